"""CPU FP64 oracle (test infrastructure only; see tpcg_oracle.py)."""
from .tpcg_oracle import *  # noqa: F401,F403
