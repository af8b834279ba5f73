"""Shared helpers of the test suite (layout conversion between the CUDA path and the oracle)."""
import numpy as np


def to_oracle(a_zyx):
    """Storage order (nz, ny, nx) -> the paper's (n, q, t) indexing used by the oracle."""
    return np.ascontiguousarray(np.asarray(a_zyx).transpose(2, 1, 0))


def from_oracle(a_nqt):
    return np.ascontiguousarray(np.asarray(a_nqt).transpose(2, 1, 0))


def oracle_bcs(bcs, nz):
    return (bcs[0], bcs[1], None if nz == 1 else bcs[2])


def oracle_shape(nx, ny, nz):
    return (nx, ny, nz)


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0)
