"""The CG scalars of the mixed forms against FP64 dot products of the same vectors (Algorithm 1, Sec. 4.1).

The mixed forms keep R, U and the stop test in FP64 (exact integer where the stencil runs on the
fixed-point direction) but accumulate <W,P>, rho, ||R||^2 and sum(R) per thread in FP32 (combined in
FP64) and take rho = <R~, Z> from the FP16/BF16 copy R~ of R that the preconditioner read.  For the
first iterations of a solve this test reads the device's alpha_s, beta_s, rho_s and <W_s, P_s> back
through the C ABI (tpcg_plan_cg_scalars), the vectors they came from (tpcg_plan_cg_vectors), and
recomputes each scalar in FP64 on the host with the oracle's assembled operator:
    <W_s, P_s> = <L P_s, P_s>,   rho_s = <R_s, Z_s> - mean(Z_s) sum(R_s),
    alpha_s = rho_s / <W_s, P_s>,   beta_s = rho_s / rho_{s-1},
where R_s = R_{s+1} + alpha_s L P_s is recovered from the residual the update wrote.  The bounds are
those of the arithmetic: FP32 partial sums of a few hundred terms per thread (relative error a few
times 2^-24 times their count's square root) and, for rho, the rounding of R~ (relative 2^-11 FP16,
2^-8 BF16 per entry, uncorrelated with Z, so of order 2^-11 / sqrt(N) on the sum).  The FP64 form is
checked the same way at FP64 accuracy, which validates the readback itself.
"""
import numpy as np
import pytest
import torch

import oracle as o
from inputs import synth
from tests._util import from_oracle, to_oracle

pytestmark = pytest.mark.gpu


def _run(prec, shape, bcs, maxit, eta):
    from paper_2501_03377_gb300 import Plan

    nx, ny, nz = shape
    pl = Plan(nx, ny, nz, bcs, prec=prec)
    ed = torch.from_numpy(eta).cuda()
    ud = torch.zeros_like(ed)
    st, info = pl.solve(ed, ud, tol=1e-14, maxit=maxit, zero_guess=True)
    sc = pl.cg_scalars()
    R, Z, P = (v.cpu().numpy() for v in pl.cg_vectors())
    pl.close()
    return st, info, sc, R, Z, P


def _fp64_scalars(L, R1, Z, P, alpha, singular):
    """FP64 <L P, P>, rho_s = <R_s, Z_s'> of the vectors the device held (oracle ordering), and ||R_s||."""
    p = o.vec(to_oracle(P))
    lp = L @ p
    wp = float(p @ lp)
    r_s = o.vec(to_oracle(R1)) + alpha * lp  # R_s from R_{s+1} = R_s - alpha_s L P_s
    z = o.vec(to_oracle(Z))
    rho = float(r_s @ z) - (float(z.mean()) * float(r_s.sum()) if singular else 0.0)
    return wp, rho, float(np.linalg.norm(r_s))


CASES = [
    ("fp16", (128, 128, 64), ("P", "P", "N")),
    ("bf16", (128, 128, 64), ("P", "P", "N")),
    ("fp16", (96, 64, 40), ("D", "ND", "N")),
    ("fp64", (64, 64, 32), ("P", "P", "N")),
    ("bf16x3", (128, 128, 64), ("P", "P", "N")),
]


@pytest.mark.parametrize("prec,shape,bcs", CASES)
def test_cg_scalars_match_fp64_dots(prec, shape, bcs):
    nx, ny, nz = shape
    eta = synth.defect_rhs(nx, ny, nz, bcs, 60, 1.5, seed=31, noise_std=1e-3)
    L = o.kron_sum(shape, bcs)
    singular = o.is_singular(shape, bcs)
    rho_ref_prev = None
    rows = []
    for s in range(1, 5):
        st, info, sc, R1, Z, P = _run(prec, shape, bcs, s, eta)
        if info["iters"] < s:  # converged before s iterations
            break
        assert sc["iter"] == s
        wp, rho, rn = _fp64_scalars(L, R1, Z, P, sc["alpha"], singular)
        if rn < 1e-9 * info["eta_norm"]:
            # R_s is at the FP64 rounding floor (the FP64 form after one iteration): the host's
            # reconstruction R_{s+1} + alpha L P cancels to noise, there is nothing left to compare
            break
        e_wp = abs(sc["wp"] - wp) / wp
        e_rho = abs(sc["rho"] - rho) / rho
        e_alpha = abs(sc["alpha"] - rho / wp) / (rho / wp)
        e_beta = abs(sc["beta"] - rho / rho_ref_prev) / (rho / rho_ref_prev) if rho_ref_prev else 0.0
        rows.append((s, e_wp, e_rho, e_alpha, e_beta))
        rho_ref_prev = rho
    print(f"\n{prec} {shape} {bcs}: iteration, rel. error of <W,P>, rho, alpha, beta vs FP64 dots")
    for r in rows:
        print("  s=%d  %.2e  %.2e  %.2e  %.2e" % r)
    # (the split form reaches the FP64 floor after three iterations: two comparable ones)
    assert len(rows) >= {"fp64": 1, "bf16x3": 2}.get(prec, 3)
    N = nx * ny * nz
    if prec == "fp64":
        bound_wp = bound_rho = 1e-12
    else:
        bound_wp = 1e-7  # FP32 partial sums per thread of exact integer differences (measured ~5e-9)
        # R~ rounding (uncorrelated with Z) plus FP32 partial sums (measured 1e-7..3e-6 FP16, 5e-6..1e-5 BF16)
        ulp = {"fp16": 2.0 ** -11, "bf16x3": 2.0 ** -16}.get(prec, 2.0 ** -8)
        bound_rho = max(1e-5, 50 * ulp / np.sqrt(N))
    for s, e_wp, e_rho, e_alpha, e_beta in rows:
        assert e_wp <= bound_wp, (s, e_wp)
        assert e_rho <= bound_rho, (s, e_rho)
        assert e_alpha <= bound_wp + bound_rho, (s, e_alpha)
        assert e_beta <= 2 * bound_rho, (s, e_beta)
