"""What the mixed forms' departures from FP64 CG scalars cost in iterations (Algorithm 1, Sec. 4.1), on CPU.

The mixed forms run Algorithm 1 with an FP16 (or BF16) tensor-core preconditioner and keep R, U and
the stop test in FP64, with three departures:
  (a) the direction is stored as 20-bit fixed point, P_s = 2^-kp round(2^kp (Z_s + beta_s P_{s-1})),
      |P_int| <= 2^20, and W = L P_s is the exact stencil of that P (so U and R stay consistent);
  (b) rho_s = <R~_s, Z_s> with R~_s the FP16 copy of R_s (scaled by 2^shift) that the preconditioner
      read, instead of the FP64 R_s;
  (c) the scalars are accumulated per thread in FP32 (combined in FP64) -- measured against FP64 dots
      on the GPU by tests/test_gpu_precision.py, relative error ~1e-7, not emulated here.
This experiment runs the same PCG with the emulated FP16 preconditioner (the device's rounding
points, tests/_tc_emulation.py) and every combination of (a) and (b) against the all-FP64-scalar
variant, and a wider 30-bit direction in place of (a).  It pins that neither departure changes the
iteration count to 1e-10 and that the true residual history agrees to a factor well inside one
iteration's reduction.
"""
import numpy as np
import pytest

import oracle as o
from inputs import synth
from tests._tc_emulation import emulate_precond, f16_from_f64, lp_shift, split_f64
from tests._util import oracle_bcs, to_oracle


def _fixed(P, bound, bits):
    """P rounded to fixed point with |P_int| <= 2^bits (exponent from the bound, as the device does)."""
    if bound <= 0:
        return P
    kp = (bits - 1) - int(np.floor(np.log2(bound)))
    return np.ldexp(np.rint(np.ldexp(P, kp)), -kp)


def _pcg(shape, bcs, H, prec, dir_bits, rho_from_copy, tol=1e-10, maxit=30):
    L = o.kron_sum(shape, bcs)
    Vs, lams, _ = o.pinv_init(shape, bcs)
    # the null eigenvalue of a P/N axis is exactly 0 on the device (closed forms); eigh leaves ~1e-16
    lams = [np.where(np.abs(lam) < 1e-12, 0.0, lam) for lam in lams]
    singular = o.is_singular(shape, bcs)
    H = o.center(H) if singular else H.copy()
    hn = np.linalg.norm(H)

    def apply_l(X):
        return o.unvec(L @ o.vec(X), shape)

    def M(R):
        return emulate_precond(R, Vs, lams, singular, prec, slices=True).astype(np.float64)

    def rho_of(R, Z):
        Zc = o.center(Z) if singular else Z
        if not rho_from_copy:
            return float(np.vdot(R, Zc))
        if prec == "fp16":
            s = lp_shift(R)
            Rt = np.ldexp(f16_from_f64(R, s).astype(np.float64), -s)
        elif prec == "bf16x3":
            hi, lo = split_f64(R)
            Rt = hi.astype(np.float64) + lo.astype(np.float64)
        else:
            from tests._tc_emulation import bf16_from_f64

            Rt = bf16_from_f64(R).astype(np.float64)
        return float(np.vdot(Rt, Zc))

    U = np.zeros(shape)
    R = H.copy()
    Z = M(R)
    rho = rho_of(R, Z)
    P = None
    hist = [1.0]
    for s in range(1, maxit + 1):
        Zc = o.center(Z) if singular else Z
        if P is None:
            Pn = Zc
            bound = np.abs(Z).max()
        else:
            beta = rho / rho_prev
            Pn = Zc + beta * P
            bound = np.abs(Z).max() + abs(beta) * np.abs(P).max()
        P = _fixed(Pn, bound, dir_bits) if dir_bits else Pn
        W = apply_l(P)
        alpha = rho / float(np.vdot(W, P))
        U = U + alpha * P
        R = R - alpha * W
        hist.append(np.linalg.norm(H - apply_l(U)) / hn)
        if hist[-1] <= tol:
            return s, hist
        Z = M(R)
        rho_prev, rho = rho, rho_of(R, Z)
    return maxit, hist


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_direction_rounding_and_rho_copy_leave_iterations_unchanged(prec):
    shape, bcs = (64, 64, 32), ("P", "P", "N")
    eta = synth.defect_rhs(*shape, bcs, 120, (1.0, 4.0), seed=5, mode="charge")
    H = to_oracle(eta)
    runs = {}
    for name, bits, copy in (("fp64 scalars", 0, False), ("20-bit P", 20, False), ("30-bit P", 30, False),
                             ("rho from copy", 0, True), ("20-bit P + rho from copy", 20, True)):
        runs[name] = _pcg(shape, bcs, H, prec, bits, copy)
    ref_it, ref_h = runs["fp64 scalars"]
    print(f"\n{prec} {shape} {bcs}: iterations to 1e-10 and true residual per iteration")
    for name, (it, h) in runs.items():
        print(f"  {name:26s} {it:3d}  " + " ".join(f"{x:.1e}" for x in h))
    for name, (it, h) in runs.items():
        assert it == ref_it, (name, it, ref_it)
        # per-iteration agreement while the residual is above the FP64 floor: well inside one iteration's
        # reduction (the FP16 preconditioner removes 2-3 orders of magnitude per iteration here)
        for a, b in zip(h[1:], ref_h[1:]):
            if max(a, b) > 1e-13:
                assert 0.5 <= a / b <= 2.0, (name, a, b)


def test_split_pair_represents_fp64_to_2_pow_minus_16():
    """hi = bf16(x), lo = bf16(x - hi): a BF16 word has 8 significant bits, so rounding to nearest leaves
    |x - hi| <= 2^-8 |x| and |x - (hi + lo)| <= 2^-8 |x - hi| <= 2^-16 |x| for values in the normal range."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal(100000) * np.exp2(rng.integers(-60, 60, 100000))
    hi, lo = split_f64(x)
    err = np.abs(x - (hi.astype(np.float64) + lo.astype(np.float64)))
    assert np.all(np.abs(x - hi) <= np.ldexp(np.abs(x), -8))
    assert np.all(err <= np.ldexp(np.abs(x), -16))
    assert np.median(err / np.abs(x)) < 2.0 ** -17.5  # uniformly spread rounding: well inside the bound
    # exactly representable values split with lo = 0
    h2, l2 = split_f64(np.array([1.0, -0.5, 3.0, 2.0 ** -100]))
    assert np.all(l2 == 0) and np.array_equal(h2, np.array([1.0, -0.5, 3.0, 2.0 ** -100], np.float32))


@pytest.mark.parametrize("shape,bcs", [((32, 24, 16), ("P", "P", "N")), ((20, 30, 1), ("D", "N", "N")),
                                       ((17, 9, 12), ("ND", "D", "DN"))])
def test_split_form_emulation_is_accurate_to_about_2_pow_minus_16(shape, bcs):
    """Algorithm 7 in the split form (three BF16 products per K step, the lo.lo term dropped) against the
    FP64 pseudoinverse: each product is accurate to about 2^-16 relative (the dropped term and the split
    of its output), so six products leave the relative error of Z near 1e-5, against about 1e-2 for one
    BF16 word per operand."""
    nx, ny, nz = shape
    sh, ob = (nx, ny, nz), oracle_bcs(bcs, nz)
    singular = o.is_singular(sh, ob)
    r = to_oracle(synth.random_field(nx, ny, nz, seed=4))
    if singular:
        r = o.center(r)
    Vs, lams, G = o.pinv_init(sh, ob)
    lams = [np.where(np.abs(lam) < 1e-12, 0.0, lam) for lam in lams]
    ref = o.pinv_apply(r, Vs, G)

    def rel(z):
        z = z.astype(np.float64)
        if singular:
            z = o.center(z)
        return np.linalg.norm(z - ref) / np.linalg.norm(ref)

    e = rel(emulate_precond(r, Vs, lams, singular, "bf16x3"))
    e1 = rel(emulate_precond(r, Vs, lams, singular, "bf16"))
    print(f"\nsplit form {shape} {bcs}: |Z - Z_fp64| / |Z_fp64| = {e:.2e} (one BF16 word: {e1:.2e})")
    assert e1 > 100 * e
    assert e <= 3e-5


def test_split_form_needs_three_iterations():
    """The split form as the preconditioner of the mixed PCG (20-bit direction, rho from the hi + lo copy of
    R): the true residual falls below 1e-10 in three iterations on the 64x64x32 P/P/N workload where the
    one-word forms need six (FP16) and eleven (BF16)."""
    shape, bcs = (64, 64, 32), ("P", "P", "N")
    eta = synth.defect_rhs(*shape, bcs, 120, (1.0, 4.0), seed=5, mode="charge")
    it, h = _pcg(shape, bcs, to_oracle(eta), "bf16x3", 20, True)
    it16, _ = _pcg(shape, bcs, to_oracle(eta), "fp16", 20, True)
    print(f"\nsplit form: {it} iterations (FP16: {it16}); residuals " + " ".join(f"{x:.1e}" for x in h))
    assert it <= 3 < it16
