"""Numpy emulation of the mixed tensor-core preconditioner (Algorithm 7) with the device's rounding points.

Test infrastructure shared by the GPU parity tests and the CPU experiments on the precision readings:
BF16 / FP16 / TF32 rounding of FP64 and FP32 values (nearest even), mode products in FP32, the
power-of-two scalings of the FP16 form, the hi/lo BF16 pairs of the split form, and the order in which
each launch sequence rounds its intermediates.
"""
import numpy as np


def bf16_from_f64(x):
    """Round float64 -> bfloat16 (nearest-even) in one step; returned as float32."""
    x = np.asarray(x, dtype=np.float64)
    u = x.view(np.uint64)
    sign = (u >> np.uint64(63)) << np.uint64(15)
    e = ((u >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    eb = e - 1023 + 127
    mant = u & np.uint64(0xFFFFFFFFFFFFF)
    top = (mant >> np.uint64(45)).astype(np.uint64)
    rest = mant & np.uint64((1 << 45) - 1)
    half = np.uint64(1 << 44)
    bits = (np.clip(eb, 0, 255).astype(np.uint64) << np.uint64(7)) | top
    up = (rest > half) | ((rest == half) & ((top & np.uint64(1)) == np.uint64(1)))
    bits = bits + up.astype(np.uint64)
    bits = np.where(eb <= 0, np.uint64(0), bits)
    b16 = (sign | bits).astype(np.uint32)
    return (b16 << np.uint32(16)).view(np.float32)


def bf16_from_f32(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)
    return (u.astype(np.uint32) << np.uint32(16)).view(np.float32)


def mode(M, X, m):
    """M x_m X in float32 (float32 accumulation)."""
    Y = np.tensordot(M.astype(np.float32), np.moveaxis(X, m, 0).astype(np.float32), axes=(1, 0))
    return np.moveaxis(Y, 0, m).astype(np.float32)


def f16_from_f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


def f16_from_f64(x, shift=0):
    """x * 2^shift rounded once to binary16 (nearest-even), returned as float32."""
    return np.ldexp(np.asarray(x, dtype=np.float64), shift).astype(np.float16).astype(np.float32)


def tf32_from(x):
    """Round to TF32 (11 significant bits, FP32's exponent range), nearest even; returned as float32."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.round(np.ldexp(m, 11)), e - 11).astype(np.float32)


def lp_shift(r):
    rms = np.sqrt(np.mean(np.asarray(r, dtype=np.float64) ** 2))
    return 0 if rms == 0 else int(np.clip(-np.floor(np.log2(rms)) - 1, -120, 120))


def fp16_gscale_exponent(lams, N):
    cands = [np.unique(np.asarray(l))[:2] for l in lams]
    sums = [x + y + z for x in cands[0] for y in cands[1] for z in cands[2] if x + y + z > 1e-300]
    bound = np.sqrt(N) / min(sums)
    return max(0, int(np.ceil(np.log2(bound / 16384.0))))


def split_f64(x):
    """x -> (hi, lo) = (bf16(x), bf16(x - hi)), each rounded once from FP64; returned as float32."""
    x = np.asarray(x, dtype=np.float64)
    hi = bf16_from_f64(x)
    return hi, bf16_from_f64(x - hi.astype(np.float64))


def split_f32(x):
    """The same split of FP32 values (x - hi is exact in FP32)."""
    x = np.asarray(x, dtype=np.float32)
    hi = bf16_from_f32(x)
    return hi, bf16_from_f32((x - hi).astype(np.float32))


def mode_split(M, X, m):
    """Split-form mode product: hi.hi + lo.hi + hi.lo of the BF16 pairs M = (Mh, Ml), X = (Xh, Xl),
    summed in FP64 and rounded once to FP32 (the device accumulates in FP32, in its own order)."""
    (Mh, Ml), (Xh, Xl) = M, X

    def prod(A, B):
        Y = np.tensordot(A.astype(np.float64), np.moveaxis(B, m, 0).astype(np.float64), axes=(1, 0))
        return np.moveaxis(Y, 0, m)

    return (prod(Mh, Xh) + prod(Ml, Xh) + prod(Mh, Xl)).astype(np.float32)


def emulate_split_precond(r_nqt, Vs, lams, singular):
    """The split BF16 form of Algorithm 7, one launch per mode product (x, y, z forward; G; z, y, x
    backward): R and the eigenbases split from FP64, every intermediate split from FP32, G applied in
    FP32 before the split, Z in FP32."""
    three_d = r_nqt.shape[2] > 1
    VT = [split_f64(np.asarray(V, dtype=np.float64).T) for V in Vs]
    VV = [split_f64(np.asarray(V, dtype=np.float64)) for V in Vs]
    F = split_f64(r_nqt)
    F = split_f32(mode_split(VT[0], F, 0))
    F = mode_split(VT[1], F, 1)
    if three_d:
        F = mode_split(VT[2], split_f32(F), 2)
    la = [np.asarray(l, dtype=np.float32) for l in lams]
    S = (la[0][:, None, None] + la[1][None, :, None]) + la[2][None, None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        F = (F * (np.float32(1.0) / S).astype(np.float32)).astype(np.float32)
    if singular:
        F[0, 0, 0] = 0.0
    F = split_f32(F)
    if three_d:
        F = split_f32(mode_split(VV[2], F, 2))
    F = split_f32(mode_split(VV[1], F, 1))
    return mode_split(VV[0], F, 0)


def emulate_precond(r_nqt, Vs, lams, singular, prec="bf16", slices=False):
    """The tensor-core form of Algorithm 7 with its rounding points (BF16, or FP16 with the
    power-of-two scalings that keep every intermediate in range).  slices: the frontal-slice launch
    sequence, whose backward x product precedes the backward y product."""
    if prec == "bf16x3":
        return emulate_split_precond(r_nqt, Vs, lams, singular)
    three_d = r_nqt.shape[2] > 1
    if prec == "bf16":
        rin, rd, Vb = (lambda x: bf16_from_f64(x)), bf16_from_f32, [bf16_from_f64(V) for V in Vs]
        s, sG = 0, 0
    elif prec == "tf32":
        rin, rd, Vb = tf32_from, tf32_from, [tf32_from(V) for V in Vs]
        s, sG = 0, 0
    else:
        s = lp_shift(r_nqt)
        sG = fp16_gscale_exponent(lams, r_nqt.size)
        rin, rd, Vb = (lambda x: f16_from_f64(x, s)), f16_from_f32, [f16_from_f64(V) for V in Vs]
    F = rin(r_nqt)
    F = rd(mode(Vb[0].T, F, 0))
    F = mode(Vb[1].T, F, 1)
    if three_d:
        F = rd(F)
        F = mode(Vb[2].T, F, 2)
    la = [np.asarray(l, dtype=np.float32) for l in lams]
    S = (la[0][:, None, None] + la[1][None, :, None]) + la[2][None, None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        g = ((np.float32(1.0) / S).astype(np.float32) * np.float32(2.0 ** -sG)).astype(np.float32)
        F = (F * g).astype(np.float32)
    if singular:
        F[0, 0, 0] = 0.0
    F = rd(F)
    if three_d:
        F = rd(mode(Vb[2], F, 2))
    if slices:
        F = rd(mode(Vb[0], F, 0))
        return (mode(Vb[1], F, 1) * np.float32(2.0 ** (sG - s))).astype(np.float32)
    F = rd(mode(Vb[1], F, 1))
    return (mode(Vb[0], F, 0) * np.float32(2.0 ** (sG - s))).astype(np.float32)
