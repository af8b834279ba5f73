"""GPU parity of the mixed tensor-core forms (BF16, FP16 scaled, TF32, split BF16), called through the C ABI.

Two references:
  * a numpy emulation of the same BF16 pipeline (identical rounding points:
    R and the eigenbases rounded FP64 -> BF16 once, FP32 accumulation, every
    intermediate rounded FP32 -> BF16, G applied in FP32 before rounding).
    Only the FP32 summation order differs, which flips an occasional BF16
    rounding; bar: relative 2-norm difference <= 4e-3 (one BF16 ulp is 2^-8
    = 3.9e-3 relative, and flips are rare and uncorrelated);
  * the FP64 oracle.  The BF16 preconditioner itself is only accurate to
    ~1e-2 (reported); PCG with FP64 residuals, inner products and updates
    must still reach the FP64 bars: solution error <= 1e-9, true residual
    <= tol.
The split form (hi/lo BF16 words, three MMAs per K step) is emulated with its products summed in FP64
and rounded once to FP32.  The tensor core accumulates in FP32 but not as a sequence of correctly
rounded FP32 additions, and its differences from the emulation (measured up to 1.1e-5 at K = 130) are
of the size of the form's own error against the oracle (the dropped lo.lo terms and the 2^-16 split of
every intermediate: about 1e-5).  Bars: 3e-5 against the emulation, 6e-5 against the oracle -- three
orders of magnitude below the one-word BF16 form, which is what the form is for.
"""
import numpy as np
import pytest

import oracle as o
from inputs import synth
from tests._tc_emulation import emulate_precond
from tests._util import from_oracle, oracle_bcs, rel_err, to_oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03377_gb300 import build

    build.build()


def _plan(nx, ny, nz, bcs, prec="bf16", h=(1.0, 1.0, 1.0)):
    from paper_2501_03377_gb300 import Plan

    return Plan(nx, ny, nz, bcs, h, prec)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float64)


def uses_slices(pl, nz):
    """The plan applies its preconditioner by the frontal-slice launches (three, or four when the z
    axis exceeds 128 points); one launch per mode product otherwise (five or six in 3D)."""
    return nz > 1 and pl.precond_launches() <= 4



def emulate_bf16_precond(r_nqt, Vs, lams, singular):
    return emulate_precond(r_nqt, Vs, lams, singular, "bf16")


def plan_bases(pl, shape):
    Vs, lams = [], []
    for ax, l in enumerate(shape):
        lam, V = pl.eigenpairs(ax)
        Vs.append(np.array(V).reshape(l, l))
        lams.append(np.array(lam))
    return Vs, lams


CASES = [
    ((16, 16, 16), ("P", "N", "P")),
    ((64, 64, 32), ("P", "P", "N")),
    ((37, 9, 5), ("N", "N", "N")),
    ((33, 7, 19), ("ND", "P", "D")),
    ((20, 30, 1), ("P", "P", "P")),
    ((64, 64, 1), ("D", "D", "D")),
    ((3, 3, 3), ("D", "N", "DN")),
    ((130, 70, 24), ("DN", "P", "N")),
    ((256, 256, 8), ("P", "P", "N")),
    ((96, 160, 96), ("N", "D", "P")),
    ((200, 40, 256), ("P", "N", "D")),
    ((16, 3, 3), ("P", "D", "N")),        # frontal slices with a 3-point y axis: one padded N block
    ((48, 40, 200), ("N", "P", "D")),     # z axis past 128: the tube products as two launches
    ((256, 40, 200), ("DN", "N", "P")),
    ((32, 256, 3), ("P", "P", "N")),
]


@pytest.mark.parametrize("slices", [1, 0])
@pytest.mark.parametrize("prec", ["bf16", "fp16", "tf32", "bf16x3"])
@pytest.mark.parametrize("shape,bcs", CASES)
def test_precond_tc_matches_emulation_and_oracle(shape, bcs, prec, slices):
    from paper_2501_03377_gb300 import binding as b

    if prec == "bf16x3" and slices == 1:
        pytest.skip("the split form runs one launch per mode product: the same launches as slices=0")
    nx, ny, nz = shape
    r = synth.random_field(nx, ny, nz, seed=21)
    pl = _plan(nx, ny, nz, bcs, prec)
    pl.set_option(b.TPCG_OPT_SLICES, slices)
    sl = uses_slices(pl, nz)
    if slices == 0 or prec in ("tf32", "bf16x3"):  # TF32 and split: one launch per mode product
        assert not sl
    elif nz > 1 and nx % 16 == 0:
        assert sl
    rd = _dev(r)
    zd = torch.empty_like(rd)
    pl.precond(rd, zd)
    torch.cuda.synchronize()
    z = zd.cpu().numpy()
    sh = (nx, ny, nz)
    ob = oracle_bcs(bcs, nz)
    Vs, lams = plan_bases(pl, sh)
    emu = from_oracle(emulate_precond(to_oracle(r), Vs, lams, o.is_singular(sh, ob), prec, slices=sl))
    e_emu = rel_err(z, emu)
    Vo, _, G = o.pinv_init(sh, ob)
    ref = from_oracle(o.pinv_apply(to_oracle(r), Vo, G))
    e_ref = rel_err(z, ref)
    print(f"{prec} {shape} {bcs} slices={int(sl)}: |z - emulation| = {e_emu:.2e}, |z - fp64 oracle| = {e_ref:.2e}")
    # one ulp: 2^-8 (BF16), 2^-11 (FP16, TF32); summation-order flips are rare; split: FP32 sums (above)
    assert e_emu <= {"bf16": 4e-3, "fp16": 5e-4, "tf32": 5e-4, "bf16x3": 3e-5}[prec]
    assert e_ref <= {"bf16": 5e-2, "bf16x3": 6e-5}.get(prec, 6e-3)


SOLVE_CASES = [
    ((16, 16, 16), ("P", "N", "P")),
    ((37, 9, 5), ("N", "N", "N")),
    ((33, 7, 19), ("ND", "P", "D")),
    ((20, 30, 1), ("P", "P", "P")),
    ((64, 64, 32), ("P", "P", "DN")),
    ((96, 64, 40), ("D", "ND", "N")),
]


@pytest.mark.parametrize("prec", ["bf16", "fp16", "tf32", "bf16x3"])
@pytest.mark.parametrize("shape,bcs", SOLVE_CASES)
def test_solve_tc_matches_oracle(shape, bcs, prec):
    nx, ny, nz = shape
    eta = synth.defect_rhs(nx, ny, nz, bcs, 8, 1.5, seed=22, noise_std=1e-3)
    pl = _plan(nx, ny, nz, bcs, prec)
    ed = _dev(eta)
    ud = torch.zeros_like(ed)
    st, info = pl.solve(ed, ud, tol=1e-10, maxit=60, zero_guess=True)
    assert st == 0, info
    sh = (nx, ny, nz)
    ob = oracle_bcs(bcs, nz)
    res = o.pcg(sh, ob, (1, 1, 1), to_oracle(eta), tol=1e-13)
    u = ud.cpu().numpy()
    err = rel_err(u, from_oracle(res.U))
    print(f"{prec} {shape} {bcs}: iters={info['iters']} rel_res_true={info['rel_res_true']:.2e} rel_err={err:.2e}")
    assert err <= 1e-9
    L = o.kron_sum(sh, ob)
    etah = to_oracle(eta) - (to_oracle(eta).mean() if o.is_singular(sh, ob) else 0.0)
    true_res = np.linalg.norm(o.vec(etah) - L @ o.vec(to_oracle(u))) / np.linalg.norm(etah)
    assert true_res <= 1e-10
    if o.is_singular(sh, ob):
        assert abs(u.mean()) <= 1e-14 * np.abs(u).max()


@pytest.mark.parametrize("prec", ["bf16", "fp16", "bf16x3"])
def test_tc_solve_deterministic(prec):
    nx, ny, nz, bcs = 64, 48, 32, ("P", "P", "N")
    eta = synth.defect_rhs(nx, ny, nz, bcs, 20, 1.5, seed=23)
    pl = _plan(nx, ny, nz, bcs, prec)
    ed = _dev(eta)
    outs = []
    for _ in range(2):
        ud = torch.zeros_like(ed)
        st, info = pl.solve(ed, ud, tol=1e-10, maxit=60, zero_guess=True)
        assert st == 0
        outs.append(ud.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("prec,nz", [("bf16", 128), ("fp16", 128), ("fp16", 256), ("tf32", 128), ("bf16x3", 128),
                                     ("bf16x3", 256)])
def test_cuboid_256_tc_full_size(prec, nz):
    """256x256x128 P/P/N cuboid (singular), mixed forms, tol 1e-10, in the bench's launch configuration,
    and the 256x256x256 cube (the z axis past 128 points: the tube products as two launches).
    Checked by properties that hold at any size (true residual recomputed on the host with the
    assembled operator, zero mean) and against the oracle's direct pseudoinverse solution."""
    w = synth.workload_cuboid_256(seed=0, nz=nz)
    pl = _plan(w["nx"], w["ny"], w["nz"], w["bcs"], prec)
    if prec == "tf32":
        assert pl.precond_launches() == 6
    elif prec == "bf16x3":  # the z products around G fused while the z axis has at most 128 points
        assert pl.precond_launches() == (5 if nz <= 128 else 6)
    else:
        assert uses_slices(pl, nz) and pl.precond_launches() == (3 if nz <= 128 else 4)
    ed = _dev(w["eta"])
    ud = torch.zeros_like(ed)
    st, info = pl.solve(ed, ud, tol=1e-10, maxit=60, zero_guess=True)
    assert st == 0, info
    u = ud.cpu().numpy()
    sh = (256, 256, nz)
    L = o.kron_sum(sh, w["bcs"])
    etah = o.center(to_oracle(w["eta"]))
    true_res = np.linalg.norm(o.vec(etah) - L @ o.vec(to_oracle(u))) / np.linalg.norm(etah)
    print(f"256x256x{nz} {prec}: iters={info['iters']} rel_res_true={true_res:.2e}")
    assert true_res <= 1e-10
    if prec == "bf16x3":  # the split form's purpose: the refinement needs at most three iterations
        assert info["iters"] <= 3
    assert abs(u.mean()) <= 1e-14 * np.abs(u).max()
    Vs, _, G = o.pinv_init(sh, w["bcs"])
    direct = o.center(o.pinv_apply(etah, Vs, G))
    assert rel_err(to_oracle(u), direct) <= 1e-9


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_host_stream_matches_host_solves(prec):
    """tpcg_solve_host_stream overlaps the copies of neighbouring solves; every solution is bitwise the
    one tpcg_solve_host returns for the same right-hand side (same plan, same launch configuration),
    across more solves than its two buffer slots, with a zero and with a given initial guess."""
    nx, ny, nz, bcs = 64, 48, 24, ("P", "P", "N")
    pl = _plan(nx, ny, nz, bcs, prec=prec)
    etas = [torch.from_numpy(synth.defect_rhs(nx, ny, nz, bcs, 20, 1.5, seed=40 + i).copy()).pin_memory()
            for i in range(5)]
    outs = [torch.zeros_like(e).pin_memory() for e in etas]
    st, infos = pl.solve_host_stream(etas, outs, tol=1e-10, maxit=40, zero_guess=True)
    assert st == 0 and len(infos) == 5
    for e, u, info in zip(etas, outs, infos):
        ref = torch.zeros_like(e).pin_memory()
        st1, info1 = pl.solve_host(e, ref, tol=1e-10, maxit=40, zero_guess=True)
        assert st1 == 0 and info["status"] == 0 and info["iters"] == info1["iters"]
        assert info["rel_res_true"] <= 1e-10
        assert torch.equal(u, ref)
    # warm starts (half of each solution): the initial guesses are read from the output buffers
    guesses = [(0.5 * u).pin_memory() for u in outs[:3]]
    outs = [g.clone().pin_memory() for g in guesses]
    st, infos = pl.solve_host_stream(etas[:3], outs, tol=1e-10, maxit=40)
    assert st == 0
    for e, g, u in zip(etas[:3], guesses, outs):
        ref = g.clone().pin_memory()
        st1, _ = pl.solve_host(e, ref, tol=1e-10, maxit=40)
        assert st1 == 0
        assert torch.equal(u, ref)


def test_host_stream_rejects_bad_arguments():
    pl = _plan(16, 16, 8, ("P", "P", "N"), prec="fp16")
    e = torch.zeros(8, 16, 16, dtype=torch.float64).pin_memory()
    u = torch.zeros_like(e).pin_memory()
    from paper_2501_03377_gb300 import binding as b

    assert pl.solve_host_stream([], [], tol=1e-10)[0] == 0
    assert b.tpcg_solve_host_stream(pl.handle, [e.data_ptr()], [u.data_ptr()], 2.0, 10, 0)[0] == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_solve_host_stream(pl.handle, [e.data_ptr()], [0], 1e-10, 10, 0)[0] == b.TPCG_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        pl.solve_host_stream([e], [], tol=1e-10)


def test_caller_arrays_need_only_8_byte_alignment():
    """Device arrays of doubles are only guaranteed 8-byte alignment: the kernels that move the caller's
    eta and U as 16-byte pairs must hand over to their one-point forms when a pointer does not allow it.
    The solve from offset buffers must succeed and agree with the aligned solve."""
    nx, ny, nz, bcs = 64, 48, 24, ("P", "P", "N")
    pl = _plan(nx, ny, nz, bcs, prec="fp16")
    eta = synth.defect_rhs(nx, ny, nz, bcs, 20, 1.5, seed=61)
    ea = torch.from_numpy(eta.copy()).cuda()
    ua = torch.zeros_like(ea)
    st, _ = pl.solve(ea, ua, tol=1e-10, maxit=40, zero_guess=True)
    assert st == 0
    buf_e = torch.zeros(ea.numel() + 1, dtype=torch.float64, device="cuda")
    buf_u = torch.zeros_like(buf_e)
    eb = buf_e[1:].view(nz, ny, nx)
    ub = buf_u[1:].view(nz, ny, nx)
    eb.copy_(ea)
    assert eb.data_ptr() % 16 == 8 and ub.data_ptr() % 16 == 8
    st2, info2 = pl.solve(eb, ub, tol=1e-10, maxit=40, zero_guess=True)
    assert st2 == 0 and info2["rel_res_true"] <= 1e-10
    assert rel_err(ub.cpu().numpy(), ua.cpu().numpy()) <= 1e-9
    ub.mul_(0.5)  # warm start from the offset buffer: the eta sum and the update read U
    st3, info3 = pl.solve(eb, ub, tol=1e-10, maxit=40)
    assert st3 == 0 and info3["rel_res_true"] <= 1e-10
    assert rel_err(ub.cpu().numpy(), ua.cpu().numpy()) <= 1e-9


@pytest.mark.parametrize("defer", [0, 1])
@pytest.mark.parametrize("maxit", [1, 2, 9])
def test_unconverged_iterate_is_the_reported_one(maxit, defer):
    """A solve stopped by maxit returns an iterate with every recorded U += alpha P step applied (the mixed
    forms apply them in one pass before the host reads U): the true residual of the returned U, computed
    here with the operator, equals the reported one.  maxit = 9 also crosses the ring of recorded
    directions (applied every seventh step)."""
    nx, ny, nz, bcs = 40, 36, 20, ("P", "D", "N")
    pl = _plan(nx, ny, nz, bcs, prec="bf16")
    from paper_2501_03377_gb300 import binding as b

    pl.set_option(b.TPCG_OPT_DEFER_U, defer)
    eta = synth.defect_rhs(nx, ny, nz, bcs, 12, 1.5, seed=71)
    ed = torch.from_numpy(eta.copy()).cuda()
    ud = torch.zeros_like(ed)
    st, info = pl.solve(ed, ud, tol=1e-14, maxit=maxit, zero_guess=True)
    assert st == 4 and info["iters"] == maxit  # TPCG_ERR_NOT_CONVERGED
    w = torch.zeros_like(ed)
    pl.laplacian(ud, w)
    eta_hat = ed - info["removed_mean"]
    res = torch.linalg.vector_norm(eta_hat - w).item() / torch.linalg.vector_norm(eta_hat).item()
    assert abs(res - info["rel_res_true"]) <= 1e-6 * info["rel_res_true"] + 1e-15



@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("case", [((64, 48, 24), ("P", "P", "N"), True), ((37, 9, 5), ("N", "N", "N"), True),
                                  ((33, 7, 19), ("ND", "P", "D"), False)])
def test_deferred_u_is_bitwise_the_in_place_update(prec, case):
    """TPCG_OPT_DEFER_U records U += alpha P and forms U with the same FP64 operations in the same order:
    the solution, the iteration count and the reported residual are bitwise those of the in-place update,
    from a zero and from a given initial guess, for even and odd nx (both update kernels)."""
    from paper_2501_03377_gb300 import binding as b

    (nx, ny, nz), bcs, zero = case
    eta = synth.defect_rhs(nx, ny, nz, bcs, 10, 1.5, seed=81)
    ed = torch.from_numpy(eta.copy()).cuda()
    outs = []
    for defer in (0, 1):
        pl = _plan(nx, ny, nz, bcs, prec=prec)
        pl.set_option(b.TPCG_OPT_DEFER_U, defer)
        ud = torch.zeros_like(ed) if zero else torch.from_numpy(0.1 * synth.random_field(nx, ny, nz, seed=82)).cuda()
        st, info = pl.solve(ed, ud, tol=1e-11, maxit=60, zero_guess=zero)
        assert st == 0
        outs.append((ud.cpu().numpy(), info))
    (u0, i0), (u1, i1) = outs
    assert np.array_equal(u0, u1)
    assert i0["iters"] == i1["iters"] and i0["rel_res_true"] == i1["rel_res_true"]


FUSE_CASES = [
    ((16, 16, 16), ("P", "N", "P")),
    ((64, 64, 32), ("P", "P", "N")),
    ((9, 16, 48), ("P", "N", "D")),       # 144 rows: a ragged last tile; 48 columns: one partial K tile
    ((96, 160, 96), ("N", "D", "P")),
    ((64, 64, 1), ("D", "D", "D")),       # 2D: the pair runs along y
    ((48, 80, 1), ("P", "N", "P")),
    ((256, 256, 128), ("P", "P", "N")),
    ((37, 9, 5), ("N", "N", "N")),        # not fusable: the option changes nothing
]


@pytest.mark.parametrize("slices", [0, 1])
@pytest.mark.parametrize("prec", ["fp16", "bf16", "bf16x3"])
@pytest.mark.parametrize("shape,bcs", FUSE_CASES)
def test_fused_pair_is_bitwise_the_two_passes(shape, bcs, prec, slices):
    """TPCG_OPT_FUSE_G runs the forward and the backward mode product around G in one kernel: the same
    MMAs in the same order and the same rounding of the intermediate, so Z is bitwise that of one launch
    per pass.  With the frontal-slice launches the z products and G form one tube-pair launch instead of
    two single tube passes, with the same guarantee.  The split form (no frontal-slice launches) fuses the
    pair with its own kernel, both split eigenbases resident and one buffer for the intermediate."""
    from paper_2501_03377_gb300 import binding as b

    nx, ny, nz = shape
    r = synth.random_field(nx, ny, nz, seed=91)
    rd = _dev(r)
    outs = []
    for fuse in (0, 1):
        pl = _plan(nx, ny, nz, bcs, prec)
        pl.set_option(b.TPCG_OPT_SLICES, slices)
        pl.set_option(b.TPCG_OPT_FUSE_G, fuse)
        zd = torch.full_like(rd, float("nan"))
        pl.precond(rd, zd)
        torch.cuda.synchronize()
        outs.append(zd.cpu().numpy())
    assert np.isfinite(outs[1]).all()
    assert np.array_equal(outs[0], outs[1])
    if slices and prec != "bf16x3" and nz > 1 and nx % 16 == 0:
        assert pl.precond_launches() == (3 if nz <= 128 else 4)
    else:
        fusable = shape != (37, 9, 5)
        full = 6 if nz > 1 else 4
        assert pl.precond_launches() == full - (1 if fusable else 0)


@pytest.mark.parametrize("prec", ["fp16", "bf16", "bf16x3"])
def test_fused_pair_solve_is_bitwise(prec):
    from paper_2501_03377_gb300 import binding as b

    nx, ny, nz, bcs = 64, 48, 32, ("P", "P", "N")
    eta = synth.defect_rhs(nx, ny, nz, bcs, 12, 1.5, seed=92)
    ed = _dev(eta)
    outs = []
    for fuse in (0, 1):
        pl = _plan(nx, ny, nz, bcs, prec)
        pl.set_option(b.TPCG_OPT_FUSE_G, fuse)
        ud = torch.zeros_like(ed)
        st, info = pl.solve(ed, ud, tol=1e-10, maxit=60, zero_guess=True)
        assert st == 0
        outs.append((ud.cpu().numpy(), info["iters"], info["rel_res_true"]))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1:] == outs[1][1:]


def test_plan_option_rejects_bad_values():
    from paper_2501_03377_gb300 import binding as b

    pl = _plan(16, 16, 8, ("P", "P", "N"), prec="fp16")
    assert b.tpcg_plan_set_option(pl.handle, b.TPCG_OPT_DEFER_U, 2) == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_plan_set_option(pl.handle, 99, 1) == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_plan_set_option(pl.handle, b.TPCG_OPT_DEFER_U, 1) == b.TPCG_OK
    assert b.tpcg_plan_set_option(pl.handle, b.TPCG_OPT_FUSE_G, 2) == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_plan_set_option(pl.handle, b.TPCG_OPT_FUSE_G, 0) == b.TPCG_OK
    assert b.tpcg_plan_set_option(pl.handle, b.TPCG_OPT_SLICES, 2) == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_plan_set_option(pl.handle, b.TPCG_OPT_SLICES, 0) == b.TPCG_OK


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_defer_u_set_between_solves_is_bitwise(prec):
    """TPCG_OPT_DEFER_U switched on between two solves of one plan (the direction storage is replaced
    once the first solve's work has finished): the second solve equals, bitwise, the same solve on a
    plan that had the option from the start, and the in-place update of a fresh plan."""
    from paper_2501_03377_gb300 import binding as b

    nx, ny, nz, bcs = 64, 48, 32, ("P", "P", "N")
    e1 = _dev(synth.defect_rhs(nx, ny, nz, bcs, 12, 1.5, seed=93))
    e2 = _dev(synth.defect_rhs(nx, ny, nz, bcs, 12, 1.5, seed=94))
    pl = _plan(nx, ny, nz, bcs, prec)
    u1 = torch.zeros_like(e1)
    assert pl.solve(e1, u1, tol=1e-10, maxit=60, zero_guess=True)[0] == 0
    pl.set_option(b.TPCG_OPT_DEFER_U, 1)
    u2 = torch.zeros_like(e2)
    st, info = pl.solve(e2, u2, tol=1e-10, maxit=60, zero_guess=True)
    assert st == 0
    outs = []
    for defer in (1, 0):
        q = _plan(nx, ny, nz, bcs, prec)
        q.set_option(b.TPCG_OPT_DEFER_U, defer)
        u = torch.zeros_like(e2)
        stq, iq = q.solve(e2, u, tol=1e-10, maxit=60, zero_guess=True)
        assert stq == 0 and iq["iters"] == info["iters"]
        outs.append(u.cpu().numpy())
    assert np.array_equal(u2.cpu().numpy(), outs[0])
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("shape,bcs", [((64, 64, 32), ("P", "P", "N")), ((37, 9, 5), ("N", "N", "N")),
                                       ((96, 64, 160), ("D", "P", "N"))])
def test_autotune_picks_a_sequence_caches_it_and_solves(shape, bcs, tmp_path):
    """tpcg_plan_autotune times the distinct launch sequences, keeps the fastest, appends it to the cache
    file; a second plan of the same grid takes it from the cache; solves after tuning still meet the bars."""
    from paper_2501_03377_gb300 import binding as b

    nx, ny, nz = shape
    cache = str(tmp_path / "tune.txt")
    pl = _plan(nx, ny, nz, bcs, "fp16")
    r1 = pl.autotune(cache, applies=3)
    assert r1["from_cache"] == 0 and r1["candidates"] >= 1 and r1["us_per_apply"] > 0
    assert r1["candidates"] <= (4 if nx % 16 == 0 else 2)
    q = _plan(nx, ny, nz, bcs, "fp16")
    r2 = q.autotune(cache, applies=3)
    assert r2["from_cache"] == 1 and (r2["slices"], r2["fuse_g"]) == (r1["slices"], r1["fuse_g"])
    assert open(cache).read().count("\n") == 1
    eta = synth.defect_rhs(nx, ny, nz, bcs, 8, 1.5, seed=95)
    ed = _dev(eta)
    ud = torch.zeros_like(ed)
    st, info = q.solve(ed, ud, tol=1e-10, maxit=60, zero_guess=True)
    assert st == 0 and info["rel_res_true"] <= 1e-10
    f64 = _plan(nx, ny, nz, bcs, "fp64")
    assert f64.autotune(None)["candidates"] == 0
    assert b.tpcg_plan_autotune(pl.handle, None, 0)[0] == b.TPCG_ERR_INVALID_ARG
