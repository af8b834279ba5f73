"""GPU parity of the FP64 path against the CPU oracle, called through the C ABI.

Tolerances (FP64 throughout, different summation orders on the two sides):
  * stencil: max |w_gpu - w_oracle| <= 1e-13 * max |w_oracle|;
  * preconditioner: relative 2-norm error <= 1e-12 (six dense mode products
    of length <= 256, each adding O(l * 2^-53) relative error);
  * solve: relative solution error <= 1e-9 and true relative residual <= tol
    (the bars of the solver specification).
"""
import itertools

import numpy as np
import pytest

import oracle as o
from inputs import synth
from tests._util import from_oracle, oracle_bcs, rel_err, to_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03377_gb300 import build

    build.build()


def _plan(nx, ny, nz, bcs, h=(1.0, 1.0, 1.0), prec="fp64"):
    from paper_2501_03377_gb300 import Plan

    return Plan(nx, ny, nz, bcs, h, prec)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float64)


ALL_BCS = list(itertools.product(o.BCS, repeat=3))


@pytest.mark.parametrize("bcs", ALL_BCS)
def test_stencil_all_bc_triples(bcs):
    nx, ny, nz = 37, 11, 6  # ragged against the 32 x 8 tiles
    h = (1.0, 0.5, 2.0)
    x = synth.random_field(nx, ny, nz, seed=11)
    pl = _plan(nx, ny, nz, bcs, h)
    xd = _dev(x)
    wd = torch.empty_like(xd)
    pl.laplacian(xd, wd)
    torch.cuda.synchronize()
    L = o.kron_sum((nx, ny, nz), bcs, h)
    ref = from_oracle(o.unvec(L @ o.vec(to_oracle(x)), (nx, ny, nz)))
    got = wd.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("shape", [(3, 3, 3), (3, 5, 1), (64, 64, 1), (33, 17, 1), (256, 8, 3), (8, 256, 4)])
@pytest.mark.parametrize("bcs", [("P", "N", "D"), ("DN", "ND", "P"), ("N", "N", "N")])
def test_stencil_shapes(shape, bcs):
    nx, ny, nz = shape
    x = synth.random_field(nx, ny, nz, seed=12)
    pl = _plan(nx, ny, nz, bcs)
    xd = _dev(x)
    wd = torch.empty_like(xd)
    pl.laplacian(xd, wd)
    torch.cuda.synchronize()
    L = o.kron_sum((nx, ny, nz), oracle_bcs(bcs, nz))
    ref = from_oracle(o.unvec(L @ o.vec(to_oracle(x)), (nx, ny, nz)))
    assert np.abs(wd.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("n", [3, 4, 5, 64, 65, 128, 255, 256])
@pytest.mark.parametrize("bc", o.BCS)
def test_plan_eigenpairs_diagonalise_lap1d(n, bc):
    pl = _plan(n, 3, 1, (bc, "D", "D"), (0.5, 1.0, 1.0))
    lam, V = pl.eigenpairs(0)
    lam = np.array(lam)
    V = np.array(V).reshape(n, n)
    L = o.lap1d(n, bc, 0.5)
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-14 * n
    assert np.abs(L @ V - V * lam).max() <= 1e-12 * 4 / 0.25
    assert np.abs(np.sort(lam) - np.linalg.eigvalsh(L)).max() <= 1e-12 * 4 / 0.25
    if bc in ("P", "N"):
        assert lam[0] == 0.0 and np.allclose(V[:, 0], 1 / np.sqrt(n))


PRECOND_CASES = [
    ((12, 10, 8), ("P", "N", "P")),
    ((16, 16, 16), ("D", "DN", "ND")),
    ((37, 9, 5), ("N", "N", "N")),
    ((20, 30, 1), ("P", "P", "P")),
    ((64, 64, 1), ("D", "D", "D")),
    ((33, 7, 19), ("ND", "P", "D")),
]


@pytest.mark.parametrize("shape,bcs", PRECOND_CASES)
def test_precond_fp64_matches_oracle(shape, bcs):
    nx, ny, nz = shape
    r = synth.random_field(nx, ny, nz, seed=13)
    pl = _plan(nx, ny, nz, bcs)
    rd = _dev(r)
    zd = torch.empty_like(rd)
    pl.precond(rd, zd)
    torch.cuda.synchronize()
    sh = (nx, ny, nz)
    Vs, _, G = o.pinv_init(sh, oracle_bcs(bcs, nz))
    ref = from_oracle(o.pinv_apply(to_oracle(r), Vs, G))
    assert rel_err(zd.cpu().numpy(), ref) <= 1e-12


SOLVE_CASES = [
    ((12, 10, 8), ("P", "N", "P")),
    ((16, 16, 16), ("D", "DN", "ND")),
    ((37, 9, 5), ("N", "N", "N")),
    ((20, 30, 1), ("P", "P", "P")),
    ((33, 7, 19), ("ND", "P", "D")),
    ((40, 24, 12), ("P", "P", "DN")),
]


@pytest.mark.parametrize("shape,bcs", SOLVE_CASES)
def test_solve_fp64_matches_oracle(shape, bcs):
    nx, ny, nz = shape
    eta = synth.defect_rhs(nx, ny, nz, bcs, 6, 1.5, seed=14, noise_std=1e-3)
    pl = _plan(nx, ny, nz, bcs)
    ed = _dev(eta)
    ud = torch.zeros_like(ed)
    st, info = pl.solve(ed, ud, tol=1e-10, maxit=30, zero_guess=True)
    assert st == 0, info
    sh = (nx, ny, nz)
    ob = oracle_bcs(bcs, nz)
    res = o.pcg(sh, ob, (1, 1, 1), to_oracle(eta), tol=1e-13)
    u = ud.cpu().numpy()
    assert rel_err(u, from_oracle(res.U)) <= 1e-9
    L = o.kron_sum(sh, ob)
    etah = to_oracle(eta) - (to_oracle(eta).mean() if o.is_singular(sh, ob) else 0.0)
    true_res = np.linalg.norm(o.vec(etah) - L @ o.vec(to_oracle(u))) / np.linalg.norm(etah)
    assert true_res <= 1e-10
    # both sides evaluate the residual in FP64 with different summation orders: agree to
    # 1% or to the rounding floor of the evaluation (~1e-14 relative)
    assert abs(info["rel_res_true"] - true_res) <= 1e-2 * true_res + 1e-14
    assert info["iters"] <= 4
    if o.is_singular(sh, ob):
        assert abs(u.mean()) <= 1e-14 * np.abs(u).max()
        assert abs(info["removed_mean"] - eta.mean()) <= 1e-12 * abs(eta).max()


def test_solve_2d_dirichlet_workload():
    """The 2D 64x64 Dirichlet workload (8 blobs, tol 1e-12) at full size."""
    w = synth.workload_2d_dirichlet(seed=0)
    pl = _plan(w["nx"], w["ny"], w["nz"], w["bcs"])
    ed = _dev(w["eta"])
    ud = torch.zeros_like(ed)
    st, info = pl.solve(ed, ud, tol=w["tol"], maxit=30, zero_guess=True)
    assert st == 0
    sh = (64, 64, 1)
    ob = ("D", "D", None)
    ref = o.pcg(sh, ob, (1, 1, 1), to_oracle(w["eta"]), tol=1e-14)
    assert rel_err(ud.cpu().numpy(), from_oracle(ref.U)) <= 1e-9
    assert info["rel_res_true"] <= 1e-12


def test_warm_start_and_host_buffers():
    nx, ny, nz, bcs = 24, 20, 10, ("P", "P", "N")
    eta = synth.defect_rhs(nx, ny, nz, bcs, 10, 1.5, seed=15)
    pl = _plan(nx, ny, nz, bcs)
    ed = _dev(eta)
    u0 = _dev(synth.random_field(nx, ny, nz, seed=16))
    st, info = pl.solve(ed, u0, tol=1e-11, maxit=30)
    assert st == 0
    u1 = torch.zeros_like(ed)
    st, _ = pl.solve(ed, u1, tol=1e-11, maxit=30, zero_guess=True)
    assert st == 0
    assert rel_err(u0.cpu().numpy(), u1.cpu().numpy()) <= 1e-9
    eh = torch.from_numpy(eta.copy()).pin_memory()
    uh = torch.zeros_like(eh).pin_memory()
    st, info_h = pl.solve_host(eh, uh, tol=1e-11, maxit=30, zero_guess=True)
    assert st == 0
    assert np.array_equal(uh.numpy(), u1.cpu().numpy())  # same launch configuration: bitwise equal


def test_zero_rhs_gives_zero_solution():
    pl = _plan(16, 16, 8, ("P", "P", "P"))
    ed = _dev(np.full((8, 16, 16), 3.0))  # constant: centred to exactly zero
    ud = _dev(synth.random_field(16, 16, 8, seed=17))
    st, info = pl.solve(ed, ud, tol=1e-10, maxit=10)
    assert st == 0
    assert torch.count_nonzero(ud).item() == 0


def test_nan_rhs_reports_breakdown():
    pl = _plan(16, 16, 8, ("D", "P", "N"))
    eta = synth.random_field(16, 16, 8, seed=18)
    eta[3, 4, 5] = np.nan
    ed = _dev(eta)
    ud = torch.zeros_like(ed)
    st, info = pl.solve(ed, ud, tol=1e-10, maxit=10, zero_guess=True)
    assert st == 5  # TPCG_ERR_BREAKDOWN


def test_maxit_reports_not_converged():
    pl = _plan(32, 32, 16, ("D", "N", "DN"))
    ed = _dev(synth.random_field(32, 32, 16, seed=19))
    ud = torch.zeros_like(ed)
    st, info = pl.solve(ed, ud, tol=1e-15 * 1.0001, maxit=1, zero_guess=True)
    assert st in (0, 4)
    if st == 4:
        assert info["iters"] == 1


def test_invalid_arguments():
    from paper_2501_03377_gb300 import binding as b

    pl = _plan(8, 8, 8, ("P", "P", "N"))
    ed = _dev(np.zeros((8, 8, 8)))
    assert b.tpcg_solve(pl.handle, ed.data_ptr(), ed.data_ptr() + 0, 0.0, 10, 0)[0] == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_solve(pl.handle, ed.data_ptr(), ed.data_ptr(), 1e-10, 0, 0)[0] == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_solve(pl.handle, 0, ed.data_ptr(), 1e-10, 5, 0)[0] == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_precond_apply(pl.handle, ed.data_ptr(), ed.data_ptr()) == b.TPCG_ERR_INVALID_ARG


def test_rhs_add_bc_matches_oracle():
    nx, ny, nz, bcs, h = 12, 9, 7, ("DN", "ND", "D"), (0.5, 2.0, 1.5)
    eta = synth.random_field(nx, ny, nz, seed=20)
    bv = [0.3, -0.5, 1.25, 2.0, -1.0, 0.75]
    pl = _plan(nx, ny, nz, bcs, h)
    ed = _dev(eta)
    pl.rhs_add_bc(ed, bv)
    torch.cuda.synchronize()
    ref = from_oracle(o.rhs_add_bc(to_oracle(eta), bcs, h, bv))
    assert np.abs(ed.cpu().numpy() - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("nx,ny,nz,bcs,h,bv", [
    (12, 9, 7, ("DN", "ND", "D"), (0.5, 2.0, 1.5), [0.3, -0.5, 1.25, 2.0, -1.0, 0.75]),
    (33, 17, 9, ("P", "N", "P"), (1.0, 0.7, 1.3), None),
    (40, 24, 1, ("D", "N", "P"), (1.0, 1.0, 1.0), [1.0, -2.0, 0.5, 0.25, 0.0, 0.0]),
    (16, 16, 8, ("N", "N", "N"), (1.0, 1.0, 1.0), [0.1, 0.2, -0.3, 0.4, 0.5, -0.6]),
])
def test_efield_matches_oracle(nx, ny, nz, bcs, h, bv):
    """epsilon = -grad(ups) (Sec. 2) with the face data of Sec. 3.4.2, every component."""
    ups = synth.random_field(nx, ny, nz, seed=21)
    pl = _plan(nx, ny, nz, bcs, h)
    ud = _dev(ups)
    ex, ey = torch.empty_like(ud), torch.empty_like(ud)
    ez = torch.empty_like(ud) if nz > 1 else None
    pl.efield(ud, ex, ey, ez, bval=bv)
    torch.cuda.synchronize()
    ref = o.efield(to_oracle(ups), oracle_bcs(bcs, nz), h, bv)
    got = [ex, ey] + ([ez] if ez is not None else [])
    assert len(ref) == len(got)
    for g, r in zip(got, ref):
        r = from_oracle(r)
        assert np.abs(g.cpu().numpy() - r).max() <= 1e-14 * max(1.0, np.abs(r).max())


def test_efield_of_solution_recovers_gauss_law():
    """div(epsilon) of the computed potential reproduces eta_hat on a periodic grid (the discrete
    divergence of the central-difference field is the wide-stencil Laplacian, so compare spectrally
    smooth data): the field's divergence correlates with eta at the level of the discretisation."""
    nx, ny, nz = 32, 32, 16
    w = synth.defect_rhs(nx, ny, nz, ("P", "P", "P"), 6, 3.0, seed=22)
    pl = _plan(nx, ny, nz, ("P", "P", "P"))
    ed = _dev(w)
    ud = torch.zeros_like(ed)
    st, info = pl.solve(ed, ud, tol=1e-12, maxit=20, zero_guess=True)
    assert st == 0, info
    ex, ey, ez = (torch.empty_like(ud) for _ in range(3))
    pl.efield(ud, ex, ey, ez)
    torch.cuda.synchronize()
    ref = o.efield(to_oracle(ud.cpu().numpy()), ("P", "P", "P"), (1.0, 1.0, 1.0))
    for g, r in zip((ex, ey, ez), ref):
        assert np.abs(g.cpu().numpy() - from_oracle(r)).max() <= 1e-14 * max(1.0, np.abs(r).max())
    # discrete Gauss law: central divergence of the central-difference field = eta_hat to O(h^2)
    div = sum(np.roll(f.cpu().numpy(), -1, axis=a) - np.roll(f.cpu().numpy(), 1, axis=a)
              for f, a in ((ex, 2), (ey, 1), (ez, 0))) / 2.0
    eta_hat = w - w.mean()
    assert np.corrcoef(div.ravel(), eta_hat.ravel())[0, 1] > 0.9


def test_efield_argument_errors():
    from paper_2501_03377_gb300 import binding as b

    pl = _plan(8, 8, 8, ("P", "P", "N"))
    ud = _dev(np.zeros((8, 8, 8)))
    e = torch.empty_like(ud)
    assert b.tpcg_efield(pl.handle, ud.data_ptr(), None, e.data_ptr(), e.data_ptr(), 0) == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_efield(pl.handle, ud.data_ptr(), None, ud.data_ptr(), e.data_ptr(), e.data_ptr()) == \
        b.TPCG_ERR_INVALID_ARG


def test_film_workload_fp64_full_size():
    """128x128x64 film, P/P/DN, FP64 form, tol 1e-10, against the oracle at full size."""
    w = synth.workload_film_128(seed=0)
    pl = _plan(w["nx"], w["ny"], w["nz"], w["bcs"])
    ed = _dev(w["eta"])
    ud = torch.zeros_like(ed)
    st, info = pl.solve(ed, ud, tol=w["tol"], maxit=20, zero_guess=True)
    assert st == 0, info
    sh = (128, 128, 64)
    ref = o.pcg(sh, w["bcs"], (1, 1, 1), to_oracle(w["eta"]), tol=1e-13)
    assert rel_err(ud.cpu().numpy(), from_oracle(ref.U)) <= 1e-9
    assert info["rel_res_true"] <= 1e-10


# ---------------------------------------------------------------- comparators (Sec. 4.3.1, Experiment 2)
@pytest.mark.parametrize("p,omega", [(1, 1.0), (2, 1.3), (3, 1.3), (4, 2.0)])
@pytest.mark.parametrize("nx,ny,nz,bcs,h", [(12, 9, 7, ("DN", "ND", "D"), (0.5, 2.0, 1.5)),
                                            (33, 17, 9, ("P", "N", "P"), (1.0, 1.0, 1.0)),
                                            (40, 24, 1, ("D", "N", "P"), (1.0, 0.7, 1.0))])
def test_jacobi_precond_apply_matches_oracle(p, omega, nx, ny, nz, bcs, h):
    r = synth.random_field(nx, ny, nz, seed=23)
    pl = _plan(nx, ny, nz, bcs, h)
    pl.set_precond("jacobi", p, omega)
    rd = _dev(r)
    zd = torch.empty_like(rd)
    pl.precond(rd, zd)
    torch.cuda.synchronize()
    ob = oracle_bcs(bcs, nz)
    Os, Dinv = o.jacobi_init((nx, ny, nz), ob, h, omega)
    ref = from_oracle(o.jacobi_apply(to_oracle(r), Os, Dinv, p))
    assert np.abs(zd.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()


def test_none_precond_is_identity():
    r = synth.random_field(16, 12, 8, seed=24)
    pl = _plan(16, 12, 8, ("P", "D", "N"))
    pl.set_precond("none")
    rd = _dev(r)
    zd = torch.zeros_like(rd)
    pl.precond(rd, zd)
    torch.cuda.synchronize()
    assert torch.equal(zd, rd)


@pytest.mark.parametrize("kind", ["none", "jacobi"])
@pytest.mark.parametrize("nx,ny,nz,bcs", [(24, 20, 12, ("P", "P", "N")), (20, 16, 1, ("D", "DN", "P"))])
def test_comparator_solves_match_oracle(kind, nx, ny, nz, bcs):
    eta = synth.defect_rhs(nx, ny, nz, bcs, 4, 2.0, seed=25)
    pl = _plan(nx, ny, nz, bcs)
    pl.set_precond(kind, 3, 1.3)
    ed = _dev(eta)
    ud = torch.zeros_like(ed)
    st, info = pl.solve(ed, ud, tol=1e-10, maxit=2000, zero_guess=True)
    assert st == 0, info
    assert info["rel_res_true"] <= 1e-10
    ref = o.pcg((nx, ny, nz), oracle_bcs(bcs, nz), (1, 1, 1), to_oracle(eta), tol=1e-13, maxit=4000, precond=kind)
    assert rel_err(ud.cpu().numpy(), from_oracle(ref.U)) <= 1e-7


def test_comparator_ordering_on_gpu():
    """Experiment 2, qualitatively: p-inv needs the fewest iterations, then Jacobi(3, 1.3), then CG."""
    nx, ny, nz, bcs = 100, 50, 1, ("P", "P", "P")
    eta = synth.defect_rhs(nx, ny, nz, bcs, 10, 2.0, seed=26)
    iters = {}
    for kind in ("pinv", "jacobi", "none"):
        pl = _plan(nx, ny, nz, bcs)
        pl.set_precond(kind, 3, 1.3)
        ud = torch.zeros((nz, ny, nx), dtype=torch.float64, device="cuda")
        st, info = pl.solve(_dev(eta), ud, tol=1e-10, maxit=5000, zero_guess=True)
        assert st == 0, (kind, info)
        iters[kind] = info["iters"]
    assert iters["pinv"] < iters["jacobi"] < iters["none"], iters


def test_set_precond_argument_errors():
    from paper_2501_03377_gb300 import Plan, binding as b

    pl = _plan(8, 8, 8, ("P", "P", "N"))
    assert b.tpcg_plan_set_precond(pl.handle, 7, 3, 1.3) == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_plan_set_precond(pl.handle, b.TPCG_PRECOND_JACOBI, 0, 1.3) == b.TPCG_ERR_INVALID_ARG
    assert b.tpcg_plan_set_precond(pl.handle, b.TPCG_PRECOND_JACOBI, 3, 0.5) == b.TPCG_ERR_INVALID_ARG
    mixed = Plan(16, 16, 16, ("P", "P", "N"), prec="fp16")
    assert b.tpcg_plan_set_precond(mixed.handle, b.TPCG_PRECOND_NONE, 3, 1.3) == b.TPCG_ERR_UNSUPPORTED
    assert b.tpcg_plan_set_precond(mixed.handle, b.TPCG_PRECOND_PINV, 3, 1.3) == b.TPCG_OK
