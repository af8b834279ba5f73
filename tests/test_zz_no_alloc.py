"""The allocation-free residual check against the solver's own report.

tpcg_residual_norms_noalloc is for callers that cannot allocate device memory
when they verify a solution (a time-stepping loop that must not trigger the
synchronisation an allocation can cause, or an application whose device
memory budget is fixed at start-up); it keeps its scratch in a static device
array instead of a plan.  This file is collected
last so that a run stopping at the first failure has run every other test.
It must pass alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

from inputs import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_03377_gb300 import build

    build.build()


@pytest.mark.parametrize("shape,bcs,prec,h", [((40, 24, 12), ("P", "P", "N"), "fp64", (1.0, 1.0, 1.0)),
                                              ((33, 17, 9), ("D", "ND", "DN"), "fp16", (1.0, 1.0, 1.0)),
                                              ((36, 20, 10), ("N", "DN", "P"), "fp64", (1.0, 0.5, 2.0)),
                                              ((64, 64, 1), ("D", "D", "D"), "bf16", (1.0, 1.0, 1.0))])
def test_noalloc_residual_matches_solver_report_twice(shape, bcs, prec, h):
    """Two calls in a row against the solver's report and against the residual recomputed on the host
    with the oracle's assembled operator (unequal spacings included: an axis mix-up of h fails)."""
    import oracle as o
    from paper_2501_03377_gb300 import Plan, binding

    nx, ny, nz = shape
    eta = synth.defect_rhs(nx, ny, nz, bcs, 6, 1.5, seed=31, noise_std=1e-3) + 1e-7  # nonzero mean
    pl = Plan(nx, ny, nz, bcs, h=h, prec=prec)
    ed = torch.from_numpy(eta).cuda()
    ud = torch.zeros_like(ed)
    st, info = pl.solve(ed, ud, tol=1e-10, maxit=60, zero_guess=True)
    assert st == 0, info
    stream = torch.cuda.current_stream().cuda_stream
    results = []
    for _ in range(2):  # two calls in a row share the static scratch
        out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        rc = binding.tpcg_residual_norms_noalloc(nx, ny, nz, bcs, h, ed.data_ptr(), ud.data_ptr(),
                                                 out.data_ptr(), stream)
        assert rc == 0
        torch.cuda.synchronize()
        results.append(out.cpu().numpy())
    for res in results:
        rel = res[0] / res[1]
        # the same tolerance the solver tests use for two FP64 residual evaluations
        assert abs(rel - info["rel_res_true"]) <= 1e-2 * info["rel_res_true"] + 1e-14
        assert abs(res[1] - info["eta_norm"]) <= 1e-12 * info["eta_norm"]
        assert abs(res[2] - info["removed_mean"]) <= 1e-12 * np.abs(eta).max()
    assert np.array_equal(results[0], results[1])
    # the host residual with the oracle's assembled Kronecker sum (x fastest: the oracle's (n, q, t) order)
    ob = (bcs[0], bcs[1], None if nz == 1 else bcs[2])
    L = o.kron_sum((nx, ny, nz), ob, h)
    e = eta.transpose(2, 1, 0)
    eh = e - (e.mean() if o.is_singular((nx, ny, nz), ob) else 0.0)
    u = ud.cpu().numpy().transpose(2, 1, 0)
    r_host = np.linalg.norm(o.vec(eh) - L @ o.vec(u))
    n_host = np.linalg.norm(o.vec(eh))
    for res in results:
        assert abs(res[1] - n_host) <= 1e-12 * n_host
        # two FP64 evaluations of a residual ~1e-10 of ||eta||: they differ by rounding of L u (~1e-16 of
        # ||L u|| ~ ||eta||), i.e. up to a few 1e-6 relative to the residual itself
        assert abs(res[0] - r_host) <= 1e-2 * r_host + 1e-14 * n_host


def test_noalloc_rejects_bad_arguments():
    from paper_2501_03377_gb300 import binding

    t = torch.zeros((4, 4, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    rc = binding.tpcg_residual_norms_noalloc(2, 4, 4, "PPN", (1, 1, 1), t.data_ptr(), t.data_ptr(), out.data_ptr(), 0)
    assert rc == binding.TPCG_ERR_INVALID_ARG
    for h in ((1, float("inf"), 1), (1, float("nan"), 1), (0, 1, 1)):  # spacing rules of tpcg_plan_create
        rc = binding.tpcg_residual_norms_noalloc(4, 4, 4, "PPN", h, t.data_ptr(), t.data_ptr(), out.data_ptr(), 0)
        assert rc == binding.TPCG_ERR_INVALID_ARG
    rc = binding.tpcg_residual_norms_noalloc(65536, 65536, 4, "PPN", (1, 1, 1), t.data_ptr(), t.data_ptr(),
                                             out.data_ptr(), 0)
    assert rc == binding.TPCG_ERR_UNSUPPORTED
