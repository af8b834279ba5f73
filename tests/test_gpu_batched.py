"""tpcg_solve_batched: many independent solves of different grids and BCs in one call.

Every batched result must equal the result of tpcg_solve on the same input
bitwise (same kernels, same launch configuration, deterministic reductions),
and small cases must match the oracle at the solver's bars.
"""
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


def _make_batch(specs, prec, streams=True):
    from paper_2501_03377_gb300 import Plan

    plans, etas, ups, keep = [], [], [], []
    for spec in specs:
        nx, ny, nz, bcs, nrhs = spec["nx"], spec["ny"], spec["nz"], spec["bcs"], spec["nrhs"]
        st = torch.cuda.Stream() if streams else torch.cuda.current_stream()
        keep.append(st)
        plans.append(Plan(nx, ny, nz, bcs, prec=prec, stream=st.cuda_stream))
        rhs = np.stack([synth.batched_rhs(spec, r) for r in range(nrhs)])
        e = torch.from_numpy(rhs).cuda()
        etas.append(e)
        ups.append(torch.zeros_like(e))
    return plans, etas, ups, keep


def _run_batch(plans, etas, ups, specs, tol=1e-10, maxit=60, flags=1):
    from paper_2501_03377_gb300 import binding

    torch.cuda.synchronize()
    st, infos = binding.tpcg_solve_batched([p.handle for p in plans], [s["nrhs"] for s in specs],
                                           [e.data_ptr() for e in etas], [u.data_ptr() for u in ups],
                                           [tol] * len(plans), maxit, flags)
    torch.cuda.synchronize()
    return st, infos


SMALL = [dict(nx=16, ny=12, nz=8, bcs=("P", "N", "P"), nrhs=2, seed=1),
         dict(nx=24, ny=16, nz=1, bcs=("D", "DN", "D"), nrhs=1, seed=2),
         dict(nx=20, ny=20, nz=10, bcs=("N", "N", "N"), nrhs=3, seed=3),
         dict(nx=33, ny=9, nz=7, bcs=("ND", "P", "D"), nrhs=1, seed=4),
         dict(nx=32, ny=32, nz=16, bcs=("P", "P", "DN"), nrhs=2, seed=5)]


@pytest.mark.parametrize("prec", ["fp64", "fp16", "bf16", "tf32", "bf16x3"])
def test_batched_equals_solo_and_oracle(prec):
    from paper_2501_03377_gb300 import Plan

    plans, etas, ups, _ = _make_batch(SMALL, prec)
    st, infos = _run_batch(plans, etas, ups, SMALL)
    assert st == 0, [i["status"] for i in infos]
    k = 0
    for spec, e, u in zip(SMALL, etas, ups):
        solo = Plan(spec["nx"], spec["ny"], spec["nz"], spec["bcs"], prec=prec)
        sh = (spec["nx"], spec["ny"], spec["nz"])
        ob = oracle_bcs(spec["bcs"], spec["nz"])
        for r in range(spec["nrhs"]):
            us = torch.zeros_like(e[r])
            st1, info1 = solo.solve(e[r].contiguous(), us, tol=1e-10, maxit=60, zero_guess=True)
            assert st1 == 0
            assert torch.equal(us, u[r]), (spec, r)
            assert infos[k]["iters"] == info1["iters"]
            ref = o.pcg(sh, ob, (1, 1, 1), to_oracle(e[r].cpu().numpy()), tol=1e-13)
            assert rel_err(u[r].cpu().numpy(), from_oracle(ref.U)) <= 1e-9
            assert infos[k]["rel_res_true"] <= 1e-10
            k += 1


def test_batched_same_plan_twice_and_argument_errors():
    from paper_2501_03377_gb300 import Plan, binding

    spec = dict(nx=16, ny=16, nz=8, bcs=("P", "D", "N"), nrhs=1, seed=7)
    pl = Plan(16, 16, 8, spec["bcs"], prec="fp16")
    e1 = torch.from_numpy(synth.batched_rhs(spec, 0)[None]).cuda()
    e2 = torch.from_numpy(synth.batched_rhs(spec, 1)[None]).cuda()
    u1, u2 = torch.zeros_like(e1), torch.zeros_like(e2)
    st, infos = binding.tpcg_solve_batched([pl.handle, pl.handle], [1, 1], [e1.data_ptr(), e2.data_ptr()],
                                           [u1.data_ptr(), u2.data_ptr()], [1e-10, 1e-10], 60, 1)
    torch.cuda.synchronize()
    assert st == 0 and len(infos) == 2
    for e, u in ((e1, u1), (e2, u2)):
        us = torch.zeros_like(e[0])
        pl.solve(e[0].contiguous(), us, tol=1e-10, maxit=60, zero_guess=True)
        assert torch.equal(us, u[0])
    assert binding.tpcg_solve_batched([pl.handle], [1], [e1.data_ptr()], [u1.data_ptr()], [0.0], 60, 1)[0] == \
        binding.TPCG_ERR_INVALID_ARG
    assert binding.tpcg_solve_batched([pl.handle], [1], [e1.data_ptr()], [u1.data_ptr()], [1e-10], 0, 1)[0] == \
        binding.TPCG_ERR_INVALID_ARG


@pytest.mark.parametrize("prec,grain", [("fp16", 4), ("bf16x3", 4), ("bf16x3", 16)])
def test_batched_48_mixed_solves(prec, grain):
    """48 independent solves, grids {64..160}^2 x {32..96}, BC per axis from {P,D,N,DN,ND}, 1-8 RHS each,
    FP16 or split BF16 mixed preconditioner (the bench's batched record runs the latter at sweep grain 16),
    tol 1e-10; a sample of them is re-solved alone (same grain) and must match bitwise."""
    from paper_2501_03377_gb300 import Plan, binding

    specs = synth.batched_specs(seed=0)
    plans, etas, ups, _ = _make_batch(specs, prec)
    for pl in plans:
        pl.set_option(binding.TPCG_OPT_SWEEP_GRAIN, grain)
    st, infos = _run_batch(plans, etas, ups, specs)
    assert st == 0, [i["status"] for i in infos if i["status"]]
    assert len(infos) == sum(s["nrhs"] for s in specs)
    assert max(i["rel_res_true"] for i in infos) <= 1e-10
    for s in (0, 7, 23, 47):
        spec = specs[s]
        solo = Plan(spec["nx"], spec["ny"], spec["nz"], spec["bcs"], prec=prec)
        solo.set_option(binding.TPCG_OPT_SWEEP_GRAIN, grain)
        us = torch.zeros_like(etas[s][0])
        solo.solve(etas[s][0].contiguous(), us, tol=1e-10, maxit=60, zero_guess=True)
        assert torch.equal(us, ups[s][0])
        if o.is_singular((spec["nx"], spec["ny"], spec["nz"]), spec["bcs"]):
            assert abs(ups[s][0].mean().item()) <= 1e-14 * ups[s][0].abs().max().item()
    # every spec: the true residual of its last right-hand side recomputed on the host with the oracle's
    # assembled Kronecker sum (independent of the GPU's own residual check)
    for spec, e, u in zip(specs, etas, ups):
        sh = (spec["nx"], spec["ny"], spec["nz"])
        L = o.kron_sum(sh, spec["bcs"])
        r = spec["nrhs"] - 1
        eh = to_oracle(e[r].cpu().numpy())
        if o.is_singular(sh, spec["bcs"]):
            eh = o.center(eh)
        res = np.linalg.norm(o.vec(eh) - L @ o.vec(to_oracle(u[r].cpu().numpy()))) / np.linalg.norm(eh)
        assert res <= 1e-10, (spec, res)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_sweep_grain_range_and_results(prec):
    """TPCG_OPT_SWEEP_GRAIN accepts 1..64 only; at the extremes the solve still matches the oracle, and a grain
    is bitwise reproducible (two solves at grain 64 agree)."""
    from paper_2501_03377_gb300 import Plan, binding
    from paper_2501_03377_gb300.binding import TpcgError

    spec = dict(nx=40, ny=24, nz=12, bcs=("P", "P", "N"), nrhs=1, seed=11)
    pl = Plan(spec["nx"], spec["ny"], spec["nz"], spec["bcs"], prec=prec)
    for bad in (0, 65, -3):
        with pytest.raises(TpcgError):
            pl.set_option(binding.TPCG_OPT_SWEEP_GRAIN, bad)
    e = torch.from_numpy(synth.batched_rhs(spec, 0)).cuda()
    ref = o.pcg((40, 24, 12), oracle_bcs(spec["bcs"], 12), (1, 1, 1), to_oracle(e.cpu().numpy()), tol=1e-13)
    outs = []
    for grain in (1, 64, 64, 4):
        pl.set_option(binding.TPCG_OPT_SWEEP_GRAIN, grain)
        u = torch.zeros_like(e)
        st, info = pl.solve(e, u, tol=1e-10, maxit=60, zero_guess=True)
        assert st == 0 and info["rel_res_true"] <= 1e-10
        assert rel_err(u.cpu().numpy(), from_oracle(ref.U)) <= 1e-9
        outs.append(u)
    assert torch.equal(outs[1], outs[2])
    pl.close()
