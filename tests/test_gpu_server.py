"""tpcg_server_*: continuous batching of independent solves with warm-started sessions.

The central property: every result of a mixed request stream equals the
result of the same session's requests run alone (same plans, same launch
configurations, deterministic reductions, warm starts in submission order).
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


SESSIONS = [  # (seed, nx, ny, nz, bcs, prec)
    (11, 32, 24, 16, ("P", "P", "N"), "fp16"),
    (12, 40, 40, 1, ("D", "D", "D"), "fp64"),
    (13, 24, 32, 20, ("N", "D", "DN"), "bf16"),
    (14, 48, 16, 12, ("P", "N", "P"), "fp16"),
    (15, 40, 24, 16, ("P", "P", "N"), "bf16x3"),
    (16, 33, 20, 12, ("ND", "P", "D"), "tf32"),
]
STEPS = 3


def _session_rhs():
    out = []
    for seed, nx, ny, nz, bcs, prec in SESSIONS:
        s = synth.ServingSession(seed, nx, ny, nz, bcs, n_defects=30)
        steps = []
        for _ in range(STEPS):
            steps.append(s.rhs())
            s.step()
        out.append(steps)
    return out


def _run(server, order, rhs):
    tickets = {}
    for (si, k) in order:
        seed, nx, ny, nz, bcs, prec = SESSIONS[si]
        tickets[(si, k)] = server.submit(rhs[si][k], bcs, prec=prec, session=100 + si, tol=1e-10, maxit=60)
    res = {}
    for key, t in tickets.items():
        st, u, info = server.wait(t, timeout_s=60.0)
        assert st == 0, (key, st, info)
        res[key] = (u, info)
    return res


def test_server_mix_equals_alone_and_oracle():
    from paper_2501_03377_gb300 import Server

    rhs = _session_rhs()
    mix_order = [(si, k) for k in range(STEPS) for si in range(len(SESSIONS))]
    srv = Server(max_slots=4)
    mixed = _run(srv, mix_order, rhs)
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == len(mix_order) and stats["failed"] == 0
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    for si in range(len(SESSIONS)):
        alone_srv = Server(max_slots=1)
        alone = _run(alone_srv, [(si, k) for k in range(STEPS)], rhs)
        alone_srv.close()
        for k in range(STEPS):
            assert np.array_equal(alone[(si, k)][0], mixed[(si, k)][0]), (si, k)
            assert alone[(si, k)][1]["iters"] == mixed[(si, k)][1]["iters"]
    for si, (seed, nx, ny, nz, bcs, prec) in enumerate(SESSIONS):
        sh, ob = (nx, ny, nz), oracle_bcs(bcs, nz)
        for k in range(STEPS):
            ref = o.pcg(sh, ob, (1, 1, 1), to_oracle(rhs[si][k]), tol=1e-13)
            assert rel_err(mixed[(si, k)][0], from_oracle(ref.U)) <= 1e-9
            assert mixed[(si, k)][1]["rel_res_true"] <= 1e-10
        # warm starts from the previous step's solution need no more iterations than the cold first step
        assert max(mixed[(si, k)][1]["iters"] for k in range(1, STEPS)) <= mixed[(si, 0)][1]["iters"]


def test_server_admission_budget():
    from paper_2501_03377_gb300 import Server, binding

    eta = synth.defect_rhs(64, 64, 32, ("P", "P", "N"), 10, 1.5, seed=3)
    tiny = Server(hbm_budget=1 << 20, max_slots=2)
    t = tiny.submit(eta, ("P", "P", "N"), prec="fp16")
    st, u, info = tiny.wait(t, 30.0)
    assert st == binding.TPCG_ERR_ADMISSION
    assert tiny.stats()["rejected"] == 1
    tiny.close()
    # room for about one plan at a time: requests of different grids still all complete
    small = Server(hbm_budget=40 << 20, max_slots=4)
    shapes = [(48, 40, 24), (40, 48, 24), (32, 32, 32), (48, 40, 24)]
    tickets = [small.submit(synth.defect_rhs(nx, ny, nz, ("P", "D", "N"), 8, 1.5, seed=i), ("P", "D", "N"))
               for i, (nx, ny, nz) in enumerate(shapes)]
    for t in tickets:
        st, u, info = small.wait(t, 60.0)
        assert st == 0 and info["rel_res_true"] <= 1e-10
    assert small.stats()["device_bytes"] <= 40 << 20
    small.close()


def test_server_poll_pending_and_unknown_ticket():
    from paper_2501_03377_gb300 import Server, binding

    srv = Server(max_slots=2)
    eta = synth.defect_rhs(128, 128, 64, ("P", "P", "DN"), 50, 1.5, seed=4)
    t = srv.submit(eta, ("P", "P", "DN"), prec="fp64")
    first = srv.poll(t)[0]
    assert first in (binding.TPCG_PENDING, 0)
    st, u, info = srv.wait(t, 60.0)
    assert st == 0
    assert binding.tpcg_server_poll(srv.handle, t, 0)[0] == binding.TPCG_ERR_UNKNOWN_TICKET
    assert binding.tpcg_server_poll(srv.handle, 987654, 0)[0] == binding.TPCG_ERR_UNKNOWN_TICKET
    srv.close()


def test_server_borrowed_rhs_equal_copied():
    from paper_2501_03377_gb300 import Server

    bcs = ("P", "D", "N")
    eta = synth.defect_rhs(40, 32, 16, bcs, 10, 1.5, seed=5)
    srv = Server(max_slots=3)
    t_copy = srv.submit(eta, bcs)
    eh = torch.from_numpy(eta.copy()).pin_memory()
    t_host = srv.submit(eh, bcs, borrow=True)
    ed = torch.from_numpy(eta.copy()).cuda()
    t_dev = srv.submit(ed, bcs, borrow=True)
    out = [srv.wait(t, 60.0) for t in (t_copy, t_host, t_dev)]
    srv.close()
    assert all(st == 0 for st, _, _ in out)
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][1], out[2][1])
