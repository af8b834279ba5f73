#!/usr/bin/env python
"""Benchmark of the PCG hot path: solves/s on the 256x256xnz P/P/N cuboid.

One step = one complete solve (Algorithm 1 with the pseudoinverse
preconditioner, zero initial guess, tol 1e-10) of a synthetic charged-defect
right-hand side already resident in HBM, each step its own 67 MB copy (four
seeded right-hand sides in rotation), so every step's data exceed the 129 MB
L2.  The timed steps go through tpcg_solve_batched spread over --concurrency
plans (default 5; sweep grain 32 on them), each on its own stream: the library runs the queues of
different plans concurrently.  single_plan reports the same steps solved one
after the other on one plan with tpcg_solve.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec bf16x3|fp16|bf16|tf32|fp64] [--nz 128]
    python bench.py --impl reference   # the CPU oracle as the reference arm

Multi-GPU: replicas only (each rank solves its own right-hand sides; no data
collective); value = all solves of all ranks / max-over-ranks time.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "256\u00b3 solves/s at rel-res 1e-10, TC-mixed vs FP64 PCG; serving p50/p99 ms"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12  # SMs x FP64 FMA/clk/SM x 2 flop x max SM clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 200; the reference arm, one full oracle solve per step: 20)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="auto", choices=["auto", "fp16", "bf16", "tf32", "bf16x3", "fp64"])
    ap.add_argument("--no-bf16-compare", action="store_true")
    ap.add_argument("--nz", type=int, default=128)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=2000)
    ap.add_argument("--serving-rate", type=float, default=200.0)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-comparators", action="store_true")
    ap.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-solves", type=int, default=10, help="oracle solves of the cpu_baseline (all cores)")
    ap.add_argument("--no-cube", action="store_true", help="skip the 256x256x256 record")
    ap.add_argument("--no-variants", action="store_true", help="skip the odd-nx / unequal-spacing record")
    ap.add_argument("--sweep-grain", type=int, default=32,
                    help="TPCG_OPT_SWEEP_GRAIN of the concurrent timed plans (0: the library's default; a single "
                         "plan keeps the default)")
    ap.add_argument("--concurrency", type=int, default=5,
                    help="plans (each on its own stream) the timed steps are spread over")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 20 if args.impl == "reference" else 200
    return args


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 50 ms) during the timed region: start() returns once the first sample has
    arrived, and stop() keeps the samples that arrived after that (all of them if none did)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.skip = 0

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
            return
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.005)
        self.skip = len(self.lines)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines[self.skip:] or self.lines
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload(nz, seeds):
    from inputs import synth

    return [synth.workload_cuboid_256(seed=s, nz=nz) for s in seeds]


def cpu_oracle_solves(w, tol, k):
    """k oracle solves (operator and eigenbases built once, outside the timed part): (seconds, result)."""
    import oracle as o

    sh = (w["nx"], w["ny"], w["nz"])
    L = o.kron_sum(sh, w["bcs"])
    pinv = o.pinv_init(sh, w["bcs"])
    H = w["eta"].transpose(2, 1, 0)
    total, res = 0.0, None
    for _ in range(k):
        t0 = time.perf_counter()
        res = o.pcg(sh, w["bcs"], (1.0, 1.0, 1.0), H, tol=tol, L=L, pinv=pinv)
        total += time.perf_counter() - t0
    return total, res


def cpu_oracle_solve(w, tol):
    """One oracle solve (operator and eigenbases built outside the timed part)."""
    return cpu_oracle_solves(w, tol, 1)


def cpu_one_thread(nz, tol, k):
    """The oracle on one host core: a child process with every BLAS/OpenMP pool limited to one thread
    (the limits must be set before numpy loads).  Returns (solves/s, k) or None."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", NUMEXPR_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", str(k), "--nz", str(nz), "--tol", str(tol)]
    try:
        out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
        d = json.loads(out.stdout.strip().splitlines()[-1])
        return k / d["seconds"], k
    except Exception:
        return None


def oracle_sample(args):
    """--oracle-sample K: K oracle solves of the bench workload on this process's threads (JSON line)."""
    w = workload(args.nz, [0])[0]
    secs, res = cpu_oracle_solves(w, args.tol, args.oracle_sample)
    print(json.dumps({"seconds": secs, "solves": args.oracle_sample, "iters": res.iters}), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return
    ws = workload(args.nz, [0])
    w = ws[0]
    cores = len(os.sched_getaffinity(0))
    for _ in range(max(0, min(args.warmup, 1))):
        cpu_oracle_solve(w, args.tol)
    times = []
    for _ in range(args.steps):
        dt, res = cpu_oracle_solve(w, args.tol)
        times.append(dt)
    total = sum(times)
    value = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "grid": [w["nx"], w["ny"], w["nz"]], "bcs": ",".join(w["bcs"]),
                   "tol": args.tol, "form": "oracle (numpy/scipy FP64 on host cores)"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full oracle solves of {w['name']} (seed 0), operator prebuilt"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "oracle_iters": res.iters, "oracle_true_res": res.true_res[-1],
    }
    print(json.dumps(line), flush=True)


def pick_prec(args):
    if args.prec != "auto":
        return args.prec
    from paper_2501_03377_gb300 import Plan

    # the split BF16 form first: its three refinement iterations beat the six of the FP16 form (measured on the
    # 256x256x128 cuboid: 950 against 833 solves/s on one plan)
    for prec in ("bf16x3", "fp16", "bf16"):
        try:
            Plan(16, 16, 16, ("P", "P", "N"), prec=prec).close()
            return prec
        except Exception:
            pass
    return "fp64"


def time_steps(plan, etas, ups, steps, tol, torch, barrier, sampler=None):
    """Run `steps` solves between synchronised barriers; returns (seconds, infos)."""
    infos = []
    barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()  # the plan issues its work on torch's current stream
    for s in range(steps):
        st, info = plan.solve(etas[s % len(etas)], ups, tol=tol, maxit=60, zero_guess=True)
        infos.append((st, info))
    e1.record()
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3
    clocks = sampler.stop() if sampler else None
    barrier()
    return dt, infos, clocks


def _pct(v, p):
    import numpy as np

    return float(np.percentile(np.asarray(v, dtype=np.float64), p)) if len(v) else None


def serving_stream(args, prec, torch):
    """One request stream: Poisson arrivals at --serving-rate from 16 warm-started sessions (grids 64..256 x
    64..256 x 32..192, random BCs); every request is the session's next time step, 1% of its defects moved
    since the previous step.  Each session keeps two pinned right-hand-side buffers (lent to the server):
    the buffer of step k held step k-2 and is brought to step k by the moves of steps k-1 and k, after step
    k-2's request has finished.  The field is scaled to the paper's norm on the first step, and that scale
    is kept (warm starts see a consistent time series)."""
    import numpy as np

    from inputs import synth
    from paper_2501_03377_gb300 import Server

    sessions = synth.serving_sessions(seed=0)
    scales = [ses.paper_scale() for ses in sessions]
    bufs = []
    for ses, sc in zip(sessions, scales):
        f = torch.from_numpy(sc * synth.gaussian_defects(
            (ses.nz, ses.ny, ses.nx), tuple(b == "P" for b in ses.bcs), ses.centres,
            np.full(len(ses.charges), ses.sigma), ses.charges, "charge")).pin_memory()
        bufs.append([f, f.clone().pin_memory()])
    state = [[0, 0] for _ in sessions]       # step each buffer holds
    moves = [[None] for _ in sessions]       # moves[i][k]: the moves of step k (k >= 1)
    pending = [[None, None] for _ in sessions]  # ticket of the request that borrowed each buffer
    steps = [0] * len(sessions)
    n = args.serving_requests
    arrivals = synth.poisson_arrivals(args.serving_rate, n, seed=1)
    order = np.random.default_rng(2).integers(0, len(sessions), size=n)
    srv = Server(max_slots=8)
    results = {}

    def collect(t):
        st, _, info = srv.wait(t, 600.0, want=False)
        results[t] = (st, info)

    # warm-up outside the measurement: one request per session builds its plan and session state (step 0)
    for i, ses in enumerate(sessions):
        collect(srv.submit(bufs[i][0], ses.bcs, prec=prec, session=i + 1, borrow=True))
    srv.reset_stats()
    results.clear()
    tickets, lag = [], []
    t0 = time.perf_counter()
    for k in range(n):
        i = int(order[k])
        ses = sessions[i]
        steps[i] += 1
        step = steps[i]
        moves[i].append(ses.step())
        b = step % 2
        if pending[i][b] is not None:  # the request of step - 2 still borrows this buffer
            collect(pending[i][b])
        buf = bufs[i][b]
        a = buf.numpy()
        for m in range(state[i][b] + 1, step + 1):
            ses.apply_moves(a, moves[i][m], scales[i])
        state[i][b] = step
        delay = t0 + arrivals[k] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        lag.append(max(0.0, -delay) * 1e3)
        t = srv.submit(buf, ses.bcs, prec=prec, session=i + 1, borrow=True)
        pending[i][b] = t
        tickets.append(t)
    for t in tickets:
        if t not in results:
            collect(t)
    stats = srv.stats()
    tim = srv.timings()
    srv.close()
    ok = [results[t] for t in tickets]
    worst = max((info["rel_res_true"] for st, info in ok if info), default=None)
    iters = [info["iters"] for st, info in ok if info]
    total = [r["total_ms"] for r in tim]
    out = {"requests": n, "rate_hz": args.serving_rate, "sessions": len(sessions), "form": prec,
           "p50_ms": stats["p50_ms"], "p99_ms": stats["p99_ms"], "mean_ms": stats["mean_ms"],
           "solves_per_s": stats["completed"] / stats["elapsed_s"] if stats["elapsed_s"] else None,
           "offered_span_s": float(arrivals[-1]), "failed": sum(1 for st, _ in ok if st != 0),
           "worst_rel_res_true": worst, "mean_iters": float(np.mean(iters)) if iters else None,
           "submit_lag_p99_ms": _pct(lag, 99),
           "plan_builds": sum(r["plan_built"] for r in tim)}
    # where the latency goes: mean of each cause overall, over the slowest 1 %, and per grid
    causes = ("queue_ms", "build_ms", "solve_ms", "copy_ms")
    out["mean_by_cause_ms"] = {c: float(np.mean([r[c] for r in tim])) for c in causes} if tim else None
    if tim:
        cut = _pct(total, 99)
        tail = [r for r in tim if r["total_ms"] >= cut]
        out["p99_tail_by_cause_ms"] = {c: float(np.mean([r[c] for r in tail])) for c in causes}
        out["p99_tail_grids"] = sorted({f"{r['nx']}x{r['ny']}x{r['nz']}" for r in tail})
        grids = {}
        for r in tim:
            grids.setdefault((r["nx"], r["ny"], r["nz"]), []).append(r)
        out["by_grid"] = {f"{g[0]}x{g[1]}x{g[2]}": {
            "requests": len(v), "p50_ms": _pct([r["total_ms"] for r in v], 50),
            "p99_ms": _pct([r["total_ms"] for r in v], 99),
            "solve_p50_ms": _pct([r["solve_ms"] for r in v], 50),
            "queue_p50_ms": _pct([r["queue_ms"] for r in v], 50),
            "mean_iters": float(np.mean([r["iters"] for r in v]))} for g, v in sorted(grids.items(), key=lambda kv: kv[0][0] * kv[0][1] * kv[0][2])}
    out["latency_note"] = ("submit call -> solution in pinned host memory (H2D of the lent pinned eta, the solve, "
                           "D2H); one warm-up request per session excluded; causes from tpcg_server_get_timings")
    return out


def run_serving(args, prec, torch):
    """The serving record: the mixed form and the FP64 form on the same request stream."""
    return {f"mixed_{prec}": serving_stream(args, prec, torch), "fp64": serving_stream(args, "fp64", torch)}


def run_comparators(torch, steps=3):
    """Experiment 2 on synthetic data: PCG with M = I, Jacobi(3, 1.3) and the pseudoinverse (FP64 and
    the mixed tensor-core form) on the 128x128x64 film (P/P/DN, 200 charged defects), tol 1e-10."""
    from paper_2501_03377_gb300 import Plan
    from inputs import synth

    w = synth.workload_film_128(seed=0)
    eta = torch.from_numpy(w["eta"]).cuda()
    ups = torch.zeros_like(eta)
    out = {"workload": w["name"], "tol": w["tol"]}
    for name, prec, kind in (("cg", "fp64", "none"), ("jacobi_3_1.3", "fp64", "jacobi"),
                             ("pinv_fp64", "fp64", "pinv"), ("pinv_fp16", "fp16", "pinv")):
        pl = Plan(w["nx"], w["ny"], w["nz"], w["bcs"], prec=prec)
        pl.set_precond(kind, 3, 1.3)
        pl.solve(eta, ups, tol=w["tol"], maxit=5000, zero_guess=True)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        infos = [pl.solve(eta, ups, tol=w["tol"], maxit=5000, zero_guess=True)[1] for _ in range(steps)]
        e1.record()
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) / 1e3
        out[name] = {"solves_per_s": steps / dt, "ms_per_solve": 1e3 * dt / steps, "iters": infos[-1]["iters"],
                     "rel_res_true": max(i["rel_res_true"] for i in infos),
                     "status": max(i["status"] for i in infos)}
        pl.close()
    return out


def run_efield(plan, ups, torch, reps=10):
    """epsilon = -grad(ups) on the bench grid: algorithmic bytes 32 per point (ups in, three components out)."""
    nz, ny, nx = ups.shape
    ex, ey, ez = (torch.empty_like(ups) for _ in range(3))
    plan.efield(ups, ex, ey, ez)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        plan.efield(ups, ex, ey, ez)
    e1.record()
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3 / reps
    return {"us_per_call": 1e6 * dt, "achieved_gbs": 32.0 * nx * ny * nz / dt / 1e9, "unit": "GB/s",
            "bytes_per_point": 32}


def run_laplacian(ups, torch, hbm_peak, reps=10):
    """The FP64 form's stencil w = L x (tpcg_apply_laplacian) on the bench grid: 16 B per point (x in, w out)."""
    from paper_2501_03377_gb300 import Plan

    nz, ny, nx = ups.shape
    p64 = Plan(nx, ny, nz, ("P", "P", "N"), prec="fp64")
    x = torch.randn_like(ups)
    w = torch.empty_like(ups)
    p64.laplacian(x, w)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        p64.laplacian(x, w)
    e1.record()
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3 / reps
    p64.close()
    gbs = 16.0 * nx * ny * nz / dt / 1e9
    return {"kernel": "k_apply_laplacian", "us_per_call": 1e6 * dt, "achieved_gbs": gbs, "unit": "GB/s",
            "bytes_per_point": 16, "frac": gbs / hbm_peak}


def run_variants(args, prec, torch, hbm_peak, steps=10):
    """The stencil variants off the main workload's path: odd nx (one-point-per-thread direction and update,
    the per-pass tensor-core sequence) and unequal spacings (three stencil weights), 255 x 256 x 128 P/P/N with
    h = (1, 0.5, 2), 2000 charged defects; one plan, tpcg_solve, with the per-kernel fractions of an
    instrumented pass."""
    from inputs import synth
    from paper_2501_03377_gb300 import Plan

    dev = torch.device("cuda", torch.cuda.current_device())
    nx, ny, nz, bcs, h = 255, 256, 128, ("P", "P", "N"), (1.0, 0.5, 2.0)
    etas = [torch.from_numpy(synth.defect_rhs(nx, ny, nz, bcs, 2000, (1.0, 4.0), seed=s)).to(dev) for s in range(4)]
    ups = torch.zeros_like(etas[0])
    pl = Plan(nx, ny, nz, bcs, h=h, prec=prec)
    nobar = lambda: None  # noqa: E731
    for s in range(3):
        pl.solve(etas[s % 4], ups, tol=args.tol, maxit=60, zero_guess=True)
    dt, infos, _ = time_steps(pl, etas, ups, steps, args.tol, torch, nobar)
    pl.profile_begin()
    _, pinfos, _ = time_steps(pl, etas, ups, steps, args.tol, torch, nobar)
    kst = pl.profile_end()
    N = nx * ny * nz
    iters = sum(i["iters"] for (_, i) in pinfos)
    applies = sum(i["precond_applies"] for (_, i) in pinfos)
    checks = sum(i.get("checks", 0) for (_, i) in pinfos)
    kernels = {}
    for k, v in kst.items():
        amount, unit, bound, _ = kernel_work(k, prec, N, (nx, ny, nz), iters, applies, steps, checks,
                                             pl.precond_launches())
        rec = {"launches": v["launches"], "ms": round(v["total_ms"], 4)}
        if amount is not None and unit == "GB":
            rec["frac"] = round(amount / (v["total_ms"] / 1e3) / hbm_peak, 4)
        kernels[k] = rec
    out = {"grid": [nx, ny, nz], "bcs": ",".join(bcs), "h": list(h), "form": f"mixed-{prec}",
           "value": steps / dt, "unit": "solves/s", "ms_per_solve": 1e3 * dt / steps,
           "iters_per_solve": sum(i["iters"] for (_, i) in infos) / steps,
           "worst_rel_res_true": max(i["rel_res_true"] for (_, i) in infos),
           "failed": sum(1 for (st, _) in infos if st != 0), "tc_launches_per_apply": pl.precond_launches(),
           "kernels": kernels}
    pl.close()
    return out


def run_batched(prec, torch):
    """48 independent solves, grids {64..160}^2 x {32..96}, random BCs, 1-8 right-hand sides each."""
    import numpy as np

    from inputs import synth
    from paper_2501_03377_gb300 import Plan, binding

    specs = synth.batched_specs(seed=0)
    plans, etas, ups, streams = [], [], [], []
    for sp in specs:
        st = torch.cuda.Stream()
        streams.append(st)
        plans.append(Plan(sp["nx"], sp["ny"], sp["nz"], sp["bcs"], prec=prec, stream=st.cuda_stream))
        e = torch.from_numpy(np.stack([synth.batched_rhs(sp, r) for r in range(sp["nrhs"])])).cuda()
        etas.append(e)
        ups.append(torch.zeros_like(e))
    # the launch sequence of every plan chosen by the autotuner (timed once per grid; the choices of this
    # run are cached in a temporary file shared by plans of the same grid)
    import tempfile

    with tempfile.TemporaryDirectory() as td:
        cache = os.path.join(td, "tpcg_tune.txt")
        tunes = [pl.autotune(cache, applies=5) for pl in plans]
    # many small plans at once: the sweeps of each take fewer, fuller blocks so that the streams' kernels
    # share the SMs (the plan option's grain; 16 measured faster than the default 4 on this batch)
    grain = 16
    for pl in plans:
        pl.set_option(binding.TPCG_OPT_SWEEP_GRAIN, grain)
    torch.cuda.synchronize()
    chosen = {}
    for tu in tunes:
        k = f"slices={tu['slices']},fuse_g={tu['fuse_g']}"
        chosen[k] = chosen.get(k, 0) + 1
    args = ([p.handle for p in plans], [sp["nrhs"] for sp in specs], [e.data_ptr() for e in etas],
            [u.data_ptr() for u in ups], [1e-10] * len(specs), 60, binding.TPCG_ZERO_GUESS)
    binding.tpcg_solve_batched(*args)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, infos = binding.tpcg_solve_batched(*args)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    nrhs = sum(sp["nrhs"] for sp in specs)
    points = sum(sp["nrhs"] * sp["nx"] * sp["ny"] * sp["nz"] for sp in specs)
    return {"solves": len(specs), "rhs": nrhs, "form": f"mixed-{prec}", "sweep_grain": grain, "seconds": dt,
            "rhs_per_s": nrhs / dt,
            "mpoints_per_s": points / dt / 1e6, "status": st,
            "worst_rel_res_true": max(i["rel_res_true"] for i in infos),
            "mean_iters": float(np.mean([i["iters"] for i in infos])),
            "autotuned_sequences": chosen, "autotune_timed": sum(t["candidates"] for t in tunes)}


# DRAM bytes (read + write) per launch measured by ncu on the 256x256x128 workload, per mixed form (one
# capture per kernel; ncu flushes the caches before each launch).  Summaries and commands are under
# profiles/.  Remove an entry when its kernel changes.
NCU_TRAFFIC_PER_LAUNCH = {
    "fp16": {
        # tensor-core launches: mean over the three launches of one application (frontal-slice sequence): the
        # forward x-y pair (17.1 MB), the tube pair (16.9 MB) and the backward x-y pair (34.7 MB)
        "modeprod_tc": (17.1e6 + 16.9e6 + 34.7e6) / 3,
        "update": 275.0e6,  # the in-place update the instrumented (one-plan) pass runs
        "form_u": 248.0e6,  # the formation before a check (six recorded directions; TPCG_OPT_DEFER_U)
        "direction": 76.2e6,
        "true_residual": 197.8e6,  # a launch that checks (the others return at once)
    },
    "bf16x3": {
        # the five launches of one application (one per mode product, the z pair around G fused): 33.7-33.9 MB
        # read each (the hi and lo planes of the input), under 0.9 MB written (the outputs stay in L2 until the
        # next launch reads them)
        "modeprod_tc": 172.24e6 / 5,
    },
}


def kernel_work(kind, plan_prec, N, dims, iters_total, applies_total, solves, checks_total, launches=None):
    """Algorithmic work of one kernel kind over the timed region: (amount, unit, bound, launches that did
    the work).

    Bytes are the data each kernel must move once per grid point (halo re-reads and
    reduction scratch excluded); flops are the FP64 operations of the FP64 form."""
    n, q, t = dims
    mixed = plan_prec != "fp64"
    # bytes per point of a tensor-core operand (and of the copy of R): FP16/BF16 2, TF32 4, split BF16 pair 4
    lpb = {"fp16": 2, "bf16": 2, "tf32": 4, "bf16x3": 4}.get(plan_prec, 0)
    if kind == "modeprod_f64":
        return applies_total * 4.0 * N * (n + q + t + 0.25) / 1e12, "TFLOP", "alu", applies_total * (6 if t > 1 else 4)
    if kind == "modeprod_tc":
        # the per-point figure of the scope table for one application of the mixed preconditioner: about
        # 30 B (2560 flop / ~30 B at 256x256x128), whatever the launch sequence fuses
        npass = launches or (6 if t > 1 else 4)
        return applies_total * 30.0 * N / 1e9, "GB", "hbm", applies_total * npass
    if kind == "modeprod_tc_design":
        # the launch sequence's own algorithmic bytes per application (3D): every launch but the last reads +
        # writes one operand per point (lpb + lpb); the last reads its input (lpb) and the copy of R (lpb) and
        # writes Z in FP32 (4 B).  `launches` is the plan's count per application.  FP16/BF16: three with the
        # frontal-slice launches (16 B per point), four when the z products run as two launches (20 B), five or
        # six with one launch per mode product (24 or 28 B); 4-byte operands: TF32 six launches (52 B), split BF16
        # five with the z pair around G fused (44 B), six when the z axis exceeds 128 points
        npass = launches or (6 if t > 1 else 4)
        per_apply = ((npass - 1) * 2 * lpb + 2 * lpb + 4) * N
        return applies_total * per_apply / 1e9, "GB", "hbm", applies_total * npass
    if kind == "direction":
        if mixed:  # Z (FP32) + P_old (int32) in, P (int32) out
            return iters_total * 12.0 * N / 1e9, "GB", "hbm", iters_total
        # FP64 form: FP64 flops per point: P = (Z - m) + beta P_old (3), 7-point stencil (7), <W, P> (2)
        return iters_total * 12.0 * N / 1e12, "TFLOP", "alu", iters_total
    if kind == "update":
        # the instrumented plan updates U in place: mixed P (4) + R (8+8) + U (8+8) + tensor-core copy of R
        # (lpb); FP64 form: P and W (8+8) + R + U
        per = (4 + 16 + 16 + lpb) if mixed else (16 + 16 + 16)
        return iters_total * per * N / 1e9, "GB", "hbm", iters_total
    if kind == "form_u":
        # mixed forms, zero initial guess: once per check, the recorded directions (4 B each) in and U (8) out
        return (4.0 * iters_total + 8.0 * checks_total) * N / 1e9, "GB", "hbm", checks_total
    if kind == "true_residual":
        # eta (8) + U (8) in, R (8) + tensor-core copy (lpb, mixed) out
        return checks_total * (24 + lpb) * N / 1e9, "GB", "hbm", checks_total
    if kind == "eta_sum":
        return solves * 8.0 * N / 1e9, "GB", "hbm", solves
    if kind == "init_residual":  # zero initial guess: eta in, R (+ tensor-core copy) out
        return solves * (16 + lpb) * N / 1e9, "GB", "hbm", solves
    if kind == "center":
        return solves * 16.0 * N / 1e9, "GB", "hbm", solves
    return None, None, None, None


def run_cube(args, prec, torch, hbm_peak, peak_src):
    """The metric's 256^3 label: the 256x256x256 P/P/N cube (2000 defects), the mixed form on one plan and
    on `concurrency` plans (tpcg_solve_batched, TPCG_OPT_DEFER_U), the FP64 form on one plan, and the
    roofline of the tensor-core launches at this shape (CUDA events of an instrumented pass)."""
    from paper_2501_03377_gb300 import Plan
    from paper_2501_03377_gb300.binding import (TPCG_OPT_DEFER_U, TPCG_OPT_SWEEP_GRAIN, TPCG_ZERO_GUESS,
                                                tpcg_solve_batched)

    dev = torch.device("cuda", torch.cuda.current_device())
    ws = workload(256, [0, 1, 2, 3])
    w0 = ws[0]
    nx, ny, nz = w0["nx"], w0["ny"], w0["nz"]
    N = nx * ny * nz
    etas = [torch.from_numpy(w["eta"]).to(dev) for w in ws]
    ups = torch.zeros_like(etas[0])
    steps = max(4, min(args.steps, 12))
    nobar = lambda: None  # noqa: E731
    out = {"workload": w0["name"], "grid": [nx, ny, nz], "bcs": ",".join(w0["bcs"]), "tol": args.tol}
    pl = Plan(nx, ny, nz, w0["bcs"], prec=prec)
    for s in range(3):
        pl.solve(etas[s % 4], ups, tol=args.tol, maxit=60, zero_guess=True)
    dt, infos, _ = time_steps(pl, etas, ups, steps, args.tol, torch, nobar)
    out[f"mixed_{prec}"] = {"value": steps / dt, "unit": "solves/s", "ms_per_solve": 1e3 * dt / steps, "steps": steps,
                            "api": "tpcg_solve, one plan", "mpoints_per_s": steps * N / dt / 1e6,
                            "iters_per_solve": sum(i["iters"] for (_, i) in infos) / steps,
                            "worst_rel_res_true": max(i["rel_res_true"] for (_, i) in infos),
                            "failed": sum(1 for (st, _) in infos if st != 0),
                            "tc_launches_per_apply": pl.precond_launches()}
    # tensor-core roofline at this shape
    pl.profile_begin()
    _, pinfos, _ = time_steps(pl, etas, ups, steps, args.tol, torch, nobar)
    kst = pl.profile_end()
    applies = sum(i["precond_applies"] for (_, i) in pinfos)
    iters = sum(i["iters"] for (_, i) in pinfos)
    checks = sum(i.get("checks", 0) for (_, i) in pinfos)
    if "modeprod_tc" in kst:
        amount, unit, bound, worked = kernel_work("modeprod_tc", prec, N, (nx, ny, nz), iters, applies, steps, checks,
                                                  pl.precond_launches())
        secs = kst["modeprod_tc"]["total_ms"] / 1e3
        out["roofline_tc"] = {"kernel": "modeprod_tc", "bound": "hbm", "achieved": amount / secs, "peak": hbm_peak,
                              "unit": "GB/s", "frac": amount / secs / hbm_peak, "peak_source": f"{peak_src} hbm_gbs",
                              "us_per_apply": 1e6 * secs / max(1, applies),
                              "algorithmic_bytes_per_apply": amount * 1e9 / max(1, applies)}
    pl.close()
    # several plans on their own streams (the headline's launch configuration)
    conc = max(1, args.concurrency)
    cs = [torch.cuda.Stream() for _ in range(conc)]
    cps = [Plan(nx, ny, nz, w0["bcs"], prec=prec, stream=c.cuda_stream) for c in cs]
    if conc > 1:
        for cp in cps:
            cp.set_option(TPCG_OPT_DEFER_U, 1)
            if args.sweep_grain:
                cp.set_option(TPCG_OPT_SWEEP_GRAIN, args.sweep_grain)
    counts = [steps // conc + (1 if q < steps % conc else 0) for q in range(conc)]
    E = [torch.stack([etas[(sum(counts[:q]) + r) % 4] for r in range(max(1, counts[q]))]).contiguous()
         for q in range(conc)]
    Uc = [torch.zeros_like(e) for e in E]
    bat = lambda ns: tpcg_solve_batched([cp.handle for cp in cps], ns, [e.data_ptr() for e in E],  # noqa: E731
                                        [u.data_ptr() for u in Uc], [args.tol] * conc, 60, TPCG_ZERO_GUESS)
    bat([1] * conc)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    st_b, binfos = bat(counts)
    e1.record()
    torch.cuda.synchronize()
    dtb = e0.elapsed_time(e1) / 1e3
    out[f"mixed_{prec}_{conc}_plans"] = {"value": steps / dtb, "unit": "solves/s", "steps": steps, "status": st_b,
                                         "worst_rel_res_true": max(i["rel_res_true"] for i in binfos)}
    for cp in cps:
        cp.close()
    del E, Uc
    # the plain FP64 form
    p64 = Plan(nx, ny, nz, w0["bcs"], prec="fp64")
    p64.solve(etas[0], ups, tol=args.tol, maxit=60, zero_guess=True)
    k64 = 3
    dt64, inf64, _ = time_steps(p64, etas, ups, k64, args.tol, torch, nobar)
    out["fp64"] = {"value": k64 / dt64, "unit": "solves/s", "steps": k64,
                   "iters_per_solve": sum(i["iters"] for (_, i) in inf64) / k64,
                   "worst_rel_res_true": max(i["rel_res_true"] for (_, i) in inf64)}
    p64.close()
    out["mixed_over_fp64"] = out[f"mixed_{prec}"]["value"] / out["fp64"]["value"]
    return out


def max_over_ranks(x, world, torch, device):
    """Largest value of a per-rank float over all ranks (the whole-job clock is the slowest rank)."""
    if world <= 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, seconds):
    """Units all ranks processed per second of the slowest rank (weak scaling: `steps` per rank)."""
    return world * steps / seconds


def run_ours(args, rank, world, torch):
    from paper_2501_03377_gb300 import Plan
    from paper_2501_03377_gb300.binding import (TPCG_OPT_DEFER_U, TPCG_OPT_SWEEP_GRAIN, TPCG_ZERO_GUESS,
                                                tpcg_solve_batched)

    dev = torch.device("cuda", torch.cuda.current_device())
    prec = pick_prec(args)
    hbm_peak, bf16_peak, bf16_sus, peak_src = peaks()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    ws = workload(args.nz, [rank * 4 + i for i in range(4)])
    w0 = ws[0]
    nx, ny, nz = w0["nx"], w0["ny"], w0["nz"]
    N = nx * ny * nz
    etas = [torch.from_numpy(w["eta"]).to(dev) for w in ws]
    ups = torch.zeros_like(etas[0])
    plan = Plan(nx, ny, nz, w0["bcs"], prec=prec)

    # warm-up, then the timed regions (clean: no instrumentation)
    for s in range(args.warmup):
        plan.solve(etas[s % 4], ups, tol=args.tol, maxit=60, zero_guess=True)
    torch.cuda.synchronize()
    # one plan, solves one after the other (reported as single_plan)
    dt1, _, _ = time_steps(plan, etas, ups, args.steps, args.tol, torch, barrier)
    dt1 = max_over_ranks(dt1, world, torch, dev)
    single = {"value": whole_job_rate(world, args.steps, dt1), "unit": "solves/s", "ms_per_solve": 1e3 * dt1 / args.steps,
              "api": "tpcg_solve, one plan"}

    # the timed region: the steps through tpcg_solve_batched over `concurrency` plans, each on its own
    # stream (the library runs the queues of different plans concurrently); the right-hand sides are the
    # four seeded ones in rotation, each step its own 67 MB copy in HBM
    conc = max(1, args.concurrency)
    cstreams = [torch.cuda.Stream() for _ in range(conc)]
    cplans = [Plan(nx, ny, nz, w0["bcs"], prec=prec, stream=cs.cuda_stream) for cs in cstreams]
    if prec != "fp64" and conc > 1:  # several plans in flight: record U += alpha P and form U before each check
        for cp in cplans:
            cp.set_option(TPCG_OPT_DEFER_U, 1)
    if args.sweep_grain and conc > 1:  # several plans in flight: fuller blocks so that their kernels share SMs
        for cp in cplans:
            cp.set_option(TPCG_OPT_SWEEP_GRAIN, args.sweep_grain)
    counts = [args.steps // conc + (1 if q < args.steps % conc else 0) for q in range(conc)]
    firsts = [sum(counts[:q]) for q in range(conc)]
    E = [torch.stack([etas[(firsts[q] + r) % 4] for r in range(max(1, counts[q]))]).contiguous() for q in range(conc)]
    Uc = [torch.zeros_like(e) for e in E]

    def batched(ns):
        return tpcg_solve_batched([cp.handle for cp in cplans], ns, [e.data_ptr() for e in E],
                                  [u.data_ptr() for u in Uc], [args.tol] * conc, 60, TPCG_ZERO_GUESS)

    batched([1] * conc)  # warm-up: one solve per plan
    torch.cuda.synchronize()
    l0 = sum(cp.launch_count() for cp in cplans)
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    st_b, binfos = batched(counts)
    e1.record()
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3
    clocks = sampler.stop() if sampler else None
    barrier()
    launches = sum(cp.launch_count() for cp in cplans) - l0
    infos = [(i["status"], i) for i in binfos]
    bad = [i for (st, i) in infos if st != 0] + ([{"status": st_b}] if st_b != 0 else [])
    worst_res = max(i["rel_res_true"] for (_, i) in infos)
    iters_total = sum(i["iters"] for (_, i) in infos)
    applies_total = sum(i["precond_applies"] for (_, i) in infos)

    dt = max_over_ranks(dt, world, torch, dev)
    value = whole_job_rate(world, args.steps, dt)

    # instrumented pass (same steps): per-kernel device time with CUDA events on the plan's stream
    plan.profile_begin()
    _, pinfos, _ = time_steps(plan, etas, ups, args.steps, args.tol, torch, barrier)
    kstats = plan.profile_end()
    p_iters = sum(i["iters"] for (_, i) in pinfos)
    p_applies = sum(i["precond_applies"] for (_, i) in pinfos)
    total_k = sum(v["total_ms"] for v in kstats.values()) or 1.0
    kernels = {k: {"launches": v["launches"], "ms": round(v["total_ms"], 4),
                   "share": round(v["total_ms"] / total_k, 4)} for k, v in sorted(kstats.items(), key=lambda kv: -kv[1]["total_ms"])}
    p_checks = sum(i.get("checks", 0) for (_, i) in pinfos)
    dom = max(kstats, key=lambda k: kstats[k]["total_ms"])

    def roof(kind):
        amount, unit, bound, worked = kernel_work(kind, prec, N, (nx, ny, nz), p_iters, p_applies, args.steps,
                                                  p_checks, plan.precond_launches())
        if amount is None:
            return None
        secs = kstats[kind]["total_ms"] / 1e3
        achieved = amount / secs
        if unit == "TFLOP":
            peak = FP64_PEAK_TFLOPS if bound == "alu" else bf16_sus
            return {"kernel": kind, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None,
                    "peak_source": "derived FP64: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz" if bound == "alu"
                    else f"{peak_src} bf16 sustained"}
        traffic = NCU_TRAFFIC_PER_LAUNCH.get(prec, {}).get(kind) if nz == 128 else None
        return {"kernel": kind, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic,
                "traffic_unit": "DRAM bytes per launch (ncu, cold caches)" if traffic else None,
                "algorithmic_bytes_per_launch": amount * 1e9 / worked if worked else None,
                "peak_source": f"{peak_src} hbm_gbs"}

    roofline = roof(dom)
    if dom == "modeprod_tc" and roofline is not None:
        kstats["modeprod_tc_design"] = kstats["modeprod_tc"]
        rd = roof("modeprod_tc_design")
        del kstats["modeprod_tc_design"]
        roofline["model"] = "30 B per point per preconditioner application (scope-table figure)"
        roofline["design_model"] = {"bytes_per_point": rd["algorithmic_bytes_per_launch"] * plan.precond_launches() / N,
                                    "achieved": rd["achieved"], "frac": rd["frac"]}
    for k in kernels:
        r = roof(k)
        if r is not None:
            kernels[k]["achieved"] = round(r["achieved"], 2)
            kernels[k]["unit"] = r["unit"]
            kernels[k]["frac"] = round(r["frac"], 4)

    # end to end through the public API with host buffers (pinned): tpcg_solve_host_stream takes the
    # steps' right-hand sides from host memory and returns every solution to host memory, the copies in
    # and out of neighbouring solves overlapping the solves; all copies lie inside the timed region
    # the same plans as the timed region, one host thread each (the library calls release the interpreter)
    eh = [torch.from_numpy(w["eta"].copy()).pin_memory() for w in ws]
    uh = [[torch.zeros_like(eh[0]).pin_memory() for _ in range(2)] for _ in range(conc)]
    e2e_out = [None] * conc

    def host_stream(q, n, first):
        e2e_out[q] = cplans[q].solve_host_stream([eh[(first + r) % 4] for r in range(n)],
                                                 [uh[q][r % 2] for r in range(n)], tol=args.tol, maxit=60,
                                                 zero_guess=True)

    def host_streams(ns):
        ths = [threading.Thread(target=host_stream, args=(q, ns[q], firsts[q])) for q in range(conc) if ns[q] > 0]
        for t in ths:
            t.start()
        for t in ths:
            t.join()

    host_streams([1] * conc)  # warm-up
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2e_out = [None] * conc
    e0.record()
    host_streams(counts)
    e1.record()
    torch.cuda.synchronize()
    e2e_dt = e0.elapsed_time(e1) / 1e3
    e2e_dt = max_over_ranks(e2e_dt, world, torch, dev)
    e2e_infos = [i for r in e2e_out if r for i in r[1]]
    e2e = {"value": whole_job_rate(world, args.steps, e2e_dt), "unit": "solves/s", "h2d_bytes_per_step": 8 * N,
           "d2h_bytes_per_step": 8 * N, "api": f"tpcg_solve_host_stream on {conc} plans, one host thread each",
           "status": max((r[0] for r in e2e_out if r), default=0),
           "worst_rel_res_true": max(i["rel_res_true"] for i in e2e_infos)}

    # the other mixed forms, same workload and timing rules (one plan each), with the preconditioner's time
    # per application from an instrumented pass
    def form_record(fprec):
        pf = Plan(nx, ny, nz, w0["bcs"], prec=fprec)
        for s in range(args.warmup):
            pf.solve(etas[s % 4], ups, tol=args.tol, maxit=60, zero_guess=True)
        dtf, inff, _ = time_steps(pf, etas, ups, args.steps, args.tol, torch, barrier)
        dtf = max_over_ranks(dtf, world, torch, dev)
        pf.profile_begin()
        _, pinf, _ = time_steps(pf, etas, ups, min(args.steps, 6), args.tol, torch, barrier)
        kst = pf.profile_end()
        applies = sum(i["precond_applies"] for (_, i) in pinf)
        rec = {"value": whole_job_rate(world, args.steps, dtf), "unit": "solves/s", "steps": args.steps,
               "ms_per_solve": 1e3 * dtf / args.steps, "api": "tpcg_solve, one plan",
               "iters_per_solve": sum(i["iters"] for (_, i) in inff) / args.steps,
               "worst_rel_res_true": max(i["rel_res_true"] for (_, i) in inff),
               "failed": sum(1 for (st, _) in inff if st != 0),
               "tc_launches_per_apply": pf.precond_launches(),
               "precond_us_per_apply": 1e3 * kst["modeprod_tc"]["total_ms"] / max(1, applies)
               if "modeprod_tc" in kst else None}
        pf.close()
        return rec

    forms = {}
    if prec != "fp64" and not args.no_bf16_compare:
        for fprec in ("fp16", "bf16", "tf32", "bf16x3"):
            if fprec != prec:
                forms[f"{fprec}_form"] = form_record(fprec)

    # the plain FP64 form for comparison (fewer steps: it is ~100x slower)
    fp64_cmp = None
    if prec != "fp64" and not args.no_fp64_compare:
        p64 = Plan(nx, ny, nz, w0["bcs"], prec="fp64")
        for s in range(3):
            p64.solve(etas[s % 4], ups, tol=args.tol, maxit=60, zero_guess=True)
        k64 = max(3, min(args.steps, 6))
        dt64, inf64, _ = time_steps(p64, etas, ups, k64, args.tol, torch, barrier)
        dt64 = max_over_ranks(dt64, world, torch, dev)
        fp64_cmp = {"value": whole_job_rate(world, k64, dt64), "unit": "solves/s", "steps": k64,
                    "iters_per_solve": sum(i["iters"] for (_, i) in inf64) / k64,
                    "worst_rel_res_true": max(i["rel_res_true"] for (_, i) in inf64)}
        p64.close()

    serving = batched = comparators = efield = laplacian = variants = None
    if rank == 0 and world == 1 and prec != "fp64":
        if args.serving_requests > 0:
            serving = run_serving(args, prec, torch)
        if not args.no_batched:
            batched = run_batched(prec, torch)
        if not args.no_comparators:
            comparators = run_comparators(torch)
        efield = run_efield(plan, ups, torch)
        laplacian = run_laplacian(ups, torch, hbm_peak)
        if not args.no_variants:
            variants = run_variants(args, prec, torch, hbm_peak)
    cube = None
    if rank == 0 and world == 1 and prec != "fp64" and nz == 128 and not args.no_cube:
        cube = run_cube(args, prec, torch, hbm_peak, peak_src)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        k = max(1, args.cpu_solves)
        dtc, res = cpu_oracle_solves(ws[0], args.tol, k)
        one = cpu_one_thread(nz, args.tol, max(1, k // 5))
        cpu = {"value": k / dtc, "unit": "solves/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
               "sample": f"{k} full oracle solves of {w0['name']} (seed 0), operator and eigenbases built once "
                         f"outside the timing; {res.iters} PCG iteration(s) each; BLAS threads = all cores",
               "one_thread": None if one is None else {
                   "value": one[0], "unit": "solves/s", "cores": 1,
                   "sample": f"{one[1]} oracle solves in a child process with BLAS/OpenMP limited to 1 thread"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else f"f64+{prec}(tensor)", "data": "synthetic",
            "config": {"workload": w0["name"], "grid": [nx, ny, nz], "bcs": ",".join(w0["bcs"]), "tol": args.tol,
                       "form": "fp64" if prec == "fp64" else f"mixed-{prec}",
                       "rhs": "2000 Gaussian defects sigma~U(1,4) cells, charges +-1, ||eta||=1/N",
                       "l2": "every step its own 67 MB right-hand side (4 seeded ones in rotation) + ~0.3 GB "
                             "workspace per plan > 129 MB L2",
                       "parallelism": f"replicas x{world}",
                       "concurrency": f"{conc} plans on {conc} streams (tpcg_solve_batched)"
                                      + (", TPCG_OPT_DEFER_U" if prec != "fp64" and conc > 1 else "")
                                      + (f", TPCG_OPT_SWEEP_GRAIN {args.sweep_grain}"
                                         if args.sweep_grain and conc > 1 else "")},
            "mpoints_per_s": value * N / 1e6,
            "iters_per_solve": iters_total / args.steps, "precond_applies_per_solve": applies_total / args.steps,
            "worst_rel_res_true": worst_res, "failed_solves": len(bad),
            "gpu_launches": launches, "single_plan": single,
            "roofline": roofline, "kernels": kernels,
            "e2e": e2e, "cpu_baseline": cpu, "fp64_form": fp64_cmp, **forms,
            "serving": serving, "batched": batched, "comparators": comparators, "efield": efield,
            "laplacian_fp64": laplacian, "variants": variants,
            "cube_256": cube, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    plan.close()


def main():
    args = parse()
    if args.oracle_sample:
        oracle_sample(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2501_03377_gb300 import build

    build.build()
    run_ours(args, rank, world, torch)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
