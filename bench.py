#!/usr/bin/env python
"""PASD ADMM iterations/s on the 200x200x200 workload, one JSON line.

Workload: a planted 200^3 tensor (Tucker core 10^3 with N(0,1) entries,
orthonormal Gaussian-QR factors, 20% of the entries corrupted by
U[-1,1] * max|L0|), rank bounds R_n = 20, lambda = 1/200, alpha_n = 1/3, run to
relative residual 1e-6 (max_n ||T - Z_n - E||_F / ||T||_F). Synthetic, seeded.

A step is one whole solve of that workload through pasd_solve with the inputs
resident in HBM (initialisation, every ADMM loop body until the stop rule, the
output pass), so every timed step holds the idle, active and converging loop
bodies of the trajectory; the metric counts loop bodies per second. The tensors
the loop streams (T, E, G_1..G_3: 160 MB) exceed the 129 MB L2, so no L2 flush is
added between steps.

Extra keys: roofline of the dominant kernel (algorithmic bytes of the fused
elementwise pass, the bandwidth floor's (2N + 2) 4 D + 4 sum_n R_n P_n, over its
CUDA-event durations, every launch of one solve, with the idle and active bodies
also reported apart; impl_frac counts the bytes this design's pass moves
instead, one more read of E and only the kept rows of Vrot), clocks sampled during the timed
region, e2e (whole solves through pasd_solve_host with pinned host buffers),
cpu_baseline (the FP64 oracle on the host cores, a bounded sample), table1 (the
paper's Table 1 workloads, 100^3 and 50^4, with the paper's own PASD results as
context), video (whole solves on the 144x176x3x300 colour-video shape, FP32 and
mixed), batched (64 uneven tensors, 8 of them hyperspectral-shaped, submitted at
once) and serving (a Poisson trace of distinct requests through pasd_submit /
pasd_poll: solves/s and p50 / p99 latency, against the same requests solved one
at a time); the shorter summaries come last on the line. Opt-in: --sweep (solve
time against cube size) and --phase (the phase-transition map of the paper's
Fig. 1 setting).

--impl reference times the FP64 oracle (the method as the paper defines it),
each step one loop body on the same 200^3 workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PASD iters/s @200^3"
UNIT = "iters/s"
DIMS = (200, 200, 200)
RANKS = (20, 20, 20)
ALPHA = (1 / 3, 1 / 3, 1 / 3)
LAMBDA = 1 / 200
TOL = 1e-6
CONFIG = {"workload": "planted Tucker(10,10,10) + 20% sparse U[-1,1]*max|L0|, 200x200x200 float32, "
                      "R_n=20, lambda=1/200, alpha_n=1/3, run to relative residual 1e-6 (seed 1)",
          "dims": list(DIMS), "rank_bounds": list(RANKS), "stop": "fro_rel 1e-6",
          "l2": "working set 160 MB > 129 MB L2, no flush"}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


FUSED_SOURCES = ("fused_tma.cu", "fused.cu", "tma.cuh")   # the kernel, its tile planner, its copy wrappers


def _fused_src_hash():
    h = hashlib.sha256()
    for f in FUSED_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1712_09999_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def _fused_traffic():
    """DRAM bytes of one fused-pass launch in an idle body and in an active body,
    from the committed ncu summary, if the kernel sources still match the ones
    that were profiled; else (None, None)."""
    p = os.path.join(ROOT, "profiles", "fused_pass_200cube_traffic.json")
    if not os.path.exists(p):
        return None, None
    d = json.load(open(p))
    if _fused_src_hash() != d.get("fused_src_sha256"):
        return None, None
    return d.get("traffic_bytes_idle_launch"), d.get("traffic_bytes_active_launch")


class ClockSampler:
    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.06)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_iters_per_s(T, seconds: float):
    """The FP64 oracle on the host cores: loop bodies of the same workload."""
    import numpy as np
    from oracle import pasd_oracle as O
    p = O.Params.from_alpha_lambda(RANKS, ALPHA, LAMBDA, stop="fixed", max_iter=10 ** 6)
    t64 = T.astype(np.float64)
    st = O.init_state(t64, p.ranks, p.mu0)
    O.step(t64, st, p)                       # first body (untimed warm-up)
    n = 0
    t0 = time.perf_counter()
    while True:
        O.step(t64, st, p)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            return n / el, n, el


ONE_CORE_ENV = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                                  "BLIS_NUM_THREADS", "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS")}


def _oracle_one_core(seconds: float):
    """The same oracle timing with every BLAS/OpenMP pool limited to one thread. The
    limits must be set before numpy loads its BLAS, so this runs in a child process
    (this script with --oracle-one-core); returns (bodies/s, bodies, seconds) or None."""
    env = dict(os.environ, **ONE_CORE_ENV)
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-one-core", str(seconds)],
                           env=env, capture_output=True, text=True, timeout=seconds + 300)
        out = json.loads(r.stdout.strip().splitlines()[-1])
        return out["value"], out["bodies"], out["seconds"]
    except Exception:
        return None


def run_oracle_one_core(seconds: float):
    from paper_1712_09999_gb300 import synth
    v, n, el = _oracle_iters_per_s(synth.cube_200(1).T, seconds)
    print(json.dumps({"value": v, "bodies": n, "seconds": el}), flush=True)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    from paper_1712_09999_gb300 import synth
    from oracle import pasd_oracle as O
    pr = synth.cube_200(1)
    t64 = pr.T.astype(np.float64)
    p = O.Params.from_alpha_lambda(RANKS, ALPHA, LAMBDA, stop="fixed", max_iter=10 ** 6)
    st = O.init_state(t64, p.ranks, p.mu0)
    tw = time.perf_counter()
    for _ in range(args.warmup):
        O.step(t64, st, p)
    per = (time.perf_counter() - tw) / max(1, args.warmup)
    # each step is a full FP64 loop body on the host: bound the timed run to ~2 minutes
    steps = max(1, min(args.steps, int(120.0 / max(per, 1e-9))))
    t0 = time.perf_counter()
    for _ in range(steps):
        O.step(t64, st, p)
    el = time.perf_counter() - t0
    v = steps / el
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "steps_requested": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * el / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": dict(CONFIG, step="one FP64 loop body on the host cores (a bounded sample of the "
                                        "181-body solve, whose bodies/s the metric counts)"),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{steps} FP64 loop bodies of the 200^3 workload "
                                       f"after {args.warmup} warm-up bodies"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


def _serving(P, torch, ctx, args):
    """Continuous-batching service on a Poisson trace of distinct requests: every
    request is its own planted cube (side log-uniform on 32-256, Tucker ranks
    3-20, R = floor(1.2 r), 5-30% corruption U[-1,1] max|L0|) with its own
    precision (FP32 or mixed, Bernoulli(1/2)), served through pasd_submit /
    pasd_poll with the idle-start skip. Plans are made per request before the
    trace (a service keeps its plans; plan set-up is not in the latency). The same
    requests solved one at a time are the baselines: the plain FP32 path, and the
    FP32 path with the skip (the served flags)."""
    import numpy as np
    from paper_1712_09999_gb300 import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    n_req = int(args.serve_rate * args.serve_seconds)
    specs = synth.serving_mix(n_req, seed=4)
    precs = synth.request_precisions(n_req, seed=7)
    tg = time.perf_counter()
    Ts = [synth.planted_device(sp.dims, sp.tucker, sp.rho, sp.seed, dev, scale="max")[0] for sp in specs]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - tg

    def timed_solve(plan, q, L, E):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        r = P.pasd_solve(plan, Ts[q], L, E)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    def serial(flags, precision_of):
        ms_all, iters, plans = [], [], []
        for q, sp in enumerate(specs):
            plan, _ = P.pasd_plan(ctx, P.make_params(sp.dims, sp.rank_bounds, max_iter=1000,
                                                     precision=precision_of(q), flags=flags))
            L = torch.empty_like(Ts[q])
            E = torch.empty_like(Ts[q])
            P.pasd_solve(plan, Ts[q], L, E)              # allocation, graph capture, warm-up
            ms, r = timed_solve(plan, q, L, E)
            ms_all.append(ms)
            iters.append(int(r.iters))
            plans.append((plan, L, E))
        return ms_all, iters, plans

    plain_ms, plain_iters, plain_plans = serial(0, lambda q: P.PREC_FP32)
    for plan, _, _ in plain_plans:
        P.pasd_plan_destroy(plan)
    skip_ms, _, _tmp = serial(P.F_SKIP_IDLE, lambda q: P.PREC_FP32)
    for plan, _, _ in _tmp:
        P.pasd_plan_destroy(plan)
    # served plans: per-request precision, the skip; warmed by one solve each
    _, _, slots = serial(P.F_SKIP_IDLE, lambda q: P.PREC_MIXED if precs[q] else P.PREC_FP32)

    def run(rate, n):
        arr = synth.poisson_arrivals(rate, n, seed=5)
        pending = {}
        lat, finish, bad = [], [], 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        i = 0
        while i < n or pending:
            now = time.perf_counter() - t0
            while i < n and arr[i] <= now:
                plan, L, E = slots[i]
                pending[P.pasd_submit(ctx, plan, Ts[i], L, E)] = float(arr[i])
                i += 1
            for tk in list(pending):
                st, _ = P.pasd_poll(ctx, tk)
                if st != P.PENDING:
                    f = time.perf_counter() - t0
                    lat.append(f - pending.pop(tk))
                    finish.append(f)
                    bad += st not in (P.OK, P.NOT_CONVERGED)
            time.sleep(0.0002)
        span = max(finish) - float(arr[0])
        return {"rate": rate, "n": n, "solves_per_s": round(n / span, 1),
                "p50_ms": round(1000 * _percentile(lat, 50), 1), "p99_ms": round(1000 * _percentile(lat, 99), 1),
                "failed": bad}

    over = run(args.serve_rate, n_req)
    low_n = max(1, int(args.serve_low_rate * args.serve_seconds))
    low = run(args.serve_low_rate, low_n)
    for plan, _, _ in slots:
        P.pasd_plan_destroy(plan)
    serial_plain = n_req / (sum(plain_ms) / 1000.0)
    serial_skip = n_req / (sum(skip_ms) / 1000.0)
    return {"trace": f"{n_req} distinct requests, Poisson {args.serve_rate:g}/s for {args.serve_seconds:g} s "
                     f"(reduced from 60 s), cubes 32-256 log-uniform, Tucker 3-20, R=floor(1.2r), 5-30% "
                     f"corruption, {int(precs.sum())} mixed / {n_req - int(precs.sum())} FP32, idle-start skip",
            "served": over, "below_capacity": low,
            "serial_plain_fp32_solves_per_s": round(serial_plain, 1),
            "serial_fp32_skip_solves_per_s": round(serial_skip, 1),
            "served_over_serial_plain": round(over["solves_per_s"] / serial_plain, 2),
            "iters_mean": round(float(np.mean(plain_iters)), 1), "generation_s": round(gen_s, 1)}


def _batched(P, torch, ctx, args):
    """The batched workload: 56 planted tensors with uneven sides (32-160 per mode)
    and 8 hyperspectral-shaped 128x128x191 cubes, all 64 submitted at once through
    pasd_submit (one stream per solve, overlapping on the GPU; one captured graph
    per loop body), with the FP32 path and with mixed precision (both with the
    idle-start skip), against the same solves run one at a time with the plain
    FP32 path and with the FP32 path plus the skip (the batched flags). Recovery
    error is against the planted low-rank part."""
    import numpy as np
    from paper_1712_09999_gb300 import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    specs = synth.batch_mix(seed=3)
    tg = time.perf_counter()
    probs = [synth.serving_problem(sp) for sp in specs]
    gen_s = time.perf_counter() - tg
    Ts = [torch.from_numpy(pr.T).to(dev) for pr in probs]
    L0s = [torch.from_numpy(pr.L0).to(dev) for pr in probs]

    def serial(flags):
        ms_all = []
        for q, sp in enumerate(specs):
            plan, _ = P.pasd_plan(ctx, P.make_params(sp.dims, sp.rank_bounds, max_iter=1000, flags=flags))
            L = torch.empty_like(Ts[q])
            E = torch.empty_like(Ts[q])
            P.pasd_solve(plan, Ts[q], L, E)              # allocation, graph capture, warm-up
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            P.pasd_solve(plan, Ts[q], L, E)
            e1.record()
            torch.cuda.synchronize()
            ms_all.append(e0.elapsed_time(e1))
            P.pasd_plan_destroy(plan)
        return len(specs) / (sum(ms_all) / 1000.0)

    serial_plain = serial(0)
    serial_skip = serial(P.F_SKIP_IDLE)

    def batch(precision, cx):
        plans, Ls, Es = [], [], []
        for q, sp in enumerate(specs):
            plan, _ = P.pasd_plan(cx, P.make_params(sp.dims, sp.rank_bounds, max_iter=1000,
                                                    precision=precision, flags=P.F_SKIP_IDLE))
            L = torch.empty_like(Ts[q])
            E = torch.empty_like(Ts[q])
            P.pasd_solve(plan, Ts[q], L, E)          # allocation, graph capture, warm-up
            plans.append(plan)
            Ls.append(L)
            Es.append(E)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pending = {P.pasd_submit(cx, plans[q], Ts[q], Ls[q], Es[q]): q for q in range(len(specs))}
        bad, iters, skipped, batched = 0, [0] * len(specs), [0] * len(specs), 0
        while pending:
            for tk in list(pending):
                st, r = P.pasd_poll(cx, tk)
                if st != P.PENDING:
                    q = pending.pop(tk)
                    bad += st not in (P.OK, P.NOT_CONVERGED)
                    iters[q], skipped[q] = int(r.iters), int(r.skipped)
                    batched += int(r.batched)
            time.sleep(0.0002)
        wall = time.perf_counter() - t0
        rse = [float(torch.linalg.vector_norm(Ls[q].double() - L0s[q]) / torch.linalg.vector_norm(L0s[q]))
               for q in range(len(specs))]
        for plan in plans:
            P.pasd_plan_destroy(plan)
        return {"solves_per_s": round(len(specs) / wall, 1), "failed": bad, "in_batched_executor": batched,
                "rse_median": float(np.median(rse)), "iters": sum(iters), "skipped": sum(skipped)}, Ls

    fp32, l32 = batch(P.PREC_FP32, ctx)
    mixed, lmx = batch(P.PREC_MIXED, ctx)
    # the same FP32 solves with every solve on a stream of its own (no batched executor)
    os.environ["PASD_NO_BATCH"] = "1"
    ctx_streams = P.pasd_ctx_create(torch.cuda.current_device())
    del os.environ["PASD_NO_BATCH"]
    fp32_streams, _ = batch(P.PREC_FP32, ctx_streams)
    P.pasd_ctx_destroy(ctx_streams)
    mixed["L_rel_vs_fp32_max"] = max(float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
                                     for a, b in zip(lmx, l32))
    return {"workload": "64 solves at once: 56 planted (sides U{32..160}, Tucker 3-15, 5-30%) + 8 hyperspectral "
                        "128x128x191 (salt and pepper), seed 3, idle-start skip",
            "fp32": fp32, "fp32_own_streams": fp32_streams, "mixed": mixed,
            "serial_plain_fp32_solves_per_s": round(serial_plain, 1),
            "serial_fp32_skip_solves_per_s": round(serial_skip, 1),
            "generation_s": round(gen_s, 1)}


# PASD's own results in the paper's Table 1 (RSE, seconds per solve; Matlab 8.1 on an
# Intel Xeon E5-2620 at 2.0 GHz, averages over its own random tensors): context only.
PAPER_TABLE1 = {("100^3", 0.05): (1.12e-7, 54.89), ("100^3", 0.10): (1.28e-7, 55.95),
                ("100^3", 0.20): (1.44e-7, 57.65), ("50^4", 0.05): (2.99e-3, 469.46),
                ("50^4", 0.10): (8.33e-3, 483.37), ("50^4", 0.20): (4.27e-2, 544.28)}


def _table1(P, torch, ctx, args):
    """The paper's Table 1 workloads: 100^3 and 50^4, Tucker rank 10, R_n = 12,
    U[-1,1] additive corruption on 5/10/20% of entries, paper-default lambda_n,
    Algorithm 1's stop test with eps = 1e-5, at most 1000 bodies; one solve each
    (plain FP32 path), time per solve by CUDA events, recovery error."""
    from paper_1712_09999_gb300 import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    rows = []
    for name, dims in (("100^3", (100,) * 3), ("50^4", (50,) * 4)):
        for rho in (0.05, 0.10, 0.20):
            pr = synth.table1(dims, rho, seed=7)
            T = torch.from_numpy(pr.T).to(dev)
            L0 = torch.from_numpy(pr.L0).to(dev)
            plan, _ = P.pasd_plan(ctx, P.make_params(dims, (12,) * len(dims), tol=1e-5, max_iter=1000))
            L = torch.empty_like(T)
            E = torch.empty_like(T)
            P.pasd_solve(plan, T, L, E)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            r = P.pasd_solve(plan, T, L, E)
            e1.record()
            torch.cuda.synchronize()
            P.pasd_plan_destroy(plan)
            rse = float(torch.linalg.vector_norm(L.double() - L0) / torch.linalg.vector_norm(L0))
            prse, psec = PAPER_TABLE1[(name, rho)]
            rows.append([name, rho, int(r.iters), int(r.status), round(e0.elapsed_time(e1), 2),
                         float("%.3g" % rse), prse, psec])
    return {"workload": "Table 1 family: Tucker rank 10, R_n = 12, U[-1,1] additive corruption, paper lambda_n, "
                        "eps = 1e-5 (seed 7); paper: Matlab 8.1, Xeon E5-2620 2.0 GHz (context only)",
            "columns": ["size", "rho", "iters", "status", "ms_per_solve", "rse", "paper_rse", "paper_s_per_solve"],
            "rows": rows}


def _sweep(P, torch, ctx, args):
    """Solve time against cube size (Tucker rank 10, R_n = 12, 10% U[-1,1]
    corruption, paper-default lambda_n, eps = 1e-5), inputs generated on the GPU."""
    from paper_1712_09999_gb300 import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    rows = []
    for side in args.sweep_sides:
        T, L0 = synth.planted_device((side,) * 3, (10,) * 3, 0.10, 11, dev)
        plan, footprint = P.pasd_plan(ctx, P.make_params(T.shape, (12,) * 3, tol=1e-5, max_iter=1000))
        L = torch.empty_like(T)
        E = torch.empty_like(T)
        P.pasd_solve(plan, T, L, E)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        r = P.pasd_solve(plan, T, L, E)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        P.pasd_plan_destroy(plan)
        rse = float(torch.linalg.vector_norm(L.double() - L0.double()) / torch.linalg.vector_norm(L0.double()))
        rows.append({"side": side, "iters": int(r.iters), "ms_per_solve": round(ms, 2),
                     "us_per_body": round(1000 * ms / max(1, r.iters), 1), "rse": rse,
                     "footprint_gb": round(footprint / 1e9, 2)})
        del T, L0, L, E
        torch.cuda.empty_cache()
    return {"workload": "cubes, Tucker rank 10, R_n = 12, 10% U[-1,1] corruption, paper lambda_n, eps = 1e-5, "
                        "generated on the GPU (seed 11)", "rows": rows}


def _phase(P, torch, ctx, args, ranks=None, rhos=None, trials=None):
    """Phase-transition map on 100^3 (the paper's Fig. 1 setting with this
    repository's random streams): Tucker rank r = 2..50 step 2 (R_n = floor(1.2 r)),
    corruption fraction 2..50% step 2 (U[-1,1] additive), `phase_trials` trials per
    cell, success when the recovery error is at most 1e-3. Solves run through
    pasd_submit, `phase_slots` at a time per rank, with the idle-start skip. The
    default run maps a coarser grid (`ranks`, `rhos`, `trials` given)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_1712_09999_gb300 import synth
    ranks = ranks or list(range(2, 51, 2))
    rhos = rhos or [k / 100 for k in range(2, 51, 2)]
    trials = trials or args.phase_trials
    grid = []
    t0 = time.perf_counter()
    n_solves = 0
    for r in ranks:
        R = int(1.2 * r)
        slots = []
        for _ in range(min(args.phase_slots, len(rhos) * trials)):
            plan, _ = P.pasd_plan(ctx, P.make_params((100,) * 3, (R,) * 3, tol=1e-5, max_iter=1000,
                                                     flags=P.F_SKIP_IDLE))
            slots.append((plan, torch.empty((100,) * 3, device=dev), torch.empty((100,) * 3, device=dev)))
        jobs = [(rho, tr) for rho in rhos for tr in range(trials)]
        ok = {rho: 0 for rho in rhos}
        free = list(range(len(slots)))
        pending = {}
        k = 0
        while k < len(jobs) or pending:
            while free and k < len(jobs):
                rho, tr = jobs[k]
                T, L0 = synth.planted_device((100,) * 3, (r,) * 3, rho, 100000 + 1000 * r + 10 * int(rho * 100) + tr, dev)
                torch.cuda.current_stream().synchronize()   # the solve's own stream reads T
                sl = free.pop()
                plan, L, E = slots[sl]
                pending[P.pasd_submit(ctx, plan, T, L, E)] = (sl, rho, T, L0)
                k += 1
            for tk in list(pending):
                st, _ = P.pasd_poll(ctx, tk)
                if st != P.PENDING:
                    sl, rho, T, L0 = pending.pop(tk)
                    L = slots[sl][1]
                    rse = float(torch.linalg.vector_norm(L.double() - L0.double()) / torch.linalg.vector_norm(L0.double()))
                    ok[rho] += int(st in (P.OK, P.NOT_CONVERGED) and rse <= 1e-3)
                    free.append(sl)
                    n_solves += 1
            time.sleep(0.0001)
        for plan, _, _ in slots:
            P.pasd_plan_destroy(plan)
        grid.append([ok[rho] / trials for rho in rhos])
    return {"workload": f"100^3, Tucker rank r in {ranks} (R = floor(1.2 r)), corruption {rhos}, "
                        f"{trials} trials per cell, success: RSE <= 1e-3", "ranks": ranks,
            "rhos": rhos, "success": grid, "solves": n_solves, "seconds": round(time.perf_counter() - t0, 1)}


def _video(P, torch, ctx, args):
    """Loop bodies per second on the colour-video shape 144x176x3x300, R = (20, 20, 3, 5),
    the paper's default lambda_n, over one whole solve to Algorithm 1's stop rule
    (eps = 1e-5), FP32 and mixed precision; per-kernel milliseconds per body from
    CUDA events over the same trajectory."""
    import numpy as np
    from paper_1712_09999_gb300 import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    pr = synth.video()
    T = torch.from_numpy(pr.T).to(dev)
    stream = torch.cuda.current_stream()
    out = {"workload": "video 144x176x3x300 (rank-1 background, 16 moving rectangles, 5% voxels, seed 2), "
                       "R=(20,20,3,5), paper lambda_n, whole solve to eps=1e-5"}
    for name, prec in (("fp32", P.PREC_FP32), ("mixed", P.PREC_MIXED)):
        plan, footprint = P.pasd_plan(ctx, P.make_params(pr.T.shape, (20, 20, 3, 5), max_iter=1000, precision=prec))
        L = torch.empty_like(T)
        E = torch.empty_like(T)
        P.pasd_solve(plan, T, L, E, stream)          # allocation, graph capture, warm-up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = P.pasd_solve(plan, T, L, E, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        rse = float(torch.linalg.vector_norm(L.double() - torch.from_numpy(pr.L0).to(dev)) /
                    float(np.linalg.norm(pr.L0)))
        P.pasd_begin(plan, T, stream)
        per = P.pasd_profile_iterations(plan, int(r.iters), stream)
        info = P.pasd_plan_info(plan)
        P.pasd_plan_destroy(plan)
        out[name] = {"iters_per_s": round(r.iters / (ms / 1000.0), 1), "iters": int(r.iters),
                     "ms_per_solve": round(ms, 2), "rse": rse, "kept": list(r.kept)[:4],
                     "kernel_us_per_body": {k: round(1000 * v / r.iters, 1) for k, v in per.items()},
                     "plan": {k: info[k] for k in ("autotune", "apass_cols_per_thread", "apass_row_groups")}}
        out["footprint_bytes"] = footprint
    return out


def _job_time_and_value(ms: float, steps: int, world: int, dist, device):
    """The job's timed region is the slowest rank's (max over ranks of `ms`);
    the throughput counts the steps of every rank (one replica per rank, no
    data-path collective). With dist None the rank is alone."""
    if dist is not None:
        import torch
        t = torch.tensor([float(ms)], device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * steps / (ms / 1000.0)


def _bodies_launched(k: int, chunk: int, max_iter: int) -> int:
    """Loop bodies pasd_solve enqueues for a solve that stops after k bodies: it
    launches `chunk` bodies, then keeps one chunk in flight while it reads the
    device stop flag of the previous one, so it sees the flag of body k only
    after launching the chunk that follows; bodies past the stop return at once."""
    launched = min(chunk, max_iter)
    while True:
        seen = launched
        if launched < max_iter:
            launched += min(chunk, max_iter - launched)
        if seen >= k or launched >= max_iter:
            return launched


def run_ours(args):
    import numpy as np
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import __graft_entry__ as ge
    ge.build()
    from paper_1712_09999_gb300 import pasd as P
    from paper_1712_09999_gb300 import synth

    pr = synth.cube_200(1)
    T_host = torch.from_numpy(pr.T).pin_memory()
    T = T_host.to(dev)
    ctx = P.pasd_ctx_create(torch.cuda.current_device())
    stream = torch.cuda.current_stream()

    # A step is one whole solve of the workload (pasd_solve on device buffers:
    # initialisation, every loop body until the stop rule, the output pass), so
    # the timed region holds the idle, active and converging bodies of each
    # trajectory; the metric counts loop bodies.
    sp = P.make_params(DIMS, RANKS, alpha=ALPHA, lam=LAMBDA, stop=P.STOP_FRO_REL, tol=TOL, max_iter=1000)
    plan, footprint = P.pasd_plan(ctx, sp)
    L = torch.empty_like(T)
    E = torch.empty_like(T)
    r = P.pasd_solve(plan, T, L, E, stream)          # allocation, graph capture
    k_conv = int(r.iters)
    for _ in range(args.warmup):
        P.pasd_solve(plan, T, L, E, stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    time.sleep(0.15)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    iters = 0
    for _ in range(args.steps):
        iters += int(P.pasd_solve(plan, T, L, E, stream).iters)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    assert iters == args.steps * k_conv
    ms, value = _job_time_and_value(ev0.elapsed_time(ev1), iters, world, dist, dev)
    lpi = P.pasd_launches_per_iter(plan)
    launches_per_solve = 3 + _bodies_launched(k_conv, 8, 1000) * lpi + 1

    # dominant kernel: per-kernel CUDA-event durations for every body of one solve,
    # the trajectory each timed step runs (idle and active bodies alike)
    P.pasd_begin(plan, T, stream)
    per_body = [P.pasd_profile_iterations(plan, 1, stream) for _ in range(k_conv)]
    D = int(np.prod(DIMS))
    N = len(DIMS)
    tr = np.zeros((k_conv, P.TRACE_STRIDE))
    P.pasd_state_get(plan, P.STATE_TRACE, 0, tr)
    kept = tr[:, 5:5 + N]
    # algorithmic bytes of one fused pass, the bandwidth floor's second phase: read T
    # and Y_1..Y_N, write E and Y_1..Y_N, read the rank-R_n refold operands once:
    # (2N + 2) 4 D + 4 sum_n R_n P_n, the same for every body
    alg = np.full(k_conv, (2 * N + 2) * 4.0 * D + 4.0 * sum(R * (D // I) for R, I in zip(RANKS, DIMS)))
    # bytes this design's pass moves: also the previous E (the multiplier update reads
    # it, the multipliers being stored as G_n) and only the kept rows of each Vrot_n
    impl = np.array([(2 * N + 3) * 4 * D + 4 * sum(float(s) * (D // I) for s, I in zip(kept[b], DIMS))
                     for b in range(k_conv)])
    fused = np.array([pb["fused"] for pb in per_body]) / 1000.0        # seconds per launch
    active = kept.sum(axis=1) > 0
    peak, peak_kind = _peaks()

    def phase(mask):
        return {"bodies": int(mask.sum()), "launch_us": round(float(fused[mask].mean() * 1e6), 1),
                "frac": round(float(alg[mask].sum() / fused[mask].sum() / 1e9 / peak), 3)}

    achieved = float(alg.sum() / fused.sum() / 1e9)
    impl_achieved = float(impl.sum() / fused.sum() / 1e9)
    tr_idle, tr_active = _fused_traffic()
    traffic = None
    if tr_idle is not None and tr_active is not None:
        traffic = (tr_idle * int((~active).sum()) + tr_active * int(active.sum())) / k_conv
    roofline = {"bound": "hbm", "kernel": "fused elementwise pass",
                "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "peak_kind": peak_kind, "traffic": traffic, "alg_bytes_per_launch": float(alg.mean()),
                "impl_bytes_per_launch": float(impl.mean()), "impl_frac": round(impl_achieved / peak, 4),
                "launch_ms": float(fused.mean() * 1000),
                "averaged_over": f"every launch of one {k_conv}-body solve",
                "phases": {"idle": phase(~active), "active": phase(active)},
                "kernel_us_per_body": {k: round(1000 * float(np.mean([pb[k] for pb in per_body])), 1)
                                       for k in per_body[0]}}

    # e2e: whole solves through the public host-buffer entry point, pinned host buffers
    Lh = torch.empty(DIMS, dtype=torch.float32).pin_memory()
    Eh = torch.empty(DIMS, dtype=torch.float32).pin_memory()
    P.pasd_solve_host(plan, T_host, Lh, Eh, stream)       # staging allocation
    it_sum, t_sum = 0, 0.0
    for _ in range(max(1, args.e2e_solves)):
        t0 = time.perf_counter()
        rr = P.pasd_solve_host(plan, T_host, Lh, Eh, stream)
        t_sum += time.perf_counter() - t0
        it_sum += rr.iters
    e2e_v = world * it_sum / t_sum
    e2e = {"value": round(e2e_v, 1), "unit": UNIT, "h2d_bytes_per_step": 4 * D, "d2h_bytes_per_step": 8 * D,
           "note": f"whole solves via pasd_solve_host from pinned host memory: a step is one solve "
                   f"({k_conv} bodies) with one T upload and one L, E download"}

    line = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(CONFIG, step=f"one whole solve ({k_conv} loop bodies)",
                           ms_per_body=round(ms / iters, 4),
                           parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                           footprint_bytes=footprint),
            "gpu_launches": args.steps * launches_per_solve, "clocks": clocks, "roofline": roofline, "e2e": e2e,
            "plan": P.pasd_plan_info(plan)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, n, el = _oracle_iters_per_s(pr.T, args.cpu_seconds)
        line["cpu_baseline"] = {"value": round(v, 3), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"{n} FP64 loop bodies of the 200^3 workload in {el:.1f} s "
                                          "(numpy/LAPACK, BLAS threads = all cores)"}
        one = _oracle_one_core(args.cpu_seconds)
        if one is not None:
            line["cpu_baseline"]["single_core"] = {
                "value": round(one[0], 3), "unit": UNIT, "cores": 1,
                "sample": f"{one[1]} FP64 loop bodies in {one[2]:.1f} s, one BLAS/OpenMP thread"}
    if rank == 0 and not args.no_table1:
        line["table1"] = _table1(P, torch, ctx, args)
    if rank == 0 and args.sweep:
        line["sweep"] = _sweep(P, torch, ctx, args)
    if rank == 0 and args.phase:
        line["phase"] = _phase(P, torch, ctx, args)
    elif rank == 0 and not args.no_phase_small:
        # a coarse cut of the phase map (Fig. 1 setting) in every default run
        line["phase_small"] = _phase(P, torch, ctx, args, ranks=[6, 14, 22, 30, 38, 46],
                                     rhos=[0.05, 0.15, 0.25, 0.35, 0.45], trials=2)
    if rank == 0 and not args.no_video:
        line["video"] = _video(P, torch, ctx, args)
    if rank == 0 and not args.no_batched:
        line["batched"] = _batched(P, torch, ctx, args)
    if rank == 0 and not args.no_serving:
        line["serving"] = _serving(P, torch, ctx, args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    P.pasd_plan_destroy(plan)
    P.pasd_ctx_destroy(ctx)
    if dist is not None:
        dist.destroy_process_group()


def run_profile_workload(args):
    """For ncu: plan a workload, run `pre` loop bodies, then `iters` more, exit.
    --workload cube200 (default): the 200^3 workload; video: the 144x176x3x300
    colour-video shape with R = (20, 20, 3, 5). Launch order per body: polar,
    A-pass (one launch per group of modes with the same padded rank), SVT, Vrot
    (one launch per rank bucket), fused pass, M-pass, finalize; pasd_begin
    launches 3 kernels first. --mixed
    plans it with mixed precision."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_1712_09999_gb300 import pasd as P
    from paper_1712_09999_gb300 import synth
    torch.cuda.set_device(0)
    prec = P.PREC_MIXED if args.mixed else P.PREC_FP32
    if args.workload == "video":
        pr = synth.video()
        params = P.make_params(pr.T.shape, (20, 20, 3, 5), stop=P.STOP_FIXED_ITERS,
                               max_iter=args.pre + args.iters + 1, precision=prec)
    else:
        pr = synth.cube_200(1)
        params = P.make_params(DIMS, RANKS, alpha=ALPHA, lam=LAMBDA, stop=P.STOP_FIXED_ITERS,
                               max_iter=args.pre + args.iters + 1, precision=prec)
    T = torch.from_numpy(pr.T).cuda()
    ctx = P.pasd_ctx_create(0)
    plan, _ = P.pasd_plan(ctx, params)
    P.pasd_begin(plan, T)
    P.pasd_iterate(plan, args.pre)
    P.pasd_iterate(plan, args.iters)
    torch.cuda.synchronize()
    print(json.dumps({"profile_workload": args.workload, "pre": args.pre, "iters": args.iters,
                      "launches_per_iter": P.pasd_launches_per_iter(plan)}))
    P.pasd_plan_destroy(plan)
    P.pasd_ctx_destroy(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile-workload", action="store_true",
                    help="run loop bodies of the 200^3 workload for an external profiler and exit")
    ap.add_argument("--pre", type=int, default=120)
    ap.add_argument("--iters", type=int, default=2)
    ap.add_argument("--mixed", action="store_true", help="--profile-workload with mixed precision")
    ap.add_argument("--workload", default="cube200", choices=["cube200", "video"],
                    help="--profile-workload: which workload")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20, help="timed whole solves")
    ap.add_argument("--warmup", type=int, default=3, help="untimed whole solves before the timed ones")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-solves", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the served-throughput measurement")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrival rate (requests/s)")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="arrival window (s)")
    ap.add_argument("--serve-low-rate", type=float, default=40.0,
                    help="second arrival rate, below capacity, for service-time latencies")
    ap.add_argument("--no-video", action="store_true", help="skip the video-shape measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-workload measurement")
    ap.add_argument("--no-table1", action="store_true", help="skip the paper's Table 1 workloads")
    ap.add_argument("--sweep", action="store_true", help="solve time against cube size")
    ap.add_argument("--sweep-sides", type=int, nargs="+", default=[100, 200, 300, 400, 500, 600, 800])
    ap.add_argument("--phase", action="store_true", help="phase-transition map on 100^3")
    ap.add_argument("--phase-trials", type=int, default=10)
    ap.add_argument("--no-phase-small", action="store_true", help="skip the coarse phase map of the default run")
    ap.add_argument("--phase-slots", type=int, default=16)
    ap.add_argument("--oracle-one-core", type=float, default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_one_core is not None:
        run_oracle_one_core(args.oracle_one_core)
        return
    if args.profile_workload:
        run_profile_workload(args)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
