"""Benchmark of the matrix-free conic solver's hot path on one B300.

Workload: the large sparse LP (m = 1,000,000 rows, n = 2,500,000 columns, power-law column degrees
on {2..200} with mean 8, about 20M nonzeros, N(0,1) values, K = R^n_+), FP32 sweep with FP64
residual reductions. One step = one check interval of the solve loop: 25 iterations (each a
column-order and a row-order sweep over all nonzeros, with the cone projection and the dual
updates fused in) followed by one FP64 residual evaluation read back to the host.

Metric: A-nonzero updates per second = o x iterations / second (each iteration updates every
nonzero's contribution in both sweeps; counted once). Also reported: the HBM roofline of the
dominant sweep kernel, time to 1e-6 relative KKT residual where reached, an end-to-end number
through the C ABI from host arrays, and the FP64 CPU oracle timed on this host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ITERS_PER_STEP = 25
METRIC = "A-nonzero updates/s (o x iterations / s)"
UNIT = "updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mfs", choices=["mfs", "reference"])
    ap.add_argument("--workload", default="large_lp", choices=["large_lp", "socp"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the extra workloads (batched LPs, shared-A family, MLP step)")
    ap.add_argument("--sweep", default="auto", choices=["auto", "chunked", "staged"],
                    help="sweep kernels of the large LP's FP32 iteration (auto: the library's choice, staged passes on this instance)")
    ap.add_argument("--l2-keep", type=int, default=1, choices=[0, 1],
                    help="settings.l2_keep of the large-LP solvers: raise the context's persisting-L2 set-aside "
                         "while they exist, so that the staged passes keep the iterate's vectors in L2 (each "
                         "is closed before the next section runs)")
    ap.add_argument("--warm-start", type=int, default=4096, metavar="TRAIN",
                    help="learned warm-start experiment with TRAIN training solves (0 skips it; 50000 is the "
                         "full experiment, about 15 minutes)")
    ap.add_argument("--warm-start-test", type=int, default=128,
                    help="held-out members solved to 1e-6 by each arm (cold, network, mean, nearest; 1000 "
                         "in the full experiment)")
    ap.add_argument("--section", default="all", choices=["all", "small", "socp", "paper", "batch", "shared", "mlp", "ruiz"],
                    help="run only one extra workload and print its line (for profiling)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="large LP with m and n scaled by this factor (a smaller case for profiler captures; "
                         "the bench line is quoted at 1.0)")
    ap.add_argument("--tts-iters", type=int, default=300000,
                    help="also solve to 1e-6 KKT from the cold start with at most this many iterations (0: skip)")
    return ap.parse_args()


def dist_env():
    from paper_2203_05027_b300 import replicas
    return replicas.env()


def make_problem(name, seed, scale=1.0):
    from paper_2203_05027_b300 import instances as I
    if name == "large_lp":
        if scale != 1.0:
            return I.large_lp(seed, m=int(1_000_000 * scale), n=int(2_500_000 * scale))
        return I.large_lp(seed)
    return I.socp(seed)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def load_peaks_raw():
    """bf16 tensor-core peak (TFLOP/s): the measured burst figure, else the nominal fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            pk = json.load(f)
        return {"bf16_tflops": float(pk.get("bf16_tflops", 1800.0)), "hbm_gbs": float(pk.get("hbm_gbs", 6400.0))}
    return {"bf16_tflops": 1800.0, "hbm_gbs": 6400.0}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hashes(names):
    import hashlib
    out = {}
    for name in names:
        with open(os.path.join(ROOT, "paper_2203_05027_b300", "csrc", name), "rb") as f:
            out[name] = hashlib.sha256(f.read()).hexdigest()[:16]
    return out


def recorded_traffic(kernel, m, n, o):
    """DRAM bytes of one launch of `kernel` from the committed ncu record, or None when there is
    none, it was taken on another instance (m, n, o), or one of the sources it was captured from
    has changed since."""
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(tpath):
        return None
    with open(tpath) as f:
        doc = json.load(f)
    if not doc.get("workload", "").startswith(f"large_lp m={m} n={n} o={o} "):
        return None
    rec = doc.get("kernels", {}).get(kernel)
    if not rec or rec.get("sources") != kernel_source_hashes(sorted(rec.get("sources", {}))):
        return None
    return rec["dram_bytes"]


def kernel_roofline(s, info, peak, peak_kind, m, n, o, sm_mhz, num_sms=148):
    """Time each kernel of an iteration on the solver's stream with CUDA events (library hook,
    kernel by kernel) and relate the dominant one's algorithmic bytes to the measured HBM copy
    bandwidth. A pass in parts splits its bytes: the staged kernel streams the entries and the
    gathered vector, the combine reads and writes the iterate's vectors. Also relates the launch
    time to the L2-request floor of the random gathers (one 4-byte gather, hence one L2 request,
    per nonzero; one request per SM cycle)."""
    from paper_2203_05027_b300 import mfs
    t = s.time_kernel_split(50)
    col_staged = info.get("sweep_col") == mfs.SWEEP_STAGED
    row_staged = info.get("sweep_row") == mfs.SWEEP_STAGED
    col_split = col_staged and info.get("col_parts", 1) > 1
    row_split = row_staged and info.get("row_parts", 1) > 1
    kernels = [
        {"kernel": "k_staged<0>" if col_staged else "k_col_sweep", "ms": t["col_main_ms"],
         "bytes": 8 * o + 4 * m if col_split else 8 * o + 32 * n + 4 * m},
        # a pass's second kernel: the combine of a pass in parts, the long chunks of a chunked
        # sweep (a staged pass in one part has none: the interval is the gap between two events)
        {"kernel": "k_col_combine" if col_split else "k_col_long",
         "ms": t["col_second_ms"] if (col_split or not col_staged) else 0.0, "bytes": 28 * n if col_split else 0},
        {"kernel": "k_staged<1>" if row_staged else "k_row_sweep", "ms": t["row_main_ms"],
         "bytes": 8 * o + 4 * n if row_split else 8 * o + 4 * n + 20 * m},
        {"kernel": "k_row_combine" if row_split else "k_row_long",
         "ms": t["row_second_ms"] if (row_split or not row_staged) else 0.0, "bytes": 20 * m if row_split else 0},
    ]
    dom = max(kernels, key=lambda k: k["ms"])
    achieved = dom["bytes"] / (dom["ms"] * 1e-3) / 1e9
    it_gbs = info["bytes_per_iter"] / (t["iter_ms"] * 1e-3) / 1e9
    traffic = recorded_traffic(dom["kernel"], m, n, o)
    clock_hz = (sm_mhz or 2032.0) * 1e6
    floor_ms = o / (num_sms * clock_hz) * 1e3
    col_ms = kernels[0]["ms"] + kernels[1]["ms"]
    row_ms = kernels[2]["ms"] + kernels[3]["ms"]
    return {"bound": "hbm", "kernel": dom["kernel"], "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_kind,
            "traffic": traffic, "algorithmic_bytes": dom["bytes"],
            "launch_ms": round(dom["ms"], 5),
            "kernels_ms": {k["kernel"]: round(k["ms"], 5) for k in kernels if k["ms"] > 0},
            "col_ms": round(col_ms, 5), "row_ms": round(row_ms, 5),
            "col_pass_frac": round((8 * o + 32 * n + 4 * m) / (col_ms * 1e-3) / 1e9 / peak, 4),
            "row_pass_frac": round((8 * o + 4 * n + 20 * m) / (row_ms * 1e-3) / 1e9 / peak, 4),
            "iteration_ms": round(t["iter_ms"], 5), "iteration_gbs": round(it_gbs, 1),
            "gather_request_floor_ms": round(floor_ms, 5),
            "frac_of_gather_request_floor": round(floor_ms / dom["ms"], 4)}


def cpu_baseline(prob, iters=3):
    """The FP64 CPU oracle (literal Algorithm 1, single thread) on the same instance: a bounded
    sample of `iters` iterations."""
    import oracle
    orc = oracle.make_oracle(prob)
    t0 = time.perf_counter()
    orc.iterate(iters)
    dt = time.perf_counter() - t0
    return {"value": orc.o * iters / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{iters} literal FP64 iterations of the oracle on the full instance "
                      f"({dt:.2f} s, set-up not timed)"}


def batch_workload(stream, seed, iters=100, tts_iters=300_000, extend_iters=1_000_000):
    """Extra workload: 4096 LPs with m log-uniform on [50, 5000], n = 2.5m, 5 nonzeros per column,
    solved together by one persistent launch (FP32 sweep). The autotuner picks threads per CTA and
    CTAs per SM; then `iters` iterations of the whole batch are timed with CUDA events, and a fresh
    batch is solved to relative KKT 1e-6 (at most `tts_iters` iterations per instance)."""
    import torch
    from paper_2203_05027_b300 import instances as I, mfs
    probs = I.batch_lps(4096, seed=seed)
    bt = mfs.Batch(probs, precision="fp32", check_every=50, stream=stream.cuda_stream)
    info = bt.info()
    tuned = bt.tune(20)
    bt.iterate(3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    bt.iterate(iters)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # both orders of A: a 4-byte value and a 2- or 4-byte local index per nonzero and order
    bytes_iter = 2 * (4 + info["index_bytes"]) * info["total_nnz"] + 36 * info["total_n"] + 24 * info["total_m"]
    bt.close()
    # time to 1e-6 from the cold start, every instance tested inside the launch at the tuned interval
    if not tts_iters:
        return {"ms_per_batch_iteration": round(ms / iters, 5), "tuning": tuned}
    bt2 = mfs.Batch(probs, precision="fp32", check_every=tuned["check_every"], stream=stream.cuda_stream)
    bt2.set_tuning(tuned["threads"], tuned["ctas_per_sm"], tuned["check_every"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its, sts = bt2.solve(1e-6, tts_iters)
    torch.cuda.synchronize()
    tts_s = time.perf_counter() - t0
    kkt = np.array([r["kkt"] for r in bt2.residuals()])
    ok = its[sts == 0]
    left = sts != 0
    ms_ = np.array([p["m"] for p in probs])
    # the members at the cap continue from where they stopped (a second solve; those already at
    # tol leave at their first check), up to extend_iters more iterations each
    ext = None
    if left.any() and extend_iters:
        t1 = time.perf_counter()
        its2, sts2 = bt2.solve(1e-6, extend_iters)
        torch.cuda.synchronize()
        more = left & (sts2 == 0)
        tot = (its + its2)[more]
        kkt2 = np.array([r["kkt"] for r in bt2.residuals()])
        # the instances still above tol, one by one: their KKT decay over the extra iterations
        # (log-linear rate) and the iterations that rate would still need to reach tol
        still = left & (sts2 != 0)
        rate = np.log(kkt[still] / kkt2[still]) / float(extend_iters)
        need = np.where(rate > 0, np.log(np.maximum(kkt2[still], 1e-6) / 1e-6) / np.where(rate > 0, rate, 1.0), np.inf)
        per = [{"m": int(ms_[t]), "kkt_at_cap": float(kkt[t]), "kkt_now": float(kkt2[t]),
                "more_iterations_at_rate": (float(f"{v:.3g}") if np.isfinite(v) else None)}
               for t, v in zip(np.flatnonzero(still), need)]
        ext = {"extra_max_iter": extend_iters, "seconds": round(time.perf_counter() - t1, 3),
               "converged": int(more.sum()), "of": int(left.sum()),
               "converged_total": int(ok.size + more.sum()),
               "total_iterations_median": float(np.median(tot)) if tot.size else None,
               "total_iterations_max": int(tot.max()) if tot.size else None,
               "still_above_tol_kkt_max": float(kkt2[still].max()) if still.any() else None,
               "still_above_tol": {"count": int(still.sum()),
                                   "m_median": float(np.median(ms_[still])) if still.any() else None,
                                   "decreasing": int((rate > 0).sum()),
                                   "more_iterations_median": (float(np.median(need)) if still.any() and
                                                              np.isfinite(np.median(need)) else None),
                                   "instances": per}}
    bt2.close()
    tts = {"tol": 1e-6, "max_iter": tts_iters, "seconds": round(tts_s, 3), "converged": int(ok.size),
           "instances_per_s": round(ok.size / tts_s, 1),
           "iterations_median": float(np.median(ok)) if ok.size else None,
           "iterations_p90": float(np.percentile(ok, 90)) if ok.size else None,
           # every instance's outcome: those that reached the cap first, by their KKT residual there
           "at_cap": {"count": int(left.sum()),
                      "kkt_median": float(np.median(kkt[left])) if left.any() else None,
                      "kkt_max": float(kkt[left].max()) if left.any() else None,
                      "below_1e-5": int((kkt[left] <= 1e-5).sum()), "below_1e-4": int((kkt[left] <= 1e-4).sum()),
                      "m_median": float(np.median(ms_[left])) if left.any() else None},
           "at_cap_continued": ext}
    out = {"workload": "batch_lps 4096 instances, m log-uniform [50, 5000], n = 2.5 m, 5 nnz/col",
           "total_nnz": info["total_nnz"], "total_m": info["total_m"], "total_n": info["total_n"],
           "iterations": iters, "ms_per_batch_iteration": round(ms / iters, 5),
           "value": info["total_nnz"] * iters / (ms * 1e-3), "unit": UNIT, "tuning": tuned,
           "algorithmic_gbs": round(bytes_iter / (ms / iters * 1e-3) / 1e9, 1), "time_to_1e-6": tts}
    return out


def ruiz_workload(stream, seed, max_iter=600_000):
    """Convergence variant outside the paper: Ruiz equilibration (10 passes, mfs_ruiz_scale) of a
    power-law LP (m = 2000, n = 5000, the large LP's construction at a smaller size), solved to
    relative KKT 1e-6 in FP64 with and without it; the scaled solve's point is mapped back and judged
    by the original problem's residuals (a solver of the original warm-started there)."""
    import torch
    from paper_2203_05027_b300 import instances as I, mfs
    prob = I.large_lp(3 + seed, m=2000, n=5000)
    out = {"workload": "power-law LP m=2000 n=5000, FP64, to relative KKT 1e-6, checks every 50",
           "passes": 10}
    for name, scaled in (("plain", False), ("ruiz", True)):
        t0 = time.perf_counter()
        if scaled:
            q, d, e = mfs.ruiz_scale(prob, passes=10)
        else:
            q = prob
        s = mfs.Solver(q, precision="fp64", polish_iters=0, check_every=50, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        st, its = s.solve(1e-6, max_iter)
        torch.cuda.synchronize()
        rec = {"status": st, "iterations": its, "seconds": round(time.perf_counter() - t1, 3),
               "setup_seconds": round(t1 - t0, 3)}
        if scaled:
            sol = s.solution()
            x, lam, z, dl = mfs.ruiz_unscale(d, e, sol["x"], sol["lam"], sol["z"], sol["delta"])
            o = mfs.Solver(prob, precision="fp64", polish_iters=0, stream=stream.cuda_stream)
            o.warm_start(x, lam, z, dl)
            rec["kkt_original"] = o.residuals()["kkt"]
            o.close()
        else:
            rec["kkt_original"] = s.residuals()["kkt"]
        s.close()
        out[name] = rec
    return out


def socp_workload(stream, seed, iters=250):
    """Extra workload: the sparse SOCP (n = 1,000,000 in Lorentz cones of sizes 3..64, m = 400,000 rows
    with 10 nonzeros each), FP32 sweep: `iters` iterations timed with CUDA events (one FP64 residual
    check every 25)."""
    import torch
    from paper_2203_05027_b300 import instances as I, mfs
    prob = I.socp(seed)
    s = mfs.Solver(prob, precision="fp32", polish_iters=0, check_every=25, stream=stream.cuda_stream)
    info = s.info()
    s.iterate(50)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(iters // 25):
        s.iterate(25)
        s.residuals()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iters
    t = s.time_kernels(50)
    o, m, n = info["o"], info["m"], info["n"]
    s.close()
    s = mfs.Solver(prob, precision="fp32", polish_iters=0, check_every=50, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, its = s.solve(1e-6, 100_000)
    torch.cuda.synchronize()
    tts = {"status": st, "iterations": its, "seconds": round(time.perf_counter() - t0, 4), "kkt": s.residuals()["kkt"]}
    s.close()
    return {"workload": f"socp n={n} m={m} o={o}, {len(prob['cones'])} cones", "ms_per_iteration": round(ms, 5),
            "time_to_1e-6": tts,
            "value": o / (ms * 1e-3), "unit": UNIT,
            "algorithmic_gbs": round((16 * o + 36 * n + 24 * m) / (ms * 1e-3) / 1e9, 1),
            "kernel_us": {k.replace("_ms", ""): round(v * 1e3, 2) for k, v in t.items()}}


def paper_family_workload(stream, seed, cap=50_000):
    """Extra workload: the paper's own random family (Sec. V) at its largest size, 1e7 nonzeros:
    LP at 1 % and 0.1 % density and the (K_4)^{n/4} SOCP at 0.1 %; per-iteration time and the
    iterations and seconds to relative KKT 1e-3 (the paper's SCS tolerance) and 1e-6."""
    import torch
    from paper_2203_05027_b300 import instances as I, mfs
    out = []
    for m, n, dens, cone in ((10_000, 100_000, 0.01, "lp"), (30_000, 333_332, 0.001, "lp"),
                             (30_000, 333_332, 0.001, "soc4")):
        prob = I.paper_instance(m, n, dens, cone, seed=seed)
        s = mfs.Solver(prob, precision="fp32", polish_iters=0, check_every=100, stream=stream.cuda_stream)
        o = s.info()["o"]
        t = s.time_kernels(50)
        rec = {"cone": cone, "m": m, "n": n, "density": dens, "o": o,
               "us_per_iteration": round(t["iter_ms"] * 1e3, 2)}
        s.close()
        for tol in (1e-3, 1e-6):
            s = mfs.Solver(prob, precision="fp32", polish_iters=0, check_every=100, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, its = s.solve(tol, cap)
            torch.cuda.synchronize()
            rec[f"to_{tol:g}"] = {"status": st, "iterations": its, "seconds": round(time.perf_counter() - t0, 3)}
            s.close()
        out.append(rec)
    return {"workload": "paper's random family, 1e7 nonzeros, FP32", "instances": out}


def small_workload(stream, seed, iters=2000):
    """Extra workload: the 200 x 500 LP (5 nonzeros per column), 2000 FP64 iterations, through the
    single-instance path (kernels per iteration under a CUDA graph) and as a batch of one (one CTA,
    the instance in shared memory, all iterations in one launch)."""
    import torch
    from paper_2203_05027_b300 import instances as I, mfs
    p = I.small_lp(seed)
    out = {"workload": "small LP m=200 n=500 5 nnz/col, FP64", "iterations": iters}
    s = mfs.Solver(p, precision="fp64", check_every=iters, polish_iters=0, stream=stream.cuda_stream)
    s.iterate(iters)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.iterate(iters)
    e1.record(stream)
    torch.cuda.synchronize()
    out["single_path_us_per_iteration"] = round(e0.elapsed_time(e1) * 1e3 / iters, 3)
    s.close()
    bt = mfs.Batch([p], precision="fp64", check_every=iters, stream=stream.cuda_stream)
    bt.iterate(iters)
    torch.cuda.synchronize()
    e0.record(stream)
    bt.iterate(iters)
    e1.record(stream)
    torch.cuda.synchronize()
    out["one_cta_us_per_iteration"] = round(e0.elapsed_time(e1) * 1e3 / iters, 3)
    bt.close()
    return out


def shared_workload(stream, seed, count=1024, iters=200):
    """Extra workload: `count` members of the parametric LP family (A fixed, m = 20,000, n = 50,000,
    8 nonzeros per column; b and c moved by theta ~ N(0, I_32)) iterated together by the shared-A
    solver (FP32 sweep); `iters` iterations timed with CUDA events."""
    import torch
    from paper_2203_05027_b300 import mfs, warmstart as W
    fam = W.family(seed)
    base = fam["base"]
    sh = mfs.Shared(base, count, check_every=iters, precision="fp32", stream=stream.cuda_stream)
    sh.set_data(*W.data_of(fam, W.thetas(count, seed + 1)))
    sh.iterate(20)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sh.iterate(iters)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iters
    o, m, n = len(base["row"]), base["m"], base["n"]
    bytes_iter = count * (36 * n + 24 * m) + 16 * o
    sh.close()
    return {"workload": f"parametric LP family, {count} members sharing A (m={m}, n={n}, o={o})",
            "ms_per_iteration": round(ms, 5), "us_per_member_iteration": round(ms * 1e3 / count, 4),
            "value": o * count / (ms * 1e-3), "unit": UNIT,
            "algorithmic_gbs": round(bytes_iter / (ms * 1e-3) / 1e9, 1)}


def mlp_workload(stream, peaks, batch=256, steps=20):
    """Extra workload: one Adam training step of the warm-start network (32 -> 512 -> 512 -> 70,000,
    BF16 tensor-core GEMMs, FP32 master weights) on a batch of 256, and its forward pass; FLOPs are
    those of the six GEMMs (2 B (32*512 + 512*512 + 512*70000) forward, twice that backward)."""
    import torch
    from paper_2203_05027_b300 import mfs
    din, width, dout = 32, 512, 70_000
    net = mfs.MLP(din, width, dout, batch, seed=0, stream=stream.cuda_stream)
    g = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn((batch, din), device="cuda", generator=g)
    T = torch.randn((batch, dout), device="cuda", generator=g)
    Y = torch.empty((batch, dout), device="cuda")
    for _ in range(3):
        net.train_step(batch, X.data_ptr(), T.data_ptr(), 1e-4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        net.train_step(batch, X.data_ptr(), T.data_ptr(), 1e-4)
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1) / steps
    e0.record(stream)
    for _ in range(steps):
        net.forward(batch, X.data_ptr(), Y.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / steps
    net.close()
    fwd_flop = 2.0 * batch * (din * width + width * width + width * dout)
    peak = peaks.get("bf16_tflops")
    tf_train = 3 * fwd_flop / (train_ms * 1e-3) / 1e12
    # bytes a training step must move (output layer dominates): W3 in BF16 for the forward and the
    # input-gradient GEMMs, its FP32 value and Adam moments read and written, its BF16 copies
    # written (row- and column-major), targets read, loss gradient written and read
    dw = dout * width
    step_bytes = 2 * dw * 2 + 24 * dw + 2 * dw * 2 + 4 * batch * dout + 2 * batch * dout * 2
    return {"workload": f"MLP {din}-{width}-{width}-{dout}, batch {batch}",
            "train_step_ms": round(train_ms, 4), "forward_ms": round(fwd_ms, 4),
            "train_tflops": round(tf_train, 1), "forward_tflops": round(fwd_flop / (fwd_ms * 1e-3) / 1e12, 1),
            "bf16_peak_tflops": peak, "train_frac_of_measured_peak": round(tf_train / peak, 4) if peak else None,
            "train_step_bytes": step_bytes, "train_gbs": round(step_bytes / (train_ms * 1e-3) / 1e9, 1),
            "train_frac_of_measured_hbm": round(step_bytes / (train_ms * 1e-3) / 1e9 / peaks.get("hbm_gbs", 6485.5), 4),
            "note": "train step = forward, loss, backward GEMMs, transposes, Adam on 36M FP32 parameters, "
                    "and a host read of the loss; the step is bound by HBM (K <= 512), not by the tensor cores"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    prob = make_problem(args.workload, 0)
    import oracle
    orc = oracle.make_oracle(prob)
    for _ in range(max(args.warmup, 0)):
        orc.iterate(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.iterate(1)
    dt = time.perf_counter() - t0
    value = orc.o * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "m": prob["m"], "n": prob["n"],
                                              "o": orc.o, "step": "1 literal FP64 iteration of the CPU oracle"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": value,
                             "sample": f"{args.steps} timed oracle iterations after {args.warmup} warm-up"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    from paper_2203_05027_b300 import build, mfs
    build.build()
    mfs.load()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    if args.section != "all":
        stream = torch.cuda.current_stream()
        fn = {"small": lambda: small_workload(stream, rank), "batch": lambda: batch_workload(stream, rank),
              "socp": lambda: socp_workload(stream, rank), "paper": lambda: paper_family_workload(stream, rank), "shared": lambda: shared_workload(stream, rank),
              "mlp": lambda: mlp_workload(stream, load_peaks_raw()), "ruiz": lambda: ruiz_workload(stream, rank)}[args.section]
        if rank == 0:
            print(json.dumps({"section": args.section, **fn()}), flush=True)
        return

    # replicas only: each rank solves its own instance (seeded by rank), no data-path collective
    prob = make_problem(args.workload, rank, args.scale)
    stream = torch.cuda.current_stream()
    s = mfs.Solver(prob, precision="fp32", polish_iters=0, check_every=ITERS_PER_STEP,
                   stream=stream.cuda_stream, sweep=args.sweep, l2_keep=bool(args.l2_keep))
    info = s.info()
    o, m, n = info["o"], info["m"], info["n"]

    def step():
        s.iterate(ITERS_PER_STEP)
        return s.residuals()

    for _ in range(max(args.warmup, 3)):
        step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            r = step()
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    from paper_2203_05027_b300 import replicas
    ms = replicas.max_over_ranks(ev0.elapsed_time(ev1), dist, device="cuda")
    iters = args.steps * ITERS_PER_STEP
    value = replicas.job_throughput(o * iters, world, ms)

    peak, peak_kind = load_peaks()
    clocks = clk.summary()
    roof = kernel_roofline(s, info, peak, peak_kind, m, n, o, clocks["sm_mhz"],
                           torch.cuda.get_device_properties(local).multi_processor_count)
    # per step: the sweeps of ITERS_PER_STEP iterations + 2 residual kernels (+ big cones) + finalize
    launches_per_step = ITERS_PER_STEP * info["launches_per_iter"] + 3 + (1 if info["nbig"] else 0)
    s.close()  # with l2_keep, its raised L2 set-aside would shrink the L2 of the sections below

    extra = {}
    if args.tts_iters:
        # time to 1e-6 relative KKT residual from the cold (zero) start: FP32 sweep, FP64 checks
        # every 250 iterations, FP64 polish if the FP32 iterate stalls; the set-up (create) is
        # reported apart.
        tc = time.perf_counter()
        s2 = mfs.Solver(prob, precision="fp32", polish_iters=200, check_every=250, stream=stream.cuda_stream,
                        sweep=args.sweep, l2_keep=bool(args.l2_keep))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, its = s2.solve(1e-6, args.tts_iters)
        torch.cuda.synchronize()
        t_solve = time.perf_counter() - t0
        r2 = s2.residuals()
        s2.set_precision("fp32")  # the polish ends in FP64; the FP32 sweeps are what the solve ran
        i2 = s2.info()
        extra["time_to_1e-6"] = {"start": "cold", "status": st, "iterations": its,
                                 "seconds": round(t_solve, 3), "kkt": r2["kkt"],
                                 "pobj": r2["pobj"], "dobj": r2["dobj"],
                                 "sweep": "staged" if i2["sweep_col"] == mfs.SWEEP_STAGED else "chunked",
                                 "create_seconds": round(t0 - tc, 3)}
        s2.close()
        if i2["sweep_col"] == mfs.SWEEP_STAGED or i2["sweep_row"] == mfs.SWEEP_STAGED:
            # the other kernels of the same iteration, for comparison: one warp per chunk of at most
            # 256 nonzeros, every gather an L2 request (a solver without staged passes, so the
            # context's L2 set-aside is at its default)
            s2 = mfs.Solver(prob, precision="fp32", polish_iters=0, stream=stream.cuda_stream, sweep="chunked")
            s2.time_kernels(3)
            tk = s2.time_kernels(20)
            s2.close()
            col_bytes = 8 * o + 32 * n + 4 * m
            extra["chunked_sweeps"] = {
                "col_us": round(tk["col_ms"] * 1e3, 1), "row_us": round(tk["row_ms"] * 1e3, 1),
                "iteration_us": round(tk["iter_ms"] * 1e3, 1),
                "col_gbs": round(col_bytes / (tk["col_ms"] * 1e-3) / 1e9, 1),
                "col_frac_of_measured_hbm": round(col_bytes / (tk["col_ms"] * 1e-3) / 1e9 / peak, 4),
                "note": "k_col_sweep / k_row_sweep (--sweep chunked) on the same instance; same iteration"}
        # a convergence variant outside the paper (residual-balanced mu), reported apart
        s4 = mfs.Solver(prob, precision="fp32", polish_iters=200, check_every=250, stream=stream.cuda_stream,
                        sweep=args.sweep, adapt_mu=4, l2_keep=bool(args.l2_keep))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st4, its4 = s4.solve(1e-6, args.tts_iters)
        torch.cuda.synchronize()
        t4 = time.perf_counter() - t0
        h4, _ = s4.history()
        extra["variant_balanced_mu"] = {
            "rule": "mu doubled / halved at checks 4, 8, 16, ... (every 250 iterations) when the primal and dual "
                    "relative residuals differ by more than 5x; not the paper's method (fixed mu)",
            "status": st4, "iterations": its4, "seconds": round(t4, 3), "kkt": s4.residuals()["kkt"],
            "mu_final": h4[-1]["mu"] if h4 else None}
        s4.close()
        extra["variant_ruiz"] = ruiz_workload(stream, rank)

    if not args.no_batch:
        extra["batch_lps"] = batch_workload(stream, rank)
        extra["small_lp"] = small_workload(stream, rank)
        extra["socp"] = socp_workload(stream, rank)
        extra["paper_family"] = paper_family_workload(stream, rank)
        extra["shared_param_lp"] = shared_workload(stream, rank)
        extra["mlp"] = mlp_workload(stream, load_peaks_raw())
    if args.warm_start and not args.no_batch:
        from paper_2203_05027_b300 import warmstart as W
        ws = W.run(train=args.warm_start, test=args.warm_start_test, seed=rank,
                   log=lambda t: print(t, file=sys.stderr, flush=True))
        full = args.warm_start >= 50_000 and args.warm_start_test >= 1000
        extra["warm_start"] = {"workload": f"parametric LP family (m=20000, n=50000), {args.warm_start} training "
                                           f"solves, {args.warm_start_test} held-out members, to 1e-6"
                                           + ("" if full else " (scaled from 50,000 and 1,000)"),
                               "arms": "cold: zero start; mlp: the trained network's prediction; mean: the mean "
                                       "training solution; nearest: the solution of the nearest training theta",
                               **{k: v for k, v in ws.items() if k != "stage"}}

    e2e = e2e_dev = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s3 = mfs.Solver(prob, precision="fp32", polish_iters=0, check_every=ITERS_PER_STEP,
                        stream=stream.cuda_stream, sweep=args.sweep, l2_keep=bool(args.l2_keep))
        for _ in range(args.steps):
            s3.iterate(ITERS_PER_STEP)
            s3.residuals()
        sol = s3.solution()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        s3.close()
        # the COO crosses as int32 row and column indices (narrowed by the host) and FP64 values
        h2d = prob["row"].size * (4 + 4 + 8) + 8 * (m + n) + 16 * len(prob["cones"])
        d2h = 168 * args.steps + 8 * (3 * n + m)
        e2e = {"value": world * o * iters / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(d2h / args.steps),
               "seconds": round(dt, 3),
               "scope": "mfs_create from host COO (set-up + upload) + all steps + mfs_get_solution to host"}

        # the same, for a caller whose COO, b and c are already in device memory (mfs_create_device):
        # no input crosses from the host; the solution still comes back
        dev_in = {k: torch.from_numpy(np.ascontiguousarray(prob[k], dtype=np.int64)).cuda() for k in ("row", "col")}
        dev_in.update({k: torch.from_numpy(np.ascontiguousarray(prob[k], dtype=np.float64)).cuda()
                       for k in ("val", "b", "c")})
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s5 = mfs.Solver.from_device(m, n, prob["row"].size, dev_in["row"].data_ptr(), dev_in["col"].data_ptr(),
                                    dev_in["val"].data_ptr(), dev_in["b"].data_ptr(), dev_in["c"].data_ptr(),
                                    prob["cones"], precision="fp32", polish_iters=0, check_every=ITERS_PER_STEP,
                                    stream=stream.cuda_stream, sweep=args.sweep, l2_keep=bool(args.l2_keep))
        for _ in range(args.steps):
            s5.iterate(ITERS_PER_STEP)
            s5.residuals()
        sol = s5.solution()
        torch.cuda.synchronize()
        dt5 = time.perf_counter() - t0
        s5.close()
        del dev_in
        e2e_dev = {"value": world * o * iters / dt5, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": int(d2h / args.steps), "seconds": round(dt5, 3),
                   "scope": "mfs_create_device from device COO (set-up on the GPU) + all steps + mfs_get_solution "
                            "to host"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(prob)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 reductions)", "data": "synthetic",
                "config": {"workload": args.workload, "m": m, "n": n, "o": o,
                           "iterations_per_step": ITERS_PER_STEP, "precision": "fp32 sweep + fp64 residuals",
                           "sweeps": {"col": "staged" if info["sweep_col"] == mfs.SWEEP_STAGED else "chunked",
                                      "row": "staged" if info["sweep_row"] == mfs.SWEEP_STAGED else "chunked"},
                           "l2": "inputs larger than L2 (A in both orders is %.0f MB in FP32)" % (16 * o / 1e6),
                           "l2_keep": bool(args.l2_keep),
                           "parallelism": f"replicas{world}"},
                "kkt_after_timed_region": r["kkt"],
                "roofline": roof, "gpu_launches": launches_per_step * args.steps,
                "clocks": clocks, "e2e": e2e, "e2e_device_input": e2e_dev, "cpu_baseline": cpu}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
