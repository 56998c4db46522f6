"""Throughput of the GB300 SFT Morlet scalogram (one JSON line on rank 0).

Workload (default): the batched scalogram -- 256 float32 signals with lengths log-uniform in
[1024, 1048576] (seed 2), 32 scales sigma = 2^(3 + j/3), omega0 = 6/sigma, K = 4, compensated FP32
(FP32 scan, two-float carries and prefix sums), complex64 outputs, one graph-captured forward per
step on the schedule MORLET_FLAG_AUTOTUNE picks (on this batch: the tile sums, then start-state
work items of the warp scan for every row). A step is one whole transform of the batch (all
hot-path steps: load, rotation, scan, start states, combine, store). Metric: complex output samples per second; the roofline counts the algorithmic
12 bytes per output (4-byte input read + 8-byte output write) against the measured copy bandwidth.

--impl reference times the CPU oracle (double-double kernel-integral SFT, oracle/sft_dd.c) on a
bounded sample of the same workload, on the host cores. Under torchrun (N > 1) every rank runs its
own copy of the batch (rows are independent: weak scaling, no collective on the data path).
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

import workloads as WL  # noqa: E402

BYTES_PER_OUTPUT = 12  # 4 B real FP32 input + 8 B complex64 output


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region (clocks and throttle reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()  # the sampler is running before the timed region starts
            while not self.lines and time.time() - t0 < 5.0:
                time.sleep(0.01)
            self.lines.clear()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [a.strip() for a in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline(w, max_seconds=15.0, threads=0):
    """Time the oracle's O-SFT (double-double kernel integral) on the host cores, on a bounded sample:
    whole (signal, scale) rows of the same batch, signals taken in order in groups of 8 until about
    `max_seconds` of wall time have been spent."""
    from oracle import morlet as om
    from oracle import sft_dd
    sft_dd.build()
    fits = [om.fit_direct(s, w.xi, w.K) for s in w.sigmas]
    done, tot, used, dt = 0, 0, 1, 0.0
    while done < len(w.signals) and dt < max_seconds:
        grp = w.signals[done:done + 8]
        t = time.perf_counter()
        _, used = sft_dd.sft_batch(grp, fits, threads)
        dt += time.perf_counter() - t
        tot += sum(len(x) for x in grp) * len(fits)
        done += len(grp)
    return {"value": tot / dt, "unit": "output samples/s", "cores": int(used), "kind": "oracle",
            "sample": f"first {done} of {len(w.signals)} signals x {len(fits)} scales "
                      f"({tot} outputs), double-double O-SFT, {dt:.1f} s"}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int, device) -> float:
    """The largest of the ranks' values (x itself on one rank): a job of replicas takes as long as its
    slowest rank."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, ws: int, seconds: float) -> float:
    """Whole-job throughput of ws replicas that each processed units_per_rank units, the job taking
    `seconds` (the max over ranks)."""
    return ws * units_per_rank / seconds


def run_reference(args, ws, rank):
    """The oracle as the reference arm: each step is a bounded sample of the workload on the host."""
    if rank != 0:
        return
    w = WL.c3_scalogram()
    budget = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(w, max_seconds=min(budget, 5.0))
    vals, walls = [], []
    last = None
    for _ in range(args.steps):
        t = time.perf_counter()
        last = cpu_baseline(w, max_seconds=budget)
        walls.append(time.perf_counter() - t)
        vals.append(last["value"])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": "Morlet output samples/s (batched scalogram, compensated FP32, % HBM roofline)",
            "value": v, "unit": "output samples/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(walls), "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (double-double)", "data": "synthetic",
            "config": {"workload": "c3_scalogram_256sig_32scales_K4 (bounded host sample per step)"},
            "cpu_baseline": {**last, "value": v},
            "e2e": {"value": v, "unit": "output samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--workload", default="c3", choices=["c3", "c3_small"],
                    help="c3: the full batched scalogram; c3_small: 64 signals clipped to 65536 samples (profiling)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default row thresholds instead of timing them at plan time")
    ap.add_argument("--thresholds", default=None,
                    help="LS:SS sets the row thresholds (lane-chunk rows L <= LS, start-state rows L > SS) "
                         "instead of autotuning them; profiling runs pass the pair the autotuner keeps")
    ap.add_argument("--scales", default=None,
                    help="a:b keeps scales a..b-1 of the workload (profiling one kernel's rows); default all")
    ap.add_argument("--schedule", default=None,
                    help="SEG:SS:ORDER sets the window-segment length (8/12/16 L), the start-state item "
                         "size (tiles) and the scale order (0/1) instead of autotuning them")
    ap.add_argument("--only", default=None,
                    help="run only the named secondary measurement (profiling) and print it")
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    import __graft_entry__
    import paper_2110_11866_gb300 as m
    __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if args.only:
        st = torch.cuda.Stream(dev)
        print(json.dumps(secondary(m, torch, dev, st, only=args.only)), flush=True)
        return
    w = WL.c3_scalogram() if args.workload == "c3" else WL.c3_scalogram(n_signals=64, max_len=65536)
    wname = w.name if args.workload == "c3" else "c3_small_64sig_max65536_32scales_K4"
    if args.scales:
        a, b = (int(v) for v in args.scales.split(":"))
        w = WL.Workload(w.name, w.signals, w.sigmas[a:b], w.K)
        wname += f"_scales{a}-{b}"
    lens, sigmas = w.lengths, w.sigmas
    n_out = w.n_outputs
    x_host = torch.from_numpy(w.concat()).pin_memory()
    x = x_host.to(dev)
    t_plan = time.perf_counter()
    tune = not args.no_autotune and args.thresholds is None and args.schedule is None
    plan = m.morlet_plan(lens, sigmas, xi=w.xi, K=w.K, precision=m.MORLET_FP32_COMP, form=args.form,
                         flags=m.MORLET_FLAG_AUTOTUNE if tune else 0)
    if args.thresholds:
        ls_max, ss_min = (int(v) for v in args.thresholds.split(":"))
        m.morlet_plan_set_row_thresholds(plan, ls_max, ss_min)
    if args.schedule:
        seg, sst, order = (int(v) for v in args.schedule.split(":"))
        m.morlet_plan_set_schedule(plan, seg, sst, order, 0)
    t_plan = time.perf_counter() - t_plan
    pst = m.morlet_plan_stats(plan)
    sched = m.morlet_plan_schedule(plan)
    W = torch.empty(n_out, dtype=torch.complex64, device=dev)
    st = torch.cuda.Stream(dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    with torch.cuda.stream(st):
        for _ in range(args.warmup):
            m.morlet_forward(plan, x, W, st)
    st.synchronize()
    err = m.morlet_last_device_error(plan, st)
    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e0.record(st)
    for k in range(args.steps):
        ev[k].record(st)
        m.morlet_forward(plan, x, W, st)
    ev[args.steps].record(st)
    e1.record(st)
    st.synchronize()
    barrier()
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    per_launch = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    ms = max_over_ranks(ms, ws, dev)
    err = err or m.morlet_last_device_error(plan, st)
    value = job_rate(n_out, ws, ms * 1e-3)
    peak, peak_kind = _peaks()
    launch_ms = statistics.mean(per_launch)
    achieved = n_out * BYTES_PER_OUTPUT / (launch_ms * 1e-3) / 1e9
    # DRAM traffic per step from the committed ncu capture of the same kernels (dram bytes read +
    # written per output, scaled by this workload's outputs); null once the sources have changed
    traffic = None
    tf = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tf):
        try:
            with open(tf) as f:
                tj = json.load(f)
            if tj.get("source_hash") == m.source_hash():
                traffic = float(tj["bytes_per_output"]) * n_out
        except Exception:
            traffic = None

    # correctness of the measured output: whole (signal, scale) rows against the oracle's O-SFT
    # (double-double kernel integral, the oracle's own fit), error over the oracle's row maximum
    worst, err_rows = headline_error(W, w, lens, sigmas)
    S = len(sigmas)

    # end to end through the same C ABI with host buffers: H2D of x, transform, D2H of W, every step.
    # Two steps are in flight, as a streaming user would run them: step k + 1's input copy and
    # transform run on `st` while step k's scalogram is copied back on a second stream (two plans with
    # the same schedule, two device buffer pairs; a buffer pair is reused only after its copy-out has
    # finished). CUDA events split each step into its copy-in, compute and copy-out phases.
    sc = m.morlet_plan_schedule(plan)
    plan2 = m.morlet_plan(lens, sigmas, xi=w.xi, K=w.K, precision=m.MORLET_FP32_COMP, form=args.form)
    if args.form != 1:  # the rotating form (the default): the schedule of the timed plan
        m.morlet_plan_set_row_thresholds(plan2, sc["lane_chunk_max_L"], sc["start_state_min_L"])
        m.morlet_plan_set_schedule(plan2, sc["seg_mult"], sc["ss_tiles_max"], sc["order"], sc["asft_chains"])
    x2, W2 = torch.empty_like(x), torch.empty_like(W)
    bx, bw, bp = (x, x2), (W, W2), (plan, plan2)
    so = torch.cuda.Stream(dev)
    out_host = torch.empty(n_out, dtype=torch.complex64).pin_memory()
    with torch.cuda.stream(st):  # warm the second plan's graph
        m.morlet_forward(plan2, x2, W2, st)
    torch.cuda.synchronize(dev)
    barrier()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.e2e_steps)]
    t0 = time.perf_counter()
    for k in range(args.e2e_steps):
        b = k % 2
        with torch.cuda.stream(st):
            evs[k][0].record(st)
            bx[b].copy_(x_host, non_blocking=True)
            evs[k][1].record(st)
            if k >= 2:
                st.wait_event(evs[k - 2][5])  # step k - 2's copy-out has read W[b]
            evs[k][2].record(st)
            m.morlet_forward(bp[b], bx[b], bw[b], st)
            evs[k][3].record(st)
        so.wait_event(evs[k][3])
        with torch.cuda.stream(so):
            evs[k][4].record(so)
            out_host.copy_(bw[b], non_blocking=True)
            evs[k][5].record(so)
    so.synchronize()
    st.synchronize()
    t1 = time.perf_counter()
    barrier()
    e2e_s = (t1 - t0) / args.e2e_steps
    e2e_s = max_over_ranks(e2e_s, ws, dev)
    h2d_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    cmp_ms = statistics.mean(e[2].elapsed_time(e[3]) for e in evs)
    d2h_ms = statistics.mean(e[4].elapsed_time(e[5]) for e in evs)
    h2d_b, d2h_b = int(x_host.numel() * 4), int(n_out * 8)
    e2e = {"value": job_rate(n_out, ws, e2e_s), "unit": "output samples/s",
           "h2d_bytes_per_step": h2d_b, "d2h_bytes_per_step": d2h_b,
           "ms_per_step": 1e3 * e2e_s, "h2d_ms": h2d_ms, "compute_ms": cmp_ms, "d2h_ms": d2h_ms,
           "h2d_GBps": h2d_b / (h2d_ms * 1e-3) / 1e9, "d2h_GBps": d2h_b / (d2h_ms * 1e-3) / 1e9,
           "steps_in_flight": 2,
           "note": "pinned host buffers; two steps in flight (step k + 1's copy-in and transform overlap "
                   "step k's copy-out); the three phases are CUDA-event times, ms_per_step the host wall time "
                   "per step"}
    del out_host, x2, W2, plan2

    extras = {}
    if not args.no_extras and rank == 0:
        extras = secondary(m, torch, dev, st)

    stats = m.morlet_plan_stats(plan)
    if rank == 0:
        line = {
            "metric": "Morlet output samples/s (batched scalogram, compensated FP32, % HBM roofline)",
            "value": value, "unit": "output samples/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wname,
                       "signals": len(lens),
                       "samples": int(sum(lens)), "scales": S, "K": w.K, "outputs_per_step": n_out,
                       "precision": "FP32 scan (packed term pairs), two-float carries", "form": "rotating" if args.form != 1 else "kernel-integral",
                       "l2": f"inputs {4 * sum(lens) / 1e6:.0f} MB + outputs {8 * n_out / 1e9:.2f} GB per step "
                             "exceed the 129 MB L2 (no flush between steps)",
                       "parallelism": f"replicas x{ws}", "plan_seconds": round(t_plan, 2),
                       "autotune": tune,
                       "schedule": sched,
                       "row_thresholds": {"lane_chunk_max_L": pst["lane_chunk_max_L"],
                                          "start_state_min_L": pst["start_state_min_L"]}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "forward step, whole graph (" + ", ".join(
                             k for k, on in (("lane-chunk scan", stats.get("rows_lane_chunk", 0) > 0),
                                             ("warp scan", stats.get("rows_window", 0) + stats.get("rows_start_state", 0) > 0),
                                             ("tile sums", stats.get("prefix_items", 0) > 0),
                                             ("look-back scan", stats.get("rows_lookback", 0) > 0)) if on) + ")",
                         "algorithmic_bytes_per_output": BYTES_PER_OUTPUT,
                         "strict_floor_bytes_per_output": 8 + 4 / S,
                         "strict_floor_frac": achieved * (8 + 4 / S) / BYTES_PER_OUTPUT / peak},
            "clocks": ck, "e2e": e2e, "gpu_launches": args.steps * stats["launches"],
            "device_error": err, "max_rel_err_vs_oracle": worst,
            "error_check": err_rows,
            "launch_shape": stats,
        }
        line.update(extras)
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def _row_err(got, ref):
    """max over rows of max|got - ref| / max|ref| (the oracle's maximum in the denominator)."""
    got = np.atleast_2d(np.asarray(got))
    ref = np.atleast_2d(np.asarray(ref))
    return float((np.abs(got - ref).max(axis=1) / np.maximum(np.abs(ref).max(axis=1), 1e-300)).max())


def headline_error(W, w, lens, sigmas):
    """Error of the measured scalogram on whole rows: three signals (the longest, the shortest and the
    median length) at every scale against the oracle's O-SFT (double-double kernel integral with the
    oracle's own fit); each row's error is over the oracle's maximum of that row."""
    from oracle import morlet as om
    from oracle import sft_dd
    fits = [om.fit_direct(s, w.xi, w.K) for s in sigmas]
    S = len(sigmas)
    offs = np.concatenate([[0], np.cumsum(lens)])
    order = np.argsort(lens)
    pick = [int(order[-1]), int(order[0]), int(order[len(order) // 2])]
    worst = 0.0
    for i in pick:
        ref, _ = sft_dd.sft_batch([w.signals[i]], fits)
        n = lens[i]
        got = W[S * int(offs[i]):S * int(offs[i]) + S * n].cpu().numpy()
        worst = max(worst, _row_err(got.reshape(S, n), ref.reshape(S, n)))
    return worst, {"rows": f"signals {pick} (lengths {[lens[i] for i in pick]}) x all {S} scales, every output",
                   "oracle": "double-double O-SFT (kernel integral, Sec. II-B), error over the row's oracle max"}


def _timed(torch, fn, st, reps=5, warm=2):
    """Mean CUDA-event time (ms) of fn() on stream st over `reps` calls after `warm` warm-up calls."""
    for _ in range(warm):
        fn()
    st.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        fn()
    b.record(st)
    st.synchronize()
    return a.elapsed_time(b) / reps


def _fp64_ops_per_output():
    """FP64 operations per output of the FP64 path (ncu instruction counts of its scan kernel,
    profiles/fp64_ops.json), or None once the CUDA sources have changed."""
    try:
        import paper_2110_11866_gb300 as m
        with open(os.path.join(ROOT, "profiles", "fp64_ops.json")) as f:
            j = json.load(f)
        if j.get("source_hash") == m.source_hash():
            return float(j["fp64_ops_per_output"])
    except Exception:
        pass
    return None


def secondary(m, torch, dev, st, only=None):
    """The other forms on the same GPU, each with its rate and its error against the oracle:
    - the plain FP64 and compensated FP32 single-signal forms (2^24 samples, sigma = 8192, K = 6),
      the FP64 one also as a fraction of the measured FP64 FMA rate;
    - the kernel-integral form (modulate, prefix-scan, difference) on the full scalogram;
    - the adjoint (morlet_backward) on the 64 x 65536 batch at 16 scales;
    - Gaussian smoothing by the SFT and its first derivative by the ASFT on that batch;
    - the multiplication method, the ASFT and the direct method on the scalogram's scales with
      L <= 4096, and the full scalogram by the ASFT and with edge extension;
    - separable 2-D Gaussian filtering of a 4096 x 4096 image.
    Errors are max|got - oracle| / max|oracle| over whole rows (or the stated part of them). The
    batched forms are planned with MORLET_FLAG_AUTOTUNE, like the headline; their keys carry the
    schedule the tuner chose."""
    from oracle import morlet as om
    from oracle import sft_dd
    out = {}
    peak, _ = _peaks()

    def want(name):
        return only is None or only == name

    def guard(name, fn):
        if not want(name):
            return
        try:
            out[name] = fn()
        except Exception as e:  # context only; never hides the headline
            out[name] = {"error": f"{type(e).__name__}: {e}"}

    # ---- single long signal, FP64 and compensated FP32 ----
    x5 = WL.c5_pink()
    M5 = 1 << 21  # the oracle runs on the first 2^21 samples; outputs n < M5 - L see only those

    def single(prec):
        f64 = prec == m.MORLET_FP64
        sg, K = 8192.0, 6
        p = m.morlet_plan([len(x5)], [sg], K=K, precision=prec)
        xi = torch.from_numpy(x5.astype(np.float64) if f64 else x5).to(dev)
        Wt = torch.empty(len(x5), dtype=torch.complex128 if f64 else torch.complex64, device=dev)
        t = _timed(torch, lambda: m.morlet_forward(p, xi, Wt, st), st)
        fit = om.fit_direct(sg, 6.0, K)
        ref = sft_dd.sft_direct_method(x5[:M5].astype(np.float64), fit)[:M5 - fit["L"]]
        got = Wt[:M5 - fit["L"]].cpu().numpy()
        r = {"workload": "c5_pink_N16777216_sigma8192_K6", "ms": t, "value": len(x5) / (t * 1e-3),
             "unit": "output samples/s", "max_rel_err_vs_oracle": _row_err(got, ref),
             "error_on": f"outputs 0..{M5 - fit['L'] - 1} (oracle O-SFT on the first {M5} samples)",
             "kernel": m.morlet_plan_stats(p)}
        if f64:
            rate = m.morlet_measure_fp64_rate(st)
            ops = _fp64_ops_per_output()
            r["fp64_fma_peak_flops_measured"] = rate
            if ops is not None:
                r["fp64_ops_per_output"] = ops
                r["fp64_achieved_flops"] = ops * r["value"]
                r["fp64_frac_of_measured"] = ops * r["value"] / rate
        del Wt, p
        return r

    guard("fp64_single_signal", lambda: single(m.MORLET_FP64))
    guard("fp32comp_single_signal", lambda: single(m.MORLET_FP32_COMP))

    w3 = WL.c3_scalogram()
    lens3 = w3.lengths
    offs3 = np.concatenate([[0], np.cumsum(lens3)])
    order3 = np.argsort(lens3)
    long_i, mid_i = int(order3[-1]), int(order3[len(order3) // 2])

    def rows_of(Wt, i, S):
        n = lens3[i]
        return Wt[S * int(offs3[i]):S * int(offs3[i]) + S * n].cpu().numpy().reshape(S, n)

    # ---- kernel-integral form on the full scalogram ----
    def kernel_integral():
        S = len(w3.sigmas)
        x = torch.from_numpy(w3.concat()).to(dev)
        Wt = torch.empty(w3.n_outputs, dtype=torch.complex64, device=dev)
        p = m.morlet_plan(lens3, w3.sigmas, K=4, precision=m.MORLET_FP32_COMP, form=m.MORLET_FORM_KERNEL)
        t = _timed(torch, lambda: m.morlet_forward(p, x, Wt, st), st)
        fits = [om.fit_direct(sg, 6.0, 4) for sg in w3.sigmas]
        err = 0.0
        for i in (long_i, mid_i):
            ref, _ = sft_dd.sft_batch([w3.signals[i]], fits)
            err = max(err, _row_err(rows_of(Wt, i, S), ref.reshape(S, lens3[i])))
        v = w3.n_outputs / (t * 1e-3)
        del Wt, x, p
        return {"workload": "c3 scalogram (256 signals x 32 scales, K = 4), kernel-integral form "
                            "(CTA decoupled look-back, phases anchored per tile), compensated FP32",
                "ms": t, "value": v, "unit": "output samples/s",
                "hbm_frac_at_12B_per_output": 12.0 * v / 1e9 / peak,
                "max_rel_err_vs_oracle": err, "error_on": f"signals {long_i}, {mid_i} x 32 scales, every output"}

    guard("kernel_integral_c3", kernel_integral)

    # ---- adjoint on the differentiation batch ----
    w4 = WL.c4_batch()
    lens4 = w4.lengths
    B4, S4, N4 = len(lens4), len(w4.sigmas), lens4[0]

    def adjoint():
        x = torch.from_numpy(np.concatenate(w4.signals)).to(dev)
        p = m.morlet_plan(lens4, w4.sigmas, K=4, precision=m.MORLET_FP32_COMP)
        rng = np.random.default_rng(8)
        g = torch.from_numpy((rng.standard_normal(B4 * S4 * N4) + 1j * rng.standard_normal(B4 * S4 * N4))
                             .astype(np.complex64)).to(dev)
        gx = torch.empty(B4 * N4, dtype=torch.float32, device=dev)
        t = _timed(torch, lambda: m.morlet_backward(p, g, gx, st), st)
        fits = [om.fit_direct(sg, 6.0, 4) for sg in w4.sigmas]
        gh = g.view(B4, S4, N4).cpu().numpy().astype(np.complex128)
        gxh = gx.view(B4, N4).cpu().numpy()
        err = 0.0
        for b in (0, B4 - 1):
            ref = sum(sft_dd.adjoint_sft(gh[b, s], fits[s]) for s in range(S4))
            err = max(err, _row_err(gxh[b], ref))
        n_g = B4 * S4 * N4
        v = n_g / (t * 1e-3)
        alg = 8.0 * n_g + 4.0 * B4 * N4
        del g, gx, x, p
        return {"workload": "c4 batch 64 x 65536, 16 scales, K = 4: gx = adjoint(gW) (gW split into 32 real "
                            "planes, their real-output transforms in one launch, the planes summed in order)",
                "ms": t, "value": v, "unit": "gW samples/s",
                "algorithmic_bytes": alg, "hbm_frac": alg / (t * 1e-3) / 1e9 / peak,
                "max_rel_err_vs_oracle": err, "error_on": "signals 0 and 63, every coordinate (sum over the 16 scales)"}

    guard("adjoint_c4", adjoint)

    # ---- Gaussian smoothing (SFT) and first derivative (ASFT), real output ----
    def gauss(tr, dv, prec):
        x = torch.from_numpy(np.concatenate(w4.signals)).to(dev)
        n4 = B4 * N4 * S4
        y = torch.empty(n4, dtype=torch.float32, device=dev)
        p = m.morlet_plan(lens4, w4.sigmas, K=7, method=m.MORLET_GAUSS, transform=tr, deriv=dv, precision=prec,
                          flags=m.MORLET_FLAG_AUTOTUNE)
        sched = m.morlet_plan_schedule(p)
        t = _timed(torch, lambda: m.morlet_forward(p, x, y, st), st)
        err = 0.0
        for b in (0, B4 - 1):
            got = y[b * S4 * N4:(b + 1) * S4 * N4].cpu().numpy().reshape(S4, N4)
            xb = w4.signals[b].astype(np.float64)
            for s, sg in enumerate(w4.sigmas):
                if tr == m.MORLET_SFT:
                    ref = sft_dd.sft_gauss(xb, om.fit_gauss(sg, 6, dv))
                else:
                    ref = sft_dd.asft_gauss(xb, om.fit_gauss_asft(sg, 6, dv, om.default_n0(sg)))
                err = max(err, _row_err(got[s], ref))
        del y, x, p
        return {"workload": "c4 batch 64 x 65536 float32, 16 scales, P = 6 (7 terms)", "ms": t, "schedule": sched,
                "value": n4 / (t * 1e-3), "unit": "output samples/s",
                "hbm_frac_at_8B_per_output": 8.0 * n4 / (t * 1e-3) / 1e9 / peak,
                "max_rel_err_vs_oracle": err, "error_on": "signals 0 and 63 x 16 scales, every output"}

    guard("gauss_sft_c4_batch", lambda: gauss(m.MORLET_SFT, 0, m.MORLET_FP32_COMP))
    guard("gauss_asft_deriv1_c4_batch", lambda: gauss(m.MORLET_ASFT, 1, m.MORLET_FP32_PLAIN))

    # ---- multiplication method, ASFT and direct method on the scales with L <= 4096 ----
    sig22 = [v for v in w3.sigmas if 4 * v <= 4096]
    short_i = int(order3[0])

    def scales22(meth, prec, tr, fl):
        S = len(sig22)
        n3 = sum(lens3) * S
        x = torch.from_numpy(w3.concat()).to(dev)
        Wt = torch.empty(n3, dtype=torch.complex64, device=dev)
        p = m.morlet_plan(lens3, sig22, K=4, method=meth, precision=prec, transform=tr,
                          flags=fl | m.MORLET_FLAG_AUTOTUNE)
        sched = m.morlet_plan_schedule(p)
        t = _timed(torch, lambda: m.morlet_forward(p, x, Wt, st), st)
        err = 0.0
        picks = (short_i, mid_i) if meth == m.MORLET_MULTIPLY else (long_i, mid_i)
        for i in picks:
            xd = w3.signals[i].astype(np.float64)
            got = rows_of(Wt, i, S)
            for s, sg in enumerate(sig22):
                if meth == m.MORLET_MULTIPLY:
                    ref = om.morlet_multiply_direct(xd, om.fit_multiply(sg, 6.0, 4))
                elif tr == m.MORLET_ASFT:
                    ref = sft_dd.asft_direct_method(xd, om.fit_direct(sg, 6.0, 4), sg, 6.0, om.default_n0(sg))
                else:
                    ref = sft_dd.sft_direct_method(xd, om.fit_direct(sg, 6.0, 4))
                err = max(err, _row_err(got[s], ref))
        del Wt, x, p
        return {"workload": f"c3 signals, the {S} scales with L <= 4096, K = 4", "ms": t, "schedule": sched,
                "value": n3 / (t * 1e-3), "unit": "output samples/s",
                "hbm_frac_at_12B_per_output": 12.0 * n3 / (t * 1e-3) / 1e9 / peak,
                "max_rel_err_vs_oracle": err,
                "error_on": f"signals {list(picks)} (lengths {[lens3[i] for i in picks]}) x {S} scales, every output"}

    guard("multiply_K4_c3_L4096", lambda: scales22(m.MORLET_MULTIPLY, m.MORLET_FP32_PLAIN, m.MORLET_SFT, 0))
    guard("asft_K4_c3_L4096", lambda: scales22(m.MORLET_DIRECT, m.MORLET_FP32_PLAIN, m.MORLET_ASFT, 0))
    guard("asft_K4_c3_L4096_row_chains",
          lambda: scales22(m.MORLET_DIRECT, m.MORLET_FP32_PLAIN, m.MORLET_ASFT, m.MORLET_FLAG_NO_HALO))
    guard("direct_K4_c3_L4096", lambda: scales22(m.MORLET_DIRECT, m.MORLET_FP32_COMP, m.MORLET_SFT, 0))

    # ---- the full scalogram with edge extension, and by the ASFT ----
    def full(what, kw, edge):
        S = len(w3.sigmas)
        x = torch.from_numpy(w3.concat()).to(dev)
        Wt = torch.empty(w3.n_outputs, dtype=torch.complex64, device=dev)
        kw = dict(kw)
        kw["flags"] = kw.get("flags", 0) | m.MORLET_FLAG_AUTOTUNE
        p = m.morlet_plan(lens3, w3.sigmas, K=4, **kw)
        sched = m.morlet_plan_schedule(p)
        t = _timed(torch, lambda: m.morlet_forward(p, x, Wt, st), st)
        err = 0.0
        for i in (long_i, mid_i):
            xd = w3.signals[i].astype(np.float64)
            got = rows_of(Wt, i, S)
            for s, sg in enumerate(w3.sigmas):
                fit = om.fit_direct(sg, 6.0, 4)
                if edge:
                    E = fit["L"]
                    ref = sft_dd.sft_direct_method(om.edge_extended(xd, E), fit)[E:E + len(xd)]
                else:
                    ref = sft_dd.asft_direct_method(xd, fit, sg, 6.0, om.default_n0(sg))
                err = max(err, _row_err(got[s], ref))
        del Wt, x, p
        v = w3.n_outputs / (t * 1e-3)
        return {"workload": f"c3 scalogram (256 signals x 32 scales, K = 4) {what}", "ms": t, "value": v,
                "schedule": sched,
                "unit": "output samples/s", "hbm_frac_at_12B_per_output": 12.0 * v / 1e9 / peak,
                "max_rel_err_vs_oracle": err,
                "error_on": f"signals {long_i}, {mid_i} (lengths {lens3[long_i]}, {lens3[mid_i]}) x 32 scales, every output"}

    # ---- the full scalogram by the multiplication method (windows up to L = 41286) ----
    def multiply_full():
        S = len(w3.sigmas)
        x = torch.from_numpy(w3.concat()).to(dev)
        Wt = torch.empty(w3.n_outputs, dtype=torch.complex64, device=dev)
        p = m.morlet_plan(lens3, w3.sigmas, K=4, method=m.MORLET_MULTIPLY, precision=m.MORLET_FP32_PLAIN,
                          flags=m.MORLET_FLAG_AUTOTUNE)
        sched = m.morlet_plan_schedule(p)
        t = _timed(torch, lambda: m.morlet_forward(p, x, Wt, st), st)
        err = 0.0
        rng = np.random.default_rng(7)
        for i in (short_i, mid_i, long_i):
            xd = w3.signals[i].astype(np.float64)
            got = rows_of(Wt, i, S)
            n = lens3[i]
            # the shortest signal whole; the others at 512 positions (both ends, the middle, random)
            idx = None if n <= 4096 else np.unique(np.concatenate([[0, 1, n // 2, n - 2, n - 1],
                                                                   rng.integers(0, n, 507)]))
            for s, sg in enumerate(w3.sigmas):
                ref = om.morlet_multiply_direct(xd, om.fit_multiply(sg, 6.0, 4), idx)
                err = max(err, _row_err(got[s] if idx is None else got[s][idx], ref))
        del Wt, x, p
        v = w3.n_outputs / (t * 1e-3)
        return {"workload": "c3 scalogram (256 signals x 32 scales) by the multiplication method, K = 4 "
                            "(7 non-harmonic terms, FP32)", "ms": t, "value": v, "schedule": sched,
                "unit": "output samples/s", "hbm_frac_at_12B_per_output": 12.0 * v / 1e9 / peak,
                "max_rel_err_vs_oracle": err,
                "error_on": f"signal {short_i} (length {lens3[short_i]}) x 32 scales, every output; signals "
                            f"{mid_i}, {long_i} x 32 scales at 512 positions each (denominator: the oracle's "
                            f"maximum over those positions)"}

    guard("multiply_K4_c3", multiply_full)
    guard("edge_extension_c3", lambda: full("with edge extension",
                                            dict(precision=m.MORLET_FP32_COMP, flags=m.MORLET_FLAG_EDGE), True))
    guard("asft_K4_c3", lambda: full("by the ASFT (FP32)",
                                     dict(precision=m.MORLET_FP32_PLAIN, transform=m.MORLET_ASFT), False))

    # ---- separable 2-D Gaussian filtering ----
    def filter2d():
        ny = nx = 4096
        img = np.random.default_rng(9).standard_normal((ny, nx)).astype(np.float32)
        im = torch.from_numpy(img).to(dev)
        oi = torch.empty_like(im)
        t = _timed(torch, lambda: m.gauss_filter_2d(im, ny, nx, 8.0, 6, 0, 0, m.MORLET_FP32_COMP, oi, st), st)
        # the oracle on a 512 x 512 corner block of a cropped image: output pixels at least L from the
        # crop's inner edges see only pixels inside it
        L = om.window_half(8.0)
        c = 512 + L
        ref = om.gauss_filter_2d_direct(img[:c, :c].astype(np.float64), 8.0, 6, 0, 0)[:512, :512]
        got = oi[:512, :512].cpu().numpy()
        err = float(np.abs(got - ref).max() / np.abs(ref).max())
        del im, oi
        return {"workload": "4096 x 4096 float32 image, sigma = 8, P = 6, G along both axes", "ms": t,
                "value": ny * nx / (t * 1e-3), "unit": "pixels/s", "max_rel_err_vs_oracle": err,
                "error_on": "the 512 x 512 corner block (both image edges), every pixel"}

    guard("gauss_filter_2d_4096", filter2d)
    return out


if __name__ == "__main__":
    main()
