"""Throughput of the GB300 SFT Morlet scalogram (one JSON line on rank 0).

Workload (default): the batched scalogram -- 256 float32 signals with lengths log-uniform in
[1024, 1048576] (seed 2), 32 scales sigma = 2^(3 + j/3), omega0 = 6/sigma, K = 4, compensated FP32
(FP32 scan, two-float carries and prefix sums), complex64 outputs, one graph-captured forward per
step (lane-chunk kernel, two warp-scan launches, tile-sum kernel). A step is one whole transform of the batch (all
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
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--workload", default="c3", choices=["c3", "c3_small"],
                    help="c3: the full batched scalogram; c3_small: 64 signals clipped to 65536 samples (profiling)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default row thresholds instead of timing them at plan time")
    ap.add_argument("--thresholds", default=None,
                    help="LS:SS sets the row thresholds (lane-chunk rows L <= LS, start-state rows L > SS) "
                         "instead of autotuning them; profiling runs pass the pair the autotuner keeps")
    ap.add_argument("--scales", default=None,
                    help="a:b keeps scales a..b-1 of the workload (profiling one kernel's rows); default all")
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
    tune = not args.no_autotune and args.thresholds is None
    plan = m.morlet_plan(lens, sigmas, xi=w.xi, K=w.K, precision=m.MORLET_FP32_COMP, form=args.form,
                         flags=m.MORLET_FLAG_AUTOTUNE if tune else 0)
    if args.thresholds:
        ls_max, ss_min = (int(v) for v in args.thresholds.split(":"))
        m.morlet_plan_set_row_thresholds(plan, ls_max, ss_min)
    t_plan = time.perf_counter() - t_plan
    pst = m.morlet_plan_stats(plan)
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

    # sampled correctness of the measured output against the oracle's direct sums
    from oracle import morlet as om
    rng = np.random.default_rng(1)
    worst = 0.0
    offs = np.concatenate([[0], np.cumsum(lens)])
    S = len(sigmas)
    for i in rng.choice(len(lens), 3, replace=False):
        s = int(rng.integers(S))
        fit = om.fit_direct(sigmas[s], w.xi, w.K)
        Ni = lens[i]
        idx = rng.integers(0, Ni, 8)
        ref = om.morlet_sft_direct(w.signals[i].astype(np.float64), fit, idx)
        row0 = S * int(offs[i]) + s * Ni
        got = W[row0 + torch.from_numpy(idx).to(dev)].cpu().numpy()
        worst = max(worst, float(np.abs(got - ref).max() / float(W[row0:row0 + Ni].abs().max().item())))

    # end to end through the same C ABI with host buffers: H2D of x, transform, D2H of W
    out_host = torch.empty(n_out, dtype=torch.complex64).pin_memory()
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        with torch.cuda.stream(st):
            x.copy_(x_host, non_blocking=True)
            m.morlet_forward(plan, x, W, st)
            out_host.copy_(W, non_blocking=True)
        st.synchronize()
    t1 = time.perf_counter()
    barrier()
    e2e_s = (t1 - t0) / args.e2e_steps
    e2e_s = max_over_ranks(e2e_s, ws, dev)
    e2e = {"value": job_rate(n_out, ws, e2e_s), "unit": "output samples/s",
           "h2d_bytes_per_step": int(x_host.numel() * 4), "d2h_bytes_per_step": int(n_out * 8)}
    del out_host

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
                       "row_thresholds": {"lane_chunk_max_L": pst["lane_chunk_max_L"],
                                          "start_state_min_L": pst["start_state_min_L"]}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "forward step (lane-chunk, warp-scan and tile-sum kernels, one graph)",
                         "algorithmic_bytes_per_output": BYTES_PER_OUTPUT,
                         "strict_floor_bytes_per_output": 8 + 4 / S,
                         "strict_floor_frac": achieved * (8 + 4 / S) / BYTES_PER_OUTPUT / peak},
            "clocks": ck, "e2e": e2e, "gpu_launches": args.steps * stats["launches"],
            "device_error": err, "max_rel_err_sampled_vs_oracle": worst,
            "launch_shape": stats,
        }
        line.update(extras)
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def secondary(m, torch, dev, st):
    """Context numbers on the same GPU: the plain FP64 and compensated FP32 single-signal forms (one
    2^24-sample signal, sigma = 8192, K = 6) at their stated accuracy, Gaussian smoothing by the SFT
    and by the ASFT on the 64 x 65536 batch, and the multiplication method beside the direct method."""
    out = {}
    try:
        x5 = WL.c5_pink()
        xs = torch.from_numpy(x5.astype(np.float64)).to(dev)
        for name, prec, dt, ct in (("fp64_single_signal", m.MORLET_FP64, torch.float64, torch.complex128),
                                   ("fp32comp_single_signal", m.MORLET_FP32_COMP, torch.float32, torch.complex64)):
            p = m.morlet_plan([len(x5)], [8192.0], K=6, precision=prec)
            xi = xs.to(dt)
            Wt = torch.empty(len(x5), dtype=ct, device=dev)
            for _ in range(2):
                m.morlet_forward(p, xi, Wt, st)
            st.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            for _ in range(5):
                m.morlet_forward(p, xi, Wt, st)
            b.record(st)
            st.synchronize()
            t = a.elapsed_time(b) / 5
            out[name] = {"workload": "c5_pink_N16777216_sigma8192_K6", "ms": t,
                         "value": len(x5) / (t * 1e-3), "unit": "output samples/s"}
            del Wt, p
        # Gaussian smoothing (eq. GsSFT) and its first derivative by the ASFT (eq. gddAsft) on the
        # 64 x 65536 batch at 16 scales: real output, 4 B read + 4 B written per output
        peak, _ = _peaks()
        w4 = WL.c4_batch()
        lens4 = [len(v) for v in w4.signals]
        n4 = sum(lens4) * len(w4.sigmas)
        x4 = torch.from_numpy(np.concatenate(w4.signals)).to(dev)
        y4 = torch.empty(n4, dtype=torch.float32, device=dev)
        for name, tr, dv, prec in (("gauss_sft_c4_batch", m.MORLET_SFT, 0, m.MORLET_FP32_COMP),
                                   ("gauss_asft_deriv1_c4_batch", m.MORLET_ASFT, 1, m.MORLET_FP32_PLAIN)):
            p = m.morlet_plan(lens4, w4.sigmas, K=7, method=m.MORLET_GAUSS, transform=tr, deriv=dv,
                              precision=prec)
            for _ in range(2):
                m.morlet_forward(p, x4, y4, st)
            st.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            for _ in range(5):
                m.morlet_forward(p, x4, y4, st)
            b.record(st)
            st.synchronize()
            t = a.elapsed_time(b) / 5
            out[name] = {"workload": "c4 batch 64 x 65536 float32, 16 scales, P = 6 (7 terms)", "ms": t,
                         "value": n4 / (t * 1e-3), "unit": "output samples/s",
                         "hbm_frac_at_8B_per_output": 8.0 * n4 / (t * 1e-3) / 1e9 / peak}
            del p
        del y4, x4
        # the multiplication method (Sec. III-B, K = 4 Gaussian terms: 7 non-harmonic terms) and the
        # ASFT (Sec. II-C, K = 4) beside the direct method (K = 4) on the scalogram's scales with
        # L <= 4096 (22 scales)
        w3 = WL.c3_scalogram()
        sig3 = [v for v in w3.sigmas if 4 * v <= 4096]
        n3 = sum(w3.lengths) * len(sig3)
        x3 = torch.from_numpy(w3.concat()).to(dev)
        W3 = torch.empty(n3, dtype=torch.complex64, device=dev)
        # (the ASFT also with MORLET_FLAG_NO_HALO: one look-back chain per row instead of window segments)
        for name, meth, prec, tr, fl in (
                ("multiply_K4_c3_L4096", m.MORLET_MULTIPLY, m.MORLET_FP32_PLAIN, m.MORLET_SFT, 0),
                ("asft_K4_c3_L4096", m.MORLET_DIRECT, m.MORLET_FP32_PLAIN, m.MORLET_ASFT, 0),
                ("asft_K4_c3_L4096_row_chains", m.MORLET_DIRECT, m.MORLET_FP32_PLAIN, m.MORLET_ASFT,
                 m.MORLET_FLAG_NO_HALO),
                ("direct_K4_c3_L4096", m.MORLET_DIRECT, m.MORLET_FP32_COMP, m.MORLET_SFT, 0)):
            p = m.morlet_plan(w3.lengths, sig3, K=4, method=meth, precision=prec, transform=tr, flags=fl)
            for _ in range(2):
                m.morlet_forward(p, x3, W3, st)
            st.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            for _ in range(5):
                m.morlet_forward(p, x3, W3, st)
            b.record(st)
            st.synchronize()
            t = a.elapsed_time(b) / 5
            out[name] = {"workload": f"c3 signals, the {len(sig3)} scales with L <= 4096, K = 4", "ms": t,
                         "value": n3 / (t * 1e-3), "unit": "output samples/s",
                         "hbm_frac_at_12B_per_output": 12.0 * n3 / (t * 1e-3) / 1e9 / peak}
            del p
        del W3, x3
        # the full scalogram with edge extension (MORLET_FLAG_EDGE: padded copy + centre-only rows),
        # and the full scalogram by the ASFT (FP32)
        x1 = torch.from_numpy(w3.concat()).to(dev)
        n1 = w3.n_outputs
        W1 = torch.empty(n1, dtype=torch.complex64, device=dev)
        for name, what, kw in (("edge_extension_c3", "with edge extension",
                                dict(precision=m.MORLET_FP32_COMP, flags=m.MORLET_FLAG_EDGE)),
                               ("asft_K4_c3", "by the ASFT (FP32)",
                                dict(precision=m.MORLET_FP32_PLAIN, transform=m.MORLET_ASFT))):
            p = m.morlet_plan(w3.lengths, w3.sigmas, K=4, **kw)
            for _ in range(2):
                m.morlet_forward(p, x1, W1, st)
            st.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            for _ in range(5):
                m.morlet_forward(p, x1, W1, st)
            b.record(st)
            st.synchronize()
            t = a.elapsed_time(b) / 5
            out[name] = {"workload": f"c3 scalogram (256 signals x 32 scales, K = 4) {what}",
                         "ms": t, "value": n1 / (t * 1e-3), "unit": "output samples/s",
                         "hbm_frac_at_12B_per_output": 12.0 * n1 / (t * 1e-3) / 1e9 / peak}
            del p
        del W1, x1
        # separable 2-D Gaussian filtering of a 4096 x 4096 image (rows, transpose, columns, transpose)
        ny = nx = 4096
        im = torch.randn(ny, nx, device=dev, dtype=torch.float32)
        oi = torch.empty_like(im)
        for _ in range(2):
            m.gauss_filter_2d(im, ny, nx, 8.0, 6, 0, 0, m.MORLET_FP32_COMP, oi, st)
        st.synchronize()
        a.record(st)
        for _ in range(5):
            m.gauss_filter_2d(im, ny, nx, 8.0, 6, 0, 0, m.MORLET_FP32_COMP, oi, st)
        b.record(st)
        st.synchronize()
        t = a.elapsed_time(b) / 5
        out["gauss_filter_2d_4096"] = {"workload": "4096 x 4096 float32 image, sigma = 8, P = 6, G along both axes",
                                       "ms": t, "value": ny * nx / (t * 1e-3), "unit": "pixels/s"}
        del im, oi
    except Exception as e:  # context only; never hides the headline
        out["secondary_error"] = str(e)
    return out


if __name__ == "__main__":
    main()
