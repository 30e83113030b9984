"""Benchmark: batched ion-steps/s of the REED-MD track stepper on GB300.

A "step" is one pass of the whole hot path over one batch: reed_run of the
workload's primaries (4096 As ions at 10 keV into Si at 300 K, Tersoff
target, 5x5x5-cell window) followed to the end of every track.  Each timed
step runs a fresh batch (primary ids step*n ... ) in the mixed-precision form.

Reported beside it: the plain FP64 GPU path on the same 4096-ion batch as
the first timed step (the metric's comparison), the range-profile error of
both forms against the oracle's stored ranges of this workload (mean,
straggle, KS p, with their sampling errors), the FP32-ALU and SFU rooflines
of the stepper kernel, the CPU oracle timed on the host cores, and an
end-to-end figure through the public API with host buffers.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank runs its own shard of primaries (weak scaling).
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

METRIC = "batched ion-steps/s on 1 GB300, chosen vs plain FP64 path, range-profile KS p>0.01"
WORKLOAD = "as10kev_si_300k_tersoff"
# Algorithmic FP32 work per unit (see the design notes): ZBL ion-target pair
# 35 ops, integrated atom update 12 FMA = 24 ops, Tersoff bond-angle triplet 60 ops.
OPS_PAIR, OPS_MOVE, OPS_TRIPLET = 35, 24, 60
# Algorithmic SFU (transcendental) work per unit: ZBL pair 4 ex2 + 1 rsqrt,
# Tersoff bond-angle term one reciprocal (the angular function g).
SFU_PAIR, SFU_TRIPLET = 5, 1
SMS, FP32_LANES = 152, 128
# DRAM bytes (read + write) of one bench launch of the stepper kernel (4096
# ions), from the one-pass ncu capture of that launch (dram__bytes_read.sum
# 680,192 B + dram__bytes_write.sum 0 B; the Tersoff summary under profiles/
# gives the command).  None once the kernel changes.
TRAFFIC_PER_LAUNCH = 680192


def _ion_name(w):
    return {5.0: "B-11", 33.0: "As-75", 18.0: "Ar-40", 92.0: "U-235", 36.0: "Kr"}.get(w["ion"]["Z"],
                                                                                    "Z=%g" % w["ion"]["Z"])


def _target_name(w):
    if w["lattice"] == "diamond":
        base = "Si(100)"
    else:
        base = "%s fluorite" % ("UO2" if w["species"][0]["Z"] == 92.0 else "CeO2")
    if w.get("target") == "bulk":
        base += " (bulk, on-lattice recoils)"
    temp = "300 K sigma %.3f A" % w["sigma"] if w["sigma"] > 0 else "0 K"
    model = {"none": "ZBL ion-target only", "tersoff": "Tersoff+ZBL", "buckingham": "Buckingham+ZBL"}[w["tt"]]
    return "%s %s, %s" % (base, temp, model)


def _window_atoms(w):
    return w["n"] ** 3 * (8 if w["lattice"] == "diamond" else 12)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _ks(a, b):
    from scipy import stats
    if len(a) < 2 or len(b) < 2:
        return None
    return float(stats.ks_2samp(a, b).pvalue)


def cpu_baseline(w, n_ions, threads, step_cap):
    """The oracle on the host cores on a bounded sample (n_ions primaries, at
    most step_cap steps each); ion-steps/s."""
    from oracle import oracle as O
    p = O.params(dict(w, step_cap=step_cap))
    t0 = time.perf_counter()
    r = O.run(p, n_ions, seed=w["seed"], first_id=0, threads=threads, records=False)
    dt = time.perf_counter() - t0
    return r["steps"] / dt, r["steps"], dt


def _merge_stats(a, b):
    """Counters of two contexts' runs added (launch fields from the first)."""
    out = dict(a)
    for k, v in b.items():
        if k in ("threads_per_track", "ctas_per_sm", "grid", "smem_bytes", "kernel_ms"):
            continue
        if isinstance(v, list):
            out[k] = [x + y for x, y in zip(a[k], v)]
        elif isinstance(v, (int, float)):
            out[k] = a[k] + v
    return out


def _golden():
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    import make_range_goldens as G
    return G


def oracle_parity(w, forms):
    """Mean, straggle and two-sample KS p of the range profile of each GPU
    form against the oracle's ranges of the same workload, stored by
    tests/golden/make_range_goldens.py, and the paired comparison on the
    primaries both sides ran (the GPU forms run the oracle's primaries: the
    same seed and ids, so the same launch draws).  forms: {name: records}."""
    try:
        G = _golden()
        ids, z, st, _ = G.read(w["name"])
    except (ImportError, OSError) as e:
        return {"workload": w["name"], "unavailable": "no stored oracle ranges (%s)" % e}
    ids, z, st = np.asarray(ids), np.asarray(z), np.asarray(st)
    zo = z[st == 1]
    out = {"workload": w["name"], "oracle_ions": len(ids), "oracle_mean_A": float(np.mean(zo)),
           "oracle_straggle_A": float(np.std(zo)), "source": "tests/golden/ranges_%s.txt (FP64 C oracle)" % w["name"]}
    for name, rec in forms.items():
        zg = rec["z"][rec["status"] == 1]
        if len(zg) < 2:
            continue
        res = {"ions": len(rec), "mean_rel_err": float(np.mean(zg) / np.mean(zo) - 1),
               "straggle_rel_err": float(np.std(zg) / np.std(zo) - 1), "ks_p": _ks(zg, zo),
               # sampling errors as for independent samples (an upper bound here)
               "mean_rel_se": float(np.hypot(_se_mean(zg), _se_mean(zo))),
               "straggle_rel_se": float(np.hypot(_se_std(zg), _se_std(zo)))}
        # paired: the same primary on both sides, both stopped
        r = rec[np.argsort(rec["id"])]
        k = r["id"] < len(ids)
        r = r[k]
        both = (r["status"] == 1) & (st[r["id"]] == 1)
        if both.sum() > 2:
            a, b = r["z"][both], z[r["id"][both]]
            d = a - b
            res["paired"] = {"primaries": int(both.sum()), "mean_rel_err": float(d.mean() / b.mean()),
                             "mean_rel_se": float(d.std(ddof=1) / np.sqrt(len(d)) / b.mean()),
                             "correlation": float(np.corrcoef(a, b)[0, 1])}
        out[name] = res
    return out


def _se_mean(z):
    return np.std(z) / np.sqrt(len(z)) / np.mean(z)


def _se_std(z):
    # relative standard error of the sample standard deviation: sqrt((kurtosis - 1) / (4 n))
    d = z - np.mean(z)
    kurt = np.mean(d ** 4) / np.mean(d ** 2) ** 2
    return np.sqrt(max(kurt - 1.0, 0.0) / (4 * len(z)))


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_0810_4737_gb300.workloads import workload
    w = workload(args.workload)
    threads = os.cpu_count() or 1
    n = args.ref_ions or threads
    for _ in range(args.warmup):
        cpu_baseline(w, n, threads, 50)
    vals, steps_tot, t_tot = [], 0, 0.0
    for _ in range(args.steps):
        v, st, dt = cpu_baseline(w, n, threads, args.cpu_steps)
        vals.append(v)
        steps_tot += st
        t_tot += dt
    value = steps_tot / t_tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ion-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "ions_per_step": n, "ion": _ion_name(w), "energy_eV": w["energy"],
                       "target": _target_name(w), "window_atoms": _window_atoms(w),
                       "sample": "%d primaries x first %d steps per step" % (n, args.cpu_steps)},
            "cpu_baseline": {"value": value, "unit": "ion-steps/s", "cores": threads, "kind": "oracle",
                             "sample": "%d primaries of %s, first %d steps each, per step; FP64 C oracle, OpenMP"
                                       % (n, w["name"], args.cpu_steps)},
            "e2e": {"value": value, "unit": "ion-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--ions", type=int, default=0, help="primaries per step per GPU (0: the workload's)")
    ap.add_argument("--fp64-ions", type=int, default=-1,
                    help="primaries of the plain FP64 path (-1: the whole batch of a step, 0: skip)")
    ap.add_argument("--cpu-ions", type=int, default=0, help="oracle sample primaries (0: one per host core)")
    ap.add_argument("--cpu-steps", type=int, default=1200, help="oracle sample: steps per primary")
    ap.add_argument("--ref-ions", type=int, default=0, help="reference arm primaries per step (0: one per core)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--threads", type=int, default=0, help="threads per track (0: autotune)")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="CTAs per SM (0: autotune)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_0810_4737_gb300 import build, reed as R
    from paper_0810_4737_gb300.workloads import workload
    if rank == 0 or ws == 1:
        build.build()
    if ws > 1:
        dist.barrier()
    w = workload(args.workload)
    n = args.ions or w["n_ions"]
    stream = torch.cuda.Stream()   # (pool streams: they do not synchronise with each other)
    sh = ctypes_stream(stream)
    # consecutive batches alternate between two contexts and streams, each
    # driven by its own host thread (reed_run blocks its caller): a batch's
    # launch takes the SMs its predecessor's last tracks leave idle
    stream2 = torch.cuda.Stream()
    sh2 = ctypes_stream(stream2)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 129 MB L2

    ctx = R.Reed(w)
    ctx2 = R.Reed(w)
    lanes = [(ctx, stream, sh), (ctx2, stream2, sh2)]
    first = rank * 10_000_000
    # launch configuration: given, or timed trials of every candidate (not part of a step)
    tune = []
    launch = dict(threads=args.threads, ctas_per_sm=args.ctas_per_sm)
    if not (args.threads and args.ctas_per_sm):
        tune = ctx.autotune(n_trial=2 * 152 * 2, seed=w["seed"] + 1, step_cap=1500, stream=None)
        best = max(tune, key=lambda t: t[2])
        launch = dict(threads=best[0], ctas_per_sm=best[1])

    def batch(lane, step_idx):
        c, s, h = lanes[lane]
        c.run(n_ions=n, seed=w["seed"], first_id=first + step_idx * n, record=False, stream=h, **launch)

    def pipelined(steps, first_step, work):
        errs = []

        def lane_work(lane):
            try:
                for i in range(lane, steps, 2):
                    work(lane, first_step + i)
            except Exception as e:   # re-raised below
                errs.append(e)
        th = [threading.Thread(target=lane_work, args=(k,)) for k in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        if errs:
            raise errs[0]

    for i in range(args.warmup):
        batch(0, i)
    torch.cuda.synchronize()
    ctx.reset()
    # measured throughput of the units that bound the stepper (roofline denominators)
    peaks = R.reed_peaks() if rank == 0 else None
    # ---- timed region: K batches one after another on one stream and
    # context, each after an L2 flush, device-timed with CUDA events on the
    # launch stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    kernel_ms = []
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()                     # L2 flush between timed steps (outside the events)
        ev[i][0].record(stream)
        batch(0, args.warmup + i)
        ev[i][1].record(stream)
        kernel_ms.append(ctx.stats()["kernel_ms"])
    torch.cuda.synchronize()
    clk = clocks.stop()
    if ws > 1:
        dist.barrier()
    tot_ms = sum(a.elapsed_time(b) for a, b in ev)
    st = ctx.stats()
    steps_done = st["steps"]
    # ---- the same number of batches streamed back to back over two contexts
    # (one host thread each): a batch's launch takes the SMs its
    # predecessor's last tracks leave idle.  Not the headline: overlapping
    # batches leave no point between them for an L2 flush.
    pipe = None
    if args.steps >= 2:
        ctx.reset()
        ctx2.reset()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            flush.zero_()
        p0.record(stream)
        stream2.wait_event(p0)
        pipelined(args.steps, args.warmup + args.steps, batch)
        p1[0].record(stream)
        p1[1].record(stream2)
        torch.cuda.synchronize()
        pipe_ms = max(p0.elapsed_time(e) for e in p1)
        pst = _merge_stats(ctx.stats(), ctx2.stats())
        pipe = {"value": pst["steps"] / (pipe_ms * 1e-3), "unit": "ion-steps/s", "ms_per_step": pipe_ms / args.steps,
                "batches": args.steps,
                "note": "the same number of batches back to back over two contexts and streams, one host thread "
                        "each (reed_run blocks its caller); L2 flushed once before the first (overlapping batches "
                        "leave no point between them), device time from the first launch to the last end"}
    if ws > 1:
        t = torch.tensor([tot_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
        c = torch.tensor([steps_done], device="cuda", dtype=torch.float64)
        dist.all_reduce(c)
        steps_done = int(c.item())
    value = steps_done / (tot_ms * 1e-3)
    pairs_per_s = (st["pair_evals"] + st["bond_evals"]) * ws / (tot_ms * 1e-3)
    # roofline of the stepper kernel (FP32 ALU)
    flops = OPS_PAIR * st["pair_evals"] + OPS_MOVE * st["atom_updates"] + OPS_TRIPLET * st["triplets"]
    sfu_ops = SFU_PAIR * st["pair_evals"] + SFU_TRIPLET * st["triplets"]
    kern_s = sum(kernel_ms) * 1e-3
    achieved = flops / kern_s / 1e12
    derived = SMS * FP32_LANES * 2 * 2070e6 / 1e12
    # ---- end to end through the public API with host buffers
    e2e = None
    if rank == 0:
        import ctypes
        ctx.reset()
        nb = int(w["n_bins"])
        prof = torch.empty(nb + 3, dtype=torch.float64, pin_memory=True)   # the step's result, pinned host
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_steps = 0
        for i in range(args.steps):
            ctx.run(n_ions=n, seed=w["seed"], first_id=first + (100 + i) * n, record=False, stream=sh, **launch)
            ptr = prof.data_ptr()
            R._check(R.lib().reed_range_profile(ctx.ctx, ptr, nb, ptr + 8 * nb), ctx.ctx)   # device -> host
            e2e_steps = ctx.stats()["steps"]            # device -> host
        dt = time.perf_counter() - t0
        # inputs: the run's parameters (options, beam, counts: kernel arguments; the
        # method has no bulk input -- every atom is generated on the device)
        h2d = ctypes.sizeof(R.reed_run_opts) + 8 * 8
        d2h = 8 * (nb + 3) + ctypes.sizeof(R.reed_stats_t)
        e2e = {"value": e2e_steps / dt, "unit": "ion-steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "note": "reed_run + reed_range_profile (into pinned host memory) + reed_stats per step, host wall clock"}
    # ---- the plain FP64 path on a full batch, and the mixed form on the same
    # primaries: the oracle's stored ones (its seed, ids 0..m-1), so that both
    # profiles can also be paired with the oracle's track by track
    fp64, forms = None, {}
    m = n if args.fp64_ions < 0 else args.fp64_ions
    if rank == 0 and m > 0:
        try:
            pseed = _golden().SEED
        except ImportError:
            pseed = w["seed"]
        with R.Reed(w) as c64, R.Reed(w) as c32:
            # (the FP64 path runs in the library's default launch shape)
            c64.run(n_ions=m, seed=pseed, first_id=0, precision=R.PREC_FP64, stream=sh)
            s64 = c64.stats()
            r64 = c64.records()
            c32.run(n_ions=m, seed=pseed, first_id=0, precision=R.PREC_MIXED, stream=sh, **launch)
            s32 = c32.stats()
            r32 = c32.records()
        z64 = r64["z"][r64["status"] == R.STOPPED]
        z32 = r32["z"][r32["status"] == R.STOPPED]
        forms = {"mixed": r32, "fp64": r64}
        f64ops = OPS_PAIR * s64["pair_evals"] + OPS_MOVE * s64["atom_updates"] + OPS_TRIPLET * s64["triplets"]
        a64 = f64ops / (s64["kernel_ms"] * 1e-3) / 1e12
        v64 = s64["steps"] / (s64["kernel_ms"] * 1e-3)
        v32 = s32["steps"] / (s32["kernel_ms"] * 1e-3)
        fp64 = {"value": v64, "unit": "ion-steps/s", "sample_ions": m,
                "sample": "%d primaries of the workload (the oracle's stored primaries 0..%d, seed %d)" % (m, m - 1, pseed),
                "roofline": {"bound": "fp64", "achieved": a64, "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                             "frac": a64 / peaks["fp64_tflops"], "peak_source": "measured FP64 FMA stream (reed_peaks)"},
                "launch": {"threads_per_track": s64["threads_per_track"], "ctas_per_sm": s64["ctas_per_sm"],
                           "grid": s64["grid"]},
                "mixed_same_sample": v32, "mixed_over_fp64": v32 / v64,
                "ks_p_mixed_vs_fp64": _ks(z32, z64),
                "mean_depth_A": [float(np.mean(z32)) if len(z32) else None, float(np.mean(z64)) if len(z64) else None]}
    # ---- per-profile error of both GPU forms against the oracle's stored
    # ranges of this workload
    parity = oracle_parity(w, forms) if rank == 0 and forms else None
    # ---- CPU oracle on the host cores (bounded sample)
    cpu = None
    if rank == 0 and not args.no_cpu:
        threads = os.cpu_count() or 1
        ci = args.cpu_ions or threads
        v, stp, dt = cpu_baseline(w, ci, threads, args.cpu_steps)
        v1, stp1, dt1 = cpu_baseline(w, 1, 1, args.cpu_steps // 2)
        cpu = {"value": v, "unit": "ion-steps/s", "cores": threads, "kind": "oracle",
               "sample": "%d primaries of %s, first %d steps each (%d ion-steps, %.1f s); FP64 C oracle, OpenMP"
                         % (ci, w["name"], args.cpu_steps, stp, dt),
               "one_thread": {"value": v1, "sample": "1 primary, first %d steps (%.1f s)" % (stp1, dt1)}}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "ion-steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["name"], "ions_per_step_per_gpu": n, "ion": _ion_name(w), "energy_eV": w["energy"],
                       "target": _target_name(w), "window_atoms": _window_atoms(w),
                       "parallelism": "replicas (independent primaries per GPU)",
                       "l2": "flushed between timed steps (256 MB write)",
                       "precision": "FP32 forces/atoms, FP64 ion position/time/energy accumulation"},
            "pair_forces_per_s": pairs_per_s,
            "autotune": [{"threads_per_track": t, "ctas_per_sm": c, "ion_steps_per_s": v} for t, c, v in tune],
            "gpu_launches": args.steps,
            "clocks": clk,
            "sfu": {"achieved_gops": sfu_ops / kern_s / 1e9, "peak_gops": peaks["ex2_gops"],
                    "frac": sfu_ops / kern_s / 1e9 / peaks["ex2_gops"],
                    "peak_source": "measured ex2.approx stream (reed_peaks)",
                    "units": "algorithmic: 5 per ion-target pair (4 ex2 + rsqrt), 1 per Tersoff bond-angle term"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s",
                         "frac": achieved / peaks["fp32_tflops"], "traffic": TRAFFIC_PER_LAUNCH if w["name"] == WORKLOAD and n == 4096 else None,
                         "peak_source": "measured FP32 FMA stream (reed_peaks, burst) at %.0f MHz; derived "
                                        "152 SM x 128 lanes x 2 x 2070 MHz = %.1f" % (peaks["sm_mhz"], derived),
                         "kernel": "reed_track_kernel<float, %s>" % w["tt"].upper(),
                         "kernel_ms_per_launch": sum(kernel_ms) / len(kernel_ms)},
            "pipelined": pipe,
            "peaks": peaks,
            "fp64_path": fp64,
            "oracle_parity": parity,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "stats": {k: st[k] for k in ("primaries", "tracks", "steps", "pair_evals", "bond_evals", "triplets",
                                         "atom_updates", "shifts", "rebuilds", "list_refreshes", "nb_overflow", "bond_cap_overflow", "nb_spilled",
                                         "threads_per_track", "ctas_per_sm", "grid", "smem_bytes", "phase_cycles",
                                         "centre_class")},
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    ctx2.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def ctypes_stream(stream):
    """cudaStream_t handle of a torch stream, for the C ABI."""
    return int(stream.cuda_stream) or None


if __name__ == "__main__":
    sys.exit(main())
