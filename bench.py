#!/usr/bin/env python
"""Benchmark of the MGARD+ hot path on GB300.

One step = one pass of the whole path over the 513^3 FP32 k^-5/3 Gaussian
random field (540 MB, larger than the 129 MB L2, so no flush is needed):
value range -> decomposition to the 3^3 coarsest level (L = 8) ->
level-wise quantization -> dequantization -> recomposition, at an L-inf bound
cycling through {1e-2, 1e-3, 1e-4, 1e-5} x range.  `value` is field bytes per
step time (GB/s) with the field resident in HBM; `dec_rec_gbs` is field
bytes / (decompose + recompose time) alone; `e2e` is the same step through the
host-buffer C entry points (mgard_compress_host_packed /
mgard_decompress_host_packed: the labels cross the link as their packed
lossless stream) with the copies inside the timed region; `quality` gives the
compression ratio, bits per value and PSNR of that stream per bound.  Inside the timed region only the
dominant kernel's launches carry timing events (its `roofline` figures come
from them); the per-kernel and per-phase split comes from passes outside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun, one rank per GPU) every rank runs its own field:
single fields do not shard, so ranks are independent replicas and `value`
is the bytes of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("decompose+recompose GB/s and % HBM roofline (FP32 vs FP64 GPU, at stated "
          "L∞ bound)")
DIMS = (513, 513, 513)
BOUNDS = (1e-2, 1e-3, 1e-4, 1e-5)
FALLBACK_HBM = 6800.0
QUANT_KERNELS = ("quantize_kernel", "dequantize_kernel", "minmax_partial_kernel")


# The paper's own figures with the hardware it names (Section 6; one core of
# a 2x8-core Xeon E5-2650 node of the Rhea cluster, FP32): context only, not
# a target and not comparable to this GPU's throughput.
PAPER_CONTEXT = {
    "hardware": "Rhea cluster node, 2x8-core Intel Xeon E5-2650, 128 GB (CPU, per core)",
    "decomposition_speedup_vs_mgard": {"Hurricane": 20, "NYX": 28, "SCALE-LETKF": 39, "QMCPACK": 71},
    "recomposition_speedup_vs_mgard": {"Hurricane": 22, "NYX": 30, "SCALE-LETKF": 41, "QMCPACK": 80},
    "whole_compressor_mb_per_s_at_psnr_60": {"Hurricane": 96.03, "NYX": 94.23, "SCALE-LETKF": 104.82,
                                             "QMCPACK": 100.30},
    "note": "Fig. 7 and Table 5 of the paper; another machine and a wider pipeline (SZ and a "
            "lossless back end included in the whole-compressor figure)",
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="single", choices=["single", "batched", "serving"],
                    help="single: the 513^3 field (default); batched: 256 uneven fields; "
                         "serving: a Poisson request stream")
    ap.add_argument("--serving-requests", type=int, default=2000, help=argparse.SUPPRESS)
    ap.add_argument("--case-dims", default="513x513x513",
                    help="field shape of --kernel-case, e.g. 513x513x257 or 288x115x69x69")
    ap.add_argument("--batch-count", type=int, default=256, help=argparse.SUPPRESS)
    ap.add_argument("--kernel-case", action="store_true",
                    help="only one compression round trip of a --case-dims FP32 field, 3D or "
                         "4D (for ncu captures)")
    ap.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-reps", type=int, default=3, help=argparse.SUPPRESS)
    return ap.parse_args()


def config_dict():
    return {
        "workload": "513^3 FP32 k^-5/3 Gaussian random field, full depth (L=8, 3^3 coarsest), "
                    "range+decompose+quantize+dequantize+recompose per step",
        "dims": list(DIMS),
        "bounds_rel": list(BOUNDS),
        "stop_level": 0,
        "l2": "inputs larger than L2 (540 MB field, 1.08 GB labels); no flush",
        "parallelism": "replicas (one independent field per GPU)",
    }


# ------------------------------------------------------------ oracle leg ---

def oracle_sample(n: int, reps: int):
    """Time the FP64 oracle (as it stands) on an n^3 sample of the same
    workload: range, decompose, quantize, dequantize, recompose."""
    import numpy as np
    from oracle import mgard_oracle as O
    from paper_2010_05872_gb300 import fields as F
    u = F.grf_field((n, n, n), seed=F.SEED_LARGE)
    H = O.Hierarchy(u.shape)
    O.level_tolerances(H, 0, 1.0)  # warms the tables
    times = []
    for i in range(reps):
        rel = BOUNDS[i % len(BOUNDS)]
        t0 = time.perf_counter()
        tau = rel * O.value_range(u)
        taus = O.level_tolerances(H, 0, tau)
        umc = O.decompose(u, H, 0)
        k = O.quantize(umc, H, 0, taus)
        rec = O.recompose(O.dequantize(k, H, 0, taus, dtype=np.float32).astype(np.float64), H, 0)
        times.append(time.perf_counter() - t0)
        assert np.abs(rec - u).max() <= tau
    return u.nbytes, times


def oracle_parity(cases):
    """The FP32 (or FP64) GPU results of the benchmarked configurations
    against the FP64 oracle, after every timed region: per case, the
    decomposition's max error relative to max|u|, and per bound the GPU
    recomposition of the bound's dequantized labels against the oracle's
    recomposition of the same labels (relative to max|u| and to tau).  Each
    case: {"name", "u" (host field), "coords", "stop", "coeffs" (GPU
    decomposition), "bounds": {rel: (tau, dequantized labels, GPU
    reconstruction)}}."""
    import numpy as np
    from oracle import mgard_oracle as O
    out = {}
    for c in cases:
        u = c["u"].astype(np.float64)
        H = O.Hierarchy(u.shape, c["coords"])
        scale = float(np.abs(u).max())
        t0 = time.perf_counter()
        exp = O.decompose(u, H, c["stop"])
        res = {"decompose_rel": float(np.abs(c["coeffs"].astype(np.float64) - exp).max()) / scale}
        del exp
        per = {}
        for rel, (tau, deq, rec) in c["bounds"].items():
            rec_o = O.recompose(deq.astype(np.float64), H, c["stop"])
            d = float(np.abs(rec.astype(np.float64) - rec_o).max())
            per[f"{rel:g}"] = {"recompose_same_labels_rel": d / scale,
                               "recompose_same_labels_over_tau": d / tau,
                               "linf_over_tau": float(np.abs(rec.astype(np.float64) - u).max()) / tau}
        res["bounds"] = per
        res["oracle_seconds"] = time.perf_counter() - t0
        out[c["name"]] = res
    return out


def cpu_baseline_subprocess(n: int, reps: int):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    res = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", str(n),
                          "--oracle-reps", str(reps)], capture_output=True, text=True, env=env,
                         timeout=900)
    if res.returncode != 0:
        return {"value": None, "error": res.stderr[-400:]}
    return json.loads(res.stdout.strip().splitlines()[-1])


def cpu_baseline_all_cores(n: int, procs: int):
    """The same oracle sample in `procs` concurrent single-thread processes
    (one per host core): aggregate GB/s = the processes' bytes over the
    longest process's timed seconds."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", str(n), "--oracle-reps", "1"]
    ps = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
          for _ in range(procs)]
    outs = []
    for p in ps:
        out, err = p.communicate(timeout=900)
        if p.returncode != 0:
            return {"value": None, "error": err[-400:]}
        outs.append(json.loads(out.strip().splitlines()[-1]))
    longest = max(o["seconds"] for o in outs)
    nbytes = sum(o["value"] * o["seconds"] * 1e9 for o in outs)
    return {"value": nbytes / longest / 1e9, "unit": "GB/s", "cores": procs, "kind": "oracle",
            "seconds": longest,
            "sample": f"{procs} concurrent single-thread processes, each one {n}^3 FP32 k^-5/3 "
                      f"field (same recipe as the 513^3 workload), full depth, range+decompose+"
                      f"quantize+dequantize+recompose in FP64; bytes of all over the longest "
                      f"process's time"}


def run_oracle_sample_cli(args):
    nbytes, times = oracle_sample(args.oracle_sample, args.oracle_reps)
    total = sum(times)
    print(json.dumps({"value": nbytes * len(times) / total / 1e9, "unit": "GB/s", "cores": 1,
                      "kind": "oracle", "seconds": total,
                      "sample": f"{args.oracle_sample}^3 FP32 k^-5/3 field (same recipe as the "
                                f"513^3 workload), full depth, range+decompose+quantize+"
                                f"dequantize+recompose in FP64, {len(times)} reps, 1 thread"}))


def run_reference(args, rank):
    """The oracle on the host cores as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    # Calibrate on a small sample, then size the per-step sample so that
    # warmup + steps finish within about two minutes.
    _, t = oracle_sample(33, 1)
    per_node = t[0] / 33 ** 3
    n = 33
    for cand in (65, 129, 257):
        if per_node * cand ** 3 * (args.steps + args.warmup) <= 120.0:
            n = cand
    nbytes, times = oracle_sample(n, args.warmup + args.steps)
    timed = times[args.warmup:]
    total = sum(timed)
    value = nbytes * len(timed) / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(timed), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(),
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"{n}^3 FP32 k^-5/3 field per step (the 513^3 workload's "
                                   f"recipe at a size one host core runs in seconds), full depth, "
                                   f"range+decompose+quantize+dequantize+recompose in FP64"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------- clocks ---

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(device_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append((time.perf_counter(), parts))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        inside = [p for (t, p) in self.samples if t0 <= t <= t1]
        used = inside if len(inside) >= 3 else [p for (_, p) in self.samples]
        if not used:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(p[0]) for p in used if num(p[0]) is not None]
        mx = [num(p[1]) for p in used if num(p[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in used for i in range(4) if p[4 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(used), "samples_in_timed_region": len(inside),
                "power_w_max": max((num(p[2]) or 0.0) for p in used)}


# ------------------------------------------------------------- GPU leg ---

def src_hash(source=None):
    """Hash of the kernel sources: every file under csrc/, or, given one
    translation unit, that file and the local headers it includes."""
    csrc = os.path.join(ROOT, "paper_2010_05872_gb300", "csrc")
    if source is None:
        files = sorted(glob.glob(os.path.join(csrc, "*")))
    else:
        seen, todo = set(), [source]
        while todo:
            name = todo.pop()
            if name in seen or not os.path.exists(os.path.join(csrc, name)):
                continue
            seen.add(name)
            with open(os.path.join(csrc, name)) as fh:
                todo += re.findall(r'^\s*#include\s+"([^"]+)"', fh.read(), re.M)
        files = [os.path.join(csrc, n) for n in sorted(seen)]
    h = hashlib.sha256()
    for f in files:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM, "fallback"


def traffic_for(kernel, level):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rows = json.load(fh)
    except (OSError, ValueError):
        return None
    for r in rows:
        if (r.get("kernel") == kernel and r.get("level") == level
                and r.get("src_hash") == src_hash(r.get("source"))):
            return r.get("dram_bytes_per_launch")
    return None


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2010_05872_gb300 import binding as B
    from paper_2010_05872_gb300 import build as build_mod
    from paper_2010_05872_gb300 import fields as F

    torch.cuda.set_device(local_rank)
    build_mod.build()
    B.lib()
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()

    u_host = F.grf_field(DIMS, seed=F.SEED_LARGE + rank)
    nbytes = u_host.nbytes
    u = torch.from_numpy(u_host).to(dev)
    x = u.clone()
    ws = B.workspace(DIMS, torch.float32, dev)
    labels = torch.empty(DIMS, dtype=torch.int64, device=dev)

    # A step waits on nothing: the range stays on the device, where the
    # quantizer forms tau = rel x (max - min) and its level tolerances (the
    # same values as the host's), and the labels' flags are read once per
    # batch of steps (quantize_status after each loop below).
    rng = torch.empty(2, dtype=torch.float64, device=dev)
    lo_u, hi_u = B.value_range(u)

    def step(buf, rel, ev=None):
        if ev:
            ev[0].record(stream)
        B.value_range_async(buf, rng)
        if ev:
            ev[1].record(stream)
        B.decompose(buf, None, 0, ws)
        if ev:
            ev[2].record(stream)
        B.quantize_rel_async(buf, rel, rng, None, 0, labels)
        if ev:
            ev[3].record(stream)
        B.dequantize_rel(labels, rel, rng, buf.dtype, None, 0, out=buf)
        if ev:
            ev[4].record(stream)
        B.recompose(buf, None, 0, ws)
        if ev:
            ev[5].record(stream)
        return rel * (hi_u - lo_u)  # the tau the device formed (the input's range)

    # Correctness of the timed configuration: L-inf error per bound.
    linf = {}
    for rel in BOUNDS:
        x.copy_(u)
        tau = step(x, rel)
        B.quantize_status()
        err = (x.double() - u.double()).abs().max().item()
        linf[f"{rel:g}"] = err / tau
        assert err <= tau, (rel, err, tau)

    # The results the oracle leg compares with the FP64 oracle (after every
    # timed region): the decomposition and, per bound, the dequantized labels
    # and the reconstruction.
    want_parity = rank == 0 and world == 1 and not args.no_cpu_baseline
    parity_cases = []
    if want_parity:
        lo2, hi2 = B.value_range(u)
        x.copy_(u)
        B.decompose(x, None, 0, ws)
        c2 = {"name": "513cubed_fp32", "u": u_host, "coords": None, "stop": 0,
              "coeffs": x.cpu().numpy(), "bounds": {}}
        for rel in BOUNDS:
            tau = rel * (hi2 - lo2)
            x.copy_(u)
            B.decompose(x, None, 0, ws)
            B.quantize(x, tau, None, 0, labels)
            B.dequantize(labels, tau, x.dtype, None, 0, out=x)
            deq = x.cpu().numpy()
            B.recompose(x, None, 0, ws)
            c2["bounds"][rel] = (tau, deq, x.cpu().numpy())
        parity_cases.append(c2)
    x.copy_(u)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    clocks = ClockSampler(local_rank)
    for i in range(args.warmup):
        step(x, BOUNDS[i % 4])
    torch.cuda.synchronize()
    B.quantize_status()

    # Per-kernel breakdown, outside the timed region: every launch bracketed
    # by trace events (they cost about 2 us of device time per launch, which
    # is why the timed region brackets the dominant kernel alone).
    kb = max(8, min(args.steps, 40))
    B.mgard_trace_select(-1)
    B.mgard_trace_enable(True)
    for i in range(kb):
        step(x, BOUNDS[i % 4])
    torch.cuda.synchronize()
    B.quantize_status()
    B.mgard_trace_enable(False)
    trace = B.mgard_trace_read()
    # Phase split, also outside the timed region: six events per step, no trace.
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(kb)]
    for i in range(kb):
        step(x, BOUNDS[i % 4], evs[i])
    torch.cuda.synchronize()
    B.quantize_status()
    phase = {k: 0.0 for k in ("range", "decompose", "quantize", "dequantize", "recompose")}
    for e in evs:
        for j, k in enumerate(phase):
            phase[k] += e[j].elapsed_time(e[j + 1]) / kb
    # The metric is decompose + recompose: the roofline block describes the
    # transform kernel with the largest summed device time; the quantizer's
    # largest kernel is reported beside it.
    transform = [r for r in trace if r["kernel"] not in QUANT_KERNELS]
    top = max(transform, key=lambda r: r["total_ms"])
    qtop = max((r for r in trace if r["kernel"] in QUANT_KERNELS), key=lambda r: r["total_ms"])

    # Timed region: K steps; only the dominant kernel's launches bracketed.
    barrier()
    torch.cuda.synchronize()
    B.mgard_trace_select(top["kind"], top["level"])
    B.mgard_trace_enable(True)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")
    start.record(stream)
    for i in range(args.steps):
        step(x, BOUNDS[i % 4])
    end.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    B.quantize_status()
    B.mgard_trace_enable(False)
    launches = B.mgard_trace_kernel_launches()
    timed_top = [r for r in B.mgard_trace_read()
                 if r["kind"] == top["kind"] and r["level"] == top["level"]][0]
    B.mgard_trace_select(-1)
    barrier()
    torch.cuda.synchronize()
    clocks.stop()
    elapsed_ms = start.elapsed_time(end)

    if world > 1:
        t = torch.tensor([elapsed_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed_ms = t.item()
    ms_per_step = elapsed_ms / args.steps
    value = world * nbytes * args.steps / (elapsed_ms * 1e-3) / 1e9
    dec_rec_gbs = nbytes / ((phase["decompose"] + phase["recompose"]) * 1e-3) / 1e9

    # Dominant kernel (largest summed device time in the breakdown pass) and
    # its roofline, from its event-timed launches inside the timed region.
    peak, peak_src = measured_peak()
    tt = timed_top
    achieved = (tt["bytes"] / tt["launches"]) / (tt["total_ms"] / tt["launches"] * 1e-3) / 1e9
    total_kernel_ms = sum(r["total_ms"] for r in trace)
    # Whole-path roofline on the path's algorithmic byte count
    # B_alg = 2 (decompose + recompose) x 2 s sum_{l > l~} #N_l.
    b_alg = path_bytes(DIMS, 0, 4)
    dec_rec_ms = phase["decompose"] + phase["recompose"]
    path_frac = b_alg / (dec_rec_ms * 1e-3) / 1e9 / peak
    # The same against the nominal HBM3e bandwidth (7.9 TB/s), as a second column.
    path_frac_nominal = b_alg / (dec_rec_ms * 1e-3) / 1e9 / 7900.0
    roofline = {
        "bound": "hbm", "kernel": top["kernel"], "level": top["level"],
        "achieved": achieved, "peak": peak, "peak_source": f"{peak_src} HBM copy bandwidth",
        "unit": "GB/s", "frac": achieved / peak,
        "traffic": traffic_for(top["kernel"], top["level"]),
        "alg_bytes_per_launch": tt["bytes"] / tt["launches"],
        "avg_launch_ms": tt["total_ms"] / tt["launches"],
        "launches_timed": tt["launches"],
        "share_of_kernel_time": top["total_ms"] / total_kernel_ms,
        "path": {"what": "decompose + recompose of the 513^3 FP32 field (the metric's path)",
                 "alg_bytes": b_alg, "ms": dec_rec_ms, "achieved": b_alg / (dec_rec_ms * 1e-3) / 1e9,
                 "frac": path_frac},
        "quantizer_top": {"kernel": qtop["kernel"], "level": qtop["level"],
                          "achieved": qtop["bytes"] / (qtop["total_ms"] * 1e-3) / 1e9,
                          "frac": qtop["bytes"] / (qtop["total_ms"] * 1e-3) / 1e9 / peak,
                          "traffic": traffic_for(qtop["kernel"], qtop["level"]),
                          "source": "breakdown pass (every launch event-timed)"},
    }

    kinds = {}
    for r in trace:
        kinds[r["kernel"]] = kinds.get(r["kernel"], 0.0) + r["total_ms"] / kb
    all_kernels = sorted(({"kernel": r["kernel"], "level": r["level"], "launches": r["launches"],
                           "ms_per_step": r["total_ms"] / kb,
                           "gbs": r["bytes"] / (r["total_ms"] * 1e-3) / 1e9} for r in trace),
                         key=lambda d: -d["ms_per_step"])
    kernels = all_kernels[:12]
    # The whole breakdown, one row per (kernel, level), on stderr.
    for d in all_kernels:
        print(f"# {d['kernel']:26s} L{d['level']:3d} launches/step {d['launches'] / kb:5.2f} "
              f"{d['ms_per_step'] * 1e3:8.1f} us/step {d['gbs']:7.0f} GB/s", file=sys.stderr)

    # Plain FP64 GPU path on the same input.
    del labels
    x64 = u.double()
    u64 = x64.clone()
    labels = torch.empty(DIMS, dtype=torch.int64, device=dev)
    ws = B.workspace(DIMS, torch.float64, dev)
    k64 = max(3, args.steps // 40)
    for i in range(2):
        step(x64, BOUNDS[i])
    ev64 = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(k64)]
    torch.cuda.synchronize()
    for i in range(k64):
        step(x64, BOUNDS[i % 4], ev64[i])
    torch.cuda.synchronize()
    B.quantize_status()
    ph64 = {k: sum(e[j].elapsed_time(e[j + 1]) for e in ev64) for j, k in enumerate(phase)}
    t64 = sum(ph64.values()) / k64
    x64.copy_(u64)
    tau64 = step(x64, 1e-3)
    B.quantize_status()
    # The FP64 path against both roofs: HBM on its own bytes (8 B per value)
    # and the measured FP64 FMA rate on the path's algorithmic flops.
    dr64 = (ph64["decompose"] + ph64["recompose"]) / k64
    dfma = B.mgard_trace_fma_rate(B.F64)
    flops = path_flops(DIMS, 0)
    b64 = path_bytes(DIMS, 0, 8)
    t_hbm, t_alu = b64 / (peak * 1e9), flops / dfma
    fp64 = {
        "ms_per_step": t64, "value_gbs_f32_bytes": nbytes / (t64 * 1e-3) / 1e9,
        "value_gbs_own_bytes": 2 * nbytes / (t64 * 1e-3) / 1e9,
        "dec_rec_ms": dr64,
        "dec_rec_gbs": nbytes / (dr64 * 1e-3) / 1e9,
        "linf_over_tau_1e-3": (x64 - u64).abs().max().item() / tau64,
        "steps": k64,
        "roofline": {
            **({"bound": "alu", "achieved": flops / (dr64 * 1e-3) / 1e12, "peak": dfma / 1e12,
                "unit": "TFLOP/s", "frac": t_alu / (dr64 * 1e-3)} if t_alu > t_hbm else
               {"bound": "hbm", "achieved": b64 / (dr64 * 1e-3) / 1e9, "peak": peak,
                "unit": "GB/s", "frac": t_hbm / (dr64 * 1e-3)}),
            "alg_flops": flops, "alg_bytes": b64,
            "fp64_fma_peak_tflops": dfma / 1e12,
            "fp32_fma_peak_tflops": B.mgard_trace_fma_rate(B.F32) / 1e12,
            "roof_ms": {"hbm": t_hbm * 1e3, "fp64_fma": t_alu * 1e3},
            "hbm_frac": t_hbm / (dr64 * 1e-3),
            "note": ("decompose + recompose of the 513^3 field in FP64; FMA peaks measured live "
                     "(mgard_trace_fma_rate: independent dependent-FMA chains, best of 3); flops "
                     "counted per level from the method's steps (bench.path_flops)"),
        },
    }
    del x64, u64, labels

    # The other single-field configurations: 500x500x100 FP32 with geometric
    # z (stopping levels 3 and 0) and 65^3 FP64 (full depth), each timed
    # (median of untimed-region runs) with its L-inf check at 1e-3 x range.
    nonuniform = {}
    dims3 = (500, 500, 100)
    coords3 = [F.uniform_coords(500), F.uniform_coords(500), F.geometric_coords(100, 1.03)]
    u3h = F.front_field(dims3, coords3)
    for stop3 in (3, 0):
        r3, c3 = measure_config(B, torch, stream, u3h, coords3, stop3, reps=10,
                                keep=want_parity)
        r3["path_roofline_frac_dec_rec"] = (path_bytes(dims3, stop3, 4) /
                                            ((r3["decompose_ms"] + r3["recompose_ms"]) * 1e-3)
                                            / 1e9 / peak)
        r3["alg_bytes"] = path_bytes(dims3, stop3, 4)
        nonuniform[f"stop{stop3}"] = r3
        if c3:
            c3["name"] = f"500x500x100_fp32_stop{stop3}"
            parity_cases.append(c3)
    nonuniform["note"] = ("500x500x100 FP32, x/y uniform, z geometric (ratio 1.03), sinusoids + "
                          "tanh front; stands in for the paper's Hurricane shape; median of 10 "
                          "runs per direction; path fraction on 2 x 2 s sum_{l>l~} #N_l of "
                          "measured HBM")
    u1h = F.sinusoid_field((65, 65, 65), seed=F.SEED_TINY)
    tiny, c1 = measure_config(B, torch, stream, u1h, None, 0, reps=20, keep=want_parity)
    tiny["note"] = ("65^3 FP64 sinusoids + noise, full depth (L=5); latency-bound, so reported "
                    "as time: decompose + quantize + dequantize + recompose")
    if c1:
        c1["name"] = "65cubed_fp64"
        parity_cases.append(c1)

    # Adaptive stopping level (Algorithm 1): the level chosen per bound, and
    # at 1e-3 x range the time of the adaptive decomposition against the
    # plain one at that level and the sampled-error kernels' share.
    ws = B.workspace(DIMS, torch.float32, dev)
    rng_lo, rng_hi = B.value_range(u)
    adaptive = {"stop_level": {}}
    for rel in BOUNDS:
        x.copy_(u)
        stop_a, _ = B.decompose_adaptive(x, rel * (rng_hi - rng_lo), None, ws)
        adaptive["stop_level"][f"{rel:g}"] = stop_a
    tau_a = 1e-3 * (rng_hi - rng_lo)
    ka = max(3, min(args.steps // 40, 10))
    t_ad, t_pl = [], []
    for i in range(ka):
        x.copy_(u)
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        stop_a, sums_a = B.decompose_adaptive(x, tau_a, None, ws)
        eb.record(stream)
        torch.cuda.synchronize()
        t_ad.append(ea.elapsed_time(eb))
    # The sampling kernels' own time, from a traced run of the same calls.
    B.mgard_trace_select(-1)
    B.mgard_trace_enable(True)
    for i in range(ka):
        x.copy_(u)
        B.decompose_adaptive(x, tau_a, None, ws)
    torch.cuda.synchronize()
    B.mgard_trace_enable(False)
    pe = [r for r in B.mgard_trace_read() if r["kernel"] == "prediction_errors_kernel"]
    for i in range(ka):
        x.copy_(u)
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        B.decompose(x, None, stop_a, ws)
        eb.record(stream)
        torch.cuda.synchronize()
        t_pl.append(ea.elapsed_time(eb))
    adaptive.update({
        "bound_rel": 1e-3, "stop": stop_a,
        "adaptive_ms": statistics.median(t_ad), "plain_at_stop_ms": statistics.median(t_pl),
        "sampling_ms": sum(r["total_ms"] for r in pe) / ka,
        "sampling_ms_by_level": {str(r["level"]): r["total_ms"] / ka for r in pe},
        "sampled_levels": int(sum(r["launches"] for r in pe) / ka),
        "note": ("median of %d untraced runs each; sampling_ms from traced runs (event pairs "
                 "inflate the small levels); the adaptive call waits on the host once per level "
                 "above 2e7 nodes and once for all smaller levels" % ka),
    })
    x.copy_(u)

    # Progressive recomposition and analysis on reduced representations
    # (the iso-surface use case): Q_k u for k = L .. L-3 from the decomposed
    # field, and the iso-surface area at the field's mean on each.
    B.decompose(x, None, 0, ws)
    torch.cuda.synchronize()
    iso = float(u.double().mean().item())
    n_lv = B.mgard_num_levels(DIMS)
    progressive = {"iso": "mean", "levels": {}}
    area_full = None
    for k in range(n_lv, n_lv - 4, -1):
        _, axes = B.level_grid(DIMS, None, k)
        tr, ti = [], []
        for i in range(3):
            ea, eb, ec = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            ea.record(stream)
            qk = B.recompose_partial(x, k, None, 0, ws)
            eb.record(stream)
            area = B.iso_area(qk, iso, axes)
            ec.record(stream)
            torch.cuda.synchronize()
            tr.append(ea.elapsed_time(eb))
            ti.append(eb.elapsed_time(ec))
            del qk
        if area_full is None:
            area_full = area
        progressive["levels"][str(k)] = {
            "recompose_ms": statistics.median(tr), "iso_area_ms": statistics.median(ti),
            "area": area, "area_rel_diff_vs_full": area / area_full - 1.0}
    x.copy_(u)

    # 4D grids (QMCPACK's shape, 288 x 115 x 69 x 69 FP32): the time of
    # the decomposition and recomposition, and one compressed round trip at
    # 1e-3 x range (labels packed for the rate).
    dims4 = (288, 115, 69, 69)
    u4 = F.grf_field_device(dims4, seed=F.SEED_LARGE + 4 + rank, device=dev)
    x4 = u4.clone()
    ws4 = B.workspace_4d(dims4, torch.float32, dev)
    nb4 = u4.numel() * 4
    B.decompose_4d(x4, None, 0, ws4)
    B.recompose_4d(x4, None, 0, ws4)
    t_d4, t_r4 = [], []
    for i in range(5):
        x4.copy_(u4)
        ea, eb, ec = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        ea.record(stream)
        B.decompose_4d(x4, None, 0, ws4)
        eb.record(stream)
        B.recompose_4d(x4, None, 0, ws4)
        ec.record(stream)
        torch.cuda.synchronize()
        t_d4.append(ea.elapsed_time(eb))
        t_r4.append(eb.elapsed_time(ec))
    md4, mr4 = statistics.median(t_d4), statistics.median(t_r4)
    lo4, hi4 = B.value_range(u4)
    tau4 = 1e-3 * (hi4 - lo4)
    x4.copy_(u4)
    B.decompose_4d(x4, None, 0, ws4)
    lab4, _ = B.quantize_4d(x4, tau4)
    pk4 = B.pack_labels(lab4)
    B.dequantize_4d(lab4, tau4, torch.float32, out=x4)
    B.recompose_4d(x4, None, 0, ws4)
    err4 = float((x4.double() - u4.double()).abs().max().item())
    peak4, _ = measured_peak()
    sizes4, n4 = [], list(dims4)
    while min(n4) > 3:
        sizes4.append(int(np.prod(n4)))
        n4 = [v // 2 + 1 for v in n4]
    b_alg4 = 2 * 2 * 4 * sum(sizes4)
    nd4 = {"dims": list(dims4), "levels": B.mgard_num_levels_4d(dims4),
           "decompose_ms": md4, "recompose_ms": mr4,
           "dec_rec_gbs": nb4 / ((md4 + mr4) * 1e-3) / 1e9,
           "path_roofline_frac_dec_rec": b_alg4 / ((md4 + mr4) * 1e-3) / 1e9 / peak4,
           "bits_per_value_1e-3": 8.0 * len(pk4) / u4.numel(),
           "linf_over_tau_1e-3": err4 / tau4,
           "note": ("median of 5 runs; dec_rec_gbs = field bytes / (decompose + recompose) as "
                    "for 1-3D; path fraction = one read and one write of every decomposed level "
                    "per transform over the time, of measured HBM; synthetic k^-5/3 Gaussian "
                    "random field")}
    del u4, x4, ws4, lab4, pk4

    # End to end through the host-buffer entry points: the packed path (the
    # labels' lossless stream crosses the link) is the headline, the int64
    # label path beside it.
    ws = B.workspace(DIMS, torch.float32, dev)
    labels = torch.empty(DIMS, dtype=torch.int64, device=dev)
    cnt = int(np.prod(DIMS))
    cap = B.pack_bound(cnt)
    d_stream = torch.empty(cap, dtype=torch.uint8, device=dev)
    h_field = torch.from_numpy(u_host).pin_memory()
    h_labels = torch.empty(DIMS, dtype=torch.int64).pin_memory()
    h_stream = torch.empty(cap, dtype=torch.uint8).pin_memory()
    h_out = torch.empty(DIMS, dtype=torch.float32).pin_memory()
    ke = max(3, args.steps // 40)
    sizes = {}

    # One lane = one field in flight: its stream and its device and pinned
    # host buffers (the input field is shared, read only).
    lane0 = (stream, x, labels, d_stream, ws, h_stream, h_out)

    def packed_round_trip(rel, lane):
        s_l, x_l, lab_l, ds_l, ws_l, hs_l, ho_l = lane
        rc, nb, tau = B.mgard_compress_host_packed(
            DIMS, None, B.F32, 0, rel, h_field.data_ptr(), hs_l.data_ptr(), cap,
            x_l.data_ptr(), lab_l.data_ptr(), ds_l.data_ptr(), cap, ws_l.data_ptr(),
            ws_l.numel(), s_l.cuda_stream)
        assert rc == 0, rc
        sizes[rel] = nb
        rc = B.mgard_decompress_host_packed(
            DIMS, None, B.F32, 0, tau, hs_l.data_ptr(), nb, ho_l.data_ptr(),
            x_l.data_ptr(), lab_l.data_ptr(), ds_l.data_ptr(), cap, ws_l.data_ptr(),
            ws_l.numel(), s_l.cuda_stream)
        assert rc == 0, rc
        return tau

    def e2e_step(rel, packed=True):
        if packed:
            return packed_round_trip(rel, lane0)
        rc, tau = B.mgard_compress_host(DIMS, None, B.F32, 0, rel, h_field.data_ptr(),
                                        h_labels.data_ptr(), x.data_ptr(), labels.data_ptr(),
                                        ws.data_ptr(), ws.numel(), stream.cuda_stream)
        assert rc == 0, rc
        rc = B.mgard_decompress_host(DIMS, None, B.F32, 0, tau, h_labels.data_ptr(),
                                     h_out.data_ptr(), x.data_ptr(), labels.data_ptr(),
                                     ws.data_ptr(), ws.numel(), stream.cuda_stream)
        assert rc == 0, rc
        return tau

    def timed_e2e(packed):
        e2e_step(1e-3, packed)
        torch.cuda.synchronize()
        barrier()
        es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        es.record(stream)
        for i in range(ke):
            e2e_step(BOUNDS[i % 4], packed)
        ee.record(stream)
        torch.cuda.synchronize()
        ms = es.elapsed_time(ee)
        if world > 1:
            t = torch.tensor([ms], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = t.item()
        return ms

    def timed_e2e_lanes(lanes, steps):
        """The packed round trip with len(lanes) fields in flight: lane q
        runs steps q, q + len(lanes), .. on a host thread of its own (the
        calls release the interpreter lock), so one field's upload overlaps
        another's download and device work.  Events on lane 0's stream
        bracket all of them (lane q's stream waits for the start event; lane
        0's stream waits for every lane's end)."""
        import threading
        for lane in lanes:
            packed_round_trip(1e-3, lane)
        torch.cuda.synchronize()
        barrier()
        es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        es.record(lanes[0][0])
        for lane in lanes[1:]:
            lane[0].wait_event(es)
        errors = []

        def run(q):
            try:
                for i in range(q, steps, len(lanes)):
                    packed_round_trip(BOUNDS[i % 4], lanes[q])
            except BaseException as exc:  # re-raised below
                errors.append(exc)

        threads = [threading.Thread(target=run, args=(q,)) for q in range(len(lanes))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        if errors:
            raise errors[0]
        for lane in lanes[1:]:
            done = torch.cuda.Event()
            done.record(lane[0])
            lanes[0][0].wait_event(done)
        ee.record(lanes[0][0])
        torch.cuda.synchronize()
        ms = es.elapsed_time(ee)
        if world > 1:
            t = torch.tensor([ms], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = t.item()
        return ms

    e2e_serial_ms = timed_e2e(True)
    stream_bytes = sum(sizes[BOUNDS[i % 4]] for i in range(ke)) / ke
    # Further fields in flight, each on its own stream and buffers (1, 2, 3
    # and 4 fields: 48, 76, 81 and 91 GB/s on GB300).
    lanes_in_flight = 4
    extra = [(torch.cuda.Stream(device=dev), torch.empty_like(x), torch.empty_like(labels),
              torch.empty_like(d_stream), torch.empty_like(ws),
              torch.empty(cap, dtype=torch.uint8).pin_memory(),
              torch.empty(DIMS, dtype=torch.float32).pin_memory())
             for _ in range(lanes_in_flight - 1)]
    ke2 = lanes_in_flight * max(ke, 6)  # enough steps per field to amortize filling the pipeline
    e2e_ms = timed_e2e_lanes([lane0] + extra, ke2) * ke / ke2
    del extra
    # Rate and distortion per bound (Section 6, "Quality"): compression
    # ratio and bits per value of the packed stream, PSNR and L-inf / tau of
    # the reconstruction.
    quality = {}
    u64 = u.double()
    rng_u = float((u64.max() - u64.min()).item())
    for rel in BOUNDS:
        tau = e2e_step(rel, True)
        rec = torch.from_numpy(h_out.numpy()).to(dev).double()
        mse = float(((rec - u64) ** 2).mean().item())
        quality[f"{rel:g}"] = {
            "compression_ratio": nbytes / sizes[rel], "bits_per_value": 8.0 * sizes[rel] / cnt,
            "psnr_db": 20 * np.log10(rng_u) - 10 * np.log10(mse),
            "linf_over_tau": float((rec - u64).abs().max().item()) / tau}
        del rec
        # The same labels through the Huffman stage, their order-0 entropy
        # and Section 4.1's cost estimate (R = range of the coefficients).
        flat = labels.reshape(-1)
        hs = B.huffman_encode(flat)
        x.copy_(u)
        B.decompose(x, None, 0, ws)
        clo, chi = B.value_range(x)
        taus_q = B.mgard_level_tolerances(DIMS, None, 0, tau)
        quality[f"{rel:g}"].update({
            "huffman_bits_per_value": 8.0 * hs.numel() / cnt,
            "huffman_compression_ratio": nbytes / hs.numel(),
            "entropy_bits_per_value": B.label_entropy(flat),
            "cost_model_bits_per_value": B.cost_model(DIMS, 0, taus_q, chi - clo) / cnt})
        del hs
    # Huffman stage throughput on the 1e-3 labels (median of 3).
    e2e_step(1e-3, True)
    flat = labels.reshape(-1)
    t_he, t_hd = [], []
    for i in range(3):
        ea, eb, ec = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        ea.record(stream)
        hs = B.huffman_encode(flat)
        eb.record(stream)
        back = B.huffman_decode(hs, cnt)
        ec.record(stream)
        torch.cuda.synchronize()
        t_he.append(ea.elapsed_time(eb))
        t_hd.append(eb.elapsed_time(ec))
    assert torch.equal(back, flat)
    huffman = {"encode_ms": statistics.median(t_he), "decode_ms": statistics.median(t_hd),
               "labels_gbs_encode": 8 * cnt / (statistics.median(t_he) * 1e-3) / 1e9,
               "labels_gbs_decode": 8 * cnt / (statistics.median(t_hd) * 1e-3) / 1e9,
               "stream_bytes_1e-3": int(hs.numel()),
               "note": "int64 labels of the 513^3 field at 1e-3 x range; the encoder waits twice "
                       "(for the histogram, from which the host builds the code, and for the chunk sizes)"}
    del hs, back
    e2e = {"value": world * nbytes * ke / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": nbytes + stream_bytes, "d2h_bytes_per_step": stream_bytes + nbytes,
           "ms_per_step": e2e_ms / ke, "steps": ke2, "fields_in_flight": lanes_in_flight,
           "path": "mgard_compress_host_packed + mgard_decompress_host_packed",
           "serial": {"value": world * nbytes * ke / (e2e_serial_ms * 1e-3) / 1e9,
                      "ms_per_step": e2e_serial_ms / ke, "steps": ke, "fields_in_flight": 1},
           "note": ("every step uploads the field from pinned host memory, compresses, downloads "
                    "the packed stream, uploads it again, decompresses and downloads the field; "
                    "one host thread per field in flight, each on a stream of its own (value), "
                    "or one field at a time (serial)"),
           "linf_over_tau_1e-3": quality["0.001"]["linf_over_tau"]}
    e2e_u_ms = timed_e2e(False)
    e2e_unpacked = {"value": world * nbytes * ke / (e2e_u_ms * 1e-3) / 1e9, "unit": "GB/s",
                    "h2d_bytes_per_step": nbytes + 8 * cnt, "d2h_bytes_per_step": 8 * cnt + nbytes,
                    "ms_per_step": e2e_u_ms / ke,
                    "path": "mgard_compress_host + mgard_decompress_host (int64 labels)"}

    if rank != 0:
        return
    cpu = cpu_all = None
    fp32_err = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_subprocess(257, 3)
        cpu_all = cpu_baseline_all_cores(257, os.cpu_count() or 1)
        fp32_err = oracle_parity(parity_cases)
        fp32_err["note"] = ("GPU results against the FP64 oracle, computed after the timed "
                            "regions: decompose_rel = max |GPU decomposition - oracle| / max|u|; "
                            "per bound, the GPU recomposition of the GPU's dequantized labels "
                            "against the oracle's recomposition of the same labels, and the "
                            "GPU reconstruction's L-inf error over tau")
        del parity_cases
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_dict(),
        "dec_rec_gbs": dec_rec_gbs,
        "phases_ms_per_step": phase,
        "path_roofline_frac_dec_rec": path_frac,
        "path_roofline_frac_dec_rec_nominal_7900": path_frac_nominal,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "e2e": e2e,
        "e2e_int64_labels": e2e_unpacked,
        "quality": quality,
        "gpu_launches": launches,
        "clocks": clocks.summary(t0, t1),
        "fp32_err_vs_oracle": fp32_err,
        "fp64": fp64,
        "nonuniform": nonuniform,
        "tiny": tiny,
        "adaptive": adaptive,
        "progressive": progressive,
        "nd4": nd4,
        "huffman": huffman,
        "paper_context": PAPER_CONTEXT,
        "linf_over_tau": linf,
        "top_kernels": kernels,
        "kinds_ms_per_step": {k: round(v, 4) for k, v in sorted(kinds.items(), key=lambda kv: -kv[1])},
        "breakdown_steps": kb,
        "src_hash": src_hash(),
    }
    print(json.dumps(line))


def measure_config(B, torch, stream, u_host, coords, stop, reps, keep):
    """Time decompose, quantize, dequantize and recompose of one field at
    1e-3 x range (median of `reps` runs, events on the stream) and check the
    L-inf bound.  With `keep`, also return the field, the decomposition, the
    dequantized labels and the reconstruction for the oracle comparison."""
    import numpy as np
    dims = u_host.shape
    dt = torch.float64 if u_host.dtype == np.float64 else torch.float32
    u = torch.from_numpy(u_host).cuda()
    x = u.clone()
    ws = B.workspace(dims, dt)
    labels = torch.empty(dims, dtype=torch.int64, device=u.device)
    lo, hi = B.value_range(u)
    tau = 1e-3 * (hi - lo)
    B.decompose(x, coords, stop, ws)
    B.recompose(x, coords, stop, ws)
    ph = {k: [] for k in ("decompose", "quantize", "dequantize", "recompose")}
    for _ in range(reps):
        x.copy_(u)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        B.decompose(x, coords, stop, ws)
        ev[1].record(stream)
        B.quantize(x, tau, coords, stop, labels)
        ev[2].record(stream)
        B.dequantize(labels, tau, dt, coords, stop, out=x)
        ev[3].record(stream)
        B.recompose(x, coords, stop, ws)
        ev[4].record(stream)
        torch.cuda.synchronize()
        for j, k in enumerate(ph):
            ph[k].append(ev[j].elapsed_time(ev[j + 1]))
    med = {k: statistics.median(v) for k, v in ph.items()}
    err = float((x.double() - u.double()).abs().max().item())
    assert err <= tau, (dims, stop, err, tau)
    nbytes = u_host.nbytes
    res = {"dims": list(dims), "stop_level": stop, "dtype": "f64" if dt == torch.float64 else "f32",
           "decompose_ms": med["decompose"], "recompose_ms": med["recompose"],
           "quantize_ms": med["quantize"], "dequantize_ms": med["dequantize"],
           "total_ms": sum(med.values()),
           "dec_rec_gbs": nbytes / ((med["decompose"] + med["recompose"]) * 1e-3) / 1e9,
           "linf_over_tau_1e-3": err / tau, "tau": tau}
    case = None
    if keep:
        rec = x.cpu().numpy()
        x.copy_(u)
        B.decompose(x, coords, stop, ws)
        coeffs = x.cpu().numpy()
        B.quantize(x, tau, coords, stop, labels)
        B.dequantize(labels, tau, dt, coords, stop, out=x)
        case = {"u": u_host, "coords": coords, "stop": stop, "coeffs": coeffs,
                "bounds": {1e-3: (tau, x.cpu().numpy(), rec)}}
    return res, case


def run_kernel_case(args):
    """One small self-contained command for the ncu captures: value range,
    decompose, quantize (1e-3 x range), dequantize and recompose of a k^-5/3
    FP32 field of --case-dims (default the 513^3 workload)."""
    import torch
    from paper_2010_05872_gb300 import binding as B
    from paper_2010_05872_gb300 import build as build_mod
    from paper_2010_05872_gb300 import fields as F
    build_mod.build()
    dims = tuple(int(v) for v in args.case_dims.split("x"))
    if len(dims) == 4:
        u = F.grf_field_device(dims, seed=F.SEED_LARGE + 4)
        ws = B.workspace_4d(dims, torch.float32)
    else:
        u = torch.from_numpy(F.grf_field(dims, seed=F.SEED_LARGE)).cuda()
        ws = B.workspace(dims, torch.float32)
    x = u.clone()

    def step():
        lo, hi = B.value_range(x)
        if len(dims) == 4:
            B.decompose_4d(x, None, 0, ws)
            labels, _ = B.quantize_4d(x, 1e-3 * (hi - lo))
            B.dequantize_4d(labels, 1e-3 * (hi - lo), torch.float32, out=x)
            B.recompose_4d(x, None, 0, ws)
            return
        B.decompose(x, None, 0, ws)
        labels, _ = B.quantize(x, 1e-3 * (hi - lo))
        B.dequantize(labels, 1e-3 * (hi - lo), torch.float32, out=x)
        B.recompose(x, None, 0, ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(args.steps):
        step()
    e.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = s.elapsed_time(e) / args.steps
    err = (x - u).abs().max().item() / (u.max() - u.min()).item()
    print(json.dumps({"kernel_case": "x".join(map(str, dims)) + " FP32 range+dec+quant+dequant+rec",
                      "ms_per_step": ms, "linf_over_range": err}))


def level_sizes(dims):
    """Node counts of the levels L, L-1, ..., 0 of a grid (every axis
    coarsened n -> n // 2 + 1 until the smallest axis has 3 nodes)."""
    out, n = [], list(dims)
    while True:
        out.append(list(n))
        if min(n) <= 3:
            return out
        n = [v // 2 + 1 for v in n]


def path_bytes(dims, stop, es):
    """Algorithmic bytes of decompose + recompose: one read and one write of
    every decomposed level's grid per direction, 2 x 2 s sum_{l > l~} #N_l."""
    shapes = level_sizes(dims)
    L = len(shapes) - 1
    return 2 * 2 * es * sum(int(np_prod(shapes[L - l])) for l in range(stop + 1, L + 1))


def path_flops(dims, stop):
    """Algorithmic flops of decompose + recompose of a 3D grid (an FMA counts
    2), per level l with fine sizes n and coarse sizes m: the multilinear
    interpolant and the coefficient subtraction, 3 per coefficient node
    (2 per interpolated value along one axis, 1 for the difference); the
    load vector, 10 per output of a 5-tap restriction along each axis
    (outputs n0 n1 m2, n0 m1 m2, m0 m1 m2); the tridiagonal solves, 4 per
    coarse node per axis; the correction, 1 per coarse node.  Recomposition
    has the same count."""
    shapes = level_sizes(dims)
    L = len(shapes) - 1
    total = 0
    for l in range(stop + 1, L + 1):
        n, m = shapes[L - l], shapes[L - l + 1]
        nf, nc = np_prod(n), np_prod(m)
        total += (3 * (nf - nc) + 10 * (n[0] * n[1] * m[2] + n[0] * m[1] * m[2] + nc)
                  + 12 * nc + nc)
    return 2 * total


def np_prod(v):
    out = 1
    for x in v:
        out *= int(x)
    return out


def level_nodes(dims):
    """Sum over the decomposed levels l = 1..L of the level-l node count."""
    import numpy as np
    n, tot = list(dims), 0
    while min(n) > 3:
        tot += int(np.prod(n))
        n = [v // 2 + 1 for v in n]
    return tot


def lpt_assign(weights, world):
    """Longest-processing-time-first assignment of items to `world` ranks."""
    order = sorted(range(len(weights)), key=lambda i: -weights[i])
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: load[q])
        parts[r].append(i)
        load[r] += weights[i]
    return [sorted(p) for p in parts]


def serving_assign(sizes, world):
    """Online partition of a request stream over `world` ranks: each request,
    in arrival order, goes to the rank with the fewest bytes assigned so far
    (the lowest rank on a tie).  Every rank computes the same assignment."""
    load = [0] * world
    out = []
    for b in sizes:
        r = min(range(world), key=lambda q: (load[q], q))
        out.append(r)
        load[r] += int(b)
    return out


def run_batched(args, rank, world, local_rank):
    """Batched workload: 256 FP32 fields, each axis from U{33..257}, k^-5/3
    fields; decompose + recompose of all fields per step, in one persistent
    launch each (CUDA graph), tile shapes from the autotuner; compared with
    per-field launch sequences on the same fields."""
    import numpy as np
    import torch
    from paper_2010_05872_gb300 import binding as B
    from paper_2010_05872_gb300 import build as build_mod
    from paper_2010_05872_gb300 import fields as F
    build_mod.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    shapes, bounds = F.batched_shapes()
    shapes, bounds = shapes[:args.batch_count], bounds[:args.batch_count]
    mine = lpt_assign([float(np.prod(sh)) for sh in shapes], world)[rank]
    xs = [F.grf_field_device(shapes[i], F.SEED_BATCHED + i, device=dev) for i in mine]
    orig = [x.clone() for x in xs]
    nbytes = sum(x.numel() * 4 for x in xs)
    b_alg = sum(2 * 2 * 4 * level_nodes(x.shape) for x in xs)
    ws = B.batch_workspace(xs)
    t0 = time.perf_counter()
    choice = B.batch_autotune(xs, ws)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        B.batch_decompose(xs, ws)
        B.batch_recompose(xs, ws)
    for x, o in zip(xs, orig):
        x.copy_(o)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    c0 = time.perf_counter()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        B.batch_decompose(xs, ws)
        ev[i][1].record(stream)
        B.batch_recompose(xs, ws)
        ev[i][2].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    c1 = time.perf_counter()
    barrier()
    clocks.stop()
    stats = B.mgard_batch_stats()  # of the last launch (a recomposition)
    elapsed = start.elapsed_time(end)
    dec_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / args.steps
    rec_ms = sum(e[1].elapsed_time(e[2]) for e in ev) / args.steps
    if world > 1:
        t = torch.tensor([elapsed], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed = t.item()
    ms = elapsed / args.steps
    # The same fields through per-field launch sequences.
    for x, o in zip(xs, orig):
        x.copy_(o)
    wss = [B.workspace(tuple(x.shape), torch.float32) for x in xs]
    pf_steps = max(1, min(args.steps, 3))
    for x, w in zip(xs, wss):
        B.decompose(x, None, 0, w)
        B.recompose(x, None, 0, w)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(pf_steps):
        for x, w in zip(xs, wss):
            B.decompose(x, None, 0, w)
            B.recompose(x, None, 0, w)
    s1.record(stream)
    torch.cuda.synchronize()
    pf_ms = s0.elapsed_time(s1) / pf_steps
    del wss
    # Checks outside the timed region: batched against per-field results,
    # and the L-infinity bound of every field at its own bound.
    for x, o in zip(xs, orig):
        x.copy_(o)
    ref = [o.clone() for o in orig[:8]]
    for r in ref:
        B.decompose(r)
    B.batch_decompose(xs, ws)
    torch.cuda.synchronize()
    dev_rel = max(((x - r).abs().max() / r.abs().max()).item() for x, r in zip(xs, ref))
    del ref
    worst = 0.0
    for j, (x, o) in enumerate(zip(xs, orig)):
        lo, hi = B.value_range(o)
        tau = bounds[mine[j]] * (hi - lo)
        labels, _ = B.quantize(x, tau)
        B.dequantize(labels, tau, torch.float32, out=x)
        del labels
    B.batch_recompose(xs, ws)
    for j, (x, o) in enumerate(zip(xs, orig)):
        lo, hi = B.value_range(o)
        tau = bounds[mine[j]] * (hi - lo)
        worst = max(worst, (x.double() - o.double()).abs().max().item() / tau)
    peak, src = measured_peak()
    value = world * nbytes * args.steps / (elapsed * 1e-3) / 1e9  # fields per rank are balanced
    achieved = b_alg / ((dec_ms + rec_ms) * 1e-3) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": "batched decompose+recompose GB/s and % HBM roofline (FP32)",
            "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "%d FP32 3D fields, axes U{33..257}, k^-5/3 fields, full depth, "
                                   "decompose + recompose per step, one persistent launch each"
                                   % len(shapes),
                       "fields": len(shapes), "fields_this_rank": len(xs),
                       "field_bytes_this_rank": nbytes,
                       "l2": "inputs larger than L2 (%.1f GB per rank); no flush" % (nbytes / 1e9),
                       "parallelism": "fields sharded over ranks (longest first)"},
            "dec_ms": dec_ms, "rec_ms": rec_ms,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "peak_source": src + " HBM copy bandwidth",
                         "alg_bytes_per_step": b_alg},
            "per_field_launches_ms_per_step": pf_ms,
            "speedup_vs_per_field": pf_ms / ms,
            "autotune": {"lv_planes": choice[0], "finish_pairs": choice[1], "solve_rows": choice[2],
                         "seg_groups": choice[3], "seconds": tune_s},
            "max_rel_diff_vs_per_field_fp32": dev_rel,
            "linf_over_tau_max": worst,
            "gpu_launches": 2 * args.steps,
            "tile_stats_last_recompose": {k: {"tiles": v[0], "wait_ms_per_cta": v[1] / 2.07e6 / (152 * 2),
                                             "run_ms_per_cta": v[2] / 2.07e6 / (152 * 2)}
                                          for k, v in stats.items()},
            "clocks": clocks.summary(c0, c1),
        }))


def run_serving(args, rank=0, world=1, local_rank=0):
    """Serving workload: a seeded Poisson stream (mean 200 requests/s) of
    compress / decompress requests on FP32 k^-5/3 fields, 2D sides from
    {1024, 1025, 2048, 2049, 4096} or 3D sides from {129, 257, 513}, bounds
    from {1e-2, 1e-3, 1e-4} x range, admitted against a 120 GB HBM budget by
    the library's serving loop; p50 / p99 latency and aggregate GB/s.  With
    N > 1 ranks the stream is partitioned over the ranks by bytes
    (`serving_assign`), each rank serving its share on its own GPU; rank 0
    merges the latencies and reports all ranks' bytes over the slowest
    rank's wall time (no collective on the data path)."""
    import numpy as np
    import torch
    from paper_2010_05872_gb300 import binding as B
    from paper_2010_05872_gb300 import build as build_mod
    from paper_2010_05872_gb300 import fields as F
    build_mod.build()
    torch.cuda.set_device(local_rank)
    rng = np.random.default_rng(F.SEED_SERVING)
    shapes = [(s, s) for s in (1024, 1025, 2048, 2049, 4096)] + [(s, s, s) for s in (129, 257, 513)]
    nreq = args.serving_requests
    gaps = rng.exponential(1.0 / 200.0, size=nreq)
    arrive = np.cumsum(gaps)
    kinds = rng.random(nreq) < 0.5                     # True: compress
    is3d = rng.random(nreq) < 0.5
    pick = np.where(is3d, 5 + rng.integers(0, 3, nreq), rng.integers(0, 5, nreq))
    rels = rng.choice([1e-2, 1e-3, 1e-4], size=nreq)
    sizes = [4 * int(np.prod(shapes[int(i)])) for i in pick]
    assign = serving_assign(sizes, world)
    mine = [k for k in range(nreq) if assign[k] == rank]
    # One field per shape (pinned), compressed once beforehand: the inputs of
    # the decompress requests.  Output buffers are recycled per shape.
    fields, packed, pools = [], [], []
    srv = B.Server(hbm_budget=120 << 30, slots=8)
    for i, shp in enumerate(shapes):
        f = F.grf_field_device(shp, F.SEED_SERVING + i).cpu().ravel().pin_memory()
        fields.append(f)
        lab = torch.empty(f.numel(), dtype=torch.int64).pin_memory()
        srv.submit(B.OP_COMPRESS, shp, f, lab, rel_bound=1e-3)
        srv.drain()
        (_, st, _, tau), = srv.poll()
        assert st == 0
        packed.append((lab, tau))
        pools.append([torch.empty(f.numel(), dtype=torch.int64).pin_memory() for _ in range(3)])
    free = [list(range(3)) for _ in shapes]
    inflight = {}
    lat = {"compress": [], "decompress": []}
    nbytes = 0
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    m = 0
    done_n = 0
    first_arrival = None
    last_done = arrive[0]
    while done_n < len(mine):
        now = time.perf_counter() - t0
        while m < len(mine) and arrive[mine[m]] <= now and free[pick[mine[m]]]:
            k = mine[m]
            i = int(pick[k])
            slot = free[i].pop()
            buf = pools[i][slot]
            if kinds[k]:
                rid = srv.submit(B.OP_COMPRESS, shapes[i], fields[i], buf, rel_bound=float(rels[k]))
            else:
                rid = srv.submit(B.OP_DECOMPRESS, shapes[i], packed[i][0], buf.view(torch.float32)[
                    :fields[i].numel()], tau=packed[i][1])
            inflight[rid] = (i, slot, "compress" if kinds[k] else "decompress", arrive[k])
            if first_arrival is None:
                first_arrival = now
            m += 1
        for rid, st, l, _ in srv.poll():
            i, slot, kind, a = inflight.pop(rid)
            assert st == 0, st
            free[i].append(slot)
            # Latency from the request's scheduled arrival (queueing for a
            # host buffer included) to completion.
            lat[kind].append(time.perf_counter() - t0 - a)
            nbytes += fields[i].numel() * 4
            done_n += 1
            last_done = time.perf_counter() - t0
        time.sleep(0.0002)
    wall = last_done - arrive[0]
    counters = srv.counters()
    # Mix vs alone: this rank's first 16 request kinds again, one at a time.
    same = True
    for j in mine[:16]:
        i = int(pick[j])
        if kinds[j]:
            a = torch.empty(fields[i].numel(), dtype=torch.int64).pin_memory()
            b = torch.empty_like(a).pin_memory()
            srv.submit(B.OP_COMPRESS, shapes[i], fields[i], a, rel_bound=float(rels[j]))
            srv.drain()
            srv.poll()
            srv2 = B.Server(hbm_budget=120 << 30, slots=1)
            srv2.submit(B.OP_COMPRESS, shapes[i], fields[i], b, rel_bound=float(rels[j]))
            srv2.drain()
            srv2.poll()
            srv2.close()
            same = same and torch.equal(a, b)
    srv.close()
    if world > 1:
        parts = [None] * world
        torch.distributed.all_gather_object(parts, (lat, nbytes, wall, counters, same))
        if rank != 0:
            return
        lat = {kk: [v for p in parts for v in p[0][kk]] for kk in lat}
        nbytes = sum(p[1] for p in parts)
        wall = max(p[2] for p in parts)
        counters = {"peak_running": max(p[3]["peak_running"] for p in parts),
                    "peak_bytes": max(p[3]["peak_bytes"] for p in parts)}
        same = all(p[4] for p in parts)
    allat = sorted(lat["compress"] + lat["decompress"])

    def pct(v, q):
        v = sorted(v)
        return 1e3 * v[min(len(v) - 1, int(q * len(v)))] if v else None

    print(json.dumps({
        "metric": "serving aggregate GB/s (field bytes) with p50/p99 latency",
        "value": nbytes / wall / 1e9, "unit": "GB/s", "n_gpus": world, "steps": nreq, "warmup": len(shapes),
        "ms_per_step": 1e3 * wall / nreq, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "Poisson 200 req/s, %d requests, 50%% compress / 50%% decompress, "
                               "2D sides {1024,1025,2048,2049,4096} or 3D sides {129,257,513}, "
                               "k^-5/3 FP32 fields, bounds {1e-2,1e-3,1e-4} x range" % nreq,
                   "hbm_budget_gb": 120, "slots": 8,
                   "parallelism": "requests partitioned over ranks by bytes (serving_assign)"},
        "latency_ms": {"p50": pct(allat, 0.5), "p99": pct(allat, 0.99),
                       "compress_p50": pct(lat["compress"], 0.5), "compress_p99": pct(lat["compress"], 0.99),
                       "decompress_p50": pct(lat["decompress"], 0.5),
                       "decompress_p99": pct(lat["decompress"], 0.99)},
        "peak_running": counters["peak_running"], "peak_bytes_gb": counters["peak_bytes"] / 1e9,
        "wall_s": wall, "same_alone_and_in_mix": same,
    }))


def main():
    args = parse_args()
    if args.kernel_case:
        run_kernel_case(args)
        return
    if args.oracle_sample:
        run_oracle_sample_cli(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "serving":
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        try:
            run_serving(args, rank, world, local_rank)
        finally:
            if world > 1:
                import torch
                torch.distributed.destroy_process_group()
        return
    if args.workload == "batched":
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        try:
            run_batched(args, rank, world, local_rank)
        finally:
            if world > 1:
                import torch
                torch.distributed.destroy_process_group()
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
