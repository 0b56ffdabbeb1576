#!/usr/bin/env python3
"""Benchmark of the ISRS EGN NLI integrator on GB300.

Metric: NLI eta channel-evaluations per second on the 120-channel C+L link
(120 ch x 64 GBd on a 75 GHz grid, 9 THz, 10 x 80 km SSMF, 2 dBm/ch, formats
from splitmix64 seed 0, 32 x 32 Gauss-Legendre points per island, dz = 1 km,
EGN terms).  One step = one full evaluation of the hot path (island planner,
D/G/H pass, E pass, F pass, assembly) for all 120 channels.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32c|fp64]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Multi-GPU: every rank evaluates its own copy of the link (replicas; the work
does not exchange data), value = channel-evals of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NLI eta channel-evals/sec (120ch C+L)"
UNIT = "channel-evals/s"
WORKLOAD = ("120ch x 64GBd C+L on 75GHz grid (9 THz), 10x80km SSMF, 2 dBm/ch, seeded formats, "
            "32x32 Gauss-Legendre per island, dz=1km, EGN (D+E+F+G+H)")
SM_COUNT_GB300 = 152
FP32_LANES_PER_SM = 128
MUFU_PER_POINT = 6  # D-only point path of the FP32C D/G/H pass: sin x 3, cos x 2, rcp x 1


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.lines = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", self.gpu_id], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_median": statistics.median(power), "reasons": sorted(reasons)}


def gpu_id_for_smi(local_rank: int) -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        return vis.split(",")[local_rank if local_rank < len(vis.split(",")) else 0]
    return str(local_rank)


# --------------------------------------------------------------------------- pipe peaks

# launch shape and rounds per thread of each throughput probe: full occupancy
# (2048 threads per SM), about 10 ms per launch on a GB300
PROBES = {"ffma": 160000, "ffma2": 80000, "dfma": 2500, "mufu_sin": 20000, "mufu_ex2": 20000, "mufu_rcp": 20000,
          "fma_mix": 53000}
PROBE_THREADS = 256


def measure_peaks(kinds, stream, reps: int = 5, sampler=None) -> dict:
    """Throughput of the arithmetic pipes with the library's probe kernels
    (egn_probe_launch), CUDA events on `stream`: best of `reps` launches after one
    warm-up.  TFLOP/s for the FMA probes, Gop/s for the MUFU probes, and the
    same per SM per clock at the median SM clock sampled meanwhile."""
    import torch
    from paper_2412_11614_gb300 import egn
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = sms * (2048 // PROBE_THREADS)
    sink = torch.empty(blocks * PROBE_THREADS, dtype=torch.float64, device="cuda")
    out = {}
    smi = sampler
    if smi is not None:
        smi.start()
        time.sleep(0.3)
    for kind in kinds:
        iters = PROBES[kind]
        ops = egn.probe_ops(kind, blocks, PROBE_THREADS, iters)
        with torch.cuda.stream(stream):
            egn.probe_launch(kind, blocks, PROBE_THREADS, iters, sink, stream.cuda_stream)
            best = None
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                egn.probe_launch(kind, blocks, PROBE_THREADS, iters, sink, stream.cuda_stream)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
        rate = ops / (best * 1e-3)
        out[kind] = {"ms": best, "ops_per_launch": ops,
                     ("tflops" if "fma" in kind else "gops"): rate / (1e12 if "fma" in kind else 1e9)}
    clocks = smi.stop() if smi is not None else {}
    mhz = clocks.get("sm_mhz")
    for kind, r in out.items():
        rate = r["ops_per_launch"] / (r["ms"] * 1e-3)
        r["per_sm_per_clock"] = rate / (sms * mhz * 1e6) if mhz else None
    return {"probes": out, "sms": sms, "blocks": blocks, "threads": PROBE_THREADS, "clocks": clocks}


# --------------------------------------------------------------------------- ranks

def aggregate_ranks(ms_local: float, evals_local: int, device=None):
    """Replicas: every rank evaluated its own link.  Returns (max-over-ranks step
    time [ms], channel-evals of all ranks per second, world size).  Works with any
    initialised torch.distributed backend (NCCL on GPUs, gloo on CPU)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return ms_local, evals_local / (ms_local * 1e-3), 1
    world = dist.get_world_size()
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([float(evals_local)], dtype=torch.float64, device=device)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    return ms, float(e.item()) / (ms * 1e-3), world


# --------------------------------------------------------------------------- oracle timing

def host_cpu() -> str:
    """The host CPU as /proc/cpuinfo names it: the model name on x86, the
    implementer and part numbers on Arm; the machine type elsewhere."""
    import platform
    fields = {}
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                k, _, v = ln.partition(":")
                fields.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    if fields.get("model name"):
        return fields["model name"]
    if fields.get("CPU implementer"):
        return (f"{platform.machine()} (implementer {fields['CPU implementer']}, "
                f"part {fields.get('CPU part', '?')})")
    return platform.machine() or "unknown"


def oracle_rate(wl, target_s: float, seed: int = 0):
    """Time the FP64 CPU oracle (as it stands) on a seeded sample of islands of the
    workload, on all host cores (one island per thread).  Returns (channel-evals/s,
    threads, sample description, islands/channel)."""
    import concurrent.futures as cf
    import numpy as np
    from oracle import oracle as O

    pb = O.Problem(wl)
    rng = np.random.default_rng(seed)
    n_ch = pb.n_ch
    cois = rng.choice(n_ch, size=min(4, n_ch), replace=False)
    pool = []
    per = []
    for n in cois:
        isl = pb.islands(int(n))
        per.append(len(isl))
        pool += [(int(n), *map(int, t)) for t in isl]
    avg_isl = float(np.mean(per))
    threads = os.cpu_count() or 1
    order = rng.permutation(len(pool))
    ex = cf.ThreadPoolExecutor(max_workers=threads)
    # calibrate on a small batch, then size the sample to ~target_s seconds
    calib = [pool[i] for i in order[: 2 * threads]]
    t0 = time.perf_counter()
    list(ex.map(lambda t: pb.island_terms(*t), calib))
    dt = time.perf_counter() - t0
    per_isl = dt / len(calib)
    n_sample = int(max(threads, min(len(pool) - len(calib), target_s / per_isl)))
    sample = [pool[i] for i in order[len(calib): len(calib) + n_sample]]
    t0 = time.perf_counter()
    list(ex.map(lambda t: pb.island_terms(*t), sample))
    dt = time.perf_counter() - t0
    ex.shutdown()
    rate = (len(sample) / avg_isl) / dt
    desc = (f"{len(sample)} islands drawn (seed {seed}) from COIs {sorted(int(c) for c in cois)} of the timed "
            f"workload ({avg_isl:.0f} islands/channel on average), segment-form mu, all D..H terms per island; "
            f"{dt:.1f} s wall on {threads} threads")
    return rate, threads, desc, avg_isl, dt


# --------------------------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2412_11614_gb300 import workloads as W
    wl = W.config_cl()
    rates = []
    threads = os.cpu_count() or 1
    desc = ""
    per_step = max(3.0, 150.0 / max(1, args.steps + args.warmup))
    for i in range(args.warmup + args.steps):
        r, threads, desc, _, _ = oracle_rate(wl, per_step, seed=i)
        if i >= args.warmup:
            rates.append(r)
    value = statistics.mean(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * 120 / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "fp64 CPU oracle", "n_ch": 120},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
                         "cpu": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    emit(line, args.jsonl)
    return 0


def emit(line: dict, jsonl: str = None) -> None:
    """Print the JSON line; with `jsonl`, also append it to that file with a hash of
    its workload and configuration (the same workload and options hash alike)."""
    print(json.dumps(line), flush=True)
    if jsonl:
        key = json.dumps({k: line.get(k) for k in ("metric", "impl", "config", "workload", "n_gpus", "dtype")},
                         sort_keys=True)
        rec = dict(line, config_hash=hashlib.sha256(key.encode()).hexdigest()[:16], time_unix=time.time())
        with open(jsonl, "a") as f:
            f.write(json.dumps(rec) + "\n")


# --------------------------------------------------------------------------- our arm

def flops_per_point(precision: str, K: int) -> float:
    """Algorithmic FLOPs per quadrature point of the D/G/H pass (FMA = 2 FLOPs):
    the segment sum of Eq. 8 by the real second-order recurrence, 2 FMA per
    segment (4 K), in both precisions.  The per-point phase, trigonometry and
    weights are not counted."""
    return 4.0 * K


def timed_evals(ln, opts, n_ch, stream, flush, steps: int, warm: int, detail: dict = None):
    """Device ms per evaluation (egn_nli_eta_device, CUDA events on `stream`, L2
    flushed before each) and the last evaluation's eta.  With `detail`, also the
    per-evaluation times and the last evaluation's per-stage times (profiling is
    switched on for the evaluations)."""
    import torch
    ws = torch.empty(ln.workspace_size(opts), dtype=torch.uint8, device="cuda")
    eta = torch.empty(n_ch, dtype=torch.float64, device="cuda")
    pnli = torch.empty(n_ch, dtype=torch.float64, device="cuda")
    times, enq = [], []
    with torch.cuda.stream(stream):
        for i in range(warm + steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t0 = time.perf_counter()
            ln.nli_eta_device(opts, ws, eta, pnli)
            t1 = time.perf_counter()
            e1.record(stream)
            e1.synchronize()
            if i >= warm:
                times.append(e0.elapsed_time(e1))
                enq.append((t1 - t0) * 1e3)
    if detail is not None:
        detail["ms_each"] = times
        detail["enqueue_ms_each"] = enq  # host time of the call (the device waits meanwhile)
        detail["stage_ms"] = {k: float(v) for k, v in ln.last_timings().items()}
    return statistics.mean(times), eta.cpu().numpy()


def fp64_denominator(args, wl, ln, eta32, value, stream, flush) -> dict:
    """The metric's denominator and precision gate: the plain FP64 GPU integrator
    (EGN_PREC_FP64) on the same link and GPU, its channel-evals/s, FP32C's speed-up
    over it and FP32C's per-channel error against it in dB (every channel); then
    the launch-power sweep -2..+4 dBm/ch (1 dB steps) of the same link in FP32C,
    each power against one FP64 evaluation (ISRS strength grows with the total
    power, Eq. 12)."""
    import numpy as np
    from paper_2412_11614_gb300 import egn, workloads as W
    n_ch = wl.n_ch
    o64 = egn.make_opts(gl_order=wl.gl_order, dz_km=wl.dz_km, precision=egn.EGN_PREC_FP64, terms=egn.EGN_TERMS_EGN,
                        stream=stream.cuda_stream)
    o32 = egn.make_opts(gl_order=wl.gl_order, dz_km=wl.dz_km, precision=egn.EGN_PREC_FP32C, terms=egn.EGN_TERMS_EGN,
                        stream=stream.cuda_stream)
    ms64, eta64 = timed_evals(ln, o64, n_ch, stream, flush, steps=args.fp64_steps, warm=1)
    err = np.abs(10 * np.log10(eta32 / eta64))
    out = {"fp64_gpu": {"ms_per_step": ms64, "value": n_ch / (ms64 * 1e-3), "unit": UNIT, "steps": args.fp64_steps,
                        "warmup": 1, "dtype": "f64",
                        "note": "plain FP64 GPU integrator (EGN_PREC_FP64), same link, same GPU, CUDA events, "
                                "L2 flushed between steps"},
           "speedup_vs_fp64_gpu": value / (n_ch / (ms64 * 1e-3)),
           "max_db_vs_fp64": float(err.max()), "mean_db_vs_fp64": float(err.mean()),
           "worst_channel_vs_fp64": int(err.argmax())}
    if not args.no_ridge:
        # the ridge-resolving node rule (FP64) on the same link: its time per evaluation and
        # how far the configured 32 x 32 rule's eta lies from it (the rule's discretisation error)
        ln.set_node_rule(egn.EGN_RULE_RIDGE, 4)
        orr = egn.make_opts(gl_order=args.ridge_nodes, dz_km=wl.dz_km, precision=egn.EGN_PREC_FP64,
                            terms=egn.EGN_TERMS_EGN, stream=stream.cuda_stream)
        ln.set_profiling(True)
        det64, det32 = {}, {}
        msr, etar = timed_evals(ln, orr, n_ch, stream, flush, steps=1, warm=1, detail=det64)
        # and in FP32C (the same rule; identical spans): time and distance from the FP64 result
        orr32 = egn.make_opts(gl_order=args.ridge_nodes, dz_km=wl.dz_km, precision=egn.EGN_PREC_FP32C,
                              terms=egn.EGN_TERMS_EGN, stream=stream.cuda_stream)
        msr32, etar32 = timed_evals(ln, orr32, n_ch, stream, flush, steps=3, warm=1, detail=det32)
        ln.set_node_rule(egn.EGN_RULE_GL)
        dr = 10 * np.log10(eta64 / etar)
        d32 = np.abs(10 * np.log10(etar32 / etar))
        out["ridge_rule"] = {"nodes_per_piece": args.ridge_nodes, "n_min": 4, "precision": "fp64",
                             "ms_per_step": msr, "value": n_ch / (msr * 1e-3), "unit": UNIT,
                             "gl32_minus_ridge_db": {"mean": float(dr.mean()), "min": float(dr.min()),
                                                     "max": float(dr.max()), "edge": float(dr[0]),
                                                     "centre": float(dr[n_ch // 2])},
                             "eta_db_sample": [float(10 * np.log10(x)) for x in etar[:: 30]],
                             "stage_ms": det64["stage_ms"],
                             "fp32c": {"ms_per_step": msr32, "value": n_ch / (msr32 * 1e-3), "unit": UNIT,
                                       "ms_each": det32["ms_each"], "enqueue_ms_each": det32["enqueue_ms_each"],
                                       "stage_ms": det32["stage_ms"],
                                       "speedup_vs_fp64": msr / msr32, "max_db_vs_fp64": float(d32.max()),
                                       "mean_db_vs_fp64": float(d32.mean())}}
    if args.no_sweep:
        return out
    sweep = {"p_dbm": [], "ms_fp32c": [], "ms_fp64": [], "channel_evals_per_s_fp32c": [], "max_abs_db_vs_fp64": [],
             "mean_abs_db_vs_fp64": [], "worst_channel": [], "delta_rho_db_per_span": []}
    for p_dbm in range(-2, 5):
        wp = W.config_cl(n_ch=n_ch, p_dbm=float(p_dbm))
        lp = egn.link_from_workload(wp)
        m32, e32 = timed_evals(lp, o32, n_ch, stream, flush, steps=3, warm=1)
        m64, e64 = timed_evals(lp, o64, n_ch, stream, flush, steps=1, warm=0)
        lp.close()
        d = np.abs(10 * np.log10(e32 / e64))
        ptot = sum(wp.launch_power_w)
        sp = wp.spans[0]
        a = sp.alpha_db_km * math.log(10) / 10
        leff = (1 - math.exp(-a * sp.length_m * 1e-3)) / a
        btot = (wp.centre_hz[-1] - wp.centre_hz[0]) * 1e-12 * n_ch / (n_ch - 1)
        sweep["p_dbm"].append(p_dbm)
        sweep["ms_fp32c"].append(m32)
        sweep["ms_fp64"].append(m64)
        sweep["channel_evals_per_s_fp32c"].append(n_ch / (m32 * 1e-3))
        sweep["max_abs_db_vs_fp64"].append(float(d.max()))
        sweep["mean_abs_db_vs_fp64"].append(float(d.mean()))
        sweep["worst_channel"].append(int(d.argmax()))
        sweep["delta_rho_db_per_span"].append(10 * math.log10(math.e) * ptot * sp.cr_per_w_km_thz * leff * btot)
    out["config3_power_sweep"] = dict(sweep, workload="the benchmark link at -2..+4 dBm/ch, FP32C against the plain "
                                                      "FP64 GPU integrator, every channel")
    return out


def run_mu_compare(args):
    """The three forms of mu on the same GPU (Sec. III): FP64 integral form (Eq. 23,
    the paper's numerical reference), FP64 segment (Eq. 7-10) and Maclaurin
    (Eq. 4-6) closed forms, and the FP32C segment path, on Table I links of
    n_ch channels of the 10.1 GHz grid around 1550 nm.  Prints one JSON line per
    link: device ms per evaluation, the time reduction of each closed form
    against the integral form, and the per-channel error of each closed form
    against the integral form in dB (Fig. 8-10 analogues)."""
    import numpy as np
    import torch
    from paper_2412_11614_gb300 import _build, egn, workloads as W
    _build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    for n_spans, cr in ((1, 0.28), (1, 1.12), (10, 1.12)):
        wl = W.table1(n_spans=n_spans, cr=cr, fmt="QPSK", gl_order=args.mu_gl, n_ch=args.mu_n_ch)
        ln = egn.link_from_workload(wl)
        res, ms = {}, {}
        for name, form, prec in (("fp64_integral", egn.EGN_MU_INTEGRAL, egn.EGN_PREC_FP64),
                                 ("fp64_segment", egn.EGN_MU_SEGMENT, egn.EGN_PREC_FP64),
                                 ("fp64_maclaurin", egn.EGN_MU_MACLAURIN, egn.EGN_PREC_FP64),
                                 ("fp32c_segment", egn.EGN_MU_SEGMENT, egn.EGN_PREC_FP32C)):
            opts = egn.make_opts(gl_order=wl.gl_order, dz_km=wl.dz_km, precision=prec, terms=egn.EGN_TERMS_EGN,
                                 stream=stream.cuda_stream, mu_form=form)
            ws = torch.empty(ln.workspace_size(opts), dtype=torch.uint8, device="cuda")
            eta = torch.empty(wl.n_ch, dtype=torch.float64, device="cuda")
            pn = torch.empty(wl.n_ch, dtype=torch.float64, device="cuda")
            reps = 1 if form == egn.EGN_MU_INTEGRAL else 5
            with torch.cuda.stream(stream):
                if form != egn.EGN_MU_INTEGRAL:
                    ln.nli_eta_device(opts, ws, eta, pn)
                t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                t0.record(stream)
                for _ in range(reps):
                    ln.nli_eta_device(opts, ws, eta, pn)
                t1.record(stream)
            t1.synchronize()
            ms[name] = t0.elapsed_time(t1) / reps
            res[name] = eta.cpu().numpy()
        ref = 10 * np.log10(res["fp64_integral"])
        err = {k: 10 * np.log10(v) - ref for k, v in res.items() if k != "fp64_integral"}
        line = {"workload": f"Table I: {wl.n_ch} ch x 10 GBd at 10.1 GHz, {n_spans} x 100 km, Cr {cr}, QPSK, "
                            f"{wl.gl_order} x {wl.gl_order} Gauss-Legendre, dz 1 km",
                "ms_per_eval": ms,
                "time_reduction_vs_integral": {k: 1.0 - ms[k] / ms["fp64_integral"] for k in ms if k != "fp64_integral"},
                "mae_db_vs_integral": {k: float(np.mean(np.abs(v))) for k, v in err.items()},
                "max_abs_db_vs_integral": {k: float(np.max(np.abs(v))) for k, v in err.items()},
                "islands": ln.island_count()[0]}
        print(json.dumps(line), flush=True)
        ln.close()
    return 0


def run_batch_compare(args):
    """Many links at once (egn_batch_*): the same links evaluated one after the
    other through egn_nli_eta_device on one stream, against one launch of the
    batch's CUDA graph (every link an independent branch).  Links: the C+L grid
    cut to 8..48 channels, 1..10 spans, FP32C.  Prints one JSON line."""
    import numpy as np
    import torch
    from paper_2412_11614_gb300 import _build, egn, workloads as W
    _build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    if args.batch_random:  # seeded heterogeneous links: 20-200 ch, 1-30 spans of drawn lengths and fibres
        gl = 16
        wls = [W.random_link(i + 1, gl_order=gl) for i in range(args.batch_links)]
        desc = (f"{len(wls)} seeded random links (20-200 ch, 32-96 GBd, 1-30 SSMF/PSCF spans of 50-120 km, "
                f"tilted rippled powers), {gl} x {gl} GL, FP32C, EGN")
    else:
        gl = 32
        wls = [W.config_cl(n_ch=8 + 8 * (i % 6), n_spans=1 + (i % 10), seed=i) for i in range(args.batch_links)]
        desc = "C+L grid cut to 8..48 channels, 1..10 x 80 km, 32 x 32 GL, FP32C, EGN"
    links = [egn.link_from_workload(w) for w in wls]
    opts = egn.make_opts(gl_order=gl, precision=egn.EGN_PREC_FP32C, stream=stream.cuda_stream)
    ws = [torch.empty(ln.workspace_size(opts), dtype=torch.uint8, device="cuda") for ln in links]
    outs = [(torch.empty(ln.n_ch, dtype=torch.float64, device="cuda"),
             torch.empty(ln.n_ch, dtype=torch.float64, device="cuda")) for ln in links]

    def one_by_one():
        for ln, w, (e, p) in zip(links, ws, outs):
            ln.nli_eta_device(opts, w, e, p)

    b = egn.Batch(links, opts)

    def timed(fn, reps):
        with torch.cuda.stream(stream):
            for _ in range(1 if args.batch_random else 3):
                fn()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(reps):
                fn()
            t1.record(stream)
        t1.synchronize()
        return t0.elapsed_time(t1) / reps

    reps = 2 if args.batch_random else args.steps
    smi = ClockSampler(gpu_id_for_smi(0))
    smi.start()
    time.sleep(0.3)
    seq_ms = timed(one_by_one, reps)
    graph_ms = timed(lambda: b.launch(stream.cuda_stream), reps)
    clocks = smi.stop()
    got = b.read(stream.cuda_stream)
    same = all(np.array_equal(g[0], o[0].cpu().numpy()) for g, o in zip(got, outs))
    n_ch = int(b.offsets[-1])
    print(json.dumps({"links": len(links), "channels": n_ch,
                      "span_types": [len({(s.length_m, s.alpha_db_km, s.D_ps_nm_km) for s in w.spans}) for w in wls],
                      "workload": desc,
                      "ms_one_by_one": seq_ms, "ms_graph": graph_ms, "speedup": seq_ms / graph_ms,
                      "channel_evals_per_s_graph": n_ch / (graph_ms * 1e-3), "results_identical": same,
                      "clocks": clocks}), flush=True)
    b.close()
    return 0


def gemm_roofline(g: int, reps: int) -> dict:
    """The surrogate's tensor-core GEMM on its own: g^3 BF16 (random inputs),
    FP32 accumulation, BF16 output with a bias, CUDA-event time per launch
    against the measured BF16 peak."""
    import torch
    from paper_2412_11614_gb300 import mlp
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    ga = torch.randn((g, g), device="cuda").to(torch.bfloat16)
    gb = torch.randn((g, g), device="cuda").to(torch.bfloat16)
    gout = torch.empty((g, g), dtype=torch.bfloat16, device="cuda")
    gbias = torch.zeros(g, dtype=torch.float32, device="cuda")
    for _ in range(3):
        mlp.gemm(ga, gb, gout, mlp.EPI_BIAS, bias=gbias, err=err)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        mlp.gemm(ga, gb, gout, mlp.EPI_BIAS, bias=gbias, err=err)
    e1.record()
    e1.synchronize()
    if int(err.item()):
        raise RuntimeError("a bounded wait of the GEMM ran out")
    ms = e0.elapsed_time(e1) / reps
    tflops = 2.0 * g ** 3 / (ms * 1e-3) / 1e12
    peaks = {}
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    peak = peaks.get("bf16_tflops")
    return {"m_n_k": g, "ms": ms, "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                                              "frac": tflops / peak if peak else None,
                                              "peak_note": "measured cuBLAS bf16 burst" if peak else "no measured peak"}}


def run_surrogate(args):
    """MLP surrogate end to end: labels of seeded 120-channel links from the
    FP32C integrator (batches of links), training on the tensor-core kernels,
    accuracy on held-out links, and inference throughput against the
    integrator's.  Prints one JSON line."""
    import numpy as np
    import torch
    from paper_2412_11614_gb300 import _build, egn, surrogate as S, workloads as W
    _build.build()
    torch.cuda.set_device(0)
    ridge = args.sur_rule == "ridge"
    rule = egn.EGN_RULE_RIDGE if ridge else egn.EGN_RULE_GL
    opts = egn.make_opts(gl_order=args.ridge_nodes if ridge else 32, precision=egn.EGN_PREC_FP32C)
    rule_txt = (f"the ridge-resolving rule, {args.ridge_nodes} nodes per piece" if ridge else "32 x 32 GL")
    train_w = [W.surrogate_link(i + 1) for i in range(args.sur_train)]
    test_w = [W.surrogate_link(1000001 + i) for i in range(args.sur_test)]
    t0 = time.perf_counter()
    seeds = [i + 1 for i in range(args.sur_train)] + [1000001 + i for i in range(args.sur_test)]
    cached = bool(args.sur_labels and os.path.exists(os.path.join(args.sur_labels, "index.json")))
    if args.sur_labels:  # sharded label files with a resume index
        lab = list(S.generate_labels(args.sur_labels, seeds, opts, rule=rule))
    else:
        lab = []
        for i in range(0, len(train_w) + len(test_w), 64):
            lab += S.labels((train_w + test_w)[i:i + 64], opts, rule)
    label_s = time.perf_counter() - t0
    xtr = np.concatenate([S.features(w) for w in train_w])
    ytr = np.concatenate(lab[:len(train_w)])
    xte = np.concatenate([S.features(w) for w in test_w])
    yte = np.concatenate(lab[len(train_w):])
    model = S.Surrogate(seed=0)
    model.fit_normalisation(xtr, ytr)
    bs = 8192
    steps = args.sur_steps
    t0 = time.perf_counter()
    losses = S.train(model, xtr, ytr, steps, batch_rows=bs, seed=0)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    pred = model.predict_rows(xte)
    err = pred - yte
    # inference throughput: forward passes over a large block of rows, CUDA events
    big = np.tile(xte, (max(1, (1 << 20) // len(xte)), 1))
    model.predict_rows(big)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows, _ = model._load_inputs(big, None)
    e0.record()
    reps = 10
    for _ in range(reps):
        model._forward(None)
        S.K.head(model.h[S.LAYERS], model.w_out, model.b_out, model.y)
    e1.record()
    e1.synchronize()
    inf_ms = e0.elapsed_time(e1) / reps
    flops = 2.0 * rows * (S.F_PAD * S.HIDDEN + (S.LAYERS - 1) * S.HIDDEN * S.HIDDEN + S.HIDDEN)
    gemm = gemm_roofline(8192, 5)
    # the per-link network (n_ch powers + span count + span length + Cr -> 3 x 512 GELU -> n_ch)
    # on the same training and held-out links
    ltr = np.stack([S.link_features(w) for w in train_w])
    lte = np.stack([S.link_features(w) for w in test_w])
    ytr_l = np.stack(lab[:len(train_w)])
    yte_l = np.stack(lab[len(train_w):])
    lmodel = S.LinkSurrogate(n_ch=ytr_l.shape[1], seed=0)
    lmodel.fit_normalisation(ltr, ytr_l)
    t0 = time.perf_counter()
    llosses = S.train(lmodel, ltr, ytr_l, args.sur_steps, batch_rows=min(512, len(ltr)), seed=0)
    torch.cuda.synchronize()
    ltrain_s = time.perf_counter() - t0
    lerr = lmodel.predict_rows(lte) - yte_l
    base_err = yte_l - ytr_l.mean(axis=0)  # no network: each channel's mean training label
    big_l = np.tile(lte, (max(1, 8192 // len(lte)), 1))
    lmodel.predict_rows(big_l)
    lrows, lrows_pad = lmodel._load_inputs(big_l, None)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        lmodel._forward(lrows, lrows_pad, None)
        S.K.outputs(lmodel.acc, lrows, lrows_pad, lmodel.n_ch, lmodel.b_out, lmodel.y)
    e1.record()
    e1.synchronize()
    linf_ms = e0.elapsed_time(e1) / reps
    link_net = {"network": f"{lmodel.n_in} inputs (powers, span count, span length, Cr) -> 3 x 512 GELU -> "
                           f"{lmodel.n_ch} outputs, BF16 tensor cores",
                "train_steps": args.sur_steps, "batch_links": min(512, len(ltr)), "train_seconds": ltrain_s,
                "loss_first": llosses[0], "loss_last": float(np.mean(llosses[-20:])),
                "heldout_mae_db": float(np.mean(np.abs(lerr))),
                "heldout_p99_abs_db": float(np.quantile(np.abs(lerr), 0.99)),
                "heldout_max_abs_db": float(np.max(np.abs(lerr))),
                "inference_links": lrows, "inference_ms": linf_ms,
                "inference_channel_evals_per_s": lrows * lmodel.n_ch / (linf_ms * 1e-3)}
    print(json.dumps({
        "workload": f"surrogate: {args.sur_train} training + {args.sur_test} held-out seeded 120-ch C+L links "
                    "(1-30 identical SSMF spans of 50-120 km, Cr 0.014-0.042, tilted rippled powers); labels from "
                    f"the FP32C integrator, {rule_txt}, dz 1 km",
        "labels": "read (or resumed) from the label directory" if cached else "computed by the integrator in this run",
        "label_seconds": None if cached else label_s,
        "label_channel_evals_per_s": None if cached else 120 * (args.sur_train + args.sur_test) / label_s,
        "train_steps": steps, "batch_rows": bs, "train_seconds": train_s,
        "loss_first": losses[0], "loss_last": float(np.mean(losses[-20:])),
        "heldout_mae_db": float(np.mean(np.abs(err))), "heldout_p99_abs_db": float(np.quantile(np.abs(err), 0.99)),
        "heldout_max_abs_db": float(np.max(np.abs(err))),
        "inference_rows": rows, "inference_ms": inf_ms, "inference_channel_evals_per_s": rows / (inf_ms * 1e-3),
        "inference_tflops": flops / (inf_ms * 1e-3) / 1e12,
        "gemm_8192": gemm,
        "per_link_network": link_net,
        "no_network_baseline": {"what": "each channel's mean training label",
                                "heldout_mae_db": float(np.mean(np.abs(base_err)))}}), flush=True)
    return 0


def run_ridge_types(args):
    """The benchmark's 120-channel C+L grid over ten spans of three types (80, 70
    and 90 km in turn, the 70 km spans with 0.17 dB/km and 20 ps/nm/km): the
    configured 32 x 32 rule and the ridge-resolving rule (--ridge-nodes per
    piece), each in FP32C and FP64, device ms per evaluation (CUDA events, L2
    flushed between steps), FP32C against FP64 per channel and the configured
    rule against the resolved one.  Prints one JSON line."""
    import numpy as np
    import torch
    from paper_2412_11614_gb300 import _build, egn, workloads as W
    _build.build()
    torch.cuda.set_device(0)
    wl = W.config_cl(n_ch=args.n_ch)
    for i, sp in enumerate(wl.spans):
        sp.length_m = (80e3, 70e3, 90e3)[i % 3]
        if i % 3 == 1:
            sp.alpha_db_km = 0.17
            sp.D_ps_nm_km = 20.0
    ln = egn.link_from_workload(wl)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
    ms, eta = {}, {}
    for rule, nodes in (("gl32", 32), ("ridge", args.ridge_nodes)):
        ln.set_node_rule(egn.EGN_RULE_RIDGE if rule == "ridge" else egn.EGN_RULE_GL, 4)
        for prec, pr in (("fp32c", egn.EGN_PREC_FP32C), ("fp64", egn.EGN_PREC_FP64)):
            o = egn.make_opts(gl_order=nodes, dz_km=wl.dz_km, precision=pr, terms=egn.EGN_TERMS_EGN,
                              stream=stream.cuda_stream)
            steps = 3 if prec == "fp32c" else 1
            ms[(rule, prec)], eta[(rule, prec)] = timed_evals(ln, o, wl.n_ch, stream, flush, steps=steps, warm=1)
    ln.close()
    db = lambda a, b: np.abs(10 * np.log10(a / b))  # noqa: E731
    d = 10 * np.log10(eta[("gl32", "fp64")] / eta[("ridge", "fp64")])
    print(json.dumps({
        "workload": f"{wl.n_ch}ch x 64GBd C+L on 75GHz grid, 10 spans of three types (80/70/90 km; the 70 km spans "
                    "0.17 dB/km, 20 ps/nm/km), 2 dBm/ch, EGN, dz=1km",
        "ms": {f"{r}_{p}": v for (r, p), v in ms.items()},
        "channel_evals_per_s": {f"{r}_{p}": wl.n_ch / (v * 1e-3) for (r, p), v in ms.items()},
        "ridge_nodes_per_piece": args.ridge_nodes,
        "ridge_fp32c_max_db_vs_fp64": float(db(eta[("ridge", "fp32c")], eta[("ridge", "fp64")]).max()),
        "gl32_fp32c_max_db_vs_fp64": float(db(eta[("gl32", "fp32c")], eta[("gl32", "fp64")]).max()),
        "gl32_minus_ridge_db": {"mean": float(d.mean()), "min": float(d.min()), "max": float(d.max())}}), flush=True)
    return 0


def run_dz_sweep(args):
    """The segment length trade-off of Sec. III-D on the GPU (Fig. 11 and 12
    analogues).  Table I links (31 central channels, Cr 1.12, QPSK, 1 and 10
    spans): the segment form at dz = 1..7 km in FP64 and FP32C and the Maclaurin
    form, each against the FP64 integral form.  Table II (101 ch x 100 GBd, about
    10 THz): the same against the FP64 segment form at dz = 0.125 km (the integral
    form's quarter-period pieces number ~1e6 per point there).  Errors per channel
    in dB, device ms per evaluation.  One JSON line per link."""
    import numpy as np
    import torch
    from paper_2412_11614_gb300 import _build, egn, workloads as W
    _build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()

    def evaluate(ln, n_ch, reps, **kw):
        opts = egn.make_opts(gl_order=16, stream=stream.cuda_stream, **kw)
        ws = torch.empty(ln.workspace_size(opts), dtype=torch.uint8, device="cuda")
        eta = torch.empty(n_ch, dtype=torch.float64, device="cuda")
        pn = torch.empty(n_ch, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            if reps > 1:
                ln.nli_eta_device(opts, ws, eta, pn)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(reps):
                ln.nli_eta_device(opts, ws, eta, pn)
            t1.record(stream)
        t1.synchronize()
        return eta.cpu().numpy(), t0.elapsed_time(t1) / reps

    cases = [("Table I, 31 ch, 1 x 100 km, Cr 1.12, QPSK", W.table1(n_spans=1, cr=1.12, fmt="QPSK", gl_order=16, n_ch=31),
              dict(mu_form=egn.EGN_MU_INTEGRAL, precision=egn.EGN_PREC_FP64), "FP64 integral form"),
             ("Table I, 31 ch, 10 x 100 km, Cr 1.12, QPSK", W.table1(n_spans=10, cr=1.12, fmt="QPSK", gl_order=16, n_ch=31),
              dict(mu_form=egn.EGN_MU_INTEGRAL, precision=egn.EGN_PREC_FP64), "FP64 integral form"),
             ("Table II, 101 ch x 100 GBd at 101 GHz, 1 x 100 km, QPSK", W.table2(fmt="QPSK", gl_order=16),
              dict(dz_km=0.125, precision=egn.EGN_PREC_FP64), "FP64 segment form, dz 0.125 km")]
    for name, wl, ref_kw, ref_name in cases:
        ln = egn.link_from_workload(wl)
        n = wl.n_ch
        ref, ref_ms = evaluate(ln, n, 1, **ref_kw)
        rdb = 10 * np.log10(ref)
        rows = {}
        for label, kw in ([(f"segment fp64 dz {d}", dict(dz_km=float(d), precision=egn.EGN_PREC_FP64)) for d in range(1, 8)] +
                          [(f"segment fp32c dz {d}", dict(dz_km=float(d), precision=egn.EGN_PREC_FP32C)) for d in range(1, 8)] +
                          [("maclaurin fp64", dict(mu_form=egn.EGN_MU_MACLAURIN, precision=egn.EGN_PREC_FP64))]):
            eta, ms = evaluate(ln, n, 3, **kw)
            err = 10 * np.log10(eta) - rdb
            rows[label] = {"ms": ms, "mae_db": float(np.mean(np.abs(err))), "max_abs_db": float(np.max(np.abs(err)))}
        print(json.dumps({"workload": name + ", 16 x 16 Gauss-Legendre, EGN", "reference": ref_name,
                          "reference_ms": ref_ms, "results": rows}), flush=True)
        ln.close()
    return 0


def run_f3d(args):
    """The f-integrated (3-D) EGN of Eq. 17-21 on the 120-channel link: n_f
    Gauss-Legendre nodes over each COI band, each a full evaluation with the
    islands planned at that frequency (egn_nli_eta_3d, host API, wall clock),
    and its difference from the white-NLI value.  One JSON line."""
    import numpy as np
    import torch
    from paper_2412_11614_gb300 import _build, egn, workloads as W
    _build.build()
    torch.cuda.set_device(0)
    wl = W.config_cl(n_ch=args.n_ch)
    ln = egn.link_from_workload(wl)
    prec = egn.EGN_PREC_FP32C if args.precision == "fp32c" else egn.EGN_PREC_FP64
    opts = egn.make_opts(gl_order=wl.gl_order, dz_km=wl.dz_km, precision=prec, terms=egn.EGN_TERMS_EGN)
    white, _ = ln.nli_eta(opts)
    ln.nli_eta_3d(opts, args.f3d)  # warm-up (tables, workspace)
    reps = max(1, args.steps)
    t0 = time.perf_counter()
    for _ in range(reps):
        e3, _ = ln.nli_eta_3d(opts, args.f3d)
    dt = (time.perf_counter() - t0) / reps
    diff = 10 * np.log10(e3 / white)
    print(json.dumps({
        "workload": f"{wl.n_ch}ch C+L link of the benchmark, f-integrated EGN, {args.f3d} Gauss-Legendre nodes "
                    f"per COI band, {args.precision}",
        "n_f": args.f3d, "seconds_per_evaluation": dt, "channel_evals_per_s": wl.n_ch / dt,
        "f3d_minus_white_db": {"mean": float(diff.mean()), "min": float(diff.min()), "max": float(diff.max()),
                               "centre": float(diff[wl.n_ch // 2]), "edge": float(diff[0])}}), flush=True)
    ln.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32c", choices=["fp32c", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the plain FP64 GPU integrator leg and the launch-power sweep")
    ap.add_argument("--no-sweep", action="store_true", help="skip the -2..+4 dBm/ch launch-power sweep")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-ridge", action="store_true", help="skip the ridge-resolving rule (FP64 and FP32C evaluations)")
    ap.add_argument("--ridge-nodes", type=int, default=16, help="nodes per piece of the ridge-resolving rule")
    ap.add_argument("--ridge-types", action="store_true",
                    help="both node rules in both precisions on the 120-channel grid over spans of three types")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the FP32, FP32x2, FP64 and MUFU pipe peaks with the probe kernels")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--n-ch", type=int, default=120, help="channels of the C+L grid (120 = the benchmark)")
    ap.add_argument("--points-per-thread", type=int, default=4, choices=[2, 4, 8],
                    help="launch-shape tuning of the FP32C D/G/H pass")
    ap.add_argument("--mu-compare", action="store_true",
                    help="time and compare the integral, segment and Maclaurin forms of mu (Table I links)")
    ap.add_argument("--mu-n-ch", type=int, default=31)
    ap.add_argument("--mu-gl", type=int, default=16)
    ap.add_argument("--batch", action="store_true",
                    help="time a batch of small links: one by one vs one graph launch")
    ap.add_argument("--batch-links", "--links", type=int, default=24, dest="batch_links")
    ap.add_argument("--batch-random", action="store_true", help="the batch is seeded heterogeneous random links")
    ap.add_argument("--dz-sweep", action="store_true", help="segment length trade-off on Table I and II links")
    ap.add_argument("--gemm", type=int, default=0, metavar="G", help="time the surrogate's G^3 tensor-core GEMM")
    ap.add_argument("--jsonl", default=None, metavar="PATH",
                    help="also append the JSON line, with a hash of its workload and configuration, to PATH")
    ap.add_argument("--f3d", type=int, default=0, metavar="NF",
                    help="time the f-integrated EGN with NF nodes per COI band against the white-NLI value")
    ap.add_argument("--surrogate", action="store_true", help="train and evaluate the MLP surrogate")
    ap.add_argument("--sur-train", type=int, default=4096)
    ap.add_argument("--sur-test", type=int, default=256)
    ap.add_argument("--sur-steps", type=int, default=2000)
    ap.add_argument("--sur-rule", choices=("gl", "ridge"), default="gl",
                    help="node rule of the surrogate's labels (ridge: --ridge-nodes per piece)")
    ap.add_argument("--sur-labels", default=None,
                    help="directory of sharded label files with a resume index (labels computed only where missing)")
    args = ap.parse_args()
    if args.peaks:
        import torch
        from paper_2412_11614_gb300 import _build
        _build.build()
        torch.cuda.set_device(0)
        st = torch.cuda.Stream()
        res = measure_peaks(list(PROBES), st, reps=max(5, args.steps), sampler=ClockSampler(gpu_id_for_smi(0)))
        res["gpu"] = torch.cuda.get_device_name(0)
        print(json.dumps(res), flush=True)
        return 0
    if args.surrogate:
        return run_surrogate(args)
    if args.ridge_types:
        return run_ridge_types(args)
    if args.f3d:
        return run_f3d(args)
    if args.dz_sweep:
        return run_dz_sweep(args)
    if args.gemm:
        import torch
        from paper_2412_11614_gb300 import _build
        _build.build()
        torch.cuda.set_device(0)
        print(json.dumps(gemm_roofline(args.gemm, args.steps)), flush=True)
        return 0
    if args.mu_compare:
        return run_mu_compare(args)
    if args.batch:
        return run_batch_compare(args)
    if args.warmup < 3:
        log("warmup raised to 3 (timing rule)")
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2412_11614_gb300 import _build, egn, workloads as W
    _build.build()
    prec = egn.EGN_PREC_FP32C if args.precision == "fp32c" else egn.EGN_PREC_FP64
    wl = W.config_cl(n_ch=args.n_ch)
    n_ch = wl.n_ch
    stream = torch.cuda.Stream()

    # inputs resident: link, comb, workspace, outputs
    ln = egn.link_from_workload(wl)
    opts = egn.make_opts(gl_order=wl.gl_order, dz_km=wl.dz_km, precision=prec, terms=egn.EGN_TERMS_EGN,
                         stream=stream.cuda_stream)
    n_isl, _, n_half, n_e, n_f = ln.island_count()
    ws = torch.empty(ln.workspace_size(opts), dtype=torch.uint8, device="cuda")
    eta = torch.empty(n_ch, dtype=torch.float64, device="cuda")
    pnli = torch.empty(n_ch, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    ln.set_profiling(True)
    ln.set_tuning(egn.EGN_TUNE_FP32C_POINTS_PER_THREAD, args.points_per_thread)

    def step():
        ln.nli_eta_device(opts, ws, eta, pnli)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            step()
    stream.synchronize()

    smi = ClockSampler(gpu_id_for_smi(local))
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stage = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    smi.start()
    time.sleep(0.3)
    t_wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            step()
            ends[i].record(stream)
            ends[i].synchronize()
            stage.append(ln.last_timings())
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    clocks = smi.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms, value, _ = aggregate_ranks(statistics.mean(step_ms), n_ch, device="cuda")

    # dominant kernel: the D/G/H integrator pass
    dgh_ms = statistics.mean(s["integrate_dgh"] for s in stage)
    n = wl.gl_order
    points = n_half * n * n  # islands evaluated (n1 <= n2); each has 1 or 2 outer panels: n x n points
    K = math.ceil(80.0 / wl.dz_km)
    flops = points * flops_per_point(args.precision, K)
    clk = clocks.get("sm_max_mhz") or 2070.0
    # measured pipe peaks (the library's probe kernels, this run, this GPU)
    peaks = measure_peaks(["ffma", "ffma2", "dfma", "mufu_sin"], stream, sampler=ClockSampler(gpu_id_for_smi(local)))
    pr = peaks["probes"]
    pclk = peaks["clocks"].get("sm_mhz")
    if args.precision == "fp32c":
        best = max(("ffma", "ffma2"), key=lambda k: pr[k]["tflops"])
        peak = pr[best]["tflops"]
        peak_note = (f"measured in this run: FP32 FMA probe ({'fma.rn.f32x2' if best == 'ffma2' else 'fma.rn.f32'} "
                     f"chains, egn_probe_launch, best of 5) at a median {pclk} MHz; derived "
                     f"152 SMs x 128 lanes x 2 FLOP x {clk:.0f} MHz = "
                     f"{SM_COUNT_GB300 * FP32_LANES_PER_SM * 2 * clk * 1e6 / 1e12:.1f}")
    else:
        peak = pr["dfma"]["tflops"]
        peak_note = f"measured in this run: FP64 FMA probe (fma.rn.f64 chains, egn_probe_launch) at a median {pclk} MHz"
    achieved = flops / (dgh_ms * 1e-3) / 1e12
    # DRAM bytes (read + write) of one FP32C D/G/H launch on the 120-channel
    # workload, from one ncu capture of that launch (dram__bytes_read.sum +
    # dram__bytes_write.sum); island keys and lists are read once, the terms
    # written stay in L2.  Valid for this kernel version only.
    traffic = 22996992 + 486656 if (args.precision == "fp32c" and n_ch == 120) else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_unit": "bytes per launch", "kernel": "integrate D/G/H pass",
                "peak_note": peak_note,
                "kernel_ms": dgh_ms, "flops_per_launch": flops,
                "peaks_measured": {k: {kk: v for kk, v in r.items() if kk != "ops_per_launch"} for k, r in pr.items()},
                "stage_ms": {k: statistics.mean(s[k] for s in stage) for k in stage[0]}}
    if args.precision == "fp32c":
        # special-function unit: per point of the D-only path one sine of the segment
        # angle, two sines of the phased array, one reciprocal and two cosines of the
        # raised-cosine shapes (the c_k table exponentials are not counted)
        mufu = points * MUFU_PER_POINT
        sfu_gops = mufu / (dgh_ms * 1e-3) / 1e9
        roofline.update({"sfu_achieved_gops": sfu_gops, "sfu_peak_gops": pr["mufu_sin"]["gops"],
                         "sfu_frac": sfu_gops / pr["mufu_sin"]["gops"], "sfu_ops_per_point": MUFU_PER_POINT,
                         "sfu_peak_note": "measured in this run: sin.approx.f32 probe (egn_probe_launch)"})

    # end to end through the host API: pinned inputs -> egn_set_wdm -> egn_nli_eta -> host outputs
    e2e_steps = args.e2e_steps or max(3, min(args.steps, 5))
    mom = [egn.egn_format_moments(f) for f in wl.formats]
    host_in = {k: torch.tensor(v, dtype=torch.float64).pin_memory() for k, v in
               dict(c=wl.centre_hz, r=wl.symbol_rate_baud, p=wl.launch_power_w, phi=[m[0] for m in mom],
                    psi=[m[1] for m in mom]).items()}
    ln2 = egn.Link(wl.spans)
    hopts = egn.make_opts(gl_order=wl.gl_order, dz_km=wl.dz_km, precision=prec, terms=egn.EGN_TERMS_EGN)
    for _ in range(2):
        ln2.set_wdm(*(host_in[k].numpy() for k in ("c", "r", "p", "phi", "psi")), wl.rolloff)
        ln2.nli_eta(hopts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ln2.set_wdm(*(host_in[k].numpy() for k in ("c", "r", "p", "phi", "psi")), wl.rolloff)
        e_host, _ = ln2.nli_eta(hopts)
    e2e_ms, e2e_value, _ = aggregate_ranks(1e3 * (time.perf_counter() - t0) / e2e_steps, n_ch, device="cuda")
    e2e_s = e2e_ms * 1e-3
    n_rows = n_ch * n_ch
    h2d = 5 * n_ch * 8 + 6 * n_ch * 8 + 2 * K * 8 + 2 * K * 4  # inputs + channel table + segment tables
    d2h = 3 * (n_rows + 1) * 4 + 2 * n_ch * 8 + 4             # island counts + eta, P_NLI + status
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "ms_per_step": e2e_s * 1e3, "api": "egn_set_wdm + egn_nli_eta (host buffers)"}
    ln2.close()

    extras = {}
    if rank == 0 and args.precision == "fp32c" and not args.no_fp64:
        extras = fp64_denominator(args, wl, ln, eta.cpu().numpy(), value / world, stream, flush)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, threads, desc, _, _ = oracle_rate(wl, 15.0)
        cpu = {"value": r, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc, "cpu": host_cpu()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32c" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if n_ch == 120 else WORKLOAD.replace("120ch", f"{n_ch}ch"),
                       "precision": args.precision, "points_per_thread": args.points_per_thread, "n_ch": n_ch,
                       "islands": n_isl,
                       "islands_evaluated": n_half, "e_islands": n_e, "f_islands": n_f, "points_per_step": points, "segments_K": K,
                       "l2": "flushed between steps (256 MB write outside the per-step events)",
                       "parallelism": f"replicas x{world}"},
            # per step: planner count, scan, emit; grouping count, tile scan, scan,
            # scatter; D/G/H, E, F; assembly
            "gpu_launches": 11 * args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "wall_s_timed_region": t_wall,
            "eta_db_sample": [float(10 * np.log10(x)) for x in eta.cpu().numpy()[:: 30]],
        }
        line.update(extras)
        emit(line, args.jsonl)
    ln.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
