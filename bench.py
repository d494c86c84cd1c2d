"""Benchmark of the hot path on the production-size workload.

Workload (one "step"): 16 sub-batches x 65536 forward rays on a misaligned
magnetar-like rotator (B0 = 1.6e14 G, P = 3.76 s, theta_m = 30 deg,
M = 1.5 Msun, R = 11 km), axion masses log-uniform in [1e-6, 5e-3] eV (one per
sub-batch, seed 1), rotation phase uniform per ray: conversion-surface
sampling (FP64) -> Dormand-Prince 5(4) trace to r = 1000 R (FP64 at rtol
1e-10, and mixed FP32/FP64 at rtol 1e-8) -> fixed-point binning into
64 x 32 x 128 (theta, phi, frequency) bins per sub-batch.  Inputs are
synthetic (SplitMix64 uniforms) and resident in HBM when the timed region
starts; the L2 is flushed (256 MiB write) before every timed step.

Reported: accepted ray-steps/s (value) of the fastest precision whose binned
flux is within 1e-6 (relative L1) of the FP64 oracle run on the same
uniforms, rays/s, the roofline of the trace kernel (FP64 or FP32 ALU), an
end-to-end number through the C ABI with host buffers, the oracle timed on
the host cores (cpu_baseline: the whole workload), and two further legs: the
backward image plane (1024 x 1024 pixels at 60 deg, impact parameters to
50 R, with oracle-checked pixels) and the adjoint gradient of a smoothed line
flux (2^18 rays; adjoint/forward time ratio, checkpoint memory).
``--impl reference`` times the oracle alone (the CPU reference arm) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ray-steps/s & rays/s at 1e-6 rel. flux err; mixed vs FP64; adjoint/forward ratio"
UNIT = "ray-steps/s"
NBINS = (64, 32, 128)
# ALU peaks: measured at the start of every run by rt_measure_alu_peak
# (independent FMA chains on every SM, CUDA events), which replaces these
# nominal values derived from the unit counts and the maximum clock (152 SMs x
# 2070 MHz; FP64 4 flop/clk/SM = 1.26 TFLOP/s; FP32 128 lanes x 2 flop/clk/SM
# = 80.5 TFLOP/s); both are reported.
SMS, CLK = 152, 2.070e9
FP64_KERNELS = "trace_fp64_kernel + tail_fp64_kernel (one trace call)"
PRECISIONS = ("fp64", "mixed", "df")
# arithmetic type of each path: FP64; FP32 stages with a double-float state;
# double-float (pairs of FP32) throughout
DTYPE = {"fp64": "f64", "mixed": "f32 (state f32x2)", "df": "f32x2"}
LC_CUT_KM = 0.0      # backward IR cut on the conversion length (Sec. 4.4): none
NOMINAL = {"fp64": SMS * 4 * CLK, "fp32": SMS * 256 * CLK}
PEAK = dict(NOMINAL)
PEAK_SOURCE = {"fp64": "nominal: 152 SMs x 4 FP64 flop/clk x 2070 MHz",
               "fp32": "nominal: 152 SMs x 256 FP32 flop/clk x 2070 MHz"}


def _measure_peaks(rt, stream):
    """Measured FP64 / FP32 multiply-add rates of this GPU, with the SM clock
    sampled while they run; they become the roofline denominators."""
    clk = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    m = rt.rt_measure_alu_peak(stream=stream)
    c = clk.stop()
    PEAK["fp64"], PEAK["fp32"] = m["fp64_flops"], m["fp32_flops"]
    for k, kk in (("fp64", "fp64_ms"), ("fp32", "fp32_ms")):
        PEAK_SOURCE[k] = (f"measured on this GPU by rt_measure_alu_peak (8 independent FMA "
                          f"chains per thread, every SM, one {m[kk]:.0f} ms launch timed with "
                          f"CUDA events; SM clock median {c['sm_mhz']} MHz); nominal "
                          f"{NOMINAL[k] / 1e12:.2f} TFLOP/s")
    return {"fp64_tflops": m["fp64_flops"] / 1e12, "fp32_tflops": m["fp32_flops"] / 1e12,
            "fp64_ms": m["fp64_ms"], "fp32_ms": m["fp32_ms"], "clocks": c,
            "nominal_fp64_tflops": NOMINAL["fp64"] / 1e12,
            "nominal_fp32_tflops": NOMINAL["fp32"] / 1e12}

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the trace
# kernel per traced ray, from one single-pass ncu capture of that kernel alone
# (one launch, caches flushed by ncu before it) on 2^21 rays of the heaviest
# benchmark star, cost-ordered claims, default launch shape and refill:
#   python profile_case.py --config config1 --precision <p> --claim-order cost --n 2097152
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none \
#       -k regex:<kernel> -s 1 -c 1 <the same command>
# (2^21 rays hold 134 MB of state, more than L2).  The bench scales it by the
# rays a launch traces; valid for the kernel sources with the given SHA-256
# prefix (null once they change).
TRAFFIC = {
    # precision -> (sources, digest, kernel, bytes per traced ray)
    "fp64": (('rt_device.cuh', 'rt_integrator.cuh', 'rt_trace.cu', 'rt_internal.h'),
             "ecbf401b4b0b6157", "trace_fp64_kernel", 334305792 / 2096328),
    "mixed": (('rt_device.cuh', 'rt_integrator.cuh', 'rt_backward.cuh', 'rt_trace_mixed.cu',
               'rt_internal.h'),
              "3283184d3aa6675e", "trace_mixed_kernel", 249587456 / 2096328),
    "df": (('rt_device.cuh', 'rt_integrator.cuh', 'rt_df.cuh', 'rt_trace_df.cu', 'rt_internal.h'),
           "f6456f701275e339", "trace_df_kernel", 392003840 / 2096328),
}


def _traffic(prec, rays):
    """DRAM bytes of the trace kernel for a launch tracing `rays` rays."""
    import hashlib
    files, digest, _, per_ray = TRAFFIC[prec]
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2309_08655_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if per_ray is None or h.hexdigest()[:16] != digest:
        return None
    return per_ray * rays


CLAIM = {"index": 0, "cost": 1}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=1 << 16,
                    help="rays per sub-batch in the CPU baseline (65536 = the whole "
                         "workload, which also gives the flux error against the oracle)")
    ap.add_argument("--no-backward", action="store_true",
                    help="skip the backward image-plane measurement")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint (gradient) measurement")
    ap.add_argument("--no-twisted", action="store_true",
                    help="skip the twisted-magnetosphere (Eq. neMag) workload")
    ap.add_argument("--claim-order", choices=["index", "cost"], default="cost",
                    help="order in which the FP64 kernels claim rays (rt_trace_opts.claim_order)")
    ap.add_argument("--no-rotating", action="store_true",
                    help="skip the rigidly rotating magnetosphere workload")
    ap.add_argument("--no-uneven", action="store_true",
                    help="skip the 256-instance uneven batch measurement")
    ap.add_argument("--no-equal-accuracy", action="store_true",
                    help="skip the mixed-vs-FP64 comparison at equal flux accuracy")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
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
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _flops_per_attempt(rt):
    return rt.rt_flops_per_step(0, 0)


def _roofline(prec, fl, fl_df, attempts, rays, promoted_attempts, t):
    """ALU roofline of one trace call of `t` seconds: counted operations per
    attempt (and per ray for the initial step) against the measured peak of
    the pipe that executes them."""
    if prec == "fp64":
        flops = attempts * fl[1] + rays * fl[2]
        r = {"kernel": FP64_KERNELS, "peak": PEAK["fp64"], "peak_source": PEAK_SOURCE["fp64"],
             "flops_per_attempt": fl[1]}
    elif prec == "mixed":
        flops = (attempts - promoted_attempts) * fl[1] + rays * fl[2]
        r = {"kernel": "trace_mixed_kernel (+ FP64 pass for promoted rays)", "peak": PEAK["fp32"],
             "peak_source": PEAK_SOURCE["fp32"], "flops_per_attempt": fl[1]}
    else:
        # the FP32 operations the double-float arithmetic executes; the FP64
        # operations they stand for reported beside them
        flops = attempts * fl_df[1] + rays * (2 * fl_df[0] + 600)
        r = {"kernel": "trace_df_kernel", "peak": PEAK["fp32"], "peak_source": PEAK_SOURCE["fp32"],
             "flops_per_attempt": fl_df[1],
             "flops_counted": "FP32 operations of the double-float arithmetic (sum 11, product 10, "
                              "rsqrt 24; rt_flops_per_step_df)",
             "fp64_equivalent_flops_per_attempt": fl[1],
             "fp64_equivalent_tflops": (attempts * fl[1] + rays * fl[2]) / t / 1e12}
    r.update({"bound": "alu", "achieved": flops / t / 1e12, "unit": "TFLOP/s",
              "frac": flops / t / r["peak"], "traffic": _traffic(prec, rays),
              "traffic_kernel": TRAFFIC[prec][2]})
    r["peak"] = r["peak"] / 1e12
    return r


class _Pipelined:
    """K copies of one step's batch (16 sub-batches) as one batch: one sampling
    launch per sub-batch, one persistent trace launch, one binning pass per
    sub-batch."""

    def __init__(self, rt, stars, nper, nsub, K, u, dev, stream, nbins, cfg, ws=1):
        import torch
        self.rt, self.stream, self.nbins, self.cfg = rt, stream, nbins, cfg
        self.stars = list(stars) * K
        self.batch = rt.Batch(self.stars, [nper] * (nsub * K))
        self.ws, self.nper = ws, nper
        if ws > 1:        # this rank's share of every star's rays (see run_ours)
            rt.rt_batch_set_norm(self.batch, [ws * nper] * (nsub * K))
        N = nsub * nper
        self.u = u.repeat(1, K).contiguous()
        f64 = torch.float64
        self.st = torch.empty((8, K * N), dtype=f64, device=dev)
        self.w = torch.empty(K * N, dtype=f64, device=dev)
        self.s = torch.empty(K * N, dtype=torch.uint8, device=dev)
        self.hist = torch.empty((K * nsub,) + tuple(nbins), dtype=f64, device=dev)
        self.hist_host = torch.empty(self.hist.shape, dtype=f64).pin_memory()
        self.oor = torch.empty(K * nsub, dtype=f64, device=dev)
        self.ctr = torch.zeros(8, dtype=torch.int64, device=dev)
        self.ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        self.acc = (torch.empty((K * nsub, rt.bin_acc_entries(*nbins)), dtype=torch.int64,
                                device=dev) if ws > 1 else None)

    def run(self, opts):
        rt, cs = self.rt, self.stream
        self.ctr.zero_()
        rt.rt_sample_batch(self.batch, self.u, self.st, self.w, self.s, stream=cs)
        self.ev[0].record(cs)
        rt.rt_trace_batch(self.batch, self.st, self.s, None, None, self.ctr, opts, stream=cs)
        self.ev[1].record(cs)
        if self.ws > 1:
            from paper_2309_08655_gb300 import shard
            ns = len(self.stars)
            shard.bin_sharded(rt, self.stars, [j * self.nper for j in range(ns + 1)],
                              self.batch.N, [self.ws * self.nper] * ns, self.st, self.w, self.s,
                              self.nbins, self.cfg["nu_lo"], self.cfg["nu_hi"], self.acc,
                              self.hist, self.oor, stream=cs)
        else:
            rt.rt_bin_batch(self.batch, self.st, self.w, self.s, *self.nbins, self.cfg["nu_lo"],
                            self.cfg["nu_hi"], self.hist, self.oor, stream=cs)


def _workload():
    from paper_2309_08655_gb300 import inputs as I
    cfg = I.CONFIG1
    return cfg, I.stars_config1(cfg["seed"], cfg["nsub"])


def _oracle_sample_run(stars, cfg, per_sub, nthreads, seed_base=None, want_hist=False,
                       states=None):
    """Oracle on the first ``per_sub`` rays of each non-empty sub-batch
    (sampling, tracing and binning, as on the GPU).  Returns (accepted steps,
    traced rays, seconds, per-sub-batch histograms or None); with a dict
    ``states``, also each sub-batch's end states and statuses in it."""
    import numpy as np
    import oracle
    from paper_2309_08655_gb300 import inputs as I
    steps = rays = 0
    hists = np.zeros((len(stars),) + NBINS) if want_hist else None
    base = cfg["seed"] * 1000 if seed_base is None else seed_base
    t0 = time.perf_counter()
    for j, kw in enumerate(stars):
        sv = oracle.star_vector(**kw)
        u = I.sample_uniforms(base + j, per_sub)
        st, w, s = oracle.sample(sv, u, nthreads)
        if not (s == oracle.RAY_READY).any():
            continue
        na, nr, _ = oracle.trace_forward(sv, oracle.trace_opts(rtol=cfg["rtol"],
                                         r_out_over_R=cfg["r_out_over_R"]), st, s, nthreads)
        h, _ = oracle.bin_rays(sv, st, w, s, *NBINS, cfg["nu_lo"], cfg["nu_hi"])
        if want_hist:
            hists[j] = h
        if states is not None:
            states[j] = (st, s)
        steps += int(na.sum())
        rays += int(np.sum(s != oracle.RAY_NO_ROOT))
    return steps, rays, time.perf_counter() - t0, hists


def _cpu_baseline(stars, cfg, per_sub, states=None):
    nthreads = os.cpu_count() or 1
    full = per_sub >= cfg["n_per_sub"]
    steps, rays, dt, hists = _oracle_sample_run(stars, cfg, min(per_sub, cfg["n_per_sub"]),
                                                nthreads, want_hist=full,
                                                states=states if full else None)
    what = ("the whole workload" if full else f"the first {per_sub} rays of each sub-batch")
    return {"value": steps / dt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "rays_per_s": rays / dt, "seconds": dt,
            "sample": f"{what} (16 sub-batches; empty ones sample only): {rays} traced rays, "
                      f"{steps} accepted steps, FP64 at rtol {cfg['rtol']:g}"}, hists


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    cfg, stars = _workload()
    per = 512
    for _ in range(args.warmup):
        _oracle_sample_run(stars, cfg, 64, os.cpu_count() or 1)
    tot_steps = tot_rays = 0
    tot_t = 0.0
    for _ in range(args.steps):
        s, r, dt, _ = _oracle_sample_run(stars, cfg, per, os.cpu_count() or 1)
        tot_steps += s
        tot_rays += r
        tot_t += dt
    v = tot_steps / tot_t
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": cfg["name"] + " (bounded sample)", "rays_per_sub_batch": per,
                   "rtol": cfg["rtol"], "r_out_over_R": cfg["r_out_over_R"]},
        "rays_per_s": tot_rays / tot_t,
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count() or 1,
                         "kind": "oracle",
                         "sample": f"first {per} rays of each of the 16 sub-batches per step"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line, default=_plain))


def run_ours(args):
    import numpy as np
    import torch

    from paper_2309_08655_gb300 import build as B
    from paper_2309_08655_gb300 import inputs as I
    from paper_2309_08655_gb300 import rt
    from paper_2309_08655_gb300 import shard

    ws, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B.build()
    dev = torch.device("cuda", local)
    cfg, stars_kw = _workload()
    nsub, nper = cfg["nsub"], cfg["n_per_sub"]
    N = nsub * nper
    nth, nph, nnu = NBINS
    stars = [rt.Star(rt.make_params(**kw)) for kw in stars_kw]
    batch = rt.Batch(stars, [nper] * nsub)
    # weak scaling: on N ranks every star carries N x 65536 rays, rank r the
    # contiguous range r (its uniforms, the whole workload's weight
    # normalisation); the per-star spectra are combined exactly at the end of
    # each step (int64 all-reduce of the fixed-point sums)
    first, _ = shard.ray_range(ws * nper, ws, rank)
    seeds = [cfg["seed"] * 1000 + j for j in range(nsub)]
    u_host = torch.from_numpy(np.ascontiguousarray(np.concatenate(
        [I.sample_uniforms(sd, nper, first) for sd in seeds], axis=1))).pin_memory()
    u = u_host.to(dev)
    if ws > 1:
        rt.rt_batch_set_norm(batch, [ws * nper] * nsub)
    acc = torch.empty((nsub, rt.bin_acc_entries(*NBINS)), dtype=torch.int64, device=dev)
    offsets = [j * nper for j in range(nsub + 1)]
    st = torch.empty((8, N), dtype=torch.float64, device=dev)
    w = torch.empty(N, dtype=torch.float64, device=dev)
    s = torch.empty(N, dtype=torch.uint8, device=dev)
    hist = torch.empty((nsub, nth, nph, nnu), dtype=torch.float64, device=dev)
    oor = torch.empty(nsub, dtype=torch.float64, device=dev)
    ctr = torch.zeros(8, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    opts = {
        "fp64": rt.make_opts(rtol=cfg["rtol"], r_out_over_R=cfg["r_out_over_R"],
                             precision=rt.PREC_FP64, max_steps=cfg["max_steps"],
                             claim_order=CLAIM[args.claim_order]),
        "mixed": rt.make_opts(rtol=cfg["rtol_mixed"], r_out_over_R=cfg["r_out_over_R"],
                              precision=rt.PREC_MIXED, max_steps=cfg["max_steps"],
                              claim_order=CLAIM[args.claim_order]),
        "df": rt.make_opts(rtol=cfg["rtol"], r_out_over_R=cfg["r_out_over_R"],
                           precision=rt.PREC_DF, max_steps=cfg["max_steps"],
                           claim_order=CLAIM[args.claim_order]),
    }
    ev_t = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # kernels of one trace call: FP64 cost-ordered = express select + rank +
    # persistent + tail; FP64 index order = persistent + tail; mixed = FP32 +
    # FP64 pass + tail.  A pipelined run of K steps: one sampling launch and
    # three binning launches per star-step, plus one trace call.
    trace_launches = {"fp64": 4 if args.claim_order == "cost" else 2, "mixed": 3, "df": 1}

    def step(prec, uin=None):
        ctr.zero_()
        rt.rt_sample_batch(batch, u if uin is None else uin, st, w, s, stream=stream)
        ev_t[0].record(stream)
        rt.rt_trace_batch(batch, st, s, None, None, ctr, opts[prec], stream=stream)
        ev_t[1].record(stream)
        if ws > 1:
            shard.bin_sharded(rt, stars, offsets, N, [ws * nper] * nsub, st, w, s, NBINS,
                              cfg["nu_lo"], cfg["nu_hi"], acc, hist, oor, stream=stream)
        else:
            rt.rt_bin_batch(batch, st, w, s, nth, nph, nnu, cfg["nu_lo"], cfg["nu_hi"], hist,
                            oor, stream=stream)

    res = {}
    fl = _flops_per_attempt(rt)
    fl_df = rt.rt_flops_per_step_df(0, 0)
    peaks = _measure_peaks(rt, stream)
    clocks = Clocks(local)
    clocks.start()
    for prec in PRECISIONS:
        for _ in range(args.warmup):
            step(prec)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t_steps, t_trace, c_sum = [], [], np.zeros(8)
        for _ in range(args.steps):
            flush.fill_(1)                  # L2 flush, outside the timed events
            e0.record(stream)
            step(prec)
            e1.record(stream)
            torch.cuda.synchronize()
            t_steps.append(e0.elapsed_time(e1) / 1e3)
            t_trace.append(ev_t[0].elapsed_time(ev_t[1]) / 1e3)
            c_sum += ctr.cpu().numpy()
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        T, acc_all, rays_all = shard.reduce_totals(sum(t_steps), c_sum[0], c_sum[2], dev)
        attempts = (c_sum[0] + c_sum[1]) / args.steps
        rays_launch = c_sum[2] / args.steps
        promoted_attempts = c_sum[5] / args.steps
        t_tr = statistics.mean(t_trace)
        roof = _roofline(prec, fl, fl_df, attempts, rays_launch, promoted_attempts, t_tr)
        if prec == "mixed":
            roof.update({"promoted_rays_per_step": c_sum[4] / args.steps,
                         "promoted_fp64_attempts_per_step": promoted_attempts})
        roof.update({"attempts_per_launch": attempts, "trace_ms_per_launch": 1e3 * t_tr})
        res[prec] = {"value": acc_all / T, "rays_per_s": rays_all / T,
                     "ms_per_step": 1e3 * T / args.steps, "roofline": roof,
                     "accepted_steps_per_step": c_sum[0] / args.steps,
                     "rejected_steps_per_step": c_sum[1] / args.steps,
                     "rtol": opts[prec].rtol,
                     "hist": hist.cpu().numpy().copy(),
                     "end": (st.cpu().numpy().copy(), s.cpu().numpy().copy()),
                     "statuses": np.bincount(s.cpu().numpy(), minlength=8).tolist()}
    hists = {p: res[p].pop("hist") for p in PRECISIONS}
    ends = {p: res[p].pop("end") for p in PRECISIONS}
    # continuous batching: the K steps' batches (16 sub-batches each) in one
    # persistent launch, so the bulk of later batches overlaps the long rays of
    # earlier ones; the same work per step (rays that finish in the six-lane
    # tail kernel may differ from one launch per step by rounding)
    K = min(args.steps, 64)
    P = _Pipelined(rt, stars, nper, nsub, K, u, dev, stream, NBINS, cfg, ws)
    for prec in PRECISIONS:
        P.run(opts[prec])                   # untimed pass of this path
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        flush.fill_(1)
        e0.record(stream)
        P.run(opts[prec])
        e1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        c = P.ctr.cpu().numpy()
        T, acc_all, rays_all = shard.reduce_totals(e0.elapsed_time(e1) / 1e3, c[0], c[2], dev)
        t_tr = P.ev[0].elapsed_time(P.ev[1]) / 1e3
        attempts = c[0] + c[1]
        roof = _roofline(prec, fl, fl_df, attempts, c[2], c[5], t_tr)
        roof.update({"attempts_per_launch": attempts, "trace_ms_per_launch": 1e3 * t_tr,
                     "steps_per_launch": K})
        hp = P.hist.cpu().numpy()
        same = all(np.array_equal(hp[k * nsub:(k + 1) * nsub], hists[prec]) for k in range(K))
        res[prec]["pipelined"] = {"value": acc_all / T, "rays_per_s": rays_all / T,
                                  "ms_per_step": 1e3 * T / K, "steps_per_launch": K,
                                  "roofline": roof, "hist_equal_to_sequential": bool(same)}
    clk = clocks.stop()

    def l1(a, b):
        return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))

    res["mixed"]["flux_l1_vs_fp64"] = l1(hists["mixed"], hists["fp64"])
    res["df"]["flux_l1_vs_fp64"] = l1(hists["df"], hists["fp64"])
    equal_acc = None
    if ws == 1 and not args.no_equal_accuracy:
        equal_acc = _equal_accuracy(rt, batch, u, st, w, s, hist, oor, ctr, cfg, stream,
                                    hists["mixed"], res["mixed"]["roofline"]["trace_ms_per_launch"],
                                    l1)
    # the oracle on the same workload: the CPU baseline and, when it covers the
    # whole workload, the flux error of each precision against it
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        or_states = {}
        cpu, h_or = _cpu_baseline(stars_kw, cfg, args.cpu_sample, or_states)
        if h_or is not None and ws == 1:
            for p in PRECISIONS:
                res[p]["flux_l1_vs_oracle"] = l1(hists[p], h_or)
            res["mixed"]["endpoint_error_vs_oracle"] = _endpoint_errors(ends, or_states, nper)
    # headline: the fastest precision whose binned flux is within 1e-6 (relative
    # L1) of the FP64 oracle; without the oracle, of the FP64 GPU path
    ok = [p for p in PRECISIONS
          if res[p].get("flux_l1_vs_oracle", res[p].get("flux_l1_vs_fp64", 0.0)) <= 1e-6]
    head = min(ok, key=lambda p: res[p]["pipelined"]["ms_per_step"]) if ok else "fp64"
    # end to end through the C ABI with host buffers: H2D of the K steps'
    # uniforms from pinned memory, the pipelined launch, D2H of the histograms
    flush.fill_(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(K):
        P.u[:, k * N:(k + 1) * N].copy_(u_host, non_blocking=True)
    P.run(opts[head])
    P.hist_host.copy_(P.hist, non_blocking=True)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    t_e2e_all, acc_e2e, _ = shard.reduce_totals(t_e2e, float(P.ctr[0]), 0.0, dev)
    e2e_val = acc_e2e / t_e2e_all
    # the further legs run on a single GPU only (a scaling run times the main step)
    back = None
    if ws == 1 and not args.no_backward:
        back = _backward_leg(args, dev, stream, fl, rank)
    adj = None
    if ws == 1 and not args.no_adjoint:
        adj = _adjoint_leg(args, dev)
    uneven = None
    if ws == 1 and not args.no_uneven:
        uneven = _uneven_leg(args, dev)
    twisted = None
    if ws == 1 and not args.no_twisted:
        twisted = _twisted_leg(args, dev, stream)
    rotating = None
    if ws == 1 and not args.no_rotating:
        rotating = _rotating_leg(args, dev, stream)
    if rank != 0:
        return
    H = res[head]
    HP = H["pipelined"]
    line = {
        "metric": METRIC, "value": HP["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": HP["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[head],
        "data": "synthetic",
        "config": {"workload": cfg["name"], "rays_per_step": N, "sub_batches": nsub,
                   "parallelism": ("single GPU" if ws == 1 else
                                   f"each star's rays split into {ws} contiguous ranges, one per "
                                   f"rank; per-star int64 fixed-point spectra all-reduced (MAX "
                                   f"of the largest weight, then SUM) every step"),
                   "rtol": H["rtol"], "r_out_over_R": cfg["r_out_over_R"],
                   "max_steps": cfg["max_steps"], "bins": list(NBINS), "precision": head,
                   "launch": f"continuous batching: the {K} timed steps' 16 sub-batches each "
                             f"in one persistent trace launch (per-step histograms compared "
                             f"with one launch per step, whose numbers are under "
                             f"'{head}' -> 'ms_per_step')",
                   "claim_order": args.claim_order,
                   "l2": f"inputs larger than L2 ({K} x 117 MB) and L2 flushed (256 MiB "
                         f"write) before the timed region"},
        "rays_per_s": HP["rays_per_s"],
        "flux_l1_vs_oracle": H.get("flux_l1_vs_oracle"),
        "roofline": HP["roofline"],
        "fp64": res["fp64"], "mixed": res["mixed"], "df": res["df"],
        "mixed_vs_fp64_rays_per_s": res["mixed"]["rays_per_s"] / res["fp64"]["rays_per_s"],
        "df_vs_fp64_rays_per_s": res["df"]["rays_per_s"] / res["fp64"]["rays_per_s"],
        "mixed_vs_fp64_equal_accuracy": equal_acc,
        "backward": back,
        "adjoint_forward_ratio": adj["adjoint_forward_ratio"] if adj else None,
        "adjoint": adj,
        "uneven_batch": uneven,
        "twisted_magnetosphere": twisted,
        "rotating_magnetosphere": rotating,
        "cpu_baseline": cpu,
        "alu_peaks": peaks,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": u_host.numel() * 8,
                "d2h_bytes_per_step": hist.numel() * 8},
        "gpu_launches": 4 * nsub * K + trace_launches[head],
        "clocks": clk,
    }
    print(json.dumps(line, default=_plain))


def _equal_accuracy(rt, batch, u, st, w, s, hist, oor, ctr, cfg, stream, hist_mixed,
                    ms_mixed, l1):  # ms_mixed: the mixed path's trace call
    """The mixed path against the plain FP64 path at equal binned-flux
    accuracy.  Reference: the FP64 flux at rtol 1e-12.  The FP64 path's
    distance from it and its time at rtol 1e-8, 1e-9, 1e-10; the mixed path's
    at its default rtol (the main leg's run) and at rtol 1e-9; the
    double-float path's at rtol 1e-9 and 1e-10.  For each mixed or
    double-float row the loosest FP64 rtol at least as close to the reference
    (the tightest one tried if none is) sets the FP64 time of its ratio.  One
    launch per step for both, as the mixed path's own timing."""
    import torch
    nth, nph, nnu = NBINS

    def run(rtol, prec):
        o = rt.make_opts(rtol=rtol, r_out_over_R=cfg["r_out_over_R"], precision=prec,
                         max_steps=cfg["max_steps"] * 4, claim_order=CLAIM["cost"])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctr.zero_()
        rt.rt_sample_batch(batch, u, st, w, s, stream=stream)
        e0.record(stream)
        rt.rt_trace_batch(batch, st, s, None, None, ctr, o, stream=stream)
        e1.record(stream)
        rt.rt_bin_batch(batch, st, w, s, nth, nph, nnu, cfg["nu_lo"], cfg["nu_hi"], hist, oor,
                        stream=stream)
        torch.cuda.synchronize()
        return hist.cpu().numpy().copy(), e0.elapsed_time(e1), int(ctr[0]), int(ctr[4])

    h_ref, t_ref, _, _ = run(1e-12, rt.PREC_FP64)
    rows = []
    for rtol in (1e-8, 1e-9, 1e-10):
        h, t, acc, _ = run(rtol, rt.PREC_FP64)
        rows.append({"rtol": rtol, "flux_l1_vs_rtol1e-12": l1(h, h_ref), "trace_ms": t,
                     "accepted_steps": acc})
    mixed = [{"rtol": cfg["rtol_mixed"], "flux_l1_vs_rtol1e-12": l1(hist_mixed, h_ref),
              "trace_ms": ms_mixed}]
    h, t, acc, promoted = run(1e-9, rt.PREC_MIXED)
    mixed.append({"rtol": 1e-9, "flux_l1_vs_rtol1e-12": l1(h, h_ref), "trace_ms": t,
                  "accepted_steps": acc, "promoted_rays": promoted})
    df = []
    for rtol in (1e-9, 1e-10):
        h, t, acc, _ = run(rtol, rt.PREC_DF)
        df.append({"rtol": rtol, "flux_l1_vs_rtol1e-12": l1(h, h_ref), "trace_ms": t,
                   "accepted_steps": acc})
    for m in mixed + df:
        ok = [r for r in rows if r["flux_l1_vs_rtol1e-12"] <= m["flux_l1_vs_rtol1e-12"]]
        pick = ok[0] if ok else rows[-1]
        m.update({"fp64_rtol_at_equal_accuracy": pick["rtol"],
                  "fp64_at_least_as_accurate": bool(ok),
                  "speedup_vs_fp64": pick["trace_ms"] / m["trace_ms"]})
    return {"reference": "FP64 rtol 1e-12 binned flux (trace %.0f ms)" % t_ref,
            "mixed_rtol": cfg["rtol_mixed"],
            "mixed_flux_l1_vs_rtol1e-12": mixed[0]["flux_l1_vs_rtol1e-12"],
            "mixed_trace_ms": ms_mixed, "fp64": rows, "mixed": mixed, "df": df,
            "fp64_rtol_at_equal_accuracy": mixed[0]["fp64_rtol_at_equal_accuracy"],
            "fp64_at_least_as_accurate": mixed[0]["fp64_at_least_as_accurate"],
            "speedup_mixed_vs_fp64": mixed[0]["speedup_vs_fp64"],
            "launch": "one persistent launch per step, both paths (cost-ordered claims); "
                      "times of the trace call (persistent launch and its second pass)"}


def _endpoint_errors(ends, or_states, nper):
    """Per-ray relative end-point error max(|dx|/|x|, |dk|/|k|) of the mixed
    path against the FP64 oracle (the same uniforms), over the rays that
    escape in both: distribution over all of them, and over the rays whose
    FP64 GPU end point reproduces the oracle's to 1e-10 (the rays whose end
    point is insensitive to rounding, the well-conditioned set)."""
    import numpy as np
    st_m, s_m = ends["mixed"]
    st_d, s_d = ends["fp64"]
    err_all, err_wc = [], []
    for j, (st_o, s_o) in or_states.items():
        sl = slice(j * nper, (j + 1) * nper)
        ok = (s_o == 1) & (s_m[sl] == 1) & (s_d[sl] == 1)
        if not ok.any():
            continue

        def rel(a, b):
            dx = np.linalg.norm(a[:3] - b[:3], axis=0) / np.linalg.norm(b[:3], axis=0)
            dk = np.linalg.norm(a[3:6] - b[3:6], axis=0) / np.linalg.norm(b[3:6], axis=0)
            return np.maximum(dx, dk)
        em = rel(st_m[:, sl][:, ok], st_o[:, ok])
        ed = rel(st_d[:, sl][:, ok], st_o[:, ok])
        err_all.append(em)
        err_wc.append(em[ed <= 1e-10])
    out = {}
    for name, e in (("all_escaped", err_all), ("fp64_reproducible", err_wc)):
        e = np.concatenate(e) if e else np.zeros(0)
        out[name] = {"rays": int(e.size),
                     "within_1e-6": float((e <= 1e-6).mean()) if e.size else None,
                     "within_1e-5": float((e <= 1e-5).mean()) if e.size else None,
                     "p50_p90_p99_max": [float(np.percentile(e, q)) for q in (50, 90, 99)] +
                                        [float(e.max())] if e.size else None}
    return out


def _plain(o):
    """numpy scalars and arrays in the JSON line."""
    import numpy as np
    if isinstance(o, np.integer):
        return int(o)
    if isinstance(o, np.floating):
        return float(o)
    if isinstance(o, (np.bool_,)):
        return bool(o)
    if isinstance(o, np.ndarray):
        return o.tolist()
    raise TypeError(type(o).__name__)


def _twisted_leg(args, dev, stream):
    """The benchmark's 16 x 65536-ray step with the twisted magnetar density
    of Sec. 6 (Eq. neMag) in place of Goldreich-Julian: model M2's charge
    multiplicity lambda = 20 with twist psi = 0.2 (plasma_a = 4), open field
    lines excised.  Every sub-batch mass (1e-6 .. 5e-3 eV) then has a
    conversion surface.  One launch per step, FP64 and mixed precision."""
    import numpy as np
    import torch

    from paper_2309_08655_gb300 import inputs as I
    from paper_2309_08655_gb300 import rt
    cfg = I.CONFIG1
    nsub, nper = cfg["nsub"], cfg["n_per_sub"]
    N = nsub * nper
    kws = I.stars_config1(cfg["seed"], nsub)
    for kw in kws:
        kw.update(plasma=rt.PLASMA_TWISTED, plasma_a=4.0)
    stars = [rt.Star(rt.make_params(**kw)) for kw in kws]
    batch = rt.Batch(stars, [nper] * nsub)
    u = torch.from_numpy(np.ascontiguousarray(np.concatenate(
        [I.sample_uniforms(cfg["seed"] * 1000 + j, nper) for j in range(nsub)], axis=1))).to(dev)
    st = torch.empty((8, N), dtype=torch.float64, device=dev)
    w = torch.empty(N, dtype=torch.float64, device=dev)
    s = torch.empty(N, dtype=torch.uint8, device=dev)
    ctr = torch.zeros(8, dtype=torch.int64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": "forward_misaligned_16x65536_twisted_lambda20_psi0.2",
           "empty_sub_batches": int(sum(1 for x in stars if x.info()["empty"]))}
    for name, prec, rtol in (("fp64", rt.PREC_FP64, cfg["rtol"]),
                             ("mixed", rt.PREC_MIXED, cfg["rtol_mixed"])):
        opts = rt.make_opts(rtol=rtol, r_out_over_R=cfg["r_out_over_R"], precision=prec,
                            max_steps=cfg["max_steps"])
        rt.rt_sample_batch(batch, u, st, w, s, stream=stream)
        rt.rt_trace_batch(batch, st, s, None, None, None, opts, stream=stream)   # warm-up
        torch.cuda.synchronize()
        ctr.zero_()
        e0.record(stream)
        rt.rt_sample_batch(batch, u, st, w, s, stream=stream)
        rt.rt_trace_batch(batch, st, s, None, None, ctr, opts, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        c = ctr.cpu().numpy()
        out[name] = {"rtol": rtol, "ms_per_step": 1e3 * t, "ray_steps_per_s": c[0] / t,
                     "rays_per_s": c[2] / t, "accepted_steps": int(c[0]),
                     "rays_traced": int(c[2]), "promoted": int(c[4]),
                     "statuses": np.bincount(s.cpu().numpy(), minlength=8).tolist()}
    return out


def _rotating_leg(args, dev, stream):
    """The benchmark's 16 x 65536-ray step with the magnetosphere turning
    while the photons fly (the cos(Omega t) of Eq. GJDensity kept during the
    flight, Eq. Hamilton on x, k, t, k_t): one batch, FP64, one launch per
    step.  Reports the speed and the Doppler shift of the escaping photons in
    units of the natural line width v0^2 / 2."""
    import numpy as np
    import torch

    from paper_2309_08655_gb300 import inputs as I
    from paper_2309_08655_gb300 import rt
    cfg = I.CONFIG1
    nsub, nper = cfg["nsub"], cfg["n_per_sub"]
    N = nsub * nper
    kws = I.stars_config1(cfg["seed"], nsub)
    for kw in kws:
        kw.update(rotation=rt.ROTATION_RIGID)
    stars = [rt.Star(rt.make_params(**kw)) for kw in kws]
    batch = rt.Batch(stars, [nper] * nsub)
    u = torch.from_numpy(np.ascontiguousarray(np.concatenate(
        [I.sample_uniforms(cfg["seed"] * 1000 + j, nper) for j in range(nsub)], axis=1))).to(dev)
    st = torch.empty((8, N), dtype=torch.float64, device=dev)
    w = torch.empty(N, dtype=torch.float64, device=dev)
    s = torch.empty(N, dtype=torch.uint8, device=dev)
    ctr = torch.zeros(8, dtype=torch.int64, device=dev)
    opts = rt.make_opts(rtol=cfg["rtol"], r_out_over_R=cfg["r_out_over_R"],
                        max_steps=cfg["max_steps"], claim_order=CLAIM[args.claim_order])
    rt.rt_sample_batch(batch, u, st, w, s, stream=stream)
    delta0 = st[6].clone()
    rt.rt_trace_batch(batch, st, s, None, None, None, opts, stream=stream)   # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rt.rt_sample_batch(batch, u, st, w, s, stream=stream)
    rt.rt_trace_batch(batch, st, s, None, None, ctr, opts, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    c = ctr.cpu().numpy()
    status = s.cpu().numpy()
    esc = status == rt.RAY_ESCAPED
    width = 0.5 * (kws[0].get("v0_kms", 200.0) / 299792.458) ** 2
    shift = np.abs((st[6] - delta0).cpu().numpy()[esc]) / width
    out = {"workload": "forward_misaligned_16x65536_rotating", "precision": "fp64",
           "rtol": cfg["rtol"], "ms_per_step": 1e3 * t, "ray_steps_per_s": c[0] / t,
           "rays_per_s": c[2] / t, "accepted_steps": int(c[0]), "rejected_steps": int(c[1]),
           "rays_traced": int(c[2]),
           "statuses": np.bincount(status, minlength=8).tolist(),
           "doppler_shift_in_line_widths_p50_p90_max": [float(np.percentile(shift, 50)),
                                                        float(np.percentile(shift, 90)),
                                                        float(shift.max())],
           "launch": "one persistent launch per step (one lane per ray, no tail mode)"}
    # continuous batching: the K steps' 16 sub-batches in one batch, one launch
    K = max(1, args.steps)
    del st, w, s
    batchK = rt.Batch(stars * K, [nper] * (nsub * K))
    uK = u.repeat(1, K)
    stK = torch.empty((8, N * K), dtype=torch.float64, device=dev)
    wK = torch.empty(N * K, dtype=torch.float64, device=dev)
    sK = torch.empty(N * K, dtype=torch.uint8, device=dev)
    ctr.zero_()
    torch.cuda.synchronize()
    e0.record(stream)
    rt.rt_sample_batch(batchK, uK, stK, wK, sK, stream=stream)
    rt.rt_trace_batch(batchK, stK, sK, None, None, ctr, opts, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    tK = e0.elapsed_time(e1) / 1e3
    cK = ctr.cpu().numpy()
    out["pipelined"] = {"steps_per_launch": K, "ms_per_step": 1e3 * tK / K,
                        "ray_steps_per_s": cK[0] / tK, "rays_per_s": cK[2] / tK,
                        "accepted_steps_equal_to_K_single_steps": bool(cK[0] == K * c[0])}
    return out


def _uneven_leg(args, dev):
    """256 star/axion instances with ray counts log-uniform in [1e3, 1e6]:
    the 128 forward instances (rays) and the 128 backward images (pixels) in
    ONE persistent launch with one work queue (mixed precision, rtol 1e-8,
    plus the FP64 pass for promoted rays and pixels), sample -> trace -> bin
    captured in one CUDA graph.  Latency of an instance = GPU global-timer
    stamp of its last ray or pixel minus the start of the launch.  The
    autotuner's shape is recorded for the rays-only launch of the same
    forward instances (also timed, for comparison)."""
    import numpy as np
    import torch

    from paper_2309_08655_gb300 import inputs as I
    from paper_2309_08655_gb300 import rt
    insts = I.instances_config3()
    fwd = [x for x in insts if x["mode"] == "forward"]
    bwd = [x for x in insts if x["mode"] == "backward"]
    stars = [rt.Star(rt.make_params(**x["star"])) for x in fwd]
    counts = [x["n"] for x in fwd]
    batch = rt.Batch(stars, counts)
    N = batch.N
    u = torch.from_numpy(np.ascontiguousarray(np.concatenate(
        [I.sample_uniforms(x["seed"], x["n"]) for x in fwd], axis=1))).to(dev)
    st = torch.empty((8, N), dtype=torch.float64, device=dev)
    w = torch.empty(N, dtype=torch.float64, device=dev)
    s = torch.empty(N, dtype=torch.uint8, device=dev)
    nth, nph, nnu = NBINS
    hist = torch.empty((len(fwd), nth, nph, nnu), dtype=torch.float64, device=dev)
    oor = torch.empty(len(fwd), dtype=torch.float64, device=dev)
    ctr = torch.zeros(8, dtype=torch.int64, device=dev)
    nts = len(fwd) + len(bwd)
    ts = torch.zeros(1 + nts, dtype=torch.int64, device=dev)
    opts = rt.make_opts(rtol=1e-8, precision=rt.PREC_MIXED, timestamps=ts)
    rt.rt_sample_batch(batch, u, st, w, s)
    tune = rt.rt_batch_autotune(batch, st, s, opts, rays_per_star=256)
    # rays only (the autotuned launch), for comparison
    graph_f = rt.Graph(batch, u, st, w, s, ctr, opts, nth, nph, nnu, 0.0, 9.0, hist, oor)
    graph_f.launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    graph_f.launch()
    e1.record()
    torch.cuda.synchronize()
    t_rays_only = e0.elapsed_time(e1) / 1e3
    # backward images: one star each, bmax from the largest conversion radius
    bstars, descs = [], []
    for x in bwd:
        sb = rt.Star(rt.make_params(**x["star"]))
        r_max = max((2.0 * sb.info()["wp2_coef"]) ** (1.0 / 3.0), 1.5)
        bstars.append(sb)
        descs.append((x["side"], x["side"], x["incl"], 1e4, 1.3 * r_max, 0.0))
    P = sum(d[0] * d[1] for d in descs)
    image = torch.empty(P, dtype=torch.float64, device=dev)
    ist = torch.empty(P, dtype=torch.uint8, device=dev)
    rt.rt_batch_set_images(batch, bstars, descs, image, ist)
    # tune the launch that is timed: rays and pixels in one queue (the first
    # 256 rays of every forward instance and a 16 x 16 copy of every image)
    rt.rt_sample_batch(batch, u, st, w, s)
    tune_img = rt.rt_batch_autotune(batch, st, s, opts, rays_per_star=256)
    graph = rt.Graph(batch, u, st, w, s, ctr, opts, nth, nph, nnu, 0.0, 9.0, hist, oor)
    graph.launch()                                     # warm-up
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    e0.record()
    graph.launch()
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    t_wall = time.perf_counter() - t_wall
    tt = ts.cpu().numpy().astype(np.int64)
    c = ctr.cpu().numpy()
    t0 = int(tt[0])
    lat = np.array([(int(tt[1 + k]) - t0) / 1e6 for k in range(nts) if tt[1 + k] > 0])
    steps = float(c[0])
    return {"workload": "uneven_256_instances_128fwd_128bwd", "instances": len(insts),
            "forward_rays": int(N), "backward_pixels": int(P),
            "empty_forward_instances": int(sum(1 for x in stars if x.info()["empty"])),
            "precision": "mixed (rtol 1e-8), FP64 pass for promoted rays and pixels",
            "launch": "rays and pixels of all 256 instances in one persistent launch, "
                      "one queue; sample -> trace -> bin replayed from one CUDA graph",
            "autotuned": {"block": tune_img["block"], "blocks_per_sm": tune_img["blocks_per_sm"],
                          "refill_min": tune_img["refill_min"],
                          "rays_per_claim": tune_img["rays_per_claim"],
                          "candidates": len(tune_img["candidates_ms"]),
                          "candidates_ms": tune_img["candidates_ms"],
                          "tuned_on": "first 256 rays of each forward instance and a 16 x 16 "
                                      "copy of each image, rays and pixels in one launch"},
            "autotuned_rays_only": {"block": tune["block"],
                                    "blocks_per_sm": tune["blocks_per_sm"],
                                    "refill_min": tune["refill_min"],
                                    "rays_per_claim": tune["rays_per_claim"],
                                    "candidates": len(tune["candidates_ms"]),
                                    "seconds_rays_only": t_rays_only},
            "seconds": t, "wall_seconds": t_wall, "ray_steps_per_s": steps / t,
            "accepted_steps": steps, "items_finished": int(c[2]),
            "promoted_to_fp64": int(c[4]),
            "latency_ms": {"p50": float(np.percentile(lat, 50)),
                           "p90": float(np.percentile(lat, 90)), "max": float(lat.max()),
                           "instances_timed": int(lat.size)}}


def _adjoint_leg(args, dev):
    """Differentiable trace: 2^18 forward rays on the misaligned magnetar-like
    star at m_a = 1e-5 eV; the line flux toward inclination 1.1 rad smoothed
    with a von Mises-Fisher kernel one theta-bin wide (kappa = (64/pi)^2) and
    its gradient with respect to (m_a, B0, theta_m, M, R, inclination) by the
    adjoint (rt_flux_gradient).  Times one forward (sample + trace + functional)
    and one gradient after a warm-up of each on a smaller sample."""
    import numpy as np
    import torch

    from paper_2309_08655_gb300 import flux
    from paper_2309_08655_gb300 import inputs as I
    from paper_2309_08655_gb300 import rt
    kw = I.stars_config1()[0]
    kw.update(m_a_eV=1e-5)
    n = 1 << 18
    kappa = (64.0 / math.pi) ** 2
    p = torch.tensor([kw["m_a_eV"], kw["B0_G"], kw["theta_m"], kw["M_sun"], kw["R_km"], 1.1],
                     dtype=torch.float64)
    u = torch.from_numpy(I.sample_uniforms(4000, n)).to(dev)
    grad = torch.empty(6, dtype=torch.float64, device=dev)
    F2 = torch.empty(1, dtype=torch.float64, device=dev)
    uw = u[:, :4096].contiguous()
    Fw, nw, sw, iw, ow = flux.flux_forward(p, kw, uw, kappa)
    rt.rt_flux_gradient(sw, 4096, uw, nw, iw, kappa, grad, F2, opts=ow)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    F, nacc, star, incl, opts = flux.flux_forward(p, kw, u, kappa)
    torch.cuda.synchronize()
    t_f = time.perf_counter() - t0
    def run(prec, tape_max_bytes):
        o = rt.make_opts(rtol=opts.rtol, precision=prec)
        rt.rt_flux_gradient(sw, 4096, uw, nw, iw, kappa, grad, F2, opts=o,
                            tape_max_bytes=tape_max_bytes)    # warm-up
        ctr = torch.zeros(8, dtype=torch.int64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nb = rt.rt_flux_gradient(star, n, u, nacc, incl, kappa, grad, F2, counters=ctr, opts=o,
                                 tape_max_bytes=tape_max_bytes)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, grad.cpu().numpy().copy(), nb, ctr.cpu().numpy()

    # the backward sweep in FP64, double-float and mixed over the full step tape
    # (one FP64 replay), and in FP64 over the checkpointed recompute
    t_g, g, nbytes, c = run(rt.PREC_FP64, -1)
    t_df, gdf, _, _ = run(rt.PREC_DF, -1)
    t_mx, gmx, _, _ = run(rt.PREC_MIXED, -1)
    t_ck, gck, nb_ck, _ = run(rt.PREC_FP64, 0)
    errmx = np.abs(gmx - g) / np.abs(g)
    errdf = np.abs(gdf - g) / np.abs(g)
    errck = np.abs(gck - g) / np.abs(g)
    na = nacc.cpu().numpy()
    # the full-size gradient against central finite differences of the GPU
    # forward pipeline (relative step 1e-6, 1e-6 rad for the angles, rtol 1e-12
    # so that the controller's discrete decisions do not move F measurably)
    t0 = time.perf_counter()
    pd = p.detach()
    hs = 1e-6 * np.abs(pd.numpy())
    hs[2] = hs[5] = 1e-6
    g_fd = np.zeros(6)
    for k in range(6):
        e = torch.zeros(6, dtype=torch.float64)
        e[k] = hs[k]
        Fp = float(flux.flux_forward(pd + e, kw, u, kappa, rtol=1e-12)[0].cpu()[0])
        Fm = float(flux.flux_forward(pd - e, kw, u, kappa, rtol=1e-12)[0].cpu()[0])
        g_fd[k] = (Fp - Fm) / (2.0 * hs[k])
    t_fd = time.perf_counter() - t0
    err_fd = np.abs(g - g_fd) / np.abs(g_fd)
    def named(v):
        return dict(zip(flux.PARAM_NAMES, [float(x) for x in v]))

    return {"workload": "adjoint_2^18_rays_ma1e-5_incl1.1_vmf_one_theta_bin",
            "precision": "fp64 replay, fp64 backward sweep", "rays": n,
            "F_W_per_sr": float(F.cpu()[0]), "grad": named(g),
            "t_forward_s": t_f, "t_gradient_s": t_g, "adjoint_forward_ratio": t_g / t_f,
            "store": "full step tape", "store_MiB": nbytes / 2 ** 20,
            "forward_steps": {"mean": float(na.mean()), "max": int(na.max())},
            "replayed_attempts": int(c[0]), "rays_left_out": int(c[4]),
            "df_sweep": {"t_gradient_s": t_df, "adjoint_forward_ratio": t_df / t_f,
                         "vs_fp64_sweep_error": named(errdf)},
            "mixed_sweep": {"t_gradient_s": t_mx, "adjoint_forward_ratio": t_mx / t_f,
                            "vs_fp64_sweep_error": named(errmx),
                            "note": "adjoint of the state in FP64, the tangents of r_s, the "
                                    "omega_p^2 coefficient and the magnetic axis in FP32"},
            "checkpoints_fp64_sweep": {"t_gradient_s": t_ck, "adjoint_forward_ratio": t_ck / t_f,
                                       "store_MiB": nb_ck / 2 ** 20,
                                       "vs_tape_relative_difference": named(errck),
                                       "note": "a checkpoint every 32 accepted steps and a "
                                               "replay per segment (the store used when the "
                                               "tape does not fit)"},
            "vs_central_differences": {"relative_error": named(err_fd), "seconds": t_fd,
                                       "note": "12 forward runs at rtol 1e-12, all 2^18 rays; "
                                               "against the FP64 sweep"},
            "note": "forward trace and replay FP64; gradient timings include sampling with "
                    "tangents, the replay onto the tape, the sweep's dual-number Jacobian "
                    "products and the sums"}


def _backward_leg(args, dev, stream, fl, rank):
    """Backward image plane: 1024 x 1024 pixels at inclination 60 deg, plane at
    1e4 R, impact parameters up to 50 R, on the aligned 200 km-surface star
    (FP64, rtol 1e-10; and mixed precision, rtol 1e-8, compared with it).  No
    conversion-length cut: on this 200 km surface the paper's 1 km cut would
    remove all but 56 of the 11212 crossings.  Near-tangent crossings make a
    few pixels very bright and sensitive to rounding, so the mixed image is also
    compared on the pixels whose crossing count agrees.  A seeded sample of the
    FP64 pixels is recomputed by the oracle on rank 0."""
    import numpy as np
    import torch

    from paper_2309_08655_gb300 import inputs as I
    from paper_2309_08655_gb300 import rt
    kw = I.star_config0()
    star = rt.Star(rt.make_params(**kw))
    nx = ny = 1024
    incl, D, bmax = math.radians(60.0), 1e4, 50.0
    opts = rt.make_opts(rtol=1e-10, precision=rt.PREC_FP64)
    img = torch.empty((ny, nx), dtype=torch.float64, device=dev)
    st = torch.empty((ny, nx), dtype=torch.uint8, device=dev)
    nc = torch.empty((ny, nx), dtype=torch.int32, device=dev)
    ctr = torch.zeros(8, dtype=torch.int64, device=dev)
    rt.rt_trace_backward(star, 128, 128, incl, D, bmax, img, st, nc, ctr,
                         Lc_cut_km=LC_CUT_KM, opts=opts,
                         stream=stream)                                    # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    ctr.zero_()
    e0.record(stream)
    for _ in range(reps):
        rt.rt_trace_backward(star, nx, ny, incl, D, bmax, img, st, nc, ctr,
                             Lc_cut_km=LC_CUT_KM, opts=opts, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    c = ctr.cpu().numpy() / reps
    out = {"workload": "backward_image_1024x1024_incl60_b50R", "precision": "fp64",
           "ms_per_image": 1e3 * t, "pixels_per_s": nx * ny / t,
           "ray_steps_per_s": c[0] / t, "accepted_steps": c[0], "rejected_steps": c[1],
           "crossings": c[6], "extremum_searches": c[5], "dP_dOmega_W_per_sr": float(img.sum()),
           "roofline": {"kernel": "backward_kernel", "bound": "alu",
                        "achieved": (c[0] + c[1]) * fl[1] / t / 1e12, "peak": PEAK["fp64"] / 1e12,
                        "unit": "TFLOP/s", "frac": (c[0] + c[1]) * fl[1] / t / PEAK["fp64"],
                        "traffic": None,
                        "note": "integrator flops only; the crossing search is not counted"}}
    # the same image in mixed precision (FP32 stages, rtol 1e-8; FP64 crossing
    # search, bisection and estimator; floor pixels re-traced in FP64)
    om = rt.make_opts(rtol=1e-8, precision=rt.PREC_MIXED)
    img_m = torch.empty_like(img)
    st_m = torch.empty_like(st)
    nc_m = torch.empty_like(nc)
    rt.rt_trace_backward(star, 128, 128, incl, D, bmax, img_m, st_m, nc_m, None,
                         Lc_cut_km=LC_CUT_KM, opts=om,
                         stream=stream)                                    # warm-up
    torch.cuda.synchronize()
    ctr.zero_()
    e0.record(stream)
    for _ in range(reps):
        rt.rt_trace_backward(star, nx, ny, incl, D, bmax, img_m, st_m, nc_m, ctr,
                             Lc_cut_km=LC_CUT_KM, opts=om, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    tm = e0.elapsed_time(e1) / 1e3 / reps
    cm = ctr.cpu().numpy() / reps
    same = (nc_m == nc) & (st_m == st)
    litm = same & (nc > 0)
    relm = ((img_m - img).abs() / img.abs().clamp_min(1e-300))[litm]
    out["mixed"] = {"rtol": 1e-8, "ms_per_image": 1e3 * tm, "pixels_per_s": nx * ny / tm,
                    "ray_steps_per_s": cm[0] / tm, "accepted_steps": cm[0],
                    "rejected_steps": cm[1], "pixels_to_fp64": cm[4], "crossings": cm[6],
                    "extremum_searches": cm[5],
                    "dP_dOmega_W_per_sr": float(img_m.sum()),
                    "total_rel_diff_vs_fp64": float(abs(img_m.sum() - img.sum()) / img.sum()),
                    "total_rel_diff_same_crossings":
                        float(abs(img_m[same].sum() - img[same].sum()) / img[same].sum()),
                    "pixels_differing_in_crossings": int((~same).sum()),
                    "pixels_same_crossings": float(same.double().mean()),
                    "pixel_rel_diff_p50_p99": [float(torch.quantile(relm, q)) for q in (0.5, 0.99)]
                    if relm.numel() else None,
                    "speedup_vs_fp64": t / tm}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        img_h, nc_h = img.cpu().numpy(), nc.cpu().numpy()
        rng = np.random.default_rng(60)
        lit = np.flatnonzero(nc_h.ravel() > 0)
        pick = np.concatenate([rng.choice(lit, size=min(48, lit.size), replace=False),
                               rng.choice(nx * ny, size=16, replace=False)])
        j, i = np.divmod(pick, nx)
        db = 2.0 * bmax / nx
        b = np.stack([-bmax + (i + 0.5) * db, -bmax + (j + 0.5) * db], 1)
        t0 = time.perf_counter()
        v, _, nco = oracle.backward_points(oracle.star_vector(**kw), oracle.trace_opts(rtol=1e-10),
                                           b, incl, D, Lc_cut_km=LC_CUT_KM)
        t_or = time.perf_counter() - t0
        ref = v * db * db
        got = img_h.ravel()[pick]
        rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
        rel[(ref == 0) & (got == 0)] = 0.0
        out["oracle_sample"] = {"pixels": int(pick.size), "lit": int(min(48, lit.size)),
                                "median_rel_diff": float(np.median(rel)),
                                "max_rel_diff": float(rel.max()),
                                "within_1e-8": int((rel <= 1e-8).sum()),
                                "ncross_equal": int((nco == nc_h.ravel()[pick]).sum()),
                                "oracle_pixels_per_s": pick.size / t_or}
    return out


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
