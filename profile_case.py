"""Small, self-contained forward case for kernel profiling (ncu) and quick timing.

    python profile_case.py --precision fp64 --n 1024
    python profile_case.py --mode backward --n 65536
    python profile_case.py --mode adjoint --n 4096
    python profile_case.py --config config1 --rotating --n 65536
    python profile_case.py --config config1 --claim-order cost --n 65536

Forward: samples n rays of the aligned 200 km-surface star (seed 0), traces
them once in the requested precision (one persistent trace launch, after one
untimed warm-up launch on a copy) and bins them; --rotating keeps the
magnetosphere turning during the flight (FP64 only).  config1 is the
misaligned magnetar-like star of the largest sub-batch mass.  Backward: an image of about
n pixels (square) of the same star at inclination 60 deg, plane at 1e4 R,
impact parameters up to 50 R, in the requested precision (one warm-up launch
on an image of at most 32 x 32 pixels first).
Adjoint: n rays of the misaligned magnetar-like star at m_a = 1e-5 eV, the
smoothed line flux toward 1.1 rad (kappa 4) and its gradient (one warm-up
gradient on 256 rays first), the backward sweep in the requested precision,
on the full step tape or (--store checkpoints) the checkpointed recompute.
Prints the trace time and step counts.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from paper_2309_08655_gb300 import inputs as I
from paper_2309_08655_gb300 import rt
from paper_2309_08655_gb300.build import build


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", choices=["fp64", "mixed", "df"], default="fp64")
    ap.add_argument("--store", choices=["tape", "checkpoints"], default="tape",
                    help="adjoint mode: the full step tape or the checkpointed recompute")
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--rtol", type=float, default=None)
    ap.add_argument("--config", choices=["config0", "config1"], default="config0")
    ap.add_argument("--mode", choices=["forward", "backward", "adjoint"], default="forward")
    ap.add_argument("--rotating", action="store_true")
    ap.add_argument("--claim-order", choices=["index", "cost"], default="index")
    a = ap.parse_args()
    build()
    dev = torch.device("cuda:0")
    if a.mode == "backward":
        return backward(a, dev)
    if a.mode == "adjoint":
        return adjoint(a, dev)
    if a.config == "config0":
        kw = I.star_config0()
    else:
        kw = I.stars_config1()[15]
    if a.rotating:
        kw.update(rotation=rt.ROTATION_RIGID)
    u = torch.from_numpy(I.sample_uniforms(0, a.n)).to(dev)
    star = rt.Star(rt.make_params(**kw))
    st = torch.empty((8, a.n), dtype=torch.float64, device=dev)
    w = torch.empty(a.n, dtype=torch.float64, device=dev)
    s = torch.empty(a.n, dtype=torch.uint8, device=dev)
    rt.rt_sample_conversion_surface(star, a.n, u, st, w, s)
    prec = {"fp64": rt.PREC_FP64, "mixed": rt.PREC_MIXED, "df": rt.PREC_DF}[a.precision]
    rtol = a.rtol if a.rtol is not None else (1e-8 if prec == rt.PREC_MIXED else 1e-10)
    opts = rt.make_opts(rtol=rtol, precision=prec,
                        claim_order=rt.CLAIM_COST if a.claim_order == "cost" else rt.CLAIM_INDEX)
    st0, s0 = st.clone(), s.clone()
    rt.rt_trace_forward(star, a.n, st0, s0, opts=opts)          # warm-up
    ctr = torch.zeros(8, dtype=torch.int64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    rt.rt_trace_forward(star, a.n, st, s, counters=ctr, opts=opts)
    e1.record()
    hist = torch.empty((64, 32, 128), dtype=torch.float64, device=dev)
    oor = torch.empty(1, dtype=torch.float64, device=dev)
    rt.rt_bin_spectrum(star, a.n, st, w, s, 64, 32, 128, 0.0, 9.0, hist, None, None, oor)
    torch.cuda.synchronize()
    c = ctr.cpu().numpy()
    print(json.dumps({"precision": a.precision, "n": a.n, "rtol": rtol,
                      "trace_ms": e0.elapsed_time(e1), "accepted": int(c[0]),
                      "rejected": int(c[1]), "rays": int(c[2]), "promoted": int(c[4]),
                      "statuses": np.bincount(s.cpu().numpy(), minlength=8).tolist()}))


def backward(a, dev):
    import math
    kw = I.star_config0()
    star = rt.Star(rt.make_params(**kw))
    side = max(1, int(round(math.sqrt(a.n))))
    prec = rt.PREC_FP64 if a.precision == "fp64" else rt.PREC_MIXED
    rtol = a.rtol if a.rtol is not None else (1e-10 if prec == rt.PREC_FP64 else 1e-8)
    opts = rt.make_opts(rtol=rtol, precision=prec)
    incl, D, bmax = math.radians(60.0), 1e4, 50.0
    img = torch.empty((side, side), dtype=torch.float64, device=dev)
    st = torch.empty((side, side), dtype=torch.uint8, device=dev)
    nc = torch.empty((side, side), dtype=torch.int32, device=dev)
    ctr = torch.zeros(8, dtype=torch.int64, device=dev)
    w = min(side, 32)
    rt.rt_trace_backward(star, w, w, incl, D, bmax, img, st, nc, ctr, opts=opts)     # warm-up
    ctr.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    rt.rt_trace_backward(star, side, side, incl, D, bmax, img, st, nc, ctr, opts=opts)
    e1.record()
    torch.cuda.synchronize()
    c = ctr.cpu().numpy()
    print(json.dumps({"mode": "backward", "precision": a.precision, "pixels": side * side,
                      "rtol": rtol, "promoted": int(c[4]),
                      "trace_ms": e0.elapsed_time(e1), "accepted": int(c[0]),
                      "rejected": int(c[1]), "pixels_done": int(c[2]), "crossings": int(c[6]),
                      "dP_dOmega": float(img.sum()),
                      "statuses": np.bincount(st.cpu().numpy().ravel(), minlength=8).tolist()}))


def adjoint(a, dev):
    from paper_2309_08655_gb300 import flux
    kw = I.stars_config1()[0]
    kw.update(m_a_eV=1e-5)
    p = torch.tensor([kw["m_a_eV"], kw["B0_G"], kw["theta_m"], kw["M_sun"], kw["R_km"], 1.1],
                     dtype=torch.float64)
    grad = torch.empty(6, dtype=torch.float64, device=dev)
    F2 = torch.empty(1, dtype=torch.float64, device=dev)
    uw = torch.from_numpy(I.sample_uniforms(4, 256)).to(dev)
    Fw, nw, sw, iw, ow = flux.flux_forward(p, kw, uw, 4.0)
    # the backward sweep's arithmetic: --precision fp64, df or mixed (FP32)
    prec = {"fp64": rt.PREC_FP64, "mixed": rt.PREC_MIXED, "df": rt.PREC_DF}[a.precision]
    og = rt.make_opts(rtol=ow.rtol, precision=prec)
    tmb = -1 if a.store == "tape" else 0
    rt.rt_flux_gradient(sw, 256, uw, nw, iw, 4.0, grad, F2, opts=og,
                        tape_max_bytes=tmb)      # warm-up
    u = torch.from_numpy(I.sample_uniforms(4, a.n)).to(dev)
    F, nacc, star, incl, opts = flux.flux_forward(p, kw, u, 4.0)
    ctr = torch.zeros(8, dtype=torch.int64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    nb = rt.rt_flux_gradient(star, a.n, u, nacc, incl, 4.0, grad, F2, counters=ctr, opts=og,
                             tape_max_bytes=tmb)
    e1.record()
    torch.cuda.synchronize()
    na = nacc.cpu().numpy()
    print(json.dumps({"mode": "adjoint", "precision": a.precision, "store": a.store,
                      "rays": a.n, "gradient_ms": e0.elapsed_time(e1),
                      "replayed_attempts": int(ctr.cpu()[0]), "store_bytes": nb,
                      "nacc_max": int(na.max()), "nacc_mean": float(na.mean()),
                      "F": float(F.cpu()[0]), "grad": grad.cpu().tolist()}))


if __name__ == "__main__":
    main()
