"""Thin ctypes binding of the C ABI in ``include/rt.h`` (same function names).

Only argument marshalling happens here: torch tensors provide device memory
(``data_ptr()``) and the stream (``torch.cuda.current_stream()``); every step
of the computation runs in the CUDA library.  If the library is missing or a
CUDA device is absent, calls raise ``RtError`` -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

from .build import library_path

STATE_ROWS = 8
UNIFORM_ROWS = 6

RT_OK, RT_EINVAL, RT_ENOMEM, RT_ECUDA, RT_EEMPTY_SURFACE, RT_EPARTIAL, RT_EUNSUPPORTED = range(7)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EEMPTY_SURFACE", "EPARTIAL", "EUNSUPPORTED"]
(RAY_READY, RAY_ESCAPED, RAY_CAPTURED, RAY_NO_ROOT, RAY_MAXSTEPS, RAY_NAN, RAY_STIFF,
 RAY_LAMBDA_END) = range(8)
RAY_NSTATUS = 8
PREC_FP64, PREC_MIXED, PREC_DF = 0, 1, 2
CLAIM_INDEX, CLAIM_COST = 0, 1
(PLASMA_GJ, PLASMA_VACUUM, PLASMA_HOMOG, PLASMA_LINEAR_Z, PLASMA_RADIAL,
 PLASMA_TWISTED) = range(6)
WEIGHT_PAG, WEIGHT_UNIT_P, WEIGHT_RENORM = 0, 1, 2
ROTATION_SNAPSHOT, ROTATION_RIGID = 0, 1
DISP_ANISO, DISP_ISO = 0, 1
METRIC_FULL, METRIC_FLAT = 0, 1


class RtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class rt_star_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in [
        "M_sun", "R_km", "B0_G", "P_s", "theta_m_rad", "psi_rad", "m_a_eV", "g_agg_GeVinv",
        "rho_dm_GeV_cm3", "v0_kms"]] + [(k, ctypes.c_int32) for k in [
            "dispersion", "resonance", "fa_model", "weight_mode", "prop_metric", "phase_mode",
            "plasma", "rotation"]] + [("plasma_a", ctypes.c_double)]


class rt_image_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("incl_rad", ctypes.c_double),
                ("dist_over_R", ctypes.c_double), ("bmax_over_R", ctypes.c_double),
                ("Lc_cut_km", ctypes.c_double)]


class rt_trace_opts(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in [
        "rtol", "atol", "r_out_over_R", "lambda_max", "r_capture_over_R"]] + [
        (k, ctypes.c_int32) for k in ["precision", "max_steps", "block", "blocks_per_sm", "tail",
                                      "claim_order"]] + [
        ("timestamps", ctypes.c_void_p), ("refill_min", ctypes.c_int32),
        ("rays_per_claim", ctypes.c_int32)]


_lib = None
_vp = ctypes.c_void_p


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RtError(RT_ECUDA, f"CUDA library not built ({path}); run "
                                    "paper_2309_08655_gb300.build.build()")
        L = ctypes.CDLL(path)
        L.rt_init_star.restype = ctypes.c_int
        L.rt_init_star.argtypes = [ctypes.POINTER(rt_star_params), ctypes.POINTER(_vp)]
        L.rt_destroy_star.restype = None
        L.rt_destroy_star.argtypes = [_vp]
        L.rt_star_info.restype = ctypes.c_int
        L.rt_star_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
        L.rt_sample_conversion_surface.restype = ctypes.c_int
        L.rt_sample_conversion_surface.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp]
        L.rt_sample_conversion_surface_part.restype = ctypes.c_int
        L.rt_sample_conversion_surface_part.argtypes = [_vp, ctypes.c_int64, ctypes.c_int64, _vp,
                                                        _vp, _vp, _vp, _vp]
        L.rt_bin_part_max.restype = ctypes.c_int
        L.rt_bin_part_max.argtypes = [ctypes.c_int64, _vp, _vp, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, _vp, _vp]
        L.rt_bin_part_accumulate.restype = ctypes.c_int
        L.rt_bin_part_accumulate.argtypes = [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                             _vp, _vp, _vp,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_double, ctypes.c_double, _vp, _vp]
        L.rt_bin_part_finalize.restype = ctypes.c_int
        L.rt_bin_part_finalize.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, _vp]
        L.rt_trace_forward.restype = ctypes.c_int
        L.rt_trace_forward.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp,
                                       ctypes.POINTER(rt_trace_opts), _vp]
        L.rt_bin_spectrum.restype = ctypes.c_int
        L.rt_bin_spectrum.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                      ctypes.c_double, _vp, _vp, _vp, _vp, _vp]
        L.rt_trace_backward.restype = ctypes.c_int
        L.rt_trace_backward.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double, _vp,
                                        _vp, _vp, _vp, ctypes.POINTER(rt_trace_opts), _vp]
        L.rt_bin_spectrum_noalloc.restype = ctypes.c_int
        L.rt_bin_spectrum_noalloc.argtypes = [ctypes.POINTER(rt_star_params), ctypes.c_int64,
                                              _vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                              _vp, _vp, _vp, _vp, _vp]
        L.rt_flops_per_step.restype = ctypes.c_int
        L.rt_flops_per_step.argtypes = [ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_double)]
        L.rt_flops_per_step_df.restype = ctypes.c_int
        L.rt_flops_per_step_df.argtypes = [ctypes.c_int32, ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_double)]
        L.rt_flux_value.restype = ctypes.c_int
        L.rt_flux_value.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, ctypes.c_double,
                                    ctypes.c_double, _vp, _vp, _vp]
        L.rt_flux_gradient.restype = ctypes.c_int
        L.rt_flux_gradient.argtypes = [_vp, ctypes.c_int64, _vp, _vp, ctypes.c_double,
                                       ctypes.c_double, ctypes.POINTER(rt_trace_opts), _vp, _vp,
                                       _vp, _vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                       _vp]
        L.rt_timestamps_reset.restype = ctypes.c_int
        L.rt_timestamps_reset.argtypes = [_vp, ctypes.c_int32, _vp]
        L.rt_batch_graph_create.restype = ctypes.c_int
        L.rt_batch_graph_create.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp,
                                            ctypes.POINTER(rt_trace_opts), ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                            ctypes.c_double, _vp, _vp, ctypes.POINTER(_vp)]
        L.rt_graph_launch.restype = ctypes.c_int
        L.rt_graph_launch.argtypes = [_vp, _vp]
        L.rt_graph_destroy.restype = None
        L.rt_graph_destroy.argtypes = [_vp]
        L.rt_batch_autotune.restype = ctypes.c_int
        L.rt_batch_autotune.argtypes = [_vp, _vp, _vp, ctypes.POINTER(rt_trace_opts),
                                        ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_int32, _vp]
        L.rt_count_status.restype = ctypes.c_int
        L.rt_count_status.argtypes = [ctypes.c_int64, _vp, ctypes.POINTER(ctypes.c_int64), _vp]
        L.rt_init_batch.restype = ctypes.c_int
        L.rt_init_batch.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_vp)]
        L.rt_destroy_batch.restype = None
        L.rt_destroy_batch.argtypes = [_vp]
        L.rt_sample_batch.restype = ctypes.c_int
        L.rt_sample_batch.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
        L.rt_batch_set_norm.restype = ctypes.c_int
        L.rt_batch_set_norm.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
        L.rt_trace_batch.restype = ctypes.c_int
        L.rt_trace_batch.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp,
                                     ctypes.POINTER(rt_trace_opts), _vp]
        L.rt_bin_batch.restype = ctypes.c_int
        L.rt_bin_batch.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_double, ctypes.c_double, _vp, _vp,
                                   _vp]
        L.rt_batch_set_images.restype = ctypes.c_int
        L.rt_batch_set_images.argtypes = [_vp, ctypes.c_int32, ctypes.POINTER(_vp),
                                          ctypes.POINTER(rt_image_desc), _vp, _vp, _vp]
        L.rt_hamilton_rhs.restype = ctypes.c_int
        L.rt_hamilton_rhs.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp]
        L.rt_measure_alu_peak.restype = ctypes.c_int
        L.rt_measure_alu_peak.argtypes = [ctypes.c_int64, ctypes.c_int64,
                                          ctypes.POINTER(ctypes.c_double), _vp]
        L.rt_last_error.restype = ctypes.c_char_p
        L.rt_last_error.argtypes = []
        L.rt_version.restype = ctypes.c_int32
        L.rt_version.argtypes = []
        _lib = L
    return _lib


def _check(status: int, allow=(RT_OK,)) -> int:
    if status not in allow:
        raise RtError(status, lib().rt_last_error().decode())
    return status


def _ptr(t):
    """Device pointer of a tensor (or None / int)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_params(**kw) -> rt_star_params:
    """rt_star_params from keyword arguments; unspecified fields are 0 except
    the paper's fiducial values for the coupling, density and dispersion."""
    p = rt_star_params()
    p.g_agg_GeVinv = 1e-12
    p.rho_dm_GeV_cm3 = 0.45
    p.v0_kms = 200.0
    alias = {"theta_m": "theta_m_rad", "psi": "psi_rad", "g_GeVinv": "g_agg_GeVinv",
             "rho_GeV_cm3": "rho_dm_GeV_cm3"}
    for k, v in kw.items():
        setattr(p, alias.get(k, k), v)
    return p


def make_opts(rtol=1e-10, atol=None, r_out_over_R=1000.0, lambda_max=0.0, r_capture_over_R=1.0,
              precision=PREC_FP64, max_steps=100000, block=0, blocks_per_sm=0,
              timestamps=None, tail=0, claim_order=0, refill_min=0,
              rays_per_claim=0) -> rt_trace_opts:
    o = rt_trace_opts()
    o.rtol = rtol
    o.atol = rtol if atol is None else atol
    o.r_out_over_R = r_out_over_R
    o.lambda_max = lambda_max
    o.r_capture_over_R = r_capture_over_R
    o.precision = precision
    o.max_steps = max_steps
    o.block = block
    o.blocks_per_sm = blocks_per_sm
    o.tail = tail
    o.claim_order = claim_order
    o.timestamps = _ptr(timestamps)
    o.refill_min = refill_min
    o.rays_per_claim = rays_per_claim
    return o


class Star:
    """Owning wrapper of an ``rt_star`` handle."""

    def __init__(self, params: rt_star_params | None = None, **kw):
        if params is None:
            params = make_params(**kw)
        h = _vp()
        _check(lib().rt_init_star(ctypes.byref(params), ctypes.byref(h)))
        self.handle = h
        self.params = params

    def info(self) -> dict:
        out = (ctypes.c_double * 8)()
        _check(lib().rt_star_info(self.handle, out))
        keys = ["rs_over_R", "wp2_coef", "B0_eV2", "R_inv_eV", "n_inf_eV3", "v0",
                "wp2_surface_max", "empty"]
        return dict(zip(keys, list(out)))

    def close(self):
        if getattr(self, "handle", None):
            lib().rt_destroy_star(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rt_init_star(params: rt_star_params) -> Star:
    return Star(params)


def rt_destroy_star(star: Star) -> None:
    star.close()


def rt_sample_conversion_surface(star: Star, n, uniforms, state, weight, status, stream=None,
                                 allow_empty=True) -> int:
    allow = (RT_OK, RT_EEMPTY_SURFACE) if allow_empty else (RT_OK,)
    return _check(lib().rt_sample_conversion_surface(
        star.handle, int(n), _ptr(uniforms), _ptr(state), _ptr(weight), _ptr(status),
        _stream(stream)), allow)


def rt_sample_conversion_surface_part(star: Star, n, n_norm, uniforms, state, weight, status,
                                      stream=None, allow_empty=True) -> int:
    allow = (RT_OK, RT_EEMPTY_SURFACE) if allow_empty else (RT_OK,)
    return _check(lib().rt_sample_conversion_surface_part(
        star.handle, int(n), int(n_norm), _ptr(uniforms), _ptr(state), _ptr(weight),
        _ptr(status), _stream(stream)), allow)


def bin_acc_entries(nth, nph, nnu) -> int:
    """RT_BIN_ACC_ENTRIES: int64 entries of a sharded binning's sums."""
    return 2 + nth * nph * nnu + nth * nph + nnu


def rt_bin_part_max(n, weight, status, nth, nph, nnu, acc, stream=None) -> int:
    return _check(lib().rt_bin_part_max(int(n), _ptr(weight), _ptr(status), int(nth), int(nph),
                                        int(nnu), _ptr(acc), _stream(stream)))


def rt_bin_part_accumulate(star: Star, n, n_total, state, weight, status, nth, nph, nnu, nu_lo,
                           nu_hi, acc, ld=None, stream=None) -> int:
    """ld: row stride of the SoA state (default n)."""
    return _check(lib().rt_bin_part_accumulate(
        star.handle, int(n), int(n if ld is None else ld), int(n_total), _ptr(state),
        _ptr(weight), _ptr(status), int(nth),
        int(nph), int(nnu), float(nu_lo), float(nu_hi), _ptr(acc), _stream(stream)))


def rt_bin_part_finalize(nth, nph, nnu, n_total, acc, hist, sky=None, spec=None,
                         out_of_range=None, stream=None) -> int:
    return _check(lib().rt_bin_part_finalize(
        int(nth), int(nph), int(nnu), int(n_total), _ptr(acc), _ptr(hist), _ptr(sky), _ptr(spec),
        _ptr(out_of_range), _stream(stream)))


def rt_trace_forward(star: Star, n, state, status, nacc=None, nrej=None, counters=None,
                     opts: rt_trace_opts | None = None, stream=None) -> int:
    if opts is None:
        opts = make_opts()
    return _check(lib().rt_trace_forward(
        star.handle, int(n), _ptr(state), _ptr(status), _ptr(nacc), _ptr(nrej), _ptr(counters),
        ctypes.byref(opts), _stream(stream)))


def rt_bin_spectrum(star: Star, n, state, weight, status, nth, nph, nnu, nu_lo, nu_hi, hist,
                    sky=None, spec=None, out_of_range=None, stream=None) -> int:
    return _check(lib().rt_bin_spectrum(
        star.handle, int(n), _ptr(state), _ptr(weight), _ptr(status), int(nth), int(nph),
        int(nnu), float(nu_lo), float(nu_hi), _ptr(hist), _ptr(sky), _ptr(spec),
        _ptr(out_of_range), _stream(stream)))


def rt_trace_backward(star: Star, nx, ny, incl_rad, dist_over_R, bmax_over_R, image, status,
                      ncross=None, counters=None, Lc_cut_km=0.0,
                      opts: rt_trace_opts | None = None, stream=None) -> int:
    if opts is None:
        opts = make_opts()
    return _check(lib().rt_trace_backward(
        star.handle, int(nx), int(ny), float(incl_rad), float(dist_over_R), float(bmax_over_R),
        float(Lc_cut_km), _ptr(image), _ptr(status), _ptr(ncross), _ptr(counters),
        ctypes.byref(opts), _stream(stream)))


def rt_bin_spectrum_noalloc(params: rt_star_params, n, state, weight, status, nth, nph, nnu,
                            nu_lo, nu_hi, hist, sky=None, spec=None, out_of_range=None,
                            stream=None) -> int:
    return _check(lib().rt_bin_spectrum_noalloc(
        ctypes.byref(params), int(n), _ptr(state), _ptr(weight), _ptr(status), int(nth),
        int(nph), int(nnu), float(nu_lo), float(nu_hi), _ptr(hist), _ptr(sky), _ptr(spec),
        _ptr(out_of_range), _stream(stream)))


def rt_flops_per_step(dispersion: int, plasma: int) -> list[float]:
    out = (ctypes.c_double * 4)()
    _check(lib().rt_flops_per_step(int(dispersion), int(plasma), out))
    return list(out)


def rt_flops_per_step_df(dispersion: int, plasma: int) -> list[float]:
    out = (ctypes.c_double * 2)()
    _check(lib().rt_flops_per_step_df(int(dispersion), int(plasma), out))
    return list(out)


def rt_flux_value(star: Star, n, state, weight, status, incl_rad, kappa, F_ray, F,
                  stream=None) -> int:
    return _check(lib().rt_flux_value(star.handle, int(n), _ptr(state), _ptr(weight),
                                      _ptr(status), float(incl_rad), float(kappa), _ptr(F_ray),
                                      _ptr(F), _stream(stream)))


def rt_flux_gradient(star: Star, n, uniforms, nacc, incl_rad, kappa, grad, F, status=None,
                     counters=None, opts: rt_trace_opts | None = None, stream=None,
                     tape_max_bytes: int = -1) -> int:
    """Returns the bytes of the store used (the full step tape, or the
    checkpoints when the tape exceeds ``tape_max_bytes``; -1: half of the free
    device memory, 0: checkpoints always)."""
    if opts is None:
        opts = make_opts()
    nbytes = ctypes.c_int64(0)
    _check(lib().rt_flux_gradient(star.handle, int(n), _ptr(uniforms), _ptr(nacc),
                                  float(incl_rad), float(kappa), ctypes.byref(opts), _ptr(grad),
                                  _ptr(F), _ptr(status), _ptr(counters), int(tape_max_bytes),
                                  ctypes.byref(nbytes), _stream(stream)))
    return int(nbytes.value)


def rt_timestamps_reset(timestamps, n_instances, stream=None) -> int:
    return _check(lib().rt_timestamps_reset(_ptr(timestamps), int(n_instances), _stream(stream)))


class Graph:
    """Owning wrapper of an ``rt_graph`` (a captured sample -> trace -> bin step)."""

    def __init__(self, batch, uniforms, state, weight, status, counters, opts, nth, nph, nnu,
                 nu_lo, nu_hi, hist, out_of_range):
        h = _vp()
        _check(lib().rt_batch_graph_create(batch.handle, _ptr(uniforms), _ptr(state),
                                           _ptr(weight), _ptr(status), _ptr(counters),
                                           ctypes.byref(opts), int(nth), int(nph), int(nnu),
                                           float(nu_lo), float(nu_hi), _ptr(hist),
                                           _ptr(out_of_range), ctypes.byref(h)))
        self.handle = h
        self.keep = (batch, opts)      # the graph refers to both

    def launch(self, stream=None) -> int:
        return _check(lib().rt_graph_launch(self.handle, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            lib().rt_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rt_batch_graph_create(batch, uniforms, state, weight, status, counters, opts, nth, nph, nnu,
                          nu_lo, nu_hi, hist, out_of_range) -> Graph:
    return Graph(batch, uniforms, state, weight, status, counters, opts, nth, nph, nnu, nu_lo,
                 nu_hi, hist, out_of_range)


def rt_graph_launch(graph: Graph, stream=None) -> int:
    return graph.launch(stream)


def rt_graph_destroy(graph: Graph) -> None:
    graph.close()


def rt_batch_autotune(batch, state, status, opts, rays_per_star=2048, stream=None) -> dict:
    blk = ctypes.c_int32(0)
    bps = ctypes.c_int32(0)
    refill = ctypes.c_int32(0)
    claim = ctypes.c_int32(0)
    ms = ctypes.c_double(0.0)
    nc = ctypes.c_int32(0)
    cand = (ctypes.c_double * 64)()
    _check(lib().rt_batch_autotune(batch.handle, _ptr(state), _ptr(status), ctypes.byref(opts),
                                   int(rays_per_star), ctypes.byref(blk), ctypes.byref(bps),
                                   ctypes.byref(refill), ctypes.byref(claim), ctypes.byref(ms),
                                   ctypes.byref(nc), cand, 64, _stream(stream)))
    return {"block": blk.value, "blocks_per_sm": bps.value, "refill_min": refill.value,
            "rays_per_claim": claim.value, "ms": ms.value,
            "candidates_ms": list(cand)[:min(nc.value, 64)]}


def rt_count_status(n, status, stream=None) -> tuple[int, list[int]]:
    counts = (ctypes.c_int64 * RAY_NSTATUS)()
    st = _check(lib().rt_count_status(int(n), _ptr(status), counts, _stream(stream)),
                (RT_OK, RT_EPARTIAL))
    return st, list(counts)


class Batch:
    """Owning wrapper of an ``rt_batch``: stars traced in one persistent launch."""

    def __init__(self, stars: list[Star], counts: list[int]):
        n = len(stars)
        arr = (_vp * n)(*[s.handle for s in stars])
        cnt = (ctypes.c_int64 * n)(*[int(c) for c in counts])
        h = _vp()
        _check(lib().rt_init_batch(arr, n, cnt, ctypes.byref(h)))
        self.handle = h
        self.stars = list(stars)        # the handles must outlive the batch
        self.counts = list(counts)
        self.N = int(sum(counts))

    def close(self):
        if getattr(self, "handle", None):
            lib().rt_destroy_batch(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rt_init_batch(stars, counts) -> Batch:
    return Batch(stars, counts)


def rt_destroy_batch(batch: Batch) -> None:
    batch.close()


def rt_sample_batch(batch: Batch, uniforms, state, weight, status, stream=None) -> int:
    return _check(lib().rt_sample_batch(batch.handle, _ptr(uniforms), _ptr(state), _ptr(weight),
                                        _ptr(status), _stream(stream)),
                  (RT_OK, RT_EEMPTY_SURFACE))


def rt_batch_set_norm(batch: Batch, n_norm=None) -> int:
    """Per-star weight normalisation counts (None: the ray counts)."""
    if n_norm is None:
        return _check(lib().rt_batch_set_norm(batch.handle, None))
    arr = (ctypes.c_int64 * len(n_norm))(*[int(v) for v in n_norm])
    return _check(lib().rt_batch_set_norm(batch.handle, arr))


def rt_trace_batch(batch: Batch, state, status, nacc=None, nrej=None, counters=None,
                   opts: rt_trace_opts | None = None, stream=None) -> int:
    if opts is None:
        opts = make_opts()
    return _check(lib().rt_trace_batch(batch.handle, _ptr(state), _ptr(status), _ptr(nacc),
                                       _ptr(nrej), _ptr(counters), ctypes.byref(opts),
                                       _stream(stream)))


def rt_bin_batch(batch: Batch, state, weight, status, nth, nph, nnu, nu_lo, nu_hi, hist,
                 out_of_range, stream=None) -> int:
    return _check(lib().rt_bin_batch(batch.handle, _ptr(state), _ptr(weight), _ptr(status),
                                     int(nth), int(nph), int(nnu), float(nu_lo), float(nu_hi),
                                     _ptr(hist), _ptr(out_of_range), _stream(stream)))


def rt_batch_set_images(batch: Batch, stars, descs, image, img_status, ncross=None) -> int:
    """descs: (nx, ny, incl_rad, dist_over_R, bmax_over_R, Lc_cut_km) per image."""
    n = len(stars)
    arr = (_vp * max(n, 1))(*[s.handle for s in stars])
    d = (rt_image_desc * max(n, 1))(*[rt_image_desc(int(x[0]), int(x[1]), float(x[2]),
                                                    float(x[3]), float(x[4]), float(x[5]))
                                      for x in descs])
    r = _check(lib().rt_batch_set_images(batch.handle, n, arr, d, _ptr(image), _ptr(img_status),
                                         _ptr(ncross)))
    batch.image_stars = list(stars)     # the handles must outlive the batch
    batch.nimg = n
    return r


def rt_hamilton_rhs(star: Star, n, state, H, dydl, stream=None) -> int:
    return _check(lib().rt_hamilton_rhs(star.handle, int(n), _ptr(state), _ptr(H), _ptr(dydl),
                                        _stream(stream)))


def rt_measure_alu_peak(iters64=7500, iters32=560000, stream=None) -> dict:
    """Measured FP64 / FP32 multiply-add throughput of the current GPU (the
    defaults run each timed kernel for ~0.15 s on a GB300)."""
    out = (ctypes.c_double * 4)()
    _check(lib().rt_measure_alu_peak(int(iters64), int(iters32), out, _stream(stream)))
    return {"fp64_flops": out[0], "fp32_flops": out[1], "fp64_ms": out[2], "fp32_ms": out[3]}


def rt_last_error() -> str:
    return lib().rt_last_error().decode()


def rt_version() -> int:
    return int(lib().rt_version())


EXPORTED = ["rt_init_star", "rt_destroy_star", "rt_star_info", "rt_sample_conversion_surface",
            "rt_trace_forward", "rt_bin_spectrum", "rt_count_status", "rt_last_error",
            "rt_version", "rt_init_batch", "rt_destroy_batch", "rt_sample_batch",
            "rt_trace_batch", "rt_bin_batch", "rt_trace_backward", "rt_bin_spectrum_noalloc",
            "rt_flops_per_step", "rt_flux_value", "rt_flux_gradient", "rt_timestamps_reset",
            "rt_batch_graph_create", "rt_graph_launch", "rt_graph_destroy", "rt_batch_autotune",
            "rt_batch_set_images", "rt_sample_conversion_surface_part", "rt_bin_part_max",
            "rt_bin_part_accumulate", "rt_bin_part_finalize", "rt_batch_set_norm",
            "rt_measure_alu_peak", "rt_hamilton_rhs", "rt_flops_per_step_df"]
