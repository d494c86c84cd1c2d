"""FP64 CPU oracle for the forward/backward axion ray tracer (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does: it fails
loudly when its CUDA library is missing.

The C++ sources in this directory implement the method of McDonald & Witte,
"Generalized Ray Tracing for Axions in Astrophysical Plasmas", in plain FP64:
Hamilton's equations (Eq. Hamilton) of the strong-field Hamiltonian
(Eq. StrongBHam) on Schwarzschild (Eq. SchwarzshildMetric1), differentiated by
dual numbers; the conversion-surface sampler and power weight (Sec. 3-4); an
adaptive Dormand-Prince 5(4) integrator; binning (Sec. 2.2); and the backward
image-plane estimator (Sec. 2.1).  This module builds ``liboracle.so`` with
g++ and wraps it with ctypes.

Parity status of each oracle function (what pins it) is listed in the test
files ``tests/test_oracle_*.py``.  The absolute normalisation of the
anisotropic weight (Eq. CPAnisoCurved is an ansatz of the paper) is parity
unpinned beyond the checks named there.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = ["or_oracle.cpp"]
_HDR = ["or_dual.hpp", "or_model.hpp", "or_dopri.hpp"]

# parameter-vector layout (or_model.hpp) and trace options (or_oracle.cpp)
STAR_KEYS = [
    "M_sun", "R_km", "B0_G", "P_s", "theta_m", "psi", "m_a_eV", "g_GeVinv",
    "rho_GeV_cm3", "v0_kms", "dispersion", "resonance", "fa_model", "weight_mode",
    "prop_metric", "phase_mode", "plasma", "plasma_a", "rotation",
]
STAR_DEFAULTS = dict(
    M_sun=1.0, R_km=10.0, B0_G=1e14, P_s=1.0, theta_m=0.0, psi=0.0, m_a_eV=1e-5,
    g_GeVinv=1e-12, rho_GeV_cm3=0.45, v0_kms=200.0, dispersion=0, resonance=0,
    fa_model=0, weight_mode=0, prop_metric=0, phase_mode=0, plasma=0, plasma_a=0.0,
    rotation=0,
)
ROTATION_SNAPSHOT, ROTATION_RIGID = 0, 1
DISP_ANISO, DISP_ISO = 0, 1
PLASMA_GJ, PLASMA_VACUUM, PLASMA_HOMOG, PLASMA_LINEAR_Z, PLASMA_RADIAL, PLASMA_TWISTED = range(6)
RAY_READY, RAY_ESCAPED, RAY_CAPTURED, RAY_NO_ROOT = 0, 1, 2, 3
RAY_MAXSTEPS, RAY_NAN, RAY_STIFF, RAY_LAMBDA_END = 4, 5, 6, 7

_lib = None
_lib_contracted = None
# The "contracted" build is the same source compiled with fused multiply-add
# contraction: a second, equally valid FP64 evaluation of every formula.  The
# spread between the two builds measures how much a ray's end point moves under
# rounding-level changes of every operation; the GPU tests compare the CUDA
# path's deviations against that spread.
_SO_CONTRACTED = os.path.join(_HERE, "liboracle_contracted.so")


def _flags(variant: str) -> list[str]:
    if variant == "contracted":
        import platform
        extra = ["-mfma"] if platform.machine() in ("x86_64", "AMD64") else []
        return ["-ffp-contract=fast"] + extra
    return ["-ffp-contract=off"]


def build(force: bool = False, variant: str = "strict") -> str:
    """Compile liboracle.so in place (g++, FP64; the reference build has no
    FMA contraction)."""
    so = _SO if variant == "strict" else _SO_CONTRACTED
    srcs = [os.path.join(_HERE, s) for s in _SRC]
    deps = srcs + [os.path.join(_HERE, h) for h in _HDR]
    if not force and os.path.exists(so):
        so_t = os.path.getmtime(so)
        if all(os.path.getmtime(d) <= so_t for d in deps):
            return so
    tmp = so + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", *_flags(variant), "-fPIC", "-shared", "-pthread",
           "-o", tmp] + srcs
    subprocess.check_call(cmd, cwd=_HERE)
    os.replace(tmp, so)
    return so


def lib_contracted():
    global _lib_contracted
    if _lib_contracted is None:
        build(variant="contracted")
        L = ctypes.CDLL(_SO_CONTRACTED)
        dp = ctypes.POINTER(ctypes.c_double)
        L.or_trace_forward.restype = None
        L.or_trace_forward.argtypes = [dp, dp, ctypes.c_long, dp, ctypes.POINTER(ctypes.c_uint8),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       dp, ctypes.c_int]
        L.or_trace_backward.restype = None
        L.or_trace_backward.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double, dp,
                                        ctypes.POINTER(ctypes.c_uint8),
                                        ctypes.POINTER(ctypes.c_int), ctypes.c_int]
        L.or_backward_points.restype = None
        L.or_backward_points.argtypes = [dp, dp, ctypes.c_long, dp, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, dp,
                                         ctypes.POINTER(ctypes.c_uint8),
                                         ctypes.POINTER(ctypes.c_int), ctypes.c_int]
        _lib_contracted = L
    return _lib_contracted


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        ip = ctypes.POINTER(ctypes.c_int)
        L.or_sample.restype = ctypes.c_long
        L.or_sample.argtypes = [dp, ctypes.c_long, dp, dp, dp, u8p, ctypes.c_int]
        L.or_sample_parts.restype = None
        L.or_sample_parts.argtypes = [dp, ctypes.c_long, dp, dp, ctypes.c_int]
        L.or_sample_parts_count.restype = ctypes.c_int
        L.or_sample_parts_count.argtypes = []
        L.or_trace_forward.restype = None
        L.or_trace_forward.argtypes = [dp, dp, ctypes.c_long, dp, u8p, ip, ip, dp, ctypes.c_int]
        L.or_trace_rk4.restype = None
        L.or_trace_rk4.argtypes = [dp, ctypes.c_long, dp, dp, ctypes.c_long, ctypes.c_int]
        L.or_hamiltonian.restype = None
        L.or_hamiltonian.argtypes = [dp, ctypes.c_long, dp, dp, dp]
        L.or_plasma_freq2.restype = None
        L.or_plasma_freq2.argtypes = [dp, ctypes.c_long, dp, ctypes.c_double, dp]
        L.or_photon_energy.restype = ctypes.c_double
        L.or_photon_energy.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double]
        L.or_maxwell_speed.restype = ctypes.c_double
        L.or_maxwell_speed.argtypes = [ctypes.c_int, ctypes.c_double]
        L.or_resonance_h.restype = ctypes.c_double
        L.or_resonance_h.argtypes = [dp, dp, dp, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, dp]
        L.or_resonance_root.restype = ctypes.c_int
        L.or_resonance_root.argtypes = [dp, dp, dp, ctypes.c_double, ctypes.c_double, dp]
        L.or_star_constants.restype = None
        L.or_star_constants.argtypes = [dp, dp]
        L.or_bin.restype = None
        L.or_bin.argtypes = [dp, ctypes.c_long, dp, dp, u8p, ctypes.c_int, ctypes.c_int,
                             ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        L.or_trace_backward.restype = None
        L.or_trace_backward.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double, dp,
                                        u8p, ip, ctypes.c_int]
        L.or_backward_points.restype = None
        L.or_backward_points.argtypes = [dp, dp, ctypes.c_long, dp, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, dp, u8p, ip,
                                         ctypes.c_int]
        L.or_dp5_tableau.restype = None
        L.or_dp5_tableau.argtypes = [dp, dp, dp, dp, dp, dp]
        L.or_dp5_linear.restype = ctypes.c_long
        L.or_dp5_linear.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.or_dp5_linear_dense.restype = None
        L.or_dp5_linear_dense.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def star_vector(**kw) -> np.ndarray:
    p = dict(STAR_DEFAULTS)
    for k, v in kw.items():
        if k not in p:
            raise KeyError(k)
        p[k] = v
    return np.array([float(p[k]) for k in STAR_KEYS], dtype=np.float64)


def trace_opts(rtol=1e-10, atol=None, r_out_over_R=1000.0, max_steps=100000, lambda_max=0.0,
               r_capture_over_R=1.0, crossing_grid=0) -> np.ndarray:
    """crossing_grid: 0 = the exhaustive backward crossing search; n > 0 = a
    plain sign test at n points per step (a comparison baseline only)."""
    if atol is None:
        atol = rtol
    return np.array([rtol, atol, r_out_over_R, max_steps, lambda_max, r_capture_over_R,
                     crossing_grid], dtype=np.float64)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


SAMPLE_PARTS = ["ok", "r", "n0", "n1", "n2", "khat0", "khat1", "khat2", "E", "K2", "wp2",
                "cos2", "Bmag", "dhdr", "gradh0", "gradh1", "gradh2", "Psi", "W1", "w", "A",
                "kinf", "omega_inf", "shape"]


def sample_parts(star: np.ndarray, u: np.ndarray, nthreads: int | None = None) -> dict:
    """Intermediate quantities of each sample (scaled units: r in R, E and
    momenta in m_a, dhdr in m_a / R, gradh = dh/d(x/R) in m_a; Bmag [eV^2],
    Psi [eV^3], w [W]); 'ok' is 0 for samples without a resonance."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    n = u.shape[1]
    L = lib()
    k = L.or_sample_parts_count()
    assert k == len(SAMPLE_PARTS)
    out = np.zeros((n, k))
    L.or_sample_parts(_dp(star), n, _dp(u), _dp(out), nthreads or default_threads())
    return {name: out[:, j] for j, name in enumerate(SAMPLE_PARTS)}


def sample(star: np.ndarray, u: np.ndarray, nthreads: int | None = None):
    """u: (6, n) uniforms in (0, 1).  Returns (state (8, n), weight (n,), status (n,))."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    n = u.shape[1]
    state = np.zeros((8, n))
    w = np.zeros(n)
    st = np.zeros(n, dtype=np.uint8)
    lib().or_sample(_dp(star), n, _dp(u), _dp(state), _dp(w), _u8(st),
                    nthreads or default_threads())
    return state, w, st


def trace_forward(star: np.ndarray, opts: np.ndarray, state: np.ndarray, status: np.ndarray,
                  nthreads: int | None = None, variant: str = "strict"):
    """Traces READY rays in place.  Returns (nacc, nrej, lambda_end)."""
    assert state.flags.c_contiguous and state.dtype == np.float64 and state.shape[0] == 8
    assert status.dtype == np.uint8
    n = state.shape[1]
    nacc = np.zeros(n, dtype=np.int32)
    nrej = np.zeros(n, dtype=np.int32)
    lam = np.zeros(n)
    L = lib() if variant == "strict" else lib_contracted()
    L.or_trace_forward(_dp(star), _dp(opts), n, _dp(state), _u8(status), _ip(nacc), _ip(nrej),
                       _dp(lam), nthreads or default_threads())
    return nacc, nrej, lam


def trace_rk4(star, state, lam_end, nsteps, nthreads=None):
    n = state.shape[1]
    lam_end = np.ascontiguousarray(lam_end, dtype=np.float64)
    lib().or_trace_rk4(_dp(star), n, _dp(state), _dp(lam_end), int(nsteps),
                       nthreads or default_threads())


def hamiltonian(star, state, with_rhs=False):
    state = np.ascontiguousarray(state, dtype=np.float64)
    n = state.shape[1]
    H = np.zeros(n)
    d = np.zeros((6, n)) if with_rhs else None
    lib().or_hamiltonian(_dp(star), n, _dp(state), _dp(H), _dp(d) if with_rhs else None)
    return (H, d) if with_rhs else H


def plasma_freq2(star, x_km, psi=0.0):
    x_km = np.ascontiguousarray(x_km, dtype=np.float64)
    n = x_km.shape[1]
    out = np.zeros(n)
    lib().or_plasma_freq2(_dp(star), n, _dp(x_km), float(psi), _dp(out))
    return out


def photon_energy(dispersion, K2, wp2, cos2):
    return lib().or_photon_energy(int(dispersion), float(K2), float(wp2), float(cos2))


def maxwell_speed(u, fa_model=0):
    return lib().or_maxwell_speed(int(fa_model), float(u))


def resonance_h(star, n, khat, omega_inf, psi, r):
    n = np.ascontiguousarray(n, dtype=np.float64)
    khat = np.ascontiguousarray(khat, dtype=np.float64)
    d = ctypes.c_double(0.0)
    h = lib().or_resonance_h(_dp(star), _dp(n), _dp(khat), float(omega_inf), float(psi),
                             float(r), ctypes.byref(d))
    return h, d.value


def resonance_root(star, n, khat, omega_inf, psi=0.0):
    n = np.ascontiguousarray(n, dtype=np.float64)
    khat = np.ascontiguousarray(khat, dtype=np.float64)
    r = ctypes.c_double(0.0)
    ok = lib().or_resonance_root(_dp(star), _dp(n), _dp(khat), float(omega_inf), float(psi),
                                 ctypes.byref(r))
    return r.value if ok else None


def star_constants(star):
    out = np.zeros(6)
    lib().or_star_constants(_dp(star), _dp(out))
    return dict(rs_over_R=out[0], wp2_coef=out[1], B0_eV2=out[2], R_inv_eV=out[3],
                n_inf_eV3=out[4], n_gj_coef_cm3=out[5])


def line_flux(star, state, weight, status, incl, kappa):
    """The smoothed line flux toward o = (sin incl, 0, cos incl) [W / sr]:
    F = sum over ESCAPED rays of w K(khat . o), K(mu) = C exp(kappa (mu - 1)),
    C = kappa / (2 pi (1 - exp(-2 kappa))), the von Mises-Fisher kernel of
    unit mass on the sphere; khat the static orthonormal-frame momentum
    direction at the end point (the direction binning uses, Sec. 2.2).  The
    paper differentiates nothing: this is the functional whose gradient the
    library's adjoint computes, written from its definition."""
    sv = np.asarray(star, dtype=np.float64)
    R_km = sv[STAR_KEYS.index("R_km")]
    rs = 0.0 if sv[STAR_KEYS.index("prop_metric")] == 1 else star_constants(sv)["rs_over_R"]
    esc = np.asarray(status) == RAY_ESCAPED
    x = np.asarray(state)[:3, esc] / R_km
    k = np.asarray(state)[3:6, esc]
    r = np.sqrt((x * x).sum(0))
    n = x / r
    A = 1.0 - rs / r
    ko = k + (np.sqrt(A) - 1.0) * (n * k).sum(0) * n
    mu = (ko[0] * np.sin(incl) + ko[2] * np.cos(incl)) / np.sqrt((ko * ko).sum(0))
    C = kappa / (2.0 * np.pi * -np.expm1(-2.0 * kappa))
    return float((np.asarray(weight)[esc] * C * np.exp(kappa * (mu - 1.0))).sum())


def bin_rays(star, state, weight, status, nth=64, nph=32, nnu=128, nu_lo=0.0, nu_hi=9.0):
    state = np.ascontiguousarray(state, dtype=np.float64)
    weight = np.ascontiguousarray(weight, dtype=np.float64)
    status = np.ascontiguousarray(status, dtype=np.uint8)
    n = state.shape[1]
    hist = np.zeros((nth, nph, nnu))
    oor = np.zeros(1)
    lib().or_bin(_dp(star), n, _dp(state), _dp(weight), _u8(status), nth, nph, nnu,
                 float(nu_lo), float(nu_hi), _dp(hist), _dp(oor))
    return hist, float(oor[0])


def dp5_tableau():
    c, b, bh, e, d = (np.zeros(7) for _ in range(5))
    a = np.zeros((7, 6))
    lib().or_dp5_tableau(_dp(c), _dp(a), _dp(b), _dp(bh), _dp(e), _dp(d))
    return dict(c=c, a=a, b=b, bh=bh, e=e, d=d)


def dp5_linear(M, y0, T, rtol, atol=None):
    M = np.ascontiguousarray(M, dtype=np.float64)
    y = np.array(y0, dtype=np.float64)
    nacc = lib().or_dp5_linear(_dp(M), _dp(y), float(T), float(rtol),
                               float(rtol if atol is None else atol))
    return y, nacc


def dp5_linear_dense(M, y0, h, th):
    M = np.ascontiguousarray(M, dtype=np.float64)
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    out = np.zeros(6)
    lib().or_dp5_linear_dense(_dp(M), _dp(y0), float(h), float(th), _dp(out))
    return out


def trace_backward(star, opts, nx, ny, incl, dist_over_R=1e4, bmax_over_R=50.0, Lc_cut_km=0.0,
                   nthreads=None, variant: str = "strict"):
    """Backward image (ny, nx) of pixel contributions to dP/dOmega [W/sr] at
    inclination incl (rad) from the rotation axis; returns (image, status, ncross)."""
    img = np.zeros((ny, nx))
    st = np.zeros((ny, nx), dtype=np.uint8)
    nc = np.zeros((ny, nx), dtype=np.int32)
    L = lib() if variant == "strict" else lib_contracted()
    L.or_trace_backward(_dp(star), _dp(opts), int(nx), int(ny), float(incl),
                            float(dist_over_R), float(bmax_over_R), float(Lc_cut_km), _dp(img),
                            _u8(st), _ip(nc), nthreads or default_threads())
    return img, st, nc


def backward_points(star, opts, b, incl, dist_over_R=1e4, Lc_cut_km=0.0, nthreads=None,
                    variant: str = "strict"):
    """Backward integrand at plane points b (n, 2) in units of R: dP/dOmega per
    unit plane area [W / sr / R^2]; returns (value, status, ncross)."""
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1, 2)
    n = b.shape[0]
    v = np.zeros(n)
    st = np.zeros(n, dtype=np.uint8)
    nc = np.zeros(n, dtype=np.int32)
    L = lib() if variant == "strict" else lib_contracted()
    L.or_backward_points(_dp(star), _dp(opts), n, _dp(b), float(incl), float(dist_over_R),
                             float(Lc_cut_km), _dp(v), _u8(st), _ip(nc),
                             nthreads or default_threads())
    return v, st, nc
