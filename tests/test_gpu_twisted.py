"""The twisted magnetar magnetosphere (Sec. 6, Eq. neMag: n_e = lambda psi
sin^2 theta B0 (R/r)^3 / (e r), no conversion on open field lines) on the GPU
against the FP64 oracle, through the C ABI: conversion-surface samples and
weights (1e-12 / 1e-11, the same statuses, excision included), FP64 forward
end points (1e-10 on the well-conditioned set, one lane per ray and in tail
mode), binned flux (1e-4), the mixed-precision kernel, and backward pixels
(1e-8 on the well-conditioned pixels).  The axion masses put the conversion
surface between 1 and 3 R, where the Goldreich-Julian density of the same star
has no resonance at all."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2309_08655_gb300 import inputs as I  # noqa: E402
from paper_2309_08655_gb300 import rt  # noqa: E402

from . import gpu_util as G  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2309_08655_gb300.build import build
    build()
    assert torch.cuda.is_available()


def _star(m_a=1e-3, dispersion=0, P_s=3.76, theta_m=math.radians(30.0), phase_mode=1):
    """The misaligned magnetar-like star of the benchmark (B0 = 1.6e14 G,
    30 deg, M = 1.5 Msun, R = 11 km) with the twisted density, lambda psi = 0.2."""
    kw = I.star_config0()
    kw.update(M_sun=1.5, R_km=11.0, B0_G=1.6e14, P_s=P_s, theta_m=theta_m, m_a_eV=m_a,
              phase_mode=phase_mode, plasma=rt.PLASMA_TWISTED, plasma_a=0.2,
              dispersion=dispersion)
    return kw


@pytest.mark.parametrize("m_a,dispersion,P_s", [(1e-3, 0, 3.76), (2e-3, 1, 3.76),
                                                 (1e-3, 0, 5.8e-4)])
def test_twisted_samples_and_weights(oracle, m_a, dispersion, P_s):
    kw = _star(m_a, dispersion, P_s)
    u = I.sample_uniforms(300, 3000)
    star, st_d, w_d, s_d, code = G.gpu_sample(kw, u)
    assert code == rt.RT_OK
    st_g, w_g, s_g = G.to_np(st_d, w_d, s_d)
    st_o, w_o, s_o = oracle.sample(oracle.star_vector(**kw), u)
    assert np.array_equal(s_g, s_o)
    ok = s_o == oracle.RAY_READY
    assert ok.sum() > 300
    assert G.rel_state_diff(st_g[:, ok], st_o[:, ok]).max() < 1e-12
    assert np.abs(w_g[ok] / w_o[ok] - 1).max() < 1e-11
    assert np.all(w_g[~ok] == 0)
    # the Goldreich-Julian density of the same (slow) star has no resonance here
    if P_s > 1.0:
        gj = dict(kw, plasma=rt.PLASMA_GJ, plasma_a=0.0)
        assert rt.Star(rt.make_params(**gj)).info()["empty"]


def test_twisted_open_field_lines_cut_samples():
    """A millisecond rotator's light cylinder cuts the surface: fewer samples,
    and the samples kept are exactly those of the slow rotator whose field line
    stays inside it."""
    u = I.sample_uniforms(301, 3000)
    _, st_s, w_s, s_s, _ = G.gpu_sample(_star(P_s=3.76), u)
    _, st_f, w_f, s_f, _ = G.gpu_sample(_star(P_s=5.8e-4), u)
    st_s, w_s, s_s, st_f, w_f, s_f = G.to_np(st_s, w_s, s_s, st_f, w_f, s_f)
    kept = s_f == rt.RAY_READY
    assert 0 < kept.sum() < (s_s == rt.RAY_READY).sum()
    assert np.array_equal(st_f[:, kept], st_s[:, kept])
    assert np.array_equal(w_f[kept], w_s[kept])


@pytest.mark.parametrize("dispersion", [0, 1])
def test_twisted_trace_and_flux_fp64(oracle, dispersion):
    kw = _star(1e-3, dispersion)
    sv = oracle.star_vector(**kw)
    u = I.sample_uniforms(302, 2048)
    st0, w0, s0 = oracle.sample(sv, u)
    ref, sref, good, spread = G.well_conditioned(oracle, sv, st0, s0, 1e-10)
    star = rt.Star(rt.make_params(**kw))
    out = {}
    for tail in (1, 0):
        st_d = torch.from_numpy(st0.copy()).cuda()
        s_d = torch.from_numpy(s0.copy()).cuda()
        G.gpu_trace(star, st_d, s_d, rtol=1e-10, tail=tail)
        out[tail] = G.to_np(st_d, s_d)
    traced = s0 == oracle.RAY_READY
    for tail, (st_g, s_g) in out.items():
        assert (s_g[traced] == sref[traced]).mean() > 0.99
        g = good & traced & (s_g == sref)
        assert g.sum() > 0.3 * traced.sum()
        assert G.rel_state_diff(st_g[:, g], ref[:, g]).max() < 1e-10, tail
    # binned flux against the oracle's
    w_d = torch.from_numpy(w0.copy()).cuda()
    st_d = torch.from_numpy(out[1][0].copy()).cuda()
    s_d = torch.from_numpy(out[1][1].copy()).cuda()
    hist, _, _, _ = G.gpu_bin(star, st_d, w_d, s_d)
    h_o, _ = oracle.bin_rays(sv, ref, w0, sref)
    assert np.abs(hist - h_o).sum() / h_o.sum() < 1e-4


def test_twisted_trace_mixed(oracle):
    """FP32 stages: the same statuses for nearly every ray and the binned flux
    within 1e-4 of the oracle's (the FP32 floor moves end points by ~1e-7)."""
    kw = _star(1e-3, 0)
    sv = oracle.star_vector(**kw)
    u = I.sample_uniforms(303, 2048)
    st0, w0, s0 = oracle.sample(sv, u)
    ref = st0.copy()
    sref = s0.copy()
    oracle.trace_forward(sv, oracle.trace_opts(rtol=1e-10), ref, sref)
    star = rt.Star(rt.make_params(**kw))
    st_d = torch.from_numpy(st0.copy()).cuda()
    s_d = torch.from_numpy(s0.copy()).cuda()
    G.gpu_trace(star, st_d, s_d, rtol=1e-8, precision=rt.PREC_MIXED)
    st_g, s_g = G.to_np(st_d, s_d)
    traced = s0 == oracle.RAY_READY
    assert (s_g[traced] == sref[traced]).mean() > 0.99
    same = traced & (s_g == sref)
    d = G.rel_state_diff(st_g[:, same], ref[:, same])
    assert np.percentile(d, 90) < 1e-5
    hist, _, _, _ = G.gpu_bin(star, st_d, torch.from_numpy(w0.copy()).cuda(), s_d)
    h_o, _ = oracle.bin_rays(sv, ref, w0, sref)
    assert np.abs(hist - h_o).sum() / h_o.sum() < 1e-4


def test_twisted_backward_pixels(oracle):
    """Backward image of the twisted magnetosphere: FP64 pixels against the
    oracle on the well-conditioned set, and the mixed image close to FP64."""
    kw = _star(1e-3, 0, phase_mode=0)
    kw.update(psi=0.4)
    nx, ny, incl, D, bmax = 20, 18, 1.0, 1e4, 2.0
    sv = oracle.star_vector(**kw)
    o = oracle.trace_opts(rtol=1e-10)
    ia, sa, na = oracle.trace_backward(sv, o, nx, ny, incl, D, bmax, 0.0)
    ib, sb, nb = oracle.trace_backward(sv, o, nx, ny, incl, D, bmax, 0.0, variant="contracted")
    star = rt.Star(rt.make_params(**kw))
    res = {}
    for prec, rtol in ((rt.PREC_FP64, 1e-10), (rt.PREC_MIXED, 1e-8)):
        img = torch.empty((ny, nx), dtype=torch.float64, device=G.dev())
        st = torch.empty((ny, nx), dtype=torch.uint8, device=G.dev())
        nc = torch.empty((ny, nx), dtype=torch.int32, device=G.dev())
        rt.rt_trace_backward(star, nx, ny, incl, D, bmax, img, st, nc, None,
                             opts=rt.make_opts(rtol=rtol, precision=prec))
        torch.cuda.synchronize()
        res[prec] = G.to_np(img, st, nc)
    ig, sg, ng = res[rt.PREC_FP64]
    scale = np.maximum(np.abs(ia), 1e-300)
    good = (sa == sb) & (na == nb) & (np.abs(ia - ib) / scale <= 1e-10)
    lit = na > 0
    assert lit.mean() > 0.1 and good[lit].mean() > 0.8
    assert np.array_equal(ng[good], na[good])
    assert (np.abs(ig - ia) / scale)[good].max() <= 1e-8
    im, sm, nm = res[rt.PREC_MIXED]
    same = (nm == ng) & (sm == sg)
    assert same.mean() > 0.95
    assert abs(im.sum() - ig.sum()) <= 1e-3 * abs(ig.sum())
