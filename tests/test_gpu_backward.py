"""Parity of the CUDA backward image-plane tracer (Sec. 2.1, Eq. BackPower;
every resonance crossing, Sec. 5.1.3) with the FP64 oracle, through the C ABI.

Both sides trace one time-reversed ray per pixel centre from the same plane
and sum sqrt(A) Psi |dt/dl| / |dg/dl| over the sign changes of g = E_gamma -
E_a.  A pixel's value is a smooth function of the ray except where a crossing
pair appears or disappears (a ray grazing the resonance): there two equally
valid FP64 evaluations disagree.  The well-conditioned set is therefore the
pixels on which the oracle's strict build and its FMA-contracted build agree
in status and crossing count and to 1e-10 in value; on it the GPU must agree
to 1e-8 relative (the factor 100 between the two bounds is the one the
forward end-point tests use).  The image total is compared with a bound of
ten times the strict-contracted spread of the total.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2309_08655_gb300 import rt  # noqa: E402

from . import gpu_util as G  # noqa: E402

RTOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2309_08655_gb300.build import build
    build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _star(dispersion, theta_m=0.5, psi=0.4, m_a_eV=1e-5, fa_model=0):
    """B0 = 1e14 G, P = 1 s, M = 1.4 Msun, R = 10 km; with m_a = 1e-5 eV the
    conversion surface lies within 2 R (a plane 4 R wide sees all of it)."""
    return dict(M_sun=1.4, R_km=10.0, B0_G=1e14, P_s=1.0, theta_m=theta_m, psi=psi,
                m_a_eV=m_a_eV, g_GeVinv=1e-12, rho_GeV_cm3=0.45, v0_kms=200.0,
                dispersion=dispersion, resonance=0, fa_model=fa_model, weight_mode=0,
                prop_metric=0, phase_mode=0, plasma=0, plasma_a=0.0)


def gpu_backward(kw, nx, ny, incl, D, bmax, Lc_cut_km=0.0, rtol=RTOL, precision=rt.PREC_FP64):
    star = rt.Star(rt.make_params(**kw))
    img = torch.full((ny, nx), float("nan"), dtype=torch.float64, device=G.dev())
    st = torch.full((ny, nx), 255, dtype=torch.uint8, device=G.dev())
    nc = torch.full((ny, nx), -1, dtype=torch.int32, device=G.dev())
    ctr = torch.zeros(8, dtype=torch.int64, device=G.dev())
    rt.rt_trace_backward(star, nx, ny, incl, D, bmax, img, st, nc, ctr, Lc_cut_km=Lc_cut_km,
                         opts=rt.make_opts(rtol=rtol, precision=precision))
    torch.cuda.synchronize()
    return img.cpu().numpy(), st.cpu().numpy(), nc.cpu().numpy(), ctr.cpu().numpy()


def oracle_backward(oracle, kw, nx, ny, incl, D, bmax, Lc_cut_km=0.0, rtol=RTOL):
    sv = oracle.star_vector(**kw)
    o = oracle.trace_opts(rtol=rtol)
    a = oracle.trace_backward(sv, o, nx, ny, incl, D, bmax, Lc_cut_km)
    b = oracle.trace_backward(sv, o, nx, ny, incl, D, bmax, Lc_cut_km, variant="contracted")
    return a, b


def _compare(a, b, g, min_good=0.9):
    (ia, sa, na), (ib, sb, nb) = a, b
    ig, sg, ng, ctr = g
    scale = np.maximum(np.abs(ia), 1e-300)
    spread = np.abs(ia - ib) / scale
    good = (sa == sb) & (na == nb) & (spread <= 1e-10)
    lit = na > 0
    if lit.any():
        assert good[lit].mean() >= min_good, good[lit].mean()
    assert np.array_equal(sg[good], sa[good])
    assert np.array_equal(ng[good], na[good])
    rel = np.abs(ig - ia) / scale
    assert np.all(np.isfinite(ig))
    worst = rel[good].max() if good.any() else 0.0
    assert worst <= 1e-8, worst
    tot_spread = abs(ia.sum() - ib.sum())
    assert abs(ig.sum() - ia.sum()) <= 10.0 * tot_spread + 1e-9 * abs(ia.sum()), (
        ig.sum(), ia.sum(), tot_spread)
    assert int(ctr[2]) == ia.size                       # every pixel finished
    assert int(ctr[6]) == int(ng.sum())                 # crossings counted
    return good


@pytest.mark.parametrize("dispersion", [0, 1])
def test_backward_parity_misaligned(oracle, dispersion):
    kw = _star(dispersion)
    args = (24, 20, 1.0, 1e4, 2.0)       # ragged: nx != ny, neither a warp multiple
    a, b = oracle_backward(oracle, kw, *args)
    g = gpu_backward(kw, *args)
    _compare(a, b, g)
    # the plane sees the emission; a ray leaves the resonance as often as it
    # enters it (the plasma reflects it before it reaches the star)
    assert (a[2] > 0).mean() > 0.2
    assert a[0].sum() > 0
    assert np.all(g[2] % 2 == 0)


def test_backward_parity_aligned_pole_on(oracle):
    """Aligned rotator seen from the rotation axis: the image is symmetric
    under the reflection of the plane's e2 axis (y -> -y) and, with an even
    grid, under b -> -b."""
    kw = _star(0, theta_m=0.0, psi=0.0)
    args = (16, 16, 0.0, 1e4, 2.0)
    a, b = oracle_backward(oracle, kw, *args)
    g = gpu_backward(kw, *args)
    good = _compare(a, b, g)
    img = g[0]
    sym = good & good[::-1, ::-1]
    assert np.allclose(img[sym], img[::-1, ::-1][sym], rtol=1e-8, atol=0)


def test_backward_conversion_length_cut(oracle):
    kw = _star(0)
    args = (16, 12, 0.7, 1e4, 2.0)
    full = gpu_backward(kw, *args)
    a, b = oracle_backward(oracle, kw, *args, Lc_cut_km=1.0)
    g = gpu_backward(kw, *args, Lc_cut_km=1.0)
    _compare(a, b, g)
    # the cut only removes crossings
    assert np.all(g[2] <= full[2])
    assert g[0].sum() < full[0].sum()


def test_backward_single_pixel_and_empty_ray(oracle):
    """One pixel; and a pixel whose ray never meets the conversion surface
    (b far outside it) contributes exactly zero."""
    kw = _star(1)
    a, b = oracle_backward(oracle, kw, 1, 1, 0.3, 1e4, 0.5)
    g = gpu_backward(kw, 1, 1, 0.3, 1e4, 0.5)
    assert g[1][0, 0] == a[1][0, 0]
    assert a[2][0, 0] > 0
    if a[2][0, 0] == b[2][0, 0] and abs(a[0][0, 0] - b[0][0, 0]) <= 1e-10 * abs(a[0][0, 0]):
        assert abs(g[0][0, 0] - a[0][0, 0]) <= 1e-8 * abs(a[0][0, 0])
    # a 2 x 1 plane 20 R wide: both pixel centres at |b| = 5 R miss the surface
    g2 = gpu_backward(kw, 2, 1, 0.3, 1e4, 10.0)
    assert np.all(g2[0] == 0.0) and np.all(g2[2] == 0)
    assert np.all(g2[1] == rt.RAY_ESCAPED)


def test_backward_rejects_bad_arguments():
    kw = _star(0)
    star = rt.Star(rt.make_params(**kw))
    img = torch.zeros((4, 4), dtype=torch.float64, device=G.dev())
    st = torch.zeros((4, 4), dtype=torch.uint8, device=G.dev())
    with pytest.raises(rt.RtError):
        rt.rt_trace_backward(star, 4, 4, 0.3, 5.0, 6.0, img, st)        # plane inside the box
    with pytest.raises(rt.RtError):
        rt.rt_trace_backward(star, 4, 4, math.nan, 1e4, 6.0, img, st)


# --- mixed precision (FP32 stages, FP64 state, crossing search and estimator) --


@pytest.mark.parametrize("dispersion", [0, 1])
def test_backward_mixed_close_to_fp64(dispersion):
    """The mixed-precision image against the FP64 kernel's on the same plane:
    the FP32 stages move each ray by ~1e-7 of its path (rtol 1e-8), so pixels
    whose crossing count agrees agree to 1e-4 relative, the pixels whose count
    differs (a crossing pair at a grazing ray) are rare, and the image total
    agrees to 1e-3."""
    kw = _star(dispersion)
    args = (40, 36, 1.0, 1e4, 2.0)
    f = gpu_backward(kw, *args)
    m = gpu_backward(kw, *args, rtol=1e-8, precision=rt.PREC_MIXED)
    (i64, s64, n64, c64), (im, sm, nm, cm) = f, m
    assert np.all(np.isfinite(im))
    assert np.all((sm == rt.RAY_ESCAPED) | (sm == rt.RAY_CAPTURED))
    assert int(cm[2]) + 0 == im.size              # every pixel finished once
    same = (nm == n64) & (sm == s64)
    assert same.mean() >= 0.98, same.mean()
    lit = same & (n64 > 0)
    rel = np.abs(im[lit] - i64[lit]) / np.abs(i64[lit])
    assert np.percentile(rel, 99) <= 1e-4, np.percentile(rel, 99)
    assert abs(im.sum() - i64.sum()) <= 1e-3 * abs(i64.sum())
    assert np.all(nm % 2 == 0)


def test_backward_mixed_hands_floor_pixels_to_fp64():
    """At a tolerance below the FP32 rounding floor pixels are handed to the
    FP64 kernel (counter 4) and traced again from the plane there: every pixel
    still ends once with a final status, and the handed pixels' values are
    those of the FP64 kernel (bitwise), so the image matches it closely."""
    kw = _star(0)
    args = (16, 16, 1.0, 1e4, 2.0)
    f = gpu_backward(kw, *args, rtol=1e-12)
    m = gpu_backward(kw, *args, rtol=1e-12, precision=rt.PREC_MIXED)
    assert int(m[3][4]) > 0
    assert int(m[3][2]) == 16 * 16
    # final statuses only (at this tolerance some rays exhaust max_steps)
    assert np.all(np.isin(m[1], [rt.RAY_ESCAPED, rt.RAY_CAPTURED, rt.RAY_MAXSTEPS]))
    eq = (m[0] == f[0]) & (m[2] == f[2]) & (m[1] == f[1])
    assert eq.mean() >= int(m[3][4]) / (16 * 16) - 1e-12
    done = np.isin(m[1], [rt.RAY_ESCAPED, rt.RAY_CAPTURED]) & (m[1] == f[1]) & (m[2] == f[2])
    assert abs(m[0][done].sum() - f[0][done].sum()) <= 1e-3 * abs(f[0][done].sum())


@pytest.mark.parametrize("precision", [rt.PREC_FP64, rt.PREC_MIXED])
def test_grazing_pairs_counted_to_the_closed_form_rim(oracle, precision):
    """Flat space, isotropic spherical medium (omega_p^2 = 8 m_a^2 (R/r)^3):
    the ray of impact parameter b reaches the resonance sphere r_c = 2 R iff
    b <= b_rim = r_c sqrt(W^2 - 1) / W (its angular momentum b W is
    conserved).  Just inside the rim its two crossings merge at the turning
    point, between two samples of the sign of g: the search must still count
    both, none just outside, and agree with the oracle's value.  At a
    relative distance eps from the rim, g peaks at about -eps v0^2 (outside)
    at the turning point, so the test resolves eps down to 1e-8 in FP64 and
    1e-4 with FP32 stages (trajectory error ~1e-7); near the rim the pixel
    value is sensitive to the ray as ~1 / (2 eps), which sets its tolerance."""
    v0_kms = 30000.0
    kw = dict(M_sun=0.0, R_km=10.0, B0_G=1e14, P_s=1.0, theta_m=0.3, m_a_eV=1e-5,
              dispersion=1, fa_model=1, plasma=rt.PLASMA_RADIAL, plasma_a=8.0, v0_kms=v0_kms)
    v0 = v0_kms / 299792.458
    W = math.sqrt(1.0 + v0 * v0)
    b_rim = 2.0 * math.sqrt(W * W - 1.0) / W
    fp64 = precision == rt.PREC_FP64
    rtol = 1e-10 if fp64 else 1e-8
    eps_in = [1e-2, 1e-3, 1e-4] + ([1e-5, 1e-6, 1e-7, 1e-8] if fp64 else [])
    sv = oracle.star_vector(**kw)
    for eps in eps_in:
        b = b_rim * (1.0 - eps)
        # two pixels of a 2 x 1 image, centred at (-b, 0) and (b, 0)
        img, st, nc, ctr = gpu_backward(kw, 2, 1, 0.7, 1e4, 2.0 * b, rtol=rtol,
                                        precision=precision)
        assert np.all(st == rt.RAY_ESCAPED)
        assert np.all(nc == 2), (eps, nc)
        if fp64 and eps >= 1e-6:
            v, _, nco = oracle.backward_points(sv, oracle.trace_opts(rtol=rtol),
                                               [[-b, 0.0], [b, 0.0]], 0.7)
            assert np.all(nco == 2)
            ref = v * (2.0 * b) * (4.0 * b)          # pixel area 2b x 4b
            assert np.abs(img.ravel() / ref - 1).max() < 2e-10 / eps, (eps, img, ref)
    for eps in ((1e-2, 1e-5, 1e-8) if fp64 else (1e-2, 1e-3, 1e-4)):
        img, st, nc, ctr = gpu_backward(kw, 2, 1, 0.7, 1e4, 2.0 * b_rim * (1.0 + eps),
                                        rtol=rtol, precision=precision)
        assert np.all(nc == 0) and np.all(img == 0.0)


def test_forward_and_backward_agree_at_the_equator_full_resolution():
    """The paper's forward/backward consistency (Sec. 2.4) at sizes the
    oracle cannot reach: the config-0 star (aligned Goldreich-Julian,
    anisotropic), forward dP/dOmega binned over the flat equatorial band
    87.5 - 92.5 deg from 2^21 rays, against the backward image total averaged
    over the band's inclinations (four Gauss points in cos over 87.5 - 90 deg,
    the star being mirror symmetric) at 2048 x 512 pixels over +-12 R.  Both
    paths are parity-tested against the oracle pixel by pixel and ray by ray;
    here they must agree with each other within 3 % plus three Monte-Carlo
    errors (pixel-centre sums resolve the bright rims to ~3 % at this size)."""
    from paper_2309_08655_gb300 import inputs as I
    kw = I.star_config0()
    n = 1 << 21
    u = I.sample_uniforms(79, n)
    star, st, w, s, _ = G.gpu_sample(kw, u)
    G.gpu_trace(star, st, s, rtol=1e-9)
    st_g, w_g, s_g = G.to_np(st, w, s)
    esc = s_g == rt.RAY_ESCAPED
    x = st_g[:3] / kw["R_km"]
    r = np.linalg.norm(x, axis=0)
    r[r == 0] = 1.0
    nv = x / r
    A = 1.0 - 2.0 * kw["M_sun"] * 1.4766250 / kw["R_km"] / r
    ko = st_g[3:6] + (np.sqrt(np.clip(A, 1e-12, 1)) - 1) * (nv * st_g[3:6]).sum(0) * nv
    th = np.degrees(np.arccos(np.clip(ko[2] / np.maximum(np.linalg.norm(ko, axis=0), 1e-300),
                                      -1, 1)))
    m = esc & (th >= 87.5) & (th < 92.5)
    dOm = 2 * math.pi * 2 * math.cos(math.radians(87.5))
    fwd = w_g[m].sum() / dOm
    sig = np.std(np.where(m, w_g, 0.0)) * math.sqrt(n) / dOm
    c, wc = np.polynomial.legendre.leggauss(4)
    ca, cb = 0.0, math.cos(math.radians(87.5))
    bwd = 0.0
    for ci, wi in zip(c, wc):
        cc = 0.5 * (ca + cb) + 0.5 * (cb - ca) * ci
        img, st_i, nc, ctr = gpu_backward(kw, 2048, 512, math.acos(cc), 1e4, 12.0, rtol=1e-9)
        assert not (nc[0].any() or nc[-1].any() or nc[:, 0].any() or nc[:, -1].any())
        bwd += 0.5 * wi * img.sum()
    print(f"equatorial band: forward {fwd:.5e} +- {sig:.1e}, backward {bwd:.5e}, "
          f"ratio {bwd / fwd:.4f}")
    assert abs(bwd / fwd - 1.0) < 0.03 + 3.0 * sig / fwd, (bwd, fwd, sig)
