"""Batched persistent launch over several stars with uneven ray counts: the
batch path (one sampling pass per star, ONE trace launch over all stars, per
star histograms) reproduces the single-star path bit for bit in FP64 with one
lane per ray throughout (tail = 1), and to rounding with the six-lane tail
mode (which rays are parked depends on the launch), and agrees with the
oracle on the sampled states."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2309_08655_gb300 import inputs as I  # noqa: E402
from paper_2309_08655_gb300 import rt  # noqa: E402

from . import gpu_util as G  # noqa: E402

NB = (16, 8, 32)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2309_08655_gb300.build import build
    build()
    assert torch.cuda.is_available()


def _setup():
    kws = I.stars_config1()
    pick = [5, 0, 13, 2]             # light, empty surface, medium, heavy axion
    counts = [300, 257, 1000, 513]   # uneven, ragged
    stars_kw = [kws[j] for j in pick]
    us = [I.sample_uniforms(2000 + j, c) for j, c in zip(pick, counts)]
    return stars_kw, counts, us


@pytest.mark.parametrize("tail", [1, 0])
def test_batch_equals_single_star_path(oracle, tail):
    stars_kw, counts, us = _setup()
    dev = torch.device("cuda:0")
    N = sum(counts)
    stars = [rt.Star(rt.make_params(**kw)) for kw in stars_kw]
    batch = rt.Batch(stars, counts)
    u_all = torch.from_numpy(np.ascontiguousarray(np.concatenate(us, axis=1))).to(dev)
    st = torch.empty((8, N), dtype=torch.float64, device=dev)
    w = torch.empty(N, dtype=torch.float64, device=dev)
    s = torch.empty(N, dtype=torch.uint8, device=dev)
    assert rt.rt_sample_batch(batch, u_all, st, w, s) == rt.RT_OK
    ctr = torch.zeros(8, dtype=torch.int64, device=dev)
    rt.rt_trace_batch(batch, st, s, counters=ctr, opts=rt.make_opts(rtol=1e-10, tail=tail))
    hist = torch.empty((len(stars),) + NB, dtype=torch.float64, device=dev)
    oor = torch.empty(len(stars), dtype=torch.float64, device=dev)
    rt.rt_bin_batch(batch, st, w, s, *NB, 0.0, 9.0, hist, oor)
    torch.cuda.synchronize()
    st_b, s_b, w_b, h_b = G.to_np(st, s, w, hist)
    off = np.concatenate([[0], np.cumsum(counts)])
    traced = 0
    for j, kw in enumerate(stars_kw):
        star, st1, w1, s1, _ = G.gpu_sample(kw, us[j])
        G.gpu_trace(star, st1, s1, rtol=1e-10, tail=tail)
        h1 = G.gpu_bin(star, st1, w1, s1, *NB)[0]
        a, b = off[j], off[j + 1]
        assert np.array_equal(w_b[a:b], w1.cpu().numpy())
        if tail == 1:
            assert np.array_equal(st_b[:, a:b], st1.cpu().numpy())
            assert np.array_equal(s_b[a:b], s1.cpu().numpy())
            assert np.array_equal(h_b[j], h1)
        else:
            s1n = s1.cpu().numpy()
            same = s_b[a:b] == s1n
            assert same.mean() > 0.99
            tr = same & (s1n != rt.RAY_NO_ROOT)
            if tr.any():
                d = G.rel_state_diff(st_b[:, a:b][:, tr], st1.cpu().numpy()[:, tr])
                assert np.median(d) < 1e-12
            if h1.sum() > 0:
                assert np.abs(h_b[j] - h1).sum() / h1.sum() < 1e-4
        traced += int((s1.cpu().numpy() != rt.RAY_NO_ROOT).sum())
        # sampled states agree with the oracle
        so, wo, sto = oracle.sample(oracle.star_vector(**kw), us[j])
        assert np.array_equal(sto == rt.RAY_NO_ROOT, s_b[a:b] == rt.RAY_NO_ROOT)
        assert np.allclose(wo, w_b[a:b], rtol=1e-9, atol=0)
    assert int(ctr[2]) == traced


def test_batch_mixed_runs_every_ray_once():
    stars_kw, counts, us = _setup()
    dev = torch.device("cuda:0")
    N = sum(counts)
    stars = [rt.Star(rt.make_params(**kw)) for kw in stars_kw]
    batch = rt.Batch(stars, counts)
    u_all = torch.from_numpy(np.ascontiguousarray(np.concatenate(us, axis=1))).to(dev)
    st = torch.empty((8, N), dtype=torch.float64, device=dev)
    w = torch.empty(N, dtype=torch.float64, device=dev)
    s = torch.empty(N, dtype=torch.uint8, device=dev)
    rt.rt_sample_batch(batch, u_all, st, w, s)
    ready = int((s == rt.RAY_READY).sum())
    ctr = torch.zeros(8, dtype=torch.int64, device=dev)
    rt.rt_trace_batch(batch, st, s, counters=ctr,
                      opts=rt.make_opts(rtol=1e-8, precision=rt.PREC_MIXED))
    torch.cuda.synchronize()
    c = ctr.cpu().numpy()
    assert c[2] == ready
    assert int((s == rt.RAY_READY).sum()) == 0 and int((s >= rt.RAY_NSTATUS).sum()) == 0


def _images():
    """Three backward images of two stars (one of them also a forward star of
    the batch), ragged sizes."""
    kw_a = dict(I.star_config0())
    kw_b = dict(M_sun=1.4, R_km=10.0, B0_G=1e14, P_s=1.0, theta_m=0.5, psi=0.4, m_a_eV=1e-5,
                g_GeVinv=1e-12, rho_GeV_cm3=0.45, v0_kms=200.0, dispersion=0, resonance=0,
                fa_model=0, weight_mode=0, prop_metric=0, phase_mode=0, plasma=0,
                plasma_a=0.0)
    descs = [(12, 10, 1.0, 1e4, 2.0, 0.0), (7, 9, 0.3, 1e4, 25.0, 0.0),
             (16, 16, 1.2, 1e4, 2.0, 1.0)]
    return [kw_b, kw_a, kw_b], descs


@pytest.mark.parametrize("precision", [rt.PREC_FP64, rt.PREC_MIXED])
def test_batch_with_images_matches_separate_calls(precision):
    """Rays and pixels in one persistent launch (one queue) against
    rt_trace_batch on the rays alone (one lane per ray, tail = 1) and
    rt_trace_backward on each image alone.  Every item is traced by the same
    integrator code whichever lane takes it, but the code is compiled into a
    different kernel, so results agree to rounding amplified by each ray's
    conditioning (the bound of the tail-mode test): identical statuses and
    crossing counts on nearly every item, end points and pixel values to 1e-9
    (FP64) or 1e-5 (FP32 stages) for 90 % of them, and totals.  The counters
    add rays and pixels; the timestamps cover both."""
    stars_kw, counts, us = _setup()
    dev = torch.device("cuda:0")
    N = sum(counts)
    mixed = precision == rt.PREC_MIXED
    rtol = 1e-8 if mixed else 1e-10
    tol = 1e-5 if mixed else 1e-9
    opts = rt.make_opts(rtol=rtol, precision=precision, tail=1)
    stars = [rt.Star(rt.make_params(**kw)) for kw in stars_kw]
    u_all = torch.from_numpy(np.ascontiguousarray(np.concatenate(us, axis=1))).to(dev)
    b0 = rt.Batch(stars, counts)
    st = torch.empty((8, N), dtype=torch.float64, device=dev)
    w = torch.empty(N, dtype=torch.float64, device=dev)
    s = torch.empty(N, dtype=torch.uint8, device=dev)
    rt.rt_sample_batch(b0, u_all, st, w, s)
    rt.rt_trace_batch(b0, st, s, opts=opts)
    torch.cuda.synchronize()
    st_r, s_r = G.to_np(st, s)
    ikw, descs = _images()
    istars = [rt.Star(rt.make_params(**kw)) for kw in ikw]
    sep = []
    for sb, d in zip(istars, descs):
        img = torch.empty((d[1], d[0]), dtype=torch.float64, device=dev)
        sti = torch.empty((d[1], d[0]), dtype=torch.uint8, device=dev)
        nci = torch.empty((d[1], d[0]), dtype=torch.int32, device=dev)
        rt.rt_trace_backward(sb, d[0], d[1], d[2], d[3], d[4], img, sti, nci, None,
                             Lc_cut_km=d[5], opts=opts)
        torch.cuda.synchronize()
        sep.append([a.ravel() for a in G.to_np(img, sti, nci)])
    img_s, ist_s, inc_s = (np.concatenate([x[k] for x in sep]) for k in range(3))
    P = img_s.size
    batch = rt.Batch(stars, counts)
    image = torch.full((P,), float("nan"), dtype=torch.float64, device=dev)
    ist = torch.full((P,), 255, dtype=torch.uint8, device=dev)
    inc = torch.full((P,), -1, dtype=torch.int32, device=dev)
    rt.rt_batch_set_images(batch, istars, descs, image, ist, inc)
    rt.rt_sample_batch(batch, u_all, st, w, s)
    ctr = torch.zeros(8, dtype=torch.int64, device=dev)
    ts = torch.zeros(1 + len(stars) + len(descs), dtype=torch.int64, device=dev)
    rt.rt_timestamps_reset(ts, len(stars) + len(descs))
    o2 = rt.make_opts(rtol=rtol, precision=precision, tail=1, timestamps=ts)
    rt.rt_trace_batch(batch, st, s, counters=ctr, opts=o2)
    torch.cuda.synchronize()
    st_u, s_u, img_u, ist_u, inc_u, c, t = G.to_np(st, s, image, ist, inc, ctr, ts)
    # rays
    traced = (s_r != rt.RAY_NO_ROOT) & (s_r != rt.RAY_READY)
    same = traced & (s_u == s_r)
    assert same.sum() >= 0.99 * traced.sum()
    d = G.rel_state_diff(st_u[:, same], st_r[:, same])
    assert np.percentile(d, 90) <= tol, np.percentile(d, 90)
    # pixels
    assert np.all(np.isin(ist_u, [rt.RAY_ESCAPED, rt.RAY_CAPTURED, rt.RAY_MAXSTEPS]))
    psame = (ist_u == ist_s) & (inc_u == inc_s)
    assert psame.mean() >= 0.98, psame.mean()
    lit = psame & (inc_s > 0)
    rel = np.abs(img_u[lit] - img_s[lit]) / np.abs(img_s[lit])
    assert np.percentile(rel, 90) <= tol, np.percentile(rel, 90)
    assert abs(img_u.sum() - img_s.sum()) <= 1e3 * tol * abs(img_s.sum())
    assert int(c[2]) == int(traced.sum()) + P          # every item finished once
    assert int(c[6]) == int(inc_u.sum())
    assert t[0] > 0 and np.all(t[1 + len(stars):] >= t[0])
    # removing the images gives the rays-only launch back (bitwise)
    rt.rt_batch_set_images(batch, [], [], None, None)
    rt.rt_sample_batch(batch, u_all, st, w, s)
    rt.rt_trace_batch(batch, st, s, opts=opts)
    torch.cuda.synchronize()
    assert np.array_equal(G.to_np(st)[0], st_r)


def test_batch_set_images_rejects_bad_geometry():
    stars_kw, counts, _ = _setup()
    dev = torch.device("cuda:0")
    stars = [rt.Star(rt.make_params(**kw)) for kw in stars_kw]
    batch = rt.Batch(stars, counts)
    ikw, descs = _images()
    istars = [rt.Star(rt.make_params(**kw)) for kw in ikw]
    img = torch.empty(1000, dtype=torch.float64, device=dev)
    st = torch.empty(1000, dtype=torch.uint8, device=dev)
    with pytest.raises(rt.RtError):
        rt.rt_batch_set_images(batch, istars[:1], [(4, 4, 0.3, 5.0, 6.0, 0.0)], img, st)
    with pytest.raises(rt.RtError):
        rt.rt_batch_set_images(batch, istars[:1], [(0, 4, 0.3, 1e4, 6.0, 0.0)], img, st)
