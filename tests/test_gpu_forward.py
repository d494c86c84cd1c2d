"""Parity of the CUDA forward path (sampling, FP64 tracing, binning) with the
FP64 oracle on the same seeded inputs, through the C ABI.

Tolerances: FP64 end points 1e-10 relative on the well-conditioned set (rays
whose oracle end point moves by at most 1e-12 between the oracle's strict FP64
build and the same source compiled with FMA contraction -- two equally valid
FP64 evaluations; 99.6 % of the config-0 rays, so the set must hold at least
98 % of the traced rays); binned flux 1e-4 relative L1; sampled states and
weights 1e-12 (both sides take the same FP64 root, differing only in
rounding).
"""
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
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _star_vec(oracle, kw):
    return oracle.star_vector(**kw)


def _config0(n=4096, first=0):
    kw = I.star_config0()
    u = I.sample_uniforms(I.CONFIG0["seed"], n, first)
    return kw, u


def test_sample_parity_config0(oracle):
    kw, u = _config0()
    star, st_d, w_d, s_d, code = G.gpu_sample(kw, u)
    assert code == rt.RT_OK
    st_g, w_g, s_g = G.to_np(st_d, w_d, s_d)
    st_o, w_o, s_o = oracle.sample(_star_vec(oracle, kw), u)
    assert np.array_equal(s_g, s_o)
    ok = s_o == oracle.RAY_READY
    assert ok.sum() > 3000
    assert G.rel_state_diff(st_g[:, ok], st_o[:, ok]).max() < 1e-12
    assert np.abs(st_g[6] / st_o[6] - 1).max() < 1e-12      # delta (Maxwellian speed)
    assert np.array_equal(st_g[7], st_o[7])
    assert np.abs(w_g[ok] / w_o[ok] - 1).max() < 1e-11
    assert np.all(w_g[~ok] == 0)


@pytest.mark.parametrize("sub", [0, 5, 7, 13])
def test_sample_parity_misaligned_rotator(oracle, sub):
    kw = I.stars_config1()[sub]
    u = I.sample_uniforms(100 + sub, 2048)
    star, st_d, w_d, s_d, code = G.gpu_sample(kw, u)
    st_g, w_g, s_g = G.to_np(st_d, w_d, s_d)
    st_o, w_o, s_o = oracle.sample(_star_vec(oracle, kw), u)
    info = star.info()
    if info["empty"]:
        assert code == rt.RT_EEMPTY_SURFACE
        assert np.all(s_g == rt.RAY_NO_ROOT) and np.all(w_g == 0)
    else:
        assert code == rt.RT_OK
    assert np.array_equal(s_g, s_o)
    ok = s_o == oracle.RAY_READY
    if ok.any():
        assert G.rel_state_diff(st_g[:, ok], st_o[:, ok]).max() < 1e-12
        assert np.abs(w_g[ok] / w_o[ok] - 1).max() < 1e-11
    assert np.allclose(st_g[7], st_o[7], rtol=0, atol=1e-15)


def _trace_parity(oracle, kw, u, rtol=1e-10, **topt):
    """GPU and oracle trace the same (oracle-sampled) initial states."""
    sv = _star_vec(oracle, kw)
    st0, w0, s0 = oracle.sample(sv, u)
    ref, sref, good, spread = G.well_conditioned(oracle, sv, st0, s0, rtol, **topt)
    star = rt.Star(rt.make_params(**kw))
    st_d = torch.from_numpy(st0.copy()).cuda()
    s_d = torch.from_numpy(s0.copy()).cuda()
    nacc, nrej, ctr = G.gpu_trace(star, st_d, s_d, rtol=rtol, **_gpu_opts(topt))
    st_g, s_g, na = G.to_np(st_d, s_d, nacc)
    _trace_parity.spread = spread
    return st0, s0, ref, sref, good, st_g, s_g, na, ctr.cpu().numpy()


def _gpu_opts(topt):
    m = {"r_out_over_R": "r_out_over_R", "max_steps": "max_steps", "lambda_max": "lambda_max",
         "r_capture_over_R": "r_capture_over_R"}
    return {m[k]: v for k, v in topt.items()}


def test_trace_parity_config0_fp64(oracle):
    kw, u = _config0()
    st0, s0, ref, sref, good, st_g, s_g, na, ctr = _trace_parity(oracle, kw, u, rtol=1e-10)
    traced = s0 == oracle.RAY_READY
    # statuses agree (up to the rare ill-conditioned grazing ray)
    assert (s_g[traced] == sref[traced]).mean() > 0.995
    # well-conditioned set (oracle strict vs contracted within 1e-12): 1e-10
    g = good & traced & (s_g == sref)
    assert g.sum() > 0.98 * traced.sum()          # oracle: 99.6 % well-conditioned
    d = G.rel_state_diff(st_g[:, g], ref[:, g])
    assert d.max() < 1e-10, np.sort(d)[-5:]
    # all rays: GPU deviations are of the size of the oracle's own spread
    # between two valid FP64 evaluations (rounding amplified by the ray)
    spread = _trace_parity.spread
    m = traced & (s_g == sref)
    dev_all = G.rel_state_diff(st_g[:, m], ref[:, m])
    for q in (50, 90, 99):
        assert np.percentile(dev_all, q) <= 10 * np.percentile(spread[m], q) + 1e-12, q
    # the step counters add up
    assert ctr[2] == traced.sum()
    assert ctr[0] == na.sum()
    assert ctr[3] == (s_g == rt.RAY_ESCAPED).sum()


def test_bin_parity_config0(oracle):
    kw, u = _config0()
    sv = _star_vec(oracle, kw)
    star, st_d, w_d, s_d, _ = G.gpu_sample(kw, u)
    G.gpu_trace(star, st_d, s_d, rtol=1e-10)
    hist, sky, spec, oor = G.gpu_bin(star, st_d, w_d, s_d)
    st_o, w_o, s_o = oracle.sample(sv, u)
    oracle.trace_forward(sv, oracle.trace_opts(rtol=1e-10), st_o, s_o)
    h_o, oor_o = oracle.bin_rays(sv, st_o, w_o, s_o)
    l1 = np.abs(hist - h_o).sum() / h_o.sum()
    assert l1 < 1e-4, l1
    w_g = w_d.cpu().numpy()
    s_g = s_d.cpu().numpy()
    esc = w_g[s_g == rt.RAY_ESCAPED].sum()
    assert abs(hist.sum() + oor - esc) <= 1e-9 * esc
    assert np.allclose(sky, hist.sum(axis=2), rtol=1e-12, atol=0)
    assert np.allclose(spec, hist.sum(axis=(0, 1)), rtol=1e-12, atol=0)


@pytest.mark.parametrize("n", [1, 31, 33, 257])
def test_ragged_sizes(oracle, n):
    kw, u = _config0(n, first=777)
    st0, s0, ref, sref, good, st_g, s_g, na, ctr = _trace_parity(oracle, kw, u)
    traced = s0 == 0
    assert ctr[2] == traced.sum()                      # every lane of the ragged tail ran
    assert (s_g[traced] == sref[traced]).mean() >= (0.95 if n > 30 else 1.0)
    g = good & traced & (s_g == sref)
    if g.any():
        assert G.rel_state_diff(st_g[:, g], ref[:, g]).max() < 1e-10


def test_zero_rays_and_empty_surface():
    kw = I.star_config0()
    star = rt.Star(rt.make_params(**kw))
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    assert rt.rt_sample_conversion_surface(star, 0, e, e, e, e) == rt.RT_OK
    assert rt.rt_trace_forward(star, 0, e, e) == rt.RT_OK
    heavy = dict(kw, m_a_eV=1e-3)
    u = I.sample_uniforms(9, 512)
    star2, st, w, s, code = G.gpu_sample(heavy, u)
    assert code == rt.RT_EEMPTY_SURFACE
    assert bool((s == rt.RAY_NO_ROOT).all()) and float(w.abs().sum()) == 0.0
    nacc, nrej, ctr = G.gpu_trace(star2, st, s)
    assert int(ctr[2]) == 0 and bool((s == rt.RAY_NO_ROOT).all())


def test_max_steps_bound_matches_oracle(oracle):
    kw, u = _config0(256, first=4096)
    st0, s0, ref, sref, good, st_g, s_g, na, ctr = _trace_parity(oracle, kw, u, max_steps=40)
    traced = s0 == 0
    assert np.array_equal(s_g[traced], sref[traced])
    assert (s_g == rt.RAY_MAXSTEPS).sum() > 10
    code, counts = rt.rt_count_status(256, torch.from_numpy(s_g).cuda())
    assert code == rt.RT_EPARTIAL and counts[rt.RAY_MAXSTEPS] == (s_g == rt.RAY_MAXSTEPS).sum()


def test_invalid_arguments_are_rejected_on_the_host():
    kw = I.star_config0()
    star = rt.Star(rt.make_params(**kw))
    st = torch.zeros((8, 4), dtype=torch.float64, device="cuda")
    s = torch.zeros(4, dtype=torch.uint8, device="cuda")
    with pytest.raises(rt.RtError) as e:
        rt.rt_trace_forward(star, 4, st, s, opts=rt.make_opts(rtol=-1.0))
    assert e.value.status == rt.RT_EINVAL
    with pytest.raises(rt.RtError) as e:
        rt.rt_trace_forward(star, 4, st.cpu(), s)      # host memory is refused
    assert e.value.status == rt.RT_EINVAL
    with pytest.raises(rt.RtError) as e:
        rt.rt_bin_spectrum(star, 4, st, st[0], s, 0, 32, 128, 0.0, 9.0, st)
    assert e.value.status == rt.RT_EINVAL


def test_deterministic_bitwise():
    kw, u = _config0(2048)
    outs = []
    for _ in range(2):
        star, st, w, s, _ = G.gpu_sample(kw, u)
        G.gpu_trace(star, st, s)
        h = G.gpu_bin(star, st, w, s)[0]
        outs.append((st.cpu().numpy(), s.cpu().numpy(), h))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][2], outs[1][2])


def test_closed_form_media_on_gpu():
    # flat space, planar-stratified isotropic plasma omega_p^2 = a z: parabola
    a = 0.02
    kw = dict(M_sun=0.0, R_km=1.0, B0_G=1e14, P_s=1.0, m_a_eV=1e-5, dispersion=1, plasma=3,
              plasma_a=a)
    star = rt.Star(rt.make_params(**kw))
    k0 = np.array([0.3, 0.1, 0.6])
    x0 = np.array([0.0, 0.0, 10.0])
    om2 = (k0**2).sum() + a * x0[2]
    st = np.zeros((8, 1))
    st[:3, 0] = x0
    st[3:6, 0] = k0 * 1e-5
    st[6, 0] = np.sqrt(om2) - 1
    st_d = torch.from_numpy(st).cuda()
    s_d = torch.zeros(1, dtype=torch.uint8, device="cuda")
    lam = 40.0
    G.gpu_trace(star, st_d, s_d, rtol=1e-12, lambda_max=lam, r_out_over_R=1e9,
                r_capture_over_R=1e-3)
    out = st_d.cpu().numpy()[:, 0]
    assert int(s_d.cpu()[0]) == rt.RAY_LAMBDA_END
    assert np.allclose(out[:2], x0[:2] + 2 * k0[:2] * lam, atol=1e-9)
    assert abs(out[2] - (x0[2] + 2 * k0[2] * lam - a * lam**2)) < 1e-8
    assert abs(out[5] / 1e-5 - (k0[2] - a * lam)) < 1e-11


@pytest.mark.parametrize("which", ["config0", "misaligned"])
def test_tail_mode_matches_one_lane_per_ray(oracle, which):
    """The six-lanes-per-ray tail kernel continues parked rays with the same
    steps and decisions; only summation order differs, so end points agree to
    rounding amplified by each ray's conditioning: 1e-10 on the
    well-conditioned set, identical statuses and step counts there, and both
    modes agree with the oracle."""
    if which == "config0":
        kw = I.star_config0()
        u = I.sample_uniforms(9, 4096)
    else:
        kw = I.stars_config1()[5]
        u = I.sample_uniforms(1009, 4096)
    sv = _star_vec(oracle, kw)
    st0, w0, s0 = oracle.sample(sv, u)
    ref, sref, good, spread = G.well_conditioned(oracle, sv, st0, s0, 1e-10)
    star = rt.Star(rt.make_params(**kw))
    out = {}
    for tail in (0, 1):
        st_d = torch.from_numpy(st0.copy()).cuda()
        s_d = torch.from_numpy(s0.copy()).cuda()
        nacc, nrej, ctr = G.gpu_trace(star, st_d, s_d, rtol=1e-10, tail=tail)
        out[tail] = G.to_np(st_d, s_d, nacc) + [ctr.cpu().numpy()]
    (st_a, s_a, na_a, c_a), (st_b, s_b, na_b, c_b) = out[0], out[1]
    traced = s0 == oracle.RAY_READY
    g = good & traced & (s_a == sref) & (s_b == sref)
    assert g.sum() > 0.9 * traced.sum()
    assert np.array_equal(na_a[g], na_b[g])
    assert G.rel_state_diff(st_a[:, g], st_b[:, g]).max() < 1e-10
    assert G.rel_state_diff(st_a[:, g], ref[:, g]).max() < 1e-10
    assert c_a[2] == c_b[2] == traced.sum()          # every ray finished once
    assert abs(int(c_a[0]) - int(c_b[0])) <= 0.01 * int(c_b[0])


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("which", ["misaligned_gj", "twisted_iso", "flat_sphere"])
def test_unit_probability_weights(oracle, which, mode):
    """RT_WEIGHT_UNIT_P (conversion probability set to one) and
    RT_WEIGHT_RENORM (times R_i of Eq. reweight): the same samples as the
    default mode, weights against the oracle's to 1e-11; the oracle
    differentiates h = E_gamma - E_a by dual numbers, the GPU dG by dual
    numbers and divides by the same factor as for h'."""
    if which == "misaligned_gj":
        kw = I.stars_config1()[5]
    elif which == "twisted_iso":
        kw = I.star_config0()
        kw.update(M_sun=1.5, R_km=11.0, B0_G=1.6e14, P_s=3.76, theta_m=0.5, m_a_eV=1e-3,
                  phase_mode=1, plasma=rt.PLASMA_TWISTED, plasma_a=0.2, dispersion=1)
    else:
        kw = I.star_config0()
        kw.update(M_sun=0.0, m_a_eV=1e-5, plasma=rt.PLASMA_RADIAL, plasma_a=8.0, dispersion=1)
    kw = dict(kw, weight_mode=mode)
    u = I.sample_uniforms(500, 2048)
    star, st_d, w_d, s_d, code = G.gpu_sample(kw, u)
    st_g, w_g, s_g = G.to_np(st_d, w_d, s_d)
    st_o, w_o, s_o = oracle.sample(_star_vec(oracle, kw), u)
    assert np.array_equal(s_g, s_o)
    ok = s_o == oracle.RAY_READY
    assert ok.sum() > 200
    assert G.rel_state_diff(st_g[:, ok], st_o[:, ok]).max() < 1e-12
    assert np.abs(w_g[ok] / w_o[ok] - 1).max() < 1e-11
    # the default mode samples the same states with other weights
    _, st_p, w_p, s_p, _ = G.gpu_sample(dict(kw, weight_mode=rt.WEIGHT_PAG), u)
    assert np.array_equal(G.to_np(s_p)[0], s_g)
    assert not np.allclose(G.to_np(w_p)[0][ok], w_g[ok])
    # the backward tracer and the gradient need the conversion probability
    img = torch.empty((2, 2), dtype=torch.float64, device=G.dev())
    st2 = torch.empty((2, 2), dtype=torch.uint8, device=G.dev())
    with pytest.raises(rt.RtError):
        rt.rt_trace_backward(star, 2, 2, 0.3, 1e4, 3.0, img, st2)


@pytest.mark.parametrize("dispersion", [0, 1])
def test_flat_propagation_mode(oracle, dispersion):
    """App. B's first approximation (RT_METRIC_FLAT): photons start with the
    momenta of the curved-space resonance but propagate with M = 0 in
    Hamilton's equations.  End points against the oracle's same mode (1e-10 on
    the well-conditioned set), and they differ from the curved propagation."""
    kw = dict(I.star_config0(), prop_metric=1, dispersion=dispersion)
    u = I.sample_uniforms(600, 1024)
    st0, s0, ref, sref, good, st_g, s_g, na, ctr = _trace_parity(oracle, kw, u, rtol=1e-10)
    traced = s0 == oracle.RAY_READY
    assert (s_g[traced] == sref[traced]).mean() > 0.99
    g = good & traced & (s_g == sref)
    assert g.sum() > 0.3 * traced.sum()
    assert G.rel_state_diff(st_g[:, g], ref[:, g]).max() < 1e-10
    cur = _trace_parity(oracle, dict(kw, prop_metric=0), u, rtol=1e-10)
    esc = traced & (s_g == rt.RAY_ESCAPED) & (cur[6] == rt.RAY_ESCAPED)
    assert esc.sum() > 100
    assert np.median(G.rel_state_diff(st_g[:, esc], cur[5][:, esc])) > 1e-6


def test_claim_order_does_not_change_results():
    # the star of the benchmark whose rays include the longest null-cone rays
    kw = I.stars_config1()[15]
    star, st_d, w_d, s_d, code = G.gpu_sample(kw, I.sample_uniforms(500, 8192))
    out = {}
    for order in (rt.CLAIM_COST, rt.CLAIM_INDEX):
        st, s = st_d.clone(), s_d.clone()
        nacc, nrej, ctr = G.gpu_trace(star, st, s, rtol=1e-10, tail=1, claim_order=order)
        out[order] = G.to_np(st, s, nacc, nrej, ctr)
    a, b = out[rt.CLAIM_COST], out[rt.CLAIM_INDEX]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)                 # one lane per ray: bitwise
    with pytest.raises(rt.RtError) as e:
        G.gpu_trace(star, st_d.clone(), s_d.clone(), claim_order=2)
    assert e.value.status == rt.RT_EINVAL


def test_claim_order_does_not_change_mixed_results():
    """Cost-ordered claims in the mixed-precision kernel (FP32 stages): the
    rays nearest the null cone are claimed first; one lane per ray, every
    ray's end point, status and step counts are bitwise those of index order
    (also for the rays handed to the FP64 pass)."""
    kw = I.stars_config1()[15]
    star, st_d, w_d, s_d, code = G.gpu_sample(kw, I.sample_uniforms(502, 8192))
    out = {}
    for order in (rt.CLAIM_COST, rt.CLAIM_INDEX):
        st, s = st_d.clone(), s_d.clone()
        nacc, nrej, ctr = G.gpu_trace(star, st, s, rtol=1e-8, precision=rt.PREC_MIXED, tail=1,
                                      claim_order=order)
        out[order] = G.to_np(st, s, nacc, nrej, ctr)
    a, b = out[rt.CLAIM_COST], out[rt.CLAIM_INDEX]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_express_lane_matches_index_order(oracle):
    # cost order in tail mode: the rays nearest the null cone run six lanes per
    # ray from the start (express lane), the others one lane per ray
    kw = I.stars_config1()[15]
    u = I.sample_uniforms(501, 16384)
    sv = oracle.star_vector(**kw)
    star, st_d, w_d, s_d, code = G.gpu_sample(kw, u)
    out = {}
    for name, order in (("cost", rt.CLAIM_COST), ("cost_again", rt.CLAIM_COST),
                        ("index", rt.CLAIM_INDEX)):
        st, s = st_d.clone(), s_d.clone()
        nacc, nrej, ctr = G.gpu_trace(star, st, s, rtol=1e-10, claim_order=order)
        out[name] = G.to_np(st, s, nacc, ctr)
    a, b, c = out["cost"], out["cost_again"], out["index"]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)                    # reproducible
    traced = s_d.cpu().numpy() == rt.RAY_READY
    assert a[3][2] == traced.sum() == c[3][2]          # every ray traced once
    assert (a[1][traced] == c[1][traced]).mean() > 0.999
    m = traced & (a[1] == c[1]) & (a[1] == rt.RAY_ESCAPED)
    d = G.rel_state_diff(a[0][:, m], c[0][:, m])
    assert np.median(d) < 1e-13 and np.percentile(d, 99) < 1e-9
    # the express rays themselves against the oracle
    st0 = st_d.cpu().numpy()
    x = st0[:3] / kw["R_km"]
    r = np.linalg.norm(x, axis=0)
    tm = kw["theta_m"]
    mvec = np.array([np.sin(tm) * np.cos(st0[7]), np.sin(tm) * np.sin(st0[7]),
                     np.full(st0.shape[1], np.cos(tm))])
    n = x / np.where(r > 0, r, 1)
    mu = (mvec * n).sum(0)
    F = 3 * n[2] * mu - mvec[2]
    cc = 6 * mu * n[2]
    g = np.array([3 * n[2] * mvec[0] - cc * n[0], 3 * n[2] * mvec[1] - cc * n[1],
                  3 * (mu + n[2] * mvec[2]) - cc * n[2]])
    dist = np.abs(F) / np.maximum(np.linalg.norm(g, axis=0), 1e-300)
    near = np.where(traced & (dist < 1e-3))[0]
    assert near.size > 5
    ref, sref, good, spread = G.well_conditioned(oracle, sv, st0[:, near].copy(),
                                                 s_d.cpu().numpy()[near].copy(), 1e-10)
    gsel = good & (sref == a[1][near])
    if gsel.any():
        assert G.rel_state_diff(a[0][:, near][:, gsel], ref[:, gsel]).max() < 1e-10
