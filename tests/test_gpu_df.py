"""Double-float tracing (RT_PREC_DF) against the FP64 oracle and the GPU's
own FP64 path.

The double-float integrator takes the FP64 integrator's steps, events and
decisions with every operation in double-float arithmetic (unit roundoff
2^-48 instead of 2^-53).  Bars:
* end points vs the oracle on the well-conditioned set (the rays whose oracle
  end point moves by <= 1e-12 between two valid FP64 evaluations): 1e-10 for
  99.9 % of them, the FP64 path's bar -- the larger rounding (x32) stays below
  it on rays that amplify rounding by at most 1e-12 / 2^-53 ~ 1e4 (x 3.6e-15 =
  3.6e-11) -- and 1e-6 for all (a step decision on a near-tie may flip);
* binned flux vs the oracle: 1e-8 relative L1 (config 0 and a misaligned
  production sub-batch);
* statuses as the FP64 path's (99.5 %);
* claim order (with the express warps of cost order), claim size, refill
  threshold and batching change nothing, bit for bit (one lane per ray: a
  ray's arithmetic does not depend on its neighbours).
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


def _trace(kw, st0, s0, **opts):
    star = rt.Star(rt.make_params(**kw))
    st_d = torch.from_numpy(st0.copy()).cuda()
    s_d = torch.from_numpy(s0.copy()).cuda()
    nacc, nrej, ctr = G.gpu_trace(star, st_d, s_d, **opts)
    st_g, s_g, na = G.to_np(st_d, s_d, nacc)
    return star, st_g, s_g, na, ctr.cpu().numpy()


@pytest.mark.parametrize("which", ["config0", "misaligned"])
def test_df_end_points_match_oracle(oracle, which):
    if which == "config0":
        kw, u = I.star_config0(), I.sample_uniforms(0, 4096)
    else:
        kw, u = dict(I.stars_config1()[0], m_a_eV=1e-5), I.sample_uniforms(3, 2048)
    sv = oracle.star_vector(**kw)
    st0, w0, s0 = oracle.sample(sv, u)
    ref, sref, good, spread = G.well_conditioned(oracle, sv, st0, s0, 1e-10)
    _, st_g, s_g, na, ctr = _trace(kw, st0, s0, rtol=1e-10, precision=rt.PREC_DF)
    traced = s0 == oracle.RAY_READY
    assert traced.sum() > 500
    assert (s_g[traced] == sref[traced]).mean() > 0.995
    g = good & traced & (s_g == sref)
    assert g.sum() > 0.9 * traced.sum()
    d = G.rel_state_diff(st_g[:, g], ref[:, g])
    # double-float rounding (2^-48, 32 x FP64's) can flip a step decision that
    # sits on a near-tie (accept/reject, a null-cone side): ~1 ray in 4000,
    # which then ends within the integration tolerance's reach (3e-7 seen)
    assert np.quantile(d, 0.999) < 1e-10, np.sort(d)[-5:]
    assert d.max() < 1e-6, np.sort(d)[-5:]
    assert ctr[2] == traced.sum()
    assert ctr[0] == na.sum()
    assert ctr[3] == (s_g == rt.RAY_ESCAPED).sum()


@pytest.mark.parametrize("which", ["config0", "misaligned"])
def test_df_binned_flux_matches_oracle(oracle, which):
    if which == "config0":
        kw, u = I.star_config0(), I.sample_uniforms(0, 4096)
    else:
        kw, u = I.stars_config1()[5], I.sample_uniforms(5, 4096)
    star, st_d, w_d, s_d, _ = G.gpu_sample(kw, u)
    G.gpu_trace(star, st_d, s_d, rtol=1e-10, precision=rt.PREC_DF)
    h_g = G.gpu_bin(star, st_d, w_d, s_d)[0]
    sv = oracle.star_vector(**kw)
    st_o, w_o, s_o = oracle.sample(sv, u)
    oracle.trace_forward(sv, oracle.trace_opts(rtol=1e-10), st_o, s_o)
    h_o = oracle.bin_rays(sv, st_o, w_o, s_o)[0]
    assert h_o.sum() > 0
    l1 = np.abs(h_g - h_o).sum() / np.abs(h_o).sum()
    assert l1 < 1e-8, l1


def test_df_agrees_with_fp64_gpu_path():
    kw = dict(I.stars_config1()[0], m_a_eV=1e-5)
    star, st_d, w_d, s_d, _ = G.gpu_sample(kw, I.sample_uniforms(7, 8192))
    st64, s64 = st_d.clone(), s_d.clone()
    G.gpu_trace(star, st64, s64, rtol=1e-10, tail=1)
    G.gpu_trace(star, st_d, s_d, rtol=1e-10, precision=rt.PREC_DF)
    a, sa, b, sb = G.to_np(st_d, s_d, st64, s64)
    same = sa == sb
    assert same.mean() > 0.995
    esc = same & (sb == rt.RAY_ESCAPED)
    d = G.rel_state_diff(a[:, esc], b[:, esc])
    assert np.median(d) < 1e-12 and np.percentile(d, 90) < 1e-10, np.percentile(d, [50, 90, 99])


def test_df_claim_order_and_batch_are_bitwise_neutral():
    kws = [I.stars_config1()[j] for j in (0, 2, 5)]
    n = 3000
    dev = G.dev()
    outs = []
    for kw, seed in zip(kws, (41, 42, 43)):
        star, st_d, w_d, s_d, _ = G.gpu_sample(kw, I.sample_uniforms(seed, n))
        a, sa = st_d.clone(), s_d.clone()
        G.gpu_trace(star, a, sa, rtol=1e-10, precision=rt.PREC_DF, claim_order=rt.CLAIM_INDEX)
        b, sb = st_d.clone(), s_d.clone()
        G.gpu_trace(star, b, sb, rtol=1e-10, precision=rt.PREC_DF, claim_order=rt.CLAIM_COST)
        assert torch.equal(a, b) and torch.equal(sa, sb)
        # cost order with the express warps, several rays per claim and a refill
        # threshold: the queues change hands between phases without losing a ray
        c, sc = st_d.clone(), s_d.clone()
        G.gpu_trace(star, c, sc, rtol=1e-10, precision=rt.PREC_DF, claim_order=rt.CLAIM_COST,
                    rays_per_claim=4, refill_min=8)
        assert torch.equal(a, c) and torch.equal(sa, sc)
        outs.append((st_d, s_d, a, sa))
    # the three stars in one batch: bitwise the per-star calls
    stars = [rt.Star(rt.make_params(**kw)) for kw in kws]
    batch = rt.Batch(stars, [n] * 3)
    st = torch.cat([o[0] for o in outs], dim=1).contiguous()
    s = torch.cat([o[1] for o in outs]).contiguous()
    ctr = torch.zeros(8, dtype=torch.int64, device=dev)
    rt.rt_trace_batch(batch, st, s, None, None, ctr,
                      rt.make_opts(rtol=1e-10, precision=rt.PREC_DF, claim_order=rt.CLAIM_COST))
    torch.cuda.synchronize()
    assert torch.equal(st, torch.cat([o[2] for o in outs], dim=1))
    assert torch.equal(s, torch.cat([o[3] for o in outs]))


def test_df_unsupported_calls_are_rejected_on_the_host():
    kw = I.star_config0()
    star = rt.Star(rt.make_params(**kw))
    dev = G.dev()
    img = torch.empty((4, 4), dtype=torch.float64, device=dev)
    ist = torch.empty((4, 4), dtype=torch.uint8, device=dev)
    with pytest.raises(rt.RtError) as e:
        rt.rt_trace_backward(star, 4, 4, 1.0, 1e4, 50.0, img, ist, None, None,
                             opts=rt.make_opts(precision=rt.PREC_DF))
    assert e.value.status == rt.RT_EUNSUPPORTED
    st = torch.zeros((8, 4), dtype=torch.float64, device=dev)
    s = torch.zeros(4, dtype=torch.uint8, device=dev)
    with pytest.raises(rt.RtError) as e:
        rt.rt_trace_forward(star, 4, st, s, None, None, None,
                            rt.make_opts(precision=rt.PREC_DF, lambda_max=1.0))
    assert e.value.status == rt.RT_EUNSUPPORTED
