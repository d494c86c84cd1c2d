"""Batched launch machinery: CUDA-graph replay of a sample -> trace -> bin step,
the launch-shape autotuner, and per-instance completion timestamps.

Each ray is integrated independently by one thread, so neither replaying a
captured graph nor changing the launch shape may change any result: both
are compared bitwise with the direct calls."""
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


def _setup(prec=rt.PREC_FP64, n_per=1024, rotation=rt.ROTATION_SNAPSHOT):
    kws = I.stars_config1()[:6]          # masses 4e-4 .. 1.4e-6 eV, some surfaces empty
    for k in kws:
        k.update(rotation=rotation)
    counts = [n_per, 3 * n_per // 2, n_per // 2, n_per, 7, n_per]   # uneven, one tiny
    stars = [rt.Star(rt.make_params(**k)) for k in kws]
    b = rt.Batch(stars, counts)
    N = b.N
    u = torch.from_numpy(np.ascontiguousarray(np.concatenate(
        [I.sample_uniforms(50 + j, c) for j, c in enumerate(counts)], axis=1))).to(G.dev())
    bufs = dict(
        st=torch.empty((8, N), dtype=torch.float64, device=G.dev()),
        w=torch.empty(N, dtype=torch.float64, device=G.dev()),
        s=torch.empty(N, dtype=torch.uint8, device=G.dev()),
        hist=torch.empty((len(stars),) + NB, dtype=torch.float64, device=G.dev()),
        oor=torch.empty(len(stars), dtype=torch.float64, device=G.dev()),
        ctr=torch.zeros(8, dtype=torch.int64, device=G.dev()))
    rtol = 1e-10 if prec == rt.PREC_FP64 else 1e-8
    return b, stars, u, bufs, rtol


def _direct(b, u, B, opts):
    B["ctr"].zero_()
    rt.rt_sample_batch(b, u, B["st"], B["w"], B["s"])
    rt.rt_trace_batch(b, B["st"], B["s"], None, None, B["ctr"], opts)
    rt.rt_bin_batch(b, B["st"], B["w"], B["s"], *NB, 0.0, 9.0, B["hist"], B["oor"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().copy() for k, v in B.items()}


@pytest.mark.parametrize("case", ["fp64", "mixed", "fp64_cost_order", "rotating"])
def test_graph_replay_equals_direct_calls(case):
    # cost order: the express lane's selection and ranking are captured too;
    # rotating: a batch of rigidly rotating magnetospheres (its own kernel)
    prec = rt.PREC_MIXED if case == "mixed" else rt.PREC_FP64
    rot = rt.ROTATION_RIGID if case == "rotating" else rt.ROTATION_SNAPSHOT
    b, stars, u, B, rtol = _setup(prec, rotation=rot)
    opts = rt.make_opts(rtol=rtol, precision=prec,
                        claim_order=rt.CLAIM_COST if case == "fp64_cost_order" else rt.CLAIM_INDEX)
    ref = _direct(b, u, B, opts)
    for v in B.values():
        v.fill_(0)
    g = rt.Graph(b, u, B["st"], B["w"], B["s"], B["ctr"], opts, *NB, 0.0, 9.0, B["hist"],
                 B["oor"])
    for _ in range(2):                      # replays are repeatable
        g.launch()
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in B.items()}
        for k in ref:
            np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    g.close()


def test_autotune_choice_is_valid_and_result_invariant():
    b, stars, u, B, rtol = _setup()
    opts = rt.make_opts(rtol=rtol)
    ref = _direct(b, u, B, opts)
    rt.rt_sample_batch(b, u, B["st"], B["w"], B["s"])
    tune = rt.rt_batch_autotune(b, B["st"], B["s"], opts, rays_per_star=128)
    assert tune["block"] in (32, 64, 128)
    assert tune["blocks_per_sm"] >= 1
    assert tune["refill_min"] in (1, 2, 4, 8, 16)
    assert tune["rays_per_claim"] in (1, 2, 4, 8)
    assert len(tune["candidates_ms"]) >= 3 + 4 + 3       # shapes, thresholds, claim sizes
    assert tune["ms"] == pytest.approx(min(tune["candidates_ms"]))
    got = _direct(b, u, B, opts)               # opts fields 0: the tuned launch
    for k in ("st", "s", "hist", "oor", "ctr"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


@pytest.mark.parametrize("refill, claim", [(1, 1), (8, 1), (1, 4), (16, 8), (32, 64)])
def test_refill_threshold_and_claim_size_do_not_change_results(refill, claim):
    """One lane per ray (tail = 1): every ray's integration is independent of
    the lane and the moment it is claimed, so any refill threshold and claim
    size give bitwise the same end states (FP64 and mixed precision)."""
    for prec in (rt.PREC_FP64, rt.PREC_MIXED):
        b, stars, u, B, rtol = _setup(prec)
        ref = _direct(b, u, B, rt.make_opts(rtol=rtol, precision=prec, tail=1))
        got = _direct(b, u, B, rt.make_opts(rtol=rtol, precision=prec, tail=1,
                                            refill_min=refill, rays_per_claim=claim))
        for k in ("st", "s", "hist", "oor", "ctr"):
            np.testing.assert_array_equal(got[k], ref[k], err_msg=(prec, k))


def test_autotune_with_images_tunes_the_joint_launch():
    """With backward images set, the autotuner times rays and (coarse copies
    of) pixels in one launch and stores the choice for that launch; results of
    the tuned launch equal those of the default one."""
    b, stars, u, B, rtol = _setup(rt.PREC_MIXED)
    kw = dict(M_sun=1.4, R_km=10.0, B0_G=1e14, P_s=1.0, theta_m=0.5, psi=0.4, m_a_eV=1e-5)
    istars = [rt.Star(rt.make_params(**kw)), rt.Star(rt.make_params(**dict(kw, theta_m=0.2)))]
    descs = [(40, 30, 1.0, 1e4, 2.0, 0.0), (17, 23, 0.4, 1e4, 2.0, 0.0)]
    P = sum(d[0] * d[1] for d in descs)
    img = torch.zeros(P, dtype=torch.float64, device=G.dev())
    ist = torch.zeros(P, dtype=torch.uint8, device=G.dev())
    rt.rt_batch_set_images(b, istars, descs, img, ist)
    opts = rt.make_opts(rtol=rtol, precision=rt.PREC_MIXED)
    ref = _direct(b, u, B, opts)
    ref_img = img.cpu().numpy().copy()
    rt.rt_sample_batch(b, u, B["st"], B["w"], B["s"])
    tune = rt.rt_batch_autotune(b, B["st"], B["s"], opts, rays_per_star=64)
    assert tune["block"] in (64, 128, 256) and tune["blocks_per_sm"] >= 1
    assert tune["refill_min"] in (1, 2, 4, 8, 16) and tune["rays_per_claim"] in (1, 2, 4, 8)
    img.zero_()
    got = _direct(b, u, B, opts)
    for k in ("st", "s", "hist", "oor", "ctr"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    np.testing.assert_array_equal(img.cpu().numpy(), ref_img)
    assert ref_img.sum() > 0


def test_instance_timestamps():
    b, stars, u, B, rtol = _setup()
    ts = torch.zeros(1 + len(stars), dtype=torch.int64, device=G.dev())
    opts = rt.make_opts(rtol=rtol, timestamps=ts)
    rt.rt_timestamps_reset(ts, len(stars))
    rt.rt_sample_batch(b, u, B["st"], B["w"], B["s"])
    traced = [bool((B["s"][o:o2] == 0).any()) for o, o2 in zip(
        np.cumsum([0] + list(b.counts))[:-1], np.cumsum(b.counts))]
    rt.rt_trace_batch(b, B["st"], B["s"], None, None, None, opts)
    torch.cuda.synchronize()
    t = ts.cpu().numpy().view(np.uint64)
    assert t[0] < np.uint64(2 ** 63)
    for k, tr in enumerate(traced):
        if tr:
            assert t[1 + k] >= t[0]
            assert (t[1 + k] - t[0]) < np.uint64(60 * 10 ** 9)
        else:
            assert t[1 + k] == 0
