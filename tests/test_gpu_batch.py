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
