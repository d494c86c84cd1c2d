"""One workload split into contiguous ray ranges (the multi-GPU partition),
run here shard after shard on one GPU through the C ABI: every shard samples
its range with the whole workload's weight normalisation, traces it, and bins
it into int64 fixed-point sums; the sums are reduced exactly (MAX of the
largest weight, then SUM) and finalised.  The result must be bitwise that of
one sampling, tracing and binning call over all rays.  Tracing runs one lane
per ray (tail = 1), where each ray's end point does not depend on which other
rays share its launch."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2309_08655_gb300 import inputs as I  # noqa: E402
from paper_2309_08655_gb300 import rt  # noqa: E402
from paper_2309_08655_gb300 import shard  # noqa: E402

from . import gpu_util as G  # noqa: E402

NB = (64, 32, 128)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2309_08655_gb300.build import build
    build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _whole(kw, u, opts):
    star, st, w, s, _ = G.gpu_sample(kw, u)
    G.gpu_trace(star, st, s, **opts)
    h, sky, spec, oor = G.gpu_bin(star, st, w, s, *NB)
    return star, st, w, s, h, sky, spec, oor


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_spectrum_equals_one_call_bitwise(world):
    kw = I.star_config0()
    n = 4096 + 37                                   # shards of unequal size
    u = I.sample_uniforms(11, n)
    opts = dict(rtol=1e-10, tail=1)
    star, st1, w1, s1, h1, sky1, spec1, oor1 = _whole(kw, u, opts)
    dev = G.dev()
    E = rt.bin_acc_entries(*NB)
    accs, parts = [], []
    for r in range(world):
        f, c = shard.ray_range(n, world, r)
        ud = torch.from_numpy(np.ascontiguousarray(u[:, f:f + c])).to(dev)
        st = torch.empty((8, c), dtype=torch.float64, device=dev)
        w = torch.empty(c, dtype=torch.float64, device=dev)
        s = torch.empty(c, dtype=torch.uint8, device=dev)
        rt.rt_sample_conversion_surface_part(star, c, n, ud, st, w, s)
        G.gpu_trace(star, st, s, **opts)
        acc = torch.full((E,), -7, dtype=torch.int64, device=dev)   # cleared by the call
        rt.rt_bin_part_max(c, w, s, *NB, acc)
        accs.append(acc)
        parts.append((f, c, st, w, s))
    torch.cuda.synchronize()
    # the same weights and end points as the single call, bit for bit
    for f, c, st, w, s in parts:
        assert torch.equal(w, w1[f:f + c])
        assert torch.equal(s, s1[f:f + c])
        assert torch.equal(st, st1[:, f:f + c])
    wmax = torch.stack([a[0] for a in accs]).max()            # the MAX all-reduce
    for a, (f, c, st, w, s) in zip(accs, parts):
        a[0] = wmax
        rt.rt_bin_part_accumulate(star, c, n, st, w, s, *NB, 0.0, 9.0, a)
    tot = torch.stack(accs).sum(0)                            # the SUM all-reduce
    tot[0] = wmax
    hist = torch.empty(NB, dtype=torch.float64, device=dev)
    sky = torch.empty(NB[:2], dtype=torch.float64, device=dev)
    spec = torch.empty(NB[2], dtype=torch.float64, device=dev)
    oor = torch.empty(1, dtype=torch.float64, device=dev)
    rt.rt_bin_part_finalize(*NB, n, tot, hist, sky, spec, oor)
    torch.cuda.synchronize()
    assert h1.sum() > 0
    assert np.array_equal(hist.cpu().numpy(), h1)
    assert np.array_equal(sky.cpu().numpy(), sky1)
    assert np.array_equal(spec.cpu().numpy(), spec1)
    assert float(oor.cpu()[0]) == oor1


def test_one_shard_is_rt_bin_spectrum_bitwise():
    kw = I.stars_config1()[5]                    # m_a = 1.4e-6 eV: a non-empty surface
    u = I.sample_uniforms(12, 3000)
    star, st, w, s, h1, sky1, spec1, oor1 = _whole(kw, u, dict(rtol=1e-10))
    dev = G.dev()
    acc = torch.empty(rt.bin_acc_entries(*NB), dtype=torch.int64, device=dev)
    rt.rt_bin_part_max(3000, w, s, *NB, acc)
    rt.rt_bin_part_accumulate(star, 3000, 3000, st, w, s, *NB, 0.0, 9.0, acc)
    hist = torch.empty(NB, dtype=torch.float64, device=dev)
    oor = torch.empty(1, dtype=torch.float64, device=dev)
    rt.rt_bin_part_finalize(*NB, 3000, acc, hist, None, None, oor)
    torch.cuda.synchronize()
    assert h1.sum() > 0
    assert np.array_equal(hist.cpu().numpy(), h1)
    assert float(oor.cpu()[0]) == oor1


def test_batch_shards_with_norm_match_the_whole_batch():
    """Two stars, each split over two batches (ranks) with rt_batch_set_norm,
    binned with shard.bin_sharded's phases and the sums added: bitwise the
    per-star histograms of one batch holding all rays."""
    kws = [I.stars_config1()[j] for j in (0, 2)]
    nper = 1500
    dev = G.dev()
    stars = [rt.Star(rt.make_params(**kw)) for kw in kws]
    opts = rt.make_opts(rtol=1e-10, tail=1)

    def run(first, count, norm):
        b = rt.Batch(stars, [count] * 2)
        if norm is not None:
            rt.rt_batch_set_norm(b, [norm] * 2)
        u = np.concatenate([I.sample_uniforms(20 + j, count, first) for j in range(2)], axis=1)
        ud = torch.from_numpy(np.ascontiguousarray(u)).to(dev)
        N = 2 * count
        st = torch.empty((8, N), dtype=torch.float64, device=dev)
        w = torch.empty(N, dtype=torch.float64, device=dev)
        s = torch.empty(N, dtype=torch.uint8, device=dev)
        rt.rt_sample_batch(b, ud, st, w, s)
        rt.rt_trace_batch(b, st, s, None, None, None, opts)
        return b, st, w, s

    b, st, w, s = run(0, nper, None)
    href = torch.empty((2,) + NB, dtype=torch.float64, device=dev)
    oref = torch.empty(2, dtype=torch.float64, device=dev)
    rt.rt_bin_batch(b, st, w, s, *NB, 0.0, 9.0, href, oref)
    E = rt.bin_acc_entries(*NB)
    half = [shard.ray_range(nper, 2, r) for r in range(2)]
    runs = [run(f, c, nper) for f, c in half]
    accs = []
    for (f, c), (bb, st2, w2, s2) in zip(half, runs):
        acc = torch.empty((2, E), dtype=torch.int64, device=dev)
        for j in range(2):
            rt.rt_bin_part_max(c, w2[j * c:], s2[j * c:], *NB, acc[j])
        accs.append(acc)
    wmax = torch.maximum(accs[0][:, 0], accs[1][:, 0])
    for (f, c), (bb, st2, w2, s2), acc in zip(half, runs, accs):
        acc[:, 0] = wmax
        for j in range(2):
            rt.rt_bin_part_accumulate(stars[j], c, nper, st2[:, j * c:], w2[j * c:], s2[j * c:],
                                      *NB, 0.0, 9.0, acc[j], ld=2 * c)
    tot = accs[0] + accs[1]
    tot[:, 0] = wmax
    hist = torch.empty((2,) + NB, dtype=torch.float64, device=dev)
    oor = torch.empty(2, dtype=torch.float64, device=dev)
    for j in range(2):
        rt.rt_bin_part_finalize(*NB, nper, tot[j], hist[j], None, None, oor[j:j + 1])
    torch.cuda.synchronize()
    assert float(href.sum()) > 0
    assert torch.equal(hist, href)
    assert torch.equal(oor, oref)


def test_part_argument_errors():
    kw = I.star_config0()
    star = rt.Star(rt.make_params(**kw))
    dev = G.dev()
    x = torch.zeros(64, dtype=torch.float64, device=dev)
    s = torch.zeros(64, dtype=torch.uint8, device=dev)
    with pytest.raises(rt.RtError) as e:
        rt.rt_sample_conversion_surface_part(star, 8, 4, x, x, x, s)     # n_norm < n
    assert e.value.status == rt.RT_EINVAL
    acc = torch.zeros(rt.bin_acc_entries(*NB), dtype=torch.int64, device=dev)
    with pytest.raises(rt.RtError) as e:
        rt.rt_bin_part_accumulate(star, 8, 4, x, x, s, *NB, 0.0, 9.0, acc)   # n_total < n
    assert e.value.status == rt.RT_EINVAL
    host = np.zeros(rt.bin_acc_entries(*NB), dtype=np.int64)
    with pytest.raises(rt.RtError) as e:
        rt.rt_bin_part_max(8, x, s, *NB, host.ctypes.data)             # host memory
    assert e.value.status == rt.RT_EINVAL
    b = rt.Batch([star], [16])
    with pytest.raises(rt.RtError) as e:
        rt.rt_batch_set_norm(b, [8])
    assert e.value.status == rt.RT_EINVAL
