"""rt_bin_spectrum_noalloc: the binning entry point for callers that cannot
allocate device memory (its accumulator is a static device array).

Checks through the C ABI that two calls in a row each reproduce the output of
rt_bin_spectrum on the same rays (the second call on different inputs, so a
leftover sum from the first call would show), and that an oversized histogram
is refused.  Named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2309_08655_gb300 import inputs as I  # noqa: E402
from paper_2309_08655_gb300 import rt  # noqa: E402

from . import gpu_util as G  # noqa: E402

NTH, NPH, NNU = 64, 32, 128


@pytest.fixture(scope="module")
def L():
    from paper_2309_08655_gb300.build import build
    build()
    assert torch.cuda.is_available()
    lib = rt.lib()
    f = lib.rt_bin_spectrum_noalloc
    f.restype = ctypes.c_int
    vp = ctypes.c_void_p
    f.argtypes = [ctypes.POINTER(rt.rt_star_params), ctypes.c_int64, vp, vp, vp, ctypes.c_int32,
                  ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double, vp, vp, vp,
                  vp, vp]
    return lib


def _noalloc(L, params, st, w, s):
    n = st.shape[1]
    dev = st.device
    hist = torch.full((NTH, NPH, NNU), -1.0, dtype=torch.float64, device=dev)
    sky = torch.empty((NTH, NPH), dtype=torch.float64, device=dev)
    spec = torch.empty(NNU, dtype=torch.float64, device=dev)
    oor = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    code = L.rt_bin_spectrum_noalloc(ctypes.byref(params), n, st.data_ptr(), w.data_ptr(),
                                     s.data_ptr(), NTH, NPH, NNU, 0.0, 9.0, hist.data_ptr(),
                                     sky.data_ptr(), spec.data_ptr(), oor.data_ptr(), stream)
    torch.cuda.synchronize()
    assert code == rt.RT_OK, L.rt_last_error()
    return hist.cpu().numpy(), sky.cpu().numpy(), spec.cpu().numpy(), float(oor.cpu()[0])


def test_noalloc_matches_rt_bin_spectrum_on_two_calls(L):
    kw = I.star_config0()
    params = rt.make_params(**kw)
    u = I.sample_uniforms(0, 2048)
    star, st, w, s, _ = G.gpu_sample(kw, u)
    G.gpu_trace(star, st, s, rtol=1e-10)
    # call 1: all rays; call 2: a different input (half of the escaped rays
    # marked captured), which must not see the first call's sums
    s2 = s.clone()
    s2[::2] = torch.where(s2[::2] == rt.RAY_ESCAPED, rt.RAY_CAPTURED, s2[::2])
    for status in (s, s2):
        ref = G.gpu_bin(star, st, w, status, NTH, NPH, NNU, 0.0, 9.0)
        got = _noalloc(L, params, st, w, status)
        h_ref, h = ref[0], got[0]
        assert h_ref.sum() > 0
        assert np.abs(h - h_ref).sum() <= 1e-12 * np.abs(h_ref).sum()
        assert np.allclose(got[1], ref[1], rtol=1e-12, atol=0)
        assert np.allclose(got[2], ref[2], rtol=1e-12, atol=0)
        assert abs(got[3] - ref[3]) <= 1e-12 * max(abs(ref[3]), 1e-300)


def test_noalloc_refuses_oversized_histograms(L):
    params = rt.make_params(**I.star_config0())
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    code = L.rt_bin_spectrum_noalloc(ctypes.byref(params), 0, x.data_ptr(), x.data_ptr(),
                                     x.data_ptr(), 128, 64, 128, 0.0, 9.0, x.data_ptr(), None,
                                     None, x.data_ptr(), None)
    assert code == rt.RT_EINVAL
    assert b"RT_BIN_NOALLOC_MAX_ENTRIES" in L.rt_last_error()


def test_noalloc_refuses_host_arrays_and_bad_params(L):
    """Host memory in place of a device array, or parameters that
    rt_init_star would refuse, come back as RT_EINVAL before any launch; a
    correct call right after still matches rt_bin_spectrum."""
    params = rt.make_params(**I.star_config0())
    host = np.zeros(8 * 64, dtype=np.float64)
    hp = host.ctypes.data
    d = torch.zeros(8 * 64, dtype=torch.float64, device="cuda")
    s = torch.zeros(64, dtype=torch.uint8, device="cuda")
    for args in [(hp, d.data_ptr(), s.data_ptr()), (d.data_ptr(), hp, s.data_ptr()),
                 (d.data_ptr(), d.data_ptr(), host.ctypes.data)]:
        code = L.rt_bin_spectrum_noalloc(ctypes.byref(params), 64, *args, 4, 4, 4, 0.0, 9.0,
                                         d.data_ptr(), None, None, d.data_ptr(), None)
        assert code == rt.RT_EINVAL, L.rt_last_error()
    code = L.rt_bin_spectrum_noalloc(ctypes.byref(params), 64, d.data_ptr(), d.data_ptr(),
                                     s.data_ptr(), 4, 4, 4, 0.0, 9.0, hp, None, None,
                                     d.data_ptr(), None)
    assert code == rt.RT_EINVAL and b"d_hist" in L.rt_last_error()
    bad = rt.make_params(**dict(I.star_config0(), v0_kms=4e5))      # faster than light
    code = L.rt_bin_spectrum_noalloc(ctypes.byref(bad), 64, d.data_ptr(), d.data_ptr(),
                                     s.data_ptr(), 4, 4, 4, 0.0, 9.0, d.data_ptr(), None, None,
                                     d.data_ptr(), None)
    assert code == rt.RT_EINVAL
    torch.cuda.synchronize()
    test_noalloc_matches_rt_bin_spectrum_on_two_calls(L)
