"""The C ABI library: builds for sm_103a, loads, exports every symbol that
include/rt.h declares, and validates arguments on the host (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2309_08655_gb300 import build as B
from paper_2309_08655_gb300 import rt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return rt.lib()


def _declared_functions():
    txt = open(os.path.join(ROOT, "include", "rt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(L):
    names = _declared_functions()
    assert "rt_trace_forward" in names and len(names) >= 8
    for name in names:
        assert hasattr(L, name), name
    for name in rt.EXPORTED:
        assert name in names


def test_struct_layouts_match_header():
    # 10 doubles, 8 int32, 1 double / 5 doubles, 4 int32 (no padding surprises)
    assert ctypes.sizeof(rt.rt_star_params) == 10 * 8 + 8 * 4 + 8
    # + the timestamps pointer and the two work-claiming knobs after it
    assert ctypes.sizeof(rt.rt_trace_opts) == 5 * 8 + 6 * 4 + 8 + 2 * 4
    assert rt.rt_trace_opts.refill_min.offset == 72
    assert rt.rt_star_params.plasma_a.offset == 112
    assert rt.rt_star_params.rotation.offset == 108


def test_version_and_error_paths_without_gpu(L):
    assert rt.rt_version() >= 20000
    with pytest.raises(rt.RtError) as e:
        rt.Star(rt.make_params(M_sun=1.4, R_km=10.0, B0_G=1e14, P_s=1.0, m_a_eV=-1.0))
    assert e.value.status == rt.RT_EINVAL and "m_a_eV" in str(e.value)
    with pytest.raises(rt.RtError) as e:
        rt.Star(rt.make_params(M_sun=5.0, R_km=10.0, B0_G=1e14, P_s=1.0, m_a_eV=1e-5))
    assert e.value.status == rt.RT_EINVAL          # R below the Schwarzschild radius
    with pytest.raises(rt.RtError) as e:
        rt.Star(rt.make_params(M_sun=1.4, R_km=10.0, B0_G=1e14, P_s=1.0, m_a_eV=1e-5,
                               dispersion=7))
    assert e.value.status == rt.RT_EUNSUPPORTED
    with pytest.raises(rt.RtError) as e:
        rt.Star(rt.make_params(M_sun=1.4, R_km=10.0, B0_G=1e14, P_s=1.0, m_a_eV=1e-5,
                               rotation=2))
    assert e.value.status == rt.RT_EUNSUPPORTED and "rotation" in str(e.value)
    st = L.rt_trace_forward(None, 10, None, None, None, None, None, None, None)
    assert st == rt.RT_EINVAL
    st = L.rt_init_star(None, ctypes.byref(ctypes.c_void_p()))
    assert st == rt.RT_EINVAL and b"NULL" in L.rt_last_error()
    # the gradient: a NULL star is refused before anything touches a GPU
    nb = ctypes.c_int64(0)
    st = L.rt_flux_gradient(None, 16, None, None, 1.0, 4.0, ctypes.byref(rt.make_opts()), None,
                            None, None, None, -1, ctypes.byref(nb), None)
    assert st == rt.RT_EINVAL and b"NULL" in L.rt_last_error()


def test_objects_are_sm103a():
    # every object is compiled for sm_103a only (one -gencode)
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(B.library_path())


def test_noalloc_rejects_bad_params_and_host_arrays_without_launch(L):
    """rt_bin_spectrum_noalloc validates the star parameters as rt_init_star
    does, and every array as device memory of the current device, before
    anything is enqueued (a host pointer must come back as RT_EINVAL, never
    reach a kernel)."""
    import numpy as np
    vp = ctypes.c_void_p
    f = L.rt_bin_spectrum_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(rt.rt_star_params), ctypes.c_int64, vp, vp, vp, ctypes.c_int32,
                  ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double, vp, vp, vp,
                  vp, vp]
    host = np.zeros(8 * 16, dtype=np.float64)
    hp = host.ctypes.data
    bad = rt.make_params(M_sun=float("nan"), R_km=10.0, B0_G=1e14, P_s=1.0, m_a_eV=1e-5)
    assert f(ctypes.byref(bad), 16, hp, hp, hp, 4, 4, 4, 0.0, 9.0, hp, None, None, hp,
             None) == rt.RT_EINVAL
    assert b"non-finite" in L.rt_last_error()
    inside = rt.make_params(M_sun=5.0, R_km=10.0, B0_G=1e14, P_s=1.0, m_a_eV=1e-5)
    assert f(ctypes.byref(inside), 16, hp, hp, hp, 4, 4, 4, 0.0, 9.0, hp, None, None, hp,
             None) == rt.RT_EINVAL                  # R inside the Schwarzschild radius
    good = rt.make_params(M_sun=1.4, R_km=10.0, B0_G=1e14, P_s=1.0, m_a_eV=1e-5)
    assert f(ctypes.byref(good), 16, hp, hp, hp, 4, 4, 4, 0.0, 9.0, hp, None, None, hp,
             None) == rt.RT_EINVAL                  # host arrays
    assert b"d_state" in L.rt_last_error()
    assert f(ctypes.byref(good), 0, None, None, None, 4, 4, 4, 0.0, 9.0, hp, None, None, hp,
             None) == rt.RT_EINVAL                  # host output, no rays
    assert b"d_hist" in L.rt_last_error()


def _declared_arities():
    """Parameter counts of the functions include/rt.h declares (comments
    stripped; `(void)` counts as none)."""
    txt = open(os.path.join(ROOT, "include", "rt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    txt = re.sub(r"//[^\n]*", "", txt)
    out = {}
    for m in re.finditer(r"\b(rt_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", txt):
        args = " ".join(m.group(2).split())
        out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_argument_counts_match_header(L):
    """Every function the binding types takes as many arguments as rt.h
    declares: a signature change on one side only fails here, on the CPU."""
    ar = _declared_arities()
    assert ar.get("rt_flux_gradient") == 14 and ar.get("rt_trace_forward") == 9
    typed = 0
    for name, n in ar.items():
        fn = getattr(L, name)
        if fn.argtypes is None:
            continue
        typed += 1
        assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)
    assert typed >= 20
