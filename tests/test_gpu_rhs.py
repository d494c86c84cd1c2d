"""Hamilton's equations on the GPU (the analytic right-hand side the FP64
integrators step with, exported by rt_hamilton_rhs) against the oracle's
derivatives of the plain Hamiltonian by dual numbers, point by point.

Points: just above the stellar surface, on both flanks of the
Goldreich-Julian null cone (where the density's gradient jumps; each side
differentiates its own smooth continuation), on the conversion surface itself
(samples of the resonance), and far out; every plasma model and both
dispersions.  Both sides evaluate the same function in FP64 in different
ways, so they agree to rounding: 1e-12 relative per block (dx/dl, dk/dl),
H to 1e-12 of the size of its largest term.
"""
import math
import zlib

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


def _unit(v):
    return v / np.linalg.norm(v, axis=0)


def _points(kw, rng, n=512):
    """State columns (x km, k eV, delta, psi): shells near the surface and far
    out, random momenta around the local photon energy."""
    R, ma = kw["R_km"], kw["m_a_eV"]
    r = np.concatenate([1.0 + 0.05 * rng.random(n // 4), 1.5 + 30 * rng.random(n // 2),
                        200.0 + 800.0 * rng.random(n - n // 4 - n // 2)])
    x = _unit(rng.standard_normal((3, n))) * r * R
    k = rng.standard_normal((3, n)) * (0.3 + rng.random(n)) * ma
    st = np.zeros((8, n))
    st[:3], st[3:6] = x, k
    st[6] = 1e-7 * rng.random(n)
    st[7] = 2 * math.pi * rng.random(n) if kw.get("phase_mode", 0) else kw.get("psi", 0.0)
    return st


def _null_cone_points(kw, rng, n=256):
    """Points within 1e-7 .. 1e-3 rad of the cone 3 cos(th) (m.n) = cos(th_m),
    on both sides."""
    R, ma = kw["R_km"], kw["m_a_eV"]
    psi = kw.get("psi", 0.0)
    tm = kw["theta_m"]
    m = np.array([math.sin(tm) * math.cos(psi), math.sin(tm) * math.sin(psi), math.cos(tm)])
    out = []
    while len(out) < n:
        nv = _unit(rng.standard_normal(3))
        F = 3 * nv[2] * (m @ nv) - m[2]
        # walk along the polar angle to the cone by bisection on F
        th0, ph = math.acos(nv[2]), math.atan2(nv[1], nv[0])

        def Fat(th):
            v = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
            return 3 * v[2] * (m @ v) - m[2], v

        lo, hi = 0.0, th0
        if Fat(lo)[0] * F > 0:
            lo, hi = th0, math.pi
            if Fat(hi)[0] * F > 0:
                continue
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if Fat(mid)[0] * Fat(lo)[0] > 0:
                lo = mid
            else:
                hi = mid
        off = 10 ** rng.uniform(-7, -3) * rng.choice([-1, 1])
        _, v = Fat(0.5 * (lo + hi) + off)
        out.append(v * (1.0 + 20 * rng.random()) * R)
    x = np.array(out).T
    k = rng.standard_normal((3, n)) * ma
    st = np.zeros((8, n))
    st[:3], st[3:6] = x, k
    st[7] = psi
    return st


def _compare(oracle, kw, st):
    sv = oracle.star_vector(**kw)
    H_o, d_o = oracle.hamiltonian(sv, st, with_rhs=True)
    star = rt.Star(rt.make_params(**kw))
    n = st.shape[1]
    sd = torch.from_numpy(np.ascontiguousarray(st)).to(G.dev())
    H = torch.empty(n, dtype=torch.float64, device=G.dev())
    d = torch.empty((6, n), dtype=torch.float64, device=G.dev())
    rt.rt_hamilton_rhs(star, n, sd, H, d)
    torch.cuda.synchronize()
    H_g, d_g = H.cpu().numpy(), d.cpu().numpy()
    ex = np.linalg.norm(d_g[:3] - d_o[:3], axis=0) / np.linalg.norm(d_o[:3], axis=0)
    ek = np.linalg.norm(d_g[3:] - d_o[3:], axis=0) / np.linalg.norm(d_o[3:], axis=0)
    # H = -W^2/A + |k|^2 + plasma terms: the size of its largest term bounds
    # the rounding of the sum (the plasma term reaches ~1e4 m_a^2 at the surface)
    W2 = (1.0 + st[6]) ** 2
    eH = np.abs(H_g - H_o) / (W2 + np.sum((st[3:6] / kw["m_a_eV"]) ** 2, axis=0) + np.abs(H_o))
    return ex, ek, eH


def _stars():
    c0 = I.star_config0()
    c1 = dict(I.stars_config1()[0], m_a_eV=1e-5)
    return {
        "gj_aligned_aniso": c0,
        "gj_misaligned_aniso": c1,
        "gj_misaligned_iso": dict(c1, dispersion=1),
        "twisted_aniso": dict(I.stars_config1()[9], plasma=rt.PLASMA_TWISTED, plasma_a=4.0),
        "radial_iso": dict(c0, plasma=rt.PLASMA_RADIAL, plasma_a=8.0, dispersion=1, M_sun=0.0),
        "homog_aniso": dict(c0, plasma=rt.PLASMA_HOMOG, plasma_a=0.5, theta_m=0.4),
        "linear_z_iso": dict(c0, plasma=rt.PLASMA_LINEAR_Z, plasma_a=0.01, dispersion=1,
                             M_sun=0.0),
        "flat_propagation": dict(c1, prop_metric=rt.METRIC_FLAT),
    }


@pytest.mark.parametrize("name", list(_stars()))
def test_rhs_matches_oracle_dual_numbers(oracle, name):
    kw = _stars()[name]
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    ex, ek, eH = _compare(oracle, kw, _points(kw, rng))
    assert ex.max() < 1e-12 and ek.max() < 1e-12, (ex.max(), ek.max())
    assert eH.max() < 1e-12, eH.max()


@pytest.mark.parametrize("name", ["gj_aligned_aniso", "gj_misaligned_aniso", "gj_misaligned_iso"])
def test_rhs_on_both_flanks_of_the_null_cone(oracle, name):
    kw = _stars()[name]
    rng = np.random.default_rng(7)
    ex, ek, eH = _compare(oracle, kw, _null_cone_points(kw, rng))
    assert ex.max() < 1e-12 and ek.max() < 1e-12, (ex.max(), ek.max())
    assert eH.max() < 1e-12


@pytest.mark.parametrize("name", ["gj_aligned_aniso", "gj_misaligned_aniso", "twisted_aniso"])
def test_rhs_on_the_conversion_surface(oracle, name):
    kw = _stars()[name]
    sv = oracle.star_vector(**kw)
    st, w, s = oracle.sample(sv, I.sample_uniforms(90, 1024))
    ok = s == oracle.RAY_READY
    assert ok.sum() > 200
    ex, ek, eH = _compare(oracle, kw, st[:, ok])
    assert ex.max() < 1e-12 and ek.max() < 1e-12, (ex.max(), ek.max())
    assert eH.max() < 1e-12          # on shell: H is a cancellation of O(1) terms
