"""Pins of the oracle's line-flux functional (oracle.line_flux), the CPU
reference for the adjoint gradient's functional:

* the von Mises-Fisher kernel has unit mass on the sphere for any width: rays
  spread uniformly over the sky (a Fibonacci lattice) with weights summing to
  one give F = 1 / (4 pi);
* kappa -> 0: F -> (sum of escaped weights) / (4 pi);
* a ray travelling exactly toward the observer contributes w C, C = kappa /
  (2 pi (1 - exp(-2 kappa)));
* the direction is that of the static orthonormal frame: a radial covariant
  momentum keeps its direction under the frame change (only its length
  scales by sqrt(A)), a tangential one is unchanged, and rays that did not
  escape contribute nothing.
"""
import math

import numpy as np
import pytest


def _flat(oracle):
    return oracle.star_vector(M_sun=0.0, R_km=10.0, m_a_eV=1e-5)


def _rays(dirs, r_R=1000.0, R_km=10.0, ma=1e-5):
    st = np.zeros((8, dirs.shape[1]))
    st[:3] = dirs * r_R * R_km
    st[3:6] = dirs * ma
    return st


def _fibonacci(n):
    i = np.arange(n) + 0.5
    z = 1 - 2 * i / n
    ph = math.pi * (1 + 5 ** 0.5) * i
    s = np.sqrt(1 - z * z)
    return np.stack([s * np.cos(ph), s * np.sin(ph), z])


@pytest.mark.parametrize("kappa", [0.1, 4.0, (64 / math.pi) ** 2])
def test_kernel_has_unit_mass(oracle, kappa):
    n = 200000
    d = _fibonacci(n)
    st = _rays(d)
    w = np.full(n, 1.0 / n)
    s = np.full(n, oracle.RAY_ESCAPED, dtype=np.uint8)
    for incl in (0.3, 1.1, 2.9):
        F = oracle.line_flux(_flat(oracle), st, w, s, incl, kappa)
        assert abs(F * 4 * math.pi - 1) < 1e-3, (kappa, incl, F)


def test_small_kappa_limit_and_status_mask(oracle):
    rng = np.random.default_rng(3)
    d = rng.standard_normal((3, 500))
    d /= np.linalg.norm(d, axis=0)
    st = _rays(d)
    w = rng.random(500)
    s = np.where(rng.random(500) < 0.7, oracle.RAY_ESCAPED, oracle.RAY_CAPTURED).astype(np.uint8)
    F = oracle.line_flux(_flat(oracle), st, w, s, 0.8, 1e-9)
    assert abs(F / (w[s == oracle.RAY_ESCAPED].sum() / (4 * math.pi)) - 1) < 1e-8


def test_ray_toward_the_observer_and_the_orthonormal_direction(oracle):
    kappa, incl = 37.0, 1.1
    o = np.array([math.sin(incl), 0.0, math.cos(incl)])
    C = kappa / (2 * math.pi * (1 - math.exp(-2 * kappa)))
    sv = oracle.star_vector(M_sun=1.4, R_km=10.0, m_a_eV=1e-5)
    s1 = np.array([oracle.RAY_ESCAPED], dtype=np.uint8)
    # at r = 3 R (A = 1 - r_s / 3R): radial momentum along o keeps its direction
    st = np.zeros((8, 1))
    st[:3, 0] = o * 30.0
    st[3:6, 0] = o * 2e-5
    assert abs(oracle.line_flux(sv, st, [2.5], s1, incl, kappa) / (2.5 * C) - 1) < 1e-14
    # tangential momentum along o at a position perpendicular to it: unchanged
    e = np.array([math.cos(incl), 0.0, -math.sin(incl)])
    st[:3, 0] = e * 30.0
    assert abs(oracle.line_flux(sv, st, [2.5], s1, incl, kappa) / (2.5 * C) - 1) < 1e-14
    # a mixed momentum: the radial part is scaled by sqrt(A) before normalising
    rs = oracle.star_constants(sv)["rs_over_R"]
    A = 1 - rs / 3.0
    k = 0.6 * o + 0.8 * e
    st[3:6, 0] = k * 1e-5
    ko = 0.6 * o + 0.8 * math.sqrt(A) * e
    mu = ko @ o / np.linalg.norm(ko)
    expect = 2.5 * C * math.exp(kappa * (mu - 1))
    assert abs(oracle.line_flux(sv, st, [2.5], s1, incl, kappa) / expect - 1) < 1e-12
