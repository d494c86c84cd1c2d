"""Pins of the oracle's anisotropic forward weight (Sec. 4.2, Eq. PowerCurved
with the ansatz Eq. CPAnisoCurved and the angle Eq. AngleDefAniso) against
things that do not use the oracle's collapsed form:

* The shape factor E^4 sin^2(th) / D, D = cos^2(th) w_p^2 (w_p^2 - 2 E^2) +
  E^4, of the strong-field probability belongs to the Langmuir-O mode (Eq.
  LOEnergy).  That mode's energy is the larger root of the dispersion
  polynomial F(E^2) = E^4 - (w_p^2 + k^2) E^2 + k^2 w_p^2 cos^2(th), and
  eliminating k^2 with F = 0 gives D = F'(E^2) (E^2 - w_p^2 cos^2(th)).  So at
  every sample the oracle's shape factor times (2 E^2 - w_p^2 - k^2)
  (E^2 - w_p^2 cos^2(th)) must equal E^4 sin^2(th), and F must vanish: a sign
  slip in D or sin and cos exchanged fails.
* The uncollapsed integrand.  Each sample's weight must equal the paper's
  integrand sqrt|h_k| cos(th_n) v_a omega P_agamma f_a, evaluated literally,
  divided by the sampling density: sqrt|h_k| as printed (with its A^{1/2})
  from the partial derivatives of the conversion radius r_k(theta, phi),
  taken here by finite differences of the oracle's root at neighbouring
  directions (the leaf of fixed khat and omega_inf); cos(th_n), v_a = |k| / E,
  omega = E and P_agamma with the proper-frame gradient dE of E_gamma - E_a
  on the leaf.  The divergence of P_agamma cancels against cos(th_n) here
  term by term, as the text after Eq. AngleDefAniso states.
"""
import math

import numpy as np
import pytest

from paper_2309_08655_gb300 import inputs as I

HBARC_EV_KM = 1.973269804e-10
HBAR_EV_S = 6.582119569e-16
EV_J = 1.602176634e-19


def _stars():
    c1 = I.stars_config1()
    tw = dict(c1[9], plasma=5, plasma_a=4.0)          # twisted magnetosphere, m_a ~ 1e-4 eV
    return {"config0": I.star_config0(), "misaligned_1": dict(c1[0], m_a_eV=1e-5),
            "misaligned_5": c1[5],
            "twisted": tw}


@pytest.mark.parametrize("name", ["config0", "misaligned_1", "misaligned_5", "twisted"])
def test_shape_factor_is_the_lo_mode_derivative(oracle, name):
    sv = oracle.star_vector(**_stars()[name])
    p = oracle.sample_parts(sv, I.sample_uniforms(71, 512))
    ok = p["ok"] == 1
    assert ok.sum() > 100
    E2, k2, w2, c2 = p["E"][ok] ** 2, p["K2"][ok], p["wp2"][ok], p["cos2"][ok]
    F = E2 * E2 - (w2 + k2) * E2 + k2 * w2 * c2
    assert np.abs(F / (E2 * E2)).max() < 1e-12
    lhs = p["shape"][ok] * (2 * E2 - w2 - k2) * (E2 - w2 * c2)
    rhs = E2 * E2 * (1 - c2)
    assert np.abs(lhs / rhs - 1).max() < 1e-10
    # the Langmuir-O root is the larger one: F'(E^2) > 0
    assert np.all(2 * E2 - w2 - k2 > 0)


def _root_radius(oracle, sv, u):
    p = oracle.sample_parts(sv, u)
    return p["r"], p["ok"] == 1


@pytest.mark.parametrize("name", ["config0", "misaligned_5", "twisted"])
def test_weight_equals_the_literal_power_integrand(oracle, name):
    kw = _stars()[name]
    sv = oracle.star_vector(**kw)
    n = 48
    u = I.sample_uniforms(72, n)
    p = oracle.sample_parts(sv, u)
    ok = p["ok"] == 1
    # partial derivatives of r_k(theta, phi) on the leaf (khat, omega_inf
    # fixed): fourth-order central differences of the oracle's root in the
    # direction uniforms (cos theta = 1 - 2 u0, phi = 2 pi u1)
    # (two step sizes: where they disagree the stencil straddles the kink of
    # the Goldreich-Julian density on its null cone and the sample is skipped)
    drdu, fd_err = [], np.zeros(n)
    for row in (0, 1):
        est = []
        for d in (1e-4, 2.5e-5):
            rs = []
            for k in (-2, -1, 1, 2):
                uu = u.copy()
                uu[row] = u[row] + k * d
                r, okk = _root_radius(oracle, sv, uu)
                ok &= okk
                rs.append(r)
            est.append((rs[0] - 8 * rs[1] + 8 * rs[2] - rs[3]) / (12 * d))
        drdu.append(est[0])
        fd_err = np.maximum(fd_err, np.abs(est[0] - est[1]) / np.maximum(np.abs(est[0]), p["r"]))
    smooth = fd_err < 1e-9
    assert (ok & smooth).sum() >= 0.85 * ok.sum() and ok.sum() > 20
    ok &= smooth
    r = p["r"]
    nz = p["n2"]
    sin_t = np.sqrt(1 - nz * nz)
    r_th = drdu[0] * sin_t / 2.0           # du0 / dtheta = sin(theta) / 2
    r_ph = drdu[1] / (2 * math.pi)         # du1 / dphi = 1 / (2 pi)
    A = p["A"]
    # Eq. PowerCurved's surface measure, sqrt|h_k| as printed [R^2]
    hk = np.sqrt(A) * r * np.sqrt(r * r * sin_t ** 2 + (r_th ** 2 * sin_t ** 2 + r_ph ** 2) / A)
    # proper-frame gradient of E_gamma - E_a on the leaf [m_a / R]
    nv = np.stack([p["n0"], p["n1"], p["n2"]])
    gh = np.stack([p["gradh0"], p["gradh1"], p["gradh2"]])
    gp = gh + (np.sqrt(A) - 1) * (nv * gh).sum(0) * nv
    dE = np.linalg.norm(gp, axis=0)
    khat = np.stack([p["khat0"], p["khat1"], p["khat2"]])
    k = np.sqrt(p["K2"])                    # local axion = photon momentum [m_a]
    E = p["E"]
    kdE = k * (khat * gp).sum(0)            # k . dE
    # physical units
    ma = kw["m_a_eV"]
    R_eV = kw["R_km"] / HBARC_EV_KM
    g = kw.get("g_GeVinv", 1e-12) * 1e-9
    hbarc_cm = HBARC_EV_KM * 1e5
    n_inf = kw.get("rho_GeV_cm3", 0.45) * 1e9 * hbarc_cm ** 3 / ma
    B = p["Bmag"]
    w2, c2 = p["wp2"], p["cos2"]
    D = c2 * w2 * (w2 - 2 * E * E) + E ** 4
    P_ag = (0.5 * math.pi * g * g * B * B * E ** 4 * (1 - c2) / D) * (E * ma) / (
        np.abs(kdE) * ma * ma / R_eV)                       # Eq. CPAnisoCurved
    cos_n = kdE / (k * dE)                                   # Eq. AngleDefAniso
    v_a = k / E
    omega = E * ma
    integrand = hk * R_eV ** 2 * np.abs(cos_n) * v_a * omega * P_ag      # [eV^3 ... per k]
    # the sampling density of (theta, phi), khat and |k_inf|, and the momentum
    # volume: d^3k_loc = k_loc k_inf / A dk_inf dOmega_k; f_a / pdf(k_inf) =
    # n_inf / (4 pi k_inf^2)
    kinf = p["kinf"] * ma
    mom = k * ma * kinf / A
    fa_pdf = n_inf / (4 * math.pi * kinf ** 2)
    w_lit = (4 * math.pi) ** 2 / sin_t * integrand * mom * fa_pdf / n * EV_J / HBAR_EV_S
    rel = np.abs(w_lit[ok] / p["w"][ok] - 1)
    assert rel.max() < 1e-8, np.sort(rel)[-5:]
    # the cancellation is not trivial: cos(th_n) spans a wide range
    assert np.abs(cos_n[ok]).min() < 0.3 and np.abs(cos_n[ok]).max() > 0.7
