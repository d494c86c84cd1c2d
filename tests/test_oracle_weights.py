"""Pins of the oracle's conversion-surface weights and binning.

* Isotropic plasma (Eq. DispIsotropic, Eq. ProbIsoCurved): the resonance is
  the single surface omega_p = m_a and the total power reduces to a
  two-dimensional quadrature over that surface times a one-dimensional
  momentum integral (the analytic reduction of Sec. 4.4); the Monte-Carlo sum
  of the oracle's weights must agree within its statistical error.
* The delta-function Jacobian 1/|dh/dr| against a smeared delta integrated by
  quadrature.
* Binning: the histogram conserves the escaped weight, and bin conventions.
"""
import numpy as np
import pytest
from scipy import integrate

HBARC_EV_KM = 1.973269804e-10
HBAR_EV_S = 6.582119569e-16
EV_J = 1.602176634e-19
C_KM_S = 299792.458


def _iso_power_quadrature(oracle, star_kw):
    """P = (8 pi / 3) pi g^2 int dOmega r0^2 |B|^2 I_k(r0) / |d_r omega_p^2|  [W]."""
    star = oracle.star_vector(**star_kw)
    c = oracle.star_constants(star)
    m = star_kw["m_a_eV"]
    R = star_kw["R_km"] / HBARC_EV_KM                       # eV^-1
    rs = c["rs_over_R"]
    Cp = c["wp2_coef"] * m * m                              # eV^2
    B0 = c["B0_eV2"]
    g = star_kw.get("g_GeVinv", 1e-12) * 1e-9
    n_inf = c["n_inf_eV3"]
    k0 = m * star_kw.get("v0_kms", 200.0) / C_KM_S

    def I_k(r_over_R):
        A = 1 - rs / r_over_R

        def f(kinf):
            k = np.sqrt((m * m + kinf * kinf) / A - m * m)
            E2 = (m * m + kinf * kinf) / A
            return (k * kinf / A) * E2 * np.exp(-(kinf / k0) ** 2)

        val, _ = integrate.quad(f, 0, 12 * k0, epsrel=1e-11, epsabs=0, limit=200)
        return n_inf * val / (np.pi * k0 * k0) ** 1.5

    def integrand(th):
        F = abs(3 * np.cos(th) ** 2 - 1)
        r0 = (Cp * F / (m * m)) ** (1.0 / 3.0)              # units of R
        if r0 <= 1.0:
            return 0.0
        Bmag = 0.5 * B0 / r0**3 * np.sqrt(3 * np.cos(th) ** 2 + 1)
        dwp2 = 3 * m * m / (r0 * R)                         # |d_r omega_p^2| [eV^3]
        return np.sin(th) * (r0 * R) ** 2 * Bmag**2 * I_k(r0) / dwp2

    thc = np.arccos(1 / np.sqrt(3))
    tot = 0.0
    for a, b in [(0, thc), (thc, np.pi - thc), (np.pi - thc, np.pi)]:
        v, _ = integrate.quad(integrand, a, b, epsrel=1e-9, limit=200)
        tot += v
    P = (8 * np.pi / 3) * np.pi * g * g * 2 * np.pi * tot    # eV^2
    return P * EV_J / HBAR_EV_S


# (lighter axions put the surface near the null cone of the Goldreich-Julian
# density where |B|^2 r0^3 grows like 1 / |3 cos^2 th - 1|; the uniform-angle
# estimator is then heavy-tailed and needs far more samples)
@pytest.mark.parametrize("m_a", [4e-6, 1e-5])
def test_isotropic_total_power_matches_surface_quadrature(oracle, m_a):
    kw = dict(M_sun=1.4, R_km=10.0, B0_G=1e14, P_s=1.0, m_a_eV=m_a, dispersion=1)
    star = oracle.star_vector(**kw)
    n = 40000
    u = np.random.default_rng(21).random((6, n))
    st, w, status = oracle.sample(star, u)
    W = w * n                          # per-sample estimator of P
    mc, sig = W.mean(), W.std() / np.sqrt(n)
    quad = _iso_power_quadrature(oracle, kw)
    assert sig / mc < 0.05
    assert abs(mc - quad) < 4 * sig, (mc, quad, sig)


def test_delta_jacobian_against_smeared_delta(oracle):
    star = oracle.star_vector(M_sun=1.4, R_km=10.0, B0_G=1e14, P_s=1.0, m_a_eV=1.094e-6,
                              theta_m=0.4)
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(12):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        kh = rng.normal(size=3)
        kh /= np.linalg.norm(kh)
        om = 1.0 + 2e-7
        psi = 0.7
        r = oracle.resonance_root(star, n, kh, om, psi)
        if r is None:
            continue
        h0, dh = oracle.resonance_h(star, n, kh, om, psi, r)
        assert abs(h0) < 1e-12
        # int dr delta_eps(h(r)) -> 1/|h'(r*)| as eps -> 0 (Gaussian delta)
        eps = 1e-6 * abs(dh) * r
        hw = 8 * eps / abs(dh)
        f = lambda rr: np.exp(-0.5 * (oracle.resonance_h(star, n, kh, om, psi, rr)[0] / eps) ** 2)
        val, _ = integrate.quad(f, r - hw, r + hw, epsabs=0, epsrel=1e-10, points=[r], limit=200)
        val /= np.sqrt(2 * np.pi) * eps
        assert abs(val * abs(dh) - 1) < 1e-6
        checked += 1
    assert checked >= 6


def _escaped_state(oracle, star, dirs, deltas, r_km=1e4):
    n = dirs.shape[1]
    st = np.zeros((8, n))
    st[:3] = dirs * r_km
    m = star[oracle.STAR_KEYS.index("m_a_eV")]
    st[3:6] = dirs * m
    st[6] = deltas
    return np.ascontiguousarray(st)


def test_binning_conserves_escaped_weight_and_edges(oracle):
    star = oracle.star_vector(M_sun=0.0, R_km=10.0, m_a_eV=1e-5)
    v0 = 200.0 / C_KM_S
    y_unit = 0.5 * v0 * v0
    # directions and frequencies placed well inside bins (a round trip through
    # acos/atan2 cannot land exactly on an edge)
    d = 1e-7
    th = np.array([0.0, np.pi / 64 + d, np.pi - 1e-12, 1.0, 2.0, 1.0, 1.0])
    ph = np.array([0.0, 2 * np.pi / 32 + d, -1e-9, 3.0, 5.0, 1.0, 1.0])
    dirs = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    ys = np.array([0.0, 9.0 / 128 + d, 1.0, 8.999, 4.0, 9.0 + d, 12.0])
    st = _escaped_state(oracle, star, dirs, ys * y_unit)
    w = np.array([1.0, 2.0, 4.0, 8.0, 16.0, 32.0, 64.0])
    status = np.array([1, 1, 1, 1, 1, 1, 2], dtype=np.uint8)
    hist, oor = oracle.bin_rays(star, st, w, status)
    assert hist.sum() + oor == pytest.approx(w[status == 1].sum(), rel=1e-15)
    assert oor == 32.0                     # y >= 9 is outside [0, 9); the captured ray is dropped
    assert hist[0, 0, 0] == 1.0
    assert hist[1, 1, 1] == 2.0
    assert hist[63, 31, 14] == 4.0         # theta = pi -> last bin, phi wraps below 2 pi
    assert hist[int(1.0 / (np.pi / 64)), int(3.0 / (2 * np.pi / 32)), 127] == 8.0
    assert hist[int(2.0 / (np.pi / 64)), int(5.0 / (2 * np.pi / 32)), int(4.0 / (9 / 128))] == 16.0


def _iso_power_quadrature_twisted(oracle, star_kw):
    """The same reduction for the twisted magnetosphere (Sec. 6, Eq. neMag):
    omega_p^2 = C sin^2(th) (R/r)^4 on an aligned rotator, resonance surface
    r0(th) = (C sin^2 th / m_a^2)^(1/4), |d_r omega_p^2| = 4 m_a^2 / r0, and no
    conversion where r0 / sin^2 th >= c / Omega (open field lines)."""
    star = oracle.star_vector(**star_kw)
    c = oracle.star_constants(star)
    m = star_kw["m_a_eV"]
    R = star_kw["R_km"] / HBARC_EV_KM
    rs = c["rs_over_R"]
    coef = oracle.plasma_freq2(star, np.array([[star_kw["R_km"]], [0.0], [0.0]]))[0]
    B0 = c["B0_eV2"]
    g = star_kw.get("g_GeVinv", 1e-12) * 1e-9
    n_inf = c["n_inf_eV3"]
    k0 = m * star_kw.get("v0_kms", 200.0) / C_KM_S
    r_lc = C_KM_S * star_kw["P_s"] / (2 * np.pi) / star_kw["R_km"]

    def I_k(r_over_R):
        A = 1 - rs / r_over_R

        def f(kinf):
            k = np.sqrt((m * m + kinf * kinf) / A - m * m)
            E2 = (m * m + kinf * kinf) / A
            return (k * kinf / A) * E2 * np.exp(-(kinf / k0) ** 2)

        val, _ = integrate.quad(f, 0, 12 * k0, epsrel=1e-11, epsabs=0, limit=200)
        return n_inf * val / (np.pi * k0 * k0) ** 1.5

    def integrand(th):
        s2 = np.sin(th) ** 2
        r0 = (coef * s2) ** 0.25
        if r0 <= 1.0 or r0 / s2 >= r_lc:
            return 0.0
        Bmag = 0.5 * B0 / r0**3 * np.sqrt(3 * np.cos(th) ** 2 + 1)
        dwp2 = 4 * m * m / (r0 * R)
        return np.sin(th) * (r0 * R) ** 2 * Bmag**2 * I_k(r0) / dwp2

    tot, _ = integrate.quad(integrand, 0, np.pi, epsrel=1e-9, limit=400)
    P = (8 * np.pi / 3) * np.pi * g * g * 2 * np.pi * tot
    return P * EV_J / HBAR_EV_S


@pytest.mark.parametrize("P_s", [3.76, 5.8e-4])
def test_isotropic_twisted_power_matches_surface_quadrature(oracle, P_s):
    """Twisted magnetar density, isotropic dispersion: the Monte-Carlo total of
    the oracle's weights against the surface quadrature, with the light
    cylinder far away (3.76 s) and cutting the surface (0.58 ms: r_LC = 2.5 R
    against a surface at 1.6 R on the magnetic equator)."""
    kw = dict(M_sun=1.5, R_km=11.0, B0_G=1.6e14, P_s=P_s, m_a_eV=1e-3, dispersion=1,
              plasma=5, plasma_a=0.2)
    star = oracle.star_vector(**kw)
    n = 40000
    u = np.random.default_rng(22).random((6, n))
    st, w, status = oracle.sample(star, u)
    W = w * n
    mc, sig = W.mean(), W.std() / np.sqrt(n)
    quad = _iso_power_quadrature_twisted(oracle, kw)
    assert sig / mc < 0.05
    assert abs(mc - quad) < 4 * sig, (mc, quad, sig)


def test_unit_probability_weights_give_the_axion_flux_through_the_surface(oracle):
    """With the conversion probability set to one (weight_mode 1), the power is
    the axion energy flux through the conversion surface, int dSigma int d^3k
    f_a |cos theta_n| v_a omega = int dSigma n_inf <|k| |cos|>.  Flat space
    (M = 0), isotropic dispersion and the spherical test medium a (R/r)^3 make
    the surface the sphere r0 = a^(1/3) R, so the total is
    4 pi r0^2 n_inf <|k|> / 2 with <|k|> = 2 k0 / sqrt(pi) for the Maxwellian."""
    kw = dict(M_sun=0.0, R_km=10.0, B0_G=1e14, P_s=1.0, m_a_eV=1e-5, dispersion=1,
              plasma=4, plasma_a=8.0, weight_mode=1)
    star = oracle.star_vector(**kw)
    c = oracle.star_constants(star)
    n = 40000
    u = np.random.default_rng(23).random((6, n))
    st, w, status = oracle.sample(star, u)
    assert np.all(status == oracle.RAY_READY)
    W = w * n
    mc, sig = W.mean(), W.std() / np.sqrt(n)
    m = kw["m_a_eV"]
    r0 = 2.0 * kw["R_km"] / HBARC_EV_KM                      # a^(1/3) = 2, in eV^-1
    k0 = m * 200.0 / C_KM_S
    P = 4 * np.pi * r0 ** 2 * c["n_inf_eV3"] * k0 / np.sqrt(np.pi) * EV_J / HBAR_EV_S
    assert sig / mc < 0.02
    assert abs(mc - P) < 4 * sig, (mc, P, sig)
    # the per-sample weight is |k cos| per unit of the surface-and-momentum
    # measure: independent of B0 and the coupling, unlike the default weights
    st2, w2, _ = oracle.sample(oracle.star_vector(**dict(kw, B0_G=3e14, g_GeVinv=5e-12)), u)
    assert np.array_equal(w2, w)
    _, w_pag, _ = oracle.sample(oracle.star_vector(**dict(kw, weight_mode=0)), u)
    assert not np.allclose(w_pag, w)


def test_renormalised_weights_count_surface_crossings(oracle):
    """weight_mode 2 (Eq. reweight): the unit-probability weight times
    R_i = (1 cm^-3 / n_a(r_i)) (m_a / |k_a|) / sqrt(1 - r_s / r_i).  In flat
    space (n_a = n_inf, A = 1) the product no longer depends on the axion
    speed: the total is 4 pi r0^2 m_a (1 cm^-3) <|cos|> = 2 pi r0^2 m_a cm^-3
    on the sphere r0 = a^(1/3) R, for any velocity distribution."""
    hbarc_cm = HBARC_EV_KM * 1e5
    for fa_model, v0 in ((0, 200.0), (0, 600.0), (1, 200.0)):
        kw = dict(M_sun=0.0, R_km=10.0, B0_G=1e14, P_s=1.0, m_a_eV=1e-5, dispersion=1,
                  plasma=4, plasma_a=8.0, weight_mode=2, fa_model=fa_model, v0_kms=v0)
        star = oracle.star_vector(**kw)
        n = 40000
        u = np.random.default_rng(24).random((6, n))
        st, w, status = oracle.sample(star, u)
        W = w * n
        mc, sig = W.mean(), W.std() / np.sqrt(n)
        r0 = 2.0 * kw["R_km"] / HBARC_EV_KM
        P = 2 * np.pi * r0 ** 2 * kw["m_a_eV"] * hbarc_cm ** 3 * EV_J / HBAR_EV_S
        assert sig / mc < 0.02
        assert abs(mc - P) < 4 * sig, (fa_model, v0, mc, P, sig)


def test_renormalised_weights_in_curved_space(oracle):
    """With M > 0 the factor uses the focused density n_inf k_c / k0,
    k_c^2 = k0^2 + m_a^2 r_s / r (Sec. 4.3), the sample's own local momentum
    and the redshift; checked sample by sample against the unit weights."""
    kw = dict(M_sun=1.4, R_km=10.0, B0_G=1e14, P_s=1.0, m_a_eV=1e-5, dispersion=0)
    u = np.random.default_rng(25).random((6, 2000))
    st1, w1, s1 = oracle.sample(oracle.star_vector(**dict(kw, weight_mode=1)), u)
    st2, w2, s2 = oracle.sample(oracle.star_vector(**dict(kw, weight_mode=2)), u)
    assert np.array_equal(s1, s2) and np.array_equal(st1, st2)
    ok = s1 == oracle.RAY_READY
    c = oracle.star_constants(oracle.star_vector(**kw))
    R = 10.0
    r = np.linalg.norm(st1[:3, ok], axis=0) / R
    A = 1 - c["rs_over_R"] / r
    m = 1e-5
    # |k_a| from the covariant state: k_o = k + (sqrt(A) - 1)(n.k) n
    n = st1[:3, ok] / (r * R)
    k = st1[3:6, ok]
    kn = (n * k).sum(0)
    ko = k + (np.sqrt(A) - 1) * kn * n
    ka = np.linalg.norm(ko, axis=0)
    k0 = m * 200.0 / C_KM_S
    kc = np.sqrt(k0 ** 2 + m ** 2 * c["rs_over_R"] / r)
    Ri = (HBARC_EV_KM * 1e5) ** 3 / (c["n_inf_eV3"] * kc / k0) * (m / ka) / np.sqrt(A)
    assert np.allclose(w2[ok], w1[ok] * Ri, rtol=1e-12)
