"""Pins of the oracle's plasma, Hamiltonian, dispersion and sampler.

Each check compares the oracle with something it does not compute itself:
finite differences, the algebraic dispersion relation, a number the paper
prints, scipy's Maxwell distribution, or a special case with a closed form.
"""
import os

import numpy as np
import pytest
from scipy import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_states(oracle, star, n, seed, rmin=15.0, rmax=400.0):
    """Random physical states (8, n) at radii in [rmin, rmax] km (R = 10 km)."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    r = rng.uniform(rmin, rmax, n)
    k = rng.normal(size=(3, n))
    m_a = star[oracle.STAR_KEYS.index("m_a_eV")]
    st = np.zeros((8, n))
    st[:3] = d * r
    st[3:6] = k * m_a
    st[6] = rng.uniform(0, 1e-6, n)
    st[7] = rng.uniform(0, 2 * np.pi, n)
    return st


STARS = {
    "gj_aligned_aniso": dict(M_sun=1.4, m_a_eV=1e-5),
    "gj_misaligned_aniso": dict(M_sun=1.5, R_km=10.0, theta_m=0.5, m_a_eV=2e-5, B0_G=1.6e14,
                                P_s=3.76),
    "gj_iso": dict(M_sun=1.0, dispersion=1, m_a_eV=1e-5),
    "flat_aniso": dict(M_sun=0.0, m_a_eV=1e-5, theta_m=0.3),
    "linear_iso_flat": dict(M_sun=0.0, dispersion=1, plasma=3, plasma_a=0.02),
}


@pytest.mark.parametrize("name", list(STARS))
def test_dual_gradient_matches_central_differences(oracle, name):
    star = oracle.star_vector(**STARS[name])
    R = star[oracle.STAR_KEYS.index("R_km")]
    m_a = star[oracle.STAR_KEYS.index("m_a_eV")]
    st = _random_states(oracle, star, 16, seed=1)
    H0, rhs = oracle.hamiltonian(star, st, with_rhs=True)
    eps = 1e-6
    for c in range(6):
        sp, sm = st.copy(), st.copy()
        scale = R if c < 3 else m_a
        sp[c] += eps * scale
        sm[c] -= eps * scale
        fd = (oracle.hamiltonian(star, sp) - oracle.hamiltonian(star, sm)) / (2 * eps)
        # dx/dl = dH/dk, dk/dl = -dH/dx
        ad = rhs[c + 3] if c < 3 else rhs[c - 3]
        ad = -ad if c < 3 else ad
        err = np.abs(fd - ad) / (1.0 + np.abs(ad))
        assert err.max() < 1e-6, (name, c, err.max())


@pytest.mark.parametrize("cos2", [0.0, 0.13, 0.5, 0.87, 1.0])
@pytest.mark.parametrize("K2,wp2", [(0.3, 1.2), (2.0, 0.5), (1.0, 1.0), (1e-3, 4.0)])
def test_lo_energy_solves_dispersion_relation(oracle, K2, wp2, cos2):
    E = oracle.photon_energy(0, K2, wp2, cos2)
    w2 = E * E
    # Eq. AnisotrpoicDisp: w^2 (w^2 - |k|^2 - wp^2) + |k|^2 wp^2 cos^2 = 0
    res = w2 * (w2 - K2 - wp2) + K2 * wp2 * cos2
    assert abs(res) < 1e-13 * (1 + w2 * w2)
    # LO is the upper root: at least max(|k|^2 cos^2, wp^2) ... and the limits
    assert w2 >= wp2 - 1e-14
    if cos2 == 1.0:
        assert np.isclose(w2, max(K2, wp2), rtol=1e-14)
    if cos2 == 0.0:
        assert np.isclose(w2, K2 + wp2, rtol=1e-14)
    assert np.isclose(oracle.photon_energy(1, K2, wp2, cos2) ** 2, K2 + wp2, rtol=1e-14)


def test_gj_normalisation_matches_paper_estimate(oracle):
    rows = np.loadtxt(os.path.join(GOLDEN, "gj_density.txt"), ndmin=2)
    for P, B0, n_paper, prec in rows:
        c = oracle.star_constants(oracle.star_vector(P_s=P, B0_G=B0))
        assert abs(c["n_gj_coef_cm3"] / n_paper - 1) < prec
        # the other common convention (field B0 at the equator, or n = Omega B/(2 pi e c)
        # with |B| = B0 at the pole) doubles it and falls outside the quoted precision
        assert abs(2 * c["n_gj_coef_cm3"] / n_paper - 1) > prec


def test_gj_density_angular_structure(oracle):
    star = oracle.star_vector(M_sun=1.4, m_a_eV=1e-5)
    R = 10.0
    th = np.linspace(0.01, np.pi - 0.01, 101)
    r = 3.0 * R
    x = np.stack([r * np.sin(th), np.zeros_like(th), r * np.cos(th)])
    wp2 = oracle.plasma_freq2(star, x)
    coef = oracle.star_constants(star)["wp2_coef"]
    expect = coef * (R / r) ** 3 * np.abs(3 * np.cos(th) ** 2 - 1)
    assert np.allclose(wp2, expect, rtol=1e-13)
    # vanishes on the null cone 3 cos^2 th = 1
    thn = np.arccos(1 / np.sqrt(3))
    xn = np.array([[r * np.sin(thn)], [0.0], [r * np.cos(thn)]])
    assert oracle.plasma_freq2(star, xn)[0] < 1e-12 * coef
    # misaligned star at phase psi: the pole moves to the magnetic axis
    tm, psi = 0.4, 1.1
    star2 = oracle.star_vector(M_sun=1.4, m_a_eV=1e-5, theta_m=tm)
    mhat = np.array([np.sin(tm) * np.cos(psi), np.sin(tm) * np.sin(psi), np.cos(tm)])
    xm = (mhat * r)[:, None]
    # at the magnetic pole: |3 cos(th) (m.n) - cos(th_m)| = |3 cos(tm) - cos(tm)| = 2 cos(tm)
    assert np.isclose(oracle.plasma_freq2(star2, xm, psi)[0],
                      coef * (R / r) ** 3 * 2 * np.cos(tm), rtol=1e-13)


def test_config0_axion_mass_puts_polar_surface_at_200km(oracle):
    star = oracle.star_vector(M_sun=1.4, R_km=10.0, B0_G=1e14, P_s=1.0, m_a_eV=1.094e-6)
    x = np.array([[0.0], [0.0], [200.0]])
    assert abs(oracle.plasma_freq2(star, x)[0] - 1.0) < 2e-3


def test_maxwell_speed_matches_scipy(oracle):
    us = np.array([1e-6, 0.01, 0.1, 0.3, 0.5, 0.7, 0.9, 0.99, 1 - 1e-9])
    ref = stats.maxwell.ppf(us, scale=1 / np.sqrt(2))
    got = np.array([oracle.maxwell_speed(u) for u in us])
    assert np.allclose(got, ref, rtol=1e-9)
    assert oracle.maxwell_speed(0.3, fa_model=1) == 1.0


def _perp_and_par(oracle, star, n, psi=0.0):
    """Unit vectors perpendicular and parallel to the dipole field direction at n."""
    tm = star[oracle.STAR_KEYS.index("theta_m")]
    m = np.array([np.sin(tm) * np.cos(psi), np.sin(tm) * np.sin(psi), np.cos(tm)])
    b = 3 * (m @ n) * n - m
    b /= np.linalg.norm(b)
    p = np.cross(b, [0.3, -0.2, 0.9])
    p /= np.linalg.norm(p)
    return p, b


@pytest.mark.parametrize("theta", [0.2, 0.7, 1.3, 2.5])
def test_resonance_special_cases(oracle, theta):
    star = oracle.star_vector(M_sun=1.4, R_km=10.0, m_a_eV=1.094e-6)
    n = np.array([np.sin(theta) * np.cos(0.4), np.sin(theta) * np.sin(0.4), np.cos(theta)])
    kperp, kpar = _perp_and_par(oracle, star, n)
    omega_inf = 1.0 + 3e-7
    rs = oracle.star_constants(star)["rs_over_R"]
    for khat, kind in [(kperp, "perp"), (kpar, "par")]:
        r = oracle.resonance_root(star, n, khat, omega_inf)
        if r is None:
            continue
        x = (n * r * 10.0)[:, None]
        wp2 = oracle.plasma_freq2(star, x)[0]
        A = 1 - rs / r
        E2 = omega_inf**2 / A
        if kind == "perp":
            # theta_B = 90 deg: the resonance is exactly omega_p = m_a
            assert abs(wp2 - 1.0) < 1e-12
        else:
            # theta_B = 0: omega_p = omega (the local photon energy)
            assert abs(wp2 / E2 - 1.0) < 1e-12


def test_sampled_points_are_on_shell_and_matched(oracle):
    star = oracle.star_vector(M_sun=1.4, R_km=10.0, B0_G=1e14, P_s=1.0, m_a_eV=1.094e-6)
    rng = np.random.default_rng(7)
    u = rng.random((6, 512))
    st, w, status = oracle.sample(star, u)
    ok = status == oracle.RAY_READY
    assert ok.sum() > 400
    H = oracle.hamiltonian(star, st[:, ok])
    # photon on shell (H = 0) with the axion's k_mu: E_gamma = E_a = sqrt(m_a^2 + |k|^2)
    assert np.abs(H).max() < 1e-12
    assert np.all(w[ok] > 0) and np.all(w[~ok] == 0)
    # misaligned rotator with random phases
    star2 = oracle.star_vector(M_sun=1.5, R_km=11.0, B0_G=1.6e14, P_s=3.76, theta_m=np.pi / 6,
                               phase_mode=1, m_a_eV=2e-5)
    st2, w2, status2 = oracle.sample(star2, u)
    ok2 = status2 == oracle.RAY_READY
    assert ok2.sum() > 100
    assert np.abs(oracle.hamiltonian(star2, st2[:, ok2])).max() < 1e-12
    assert np.allclose(st2[7], 2 * np.pi * u[5])


def test_empty_surface_gives_no_roots(oracle):
    # polar surface omega_p of this star is ~6.4e-5 eV: a heavier axion has no resonance
    star = oracle.star_vector(M_sun=1.5, R_km=11.0, B0_G=1.6e14, P_s=3.76, theta_m=np.pi / 6,
                              phase_mode=1, m_a_eV=2e-4)
    u = np.random.default_rng(3).random((6, 256))
    st, w, status = oracle.sample(star, u)
    assert np.all(status == oracle.RAY_NO_ROOT) and np.all(w == 0)


# --- twisted magnetar magnetosphere (Sec. 6, Eq. neMag) ----------------------


def _n_e_cm3(wp2, m_a):
    """n_e [cm^-3] from omega_p^2 / m_a^2: n_e = omega_p^2 m_e / e^2 (e^2 = 4 pi alpha)."""
    alpha = 7.2973525693e-3
    hbarc_cm = 1.973269804e-10 * 1e5
    n_ev3 = wp2 * m_a ** 2 * 510998.95 / (4 * np.pi * alpha)
    return n_ev3 / hbarc_cm ** 3


def test_twisted_density_matches_paper_estimate(oracle):
    rows = np.loadtxt(os.path.join(GOLDEN, "twisted_density.txt"), ndmin=2)
    for lam, psi, B0, R, n_paper, prec, ratio_paper, lprec in rows:
        m_a = 1e-4
        star = oracle.star_vector(R_km=R, B0_G=B0, P_s=3.76, m_a_eV=m_a, plasma=5,
                                  plasma_a=lam * psi)
        # on the magnetic equator (sin^2 theta = 1) of the surface, aligned rotator
        x = np.array([[R], [0.0], [0.0]])
        n_e = _n_e_cm3(oracle.plasma_freq2(star, x)[0], m_a)
        assert abs(n_e / n_paper - 1) < prec, n_e
        # against the Goldreich-Julian density at the pole of the same star
        gj = oracle.star_vector(R_km=R, B0_G=B0, P_s=3.76, m_a_eV=m_a)
        n_gj = _n_e_cm3(oracle.plasma_freq2(gj, np.array([[0.0], [0.0], [R]]))[0], m_a)
        assert abs(np.log10(n_e / n_gj / (lam * ratio_paper))) < lprec, n_e / n_gj


def test_twisted_density_angular_and_radial_structure(oracle):
    """omega_p^2 = c sin^2(theta_mag) (R/r)^4, linear in lambda psi and B0,
    1/m_a^2, independent of the rotation period, following the magnetic axis."""
    R = 11.0
    base = dict(R_km=R, B0_G=1.6e14, P_s=3.76, m_a_eV=1e-3, plasma=5, plasma_a=0.2)
    star = oracle.star_vector(**base)
    th = np.linspace(0.0, np.pi, 37)
    r = np.array([1.0, 1.7, 4.2]) * R
    pts = np.concatenate([np.stack([rr * np.sin(th), np.zeros_like(th), rr * np.cos(th)])
                          for rr in r], axis=1)
    wp2 = oracle.plasma_freq2(star, pts)
    c = oracle.plasma_freq2(star, np.array([[R], [0.0], [0.0]]))[0]
    rr = np.repeat(r, th.size)
    tt = np.tile(th, r.size)
    assert np.allclose(wp2, c * np.sin(tt) ** 2 * (R / rr) ** 4, rtol=1e-12, atol=1e-14 * c)
    for k, f in (("plasma_a", 3.0), ("B0_G", 2.5), ("m_a_eV", 0.5), ("P_s", 7.0)):
        kw = dict(base)
        kw[k] = base[k] * f
        c2 = oracle.plasma_freq2(oracle.star_vector(**kw), np.array([[R], [0.0], [0.0]]))[0]
        expect = {"plasma_a": f, "B0_G": f, "m_a_eV": 1 / f ** 2, "P_s": 1.0}[k]
        assert np.isclose(c2 / c, expect, rtol=1e-13), k
    # misaligned: zero on the magnetic axis at phase psi, maximal across it
    tm, ph = 0.5, 2.0
    s2 = oracle.star_vector(**dict(base, theta_m=tm))
    mh = np.array([np.sin(tm) * np.cos(ph), np.sin(tm) * np.sin(ph), np.cos(tm)])
    assert oracle.plasma_freq2(s2, (2 * R * mh)[:, None], ph)[0] < 1e-14 * c
    e = np.cross(mh, [0.0, 0.0, 1.0])
    e /= np.linalg.norm(e)
    assert np.isclose(oracle.plasma_freq2(s2, (2 * R * e)[:, None], ph)[0], c / 16, rtol=1e-12)


def test_twisted_open_field_lines_are_excluded(oracle):
    """Samples whose conversion point lies on an open field line (the dipole
    line r / sin^2 theta = L reaching the light cylinder, L >= c / Omega) get
    no resonance and weight 0; all others are kept unchanged."""
    from paper_2309_08655_gb300 import inputs as I
    R = 10.0
    base = dict(R_km=R, B0_G=1e14, m_a_eV=1e-3, plasma=5, plasma_a=0.2, theta_m=0.3,
                psi=0.7)
    u = I.sample_uniforms(77, 4000)
    slow = oracle.star_vector(**dict(base, P_s=10.0))          # r_LC ~ 4.8e4 R
    fast = oracle.star_vector(**dict(base, P_s=4.5e-4))        # r_LC ~ 2.1 R
    st_s, w_s, s_s = oracle.sample(slow, u)
    st_f, w_f, s_f = oracle.sample(fast, u)
    r_lc = 299792.458 * 4.5e-4 / (2 * np.pi) / R
    mh = np.array([np.sin(0.3) * np.cos(0.7), np.sin(0.3) * np.sin(0.7), np.cos(0.3)])
    ok = s_s == oracle.RAY_READY
    assert ok.sum() > 1000
    x = st_s[:3] / R
    r = np.linalg.norm(x, axis=0)
    with np.errstate(invalid="ignore", divide="ignore"):     # r = 0 where no root
        cos_t = (mh[:, None] * x).sum(0) / r
        L = r / (1 - cos_t ** 2)
    assert np.any(ok & (L >= r_lc)) and np.any(ok & (L < r_lc))
    open_ = ok & (L >= r_lc)
    assert np.all(s_f[open_] == oracle.RAY_NO_ROOT) and np.all(w_f[open_] == 0.0)
    keep = ok & (L < r_lc)
    assert np.all(s_f[keep] == oracle.RAY_READY)
    assert np.array_equal(st_f[:, keep], st_s[:, keep]) and np.array_equal(w_f[keep], w_s[keep])
