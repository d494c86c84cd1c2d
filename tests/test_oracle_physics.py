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
