"""Pins of the oracle's ray integration against closed forms and invariants.

* flat space, homogeneous isotropic plasma: straight lines, constant k;
* flat space, planar-stratified plasma omega_p^2 = a z: a parabola with
  conserved k_x, k_y (Snell) and the turning point omega^2 - a z* = k_x^2 + k_y^2;
* vacuum Schwarzschild: azimuth swept between two crossings of r = X against
  an independent quadrature of the orbit integral, and capture exactly below
  the critical impact parameter 3 sqrt(3) GM;
* invariants along production rays: H = 0, k_t (by construction) and, for an
  aligned rotator, L_z = x k_y - y k_x;
* time reversal, and a brute-force fixed-step RK4 with Richardson
  extrapolation.
"""
import numpy as np
import pytest
from scipy import integrate, optimize

GM_SUN_KM = 1.4766250


def _state(x_km, k_scaled, m_a, delta=0.0, psi=0.0):
    n = x_km.shape[1]
    st = np.zeros((8, n))
    st[:3] = x_km
    st[3:6] = k_scaled * m_a
    st[6] = delta
    st[7] = psi
    return np.ascontiguousarray(st)


def test_flat_homogeneous_plasma_straight_lines(oracle):
    a = 0.5
    star = oracle.star_vector(M_sun=0.0, R_km=1.0, dispersion=1, plasma=2, plasma_a=a,
                              m_a_eV=1e-5)
    rng = np.random.default_rng(0)
    n = 8
    x0 = rng.uniform(5, 10, size=(3, n))
    k0 = rng.normal(size=(3, n)) * 0.4
    omega = np.sqrt((k0**2).sum(0) + a)            # -omega^2 + |k|^2 + a = 0
    st = _state(x0, k0, 1e-5, delta=omega - 1.0)
    lam = 3.0
    status = np.zeros(n, dtype=np.uint8)
    oracle.trace_forward(star, oracle.trace_opts(rtol=1e-12, lambda_max=lam, r_out_over_R=1e9,
                                                 r_capture_over_R=1e-3), st, status)
    assert np.all(status == oracle.RAY_LAMBDA_END)
    # dx/dl = 2k (units of R and m_a), dk/dl = 0
    assert np.allclose(st[:3], x0 + 2 * k0 * lam, rtol=0, atol=1e-10)
    assert np.allclose(st[3:6] / 1e-5, k0, rtol=0, atol=1e-12)


def test_flat_linear_plasma_parabola_and_turning_point(oracle):
    a = 0.02
    star = oracle.star_vector(M_sun=0.0, R_km=1.0, dispersion=1, plasma=3, plasma_a=a,
                              m_a_eV=1e-5)
    x0 = np.array([[0.0], [0.0], [10.0]])
    k0 = np.array([[0.3], [0.1], [0.6]])
    omega2 = (k0**2).sum() + a * x0[2, 0]
    st = _state(x0, k0, 1e-5, delta=np.sqrt(omega2) - 1.0)
    lam = 40.0
    status = np.zeros(1, dtype=np.uint8)
    oracle.trace_forward(star, oracle.trace_opts(rtol=1e-12, lambda_max=lam, r_out_over_R=1e9,
                                                 r_capture_over_R=1e-3), st, status)
    assert status[0] == oracle.RAY_LAMBDA_END
    # H = -w^2 + k^2 + a z: dk_z/dl = -a, dz/dl = 2 k_z -> z = z0 + 2 kz0 l - a l^2
    x_exp = x0[:2, 0] + 2 * k0[:2, 0] * lam
    z_exp = x0[2, 0] + 2 * k0[2, 0] * lam - a * lam**2
    assert np.allclose(st[:2, 0], x_exp, atol=1e-9)
    assert abs(st[2, 0] - z_exp) < 1e-9 * (1 + abs(z_exp))
    assert np.allclose(st[3:5, 0] / 1e-5, k0[:2, 0], atol=1e-12)   # Snell: k_x, k_y conserved
    assert abs(st[5, 0] / 1e-5 - (k0[2, 0] - a * lam)) < 1e-11
    # turning point: the ray turns at k_z = 0, where omega^2 - a z* = k_x^2 + k_y^2
    lam_t = k0[2, 0] / a
    z_t = x0[2, 0] + 2 * k0[2, 0] * lam_t - a * lam_t**2
    assert abs(omega2 - a * z_t - (k0[0, 0] ** 2 + k0[1, 0] ** 2)) < 1e-12


def _vacuum_star(M_sun, R_km):
    return dict(M_sun=M_sun, R_km=R_km, dispersion=1, plasma=1, m_a_eV=1e-5)


def _vacuum_ray(rs, X, b):
    """Photon at (X, 0, 0) with impact parameter b (same length unit), omega_inf = 1."""
    A = 1 - rs / X
    ky = b / X                      # L = X k_y = b omega_inf
    kr = -np.sqrt((1.0 / A - ky**2) / A)
    return np.array([X, 0.0, 0.0]), np.array([kr, ky, 0.0])


def _exact_sweep(rs, X, b):
    """2 int_{r0}^{X} dr / (r^2 sqrt(1/b^2 - A/r^2)), in u = 1/r.

    G(u) = 1/b^2 - u^2 + rs u^3 = (u0 - u) Q(u) with
    Q(u) = (1 - rs u0)(u + u0) - rs u^2, so the integrand is
    (u0 - u)^(-1/2) Q(u)^(-1/2) with an integrable end-point singularity.
    """
    G = lambda u: 1 / b**2 - u**2 + rs * u**3
    u0 = optimize.brentq(G, 1 / X, 2 / (3 * rs), xtol=1e-300, rtol=1e-15)
    Q = lambda u: (1 - rs * u0) * (u + u0) - rs * u * u
    val, err = integrate.quad(lambda u: 1 / np.sqrt(Q(u)), 1 / X, u0, weight="alg",
                              wvar=(0.0, -0.5), epsabs=1e-15, epsrel=1e-14, limit=200)
    return 2 * val


@pytest.mark.parametrize("b_over_rs", [30.0, 300.0, 3000.0])
def test_vacuum_schwarzschild_sweep_matches_orbit_integral(oracle, b_over_rs):
    M = 1.0
    rs_km = 2 * M * GM_SUN_KM
    R_km = 1.01 * rs_km
    star = oracle.star_vector(**_vacuum_star(M, R_km))
    rs = rs_km / R_km
    X = 1e5 * rs
    b = b_over_rs * rs
    x0, k0 = _vacuum_ray(rs, X, b)
    st = _state(x0[:, None] * R_km, k0[:, None], 1e-5)
    status = np.zeros(1, dtype=np.uint8)
    oracle.trace_forward(star, oracle.trace_opts(rtol=1e-13, r_out_over_R=X * (1 - 1e-12)), st,
                         status)
    assert status[0] == oracle.RAY_ESCAPED
    phi = np.arctan2(st[1, 0], st[0, 0]) % (2 * np.pi)
    exact = _exact_sweep(rs, X, b)
    assert abs(phi - exact) < 1e-9, (phi, exact)


def test_orbit_integral_reduces_to_weak_field_deflection():
    # pins the quadrature reference itself against the weak-field series
    # alpha = 4 m/b + (15 pi/4) (m/b)^2 + (128/3) (m/b)^3 + O((m/b)^4), m = GM
    rs = 1.0
    for b in [1e2, 1e3, 1e4]:
        X = 1e12
        alpha = _exact_sweep(rs, X, b) - np.pi + 2 * np.arcsin(b / X)
        GMb = 0.5 * rs / b
        approx = 4 * GMb + 15 * np.pi / 4 * GMb**2 + 128 / 3 * GMb**3
        assert abs(alpha - approx) < 200 * GMb**4 + 1e-13


@pytest.mark.parametrize("frac,expect", [(0.99, 2), (1.01, 1)])
def test_photon_sphere_capture_threshold(oracle, frac, expect):
    M = 1.0
    rs_km = 2 * M * GM_SUN_KM
    R_km = 1.01 * rs_km                   # capture sphere inside the photon sphere
    star = oracle.star_vector(**_vacuum_star(M, R_km))
    rs = rs_km / R_km
    X = 2000 * rs
    b = frac * 1.5 * np.sqrt(3) * rs       # b_crit = 3 sqrt(3) GM
    x0, k0 = _vacuum_ray(rs, X, b)
    st = _state(x0[:, None] * R_km, k0[:, None], 1e-5)
    status = np.zeros(1, dtype=np.uint8)
    oracle.trace_forward(star, oracle.trace_opts(rtol=1e-12, r_out_over_R=X * (1 - 1e-9)), st,
                         status)
    assert status[0] == expect


def _config0_star(oracle, **kw):
    p = dict(M_sun=1.4, R_km=10.0, B0_G=1e14, P_s=1.0, m_a_eV=1.094e-6)
    p.update(kw)
    return oracle.star_vector(**p)


def test_invariants_on_production_rays(oracle):
    star = _config0_star(oracle)
    u = np.random.default_rng(11).random((6, 96))
    st, w, status = oracle.sample(star, u)
    Lz0 = st[0] * st[4] - st[1] * st[3]
    rtol = 1e-12
    nacc, nrej, lam = oracle.trace_forward(star, oracle.trace_opts(rtol=rtol), st, status)
    esc = status == oracle.RAY_ESCAPED
    assert esc.sum() > 60
    H = oracle.hamiltonian(star, st[:, esc])
    # H / m_a^2 = 0 up to the accumulated local errors
    assert np.all(np.abs(H) < 50 * rtol * nacc[esc])
    # aligned rotator: axisymmetric H, so L_z is conserved
    Lz = st[0] * st[4] - st[1] * st[3]
    scale = np.abs(st[0] * st[4]) + np.abs(st[1] * st[3]) + 1e-30
    assert np.all(np.abs(Lz - Lz0)[esc] / scale[esc] < 50 * rtol * nacc[esc])


def _lambda_limited(oracle, star, st0, lam, rtol):
    st = st0.copy()
    s = np.zeros(st0.shape[1], dtype=np.uint8)
    nacc, _, _ = oracle.trace_forward(
        star, oracle.trace_opts(rtol=rtol, lambda_max=lam, r_out_over_R=1e9,
                                r_capture_over_R=1.0), st, s)
    return st, s == oracle.RAY_LAMBDA_END, nacc


def _well_conditioned(oracle, star, st0, lam):
    """Rays whose end state moves by < 1e-12 (relative) between rtol 1e-12 and 1e-13.

    Rays that graze the kink of |Omega . B| on the Goldreich-Julian null cone or
    bounce near the surface amplify any perturbation; the comparisons below are
    stated on the well-conditioned set, as the parity tests are.
    """
    a, ka, _ = _lambda_limited(oracle, star, st0, lam, 1e-12)
    b, kb, _ = _lambda_limited(oracle, star, st0, lam, 1e-13)
    scale = np.abs(st0[:6]).max(axis=0)
    cond = np.abs(a[:6] - b[:6]).max(axis=0) / scale
    return b, ka & kb & (cond < 1e-12)


def test_time_reversal(oracle):
    star = _config0_star(oracle, theta_m=0.5, phase_mode=1)
    u = np.random.default_rng(12).random((6, 48))
    st0, w, status = oracle.sample(star, u)
    st0 = np.ascontiguousarray(st0[:, status == oracle.RAY_READY])
    lam = 5.0
    fwd, good = _well_conditioned(oracle, star, st0, lam)
    fwd[3:6] *= -1.0                      # k_i -> -k_i, k_t kept: H(x, -k) = H(x, k)
    back, kb, _ = _lambda_limited(oracle, star, fwd, lam, 1e-13)
    good &= kb
    assert good.sum() > 20
    back[3:6] *= -1.0
    dx = np.linalg.norm(back[:3] - st0[:3], axis=0) / np.linalg.norm(st0[:3], axis=0)
    dk = np.linalg.norm(back[3:6] - st0[3:6], axis=0) / np.linalg.norm(st0[3:6], axis=0)
    assert dx[good].max() < 1e-9 and dk[good].max() < 1e-9


def test_brute_force_rk4_richardson(oracle):
    star = _config0_star(oracle, theta_m=0.3)
    u = np.random.default_rng(13).random((6, 24))
    st0, w, status = oracle.sample(star, u)
    st0 = np.ascontiguousarray(st0[:, status == oracle.RAY_READY][:, :16])
    n = st0.shape[1]
    lam = 6.0
    dp5, good = _well_conditioned(oracle, star, st0, lam)
    a = st0.copy()
    b = st0.copy()
    oracle.trace_rk4(star, a, np.full(n, lam), 4000)
    oracle.trace_rk4(star, b, np.full(n, lam), 8000)
    rich = (16 * b - a) / 15
    scale = np.abs(st0[:6]).max(axis=0)
    err = np.abs(rich[:6] - dp5[:6]).max(axis=0) / scale
    # compare only where the brute force has itself converged (its Richardson
    # error estimate |b - a| / 15 is small): a fixed step loses its order where
    # the ray crosses the kink of |Omega . B| on the null cone
    good &= np.abs(b[:6] - a[:6]).max(axis=0) / 15 / scale < 1e-10
    assert good.sum() >= 8
    assert err[good].max() < 1e-11, err[good]


def test_flat_propagation_keeps_vacuum_rays_straight(oracle):
    """With M > 0 in the initial conditions but flat propagation (App. B) and
    no plasma, H = -W^2 + |k|^2 and a ray is the straight line x + 2 k l with
    constant k, whatever the mass."""
    star = oracle.star_vector(M_sun=1.4, R_km=10.0, m_a_eV=1e-5, plasma=1, prop_metric=1,
                              dispersion=1)
    x0 = np.array([3.0, -2.0, 5.0]) * 10.0                  # km
    k0 = np.array([0.3, 0.4, -0.1]) * 1e-5                  # eV, covariant
    st = np.zeros((8, 1))
    st[:3, 0] = x0
    st[3:6, 0] = k0
    st[6, 0] = 0.0
    s = np.zeros(1, dtype=np.uint8)
    lam = 2.0
    oracle.trace_forward(star, oracle.trace_opts(rtol=1e-12, lambda_max=lam, r_out_over_R=1e6),
                         st, s)
    assert s[0] == oracle.RAY_LAMBDA_END
    xs = x0 / 10.0 + 2.0 * (k0 / 1e-5) * lam
    assert np.allclose(st[:3, 0] / 10.0, xs, rtol=1e-12, atol=1e-12)
    assert np.allclose(st[3:6, 0], k0, rtol=1e-13, atol=0)
