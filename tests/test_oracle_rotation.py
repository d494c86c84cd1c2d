"""Pins of the oracle's rigidly rotating magnetosphere (the cos(Omega t) of
Eq. GJDensity kept during the flight, Eq. Hamilton for all four canonical
pairs, state (x, k, t, k_t)).

* flat vacuum: straight lines at the speed of light, so the clock that the
  rotation phase records equals the distance travelled (dt/dl = dH/dk_t);
* radial vacuum Schwarzschild: the coordinate time from r0 to r_out is the
  closed form r_out - r0 + r_s ln((r_out - r_s)/(r0 - r_s)) (Shapiro delay);
* flat homogeneous isotropic plasma: the clock advances at 1 / v_g with the
  group velocity |k| / omega;
* production rays of a misaligned Goldreich-Julian star: H stays on shell at
  the end point with the end point's own t and k_t, and the energy in the
  corotating frame omega - Omega L_z is conserved (H depends on t only
  through phi - Omega t), while omega itself is Doppler shifted;
* an aligned rotator: the rotating integration is the static one bit for bit
  (H does not depend on t).
"""
import numpy as np

C_KM_S = 299792.458
GM_SUN_KM = 1.4766250


def _state(x_km, k_scaled, m_a, delta=0.0, psi=0.0):
    n = x_km.shape[1]
    st = np.zeros((8, n))
    st[:3] = x_km
    st[3:6] = k_scaled * m_a
    st[6] = delta
    st[7] = psi
    return np.ascontiguousarray(st)


def _omega_R(P_s, R_km):
    return 2.0 * np.pi / P_s * R_km / C_KM_S


def test_flat_vacuum_clock_is_distance(oracle):
    P, R, ma = 1e-3, 10.0, 1e-5
    star = oracle.star_vector(M_sun=0.0, R_km=R, P_s=P, plasma=oracle.PLASMA_VACUUM,
                              theta_m=0.7, rotation=oracle.ROTATION_RIGID, m_a_eV=ma)
    rng = np.random.default_rng(11)
    n = 6
    x0 = rng.uniform(2, 4, size=(3, n))
    k0 = rng.normal(size=(3, n))
    om = np.sqrt((k0**2).sum(0))
    psi0 = rng.uniform(0, 2 * np.pi, n)
    st = _state(x0 * R, k0, ma, delta=om - 1.0, psi=psi0)
    status = np.zeros(n, dtype=np.uint8)
    oracle.trace_forward(star, oracle.trace_opts(rtol=1e-12, r_out_over_R=200.0,
                                                 r_capture_over_R=1e-3), st, status)
    assert np.all(status == oracle.RAY_ESCAPED)
    dist = np.linalg.norm(st[:3] / R - x0, axis=0)
    t = (st[7] - psi0) / _omega_R(P, R)
    assert np.allclose(t, dist, rtol=1e-10, atol=0)
    assert np.allclose(st[6], om - 1.0, rtol=0, atol=1e-15)    # vacuum: dk_t/dl = 0


def test_radial_schwarzschild_shapiro_delay(oracle):
    P, R, M, ma = 1e-3, 10.0, 1.4, 1e-5
    rs = 2 * M * GM_SUN_KM / R
    star = oracle.star_vector(M_sun=M, R_km=R, P_s=P, plasma=oracle.PLASMA_VACUUM,
                              theta_m=0.3, rotation=oracle.ROTATION_RIGID, m_a_eV=ma)
    r0 = np.array([1.5, 3.0, 7.0])
    n = r0.size
    dirs = np.array([[0.0, 0.0, 1.0], [0.6, 0.0, 0.8], [0.0, -1.0, 0.0]]).T
    om = 1.3
    A0 = 1 - rs / r0
    # radial null ray: -om^2 / A + A k_r^2 = 0, covariant k = k_r n
    st = _state(dirs * r0 * R, dirs * (om / A0), ma, delta=om - 1.0, psi=0.25)
    status = np.zeros(n, dtype=np.uint8)
    r_out = 1000.0
    oracle.trace_forward(star, oracle.trace_opts(rtol=1e-12, r_out_over_R=r_out), st, status)
    assert np.all(status == oracle.RAY_ESCAPED)
    t = (st[7] - 0.25) / _omega_R(P, R)
    expect = r_out - r0 + rs * np.log((r_out - rs) / (r0 - rs))
    assert np.allclose(t, expect, rtol=1e-9, atol=0)


def test_flat_homogeneous_plasma_group_delay(oracle):
    P, R, ma, a = 1e-3, 10.0, 1e-5, 0.5
    star = oracle.star_vector(M_sun=0.0, R_km=R, P_s=P, plasma=oracle.PLASMA_HOMOG,
                              plasma_a=a, dispersion=oracle.DISP_ISO,
                              rotation=oracle.ROTATION_RIGID, m_a_eV=ma)
    rng = np.random.default_rng(5)
    n = 5
    x0 = rng.uniform(2, 4, size=(3, n))
    k0 = rng.normal(size=(3, n)) * 0.5
    om = np.sqrt((k0**2).sum(0) + a)
    st = _state(x0 * R, k0, ma, delta=om - 1.0, psi=0.0)
    status = np.zeros(n, dtype=np.uint8)
    oracle.trace_forward(star, oracle.trace_opts(rtol=1e-12, r_out_over_R=100.0,
                                                 r_capture_over_R=1e-3), st, status)
    assert np.all(status == oracle.RAY_ESCAPED)
    dist = np.linalg.norm(st[:3] / R - x0, axis=0)
    t = st[7] / _omega_R(P, R)
    vg = np.sqrt((k0**2).sum(0)) / om
    assert np.allclose(t, dist / vg, rtol=1e-10, atol=0)


def _misaligned_rays(oracle, rotation, theta_m=0.6, n=24, seed=3):
    P, R, ma = 1.0, 10.0, 1e-5
    star = oracle.star_vector(M_sun=1.0, R_km=R, P_s=P, theta_m=theta_m, m_a_eV=ma,
                              phase_mode=1, rotation=rotation)
    u = np.random.default_rng(seed).uniform(size=(6, n))
    st, w, status = oracle.sample(star, u)
    ok = status == oracle.RAY_READY
    st0 = st.copy()
    oracle.trace_forward(star, oracle.trace_opts(rtol=1e-10), st, status)
    return star, st0, st, status, ok, _omega_R(P, R), R, ma


def test_misaligned_rotator_on_shell_and_corotating_energy(oracle):
    star, st0, st, status, ok, wR, R, ma = _misaligned_rays(oracle, oracle.ROTATION_RIGID)
    esc = ok & (status == oracle.RAY_ESCAPED)
    assert esc.sum() >= 10
    # H = 0 at the end point, evaluated with its own omega = -k_t and phase
    H0 = oracle.hamiltonian(star, st0[:, ok])
    H = oracle.hamiltonian(star, st[:, esc])
    assert np.max(np.abs(H0)) < 1e-9
    assert np.max(np.abs(H)) < 1e-8
    # omega - Omega L_z conserved, L_z = x k_y - y k_x in units of R m_a
    Lz = lambda s: (s[0] * s[4] - s[1] * s[3]) / (R * ma)
    d_om = st[6, esc] - st0[6, esc]
    d_J = d_om - wR * (Lz(st[:, esc]) - Lz(st0[:, esc]))
    assert np.max(np.abs(d_J)) < 1e-11
    # ... while the frequency itself moves (Doppler shift by the turning plasma)
    assert np.max(np.abs(d_om)) > 1e-7


def test_aligned_rotator_is_the_static_trace(oracle):
    _, _, st_r, status_r, ok, _, _, _ = _misaligned_rays(oracle, oracle.ROTATION_RIGID,
                                                         theta_m=0.0, n=12, seed=4)
    _, _, st_s, status_s, _, _, _, _ = _misaligned_rays(oracle, oracle.ROTATION_SNAPSHOT,
                                                        theta_m=0.0, n=12, seed=4)
    assert ok.sum() >= 6
    assert np.array_equal(status_r, status_s)
    assert np.array_equal(st_r[:6, ok], st_s[:6, ok])
    assert np.allclose(st_r[6, ok], st_s[6, ok], rtol=0, atol=1e-15)
