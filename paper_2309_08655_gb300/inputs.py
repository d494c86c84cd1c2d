"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle and the benchmark.

This module holds no arithmetic of the method: only a counter-based uniform
generator and the parameter sets of the synthetic workloads (stars shaped on
the paper's fiducial and magnetar parameters, Sec. 5 and Sec. 6).

Uniforms: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  Output i of stream ``seed`` is
``mix(seed * 2^32 + (i + 1) * 0x9E3779B97F4A7C15)``; the top 53 bits give
``(k + 0.5) * 2^-53``, so every uniform lies strictly inside (0, 1).
Each conversion sample j draws the six uniforms 6j .. 6j + 5 of its stream.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start + count - 1 of stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
        z = np.uint64((seed << 32) & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, start: int, count: int) -> np.ndarray:
    z = splitmix64(seed, start, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def sample_uniforms(seed: int, n: int, first: int = 0) -> np.ndarray:
    """Uniforms of samples first .. first + n - 1, SoA (6, n) float64."""
    u = uniforms(seed, 6 * first, 6 * n)
    return np.ascontiguousarray(u.reshape(n, 6).T)


# --- synthetic workloads -----------------------------------------------------
# Star dictionaries use the keys of the C-ABI parameter block (include/rt.h).

def star_config0() -> dict:
    """Aligned non-rotating-snapshot neutron star: M = 1.4 Msun, R = 10 km,
    B0 = 1e14 G, P = 1 s, Goldreich-Julian plasma, anisotropic dispersion.
    m_a = 1.094e-6 eV places the polar resonance (omega_p = m_a) at 200 km."""
    return dict(M_sun=1.4, R_km=10.0, B0_G=1e14, P_s=1.0, theta_m=0.0, psi=0.0,
                m_a_eV=1.094e-6, g_GeVinv=1e-12, rho_GeV_cm3=0.45, v0_kms=200.0,
                dispersion=0, resonance=0, fa_model=0, weight_mode=0, prop_metric=0,
                phase_mode=0, plasma=0, plasma_a=0.0)


CONFIG0 = dict(name="forward_aligned_4096", n=4096, seed=0, rtol=1e-10, r_out_over_R=1000.0,
               nth=64, nph=32, nnu=128, nu_lo=0.0, nu_hi=9.0)


def config1_masses(seed: int = 1, nsub: int = 16) -> np.ndarray:
    """Axion masses of the sub-batches, log-uniform in [1e-6, 5e-3] eV."""
    u = uniforms(seed, 1 << 40, nsub)
    lo, hi = math.log(1e-6), math.log(5e-3)
    return np.exp(lo + u * (hi - lo))


def stars_config1(seed: int = 1, nsub: int = 16) -> list[dict]:
    """Misaligned magnetar-like rotator (B0 = 1.6e14 G, P = 3.76 s,
    theta_m = 30 deg, M = 1.5 Msun, R = 11 km), one star per axion mass,
    rotation phase drawn per ray (period average)."""
    out = []
    for m in config1_masses(seed, nsub):
        s = star_config0()
        s.update(M_sun=1.5, R_km=11.0, B0_G=1.6e14, P_s=3.76, theta_m=math.radians(30.0),
                 m_a_eV=float(m), phase_mode=1)
        out.append(s)
    return out


CONFIG1 = dict(name="forward_misaligned_16x65536", nsub=16, n_per_sub=1 << 16, seed=1,
               rtol=1e-10, rtol_mixed=1e-8, r_out_over_R=1000.0, max_steps=100000, nth=64,
               nph=32, nnu=128, nu_lo=0.0, nu_hi=9.0)


def instances_config3(seed: int = 3, n: int = 256) -> list[dict]:
    """Uneven batch of star/axion configurations: B0 log-uniform in
    [1e12, 1e15] G, P uniform in [0.1, 10] s, misalignment uniform in
    [0, 90] deg, m_a log-uniform in [1e-6, 5e-3] eV, M = 1.4 Msun, R = 10 km;
    ray counts log-uniform in [1e3, 1e6]; odd instances are backward images
    (side ceil(sqrt(N)), observer direction uniform on the sphere), even ones
    forward batches with a uniform rotation phase per ray."""
    u = uniforms(seed, 1 << 41, 7 * n).reshape(n, 7)
    out = []
    for i in range(n):
        v = u[i]
        B0 = math.exp(math.log(1e12) + v[0] * (math.log(1e15) - math.log(1e12)))
        P = 0.1 + v[1] * (10.0 - 0.1)
        th = v[2] * 0.5 * math.pi
        ma = math.exp(math.log(1e-6) + v[3] * (math.log(5e-3) - math.log(1e-6)))
        N = int(round(math.exp(math.log(1e3) + v[4] * (math.log(1e6) - math.log(1e3)))))
        star = star_config0()
        star.update(M_sun=1.4, R_km=10.0, B0_G=B0, P_s=P, theta_m=th, m_a_eV=ma,
                    phase_mode=1 if i % 2 == 0 else 0, psi=2.0 * math.pi * v[6])
        inst = dict(star=star, n=N, mode="backward" if i % 2 else "forward",
                    seed=seed * 100000 + i)
        if i % 2:
            inst["side"] = int(math.ceil(math.sqrt(N)))
            inst["incl"] = math.acos(1.0 - 2.0 * v[5])
        out.append(inst)
    return out
