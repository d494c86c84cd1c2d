"""The seeded input generator: SplitMix64 reference values and ranges."""
import numpy as np

from paper_2309_08655_gb300 import inputs as I


def test_splitmix64_reference_sequence():
    # SplitMix64 seeded with state 0 (Steele, Lea & Flood 2014): first outputs
    z = I.splitmix64(0, 0, 3)
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4
    assert int(z[2]) == 0x06C45D188009454F


def test_uniform_layout_and_range():
    u = I.sample_uniforms(3, 1000)
    assert u.shape == (6, 1000)
    assert np.all((u > 0) & (u < 1))
    flat = I.uniforms(3, 0, 6000)
    assert np.array_equal(u[:, 7], flat[42:48])
    # chunked generation equals one-shot generation
    assert np.array_equal(I.sample_uniforms(3, 10, first=990), u[:, 990:])
    assert abs(u.mean() - 0.5) < 0.02


def test_config1_masses_log_uniform_in_range():
    m = I.config1_masses()
    assert m.shape == (16,)
    assert np.all((m >= 1e-6) & (m <= 5e-3))
