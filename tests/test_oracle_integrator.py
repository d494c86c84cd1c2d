"""Pins of the oracle's Dormand-Prince 5(4) integrator against mathematics.

The Butcher-tree order conditions fix every tableau coefficient; the
continuous extension is checked for its order; the adaptive loop is checked on
a linear system with a closed-form solution (matrix exponential).
"""
import numpy as np
import pytest
from scipy.linalg import expm


@pytest.fixture(scope="module")
def tab(oracle):
    return oracle.dp5_tableau()


def _order_conditions(b, A, c, order):
    """Residuals of the rooted-tree order conditions up to ``order`` (<= 5)."""
    ac = A @ c
    ac2 = A @ c**2
    ac3 = A @ c**3
    aac = A @ ac
    res = [b.sum() - 1.0]
    if order >= 2:
        res += [b @ c - 1 / 2]
    if order >= 3:
        res += [b @ c**2 - 1 / 3, b @ ac - 1 / 6]
    if order >= 4:
        res += [b @ c**3 - 1 / 4, b @ (c * ac) - 1 / 8, b @ ac2 - 1 / 12, b @ aac - 1 / 24]
    if order >= 5:
        res += [
            b @ c**4 - 1 / 5,
            b @ (c**2 * ac) - 1 / 10,
            b @ (c * ac2) - 1 / 15,
            b @ (c * aac) - 1 / 30,
            b @ (ac * ac) - 1 / 20,
            b @ ac3 - 1 / 20,
            b @ (A @ (c * ac)) - 1 / 40,
            b @ (A @ ac2) - 1 / 60,
            b @ (A @ aac) - 1 / 120,
        ]
    return np.array(res)


def _full_A(tab):
    A = np.zeros((7, 7))
    A[:, :6] = tab["a"]
    return A


def test_row_sums_equal_nodes(tab):
    A = _full_A(tab)
    assert np.allclose(A.sum(axis=1), tab["c"], atol=1e-15)


def test_fifth_order_conditions(tab):
    res = _order_conditions(tab["b"], _full_A(tab), tab["c"], 5)
    assert np.abs(res).max() < 1e-14


def test_embedded_is_fourth_not_fifth_order(tab):
    A = _full_A(tab)
    assert np.abs(_order_conditions(tab["bh"], A, tab["c"], 4)).max() < 1e-14
    assert np.abs(_order_conditions(tab["bh"], A, tab["c"], 5)).max() > 1e-4


def test_error_weights_are_difference(tab):
    assert np.allclose(tab["e"], tab["b"] - tab["bh"], atol=1e-16, rtol=0)


def test_fsal_last_row_equals_b(tab):
    assert np.allclose(tab["a"][6, :6], tab["b"][:6], atol=0, rtol=0)
    assert tab["b"][6] == 0.0


def _rotation_matrix():
    M = np.zeros((6, 6))
    for i, w in enumerate([1.0, 2.0, 3.0]):
        M[2 * i, 2 * i + 1] = w
        M[2 * i + 1, 2 * i] = -w
    return M


@pytest.mark.parametrize("rtol", [1e-8, 1e-10, 1e-12])
def test_adaptive_linear_system_matches_expm(oracle, rtol):
    M = _rotation_matrix() + 0.05 * np.eye(6)
    y0 = np.array([1.0, 0.0, 0.5, -0.3, 0.2, 0.7])
    T = 7.0
    y, nacc = oracle.dp5_linear(M, y0, T, rtol)
    exact = expm(M * T) @ y0
    err = np.abs(y - exact).max()
    assert nacc > 10
    # global error of a tolerance-proportional method: a modest multiple of rtol
    assert err < 200 * rtol, (err, nacc)


def test_dense_output_endpoints_and_order(oracle):
    M = _rotation_matrix()
    y0 = np.array([1.0, 0.0, 0.5, -0.3, 0.2, 0.7])
    e_end = []
    for h in [0.2, 0.1]:
        y_end = oracle.dp5_linear_dense(M, y0, h, 1.0)
        e_end.append(np.abs(y_end - expm(M * h) @ y0).max())
        assert np.allclose(oracle.dp5_linear_dense(M, y0, h, 0.0), y0, atol=1e-15)
    # at th = 1 the extension is the 5th-order solution: local error O(h^6)
    assert 45 < e_end[0] / e_end[1] < 90, e_end
    # local error of the continuous extension at th = 0.4 is O(h^5)
    errs = []
    for h in [0.4, 0.2, 0.1]:
        yd = oracle.dp5_linear_dense(M, y0, h, 0.4)
        errs.append(np.abs(yd - expm(M * 0.4 * h) @ y0).max())
    ratio1, ratio2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 20 < ratio1 < 45 and 20 < ratio2 < 45, errs
