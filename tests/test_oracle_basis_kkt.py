"""Pins of the oracle's basis and KKT pieces against the mathematics, not itself.

- Bernstein tables against scipy's BPoly (a library routine) and against
  partition of unity, endpoint interpolation and linear precision.
- Gauss-Jordan inverse and the KKT inverse against LAPACK (numpy.linalg).
- F^T F of the dense stacked F against its closed form n_o P^T P + Pd^T Pd + Pdd^T Pdd.
"""
import numpy as np
import pytest
from scipy.interpolate import BPoly

from oracle import am


@pytest.mark.parametrize("n_p,T", [(50, 5.0), (100, 10.0), (75, 7.5), (150, 20.0), (1000, 10.0)])
def test_bernstein_against_scipy_bpoly(n_p, T):
    P, Pd, Pdd = am.bernstein(n_p, T)
    t = np.linspace(0.0, T, n_p)
    for i in range(11):
        c = np.zeros((11, 1)); c[i, 0] = 1.0
        bp = BPoly(c, [0.0, T])
        np.testing.assert_allclose(P[:, i], bp(t), atol=1e-13)
        np.testing.assert_allclose(Pd[:, i], bp.derivative()(t), atol=1e-12)
        np.testing.assert_allclose(Pdd[:, i], bp.derivative(2)(t), atol=1e-11)


def test_bernstein_partition_endpoints_linear_precision():
    P, Pd, Pdd = am.bernstein(100, 10.0)
    np.testing.assert_allclose(P.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose(Pd.sum(1), 0.0, atol=1e-13)
    np.testing.assert_allclose(Pdd.sum(1), 0.0, atol=1e-13)
    np.testing.assert_array_equal(P[0], np.eye(11)[0])
    np.testing.assert_array_equal(P[-1], np.eye(11)[10])
    # linear coefficients -> exactly linear trajectory with constant velocity
    c = 2.0 + 3.0 * np.arange(11) / 10.0
    tau = np.linspace(0.0, 1.0, 100)
    np.testing.assert_allclose(P @ c, 2.0 + 3.0 * tau, atol=1e-13)
    np.testing.assert_allclose(Pd @ c, 3.0 / 10.0, atol=1e-12)
    np.testing.assert_allclose(Pdd @ c, 0.0, atol=1e-12)


def test_derivatives_central_differences():
    # a very fine grid: central differences of P reproduce Pd, of Pd reproduce Pdd
    n_p, T = 200001, 4.0
    P, Pd, Pdd = am.bernstein(n_p, T)
    h = T / (n_p - 1)
    k = np.arange(1000, n_p - 1000, 997)
    np.testing.assert_allclose((P[k + 1] - P[k - 1]) / (2 * h), Pd[k], atol=1e-8)
    np.testing.assert_allclose((Pd[k + 1] - Pd[k - 1]) / (2 * h), Pdd[k], atol=1e-7)


def test_gauss_jordan_against_lapack():
    rng = np.random.default_rng(3)
    for n in (3, 8, 15):
        A = rng.normal(size=(n, n)) + n * np.eye(n)
        np.testing.assert_allclose(am.invert(A), np.linalg.inv(A), rtol=1e-12, atol=1e-12)
    # needs pivoting: zero leading entry
    A = np.array([[0.0, 1.0, 2.0], [1.0, 0.0, 3.0], [4.0, -3.0, 8.0]])
    np.testing.assert_allclose(am.invert(A) @ A, np.eye(3), atol=1e-13)
    with pytest.raises(np.linalg.LinAlgError):
        am.invert(np.ones((4, 4)))


@pytest.mark.parametrize("cost_mode", [0, 1])
def test_kkt_structure_and_inverse(cost_mode):
    n_p, T, n_o, rho = 100, 10.0, 50, 1.0
    K, Ki = am.kkt(2, n_p, T, n_o, rho=rho, cost_mode=cost_mode)
    P, Pd, Pdd = am.bernstein(n_p, T)
    # F^T F of the stacked F equals the closed form (F never needs materialising)
    M = n_o * P.T @ P + Pd.T @ Pd + Pdd.T @ Pdd
    Q = (Pdd.T @ Pdd + P.T @ P) if cost_mode == 0 else np.eye(11)
    np.testing.assert_allclose(K[:11, :11], Q + rho * M, rtol=1e-12)
    A = np.stack([P[0], Pd[0], Pdd[0], P[-1]])
    np.testing.assert_array_equal(K[11:, :11], A)
    np.testing.assert_array_equal(K[:11, 11:], A.T)
    np.testing.assert_array_equal(K[11:, 11:], 0.0)
    # inverse against LAPACK's solve of the same system
    rhs = np.random.default_rng(0).normal(size=(15, 7))
    np.testing.assert_allclose(Ki @ rhs, np.linalg.solve(K, rhs), rtol=1e-9, atol=1e-12)
