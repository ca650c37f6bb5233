"""Pins for the oracle's Householder least squares (Sec. 2.3, "via QR or SVD").

QR is checked by rebuilding Q from the stored reflectors in plain numpy; the
solve is checked against LAPACK (numpy.linalg.lstsq), against the regularised
normal equations solved by numpy.linalg.solve, and on consistent systems.
"""
import numpy as np
import pytest

import oracle

rng = np.random.default_rng(7)


def _q_from_reflectors(packed, tau):
    m, n = packed.shape
    Q = np.eye(m)
    for j in range(n):
        v = np.zeros(m)
        v[j] = 1.0
        v[j + 1:] = packed[j + 1:, j]
        H = np.eye(m) - tau[j] * np.outer(v, v)
        Q = Q @ H
    return Q


@pytest.mark.parametrize("m,n", [(12, 5), (40, 17), (9, 9)])
def test_qr_reconstructs_and_is_orthogonal(m, n):
    A = rng.standard_normal((m, n))
    packed, tau = oracle.qr(A)
    Q = _q_from_reflectors(packed, tau)
    R = np.triu(packed[:n, :])
    np.testing.assert_allclose(Q.T @ Q, np.eye(m), atol=1e-13)
    np.testing.assert_allclose(Q[:, :n] @ R, A, atol=1e-12)
    # LAPACK sign convention: R_jj has the opposite sign of the pivot it replaced
    assert np.all(np.abs(np.diag(R)) > 0)


def test_qr_column_already_reduced_gives_identity_reflector():
    A = np.zeros((6, 3))
    A[0, 0] = 2.0
    A[:, 1] = rng.standard_normal(6)
    A[:, 2] = rng.standard_normal(6)
    packed, tau = oracle.qr(A)
    assert tau[0] == 0.0
    np.testing.assert_allclose(np.abs(np.diag(packed[:3])), np.abs(np.linalg.qr(A)[1].diagonal()),
                               rtol=1e-13)


@pytest.mark.parametrize("m,n,nrhs", [(12, 5, 1), (30, 11, 3), (64, 20, 2)])
def test_lstsq_matches_lapack(m, n, nrhs):
    A = rng.standard_normal((m, n))
    B = rng.standard_normal((m, nrhs))
    ref = np.linalg.lstsq(A, B, rcond=None)[0]
    got = oracle.lstsq(A, B)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_lstsq_regularised_matches_normal_equations():
    m, n, mu = 25, 9, 0.3
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    ref = np.linalg.solve(A.T @ A + mu * np.eye(n), A.T @ b)
    got = oracle.lstsq(A, b, mu=mu)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_lstsq_long_double_normal_equations_tiny():
    # brute force in extended precision on a small well-conditioned system
    m, n = 12, 5
    A = 0.5 * rng.standard_normal((m, n)) + np.eye(m, n) * 3
    b = rng.standard_normal(m)
    Al = A.astype(np.longdouble)
    G = Al.T @ Al
    rhs = Al.T @ b.astype(np.longdouble)
    # Gaussian elimination in long double (no pivoting needed: G is SPD)
    G = G.copy(); rhs = rhs.copy()
    for k in range(n):
        for i in range(k + 1, n):
            f = G[i, k] / G[k, k]
            G[i, k:] -= f * G[k, k:]
            rhs[i] -= f * rhs[k]
    x = np.zeros(n, dtype=np.longdouble)
    for i in range(n - 1, -1, -1):
        x[i] = (rhs[i] - G[i, i + 1:] @ x[i + 1:]) / G[i, i]
    got = oracle.lstsq(A, b)
    np.testing.assert_allclose(got, x.astype(np.float64), rtol=1e-13, atol=1e-13)


def test_consistent_system_recovers_coefficients():
    m, n = 50, 12
    A = rng.standard_normal((m, n))
    beta0 = rng.standard_normal(n)
    got = oracle.lstsq(A, A @ beta0)
    np.testing.assert_allclose(got, beta0, rtol=1e-12, atol=1e-12)


def test_apply_qt_and_backsolve_compose_to_lstsq():
    m, n = 20, 6
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    packed, tau = oracle.qr(A)
    y = oracle.apply_qt(packed, tau, b)
    x = oracle.backsolve(packed, y)
    np.testing.assert_allclose(x, np.linalg.lstsq(A, b, rcond=None)[0], rtol=1e-12)
    # the tail of Q^T b is the residual's norm
    np.testing.assert_allclose(np.linalg.norm(y[n:]), np.linalg.norm(A @ x - b), rtol=1e-12)
