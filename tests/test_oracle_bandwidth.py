"""Pins of the oracle's feature-weight gradient (learnable bandwidth, App. "Learnable
Bandwidth via Reparameterisation", Alg. 2) against finite differences.

1. The bilinear form F(W, b) = sum_ij w_ij A_ij(W, b) is differentiated by central
   differences of the oracle's assembled operator (itself pinned by closed forms),
   for operators of even, odd and mixed orders in d = 1, 2, 3.
2. The outer loss L(sigma) = ||A(sigma) beta*(sigma) - rhs||^2, with beta* the exact
   (regularised) least-squares solution, is differentiated by central differences in
   sigma (W = sigma W_hat) and in the entries of a lower-triangular L (W_j = L W_hat_j),
   with mu = 0 (envelope theorem) and mu > 0 (the extra adjoint term).
"""
import math

import numpy as np
import pytest

import oracle

OPS = [
    ("laplacian 2d", [[2, 0], [0, 2]], [1.0, 1.0]),
    ("advection + mixed 2d", [[1, 0], [1, 1], [0, 0]], [0.7, -1.3, 2.0]),
    ("biharmonic 1d + u", [[4], [0]], [1.0, 3.0]),
    ("d = 3 mixed orders", [[1, 0, 2], [0, 3, 0], [0, 0, 1]], [0.5, -0.25, 1.5]),
]


def _bilinear(x, alpha, coef, rw, W, b, scale, wts):
    A = oracle.assemble(x, alpha, coef, W, b, scale, row_weight=rw)
    return float(np.sum(wts * A))


@pytest.mark.parametrize("name,alpha,coef", OPS)
def test_weight_grad_is_the_derivative_of_the_bilinear_form(name, alpha, coef):
    d = len(alpha[0])
    rng = np.random.default_rng(7 + d)
    n, nf = 11, 6
    x = rng.random((n, d))
    W = 2.0 * rng.standard_normal((nf, d))
    b = 2 * math.pi * rng.random(nf)
    r, Av = rng.standard_normal(n), rng.standard_normal(n)
    beta, v = rng.standard_normal(nf), rng.standard_normal(nf)
    c_v, c_rb, c_av = 0.3, -2.0, 1.7
    rw, scale = 1.9, 1 / math.sqrt(nf)
    wts = np.outer(r, c_v * v + c_rb * beta) + c_av * np.outer(Av, beta)
    gW, gb = oracle.weight_grad(x, alpha, coef, rw, W, b, scale, r, beta, v=v, Av=Av,
                                c_v=c_v, c_rb=c_rb, c_av=c_av)
    h = 1e-6
    for j in range(nf):
        for k in range(d):
            Wp, Wm = W.copy(), W.copy()
            Wp[j, k] += h
            Wm[j, k] -= h
            fd = (_bilinear(x, alpha, coef, rw, Wp, b, scale, wts)
                  - _bilinear(x, alpha, coef, rw, Wm, b, scale, wts)) / (2 * h)
            assert abs(gW[j, k] - fd) <= 1e-7 * max(1.0, abs(fd)), (name, j, k, gW[j, k], fd)
        bp, bm = b.copy(), b.copy()
        bp[j] += h
        bm[j] -= h
        fd = (_bilinear(x, alpha, coef, rw, W, bp, scale, wts)
              - _bilinear(x, alpha, coef, rw, W, bm, scale, wts)) / (2 * h)
        assert abs(gb[j] - fd) <= 1e-7 * max(1.0, abs(fd)), (name, j, gb[j], fd)


def _problem(seed=3):
    """A small Helmholtz-like system: interior rows Lap + 16 on 48 points, boundary rows
    (weight 10) on 16 points of the unit square's edges, 14 features."""
    rng = np.random.default_rng(seed)
    x_int = rng.random((48, 2))
    t = rng.random(16)
    x_bc = np.stack([np.concatenate([t[:4], np.ones(4), t[8:12], np.zeros(4)]),
                     np.concatenate([np.zeros(4), t[4:8], np.ones(4), t[12:]])], axis=1)
    W_hat = rng.standard_normal((14, 2))
    b = 2 * math.pi * rng.random(14)
    rhs = np.concatenate([np.sin(3 * x_int[:, 0]) * np.cos(2 * x_int[:, 1]),
                          10.0 * (x_bc[:, 0] * x_bc[:, 1] + 0.5)])
    return x_int, x_bc, W_hat, b, rhs


ALPHA_INT, COEF_INT = [[2, 0], [0, 2], [0, 0]], [1.0, 1.0, 16.0]


def _outer_loss(W, x_int, x_bc, b, rhs, mu):
    scale = 1 / math.sqrt(W.shape[0])
    A = np.vstack([oracle.assemble(x_int, ALPHA_INT, COEF_INT, W, b, scale),
                   oracle.assemble(x_bc, [[0, 0]], [1.0], W, b, scale, row_weight=10.0)])
    beta = oracle.lstsq(A, rhs, mu)
    r = rhs - A @ beta
    return float(r @ r), A, beta, r


def _outer_grad_W(W, x_int, x_bc, b, rhs, mu):
    """dL/dW of the outer loss by the adjoint formula: weights (c_v, c_rb, c_av) =
    (-2 mu, -2, 2 mu) with v = (A^T A + mu I)^{-1} beta, summed over both row blocks."""
    L, A, beta, r = _outer_loss(W, x_int, x_bc, b, rhs, mu)
    n = W.shape[0]
    scale = 1 / math.sqrt(n)
    v = np.linalg.solve(A.T @ A + mu * np.eye(n), beta) if mu > 0 else None
    Av = A @ v if mu > 0 else None
    m_int = x_int.shape[0]
    gW = np.zeros_like(W)
    for rows, alpha, coef, rw in ((slice(0, m_int), ALPHA_INT, COEF_INT, 1.0),
                                  (slice(m_int, None), [[0, 0]], [1.0], 10.0)):
        xs = x_int if rows.start == 0 else x_bc
        g, _ = oracle.weight_grad(xs, alpha, coef, rw, W, b, scale, r[rows], beta,
                                  v=v, Av=None if Av is None else Av[rows],
                                  c_v=-2 * mu, c_rb=-2.0, c_av=2 * mu)
        gW += g
    return gW


@pytest.mark.parametrize("mu", [0.0, 1e-3])
def test_outer_loss_gradient_in_sigma(mu):
    """dL/dsigma = sum_jk dL/dW_jk W_hat_jk (W = sigma W_hat, eq. reparam_scalar)."""
    x_int, x_bc, W_hat, b, rhs = _problem()
    sigma = 2.0
    gW = _outer_grad_W(sigma * W_hat, x_int, x_bc, b, rhs, mu)
    g = float(np.sum(gW * W_hat))
    h = 1e-5
    fd = (_outer_loss((sigma + h) * W_hat, x_int, x_bc, b, rhs, mu)[0]
          - _outer_loss((sigma - h) * W_hat, x_int, x_bc, b, rhs, mu)[0]) / (2 * h)
    assert abs(g - fd) <= 1e-6 * max(abs(fd), 1e-3), (g, fd)


@pytest.mark.parametrize("mu", [0.0, 1e-3])
def test_outer_loss_gradient_in_cholesky_factor(mu):
    """dL/dL_ab = sum_j dL/dW_ja W_hat_jb for W_j = L W_hat_j (eq. reparam_cholesky)."""
    x_int, x_bc, W_hat, b, rhs = _problem(5)
    Lc = np.array([[2.0, 0.0], [0.7, 1.4]])
    gW = _outer_grad_W(W_hat @ Lc.T, x_int, x_bc, b, rhs, mu)
    G = gW.T @ W_hat
    h = 1e-6
    for a, c in ((0, 0), (1, 0), (1, 1)):
        Lp, Lm = Lc.copy(), Lc.copy()
        Lp[a, c] += h
        Lm[a, c] -= h
        fd = (_outer_loss(W_hat @ Lp.T, x_int, x_bc, b, rhs, mu)[0]
              - _outer_loss(W_hat @ Lm.T, x_int, x_bc, b, rhs, mu)[0]) / (2 * h)
        assert abs(G[a, c] - fd) <= 1e-6 * max(abs(fd), 1e-3), (a, c, G[a, c], fd)
