"""Pins for the oracle's operator assembly (eq. cyclic, Corollary 1).

Every expected value here is computed independently of the oracle: numpy's sin
and cos of closed forms, or central finite differences of the bare feature
sin(W.x + b) written in this file.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2602_10541_gb300 import workloads as wl

rng = np.random.default_rng(12345)


def _setup(d, n_rows=7, n_feat=5, sigma=1.5):
    x = rng.random((n_rows, d))
    W = sigma * rng.standard_normal((n_feat, d))
    b = rng.uniform(0, 2 * math.pi, n_feat)
    return x, W, b


@pytest.mark.parametrize("d", [1, 2, 3, 5])
def test_laplacian_closed_form(d):
    # Corollary 1: Lap phi_j = -|W_j|^2 sin(W_j.x + b_j)
    x, W, b = _setup(d)
    alpha = 2 * np.eye(d, dtype=np.int32)
    A = oracle.assemble(x, alpha, np.ones(d), W, b, scale=0.7)
    z = x @ W.T + b
    ref = 0.7 * (-(W ** 2).sum(1))[None, :] * np.sin(z)
    np.testing.assert_allclose(A, ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_biharmonic_closed_form(d):
    # Corollary 1: Lap^2 phi_j = |W_j|^4 sin z, the operator sum_{k,l} d^2_k d^2_l
    x, W, b = _setup(d)
    alpha = np.array([2 * (np.eye(d, dtype=int)[k] + np.eye(d, dtype=int)[l])
                      for k in range(d) for l in range(d)], np.int32)
    A = oracle.assemble(x, alpha, np.ones(len(alpha)), W, b, scale=1.0)
    ref = ((W ** 2).sum(1) ** 2)[None, :] * np.sin(x @ W.T + b)
    np.testing.assert_allclose(A, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("d", [1, 2, 4])
def test_advection_closed_form(d):
    # Corollary 1: v . grad phi_j = (v . W_j) cos z
    x, W, b = _setup(d)
    v = rng.standard_normal(d)
    A = oracle.assemble(x, np.eye(d, dtype=np.int32), v, W, b, scale=1.0)
    ref = (W @ v)[None, :] * np.cos(x @ W.T + b)
    np.testing.assert_allclose(A, ref, rtol=1e-13, atol=1e-13)


def _fd_derivative(x, Wj, bj, alpha, h):
    """Central finite-difference D^alpha of sin(Wj.x + bj), one axis at a time
    (nested stencils: first derivative [-1, 0, 1]/2h, second [1, -2, 1]/h^2)."""
    d = len(alpha)
    stencils = []
    for k in range(d):
        a = alpha[k]
        if a == 0:
            stencils.append([(0, 1.0)])
        elif a == 1:
            stencils.append([(-1, -0.5 / h), (1, 0.5 / h)])
        elif a == 2:
            stencils.append([(-1, 1 / h ** 2), (0, -2 / h ** 2), (1, 1 / h ** 2)])
        elif a == 3:
            stencils.append([(-2, -0.5 / h ** 3), (-1, 1 / h ** 3), (1, -1 / h ** 3),
                             (2, 0.5 / h ** 3)])
        else:
            raise ValueError
    acc = 0.0
    for combo in itertools.product(*stencils):
        shift = np.array([c[0] for c in combo], float) * h
        w = np.prod([c[1] for c in combo])
        acc += w * math.sin(float(Wj @ (x + shift)) + bj)
    return acc


@pytest.mark.parametrize("alpha", [(1, 0), (0, 1), (2, 0), (1, 1), (2, 1), (3, 0),
                                   (1, 2), (0, 3), (2, 2), (1, 1, 1), (2, 0, 1)])
def test_single_term_matches_finite_differences(alpha):
    d = len(alpha)
    x, W, b = _setup(d, n_rows=3, n_feat=3, sigma=0.8)
    A = oracle.assemble(x, np.array([alpha], np.int32), [1.0], W, b, scale=1.0)
    order = sum(alpha)
    # Richardson on the O(h^2) stencils
    for i in range(3):
        for j in range(3):
            h = 2e-2
            f1 = _fd_derivative(x[i], W[j], b[j], alpha, h)
            f2 = _fd_derivative(x[i], W[j], b[j], alpha, h / 2)
            fd = (4 * f2 - f1) / 3
            assert abs(A[i, j] - fd) <= 1e-6 * (1 + np.abs(W[j]).max() ** order), (i, j)


def test_zero_weights_special_case():
    # W = 0: every derivative term vanishes, A = scale * c_0 * sin(b_j)
    d = 2
    x, _, b = _setup(d)
    W = np.zeros((5, d))
    alpha = np.array([[0, 0], [2, 0], [1, 1]], np.int32)
    A = oracle.assemble(x, alpha, [3.0, 5.0, 7.0], W, b, scale=0.5, row_weight=2.0)
    np.testing.assert_allclose(A, np.broadcast_to(2.0 * 0.5 * 3.0 * np.sin(b), A.shape),
                               rtol=1e-15)


def test_cyclic_table_one_dimension():
    # d = 1, W = 1: D^n sin(x + b) runs through sin, cos, -sin, -cos (period 4)
    x = np.array([[0.3], [1.1]])
    b = np.array([0.2])
    z = x[:, 0] + 0.2
    table = [np.sin(z), np.cos(z), -np.sin(z), -np.cos(z)]
    for n in range(9):
        A = oracle.assemble(x, np.array([[n]], np.int32), [1.0], np.ones((1, 1)), b, 1.0)
        np.testing.assert_allclose(A[:, 0], table[n % 4], rtol=0, atol=1e-15)


def test_per_point_coefficient_adds_to_term():
    d = 2
    x, W, b = _setup(d)
    alpha = np.array([[2, 0], [0, 2], [0, 0]], np.int32)
    c_i = rng.standard_normal(x.shape[0])
    cpt = np.zeros((3, x.shape[0]))
    cpt[2] = c_i
    A = oracle.assemble(x, alpha, [1.0, 1.0, 0.0], W, b, 0.3, coef_pt=cpt)
    ref = 0.3 * (-(W ** 2).sum(1)[None, :] + c_i[:, None]) * np.sin(x @ W.T + b)
    np.testing.assert_allclose(A, ref, rtol=1e-13, atol=1e-13)


def test_eval_u_matches_definition():
    x, W, b = _setup(3)
    beta = rng.standard_normal(5)
    u = oracle.eval_u(x, W, b, 0.25, beta)
    np.testing.assert_allclose(u, 0.25 * np.sin(x @ W.T + b) @ beta, rtol=1e-13)


def test_eval_u_agrees_with_the_identity_operator_and_central_differences():
    """u = sum_j beta_j scale sin(W_j . x + b_j) evaluated by eval_u equals the identity
    operator's assembled rows times beta (a separate code path, pinned by the closed
    forms above), and central differences of eval_u in x (h = 1e-4, error O(h^2))
    reproduce the assembled Laplacian rows times beta: a wrong scale, sign or argument
    in eval_u fails one of the two."""
    d = 3
    x, W, b = _setup(d)
    beta = rng.standard_normal(W.shape[0])
    u = oracle.eval_u(x, W, b, 0.25, beta)
    A_id = oracle.assemble(x, np.zeros((1, d), np.int32), [1.0], W, b, 0.25)
    np.testing.assert_allclose(u, A_id @ beta, rtol=1e-12, atol=1e-14)
    h = 1e-4
    lap_fd = np.zeros(x.shape[0])
    for k in range(d):
        e = np.zeros(d)
        e[k] = h
        lap_fd += (oracle.eval_u(x + e, W, b, 0.25, beta) - 2 * u + oracle.eval_u(x - e, W, b, 0.25, beta)) / h ** 2
    A_lap = oracle.assemble(x, (2 * np.eye(d, dtype=np.int32)), [1.0] * d, W, b, 0.25)
    ref = A_lap @ beta
    assert np.abs(lap_fd - ref).max() <= 1e-5 * np.abs(ref).max() + 1e-9


def test_workload_generators_are_deterministic_and_shaped():
    a = wl.helmholtz2d(n_int=64, n_bc=16, n_feat=8)
    c = wl.helmholtz2d(n_int=64, n_bc=16, n_feat=8)
    np.testing.assert_array_equal(a.W, c.W)
    np.testing.assert_array_equal(a.x_int, c.x_int)
    assert a.x_bc.shape == (16, 2)
    # each boundary point lies on an edge of the unit square
    on_edge = np.isclose(a.x_bc, 0) | np.isclose(a.x_bc, 1)
    assert on_edge.any(axis=1).all()
    u = wl.uniform(1, "s", 200000)
    assert 0.49 < u.mean() < 0.51 and u.min() >= 0 and u.max() < 1
    g = wl.normal(1, "n", 200000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1) < 0.01
