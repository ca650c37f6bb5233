"""Pins for the manufactured problems and end-to-end linear solves of the oracle.

f = L[u*] is checked by finite differences of u*; full solves are checked
against the exact solutions on an independent test set (Sec. 3.1 protocol) and
against the paper's printed error levels (tests/golden/paper_reported.txt).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2602_10541_gb300 import workloads as wl
from tests.golden.paper import reported

rng = np.random.default_rng(99)


def _fd_laplacian(fun, x, h=4e-3):
    """Five-point-per-axis second differences with one Richardson step (O(h^4))."""
    def lap(hh):
        n, d = x.shape
        out = np.zeros(n)
        for k in range(d):
            e = np.zeros(d)
            e[k] = hh
            out += (fun(x + e) - 2 * fun(x) + fun(x - e)) / hh ** 2
        return out
    return (4 * lap(h / 2) - lap(h)) / 3


@pytest.mark.parametrize("prob,d,params,op", [
    (oracle.POISSON_1D, 1, (), lambda lap, u: -lap),
    (oracle.HELMHOLTZ_2D, 2, (4.0,), lambda lap, u: lap + 16.0 * u),
    (oracle.POISSON_5D, 5, (), lambda lap, u: -lap),
])
def test_source_is_operator_of_exact_solution(prob, d, params, op):
    x = 0.1 + 0.8 * rng.random((50, d))
    ue = lambda y: oracle.problem_exact(prob, y, params)
    lap = _fd_laplacian(ue, x)
    f = oracle.problem_source(prob, x, params)
    np.testing.assert_allclose(f, op(lap, ue(x)), rtol=2e-5, atol=2e-4)


def test_exact_solution_special_values():
    # u*(1/4) = sin(pi/2) + 0.5 sin(3 pi/2) = 0.5 ; Helmholtz u*(1/2, 1/4) = 1 + 0.3 cos(7 pi / 4)
    np.testing.assert_allclose(oracle.problem_exact(oracle.POISSON_1D, [[0.25]]), [0.5], atol=1e-15)
    np.testing.assert_allclose(oracle.problem_exact(oracle.HELMHOLTZ_2D, [[0.5, 0.25]], (4.0,)),
                               [1.0 + 0.3 * math.cos(1.75 * math.pi)], atol=1e-15)
    x = np.full((1, 5), 0.5)
    np.testing.assert_allclose(oracle.problem_exact(oracle.POISSON_5D, x), [5.0 + 0.5 ** 5], atol=1e-14)
    # Dirichlet data vanish on the 1-D ends
    np.testing.assert_allclose(oracle.problem_exact(oracle.POISSON_1D, [[0.0], [1.0]]), 0, atol=1e-15)


def test_gauss_source_gradient_matches_finite_differences():
    x = rng.random((40, 2))
    theta = wl.gauss_theta(5, "t")
    w = rng.standard_normal(40)
    g = oracle.gauss_source_grad(x, theta, w)
    h = 1e-6
    for q in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[q] += h
        tm[q] -= h
        fd = (w @ oracle.problem_source(oracle.GAUSS_SOURCE_2D, x, tp)
              - w @ oracle.problem_source(oracle.GAUSS_SOURCE_2D, x, tm)) / (2 * h)
        assert abs(g[q] - fd) <= 1e-6 * (1 + abs(fd)), q


def _linear_system(w, bc_exact=True):
    A_int = oracle.assemble(w.x_int, w.alpha, w.coef, w.W, w.b, w.scale)
    A_bc = oracle.assemble(w.x_bc, np.zeros((1, w.d), np.int32), [1.0], w.W, w.b, w.scale,
                           row_weight=w.lam_bc)
    f = oracle.problem_source(w.problem, w.x_int, w.params)
    g = oracle.problem_exact(w.problem, w.x_bc, w.params) if bc_exact else np.zeros(w.n_bc)
    return np.vstack([A_int, A_bc]), np.concatenate([f, w.lam_bc * g])


def _rel_l2(w, beta):
    u = oracle.eval_u(w.x_test, w.W, w.b, w.scale, beta)
    ue = oracle.problem_exact(w.problem, w.x_test, w.params)
    return np.linalg.norm(u - ue) / np.linalg.norm(ue)


def test_poisson1d_full_size_solution_error():
    w = wl.poisson1d()
    A, rhs = _linear_system(w)
    beta = oracle.lstsq(A, rhs)
    err = _rel_l2(w, beta)
    assert err < 1e-6, err


def test_helmholtz2d_small_solution_error():
    w = wl.helmholtz2d(n_int=1536, n_bc=256, n_feat=384)
    A, rhs = _linear_system(w)
    beta = oracle.lstsq(A, rhs)
    err = _rel_l2(w, beta)
    assert err < reported()["helmholtz2d_rel_l2"], err


def test_poisson5d_small_solution_error():
    # 512 features resolve the 5-D solution only coarsely (LAPACK gives the same
    # level); the error falls with size (4.2e-6 at 32768+4096 rows x 4096 features)
    w = wl.poisson5d(n_int=2048, n_bc=512, n_feat=512)
    A, rhs = _linear_system(w)
    beta = oracle.lstsq(A, rhs)
    err = _rel_l2(w, beta)
    ref = np.linalg.lstsq(A, rhs, rcond=None)[0]
    assert err < 2e-2, err
    assert abs(err - _rel_l2(w, ref)) < 0.05 * err


def test_normalisation_keeps_coefficients_order_one():
    # Sec. 2.1 / ablation: with the 1/sqrt(N) scale the coefficients stay moderate,
    # without it they are sqrt(N) times larger for the same fit
    w = wl.helmholtz2d(n_int=512, n_bc=128, n_feat=128)
    A, rhs = _linear_system(w)
    beta = oracle.lstsq(A, rhs)
    beta_unscaled = oracle.lstsq(A / w.scale, rhs)
    np.testing.assert_allclose(beta_unscaled * math.sqrt(w.n_feat), beta, rtol=1e-6, atol=1e-6)
