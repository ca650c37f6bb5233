"""Pins of the oracle's variable-coefficient problem (Sec. 3.8: div(nu grad u), expanded
as nu Lap u + grad nu . grad u, the operator written as per-point terms).

- nu and its gradient equal the closed form written here, and grad nu matches central
  differences of the oracle's nu;
- the source equals div(nu grad u*) computed in flux form by nested central differences
  (nu times the difference gradient of u*, then the difference divergence), which shares
  no step with the expanded form the oracle evaluates;
- the per-point assembly (coef_pt) of the expanded operator, solved by the oracle's least
  squares, recovers u* on a test set.
"""
import math

import numpy as np

import oracle
from paper_2602_10541_gb300 import workloads as wl


def _u_star(x):
    return np.sin(np.pi * x[:, 0]) * np.sin(2 * np.pi * x[:, 1]) + x[:, 0] * x[:, 1]


def test_coefficient_fields():
    w = wl.varcoef2d(n_int=200, n_bc=8, n_feat=8, a=0.7)
    x = w.x_int
    nu = oracle.problem_coef(w.problem, -1, x, w.params)
    np.testing.assert_allclose(nu, 1 + 0.7 * (x[:, 0] ** 2 + 0.5 * x[:, 1] ** 2), rtol=0, atol=1e-15)
    h = 1e-5
    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        fd = (oracle.problem_coef(w.problem, -1, x + e, w.params)
              - oracle.problem_coef(w.problem, -1, x - e, w.params)) / (2 * h)
        np.testing.assert_allclose(oracle.problem_coef(w.problem, k, x, w.params), fd, rtol=0, atol=1e-9)
    np.testing.assert_allclose(oracle.problem_exact(w.problem, x, w.params), _u_star(x), rtol=0, atol=1e-15)


def test_source_is_the_divergence_of_the_flux():
    w = wl.varcoef2d(n_int=300, n_bc=8, n_feat=8, a=1.0)
    x = w.x_int
    h = 1e-4

    def flux(y):
        nu = oracle.problem_coef(w.problem, -1, y, w.params)
        g = np.zeros_like(y)
        for k in range(2):
            e = np.zeros(2)
            e[k] = h
            g[:, k] = (_u_star(y + e) - _u_star(y - e)) / (2 * h)
        return nu[:, None] * g

    div = np.zeros(len(x))
    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        div += (flux(x + e)[:, k] - flux(x - e)[:, k]) / (2 * h)
    f = oracle.problem_source(w.problem, x, w.params)
    assert np.abs(f - div).max() <= 1e-5 * np.abs(f).max()


def _varcoef_operator(w, x):
    nu = oracle.problem_coef(w.problem, -1, x, w.params)
    nux = oracle.problem_coef(w.problem, 0, x, w.params)
    nuy = oracle.problem_coef(w.problem, 1, x, w.params)
    alpha = [[2, 0], [0, 2], [1, 0], [0, 1]]
    coef_pt = np.stack([nu, nu, nux, nuy])          # [n_terms][n_rows]
    return oracle.assemble(x, alpha, np.zeros(4), w.W, w.b, w.scale, coef_pt=coef_pt)


def test_varcoef_solve_recovers_u_star():
    w = wl.varcoef2d(n_int=900, n_bc=200, n_feat=200)
    A = np.vstack([_varcoef_operator(w, w.x_int),
                   oracle.assemble(w.x_bc, [[0, 0]], [1.0], w.W, w.b, w.scale, row_weight=w.lam_bc)])
    rhs = np.concatenate([oracle.problem_source(w.problem, w.x_int, w.params),
                          w.lam_bc * oracle.problem_exact(w.problem, w.x_bc, w.params)])
    beta = oracle.lstsq(A, rhs)
    u = oracle.eval_u(w.x_test, w.W, w.b, w.scale, beta)
    ue = _u_star(w.x_test)
    err = np.linalg.norm(u - ue) / np.linalg.norm(ue)
    assert err < 1e-4, err
