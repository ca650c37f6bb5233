"""Pins for the oracle's Newton-Raphson (Sec. 2.4) and adjoint (Sec. 2.5, 4.4).

Bratu has no closed form: the oracle's Newton solution is compared with an
independent second-order finite-difference Newton solve (5-point Laplacian,
sparse direct solves, one Richardson step between grids h and h/2).  The adjoint
gradients are compared with central finite differences (h = 1e-6) of the loss
through the oracle's forward map.
"""
import math

import numpy as np
import pytest
import oracle
from paper_2602_10541_gb300 import workloads as wl
from tests.golden import bratu as golden_bratu


@pytest.fixture(scope="module")
def bratu_reference():
    return golden_bratu.bratu_reference(128)


def test_bratu_reference_center_value(bratu_reference):
    # the classical lambda = 1 Bratu solution peaks near 0.0784 at the centre
    c = float(bratu_reference([[0.5, 0.5]])[0])
    assert 0.078 < c < 0.079


def test_newton_bratu_matches_finite_differences(bratu_reference):
    w = wl.bratu2d(n_int=1200, n_bc=256, n_feat=320)
    w.W = w.W * (2.0 / 6.0)          # the paper's Bratu bandwidth sigma = 2 suits this small N
    f = np.zeros(w.n_int)
    g = np.zeros(w.n_bc)
    beta, status, iters, hist = oracle.newton(w.x_int, w.x_bc, w.alpha, w.coef, oracle.NL_EXP,
                                              1.0, w.lam_bc, f, g, w.W, w.b, w.scale,
                                              mu=1e-10, max_iter=15, tol=1e-10)
    # 320 features cannot zero the residual at 1456 rows: after the first steps the
    # iteration sits on the approximation floor (the plateau of Sec. 3.3), so it
    # may stop on max_iter (1) as well as on the step test (0) or line search (2)
    assert status in (0, 1, 2), status
    assert iters <= 15
    # residual falls by orders of magnitude in the first iteration (Sec. 3.3)
    assert hist[1] < 1e-2 * hist[0]
    assert np.all(np.diff(hist) <= 0)          # Armijo: never increases
    xt = w.x_test
    u = oracle.eval_u(xt, w.W, w.b, w.scale, beta)
    ref = bratu_reference(xt)
    err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    assert err < 2e-3, err
    uc = oracle.eval_u([[0.5, 0.5]], w.W, w.b, w.scale, beta)[0]
    assert abs(uc - float(bratu_reference([[0.5, 0.5]])[0])) < 2e-4


def test_newton_on_linear_problem_is_one_regularised_solve():
    w = wl.helmholtz2d(n_int=400, n_bc=80, n_feat=60)
    f = oracle.problem_source(w.problem, w.x_int, w.params)
    g = oracle.problem_exact(w.problem, w.x_bc, w.params)
    beta, status, iters, hist = oracle.newton(w.x_int, w.x_bc, w.alpha, w.coef, oracle.NL_NONE,
                                              0.0, w.lam_bc, f, g, w.W, w.b, w.scale,
                                              mu=1e-8, max_iter=1, tol=0.0)
    A_int = oracle.assemble(w.x_int, w.alpha, w.coef, w.W, w.b, w.scale)
    A_bc = oracle.assemble(w.x_bc, np.zeros((1, 2), np.int32), [1.0], w.W, w.b, w.scale,
                           row_weight=w.lam_bc)
    A = np.vstack([A_int, A_bc])
    rhs = np.concatenate([f, w.lam_bc * g])
    ref = np.linalg.solve(A.T @ A + 1e-8 * np.eye(w.n_feat), A.T @ rhs)
    np.testing.assert_allclose(beta, ref, rtol=1e-7, atol=1e-7 * np.abs(ref).max())


def _inverse_setup(n_int=300, n_bc=48, n_feat=80, sigma=4.0):
    w = wl.inverse_instance(0, n_int=n_int, n_feat=n_feat)
    w.W = w.W * (sigma / 8.0)
    x_bc = w.x_bc[:n_bc]
    A_int = oracle.assemble(w.x_int, w.alpha, w.coef, w.W, w.b, w.scale)
    A_bc = oracle.assemble(x_bc, np.zeros((1, 2), np.int32), [1.0], w.W, w.b, w.scale,
                           row_weight=w.lam_bc)
    Hs = oracle.assemble(w.sensors, np.zeros((1, 2), np.int32), [1.0], w.W, w.b, w.scale)
    return w, x_bc, np.vstack([A_int, A_bc]), Hs


def _loss(A, Hs, x_int, n_bc, theta, y, mu):
    f = oracle.problem_source(oracle.GAUSS_SOURCE_2D, x_int, theta)
    rhs = np.concatenate([f, np.zeros(n_bc)])
    return oracle.inverse_adjoint(A, rhs, Hs, y, mu)


def test_adjoint_source_gradient_matches_central_differences():
    w, x_bc, A, Hs = _inverse_setup()
    mu = 1e-10
    y = _loss(A, Hs, w.x_int, len(x_bc), w.params, np.zeros(64), mu)["u_s"] + w.noise
    out = _loss(A, Hs, w.x_int, len(x_bc), w.theta0, y, mu)
    grad = oracle.gauss_source_grad(w.x_int, w.theta0, out["grad_rhs"][: w.n_int])
    # v solves the regularised normal equations (A^T A + mu I) v = grad_beta
    gb = Hs.T @ (2 * (out["u_s"] - y) / 64)
    np.testing.assert_allclose((A.T @ A + mu * np.eye(A.shape[1])) @ out["v"], gb,
                               rtol=1e-6, atol=1e-9 * np.abs(gb).max())
    h = 1e-6
    for q in range(16):
        tp, tm = w.theta0.copy(), w.theta0.copy()
        tp[q] += h
        tm[q] -= h
        fd = (_loss(A, Hs, w.x_int, len(x_bc), tp, y, mu)["loss"]
              - _loss(A, Hs, w.x_int, len(x_bc), tm, y, mu)["loss"]) / (2 * h)
        assert abs(grad[q] - fd) <= 2e-5 * np.abs(grad).max(), (q, grad[q], fd)


def test_adjoint_coefficient_gradient_matches_central_differences():
    w, x_bc, A, Hs = _inverse_setup(n_int=200, n_bc=40, n_feat=30, sigma=3.0)
    mu = 1e-8
    f = oracle.problem_source(oracle.GAUSS_SOURCE_2D, w.x_int, w.theta0)
    rhs = np.concatenate([f, np.zeros(len(x_bc))])
    y = np.linspace(-0.1, 0.1, 64)
    out = oracle.inverse_adjoint(A, rhs, Hs, y, mu)
    Av = A @ out["v"]
    n_int = w.n_int
    for t in range(2):
        g = oracle.term_coef_grad(w.x_int, w.alpha[t], w.W, w.b, w.scale, out["resid"][:n_int],
                                  Av[:n_int], out["v"], out["beta"])
        h = 1e-6
        losses = []
        for sgn in (1, -1):
            coef = w.coef.copy()
            coef[t] += sgn * h
            Ai = oracle.assemble(w.x_int, w.alpha, coef, w.W, w.b, w.scale)
            Ap = np.vstack([Ai, A[n_int:]])
            losses.append(oracle.inverse_adjoint(Ap, rhs, Hs, y, mu)["loss"])
        fd = (losses[0] - losses[1]) / (2 * h)
        assert abs(g - fd) <= 1e-5 * (abs(fd) + 1e-12), (t, g, fd)


def _u_star(x):
    """u* = sin(pi x) sin(pi y) + x y / 2 of the cubic problems, written out here."""
    return np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) + 0.5 * x[:, 0] * x[:, 1]


@pytest.mark.parametrize("name", ["nlpoisson2d", "nlhelmholtz2d"])
def test_cubic_sources_match_the_operator_on_u_star(name):
    """f of the cubic problems = L[u*] + lam u*^3, with L[u*] by central differences
    of the closed form (h = 1e-4, error O(h^2))."""
    w = getattr(wl, name)(n_int=200, n_bc=8, n_feat=8)
    x = w.x_int
    h = 1e-4
    lap = np.zeros(len(x))
    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        lap += (_u_star(x + e) - 2 * _u_star(x) + _u_star(x - e)) / h ** 2
    u = _u_star(x)
    lam = w.nl_lam
    ref = (-lap + lam * u ** 3) if name == "nlpoisson2d" else (lap + 9.0 * u + lam * u ** 3)
    f = oracle.problem_source(w.problem, x, w.params)
    np.testing.assert_allclose(f, ref, rtol=0, atol=1e-5 * np.abs(ref).max())
    np.testing.assert_allclose(oracle.problem_exact(w.problem, w.x_bc, w.params), _u_star(w.x_bc),
                               rtol=0, atol=1e-15)


@pytest.mark.parametrize("name", ["nlpoisson2d", "nlhelmholtz2d"])
def test_newton_cubic_recovers_the_manufactured_solution(name):
    """Newton from beta = 0 on the cubic problems (Sec. 3.3, mu = 1e-10, backtracking)
    converges, and u agrees with u* on the test set to the basis' accuracy."""
    w = getattr(wl, name)(n_int=1200, n_bc=256, n_feat=320)
    f = oracle.problem_source(w.problem, w.x_int, w.params)
    g = _u_star(w.x_bc)
    beta, status, iters, hist = oracle.newton(w.x_int, w.x_bc, w.alpha, w.coef, oracle.NL_CUBIC, w.nl_lam,
                                              w.lam_bc, f, g, w.W, w.b, w.scale, mu=w.mu, max_iter=20,
                                              tol=1e-10)
    assert hist[-1] < 1e-3 * hist[0]
    u = oracle.eval_u(w.x_test, w.W, w.b, w.scale, beta)
    ue = _u_star(w.x_test)
    err = np.linalg.norm(u - ue) / np.linalg.norm(ue)
    assert err < 1e-6, (status, iters, err)


# ---------------------------------------------------------------------------
# The 1-D Newton problems of Sec. 3.3 (Allen-Cahn eps = 0.1, steady Burgers nu = 0.1)
# in true solver mode: f = 0 and the Dirichlet data of a kink that solves each
# equation exactly, written out here: tanh(s/sqrt(2 eps)) and -tanh(s/(2 nu)).
# ---------------------------------------------------------------------------

def _kink(name, x, c):
    s = x[:, 0] - 0.5
    return np.tanh(s / math.sqrt(2 * c)) if name == "allen_cahn1d" else -np.tanh(s / (2 * c))


@pytest.mark.parametrize("name,c", [("allen_cahn1d", 0.1), ("allen_cahn1d", 0.03),
                                    ("burgers1d", 0.1), ("burgers1d", 0.5)])
def test_1d_kinks_solve_their_equations(name, c):
    """The oracle's u* of problems 8 and 9 equals the kink and zeroes the equation:
    eps u'' + u - u^3 (Allen-Cahn) and u u' - nu u'' (Burgers) by central differences
    of the oracle's own u* (h = 1e-4), and the source is 0."""
    w = getattr(wl, name)(n_int=300, n_feat=4)
    x = w.x_int
    prob = w.problem
    u = lambda y: oracle.problem_exact(prob, y, [c])
    np.testing.assert_allclose(u(x), _kink(name, x, c), rtol=0, atol=1e-15)
    h = 1e-4
    e = np.array([[h]])
    up, u0, um = u(x + e), u(x), u(x - e)
    d1 = (up - um) / (2 * h)
    d2 = (up - 2 * u0 + um) / h ** 2
    res = (c * d2 + u0 - u0 ** 3) if name == "allen_cahn1d" else (u0 * d1 - c * d2)
    scale = np.abs(c * d2).max()
    assert np.abs(res).max() < 1e-5 * scale
    np.testing.assert_array_equal(oracle.problem_source(prob, x, [c]), np.zeros(len(x)))


def _solve_1d(w, stages, iters, warm=True):
    f = np.zeros(w.n_int)
    g = oracle.problem_exact(w.problem, w.x_bc, w.params)
    beta = None
    if warm:   # warm start: the linear part alone (one Newton step with N = 0 is that solve)
        beta, *_ = oracle.newton(w.x_int, w.x_bc, w.alpha, stages[0], oracle.NL_NONE, 0.0,
                                 w.lam_bc, f, g, w.W, w.b, w.scale, mu=w.mu, max_iter=1, tol=0.0)
    hists = []
    for coef in stages:
        beta, status, iters_done, hist = oracle.newton(w.x_int, w.x_bc, w.alpha, coef, w.nl_kind,
                                                       w.nl_lam, w.lam_bc, f, g, w.W, w.b, w.scale,
                                                       mu=w.mu, max_iter=iters, tol=1e-12, beta0=beta)
        hists.append(hist)
    return beta, hists


def test_newton_allen_cahn_recovers_the_kink():
    """Newton (warm start, mu = 1e-10, backtracking) on eps u'' + u - u^3 = 0 converges to
    the kink; with the cubic's Jacobian term 3 lam u^2 the residual drops by orders of
    magnitude per step once close (a wrong Jacobian stalls to linear convergence)."""
    w = wl.allen_cahn1d(n_int=600, n_feat=300)
    beta, (hist,) = _solve_1d(w, [w.coef], 25)
    assert np.all(np.diff(hist) <= 0)
    assert hist[2] < 1e-3 * hist[0], hist       # two quadratic steps reach the floor
    u = oracle.eval_u(w.x_test, w.W, w.b, w.scale, beta)
    ue = _kink("allen_cahn1d", w.x_test, 0.1)
    err = np.linalg.norm(u - ue) / np.linalg.norm(ue)
    assert err < 2e-5, err


def test_newton_burgers_jacobian_converges_quadratically():
    """At nu = 1 the Burgers step with J = -nu phi'' + u' phi + u phi' (both per-point
    terms) reaches the approximation floor within two steps from the linear warm
    start: each accepted step squares the error.  Dropping either term of the
    Jacobian or flipping its sign leaves a contraction far slower than that."""
    w = wl.burgers1d(n_int=600, n_feat=300)
    _, (hist,) = _solve_1d(w, [np.array([-1.0])], 3)
    assert hist[2] < 1e-6 * hist[0], hist


def test_newton_burgers_continuation_recovers_the_shock():
    """Continuation nu = 1, 0.5, 0.2, 0.1 (Sec. 2.4), each stage warm-started from the
    previous one, ends at the viscous shock -tanh((x - 1/2)/(2 nu))."""
    w = wl.burgers1d(n_int=600, n_feat=300)
    beta, hists = _solve_1d(w, list(wl.burgers_stage_coef(0.1)), 12)
    for h in hists:
        assert np.all(np.diff(h) <= 0)
    u = oracle.eval_u(w.x_test, w.W, w.b, w.scale, beta)
    ue = _kink("burgers1d", w.x_test, 0.1)
    err = np.linalg.norm(u - ue) / np.linalg.norm(ue)
    assert err < 1e-4, err
