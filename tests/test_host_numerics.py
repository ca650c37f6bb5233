"""Host-side checks of two numerical facts the GPU path relies on (no GPU):

* the thin-Q reading of the batched inverse evaluation: for y = [s; 0; 0] (zero past the
  interior rows), the first n entries of Q^T y equal Qi^T s, and the interior rows of
  Q [w; 0] equal Qi w, Qi being the interior rows of Q's first n columns;
* the error-free transformations of the double-float arithmetic (csrc/dfloat.cuh), done
  here in IEEE binary32 with round-to-nearest (numpy float32), are exact: two-sum,
  fast two-sum and the FMA product error leave no rounding, checked in exact rationals.
"""
from fractions import Fraction

import numpy as np


def test_thin_q_identities_of_the_inverse_evaluation():
    rng = np.random.default_rng(5)
    n_int, n_bc, n = 60, 12, 25
    mu = 1e-3
    A = rng.standard_normal((n_int + n_bc, n))
    Aug = np.vstack([A, np.sqrt(mu) * np.eye(n)])
    Q, R = np.linalg.qr(Aug, mode="complete")
    Qi = Q[:n_int, :n]
    s = rng.standard_normal(n_int)
    y = np.concatenate([s, np.zeros(n_bc + n)])
    np.testing.assert_allclose((Q.T @ y)[:n], Qi.T @ s, rtol=1e-12, atol=1e-13)
    w = rng.standard_normal(n)
    z = Q @ np.concatenate([w, np.zeros(n_int + n_bc)])
    np.testing.assert_allclose(z[:n_int], Qi @ w, rtol=1e-12, atol=1e-13)
    # and the evaluation's beta through Qi equals the regularised least-squares solution
    beta = np.linalg.solve(R[:n, :n], Qi.T @ s)
    rhs = np.concatenate([s, np.zeros(n_bc)])
    ref = np.linalg.solve(A.T @ A + mu * np.eye(n), A.T @ rhs)
    np.testing.assert_allclose(beta, ref, rtol=1e-9, atol=1e-11)


def _two_sum(a, b):
    s = np.float32(a + b)
    bb = np.float32(s - a)
    e = np.float32(np.float32(a - np.float32(s - bb)) + np.float32(b - bb))
    return s, e


def _fast_two_sum(a, b):
    s = np.float32(a + b)
    return s, np.float32(b - np.float32(s - a))


def _fma32(a, b, c):
    # a * b + c rounded once to binary32 (the exact value fits a double here)
    return np.float32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def test_double_float_error_free_transformations_are_exact():
    rng = np.random.default_rng(7)
    for _ in range(2000):
        a, b = np.float32(rng.standard_normal() * 10.0 ** rng.integers(-8, 8)), \
            np.float32(rng.standard_normal() * 10.0 ** rng.integers(-8, 8))
        s, e = _two_sum(a, b)
        assert Fraction(float(s)) + Fraction(float(e)) == Fraction(float(a)) + Fraction(float(b))
        hi, lo = (a, b) if abs(a) >= abs(b) else (b, a)
        s, e = _fast_two_sum(hi, lo)
        assert Fraction(float(s)) + Fraction(float(e)) == Fraction(float(hi)) + Fraction(float(lo))
        p = np.float32(a * b)
        e = _fma32(a, b, -p)
        assert Fraction(float(p)) + Fraction(float(e)) == Fraction(float(a)) * Fraction(float(b))
