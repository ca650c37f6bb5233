"""Seeded synthetic workloads shaped like the paper's PDE problems.

This module only draws numbers: collocation points, frozen features W and b,
test points, source parameters and sensor noise.  It holds none of the method's
arithmetic (no features, no operators, no solves), so the CPU oracle and the GPU
path can both take their inputs from it.

Random streams are counter based: the i-th draw of a named stream is
SplitMix64(key + (i + 1) * 0x9E3779B97F4A7C15) with key derived from the
workload seed and the stream's name, and normals come from the Box-Muller
transform of two uniform streams.  Every array is therefore reproducible on its
own, independent of the sizes of the others.

Frozen features follow Sec. 2.1 (W_j ~ N(0, sigma^2 I_d), b_j ~ U(0, 2 pi));
collocation follows Alg. 1 (interior points in the domain, boundary points on
its faces); errors are measured on an independent test set of 5000 points
drawn with a different seed (Sec. 3.1).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, name: str) -> np.uint64:
    h = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    for ch in name.encode():
        with np.errstate(over="ignore"):
            h = _mix(h ^ np.uint64(ch) ^ (np.uint64(len(name)) << np.uint64(56)))
    return np.uint64(h)


def uniform(seed: int, name: str, n: int) -> np.ndarray:
    """n uniforms in [0, 1) from the named counter-based stream."""
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix(_key(seed, name) + i * _GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, name: str, n: int) -> np.ndarray:
    """n standard normals (Box-Muller on two uniform streams)."""
    u1 = 1.0 - uniform(seed, name + "/u1", n)      # (0, 1]
    u2 = uniform(seed, name + "/u2", n)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def box_boundary(seed: int, name: str, n: int, d: int, per_face: bool) -> np.ndarray:
    """Points on the faces of [0,1]^d.  per_face=True: n/(2d) points on each face in
    the order (x_0=0, x_0=1, x_1=0, x_1=1, ...) except for d == 2 where the faces
    go y=0, x=1, y=1, x=0 (the edges walked in turn).  per_face=False: each point
    picks its face uniformly among the 2d faces, face f meaning x_{f//2} = f%2."""
    x = uniform(seed, name + "/pos", n * d).reshape(n, d)
    if per_face:
        faces = np.repeat(np.arange(2 * d), n // (2 * d))
        faces = np.concatenate([faces, np.arange(n - faces.size) % (2 * d)])
        if d == 2:
            walk = np.array([(1, 0), (0, 1), (1, 1), (0, 0)])   # (axis, value) per edge
            axis, val = walk[faces, 0], walk[faces, 1]
        else:
            axis, val = faces // 2, faces % 2
    else:
        faces = np.minimum((uniform(seed, name + "/face", n) * (2 * d)).astype(np.int64),
                           2 * d - 1)
        axis, val = faces // 2, faces % 2
    x[np.arange(n), axis] = val.astype(np.float64)
    return x


@dataclass
class Workload:
    """One linear or nonlinear PDE problem in the paper's form L[u] (+ N[u]) = f
    with Dirichlet rows B[u] = u = g weighted by lam_bc (eq. linear_system)."""
    name: str
    problem: int                    # problem id shared by the rhs kernels and the oracle
    d: int
    n_int: int
    n_bc: int
    n_feat: int
    sigma: float
    lam_bc: float
    alpha: np.ndarray               # [n_terms][d] multi-indices of the interior operator L
    coef: np.ndarray                # [n_terms] coefficients of L
    params: np.ndarray              # problem parameters (k for Helmholtz, theta for sources)
    seed: int
    mu: float = 0.0
    nl_kind: int = 0                # 0 none, 1 exp, 2 cubic, 3 Burgers (u u_x0)
    nl_lam: float = 0.0
    pp_alpha: np.ndarray = None     # [n_pp][d] per-point terms of L (variable coefficients)
    pp_kinds: tuple = None          # rhs kinds giving each per-point coefficient at x_int
    x_int: np.ndarray = field(default=None, repr=False)
    x_bc: np.ndarray = field(default=None, repr=False)
    W: np.ndarray = field(default=None, repr=False)
    b: np.ndarray = field(default=None, repr=False)
    x_test: np.ndarray = field(default=None, repr=False)

    @property
    def n_rows(self) -> int:
        return self.n_int + self.n_bc

    @property
    def scale(self) -> float:
        """1/sqrt(N) of eq. approximation (N = number of features)."""
        return 1.0 / math.sqrt(self.n_feat)


def _features(seed, n_feat, d, sigma):
    W = sigma * normal(seed, "W", n_feat * d).reshape(n_feat, d)
    b = 2.0 * math.pi * uniform(seed, "b", n_feat)
    return W, b


def _laplacian_terms(d, sign):
    alpha = 2 * np.eye(d, dtype=np.int32)
    return alpha, np.full(d, float(sign))


SEED0 = 20260210


def poisson1d(n_int=256, n_feat=128):
    """-u'' = f on [0,1], equispaced interior x_i = i/(n_int+1), both ends as
    boundary rows with weight 1; sigma = 10; FP64."""
    s = SEED0 + 1
    w = Workload("poisson1d", 1, 1, n_int, 2, n_feat, 10.0, 1.0,
                 np.array([[2]], np.int32), np.array([-1.0]), np.zeros(0), s)
    w.x_int = (np.arange(1, n_int + 1, dtype=np.float64) / (n_int + 1)).reshape(-1, 1)
    w.x_bc = np.array([[0.0], [1.0]])
    w.W, w.b = _features(s, n_feat, 1, w.sigma)
    w.x_test = uniform(s + 200, "test", 5000).reshape(-1, 1)
    return w


def helmholtz2d(n_int=8192, n_bc=1024, n_feat=2048, k=4.0, seed_offset=0):
    """Lap u + k^2 u = f on [0,1]^2, uniform-random interior, n_bc/4 uniform points per
    edge, sigma = 8, boundary weight 100."""
    s = SEED0 + 2 + seed_offset
    alpha = np.array([[2, 0], [0, 2], [0, 0]], np.int32)
    w = Workload("helmholtz2d", 2, 2, n_int, n_bc, n_feat, 8.0, 100.0, alpha,
                 np.array([1.0, 1.0, k * k]), np.array([k]), s)
    w.x_int = uniform(s + 100, "x_int", n_int * 2).reshape(n_int, 2)
    w.x_bc = box_boundary(s + 100, "x_bc", n_bc, 2, per_face=True)
    w.W, w.b = _features(s, n_feat, 2, w.sigma)
    w.x_test = uniform(s + 200, "test", 5000 * 2).reshape(-1, 2)
    return w


def poisson5d(n_int=32768, n_bc=4096, n_feat=4096, seed_offset=0):
    """-Lap u = f on [0,1]^5, uniform-random interior, boundary points on a face
    chosen uniformly among the 10, sigma = 3, boundary weight 100."""
    s = SEED0 + 3 + 1000 * seed_offset
    alpha, coef = _laplacian_terms(5, -1.0)
    w = Workload("poisson5d", 3, 5, n_int, n_bc, n_feat, 3.0, 100.0, alpha, coef,
                 np.zeros(0), s)
    w.x_int = uniform(s + 100, "x_int", n_int * 5).reshape(n_int, 5)
    w.x_bc = box_boundary(s + 100, "x_bc", n_bc, 5, per_face=False)
    w.W, w.b = _features(s, n_feat, 5, w.sigma)
    w.x_test = uniform(s + 200, "test", 5000 * 5).reshape(-1, 5)
    return w


def bratu2d(n_int=8192, n_bc=1024, n_feat=2048, lam=1.0):
    """Lap u + lam e^u = 0 on [0,1]^2, u = 0 on the boundary; Newton from beta = 0,
    mu = 1e-10, sigma = 6, boundary weight 100."""
    s = SEED0 + 4
    alpha, coef = _laplacian_terms(2, 1.0)
    w = Workload("bratu2d", 4, 2, n_int, n_bc, n_feat, 6.0, 100.0, alpha, coef,
                 np.array([lam]), s, mu=1e-10, nl_kind=1, nl_lam=lam)
    w.x_int = uniform(s + 100, "x_int", n_int * 2).reshape(n_int, 2)
    w.x_bc = box_boundary(s + 100, "x_bc", n_bc, 2, per_face=True)
    w.W, w.b = _features(s, n_feat, 2, w.sigma)
    w.x_test = uniform(s + 200, "test", 5000 * 2).reshape(-1, 2)
    return w


def nlpoisson2d(n_int=8192, n_bc=1024, n_feat=2048, lam=1.0):
    """-Lap u + lam u^3 = f on [0,1]^2 (Sec. 3.3 NL-Poisson, sigma = 3), manufactured
    u* = sin(pi x) sin(pi y) + x y / 2 with Dirichlet data u* (problem 6); Newton from
    beta = 0, mu = 1e-10, boundary weight 100."""
    s = SEED0 + 6
    alpha, coef = _laplacian_terms(2, -1.0)
    w = Workload("nlpoisson2d", 6, 2, n_int, n_bc, n_feat, 3.0, 100.0, alpha, coef,
                 np.array([lam]), s, mu=1e-10, nl_kind=2, nl_lam=lam)
    w.x_int = uniform(s + 100, "x_int", n_int * 2).reshape(n_int, 2)
    w.x_bc = box_boundary(s + 100, "x_bc", n_bc, 2, per_face=True)
    w.W, w.b = _features(s, n_feat, 2, w.sigma)
    w.x_test = uniform(s + 200, "test", 5000 * 2).reshape(-1, 2)
    return w


def nlhelmholtz2d(n_int=8192, n_bc=1024, n_feat=2048, k=3.0, lam=1.0):
    """Lap u + k^2 u + lam u^3 = f on [0,1]^2 (Sec. 3.3 NL-Helmholtz, k = 3, sigma = 5),
    the same manufactured u* (problem 7); Newton from beta = 0, mu = 1e-10, boundary
    weight 100."""
    s = SEED0 + 7
    alpha = np.array([[2, 0], [0, 2], [0, 0]], np.int32)
    w = Workload("nlhelmholtz2d", 7, 2, n_int, n_bc, n_feat, 5.0, 100.0, alpha,
                 np.array([1.0, 1.0, k * k]), np.array([k, lam]), s, mu=1e-10, nl_kind=2, nl_lam=lam)
    w.x_int = uniform(s + 100, "x_int", n_int * 2).reshape(n_int, 2)
    w.x_bc = box_boundary(s + 100, "x_bc", n_bc, 2, per_face=True)
    w.W, w.b = _features(s, n_feat, 2, w.sigma)
    w.x_test = uniform(s + 200, "test", 5000 * 2).reshape(-1, 2)
    return w


def allen_cahn1d(n_int=5000, n_feat=1500, eps=0.1):
    """eps u'' + u - u^3 = 0 on [0,1] (Sec. 3.3 Allen-Cahn, eps = 0.1, sigma = 3) in true
    solver mode (f = 0), Dirichlet data from the kink u* = tanh((x - 1/2)/sqrt(2 eps))
    (problem 8); interior points uniform-random, the two ends as boundary rows; Newton
    warm-started from the linear part, mu = 1e-10, boundary weight 100."""
    s = SEED0 + 8
    w = Workload("allen_cahn1d", 8, 1, n_int, 2, n_feat, 3.0, 100.0,
                 np.array([[2], [0]], np.int32), np.array([eps, 1.0]), np.array([eps]), s,
                 mu=1e-10, nl_kind=2, nl_lam=-1.0)
    w.x_int = uniform(s + 100, "x_int", n_int).reshape(n_int, 1)
    w.x_bc = np.array([[0.0], [1.0]])
    w.W, w.b = _features(s, n_feat, 1, w.sigma)
    w.x_test = uniform(s + 200, "test", 5000).reshape(-1, 1)
    return w


BURGERS_STAGES = (1.0, 0.5, 0.2, 0.1)


def burgers1d(n_int=5000, n_feat=1500, nu=0.1):
    """u u' - nu u'' = 0 on [0,1] (Sec. 3.3 steady Burgers, nu = 0.1, sigma = 10) in true
    solver mode (f = 0), Dirichlet data from the viscous shock u* = -tanh((x - 1/2)/(2 nu))
    (problem 9); Newton with continuation in nu over BURGERS_STAGES (ending at nu),
    warm-started from the linear part, mu = 1e-10, boundary weight 100.  coef holds the
    target -nu of the term D^2."""
    s = SEED0 + 9
    w = Workload("burgers1d", 9, 1, n_int, 2, n_feat, 10.0, 100.0,
                 np.array([[2]], np.int32), np.array([-nu]), np.array([nu]), s,
                 mu=1e-10, nl_kind=3, nl_lam=1.0)
    w.x_int = uniform(s + 100, "x_int", n_int).reshape(n_int, 1)
    w.x_bc = np.array([[0.0], [1.0]])
    w.W, w.b = _features(s, n_feat, 1, w.sigma)
    w.x_test = uniform(s + 200, "test", 5000).reshape(-1, 1)
    return w


def burgers_stage_coef(nu=0.1):
    """Continuation coefficients of the term D^2 per stage: -nu_k for nu_k in
    BURGERS_STAGES down to nu."""
    stages = [v for v in BURGERS_STAGES if v > nu] + [nu]
    return np.array([[-v] for v in stages])


def varcoef2d(n_int=8192, n_bc=1024, n_feat=2048, a=1.0):
    """div(nu grad u) = f on [0,1]^2 with nu = 1 + a (x^2 + y^2/2) (the variable-coefficient
    form of Sec. 3.8, expanded as nu Lap u + grad nu . grad u), manufactured
    u* = sin(pi x) sin(2 pi y) + x y (problem 10); the operator is four per-point terms
    with coefficients nu, nu, d nu/dx, d nu/dy on D^(2,0), D^(0,2), D^(1,0), D^(0,1);
    points as helmholtz2d, sigma = 6, boundary weight 100."""
    s = SEED0 + 10
    w = Workload("varcoef2d", 10, 2, n_int, n_bc, n_feat, 6.0, 100.0,
                 np.zeros((1, 2), np.int32), np.zeros(1), np.array([a]), s,
                 pp_alpha=np.array([[2, 0], [0, 2], [1, 0], [0, 1]], np.int32),
                 pp_kinds=(2, 2, 3, 4))
    w.x_int = uniform(s + 100, "x_int", n_int * 2).reshape(n_int, 2)
    w.x_bc = box_boundary(s + 100, "x_bc", n_bc, 2, per_face=True)
    w.W, w.b = _features(s, n_feat, 2, w.sigma)
    w.x_test = uniform(s + 200, "test", 5000 * 2).reshape(-1, 2)
    return w


def gauss_theta(seed: int, name: str, n_src: int = 4) -> np.ndarray:
    """theta_k = (c_kx, c_ky, w_k, a_k): centres U(0.2,0.8)^2, widths U(0.05,0.15),
    amplitudes U(0.5,2)."""
    u = uniform(seed, name, 4 * n_src).reshape(n_src, 4)
    th = np.empty((n_src, 4))
    th[:, 0] = 0.2 + 0.6 * u[:, 0]
    th[:, 1] = 0.2 + 0.6 * u[:, 1]
    th[:, 2] = 0.05 + 0.10 * u[:, 2]
    th[:, 3] = 0.5 + 1.5 * u[:, 3]
    return th.reshape(-1)


def perturb_theta(seed: int, name: str, theta: np.ndarray) -> np.ndarray:
    """Evaluation point theta_0: centres moved by U(-0.05, 0.05), widths and
    amplitudes scaled by U(0.9, 1.1)."""
    th = theta.reshape(-1, 4).copy()
    u = uniform(seed, name, th.size).reshape(th.shape)
    th[:, 0:2] += 0.1 * u[:, 0:2] - 0.05
    th[:, 2:4] *= 0.9 + 0.2 * u[:, 2:4]
    return th.reshape(-1)


def inverse_instance(q: int, n_int=None, n_feat=None, seed_offset=0):
    """Instance q of the batched steady inverse heat-source problem:
    -Lap u = s(x; theta) on [0,1]^2, u = 0 on the boundary (weight 100),
    n_int ~ U{1024..8192}, n_feat ~ U{512..2048}, n_bc = n_int / 8 (a multiple of 4,
    walked by edge), sigma = 8, mu = 1e-10; 64 sensors U(0.05, 0.95)^2;
    observation noise N(0, 1e-3^2) (returned, to be added to the forward values)."""
    s = SEED0 + 5 + seed_offset
    tag = f"inst{q}"
    if n_int is None:
        n_int = 1024 + int(uniform(s, tag + "/nint", 1)[0] * (8192 - 1024 + 1))
    if n_feat is None:
        n_feat = 512 + int(uniform(s, tag + "/nfeat", 1)[0] * (2048 - 512 + 1))
    n_bc = max(4, (n_int // 8) // 4 * 4)
    alpha, coef = _laplacian_terms(2, -1.0)
    theta = gauss_theta(s + 300, tag + "/theta")
    w = Workload(f"inverse2d[{q}]", 5, 2, n_int, n_bc, n_feat, 8.0, 100.0, alpha, coef,
                 theta, s, mu=1e-10)
    w.x_int = uniform(s + 100, tag + "/x_int", n_int * 2).reshape(n_int, 2)
    w.x_bc = box_boundary(s + 100, tag + "/x_bc", n_bc, 2, per_face=True)
    w.W = 8.0 * normal(s, tag + "/W", n_feat * 2).reshape(n_feat, 2)
    w.b = 2.0 * math.pi * uniform(s, tag + "/b", n_feat)
    w.x_test = uniform(s + 200, tag + "/test", 5000 * 2).reshape(-1, 2)
    w.sensors = 0.05 + 0.9 * uniform(s + 300, tag + "/sensors", 64 * 2).reshape(64, 2)
    w.noise = 1e-3 * normal(s + 300, tag + "/noise", 64)
    w.theta0 = perturb_theta(s + 300, tag + "/theta0", theta)
    return w


CONFIGS = {
    "poisson1d": poisson1d,
    "helmholtz2d": helmholtz2d,
    "poisson5d": poisson5d,
    "bratu2d": bratu2d,
}
