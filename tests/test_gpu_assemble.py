"""GPU parity of the operator assembly (eq. cyclic; eq. linear_system) against the
FP64 CPU oracle, through the C ABI.

Error per entry is measured relative to the entry's magnitude without the
trigonometric factor, |A_ij - ref_ij| / (rw * s * sum_t |c_t + pp| prod_k |W_jk|^alpha_tk),
because an entry near a zero of sin has no meaningful relative error.  Bars: 1e-5
for the FP32 kernel (reference built from the FP32-rounded inputs, so input
rounding is not charged to the kernel) and 1e-12 for the FP64 kernel.  Layout is
checked bit-exactly: rows outside the written block keep a sentinel.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2602_10541_gb300 import fastlsq as fl
from paper_2602_10541_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
SENTINEL = 12345.0


@pytest.fixture(scope="module")
def ctx():
    return fl.Context(0)


def _mag(x_rows, alpha, coef, W, scale, rw, cpt=None):
    """rw * s * sum_t |c_t (+ pp)| * prod_k |W_jk|^alpha_tk  -> (n_rows, n_feat)"""
    n = x_rows
    out = np.zeros((n, W.shape[0]))
    for t in range(alpha.shape[0]):
        mono = np.prod(np.abs(W) ** alpha[t][None, :], axis=1)
        c = np.full(n, abs(coef[t])) if cpt is None else np.abs(coef[t] + cpt[t])
        out += c[:, None] * mono[None, :]
    return rw * scale * out


CASES = {
    "poisson1d": (1, 10.0, [[2]], [-1.0]),
    "helmholtz2d": (2, 8.0, [[2, 0], [0, 2], [0, 0]], [1.0, 1.0, 16.0]),
    "poisson5d": (5, 3.0, (2 * np.eye(5, dtype=int)).tolist(), [-1.0] * 5),
    "biharmonic2d": (2, 2.0, [[4, 0], [2, 2], [0, 4]], [1.0, 2.0, 1.0]),
    "advection_mixed3d": (3, 2.0, [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1], [2, 0, 1], [0, 0, 0]],
                          [0.3, -1.2, 0.7, 0.05, -0.4, 2.0]),
}


@pytest.mark.parametrize("dtype", [fl.F32, fl.F64])
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("row_offset", [0, 5])
def test_assemble_matches_oracle(ctx, dtype, case, row_offset):
    d, sigma, alpha, coef = CASES[case]
    alpha = np.array(alpha, np.int32)
    coef = np.array(coef)
    rng = np.random.default_rng(hash((case, row_offset)) % 2**32)
    n_rows, n_feat = 301, 77                      # ragged against the 128 x 64 tile
    x = rng.random((n_rows, d))
    W = sigma * rng.standard_normal((n_feat, d))
    b = rng.uniform(0, 2 * math.pi, n_feat)
    scale, rw = 1 / math.sqrt(n_feat), 3.0
    tdt = torch.float32 if dtype == fl.F32 else torch.float64
    ld = row_offset + n_rows + 3
    A = torch.full((n_feat, ld), SENTINEL, dtype=tdt, device=DEV)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=DEV)
    fl.fastlsq_assemble(ctx, dtype, t(x), fl.Op(alpha, coef), rw, t(W), t(b), scale, A, row_offset)
    torch.cuda.synchronize()
    got = A.cpu().numpy().astype(np.float64).T             # (ld, n_feat)
    if dtype == fl.F32:
        r32 = lambda a: a.astype(np.float32).astype(np.float64)
        xr, Wr, br = r32(x), r32(W), r32(b)
        tol = 1e-5
    else:
        xr, Wr, br = x, W, b
        tol = 1e-12
    ref = oracle.assemble(xr, alpha, coef, Wr, br, scale, row_weight=rw)
    block = got[row_offset: row_offset + n_rows]
    err = np.abs(block - ref) / _mag(n_rows, alpha, coef, Wr, scale, rw)
    assert err.max() <= tol, err.max()
    # layout: nothing outside the block was written
    assert np.all(got[:row_offset] == SENTINEL)
    assert np.all(got[row_offset + n_rows:] == SENTINEL)


@pytest.mark.parametrize("ctas", [1, 2])
def test_fp64_assembly_persistent_grid_is_identical(ctx, ctas):
    """The persistent FP64 assembly grid (k CTAs per SM looping over the 128 x 64 tiles)
    writes the same entries as one CTA per tile, bit for bit, on a ragged operator
    with more tiles than the grid (2,000 + 300 rows x 700 features) and a per-point term."""
    d, n_rows, n_feat = 3, 2300, 700
    rng = np.random.default_rng(11)
    x = rng.random((n_rows, d))
    W = 4 * rng.standard_normal((n_feat, d))
    b = rng.uniform(0, 2 * math.pi, n_feat)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=DEV)
    op = fl.Op([[2, 0, 0], [0, 2, 0], [0, 0, 1]], [1.0, 1.0, -0.5], pp_alpha=[[0, 0, 0]],
               pp_coef=[t(rng.standard_normal(n_rows))])
    out = []
    for k in (0, ctas):
        fl.fastlsq_set_option(ctx, fl.OPT_FP64_ASSEMBLY_CTAS, k)
        A = torch.full((n_feat, n_rows + 5), SENTINEL, dtype=torch.float64, device=DEV)
        try:
            fl.fastlsq_assemble(ctx, fl.F64, t(x), op, 2.0, t(W), t(b), 0.1, A, 5)
        finally:
            fl.fastlsq_set_option(ctx, fl.OPT_FP64_ASSEMBLY_CTAS, 0)
        torch.cuda.synchronize()
        out.append(A.cpu())
    assert torch.equal(out[0], out[1])
    assert torch.all(out[1][:, :5] == SENTINEL)


@pytest.mark.parametrize("dtype", [fl.F32, fl.F64])
def test_per_point_terms(ctx, dtype):
    # Newton Jacobian form: L = Lap plus per-point terms c_i phi_j (alpha = 0) and
    # e_i d/dx phi_j (odd order, cos path)
    d, n_rows, n_feat = 2, 257, 65
    rng = np.random.default_rng(3)
    x = rng.random((n_rows, d))
    W = 6 * rng.standard_normal((n_feat, d))
    b = rng.uniform(0, 2 * math.pi, n_feat)
    c = rng.standard_normal(n_rows)
    e = rng.standard_normal(n_rows)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=DEV)
    ct, et = t(c), t(e)
    op = fl.Op([[2, 0], [0, 2]], [1.0, 1.0], pp_alpha=[[0, 0], [1, 0]], pp_coef=[ct, et])
    tdt = torch.float32 if dtype == fl.F32 else torch.float64
    A = torch.zeros((n_feat, n_rows), dtype=tdt, device=DEV)
    scale = 1 / math.sqrt(n_feat)
    fl.fastlsq_assemble(ctx, dtype, t(x), op, 1.0, t(W), t(b), scale, A, 0)
    torch.cuda.synchronize()
    got = A.cpu().numpy().astype(np.float64).T
    if dtype == fl.F32:
        r32 = lambda a: a.astype(np.float32).astype(np.float64)
        x, W, b, c, e = r32(x), r32(W), r32(b), r32(c), r32(e)
    alpha = np.array([[2, 0], [0, 2], [0, 0], [1, 0]], np.int32)
    coef = np.array([1.0, 1.0, 0.0, 0.0])
    cpt = np.zeros((4, n_rows))
    cpt[2], cpt[3] = c, e
    ref = oracle.assemble(x, alpha, coef, W, b, scale, coef_pt=cpt)
    err = np.abs(got - ref) / _mag(n_rows, alpha, coef, W, scale, 1.0, cpt)
    assert err.max() <= (1e-5 if dtype == fl.F32 else 1e-12), err.max()


@pytest.mark.parametrize("name", ["helmholtz2d", "poisson5d"])
def test_full_size_sampled_entries(ctx, name):
    """Full-size operator (the bench's launch configuration), checked on a random
    64 x 64 block of rows and columns against the oracle."""
    w = wl.CONFIGS[name]()
    rng = np.random.default_rng(11)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)
    A = fl.colmajor(w.n_rows, w.n_feat, torch.float32, DEV)
    fl.fastlsq_assemble(ctx, fl.F32, t(w.x_int), fl.Op(w.alpha, w.coef), 1.0, t(w.W), t(w.b),
                        w.scale, A, 0)
    fl.fastlsq_assemble(ctx, fl.F32, t(w.x_bc), fl.Op.identity(w.d), w.lam_bc, t(w.W), t(w.b),
                        w.scale, A, w.n_int)
    torch.cuda.synchronize()
    rows_i = np.sort(rng.choice(w.n_int, 48, replace=False))
    rows_b = np.sort(rng.choice(w.n_bc, 16, replace=False))
    cols = np.sort(rng.choice(w.n_feat, 64, replace=False))
    r32 = lambda a: a.astype(np.float32).astype(np.float64)
    Ac = A[torch.as_tensor(cols, device=DEV)].cpu().numpy().astype(np.float64)   # (64, ld)
    Wc, bc = r32(w.W[cols]), r32(w.b[cols])
    ref_i = oracle.assemble(r32(w.x_int[rows_i]), w.alpha, w.coef, Wc, bc, w.scale)
    ref_b = oracle.assemble(r32(w.x_bc[rows_b]), np.zeros((1, w.d), np.int32), [1.0], Wc, bc,
                            w.scale, row_weight=w.lam_bc)
    got_i = Ac[:, rows_i].T
    got_b = Ac[:, w.n_int + rows_b].T
    mag_i = _mag(len(rows_i), w.alpha, w.coef, Wc, w.scale, 1.0)
    mag_b = np.full(ref_b.shape, w.lam_bc * w.scale)
    assert (np.abs(got_i - ref_i) / mag_i).max() <= 1e-5
    assert (np.abs(got_b - ref_b) / mag_b).max() <= 1e-5


def test_eval_and_rhs_match_oracle(ctx):
    w = wl.helmholtz2d(n_int=333, n_bc=64, n_feat=150)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)
    beta = np.random.default_rng(5).standard_normal(w.n_feat)
    u = torch.empty(w.x_test.shape[0], dtype=torch.float64, device=DEV)
    fl.fastlsq_eval(ctx, t(w.x_test), t(w.W), t(w.b), w.scale, t(beta), u)
    ref = oracle.eval_u(w.x_test, w.W, w.b, w.scale, beta)
    np.testing.assert_allclose(u.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    for prob, d, params in [(oracle.POISSON_1D, 1, ()), (oracle.HELMHOLTZ_2D, 2, (4.0,)),
                            (oracle.POISSON_5D, 5, ()), (oracle.GAUSS_SOURCE_2D, 2,
                                                         tuple(wl.gauss_theta(1, "g")))]:
        x = np.random.default_rng(prob).random((123, d))
        for kind in (fl.RHS_SOURCE, fl.RHS_EXACT):
            out = torch.empty(123, dtype=torch.float64, device=DEV)
            fl.fastlsq_rhs(ctx, prob, kind, params, t(x), 2.5, out)
            if kind == fl.RHS_SOURCE:
                ref = 2.5 * oracle.problem_source(prob, x, params)
            else:
                ref = 2.5 * oracle.problem_exact(prob, x, params)
            np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("case", list(CASES))
def test_eval_op_matches_oracle(ctx, case):
    """(L u)(x) at arbitrary points (gradients, Laplacians, mixed odd/even operators)
    against the oracle's assembled operator times beta, FP64 bar 1e-12 of the
    magnitude sum |L phi_j(x)| |beta_j|."""
    d, sigma, alpha, coef = CASES[case]
    rng = np.random.default_rng(len(case) * 7 + d)
    n, nf = 777, 150
    x = rng.random((n, d))
    W = sigma * rng.standard_normal((nf, d))
    b = 2 * math.pi * rng.random(nf)
    beta = rng.standard_normal(nf)
    scale = 1.0 / math.sqrt(nf)
    alpha, coef = np.array(alpha, np.int32), np.array(coef)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)
    u = torch.empty(n, dtype=torch.float64, device=DEV)
    fl.fastlsq_eval_op(ctx, t(x), fl.Op(alpha, coef), t(W), t(b), scale, t(beta), u)
    A = oracle.assemble(x, alpha, coef, W, b, scale)
    ref = A @ beta
    mag = _mag(n, alpha, coef, W, scale, 1.0) @ np.abs(beta)
    assert np.all(np.abs(u.cpu().numpy() - ref) <= 1e-12 * mag)


def test_eval_op_gradient_and_identity(ctx):
    """The identity operator reproduces fastlsq_eval; the gradient components of u
    agree with central differences of fastlsq_eval (h = 1e-5, O(h^2)); per-point terms
    are refused."""
    w = wl.helmholtz2d(n_int=64, n_bc=16, n_feat=200)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)
    beta = np.random.default_rng(3).standard_normal(w.n_feat)
    x = w.x_test[:500]
    u0 = torch.empty(len(x), dtype=torch.float64, device=DEV)
    ui = torch.empty(len(x), dtype=torch.float64, device=DEV)
    fl.fastlsq_eval(ctx, t(x), t(w.W), t(w.b), w.scale, t(beta), u0)
    fl.fastlsq_eval_op(ctx, t(x), fl.Op.identity(2), t(w.W), t(w.b), w.scale, t(beta), ui)
    np.testing.assert_allclose(ui.cpu().numpy(), u0.cpu().numpy(), rtol=0, atol=1e-13 * u0.abs().max().item())
    h = 1e-5
    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        up = torch.empty(len(x), dtype=torch.float64, device=DEV)
        um = torch.empty(len(x), dtype=torch.float64, device=DEV)
        fl.fastlsq_eval(ctx, t(x + e), t(w.W), t(w.b), w.scale, t(beta), up)
        fl.fastlsq_eval(ctx, t(x - e), t(w.W), t(w.b), w.scale, t(beta), um)
        fd = ((up - um) / (2 * h)).cpu().numpy()
        g = torch.empty(len(x), dtype=torch.float64, device=DEV)
        alpha = np.zeros((1, 2), np.int32)
        alpha[0, k] = 1
        fl.fastlsq_eval_op(ctx, t(x), fl.Op(alpha, [1.0]), t(w.W), t(w.b), w.scale, t(beta), g)
        np.testing.assert_allclose(g.cpu().numpy(), fd, rtol=0, atol=1e-6 * np.abs(fd).max())
    with pytest.raises(fl.FastLSQError):
        fl.fastlsq_eval_op(ctx, t(x), fl.Op(np.zeros((1, 2), np.int32), [1.0], [[0, 0]],
                                            [t(np.zeros(len(x)))]),
                           t(w.W), t(w.b), w.scale, t(beta), ui)
