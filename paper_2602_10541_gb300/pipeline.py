"""Compose the C-ABI calls into the paper's pipelines (Alg. 1; Sec. 2.4; Sec. 3.8).

Orchestration only: every number is produced by libfastlsq kernels through the
binding in ``fastlsq.py``.  Used by the tests, ``bench.py`` and the smoke check.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import fastlsq as fl
from .workloads import Workload


@dataclass
class DeviceProblem:
    """A workload's inputs resident on the GPU (float64)."""
    w: Workload
    x_int: torch.Tensor
    x_bc: torch.Tensor
    W: torch.Tensor
    b: torch.Tensor
    x_test: torch.Tensor
    op_int: fl.Op
    op_bc: fl.Op


def upload(w: Workload, device="cuda:0", ctx=None) -> DeviceProblem:
    """Copy a workload's inputs to the GPU.  A workload with per-point terms (variable
    coefficients) needs ctx: their coefficients at the interior points are evaluated
    on the GPU from the problem catalogue (fastlsq_rhs with the workload's kinds)."""
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)
    x_int = t(w.x_int)
    op_int = fl.Op(w.alpha, w.coef)
    if w.pp_alpha is not None:
        if ctx is None:
            raise ValueError("upload: a workload with per-point terms needs a context")
        pp = []
        for kind in w.pp_kinds:
            c = torch.empty(w.n_int, dtype=torch.float64, device=device)
            fl.fastlsq_rhs(ctx, w.problem, kind, w.params, x_int, 1.0, c)
            pp.append(c)
        op_int = fl.Op(w.alpha, w.coef, pp_alpha=w.pp_alpha, pp_coef=pp)
    return DeviceProblem(w, x_int, t(w.x_bc), t(w.W), t(w.b), t(w.x_test), op_int,
                         fl.Op.identity(w.d))


class LinearSolver:
    """One linear PDE solve (Alg. 1): rhs, operator assembly (FP32 for the factor,
    FP64 for the refinement residual) and the least-squares solve.  Buffers are
    allocated once so that repeated solves (and CUDA-graph capture) reuse them."""

    def __init__(self, ctx: fl.Context, dp: DeviceProblem, prec=fl.PREC_MIXED, max_refine=2,
                 mu=None, refine_mode=fl.REFINE_CLASSICAL, refine_tol=1e-10, overlap=True):
        self.ctx, self.dp, self.prec, self.max_refine = ctx, dp, prec, max_refine
        self.refine_mode, self.refine_tol = refine_mode, refine_tol
        w = dp.w
        self.m, self.n = w.n_rows, w.n_feat
        self.mu = w.mu if mu is None else mu
        dev = dp.W.device
        self.A64 = fl.colmajor(self.m, self.n, torch.float64, dev)
        self.A32 = fl.colmajor(self.m, self.n, torch.float32, dev) if prec == fl.PREC_MIXED else None
        self.rhs = torch.empty((1, self.A64.shape[1]), dtype=torch.float64, device=dev)
        self.beta = torch.zeros((1, self.n), dtype=torch.float64, device=dev)
        self.stats = None
        # MIXED: the FP64 operator, read only by the refinement, is assembled on a
        # side stream while the FP32 factorisation runs
        self.side = None
        if overlap and self.A32 is not None:
            lo, _ = torch.cuda.Stream.priority_range()
            self.side = torch.cuda.Stream(device=dev, priority=lo)
            self.ev_fp32 = torch.cuda.Event()
            self.ev_fp64 = torch.cuda.Event()

    def _assemble_one(self, dtype, A):
        ctx, dp, w = self.ctx, self.dp, self.dp.w
        fl.fastlsq_assemble(ctx, dtype, dp.x_int, dp.op_int, 1.0, dp.W, dp.b, w.scale, A, 0)
        fl.fastlsq_assemble(ctx, dtype, dp.x_bc, dp.op_bc, w.lam_bc, dp.W, dp.b, w.scale, A, w.n_int)

    def assemble(self):
        if self.A32 is not None:
            self._assemble_one(fl.F32, self.A32)
        if self.side is None:
            self._assemble_one(fl.F64, self.A64)
            return
        # the side stream starts after the FP32 assembly (the context's column
        # prefactors are free again, and the previous solve's reads of A64 are done)
        main = self.ctx.stream
        self.ev_fp32.record(main)
        self.side.wait_event(self.ev_fp32)
        fl.fastlsq_set_stream(self.ctx, self.side)
        try:
            self._assemble_one(fl.F64, self.A64)
        finally:
            fl.fastlsq_set_stream(self.ctx, main)
        self.ev_fp64.record(self.side)

    def build_rhs(self):
        ctx, dp, w = self.ctx, self.dp, self.dp.w
        r = self.rhs[0]
        fl.fastlsq_rhs(ctx, w.problem, fl.RHS_SOURCE, w.params, dp.x_int, 1.0, r[: w.n_int])
        fl.fastlsq_rhs(ctx, w.problem, fl.RHS_EXACT, w.params, dp.x_bc, w.lam_bc,
                       r[w.n_int: w.n_rows])

    def solve(self, stats=False, keep=False):
        A = self.A32 if self.prec == fl.PREC_MIXED else self.A64
        if self.side is not None:     # the waits are queued by the call itself
            fl.fastlsq_set_refine_event(self.ctx, self.ev_fp64)
        try:
            rc, fac, st = fl.fastlsq_lstsq(self.ctx, self.prec, A, self.m, self.mu, self.rhs, self.beta,
                                           A_refine=self.A64,
                                           max_refine=(self.max_refine if self.prec == fl.PREC_MIXED
                                                       or self.refine_mode == fl.REFINE_CGLS else 0),
                                           keep=keep, stats=stats, refine_mode=self.refine_mode,
                                           refine_tol=self.refine_tol)
        finally:
            if self.side is not None:
                fl.fastlsq_set_refine_event(self.ctx, None)
        self.stats = st
        return fac

    def step(self, stats=False):
        self.build_rhs()
        self.assemble()
        return self.solve(stats=stats)

    def outer_grad(self, W_hat, fac=None, max_iter=0):
        """Gradient of the outer loss ||A beta* - rhs||^2 of Alg. 2 (learnable bandwidth)
        after a solve: r = rhs - A beta (FP64 operator), for mu > 0 the adjoint vector
        v = (A^T A + mu I)^{-1} beta and A v from the kept factor `fac`, then the
        feature-weight gradient of both row blocks and its contraction with W_hat.
        Returns (r [m], gW [n_feat][d], out [d*d + 1]): out[a*d + c] = dL/dL_ac for
        W_j = L W_hat_j, out[d*d] = dL/dsigma for W = sigma W_hat."""
        ctx, dp, w = self.ctx, self.dp, self.dp.w
        dev = dp.W.device
        beta = self.beta[0]
        r = torch.empty(self.m, dtype=torch.float64, device=dev)
        fl.fastlsq_residual(ctx, self.A64, self.m, beta, self.rhs[0], r)
        v = Av = None
        if self.mu > 0:
            if fac is None:
                raise ValueError("outer_grad: mu > 0 needs the kept factor")
            v = torch.empty(self.n, dtype=torch.float64, device=dev)
            Av = torch.empty(self.m, dtype=torch.float64, device=dev)
            fl.fastlsq_backward(ctx, fac, beta, v, Av, self.A64, max_iter=max_iter)
        gW = torch.zeros((self.n, w.d), dtype=torch.float64, device=dev)
        gb = torch.zeros(self.n, dtype=torch.float64, device=dev)
        cf = dict(c_v=-2.0 * self.mu, c_rb=-2.0, c_av=2.0 * self.mu)
        ni = w.n_int
        fl.fastlsq_weight_grad(ctx, dp.x_int, dp.op_int, 1.0, dp.W, dp.b, w.scale, r[:ni], beta, gW, gb,
                               v=v, Av=None if Av is None else Av[:ni], **cf)
        fl.fastlsq_weight_grad(ctx, dp.x_bc, dp.op_bc, w.lam_bc, dp.W, dp.b, w.scale, r[ni:], beta, gW,
                               gb, v=v, Av=None if Av is None else Av[ni:], **cf)
        out = torch.empty(w.d * w.d + 1, dtype=torch.float64, device=dev)
        W_hat = torch.as_tensor(np.ascontiguousarray(W_hat), dtype=torch.float64, device=dev)
        fl.fastlsq_bandwidth_grad(ctx, gW, W_hat, out)
        return r, gW, out

    def u_test(self, beta=None):
        dp = self.dp
        u = torch.empty(dp.x_test.shape[0], dtype=torch.float64, device=dp.W.device)
        fl.fastlsq_eval(self.ctx, dp.x_test, dp.W, dp.b, dp.w.scale,
                        self.beta[0] if beta is None else beta, u)
        return u

    def u_exact_test(self):
        dp = self.dp
        u = torch.empty(dp.x_test.shape[0], dtype=torch.float64, device=dp.W.device)
        fl.fastlsq_rhs(self.ctx, dp.w.problem, fl.RHS_EXACT, dp.w.params, dp.x_test, 1.0, u)
        return u


class ConcurrentSolves:
    """Independent linear solves queued together, each on its own context and stream.

    One solve's critical path is its chain of panel factorisations, each on one
    cluster of at most 16 SMs; the trailing updates fill part of the rest.  Solves of
    independent instances (other seeds, parameters or right-hand-side operators) on
    separate streams fill the remaining SMs.  step() forks from `origin` (a stream)
    and joins back into it, so events recorded on `origin` around it time the batch.
    With several solves in flight, turn look-ahead off in their contexts
    (OPT_LOOKAHEAD = 0): the other solves already fill the SMs beside each panel, and
    one update pass per panel is cheaper than the split one (helmholtz2d, 8 solves:
    272 solves/s without look-ahead against 243 with it, same kernels)."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.ev_fork = torch.cuda.Event()
        self.ev_done = [torch.cuda.Event() for _ in self.solvers]

    def step(self, origin=None):
        origin = torch.cuda.current_stream() if origin is None else origin
        self.ev_fork.record(origin)
        for sv, ev in zip(self.solvers, self.ev_done):
            s = sv.ctx.stream
            s.wait_event(self.ev_fork)
            with torch.cuda.stream(s):
                sv.step()
            ev.record(s)
        for ev in self.ev_done:
            origin.wait_event(ev)


def tuned(kernel: str, default: dict) -> dict:
    """The launch shape the autotuner recorded for a kernel (tuning.json next to this
    module, written by ``python -m paper_2602_10541_gb300.tune``), else `default`."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")
    if os.path.exists(path):
        entry = json.load(open(path)).get(kernel)
        if entry:
            return {k: entry.get(k, v) for k, v in default.items()}
    return dict(default)


class InverseBatch:
    """Instances of the batched inverse heat-source problem (Sec. 3.8, steady form) on
    the GPU behind one pre-factored plan: setup factors every operator once (FP64),
    each evaluation is one persistent launch over all instances (loss, beta, dL/dtheta
    per instance).  Observations come from the forward map at the instances' true
    parameters plus their noise; evaluations start at their perturbed parameters."""

    def __init__(self, ctx, workloads, device="cuda:0", mu=1e-10, bc_weight=100.0, launch=None, thin_q=True):
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)
        self.ctx, self.ws = ctx, list(workloads)
        self.inst = [dict(x_int=t(w.x_int), x_bc=t(w.x_bc), W=t(w.W), b=t(w.b), sensors=t(w.sensors),
                          y_obs=torch.zeros(w.sensors.shape[0], dtype=torch.float64, device=device),
                          theta=t(w.params), beta=torch.zeros(w.n_feat, dtype=torch.float64, device=device),
                          loss=torch.zeros(1, dtype=torch.float64, device=device),
                          dtheta=torch.zeros(w.params.size, dtype=torch.float64, device=device))
                     for w in self.ws]
        self.n_src = self.ws[0].params.size // 4
        self.launch = launch or tuned("inverse_eval", {"threads": 256, "ctas_per_sm": 1, "cluster": 1})
        self.thin_q = bool(thin_q)
        fl.fastlsq_set_option(ctx, fl.OPT_INVERSE_THIN_Q, int(self.thin_q))
        self.plan = fl.fastlsq_inverse_prepare(ctx, self.inst, fl.Op(self.ws[0].alpha, self.ws[0].coef),
                                               self.n_src, mu=mu, bc_weight=bc_weight)
        self.device = device

    def eval(self):
        fl.fastlsq_inverse_eval(self.ctx, self.plan, **self.launch)

    def observe(self):
        """y_obs = u(sensors) at the true parameters + the instance's noise; theta set to
        the perturbed evaluation point theta_0."""
        self.eval()
        for d, w in zip(self.inst, self.ws):
            u_s = torch.empty(d["sensors"].shape[0], dtype=torch.float64, device=self.device)
            fl.fastlsq_eval(self.ctx, d["sensors"], d["W"], d["b"], w.scale, d["beta"], u_s)
            d["y_obs"].copy_(u_s + torch.as_tensor(w.noise, device=self.device))
            d["theta"].copy_(torch.as_tensor(w.theta0, device=self.device))

    def close(self):
        self.plan.close()


def newton_solve(ctx, dp: DeviceProblem, f, g, prec=fl.PREC_MIXED, max_iter=30, tol=1e-10,
                 stage_coef=None, warm=True, max_refine=64, refine_tol=1e-13):
    """Newton-Raphson with the refinements of Sec. 2.4 on a device problem: warm start
    from the linear part (one regularised solve with N dropped, i.e. a Newton step with
    no nonlinearity from beta = 0), then fastlsq_newton, or with stage_coef
    ([n_stages][n_terms]) fastlsq_newton_continuation with max_iter iterations per
    stage.  f, g: device sources and Dirichlet data.  Returns (beta, status, stats),
    stats a list (one per stage)."""
    w = dp.w
    beta = torch.zeros(w.n_feat, dtype=torch.float64, device=dp.W.device)
    first = w.coef if stage_coef is None else np.asarray(stage_coef, dtype=np.float64)[0]
    common = dict(mu=w.mu, prec=prec, max_refine=max_refine, refine_tol=refine_tol)
    if warm:
        fl.fastlsq_newton(ctx, dp.x_int, dp.x_bc, fl.Op(w.alpha, first), fl.NL_NONE, 0.0,
                          w.lam_bc, f, g, dp.W, dp.b, w.scale, beta, max_iter=1, tol=0.0, **common)
    if stage_coef is None:
        rc, st = fl.fastlsq_newton(ctx, dp.x_int, dp.x_bc, dp.op_int, w.nl_kind, w.nl_lam,
                                   w.lam_bc, f, g, dp.W, dp.b, w.scale, beta, max_iter=max_iter,
                                   tol=tol, **common)
        return beta, rc, [st]
    rc, sts = fl.fastlsq_newton_continuation(ctx, dp.x_int, dp.x_bc, dp.op_int, stage_coef,
                                             w.nl_kind, w.nl_lam, w.lam_bc, f, g, dp.W, dp.b,
                                             w.scale, beta, max_iter=max_iter, tol=tol, **common)
    return beta, rc, sts


def rel_l2(a, b) -> float:
    """Relative L2 difference ||a - b|| / ||b||, computed on the host."""
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)
    b = b.detach().cpu().numpy() if isinstance(b, torch.Tensor) else np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def main(argv=None):
    """Command line: run a few linear solves of a named workload and print the error
    of the last one on the test set, e.g. as the program under a profiler:
    ``python -m paper_2602_10541_gb300.pipeline helmholtz2d --prec mixed --steps 2``;
    ``... random --rows 36864 --cols 256`` factors a random MIXED matrix of that shape;
    ``... inverse --instances 16`` runs gradient evaluations of a batch of inverse-problem
    instances."""
    import argparse

    from . import workloads as wl

    ap = argparse.ArgumentParser(prog="python -m paper_2602_10541_gb300.pipeline")
    ap.add_argument("workload", choices=["poisson1d", "helmholtz2d", "poisson5d", "random", "inverse"])
    ap.add_argument("--prec", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--refine", type=int, default=2)
    ap.add_argument("--refine-mode", choices=["classical", "cgls"], default="classical")
    ap.add_argument("--tensor-core", type=int, default=1, choices=[0, 1, 2],
                    help="1 (default): blocked tcgen05 updates; 2: panel-by-panel TF32x3; 0: SIMT FP32")
    ap.add_argument("--lookahead", type=int, default=1, choices=[0, 1],
                    help="1 (the library default): factor the next panel on a second stream")
    ap.add_argument("--rows", type=int, default=36864, help="random: rows")
    ap.add_argument("--cols", type=int, default=256, help="random: columns")
    ap.add_argument("--instances", type=int, default=16, help="inverse: instances")
    ap.add_argument("--cluster", type=int, default=0, choices=[0, 1, 2, 4],
                    help="inverse: CTAs per instance (0: the tuned launch)")
    a = ap.parse_args(argv)
    ctx = fl.Context(0)
    fl.fastlsq_set_option(ctx, fl.OPT_TENSOR_CORE, a.tensor_core)
    fl.fastlsq_set_option(ctx, fl.OPT_LOOKAHEAD, a.lookahead)
    if a.workload == "random":
        g = torch.Generator("cuda:0").manual_seed(1)
        A = fl.colmajor(a.rows, a.cols, torch.float32, "cuda:0", zero=True)
        A[:, : a.rows] = torch.randn((a.cols, a.rows), generator=g, device="cuda:0")
        for _ in range(a.steps):
            _, fac, st = fl.fastlsq_lstsq(ctx, fl.PREC_MIXED, A, a.rows, 0.0, None, None,
                                          A_refine=A.double(), keep=True, stats=True)
            fl.fastlsq_factor_destroy(ctx, fac)
        torch.cuda.synchronize()
        print(f"random {a.rows} x {a.cols}: panel width {st.nb}, trailing-update mode {st.tensor_core}")
        return
    if a.workload == "inverse":
        batch = InverseBatch(ctx, [wl.inverse_instance(q) for q in range(a.instances)])
        if a.cluster:
            batch.launch = {**batch.launch, "cluster": a.cluster}
        batch.observe()
        for _ in range(a.steps):
            batch.eval()
        torch.cuda.synchronize()
        print(f"inverse: {a.instances} instances, mean loss "
              f"{sum(d['loss'].item() for d in batch.inst) / a.instances:.4e}")
        batch.close()
        return
    dp = upload(wl.CONFIGS[a.workload]())
    s = LinearSolver(ctx, dp, prec=fl.PREC_MIXED if a.prec == "mixed" else fl.PREC_FP64,
                     max_refine=a.refine,
                     refine_mode=fl.REFINE_CGLS if a.refine_mode == "cgls" else fl.REFINE_CLASSICAL)
    for _ in range(a.steps):
        s.step()
    torch.cuda.synchronize()
    print(f"{a.workload} {a.prec}: rel L2 error vs exact on the test set "
          f"{rel_l2(s.u_test(), s.u_exact_test()):.3e}")


if __name__ == "__main__":
    main()
