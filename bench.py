#!/usr/bin/env python
"""Benchmark of the FastLSQ hot path on GB300 (one JSON line on rank 0).

Headline workload (default `--workload poisson5d`): the 5-D Poisson problem
-Lap u = f on [0,1]^5, manufactured u* = sum_k sin(pi x_k) + prod_k x_k, 32768
uniform-random interior points + 4096 boundary points (uniform over the 10 faces,
weight 100), 4096 frozen features W ~ N(0, 9 I), b ~ U(0, 2 pi): the largest of the
linear configurations.  One step = `--instances` independent whole linear PDE solves
(Alg. 1; other seeds, each on its own context and stream): right-hand side, operator
assembly (FP32 for the factor, FP64 for the refinement residual), two-level blocked
Householder QR (tensor-core outer-block updates), triangular solve and two steps of
FP64 iterative refinement, all in libfastlsq kernels through the C ABI.
`--workload helmholtz2d` runs the 2-D Helmholtz configuration instead (9216 x 2048).

`value` is device-timed solves/s with inputs resident in HBM (L2 flushed between
steps, outside the per-step events); `e2e` is the same metric through the C ABI
with host buffers (H2D of the points and features, D2H of beta inside the timed
step).  `roofline` describes the factorisation's trailing update on the tensor
cores (the Y pass and the update pass of the outer blocks), measured with CUDA
events inside the timed region; `kernels` gives every kernel class.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PDE solves/s at <=1e-6 rel L2 err vs FP64 GPU path; assembly Gentries/s"
WORKLOADS = {
    "poisson5d": dict(
        desc=("poisson5d: -Lap u = f, [0,1]^5, 32768 interior + 4096 boundary rows (weight 100), "
              "4096 features sigma=3"),
        rows=32768 + 4096, feat=4096, instances=4,
        # the CPU oracle's bounded samples (same recipe, fewer rows and features); their
        # times are scaled to the full workload by the QR work ratio m n^2
        cpu_sample=dict(n_int=4096, n_bc=512, n_feat=1024),
        ref_sample=dict(n_int=2048, n_bc=256, n_feat=512)),
    "helmholtz2d": dict(
        desc=("helmholtz2d: Lap u + k^2 u = f, k=4, [0,1]^2, 8192 interior + 1024 boundary rows "
              "(weight 100), 2048 features sigma=8"),
        rows=8192 + 1024, feat=2048, instances=8,
        cpu_sample=None,                     # the full workload: one solve is about 20 s
        ref_sample=dict(n_int=2048, n_bc=256, n_feat=512)),
}


def _scale_ratio(name, sample):
    """QR work (m n^2) of the full workload over that of the sample (1 for the full size)."""
    if sample is None:
        return 1.0
    cfg = WORKLOADS[name]
    return cfg["rows"] * cfg["feat"] ** 2 / ((sample["n_int"] + sample["n_bc"]) * sample["n_feat"] ** 2)


def _oracle_solve_seconds(name, sample):
    """One oracle solve of the workload (or of its sample): assembly, rhs, QR, solve."""
    import oracle
    from paper_2602_10541_gb300 import workloads as wl
    w = getattr(wl, name)(**(sample or {}))
    t0 = time.perf_counter()
    A_int = oracle.assemble(w.x_int, w.alpha, w.coef, w.W, w.b, w.scale)
    A_bc = oracle.assemble(w.x_bc, np.zeros((1, w.d), np.int32), [1.0], w.W, w.b, w.scale,
                           row_weight=w.lam_bc)
    f = oracle.problem_source(w.problem, w.x_int, w.params)
    g = oracle.problem_exact(w.problem, w.x_bc, w.params)
    oracle.lstsq(np.vstack([A_int, A_bc]), np.concatenate([f, w.lam_bc * g]))
    return time.perf_counter() - t0


def _sample_text(name, sample, seconds=None):
    if sample is None:
        return f"one oracle solve of the full {name} workload" + (f" ({seconds:.1f} s)" if seconds else "")
    r = _scale_ratio(name, sample)
    return (f"{name} with {sample['n_int']}+{sample['n_bc']} rows x {sample['n_feat']} features"
            + (f" ({seconds:.1f} s)" if seconds else "")
            + f"; time x{r:.0f}: extrapolated to the full workload by the QR work ratio m n^2")


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _job_throughput(total_ms, steps, world, device=None):
    """Whole-job solves/s over `world` replicas: each rank solved `steps` instances in
    total_ms of device time; the job takes as long as its slowest rank (max over ranks)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * steps / (total_ms / 1e3), total_ms


def run_reference(args):
    rank, world, _ = _dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    name = args.workload
    sample = WORKLOADS[name]["ref_sample"]
    ratio = _scale_ratio(name, sample)
    for _ in range(max(0, args.warmup)):
        _oracle_solve_seconds(name, sample)
    ts = [_oracle_solve_seconds(name, sample) for _ in range(args.steps)]
    total = sum(ts) * ratio
    value = args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[name]["desc"], "impl": "FP64 CPU oracle (plain C, 1 thread)"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "cpu": _cpu_model(),
                             "sample": _sample_text(name, sample) + " (per step)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def _src_sha(names):
    """Hash of a kernel class's sources (the .cu file and the headers its kernels use)."""
    h = hashlib.sha256()
    for name in (names,) if isinstance(names, str) else names:
        with open(os.path.join(ROOT, "paper_2602_10541_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


KERNEL_SRC = {"panel": "panel_row.cu", "trail_simt": "qr.cu",
              "trail_tc": ("tc_update.cu", "trail_z.cuh", "tc_common.cuh"),
              "block_prep": ("tc_block.cu", "tc_common.cuh"), "block_y": ("tc_block.cu", "tc_common.cuh"),
              "block_u": ("tc_block.cu", "tc_common.cuh"),
              "apply_q": "apply_q.cu", "trsv": "refine.cu", "residual": "qr.cu",
              "assemble_f32": "assemble.cu", "assemble_f64": "assemble.cu", "copy_in": "qr.cu"}

BLK = 128          # outer block width of the blocked factorisation
SPLIT_PRODUCTS = 6  # bf16 products per fp32 product in the three-part split


def _blocked_flops(m_aug, n, nrhs):
    """Algorithmic flops of the outer-block updates of one factorisation: the Y pass
    Y = V^T [V | C] (2 m_p nbk n_ext per block, the block's own V^T V included) and the
    update pass C -= V Z (2 m_p nbk n_tr per block)."""
    y = u = 0.0
    for k in range(0, n, BLK):
        nbk = min(BLK, n - k)
        mp, n_ext = m_aug - k, n + nrhs - k
        n_tr = n_ext - nbk
        if n_tr <= 0:
            continue
        y += 2.0 * mp * nbk * n_ext
        u += 2.0 * mp * nbk * n_tr
    return y, u


def _block_launches(n, nrhs):
    """Y-pass plus update-pass launches of one factorisation (blocks with columns right of them)."""
    return 2 * sum(1 for k in range(0, n, BLK) if n + nrhs - k - min(BLK, n - k) > 0)


def _inner_flops(m_aug, n, nb):
    """Flops of the SIMT updates inside the outer blocks (4 m_p nb n_c per panel)."""
    f = 0.0
    for k in range(0, n, BLK):
        nbk = min(BLK, n - k)
        for kp in range(k, k + nbk, nb):
            c = min(nb, n - kp)
            f += 4.0 * (m_aug - kp) * c * (k + nbk - (kp + c))
    return f


def _algorithmic(kernel, m, n, m_aug, nb, nrhs, refine, nb_elem, blocked=True):
    """(unit, amount per solve) of the algorithmic cost of one kernel class in one
    solve: flops for the contractions (the tensor-core classes in bf16 products: six per
    fp32 product of the three-part split), bytes for memory-bound kernels (each operand
    moved once)."""
    e = nb_elem
    panels = [(k, min(nb, n - k)) for k in range(0, n, nb)]
    if kernel == "assemble_f32":
        return "bytes", 4.0 * m * n                     # each entry written once
    if kernel == "assemble_f64":
        return "bytes", 8.0 * m * n
    if kernel == "panel":                              # slice read + written once per panel
        return "bytes", sum(2.0 * (m_aug - k) * c * e for k, c in panels)
    if kernel == "block_y":
        return "flops", SPLIT_PRODUCTS * _blocked_flops(m_aug, n, nrhs)[0]
    if kernel == "block_u":
        return "flops", SPLIT_PRODUCTS * _blocked_flops(m_aug, n, nrhs)[1]
    if kernel == "block_prep":                         # V images written (12 B per V entry)
        return "bytes", sum(12.0 * (m_aug - k) * min(BLK, n - k) for k in range(0, n, BLK))
    if kernel == "trail_simt":
        if blocked:
            return "flops", _inner_flops(m_aug, n, nb)
        return "flops", sum(4.0 * (m_aug - k) * c * (n + nrhs - (k + c)) for k, c in panels)
    if kernel == "trail_tc":                           # panel-by-panel TF32x3: C read twice, written once
        return "bytes", sum((12.0 * (n + nrhs - (k + c)) + 4.0 * c + 8.0 * 32) * (m_aug - k)
                            for k, c in panels)
    if kernel == "apply_q":                            # V read twice per application
        return "bytes", refine * sum(2.0 * (m_aug - k) * c * e for k, c in panels)
    if kernel == "trsv":                               # upper triangle read once per solve
        return "bytes", (1 + refine) * 0.5 * n * n * e
    if kernel == "residual":                           # FP64 operator read once per residual
        return "bytes", refine * 8.0 * m * n
    if kernel == "copy_in":
        return "bytes", (4.0 + e) * m * n
    return "bytes", 0.0


def _secondary(fl, pl, wl, torch, ctx, dev, n_inverse):
    """The other rows of the hot path, timed outside the headline step: the full-size
    Bratu Newton run (Jacobian reassembled every step) in MIXED and FP64, and a batch of
    inverse-problem instances (factor, solve, sensor loss, adjoint gradient)."""
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    out = {}
    w = wl.bratu2d()
    xi, xb, W, b = t(w.x_int), t(w.x_bc), t(w.W), t(w.b)
    zi, zb = torch.zeros(w.n_int, dtype=torch.float64, device=dev), torch.zeros(w.n_bc, dtype=torch.float64, device=dev)
    xt = t(w.x_test)
    us = {}
    for name, prec in (("mixed", fl.PREC_MIXED), ("fp64", fl.PREC_FP64)):
        beta = torch.zeros(w.n_feat, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st = fl.fastlsq_newton(ctx, xi, xb, fl.Op(w.alpha, w.coef), fl.NL_EXP, w.nl_lam, w.lam_bc,
                                   zi, zb, W, b, w.scale, beta, max_iter=15, tol=1e-10, mu=w.mu,
                                   prec=prec, max_refine=64, refine_tol=1e-13)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        u = torch.empty(xt.shape[0], dtype=torch.float64, device=dev)
        fl.fastlsq_eval(ctx, xt, W, b, w.scale, beta, u)
        us[name] = u
        out[f"newton_{name}"] = {"seconds": sec, "iters": int(st.iters), "status": int(st.status),
                                 "res_norm_first": float(st.res_norm[0]),
                                 "res_norm_last": float(st.res_norm[st.iters]),
                                 "last_step_rel": float(st.step_rel[max(0, st.iters - 1)])}
    out["newton_mixed"]["rel_l2_vs_fp64_gpu"] = pl.rel_l2(us["mixed"], us["fp64"])
    out["newton_workload"] = ("bratu2d: Lap u + e^u = 0, [0,1]^2, 8192 interior + 1024 boundary rows, "
                              "2048 features sigma=6, mu=1e-10, Newton from beta=0, <=15 iterations")
    # inverse problem: observations from the forward map at theta_true, gradients at theta_0
    # the cubic Newton problems (Sec. 3.3 NL-Poisson, NL-Helmholtz k = 3): N(u) = u^3,
    # manufactured u*, sources and Dirichlet data from the GPU's problem catalogue
    for name, precs in (("nlpoisson2d", (("mixed", fl.PREC_MIXED), ("fp64", fl.PREC_FP64))),
                        ("nlhelmholtz2d", (("mixed", fl.PREC_MIXED),))):
        wc = getattr(wl, name)()
        xi, xb, Wc, bc, xt = t(wc.x_int), t(wc.x_bc), t(wc.W), t(wc.b), t(wc.x_test)
        f = torch.empty(wc.n_int, dtype=torch.float64, device=dev)
        g = torch.empty(wc.n_bc, dtype=torch.float64, device=dev)
        ue = torch.empty(xt.shape[0], dtype=torch.float64, device=dev)
        fl.fastlsq_rhs(ctx, wc.problem, fl.RHS_SOURCE, wc.params, xi, 1.0, f)
        fl.fastlsq_rhs(ctx, wc.problem, fl.RHS_EXACT, wc.params, xb, 1.0, g)
        fl.fastlsq_rhs(ctx, wc.problem, fl.RHS_EXACT, wc.params, xt, 1.0, ue)
        for pname, prec in precs:
            beta = torch.zeros(wc.n_feat, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, st = fl.fastlsq_newton(ctx, xi, xb, fl.Op(wc.alpha, wc.coef), fl.NL_CUBIC, wc.nl_lam, wc.lam_bc,
                                       f, g, Wc, bc, wc.scale, beta, max_iter=12, tol=1e-10, mu=wc.mu,
                                       prec=prec, max_refine=64, refine_tol=1e-13)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            u = torch.empty(xt.shape[0], dtype=torch.float64, device=dev)
            fl.fastlsq_eval(ctx, xt, Wc, bc, wc.scale, beta, u)
            out[f"newton_{name}_{pname}"] = {
                "seconds": sec, "iters": int(st.iters), "status": int(st.status),
                "seconds_per_iter": sec / max(1, int(st.iters)),
                "rel_l2_vs_exact": pl.rel_l2(u, ue), "last_step_rel": float(st.step_rel[max(0, st.iters - 1)]),
                "workload": (f"{name}: 8192 interior + 1024 boundary rows, 2048 features sigma={wc.sigma:g}, "
                             "u^3 term, manufactured u* = sin(pi x) sin(pi y) + x y / 2, mu=1e-10, <=12 iterations")}

    # the 1-D problems of Sec. 3.3 in true solver mode (f = 0, Dirichlet data of the exact
    # kink): Allen-Cahn eps = 0.1 (30 iterations) and steady Burgers nu = 0.1 with
    # continuation nu = 1, 0.5, 0.2, 0.1 (12 iterations per stage, 48 in all), both
    # warm-started from the linear part, 5000 interior points, 1500 features
    for name, stages, iters in (("allen_cahn1d", None, 30),
                                ("burgers1d", wl.burgers_stage_coef(0.1), 12)):
        w1 = getattr(wl, name)()
        dp1 = pl.upload(w1, dev)
        f1 = torch.zeros(w1.n_int, dtype=torch.float64, device=dev)
        g1 = torch.empty(w1.n_bc, dtype=torch.float64, device=dev)
        ue1 = torch.empty(dp1.x_test.shape[0], dtype=torch.float64, device=dev)
        fl.fastlsq_rhs(ctx, w1.problem, fl.RHS_EXACT, w1.params, dp1.x_bc, 1.0, g1)
        fl.fastlsq_rhs(ctx, w1.problem, fl.RHS_EXACT, w1.params, dp1.x_test, 1.0, ue1)
        for pname, prec in (("mixed", fl.PREC_MIXED), ("fp64", fl.PREC_FP64)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            beta, rc, sts = pl.newton_solve(ctx, dp1, f1, g1, prec=prec, max_iter=iters, tol=1e-10,
                                            stage_coef=stages)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            u = torch.empty(dp1.x_test.shape[0], dtype=torch.float64, device=dev)
            fl.fastlsq_eval(ctx, dp1.x_test, dp1.W, dp1.b, w1.scale, beta, u)
            n_it = sum(int(st.iters) for st in sts) + 1          # + the warm-start solve
            out[f"newton_{name}_{pname}"] = {
                "seconds": sec, "iters": n_it, "status": int(rc), "seconds_per_iter": sec / n_it,
                "rel_l2_vs_exact": pl.rel_l2(u, ue1),
                "workload": (f"{name}: {w1.n_int} interior + 2 boundary rows, {w1.n_feat} features "
                             f"sigma={w1.sigma:g}, f = 0, exact kink as Dirichlet data, mu=1e-10, warm start, "
                             + (f"<= {iters} iterations" if stages is None else
                                f"continuation nu = {', '.join(f'{-c[0]:g}' for c in stages)}, "
                                f"<= {iters} iterations per stage"))}

    # variable-coefficient operator (Sec. 3.8): div(nu grad u) = f as nu Lap u + grad nu .
    # grad u, four per-point terms assembled on the fly from the coefficient fields; MIXED
    # solves (2 refinement steps) timed one at a time, error vs u* and vs the FP64 solve
    wv = wl.varcoef2d()
    dpv = pl.upload(wv, dev, ctx=ctx)
    sv_m = pl.LinearSolver(ctx, dpv, prec=fl.PREC_MIXED, max_refine=2)
    for _ in range(3):
        sv_m.step()
    n_v = 10
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_v):
        sv_m.step()
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / n_v
    u_vm = sv_m.u_test()
    ue_v = sv_m.u_exact_test()
    sv_d = pl.LinearSolver(ctx, dpv, prec=fl.PREC_FP64)
    sv_d.step()
    u_vd = sv_d.u_test()
    out["varcoef2d"] = {
        "seconds_per_solve": sec, "solves_per_s": 1.0 / sec, "rel_l2_vs_exact": pl.rel_l2(u_vm, ue_v),
        "rel_l2_vs_fp64_gpu": pl.rel_l2(u_vm, u_vd), "fp64_rel_l2_vs_exact": pl.rel_l2(u_vd, ue_v),
        "workload": ("varcoef2d: div(nu grad u) = f, nu = 1 + x^2 + y^2/2, u* = sin(pi x) sin(2 pi y) + x y, "
                     "8192 interior + 1024 boundary rows, 2048 features sigma=6; per-point coefficient "
                     "terms nu, nu, nu_x, nu_y; MIXED, 2 refinement steps, one solve at a time")}
    del sv_m, sv_d, dpv

    # learnable bandwidth (Alg. 2): the gradient of the outer loss ||A beta* - rhs||^2 in
    # sigma (W = sigma W_hat) after each solve: residual, adjoint vector v (PCG), the
    # feature-weight gradient of both row blocks (on the fly, FP64) and the contraction
    # with W_hat.  Tikhonov mu = 1e-6: with much smaller mu the quantity is not
    # determined in FP64 at this size.  The whole evaluation (rhs, assembly, MIXED solve
    # refined by CGLS, gradient) is timed, the gradient alone too, and the gradient is
    # checked against central differences of the loss (h = 1e-4 sigma)
    import copy as _copy
    wbw = wl.helmholtz2d()
    wbw.mu = 1e-6
    W_hat = wbw.W / wbw.sigma

    def _bw_solver(sig):
        wq = _copy.copy(wbw)
        wq.W = sig * W_hat
        return pl.LinearSolver(ctx, pl.upload(wq, dev), prec=fl.PREC_MIXED, mu=wbw.mu, max_refine=64,
                               refine_mode=fl.REFINE_CGLS, refine_tol=1e-13)

    def _bw_once(sb):
        sb.build_rhs()
        sb.assemble()
        fac = sb.solve(keep=True)
        r, _, gout = sb.outer_grad(W_hat, fac=fac, max_iter=64)
        fl.fastlsq_factor_destroy(ctx, fac)
        return r, gout

    sb = _bw_solver(wbw.sigma)
    for _ in range(2):
        _bw_once(sb)
    n_bw = 5
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_bw):
        r_bw, gout = _bw_once(sb)
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / n_bw
    fac = sb.solve(keep=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_bw):
        sb.outer_grad(W_hat, fac=fac, max_iter=64)
    torch.cuda.synchronize()
    sec_g = (time.perf_counter() - t0) / n_bw
    fl.fastlsq_factor_destroy(ctx, fac)
    g_sigma = float(gout[-1].item())
    hb = 1e-4 * wbw.sigma
    lp = _bw_once(_bw_solver(wbw.sigma + hb))[0]
    lm = _bw_once(_bw_solver(wbw.sigma - hb))[0]
    fd = (float((lp * lp).sum()) - float((lm * lm).sum())) / (2 * hb)
    out["bandwidth_grad"] = {
        "seconds_per_eval": sec, "evals_per_s": 1.0 / sec, "gradient_ms": 1e3 * sec_g,
        "dL_dsigma": g_sigma, "fd_dL_dsigma": fd, "rel_diff_vs_fd": abs(g_sigma - fd) / abs(fd),
        "workload": ("helmholtz2d (9216 x 2048, sigma = 8, Tikhonov mu = 1e-6): outer loss "
                     "||A beta* - rhs||^2 of the learnable-bandwidth loop; per evaluation rhs, FP32+FP64 "
                     "assembly, MIXED solve with CGLS refinement, residual, v by PCG, dL/dW (FP64, on the "
                     "fly) and dL/dsigma; checked against central differences of the loss")}
    del sb

    # cached re-solves (App. G.5): factor the helmholtz2d operator once, then solve for
    # new right-hand sides (Q^T b, R^{-1}, two refinement steps) against the kept factor
    wr = wl.helmholtz2d()
    dpr = pl.upload(wr, dev)
    sr = pl.LinearSolver(ctx, dpr, prec=fl.PREC_MIXED, max_refine=2)
    sr.build_rhs()
    sr.assemble()
    fac = sr.solve(keep=True)
    n_resolve = 20
    rhs = sr.rhs.repeat(n_resolve, 1) * torch.linspace(0.5, 1.5, n_resolve, dtype=torch.float64,
                                                      device=dev).unsqueeze(1)
    betas = torch.zeros((n_resolve, wr.n_feat), dtype=torch.float64, device=dev)
    fl.fastlsq_factor_solve(ctx, fac, rhs[:1], betas[:1], max_refine=2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fl.fastlsq_factor_solve(ctx, fac, rhs, betas, max_refine=2)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    # the solution is linear in the right-hand side: u(1.5 b) = 1.5 u(b) on the test set
    # (beta itself is not determined elementwise: the system's condition number is large)
    fl.fastlsq_factor_destroy(ctx, fac)
    u_a = sr.u_test()
    u_b = sr.u_test(beta=betas[-1])
    lin = pl.rel_l2(u_b, 1.5 * u_a)
    out["resolve"] = {"rhs": n_resolve, "seconds": sec, "resolves_per_s": n_resolve / sec,
                      "u_rel_diff_scaled_rhs": lin,
                      "workload": ("helmholtz2d (9216 x 2048) MIXED factor kept; 20 right-hand sides, each Q^T b, "
                                   "R^{-1} and 2 classical refinement steps")}
    # L u at arbitrary points (the gradient of the helmholtz2d solution at 200,000 points)
    xg = torch.rand((200000, 2), dtype=torch.float64, device=dev, generator=torch.Generator(dev).manual_seed(7))
    gx = torch.empty(200000, dtype=torch.float64, device=dev)
    ops = [fl.Op([[1, 0]], [1.0]), fl.Op([[0, 1]], [1.0])]
    for o in ops:
        fl.fastlsq_eval_op(ctx, xg, o, dpr.W, dpr.b, wr.scale, sr.beta[0], gx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for o in ops:
        fl.fastlsq_eval_op(ctx, xg, o, dpr.W, dpr.b, wr.scale, sr.beta[0], gx)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    out["eval_grad"] = {"points": 200000, "components": 2, "seconds": sec,
                        "point_feature_pairs_per_s": 2 * 200000 * wr.n_feat / sec,
                        "workload": "d u/dx and d u/dy of the helmholtz2d solution (2048 features) at 200,000 points, FP64"}
    del sr, dpr

    out["inverse"] = _inverse_row(fl, pl, wl, torch, ctx, dev, n_inverse)
    return out


def _inverse_eval_fma(shapes, thin_q):
    """FP64 FMAs of one evaluation of a batch of (n_int, n_bc, n_feat) instances.  Thin-Q
    plan (the default): Qi^T s and Qi w over the interior rows (n_int n each) and two
    triangular solves (n^2 / 2 each): 2 n_int n + n^2 per instance.  Reflector plan: Q^T
    and Q each a dot pass and an update pass over the reflectors (2 (m_aug n - n^2 / 2)
    each) and the two solves: 4 m_aug n, m_aug = interior + boundary + Tikhonov rows."""
    if thin_q:
        return sum(2.0 * ni * n + float(n) ** 2 for ni, nb, n in shapes)
    return sum(4.0 * (ni + nb + n) * n for ni, nb, n in shapes)


def _inverse_row(fl, pl, wl, torch, ctx, dev, n_inst):
    """The batched inverse heat-source configuration: n_inst instances drawn with its
    recipe, factored once (FP64 QR, kept), then gradient evaluations of the whole batch,
    each one persistent launch, replayed from a captured CUDA graph and timed with
    events.  Reports factorisations/s of the setup and gradient evaluations/s (one
    evaluation = loss and dL/dtheta of one instance)."""
    ws = [wl.inverse_instance(q) for q in range(n_inst)]
    # a context of its own on a non-default stream (graph capture needs one)
    ctx = fl.Context(torch.device(dev).index or 0, stream=torch.cuda.Stream(device=dev))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch = pl.InverseBatch(ctx, ws, device=dev)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    batch.observe()
    for _ in range(2):
        batch.eval()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=ctx.stream):
        batch.eval()
    reps = 10
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(ctx.stream):                # replay() runs on the current stream
        g.replay()
        a.record(ctx.stream)
        for _ in range(reps):
            g.replay()
        b.record(ctx.stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    thin_q = batch.thin_q
    fma = _inverse_eval_fma([(w.n_int, w.n_bc, w.n_feat) for w in ws], thin_q)
    tfma = fma / (ms / 1e3) / 1e12
    out = {"instances": n_inst, "setup_s": setup_s, "factorizations_per_s": n_inst / setup_s,
           "ms_per_batch_eval": ms, "gradient_evals_per_s": n_inst / (ms / 1e3),
           "plan": "thin Q of the interior rows" if thin_q else "reflectors",
           "roofline": {"bound": "fp64", "achieved": tfma, "unit": "TFMA/s", "peak": 0.625,
                        "frac": tfma / 0.625, "work_fma_per_eval": fma,
                        "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (0.625 TFMA/s); a cuBLAS DGEMM "
                                       "on this pool measured 1.10 TFLOP/s"},
           "launch": batch.launch,
           "rows_range": [int(min(w.n_int for w in ws)), int(max(w.n_int for w in ws))],
           "features_range": [int(min(w.n_feat for w in ws)), int(max(w.n_feat for w in ws))],
           "loss_mean": float(sum(d["loss"].item() for d in batch.inst) / n_inst),
           "workload": ("steady inverse heat source -Lap u = s(x; theta), 4 Gaussians (16 parameters), "
                        "n_int ~ U{1024..8192}, n_feat ~ U{512..2048}, sigma = 8, mu = 1e-10, 64 sensors; "
                        "FP64 factor of [A; sqrt(mu) I] kept with the thin Q of its interior rows, per "
                        "evaluation Qi^T s, R^-1, R^-T, Qi w and the source gradient in one persistent "
                        "launch (CUDA graph replay)")}
    batch.close()
    del g
    ctx.close()
    return out


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
        return p, "of measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "of fallback"


def _traffic(cls):
    """ncu DRAM bytes per bf16 tensor flop of a kernel class, if a capture of the current
    sources is on record (profiles/ncu_traffic.json).  Both passes stream their operand
    once per launch (the Y pass reads the block's rows of [V | C], the update pass reads
    and writes C), so their traffic grows with the launch's flops at a fixed block
    width and a capture on a smaller workload scales to the bench's."""
    tpath = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(tpath):
        return None, None
    info = json.load(open(tpath)).get(cls)
    if not info or info.get("src_sha") != _src_sha(KERNEL_SRC.get(cls, "qr.cu")):
        return None, None
    return info.get("bytes_per_tensor_flop"), info.get("captured_on")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="poisson5d", choices=sorted(WORKLOADS))
    ap.add_argument("--refine", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tensor-core", type=int, default=1, choices=[0, 1, 2],
                    help="1: two-level blocked QR with tcgen05 outer-block updates (three-part "
                         "bf16 split); 2: panel-by-panel tcgen05 TF32x3; 0: SIMT FP32")
    ap.add_argument("--trsv-fp32", type=int, default=1, choices=[0, 1],
                    help="1: FP32 substitution in the triangular solves of classical refinement")
    ap.add_argument("--no-extras", action="store_true", help="skip the other rows of the hot path")
    ap.add_argument("--inverse-instances", type=int, default=256)
    ap.add_argument("--instances", type=int, default=0,
                    help="independent full-size solves per step, each on its own stream "
                         "(0: the workload's default, 4 for poisson5d, 8 for helmholtz2d)")
    ap.add_argument("--overlap", type=int, default=1, choices=[0, 1],
                    help="assemble the FP64 operator on a side stream during the factorisation")
    ap.add_argument("--fused-lookahead", type=int, default=1, choices=[0, 1],
                    help="with look-ahead, 1: panels apply the previous panel's update in their prologue")
    ap.add_argument("--split-rows", type=int, default=256,
                    help="least rows per split of the SIMT updates inside an outer block")
    ap.add_argument("--lookahead", type=int, default=0, choices=[0, 1],
                    help="panel-by-panel modes: 1 factors the next panel on a second stream")
    ap.add_argument("--asm64-ctas", type=int, default=0, choices=range(0, 9),
                    help="FP64 assembly: 0 one CTA per tile; k a persistent grid of k CTAs per SM")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2602_10541_gb300 import _build
    from paper_2602_10541_gb300 import fastlsq as fl
    from paper_2602_10541_gb300 import pipeline as pl
    from paper_2602_10541_gb300 import workloads as wl

    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    if not _build.up_to_date():
        _build.build()
    name = args.workload
    cfg = WORKLOADS[name]
    make = getattr(wl, name)
    stream = torch.cuda.current_stream(local)
    # each rank solves its own instances (replicas: a solve does not shard); a step is
    # B independent full-size solves, one context and stream each
    _, hi_prio = torch.cuda.Stream.priority_range()
    B = args.instances if args.instances > 0 else cfg["instances"]
    ctxs, solvers = [], []
    for i in range(B):
        c = fl.Context(local, stream=torch.cuda.Stream(device=local, priority=hi_prio))
        fl.fastlsq_set_option(c, fl.OPT_TENSOR_CORE, args.tensor_core)
        fl.fastlsq_set_option(c, fl.OPT_TRSV_FP32, args.trsv_fp32)
        fl.fastlsq_set_option(c, fl.OPT_LOOKAHEAD, args.lookahead)
        fl.fastlsq_set_option(c, fl.OPT_SPLIT_ROWS, args.split_rows)
        fl.fastlsq_set_option(c, fl.OPT_FUSED_LOOKAHEAD, args.fused_lookahead)
        fl.fastlsq_set_option(c, fl.OPT_FP64_ASSEMBLY_CTAS, args.asm64_ctas)
        wi = make(seed_offset=rank * B + i)
        with torch.cuda.stream(c.stream):
            dpi = pl.upload(wi, dev)
            solvers.append(pl.LinearSolver(c, dpi, prec=fl.PREC_MIXED, max_refine=args.refine,
                                           overlap=bool(args.overlap)))
        ctxs.append(c)
    torch.cuda.synchronize()
    ctx, solver = ctxs[0], solvers[0]          # instance 0: profiles, accuracy, assembly alone
    dp, w = solver.dp, solver.dp.w
    batch = pl.ConcurrentSolves(solvers)
    m, n = w.n_rows, w.n_feat
    m_aug = m + (n if w.mu > 0 else 0)

    for _ in range(args.warmup):
        batch.step(stream)
    torch.cuda.synchronize()

    # per-class device times of instance 0 (a pre-pass with events on every class)
    fl.fastlsq_profile_enable(ctx, None)
    for _ in range(2):
        batch.step(stream)
    prof_pre = fl.fastlsq_profile_read(ctx)
    dominant = max(prof_pre, key=lambda k: prof_pre[k][1])
    # inside the timed region, events on the tensor-core update classes only
    tc_classes = ["block_y", "block_u"] if args.tensor_core == 1 else (
        ["trail_tc"] if args.tensor_core == 2 else ["trail_simt"])
    fl.fastlsq_profile_enable(ctx, tc_classes)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))                         # evict L2 (outside the step events)
        ev_s[i].record(stream)
        batch.step(stream)
        ev_e[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [ev_s[i].elapsed_time(ev_e[i]) for i in range(args.steps)]
    total_ms = sum(step_ms)
    prof = fl.fastlsq_profile_read(ctx)
    fl.fastlsq_profile_enable(ctx, [])
    launches = B * sum(v[0] for v in prof.values())     # instances run the same launches
    value, total_ms = _job_throughput(total_ms, args.steps, world, dev)
    value *= B

    with torch.cuda.stream(ctx.stream):
        solver.solve(stats=True)
    solve_stats = solver.stats
    nb = solve_stats.nb
    blocked = args.tensor_core == 1
    peaks, peak_tag = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    nsm = torch.cuda.get_device_properties(local).multi_processor_count

    # roofline of the factorisation's trailing update (the contraction of Sec. 2.3's QR):
    # algorithmic flops per launch over the event time of its launches in the timed region
    units = 0.0
    for cls in tc_classes:
        units += _algorithmic(cls, m, n, m_aug, nb, 1, args.refine, 4, blocked)[1]
    tc_launches = sum(prof[c][0] for c in tc_classes)
    tc_ms = sum(prof[c][1] for c in tc_classes)
    if args.tensor_core == 1:
        bound, unit = "tensor", "TFLOP/s"
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0))
        peak_src = f"MEASURED_PEAKS.json bf16_tflops_sustained ({peak_tag}): bf16 operands"
        work_note = ("bf16 tensor flops: 6 products (three-part split) x 2 m_p nbk n per outer block, "
                     "Y pass (n = columns right of the block plus the block's own) and update pass")
    elif args.tensor_core == 2:
        bound, unit = "tensor", "TFLOP/s"
        peak = 0.5 * peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0))
        peak_src = f"MEASURED_PEAKS.json bf16_tflops_sustained x 0.5 (nominal tf32 : bf16) ({peak_tag})"
        units = sum(3 * 4.0 * (m_aug - k) * min(nb, n - k) * (n + 1 - (k + min(nb, n - k)))
                    for k in range(0, n, nb))
        work_note = "tf32 tensor flops: 3 products (TF32x3) x 4 m_p nb n_c per panel"
    else:
        bound, unit = "alu", "TFLOP/s"
        peak = 2.0 * 128 * nsm * sm_mhz * 1e6 / 1e12
        peak_src = f"derived: {nsm} SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz"
        work_note = "FP32 flops: 4 m_p nb n_c per panel"
    per_launch = units * args.steps / max(1, tc_launches)
    achieved = units * args.steps / (tc_ms / 1e3) / 1e12 if tc_ms > 0 else 0.0
    traffic = None
    tsrc = None
    if args.tensor_core == 1:
        ty, sy = _traffic("block_y")
        tu, su = _traffic("block_u")
        if ty is not None and tu is not None:
            fy = _algorithmic("block_y", m, n, m_aug, nb, 1, args.refine, 4, blocked)[1]
            fu = _algorithmic("block_u", m, n, m_aug, nb, 1, args.refine, 4, blocked)[1]
            traffic = (ty * fy + tu * fu) / max(1, _block_launches(n, 1))
            tsrc = f"ncu DRAM bytes per bf16 tensor flop on {sy}, scaled to this workload's launches"
    roofline = {"kernel": "+".join(tc_classes), "bound": bound, "achieved": achieved, "peak": peak,
                "unit": unit, "frac": achieved / peak, "traffic": traffic, "traffic_source": tsrc,
                "launches": tc_launches, "avg_launch_us": 1e3 * tc_ms / max(1, tc_launches),
                "work_per_launch": per_launch, "work": work_note, "peak_source": peak_src,
                "algorithmic_fp32_tflops": achieved / (SPLIT_PRODUCTS if args.tensor_core == 1 else
                                                       (3 if args.tensor_core == 2 else 1)),
                "dominant_class_of_step": dominant,
                "concurrent_instances": B}     # each launch shares the GPU with B - 1 other solves
    breakdown = {k: {"launches_per_solve": v[0] / 2.0, "ms_per_solve": v[1] / 2.0}
                 for k, v in prof_pre.items() if v[0]}
    for kname, v in breakdown.items():
        ukind, amount = _algorithmic(kname, m, n, m_aug, nb, 1, args.refine, 4, blocked)
        if amount <= 0 or v["ms_per_solve"] <= 0:
            continue
        if ukind == "flops":
            if kname in ("block_y", "block_u"):
                pk, bd = peaks.get("bf16_tflops_sustained", 1700.0), "tensor"
            else:
                pk, bd = 2.0 * 128 * nsm * sm_mhz * 1e6 / 1e12, "alu"
            v["roofline"] = {"achieved": amount / (v["ms_per_solve"] / 1e3) / 1e12, "peak": pk,
                             "unit": "TFLOP/s", "bound": bd}
        else:
            v["roofline"] = {"achieved": amount / (v["ms_per_solve"] / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                             "bound": "hbm"}
        v["roofline"]["frac"] = v["roofline"]["achieved"] / v["roofline"]["peak"]

    # accuracy: mixed result vs the plain FP64 GPU path and vs the exact solution
    # (instance 0, on the default stream from here on except in the end-to-end batch)
    torch.cuda.synchronize()
    s0 = ctx.stream
    fl.fastlsq_set_stream(ctx, stream)
    u_mixed = solver.u_test()
    ue = solver.u_exact_test()
    s64 = pl.LinearSolver(ctx, dp, prec=fl.PREC_FP64)
    fl.fastlsq_set_option(ctx, fl.OPT_LOOKAHEAD, 1)   # one solve alone: the library default
    torch.cuda.synchronize()
    t64 = time.perf_counter()
    s64.step()
    torch.cuda.synchronize()
    fp64_ms = 1e3 * (time.perf_counter() - t64)
    fl.fastlsq_set_option(ctx, fl.OPT_LOOKAHEAD, args.lookahead)
    u64 = s64.u_test()
    accuracy = {"rel_l2_vs_fp64_gpu": pl.rel_l2(u_mixed, u64), "rel_l2_vs_exact": pl.rel_l2(u_mixed, ue),
                "fp64_gpu_rel_l2_vs_exact": pl.rel_l2(u64, ue), "fp64_gpu_ms_per_solve": fp64_ms,
                "fp64_gpu_solves_per_s": 1e3 / fp64_ms,
                "resid_norms": list(solve_stats.resid_norm[: args.refine + 1])}
    del s64
    torch.cuda.empty_cache()

    # one solve alone (instance 0, the library defaults: look-ahead on), for the latency
    # of a solve
    fl.fastlsq_set_option(ctx, fl.OPT_LOOKAHEAD, 1)
    torch.cuda.synchronize()
    one = []
    for _ in range(4):
        t0 = time.perf_counter()
        solver.step()
        torch.cuda.synchronize()
        one.append(time.perf_counter() - t0)
    fl.fastlsq_set_option(ctx, fl.OPT_LOOKAHEAD, args.lookahead)
    single = {"ms_per_solve": 1e3 * min(one[1:]), "solves_per_s": 1.0 / min(one[1:]), "lookahead": True}

    # assembly alone (FP32 operator, both row blocks), Gentries/s
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    asm_ms = 0.0
    for i in range(args.steps):
        flush.fill_(float(i))
        ea.record(stream)
        fl.fastlsq_assemble(ctx, fl.F32, dp.x_int, dp.op_int, 1.0, dp.W, dp.b, w.scale, solver.A32, 0)
        fl.fastlsq_assemble(ctx, fl.F32, dp.x_bc, dp.op_bc, w.lam_bc, dp.W, dp.b, w.scale,
                            solver.A32, w.n_int)
        eb.record(stream)
        torch.cuda.synchronize()
        asm_ms += ea.elapsed_time(eb)
    asm_rate = args.steps * m * n / (asm_ms / 1e3)
    sfu = nsm * 16 * sm_mhz * 1e6
    assembly = {"gentries_per_s": asm_rate / 1e9, "entries": m * n,
                "hbm_write_gbs": 4 * asm_rate / 1e9, "hbm_frac": 4 * asm_rate / 1e9 / hbm,
                "sfu_bound_gentries_per_s": sfu / 1e9, "sfu_frac": asm_rate / sfu,
                "sfu_bound_source": f"derived: {nsm} SMs x 16 sin/clk x {sm_mhz:.0f} MHz"}

    # end to end through the C ABI with host buffers: every instance's inputs from
    # pinned host memory, its solution back, each step
    torch.cuda.synchronize()
    fl.fastlsq_set_stream(ctx, s0)
    pin = lambda t: t.detach().cpu().pin_memory()
    h_in = [[pin(t) for t in (sv.dp.x_int, sv.dp.x_bc, sv.dp.W, sv.dp.b)] for sv in solvers]
    h_beta = [torch.empty_like(sv.beta, device="cpu").pin_memory() for sv in solvers]
    bi = sum(t.numel() * t.element_size() for h in h_in for t in h)
    bo = sum(t.numel() * t.element_size() for t in h_beta)
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        for sv, h in zip(solvers, h_in):
            for d, hh in zip((sv.dp.x_int, sv.dp.x_bc, sv.dp.W, sv.dp.b), h):
                d.copy_(hh, non_blocking=True)
        batch.step(stream)
        for sv, hb in zip(solvers, h_beta):
            hb.copy_(sv.beta, non_blocking=True)
        stream.synchronize()
    e2e_s = time.perf_counter() - t0
    fl.fastlsq_set_stream(ctx, stream)
    e2e = {"value": world * B * e2e_steps / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": bi,
           "d2h_bytes_per_step": bo}
    del batch, solvers, solver
    torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        sample = cfg["cpu_sample"]
        t = _oracle_solve_seconds(name, sample)
        cpu = {"value": 1.0 / (t * _scale_ratio(name, sample)), "unit": "solves/s", "cores": 1,
               "kind": "oracle", "cpu": _cpu_model(), "nproc": os.cpu_count(),
               "sample": _sample_text(name, sample, t)}

    extras = None
    if rank == 0 and not args.no_extras:
        # one solve, Newton run or instance at a time: look-ahead on (the library default)
        fl.fastlsq_set_option(ctx, fl.OPT_LOOKAHEAD, 1)
        extras = _secondary(fl, pl, wl, torch, ctx, dev, args.inverse_instances)
        if name != "helmholtz2d":
            extras["helmholtz2d_concurrent"] = _helmholtz_row(fl, pl, wl, torch, dev, local, args)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": cfg["desc"], "n_rows": m, "n_feat": n,
                           "precision": (f"mixed: FP32 assembly and Householder QR (outer-block updates on "
                                         f"tcgen05, three-part bf16 split), FP64 residual, {args.refine} "
                                         f"refinement steps"),
                           "tensor_core_updates": int(solve_stats.tensor_core),
                           "panel_nb": nb, "outer_block": BLK if blocked else None,
                           "lookahead": bool(args.lookahead), "split_rows": args.split_rows,
                           "fp64_assembly_ctas_per_sm": args.asm64_ctas,
                           "fused_lookahead": bool(args.fused_lookahead),
                           "l2": "flushed between steps (256 MiB write outside the step events)",
                           "instances_per_step": B,
                           "concurrency": (f"{B} independent instances (seeds) of the workload per step, "
                                           "each on its own context and stream"),
                           "parallelism": "replicas" if world > 1 else "single"},
                "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
                "clocks": clk, "accuracy": accuracy, "single_solve": single, "assembly": assembly,
                "kernels": breakdown, "other_rows": extras, "wall_s_timed": wall}
        print(json.dumps(line), flush=True)
    for c in ctxs:
        c.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def _helmholtz_row(fl, pl, wl, torch, dev, local, args):
    """The 2-D Helmholtz configuration (9216 x 2048) as a row: 8 concurrent solves per
    step, device-timed, and the MIXED solution against the FP64 GPU path."""
    _, hi_prio = torch.cuda.Stream.priority_range()
    ctxs, solvers = [], []
    for i in range(8):
        c = fl.Context(local, stream=torch.cuda.Stream(device=local, priority=hi_prio))
        fl.fastlsq_set_option(c, fl.OPT_TENSOR_CORE, args.tensor_core)
        fl.fastlsq_set_option(c, fl.OPT_LOOKAHEAD, 0)
        with torch.cuda.stream(c.stream):
            solvers.append(pl.LinearSolver(c, pl.upload(wl.helmholtz2d(seed_offset=i), dev),
                                           prec=fl.PREC_MIXED, max_refine=args.refine))
        ctxs.append(c)
    batch = pl.ConcurrentSolves(solvers)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        batch.step(stream)
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = 10
    torch.cuda.synchronize()
    ea.record(stream)
    for _ in range(steps):
        batch.step(stream)
    eb.record(stream)
    torch.cuda.synchronize()
    ms = ea.elapsed_time(eb)
    s0 = solvers[0]
    torch.cuda.synchronize()
    fl.fastlsq_set_stream(s0.ctx, stream)
    um = s0.u_test()
    s64 = pl.LinearSolver(s0.ctx, s0.dp, prec=fl.PREC_FP64)
    s64.step()
    u64 = s64.u_test()
    ue = s0.u_exact_test()
    out = {"solves_per_s": 8 * steps / (ms / 1e3), "instances_per_step": 8,
           "rel_l2_vs_fp64_gpu": pl.rel_l2(um, u64), "rel_l2_vs_exact": pl.rel_l2(um, ue),
           "workload": WORKLOADS["helmholtz2d"]["desc"]}
    torch.cuda.synchronize()
    for c in ctxs:
        c.close()
    return out


if __name__ == "__main__":
    main()
