"""A whole MIXED linear-solve step (rhs, FP32 assembly, FP64 assembly on the side stream,
QR with look-ahead on the context's second stream, tensor-core trailing updates, solve and
classical refinement) issues no host synchronisation, so it can be captured into a CUDA graph;
a replay reproduces the eager step's beta bit for bit.  (Runs late in the suite: a failed
capture would end the stream's capture with an error rather than a fault.)"""
import numpy as np
import pytest
import torch

from paper_2602_10541_gb300 import fastlsq as fl
from paper_2602_10541_gb300 import pipeline as pl
from paper_2602_10541_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_linear_solve_step_replays_from_a_cuda_graph():
    s = torch.cuda.Stream()
    ctx = fl.Context(0, stream=s)
    w = wl.helmholtz2d(n_int=2048, n_bc=256, n_feat=512)
    with torch.cuda.stream(s):
        dp = pl.upload(w, "cuda:0")
        sv = pl.LinearSolver(ctx, dp, prec=fl.PREC_MIXED, max_refine=2)
        for _ in range(2):                      # workspaces and kernel attributes set up
            sv.step()
        sv.step()
    torch.cuda.synchronize()
    beta_eager = sv.beta.clone()
    sv.beta.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sv.step()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(sv.beta, beta_eager)
    sv.beta.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(sv.beta, beta_eager)
    u, ue = sv.u_test(), sv.u_exact_test()      # on the context's stream
    torch.cuda.synchronize()
    assert pl.rel_l2(u, ue) < 1e-6
