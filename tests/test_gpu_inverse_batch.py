"""The pre-factored batch of inverse-problem instances (Sec. 3.8: factor once, two
triangular solves per evaluation; Sec. 2.5: gradients through the solve) evaluated in
one persistent launch, against the FP64 oracle.

Instances follow the batched configuration's recipe (W ~ N(0, 8^2 I), uneven numbers
of points and features, one with fewer rows than features before the sqrt(mu) rows),
at sizes the oracle factors in seconds.  Bars: the loss to 1e-6 relative (the loss is
a mean of squared residuals of the size of the noise, so an absolute error delta in
u_s moves it by about 2 delta / 1e-3); dL/dtheta to 2e-5 of its largest component
against the oracle's adjoint (the accuracy the FP64 forward map itself reaches, its
condition number being near 1e8), and against central differences (h = 1e-6) of the
GPU loss; beta to 1e-6 of its size on the sensors (u_s)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_10541_gb300 import fastlsq as fl
from paper_2602_10541_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
MU = 1e-10
OP = fl.Op([[2, 0], [0, 2]], [-1.0, -1.0])

# (n_int, n_feat): 400 interior + 48 boundary rows against 520 features is the case
# with fewer rows than features before the sqrt(mu) rows
SHAPES = [(1024, 512), (1800, 384), (400, 520), (2048, 512), (1300, 200), (800, 700), (500, 600),
          (1536, 256)]


@pytest.fixture(scope="module")
def ctx():
    return fl.Context(0)


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _oracle(w, theta, y):
    A_int = oracle.assemble(w.x_int, w.alpha, w.coef, w.W, w.b, w.scale)
    A_bc = oracle.assemble(w.x_bc, np.zeros((1, 2), np.int32), [1.0], w.W, w.b, w.scale,
                           row_weight=w.lam_bc)
    A = np.vstack([A_int, A_bc])
    Hs = oracle.assemble(w.sensors, np.zeros((1, 2), np.int32), [1.0], w.W, w.b, w.scale)
    f = oracle.problem_source(oracle.GAUSS_SOURCE_2D, w.x_int, theta)
    out = oracle.inverse_adjoint(A, np.concatenate([f, np.zeros(w.n_bc)]), Hs, y, MU)
    out["dtheta"] = oracle.gauss_source_grad(w.x_int, theta, out["grad_rhs"][: w.n_int])
    return out


def _device(w, y, theta):
    return dict(x_int=_t(w.x_int), x_bc=_t(w.x_bc), W=_t(w.W), b=_t(w.b), sensors=_t(w.sensors),
                y_obs=_t(y), theta=_t(theta),
                beta=torch.zeros(w.n_feat, dtype=torch.float64, device=DEV),
                loss=torch.zeros(1, dtype=torch.float64, device=DEV),
                dtheta=torch.zeros(16, dtype=torch.float64, device=DEV))


@pytest.fixture(scope="module")
def batch():
    cases, dev = [], []
    for q, (ni, nf) in enumerate(SHAPES):
        w = wl.inverse_instance(q, n_int=ni, n_feat=nf)
        y = _oracle(w, w.params, np.zeros(64))["u_s"] + w.noise
        cases.append((w, y, _oracle(w, w.theta0, y)))
        dev.append(_device(w, y, w.theta0))
    return cases, dev


@pytest.mark.parametrize("thin_q", [1, 0])
@pytest.mark.parametrize("threads,ctas,cluster", [(256, 1, 1), (512, 1, 1), (256, 2, 1), (256, 1, 2),
                                                  (512, 1, 2), (512, 2, 4)])
def test_persistent_batch_matches_oracle(ctx, batch, threads, ctas, cluster, thin_q):
    """Both forms of the plan: the explicit thin Q of the interior rows (default) and
    the reflectors alone."""
    cases, dev = batch
    fl.fastlsq_set_option(ctx, fl.OPT_INVERSE_THIN_Q, thin_q)
    try:
        plan = fl.fastlsq_inverse_prepare(ctx, dev, OP, 4, mu=MU)
    finally:
        fl.fastlsq_set_option(ctx, fl.OPT_INVERSE_THIN_Q, 1)
    for d in dev:
        d["loss"].zero_()
        d["dtheta"].zero_()
    fl.fastlsq_inverse_eval(ctx, plan, threads=threads, ctas_per_sm=ctas, cluster=cluster)
    torch.cuda.synchronize()
    for (w, y, ref), d in zip(cases, dev):
        assert abs(d["loss"].item() - ref["loss"]) <= 1e-6 * ref["loss"], (w.name, d["loss"].item(), ref["loss"])
        u_s = oracle.eval_u(w.sensors, w.W, w.b, w.scale, d["beta"].cpu().numpy())
        assert np.abs(u_s - ref["u_s"]).max() <= 1e-6 * np.abs(ref["u_s"]).max(), w.name
        g = d["dtheta"].cpu().numpy()
        assert np.abs(g - ref["dtheta"]).max() <= 2e-5 * np.abs(ref["dtheta"]).max(), (w.name, g, ref["dtheta"])
    plan.close()


def test_persistent_batch_gradient_matches_central_differences(ctx, batch):
    """dL/dtheta of one instance against FP64 central differences of the GPU loss
    (h = 1e-6 on every parameter), both from the persistent evaluation."""
    cases, dev = batch
    q = 3                                                  # 2048 + 256 rows x 512 features
    d = dev[q]
    plan = fl.fastlsq_inverse_prepare(ctx, [d], OP, 4, mu=MU)
    theta0 = d["theta"].clone()
    fl.fastlsq_inverse_eval(ctx, plan)
    torch.cuda.synchronize()
    g = d["dtheta"].cpu().numpy().copy()
    h = 1e-6
    fd = np.zeros(16)
    for k in range(16):
        vals = []
        for sgn in (1.0, -1.0):
            d["theta"].copy_(theta0)
            d["theta"][k] += sgn * h
            fl.fastlsq_inverse_eval(ctx, plan)
            torch.cuda.synchronize()
            vals.append(d["loss"].item())
        fd[k] = (vals[0] - vals[1]) / (2 * h)
    d["theta"].copy_(theta0)
    plan.close()
    assert np.abs(g - fd).max() <= 1e-4 * np.abs(fd).max(), (g, fd)


@pytest.mark.parametrize("thin_q,cluster", [(1, 1), (1, 2), (0, 2)])
def test_persistent_batch_replays_from_a_cuda_graph(ctx, batch, thin_q, cluster):
    """The evaluation allocates nothing and never synchronises: captured once, a replay
    after theta changes gives the eager results bit for bit (at a fixed cluster size
    the sums run in a fixed order)."""
    cases, dev = batch
    s = torch.cuda.Stream()
    gctx = fl.Context(0, stream=s)
    fl.fastlsq_set_option(gctx, fl.OPT_INVERSE_THIN_Q, thin_q)
    sub = dev[:4]
    with torch.cuda.stream(s):
        plan = fl.fastlsq_inverse_prepare(gctx, sub, OP, 4, mu=MU)
        fl.fastlsq_inverse_eval(gctx, plan, cluster=cluster)   # kernel attributes set before capture
    torch.cuda.synchronize()
    theta_b = [d["theta"].clone() * 1.01 for d in sub]
    for d, tb in zip(sub, theta_b):
        d["theta"].copy_(tb)
    with torch.cuda.stream(s):
        fl.fastlsq_inverse_eval(gctx, plan, cluster=cluster)
    torch.cuda.synchronize()
    eager = [(d["loss"].clone(), d["dtheta"].clone(), d["beta"].clone()) for d in sub]
    for d in sub:
        d["loss"].zero_()
        d["dtheta"].zero_()
        d["beta"].zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fl.fastlsq_inverse_eval(gctx, plan, cluster=cluster)
    g.replay()
    torch.cuda.synchronize()
    for d, (l, dt, b) in zip(sub, eager):
        assert torch.equal(d["loss"], l) and torch.equal(d["dtheta"], dt) and torch.equal(d["beta"], b)
    for (w, _, _), d in zip(cases[:4], sub):
        d["theta"].copy_(_t(w.theta0))
    plan.close()
    gctx.close()


def test_inverse_plan_rejects_bad_arguments(ctx, batch):
    _, dev = batch
    with pytest.raises(fl.FastLSQError) as e:
        fl.fastlsq_inverse_prepare(ctx, dev[:1], OP, 0, mu=MU)
    assert e.value.code == -1
    with pytest.raises(fl.FastLSQError) as e:
        fl.fastlsq_inverse_prepare(ctx, dev[:1], OP, 4, mu=0.0)
    assert e.value.code == -1
    plan = fl.fastlsq_inverse_prepare(ctx, dev[:1], OP, 4, mu=MU)
    with pytest.raises(fl.FastLSQError) as e:
        fl.fastlsq_inverse_eval(ctx, plan, threads=128)
    assert e.value.code == -1
    with pytest.raises(fl.FastLSQError) as e:
        fl.fastlsq_inverse_eval(ctx, plan, cluster=3)
    assert e.value.code == -1
    plan.close()
    fl.fastlsq_sync(ctx)
