"""fastlsq_eval_noalloc, the evaluation entry point whose scratch is a fixed array
inside the library (no device allocation), against fastlsq_eval on the same inputs.
It exists for callers that cannot call cudaMalloc mid-run: a service holding all of its
device memory from start-up, which must not fail or stall on an allocation during a
request, or code inside a custom allocator's callbacks, which must not re-enter it.

Collected last (file name) so that it also runs after every other GPU test in the
same process; it passes alone as well.
"""
import numpy as np
import pytest
import torch

from paper_2602_10541_gb300 import fastlsq as fl

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _inputs(rng, n_eval, n_feat, d):
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)
    return (t(rng.uniform(0.0, 1.0, (n_eval, d))), t(rng.normal(0.0, 8.0, (n_feat, d))),
            t(rng.uniform(0.0, 2 * np.pi, n_feat)), t(rng.normal(0.0, 1.0, n_feat)))


def test_noalloc_eval_equals_eval_on_two_calls_in_a_row():
    ctx = fl.Context(0)
    rng = np.random.default_rng(2026)
    # two calls in a row with different shapes (the second reuses the scratch the
    # first wrote), each compared with the allocating entry point bit for bit
    for n_eval, n_feat, d in ((5000, 2048, 2), (777, 300, 5)):
        x, W, b, beta = _inputs(rng, n_eval, n_feat, d)
        scale = 1.0 / np.sqrt(n_feat)
        u_ref = torch.empty(n_eval, dtype=torch.float64, device=DEV)
        u = torch.full((n_eval,), float("nan"), dtype=torch.float64, device=DEV)
        fl.fastlsq_eval(ctx, x, W, b, scale, beta, u_ref)
        fl.fastlsq_eval_noalloc(ctx, x, W, b, scale, beta, u)
        torch.cuda.synchronize()
        assert torch.equal(u, u_ref)


def test_noalloc_eval_rejects_requests_beyond_its_scratch():
    ctx = fl.Context(0)
    rng = np.random.default_rng(7)
    n_feat = 2048                           # 16 column splits of 128
    n_eval = (1 << 19) // 16 + 1            # one point more than the scratch holds
    x, W, b, beta = _inputs(rng, n_eval, n_feat, 2)
    u = torch.zeros(n_eval, dtype=torch.float64, device=DEV)
    with pytest.raises(fl.FastLSQError):
        fl.fastlsq_eval_noalloc(ctx, x, W, b, 1.0, beta, u)
    assert float(u.abs().max()) == 0.0      # nothing was launched


def test_noalloc_eval_rejects_too_many_features():
    """More features than the library's limit (16384) is an invalid argument, not a
    launch with a column grid past the hardware's limit."""
    ctx = fl.Context(0)
    rng = np.random.default_rng(11)
    x, W, b, beta = _inputs(rng, 1, 16385, 2)
    u = torch.zeros(1, dtype=torch.float64, device=DEV)
    with pytest.raises(fl.FastLSQError) as e:
        fl.fastlsq_eval_noalloc(ctx, x, W, b, 1.0, beta, u)
    assert e.value.code == -1
    with pytest.raises(fl.FastLSQError) as e:
        fl.fastlsq_eval(ctx, x, W, b, 1.0, beta, u)
    assert e.value.code == -1
