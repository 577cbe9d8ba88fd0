"""Ladder-predictor MLP kernels (fp32) against the float64 oracle.

Tolerance: every output is a sum of at most ~260 fp32 products per layer,
four layers deep, so the relative error of fp32 against float64 is a few
times K * 2^-24 ~ 2e-5; the tests allow 2e-4 (relative, per tensor norm)."""
import numpy as np
import pytest

from paper_2503_10302_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 2e-4


@pytest.fixture(scope="module")
def pc():
    from paper_2503_10302_gb300 import build, pcomp
    build.build()
    return pcomp


def _data(B, seed):
    from oracle import mlp
    rng = np.random.default_rng(seed)
    X = np.zeros((B, mlp.N_IN), np.float32)
    X[:, 0] = rng.choice([6, 8, 10, 12, 14, 16], size=B) / 16
    X[:, 1] = 0.5 + 0.02 * rng.normal(size=B)
    X[:, 2] = 0.5 + 0.02 * rng.normal(size=B)
    h = rng.random(size=(B, 4, 64)) ** 4
    X[:, 3:] = (h / h.sum(-1, keepdims=True)).reshape(B, -1)
    Y = (0.5 + np.cumsum(0.04 + 0.05 * rng.random(size=(B, 32)), axis=1)).astype(np.float32)
    return X, Y


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("B", [1, 37, 256])
def test_forward_matches_oracle(pc, B):
    from oracle import mlp
    params = W.mlp_init(mlp.SIZES, 1)
    X, _ = _data(B, B)
    ctx = pc.Context(0, 0)
    m = pc.Mlp(ctx.h, params, beta_min=0.1)
    beta = m.forward(X)
    ref, _ = mlp.forward(params, X.astype(np.float64), beta_min=0.1)
    assert _rel(beta, ref) < TOL
    m.close()
    ctx.close()


def test_gradients_match_oracle(pc):
    from oracle import mlp
    params = W.mlp_init(mlp.SIZES, 2)
    params = [(w, b + 0.01) for w, b in params]
    X, Y = _data(64, 3)
    ctx = pc.Context(0, 0)
    m = pc.Mlp(ctx.h, params)
    loss, grads = m.grads(X, Y)
    loss_ref, grads_ref = mlp.loss_and_grads(params, X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss - loss_ref) < TOL * loss_ref
    for (gW, gb), (rW, rb) in zip(grads, grads_ref):
        assert _rel(gW, rW) < TOL and _rel(gb, rb) < TOL
    m.close()
    ctx.close()


def test_adam_steps_match_oracle(pc):
    """Three train steps; the oracle's Adam is fed the GPU's own fp32
    gradients (deterministic: fixed-order reductions), so the comparison
    isolates the update arithmetic (fp32 vs float64: ~1e-6 relative)."""
    from oracle import mlp
    params = W.mlp_init(mlp.SIZES, 4)
    X, Y = _data(128, 5)
    ctx = pc.Context(0, 0)
    m = pc.Mlp(ctx.h, params)
    state = {}
    ref = [(w.astype(np.float64), b.astype(np.float64)) for w, b in params]
    for _ in range(3):
        _, g = m.grads(X, Y)
        ref = mlp.adam_step(ref, [(gw.astype(np.float64), gb.astype(np.float64)) for gw, gb in g], state,
                            lr=1e-3)
        m.train_step(X, Y, lr=1e-3)
        ref = [(w, b) for w, b in ref]
        got = m.params()
        for (w, b), (rw, rb) in zip(got, ref):
            assert _rel(w, rw) < 1e-5 and _rel(b, rb) < 1e-5
        # continue the oracle from the GPU's parameters to keep both on one trajectory
        ref = [(w.astype(np.float64), b.astype(np.float64)) for w, b in got]
    m.close()
    ctx.close()


def test_training_reduces_loss(pc):
    from oracle import mlp
    params = W.mlp_init(mlp.SIZES, 6)
    X, Y = _data(256, 7)
    ctx = pc.Context(0, 0)
    m = pc.Mlp(ctx.h, params)
    losses = [m.train_step(X, Y, lr=1e-3) for _ in range(200)]
    assert losses[-1] < 0.05 * losses[0]
    m.close()
    ctx.close()
