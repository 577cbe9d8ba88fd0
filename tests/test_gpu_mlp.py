"""Ladder-predictor MLP kernels (fp32) against the float64 oracle, element
by element.

Tolerance.  Every value is built from dot products of at most K = 259
terms (or the batch, for weight gradients), four layers deep.  The fp32
rounding error of such a sum is at most about K * 2^-24 times the sum of
its terms' magnitudes, so an entry of a tensor b is compared as

    |gpu - oracle| <= RTOL * |oracle| + ATOL,   ATOL = 4 * K * 2^-24 * max|b|

with RTOL = 1e-4 and K the longest reduction behind the tensor (the factor
4 for the four layers).  A norm would hide one wrong row or column; this
bound does not.
"""
import numpy as np
import pytest

from paper_2503_10302_gb300 import workloads as W

pytestmark = pytest.mark.gpu
RTOL = 1e-4


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


def _close(a, b, K, what=""):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    atol = 4 * K * 2.0 ** -24 * np.abs(b).max()
    bound = RTOL * np.abs(b) + atol
    bad = np.abs(a - b) > bound
    assert not bad.any(), (what, int(bad.sum()), float((np.abs(a - b) / bound).max()),
                           np.argwhere(bad)[:4].tolist())


@pytest.mark.parametrize("B", [1, 37, 256])
def test_forward_matches_oracle(pc, B):
    from oracle import mlp
    params = W.mlp_init(mlp.SIZES, 1)
    X, _ = _data(B, B)
    ctx = pc.Context(0, 0)
    m = pc.Mlp(ctx.h, params, beta_min=0.1)
    beta = m.forward(X)
    ref, _ = mlp.forward(params, X.astype(np.float64), beta_min=0.1)
    _close(beta, ref, 259, "beta")
    m.close()
    ctx.close()


@pytest.mark.parametrize("B", [64, 300])
def test_gradients_match_oracle(pc, B):
    from oracle import mlp
    params = W.mlp_init(mlp.SIZES, 2)
    params = [(w, b + 0.01) for w, b in params]
    X, Y = _data(B, 3)
    ctx = pc.Context(0, 0)
    m = pc.Mlp(ctx.h, params)
    loss, grads = m.grads(X, Y)
    loss_ref, grads_ref = mlp.loss_and_grads(params, X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss - loss_ref) <= RTOL * loss_ref
    K = max(259, B)
    for l, ((gW, gb), (rW, rb)) in enumerate(zip(grads, grads_ref)):
        _close(gW, rW, K, f"dW{l}")
        _close(gb, rb, K, f"db{l}")
    m.close()
    ctx.close()


def test_training_trajectory_matches_oracle(pc):
    """Five Adam steps on the GPU and five in the oracle (its own float64
    gradients), from the same start; parameters compared after every step."""
    from oracle import mlp
    params = W.mlp_init(mlp.SIZES, 4)
    X, Y = _data(128, 5)
    ctx = pc.Context(0, 0)
    m = pc.Mlp(ctx.h, params)
    state = {}
    ref = [(w.astype(np.float64), b.astype(np.float64)) for w, b in params]
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    for step in range(5):
        loss = m.train_step(X, Y, lr=1e-3)
        loss_ref, g = mlp.loss_and_grads(ref, X64, Y64)
        assert abs(loss - loss_ref) <= RTOL * loss_ref, step
        ref = mlp.adam_step(ref, g, state, lr=1e-3)
        for l, ((w, b), (rw, rb)) in enumerate(zip(m.params(), ref)):
            _close(w, rw, 259, f"W{l} step {step}")
            _close(b, rb, 259, f"b{l} step {step}")
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
