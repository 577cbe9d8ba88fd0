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
    m = pc.Mlp(ctx, params, beta_min=0.1)
    beta = m.forward(X)
    ref, _ = mlp.forward(params, X.astype(np.float64), beta_min=0.1)
    _close(beta, ref, 259, "beta")
    m.close()
    ctx.close()


@pytest.mark.parametrize("B,gw", [(64, 0.0), (300, 0.0), (64, 0.05), (300, 0.3)])
def test_gradients_match_oracle(pc, B, gw):
    """Gradients of the squared ladder error, and with the relative-gap
    term (its gap_weight gw)."""
    from oracle import mlp
    params = W.mlp_init(mlp.SIZES, 2)
    params = [(w, b + 0.01) for w, b in params]
    X, Y = _data(B, 3)
    ctx = pc.Context(0, 0)
    m = pc.Mlp(ctx, params)
    m.set_gap_weight(gw)
    loss, grads = m.grads(X, Y)
    loss_ref, grads_ref = mlp.loss_and_grads(params, X.astype(np.float64), Y.astype(np.float64), gap_weight=gw)
    assert abs(loss - loss_ref) <= RTOL * loss_ref
    K = max(259, B)
    for l, ((gW, gb), (rW, rb)) in enumerate(zip(grads, grads_ref)):
        _close(gW, rW, K, f"dW{l}")
        _close(gb, rb, K, f"db{l}")
    m.close()
    ctx.close()


def _oracle_trajectory(params, X, Y, steps, lr, perturb=None):
    """Oracle Adam trajectory (float64); perturb(step, l, k, g) may move
    each gradient before its update.  Returns the parameters after each
    step."""
    from oracle import mlp
    state = {}
    p = [(w.astype(np.float64), b.astype(np.float64)) for w, b in params]
    out = []
    for step in range(steps):
        _, g = mlp.loss_and_grads(p, X, Y)
        if perturb is not None:
            g = [tuple(perturb(step, l, k, gk) for k, gk in enumerate(gl)) for l, gl in enumerate(g)]
        p = mlp.adam_step(p, g, state, lr=lr)
        out.append(p)
    return out


def test_training_trajectory_matches_oracle(pc):
    """Five Adam steps on the GPU and five in the oracle (its own float64
    gradients), from the same start; parameters compared element by element
    after every step.

    Adam divides each gradient by its own running magnitude, so an element
    whose gradient is no larger than its fp32 rounding error can move by up
    to lr per step in either implementation.  The tolerance therefore adds
    to RTOL * |p| + ATOL the spread of the oracle's own trajectory when
    every gradient element is moved by its fp32 error bound
    (RTOL |g| + 4 K 2^-24 max|g|, the bound the gradient test checks),
    taken over the all-up, all-down and four random-sign perturbations."""
    from oracle import mlp
    params = W.mlp_init(mlp.SIZES, 4)
    X, Y = _data(128, 5)
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    steps, lr, K = 5, 1e-3, 259
    ref = _oracle_trajectory(params, X64, Y64, steps, lr)
    spread = [[np.zeros_like(w), np.zeros_like(b)] for w, b in ref[0]]
    spread = [[[np.zeros_like(t) for t in layer] for layer in spread] for _ in range(steps)]
    rng = np.random.default_rng(0)
    signs = [lambda g: np.ones_like(g), lambda g: -np.ones_like(g)] + \
            [lambda g: rng.choice([-1.0, 1.0], size=g.shape) for _ in range(4)]
    for sign in signs:
        def perturb(step, l, k, g, sign=sign):
            return g + sign(g) * (RTOL * np.abs(g) + 4 * K * 2.0 ** -24 * np.abs(g).max())
        alt = _oracle_trajectory(params, X64, Y64, steps, lr, perturb)
        for t in range(steps):
            for l in range(4):
                for k in range(2):
                    spread[t][l][k] = np.maximum(spread[t][l][k], np.abs(alt[t][l][k] - ref[t][l][k]))
    ctx = pc.Context(0, 0)
    m = pc.Mlp(ctx, params)
    for step in range(steps):
        loss = m.train_step(X, Y, lr=lr)
        loss_ref, _ = mlp.loss_and_grads(ref[step - 1] if step else
                                         [(w.astype(np.float64), b.astype(np.float64)) for w, b in params],
                                         X64, Y64)
        assert abs(loss - loss_ref) <= 1e-3 * loss_ref, step
        for l, ((w, b), (rw, rb)) in enumerate(zip(m.params(), ref[step])):
            for k, (a, r) in enumerate(((w, rw), (b, rb))):
                a = np.asarray(a, np.float64)
                bound = RTOL * np.abs(r) + 4 * K * 2.0 ** -24 * np.abs(r).max() + 2 * spread[step][l][k]
                bad = np.abs(a - r) > bound
                assert not bad.any(), (step, l, k, int(bad.sum()), float((np.abs(a - r) / bound).max()))
    m.close()
    ctx.close()


def test_training_reduces_loss(pc):
    from oracle import mlp
    params = W.mlp_init(mlp.SIZES, 6)
    X, Y = _data(256, 7)
    ctx = pc.Context(0, 0)
    m = pc.Mlp(ctx, params)
    losses = [m.train_step(X, Y, lr=1e-3) for _ in range(200)]
    assert losses[-1] < 0.05 * losses[0]
    m.close()
    ctx.close()
