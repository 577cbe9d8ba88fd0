"""Pins for the oracle of the learned ladder predictor: gradients against
central finite differences and against torch.autograd (float64), Adam against
torch.optim.Adam, and the feature and resampling helpers against brute force."""
import itertools

import numpy as np
import pytest

from oracle import mlp
from paper_2503_10302_gb300 import workloads as W


def _params(sizes, seed):
    return [(W.astype(np.float64), b.astype(np.float64) + 0.01) for W, b in W_init(sizes, seed)]


def W_init(sizes, seed):
    return W.mlp_init(sizes, seed)


@pytest.mark.parametrize("gw", [0.0, 0.3])
def test_gradients_match_finite_differences(gw):
    sizes = (7, 6, 5, 4, 3)
    params = _params(sizes, 1)
    rng = np.random.default_rng(0)
    X = rng.normal(size=(4, 7))
    Y = np.cumsum(np.abs(rng.normal(size=(4, 3))), axis=1)
    loss, grads = mlp.loss_and_grads(params, X, Y, beta_min=0.1, gap_weight=gw)
    eps = 1e-6
    for li in range(4):
        for k in range(2):
            p = params[li][k]
            g = grads[li][k]
            for idx in itertools.islice(np.ndindex(p.shape), 0, None, 3):
                old = p[idx]
                p[idx] = old + eps
                lp, _ = mlp.loss_and_grads(params, X, Y, 0.1, gw)
                p[idx] = old - eps
                lm, _ = mlp.loss_and_grads(params, X, Y, 0.1, gw)
                p[idx] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - g[idx]) < 1e-6 * max(1.0, abs(fd)), (li, k, idx)


@pytest.mark.parametrize("gw", [0.0, 0.05])
def test_gradients_match_autograd_full_size(gw):
    torch = pytest.importorskip("torch")
    params = _params(mlp.SIZES, 2)
    rng = np.random.default_rng(1)
    X = rng.random(size=(8, mlp.N_IN))
    Y = np.cumsum(rng.random(size=(8, 32)) * 0.1, axis=1) + 0.5
    loss, grads = mlp.loss_and_grads(params, X, Y, gap_weight=gw)
    tp = [(torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True)) for W, b in params]
    h = torch.tensor(X)
    for i, (Wt, bt) in enumerate(tp):
        h = h @ Wt.T + bt
        if i < 3:
            h = torch.relu(h)
    beta = torch.cumsum(torch.nn.functional.softplus(h), dim=1)
    Yt = torch.tensor(Y)
    tl = ((beta - Yt) ** 2).mean()
    if gw:   # the gap term written with torch's own ops: differences of the ladders
        gaps, d = torch.diff(beta, dim=1), torch.diff(Yt, dim=1)
        tl = tl + gw * (((gaps - d) / d) ** 2).mean()
    tl.backward()
    assert abs(tl.item() - loss) < 1e-12 * max(1, loss)
    for (Wt, bt), (gW, gb) in zip(tp, grads):
        assert np.allclose(Wt.grad.numpy(), gW, rtol=1e-10, atol=1e-14)
        assert np.allclose(bt.grad.numpy(), gb, rtol=1e-10, atol=1e-14)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    params = _params((5, 4, 4, 4, 3), 3)
    rng = np.random.default_rng(2)
    tp = [torch.tensor(a.copy(), requires_grad=True) for pr in params for a in pr]
    opt = torch.optim.Adam(tp, lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    state = {}
    cur = params
    for step in range(5):
        grads = [(rng.normal(size=W.shape), rng.normal(size=b.shape)) for W, b in cur]
        cur = mlp.adam_step(cur, grads, state, lr=1e-2)
        for t, g in zip(tp, [a for pr in grads for a in pr]):
            t.grad = torch.tensor(g)
        opt.step()
    for t, a in zip(tp, [a for pr in cur for a in pr]):
        assert np.allclose(t.detach().numpy(), a, rtol=1e-12, atol=1e-14)


def test_monotone_head():
    params = _params(mlp.SIZES, 4)
    X = np.random.default_rng(3).normal(size=(5, mlp.N_IN))
    beta, _ = mlp.forward(params, X, beta_min=0.2)
    assert (np.diff(beta, axis=1) > 0).all() and (beta[:, 0] > 0.2).all()


def test_instance_features_brute_force():
    dims = (4, 6, 4)
    Lx, Ly, Lz = dims
    J = W.ea_couplings(dims, 5, 0)
    idx = lambda x, y, z: (x % Lx) + Lx * ((y % Ly) + Ly * (z % Lz))
    unit = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    fr = 0
    for z, y, x in itertools.product(range(Lz), range(Ly), range(Lx)):
        for a, b in ((0, 1), (0, 2), (1, 2)):
            ea, eb = unit[a], unit[b]
            r = (x, y, z)
            ra = tuple(r[i] + ea[i] for i in range(3))
            rb = tuple(r[i] + eb[i] for i in range(3))
            prod = J[idx(*r), a] * J[idx(*ra), b] * J[idx(*rb), a] * J[idx(*r), b]
            fr += prod < 0
    f = mlp.instance_features(dims, J)
    assert f[2] == fr / (3 * 96)
    assert f[1] == (J > 0).mean()
    ferro = np.ones((64, 3), np.int8)
    assert list(mlp.instance_features((4, 4, 4), ferro)) == [0.25, 1.0, 0.0]


def test_resample_ladder():
    b = np.linspace(0.5, 3.0, 20)
    r = mlp.resample_ladder(b, 32)
    assert r[0] == 0.5 and r[-1] == 3.0 and np.allclose(np.diff(r), 2.5 / 31)
    b32 = np.sort(np.random.default_rng(0).random(32))
    assert np.allclose(mlp.resample_ladder(b32, 32), b32, rtol=0, atol=1e-15)
