"""Oracle for the learned beta-ladder predictor (test infrastructure only).

A plain float64 numpy restatement of the small network that maps instance
features and pilot-run energy histograms to a 32-point beta ladder, its
gradient and one Adam step.  The paper has no learned component; its
grounding is the observation (Sec. "Temperature profile and swap acceptance
rate in APT", Fig. S12) that adaptive ladders are nearly the same across
instances of one size, which makes them learnable from cheap features.

Network: x (259) -> 256 -> 256 -> 256 (ReLU each) -> o (32).
Monotone head: beta_k = beta_min + sum_{m<=k} softplus(o_m).
Loss: mean over batch and the 32 outputs of (beta_k - y_k)^2, plus
gap_weight times the mean over batch and the 31 gaps k >= 1 of
((g_k - d_k) / d_k)^2, with g_k = softplus(o_k) = beta_k - beta_{k-1} and
d_k = y_k - y_{k-1} the target's gap (the swap acceptance of a pair depends
on its gap; the squared error of the cumulative ladder alone barely
constrains gap errors that cancel between neighbours).

Features of an instance (also restated here): [L/16, fraction of J > 0,
fraction of frustrated plaquettes, 4 x 64 normalised pilot histograms].
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np

N_OUT = 32
N_HIST = 4 * 64
N_IN = 3 + N_HIST
SIZES = (N_IN, 256, 256, 256, N_OUT)


def softplus(x):
    return np.maximum(x, 0.0) + np.log1p(np.exp(-np.abs(x)))


def sigmoid(x):
    return 0.5 * (1.0 + np.tanh(0.5 * x))


def forward(params: Sequence[Tuple[np.ndarray, np.ndarray]], X: np.ndarray, beta_min: float = 0.0):
    """params: [(W [out,in], b [out])] * 4; X: [B, 259].  Returns (beta, cache)."""
    acts = [np.asarray(X, np.float64)]
    pre = []
    h = acts[0]
    for li, (W, b) in enumerate(params):
        z = h @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        pre.append(z)
        h = np.maximum(z, 0.0) if li < len(params) - 1 else z
        acts.append(h)
    o = acts[-1]
    beta = beta_min + np.cumsum(softplus(o), axis=1)
    return beta, (acts, pre)


def loss_and_grads(params, X, Y, beta_min: float = 0.0, gap_weight: float = 0.0):
    """Loss (squared ladder error plus gap_weight times the squared relative
    gap error) and gradients w.r.t. every W and b."""
    beta, (acts, pre) = forward(params, X, beta_min)
    Y = np.asarray(Y, np.float64)
    diff = beta - Y
    loss = float((diff ** 2).mean())
    g_beta = 2.0 * diff / diff.size
    # beta_k = sum_{m<=k} softplus(o_m)  =>  dL/do_m = sigmoid(o_m) sum_{k>=m} dL/dbeta_k
    g = sigmoid(pre[-1]) * np.cumsum(g_beta[:, ::-1], axis=1)[:, ::-1]
    if gap_weight:
        o = pre[-1][:, 1:]
        d = np.diff(Y, axis=1)
        r = (softplus(o) - d) / d
        loss += gap_weight * float((r ** 2).mean())
        # d softplus(o) / do = sigmoid(o)
        g[:, 1:] += gap_weight * 2.0 * r / d * sigmoid(o) / r.size
    grads: List[Tuple[np.ndarray, np.ndarray]] = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W = np.asarray(params[li][0], np.float64)
        grads[li] = (g.T @ acts[li], g.sum(0))
        if li > 0:
            g = (g @ W) * (pre[li - 1] > 0)
    return loss, grads


def adam_step(params, grads, state: Dict, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) in place on float64 copies of params."""
    t = state.get("t", 0) + 1
    state["t"] = t
    if "m" not in state:
        state["m"] = [[np.zeros_like(W, np.float64), np.zeros_like(b, np.float64)] for W, b in params]
        state["v"] = [[np.zeros_like(W, np.float64), np.zeros_like(b, np.float64)] for W, b in params]
    new = []
    for li, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        out = []
        for k, (p, g) in enumerate(((W, gW), (b, gb))):
            m = state["m"][li][k] = b1 * state["m"][li][k] + (1 - b1) * g
            v = state["v"][li][k] = b2 * state["v"][li][k] + (1 - b2) * g * g
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            out.append(np.asarray(p, np.float64) - lr * mh / (np.sqrt(vh) + eps))
        new.append(tuple(out))
    return new


def instance_features(dims, J) -> np.ndarray:
    """[L/16, fraction of J>0, frustrated-plaquette fraction] of a periodic lattice."""
    Lx, Ly, Lz = (int(v) for v in dims)
    N = Lx * Ly * Lz
    Jg = np.asarray(J, np.int64).reshape(Lz, Ly, Lx, 3)
    frust = 0
    # plaquette in the (a, b) plane at site r: J_a(r) J_b(r+a) J_a(r+b) J_b(r)
    axis_of = {0: 2, 1: 1, 2: 0}       # array axis of lattice direction x, y, z
    for a in range(3):
        for b in range(a + 1, 3):
            ja, jb = Jg[..., a], Jg[..., b]
            prod = ja * np.roll(jb, -1, axis=axis_of[a]) * np.roll(ja, -1, axis=axis_of[b]) * jb
            frust += int((prod < 0).sum())
    return np.array([np.cbrt(float(N)) / 16.0, float((np.asarray(J) > 0).mean()), frust / (3.0 * N)], np.float64)


def histogram_features(counts: np.ndarray) -> np.ndarray:
    """[4, 64] integer counts -> per-temperature normalised, flattened."""
    c = np.asarray(counts, np.float64)
    return (c / np.maximum(c.sum(axis=1, keepdims=True), 1.0)).reshape(-1)


def resample_ladder(beta: np.ndarray, n: int = N_OUT) -> np.ndarray:
    """Piecewise-linear resampling of a ladder to n points in normalised
    index, keeping both endpoints."""
    beta = np.asarray(beta, np.float64)
    if len(beta) == 1:
        return np.full(n, beta[0])
    pos = np.arange(n, dtype=np.float64) * (len(beta) - 1) / (n - 1)
    lo = np.minimum(np.floor(pos).astype(np.int64), len(beta) - 2)
    w = pos - lo
    return beta[lo] * (1.0 - w) + beta[lo + 1] * w
