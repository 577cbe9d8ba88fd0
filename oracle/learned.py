"""Oracle of the learned beta ladder and its judge (test infrastructure only).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg
may import this module.  It composes the oracle's own pieces, in the order
the library's learned-ladder call takes them, from plain restatements:

1. pilot histograms of a short run at four fixed temperatures
   (``oracle.pilot_hist``);
2. the network's input: [cbrt(N)/16, fraction of J > 0, fraction of
   frustrated plaquettes] and the histograms, each temperature's counts
   divided by their total (``mlp.instance_features``,
   ``mlp.histogram_features``);
3. the network in float64 (``mlp.forward``), whose cumulative-softplus head
   makes a ladder of 32 betas;
4. a strictly increasing ladder: beta_0 = max(b_0, 0), then
   beta_k = max(b_k, beta_{k-1} + 1e-6);
5. the judge: the first attempts of APT with ICM (Algorithm S2) on that
   ladder, and the swap acceptance of every temperature pair pooled over the
   labels; a ladder passes iff every attempted pair has
   accepts >= floor * attempts.  The adaptive procedure (Methods "APT
   details") aims at a flat acceptance erfc(alpha/2), about 0.38 at the
   paper's alpha = 1.25 (Supplementary "Temperature profile and swap
   acceptance rate in APT"), which is what the floor is measured against;
6. the fallback of a rejected ladder: the adaptive procedure of
   Algorithm S2's preprocessing, resampled to 32 points.

The paper has no learned component; its ground is that ladders of one size
are nearly the same across instances (Fig. S12).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

from . import adaptive_ladder, pilot_hist, Apt
from . import mlp

LADDER_GAP = 1e-6


def features(dims_list, J_list, pilot_betas, entry0=0, seed=0, chains=8, sweeps=256, burn=128) -> np.ndarray:
    """Network inputs [n][259] (float64) of the instances: steps 1 and 2."""
    X = np.zeros((len(J_list), mlp.N_IN), np.float64)
    for i, (d, J) in enumerate(zip(dims_list, J_list)):
        counts = pilot_hist(d, J, pilot_betas, entry=entry0 + i, seed=seed, chains_per_beta=chains,
                            sweeps=sweeps, burn=burn, n_bins=64)
        X[i, :3] = mlp.instance_features(d, J)
        X[i, 3:] = mlp.histogram_features(counts)
    return X


def monotone(beta: np.ndarray, gap: float = LADDER_GAP) -> np.ndarray:
    """Step 4: beta_0 = max(b_0, 0), beta_k = max(b_k, beta_{k-1} + gap)."""
    b = np.array(beta, np.float64, copy=True)
    for row in np.atleast_2d(b):
        row[0] = max(row[0], 0.0)
        for k in range(1, row.size):
            if not row[k] >= row[k - 1] + gap:
                row[k] = row[k - 1] + gap
    return b


def predict(params, X, beta_min=0.0) -> np.ndarray:
    """Step 3 and 4: the network's ladders, made strictly increasing."""
    beta, _ = mlp.forward(params, X, beta_min)
    return monotone(beta)


def judge(dims_list, J_list, betas, entry0=0, seed=0, n_labels=2, attempts=200, floor=0.19,
          threads=0) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """Step 5.  Returns (attempts [n][T-1], accepts [n][T-1], pooled
    acceptance [n][T-1] (-1 where never attempted), pass [n])."""
    betas = [np.asarray(b, np.float64) for b in betas]
    apt = Apt(np.asarray(dims_list, np.int32).reshape(-1, 3), J_list, betas, n_labels, seed=seed, entry0=entry0)
    apt.run(attempts, 1, n_labels >= 2, threads)
    n = len(J_list)
    T = len(betas[0])
    att = np.zeros((n, T - 1), np.int64)
    acc = np.zeros((n, T - 1), np.int64)
    rate = np.full((n, T - 1), -1.0)
    ok = np.ones(n, bool)
    for i in range(n):
        a, c, _ = apt.stats(i)
        att[i], acc[i] = a.sum(axis=1), c.sum(axis=1)
        for r in range(T - 1):
            if att[i, r] <= 0:
                continue
            rate[i, r] = float(acc[i, r]) / float(att[i, r])
            if float(acc[i, r]) < floor * float(att[i, r]):
                ok[i] = False
    return att, acc, rate, ok


def fallback(dims, J, entry, seed=0, beta0=0.5, alpha=1.25, n_chains=32, sweeps=2000, tail=500, tol=1.0,
             max_len=64) -> np.ndarray:
    """Step 6: the adaptive ladder resampled to 32 points."""
    b, _, _ = adaptive_ladder(dims, J, entry=entry, seed=seed, beta0=beta0, alpha=alpha, n_chains=n_chains,
                              sweeps=sweeps, tail=tail, tol=tol, max_len=max_len)
    return mlp.resample_ladder(b, mlp.N_OUT)


def learned_ladder(params, dims_list, J_list, pilot_betas, entry0=0, seed=0, beta_min=0.0, pilot_chains=8,
                   pilot_sweeps=256, pilot_burn=128, probe_attempts=200, probe_labels=2, acc_floor=0.19,
                   ladder_kw=None, threads=0):
    """Steps 1-6: (ladders [n][32], pooled acceptances [n][31], fallback [n])."""
    ladder_kw = dict(ladder_kw or {})
    X = features(dims_list, J_list, pilot_betas, entry0, seed, pilot_chains, pilot_sweeps, pilot_burn)
    beta = predict(params, X, beta_min)
    n = len(J_list)
    fb = np.zeros(n, bool)
    rate = np.full((n, mlp.N_OUT - 1), -1.0)
    if probe_attempts <= 0:
        return beta, rate, fb
    _, _, rate, ok = judge(dims_list, J_list, list(beta), entry0, seed, probe_labels, probe_attempts, acc_floor,
                           threads)
    for i in np.flatnonzero(~ok):
        beta[i] = fallback(dims_list[i], J_list[i], entry0 + int(i), seed, **ladder_kw)
        fb[i] = True
    return beta, rate, fb
