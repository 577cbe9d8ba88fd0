"""The learned beta ladder: training set, GPU training, weights file, and the
time-to-target comparison of ladders.

Everything numeric runs in the C-ABI library: adaptive ladders
(pc_adaptive_ladder, Algorithm S2's preprocessing), the network's inputs
(pc_learned_features: pilot histograms and instance features on the
device), training (pc_mlp_train_step_dev: hand-written fp32 forward,
backward and Adam kernels), inference with its judge and fallback
(pc_learned_ladder) and the APT+ICM runs to a target energy.  This module
only orders the calls and times them.

Run ``python -m paper_2503_10302_gb300.ladder --help``.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time
from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import pcomp
from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(_HERE, "weights", "ladder_mlp.bin")
MEANS = os.path.join(_HERE, "weights", "ladder_means.json")

# Pilot design of the network's inputs: 4 temperatures geometric over
# [0.2, 3.0], 8 chains each, 256 sweeps of which the last 128 are counted.
PILOT_BETAS = W.geometric_ladder(4, 0.2, 3.0)
PILOT_KW = dict(pilot_chains=8, pilot_sweeps=256, pilot_burn=128)
# Adaptive procedure (Methods "APT details": beta_0 = 0.5, alpha = 1.25;
# the paper uses 100 chains, 10^4 sweeps and a tail of 10^3; these reduced
# settings are used for the training labels and for the adaptive arm alike).
LADDER_KW = dict(beta0=0.5, alpha=1.25, n_chains=32, sweeps=2000, tail=500, tol=1.0, max_len=64)
# Judge: 500 probe attempts with 2 labels.  The adaptive procedure spaces
# temperatures so that dbeta sigma_E = alpha, whose acceptance for Gaussian
# energies is erfc(alpha / 2) = 0.377 at alpha = 1.25; a pair fails when its
# acceptance is below erfc(1.25 alpha) = 0.027, that of a gap 2.5 times the
# adaptive one.  (The adaptive ladders themselves, resampled to 32 points,
# accept 0.07-0.13 at their coldest pair at L = 16, so a floor of half the
# design acceptance would reject them too.)
JUDGE_KW = dict(probe_attempts=500, probe_labels=2, acc_floor=math.erfc(1.25 * 1.25))
SIZES = (6, 8, 10, 12, 14, 16)
# Weight of the relative-gap term of the training loss (pc_mlp_set_gap_weight):
# without it the network's hottest gaps ripple (pairs accepting alternately
# about 0.13 and 0.8 at L = 16) because the squared error of the cumulative
# ladder barely constrains gap errors that cancel between neighbours.
GAP_WEIGHT = 0.05


def _ctx(seed: int) -> pcomp.Context:
    return pcomp.Context(0, seed)


def training_set(n: int, sizes: Sequence[int] = SIZES, seed: int = W.SEED_TRAIN, chunk: int = 4096,
                 ladder_kw=None) -> Dict:
    """n generated periodic +-J instances (even L drawn uniformly from
    `sizes`), their adaptive ladders resampled to 32 points (the targets)
    and the network's inputs.  Instance i draws entry i for the ladder and
    for the pilot run."""
    ladder_kw = dict(LADDER_KW, **(ladder_kw or {}))
    rng = np.random.Generator(np.random.Philox(key=[seed, 0xEEEE]))
    Ls = rng.choice(np.asarray(sizes), size=n)
    X = np.zeros((n, 259), np.float32)
    Y = np.zeros((n, 32), np.float32)
    lens = np.zeros(n, np.int32)
    t_lad = t_feat = 0.0
    ctx = _ctx(seed)
    for s0 in range(0, n, chunk):
        idx = range(s0, min(n, s0 + chunk))
        dims = np.array([[Ls[i]] * 3 for i in idx], np.int32)
        J = [W.ea_couplings((int(Ls[i]),) * 3, seed, i) for i in idx]
        t0 = time.perf_counter()
        lad = pcomp.pc_adaptive_ladder(ctx.h, dims, J, entry0=s0, **ladder_kw)
        t_lad += time.perf_counter() - t0
        t0 = time.perf_counter()
        X[s0:s0 + len(J)] = pcomp.pc_learned_features(ctx.h, dims, J, PILOT_BETAS, entry0=s0, **PILOT_KW)
        t_feat += time.perf_counter() - t0
        for k, (b, _, _) in enumerate(lad):
            Y[s0 + k] = pcomp.pc_resample_ladder(b, 32)
            lens[s0 + k] = len(b)
    ctx.close()
    return {"X": X, "Y": Y, "L": Ls, "len": lens, "ladder_seconds": t_lad, "feature_seconds": t_feat,
            "ladder_kw": ladder_kw}


def train(X: np.ndarray, Y: np.ndarray, epochs: int = 60, batch: int = 256, lr: float = 1e-3, seed: int = 21,
          gap_weight: float = GAP_WEIGHT):
    """Adam on the GPU kernels over shuffled minibatches, the learning rate
    decaying tenfold over the epochs.  Returns (network, context, loss of
    the last minibatch of each epoch, seconds)."""
    import torch
    params = W.mlp_init(pcomp.MLP_SIZES, seed)
    ctx = _ctx(seed)
    stream = torch.cuda.Stream()
    pcomp.pc_set_stream(ctx.h, stream.cuda_stream)
    m = pcomp.Mlp(ctx, params)
    m.set_gap_weight(gap_weight)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    loss = torch.zeros(1, device="cuda")
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    hist = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).cuda()
        Xp, Yp = Xd[perm].contiguous(), Yd[perm].contiguous()
        torch.cuda.synchronize()
        lr_ep = lr * (0.1 ** (ep / max(1, epochs - 1)))
        for b0 in range(0, n - batch + 1, batch):
            m.train_step_dev(batch, Xp[b0:].data_ptr(), Yp[b0:].data_ptr(), lr_ep, loss.data_ptr())
        torch.cuda.synchronize()
        hist.append(float(loss.item()))
    return m, ctx, hist, time.perf_counter() - t0


def mean_ladders(Y: np.ndarray, Ls: np.ndarray) -> Dict[str, List[float]]:
    """Per-size mean of the training ladders: the input-free baseline that
    knows the size only."""
    return {str(int(L)): [float(v) for v in Y[Ls == L].mean(axis=0)] for L in sorted(set(int(x) for x in Ls))}


def load_means(path: str = MEANS) -> Dict[int, np.ndarray]:
    with open(path) as f:
        d = json.load(f)
    return {int(k): np.asarray(v, np.float64) for k, v in d["mean_ladders"].items()}


def best_energies(dims, J_list, betas, runs: int = 10, sweeps: int = 20000, spp: int = 10,
                  seed: int = 100) -> np.ndarray:
    """E_best of each instance: the minimum over `runs` independent APT+ICM
    runs with sweep-to-swap ratio `spp` (Methods "Instances": the best over
    long runs at ratio 10).  Run r of instance i is problem r*n + i of one
    batch, drawing with its own entry id."""
    n = len(J_list)
    ctx = _ctx(seed)
    d = np.tile(np.asarray(dims, np.int32).reshape(n, 3), (runs, 1))
    pcomp.pc_apt_load(ctx.h, d, list(J_list) * runs, list(betas) * runs, 2, 0)
    pcomp.pc_apt_run(ctx.h, max(1, sweeps // spp), spp, True)
    E, _ = pcomp.pc_apt_get_best_all(ctx.h, n * runs)
    ctx.close()
    return E.reshape(runs, n).min(axis=0)


def run_to_target(dims, J_list, betas, targets, max_sweeps: int = 100000, chunk: int = 128,
                  seed: int = 7, entry0: int = 0) -> Tuple[np.ndarray, np.ndarray, float]:
    """APT+ICM, one sweep per attempt, 2 labels, until every instance has
    reached its target or max_sweeps.  Returns (hit sweep per instance, -1 if
    missed; measured seconds from the start of the run to the end of the
    chunk in which each instance's hit was seen, inf if missed; seconds per
    sweep of the batch)."""
    n = len(J_list)
    ctx = _ctx(seed)
    pcomp.pc_apt_load(ctx.h, dims, J_list, betas, 2, entry0)
    for i, t in enumerate(targets):
        pcomp.pc_apt_set_target(ctx.h, i, int(t))
    pcomp.pc_synchronize(ctx.h)
    t0 = time.perf_counter()
    done = 0
    hit = np.full(n, -1, np.int64)
    t_hit = np.full(n, np.inf)
    while done < max_sweeps:
        pcomp.pc_apt_run(ctx.h, chunk, 1, True)
        done += chunk
        _, hit = pcomp.pc_apt_get_best_all(ctx.h, n)     # synchronises the stream
        now = time.perf_counter() - t0
        t_hit[(hit >= 0) & np.isinf(t_hit)] = now
        if (hit >= 0).all():
            break
    total = time.perf_counter() - t0
    ctx.close()
    return hit, t_hit, total / done


def eval_set(n: int, L: int, seed: int = W.SEED_EVAL):
    dims = np.tile(np.array([L, L, L], np.int32), (n, 1))
    J = [W.ea_couplings((L, L, L), seed, i) for i in range(n)]
    return dims, J


def construct(arm: str, dims, J, net=None, means=None, entry0: int = 1 << 20, seed: int = 11,
              judge_kw=None) -> Tuple[List[np.ndarray], float, Dict, np.ndarray]:
    """Ladders of one arm, the wall time to construct them (one batch) and
    the time at which each instance's ladder was ready: the learned arm
    reports it per instance (after the judge, or after a fallback); the
    adaptive arm's instances all wait for the batch."""
    info: Dict = {}
    n = len(J)
    if arm == "geometric":
        return [W.geometric_ladder(32, 0.2, 3.0)] * n, 0.0, info, np.zeros(n)
    if arm == "mean":
        L = int(dims[0][0])
        return [means[L] + 0.0] * n, 0.0, info, np.zeros(n)
    owner = None if arm == "learned" else _ctx(seed)
    h = net.ctx if owner is None else owner.h
    pcomp.pc_synchronize(h)
    t0 = time.perf_counter()
    ready = None
    if arm == "adaptive":
        lad = pcomp.pc_adaptive_ladder(h, dims, J, entry0=entry0, **LADDER_KW)
        betas = [pcomp.pc_resample_ladder(b, 32) for b, _, _ in lad]
        info["ladder_lengths"] = [len(b) for b, _, _ in lad]
    elif arm == "learned":
        beta, acc, fb, ready = pcomp.pc_learned_ladder(h, net, dims, J, PILOT_BETAS, entry0=entry0, **PILOT_KW,
                                                       **dict(JUDGE_KW, **(judge_kw or {})), **LADDER_KW,
                                                       with_ready=True)
        betas = list(beta)
        info["fallback"] = int(fb.sum())
        info["min_pair_acceptance"] = float(np.where(acc >= 0, acc, 1.0).min())
        info["median_min_pair_acceptance"] = float(np.median(np.where(acc >= 0, acc, 1.0).min(axis=1)))
    else:
        raise ValueError(arm)
    dt = time.perf_counter() - t0
    if owner is not None:
        owner.close()
    return betas, dt, info, (np.full(n, dt) if ready is None else ready)


def compare(net, means, n_eval: int = 128, L: int = 16, rho: float = 1e-3, best_runs: int = 10,
            best_sweeps: int = 20000, max_sweeps: int = 100000,
            arms: Sequence[str] = ("learned", "adaptive", "geometric", "mean")) -> Dict:
    """Time to rho_E <= rho (Eq. rho_E_f) on n_eval held-out L^3 instances,
    one APT+ICM batch per arm.  An instance's time is the time its ladder
    was ready plus the measured run time up to the chunk in which it
    reached the target.  E_best is the best over best_runs runs on the
    adaptive ladders (sweep-to-swap ratio 10)."""
    dims, J = eval_set(n_eval, L)
    N = L ** 3
    ladders = {}
    for arm in arms:
        ladders[arm] = construct(arm, dims, J, net, means)
    t0 = time.perf_counter()
    e_best = best_energies(dims, J, ladders["adaptive"][0] if "adaptive" in ladders else ladders[arms[0]][0],
                           best_runs, best_sweeps)
    t_best = time.perf_counter() - t0
    targets = np.floor(e_best + rho * N).astype(np.int64)
    out = {"n_eval": n_eval, "L": L, "rho_target": rho, "best_runs": best_runs, "best_sweeps": best_sweeps,
           "e_best_seconds": t_best, "max_sweeps": max_sweeps, "adaptive_settings": LADDER_KW,
           "judge": JUDGE_KW, "pilot": PILOT_KW}
    for arm in arms:
        betas, t_lad, info, ready = ladders[arm]
        hit, t_hit, t_sweep = run_to_target(dims, J, betas, targets, max_sweeps)
        ok = hit >= 0
        tt = ready + t_hit
        out[arm] = dict(info, ladder_seconds=t_lad, apt_seconds_per_sweep=t_sweep, hit_fraction=float(ok.mean()),
                        median_hit_sweep=float(np.median(np.where(ok, hit, max_sweeps))),
                        median_time_to_target_s=float(np.median(tt)),
                        time_to_90pct_s=float(np.quantile(tt, 0.9)),
                        hit_sweeps=[int(h) for h in hit])
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("what", choices=["train", "compare"])
    ap.add_argument("--n-train", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--n-eval", type=int, default=128)
    ap.add_argument("--L", type=int, default=16)
    ap.add_argument("--best-runs", type=int, default=10)
    ap.add_argument("--best-sweeps", type=int, default=20000)
    ap.add_argument("--max-sweeps", type=int, default=100000)
    ap.add_argument("--dump", help="train: also save the training set (X, Y, L) to this .npz")
    ap.add_argument("--json", help="compare: also write the full results (per-instance hit sweeps) here")
    args = ap.parse_args()
    if args.what == "train":
        ts = training_set(args.n_train)
        if args.dump:
            np.savez_compressed(args.dump, X=ts["X"], Y=ts["Y"], L=ts["L"], len=ts["len"])
        m, ctx, hist, t_train = train(ts["X"], ts["Y"], epochs=args.epochs)
        os.makedirs(os.path.dirname(args.out), exist_ok=True)
        m.save(args.out)
        meta = {"n_train": args.n_train, "sizes": list(SIZES), "epochs": args.epochs, "seed": W.SEED_TRAIN,
                "gap_weight": GAP_WEIGHT,
                "ladder_kw": ts["ladder_kw"], "pilot_betas": [float(b) for b in PILOT_BETAS], "pilot": PILOT_KW,
                "ladder_seconds": ts["ladder_seconds"], "feature_seconds": ts["feature_seconds"],
                "train_seconds": t_train, "loss_first_last": [hist[0], hist[-1]],
                "mean_ladders": mean_ladders(ts["Y"], ts["L"]),
                "mean_ladder_len": {str(L): float(ts["len"][ts["L"] == L].mean()) for L in SIZES}}
        with open(os.path.join(os.path.dirname(args.out), "ladder_means.json"), "w") as f:
            json.dump(meta, f, indent=1)
        print(json.dumps({k: v for k, v in meta.items() if k != "mean_ladders"}, indent=1))
        m.close()
        ctx.close()
    else:
        ctx = _ctx(5)
        net = pcomp.Mlp(ctx, path=args.out)
        out = compare(net, load_means(os.path.join(os.path.dirname(args.out), "ladder_means.json")),
                      args.n_eval, args.L, best_runs=args.best_runs, best_sweeps=args.best_sweeps,
                      max_sweeps=args.max_sweeps)
        if args.json:
            with open(args.json, "w") as f:
                json.dump(out, f)
        print(json.dumps({k: ({kk: vv for kk, vv in v.items() if kk != "hit_sweeps"} if isinstance(v, dict)
                              else v) for k, v in out.items()}, indent=1))
        net.close()
        ctx.close()


if __name__ == "__main__":
    main()
