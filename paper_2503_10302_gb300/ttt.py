"""Throughput and time-to-target measurements on the C ABI.

* APT+ICM spin flips per ns (with and without the cluster moves; the
  paper's flip counters exclude swap/ICM time, Methods "FPGA details").
* Time to a target residual energy rho_E = (E - E_best)/N (Eq. rho_E_f)
  with E_best the best energy over independent long runs (Methods
  "Instances": best over an APT+ICM run with sweep-to-swap ratio 10).
* The learned-ladder pipeline lives in ``ladder.py`` (training, weights,
  learned vs adaptive ladders by wall time to the target).

Run ``python -m paper_2503_10302_gb300.ttt --help``.
"""
from __future__ import annotations

import argparse
import json
import time
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import pcomp
from . import workloads as W

class DeviceTimer:
    """CUDA-event timing of work enqueued on the context's torch stream."""

    def __init__(self, ctx: pcomp.Context):
        import torch
        self.torch = torch
        self.stream = torch.cuda.Stream()
        pcomp.pc_set_stream(ctx.h, self.stream.cuda_stream)

    def time(self, fn) -> float:
        t = self.torch
        a, b = t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)
        t.cuda.synchronize()
        a.record(self.stream)
        fn()
        b.record(self.stream)
        t.cuda.synchronize()
        return a.elapsed_time(b) * 1e-3


def apt_throughput(batch: W.AptBatch, sweeps: int = 200, icm: bool = True, seed: int = 1,
                   shape: Optional[Tuple[int, int, int, int]] = None) -> Dict:
    """shape: (threads, thread chunks, split preference, split groups) as
    pc_apt_set_launch takes them; None keeps the default placement."""
    ctx = pcomp.Context(0, seed)
    timer = DeviceTimer(ctx)
    pcomp.pc_apt_load(ctx.h, batch.dims, batch.J, batch.betas, batch.n_labels, 0)
    if shape is not None:
        pcomp.pc_apt_set_launch(ctx.h, *shape)
    pcomp.pc_apt_run(ctx.h, 20, 1, icm)            # warm (also builds the graph)
    dt = timer.time(lambda: pcomp.pc_apt_run(ctx.h, sweeps, 1, icm))
    flips = batch.spins_per_sweep() * sweeps
    ctx.close()
    return {"flips_per_ns": flips / dt / 1e9, "seconds": dt, "sweeps": sweeps, "icm": icm,
            "spins_per_sweep": batch.spins_per_sweep()}


def best_energies(batch: W.AptBatch, n_runs: int, sweeps: int, spp: int = 10, seed0: int = 100) -> np.ndarray:
    """Minimum over n_runs independent APT+ICM runs of each instance's best energy."""
    best = None
    for r in range(n_runs):
        ctx = pcomp.Context(0, seed0 + r)
        pcomp.pc_apt_load(ctx.h, batch.dims, batch.J, batch.betas, batch.n_labels, 0)
        pcomp.pc_apt_run(ctx.h, max(1, sweeps // spp), spp, True)
        E, _ = pcomp.pc_apt_get_best_all(ctx.h, batch.n)
        best = E if best is None else np.minimum(best, E)
        ctx.close()
    return best


def run_to_target(batch: W.AptBatch, targets: np.ndarray, max_sweeps: int, chunk: int = 128,
                  seed: int = 7) -> Tuple[np.ndarray, np.ndarray, float, float]:
    """APT+ICM (sweep-to-swap 1) until every instance has E <= target or the
    sweep budget ends.  Returns (hit sweep per instance, -1 if missed;
    measured seconds from the start of the run to the end of the chunk in
    which each instance's hit was seen, inf if missed; seconds per sweep of
    the batch; total seconds)."""
    ctx = pcomp.Context(0, seed)
    pcomp.pc_apt_load(ctx.h, batch.dims, batch.J, batch.betas, batch.n_labels, 0)
    for i, t in enumerate(targets):
        pcomp.pc_apt_set_target(ctx.h, i, int(t))
    pcomp.pc_synchronize(ctx.h)
    t0 = time.perf_counter()
    done = 0
    hit = np.full(batch.n, -1, np.int64)
    t_hit = np.full(batch.n, np.inf)
    while done < max_sweeps:
        pcomp.pc_apt_run(ctx.h, chunk, 1, True)
        done += chunk
        _, hit = pcomp.pc_apt_get_best_all(ctx.h, batch.n)     # synchronises the stream
        t_hit[(hit >= 0) & np.isinf(t_hit)] = time.perf_counter() - t0
        if (hit >= 0).all():
            break
    total = time.perf_counter() - t0
    ctx.close()
    return hit, t_hit, total / done, total


def adaptive_ladders(dims, J_list, n_chains=32, sweeps=2000, tail=500, seed=11, entry0=0,
                     max_len=64) -> Tuple[List[np.ndarray], float]:
    ctx = pcomp.Context(0, seed)
    t0 = time.perf_counter()
    res = pcomp.pc_adaptive_ladder(ctx.h, dims, J_list, entry0=entry0, beta0=0.5, alpha=1.25,
                                   n_chains=n_chains, sweeps=sweeps, tail=tail, tol=1.0,
                                   max_len=max_len)
    dt = time.perf_counter() - t0
    ctx.close()
    return [b for b, _, _ in res], dt


def c3_time_to_target(n_inst=64, L=12, rho=1e-3, best_runs=10, best_sweeps=100000,
                      max_sweeps=100000, labels=2) -> Dict:
    """64 instances of L = 12, adaptive ladder resampled to 32 temperatures x
    `labels` ICM labels (4: the paper's setting, 128 replicas per problem)."""
    dims = np.tile(np.array([L, L, L], np.int32), (n_inst, 1))
    J = [W.ea_couplings((L, L, L), W.SEED_INSTANCES, i) for i in range(n_inst)]
    ladders, t_lad = adaptive_ladders(dims, J)
    betas = [pcomp.pc_resample_ladder(b, 32) for b in ladders]
    batch = W.AptBatch(dims, J, betas, labels)
    e_best = best_energies(W.AptBatch(dims, J, betas, 2), best_runs, best_sweeps)
    N = L ** 3
    targets = np.floor(e_best + rho * N).astype(np.int64)
    hit, t_hit, t_sweep, total = run_to_target(batch, targets, max_sweeps)
    ok = hit >= 0
    # per instance: the batch's ladder construction, then the measured run
    # time to the end of the chunk in which the instance reached its target
    t_inst = t_lad + t_hit
    return {"instances": n_inst, "L": L, "labels": labels, "rho_target": rho, "ladder_seconds": t_lad,
            "ladder_lengths": [len(b) for b in ladders], "apt_seconds_per_sweep": t_sweep,
            "hit_fraction": float(ok.mean()),
            "median_hit_sweep": float(np.median(hit[ok])) if ok.any() else None,
            "median_time_to_target_s": float(np.median(t_inst)) if ok.mean() > 0.5 else None,
            "e_best_per_spin_mean": float((e_best / N).mean())}


def evt_median_gaussian(mu: float, sd: float, r: int) -> float:
    """Median of the minimum of r independent N(mu, sd^2) draws (Eq.
    EVTmedianFinal): F_min(x) = 1 - (1 - Phi((x - mu)/sd))^r = 1/2 gives
    x = mu + sqrt(2) sd erfc^-1(2^((r - 1)/r))."""
    from scipy.special import erfcinv
    return mu + np.sqrt(2.0) * sd * float(erfcinv(2.0 ** ((r - 1) / r)))


def c2_residual_vs_R(L=8, P=64, R=256, T=0.05, sweeps=10000, best_runs=10, best_sweeps=100000,
                     Rs=(1, 4, 16, 64, 256)) -> Dict:
    """DT-SQA on one L = 8 instance: residual energy of the best slice of a
    run, and of the best of R independent runs as R grows.  E_best: best of
    APT+ICM runs on the same instance.  The Gaussian extreme-value median of
    the best of R (Eq. EVTmedianFinal) is reported beside the measurement."""
    wl = W.sqa_workload(L, P, R, T, sweeps)
    N = L ** 3
    ctx = pcomp.Context(0, 31)
    timer = DeviceTimer(ctx)
    pcomp.pc_sqa_setup(ctx.h, wl.dims, wl.J, P, T, wl.gamma)
    import torch
    E_dev = torch.empty((R, P), dtype=torch.int32, device="cuda")
    C_dev = torch.empty((R, P), dtype=torch.int32, device="cuda")
    dt = timer.time(lambda: pcomp.pc_sqa_run_dev(ctx.h, R, 0, E_dev.data_ptr()))
    E = E_dev.cpu().numpy().astype(np.int64)
    # replica-direction correlation of the final states (Fig. S17), same runs
    pcomp.pc_sqa_run_corr_dev(ctx.h, R, 0, E_dev.data_ptr(), C_dev.data_ptr())
    pcomp.pc_synchronize(ctx.h)
    C_r = C_dev.cpu().numpy().astype(np.float64).mean(axis=0) / N
    # C_r at the end of shorter anneals (the same schedule compressed to t_a
    # sweeps), as in Fig. S17's dependence on the annealing time
    C_ta = {}
    for ta in (10, 100, 1000):
        g = W.linear_gamma_schedule(ta)
        pcomp.pc_sqa_setup(ctx.h, wl.dims, wl.J, P, T, g)
        pcomp.pc_sqa_run_corr_dev(ctx.h, R, 0, E_dev.data_ptr(), C_dev.data_ptr())
        pcomp.pc_synchronize(ctx.h)
        c = C_dev.cpu().numpy().astype(np.float64).mean(axis=0) / N
        C_ta[str(ta)] = [float(x) for x in c[: P // 2 + 1]]
    ctx.close()
    ladder, _ = adaptive_ladders(np.array([[L] * 3], np.int32), [wl.J])
    batch = W.AptBatch(np.array([[L] * 3], np.int32), [wl.J], [pcomp.pc_resample_ladder(ladder[0], 32)], 2)
    e_best = int(best_energies(batch, best_runs, best_sweeps)[0])
    run_best = E.min(axis=1)
    e_best = min(e_best, int(run_best.min()))
    rho_run = (run_best - e_best) / N
    mu, sd = float(rho_run.mean()), float(rho_run.std(ddof=1))
    # the Gaussian-fit check behind the EVT median: shape of the per-run
    # residual-energy distribution (Sec. S2: it skews left at long anneals)
    from scipy import stats as sst
    gauss = {"skewness": float(sst.skew(rho_run)), "excess_kurtosis": float(sst.kurtosis(rho_run)),
             "shapiro_p": float(sst.shapiro(rho_run).pvalue) if rho_run.size >= 3 else None}
    out = {"L": L, "P": P, "R": R, "T": T, "sweeps": sweeps, "anneal_seconds": dt,
           "flips_per_ns": N * P * R * sweeps / dt / 1e9, "e_best": e_best,
           "rho_single_run": {"mean": mu, "std": sd, "gaussian_check": gauss}, "best_of_R": {},
           "C_r_mean_over_runs": [float(x) for x in C_r[: P // 2 + 1]],
           "C_r_by_anneal_sweeps": C_ta,
           "C_r_length_1_over_e": int(np.argmax(C_r[: P // 2 + 1] < np.exp(-1.0))) or None}
    for r in Rs:
        g = rho_run[: (R // r) * r].reshape(-1, r).min(axis=1)
        pred = evt_median_gaussian(mu, sd, r)
        out["best_of_R"][str(r)] = {"groups": int(g.size), "mean": float(g.mean()),
                                    "median": float(np.median(g)), "evt_median_gaussian": pred,
                                    "hit_fraction_rho_le_1e-3": float((g <= 1e-3).mean())}
    return out


def c4_mixed_time_to_target(rho=1e-3, best_runs=10, best_sweeps=20000, max_sweeps=100000) -> Dict:
    """256 mixed-size instances (L in {6..16}, 24-32 geometric temperatures
    x 2): flips/ns of the fused kernel and per-instance time to rho_E."""
    batch = W.apt_mixed_batch()
    tp = apt_throughput(batch, 300, True)
    e_best = best_energies(batch, best_runs, best_sweeps)
    Ns = np.array([int(np.prod(d)) for d in batch.dims])
    targets = np.floor(e_best + rho * Ns).astype(np.int64)
    hit, t_hit, t_sweep, total = run_to_target(batch, targets, max_sweeps)
    ok = hit >= 0
    per_L = {}
    for Lv in sorted(set(int(d[0]) for d in batch.dims)):
        sel = np.array([int(d[0]) == Lv for d in batch.dims])
        h = hit[sel & ok]
        frac = float((hit[sel] >= 0).mean())
        per_L[str(Lv)] = {"instances": int(sel.sum()), "hit_fraction": frac,
                          "median_hit_sweep": float(np.median(h)) if h.size else None,
                          # measured, per instance, to the end of the chunk of its hit
                          "median_time_s": float(np.median(t_hit[sel])) if frac > 0.5 else None}
    return {"flips_per_ns_icm": tp["flips_per_ns"], "apt_seconds_per_sweep": t_sweep,
            "hit_fraction": float(ok.mean()), "per_L": per_L}


def graph_apt_throughput(graphs: Sequence[W.Graph], n_temps: int = 32, labels: int = 2, sweeps: int = 200,
                         icm: bool = True, seed: int = 1) -> Dict:
    """APT (+ICM) on general graphs: sweep updates per ns, end to end."""
    ctx = pcomp.Context(0, seed)
    timer = DeviceTimer(ctx)
    betas = [W.geometric_ladder(n_temps, 0.2, 3.0)] * len(graphs)
    pcomp.pc_gapt_load(ctx.h, [(g.rp, g.col, g.w) for g in graphs], betas, labels, 0)
    pcomp.pc_gapt_run(ctx.h, 10, 1, icm)
    dt = timer.time(lambda: pcomp.pc_gapt_run(ctx.h, sweeps, 1, icm))
    colours = max(int(pcomp.pc_gapt_get_colours(ctx.h, i, g.n).max()) + 1 for i, g in enumerate(graphs))
    ctx.close()
    per_sweep = sum(g.n for g in graphs) * n_temps * labels
    return {"flips_per_ns": per_sweep * sweeps / dt / 1e9, "seconds": dt, "sweeps": sweeps, "icm": icm,
            "spins_per_sweep": per_sweep, "colours": colours, "problems": len(graphs)}


def graph_sqa_throughput(g: W.Graph, P: int = 64, R: int = 4864, sweeps: int = 1000, T: float = 0.05,
                         seed: int = 1) -> Dict:
    """DT-SQA on a graph: spin updates per ns of one anneal (launch, tables
    and the copies of its inputs and outputs included)."""
    ctx = pcomp.Context(0, seed)
    gamma = W.linear_gamma_schedule(sweeps)
    pcomp.pc_gsqa_anneal(ctx.h, g.rp, g.col, g.w, P, T, gamma[:10], R)
    t0 = time.perf_counter()
    E = pcomp.pc_gsqa_anneal(ctx.h, g.rp, g.col, g.w, P, T, gamma, R)
    dt = time.perf_counter() - t0
    ctx.close()
    flips = g.n * P * R * sweeps
    return {"flips_per_ns": flips / dt / 1e9, "seconds": dt, "sweeps": sweeps, "P": P, "R": R, "n": g.n,
            "min_energy": int(E.min())}


def gsqa_embedded_scaling(dims=(15, 15, 12), n_inst: int = 4, Ps=(16, 64), tas=(100, 1000, 10000),
                          runs: int = 256, T: float = 0.05, best_runs: int = 4,
                          best_sweeps: int = 20000) -> Dict:
    """DT-SQA on dimer embeddings of logical +-J lattices (4 colours,
    couplings of strength 2), the embedded-instance setting of Fig. S15:
    residual energy per p-bit of the best slice, rho = (E_min - E_best)/n,
    against the annealing time t_a for P Trotter replicas, and the fitted
    slope kappa_f of log rho against log t_a.  E_best: the best of APT+ICM
    runs on the same graphs (sweep-to-swap ratio 10) and of every anneal."""
    graphs = [W.dimer_embedding(dims, W.ea_couplings(dims, W.SEED_INSTANCES, i)) for i in range(n_inst)]
    trip = [(g.rp, g.col, g.w) for g in graphs]
    best = np.full(n_inst, np.iinfo(np.int64).max, np.int64)
    t0 = time.perf_counter()
    for r in range(best_runs):
        ctx = pcomp.Context(0, 200 + r)
        pcomp.pc_gapt_load(ctx.h, trip, [W.geometric_ladder(32, 0.2, 3.0)] * n_inst, 2, 0)
        pcomp.pc_gapt_run(ctx.h, max(1, best_sweeps // 10), 10, True)
        for i, g in enumerate(graphs):
            best[i] = min(best[i], pcomp.pc_gapt_get_best(ctx.h, i, g.n)["E"])
        ctx.close()
    t_best = time.perf_counter() - t0
    emin = {}
    secs = {}
    for P in Ps:
        for ta in tas:
            gamma = W.linear_gamma_schedule(ta)
            ctx = pcomp.Context(0, 300 + P)
            t0 = time.perf_counter()
            emin[(P, ta)] = np.stack([pcomp.pc_gsqa_anneal(ctx.h, g.rp, g.col, g.w, P, T, gamma, runs).min(axis=1)
                                      for g in graphs])   # [inst][run]
            secs[(P, ta)] = time.perf_counter() - t0
            ctx.close()
            best = np.minimum(best, emin[(P, ta)].min(axis=1))
    n = graphs[0].n
    out = {"dims_logical": list(dims), "p_bits": n, "instances": n_inst, "runs": runs, "T": T,
           "apt_best_seconds": t_best, "e_best_per_pbit": [float(b / n) for b in best], "by_P": {}}
    for P in Ps:
        rows = []
        for ta in tas:
            rho = (emin[(P, ta)] - best[:, None]) / n
            rows.append({"t_a": ta, "rho_mean": float(rho.mean()), "rho_median": float(np.median(rho)),
                         "hit_fraction_rho_0": float((rho == 0).mean()), "seconds": secs[(P, ta)]})
        r = np.array([max(x["rho_mean"], 1e-12) for x in rows])
        kappa = float(-np.polyfit(np.log(np.array(tas, float)), np.log(r), 1)[0])
        out["by_P"][str(P)] = {"rows": rows, "kappa_f": kappa}
    return out


def graph_workloads(name: str) -> List[W.Graph]:
    if name == "dimer_64xL8":
        return [W.dimer_embedding((8, 8, 8), W.ea_couplings((8, 8, 8), W.SEED_INSTANCES, i)) for i in range(64)]
    if name == "lattice15x15x12_64":
        d = (15, 15, 12)
        return [W.lattice_graph(d, (1, 1, 1), W.ea_couplings(d, W.SEED_INSTANCES, i))[0] for i in range(64)]
    if name == "lattice12_64":
        d = (12, 12, 12)
        return [W.lattice_graph(d, (1, 1, 1), W.ea_couplings(d, W.SEED_INSTANCES, i))[0] for i in range(64)]
    if name == "random4096_152":
        return [W.sparse_random_graph(4096, 6.0, i, wmax=3) for i in range(152)]
    raise ValueError(name)


def graph_time_to_target(name: str = "dimer_64xL8", labels: int = 2, rho: float = 1e-3, best_runs: int = 10,
                         best_sweeps: int = 20000, max_sweeps: int = 100000, chunk: int = 256,
                         adaptive: bool = False) -> Dict:
    """Time to rho_E <= rho on a graph workload with APT+ICM on the general-
    graph kernels: 32 geometric temperatures 0.2-3.0, or (adaptive) the
    adaptive ladder resampled to 32 with its construction time included;
    E_best = the minimum over best_runs runs with sweep-to-swap ratio 10."""
    graphs = graph_workloads(name)
    trip = [(g.rp, g.col, g.w) for g in graphs]
    n_prob = len(graphs)
    t_lad = 0.0
    if adaptive:
        # Algorithm S2's preprocessing on the graph kernels, resampled to 32 temperatures
        ctx = pcomp.Context(0, 11)
        t0 = time.perf_counter()
        lad = pcomp.pc_graph_adaptive_ladder(ctx.h, trip, beta0=0.5, alpha=1.25, n_chains=32, sweeps=2000,
                                             tail=500, tol=1.0, max_len=64)
        t_lad = time.perf_counter() - t0
        ctx.close()
        betas = [pcomp.pc_resample_ladder(b, 32) for b, _, _ in lad]
    else:
        betas = [W.geometric_ladder(32, 0.2, 3.0)] * n_prob
    best = np.full(n_prob, np.iinfo(np.int64).max, np.int64)
    for r in range(best_runs):
        ctx = pcomp.Context(0, 100 + r)
        pcomp.pc_gapt_load(ctx.h, trip, betas, 2, 0)
        pcomp.pc_gapt_run(ctx.h, max(1, best_sweeps // 10), 10, True)
        for i, g in enumerate(graphs):
            best[i] = min(best[i], pcomp.pc_gapt_get_best(ctx.h, i, g.n)["E"])
        ctx.close()
    n = np.array([g.n for g in graphs])
    targets = np.floor(best + rho * n).astype(np.int64)
    ctx = pcomp.Context(0, 7)
    pcomp.pc_gapt_load(ctx.h, trip, betas, labels, 0)
    for i, t in enumerate(targets):
        pcomp.pc_gapt_set_target(ctx.h, i, int(t))
    pcomp.pc_synchronize(ctx.h)
    t0 = time.perf_counter()
    done = 0
    hit = np.full(n_prob, -1, np.int64)
    t_hit = np.full(n_prob, np.inf)
    while done < max_sweeps:
        pcomp.pc_gapt_run(ctx.h, chunk, 1, True)
        done += chunk
        hit = np.array([pcomp.pc_gapt_get_best(ctx.h, i, g.n)["hit_sweep"] for i, g in enumerate(graphs)])
        t_hit[(hit >= 0) & np.isinf(t_hit)] = time.perf_counter() - t0
        if (hit >= 0).all():
            break
    total = time.perf_counter() - t0
    ctx.close()
    ok = hit >= 0
    t_sweep = total / done
    return {"workload": name, "problems": n_prob, "labels": labels, "rho_target": rho, "adaptive": adaptive,
            "ladder_seconds": t_lad, "ladder_lengths": [len(b) for b in betas] if adaptive else None,
            "apt_seconds_per_sweep": t_sweep, "hit_fraction": float(ok.mean()),
            "median_hit_sweep": float(np.median(hit[ok])) if ok.any() else None,
            # measured per instance: ladder construction, then the run to the
            # end of the chunk in which the instance reached its target
            "median_time_to_target_s": float(np.median(t_lad + t_hit)) if ok.mean() > 0.5 else None,
            "e_best_per_spin_mean": float((best / n).mean())}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("what", choices=["throughput", "graph", "graph-ttt", "gsqa-embedded", "c2", "c3", "c4",
                                     "all"])
    ap.add_argument("--graph", choices=["dimer_64xL8", "lattice15x15x12_64", "lattice12_64", "random4096_152"])
    ap.add_argument("--graph-labels", type=int, choices=[2, 4], help="graph: one label count only")
    ap.add_argument("--no-sqa", action="store_true", help="graph: skip the DT-SQA lines")
    ap.add_argument("--sqa-only", action="store_true", help="graph: only the DT-SQA lines")
    ap.add_argument("--adaptive", action="store_true", help="graph-ttt: adaptive ladders instead of geometric")
    ap.add_argument("--sweeps", type=int, default=200)
    ap.add_argument("--batch", choices=["apt_plain_L4", "apt_icm_64xL12", "apt_icm_mixed256"])
    ap.add_argument("--icm", type=int, choices=[0, 1])
    ap.add_argument("--shape", help="throughput: threads,chunks,split_pref,split_groups (pc_apt_set_launch)")
    ap.add_argument("--best-runs", type=int, default=10)
    ap.add_argument("--best-sweeps", type=int, default=20000)
    ap.add_argument("--max-sweeps", type=int, default=100000)
    ap.add_argument("--labels", type=int, default=2, choices=[2, 4], help="ICM labels (c3)")
    args = ap.parse_args()
    out = {}
    if args.what in ("throughput", "all"):
        batches = {"apt_plain_L4": lambda: W.apt_single(L=4),
                   "apt_icm_64xL12": lambda: W.apt_uniform_batch(64, 12, 32),
                   "apt_icm_mixed256": lambda: W.apt_mixed_batch()}
        names = [args.batch] if args.batch else list(batches)
        for name in names:
            batch = batches[name]()
            for icm in ((True, False) if args.icm is None else (bool(args.icm),)):
                shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else None
                out[f"{name}_icm{int(icm)}"] = apt_throughput(batch, args.sweeps, icm, shape=shape)
    if args.what in ("graph", "all") and not args.sqa_only:
        names = [args.graph] if args.graph else ["dimer_64xL8", "lattice15x15x12_64", "lattice12_64",
                                                 "random4096_152"]
        for name in names:
            graphs = graph_workloads(name)
            for labels in ((2, 4) if args.graph_labels is None else (args.graph_labels,)):
                for icm in ((True, False) if args.icm is None else (bool(args.icm),)):
                    out[f"graph_{name}_A{labels}_icm{int(icm)}"] = graph_apt_throughput(
                        graphs, 32, labels, args.sweeps, icm)
    if args.what in ("graph", "all") and not args.no_sqa:
        out["graph_sqa_dimerL4_P64"] = graph_sqa_throughput(
            W.dimer_embedding((4, 4, 4), W.ea_couplings((4, 4, 4), W.SEED_INSTANCES, 0)), 64, 4864, 1000)
        # an embedding of the paper's 15 x 15 x 12 shape (5400 p-bits, 4 colours): a run
        # group's slices are split over a CTA cluster
        d = (15, 15, 12)
        out["graph_sqa_dimer15x15x12_P64"] = graph_sqa_throughput(
            W.dimer_embedding(d, W.ea_couplings(d, W.SEED_INSTANCES, 0)), 64, 4864, 1000)
        out["graph_sqa_lattice5x5x4_P65"] = graph_sqa_throughput(
            W.lattice_graph((5, 5, 4), (1, 1, 1), W.ea_couplings((5, 5, 4), W.SEED_INSTANCES, 0))[0], 65, 4864,
            1000)
    if args.what == "graph-ttt":
        for name in ([args.graph] if args.graph else ["dimer_64xL8", "lattice15x15x12_64"]):
            for labels in ((2, 4) if args.graph_labels is None else (args.graph_labels,)):
                out[f"gttt_{name}_A{labels}{'_adaptive' if args.adaptive else ''}"] = graph_time_to_target(
                    name, labels, best_runs=args.best_runs, best_sweeps=args.best_sweeps,
                    max_sweeps=args.max_sweeps, adaptive=args.adaptive)
    if args.what == "gsqa-embedded":
        out["gsqa_embedded"] = gsqa_embedded_scaling()
    if args.what in ("c2", "all"):
        out["c2"] = c2_residual_vs_R()
    if args.what in ("c3", "all"):
        out["c3"] = c3_time_to_target(labels=args.labels)
    if args.what in ("c4", "all"):
        out["c4"] = c4_mixed_time_to_target()
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
