"""Seeded synthetic inputs shared by the tests, the bench and the CPU oracle.

This module holds input generators only: the coupling realisations of the
3D Edwards-Anderson +-J model (each J_ij drawn from {-1,+1} with equal
probability on nearest-neighbour bonds of a periodic simple-cubic lattice),
the geometric beta ladders and the linear transverse-field schedules that the
workloads name, and the workload shapes themselves.  None of the method's
arithmetic (sweeps, thresholds, swaps, cluster moves, energies, ladders) lives
here; the random numbers the method itself draws come from each side's own
Philox4x32-10.

Coupling layout used everywhere: ``J[lin, d]`` is the coupling of the forward
bond of site ``lin = x + Lx*(y + Ly*z)`` along axis d (0:+x, 1:+y, 2:+z),
int8 in {-1,+1}; with periodic boundaries every site has all three.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence, Tuple

import numpy as np

# seed streams for instance families (instance i of a family uses [family, i])
SEED_INSTANCES = 1000
SEED_TRAIN = 2000
SEED_EVAL = 3000
SEED_MIXED = 4000


def ea_couplings(dims: Sequence[int], seed: int, index: int = 0) -> np.ndarray:
    """+-J couplings for one periodic lattice, shape [N, 3], int8."""
    lx, ly, lz = (int(v) for v in dims)
    n = lx * ly * lz
    rng = np.random.Generator(np.random.Philox(key=[seed, index]))
    bits = rng.integers(0, 2, size=(n, 3), dtype=np.int8)
    return (2 * bits - 1).astype(np.int8)


def geometric_ladder(n_temps: int, beta_min: float = 0.2, beta_max: float = 3.0) -> np.ndarray:
    """beta_r = beta_min * (beta_max/beta_min)**(r/(n-1)), r = 0..n-1."""
    if n_temps == 1:
        return np.array([beta_min], dtype=np.float64)
    r = np.arange(n_temps, dtype=np.float64) / (n_temps - 1)
    return beta_min * (beta_max / beta_min) ** r


def linear_gamma_schedule(n_sweeps: int, gamma0: float = 3.0, gamma1: float = 1e-3) -> np.ndarray:
    """Gamma_s = gamma0 + (gamma1 - gamma0) * s/(S-1), s = 0..S-1."""
    if n_sweeps == 1:
        return np.array([gamma0], dtype=np.float64)
    s = np.arange(n_sweeps, dtype=np.float64)
    return gamma0 + (gamma1 - gamma0) * s / (n_sweeps - 1)


@dataclasses.dataclass
class AptBatch:
    """A batch of APT problems: one entry per instance."""
    dims: np.ndarray          # [n, 3] int32
    J: List[np.ndarray]       # per instance [N, 3] int8
    betas: List[np.ndarray]   # per instance [n_temps] float64
    n_labels: int

    @property
    def n(self) -> int:
        return len(self.J)

    def spins_per_sweep(self) -> int:
        return int(sum(int(np.prod(d)) * len(b) * self.n_labels for d, b in zip(self.dims, self.betas)))


def apt_single(L: int = 4, n_temps: int = 8, n_labels: int = 2, seed: int = SEED_INSTANCES,
               index: int = 0) -> AptBatch:
    """One periodic L^3 instance with a geometric 0.2-3.0 ladder."""
    dims = np.array([[L, L, L]], dtype=np.int32)
    return AptBatch(dims, [ea_couplings((L, L, L), seed, index)], [geometric_ladder(n_temps)], n_labels)


def apt_uniform_batch(n_inst: int, L: int, n_temps: int, n_labels: int = 2,
                      seed: int = SEED_INSTANCES) -> AptBatch:
    dims = np.tile(np.array([L, L, L], dtype=np.int32), (n_inst, 1))
    J = [ea_couplings((L, L, L), seed, i) for i in range(n_inst)]
    return AptBatch(dims, J, [geometric_ladder(n_temps) for _ in range(n_inst)], n_labels)


def apt_mixed_batch(n_inst: int = 256, sizes: Sequence[int] = (6, 8, 10, 12, 14, 16),
                    temps: Tuple[int, int] = (24, 32), n_labels: int = 2,
                    seed: int = SEED_MIXED) -> AptBatch:
    """Mixed-size batch: L uniform over `sizes`, n_temps uniform over [temps]."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 0xFFFF]))
    Ls = rng.choice(np.asarray(sizes), size=n_inst)
    nts = rng.integers(temps[0], temps[1] + 1, size=n_inst)
    dims = np.stack([Ls, Ls, Ls], axis=1).astype(np.int32)
    J = [ea_couplings((int(L),) * 3, seed, i) for i, L in enumerate(Ls)]
    return AptBatch(dims, J, [geometric_ladder(int(t)) for t in nts], n_labels)


@dataclasses.dataclass
class SqaWorkload:
    dims: Tuple[int, int, int]
    J: np.ndarray            # [N, 3] int8
    P: int                   # Trotter slices
    R: int                   # independent runs
    T: float                 # temperature
    gamma: np.ndarray        # [S] float64

    def flips_per_anneal(self) -> int:
        return int(np.prod(self.dims)) * self.P * self.R * len(self.gamma)


def sqa_workload(L: int = 8, P: int = 64, R: int = 256, T: float = 0.05, n_sweeps: int = 10000,
                 gamma0: float = 3.0, gamma1: float = 1e-3, seed: int = SEED_INSTANCES,
                 index: int = 0) -> SqaWorkload:
    return SqaWorkload((L, L, L), ea_couplings((L, L, L), seed, index), P, R, T,
                       linear_gamma_schedule(n_sweeps, gamma0, gamma1))


def random_spins(n: int, seed: int) -> np.ndarray:
    """+-1 int8 spins (used only for host-logic tests of energy routines)."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 0xABCD]))
    return (2 * rng.integers(0, 2, size=n, dtype=np.int8) - 1).astype(np.int8)


def mlp_init(sizes: Sequence[int], seed: int) -> List[Tuple[np.ndarray, np.ndarray]]:
    """He-uniform initial weights [out, in] and zero biases, float32."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 0x4D4C50]))
    params = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        bound = np.sqrt(6.0 / fan_in)
        W = rng.uniform(-bound, bound, size=(fan_out, fan_in)).astype(np.float32)
        params.append((W, np.zeros(fan_out, dtype=np.float32)))
    return params


def pad_odd_open(dims, periodic, J) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """An instance with odd lengths on open axes (e.g. the paper's 15 x 15 x 12,
    open in x and y) as an even-length lattice whose extra end layers are
    vacancies.  Returns (padded dims, present [N_pad], J [N_pad][3]); the
    original site (x, y, z) keeps its coordinates.  Odd periodic lengths are
    not bipartite and are refused."""
    dims = [int(v) for v in dims]
    per = [int(bool(v)) for v in periodic]
    for a in range(3):
        if dims[a] % 2 and per[a]:
            raise ValueError("odd length on a periodic axis: the lattice is not bipartite")
    pd = [v + (v % 2) for v in dims]
    J = np.asarray(J, np.int8).reshape(dims[2], dims[1], dims[0], 3)
    Jp = np.ones((pd[2], pd[1], pd[0], 3), np.int8)
    Jp[: dims[2], : dims[1], : dims[0]] = J
    present = np.zeros((pd[2], pd[1], pd[0]), np.uint8)
    present[: dims[2], : dims[1], : dims[0]] = 1
    return np.array(pd, np.int32), present.ravel(), Jp.reshape(-1, 3)


def random_vacancies(dims, fraction: float, seed: int) -> np.ndarray:
    """present [N] with about `fraction` of the sites missing (seeded)."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 0xEEEE]))
    return (rng.random(int(np.prod(dims))) >= fraction).astype(np.uint8)


# ---------------------------------------------------------------- general sparse graphs
SEED_GRAPHS = 5000


@dataclasses.dataclass
class Graph:
    """A symmetric sparse graph in CSR form: the neighbours of v are
    ``col[rp[v]:rp[v+1]]`` (ascending) with integer weights ``w`` (nonzero,
    equal in both directions)."""
    rp: np.ndarray    # [n + 1] int32
    col: np.ndarray   # [m] int32
    w: np.ndarray     # [m] int8

    @property
    def n(self) -> int:
        return len(self.rp) - 1

    def edges(self) -> List[Tuple[int, int, int]]:
        """(u, v, w) with u < v, each edge once."""
        out = []
        for v in range(self.n):
            for q in range(self.rp[v], self.rp[v + 1]):
                if self.col[q] > v:
                    out.append((v, int(self.col[q]), int(self.w[q])))
        return out


def csr_from_edges(n: int, edges, weights=None) -> Graph:
    """Symmetric CSR from an undirected edge list; repeated pairs are merged by
    adding their weights and zero-weight pairs are dropped."""
    acc = {}
    edges = list(edges)
    weights = [1] * len(edges) if weights is None else list(weights)
    for (u, v), wt in zip(edges, weights):
        u, v = int(u), int(v)
        if u == v:
            raise ValueError("self-loop")
        key = (min(u, v), max(u, v))
        acc[key] = acc.get(key, 0) + int(wt)
    adj = [[] for _ in range(n)]
    for (u, v), wt in acc.items():
        if wt == 0:
            continue
        if not -127 <= wt <= 127:
            raise ValueError("weight out of int8 range")
        adj[u].append((v, wt))
        adj[v].append((u, wt))
    rp = np.zeros(n + 1, np.int32)
    col, w = [], []
    for v in range(n):
        for u, wt in sorted(adj[v]):
            col.append(u)
            w.append(wt)
        rp[v + 1] = len(col)
    return Graph(rp, np.asarray(col, np.int32), np.asarray(w, np.int8))


def lattice_graph(dims, periodic, J, present=None) -> Tuple[Graph, np.ndarray]:
    """The bond graph of a 3D lattice with couplings J [N][3] (forward bonds
    +x, +y, +z) and optional vacancies; any lengths, odd periodic ones
    included.  Vertices are the present sites in lin order; returns the graph
    and the lin of every vertex."""
    lx, ly, lz = (int(v) for v in dims)
    per = [1, 1, 1] if periodic is None else [int(bool(v)) for v in periodic]
    N = lx * ly * lz
    pres = np.ones(N, bool) if present is None else np.asarray(present).ravel().astype(bool)
    sites = np.flatnonzero(pres).astype(np.int32)
    vid = -np.ones(N, np.int64)
    vid[sites] = np.arange(len(sites))
    J = np.asarray(J, np.int8).reshape(N, 3)
    L = (lx, ly, lz)
    edges, ws = [], []
    for lin in sites:
        c = [lin % lx, (lin // lx) % ly, lin // (lx * ly)]
        for a in range(3):
            cc = list(c)
            cc[a] += 1
            if cc[a] == L[a]:
                if not per[a]:
                    continue
                cc[a] = 0
            nb = cc[0] + lx * (cc[1] + ly * cc[2])
            if nb == lin or not pres[nb]:
                continue
            edges.append((vid[lin], vid[nb]))
            ws.append(int(J[lin, a]))
    return csr_from_edges(len(sites), edges, ws), sites


def random_graph(n: int, mean_degree: float, seed: int, wmax: int = 1, index: int = 0) -> Graph:
    """Erdos-Renyi graph G(n, p = mean_degree / (n - 1)) with weights drawn
    uniformly from {-wmax..wmax} without 0."""
    rng = np.random.Generator(np.random.Philox(key=[SEED_GRAPHS + seed, index]))
    p = min(1.0, mean_degree / max(n - 1, 1))
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(len(iu)) < p
    mags = rng.integers(1, wmax + 1, size=int(keep.sum()))
    signs = 2 * rng.integers(0, 2, size=int(keep.sum())) - 1
    return csr_from_edges(n, zip(iu[keep], ju[keep]), mags * signs)


def sparse_random_graph(n: int, mean_degree: float, seed: int, wmax: int = 1, index: int = 0) -> Graph:
    """A large sparse random graph: n * mean_degree / 2 vertex pairs drawn
    uniformly (self-pairs dropped, repeated pairs merged), weights drawn
    uniformly from {-wmax..wmax} without 0 (the sum of a repeated pair's
    weights, zero sums dropped)."""
    rng = np.random.Generator(np.random.Philox(key=[SEED_GRAPHS + seed, 0x5A00 + index]))
    m = int(round(n * mean_degree / 2))
    u = rng.integers(0, n, size=m)
    v = rng.integers(0, n, size=m)
    keep = u != v
    mags = rng.integers(1, wmax + 1, size=m)
    signs = 2 * rng.integers(0, 2, size=m) - 1
    return csr_from_edges(n, zip(u[keep], v[keep]), (mags * signs)[keep])


def random_biases(n: int, hmax: int, seed: int) -> np.ndarray:
    """Biases h [n] drawn uniformly from {-hmax..hmax}."""
    rng = np.random.Generator(np.random.Philox(key=[SEED_GRAPHS + seed, 0xB1A5]))
    return rng.integers(-hmax, hmax + 1, size=n).astype(np.int8)


def dimer_embedding(dims, J, ferro: int = 2) -> Graph:
    """A logical periodic +-J lattice embedded with dimers, in the manner of
    annealer embeddings: logical spin i becomes physical spins 2i and 2i+1
    joined by a ferromagnetic coupling of strength `ferro`.  The logical bond
    along +x joins the first halves and along +y the second halves, each with
    J; the bond along +z is split over two couplers, from both halves of i to
    the second half of its neighbour, each with J.  The split couplers close
    triangles with the chains, so the graph is not bipartite."""
    lx, ly, lz = (int(v) for v in dims)
    N = lx * ly * lz
    J = np.asarray(J, np.int8).reshape(N, 3)
    edges, ws = [], []
    for lin in range(N):
        edges.append((2 * lin, 2 * lin + 1))
        ws.append(ferro)
        c = [lin % lx, (lin // lx) % ly, lin // (lx * ly)]
        for a in range(3):
            cc = list(c)
            cc[a] = (cc[a] + 1) % (lx, ly, lz)[a]
            nb = cc[0] + lx * (cc[1] + ly * cc[2])
            pairs = ((0, 0),) if a == 0 else (((1, 1),) if a == 1 else ((0, 1), (1, 1)))
            for hi, hj in pairs:
                edges.append((2 * lin + hi, 2 * nb + hj))
                ws.append(int(J[lin, a]))
    return csr_from_edges(2 * N, edges, ws)
