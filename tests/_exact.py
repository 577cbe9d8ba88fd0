"""Brute-force helpers for the oracle pins: explicit bond lists of tiny
lattices and exact Boltzmann distributions by enumerating all 2^n states."""
import itertools

import numpy as np


def lattice_edges(dims, periodic=(1, 1, 1)):
    """(i, j, axis) for every forward bond; site index x + Lx*(y + Ly*z)."""
    Lx, Ly, Lz = dims
    idx = lambda x, y, z: x + Lx * (y + Ly * z)
    edges = []
    for z, y, x in itertools.product(range(Lz), range(Ly), range(Lx)):
        c = [x, y, z]
        for a in range(3):
            d = list(c)
            d[a] += 1
            if d[a] == dims[a]:
                if not periodic[a]:
                    continue
                d[a] = 0
            edges.append((idx(*c), idx(*d), a))
    return edges


def all_states(n):
    """[2^n, n] int8 +-1; state index k has spin i = +1 iff bit i of k is set."""
    k = np.arange(2 ** n, dtype=np.int64)[:, None]
    return (2 * ((k >> np.arange(n)) & 1) - 1).astype(np.int8)


def state_index(spins):
    s = np.asarray(spins)
    return ((s > 0).astype(np.int64) << np.arange(s.shape[-1])).sum(-1)


def energies(edges, J, h, states):
    E = np.zeros(states.shape[0], dtype=np.int64)
    for (i, j, a) in edges:
        E -= int(J[i, a]) * states[:, i].astype(np.int64) * states[:, j]
    if h is not None:
        E -= (states.astype(np.int64) * np.asarray(h, np.int64)[None, :]).sum(1)
    return E


def boltzmann(E, beta):
    w = np.exp(-beta * (E - E.min()).astype(np.float64))
    return w / w.sum()


def batch_mean_stderr(x, n_batches=32):
    """Mean and batch-means standard error of a (time-ordered) sample."""
    x = np.asarray(x, np.float64)
    m = len(x) // n_batches
    b = x[: m * n_batches].reshape(n_batches, m).mean(1)
    return float(x.mean()), float(b.std(ddof=1) / np.sqrt(n_batches))
