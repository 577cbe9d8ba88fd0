"""Pins for the CPU oracle against facts fixed by the paper and mathematics.

Each test checks the oracle against something other than itself: an
independent Philox implementation, closed forms evaluated with mpmath,
exact Boltzmann distributions by enumeration, lattice graphs built by
networkx, and invariants of the moves.  Statistical checks use fixed seeds
and 5-sigma (or chi-square p > 1e-6) margins.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2503_10302_gb300 import workloads as W
from tests import _exact as X

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 50


# ---------------------------------------------------------------- Philox
_TRITON_PHILOX = r"""
import json, sys
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def k(out, cin, seed_ptr, n: tl.constexpr):
    offs = tl.arange(0, n)
    c0 = tl.load(cin + offs * 4 + 0).to(tl.uint32)
    c1 = tl.load(cin + offs * 4 + 1).to(tl.uint32)
    c2 = tl.load(cin + offs * 4 + 2).to(tl.uint32)
    c3 = tl.load(cin + offs * 4 + 3).to(tl.uint32)
    seed = tl.load(seed_ptr).to(tl.uint64)
    r0, r1, r2, r3 = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out + offs * 4 + 0, r0.to(tl.int64))
    tl.store(out + offs * 4 + 1, r1.to(tl.int64))
    tl.store(out + offs * 4 + 2, r2.to(tl.int64))
    tl.store(out + offs * 4 + 3, r3.to(tl.int64))

req = json.loads(sys.stdin.read())
ctr = np.array(req["ctr"], dtype=np.int64)
n = ctr.shape[0]
out = torch.zeros(n * 4, dtype=torch.int64)
k[(1,)](out, torch.tensor(ctr.reshape(-1)), torch.tensor([req["seed"]], dtype=torch.int64), n)
print(json.dumps((out.numpy() & 0xFFFFFFFF).tolist()))
"""


def _triton_philox(ctr, seed):
    """Triton's Philox4x32 run by its CPU interpreter in a child process (the
    interpreter must be selected before triton is imported)."""
    import json
    import os
    import subprocess
    import sys
    pytest.importorskip("triton")
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _TRITON_PHILOX], input=json.dumps(
        {"ctr": ctr.astype(np.int64).tolist(), "seed": int(seed)}), capture_output=True, text=True,
        env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.array(json.loads(r.stdout), dtype=np.uint64).astype(np.uint32).reshape(-1, 4)


def test_philox_matches_independent_implementation(orc):
    """Oracle Philox4x32-10 == Triton's Philox4x32 (10 rounds), a separately
    written implementation of Salmon et al.'s generator."""
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2 ** 32, size=(16, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    for seed in (0, 123456789, (0xDEADBEEF << 32) | 0x12345678, 2 ** 64 - 1):
        # triton's seed is int64 on the host side; pass the same bit pattern
        s64 = seed - 2 ** 64 if seed >= 2 ** 63 else seed
        ref = _triton_philox(ctr, s64)
        got = orc.philox(ctr, seed)
        assert np.array_equal(ref, got), seed


def test_philox_words_are_uniform(orc):
    ctr = np.zeros((1 << 14, 4), np.uint32)
    ctr[:, 0] = np.arange(1 << 14)
    x = orc.philox(ctr, 42)
    halves = np.concatenate([(x & 0xFFFF).ravel(), (x >> 16).ravel()])
    counts = np.bincount(halves >> 12, minlength=16)
    assert stats.chisquare(counts).pvalue > 1e-6


# ---------------------------------------------------------------- thresholds
def _floor_2_32(p):
    v = mpmath.floor(p * mpmath.mpf(2) ** 32)
    frac = p * mpmath.mpf(2) ** 32 - v
    return int(v), float(frac)


@pytest.mark.parametrize("beta", [0.2, 0.3125, 0.5, 1.0, 1.7, 3.0])
def test_pbit_threshold_closed_form(orc, beta):
    """Eq. neuron: P(+1) = (1 + tanh(beta I))/2; threshold = floor(2^32 P)."""
    for I in range(-8, 9):
        p = (1 + mpmath.tanh(mpmath.mpf(beta) * I)) / 2
        exact, frac = _floor_2_32(p)
        exact = min(exact, 2 ** 32 - 1)
        got = orc.pbit_threshold(beta, I)
        if min(frac, 1 - frac) < 1e-5:
            assert abs(got - exact) <= 1
        else:
            assert got == exact, (beta, I, got, exact)
    assert orc.pbit_threshold(beta, 0) == 2 ** 31


def test_swap_threshold_closed_form(orc):
    for dbeta in (0.01, 0.05, 0.125, 0.4):
        for dE in (-2, -4, -8, -30, -100, -400):
            exact, frac = _floor_2_32(mpmath.exp(mpmath.mpf(dbeta) * dE))
            got = orc.swap_threshold(dbeta, dE)
            if min(frac, 1 - frac) < 1e-5:
                assert abs(got - exact) <= 1
            else:
                assert got == exact


def test_jperp_closed_form(orc):
    """Eq. S.3 scaled by P: J_perp = -(P T/2) ln tanh(Gamma/(P T)), Q16.16."""
    for (g, P, T) in [(3.0, 64, 0.05), (1e-3, 64, 0.05), (0.5, 16, 0.1), (1.0, 8, 0.5)]:
        pt = mpmath.mpf(P) * mpmath.mpf(T)
        jp = -(pt / 2) * mpmath.log(mpmath.tanh(mpmath.mpf(g) / pt))
        assert orc.jperp_q(g, P, T) == int(mpmath.nint(jp * 65536))
    # schedule endpoints of the P = 64, T = 0.05 workload
    assert abs(orc.jperp_q(3.0, 64, 0.05) / 65536 - 0.4941) < 2e-3
    assert abs(orc.jperp_q(1e-3, 64, 0.05) / 65536 - 12.907) < 2e-2
    gs = np.linspace(3.0, 1e-3, 50)
    q = [orc.jperp_q(g, 64, 0.05) for g in gs]
    assert all(a < b for a, b in zip(q, q[1:]))


def test_sqa_threshold_closed_form(orc):
    beta_eff = 1 / (64 * 0.05)
    for jq in (0, 16207, 845875):
        for I in range(-6, 7, 2):
            for n in (-2, 0, 2):
                h = mpmath.mpf(I) + mpmath.mpf(jq) / 65536 * n
                p = 1 / (1 + mpmath.exp(-2 * mpmath.mpf(beta_eff) * h))
                exact, frac = _floor_2_32(p)
                exact = min(exact, 2 ** 32 - 1)
                got = orc.sqa_threshold(beta_eff, I, jq, n)
                assert abs(got - exact) <= (1 if min(frac, 1 - frac) < 1e-5 else 0)


# ---------------------------------------------------------------- energy
def _nx_energy(dims, J, s):
    """Energy over the edges of networkx's periodic grid graph (L >= 3)."""
    nx = pytest.importorskip("networkx")
    Lx, Ly, Lz = dims
    G = nx.grid_graph(dim=[Lz, Ly, Lx], periodic=True)  # nodes (x, y, z)
    idx = lambda c: c[0] + Lx * (c[1] + Ly * c[2])
    E = 0
    for u, v in G.edges():
        a = [k for k in range(3) if u[k] != v[k]][0]
        lo, hi = (u, v) if (u[a] + 1) % dims[a] == v[a] else (v, u)
        E -= int(J[idx(lo), a]) * int(s[idx(lo)]) * int(s[idx(hi)])
    return E


@pytest.mark.parametrize("dims", [(4, 4, 4), (6, 4, 8), (4, 6, 6)])
def test_energy_matches_graph_enumeration(orc, dims):
    J = W.ea_couplings(dims, 11, 0)
    for k in range(3):
        s = W.random_spins(int(np.prod(dims)), 100 + k)
        assert orc.energy(dims, J, s) == _nx_energy(dims, J, s)


def test_energy_invariants(orc):
    dims = (4, 4, 4)
    N = 64
    ferro = np.ones((N, 3), np.int8)
    assert orc.energy(dims, ferro, np.ones(N, np.int8)) == -3 * N
    J = W.ea_couplings(dims, 5, 0)
    s = W.random_spins(N, 9)
    assert orc.energy(dims, J, s) == orc.energy(dims, J, -s)       # global flip, h = 0
    assert orc.energy(dims, J, np.ones(N, np.int8)) == -int(J.sum())
    # all energies of one instance share the parity of the bond count
    e = [orc.energy(dims, J, W.random_spins(N, k)) for k in range(20)]
    assert len({v % 2 for v in e}) == 1


# ---------------------------------------------------------------- sampler
def _sample_states(orc, dims, J, beta, n_chains, n_sweeps, burn, h=None, periodic=(1, 1, 1)):
    """Chains = independent entries of the same problem; one state per sweep."""
    apt = orc.Apt(np.tile(np.asarray(dims), (n_chains, 1)), [J] * n_chains,
                  [np.array([beta])] * n_chains, n_labels=1, seed=3,
                  h_list=None if h is None else [h] * n_chains,
                  periodic=np.tile(np.asarray(periodic), (n_chains, 1)))
    apt.run(burn, icm=False)
    out = []
    for _ in range(n_sweeps):
        apt.run(1, icm=False)
        out.append(np.stack([apt.state(i)[0][0] for i in range(n_chains)]))
    return np.stack(out)  # [sweeps, chains, N]


def _check_distribution(samples, p_exact, what, fold_global_flip=False):
    k = X.state_index(samples.reshape(-1, samples.shape[-1]))
    if fold_global_flip:
        # with h = 0, exp(-beta E) is symmetric under s -> -s; a Gibbs chain
        # hops between a low state and its mirror image slowly, so compare
        # the distribution of the mirror-pair classes
        full = len(p_exact) - 1
        k = np.minimum(k, full - k)
        pf = np.zeros_like(p_exact)
        np.add.at(pf, np.minimum(np.arange(len(p_exact)), full - np.arange(len(p_exact))), p_exact)
        p_exact = pf
    counts = np.bincount(k, minlength=len(p_exact)).astype(np.float64)
    n = counts.sum()
    mask = p_exact * n >= 5
    exp = p_exact[mask] * n
    obs = counts[mask]
    rest_o, rest_e = counts[~mask].sum(), p_exact[~mask].sum() * n
    if rest_e > 0:
        obs = np.append(obs, rest_o)
        exp = np.append(exp, rest_e)
    chi2 = ((obs - exp) ** 2 / exp).sum()
    # consecutive sweeps of one chain are correlated; inflate by 2x
    pval = stats.chi2.sf(chi2 / 2.0, len(obs) - 1)
    assert pval > 1e-6, (what, chi2, len(obs))
    tv = 0.5 * np.abs(counts / n - p_exact).sum()
    return tv


@pytest.mark.parametrize("beta", [0.3, 1.0])
def test_gibbs_sampler_matches_enumeration_periodic(orc, beta):
    """p-bit sweeps sample exp(-beta E) (Eq. boltz_prob) on the 8-spin 2x2x2
    periodic lattice (double bonds on length-2 axes)."""
    dims = (2, 2, 2)
    J = W.ea_couplings(dims, 21, 0)
    E = X.energies(X.lattice_edges(dims), J, None, X.all_states(8))
    p = X.boltzmann(E, beta)
    s = _sample_states(orc, dims, J, beta, n_chains=32, n_sweeps=1500, burn=20)
    tv = _check_distribution(s, p, f"beta={beta}", fold_global_flip=True)
    assert tv < 0.02
    Es = np.array([[orc.energy(dims, J, s[t, c]) for c in range(0, 32, 4)] for t in range(0, 1500, 3)])
    m, se = X.batch_mean_stderr(Es.T.ravel())
    assert abs(m - (p * E).sum()) < 5 * se + 1e-9


def test_vacancies_remove_their_bonds(orc):
    """A vacancy (missing spin) has no bonds: the lattice energy equals the
    explicit graph energy over the bonds between present sites, whatever
    the vacancy spins are."""
    rng = np.random.default_rng(3)
    for dims, per in (((4, 4, 4), (1, 1, 1)), ((4, 2, 6), (0, 1, 0)), ((6, 4, 2), (0, 0, 1))):
        J = W.ea_couplings(dims, 61, 0)
        N = int(np.prod(dims))
        present = (rng.random(N) > 0.2).astype(np.uint8)
        edges = [e for e in X.lattice_edges(dims, per) if present[e[0]] and present[e[1]]]
        for _ in range(5):
            s = rng.choice(np.array([-1, 1], np.int8), size=N)
            want = int(X.energies(edges, J, None, s[None, :])[0])
            assert orc.energy(dims, J, s, periodic=per, present=present) == want
            s2 = s.copy()
            s2[present == 0] *= -1          # vacancy spins do not count
            assert orc.energy(dims, J, s2, periodic=per, present=present) == want


def test_gibbs_sampler_with_vacancies_matches_enumeration(orc):
    """The present spins of a lattice with vacancies sample exp(-beta E) of
    the graph without them (12 present spins of a 2x2x4 lattice)."""
    dims, per = (2, 2, 4), (0, 0, 1)
    J = W.ea_couplings(dims, 62, 0)
    present = np.ones(16, np.uint8)
    present[[3, 9, 14, 6]] = 0
    keep = np.flatnonzero(present)
    beta = 0.7
    edges = [e for e in X.lattice_edges(dims, per) if present[e[0]] and present[e[1]]]
    n = 32
    apt = orc.Apt(np.tile(dims, (n, 1)), [J] * n, [np.array([beta])] * n, n_labels=1, seed=8,
                  periodic=np.tile(per, (n, 1)), present_list=[present] * n)
    apt.run(20, icm=False)
    Es = []
    for _ in range(1500):
        apt.run(1, icm=False)
        for i in range(0, n, 2):
            s, e, _ = apt.state(i)
            Es.append(e[0])
    # exact mean energy over the 2^12 states of the present spins
    sub = X.all_states(len(keep))
    states = np.ones((sub.shape[0], 16), np.int8)
    states[:, keep] = sub
    E = X.energies(edges, J, None, states)
    p = X.boltzmann(E, beta)
    m, se = X.batch_mean_stderr(np.array(Es, float).reshape(1500, n // 2).T.ravel())
    assert abs(m - (p * E).sum()) < 5 * se


def test_icm_with_vacancies_keeps_product_boltzmann(orc):
    """Two labels with ICM on a lattice with vacancies: each replica keeps
    exp(-beta E) of the graph without the missing spins."""
    dims, per = (2, 2, 4), (1, 1, 1)
    J = W.ea_couplings(dims, 63, 0)
    present = np.ones(16, np.uint8)
    present[[2, 13]] = 0
    keep = np.flatnonzero(present)
    beta = 0.9
    edges = [e for e in X.lattice_edges(dims, per) if present[e[0]] and present[e[1]]]
    sub = X.all_states(len(keep))
    states = np.ones((sub.shape[0], 16), np.int8)
    states[:, keep] = sub
    E = X.energies(edges, J, None, states)
    p = X.boltzmann(E, beta)
    n = 24
    apt = orc.Apt(np.tile(dims, (n, 1)), [J] * n, [np.array([beta])] * n, n_labels=2, seed=5,
                  present_list=[present] * n)
    apt.run(10, icm=True)
    Ea = []
    for _ in range(1200):
        apt.run(1, icm=True)
        for i in range(n):
            s, e, _ = apt.state(i)
            assert e[0] == orc.energy(dims, J, s[0], present=present)
            Ea.append(e[0])
    _, _, icm = apt.stats(0)
    assert icm[1] + icm[2] > 0
    m, se = X.batch_mean_stderr(np.array(Ea, float).reshape(1200, n).T.ravel())
    assert abs(m - (p * E).sum()) < 5 * se


def test_gibbs_sampler_open_lattice_with_field(orc):
    """Open x, y / periodic z with integer fields: 16 spins, exact by enumeration."""
    dims, per = (2, 2, 4), (0, 0, 1)
    J = W.ea_couplings(dims, 31, 0)
    rng = np.random.default_rng(4)
    h = rng.integers(-1, 2, size=16).astype(np.int8)
    beta = 0.6
    E = X.energies(X.lattice_edges(dims, per), J, h, X.all_states(16))
    p = X.boltzmann(E, beta)
    s = _sample_states(orc, dims, J, beta, n_chains=32, n_sweeps=1500, burn=20, h=h, periodic=per)
    flat = s.reshape(-1, 16)
    Es = E[X.state_index(flat)]
    m, se = X.batch_mean_stderr(Es.reshape(1500, 32).T.ravel())
    assert abs(m - (p * E).sum()) < 5 * se
    mag = flat.astype(np.float64).mean(0)
    mag_exact = (p[:, None] * X.all_states(16)).sum(0)
    assert np.abs(mag - mag_exact).max() < 0.05


def test_single_spin_in_field(orc):
    """One spin, no bonds: P(+1) = 1/(1 + exp(-2 beta h))."""
    dims, per = (1, 1, 1), (0, 0, 0)
    J = np.zeros((1, 3), np.int8)
    for h0, beta in [(1, 0.4), (-2, 0.3)]:
        s = _sample_states(orc, dims, J, beta, 64, 400, 0, h=np.array([h0], np.int8), periodic=per)
        frac = (s > 0).mean()
        p = 1 / (1 + math.exp(-2 * beta * h0))
        n = s.size
        assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / n)


def test_ring_mean_energy_closed_form(orc):
    """1D +-J ring: Z = 2^N [prod cosh(beta J) + prod sinh(beta J)]."""
    N = 16
    dims, per = (N, 1, 1), (1, 0, 0)
    J = np.zeros((N, 3), np.int8)
    J[:, 0] = W.ea_couplings((N, 1, 1), 41, 0)[:, 0]
    sgn = int(np.prod(J[:, 0]))
    for beta in (0.4, 1.2):
        C, S = math.cosh(beta) ** N, sgn * math.sinh(beta) ** N
        e_exact = -(N * C * math.tanh(beta) + N * S / math.tanh(beta)) / (C + S)
        s = _sample_states(orc, dims, J, beta, 16, 1500, 20, periodic=per)
        idx = np.arange(N)
        Es = -(J[idx, 0][None, None, :] * s * np.roll(s, -1, axis=2)).sum(-1)
        m, se = X.batch_mean_stderr(Es.T.ravel())
        assert abs(m - e_exact) < 5 * se


# ---------------------------------------------------------------- swaps
def test_parallel_tempering_stationary_per_temperature(orc):
    """Sweeps + replica exchange keep each temperature's marginal at
    exp(-beta_r E); the sampled swap acceptance equals the exact
    E[min(1, exp(dbeta dE))] under the product measure."""
    dims = (2, 2, 2)
    J = W.ea_couplings(dims, 51, 0)
    betas = np.array([0.25, 0.7, 1.3])
    E = X.energies(X.lattice_edges(dims), J, None, X.all_states(8))
    n_ch, n_sw = 32, 2000
    apt = orc.Apt(np.tile([2, 2, 2], (n_ch, 1)), [J] * n_ch, [betas] * n_ch, n_labels=1, seed=9)
    apt.run(20, icm=False)
    per_t = [[] for _ in betas]
    for _ in range(n_sw):
        apt.run(1, icm=False)
        for i in range(n_ch):
            s, e, temp = apt.state(i)
            for b in range(3):
                per_t[temp[b]].append(X.state_index(s[b]))
    for r, beta in enumerate(betas):
        p = X.boltzmann(E, beta)
        k = np.array(per_t[r])
        Es = E[k]
        m, se = X.batch_mean_stderr(Es.reshape(n_sw, n_ch).T.ravel())
        assert abs(m - (p * E).sum()) < 5 * se, r
    att = np.zeros((2, 1)); acc = np.zeros((2, 1))
    for i in range(n_ch):
        a, c, _ = apt.stats(i)
        att += a; acc += c
    for r in range(2):
        p0, p1 = X.boltzmann(E, betas[r]), X.boltzmann(E, betas[r + 1])
        dE = E[None, :] - E[:, None]            # E_{r+1} - E_r
        acc_exact = (p0[:, None] * p1[None, :] * np.minimum(1, np.exp((betas[r + 1] - betas[r]) * dE))).sum()
        rate = acc[r, 0] / att[r, 0]
        assert abs(rate - acc_exact) < 5 * math.sqrt(acc_exact * (1 - acc_exact) / att[r, 0]) * 2


def test_swap_parity_schedule(orc):
    """Even attempts pair (0,1),(2,3)..; odd attempts (1,2),(3,4).. (Methods)."""
    b = W.apt_single(L=4, n_temps=6)
    apt = orc.Apt(b.dims, b.J, b.betas, n_labels=2, seed=1)
    apt.run(1, icm=False)
    att, _, _ = apt.stats(0)
    assert att[:, 0].tolist() == [1, 0, 1, 0, 1]
    apt.run(1, icm=False)
    att, _, _ = apt.stats(0)
    assert att[:, 0].tolist() == [1, 1, 1, 1, 1]
    assert (att[:, 0] == att[:, 1]).all()


# ---------------------------------------------------------------- ICM
def _components(dims, mask):
    nx = pytest.importorskip("networkx")
    Lx, Ly, Lz = dims
    G = nx.grid_graph(dim=[Lz, Ly, Lx], periodic=True)
    idx = lambda c: c[0] + Lx * (c[1] + Ly * c[2])
    H = G.subgraph([v for v in G.nodes if mask[idx(v)]])
    return [sorted(idx(v) for v in comp) for comp in nx.connected_components(H)]


def test_icm_moves_a_connected_component(orc):
    dims = (4, 4, 4)
    N = 64
    J = W.ea_couplings(dims, 61, 0)
    rng = np.random.default_rng(2)
    seen = {0: 0, 1: 0, 2: 0}
    for t in range(300):
        sa = W.random_spins(N, 1000 + t)
        # mismatch densities from sparse to dense
        flip = rng.random(N) < (0.05 + 0.9 * (t % 10) / 10)
        sb = np.where(flip, -sa, sa).astype(np.int8)
        if t % 37 == 0:
            sb = sa.copy()
        br, size, a2, b2 = orc.icm_apply(dims, sa, sb, seed=5, t=t)
        seen[br] += 1
        Ea, Eb = orc.energy(dims, J, sa), orc.energy(dims, J, sb)
        Ea2, Eb2 = orc.energy(dims, J, a2), orc.energy(dims, J, b2)
        mism = sa != sb
        comps = _components(dims, mism)
        if br == 0:
            assert not mism.any() and (a2 == sa).all() and (b2 == sb).all()
            continue
        if br == 1:
            flipped = np.nonzero(a2 != sa)[0].tolist()
            assert flipped == np.nonzero(b2 != sb)[0].tolist()
            assert flipped in comps and len(flipped) == size and 2 * size <= N
            assert Ea + Eb == Ea2 + Eb2                      # isoenergetic
            assert ((a2 != b2) == mism).all()                # overlap preserved
        else:
            assert 2 * size > N and size in [len(c) for c in comps]
            fa, fb = (a2 == -sa).all(), (b2 == -sb).all()
            assert fa != fb and ((a2 == sa).all() or (b2 == sb).all())
            assert Ea == Ea2 and Eb == Eb2                   # h = 0: global flip
    assert all(v > 0 for v in seen.values()), seen


def test_icm_seed_is_uniform_over_mismatch_sites(orc):
    """The chosen cluster is the component of a uniform mismatch site, so a
    component is chosen with probability size / n_minus."""
    dims = (4, 4, 4)
    N = 64
    sa = np.ones(N, np.int8)
    sb = sa.copy()
    blobs = [[0, 1, 2, 3], [42], [23, 39]]   # three separate clusters
    for c in blobs:
        sb[c] = -1
    comps = _components(dims, sa != sb)
    assert len(comps) == 3
    counts = {tuple(c): 0 for c in comps}
    n = 6000
    for t in range(n):
        br, size, a2, b2 = orc.icm_apply(dims, sa, sb, seed=77, t=t)
        counts[tuple(np.nonzero(a2 != sa)[0].tolist())] += 1
    nminus = sum(len(c) for c in comps)
    obs = np.array([counts[tuple(c)] for c in comps], np.float64)
    exp = np.array([len(c) / nminus * n for c in comps])
    assert stats.chisquare(obs, exp).pvalue > 1e-6


def test_icm_cluster_seed_is_uniform_over_clusters(orc):
    """Under the cluster-seed rule ("randomly pick one cluster" read as a
    uniform cluster) each of the three mismatch clusters is chosen with
    probability 1/3 whatever its size, and the number of choices is the
    number of networkx components of the mismatch set."""
    dims = (4, 4, 4)
    N = 64
    sa = np.ones(N, np.int8)
    sb = sa.copy()
    for c in [[0, 1, 2, 3], [42], [23, 39]]:
        sb[c] = -1
    comps = _components(dims, sa != sb)
    assert orc.icm_choice(dims, sa, sb, 0, cluster_seed=True)[1] == len(comps) == 3
    counts = {tuple(c): 0 for c in comps}
    n = 6000
    for t in range(n):
        br, size, a2, b2 = orc.icm_apply_rules(dims, sa, sb, seed=77, t=t, cluster_seed=True)
        counts[tuple(np.nonzero(a2 != sa)[0].tolist())] += 1
    obs = np.array([counts[tuple(c)] for c in comps], np.float64)
    assert stats.chisquare(obs, np.full(3, n / 3)).pvalue > 1e-6
    rng = np.random.default_rng(5)
    for t in range(40):     # random overlaps: choices = components, chosen set = a component
        sa = W.random_spins(N, 3000 + t)
        sb = np.where(rng.random(N) < 0.1 + 0.02 * t, -sa, sa).astype(np.int8)
        comps = _components(dims, sa != sb)
        br, nc, size, a2, b2 = orc.icm_choice(dims, sa, sb, 0, big_cluster_rule=False, cluster_seed=True)
        assert nc == len(comps)
        if nc:
            k = int(rng.integers(nc))
            br, _, size, a2, b2 = orc.icm_choice(dims, sa, sb, k, big_cluster_rule=False, cluster_seed=True)
            assert br == 1 and np.nonzero(a2 != sa)[0].tolist() in comps


def _icm_moves(orc, dims, sa, sb, big, seed_rule):
    """{y: T[x -> y]} of one ICMop from x = (s^a, s^b), from the oracle's
    move with each of its random choices (seed choice k, replica bit)
    weighted uniformly; y = (index of s^a', index of s^b')."""
    _, n, _, _, _ = orc.icm_choice(dims, sa, sb, 0, False, big, seed_rule)
    if n == 0:
        return {(int(X.state_index(sa)), int(X.state_index(sb))): 1.0}
    out = {}
    for k in range(n):
        for fb in (0, 1):
            _, _, _, a2, b2 = orc.icm_choice(dims, sa, sb, k, fb, big, seed_rule)
            y = (int(X.state_index(a2)), int(X.state_index(b2)))
            out[y] = out.get(y, 0.0) + 0.5 / n
    return out


@pytest.mark.parametrize("seed_rule", [False, True])
def test_icm_transition_matrix_is_symmetric_without_big_cluster_rule(orc, seed_rule):
    """With the big-cluster branch off, ICMop is an exact symmetric move
    on pairs of states (a cluster flip keeps the overlap, hence the set of
    choices): T[x -> y] = T[y -> x] on a 2 x 2 x 2 lattice for every one of
    the 256 overlaps, with 16 seeded s^a each, for the site seed and the
    cluster seed; rows sum to 1 and every move keeps E_a + E_b, so the
    product Boltzmann law at one temperature is stationary.  With the
    branch on, T is not symmetric: a cluster of 7 of the 8 spins flips one
    whole replica, and no move leads back."""
    dims = (2, 2, 2)
    states = X.all_states(8)
    J = W.ea_couplings(dims, 62, 0)
    E = X.energies(X.lattice_edges(dims), J, None, states)
    rng = np.random.default_rng(9)
    for iq in range(256):
        q = states[iq]
        for ia in rng.choice(256, size=16, replace=False):
            sa = states[ia]
            sb = (sa * q).astype(np.int8)
            x = (int(ia), int(X.state_index(sb)))
            fwd = _icm_moves(orc, dims, sa, sb, False, seed_rule)
            assert abs(sum(fwd.values()) - 1.0) < 1e-12
            for y, p in fwd.items():
                back = _icm_moves(orc, dims, states[y[0]], states[y[1]], False, seed_rule)
                assert abs(back.get(x, 0.0) - p) < 1e-12, (x, y)
                assert E[x[0]] + E[x[1]] == E[y[0]] + E[y[1]]
    sa = states[0]
    sb = sa.copy()
    sb[:7] = -sb[:7]                    # one mismatch cluster of 7 sites
    x = (0, int(X.state_index(sb)))
    fwd = _icm_moves(orc, dims, sa, sb, True, False)
    assert any(_icm_moves(orc, dims, states[y[0]], states[y[1]], True, False).get(x, 0.0) != p
               for y, p in fwd.items())


def test_joint_label_swaps_keep_product_boltzmann(orc):
    """Joint swaps (one decision moves both labels of a temperature pair):
    each temperature's marginal stays exp(-beta_r E), and the acceptance
    equals E[min(1, exp(dbeta (dE_1 + dE_2)))] under the product measure,
    computed exactly from the convolution of the two labels' dE laws."""
    dims = (2, 2, 2)
    J = W.ea_couplings(dims, 53, 0)
    betas = np.array([0.3, 0.8, 1.4])
    E = X.energies(X.lattice_edges(dims), J, None, X.all_states(8))
    n_ch, n_sw = 32, 1500
    apt = orc.Apt(np.tile([2, 2, 2], (n_ch, 1)), [J] * n_ch, [betas] * n_ch, n_labels=2, seed=12)
    apt.set_joint_swap(True)
    apt.run(20, icm=False)
    per_t = [[] for _ in betas]
    for _ in range(n_sw):
        apt.run(1, icm=False)
        for i in range(n_ch):
            s, e, temp = apt.state(i)
            for b in range(6):
                per_t[temp[b]].append(e[b])
    for r, beta in enumerate(betas):
        p = X.boltzmann(E, beta)
        m, se = X.batch_mean_stderr(np.array(per_t[r], float).reshape(n_sw, n_ch * 2).T.ravel())
        assert abs(m - (p * E).sum()) < 5 * se, r
    att = np.zeros((2, 2)); acc = np.zeros((2, 2))
    for i in range(n_ch):
        a, c, _ = apt.stats(i)
        att += a; acc += c
        assert np.array_equal(a[:, 0], a[:, 1]) and np.array_equal(c[:, 0], c[:, 1])
    for r in range(2):
        p0, p1 = X.boltzmann(E, betas[r]), X.boltzmann(E, betas[r + 1])
        # law of dE = E_{r+1} - E_r for one label
        law = {}
        for ea, pa in zip(E, p0):
            for eb, pb in zip(E, p1):
                law[eb - ea] = law.get(eb - ea, 0.0) + pa * pb
        db = betas[r + 1] - betas[r]
        acc_exact = sum(q1 * q2 * min(1.0, math.exp(db * (d1 + d2)))
                        for d1, q1 in law.items() for d2, q2 in law.items())
        rate = acc[r, 0] / att[r, 0]
        assert abs(rate - acc_exact) < 10 * math.sqrt(acc_exact * (1 - acc_exact) / att[r, 0])


def test_icm_keeps_product_boltzmann(orc):
    """Two labels at one temperature with sweeps + ICM: each replica's
    marginal stays exp(-beta E) and the pair is independent."""
    dims = (2, 2, 2)
    J = W.ea_couplings(dims, 71, 0)
    beta = 0.9
    E = X.energies(X.lattice_edges(dims), J, None, X.all_states(8))
    p = X.boltzmann(E, beta)
    n_ch, n_sw = 32, 1500
    apt = orc.Apt(np.tile([2, 2, 2], (n_ch, 1)), [J] * n_ch, [np.array([beta])] * n_ch, n_labels=2, seed=4)
    apt.run(10, icm=True)
    Ea, Eb = [], []
    for _ in range(n_sw):
        apt.run(1, icm=True)
        for i in range(n_ch):
            _, e, _ = apt.state(i)
            Ea.append(e[0]); Eb.append(e[1])
    _, _, icm = apt.stats(0)
    assert icm[1] + icm[2] > 0
    mean = (p * E).sum()
    for arr in (Ea, Eb):
        m, se = X.batch_mean_stderr(np.array(arr).reshape(n_sw, n_ch).T.ravel())
        assert abs(m - mean) < 5 * se
    cov = np.cov(np.array(Ea, float), np.array(Eb, float))[0, 1]
    var = (p * E ** 2).sum() - mean ** 2
    assert abs(cov) < 0.1 * var


def test_icm_pairing_is_a_uniform_random_partition(orc):
    """Four labels: every draw is one of the three perfect matchings of
    {0,1,2,3}, each with probability 1/3 (chi-square, 2 d.o.f.); two labels
    always pair (0, 1)."""
    counts = np.zeros(3)
    allowed = {(0, 1, 2, 3): 0, (0, 2, 1, 3): 1, (0, 3, 1, 2): 2}
    for r in range(40):
        for t in range(300):
            m, q = orc.icm_pairing(13, 5, r, t, 4)
            assert allowed[tuple(q)] == m
            counts[m] += 1
            assert orc.icm_pairing(13, 5, r, t, 2) == (0, [0, 1])
    exp = counts.sum() / 3
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 13.8      # p = 0.001 for 2 degrees of freedom


def test_icm_four_labels_keep_product_boltzmann(orc):
    """Four labels at one temperature with sweeps + two random-pair ICMs per
    attempt: every label's marginal stays exp(-beta E), and labels stay
    uncorrelated."""
    dims = (2, 2, 2)
    J = W.ea_couplings(dims, 73, 0)
    beta = 0.8
    E = X.energies(X.lattice_edges(dims), J, None, X.all_states(8))
    p = X.boltzmann(E, beta)
    n_ch, n_sw = 24, 1200
    apt = orc.Apt(np.tile([2, 2, 2], (n_ch, 1)), [J] * n_ch, [np.array([beta])] * n_ch, n_labels=4, seed=6)
    apt.run(10, icm=True)
    Es = [[] for _ in range(4)]
    for _ in range(n_sw):
        apt.run(1, icm=True)
        for i in range(n_ch):
            s, e, _ = apt.state(i)
            for a in range(4):
                assert e[a] == orc.energy(dims, J, s[a])
                Es[a].append(e[a])
    _, _, icm = apt.stats(0)
    assert icm[1] + icm[2] > 0 and icm.sum() == 2 * (n_sw + 10)
    mean = (p * E).sum()
    var = (p * E ** 2).sum() - mean ** 2
    for arr in Es:
        m, se = X.batch_mean_stderr(np.array(arr).reshape(n_sw, n_ch).T.ravel())
        assert abs(m - mean) < 5 * se
    for a in range(4):
        for b in range(a + 1, 4):
            assert abs(np.cov(np.array(Es[a], float), np.array(Es[b], float))[0, 1]) < 0.1 * var


# ---------------------------------------------------------------- APT run
def test_apt_energies_and_best_consistent(orc):
    b = W.apt_single(L=4)
    apt = orc.Apt(b.dims, b.J, b.betas, n_labels=2, seed=0)
    apt.run(200)
    s, E, temp = apt.state(0)
    for k in range(s.shape[0]):
        assert E[k] == orc.energy((4, 4, 4), b.J[0], s[k])
    assert sorted(temp.tolist()) == sorted(list(range(8)) * 2)
    best = apt.best(0)
    assert best["E"] == orc.energy((4, 4, 4), b.J[0], best["spins"]) and best["E"] <= E.min()
    assert 0 < best["sweep"] <= 200


def test_apt_thread_count_invariance(orc):
    b = W.apt_uniform_batch(6, 4, 5)
    res = []
    for th in (1, 3):
        apt = orc.Apt(b.dims, b.J, b.betas, n_labels=2, seed=8)
        apt.run(50, threads=th)
        res.append([apt.state(i) for i in range(6)])
    for x, y in zip(*res):
        for u, v in zip(x, y):
            assert np.array_equal(u, v)


def test_apt_resume_equals_single_run(orc):
    b = W.apt_single(L=4)
    a1 = orc.Apt(b.dims, b.J, b.betas, seed=2); a1.run(60)
    a2 = orc.Apt(b.dims, b.J, b.betas, seed=2); a2.run(25); a2.run(35)
    for u, v in zip(a1.state(0), a2.state(0)):
        assert np.array_equal(u, v)
    assert a1.best(0)["E"] == a2.best(0)["E"]


def test_apt_finds_ground_state_of_tiny_instance(orc):
    """APT+ICM reaches the exact ground energy of a 2x2x4 periodic instance."""
    dims = (2, 2, 4)
    J = W.ea_couplings(dims, 81, 0)
    E = X.energies(X.lattice_edges(dims), J, None, X.all_states(16))
    apt = orc.Apt(np.array([dims]), [J], [W.geometric_ladder(6)], seed=0)
    apt.set_target(0, int(E.min()))
    apt.run(300)
    best = apt.best(0)
    assert best["E"] == E.min() and 0 < best["hit_sweep"] <= best["sweep"]


# ---------------------------------------------------------------- DT-SQA
def test_sqa_decoupled_rings_closed_form(orc):
    """J = 0: every site is a P-ring with coupling J_perp at beta_eff, so
    <s_k s_k+1> = (t + t^(P-1)) / (1 + t^P), t = tanh(beta_eff J_perp)."""
    dims = (2, 2, 2)
    J = np.zeros((8, 3), np.int8)
    P, T, g = 8, 0.5, 1.5
    jq = orc.jperp_q(g, P, T)
    t = math.tanh(jq / 65536 / (P * T))
    corr_exact = (t + t ** (P - 1)) / (1 + t ** P)
    R = 256
    E, s = orc.sqa_anneal(dims, J, P, T, np.full(60, g), R, seed=3, want_spins=True)
    c = (s * np.roll(s, -1, axis=1)).astype(np.float64).mean(axis=(1, 2))   # per run
    assert abs(c.mean() - corr_exact) < 5 * c.std(ddof=1) / math.sqrt(R)
    assert (E == 0).all()


@pytest.mark.parametrize("gamma", [0.4, 50.0])
def test_sqa_matches_enumeration(orc, gamma):
    """Ring of 4 spins x 4 slices (16 spins): the joint state distribution is
    exp(-H_C/(P T)) with H_C of Eq. S.3 (scaled by P), exact by enumeration."""
    dims, per = (4, 1, 1), (1, 0, 0)
    N, P, T = 4, 4, 0.3
    J = np.zeros((N, 3), np.int8)
    J[:, 0] = np.array([1, -1, 1, 1], np.int8)
    jq = orc.jperp_q(gamma, P, T)
    st = X.all_states(N * P).reshape(-1, P, N)    # state k: slice-major
    Hc = np.zeros(st.shape[0])
    for k in range(P):
        for i in range(N):
            Hc -= J[i, 0] * st[:, k, i] * st[:, k, (i + 1) % N]
            Hc -= jq / 65536 * st[:, k, i] * st[:, (k + 1) % P, i]
    p = np.exp(-(Hc - Hc.min()) / (P * T)); p /= p.sum()
    R = 3000
    _, s = orc.sqa_anneal(dims, J, P, T, np.full(40, gamma), R, seed=6, want_spins=True, periodic=per)
    k = X.state_index(s.reshape(R, P * N))
    counts = np.bincount(k, minlength=p.size).astype(float)
    # compare on the H_C levels (few categories, exact probabilities)
    levels, inv = np.unique(np.round(Hc, 9), return_inverse=True)
    pl = np.bincount(inv, weights=p)
    ol = np.bincount(inv, weights=counts)
    mask = pl * R >= 5
    obs = np.append(ol[mask], ol[~mask].sum())
    exp = np.append(pl[mask] * R, pl[~mask].sum() * R)
    if exp[-1] == 0:
        obs, exp = obs[:-1], exp[:-1]
    assert stats.chisquare(obs, exp).pvalue > 1e-6


def test_sqa_slices_align_when_transverse_field_vanishes(orc):
    dims = (4, 4, 4)
    J = W.ea_couplings(dims, 91, 0)
    # P T = 3.2 as in the 64-slice, T = 0.05 workload: J_perp grows to ~12.9
    _, s = orc.sqa_anneal(dims, J, 16, 0.2, W.linear_gamma_schedule(300), 4, seed=1, want_spins=True)
    agree = (s == s[:, :1, :]).mean()
    assert agree > 0.99


# ---------------------------------------------------------------- ladder
def test_adaptive_ladder_first_step_closed_form(orc):
    """On a +-J ring Var(E) = d^2 ln Z / d beta^2 is known, so the first
    ladder step beta_1 - beta_0 = alpha / sigma_E pins the standard-deviation
    reading of sigma_E and the alpha/sigma_E rule (Algorithm S2)."""
    N = 64
    dims, per = (N, 1, 1), (1, 0, 0)
    J = np.zeros((N, 3), np.int8)
    J[:, 0] = W.ea_couplings((N, 1, 1), 43, 0)[:, 0]
    sgn = int(np.prod(J[:, 0]))
    b0 = 0.5
    lnZ = lambda b: mpmath.log(mpmath.cosh(b) ** N + sgn * mpmath.sinh(b) ** N)
    var = float(mpmath.diff(lnZ, mpmath.mpf(b0), 2))
    beta, sig, ok = orc.adaptive_ladder(dims, J, beta0=b0, alpha=1.25, n_chains=64, sweeps=600,
                                        tail=500, tol=1.0, max_len=3, periodic=per)
    assert abs(sig[0] - math.sqrt(var)) < 0.05 * math.sqrt(var)
    assert beta[1] == pytest.approx(b0 + 1.25 / sig[0], rel=1e-12)


def test_adaptive_ladder_stop_rules(orc):
    dims = (4, 4, 4)
    zero = np.zeros((64, 3), np.int8)
    beta, sig, ok = orc.adaptive_ladder(dims, zero, n_chains=8, sweeps=20, tail=10)
    assert ok and len(beta) == 1 and sig[0] == 0.0
    J = W.ea_couplings(dims, 3, 0)
    beta, sig, ok = orc.adaptive_ladder(dims, J, n_chains=8, sweeps=40, tail=20, max_len=3)
    assert not ok and len(beta) == 3
    beta, sig, ok = orc.adaptive_ladder(dims, J, n_chains=16, sweeps=200, tail=100, max_len=64)
    assert ok and np.all(np.diff(beta) > 0) and sig[-1] < 1.0 <= sig[-2]
    assert sig[0] > sig[len(sig) // 2] > sig[-1]     # sigma_E falls with beta (Fig. S12)


# ---------------------------------------------------------------- pilot histograms
def test_pilot_histogram_totals_and_limits(orc):
    dims = (4, 4, 4)
    J = W.ea_couplings(dims, 3, 0)
    betas = W.geometric_ladder(4)
    c = orc.pilot_hist(dims, J, betas, chains_per_beta=4, sweeps=40, burn=10)
    assert (c.sum(1) == 4 * 30).all()
    zero = np.zeros((64, 3), np.int8)
    # free spins in a unit field at beta = 20 align: E = -N -> bin floor(64*2/3) = 42
    c = orc.pilot_hist(dims, zero, np.array([20.0]), chains_per_beta=4, sweeps=20, burn=10,
                       h=np.ones(64, np.int8))
    assert c[0, 42] == 4 * 10
    zero = np.zeros((64, 3), np.int8)
    c = orc.pilot_hist(dims, zero, np.array([1.0]), chains_per_beta=2, sweeps=5, burn=0)
    assert c[0, 63] == 10             # E = 0 -> last bin


def test_odd_open_lattice_equals_padded_lattice_with_vacancies(orc):
    """An odd open length (the paper's 15 x 15 x 12 is open in x, y) padded
    with a vacant end layer has the same energy function as the odd
    lattice itself."""
    rng = np.random.default_rng(9)
    for dims, per in (((5, 7, 4), (0, 0, 1)), ((3, 3, 3), (0, 0, 0)), ((15, 15, 12), (0, 0, 1))):
        J = W.ea_couplings(dims, 64, 0)
        pd, present, Jp = W.pad_odd_open(dims, per, J)
        for _ in range(3):
            s = rng.choice(np.array([-1, 1], np.int8), size=int(np.prod(dims)))
            sp = rng.choice(np.array([-1, 1], np.int8), size=int(np.prod(pd)))
            sp.reshape(pd[2], pd[1], pd[0])[: dims[2], : dims[1], : dims[0]] = s.reshape(dims[2], dims[1], dims[0])
            assert orc.energy(dims, J, s, periodic=per) == orc.energy(pd, Jp, sp, periodic=per, present=present)
    with pytest.raises(ValueError):
        W.pad_odd_open((5, 4, 4), (1, 1, 1), W.ea_couplings((5, 4, 4), 1, 0))
