"""Pins for the oracle's general-graph path (DSATUR colouring, graph-coloured
Gibbs sweeps, APT with ICM on graphs, DT-SQA on the replicated network).

Each test checks the oracle against something other than itself: colourings
worked by hand, brute-force chromatic numbers, the colouring theorems for
bipartite graphs, cycles, wheels and complete graphs, the lattice oracle's
energy, networkx components, and exact Boltzmann distributions by
enumeration.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

from paper_2503_10302_gb300 import workloads as W
from tests import _exact as X

nx = pytest.importorskip("networkx")


def _graph(n, edges, weights=None):
    return W.csr_from_edges(n, edges, weights)


def _proper(g, colour):
    return all(colour[v] != colour[g.col[q]] for v in range(g.n) for q in range(g.rp[v], g.rp[v + 1]))


def _chromatic_number(g):
    """Smallest k with a proper k-colouring, by backtracking (tiny graphs)."""
    n = g.n
    nbrs = [list(g.col[g.rp[v]:g.rp[v + 1]]) for v in range(n)]
    for k in range(1, n + 1):
        col = [-1] * n

        def bt(v):
            if v == n:
                return True
            for c in range(k):
                if all(col[u] != c for u in nbrs[v]):
                    col[v] = c
                    if bt(v + 1):
                        return True
            col[v] = -1
            return False
        if bt(0):
            return k
    return n


def _cycle(n):
    return _graph(n, [(i, (i + 1) % n) for i in range(n)])


def _wheel(rim):
    return _graph(rim + 1, [(i, (i + 1) % rim) for i in range(rim)] + [(rim, i) for i in range(rim)])


# ---------------------------------------------------------------- DSATUR
def test_dsatur_hand_worked_examples(orc):
    """Colourings traced by hand with the rule: largest saturation, then the
    largest degree among uncoloured vertices, then the smallest index; the
    smallest free colour."""
    # path 0-1-2: vertex 1 first (degree 2), then 0, then 2
    c, C = orc.dsatur(*(lambda g: (g.rp, g.col))(_graph(3, [(0, 1), (1, 2)])))
    assert list(c) == [1, 0, 1] and C == 2
    # 5-cycle: 0 -> 0, 1 -> 1, 2 -> 0, 3 -> 1, 4 -> 2
    g = _cycle(5)
    c, C = orc.dsatur(g.rp, g.col)
    assert list(c) == [0, 1, 0, 1, 2] and C == 3
    # star with centre 3: centre first, leaves share colour 1
    g = _graph(5, [(3, 0), (3, 1), (3, 2), (3, 4)])
    c, C = orc.dsatur(g.rp, g.col)
    assert list(c) == [1, 1, 1, 0, 1] and C == 2
    # isolated vertices all take colour 0
    g = _graph(4, [])
    c, C = orc.dsatur(g.rp, g.col)
    assert list(c) == [0, 0, 0, 0] and C == 1


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 8, 9, 10, 11])
def test_dsatur_exact_on_cycles_wheels_complete(orc, n):
    """Known chromatic numbers: C_n is 2 (even) or 3 (odd); the wheel with
    n rim vertices is 3 (even n) or 4 (odd n); K_n is n.  DSATUR is exact on
    all three families."""
    g = _cycle(n)
    c, C = orc.dsatur(g.rp, g.col)
    assert _proper(g, c) and C == (2 if n % 2 == 0 else 3)
    g = _wheel(n)
    c, C = orc.dsatur(g.rp, g.col)
    assert _proper(g, c) and C == (3 if n % 2 == 0 else 4)
    g = _graph(n, list(itertools.combinations(range(n), 2)))
    c, C = orc.dsatur(g.rp, g.col)
    assert _proper(g, c) and C == n


def test_dsatur_exact_on_bipartite_graphs(orc):
    """Brelaz (1979): DSATUR colours every bipartite graph with 2 colours.
    Random trees, random bipartite graphs and even periodic lattices."""
    rng = np.random.default_rng(5)
    for trial in range(20):
        n = int(rng.integers(2, 60))
        tree = [(v, int(rng.integers(0, v))) for v in range(1, n)]
        g = _graph(n, tree)
        c, C = orc.dsatur(g.rp, g.col)
        assert _proper(g, c) and C == 2
        a, b = int(rng.integers(1, 20)), int(rng.integers(1, 20))
        E = [(i, a + j) for i in range(a) for j in range(b) if rng.random() < 0.3]
        if E:
            g = _graph(a + b, E)
            c, C = orc.dsatur(g.rp, g.col)
            assert _proper(g, c) and C == 2
    for dims, per in [((4, 4, 4), (1, 1, 1)), ((6, 4, 2), (1, 1, 1)), ((5, 3, 4), (0, 0, 1))]:
        g, _ = W.lattice_graph(dims, per, np.ones((int(np.prod(dims)), 3), np.int8))
        c, C = orc.dsatur(g.rp, g.col)
        assert _proper(g, c) and C == 2


def test_dsatur_odd_periodic_lattice_needs_three_colours(orc):
    """An odd periodic length closes odd cycles, so 2 colours are impossible;
    DSATUR finds 3 (the Methods' remark that missing spins and embeddings
    need graph colouring)."""
    for dims in [(5, 5, 4), (3, 3, 3), (7, 4, 4)]:
        g, _ = W.lattice_graph(dims, (1, 1, 1), W.ea_couplings(dims, 1000))
        c, C = orc.dsatur(g.rp, g.col)
        assert _proper(g, c) and C == 3


def test_dsatur_valid_and_within_bounds_on_random_graphs(orc):
    """Proper, at least the chromatic number (brute force) and at most
    max degree + 1."""
    for seed in range(40):
        n = 5 + seed % 5
        g = W.random_graph(n, 1.0 + (seed % 7) * 0.6, seed, wmax=3)
        c, C = orc.dsatur(g.rp, g.col)
        deg = np.diff(g.rp)
        assert _proper(g, c)
        assert _chromatic_number(g) <= C <= int(deg.max(initial=0)) + 1
        assert set(c.tolist()) == set(range(C))


def test_dimer_embedding_needs_four_colours(orc):
    """The synthetic dimer embedding (chains of strength 2, split couplers)
    is not bipartite; like the paper's embedded instances it takes four
    colours, and a proper colouring with them exists."""
    for L in (4, 6):
        g = W.dimer_embedding((L, L, L), W.ea_couplings((L, L, L), 1000))
        c, C = orc.dsatur(g.rp, g.col)
        assert _proper(g, c) and C == 4
        assert set(np.abs(g.w).tolist()) == {1, 2}


def test_graph_check_rejects_malformed_graphs(orc):
    g = _cycle(4)
    assert orc.graph_check(g.rp, g.col, g.w)
    assert not orc.graph_check([0, 1, 1], [1], [1])                      # one direction only
    assert not orc.graph_check([0, 1, 2], [0, 1], [1, 1])                # self loops
    assert not orc.graph_check([0, 2, 4], [1, 1, 0, 0], [1, 1, 1, 1])    # repeated neighbour
    assert not orc.graph_check([0, 1, 2], [1, 0], [1, 2])                # asymmetric weights
    assert not orc.graph_check([0, 1, 2], [1, 0], [0, 0])                # zero weight


# ---------------------------------------------------------------- replicated colouring
def test_sqa_replicated_colouring_is_proper(orc):
    """Algorithm S1 colours the replicated network from one replica's
    colormap: proper on in-slice and (periodic) inter-slice edges, with
    max(C, 2) colours for even P and max(C, 3) for odd P (the paper's extra
    colour for an odd number of replicas)."""
    graphs = [_graph(1, []), _graph(2, [(0, 1)]), _cycle(5), _wheel(5),
              W.dimer_embedding((2, 2, 2), W.ea_couplings((2, 2, 2), 1000))]
    for g in graphs:
        base, C = orc.dsatur(g.rp, g.col)
        for P in range(2, 10):
            cols, Cp = orc.graph_sqa_colouring(base, P)
            assert Cp == max(C, 3 if P % 2 else 2)
            assert cols.min() >= 0 and cols.max() < Cp
            for k in range(P):
                assert _proper(g, cols[k])
                assert np.all(cols[k] != cols[(k + 1) % P])


# ---------------------------------------------------------------- energy
@pytest.mark.parametrize("dims,per", [((4, 4, 4), (1, 1, 1)), ((2, 2, 2), (1, 1, 1)),
                                      ((3, 4, 2), (0, 1, 1)), ((4, 2, 3), (1, 1, 0))])
def test_graph_energy_equals_lattice_energy(orc, dims, per):
    """The bond graph of a lattice (double bonds of length-2 periodic axes
    merged, vacancies removed) has the lattice oracle's energy."""
    N = int(np.prod(dims))
    rng = np.random.default_rng(3)
    for trial in range(5):
        J = W.ea_couplings(dims, 77, trial)
        present = None if trial < 2 else W.random_vacancies(dims, 0.25, trial)
        g, sites = W.lattice_graph(dims, per, J, present)
        s = rng.choice(np.array([-1, 1], np.int8), size=N)
        if present is not None:
            s = np.where(present > 0, s, 1).astype(np.int8)
        e_lat = orc.energy(dims, J, s, periodic=per, present=present)
        assert orc.graph_energy(g.rp, g.col, g.w, s[sites]) == e_lat


def test_graph_energy_matches_networkx_with_biases(orc):
    for seed in range(5):
        g = W.random_graph(30, 3.0, seed, wmax=5)
        h = W.random_biases(g.n, 3, seed)
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        for u, v, w in g.edges():
            G.add_edge(u, v, weight=w)
        s = np.random.default_rng(seed).choice(np.array([-1, 1], np.int8), size=g.n)
        ref = -sum(d["weight"] * int(s[u]) * int(s[v]) for u, v, d in G.edges(data=True))
        ref -= sum(int(h[v]) * int(s[v]) for v in G.nodes)
        assert orc.graph_energy(g.rp, g.col, g.w, s, h) == ref


# ---------------------------------------------------------------- sampler
def _frustrated_graph(seed=11):
    """7 vertices, odd cycles (3 colours), weights in +-{1,2,3}."""
    rng = np.random.default_rng(seed)
    E = [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 5), (5, 6), (6, 2), (1, 4), (0, 6)]
    w = rng.integers(1, 4, size=len(E)) * (2 * rng.integers(0, 2, size=len(E)) - 1)
    return _graph(7, E, w)


def _exact_graph_energies(g, h=None):
    st = X.all_states(g.n)
    E = np.zeros(st.shape[0], np.int64)
    for u, v, w in g.edges():
        E -= w * st[:, u].astype(np.int64) * st[:, v]
    if h is not None:
        E -= (st.astype(np.int64) * np.asarray(h, np.int64)[None, :]).sum(1)
    return E


def _chi2_states(k, p, what, inflate=2.0):
    counts = np.bincount(k, minlength=len(p)).astype(float)
    n = counts.sum()
    mask = p * n >= 5
    obs = np.append(counts[mask], counts[~mask].sum())
    exp = np.append(p[mask] * n, p[~mask].sum() * n)
    if exp[-1] == 0:
        obs, exp = obs[:-1], exp[:-1]
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert stats.chi2.sf(chi2 / inflate, len(obs) - 1) > 1e-6, (what, chi2, len(obs))


@pytest.mark.parametrize("beta", [0.25, 0.6])
def test_graph_gibbs_sampler_matches_enumeration(orc, beta):
    """Graph-coloured sweeps with weights and biases sample exp(-beta E)
    over all 2^7 states of a 3-colour frustrated graph."""
    g = _frustrated_graph()
    h = np.array([1, -2, 0, 1, 0, -1, 2], np.int8)
    E = _exact_graph_energies(g, h)
    p = X.boltzmann(E, beta)
    n_ch, n_sw = 48, 800
    apt = orc.GApt([(g.rp, g.col, g.w)] * n_ch, [np.array([beta])] * n_ch, n_labels=1, seed=5,
                   h_list=[h] * n_ch)
    apt.run(20, icm=False)
    ks = []
    for _ in range(n_sw):
        apt.run(1, icm=False)
        ks.append([X.state_index(apt.state(i)[0][0]) for i in range(n_ch)])
    _chi2_states(np.array(ks).ravel(), p, ("gibbs", beta))


def test_graph_parallel_tempering_stationary_per_temperature(orc):
    """Sweeps + replica exchange on a graph keep each temperature at
    exp(-beta_r E), and the swap acceptance equals its exact expectation."""
    g = _frustrated_graph(13)
    E = _exact_graph_energies(g)
    betas = np.array([0.2, 0.5, 1.1])
    n_ch, n_sw = 32, 1500
    apt = orc.GApt([(g.rp, g.col, g.w)] * n_ch, [betas] * n_ch, n_labels=1, seed=8)
    apt.run(20, icm=False)
    per_t = [[] for _ in betas]
    for _ in range(n_sw):
        apt.run(1, icm=False)
        for i in range(n_ch):
            s, _, _ = apt.state(i)
            for r in range(3):
                per_t[r].append(X.state_index(s[r]))
    for r, beta in enumerate(betas):
        pr = X.boltzmann(E, beta)
        Es = E[np.array(per_t[r])]
        m, se = X.batch_mean_stderr(Es.reshape(n_sw, n_ch).T.ravel())
        assert abs(m - (pr * E).sum()) < 5 * se, r
    att = np.zeros((2, 1)); acc = np.zeros((2, 1))
    for i in range(n_ch):
        a, c, _ = apt.stats(i)
        att += a; acc += c
    for r in range(2):
        p0, p1 = X.boltzmann(E, betas[r]), X.boltzmann(E, betas[r + 1])
        dE = E[None, :] - E[:, None]
        acc_exact = (p0[:, None] * p1[None, :] * np.minimum(1, np.exp((betas[r + 1] - betas[r]) * dE))).sum()
        rate = acc[r, 0] / att[r, 0]
        assert abs(rate - acc_exact) < 10 * math.sqrt(acc_exact * (1 - acc_exact) / att[r, 0])


# ---------------------------------------------------------------- ICM
def test_graph_icm_moves_a_connected_component(orc):
    """The flipped set is the networkx connected component, in the mismatch
    subgraph, of a mismatch vertex; E_a + E_b is conserved (h = 0); a
    cluster of more than n/2 vertices flips one whole replica instead."""
    rng = np.random.default_rng(21)
    seen = {1: 0, 2: 0}
    for trial in range(60):
        g = W.random_graph(40, 2.5, trial, wmax=2)
        colour, _ = orc.dsatur(g.rp, g.col)
        sa = rng.choice(np.array([-1, 1], np.int8), size=g.n)
        sb = np.where(rng.random(g.n) < 0.3 + 0.4 * (trial % 2), -sa, sa).astype(np.int8)
        br, size, a2, b2 = orc.gicm_apply(g.rp, g.col, colour, sa, sb, seed=3, entry=trial, r=1, t=trial)
        mism = np.flatnonzero(sa != sb)
        if len(mism) == 0:
            assert br == 0
            continue
        G = nx.Graph()
        G.add_nodes_from(mism.tolist())
        G.add_edges_from((u, v) for u, v, _ in g.edges() if sa[u] != sb[u] and sa[v] != sb[v])
        Ea = orc.graph_energy(g.rp, g.col, g.w, sa) + orc.graph_energy(g.rp, g.col, g.w, sb)
        Eb = orc.graph_energy(g.rp, g.col, g.w, a2) + orc.graph_energy(g.rp, g.col, g.w, b2)
        assert Ea == Eb
        seen[br] += 1
        if br == 1:
            flipped = np.flatnonzero(a2 != sa)
            assert np.array_equal(flipped, np.flatnonzero(b2 != sb))
            comp = nx.node_connected_component(G, int(flipped[0]))
            assert sorted(comp) == flipped.tolist() and size == len(comp) and 2 * size <= g.n
        else:
            assert 2 * size > g.n
            assert (np.array_equal(a2, -sa) and np.array_equal(b2, sb)) or \
                   (np.array_equal(b2, -sb) and np.array_equal(a2, sa))
    assert seen[1] > 5 and seen[2] > 2


def test_graph_icm_seed_is_uniform_over_mismatch_vertices(orc):
    """With an edgeless mismatch set every cluster is one vertex, so the
    flipped vertex is the seed: uniform over the mismatch vertices."""
    g = _cycle(24)
    colour, _ = orc.dsatur(g.rp, g.col)
    sa = np.ones(24, np.int8)
    sb = sa.copy()
    mism = [0, 2, 5, 9, 12, 17, 20]          # no two adjacent on the cycle
    sb[mism] = -1
    counts = np.zeros(24)
    for t in range(7000):
        br, size, a2, _ = orc.gicm_apply(g.rp, g.col, colour, sa, sb, seed=1, entry=0, r=0, t=t)
        assert br == 1 and size == 1
        counts[np.flatnonzero(a2 != sa)[0]] += 1
    assert counts[mism].sum() == 7000
    assert stats.chisquare(counts[mism]).pvalue > 1e-6


@pytest.mark.parametrize("labels", [2, 4])
def test_graph_icm_keeps_product_boltzmann(orc, labels):
    """Sweeps + ICM at one temperature: every label's marginal stays
    exp(-beta E), with 2 labels and with 4 labels in random pairs."""
    g = _frustrated_graph(17)
    E = _exact_graph_energies(g)
    beta = 0.8
    p = X.boltzmann(E, beta)
    n_ch, n_sw = 32, 1000
    apt = orc.GApt([(g.rp, g.col, g.w)] * n_ch, [np.array([beta])] * n_ch, n_labels=labels, seed=4)
    apt.run(10, icm=True)
    ks = [[] for _ in range(labels)]
    for _ in range(n_sw):
        apt.run(1, icm=True)
        for i in range(n_ch):
            s, _, _ = apt.state(i)
            for a in range(labels):
                ks[a].append(X.state_index(s[a]))
    _, _, icm = apt.stats(0)
    assert icm[1] + icm[2] > 0
    for a in range(labels):
        _chi2_states(np.array(ks[a]), p, ("icm", labels, a), inflate=3.0)


# ---------------------------------------------------------------- APT bookkeeping
def test_graph_apt_energies_best_and_resume(orc):
    g = W.random_graph(60, 3.0, 2, wmax=2)
    betas = W.geometric_ladder(6, 0.3, 2.5)
    a1 = orc.GApt([(g.rp, g.col, g.w)] * 2, [betas] * 2, n_labels=2, seed=12)
    a1.run(30, icm=True)
    a2 = orc.GApt([(g.rp, g.col, g.w)] * 2, [betas] * 2, n_labels=2, seed=12)
    a2.run(12, icm=True, threads=1)
    a2.run(18, icm=True, threads=2)
    for i in range(2):
        s1, E1, c1 = a1.state(i)
        s2, E2, _ = a2.state(i)
        assert np.array_equal(s1, s2) and np.array_equal(E1, E2)
        assert _proper(g, c1)
        for b in range(len(E1)):
            assert E1[b] == orc.graph_energy(g.rp, g.col, g.w, s1[b])
        best = a1.best(i)
        assert best["E"] <= E1.min()
        assert best["E"] == orc.graph_energy(g.rp, g.col, g.w, best["spins"])


def test_graph_apt_refuses_icm_with_biases(orc):
    g = _cycle(6)
    apt = orc.GApt([(g.rp, g.col, g.w)], [np.array([0.5, 1.0])], n_labels=2,
                   h_list=[np.array([1, 0, 0, 0, 0, 0], np.int8)])
    with pytest.raises(ValueError):
        apt.run(1, icm=True)
    apt.run(1, icm=False)


# ---------------------------------------------------------------- DT-SQA on graphs
@pytest.mark.parametrize("P,gamma", [(3, 0.4), (2, 0.8), (4, 0.3)])
def test_graph_sqa_matches_enumeration(orc, P, gamma):
    """Triangle with weights and biases, P slices (P = 3 needs the extra
    colour): the joint distribution of all 3P spins is exp(-H_C/(P T)) with
    H_C of Eq. S.3 scaled by P, exact by enumeration."""
    g = _graph(3, [(0, 1), (1, 2), (2, 0)], [1, -2, 1])
    h = np.array([1, 0, -1], np.int8)
    n, T = 3, 0.4
    jq = orc.jperp_q(gamma, P, T)
    st = X.all_states(n * P).reshape(-1, P, n).astype(np.float64)
    Hc = np.zeros(st.shape[0])
    for k in range(P):
        for u, v, w in g.edges():
            Hc -= w * st[:, k, u] * st[:, k, v]
        Hc -= (st[:, k, :] * h[None, :]).sum(1)
        if P > 2 or k == 0:
            # with P = 2 slices k-1 and k+1 are the same slice: two bonds
            Hc -= (jq / 65536) * (st[:, k, :] * st[:, (k + 1) % P, :]).sum(1) * (2 if P == 2 else 1)
    p = np.exp(-(Hc - Hc.min()) / (P * T))
    p /= p.sum()
    R = 4000
    _, s = orc.gsqa_anneal(g.rp, g.col, g.w, P, T, np.full(400, gamma), R, seed=9, h=h, want_spins=True)
    k = X.state_index(s.reshape(R, P * n))
    levels, inv = np.unique(np.round(Hc, 9), return_inverse=True)
    pl = np.bincount(inv, weights=p)
    ol = np.bincount(inv, weights=np.bincount(k, minlength=p.size).astype(float))
    mask = pl * R >= 5
    obs = np.append(ol[mask], ol[~mask].sum())
    exp = np.append(pl[mask] * R, pl[~mask].sum() * R)
    if exp[-1] == 0:
        obs, exp = obs[:-1], exp[:-1]
    assert stats.chisquare(obs, exp).pvalue > 1e-6


def test_graph_sqa_energies_are_slice_energies(orc):
    g = W.dimer_embedding((2, 2, 2), W.ea_couplings((2, 2, 2), 1000))
    h = W.random_biases(g.n, 1, 4)
    E, s = orc.gsqa_anneal(g.rp, g.col, g.w, 5, 0.2, W.linear_gamma_schedule(30), 3, seed=2, h=h,
                           want_spins=True)
    for r in range(3):
        for k in range(5):
            assert E[r, k] == orc.graph_energy(g.rp, g.col, g.w, s[r, k], h)


# ---------------------------------------------------------------- adaptive ladder on graphs
def test_graph_adaptive_ladder_first_step_matches_enumeration(orc):
    """sigma_E at beta_0 equals the standard deviation of E under the exact
    Boltzmann law of a 7-vertex frustrated graph with weights and biases, and
    beta_1 = beta_0 + alpha / sigma_E (Algorithm S2 preprocessing)."""
    g = _frustrated_graph(23)
    h = np.array([1, 0, -1, 0, 2, 0, -1], np.int8)
    E = _exact_graph_energies(g, h).astype(np.float64)
    b0 = 0.4
    p = X.boltzmann(E.astype(np.int64), b0)
    sd = math.sqrt((p * E ** 2).sum() - (p * E).sum() ** 2)
    beta, sig, ok = orc.graph_adaptive_ladder(g.rp, g.col, g.w, h=h, beta0=b0, alpha=1.25, n_chains=128,
                                              sweeps=700, tail=600, tol=0.1, max_len=2)
    assert abs(sig[0] - sd) < 0.04 * sd, (sig[0], sd)
    assert beta[1] == pytest.approx(b0 + 1.25 / sig[0], rel=1e-12)


def test_graph_adaptive_ladder_stop_rules(orc):
    g0 = _graph(9, [])
    beta, sig, ok = orc.graph_adaptive_ladder(g0.rp, g0.col, g0.w, n_chains=8, sweeps=20, tail=10)
    assert ok and len(beta) == 1 and sig[0] == 0.0
    g = W.dimer_embedding((4, 4, 4), W.ea_couplings((4, 4, 4), 1000, 6))
    beta, sig, ok = orc.graph_adaptive_ladder(g.rp, g.col, g.w, n_chains=8, sweeps=40, tail=20, max_len=3)
    assert not ok and len(beta) == 3
    beta, sig, ok = orc.graph_adaptive_ladder(g.rp, g.col, g.w, n_chains=32, sweeps=300, tail=200, max_len=64)
    assert ok and np.all(np.diff(beta) > 0) and sig[-1] < 1.0 <= sig[-2]
