"""APT + ICM and DT-SQA on general sparse graphs, GPU against the CPU oracle:
bit-exact spins, energies, best energies and states, hit sweeps, swap and
ICM statistics, for DSATUR-coloured graphs with 1 to 4 colours (odd periodic
lattices, dimer embeddings with couplings of strength 2, random weighted
graphs with biases) and odd and even numbers of Trotter slices."""
import numpy as np
import pytest

from paper_2503_10302_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    from paper_2503_10302_gb300 import build, pcomp
    build.build()
    return pcomp


def _trip(g):
    return (g.rp, g.col, g.w)


def _compare(pc, ctx, o, graphs, betas, A):
    for i, g in enumerate(graphs):
        T = len(betas[i])
        E1 = pc.pc_gapt_get_energies(ctx.h, i, T, A)
        s1 = pc.pc_gapt_get_spins(ctx.h, i, T, A, g.n)
        s2, E2, c2 = o.state(i)
        assert np.array_equal(pc.pc_gapt_get_colours(ctx.h, i, g.n), c2), ("colours", i)
        assert np.array_equal(E1, E2), ("energies", i, E1, E2)
        assert np.array_equal(s1, s2), ("spins", i)
        b1, b2 = pc.pc_gapt_get_best(ctx.h, i, g.n), o.best(i)
        for key in ("E", "sweep", "buf", "hit_sweep"):
            assert b1[key] == b2[key], (key, i, b1[key], b2[key])
        if b2["sweep"] >= 0:
            assert np.array_equal(b1["spins"], b2["spins"]), ("best spins", i)
        att, acc, icm = pc.pc_gapt_get_stats(ctx.h, i, T, A)
        att2, acc2, icm2 = o.stats(i)
        assert np.array_equal(att, att2) and np.array_equal(acc, acc2), ("swap stats", i)
        assert np.array_equal(icm, icm2), ("icm stats", i, icm, icm2)


def _mixed_graphs():
    """Several tiles of work per colour and ragged tails: graphs whose colour
    classes are not multiples of 8 vertices."""
    return [W.lattice_graph((5, 5, 4), (1, 1, 1), W.ea_couplings((5, 5, 4), 1000, 0))[0],
            W.dimer_embedding((4, 4, 4), W.ea_couplings((4, 4, 4), 1000, 1)),
            W.random_graph(333, 4.0, 7, wmax=3),
            W.lattice_graph((6, 6, 6), (0, 1, 1), W.ea_couplings((6, 6, 6), 1000, 2),
                            W.random_vacancies((6, 6, 6), 0.15, 5))[0]]


@pytest.mark.parametrize("A,icm,spp", [(2, True, 1), (4, True, 1), (1, False, 1), (2, False, 3),
                                       (2, True, 2)])
def test_gapt_matches_oracle(pc, orc, A, icm, spp):
    graphs = _mixed_graphs()
    betas = [W.geometric_ladder(T, 0.2, 3.0) for T in (32, 17, 24, 9)]
    seed = 1234 + A
    ctx = pc.Context(0, seed)
    pc.pc_gapt_load(ctx.h, [_trip(g) for g in graphs], betas, A, 5)
    o = orc.GApt([_trip(g) for g in graphs], betas, n_labels=A, seed=seed, entry0=5)
    _compare(pc, ctx, o, graphs, betas, A)          # initial states and energies
    for i, g in enumerate(graphs):
        o.set_target(i, -int(1.2 * g.n))
        pc.pc_gapt_set_target(ctx.h, i, -int(1.2 * g.n))
    for n_sw in (1, 7, 40):
        pc.pc_gapt_run(ctx.h, n_sw, spp, icm)
        o.run(n_sw, spp, icm)
        _compare(pc, ctx, o, graphs, betas, A)
    ctx.close()


def test_gapt_with_biases_and_joint_swaps(pc, orc):
    graphs = [W.random_graph(200, 5.0, 11, wmax=4), W.random_graph(77, 2.0, 12, wmax=2)]
    hs = [W.random_biases(g.n, 3, 20 + i) for i, g in enumerate(graphs)]
    betas = [W.geometric_ladder(20, 0.1, 2.0), W.geometric_ladder(31, 0.3, 4.0)]
    ctx = pc.Context(0, 99)
    pc.pc_gapt_load(ctx.h, [_trip(g) for g in graphs], betas, 2, 0, h_list=hs)
    o = orc.GApt([_trip(g) for g in graphs], betas, n_labels=2, seed=99, h_list=hs)
    pc.pc_gapt_set_joint_swap(ctx.h, True)
    o.set_joint_swap(True)
    pc.pc_gapt_run(ctx.h, 30, 1, False)
    o.run(30, 1, False)
    _compare(pc, ctx, o, graphs, betas, 2)
    pc.pc_gapt_set_joint_swap(ctx.h, False)
    o.set_joint_swap(False)
    pc.pc_gapt_run(ctx.h, 20, 2, False)
    o.run(20, 2, False)
    _compare(pc, ctx, o, graphs, betas, 2)
    with pytest.raises(RuntimeError):
        pc.pc_gapt_run(ctx.h, 1, 1, True)           # ICM refuses biases
    ctx.close()


def test_gapt_given_colormap_and_edge_cases(pc, orc):
    """A caller's colormap (here 4 colours on a bipartite graph), a graph
    without edges (1 colour) and one temperature."""
    g1 = W.lattice_graph((4, 4, 4), (1, 1, 1), W.ea_couplings((4, 4, 4), 1000, 3))[0]
    lin = np.arange(64)
    col1 = (((lin % 4) + (lin // 4) % 4 + lin // 16) % 2 + 2 * (lin % 3 == 0)).astype(np.int32)
    g2 = W.csr_from_edges(13, [])
    graphs, colours = [g1, g2], [col1, None]
    betas = [W.geometric_ladder(8, 0.2, 3.0), np.array([0.7])]
    ctx = pc.Context(0, 3)
    cl = [col1, orc.dsatur(g2.rp, g2.col)[0]]
    pc.pc_gapt_load(ctx.h, [_trip(g) for g in graphs], betas, 2, 0, colours=cl)
    o = orc.GApt([_trip(g) for g in graphs], betas, n_labels=2, seed=3, colours=cl)
    for _ in range(3):
        pc.pc_gapt_run(ctx.h, 9, 1, True)
        o.run(9, 1, True)
        _compare(pc, ctx, o, graphs, betas, 2)
    ctx.close()


def test_gapt_refuses_bad_input(pc):
    ctx = pc.Context(0, 0)
    g = W.csr_from_edges(4, [(0, 1), (1, 2), (2, 3), (3, 0)])
    bad_colour = [np.zeros(4, np.int32)]
    with pytest.raises(RuntimeError):
        pc.pc_gapt_load(ctx.h, [_trip(g)], [np.array([0.5, 1.0])], 2, 0, colours=bad_colour)
    with pytest.raises(RuntimeError):
        pc.pc_gapt_load(ctx.h, [_trip(g)], [np.array([1.0, 0.5])], 2)    # not increasing
    with pytest.raises(RuntimeError):
        pc.pc_gapt_load(ctx.h, [_trip(g)], [np.linspace(0.1, 1, 33)], 2)  # 33 temperatures
    heavy = W.csr_from_edges(3, [(0, 1), (1, 2)], [100, 100])
    with pytest.raises(RuntimeError):
        pc.pc_gapt_load(ctx.h, [_trip(heavy)], [np.array([0.5])], 1)    # |field| > 127
    ctx.close()


@pytest.mark.parametrize("P", [2, 3, 4, 5, 8])
def test_gsqa_matches_oracle(pc, orc, P):
    cases = [(W.dimer_embedding((2, 2, 2), W.ea_couplings((2, 2, 2), 1000, 4)), None),
             (W.random_graph(70, 3.0, 8, wmax=3), W.random_biases(70, 2, 8)),
             (W.lattice_graph((3, 3, 4), (1, 1, 1), W.ea_couplings((3, 3, 4), 1000, 5))[0], None)]
    gamma = W.linear_gamma_schedule(37, 3.0, 0.05)
    for gi, (g, h) in enumerate(cases):
        R = 45
        ctx = pc.Context(0, 17 + gi)
        E1, s1 = pc.pc_gsqa_anneal(ctx.h, g.rp, g.col, g.w, P, 0.3, gamma, R, run0=16, h=h, want_spins=True)
        E2, s2 = orc.gsqa_anneal(g.rp, g.col, g.w, P, 0.3, gamma, R, run0=16, seed=17 + gi, h=h,
                                 want_spins=True)
        assert np.array_equal(s1, s2), (P, gi)
        assert np.array_equal(E1, E2), (P, gi)
        ctx.close()


def test_gsqa_refuses_unaligned_run_ids(pc):
    g = W.random_graph(20, 2.0, 1)
    ctx = pc.Context(0, 1)
    with pytest.raises(RuntimeError):
        pc.pc_gsqa_anneal(ctx.h, g.rp, g.col, g.w, 4, 0.5, np.full(3, 1.0), 8, run0=3)
    ctx.close()


def test_gsqa_heavy_weights_take_the_wide_planes(pc, orc):
    """Field bounds above 7 take 7 bit planes and an unreplicated table."""
    g = W.random_graph(50, 3.0, 21, wmax=9)
    gamma = W.linear_gamma_schedule(25, 3.0, 0.1)
    ctx = pc.Context(0, 9)
    E1, s1 = pc.pc_gsqa_anneal(ctx.h, g.rp, g.col, g.w, 6, 0.4, gamma, 40, run0=8, want_spins=True)
    E2, s2 = orc.gsqa_anneal(g.rp, g.col, g.w, 6, 0.4, gamma, 40, run0=8, seed=9, want_spins=True)
    assert np.array_equal(s1, s2) and np.array_equal(E1, E2)
    ctx.close()


@pytest.mark.parametrize("case", ["dimer_P512", "random_odd_P203", "dimer_15x15x24_P16"])
def test_gsqa_cluster_split_matches_oracle(pc, orc, case):
    """Anneals too large for one CTA: the slices of a run group are split over
    a cluster of 2 (dimer embedding, P = 512), 8 (1000-vertex graph with heavy
    weights, odd P = 203) or 4 CTAs (10800-p-bit embedding whose graph is read
    from global memory), boundary slices read through distributed shared
    memory."""
    if case == "dimer_P512":
        g, P, sw, h = W.dimer_embedding((4, 4, 4), W.ea_couplings((4, 4, 4), 1000, 12)), 512, 12, None
    elif case == "dimer_15x15x24_P16":
        # 10800 p-bits: the graph itself stays in global memory (read through L1)
        d = (15, 15, 24)
        g, P, sw, h = W.dimer_embedding(d, W.ea_couplings(d, 1000, 13)), 16, 3, None
    else:
        g, P, sw = W.sparse_random_graph(1000, 4.0, 5, wmax=6), 203, 8
        h = W.random_biases(g.n, 2, 5)
    gamma = W.linear_gamma_schedule(sw, 2.0, 0.2)
    R = 40
    ctx = pc.Context(0, 31)
    E1, s1 = pc.pc_gsqa_anneal(ctx.h, g.rp, g.col, g.w, P, 0.2, gamma, R, run0=24, h=h, want_spins=True)
    E2, s2 = orc.gsqa_anneal(g.rp, g.col, g.w, P, 0.2, gamma, R, run0=24, seed=31, h=h, want_spins=True)
    assert np.array_equal(s1, s2) and np.array_equal(E1, E2)
    ctx.close()


def test_gsqa_zero_sweeps_is_the_initial_state(pc, orc):
    g = W.random_graph(40, 2.0, 3)
    ctx = pc.Context(0, 5)
    E1, s1 = pc.pc_gsqa_anneal(ctx.h, g.rp, g.col, g.w, 3, 0.5, np.zeros(0), 33, want_spins=True)
    E2, s2 = orc.gsqa_anneal(g.rp, g.col, g.w, 3, 0.5, np.zeros(0), 33, seed=5, want_spins=True)
    assert np.array_equal(s1, s2) and np.array_equal(E1, E2)
    ctx.close()


def test_gapt_large_graph_reads_adjacency_from_global_memory(pc, orc):
    """A graph whose vertex table and adjacency do not fit in shared memory
    next to its 4 labels of spin words: the kernel reads them through the L1
    cache instead (the same results)."""
    g = W.sparse_random_graph(7000, 6.0, 2, wmax=2)
    betas = [W.geometric_ladder(32, 0.2, 3.0)]
    ctx = pc.Context(0, 41)
    pc.pc_gapt_load(ctx.h, [_trip(g)], betas, 4, 0)
    o = orc.GApt([_trip(g)], betas, n_labels=4, seed=41)
    for n_sw in (2, 6):
        pc.pc_gapt_run(ctx.h, n_sw, 1, True)
        o.run(n_sw, 1, True)
        _compare(pc, ctx, o, [g], betas, 4)
    ctx.close()



@pytest.mark.parametrize("n_chains", [24, 40, 100])
def test_graph_adaptive_ladder_matches_oracle(pc, orc, n_chains):
    """Identical betas and sigmas: the chains' post-sweep energy sums are
    exact integers on both sides and sigma_E follows the same formula."""
    graphs = [W.dimer_embedding((2, 2, 2), W.ea_couplings((2, 2, 2), 1000, 8)),
              W.random_graph(90, 3.0, 9, wmax=2),
              W.lattice_graph((3, 3, 4), (1, 1, 1), W.ea_couplings((3, 3, 4), 1000, 9))[0]]
    hs = [np.zeros(graphs[0].n, np.int8), W.random_biases(graphs[1].n, 2, 9), np.zeros(graphs[2].n, np.int8)]
    ctx = pc.Context(0, 77)
    out = pc.pc_graph_adaptive_ladder(ctx.h, [_trip(g) for g in graphs], entry0=3, n_chains=n_chains,
                                      sweeps=120, tail=60, max_len=6, h_list=hs)
    for i, g in enumerate(graphs):
        b2, s2, ok2 = orc.graph_adaptive_ladder(g.rp, g.col, g.w, h=hs[i], entry=3 + i, seed=77,
                                                n_chains=n_chains, sweeps=120, tail=60, max_len=6)
        b1, s1, ok1 = out[i]
        assert ok1 == ok2 and np.array_equal(b1, b2) and np.array_equal(s1, s2), (i, b1, b2)
    ctx.close()


def test_gapt_fuzz_shapes(pc, orc):
    """Random shapes against the oracle: isolated vertices, a star with a hub
    of degree 120, heavy weights (field bounds up to 127), biases, 1 to 32
    temperatures and every label count."""
    rng = np.random.default_rng(123)
    for trial in range(12):
        A = [1, 2, 4][trial % 3]
        kind = trial % 4
        if kind == 0:
            g = W.csr_from_edges(1 + trial, [])
        elif kind == 1:
            leaves = 120
            g = W.csr_from_edges(leaves + 1, [(0, i) for i in range(1, leaves + 1)])
        elif kind == 2:
            g = W.random_graph(int(rng.integers(20, 700)), float(rng.uniform(1, 8)), 300 + trial, wmax=2)
        else:
            g = W.random_graph(40, 3.0, 400 + trial, wmax=25)
        deg = np.diff(g.rp)
        bound = np.array([np.abs(g.w[g.rp[v]:g.rp[v + 1]]).sum() for v in range(g.n)])
        hmax = int(max(0, min(5, 127 - bound.max())))
        h = W.random_biases(g.n, hmax, trial) if (trial % 2 and hmax) else None
        T = int(rng.integers(1, 33))
        betas = [np.sort(rng.uniform(0.05, 2.5, T)) + np.arange(T) * 1e-3]
        icm = A >= 2 and h is None
        ctx = pc.Context(0, 500 + trial)
        pc.pc_gapt_load(ctx.h, [_trip(g)], betas, A, trial, h_list=None if h is None else [h])
        o = orc.GApt([_trip(g)], betas, n_labels=A, seed=500 + trial, entry0=trial,
                     h_list=None if h is None else [h])
        pc.pc_gapt_run(ctx.h, 5, 1 + trial % 2, icm)
        o.run(5, 1 + trial % 2, icm)
        _compare(pc, ctx, o, [g], betas, A)
        ctx.close()
        assert deg.max(initial=0) <= 200
