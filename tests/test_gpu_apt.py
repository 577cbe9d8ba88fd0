"""Adaptive parallel tempering + ICM, the adaptive ladder and the pilot
histograms on the GPU against the CPU oracle: bit-exact spins, energies,
temperature assignments, swap/ICM statistics, best energies and hit sweeps."""
import numpy as np
import pytest

from paper_2503_10302_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    from paper_2503_10302_gb300 import build, pcomp
    build.build()
    return pcomp


def _compare(pc, orc_apt, ctx, batch, insts=None, entry0=0):
    """GPU problem i vs oracle problem i - entry0 offset mapping."""
    insts = [(i, i) for i in range(batch.n)] if insts is None else insts
    for gi, oi in insts:
        N = int(np.prod(batch.dims[gi]))
        T = len(batch.betas[gi])
        B = T * batch.n_labels
        s, E, t = pc.pc_apt_get_state(ctx.h, gi, N, B)
        s2, E2, t2 = orc_apt.state(oi)
        assert np.array_equal(t, t2), ("temps", gi)
        assert np.array_equal(E, E2), ("energies", gi)
        assert np.array_equal(s, s2), ("spins", gi)
        b1 = pc.pc_apt_get_best(ctx.h, gi, N)
        b2 = orc_apt.best(oi)
        for key in ("E", "sweep", "buf", "hit_sweep"):
            assert b1[key] == b2[key], (key, gi, b1[key], b2[key])
        if b2["sweep"] >= 0:
            assert np.array_equal(b1["spins"], b2["spins"]), ("best spins", gi)
        att, acc, icm = pc.pc_apt_get_stats(ctx.h, gi, T, batch.n_labels)
        att2, acc2, icm2 = orc_apt.stats(oi)
        assert np.array_equal(att, att2) and np.array_equal(acc, acc2), ("swap stats", gi)
        assert np.array_equal(icm, icm2), ("icm stats", gi, icm, icm2)


def test_tables_equal_oracle(pc, orc):
    b = W.apt_uniform_batch(2, 4, 12)
    b.betas[1] = W.geometric_ladder(12, 0.1, 5.0)
    ctx = pc.Context(0, 0)
    pc.pc_apt_load(ctx.h, b.dims, b.J, b.betas, 2, 0)
    for i in range(2):
        tab = pc.pc_apt_get_pbit_table(ctx.h, i, 12)
        for t, beta in enumerate(b.betas[i]):
            assert [int(v) for v in tab[t]] == [orc.pbit_threshold(beta, 2 * c - 6) for c in range(7)]
        for r in range(11):
            sw = pc.pc_apt_get_swap_table(ctx.h, i, r)
            db = b.betas[i][r + 1] - b.betas[i][r]
            # entry k: dE = -2k; the table ends where the threshold reaches 0
            # or at |dE| = 6N, the largest gap two states can have
            ref = [orc.swap_threshold(db, -2 * k) for k in range(1, len(sw) + 1)]
            assert sw[0] == 0xFFFFFFFF and list(sw[1:]) == ref[:-1]
            assert ref[-1] == 0 or len(sw) == 3 * 64 + 1
    ctx.close()


def test_initial_state_equals_oracle(pc, orc):
    b = W.apt_uniform_batch(3, 6, 9)
    ctx = pc.Context(0, 11)
    pc.pc_apt_load(ctx.h, b.dims, b.J, b.betas, 2, 5)
    apt = orc.Apt(b.dims, b.J, b.betas, 2, seed=11, entry0=5)
    _compare(pc, apt, ctx, b, [(i, i) for i in range(3)])
    ctx.close()


def test_c1_full_run_bit_exact(pc, orc):
    """One L = 4 instance, 8 temperatures x 2 replicas, swap + ICM every
    sweep, 1e4 sweeps; compared after 100 and after 10000 sweeps."""
    b = W.apt_single(L=4, n_temps=8)
    ctx = pc.Context(0, 0)
    pc.pc_apt_load(ctx.h, b.dims, b.J, b.betas, 2, 0)
    apt = orc.Apt(b.dims, b.J, b.betas, 2, seed=0)
    pc.pc_apt_run(ctx.h, 100, 1, True)
    apt.run(100)
    _compare(pc, apt, ctx, b, [(0, 0)])
    pc.pc_apt_run(ctx.h, 9900, 1, True)
    apt.run(9900)
    _compare(pc, apt, ctx, b, [(0, 0)])
    assert pc.pc_apt_progress(ctx.h) == (10000, 10000)
    ctx.close()


@pytest.mark.parametrize("spp,icm,labels", [(1, False, 2), (3, True, 2), (2, False, 1), (1, True, 4),
                                            (2, False, 4)])
def test_apt_variants(pc, orc, spp, icm, labels):
    b = W.apt_uniform_batch(2, 6, 7, n_labels=labels)
    ctx = pc.Context(0, 3)
    pc.pc_apt_load(ctx.h, b.dims, b.J, b.betas, labels, 0)
    apt = orc.Apt(b.dims, b.J, b.betas, labels, seed=3)
    pc.pc_apt_run(ctx.h, 150, spp, icm)
    apt.run(150, spp, icm)
    _compare(pc, apt, ctx, b, [(0, 0), (1, 1)])
    ctx.close()


def test_mixed_shapes_batch(pc, orc):
    """Uneven shapes and ladder lengths in one launch, incl. the largest
    supported problem (16^3 spins x 64 replicas)."""
    shapes = [(4, 4, 4), (6, 6, 6), (8, 8, 8), (4, 6, 8), (2, 4, 6), (10, 10, 10), (16, 16, 16)]
    temps = [5, 9, 16, 11, 3, 24, 32]
    dims = np.array(shapes, np.int32)
    J = [W.ea_couplings(s, 7, i) for i, s in enumerate(shapes)]
    betas = [W.geometric_ladder(t) for t in temps]
    b = W.AptBatch(dims, J, betas, 2)
    ctx = pc.Context(0, 21)
    pc.pc_apt_load(ctx.h, dims, J, betas, 2, 100)
    apt = orc.Apt(dims, J, betas, 2, seed=21, entry0=100)
    pc.pc_apt_run(ctx.h, 30, 1, True)
    apt.run(30, threads=8)
    _compare(pc, apt, ctx, b, [(i, i) for i in range(len(shapes))])
    ctx.close()


@pytest.mark.parametrize("tpb", [64, 512])
def test_elongated_and_thin_lattices_with_icm(pc, orc, tpb):
    """Long axes (Lx = 32), axes of length 2 (double bonds) and, at 64
    threads, several 2x2x2 fill blocks and chunks per thread."""
    shapes = [(32, 4, 4), (2, 2, 2), (8, 2, 4), (4, 16, 2), (16, 16, 16)]
    temps = [8, 4, 7, 12, 16]
    dims = np.array(shapes, np.int32)
    J = [W.ea_couplings(s, 8, i) for i, s in enumerate(shapes)]
    betas = [W.geometric_ladder(t) for t in temps]
    b = W.AptBatch(dims, J, betas, 2)
    ctx = pc.Context(0, 23)
    pc.pc_apt_load(ctx.h, dims, J, betas, 2, 40)
    pc.pc_apt_set_block_threads(ctx.h, tpb)
    apt = orc.Apt(dims, J, betas, 2, seed=23, entry0=40)
    pc.pc_apt_run(ctx.h, 25, 1, True)
    apt.run(25, threads=8)
    _compare(pc, apt, ctx, b, [(i, i) for i in range(len(shapes))])
    ctx.close()


def test_four_labels_sixteen_temperatures_with_icm(pc, orc):
    """The paper's four ICM labels (two random pairs per temperature) at the
    largest ladder one CTA holds (16 x 4 = 64 replicas), incl. a ragged
    ladder (11 temperatures)."""
    shapes = [(8, 8, 8), (6, 6, 6), (4, 4, 8)]
    temps = [16, 11, 9]
    dims = np.array(shapes, np.int32)
    J = [W.ea_couplings(s, 9, i) for i, s in enumerate(shapes)]
    betas = [W.geometric_ladder(t) for t in temps]
    b = W.AptBatch(dims, J, betas, 4)
    ctx = pc.Context(0, 29)
    pc.pc_apt_load(ctx.h, dims, J, betas, 4, 7)
    apt = orc.Apt(dims, J, betas, 4, seed=29, entry0=7)
    pc.pc_apt_run(ctx.h, 60, 1, True)
    apt.run(60, threads=8)
    _compare(pc, apt, ctx, b, [(i, i) for i in range(len(shapes))])
    ctx.close()


@pytest.mark.parametrize("labels", [2, 4])
def test_open_boundaries_with_icm(pc, orc, labels):
    """Open axes (the paper's instances are open in x and y): absent bonds,
    odd local fields at the faces, energies over the present bonds, and ICM
    clusters that do not wrap."""
    shapes = [(8, 8, 8), (6, 4, 8), (4, 4, 4), (2, 4, 6), (12, 12, 4)]
    per = [(0, 0, 1), (0, 1, 1), (0, 0, 0), (1, 1, 0), (0, 0, 1)]
    temps = [8, 12, 5, 7, 16]
    dims = np.array(shapes, np.int32)
    J = [W.ea_couplings(s, 10, i) for i, s in enumerate(shapes)]
    betas = [W.geometric_ladder(t) for t in temps]
    b = W.AptBatch(dims, J, betas, labels)
    ctx = pc.Context(0, 31)
    pc.pc_apt_load_bc(ctx.h, dims, per, J, betas, labels, 3)
    apt = orc.Apt(dims, J, betas, labels, seed=31, entry0=3, periodic=np.array(per, np.uint8))
    pc.pc_apt_run(ctx.h, 40, 1, True)
    apt.run(40, threads=8)
    _compare(pc, apt, ctx, b, [(i, i) for i in range(len(shapes))])
    for i, s in enumerate(shapes):   # energies really are open-lattice energies
        st, E, _ = pc.pc_apt_get_state(ctx.h, i, int(np.prod(s)), temps[i] * labels)
        assert E[0] == orc.energy(s, J[i], st[0], periodic=per[i])
    ctx.close()


@pytest.mark.parametrize("labels,icm", [(2, True), (4, True), (1, False)])
def test_joint_label_swaps(pc, orc, labels, icm):
    """The joint swap rule (one decision per temperature pair for all labels)
    against the oracle, across a graph-replayed chunk (140 attempts)."""
    b = W.apt_uniform_batch(3, 4, 8 if labels == 4 else 13, n_labels=labels)
    ctx = pc.Context(0, 17)
    pc.pc_apt_load(ctx.h, b.dims, b.J, b.betas, labels, 0)
    pc.pc_apt_set_joint_swap(ctx.h, True)
    apt = orc.Apt(b.dims, b.J, b.betas, labels, seed=17)
    apt.set_joint_swap(True)
    pc.pc_apt_run(ctx.h, 140, 1, icm)
    apt.run(140, 1, icm, threads=8)
    _compare(pc, apt, ctx, b)
    ctx.close()


@pytest.mark.parametrize("big,cseed,labels,pref", [(False, False, 2, 1), (True, True, 2, 1), (False, True, 4, 2),
                                                    (True, True, 2, 2), (False, False, 4, 1)])
def test_icm_rules_match_oracle(pc, orc, big, cseed, labels, pref):
    """The ICMop switches (big-cluster branch on or off; seed at a uniform
    mismatch site or at a uniform cluster) against the oracle with the same
    switches, with open boundaries and vacancies, one-CTA and two-CTA
    placements, across a graph-replayed chunk (140 attempts)."""
    shapes = [(8, 8, 8), (6, 6, 6), (4, 4, 8), (12, 12, 4)]
    per = [(1, 1, 1), (0, 0, 1), (1, 1, 1), (0, 1, 1)]
    dims = np.array(shapes, np.int32)
    J = [W.ea_couplings(s, 15, i) for i, s in enumerate(shapes)]
    present = [W.random_vacancies(s, 0.05, i) if i == 2 else None for i, s in enumerate(shapes)]
    present = [np.ones(int(np.prod(s)), np.uint8) if p_ is None else p_ for s, p_ in zip(shapes, present)]
    temps = [16, 12, 9, 16] if labels == 4 else [24, 12, 9, 20]
    betas = [W.geometric_ladder(t) for t in temps]
    b = W.AptBatch(dims, J, betas, labels)
    ctx = pc.Context(0, 53)
    pc.pc_apt_load_bc(ctx.h, dims, per, J, betas, labels, 6, present_list=present)
    pc.pc_apt_set_split(ctx.h, pref)
    pc.pc_apt_set_icm_rules(ctx.h, big, cseed)
    apt = orc.Apt(dims, J, betas, labels, seed=53, entry0=6, periodic=np.array(per, np.uint8),
                  present_list=present)
    apt.set_icm_rules(big, cseed)
    pc.pc_apt_run(ctx.h, 140, 1, True)
    apt.run(140, threads=8)
    _compare(pc, apt, ctx, b)
    ctx.close()


@pytest.mark.parametrize("labels,joint", [(2, False), (4, False), (2, True), (1, False)])
def test_split_placement_is_bit_identical_and_matches_oracle(pc, orc, labels, joint):
    """The same batch as one CTA per problem and as two-CTA clusters that
    split the temperatures (even and uneven halves: 13, 24 and 32
    temperatures), across a graph-replayed chunk, against the oracle."""
    temps = [13, 24, 32] if labels < 4 else [13, 16, 12]
    shapes = [(6, 6, 6), (8, 8, 8), (4, 6, 8)]
    dims = np.array(shapes, np.int32)
    J = [W.ea_couplings(s, 11, i) for i, s in enumerate(shapes)]
    betas = [W.geometric_ladder(t) for t in temps]
    b = W.AptBatch(dims, J, betas, labels)
    res = []
    for pref in (1, 2):
        ctx = pc.Context(0, 37)
        pc.pc_apt_load(ctx.h, dims, J, betas, labels, 2)
        pc.pc_apt_set_split(ctx.h, pref)
        assert pc.pc_apt_is_split(ctx.h) == (pref == 2)
        pc.pc_apt_set_joint_swap(ctx.h, joint)
        pc.pc_apt_run(ctx.h, 150, 1, labels > 1)
        res.append([pc.pc_apt_get_state(ctx.h, i, int(np.prod(s)), temps[i] * labels) for i, s in enumerate(shapes)]
                   + [pc.pc_apt_get_best(ctx.h, i, int(np.prod(s)))["E"] for i, s in enumerate(shapes)])
        if pref == 2:
            apt = orc.Apt(dims, J, betas, labels, seed=37, entry0=2)
            apt.set_joint_swap(joint)
            apt.run(150, 1, labels > 1, threads=8)
            _compare(pc, apt, ctx, b)
        ctx.close()
    for x, y in zip(*res):
        if isinstance(x, tuple):
            for u, v in zip(x, y):
                assert np.array_equal(u, v)
        else:
            assert x == y


def test_four_labels_thirty_two_temperatures(pc, orc):
    """The paper's APT shape: 32 temperatures x 4 ICM labels = 128 replicas
    per problem (two CTAs per problem), with open x, y boundaries; 260
    attempts (two graph replays and a remainder)."""
    shapes = [(8, 8, 8), (6, 6, 4)]
    per = [(0, 0, 1), (1, 1, 1)]
    dims = np.array(shapes, np.int32)
    J = [W.ea_couplings(s, 12, i) for i, s in enumerate(shapes)]
    betas = [W.geometric_ladder(32), W.geometric_ladder(27)]
    b = W.AptBatch(dims, J, betas, 4)
    ctx = pc.Context(0, 41)
    pc.pc_apt_load_bc(ctx.h, dims, per, J, betas, 4, 0)
    assert pc.pc_apt_is_split(ctx.h)
    apt = orc.Apt(dims, J, betas, 4, seed=41, periodic=np.array(per, np.uint8))
    pc.pc_apt_run(ctx.h, 60, 1, True)
    apt.run(60, threads=8)
    _compare(pc, apt, ctx, b)
    pc.pc_apt_run(ctx.h, 200, 1, True)
    apt.run(200, threads=8)
    _compare(pc, apt, ctx, b)
    ctx.close()


@pytest.mark.parametrize("groups", [1, 3])
def test_uneven_split_requests_respect_the_cta_limit(pc, orc, groups):
    """32 temperatures x 4 labels: an uneven split would put 12 groups (96
    replicas) in one CTA, so it falls back to the even split (8 groups
    each); results equal the oracle's."""
    shapes = [(6, 6, 6), (4, 4, 8)]
    dims = np.array(shapes, np.int32)
    J = [W.ea_couplings(s, 17, i) for i, s in enumerate(shapes)]
    betas = [W.geometric_ladder(32), W.geometric_ladder(30)]
    b = W.AptBatch(dims, J, betas, 4)
    ctx = pc.Context(0, 59)
    pc.pc_apt_load(ctx.h, dims, J, betas, 4, 0)
    pc.pc_apt_set_launch(ctx.h, 512, 0, 2, groups)
    apt = orc.Apt(dims, J, betas, 4, seed=59)
    pc.pc_apt_run(ctx.h, 30, 1, True)
    apt.run(30, threads=8)
    _compare(pc, apt, ctx, b)
    ctx.close()


@pytest.mark.parametrize("labels,pref", [(2, 1), (2, 2), (4, 2)])
def test_vacancies_and_odd_open_lattices(pc, orc, labels, pref):
    """Missing spins (random vacancies) and odd open lengths padded with a
    vacant layer (5 x 7 x 4, and the paper's 15 x 15 x 12 shape), with ICM,
    one-CTA and two-CTA placements."""
    cases = [((8, 8, 8), (1, 1, 1), None), ((5, 7, 4), (0, 0, 1), "odd"), ((6, 6, 6), (0, 1, 1), None),
             ((15, 15, 12), (0, 0, 1), "odd")]
    dims, per, J, present, temps = [], [], [], [], []
    for i, (d, p_, kind) in enumerate(cases):
        Ji = W.ea_couplings(d, 13, i)
        if kind == "odd":
            pd, pres, Jp = W.pad_odd_open(d, p_, Ji)
        else:
            pd, pres, Jp = np.array(d, np.int32), W.random_vacancies(d, 0.08, i), Ji
        dims.append(pd); per.append(p_); J.append(Jp); present.append(pres)
        temps.append(16 if labels == 4 else 12 + 4 * i)
    dims = np.array(dims, np.int32)
    betas = [W.geometric_ladder(t) for t in temps]
    b = W.AptBatch(dims, J, betas, labels)
    ctx = pc.Context(0, 43)
    pc.pc_apt_load_bc(ctx.h, dims, per, J, betas, labels, 0, present_list=present)
    pc.pc_apt_set_split(ctx.h, pref)
    apt = orc.Apt(dims, J, betas, labels, seed=43, periodic=np.array(per, np.uint8), present_list=present)
    pc.pc_apt_run(ctx.h, 30, 1, True)
    apt.run(30, threads=8)
    _compare(pc, apt, ctx, b)
    ctx.close()


def test_resume_and_chunking(pc, orc):
    """140 attempts in one call (graph replay + remainder) == 60 + 80."""
    b = W.apt_single(L=6, n_temps=10)
    c1 = pc.Context(0, 2)
    pc.pc_apt_load(c1.h, b.dims, b.J, b.betas, 2, 0)
    pc.pc_apt_run(c1.h, 140, 1, True)
    c2 = pc.Context(0, 2)
    pc.pc_apt_load(c2.h, b.dims, b.J, b.betas, 2, 0)
    pc.pc_apt_run(c2.h, 60, 1, True)
    pc.pc_apt_run(c2.h, 80, 1, True)
    for x, y in zip(pc.pc_apt_get_state(c1.h, 0, 216, 20), pc.pc_apt_get_state(c2.h, 0, 216, 20)):
        assert np.array_equal(x, y)
    c1.close()
    c2.close()


def test_target_hit_sweep(pc, orc):
    b = W.apt_single(L=4, n_temps=8)
    ctx = pc.Context(0, 4)
    pc.pc_apt_load(ctx.h, b.dims, b.J, b.betas, 2, 0)
    apt = orc.Apt(b.dims, b.J, b.betas, 2, seed=4)
    pc.pc_apt_run(ctx.h, 300, 1, True)
    apt.run(300)
    e_best = apt.best(0)["E"]
    for tgt in (e_best + 8, e_best):
        pc.pc_apt_set_target(ctx.h, 0, tgt)
        apt.set_target(0, tgt)
    pc.pc_apt_run(ctx.h, 700, 1, True)
    apt.run(700)
    _compare(pc, apt, ctx, b, [(0, 0)])
    E, hit = pc.pc_apt_get_best_all(ctx.h, 1)
    assert E[0] == apt.best(0)["E"] and hit[0] == apt.best(0)["hit_sweep"]
    ctx.close()


@pytest.mark.parametrize("pref", [0, 1])
def test_c3_shape_sampled(pc, orc, pref):
    """64 instances of L = 12 with 32 x 2 replicas (the APT+ICM batch
    shape), in its default placement (two-CTA clusters: the batch fills at
    most half the SMs) and in one CTA per problem; 260 attempts = two
    replays of the 128-attempt CUDA graph and a remainder.  Instances 0, 31
    and 63 re-computed by the oracle."""
    b = W.apt_uniform_batch(64, 12, 32)
    ctx = pc.Context(0, 9)
    pc.pc_apt_load(ctx.h, b.dims, b.J, b.betas, 2, 0)
    pc.pc_apt_set_split(ctx.h, pref)
    pc.pc_apt_run(ctx.h, 260, 1, True)
    for i in (0, 31, 63):
        apt = orc.Apt(b.dims[i:i + 1], b.J[i:i + 1], b.betas[i:i + 1], 2, seed=9, entry0=i)
        apt.run(260)
        _compare(pc, apt, ctx, b, [(i, 0)])
    ctx.close()


def test_sweep_to_swap_ratio_ten(pc, orc):
    """Ten sweeps per swap attempt (the ratio the paper uses to find the
    best energies, Methods "Instances"), 130 attempts (a graph replay and a
    remainder), with ICM, against the oracle."""
    shapes = [(6, 6, 6), (4, 4, 8), (8, 8, 8)]
    dims = np.array(shapes, np.int32)
    J = [W.ea_couplings(s, 14, i) for i, s in enumerate(shapes)]
    betas = [W.geometric_ladder(t) for t in (12, 7, 20)]
    b = W.AptBatch(dims, J, betas, 2)
    ctx = pc.Context(0, 47)
    pc.pc_apt_load(ctx.h, dims, J, betas, 2, 11)
    apt = orc.Apt(dims, J, betas, 2, seed=47, entry0=11)
    pc.pc_apt_run(ctx.h, 130, 10, True)
    apt.run(130, 10, True, threads=8)
    _compare(pc, apt, ctx, b)
    assert pc.pc_apt_progress(ctx.h) == (1300, 130)
    ctx.close()


@pytest.mark.parametrize("pref", [1, 2])
def test_sweep_to_swap_ratio_516(pc, orc, pref):
    """516 sweeps per swap attempt (the largest ratio of the paper's
    sweep-to-swap study, Supplementary "APT Algorithm with ICM"), 5 attempts
    in one call and 2 more in a second (2580 + 1032 sweeps), with ICM,
    against the oracle; one CTA per problem (pref 1) and two-CTA clusters
    (pref 2)."""
    shapes = [(6, 6, 6), (4, 4, 8), (8, 8, 8)]
    dims = np.array(shapes, np.int32)
    J = [W.ea_couplings(s, 15, i) for i, s in enumerate(shapes)]
    betas = [W.geometric_ladder(t) for t in (12, 10, 16)]   # >= 9 each, so that pref 2 splits
    b = W.AptBatch(dims, J, betas, 2)
    ctx = pc.Context(0, 48)
    pc.pc_apt_load(ctx.h, dims, J, betas, 2, 5)
    pc.pc_apt_set_split(ctx.h, pref)
    assert pc.pc_apt_is_split(ctx.h) == (pref == 2)
    apt = orc.Apt(dims, J, betas, 2, seed=48, entry0=5)
    pc.pc_apt_run(ctx.h, 5, 516, True)
    apt.run(5, 516, True, threads=8)
    _compare(pc, apt, ctx, b)
    pc.pc_apt_run(ctx.h, 2, 516, True)
    apt.run(2, 516, True, threads=8)
    _compare(pc, apt, ctx, b)
    assert pc.pc_apt_progress(ctx.h) == (7 * 516, 7)
    ctx.close()


@pytest.mark.parametrize("spp", [1, 10])
def test_more_than_32_sites_per_thread(pc, orc, spp):
    """64 threads per CTA in two chunks of 32 on a 16^3 lattice (2048 sites
    per colour): each thread sweeps 64 sites, so its byte-lane energy counts
    are reduced in two blocks of 32 sites, and the flood fill runs several
    2x2x2 blocks per thread; with ICM, against the oracle."""
    shapes = [(16, 16, 16), (6, 6, 6)]
    dims = np.array(shapes, np.int32)
    J = [W.ea_couplings(s, 16, i) for i, s in enumerate(shapes)]
    betas = [W.geometric_ladder(16), W.geometric_ladder(12)]
    b = W.AptBatch(dims, J, betas, 2)
    ctx = pc.Context(0, 49)
    pc.pc_apt_load(ctx.h, dims, J, betas, 2, 2)
    pc.pc_apt_set_launch(ctx.h, 64, 2, 1, 0)
    apt = orc.Apt(dims, J, betas, 2, seed=49, entry0=2)
    n = 24 if spp == 1 else 4
    pc.pc_apt_run(ctx.h, n, spp, True)
    apt.run(n, spp, True, threads=8)
    _compare(pc, apt, ctx, b)
    ctx.close()


def test_c4_mixed_batch_sampled(pc, orc):
    """256 instances, L uniform over {6..16}, 24-32 temperatures x 2, 140
    attempts (a graph replay and a remainder); the smallest, the largest and
    a middle instance re-computed by the oracle."""
    b = W.apt_mixed_batch()
    ctx = pc.Context(0, 17)
    pc.pc_apt_load(ctx.h, b.dims, b.J, b.betas, 2, 0)
    pc.pc_apt_run(ctx.h, 140, 1, True)
    work = [int(np.prod(d)) * len(t) for d, t in zip(b.dims, b.betas)]
    picks = {int(np.argmin(work)), int(np.argmax(work)), 128}
    for i in picks:
        apt = orc.Apt(b.dims[i:i + 1], b.J[i:i + 1], b.betas[i:i + 1], 2, seed=17, entry0=i)
        apt.run(140)
        _compare(pc, apt, ctx, b, [(i, 0)])
    ctx.close()


@pytest.mark.parametrize("labels", [2, 4])
def test_launch_shape_does_not_change_results(pc, orc, labels):
    """Shapes the autotuner chooses from (one CTA or two-CTA clusters split
    evenly or unevenly, 256/384/512 threads, thread chunks 0/1/2/4; also 320
    and 448 threads) and the autotuner's own choice give bit-identical
    chains, equal to the oracle's."""
    shapes = [(8, 8, 8), (6, 6, 6), (4, 4, 8)]
    temps = [20, 12, 9] if labels == 2 else [16, 12, 9]
    dims = np.array(shapes, np.int32)
    J = [W.ea_couplings(s, 16, i) for i, s in enumerate(shapes)]
    betas = [W.geometric_ladder(t) for t in temps]
    b = W.AptBatch(dims, J, betas, labels)
    ref = None
    shapes_run = [(sp, tpb, nch, 0) for sp in (1, 2) for tpb in (256, 384, 512) for nch in (0, 1, 2, 4)]
    shapes_run += [(1, 320, 1, 0), (2, 448, 1, 0), (2, 512, 0, 1), (2, 256, 2, 3), None]
    for shape in shapes_run:
        ctx = pc.Context(0, 13)
        pc.pc_apt_load(ctx.h, dims, J, betas, labels, 0)
        if shape is None:
            tpb, nch, split, grp = pc.pc_apt_autotune(ctx.h, 8, True)
            assert tpb in (256, 320, 384, 448, 512) and nch in (0, 1, 2, 4) and grp in (0, 1, 2, 3)
        else:
            sp, tpb, nch, grp = shape
            pc.pc_apt_set_launch(ctx.h, tpb, nch, sp, grp)
            assert pc.pc_apt_is_split(ctx.h) == (sp == 2)
        pc.pc_apt_run(ctx.h, 40, 1, True)
        got = [pc.pc_apt_get_state(ctx.h, i, int(np.prod(s)), t * labels) for i, (s, t) in enumerate(zip(shapes, temps))]
        if ref is None:
            ref = got
            apt = orc.Apt(dims, J, betas, labels, seed=13)
            apt.run(40, threads=8)
            _compare(pc, apt, ctx, b)
        else:
            for x, y in zip(ref, got):
                for u, v in zip(x, y):
                    assert np.array_equal(u, v), shape
        ctx.close()


@pytest.mark.parametrize("labels", [2, 4])
def test_mixed_placement_matches_oracle(pc, orc, labels):
    """Split preference 3: the two 8^3 problems (20 temperatures) run as
    two-CTA clusters in one launch, the 150 problems of 4^3 (9 temperatures,
    below the batch's mean work per SM) as one CTA each in a second launch
    on a second stream; 40 and 130 attempts in both orders (130 = a captured
    graph with both launches, and a remainder), with ICM, against the
    oracle."""
    shapes = [(8, 8, 8)] * 2 + [(4, 4, 4)] * 150
    temps = [20, 20] + [9] * 150
    dims = np.array(shapes, np.int32)
    J = [W.ea_couplings(s_, 17, i) for i, s_ in enumerate(shapes)]
    betas = [W.geometric_ladder(t) for t in temps]
    b = W.AptBatch(dims, J, betas, labels)
    ctx = pc.Context(0, 51)
    pc.pc_apt_load(ctx.h, dims, J, betas, labels, 4)
    pc.pc_apt_set_split(ctx.h, 3)
    assert pc.pc_apt_is_split(ctx.h) == 2
    apt = orc.Apt(dims, J, betas, labels, seed=51, entry0=4)
    # with 2 labels the first launch after the placement change is the
    # captured graph
    first, second = (130, 40) if labels == 2 else (40, 130)
    pc.pc_apt_run(ctx.h, first, 1, True)
    apt.run(first, 1, True, threads=8)
    _compare(pc, apt, ctx, b, [(i, i) for i in (0, 1, 2, 77, 151)])
    pc.pc_apt_run(ctx.h, second, 1, True)
    apt.run(second, 1, True, threads=8)
    _compare(pc, apt, ctx, b)
    ctx.close()


def test_swap_tables_unstaged_where_they_do_not_fit(pc, orc):
    """32 temperatures x 4 labels on a 16^3 lattice (the paper's label
    count): a two-CTA cluster with staged swap tables would exceed shared
    memory, so this batch reads them from global memory; with ICM, against
    the oracle."""
    dims = np.array([(16, 16, 16)], np.int32)
    J = [W.ea_couplings((16, 16, 16), 18, 0)]
    betas = [W.geometric_ladder(32)]
    b = W.AptBatch(dims, J, betas, 4)
    ctx = pc.Context(0, 53)
    pc.pc_apt_load(ctx.h, dims, J, betas, 4, 1)
    assert pc.pc_apt_is_split(ctx.h) == 1
    apt = orc.Apt(dims, J, betas, 4, seed=53, entry0=1)
    pc.pc_apt_run(ctx.h, 12, 1, True)
    apt.run(12, 1, True, threads=8)
    _compare(pc, apt, ctx, b)
    ctx.close()


def test_checkpoint_resume_bit_exact(pc, tmp_path):
    """200 attempts == 90, save, restore into a fresh context, 110 more."""
    b = W.apt_uniform_batch(2, 6, 12)
    c1 = pc.Context(0, 8)
    pc.pc_apt_load(c1.h, b.dims, b.J, b.betas, 2, 0)
    pc.pc_apt_run(c1.h, 200, 1, True)
    c2 = pc.Context(0, 8)
    pc.pc_apt_load(c2.h, b.dims, b.J, b.betas, 2, 0)
    pc.pc_apt_run(c2.h, 90, 1, True)
    path = str(tmp_path / "apt.ckpt")
    pc.pc_apt_save(c2.h, path)
    c2.close()
    c3 = pc.Context(0, 8)
    pc.pc_apt_load(c3.h, b.dims, b.J, b.betas, 2, 0)
    pc.pc_apt_restore(c3.h, path)
    pc.pc_apt_run(c3.h, 110, 1, True)
    assert pc.pc_apt_progress(c3.h) == pc.pc_apt_progress(c1.h)
    for i in range(2):
        for u, v in zip(pc.pc_apt_get_state(c1.h, i, 216, 24), pc.pc_apt_get_state(c3.h, i, 216, 24)):
            assert np.array_equal(u, v)
        assert pc.pc_apt_get_best(c1.h, i, 216)["E"] == pc.pc_apt_get_best(c3.h, i, 216)["E"]
        for u, v in zip(pc.pc_apt_get_stats(c1.h, i, 12, 2), pc.pc_apt_get_stats(c3.h, i, 12, 2)):
            assert np.array_equal(u, v)
    c4 = pc.Context(0, 9)    # another seed: refused
    pc.pc_apt_load(c4.h, b.dims, b.J, b.betas, 2, 0)
    with pytest.raises(pc.PcompError):
        pc.pc_apt_restore(c4.h, path)
    c1.close(); c3.close(); c4.close()


def test_apt_rejects_bad_input(pc):
    ctx = pc.Context(0, 0)
    J = [W.ea_couplings((4, 4, 4), 1, 0)]
    with pytest.raises(pc.PcompError):
        pc.pc_apt_run(ctx.h, 10, 1, True)                          # before load
    with pytest.raises(pc.PcompError):
        pc.pc_apt_load(ctx.h, [(4, 4, 4)], J, [W.geometric_ladder(33)], 2, 0)   # > 32 temperatures
    with pytest.raises(pc.PcompError):   # 128 replicas need two CTAs; 5 temperatures cannot split
        pc.pc_apt_load(ctx.h, [(4, 4, 4)] * 2, J * 2, [W.geometric_ladder(32), W.geometric_ladder(5)], 4, 0)
    with pytest.raises(pc.PcompError):
        pc.pc_apt_load(ctx.h, [(4, 4, 4)], J, [np.array([1.0, 0.5])], 2, 0)     # not increasing
    with pytest.raises(pc.PcompError):
        pc.pc_apt_load(ctx.h, [(5, 4, 4)], [W.ea_couplings((5, 4, 4), 1, 0)], [np.ones(1)], 2, 0)
    pc.pc_apt_load(ctx.h, [(4, 4, 4)], J, [W.geometric_ladder(4)], 1, 0)
    with pytest.raises(pc.PcompError):
        pc.pc_apt_run(ctx.h, 5, 1, True)                           # ICM needs 2 labels
    ctx.close()


# ---------------------------------------------------------------- ladder / pilot
def test_adaptive_ladder_bit_exact(pc, orc):
    shapes = [(4, 4, 4), (6, 6, 6), (4, 4, 8)]
    J = [W.ea_couplings(s, 3, i) for i, s in enumerate(shapes)]
    ctx = pc.Context(0, 5)
    res = pc.pc_adaptive_ladder(ctx.h, shapes, J, entry0=10, n_chains=20, sweeps=60, tail=30,
                                max_len=40)
    for i, s in enumerate(shapes):
        beta, sig, ok = orc.adaptive_ladder(s, J[i], entry=10 + i, seed=5, n_chains=20, sweeps=60,
                                            tail=30, max_len=40)
        assert res[i][2] == ok
        assert np.array_equal(res[i][0], beta) and np.array_equal(res[i][1], sig)
    ctx.close()


def test_adaptive_ladder_many_chains(pc, orc):
    """100 chains (more than one CTA's 64 replicas), paper's beta_0 and alpha."""
    J = W.ea_couplings((6, 6, 6), 3, 9)
    ctx = pc.Context(0, 6)
    res = pc.pc_adaptive_ladder(ctx.h, [(6, 6, 6)], [J], n_chains=100, sweeps=40, tail=20, max_len=6)
    beta, sig, ok = orc.adaptive_ladder((6, 6, 6), J, seed=6, n_chains=100, sweeps=40, tail=20, max_len=6)
    assert np.array_equal(res[0][0], beta) and np.array_equal(res[0][1], sig) and res[0][2] == ok
    ctx.close()


def test_pilot_histograms_bit_exact(pc, orc):
    shapes = [(4, 4, 4), (8, 8, 8)]
    J = [W.ea_couplings(s, 4, i) for i, s in enumerate(shapes)]
    betas = W.geometric_ladder(4)
    ctx = pc.Context(0, 8)
    got = pc.pc_pilot_hist(ctx.h, shapes, J, betas, entry0=3, chains_per_beta=8, sweeps=50, burn=20)
    for i, s in enumerate(shapes):
        ref = orc.pilot_hist(s, J[i], betas, entry=3 + i, seed=8, chains_per_beta=8, sweeps=50, burn=20)
        assert np.array_equal(got[i], ref)
    ctx.close()


def test_features_and_resampling_match_oracle(pc):
    from oracle import mlp
    for i, s in enumerate([(4, 4, 4), (6, 8, 4), (16, 16, 16)]):
        J = W.ea_couplings(s, 12, i)
        f = pc.pc_instance_features(s, J)
        ref = mlp.instance_features(s, J)
        assert f[1] == ref[1] and f[2] == ref[2] and abs(f[0] - ref[0]) < 1e-15
    for ln in (1, 2, 20, 33, 34):
        beta = np.sort(np.random.default_rng(ln).random(ln)) + 0.5
        assert np.array_equal(pc.pc_resample_ladder(beta, 32), mlp.resample_ladder(beta, 32))
