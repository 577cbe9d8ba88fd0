"""DT-SQA on the GPU against the oracle: bit-exact energies and spins."""
import numpy as np
import pytest

from paper_2503_10302_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    from paper_2503_10302_gb300 import build, pcomp
    build.build()
    return pcomp


def test_device_philox_equals_oracle(pc, orc):
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    for seed in (0, 0x123456789ABCDEF):
        ctx = pc.Context(0, seed)
        assert np.array_equal(pc.pc_philox(ctx.h, ctr), orc.philox(ctr, seed))
        ctx.close()


def test_sqa_tables_equal_oracle(pc, orc):
    wl = W.sqa_workload(L=4, P=64, R=1, n_sweeps=57)
    ctx = pc.Context(0, 1)
    pc.pc_sqa_setup(ctx.h, wl.dims, wl.J, wl.P, wl.T, wl.gamma)
    beta_eff = 1.0 / (wl.P * wl.T)
    for s in (0, 1, 28, 56):
        tab, jq = pc.pc_sqa_get_table(ctx.h, s)
        assert jq == orc.jperp_q(wl.gamma[s], wl.P, wl.T)
        for m, n in enumerate((-2, 0, 2)):
            for c in range(7):
                assert tab[m, c] == orc.sqa_threshold(beta_eff, 2 * c - 6, jq, n)
    ctx.close()


def _check_all_rows(pc, orc, ctx, wl):
    beta_eff = 1.0 / (wl.P * wl.T)
    for s in range(len(wl.gamma)):
        tab, jq = pc.pc_sqa_get_table(ctx.h, s)
        assert jq == orc.jperp_q(wl.gamma[s], wl.P, wl.T), s
        for m, n in enumerate((-2, 0, 2)):
            for c in range(7):
                assert tab[m, c] == orc.sqa_threshold(beta_eff, 2 * c - 6, jq, n), (s, m, c)


def test_sqa_long_schedules_threaded_rows_and_reused_buffers(pc, orc):
    """Long schedules build their table rows on several host threads, in
    splits that do not divide the schedule evenly; later setups on the same
    context reuse (or grow) the device buffers.  Every row equals the
    oracle's, and an anneal after a shrinking setup stays bit-exact."""
    ctx = pc.Context(0, 21)
    for L, P, S in ((4, 64, 1531), (6, 32, 4099), (4, 16, 1031)):
        wl = W.sqa_workload(L=L, P=P, R=1, n_sweeps=S, index=S)
        pc.pc_sqa_setup(ctx.h, wl.dims, wl.J, wl.P, wl.T, wl.gamma)
        _check_all_rows(pc, orc, ctx, wl)
    dims, P, R, S, seed = (4, 4, 4), 16, 3, 20, 21
    J = W.ea_couplings(dims, W.SEED_INSTANCES, seed)
    gamma = W.linear_gamma_schedule(S)
    E_ref = orc.sqa_anneal(dims, J, P, 0.05, gamma, R, run0=0, seed=seed)
    pc.pc_sqa_setup(ctx.h, dims, J, P, 0.05, gamma)
    E = pc.pc_sqa_run(ctx.h, R, 0, P, int(np.prod(dims)))
    ctx.close()
    assert np.array_equal(E, E_ref)


CASES = [
    # dims, P, R, sweeps, seed
    ((4, 4, 4), 16, 6, 40, 0),
    ((8, 8, 8), 64, 3, 12, 5),
    ((6, 4, 2), 32, 5, 30, 7),
    ((2, 2, 2), 16, 4, 25, 9),
    ((4, 6, 8), 48, 3, 15, 11),
    ((10, 10, 10), 128, 2, 4, 13),
]


@pytest.mark.parametrize("dims,P,R,S,seed", CASES)
def test_sqa_bit_exact(pc, orc, dims, P, R, S, seed):
    J = W.ea_couplings(dims, W.SEED_INSTANCES, seed)
    gamma = W.linear_gamma_schedule(S)
    N = int(np.prod(dims))
    run0 = 17 * seed
    E_ref, s_ref = orc.sqa_anneal(dims, J, P, 0.05, gamma, R, run0=run0, seed=seed,
                                  want_spins=True)
    ctx = pc.Context(0, seed)
    pc.pc_sqa_setup(ctx.h, dims, J, P, 0.05, gamma)
    E, s = pc.pc_sqa_run(ctx.h, R, run0, P, N, want_spins=True)
    ctx.close()
    assert np.array_equal(s, s_ref)
    assert np.array_equal(E, E_ref)


@pytest.mark.parametrize("dims,P,R,S,seed", [CASES[0], CASES[2], CASES[5]])
def test_replica_correlation_matches_oracle_spins(pc, orc, dims, P, R, S, seed):
    """Fig. S17's C_r from the device reduction equals N^-1 sum_i s_i0 s_ir
    computed from the oracle's final spins."""
    import torch
    J = W.ea_couplings(dims, W.SEED_INSTANCES, seed)
    gamma = W.linear_gamma_schedule(S)
    N = int(np.prod(dims))
    E_ref, s_ref = orc.sqa_anneal(dims, J, P, 0.05, gamma, R, run0=3, seed=seed, want_spins=True)
    want = np.einsum("rn,rkn->rk", s_ref[:, 0, :].astype(np.int64), s_ref.astype(np.int64))
    ctx = pc.Context(0, seed)
    pc.pc_sqa_setup(ctx.h, dims, J, P, 0.05, gamma)
    E = torch.zeros((R, P), dtype=torch.int32, device="cuda")
    C = torch.zeros((R, P), dtype=torch.int32, device="cuda")
    pc.pc_sqa_run_corr_dev(ctx.h, R, 3, E.data_ptr(), C.data_ptr())
    torch.cuda.synchronize()
    ctx.close()
    assert np.array_equal(E.cpu().numpy(), E_ref)
    got = C.cpu().numpy()
    assert np.array_equal(got, want)
    assert (got[:, 0] == N).all()


@pytest.mark.parametrize("dims,per,P,R,S", [((8, 8, 4), (0, 0, 1), 32, 4, 20),
                                              ((4, 6, 8), (0, 1, 0), 16, 3, 30),
                                              ((6, 6, 6), (0, 0, 0), 64, 2, 12)])
def test_sqa_open_boundaries_bit_exact(pc, orc, dims, per, P, R, S):
    """Open axes (the paper's instances are open in x and y): absent bonds,
    odd in-slice fields at the faces, slice energies over the present bonds."""
    J = W.ea_couplings(dims, W.SEED_INSTANCES, 77)
    gamma = W.linear_gamma_schedule(S)
    N = int(np.prod(dims))
    E_ref, s_ref = orc.sqa_anneal(dims, J, P, 0.05, gamma, R, run0=5, seed=3, want_spins=True,
                                  periodic=np.array(per, np.uint8))
    ctx = pc.Context(0, 3)
    pc.pc_sqa_setup_bc(ctx.h, dims, per, J, P, 0.05, gamma)
    E, s = pc.pc_sqa_run(ctx.h, R, 5, P, N, want_spins=True)
    ctx.close()
    assert np.array_equal(s, s_ref)
    assert np.array_equal(E, E_ref)
    assert E[0, 0] == orc.energy(dims, J, s_ref[0, 0], periodic=per)


@pytest.mark.parametrize("dims,per,kind", [((8, 8, 8), (1, 1, 1), "vac"), ((7, 5, 4), (0, 0, 1), "odd")])
def test_sqa_vacancies_and_odd_open_lattice(pc, orc, dims, per, kind):
    """Missing spins and an odd open lattice padded with a vacant layer."""
    J = W.ea_couplings(dims, W.SEED_INSTANCES, 78)
    if kind == "odd":
        dims, present, J = W.pad_odd_open(dims, per, J)
    else:
        present = W.random_vacancies(dims, 0.1, 5)
    gamma = W.linear_gamma_schedule(15)
    N = int(np.prod(dims))
    E_ref, s_ref = orc.sqa_anneal(dims, J, 32, 0.05, gamma, 3, run0=2, seed=4, want_spins=True,
                                  periodic=np.array(per, np.uint8), present=present)
    ctx = pc.Context(0, 4)
    pc.pc_sqa_setup_bc(ctx.h, dims, per, J, 32, 0.05, gamma, present=present)
    E, s = pc.pc_sqa_run(ctx.h, 3, 2, 32, N, want_spins=True)
    ctx.close()
    assert np.array_equal(s, s_ref)
    assert np.array_equal(E, E_ref)


def test_sqa_zero_sweeps_is_random_init(pc, orc):
    dims, P = (4, 4, 4), 16
    J = W.ea_couplings(dims, 1, 0)
    E_ref, s_ref = orc.sqa_anneal(dims, J, P, 0.05, np.zeros(0), 3, seed=2, want_spins=True)
    ctx = pc.Context(0, 2)
    pc.pc_sqa_setup(ctx.h, dims, J, P, 0.05, np.zeros(0))
    E, s = pc.pc_sqa_run(ctx.h, 3, 0, P, 64, want_spins=True)
    assert np.array_equal(s, s_ref) and np.array_equal(E, E_ref)
    ctx.close()


def test_sqa_rejects_bad_shapes(pc):
    ctx = pc.Context(0, 0)
    J = W.ea_couplings((4, 4, 4), 1, 0)
    for dims, P in (((4, 4, 4), 24), ((5, 4, 4), 16), ((4, 4, 4), 0), ((4, 4, 4), 144)):
        with pytest.raises(pc.PcompError):
            pc.pc_sqa_setup(ctx.h, dims, W.ea_couplings(dims, 1, 0), P, 0.05, np.ones(3))
    with pytest.raises(pc.PcompError):
        pc.pc_sqa_setup(ctx.h, (4, 4, 4), J, 16, 0.05, np.array([1.0, 0.0]))
    ctx.close()


def test_sqa_full_size_sampled_runs(pc, orc):
    """The L=8, P=64, R=256, 1e4-sweep anneal in the bench's launch
    configuration; runs 0, 137 and 255 re-computed by the oracle."""
    wl = W.sqa_workload()
    N = 512
    ctx = pc.Context(0, 0)
    pc.pc_sqa_setup(ctx.h, wl.dims, wl.J, wl.P, wl.T, wl.gamma)
    E = pc.pc_sqa_run(ctx.h, wl.R, 0, wl.P, N)
    ctx.close()
    assert (E % 2 == (3 * N) % 2).all() and (E >= -3 * N).all()
    picks = [0, 137, 255]
    for r in picks:
        E_ref = orc.sqa_anneal(wl.dims, wl.J, wl.P, wl.T, wl.gamma, 1, run0=r, seed=0)
        assert np.array_equal(E[r], E_ref[0]), r


def test_bounded_wait_reports_timeout_and_context_survives(pc, orc):
    """Every wait for a previous chunk runs out (nothing sets its flag); the
    kernel returns, the host reports PC_EDEVICE, and the next anneal on the
    same context is still bit-exact."""
    dims, P = (4, 4, 4), 16
    J = W.ea_couplings(dims, 2, 0)
    gamma = W.linear_gamma_schedule(20)
    ctx = pc.Context(0, 5)
    pc.pc_sqa_setup(ctx.h, dims, J, P, 0.05, gamma)
    assert pc.pc_sqa_selftest_wait(ctx.h) == pc.PC_EDEVICE
    pc.pc_sqa_setup(ctx.h, dims, J, P, 0.05, gamma)
    E = pc.pc_sqa_run(ctx.h, 3, 0, P, 64)
    assert np.array_equal(E, orc.sqa_anneal(dims, J, P, 0.05, gamma, 3, seed=5))
    ctx.close()
