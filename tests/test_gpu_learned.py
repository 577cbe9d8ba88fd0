"""The learned ladder behind the C ABI (pc_learned_ladder, pc_ladder_judge)
against the oracle's composition of the same steps (oracle/learned.py).

* Ladders: the network runs in fp32 on the GPU and in float64 in the
  oracle, so the ladders agree within a tolerance, element by element.  A
  ladder entry is a cumulative sum of at most 32 softplus terms, each the
  output of four layers whose dot products have at most 259 terms; fp32
  rounding of such a sum is bounded by K * 2^-24 of the sum of the terms'
  magnitudes (K = 259), a few 1e-5 relative.  The tests allow
  |gpu - oracle| <= 1e-4 * |oracle| + 1e-5 * max|oracle| per entry.
* The judge is integer work given a ladder (APT chains are bit-exact), so
  on the same ladders its acceptances and decisions must be identical.
* The fallback ladder is the adaptive ladder (bit-exact) resampled in
  double, so it must be identical too.
"""
import numpy as np
import pytest

from paper_2503_10302_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL, ATOL_REL = 1e-4, 1e-5
PILOT = W.geometric_ladder(4, 0.2, 3.0)
KW = dict(n_chains=8, sweeps=80, tail=40, max_len=24)


@pytest.fixture(scope="module")
def pc():
    from paper_2503_10302_gb300 import build, pcomp
    build.build()
    return pcomp


@pytest.fixture(scope="module")
def ol(orc):
    from oracle import learned
    return learned


def _params(seed, scale=0.5):
    from oracle import mlp
    return [(w * scale, b + 0.01) for w, b in W.mlp_init(mlp.SIZES, seed)]


def _close(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    bound = RTOL * np.abs(b) + ATOL_REL * np.abs(b).max()
    assert (np.abs(a - b) <= bound).all(), float((np.abs(a - b) / bound).max())


def _instances():
    dims = [(4, 4, 4), (6, 6, 6), (8, 8, 8), (4, 6, 8), (6, 4, 4)]
    J = [W.ea_couplings(d, 71, i) for i, d in enumerate(dims)]
    return dims, J


def test_learned_ladder_matches_oracle_composition(pc, ol):
    """Pilot histograms -> features -> network -> monotone ladder, on the
    device, against the oracle's composition (no judge)."""
    dims, J = _instances()
    params = _params(41)
    ctx = pc.Context(0, 6)
    m = pc.Mlp(ctx, params, beta_min=0.05)
    beta, acc, fb = pc.pc_learned_ladder(ctx.h, m, dims, J, PILOT, entry0=9, pilot_sweeps=96, pilot_burn=32,
                                         probe_attempts=0)
    ref, _, _ = ol.learned_ladder(params, dims, J, PILOT, entry0=9, seed=6, beta_min=0.05, pilot_sweeps=96,
                                  pilot_burn=32, probe_attempts=0)
    _close(beta, ref)
    assert (np.diff(beta, axis=1) > 0).all() and not fb.any() and (acc == -1).all()
    # the device features are the oracle's features rounded once to fp32
    # (cbrt may differ by an ulp between the device and libm)
    X_ref = ol.features(dims, J, PILOT, 9, 6, 8, 96, 32)
    X = pc.pc_learned_features(ctx.h, dims, J, PILOT, entry0=9, pilot_sweeps=96, pilot_burn=32)
    assert np.array_equal(X[:, 1:], X_ref[:, 1:].astype(np.float32))
    assert np.allclose(X[:, 0], X_ref[:, 0], rtol=2.0 ** -23, atol=0)
    m.close()
    ctx.close()


def test_ladder_judge_is_bit_exact(pc, ol):
    """pc_ladder_judge on ladders the oracle made: geometric, one with an
    enormous gap (fails), and the oracle's learned ladders; two and four
    labels; across a 128-attempt chunk boundary."""
    dims, J = _instances()
    params = _params(42)
    lad, _, _ = ol.learned_ladder(params, dims, J, PILOT, entry0=3, seed=8, pilot_sweeps=64, pilot_burn=16,
                                  probe_attempts=0)
    gap = np.concatenate([np.linspace(0.02, 0.05, 16), np.linspace(8.0, 8.5, 16)])
    ladders = [lad[0], gap, W.geometric_ladder(32, 0.2, 3.0), lad[3], lad[4]]
    for labels in (2, 4):
        ctx = pc.Context(0, 8)
        acc, ok = pc.pc_ladder_judge(ctx.h, dims, J, ladders, entry0=3, n_labels=labels, probe_attempts=150,
                                     acc_floor=0.2)
        _, _, rate, ok_ref = ol.judge(dims, J, ladders, entry0=3, seed=8, n_labels=labels, attempts=150,
                                      floor=0.2, threads=8)
        assert np.array_equal(acc, rate), labels
        assert np.array_equal(ok, ok_ref) and not ok[1]
        ctx.close()


def test_learned_ladder_fallback_is_exact(pc, ol):
    """A floor above 1 rejects every predicted ladder: each instance gets
    its adaptive ladder resampled to 32 points, identical to the oracle's.
    A network whose ladder has one enormous gap is rejected, and the
    rejected instances fall back with their own entry ids."""
    dims, J = _instances()
    ctx = pc.Context(0, 12)
    m = pc.Mlp(ctx, _params(43))
    beta, acc, fb = pc.pc_learned_ladder(ctx.h, m, dims, J, PILOT, entry0=20, pilot_sweeps=64, pilot_burn=16,
                                         probe_attempts=30, acc_floor=1.5, **KW)
    assert fb.all()
    for i in range(len(J)):
        assert np.array_equal(beta[i], ol.fallback(dims[i], J[i], 20 + i, 12, **KW)), i
    m.close()
    # a network whose ladder jumps from beta 0.78 to 3.8 between outputs 15
    # and 16 (softplus(3) = 3.05): on 6^3 and 8^3 lattices that pair
    # accepts about a tenth of its swaps (a 4^3 lattice visits its ground
    # state at beta 0.78 often enough to accept a quarter), well under the
    # floor of 0.5, so both instances fall back, as in the oracle
    params = _params(44, scale=0.0)
    params[-1] = (params[-1][0], np.where(np.arange(32) == 16, 3.0, -3.0).astype(np.float32))
    m = pc.Mlp(ctx, params)
    beta, acc, fb = pc.pc_learned_ladder(ctx.h, m, dims[1:3], J[1:3], PILOT, entry0=20, pilot_sweeps=64,
                                         pilot_burn=16, probe_attempts=200, acc_floor=0.5, **KW)
    _, rate_ref, fb_ref = ol.learned_ladder(params, dims[1:3], J[1:3], PILOT, entry0=20, seed=12,
                                            pilot_sweeps=64, pilot_burn=16, probe_attempts=200, acc_floor=0.5,
                                            ladder_kw=KW, threads=8)
    assert fb.all() and fb_ref.all(), (fb, fb_ref)
    assert (acc[:, 15] < 0.25).all() and (rate_ref[:, 15] < 0.25).all(), (acc[:, 15], rate_ref[:, 15])
    for i in range(2):
        assert np.array_equal(beta[i], ol.fallback(dims[1 + i], J[1 + i], 20 + i, 12, **KW))
    m.close()
    ctx.close()


def test_weights_file_round_trip(pc, tmp_path):
    from oracle import mlp
    params = _params(45)
    ctx = pc.Context(0, 0)
    m = pc.Mlp(ctx, params, beta_min=0.25)
    path = str(tmp_path / "w.bin")
    m.save(path)
    m2 = pc.Mlp(ctx, path=path)
    for (a, b), (c, d) in zip(m.params(), m2.params()):
        assert np.array_equal(a, c) and np.array_equal(b, d)
    X = np.random.default_rng(0).random((3, mlp.N_IN)).astype(np.float32)
    assert np.array_equal(m.forward(X), m2.forward(X))
    with open(path, "r+b") as f:
        f.truncate(1000)
    with pytest.raises(pc.PcompError):
        pc.Mlp(ctx, path=path)
    m.close()
    m2.close()
    ctx.close()


def test_trained_network_gains_over_the_methods_without_it(pc):
    """What the committed network (trained on the GPU by this library's
    kernels on 20 000 instances with L = 6 .. 16) gains, on 32 held-out
    L = 16 instances: time to rho_E <= 1e-3 (Eq. rho_E_f), construction of
    the ladder included, per instance, measured.

    * Against the adaptive procedure (Algorithm S2's preprocessing, which
      the network replaces): no more sweeps to the target, within the
      sampling noise of a median over 32 instances (a factor 1.25), and less
      wall time (the pilot run, network and judge cost a fraction of the
      adaptive procedure).
    * Against the input-free geometric ladder 0.2 .. 3.0 (the range of the
      pilot temperatures): strictly fewer sweeps to the target.
    The per-size mean of the training ladders is reported, not asserted."""
    from paper_2503_10302_gb300 import ladder
    ctx = pc.Context(0, 5)
    net = pc.Mlp(ctx, path=ladder.WEIGHTS)
    res = ladder.compare(net, ladder.load_means(), n_eval=32, L=16, best_runs=10, best_sweeps=20000,
                         max_sweeps=100000)
    net.close()
    ctx.close()
    lrn, ada, geo = res["learned"], res["adaptive"], res["geometric"]
    summary = {k: (v["median_hit_sweep"], round(v["median_time_to_target_s"], 4), v["hit_fraction"])
               for k, v in res.items() if isinstance(v, dict) and "median_hit_sweep" in v}
    print(summary)
    assert lrn["hit_fraction"] >= ada["hit_fraction"] - 1 / 32, summary
    assert lrn["median_hit_sweep"] <= 1.25 * ada["median_hit_sweep"], summary
    assert lrn["median_time_to_target_s"] < ada["median_time_to_target_s"], summary
    assert lrn["median_hit_sweep"] < geo["median_hit_sweep"], summary
