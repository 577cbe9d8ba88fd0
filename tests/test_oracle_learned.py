"""Pins for the oracle of the learned ladder and its judge (oracle/learned.py).

The composition's steps are each pinned elsewhere (pilot histograms,
features, the network, the adaptive ladder, resampling); these tests pin
what the composition adds: the monotone rule, the judge's pooled swap
acceptance against the exact acceptance by enumeration, the judge's
decisions on ladders whose acceptance the mathematics fixes near 0 or 1,
and the fallback switch.
"""
import math

import numpy as np
import pytest

from paper_2503_10302_gb300 import workloads as W
from tests import _exact as X


@pytest.fixture(scope="module")
def ol(orc):
    from oracle import learned
    return learned


def test_monotone_rule(ol):
    b = np.array([[-0.5, 0.2, 0.2, 0.1, 3.0],
                  [0.3, 0.3 + 1e-7, 0.9, 0.9 + 2e-6, 5.0]])
    got = ol.monotone(b)
    assert got[0].tolist() == [0.0, 0.2, 0.2 + 1e-6, 0.2 + 2e-6, 3.0]
    assert got[1].tolist() == [0.3, 0.3 + 1e-6, 0.9, 0.9 + 2e-6, 5.0]
    assert (np.diff(got, axis=1) > 0).all()
    inc = np.cumsum(np.full((3, 32), 0.05), axis=1)   # already increasing: unchanged
    assert np.array_equal(ol.monotone(inc), inc)


def test_judge_rate_equals_exact_acceptance(ol):
    """Pooled acceptance of a two-temperature ladder with two labels and ICM
    against E[min(1, exp(dbeta dE))] under the product Boltzmann measure,
    enumerated over the 256 states of a 2x2x2 lattice."""
    dims = (2, 2, 2)
    J = W.ea_couplings(dims, 52, 0)
    betas = np.array([0.3, 0.8])
    E = X.energies(X.lattice_edges(dims), J, None, X.all_states(8))
    p0, p1 = X.boltzmann(E, betas[0]), X.boltzmann(E, betas[1])
    dE = E[None, :] - E[:, None]
    exact = (p0[:, None] * p1[None, :] * np.minimum(1, np.exp((betas[1] - betas[0]) * dE))).sum()
    n = 16
    att, acc, rate, ok = ol.judge([dims] * n, [J] * n, [betas] * n, seed=3, n_labels=2, attempts=2000,
                                  floor=0.0)
    assert ok.all()
    assert (att[:, 0] == 2 * 1000).all()          # even attempts only, two labels
    pooled = acc.sum() / att.sum()
    assert abs(rate[0, 0] - acc[0, 0] / att[0, 0]) == 0
    se = math.sqrt(exact * (1 - exact) / att.sum())
    assert abs(pooled - exact) < 10 * se          # swaps are correlated in time: 10 naive sigmas


def test_judge_decisions_at_fixed_acceptance(ol):
    """A ladder with one enormous gap (beta 0.05 -> 8 on a 4^3 lattice) has
    an acceptance near 0 at that pair and fails any positive floor; a ladder
    packed into [0.5, 0.51] accepts nearly every swap and passes a floor of
    0.9; floor 0 passes everything and a floor above 1 fails everything."""
    dims = (4, 4, 4)
    J = [W.ea_couplings(dims, 53, i) for i in range(3)]
    gap = np.concatenate([np.linspace(0.02, 0.05, 16), np.linspace(8.0, 8.5, 16)])
    dense = np.linspace(0.5, 0.51, 32)
    ladders = [gap, dense, dense]
    att, acc, rate, ok = ol.judge([dims] * 3, J, ladders, seed=1, attempts=300, floor=0.9)
    assert not ok[0] and ok[1] and ok[2]
    assert rate[0, 15] < 0.01 and rate[1].min() > 0.9
    _, _, _, ok0 = ol.judge([dims] * 3, J, ladders, seed=1, attempts=300, floor=0.0)
    _, _, _, ok2 = ol.judge([dims] * 3, J, ladders, seed=1, attempts=300, floor=1.01)
    assert ok0.all() and not ok2.any()
    # a single attempt leaves the odd pairs unattempted: reported as -1, not judged
    _, _, r1, _ = ol.judge([dims], J[:1], [dense], seed=1, attempts=1, floor=0.0)
    assert (r1[0, 1::2] == -1).all() and (r1[0, 0::2] >= 0).all()


def test_learned_ladder_fallback_switch(ol):
    """Floor 0: the network's ladders are kept; a floor above 1: every
    instance falls back to its resampled adaptive ladder."""
    from oracle import mlp
    params = W.mlp_init(mlp.SIZES, 31)
    params = [(w * 0.5, b) for w, b in params]
    dims = [(4, 4, 4), (4, 4, 6)]
    J = [W.ea_couplings(d, 54, i) for i, d in enumerate(dims)]
    pb = W.geometric_ladder(4, 0.2, 3.0)
    kw = dict(n_chains=8, sweeps=60, tail=30, max_len=20)
    b0, r0, f0 = ol.learned_ladder(params, dims, J, pb, entry0=5, seed=2, pilot_sweeps=40, pilot_burn=20,
                                   probe_attempts=20, acc_floor=0.0, ladder_kw=kw)
    X_ = ol.features(dims, J, pb, 5, 2, 8, 40, 20)
    assert not f0.any() and np.array_equal(b0, ol.predict(params, X_))
    assert (np.diff(b0, axis=1) > 0).all()
    b1, _, f1 = ol.learned_ladder(params, dims, J, pb, entry0=5, seed=2, pilot_sweeps=40, pilot_burn=20,
                                  probe_attempts=20, acc_floor=1.5, ladder_kw=kw)
    assert f1.all()
    for i in range(2):
        assert np.array_equal(b1[i], ol.fallback(dims[i], J[i], 5 + i, 2, **kw))
