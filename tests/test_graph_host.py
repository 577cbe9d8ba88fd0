"""Host logic of the general-graph path, without a GPU: the library's DSATUR
(its own C++ with an ordered set) colours exactly like the oracle's plain
O(n^2) restatement, and malformed graphs are refused."""
import itertools

import numpy as np
import pytest

from paper_2503_10302_gb300 import workloads as W


@pytest.fixture(scope="module")
def pc():
    from paper_2503_10302_gb300 import build, pcomp
    build.build()
    return pcomp


def _graphs():
    out = [W.csr_from_edges(5, [(i, (i + 1) % 5) for i in range(5)]),
           W.csr_from_edges(6, list(itertools.combinations(range(6), 2))),
           W.csr_from_edges(4, [])]
    for seed in range(30):
        out.append(W.random_graph(20 + 13 * seed, 1.5 + (seed % 6), seed, wmax=3))
    for L in (4, 6):
        out.append(W.dimer_embedding((L, L, L), W.ea_couplings((L, L, L), 1000)))
    for dims in [(5, 5, 4), (3, 3, 3), (8, 8, 8)]:
        out.append(W.lattice_graph(dims, (1, 1, 1), W.ea_couplings(dims, 1000))[0])
    pres = W.random_vacancies((6, 6, 6), 0.2, 3)
    out.append(W.lattice_graph((6, 6, 6), (0, 1, 1), W.ea_couplings((6, 6, 6), 1000), pres)[0])
    return out


def test_library_dsatur_equals_oracle(pc, orc):
    for g in _graphs():
        c1, C1 = pc.pc_graph_dsatur(g.rp, g.col)
        c2, C2 = orc.dsatur(g.rp, g.col)
        assert C1 == C2 and np.array_equal(c1, c2)


def test_library_refuses_malformed_graphs(pc):
    bad = [([0, 1, 1], [1]),                    # one direction only
           ([0, 1, 2], [0, 1]),                 # self-loops
           ([0, 2, 4], [1, 1, 0, 0]),           # repeated neighbour
           ([1, 1, 2], [1, 0])]                 # row_ptr[0] != 0
    for rp, col in bad:
        with pytest.raises(RuntimeError):
            pc.pc_graph_dsatur(rp, col)
    # K_33 needs 33 colours, one more than the library holds
    g = W.csr_from_edges(33, list(itertools.combinations(range(33), 2)))
    with pytest.raises(RuntimeError):
        pc.pc_graph_dsatur(g.rp, g.col)
