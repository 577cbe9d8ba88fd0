"""The C-ABI library builds, loads without a GPU and exports every symbol
that include/pcomp.h declares; host-side table builders agree with the
oracle's (each side has its own code)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pcomp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def so():
    from paper_2503_10302_gb300 import build
    build.build()
    from paper_2503_10302_gb300 import pcomp
    return pcomp.lib()


def test_every_declared_symbol_is_exported(so):
    names = _declared()
    assert len(names) > 20
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2503_10302_gb300 import pcomp
    assert set(_declared()) == set(pcomp.SIGNATURES)


def test_host_thresholds_equal_oracle(so, orc):
    from paper_2503_10302_gb300 import pcomp
    for beta in (0.2, 0.3125, 0.77, 1.5, 3.0):
        for I in range(-6, 7):
            assert pcomp.pc_pbit_threshold(beta, I) == orc.pbit_threshold(beta, I)
    for db in (0.013, 0.1, 0.37):
        for dE in range(-400, 0, 2):
            assert pcomp.pc_swap_threshold(db, dE) == orc.swap_threshold(db, dE)
    for g in np.linspace(3.0, 1e-3, 101):
        for (P, T) in ((64, 0.05), (16, 0.2), (32, 1.0)):
            assert pcomp.pc_jperp_q(g, P, T) == orc.jperp_q(g, P, T)


def test_no_gpu_errors_are_reported_not_raised(so):
    """Without a GPU pc_create fails with a status, never aborts."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2503_10302_gb300 import pcomp
    with pytest.raises(pcomp.PcompError):
        pcomp.pc_create(0, 0)
