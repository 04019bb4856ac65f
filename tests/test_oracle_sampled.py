"""Pin the oracle's sampled-site Wilson operator (index-based) to the
whole-lattice one (shift-based) on small lattices, including the time
boundary and an L = 2 extent (CPU only)."""
import numpy as np
import pytest

from oracle import lattice, sampled, wilson
from paper_1702_00124_gb300 import synthetic


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 10)])
@pytest.mark.parametrize("dagger", [False, True])
def test_hop_at_matches_full(dims, dagger):
    U = synthetic.gauge_field(dims, 0.6, 61)
    f = synthetic.spinor_field(dims, 62)
    ref = wilson.hop(U, f, dagger=dagger).reshape(-1, 4, 3)
    idx = np.arange(int(np.prod(dims)))
    assert np.max(np.abs(sampled.hop_at(U, f, idx, dagger) - ref)) < 1e-13


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 6, 10)])
def test_khat_at_matches_full(dims):
    U = synthetic.gauge_field(dims, 0.5, 63)
    f = lattice.mask(synthetic.spinor_field(dims, 64), dims, 0)
    ref = wilson.apply_Khat(U, f, 0.13).reshape(-1, 4, 3)
    par = lattice.parity(dims).reshape(-1)
    idx = np.flatnonzero(par == 0)[::3]
    assert np.max(np.abs(sampled.khat_at(U, f, 0.13, idx) - ref[idx])) < 1e-12
