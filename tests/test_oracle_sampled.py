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


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 10)])
def test_dre_ydx_at_matches_full(dims):
    """The per-link force derivative (explicit neighbour indices, one link at a
    time) against the whole-lattice one (shifts), at every link of the lattice,
    time-boundary links included; the latter is pinned by finite differences."""
    from oracle import force
    U = synthetic.gauge_field(dims, 0.6, 65)
    X = synthetic.spinor_field(dims, 66)
    Y = synthetic.spinor_field(dims, 67)
    ref = force.dre_ydx(U, Y, X).reshape(-1, 4, 8)
    V = int(np.prod(dims))
    idx = np.repeat(np.arange(V), 4)
    mu = np.tile(np.arange(4), V)
    got = sampled.dre_ydx_at(U, Y, X, idx, mu)
    assert np.max(np.abs(got - ref[idx, mu])) < 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 6, 10)])
def test_xy_force_at_matches_full(dims):
    """The PLAIN and HASENBUSCH force from given X, Y (and phi) at sampled links
    against the oracle's whole-lattice form -2 dRe(Y^dag M_hat X) [+ 2 dRe(phi^dag M_h X)]."""
    from oracle import force
    U = synthetic.gauge_field(dims, 0.5, 68)
    X = lattice.mask(synthetic.spinor_field(dims, 69), dims, 0)
    Y = lattice.mask(synthetic.spinor_field(dims, 70), dims, 0)
    phi = lattice.mask(synthetic.spinor_field(dims, 71), dims, 0)
    k, kh = 0.13, 0.12
    plain = (-2 * force._dre_mhat(U, Y, X, k)).reshape(-1, 4, 8)
    hasen = plain + (2 * force._dre_mhat(U, phi, X, kh)).reshape(-1, 4, 8)
    rng = np.random.default_rng(3)
    V = int(np.prod(dims))
    idx = rng.choice(V, 64, replace=False)
    mu = rng.integers(0, 4, 64)
    got = sampled.xy_force_at(U, X, Y, k, idx, mu)
    assert np.max(np.abs(got - plain[idx, mu])) < 1e-13 * np.max(np.abs(plain))
    got = sampled.xy_force_at(U, X, Y, k, idx, mu, phi_e=phi, kappa_h=kh)
    assert np.max(np.abs(got - hasen[idx, mu])) < 1e-13 * np.max(np.abs(hasen))
