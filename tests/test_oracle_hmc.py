"""Pins for the oracle's integrators, Hamiltonian and Metropolis test (CPU only).

  * The generalised multi-scale scheme reproduces the worked example printed
    in Section 3.2 (tests/golden/generalised_scheme_example.txt).
  * Reversibility: forward, flip P, forward again returns to the start.
  * Energy conservation of a second-order integrator: halving the step
    divides |dH| by about 4 (ratio in [3, 5]) for leapfrog and Omelyan 2MN;
    a wrong force sign or normalisation breaks this (dH would not vanish).
  * T[eps] keeps links in SU(3).
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import lattice, hmc, actions, force, su3
from paper_1702_00124_gb300 import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "generalised_scheme_example.txt")


def _read_golden():
    ops = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        if f[0] == "T":
            ops.append(("T", Fraction(f[1])))
        else:
            ops.append(("S", int(f[1]), Fraction(f[2])))
    return ops


def test_generalised_scheme_printed_example():
    tau = 1.0
    I1 = hmc.merge_adjacent(hmc.leapfrog(2, tau, 1))
    I2 = hmc.merge_adjacent(hmc.leapfrog(3, tau, 2))
    ops = hmc.generalised([I1, I2], tau)
    want = _read_golden()
    assert len(ops) == len(want)
    for a, b in zip(ops, want):
        assert a[0] == b[0]
        if a[0] == "T":
            assert abs(a[1] - float(b[1])) < 1e-12
        else:
            assert a[1] == b[1] and abs(a[2] - float(b[2])) < 1e-12


def test_nested_structure():
    """I_nested: S_1[h1/2] (S_2[h2/2] T[h2] S_2[h2/2])^m S_1[h1/2], h2 = h1/m."""
    ops = hmc.nested([(0, 2), (1, 3)], 1.0)
    h1 = 0.5
    h2 = h1 / 3
    step = [("S", 0, h1 / 2)] + [("S", 1, h2 / 2), ("T", h2), ("S", 1, h2 / 2)] * 3 + [("S", 0, h1 / 2)]
    assert len(ops) == 2 * len(step)
    for a, b in zip(ops, step * 2):
        assert a[0] == b[0] and abs(a[-1] - b[-1]) < 1e-15
    assert abs(sum(o[1] for o in ops if o[0] == "T") - 1.0) < 1e-14


@pytest.fixture(scope="module")
def md_setup():
    dims = (4, 4, 4, 4)
    U = synthetic.gauge_field(dims, 0.3, 91)
    P = synthetic.momenta(dims, 92)
    chi = lattice.mask(synthetic.spinor_field(dims, 93), dims, 0)
    beta = 5.6
    t = actions.term("plain", 0.12)
    phi = actions.heatbath(U, t, chi)

    def H(U_, P_):
        return hmc.kinetic(P_) + force.gauge_action(U_, beta) + actions.action(U_, t, phi)[0]

    def forces(g, U_):
        return force.gauge_force(U_, beta) if g == 0 else force.fermion_force(U_, t, phi)

    return U, P, H, forces


def _run(md_setup, ops):
    U, P, H, forces = md_setup
    U1, P1 = hmc.integrate(U, P, ops, forces)
    return H(U1, P1) - H(U, P), U1, P1


@pytest.mark.parametrize("kind", ["leapfrog", "omelyan"])
def test_dH_scales_as_eps_squared(md_setup, kind):
    tau = 0.25
    dh = []
    for n in (2, 4):
        ops = hmc.nested([(1, n), (0, 2)], tau, kind)
        dh.append(abs(_run(md_setup, ops)[0]))
    ratio = dh[0] / dh[1]
    assert 3.0 <= ratio <= 5.0, (dh, ratio)


def test_reversibility(md_setup):
    U, P, H, forces = md_setup
    ops = hmc.nested([(1, 3), (0, 2)], 0.3, "omelyan")
    U1, P1 = hmc.integrate(U, P, ops, forces)
    U2, P2 = hmc.integrate(U1, -P1, ops, forces)
    assert np.max(np.abs(U2 - U)) < 1e-10
    assert np.max(np.abs(-P2 - P)) < 1e-9
    eye = np.eye(3)
    assert np.max(np.abs(U1 @ su3.dagger(U1) - eye)) < 1e-14


@pytest.mark.parametrize("kind", ["leapfrog", "omelyan"])
def test_generalised_scheme_reversible(md_setup, kind):
    """Section 3.2's overlay with step counts whose events coincide in time (2 and 4
    steps): the list of operations is not a palindrome at the ties, but coincident S
    steps commute, so integrating back with -P returns to the start."""
    U, P, H, forces = md_setup
    mk = hmc.leapfrog if kind == "leapfrog" else hmc.omelyan
    ops = hmc.generalised([mk(2, 0.3, 1), mk(4, 0.3, 0)], 0.3)
    U1, P1 = hmc.integrate(U, P, ops, forces)
    U2, P2 = hmc.integrate(U1, -P1, ops, forces)
    assert np.max(np.abs(U2 - U)) < 1e-10
    assert np.max(np.abs(-P2 - P)) < 1e-9


def test_metropolis():
    assert hmc.metropolis(-0.1, 0.999)
    assert hmc.metropolis(0.5, 0.5)          # exp(-0.5) = 0.607 > 0.5
    assert not hmc.metropolis(0.5, 0.61)
