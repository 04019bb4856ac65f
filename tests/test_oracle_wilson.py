"""Pins for the oracle's gamma basis and Wilson operator (CPU only).

What pins what:
  * Clifford algebra and hermiticity fix the gamma matrices up to basis.
  * The free-field (U = 1) plane-wave spectrum in closed form fixes D, M,
    the time-boundary sign, M_hat and K_hat (a dropped term, a wrong sign or
    a transposed gamma changes the eigenvalues).
  * The adjoint dot-product test and gamma_5 hermiticity tie D^dag (coded as
    its own stencil) to D.
  * Gauge covariance ties the link placement (U(x) vs U(x-mu)^dag) down.
  * det M = det M_hat, densely on 2^4, ties the even-odd Schur complement to M.
"""
import numpy as np
import pytest

from oracle import lattice, wilson
from oracle.dirac import GAMMA, GAMMA5
from oracle.cg import dense_matrix, vdot
from paper_1702_00124_gb300 import synthetic


def test_clifford_algebra():
    eye = np.eye(4)
    for mu in range(4):
        assert np.allclose(GAMMA[mu], GAMMA[mu].conj().T)
        for nu in range(4):
            anti = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
            assert np.allclose(anti, 2 * eye * (mu == nu))
    assert np.allclose(GAMMA5, np.diag([1, 1, -1, -1]))


def _plane_wave(dims, n, u):
    lx, ly, lz, lt = dims
    p = np.array([2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz,
                  (2 * n[3] + 1) * np.pi / lt])
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx),
                             indexing="ij")
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return p, ph[..., None, None] * u[None, None, None, None]


def _unit_gauge(dims):
    U = np.zeros(lattice.shape(dims) + (4, 3, 3), dtype=np.complex128)
    U[...] = np.eye(3)
    return U


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 1), (3, 1, 1, 2)])
def test_free_field_M_closed_form(n):
    dims = (4, 4, 6, 8)
    rng = np.random.default_rng(1)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    kappa = 0.13
    p, f = _plane_wave(dims, n, u)
    Mp = (1 - 2 * kappa * np.cos(p).sum()) * np.eye(4) + 2j * kappa * sum(
        GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
    out = wilson.apply_M(_unit_gauge(dims), f, kappa)
    ref = np.einsum("st,...tc->...sc", Mp, f)
    assert np.max(np.abs(out - ref)) < 1e-13
    # K(p) = (1 - 2 kappa sum cos)^2 + 4 kappa^2 sum sin^2, times the identity
    Kp = Mp.conj().T @ Mp
    kclosed = (1 - 2 * kappa * np.cos(p).sum()) ** 2 + 4 * kappa ** 2 * np.sum(np.sin(p) ** 2)
    assert np.allclose(Kp, kclosed * np.eye(4), atol=1e-14)


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 2, 0, 3), (2, 1, 3, 0)])
def test_free_field_Mhat_spectrum(n):
    """On even plane waves M_hat = 1 - kappa^2 D(p)^2 with eigenvalues
    1 - kappa^2 (a -/+ i|b|)^2, a = 2 sum cos p, b = 2 sin p."""
    dims = (4, 4, 4, 8)
    kappa = 0.124
    p, _ = _plane_wave(dims, n, np.zeros((4, 3)))
    a = 2 * np.cos(p).sum()
    b = 2 * np.sin(p)
    nb = np.sqrt(np.sum(b ** 2))
    Dp = a * np.eye(4) - 1j * sum(GAMMA[mu] * b[mu] for mu in range(4))
    Mh = np.eye(4) - kappa ** 2 * Dp @ Dp
    ev = np.linalg.eigvals(Mh)
    closed = np.array([1 - kappa ** 2 * (a - 1j * nb) ** 2] * 2 +
                      [1 - kappa ** 2 * (a + 1j * nb) ** 2] * 2)
    # same multiset: every closed-form value matched by an eigenvalue, and vice versa
    assert np.max(np.min(np.abs(ev[:, None] - closed[None, :]), axis=1)) < 1e-12
    assert np.max(np.min(np.abs(closed[:, None] - ev[None, :]), axis=1)) < 1e-12
    U = _unit_gauge(dims)
    rng = np.random.default_rng(2)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    _, f = _plane_wave(dims, n, u)
    fe = lattice.mask(f, dims, 0)
    out = wilson.apply_Mhat(U, fe, kappa)
    ref = lattice.mask(np.einsum("st,...tc->...sc", Mh, f), dims, 0)
    assert np.max(np.abs(out - ref)) < 1e-13
    outK = wilson.apply_Khat(U, fe, kappa)
    refK = lattice.mask(np.einsum("st,...tc->...sc", Mh.conj().T @ Mh, f), dims, 0)
    assert np.max(np.abs(outK - refK)) < 1e-13


@pytest.fixture(scope="module")
def rand44():
    dims = (4, 4, 4, 4)
    U = synthetic.gauge_field(dims, 0.5, 11)
    psi = synthetic.spinor_field(dims, 12)
    chi = synthetic.spinor_field(dims, 13)
    return dims, U, psi, chi


def test_adjoint_dot_product(rand44):
    dims, U, psi, chi = rand44
    lhs = vdot(psi, wilson.hop(U, chi))
    rhs = vdot(wilson.hop(U, psi, dagger=True), chi)
    assert abs(lhs - rhs) < 1e-14 * abs(lhs) * 10
    k = 0.12
    lhs = vdot(psi, wilson.apply_M(U, chi, k))
    rhs = vdot(wilson.apply_M(U, psi, k, dagger=True), chi)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_gamma5_hermiticity(rand44):
    dims, U, psi, _ = rand44
    g5 = lambda v: np.einsum("st,...tc->...sc", GAMMA5, v)
    assert np.max(np.abs(wilson.hop(U, psi, dagger=True) - g5(wilson.hop(U, g5(psi))))) < 1e-13


def test_gauge_covariance(rand44):
    dims, U, psi, _ = rand44
    g = synthetic.gauge_field(dims, 1.0, 99)[..., 0, :, :]   # random SU(3) per site
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ lattice.shift(g, mu, +1).conj().swapaxes(-1, -2)
    G = lambda v: np.einsum("...ab,...sb->...sa", g, v)
    assert np.max(np.abs(wilson.hop(Ug, G(psi)) - G(wilson.hop(U, psi)))) < 1e-13


def test_two_site_direction_adds_both_hops():
    """On an L = 2 extent x+mu and x-mu coincide: both hops must be added."""
    dims = (2, 2, 2, 2)
    U = synthetic.gauge_field(dims, 0.7, 5)
    psi = synthetic.spinor_field(dims, 6)
    mat, _ = dense_matrix(lambda v: wilson.hop(U, v), np.ones(psi.shape, bool))
    # D is Hermitian up to gamma_5: D^dag = g5 D g5
    g5 = np.kron(np.eye(16), np.kron(GAMMA5, np.eye(3)))
    assert np.allclose(mat.conj().T, g5 @ mat @ g5, atol=1e-13)
    # each 12x12 block couples a site to its 4 distinct neighbours with
    # (1-g)U + (1+g)U'^dag: its rank is 12 (sum of two rank-6 pieces)
    blk = mat[:12, 12:24]          # site 0 -> site 1 (x-neighbour both ways)
    assert np.linalg.matrix_rank(blk, tol=1e-10) == 12


def test_det_M_equals_det_Mhat():
    dims = (2, 2, 2, 2)
    U = synthetic.gauge_field(dims, 0.6, 21)
    k = 0.11
    shp = lattice.shape(dims) + (4, 3)
    full, _ = dense_matrix(lambda v: wilson.apply_M(U, v, k), np.ones(shp, bool))
    ev = lattice.parity(dims) == 0
    sup = np.broadcast_to(ev[..., None, None], shp)
    half, _ = dense_matrix(lambda v: wilson.apply_Mhat(U, v, k), sup)
    s1, l1 = np.linalg.slogdet(full)
    s2, l2 = np.linalg.slogdet(half)
    assert abs(l1 - l2) < 1e-12 and abs(s1 - s2) < 1e-12
