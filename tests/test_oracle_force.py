"""Pins for the oracle's actions, heat bath and forces (CPU only).

  * Heat bath: S(phi(chi)) = chi^dag chi for every term kind (the action and
    the heat bath are computed by different routes).
  * Determinant identities of mass preconditioning and polynomial filtering
    (Section 2, Sections 3.3 and 4.1-4.2): the Gaussian integrals of the PF-MP,
    2PF, 2MP and 1PF-2MP terms multiply to det K_hat, checked densely on 2^4.
  * Gauge invariance of every action term under random SU(3) transforms.
  * Forces: central finite differences of the actions in extended precision
    (long double, solves to 1e-18), step 1e-5, on links that include the
    antiperiodic time boundary; tolerance 1e-9 relative.
"""
import numpy as np
import pytest

from oracle import lattice, su3, wilson, actions, force
from oracle.cg import dense_matrix, vdot
from oracle.poly import ChebyshevFilter
from paper_1702_00124_gb300 import synthetic

LD = np.clongdouble


def _terms(kappa, kappa_h, n=4):
    from oracle.poly import RatioFilter
    pf = ChebyshevFilter(n, 0.05, 5.0)
    q = RatioFilter(ChebyshevFilter(8, 0.05, 5.0), ChebyshevFilter(2, 0.05, 5.0))
    return [actions.term("plain", kappa),
            actions.term("hasenbusch", kappa, kappa_h),
            actions.term("poly", kappa_h, poly=pf),
            actions.term("filtered", kappa_h, poly=pf),
            actions.term("ratio", kappa_h, poly=q)]


@pytest.fixture(scope="module")
def setup44():
    dims = (4, 4, 4, 4)
    U = synthetic.gauge_field(dims, 0.5, 41)
    chi = lattice.mask(synthetic.spinor_field(dims, 42), dims, 0)
    return dims, U, chi


@pytest.mark.parametrize("i", range(5))
def test_heatbath_gives_chi_norm(setup44, i):
    dims, U, chi = setup44
    t = _terms(0.125, 0.115)[i]
    phi = actions.heatbath(U, t, chi)
    S, _ = actions.action(U, t, phi)
    assert abs(S - vdot(chi, chi).real) < 1e-10 * vdot(chi, chi).real


@pytest.mark.parametrize("i", range(5))
def test_gauge_invariance(setup44, i):
    dims, U, chi = setup44
    t = _terms(0.125, 0.115)[i]
    g = synthetic.gauge_field(dims, 1.0, 77)[..., 1, :, :]
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ su3.dagger(lattice.shift(g, mu, +1))
    phi = chi
    phig = np.einsum("...ab,...sb->...sa", g, phi)
    S1, _ = actions.action(U, t, phi)
    S2, _ = actions.action(Ug, t, phig)
    assert abs(S1 - S2) < 1e-11 * abs(S1)


def test_pfmp_determinant_identity():
    """det P(J)^-1 . det(P(J) J) . det(J K^-1)^-1 ... = det K_hat (PF-MP, Section 4.1):
    the Gaussian integral of exp(-phi^dag A phi) is proportional to det A^-1."""
    dims = (2, 2, 2, 2)
    U = synthetic.gauge_field(dims, 0.6, 51)
    k, kh = 0.12, 0.10
    pf = ChebyshevFilter(6, 0.02, 6.0)
    shp = lattice.shape(dims) + (4, 3)
    sup = np.broadcast_to((lattice.parity(dims) == 0)[..., None, None], shp)
    D = lambda op: dense_matrix(op, sup)[0]
    K = D(lambda v: wilson.apply_Khat(U, v, k))
    J = D(lambda v: wilson.apply_Khat(U, v, kh))
    Mh = D(lambda v: wilson.apply_Mhat(U, v, kh))
    PJ = D(lambda v: pf.apply(lambda w: wilson.apply_Khat(U, w, kh), v))
    A_poly = PJ
    A_filt = np.linalg.inv(PJ @ J)
    A_hb = Mh @ np.linalg.inv(K) @ Mh.conj().T
    logdet = lambda A: np.linalg.slogdet(A)[1]
    lhs = -(logdet(A_poly) + logdet(A_filt) + logdet(A_hb))
    assert abs(lhs - logdet(K)) < 1e-9 * abs(logdet(K))
    # the dense P(J) matches the filter's scalar closed form on J's eigenvalues
    w, v = np.linalg.eigh(J)
    assert np.allclose(PJ, (v * pf.value(w)) @ v.conj().T, atol=1e-10 * np.abs(PJ).max())


def test_2pf_determinant_identity():
    """2PF (Section 3.3): det P_1^-1 . det Q^-1 . det(P_2 K) = det K with Q = P_2 / P_1."""
    from oracle.poly import RatioFilter
    dims = (2, 2, 2, 2)
    U = synthetic.gauge_field(dims, 0.6, 52)
    k = 0.12
    p1, p2 = ChebyshevFilter(2, 0.02, 6.0), ChebyshevFilter(8, 0.02, 6.0)
    q = RatioFilter(p2, p1)
    shp = lattice.shape(dims) + (4, 3)
    sup = np.broadcast_to((lattice.parity(dims) == 0)[..., None, None], shp)
    D = lambda op: dense_matrix(op, sup)[0]
    Kop = lambda w: wilson.apply_Khat(U, w, k)
    K = D(Kop)
    P1 = D(lambda v: p1.apply(Kop, v))
    Q = D(lambda v: q.apply(Kop, v))
    P2K = D(lambda v: p2.apply(Kop, Kop(v)))
    logdet = lambda A: np.linalg.slogdet(A)[1]
    lhs = -(logdet(P1) + logdet(Q) - logdet(P2K))
    assert abs(lhs - logdet(K)) < 1e-9 * abs(logdet(K))
    assert np.allclose(P1 @ Q, D(lambda v: p2.apply(Kop, v)), atol=1e-9 * np.abs(P1 @ Q).max())


@pytest.mark.parametrize("with_filter", [False, True], ids=["2MP", "1PF-2MP"])
def test_two_mass_determinant_identity(with_filter):
    """2MP (Section 3.3) and 1PF-2MP (Section 4.2) with kappa_1 < kappa_2 < kappa:
    J_1^-1 (or P(J_1) and [P(J_1) J_1]^-1), M_1 J_2^-1 M_1^dag and M_2 K^-1 M_2^dag,
    the Hermitian reading of "J_1 J_2^-1" and "J_2 K^-1"; their Gaussian integrals
    multiply to det K_hat."""
    dims = (2, 2, 2, 2)
    U = synthetic.gauge_field(dims, 0.6, 53)
    k, k2, k1 = 0.125, 0.115, 0.10
    pf = ChebyshevFilter(4, 0.02, 6.0)
    shp = lattice.shape(dims) + (4, 3)
    sup = np.broadcast_to((lattice.parity(dims) == 0)[..., None, None], shp)
    D = lambda op: dense_matrix(op, sup)[0]
    K = D(lambda v: wilson.apply_Khat(U, v, k))
    J1 = D(lambda v: wilson.apply_Khat(U, v, k1))
    J2 = D(lambda v: wilson.apply_Khat(U, v, k2))
    M1 = D(lambda v: wilson.apply_Mhat(U, v, k1))
    M2 = D(lambda v: wilson.apply_Mhat(U, v, k2))
    if with_filter:
        PJ = D(lambda v: pf.apply(lambda w: wilson.apply_Khat(U, w, k1), v))
        first = [PJ, np.linalg.inv(PJ @ J1)]
    else:
        first = [np.linalg.inv(J1)]
    forms = first + [M1 @ np.linalg.inv(J2) @ M1.conj().T, M2 @ np.linalg.inv(K) @ M2.conj().T]
    logdet = lambda A: np.linalg.slogdet(A)[1]
    lhs = -sum(logdet(A) for A in forms)
    assert abs(lhs - logdet(K)) < 1e-9 * abs(logdet(K))
    # the oracle's hasenbusch term evaluates the same quadratic form
    phi = lattice.mask(synthetic.spinor_field(dims, 54), dims, 0)
    v = phi.reshape(-1)[dense_matrix(lambda x: x, sup)[1]]
    S, _ = actions.action(U, actions.term("hasenbusch", k2, k1), phi, tol=1e-14)
    assert abs(S - np.vdot(v, forms[-2] @ v).real) < 1e-10 * abs(S)


def _fd_check(U, action_of_U, F, links, h=1e-5, rtol=1e-9):
    ULD = U.astype(LD)
    T = su3.generators(LD)
    scale = np.sqrt(np.mean(F.astype(np.float64) ** 2))
    for (t, z, y, x, mu, a) in links:
        vals = []
        for s in (+1, -1):
            V = ULD.copy()
            R = su3.expm(1j * LD(s * h) * T[a])
            V[t, z, y, x, mu] = R @ V[t, z, y, x, mu]
            vals.append(action_of_U(V))
        fd = np.real(vals[0] - vals[1]) / (2 * LD(h))
        f = F[t, z, y, x, mu, a]
        assert abs(float(fd) - float(f)) <= rtol * max(abs(float(fd)), scale), \
            (t, z, y, x, mu, a, float(fd), float(f))


def _links(dims, n, seed):
    rng = np.random.default_rng(seed)
    lt = dims[3]
    out = [(lt - 1, 0, 1, 0, 3, 2), (lt - 1, 1, 0, 1, 3, 7), (0, 1, 1, 0, 0, 0)]
    for _ in range(n):
        out.append((int(rng.integers(dims[3])), int(rng.integers(dims[2])),
                    int(rng.integers(dims[1])), int(rng.integers(dims[0])),
                    int(rng.integers(4)), int(rng.integers(8))))
    return out


@pytest.mark.parametrize("i", range(5))
def test_fermion_force_finite_difference(i):
    dims = (2, 2, 2, 4)
    U = synthetic.gauge_field(dims, 0.5, 61)
    chi = lattice.mask(synthetic.spinor_field(dims, 62), dims, 0)
    t = _terms(0.125, 0.11)[i]
    F = force.fermion_force(U.astype(LD), t, chi.astype(LD), tol=1e-18)
    act = lambda V: actions.action(V, t, chi.astype(LD), tol=1e-18)[0]
    _fd_check(U, act, F, _links(dims, 4, i))


def test_plain_force_finite_difference_4444():
    dims = (4, 4, 4, 4)
    U = synthetic.gauge_field(dims, 0.5, 71)
    chi = lattice.mask(synthetic.spinor_field(dims, 72), dims, 0)
    t = actions.term("plain", 0.12)
    F = force.fermion_force(U.astype(LD), t, chi.astype(LD), tol=1e-18)
    act = lambda V: actions.action(V, t, chi.astype(LD), tol=1e-18)[0]
    _fd_check(U, act, F, _links(dims, 2, 5))


def test_gauge_force_finite_difference():
    dims = (2, 2, 4, 4)
    U = synthetic.gauge_field(dims, 0.7, 81)
    F = force.gauge_force(U.astype(LD), 5.6)
    _fd_check(U, lambda V: force.gauge_action(V, 5.6), F, _links(dims, 6, 9))


def test_gauge_action_closed_form():
    """U = 1 gives S_G = 0.  x-links U_x = exp(i th y D), D = diag(1,-1,0), others 1:
    (x,y) plaquettes are exp(-i th D) except the wrapped row, which carries
    exp(i th (Ly-1) D); every other plane is trivial."""
    dims = (2, 4, 2, 2)
    U = np.zeros(lattice.shape(dims) + (4, 3, 3), dtype=np.complex128)
    U[...] = np.eye(3)
    assert abs(force.gauge_action(U, 5.6)) < 1e-12
    th, ly = 0.3, dims[1]
    d = np.array([1.0, -1.0, 0.0])
    for y in range(ly):
        U[:, :, y, :, 0] = np.diag(np.exp(1j * th * y * d))
    vol = int(np.prod(dims))
    per = lambda a: (2.0 / 3.0) * (1 - np.cos(a))
    closed = 5.6 * vol / ly * ((ly - 1) * per(th) + per((ly - 1) * th))
    assert abs(force.gauge_action(U, 5.6) - closed) < 1e-12 * closed
