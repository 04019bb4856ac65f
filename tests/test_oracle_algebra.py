"""Pins for the oracle's SU(3) helpers, CG, Chebyshev filter and RNG (CPU only).

  * expm is checked against scipy.linalg.expm (a library routine); the
    generators against tr(T_a T_b) = delta_ab / 2 and the su(3) structure
    [T_1, T_2] = i T_3.
  * CG is checked against a dense LU solve on a 2^4 lattice.
  * The filter's root product is checked against the closed form
    (1 - R(x)) / x built from numpy's Chebyshev basis, its minimax error
    bound, its positivity for even degree, the root-subset property that
    makes Q = P_2 / P_1 a polynomial for the paper's orders, and, as an
    operator, against the free-field eigenvalues of K_hat.
  * Philox4x64-10 is checked against numpy's Philox bit generator; the
    Gaussian draws against their first moments.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import lattice, su3, wilson, philox
from oracle.cg import cg, dense_matrix
from oracle.poly import ChebyshevFilter
from paper_1702_00124_gb300 import synthetic


def test_generators():
    T = su3.T
    for a in range(8):
        for b in range(8):
            assert abs(np.trace(T[a] @ T[b]) - 0.5 * (a == b)) < 1e-15
        assert abs(np.trace(T[a])) < 1e-15
        assert np.allclose(T[a], T[a].conj().T)
    assert np.allclose(T[0] @ T[1] - T[1] @ T[0], 1j * T[2])
    p = np.random.default_rng(0).standard_normal((5, 8))
    assert np.allclose(su3.matrix_to_alg(su3.alg_to_matrix(p)), p)


def test_expm_against_scipy():
    rng = np.random.default_rng(3)
    for scale in (0.01, 0.7, 3.0, 12.0):
        p = rng.standard_normal((20, 8)) * scale
        A = 1j * su3.alg_to_matrix(p)
        ref = np.stack([scipy.linalg.expm(a) for a in A])
        out = su3.expm(A)
        assert np.max(np.abs(out - ref)) < 1e-13 * max(1.0, scale)
        assert np.allclose(np.linalg.det(out), 1.0, atol=1e-12)


def test_reunitarize():
    U = synthetic.gauge_field((2, 2, 2, 2), 0.8, 7)
    V = su3.reunitarize(U)
    assert np.max(np.abs(V - U)) < 1e-14          # identity on SU(3)
    W = su3.reunitarize(U + 1e-3 * np.random.default_rng(1).standard_normal(U.shape))
    eye = np.eye(3)
    assert np.max(np.abs(W @ su3.dagger(W) - eye)) < 1e-14
    assert np.max(np.abs(np.linalg.det(W) - 1)) < 1e-14


def test_cg_against_dense_solve():
    dims = (2, 2, 2, 2)
    U = synthetic.gauge_field(dims, 0.5, 31)
    k = 0.12
    shp = lattice.shape(dims) + (4, 3)
    sup = np.broadcast_to((lattice.parity(dims) == 0)[..., None, None], shp)
    K = lambda v: wilson.apply_Khat(U, v, k)
    mat, idx = dense_matrix(K, sup)
    b = lattice.mask(synthetic.spinor_field(dims, 32), dims, 0)
    x, info = cg(K, b, 1e-13)
    ref = np.linalg.solve(mat, b.reshape(-1)[idx])
    assert info["rel_resid"] <= 1e-13
    assert np.linalg.norm(x.reshape(-1)[idx] - ref) / np.linalg.norm(ref) < 1e-11
    assert np.allclose(mat, mat.conj().T, atol=1e-14)     # K_hat Hermitian
    assert np.min(np.linalg.eigvalsh(mat)) > 0


@pytest.mark.parametrize("n,eps,lam", [(4, 0.005, 8.0), (16, 0.005, 8.0), (24, 0.005, 8.0),
                                       (10, 0.05, 5.0)])
def test_filter_closed_form(n, eps, lam):
    p = ChebyshevFilter(n, eps, lam)
    x = np.concatenate([np.linspace(eps, lam, 257), [1e-4, 0.001, 9.0, 20.0]])
    prod = p.value_product(x)
    closed = p.value(x)
    assert np.max(np.abs(prod.imag)) < 1e-9 * np.max(np.abs(closed))
    assert np.max(np.abs(prod.real - closed) / np.abs(closed)) < 1e-10
    xin = np.linspace(eps, lam, 2001)
    err = np.max(np.abs(1 - xin * p.value(xin)))
    assert err <= p.error_bound() * (1 + 1e-9)
    assert err >= p.error_bound() * (1 - 1e-6)      # equioscillation reaches the bound
    assert np.all(p.value(np.linspace(1e-6, 50, 5001)) > 0)   # even degree: positive
    # roots come in conjugate pairs: z_k = conj(z_{n+1-k})
    z = p.roots()
    assert np.max(np.abs(z - z[::-1].conj())) < 1e-12


@pytest.mark.parametrize("p1,p2", [(4, 24), (4, 34), (4, 54), (4, 20)])
def test_root_subset_for_ratio_filter(p1, p2):
    """Q = P_2 / P_1 is a polynomial iff the roots of P_1 are roots of P_2; with
    t_k = 2 pi k/(n+1) that holds when (p1 + 1) divides (p2 + 1)."""
    a = ChebyshevFilter(p1, 0.005, 8.0).roots()
    b = ChebyshevFilter(p2, 0.005, 8.0).roots()
    contained = all(np.min(np.abs(b - z)) < 1e-12 for z in a)
    assert contained == ((p2 + 1) % (p1 + 1) == 0)


@pytest.mark.parametrize("lo,hi", [(4, 24), (4, 54), (2, 8)])
def test_ratio_filter_is_polynomial(lo, hi):
    """Q = P_hi / P_lo (Section 3.3): the root product of the leftover roots equals
    the ratio of the two closed forms, and its roots come in conjugate pairs."""
    from oracle.poly import RatioFilter
    q = RatioFilter(ChebyshevFilter(hi, 0.005, 8.0), ChebyshevFilter(lo, 0.005, 8.0))
    assert q.n == hi - lo
    x = np.concatenate([np.linspace(0.005, 8.0, 101), [0.001, 12.0]])
    closed = q.value(x)
    prod = q.value_product(x)
    assert np.max(np.abs(prod.imag)) < 1e-9 * np.max(np.abs(closed))
    assert np.max(np.abs(prod.real - closed) / np.abs(closed)) < 1e-9
    z = q.roots()
    assert np.max([np.min(np.abs(z - w.conj())) for w in z]) < 1e-12
    # as an operator: a diagonal "K" gives the scalar values
    assert np.allclose(q.apply(lambda v: x * v, np.ones_like(x)), closed, rtol=1e-10)


def test_filter_on_free_field_modes():
    dims = (4, 4, 4, 8)
    kappa = 0.12
    U = np.zeros(lattice.shape(dims) + (4, 3, 3), dtype=np.complex128)
    U[...] = np.eye(3)
    pf = ChebyshevFilter(8, 0.01, 4.0)
    n = (1, 2, 1, 1)
    p = np.array([2 * np.pi * n[0] / 4, 2 * np.pi * n[1] / 4, 2 * np.pi * n[2] / 4,
                  (2 * n[3] + 1) * np.pi / 8])
    a = 2 * np.cos(p).sum()
    nb = 2 * np.sqrt(np.sum(np.sin(p) ** 2))
    lamK = abs(1 - kappa ** 2 * (a - 1j * nb) ** 2) ** 2   # both K eigenvalues coincide
    t, z, y, x = np.meshgrid(*[np.arange(s) for s in lattice.shape(dims)], indexing="ij")
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    # a K_hat eigenvector: even plane wave with spinor in the |b| eigenspace of g.b
    from oracle.dirac import GAMMA
    gb = sum(GAMMA[mu] * 2 * np.sin(p[mu]) for mu in range(4))
    w, v = np.linalg.eigh(gb)
    u = np.outer(v[:, -1], np.array([1.0, 0.5j, -0.25]))
    f = lattice.mask(ph[..., None, None] * u, dims, 0)
    K = lambda vv: wilson.apply_Khat(U, vv, kappa)
    assert np.max(np.abs(K(f) - lamK * f)) < 1e-12
    out = pf.apply(K, f)
    assert np.max(np.abs(out - pf.value(lamK) * f)) < 1e-11 * abs(pf.value(lamK))


def test_philox_matches_numpy():
    key, stream = 12345, 7
    bg = np.random.Philox(key=np.array([key, 0], dtype=np.uint64),
                          counter=np.array([0, stream, 0, 0], dtype=np.uint64))
    raw = bg.random_raw(40).reshape(10, 4)       # blocks with counters 1..10
    j = np.arange(1, 11, dtype=np.uint64)
    z = np.zeros(10, dtype=np.uint64)
    mine = np.stack(philox.philox4x64_10(j, np.full(10, stream, np.uint64), z, z,
                                         np.uint64(key), np.uint64(0)), axis=1)
    assert np.array_equal(mine, raw)


def test_gaussian_moments():
    g = philox.gaussian_field(400_000, 99, 3)
    assert abs(g.mean()) < 0.01
    assert abs(g.var() - 1) < 0.01
    assert abs(np.mean(g ** 4) - 3) < 0.05
    g2 = philox.gaussian_field(400_000, 99, 4)
    assert abs(np.mean(g * g2)) < 0.01
