"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the method: it only draws the random
numbers that make up a workload and lays them out in the canonical host
formats below.  Both the oracle (``oracle/``) and the CUDA path read its
output; neither computes anything here.

Canonical host layouts (``dims = (Lx, Ly, Lz, Lt)``, arrays indexed
``[t, z, y, x, ...]``, direction index mu = 0..3 for x, y, z, t):

* gauge field  ``U[t,z,y,x,mu,a,b]``  complex128, SU(3) link U_mu(x)
* spinor       ``psi[t,z,y,x,s,c]``   complex128, spin s = 0..3, colour c = 0..2
* algebra      ``P[t,z,y,x,mu,k]``    float64, coordinates of P = sum_k P_k T_k
                                       with T_k = lambda_k / 2 (Gell-Mann)

Gauge links follow the recipe U = exp(i a H), H = sum_k h_k lambda_k/2 with
h_k ~ N(0,1) per link (a Gaussian traceless Hermitian matrix); the matrix
exponential is numpy's Hermitian eigendecomposition.  Spinors have N(0,1)
real and imaginary parts; momenta N(0,1) per algebra coordinate, i.e.
P ~ exp(-sum tr P^2) as in Section 2 of the paper.  Seeds are
170200124 + workload index.
"""
import numpy as np

SEED_BASE = 170200124

# Gell-Mann matrices: the basis in which H and the momenta are drawn.
_LAMBDA = np.zeros((8, 3, 3), dtype=np.complex128)
_LAMBDA[0][0, 1] = _LAMBDA[0][1, 0] = 1
_LAMBDA[1][0, 1], _LAMBDA[1][1, 0] = -1j, 1j
_LAMBDA[2][0, 0], _LAMBDA[2][1, 1] = 1, -1
_LAMBDA[3][0, 2] = _LAMBDA[3][2, 0] = 1
_LAMBDA[4][0, 2], _LAMBDA[4][2, 0] = -1j, 1j
_LAMBDA[5][1, 2] = _LAMBDA[5][2, 1] = 1
_LAMBDA[6][1, 2], _LAMBDA[6][2, 1] = -1j, 1j
_LAMBDA[7][0, 0] = _LAMBDA[7][1, 1] = 1 / np.sqrt(3)
_LAMBDA[7][2, 2] = -2 / np.sqrt(3)


def lattice_shape(dims):
    lx, ly, lz, lt = dims
    return (lt, lz, ly, lx)


def gauge_field(dims, a, seed, chunk=1 << 18):
    """Links U = exp(i a H) with H Gaussian traceless Hermitian, per link."""
    shp = lattice_shape(dims) + (4,)
    n = int(np.prod(shp))
    rng = np.random.default_rng(seed)
    h = rng.standard_normal((n, 8))
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for s in range(0, n, chunk):
        hh = np.einsum("nk,kab->nab", h[s:s + chunk], _LAMBDA) * 0.5
        w, v = np.linalg.eigh(hh)
        out[s:s + chunk] = np.einsum("nak,nk,nbk->nab", v, np.exp(1j * a * w), v.conj())
    return out.reshape(shp + (3, 3))


def spinor_field(dims, seed):
    """Complex Gaussian spinor with unit variance per real component."""
    rng = np.random.default_rng(seed)
    shp = lattice_shape(dims) + (4, 3)
    re = rng.standard_normal(shp)
    im = rng.standard_normal(shp)
    return re + 1j * im


def momenta(dims, seed):
    """Algebra coordinates P_k ~ N(0,1) per link."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(lattice_shape(dims) + (4, 8))


def uniform(seed):
    """One uniform draw in [0,1) for a Metropolis test."""
    return float(np.random.default_rng(seed).random())


# Workloads: each is a dict of plain parameters, no arithmetic.
WORKLOADS = {
    "c1_4x4x4x4": dict(dims=(4, 4, 4, 4), a=0.3, kappa=0.12, seed=SEED_BASE + 0),
    "c2_8x8x8x16": dict(dims=(8, 8, 8, 16), a=0.5, kappa=0.13, seed=SEED_BASE + 1),
    "c3_16x16x16x32": dict(dims=(16, 16, 16, 32), a=0.5, kappa=0.135, kappa_h=0.125,
                           poly=dict(n=16, eps=0.005, lam=8.0), nrhs=3, seed=SEED_BASE + 2),
    "c5_32x32x32x64": dict(dims=(32, 32, 32, 64), a=0.5, kappa=0.136, kappa_h=0.128,
                           poly=dict(n=24, eps=0.005, lam=8.0), beta=5.6, tau=1.0,
                           n_outer=10, seed=SEED_BASE + 4),
}


def batched_workload(seed=SEED_BASE + 3):
    """24 independent lattices of uneven volume with kappa ~ U[0.125, 0.135]."""
    rng = np.random.default_rng(seed)
    lats = [(8, 8, 8, 8)] * 8 + [(12, 12, 12, 24)] * 8 + [(16, 16, 16, 32)] * 8
    kappas = rng.uniform(0.125, 0.135, size=len(lats))
    return [dict(dims=d, a=0.4, kappa=float(k), nrhs=4, seed=seed * 100 + i)
            for i, (d, k) in enumerate(zip(lats, kappas))]
