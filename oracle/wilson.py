"""Wilson-Dirac operator for the oracle (test infrastructure only).

Section 2 of the paper: the two-flavour fermion action is built on the
fermion matrix M and K = M^dag M; Section 3.1: Wilson fermions with hopping
parameter kappa and even-odd preconditioning.  With Wilson parameter r = 1

    M = 1 - kappa D,
    (D psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
                        + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ],

fermions antiperiodic in time.  D^dag is coded here as its own transposed
stencil (not as gamma_5 D gamma_5) so that the adjoint identities the tests
check are not true by construction:

    (D^dag psi)(x) = sum_mu [ (1 + gamma_mu) U_mu(x) psi(x+mu)
                            + (1 - gamma_mu) U_mu(x-mu)^dag psi(x-mu) ].

Even-odd: D only couples sites of opposite parity, so with M acting on
(even, odd) blocks the Schur complement on even sites is

    M_hat = 1 - kappa^2 D_eo D_oe,   K_hat = M_hat^dag M_hat,

and det M = det M_hat (the diagonal blocks are the identity).  Half-lattice
vectors are full-lattice arrays that vanish on odd sites.
"""
import numpy as np

from .dirac import GAMMA
from .lattice import shift, mask, dims_of


def _colour(Umat, psi):
    """U psi on every spin component: (U psi_s)_a = sum_b U[...,a,b] psi[...,s,b]."""
    return np.matmul(psi, np.swapaxes(Umat, -1, -2))


def _colour_dag(Umat, psi):
    """U^dag psi on every spin component: sum_b conj(U[...,b,a]) psi[...,s,b]."""
    return np.matmul(psi, Umat.conj())


def _spin(g, psi):
    """(g psi)_s = sum_t g[s,t] psi[...,t,c]."""
    return np.matmul(g, psi)


def hop(U, psi, dagger=False):
    """D psi (dagger=False) or D^dag psi (dagger=True), full lattice."""
    out = np.zeros_like(psi)
    sgn = 1 if dagger else -1
    for mu in range(4):
        g = GAMMA[mu].astype(psi.dtype)
        fw = _colour(U[..., mu, :, :], shift(psi, mu, +1, antiperiodic=True))
        out += fw + sgn * _spin(g, fw)
        Ub = shift(U[..., mu, :, :], mu, -1)
        bw = _colour_dag(Ub, shift(psi, mu, -1, antiperiodic=True))
        out += bw - sgn * _spin(g, bw)
    return out


def apply_M(U, psi, kappa, dagger=False):
    """Full Wilson matrix M = 1 - kappa D (or M^dag)."""
    return psi - kappa * hop(U, psi, dagger)


def apply_Mhat(U, psi_e, kappa, dagger=False):
    """Even-odd preconditioned M_hat = 1 - kappa^2 D_eo D_oe (or M_hat^dag)."""
    dims = dims_of(psi_e)
    t = mask(hop(U, psi_e, dagger), dims, 1)
    return psi_e - kappa ** 2 * mask(hop(U, t, dagger), dims, 0)


def apply_Khat(U, psi_e, kappa):
    """K_hat = M_hat^dag M_hat on even sites; one K_hat is the unit N_mat counts."""
    return apply_Mhat(U, apply_Mhat(U, psi_e, kappa), kappa, dagger=True)


def expand_odd(U, v_e, dagger=False):
    """Full-lattice vector (v_e, D_oe v_e) (dagger: (v_e, D^dag_oe v_e))."""
    dims = dims_of(v_e)
    return v_e + mask(hop(U, v_e, dagger), dims, 1)
