"""Fermion and gauge forces for the oracle (test infrastructure only).

Force convention (the paper writes F = dS/dU schematically, Section 2):
for the link U_mu(x) rotated as U -> exp(i w T_a) U,

    F_a(x, mu) = d S / d w |_{w=0},   F = sum_a F_a T_a,

so that with H = sum tr P^2 + S the steps T[eps]: U -> exp(i eps P) U and
S[eps]: P -> P - eps F are Hamilton's equations.  Forces are stored as the
eight coordinates F_a per link.

Two-flavour term (Section 2): dS_F = -phi^dag K^-1 (dK) K^-1 phi.  With
X = K_hat^-1 phi and Y = M_hat X this is 2 kappa^2 Re(Y~^dag dD X~) for the
full-lattice vectors X~ = (X, D_oe X), Y~ = (Y, D^dag_oe Y).  The per-link
derivative of Re(Y^dag D X) is

    Re( i tr(T_a W) ),  W = U_mu(x) A1 - A2 U_mu(x)^dag,
    A1 = sum_s [(1 - gamma_mu) X(x+mu)]_s Y_s(x)^dag,
    A2 = sum_s [(1 + gamma_mu) X(x)]_s Y_s(x+mu)^dag,

with the time-boundary sign on the shifted fields.  Pinned by central finite
differences of the actions in extended precision (tests/test_oracle_force.py).
"""
import numpy as np

from . import wilson
from .actions import K_op, filtered_op
from .cg import cg
from .dirac import GAMMA, spin_mul
from .lattice import shift, mask, dims_of
from .su3 import project_ta, dagger


def dre_ydx(U, Y, X):
    """Per link (x, mu) and generator a: d/dw Re(Y^dag D X)."""
    out = np.zeros(U.shape[:4] + (4, 8), dtype=np.real(np.zeros(1, X.dtype)).dtype)
    for mu in range(4):
        g = GAMMA[mu]
        Xf = shift(X, mu, +1, antiperiodic=True)
        A1 = np.einsum("...sa,...sb->...ab", Xf - spin_mul(g, Xf), Y.conj())
        Yf = shift(Y, mu, +1, antiperiodic=True)
        A2 = np.einsum("...sa,...sb->...ab", X + spin_mul(g, X), Yf.conj())
        Um = U[..., mu, :, :]
        out[..., mu, :] = project_ta(Um @ A1 - A2 @ dagger(Um))
    return out


def _dre_mhat(U, A, B, kappa):
    """Per-link d/dw Re(A^dag M_hat B) for even A, B: -kappa^2 Re(A~^dag dD B~)."""
    At = wilson.expand_odd(U, A, dagger=True)
    Bt = wilson.expand_odd(U, B)
    return -kappa ** 2 * dre_ydx(U, At, Bt)


def poly_force(U, kappa, roots, scale, v):
    """Force of S = v^dag Q(K_hat) v with Q = scale * prod_k (K_hat - r_k).

    dS = scale * sum_k Re(L_k^dag dK R_k), L_k = prod_{j<k} (K - r_j^*) v,
    R_k = prod_{j>k} (K - r_j) v, and Re(L^dag dK R) = Re((M R)^dag dM L) +
    Re((M L)^dag dM R)."""
    K = K_op(U, kappa)
    m = len(roots)
    R = [None] * m
    R[m - 1] = v
    for k in range(m - 1, 0, -1):
        R[k - 1] = K(R[k]) - roots[k] * R[k]
    F = 0
    L = v
    for k in range(m):
        ML = wilson.apply_Mhat(U, L, kappa)
        MR = wilson.apply_Mhat(U, R[k], kappa)
        F = F + scale * (_dre_mhat(U, MR, L, kappa) + _dre_mhat(U, ML, R[k], kappa))
        L = K(L) - np.conj(roots[k]) * L
    return F


def fermion_force(U, t, phi, tol=1e-14):
    """F_a(x, mu) = dS/dw for one action term (kinds as in oracle.actions)."""
    k = t["kind"]
    kap = t["kappa"]
    K = K_op(U, kap)
    if k in ("plain", "hasenbusch"):
        psi = phi if k == "plain" else wilson.apply_Mhat(U, phi, t["kappa_h"], dagger=True)
        X, _ = cg(K, psi, tol)
        Y = wilson.apply_Mhat(U, X, kap)
        F = -2 * _dre_mhat(U, Y, X, kap)
        if k == "hasenbusch":
            F = F + 2 * _dre_mhat(U, phi, X, t["kappa_h"])
        return F
    p = t["poly"]
    if k in ("poly", "ratio"):
        return poly_force(U, kap, p.roots(), p.scale(), phi)
    if k == "filtered":
        X, _ = cg(filtered_op(U, kap, p), phi, tol)
        return -poly_force(U, kap, p.roots_times_x(), p.scale(), X)
    raise ValueError(k)


# --------------------------------------------------------------------------
# Gauge action: the paper names S_G only (Section 2); the workloads use the
# Wilson plaquette action S_G = beta sum_{x, mu<nu} (1 - Re tr U_munu(x) / 3).

def plaquette_field(U, mu, nu):
    Um, Un = U[..., mu, :, :], U[..., nu, :, :]
    return Um @ shift(Un, mu, +1) @ dagger(shift(Um, nu, +1)) @ dagger(Un)


def gauge_action(U, beta):
    s = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            s = s + np.sum(1 - np.trace(plaquette_field(U, mu, nu), axis1=-2, axis2=-1).real / 3)
    return beta * s


def staple(U, mu):
    A = 0
    Um = U[..., mu, :, :]
    for nu in range(4):
        if nu == mu:
            continue
        Un = U[..., nu, :, :]
        A = A + shift(Un, mu, +1) @ dagger(shift(Um, nu, +1)) @ dagger(Un)
        Un_m = shift(Un, nu, -1)
        A = A + dagger(shift(Un_m, mu, +1)) @ dagger(shift(Um, nu, -1)) @ Un_m
    return A


def gauge_force(U, beta):
    """dS_G/dw = -(beta/3) Re(i tr(T_a U_mu(x) A_mu(x))), A the staple sum."""
    out = np.zeros(U.shape[:4] + (4, 8), dtype=np.real(np.zeros(1, U.dtype)).dtype)
    for mu in range(4):
        out[..., mu, :] = -(beta / 3) * project_ta(U[..., mu, :, :] @ staple(U, mu))
    return out
