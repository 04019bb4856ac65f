"""Pseudofermion action terms and their heat bath, for the oracle (test
infrastructure only).

Every fermion term of the paper's actions is one of four kinds, each on the
even-site operator K_hat(kappa) = M_hat^dag M_hat:

  plain       S = phi^dag K^-1 phi                       (Section 2, two-flavour S_F)
  hasenbusch  S = phi^dag M_h K^-1 M_h^dag phi           (Section 2, "phi^dag J K^-1 phi")
  poly        S = phi^dag P(K) phi                       (Section 2, polynomial filter S_1)
  filtered    S = phi^dag [P(K) K]^-1 phi                (Section 2, filtered S_2)
  ratio       S = phi^dag Q(K) phi, Q = P_hi / P_lo      (Section 3.3, S_2PF middle term)

Readings of the paper:
  * "phi^dag J K^-1 phi" (Sections 2 and 4.1) is not Hermitian as printed; it
    is read as phi^dag M_h K^-1 M_h^dag phi with J = M_h^dag M_h = K_hat(kappa_h),
    whose Gaussian integral gives det K / det J as mass preconditioning needs.
  * The printed filtered term drops its trailing phi_2; it is restored.
  * For even-odd preconditioning P(K) means P(K_hat).
  * The heavier mass means kappa_h < kappa (Section 2); the "kappa' > kappa"
    of Section 4.1 is read as the same heavier-mass condition.
Composite actions: 1MP = [plain(k'), hasenbusch(k, k')]; 1PF = [poly(k), filtered(k)];
2MP = [plain(k1), hasenbusch(k2, k1), hasenbusch(k, k2)];
PF-MP (Section 4.1) = [poly(k'), filtered(k'), hasenbusch(k, k')];
2PF (Section 3.3) = [poly(P_1, k), ratio(P_2/P_1, k), filtered(P_2, k)];
1PF-2MP (Section 4.2) = [poly(k1), filtered(k1), hasenbusch(k2, k1), hasenbusch(k, k2)];
2PF-1MP (Section 4.2) = [poly(P_1, k'), ratio(P_2/P_1, k'), filtered(P_2, k'), hasenbusch(k, k')].

Heat bath (Section 2: phi is drawn from exp(-S_F) by way of Gaussian chi,
exp(-chi^dag chi)); each phi below makes S(phi) = chi^dag chi:
  plain       phi = M^dag chi
  hasenbusch  phi = M_h J^-1 M^dag chi          (= M_h^-dag M^dag chi)
  poly        phi = P^-1 C^dag chi              (= C^-1 chi, P = C^dag C)
  filtered    phi = C^dag M^dag chi
"""
import numpy as np

from . import wilson
from .cg import cg, vdot
from .lattice import mask, dims_of


def term(kind, kappa, kappa_h=None, poly=None):
    return dict(kind=kind, kappa=kappa, kappa_h=kappa_h, poly=poly)


def even(v):
    return mask(v, dims_of(v), 0)


def K_op(U, kappa):
    return lambda v: wilson.apply_Khat(U, v, kappa)


def filtered_op(U, kappa, poly):
    K = K_op(U, kappa)
    return lambda v: poly.apply(K, K(v))


def action(U, t, phi, tol=1e-14):
    """S for one term; returns (S, aux) with the solutions used by the force."""
    k = t["kind"]
    K = K_op(U, t["kappa"])
    if k == "plain":
        X, info = cg(K, phi, tol)
        return vdot(phi, X).real, dict(X=X, info=info)
    if k == "hasenbusch":
        psi = wilson.apply_Mhat(U, phi, t["kappa_h"], dagger=True)
        X, info = cg(K, psi, tol)
        return vdot(psi, X).real, dict(X=X, info=info)
    if k in ("poly", "ratio"):
        return vdot(phi, t["poly"].apply(K, phi)).real, {}
    if k == "filtered":
        X, info = cg(filtered_op(U, t["kappa"], t["poly"]), phi, tol)
        return vdot(phi, X).real, dict(X=X, info=info)
    raise ValueError(k)


def heatbath(U, t, chi, tol=1e-14):
    """phi with S(phi) = chi^dag chi, for chi on even sites."""
    k = t["kind"]
    kap = t["kappa"]
    if k == "plain":
        return wilson.apply_Mhat(U, chi, kap, dagger=True)
    if k == "hasenbusch":
        y = wilson.apply_Mhat(U, chi, kap, dagger=True)
        w, _ = cg(K_op(U, t["kappa_h"]), y, tol)
        return wilson.apply_Mhat(U, w, t["kappa_h"])
    K = K_op(U, kap)
    if k in ("poly", "ratio"):
        y = t["poly"].apply_half(K, chi, dagger=True)
        phi, _ = cg(lambda v: t["poly"].apply(K, v), y, tol)
        return phi
    if k == "filtered":
        return t["poly"].apply_half(K, wilson.apply_Mhat(U, chi, kap, dagger=True), dagger=True)
    raise ValueError(k)
