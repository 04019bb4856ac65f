"""Wilson operator at sampled sites, for the oracle (test infrastructure only).

The same definitions as `oracle.wilson` (Section 3.1 of the paper: Wilson
fermions, even-odd preconditioning), written per site with explicit
neighbour indices instead of whole-lattice shifts, so that D and K_hat can be
evaluated at a few hundred sites of a 32^3 x 64 lattice:

    (D f)(x) = sum_mu [ (1 - g_mu) U_mu(x) s_+ f(x+mu) + (1 + g_mu) U_mu(x-mu)^dag s_- f(x-mu) ]

with s_+- = -1 when the hop crosses the time boundary (antiperiodic fermions).
K_hat at a set S of even sites needs M_hat f on the even sites within two hops
of S, which needs D f on the odd sites within three hops; the functions below
fill exactly those sites.  Pinned against `oracle.wilson` on small lattices
(tests/test_oracle_sampled.py).
"""
import numpy as np

from .dirac import GAMMA


def _coords(dims, idx):
    lx, ly, lz, lt = dims
    t, r = np.divmod(idx, lx * ly * lz)
    z, r = np.divmod(r, lx * ly)
    y, x = np.divmod(r, lx)
    return [x, y, z, t]


def _flat(dims, c):
    lx, ly, lz, lt = dims
    return ((c[3] * lz + c[2]) * ly + c[1]) * lx + c[0]


def neighbour(dims, idx, mu, step):
    """Flat index of x + step*mu and the fermion sign of that hop."""
    c = _coords(dims, idx)
    L = dims[mu]
    v = c[mu] + step
    sign = np.ones(len(idx))
    if mu == 3:
        sign = np.where((v < 0) | (v >= L), -1.0, 1.0)
    c[mu] = v % L
    return _flat(dims, c), sign


def hop_at(U, f, idx, dagger=False):
    """(D f)(x) (or D^dag) at the flat site indices idx; U and f full-lattice arrays."""
    dims = (U.shape[3], U.shape[2], U.shape[1], U.shape[0])
    Uf = U.reshape(-1, 4, 3, 3)
    ff = f.reshape(-1, 4, 3)
    out = np.zeros((len(idx), 4, 3), dtype=f.dtype)
    sg = 1 if dagger else -1
    for mu in range(4):
        g = GAMMA[mu]
        nb, s = neighbour(dims, idx, mu, +1)
        # U_mu(x) f(x+mu): colour index contracted per spin component
        v = np.einsum("nab,nsb->nsa", Uf[idx, mu], ff[nb]) * s[:, None, None]
        out += v + sg * np.einsum("st,ntc->nsc", g, v)
        nb, s = neighbour(dims, idx, mu, -1)
        w = np.einsum("nba,nsb->nsa", Uf[nb, mu].conj(), ff[nb]) * s[:, None, None]
        out += w - sg * np.einsum("st,ntc->nsc", g, w)
    return out


def _ball(dims, idx, radius):
    """All sites within `radius` hops of idx, by hop distance: list of index arrays."""
    shells = [np.unique(idx)]
    seen = set(shells[0].tolist())
    for _ in range(radius):
        nxt = []
        for mu in range(4):
            for st in (+1, -1):
                nxt.append(neighbour(dims, shells[-1], mu, st)[0])
        nxt = np.unique(np.concatenate(nxt))
        shells.append(nxt)
        seen.update(nxt.tolist())
    return shells


def khat_at(U, f_even, kappa, idx):
    """K_hat f at the even sites idx (f_even vanishes on odd sites)."""
    dims = (U.shape[3], U.shape[2], U.shape[1], U.shape[0])
    shells = _ball(dims, idx, 4)
    # hop distance k from idx: shells[k]; even sites at even k, odd at odd k
    need_D1 = np.unique(np.concatenate(shells[1:4:2]))        # odd sites within 3 hops
    need_M = np.unique(np.concatenate(shells[0:3:2]))         # even sites within 2 hops
    need_D2 = np.unique(shells[1])                            # odd sites within 1 hop
    shape = f_even.shape
    t = np.zeros_like(f_even).reshape(-1, 4, 3)
    t[need_D1] = hop_at(U, f_even, need_D1)
    m = np.zeros_like(f_even).reshape(-1, 4, 3)
    m[need_M] = f_even.reshape(-1, 4, 3)[need_M] - kappa ** 2 * hop_at(U, t.reshape(shape), need_M)
    u = np.zeros_like(f_even).reshape(-1, 4, 3)
    u[need_D2] = hop_at(U, m.reshape(shape), need_D2, dagger=True)
    return m[idx] - kappa ** 2 * hop_at(U, u.reshape(shape), idx, dagger=True)


# ---------------------------------------------------------------------------
# Fermion force at sampled links.
#
# Section 2 of the paper gives the two-flavour force as
# -phi^dag K^-1 (dK/dU) K^-1 phi.  With X = K_hat^-1 phi and Y = M_hat X it is
# 2 kappa^2 Re(Y~^dag dD X~) on the full-lattice vectors X~ = (X, D_oe X) and
# Y~ = (Y, D^dag_oe Y).  For the link U_mu(x) rotated as exp(i w T_a) U_mu(x)
# only the two hops across that link depend on w:
#
#   Re(Y~^dag D X~) contains  Y~(x)^dag (1 - g_mu) U_mu(x) s X~(x+mu)
#                           + Y~(x+mu)^dag (1 + g_mu) U_mu(x)^dag s X~(x),
#
# s = -1 when x+mu crosses the time boundary.  Differentiating in w at w = 0
# (d U/dw = i T_a U, d U^dag/dw = -i U^dag T_a) gives, written here term by
# term per link rather than by whole-lattice shifts,
#
#   dS_a = Re[ i s ( Y~(x)^dag (1 - g_mu) T_a U X~(x+mu)
#                  - Y~(x+mu)^dag (1 + g_mu) U^dag T_a X~(x) ) ].

def dre_ydx_at(U, Yt, Xt, idx, mu):
    """d/dw_a Re(Y~^dag D X~) for the links (idx[i], mu[i]), every generator a.

    Yt, Xt: full-lattice spinor arrays, needed at the sites idx and idx + mu.
    Returns an array [len(idx), 8]."""
    from .su3 import generators
    dims = (U.shape[3], U.shape[2], U.shape[1], U.shape[0])
    Uf = U.reshape(-1, 4, 3, 3)
    Yf = Yt.reshape(-1, 4, 3)
    Xf = Xt.reshape(-1, 4, 3)
    T = generators(Yt.dtype)
    idx = np.asarray(idx)
    mu = np.asarray(mu)
    out = np.zeros((len(idx), 8))
    for i, (x, m) in enumerate(zip(idx, mu)):
        nb, s = neighbour(dims, np.array([x]), int(m), +1)
        nb, s = int(nb[0]), float(s[0])
        g = GAMMA[int(m)]
        Ul = Uf[x, m]
        one = np.eye(4)
        for a in range(8):
            # Y~(x)^dag (1 - g) [T_a U X~(x+mu)], colour acting per spin component
            v1 = (T[a] @ Ul @ Xf[nb].T).T               # [spin, colour]
            t1 = np.vdot(Yf[x], (one - g) @ v1)
            # Y~(x+mu)^dag (1 + g) [U^dag T_a X~(x)]
            v2 = (Ul.conj().T @ T[a] @ Xf[x].T).T
            t2 = np.vdot(Yf[nb], (one + g) @ v2)
            out[i, a] = np.real(1j * s * (t1 - t2))
    return out


def expand_at(U, v_e, sites, dagger=False):
    """The full-lattice vector (v_e, D_oe v_e) (dagger: D^dag_oe) filled at `sites`
    only (v_e itself on even sites, the hop on odd ones); zero elsewhere."""
    dims = (U.shape[3], U.shape[2], U.shape[1], U.shape[0])
    lx, ly, lz, lt = dims
    c = [np.asarray(sites) % lx, (np.asarray(sites) // lx) % ly, (np.asarray(sites) // (lx * ly)) % lz,
         np.asarray(sites) // (lx * ly * lz)]
    par = (c[0] + c[1] + c[2] + c[3]) % 2
    out = np.zeros_like(v_e).reshape(-1, 4, 3)
    ev, od = np.asarray(sites)[par == 0], np.asarray(sites)[par == 1]
    out[ev] = v_e.reshape(-1, 4, 3)[ev]
    if len(od):
        out[od] = hop_at(U, v_e, od, dagger)
    return out.reshape(v_e.shape)


def xy_force_at(U, X_e, Y_e, kappa, idx, mu, phi_e=None, kappa_h=None):
    """Force of the PLAIN term from given X, Y at the links (idx, mu):
    2 kappa^2 Re(Y~^dag dD X~); with phi_e (HASENBUSCH) also the term
    -2 kappa_h^2 Re(phi~^dag dD X~) of +2 Re(phi^dag dM_h X)."""
    dims = (U.shape[3], U.shape[2], U.shape[1], U.shape[0])
    fwd = np.array([neighbour(dims, np.array([x]), int(m), +1)[0][0] for x, m in zip(idx, mu)])
    sites = np.unique(np.concatenate([np.asarray(idx), fwd]))
    Xt = expand_at(U, X_e, sites)
    Yt = expand_at(U, Y_e, sites, dagger=True)
    F = 2 * kappa ** 2 * dre_ydx_at(U, Yt, Xt, idx, mu)
    if phi_e is not None:
        Pt = expand_at(U, phi_e, sites, dagger=True)
        F = F - 2 * kappa_h ** 2 * dre_ydx_at(U, Pt, Xt, idx, mu)
    return F
