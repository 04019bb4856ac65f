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
