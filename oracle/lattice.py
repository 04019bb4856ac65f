"""Lattice geometry for the oracle (test infrastructure only).

Fields are numpy arrays indexed [t, z, y, x, ...] for dims = (Lx, Ly, Lz, Lt);
direction mu = 0, 1, 2, 3 is x, y, z, t.  Gauge links are periodic in every
direction; fermion fields are periodic in space and antiperiodic in time
(the boundary conditions of the workloads; the paper, Section 3.1, uses the
Wilson action on a 16^3 x 32 lattice without stating them).
"""
import numpy as np

AXIS = {0: 3, 1: 2, 2: 1, 3: 0}   # direction mu -> array axis


def shape(dims):
    lx, ly, lz, lt = dims
    return (lt, lz, ly, lx)


def dims_of(field):
    lt, lz, ly, lx = field.shape[:4]
    return (lx, ly, lz, lt)


def shift(field, mu, step, antiperiodic=False):
    """g(x) = field(x + step * mu_hat), step = +1 or -1.

    With antiperiodic=True and mu = 3 the value fetched across the time
    boundary is negated (fermion boundary condition)."""
    ax = AXIS[mu]
    g = np.roll(field, -step, axis=ax)
    if antiperiodic and mu == 3:
        n = field.shape[ax]
        idx = [slice(None)] * field.ndim
        idx[ax] = n - 1 if step == +1 else 0
        g[tuple(idx)] *= -1
    return g


def parity(dims):
    """Array [t,z,y,x] of (x+y+z+t) mod 2."""
    lt, lz, ly, lx = shape(dims)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx),
                             indexing="ij")
    return (x + y + z + t) % 2


def mask(field, dims, p):
    """Keep the sites of parity p, zero elsewhere."""
    m = (parity(dims) == p)
    m = m.reshape(m.shape + (1,) * (field.ndim - 4))
    return np.where(m, field, 0)
