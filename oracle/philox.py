"""Counter-based Gaussian draws for the oracle (test infrastructure only).

Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11, section 3.3) written from its published definition:
ten rounds of two 64x64->128 multiplications with the round keys bumped by
the Weyl constants between rounds.  The method's random draws (pseudofermion
heat bath chi and momenta P, Section 2 of the paper: chi ~ exp(-chi^dag chi),
P ~ exp(-sum tr P^2)) are generated from it so that the oracle and the CUDA
path can each produce the same field independently.

Field-draw convention (shared by definition, not by code, with the CUDA path):
  real element e of a field, in its lexicographic flat real layout, is
  Gaussian number (e mod 4) of Philox block j = e div 4, drawn with
  counter (j, stream, 0, 0) and key (seed, 0).  The four 64-bit words
  x0..x3 of a block give uniforms u_k = ((x_k >> 11) + 1/2) 2^-53 in (0,1)
  and Box-Muller pairs
     g0 = sqrt(-2 ln u0) cos(2 pi u1),  g1 = sqrt(-2 ln u0) sin(2 pi u1),
     g2 = sqrt(-2 ln u2) cos(2 pi u3),  g3 = sqrt(-2 ln u2) sin(2 pi u3).

Pinned against numpy's own Philox bit generator (tests/test_oracle_algebra.py).
Only tests/, bench.py's CPU-baseline leg and the smoke check may import this.
"""
import numpy as np

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)
_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo64(a, b):
    """Full 128-bit product of uint64 arrays, returned as (hi, lo)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    a_lo, a_hi = a & _MASK32, a >> _S32
    b_lo, b_hi = b & _MASK32, b >> _S32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> _S32) + (lh & _MASK32) + (hl & _MASK32)
    lo = (ll & _MASK32) | ((mid & _MASK32) << _S32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    return hi, lo


def philox4x64_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on counter words (c0..c3) under key (k0, k1)."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64).copy() for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64).copy()
    k1 = np.asarray(k1, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        for r in range(10):
            if r > 0:
                k0 = k0 + W0
                k1 = k1 + W1
            hi0, lo0 = _mulhilo64(M0, c0)
            hi1, lo1 = _mulhilo64(M1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def gaussian_field(n_real, seed, stream):
    """n_real standard normal reals in the field-draw convention above."""
    nblk = (n_real + 3) // 4
    j = np.arange(nblk, dtype=np.uint64)
    z = np.zeros(nblk, dtype=np.uint64)
    x = philox4x64_10(j, np.full(nblk, stream, dtype=np.uint64), z, z,
                      np.uint64(seed), np.uint64(0))
    u = [((xk >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53 for xk in x]
    r0 = np.sqrt(-2.0 * np.log(u[0]))
    r2 = np.sqrt(-2.0 * np.log(u[2]))
    g = np.empty((nblk, 4))
    g[:, 0] = r0 * np.cos(2.0 * np.pi * u[1])
    g[:, 1] = r0 * np.sin(2.0 * np.pi * u[1])
    g[:, 2] = r2 * np.cos(2.0 * np.pi * u[3])
    g[:, 3] = r2 * np.sin(2.0 * np.pi * u[3])
    return g.reshape(-1)[:n_real]
