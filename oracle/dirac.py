"""Gamma matrices for the oracle (test infrastructure only).

The paper (Section 3.1) uses Wilson fermions without fixing a spinor basis.
Reading: the chiral DeGrand-Rossi basis, gamma_5 = gamma_1 gamma_2 gamma_3
gamma_4.  Every quantity the tests compare (spectra, actions, forces) is
basis independent; the CUDA path states the same basis on its own.
Pinned by tests/test_oracle_wilson.py (Clifford algebra, hermiticity,
gamma_5 = diag(1,1,-1,-1)).
"""
import numpy as np

GAMMA = np.zeros((4, 4, 4), dtype=np.complex128)
# gamma_1 (x)
GAMMA[0][0, 3], GAMMA[0][1, 2], GAMMA[0][2, 1], GAMMA[0][3, 0] = 1j, 1j, -1j, -1j
# gamma_2 (y)
GAMMA[1][0, 3], GAMMA[1][1, 2], GAMMA[1][2, 1], GAMMA[1][3, 0] = -1, 1, 1, -1
# gamma_3 (z)
GAMMA[2][0, 2], GAMMA[2][1, 3], GAMMA[2][2, 0], GAMMA[2][3, 1] = 1j, -1j, -1j, 1j
# gamma_4 (t)
GAMMA[3][0, 2], GAMMA[3][1, 3], GAMMA[3][2, 0], GAMMA[3][3, 1] = 1, 1, 1, 1

GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]


def spin_mul(g, psi):
    """Apply a 4x4 spin matrix to psi[..., s, c]."""
    return np.einsum("st,...tc->...sc", g.astype(psi.dtype), psi)
