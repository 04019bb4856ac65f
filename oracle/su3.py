"""SU(3) helpers for the oracle (test infrastructure only).

Generators T_a = lambda_a / 2 (Gell-Mann), tr(T_a T_b) = delta_ab / 2.
Momenta and forces are Hermitian traceless matrices X = sum_a x_a T_a stored
by their eight coordinates x_a = 2 tr(T_a X).  With that normalisation
sum tr P^2 = (1/2) sum_a p_a^2, so P ~ exp(-sum tr P^2) (Section 2) means
p_a ~ N(0,1).

The link update of T[eps] (Section 2, eq. for T-hat) needs exp(i eps P).
The oracle uses the definition of the exponential: the Taylor series, after
scaling the argument by 2^-s to norm <= 1/2, followed by s squarings
(pinned against scipy.linalg.expm).  Reunitarisation: Gram-Schmidt on the
first two rows, third row = (r1 x r2)^*.
"""
import numpy as np

LAMBDA = np.zeros((8, 3, 3), dtype=np.complex128)
LAMBDA[0][0, 1] = LAMBDA[0][1, 0] = 1
LAMBDA[1][0, 1], LAMBDA[1][1, 0] = -1j, 1j
LAMBDA[2][0, 0], LAMBDA[2][1, 1] = 1, -1
LAMBDA[3][0, 2] = LAMBDA[3][2, 0] = 1
LAMBDA[4][0, 2], LAMBDA[4][2, 0] = -1j, 1j
LAMBDA[5][1, 2] = LAMBDA[5][2, 1] = 1
LAMBDA[6][1, 2], LAMBDA[6][2, 1] = -1j, 1j
LAMBDA[7][0, 0] = LAMBDA[7][1, 1] = 1 / np.sqrt(3)
LAMBDA[7][2, 2] = -2 / np.sqrt(3)
T = LAMBDA / 2


def generators(dtype=np.complex128):
    """T_a in the requested precision (lambda_8 rebuilt exactly in that precision)."""
    if dtype == np.complex128:
        return T
    t = LAMBDA.astype(dtype) / 2
    r3 = np.sqrt(np.array(3, dtype=np.real(np.zeros(1, dtype)).dtype))
    t[7] = np.diag(np.array([1, 1, -2], dtype=dtype)) / (2 * r3)
    return t


def alg_to_matrix(p, dtype=np.complex128):
    """sum_a p_a T_a for p[..., 8]."""
    return np.einsum("...a,aij->...ij", p.astype(dtype), generators(dtype))


def matrix_to_alg(X):
    """x_a = Re 2 tr(T_a X)."""
    return 2 * np.einsum("aij,...ji->...a", generators(X.dtype), X).real


def dagger(A):
    return np.swapaxes(A.conj(), -1, -2)


def expm(A):
    """exp(A) for a stack of 3x3 matrices: scaling, Taylor series, squaring."""
    A = np.asarray(A)
    norm = np.max(np.abs(A).sum(axis=-1), axis=-1)   # max row sum per matrix
    s = int(np.ceil(np.log2(max(float(norm.max()), 1e-300) / 0.5))) if norm.max() > 0.5 else 0
    B = A / (2 ** s)
    eye = np.broadcast_to(np.eye(3, dtype=A.dtype), A.shape)
    term = eye.copy()
    out = eye.copy()
    tiny = np.finfo(A.real.dtype).eps
    for k in range(1, 40):
        term = term @ B / k
        out = out + term
        if np.max(np.abs(term)) < tiny * 1e-3:
            break
    for _ in range(s):
        out = out @ out
    return out


def reunitarize(U):
    """Project onto SU(3): Gram-Schmidt on rows 0 and 1, row 2 = (r0 x r1)^*."""
    r0 = U[..., 0, :]
    r0 = r0 / np.sqrt(np.sum(np.abs(r0) ** 2, axis=-1, keepdims=True))
    r1 = U[..., 1, :]
    r1 = r1 - np.sum(r0.conj() * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.sqrt(np.sum(np.abs(r1) ** 2, axis=-1, keepdims=True))
    r2 = np.cross(r0, r1).conj()
    return np.stack([r0, r1, r2], axis=-2)


def project_ta(W):
    """Coordinates of the force from W: x_a = Re(i tr(T_a W)) = (i/2) tr(T_a (W - W^dag))."""
    return np.real(1j * np.einsum("aij,...ji->...a", generators(W.dtype), W))
