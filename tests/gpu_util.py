"""Helpers for the GPU parity tests: move seeded synthetic fields to the
device through the library's own pack/unpack entry points and compare with
the oracle.  Not a test module."""
import numpy as np
import torch

from oracle import lattice


def dev(a):
    """numpy complex128/float64 array -> contiguous float64 CUDA tensor (same bytes)."""
    a = np.ascontiguousarray(a)
    if np.iscomplexobj(a):
        a = a.view(np.float64)
    return torch.from_numpy(a.copy()).to("cuda")


def host_c(t, shape):
    """float64 CUDA tensor -> complex128 numpy array of the given shape."""
    return t.cpu().numpy().view(np.complex128).reshape(shape)


def spinor_shape(dims):
    return lattice.shape(dims) + (4, 3)


def pack(lat, psi, parity):
    eo = lat.half_spinor()
    lat.wd_spinor_pack(parity, dev(psi), eo)
    return eo


def unpack(lat, eo, parity):
    dims = lat.dims
    lex = torch.zeros(2 * int(np.prod(spinor_shape(dims))), dtype=torch.float64, device="cuda")
    lat.wd_spinor_unpack(parity, eo, lex)
    return host_c(lex, spinor_shape(dims))


def alg_to_dev(lat, P):
    eo = lat.algebra_field()
    lat.wd_algebra_pack(dev(P), eo)
    return eo


def alg_to_host(lat, eo):
    lex = torch.zeros(64 * lat.Vh, dtype=torch.float64, device="cuda")
    lat.wd_algebra_unpack(eo, lex)
    return lex.cpu().numpy().reshape(lattice.shape(lat.dims) + (4, 8))


def site_rel_err(out, ref, parity=None, dims=None):
    """max over sites of |out(x) - ref(x)|_2 / max(|ref(x)|_2, 1e-3 rms_x |ref|)."""
    d = np.sqrt(np.sum(np.abs(out - ref) ** 2, axis=(-2, -1)))
    r = np.sqrt(np.sum(np.abs(ref) ** 2, axis=(-2, -1)))
    if parity is not None:
        m = lattice.parity(dims) == parity
        d, r = d[m], r[m]
    floor = 1e-3 * np.sqrt(np.mean(r ** 2))
    return float(np.max(d / np.maximum(r, floor)))


def rel_norm_err(out, ref):
    return float(np.linalg.norm((out - ref).reshape(-1)) / np.linalg.norm(ref.reshape(-1)))
