"""The allocation-free K_hat entry point (mdagm_apply_noalloc) against the
context-based mdagm_apply.

mdagm_apply_noalloc serves callers that cannot allocate device memory (their
device memory belongs to another pool manager, or they cannot afford the
synchronisation of cudaMalloc, or must not fail on allocation): its scratch
is a fixed static device array.  Checked here through the C ABI: two calls in
a row on different inputs each match mdagm_apply to the FP64 tolerance of
the operator tests (1e-12 per site), so does a call with in and out the same
buffer, and a lattice beyond the fixed scratch size or with an odd, zero or
negative extent is rejected before any launch.  Collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import lattice
from paper_1702_00124_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _gauge_eo(U, dims):
    """Lexicographic links -> complex [4][2][9][Vh] even-odd layout (test-side reshuffle)."""
    V = int(np.prod(dims))
    Vh = V // 2
    Uf = U.reshape(V, 4, 9)
    par = lattice.parity(dims).reshape(-1)
    cb = np.arange(V) // 2
    eo = np.zeros((4, 2, 9, Vh), dtype=np.complex128)
    for p in (0, 1):
        m = par == p
        eo[:, p][:, :, cb[m]] = Uf[m].transpose(1, 2, 0)
    return eo


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 6, 10)], ids=["8x8x8x8", "6x4x6x10"])
def test_noalloc_matches_mdagm_apply(dims):
    import torch
    from paper_1702_00124_gb300 import wdhmc as wd
    from tests import gpu_util as gu
    U = synthetic.gauge_field(dims, 0.5, 3100 + dims[3])
    lat = wd.Lattice(dims)
    lat.wd_gauge_load(gu.dev(U))
    G = gu.dev(_gauge_eo(U, dims))
    d = (C.c_int * 4)(*dims)
    kappa = 0.13
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, seed in enumerate((3200, 3201)):          # two calls in a row
        x = gu.pack(lat, synthetic.spinor_field(dims, seed + dims[3]), 0)
        ref = lat.half_spinor()
        lat.mdagm_apply(kappa, wd.F64, 1, x, ref)
        out = lat.half_spinor()
        rc = wd.lib.mdagm_apply_noalloc(d, C.c_void_p(G.data_ptr()), kappa, C.c_void_p(x.data_ptr()),
                                        C.c_void_p(out.data_ptr()), stream)
        assert rc == 0, wd.lib.wd_last_error().decode()
        torch.cuda.synchronize()
        err = gu.site_rel_err(gu.unpack(lat, out, 0), gu.unpack(lat, ref, 0), 0, dims)
        assert err < 1e-12, (call, err)
    # in and out may be the same buffer: out is written only by the last launch
    io = x.clone()
    rc = wd.lib.mdagm_apply_noalloc(d, C.c_void_p(G.data_ptr()), kappa, C.c_void_p(io.data_ptr()),
                                    C.c_void_p(io.data_ptr()), stream)
    assert rc == 0, wd.lib.wd_last_error().decode()
    torch.cuda.synchronize()
    assert gu.site_rel_err(gu.unpack(lat, io, 0), gu.unpack(lat, ref, 0), 0, dims) < 1e-12
    lat.close()


def test_noalloc_rejects_oversized_lattice():
    import torch
    from paper_1702_00124_gb300 import wdhmc as wd
    d = (C.c_int * 4)(16, 16, 16, 18)           # 36864 sites per parity > 32768
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    rc = wd.lib.mdagm_apply_noalloc(d, p, 0.12, p, p, None)
    assert rc == 1
    assert "32768" in wd.lib.wd_last_error().decode()


@pytest.mark.parametrize("dims", [(4, 4, 4, 5), (4, 0, 4, 4), (3, 4, 4, 4), (4, 4, -2, 4)],
                         ids=["odd_t", "zero", "odd_x", "negative"])
def test_noalloc_rejects_bad_extents(dims):
    """Odd, zero or negative extents are rejected with WD_ERR_ARG before any work."""
    import torch
    from paper_1702_00124_gb300 import wdhmc as wd
    d = (C.c_int * 4)(*dims)
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    rc = wd.lib.mdagm_apply_noalloc(d, p, 0.12, p, p, None)
    assert rc == 1
    assert "even" in wd.lib.wd_last_error().decode()
    torch.cuda.synchronize()
    assert float(buf.abs().sum()) == 0.0
