"""GPU parity of the Wilson operator kernels against the oracle.

Tolerances (per-site relative error |d(x)| / max(|ref(x)|, 1e-3 rms|ref|)):
FP64 1e-12, FP32 1e-5, FP16 with per-site norm 3e-3, BF16 with per-site norm
3e-2, double-float (two FP32 words, error-free arithmetic) 1e-12.  Lattices: 2^4 (x+mu = x-mu), 4^4, 6x4x6x10 (Vh = 720, a ragged last
block of 128 threads), 8^3x16.
"""
import numpy as np
import pytest

from oracle import lattice, wilson
from paper_1702_00124_gb300 import synthetic

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 3e-3, 3: 3e-2, 4: 1e-12}   # 4: double-float
LATS = [(2, 2, 2, 2), (4, 4, 4, 4), (6, 4, 6, 10), (8, 8, 8, 16)]


@pytest.fixture(scope="module", params=LATS, ids=lambda d: "x".join(map(str, d)))
def setup(request):
    from paper_1702_00124_gb300 import wdhmc
    from tests import gpu_util as gu
    dims = request.param
    U = synthetic.gauge_field(dims, 0.5, 1000 + dims[3])
    psi = synthetic.spinor_field(dims, 2000 + dims[3])
    lat = wdhmc.Lattice(dims)
    lat.wd_gauge_load(gu.dev(U))
    yield dims, U, psi, lat, gu, wdhmc
    lat.close()


def test_pack_roundtrip(setup):
    dims, U, psi, lat, gu, wd = setup
    for par in (0, 1):
        eo = gu.pack(lat, psi, par)
        back = gu.unpack(lat, eo, par)
        assert np.array_equal(back, lattice.mask(psi, dims, par))
    import torch
    Ub = torch.zeros(2 * U.size, dtype=torch.float64, device="cuda")
    lat.wd_gauge_store(Ub)
    assert np.array_equal(gu.host_c(Ub, U.shape), U)


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("dagger", [False, True])
def test_hop(setup, prec, dagger):
    dims, U, psi, lat, gu, wd = setup
    for out_par in (0, 1):
        src = lattice.mask(psi, dims, 1 - out_par)
        ref = lattice.mask(wilson.hop(U, src, dagger=dagger), dims, out_par)
        eo = gu.pack(lat, psi, 1 - out_par)
        out = lat.half_spinor()
        lat.wd_hop(out_par, dagger, prec, eo, out)
        got = gu.unpack(lat, out, out_par)
        assert gu.site_rel_err(got, ref, out_par, dims) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("dagger", [False, True])
def test_mhat(setup, prec, dagger):
    dims, U, psi, lat, gu, wd = setup
    k = 0.13
    src = lattice.mask(psi, dims, 0)
    ref = wilson.apply_Mhat(U, src, k, dagger=dagger)
    eo = gu.pack(lat, psi, 0)
    out = lat.half_spinor()
    lat.wd_apply(k, dagger, prec, eo, out)
    assert gu.site_rel_err(gu.unpack(lat, out, 0), ref, 0, dims) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_khat(setup, prec):
    dims, U, psi, lat, gu, wd = setup
    k = 0.12
    src = lattice.mask(psi, dims, 0)
    ref = wilson.apply_Khat(U, src, k)
    eo = gu.pack(lat, psi, 0)
    out = lat.half_spinor()
    lat.mdagm_apply(k, prec, 1, eo, out)
    assert gu.site_rel_err(gu.unpack(lat, out, 0), ref, 0, dims) < TOL[prec]


def test_khat_recon12(setup):
    dims, U, psi, lat, gu, wd = setup
    k = 0.125
    src = lattice.mask(psi, dims, 0)
    ref = wilson.apply_Khat(U, src, k)
    eo = gu.pack(lat, psi, 0)
    out = lat.half_spinor()
    lat.wd_set_recon(wd.RECON_12)
    try:
        lat.mdagm_apply(k, wd.F32, 1, eo, out)
    finally:
        lat.wd_set_recon(wd.RECON_18)
    assert gu.site_rel_err(gu.unpack(lat, out, 0), ref, 0, dims) < 2e-5


def test_khat_multi_rhs(setup):
    dims, U, psi, lat, gu, wd = setup
    import torch
    k = 0.12
    psi2 = synthetic.spinor_field(dims, 77)
    a, b = gu.pack(lat, psi, 0), gu.pack(lat, psi2, 0)
    x = torch.cat([a, b])
    out = torch.zeros_like(x)
    lat.mdagm_apply(k, wd.F64, 2, x, out)
    for i, p in enumerate((psi, psi2)):
        ref = wilson.apply_Khat(U, lattice.mask(p, dims, 0), k)
        got = gu.unpack(lat, out[i * 24 * lat.Vh:(i + 1) * 24 * lat.Vh].contiguous(), 0)
        assert gu.site_rel_err(got, ref, 0, dims) < 1e-12
