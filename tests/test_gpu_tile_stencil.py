"""GPU parity of the two kernels of the 12-real-link stencil (Section 3.1,
Wilson fermions with even-odd preconditioning) against the oracle:
WD_STENCIL_TILE (512-site tiles of links and neighbour-spinor faces copied into
a ring of shared-memory stages by bulk asynchronous copies) and
WD_STENCIL_THREAD (the default: one thread per site, per-thread link staging).

Lattices are ones the tile kernel accepts (Lx/2 a multiple of 4 dividing the
512-site tile in at most 32 rows, Vh a multiple of 512), small enough for the
oracle, and chosen so that faces wrap: 32x2x2x16 (extents of 2: the forward
and backward neighbours coincide; a tile spans several z and t), 32x4x6x8
(6 tiles; y and z faces cross planes) and 64x2x4x8 (16 rows per tile).

Tolerances (per-site relative error |d(x)| / max(|ref(x)|, 1e-3 rms|ref|)):
FP32 1e-5 per hop and 2e-5 for M_hat and K_hat, FP16 3e-3 (6e-3 for K_hat),
BF16 3e-2 (6e-2 for K_hat), as for the other FP32 and 16-bit operator tests;
the two kernels against each other 1e-6 (FP32 arithmetic in the same order per
site, rounding of FMA contractions may differ); the Chebyshev filter at FP32
1e-5; mixed-precision CG reaches the true relative residual 1e-10 recomputed by
the oracle.  The bounded barrier wait of the tile kernel is shown to expire
with WD_ERR_TIMEOUT (a barrier nothing arrives at, 50 ms bound) and to leave
the context usable.
"""
import numpy as np
import pytest

from oracle import lattice, wilson
from oracle.cg import cg
from oracle.poly import ChebyshevFilter
from paper_1702_00124_gb300 import synthetic

pytestmark = pytest.mark.gpu

LATS = [(32, 2, 2, 16), (32, 4, 6, 8), (64, 2, 4, 8)]
HOP_TOL = {1: 1e-5, 2: 3e-3, 3: 3e-2}
STENCILS = {"tile": 1, "thread": 0}


@pytest.fixture(scope="module", params=LATS, ids=lambda d: "x".join(map(str, d)))
def setup(request):
    from paper_1702_00124_gb300 import wdhmc
    from tests import gpu_util as gu
    dims = request.param
    U = synthetic.gauge_field(dims, 0.5, 3000 + dims[3])
    psi = synthetic.spinor_field(dims, 4000 + dims[3])
    lat = wdhmc.Lattice(dims)
    lat.wd_gauge_load(gu.dev(U))
    lat.wd_set_recon(wdhmc.RECON_12)
    yield dims, U, psi, lat, gu, wdhmc
    lat.close()


def _with(lat, stencil, fn):
    lat.wd_set_stencil(stencil)
    try:
        return fn()
    finally:
        lat.wd_set_stencil(0)


@pytest.mark.parametrize("stencil", list(STENCILS), ids=list(STENCILS))
@pytest.mark.parametrize("prec", [1, 2, 3], ids=["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("dagger", [False, True])
def test_hop(setup, stencil, prec, dagger):
    dims, U, psi, lat, gu, wd = setup
    for out_par in (0, 1):
        src = lattice.mask(psi, dims, 1 - out_par)
        ref = lattice.mask(wilson.hop(U, src, dagger=dagger), dims, out_par)
        eo = gu.pack(lat, psi, 1 - out_par)
        out = lat.half_spinor()
        _with(lat, STENCILS[stencil], lambda: lat.wd_hop(out_par, dagger, prec, eo, out))
        assert gu.site_rel_err(gu.unpack(lat, out, out_par), ref, out_par, dims) < HOP_TOL[prec]
    assert lat.wd_kernel_status() == 0


@pytest.mark.parametrize("stencil", list(STENCILS), ids=list(STENCILS))
@pytest.mark.parametrize("prec", [1, 2, 3], ids=["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("dagger", [False, True])
def test_mhat(setup, stencil, prec, dagger):
    dims, U, psi, lat, gu, wd = setup
    k = 0.13
    ref = wilson.apply_Mhat(U, lattice.mask(psi, dims, 0), k, dagger=dagger)
    eo = gu.pack(lat, psi, 0)
    out = lat.half_spinor()
    _with(lat, STENCILS[stencil], lambda: lat.wd_apply(k, dagger, prec, eo, out))
    assert gu.site_rel_err(gu.unpack(lat, out, 0), ref, 0, dims) < 2 * HOP_TOL[prec]


@pytest.mark.parametrize("stencil", list(STENCILS), ids=list(STENCILS))
@pytest.mark.parametrize("prec", [1, 2, 3], ids=["fp32", "fp16", "bf16"])
def test_khat(setup, stencil, prec):
    dims, U, psi, lat, gu, wd = setup
    k = 0.125
    ref = wilson.apply_Khat(U, lattice.mask(psi, dims, 0), k)
    eo = gu.pack(lat, psi, 0)
    out = lat.half_spinor()
    _with(lat, STENCILS[stencil], lambda: lat.mdagm_apply(k, prec, 1, eo, out))
    assert gu.site_rel_err(gu.unpack(lat, out, 0), ref, 0, dims) < 2 * HOP_TOL[prec]


def test_tile_matches_thread_kernel(setup):
    """Both kernels do the same FP32 operations per site in the same order."""
    dims, U, psi, lat, gu, wd = setup
    eo = gu.pack(lat, psi, 0)
    outs = {}
    for name, st in STENCILS.items():
        o = lat.half_spinor()
        _with(lat, st, lambda: lat.mdagm_apply(0.13, wd.F32, 1, eo, o))
        outs[name] = gu.unpack(lat, o, 0)
    assert gu.site_rel_err(outs["tile"], outs["thread"], 0, dims) < 1e-6


@pytest.mark.parametrize("stencil", list(STENCILS), ids=list(STENCILS))
def test_poly_filter_fp32(setup, stencil):
    """P(K_hat) v in FP32: its recurrence runs the last hop of every K_hat fused
    with the Chebyshev step (four epilogue vectors through the stage ring)."""
    dims, U, psi, lat, gu, wd = setup
    k, poly = 0.125, (16, 0.005, 8.0)
    v = lattice.mask(psi, dims, 0)
    ref = ChebyshevFilter(*poly).apply(lambda x: wilson.apply_Khat(U, x, k), v)
    out = lat.half_spinor()
    eo = gu.pack(lat, psi, 0)
    _with(lat, STENCILS[stencil], lambda: lat.poly_filter_apply(k, poly, wd.F32, eo, out))
    assert gu.site_rel_err(gu.unpack(lat, out, 0), ref, 0, dims) < 1e-5


@pytest.mark.parametrize("stencil", list(STENCILS), ids=list(STENCILS))
@pytest.mark.parametrize("prec", [1, 3], ids=["fp32", "bf16"])
def test_mixed_cg(setup, stencil, prec):
    """Mixed-precision CG: its M_hat hop carries the |M_hat p|^2 grid sum."""
    dims, U, psi, lat, gu, wd = setup
    k = 0.13
    b = wilson.apply_Mhat(U, lattice.mask(psi, dims, 0), k, dagger=True)
    be = gu.pack(lat, b, 0)
    x = lat.half_spinor()
    info = _with(lat, STENCILS[stencil],
                 lambda: lat.cg_solve(k, be, x, wd.cg_params(tol=1e-10, prec=prec, maxiter=20000)))
    xh = gu.unpack(lat, x, 0)
    true_rel = np.linalg.norm(b - wilson.apply_Khat(U, xh, k)) / np.linalg.norm(b)
    assert true_rel <= 1.01e-10, (true_rel, info)
    x_ref, _ = cg(lambda v: wilson.apply_Khat(U, v, k), b, 1e-13)
    assert gu.rel_norm_err(xh, x_ref) < 1e-8


def test_stencil_argument_checked(setup):
    dims, U, psi, lat, gu, wd = setup
    with pytest.raises(wd.WdError) as e:
        lat.wd_set_stencil(2)
    assert e.value.code == 1


def test_bounded_wait_expires_and_context_stays_usable(setup):
    """A barrier wait that nothing completes ends after its bound (50 ms here)
    with WD_ERR_TIMEOUT in the device error word; the context keeps working."""
    dims, U, psi, lat, gu, wd = setup
    assert lat.wd_kernel_status() == 0
    with pytest.raises(wd.WdError) as e:
        lat.wd_selftest_wait_timeout(1000)          # below the allowed bound
    assert e.value.code == 1
    lat.wd_selftest_wait_timeout(50_000_000)
    with pytest.raises(wd.WdError) as e:
        lat.wd_kernel_status()
    assert e.value.code == 6
    assert lat.wd_kernel_status() == 0              # read and cleared
    src = lattice.mask(psi, dims, 1)
    ref = lattice.mask(wilson.hop(U, src), dims, 0)
    out = lat.half_spinor()
    _with(lat, 1, lambda: lat.wd_hop(0, False, wd.F32, gu.pack(lat, psi, 1), out))
    assert gu.site_rel_err(gu.unpack(lat, out, 0), ref, 0, dims) < 1e-5
    assert lat.wd_kernel_status() == 0
