"""GPU parity of CG (FP64 and mixed precision with FP64 reliable updates), of
the Chebyshev filter application and of the filtered solve, against the oracle.

Tolerances: solutions of both paths solved to 1e-14 agree to 1e-11 (relative
norm); mixed-precision solves reach a true relative residual <= 1e-10,
recomputed by the oracle's FP64 K_hat; the filter applied in FP64 agrees to
1e-12 per site (FP32: 1e-5).
"""
import numpy as np
import pytest

from oracle import lattice, wilson
from oracle.actions import filtered_op
from oracle.cg import cg
from oracle.poly import ChebyshevFilter
from paper_1702_00124_gb300 import synthetic

pytestmark = pytest.mark.gpu

CASES = {
    "c1_4x4x4x4": ((4, 4, 4, 4), 0.3, 0.12),
    "ragged_6x4x6x10": ((6, 4, 6, 10), 0.5, 0.125),
    "c2_8x8x8x16": ((8, 8, 8, 16), 0.5, 0.13),
}


@pytest.fixture(scope="module", params=list(CASES), ids=list(CASES))
def setup(request):
    from paper_1702_00124_gb300 import wdhmc
    from tests import gpu_util as gu
    dims, a, kappa = CASES[request.param]
    U = synthetic.gauge_field(dims, a, synthetic.SEED_BASE + dims[3])
    chi = lattice.mask(synthetic.spinor_field(dims, synthetic.SEED_BASE + 50 + dims[3]), dims, 0)
    b = wilson.apply_Mhat(U, chi, kappa, dagger=True)      # b = M^dag chi
    lat = wdhmc.Lattice(dims)
    lat.wd_gauge_load(gu.dev(U))
    x_ref, _ = cg(lambda v: wilson.apply_Khat(U, v, kappa), b, 1e-14)
    yield dict(dims=dims, U=U, b=b, kappa=kappa, lat=lat, gu=gu, wd=wdhmc, x_ref=x_ref)
    lat.close()


def _solve(s, prec, tol, **kw):
    lat, gu, wd = s["lat"], s["gu"], s["wd"]
    be = gu.pack(lat, s["b"], 0)
    x = lat.half_spinor()
    info = lat.cg_solve(s["kappa"], be, x, wd.cg_params(tol=tol, prec=prec, maxiter=20000, **kw))
    return gu.unpack(lat, x, 0), info


def test_cg_fp64_matches_oracle(setup):
    x, info = _solve(setup, 0, 1e-14)
    assert info["true_rel_resid"] <= 1e-14
    assert setup["gu"].rel_norm_err(x, setup["x_ref"]) < 1e-11


@pytest.mark.parametrize("prec", [1, 2, 3], ids=["fp32", "fp16", "bf16"])
def test_cg_mixed_reaches_true_residual(setup, prec):
    s = setup
    x, info = _solve(s, prec, 1e-10)
    r = s["b"] - wilson.apply_Khat(s["U"], x, s["kappa"])
    true_rel = np.linalg.norm(r) / np.linalg.norm(s["b"])
    assert true_rel <= 1.01e-10, (true_rel, info)
    assert abs(true_rel - info["true_rel_resid"]) < 1e-12
    err = s["gu"].rel_norm_err(x, s["x_ref"])
    assert err < 1e-8, err               # condition number of K_hat is O(10-100) here
    assert info["reliable_updates"] >= 1


def test_cg_zero_rhs(setup):
    lat, wd = setup["lat"], setup["wd"]
    b = lat.half_spinor()
    x = lat.half_spinor() + 1.0
    info = lat.cg_solve(0.12, b, x, wd.cg_params(tol=1e-10))
    assert info["iters"] == 0 and float(x.abs().max()) == 0.0


def test_cg_maxiter_reports_noconv(setup):
    lat, gu, wd = setup["lat"], setup["gu"], setup["wd"]
    be = gu.pack(lat, setup["b"], 0)
    x = lat.half_spinor()
    with pytest.raises(wd.WdError) as e:
        lat.cg_solve(setup["kappa"], be, x, wd.cg_params(tol=1e-14, maxiter=3, prec=1))
    assert e.value.code == 3


def test_cg_nan_input_reports_nan(setup):
    lat, gu, wd = setup["lat"], setup["gu"], setup["wd"]
    be = gu.pack(lat, setup["b"], 0)
    be[5] = float("nan")
    x = lat.half_spinor()
    with pytest.raises(wd.WdError) as e:
        lat.cg_solve(setup["kappa"], be, x, wd.cg_params(tol=1e-10))
    assert e.value.code == 4


@pytest.mark.parametrize("poly", [(16, 0.005, 8.0), (4, 0.05, 5.0), (0, 0.1, 4.0)])
@pytest.mark.parametrize("prec", [0, 1])
def test_poly_filter_apply(setup, poly, prec):
    s = setup
    lat, gu = s["lat"], s["gu"]
    pf = ChebyshevFilter(*poly)
    ref = pf.apply(lambda v: wilson.apply_Khat(s["U"], v, s["kappa"]), s["b"])
    be = gu.pack(lat, s["b"], 0)
    out = lat.half_spinor()
    lat.poly_filter_apply(s["kappa"], poly, prec, be, out)
    tol = 1e-12 if prec == 0 else 1e-5
    assert gu.site_rel_err(gu.unpack(lat, out, 0), ref, 0, s["dims"]) < tol


@pytest.mark.parametrize("filt", [None, (8, 0.02, 6.0)], ids=["khat", "filtered"])
def test_double_float_residual(setup, filt):
    """Reliable updates with the residual formed in double-float still deliver
    the FP64 true residual (recomputed here by the oracle's FP64 operator)."""
    s = setup
    lat, gu, wd = s["lat"], s["gu"], s["wd"]
    lat.wd_set_residual(1)
    try:
        be = gu.pack(lat, s["b"], 0)
        x = lat.half_spinor()
        info = lat.cg_solve(s["kappa"], be, x, wd.cg_params(tol=1e-10, prec=1), filt=filt)
    finally:
        lat.wd_set_residual(0)
    xh = gu.unpack(lat, x, 0)
    if filt is None:
        Ax = wilson.apply_Khat(s["U"], xh, s["kappa"])
    else:
        Ax = filtered_op(s["U"], s["kappa"], ChebyshevFilter(*filt))(xh)
    true_rel = np.linalg.norm(s["b"] - Ax) / np.linalg.norm(s["b"])
    assert true_rel <= 1.01e-10, (true_rel, info)
    assert abs(true_rel - info["true_rel_resid"]) < 1e-12


def test_filtered_solve(setup):
    s = setup
    lat, gu, wd = s["lat"], s["gu"], s["wd"]
    poly = (8, 0.02, 6.0)
    pf = ChebyshevFilter(*poly)
    x_ref, _ = cg(filtered_op(s["U"], s["kappa"], pf), s["b"], 1e-14)
    be = gu.pack(lat, s["b"], 0)
    for prec, tol, bound in ((0, 1e-13, 1e-10), (1, 1e-10, 1e-8)):
        x = lat.half_spinor()
        info = lat.cg_solve(s["kappa"], be, x, wd.cg_params(tol=tol, prec=prec), filt=poly)
        assert info["true_rel_resid"] <= tol * 1.01
        assert gu.rel_norm_err(gu.unpack(lat, x, 0), x_ref) < bound
        assert info["n_mat"] >= info["iters"] * (poly[0] + 1)
