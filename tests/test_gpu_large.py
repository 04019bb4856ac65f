"""Parity at the workloads' full sizes, in the launch configuration the bench
times (FP32 with 12-real links, FP64, BF16).

32^3 x 64: the hop and K_hat on 256 sampled sites against the oracle's
sampled-site operator, with the tolerances of the small lattices (FP64 1e-12,
FP32 1e-5, BF16 with per-site norm 3e-2 per site; measured BF16 maximum over
2048 sites about 3.5e-3 for the hop and K_hat, the same as on 8^4); the force
kernel from given X, Y at 256 sampled links (1e-12 FP64, 1e-5 FP32 per link);
the tile-staged stencil's K_hat against the oracle's sampled sites and against the
thread kernel at every site (1e-6); whole-lattice properties of the FP64 operator
(<psi, K psi> = |M psi|^2, adjointness of M_hat, 1e-12); the mixed-precision
solve's true residual recomputed with the FP64 operator.

16^3 x 32 (kappa 0.135, heavy 0.125, filter n = 16 on [0.005, 8], three
Gaussian pseudofermions): every force term against central finite differences
of the action along a random algebra direction (step 1e-5 in FP64; FP64 force
1e-6, FP32 force 1e-4 relative), and the Hasenbusch force against the oracle
(1e-9 relative, one oracle solve at this volume: slow).
"""
import numpy as np
import pytest

from oracle import lattice, sampled
from paper_1702_00124_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c5():
    import torch
    from paper_1702_00124_gb300 import wdhmc as wd
    from tests import gpu_util as gu
    dims = (32, 32, 32, 64)
    U = synthetic.gauge_field(dims, 0.5, synthetic.SEED_BASE + 4)
    lat = wd.Lattice(dims)
    lat.wd_gauge_load(torch.from_numpy(U.view(np.float64).reshape(-1)).cuda())
    psi = synthetic.spinor_field(dims, synthetic.SEED_BASE + 44)
    rng = np.random.default_rng(5)
    V = int(np.prod(dims))
    par = lattice.parity(dims).reshape(-1)
    sites = {p: np.sort(rng.choice(np.flatnonzero(par == p), 256, replace=False)) for p in (0, 1)}
    yield dict(dims=dims, U=U, lat=lat, psi=psi, sites=sites, wd=wd, gu=gu, V=V)
    lat.close()


def _rel(out, ref):
    d = np.sqrt(np.sum(np.abs(out - ref) ** 2, axis=(-2, -1)))
    r = np.sqrt(np.sum(np.abs(ref) ** 2, axis=(-2, -1)))
    return float(np.max(d / np.maximum(r, 1e-3 * np.sqrt(np.mean(r ** 2)))))


@pytest.mark.parametrize("prec,recon,tol", [(0, 0, 1e-12), (1, 1, 1e-5), (1, 0, 1e-5), (3, 1, 3e-2), (2, 1, 3e-3)],
                         ids=["fp64", "fp32_recon12", "fp32", "bf16_recon12", "fp16_recon12"])
def test_c5_hop_sampled(c5, prec, recon, tol):
    lat, gu, wd, dims = c5["lat"], c5["gu"], c5["wd"], c5["dims"]
    lat.wd_set_recon(recon)
    try:
        for out_par in (0, 1):
            src = lattice.mask(c5["psi"], dims, 1 - out_par)
            eo = gu.pack(lat, c5["psi"], 1 - out_par)
            out = lat.half_spinor()
            lat.wd_hop(out_par, False, prec, eo, out)
            got = gu.unpack(lat, out, out_par).reshape(-1, 4, 3)
            idx = c5["sites"][out_par]
            assert _rel(got[idx], sampled.hop_at(c5["U"], src, idx)) < tol
    finally:
        lat.wd_set_recon(0)


@pytest.mark.parametrize("prec,recon,tol", [(0, 0, 1e-12), (1, 1, 1e-5), (3, 1, 3e-2), (2, 1, 3e-3)],
                         ids=["fp64", "fp32_recon12", "bf16_recon12", "fp16_recon12"])
def test_c5_khat_sampled(c5, prec, recon, tol):
    lat, gu, dims = c5["lat"], c5["gu"], c5["dims"]
    k = 0.136
    f = lattice.mask(c5["psi"], dims, 0)
    lat.wd_set_recon(recon)
    try:
        eo = gu.pack(lat, c5["psi"], 0)
        out = lat.half_spinor()
        lat.mdagm_apply(k, prec, 1, eo, out)
        got = gu.unpack(lat, out, 0).reshape(-1, 4, 3)
    finally:
        lat.wd_set_recon(0)
    idx = c5["sites"][0]
    assert _rel(got[idx], sampled.khat_at(c5["U"], f, k, idx)) < tol


@pytest.mark.parametrize("prec,tol", [(1, 1e-5), (3, 3e-2)], ids=["fp32", "bf16"])
def test_c5_tile_stencil(c5, prec, tol):
    """The tile-staged kernel (WD_STENCIL_TILE) at the workload's volume: K_hat
    against the oracle at the sampled sites, and against the thread kernel at
    every site (the same FP32 operations per site: 1e-6 relative for FP32
    spinors; BF16 inputs are quantised identically, so 1e-6 holds there too)."""
    import torch
    lat, gu, wd, dims = c5["lat"], c5["gu"], c5["wd"], c5["dims"]
    k = 0.136
    f = lattice.mask(c5["psi"], dims, 0)
    lat.wd_set_recon(1)
    try:
        eo = gu.pack(lat, c5["psi"], 0)
        outs = {}
        for name, st in (("tile", wd.STENCIL_TILE), ("thread", wd.STENCIL_THREAD)):
            lat.wd_set_stencil(st)
            o = lat.half_spinor()
            lat.mdagm_apply(k, prec, 1, eo, o)
            outs[name] = o
        assert lat.wd_kernel_status() == 0
    finally:
        lat.wd_set_stencil(wd.STENCIL_THREAD)
        lat.wd_set_recon(0)
    got = gu.unpack(lat, outs["tile"], 0).reshape(-1, 4, 3)
    idx = c5["sites"][0]
    assert _rel(got[idx], sampled.khat_at(c5["U"], f, k, idx)) < tol
    a = torch.view_as_complex(outs["tile"].view(-1, 2)).view(12, -1)
    b = torch.view_as_complex(outs["thread"].view(-1, 2)).view(12, -1)
    d = torch.linalg.vector_norm(a - b, dim=0)
    r = torch.linalg.vector_norm(b, dim=0)
    rel = torch.max(d / torch.clamp(r, min=1e-3 * float(torch.sqrt(torch.mean(r ** 2)))))
    assert float(rel) < 1e-6


def test_c5_operator_properties(c5):
    import torch
    lat, wd = c5["lat"], c5["wd"]
    k = 0.136
    x, y = lat.half_spinor(), lat.half_spinor()
    lat.gaussian_draw(0, 0, 11, 1, x)
    lat.gaussian_draw(0, 0, 11, 2, y)
    Kx, Mx, Mdy = lat.half_spinor(), lat.half_spinor(), lat.half_spinor()
    lat.mdagm_apply(k, wd.F64, 1, x, Kx)
    lat.wd_apply(k, False, wd.F64, x, Mx)
    lat.wd_apply(k, True, wd.F64, y, Mdy)
    xc, yc = torch.view_as_complex(x.view(-1, 2)), torch.view_as_complex(y.view(-1, 2))
    xKx = torch.vdot(xc, torch.view_as_complex(Kx.view(-1, 2)))
    nMx = torch.vdot(torch.view_as_complex(Mx.view(-1, 2)), torch.view_as_complex(Mx.view(-1, 2)))
    assert abs(complex(xKx) - complex(nMx)) < 1e-12 * abs(complex(nMx))
    a = torch.vdot(yc, torch.view_as_complex(Mx.view(-1, 2)))
    b = torch.vdot(torch.view_as_complex(Mdy.view(-1, 2)), xc)
    assert abs(complex(a) - complex(b)) < 1e-12 * abs(complex(a))


@pytest.mark.parametrize("prec", [1, 3], ids=["fp32", "bf16"])
def test_c5_mixed_cg_true_residual(c5, prec):
    import torch
    lat, wd = c5["lat"], c5["wd"]
    k = 0.136
    chi, b = lat.half_spinor(), lat.half_spinor()
    lat.gaussian_draw(0, 0, 12, 1, chi)
    lat.wd_apply(k, True, wd.F64, chi, b)
    lat.wd_set_recon(1)
    try:
        x = lat.half_spinor()
        info = lat.cg_solve(k, b, x, wd.cg_params(tol=1e-10, prec=prec, maxiter=20000))
    finally:
        lat.wd_set_recon(0)
    Kx = lat.half_spinor()
    lat.mdagm_apply(k, wd.F64, 1, x, Kx)
    rel = float(torch.linalg.vector_norm(b - Kx) / torch.linalg.vector_norm(b))
    assert rel <= 1.01e-10 and abs(rel - info["true_rel_resid"]) < 1e-12


def _link_rel(out, ref):
    """max over sampled links of |dF(l)|_2 / max(|F_ref(l)|_2, 1e-3 rms_l |F_ref|)."""
    d = np.linalg.norm(out - ref, axis=-1)
    r = np.linalg.norm(ref, axis=-1)
    return float(np.max(d / np.maximum(r, 1e-3 * np.sqrt(np.mean(r ** 2)))))


@pytest.mark.parametrize("kind", ["plain", "hasenbusch"])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)], ids=["fp64", "fp32"])
def test_c5_force_xy_sampled(c5, kind, prec, tol):
    """The force kernel from given X, Y (fermion_force_xy, no solve) at 32^3 x 64
    against the oracle's per-link force at 256 sampled links of every direction
    (Section 2, fermion force: 2 kappa^2 Re(Y~^dag dD X~), plus the
    -2 kappa_h^2 Re(phi~^dag dD X~) term of the Hasenbusch action)."""
    lat, gu, wd, dims = c5["lat"], c5["gu"], c5["wd"], c5["dims"]
    k, kh = 0.136, 0.128
    X = lattice.mask(synthetic.spinor_field(dims, synthetic.SEED_BASE + 45), dims, 0)
    Y = lattice.mask(synthetic.spinor_field(dims, synthetic.SEED_BASE + 46), dims, 0)
    phi = lattice.mask(synthetic.spinor_field(dims, synthetic.SEED_BASE + 47), dims, 0)
    rng = np.random.default_rng(17)
    idx = rng.choice(c5["V"], 256, replace=False)
    mu = rng.integers(0, 4, 256)
    t = wd.term(wd.PLAIN, k) if kind == "plain" else wd.term(wd.HASENBUSCH, k, kh)
    F = lat.algebra_field()
    lat.fermion_force_xy(t, gu.pack(lat, phi, 0), gu.pack(lat, X, 0), gu.pack(lat, Y, 0), prec, 1.0, F)
    got = gu.alg_to_host(lat, F).reshape(-1, 4, 8)[idx, mu]
    ref = sampled.xy_force_at(c5["U"], X, Y, k, idx, mu, *((phi, kh) if kind == "hasenbusch" else ()))
    assert _link_rel(got, ref) < tol


# ---------------------------------------------------------------------------
C3 = dict(dims=(16, 16, 16, 32), a=0.5, kappa=0.135, kappa_h=0.125, poly=(16, 0.005, 8.0))


@pytest.fixture(scope="module")
def c3():
    import torch
    from paper_1702_00124_gb300 import wdhmc as wd
    from tests import gpu_util as gu
    dims = C3["dims"]
    U = synthetic.gauge_field(dims, C3["a"], synthetic.SEED_BASE + 2)
    lat = wd.Lattice(dims)
    Ud = torch.from_numpy(U.view(np.float64).reshape(-1)).cuda()
    lat.wd_gauge_load(Ud)
    terms = {"poly": wd.term(wd.POLY, C3["kappa_h"], poly=C3["poly"]),
             "filtered": wd.term(wd.FILTERED, C3["kappa_h"], poly=C3["poly"]),
             "hasenbusch": wd.term(wd.HASENBUSCH, C3["kappa"], C3["kappa_h"])}
    phis = {}
    for i, (name, t) in enumerate(terms.items()):   # three Gaussian pseudofermions
        chi = lat.half_spinor()
        lat.gaussian_draw(0, 0, synthetic.SEED_BASE + 2, 100 + i, chi)
        phi = lat.half_spinor()
        lat.pf_heatbath(t, chi, wd.cg_params(tol=1e-13), phi)
        phis[name] = phi
    yield dict(U=U, Ud=Ud, lat=lat, terms=terms, phis=phis, wd=wd, gu=gu)
    lat.close()


@pytest.mark.parametrize("name", ["poly", "filtered", "hasenbusch"])
@pytest.mark.parametrize("prec,tol", [(0, 1e-6), (1, 1e-4)], ids=["fp64", "mixed_fp32"])
def test_c3_force_vs_finite_difference(c3, name, prec, tol):
    import torch
    from paper_1702_00124_gb300.autograd import pf_action
    lat, wd = c3["lat"], c3["wd"]
    t, phi = c3["terms"][name], c3["phis"][name]
    Om = lat.algebra_field()
    lat.gaussian_draw(1, 0, 77, 5, Om)
    # the force from the autograd adjoint (forward solve keeps X, Y; backward has no solve)
    w = torch.zeros(64 * lat.Vh, dtype=torch.float64, device="cuda", requires_grad=True)
    pf_action(w, lat, t, phi, wd.cg_params(tol=1e-12, prec=prec), wd.F64 if prec == 0 else wd.F32).backward()
    deriv = float(torch.dot(w.grad, Om))
    p = wd.cg_params(tol=1e-12, prec=0)
    h = 1e-5
    S = []
    for s in (+1, -1):
        lat.wd_gauge_load(c3["Ud"])
        lat.step_T(Om, s * h)
        S.append(lat.pf_action(t, phi, p))
    lat.wd_gauge_load(c3["Ud"])
    fd = (S[0] - S[1]) / (2 * h)
    assert abs(fd - deriv) < tol * abs(fd), (name, prec, fd, deriv)


@pytest.mark.slow
def test_c3_hasenbusch_force_vs_oracle(c3):
    from oracle import actions, force
    lat, gu, wd = c3["lat"], c3["gu"], c3["wd"]
    dims = C3["dims"]
    # the same host-drawn pseudofermion for both paths
    phi = lattice.mask(synthetic.spinor_field(dims, synthetic.SEED_BASE + 2 + 500), dims, 0)
    import torch
    from paper_1702_00124_gb300.autograd import pf_action
    F_ref = force.fermion_force(c3["U"], actions.term("hasenbusch", C3["kappa"], C3["kappa_h"]), phi,
                                tol=1e-11)
    w = torch.zeros(64 * lat.Vh, dtype=torch.float64, device="cuda", requires_grad=True)
    pf_action(w, lat, c3["terms"]["hasenbusch"], gu.pack(lat, phi, 0), wd.cg_params(tol=1e-12)).backward()
    err = np.linalg.norm(gu.alg_to_host(lat, w.grad.detach()) - F_ref) / np.linalg.norm(F_ref)
    assert err < 1e-9, err
