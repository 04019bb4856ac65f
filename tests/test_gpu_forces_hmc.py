"""GPU parity of actions, heat bath, fermion and gauge forces, HMC steps,
Gaussian draws and a whole trajectory, against the oracle.

Tolerances: actions and heat bath 1e-10 relative; FP64 forces 1e-9
(Frobenius, relative); FP32 forces 1e-5; gauge action 1e-12; T step 1e-13
per link; Gaussian draws 1e-13 (same Philox words, transcendental rounding
differs); trajectory dH 1e-9 absolute and final links 1e-10.
"""
import numpy as np
import pytest

from oracle import actions, force, hmc, lattice, philox, wilson
from oracle.poly import ChebyshevFilter
from paper_1702_00124_gb300 import synthetic

pytestmark = pytest.mark.gpu

POLY = (4, 0.05, 5.0)
RATIO_HI, RATIO_LO = (8, 0.05, 5.0), (2, 0.05, 5.0)     # Q = P_8 / P_2 (Section 3.3)
KAPPA, KAPPA_H = 0.125, 0.115


def _oracle_term(kind):
    from oracle.poly import RatioFilter
    pf = ChebyshevFilter(*POLY)
    q = RatioFilter(ChebyshevFilter(*RATIO_HI), ChebyshevFilter(*RATIO_LO))
    return {0: actions.term("plain", KAPPA), 1: actions.term("hasenbusch", KAPPA, KAPPA_H),
            2: actions.term("poly", KAPPA_H, poly=pf), 3: actions.term("filtered", KAPPA_H, poly=pf),
            4: actions.term("ratio", KAPPA_H, poly=q)}[kind]


def _gpu_term(wd, kind):
    return {0: wd.term(wd.PLAIN, KAPPA), 1: wd.term(wd.HASENBUSCH, KAPPA, KAPPA_H),
            2: wd.term(wd.POLY, KAPPA_H, poly=POLY), 3: wd.term(wd.FILTERED, KAPPA_H, poly=POLY),
            4: wd.term(wd.RATIO, KAPPA_H, poly=RATIO_HI, poly_lo=RATIO_LO)}[kind]


@pytest.fixture(scope="module", params=[(4, 4, 4, 4), (6, 4, 6, 10)], ids=["4x4x4x4", "6x4x6x10"])
def setup(request):
    from paper_1702_00124_gb300 import wdhmc
    from tests import gpu_util as gu
    dims = request.param
    U = synthetic.gauge_field(dims, 0.5, 501 + dims[3])
    chi = lattice.mask(synthetic.spinor_field(dims, 502 + dims[3]), dims, 0)
    lat = wdhmc.Lattice(dims)
    lat.wd_gauge_load(gu.dev(U))
    yield dict(dims=dims, U=U, chi=chi, lat=lat, gu=gu, wd=wdhmc)
    lat.close()


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4], ids=["plain", "hasenbusch", "poly", "filtered", "ratio"])
def test_heatbath_and_action(setup, kind):
    s = setup
    lat, gu, wd = s["lat"], s["gu"], s["wd"]
    t_o, t_g = _oracle_term(kind), _gpu_term(wd, kind)
    phi_ref = actions.heatbath(s["U"], t_o, s["chi"])
    chi_e = gu.pack(lat, s["chi"], 0)
    phi = lat.half_spinor()
    lat.pf_heatbath(t_g, chi_e, wd.cg_params(tol=1e-13), phi)
    assert gu.rel_norm_err(gu.unpack(lat, phi, 0), phi_ref) < 1e-10
    S_ref, _ = actions.action(s["U"], t_o, phi_ref)
    for prec in (0, 1):
        S = lat.pf_action(t_g, phi, wd.cg_params(tol=1e-11, prec=prec))
        assert abs(S - S_ref) < 1e-10 * abs(S_ref), (prec, S, S_ref)
    chi2 = float(np.vdot(s["chi"], s["chi"]).real)
    assert abs(S_ref - chi2) < 1e-9 * chi2


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4], ids=["plain", "hasenbusch", "poly", "filtered", "ratio"])
def test_fermion_force(setup, kind):
    s = setup
    lat, gu, wd = s["lat"], s["gu"], s["wd"]
    t_o, t_g = _oracle_term(kind), _gpu_term(wd, kind)
    phi = s["chi"]                      # any even field serves as phi
    F_ref = force.fermion_force(s["U"], t_o, phi)
    phi_e = gu.pack(lat, phi, 0)
    for prec, tol in ((0, 1e-9), (1, 1e-5)):
        F = lat.algebra_field()
        lat.fermion_force(t_g, phi_e, wd.cg_params(tol=1e-13 if prec == 0 else 1e-10, prec=prec), 1.0, F)
        Fg = gu.alg_to_host(lat, F)
        err = np.linalg.norm(Fg - F_ref) / np.linalg.norm(F_ref)
        assert err < tol, (prec, err)
    # coef scales and accumulates: F += 2 * force on top of -1 * force gives +1 * force
    F = lat.algebra_field()
    p = wd.cg_params(tol=1e-13)
    lat.fermion_force(t_g, phi_e, p, -1.0, F)
    lat.fermion_force(t_g, phi_e, p, 2.0, F)
    assert np.linalg.norm(gu.alg_to_host(lat, F) - F_ref) < 1e-9 * np.linalg.norm(F_ref)


# The filter of the trajectory bench (degree 24 on [0.005, 8]: ceil(sqrt(24)) = 5
# checkpoint segments of five roots, the fused FP32 Chebyshev-step hop) and the
# two-filter pair P_24 / P_4 of Section 3.3, at the bench's heavy kappa.
BENCH_POLY, BENCH_LO, BENCH_KAPPA_H = (24, 0.005, 8.0), (4, 0.005, 8.0), 0.128


@pytest.mark.parametrize("kind", ["poly", "filtered", "ratio"])
def test_fermion_force_bench_filter(setup, kind):
    """fermion_force (solve and force) and fermion_force_xy (force from the
    oracle's X, no solve) against the oracle force at the bench's filter:
    FP64 1e-9, FP32 1e-5 (relative, Frobenius)."""
    from oracle.cg import cg
    from oracle.poly import RatioFilter
    s = setup
    lat, gu, wd = s["lat"], s["gu"], s["wd"]
    U, phi, kh = s["U"], s["chi"], BENCH_KAPPA_H
    pf = ChebyshevFilter(*BENCH_POLY)
    if kind == "poly":
        t_o, t_g = actions.term("poly", kh, poly=pf), wd.term(wd.POLY, kh, poly=BENCH_POLY)
    elif kind == "filtered":
        t_o, t_g = actions.term("filtered", kh, poly=pf), wd.term(wd.FILTERED, kh, poly=BENCH_POLY)
    else:
        q = RatioFilter(pf, ChebyshevFilter(*BENCH_LO))
        t_o = actions.term("ratio", kh, poly=q)
        t_g = wd.term(wd.RATIO, kh, poly=BENCH_POLY, poly_lo=BENCH_LO)
    phi_e = gu.pack(lat, phi, 0)
    X_e = None
    if kind == "filtered":
        # The FP64 root product of K_hat P(K_hat) at degree 24 is accurate to about
        # 1e-12 relative, so the oracle solves to 5e-12 (bounded iterations); the
        # force error this leaves is of the same order, far below 1e-9.
        X, info = cg(actions.filtered_op(U, kh, pf), phi, 5e-12, maxiter=400)
        assert info["rel_resid"] <= 5e-12, info
        F_ref = -force.poly_force(U, kh, pf.roots_times_x(), pf.scale(), X)
        X_e = gu.pack(lat, X, 0)
    else:
        F_ref = force.fermion_force(U, t_o, phi)
    nref = np.linalg.norm(F_ref)
    for prec, tol in ((0, 1e-9), (1, 1e-5)):
        F = lat.algebra_field()
        lat.fermion_force(t_g, phi_e, wd.cg_params(tol=1e-12 if prec == 0 else 1e-10, prec=prec, maxiter=4000),
                          1.0, F)
        err = np.linalg.norm(gu.alg_to_host(lat, F) - F_ref) / nref
        assert err < tol, ("fermion_force", prec, err)
        F = lat.algebra_field()
        lat.fermion_force_xy(t_g, phi_e, X_e, None, prec, 1.0, F)
        err = np.linalg.norm(gu.alg_to_host(lat, F) - F_ref) / nref
        assert err < tol, ("fermion_force_xy", prec, err)


def test_ratio_degenerate_and_invalid(setup):
    """Q = P / P = 1: S = phi^dag phi, phi = chi, zero force.  Filters whose orders
    do not nest ((n_lo + 1) not dividing (n + 1)) or whose intervals differ are
    rejected before any work."""
    s = setup
    lat, gu, wd = s["lat"], s["gu"], s["wd"]
    chi_e = gu.pack(lat, s["chi"], 0)
    t1 = wd.term(wd.RATIO, KAPPA_H, poly=RATIO_HI, poly_lo=RATIO_HI)
    p = wd.cg_params(tol=1e-12)
    phi = lat.half_spinor()
    lat.pf_heatbath(t1, chi_e, p, phi)
    assert gu.rel_norm_err(gu.unpack(lat, phi, 0), s["chi"]) < 1e-15
    chi2 = float(np.vdot(s["chi"], s["chi"]).real)
    assert abs(lat.pf_action(t1, phi, p) - chi2) < 1e-13 * chi2
    F = lat.algebra_field()
    lat.fermion_force(t1, phi, p, 1.0, F)
    assert float(F.abs().max()) == 0.0
    for hi, lo in ((RATIO_HI, (4, 0.05, 5.0)), (RATIO_HI, (2, 0.05, 6.0)), (RATIO_LO, RATIO_HI)):
        with pytest.raises(wd.WdError):
            lat.pf_action(wd.term(wd.RATIO, KAPPA_H, poly=hi, poly_lo=lo), phi, p)


def test_gauge_action_and_force(setup):
    s = setup
    lat, gu = s["lat"], s["gu"]
    beta = 5.6
    S_ref = force.gauge_action(s["U"], beta)
    assert abs(lat.gauge_action(beta) - S_ref) < 1e-12 * S_ref
    F_ref = force.gauge_force(s["U"], beta)
    for prec, tol in ((0, 1e-12), (1, 1e-5)):
        F = lat.algebra_field()
        lat.gauge_force(beta, prec, 1.0, F)
        err = np.linalg.norm(gu.alg_to_host(lat, F) - F_ref) / np.linalg.norm(F_ref)
        assert err < tol, (prec, err)


def test_steps_and_kinetic(setup):
    s = setup
    lat, gu = s["lat"], s["gu"]
    P = synthetic.momenta(s["dims"], 77)
    Pe = gu.alg_to_dev(lat, P)
    assert abs(lat.kinetic_energy(Pe) - hmc.kinetic(P)) < 1e-12 * hmc.kinetic(P)
    import torch
    for eps in (2.0, 0.3, 0.01, 1e-4):     # 2.0: angles above the series range
        lat.wd_gauge_load(gu.dev(s["U"]))
        lat.step_T(Pe, eps)
        Ub = torch.zeros(2 * s["U"].size, dtype=torch.float64, device="cuda")
        lat.wd_gauge_store(Ub)
        ref = hmc.step_T(s["U"], P, eps)
        assert np.max(np.abs(gu.host_c(Ub, s["U"].shape) - ref)) < 1e-13
    lat.wd_gauge_load(gu.dev(s["U"]))
    F = gu.alg_to_dev(lat, synthetic.momenta(s["dims"], 78))
    lat.step_S(Pe, F, 0.25)
    assert np.max(np.abs(gu.alg_to_host(lat, Pe) - hmc.step_S(P, synthetic.momenta(s["dims"], 78), 0.25))) < 1e-14


def test_gaussian_draws(setup):
    s = setup
    lat, gu = s["lat"], s["gu"]
    dims = s["dims"]
    V = int(np.prod(dims))
    seed, stream = 424242, 9
    out = lat.algebra_field()
    lat.gaussian_draw(1, 0, seed, stream, out)
    ref = philox.gaussian_field(V * 32, seed, stream).reshape(lattice.shape(dims) + (4, 8))
    assert np.max(np.abs(gu.alg_to_host(lat, out) - ref)) < 1e-13
    for par in (0, 1):
        h = lat.half_spinor()
        lat.gaussian_draw(0, par, seed, stream + 1, h)
        g = philox.gaussian_field(V * 24, seed, stream + 1)
        ref = lattice.mask(g.view(np.complex128).reshape(lattice.shape(dims) + (4, 3)), dims, par)
        assert np.max(np.abs(gu.unpack(lat, h, par) - ref)) < 1e-13


def test_bench_configuration_trajectory():
    """The bench's configuration at 4^4: PF-MP + gauge, nested Omelyan 2MN with the
    bench's level structure, FP32 forces, mixed-precision solves to 1e-10 with
    double-float residuals, 12-real FP32 links.  dH must agree with the oracle's FP64
    trajectory to 1e-4 + 1e-4 |dH| (FP32 forces move the trajectory by ~1e-6)."""
    import torch
    from paper_1702_00124_gb300 import wdhmc as wd
    from tests import gpu_util as gu
    dims = (4, 4, 4, 4)
    U0 = synthetic.gauge_field(dims, 0.3, 951)
    k, kh, beta, tau = 0.124, 0.115, 5.6, 0.5
    poly = (8, 0.02, 6.0)
    seed, traj = 321, 2
    pf = ChebyshevFilter(*poly)
    terms_o = [actions.term("poly", kh, poly=pf), actions.term("filtered", kh, poly=pf),
               actions.term("hasenbusch", k, kh)]
    terms_g = [wd.term(wd.POLY, kh, poly=poly), wd.term(wd.FILTERED, kh, poly=poly),
               wd.term(wd.HASENBUSCH, k, kh)]
    groups = [1, 0, 0]
    levels = [(0, 3), (1, 1), (-1, 2)]
    V = int(np.prod(dims))
    base = traj * 64
    P0 = philox.gaussian_field(V * 32, seed, base).reshape(lattice.shape(dims) + (4, 8))
    phis = []
    for i, t in enumerate(terms_o):
        g = philox.gaussian_field(V * 24, seed, base + 1 + i)
        # chi ~ exp(-chi^dag chi): the unit-variance draw over sqrt(2) (Section 2)
        chi = lattice.mask(g.view(np.complex128).reshape(lattice.shape(dims) + (4, 3)), dims, 0) / np.sqrt(2)
        phis.append(actions.heatbath(U0, t, chi))

    def H(U, P):
        return hmc.kinetic(P) + force.gauge_action(U, beta) + sum(
            actions.action(U, t, ph)[0] for t, ph in zip(terms_o, phis))

    def fog(grp, U):
        if grp == -1:
            return force.gauge_force(U, beta)
        return sum(force.fermion_force(U, t, ph) for t, ph, g in zip(terms_o, phis, groups) if g == grp)

    U1, P1 = hmc.integrate(U0, P0, hmc.nested(levels, tau, "omelyan"), fog)
    dH_ref = H(U1, P1) - H(U0, P0)
    lat = wd.Lattice(dims)
    lat.wd_gauge_load(gu.dev(U0))
    lat.wd_set_recon(wd.RECON_12)
    lat.wd_set_residual(1)
    ops = wd.wd_schedule_nested(1, tau, [g for g, _ in levels], [n for _, n in levels])
    p32 = wd.cg_params(tol=1e-10, prec=wd.F32, maxiter=20000)
    r = lat.hmc_trajectory(terms_g, groups, beta, ops, p32, p32, wd.F32, seed, traj, 0.0)
    assert abs(r["dH"] - dH_ref) < 1e-4 + 1e-4 * abs(dH_ref), (r["dH"], dH_ref)
    assert r["t_force_group_ms"][0] > 0 and r["t_T_ms"] > 0
    lat.close()


def test_trajectory_matches_oracle():
    """One PF-MP + gauge trajectory with a nested Omelyan 2MN schedule, every
    step in FP64: same draws (Philox), same schedule structure (the GPU merges
    commuting S steps, the oracle does not), dH and final links compared."""
    from paper_1702_00124_gb300 import wdhmc as wd
    from tests import gpu_util as gu
    dims = (4, 4, 4, 4)
    U0 = synthetic.gauge_field(dims, 0.3, 901)
    k, kh, beta, tau = 0.124, 0.115, 5.6, 0.4
    seed, traj = 123, 5
    pf = ChebyshevFilter(*POLY)
    terms_o = [actions.term("poly", kh, poly=pf), actions.term("filtered", kh, poly=pf),
               actions.term("hasenbusch", k, kh)]
    terms_g = [wd.term(wd.POLY, kh, poly=POLY), wd.term(wd.FILTERED, kh, poly=POLY),
               wd.term(wd.HASENBUSCH, k, kh)]
    groups = [1, 0, 0]                     # group 0 outer: filtered + hasenbusch; 1: poly; -1: gauge
    levels = [(0, 2), (1, 2), (-1, 2)]
    ops_g = wd.wd_schedule_nested(1, tau, [g for g, _ in levels], [n for _, n in levels])
    ops_o = hmc.nested(levels, tau, "omelyan")
    V = int(np.prod(dims))
    base = traj * 64
    P0 = philox.gaussian_field(V * 32, seed, base).reshape(lattice.shape(dims) + (4, 8))
    phis = []
    for i, t in enumerate(terms_o):
        g = philox.gaussian_field(V * 24, seed, base + 1 + i)
        # chi ~ exp(-chi^dag chi): the unit-variance draw over sqrt(2) (Section 2)
        chi = lattice.mask(g.view(np.complex128).reshape(lattice.shape(dims) + (4, 3)), dims, 0) / np.sqrt(2)
        phis.append(actions.heatbath(U0, t, chi))

    def H(U, P):
        return hmc.kinetic(P) + force.gauge_action(U, beta) + sum(
            actions.action(U, t, ph)[0] for t, ph in zip(terms_o, phis))

    def fog(grp, U):
        if grp == -1:
            return force.gauge_force(U, beta)
        return sum(force.fermion_force(U, t, ph) for t, ph, g in zip(terms_o, phis, groups) if g == grp)

    U1, P1 = hmc.integrate(U0, P0, ops_o, fog)
    dH_ref = H(U1, P1) - H(U0, P0)

    lat = wd.Lattice(dims)
    lat.wd_gauge_load(gu.dev(U0))
    p64 = wd.cg_params(tol=1e-14, maxiter=20000)
    r = lat.hmc_trajectory(terms_g, groups, beta, ops_g, p64, p64, wd.F64, seed, traj, 0.0)
    assert abs(r["dH"] - dH_ref) < 1e-9, (r["dH"], dH_ref)
    import torch
    Ub = torch.zeros(2 * U0.size, dtype=torch.float64, device="cuda")
    lat.wd_gauge_store(Ub)
    if r["accepted"]:
        assert np.max(np.abs(gu.host_c(Ub, U0.shape) - U1)) < 1e-10
    else:
        assert np.array_equal(gu.host_c(Ub, U0.shape), U0)
    assert r["n_mat"] > 0
    lat.close()


def test_two_filter_trajectory_matches_oracle():
    """2PF-1MP (Section 3.3, Section 4.2): P_1, Q = P_2 / P_1, the filtered P_2 term and
    a Hasenbusch term, on four integrator levels, every step in FP64; dH and the final
    links against the oracle's trajectory from the same draws."""
    from oracle.poly import RatioFilter
    from paper_1702_00124_gb300 import wdhmc as wd
    from tests import gpu_util as gu
    dims = (4, 4, 4, 4)
    U0 = synthetic.gauge_field(dims, 0.3, 911)
    k, kh, beta, tau = 0.124, 0.115, 5.6, 0.4
    seed, traj = 77, 3
    p1, p2 = (2, 0.02, 6.0), (8, 0.02, 6.0)
    f1, f2 = ChebyshevFilter(*p1), ChebyshevFilter(*p2)
    terms_o = [actions.term("poly", kh, poly=f1), actions.term("ratio", kh, poly=RatioFilter(f2, f1)),
               actions.term("filtered", kh, poly=f2), actions.term("hasenbusch", k, kh)]
    terms_g = [wd.term(wd.POLY, kh, poly=p1), wd.term(wd.RATIO, kh, poly=p2, poly_lo=p1),
               wd.term(wd.FILTERED, kh, poly=p2), wd.term(wd.HASENBUSCH, k, kh)]
    groups = [2, 1, 0, 0]
    levels = [(0, 2), (1, 1), (2, 1), (-1, 2)]
    V = int(np.prod(dims))
    base = traj * 64
    P0 = philox.gaussian_field(V * 32, seed, base).reshape(lattice.shape(dims) + (4, 8))
    phis = []
    for i, t in enumerate(terms_o):
        g = philox.gaussian_field(V * 24, seed, base + 1 + i)
        # chi ~ exp(-chi^dag chi): the unit-variance draw over sqrt(2) (Section 2)
        chi = lattice.mask(g.view(np.complex128).reshape(lattice.shape(dims) + (4, 3)), dims, 0) / np.sqrt(2)
        phis.append(actions.heatbath(U0, t, chi))

    def H(U, P):
        return hmc.kinetic(P) + force.gauge_action(U, beta) + sum(
            actions.action(U, t, ph)[0] for t, ph in zip(terms_o, phis))

    def fog(grp, U):
        if grp == -1:
            return force.gauge_force(U, beta)
        return sum(force.fermion_force(U, t, ph) for t, ph, g in zip(terms_o, phis, groups) if g == grp)

    U1, P1 = hmc.integrate(U0, P0, hmc.nested(levels, tau, "omelyan"), fog)
    dH_ref = H(U1, P1) - H(U0, P0)
    lat = wd.Lattice(dims)
    lat.wd_gauge_load(gu.dev(U0))
    ops = wd.wd_schedule_nested(1, tau, [g for g, _ in levels], [n for _, n in levels])
    p64 = wd.cg_params(tol=1e-14, maxiter=20000)
    r = lat.hmc_trajectory(terms_g, groups, beta, ops, p64, p64, wd.F64, seed, traj, 0.0)
    assert abs(r["dH"] - dH_ref) < 1e-9, (r["dH"], dH_ref)
    import torch
    Ub = torch.zeros(2 * U0.size, dtype=torch.float64, device="cuda")
    lat.wd_gauge_store(Ub)
    if r["accepted"]:
        assert np.max(np.abs(gu.host_c(Ub, U0.shape) - U1)) < 1e-10
    else:
        assert np.array_equal(gu.host_c(Ub, U0.shape), U0)
    lat.close()


def test_ratio_heatbath_wide_filters_mixed_precision():
    """Q = P_26 / P_8 on [0.005, 8] at kappa = 0.15: the FP32 root product loses up to
    6e-5 relative on low modes, and the mixed-precision heat bath must still converge
    (reliable-update factor of the K_hat class) and give S(phi) = chi^dag chi."""
    import torch
    from paper_1702_00124_gb300 import wdhmc as wd
    from tests import gpu_util as gu
    dims = (4, 4, 4, 8)
    U = synthetic.gauge_field(dims, 0.4, 577)
    lat = wd.Lattice(dims)
    lat.wd_gauge_load(gu.dev(U))
    t = wd.term(wd.RATIO, 0.15, poly=(26, 0.005, 8.0), poly_lo=(8, 0.005, 8.0))
    chi = lat.half_spinor()
    lat.gaussian_draw(0, 0, 5, 5, chi)
    phi = lat.half_spinor()
    lat.pf_heatbath(t, chi, wd.cg_params(tol=1e-10, prec=wd.F32, maxiter=20000), phi)
    S = lat.pf_action(t, phi, wd.cg_params(tol=1e-12))
    chi2 = float((chi * chi).sum())
    assert abs(S - chi2) < 1e-8 * chi2, (S, chi2)
    lat.close()


def test_integrate_on_caller_momenta():
    """integrate() (Section 2: T[eps] and S[eps]; Section 3.2: nested schedule) on
    caller-held momenta and pseudofermions, every step in FP64, against the
    oracle's integrator from the same links, momenta and phi: final links 1e-10,
    final momenta 1e-9 relative to max |P|."""
    import torch
    from paper_1702_00124_gb300 import wdhmc as wd
    from tests import gpu_util as gu
    dims = (4, 4, 4, 4)
    U0 = synthetic.gauge_field(dims, 0.3, 931)
    P0 = synthetic.momenta(dims, 932)
    k, kh, beta, tau = 0.124, 0.115, 5.6, 0.3
    pf = ChebyshevFilter(*POLY)
    terms_o = [actions.term("hasenbusch", k, kh), actions.term("poly", kh, poly=pf)]
    terms_g = [wd.term(wd.HASENBUSCH, k, kh), wd.term(wd.POLY, kh, poly=POLY)]
    phis = [lattice.mask(synthetic.spinor_field(dims, 933 + i), dims, 0) for i in range(2)]
    groups = [0, 1]
    levels = [(0, 2), (1, 1), (-1, 2)]

    def fog(grp, U):
        if grp == -1:
            return force.gauge_force(U, beta)
        return sum(force.fermion_force(U, t, ph) for t, ph, g in zip(terms_o, phis, groups) if g == grp)

    U1, P1 = hmc.integrate(U0, P0, hmc.nested(levels, tau, "omelyan"), fog)
    lat = wd.Lattice(dims)
    lat.wd_gauge_load(gu.dev(U0))
    Pe = gu.alg_to_dev(lat, P0)
    phis_e = [gu.pack(lat, ph, 0) for ph in phis]
    ops = wd.wd_schedule_nested(1, tau, [g for g, _ in levels], [n for _, n in levels])
    nf = lat.integrate(Pe, terms_g, groups, phis_e, beta, ops, wd.cg_params(tol=1e-14, maxiter=20000), wd.F64)
    assert nf > 0
    Ub = torch.zeros(2 * U0.size, dtype=torch.float64, device="cuda")
    lat.wd_gauge_store(Ub)
    assert np.max(np.abs(gu.host_c(Ub, U0.shape) - U1)) < 1e-10
    assert np.max(np.abs(gu.alg_to_host(lat, Pe) - P1)) < 1e-9 * np.max(np.abs(P1))
    with pytest.raises(wd.WdError):        # an op kind other than T or S
        lat.integrate(Pe, terms_g, groups, phis_e, beta, [(2, 0, 0.1)], wd.cg_params(), wd.F64)
    lat.close()


def test_trajectory_host_buffers_match_device():
    """hmc_trajectory_host (links in and out through host memory, one copy each
    way) gives the trajectory hmc_trajectory gives on the same links and draws."""
    import torch
    from paper_1702_00124_gb300 import wdhmc as wd
    from tests import gpu_util as gu
    dims = (4, 4, 4, 4)
    U0 = synthetic.gauge_field(dims, 0.3, 941)
    k, kh, beta, tau = 0.124, 0.115, 5.6, 0.4
    terms = [wd.term(wd.POLY, kh, poly=POLY), wd.term(wd.HASENBUSCH, k, kh)]
    groups = [1, 0]
    ops = wd.wd_schedule_nested(1, tau, [0, 1, -1], [2, 1, 2])
    p32 = wd.cg_params(tol=1e-10, prec=wd.F32, maxiter=20000)
    lat = wd.Lattice(dims)
    lat.wd_set_autotune(0)
    lat.wd_gauge_load(gu.dev(U0))
    r_dev = lat.hmc_trajectory(terms, groups, beta, ops, p32, p32, wd.F32, 55, 1, 0.25)
    Ub = torch.zeros(2 * U0.size, dtype=torch.float64, device="cuda")
    lat.wd_gauge_store(Ub)
    U_host = torch.from_numpy(np.ascontiguousarray(U0).view(np.float64).reshape(-1).copy()).pin_memory()
    U_out = torch.zeros_like(U_host).pin_memory()
    r_host = lat.hmc_trajectory_host(terms, groups, beta, ops, p32, p32, wd.F32, 55, 1, 0.25, U_host, U_out)
    assert abs(r_host["dH"] - r_dev["dH"]) <= 1e-12 * max(1.0, abs(r_dev["dH"]))
    assert r_host["accepted"] == r_dev["accepted"] and r_host["n_mat"] == r_dev["n_mat"]
    assert np.max(np.abs(U_out.numpy() - Ub.cpu().numpy())) < 1e-13
    U_in_place = U_host.clone().pin_memory()       # U_out may be U_in
    lat.hmc_trajectory_host(terms, groups, beta, ops, p32, p32, wd.F32, 55, 1, 0.25, U_in_place, U_in_place)
    assert np.max(np.abs(U_in_place.numpy() - Ub.cpu().numpy())) < 1e-13
    with pytest.raises(ValueError):               # device tensors are not host buffers
        lat.hmc_trajectory_host(terms, groups, beta, ops, p32, p32, wd.F32, 55, 1, 0.25, Ub, Ub)
    lat.close()
