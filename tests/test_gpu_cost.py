"""Cost driver on the GPU (Section 3.1, C = N_mat / P_acc): every action of the paper
runs a trajectory through the C ABI; each record's Metropolis decision is the host
test on its dH and uniform; the library's N_mat equals its K_hat counter; a sweep
leaves the links as it found them and orders its points by cost.  The trajectories
themselves are compared with the oracle in test_gpu_forces_hmc.py, and wd_cost with
the oracle's definition in test_cabi_host.py."""
import math

import numpy as np
import pytest

from paper_1702_00124_gb300 import synthetic

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)
POLY, POLY2 = (2, 0.02, 6.0), (8, 0.02, 6.0)


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1702_00124_gb300 import cost, wdhmc as wd
    lat = wd.Lattice(DIMS)
    U = synthetic.gauge_field(DIMS, 0.3, 4242)
    lat.wd_gauge_load(torch.from_numpy(U.view(np.float64).reshape(-1)).cuda())
    yield lat, cost, wd, torch
    lat.close()


@pytest.mark.parametrize("name", ["1PF", "1MP", "PF-MP", "2PF", "2MP", "1PF-2MP", "2PF-1MP"])
def test_every_action_runs(env, name):
    lat, cost, wd, _ = env
    terms = cost.action(name, 0.125, 0.11, POLY, POLY2, kappa_2=0.118)
    assert len(terms) == len(cost.ACTION_TERMS[name])
    ops = cost.schedule([3] + [4] * (len(terms) - 1), 8, tau=0.5)
    p = wd.cg_params(tol=1e-12, maxiter=20000)
    recs, c = cost.run(lat, terms, 5.6, ops, 3, seed=17, cg_md=p, cg_acc=p, force_prec=wd.F64)
    for r in recs:
        assert r["accepted"] == int(wd.metropolis(r["dH"], r["u"]))
        assert r["n_mat"] == r["n_mat_counter"] > 0
        assert math.isfinite(r["dH"])
    acc = np.mean([r["accepted"] for r in recs])
    assert c["p_acc"] == acc
    assert c["mean_nmat"] == np.mean([r["n_mat"] for r in recs])
    if acc > 0:
        assert abs(c["C"] - c["mean_nmat"] / acc) <= 1e-12 * c["C"]


def test_sweep_restores_links_and_orders_by_cost(env):
    lat, cost, wd, torch = env
    V = int(np.prod(DIMS))
    before = torch.empty(V * 72, dtype=torch.float64, device="cuda")
    lat.wd_gauge_store(before)
    terms = cost.action("1MP", 0.125, 0.11)
    p = wd.cg_params(tol=1e-12, maxiter=20000)
    rows = cost.sweep(lat, terms, 5.6, [([2, 4], 8), ([4, 8], 16)], 2, seed=5, tau=0.5,
                      cg_md=p, cg_acc=p, force_prec=wd.F64)
    after = torch.empty_like(before)
    lat.wd_gauge_store(after)
    assert torch.equal(before, after)
    assert [r["C_est"] for r in rows] == sorted(r["C_est"] for r in rows)
    assert {tuple(r["nsteps"]) for r in rows} == {(2, 4), (4, 8)}
    for r in rows:
        assert 0.0 <= r["p_acc"] <= 1.0 and r["mean_nmat"] > 0


def test_heatbath_noise_and_momenta_distributions(env):
    """Section 2: momenta with density exp(-sum tr P^2) and pseudofermion noise with
    density exp(-chi^dag chi).  With beta = 0 and one PLAIN term, H_0 = sum tr P^2 +
    chi^dag chi has mean 16 V (32 V coordinates, P_a ~ N(0, 1)) + 6 V (6 V complex
    components of variance 1) and standard deviation sqrt(22 V)."""
    import torch
    lat0, cost, wd, _ = env
    dims = (8, 8, 8, 8)
    V = int(np.prod(dims))
    lat = wd.Lattice(dims)
    U = synthetic.gauge_field(dims, 0.3, 99)
    lat.wd_gauge_load(torch.from_numpy(U.view(np.float64).reshape(-1)).cuda())
    ops = cost.schedule([1], 1, tau=1e-3)
    p = wd.cg_params(tol=1e-12, maxiter=20000)
    H0 = []
    for i in range(4):
        r = lat.hmc_trajectory([wd.term(wd.PLAIN, 0.12)], [0], 0.0, ops, p, p, wd.F64, 31, i, 0.5)
        H0.append(r["H0"])
    lat.close()
    assert abs(np.mean(H0) - 22 * V) < 5 * math.sqrt(22 * V / len(H0)), (np.mean(H0) / V, H0)


def test_hmc_exactness_identity(env):
    """<exp(-dH)> = 1 over an equilibrated chain (reversible, area-preserving
    integrator; momenta and pseudofermions from the conditional distributions of
    Section 2).  A wrong noise normalisation or an irreversible schedule moves it by
    orders of magnitude; 4^3 x 8, PLAIN at kappa = 0.14, leapfrog with 8 fermion and
    32 gauge steps, after pure-gauge thermalisation."""
    import torch
    _, cost, wd, _ = env
    dims = (4, 4, 4, 8)
    lat = wd.Lattice(dims)
    U = synthetic.gauge_field(dims, 0.5, 11)
    lat.wd_gauge_load(torch.from_numpy(U.view(np.float64).reshape(-1)).cuda())
    cost.run(lat, [], 5.6, wd.wd_schedule_generalised(1, 1.0, [-1], [20]), 200, 1)
    terms = [wd.term(wd.PLAIN, 0.14)]
    ops = cost.schedule([8], 32)
    cost.run(lat, terms, 5.6, ops, 40, 2, first_traj=1000)                 # settle with fermions
    _, c = cost.run(lat, terms, 5.6, ops, 160, 3, first_traj=2000)
    lat.close()
    assert c["p_acc"] > 0.5
    assert abs(c["exp_mdH"] - 1.0) < 4 * c["exp_mdH_err"] + 0.05, c
