"""Cost of an HMC action and sweeps of its step sizes (Section 3.1: C = N_mat / P_acc;
Sections 3.1-3.3 and 4.1-4.2 for the actions).

Every action here is S_G plus pseudofermion terms of the library's kinds, each on its
own integration time scale (Section 3.1: step sizes h_G < h_1 < h_2 ..., n_i steps of
term i per trajectory, tau = h_i n_i), combined by the generalised scheme of Section
3.2.  One measurement runs trajectories through hmc_trajectory (heat bath, integration,
Metropolis test, all in the library), and reduces their records with wd_cost:

    C = <N_mat> / P_acc          N_mat: K_hat multiplications the library counted
    C_est = <N_mat> / <min(1, exp(-dH))>     the same with the smoother estimator

The paper tunes the step sizes by balancing the forces of the terms (a method it only
cites); `sweep` instead scans a grid of step counts and keeps the cheapest point.
This module is orchestration over the C ABI: no arithmetic of the method runs here.
"""
import math

import numpy as np
import torch

from . import wdhmc as wd

# action name -> pseudofermion terms, outermost (coarsest step) first
ACTION_TERMS = {
    "1PF": ["filtered(P, k)", "poly(P, k)"],
    "1MP": ["hasenbusch(k over k')", "plain(k')"],
    "PF-MP": ["hasenbusch(k over k')", "filtered(P, k')", "poly(P, k')"],
    "2PF": ["filtered(P2, k)", "ratio(P2/P1, k)", "poly(P1, k)"],
    "2MP": ["hasenbusch(k over k2)", "hasenbusch(k2 over k1)", "plain(k1)"],
    "1PF-2MP": ["hasenbusch(k over k2)", "hasenbusch(k2 over k1)", "filtered(P, k1)", "poly(P, k1)"],
    "2PF-1MP": ["hasenbusch(k over k')", "filtered(P2, k')", "ratio(P2/P1, k')", "poly(P1, k')"],
}


def action(name, kappa, kappa_h=None, poly=None, poly2=None, kappa_2=None):
    """Terms of one of the paper's actions (ACTION_TERMS), outermost first.

    kappa: the quark's hopping parameter; kappa_h: the heavier kappa' (1MP, PF-MP,
    2PF-1MP) or kappa_1 (2MP, 1PF-2MP); kappa_2: the middle kappa of 2MP / 1PF-2MP
    (kappa_1 < kappa_2 < kappa); poly = (n, eps, lam) of P (or P_1); poly2 of P_2."""
    T = wd.term
    if name == "1PF":
        return [T(wd.FILTERED, kappa, poly=poly), T(wd.POLY, kappa, poly=poly)]
    if name == "1MP":
        return [T(wd.HASENBUSCH, kappa, kappa_h), T(wd.PLAIN, kappa_h)]
    if name == "PF-MP":
        return [T(wd.HASENBUSCH, kappa, kappa_h), T(wd.FILTERED, kappa_h, poly=poly),
                T(wd.POLY, kappa_h, poly=poly)]
    if name == "2PF":
        return [T(wd.FILTERED, kappa, poly=poly2), T(wd.RATIO, kappa, poly=poly2, poly_lo=poly),
                T(wd.POLY, kappa, poly=poly)]
    if name == "2MP":
        return [T(wd.HASENBUSCH, kappa, kappa_2), T(wd.HASENBUSCH, kappa_2, kappa_h), T(wd.PLAIN, kappa_h)]
    if name == "1PF-2MP":
        return [T(wd.HASENBUSCH, kappa, kappa_2), T(wd.HASENBUSCH, kappa_2, kappa_h),
                T(wd.FILTERED, kappa_h, poly=poly), T(wd.POLY, kappa_h, poly=poly)]
    if name == "2PF-1MP":
        return [T(wd.HASENBUSCH, kappa, kappa_h), T(wd.FILTERED, kappa_h, poly=poly2),
                T(wd.RATIO, kappa_h, poly=poly2, poly_lo=poly), T(wd.POLY, kappa_h, poly=poly)]
    raise ValueError(f"unknown action {name!r}; one of {sorted(ACTION_TERMS)}")


def schedule(nsteps, n_gauge, tau=1.0, kind=0):
    """Generalised scheme (Section 3.2): term i (group i) with nsteps[i] steps, the
    gauge force (group -1) with n_gauge steps, over trajectory length tau.
    kind 0 = leapfrog, 1 = Omelyan 2MN."""
    groups = list(range(len(nsteps))) + [-1]
    return wd.wd_schedule_generalised(kind, tau, groups, list(nsteps) + [n_gauge])


def run(lat, terms, beta, ops, n_traj, seed, first_traj=0, cg_md=None, cg_acc=None, force_prec=wd.F32):
    """n_traj trajectories with the Metropolis test (uniforms from a generator seeded
    by `seed`); returns the per-trajectory records and their wd_cost reduction."""
    if n_traj < 1:
        raise ValueError("n_traj must be >= 1")
    cg_md = cg_md or wd.cg_params(tol=1e-8, prec=wd.F32, maxiter=50000)
    cg_acc = cg_acc or wd.cg_params(tol=1e-10, prec=wd.F32, maxiter=50000)
    groups = list(range(len(terms)))
    rng = np.random.default_rng(seed)
    recs = []
    for i in range(n_traj):
        u = float(rng.random())
        n0 = lat.wd_nmat()
        r = lat.hmc_trajectory(terms, groups, beta, ops, cg_md, cg_acc, force_prec, seed, first_traj + i, u)
        r["u"] = u
        r["n_mat_counter"] = lat.wd_nmat() - n0
        recs.append(r)
    cost = wd.wd_cost([r["n_mat"] for r in recs], [r["accepted"] for r in recs], [r["dH"] for r in recs])
    return recs, cost


def sweep(lat, terms, beta, grid, n_traj, seed, first_traj=0, tau=1.0, kind=0, **kw):
    """For each (nsteps, n_gauge) of grid: `run` from the current links, which are
    restored before the next point, so every point starts from the same field.
    Returns rows sorted by C_est (the cheapest first)."""
    U0 = torch.empty(int(np.prod(lat.dims)) * 4 * 18, dtype=torch.float64, device="cuda")
    lat.wd_gauge_store(U0)
    rows = []
    for j, (nsteps, n_gauge) in enumerate(grid):
        lat.wd_gauge_load(U0)
        ops = schedule(nsteps, n_gauge, tau, kind)
        _, c = run(lat, terms, beta, ops, n_traj, seed + 7919 * j, first_traj + 1000 * j, **kw)
        rows.append(dict(nsteps=list(nsteps), n_gauge=n_gauge, **c))
    lat.wd_gauge_load(U0)
    return sorted(rows, key=lambda r: r["C_est"])


def main(argv=None):
    """Command line: thermalise a synthetic field with one action, then sweep the
    step counts of each requested action from that field; one JSON line per grid
    point (cost, acceptance, <exp(-dH)>) and a summary line per action."""
    import argparse
    import json
    from . import synthetic
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--dims", type=int, nargs=4, default=[8, 8, 8, 8])
    ap.add_argument("--beta", type=float, default=5.6)
    ap.add_argument("--kappa", type=float, default=0.150)
    ap.add_argument("--kappa-h", type=float, default=0.140, help="kappa' (or kappa_1 for 2MP / 1PF-2MP)")
    ap.add_argument("--kappa-2", type=float, default=0.145, help="middle kappa of 2MP / 1PF-2MP")
    ap.add_argument("--poly", type=float, nargs=3, default=[8, 0.005, 8.0], help="n eps lam of P (P_1)")
    ap.add_argument("--poly2", type=float, nargs=3, default=[26, 0.005, 8.0], help="n eps lam of P_2")
    ap.add_argument("--actions", nargs="+", default=["1PF", "1MP", "PF-MP"])
    ap.add_argument("--scales", type=int, nargs="+", default=[6, 8, 12, 16],
                    help="outermost step counts of the grid; inner terms take 2x, the gauge 4x")
    ap.add_argument("--therm-gauge", type=int, default=200, help="pure-gauge thermalisation trajectories")
    ap.add_argument("--gauge-steps", type=int, default=40, help="Omelyan steps of a pure-gauge trajectory")
    ap.add_argument("--therm", type=int, default=40, help="thermalisation trajectories with fermions")
    ap.add_argument("--traj", type=int, default=20)
    ap.add_argument("--seed", type=int, default=20170201)
    a = ap.parse_args(argv)
    poly = (int(a.poly[0]), a.poly[1], a.poly[2])
    poly2 = (int(a.poly2[0]), a.poly2[1], a.poly2[2])
    lat = wd.Lattice(a.dims)
    U = synthetic.gauge_field(a.dims, 0.3, a.seed)
    lat.wd_gauge_load(torch.from_numpy(U.view(np.float64).reshape(-1)).cuda())
    vol = int(np.prod(a.dims))

    def plaquette():
        return 1.0 - lat.gauge_action(a.beta) / (6 * vol * a.beta)

    # pure-gauge trajectories bring the links near the equilibrium plaquette cheaply,
    # then trajectories with the fermions (PF-MP, steps twice as fine as the finest
    # grid point) finish the thermalisation.  Far from equilibrium the forces are
    # large: too coarse a step there gives |dH| >> 1 and a chain that never moves
    # (dH > 0) or drifts on integration error (dH < 0).
    _, c = run(lat, [], a.beta, wd.wd_schedule_generalised(1, 1.0, [-1], [a.gauge_steps]), a.therm_gauge, a.seed)
    print(json.dumps({"thermalisation": "pure gauge", "trajectories": a.therm_gauge, "p_acc": c["p_acc"],
                      "mean_plaquette": plaquette()}), flush=True)
    terms = action("PF-MP", a.kappa, a.kappa_h, poly)
    n0 = 2 * max(a.scales)
    recs, c = run(lat, terms, a.beta, schedule([n0, 2 * n0, 2 * n0], 4 * n0), a.therm, a.seed + 1,
                  first_traj=a.therm_gauge)
    tail = wd.wd_cost([r["n_mat"] for r in recs[-10:]], [r["accepted"] for r in recs[-10:]],
                      [r["dH"] for r in recs[-10:]])
    print(json.dumps({"thermalisation": "PF-MP", "trajectories": a.therm, "p_acc": c["p_acc"],
                      "mean_plaquette": plaquette(), "last10_exp_mdH": tail["exp_mdH"],
                      "last10_exp_mdH_err": tail["exp_mdH_err"]}), flush=True)
    for i, name in enumerate(a.actions):
        terms = action(name, a.kappa, a.kappa_h, poly, poly2, a.kappa_2)
        grid = [([s] + [2 * s] * (len(terms) - 1), 4 * s) for s in a.scales]
        rows = sweep(lat, terms, a.beta, grid, a.traj, a.seed + 100 * (i + 1), first_traj=10 ** 6)
        for r in rows:
            print(json.dumps({"action": name, **r}), flush=True)
        print(json.dumps({"action": name, "best": rows[0]["nsteps"] + [rows[0]["n_gauge"]],
                          "C": rows[0]["C"], "C_est": rows[0]["C_est"]}), flush=True)
    lat.close()


if __name__ == "__main__":
    main()
