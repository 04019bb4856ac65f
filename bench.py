"""Benchmark: HMC trajectories of the polynomial-filtered, mass-preconditioned
(PF-MP) two-flavour Wilson action on a 32^3 x 64 lattice, one GB300.

A step is one full trajectory (Section 2 of the paper): momentum and
pseudofermion heat bath, H, a nested multi-time-scale Omelyan 2MN integration
of tau = 1 with 10 outer steps, H again and the Metropolis test.  Workload
(synthetic, seeded): links exp(0.5 i H), kappa = 0.136, heavy kappa' = 0.128,
Chebyshev filter of degree 24 on [0.005, 8], Wilson gauge action beta = 5.6,
action S = phi1^dag P(J) phi1 + phi2^dag [P(J) J]^-1 phi2 + phi3^dag M_J K^-1 M_J^dag phi3
(Section 4.1), mixed precision (FP32 bulk, FP64 reliable updates to a 1e-10
true residual, FP64 links, momenta and H).

Prints one JSON line.  `value` = trajectories per second (whole job);
`roofline` = the FP32 hop stencil (the dominant kernel) sampled with CUDA
events inside the timed region; `cpu_baseline` = the oracle's K_hat on a
bounded sample, scaled to a trajectory by its K_hat count; `e2e` = the same
trajectory through the C ABI from host buffers.
  --impl reference  times the oracle (the reference arm of this benchmark).
Multi-GPU (torchrun): every rank runs an independent replica (different
seed); value = all ranks' trajectories / max time.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "M†M stencil HBM GB/s and CG/force/trajectory time, mixed vs FP64 at 1e-10 resid"
WORKLOADS = {
    # name: dims, link scale a, kappa, kappa', filter (n, eps, lam), beta, outer steps
    "c5_32x32x32x64": dict(dims=(32, 32, 32, 64), a=0.5, kappa=0.136, kappa_h=0.128,
                           poly=(24, 0.005, 8.0), beta=5.6, tau=1.0, n_outer=10),
    "c3_16x16x16x32": dict(dims=(16, 16, 16, 32), a=0.5, kappa=0.136, kappa_h=0.128,
                           poly=(24, 0.005, 8.0), beta=5.6, tau=1.0, n_outer=10),
}
DEFAULT_WORKLOAD = "c5_32x32x32x64"
# Integrator levels, outermost first: (group, steps per enclosing T).
# group 0: filtered + Hasenbusch terms, group 1: P(J) term, -1: gauge action.
LEVELS = [(0, 10), (1, 1), (-1, 2)]
# Residual recomputation of the mixed-precision solves: 0 = FP64, 1 =
# double-float (2 x FP32, about 44-48 bits; b, x, r and dots stay FP64).
# At this volume the double-float hop takes 0.50-0.58 ms against 2.08 ms in FP64.
RESIDUAL_MODE = 1
# K_hat applications of one trajectory of the default workload, counted by
# the library's N_mat counter (algorithmic count; the reference arm scales
# its per-K_hat time by it).
N_MAT_PER_TRAJ = 20305
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "hop_f32_c5_32x32x32x64.md")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profiled_traffic():
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu summary."""
    try:
        for line in open(PROFILE_SUMMARY):
            if line.startswith("traffic_bytes_per_launch:"):
                v = line.split(":", 1)[1].strip()
                return None if v == "null" else float(v)
    except OSError:
        pass
    return None


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        load = [s for s in sm if s > 0.5 * max(sm)]
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_khat_seconds(reps=2):
    """Oracle K_hat on a 32^3 x 4 slab (the workload's spatial volume, 1/16 of its
    sites), seconds per application scaled to the full 32^3 x 64 lattice."""
    from oracle import lattice, wilson
    from paper_1702_00124_gb300 import synthetic
    w = WORKLOADS[DEFAULT_WORKLOAD]
    slab = (32, 32, 32, 4)
    U = synthetic.gauge_field(slab, w["a"], synthetic.SEED_BASE + 40)
    psi = lattice.mask(synthetic.spinor_field(slab, synthetic.SEED_BASE + 41), slab, 0)
    wilson.apply_Khat(U, psi, w["kappa"])          # warm
    t = time.perf_counter()
    for _ in range(reps):
        wilson.apply_Khat(U, psi, w["kappa"])
    per = (time.perf_counter() - t) / reps
    scale = np.prod(w["dims"]) / np.prod(slab)
    return per * scale, f"oracle K_hat on a 32x32x32x4 slab ({reps} applications, x{scale:.0f} volume)"


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    steps = []
    sample = ""
    for i in range(args.warmup + args.steps):
        per_khat, sample = oracle_khat_seconds(reps=1)
        if i >= args.warmup:
            steps.append(per_khat * N_MAT_PER_TRAJ)
    t_traj = float(np.mean(steps))
    value = 1.0 / t_traj
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "trajectories/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_traj * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "dims": list(w["dims"])},
            "cpu_baseline": {"value": value, "unit": "trajectories/s", "cores": 1, "kind": "oracle",
                             "sample": sample + f", scaled by N_mat = {N_MAT_PER_TRAJ} K_hat per trajectory"},
            "e2e": {"value": value, "unit": "trajectories/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def max_over_ranks(seconds, dist, device):
    """Slowest rank's timed region (every rank runs an independent replica)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def replica_throughput(world, steps, t_max):
    """Whole-job trajectories per second: all ranks' trajectories / slowest rank."""
    return world * steps / t_max


def batched_workload_run(wd):
    """The batched workload: 24 lattices (8 x 8^4, 8 x 12^3 x 24, 8 x 16^3 x 32),
    links exp(0.4 i H), kappa ~ U[0.125, 0.135], 4 Gaussian right-hand sides
    each, mixed-precision CG of all 96 systems to 1e-10 (CUDA-graph chunks)."""
    import torch
    from paper_1702_00124_gb300 import synthetic
    work = synthetic.batched_workload()
    stream = torch.cuda.current_stream()
    lats, bs, xs = [], [], []
    for w in work:
        U = synthetic.gauge_field(w["dims"], w["a"], w["seed"])
        lat = wd.Lattice(w["dims"], stream=stream)
        lat.wd_gauge_load(torch.from_numpy(U.view(np.float64).reshape(-1)).cuda())
        lat.wd_set_recon(wd.RECON_12)
        b = torch.empty(w["nrhs"] * 24 * lat.Vh, dtype=torch.float64, device="cuda")
        for r in range(w["nrhs"]):
            lat.gaussian_draw(0, 0, w["seed"], 10 + r, b[r * 24 * lat.Vh:(r + 1) * 24 * lat.Vh])
        lats.append(lat)
        bs.append(b)
        xs.append(torch.zeros_like(b))
    batch = wd.Batch(lats, [w["kappa"] for w in work], [w["nrhs"] for w in work])
    p = wd.cg_params(tol=1e-10, prec=wd.F32)
    batch.wd_batch_cg(bs, xs, p, True)          # tunes, captures the graph
    torch.cuda.synchronize()
    t = time.perf_counter()
    infos = batch.wd_batch_cg(bs, xs, p, True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    info = batch.wd_batch_info()
    out = {"s": dt, "systems": info["systems"], "systems_per_s": info["systems"] / dt,
           "max_true_rel_resid": max(i["true_rel_resid"] for i in infos),
           "max_iters": max(i["iters"] for i in infos), "block_threads": info["threads"]}
    batch.close()
    for lat in lats:
        lat.close()
    return out


def kernel_case(args):
    """K_hat alone on the workload's lattice: the launch sequence ncu captures."""
    import torch
    from paper_1702_00124_gb300 import synthetic, wdhmc as wd
    w = WORKLOADS[args.workload]
    dims = w["dims"]
    U = synthetic.gauge_field(dims, w["a"], synthetic.SEED_BASE + 4)
    lat = wd.Lattice(dims)
    U_dev = torch.from_numpy(U.view(np.float64).reshape(-1)).to("cuda")
    lat.wd_gauge_load(U_dev)
    del U_dev
    lat.wd_set_autotune(0)     # the default launch shape, as production settles on
    prec, recon = {"khat_f32_recon12": (wd.F32, 1), "khat_bf16_recon12": (wd.BF16, 1),
                   "khat_f64": (wd.F64, 0), "khat_df": (wd.DF, 0),
                   "poly_f32_recon12": (wd.F32, 1)}[args.kernel_case]
    lat.wd_set_recon(recon)
    x, y = lat.half_spinor(), lat.half_spinor()
    lat.gaussian_draw(0, 0, 1, 1, x)
    for _ in range(args.reps):
        if args.kernel_case.startswith("poly"):
            lat.poly_filter_apply(w["kappa_h"], (4, w["poly"][1], w["poly"][2]), prec, x, y)
        else:
            lat.mdagm_apply(w["kappa"], prec, 1, x, y)
    torch.cuda.synchronize()
    lat.close()
    print(f"kernel case {args.kernel_case} on {args.workload}: {args.reps} K_hat applications")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-extras", action="store_true", help="skip the mixed-vs-FP64 and e2e measurements")
    ap.add_argument("--kernel-case", choices=["khat_f32_recon12", "khat_bf16_recon12", "khat_f64", "khat_df",
                                              "poly_f32_recon12"],
                    help="only apply K_hat --reps times on the workload (for ncu captures); prints no JSON")
    ap.add_argument("--reps", type=int, default=4)
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.kernel_case:
        return kernel_case(args)

    import torch
    from paper_1702_00124_gb300 import synthetic, wdhmc as wd

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    w = WORKLOADS[args.workload]
    dims = w["dims"]
    seed = synthetic.SEED_BASE + 4 + 1000 * rank
    U = synthetic.gauge_field(dims, w["a"], seed)
    U_host = torch.from_numpy(U.view(np.float64).reshape(-1)).pin_memory()
    lat = wd.Lattice(dims)
    lat.wd_set_recon(wd.RECON_12)
    lat.wd_set_residual(RESIDUAL_MODE)
    U_dev = U_host.to("cuda", non_blocking=True)
    lat.wd_gauge_load(U_dev)
    terms = [wd.term(wd.POLY, w["kappa_h"], poly=w["poly"]), wd.term(wd.FILTERED, w["kappa_h"], poly=w["poly"]),
             wd.term(wd.HASENBUSCH, w["kappa"], w["kappa_h"])]
    groups = [1, 0, 0]
    ops = wd.wd_schedule_nested(1, w["tau"], [g for g, _ in LEVELS], [n for _, n in LEVELS])
    cg_md = wd.cg_params(tol=1e-10, prec=wd.F32, maxiter=20000)
    cg_acc = wd.cg_params(tol=1e-10, prec=wd.F32, maxiter=20000)
    traj = [0]
    results = []

    def trajectory():
        u = synthetic.uniform(seed + traj[0])
        r = lat.hmc_trajectory(terms, groups, w["beta"], ops, cg_md, cg_acc, wd.F32, seed, traj[0], u)
        traj[0] += 1
        results.append(r)
        return r

    for _ in range(args.warmup):
        trajectory()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    # every 7th hop launch: co-prime with the 4-hop cycle of K_hat, so every
    # variant (plain, xpay, dagger) is sampled
    lat.wd_profile_enable(7)
    l0, n0 = lat.wd_launch_count(), lat.wd_nmat()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        trajectory()
    e1.record(stream)
    torch.cuda.synchronize()
    elapsed = e0.elapsed_time(e1) / 1e3
    launches = lat.wd_launch_count() - l0
    nmat = (lat.wd_nmat() - n0) / args.steps
    prof = lat.wd_profile_read(wd.F32)
    prof64 = lat.wd_profile_read(wd.F64)
    counts = lat.wd_hop_counts()
    lat.wd_profile_enable(0)
    # share of the timed region spent in each hop family: all launches of the
    # family x its average sampled duration
    shares = {}
    for name, pr, n in (("k_hop_fp32", prof, counts[wd.F32]), ("k_hop_fp64", prof64, counts[wd.F64])):
        if pr["launches"]:
            shares[name] = {"launches": n, "avg_ms": pr["ms"] / pr["launches"],
                            "share": n * pr["ms"] / pr["launches"] / (elapsed * 1e3)}
    clk = clocks.stop()
    t_max = max_over_ranks(elapsed, dist, "cuda")
    timed = results[-args.steps:]
    value = replica_throughput(world, args.steps, t_max)

    hbm, peak_kind = peaks()
    achieved = prof["bytes"] / (prof["ms"] * 1e-3) / 1e9 if prof["ms"] > 0 else None
    traffic = profiled_traffic()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": (achieved / hbm) if achieved else None,
                "traffic": traffic, "kernel": "k_hop_st FP32 (all variants, links staged by cp.async), 12-real links",
                "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured" else "fallback",
                "sampled_launches": prof["launches"],
                "algorithmic_bytes_per_launch": prof["bytes"] / max(prof["launches"], 1),
                "avg_launch_ms": prof["ms"] / max(prof["launches"], 1)}

    extras = {}
    e2e = None
    cpu = None
    if rank == 0 and not args.no_extras:
        # end to end through the C ABI from pinned host buffers, one trajectory
        out_host = torch.empty_like(U_host).pin_memory()
        torch.cuda.synchronize()
        t = time.perf_counter()
        U_dev.copy_(U_host, non_blocking=True)
        lat.wd_gauge_load(U_dev)
        r = trajectory()
        lat.wd_gauge_store(U_dev)
        out_host.copy_(U_dev, non_blocking=True)
        torch.cuda.synchronize()
        dh = float(r["dH"])
        t_e2e = time.perf_counter() - t
        nbytes = U_host.numel() * 8
        e2e = {"value": 1.0 / t_e2e, "unit": "trajectories/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes + 8, "dH": dh}
        # mixed vs FP64: one CG solve and one force evaluation of the Hasenbusch term
        chi = lat.half_spinor()
        lat.gaussian_draw(0, 0, 7, 7, chi)
        b = lat.half_spinor()
        lat.wd_apply(w["kappa"], True, wd.F64, chi, b)
        F = lat.algebra_field()
        runs = (("fp64", wd.F64, 0), ("mixed_fp32_fp64resid", wd.F32, 0), ("mixed_fp32", wd.F32, RESIDUAL_MODE),
                ("mixed_bf16", wd.BF16, RESIDUAL_MODE))
        for name, prec, rmode in runs:
            lat.wd_set_residual(rmode)
            x = lat.half_spinor()
            torch.cuda.synchronize()
            t = time.perf_counter()
            info = lat.cg_solve(w["kappa"], b, x, wd.cg_params(tol=1e-10, prec=prec, maxiter=20000))
            torch.cuda.synchronize()
            extras[f"cg_{name}"] = {"s": time.perf_counter() - t, "iters": info["iters"],
                                    "reliable_updates": info["reliable_updates"],
                                    "true_rel_resid": info["true_rel_resid"]}
            if name in ("fp64", "mixed_fp32"):
                torch.cuda.synchronize()
                t = time.perf_counter()
                lat.fermion_force(terms[2], chi, wd.cg_params(tol=1e-10, prec=prec), 1.0, F)
                torch.cuda.synchronize()
                extras[f"force_hasenbusch_{name}"] = {"s": time.perf_counter() - t}
            # the filtered term's solve: the FP64-residual cost centre
            if name in ("mixed_fp32_fp64resid", "mixed_fp32"):
                x = lat.half_spinor()
                torch.cuda.synchronize()
                t = time.perf_counter()
                info = lat.cg_solve(w["kappa_h"], b, x, wd.cg_params(tol=1e-10, prec=prec), filt=w["poly"])
                torch.cuda.synchronize()
                extras[f"filtered_cg_{name}"] = {"s": time.perf_counter() - t, "iters": info["iters"],
                                                 "reliable_updates": info["reliable_updates"],
                                                 "true_rel_resid": info["true_rel_resid"]}
        lat.wd_set_residual(RESIDUAL_MODE)
        # stand-alone K_hat bandwidth per precision (10 applications each)
        out = lat.half_spinor()
        for name, prec, recon in (("fp64", wd.F64, 0), ("double_float", wd.DF, 0), ("fp32", wd.F32, 0),
                                  ("fp32_recon12", wd.F32, 1), ("bf16_recon12", wd.BF16, 1)):
            lat.wd_set_recon(recon)
            lat.wd_profile_enable(1)
            lat.mdagm_apply(w["kappa"], prec, 1, chi, out)
            lat.wd_profile_enable(1)
            for _ in range(10):
                lat.mdagm_apply(w["kappa"], prec, 1, chi, out)
            pr = lat.wd_profile_read(prec)
            extras[f"hop_{name}"] = {"GBs": pr["bytes"] / (pr["ms"] * 1e-3) / 1e9,
                                     "ms_per_hop": pr["ms"] / max(pr["launches"], 1)}
        lat.wd_set_recon(wd.RECON_12)
        lat.wd_profile_enable(0)
        extras["batched_24_lattices_x4_rhs"] = batched_workload_run(wd)
        per_khat, sample = oracle_khat_seconds(reps=2)
        cpu_traj = per_khat * nmat
        cpu = {"value": 1.0 / cpu_traj, "unit": "trajectories/s", "cores": 1, "kind": "oracle",
               "sample": sample + f", scaled by this run's N_mat = {nmat:.0f} K_hat per trajectory"}

    if rank == 0:
        acc = [int(r["accepted"]) for r in timed]
        line = {"metric": METRIC, "value": value, "unit": "trajectories/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": args.workload, "dims": list(dims), "kappa": w["kappa"],
                           "kappa_h": w["kappa_h"], "poly": list(w["poly"]), "beta": w["beta"],
                           "integrator": "nested Omelyan 2MN", "levels": LEVELS, "tau": w["tau"],
                           "action": "PF-MP + Wilson gauge",
                           "precision": "FP32 bulk (12-real links); reliable updates with b, x, r, dots in FP64 and "
                                        + ("A x in double-float (2xFP32, ~48 bits)" if RESIDUAL_MODE else "A x in FP64")
                                        + "; links, momenta, H in FP64",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "l2": "working set (1.2 GB FP64 links + FP32 copies) far above the 126 MB L2"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "hop_time_shares": shares,
                "clocks": clk,
                "trajectory": {"dH": [float(r["dH"]) for r in timed], "accepted": acc,
                               "n_mat_per_traj": nmat, "force_evals": [r["n_force_evals"] for r in timed],
                               "integrator_ops": len(ops),
                               # device time per phase of the last timed trajectory (ms)
                               "phases_ms": {"heatbath": timed[-1]["t_heatbath_ms"],
                                             "hamiltonians": timed[-1]["t_hamiltonian_ms"],
                                             "T_steps": timed[-1]["t_T_ms"],
                                             "gauge_force": timed[-1]["t_gauge_force_ms"],
                                             "force_filtered_and_hasenbusch": timed[-1]["t_force_group_ms"][0],
                                             "force_poly": timed[-1]["t_force_group_ms"][1]}},
                "breakdown": extras,
                "autotuned_hop_shapes": {str(k): list(v) for k, v in lat.tuned().items()}}
        print(json.dumps(line))
    lat.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
