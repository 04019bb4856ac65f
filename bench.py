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
events inside the timed region; `cpu_baseline` = the oracle timed on the host
cores (per kernel on one core; one K_hat of the workload over every core,
scaled to a trajectory by this run's K_hat count); `e2e` = the same
trajectories through the C ABI's host-buffer call; `breakdown` = mixed vs FP64
CG / force / trajectory at 32^3 x 64 and 16^3 x 32, the batched workload, and
the error against the FP64 oracle of a solution, a force and a dH.
  --impl reference  times the oracle (the reference arm of this benchmark).
Multi-GPU (torchrun): every rank runs an independent replica (different
seed); value = all ranks' trajectories / max time.
"""
import argparse
import json
import os
import subprocess
import sys
import platform
import tempfile
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
STENCILS = {"thread": 0, "tile": 1}
# Integrator levels, outermost first: (group, steps per enclosing T).
# group 0: filtered + Hasenbusch terms, group 1: P(J) term, -1: gauge action.
LEVELS = [(0, 10), (1, 1), (-1, 2)]
# Residual recomputation of the mixed-precision solves: 0 = FP64, 1 =
# double-float (2 x FP32, about 44-48 bits; b, x, r and dots stay FP64).
# At this volume the double-float hop takes 0.50-0.58 ms against 2.08 ms in FP64.
RESIDUAL_MODE = 1
# K_hat applications of one trajectory of the default workload: the library's
# N_mat counter over the timed trajectories of `python bench.py` (two after three
# warm-ups: 18,710; 18,710-18,800 in other runs of the same seeded chain).  The
# reference arm, which runs no GPU code, scales its per-K_hat time by it; the GPU
# arm's CPU baseline uses the count of its own run.
N_MAT_PER_TRAJ = 18710
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


def host_info():
    """Host description for the CPU legs: cores and CPU model."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model Name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or "unknown",
            "machine": platform.machine()}


# ---------------------------------------------------------------------------
# The oracle (FP64 numpy, as it stands) timed on the host cores.  Workers are
# spawned processes (the parent may hold a CUDA context) and import only numpy
# and the oracle.  A c5 K_hat's work is done as 16 slabs of 32^3 x 4 sites (the
# workload's spatial volume, 1/16 of its sites), one per task.
SLAB = (32, 32, 32, 4)
N_SLABS = 16
_W = {}


def _worker_init():
    from oracle import lattice
    from paper_1702_00124_gb300 import synthetic
    w = WORKLOADS[DEFAULT_WORKLOAD]
    _W["U"] = synthetic.gauge_field(SLAB, w["a"], synthetic.SEED_BASE + 40)
    _W["psi"] = lattice.mask(synthetic.spinor_field(SLAB, synthetic.SEED_BASE + 41), SLAB, 0)
    _W["kappa"] = w["kappa"]


def _slab_khat(_):
    from oracle import wilson
    t = time.perf_counter()
    wilson.apply_Khat(_W["U"], _W["psi"], _W["kappa"])
    return time.perf_counter() - t


def _single_thread_suite():
    """Oracle per kernel on one core (seconds): K_hat at c1, c2, c3 and the c5 slab;
    CG to a 1e-10 true residual at c1, c2; the plain-term force with its solve at c1
    and the force from given X, Y at c3.  Also returns the c2 solution and the c1 force
    (the references of the GPU error legs)."""
    from oracle import actions, force, lattice, wilson
    from oracle.cg import cg
    from paper_1702_00124_gb300 import synthetic
    out, refs = {}, {}
    for name in ("c1_4x4x4x4", "c2_8x8x8x16", "c3_16x16x16x32"):
        w = synthetic.WORKLOADS[name]
        dims, k = w["dims"], w["kappa"]
        U = synthetic.gauge_field(dims, w["a"], w["seed"])
        chi = lattice.mask(synthetic.spinor_field(dims, w["seed"] + 100), dims, 0)
        t = time.perf_counter()
        wilson.apply_Khat(U, chi, k)
        out[f"khat_{name}_s"] = time.perf_counter() - t
        b = wilson.apply_Mhat(U, chi, k, dagger=True)
        if name != "c3_16x16x16x32":
            t = time.perf_counter()
            X, info = cg(actions.K_op(U, k), b, 1e-10)
            out[f"cg_{name}_s"] = time.perf_counter() - t
            out[f"cg_{name}_iters"] = info["iters"]
            refs[f"X_{name}"] = X
        if name == "c1_4x4x4x4":
            t = time.perf_counter()
            refs["F_c1"] = force.fermion_force(U, actions.term("plain", k), b, tol=1e-12)
            out["force_plain_c1_s"] = time.perf_counter() - t
        if name == "c3_16x16x16x32":
            Y = wilson.apply_Mhat(U, chi, k)
            t = time.perf_counter()
            -2 * force._dre_mhat(U, Y, chi, k)
            out["force_xy_c3_s"] = time.perf_counter() - t
    out["khat_c5_slab_s"] = (_worker_init(), _slab_khat(0))[1]
    return out, refs


def _oracle_dH_c1():
    """dH of one FP64 oracle trajectory at 4^4 (the error leg's reference)."""
    from oracle import actions, force, hmc, lattice, philox
    from oracle.poly import ChebyshevFilter
    from paper_1702_00124_gb300 import synthetic
    c = DH_LEG
    U0 = synthetic.gauge_field(c["dims"], c["a"], c["seed"])
    pf = ChebyshevFilter(*c["poly"])
    terms = [actions.term("poly", c["kappa_h"], poly=pf), actions.term("filtered", c["kappa_h"], poly=pf),
             actions.term("hasenbusch", c["kappa"], c["kappa_h"])]
    V = int(np.prod(c["dims"]))
    base = c["traj"] * 64
    P0 = philox.gaussian_field(V * 32, c["draw_seed"], base).reshape(lattice.shape(c["dims"]) + (4, 8))
    phis = []
    for i, t in enumerate(terms):
        g = philox.gaussian_field(V * 24, c["draw_seed"], base + 1 + i)
        chi = lattice.mask(g.view(np.complex128).reshape(lattice.shape(c["dims"]) + (4, 3)), c["dims"], 0)
        phis.append(actions.heatbath(U0, t, chi / np.sqrt(2), tol=1e-12))

    def H(U, P):
        return hmc.kinetic(P) + force.gauge_action(U, c["beta"]) + sum(
            actions.action(U, t, ph, tol=1e-12)[0] for t, ph in zip(terms, phis))

    def fog(grp, U):
        if grp == -1:
            return force.gauge_force(U, c["beta"])
        return sum(force.fermion_force(U, t, ph, tol=1e-12) for t, ph, g in zip(terms, phis, c["groups"])
                   if g == grp)

    U1, P1 = hmc.integrate(U0, P0, hmc.nested(c["levels"], c["tau"], "omelyan"), fog)
    return H(U1, P1) - H(U0, P0)


# The dH error leg: PF-MP + gauge at 4^4 with the trajectory bench's structure
DH_LEG = dict(dims=(4, 4, 4, 4), a=0.3, seed=951, kappa=0.124, kappa_h=0.115, beta=5.6, tau=0.5,
              poly=(8, 0.02, 6.0), groups=[1, 0, 0], levels=[(0, 3), (1, 1), (-1, 2)], draw_seed=321, traj=2)


def spawn_pool(n):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(n, initializer=_worker_init)


def c5_khat_all_cores(pool, reps=1):
    """Wall time of one c5 K_hat's work (16 slab applications) over the pool."""
    best = None
    for _ in range(reps):
        t = time.perf_counter()
        pool.map(_slab_khat, range(N_SLABS), chunksize=1)
        dt = time.perf_counter() - t
        best = dt if best is None else min(best, dt)
    return best


def run_reference(args, rank, world):
    """The reference arm: the oracle on the host cores.  One step = one K_hat of the
    32^3 x 64 workload (16 slab applications spread over every core), the unit of the
    cost metric (Section 3.1); a trajectory is N_MAT_PER_TRAJ of them, which sets
    `value`.  ms_per_step is the step's own measured time."""
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    host = host_info()
    n = host["nproc"] or 1
    pool = spawn_pool(min(n, N_SLABS))
    try:
        for _ in range(args.warmup):
            c5_khat_all_cores(pool)
        steps = [c5_khat_all_cores(pool) for _ in range(args.steps)]
    finally:
        pool.close()
        pool.join()
    t_step = float(np.mean(steps))
    value = 1.0 / (t_step * N_MAT_PER_TRAJ)
    sample = (f"one K_hat of {args.workload} per step (16 slabs of 32x32x32x4 over {min(n, N_SLABS)} "
              f"processes); value scaled by N_mat = {N_MAT_PER_TRAJ} K_hat per trajectory")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "trajectories/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "dims": list(w["dims"])},
            "cpu_baseline": {"value": value, "unit": "trajectories/s", "cores": min(n, N_SLABS), "kind": "oracle",
                             "sample": sample, "host": host},
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
    each, mixed-precision CG of all 96 systems to 1e-10 (CUDA-graph chunks,
    reliable updates with K_hat x in double-float as in the trajectory)."""
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
        lat.wd_set_residual(RESIDUAL_MODE)
        b = torch.empty(w["nrhs"] * 24 * lat.Vh, dtype=torch.float64, device="cuda")
        for r in range(w["nrhs"]):
            lat.gaussian_draw(0, 0, w["seed"], 10 + r, b[r * 24 * lat.Vh:(r + 1) * 24 * lat.Vh])
        lats.append(lat)
        bs.append(b)
        xs.append(torch.zeros_like(b))
    batch = wd.Batch(lats, [w["kappa"] for w in work], [w["nrhs"] for w in work])
    p = wd.cg_params(tol=1e-10, prec=wd.F32)
    out = {}
    # 1: each chunk of 16 iterations as a captured graph of 8 launches per
    # iteration; 2: one persistent cooperative launch per chunk
    for mode, name in ((1, "graph"), (2, "persistent")):
        batch.wd_batch_cg(bs, xs, p, mode)          # tunes (first call), captures the graph
        torch.cuda.synchronize()
        t = time.perf_counter()
        infos = batch.wd_batch_cg(bs, xs, p, mode)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        out[name] = {"s": dt, "systems_per_s": len(infos) / dt,
                     "max_true_rel_resid": max(i["true_rel_resid"] for i in infos),
                     "max_iters": max(i["iters"] for i in infos)}
    info = batch.wd_batch_info()
    best = min(out, key=lambda k: out[k]["s"])
    out.update({"s": out[best]["s"], "systems": info["systems"], "systems_per_s": out[best]["systems_per_s"],
                "mode": best, "tuned_tile_shape": batch.wd_batch_shape()})
    batch.close()
    for lat in lats:
        lat.close()
    return out


def kernel_case(args):
    """K_hat alone on the workload's lattice: the launch sequence ncu captures."""
    import torch
    from paper_1702_00124_gb300 import synthetic, wdhmc as wd
    if args.kernel_case == "batched":
        for k in range(args.reps):
            r = batched_workload_run(wd)
            print(f"kernel case batched (24 lattices x 4 rhs, call {k}): " + json.dumps(r))
        return
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
    lat.wd_set_stencil(STENCILS[args.stencil])
    if args.profile:
        lat.wd_profile_enable(1)   # every hop launch bracketed by CUDA events (not under ncu)
    x, y = lat.half_spinor(), lat.half_spinor()
    lat.gaussian_draw(0, 0, 1, 1, x)
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(args.reps):
        # K_hat chain: each application reads what the previous one wrote, as in CG
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if args.kernel_case.startswith("poly"):
            lat.poly_filter_apply(w["kappa_h"], (4, w["poly"][1], w["poly"][2]), prec, x, y)
        else:
            lat.mdagm_apply(w["kappa"], prec, 1, x, y)
        e1.record(stream)
        x, y = y, x
        ms.append((e0, e1))
    torch.cuda.synchronize()
    t = sorted(a.elapsed_time(b) for a, b in ms[min(3, len(ms) - 1):])
    status = lat.wd_kernel_status()
    hops = lat.wd_profile_read(prec if prec != wd.DF else 4)
    lat.close()
    n_khat = 4 if args.kernel_case.startswith("poly") else 1
    hop = (f"; sampled hops (plain, xpay, dagger): {hops['launches']} launches, "
           f"{hops['ms'] / max(hops['launches'], 1):.4f} ms each, "
           f"{hops['bytes'] / max(hops['ms'], 1e-9) / 1e6:.0f} GB/s algorithmic") if args.profile else ""
    print(f"kernel case {args.kernel_case} on {args.workload} ({args.stencil} stencil): {args.reps} calls of "
          f"{n_khat} K_hat; median {t[len(t) // 2]:.4f} ms per call{hop}; kernel status {status}")


def e2e_run(lat, w, terms, groups, ops, cg_md, cg_acc, force_prec, seed, traj, n=2):
    """The same trajectories end to end through the C ABI's host-buffer call
    (hmc_trajectory_host): every trajectory copies the links in from pinned host
    memory and back out, continuing the chain of the timed region."""
    import torch
    from paper_1702_00124_gb300 import synthetic
    V = int(np.prod(w["dims"]))
    U_dev = torch.empty(V * 72, dtype=torch.float64, device="cuda")
    lat.wd_gauge_store(U_dev)
    U_host = U_dev.cpu().pin_memory()
    del U_dev
    dH = []
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(n):
        u = synthetic.uniform(seed + traj[0])
        r = lat.hmc_trajectory_host(terms, groups, w["beta"], ops, cg_md, cg_acc, force_prec, seed, traj[0], u,
                                    U_host, U_host)
        traj[0] += 1
        dH.append(float(r["dH"]))
    dt = time.perf_counter() - t
    nbytes = V * 72 * 8
    return {"value": n / dt, "unit": "trajectories/s", "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "trajectories": n, "dH": dH,
            "call": "hmc_trajectory_host (links in and out through pinned host memory, one cudaMemcpyAsync each way)"}


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    t = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t, out


def breakdown_c5(lat, w, terms):
    """At 32^3 x 64: one CG solve and one force of the Hasenbusch term in FP64, mixed
    FP32 (FP64 and double-float residuals) and mixed BF16 to 1e-10; one filtered solve;
    stand-alone K_hat bandwidth per precision."""
    from paper_1702_00124_gb300 import wdhmc as wd
    extras = {}
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
        dt, info = _timed(lambda: lat.cg_solve(w["kappa"], b, x, wd.cg_params(tol=1e-10, prec=prec, maxiter=20000)))
        extras[f"cg_{name}"] = {"s": dt, "iters": info["iters"], "reliable_updates": info["reliable_updates"],
                                "true_rel_resid": info["true_rel_resid"]}
        if name in ("fp64", "mixed_fp32"):
            dt, _ = _timed(lambda: lat.fermion_force(terms[2], chi, wd.cg_params(tol=1e-10, prec=prec), 1.0, F))
            extras[f"force_hasenbusch_{name}"] = {"s": dt}
        if name in ("mixed_fp32_fp64resid", "mixed_fp32"):
            x = lat.half_spinor()
            dt, info = _timed(lambda: lat.cg_solve(w["kappa_h"], b, x, wd.cg_params(tol=1e-10, prec=prec),
                                                   filt=w["poly"]))
            extras[f"filtered_cg_{name}"] = {"s": dt, "iters": info["iters"],
                                             "reliable_updates": info["reliable_updates"],
                                             "true_rel_resid": info["true_rel_resid"]}
    lat.wd_set_residual(RESIDUAL_MODE)
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
    return extras


def c3_legs(wd):
    """The paper's volume, 16^3 x 32, with the bench's PF-MP action: one trajectory,
    one CG solve and one force in plain FP64 and in the mixed-precision form (FP32 bulk,
    12-real links, double-float residuals, FP32 forces; the autograd adjoint for the
    force), all to a 1e-10 true residual."""
    import torch
    from paper_1702_00124_gb300 import synthetic
    from paper_1702_00124_gb300.autograd import pf_action
    w = WORKLOADS["c3_16x16x16x32"]
    seed = synthetic.SEED_BASE + 2
    U = synthetic.gauge_field(w["dims"], w["a"], seed)
    U_dev = torch.from_numpy(U.view(np.float64).reshape(-1)).cuda()
    lat = wd.Lattice(w["dims"])
    terms = [wd.term(wd.POLY, w["kappa_h"], poly=w["poly"]), wd.term(wd.FILTERED, w["kappa_h"], poly=w["poly"]),
             wd.term(wd.HASENBUSCH, w["kappa"], w["kappa_h"])]
    groups = [1, 0, 0]
    ops = wd.wd_schedule_nested(1, w["tau"], [g for g, _ in LEVELS], [n for _, n in LEVELS])
    out = {}
    modes = {"mixed": dict(recon=wd.RECON_12, resid=RESIDUAL_MODE, prec=wd.F32, fprec=wd.F32),
             "fp64": dict(recon=wd.RECON_18, resid=0, prec=wd.F64, fprec=wd.F64)}
    for name, m in modes.items():
        lat.wd_set_recon(m["recon"])
        lat.wd_set_residual(m["resid"])
        p = wd.cg_params(tol=1e-10, prec=m["prec"], maxiter=20000)
        recs = []
        for i in range(2 if name == "mixed" else 1):      # mixed: the first one warms up
            lat.wd_gauge_load(U_dev)
            dt, r = _timed(lambda: lat.hmc_trajectory(terms, groups, w["beta"], ops, p, p, m["fprec"], seed, 0, 0.5))
            recs.append((dt, r))
        dt, r = recs[-1]
        out[f"trajectory_{name}"] = {"s": dt, "dH": r["dH"], "n_mat": r["n_mat"], "force_evals": r["n_force_evals"]}
        lat.wd_gauge_load(U_dev)
        chi = lat.half_spinor()
        lat.gaussian_draw(0, 0, seed, 100, chi)
        b = lat.half_spinor()
        lat.wd_apply(w["kappa"], True, wd.F64, chi, b)
        x = lat.half_spinor()
        # every leg is timed on its second call: the first one loads its kernels
        # (lazy module loading) and settles the launch-shape tuner
        lat.cg_solve(w["kappa"], b, x, p)
        x.zero_()                                          # x is the initial guess
        dt, info = _timed(lambda: lat.cg_solve(w["kappa"], b, x, p))
        out[f"cg_hasenbusch_{name}"] = {"s": dt, "iters": info["iters"], "true_rel_resid": info["true_rel_resid"]}
        F = lat.algebra_field()
        lat.fermion_force(terms[2], chi, p, 1.0, F)
        dt, _ = _timed(lambda: lat.fermion_force(terms[2], chi, p, 1.0, F))
        out[f"force_hasenbusch_{name}"] = {"s": dt}
        wv = torch.zeros(64 * lat.Vh, dtype=torch.float64, device="cuda", requires_grad=True)
        for _ in range(2):      # torch's autograd engine starts up over the first two backward calls
            pf_action(wv, lat, terms[2], chi, p, m["fprec"]).backward()
        dt, _ = _timed(lambda: pf_action(wv, lat, terms[2], chi, p, m["fprec"]).backward())
        out[f"autograd_force_hasenbusch_{name}"] = {"s": dt}
    out["trajectory_dH_mixed_minus_fp64"] = out["trajectory_mixed"]["dH"] - out["trajectory_fp64"]["dH"]
    lat.close()
    return out


def cpu_baseline(nmat):
    """The oracle timed on the host cores (single-thread per kernel in one spawned
    process, then one c5 K_hat's work over every core); value = trajectories/s of the
    oracle at the all-core K_hat rate and this run's N_mat."""
    host = host_info()
    pool = spawn_pool(1)
    try:
        single, refs = pool.apply(_single_thread_suite)
    finally:
        pool.close()
        pool.join()
    n = min(host["nproc"] or 1, N_SLABS)
    pool = spawn_pool(n)
    try:
        c5_khat_all_cores(pool)                        # warm
        t_all = c5_khat_all_cores(pool, reps=2)
    finally:
        pool.close()
        pool.join()
    value = 1.0 / (t_all * nmat)
    cpu = {"value": value, "unit": "trajectories/s", "cores": n, "kind": "oracle",
           "sample": f"one K_hat of the 32^3 x 64 workload (16 slabs of 32x32x32x4 over {n} processes, "
                     f"{t_all:.2f} s), scaled by this run's N_mat = {nmat:.0f} K_hat per trajectory",
           "host": host, "c5_khat_all_cores_s": t_all,
           "c5_khat_single_thread_s": single["khat_c5_slab_s"] * N_SLABS,
           "per_kernel_single_thread_s": single}
    return cpu, refs


def error_legs(wd, refs, dH_ref):
    """Error against the FP64 oracle, outside the timed region: the c2 CG solution
    (FP64, mixed FP32, mixed BF16 at 1e-10), the c1 plain-term force (FP64, FP32) and
    the dH of one c1 PF-MP trajectory (FP64, and the bench's mixed configuration)."""
    import torch
    from paper_1702_00124_gb300 import synthetic

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).reshape(-1).copy()).cuda()

    def even_half(lat, lex):            # the library ignores the odd sites of lex
        eo = lat.half_spinor()
        lat.wd_spinor_pack(0, dev(lex), eo)
        return eo

    def rel(a, b):
        return float(np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(b.reshape(-1)))

    out = {}
    w = synthetic.WORKLOADS["c2_8x8x8x16"]
    dims, k = w["dims"], w["kappa"]
    lat = wd.Lattice(dims)
    lat.wd_gauge_load(dev(synthetic.gauge_field(dims, w["a"], w["seed"])))
    lat.wd_set_residual(RESIDUAL_MODE)
    b = lat.half_spinor()
    lat.wd_apply(k, True, wd.F64, even_half(lat, synthetic.spinor_field(dims, w["seed"] + 100)), b)
    X_ref = refs["X_c2_8x8x8x16"]
    for name, prec in (("fp64", wd.F64), ("mixed_fp32", wd.F32), ("mixed_bf16", wd.BF16)):
        x = lat.half_spinor()
        info = lat.cg_solve(k, b, x, wd.cg_params(tol=1e-10, prec=prec, maxiter=20000))
        lex = torch.zeros(X_ref.size * 2, dtype=torch.float64, device="cuda")
        lat.wd_spinor_unpack(0, x, lex)
        got = lex.cpu().numpy().view(np.complex128).reshape(X_ref.shape)
        out[f"c2_cg_solution_{name}"] = {"rel_err": rel(got, X_ref), "iters": info["iters"],
                                         "true_rel_resid": info["true_rel_resid"]}
    lat.close()
    w = synthetic.WORKLOADS["c1_4x4x4x4"]
    dims, k = w["dims"], w["kappa"]
    lat = wd.Lattice(dims)
    lat.wd_gauge_load(dev(synthetic.gauge_field(dims, w["a"], w["seed"])))
    phi = lat.half_spinor()
    lat.wd_apply(k, True, wd.F64, even_half(lat, synthetic.spinor_field(dims, w["seed"] + 100)), phi)
    F_ref = refs["F_c1"]
    for name, prec in (("fp64", wd.F64), ("mixed_fp32", wd.F32)):
        F = lat.algebra_field()
        lat.fermion_force(wd.term(wd.PLAIN, k), phi, wd.cg_params(tol=1e-10, prec=prec), 1.0, F)
        lex = torch.zeros(F_ref.size, dtype=torch.float64, device="cuda")
        lat.wd_algebra_unpack(F, lex)
        out[f"c1_force_{name}"] = {"rel_err": rel(lex.cpu().numpy().reshape(F_ref.shape), F_ref)}
    lat.close()
    c = DH_LEG
    U0 = synthetic.gauge_field(c["dims"], c["a"], c["seed"])
    terms = [wd.term(wd.POLY, c["kappa_h"], poly=c["poly"]), wd.term(wd.FILTERED, c["kappa_h"], poly=c["poly"]),
             wd.term(wd.HASENBUSCH, c["kappa"], c["kappa_h"])]
    ops = wd.wd_schedule_nested(1, c["tau"], [g for g, _ in c["levels"]], [n for _, n in c["levels"]])
    for name, prec, fprec, recon, resid in (("fp64", wd.F64, wd.F64, 0, 0), ("mixed", wd.F32, wd.F32, 1, 1)):
        lat = wd.Lattice(c["dims"])
        lat.wd_gauge_load(dev(U0))
        lat.wd_set_recon(recon)
        lat.wd_set_residual(resid)
        p = wd.cg_params(tol=1e-12 if prec == wd.F64 else 1e-10, prec=prec, maxiter=20000)
        r = lat.hmc_trajectory(terms, c["groups"], c["beta"], ops, p, p, fprec, c["draw_seed"], c["traj"], 0.0)
        out[f"c1_trajectory_dH_{name}"] = {"dH": r["dH"], "dH_oracle": dH_ref, "abs_err": abs(r["dH"] - dH_ref)}
        lat.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-extras", action="store_true", help="skip the mixed-vs-FP64 and e2e measurements")
    ap.add_argument("--kernel-case", choices=["khat_f32_recon12", "khat_bf16_recon12", "khat_f64", "khat_df",
                                              "poly_f32_recon12", "batched"],
                    help="only apply K_hat --reps times on the workload (for ncu captures); prints no JSON")
    ap.add_argument("--reps", type=int, default=4)
    ap.add_argument("--profile", action="store_true", help="kernel case: time every hop with CUDA events")
    ap.add_argument("--stencil", default="thread", choices=sorted(STENCILS),
                    help="kernel case: 12-real-link stencil kernel (thread: per-thread staging, the default; "
                         "tile: tile-staged bulk copies)")
    ap.add_argument("--n-outer", type=int, default=None,
                    help="outer integrator steps (default: the workload's; fewer only for short ncu launch lists)")
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
    del U_dev
    terms = [wd.term(wd.POLY, w["kappa_h"], poly=w["poly"]), wd.term(wd.FILTERED, w["kappa_h"], poly=w["poly"]),
             wd.term(wd.HASENBUSCH, w["kappa"], w["kappa_h"])]
    groups = [1, 0, 0]
    levels = [(g, (args.n_outer or w["n_outer"]) if g == 0 else n) for g, n in LEVELS]
    ops = wd.wd_schedule_nested(1, w["tau"], [g for g, _ in levels], [n for _, n in levels])
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
    profdd = lat.wd_profile_read(wd.DF)
    counts = lat.wd_hop_counts()
    lat.wd_profile_enable(0)
    # share of the timed region spent in each hop family: all launches of the
    # family x its average sampled duration
    shares = {}
    for name, pr, n in (("k_hop_fp32", prof, counts[wd.F32]), ("k_hop_fp64", prof64, counts[wd.F64]),
                        ("k_hop_dd", profdd, counts[wd.DF])):
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
        e2e = e2e_run(lat, w, terms, groups, ops, cg_md, cg_acc, wd.F32, seed, traj)
        pool = spawn_pool(1)
        refs_job = pool.apply_async(_oracle_dH_c1)
        extras.update(breakdown_c5(lat, w, terms))
        extras["c3_16x16x16x32"] = c3_legs(wd)
        extras["batched_24_lattices_x4_rhs"] = batched_workload_run(wd)
        dH_ref = refs_job.get()
        pool.close()
        pool.join()
        cpu, refs = cpu_baseline(nmat)
        extras["error_vs_fp64_oracle"] = error_legs(wd, refs, dH_ref)

    if rank == 0:
        acc = [int(r["accepted"]) for r in timed]
        line = {"metric": METRIC, "value": value, "unit": "trajectories/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": args.workload, "dims": list(dims), "kappa": w["kappa"],
                           "kappa_h": w["kappa_h"], "poly": list(w["poly"]), "beta": w["beta"],
                           "integrator": "nested Omelyan 2MN", "levels": levels, "tau": w["tau"],
                           "action": "PF-MP + Wilson gauge",
                           "precision": "FP32 bulk (12-real links); reliable updates with b, x, r, dots in FP64 and "
                                        + ("A x in double-float (2xFP32, ~48 bits)" if RESIDUAL_MODE else "A x in FP64")
                                        + "; links, momenta, H in FP64",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "l2": "inputs larger than L2: working set (1.2 GB FP64 links + FP32 copies) far above the 129 MB L2"},
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
