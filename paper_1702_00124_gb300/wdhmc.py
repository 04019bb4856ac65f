"""Thin Python binding of libwdhmc (include/wdhmc.h).

Argument marshalling only: every function forwards torch tensors' device
pointers to the C entry point of the same name and raises on a non-zero
status.  All computation happens in the CUDA library; there is no fallback:
importing this module without the built library raises.
"""
import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libwdhmc.so")

if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libwdhmc.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
lib = C.CDLL(_LIB_PATH)

F64, F32, F16, BF16, DF = 0, 1, 2, 3, 4   # DF: double-float (operator calls only)
RECON_18, RECON_12 = 0, 1
STENCIL_THREAD, STENCIL_TILE = 0, 1
PLAIN, HASENBUSCH, POLY, FILTERED, RATIO = 0, 1, 2, 3, 4
ERRORS = {1: "WD_ERR_ARG", 2: "WD_ERR_CUDA", 3: "WD_ERR_NOCONV", 4: "WD_ERR_NAN", 5: "WD_ERR_STATE",
          6: "WD_ERR_TIMEOUT"}


class WdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class wd_poly(C.Structure):
    _fields_ = [("n", C.c_int), ("eps", C.c_double), ("lam", C.c_double)]


class wd_term(C.Structure):
    _fields_ = [("kind", C.c_int), ("kappa", C.c_double), ("kappa_h", C.c_double), ("poly", wd_poly),
                ("poly_lo", wd_poly)]


class wd_cg_params(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxiter", C.c_int), ("prec", C.c_int), ("delta", C.c_double),
                ("check_every", C.c_int)]


class wd_cg_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("reliable_updates", C.c_int), ("n_mat", C.c_longlong),
                ("true_rel_resid", C.c_double)]


class wd_op(C.Structure):
    _fields_ = [("kind", C.c_int), ("group", C.c_int), ("eps", C.c_double)]


class wd_hmc_params(C.Structure):
    _fields_ = [("nterms", C.c_int), ("terms", C.POINTER(wd_term)), ("term_group", C.POINTER(C.c_int)),
                ("beta", C.c_double), ("nops", C.c_int), ("ops", C.POINTER(wd_op)),
                ("cg_md", wd_cg_params), ("cg_acc", wd_cg_params), ("force_prec", C.c_int),
                ("seed", C.c_uint64), ("traj_index", C.c_uint64), ("h0_solve", C.c_int)]


class wd_integrate_params(C.Structure):
    _fields_ = [("nterms", C.c_int), ("terms", C.POINTER(wd_term)), ("term_group", C.POINTER(C.c_int)),
                ("phi", C.POINTER(C.c_void_p)), ("beta", C.c_double), ("nops", C.c_int),
                ("ops", C.POINTER(wd_op)), ("cg_md", wd_cg_params), ("force_prec", C.c_int)]


class wd_cost_result(C.Structure):
    _fields_ = [("C", C.c_double), ("p_acc", C.c_double), ("p_acc_est", C.c_double), ("mean_nmat", C.c_double),
                ("exp_mdH", C.c_double), ("exp_mdH_err", C.c_double), ("C_est", C.c_double)]


class wd_hmc_result(C.Structure):
    _fields_ = [("H0", C.c_double), ("H1", C.c_double), ("dH", C.c_double), ("S_gauge0", C.c_double),
                ("S_gauge1", C.c_double), ("accepted", C.c_int), ("n_mat", C.c_longlong),
                ("n_force_evals", C.c_int), ("t_heatbath_ms", C.c_double), ("t_hamiltonian_ms", C.c_double),
                ("t_T_ms", C.c_double), ("t_gauge_force_ms", C.c_double),
                ("t_force_group_ms", C.c_double * 4)]


_P = C.c_void_p
_D = C.c_double
_I = C.c_int
_SIG = {
    "wd_last_error": ([], C.c_char_p),
    "wd_context_create": ([C.POINTER(C.c_int), _P, C.POINTER(_P)], _I),
    "wd_context_destroy": ([_P], _I),
    "wd_set_recon": ([_P, _I], _I),
    "wd_volume": ([_P, C.POINTER(C.c_longlong)], _I),
    "wd_gauge_load": ([_P, _P], _I),
    "wd_gauge_store": ([_P, _P], _I),
    "wd_spinor_pack": ([_P, _I, _P, _P], _I),
    "wd_spinor_unpack": ([_P, _I, _P, _P], _I),
    "wd_algebra_pack": ([_P, _P, _P], _I),
    "wd_algebra_unpack": ([_P, _P, _P], _I),
    "wd_hop": ([_P, _I, _I, _I, _P, _P], _I),
    "wd_apply": ([_P, _D, _I, _I, _P, _P], _I),
    "mdagm_apply": ([_P, _D, _I, _I, _P, _P], _I),
    "cg_solve": ([_P, _D, C.POINTER(wd_poly), _P, _P, C.POINTER(wd_cg_params), C.POINTER(wd_cg_info)], _I),
    "poly_filter_apply": ([_P, _D, C.POINTER(wd_poly), _I, _P, _P], _I),
    "pf_action": ([_P, C.POINTER(wd_term), _P, C.POINTER(wd_cg_params), C.POINTER(_D)], _I),
    "pf_heatbath": ([_P, C.POINTER(wd_term), _P, C.POINTER(wd_cg_params), _P], _I),
    "fermion_force": ([_P, C.POINTER(wd_term), _P, C.POINTER(wd_cg_params), _D, _P], _I),
    "gauge_action": ([_P, _D, C.POINTER(_D)], _I),
    "gauge_force": ([_P, _D, _I, _D, _P], _I),
    "step_T": ([_P, _P, _D], _I),
    "step_S": ([_P, _P, _P, _D], _I),
    "kinetic_energy": ([_P, _P, C.POINTER(_D)], _I),
    "gaussian_draw": ([_P, _I, _I, C.c_uint64, C.c_uint64, _P], _I),
    "metropolis": ([_D, _D, C.POINTER(_I)], _I),
    "metropolis_philox": ([_D, C.c_uint64, C.c_uint64, C.POINTER(_D), C.POINTER(_I)], _I),
    "wd_cost": ([C.POINTER(C.c_longlong), C.POINTER(_I), C.POINTER(_D), _I, C.POINTER(wd_cost_result)], _I),
    "hmc_trajectory": ([_P, C.POINTER(wd_hmc_params), _D, C.POINTER(wd_hmc_result)], _I),
    "hmc_trajectory_host": ([_P, C.POINTER(wd_hmc_params), _D, _P, _P, C.POINTER(wd_hmc_result)], _I),
    "integrate": ([_P, _P, C.POINTER(wd_integrate_params), C.POINTER(_I)], _I),
    "wd_schedule_nested": ([_I, _D, _I, C.POINTER(_I), C.POINTER(_I), C.POINTER(wd_op), _I, C.POINTER(_I)], _I),
    "wd_schedule_generalised": ([_I, _D, _I, C.POINTER(_I), C.POINTER(_I), C.POINTER(wd_op), _I,
                                 C.POINTER(_I)], _I),
    "wd_nmat": ([_P, C.POINTER(C.c_longlong), _I], _I),
    "wd_profile_enable": ([_P, _I], _I),
    "wd_profile_read": ([_P, _I, C.POINTER(C.c_longlong), C.POINTER(_D), C.POINTER(_D)], _I),
    "wd_launch_count": ([_P, C.POINTER(C.c_longlong)], _I),
    "mdagm_apply_noalloc": ([C.POINTER(C.c_int), _P, _D, _P, _P, _P], _I),
    "pf_action_xy": ([_P, C.POINTER(wd_term), _P, C.POINTER(wd_cg_params), C.POINTER(_D), _P, _P], _I),
    "fermion_force_xy": ([_P, C.POINTER(wd_term), _P, _P, _P, _I, _D, _P], _I),
    "wd_set_residual": ([_P, _I], _I),
    "wd_set_stencil": ([_P, _I], _I),
    "wd_kernel_status": ([_P, C.POINTER(C.c_uint)], _I),
    "wd_selftest_wait_timeout": ([_P, C.c_longlong], _I),
    "wd_set_autotune": ([_P, _I, C.POINTER(_I)], _I),
    "wd_tune_entry": ([_P, _I, C.POINTER(C.c_longlong), C.POINTER(_I), C.POINTER(_I)], _I),
    "wd_hop_counts": ([_P, C.POINTER(C.c_longlong)], _I),
    "wd_batch_create": ([C.POINTER(_P), _I, C.POINTER(_D), C.POINTER(_I), C.POINTER(_P)], _I),
    "wd_batch_destroy": ([_P], _I),
    "wd_batch_mdagm": ([_P, C.POINTER(_P), C.POINTER(_P)], _I),
    "wd_batch_cg": ([_P, C.POINTER(_P), C.POINTER(_P), C.POINTER(wd_cg_params), _I, C.POINTER(wd_cg_info)], _I),
    "wd_batch_info": ([_P, C.POINTER(_I), C.POINTER(_I), C.POINTER(C.c_longlong)], _I),
    "wd_batch_shape": ([_P, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)], _I),
    "wd_batch_set_shape": ([_P, _I, _I, _I], _I),
}
for _name, (_args, _res) in _SIG.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = sorted(_SIG)


def _check(code):
    if code != 0:
        raise WdError(code, lib.wd_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("tensor must live on the GPU")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def _host_ptr(a, n):
    """Address of a HOST float64 buffer of at least n elements (CPU tensor or numpy array)."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous() or a.numel() < n:
            raise ValueError(f"expected a contiguous CPU float64 tensor of >= {n} elements")
        return C.c_void_p(a.data_ptr())
    import numpy as np
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size < n:
        raise ValueError(f"expected a contiguous float64 array of >= {n} elements")
    return C.c_void_p(a.ctypes.data)


def cg_params(tol=1e-10, maxiter=10000, prec=F64, delta=0.0, check_every=0):
    """delta = 0 and check_every = 0 select the library defaults."""
    return wd_cg_params(tol, maxiter, prec, delta, check_every)


def term(kind, kappa, kappa_h=0.0, poly=None, poly_lo=None):
    def mk(q):
        return wd_poly(0, 0.0, 0.0) if q is None else wd_poly(int(q[0]), float(q[1]), float(q[2]))
    return wd_term(kind, kappa, kappa_h, mk(poly), mk(poly_lo))


def _ops_array(ops):
    arr = (wd_op * len(ops))()
    for i, o in enumerate(ops):
        arr[i] = wd_op(*o) if not isinstance(o, wd_op) else o
    return arr


def wd_schedule_nested(kind, tau, groups, steps):
    g = (C.c_int * len(groups))(*groups)
    s = (C.c_int * len(steps))(*steps)
    n = C.c_int(0)
    _check(lib.wd_schedule_nested(kind, tau, len(groups), g, s, None, 0, C.byref(n)))
    ops = (wd_op * n.value)()
    _check(lib.wd_schedule_nested(kind, tau, len(groups), g, s, ops, n.value, C.byref(n)))
    return [(o.kind, o.group, o.eps) for o in ops]


def wd_schedule_generalised(kind, tau, groups, nsteps):
    g = (C.c_int * len(groups))(*groups)
    s = (C.c_int * len(nsteps))(*nsteps)
    n = C.c_int(0)
    _check(lib.wd_schedule_generalised(kind, tau, len(groups), g, s, None, 0, C.byref(n)))
    ops = (wd_op * n.value)()
    _check(lib.wd_schedule_generalised(kind, tau, len(groups), g, s, ops, n.value, C.byref(n)))
    return [(o.kind, o.group, o.eps) for o in ops]


def metropolis(dH, u):
    a = C.c_int(0)
    _check(lib.metropolis(dH, u, C.byref(a)))
    return bool(a.value)


def metropolis_philox(dH, seed, counter):
    """(accepted, u) with u drawn from (seed, counter) by Philox4x64-10."""
    a, u = C.c_int(0), C.c_double(0)
    _check(lib.metropolis_philox(dH, seed, counter, C.byref(u), C.byref(a)))
    return bool(a.value), u.value


def wd_cost(n_mat, accepted, dH):
    """C = <N_mat> / P_acc over trajectories (host arrays; see the C header)."""
    n = len(n_mat)
    if len(accepted) != n or len(dH) != n:
        raise ValueError("n_mat, accepted and dH must have one entry per trajectory")
    r = wd_cost_result()
    _check(lib.wd_cost((C.c_longlong * max(n, 1))(*[int(v) for v in n_mat]),
                       (C.c_int * max(n, 1))(*[int(v) for v in accepted]),
                       (C.c_double * max(n, 1))(*[float(v) for v in dH]), n, C.byref(r)))
    return {k: getattr(r, k) for k, _ in wd_cost_result._fields_}


class Batch:
    """wd_batch: independent lattices (Lattice objects sharing a stream), each
    with a hopping parameter and 1..8 right-hand sides."""

    def __init__(self, lattices, kappas, nrhs):
        n = len(lattices)
        self.lattices, self.nrhs = list(lattices), list(nrhs)
        hs = (_P * n)(*[lat.h.value for lat in lattices])
        h = C.c_void_p()
        _check(lib.wd_batch_create(hs, n, (_D * n)(*kappas), (_I * n)(*nrhs), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib.wd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _ptrs(ts):
        return (_P * len(ts))(*[_ptr(t).value for t in ts])

    def wd_batch_mdagm(self, ins, outs):
        _check(lib.wd_batch_mdagm(self.h, self._ptrs(ins), self._ptrs(outs)))

    def wd_batch_cg(self, bs, xs, params, use_graph=True):
        S = sum(self.nrhs)
        infos = (wd_cg_info * S)()
        _check(lib.wd_batch_cg(self.h, self._ptrs(bs), self._ptrs(xs), C.byref(params), int(use_graph), infos))
        return [dict(iters=i.iters, reliable_updates=i.reliable_updates, n_mat=i.n_mat,
                     true_rel_resid=i.true_rel_resid) for i in infos]

    def wd_batch_info(self):
        s, t, n = C.c_int(0), C.c_int(0), C.c_longlong(0)
        _check(lib.wd_batch_info(self.h, C.byref(s), C.byref(t), C.byref(n)))
        return dict(systems=s.value, threads=t.value, launches=n.value)

    def wd_batch_set_shape(self, items_per_block, rhs_per_thread, link_staging=0):
        _check(lib.wd_batch_set_shape(self.h, items_per_block, rhs_per_thread, int(link_staging)))

    def wd_batch_shape(self):
        t, r, st = C.c_int(0), C.c_int(0), C.c_int(0)
        _check(lib.wd_batch_shape(self.h, C.byref(t), C.byref(r), C.byref(st)))
        return dict(items_per_block=t.value, rhs_per_thread=r.value, link_staging=st.value)


class Lattice:
    """One wd_ctx: a lattice, its gauge field copies and workspaces, on the
    current CUDA device and torch's current stream (or the given one)."""

    def __init__(self, dims, stream=None):
        self.dims = tuple(int(d) for d in dims)
        d = (C.c_int * 4)(*self.dims)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        h = C.c_void_p()
        _check(lib.wd_context_create(d, C.c_void_p(s.cuda_stream), C.byref(h)))
        self.h = h
        vol = (C.c_longlong * 2)()
        _check(lib.wd_volume(self.h, vol))
        self.V, self.Vh = int(vol[0]), int(vol[1])
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "h", None):
            lib.wd_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # allocation helpers (torch owns the memory)
    def half_spinor(self, zero=True):
        f = torch.zeros if zero else torch.empty
        return f(24 * self.Vh, dtype=torch.float64, device=self.device)

    def algebra_field(self, zero=True):
        f = torch.zeros if zero else torch.empty
        return f(64 * self.Vh, dtype=torch.float64, device=self.device)

    # ---- entry points ----------------------------------------------------
    def wd_set_recon(self, recon):
        _check(lib.wd_set_recon(self.h, recon))

    def wd_set_residual(self, mode):
        _check(lib.wd_set_residual(self.h, mode))

    def wd_set_stencil(self, stencil):
        _check(lib.wd_set_stencil(self.h, stencil))

    def wd_selftest_wait_timeout(self, timeout_ns):
        _check(lib.wd_selftest_wait_timeout(self.h, int(timeout_ns)))

    def wd_kernel_status(self):
        w = C.c_uint(0)
        _check(lib.wd_kernel_status(self.h, C.byref(w)))
        return w.value

    def wd_set_autotune(self, enable=-1):
        n = C.c_int(0)
        _check(lib.wd_set_autotune(self.h, enable, C.byref(n)))
        return n.value

    def tuned(self):
        """{key: (threads, minb)} chosen by the launch-shape autotuner."""
        out = {}
        for i in range(self.wd_set_autotune(-1)):
            k, t, m = C.c_longlong(0), C.c_int(0), C.c_int(0)
            _check(lib.wd_tune_entry(self.h, i, C.byref(k), C.byref(t), C.byref(m)))
            out[k.value] = (t.value, m.value)
        return out

    def wd_gauge_load(self, U_lex):
        _check(lib.wd_gauge_load(self.h, _ptr(U_lex)))

    def wd_gauge_store(self, U_lex):
        _check(lib.wd_gauge_store(self.h, _ptr(U_lex)))

    def wd_spinor_pack(self, parity, lex, eo):
        _check(lib.wd_spinor_pack(self.h, parity, _ptr(lex), _ptr(eo)))

    def wd_spinor_unpack(self, parity, eo, lex):
        _check(lib.wd_spinor_unpack(self.h, parity, _ptr(eo), _ptr(lex)))

    def wd_algebra_pack(self, lex, eo):
        _check(lib.wd_algebra_pack(self.h, _ptr(lex), _ptr(eo)))

    def wd_algebra_unpack(self, eo, lex):
        _check(lib.wd_algebra_unpack(self.h, _ptr(eo), _ptr(lex)))

    def wd_hop(self, out_parity, dagger, prec, x, out):
        _check(lib.wd_hop(self.h, out_parity, int(dagger), prec, _ptr(x), _ptr(out)))

    def wd_apply(self, kappa, dagger, prec, x, out):
        _check(lib.wd_apply(self.h, kappa, int(dagger), prec, _ptr(x), _ptr(out)))

    def mdagm_apply(self, kappa, prec, nrhs, x, out):
        _check(lib.mdagm_apply(self.h, kappa, prec, nrhs, _ptr(x), _ptr(out)))

    def cg_solve(self, kappa, b, x, params, filt=None):
        info = wd_cg_info()
        fp = C.byref(wd_poly(*filt)) if filt is not None else None
        _check(lib.cg_solve(self.h, kappa, fp, _ptr(b), _ptr(x), C.byref(params), C.byref(info)))
        return dict(iters=info.iters, reliable_updates=info.reliable_updates, n_mat=info.n_mat,
                    true_rel_resid=info.true_rel_resid)

    def poly_filter_apply(self, kappa, poly, prec, x, out):
        _check(lib.poly_filter_apply(self.h, kappa, C.byref(wd_poly(*poly)), prec, _ptr(x), _ptr(out)))

    def pf_action(self, t, phi, params):
        S = C.c_double(0)
        _check(lib.pf_action(self.h, C.byref(t), _ptr(phi), C.byref(params), C.byref(S)))
        return S.value

    def pf_action_xy(self, t, phi, params, X=None, Y=None):
        S = C.c_double(0)
        _check(lib.pf_action_xy(self.h, C.byref(t), _ptr(phi), C.byref(params), C.byref(S), _ptr(X), _ptr(Y)))
        return S.value

    def fermion_force_xy(self, t, phi, X, Y, prec, coef, F):
        _check(lib.fermion_force_xy(self.h, C.byref(t), _ptr(phi), _ptr(X), _ptr(Y), prec, coef, _ptr(F)))

    def pf_heatbath(self, t, chi, params, phi):
        _check(lib.pf_heatbath(self.h, C.byref(t), _ptr(chi), C.byref(params), _ptr(phi)))

    def fermion_force(self, t, phi, params, coef, F):
        _check(lib.fermion_force(self.h, C.byref(t), _ptr(phi), C.byref(params), coef, _ptr(F)))

    def gauge_action(self, beta):
        S = C.c_double(0)
        _check(lib.gauge_action(self.h, beta, C.byref(S)))
        return S.value

    def gauge_force(self, beta, prec, coef, F):
        _check(lib.gauge_force(self.h, beta, prec, coef, _ptr(F)))

    def step_T(self, P, eps):
        _check(lib.step_T(self.h, _ptr(P), eps))

    def step_S(self, P, F, eps):
        _check(lib.step_S(self.h, _ptr(P), _ptr(F), eps))

    def kinetic_energy(self, P):
        K = C.c_double(0)
        _check(lib.kinetic_energy(self.h, _ptr(P), C.byref(K)))
        return K.value

    def gaussian_draw(self, what, parity, seed, stream, out):
        _check(lib.gaussian_draw(self.h, what, parity, seed, stream, _ptr(out)))

    def hmc_trajectory(self, terms, groups, beta, ops, cg_md, cg_acc, force_prec, seed, traj_index, u, h0_solve=0):
        tarr = (wd_term * max(len(terms), 1))(*terms)
        garr = (C.c_int * max(len(groups), 1))(*groups)
        oarr = _ops_array(ops)
        p = wd_hmc_params(len(terms), tarr, garr, beta, len(ops), oarr, cg_md, cg_acc, force_prec, seed,
                          traj_index, h0_solve)
        r = wd_hmc_result()
        _check(lib.hmc_trajectory(self.h, C.byref(p), u, C.byref(r)))
        return self._result(r)

    @staticmethod
    def _result(r):
        out = {k: getattr(r, k) for k, _ in wd_hmc_result._fields_}
        out["t_force_group_ms"] = list(r.t_force_group_ms)
        return out

    def hmc_trajectory_host(self, terms, groups, beta, ops, cg_md, cg_acc, force_prec, seed, traj_index, u,
                            U_in, U_out, h0_solve=0):
        """hmc_trajectory with the links in and out through HOST buffers (CPU
        float64 tensors or arrays of V * 72 doubles; pinned memory for DMA)."""
        tarr = (wd_term * max(len(terms), 1))(*terms)
        garr = (C.c_int * max(len(groups), 1))(*groups)
        oarr = _ops_array(ops)
        p = wd_hmc_params(len(terms), tarr, garr, beta, len(ops), oarr, cg_md, cg_acc, force_prec, seed,
                          traj_index, h0_solve)
        r = wd_hmc_result()
        _check(lib.hmc_trajectory_host(self.h, C.byref(p), u, _host_ptr(U_in, self.V * 72),
                                       _host_ptr(U_out, self.V * 72), C.byref(r)))
        return self._result(r)

    def integrate(self, P, terms, groups, phis, beta, ops, cg_md, force_prec):
        """The integrator alone on caller-held momenta P (device algebra field),
        pseudofermions phis (device half spinors) fixed; returns the number of
        force evaluations."""
        tarr = (wd_term * max(len(terms), 1))(*terms)
        garr = (C.c_int * max(len(groups), 1))(*groups)
        parr = (C.c_void_p * max(len(phis), 1))(*[_ptr(f) for f in phis])
        oarr = _ops_array(ops)
        p = wd_integrate_params(len(terms), tarr, garr, parr, beta, len(ops), oarr, cg_md, force_prec)
        nf = C.c_int(0)
        _check(lib.integrate(self.h, _ptr(P), C.byref(p), C.byref(nf)))
        return nf.value

    def wd_nmat(self, reset=False):
        n = C.c_longlong(0)
        _check(lib.wd_nmat(self.h, C.byref(n), int(reset)))
        return n.value

    def wd_profile_enable(self, every_n):
        _check(lib.wd_profile_enable(self.h, every_n))

    def wd_profile_read(self, fmt=-1):
        n, ms, b = C.c_longlong(0), C.c_double(0), C.c_double(0)
        _check(lib.wd_profile_read(self.h, fmt, C.byref(n), C.byref(ms), C.byref(b)))
        return dict(launches=n.value, ms=ms.value, bytes=b.value)

    def wd_hop_counts(self):
        a = (C.c_longlong * 5)()
        _check(lib.wd_hop_counts(self.h, a))
        return list(a)

    def wd_launch_count(self):
        n = C.c_longlong(0)
        _check(lib.wd_launch_count(self.h, C.byref(n)))
        return n.value
