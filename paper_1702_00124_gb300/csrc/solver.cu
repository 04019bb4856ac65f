// Solver layer: the filter polynomial, its application by a three-term
// recurrence, and conjugate gradient with FP64 reliable updates.
//
// Section 2 of the paper: K = M^dag M is inverted by an iterative solver such
// as CG; polynomial filtering uses P(K) ~ K^-1 built from Chebyshev
// polynomials, and the filtered term needs [P(K) K]^-1.  Section 3.1: the
// cost unit is one multiplication by K (N_mat).
//
// Filter (reading of the paper; it prints no construction):
//   x P(x) = 1 - R(x),  R(x) = T_{n+1}(y(x)) / T_{n+1}(y0),
//   y(x) = (mu - x)/nu, y0 = mu/nu, mu = (lam+eps)/2, nu = (lam-eps)/2.
// With t_k = T_k(y0) and s_k = (1 - T_k(y(x))/t_k)/x the Chebyshev recurrence
// T_{k+1} = 2 y T_k - T_{k-1} gives, for the polynomials s_k,
//   s_1 = 1/mu,  s_{k+1} = a_k (1 + mu s_k - x s_k) - b_k s_{k-1},
//   a_k = 2 t_k / (nu t_{k+1}),  b_k = t_{k-1} / t_{k+1},
// and P = s_{n+1}: n multiplications by K.  The factored form
// P(x) = c prod_k (x - z_k), z_k = mu (1 - cos th_k) - i sqrt(eps lam) sin th_k,
// th_k = 2 pi k / (n+1), c = 2^n / (nu^{n+1} t_{n+1}) (even n), serves the
// heat bath and the force.
//
// Mixed-precision CG (reliable updates, Sleijpen & van der Vorst 1996; as used
// for lattice QCD by Clark et al. 2010): the iterated residual, search
// direction and operator run in the sloppy precision; when |r|^2 falls below
// delta^2 times its value at the last update (or below tol^2 |b|^2), the
// solution increment is folded into the FP64 x and r = b - A x is recomputed
// in FP64.  The FP64 mode is the same loop with every field in FP64.
#include <cmath>

#include "dslash_impl.cuh"

namespace wd {

int poly_coef(const wd_poly& P, PolyCoef* out) {
  if (P.n < 0 || P.n % 2 != 0) return fail(WD_ERR_ARG, "filter degree must be even and >= 0");
  if (!(P.eps > 0) || !(P.lam > P.eps)) return fail(WD_ERR_ARG, "filter interval must satisfy 0 < eps < lam");
  PolyCoef& c = *out;
  c.n = P.n;
  c.mu = 0.5 * (P.lam + P.eps);
  c.nu = 0.5 * (P.lam - P.eps);
  const double y0 = c.mu / c.nu;
  const double eta = std::acosh(y0);
  std::vector<double> t(P.n + 2);
  for (int k = 0; k <= P.n + 1; ++k) t[k] = std::cosh(k * eta);
  c.s1 = 1.0 / c.mu;
  c.a.assign(P.n + 1, 0.0);
  c.b.assign(P.n + 1, 0.0);
  for (int k = 1; k <= P.n; ++k) {
    c.a[k] = 2.0 * t[k] / (c.nu * t[k + 1]);
    c.b[k] = t[k - 1] / t[k + 1];
  }
  c.scale = std::ldexp(1.0, P.n) / (std::pow(c.nu, P.n + 1) * t[P.n + 1]);
  c.zr.resize(P.n);
  c.zi.resize(P.n);
  const double sq = std::sqrt(P.eps * P.lam);
  for (int k = 1; k <= P.n; ++k) {
    const double th = 2.0 * M_PI * k / (P.n + 1);
    c.zr[k - 1] = c.mu * (1.0 - std::cos(th));
    c.zi[k - 1] = -sq * std::sin(th);
  }
  return WD_OK;
}

// Q = P_hi / P_lo on one interval (Section 3.3).  With th_k = 2 pi k / (n + 1)
// the roots of P_lo are the roots of P_hi whose index k is a multiple of
// m = (n_hi + 1) / (n_lo + 1); Q keeps the others, in ascending k, and has
// scale c_hi / c_lo.  The kept set is closed under k -> n_hi + 1 - k (the
// conjugate root), so its first half holds one root of every conjugate pair.
int ratio_coef(const wd_poly& hi, const wd_poly& lo, PolyCoef* out) {
  PolyCoef ph, pl;
  WD_TRY(poly_coef(hi, &ph));
  WD_TRY(poly_coef(lo, &pl));
  if (hi.eps != lo.eps || hi.lam != lo.lam) return fail(WD_ERR_ARG, "ratio: both filters need the same [eps, lam]");
  if (lo.n > hi.n || (hi.n + 1) % (lo.n + 1) != 0)
    return fail(WD_ERR_ARG, "ratio: (n_lo + 1) must divide (n + 1)");
  const int m = (hi.n + 1) / (lo.n + 1);
  PolyCoef& c = *out;
  c.n = hi.n - lo.n;
  c.mu = ph.mu;
  c.nu = ph.nu;
  c.scale = ph.scale / pl.scale;
  c.s1 = 0.0;
  c.a.clear();
  c.b.clear();
  c.zr.clear();
  c.zi.clear();
  for (int k = 1; k <= hi.n; ++k) {
    if (k % m == 0) continue;
    c.zr.push_back(ph.zr[k - 1]);
    c.zi.push_back(ph.zi[k - 1]);
  }
  return WD_OK;
}

// out = Q(K) in = prod_pairs f (K^2 - 2 Re z K + |z|^2) in, f = scale^(1/pairs).
// Each factor is one recurrence-shaped update a (v + mu s - K s) - b s' with
// v = s' = x, s = K x: a = -f, mu = 2 Re z, b = -f (1 + |z|^2); in FP32 it is
// fused into the last hop of the second K.
int roots_apply_f(wd_ctx* c, double kappa, const PolyCoef& q, const Field& in, const Field& out) {
  const int f = in.fmt;
  if (f != WD_F64 && f != WD_F32 && f != WD_DD) return fail(WD_ERR_ARG, "ratio: FP64, FP32 or double-float fields");
  const int np = q.n / 2;
  if (np == 0) return axpby(c, q.scale, in, 0.0, in, out);
  const double fs = std::pow(q.scale, 1.0 / np);
  WsGuard w(c);
  Field s, ks, t1, t2;
  WD_TRY(w.get(f, &s));
  WD_TRY(w.get(f, &ks));
  WD_TRY(w.get(f, &t1));
  WD_TRY(w.get(f, &t2));
  WD_TRY(convert(c, in, out));
  for (int k = 0; k < np; ++k) {
    const double zr = q.zr[k], zi = q.zi[k];
    const double ca = -fs, cmu = 2.0 * zr, cb = -fs * (1.0 + zr * zr + zi * zi);
    WD_TRY(apply_khat(c, kappa, out, s, t1, t2, false, false));
    if (f == WD_F32) {
      WD_TRY(khat_poly_step_f32(c, kappa, s, t1, t2, out, out, ca, cmu, cb, out));
    } else {
      WD_TRY(apply_khat(c, kappa, s, ks, t1, t2, false, false));
      WD_TRY(poly_step(c, ca, cmu, cb, out, s, ks, out, out));
    }
  }
  return WD_OK;
}

int khat_any(wd_ctx* c, double kappa, const Field& in, const Field& out) {
  WsGuard w(c);
  Field t1, t2;
  WD_TRY(w.get(in.fmt, &t1));
  WD_TRY(w.get(in.fmt, &t2));
  return apply_khat(c, kappa, in, out, t1, t2, false, false);
}

// out = P(K_hat) in; in and out are FP64 or FP32 fields of one format and
// may not alias.
int poly_apply_f(wd_ctx* c, double kappa, const wd_poly& P, int /*prec*/, const Field& in,
                 const Field& out) {
  PolyCoef pc;
  WD_TRY(poly_coef(P, &pc));
  const int f = in.fmt;
  if (f != WD_F64 && f != WD_F32 && f != WD_DD) return fail(WD_ERR_ARG, "poly: FP64, FP32 or double-float fields");
  if (P.n == 0) return axpby(c, pc.s1, in, 0.0, in, out);
  WsGuard w(c);
  Field s, sp, ks, t1, t2;
  WD_TRY(w.get(f, &s));
  WD_TRY(w.get(f, &sp));
  WD_TRY(w.get(f, &ks));
  WD_TRY(w.get(f, &t1));
  WD_TRY(w.get(f, &t2));
  WD_TRY(zero(c, sp));                         // s_0 = 0
  WD_TRY(axpby(c, pc.s1, in, 0.0, in, s));     // s_1 = v / mu
  for (int k = 1; k <= P.n; ++k) {
    const Field& dst = (k == P.n) ? out : sp;  // s_{k+1} overwrites s_{k-1}
    if (f == WD_F32) {
      // FP32: the step is fused into the last hop of K_hat
      WD_TRY(khat_poly_step_f32(c, kappa, s, t1, t2, in, sp, pc.a[k], pc.mu, pc.b[k], dst));
    } else {
      WD_TRY(apply_khat(c, kappa, s, ks, t1, t2, false, false));
      WD_TRY(poly_step(c, pc.a[k], pc.mu, pc.b[k], in, s, ks, sp, dst));
    }
    if (k < P.n) std::swap(s, sp);
  }
  return WD_OK;
}

// ----------------------------------------------------------------------------
// operators for CG
enum OpKind { OP_K = 0, OP_KP = 1, OP_R = 3 };

struct Op {
  OpKind kind;
  double kappa;
  wd_poly poly;
  const PolyCoef* roots = nullptr;   // OP_R: Q in factored form
};

static int op_apply(wd_ctx* c, const Op& op, const Field& in, const Field& out, bool in_cg) {
  WsGuard w(c);
  if (op.kind == OP_K) {
    Field t1, t2;
    WD_TRY(w.get(in.fmt, &t1));
    WD_TRY(w.get(in.fmt, &t2));
    // inside CG the second hop also forms pAp = |M_hat p|^2 and alpha
    WD_TRY(apply_khat(c, op.kappa, in, out, t1, t2, in_cg, in_cg));
    return WD_OK;
  }
  if (op.kind == OP_R) {
    WD_TRY(roots_apply_f(c, op.kappa, *op.roots, in, out));
  } else {
    Field s;
    WD_TRY(w.get(in.fmt, &s));
    WD_TRY(poly_apply_f(c, op.kappa, op.poly, in.fmt, in, s));
    WD_TRY(khat_any(c, op.kappa, s, out));
  }
  if (in_cg) WD_TRY(cg_dot_pap(c, in, out));
  return WD_OK;
}

static int upload_state(wd_ctx* c) {
  WD_CUDA(cudaMemcpyAsync(c->cgs, c->cgs_host, sizeof(CGState), cudaMemcpyHostToDevice, c->stream));
  return WD_OK;
}
static int download_state(wd_ctx* c) {
  WD_CUDA(cudaMemcpyAsync(c->cgs_host, c->cgs, sizeof(CGState), cudaMemcpyDeviceToHost, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  return WD_OK;
}

// r = b - A x with b, x, r in FP64, returns |r|^2.  A x is formed in FP64, or,
// when the context selects it, in double-float (x split exactly enough into
// two FP32 words, the operator applied with error-free FP32 arithmetic, the
// result rejoined in FP64): about 48 significant bits on the FP32 pipes.
static int true_residual(wd_ctx* c, const Op& op, const Field& b, const Field& x, const Field& r,
                         const Field& t, double* rr) {
  if (c->resid_dd && c->gauge_dd) {
    WsGuard w(c);
    Field xd, td;
    WD_TRY(w.get(WD_DD, &xd));
    WD_TRY(w.get(WD_DD, &td));
    WD_TRY(convert(c, x, xd));
    WD_TRY(op_apply(c, op, xd, td, false));
    WD_TRY(convert(c, td, t));
  } else {
    WD_TRY(op_apply(c, op, x, t, false));
  }
  WD_TRY(axpby(c, 1.0, b, -1.0, t, r));
  return norm2(c, r, rr);
}

// Default reliable-update factor per sloppy precision: the iterated residual
// of FP32 stays faithful over larger reductions than that of 16-bit storage.
// The Chebyshev-recurrence operator K P is well conditioned, accurate to a few
// u_FP32 in FP32, and its FP64 application costs n+1 FP64 K_hat, so it
// recomputes the residual less often.  The root product Q = P_2 / P_1 is
// not: each real quadratic factor loses about u / |z|^2 on low modes, up to
// 6e-5 relative for P_26 / P_8 on [0.005, 8], and a sloppy cycle asked to gain
// 1e-5 stalls; it takes the K_hat factor.
static double default_delta(int prec, OpKind kind) {
  if (kind == OP_KP && prec == WD_F32) return 1e-5;
  switch (prec) {
    case WD_F32: return 1e-3;
    case WD_F16: return 5e-2;
    case WD_BF16: return 1e-1;
    default: return 1e-1;
  }
}

static int cg_core(wd_ctx* c, const Op& op, const Field& b, const Field& x, const wd_cg_params& p,
                   wd_cg_info* info, bool x_zero = false) {
  if (!(p.tol > 0) || p.maxiter < 1) return fail(WD_ERR_ARG, "cg: tol must be > 0 and maxiter >= 1");
  int prec = p.prec;
  if (prec < WD_F64 || prec > WD_BF16) return fail(WD_ERR_ARG, "cg: unknown precision");
  if (op.kind != OP_K && (prec == WD_F16 || prec == WD_BF16)) prec = WD_F32;  // poly in FP32
  const int accf = (prec == WD_F64) ? WD_F64 : WD_F32;
  const double delta = (p.delta > 0 && p.delta < 1) ? p.delta : default_delta(prec, op.kind);
  const int check = p.check_every > 0 ? p.check_every : (op.kind == OP_K ? 16 : 1);
  const long long nmat0 = c->nmat;

  wd_cg_info inf{};
  double bb;
  WD_TRY(norm2(c, b, &bb));
  if (bb == 0.0) {
    WD_TRY(zero(c, x));
    if (info) *info = inf;
    return WD_OK;
  }
  const double stop_rr = p.tol * p.tol * bb;
  // In the last sloppy cycle the iterated residual drifts from the true one by
  // about u_sloppy times the residual the cycle started from, which for the
  // polynomial operators is a sizeable part of tol.  A cycle that would end
  // within a factor 10 of tol therefore runs on to 0.3 tol: one or two cheap
  // iterations instead of one more cycle and one more FP64-accurate residual
  // (n+1 K_hat in double-float or FP64).
  const double final_rr = (op.kind != OP_K ? 0.09 : 1.0) * stop_rr;
  auto next_target = [&](double rr_now) {
    if (prec == WD_F64) return stop_rr;
    const double t = delta * delta * rr_now;
    return t < 100.0 * stop_rr ? final_rr : t;
  };
  WsGuard w(c);
  Field r, t, xs, rs, ps, aps;
  WD_TRY(w.get(WD_F64, &r));
  WD_TRY(w.get(WD_F64, &t));
  double rr;
  if (x_zero) {   // r = b without applying A
    WD_TRY(zero(c, x));
    WD_TRY(convert(c, b, r));
    rr = bb;
  } else {
    WD_TRY(true_residual(c, op, b, x, r, t, &rr));
  }
  if (!std::isfinite(rr)) return fail(WD_ERR_NAN, "cg: non-finite initial residual");
  int status = WD_OK;
  if (rr > stop_rr) {
    WD_TRY(w.get(accf, &xs));
    WD_TRY(w.get(accf, &rs));
    WD_TRY(w.get(prec, &ps));
    WD_TRY(w.get(accf, &aps));
    WD_TRY(zero(c, xs));
    WD_TRY(convert(c, r, rs));
    WD_TRY(convert(c, r, ps));
    CGState& st = *c->cgs_host;
    st = CGState{};
    st.rr = rr;
    st.rr_old = rr;
    st.stop_rr = stop_rr;
    st.upd_rr = next_target(rr);
    st.flag = 0;
    st.iter = 0;
    st.maxiter = p.maxiter;
    WD_TRY(upload_state(c));
    for (;;) {
      for (int k = 0; k < check; ++k) {
        WD_TRY(op_apply(c, op, ps, aps, true));
        WD_TRY(cg_update(c, xs, rs, ps, aps));
        WD_TRY(cg_pupdate(c, rs, ps));
      }
      WD_TRY(download_state(c));
      if (st.flag & FLAG_TIMEOUT) { status = fail(WD_ERR_TIMEOUT, "cg: a bounded stencil wait expired"); break; }
      if (st.flag & FLAG_NAN) { status = fail(WD_ERR_NAN, "cg: non-finite value in the iteration"); break; }
      if (st.flag == 0) continue;
      // fold the sloppy increment into x and recompute the FP64 residual
      WD_TRY(convert(c, xs, t));
      WD_TRY(axpby(c, 1.0, x, 1.0, t, x));
      WD_TRY(true_residual(c, op, b, x, r, t, &rr));
      inf.reliable_updates += 1;
      if (!std::isfinite(rr)) { status = fail(WD_ERR_NAN, "cg: non-finite true residual"); break; }
      if (rr <= stop_rr) break;
      if (st.flag & FLAG_MAXITER) { status = fail(WD_ERR_NOCONV, "cg: maxiter reached"); break; }
      WD_TRY(zero(c, xs));
      WD_TRY(convert(c, r, rs));
      st.beta = rr / st.rr_old;
      st.rr = rr;
      st.upd_rr = next_target(rr);
      st.flag = 0;
      WD_TRY(upload_state(c));
      WD_TRY(cg_pupdate(c, rs, ps));
    }
    inf.iters = st.iter;
  }
  inf.true_rel_resid = std::sqrt(rr / bb);
  inf.n_mat = c->nmat - nmat0;
  if (info) *info = inf;
  return status;
}

int cg_solve_f(wd_ctx* c, double kappa, const wd_poly* filt, const Field& b, const Field& x,
               const wd_cg_params& p, wd_cg_info* info, bool x_zero) {
  Op op{filt ? OP_KP : OP_K, kappa, filt ? *filt : wd_poly{0, 0, 0}};
  if (filt) {
    PolyCoef pc;
    WD_TRY(poly_coef(*filt, &pc));
  }
  return cg_core(c, op, b, x, p, info, x_zero);
}

// CG on Q(K_hat) (heat bath of the ratio term), from x = 0
int cg_solve_ratio(wd_ctx* c, double kappa, const PolyCoef& q, const Field& b, const Field& x,
                   const wd_cg_params& p, wd_cg_info* info) {
  Op op{OP_R, kappa, wd_poly{0, 0, 0}, &q};
  return cg_core(c, op, b, x, p, info, true);
}

}  // namespace wd
