// Pseudofermion terms (actions, heat bath, forces), HMC trajectory and
// integrator schedules.
//
// Terms (Section 2 of the paper; Section 4.1 for PF-MP), each on
// K = K_hat(kappa) = M_hat^dag M_hat:
//   PLAIN       S = phi^dag K^-1 phi                 heat bath phi = M^dag chi
//   HASENBUSCH  S = phi^dag M_h K^-1 M_h^dag phi     phi = M_h J^-1 M^dag chi, J = K_hat(kappa_h)
//   POLY        S = phi^dag P(K) phi                 phi = P^-1 C^dag chi, P = C^dag C
//   FILTERED    S = phi^dag [P(K) K]^-1 phi          phi = C^dag M^dag chi
//   RATIO       S = phi^dag Q(K) phi, Q = P / P_lo   phi = Q^-1 D^dag chi, Q = D^dag D
// with C = sqrt(c) prod_{k <= n/2} (K - z_k) and D the same product over the
// first half of Q's roots (Section 3.3).  Actions use the variational
// estimate S = 2 Re(b^dag X) - X^dag A X of b^dag A^-1 b, whose error is
// quadratic in the solver residual.
//
// Forces: F_a = dS/dw, w the angle of U_mu(x) -> exp(i w T_a) U_mu(x).  With
// X = A^-1 psi and Y = M_hat X:
//   PLAIN       F = 2 kappa^2 Re(Y~^dag dD X~)
//   HASENBUSCH  same with psi = M_h^dag phi, plus -2 kappa_h^2 Re(phi~^dag dD X~)
//   POLY        S = v^dag Q(K) v, Q = s prod_k (K - r_k):
//               dS = s sum_k Re(L_k^dag dK R_k), L_k = prod_{j<k} (K - r_j^*) v,
//               R_k = prod_{j>k} (K - r_j) v
//   FILTERED    minus the POLY force of Q(x) = x P(x) at v = X
//   RATIO       the POLY force with Q's roots and scale
// where A~ = (A, D^dag_oe A) and B~ = (B, D_oe B) extend even fields to the
// full lattice.  Only X and Y are kept per PLAIN/HASENBUSCH term; for
// polynomial terms the vectors R_k are recomputed segment by segment from
// ceil(sqrt(m)) checkpoints instead of being stored; the rebuild of a segment
// applies K_hat to its vectors, and the odd-site halves that K_hat forms on the
// way (D_oe R, M_hat R, D^dag_oe M_hat R) are kept for that segment's forces,
// so each root costs four hops in the forward pass instead of seven.
#include <algorithm>
#include <cmath>
#include <map>

#include "dslash_impl.cuh"

namespace wd {

static int check_term(const wd_term* t) {
  if (t == nullptr) return fail(WD_ERR_ARG, "term is null");
  if (t->kind < WD_TERM_PLAIN || t->kind > WD_TERM_RATIO) return fail(WD_ERR_ARG, "unknown term kind");
  PolyCoef pc;
  if (t->kind == WD_TERM_POLY || t->kind == WD_TERM_FILTERED) WD_TRY(poly_coef(t->poly, &pc));
  if (t->kind == WD_TERM_RATIO) WD_TRY(ratio_coef(t->poly, t->poly_lo, &pc));
  return WD_OK;
}

static int check_cg(const wd_cg_params* p) {
  if (p == nullptr) return fail(WD_ERR_ARG, "cg params are null");
  if (!(p->tol > 0) || p->maxiter < 1) return fail(WD_ERR_ARG, "cg params: tol > 0 and maxiter >= 1 required");
  if (p->prec < WD_F64 || p->prec > WD_BF16) return fail(WD_ERR_ARG, "cg params: unknown precision");
  return WD_OK;
}

static int force_fmt(const wd_cg_params& p) { return p.prec == WD_F64 ? WD_F64 : WD_F32; }

// F += coef * d/dw Re(A^dag M_hat B) = coef * (-kappa^2) Re(A~^dag dD B~)
static int mhat_outer(wd_ctx* c, double kappa, const Field& A, const Field& B, double coef, double* F) {
  WsGuard w(c);
  Field Ao, Bo;
  WD_TRY(w.get(A.fmt, &Ao));
  WD_TRY(w.get(A.fmt, &Bo));
  WD_TRY(hop(c, 1, true, A, Ao, nullptr, 0.0, false, false));
  WD_TRY(hop(c, 1, false, B, Bo, nullptr, 0.0, false, false));
  return force_outer(c, -coef * kappa * kappa, A, Ao, B, Bo, F, A.fmt);
}

static int mhat(wd_ctx* c, double kappa, bool dag, const Field& in, const Field& out) {
  WsGuard w(c);
  Field t;
  WD_TRY(w.get(in.fmt, &t));
  return apply_mhat(c, kappa, dag, in, out, t, false);
}

// out = K x - z x  (z complex; conj_z selects conj(z))
static int k_minus(wd_ctx* c, double kappa, double zr, double zi, const Field& x, const Field& out) {
  WsGuard w(c);
  Field k;
  WD_TRY(w.get(x.fmt, &k));
  WD_TRY(khat_any(c, kappa, x, k));
  return caxpby(c, 1.0, 0.0, k, -zr, -zi, x, out);
}

// Force of S = v^dag Q(K) v, Q = scale prod_k (K - r_k), added with coef.
static int poly_force(wd_ctx* c, double kappa, const std::vector<double>& rr, const std::vector<double>& ri,
                      double scale, const Field& v, double coef, double* F) {
  const int m = (int)rr.size();
  const int f = v.fmt;
  const int seg = std::max(1, (int)std::ceil(std::sqrt((double)m)));
  const int nseg = (m + seg - 1) / seg;
  WsGuard w(c);
  // buf: the R of one segment; ro / mr / mro: D_oe R, M_hat R and D^dag_oe M_hat R
  // of those R, formed while K_hat is applied to them in the segment rebuild
  std::vector<Field> cp(nseg), buf(seg), ro(seg), mr(seg), mro(seg);
  Field L, Ln, ML, cur, Lo, MLo, KR;
  for (auto& x : cp) WD_TRY(w.get(f, &x));
  for (auto* v : {&buf, &ro, &mr, &mro})
    for (auto& x : *v) WD_TRY(w.get(f, &x));
  for (Field* x : {&L, &Ln, &ML, &cur, &Lo, &MLo, &KR}) WD_TRY(w.get(f, x));
  const double k2 = kappa * kappa;
  auto seg_end = [&](int s) { return std::min((s + 1) * seg, m) - 1; };
  // backward pass: R_{m-1} = v, R_{k-1} = (K - r_k) R_k; keep R at segment ends
  WD_TRY(convert(c, v, cur));
  for (int s = nseg - 1, k = m - 1; k >= 0; --k) {
    if (s >= 0 && k == seg_end(s)) { WD_TRY(convert(c, cur, cp[s])); --s; }
    if (k > 0) WD_TRY(k_minus(c, kappa, rr[k], ri[k], cur, cur));
  }
  // forward pass over k with L_k; R_k rebuilt from the segment's checkpoint
  WD_TRY(convert(c, v, L));
  for (int s = 0; s < nseg; ++s) {
    const int a = s * seg, b = seg_end(s);
    WD_TRY(convert(c, cp[s], buf[b - a]));
    // R_{a+j-1} = (K - r_{a+j}) R_{a+j}, keeping the hops of each K R_{a+j}
    for (int j = b - a; j >= 1; --j) {
      WD_TRY(hop(c, 1, false, buf[j], ro[j], nullptr, 0.0, false, false));
      WD_TRY(hop(c, 0, false, ro[j], mr[j], &buf[j], -k2, false, false));
      WD_TRY(hop(c, 1, true, mr[j], mro[j], nullptr, 0.0, false, false));
      WD_TRY(hop(c, 0, true, mro[j], KR, &mr[j], -k2, false, false));
      c->nmat += 1;
      WD_TRY(caxpby(c, 1.0, 0.0, KR, -rr[a + j], -ri[a + j], buf[j], buf[j - 1]));
    }
    for (int k = a; k <= b; ++k) {
      const int j = k - a;
      const Field& R = buf[j];
      // Lo = D_oe L, ML = M_hat L, MLo = D^dag_oe ML (the odd halves of L~ and
      // (M L)~), and the same for R (kept from the rebuild except for its
      // first vector): each used twice below
      WD_TRY(hop(c, 1, false, L, Lo, nullptr, 0.0, false, false));
      WD_TRY(hop(c, 0, false, Lo, ML, &L, -k2, false, false));
      WD_TRY(hop(c, 1, true, ML, MLo, nullptr, 0.0, false, false));
      if (j == 0) {
        WD_TRY(hop(c, 1, false, R, ro[0], nullptr, 0.0, false, false));
        WD_TRY(hop(c, 0, false, ro[0], mr[0], &R, -k2, false, false));
        WD_TRY(hop(c, 1, true, mr[0], mro[0], nullptr, 0.0, false, false));
      }
      // Re((M R)~^dag dD L~) and Re((M L)~^dag dD R~), one pass over the links
      const double cf[2] = {-coef * scale * k2, -coef * scale * k2};
      const Field Ye[2] = {mr[j], ML}, Yo[2] = {mro[j], MLo}, Xe[2] = {L, R}, Xo[2] = {Lo, ro[j]};
      WD_TRY(force_outer2(c, cf, Ye, Yo, Xe, Xo, F));
      if (k < m - 1) {
        // K L = M^dag (M L) = ML - kappa^2 D^dag_eo MLo: one more hop
        WD_TRY(hop(c, 0, true, MLo, Ln, &ML, -k2, false, false));
        c->nmat += 1;
        WD_TRY(caxpby(c, 1.0, 0.0, Ln, -rr[k], ri[k], L, Ln));   // (K - conj r_k) L
        std::swap(L, Ln);
      }
    }
  }
  return WD_OK;
}

// C^dag v = sqrt(c) prod_{k<=n/2} (K - conj z_k) v (FP64 fields; the factors in
// double-float when the context selects it for FP64-accurate operators)
static int apply_cdag(wd_ctx* c, double kappa, const PolyCoef& pc, const Field& v, const Field& out) {
  if (c->resid_dd && c->gauge_dd) {
    WsGuard w(c);
    Field a;
    WD_TRY(w.get(WD_DD, &a));
    WD_TRY(convert(c, v, a));
    WD_TRY(axpby(c, std::sqrt(pc.scale), a, 0.0, a, a));
    for (int k = 0; k < pc.n / 2; ++k) WD_TRY(k_minus(c, kappa, pc.zr[k], -pc.zi[k], a, a));
    return convert(c, a, out);
  }
  WD_TRY(axpby(c, std::sqrt(pc.scale), v, 0.0, v, out));
  for (int k = 0; k < pc.n / 2; ++k) WD_TRY(k_minus(c, kappa, pc.zr[k], -pc.zi[k], out, out));
  return WD_OK;
}

static int solve(wd_ctx* c, double kappa, const wd_poly* filt, const Field& b, const Field& x,
                 const wd_cg_params& p) {
  wd_cg_info info;
  return cg_solve_f(c, kappa, filt, b, x, p, &info, true);
}

// FP64-accurate operator applications on FP64 fields for the actions and the
// heat bath: in FP64, or in double-float when the context selects it for its
// residuals (the same accuracy class, about 1e-13 relative).
static int poly_apply_hp(wd_ctx* c, double kappa, const wd_poly& P, const Field& in, const Field& out) {
  if (!(c->resid_dd && c->gauge_dd)) return poly_apply_f(c, kappa, P, WD_F64, in, out);
  WsGuard w(c);
  Field a, b;
  WD_TRY(w.get(WD_DD, &a));
  WD_TRY(w.get(WD_DD, &b));
  WD_TRY(convert(c, in, a));
  WD_TRY(poly_apply_f(c, kappa, P, WD_DD, a, b));
  return convert(c, b, out);
}

static int roots_apply_hp(wd_ctx* c, double kappa, const PolyCoef& q, const Field& in, const Field& out) {
  if (!(c->resid_dd && c->gauge_dd)) return roots_apply_f(c, kappa, q, in, out);
  WsGuard w(c);
  Field a, b;
  WD_TRY(w.get(WD_DD, &a));
  WD_TRY(w.get(WD_DD, &b));
  WD_TRY(convert(c, in, a));
  WD_TRY(roots_apply_f(c, kappa, q, a, b));
  return convert(c, b, out);
}

static int khat_hp(wd_ctx* c, double kappa, const Field& in, const Field& out) {
  if (!(c->resid_dd && c->gauge_dd)) return khat_any(c, kappa, in, out);
  WsGuard w(c);
  Field a, b;
  WD_TRY(w.get(WD_DD, &a));
  WD_TRY(w.get(WD_DD, &b));
  WD_TRY(convert(c, in, a));
  WD_TRY(khat_any(c, kappa, a, b));
  return convert(c, b, out);
}

// S of one term; when Xo / Yo are given, also the solution X = A^-1 psi and
// (PLAIN, HASENBUSCH) Y = M_hat X, the only vectors the force needs.
int term_action(wd_ctx* c, const wd_term& t, const Field& phi, const wd_cg_params& p, double* S,
                const Field* Xo = nullptr, const Field* Yo = nullptr) {
  WsGuard w(c);
  Field b, X, AX, tmp;
  WD_TRY(w.get(WD_F64, &b));
  WD_TRY(w.get(WD_F64, &X));
  WD_TRY(w.get(WD_F64, &AX));
  double re, xax;
  switch (t.kind) {
    case WD_TERM_PLAIN:
    case WD_TERM_HASENBUSCH: {
      if (t.kind == WD_TERM_PLAIN) WD_TRY(convert(c, phi, b));
      else WD_TRY(mhat(c, t.kappa_h, true, phi, b));
      WD_TRY(solve(c, t.kappa, nullptr, b, X, p));
      WD_TRY(mhat(c, t.kappa, false, X, AX));       // |M X|^2 = X^dag K X
      WD_TRY(dot(c, b, X, &re, nullptr));
      WD_TRY(norm2(c, AX, &xax));
      *S = 2.0 * re - xax;
      if (Xo) WD_TRY(convert(c, X, *Xo));
      if (Yo) WD_TRY(convert(c, AX, *Yo));
      return WD_OK;
    }
    case WD_TERM_POLY: {
      WD_TRY(poly_apply_hp(c, t.kappa, t.poly, phi, AX));
      WD_TRY(dot(c, phi, AX, &re, nullptr));
      *S = re;
      return WD_OK;
    }
    case WD_TERM_RATIO: {
      PolyCoef q;
      WD_TRY(ratio_coef(t.poly, t.poly_lo, &q));
      WD_TRY(roots_apply_hp(c, t.kappa, q, phi, AX));
      WD_TRY(dot(c, phi, AX, &re, nullptr));
      *S = re;
      return WD_OK;
    }
    case WD_TERM_FILTERED: {
      WD_TRY(w.get(WD_F64, &tmp));
      WD_TRY(solve(c, t.kappa, &t.poly, phi, X, p));
      WD_TRY(poly_apply_hp(c, t.kappa, t.poly, X, tmp));
      WD_TRY(khat_hp(c, t.kappa, tmp, AX));
      WD_TRY(dot(c, phi, X, &re, nullptr));
      WD_TRY(dot(c, X, AX, &xax, nullptr));
      *S = 2.0 * re - xax;
      if (Xo) WD_TRY(convert(c, X, *Xo));
      return WD_OK;
    }
  }
  return fail(WD_ERR_ARG, "unknown term kind");
}

int term_heatbath(wd_ctx* c, const wd_term& t, const Field& chi, const wd_cg_params& p, const Field& phi) {
  WsGuard w(c);
  Field y, z;
  WD_TRY(w.get(WD_F64, &y));
  switch (t.kind) {
    case WD_TERM_PLAIN:
      return mhat(c, t.kappa, true, chi, phi);
    case WD_TERM_HASENBUSCH:
      WD_TRY(w.get(WD_F64, &z));
      WD_TRY(mhat(c, t.kappa, true, chi, y));
      WD_TRY(solve(c, t.kappa_h, nullptr, y, z, p));
      return mhat(c, t.kappa_h, false, z, phi);
    case WD_TERM_POLY: {
      // phi = P^-1 C^dag chi = K [K P]^-1 C^dag chi (P and K commute): the filtered
      // operator K P is close to 1 on [eps, lam], so its solve takes a few
      // iterations where CG on P(K) itself, about as ill-conditioned as K, takes
      // as many as a K solve, each n times dearer.  The same residual bound
      // |C^dag chi - K P x| <= tol |C^dag chi| gives the same error in phi.
      PolyCoef pc;
      WD_TRY(poly_coef(t.poly, &pc));
      WD_TRY(w.get(WD_F64, &z));
      WD_TRY(apply_cdag(c, t.kappa, pc, chi, y));
      WD_TRY(solve(c, t.kappa, &t.poly, y, z, p));
      return khat_hp(c, t.kappa, z, phi);
    }
    case WD_TERM_FILTERED: {
      PolyCoef pc;
      WD_TRY(poly_coef(t.poly, &pc));
      WD_TRY(mhat(c, t.kappa, true, chi, y));
      return apply_cdag(c, t.kappa, pc, y, phi);
    }
    case WD_TERM_RATIO: {
      PolyCoef q;
      WD_TRY(ratio_coef(t.poly, t.poly_lo, &q));
      WD_TRY(apply_cdag(c, t.kappa, q, chi, y));    // D^dag chi
      WD_TRY(zero(c, phi));
      wd_cg_info info;
      return cg_solve_ratio(c, t.kappa, q, y, phi, p, &info);
    }
  }
  return fail(WD_ERR_ARG, "unknown term kind");
}

// Force from a given solution X (and Y = M_hat X, or nullptr to form it):
// no solve.  POLY and RATIO ignore X and Y.  f = FP64 or FP32 arithmetic.
int term_force_xy(wd_ctx* c, const wd_term& t, const Field& phi, const Field* X, const Field* Y, int f,
                  double coef, double* F) {
  WsGuard w(c);
  Field Xf, Yf, phif;
  switch (t.kind) {
    case WD_TERM_PLAIN:
    case WD_TERM_HASENBUSCH: {
      WD_TRY(w.get(f, &Xf));
      WD_TRY(w.get(f, &Yf));
      WD_TRY(convert(c, *X, Xf));
      if (Y) WD_TRY(convert(c, *Y, Yf));
      else WD_TRY(mhat(c, t.kappa, false, Xf, Yf));
      WD_TRY(mhat_outer(c, t.kappa, Yf, Xf, -2.0 * coef, F));
      if (t.kind == WD_TERM_HASENBUSCH) {
        WD_TRY(w.get(f, &phif));
        WD_TRY(convert(c, phi, phif));
        WD_TRY(mhat_outer(c, t.kappa_h, phif, Xf, 2.0 * coef, F));
      }
      return WD_OK;
    }
    case WD_TERM_POLY: {
      PolyCoef pc;
      WD_TRY(poly_coef(t.poly, &pc));
      WD_TRY(w.get(f, &phif));
      WD_TRY(convert(c, phi, phif));
      return poly_force(c, t.kappa, pc.zr, pc.zi, pc.scale, phif, coef, F);
    }
    case WD_TERM_RATIO: {
      PolyCoef q;
      WD_TRY(ratio_coef(t.poly, t.poly_lo, &q));
      WD_TRY(w.get(f, &phif));
      WD_TRY(convert(c, phi, phif));
      return poly_force(c, t.kappa, q.zr, q.zi, q.scale, phif, coef, F);
    }
    case WD_TERM_FILTERED: {
      PolyCoef pc;
      WD_TRY(poly_coef(t.poly, &pc));
      WD_TRY(w.get(f, &Xf));
      WD_TRY(convert(c, *X, Xf));
      std::vector<double> rr(1, 0.0), ri(1, 0.0);
      rr.insert(rr.end(), pc.zr.begin(), pc.zr.end());
      ri.insert(ri.end(), pc.zi.begin(), pc.zi.end());
      return poly_force(c, t.kappa, rr, ri, pc.scale, Xf, -coef, F);
    }
  }
  return fail(WD_ERR_ARG, "unknown term kind");
}

int term_force(wd_ctx* c, const wd_term& t, const Field& phi, const wd_cg_params& p, double coef, double* F) {
  const int f = force_fmt(p);
  WsGuard w(c);
  Field b, X;
  WD_TRY(w.get(WD_F64, &X));
  switch (t.kind) {
    case WD_TERM_PLAIN:
    case WD_TERM_HASENBUSCH:
      WD_TRY(w.get(WD_F64, &b));
      if (t.kind == WD_TERM_PLAIN) WD_TRY(convert(c, phi, b));
      else WD_TRY(mhat(c, t.kappa_h, true, phi, b));
      WD_TRY(solve(c, t.kappa, nullptr, b, X, p));
      return term_force_xy(c, t, phi, &X, nullptr, f, coef, F);
    case WD_TERM_POLY:
    case WD_TERM_RATIO:
      return term_force_xy(c, t, phi, nullptr, nullptr, f, coef, F);
    case WD_TERM_FILTERED:
      WD_TRY(solve(c, t.kappa, &t.poly, phi, X, p));
      return term_force_xy(c, t, phi, &X, nullptr, f, coef, F);
  }
  return fail(WD_ERR_ARG, "unknown term kind");
}

// ----------------------------------------------------------------------------
// schedules (Section 3.2)
struct OpV {
  int kind, group;
  double eps;
};

static void base_scheme(int kind, int n, double tau, int g, std::vector<OpV>& out) {
  const double h = tau / n;
  const double lam = 0.1931833275037836;   // Omelyan, Mryglod, Folk (2003), 2MN
  for (int i = 0; i < n; ++i) {
    if (kind == 0) {
      out.push_back({1, g, h / 2});
      out.push_back({0, 0, h});
      out.push_back({1, g, h / 2});
    } else {
      out.push_back({1, g, lam * h});
      out.push_back({0, 0, h / 2});
      out.push_back({1, g, (1 - 2 * lam) * h});
      out.push_back({0, 0, h / 2});
      out.push_back({1, g, lam * h});
    }
  }
}

static void nested_rec(int kind, double tau, int lv, int nl, const int* groups, const int* steps,
                       std::vector<OpV>& out) {
  std::vector<OpV> ops;
  base_scheme(kind, steps[lv], tau, groups[lv], ops);
  for (auto& o : ops) {
    if (o.kind == 0 && lv + 1 < nl) nested_rec(kind, o.eps, lv + 1, nl, groups, steps, out);
    else out.push_back(o);
  }
}

// S steps between two T steps commute (each force depends on U only): sum
// them per group, in order of first appearance.
static std::vector<OpV> canonical(const std::vector<OpV>& in) {
  std::vector<OpV> out;
  std::vector<OpV> run;
  auto flush = [&]() {
    for (auto& o : run) out.push_back(o);
    run.clear();
  };
  for (auto& o : in) {
    if (o.kind == 0) {
      flush();
      out.push_back(o);
    } else {
      bool merged = false;
      for (auto& r : run)
        if (r.group == o.group) { r.eps += o.eps; merged = true; break; }
      if (!merged) run.push_back(o);
    }
  }
  flush();
  return out;
}

static int emit(const std::vector<OpV>& v, wd_op* ops, int cap, int* nops) {
  if (nops) *nops = (int)v.size();
  if (ops) for (int i = 0; i < (int)v.size() && i < cap; ++i) ops[i] = wd_op{v[i].kind, v[i].group, v[i].eps};
  return WD_OK;
}

}  // namespace wd

using namespace wd;

extern "C" {

int wd_schedule_nested(int kind, double tau, int nlevels, const int* groups, const int* steps, wd_op* ops,
                       int cap, int* nops) {
  if (kind != 0 && kind != 1) return fail(WD_ERR_ARG, "kind must be 0 (leapfrog) or 1 (2MN)");
  if (nlevels < 1 || !groups || !steps || !(tau > 0)) return fail(WD_ERR_ARG, "bad schedule arguments");
  for (int i = 0; i < nlevels; ++i)
    if (steps[i] < 1) return fail(WD_ERR_ARG, "steps must be >= 1");
  std::vector<OpV> v;
  nested_rec(kind, tau, 0, nlevels, groups, steps, v);
  return emit(canonical(v), ops, cap, nops);
}

int wd_schedule_generalised(int kind, double tau, int ngroups, const int* groups, const int* nsteps,
                            wd_op* ops, int cap, int* nops) {
  if (kind != 0 && kind != 1) return fail(WD_ERR_ARG, "kind must be 0 (leapfrog) or 1 (2MN)");
  if (ngroups < 1 || !groups || !nsteps || !(tau > 0)) return fail(WD_ERR_ARG, "bad schedule arguments");
  struct Ev { double t; int pos; OpV op; };
  std::vector<Ev> ev;
  for (int i = 0; i < ngroups; ++i) {
    if (nsteps[i] < 1) return fail(WD_ERR_ARG, "nsteps must be >= 1");
    std::vector<OpV> s;
    base_scheme(kind, nsteps[i], tau, groups[i], s);
    double t = 0;
    for (auto& o : s) {
      if (o.kind == 0) t += o.eps;
      else ev.push_back({t, i, o});
    }
  }
  const double tolt = 1e-12 * tau;
  std::vector<double> times;
  for (auto& e : ev) times.push_back(e.t);
  std::sort(times.begin(), times.end());
  std::vector<double> uniq;
  for (double t : times)
    if (uniq.empty() || t - uniq.back() > tolt) uniq.push_back(t);
  std::vector<OpV> out;
  double prev = 0;
  for (double t : uniq) {
    if (t - prev > tolt) out.push_back({0, 0, t - prev});
    std::vector<Ev> here;
    for (auto& e : ev)
      if (std::fabs(e.t - t) <= tolt) here.push_back(e);
    const bool desc = t >= tau / 2 - tolt;
    std::stable_sort(here.begin(), here.end(),
                     [&](const Ev& a, const Ev& b) { return desc ? a.pos > b.pos : a.pos < b.pos; });
    for (auto& e : here) out.push_back(e.op);
    prev = t;
  }
  if (tau - prev > tolt) out.push_back({0, 0, tau - prev});
  return emit(canonical(out), ops, cap, nops);
}

int cg_solve(wd_ctx* c, double kappa, const wd_poly* filt, const double* b, double* x,
             const wd_cg_params* p, wd_cg_info* info) {
  if (!c) return fail(WD_ERR_ARG, "null context");
  if (!b || !x) return fail(WD_ERR_ARG, "b and x must be device pointers");
  WD_TRY(check_cg(p));
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  if (filt) {
    PolyCoef pc;
    WD_TRY(poly_coef(*filt, &pc));
  }
  return cg_solve_f(c, kappa, filt, wrap_f64(c, b), wrap_f64(c, x), *p, info);
}

int poly_filter_apply(wd_ctx* c, double kappa, const wd_poly* poly, int prec, const double* in, double* out) {
  if (!c || !poly || !in || !out) return fail(WD_ERR_ARG, "null argument");
  if (prec != WD_F64 && prec != WD_F32) return fail(WD_ERR_ARG, "poly_filter_apply: FP64 or FP32");
  if (in == out) return fail(WD_ERR_ARG, "poly_filter_apply: in and out must differ");
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  PolyCoef pc;
  WD_TRY(poly_coef(*poly, &pc));
  if (prec == WD_F64) return poly_apply_f(c, kappa, *poly, prec, wrap_f64(c, in), wrap_f64(c, out));
  WsGuard w(c);
  Field a, b;
  WD_TRY(w.get(WD_F32, &a));
  WD_TRY(w.get(WD_F32, &b));
  WD_TRY(convert(c, wrap_f64(c, in), a));
  WD_TRY(poly_apply_f(c, kappa, *poly, prec, a, b));
  return convert(c, b, wrap_f64(c, out));
}

int pf_action(wd_ctx* c, const wd_term* term, const double* phi, const wd_cg_params* p, double* S) {
  if (!c || !phi || !S) return fail(WD_ERR_ARG, "null argument");
  WD_TRY(check_term(term));
  WD_TRY(check_cg(p));
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  return term_action(c, *term, wrap_f64(c, phi), *p, S);
}

int pf_action_xy(wd_ctx* c, const wd_term* term, const double* phi, const wd_cg_params* p, double* S,
                 double* X, double* Y) {
  if (!c || !phi || !S) return fail(WD_ERR_ARG, "null argument");
  WD_TRY(check_term(term));
  WD_TRY(check_cg(p));
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  if ((X && (X == phi || X == Y)) || (Y && Y == phi)) return fail(WD_ERR_ARG, "phi, X and Y must differ");
  Field fx = wrap_f64(c, X), fy = wrap_f64(c, Y);
  return term_action(c, *term, wrap_f64(c, phi), *p, S, X ? &fx : nullptr, Y ? &fy : nullptr);
}

int fermion_force_xy(wd_ctx* c, const wd_term* term, const double* phi, const double* X, const double* Y,
                     int prec, double coef, double* F) {
  if (!c || !phi || !F) return fail(WD_ERR_ARG, "null argument");
  WD_TRY(check_term(term));
  if (prec != WD_F64 && prec != WD_F32) return fail(WD_ERR_ARG, "fermion_force_xy: prec must be FP64 or FP32");
  if (term->kind != WD_TERM_POLY && term->kind != WD_TERM_RATIO && !X) return fail(WD_ERR_ARG, "fermion_force_xy: X is required for this term");
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  Field fx = wrap_f64(c, X), fy = wrap_f64(c, Y);
  const bool useY = Y != nullptr && (term->kind == WD_TERM_PLAIN || term->kind == WD_TERM_HASENBUSCH);
  return term_force_xy(c, *term, wrap_f64(c, phi), X ? &fx : nullptr, useY ? &fy : nullptr, prec, coef, F);
}

int pf_heatbath(wd_ctx* c, const wd_term* term, const double* chi, const wd_cg_params* p, double* phi) {
  if (!c || !chi || !phi) return fail(WD_ERR_ARG, "null argument");
  if (chi == phi) return fail(WD_ERR_ARG, "chi and phi must differ");
  WD_TRY(check_term(term));
  WD_TRY(check_cg(p));
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  return term_heatbath(c, *term, wrap_f64(c, chi), *p, wrap_f64(c, phi));
}

int fermion_force(wd_ctx* c, const wd_term* term, const double* phi, const wd_cg_params* p, double coef,
                  double* F) {
  if (!c || !phi || !F) return fail(WD_ERR_ARG, "null argument");
  WD_TRY(check_term(term));
  WD_TRY(check_cg(p));
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  return term_force(c, *term, wrap_f64(c, phi), *p, coef, F);
}

int gauge_action(wd_ctx* c, double beta, double* S) {
  if (!c || !S) return fail(WD_ERR_ARG, "null argument");
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  double s;
  WD_TRY(gauge_action_k(c, &s));
  *S = beta * s;
  return WD_OK;
}

int gauge_force(wd_ctx* c, double beta, int prec, double coef, double* F) {
  if (!c || !F) return fail(WD_ERR_ARG, "null argument");
  if (prec != WD_F64 && prec != WD_F32) return fail(WD_ERR_ARG, "gauge_force: FP64 or FP32");
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  return gauge_force_k(c, beta, prec, coef, F);
}

int step_T(wd_ctx* c, const double* P, double eps) {
  if (!c || !P) return fail(WD_ERR_ARG, "null argument");
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  return step_T_k(c, P, eps);
}

int step_S(wd_ctx* c, double* P, const double* F, double eps) {
  if (!c || !P || !F) return fail(WD_ERR_ARG, "null argument");
  return step_S_k(c, P, F, eps);
}

int kinetic_energy(wd_ctx* c, const double* P, double* out) {
  if (!c || !P || !out) return fail(WD_ERR_ARG, "null argument");
  return kinetic_k(c, P, out);
}

int gaussian_draw(wd_ctx* c, int what, int parity, uint64_t seed, uint64_t stream, double* out) {
  if (!c || !out) return fail(WD_ERR_ARG, "null argument");
  if (what != 0 && what != 1) return fail(WD_ERR_ARG, "what must be 0 (spinor) or 1 (algebra)");
  if (what == 0 && parity != 0 && parity != 1) return fail(WD_ERR_ARG, "parity must be 0 or 1");
  return gaussian_draw_k(c, what, parity, seed, stream, out);
}

}  // extern "C"

namespace wd {

// Phase timing of a trajectory: (phase, start, stop) events on the context
// stream, read once at the end.
struct Phases {
  struct Mark { int phase; cudaEvent_t e0, e1; };
  wd_ctx* c;
  std::vector<Mark> marks;
  void begin(int phase) {
    Mark m{phase, nullptr, nullptr};
    cudaEventCreate(&m.e0);
    cudaEventCreate(&m.e1);
    cudaEventRecord(m.e0, c->stream);
    marks.push_back(m);
  }
  void end() { cudaEventRecord(marks.back().e1, c->stream); }
  ~Phases() {
    for (auto& m : marks) {
      cudaEventDestroy(m.e0);
      cudaEventDestroy(m.e1);
    }
  }
};
enum { PH_HB = 0, PH_H, PH_T, PH_GF, PH_F0 };

// The integrator on momenta P (Section 2: T[eps] U = exp(i eps P) U,
// S[eps] P = P - eps F; Section 3.2: the schedule), pseudofermions fixed.
static int run_ops(wd_ctx* c, double* P, int nterms, const wd_term* terms, const int* groups, const Field* phi,
                   double beta, int nops, const wd_op* ops, const wd_cg_params& md, int fprec, int* nf_out,
                   Phases* ph) {
  int nf = 0;
  for (int k = 0; k < nops; ++k) {
    const wd_op& o = ops[k];
    if (o.kind == 0) {
      if (ph) ph->begin(PH_T);
      WD_TRY(step_T_k(c, P, o.eps));
      if (ph) ph->end();
    } else {
      if (o.group == -1 && beta > 0) {
        if (ph) ph->begin(PH_GF);
        WD_TRY(gauge_force_k(c, beta, fprec, -o.eps, P));
        if (ph) ph->end();
        ++nf;
      }
      for (int i = 0; i < nterms; ++i) {
        if (groups[i] != o.group) continue;
        if (ph) ph->begin(o.group >= 0 && o.group < 4 ? PH_F0 + o.group : PH_GF);
        WD_TRY(term_force(c, terms[i], phi[i], md, -o.eps, P));
        if (ph) ph->end();
        ++nf;
      }
    }
  }
  if (nf_out) *nf_out = nf;
  return WD_OK;
}

static int check_ops(int nops, const wd_op* ops) {
  if (nops < 1 || !ops) return fail(WD_ERR_ARG, "empty integrator");
  for (int k = 0; k < nops; ++k)
    if (ops[k].kind != 0 && ops[k].kind != 1) return fail(WD_ERR_ARG, "op kind must be 0 (T) or 1 (S)");
  return WD_OK;
}

}  // namespace wd

extern "C" {

int integrate(wd_ctx* c, double* P, const wd_integrate_params* p, int* n_force_evals) {
  if (!c || !P || !p) return fail(WD_ERR_ARG, "null argument");
  if (p->nterms < 0 || (p->nterms > 0 && (!p->terms || !p->term_group || !p->phi))) return fail(WD_ERR_ARG, "bad terms");
  WD_TRY(check_ops(p->nops, p->ops));
  for (int i = 0; i < p->nterms; ++i) {
    WD_TRY(check_term(&p->terms[i]));
    if (!p->phi[i]) return fail(WD_ERR_ARG, "pseudofermion pointer is null");
  }
  WD_TRY(check_cg(&p->cg_md));
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  wd_cg_params md = p->cg_md;
  md.prec = p->force_prec == WD_F64 ? WD_F64 : p->cg_md.prec;
  const int fprec = p->force_prec == WD_F64 ? WD_F64 : WD_F32;
  std::vector<Field> phi(p->nterms);
  for (int i = 0; i < p->nterms; ++i) phi[i] = wrap_f64(c, p->phi[i]);
  return run_ops(c, P, p->nterms, p->terms, p->term_group, phi.data(), p->beta, p->nops, p->ops, md, fprec,
                 n_force_evals, nullptr);
}

int hmc_trajectory(wd_ctx* c, const wd_hmc_params* p, double u, wd_hmc_result* res) {
  if (!c || !p || !res) return fail(WD_ERR_ARG, "null argument");
  if (p->nterms < 0 || (p->nterms > 0 && (!p->terms || !p->term_group))) return fail(WD_ERR_ARG, "bad terms");
  WD_TRY(check_ops(p->nops, p->ops));
  if (!(u >= 0.0 && u < 1.0)) return fail(WD_ERR_ARG, "u must be in [0, 1)");
  for (int i = 0; i < p->nterms; ++i) WD_TRY(check_term(&p->terms[i]));
  WD_TRY(check_cg(&p->cg_md));
  WD_TRY(check_cg(&p->cg_acc));
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  const long Vh = c->g.Vh;
  if (!c->gauge_backup) WD_CUDA(cudaMalloc(&c->gauge_backup, sizeof(double2) * 72 * Vh));
  if (!c->mom) WD_CUDA(cudaMalloc(&c->mom, sizeof(double) * 64 * Vh));
  WD_CUDA(cudaMemcpyAsync(c->gauge_backup, c->gauge64, sizeof(double2) * 72 * Vh, cudaMemcpyDeviceToDevice,
                          c->stream));
  const long long nmat0 = c->nmat;
  const uint64_t base = p->traj_index * 64;
  wd_cg_params md = p->cg_md;
  md.prec = p->force_prec == WD_F64 ? WD_F64 : p->cg_md.prec;
  WsGuard w(c);
  std::vector<Field> phi(p->nterms);
  Field chi;
  WD_TRY(w.get(WD_F64, &chi));
  for (auto& f : phi) WD_TRY(w.get(WD_F64, &f));
  Phases ph{c, {}};
  auto begin = [&](int phase) { ph.begin(phase); };
  auto end = [&]() { ph.end(); };
  // momenta and pseudofermions
  begin(PH_HB);
  WD_TRY(gaussian_draw_k(c, 1, 0, p->seed, base, c->mom));
  double noise = 0.0;   // sum_i chi_i^dag chi_i
  for (int i = 0; i < p->nterms; ++i) {
    // chi ~ exp(-chi^dag chi) (Section 2): real and imaginary parts N(0, 1/2),
    // the unit-variance Philox draw scaled by 1/sqrt(2)
    WD_TRY(gaussian_draw_k(c, 0, 0, p->seed, base + 1 + i, (double*)chi.data));
    WD_TRY(axpby(c, M_SQRT1_2, chi, 0.0, chi, chi));
    if (!p->h0_solve) {
      double n2;
      WD_TRY(norm2(c, chi, &n2));
      noise += n2;
    }
    WD_TRY(term_heatbath(c, p->terms[i], chi, p->cg_acc, phi[i]));
  }
  end();
  // H = sum tr P^2 + S_G + sum_i S_i(phi_i).  At the start of the trajectory the
  // heat bath fixes S_i(phi_i) = chi_i^dag chi_i (to the heat bath's solver
  // tolerance), which replaces the solves unless h0_solve asks for them.
  auto hamiltonian = [&](double* H, double* SG, bool from_noise) -> int {
    double k, s, sum;
    WD_TRY(kinetic_k(c, c->mom, &k));
    sum = k;
    *SG = 0;
    if (p->beta > 0) {
      WD_TRY(gauge_action_k(c, &s));
      *SG = p->beta * s;
      sum += *SG;
    }
    if (from_noise) {
      sum += noise;
    } else {
      for (int i = 0; i < p->nterms; ++i) {
        WD_TRY(term_action(c, p->terms[i], phi[i], p->cg_acc, &s));
        sum += s;
      }
    }
    *H = sum;
    return WD_OK;
  };
  begin(PH_H);
  WD_TRY(hamiltonian(&res->H0, &res->S_gauge0, !p->h0_solve));
  end();
  int nf = 0;
  const int fprec = p->force_prec == WD_F64 ? WD_F64 : WD_F32;
  WD_TRY(run_ops(c, c->mom, p->nterms, p->terms, p->term_group, phi.data(), p->beta, p->nops, p->ops, md, fprec,
                 &nf, &ph));
  begin(PH_H);
  WD_TRY(hamiltonian(&res->H1, &res->S_gauge1, false));
  end();
  res->dH = res->H1 - res->H0;
  res->n_force_evals = nf;
  int acc = 0;
  WD_TRY(metropolis(res->dH, u, &acc));
  res->accepted = acc;
  if (!acc) {
    WD_CUDA(cudaMemcpyAsync(c->gauge64, c->gauge_backup, sizeof(double2) * 72 * Vh, cudaMemcpyDeviceToDevice,
                            c->stream));
    WD_TRY(gauge_lowprec_k(c));
  }
  res->n_mat = c->nmat - nmat0;
  WD_CUDA(cudaStreamSynchronize(c->stream));
  double t[PH_F0 + 4] = {0};
  for (auto& m : ph.marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, m.e0, m.e1) == cudaSuccess) t[m.phase] += ms;
  }
  res->t_heatbath_ms = t[PH_HB];
  res->t_hamiltonian_ms = t[PH_H];
  res->t_T_ms = t[PH_T];
  res->t_gauge_force_ms = t[PH_GF];
  for (int g = 0; g < 4; ++g) res->t_force_group_ms[g] = t[PH_F0 + g];
  return WD_OK;
}

int hmc_trajectory_host(wd_ctx* c, const wd_hmc_params* p, double u, const double* U_in, double* U_out,
                        wd_hmc_result* res) {
  if (!c || !p || !res || !U_in || !U_out) return fail(WD_ERR_ARG, "null argument");
  const size_t bytes = sizeof(double) * 72 * (size_t)c->g.V;
  if (!c->lex_stage) WD_CUDA(cudaMalloc(&c->lex_stage, bytes));
  WD_CUDA(cudaMemcpyAsync(c->lex_stage, U_in, bytes, cudaMemcpyHostToDevice, c->stream));
  WD_TRY(wd_gauge_load(c, c->lex_stage));
  WD_TRY(hmc_trajectory(c, p, u, res));
  WD_TRY(wd_gauge_store(c, c->lex_stage));
  WD_CUDA(cudaMemcpyAsync(U_out, c->lex_stage, bytes, cudaMemcpyDeviceToHost, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  return WD_OK;
}

}  // extern "C"
