// Vector kernels on half-lattice spinor fields: precision conversion, linear
// combinations, FP64 inner products (deterministic grid sums), and the fused
// conjugate-gradient updates whose scalars stay on the device.
//
// Arithmetic: FP64 when every field is FP64, FP32 otherwise; inner products
// and norms always accumulate in FP64.
#include "dslash_impl.cuh"

namespace wd {

constexpr int BL_THREADS = 256;

size_t field_bytes(int fmt, long Vh) {
  switch (fmt) {
    case WD_F64:
    case WD_DD: return (size_t)Vh * 24 * 8;
    case WD_F32: return (size_t)Vh * 24 * 4;
    default: return (size_t)Vh * 24 * 2;   // the norm array is separate
  }
}

template <class Fn>
static int with_fmt(const Field& f, Fn&& fn) {
  switch (f.fmt) {
    case WD_F64: return fn(sp64(f));
    case WD_F32: return fn(sp32(f));
    case WD_F16: return fn(sp16<__half>(f));
    case WD_BF16: return fn(sp16<__nv_bfloat16>(f));
    case WD_DD: return fn(spdd(f));
  }
  return fail(WD_ERR_ARG, "unknown field format");
}

// arithmetic of a kernel on two formats: FP64 when both are FP64, double-float
// when both are double-float, FP64 for conversions between the two, else FP32
template <class A, class B> struct Pick { using T = float; };
template <> struct Pick<SpF64, SpF64> { using T = double; };
template <> struct Pick<SpDD, SpDD> { using T = dd; };
template <> struct Pick<SpF64, SpDD> { using T = double; };
template <> struct Pick<SpDD, SpF64> { using T = double; };

// ---------------------------------------------------------------------------
template <class T, class In, class Out>
__global__ void k_convert(long n, In in, Out out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cpx<T> s[12];
  in.loadT(i, s);
  out.store(i, s);
}

int convert(wd_ctx* c, const Field& in, const Field& out) {
  const long n = c->g.Vh;
  return with_fmt(in, [&](auto I) {
    return with_fmt(out, [&](auto O) {
      using T = typename Pick<decltype(I), decltype(O)>::T;
      k_convert<T><<<nblocks(n, BL_THREADS), BL_THREADS, 0, c->stream>>>(n, I, O);
      WD_CHECK_LAUNCH();
      return (int)WD_OK;
    });
  });
}

// out = (ar + i ai) x + (br + i bi) y, all fields of one format
template <class T, class F>
__global__ void k_caxpby(long n, T ar, T ai, F x, T br, T bi, F y, F out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cpx<T> a[12], b[12];
  x.loadT(i, a);
  y.loadT(i, b);
  const cpx<T> ca = mk(ar, ai), cb = mk(br, bi);
#pragma unroll
  for (int j = 0; j < 12; ++j) a[j] = ca * a[j] + cb * b[j];
  out.store(i, a);
}

int caxpby(wd_ctx* c, double ar, double ai, const Field& x, double br, double bi, const Field& y,
           const Field& out) {
  if (x.fmt != y.fmt || x.fmt != out.fmt) return fail(WD_ERR_ARG, "caxpby: formats differ");
  const long n = c->g.Vh;
  return with_fmt(x, [&](auto X) {
    using F = decltype(X);
    using T = typename Pick<F, F>::T;
    F Y = X, O = X;
    if constexpr (std::is_same<F, SpF64>::value) { Y = sp64(y); O = sp64(out); }
    else if constexpr (std::is_same<F, SpF32>::value) { Y = sp32(y); O = sp32(out); }
    else if constexpr (std::is_same<F, SpDD>::value) { Y = spdd(y); O = spdd(out); }
    else { Y = F{(uint4*)y.data, y.norm, y.stride}; O = F{(uint4*)out.data, out.norm, out.stride}; }
    k_caxpby<T><<<nblocks(n, BL_THREADS), BL_THREADS, 0, c->stream>>>(n, (T)ar, (T)ai, X, (T)br, (T)bi, Y, O);
    WD_CHECK_LAUNCH();
    return (int)WD_OK;
  });
}

int axpby(wd_ctx* c, double a, const Field& x, double b, const Field& y, const Field& out) {
  return caxpby(c, a, 0.0, x, b, 0.0, y, out);
}

int zero(wd_ctx* c, const Field& f) {
  WD_CUDA(cudaMemsetAsync(f.data, 0, field_bytes(f.fmt, c->g.Vh), c->stream));
  if (f.norm) WD_CUDA(cudaMemsetAsync(f.norm, 0, sizeof(float) * c->g.Vh, c->stream));
  return WD_OK;
}

template <class T, class F>
__global__ void k_gamma5(long n, F in, F out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cpx<T> s[12];
  in.loadT(i, s);
#pragma unroll
  for (int j = 6; j < 12; ++j) s[j] = mk<T>(-s[j].r, -s[j].i);
  out.store(i, s);
}

int gamma5(wd_ctx* c, const Field& in, const Field& out) {
  if (in.fmt != WD_F64 || out.fmt != WD_F64) return fail(WD_ERR_ARG, "gamma5: FP64 only");
  const long n = c->g.Vh;
  k_gamma5<double><<<nblocks(n, BL_THREADS), BL_THREADS, 0, c->stream>>>(n, sp64(in), sp64(out));
  WD_CHECK_LAUNCH();
  return WD_OK;
}

// ---------------------------------------------------------------------------
// inner products
template <class T, class A, class B>
__global__ void __launch_bounds__(BL_THREADS) k_dot(long n, A a, B b, Reduce red) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (i < n) {
    cpx<T> x[12], y[12];
    a.loadT(i, x);
    b.loadT(i, y);
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      cpx<T> p = cmulc(x[j], y[j]);
      v[0] += (double)p.r;
      v[1] += (double)p.i;
    }
  }
  double tot[2];
  grid_sum<2>(red, v, tot);
}

static int fetch_host(wd_ctx* c, int nv, double* out) {
  WD_CUDA(cudaMemcpyAsync(c->host_scalar, c->red_out, sizeof(double) * nv, cudaMemcpyDeviceToHost,
                          c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < nv; ++k) out[k] = c->host_scalar[k];
  return WD_OK;
}

int dot(wd_ctx* c, const Field& a, const Field& b, double* re, double* im) {
  const long n = c->g.Vh;
  const int nb = nblocks(n, BL_THREADS);
  if (nb > RED_MAX_BLOCKS) return fail(WD_ERR_ARG, "dot: lattice too large");
  int s = with_fmt(a, [&](auto A) {
    return with_fmt(b, [&](auto B) {
      using T = typename Pick<decltype(A), decltype(B)>::T;
      k_dot<T><<<nb, BL_THREADS, 0, c->stream>>>(n, A, B, reducer(c));
      WD_CHECK_LAUNCH();
      return (int)WD_OK;
    });
  });
  if (s != WD_OK) return s;
  double v[2];
  WD_TRY(fetch_host(c, 2, v));
  if (re) *re = v[0];
  if (im) *im = v[1];
  return WD_OK;
}

int norm2(wd_ctx* c, const Field& a, double* out) { return dot(c, a, a, out, nullptr); }

// ---------------------------------------------------------------------------
// CG: x += alpha p; r -= alpha Ap; rr = |r|^2 and the scalar logic in the
// last block (beta, stop and reliable-update flags).
template <class T, class X, class P, class R, class A>
__global__ void __launch_bounds__(BL_THREADS) k_cg_update(long n, X x, P p, R r, A ap, CGState* st,
                                                          Reduce red) {
  if (st->flag != 0) return;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (i < n) {
    const T al = (T)st->alpha;
    cpx<T> xv[12], pv[12], rv[12], av[12];
    x.loadT(i, xv);
    p.loadT(i, pv);
    r.loadT(i, rv);
    ap.loadT(i, av);
    T acc = 0;
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      xv[j] = xv[j] + al * pv[j];
      rv[j] = rv[j] - al * av[j];
      acc += norm2(rv[j]);
    }
    v[0] = (double)acc;
    x.store(i, xv);
    r.store(i, rv);
  }
  double tot[1];
  if (grid_sum<1>(red, v, tot)) {
    const double rr = tot[0];
    if (!isfinite(rr)) { st->flag |= FLAG_NAN; return; }
    st->rr_old = st->rr;
    st->beta = rr / st->rr;
    st->rr = rr;
    st->iter += 1;
    if (rr <= st->upd_rr) st->flag |= FLAG_UPDATE;
    if (st->iter >= st->maxiter) st->flag |= FLAG_MAXITER;
  }
}

template <class T, class R, class P>
__global__ void k_cg_pupdate(long n, R r, P p, CGState* st) {
  if (st->flag != 0) return;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T be = (T)st->beta;
  cpx<T> rv[12], pv[12];
  r.loadT(i, rv);
  p.loadT(i, pv);
#pragma unroll
  for (int j = 0; j < 12; ++j) pv[j] = rv[j] + be * pv[j];
  p.store(i, pv);
}

template <class T, class P, class A>
__global__ void __launch_bounds__(BL_THREADS) k_cg_dot_pap(long n, P p, A ap, CGState* st, Reduce red) {
  if (st->flag != 0) return;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (i < n) {
    cpx<T> pv[12], av[12];
    p.loadT(i, pv);
    ap.loadT(i, av);
    T acc = 0;
#pragma unroll
    for (int j = 0; j < 12; ++j) acc += pv[j].r * av[j].r + pv[j].i * av[j].i;
    v[0] = (double)acc;
  }
  double tot[1];
  if (grid_sum<1>(red, v, tot)) {
    st->pAp = tot[0];
    if (!(tot[0] > 0.0) || !isfinite(tot[0])) st->flag |= FLAG_NAN;
    else st->alpha = st->rr / tot[0];
  }
}

int cg_update(wd_ctx* c, const Field& x, const Field& r, const Field& p, const Field& Ap) {
  const long n = c->g.Vh;
  const int nb = nblocks(n, BL_THREADS);
  if (x.fmt != r.fmt || x.fmt != Ap.fmt || (x.fmt != WD_F64 && x.fmt != WD_F32))
    return fail(WD_ERR_ARG, "cg_update: x, r, Ap must share FP64 or FP32");
  return with_fmt(p, [&](auto P) {
    if (x.fmt == WD_F64) {
      using T = typename Pick<SpF64, decltype(P)>::T;
      k_cg_update<T><<<nb, BL_THREADS, 0, c->stream>>>(n, sp64(x), P, sp64(r), sp64(Ap), c->cgs, reducer(c));
    } else {
      k_cg_update<float><<<nb, BL_THREADS, 0, c->stream>>>(n, sp32(x), P, sp32(r), sp32(Ap), c->cgs, reducer(c));
    }
    WD_CHECK_LAUNCH();
    return (int)WD_OK;
  });
}

int cg_pupdate(wd_ctx* c, const Field& r, const Field& p) {
  const long n = c->g.Vh;
  const int nb = nblocks(n, BL_THREADS);
  return with_fmt(p, [&](auto P) {
    if (r.fmt == WD_F64) {
      using T = typename Pick<SpF64, decltype(P)>::T;
      k_cg_pupdate<T><<<nb, BL_THREADS, 0, c->stream>>>(n, sp64(r), P, c->cgs);
    } else if (r.fmt == WD_F32) {
      k_cg_pupdate<float><<<nb, BL_THREADS, 0, c->stream>>>(n, sp32(r), P, c->cgs);
    } else {
      return fail(WD_ERR_ARG, "cg_pupdate: r must be FP64 or FP32");
    }
    WD_CHECK_LAUNCH();
    return (int)WD_OK;
  });
}

int cg_dot_pap(wd_ctx* c, const Field& p, const Field& Ap) {
  const long n = c->g.Vh;
  const int nb = nblocks(n, BL_THREADS);
  return with_fmt(p, [&](auto P) {
    return with_fmt(Ap, [&](auto A) {
      using T = typename Pick<decltype(P), decltype(A)>::T;
      k_cg_dot_pap<T><<<nb, BL_THREADS, 0, c->stream>>>(n, P, A, c->cgs, reducer(c));
      WD_CHECK_LAUNCH();
      return (int)WD_OK;
    });
  });
}

// ---------------------------------------------------------------------------
// Chebyshev recurrence step: out = a (v + mu s - Ks) - b sprev
template <class T, class F>
__global__ void k_poly_step(long n, T a, T mu, T b, F v, F s, F ks, F sp, F out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cpx<T> vv[12], sv[12], kv[12], pv[12];
  v.loadT(i, vv);
  s.loadT(i, sv);
  ks.loadT(i, kv);
  sp.loadT(i, pv);
#pragma unroll
  for (int j = 0; j < 12; ++j) vv[j] = a * (vv[j] + mu * sv[j] - kv[j]) - b * pv[j];
  out.store(i, vv);
}

int poly_step(wd_ctx* c, double a, double mu, double b, const Field& v, const Field& s,
              const Field& Ks, const Field& sprev, const Field& out) {
  const long n = c->g.Vh;
  const int nb = nblocks(n, BL_THREADS);
  if (v.fmt == WD_F64) {
    k_poly_step<double><<<nb, BL_THREADS, 0, c->stream>>>(n, a, mu, b, sp64(v), sp64(s), sp64(Ks),
                                                          sp64(sprev), sp64(out));
  } else if (v.fmt == WD_F32) {
    k_poly_step<float><<<nb, BL_THREADS, 0, c->stream>>>(n, (float)a, (float)mu, (float)b, sp32(v), sp32(s),
                                                         sp32(Ks), sp32(sprev), sp32(out));
  } else if (v.fmt == WD_DD) {
    k_poly_step<dd><<<nb, BL_THREADS, 0, c->stream>>>(n, dd(a), dd(mu), dd(b), spdd(v), spdd(s), spdd(Ks),
                                                      spdd(sprev), spdd(out));
  } else {
    return fail(WD_ERR_ARG, "poly_step: FP64, FP32 or double-float fields only");
  }
  WD_CHECK_LAUNCH();
  return WD_OK;
}

}  // namespace wd
