// FP32 instantiations of the hopping stencil (float storage and arithmetic,
// FP32 links with 18 or 12 stored reals).
#include "dslash_tt.cuh"

namespace wd {

int hop_f32(wd_ctx* c, int out_par, bool dag, const Field& in, const Field& out, const Field* y,
            double alpha, bool norm_cg, bool in_cg) {
  if (in.fmt != WD_F32 || out.fmt != WD_F32 || (y && y->fmt != WD_F32))
    return fail(WD_ERR_ARG, "hop_f32: field formats must all be FP32");
  SpF32 I = sp32(in), O = sp32(out), Y = y ? sp32(*y) : O;
  if (c->recon == WD_RECON_12) {
    if (tt_eligible(c)) return hop_tt(c, out_par, dag, I, O, Y, y != nullptr, alpha, norm_cg, in_cg);
    return hop_staged(c, out_par, dag, I, O, Y, y != nullptr, alpha, norm_cg, in_cg);
  }
  return hop_with_gauge<float>(c, out_par, dag, I, O, Y, y != nullptr, alpha, norm_cg, in_cg, false);
}

// Self-test of the bounded barrier wait: thread 0 waits on a freshly
// initialised mbarrier that nothing arrives at; the wait expires after ns and
// the kernel records it in the device error word and returns.
__global__ void k_wait_selftest(unsigned* kerr, long long ns) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_ns(&bar, 0u, ns)) atomicOr(kerr, 1u);
}

int wait_selftest(wd_ctx* c, long long ns) {
  if (c->kerr == nullptr) return fail(WD_ERR_STATE, "no device error word");
  k_wait_selftest<<<1, 32, 0, c->stream>>>(c->kerr, ns);
  WD_CHECK_LAUNCH();
  return WD_OK;
}

// Last hop of K_hat fused with the Chebyshev recurrence step (FP32):
//   Ks = y + alpha D^dag_eo x  (y = M_hat s, x = D^dag_oe y),
//   out = ca (v + cmu s - Ks) - cb sprev.
// Saves the K s vector and the separate 5-vector pass of the step kernel.
template <class G>
__global__ void __launch_bounds__(128) k_hop_poly(HopArgs<SpF32, SpF32, SpF32, G> a, SpF32 v, SpF32 s, SpF32 sp,
                                                  float ca, float cmu, float cb) {
  const long cb_ = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cb_ >= a.g.Vh) return;
  int c[4];
  a.g.coords(cb_, 0, c);
  cpx<float> acc[12];
#pragma unroll
  for (int j = 0; j < 12; ++j) acc[j] = mk<float>(0, 0);
  hop_dir<0, true>(a.g, 0, cb_, c, a.in, a.gauge, acc);
  hop_dir<1, true>(a.g, 0, cb_, c, a.in, a.gauge, acc);
  hop_dir<2, true>(a.g, 0, cb_, c, a.in, a.gauge, acc);
  hop_dir<3, true>(a.g, 0, cb_, c, a.in, a.gauge, acc);
  cpx<float> yv[12], q[12];
  a.y.loadT(cb_, yv);
  const float al = (float)a.alpha;
#pragma unroll
  for (int j = 0; j < 12; ++j) acc[j] = yv[j] + al * acc[j];   // K s
  v.loadT(cb_, yv);
  s.loadT(cb_, q);
#pragma unroll
  for (int j = 0; j < 12; ++j) yv[j] = yv[j] + cmu * q[j] - acc[j];
  sp.loadT(cb_, q);
#pragma unroll
  for (int j = 0; j < 12; ++j) yv[j] = ca * yv[j] - cb * q[j];
  a.out.store(cb_, yv);
}

// the same with the staged neighbour loads (12-real links)
__global__ void __launch_bounds__(HOP_ST_THREADS, HOP_MINB) k_hop_poly_st(HopArgs<SpF32, SpF32, SpF32, GF32R12> a, SpF32 v, SpF32 s,
                                                     SpF32 sp, float ca, float cmu, float cb) {
  extern __shared__ float4 sbuf[];
  const long cb_ = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cb_ >= a.g.Vh) return;
  Staged<HOP_NST, true, HopArgs<SpF32, SpF32, SpF32, GF32R12>> S{a, cb_, {0, 0, 0, 0}, sbuf, (int)threadIdx.x,
                                                                  (int)blockDim.x};
  a.g.coords(cb_, 0, S.c);
  cpx<float> acc[12];
#pragma unroll
  for (int j = 0; j < 12; ++j) acc[j] = mk<float>(0, 0);
  S.run(acc);
  cpx<float> yv[12], q[12];
  a.y.loadT(cb_, yv);
  const float al = (float)a.alpha;
#pragma unroll
  for (int j = 0; j < 12; ++j) acc[j] = yv[j] + al * acc[j];   // K s
  v.loadT(cb_, yv);
  s.loadT(cb_, q);
#pragma unroll
  for (int j = 0; j < 12; ++j) yv[j] = yv[j] + cmu * q[j] - acc[j];
  sp.loadT(cb_, q);
#pragma unroll
  for (int j = 0; j < 12; ++j) yv[j] = ca * yv[j] - cb * q[j];
  a.out.store(cb_, yv);
}

// out = ca (v + cmu s - K_hat s) - cb sprev for FP32 fields (t1, t2 scratch)
int khat_poly_step_f32(wd_ctx* c, double kappa, const Field& s, Field& t1, Field& t2, const Field& v,
                       const Field& sprev, double ca, double cmu, double cb, const Field& out) {
  const Field* fields[] = {&s, &t1, &t2, &v, &sprev, &out};
  for (const Field* f : fields)
    if (f->fmt != WD_F32) return fail(WD_ERR_ARG, "khat_poly_step_f32: FP32 fields only");
  const double a2 = -kappa * kappa;
  WD_TRY(hop(c, 1, false, s, t1, nullptr, 0.0, false, false));
  WD_TRY(hop(c, 0, false, t1, t2, &s, a2, false, false));
  WD_TRY(hop(c, 1, true, t2, t1, nullptr, 0.0, false, false));
  const int nb = nblocks(c->g.Vh, 128);
  if (c->recon == WD_RECON_12 && tt_eligible(c)) {
    HopArgs<SpF32, SpF32, SpF32, GF32R12> a{c->g, 0, sp32(t1), sp32(out), sp32(t2), GF32R12{c->gauge32r12, c->g.Vh},
                                            a2, reducer(c), nullptr};
    const TTPoly pe{sp32(v), sp32(s), sp32(sprev), (float)ca, (float)cmu, (float)cb};
    const Field* chk[] = {&t1, &t2, &v, &s, &sprev};
    for (const Field* f : chk)
      if (((uintptr_t)f->data & 15) != 0) return fail(WD_ERR_ARG, "khat_poly_step_f32: fields must be 16-byte aligned");
    WD_TRY((tt_launch<true, 2, false>(c, a, pe)));
  } else if (c->recon == WD_RECON_12) {
    HopArgs<SpF32, SpF32, SpF32, GF32R12> a{c->g, 0, sp32(t1), sp32(out), sp32(t2), GF32R12{c->gauge32r12, c->g.Vh},
                                            a2, reducer(c), nullptr};
    k_hop_poly_st<<<nb, HOP_ST_THREADS, HOP_STAGE_SMEM, c->stream>>>(a, sp32(v), sp32(s), sp32(sprev), (float)ca,
                                                                      (float)cmu, (float)cb);
    WD_CHECK_LAUNCH();
  } else {
    HopArgs<SpF32, SpF32, SpF32, GF32> a{c->g, 0, sp32(t1), sp32(out), sp32(t2), GF32{c->gauge32, c->g.Vh}, a2,
                                         reducer(c), nullptr};
    k_hop_poly<<<nb, 128, 0, c->stream>>>(a, sp32(v), sp32(s), sp32(sprev), (float)ca, (float)cmu, (float)cb);
    WD_CHECK_LAUNCH();
  }
  c->prof.all[WD_F32] += 1;
  c->nmat += 1;
  return WD_OK;
}

}  // namespace wd
