// FP32 instantiations of the hopping stencil (float storage and arithmetic,
// FP32 links with 18 or 12 stored reals).
#include "dslash_impl.cuh"

namespace wd {

// ----------------------------------------------------------------------------
// Staged FP32 stencil with 12-real links.  The plain kernel holds a direction's
// neighbour loads in registers, so at 88 registers (five 128-thread blocks per
// SM) too few bytes are in flight to keep HBM busy (ncu: long-scoreboard stalls
// dominate, DRAM about 70 % active).  Here every thread runs its own software
// pipeline over the eight neighbour directions: the three float4 of the link
// (and, with SPIN, the six float4 of the neighbour spinor) of direction D + NST
// are copied global -> shared with cp.async while direction D is computed, so
// NST directions are in flight without holding registers.  A thread reads only
// the shared words it copied itself, so no block barrier is needed; NST + 1
// buffers make the buffer being refilled one whose values were consumed in the
// previous step.  Links are copied with .cg (read once per hop), spinors with
// .ca (each is read by eight sites).
__device__ __forceinline__ void cpa16(float4* sdst, const float4* gsrc, bool cache_l1) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  if (cache_l1) asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
  else asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int NST, bool SPIN, bool DAG>
struct Staged {
  static constexpr int NB = NST + 1;          // buffers
  static constexpr int K = SPIN ? 9 : 3;      // float4 per direction and thread
  const HopArgs<SpF32, SpF32, SpF32, GF32R12>& a;
  long cb;
  int c[4];
  float4* buf;                                // [NB][K][blockDim.x]
  int tid, nt;

  __device__ __forceinline__ float4* slot(int b, int k) const { return buf + (b * K + k) * nt + tid; }

  template <int D> __device__ __forceinline__ long nbr() const {
    constexpr int MU = D >> 1;
    int n[4] = {c[0], c[1], c[2], c[3]};
    if constexpr ((D & 1) == 0) n[MU] = (n[MU] + 1 == a.g.L[MU]) ? 0 : n[MU] + 1;
    else n[MU] = (n[MU] == 0) ? a.g.L[MU] - 1 : n[MU] - 1;
    return a.g.cb_of(n[0], n[1], n[2], n[3]);
  }

  template <int D> __device__ __forceinline__ void issue() const {
    if constexpr (D < 8) {
      constexpr int MU = D >> 1;
      constexpr int B = D % NB;
      const long nb = nbr<D>();
      const int lpar = (D & 1) == 0 ? a.out_par : 1 - a.out_par;
      const long li = (D & 1) == 0 ? cb : nb;
      const float4* q = a.gauge.p + ((long)(MU * 2 + lpar) * 3) * a.gauge.stride + li;
#pragma unroll
      for (int j = 0; j < 3; ++j) cpa16(slot(B, (SPIN ? 6 : 0) + j), q + j * a.gauge.stride, false);
      if constexpr (SPIN) {
#pragma unroll
        for (int j = 0; j < 6; ++j) cpa16(slot(B, j), a.in.p + j * a.in.stride + nb, true);
      }
    }
    cpa_commit();                              // possibly empty: keeps one group per step
  }

  template <int D> __device__ __forceinline__ void step(cpx<float> (&acc)[12]) const {
    constexpr int MU = D >> 1;
    constexpr bool FWD = (D & 1) == 0;
    constexpr int B = D % NB;
    cpa_wait<NST - 1>();                       // direction D has landed
    cpx<float> s[12], U[9], h[6], u[6];
    if constexpr (SPIN) {
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const float4 v = *slot(B, j);
        s[2 * j] = {v.x, v.y};
        s[2 * j + 1] = {v.z, v.w};
      }
    } else {
      a.in.loadT(nbr<D>(), s);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float4 v = *slot(B, (SPIN ? 6 : 0) + j);
      U[2 * j] = {v.x, v.y};
      U[2 * j + 1] = {v.z, v.w};
    }
    issue<D + NST>();                          // refills the buffer of direction D - 1
    U[6] = conj(U[1] * U[5] - U[2] * U[4]);
    U[7] = conj(U[2] * U[3] - U[0] * U[5]);
    U[8] = conj(U[0] * U[4] - U[1] * U[3]);
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SG = FWD ? SF : -SF;
    spin_project<MU, SG>(s, h);
    if (MU == 3 && (FWD ? c[3] == a.g.L[3] - 1 : c[3] == 0)) {
#pragma unroll
      for (int j = 0; j < 6; ++j) h[j] = mk<float>(-h[j].r, -h[j].i);
    }
    if constexpr (FWD) su3_mul(U, h, u);
    else su3_dag_mul(U, h, u);
    spin_accum<MU, SG>(acc, u);
  }

  // directions 0 .. NST - 1 go out before the first step
  template <int D> __device__ __forceinline__ void prologue() const {
    if constexpr (D < NST) {
      issue<D>();
      prologue<D + 1>();
    }
  }

  __device__ __forceinline__ void run(cpx<float> (&acc)[12]) const {
    static_assert(NST >= 1 && NST <= 7, "one to seven directions in flight");
    prologue<0>();
    step<0>(acc);
    step<1>(acc);
    step<2>(acc);
    step<3>(acc);
    step<4>(acc);
    step<5>(acc);
    step<6>(acc);
    step<7>(acc);
  }
};

template <int NST, bool SPIN, bool DAG, bool XPAY, bool NORM>
__global__ void __launch_bounds__(128, 5) k_hop_st(HopArgs<SpF32, SpF32, SpF32, GF32R12> a) {
  extern __shared__ float4 sbuf[];
  if (a.st != nullptr && a.st->flag != 0) return;
  const long cb = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double part[1] = {0.0};
  if (cb < a.g.Vh) {
    Staged<NST, SPIN, DAG> S{a, cb, {0, 0, 0, 0}, sbuf, (int)threadIdx.x, (int)blockDim.x};
    a.g.coords(cb, a.out_par, S.c);
    cpx<float> acc[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) acc[j] = mk<float>(0, 0);
    S.run(acc);
    if constexpr (XPAY) {
      cpx<float> yv[12];
      a.y.loadT(cb, yv);
      const float al = (float)a.alpha;
#pragma unroll
      for (int j = 0; j < 12; ++j) acc[j] = yv[j] + al * acc[j];
    }
    if constexpr (NORM) {
#pragma unroll
      for (int j = 0; j < 12; ++j) {
        const double re = (double)acc[j].r, im = (double)acc[j].i;
        part[0] += re * re + im * im;
      }
    }
    a.out.store(cb, acc);
  }
  if constexpr (NORM) {
    double tot[1];
    if (grid_sum<1>(a.red, part, tot)) {
      CGState* st = a.st;
      if (st != nullptr) {
        st->pAp = tot[0];
        if (!(tot[0] > 0.0) || !isfinite(tot[0])) st->flag |= FLAG_NAN;
        else st->alpha = st->rr / tot[0];
      }
    }
  }
}

// staging depth and whether spinors are staged too (links always are); NST = 0
// selects the register-only kernel
constexpr int HOP_STAGES = 2;
constexpr bool HOP_STAGE_SPINOR = false;

constexpr int HOP_NST = HOP_STAGES > 0 ? HOP_STAGES : 1;
constexpr size_t HOP_STAGE_SMEM = (size_t)(HOP_NST + 1) * (HOP_STAGE_SPINOR ? 9 : 3) * 128 * sizeof(float4);

template <bool DAG, bool XPAY, bool NORM>
static void launch_st(wd_ctx* c, const HopArgs<SpF32, SpF32, SpF32, GF32R12>& a) {
  k_hop_st<HOP_NST, HOP_STAGE_SPINOR, DAG, XPAY, NORM>
      <<<nblocks(c->g.Vh, 128), 128, HOP_STAGE_SMEM, c->stream>>>(a);
}

static int hop_f32_staged(wd_ctx* c, int out_par, bool dag, const SpF32& I, const SpF32& O, const SpF32& Y,
                          bool xpay, double alpha, bool norm_cg, bool in_cg) {
  if (norm_cg && nblocks(c->g.Vh, 64) > RED_MAX_BLOCKS) return fail(WD_ERR_ARG, "lattice too large for one reduction grid");
  if (norm_cg && (dag || !xpay)) return fail(WD_ERR_ARG, "hop: the |out|^2 epilogue exists for M_hat only");
  CGState* st = (norm_cg || in_cg) ? c->cgs : nullptr;
  HopArgs<SpF32, SpF32, SpF32, GF32R12> a{c->g, out_par, I, O, Y, GF32R12{c->gauge32r12, c->g.Vh}, alpha,
                                          reducer(c), st};
  if (!dag) {
    if (!xpay) launch_st<false, false, false>(c, a);
    else if (!norm_cg) launch_st<false, true, false>(c, a);
    else launch_st<false, true, true>(c, a);
  } else {
    if (!xpay) launch_st<true, false, false>(c, a);
    else launch_st<true, true, false>(c, a);
  }
  WD_CHECK_LAUNCH();
  return WD_OK;
}

int hop_f32(wd_ctx* c, int out_par, bool dag, const Field& in, const Field& out, const Field* y,
            double alpha, bool norm_cg, bool in_cg) {
  if (in.fmt != WD_F32 || out.fmt != WD_F32 || (y && y->fmt != WD_F32))
    return fail(WD_ERR_ARG, "hop_f32: field formats must all be FP32");
  SpF32 I = sp32(in), O = sp32(out), Y = y ? sp32(*y) : O;
  if (HOP_STAGES > 0 && c->recon == WD_RECON_12)
    return hop_f32_staged(c, out_par, dag, I, O, Y, y != nullptr, alpha, norm_cg, in_cg);
  return hop_with_gauge<float>(c, out_par, dag, I, O, Y, y != nullptr, alpha, norm_cg, in_cg, false);
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
__global__ void __launch_bounds__(128, 5) k_hop_poly_st(HopArgs<SpF32, SpF32, SpF32, GF32R12> a, SpF32 v, SpF32 s,
                                                     SpF32 sp, float ca, float cmu, float cb) {
  extern __shared__ float4 sbuf[];
  const long cb_ = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cb_ >= a.g.Vh) return;
  Staged<HOP_NST, HOP_STAGE_SPINOR, true> S{a, cb_, {0, 0, 0, 0}, sbuf, (int)threadIdx.x, (int)blockDim.x};
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
  if (c->recon == WD_RECON_12) {
    HopArgs<SpF32, SpF32, SpF32, GF32R12> a{c->g, 0, sp32(t1), sp32(out), sp32(t2), GF32R12{c->gauge32r12, c->g.Vh},
                                            a2, reducer(c), nullptr};
    if (HOP_STAGES > 0)
      k_hop_poly_st<<<nb, 128, HOP_STAGE_SMEM, c->stream>>>(a, sp32(v), sp32(s), sp32(sprev), (float)ca, (float)cmu,
                                                           (float)cb);
    else
      k_hop_poly<<<nb, 128, 0, c->stream>>>(a, sp32(v), sp32(s), sp32(sprev), (float)ca, (float)cmu, (float)cb);
  } else {
    HopArgs<SpF32, SpF32, SpF32, GF32> a{c->g, 0, sp32(t1), sp32(out), sp32(t2), GF32{c->gauge32, c->g.Vh}, a2,
                                         reducer(c), nullptr};
    k_hop_poly<<<nb, 128, 0, c->stream>>>(a, sp32(v), sp32(s), sp32(sprev), (float)ca, (float)cmu, (float)cb);
  }
  WD_CHECK_LAUNCH();
  c->prof.all[WD_F32] += 1;
  c->nmat += 1;
  return WD_OK;
}

}  // namespace wd
