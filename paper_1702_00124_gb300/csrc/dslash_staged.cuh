// Staged hopping stencil for 12-real FP32 links (Section 3.1 of the paper:
// Wilson fermions, even-odd preconditioning), any spinor storage format.
//
// The register-only kernel holds a direction's neighbour loads in registers,
// so at the register count that allows five 128-thread blocks per SM too few
// bytes are in flight to keep HBM busy (long-scoreboard stalls dominate).
// Here every thread runs its own software pipeline over the eight neighbour
// directions: the three float4 of the link of direction D + NST are copied
// global -> shared with cp.async.cg while direction D is computed, so NST
// directions' links are in flight without holding registers.  A thread reads
// only the shared words it copied itself, so no block barrier is needed; NST + 1
// buffers make the buffer being refilled one whose values were consumed in the
// previous step.  Neighbour spinors are read through L1 (each is read by eight
// sites, several of them in the same block).
#pragma once
#include "dslash_impl.cuh"

namespace wd {

#ifndef WD_HOP_STAGES
#define WD_HOP_STAGES 2
#endif
#ifndef WD_HOP_SPIN_AHEAD
#define WD_HOP_SPIN_AHEAD 1
#endif
// resident 128-thread blocks per SM the register budget is set for: FP32
// spinors five (96 registers), 16-bit spinors six (80 registers; their words
// take half the registers).  Measured per hop at 32^3 x 64 in the K_hat chain:
// FP32 0.1112 ms (five, with the look-ahead below) against 0.1163 (six) and
// 0.1283 (seven); BF16 0.1070 ms (six) against 0.1104 (five).
#ifndef WD_HOP_MINB_F32
#define WD_HOP_MINB_F32 5
#endif
#ifndef WD_HOP_MINB_16
#define WD_HOP_MINB_16 6
#endif
// L2 prefetch size of the stencil's global reads: 0 none, 1 the link copies
// fetch 256-byte L2 lines, 2 the neighbour spinor reads as well
#ifndef WD_HOP_L2_256
#define WD_HOP_L2_256 0
#endif
constexpr int HOP_NST = WD_HOP_STAGES;                 // link directions in flight
// neighbour spinor of direction D + 1 loaded into registers while D is computed:
// 0 never, 1 for FP32 spinors (0.1133 -> 0.1112 ms per hop; 16-bit spinors gain
// nothing), 2 for every format
template <class In> constexpr bool spin_ahead() {
  return WD_HOP_SPIN_AHEAD >= 2 || (WD_HOP_SPIN_AHEAD == 1 && std::is_same<In, SpF32>::value);
}
template <class In> constexpr int hop_minb() {
  return std::is_same<In, SpF32>::value ? WD_HOP_MINB_F32 : WD_HOP_MINB_16;
}
constexpr int HOP_MINB = WD_HOP_MINB_F32;              // FP32 kernels outside the template
static_assert(HOP_NST >= 1 && HOP_NST <= 7, "one to seven directions in flight");
constexpr int HOP_ST_THREADS = 128;
constexpr size_t HOP_STAGE_SMEM = (size_t)(HOP_NST + 1) * 3 * HOP_ST_THREADS * sizeof(float4);

__device__ __forceinline__ void cpa16(float4* sdst, const float4* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
#if WD_HOP_L2_256 >= 1
  asm volatile("cp.async.cg.shared.global.L2::256B [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
#else
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
#endif
}

// read-only 16-byte load with the L2 prefetch size of WD_HOP_L2_256 >= 2
__device__ __forceinline__ float4 ldg_stencil(const float4* p) {
#if WD_HOP_L2_256 >= 2
  float4 v;
  asm volatile("ld.global.nc.L2::256B.v4.f32 {%0, %1, %2, %3}, [%4];\n"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
#else
  return __ldg(p);
#endif
}

// neighbour spinor of the staged stencil: FP32 through ldg_stencil, other
// formats through their own loader
template <class S> __device__ __forceinline__ void load_nbr(const S& in, long i, cpx<float> (&s)[12]) {
  in.loadT(i, s);
}
template <> __device__ __forceinline__ void load_nbr<SpF32>(const SpF32& in, long i, cpx<float> (&s)[12]) {
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const float4 v = ldg_stencil(in.p + j * in.stride + i);
    s[2 * j] = {v.x, v.y};
    s[2 * j + 1] = {v.z, v.w};
  }
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int NST, bool DAG, class A>
struct Staged {
  static constexpr int NB = NST + 1;          // buffers
  const A& a;
  long cb;
  int c[4];
  float4* buf;                                // [NB][3][blockDim.x]
  int tid, nt;

  __device__ __forceinline__ float4* slot(int b, int k) const { return buf + (b * 3 + k) * nt + tid; }

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
      const int lpar = (D & 1) == 0 ? a.out_par : 1 - a.out_par;
      const long li = (D & 1) == 0 ? cb : nbr<D>();
      const float4* q = a.gauge.p + ((long)(MU * 2 + lpar) * 3) * a.gauge.stride + li;
#pragma unroll
      for (int j = 0; j < 3; ++j) cpa16(slot(D % NB, j), q + j * a.gauge.stride);
    }
    cpa_commit();                              // possibly empty: keeps one group per step
  }

  template <int D> __device__ __forceinline__ void step(cpx<float> (&acc)[12]) const {
    cpx<float> s[12];
    load_nbr(a.in, nbr<D>(), s);
    compute<D>(acc, s);
  }

  // the same with the spinor of this direction loaded one step earlier (cur) and
  // the next direction's issued now (nxt)
  template <int D, class R> __device__ __forceinline__ void step_ahead(cpx<float> (&acc)[12], const R& cur,
                                                                       R& nxt) const {
    if constexpr (D + 1 < 8) a.in.loadRaw(nbr<D + 1>(), nxt);
    cpx<float> s[12];
    a.in.unpack(cur, s);
    compute<D>(acc, s);
  }

  template <int D> __device__ __forceinline__ void compute(cpx<float> (&acc)[12], const cpx<float> (&s)[12]) const {
    constexpr int MU = D >> 1;
    constexpr bool FWD = (D & 1) == 0;
    cpa_wait<NST - 1>();                       // direction D has landed
    cpx<float> U[9], h[6], u[6];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float4 v = *slot(D % NB, j);
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
    prologue<0>();
    using In = typename std::remove_cv<decltype(a.in)>::type;
    if constexpr (spin_ahead<In>()) {
      typename In::Raw r0, r1;
      a.in.loadRaw(nbr<0>(), r0);
      step_ahead<0>(acc, r0, r1);
      step_ahead<1>(acc, r1, r0);
      step_ahead<2>(acc, r0, r1);
      step_ahead<3>(acc, r1, r0);
      step_ahead<4>(acc, r0, r1);
      step_ahead<5>(acc, r1, r0);
      step_ahead<6>(acc, r0, r1);
      step_ahead<7>(acc, r1, r0);
    } else {
      step<0>(acc);
      step<1>(acc);
      step<2>(acc);
      step<3>(acc);
      step<4>(acc);
      step<5>(acc);
      step<6>(acc);
      step<7>(acc);
    }
  }
};

template <bool DAG, bool XPAY, bool NORM, class In, class Out, class Y>
__global__ void __launch_bounds__(HOP_ST_THREADS, hop_minb<In>()) k_hop_st(HopArgs<In, Out, Y, GF32R12> a) {
  extern __shared__ float4 sbuf[];
  if (a.st != nullptr && a.st->flag != 0) return;
  const long cb = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double part[1] = {0.0};
  if (cb < a.g.Vh) {
    Staged<HOP_NST, DAG, HopArgs<In, Out, Y, GF32R12>> S{a, cb, {0, 0, 0, 0}, sbuf, (int)threadIdx.x,
                                                         (int)blockDim.x};
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
    if constexpr (NORM) part[0] = site_norm2(acc);
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

// Launch of the staged stencil for the context's 12-real FP32 links.
template <class In, class Out, class Y>
int hop_staged(wd_ctx* c, int out_par, bool dag, const In& I, const Out& O, const Y& Yv, bool xpay, double alpha,
               bool norm_cg, bool in_cg) {
  if (norm_cg && nblocks(c->g.Vh, 64) > RED_MAX_BLOCKS) return fail(WD_ERR_ARG, "lattice too large for one reduction grid");
  if (norm_cg && (dag || !xpay)) return fail(WD_ERR_ARG, "hop: the |out|^2 epilogue exists for M_hat only");
  CGState* st = (norm_cg || in_cg) ? c->cgs : nullptr;
  HopArgs<In, Out, Y, GF32R12> a{c->g, out_par, I, O, Yv, GF32R12{c->gauge32r12, c->g.Vh}, alpha, reducer(c), st};
  const int nb = nblocks(c->g.Vh, HOP_ST_THREADS);
  if (!dag) {
    if (!xpay) k_hop_st<false, false, false><<<nb, HOP_ST_THREADS, HOP_STAGE_SMEM, c->stream>>>(a);
    else if (!norm_cg) k_hop_st<false, true, false><<<nb, HOP_ST_THREADS, HOP_STAGE_SMEM, c->stream>>>(a);
    else k_hop_st<false, true, true><<<nb, HOP_ST_THREADS, HOP_STAGE_SMEM, c->stream>>>(a);
  } else {
    if (!xpay) k_hop_st<true, false, false><<<nb, HOP_ST_THREADS, HOP_STAGE_SMEM, c->stream>>>(a);
    else k_hop_st<true, true, false><<<nb, HOP_ST_THREADS, HOP_STAGE_SMEM, c->stream>>>(a);
  }
  WD_CHECK_LAUNCH();
  return WD_OK;
}

}  // namespace wd
