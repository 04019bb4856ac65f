// Wilson hopping stencil (Section 3.1 of the paper: Wilson fermions, even-odd
// preconditioning).  One thread per output site of one parity:
//   (D psi)(x) = sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ]
// (dagger: the signs of the two projectors swap), fermion sign -1 across the
// time boundary.  The spin projector reduces each neighbour to a half spinor
// (2 x 3 complex) before the SU(3) multiply, and the lower half of the result
// is rebuilt from the upper half.  Optional epilogue: out = y + alpha * D psi,
// with the FP64 grid sum of |out|^2 (pAp = |M_hat p|^2 for CG).
#pragma once
#include <algorithm>

#include "wd_internal.cuh"

namespace wd {

constexpr int HOP_THREADS = 128;   // default block size
constexpr int HOP_MAXT = 256;      // largest block size any launch uses

template <int MU, int SG, class T>
__device__ __forceinline__ void spin_project(const cpx<T> (&s)[12], cpx<T> (&h)[6]) {
  using Gm = Gam<MU>;
  constexpr int k0 = Gm::k0 + (SG > 0 ? 0 : 2);
  constexpr int k1 = Gm::k1 + (SG > 0 ? 0 : 2);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    h[c] = s[c] + ipow<k0>(s[3 * Gm::p0 + c]);
    h[3 + c] = s[3 + c] + ipow<k1>(s[3 * Gm::p1 + c]);
  }
}

template <int MU, int SG, class T>
__device__ __forceinline__ void spin_accum(cpx<T> (&acc)[12], const cpx<T> (&u)[6]) {
  using Gm = Gam<MU>;
  constexpr int q0 = (SG > 0 ? 0 : 2) - Gm::k0;
  constexpr int q1 = (SG > 0 ? 0 : 2) - Gm::k1;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c] = acc[c] + u[c];
    acc[3 + c] = acc[3 + c] + u[3 + c];
    acc[3 * Gm::p0 + c] = acc[3 * Gm::p0 + c] + ipow<q0>(u[c]);
    acc[3 * Gm::p1 + c] = acc[3 * Gm::p1 + c] + ipow<q1>(u[3 + c]);
  }
}

template <class T>
__device__ __forceinline__ void su3_mul(const cpx<T> (&U)[9], const cpx<T> (&h)[6], cpx<T> (&o)[6]) {
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      o[3 * a + c] = U[3 * c] * h[3 * a] + U[3 * c + 1] * h[3 * a + 1] + U[3 * c + 2] * h[3 * a + 2];
}

template <class T>
__device__ __forceinline__ void su3_dag_mul(const cpx<T> (&U)[9], const cpx<T> (&h)[6], cpx<T> (&o)[6]) {
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      o[3 * a + c] = cmulc(U[c], h[3 * a]) + cmulc(U[3 + c], h[3 * a + 1]) + cmulc(U[6 + c], h[3 * a + 2]);
}

// |s|^2 of one site for a grid sum, returned in FP64.  FP32 sites are summed
// in FP32 (24 terms, relative error ~1e-6): GB300 issues FP64 at 1/64 of the
// FP32 rate, and 24 FP64 FMAs per site cost as much as the stencil's loads.
template <class T> __device__ __forceinline__ double site_norm2(const cpx<T> (&s)[12]) {
  if constexpr (std::is_same<T, float>::value) {
    float q = 0.f;
#pragma unroll
    for (int j = 0; j < 12; ++j) q = fmaf(s[j].r, s[j].r, fmaf(s[j].i, s[j].i, q));
    return (double)q;
  } else {
    double q = 0.0;
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      const double re = (double)s[j].r, im = (double)s[j].i;
      q += re * re + im * im;
    }
    return q;
  }
}

template <class In, class Out, class Y, class G>
struct HopArgs {
  Geom g;
  int out_par;
  In in;
  Out out;
  Y y;
  G gauge;
  double alpha;
  Reduce red;
  CGState* st;
};

template <int MU, bool DAG, class T, class In, class G>
__device__ __forceinline__ void hop_dir(const Geom& g, int par, long cb, const int (&c)[4], const In& in,
                                        const G& gauge, cpx<T> (&acc)[12]) {
  constexpr int SF = DAG ? +1 : -1;   // forward projector 1 + SF g_mu
  constexpr int SB = -SF;             // backward projector
  // forward neighbour x + mu
  {
    int n[4] = {c[0], c[1], c[2], c[3]};
    n[MU] = (n[MU] + 1 == g.L[MU]) ? 0 : n[MU] + 1;
    const long nb = g.cb_of(n[0], n[1], n[2], n[3]);
    cpx<T> s[12], h[6], u[6], U[9];
    in.loadT(nb, s);
    gauge.load(MU, par, cb, U);
    spin_project<MU, SF>(s, h);
    if (MU == 3 && c[3] == g.L[3] - 1) {
#pragma unroll
      for (int j = 0; j < 6; ++j) h[j] = mk<T>(-h[j].r, -h[j].i);
    }
    su3_mul(U, h, u);
    spin_accum<MU, SF>(acc, u);
  }
  // backward neighbour x - mu, link U_mu(x - mu)^dag
  {
    int n[4] = {c[0], c[1], c[2], c[3]};
    n[MU] = (n[MU] == 0) ? g.L[MU] - 1 : n[MU] - 1;
    const long nb = g.cb_of(n[0], n[1], n[2], n[3]);
    cpx<T> s[12], h[6], u[6], U[9];
    in.loadT(nb, s);
    gauge.load(MU, 1 - par, nb, U);
    spin_project<MU, SB>(s, h);
    if (MU == 3 && c[3] == 0) {
#pragma unroll
      for (int j = 0; j < 6; ++j) h[j] = mk<T>(-h[j].r, -h[j].i);
    }
    su3_dag_mul(U, h, u);
    spin_accum<MU, SB>(acc, u);
  }
}

// MAXT: the largest block size the compiled kernel may be launched with.
template <class T, bool DAG, bool XPAY, bool NORM, int MAXT, class In, class Out, class Y, class G>
__global__ void __launch_bounds__(MAXT) k_hop(HopArgs<In, Out, Y, G> a) {
  if (a.st != nullptr && a.st->flag != 0) return;
  const long cb = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double part[1] = {0.0};
  if (cb < a.g.Vh) {
    int c[4];
    a.g.coords(cb, a.out_par, c);
    cpx<T> acc[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) acc[j] = mk<T>(0, 0);
    hop_dir<0, DAG>(a.g, a.out_par, cb, c, a.in, a.gauge, acc);
    hop_dir<1, DAG>(a.g, a.out_par, cb, c, a.in, a.gauge, acc);
    hop_dir<2, DAG>(a.g, a.out_par, cb, c, a.in, a.gauge, acc);
    hop_dir<3, DAG>(a.g, a.out_par, cb, c, a.in, a.gauge, acc);
    if constexpr (XPAY) {
      cpx<T> yv[12];
      a.y.loadT(cb, yv);
      const T al = (T)a.alpha;
#pragma unroll
      for (int j = 0; j < 12; ++j) acc[j] = yv[j] + al * acc[j];
    }
    if constexpr (NORM) part[0] = site_norm2(acc);
    a.out.store(cb, acc);
  }
  if constexpr (NORM) {
    double tot[1];
    if (grid_sum<1>(a.red, part, tot)) {
      CGState* s = a.st;
      if (s != nullptr) {
        s->pAp = tot[0];
        if (!(tot[0] > 0.0) || !isfinite(tot[0])) s->flag |= FLAG_NAN;
        else s->alpha = s->rr / tot[0];
      }
    }
  }
}

// Launch-shape autotuner.  Candidates: block sizes 128 and 64 with the kernel
// compiled for at most 128 threads (FP32: 86-88 registers, no spills), and
// 256 with a kernel compiled for 256 threads (the compiler then takes up to
// 255 registers).  Register caps below the compiler's choice spill and lost
// 4-5 % inside the trajectory, so none is a candidate.  The first launches of
// a (formats, links, dagger, epilogue, volume) key outside a queued CG chunk
// cycle through the candidates (see hop_dispatch); the NORM variant reuses
// the shape of its key.
struct HopCfg {
  int threads, maxt;   // block size; the launch bound the kernel is compiled for
};
constexpr HopCfg HOP_CANDIDATES[] = {{128, 128}, {256, 256}, {64, 128}};
constexpr int HOP_NCAND = sizeof(HOP_CANDIDATES) / sizeof(HOP_CANDIDATES[0]);

template <class T, bool D, bool X, bool N, class In, class Out, class Y, class G>
void hop_launch_cfg(wd_ctx* c, HopCfg cfg, const HopArgs<In, Out, Y, G>& a) {
  const int nb = nblocks(c->g.Vh, cfg.threads);
  if (cfg.maxt == 256) k_hop<T, D, X, N, 256, In, Out, Y, G><<<nb, cfg.threads, 0, c->stream>>>(a);
  else k_hop<T, D, X, N, 128, In, Out, Y, G><<<nb, cfg.threads, 0, c->stream>>>(a);
}

// Online tuning: the first HOP_NCAND * TUNE_ROUNDS tunable launches of a key
// are real launches of the pipeline, cycling through the candidates, each
// bracketed by CUDA events (so every candidate is timed in the data flow it
// serves: inputs just written by the producing kernel, L2 as in production).
// When all samples are in, the best time per candidate decides.
// The candidate order rotates from round to round (a clock ramp or a cache
// state favours no candidate), a candidate's score is its median time, and the
// default shape is replaced only by a candidate at least 3 % faster.
constexpr int TUNE_ROUNDS = 5;

inline int tune_candidate(int sample) {
  const int round = sample / HOP_NCAND;
  return (sample + round) % HOP_NCAND;
}

inline int tune_settle(wd_ctx* c, long long key, TuneSamples& s) {
  WD_CUDA(cudaEventSynchronize(s.ev.back()));
  float med[HOP_NCAND];
  for (int k = 0; k < HOP_NCAND; ++k) {
    float t[TUNE_ROUNDS];
    int n = 0;
    for (int i = 0; i < HOP_NCAND * TUNE_ROUNDS; ++i) {
      if (tune_candidate(i) != k) continue;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, s.ev[2 * i], s.ev[2 * i + 1]);
      t[n++] = ms;
    }
    std::sort(t, t + n);
    med[k] = t[n / 2];
  }
  int pick = 0;
  for (int k = 1; k < HOP_NCAND; ++k)
    if (med[k] < 0.97f * med[pick]) pick = k;
  for (auto& e : s.ev) cudaEventDestroy(e);
  c->tune_samples.erase(key);
  c->tune[key] = {HOP_CANDIDATES[pick].threads, HOP_CANDIDATES[pick].maxt};
  return WD_OK;
}

template <class T, bool D, bool X, bool N, class In, class Out, class Y, class G>
int hop_dispatch(wd_ctx* c, long long key, bool may_tune, const HopArgs<In, Out, Y, G>& a) {
  HopCfg cfg = HOP_CANDIDATES[0];
  auto it = c->tune.find(key);
  if (it != c->tune.end()) {
    cfg = HopCfg{it->second.first, it->second.second};
  } else if (may_tune && c->autotune && !N) {
    TuneSamples& s = c->tune_samples[key];
    const int i = (int)s.ev.size() / 2;               // sample index
    cfg = HOP_CANDIDATES[tune_candidate(i)];
    cudaEvent_t e0, e1;
    WD_CUDA(cudaEventCreate(&e0));
    WD_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, c->stream);
    hop_launch_cfg<T, D, X, N>(c, cfg, a);
    cudaEventRecord(e1, c->stream);
    s.ev.push_back(e0);
    s.ev.push_back(e1);
    WD_CHECK_LAUNCH();
    if ((int)s.ev.size() == 2 * HOP_NCAND * TUNE_ROUNDS) WD_TRY(tune_settle(c, key, s));
    return WD_OK;
  }
  hop_launch_cfg<T, D, X, N>(c, cfg, a);
  WD_CHECK_LAUNCH();
  return WD_OK;
}

template <class T, class In, class Out, class Y, class G>
int launch_hop(wd_ctx* c, bool dag, bool xpay, bool norm, long long key, bool may_tune,
               const HopArgs<In, Out, Y, G>& a) {
  if (norm && nblocks(c->g.Vh, 64) > RED_MAX_BLOCKS) return fail(WD_ERR_ARG, "lattice too large for one reduction grid");
  key = key * 4 + (dag ? 2 : 0) + (xpay ? 1 : 0);
  if (!dag) {
    if (!xpay) return hop_dispatch<T, false, false, false>(c, key, may_tune, a);
    if (!norm) return hop_dispatch<T, false, true, false>(c, key, may_tune, a);
    return hop_dispatch<T, false, true, true>(c, key, may_tune, a);
  }
  if (norm) return fail(WD_ERR_ARG, "hop: the |out|^2 epilogue exists for M_hat, not M_hat^dag");
  if (!xpay) return hop_dispatch<T, true, false, false>(c, key, may_tune, a);
  return hop_dispatch<T, true, true, false>(c, key, may_tune, a);
}

// format objects from fields
inline SpF64 sp64(const Field& f) { return SpF64{(double2*)f.data, f.stride}; }
inline SpF32 sp32(const Field& f) { return SpF32{(float4*)f.data, f.stride}; }
template <class H> inline Sp16<H> sp16(const Field& f) { return Sp16<H>{(uint4*)f.data, f.norm, f.stride}; }

template <class T, class In, class Out, class Y>
int hop_with_gauge(wd_ctx* c, int out_par, bool dag, In in, Out out, Y y, bool xpay, double alpha,
                   bool norm_cg, bool in_cg, bool use64) {
  Reduce red = reducer(c);
  CGState* st = (norm_cg || in_cg) ? c->cgs : nullptr;
  // tuning key: formats of in / out / y and the link storage
  const long long base = ((long long)In::fmt * 8 + Out::fmt) * 8 + (xpay ? Y::fmt : 7);
  const bool may_tune = !in_cg;
  if constexpr (std::is_same<T, dd>::value) {
    GDD G{c->gauge_dd, c->g.Vh};
    HopArgs<In, Out, Y, GDD> a{c->g, out_par, in, out, y, G, alpha, red, st};
    return launch_hop<T>(c, dag, xpay, norm_cg, base * 4 + 3, may_tune, a);
  } else {
  if (use64) {
    GF64 G{c->gauge64, c->g.Vh};
    HopArgs<In, Out, Y, GF64> a{c->g, out_par, in, out, y, G, alpha, red, st};
    return launch_hop<T>(c, dag, xpay, norm_cg, base * 4 + 0, may_tune, a);
  }
  if (c->recon == WD_RECON_12) {
    GF32R12 G{c->gauge32r12, c->g.Vh};
    HopArgs<In, Out, Y, GF32R12> a{c->g, out_par, in, out, y, G, alpha, red, st};
    return launch_hop<T>(c, dag, xpay, norm_cg, base * 4 + 2, may_tune, a);
  }
  GF32 G{c->gauge32, c->g.Vh};
  HopArgs<In, Out, Y, GF32> a{c->g, out_par, in, out, y, G, alpha, red, st};
  return launch_hop<T>(c, dag, xpay, norm_cg, base * 4 + 1, may_tune, a);
  }
}

// per-family dispatchers (one translation unit each)
int hop_f64(wd_ctx* c, int out_par, bool dag, const Field& in, const Field& out, const Field* y,
            double alpha, bool norm_cg, bool in_cg);
int hop_f32(wd_ctx* c, int out_par, bool dag, const Field& in, const Field& out, const Field* y,
            double alpha, bool norm_cg, bool in_cg);
int hop_h16(wd_ctx* c, int out_par, bool dag, const Field& in, const Field& out, const Field* y,
            double alpha, bool norm_cg, bool in_cg);
int hop_dd(wd_ctx* c, int out_par, bool dag, const Field& in, const Field& out, const Field* y,
           double alpha, bool norm_cg, bool in_cg);
inline SpDD spdd(const Field& f) { return SpDD{(float4*)f.data, f.stride}; }

}  // namespace wd
