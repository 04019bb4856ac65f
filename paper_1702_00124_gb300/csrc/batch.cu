// Batched solves: many independent lattices of uneven volume, each with
// several right-hand sides, advanced together.
//
// Every (lattice, right-hand side) pair is one system A_s x_s = b_s with
// A_s = K_hat(kappa_s) on its lattice (Section 2 of the paper: CG on K).  The
// right-hand sides of one lattice are interleaved in memory
// (element (chunk, cb, r) at (chunk * Vh + cb) * nrhs + r), so that the lanes
// of a warp that work on the nrhs systems of one site read that site's links
// once: the link bytes per system drop by nrhs.  One launch covers all
// lattices: every block belongs to one lattice (blocks are laid out lattice
// after lattice), so per-system sums are formed per block and then added in
// block order by a second small kernel (deterministic).  CG scalars of every
// system live on the device; an iteration is eight launches, and a chunk of
// iterations can be captured once in a CUDA graph and replayed.  The bulk is
// FP32; the residual of a system is recomputed in FP64 (reliable update,
// through its lattice's own context) when its iterated residual has dropped by
// delta or below the tolerance.
#include <algorithm>
#include <cmath>
#include <new>

#include "dslash_staged.cuh"

namespace wd {

constexpr int B_MAXR = 8;   // right-hand sides per lattice

enum BField { BF_P = 0, BF_AP, BF_R, BF_X, BF_T1, BF_T2, BF_N };

struct BLat {
  Geom g;
  int nr;          // right-hand sides
  int sys0;        // first system index
  int block0;      // first block of this lattice
  int nblocks;
  int recon;       // 12 or 18 stored reals
  double kappa;
  const float4* g12;
  const float2* g18;
  float4* f[BF_N];  // interleaved FP32 half spinors, stride 6 chunks x Vh x nr
};

// format adaptor: spinor index i of one system -> interleaved element
struct SpIL {
  float4* p;
  long stride;    // Vh * nr
  int nr, r;
  template <class T> __device__ __forceinline__ void loadT(long i, cpx<T> (&s)[12]) const {
    SpF32{p, stride}.loadT(i * nr + r, s);
  }
  template <class T> __device__ __forceinline__ void store(long i, const cpx<T> (&s)[12]) const {
    SpF32{p, stride}.store(i * nr + r, s);
  }
};

struct BArgs {
  const BLat* lats;
  const int* block_lat;    // block -> lattice
  CGState* st;             // per system
  double* partial;         // [block][B_MAXR]
  int out_par;
  int use_flags;           // inside CG: systems with a stop flag do no work
};

// The RPT consecutive (site, rhs) items of this thread in block vb of the
// layout (blocks of blockDim.x * RPT items, lattice after lattice); with
// nr % RPT == 0 they belong to one site.
struct BItem {
  const BLat* L;
  long cb;
  int r0;
  bool valid;
};
__device__ __forceinline__ BItem b_item(const BArgs& a, int vb, int rpt) {
  BItem it;
  it.L = a.lats + a.block_lat[vb];
  const long item0 = (long)(vb - it.L->block0) * (blockDim.x * rpt) + (long)threadIdx.x * rpt;
  it.valid = item0 < it.L->g.Vh * it.L->nr;
  it.cb = 0;
  it.r0 = 0;
  if (it.valid) {
    const unsigned u = (unsigned)item0, nr = (unsigned)it.L->nr;   // Vh * nr < 2^31 (checked at creation)
    it.cb = (long)(u / nr);
    it.r0 = (int)(u - (unsigned)it.cb * nr);
  }
  return it;
}
// Loads of data the same kernel may have written (COH): the persistent kernel
// reads fields, sums and solver state that other blocks wrote in an earlier
// phase, which the read-only path (ld.global.nc) does not allow; ld.global.cg
// reads them from L2, after the grid barrier's fences.  Separate launches use
// the read-only path.
template <bool COH> __device__ __forceinline__ float4 bld(const float4* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}
template <bool COH> __device__ __forceinline__ void bload(const float4* f, long stride, long e, cpx<float> (&s)[12]) {
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const float4 v = bld<COH>(f + j * stride + e);
    s[2 * j] = {v.x, v.y};
    s[2 * j + 1] = {v.z, v.w};
  }
}
// inside CG, systems that carry a stop flag do no work
template <bool COH> __device__ __forceinline__ bool b_active(const BArgs& a, const BLat* L, int r) {
  if (!a.use_flags) return true;
  if constexpr (COH) return __ldcg(&a.st[L->sys0 + r].flag) == 0;
  else return a.st[L->sys0 + r].flag == 0;
}

// Per-block partial sums of every right-hand side: v[r] holds the thread's
// value for its system (zero elsewhere).  FP32 sums (warp shuffles, then the
// warps in order by lane r of warp 0), stored as FP64; GB300 issues FP64 at
// 1/64 of the FP32 rate, and eight FP64 shuffle trees per thread cost more
// than the hop itself.  Deterministic: a fixed order at every level.
__device__ __forceinline__ void b_block_partial(const BArgs& a, int vb, float (&v)[B_MAXR]) {
  __shared__ float sh[B_MAXR * 32];
#pragma unroll
  for (int k = 0; k < B_MAXR; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < B_MAXR; ++k) sh[k * 32 + wid] = v[k];
  }
  __syncthreads();
  if (wid == 0 && lane < B_MAXR) {
    const int nw = (blockDim.x + 31) >> 5;
    float t = 0.f;
    for (int w = 0; w < nw; ++w) t += sh[lane * 32 + w];
    a.partial[(long)vb * B_MAXR + lane] = (double)t;
  }
}

// One direction of the hop for RPT right-hand sides of one site: the link is
// loaded and rebuilt once and applied to the RPT neighbour spinors (consecutive
// in the interleaved layout).
template <int MU, bool DAG, int RPT, bool COH, class G>
__device__ __forceinline__ void bhop_dir(const Geom& g, int par, long cb, const int (&c)[4], const float4* in,
                                         long stride, int nr, int r0, const G& gauge, cpx<float> (&acc)[RPT][12]) {
  constexpr int SF = DAG ? +1 : -1;
#pragma unroll
  for (int fb = 0; fb < 2; ++fb) {
    const bool fwd = fb == 0;
    int n[4] = {c[0], c[1], c[2], c[3]};
    if (fwd) n[MU] = (n[MU] + 1 == g.L[MU]) ? 0 : n[MU] + 1;
    else n[MU] = (n[MU] == 0) ? g.L[MU] - 1 : n[MU] - 1;
    const long nb = g.cb_of(n[0], n[1], n[2], n[3]);
    cpx<float> U[9];
    if (fwd) gauge.load(MU, par, cb, U);
    else gauge.load(MU, 1 - par, nb, U);
    const bool flip = MU == 3 && (fwd ? c[3] == g.L[3] - 1 : c[3] == 0);
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      cpx<float> sp[12], h[6], u[6];
      bload<COH>(in, stride, nb * nr + r0 + k, sp);
      if (fwd) spin_project<MU, SF>(sp, h);
      else spin_project<MU, -SF>(sp, h);
      if (flip) {
#pragma unroll
        for (int j = 0; j < 6; ++j) h[j] = mk<float>(-h[j].r, -h[j].i);
      }
      if (fwd) {
        su3_mul(U, h, u);
        spin_accum<MU, SF>(acc[k], u);
      } else {
        su3_dag_mul(U, h, u);
        spin_accum<MU, -SF>(acc[k], u);
      }
    }
  }
}

// Batched hop; every thread handles RPT consecutive (site, rhs) items of its
// lattice (nr % RPT == 0, so they share one site) in block vb of the layout.
// Systems with a stop flag are not written.
template <bool DAG, bool XPAY, bool NORM, bool R12, int RPT, bool COH = false>
__device__ __forceinline__ void bhop_body(const BArgs& a, int vb, int fin, int fout, int fy) {
  const BItem it = b_item(a, vb, RPT);
  const BLat* L = it.L;
  float v[B_MAXR];
#pragma unroll
  for (int k = 0; k < B_MAXR; ++k) v[k] = 0.f;
  bool act[RPT];
  bool any = false;
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    act[k] = it.valid && b_active<COH>(a, L, it.r0 + k);
    any = any || act[k];
  }
  if (any) {
    const long cb = it.cb;
    const int r0 = it.r0;
    const long stride = L->g.Vh * L->nr;
    int c[4];
    L->g.coords(cb, a.out_par, c);
    cpx<float> acc[RPT][12];
#pragma unroll
    for (int k = 0; k < RPT; ++k)
#pragma unroll
      for (int j = 0; j < 12; ++j) acc[k][j] = mk<float>(0, 0);
    const float4* in = L->f[fin];
    if constexpr (R12) {
      GF32R12 G{L->g12, L->g.Vh};
      bhop_dir<0, DAG, RPT, COH>(L->g, a.out_par, cb, c, in, stride, L->nr, r0, G, acc);
      bhop_dir<1, DAG, RPT, COH>(L->g, a.out_par, cb, c, in, stride, L->nr, r0, G, acc);
      bhop_dir<2, DAG, RPT, COH>(L->g, a.out_par, cb, c, in, stride, L->nr, r0, G, acc);
      bhop_dir<3, DAG, RPT, COH>(L->g, a.out_par, cb, c, in, stride, L->nr, r0, G, acc);
    } else {
      GF32 G{L->g18, L->g.Vh};
      bhop_dir<0, DAG, RPT, COH>(L->g, a.out_par, cb, c, in, stride, L->nr, r0, G, acc);
      bhop_dir<1, DAG, RPT, COH>(L->g, a.out_par, cb, c, in, stride, L->nr, r0, G, acc);
      bhop_dir<2, DAG, RPT, COH>(L->g, a.out_par, cb, c, in, stride, L->nr, r0, G, acc);
      bhop_dir<3, DAG, RPT, COH>(L->g, a.out_par, cb, c, in, stride, L->nr, r0, G, acc);
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      if (!act[k]) continue;
      const int r = r0 + k;
      if constexpr (XPAY) {
        cpx<float> yv[12];
        bload<COH>(L->f[fy], stride, cb * L->nr + r, yv);
        const float al = (float)(-L->kappa * L->kappa);
#pragma unroll
        for (int j = 0; j < 12; ++j) acc[k][j] = yv[j] + al * acc[k][j];
      }
      if constexpr (NORM) {
        float q = 0.f;
#pragma unroll
        for (int j = 0; j < 12; ++j) q = fmaf(acc[k][j].r, acc[k][j].r, fmaf(acc[k][j].i, acc[k][j].i, q));
#pragma unroll
        for (int m = 0; m < B_MAXR; ++m)
          if (m == r) v[m] = q;
      }
      SpIL{L->f[fout], stride, L->nr, r}.store(cb, acc[k]);
    }
  }
  if constexpr (NORM) b_block_partial(a, vb, v);
}

template <bool DAG, bool XPAY, bool NORM, bool R12, int RPT>
__global__ void __launch_bounds__(256) k_bhop(BArgs a, int fin, int fout, int fy) {
  bhop_body<DAG, XPAY, NORM, R12, RPT>(a, blockIdx.x, fin, fout, fy);
}

// The batched hop on the single-lattice stencil's per-thread pipeline (one
// (site, rhs) item per thread, 12-real links): the links of the next two
// directions are copied into shared memory by cp.async while the current one
// is computed (dslash_staged.cuh); the item's lattice supplies geometry, links
// and fields.  Blocks of HOP_ST_THREADS items.
template <bool DAG, bool XPAY, bool NORM>
__global__ void __launch_bounds__(HOP_ST_THREADS, HOP_MINB) k_bhop_st(BArgs a, int fin, int fout, int fy) {
  extern __shared__ float4 sbuf[];
  const BItem it = b_item(a, blockIdx.x, 1);
  const BLat* L = it.L;
  float v[B_MAXR];
#pragma unroll
  for (int k = 0; k < B_MAXR; ++k) v[k] = 0.f;
  if (it.valid && b_active<false>(a, L, it.r0)) {
    const long stride = L->g.Vh * L->nr;
    const int r = it.r0;
    const SpIL in{L->f[fin], stride, L->nr, r}, out{L->f[fout], stride, L->nr, r};
    using HA = HopArgs<SpIL, SpIL, SpIL, GF32R12>;
    const HA ha{L->g, a.out_par, in, out, in, GF32R12{L->g12, L->g.Vh}, 0.0, Reduce{nullptr, nullptr, nullptr},
                nullptr};
    Staged<HOP_NST, DAG, HA> S{ha, it.cb, {0, 0, 0, 0}, sbuf, (int)threadIdx.x, (int)blockDim.x};
    L->g.coords(it.cb, a.out_par, S.c);
    cpx<float> acc[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) acc[j] = mk<float>(0, 0);
    S.run(acc);
    if constexpr (XPAY) {
      cpx<float> yv[12];
      SpIL{L->f[fy], stride, L->nr, r}.loadT(it.cb, yv);
      const float al = (float)(-L->kappa * L->kappa);
#pragma unroll
      for (int j = 0; j < 12; ++j) acc[j] = yv[j] + al * acc[j];
    }
    if constexpr (NORM) {
      float q = 0.f;
#pragma unroll
      for (int j = 0; j < 12; ++j) q = fmaf(acc[j].r, acc[j].r, fmaf(acc[j].i, acc[j].i, q));
#pragma unroll
      for (int m = 0; m < B_MAXR; ++m)
        if (m == r) v[m] = q;
    }
    out.store(it.cb, acc);
  }
  if constexpr (NORM) b_block_partial(a, blockIdx.x, v);
}

// x += alpha p; r -= alpha Ap; partial |r|^2 (RPT items per thread)
template <int RPT, bool COH = false>
__device__ __forceinline__ void bupdate_body(const BArgs& a, int vb) {
  const BItem it = b_item(a, vb, RPT);
  float v[B_MAXR];
#pragma unroll
  for (int k = 0; k < B_MAXR; ++k) v[k] = 0.f;
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int r = it.r0 + k;
    if (!it.valid || !b_active<COH>(a, it.L, r)) continue;
    const BLat* L = it.L;
    const long stride = L->g.Vh * L->nr;
    const long e = it.cb * L->nr + r;
    const float al = (float)(COH ? __ldcg(&a.st[L->sys0 + r].alpha) : a.st[L->sys0 + r].alpha);
    SpIL X{L->f[BF_X], stride, L->nr, r}, R{L->f[BF_R], stride, L->nr, r};
    cpx<float> xv[12], pv[12], rv[12], av[12];
    bload<COH>(L->f[BF_X], stride, e, xv);
    bload<COH>(L->f[BF_P], stride, e, pv);
    bload<COH>(L->f[BF_R], stride, e, rv);
    bload<COH>(L->f[BF_AP], stride, e, av);
    float q = 0.f;
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      xv[j] = xv[j] + al * pv[j];
      rv[j] = rv[j] - al * av[j];
      q += norm2(rv[j]);
    }
    X.store(it.cb, xv);
    R.store(it.cb, rv);
#pragma unroll
    for (int m = 0; m < B_MAXR; ++m)
      if (m == r) v[m] = q;
  }
  b_block_partial(a, vb, v);
}
__global__ void __launch_bounds__(256) k_bupdate(BArgs a) { bupdate_body<1>(a, blockIdx.x); }

// p = r + beta p (RPT items per thread)
template <int RPT, bool COH = false>
__device__ __forceinline__ void bpupdate_body(const BArgs& a, int vb) {
  const BItem it = b_item(a, vb, RPT);
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int r = it.r0 + k;
    if (!it.valid || !b_active<COH>(a, it.L, r)) continue;
    const BLat* L = it.L;
    const long stride = L->g.Vh * L->nr;
    const long e = it.cb * L->nr + r;
    const float be = (float)(COH ? __ldcg(&a.st[L->sys0 + r].beta) : a.st[L->sys0 + r].beta);
    SpIL P{L->f[BF_P], stride, L->nr, r};
    cpx<float> pv[12], rv[12];
    bload<COH>(L->f[BF_P], stride, e, pv);
    bload<COH>(L->f[BF_R], stride, e, rv);
#pragma unroll
    for (int j = 0; j < 12; ++j) pv[j] = rv[j] + be * pv[j];
    P.store(it.cb, pv);
  }
}
__global__ void __launch_bounds__(256) k_bpupdate(BArgs a) { bpupdate_body<1>(a, blockIdx.x); }

// Per-system totals of the block partials, then the CG scalar step; one block
// per system s: thread t adds the partials of blocks t, t + blockDim, ... in
// order, the block adds the threads in a fixed tree (deterministic).
// mode 0: pAp -> alpha; mode 1: |r|^2 -> beta, flags.
constexpr int BRED_THREADS = 128;
__device__ __forceinline__ void breduce_body(const BLat* lats, int nlat, CGState* st, const double* partial,
                                             int mode, int s) {
  int l = 0;
  while (l < nlat && s >= lats[l].sys0 + lats[l].nr) ++l;
  if (l >= nlat || s < lats[l].sys0) return;     // the same for the whole block
  CGState& S = st[s];
  if (__ldcg(&S.flag) != 0) return;               // read before thread 0 may change it
  const BLat& L = lats[l];
  const int r = s - L.sys0;
  double v[1] = {0.0};
  for (int b = threadIdx.x; b < L.nblocks; b += blockDim.x) v[0] += __ldcg(partial + (long)(L.block0 + b) * B_MAXR + r);
  __shared__ double sh[32];
  block_sum<1>(v, sh);
  if (threadIdx.x != 0) return;
  const double tot = v[0];
  if (!isfinite(tot)) { S.flag |= FLAG_NAN; return; }
  if (mode == 0) {
    S.pAp = tot;
    if (!(tot > 0.0)) S.flag |= FLAG_NAN;
    else S.alpha = S.rr / tot;
  } else {
    S.rr_old = S.rr;
    S.beta = tot / S.rr;
    S.rr = tot;
    S.iter += 1;
    if (tot <= S.upd_rr) S.flag |= FLAG_UPDATE;
    if (S.iter >= S.maxiter) S.flag |= FLAG_MAXITER;
  }
}
__global__ void __launch_bounds__(BRED_THREADS) k_breduce(const BLat* lats, int nlat, CGState* st,
                                                          const double* partial, int mode) {
  breduce_body(lats, nlat, st, partial, mode, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Persistent CG: one cooperative launch runs `iters` CG iterations of every
// system.  Its phases are the launches of an iteration of the graph path
// (hop, hop + pAp sums, per-system reduce, hop, hop, update + |r|^2 sums,
// reduce, p update), each looping over the same blocks of the layout (or over
// the systems), separated by grid barriers.  A cooperative launch keeps every
// block resident, so the barrier cannot wait on a block that never runs; each
// wait is still bounded (2 s) and an expiry ends the kernel with bit 1 of the
// batch's error word set.
struct GridBar {
  unsigned count, gen;
};
constexpr long long B_WAIT_NS = 2000000000LL;

__device__ __forceinline__ long long b_gtimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// all blocks arrive; false if the wait expired (then every block leaves)
__device__ __forceinline__ bool grid_barrier(GridBar* g, unsigned& gen, unsigned* kerr) {
  __shared__ int ok_sh;
  __syncthreads();                               // the block's writes happen before thread 0 arrives
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = gen + 1;
    __threadfence();
    if (atomicAdd(&g->count, 1u) == gridDim.x - 1) {
      atomicExch(&g->count, 0u);
      __threadfence();
      atomicExch(&g->gen, target);                // releases the others
    } else {
      const long long t0 = b_gtimer();
      for (unsigned k = 1; *(volatile unsigned*)&g->gen != target; ++k) {
        if ((k & 255u) == 0 && b_gtimer() - t0 > B_WAIT_NS) {
          ok = 0;
          atomicOr(kerr, 2u);
          break;
        }
      }
    }
    __threadfence();
    gen = target;
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

template <bool R12, int RPT>
__global__ void __launch_bounds__(256) k_bcg_chunk(BArgs a, int nlat, int nsys, int nvb, int iters, GridBar* gb,
                                                   unsigned* kerr) {
  unsigned gen = 0;
  if (threadIdx.x == 0) gen = *(volatile unsigned*)&gb->gen;   // before the first arrival of any block
  a.use_flags = 1;
#define WD_BSYNC() \
  if (!grid_barrier(gb, gen, kerr)) return
  for (int it = 0; it < iters; ++it) {
    a.out_par = 1;
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) bhop_body<false, false, false, R12, RPT, true>(a, vb, BF_P, BF_T1, -1);
    WD_BSYNC();
    a.out_par = 0;
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
      bhop_body<false, true, true, R12, RPT, true>(a, vb, BF_T1, BF_T2, BF_P);
      __syncthreads();                             // the block's partial-sum buffer is reused
    }
    WD_BSYNC();
    for (int sy = blockIdx.x; sy < nsys; sy += gridDim.x) {
      breduce_body(a.lats, nlat, a.st, a.partial, 0, sy);
      __syncthreads();
    }
    WD_BSYNC();
    a.out_par = 1;
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) bhop_body<true, false, false, R12, RPT, true>(a, vb, BF_T2, BF_T1, -1);
    WD_BSYNC();
    a.out_par = 0;
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) bhop_body<true, true, false, R12, RPT, true>(a, vb, BF_T1, BF_AP, BF_T2);
    WD_BSYNC();
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
      bupdate_body<RPT, true>(a, vb);
      __syncthreads();
    }
    WD_BSYNC();
    for (int sy = blockIdx.x; sy < nsys; sy += gridDim.x) {
      breduce_body(a.lats, nlat, a.st, a.partial, 1, sy);
      __syncthreads();
    }
    WD_BSYNC();
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) bpupdate_body<RPT, true>(a, vb);
    WD_BSYNC();
  }
#undef WD_BSYNC
}

// one system's slot of an interleaved field <-> a standard FP64 half spinor
__global__ void k_slot(long Vh, int nr, int r, float4* il, double2* f64, int dir /*0 get, 1 put, 2 zero*/) {
  const long cb = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= Vh) return;
  SpIL I{il, Vh * nr, nr, r};
  cpx<double> s[12];
  if (dir == 0) {
    I.loadT(cb, s);
    SpF64{f64, Vh}.store(cb, s);
  } else if (dir == 1) {
    SpF64{f64, Vh}.loadT(cb, s);
    I.store(cb, s);
  } else {
#pragma unroll
    for (int j = 0; j < 12; ++j) s[j] = mk(0.0, 0.0);
    I.store(cb, s);
  }
}

// p_s = r_s + beta p_s for one system
__global__ void k_slot_pupdate(long Vh, int nr, int r, float4* p, const float4* rr, float beta) {
  const long cb = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= Vh) return;
  SpIL P{p, Vh * nr, nr, r}, R{const_cast<float4*>(rr), Vh * nr, nr, r};
  cpx<float> pv[12], rv[12];
  P.loadT(cb, pv);
  R.loadT(cb, rv);
#pragma unroll
  for (int j = 0; j < 12; ++j) pv[j] = rv[j] + beta * pv[j];
  P.store(cb, pv);
}

}  // namespace wd

using namespace wd;

struct wd_batch {
  std::vector<wd_ctx*> ctx;
  std::vector<BLat> lat_h;
  BLat* lat_d = nullptr;
  int S = 0;                     // systems
  int threads = 128;             // items (site, rhs) per block (autotuned on first use)
  int rpt = 1;                   // right-hand sides per thread of the batched hop (autotuned)
  int staged = 0;                // 1: the hop on the per-thread link-staging pipeline (rpt 1, 128 items)
  bool tuned = false;
  std::vector<int> block_lat_h;
  int* block_lat_d = nullptr;
  int nblocks = 0;
  double* partial = nullptr;
  CGState* st_d = nullptr;
  CGState* st_h = nullptr;       // pinned
  cudaStream_t stream = nullptr; // capture-capable stream
  bool own_stream = false;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_iters = 0;
  long long launches = 0;
  int in_cg = 0;                 // launches belong to a CG iteration
  std::vector<void*> mem;
  GridBar* gbar = nullptr;       // grid barrier of the persistent CG kernel
  unsigned* kerr = nullptr;      // device error word: bit 1 = a grid-barrier wait expired
  int coop_grid = 0;             // resident blocks of the persistent kernel (0: not known yet)
  int coop_rpt = 0;              // the rhs-per-thread its grid was computed for
};

namespace wd {

static int b_layout(wd_batch* b, int threads) {
  WD_CUDA(cudaStreamSynchronize(b->stream));   // no launch may still use the old layout
  b->threads = threads;
  b->block_lat_h.clear();
  for (size_t l = 0; l < b->lat_h.size(); ++l) {
    BLat& L = b->lat_h[l];
    L.block0 = (int)b->block_lat_h.size();
    L.nblocks = nblocks(L.g.Vh * L.nr, threads);
    for (int k = 0; k < L.nblocks; ++k) b->block_lat_h.push_back((int)l);
  }
  b->nblocks = (int)b->block_lat_h.size();
  cudaFree(b->block_lat_d);
  cudaFree(b->partial);
  b->block_lat_d = nullptr;
  b->partial = nullptr;
  WD_CUDA(cudaMalloc(&b->block_lat_d, sizeof(int) * b->nblocks));
  WD_CUDA(cudaMalloc(&b->partial, sizeof(double) * B_MAXR * b->nblocks));
  WD_CUDA(cudaMemcpy(b->block_lat_d, b->block_lat_h.data(), sizeof(int) * b->nblocks, cudaMemcpyHostToDevice));
  WD_CUDA(cudaMemcpy(b->lat_d, b->lat_h.data(), sizeof(BLat) * b->lat_h.size(), cudaMemcpyHostToDevice));
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return WD_OK;
}

static BArgs b_args(wd_batch* b, int out_par) {
  return BArgs{b->lat_d, b->block_lat_d, b->st_d, b->partial, out_par, b->in_cg};
}

static int b_hop(wd_batch* b, int out_par, bool dag, int fin, int fout, int fy, bool norm) {
  const BArgs a = b_args(b, out_par);
  const bool r12 = b->lat_h[0].recon == 12;
#define WD_BH(D, X, N, R)                                                                                 \
  do {                                                                                                    \
    if (b->rpt == 4) k_bhop<D, X, N, R, 4><<<b->nblocks, b->threads / 4, 0, b->stream>>>(a, fin, fout, fy); \
    else if (b->rpt == 2) k_bhop<D, X, N, R, 2><<<b->nblocks, b->threads / 2, 0, b->stream>>>(a, fin, fout, fy); \
    else k_bhop<D, X, N, R, 1><<<b->nblocks, b->threads, 0, b->stream>>>(a, fin, fout, fy);                \
  } while (0)
  if (r12 && b->staged) {
#define WD_BS(D, X, N) k_bhop_st<D, X, N><<<b->nblocks, HOP_ST_THREADS, HOP_STAGE_SMEM, b->stream>>>(a, fin, fout, fy)
    if (!dag) {
      if (fy < 0) WD_BS(false, false, false);
      else if (norm) WD_BS(false, true, true);
      else WD_BS(false, true, false);
    } else {
      if (fy < 0) WD_BS(true, false, false);
      else WD_BS(true, true, false);
    }
#undef WD_BS
  } else if (r12) {
    if (!dag) {
      if (fy < 0) WD_BH(false, false, false, true);
      else if (norm) WD_BH(false, true, true, true);
      else WD_BH(false, true, false, true);
    } else {
      if (fy < 0) WD_BH(true, false, false, true);
      else WD_BH(true, true, false, true);
    }
  } else {
    if (!dag) {
      if (fy < 0) WD_BH(false, false, false, false);
      else if (norm) WD_BH(false, true, true, false);
      else WD_BH(false, true, false, false);
    } else {
      if (fy < 0) WD_BH(true, false, false, false);
      else WD_BH(true, true, false, false);
    }
  }
#undef WD_BH
  b->launches += 1;
  WD_CUDA(cudaGetLastError());
  return WD_OK;
}

// out = K_hat in for every system (fields of the batch), with pAp when norm
static int b_khat(wd_batch* b, int fin, int fout, bool norm) {
  WD_TRY(b_hop(b, 1, false, fin, BF_T1, -1, false));
  WD_TRY(b_hop(b, 0, false, BF_T1, BF_T2, fin, norm));
  if (norm) {
    k_breduce<<<b->S, BRED_THREADS, 0, b->stream>>>(b->lat_d, (int)b->lat_h.size(), b->st_d, b->partial, 0);
    b->launches += 1;
  }
  WD_TRY(b_hop(b, 1, true, BF_T2, BF_T1, -1, false));
  WD_TRY(b_hop(b, 0, true, BF_T1, fout, BF_T2, false));
  WD_CUDA(cudaGetLastError());
  return WD_OK;
}

static int b_iteration(wd_batch* b) {
  b->in_cg = 1;   // systems that carry a stop flag skip their work
  int s = b_khat(b, BF_P, BF_AP, true);
  if (s == WD_OK) {
    k_bupdate<<<b->nblocks, b->threads, 0, b->stream>>>(b_args(b, 0));
    k_breduce<<<b->S, BRED_THREADS, 0, b->stream>>>(b->lat_d, (int)b->lat_h.size(), b->st_d, b->partial, 1);
    k_bpupdate<<<b->nblocks, b->threads, 0, b->stream>>>(b_args(b, 0));
    b->launches += 3;
  }
  b->in_cg = 0;
  WD_TRY(s);
  WD_CUDA(cudaGetLastError());
  return WD_OK;
}

static int b_slot(wd_batch* b, int l, int r, int field, double* f64, int dir) {
  const BLat& L = b->lat_h[l];
  k_slot<<<nblocks(L.g.Vh, 128), 128, 0, b->stream>>>(L.g.Vh, L.nr, r, L.f[field], (double2*)f64, dir);
  b->launches += 1;
  WD_CUDA(cudaGetLastError());
  return WD_OK;
}

static int b_enter(wd_batch* b) {   // order the batch stream after the contexts' stream
  if (!b->own_stream) return WD_OK;
  WD_CUDA(cudaEventRecord(b->ev_in, b->ctx[0]->stream));
  WD_CUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
  return WD_OK;
}
static int b_leave(wd_batch* b) {
  if (!b->own_stream) return WD_OK;
  WD_CUDA(cudaEventRecord(b->ev_out, b->stream));
  WD_CUDA(cudaStreamWaitEvent(b->ctx[0]->stream, b->ev_out, 0));
  return WD_OK;
}

// Tile-shape tuner: time the batched K_hat for each candidate shape (items
// per block, right-hand sides per thread of the hop) and keep the fastest.
// Rounds with the candidate order rotated; median per candidate; the default
// (128 items, one rhs per thread) is replaced only by a candidate at least 3 %
// faster.  A shape with rpt > 1 needs nr % rpt == 0 on every lattice.
struct BShape {
  int threads, rpt, staged;
};
static int b_autotune(wd_batch* b) {
  constexpr int ROUNDS = 5;
  const BShape all[] = {{128, 1, 0}, {256, 1, 0}, {64, 1, 0}, {128, 2, 0}, {256, 2, 0},
                        {128, 4, 0}, {256, 4, 0}, {HOP_ST_THREADS, 1, 1}};
  std::vector<BShape> cand;
  for (const BShape& c : all) {
    bool ok = !c.staged || b->lat_h[0].recon == 12;
    for (const BLat& L : b->lat_h) ok = ok && (L.nr % c.rpt == 0);
    if (ok) cand.push_back(c);
  }
  const int NC = (int)cand.size();
  std::vector<std::vector<float>> t(NC);
  cudaEvent_t e0, e1;
  WD_CUDA(cudaEventCreate(&e0));
  WD_CUDA(cudaEventCreate(&e1));
  WD_TRY(b_khat(b, BF_P, BF_AP, false));      // warm
  for (int r = 0; r < ROUNDS; ++r) {
    for (int j = 0; j < NC; ++j) {
      const int k = (j + r) % NC;
      WD_TRY(b_layout(b, cand[k].threads));
      b->rpt = cand[k].rpt;
      b->staged = cand[k].staged;
      cudaEventRecord(e0, b->stream);
      WD_TRY(b_khat(b, BF_P, BF_AP, false));
      cudaEventRecord(e1, b->stream);
      WD_CUDA(cudaEventSynchronize(e1));
      float ms;
      cudaEventElapsedTime(&ms, e0, e1);
      t[k].push_back(ms);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::vector<float> med(NC);
  for (int k = 0; k < NC; ++k) {
    std::sort(t[k].begin(), t[k].end());
    med[k] = t[k][t[k].size() / 2];
  }
  int pick = 0;
  for (int k = 1; k < NC; ++k)
    if (med[k] < 0.97f * med[pick]) pick = k;
  WD_TRY(b_layout(b, cand[pick].threads));
  b->rpt = cand[pick].rpt;
  b->staged = cand[pick].staged;
  b->tuned = true;
  return WD_OK;
}

// Persistent mode: the resident grid of the cooperative kernel for the
// batch's tile shape (all blocks must fit at once), computed once per shape.
template <bool R12, int RPT>
static int b_coop_grid(wd_batch* b, int threads) {
  int per_sm = 0;
  WD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bcg_chunk<R12, RPT>, threads, 0));
  int dev = 0, nsm = 0;
  WD_CUDA(cudaGetDevice(&dev));
  WD_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (per_sm < 1) return fail(WD_ERR_ARG, "wd_batch_cg: the persistent kernel does not fit on an SM");
  b->coop_grid = std::max(1, std::min(per_sm * nsm, std::max(b->nblocks, b->S)));
  return WD_OK;
}
static int b_coop_prepare(wd_batch* b) {
  if (b->coop_grid > 0 && b->coop_rpt == b->rpt) return WD_OK;
  const bool r12 = b->lat_h[0].recon == 12;
  const int t = b->threads / b->rpt;
  int s;
  if (r12) s = b->rpt == 4 ? b_coop_grid<true, 4>(b, t) : b->rpt == 2 ? b_coop_grid<true, 2>(b, t) : b_coop_grid<true, 1>(b, t);
  else s = b->rpt == 4 ? b_coop_grid<false, 4>(b, t) : b->rpt == 2 ? b_coop_grid<false, 2>(b, t) : b_coop_grid<false, 1>(b, t);
  if (s == WD_OK) b->coop_rpt = b->rpt;
  return s;
}
// one chunk of `iters` CG iterations of every system in one cooperative launch
static int b_coop_chunk(wd_batch* b, int iters) {
  WD_CUDA(cudaMemsetAsync(b->gbar, 0, sizeof(GridBar), b->stream));   // a clean barrier for every launch
  BArgs a = b_args(b, 0);
  int nlat = (int)b->lat_h.size(), nsys = b->S, nvb = b->nblocks;
  void* args[] = {&a, &nlat, &nsys, &nvb, &iters, &b->gbar, &b->kerr};
  const dim3 grid(b->coop_grid), block(b->threads / b->rpt);
  const bool r12 = b->lat_h[0].recon == 12;
  void* k;
  if (r12) k = b->rpt == 4 ? (void*)k_bcg_chunk<true, 4> : b->rpt == 2 ? (void*)k_bcg_chunk<true, 2> : (void*)k_bcg_chunk<true, 1>;
  else k = b->rpt == 4 ? (void*)k_bcg_chunk<false, 4> : b->rpt == 2 ? (void*)k_bcg_chunk<false, 2> : (void*)k_bcg_chunk<false, 1>;
  WD_CUDA(cudaLaunchCooperativeKernel(k, grid, block, args, 0, b->stream));
  b->launches += 1;
  return WD_OK;
}

}  // namespace wd

extern "C" {

int wd_batch_create(wd_ctx* const* ctxs, int nlat, const double* kappas, const int* nrhs, wd_batch** out) {
  if (!ctxs || !kappas || !nrhs || !out || nlat < 1) return fail(WD_ERR_ARG, "wd_batch_create: bad arguments");
  *out = nullptr;
  for (int l = 0; l < nlat; ++l) {
    if (!ctxs[l] || !ctxs[l]->have_gauge) return fail(WD_ERR_STATE, "wd_batch_create: every context needs a gauge field");
    if (nrhs[l] < 1 || nrhs[l] > B_MAXR) return fail(WD_ERR_ARG, "wd_batch_create: 1 <= nrhs <= 8 per lattice");
    if (ctxs[l]->g.Vh * (long)nrhs[l] >= (1L << 31))
      return fail(WD_ERR_ARG, "wd_batch_create: Vh * nrhs must stay below 2^31 per lattice");
    if (ctxs[l]->stream != ctxs[0]->stream) return fail(WD_ERR_ARG, "wd_batch_create: contexts must share a stream");
  }
  wd_batch* b = new (std::nothrow) wd_batch();
  if (!b) return fail(WD_ERR_ARG, "out of host memory");
  auto bail = [&](int code) { wd_batch_destroy(b); return code; };
  b->ctx.assign(ctxs, ctxs + nlat);
  int s0 = 0;
  for (int l = 0; l < nlat; ++l) {
    wd_ctx* c = ctxs[l];
    BLat L{};
    L.g = c->g;
    L.nr = nrhs[l];
    L.sys0 = s0;
    L.recon = ctxs[0]->recon == WD_RECON_12 ? 12 : 18;
    L.kappa = kappas[l];
    L.g12 = c->gauge32r12;
    L.g18 = c->gauge32;
    for (int f = 0; f < BF_N; ++f) {
      void* p = nullptr;
      cudaError_t e = cudaMalloc(&p, sizeof(float4) * 6 * c->g.Vh * L.nr);
      if (e != cudaSuccess) return bail(cuda_fail(e, "wd_batch_create: cudaMalloc"));
      b->mem.push_back(p);
      L.f[f] = (float4*)p;
    }
    s0 += L.nr;
    b->lat_h.push_back(L);
  }
  b->S = s0;
  cudaError_t e = cudaMalloc(&b->lat_d, sizeof(BLat) * nlat);
  if (e == cudaSuccess) e = cudaMalloc(&b->st_d, sizeof(CGState) * b->S);
  if (e == cudaSuccess) e = cudaMallocHost(&b->st_h, sizeof(CGState) * b->S);
  if (e == cudaSuccess) e = cudaMemset(b->st_d, 0, sizeof(CGState) * b->S);
  if (e == cudaSuccess) e = cudaMalloc(&b->gbar, sizeof(GridBar));
  if (e == cudaSuccess) e = cudaMalloc(&b->kerr, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(b->kerr, 0, sizeof(unsigned));
  if (e != cudaSuccess) return bail(cuda_fail(e, "wd_batch_create: allocation"));
  if (ctxs[0]->stream == nullptr) {   // the legacy stream cannot be captured: use our own
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(cuda_fail(e, "wd_batch_create: stream"));
    b->own_stream = true;
  } else {
    b->stream = ctxs[0]->stream;
  }
  int s = b_layout(b, 128);
  if (s != WD_OK) return bail(s);
  *out = b;
  return WD_OK;
}

int wd_batch_destroy(wd_batch* b) {
  if (!b) return WD_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void* p : b->mem) cudaFree(p);
  cudaFree(b->lat_d);
  cudaFree(b->block_lat_d);
  cudaFree(b->partial);
  cudaFree(b->st_d);
  cudaFree(b->gbar);
  cudaFree(b->kerr);
  if (b->st_h) cudaFreeHost(b->st_h);
  if (b->own_stream) {
    cudaStreamDestroy(b->stream);
    cudaEventDestroy(b->ev_in);
    cudaEventDestroy(b->ev_out);
  }
  delete b;
  return WD_OK;
}

int wd_batch_mdagm(wd_batch* b, const double* const* in, double* const* out) {
  if (!b || !in || !out) return fail(WD_ERR_ARG, "wd_batch_mdagm: null argument");
  WD_TRY(b_enter(b));
  for (size_t l = 0; l < b->lat_h.size(); ++l) {
    const BLat& L = b->lat_h[l];
    for (int r = 0; r < L.nr; ++r)
      WD_TRY(b_slot(b, (int)l, r, BF_P, const_cast<double*>(in[l]) + (long)r * 24 * L.g.Vh, 1));
  }
  WD_TRY(b_khat(b, BF_P, BF_AP, false));
  for (size_t l = 0; l < b->lat_h.size(); ++l) {
    const BLat& L = b->lat_h[l];
    for (int r = 0; r < L.nr; ++r) WD_TRY(b_slot(b, (int)l, r, BF_AP, out[l] + (long)r * 24 * L.g.Vh, 0));
  }
  for (size_t l = 0; l < b->lat_h.size(); ++l) b->ctx[l]->nmat += b->lat_h[l].nr;
  return b_leave(b);
}

int wd_batch_cg(wd_batch* b, const double* const* bvec, double* const* x, const wd_cg_params* p, int use_graph,
                wd_cg_info* infos) {
  if (!b || !bvec || !x || !p) return fail(WD_ERR_ARG, "wd_batch_cg: null argument");
  if (!(p->tol > 0) || p->maxiter < 1) return fail(WD_ERR_ARG, "wd_batch_cg: tol > 0 and maxiter >= 1");
  if (use_graph < 0 || use_graph > 2)
    return fail(WD_ERR_ARG, "wd_batch_cg: use_graph must be 0 (launches), 1 (graph) or 2 (persistent kernel)");
  const double delta = (p->delta > 0 && p->delta < 1) ? p->delta : 1e-3;
  const int check = p->check_every > 0 ? p->check_every : 16;
  const int nlat = (int)b->lat_h.size();
  WD_TRY(b_enter(b));
  // x = 0, r = p = b (interleaved FP32); per-system |b|^2 in FP64
  std::vector<double> bb(b->S);
  std::vector<wd_cg_info> info(b->S);
  std::vector<long long> nmat0(nlat);
  for (int l = 0; l < nlat; ++l) {
    const BLat& L = b->lat_h[l];
    wd_ctx* c = b->ctx[l];
    nmat0[l] = c->nmat;
    for (int r = 0; r < L.nr; ++r) {
      const long off = (long)r * 24 * L.g.Vh;
      Field bf = wrap_f64(c, bvec[l] + off), xf = wrap_f64(c, x[l] + off);
      WD_TRY(zero(c, xf));
      WD_TRY(norm2(c, bf, &bb[L.sys0 + r]));
      WD_TRY(b_slot(b, l, r, BF_R, const_cast<double*>(bvec[l]) + off, 1));
      WD_TRY(b_slot(b, l, r, BF_P, const_cast<double*>(bvec[l]) + off, 1));
      WD_TRY(b_slot(b, l, r, BF_X, nullptr, 2));
    }
  }
  for (int s = 0; s < b->S; ++s) {
    CGState& S = b->st_h[s];
    S = CGState{};
    S.rr = S.rr_old = bb[s];
    S.stop_rr = p->tol * p->tol * bb[s];
    S.upd_rr = std::max(delta * delta * bb[s], S.stop_rr);
    S.maxiter = p->maxiter;
    S.flag = (bb[s] == 0.0) ? FLAG_DONE : 0;
  }
  WD_CUDA(cudaMemcpyAsync(b->st_d, b->st_h, sizeof(CGState) * b->S, cudaMemcpyHostToDevice, b->stream));
  if (!b->tuned) {
    // tune on K_hat p (p = b: real data); the pAp it leaves is recomputed
    WD_TRY(b_autotune(b));
  }
  // a chunk of iterations: one persistent cooperative launch (use_graph == 2),
  // or the iterations' launches as one CUDA graph (1), or plain launches (0)
  const bool persistent = use_graph == 2;
  if (persistent) WD_TRY(b_coop_prepare(b));
  if (use_graph == 1 && (b->graph == nullptr || b->graph_iters != check)) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaGraph_t g;
    WD_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const long long l0 = b->launches;
    int s = WD_OK;
    for (int k = 0; k < check && s == WD_OK; ++k) s = b_iteration(b);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    b->launches = l0;
    if (s != WD_OK) return s;
    if (e != cudaSuccess) return cuda_fail(e, "wd_batch_cg: graph capture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "wd_batch_cg: graph instantiate");
    b->graph_iters = check;
  }
  const int per_iter = 8;
  int status = WD_OK;
  for (;;) {
    if (persistent) {
      WD_TRY(b_coop_chunk(b, check));
    } else if (use_graph) {
      WD_CUDA(cudaGraphLaunch(b->graph, b->stream));
      b->launches += (long long)per_iter * check;
    } else {
      for (int k = 0; k < check; ++k) WD_TRY(b_iteration(b));
    }
    for (int l = 0; l < nlat; ++l) b->ctx[l]->nmat += (long long)check * b->lat_h[l].nr;
    WD_CUDA(cudaMemcpyAsync(b->st_h, b->st_d, sizeof(CGState) * b->S, cudaMemcpyDeviceToHost, b->stream));
    unsigned kerr_h = 0;
    if (persistent) WD_CUDA(cudaMemcpyAsync(&kerr_h, b->kerr, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream));
    WD_CUDA(cudaStreamSynchronize(b->stream));
    if (kerr_h != 0) {
      WD_CUDA(cudaMemsetAsync(b->kerr, 0, sizeof(unsigned), b->stream));
      WD_TRY(b_leave(b));
      return fail(WD_ERR_TIMEOUT, "wd_batch_cg: a grid-barrier wait of the persistent kernel expired");
    }
    bool all_done = true, changed = false;
    for (int l = 0; l < nlat && status == WD_OK; ++l) {
      const BLat& L = b->lat_h[l];
      wd_ctx* c = b->ctx[l];
      for (int r = 0; r < L.nr; ++r) {
        const int sidx = L.sys0 + r;
        CGState& S = b->st_h[sidx];
        if (S.flag == FLAG_DONE) continue;
        if (S.flag & FLAG_NAN) { status = fail(WD_ERR_NAN, "wd_batch_cg: non-finite value"); break; }
        if (S.flag == 0) { all_done = false; continue; }
        // reliable update of this system in FP64 on its own lattice
        const long off = (long)r * 24 * L.g.Vh;
        Field xf = wrap_f64(c, x[l] + off), bf = wrap_f64(c, bvec[l] + off);
        WsGuard w(c);
        Field t, rr, t1, t2;
        WD_TRY(w.get(WD_F64, &t));
        WD_TRY(w.get(WD_F64, &rr));
        WD_TRY(w.get(WD_F64, &t1));
        WD_TRY(w.get(WD_F64, &t2));
        WD_TRY(b_slot(b, l, r, BF_X, (double*)t.data, 0));
        WD_TRY(b_slot(b, l, r, BF_X, nullptr, 2));
        if (b->own_stream) {   // the context stream works on what the batch stream produced
          WD_CUDA(cudaEventRecord(b->ev_out, b->stream));
          WD_CUDA(cudaStreamWaitEvent(c->stream, b->ev_out, 0));
        }
        WD_TRY(axpby(c, 1.0, xf, 1.0, t, xf));
        if (c->resid_dd && c->gauge_dd) {
          // K_hat x in double-float when the lattice's context selects it (as
          // the single-system solver's true residual): FP64-class accuracy on
          // the FP32 pipes, b, x, r and the norm stay FP64
          Field xd, td, d1, d2;
          WD_TRY(w.get(WD_DD, &xd));
          WD_TRY(w.get(WD_DD, &td));
          WD_TRY(w.get(WD_DD, &d1));
          WD_TRY(w.get(WD_DD, &d2));
          WD_TRY(convert(c, xf, xd));
          WD_TRY(apply_khat(c, L.kappa, xd, td, d1, d2, false, false));
          WD_TRY(convert(c, td, t));
        } else {
          WD_TRY(apply_khat(c, L.kappa, xf, t, t1, t2, false, false));
        }
        WD_TRY(axpby(c, 1.0, bf, -1.0, t, rr));
        double rr2;
        WD_TRY(norm2(c, rr, &rr2));
        info[sidx].reliable_updates += 1;
        info[sidx].iters = S.iter;
        info[sidx].true_rel_resid = std::sqrt(rr2 / bb[sidx]);
        changed = true;
        if (!std::isfinite(rr2)) { status = fail(WD_ERR_NAN, "wd_batch_cg: non-finite residual"); break; }
        if (rr2 <= S.stop_rr) { S.flag = FLAG_DONE; continue; }
        if (S.flag & FLAG_MAXITER) { status = fail(WD_ERR_NOCONV, "wd_batch_cg: maxiter reached"); break; }
        all_done = false;
        WD_TRY(b_slot(b, l, r, BF_R, (double*)rr.data, 1));
        const double beta = rr2 / S.rr_old;
        k_slot_pupdate<<<nblocks(L.g.Vh, 128), 128, 0, b->stream>>>(L.g.Vh, L.nr, r, L.f[BF_P], L.f[BF_R],
                                                                    (float)beta);
        b->launches += 1;
        S.rr = rr2;
        S.upd_rr = std::max(delta * delta * rr2, S.stop_rr);
        S.flag = 0;
      }
    }
    if (status != WD_OK) break;
    if (changed) WD_CUDA(cudaMemcpyAsync(b->st_d, b->st_h, sizeof(CGState) * b->S, cudaMemcpyHostToDevice, b->stream));
    if (all_done) break;
  }
  for (int l = 0; l < nlat && infos; ++l) {
    const BLat& L = b->lat_h[l];
    for (int r = 0; r < L.nr; ++r) {
      const int sidx = L.sys0 + r;
      info[sidx].n_mat = info[sidx].iters + info[sidx].reliable_updates;
      infos[sidx] = info[sidx];
    }
  }
  WD_TRY(b_leave(b));
  return status;
}

int wd_batch_set_shape(wd_batch* b, int items_per_block, int rhs_per_thread, int link_staging) {
  if (!b) return fail(WD_ERR_ARG, "null batch");
  if (link_staging != 0 && link_staging != 1) return fail(WD_ERR_ARG, "wd_batch_set_shape: link_staging must be 0 or 1");
  if (link_staging && (items_per_block != HOP_ST_THREADS || rhs_per_thread != 1 || b->lat_h[0].recon != 12))
    return fail(WD_ERR_ARG, "wd_batch_set_shape: link staging needs 128 items per block, one rhs per thread, 12-real links");
  if (items_per_block != 64 && items_per_block != 128 && items_per_block != 256)
    return fail(WD_ERR_ARG, "wd_batch_set_shape: items_per_block must be 64, 128 or 256");
  if (rhs_per_thread != 1 && rhs_per_thread != 2 && rhs_per_thread != 4)
    return fail(WD_ERR_ARG, "wd_batch_set_shape: rhs_per_thread must be 1, 2 or 4");
  for (const BLat& L : b->lat_h)
    if (L.nr % rhs_per_thread != 0)
      return fail(WD_ERR_ARG, "wd_batch_set_shape: rhs_per_thread must divide every lattice's nrhs");
  WD_TRY(b_layout(b, items_per_block));
  b->rpt = rhs_per_thread;
  b->staged = link_staging;
  b->tuned = true;
  return WD_OK;
}

int wd_batch_shape(wd_batch* b, int* items_per_block, int* rhs_per_thread, int* link_staging) {
  if (!b) return fail(WD_ERR_ARG, "null batch");
  if (items_per_block) *items_per_block = b->threads;
  if (rhs_per_thread) *rhs_per_thread = b->rpt;
  if (link_staging) *link_staging = b->staged;
  return WD_OK;
}

int wd_batch_info(wd_batch* b, int* n_systems, int* threads, long long* launches) {
  if (!b) return fail(WD_ERR_ARG, "null batch");
  if (n_systems) *n_systems = b->S;
  if (threads) *threads = b->threads;
  if (launches) *launches = b->launches;
  return WD_OK;
}

}  // extern "C"
