// Tile-staged hopping stencil for 12-real FP32 links (Section 3.1 of the
// paper: Wilson fermions, even-odd preconditioning), fed by bulk asynchronous
// copies into shared memory.
//
// One persistent block per SM, warp-specialised:
//   - a producer warp copies, for a tile of TT_TILE consecutive output sites
//     (whole x rows), the data of one neighbour direction at a time into a ring
//     of shared-memory stages with cp.async.bulk (1-D bulk copies of the Tensor
//     Memory Accelerator; completion counted in bytes on an mbarrier): the three
//     stored rows of the tile's links of that direction and the neighbour
//     spinors, i.e. the tile's face shifted by one site in mu.  For mu = y, z, t
//     the neighbour of the site (xh, row R) is (xh, row R') with R' the
//     neighbour row, so a face is the tile's rows mapped row by row: one copy
//     per run of consecutive neighbour rows (one run, or two where the face
//     wraps around the lattice).  For mu = x the neighbours lie in the tile's
//     own rows of the other parity, which are copied as they are;
//   - TT_TILE consumer threads (one output site each) wait on the stage's full
//     barrier, read link and spinor from shared memory, apply the projector,
//     the rebuilt link and the accumulation, and release the stage on its empty
//     barrier (one arrival per warp, after the values read have been used).
// Epilogue vectors (y of out = y + alpha D in, and the Chebyshev-step operands
// v, s, s_prev) come through the same ring.  The producer runs up to NS stages
// ahead (three 72 KB stages for FP32 spinors, four 50 KB stages for 16-bit), so
// every SM keeps that much of its reads in flight without any register holding
// them, and the consumers read at shared-memory latency.
//
// Measured at 32^3 x 64 (FP32 K_hat, links 12 reals): 0.70 ms per application
// against 0.54 ms for the per-thread staged kernel (dslash_staged.cuh), which
// stays the default.  With 256-site tiles (8 consumer warps, six 36 KB stages)
// it took 0.98 ms; ncu showed DRAM traffic equal to the algorithmic bytes but
// DRAM only 35 % busy, 14 % of warps active and the consumers stalled on the
// stage barriers: the ring fills at about 37 GB/s per SM.  A producer of two
// warps issuing 16-byte cp.async per element instead of bulk copies took
// 0.74 ms (256-site tiles) and 0.82 ms (512).
//
// Every wait is bounded (about two seconds): on expiry the thread records
// WD_ERR_TIMEOUT in the context's device error word (and FLAG_TIMEOUT in the
// solver state when there is one), stops its work, and the producer waits
// (again bounded) for the copies it has issued before the block ends.
#pragma once
#include "dslash_staged.cuh"

namespace wd {

constexpr int TT_TILE = 512;                   // output sites per tile = consumer threads
constexpr int TT_THREADS = TT_TILE + 32;       // + one producer warp
constexpr long long TT_WAIT_NS = 2000000000LL; // bound of every wait

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy primitives (PTX ISA: mbarrier, cp.async.bulk)
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ long long gtimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait for the completion of the phase with the given parity; false after ns
__device__ __forceinline__ bool mbar_wait_ns(unsigned long long* b, unsigned parity, long long ns) {
  if (mbar_try(b, parity)) return true;
  const long long t0 = gtimer();
  for (unsigned k = 1;; ++k) {
    if (mbar_try(b, parity)) return true;
    if ((k & 255u) == 0 && gtimer() - t0 > ns) return false;
  }
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity) {
  return mbar_wait_ns(b, parity, TT_WAIT_NS);
}
// global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte
// aligned), completion counted on the barrier
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned long long* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(smem_u32(b))
               : "memory");
}

// ---------------------------------------------------------------------------
// spinor formats in a stage: component arrays of TT_TILE sites, as in HBM.
// copy(k, ...) issues the k-th of the NCOPY bulk copies of n sites.
template <class S> struct TTFmt;
template <> struct TTFmt<SpF32> {
  static constexpr unsigned SITE_BYTES = 96;
  static constexpr int NCOPY = 6;
  __device__ __forceinline__ static void copy(int k, unsigned dst, const SpF32& f, long src, int dsite, int n,
                                              unsigned long long* b) {
    bulk_g2s(dst + (unsigned)(k * TT_TILE + dsite) * 16u, f.p + k * f.stride + src, (unsigned)n * 16u, b);
  }
  __device__ __forceinline__ static void read(const unsigned char* base, int i, cpx<float> (&s)[12]) {
    const float4* q = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const float4 v = q[j * TT_TILE + i];
      s[2 * j] = {v.x, v.y};
      s[2 * j + 1] = {v.z, v.w};
    }
  }
  static bool aligned(const SpF32& f) { return ((uintptr_t)f.p & 15) == 0; }
};
template <class H> struct TTFmt<Sp16<H>> {
  static constexpr unsigned SITE_BYTES = 52;   // 48 bytes of 16-bit values + the FP32 norm
  static constexpr int NCOPY = 4;              // three 16-byte words per site, then the norms
  __device__ __forceinline__ static void copy(int k, unsigned dst, const Sp16<H>& f, long src, int dsite, int n,
                                              unsigned long long* b) {
    if (k < 3) bulk_g2s(dst + (unsigned)(k * TT_TILE + dsite) * 16u, f.p + k * f.stride + src, (unsigned)n * 16u, b);
    else bulk_g2s(dst + 3u * TT_TILE * 16u + (unsigned)dsite * 4u, f.nrm + src, (unsigned)n * 4u, b);
  }
  __device__ __forceinline__ static void read(const unsigned char* base, int i, cpx<float> (&s)[12]) {
    const uint4* q = reinterpret_cast<const uint4*>(base);
    const float nm = reinterpret_cast<const float*>(base + 3 * TT_TILE * 16)[i];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const uint4 v = q[j * TT_TILE + i];
      const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; ++k)
        s[4 * j + k] = {nm * H16Traits<H>::to_f((unsigned short)(w[k] & 0xffffu)),
                        nm * H16Traits<H>::to_f((unsigned short)(w[k] >> 16))};
    }
  }
  static bool aligned(const Sp16<H>& f) { return ((uintptr_t)f.p & 15) == 0 && ((uintptr_t)f.nrm & 15) == 0; }
};

constexpr unsigned TT_LINK_BYTES = 3u * TT_TILE * 16u;   // three stored rows of 12-real links
template <class In> constexpr unsigned tt_slot_bytes() { return TT_LINK_BYTES + TT_TILE * TTFmt<In>::SITE_BYTES; }
// ring depth: as many stages as fit in 227 KB of shared memory, at most 8
template <class In> constexpr int tt_stages() {
  return (int)((227u * 1024u - 1024u) / tt_slot_bytes<In>()) > 8 ? 8 : (int)((227u * 1024u - 1024u) / tt_slot_bytes<In>());
}

// Chebyshev-step epilogue operands: out = ca (v + cmu s - (y + alpha D in)) - cb s_prev
struct TTPoly {
  SpF32 v, s, sp;
  float ca, cmu, cb;
};

// Copies of one direction's stage, spread over the producer warp's lanes.
// Lane r < nr holds row R0 + r's coordinates (y, z, t) and row index R.  For
// each run of consecutive neighbour rows (a piece) the stage needs NCOPY spinor
// copies, and for a backward direction three link copies of the same rows; a
// forward direction's links are the tile's own rows (three copies).  Copy
// number k of the stage goes to lane k mod 32.
template <class In, class A>
__device__ __forceinline__ void tt_issue_dir(const A& a, int D, int lane, int nr, int Lh, int R, int y, int z, int t,
                                             int R0, unsigned dst, unsigned long long* fb) {
  const int mu = D >> 1;
  const bool fwd = (D & 1) == 0;
  int Rn = R;
  if (mu == 1) Rn = R + (fwd ? (y + 1 == a.g.L[1] ? 1 - a.g.L[1] : 1) : (y == 0 ? a.g.L[1] - 1 : -1));
  else if (mu == 2) Rn = R + a.g.L[1] * (fwd ? (z + 1 == a.g.L[2] ? 1 - a.g.L[2] : 1) : (z == 0 ? a.g.L[2] - 1 : -1));
  else if (mu == 3)
    Rn = R + a.g.L[1] * a.g.L[2] * (fwd ? (t + 1 == a.g.L[3] ? 1 - a.g.L[3] : 1) : (t == 0 ? a.g.L[3] - 1 : -1));
  const int prev = __shfl_up_sync(0xffffffffu, Rn, 1);
  const unsigned starts = __ballot_sync(0xffffffffu, lane < nr && (lane == 0 || Rn != prev + 1));
  const int np = __popc(starts);
  constexpr int NC = TTFmt<In>::NCOPY;
  const int per = fwd ? NC : NC + 3;                 // copies per piece
  const int ntup = np * per + (fwd ? 3 : 0);
  for (int k0 = 0; k0 < ntup; k0 += 32) {            // uniform over the warp
    const int k = k0 + lane;
    int p = k / per, j = k - p * per;
    if (k >= np * per) p = 0;                        // forward links, or idle lanes
    unsigned m = starts;
    for (int q = 0; q < p; ++q) m &= m - 1;
    const int r0 = __ffs(m) - 1;                     // first row of piece p
    const unsigned later = m & (m - 1);
    const int r1 = later ? __ffs(later) - 1 : nr;    // one past its last row
    const int rn0 = __shfl_sync(0xffffffffu, Rn, r0 < 0 ? 0 : r0);
    if (k < np * per) {
      const int dsite = r0 * Lh, n = (r1 - r0) * Lh;
      const long src = (long)rn0 * Lh;
      if (j < NC) {
        TTFmt<In>::copy(j, dst + TT_LINK_BYTES, a.in, src, dsite, n, fb);
      } else {
        const float4* g = a.gauge.p + (long)((mu * 2 + 1 - a.out_par) * 3 + (j - NC)) * a.gauge.stride + src;
        bulk_g2s(dst + (unsigned)((j - NC) * TT_TILE + dsite) * 16u, g, (unsigned)n * 16u, fb);
      }
    } else if (k < ntup) {
      const int jl = k - np * per;
      const float4* g = a.gauge.p + (long)((mu * 2 + a.out_par) * 3 + jl) * a.gauge.stride + (long)R0 * Lh;
      bulk_g2s(dst + (unsigned)(jl * TT_TILE) * 16u, g, TT_TILE * 16u, fb);
    }
  }
}

// EPI: 0 out = D in; 1 out = y + alpha D in; 2 the Chebyshev step above (FP32)
template <bool DAG, int EPI, bool NORM, class In, class Out, class Y>
__global__ void __launch_bounds__(TT_THREADS, 1)
    k_hop_tt(HopArgs<In, Out, Y, GF32R12> a, TTPoly pe, unsigned* kerr) {
  constexpr int NS = tt_stages<In>();
  constexpr unsigned SLOT = tt_slot_bytes<In>();
  constexpr int NEPI = EPI == 0 ? 0 : (EPI == 1 ? 1 : 4);
  constexpr int NSTG = 8 + NEPI;
  static_assert(TTFmt<Y>::SITE_BYTES <= TTFmt<In>::SITE_BYTES, "epilogue vectors fit a stage");
  extern __shared__ __align__(128) unsigned char tt_smem[];
  __shared__ __align__(8) unsigned long long full[NS], empty[NS];

  if (a.st != nullptr && a.st->flag != 0) return;   // the same for every thread
  const int tid = threadIdx.x;
  const int Lh = a.g.Lh;
  const int nr = TT_TILE / Lh;                       // rows per tile (<= 32)
  const int ntiles = (int)(a.g.Vh / TT_TILE);
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], TT_TILE / 32);            // one arrival per consumer warp
    }
    mbar_fence_init();
  }
  __syncthreads();

  bool bad = false;
  double part = 0.0;
  const unsigned base = smem_u32(tt_smem);
  if (tid >= TT_TILE) {
    // ------------------------------------------------- producer: bulk copies
    const int lane = tid - TT_TILE;
    int q = 0;
    for (int tile = blockIdx.x; tile < ntiles && !bad; tile += gridDim.x) {
      const int R0 = tile * nr;
      // coordinates of this lane's row (lanes >= nr carry a copy of row R0)
      const int R = R0 + (lane < nr ? lane : 0);
      const int y = R % a.g.L[1];
      const int zt = R / a.g.L[1];
      const int z = zt % a.g.L[2], t = zt / a.g.L[2];
      for (int st = 0; st < NSTG; ++st, ++q) {
        const int slot = q % NS;
        const unsigned ph = (unsigned)(q / NS) & 1u;
        // every lane waits; the warp leaves together if any lane's wait expired
        if (!__all_sync(0xffffffffu, mbar_wait(&empty[slot], ph ^ 1u))) { bad = true; break; }
        const unsigned dst = base + (unsigned)slot * SLOT;
        unsigned long long* fb = &full[slot];
        if (st < 8) {
          if (lane == 0) mbar_arrive_tx(fb, TT_LINK_BYTES + TT_TILE * TTFmt<In>::SITE_BYTES);
          __syncwarp();
          tt_issue_dir<In>(a, st, lane, nr, Lh, R, y, z, t, R0, dst, fb);
        } else {
          if (lane == 0) mbar_arrive_tx(fb, TT_TILE * TTFmt<Y>::SITE_BYTES);
          __syncwarp();
          const int e = st - 8;
          const long s0 = (long)R0 * Lh;
          if (lane < TTFmt<Y>::NCOPY) {
            if constexpr (EPI == 1) TTFmt<Y>::copy(lane, dst + TT_LINK_BYTES, a.y, s0, 0, TT_TILE, fb);
            if constexpr (EPI == 2) {
              const SpF32& f = e == 0 ? a.y : (e == 1 ? pe.v : (e == 2 ? pe.s : pe.sp));
              TTFmt<SpF32>::copy(lane, dst + TT_LINK_BYTES, f, s0, 0, TT_TILE, fb);
            }
          }
        }
        __syncwarp();
      }
    }
    if (lane == 0) {
      // the block must not end with copies in flight: wait for the last NS
      // stages issued (already complete unless a consumer left early)
      bool done = true;
      for (int k = 1; k <= NS && k <= q; ++k) {
        const int qq = q - k;
        if (!mbar_wait(&full[qq % NS], (unsigned)(qq / NS) & 1u)) { done = false; break; }
      }
      if (bad || !done) {
        atomicOr(kerr, 1u);
        if (a.st != nullptr) atomicOr(&a.st->flag, FLAG_TIMEOUT);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------- consumers
    const int i = tid;                       // site within the tile
    const int lane = tid & 31;
    const int ir = i / Lh, xh = i - ir * Lh;
    int q = 0;
    for (int tile = blockIdx.x; tile < ntiles && !bad; tile += gridDim.x) {
      const long cb = (long)tile * TT_TILE + i;
      const int R = tile * nr + ir;
      const int y = R % a.g.L[1];
      const int zt = R / a.g.L[1];
      const int z = zt % a.g.L[2], t = zt / a.g.L[2];
      const bool xodd = ((a.out_par + y + z + t) & 1) != 0;
      // shared-memory index of the x neighbours (same row, other parity)
      const int ixf = ir * Lh + (xodd ? (xh + 1 == Lh ? 0 : xh + 1) : xh);
      const int ixb = ir * Lh + (xodd ? xh : (xh == 0 ? Lh - 1 : xh - 1));
      cpx<float> acc[12];
#pragma unroll
      for (int j = 0; j < 12; ++j) acc[j] = mk<float>(0, 0);
#pragma unroll
      for (int D = 0; D < 8; ++D) {
        const int slot = q % NS;
        const unsigned ph = (unsigned)(q / NS) & 1u;
        if (!__all_sync(0xffffffffu, mbar_wait(&full[slot], ph))) { bad = true; break; }
        const unsigned char* sb = tt_smem + (size_t)slot * SLOT;
        const int mu = D >> 1;
        const bool fwd = (D & 1) == 0;
        const int is = mu == 0 ? (fwd ? ixf : ixb) : i;   // neighbour spinor
        const int il = fwd ? i : is;                        // link: U(x) or U(x - mu)
        cpx<float> U[9], s[12], h[6], u[6];
        const float4* L = reinterpret_cast<const float4*>(sb);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float4 v = L[j * TT_TILE + il];
          U[2 * j] = {v.x, v.y};
          U[2 * j + 1] = {v.z, v.w};
        }
        TTFmt<In>::read(sb + TT_LINK_BYTES, is, s);
        U[6] = conj(U[1] * U[5] - U[2] * U[4]);
        U[7] = conj(U[2] * U[3] - U[0] * U[5]);
        U[8] = conj(U[0] * U[4] - U[1] * U[3]);
        constexpr int SF = DAG ? +1 : -1;
        const bool flip = (mu == 3) && (fwd ? t == a.g.L[3] - 1 : t == 0);
        // the projector and its reconstruction are compile-time per direction
        switch (D) {
#define WD_TT_DIR(DD)                                                   \
  case DD: {                                                            \
    constexpr int MU_ = (DD) >> 1;                                      \
    constexpr int SG_ = ((DD) & 1) == 0 ? SF : -SF;                     \
    spin_project<MU_, SG_>(s, h);                                       \
    if (flip) {                                                         \
      _Pragma("unroll") for (int j = 0; j < 6; ++j) h[j] = mk<float>(-h[j].r, -h[j].i); \
    }                                                                   \
    if constexpr (((DD) & 1) == 0) su3_mul(U, h, u);                    \
    else su3_dag_mul(U, h, u);                                          \
    spin_accum<MU_, SG_>(acc, u);                                       \
  } break;
          WD_TT_DIR(0) WD_TT_DIR(1) WD_TT_DIR(2) WD_TT_DIR(3) WD_TT_DIR(4) WD_TT_DIR(5) WD_TT_DIR(6) WD_TT_DIR(7)
#undef WD_TT_DIR
        }
        // every value read from the stage has been used: release it (one
        // arrival per warp once all of its lanes are here)
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
        ++q;
      }
      if (bad) break;
      if constexpr (EPI >= 1) {
        const float al = (float)a.alpha;
        cpx<float> tv[EPI == 2 ? 12 : 1];
#pragma unroll
        for (int e = 0; e < NEPI; ++e) {
          const int slot = q % NS;
          const unsigned ph = (unsigned)(q / NS) & 1u;
          if (!__all_sync(0xffffffffu, mbar_wait(&full[slot], ph))) { bad = true; break; }
          const unsigned char* sb = tt_smem + (size_t)slot * SLOT + TT_LINK_BYTES;
          cpx<float> w[12];
          TTFmt<Y>::read(sb, i, w);
          if (e == 0) {
#pragma unroll
            for (int j = 0; j < 12; ++j) acc[j] = w[j] + al * acc[j];         // y + alpha D in
          } else if constexpr (EPI == 2) {
            // the same operation order as the thread kernel's Chebyshev step
            if (e == 1) {
#pragma unroll
              for (int j = 0; j < 12; ++j) tv[j] = w[j];                          // v
            } else if (e == 2) {
#pragma unroll
              for (int j = 0; j < 12; ++j) tv[j] = tv[j] + pe.cmu * w[j] - acc[j];  // v + cmu s - K s
            } else {
#pragma unroll
              for (int j = 0; j < 12; ++j) acc[j] = pe.ca * tv[j] - pe.cb * w[j];  // ca (.) - cb s_prev
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty[slot]);
          ++q;
        }
        if (bad) break;
      }
      if constexpr (NORM) part += site_norm2(acc);
      a.out.store(cb, acc);
    }
    if (bad) {
      atomicOr(kerr, 1u);
      if (a.st != nullptr) atomicOr(&a.st->flag, FLAG_TIMEOUT);
    }
  }
  if constexpr (NORM) {
    double v[1] = {part}, tot[1];
    if (grid_sum<1>(a.red, v, tot)) {
      CGState* st = a.st;
      if (st != nullptr) {
        st->pAp = tot[0];
        if (!(tot[0] > 0.0) || !isfinite(tot[0])) st->flag |= FLAG_NAN;
        else st->alpha = st->rr / tot[0];
      }
    }
  }
}

// The tile-staged kernel needs whole x rows per tile (Lx/2 divides TT_TILE,
// at most 32 rows per tile, Lx/2 a multiple of 4 so that every 16-bit norm
// copy starts on 16 bytes), a whole number of tiles and 16-byte aligned fields.
inline bool tt_eligible(const wd_ctx* c) {
  const int Lh = c->g.Lh;
  return c->stencil == WD_STENCIL_TILE && Lh >= 8 && Lh % 4 == 0 && TT_TILE % Lh == 0 && TT_TILE / Lh <= 32 &&
         c->g.Vh % TT_TILE == 0 && c->g.Vh / Lh < (1L << 30) && c->nsm > 0 && c->kerr != nullptr;
}

template <bool DAG, int EPI, bool NORM, class In, class Out, class Y>
int tt_launch(wd_ctx* c, const HopArgs<In, Out, Y, GF32R12>& a, const TTPoly& pe) {
  constexpr size_t smem = (size_t)tt_stages<In>() * tt_slot_bytes<In>();
  static unsigned long long attr_set = 0;   // per instantiation, one bit per device
  const unsigned long long bit = 1ull << (c->device & 63);
  if (!(attr_set & bit)) {
    WD_CUDA(cudaFuncSetAttribute(k_hop_tt<DAG, EPI, NORM, In, Out, Y>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    attr_set |= bit;
  }
  const long ntiles = c->g.Vh / TT_TILE;
  const int grid = (int)std::min<long>(ntiles, c->nsm);
  k_hop_tt<DAG, EPI, NORM, In, Out, Y><<<grid, TT_THREADS, smem, c->stream>>>(a, pe, c->kerr);
  WD_CHECK_LAUNCH();
  return WD_OK;
}

// out = D in (or y + alpha D in, with |out|^2 for CG) through the tile-staged kernel
template <class In, class Out, class Y>
int hop_tt(wd_ctx* c, int out_par, bool dag, const In& I, const Out& O, const Y& Yv, bool xpay, double alpha,
           bool norm_cg, bool in_cg) {
  if (norm_cg && (dag || !xpay)) return fail(WD_ERR_ARG, "hop: the |out|^2 epilogue exists for M_hat only");
  if (!TTFmt<In>::aligned(I) || (xpay && !TTFmt<Y>::aligned(Yv)))
    return fail(WD_ERR_ARG, "hop: tile-staged stencil needs 16-byte aligned fields");
  CGState* st = (norm_cg || in_cg) ? c->cgs : nullptr;
  HopArgs<In, Out, Y, GF32R12> a{c->g, out_par, I, O, Yv, GF32R12{c->gauge32r12, c->g.Vh}, alpha, reducer(c), st};
  const TTPoly pe{};
  if (!dag) {
    if (!xpay) return tt_launch<false, 0, false>(c, a, pe);
    if (!norm_cg) return tt_launch<false, 1, false>(c, a, pe);
    return tt_launch<false, 1, true>(c, a, pe);
  }
  if (!xpay) return tt_launch<true, 0, false>(c, a, pe);
  return tt_launch<true, 1, false>(c, a, pe);
}

}  // namespace wd
