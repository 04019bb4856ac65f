// Internal definitions shared by the CUDA translation units of libwdhmc.
//
// Geometry: even-odd (checkerboard) site ordering, cb = lex / 2 with
// lex = x + Lx (y + Ly (z + Lz t)); fermion time boundary antiperiodic.
// Storage formats (structure of arrays, one 16-byte or 8-byte word per
// thread per chunk so that a warp reads contiguous memory):
//   spinor F64   double2 [12][Vh]           (component j = 3 spin + colour)
//   spinor F32   float4  [6][Vh]            (components 2j, 2j+1)
//   spinor 16    uint4   [3][Vh] + float [Vh] norm: 8 half/bf16 values per
//                word, value = stored * norm, norm = max |component| of the site
//   gauge F64    double2 [4 mu][2 par][9][Vh]
//   gauge F32    float2  [4][2][9][Vh]       (18 reals)
//   gauge F32R12 float4  [4][2][3][Vh]       (rows 0,1; row 2 = (r0 x r1)^*)
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <type_traits>
#include <unordered_map>
#include <utility>
#include <vector>

#include "wdhmc.h"

namespace wd {

// ----------------------------------------------------------------------------
// complex arithmetic
template <class T> struct cpx { T r, i; };

template <class T> __host__ __device__ __forceinline__ cpx<T> mk(T r, T i) { return {r, i}; }
template <class T> __host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.r + b.r, a.i + b.i}; }
template <class T> __host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.r - b.r, a.i - b.i}; }
template <class T> __host__ __device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
template <class T> __host__ __device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return {s * a.r, s * a.i}; }
template <class T> __host__ __device__ __forceinline__ cpx<T> conj(cpx<T> a) { return {a.r, -a.i}; }
// conj(a) * b
template <class T> __host__ __device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) { return {a.r * b.r + a.i * b.i, a.r * b.i - a.i * b.r}; }
template <class T> __host__ __device__ __forceinline__ T norm2(cpx<T> a) { return a.r * a.r + a.i * a.i; }
// multiply by i^k (k mod 4)
template <int K, class T> __host__ __device__ __forceinline__ cpx<T> ipow(cpx<T> a) {
  constexpr int k = ((K % 4) + 4) % 4;
  if constexpr (k == 0) return a;
  else if constexpr (k == 1) return {-a.i, a.r};
  else if constexpr (k == 2) return {-a.r, -a.i};
  else return {a.i, -a.r};
}

// ----------------------------------------------------------------------------
// Double-float arithmetic: a value is hi + lo with two FP32 words (|lo| <=
// ulp(hi)/2), about 48 significant bits.  Sum and product follow the
// error-free transformations of Knuth (two-sum) and Dekker (two-product, here
// with an FMA); they run on the FP32 pipes, which GB300 has 60x more of than
// FP64.  Used only where an FP64-accurate operator is needed many times: the
// residual recomputation of mixed-precision solves, when selected.
struct dd {
  float hi, lo;
  dd() = default;
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dd(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ explicit dd(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};
__host__ __device__ __forceinline__ dd dd_fast2sum(float a, float b) {
  const float s = a + b;
  return dd(s, b - (s - a));
}
__host__ __device__ __forceinline__ dd dd_2sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return dd(s, (a - (s - bb)) + (b - bb));
}
// Sum with an exact two-sum of the high words and the low words added in
// FP32 (Dekker): relative error about 2^-44 unless the operands cancel.
__host__ __device__ __forceinline__ dd operator+(dd a, dd b) {
  dd s = dd_2sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return dd_fast2sum(s.hi, s.lo);
}
__host__ __device__ __forceinline__ dd& operator+=(dd& a, dd b) { return a = a + b; }
__host__ __device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__host__ __device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return dd_fast2sum(p, e);
}

// ----------------------------------------------------------------------------
// Gamma matrices, DeGrand-Rossi chiral basis (gamma_5 = diag(1,1,-1,-1)).
// Each gamma_mu has one non-zero per row; row a (a = 0,1) couples to column
// PERM[mu][a] with value i^PH[mu][a]:
//   g_x: (0,3) i   (1,2) i   (2,1) -i  (3,0) -i
//   g_y: (0,3) -1  (1,2) 1   (2,1) 1   (3,0) -1
//   g_z: (0,2) i   (1,3) -i  (2,0) -i  (3,1) i
//   g_t: (0,2) 1   (1,3) 1   (2,0) 1   (3,1) 1
// For r = (1 + s gamma_mu) psi (s = +-1) the upper half determines the rest:
//   h_a = psi_a + s g_a psi_PERM(a),  r_a = h_a,  r_PERM(a) = s conj(g_a) h_a.
template <int MU> struct Gam;
template <> struct Gam<0> { static constexpr int p0 = 3, p1 = 2, k0 = 1, k1 = 1; };
template <> struct Gam<1> { static constexpr int p0 = 3, p1 = 2, k0 = 2, k1 = 0; };
template <> struct Gam<2> { static constexpr int p0 = 2, p1 = 3, k0 = 1, k1 = 3; };
template <> struct Gam<3> { static constexpr int p0 = 2, p1 = 3, k0 = 0, k1 = 0; };

// ----------------------------------------------------------------------------
struct Geom {
  int L[4];
  int Lh;      // Lx / 2
  long V, Vh;
  // site index -> coordinates in 32-bit arithmetic (contexts have V < 2^31):
  // a 64-bit division by a runtime divisor is a long emulated sequence, and
  // every stencil thread needs three of them
  __host__ __device__ __forceinline__ void coords(long cb, int par, int c[4]) const {
    const unsigned u = (unsigned)cb, lh = (unsigned)Lh, l1 = (unsigned)L[1], l2 = (unsigned)L[2];
    const unsigned r0 = u / lh, r1 = r0 / l1, r2 = r1 / l2;
    const int xh = (int)(u - r0 * lh);
    c[1] = (int)(r0 - r1 * l1);
    c[2] = (int)(r1 - r2 * l2);
    c[3] = (int)r2;
    c[0] = 2 * xh + ((par + c[1] + c[2] + c[3]) & 1);
  }
  __host__ __device__ __forceinline__ long cb_of(int x, int y, int z, int t) const {
    return ((((long)t * L[2] + z) * L[1] + y) * L[0] + x) >> 1;
  }
  __host__ __device__ __forceinline__ long lex_of(int x, int y, int z, int t) const {
    return (((long)t * L[2] + z) * L[1] + y) * L[0] + x;
  }
};

// ----------------------------------------------------------------------------
// spinor storage formats
struct SpF64 {
  using real = double;
  static constexpr int fmt = WD_F64;
  double2* p;
  long stride;
  __device__ __forceinline__ void load(long i, cpx<double> (&s)[12]) const {
#pragma unroll
    for (int j = 0; j < 12; ++j) { double2 v = __ldg(p + j * stride + i); s[j] = {v.x, v.y}; }
  }
  template <class T> __device__ __forceinline__ void store(long i, const cpx<T> (&s)[12]) const {
#pragma unroll
    for (int j = 0; j < 12; ++j) p[j * stride + i] = make_double2((double)s[j].r, (double)s[j].i);
  }
  template <class T> __device__ __forceinline__ void loadT(long i, cpx<T> (&s)[12]) const {
#pragma unroll
    for (int j = 0; j < 12; ++j) { double2 v = __ldg(p + j * stride + i); s[j] = {(T)v.x, (T)v.y}; }
  }
};

struct SpF32 {
  using real = float;
  static constexpr int fmt = WD_F32;
  float4* p;
  long stride;
  template <class T> __device__ __forceinline__ void loadT(long i, cpx<T> (&s)[12]) const {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      float4 v = __ldg(p + j * stride + i);
      s[2 * j] = {(T)v.x, (T)v.y};
      s[2 * j + 1] = {(T)v.z, (T)v.w};
    }
  }
  template <class T> __device__ __forceinline__ void store(long i, const cpx<T> (&s)[12]) const {
#pragma unroll
    for (int j = 0; j < 6; ++j)
      p[j * stride + i] = make_float4((float)s[2 * j].r, (float)s[2 * j].i, (float)s[2 * j + 1].r,
                                      (float)s[2 * j + 1].i);
  }
  // the stored words of one site, loaded ahead of their use
  struct Raw { float4 v[6]; };
  __device__ __forceinline__ void loadRaw(long i, Raw& r) const {
#pragma unroll
    for (int j = 0; j < 6; ++j) r.v[j] = __ldg(p + j * stride + i);
  }
  template <class T> __device__ __forceinline__ static void unpack(const Raw& r, cpx<T> (&s)[12]) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      s[2 * j] = {(T)r.v[j].x, (T)r.v[j].y};
      s[2 * j + 1] = {(T)r.v[j].z, (T)r.v[j].w};
    }
  }
};

template <class H> struct H16Traits;
template <> struct H16Traits<__half> {
  static constexpr int fmt = WD_F16;
  __device__ __forceinline__ static float to_f(unsigned short u) { return __half2float(__ushort_as_half(u)); }
  __device__ __forceinline__ static unsigned short from_f(float f) { return __half_as_ushort(__float2half_rn(f)); }
};
template <> struct H16Traits<__nv_bfloat16> {
  static constexpr int fmt = WD_BF16;
  __device__ __forceinline__ static float to_f(unsigned short u) { return __bfloat162float(__ushort_as_bfloat16(u)); }
  __device__ __forceinline__ static unsigned short from_f(float f) { return __bfloat16_as_ushort(__float2bfloat16_rn(f)); }
};

template <class H> struct Sp16 {
  using real = float;
  static constexpr int fmt = H16Traits<H>::fmt;
  uint4* p;
  float* nrm;
  long stride;
  template <class T> __device__ __forceinline__ void loadT(long i, cpx<T> (&s)[12]) const {
    const float n = __ldg(nrm + i);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      uint4 v = __ldg(p + j * stride + i);
      unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        s[4 * j + q] = {(T)(n * H16Traits<H>::to_f((unsigned short)(w[q] & 0xffffu))),
                        (T)(n * H16Traits<H>::to_f((unsigned short)(w[q] >> 16)))};
      }
    }
  }
  template <class T> __device__ __forceinline__ void store(long i, const cpx<T> (&s)[12]) const {
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < 12; ++j) m = fmaxf(m, fmaxf(fabsf((float)s[j].r), fabsf((float)s[j].i)));
    const float inv = m > 0.f ? 1.f / m : 0.f;
    nrm[i] = m;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      unsigned w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        unsigned lo = H16Traits<H>::from_f((float)s[4 * j + q].r * inv);
        unsigned hi = H16Traits<H>::from_f((float)s[4 * j + q].i * inv);
        w[q] = lo | (hi << 16);
      }
      p[j * stride + i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
  // the stored words of one site (16-bit values and the norm), loaded ahead of their use
  struct Raw { uint4 v[3]; float n; };
  __device__ __forceinline__ void loadRaw(long i, Raw& r) const {
    r.n = __ldg(nrm + i);
#pragma unroll
    for (int j = 0; j < 3; ++j) r.v[j] = __ldg(p + j * stride + i);
  }
  template <class T> __device__ __forceinline__ static void unpack(const Raw& r, cpx<T> (&s)[12]) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      unsigned w[4] = {r.v[j].x, r.v[j].y, r.v[j].z, r.v[j].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        s[4 * j + q] = {(T)(r.n * H16Traits<H>::to_f((unsigned short)(w[q] & 0xffffu))),
                        (T)(r.n * H16Traits<H>::to_f((unsigned short)(w[q] >> 16)))};
      }
    }
  }
};

// Double-float spinor: float4 [12][Vh], component j = (re.hi, re.lo, im.hi, im.lo);
// 16 bytes per complex like FP64.  Internal format id WD_DD.
constexpr int WD_DD = 4;
template <class T> __device__ __forceinline__ T dd_to(dd v);
template <> __device__ __forceinline__ dd dd_to<dd>(dd v) { return v; }
template <> __device__ __forceinline__ double dd_to<double>(dd v) { return (double)v; }
template <> __device__ __forceinline__ float dd_to<float>(dd v) { return v.hi + v.lo; }
template <class T> __device__ __forceinline__ dd to_dd(T v) { return dd((double)v); }
template <> __device__ __forceinline__ dd to_dd<dd>(dd v) { return v; }
template <> __device__ __forceinline__ dd to_dd<float>(float v) { return dd(v, 0.f); }

struct SpDD {
  using real = dd;
  static constexpr int fmt = WD_DD;
  float4* p;
  long stride;
  template <class T> __device__ __forceinline__ void loadT(long i, cpx<T> (&s)[12]) const {
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      const float4 v = __ldg(p + j * stride + i);
      s[j] = {dd_to<T>(dd(v.x, v.y)), dd_to<T>(dd(v.z, v.w))};
    }
  }
  template <class T> __device__ __forceinline__ void store(long i, const cpx<T> (&s)[12]) const {
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      const dd r = to_dd(s[j].r), m = to_dd(s[j].i);
      p[j * stride + i] = make_float4(r.hi, r.lo, m.hi, m.lo);
    }
  }
};

// ----------------------------------------------------------------------------
// gauge storage formats; load U_mu(x) for site cb of parity par
struct GF64 {
  using real = double;
  const double2* p;
  long stride;
  template <class T> __device__ __forceinline__ void load(int mu, int par, long i, cpx<T> (&U)[9]) const {
    const double2* q = p + ((long)(mu * 2 + par) * 9) * stride + i;
#pragma unroll
    for (int j = 0; j < 9; ++j) { double2 v = __ldg(q + j * stride); U[j] = {(T)v.x, (T)v.y}; }
  }
};
struct GF32 {
  using real = float;
  const float2* p;
  long stride;
  template <class T> __device__ __forceinline__ void load(int mu, int par, long i, cpx<T> (&U)[9]) const {
    const float2* q = p + ((long)(mu * 2 + par) * 9) * stride + i;
#pragma unroll
    for (int j = 0; j < 9; ++j) { float2 v = __ldg(q + j * stride); U[j] = {(T)v.x, (T)v.y}; }
  }
};
// double-float links: float4 [4][2][9][Vh], entry = (re.hi, re.lo, im.hi, im.lo)
struct GDD {
  using real = dd;
  const float4* p;
  long stride;
  template <class T> __device__ __forceinline__ void load(int mu, int par, long i, cpx<T> (&U)[9]) const {
    const float4* q = p + ((long)(mu * 2 + par) * 9) * stride + i;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const float4 v = __ldg(q + j * stride);
      U[j] = {dd_to<T>(dd(v.x, v.y)), dd_to<T>(dd(v.z, v.w))};
    }
  }
};
struct GF32R12 {
  using real = float;
  const float4* p;
  long stride;
  template <class T> __device__ __forceinline__ void load(int mu, int par, long i, cpx<T> (&U)[9]) const {
    const float4* q = p + ((long)(mu * 2 + par) * 3) * stride + i;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float4 v = __ldg(q + j * stride);
      U[2 * j] = {(T)v.x, (T)v.y};
      U[2 * j + 1] = {(T)v.z, (T)v.w};
    }
    // row 2 = (row0 x row1)^*
    U[6] = conj(U[1] * U[5] - U[2] * U[4]);
    U[7] = conj(U[2] * U[3] - U[0] * U[5]);
    U[8] = conj(U[0] * U[4] - U[1] * U[3]);
  }
};

// ----------------------------------------------------------------------------
// deterministic grid reduction: every block writes its partial sums; the last
// block to finish adds them in block order and calls a finisher.
struct Reduce {
  double* partial;      // [gridDim.x * NV]
  unsigned* counter;    // zero before the launch; reset by the last block
  double* out;          // [NV] results
};

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh /* [NV*32] */) {
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k * 32 + wid] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a = lane < nw ? sh[k * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
      v[k] = a;
    }
  }
}

// Returns true in thread 0 of the last block, with tot[] = the grid sums.
template <int NV>
__device__ __forceinline__ bool grid_sum(const Reduce& r, double (&v)[NV], double (&tot)[NV]) {
  __shared__ double sh[NV * 32];
  __shared__ bool last;
  block_sum<NV>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) r.partial[blockIdx.x * NV + k] = v[k];
    __threadfence();
    unsigned prev = atomicAdd(r.counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  // the last block: sum the partials in fixed order, 2-level for determinism
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += __ldcg(r.partial + b * NV + k);
  }
  __syncthreads();
  block_sum<NV>(acc, sh);
  if (threadIdx.x != 0) return false;
#pragma unroll
  for (int k = 0; k < NV; ++k) { tot[k] = acc[k]; r.out[k] = acc[k]; }
  *r.counter = 0u;
  return true;
}

// ----------------------------------------------------------------------------
// Solver state kept on the device so that iterations can be queued without
// host round trips.  Kernels return at once when flag != 0.
enum : int { FLAG_DONE = 1, FLAG_UPDATE = 2, FLAG_NAN = 4, FLAG_MAXITER = 8, FLAG_TIMEOUT = 16 };
struct CGState {
  double rr;        // |r|^2 of the current residual
  double rr_old;    // |r|^2 one iteration earlier
  double pAp;
  double alpha, beta;
  double stop_rr;   // convergence threshold on |r|^2 (sloppy)
  double upd_rr;    // reliable-update threshold on |r|^2
  int flag;
  int iter;
  int maxiter;
  int pad;
};

// ----------------------------------------------------------------------------
// Host-side field handle for internal buffers
struct Field {
  void* data = nullptr;
  float* norm = nullptr;
  int fmt = WD_F64;
  long stride = 0;
};

size_t field_bytes(int fmt, long Vh);

// Timing events of a hop key whose launch shape is being tuned.
struct TuneSamples {
  std::vector<cudaEvent_t> ev;   // (start, stop) per sampled launch
};

// Sampled launch timing of the hop kernels, per input-spinor format.
struct Prof {
  int every = 0;
  long long seen = 0;
  static constexpr int NF = 5;      // FP64, FP32, FP16, BF16, double-float
  long long all[NF] = {0, 0, 0, 0, 0};          // every hop launch, sampled or not
  long long launches[NF] = {0, 0, 0, 0, 0};
  double ms[NF] = {0, 0, 0, 0, 0};
  double bytes[NF] = {0, 0, 0, 0, 0};
  std::vector<cudaEvent_t> ev;   // pairs, pending
  std::vector<double> ev_bytes;
  std::vector<int> ev_fmt;
};

}  // namespace wd

// The context (opaque to C callers)
struct wd_ctx {
  wd::Geom g;
  cudaStream_t stream = nullptr;
  int device = 0;
  int recon = WD_RECON_18;
  bool have_gauge = false;
  // gauge copies
  double2* gauge64 = nullptr;       // [4][2][9][Vh]
  float2* gauge32 = nullptr;        // [4][2][9][Vh]
  float4* gauge32r12 = nullptr;     // [4][2][3][Vh]
  float4* gauge_dd = nullptr;       // double-float copy [4][2][9][Vh] (on demand)
  int resid_dd = 0;                 // residual recomputation in double-float
  double2* gauge_backup = nullptr;  // FP64 links at the start of a trajectory
  double* mom = nullptr;            // momenta of a trajectory [4][2][8][Vh]
  double* lex_stage = nullptr;      // lexicographic FP64 links, staging of host-buffer calls
  // reduction scratch
  double* red_partial = nullptr;
  unsigned* red_counter = nullptr;
  double* red_out = nullptr;        // [16]
  wd::CGState* cgs = nullptr;       // device solver state
  wd::CGState* cgs_host = nullptr;  // pinned mirror
  double* host_scalar = nullptr;    // pinned scratch [16]
  // workspace pool: half-lattice vectors by format
  std::vector<wd::Field> pool;
  std::vector<bool> pool_used;
  long long nmat = 0;
  long long launches = 0;           // kernels launched by the library
  int autotune = 1;                 // time launch shapes on first use
  int stencil = WD_STENCIL_THREAD;  // 12-real-link stencil: per-thread staging or tile-staged bulk copies
  int nsm = 0;                      // multiprocessors of the device
  unsigned* kerr = nullptr;         // device error word: bit 0 = a bounded wait expired
  std::unordered_map<long long, std::pair<int, int>> tune;   // key -> (threads, minb)
  std::unordered_map<long long, wd::TuneSamples> tune_samples;   // keys being tuned
  wd::Prof prof;
};

namespace wd {

// error reporting (thread local message)
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
#define WD_CUDA(call)                                         \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return ::wd::cuda_fail(_e, #call); \
  } while (0)
// after every kernel launch: count it (context `c` in scope) and check it
#define WD_CHECK_LAUNCH()                   \
  do {                                      \
    c->launches += 1;                       \
    WD_CUDA(cudaGetLastError());            \
  } while (0)
#define WD_TRY(expr)                      \
  do {                                    \
    int _s = (expr);                      \
    if (_s != WD_OK) return _s;           \
  } while (0)

// workspace
int ws_get(wd_ctx* c, int fmt, Field* f);   // borrow a half-lattice vector
void ws_put(wd_ctx* c, const Field& f);
struct WsGuard {
  wd_ctx* c;
  std::vector<Field> held;
  explicit WsGuard(wd_ctx* cc) : c(cc) {}
  int get(int fmt, Field* f) {
    int s = ws_get(c, fmt, f);
    if (s == WD_OK) held.push_back(*f);
    return s;
  }
  ~WsGuard() { for (auto& f : held) ws_put(c, f); }
};
Field wrap_f64(wd_ctx* c, const double* p);

inline Reduce reducer(wd_ctx* c) { return Reduce{c->red_partial, c->red_counter, c->red_out}; }
constexpr int RED_MAX_BLOCKS = 1 << 16;

// bounded-wait self-test (dslash_f32.cu)
int wait_selftest(wd_ctx* c, long long ns);

// operator layer (dslash.cu)
// in_cg: the launch belongs to a queued CG iteration and returns at once when
// the solver state carries a stop flag; norm_cg: also form pAp = |out|^2.
int hop(wd_ctx* c, int out_par, bool dag, const Field& in, const Field& out, const Field* y,
        double alpha, bool norm_cg, bool in_cg);
int apply_mhat(wd_ctx* c, double kappa, bool dag, const Field& in, const Field& out, Field& tmp,
               bool norm_cg);
int apply_khat(wd_ctx* c, double kappa, const Field& in, const Field& out, Field& t1, Field& t2,
               bool norm_cg, bool in_cg = false);
double hop_bytes(int fmt_in, int fmt_out, bool xpay, int gauge_bytes_per_link, long Vh);
int khat_poly_step_f32(wd_ctx* c, double kappa, const Field& s, Field& t1, Field& t2, const Field& v,
                       const Field& sprev, double ca, double cmu, double cb, const Field& out);

// blas layer (blas.cu)
int convert(wd_ctx* c, const Field& in, const Field& out);
int axpby(wd_ctx* c, double a, const Field& x, double b, const Field& y, const Field& out);  // out = a x + b y
int caxpby(wd_ctx* c, double ar, double ai, const Field& x, double br, double bi, const Field& y,
           const Field& out);
int zero(wd_ctx* c, const Field& f);
int dot(wd_ctx* c, const Field& a, const Field& b, double* re, double* im);   // host result
int norm2(wd_ctx* c, const Field& a, double* out);                           // host result
int cg_update(wd_ctx* c, const Field& x, const Field& r, const Field& p, const Field& Ap);
int cg_pupdate(wd_ctx* c, const Field& r, const Field& p);
int cg_dot_pap(wd_ctx* c, const Field& p, const Field& Ap);
int poly_step(wd_ctx* c, double a, double mu, double b, const Field& v, const Field& s,
              const Field& Ks, const Field& sprev, const Field& out);
int gamma5(wd_ctx* c, const Field& in, const Field& out);

// solver layer (solver.cu)
int khat_any(wd_ctx* c, double kappa, const Field& in, const Field& out);   // FP64 fields
int poly_apply_f(wd_ctx* c, double kappa, const wd_poly& P, int prec, const Field& in,
                 const Field& out);
// x_zero: start from x = 0 (x is zeroed, the initial residual is b itself)
int cg_solve_f(wd_ctx* c, double kappa, const wd_poly* filt, const Field& b, const Field& x,
               const wd_cg_params& p, wd_cg_info* info, bool x_zero = false);

// kernels of other units
int pack_k(wd_ctx* c, bool unpack, int nouter, int nchunk, int chunk, int parity, const double* src,
           double* dst);
int gauge_lowprec_k(wd_ctx* c);
int gauge_force_k(wd_ctx* c, double beta, int prec, double coef, double* F);
int gauge_action_k(wd_ctx* c, double* S);
int step_T_k(wd_ctx* c, const double* P, double eps);
int step_S_k(wd_ctx* c, double* P, const double* F, double eps);
int kinetic_k(wd_ctx* c, const double* P, double* out);
int gaussian_draw_k(wd_ctx* c, int what, int parity, uint64_t seed, uint64_t stream, double* out);

// force layer (force.cu)
int force_outer(wd_ctx* c, double coef, const Field& Ye, const Field& Yo, const Field& Xe,
                const Field& Xo, double* F, int prec);
int force_outer2(wd_ctx* c, const double coef[2], const Field* Ye, const Field* Yo, const Field* Xe,
                 const Field* Xo, double* F);

// polynomial helpers (host)
struct PolyCoef {
  int n;
  double mu, nu, scale;
  std::vector<double> zr, zi;      // roots z_k, k = 1..n
  std::vector<double> a, b;        // recurrence s_{k+1} = a_k (v + mu s_k - K s_k) - b_k s_{k-1}
  double s1;                       // s_1 = 1/mu
};
int poly_coef(const wd_poly& P, PolyCoef* out);
// Q = P_hi / P_lo in factored form (no recurrence coefficients)
int ratio_coef(const wd_poly& hi, const wd_poly& lo, PolyCoef* out);
// out = Q(K_hat) in from the roots of Q, conjugate pairs as real quadratics;
// in and out of one format (FP64, FP32 or double-float) and distinct
int roots_apply_f(wd_ctx* c, double kappa, const PolyCoef& q, const Field& in, const Field& out);
int cg_solve_ratio(wd_ctx* c, double kappa, const PolyCoef& q, const Field& b, const Field& x,
                   const wd_cg_params& p, wd_cg_info* info);

// launch helpers
inline int nblocks(long n, int threads) { return (int)((n + threads - 1) / threads); }
void prof_begin(wd_ctx* c, cudaEvent_t* e0);
void prof_end(wd_ctx* c, cudaEvent_t e0, double bytes, int fmt);

}  // namespace wd
