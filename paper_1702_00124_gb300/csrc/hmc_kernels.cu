// HMC step kernels (Section 2 of the paper):
//   T[eps]: U -> exp(i eps P) U,   S[eps]: P -> P - eps F,   H = sum tr P^2 + S,
// and the Gaussian draws of momenta (P ~ exp(-sum tr P^2)) and of the heat
// bath noise chi (exp(-chi^dag chi)).
//
// exp(iQ) for Hermitian traceless Q = eps P follows the Cayley-Hamilton
// closed form of Morningstar and Peardon (Phys. Rev. D 69 (2004) 054501,
// Section III): exp(iQ) = f0 + f1 Q + f2 Q^2 with the f_j from
// c0 = det Q, c1 = tr Q^2 / 2; negative c0 is mapped to positive c0 by the
// symmetry f_j(-c0) = (-1)^j conj(f_j(c0)), which keeps the denominator
// 9u^2 - w^2 away from zero.  The product is reunitarised (Gram-Schmidt on
// rows 0 and 1, row 2 = (r0 x r1)^*) and written to the FP64 links and to
// both FP32 link copies in the same pass.
//
// Random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) with key
// (seed, 0) and counter (j, stream, 0, 0); the four words of block j give
// u_k = ((x_k >> 11) + 1/2) 2^-53 and two Box-Muller pairs, which are the
// Gaussian reals 4j..4j+3 of the field in its lexicographic real order.
#include <cmath>

#include "dslash_impl.cuh"

namespace wd {

constexpr int H_THREADS = 128;

// cos x and sin(x)/x from y = -x^2 by their Taylor series through x^14; for
// |x| <= 0.5 the first omitted terms are below 1e-18.
__device__ __forceinline__ double cos_series(double y) {
  double t = 1.0 / 87178291200.0;              // 1/14!
  t = fma(t, y, 1.0 / 479001600.0);            // 1/12!
  t = fma(t, y, 1.0 / 3628800.0);
  t = fma(t, y, 1.0 / 40320.0);
  t = fma(t, y, 1.0 / 720.0);
  t = fma(t, y, 1.0 / 24.0);
  t = fma(t, y, 0.5);
  return fma(t, y, 1.0);
}
__device__ __forceinline__ double sinc_series(double y) {
  double t = 1.0 / 1307674368000.0;            // 1/15!
  t = fma(t, y, 1.0 / 6227020800.0);           // 1/13!
  t = fma(t, y, 1.0 / 39916800.0);
  t = fma(t, y, 1.0 / 362880.0);
  t = fma(t, y, 1.0 / 5040.0);
  t = fma(t, y, 1.0 / 120.0);
  t = fma(t, y, 1.0 / 6.0);
  return fma(t, y, 1.0);
}

// Q is Hermitian and traceless: Q2 = Q^2 is Hermitian, so its diagonal is
// real and its lower triangle the conjugate of the upper one.
__device__ __forceinline__ void cayley_hamilton_exp(const cpx<double> (&Q)[9], cpx<double> (&E)[9]) {
  const double q00 = Q[0].r, q11 = Q[4].r, q22 = Q[8].r;
  const cpx<double> q01 = Q[1], q02 = Q[2], q12 = Q[5];
  const double n01 = norm2(q01), n02 = norm2(q02), n12 = norm2(q12);
  cpx<double> Q2[9];
  Q2[0] = mk(q00 * q00 + n01 + n02, 0.0);
  Q2[4] = mk(q11 * q11 + n01 + n12, 0.0);
  Q2[8] = mk(q22 * q22 + n02 + n12, 0.0);
  Q2[1] = (q00 + q11) * q01 + q02 * conj(q12);
  Q2[2] = (q00 + q22) * q02 + q01 * q12;
  Q2[5] = (q11 + q22) * q12 + conj(q01) * q02;
  Q2[3] = conj(Q2[1]);
  Q2[6] = conj(Q2[2]);
  Q2[7] = conj(Q2[5]);
  const double c1 = 0.5 * (Q2[0].r + Q2[4].r + Q2[8].r);
  // c0 = det Q = q00 q11 q22 + 2 Re(q01 q12 q02^*) - q00 |q12|^2 - q11 |q02|^2 - q22 |q01|^2
  const double c0 = q00 * q11 * q22 + 2.0 * (q01 * q12 * conj(q02)).r - q00 * n12 - q11 * n02 - q22 * n01;
  cpx<double> f0, f1, f2;
  if (c1 < 1e-24) {
    f0 = mk(1.0, 0.0);
    f1 = mk(0.0, 1.0);
    f2 = mk(-0.5, 0.0);
  } else {
    const bool neg = c0 < 0;
    const double c0a = fabs(c0);
    const double t3 = c1 / 3.0;
    const double st3 = sqrt(t3);                   // sqrt(c1/3)
    const double c0max = 2.0 * t3 * st3;           // 2 (c1/3)^{3/2}
    double r = c0a / c0max;
    r = r > 1.0 ? 1.0 : r;
    // cs = cos(th/3), th = acos(r) in [0, pi/2]: the root of 4 cs^3 - 3 cs = r
    // in [cos(pi/6), 1], where the derivative 12 cs^2 - 3 lies in [6, 9]; an
    // FP32 seed and two Newton steps in FP64
    double cs = (double)cosf(acosf((float)r) * (1.0f / 3.0f));
#pragma unroll
    for (int it = 0; it < 2; ++it) cs -= (cs * (4.0 * cs * cs - 3.0) - r) / (12.0 * cs * cs - 3.0);
    const double u = st3 * cs;
    const double u2 = u * u;
    const double w2 = c1 * (1.0 - cs) * (1.0 + cs);  // w = sqrt(c1) sin(th/3)
    double cw, xi0, cu, su;
    if (w2 <= 0.25) {
      cw = cos_series(-w2);
      xi0 = sinc_series(-w2);
    } else {
      const double w = sqrt(w2);
      double sw;
      sincos(w, &sw, &cw);
      xi0 = sw / w;
    }
    if (u2 <= 0.25) {
      cu = cos_series(-u2);
      su = u * sinc_series(-u2);
    } else {
      sincos(u, &su, &cu);
    }
    const cpx<double> e2 = mk(cu * cu - su * su, 2.0 * su * cu);   // exp(2iu)
    const cpx<double> em = mk(cu, -su);                              // exp(-iu)
    const cpx<double> h0 = (u2 - w2) * e2 + em * mk(8 * u2 * cw, 2 * u * (3 * u2 + w2) * xi0);
    const cpx<double> h1 = (2 * u) * e2 - em * mk(2 * u * cw, -(3 * u2 - w2) * xi0);
    const cpx<double> h2 = e2 - em * mk(cw, 3 * u * xi0);
    const double den = 1.0 / (9 * u2 - w2);
    f0 = den * h0;
    f1 = den * h1;
    f2 = den * h2;
    if (neg) {
      f0 = conj(f0);
      f1 = mk(-f1.r, f1.i);
      f2 = conj(f2);
    }
  }
#pragma unroll
  for (int j = 0; j < 9; ++j) E[j] = f1 * Q[j] + f2 * Q2[j];
  E[0] = E[0] + f0;
  E[4] = E[4] + f0;
  E[8] = E[8] + f0;
}

__device__ __forceinline__ void reunitarize(cpx<double> (&U)[9]) {
  double n0 = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j) n0 += norm2(U[j]);
  n0 = 1.0 / sqrt(n0);
#pragma unroll
  for (int j = 0; j < 3; ++j) U[j] = n0 * U[j];
  cpx<double> d = mk(0.0, 0.0);
#pragma unroll
  for (int j = 0; j < 3; ++j) d = d + cmulc(U[j], U[3 + j]);
#pragma unroll
  for (int j = 0; j < 3; ++j) U[3 + j] = U[3 + j] - d * U[j];
  double n1 = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j) n1 += norm2(U[3 + j]);
  n1 = 1.0 / sqrt(n1);
#pragma unroll
  for (int j = 0; j < 3; ++j) U[3 + j] = n1 * U[3 + j];
  U[6] = conj(U[1] * U[5] - U[2] * U[4]);
  U[7] = conj(U[2] * U[3] - U[0] * U[5]);
  U[8] = conj(U[0] * U[4] - U[1] * U[3]);
}

// Hermitian traceless matrix from algebra coordinates: sum_a p_a lambda_a / 2
__device__ __forceinline__ void alg_matrix(const double (&p)[8], double s, cpx<double> (&Q)[9]) {
  const double h = 0.5 * s;
  const double r3 = 0.57735026918962576451;
  Q[0] = mk(h * (p[2] + r3 * p[7]), 0.0);
  Q[4] = mk(h * (-p[2] + r3 * p[7]), 0.0);
  Q[8] = mk(h * (-2.0 * r3 * p[7]), 0.0);
  Q[1] = mk(h * p[0], -h * p[1]);
  Q[3] = mk(h * p[0], h * p[1]);
  Q[2] = mk(h * p[3], -h * p[4]);
  Q[6] = mk(h * p[3], h * p[4]);
  Q[5] = mk(h * p[5], -h * p[6]);
  Q[7] = mk(h * p[5], h * p[6]);
}

__global__ void __launch_bounds__(H_THREADS) k_step_T(Geom g, const double* P, double eps, double2* U64,
                                                      float2* U32, float4* U12, float4* Udd) {
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= 8 * g.Vh) return;
  const long cb = tid % g.Vh;
  const int mp = (int)(tid / g.Vh);   // mu * 2 + parity
  double p[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) p[a] = P[((long)mp * 8 + a) * g.Vh + cb];
  cpx<double> Q[9], E[9], U[9], V[9];
  alg_matrix(p, eps, Q);
  cayley_hamilton_exp(Q, E);
  double2* u = U64 + (long)mp * 9 * g.Vh + cb;
#pragma unroll
  for (int j = 0; j < 9; ++j) { double2 v = u[j * g.Vh]; U[j] = mk(v.x, v.y); }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) V[3 * i + j] = E[3 * i] * U[j] + E[3 * i + 1] * U[3 + j] + E[3 * i + 2] * U[6 + j];
  reunitarize(V);
#pragma unroll
  for (int j = 0; j < 9; ++j) u[j * g.Vh] = make_double2(V[j].r, V[j].i);
  float2* v32 = U32 + (long)mp * 9 * g.Vh + cb;
#pragma unroll
  for (int j = 0; j < 9; ++j) v32[j * g.Vh] = make_float2((float)V[j].r, (float)V[j].i);
  float4* v12 = U12 + (long)mp * 3 * g.Vh + cb;
#pragma unroll
  for (int j = 0; j < 3; ++j)
    v12[j * g.Vh] = make_float4((float)V[2 * j].r, (float)V[2 * j].i, (float)V[2 * j + 1].r, (float)V[2 * j + 1].i);
  if (Udd != nullptr) {
    float4* vd = Udd + (long)mp * 9 * g.Vh + cb;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const dd r(V[j].r), m(V[j].i);
      vd[j * g.Vh] = make_float4(r.hi, r.lo, m.hi, m.lo);
    }
  }
}

int step_T_k(wd_ctx* c, const double* P, double eps) {
  const long n = 8 * c->g.Vh;
  k_step_T<<<nblocks(n, H_THREADS), H_THREADS, 0, c->stream>>>(c->g, P, eps, c->gauge64, c->gauge32,
                                                                c->gauge32r12, c->gauge_dd);
  WD_CHECK_LAUNCH();
  return WD_OK;
}

__global__ void k_axpy_alg(long n, double a, const double* x, double* y) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

int step_S_k(wd_ctx* c, double* P, const double* F, double eps) {
  const long n = 64 * c->g.Vh;   // 4 mu x 2 parities x 8 coordinates
  k_axpy_alg<<<nblocks(n, 256), 256, 0, c->stream>>>(n, -eps, F, P);
  WD_CHECK_LAUNCH();
  return WD_OK;
}

__global__ void __launch_bounds__(256) k_sumsq(long n, const double* x, Reduce red) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  // 8 consecutive values per thread keeps the block count small
  for (int q = 0; q < 8; ++q) {
    const long k = i * 8 + q;
    if (k < n) v[0] += x[k] * x[k];
  }
  double tot[1];
  grid_sum<1>(red, v, tot);
}

int kinetic_k(wd_ctx* c, const double* P, double* out) {
  const long n = 64 * c->g.Vh;
  const int nb = nblocks((n + 7) / 8, 256);
  if (nb > RED_MAX_BLOCKS) return fail(WD_ERR_ARG, "kinetic: lattice too large");
  k_sumsq<<<nb, 256, 0, c->stream>>>(n, P, reducer(c));
  WD_CHECK_LAUNCH();
  WD_CUDA(cudaMemcpyAsync(c->host_scalar, c->red_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  *out = 0.5 * c->host_scalar[0];
  return WD_OK;
}

// ----------------------------------------------------------------------------
// Philox4x64-10
__device__ __forceinline__ void philox4x64(uint64_t (&x)[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint64_t hi0 = __umul64hi(M0, x[0]), lo0 = M0 * x[0];
    const uint64_t hi1 = __umul64hi(M1, x[2]), lo1 = M1 * x[2];
    const uint64_t n0 = hi1 ^ x[1] ^ k0, n2 = hi0 ^ x[3] ^ k1;
    x[0] = n0; x[1] = lo1; x[2] = n2; x[3] = lo0;
  }
}

__device__ __forceinline__ void gauss4(uint64_t j, uint64_t seed, uint64_t stream, double (&g)[4]) {
  uint64_t x[4] = {j, stream, 0ull, 0ull};
  philox4x64(x, seed, 0ull);
  double u[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) u[k] = ((double)(x[k] >> 11) + 0.5) * 0x1.0p-53;
  const double r0 = sqrt(-2.0 * log(u[0])), r2 = sqrt(-2.0 * log(u[2]));
  const double two_pi = 6.283185307179586232;
  g[0] = r0 * cos(two_pi * u[1]);
  g[1] = r0 * sin(two_pi * u[1]);
  g[2] = r2 * cos(two_pi * u[3]);
  g[3] = r2 * sin(two_pi * u[3]);
}

// spinor: lexicographic reals e = (lex * 12 + comp) * 2 + re/im; a block holds
// reals 4j..4j+3 = complex components 2q, 2q+1 of one site (q = j mod 6)
__global__ void k_draw_spinor(Geom g, int parity, uint64_t seed, uint64_t stream, double2* out) {
  const long j = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= 6 * g.V) return;
  const long lex = j / 6;
  const int q = (int)(j % 6);
  const int x = (int)(lex % g.L[0]);
  long r = lex / g.L[0];
  const int y = (int)(r % g.L[1]); r /= g.L[1];
  const int z = (int)(r % g.L[2]);
  const int t = (int)(r / g.L[2]);
  if (((x + y + z + t) & 1) != parity) return;
  double v[4];
  gauss4((uint64_t)j, seed, stream, v);
  const long cb = lex >> 1;
  out[(2 * q) * g.Vh + cb] = make_double2(v[0], v[1]);
  out[(2 * q + 1) * g.Vh + cb] = make_double2(v[2], v[3]);
}

// algebra: lexicographic reals e = (lex * 4 + mu) * 8 + a; block j covers
// coordinates 4h..4h+3 (h = j mod 2) of link (lex, mu)
__global__ void k_draw_alg(Geom g, uint64_t seed, uint64_t stream, double* out) {
  const long j = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= 8 * g.V) return;
  const int h = (int)(j & 1);
  const long lm = j >> 1;
  const int mu = (int)(lm & 3);
  const long lex = lm >> 2;
  const int x = (int)(lex % g.L[0]);
  long r = lex / g.L[0];
  const int y = (int)(r % g.L[1]); r /= g.L[1];
  const int z = (int)(r % g.L[2]);
  const int t = (int)(r / g.L[2]);
  const int par = (x + y + z + t) & 1;
  const long cb = lex >> 1;
  double v[4];
  gauss4((uint64_t)j, seed, stream, v);
#pragma unroll
  for (int k = 0; k < 4; ++k) out[((long)(mu * 2 + par) * 8 + 4 * h + k) * g.Vh + cb] = v[k];
}

int gaussian_draw_k(wd_ctx* c, int what, int parity, uint64_t seed, uint64_t stream, double* out) {
  if (what == 0) {
    const long n = 6 * c->g.V;
    k_draw_spinor<<<nblocks(n, 256), 256, 0, c->stream>>>(c->g, parity, seed, stream, (double2*)out);
  } else {
    const long n = 8 * c->g.V;
    k_draw_alg<<<nblocks(n, 256), 256, 0, c->stream>>>(c->g, seed, stream, out);
  }
  WD_CHECK_LAUNCH();
  return WD_OK;
}

}  // namespace wd
