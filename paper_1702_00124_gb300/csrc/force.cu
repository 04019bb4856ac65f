// Force kernels.
//
// Fermion force (Section 2 of the paper: dS_F/dU = -phi^dag K^-1 (dK/dU) K^-1 phi).
// Convention: F_a(x,mu) = dS/dw for U_mu(x) -> exp(i w T_a) U_mu(x), stored as
// algebra coordinates [mu][parity][a][cb].  For full-lattice fields Y, X the
// per-link derivative of Re(Y^dag D X) is
//     Re(i tr(T_a W)) = -1/2 Im tr(lambda_a W),  W = U A1 - A2 U^dag,
//     A1 = sum_s [(1 - g_mu) X(x+mu)]_s Y_s(x)^dag,
//     A2 = sum_s [(1 + g_mu) X(x)]_s Y_s(x+mu)^dag,
// with the fermion sign on links across the time boundary.  Because the
// projector (1 + s g) has rank 2, sum_s [(1+s g)X]_s Y_s^dag equals
// sum_{a=0,1} h_a(X) h_a(Y)^dag with h the half spinor of the same projector,
// so each A is two 3x3 outer products.  The kernel adds coef times this to F.
//
// Gauge force: S_G = beta sum_{x, mu<nu} (1 - Re tr U_munu / 3) (the workload's
// Wilson plaquette action; the paper names S_G only), whose derivative is
// -(beta/3) Re(i tr(T_a U_mu(x) A_mu(x))) with A the sum of the six staples.
#include "dslash_impl.cuh"

namespace wd {

constexpr int F_THREADS = 128;

template <class T>
__device__ __forceinline__ void proj_ta(const cpx<T> (&W)[9], T (&f)[8]) {
  // f_a = -1/2 Im tr(lambda_a W); W[3*i+j] = W_ij
  const T h = (T)0.5;
  f[0] = -h * (W[3].i + W[1].i);
  f[1] = -h * (W[1].r - W[3].r);
  f[2] = -h * (W[0].i - W[4].i);
  f[3] = -h * (W[6].i + W[2].i);
  f[4] = -h * (W[2].r - W[6].r);
  f[5] = -h * (W[7].i + W[5].i);
  f[6] = -h * (W[5].r - W[7].r);
  f[7] = -h * (W[0].i + W[4].i - (T)2 * W[8].i) * (T)0.57735026918962576451;
}

template <class T>
__device__ __forceinline__ void mat_mul(const cpx<T> (&A)[9], const cpx<T> (&B)[9], cpx<T> (&C)[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}
// C = A B^dag
template <class T>
__device__ __forceinline__ void mat_mul_nd(const cpx<T> (&A)[9], const cpx<T> (&B)[9], cpx<T> (&C)[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = A[3 * i] * conj(B[3 * j]) + A[3 * i + 1] * conj(B[3 * j + 1]) + A[3 * i + 2] * conj(B[3 * j + 2]);
}
// C = A^dag B
template <class T>
__device__ __forceinline__ void mat_mul_dn(const cpx<T> (&A)[9], const cpx<T> (&B)[9], cpx<T> (&C)[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[3 * i + j] = cmulc(A[i], B[j]) + cmulc(A[3 + i], B[3 + j]) + cmulc(A[6 + i], B[6 + j]);
}

// h_a(X) for the projector (1 + SG g_mu): 2 x 3 complex
template <int MU, int SG, class T>
__device__ __forceinline__ void half_of(const cpx<T> (&s)[12], cpx<T> (&h)[6]) {
  spin_project<MU, SG>(s, h);
}

// A += sum_a h_a k_a^dag
template <class T>
__device__ __forceinline__ void outer_acc(cpx<T> (&A)[9], const cpx<T> (&h)[6], const cpx<T> (&k)[6]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) A[3 * i + j] = A[3 * i + j] + h[i] * conj(k[j]) + h[3 + i] * conj(k[3 + j]);
}

template <class S, class G>
struct ForceArgs {
  Geom g;
  S Ye, Yo, Xe, Xo;
  G gauge;
  double coef;
  double* F;   // [4][2][8][Vh]
};

template <int MU, class T, class S, class G>
__device__ __forceinline__ void force_dir(const ForceArgs<S, G>& a, int par, long cb, const int (&c)[4],
                                          const cpx<T> (&Xs)[12], const cpx<T> (&Ys)[12]) {
  const Geom& g = a.g;
  int n[4] = {c[0], c[1], c[2], c[3]};
  n[MU] = (n[MU] + 1 == g.L[MU]) ? 0 : n[MU] + 1;
  const long nb = g.cb_of(n[0], n[1], n[2], n[3]);
  cpx<T> Xn[12], Yn[12];
  (par ? a.Xe : a.Xo).loadT(nb, Xn);
  (par ? a.Ye : a.Yo).loadT(nb, Yn);
  cpx<T> A1[9], A2[9], h[6], k[6];
#pragma unroll
  for (int j = 0; j < 9; ++j) { A1[j] = mk<T>(0, 0); A2[j] = mk<T>(0, 0); }
  half_of<MU, -1>(Xn, h);
  half_of<MU, -1>(Ys, k);
  outer_acc(A1, h, k);
  half_of<MU, +1>(Xs, h);
  half_of<MU, +1>(Yn, k);
  outer_acc(A2, h, k);
  cpx<T> U[9], W[9], t[9];
  a.gauge.load(MU, par, cb, U);
  mat_mul(U, A1, W);
  mat_mul_nd(A2, U, t);
  const T bc = (MU == 3 && c[3] == g.L[3] - 1) ? (T)-1 : (T)1;
#pragma unroll
  for (int j = 0; j < 9; ++j) W[j] = bc * (W[j] - t[j]);
  T f[8];
  proj_ta(W, f);
  double* F = a.F + ((long)(MU * 2 + par) * 8) * g.Vh + cb;
#pragma unroll
  for (int q = 0; q < 8; ++q) F[q * g.Vh] += a.coef * (double)f[q];
}

template <class T, class S, class G>
__global__ void __launch_bounds__(F_THREADS) k_force(ForceArgs<S, G> a) {
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= 2 * a.g.Vh) return;
  const int par = (int)(tid / a.g.Vh);
  const long cb = tid - par * a.g.Vh;
  int c[4];
  a.g.coords(cb, par, c);
  cpx<T> Xs[12], Ys[12];
  (par ? a.Xo : a.Xe).loadT(cb, Xs);
  (par ? a.Yo : a.Ye).loadT(cb, Ys);
  force_dir<0, T>(a, par, cb, c, Xs, Ys);
  force_dir<1, T>(a, par, cb, c, Xs, Ys);
  force_dir<2, T>(a, par, cb, c, Xs, Ys);
  force_dir<3, T>(a, par, cb, c, Xs, Ys);
}

int force_outer(wd_ctx* c, double coef, const Field& Ye, const Field& Yo, const Field& Xe,
                const Field& Xo, double* F, int prec) {
  const int nb = nblocks(2 * c->g.Vh, F_THREADS);
  if (Ye.fmt != Yo.fmt || Ye.fmt != Xe.fmt || Ye.fmt != Xo.fmt) return fail(WD_ERR_ARG, "force: formats differ");
  if (Ye.fmt == WD_F64 && prec == WD_F64) {
    ForceArgs<SpF64, GF64> a{c->g, sp64(Ye), sp64(Yo), sp64(Xe), sp64(Xo), GF64{c->gauge64, c->g.Vh}, coef, F};
    k_force<double><<<nb, F_THREADS, 0, c->stream>>>(a);
  } else if (Ye.fmt == WD_F32) {
    ForceArgs<SpF32, GF32> a{c->g, sp32(Ye), sp32(Yo), sp32(Xe), sp32(Xo), GF32{c->gauge32, c->g.Vh}, coef, F};
    k_force<float><<<nb, F_THREADS, 0, c->stream>>>(a);
  } else {
    return fail(WD_ERR_ARG, "force: fields must be FP64 (prec FP64) or FP32");
  }
  WD_CHECK_LAUNCH();
  return WD_OK;
}

// Two (Y, X) pairs in one pass: F += coef0 * dRe(Y0^dag D X0) + coef1 * dRe(Y1^dag D X1),
// so the links and F are read and written once for both (the polynomial-term force
// has two pairs per factor).
template <class S, class G>
struct ForceArgs2 {
  Geom g;
  S Ye[2], Yo[2], Xe[2], Xo[2];
  G gauge;
  double coef[2];
  double* F;
};

template <int MU, class T, class S, class G>
__device__ __forceinline__ void force_dir2(const ForceArgs2<S, G>& a, int par, long cb, const int (&c)[4]) {
  const Geom& g = a.g;
  int n[4] = {c[0], c[1], c[2], c[3]};
  n[MU] = (n[MU] + 1 == g.L[MU]) ? 0 : n[MU] + 1;
  const long nb = g.cb_of(n[0], n[1], n[2], n[3]);
  cpx<T> U[9];
  a.gauge.load(MU, par, cb, U);
  const T bc = (MU == 3 && c[3] == g.L[3] - 1) ? (T)-1 : (T)1;
  double fs[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    cpx<T> Xs[12], Ys[12], Xn[12], Yn[12];
    (par ? a.Xo[p] : a.Xe[p]).loadT(cb, Xs);
    (par ? a.Yo[p] : a.Ye[p]).loadT(cb, Ys);
    (par ? a.Xe[p] : a.Xo[p]).loadT(nb, Xn);
    (par ? a.Ye[p] : a.Yo[p]).loadT(nb, Yn);
    cpx<T> A1[9], A2[9], h[6], k[6];
#pragma unroll
    for (int j = 0; j < 9; ++j) { A1[j] = mk<T>(0, 0); A2[j] = mk<T>(0, 0); }
    half_of<MU, -1>(Xn, h);
    half_of<MU, -1>(Ys, k);
    outer_acc(A1, h, k);
    half_of<MU, +1>(Xs, h);
    half_of<MU, +1>(Yn, k);
    outer_acc(A2, h, k);
    cpx<T> W[9], t[9];
    mat_mul(U, A1, W);
    mat_mul_nd(A2, U, t);
#pragma unroll
    for (int j = 0; j < 9; ++j) W[j] = bc * (W[j] - t[j]);
    T f[8];
    proj_ta(W, f);
#pragma unroll
    for (int q = 0; q < 8; ++q) fs[q] += a.coef[p] * (double)f[q];
  }
  double* F = a.F + ((long)(MU * 2 + par) * 8) * g.Vh + cb;
#pragma unroll
  for (int q = 0; q < 8; ++q) F[q * g.Vh] += fs[q];
}

template <class T, class S, class G>
__global__ void __launch_bounds__(F_THREADS) k_force2(ForceArgs2<S, G> a) {
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= 2 * a.g.Vh) return;
  const int par = (int)(tid / a.g.Vh);
  const long cb = tid - par * a.g.Vh;
  int c[4];
  a.g.coords(cb, par, c);
  force_dir2<0, T>(a, par, cb, c);
  force_dir2<1, T>(a, par, cb, c);
  force_dir2<2, T>(a, par, cb, c);
  force_dir2<3, T>(a, par, cb, c);
}

int force_outer2(wd_ctx* c, const double coef[2], const Field* Ye, const Field* Yo, const Field* Xe,
                 const Field* Xo, double* F) {
  const int nb = nblocks(2 * c->g.Vh, F_THREADS);
  const int f = Ye[0].fmt;
  for (int p = 0; p < 2; ++p)
    if (Ye[p].fmt != f || Yo[p].fmt != f || Xe[p].fmt != f || Xo[p].fmt != f)
      return fail(WD_ERR_ARG, "force2: formats differ");
  if (f == WD_F64) {
    ForceArgs2<SpF64, GF64> a{c->g, {sp64(Ye[0]), sp64(Ye[1])}, {sp64(Yo[0]), sp64(Yo[1])},
                              {sp64(Xe[0]), sp64(Xe[1])}, {sp64(Xo[0]), sp64(Xo[1])},
                              GF64{c->gauge64, c->g.Vh}, {coef[0], coef[1]}, F};
    k_force2<double><<<nb, F_THREADS, 0, c->stream>>>(a);
  } else if (f == WD_F32) {
    ForceArgs2<SpF32, GF32> a{c->g, {sp32(Ye[0]), sp32(Ye[1])}, {sp32(Yo[0]), sp32(Yo[1])},
                              {sp32(Xe[0]), sp32(Xe[1])}, {sp32(Xo[0]), sp32(Xo[1])},
                              GF32{c->gauge32, c->g.Vh}, {coef[0], coef[1]}, F};
    k_force2<float><<<nb, F_THREADS, 0, c->stream>>>(a);
  } else {
    return fail(WD_ERR_ARG, "force2: fields must be FP64 or FP32");
  }
  WD_CHECK_LAUNCH();
  return WD_OK;
}

// ----------------------------------------------------------------------------
// gauge action and force
template <class T, class G>
__device__ __forceinline__ void link_at(const Geom& g, const G& gauge, int mu, const int (&c)[4], cpx<T> (&U)[9]) {
  const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
  gauge.load(mu, par, g.cb_of(c[0], c[1], c[2], c[3]), U);
}

__device__ __forceinline__ void step(const Geom& g, int (&c)[4], int mu, int d) {
  int v = c[mu] + d;
  c[mu] = v < 0 ? v + g.L[mu] : (v >= g.L[mu] ? v - g.L[mu] : v);
}

template <class T, class G>
__global__ void __launch_bounds__(F_THREADS) k_gauge_force(Geom g, G gauge, double coef, double* F) {
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= 2 * g.Vh) return;
  const int par = (int)(tid / g.Vh);
  const long cb = tid - par * g.Vh;
  int c[4];
  g.coords(cb, par, c);
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    cpx<T> A[9], t1[9], t2[9], t3[9], Ua[9], Ub[9], Uc[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) A[j] = mk<T>(0, 0);
#pragma unroll 1
    for (int nu = 0; nu < 4; ++nu) {
      if (nu == mu) continue;
      // upper staple U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
      int p[4] = {c[0], c[1], c[2], c[3]};
      step(g, p, mu, +1);
      link_at<T>(g, gauge, nu, p, Ua);
      int q[4] = {c[0], c[1], c[2], c[3]};
      step(g, q, nu, +1);
      link_at<T>(g, gauge, mu, q, Ub);
      link_at<T>(g, gauge, nu, c, Uc);
      mat_mul_nd(Ua, Ub, t1);
      mat_mul_nd(t1, Uc, t2);
#pragma unroll
      for (int j = 0; j < 9; ++j) A[j] = A[j] + t2[j];
      // lower staple U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
      int r[4] = {c[0], c[1], c[2], c[3]};
      step(g, r, nu, -1);
      int s[4] = {r[0], r[1], r[2], r[3]};
      step(g, s, mu, +1);
      link_at<T>(g, gauge, nu, s, Ua);
      link_at<T>(g, gauge, mu, r, Ub);
      link_at<T>(g, gauge, nu, r, Uc);
      mat_mul(Ub, Ua, t1);              // U_mu(x-nu) U_nu(x+mu-nu)
      mat_mul_dn(t1, Uc, t3);           // (U_mu U_nu')^dag U_nu(x-nu)
#pragma unroll
      for (int j = 0; j < 9; ++j) A[j] = A[j] + t3[j];
    }
    cpx<T> U[9], W[9];
    gauge.load(mu, par, cb, U);
    mat_mul(U, A, W);
    T f[8];
    proj_ta(W, f);
    double* Fp = F + ((long)(mu * 2 + par) * 8) * g.Vh + cb;
#pragma unroll
    for (int a = 0; a < 8; ++a) Fp[a * g.Vh] += coef * (double)f[a];
  }
}

int gauge_force_k(wd_ctx* c, double beta, int prec, double coef, double* F) {
  const int nb = nblocks(2 * c->g.Vh, F_THREADS);
  const double k = -coef * beta / 3.0;
  if (prec == WD_F64) k_gauge_force<double><<<nb, F_THREADS, 0, c->stream>>>(c->g, GF64{c->gauge64, c->g.Vh}, k, F);
  else k_gauge_force<float><<<nb, F_THREADS, 0, c->stream>>>(c->g, GF32{c->gauge32, c->g.Vh}, k, F);
  WD_CHECK_LAUNCH();
  return WD_OK;
}

template <class G>
__global__ void __launch_bounds__(F_THREADS) k_gauge_action(Geom g, G gauge, Reduce red) {
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (tid < 2 * g.Vh) {
    const int par = (int)(tid / g.Vh);
    const long cb = tid - par * g.Vh;
    int c[4];
    g.coords(cb, par, c);
    for (int mu = 0; mu < 4; ++mu) {
      for (int nu = mu + 1; nu < 4; ++nu) {
        cpx<double> Um[9], Un[9], Umn[9], Unm[9], t1[9], t2[9];
        link_at<double>(g, gauge, mu, c, Um);
        int p[4] = {c[0], c[1], c[2], c[3]};
        step(g, p, mu, +1);
        link_at<double>(g, gauge, nu, p, Un);      // U_nu(x+mu)
        int q[4] = {c[0], c[1], c[2], c[3]};
        step(g, q, nu, +1);
        link_at<double>(g, gauge, mu, q, Umn);     // U_mu(x+nu)
        link_at<double>(g, gauge, nu, c, Unm);     // U_nu(x)
        mat_mul(Um, Un, t1);
        mat_mul_nd(t1, Umn, t2);
        // Re tr(t2 Unm^dag)
        double tr = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) tr += t2[3 * i + j].r * Unm[3 * i + j].r + t2[3 * i + j].i * Unm[3 * i + j].i;
        v[0] += 1.0 - tr / 3.0;
      }
    }
  }
  double tot[1];
  grid_sum<1>(red, v, tot);
}

int gauge_action_k(wd_ctx* c, double* S) {
  const int nb = nblocks(2 * c->g.Vh, F_THREADS);
  if (nb > RED_MAX_BLOCKS) return fail(WD_ERR_ARG, "gauge action: lattice too large");
  k_gauge_action<<<nb, F_THREADS, 0, c->stream>>>(c->g, GF64{c->gauge64, c->g.Vh}, reducer(c));
  WD_CHECK_LAUNCH();
  WD_CUDA(cudaMemcpyAsync(c->host_scalar, c->red_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  *S = c->host_scalar[0];
  return WD_OK;
}

}  // namespace wd
