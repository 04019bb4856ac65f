// Double-float instantiation of the hopping stencil: spinors and links in
// double-float storage (16 bytes per complex, like FP64), arithmetic by
// error-free transformations on the FP32 pipes (about 44-48 significant bits).
//
// Arithmetic: the SU(3) x half-spinor products use the compensated dot
// product of Ogita, Rump and Oishi (2005, "Dot2") instead of one normalised
// double-float operation per step: each real component of U h is a sum of
// six products, each product is split exactly by an FMA (two-product, with
// the cross terms of the low words), the high words are summed exactly
// (two-sum) and every rounding error is added into one FP32 word.  The site's
// accumulator keeps that unnormalised form across its directions and is
// normalised once, before the store.  Links are read one row (column, for
// U^dag) at a time, where they are used, to keep the live register set small.
//
// One hop is DD_DIRS_PER_LAUNCH directions per launch (forward and backward
// hop each): the first launch writes the output, later ones add to it, the
// last applies the y + alpha D x epilogue.  All eight directions in one kernel
// overflow the instruction cache ("no instruction" stalls in ncu, 1.24 ms per
// hop at 32^3 x 64); one direction per launch re-reads and re-writes the
// partial sum three times (0.77 ms); two directions per launch took 0.60 ms,
// and 0.58 ms with the register cap of four 128-thread blocks per SM (a few
// bytes of spill in the last launch).
#include "dslash_impl.cuh"

namespace wd {

constexpr int DD_DIRS_PER_LAUNCH = 2;

// value s + c with c the collected rounding errors (not normalised)
struct lz {
  float s, c;
};
struct lzc {
  lz r, i;
};

// a += p + e for FP32 p and e: two-sum of the high words, e and the sum's
// error go to the low word
__device__ __forceinline__ void lz_add(lz& a, float p, float e) {
  const float t = a.s + p;
  const float z = t - a.s;
  a.c += ((a.s - (t - z)) + (p - z)) + e;
  a.s = t;
}
// exact product split of x y: p + e, e including the low-word cross terms
__device__ __forceinline__ void two_prod(dd x, dd y, float& p, float& e) {
  p = x.hi * y.hi;
  e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
}
__device__ __forceinline__ void lz_fma(lz& a, dd x, dd y) {
  float p, e;
  two_prod(x, y, p, e);
  lz_add(a, p, e);
}
__device__ __forceinline__ lz lz_first(dd x, dd y) {
  lz a;
  two_prod(x, y, a.s, a.c);
  return a;
}
__device__ __forceinline__ dd neg(dd x) { return dd(-x.hi, -x.lo); }
__device__ __forceinline__ dd lz_norm(const lz& a) { return dd_2sum(a.s, a.c); }

// one double-float link element U_{row,col} of U_mu(x) (x = site i of parity par)
__device__ __forceinline__ cpx<dd> link_dd(const GDD& G, int mu, int par, long i, int row, int col) {
  const float4 v = __ldg(G.p + ((long)(mu * 2 + par) * 9 + 3 * row + col) * G.stride + i);
  return {dd(v.x, v.y), dd(v.z, v.w)};
}

// a += i^K u
template <int K>
__device__ __forceinline__ void lz_add_ipow(lzc& a, const lzc& u) {
  constexpr int k = ((K % 4) + 4) % 4;
  if constexpr (k == 0) {
    lz_add(a.r, u.r.s, u.r.c);
    lz_add(a.i, u.i.s, u.i.c);
  } else if constexpr (k == 1) {
    lz_add(a.r, -u.i.s, -u.i.c);
    lz_add(a.i, u.r.s, u.r.c);
  } else if constexpr (k == 2) {
    lz_add(a.r, -u.r.s, -u.r.c);
    lz_add(a.i, -u.i.s, -u.i.c);
  } else {
    lz_add(a.r, u.i.s, u.i.c);
    lz_add(a.i, -u.r.s, -u.r.c);
  }
}

// (U h)_c (DAG = false) or (U^dag h)_c (DAG = true) for one colour vector h
// of the half spinor, from row (column) c of U
template <bool DAG>
__device__ __forceinline__ lzc su3_row_lz(const cpx<dd> (&u)[3], const cpx<dd>* h) {
  lz re, im;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const cpx<dd> v = h[k];
    // U h:     re = ur vr - ui vi, im = ur vi + ui vr
    // U^dag h: re = ur vr + ui vi, im = ur vi - ui vr
    const dd ui_re = DAG ? u[k].i : neg(u[k].i);
    const dd ui_im = DAG ? neg(u[k].i) : u[k].i;
    if (k == 0) {
      re = lz_first(u[k].r, v.r);
      im = lz_first(u[k].r, v.i);
    } else {
      lz_fma(re, u[k].r, v.r);
      lz_fma(im, u[k].r, v.i);
    }
    lz_fma(re, ui_re, v.i);
    lz_fma(im, ui_im, v.r);
  }
  return {re, im};
}

// acc += (1 + SG g_mu) (x) [U or U^dag] h, colour by colour
template <int MU, int SG, bool DAG>
__device__ __forceinline__ void mul_accum_lz(const GDD& G, int par, long i, const cpx<dd> (&h)[6],
                                             lzc (&acc)[12]) {
  using Gm = Gam<MU>;
  constexpr int q0 = (SG > 0 ? 0 : 2) - Gm::k0;
  constexpr int q1 = (SG > 0 ? 0 : 2) - Gm::k1;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cpx<dd> u[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = DAG ? link_dd(G, MU, par, i, k, c) : link_dd(G, MU, par, i, c, k);
    const lzc o0 = su3_row_lz<DAG>(u, h);
    const lzc o1 = su3_row_lz<DAG>(u, h + 3);
    lz_add_ipow<0>(acc[c], o0);
    lz_add_ipow<0>(acc[3 + c], o1);
    lz_add_ipow<q0>(acc[3 * Gm::p0 + c], o0);
    lz_add_ipow<q1>(acc[3 * Gm::p1 + c], o1);
  }
}

// forward and backward hop in direction MU (same structure as hop_dir)
template <int MU, bool DAG>
__device__ __forceinline__ void hop_dir_lz(const HopArgs<SpDD, SpDD, SpDD, GDD>& a, long cb, const int (&c)[4],
                                           lzc (&acc)[12]) {
  constexpr int SF = DAG ? +1 : -1;
  constexpr int SB = -SF;
  const Geom& g = a.g;
  {
    int n[4] = {c[0], c[1], c[2], c[3]};
    n[MU] = (n[MU] + 1 == g.L[MU]) ? 0 : n[MU] + 1;
    const long nb = g.cb_of(n[0], n[1], n[2], n[3]);
    cpx<dd> s[12], h[6];
    a.in.loadT(nb, s);
    spin_project<MU, SF>(s, h);
    if (MU == 3 && c[3] == g.L[3] - 1) {
#pragma unroll
      for (int j = 0; j < 6; ++j) h[j] = {neg(h[j].r), neg(h[j].i)};
    }
    mul_accum_lz<MU, SF, false>(a.gauge, a.out_par, cb, h, acc);
  }
  {
    int n[4] = {c[0], c[1], c[2], c[3]};
    n[MU] = (n[MU] == 0) ? g.L[MU] - 1 : n[MU] - 1;
    const long nb = g.cb_of(n[0], n[1], n[2], n[3]);
    cpx<dd> s[12], h[6];
    a.in.loadT(nb, s);
    spin_project<MU, SB>(s, h);
    if (MU == 3 && c[3] == 0) {
#pragma unroll
      for (int j = 0; j < 6; ++j) h[j] = {neg(h[j].r), neg(h[j].i)};
    }
    mul_accum_lz<MU, SB, true>(a.gauge, 1 - a.out_par, nb, h, acc);
  }
}

// directions MU0 .. MU0 + NMU - 1 of one hop
template <int MU0, int NMU, bool DAG, bool FIRST, bool LAST, bool XPAY>
__global__ void __launch_bounds__(128, 4) k_hop_dd(HopArgs<SpDD, SpDD, SpDD, GDD> a) {
  const long cb = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= a.g.Vh) return;
  int c[4];
  a.g.coords(cb, a.out_par, c);
  lzc acc[12];
  if constexpr (FIRST) {
#pragma unroll
    for (int j = 0; j < 12; ++j) acc[j] = {{0.f, 0.f}, {0.f, 0.f}};
  } else {
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      const float4 v = __ldg(a.out.p + j * a.out.stride + cb);
      acc[j] = {{v.x, v.y}, {v.z, v.w}};
    }
  }
  hop_dir_lz<MU0, DAG>(a, cb, c, acc);
  if constexpr (NMU > 1) hop_dir_lz<MU0 + 1, DAG>(a, cb, c, acc);
  if constexpr (NMU > 2) {
    hop_dir_lz<MU0 + 2, DAG>(a, cb, c, acc);
    hop_dir_lz<MU0 + 3, DAG>(a, cb, c, acc);
  }
  // normalise, apply the epilogue and store one complex at a time
  const dd al(a.alpha);
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    cpx<dd> r = {lz_norm(acc[j].r), lz_norm(acc[j].i)};
    if constexpr (LAST && XPAY) {
      const float4 v = __ldg(a.y.p + j * a.y.stride + cb);
      r = cpx<dd>{dd(v.x, v.y), dd(v.z, v.w)} + al * r;
    }
    a.out.p[j * a.out.stride + cb] = make_float4(r.r.hi, r.r.lo, r.i.hi, r.i.lo);
  }
}

template <bool DAG, bool XPAY>
static int hop_dd_split(wd_ctx* c, const HopArgs<SpDD, SpDD, SpDD, GDD>& a) {
  const int nb = nblocks(c->g.Vh, 128);
  if constexpr (DD_DIRS_PER_LAUNCH == 4) {
    k_hop_dd<0, 4, DAG, true, true, XPAY><<<nb, 128, 0, c->stream>>>(a);
  } else if constexpr (DD_DIRS_PER_LAUNCH == 2) {
    k_hop_dd<0, 2, DAG, true, false, XPAY><<<nb, 128, 0, c->stream>>>(a);
    k_hop_dd<2, 2, DAG, false, true, XPAY><<<nb, 128, 0, c->stream>>>(a);
    c->launches += 1;
  } else {
    k_hop_dd<0, 1, DAG, true, false, XPAY><<<nb, 128, 0, c->stream>>>(a);
    k_hop_dd<1, 1, DAG, false, false, XPAY><<<nb, 128, 0, c->stream>>>(a);
    k_hop_dd<2, 1, DAG, false, false, XPAY><<<nb, 128, 0, c->stream>>>(a);
    k_hop_dd<3, 1, DAG, false, true, XPAY><<<nb, 128, 0, c->stream>>>(a);
    c->launches += 3;
  }
  WD_CHECK_LAUNCH();
  return WD_OK;
}

int hop_dd(wd_ctx* c, int out_par, bool dag, const Field& in, const Field& out, const Field* y,
           double alpha, bool norm_cg, bool in_cg) {
  if (in.fmt != WD_DD || out.fmt != WD_DD || (y && y->fmt != WD_DD))
    return fail(WD_ERR_ARG, "hop_dd: field formats must all be double-float");
  if (c->gauge_dd == nullptr) return fail(WD_ERR_STATE, "hop_dd: no double-float link copy");
  if (norm_cg || in_cg) return fail(WD_ERR_ARG, "hop_dd: not used inside queued CG iterations");
  if (out.data == in.data || (y && out.data == y->data))
    return fail(WD_ERR_ARG, "hop_dd: the output accumulates in place and may not alias an input");
  SpDD I = spdd(in), O = spdd(out), Y = y ? spdd(*y) : O;
  HopArgs<SpDD, SpDD, SpDD, GDD> a{c->g, out_par, I, O, Y, GDD{c->gauge_dd, c->g.Vh}, alpha,
                                    Reduce{nullptr, nullptr, nullptr}, nullptr};
  if (!dag) return y ? hop_dd_split<false, true>(c, a) : hop_dd_split<false, false>(c, a);
  return y ? hop_dd_split<true, true>(c, a) : hop_dd_split<true, false>(c, a);
}

}  // namespace wd
