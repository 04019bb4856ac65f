// Double-float instantiation of the hopping stencil: spinors and links in
// double-float storage (16 bytes per complex, like FP64), arithmetic by
// error-free transformations on the FP32 pipes (about 44-48 significant bits).
//
// The fully unrolled eight-direction kernel is too large for the instruction
// cache in double-float (ncu: "no instruction" stalls dominate), so one hop is
// four launches, one per direction mu (forward and backward hop): the first
// writes its contribution to the output, the next two add to it, the last adds
// and applies the y + alpha D x epilogue.  Memory is idle in this ALU-bound
// kernel, so re-reading the partial sum costs nothing noticeable.
#include "dslash_impl.cuh"

namespace wd {

template <int MU, bool DAG, bool FIRST, bool LAST, bool XPAY>
__global__ void __launch_bounds__(128) k_hop_dd_mu(HopArgs<SpDD, SpDD, SpDD, GDD> a) {
  const long cb = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= a.g.Vh) return;
  int c[4];
  a.g.coords(cb, a.out_par, c);
  cpx<dd> acc[12];
  if constexpr (FIRST) {
#pragma unroll
    for (int j = 0; j < 12; ++j) acc[j] = mk<dd>(0, 0);
  } else {
    a.out.loadT(cb, acc);
  }
  hop_dir<MU, DAG>(a.g, a.out_par, cb, c, a.in, a.gauge, acc);
  if constexpr (LAST && XPAY) {
    cpx<dd> yv[12];
    a.y.loadT(cb, yv);
    const dd al(a.alpha);
#pragma unroll
    for (int j = 0; j < 12; ++j) acc[j] = yv[j] + al * acc[j];
  }
  a.out.store(cb, acc);
}

template <bool DAG, bool XPAY>
static int hop_dd_split(wd_ctx* c, const HopArgs<SpDD, SpDD, SpDD, GDD>& a) {
  const int nb = nblocks(c->g.Vh, 128);
  k_hop_dd_mu<0, DAG, true, false, XPAY><<<nb, 128, 0, c->stream>>>(a);
  k_hop_dd_mu<1, DAG, false, false, XPAY><<<nb, 128, 0, c->stream>>>(a);
  k_hop_dd_mu<2, DAG, false, false, XPAY><<<nb, 128, 0, c->stream>>>(a);
  k_hop_dd_mu<3, DAG, false, true, XPAY><<<nb, 128, 0, c->stream>>>(a);
  c->launches += 3;
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
