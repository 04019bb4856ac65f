// Double-float instantiation of the hopping stencil: spinors and links in
// double-float storage (16 bytes per complex, like FP64), arithmetic by
// error-free transformations on the FP32 pipes (about 48 significant bits).
#include "dslash_impl.cuh"

namespace wd {

int hop_dd(wd_ctx* c, int out_par, bool dag, const Field& in, const Field& out, const Field* y,
           double alpha, bool norm_cg, bool in_cg) {
  if (in.fmt != WD_DD || out.fmt != WD_DD || (y && y->fmt != WD_DD))
    return fail(WD_ERR_ARG, "hop_dd: field formats must all be double-float");
  if (c->gauge_dd == nullptr) return fail(WD_ERR_STATE, "hop_dd: no double-float link copy");
  SpDD I = spdd(in), O = spdd(out), Y = y ? spdd(*y) : O;
  return hop_with_gauge<dd>(c, out_par, dag, I, O, Y, y != nullptr, alpha, norm_cg, in_cg, false);
}

}  // namespace wd
