// FP32 instantiations of the hopping stencil (float storage and arithmetic,
// FP32 links with 18 or 12 stored reals).
#include "dslash_impl.cuh"

namespace wd {

int hop_f32(wd_ctx* c, int out_par, bool dag, const Field& in, const Field& out, const Field* y,
            double alpha, bool norm_cg, bool in_cg) {
  if (in.fmt != WD_F32 || out.fmt != WD_F32 || (y && y->fmt != WD_F32))
    return fail(WD_ERR_ARG, "hop_f32: field formats must all be FP32");
  SpF32 I = sp32(in), O = sp32(out), Y = y ? sp32(*y) : O;
  return hop_with_gauge<float>(c, out_par, dag, I, O, Y, y != nullptr, alpha, norm_cg, in_cg, false);
}

}  // namespace wd
