// FP64 instantiations of the hopping stencil (double storage, double arithmetic).
#include "dslash_impl.cuh"

namespace wd {

int hop_f64(wd_ctx* c, int out_par, bool dag, const Field& in, const Field& out, const Field* y,
            double alpha, bool norm_cg, bool in_cg) {
  if (in.fmt != WD_F64 || out.fmt != WD_F64 || (y && y->fmt != WD_F64))
    return fail(WD_ERR_ARG, "hop_f64: field formats must all be FP64");
  SpF64 I = sp64(in), O = sp64(out), Y = y ? sp64(*y) : O;
  return hop_with_gauge<double>(c, out_par, dag, I, O, Y, y != nullptr, alpha, norm_cg, in_cg, true);
}

}  // namespace wd
