// 16-bit instantiations of the hopping stencil: half or bfloat16 spinors with
// a per-site FP32 norm, FP32 arithmetic, FP32 links (12-real links on the
// staged pipeline).  The output may be 16-bit or FP32 (the last hop of K_hat
// inside mixed-precision CG writes FP32).
#include "dslash_tt.cuh"

namespace wd {

template <class H>
static int hop_h(wd_ctx* c, int out_par, bool dag, const Field& in, const Field& out, const Field* y,
                 double alpha, bool norm_cg, bool in_cg) {
  Sp16<H> I = sp16<H>(in);
  if (y && y->fmt != in.fmt) return fail(WD_ERR_ARG, "hop_h16: y must match the input format");
  Sp16<H> Y = y ? sp16<H>(*y) : I;
  if (c->recon == WD_RECON_12 && tt_eligible(c)) {
    if (out.fmt == in.fmt) return hop_tt(c, out_par, dag, I, sp16<H>(out), Y, y != nullptr, alpha, norm_cg, in_cg);
    if (out.fmt == WD_F32) return hop_tt(c, out_par, dag, I, sp32(out), Y, y != nullptr, alpha, norm_cg, in_cg);
    return fail(WD_ERR_ARG, "hop_h16: output must be 16-bit of the same kind or FP32");
  }
  if (c->recon == WD_RECON_12) {
    if (out.fmt == in.fmt) return hop_staged(c, out_par, dag, I, sp16<H>(out), Y, y != nullptr, alpha, norm_cg, in_cg);
    if (out.fmt == WD_F32) return hop_staged(c, out_par, dag, I, sp32(out), Y, y != nullptr, alpha, norm_cg, in_cg);
    return fail(WD_ERR_ARG, "hop_h16: output must be 16-bit of the same kind or FP32");
  }
  if (out.fmt == in.fmt)
    return hop_with_gauge<float>(c, out_par, dag, I, sp16<H>(out), Y, y != nullptr, alpha, norm_cg, in_cg, false);
  if (out.fmt == WD_F32)
    return hop_with_gauge<float>(c, out_par, dag, I, sp32(out), Y, y != nullptr, alpha, norm_cg, in_cg, false);
  return fail(WD_ERR_ARG, "hop_h16: output must be 16-bit of the same kind or FP32");
}

int hop_h16(wd_ctx* c, int out_par, bool dag, const Field& in, const Field& out, const Field* y,
            double alpha, bool norm_cg, bool in_cg) {
  if (in.fmt == WD_F16) return hop_h<__half>(c, out_par, dag, in, out, y, alpha, norm_cg, in_cg);
  if (in.fmt == WD_BF16) return hop_h<__nv_bfloat16>(c, out_par, dag, in, out, y, alpha, norm_cg, in_cg);
  return fail(WD_ERR_ARG, "hop_h16: input must be FP16 or BF16");
}

}  // namespace wd
