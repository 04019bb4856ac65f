// Operator layer: hop dispatch, M_hat and K_hat compositions, launch sampling.
//
// Section 3.1 (Wilson fermions, even-odd preconditioning):
//   M_hat = 1 - kappa^2 D_eo D_oe,  M_hat^dag = 1 - kappa^2 D^dag_eo D^dag_oe,
//   K_hat = M_hat^dag M_hat (the multiplication N_mat counts, Section 3.1).
#include "dslash_impl.cuh"

namespace wd {

static int spinor_bytes(int fmt) {
  switch (fmt) {
    case WD_F64:
    case WD_DD: return 192;
    case WD_F32: return 96;
    default: return 52;   // 48 bytes of 16-bit values + 4-byte norm
  }
}

double hop_bytes(int fmt_in, int fmt_out, bool xpay, int gauge_bytes_per_link, long Vh) {
  // every input site, link and output site moved once; y read once if xpay
  double per = 8.0 * gauge_bytes_per_link + spinor_bytes(fmt_in) + spinor_bytes(fmt_out) +
               (xpay ? spinor_bytes(fmt_in) : 0);
  return per * (double)Vh;
}

static int gauge_link_bytes(wd_ctx* c, int fmt_in) {
  if (fmt_in == WD_F64 || fmt_in == WD_DD) return 144;
  return c->recon == WD_RECON_12 ? 48 : 72;
}

void prof_begin(wd_ctx* c, cudaEvent_t* e0) {
  *e0 = nullptr;
  Prof& p = c->prof;
  if (p.every <= 0) return;
  if ((p.seen++ % p.every) != 0) return;
  if (p.ev.size() >= 8192) return;   // pending buffer full: skip this sample
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, c->stream);
  *e0 = e;
}

void prof_end(wd_ctx* c, cudaEvent_t e0, double bytes, int fmt) {
  if (e0 == nullptr) return;
  cudaEvent_t e1;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return; }
  cudaEventRecord(e1, c->stream);
  c->prof.ev.push_back(e0);
  c->prof.ev.push_back(e1);
  c->prof.ev_bytes.push_back(bytes);
  c->prof.ev_fmt.push_back(fmt);
}

int hop(wd_ctx* c, int out_par, bool dag, const Field& in, const Field& out, const Field* y,
        double alpha, bool norm_cg, bool in_cg) {
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  // Launches queued inside a CG chunk may return at once after convergence;
  // only launches that always do their work are sampled.
  cudaEvent_t e0 = nullptr;
  if (in.fmt >= 0 && in.fmt < Prof::NF) c->prof.all[in.fmt] += 1;
  if (!in_cg) prof_begin(c, &e0);
  int s;
  if (in.fmt == WD_F64) s = hop_f64(c, out_par, dag, in, out, y, alpha, norm_cg, in_cg);
  else if (in.fmt == WD_F32) s = hop_f32(c, out_par, dag, in, out, y, alpha, norm_cg, in_cg);
  else if (in.fmt == WD_DD) s = hop_dd(c, out_par, dag, in, out, y, alpha, norm_cg, in_cg);
  else s = hop_h16(c, out_par, dag, in, out, y, alpha, norm_cg, in_cg);
  if (s != WD_OK) return s;
  prof_end(c, e0, hop_bytes(in.fmt, out.fmt, y != nullptr, gauge_link_bytes(c, in.fmt), c->g.Vh), in.fmt);
  return WD_OK;
}

int apply_mhat(wd_ctx* c, double kappa, bool dag, const Field& in, const Field& out, Field& tmp,
               bool norm_cg) {
  WD_TRY(hop(c, 1, dag, in, tmp, nullptr, 0.0, false, false));
  return hop(c, 0, dag, tmp, out, &in, -kappa * kappa, norm_cg, false);
}

int apply_khat(wd_ctx* c, double kappa, const Field& in, const Field& out, Field& t1, Field& t2,
               bool norm_cg, bool in_cg) {
  // t2 = M_hat in (with |t2|^2 = <in, K_hat in> when norm_cg), out = M_hat^dag t2
  WD_TRY(hop(c, 1, false, in, t1, nullptr, 0.0, false, in_cg));
  WD_TRY(hop(c, 0, false, t1, t2, &in, -kappa * kappa, norm_cg, in_cg));
  WD_TRY(hop(c, 1, true, t2, t1, nullptr, 0.0, false, in_cg));
  WD_TRY(hop(c, 0, true, t1, out, &t2, -kappa * kappa, false, in_cg));
  c->nmat += 1;
  return WD_OK;
}

}  // namespace wd
