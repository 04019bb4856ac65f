// C ABI: context, error reporting, workspace pool, field layout and operator
// entry points.  Every entry validates its arguments before any launch.
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "dslash_impl.cuh"

namespace wd {

static thread_local std::string g_err = "no error";

void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  return fail(WD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int ws_get(wd_ctx* c, int fmt, Field* f) {
  for (size_t i = 0; i < c->pool.size(); ++i) {
    if (!c->pool_used[i] && c->pool[i].fmt == fmt) {
      c->pool_used[i] = true;
      *f = c->pool[i];
      return WD_OK;
    }
  }
  Field n;
  n.fmt = fmt;
  n.stride = c->g.Vh;
  WD_CUDA(cudaMalloc(&n.data, field_bytes(fmt, c->g.Vh)));
  if (fmt == WD_F16 || fmt == WD_BF16) {
    cudaError_t e = cudaMalloc(&n.norm, sizeof(float) * c->g.Vh);
    if (e != cudaSuccess) {
      cudaFree(n.data);
      return cuda_fail(e, "cudaMalloc(norm)");
    }
  }
  c->pool.push_back(n);
  c->pool_used.push_back(true);
  *f = n;
  return WD_OK;
}

void ws_put(wd_ctx* c, const Field& f) {
  for (size_t i = 0; i < c->pool.size(); ++i)
    if (c->pool[i].data == f.data) c->pool_used[i] = false;
}

Field wrap_f64(wd_ctx* c, const double* p) {
  Field f;
  f.data = const_cast<double*>(p);
  f.fmt = WD_F64;
  f.stride = c->g.Vh;
  return f;
}

}  // namespace wd

using namespace wd;

#define CHECK_CTX(c) \
  if ((c) == nullptr) return fail(WD_ERR_ARG, "null context")
#define CHECK_PTR(p) \
  if ((p) == nullptr) return fail(WD_ERR_ARG, #p " is null")

static_assert((int)WD_DF == (int)WD_DD, "the public double-float precision is the internal format");

static int ensure_gauge_dd(wd_ctx* c) {
  if (c->gauge_dd != nullptr) return WD_OK;
  WD_CUDA(cudaMalloc(&c->gauge_dd, sizeof(float4) * 72 * c->g.Vh));
  if (c->have_gauge) return gauge_lowprec_k(c);
  return WD_OK;
}

// operator entry points accept every precision including double-float
static int check_prec(wd_ctx* c, int prec) {
  if (prec < WD_F64 || prec > WD_DF) return fail(WD_ERR_ARG, "unknown precision");
  if (prec == WD_DF) return ensure_gauge_dd(c);
  return WD_OK;
}

extern "C" {

const char* wd_last_error(void) { return g_err.c_str(); }

int wd_context_create(const int dims[4], void* stream, wd_ctx** out) {
  CHECK_PTR(dims);
  CHECK_PTR(out);
  *out = nullptr;
  for (int m = 0; m < 4; ++m)
    if (dims[m] < 2 || dims[m] % 2 != 0) return fail(WD_ERR_ARG, "every lattice extent must be even and >= 2");
  if ((long long)dims[0] * dims[1] * dims[2] * dims[3] >= (1LL << 31))
    return fail(WD_ERR_ARG, "the lattice must have fewer than 2^31 sites");
  wd_ctx* c = new (std::nothrow) wd_ctx();
  if (!c) return fail(WD_ERR_ARG, "out of host memory");
  for (int m = 0; m < 4; ++m) c->g.L[m] = dims[m];
  c->g.Lh = dims[0] / 2;
  c->g.V = (long)dims[0] * dims[1] * dims[2] * dims[3];
  c->g.Vh = c->g.V / 2;
  c->stream = (cudaStream_t)stream;
  cudaGetDevice(&c->device);
  const long Vh = c->g.Vh;
  cudaError_t e = cudaSuccess;
  auto al = [&](void** p, size_t n) { if (e == cudaSuccess) e = cudaMalloc(p, n); };
  al((void**)&c->gauge64, sizeof(double2) * 72 * Vh);
  al((void**)&c->gauge32, sizeof(float2) * 72 * Vh);
  al((void**)&c->gauge32r12, sizeof(float4) * 24 * Vh);
  al((void**)&c->red_partial, sizeof(double) * 4 * RED_MAX_BLOCKS);
  al((void**)&c->red_counter, sizeof(unsigned) * 4);
  al((void**)&c->red_out, sizeof(double) * 16);
  al((void**)&c->cgs, sizeof(CGState));
  al((void**)&c->kerr, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->cgs_host, sizeof(CGState));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->host_scalar, sizeof(double) * 16);
  if (e == cudaSuccess) e = cudaMemset(c->red_counter, 0, sizeof(unsigned) * 4);
  if (e == cudaSuccess) e = cudaMemset(c->cgs, 0, sizeof(CGState));
  if (e == cudaSuccess) e = cudaMemset(c->kerr, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    std::string m = std::string("wd_context_create: ") + cudaGetErrorString(e);
    wd_context_destroy(c);
    return fail(WD_ERR_CUDA, m);
  }
  *out = c;
  return WD_OK;
}

int wd_context_destroy(wd_ctx* c) {
  if (!c) return WD_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  cudaFree(c->gauge64);
  cudaFree(c->gauge32);
  cudaFree(c->gauge32r12);
  cudaFree(c->gauge_dd);
  cudaFree(c->red_partial);
  cudaFree(c->red_counter);
  cudaFree(c->red_out);
  cudaFree(c->cgs);
  cudaFree(c->kerr);
  cudaFree(c->gauge_backup);
  cudaFree(c->mom);
  cudaFree(c->lex_stage);
  if (c->cgs_host) cudaFreeHost(c->cgs_host);
  if (c->host_scalar) cudaFreeHost(c->host_scalar);
  for (auto& f : c->pool) {
    cudaFree(f.data);
    if (f.norm) cudaFree(f.norm);
  }
  for (auto& e : c->prof.ev) cudaEventDestroy(e);
  for (auto& kv : c->tune_samples)
    for (auto& e : kv.second.ev) cudaEventDestroy(e);
  delete c;
  return WD_OK;
}

int wd_set_recon(wd_ctx* c, int recon) {
  CHECK_CTX(c);
  if (recon != WD_RECON_18 && recon != WD_RECON_12) return fail(WD_ERR_ARG, "recon must be 18 or 12");
  c->recon = recon;
  return WD_OK;
}

int wd_set_autotune(wd_ctx* c, int enable, int* n_tuned) {
  CHECK_CTX(c);
  if (enable != 0 && enable != 1 && enable != -1) return fail(WD_ERR_ARG, "enable must be 0, 1 or -1 (query)");
  if (enable >= 0) c->autotune = enable;
  if (n_tuned) *n_tuned = (int)c->tune.size();
  return WD_OK;
}

int wd_tune_entry(wd_ctx* c, int index, long long* key, int* threads, int* minb) {
  CHECK_CTX(c);
  if (index < 0 || index >= (int)c->tune.size()) return fail(WD_ERR_ARG, "index out of range");
  auto it = c->tune.begin();
  std::advance(it, index);
  if (key) *key = it->first;
  if (threads) *threads = it->second.first;
  if (minb) *minb = it->second.second;
  return WD_OK;
}

int wd_set_residual(wd_ctx* c, int mode) {
  CHECK_CTX(c);
  if (mode != 0 && mode != 1) return fail(WD_ERR_ARG, "mode must be 0 (FP64) or 1 (double-float)");
  if (mode == 1) WD_TRY(ensure_gauge_dd(c));
  c->resid_dd = mode;
  return WD_OK;
}

int wd_set_stencil(wd_ctx* c, int stencil) {
  CHECK_CTX(c);
  if (stencil != WD_STENCIL_THREAD && stencil != WD_STENCIL_TILE)
    return fail(WD_ERR_ARG, "stencil must be WD_STENCIL_THREAD (0) or WD_STENCIL_TILE (1)");
  c->stencil = stencil;
  return WD_OK;
}

int wd_kernel_status(wd_ctx* c, unsigned* word) {
  CHECK_CTX(c);
  unsigned* h = (unsigned*)c->host_scalar;
  WD_CUDA(cudaMemcpyAsync(h, c->kerr, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  const unsigned w = *h;
  if (word) *word = w;
  if (w == 0) return WD_OK;
  WD_CUDA(cudaMemsetAsync(c->kerr, 0, sizeof(unsigned), c->stream));
  WD_CUDA(cudaStreamSynchronize(c->stream));
  return fail(WD_ERR_TIMEOUT, "a bounded device-side wait expired in a stencil kernel");
}

int wd_selftest_wait_timeout(wd_ctx* c, long long timeout_ns) {
  CHECK_CTX(c);
  if (timeout_ns < 1000000LL || timeout_ns > 10000000000LL)
    return fail(WD_ERR_ARG, "timeout_ns must lie in [1e6, 1e10]");
  return wait_selftest(c, timeout_ns);
}

int wd_volume(const wd_ctx* c, long long out[2]) {
  CHECK_CTX(c);
  CHECK_PTR(out);
  out[0] = c->g.V;
  out[1] = c->g.Vh;
  return WD_OK;
}

int wd_gauge_load(wd_ctx* c, const double* U_lex) {
  CHECK_CTX(c);
  CHECK_PTR(U_lex);
  WD_TRY(pack_k(c, false, 4, 9, 2, -1, U_lex, (double*)c->gauge64));
  WD_TRY(gauge_lowprec_k(c));
  c->have_gauge = true;
  return WD_OK;
}

int wd_gauge_store(wd_ctx* c, double* U_lex) {
  CHECK_CTX(c);
  CHECK_PTR(U_lex);
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  return pack_k(c, true, 4, 9, 2, -1, (const double*)c->gauge64, U_lex);
}

int wd_spinor_pack(wd_ctx* c, int parity, const double* lex, double* eo) {
  CHECK_CTX(c);
  CHECK_PTR(lex);
  CHECK_PTR(eo);
  if (parity != 0 && parity != 1) return fail(WD_ERR_ARG, "parity must be 0 or 1");
  return pack_k(c, false, 1, 12, 2, parity, lex, eo);
}

int wd_spinor_unpack(wd_ctx* c, int parity, const double* eo, double* lex) {
  CHECK_CTX(c);
  CHECK_PTR(lex);
  CHECK_PTR(eo);
  if (parity != 0 && parity != 1) return fail(WD_ERR_ARG, "parity must be 0 or 1");
  return pack_k(c, true, 1, 12, 2, parity, eo, lex);
}

int wd_algebra_pack(wd_ctx* c, const double* lex, double* eo) {
  CHECK_CTX(c);
  CHECK_PTR(lex);
  CHECK_PTR(eo);
  return pack_k(c, false, 4, 8, 1, -1, lex, eo);
}

int wd_algebra_unpack(wd_ctx* c, const double* eo, double* lex) {
  CHECK_CTX(c);
  CHECK_PTR(lex);
  CHECK_PTR(eo);
  return pack_k(c, true, 4, 8, 1, -1, eo, lex);
}

int wd_hop(wd_ctx* c, int out_parity, int dagger, int prec, const double* in, double* out) {
  CHECK_CTX(c);
  CHECK_PTR(in);
  CHECK_PTR(out);
  if (out_parity != 0 && out_parity != 1) return fail(WD_ERR_ARG, "parity must be 0 or 1");
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  WD_TRY(check_prec(c, prec));
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  Field fi = wrap_f64(c, in), fo = wrap_f64(c, out);
  if (prec == WD_F64) return hop(c, out_parity, dagger != 0, fi, fo, nullptr, 0.0, false, false);
  WsGuard w(c);
  Field a, b;
  WD_TRY(w.get(prec, &a));
  WD_TRY(w.get(prec, &b));
  WD_TRY(convert(c, fi, a));
  WD_TRY(hop(c, out_parity, dagger != 0, a, b, nullptr, 0.0, false, false));
  return convert(c, b, fo);
}

int wd_apply(wd_ctx* c, double kappa, int dagger, int prec, const double* in, double* out) {
  CHECK_CTX(c);
  CHECK_PTR(in);
  CHECK_PTR(out);
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  WD_TRY(check_prec(c, prec));
  Field fi = wrap_f64(c, in), fo = wrap_f64(c, out);
  WsGuard w(c);
  Field t, a, b;
  WD_TRY(w.get(prec, &t));
  if (prec == WD_F64) return apply_mhat(c, kappa, dagger != 0, fi, fo, t, false);
  WD_TRY(w.get(prec, &a));
  WD_TRY(w.get(prec, &b));
  WD_TRY(convert(c, fi, a));
  WD_TRY(apply_mhat(c, kappa, dagger != 0, a, b, t, false));
  return convert(c, b, fo);
}

int mdagm_apply(wd_ctx* c, double kappa, int prec, int nrhs, const double* in, double* out) {
  CHECK_CTX(c);
  CHECK_PTR(in);
  CHECK_PTR(out);
  if (nrhs < 1) return fail(WD_ERR_ARG, "nrhs must be >= 1");
  if (!c->have_gauge) return fail(WD_ERR_STATE, "no gauge field loaded");
  WD_TRY(check_prec(c, prec));
  WsGuard w(c);
  Field t1, t2, a, b;
  WD_TRY(w.get(prec, &t1));
  WD_TRY(w.get(prec, &t2));
  if (prec != WD_F64) {
    WD_TRY(w.get(prec, &a));
    // K_hat of 16-bit input writes FP32; FP32 and double-float keep their format
    WD_TRY(w.get(prec == WD_DF ? WD_DD : WD_F32, &b));
  }
  const long stride = 24 * c->g.Vh;
  for (int k = 0; k < nrhs; ++k) {
    Field fi = wrap_f64(c, in + k * stride), fo = wrap_f64(c, out + k * stride);
    if (prec == WD_F64) {
      WD_TRY(apply_khat(c, kappa, fi, fo, t1, t2, false, false));
    } else {
      WD_TRY(convert(c, fi, a));
      WD_TRY(apply_khat(c, kappa, a, b, t1, t2, false, false));
      WD_TRY(convert(c, b, fo));
    }
  }
  return WD_OK;
}

int wd_nmat(wd_ctx* c, long long* count, int reset) {
  CHECK_CTX(c);
  if (count) *count = c->nmat;
  if (reset) c->nmat = 0;
  return WD_OK;
}

int wd_profile_enable(wd_ctx* c, int every_n) {
  CHECK_CTX(c);
  if (every_n < 0) return fail(WD_ERR_ARG, "every_n must be >= 0");
  Prof& p = c->prof;
  p.every = every_n;
  p.seen = 0;
  for (int f = 0; f < Prof::NF; ++f) { p.launches[f] = 0; p.ms[f] = 0.0; p.bytes[f] = 0.0; p.all[f] = 0; }
  for (auto& e : p.ev) cudaEventDestroy(e);
  p.ev.clear();
  p.ev_bytes.clear();
  p.ev_fmt.clear();
  return WD_OK;
}

int wd_profile_read(wd_ctx* c, int fmt, long long* launches, double* total_ms, double* bytes) {
  CHECK_CTX(c);
  if (fmt < -1 || fmt >= Prof::NF) return fail(WD_ERR_ARG, "fmt must be -1 (all), a wd_prec or 4 (double-float)");
  Prof& p = c->prof;
  for (size_t k = 0; k + 1 < p.ev.size(); k += 2) {
    float ms = 0.f;
    WD_CUDA(cudaEventSynchronize(p.ev[k + 1]));
    WD_CUDA(cudaEventElapsedTime(&ms, p.ev[k], p.ev[k + 1]));
    const int f = p.ev_fmt[k / 2];
    p.ms[f] += ms;
    p.bytes[f] += p.ev_bytes[k / 2];
    p.launches[f] += 1;
    cudaEventDestroy(p.ev[k]);
    cudaEventDestroy(p.ev[k + 1]);
  }
  p.ev.clear();
  p.ev_bytes.clear();
  p.ev_fmt.clear();
  long long n = 0;
  double ms = 0, b = 0;
  for (int f = 0; f < Prof::NF; ++f) {
    if (fmt >= 0 && f != fmt) continue;
    n += p.launches[f];
    ms += p.ms[f];
    b += p.bytes[f];
  }
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  if (bytes) *bytes = b;
  return WD_OK;
}

int wd_hop_counts(wd_ctx* c, long long counts[5]) {
  CHECK_CTX(c);
  CHECK_PTR(counts);
  for (int f = 0; f < Prof::NF; ++f) counts[f] = c->prof.all[f];
  return WD_OK;
}

int wd_launch_count(wd_ctx* c, long long* count) {
  CHECK_CTX(c);
  CHECK_PTR(count);
  *count = c->launches;
  return WD_OK;
}

int metropolis(double dH, double u, int* accept) {
  CHECK_PTR(accept);
  if (!(u >= 0.0 && u < 1.0)) return fail(WD_ERR_ARG, "u must be in [0, 1)");
  if (std::isnan(dH)) return fail(WD_ERR_NAN, "dH is NaN");
  *accept = (u < std::exp(-dH)) ? 1 : 0;
  return WD_OK;
}

}  // extern "C"

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) on the host: ten rounds of
// two 64 x 64 -> 128-bit products with the published multipliers, the key
// bumped by the published Weyl constants between rounds.
static void host_philox4x64(uint64_t (&x)[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const unsigned __int128 p0 = (unsigned __int128)M0 * x[0], p1 = (unsigned __int128)M1 * x[2];
    const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    const uint64_t n0 = hi1 ^ x[1] ^ k0, n2 = hi0 ^ x[3] ^ k1;
    x[0] = n0;
    x[1] = lo1;
    x[2] = n2;
    x[3] = lo0;
  }
}

extern "C" {

int metropolis_philox(double dH, uint64_t seed, uint64_t counter, double* u, int* accept) {
  CHECK_PTR(accept);
  uint64_t x[4] = {counter, WD_METROPOLIS_STREAM, 0ull, 0ull};
  host_philox4x64(x, seed, 0ull);
  const double uu = ((double)(x[0] >> 11) + 0.5) * 0x1.0p-53;
  if (u) *u = uu;
  return metropolis(dH, uu, accept);
}

int wd_cost(const long long* n_mat, const int* accepted, const double* dH, int n, wd_cost_result* out) {
  CHECK_PTR(n_mat);
  CHECK_PTR(accepted);
  CHECK_PTR(dH);
  CHECK_PTR(out);
  if (n < 1) return fail(WD_ERR_ARG, "wd_cost: n must be >= 1");
  double sn = 0, sa = 0, se = 0, sx = 0, sx2 = 0;
  for (int i = 0; i < n; ++i) {
    if (n_mat[i] < 0) return fail(WD_ERR_ARG, "wd_cost: n_mat must be >= 0");
    if (accepted[i] != 0 && accepted[i] != 1) return fail(WD_ERR_ARG, "wd_cost: accepted must be 0 or 1");
    if (std::isnan(dH[i])) return fail(WD_ERR_NAN, "wd_cost: dH is NaN");
    const double x = std::exp(-dH[i]);
    sn += (double)n_mat[i];
    sa += accepted[i];
    se += x < 1.0 ? x : 1.0;
    sx += x;
    sx2 += x * x;
  }
  wd_cost_result r;
  r.mean_nmat = sn / n;
  r.p_acc = sa / n;
  r.p_acc_est = se / n;
  r.C = r.p_acc > 0 ? r.mean_nmat / r.p_acc : INFINITY;
  r.C_est = r.p_acc_est > 0 ? r.mean_nmat / r.p_acc_est : INFINITY;
  r.exp_mdH = sx / n;
  const double var = n > 1 ? (sx2 - sx * sx / n) / (n - 1) : 0.0;
  r.exp_mdH_err = n > 1 ? std::sqrt((var > 0 ? var : 0.0) / n) : 0.0;
  *out = r;
  return WD_OK;
}

}  // extern "C"
