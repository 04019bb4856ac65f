// Layout kernels: lexicographic host-order fields <-> even-odd structure-of-
// arrays device fields, and the FP32 link copies derived from the FP64 links.
#include "dslash_impl.cuh"

namespace wd {

// One thread per lexicographic site.  The lexicographic field holds
// nouter * nchunk * chunk doubles per site (outer index = mu or nothing);
// the EO field is [outer][parity][nchunk][Vh] of `chunk` doubles when
// parity < 0 (both parities), or [nchunk][Vh] for one parity.
template <bool UNPACK>
__global__ void k_pack(Geom g, int nouter, int nchunk, int chunk, int parity, const double* src,
                       double* dst) {
  const long lex = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (lex >= g.V) return;
  const int x = (int)(lex % g.L[0]);
  long r = lex / g.L[0];
  const int y = (int)(r % g.L[1]); r /= g.L[1];
  const int z = (int)(r % g.L[2]);
  const int t = (int)(r / g.L[2]);
  const int par = (x + y + z + t) & 1;
  if (parity >= 0 && par != parity) return;
  const long cb = lex >> 1;
  const long per_site = (long)nouter * nchunk * chunk;
  for (int o = 0; o < nouter; ++o) {
    const long base = parity >= 0 ? 0 : (long)(o * 2 + par) * nchunk;
    for (int j = 0; j < nchunk; ++j) {
      const long eo = ((base + j) * g.Vh + cb) * chunk;
      const long lx = lex * per_site + ((long)o * nchunk + j) * chunk;
      for (int w = 0; w < chunk; ++w) {
        if (UNPACK) dst[lx + w] = src[eo + w];
        else dst[eo + w] = src[lx + w];
      }
    }
  }
}

int pack_k(wd_ctx* c, bool unpack, int nouter, int nchunk, int chunk, int parity, const double* src,
           double* dst) {
  const int nb = nblocks(c->g.V, 128);
  if (unpack) k_pack<true><<<nb, 128, 0, c->stream>>>(c->g, nouter, nchunk, chunk, parity, src, dst);
  else k_pack<false><<<nb, 128, 0, c->stream>>>(c->g, nouter, nchunk, chunk, parity, src, dst);
  WD_CHECK_LAUNCH();
  return WD_OK;
}

__global__ void k_gauge_lowprec(long n9, long Vh, const double2* U64, float2* U32, float4* U12, float4* Udd) {
  // one thread per link (mu, parity, cb): n = 8 Vh
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n9) return;
  const long mp = i / Vh, cb = i % Vh;
  const double2* u = U64 + mp * 9 * Vh + cb;
  double2 v[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) v[j] = u[j * Vh];
  if (Udd != nullptr) {
    float4* o = Udd + mp * 9 * Vh + cb;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const dd r(v[j].x), m(v[j].y);
      o[j * Vh] = make_float4(r.hi, r.lo, m.hi, m.lo);
    }
  }
  float2* o = U32 + mp * 9 * Vh + cb;
#pragma unroll
  for (int j = 0; j < 9; ++j) o[j * Vh] = make_float2((float)v[j].x, (float)v[j].y);
  float4* q = U12 + mp * 3 * Vh + cb;
#pragma unroll
  for (int j = 0; j < 3; ++j)
    q[j * Vh] = make_float4((float)v[2 * j].x, (float)v[2 * j].y, (float)v[2 * j + 1].x, (float)v[2 * j + 1].y);
}

int gauge_lowprec_k(wd_ctx* c) {
  const long n = 8 * c->g.Vh;
  k_gauge_lowprec<<<nblocks(n, 128), 128, 0, c->stream>>>(n, c->g.Vh, c->gauge64, c->gauge32, c->gauge32r12,
                                                          c->gauge_dd);
  WD_CHECK_LAUNCH();
  return WD_OK;
}

}  // namespace wd
