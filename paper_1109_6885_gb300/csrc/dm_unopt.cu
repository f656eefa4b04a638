// Step 2(b) by the paper's unoptimised route (Section 5.2, Eq. 5): every
// tuple's value is decoded through its old dictionary (U_M for main rows,
// D_dict for delta rows) and looked up in U' by binary search, instead of
// being translated through X_M / X_D (Section 5.3).  The output is the same
// packed vector; the route exists to measure what the translation tables
// save (Section 7's Opt / UnOpt comparison) and as a second, independent
// way to the same bytes.
//
// One thread owns a group of 32 consecutive output codes, exactly b' words
// of the packed output, so threads write disjoint whole words.
#include <stdint.h>

#include "../../include/dmerge.h"
#include "dm_common.cuh"
#include "dm_ctx.h"

namespace dm {

namespace {

struct SearchArgs {
  const uint32_t* main_words;
  uint64_t main_words_n;
  uint32_t b;
  uint64_t n_main;
  const uint32_t* dcodes;
  uint64_t n_delta;
  const void* um;          // U_M
  uint64_t m;
  const void* dd;          // D_dict (insertion order)
  uint64_t d;
  const void* unew;        // U'
  const uint64_t* d_u;     // |U'| (device scalar)
  const uint32_t* d_bits;  // E'_C (device scalar)
  uint32_t max_bits;
  uint32_t* out_words;
  uint32_t* status;
};

// Code i of a packed stream at b bits (plain, bounds-checked loads).
__device__ __forceinline__ uint32_t packed_code(const uint32_t* words, uint64_t nwords, uint64_t i, uint32_t b) {
  if (b == 0) return 0;
  const uint64_t bit = i * b, k = bit >> 5;
  const uint32_t lo = k < nwords ? __ldg(words + k) : 0u;
  const uint32_t hi = k + 1 < nwords ? __ldg(words + k + 1) : 0u;
  const uint32_t v = __funnelshift_r(lo, hi, (uint32_t)(bit & 31));
  return b == 32 ? v : (v & ((1u << b) - 1u));
}

template <int W>
__global__ void __launch_bounds__(256) reencode_search_kernel(SearchArgs a) {
  using K = typename KeyOf<W>::T;
  const uint32_t bo = *a.d_bits;
  const uint64_t u = *a.d_u;
  if (bo > a.max_bits || u > a.m + a.d) {
    if (blockIdx.x == 0 && threadIdx.x == 0) flag_status(a.status, ST_WIDTH);
    return;
  }
  const K* um = static_cast<const K*>(a.um);
  const K* dd = static_cast<const K*>(a.dd);
  const K* un = static_cast<const K*>(a.unew);
  const uint64_t n_out = a.n_main + a.n_delta;
  const uint64_t groups = (n_out + 31) / 32;
  const uint64_t out_total = ((n_out * bo + 127) / 128) * 4;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += stride) {
    uint64_t acc = 0, w = g * bo;
    uint32_t nb = 0;
    for (uint32_t j = 0; j < 32; ++j) {
      const uint64_t i = g * 32 + j;
      uint32_t x = 0;
      if (i < n_out) {
        K v;
        if (i < a.n_main) {
          uint32_t c = packed_code(a.main_words, a.main_words_n, i, a.b);
          if (c >= a.m) {
            flag_status(a.status, ST_CODE);
            c = (uint32_t)(a.m - 1);
          }
          v = load_key(um + c);
        } else {
          uint32_t c = __ldg(a.dcodes + (i - a.n_main));
          if (c >= a.d) {
            flag_status(a.status, ST_CODE);
            c = (uint32_t)(a.d - 1);
          }
          v = load_key(dd + c);
        }
        // Eq. 5: the position of the value in U' (the first entry not below it)
        uint64_t lo = 0, hi = u;
        while (lo < hi) {
          const uint64_t mid = (lo + hi) >> 1;
          if (key_lt(load_key(un + mid), v)) lo = mid + 1;
          else hi = mid;
        }
        x = (uint32_t)lo;
      }
      acc |= (uint64_t)x << nb;
      nb += bo;
      if (nb >= 32) {
        if (w < out_total) a.out_words[w] = (uint32_t)acc;
        ++w;
        acc >>= 32;
        nb -= 32;
      }
    }
    // the stream is padded with zeros to a whole 16-byte unit
    if (g == groups - 1)
      for (uint64_t z = groups * bo; z < out_total; ++z) a.out_words[z] = 0;
  }
}

bool aligned_to(const void* p, size_t n) { return (reinterpret_cast<uintptr_t>(p) & (n - 1)) == 0; }

}  // namespace

}  // namespace dm

extern "C" dm_status dm_reencode_search(dm_ctx* ctx, const dm_column_in* in, const dm_column_out* out,
                                        void* stream) {
  using dm::aligned_to;
  if (!ctx || !in || !out) return DM_EINVAL;
  const uint32_t w = in->value_bytes;
  if ((w != 4 && w != 8 && w != 16) || in->main_bits > 32) return DM_EINVAL;
  const uint64_t m = in->main_dict_len, d = in->delta_dict_len;
  const uint64_t n_out = in->main_rows + in->delta_rows;
  if ((in->main_rows && (!m || !in->main_dict || (in->main_bits && !in->main_packed))) ||
      (in->delta_rows && (!d || !in->delta_dict || !in->delta_codes)))
    return DM_EINVAL;
  if (in->main_bits < dm_bits_for(m) || m + d > (1ull << 32)) return DM_EINVAL;
  const size_t ka = w;
  if ((m && !aligned_to(in->main_dict, ka)) || (d && !aligned_to(in->delta_dict, ka))) return DM_EINVAL;
  if (in->main_packed && !aligned_to(in->main_packed, 16)) return DM_EINVAL;
  if (!out->d_new_dict_len || !out->d_new_bits) return DM_EINVAL;
  if (n_out && (!out->new_dict || !out->new_packed || !aligned_to(out->new_packed, 16) ||
                !aligned_to(out->new_dict, ka)))
    return DM_EINVAL;
  if (n_out == 0) return DM_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DM_ECUDA;
  dm::SearchArgs a{};
  a.main_words = static_cast<const uint32_t*>(in->main_packed);
  a.main_words_n = dm_packed_bytes(in->main_rows, in->main_bits) / 4;
  a.b = in->main_bits;
  a.n_main = in->main_rows;
  a.dcodes = in->delta_codes;
  a.n_delta = in->delta_rows;
  a.um = in->main_dict;
  a.m = m;
  a.dd = in->delta_dict;
  a.d = d;
  a.unew = out->new_dict;
  a.d_u = out->d_new_dict_len;
  a.d_bits = out->d_new_bits;
  a.max_bits = dm_bits_for(m + d);
  a.out_words = static_cast<uint32_t*>(out->new_packed);
  a.status = ctx->status;
  const uint64_t groups = (n_out + 31) / 32;
  const uint64_t want = (groups + 255) / 256, cap = (uint64_t)ctx->sm_count * 8;
  const uint32_t grid = (uint32_t)(want < cap ? want : cap);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (w) {
    case 4: dm::reencode_search_kernel<4><<<grid, 256, 0, s>>>(a); break;
    case 8: dm::reencode_search_kernel<8><<<grid, 256, 0, s>>>(a); break;
    default: dm::reencode_search_kernel<16><<<grid, 256, 0, s>>>(a); break;
  }
  ++ctx->launches;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) ctx->last_error = e;
  return e == cudaSuccess ? DM_OK : DM_ECUDA;
}
