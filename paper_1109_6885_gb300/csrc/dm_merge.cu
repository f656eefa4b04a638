// Step 1(b) and Step 2(a): merge the sorted dictionaries U_M and U_D into
// the duplicate-free U', emit the translation tables X_M and X_D, and the
// new width E'_C (Section 5.1, Section 5.3, Eq. 4).
//
// The paper parallelises the two-pointer merge by cutting both inputs at
// N_T-quantiles, merging each part locally, and fixing the output offsets
// with a counter array and a prefix sum in three phases (Section 6.2.1).
// The GPU form keeps the quantile idea at tile granularity and does it in a
// single pass:
//   * tile t owns merged positions [2048t, 2048t + 2048); its cut of U_M
//     and U_D is found by a merge-path (co-rank) search, 33-ary per warp;
//   * each thread merges 8 positions out of shared memory (ties: the main
//     value first, so a value present in both sits main-then-delta);
//   * a position is a duplicate when its key equals the previous key in
//     merged order, which covers values in both dictionaries and repeated
//     values inside D_dict alike;
//   * new code of a position = (non-duplicates at or before it) - 1, found
//     from a block scan plus a decoupled look-back over earlier tiles;
//   * U'[code] receives each non-duplicate, X_M / X_D every position.
// The last tile publishes |U'| and E'_C = ceil(log2 |U'|) as device scalars.
#include <mutex>

#include "dm_common.cuh"
#include "dm_internal.h"

namespace dm {

namespace {

// Number of U_M entries among the first k merged positions (ties: U_M
// first).  Whole warp; 32 probes per round narrow the range 33-fold.
template <class K>
__device__ uint64_t corank_warp(const K* A, uint64_t m, const K* B, uint64_t d, uint64_t k) {
  const uint32_t lane = lane_id();
  uint64_t lo = k > d ? k - d : 0, hi = k < m ? k : m;
  while (hi - lo > 32) {
    uint64_t span = hi - lo;
    uint64_t c = lo + (span * (lane + 1)) / 33;
    bool p = key_le(load_key(A + c), load_key(B + (k - 1 - c)));
    uint32_t t = __popc(__ballot_sync(0xFFFFFFFFu, p));
    uint64_t c_below = __shfl_sync(0xFFFFFFFFu, c, t > 0 ? t - 1 : 0);
    uint64_t c_at = __shfl_sync(0xFFFFFFFFu, c, t < 32 ? t : 31);
    uint64_t nlo = t > 0 ? c_below + 1 : lo;
    uint64_t nhi = t < 32 ? c_at : hi;
    lo = nlo;
    hi = nhi < nlo ? nlo : nhi;
  }
  uint64_t c = lo + lane;
  bool p = c < hi && key_le(load_key(A + c), load_key(B + (k - 1 - c)));
  return lo + __popc(__ballot_sync(0xFFFFFFFFu, p));
}

template <int W>
__global__ void __launch_bounds__(MG_THREADS) merge_kernel(MergeArgs args) {
  using K = typename KeyOf<W>::T;
  __shared__ K s_keys[MG_TILE];
  __shared__ K s_last[MG_THREADS];
  __shared__ uint32_t s_wsum[MG_THREADS / 32];
  __shared__ uint64_t s_cut[2];
  __shared__ uint64_t s_excl;
  __shared__ uint32_t s_tile;
  __shared__ K s_pred;

  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const K* A = static_cast<const K*>(args.a);
  const K* B = args.b_slot ? static_cast<const K*>(args.b_slot[0]) : static_cast<const K*>(args.b);
  const uint32_t* perm = args.b_slot ? static_cast<const uint32_t*>(args.b_slot[1]) : args.perm;
  const uint64_t m = args.m, d = args.d, n = m + d;

  if (tid == 0) s_tile = atomicAdd(args.counter, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t k0 = (uint64_t)tile * MG_TILE;
  const uint64_t k1 = k0 + MG_TILE < n ? k0 + MG_TILE : n;
  if (warp < 2) {
    uint64_t c = corank_warp(A, m, B, d, warp == 0 ? k0 : k1);
    if (lane == 0) s_cut[warp] = c;
  }
  __syncthreads();
  const uint64_t i0 = s_cut[0], i1 = s_cut[1];
  const uint64_t j0 = k0 - i0, j1 = k1 - i1;
  const uint32_t na = (uint32_t)(i1 - i0), nb = (uint32_t)(j1 - j0), nt = na + nb;
  for (uint32_t x = tid; x < na; x += MG_THREADS) s_keys[x] = load_key(A + i0 + x);
  for (uint32_t x = tid; x < nb; x += MG_THREADS) s_keys[na + x] = load_key(B + j0 + x);
  if (tid == 0 && k0 > 0) {
    // the key at merged position k0 - 1 is the larger of the two candidates
    if (i0 > 0 && j0 > 0) s_pred = key_max(load_key(A + i0 - 1), load_key(B + j0 - 1));
    else s_pred = i0 > 0 ? load_key(A + i0 - 1) : load_key(B + j0 - 1);
  }
  __syncthreads();
  const K* sA = s_keys;
  const K* sB = s_keys + na;

  // U_M must be strictly increasing
  for (uint32_t x = tid; x < na; x += MG_THREADS) {
    if (i0 + x == 0) continue;
    K prev = x > 0 ? sA[x - 1] : load_key(A + i0 - 1);
    if (!key_lt(prev, sA[x])) flag_status(args.status, ST_UNSORTED);
  }

  // this thread's 8 merged positions: cut inside the tile, then merge
  const uint32_t kk = tid * MG_ITEMS < nt ? tid * MG_ITEMS : nt;
  const uint32_t cnt = kk + MG_ITEMS < nt ? MG_ITEMS : nt - kk;
  uint32_t lo = kk > nb ? kk - nb : 0, hi = kk < na ? kk : na;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (key_le(sA[mid], sB[kk - 1 - mid])) lo = mid + 1;
    else hi = mid;
  }
  uint32_t ia = lo, ib = kk - lo;
  K key[MG_ITEMS];
  K last{};
  uint32_t src[MG_ITEMS];  // bit 31: from U_D; low bits: index inside the tile's segment
#pragma unroll
  for (int it = 0; it < MG_ITEMS; ++it) {
    if ((uint32_t)it < cnt) {
      bool takeA = ib >= nb || (ia < na && key_le(sA[ia], sB[ib]));
      if (takeA) {
        key[it] = sA[ia];
        src[it] = ia++;
      } else {
        key[it] = sB[ib];
        src[it] = 0x80000000u | ib++;
      }
      last = key[it];
    } else {
      key[it] = K{};
      src[it] = 0;
    }
  }
  if (cnt > 0) s_last[tid] = last;
  __syncthreads();

  // duplicates: equal to the previous key in merged order
  uint32_t dupmask = 0, nondup = 0;
  {
    bool has_prev = tid > 0 ? true : k0 > 0;
    K prev = tid > 0 ? s_last[tid - 1] : s_pred;
#pragma unroll
    for (int it = 0; it < MG_ITEMS; ++it) {
      if ((uint32_t)it < cnt) {
        bool dup = has_prev && key_eq(key[it], prev);
        dupmask |= (uint32_t)dup << it;
        nondup += !dup;
        prev = key[it];
        has_prev = true;
      }
    }
  }

  // block exclusive scan of the non-duplicate counts
  uint32_t inc = nondup;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t v = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= (uint32_t)o) inc += v;
  }
  if (lane == 31) s_wsum[warp] = inc;
  __syncthreads();
  uint32_t texcl = inc - nondup, ttotal = 0;
#pragma unroll
  for (int w = 0; w < MG_THREADS / 32; ++w) {
    uint32_t sw = s_wsum[w];
    if ((uint32_t)w < warp) texcl += sw;
    ttotal += sw;
  }

  // decoupled look-back over earlier tiles (warp 0, 32 tiles per step)
  if (warp == 0) {
    uint64_t excl = 0;
    if (tile == 0) {
      if (lane == 0) st_volatile(&args.lookback[0], LB_INC64 | ttotal);
    } else {
      if (lane == 0) st_volatile(&args.lookback[tile], LB_AGG64 | ttotal);
      int64_t top = (int64_t)tile - 1;  // highest tile not yet accounted for
      uint32_t spins = 0;
      while (top >= 0) {
        int64_t p = top - lane;
        uint64_t v = p >= 0 ? ld_volatile(&args.lookback[p]) : LB_INC64;
        uint32_t ready = __ballot_sync(0xFFFFFFFFu, (v >> 62) != 0);
        uint32_t incl = __ballot_sync(0xFFFFFFFFu, (v >> 62) == 2);
        // lanes up to the nearest inclusive prefix must all be published
        uint32_t need = incl ? ((incl & (0u - incl)) << 1) - 1 : 0xFFFFFFFFu;
        if ((ready & need) != need) {
          if (++spins > kSpinLimit) {
            if (lane == 0) flag_status(args.status, ST_TIMEOUT);
            break;
          }
          if (spins > 32) __nanosleep(64);
          continue;
        }
        uint64_t part = (need >> lane) & 1u ? (v & LB_MASK64) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
        excl += part;
        if (incl) break;
        top -= 32;
      }
      if (lane == 0) st_volatile(&args.lookback[tile], LB_INC64 | (excl + ttotal));
    }
    if (lane == 0) s_excl = excl;
  }
  __syncthreads();

  // codes and writes
  uint64_t c = s_excl + texcl;
  K* unew = static_cast<K*>(args.unew);
#pragma unroll
  for (int it = 0; it < MG_ITEMS; ++it) {
    if ((uint32_t)it < cnt) {
      bool dup = (dupmask >> it) & 1u;
      c += !dup;
      uint64_t code = c - 1;
      if (code >= n) {
        flag_status(args.status, ST_TIMEOUT);
        continue;
      }
      if (!dup) unew[code] = key[it];
      uint32_t s = src[it];
      if (s & 0x80000000u) {
        uint32_t pj = __ldg(perm + j0 + (s & 0x7FFFFFFFu));
        if (pj < d) args.xd[pj] = (uint32_t)code;
        else flag_status(args.status, ST_CODE);
      } else {
        args.xm[i0 + s] = (uint32_t)code;
      }
    }
  }
  if (tile == args.ntiles - 1 && tid == 0) {
    uint64_t u = s_excl + ttotal;
    *args.d_u = u;
    *args.d_bits = bits_for(u);
  }
}

template <int W>
cudaError_t launch_merge_w(const MergeArgs& a, cudaStream_t s, uint64_t* launches) {
  merge_kernel<W><<<a.ntiles, MG_THREADS, 0, s>>>(a);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace

uint32_t merge_tiles(uint64_t n) { return (uint32_t)((n + MG_TILE - 1) / MG_TILE); }

cudaError_t launch_merge(uint32_t w, const MergeArgs& a, cudaStream_t s, uint64_t* launches) {
  switch (w) {
    case 4: return launch_merge_w<4>(a, s, launches);
    case 8: return launch_merge_w<8>(a, s, launches);
    case 16: return launch_merge_w<16>(a, s, launches);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dm

// ---------------------------------------------------------------- no-alloc variant
// Scratch of dm_merge_dicts_noalloc: the look-back words of every tile of a
// merge of up to DM_NOALLOC_MAX_ENTRIES entries, then the tile counter.  It
// is static device memory of this library, present on every device that
// loads it; host code must not pass the symbol itself to a kernel (on the
// host it only names a shadow), so the device address is looked up once per
// device with cudaGetSymbolAddress.
namespace {
constexpr uint32_t kNoAllocTiles = (DM_NOALLOC_MAX_ENTRIES + dm::MG_TILE - 1) / dm::MG_TILE;
static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocTiles + 1];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
uint64_t* g_noalloc_addr[kMaxDevices] = {};
}  // namespace

extern "C" dm_status dm_merge_dicts_noalloc(uint32_t w, const void* main_dict, uint64_t m, const void* ud,
                                            const uint32_t* perm, uint64_t d, void* new_dict, uint32_t* x_main,
                                            uint32_t* x_delta, uint64_t* d_u, uint32_t* d_bits,
                                            uint32_t* d_status, void* stream) {
  if ((w != 4 && w != 8 && w != 16) || !d_u || !d_bits) return DM_EINVAL;
  if (m + d > DM_NOALLOC_MAX_ENTRIES) return DM_EINVAL;
  if ((m && (!main_dict || !x_main)) || (d && (!ud || !perm || !x_delta)) || (m + d && !new_dict)) return DM_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DM_ECUDA;
  uint64_t* scratch = nullptr;
  {
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return DM_ECUDA;
      g_noalloc_addr[dev] = static_cast<uint64_t*>(p);
    }
    scratch = g_noalloc_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (m + d == 0) {
    if (cudaMemsetAsync(d_u, 0, 8, s) != cudaSuccess || cudaMemsetAsync(d_bits, 0, 4, s) != cudaSuccess)
      return DM_ECUDA;
    return DM_OK;
  }
  const uint32_t tiles = dm::merge_tiles(m + d);
  // look-back words and tile counter must start at zero; the array keeps
  // whatever the previous call left
  if (cudaMemsetAsync(scratch, 0, (size_t)(tiles + 1) * sizeof(uint64_t), s) != cudaSuccess) return DM_ECUDA;
  dm::MergeArgs a{};
  a.a = main_dict;
  a.m = m;
  a.b = ud;
  a.perm = perm;
  a.b_slot = nullptr;
  a.d = d;
  a.unew = new_dict;
  a.xm = x_main;
  a.xd = x_delta;
  a.d_u = d_u;
  a.d_bits = d_bits;
  a.lookback = scratch;
  a.counter = reinterpret_cast<uint32_t*>(scratch + tiles);
  a.ntiles = tiles;
  a.status = d_status;
  uint64_t launches = 0;
  return dm::launch_merge(w, a, s, &launches) == cudaSuccess ? DM_OK : DM_ECUDA;
}
