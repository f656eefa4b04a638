// Step 1(a): sort the delta dictionary (Section 5.1; the tuple-id map of
// Section 5.3 becomes perm[j] = insertion code of U_D[j]).
//
// The paper walks the leaves of a CSB+ tree kept during inserts; here the
// delta dictionary is a plain insertion-order array, so Step 1(a) is a
// stable LSD radix sort of (key, insertion code) pairs with 8-bit digits:
//   * one histogram kernel counts the digits of every pass at once;
//   * one "onesweep" kernel per digit pass ranks each 2048-key tile in
//     shared memory (warp match + per-warp counters, stable), finds the
//     tile's global offset per digit by decoupled look-back over earlier
//     tiles (bounded spins), and scatters.
// A pass whose digit is the same for every key is skipped on the device
// (the histogram shows it); which buffer holds the result is therefore
// known only on the device and is published in two pointer slots.
#include "dm_common.cuh"
#include "dm_internal.h"

namespace dm {

namespace {

template <int W>
__global__ void __launch_bounds__(256) rs_hist_kernel(const typename KeyOf<W>::T* __restrict__ keys,
                                                      uint64_t d, uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[W * 256];
  for (uint32_t i = threadIdx.x; i < W * 256; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < d;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    auto k = load_key(keys + idx);
#pragma unroll
    for (int p = 0; p < W; ++p) atomicAdd(&sh[p * 256 + key_digit(k, p)], 1u);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < W * 256; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Which passes run: pass q runs when its digit is not constant over the keys;
// if none does, the last pass runs anyway so that the result is always in a
// ping-pong buffer.  Returns the mask of running passes (uniform over the block).
template <int W>
__device__ uint32_t running_passes(const uint32_t* hist, uint64_t d) {
  uint32_t mask = 0;
#pragma unroll 1
  for (int q = 0; q < W; ++q) {
    int full = __syncthreads_or((uint64_t)hist[q * 256 + threadIdx.x] == d);
    if (!full) mask |= 1u << q;
  }
  if (mask == 0) mask = 1u << (W - 1);
  return mask;
}

template <int W>
__global__ void __launch_bounds__(RS_THREADS) rs_pass_kernel(SortArgs a, int pass) {
  using K = typename KeyOf<W>::T;
  __shared__ uint32_t s_whist[RS_THREADS / 32][256];
  __shared__ uint32_t s_base[256];
  __shared__ uint32_t s_wsum[RS_THREADS / 32];
  __shared__ uint32_t s_tile;

  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t d = a.d;

  const uint32_t run = running_passes<W>(a.hist, d);
  if (!((run >> pass) & 1u)) return;
  const int e = __popc(run & ((1u << pass) - 1u));      // running passes before this one
  const int last = 31 - __clz(run);

  // select ping-pong buffers without indexing the parameter arrays
  const bool odd = e & 1;
  const K* src_k = e == 0 ? static_cast<const K*>(a.in_keys) : static_cast<const K*>(odd ? a.keys[0] : a.keys[1]);
  const uint32_t* src_v = e == 0 ? nullptr : (odd ? a.vals[0] : a.vals[1]);
  K* dst_k = static_cast<K*>(odd ? a.keys[1] : a.keys[0]);
  uint32_t* dst_v = odd ? a.vals[1] : a.vals[0];

  // exclusive scan of this pass's histogram -> first slot of every digit
  const uint32_t hval = a.hist[pass * 256 + tid];
  uint32_t inc = hval;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t n = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= (uint32_t)o) inc += n;
  }
  if (lane == 31) s_wsum[warp] = inc;
  for (uint32_t i = tid; i < (RS_THREADS / 32) * 256; i += RS_THREADS) (&s_whist[0][0])[i] = 0;
  if (tid == 0) s_tile = atomicAdd(&a.counters[pass], 1u);
  __syncthreads();
  uint32_t bstart = inc - hval;
  for (uint32_t w = 0; w < warp; ++w) bstart += s_wsum[w];
  const uint32_t tile = s_tile;

  // load: warp w owns tile items [256w, 256w + 256), round r covers 32 of them
  K key[RS_ITEMS];
  uint32_t val[RS_ITEMS], dig[RS_ITEMS], rank[RS_ITEMS];
  const uint64_t base = (uint64_t)tile * RS_TILE + warp * (RS_ITEMS * 32) + lane;
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    uint64_t idx = base + r * 32;
    bool ok = idx < d;
    if (ok) {
      key[r] = load_key(src_k + idx);
      val[r] = src_v ? __ldg(src_v + idx) : (uint32_t)idx;
      dig[r] = key_digit(key[r], pass);
    } else {
      key[r] = K{};
      val[r] = 0;
      dig[r] = 256;
    }
  }

  // stable rank inside the warp: equal digits of one round are peers,
  // rounds are processed in item order
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    uint32_t peers = __match_any_sync(0xFFFFFFFFu, dig[r]);
    uint32_t leader = __ffs(peers) - 1;
    uint32_t cnt = 0;
    if (lane == leader && dig[r] < 256) {
      cnt = s_whist[warp][dig[r]];
      s_whist[warp][dig[r]] = cnt + __popc(peers);
    }
    cnt = __shfl_sync(0xFFFFFFFFu, cnt, leader);
    rank[r] = cnt + __popc(peers & lanemask_lt());
    __syncwarp();
  }
  __syncthreads();

  // per digit (thread = digit): warp offsets inside the tile, tile count
  uint32_t tcount = 0;
#pragma unroll
  for (int w = 0; w < RS_THREADS / 32; ++w) {
    uint32_t c = s_whist[w][tid];
    s_whist[w][tid] = tcount;
    tcount += c;
  }

  // decoupled look-back over earlier tiles, digit `tid`
  uint32_t* lb = a.lookback + (uint64_t)pass * a.ntiles * 256;
  uint32_t excl = 0;
  if (tile == 0) {
    st_volatile(&lb[tid], LB_INC32 | tcount);
  } else {
    st_volatile(&lb[(uint64_t)tile * 256 + tid], LB_AGG32 | tcount);
    int64_t p = (int64_t)tile - 1;
    uint32_t spins = 0;
    bool done = false;
    while (!done && p >= 0) {
      // eight predecessors per step: independent loads
      uint32_t v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = (p - q >= 0) ? ld_volatile(&lb[(uint64_t)(p - q) * 256 + tid]) : LB_INC32;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (!done) {
          while ((v[q] >> 30) == 0) {              // not published yet
            if (++spins > kSpinLimit) {
              flag_status(a.status, ST_TIMEOUT);
              v[q] = LB_INC32;
              break;
            }
            if (spins > 32) __nanosleep(64);
            v[q] = ld_volatile(&lb[(uint64_t)(p - q) * 256 + tid]);
          }
          excl += v[q] & LB_MASK32;
          if ((v[q] >> 30) == 2) done = true;
        }
      }
      p -= 8;
    }
    st_volatile(&lb[(uint64_t)tile * 256 + tid], LB_INC32 | (excl + tcount));
  }
  s_base[tid] = bstart + excl;
  __syncthreads();

#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    if (dig[r] < 256) {
      uint64_t pos = (uint64_t)s_base[dig[r]] + s_whist[warp][dig[r]] + rank[r];
      if (pos < d) {
        dst_k[pos] = key[r];
        dst_v[pos] = val[r];
      } else {
        flag_status(a.status, ST_TIMEOUT);
      }
    }
  }
  if (pass == last && tile == 0 && tid == 0) {
    a.final_slot[0] = dst_k;
    a.final_slot[1] = dst_v;
  }
}

template <int W>
__global__ void rs_copy_kernel(void* const* slot, uint64_t d, typename KeyOf<W>::T* keys_out,
                               uint32_t* perm_out) {
  using K = typename KeyOf<W>::T;
  const K* k = static_cast<const K*>(slot[0]);
  const uint32_t* v = static_cast<const uint32_t*>(slot[1]);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (uint64_t)gridDim.x * blockDim.x) {
    keys_out[i] = k[i];
    perm_out[i] = v[i];
  }
}

template <int W>
cudaError_t launch_sort_w(const SortArgs& a, cudaStream_t s, uint32_t sm_count, uint64_t* launches) {
  using K = typename KeyOf<W>::T;
  uint32_t hblocks = (uint32_t)((a.d + 255) / 256);
  if (hblocks > sm_count * 4) hblocks = sm_count * 4;
  if (hblocks == 0) hblocks = 1;
  rs_hist_kernel<W><<<hblocks, 256, 0, s>>>(static_cast<const K*>(a.in_keys), a.d, a.hist);
  ++*launches;
  for (int p = 0; p < W; ++p) {
    rs_pass_kernel<W><<<a.ntiles, RS_THREADS, 0, s>>>(a, p);
    ++*launches;
  }
  return cudaGetLastError();
}

}  // namespace

uint32_t sort_tiles(uint64_t d) { return (uint32_t)((d + RS_TILE - 1) / RS_TILE); }

uint64_t sort_zeroed_words(uint32_t w, uint64_t d) {
  return (uint64_t)w * 256 + w + (uint64_t)w * sort_tiles(d) * 256;
}

cudaError_t launch_sort(uint32_t w, const SortArgs& a, cudaStream_t s, uint32_t sm_count, uint64_t* launches) {
  switch (w) {
    case 4: return launch_sort_w<4>(a, s, sm_count, launches);
    case 8: return launch_sort_w<8>(a, s, sm_count, launches);
    case 16: return launch_sort_w<16>(a, s, sm_count, launches);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_sort_copy_out(uint32_t w, void** final_slot, uint64_t d, void* ud_out, uint32_t* perm_out,
                                 cudaStream_t s, uint64_t* launches) {
  uint32_t blocks = (uint32_t)((d + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  if (blocks == 0) return cudaSuccess;
  ++*launches;
  switch (w) {
    case 4: rs_copy_kernel<4><<<blocks, 256, 0, s>>>(final_slot, d, static_cast<uint32_t*>(ud_out), perm_out); break;
    case 8: rs_copy_kernel<8><<<blocks, 256, 0, s>>>(final_slot, d, static_cast<uint64_t*>(ud_out), perm_out); break;
    case 16: rs_copy_kernel<16><<<blocks, 256, 0, s>>>(final_slot, d, static_cast<u128*>(ud_out), perm_out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace dm
