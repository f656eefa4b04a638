// Step 2(b): re-encode the main vector through X_M and append the delta rows
// through X_D at the new width (Section 5.3, Eq. 11; parallel form Section
// 6.2.2, which splits the N'_M output tuples evenly over threads).
//
// GPU form.  A group of 32 consecutive codes at b bits is exactly b 32-bit
// words, in the input and (at b' bits) in the output, so groups are
// independent and aligned.  A warp owns a tile of 32 groups (1024 codes);
// lane l owns group l of the tile and keeps its 32 codes in registers.
//   * tiles that are entirely main rows stream in through a 3-stage
//     pipeline of bulk (TMA) copies global -> shared, one per tile, each
//     completing on its own mbarrier; lanes read their b words from shared
//     memory with the widest aligned loads b allows;
//   * unpacking is specialised at compile time for b (the kernel is a
//     template over b = 0..32), so each code costs one or two shifts;
//   * codes are range-checked against |U_M| (clamped and flagged, never
//     faulting), then gathered from X_M — out of shared memory when X_M is
//     small, else through the read-only L1/L2 path (the paper's observation
//     that X fits in cache or not, Section 7.3, becomes smem vs L2 here);
//   * b' is produced on the device by Step 2(a), so the kernel reads it and
//     branches (warp-uniformly) to a packer specialised for b' = b or
//     b' = b + 1, or to a runtime-width packer otherwise;
//   * packed rows go to a double-buffered shared tile that one bulk copy
//     stores to global memory; the last tile is stored with clipped plain
//     stores and zero padding up to the stream's 16-byte end.
// Tiles that hold delta rows or the main/delta boundary use a plain path.
#include <mutex>

#include "dm_common.cuh"
#include "dm_internal.h"

namespace dm {

namespace {

constexpr int RE_WARPS = 8;
constexpr int RE_THREADS = RE_WARPS * 32;
constexpr int RE_STAGES = 3;
constexpr uint32_t RE_TILE = 1024;          // codes per warp tile
constexpr uint32_t RE_XSMEM_MAX = 16384;    // X_M entries staged in shared memory at most

template <int B>
__device__ __forceinline__ void load_row(const uint32_t* row, uint32_t (&w)[B > 0 ? B : 1]) {
  if constexpr (B == 0) {
    w[0] = 0;
  } else if constexpr (B % 4 == 0) {
#pragma unroll
    for (int q = 0; q < B / 4; ++q) {
      uint4 v = reinterpret_cast<const uint4*>(row)[q];
      w[4 * q] = v.x;
      w[4 * q + 1] = v.y;
      w[4 * q + 2] = v.z;
      w[4 * q + 3] = v.w;
    }
  } else if constexpr (B % 2 == 0) {
#pragma unroll
    for (int q = 0; q < B / 2; ++q) {
      uint2 v = reinterpret_cast<const uint2*>(row)[q];
      w[2 * q] = v.x;
      w[2 * q + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < B; ++q) w[q] = row[q];
  }
}

// 32 codes of b = B bits out of B words (LSB-first).
template <int B>
__device__ __forceinline__ void unpack32(const uint32_t (&w)[B > 0 ? B : 1], uint32_t (&c)[32]) {
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    if constexpr (B == 0) {
      c[j] = 0;
    } else {
      const int bit = j * B, k = bit >> 5, s = bit & 31;
      uint32_t v;
      if (s + B <= 32) v = w[k] >> s;
      else v = __funnelshift_r(w[k], w[(k + 1 < B) ? k + 1 : k], s);
      c[j] = (B == 32) ? v : (v & ((1u << (B & 31)) - 1u));
    }
  }
}

// 32 values of BO bits into BO words at `row` (shared memory).
template <int BO>
__device__ __forceinline__ void pack32(const uint32_t (&x)[32], uint32_t* row) {
  if constexpr (BO == 0) {
    return;
  } else {
    uint32_t o[BO];
#pragma unroll
    for (int k = 0; k < BO; ++k) o[k] = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int bit = j * BO, k = bit >> 5, s = bit & 31;
      o[k] |= x[j] << s;
      if (s + BO > 32) o[(k + 1 < BO) ? k + 1 : k] |= x[j] >> ((32 - s) & 31);
    }
    if constexpr (BO % 4 == 0) {
#pragma unroll
      for (int q = 0; q < BO / 4; ++q)
        reinterpret_cast<uint4*>(row)[q] = make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    } else if constexpr (BO % 2 == 0) {
#pragma unroll
      for (int q = 0; q < BO / 2; ++q) reinterpret_cast<uint2*>(row)[q] = make_uint2(o[2 * q], o[2 * q + 1]);
    } else {
#pragma unroll
      for (int q = 0; q < BO; ++q) row[q] = o[q];
    }
  }
}

// Runtime-width packer (any b' in 0..32): exactly bo words.
__device__ __forceinline__ void pack32_generic(const uint32_t (&x)[32], uint32_t bo, uint32_t* row) {
  if (bo == 0) return;
  uint64_t acc = 0;
  uint32_t nb = 0, k = 0;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    acc |= (uint64_t)x[j] << nb;
    nb += bo;
    if (nb >= 32) {
      row[k++] = (uint32_t)acc;
      acc >>= 32;
      nb -= 32;
    }
  }
}

// Code i of a packed stream (bounds-checked plain loads; boundary tiles).
__device__ __forceinline__ uint32_t code_at(const uint32_t* words, uint64_t nwords, uint64_t i, uint32_t b) {
  if (b == 0) return 0;
  uint64_t bit = i * b, k = bit >> 5;
  uint32_t lo = k < nwords ? __ldg(words + k) : 0u;
  uint32_t hi = k + 1 < nwords ? __ldg(words + k + 1) : 0u;
  uint32_t v = __funnelshift_r(lo, hi, (uint32_t)(bit & 31));
  return b == 32 ? v : (v & ((1u << b) - 1u));
}

struct Layout {
  uint32_t in_words;    // words of one input stage (32 * b)
  uint32_t out_words;   // words of one output buffer (32 * max_bits)
  uint32_t x_entries;   // X_M entries staged in shared memory (0 = none)
  uint32_t generic;     // 1: plain per-code path and runtime-width packer on every tile
};

__host__ __device__ __forceinline__ uint32_t round4(uint32_t v) { return (v + 3u) & ~3u; }

__host__ __device__ __forceinline__ uint32_t smem_bytes(const Layout& L) {
  uint32_t bars = RE_WARPS * RE_STAGES * 8;
  uint32_t per_warp = RE_STAGES * round4(L.in_words) + 2 * round4(L.out_words);
  return ((bars + 127) & ~127u) + RE_WARPS * per_warp * 4 + round4(L.x_entries) * 4;
}

template <int B>
__global__ void __launch_bounds__(RE_THREADS) reencode_kernel(ReencodeArgs a, Layout L) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem) + warp * RE_STAGES;
  uint32_t* region = reinterpret_cast<uint32_t*>(smem + ((RE_WARPS * RE_STAGES * 8 + 127) & ~127u));
  const uint32_t per_warp = RE_STAGES * round4(L.in_words) + 2 * round4(L.out_words);
  uint32_t* wbase = region + warp * per_warp;
  uint32_t* s_x = region + RE_WARPS * per_warp;

  const uint32_t bo = *a.d_bits;
  if (bo > a.max_bits) {
    if (threadIdx.x == 0) flag_status(a.status, ST_WIDTH);
    return;
  }
  const uint64_t n_out = a.n_main + a.n_delta;
  const uint64_t out_total = ((n_out * bo + 127) / 128) * 4;
  const uint64_t n_tiles = (n_out + RE_TILE - 1) / RE_TILE;
  const uint64_t full_tiles = L.generic ? 0 : a.n_main / RE_TILE;
  const uint64_t gw = (uint64_t)blockIdx.x * RE_WARPS + warp;
  const uint64_t nw = (uint64_t)gridDim.x * RE_WARPS;
  constexpr uint32_t in_bytes = 128u * B;
  const bool x_smem = L.x_entries > 0;

  if (x_smem) {
    for (uint32_t i = threadIdx.x; i < L.x_entries; i += RE_THREADS) s_x[i] = __ldg(a.xm + i);
    __syncthreads();
  }
  if (lane == 0) {
    for (int s = 0; s < RE_STAGES; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncwarp();
  if constexpr (B > 0) {
    if (lane == 0) {
      for (int s = 0; s < RE_STAGES; ++s) {
        uint64_t t = gw + (uint64_t)s * nw;
        if (t < full_tiles) {
          mbar_arrive_expect_tx(&bars[s], in_bytes);
          bulk_g2s(wbase + s * round4(L.in_words), a.main_words + t * 32 * B, in_bytes, &bars[s]);
        }
      }
    }
  }

  bool timed_out = false;
  uint32_t it = 0;
  for (uint64_t t = gw; t < n_tiles; t += nw, ++it) {
    uint32_t x[32];
    if (t < full_tiles) {
      uint32_t c[32];
      if constexpr (B > 0) {
        const uint32_t st = it % RE_STAGES;
        uint32_t* stage = wbase + st * round4(L.in_words);
        const bool ok = mbar_wait(&bars[st], (it / RE_STAGES) & 1u, a.status);
        if (!__all_sync(0xFFFFFFFFu, ok)) {
          timed_out = true;
          break;
        }
        uint32_t w[B];
        load_row<B>(stage + lane * B, w);
        __syncwarp();
        if (lane == 0) {
          uint64_t tn = t + (uint64_t)RE_STAGES * nw;
          if (tn < full_tiles) {
            mbar_arrive_expect_tx(&bars[st], in_bytes);
            bulk_g2s(stage, a.main_words + tn * 32 * B, in_bytes, &bars[st]);
          }
        }
        unpack32<B>(w, c);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) c[j] = 0;
      }
      uint32_t mx = 0;
#pragma unroll
      for (int j = 0; j < 32; ++j) mx = max(mx, c[j]);
      if (__any_sync(0xFFFFFFFFu, mx >= a.m)) {
        if (mx >= a.m) flag_status(a.status, ST_CODE);
#pragma unroll
        for (int j = 0; j < 32; ++j) c[j] = min(c[j], a.m - 1);
      }
      if (x_smem) {
#pragma unroll
        for (int j = 0; j < 32; ++j) x[j] = s_x[c[j]];
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) x[j] = __ldg(a.xm + c[j]);
      }
    } else {
      const uint64_t i0 = t * RE_TILE + lane * 32;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const uint64_t i = i0 + j;
        uint32_t v = 0;
        if (i < a.n_main) {
          uint32_t cc = code_at(a.main_words, a.main_words_n, i, B);
          if (cc >= a.m) {
            flag_status(a.status, ST_CODE);
            cc = a.m - 1;
          }
          v = __ldg(a.xm + cc);
        } else if (i < n_out) {
          uint32_t cc = __ldg(a.dcodes + (i - a.n_main));
          if (cc >= a.d) {
            flag_status(a.status, ST_CODE);
            cc = a.d - 1;
          }
          v = __ldg(a.xd + cc);
        }
        x[j] = v;
      }
    }

    uint32_t* ob = wbase + RE_STAGES * round4(L.in_words) + (it & 1u) * round4(L.out_words);
    if (lane == 0) bulk_wait_read<1>();
    __syncwarp();
    uint32_t* row = ob + lane * bo;
    if (L.generic) {
      pack32_generic(x, bo, row);
    } else if (bo == (uint32_t)B) {
      pack32<B>(x, row);
    } else if (B < 32 && bo == (uint32_t)B + 1) {
      pack32<(B < 32 ? B + 1 : 32)>(x, row);
    } else {
      pack32_generic(x, bo, row);
    }
    fence_proxy_async_smem();
    __syncwarp();
    const uint64_t w0 = t * 32 * bo;
    const uint32_t tile_words = 32 * bo;
    if (w0 + tile_words <= out_total) {
      if (lane == 0 && bo > 0) {
        bulk_s2g(a.out_words + w0, ob, tile_words * 4);
        bulk_commit();
      }
    } else {
      for (uint64_t q = lane; w0 + q < out_total; q += 32) a.out_words[w0 + q] = q < tile_words ? ob[q] : 0u;
    }
  }

  if constexpr (B > 0) {
    if (timed_out && lane == 0) {
      // let the copies already in flight land before the block exits
      for (uint32_t k = 0; k < RE_STAGES; ++k) {
        uint32_t i2 = it + k;
        uint64_t t2 = gw + (uint64_t)i2 * nw;
        if (t2 < full_tiles) mbar_wait(&bars[i2 % RE_STAGES], (i2 / RE_STAGES) & 1u, a.status);
      }
    }
  }
  if (lane == 0) bulk_wait_all();
  __syncwarp();
}

using KernelFn = void (*)(ReencodeArgs, Layout);

template <int B>
struct KernelTable {
  static void fill(KernelFn* t) {
    t[B] = reencode_kernel<B>;
    KernelTable<B - 1>::fill(t);
  }
};
template <>
struct KernelTable<-1> {
  static void fill(KernelFn*) {}
};

struct Registry {
  KernelFn fn[33];
  uint32_t smem_set[33];  // dynamic smem size already allowed per kernel
  std::mutex mu;
  Registry() {
    KernelTable<32>::fill(fn);
    for (auto& s : smem_set) s = 0;
  }
};

Registry& registry() {
  static Registry r;
  return r;
}

}  // namespace

cudaError_t launch_reencode(uint32_t b, const ReencodeArgs& a, cudaStream_t s, uint32_t sm_count, uint32_t flags,
                            uint64_t* launches) {
  if (b > 32 || a.max_bits > 32) return cudaErrorInvalidValue;
  const uint64_t n_out = a.n_main + a.n_delta;
  if (n_out == 0) return cudaSuccess;
  Layout L;
  L.in_words = 32 * b;
  L.out_words = 32 * (a.max_bits > b + 1 ? a.max_bits : b + 1);
  if (L.out_words > 32 * 32) L.out_words = 32 * 32;
  bool want_smem = (flags & DM_FLAG_X_SMEM) || (!(flags & DM_FLAG_X_GLOBAL) && a.m <= RE_XSMEM_MAX && a.n_main >= (1u << 20));
  L.x_entries = (want_smem && a.m <= RE_XSMEM_MAX && a.n_main > 0) ? a.m : 0;
  L.generic = (flags & DM_FLAG_GENERIC_REENCODE) ? 1u : 0u;
  const uint32_t bytes = smem_bytes(L);

  Registry& R = registry();
  KernelFn fn = R.fn[b];
  {
    std::lock_guard<std::mutex> g(R.mu);
    if (R.smem_set[b] < bytes) {
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e != cudaSuccess) return e;
      R.smem_set[b] = bytes;
    }
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, RE_THREADS, bytes);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t n_tiles = (n_out + RE_TILE - 1) / RE_TILE;
  uint64_t grid = (n_tiles + RE_WARPS - 1) / RE_WARPS;
  const uint64_t cap = (uint64_t)sm_count * per_sm;
  if (grid > cap) grid = cap;
  fn<<<(uint32_t)grid, RE_THREADS, bytes, s>>>(a, L);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace dm
