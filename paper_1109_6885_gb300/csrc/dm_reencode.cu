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
// Tiles of delta rows only read their codes with wide loads and map them
// through X_D; the tile at the main/delta boundary and a ragged last tile
// use a plain per-code path.
#include <string.h>

#include <algorithm>
#include <mutex>

#include "dm_common.cuh"
#include "dm_internal.h"
#include "dm_xdir.cuh"

namespace dm {

namespace {

constexpr uint32_t RE_STAGES_MAX = 4;
constexpr uint32_t RE_TILE = 1024;          // codes per warp tile
constexpr uint32_t RE_XSMEM_MAX = 16384;    // X_M entries staged in shared memory at most
// Above this many main codes X_M (4 bytes a code, 46 MB and more) starts to
// lose its place in L2 next to the streams, and the directory's crowded
// buckets read a byte table.  Below it a crowded code's X_M read is cheaper
// than the byte table's path (and Step 1 skips building the table): at 10M
// codes the merge is 10-50% faster without it, at 16M with dense steps 14%
// slower.
constexpr uint64_t RE_X8_MIN_CODES = 11u << 20;
// Input widths that can carry that many codes (the byte-table path is
// compiled into their kernels only).
constexpr bool RE_X8_B(int b) { return (1ull << b) > RE_X8_MIN_CODES; }
// Input widths whose columns can have more main codes than the direct table
// holds; only their kernels carry the directory lookup.  Without it a
// kernel fits 64 registers a thread, so two blocks can share an SM.
constexpr bool RE_DIR_B(int b) { return (1ull << b) > RE_XSMEM_MAX; }
constexpr int RE_BLOCKS_MIN(int b) { return RE_DIR_B(b) ? 1 : 2; }
// Input widths whose columns can have more main codes than the shared-memory
// directory covers; only their kernels carry the global directory lookup.
constexpr bool RE_GDIR_B(int b) { return (1ull << b) > ((uint64_t)RE_DIR_MAX << RE_DIR_SHIFT_MAX); }
// The global directory: one 8-byte entry per bucket of 2^s main codes
// (3 <= s <= 6, at most 4M entries, 32 MB, so that it stays in L2): the
// count c of new values below the bucket's first code, and the offsets in
// the bucket of its first four steps, one byte each in increasing order,
// GDIR_UNUSED past the last; GDIR_MANY marks a bucket of more than four.
// A step is a code where c grows; a code where it grows by two holds two.
// s is picked from |U_M| / |D_dict| (|D_dict| bounds the new values) for
// about 1.5 steps a bucket at most, so that few buckets are crowded.
constexpr uint32_t GDIR_SHIFT_MIN = 3, GDIR_SHIFT_MAX = 6;
constexpr uint64_t GDIR_MAX_ENTRIES = 1ull << 22;
constexpr uint32_t GDIR_UNUSED = 0x7Fu, GDIR_MANY = 0xFFFFFFFFu;
static_assert((1u << GDIR_SHIFT_MAX) <= GDIR_UNUSED, "offsets below the unused mark");

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
      if (B == 32) {
        c[j] = w[k];
      } else if (s + B == 32) {
        c[j] = w[k] >> s;                                        // the word's top field
      } else if (s + B < 32) {
        // field below the top: move it to the top, take the high B bits
        // (two multiplies, FMA pipe, instead of a shift and a mask)
        c[j] = __umulhi(w[k] * (1u << ((32 - s - B) & 31)), 1u << (B & 31));
      } else {
        const uint32_t v = __funnelshift_r(w[k], w[(k + 1 < B) ? k + 1 : k], s);
        c[j] = v & ((1u << (B & 31)) - 1u);
      }
    }
  }
}

// 32 values of BO bits into BO words at `row` (shared memory).  Fields do
// not overlap, so a field is added rather than ORed in: x * 2^s + word is
// one multiply-add (FMA pipe) instead of a shift and an OR (ALU pipe).  The
// part of a field that spills into the next word starts that word.
template <int BO>
__device__ __forceinline__ void pack32(const uint32_t (&x)[32], uint32_t* row) {
  if constexpr (BO == 0) {
    return;
  } else {
    uint32_t o[BO];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int bit = j * BO, k = bit >> 5, s = bit & 31;
      if (s == 0) o[k] = x[j];
      else o[k] = x[j] * (1u << s) + o[k];
      if (s + BO > 32) o[(k + 1 < BO) ? k + 1 : k] = x[j] >> ((32 - s) & 31);
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
  uint32_t x_mode;      // X_M lookup: 0 global gather, 1 direct table in smem, 2 directory in smem,
                        // 3 global directory (L2)
  uint32_t x_entries;   // mode 1: entries of X_M staged; mode 2: directory entries
  uint32_t dir_shift;   // modes 2, 3: main codes per directory bucket = 2^dir_shift
  uint32_t generic;     // 1: plain per-code path and runtime-width packer on every tile
  uint32_t stages;      // input bulk-copy stages per warp (2..4)
  uint32_t obufs;       // output staging buffers per warp (1..2)
};

constexpr uint32_t RE_WARPS_MAX = 16;
constexpr uint32_t RE_BAR_BYTES = RE_WARPS_MAX * RE_STAGES_MAX * 8;   // 512

__host__ __device__ __forceinline__ uint32_t round4(uint32_t v) { return (v + 3u) & ~3u; }

__host__ __device__ __forceinline__ uint32_t per_warp_words(const Layout& L) {
  return L.stages * round4(L.in_words) + L.obufs * round4(L.out_words);
}

__host__ __device__ __forceinline__ uint32_t smem_bytes(const Layout& L, uint32_t warps) {
  return RE_BAR_BYTES + warps * per_warp_words(L) * 4 + round4(L.x_entries) * 4;
}

// The X_M directory (see dm_xdir.cuh) built by a kernel of its own when
// Step 2(b) runs without the Step 1 kernel in front of it.
__global__ void xdir_build_kernel(const uint32_t* __restrict__ xm, uint32_t m, uint32_t s, uint32_t R,
                                  uint32_t* __restrict__ dir, uint8_t* __restrict__ x8) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  const bool use_x8 = x8 != nullptr && xdir_x8_pays<false>(xm, m, R);
  for (uint32_t b = t; b < R; b += nt) dir[b] = xdir_entry<false>(xm, m, s, b, use_x8);
  if (use_x8) xdir_x8_fill<false>(xm, m, s, x8, t, nt);
}

// The global directory from the finished X_M: per bucket of 2^s codes the
// count of new values below it, X_M[lo - 1] - (lo - 1), and the steps in
// it, X_M at its last code less that; with at most four, the k-th step's
// offset is the first code whose count reaches base + k (a binary search).
__global__ void gdir_build_kernel(const uint32_t* __restrict__ xm, uint32_t m, uint32_t s, uint64_t R,
                                  uint2* __restrict__ gdir) {
  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < R; b += nt) {
    const uint32_t lo = (uint32_t)(b << s);
    const uint32_t hi = (uint32_t)min((b + 1) << s, (uint64_t)m) - 1;
    const uint32_t base = lo == 0 ? 0u : __ldg(xm + lo - 1) - (lo - 1);
    const uint32_t cnt = (__ldg(xm + hi) - hi) - base;
    uint32_t offs = GDIR_UNUSED * 0x01010101u;
    if (cnt > 4) {
      offs = GDIR_MANY;
    } else {
      for (uint32_t k = 1; k <= cnt; ++k) {
        uint32_t l = lo, h = hi;
        while (l < h) {
          const uint32_t mid = l + ((h - l) >> 1);
          if (__ldg(xm + mid) - mid >= base + k) h = mid;
          else l = mid + 1;
        }
        const uint32_t sh = 8 * (k - 1);
        offs = (offs & ~(0xFFu << sh)) | ((l - lo) << sh);
      }
    }
    gdir[b] = make_uint2(offs, base);
  }
}

template <int B>
__global__ void __launch_bounds__(RE_WARPS_MAX * 32, RE_BLOCKS_MIN(B)) reencode_kernel(ReencodeArgs a, Layout L) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem) + warp * RE_STAGES_MAX;
  const uint32_t stages = L.stages;
  uint32_t* region = reinterpret_cast<uint32_t*>(smem + RE_BAR_BYTES);
  const uint32_t pw = per_warp_words(L);
  uint32_t* wbase = region + warp * pw;
  uint32_t* s_x = region + nwarps * pw;

  const uint32_t bo = *a.d_bits;
  if (bo > a.max_bits) {
    if (threadIdx.x == 0) flag_status(a.status, ST_WIDTH);
    return;
  }
  const uint64_t n_out = a.n_main + a.n_delta;
  const uint64_t out_total = ((n_out * bo + 127) / 128) * 4;
  const uint64_t n_tiles = (n_out + RE_TILE - 1) / RE_TILE;
  const uint64_t full_tiles = L.generic ? 0 : a.n_main / RE_TILE;
  const uint64_t gw = (uint64_t)blockIdx.x * nwarps + warp;
  const uint64_t nw = (uint64_t)gridDim.x * nwarps;
  constexpr uint32_t in_bytes = 128u * B;
  const uint32_t xmode = L.x_mode;
  const uint32_t dshift = L.dir_shift, dmask = (1u << L.dir_shift) - 1u;
  const uint64_t stream_policy = policy_evict_first();   // the packed streams pass through once

  // the byte table is read only where its builder wrote it: the same density
  // rule over the finished X_M decides on both sides
  const bool x8_on = RE_X8_B(B) && xmode == 2 && a.x8 != nullptr && xdir_x8_pays<false>(a.xm, a.m, L.x_entries);
  if (xmode == 1 || xmode == 2) {
    const uint32_t* src = xmode == 1 ? a.xm : a.xdir;
    for (uint32_t i = threadIdx.x; i < L.x_entries; i += blockDim.x) s_x[i] = __ldg(src + i);
    __syncthreads();
  }
  if (lane == 0) {
    for (uint32_t s = 0; s < stages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncwarp();
  if constexpr (B > 0) {
    if (lane == 0) {
      for (uint32_t s = 0; s < stages; ++s) {
        uint64_t t = gw + (uint64_t)s * nw;
        if (t < full_tiles) {
          mbar_arrive_expect_tx(&bars[s], in_bytes);
          bulk_g2s_hint(wbase + s * round4(L.in_words), a.main_words + t * 32 * B, in_bytes, &bars[s], stream_policy);
        }
      }
    }
  }

  bool timed_out = false;
  uint32_t it = 0, st = 0, ph = 0;   // iteration, its input stage, that stage's phase
  for (uint64_t t = gw; t < n_tiles; t += nw, ++it) {
    uint32_t x[32];
    if (t < full_tiles) {
      uint32_t c[32];
      if constexpr (B > 0) {
        uint32_t* stage = wbase + st * round4(L.in_words);
        const bool ok = mbar_wait(&bars[st], ph, a.status);
        if (!__all_sync(0xFFFFFFFFu, ok)) {
          timed_out = true;
          break;
        }
        uint32_t w[B];
        load_row<B>(stage + lane * B, w);
        // unpacking consumes every word read from the stage, so after it (and
        // the warp barrier) no lane has a read of the stage outstanding; the
        // proxy fence then orders those reads before the bulk copy that
        // refills the stage (generic-proxy reads, async-proxy write)
        unpack32<B>(w, c);
        __syncwarp();
        if (lane == 0) {
          fence_proxy_async_smem();
          uint64_t tn = t + (uint64_t)stages * nw;
          if (tn < full_tiles) {
            mbar_arrive_expect_tx(&bars[st], in_bytes);
            bulk_g2s_hint(stage, a.main_words + tn * 32 * B, in_bytes, &bars[st], stream_policy);
          }
        }
        if (++st == stages) {
          st = 0;
          ph ^= 1u;
        }
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
      if (RE_DIR_B(B) && xmode == 2) {
        uint32_t many = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const uint32_t e = s_x[c[j] >> dshift];
          const uint32_t y = (c[j] & dmask) * (1u << 20) + e;   // multiply-add: FMA pipe
          x[j] = c[j] + (y & 0xFFFFFu) + __umulhi(y, 2u);        // y >> 31 on the FMA pipe
          many |= (e < DIR_SLOW_BELOW ? 1u : 0u) << j;
        }
        // codes in buckets with several steps read X_M, or the byte table
        // where there is one (an X_M too large to stay in L2)
        if (__any_sync(0xFFFFFFFFu, many != 0)) {
          if (!x8_on) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if ((many >> j) & 1u) x[j] = __ldg(a.xm + c[j]);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if ((many >> j) & 1u) {
                const uint32_t e = s_x[c[j] >> dshift];
                x[j] = (e >> 20) == DIR_MANY8_TOP ? c[j] + (e & 0xFFFFFu) + __ldg(a.x8 + c[j]) : __ldg(a.xm + c[j]);
              }
          }
        }
      } else if (RE_GDIR_B(B) && xmode == 3) {
        // the global directory (L2-resident): X_M[c] = c + base + (steps at
        // or below c's offset); buckets with more than four read X_M
        // steps at or below the code's offset lo: a byte k of the offsets
        // word counts when (lo + 128) - offset_k keeps its top bit, byte by
        // byte without borrows (offsets and lo below 128)
        uint32_t many = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const uint2 e = __ldg(a.gdir + (c[j] >> dshift));
          const uint32_t lo4 = ((c[j] & dmask) * 0x01010101u) | 0x80808080u;
          x[j] = c[j] + e.y + __popc((lo4 - e.x) & 0x80808080u);
          many |= (e.x == GDIR_MANY ? 1u : 0u) << j;
        }
        if (__any_sync(0xFFFFFFFFu, many != 0)) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if ((many >> j) & 1u) x[j] = __ldg(a.xm + c[j]);
        }
      } else if (xmode == 1) {
#pragma unroll
        for (int j = 0; j < 32; ++j) x[j] = s_x[c[j]];
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) x[j] = __ldg(a.xm + c[j]);
      }
    } else if (t * RE_TILE >= a.n_main && (t + 1) * RE_TILE <= n_out) {
      // a tile of delta rows only: 32 consecutive delta codes per lane
      // (16-byte loads when aligned), range-checked, mapped through X_D
      const uint32_t* src = a.dcodes + (t * RE_TILE - a.n_main) + lane * 32;
      uint32_t c[32];
      if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const uint4 v = __ldg(reinterpret_cast<const uint4*>(src) + q);
          c[4 * q] = v.x;
          c[4 * q + 1] = v.y;
          c[4 * q + 2] = v.z;
          c[4 * q + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) c[j] = __ldg(src + j);
      }
      uint32_t mx = 0;
#pragma unroll
      for (int j = 0; j < 32; ++j) mx = max(mx, c[j]);
      if (__any_sync(0xFFFFFFFFu, mx >= a.d)) {
        if (mx >= a.d) flag_status(a.status, ST_CODE);
#pragma unroll
        for (int j = 0; j < 32; ++j) c[j] = min(c[j], a.d - 1);
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) x[j] = __ldg(a.xd + c[j]);
    } else {
      // the main/delta boundary tile and a ragged last tile, per code: a
      // lane's codes are all main rows, all delta rows (or past the end),
      // or (one lane at most) mixed; the first two classes load without
      // per-code branches, so their loads are in flight together
      const uint64_t i0 = t * RE_TILE + lane * 32;
      if (i0 + 32 <= a.n_main) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          uint32_t cc = code_at(a.main_words, a.main_words_n, i0 + j, B);
          if (cc >= a.m) {
            flag_status(a.status, ST_CODE);
            cc = a.m - 1;
          }
          x[j] = __ldg(a.xm + cc);
        }
      } else if (i0 >= a.n_main) {
        const uint64_t nd = a.n_delta;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const uint64_t r = i0 + j - a.n_main;
          uint32_t cc = r < nd ? __ldg(a.dcodes + r) : 0u;
          if (r < nd && cc >= a.d) {
            flag_status(a.status, ST_CODE);
            cc = a.d - 1;
          }
          x[j] = r < nd ? __ldg(a.xd + cc) : 0u;
        }
      } else {
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
    }

    const uint32_t obi = L.obufs == 1 ? 0u : (it & 1u);
    uint32_t* ob = wbase + stages * round4(L.in_words) + obi * round4(L.out_words);
    // the bulk store that last read this buffer must have finished reading
    if (lane == 0) {
      if (L.obufs == 1) bulk_wait_read<0>();
      else bulk_wait_read<1>();
    }
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
        bulk_s2g_hint(a.out_words + w0, ob, tile_words * 4, stream_policy);
        bulk_commit();
      }
    } else {
      for (uint64_t q = lane; w0 + q < out_total; q += 32) a.out_words[w0 + q] = q < tile_words ? ob[q] : 0u;
    }
  }

  if constexpr (B > 0) {
    if (timed_out && lane == 0) {
      // let the copies already in flight land before the block exits
      for (uint32_t k = 0; k < stages; ++k) {
        const uint64_t t2 = gw + (uint64_t)(it + k) * nw;
        const uint32_t s2 = (st + k) % stages;
        const uint32_t p2 = ph ^ ((st + k) >= stages ? 1u : 0u);
        if (t2 < full_tiles) mbar_wait(&bars[s2], p2, a.status);
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

// The raised shared-memory limit of a kernel holds for the device that was
// current when it was set, so it is kept per device.
constexpr int kRegDevices = 64;
struct Registry {
  KernelFn fn[33];
  uint32_t smem_set[kRegDevices][33];  // dynamic smem size already allowed per device and kernel
  std::mutex mu;
  Registry() {
    KernelTable<32>::fill(fn);
    for (auto& d : smem_set)
      for (auto& s : d) s = 0;
  }
};

Registry& registry() {
  static Registry r;
  return r;
}

}  // namespace

uint32_t reencode_dir_words(uint64_t m) { return m > RE_DIR_FINE_MIN_CODES ? RE_DIR_FINE_MAX : RE_DIR_MAX; }
uint64_t reencode_dir_max_codes() { return (uint64_t)RE_DIR_MAX << RE_DIR_SHIFT_MAX; }
bool reencode_wants_x8(uint64_t m) { return m > RE_X8_MIN_CODES && m <= reencode_dir_max_codes(); }

// Bucket shift of the global directory for m main codes and d delta values
// (0: no global directory).
static uint32_t gdir_shift(uint64_t m, uint64_t d) {
  if (m <= reencode_dir_max_codes()) return 0;
  uint32_t s = GDIR_SHIFT_MAX;
  while (s > GDIR_SHIFT_MIN && 2 * (d << s) > 3 * m) --s;
  while (((m + (1ull << s) - 1) >> s) > GDIR_MAX_ENTRIES) ++s;
  return s <= GDIR_SHIFT_MAX ? s : 0;
}
uint64_t reencode_gdir_entries(uint64_t m, uint64_t d) {
  const uint32_t s = gdir_shift(m, d);
  return s ? (m + (1ull << s) - 1) >> s : 0;
}

// Host-side launch plan of Step 2(b): lookup mode, block size, shared memory.
struct ReencodePlanImpl {
  Layout L;
  uint32_t warps, bytes, grid;
  KernelFn fn;
};
static_assert(sizeof(ReencodePlanImpl) <= sizeof(ReencodePlan), "plan storage");

// Default warps a block of a column whose directory is refined.
constexpr uint32_t RE_WARPS_FINE = 12;
// Shared memory of a block with a refined directory at most: the 196 KB
// carve-out level, which leaves 60 KB of the SM's 256 KB to L1.
constexpr uint32_t RE_SMEM_KEEP_L1 = 196u << 10;

cudaError_t plan_reencode(uint32_t b, const ReencodeArgs& a, uint32_t sm_count, uint32_t flags, ReencodePlan* out) {
  if (b > 32 || a.max_bits > 32) return cudaErrorInvalidValue;
  ReencodePlanImpl P{};
  const uint64_t n_out = a.n_main + a.n_delta;
  Layout& L = P.L;
  L.in_words = 32 * b;
  L.out_words = 32 * (a.max_bits > b + 1 ? a.max_bits : b + 1);
  if (L.out_words > 32 * 32) L.out_words = 32 * 32;
  L.generic = (flags & DM_FLAG_GENERIC_REENCODE) ? 1u : 0u;
  L.stages = a.tune_stages >= 2 && a.tune_stages <= RE_STAGES_MAX ? a.tune_stages : 2;
  L.obufs = a.tune_obufs == 1 || a.tune_obufs == 2 ? a.tune_obufs : 1;
  // X_M lookup: a direct table in shared memory when it is small; else the
  // shared-memory directory of its steps; never smem when asked not to
  const bool allow_smem = !(flags & DM_FLAG_X_GLOBAL) && a.n_main > 0 && !L.generic;
  const bool want_smem = (flags & DM_FLAG_X_SMEM) != 0 || a.n_main >= (1u << 20);
  if (allow_smem && want_smem && a.m <= RE_XSMEM_MAX) {
    L.x_mode = 1;
    L.x_entries = a.m;
  } else if (allow_smem && want_smem && a.xdir && RE_DIR_B((int)b) &&
             (uint64_t)a.m <= ((uint64_t)RE_DIR_MAX << RE_DIR_SHIFT_MAX)) {
    L.x_mode = 2;
    xdir_shape(a.m, &L.dir_shift, &L.x_entries);
  } else if (allow_smem && want_smem && a.gdir && RE_GDIR_B((int)b) && reencode_gdir_entries(a.m, a.d)) {
    L.x_mode = 3;   // nothing in shared memory
    L.dir_shift = gdir_shift(a.m, a.d);
  }
  // warps per block: as many as the device's shared memory allows, up to 16
  // (one block per SM); a lookup table that leaves room for fewer than 4
  // warps is dropped for the global gather
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kRegDevices ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return cudaErrorInvalidValue;
  auto fit = [&](const Layout& l, uint32_t cap) {
    const uint64_t fixed = RE_BAR_BYTES + (uint64_t)round4(l.x_entries) * 4;
    const uint64_t per = (uint64_t)per_warp_words(l) * 4;
    uint64_t w = fixed < (uint64_t)optin ? ((uint64_t)optin - fixed) / per : 0;
    return (uint32_t)(w < cap ? w : cap);
  };
  // (12 by default for directory columns of 2^22 to 11 * 2^20 main codes,
  // whose freed staging refines the directory below: Step 2(b) of a 10M-value
  // column with 30k new values took 0.233 ms against 0.348 at 16 warps, and
  // 0.143 against 0.135 with 3k)
  const bool fine = L.x_mode == 2 && a.m > RE_DIR_FINE_MIN_CODES && a.m <= RE_X8_MIN_CODES;
  const uint32_t want_warps =
      a.tune_warps >= 1 && a.tune_warps <= RE_WARPS_MAX ? a.tune_warps : (fine ? RE_WARPS_FINE : 16u);
  P.warps = fit(L, want_warps);
  if ((L.x_mode == 1 || L.x_mode == 2) && P.warps < 4) {
    L.x_mode = 0;
    L.x_entries = 0;
    L.dir_shift = 0;
    P.warps = fit(L, want_warps);
  }
  if (P.warps < 1) return cudaErrorInvalidConfiguration;
  // Above 2^22 main codes X_M is far larger than L1, so a code in a bucket
  // with several steps costs an L2 gather.  Buckets are halved while the
  // finer directory fits the scratch, leaves the block as many warps and
  // keeps its shared memory within RE_SMEM_KEEP_L1 (the L1 left beside it
  // holds the gathers in flight; a block of 227 KB halves it and slowed a
  // step-dense column's Step 2(b) from 0.47 to 0.87 ms).  With 16 warps the
  // rule leaves the directory as it is; fewer warps trade their staging
  // for finer buckets.
  if (L.x_mode == 2 && a.m > RE_DIR_FINE_MIN_CODES) {
    const uint32_t words = a.xdir_words ? a.xdir_words : RE_DIR_MAX;
    while (L.dir_shift > 0) {
      Layout l2 = L;
      l2.dir_shift = L.dir_shift - 1;
      const uint64_t n = ((uint64_t)a.m + (1ull << l2.dir_shift) - 1) >> l2.dir_shift;
      if (n > words) break;
      l2.x_entries = (uint32_t)n;
      if (fit(l2, want_warps) < P.warps || smem_bytes(l2, P.warps) > RE_SMEM_KEEP_L1) break;
      L = l2;
    }
  }
  P.bytes = smem_bytes(L, P.warps);
  Registry& R = registry();
  P.fn = R.fn[b];
  {
    std::lock_guard<std::mutex> g(R.mu);
    if (R.smem_set[dev][b] < P.bytes) {
      cudaError_t e = cudaFuncSetAttribute(P.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.bytes);
      if (e != cudaSuccess) return e;
      R.smem_set[dev][b] = P.bytes;
    }
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, P.fn, P.warps * 32, P.bytes);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t n_tiles = (n_out + RE_TILE - 1) / RE_TILE;
  uint64_t grid = (n_tiles + P.warps - 1) / P.warps;
  const uint64_t cap = (uint64_t)sm_count * per_sm;
  if (grid > cap) grid = cap;
  P.grid = (uint32_t)(grid ? grid : 1);
  memcpy(out->storage, &P, sizeof(P));
  out->needs_directory = L.x_mode == 2;
  out->dir_shift = L.dir_shift;
  out->dir_entries = L.x_mode == 2 ? L.x_entries : 0;
  out->gdir_entries = L.x_mode == 3 ? reencode_gdir_entries(a.m, a.d) : 0;
  return cudaSuccess;
}

cudaError_t launch_xdir(const ReencodePlan& plan, const ReencodeArgs& a, cudaStream_t s, uint64_t* launches) {
  ReencodePlanImpl P;
  memcpy(&P, plan.storage, sizeof(P));
  if (P.L.x_mode != 2) return cudaSuccess;
  const uint32_t work = std::max<uint32_t>(P.L.x_entries, a.x8 ? (uint32_t)((a.m + 3) / 4) : 0u);
  uint32_t blocks = (work + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  xdir_build_kernel<<<blocks, 256, 0, s>>>(a.xm, a.m, P.L.dir_shift, P.L.x_entries, a.xdir, a.x8);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_gdir(const ReencodePlan& plan, const ReencodeArgs& a, cudaStream_t s, uint64_t* launches) {
  ReencodePlanImpl P;
  memcpy(&P, plan.storage, sizeof(P));
  if (P.L.x_mode != 3 || plan.gdir_entries == 0) return cudaSuccess;
  const uint64_t blocks = std::min<uint64_t>(4096, (plan.gdir_entries + 255) / 256);
  gdir_build_kernel<<<(uint32_t)blocks, 256, 0, s>>>(a.xm, a.m, P.L.dir_shift, plan.gdir_entries, a.gdir);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_reencode_planned(const ReencodePlan& plan, const ReencodeArgs& a, cudaStream_t s,
                                    uint64_t* launches) {
  ReencodePlanImpl P;
  memcpy(&P, plan.storage, sizeof(P));
  if (a.n_main + a.n_delta == 0) return cudaSuccess;
  P.fn<<<P.grid, P.warps * 32, P.bytes, s>>>(a, P.L);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_reencode(uint32_t b, const ReencodeArgs& a, cudaStream_t s, uint32_t sm_count, uint32_t flags,
                            uint64_t* launches) {
  if (a.n_main + a.n_delta == 0) return cudaSuccess;
  ReencodePlan plan;
  cudaError_t e = plan_reencode(b, a, sm_count, flags, &plan);
  if (e == cudaSuccess) e = launch_xdir(plan, a, s, launches);
  if (e == cudaSuccess) e = launch_gdir(plan, a, s, launches);
  if (e == cudaSuccess) e = launch_reencode_planned(plan, a, s, launches);
  return e;
}

}  // namespace dm
