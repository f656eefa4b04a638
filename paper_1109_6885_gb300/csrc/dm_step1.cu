// Step 1 of the column merge in one persistent kernel: sort the delta
// dictionary (Step 1(a)), merge it with the main dictionary (Step 1(b)),
// publish the new width (Step 2(a)) and build the X_M directory used by
// Step 2(b).
//
// Step 1(a).  The paper walks the leaves of a CSB+ tree kept during inserts
// (Section 5.1); with the delta dictionary stored as an insertion-order
// array, Step 1(a) is a stable LSD radix sort of (key, insertion code)
// pairs, 8-bit digits, perm[j] = insertion code of U_D[j] being the tuple-id
// map of Section 5.3.  One sweep counts the digits of every pass; each block
// then derives the plan (first slot of every digit, passes whose digit is
// not constant).  Each pass ranks 2048-key tiles in shared memory with a
// stable warp multisplit (ballots over the digit bits), finds the tile's
// offset per digit by decoupled look-back over earlier tiles, stages the
// tile in digit order and writes it out coalesced.
//
// Step 1(b).  The paper cuts both dictionaries at N_T-quantiles and fixes
// the output offsets with a counter array and a prefix sum (Section 6.2.1).
// Here tile t owns merged positions [2048t, 2048t + 2048): a merge-path
// (co-rank) search cuts U_M and U_D, each thread merges 8 positions out of
// shared memory (ties: the main value first), a position is a duplicate
// when its key equals the previous one in merged order (values in both
// dictionaries and repeats inside D_dict alike), and its new code is the
// number of non-duplicates at or before it minus one, from a block scan
// plus a decoupled look-back.  U'[code] receives each non-duplicate, X_M /
// X_D every position; the last tile publishes |U'| and E'_C = ceil(log2|U'|).
//
// The phases are separated by grid-wide barriers (bounded spins); the
// kernel is launched cooperatively, so all its blocks are resident and
// tiles are assigned by block index.  Data written earlier in the kernel is
// read with ld.global.cg (L1 is not coherent across SMs).
#include <string.h>

#include <algorithm>
#include <mutex>

#include "dm_common.cuh"
#include "dm_internal.h"
#include "dm_xdir.cuh"

namespace dm {

namespace {

constexpr uint32_t S1_THREADS = 256;
constexpr uint32_t S1_WARPS = S1_THREADS / 32;
constexpr uint32_t S1_ITEMS = 8;                      // merge positions per thread
constexpr uint32_t S1_TILE = S1_THREADS * S1_ITEMS;   // 2048 merged positions per merge tile
constexpr uint32_t SR_ITEMS = RS_ITEMS;               // sort keys per thread
constexpr uint32_t SR_TILE = S1_THREADS * SR_ITEMS;   // sort keys per sort tile
static_assert(S1_TILE == MG_TILE && SR_TILE == RS_TILE, "tile sizes");

// ---------------------------------------------------------------- loads
template <class K>
__device__ __forceinline__ K ldcg_key(const K* p) {
  return __ldcg(p);
}
template <>
__device__ __forceinline__ u128 ldcg_key<u128>(const u128* p) {
  ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(p));
  return u128{v.x, v.y};
}
template <class K>
__device__ __forceinline__ K ld_key(const K* p, bool coherent) {
  return coherent ? ldcg_key(p) : load_key(p);
}

// ---------------------------------------------------------------- grid barrier
// Barrier `idx` of this launch: every block adds one to its own zeroed
// counter and waits (bounded) until all blocks have.  Writes before the
// barrier are fenced; reads after it see them.
__device__ void grid_barrier(uint32_t* bars, uint32_t idx, uint32_t* status) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&bars[idx], 1u);
    uint32_t spins = 0;
    while (ld_volatile(&bars[idx]) < gridDim.x) {
      if (++spins > kSpinLimit) {
        flag_status(status, ST_TIMEOUT);
        break;
      }
      if (spins > 16) __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
}

// ---------------------------------------------------------------- shared memory
template <int W>
struct SortSmem {
  using K = typename KeyOf<W>::T;
  uint32_t whist[S1_WARPS][256];   // per-warp digit counts, then warp offsets
  uint32_t tstart[256];            // tile-local first position of each digit
  uint32_t gbase[256];             // global position of the tile's first key of each digit
  uint32_t wsum[S1_WARPS];
  K keys[SR_TILE];                 // the tile in digit order
  uint32_t vals[SR_TILE];
};

template <int W>
struct MergeSmem {
  using K = typename KeyOf<W>::T;
  K keys[S1_TILE];                 // U_M segment then U_D segment
  K last[S1_THREADS];
  uint32_t perm[S1_TILE];
  uint32_t wsum[S1_WARPS];
  uint64_t cut[2];
  uint64_t excl, lb_sum;
  uint32_t nearest;
  K pred, prevA, prevB;
};

constexpr uint32_t BK_CAP = 2048;   // keys a block sorts in shared memory at once
constexpr uint32_t BK_SINGLE = 512; // at most this many keys: one block sorts them all

template <int W>
struct BucketSmem {
  using K = typename KeyOf<W>::T;
  K keys[BK_CAP];
  uint32_t vals[BK_CAP];
};

template <int W>
union Step1Smem {
  SortSmem<W> s;
  MergeSmem<W> m;
  BucketSmem<W> b;
  uint32_t hist[W * 256];
};

template <int W>
constexpr size_t step1_smem_bytes() {
  return (sizeof(Step1Smem<W>) + 15) / 16 * 16 + (size_t)W * 256 * 4 + 64;
}

// ---------------------------------------------------------------- Step 1(a)
// Digit counts of every pass (blocks below hist_blocks take part).
template <int W>
__device__ void hist_phase(const Step1Args& a, uint32_t* sh) {
  using K = typename KeyOf<W>::T;
  if (blockIdx.x >= a.hist_blocks) return;
  for (uint32_t i = threadIdx.x; i < W * 256; i += S1_THREADS) sh[i] = 0;
  __syncthreads();
  const K* keys = static_cast<const K*>(a.in_keys);
  for (uint64_t idx = (uint64_t)blockIdx.x * S1_THREADS + threadIdx.x; idx < a.d;
       idx += (uint64_t)a.hist_blocks * S1_THREADS) {
    const K k = load_key(keys + idx);
#pragma unroll
    for (int p = 0; p < W; ++p) atomicAdd(&sh[p * 256 + key_digit(k, p)], 1u);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < W * 256; i += S1_THREADS)
    if (sh[i]) atomicAdd(&a.hist[i], sh[i]);
}

// Block exclusive scan of one value per thread (256 threads).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* wsum, uint32_t* total) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t n = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= (uint32_t)o) inc += n;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t excl = inc - v, tot = 0;
#pragma unroll
  for (uint32_t w = 0; w < S1_WARPS; ++w) {
    const uint32_t sw = wsum[w];
    if (w < warp) excl += sw;
    tot += sw;
  }
  __syncthreads();
  if (total) *total = tot;
  return excl;
}

// The sort plan from the global histogram: first slot of every digit of
// every pass, and the mask of passes that run (a pass whose digit is the
// same for every key is skipped; if none remains, the last pass runs so the
// result always lands in a ping-pong buffer).  Every block computes it.
//
// It also decides between the two ways to finish the sort: when every bucket
// of the most significant digit that varies holds at most BK_CAP keys, one
// stable pass on that digit plus one sort of each bucket in shared memory
// (*msd = true); otherwise all running passes, least significant first.
template <int W>
__device__ uint32_t plan_phase(const Step1Args& a, uint32_t* s_plan, uint32_t* wsum, bool* msd) {
  const uint32_t t = threadIdx.x;
  uint32_t v[W];
#pragma unroll
  for (int p = 0; p < W; ++p) v[p] = ld_volatile(&a.hist[p * 256 + t]);
  uint32_t run = 0;
#pragma unroll
  for (int p = 0; p < W; ++p) {
    if (!__syncthreads_or((uint64_t)v[p] == a.d)) run |= 1u << p;
    s_plan[p * 256 + t] = block_excl_scan(v[p], wsum, nullptr);
  }
  run = run ? run : (1u << (W - 1));
  const int top = 31 - __clz(run);
  uint32_t vtop = 0;
#pragma unroll
  for (int p = 0; p < W; ++p)
    if (p == top) vtop = v[p];
  *msd = !__syncthreads_or(vtop > BK_CAP);
  return run;
}

// One tile of one LSD pass.
template <int W>
__device__ void pass_tile(const Step1Args& a, int pass, uint32_t tile, int e, const uint32_t* s_plan,
                          SortSmem<W>& S) {
  using K = typename KeyOf<W>::T;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t d = a.d;
  // e: passes that ran before this one (0: read the input dictionary)
  const bool odd = e & 1;
  const K* src_k = e == 0 ? static_cast<const K*>(a.in_keys) : static_cast<const K*>(odd ? a.keys[0] : a.keys[1]);
  const uint32_t* src_v = e == 0 ? nullptr : (odd ? a.vals[0] : a.vals[1]);
  K* dst_k = static_cast<K*>(odd ? a.keys[1] : a.keys[0]);
  uint32_t* dst_v = odd ? a.vals[1] : a.vals[0];

  for (uint32_t i = tid; i < S1_WARPS * 256; i += S1_THREADS) (&S.whist[0][0])[i] = 0;

  // warp w owns tile items [256w, 256w + 256), round r covers 32 of them
  K key[SR_ITEMS];
  uint32_t val[SR_ITEMS], dig[SR_ITEMS], rank[SR_ITEMS];
  const uint64_t tbase = (uint64_t)tile * SR_TILE;
  const uint64_t base = tbase + warp * (SR_ITEMS * 32) + lane;
#pragma unroll
  for (int r = 0; r < (int)SR_ITEMS; ++r) {
    const uint64_t idx = base + r * 32;
    if (idx < d) {
      key[r] = e == 0 ? load_key(src_k + idx) : ldcg_key(src_k + idx);
      val[r] = e == 0 ? (uint32_t)idx : __ldcg(src_v + idx);
      dig[r] = key_digit(key[r], pass);
    } else {
      key[r] = K{};
      val[r] = 0;
      dig[r] = 256;
    }
  }
  __syncthreads();

  // stable warp multisplit: lanes with equal digits found by ballots over
  // the digit's bits; rounds in item order, so ranks follow input order
#pragma unroll
  for (int r = 0; r < (int)SR_ITEMS; ++r) {
    const uint32_t dg = dig[r];
    uint32_t peers = __ballot_sync(0xFFFFFFFFu, dg < 256);
#pragma unroll
    for (int bit = 0; bit < 8; ++bit) {
      const uint32_t bb = __ballot_sync(0xFFFFFFFFu, (dg >> bit) & 1u);
      peers &= ((dg >> bit) & 1u) ? bb : ~bb;
    }
    const bool ok = dg < 256;
    const uint32_t leader = ok ? __ffs(peers) - 1 : lane;
    uint32_t cnt = 0;
    if (ok && lane == leader) {
      cnt = S.whist[warp][dg];
      S.whist[warp][dg] = cnt + __popc(peers);
    }
    cnt = __shfl_sync(0xFFFFFFFFu, cnt, leader);
    rank[r] = cnt + __popc(peers & lanemask_lt());
    __syncwarp();
  }
  __syncthreads();

  // per digit (thread = digit): warp offsets inside the tile, tile count,
  // tile-local start of the digit
  uint32_t tcount = 0;
#pragma unroll
  for (uint32_t w = 0; w < S1_WARPS; ++w) {
    const uint32_t c = S.whist[w][tid];
    S.whist[w][tid] = tcount;
    tcount += c;
  }
  S.tstart[tid] = block_excl_scan(tcount, S.wsum, nullptr);

  // decoupled look-back over earlier tiles for digit `tid`
  uint32_t* lb = a.sort_lb + (uint64_t)pass * a.sort_tiles * 256;
  uint32_t excl = 0;
  if (tile == 0) {
    st_volatile(&lb[tid], LB_INC32 | tcount);
  } else {
    st_volatile(&lb[(uint64_t)tile * 256 + tid], LB_AGG32 | tcount);
    int64_t p = (int64_t)tile - 1;
    uint32_t spins = 0;
    bool done = false;
    while (!done && p >= 0) {
      uint32_t v[32];   // 32 predecessors per round trip
#pragma unroll
      for (int q = 0; q < 32; ++q) v[q] = (p - q >= 0) ? ld_volatile(&lb[(uint64_t)(p - q) * 256 + tid]) : LB_INC32;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        if (!done) {
          while ((v[q] >> 30) == 0) {   // not published yet
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
      p -= 32;
    }
    st_volatile(&lb[(uint64_t)tile * 256 + tid], LB_INC32 | (excl + tcount));
  }
  S.gbase[tid] = s_plan[pass * 256 + tid] + excl;
  __syncthreads();

  // stage the tile in digit order, then write it out with consecutive
  // threads on consecutive positions of each digit's run
#pragma unroll
  for (int r = 0; r < (int)SR_ITEMS; ++r) {
    if (dig[r] < 256) {
      const uint32_t lp = S.tstart[dig[r]] + S.whist[warp][dig[r]] + rank[r];
      if (lp < SR_TILE) {
        S.keys[lp] = key[r];
        S.vals[lp] = val[r];
      }
    }
  }
  __syncthreads();
  const uint32_t nt = (uint32_t)(d - tbase < SR_TILE ? d - tbase : SR_TILE);
  for (uint32_t i = tid; i < nt; i += S1_THREADS) {
    const K k = S.keys[i];
    const uint32_t dg = key_digit(k, pass);
    const uint64_t pos = (uint64_t)S.gbase[dg] + (i - S.tstart[dg]);
    if (pos < d) {
      dst_k[pos] = k;
      dst_v[pos] = S.vals[i];
    } else {
      flag_status(a.status, ST_TIMEOUT);
    }
  }
  __syncthreads();
}

// Sort n <= BK_CAP (key, insertion code) pairs of one bucket in shared
// memory (bitonic network over pairs ordered by key, then code; codes are
// distinct, so the order is the stable one) and write them to dst at the
// same offsets.  src_v == nullptr: the codes are the positions (input
// dictionary); coherent: src was written earlier in this kernel.
template <int W>
__device__ void bucket_sort(const typename KeyOf<W>::T* src_k, const uint32_t* src_v, uint64_t off, uint32_t n,
                            bool coherent, typename KeyOf<W>::T* dst_k, uint32_t* dst_v, BucketSmem<W>& S) {
  using K = typename KeyOf<W>::T;
  const uint32_t tid = threadIdx.x;
  uint32_t N = 2;
  while (N < n) N <<= 1;
  for (uint32_t i = tid; i < N; i += S1_THREADS) {
    if (i < n) {
      S.keys[i] = coherent ? ldcg_key(src_k + off + i) : load_key(src_k + off + i);
      S.vals[i] = src_v ? (coherent ? __ldcg(src_v + off + i) : __ldg(src_v + off + i)) : (uint32_t)(off + i);
    } else {
      S.keys[i] = key_max_value<K>();
      S.vals[i] = 0xFFFFFFFFu;
    }
  }
  __syncthreads();
  for (uint32_t k = 2; k <= N; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = tid; i < (N >> 1); i += S1_THREADS) {
        const uint32_t lo = 2 * i - (i & (j - 1)), hi = lo + j;
        const bool up = (lo & k) == 0;
        const K ka = S.keys[lo], kb = S.keys[hi];
        const uint32_t va = S.vals[lo], vb = S.vals[hi];
        const bool gt = key_lt(kb, ka) || (key_eq(ka, kb) && va > vb);
        if (gt == up) {
          S.keys[lo] = kb;
          S.keys[hi] = ka;
          S.vals[lo] = vb;
          S.vals[hi] = va;
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = tid; i < n; i += S1_THREADS) {
    dst_k[off + i] = S.keys[i];
    dst_v[off + i] = S.vals[i];
  }
  __syncthreads();
}

// ---------------------------------------------------------------- Step 1(b)
// Number of U_M entries among the first k merged positions (ties: U_M
// first).  Whole warp; 32 probes per round narrow the range 33-fold.
template <class K>
__device__ uint64_t corank_warp(const K* A, uint64_t m, const K* B, uint64_t d, uint64_t k, bool bcoh) {
  const uint32_t lane = lane_id();
  uint64_t lo = k > d ? k - d : 0, hi = k < m ? k : m;
  while (hi - lo > 32) {
    const uint64_t span = hi - lo;
    const uint64_t c = lo + (span * (lane + 1)) / 33;
    const bool p = key_le(load_key(A + c), ld_key(B + (k - 1 - c), bcoh));
    const uint32_t t = __popc(__ballot_sync(0xFFFFFFFFu, p));
    const uint64_t c_below = __shfl_sync(0xFFFFFFFFu, c, t > 0 ? t - 1 : 0);
    const uint64_t c_at = __shfl_sync(0xFFFFFFFFu, c, t < 32 ? t : 31);
    const uint64_t nlo = t > 0 ? c_below + 1 : lo;
    const uint64_t nhi = t < 32 ? c_at : hi;
    lo = nlo;
    hi = nhi < nlo ? nlo : nhi;
  }
  const uint64_t c = lo + lane;
  const bool p = c < hi && key_le(load_key(A + c), ld_key(B + (k - 1 - c), bcoh));
  return lo + __popc(__ballot_sync(0xFFFFFFFFu, p));
}

template <int W>
__device__ void merge_tile(const Step1Args& a, uint32_t tile, const typename KeyOf<W>::T* B, const uint32_t* perm,
                           bool bcoh, MergeSmem<W>& S) {
  using K = typename KeyOf<W>::T;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const K* A = static_cast<const K*>(a.a);
  const uint64_t m = a.m, d = a.d, n = m + d;

  const uint64_t k0 = (uint64_t)tile * S1_TILE;
  const uint64_t k1 = k0 + S1_TILE < n ? k0 + S1_TILE : n;
  if (warp < 2) {
    const uint64_t c = corank_warp(A, m, B, d, warp == 0 ? k0 : k1, bcoh);
    if (lane == 0) S.cut[warp] = c;
  }
  __syncthreads();
  const uint64_t i0 = S.cut[0], i1 = S.cut[1];
  const uint64_t j0 = k0 - i0, j1 = k1 - i1;
  const uint32_t na = (uint32_t)(i1 - i0), nb = (uint32_t)(j1 - j0), nt = na + nb;
  // one batch of loads: both segments, their perm entries, and the keys just
  // before the tile (merge predecessor and sortedness check)
  for (uint32_t x = tid; x < na; x += S1_THREADS) S.keys[x] = load_key(A + i0 + x);
  for (uint32_t x = tid; x < nb; x += S1_THREADS) {
    S.keys[na + x] = ld_key(B + j0 + x, bcoh);
    S.perm[x] = bcoh ? __ldcg(perm + j0 + x) : __ldg(perm + j0 + x);
  }
  if (tid == 0 && i0 > 0) S.prevA = load_key(A + i0 - 1);
  if (tid == 32 && j0 > 0) S.prevB = ld_key(B + j0 - 1, bcoh);
  __syncthreads();
  const K* sA = S.keys;
  const K* sB = S.keys + na;

  // U_M must be strictly increasing
  for (uint32_t x = tid; x < na; x += S1_THREADS) {
    if (i0 + x == 0) continue;
    const K prev = x > 0 ? sA[x - 1] : S.prevA;
    if (!key_lt(prev, sA[x])) flag_status(a.status, ST_UNSORTED);
  }

  // this thread's 8 merged positions: cut inside the tile, then merge
  const uint32_t kk = tid * S1_ITEMS < nt ? tid * S1_ITEMS : nt;
  const uint32_t cnt = kk + S1_ITEMS < nt ? S1_ITEMS : nt - kk;
  uint32_t lo = kk > nb ? kk - nb : 0, hi = kk < na ? kk : na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (key_le(sA[mid], sB[kk - 1 - mid])) lo = mid + 1;
    else hi = mid;
  }
  uint32_t ia = lo, ib = kk - lo;
  K key[S1_ITEMS];
  K last{};
  uint32_t src[S1_ITEMS];   // bit 31: from U_D; low bits: index inside the tile's segment
#pragma unroll
  for (int it = 0; it < (int)S1_ITEMS; ++it) {
    if ((uint32_t)it < cnt) {
      const bool takeA = ib >= nb || (ia < na && key_le(sA[ia], sB[ib]));
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
  if (cnt > 0) S.last[tid] = last;
  __syncthreads();

  // duplicates: equal to the previous key in merged order
  uint32_t dupmask = 0, nondup = 0;
  {
    bool has_prev = tid > 0 ? true : k0 > 0;
    K prev;
    if (tid > 0) {
      prev = S.last[tid - 1];
    } else if (i0 > 0 && j0 > 0) {
      prev = key_max(S.prevA, S.prevB);   // the key at merged position k0 - 1
    } else {
      prev = i0 > 0 ? S.prevA : S.prevB;
    }
#pragma unroll
    for (int it = 0; it < (int)S1_ITEMS; ++it) {
      if ((uint32_t)it < cnt) {
        const bool dup = has_prev && key_eq(key[it], prev);
        dupmask |= (uint32_t)dup << it;
        nondup += !dup;
        prev = key[it];
        has_prev = true;
      }
    }
  }
  uint32_t ttotal = 0;
  const uint32_t texcl = block_excl_scan(nondup, S.wsum, &ttotal);

  // decoupled look-back: the whole block reads 256 predecessors per round
  // trip and sums them down to the nearest inclusive prefix
  if (tile == 0) {
    if (tid == 0) {
      st_volatile(&a.merge_lb[0], LB_INC64 | ttotal);
      S.excl = 0;
    }
  } else {
    if (tid == 0) {
      st_volatile(&a.merge_lb[tile], LB_AGG64 | ttotal);
      S.lb_sum = 0;
    }
    int64_t top = (int64_t)tile - 1;
    uint32_t spins = 0;
    for (;;) {
      const int64_t p = top - (int64_t)tid;
      const uint64_t v = p >= 0 ? ld_volatile(&a.merge_lb[p]) : LB_INC64;
      if (tid == 0) S.nearest = S1_THREADS;
      __syncthreads();
      if ((v >> 62) == 2) atomicMin(&S.nearest, tid);
      __syncthreads();
      const uint32_t nearest = S.nearest;
      const bool all_ready = __syncthreads_and(tid > nearest || (v >> 62) != 0);
      if (!all_ready) {
        if (++spins > kSpinLimit) {
          if (tid == 0) flag_status(a.status, ST_TIMEOUT);
          break;
        }
        if (spins > 32) __nanosleep(64);
        continue;
      }
      uint64_t part = tid <= nearest ? (v & LB_MASK64) : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
      if (lane == 0 && part) atomicAdd(reinterpret_cast<unsigned long long*>(&S.lb_sum), (unsigned long long)part);
      __syncthreads();
      if (nearest < S1_THREADS) break;
      top -= S1_THREADS;
    }
    __syncthreads();
    if (tid == 0) {
      S.excl = S.lb_sum;
      st_volatile(&a.merge_lb[tile], LB_INC64 | (S.lb_sum + ttotal));
    }
  }
  __syncthreads();

  // codes and writes
  uint64_t c = S.excl + texcl;
  K* unew = static_cast<K*>(a.unew);
#pragma unroll
  for (int it = 0; it < (int)S1_ITEMS; ++it) {
    if ((uint32_t)it < cnt) {
      const bool dup = (dupmask >> it) & 1u;
      c += !dup;
      const uint64_t code = c - 1;
      if (code >= n) {
        flag_status(a.status, ST_TIMEOUT);
        continue;
      }
      if (!dup) unew[code] = key[it];
      const uint32_t s = src[it];
      if (s & 0x80000000u) {
        const uint32_t pj = S.perm[s & 0x7FFFFFFFu];
        if (pj < d) a.xd[pj] = (uint32_t)code;
        else flag_status(a.status, ST_CODE);
      } else {
        a.xm[i0 + s] = (uint32_t)code;
      }
    }
  }
  if (tile == a.merge_tiles - 1 && tid == 0) {
    const uint64_t u = S.excl + ttotal;
    *a.d_u = u;
    *a.d_bits = bits_for(u);
  }
  __syncthreads();
}

// ---------------------------------------------------------------- the kernel
template <int W>
__global__ void __launch_bounds__(S1_THREADS) step1_kernel(Step1Args a) {
  using K = typename KeyOf<W>::T;
  extern __shared__ __align__(16) unsigned char dsmem[];
  Step1Smem<W>& U = *reinterpret_cast<Step1Smem<W>*>(dsmem);
  uint32_t* s_plan = reinterpret_cast<uint32_t*>(dsmem + (sizeof(Step1Smem<W>) + 15) / 16 * 16);
  uint32_t* s_wsum = s_plan + W * 256;

  uint32_t nbar = 0;
  const K* ud = static_cast<const K*>(a.b);
  const uint32_t* up = a.perm;
  bool coherent = false;
  if ((a.phases & S1_SORT) && a.d > 0) {
    K* k0 = static_cast<K*>(a.keys[0]);
    uint32_t* v0 = a.vals[0];
    if (a.d <= BK_SINGLE) {
      // a delta dictionary this small is sorted by one block
      if (blockIdx.x == 0) bucket_sort<W>(static_cast<const K*>(a.in_keys), nullptr, 0, (uint32_t)a.d, false, k0, v0, U.b);
      ud = k0;
      up = v0;
    } else {
      hist_phase<W>(a, U.hist);
      grid_barrier(a.barriers, nbar++, a.status);
      bool msd = false;
      const uint32_t run = plan_phase<W>(a, s_plan, s_wsum, &msd);
      if (msd) {
        // one stable pass on the top varying digit, then each of its 256
        // buckets sorted in shared memory in place
        const int top = 31 - __clz(run);
        for (uint32_t t = blockIdx.x; t < a.sort_tiles; t += gridDim.x) pass_tile<W>(a, top, t, 0, s_plan, U.s);
        grid_barrier(a.barriers, nbar++, a.status);
        for (uint32_t b = blockIdx.x; b < 256; b += gridDim.x) {
          const uint32_t off = s_plan[top * 256 + b];
          const uint32_t n = (b < 255 ? s_plan[top * 256 + b + 1] : (uint32_t)a.d) - off;
          if (n > 1) bucket_sort<W>(k0, v0, off, n, true, k0, v0, U.b);
        }
        ud = k0;
        up = v0;
      } else {
        int e = 0;
        for (int p = 0; p < W; ++p) {
          if (!((run >> p) & 1u)) continue;
          for (uint32_t t = blockIdx.x; t < a.sort_tiles; t += gridDim.x) pass_tile<W>(a, p, t, e, s_plan, U.s);
          grid_barrier(a.barriers, nbar++, a.status);
          ++e;
        }
        const bool last_odd = (e - 1) & 1;
        ud = static_cast<const K*>(last_odd ? a.keys[1] : a.keys[0]);
        up = last_odd ? a.vals[1] : a.vals[0];
      }
    }
    coherent = true;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.final_slot) {
      a.final_slot[0] = const_cast<K*>(ud);
      a.final_slot[1] = const_cast<uint32_t*>(up);
    }
    // the merge reads what other blocks wrote
    if (a.phases & (S1_MERGE | S1_DIR)) grid_barrier(a.barriers, nbar++, a.status);
  }
  if ((a.phases & S1_MERGE) && a.m + a.d > 0) {
    for (uint32_t t = blockIdx.x; t < a.merge_tiles; t += gridDim.x) merge_tile<W>(a, t, ud, up, coherent, U.m);
  }
  if ((a.phases & S1_DIR) && a.dir_entries > 0) {
    grid_barrier(a.barriers, nbar++, a.status);
    for (uint32_t b = blockIdx.x * S1_THREADS + threadIdx.x; b < a.dir_entries; b += gridDim.x * S1_THREADS)
      a.xdir[b] = xdir_entry<true>(a.xm, (uint32_t)a.m, a.dir_shift, b);
  }
}

template <int W>
__global__ void sort_copy_kernel(void* const* slot, uint64_t d, typename KeyOf<W>::T* keys_out, uint32_t* perm_out) {
  using K = typename KeyOf<W>::T;
  const K* k = static_cast<const K*>(slot[0]);
  const uint32_t* v = static_cast<const uint32_t*>(slot[1]);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (uint64_t)gridDim.x * blockDim.x) {
    keys_out[i] = k[i];
    perm_out[i] = v[i];
  }
}

struct Launch {
  std::mutex mu;
  bool ready[3] = {false, false, false};
  int per_sm[3] = {0, 0, 0};
};
Launch& launch_state() {
  static Launch L;
  return L;
}

template <int W>
cudaError_t prepare_w() {
  const int wi = W == 4 ? 0 : (W == 8 ? 1 : 2);
  Launch& L = launch_state();
  std::lock_guard<std::mutex> g(L.mu);
  if (L.ready[wi]) return cudaSuccess;
  const size_t smem = step1_smem_bytes<W>();
  cudaError_t e = cudaFuncSetAttribute(step1_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L.per_sm[wi], step1_kernel<W>, S1_THREADS, smem);
  if (e != cudaSuccess) return e;
  L.ready[wi] = true;
  return cudaSuccess;
}


template <int W>
cudaError_t launch_step1_w(Step1Args a, cudaStream_t s, uint32_t sm_count, uint64_t* launches) {
  const int wi = W == 4 ? 0 : (W == 8 ? 1 : 2);
  const size_t smem = step1_smem_bytes<W>();
  cudaError_t pe = prepare_w<W>();
  if (pe != cudaSuccess) return pe;
  Launch& L = launch_state();
  int per_sm;
  {
    std::lock_guard<std::mutex> g(L.mu);
    per_sm = L.per_sm[wi];
  }
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // all blocks resident at once (cooperative launch); no more blocks than
  // the largest phase has tiles
  uint64_t want = 1;
  if ((a.phases & S1_SORT) && a.d > BK_SINGLE) want = std::max<uint64_t>(want, std::max<uint64_t>(a.sort_tiles, 256));
  if (a.phases & S1_MERGE) want = std::max<uint64_t>(want, a.merge_tiles);
  if (a.phases & S1_DIR) want = std::max<uint64_t>(want, (a.dir_entries + S1_THREADS - 1) / S1_THREADS);
  uint64_t cap = (uint64_t)per_sm * sm_count;
  if (a.grid_cap && a.grid_cap < cap) cap = a.grid_cap;
  const uint32_t grid = (uint32_t)std::min(want, cap);
  a.hist_blocks = (uint32_t)std::min<uint64_t>(grid, std::max<uint64_t>(1, (a.d + 4095) / 4096));

  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(S1_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, step1_kernel<W>, a);
  ++*launches;
  return e;
}

}  // namespace

cudaError_t step1_prepare() {
  cudaError_t e = prepare_w<4>();
  if (e == cudaSuccess) e = prepare_w<8>();
  if (e == cudaSuccess) e = prepare_w<16>();
  return e;
}

uint32_t step1_capacity(uint32_t w, uint32_t sm_count) {
  if (step1_prepare() != cudaSuccess) return 0;
  Launch& L = launch_state();
  std::lock_guard<std::mutex> g(L.mu);
  const int wi = w == 4 ? 0 : (w == 8 ? 1 : 2);
  return (uint32_t)L.per_sm[wi] * sm_count;
}

uint32_t sort_tiles(uint64_t d) { return (uint32_t)((d + RS_TILE - 1) / RS_TILE); }
uint32_t merge_tiles(uint64_t n) { return (uint32_t)((n + MG_TILE - 1) / MG_TILE); }

uint64_t step1_zeroed_words(uint32_t w, uint64_t n_merge, uint64_t d) {
  // merge look-back (64-bit words), barrier counters, digit histograms,
  // sort look-back
  return 2ull * merge_tiles(n_merge) + S1_BARRIERS + (d ? (uint64_t)w * 256 + (uint64_t)w * sort_tiles(d) * 256 : 0);
}

void step1_layout(uint32_t w, uint64_t n_merge, uint64_t d, uint32_t* zero, Step1Args* a) {
  const uint32_t mt = merge_tiles(n_merge);
  a->merge_lb = reinterpret_cast<uint64_t*>(zero);
  a->merge_tiles = mt;
  a->barriers = zero + 2ull * mt;
  uint32_t* z = a->barriers + S1_BARRIERS;
  a->hist = z;
  a->sort_tiles = sort_tiles(d);
  a->sort_lb = z + (uint64_t)w * 256;
}

cudaError_t launch_step1(uint32_t w, const Step1Args& a, cudaStream_t s, uint32_t sm_count, uint64_t* launches) {
  switch (w) {
    case 4: return launch_step1_w<4>(a, s, sm_count, launches);
    case 8: return launch_step1_w<8>(a, s, sm_count, launches);
    case 16: return launch_step1_w<16>(a, s, sm_count, launches);
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
    case 4: sort_copy_kernel<4><<<blocks, 256, 0, s>>>(final_slot, d, static_cast<uint32_t*>(ud_out), perm_out); break;
    case 8: sort_copy_kernel<8><<<blocks, 256, 0, s>>>(final_slot, d, static_cast<uint64_t*>(ud_out), perm_out); break;
    case 16: sort_copy_kernel<16><<<blocks, 256, 0, s>>>(final_slot, d, static_cast<u128*>(ud_out), perm_out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace dm

// ---------------------------------------------------------------- no-alloc variant
// Scratch of dm_merge_dicts_noalloc: the look-back words of every tile of a
// merge of up to DM_NOALLOC_MAX_ENTRIES entries, then the barrier counters.
// It is static device memory of this library, present on every device that
// loads it; host code must not pass the symbol itself to a kernel (on the
// host it only names a shadow), so the device address is looked up once per
// device with cudaGetSymbolAddress.
namespace {
constexpr uint32_t kNoAllocTiles = (DM_NOALLOC_MAX_ENTRIES + dm::MG_TILE - 1) / dm::MG_TILE;
static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocTiles + dm::S1_BARRIERS / 2];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
uint64_t* g_noalloc_addr[kMaxDevices] = {};
int g_noalloc_sms[kMaxDevices] = {};
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
  int sms = 0;
  {
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return DM_ECUDA;
      if (cudaDeviceGetAttribute(&g_noalloc_sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DM_ECUDA;
      g_noalloc_addr[dev] = static_cast<uint64_t*>(p);
    }
    scratch = g_noalloc_addr[dev];
    sms = g_noalloc_sms[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (m + d == 0) {
    if (cudaMemsetAsync(d_u, 0, 8, s) != cudaSuccess || cudaMemsetAsync(d_bits, 0, 4, s) != cudaSuccess)
      return DM_ECUDA;
    return DM_OK;
  }
  // look-back words and barrier counters must start at zero; the array
  // keeps whatever the previous call left
  dm::Step1Args a{};
  dm::step1_layout(w, m + d, 0, reinterpret_cast<uint32_t*>(scratch), &a);
  const size_t used = (size_t)dm::step1_zeroed_words(w, m + d, 0) * 4;
  if (cudaMemsetAsync(scratch, 0, used, s) != cudaSuccess) return DM_ECUDA;
  a.a = main_dict;
  a.m = m;
  a.b = ud;
  a.perm = perm;
  a.d = d;
  a.unew = new_dict;
  a.xm = x_main;
  a.xd = x_delta;
  a.d_u = d_u;
  a.d_bits = d_bits;
  a.phases = dm::S1_MERGE;
  a.status = d_status;
  uint64_t launches = 0;
  return dm::launch_step1(w, a, s, (uint32_t)sms, &launches) == cudaSuccess ? DM_OK : DM_ECUDA;
}
