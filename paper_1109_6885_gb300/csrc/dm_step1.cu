// Step 1 of the column merge in one persistent kernel: sort the delta
// dictionary (Step 1(a)), merge it with the main dictionary (Step 1(b)),
// publish the new width (Step 2(a)) and build the X_M directory used by
// Step 2(b).
//
// Step 1(a).  The paper walks the leaves of a CSB+ tree kept during inserts
// (Section 5.1); with the delta dictionary stored as an insertion-order
// array, Step 1(a) sorts (key, insertion code) pairs, perm[j] = insertion
// code of U_D[j] being the tuple-id map of Section 5.3.  One sweep counts
// the 8-bit digits of every byte; each block then derives the plan (first
// slot of every digit, bytes whose digit is not constant).  When every
// bucket of the most significant varying byte holds at most 2048 keys, one
// partition pass scatters the keys into those buckets (atomic cursors) and
// each block sorts a bucket in shared memory by (key, insertion code):
// a count/scatter on the next varying byte into 256 sub-buckets, each
// finished by one thread's insertion sort, or a block merge sort when a
// sub-bucket holds more than 32 keys;
// otherwise stable LSD passes run, each ranking 1024-key tiles with a warp
// multisplit and a decoupled look-back over earlier tiles.
//
// Step 1(b).  The paper cuts both dictionaries at N_T-quantiles and fixes
// the output offsets with a counter array and a prefix sum (Section 6.2.1).
// Here tile t owns merged positions [4096t, 4096t + 4096): a merge-path
// (co-rank) search cuts U_M and U_D (ties: the main value first).  Inside
// the tile, each U_D entry is ranked against the U_M segment by binary
// search; a U_D entry is a duplicate when it equals the key before it in
// merged order (a value in both dictionaries, or a repeat inside D_dict; a
// U_M entry never is), and every position's new code follows from the
// ranks and one block scan of the non-duplicates, plus the tile's offset
// from a decoupled look-back.  U'[code] receives each non-duplicate, X_M /
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
constexpr uint32_t SR_ITEMS = RS_ITEMS;               // sort keys per thread
constexpr uint32_t SR_TILE = S1_THREADS * SR_ITEMS;   // sort keys per sort tile
static_assert(SR_TILE == RS_TILE, "tile sizes");
static_assert(mg_tile(4) % (4 * S1_THREADS) == 0 && mg_tile(16) % (4 * S1_THREADS) == 0, "merge tiles");

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
__device__ __forceinline__ uint32_t spin_limit_of(const Step1Args& a) {
  return a.spin_limit ? a.spin_limit : kSpinLimit;
}

__device__ void grid_barrier(uint32_t* bars, uint32_t idx, uint32_t* status, uint32_t limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&bars[idx], 1u);
    uint32_t spins = 0;
    while (ld_volatile(&bars[idx]) < gridDim.x) {
      if (++spins > limit) {
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
  uint32_t next;                   // split form: the tile a block takes next
};

template <int W>
struct MergeSmem {
  using K = typename KeyOf<W>::T;
  static constexpr uint32_t T = mg_tile(W);
  K keys[T];                       // U_M segment then U_D segment
  // [0, na): per U_M entry, the U_D entries placed right before it, then
  // their prefix; [na, na + nb): the U_D segment's insertion codes
  alignas(16) uint32_t ap[T];
  uint16_t rank[T];                // per U_D entry: U_M entries of the tile at or below it
  uint16_t ndx[T + 1];             // per U_D entry: non-duplicate U_D entries before it (and the total)
  uint32_t wsum[S1_WARPS];
  uint64_t cut[2];
  uint64_t excl, lb_sum;
  uint32_t nearest;
  uint32_t next_tile;
  K prevA, prevB;
};

static_assert(mg_tile(4) < 65536 && mg_tile(16) < 65536, "16-bit ranks within a tile");

// Shared memory of the split form's merge kernel (the merge phase alone),
// and its blocks per SM: three with 4- and 8-byte keys, two with 16-byte.
template <int W>
constexpr size_t merge_smem_bytes() {
  return (sizeof(MergeSmem<W>) + 15) / 16 * 16;
}
constexpr int merge_blocks_min(int w) { return w == 16 ? 2 : 3; }

constexpr uint32_t BK_CAP = 2048;     // keys a block sorts in shared memory at once
constexpr uint32_t BK_SINGLE = BK_CAP;  // at most this many keys: one block sorts them all

template <int W>
struct BucketSmem {
  using K = typename KeyOf<W>::T;
  K keys[2][BK_CAP + BK_CAP / 16];   // ping-pong buffers of the merge rounds (bk_slot layout)
  uint32_t vals[2][BK_CAP + BK_CAP / 16];
  uint32_t cnt[256];                 // sub-bucket counts, then cursors
  uint32_t wsum[S1_WARPS];
};
constexpr uint32_t BK_SUB_MAX = 32;   // largest sub-bucket one thread sorts by insertion

// The sort plan (first slot of every digit) lives in front of the sort and
// bucket phases' memory; the merge phase, which no longer needs it, reuses
// the whole union.
template <int W>
struct SortPhase {
  uint32_t plan[W * 256];
  SortSmem<W> s;
};
template <int W>
struct BucketPhase {
  uint32_t plan[W * 256];
  BucketSmem<W> b;
};

template <int W>
union Step1Smem {
  SortPhase<W> sp;
  BucketPhase<W> bp;
  MergeSmem<W> m;
  uint32_t hist[W * 256];
};

template <int W>
constexpr size_t step1_smem_bytes() {
  return (sizeof(Step1Smem<W>) + 15) / 16 * 16 + 64;
}
// The split form's histogram, pass and partition kernels: the sort phase's
// memory (the plan and one sort tile) and the scan's warp sums after it.
template <int W>
constexpr size_t sort_smem_bytes() {
  return (sizeof(SortPhase<W>) + 15) / 16 * 16 + 64;
}
constexpr int SORT_BLOCKS_MIN = 3;

// ---------------------------------------------------------------- Step 1(a)
// Digit counts of every pass (blocks below hist_blocks take part; each
// thread loads HI_ITEMS keys at once, then counts them in shared memory).
constexpr uint32_t HI_ITEMS = 8;

template <int W>
__device__ void hist_phase(const Step1Args& a, uint32_t* sh) {
  using K = typename KeyOf<W>::T;
  if (blockIdx.x >= a.hist_blocks) return;
  for (uint32_t i = threadIdx.x; i < W * 256; i += S1_THREADS) sh[i] = 0;
  __syncthreads();
  const K* keys = static_cast<const K*>(a.in_keys);
  const uint64_t stride = (uint64_t)a.hist_blocks * S1_THREADS * HI_ITEMS;
  for (uint64_t base = (uint64_t)blockIdx.x * S1_THREADS * HI_ITEMS + threadIdx.x; base < a.d; base += stride) {
    K k[HI_ITEMS];
#pragma unroll
    for (int q = 0; q < (int)HI_ITEMS; ++q) {
      const uint64_t idx = base + (uint64_t)q * S1_THREADS;
      if (idx < a.d) k[q] = load_key(keys + idx);
    }
#pragma unroll
    for (int q = 0; q < (int)HI_ITEMS; ++q) {
      if (base + (uint64_t)q * S1_THREADS < a.d) {
#pragma unroll
        for (int p = 0; p < W; ++p) atomicAdd(&sh[p * 256 + key_digit(k[q], p)], 1u);
      }
    }
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

// The sort plan from the global histogram, computed by every block: the
// mask of bytes whose digit varies (a byte whose digit is the same for every
// key is skipped; if none varies, the last one runs so the result always
// lands in a ping-pong buffer), and the first slot of every digit of the
// bytes that will be passed over.
//
// It also decides between the two ways to finish the sort: when every bucket
// of the most significant byte that varies holds at most BK_CAP keys, one
// partition on that byte plus one sort of each bucket in shared memory
// (*msd = true; only that byte's slots are computed); otherwise all varying
// bytes, least significant first.
template <int W>
__device__ uint32_t plan_phase(const Step1Args& a, uint32_t* s_plan, uint32_t* wsum, bool* msd) {
  const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
  uint32_t v[W];
#pragma unroll
  for (int p = 0; p < W; ++p) v[p] = ld_volatile(&a.hist[p * 256 + t]);
  // bytes whose digit is the same for every key: one vote for all bytes
  uint32_t cmask = 0;
#pragma unroll
  for (int p = 0; p < W; ++p) cmask |= ((uint64_t)v[p] == a.d ? 1u : 0u) << p;
  cmask = __reduce_or_sync(0xFFFFFFFFu, cmask);
  if (lane == 0) wsum[warp] = cmask;
  __syncthreads();
  cmask = 0;
#pragma unroll
  for (uint32_t w = 0; w < S1_WARPS; ++w) cmask |= wsum[w];
  __syncthreads();
  uint32_t run = ~cmask & ((1u << W) - 1u);
  run = run ? run : (1u << (W - 1));
  const int top = 31 - __clz(run);
  uint32_t vtop = 0;
#pragma unroll
  for (int p = 0; p < W; ++p)
    if (p == top) vtop = v[p];
  *msd = !__syncthreads_or(vtop > BK_CAP);
  if (*msd) {
    s_plan[top * 256 + t] = block_excl_scan(vtop, wsum, nullptr);
  } else {
#pragma unroll
    for (int p = 0; p < W; ++p)
      if ((run >> p) & 1u) s_plan[p * 256 + t] = block_excl_scan(v[p], wsum, nullptr);
  }
  __syncthreads();
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
    const uint32_t limit = spin_limit_of(a);
    bool done = false;
    while (!done && p >= 0) {
      uint32_t v[32];   // 32 predecessors per round trip
#pragma unroll
      for (int q = 0; q < 32; ++q) v[q] = (p - q >= 0) ? ld_volatile(&lb[(uint64_t)(p - q) * 256 + tid]) : LB_INC32;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        if (!done) {
          while ((v[q] >> 30) == 0) {   // not published yet
            if (++spins > limit) {
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
      flag_status(a.status, ST_INTERNAL);
    }
  }
  __syncthreads();
}

// One tile of the MSD partition on digit `top`: the input dictionary's keys
// go to their digit's bucket (its first slot from the plan), each tile
// claiming a run of every bucket with one atomic add on that bucket's cursor
// (zeroed).  The order inside a bucket is arbitrary; the bucket sort that
// follows orders by (key, insertion code).
template <int W>
__device__ void msd_tile(const Step1Args& a, int top, uint32_t tile, const uint32_t* s_plan, SortSmem<W>& S) {
  using K = typename KeyOf<W>::T;
  const uint32_t tid = threadIdx.x;
  const uint64_t d = a.d;
  const K* src = static_cast<const K*>(a.in_keys);
  K* dst_k = static_cast<K*>(a.keys[0]);
  uint32_t* dst_v = a.vals[0];
  uint32_t* cursor = a.sort_lb;
  S.tstart[tid] = 0;   // per-digit count of this tile
  __syncthreads();
  const uint64_t tbase = (uint64_t)tile * SR_TILE + tid;
  K key[SR_ITEMS];
  uint32_t dig[SR_ITEMS], rank[SR_ITEMS];
#pragma unroll
  for (int r = 0; r < (int)SR_ITEMS; ++r) {
    const uint64_t idx = tbase + (uint64_t)r * S1_THREADS;
    dig[r] = 256;
    if (idx < d) key[r] = load_key(src + idx);
  }
#pragma unroll
  for (int r = 0; r < (int)SR_ITEMS; ++r) {
    if (tbase + (uint64_t)r * S1_THREADS < d) {
      dig[r] = key_digit(key[r], top);
      rank[r] = atomicAdd(&S.tstart[dig[r]], 1u);
    }
  }
  __syncthreads();
  const uint32_t c = S.tstart[tid];
  if (c) S.gbase[tid] = s_plan[top * 256 + tid] + atomicAdd(&cursor[tid], c);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < (int)SR_ITEMS; ++r) {
    if (dig[r] < 256) {
      const uint64_t pos = (uint64_t)S.gbase[dig[r]] + rank[r];
      if (pos < d) {
        dst_k[pos] = key[r];
        dst_v[pos] = (uint32_t)(tbase + (uint64_t)r * S1_THREADS);
      } else {
        flag_status(a.status, ST_INTERNAL);
      }
    }
  }
  __syncthreads();
}

// (key, insertion code) order; codes are distinct, so it is the stable order.
template <class K>
__device__ __forceinline__ bool kv_lt(const K& ka, uint32_t va, const K& kb, uint32_t vb) {
  return key_lt(ka, kb) || (key_eq(ka, kb) && va < vb);
}

// Shared-memory slot of bucket entry i: one unused slot after every 16, so
// that threads reading or writing their own runs of consecutive entries
// spread over the banks.
__device__ __forceinline__ uint32_t bk_slot(uint32_t i) { return i + (i >> 4); }

// Sort n <= BK_CAP (key, insertion code) pairs of one bucket in shared
// memory and write them to dst at the same offsets.  Block merge sort over
// two shared buffers: the bucket is padded to N = 2^k entries with (max key,
// max code); thread t owns the I = max(1, N / threads) entries [tI, tI + I),
// sorts them by insertion, then every round merges neighbouring sorted runs
// into the other buffer, each thread producing its I outputs after a
// merge-path search.  Both run heads stay in registers, so an output costs
// one unconditional load of the next entry.  src_v == nullptr: the codes are
// the positions (input dictionary); coherent: src was written earlier in
// this kernel.
template <int W>
__device__ void bucket_sort(const typename KeyOf<W>::T* src_k, const uint32_t* src_v, uint64_t off, uint32_t n,
                            bool coherent, typename KeyOf<W>::T* dst_k, uint32_t* dst_v, BucketSmem<W>& S) {
  using K = typename KeyOf<W>::T;
  constexpr uint32_t R = BK_CAP / S1_THREADS;
  const uint32_t tid = threadIdx.x;
  uint32_t N = 2;
  while (N < n) N <<= 1;
  const uint32_t I = N > S1_THREADS ? N / S1_THREADS : 1;   // entries per thread
  const uint32_t T = N / I;                                  // threads with entries
  {
    K kr[R];
    uint32_t vr[R];
#pragma unroll
    for (uint32_t r = 0; r < R; ++r) {
      const uint32_t i = tid + r * S1_THREADS;
      kr[r] = key_max_value<K>();
      vr[r] = 0xFFFFFFFFu;
      if (i < n) {
        kr[r] = coherent ? ldcg_key(src_k + off + i) : load_key(src_k + off + i);
        vr[r] = src_v ? (coherent ? __ldcg(src_v + off + i) : __ldg(src_v + off + i)) : (uint32_t)(off + i);
      }
    }
#pragma unroll
    for (uint32_t r = 0; r < R; ++r) {
      const uint32_t i = tid + r * S1_THREADS;
      if (i < N) {
        S.keys[0][bk_slot(i)] = kr[r];
        S.vals[0][bk_slot(i)] = vr[r];
      }
    }
  }
  __syncthreads();
  if (tid < T && I > 1) {
    K* kk = S.keys[0];
    uint32_t* vv = S.vals[0];
    const uint32_t o = tid * I;
#pragma unroll 1
    for (uint32_t i = 1; i < I; ++i) {
      const K x = kk[bk_slot(o + i)];
      const uint32_t y = vv[bk_slot(o + i)];
      uint32_t j = i;
      while (j > 0) {
        const K z = kk[bk_slot(o + j - 1)];
        const uint32_t zv = vv[bk_slot(o + j - 1)];
        if (!kv_lt(x, y, z, zv)) break;
        kk[bk_slot(o + j)] = z;
        vv[bk_slot(o + j)] = zv;
        --j;
      }
      kk[bk_slot(o + j)] = x;
      vv[bk_slot(o + j)] = y;
    }
  }
  uint32_t cur = 0;
#pragma unroll 1
  for (uint32_t w = I; w < N; w <<= 1) {
    __syncthreads();
    if (tid < T) {
      const K* sk = S.keys[cur];
      const uint32_t* sv = S.vals[cur];
      K* dk = S.keys[cur ^ 1];
      uint32_t* dv = S.vals[cur ^ 1];
      // outputs [tI, tI + I) of the merged run [base, base + 2w)
      const uint32_t o = tid * I;
      const uint32_t base = o & ~(2 * w - 1);
      const uint32_t diag = o - base;
      const uint32_t a0 = base, b0 = base + w;
      // entries taken from the first run (ties go to the first run)
      uint32_t lo = diag > w ? diag - w : 0, hi = diag < w ? diag : w;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint32_t ja = bk_slot(a0 + mid), jb = bk_slot(b0 + diag - 1 - mid);
        const K xa = sk[ja], xb = sk[jb];
        const uint32_t va = sv[ja], vb = sv[jb];
        if (kv_lt(xb, vb, xa, va)) hi = mid;
        else lo = mid + 1;
      }
      uint32_t ia = a0 + lo, ib = b0 + (diag - lo);
      const uint32_t ea = a0 + w, eb = b0 + w;
      K ka = sk[bk_slot(min(ia, ea - 1))], kb = sk[bk_slot(min(ib, eb - 1))];
      uint32_t va = sv[bk_slot(min(ia, ea - 1))], vb = sv[bk_slot(min(ib, eb - 1))];
#pragma unroll 1
      for (uint32_t q = 0; q < I; ++q) {
        const bool takeA = ia < ea && (ib >= eb || !kv_lt(kb, vb, ka, va));
        dk[bk_slot(o + q)] = takeA ? ka : kb;
        dv[bk_slot(o + q)] = takeA ? va : vb;
        ia += takeA;
        ib += !takeA;
        const uint32_t nx = bk_slot(takeA ? min(ia, ea - 1) : min(ib, eb - 1));
        const K kn = sk[nx];
        const uint32_t vn = sv[nx];
        ka = takeA ? kn : ka;
        va = takeA ? vn : va;
        kb = takeA ? kb : kn;
        vb = takeA ? vb : vn;
      }
    }
    cur ^= 1;
  }
  __syncthreads();
  for (uint32_t i = tid; i < n; i += S1_THREADS) {
    dst_k[off + i] = S.keys[cur][bk_slot(i)];
    dst_v[off + i] = S.vals[cur][bk_slot(i)];
  }
  __syncthreads();
}

// Sort one bucket (as bucket_sort) by one more counting-sort level: the
// keys are counted and scattered on byte `sub` (the next byte below the
// bucket's that varies) into 256 sub-buckets, and each thread sorts one
// sub-bucket by insertion on (key, insertion code).  A bucket with a
// sub-bucket above BK_SUB_MAX keys goes to the merge sort instead.
template <int W>
__device__ void bucket_sort_sub(const typename KeyOf<W>::T* src_k, const uint32_t* src_v, uint64_t off, uint32_t n,
                                bool coherent, typename KeyOf<W>::T* dst_k, uint32_t* dst_v, int sub,
                                BucketSmem<W>& S) {
  using K = typename KeyOf<W>::T;
  constexpr uint32_t R = BK_CAP / S1_THREADS;
  const uint32_t tid = threadIdx.x;
  K kr[R];
  uint32_t vr[R], dg[R];
  S.cnt[tid] = 0;
#pragma unroll
  for (uint32_t r = 0; r < R; ++r) {
    const uint32_t i = tid + r * S1_THREADS;
    dg[r] = 256;
    if (i < n) {
      kr[r] = coherent ? ldcg_key(src_k + off + i) : load_key(src_k + off + i);
      vr[r] = src_v ? (coherent ? __ldcg(src_v + off + i) : __ldg(src_v + off + i)) : (uint32_t)(off + i);
    }
  }
  __syncthreads();
#pragma unroll
  for (uint32_t r = 0; r < R; ++r) {
    if (tid + r * S1_THREADS < n) {
      dg[r] = key_digit(kr[r], sub);
      atomicAdd(&S.cnt[dg[r]], 1u);
    }
  }
  __syncthreads();
  const uint32_t c = S.cnt[tid];
  if (__syncthreads_or(c > BK_SUB_MAX)) {
    bucket_sort<W>(src_k, src_v, off, n, coherent, dst_k, dst_v, S);
    return;
  }
  uint32_t total = 0;
  const uint32_t st = block_excl_scan(c, S.wsum, &total);
  S.cnt[tid] = st;   // cursor of sub-bucket tid
  __syncthreads();
  K* kk = S.keys[0];
  uint32_t* vv = S.vals[0];
#pragma unroll
  for (uint32_t r = 0; r < R; ++r) {
    if (dg[r] < 256) {
      const uint32_t pos = atomicAdd(&S.cnt[dg[r]], 1u);
      if (pos < BK_CAP) {
        kk[pos] = kr[r];
        vv[pos] = vr[r];
      }
    }
  }
  __syncthreads();
  // sub-bucket tid: entries [st, st + c)
#pragma unroll 1
  for (uint32_t i = 1; i < c; ++i) {
    const K x = kk[st + i];
    const uint32_t y = vv[st + i];
    uint32_t j = i;
    while (j > 0) {
      const K z = kk[st + j - 1];
      const uint32_t zv = vv[st + j - 1];
      if (!kv_lt(x, y, z, zv)) break;
      kk[st + j] = z;
      vv[st + j] = zv;
      --j;
    }
    kk[st + j] = x;
    vv[st + j] = y;
  }
  __syncthreads();
  for (uint32_t i = tid; i < n; i += S1_THREADS) {
    dst_k[off + i] = kk[i];
    dst_v[off + i] = vv[i];
  }
  __syncthreads();
}

// Whether bucket [off, off + n) of the top-byte partition is one for the
// shared-memory sort: more than one key, inside the d keys, at most BK_CAP.
// The plan guarantees the last two unless a grid barrier before it timed out
// (the histogram it read was then incomplete); such a bucket is skipped and
// flagged, so that a timed-out wait never leads to an access out of bounds.
__device__ __forceinline__ bool bucket_ok(const Step1Args& a, uint32_t off, uint32_t n) {
  if (n <= 1) return false;
  if (n > BK_CAP || (uint64_t)off + n > a.d) {
    if (threadIdx.x == 0) flag_status(a.status, ST_INTERNAL);
    return false;
  }
  return true;
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
                           bool bcoh, bool precut, MergeSmem<W>& S) {
  using K = typename KeyOf<W>::T;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const K* A = static_cast<const K*>(a.a);
  const uint64_t m = a.m, d = a.d, n = m + d;

  constexpr uint32_t T = MergeSmem<W>::T;   // merged positions per tile
  constexpr uint32_t E = T / S1_THREADS;     // U_M prefix entries per thread
  const uint64_t k0 = (uint64_t)tile * T;
  const uint64_t k1 = k0 + T < n ? k0 + T : n;
  if (precut) {
    if (tid == 0) {
      // co-ranks found by another kernel or phase; clamped to a consistent
      // pair (c0 a co-rank of k0, c1 one of k1, both segments of
      // non-negative length), which they are unless the wait that ordered
      // them timed out: then the tile is wrong but stays in bounds
      const uint64_t r0 = __ldcg(a.cuts + tile), r1 = __ldcg(a.cuts + tile + 1);
      const uint64_t c0 = min(max(r0, k0 > d ? k0 - d : (uint64_t)0), min(k0, m));
      const uint64_t lo1 = max(c0, k1 > d ? k1 - d : (uint64_t)0), hi1 = min(c0 + (k1 - k0), m);
      S.cut[0] = c0;
      S.cut[1] = min(max(r1, lo1), hi1);
    }
  } else if (warp < 2) {
    const uint64_t c = corank_warp(A, m, B, d, warp == 0 ? k0 : k1, bcoh);
    if (lane == 0) S.cut[warp] = c;
  }
  __syncthreads();
  const uint64_t i0 = S.cut[0], i1 = S.cut[1];
  const uint64_t j0 = k0 - i0, j1 = k1 - i1;
  const uint32_t na = (uint32_t)(i1 - i0), nb = (uint32_t)(j1 - j0), nt = na + nb;
  // the segments, their perm entries, and the keys just before the tile
  // (merge predecessor and sortedness check), in batches whose loads are
  // all in flight before the first store (two batches for 16-byte keys,
  // for registers)
  if (tid == 0 && i0 > 0) S.prevA = load_key(A + i0 - 1);
  if (tid == 32 && j0 > 0) S.prevB = ld_key(B + j0 - 1, bcoh);
  {
    constexpr uint32_t R = T / S1_THREADS;
    constexpr uint32_t RB = W == 16 ? R / 2 : R;   // loads per batch
#pragma unroll
    for (uint32_t r0 = 0; r0 < R; r0 += RB) {
      K kr[RB];
      uint32_t pr[RB];
#pragma unroll
      for (uint32_t r = 0; r < RB; ++r) {
        const uint32_t x = tid + (r0 + r) * S1_THREADS;
        if (x < na) {
          kr[r] = load_key(A + i0 + x);
        } else if (x < nt) {
          kr[r] = ld_key(B + j0 + (x - na), bcoh);
          pr[r] = bcoh ? __ldcg(perm + j0 + (x - na)) : __ldg(perm + j0 + (x - na));
        }
      }
#pragma unroll
      for (uint32_t r = 0; r < RB; ++r) {
        const uint32_t x = tid + (r0 + r) * S1_THREADS;
        if (x < nt) S.keys[x] = kr[r];
        if (x < na) S.ap[x] = 0;
        else if (x < nt) S.ap[x] = pr[r];
      }
    }
  }
  __syncthreads();
  const K* sA = S.keys;
  const K* sB = S.keys + na;

  // U_M must be strictly increasing
#pragma unroll 4
  for (uint32_t x = tid; x < na; x += S1_THREADS) {
    if (i0 + x == 0) continue;
    const K prev = x > 0 ? sA[x - 1] : S.prevA;
    if (!key_lt(prev, sA[x])) flag_status(a.status, ST_UNSORTED);
  }

  // Merged order inside the tile (ties: the U_M entry first).  U_D entry j
  // follows the rank_j = #{i : U_M[i] <= U_D[j]} U_M entries of the tile;
  // U_M entry i follows the U_D entries with rank <= i.  One fixed-step
  // binary search per U_D entry, spread over all threads.
  {
    const uint32_t top = na ? 1u << (31 - __clz(na)) : 0u;
    for (uint32_t j = tid; j < nb; j += S1_THREADS) {
      const K x = sB[j];
      uint32_t r = 0;
      for (uint32_t step = top; step > 0; step >>= 1) {
        const uint32_t p = r + step;
        const K v = sA[min(p, na) - 1];
        r = (p <= na && key_le(v, x)) ? p : r;
      }
      S.rank[j] = r;
      if (r < na) atomicAdd(&S.ap[r], 1u);
    }
  }
  __syncthreads();

  // duplicates: a U_D entry equal to the key before it in merged order (a
  // U_M entry never is: U_M increases and ties put it first)
  K kp{};
  if (i0 > 0 && j0 > 0) kp = key_max(S.prevA, S.prevB);   // the key at merged position k0 - 1
  else if (i0 > 0) kp = S.prevA;
  else if (j0 > 0) kp = S.prevB;
  auto nondup_at = [&](uint32_t j) -> uint32_t {
    if (j >= nb) return 0u;
    const uint32_t r = S.rank[j];
    bool has_prev = true;
    K pk;
    if (j > 0 && S.rank[j - 1] == r) pk = sB[j - 1];
    else if (r > 0) pk = sA[r - 1];
    else {
      pk = kp;
      has_prev = k0 > 0;
    }
    return has_prev && key_eq(sB[j], pk) ? 0u : 1u;
  };
  // U_D entries placed before this thread's U_M entries [Et, Et + E)
  // (entries at or past na hold insertion codes: they count as zero)
  uint32_t cinc[E];
  {
    uint32_t run = 0;
#pragma unroll
    for (uint32_t v = 0; v < E / 4; ++v) {
      const uint32_t i = E * tid + 4 * v;
      const uint4 c = reinterpret_cast<const uint4*>(S.ap)[(E / 4) * tid + v];
      cinc[4 * v] = run += i < na ? c.x : 0u;
      cinc[4 * v + 1] = run += i + 1 < na ? c.y : 0u;
      cinc[4 * v + 2] = run += i + 2 < na ? c.z : 0u;
      cinc[4 * v + 3] = run += i + 3 < na ? c.w : 0u;
    }
  }
  // the U_M prefix and the first round of U_D non-duplicates in one block
  // scan (each total is at most 4096: 16 bits), further rounds alone
  uint32_t total = 0;
  const uint32_t pex = block_excl_scan((nondup_at(tid) << 16) | cinc[E - 1], S.wsum, &total);
  {
    const uint32_t cx = pex & 0xFFFFu;
#pragma unroll
    for (uint32_t v = 0; v < E / 4; ++v) {
      const uint32_t i = E * tid + 4 * v;
      if (i + 3 < na) {
        reinterpret_cast<uint4*>(S.ap)[(E / 4) * tid + v] =
            make_uint4(cx + cinc[4 * v], cx + cinc[4 * v + 1], cx + cinc[4 * v + 2], cx + cinc[4 * v + 3]);
      } else {
#pragma unroll
        for (uint32_t q = 0; q < 4; ++q)
          if (i + q < na) S.ap[i + q] = cx + cinc[4 * v + q];
      }
    }
  }
  if (tid < nb) S.ndx[tid] = pex >> 16;
  uint32_t ndB = total >> 16;
  for (uint32_t q = 1; q * S1_THREADS < nb; ++q) {
    const uint32_t j = q * S1_THREADS + tid;
    uint32_t tq = 0;
    const uint32_t e = block_excl_scan(nondup_at(j), S.wsum, &tq);
    if (j < nb) S.ndx[j] = ndB + e;
    ndB += tq;
  }
  if (tid == 0) S.ndx[nb] = ndB;
  const uint32_t ttotal = na + ndB;

  // decoupled look-back: the whole block reads 256 predecessors per round
  // trip and sums them down to the nearest inclusive prefix
  // (a tile the test setting names publishes nothing, so that the waits
  // of the tiles after it run out)
  const bool publish = a.test_withhold != tile + 1;
  if (tile == 0) {
    if (tid == 0) {
      if (publish) st_volatile(&a.merge_lb[0], LB_INC64 | ttotal);
      S.excl = 0;
    }
  } else {
    if (tid == 0) {
      if (publish) st_volatile(&a.merge_lb[tile], LB_AGG64 | ttotal);
      S.lb_sum = 0;
    }
    int64_t top = (int64_t)tile - 1;
    uint32_t spins = 0;
    const uint32_t limit = spin_limit_of(a);
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
        if (++spins > limit) {
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
      if (publish) st_volatile(&a.merge_lb[tile], LB_INC64 | (S.lb_sum + ttotal));
    }
  }
  __syncthreads();

  // codes and writes.  U_M entry i: code = excl + i + (non-duplicate U_D
  // entries before it); U_D entry j: code = excl + rank_j + (non-duplicate
  // U_D entries before it), minus one for a duplicate (the code of the
  // equal key before it).  U' and X_M go out in U_M order (consecutive
  // threads, nearly consecutive codes); X_D is scattered through perm.
  const uint64_t excl = S.excl;
  K* unew = static_cast<K*>(a.unew);
#pragma unroll 4
  for (uint32_t x = tid; x < na; x += S1_THREADS) {
    const uint64_t code = excl + x + S.ndx[S.ap[x]];
    if (code < n) {
      unew[code] = sA[x];
      a.xm[i0 + x] = (uint32_t)code;
    } else {
      flag_status(a.status, ST_INTERNAL);
    }
  }
  for (uint32_t j = tid; j < nb; j += S1_THREADS) {
    const uint32_t before = S.ndx[j];
    const bool nondup = S.ndx[j + 1] != before;
    const uint64_t code = excl + S.rank[j] + before - (nondup ? 0u : 1u);
    if (code >= n) {
      flag_status(a.status, ST_INTERNAL);
      continue;
    }
    if (nondup) unew[code] = sB[j];
    const uint32_t pj = S.ap[na + j];
    if (pj < d) a.xd[pj] = (uint32_t)code;
    else flag_status(a.status, ST_CODE);
  }
  if (tile == a.merge_tiles - 1 && tid == 0) {
    const uint64_t u = excl + ttotal;
    *a.d_u = u;
    *a.d_bits = bits_for(u);
  }
  __syncthreads();
}

// ---------------------------------------------------------------- small dictionaries
// Steps 1(a), 1(b) and 2(a) of a column whose dictionaries are small (at most
// SM_MAX_M main and SM_MAX_D delta entries) by one block with a short code
// path.  The tiled kernel spends 20-35 us on such a column whatever its size:
// its phases and grid barriers run once through a long, cold instruction
// stream.  Here both dictionaries sit in shared memory and every code comes
// from binary searches:
//   * each delta value is ranked in U_M; the values not in U_M (the new
//     values of U') are gathered, sorted (bitonic) and counted once each;
//   * with q(x) the number of distinct new values below x, U_M[i] takes code
//     i + q(U_M[i]), a distinct new value v takes #{U_M < v} + q(v), and
//     delta entry j takes #{U_M < D[j]} + q(D[j]) (U' is the sorted union
//     without duplicates, Eq. 3; X_M and X_D give each value's position in
//     it, Section 5.3).
// Repeated delta values get one code; a U_M that is not strictly increasing
// is flagged as the tiled kernel flags it.  No wait, no look-back.
constexpr uint32_t SM_MAX_M = 4096, SM_MAX_D = 2048;

template <int W>
constexpr size_t small_smem_bytes() {
  return (size_t)(SM_MAX_M + 2 * SM_MAX_D) * W + (size_t)(2 * SM_MAX_D + 1 + S1_WARPS) * 4;
}

// First index of s[0..n) whose key is not below x (lower) or above x (upper).
template <class K>
__device__ __forceinline__ uint32_t bound_s(const K* s, uint32_t n, const K& x, bool upper) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (upper ? !key_lt(x, s[mid]) : key_lt(s[mid], x)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Exclusive scan of flag(k), k < n <= SM_MAX_D, into out[0..n]; returns the
// total (out[n]).  Every thread takes a run of consecutive k.
template <class F>
__device__ __forceinline__ uint32_t small_scan(uint32_t n, F flag, uint32_t* out, uint32_t* wsum) {
  constexpr uint32_t PER = SM_MAX_D / S1_THREADS;
  const uint32_t k0 = threadIdx.x * PER;
  uint32_t f[PER], sum = 0;
#pragma unroll
  for (uint32_t q = 0; q < PER; ++q) {
    f[q] = k0 + q < n ? flag(k0 + q) : 0u;
    sum += f[q];
  }
  uint32_t total = 0;
  uint32_t ex = block_excl_scan(sum, wsum, &total);
#pragma unroll
  for (uint32_t q = 0; q < PER; ++q) {
    if (k0 + q < n) out[k0 + q] = ex;
    ex += f[q];
  }
  if (threadIdx.x == 0) out[n] = total;
  __syncthreads();
  return total;
}

template <int W>
__global__ void __launch_bounds__(S1_THREADS) step1_small_kernel(Step1Args a) {
  using K = typename KeyOf<W>::T;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  K* sA = reinterpret_cast<K*>(smem_raw);
  K* sD = sA + SM_MAX_M;
  K* sN = sD + SM_MAX_D;
  uint32_t* lbm = reinterpret_cast<uint32_t*>(sN + SM_MAX_D);   // #{U_M < D[j]}, bit 31: D[j] is new
  uint32_t* q = lbm + SM_MAX_D;                                  // scans, SM_MAX_D + 1 words
  uint32_t* wsum = q + SM_MAX_D + 1;
  const uint32_t tid = threadIdx.x;
  const uint32_t m = (uint32_t)a.m, d = (uint32_t)a.d;
  const K* A = static_cast<const K*>(a.a);
  const K* D = static_cast<const K*>(a.in_keys);
  for (uint32_t i = tid; i < m; i += S1_THREADS) sA[i] = load_key(A + i);
  for (uint32_t j = tid; j < d; j += S1_THREADS) sD[j] = load_key(D + j);
  __syncthreads();
  bool unsorted = false;
  for (uint32_t i = tid + 1; i < m; i += S1_THREADS) unsorted |= !key_lt(sA[i - 1], sA[i]);
  if (unsorted) flag_status(a.status, ST_UNSORTED);
  for (uint32_t j = tid; j < d; j += S1_THREADS) {
    const uint32_t r = bound_s(sA, m, sD[j], true);
    const bool in_main = r > 0 && key_eq(sA[r - 1], sD[j]);
    lbm[j] = in_main ? r - 1 : (r | 0x80000000u);
  }
  __syncthreads();
  // the new values, gathered in delta order, then sorted (padded with the
  // largest key to a power of two; only the first nn are read)
  const uint32_t nn = small_scan(d, [&](uint32_t j) { return lbm[j] >> 31; }, q, wsum);
  for (uint32_t j = tid; j < d; j += S1_THREADS)
    if (lbm[j] >> 31) sN[q[j]] = sD[j];
  uint32_t np = 1;
  while (np < nn) np <<= 1;
  for (uint32_t k = nn + tid; k < np; k += S1_THREADS) sN[k] = key_max_value<K>();
  __syncthreads();
  for (uint32_t k = 2; k <= np; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = tid; i < np; i += S1_THREADS) {
        const uint32_t l = i ^ j;
        if (l > i) {
          const K x = sN[i], y = sN[l];
          if ((i & k) == 0 ? key_lt(y, x) : key_lt(x, y)) {
            sN[i] = y;
            sN[l] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  // q[k]: distinct new values among sN[0..k)
  const uint32_t nd = small_scan(nn, [&](uint32_t k) { return k == 0 || !key_eq(sN[k - 1], sN[k]) ? 1u : 0u; },
                                 q, wsum);
  const uint32_t u = m + nd;
  K* unew = static_cast<K*>(a.unew);
  for (uint32_t i = tid; i < m; i += S1_THREADS) {
    const uint32_t code = i + q[bound_s(sN, nn, sA[i], false)];
    if (code < u) {
      unew[code] = sA[i];
      a.xm[i] = code;
    } else {
      flag_status(a.status, ST_INTERNAL);
    }
  }
  for (uint32_t k = tid; k < nn; k += S1_THREADS) {
    if (k > 0 && key_eq(sN[k - 1], sN[k])) continue;
    const uint32_t code = bound_s(sA, m, sN[k], false) + q[k];
    if (code < u) unew[code] = sN[k];
    else flag_status(a.status, ST_INTERNAL);
  }
  for (uint32_t j = tid; j < d; j += S1_THREADS) {
    const uint32_t code = (lbm[j] & 0x7FFFFFFFu) + q[bound_s(sN, nn, sD[j], false)];
    if (code < u) a.xd[j] = code;
    else flag_status(a.status, ST_INTERNAL);
  }
  if (tid == 0) {
    *a.d_u = u;
    *a.d_bits = bits_for(u);
  }
}

// ---------------------------------------------------------------- the kernel
template <int W>
__global__ void __launch_bounds__(S1_THREADS, 2) step1_kernel(Step1Args a) {
  using K = typename KeyOf<W>::T;
  extern __shared__ __align__(16) unsigned char dsmem[];
  Step1Smem<W>& U = *reinterpret_cast<Step1Smem<W>*>(dsmem);
  uint32_t* s_plan = U.sp.plan;   // the same words as U.bp.plan
  uint32_t* s_wsum = reinterpret_cast<uint32_t*>(dsmem + (sizeof(Step1Smem<W>) + 15) / 16 * 16);

  uint32_t nbar = 0;
  const K* ud = static_cast<const K*>(a.b);
  const uint32_t* up = a.perm;
  bool coherent = false;
  if ((a.phases & S1_SORT) && a.d > 0) {
    K* k0 = static_cast<K*>(a.keys[0]);
    uint32_t* v0 = a.vals[0];
    if (a.d <= BK_SINGLE) {
      // a delta dictionary this small is sorted by one block
      if (blockIdx.x == 0) bucket_sort<W>(static_cast<const K*>(a.in_keys), nullptr, 0, (uint32_t)a.d, false, k0, v0, U.bp.b);
      ud = k0;
      up = v0;
    } else {
      hist_phase<W>(a, U.hist);
      grid_barrier(a.barriers, nbar++, a.status, spin_limit_of(a));
      bool msd = false;
      const uint32_t run = plan_phase<W>(a, s_plan, s_wsum, &msd);
      if (msd) {
        // one stable pass on the top varying digit, then each of its 256
        // buckets sorted in shared memory in place
        const int top = 31 - __clz(run);
        for (uint32_t t = blockIdx.x; t < a.sort_tiles; t += gridDim.x) msd_tile<W>(a, top, t, s_plan, U.sp.s);
        grid_barrier(a.barriers, nbar++, a.status, spin_limit_of(a));
        // the next byte below the top one that varies splits each bucket once more
        const uint32_t lower = run & ((1u << top) - 1u);
        const int sub = lower ? 31 - __clz(lower) : -1;
        for (uint32_t b = blockIdx.x; b < 256; b += gridDim.x) {
          const uint32_t off = s_plan[top * 256 + b];
          const uint32_t n = (b < 255 ? s_plan[top * 256 + b + 1] : (uint32_t)a.d) - off;
          if (!bucket_ok(a, off, n)) continue;
          if (sub >= 0) bucket_sort_sub<W>(k0, v0, off, n, true, k0, v0, sub, U.bp.b);
          else bucket_sort<W>(k0, v0, off, n, true, k0, v0, U.bp.b);
        }
        ud = k0;
        up = v0;
      } else {
        int e = 0;
        for (int p = 0; p < W; ++p) {
          if (!((run >> p) & 1u)) continue;
          for (uint32_t t = blockIdx.x; t < a.sort_tiles; t += gridDim.x) pass_tile<W>(a, p, t, e, s_plan, U.sp.s);
          grid_barrier(a.barriers, nbar++, a.status, spin_limit_of(a));
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
    if (a.phases & (S1_MERGE | S1_DIR)) grid_barrier(a.barriers, nbar++, a.status, spin_limit_of(a));
  }
  if ((a.phases & S1_MERGE) && a.m + a.d > 0) {
    // a merge of several waves of tiles finds every tile boundary first, one
    // warp per boundary, so that each tile starts with its loads
    const bool precut = a.cuts != nullptr && a.merge_tiles > gridDim.x;
    if (precut) {
      constexpr uint32_t T = MergeSmem<W>::T;
      const uint64_t n = a.m + a.d;
      const uint32_t lane = threadIdx.x & 31;
      const uint32_t nwt = gridDim.x * S1_WARPS;
      for (uint32_t b = blockIdx.x * S1_WARPS + (threadIdx.x >> 5); b <= a.merge_tiles; b += nwt) {
        const uint64_t k = (uint64_t)b * T < n ? (uint64_t)b * T : n;
        const uint64_t c = corank_warp(static_cast<const K*>(a.a), a.m, ud, a.d, k, coherent);
        if (lane == 0) a.cuts[b] = c;
      }
      grid_barrier(a.barriers, nbar++, a.status, spin_limit_of(a));
    }
    // block b merges tile b; further tiles (a merge of several waves) are
    // taken in index order from a counter, so that a tile's look-back only
    // waits on tiles already being merged
    uint32_t* next = a.barriers + S1_BARRIERS - 1;
    for (uint32_t t = blockIdx.x; t < a.merge_tiles;) {
      merge_tile<W>(a, t, ud, up, coherent, precut, U.m);
      if (a.merge_tiles <= gridDim.x) break;
      if (threadIdx.x == 0) U.m.next_tile = gridDim.x + atomicAdd(next, 1u);
      __syncthreads();
      t = U.m.next_tile;
    }
  }
  if ((a.phases & S1_DIR) && a.dir_entries > 0) {
    grid_barrier(a.barriers, nbar++, a.status, spin_limit_of(a));
    const bool use_x8 = a.x8 != nullptr && xdir_x8_pays<true>(a.xm, (uint32_t)a.m, a.dir_entries);
    for (uint32_t b = blockIdx.x * S1_THREADS + threadIdx.x; b < a.dir_entries; b += gridDim.x * S1_THREADS)
      a.xdir[b] = xdir_entry<true>(a.xm, (uint32_t)a.m, a.dir_shift, b, use_x8);
    if (use_x8)
      xdir_x8_fill<true>(a.xm, (uint32_t)a.m, a.dir_shift, a.x8, blockIdx.x * S1_THREADS + threadIdx.x,
                         gridDim.x * S1_THREADS);
  }
}

// ---------------------------------------------------------------- split form
// When a launch may hold only a few blocks (several merges share the GPU,
// each cooperative grid capped so that all of them fit at once) and the
// merge has more tiles than that, the merge leaves the cooperative kernel:
// the kernel sorts (or does nothing), then the kernels below find every
// tile boundary, merge the tiles on as many blocks as the device holds, and
// build the X_M directory.  The merge needs no co-residency: each block
// takes its next tile from a counter, so a tile's look-back only waits on
// tiles that running blocks have already taken.

// The sort in the same spirit, for a delta dictionary too large for a capped
// grid: one kernel per step, every block deriving the plan from the global
// histogram, tiles of a pass taken from a per-pass counter (barriers[p]),
// so that a pass's look-back only waits on tiles already taken.  A pass over
// a byte the plan skips, or the passes when the plan partitions on the top
// byte instead (and the reverse), return at once.

// The byte below `top` that varies (-1: none), and whether a large sort
// took the two-level partition (its scan's decision word).
__device__ __forceinline__ int byte_below(uint32_t run, int top) {
  const uint32_t lower = run & ((1u << top) - 1u);
  return lower ? 31 - __clz(lower) : -1;
}
__device__ __forceinline__ bool joint_chosen(const Step1Args& a) {
  return a.joff != nullptr && __ldcg(a.joff + JOINT_BINS + 1) != 0u;
}

template <int W>
__global__ void __launch_bounds__(S1_THREADS, SORT_BLOCKS_MIN) step1_hist_kernel(Step1Args a) {
  extern __shared__ __align__(16) unsigned char dsmem[];
  hist_phase<W>(a, reinterpret_cast<uint32_t*>(dsmem));   // W * 256 counters
}

template <int W>
__global__ void __launch_bounds__(S1_THREADS, SORT_BLOCKS_MIN) step1_pass_kernel(Step1Args a, int pass) {
  extern __shared__ __align__(16) unsigned char dsmem[];
  SortPhase<W>& SP = *reinterpret_cast<SortPhase<W>*>(dsmem);
  uint32_t* s_wsum = reinterpret_cast<uint32_t*>(dsmem + (sizeof(SortPhase<W>) + 15) / 16 * 16);
  bool msd = false;
  const uint32_t run = plan_phase<W>(a, SP.plan, s_wsum, &msd);
  if (msd || !((run >> pass) & 1u) || joint_chosen(a)) return;
  const int e = __popc(run & ((1u << pass) - 1u));
  for (;;) {
    if (threadIdx.x == 0) SP.s.next = atomicAdd(a.barriers + pass, 1u);
    __syncthreads();
    const uint32_t t = SP.s.next;
    __syncthreads();
    if (t >= a.sort_tiles) break;
    pass_tile<W>(a, pass, t, e, SP.plan, SP.s);
  }
}

template <int W>
__global__ void __launch_bounds__(S1_THREADS, SORT_BLOCKS_MIN) step1_msd_kernel(Step1Args a) {
  extern __shared__ __align__(16) unsigned char dsmem[];
  SortPhase<W>& SP = *reinterpret_cast<SortPhase<W>*>(dsmem);
  uint32_t* s_wsum = reinterpret_cast<uint32_t*>(dsmem + (sizeof(SortPhase<W>) + 15) / 16 * 16);
  bool msd = false;
  const uint32_t run = plan_phase<W>(a, SP.plan, s_wsum, &msd);
  if (!msd) return;
  const int top = 31 - __clz(run);
  for (uint32_t t = blockIdx.x; t < a.sort_tiles; t += gridDim.x) msd_tile<W>(a, top, t, SP.plan, SP.s);
}

// ---- two-level partition of a large sort (split form)
// When the plan's top varying byte leaves a bucket above BK_CAP keys (more
// than 256 * BK_CAP keys in all make that certain), the keys are binned on
// their two most significant varying bytes instead: a histogram of the
// JOINT_BINS bins, one block's scan of it (which also checks that every bin
// fits the shared-memory sort, else the LSD passes run as before), one
// scatter into the bins, and in-place sorts of groups of consecutive bins by
// (key, insertion code).  Three passes over the keys instead of one per
// varying byte.
static_assert(JOINT_MIN_KEYS == 256ull * BK_CAP, "a top-byte bucket above BK_CAP keys");

template <int W>
__global__ void __launch_bounds__(S1_THREADS, SORT_BLOCKS_MIN) step1_jhist_kernel(Step1Args a) {
  using K = typename KeyOf<W>::T;
  extern __shared__ __align__(16) unsigned char dsmem[];
  SortPhase<W>& SP = *reinterpret_cast<SortPhase<W>*>(dsmem);
  uint32_t* s_wsum = reinterpret_cast<uint32_t*>(dsmem + (sizeof(SortPhase<W>) + 15) / 16 * 16);
  bool msd = false;
  const uint32_t run = plan_phase<W>(a, SP.plan, s_wsum, &msd);
  const int top = 31 - __clz(run), nxt = byte_below(run, top);
  if (msd || nxt < 0) return;
  const K* keys = static_cast<const K*>(a.in_keys);
  const uint64_t stride = (uint64_t)gridDim.x * S1_THREADS;
  for (uint64_t i = (uint64_t)blockIdx.x * S1_THREADS + threadIdx.x; i < a.d; i += stride) {
    const K k = load_key(keys + i);
    atomicAdd(&a.jhist[(key_digit(k, top) << 8) | key_digit(k, nxt)], 1u);
  }
}

// One block: the bins' offsets and the decision (every bin at most BK_CAP).
template <int W>
__global__ void __launch_bounds__(S1_THREADS) step1_jscan_kernel(Step1Args a) {
  extern __shared__ __align__(16) unsigned char dsmem[];
  SortPhase<W>& SP = *reinterpret_cast<SortPhase<W>*>(dsmem);
  uint32_t* s_wsum = reinterpret_cast<uint32_t*>(dsmem + (sizeof(SortPhase<W>) + 15) / 16 * 16);
  bool msd = false;
  const uint32_t run = plan_phase<W>(a, SP.plan, s_wsum, &msd);
  const int top = 31 - __clz(run), nxt = byte_below(run, top);
  if (msd || nxt < 0) return;   // the decision word stays zero
  constexpr uint32_t PER = JOINT_BINS / S1_THREADS;
  const uint32_t b0 = threadIdx.x * PER;
  uint32_t sum = 0, mx = 0;
  for (uint32_t q = 0; q < PER; ++q) {
    const uint32_t c = a.jhist[b0 + q];
    sum += c;
    mx = max(mx, c);
  }
  uint32_t total = 0;
  uint32_t ex = block_excl_scan(sum, s_wsum, &total);
  for (uint32_t q = 0; q < PER; ++q) {
    a.joff[b0 + q] = ex;
    ex += a.jhist[b0 + q];
  }
  const bool fits = !__syncthreads_or(mx > BK_CAP);
  if (threadIdx.x == 0) {
    a.joff[JOINT_BINS] = total;
    a.joff[JOINT_BINS + 1] = fits && (uint64_t)total == a.d ? 1u : 0u;
  }
}

// Every key to its bin (a cursor per bin), in the first ping-pong buffer.
template <int W>
__global__ void __launch_bounds__(S1_THREADS, SORT_BLOCKS_MIN) step1_jscatter_kernel(Step1Args a) {
  using K = typename KeyOf<W>::T;
  extern __shared__ __align__(16) unsigned char dsmem[];
  if (!joint_chosen(a)) return;
  SortPhase<W>& SP = *reinterpret_cast<SortPhase<W>*>(dsmem);
  uint32_t* s_wsum = reinterpret_cast<uint32_t*>(dsmem + (sizeof(SortPhase<W>) + 15) / 16 * 16);
  bool msd = false;
  const uint32_t run = plan_phase<W>(a, SP.plan, s_wsum, &msd);
  const int top = 31 - __clz(run), nxt = byte_below(run, top);
  if (nxt < 0) return;
  const K* keys = static_cast<const K*>(a.in_keys);
  K* dst_k = static_cast<K*>(a.keys[0]);
  uint32_t* dst_v = a.vals[0];
  const uint64_t stride = (uint64_t)gridDim.x * S1_THREADS;
  for (uint64_t i = (uint64_t)blockIdx.x * S1_THREADS + threadIdx.x; i < a.d; i += stride) {
    const K k = load_key(keys + i);
    const uint32_t bin = (key_digit(k, top) << 8) | key_digit(k, nxt);
    const uint64_t pos = (uint64_t)__ldg(a.joff + bin) + atomicAdd(&a.jcur[bin], 1u);
    if (pos < a.d) {
      dst_k[pos] = k;
      dst_v[pos] = (uint32_t)i;
    } else {
      flag_status(a.status, ST_INTERNAL);
    }
  }
}

// Groups of jgroup consecutive bins sorted in place: a group of at most
// BK_CAP keys at once (its bins are in key order, so the group's range is),
// a larger one bin by bin (each at most BK_CAP).
template <int W>
__global__ void __launch_bounds__(S1_THREADS, 2) step1_jgroup_kernel(Step1Args a) {
  using K = typename KeyOf<W>::T;
  extern __shared__ __align__(16) unsigned char dsmem[];
  if (!joint_chosen(a)) return;
  Step1Smem<W>& U = *reinterpret_cast<Step1Smem<W>*>(dsmem);
  K* k0 = static_cast<K*>(a.keys[0]);
  uint32_t* v0 = a.vals[0];
  const uint32_t G = a.jgroup ? a.jgroup : 1u;
  const uint32_t ngroups = (JOINT_BINS + G - 1) / G;
  for (uint32_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const uint32_t b0 = g * G, b1 = min(b0 + G, JOINT_BINS);
    const uint32_t lo = __ldg(a.joff + b0), n = __ldg(a.joff + b1) - lo;
    if (n <= BK_CAP) {
      if (n > 1 && (uint64_t)lo + n <= a.d) bucket_sort<W>(k0, v0, lo, n, true, k0, v0, U.bp.b);
      continue;
    }
    for (uint32_t b = b0; b < b1; ++b) {
      const uint32_t o = __ldg(a.joff + b), nb = __ldg(a.joff + b + 1) - o;
      if (nb > 1 && nb <= BK_CAP && (uint64_t)o + nb <= a.d) bucket_sort<W>(k0, v0, o, nb, true, k0, v0, U.bp.b);
    }
  }
}

// The buckets of the top-byte partition, each sorted in shared memory; and
// where the sorted keys are, for the merge.
template <int W>
__global__ void __launch_bounds__(S1_THREADS, 2) step1_bucket_kernel(Step1Args a) {
  using K = typename KeyOf<W>::T;
  extern __shared__ __align__(16) unsigned char dsmem[];
  Step1Smem<W>& U = *reinterpret_cast<Step1Smem<W>*>(dsmem);
  uint32_t* s_wsum = reinterpret_cast<uint32_t*>(dsmem + (sizeof(Step1Smem<W>) + 15) / 16 * 16);
  bool msd = false;
  const uint32_t run = plan_phase<W>(a, U.sp.plan, s_wsum, &msd);
  K* k0 = static_cast<K*>(a.keys[0]);
  uint32_t* v0 = a.vals[0];
  if (msd) {
    const int top = 31 - __clz(run);
    const uint32_t lower = run & ((1u << top) - 1u);
    const int sub = lower ? 31 - __clz(lower) : -1;
    for (uint32_t b = blockIdx.x; b < 256; b += gridDim.x) {
      const uint32_t off = U.sp.plan[top * 256 + b];
      const uint32_t n = (b < 255 ? U.sp.plan[top * 256 + b + 1] : (uint32_t)a.d) - off;
      if (!bucket_ok(a, off, n)) continue;
      if (sub >= 0) bucket_sort_sub<W>(k0, v0, off, n, true, k0, v0, sub, U.bp.b);
      else bucket_sort<W>(k0, v0, off, n, true, k0, v0, U.bp.b);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const bool last_odd = !msd && !joint_chosen(a) && ((__popc(run) - 1) & 1);
    a.final_slot[0] = last_odd ? a.keys[1] : a.keys[0];
    a.final_slot[1] = last_odd ? a.vals[1] : a.vals[0];
  }
}

// U_D and perm for a merge that follows the sorting launch, or the caller's.
template <int W>
__device__ __forceinline__ void sorted_delta(const Step1Args& a, const typename KeyOf<W>::T** ud, const uint32_t** up) {
  using K = typename KeyOf<W>::T;
  if ((a.phases & S1_SORT) && a.d > 0) {
    *ud = static_cast<const K*>(a.final_slot[0]);
    *up = static_cast<const uint32_t*>(a.final_slot[1]);
  } else {
    *ud = static_cast<const K*>(a.b);
    *up = a.perm;
  }
}

// U_M co-rank of every tile boundary, one warp each.
template <int W>
__global__ void __launch_bounds__(S1_THREADS) step1_cut_kernel(Step1Args a) {
  using K = typename KeyOf<W>::T;
  const K* ud;
  const uint32_t* up;
  sorted_delta<W>(a, &ud, &up);
  constexpr uint32_t T = MergeSmem<W>::T;
  const uint64_t n = a.m + a.d;
  const uint32_t nwt = gridDim.x * S1_WARPS;
  for (uint32_t b = blockIdx.x * S1_WARPS + (threadIdx.x >> 5); b <= a.merge_tiles; b += nwt) {
    const uint64_t k = (uint64_t)b * T < n ? (uint64_t)b * T : n;
    const uint64_t c = corank_warp(static_cast<const K*>(a.a), a.m, ud, a.d, k, false);
    if ((threadIdx.x & 31) == 0) a.cuts[b] = c;
  }
}

// The merge tiles, each block taking the next from a counter.
template <int W>
__global__ void __launch_bounds__(S1_THREADS, merge_blocks_min(W)) step1_merge_kernel(Step1Args a) {
  using K = typename KeyOf<W>::T;
  extern __shared__ __align__(16) unsigned char dsmem[];
  Step1Smem<W>& U = *reinterpret_cast<Step1Smem<W>*>(dsmem);
  const K* ud;
  const uint32_t* up;
  sorted_delta<W>(a, &ud, &up);
  uint32_t* next = a.barriers + S1_BARRIERS - 1;
  for (;;) {
    if (threadIdx.x == 0) U.m.next_tile = atomicAdd(next, 1u);
    __syncthreads();
    const uint32_t t = U.m.next_tile;
    if (t >= a.merge_tiles) break;
    merge_tile<W>(a, t, ud, up, false, true, U.m);
  }
}

// The X_M directory (and its byte table) from the finished X_M.
__global__ void __launch_bounds__(S1_THREADS) step1_dir_kernel(Step1Args a) {
  const uint32_t t = blockIdx.x * S1_THREADS + threadIdx.x, nt = gridDim.x * S1_THREADS;
  const bool use_x8 = a.x8 != nullptr && xdir_x8_pays<false>(a.xm, (uint32_t)a.m, a.dir_entries);
  for (uint32_t b = t; b < a.dir_entries; b += nt)
    a.xdir[b] = xdir_entry<false>(a.xm, (uint32_t)a.m, a.dir_shift, b, use_x8);
  if (use_x8) xdir_x8_fill<false>(a.xm, (uint32_t)a.m, a.dir_shift, a.x8, t, nt);
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

// Kernel attributes (the raised shared-memory limit) and occupancy hold for
// the device that was current when they were set, so they are kept per
// device.
constexpr int kLaunchDevices = 64;
struct Launch {
  std::mutex mu;
  bool ready[kLaunchDevices][3] = {};
  int per_sm[kLaunchDevices][3] = {};
  int merge_per_sm[kLaunchDevices][3] = {};   // step1_merge_kernel<W>
  int sort_per_sm[kLaunchDevices][3] = {};    // step1_hist / pass / msd_kernel<W>
};
Launch& launch_state() {
  static Launch L;
  return L;
}

cudaError_t current_device(int* dev) {
  cudaError_t e = cudaGetDevice(dev);
  if (e != cudaSuccess) return e;
  return *dev >= 0 && *dev < kLaunchDevices ? cudaSuccess : cudaErrorInvalidDevice;
}

// Blocks per SM of step1_kernel<W> on the current device (its attributes set
// on first use there), or 0 with the error in *err.
template <int W>
int prepare_w(cudaError_t* err) {
  const int wi = W == 4 ? 0 : (W == 8 ? 1 : 2);
  int dev = 0;
  *err = current_device(&dev);
  if (*err != cudaSuccess) return 0;
  Launch& L = launch_state();
  std::lock_guard<std::mutex> g(L.mu);
  if (L.ready[dev][wi]) return L.per_sm[dev][wi];
  const size_t smem = step1_smem_bytes<W>();
  cudaError_t e = cudaFuncSetAttribute(step1_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step1_bucket_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step1_jgroup_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  for (const void* fn : {(const void*)step1_hist_kernel<W>, (const void*)step1_pass_kernel<W>,
                         (const void*)step1_msd_kernel<W>, (const void*)step1_jhist_kernel<W>,
                         (const void*)step1_jscan_kernel<W>, (const void*)step1_jscatter_kernel<W>})
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem_bytes<W>());
  int sort_per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sort_per_sm, step1_pass_kernel<W>, S1_THREADS,
                                                      sort_smem_bytes<W>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step1_merge_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)merge_smem_bytes<W>());
  int merge_per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&merge_per_sm, step1_merge_kernel<W>, S1_THREADS,
                                                      merge_smem_bytes<W>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step1_small_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)small_smem_bytes<W>());
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step1_kernel<W>, S1_THREADS, smem);
  *err = e;
  if (e != cudaSuccess) return 0;
  L.per_sm[dev][wi] = per_sm;
  L.merge_per_sm[dev][wi] = merge_per_sm > 0 ? merge_per_sm : 1;
  L.sort_per_sm[dev][wi] = sort_per_sm > 0 ? sort_per_sm : 1;
  L.ready[dev][wi] = true;
  return per_sm;
}


template <int W>
cudaError_t launch_step1_w(Step1Args a, cudaStream_t s, uint32_t sm_count, uint64_t* launches) {
  const size_t smem = step1_smem_bytes<W>();
  cudaError_t pe = cudaSuccess;
  const int per_sm = prepare_w<W>(&pe);
  if (pe != cudaSuccess) return pe;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // small dictionaries: one block (not with the wait-test setting, which
  // needs the tiled kernel's look-back)
  const bool merge_only_dir = !(a.phases & S1_DIR) || a.dir_entries == 0;
  if ((a.phases & S1_MERGE) && merge_only_dir && (a.d == 0 || (a.phases & S1_SORT)) && a.m <= SM_MAX_M &&
      a.d <= SM_MAX_D && a.m + a.d > 0 && a.test_withhold == 0) {
    step1_small_kernel<W><<<1, S1_THREADS, small_smem_bytes<W>(), s>>>(a);
    ++*launches;
    return cudaGetLastError();
  }
  const uint64_t full = (uint64_t)per_sm * sm_count;
  uint64_t cap = full;
  if (a.grid_cap && a.grid_cap < cap) cap = a.grid_cap;
  // a capped grid with fewer blocks than the merge has tiles, or than a
  // quarter of the sort's: the split form (a split sort implies a split merge,
  // which finds the sorted keys where the sort left them)
  const bool capped = cap < full && a.final_slot != nullptr;
  // a sort of more than four times as many tiles as the grid holds at once
  // takes the split form too, whose histogram, pass and partition kernels
  // fit three blocks to an SM (below that the split form's extra launches
  // cost more than they save)
  const bool split_sort = a.final_slot != nullptr && (a.phases & S1_SORT) && a.d > BK_SINGLE &&
                          ((capped && a.sort_tiles > 4 * cap) || a.sort_tiles > 4 * full);
  // a merge of more tiles than the cooperative grid holds at once also
  // takes the split form, uncapped: its merge kernel's blocks need no
  // co-residency and fit more to an SM (16-bit per-tile arrays, fewer
  // registers), so more latency-bound tiles are in flight
  const bool multiwave = a.final_slot != nullptr && a.merge_tiles > full;
  const bool split = (a.phases & S1_MERGE) && a.m + a.d > 0 && a.cuts != nullptr &&
                     ((capped && a.merge_tiles > cap) || multiwave || split_sort);
  Step1Args c = a;
  if (split) c.phases &= S1_SORT;
  if (split_sort) c.phases = 0;
  cudaError_t e = cudaSuccess;
  if (c.phases && !(c.phases == S1_SORT && a.d == 0)) {
    // all blocks resident at once (cooperative launch); no more blocks than
    // the largest phase has tiles
    uint64_t want = 1;
    if ((c.phases & S1_SORT) && c.d > BK_SINGLE) want = std::max<uint64_t>(want, std::max<uint64_t>(c.sort_tiles, 256));
    if (c.phases & S1_MERGE) want = std::max<uint64_t>(want, c.merge_tiles);
    if (c.phases & S1_DIR) want = std::max<uint64_t>(want, (c.dir_entries + S1_THREADS - 1) / S1_THREADS);
    const uint32_t grid = (uint32_t)std::min(want, cap);
    c.hist_blocks = (uint32_t)std::min<uint64_t>(
        grid, std::max<uint64_t>(1, (c.d + S1_THREADS * HI_ITEMS - 1) / (S1_THREADS * HI_ITEMS)));

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
    e = cudaLaunchKernelEx(&cfg, step1_kernel<W>, c);
    ++*launches;
  }
  if (e != cudaSuccess) return e;
  int dev = 0;
  if (current_device(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
  const int wi = W == 4 ? 0 : (W == 8 ? 1 : 2);
  if (split_sort) {
    const uint64_t sort_full = std::max<uint64_t>(1, (uint64_t)launch_state().sort_per_sm[dev][wi] * sm_count);
    const size_t ssm = sort_smem_bytes<W>();
    Step1Args h = a;
    h.hist_blocks =
        (uint32_t)std::min<uint64_t>(sort_full, (a.d + S1_THREADS * HI_ITEMS - 1) / (S1_THREADS * HI_ITEMS));
    step1_hist_kernel<W><<<h.hist_blocks, S1_THREADS, ssm, s>>>(h);
    ++*launches;
    const uint32_t sort_grid = (uint32_t)std::min<uint64_t>(sort_full, a.sort_tiles);
    if (a.jhist) {
      // the two-level partition; when the plan or its bins rule it out, its
      // kernels return at once and the LSD passes below run
      Step1Args j = a;
      const uint64_t per_bin = std::max<uint64_t>(1, a.d / JOINT_BINS);
      j.jgroup = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(JOINT_BINS, (BK_CAP / 2) / per_bin));
      const uint32_t ngroups = (JOINT_BINS + j.jgroup - 1) / j.jgroup;
      step1_jhist_kernel<W><<<sort_grid, S1_THREADS, ssm, s>>>(j);
      step1_jscan_kernel<W><<<1, S1_THREADS, ssm, s>>>(j);
      step1_jscatter_kernel<W><<<sort_grid, S1_THREADS, ssm, s>>>(j);
      step1_jgroup_kernel<W><<<(uint32_t)std::min<uint64_t>(full, ngroups), S1_THREADS, smem, s>>>(j);
      *launches += 4;
    }
    for (int p = 0; p < W; ++p) {
      step1_pass_kernel<W><<<sort_grid, S1_THREADS, ssm, s>>>(a, p);
      ++*launches;
    }
    step1_msd_kernel<W><<<sort_grid, S1_THREADS, ssm, s>>>(a);
    step1_bucket_kernel<W><<<(uint32_t)std::min<uint64_t>(full, 256), S1_THREADS, smem, s>>>(a);
    *launches += 2;
  }
  if (!split) return cudaGetLastError();
  const uint32_t cut_blocks = (uint32_t)std::min<uint64_t>(full, (a.merge_tiles + S1_WARPS) / S1_WARPS);
  step1_cut_kernel<W><<<cut_blocks, S1_THREADS, 0, s>>>(a);
  ++*launches;
  const uint64_t merge_full = (uint64_t)launch_state().merge_per_sm[dev][wi] * sm_count;
  step1_merge_kernel<W><<<(uint32_t)std::min<uint64_t>(std::max<uint64_t>(merge_full, 1), a.merge_tiles),
                          S1_THREADS, merge_smem_bytes<W>(), s>>>(a);
  ++*launches;
  if ((a.phases & S1_DIR) && a.dir_entries > 0) {
    const uint64_t work = std::max<uint64_t>(a.dir_entries, a.x8 ? (a.m + 3) / 4 : 0);
    step1_dir_kernel<<<(uint32_t)std::min<uint64_t>(4096, (work + S1_THREADS - 1) / S1_THREADS), S1_THREADS, 0, s>>>(a);
    ++*launches;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t step1_prepare() {
  cudaError_t e = cudaSuccess;
  prepare_w<4>(&e);
  if (e == cudaSuccess) prepare_w<8>(&e);
  if (e == cudaSuccess) prepare_w<16>(&e);
  return e;
}

uint32_t step1_capacity(uint32_t w, uint32_t sm_count) {
  cudaError_t e = cudaSuccess;
  const int per_sm = w == 4 ? prepare_w<4>(&e) : (w == 8 ? prepare_w<8>(&e) : prepare_w<16>(&e));
  return e == cudaSuccess ? (uint32_t)per_sm * sm_count : 0u;
}

uint32_t sort_tiles(uint64_t d) { return (uint32_t)((d + RS_TILE - 1) / RS_TILE); }
uint32_t merge_tiles(uint64_t n, uint32_t w) { return (uint32_t)((n + mg_tile(w) - 1) / mg_tile(w)); }

uint64_t step1_zeroed_words(uint32_t w, uint64_t n_merge, uint64_t d) {
  // merge look-back (64-bit words), barrier counters, digit histograms,
  // sort look-back
  return 2ull * merge_tiles(n_merge, w) + S1_BARRIERS + (d ? (uint64_t)w * 256 + (uint64_t)w * sort_tiles(d) * 256 : 0) +
         (d > JOINT_MIN_KEYS ? 3ull * JOINT_BINS + 2 : 0);
}

void step1_layout(uint32_t w, uint64_t n_merge, uint64_t d, uint32_t* zero, Step1Args* a) {
  const uint32_t mt = merge_tiles(n_merge, w);
  a->merge_lb = reinterpret_cast<uint64_t*>(zero);
  a->merge_tiles = mt;
  a->barriers = zero + 2ull * mt;
  uint32_t* z = a->barriers + S1_BARRIERS;
  a->hist = z;
  a->sort_tiles = sort_tiles(d);
  a->sort_lb = z + (uint64_t)w * 256;
  a->jhist = a->jcur = a->joff = nullptr;
  if (d > JOINT_MIN_KEYS) {
    uint32_t* j = a->sort_lb + (uint64_t)w * sort_tiles(d) * 256;
    a->jhist = j;
    a->jcur = j + JOINT_BINS;
    a->joff = j + 2 * JOINT_BINS;   // JOINT_BINS + 1 offsets, then the decision word
  }
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
constexpr uint32_t kNoAllocTiles = (DM_NOALLOC_MAX_ENTRIES + dm::MG_TILE_MIN - 1) / dm::MG_TILE_MIN;
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
  if (m > DM_NOALLOC_MAX_ENTRIES || d > DM_NOALLOC_MAX_ENTRIES - m) return DM_EINVAL;
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
