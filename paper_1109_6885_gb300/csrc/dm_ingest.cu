// Delta ingest (Section 4, Figure 5): tuples appended to a column's delta
// partition in arrival order, turned into the delta form the merge reads:
// D_dict, each distinct value once in order of first arrival, and one code
// per tuple (the position of its value in D_dict).  The paper keeps the
// distinct values in a CSB+ tree with the tuple ids of each value; the
// insertion-order dictionary plus codes carries the same information.
//
// GPU form:
//   1. a hash table of row indices: each slot holds the smallest row of one
//      value (the row is the key's representative, so any width needs only
//      32-bit atomics: a row reads the slot, claims it with a CAS if it is
//      empty, or lowers its row with atomicMin if its representative
//      equals the value and is a later row);
//      open addressing, linear probing, load at most one half;
//      a row's slot is final once it claims it or finds its value there,
//      so the insert also records each row's slot;
//   2. a row is a first arrival when its slot holds it; rows are cut into
//      tiles of 1024 and each tile counts its first arrivals;
//   3. one block scans the tile counts (the codes of each tile's first
//      arrivals start at its scan value) and publishes |D_dict|;
//   4. each tile numbers its first arrivals in row order, writes them to
//      D_dict and the code to their slot;
//   5. every row reads its code from its slot.
// Consecutive threads take consecutive rows, so the per-row loads and
// stores are coalesced.  Every probe loop ends after at most the table's
// size; nothing waits.  A row left without a slot (impossible at load at
// most one half) is flagged as an internal error.
#include <stdint.h>

#include "../../include/dmerge.h"
#include "dm_common.cuh"
#include "dm_ctx.h"

namespace dm {

namespace {

constexpr uint32_t IG_THREADS = 256;
constexpr uint32_t IG_PER_THREAD = 4;
constexpr uint32_t IG_TILE = IG_THREADS * IG_PER_THREAD;   // rows per tile
constexpr uint32_t IG_EMPTY = 0xFFFFFFFFu;
constexpr uint64_t IG_MAX_ROWS = 1ull << 30;
constexpr uint32_t IG_CACHE = 2048;                      // block cache entries (16 KiB)
constexpr uint64_t IG_CACHE_EMPTY = ~0ull;

// Table slots for n rows: a power of two of at least 2n (and 64).
uint64_t table_slots(uint64_t n) {
  uint64_t c = 64;
  while (c < 2 * n) c <<= 1;
  return c;
}

// MurmurHash3's 32- and 64-bit finalisers (public domain mixing steps).
__device__ __forceinline__ uint32_t mix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
__device__ __forceinline__ uint64_t mix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}
__device__ __forceinline__ uint32_t hash_key(uint32_t v) { return mix32(v); }
__device__ __forceinline__ uint32_t hash_key(uint64_t v) { return (uint32_t)mix64(v); }
__device__ __forceinline__ uint32_t hash_key(const u128& v) { return (uint32_t)mix64(v.hi ^ mix64(v.lo)); }

struct IngestArgs {
  const void* values;
  uint64_t n;
  void* dict_out;
  uint32_t* codes;
  uint64_t* d_out;
  uint32_t* table;       // [slots] smallest row of the slot's value, or IG_EMPTY
  uint32_t* slot_code;   // [slots] code of the slot's value
  uint32_t* slot_of;     // [n] each row's slot
  uint32_t* tile_first;  // [tiles] first arrivals per tile, then their exclusive scan
  uint64_t slots;
  uint32_t tiles;
  uint32_t* status;
};

// Lanes of the warp holding the same key as this lane.
__device__ __forceinline__ uint32_t match_key(uint32_t v) { return __match_any_sync(0xFFFFFFFFu, v); }
__device__ __forceinline__ uint32_t match_key(uint64_t v) {
  return __match_any_sync(0xFFFFFFFFu, (unsigned long long)v);
}
__device__ __forceinline__ uint32_t match_key(const u128& v) {
  return __match_any_sync(0xFFFFFFFFu, (unsigned long long)v.hi) &
         __match_any_sync(0xFFFFFFFFu, (unsigned long long)v.lo);
}

// Block-local cache entries, (row << 32) | slot, read and written whole.
__device__ __forceinline__ uint64_t cache_ld(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.cta.shared.b64 %0, [%1];" : "=l"(v) : "r"((uint32_t)__cvta_generic_to_shared(p)));
  return v;
}
__device__ __forceinline__ void cache_st(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.cta.shared.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(p)), "l"(v)
               : "memory");
}

// One block-stride round of 256 rows per block.  The lanes of a warp that
// hold one value elect the lowest (its smallest row); only it looks the value
// up, and the others take its slot.  The leader looks first in the block's
// cache of recent (row, slot) pairs: an entry is right for the value when the
// value of its row equals it (a slot keeps its value for good), and the
// slot's row is then at most the entry's row (rows only decrease), so
// atomicMin is needed only for a smaller row.  A frequent value thus reaches
// the table about once per block instead of once per warp.  Otherwise it
// probes the table, reading each slot before any atomic.
template <int W>
__global__ void __launch_bounds__(IG_THREADS) ingest_insert_kernel(IngestArgs a) {
  using K = typename KeyOf<W>::T;
  __shared__ uint64_t cache[IG_CACHE];
  for (uint32_t i = threadIdx.x; i < IG_CACHE; i += IG_THREADS) cache[i] = IG_CACHE_EMPTY;
  __syncthreads();
  const K* vals = static_cast<const K*>(a.values);
  const uint64_t mask = a.slots - 1;
  const uint32_t lane = threadIdx.x & 31;
  for (uint64_t base = (uint64_t)blockIdx.x * IG_THREADS; base < a.n; base += (uint64_t)gridDim.x * IG_THREADS) {
    const uint64_t r = base + threadIdx.x;
    const bool valid = r < a.n;
    const K v = load_key(vals + (valid ? r : base));
    const uint32_t group = match_key(v) & __ballot_sync(0xFFFFFFFFu, valid);
    const uint32_t leader = group ? (uint32_t)(__ffs(group) - 1) : lane;
    uint32_t slot = IG_EMPTY;
    if (valid && leader == lane) {
      const uint32_t h = hash_key(v);
      uint64_t* ce = cache + ((h >> 11) & (IG_CACHE - 1));
      const uint64_t e = cache_ld(ce);
      if (e != IG_CACHE_EMPTY && key_eq(load_key(vals + (uint32_t)(e >> 32)), v)) {
        slot = (uint32_t)e;
        if ((uint32_t)r < (uint32_t)(e >> 32)) atomicMin(a.table + slot, (uint32_t)r);
      } else {
        uint64_t s = h & mask;
        for (uint64_t p = 0; p < a.slots; ++p, s = (s + 1) & mask) {
          uint32_t cur = __ldcg(a.table + s);
          if (cur == IG_EMPTY) {
            cur = atomicCAS(a.table + s, IG_EMPTY, (uint32_t)r);
            if (cur == IG_EMPTY) {   // claimed
              slot = (uint32_t)s;
              cache_st(ce, ((uint64_t)r << 32) | s);
              break;
            }
          }
          if (key_eq(load_key(vals + cur), v)) {
            if ((uint32_t)r < cur) atomicMin(a.table + s, (uint32_t)r);
            slot = (uint32_t)s;
            cache_st(ce, ((uint64_t)min((uint32_t)r, cur) << 32) | s);
            break;
          }
        }
      }
    }
    slot = __shfl_sync(0xFFFFFFFFu, slot, leader);
    if (valid) {
      if (slot == IG_EMPTY) flag_status(a.status, ST_INTERNAL);   // cannot happen at load <= 1/2
      a.slot_of[r] = slot;
    }
  }
}

// Row q * IG_THREADS + threadIdx.x of tile t (consecutive threads, consecutive rows).
__device__ __forceinline__ uint64_t tile_row(uint32_t t, uint32_t q) {
  return (uint64_t)t * IG_TILE + (uint64_t)q * IG_THREADS + threadIdx.x;
}

// Whether row r is the first arrival of its value (its slot holds r).
__device__ __forceinline__ bool first_arrival(const IngestArgs& a, uint64_t r) {
  if (r >= a.n) return false;
  const uint32_t s = a.slot_of[r];
  return s != IG_EMPTY && __ldg(a.table + s) == (uint32_t)r;
}

// Each tile's count of first arrivals.
__global__ void __launch_bounds__(IG_THREADS) ingest_mark_kernel(IngestArgs a) {
  __shared__ uint32_t wsum[IG_THREADS / 32];
  for (uint32_t t = blockIdx.x; t < a.tiles; t += gridDim.x) {
    uint32_t cnt = 0;
#pragma unroll
    for (uint32_t q = 0; q < IG_PER_THREAD; ++q) cnt += first_arrival(a, tile_row(t, q)) ? 1u : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t tot = 0;
      for (uint32_t w = 0; w < IG_THREADS / 32; ++w) tot += wsum[w];
      a.tile_first[t] = tot;
    }
    __syncthreads();
  }
}

// Exclusive scan of the tile counts by one block; |D_dict| to *d_out.
__global__ void __launch_bounds__(IG_THREADS) ingest_scan_kernel(IngestArgs a) {
  __shared__ uint32_t wsum[IG_THREADS / 32];
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < a.tiles; base += IG_THREADS) {
    const uint32_t t = base + threadIdx.x;
    const uint32_t v = t < a.tiles ? a.tile_first[t] : 0u;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if ((threadIdx.x & 31) >= (uint32_t)o) inc += y;
    }
    if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = inc;
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (uint32_t w = 0; w < IG_THREADS / 32; ++w) {
      if (w < (threadIdx.x >> 5)) before += wsum[w];
      total += wsum[w];
    }
    const uint64_t c = carry;
    if (t < a.tiles) a.tile_first[t] = (uint32_t)(c + before + inc - v);
    __syncthreads();
    if (threadIdx.x == 0) carry = c + total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *a.d_out = carry;
}

// First arrivals numbered in row order: D_dict and their slots' codes.  A
// tile's rows go in IG_PER_THREAD rounds of IG_THREADS consecutive rows; the
// first arrivals before a row are those of earlier rounds, of earlier warps
// in its round, and of lower lanes in its warp (one ballot each).
template <int W>
__global__ void __launch_bounds__(IG_THREADS) ingest_emit_kernel(IngestArgs a) {
  using K = typename KeyOf<W>::T;
  constexpr uint32_t NW = IG_THREADS / 32;
  __shared__ uint32_t wcnt[IG_PER_THREAD * NW];
  const K* vals = static_cast<const K*>(a.values);
  K* dict = static_cast<K*>(a.dict_out);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t t = blockIdx.x; t < a.tiles; t += gridDim.x) {
    uint32_t ball[IG_PER_THREAD];
#pragma unroll
    for (uint32_t q = 0; q < IG_PER_THREAD; ++q) {
      ball[q] = __ballot_sync(0xFFFFFFFFu, first_arrival(a, tile_row(t, q)));
      if (lane == 0) wcnt[q * NW + warp] = __popc(ball[q]);
    }
    __syncthreads();
    uint32_t acc = a.tile_first[t], k = 0;
#pragma unroll
    for (uint32_t q = 0; q < IG_PER_THREAD; ++q) {
      for (; k < q * NW + warp; ++k) acc += wcnt[k];
      if ((ball[q] >> lane) & 1u) {
        const uint32_t code = acc + __popc(ball[q] & lanemask_lt());
        const uint64_t r = tile_row(t, q);
        if (code < a.n) {
          dict[code] = load_key(vals + r);
          a.slot_code[a.slot_of[r]] = code;
        } else {
          flag_status(a.status, ST_INTERNAL);
        }
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(IG_THREADS) ingest_codes_kernel(IngestArgs a) {
  for (uint64_t r = (uint64_t)blockIdx.x * IG_THREADS + threadIdx.x; r < a.n; r += (uint64_t)gridDim.x * IG_THREADS) {
    const uint32_t s = a.slot_of[r];
    a.codes[r] = s != IG_EMPTY ? __ldg(a.slot_code + s) : 0u;
  }
}

template <int W>
cudaError_t launch_ingest(const IngestArgs& a, cudaStream_t s, uint32_t sm_count, uint64_t* launches) {
  const uint64_t row_blocks = (a.n + IG_THREADS - 1) / IG_THREADS;
  const uint32_t grid = (uint32_t)(row_blocks < (uint64_t)sm_count * 8 ? row_blocks : (uint64_t)sm_count * 8);
  const uint32_t tgrid = a.tiles < sm_count * 8 ? a.tiles : sm_count * 8;
  ingest_insert_kernel<W><<<grid, IG_THREADS, 0, s>>>(a);
  ingest_mark_kernel<<<tgrid, IG_THREADS, 0, s>>>(a);
  ingest_scan_kernel<<<1, IG_THREADS, 0, s>>>(a);
  ingest_emit_kernel<W><<<tgrid, IG_THREADS, 0, s>>>(a);
  ingest_codes_kernel<<<grid, IG_THREADS, 0, s>>>(a);
  *launches += 5;
  return cudaGetLastError();
}

size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

}  // namespace dm

extern "C" size_t dm_ingest_scratch_bytes(uint32_t value_bytes, uint64_t n) {
  (void)value_bytes;
  const uint64_t slots = dm::table_slots(n);
  const uint64_t tiles = (n + dm::IG_TILE - 1) / dm::IG_TILE;
  return dm::round256(slots * 4) * 2 + dm::round256(n * 4) + dm::round256(tiles * 4 + 4);
}

namespace dm {
namespace {

// Argument checks of one column's ingest (no launch).
dm_status ingest_check(uint32_t w, const void* values, uint64_t n, const void* dict_out, const uint32_t* codes_out,
                       const uint64_t* d_dict_len) {
  if ((w != 4 && w != 8 && w != 16) || !d_dict_len || n > IG_MAX_ROWS) return DM_EINVAL;
  if (n && (!values || !dict_out || !codes_out)) return DM_EINVAL;
  if (n && ((reinterpret_cast<uintptr_t>(values) | reinterpret_cast<uintptr_t>(dict_out)) & (w - 1))) return DM_EINVAL;
  return DM_OK;
}

// One column's ingest on stream s with its scratch at `base`.
dm_status ingest_column(dm_ctx* ctx, uint32_t w, const void* values, uint64_t n, void* dict_out, uint32_t* codes_out,
                        uint64_t* d_dict_len, cudaStream_t s, void* base) {
  if (n == 0) return cudaMemsetAsync(d_dict_len, 0, 8, s) == cudaSuccess ? DM_OK : DM_ECUDA;
  IngestArgs a{};
  a.values = values;
  a.n = n;
  a.dict_out = dict_out;
  a.codes = codes_out;
  a.d_out = d_dict_len;
  a.slots = table_slots(n);
  a.tiles = (uint32_t)((n + IG_TILE - 1) / IG_TILE);
  char* p = static_cast<char*>(base);
  a.table = reinterpret_cast<uint32_t*>(p);
  p += round256(a.slots * 4);
  a.slot_code = reinterpret_cast<uint32_t*>(p);
  p += round256(a.slots * 4);
  a.slot_of = reinterpret_cast<uint32_t*>(p);
  p += round256(n * 4);
  a.tile_first = reinterpret_cast<uint32_t*>(p);
  a.status = ctx->status;
  if (cudaMemsetAsync(a.table, 0xFF, a.slots * 4, s) != cudaSuccess) return DM_ECUDA;
  cudaError_t e;
  switch (w) {
    case 4: e = launch_ingest<4>(a, s, ctx->sm_count, &ctx->launches); break;
    case 8: e = launch_ingest<8>(a, s, ctx->sm_count, &ctx->launches); break;
    default: e = launch_ingest<16>(a, s, ctx->sm_count, &ctx->launches); break;
  }
  if (e != cudaSuccess) ctx->last_error = e;
  return e == cudaSuccess ? DM_OK : DM_ECUDA;
}

}  // namespace
}  // namespace dm

extern "C" dm_status dm_ingest_delta(dm_ctx* ctx, uint32_t value_bytes, const void* values, uint64_t n,
                                     void* dict_out, uint32_t* codes_out, uint64_t* d_dict_len, void* stream) {
  if (!ctx) return DM_EINVAL;
  const dm_status st = dm::ingest_check(value_bytes, values, n, dict_out, codes_out, d_dict_len);
  if (st != DM_OK) return st;
  if (dm_ingest_scratch_bytes(value_bytes, n) > ctx->arena_bytes) return DM_ENOMEM;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DM_ECUDA;
  return dm::ingest_column(ctx, value_bytes, values, n, dict_out, codes_out, d_dict_len,
                           static_cast<cudaStream_t>(stream), ctx->arena);
}

// Branches of a table ingest: the context's side streams (as many as a table
// merge uses), each with its own scratch region.
static uint32_t ingest_branches(const dm_ctx* ctx, uint32_t ncols) {
  uint32_t b = ctx->tuning.table_branches ? ctx->tuning.table_branches : dm_ctx::kTableBranches;
  if (b > dm_ctx::kTableStreams) b = dm_ctx::kTableStreams;
  return ncols < b ? (ncols ? ncols : 1) : b;
}

extern "C" size_t dm_ingest_table_scratch_bytes(const dm_ingest_column* cols, uint32_t ncols, uint64_t n) {
  (void)cols;
  const size_t region = (dm_ingest_scratch_bytes(4, n) + 255) & ~(size_t)255;
  return region * (ncols < dm_ctx::kTableStreams ? (ncols ? ncols : 1) : dm_ctx::kTableStreams);
}

extern "C" dm_status dm_ingest_table(dm_ctx* ctx, const dm_ingest_column* cols, uint32_t ncols, uint64_t n,
                                     void* stream) {
  if (!ctx || (ncols && !cols)) return DM_EINVAL;
  for (uint32_t c = 0; c < ncols; ++c) {
    const dm_status st = dm::ingest_check(cols[c].value_bytes, cols[c].values, n, cols[c].dict_out,
                                          cols[c].codes_out, cols[c].d_dict_len);
    if (st != DM_OK) return st;
  }
  if (ncols == 0) return DM_OK;
  const uint32_t S = ingest_branches(ctx, ncols);
  const size_t region = (dm_ingest_scratch_bytes(4, n) + 255) & ~(size_t)255;
  if (region * S > ctx->arena_bytes) return DM_ENOMEM;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DM_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // columns round-robin over the side streams, which start after earlier
  // work on s and which s waits for at the end
  if (cudaEventRecord(ctx->fork, s) != cudaSuccess) return DM_ECUDA;
  for (uint32_t i = 0; i < S; ++i)
    if (cudaStreamWaitEvent(ctx->side[i], ctx->fork, 0) != cudaSuccess) return DM_ECUDA;
  dm_status st = DM_OK;
  for (uint32_t c = 0; c < ncols && st == DM_OK; ++c) {
    const uint32_t i = c % S;
    st = dm::ingest_column(ctx, cols[c].value_bytes, cols[c].values, n, cols[c].dict_out, cols[c].codes_out,
                           cols[c].d_dict_len, ctx->side[i], static_cast<char*>(ctx->arena) + (size_t)i * region);
  }
  // join every branch whatever happened, so that no work is left unordered
  for (uint32_t i = 0; i < S; ++i) {
    if (cudaEventRecord(ctx->join[i], ctx->side[i]) != cudaSuccess ||
        cudaStreamWaitEvent(s, ctx->join[i], 0) != cudaSuccess)
      st = DM_ECUDA;
  }
  return st;
}
