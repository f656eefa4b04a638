// Merge server: table merges requested over time, run with continuous
// batching on one GPU.
//
// The paper runs the merge when the delta grows past a fraction of the main
// (Section 4), on a copy of the table, committing the result atomically at
// the end while a second delta takes new inserts (Section 3); scheduling is
// left open there.  Here registered tables stay resident in device memory;
// requests are admitted by the scheduler core (dm_sched.h) into slots —
// each a context with its own stream — when a slot, the table and a
// region of the scratch pool (their HBM footprint) are free.  A host thread
// watches each slot's completion event, commits the table's new version,
// frees the region and admits more, so requests that arrive while others
// run join as soon as resources allow and overlap them on the device.
//
// Online tables are owned by the server: two copies of the main partition
// (a merge reads the committed one and writes the other, and its commit
// swaps them) and two delta partitions of raw inserted values (inserts go
// to the active one; a merge freezes it and the other takes the inserts
// that arrive while it runs).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dm_common.cuh"
#include "dm_ctx.h"
#include "dm_internal.h"
#include "dm_sched.h"

// Branches of each slot's batched table merges: slots already run side by
// side, so fewer than a table merged alone.
constexpr uint32_t kSlotBranches = 4;

namespace {

// One column of an online table: its two main copies and two deltas.
struct OnlineColumn {
  uint32_t w = 0;
  uint64_t dict_cap = 0;          // keys per main dictionary copy
  void* dict[2] = {nullptr, nullptr};
  void* packed[2] = {nullptr, nullptr};
  void* delta[2] = {nullptr, nullptr};   // delta_capacity keys each
  uint64_t u = 0;                 // |U_M| of the committed main
  uint32_t bits = 0;              // its E_C
};

}  // namespace

struct dm_server {
  int device = 0;
  dm_server_config cfg{};
  uint32_t merge_flags = 0;       // cfg.flags without the server's own bits
  bool digest = false;
  void* pool = nullptr;
  dm::Scheduler* sched = nullptr;
  // Streams of every priority the device offers, per slot: a table merge is
  // launched at a priority set by its size (fewer tuples: higher), so that
  // small merges admitted next to a large one are not queued behind its
  // kernels at block granularity.
  static constexpr int kLevels = 8;
  int levels = 1, greatest = 0;
  struct Slot {
    dm_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;            // the stream of the merge in flight
    cudaStream_t by_level[kLevels] = {};      // [0]: highest priority
    cudaEvent_t done = nullptr;
    unsigned long long* d_digest = nullptr;   // the merge's checksum (device)
    uint64_t req = 0;
    bool busy = false;
  };
  std::vector<Slot> slots;
  dm_tune_cache tune_cache;   // shared by every slot's context
  struct Table {
    std::vector<dm_column_in> in;
    std::vector<dm_column_out> out;
    uint64_t tuples = 0;
    // online tables
    bool online = false;
    uint32_t cur = 0;                    // main copy of the committed version
    uint64_t delta_cap = 0;
    std::vector<OnlineColumn> cols;
    uint32_t* iota = nullptr;            // delta codes 0..delta_cap-1
    uint64_t* scalars = nullptr;         // [ncols][2] device: |U'|, E'_C of the merge in flight
    std::vector<uint64_t> host_scalars;
    cudaEvent_t inserted[2] = {nullptr, nullptr};   // the last insert's copies into each delta
    std::vector<void*> owned;            // device allocations
  };
  std::unordered_map<uint32_t, Table> tables;
  cudaStream_t insert_stream = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

  uint64_t now() const {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0)
        .count();
  }
};

namespace {

// Priority level of a merge of `tuples` tuples: 0 (highest) below 2M tuples,
// one level lower per factor of 8 above, the lowest from there on.
int level_of(const dm_server* S, uint64_t tuples) {
  int lvl = 0;
  for (uint64_t v = tuples; v >= 2000000 && lvl < S->levels - 1; v /= 8) ++lvl;
  return lvl;
}

// ------------------------------------------------------------ output checksum
// An order-independent sum of one mixed term per 32-bit word of a merge's
// outputs: splitmix64's output function (Steele et al.) of the word's
// position tag and value.  Any change of a word or of |U'| / E'_C changes the
// sum unless two terms cancel exactly.
__device__ __forceinline__ uint64_t dg_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t dg_term(uint32_t col, uint32_t section, uint64_t i, uint32_t v) {
  const uint64_t tag = ((uint64_t)col << 40) | ((uint64_t)section << 38) | i;
  return dg_mix(tag * 0x9e3779b97f4a7c15ull + dg_mix((uint64_t)v + 0x632be59bd9b4e019ull));
}

// One column's checksum: |U'| and E'_C, the |U'| keys of U', and the packed
// vector of n_rows codes at E'_C bits (lengths from the device scalars,
// clamped to the buffers' capacities u_cap keys and b_cap bits, which a
// merge that failed may have left them above).
__global__ void digest_kernel(const uint32_t* dict, const uint64_t* d_u, uint32_t w, const uint32_t* packed,
                              const uint32_t* d_bits, uint64_t n_rows, uint32_t col, uint64_t u_cap, uint32_t b_cap,
                              unsigned long long* out) {
  const uint64_t u = min(*d_u, u_cap);
  const uint32_t b = min(*d_bits, b_cap);
  const uint64_t dict_words = u * (w / 4);
  const uint64_t packed_words = ((n_rows * b + 127) / 128) * 4;
  uint64_t acc = 0;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
  if (t == 0) {
    acc += dg_term(col, 2, 0, (uint32_t)u) + dg_term(col, 2, 1, (uint32_t)(u >> 32)) + dg_term(col, 2, 2, b);
  }
  for (uint64_t i = t; i < dict_words; i += nt) acc += dg_term(col, 0, i, __ldg(dict + i));
  for (uint64_t i = t; i < packed_words; i += nt) acc += dg_term(col, 1, i, __ldg(packed + i));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, (unsigned long long)acc);
}

cudaError_t launch_column_digest(const dm_column_in& in, const dm_column_out& out, uint32_t col,
                                 unsigned long long* d, cudaStream_t s) {
  const uint64_t n = in.main_rows + in.delta_rows;
  const uint64_t words =
      (in.main_dict_len + in.delta_dict_len) * (in.value_bytes / 4) + dm_packed_bytes(n, dm_max_bits(&in)) / 4;
  const uint32_t blocks = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(1024, (words + 2047) / 2048));
  digest_kernel<<<blocks, 256, 0, s>>>(static_cast<const uint32_t*>(out.new_dict), out.d_new_dict_len,
                                       in.value_bytes, static_cast<const uint32_t*>(out.new_packed), out.d_new_bits,
                                       n, col, in.main_dict_len + in.delta_dict_len, dm_max_bits(&in), d);
  return cudaGetLastError();
}

cudaError_t launch_digest(const std::vector<dm_column_in>& in, const std::vector<dm_column_out>& out,
                          unsigned long long* d, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), s);
  for (size_t c = 0; c < in.size() && e == cudaSuccess; ++c) e = launch_column_digest(in[c], out[c], (uint32_t)c, d, s);
  return e;
}

// ------------------------------------------------------------ online tables
// The merge of an online table's committed main with delta `k` (its first
// `rows` rows) into the other main copy.
void online_args(const dm_server* S, uint32_t table_id, const dm_server::Table& t, uint32_t k, uint64_t rows,
                 std::vector<dm_column_in>* in, std::vector<dm_column_out>* out) {
  const uint64_t main_rows = S->sched->main_rows(table_id);
  in->assign(t.cols.size(), dm_column_in{});
  out->assign(t.cols.size(), dm_column_out{});
  for (size_t c = 0; c < t.cols.size(); ++c) {
    const OnlineColumn& oc = t.cols[c];
    dm_column_in& ci = (*in)[c];
    ci.value_bytes = oc.w;
    ci.main_dict = oc.dict[t.cur];
    ci.main_dict_len = oc.u;
    ci.main_packed = oc.packed[t.cur];
    ci.main_bits = oc.bits;
    ci.main_rows = main_rows;
    ci.delta_dict = oc.delta[k];
    ci.delta_dict_len = rows;
    ci.delta_codes = t.iota;
    ci.delta_rows = rows;
    dm_column_out& co = (*out)[c];
    co.new_dict = oc.dict[t.cur ^ 1u];
    co.new_packed = oc.packed[t.cur ^ 1u];
    co.d_new_dict_len = t.scalars + 2 * c;
    co.d_new_bits = reinterpret_cast<uint32_t*>(t.scalars + 2 * c + 1);
  }
}

void free_online(dm_server::Table& t) {
  for (void* p : t.owned)
    if (p) cudaFree(p);
  t.owned.clear();
  for (auto& e : t.inserted)
    if (e) cudaEventDestroy(e);
}

// One scheduling round under the lock: collect finished slots, start
// admissible requests.  Returns true when anything changed.
bool round(dm_server* S) {
  bool progress = false;
  for (auto& sl : S->slots) {
    if (!sl.busy) continue;
    const cudaError_t e = cudaEventQuery(sl.done);
    if (e == cudaErrorNotReady) continue;
    int st = e == cudaSuccess ? (int)dm_sync_status(sl.ctx, sl.stream) : (int)DM_ECUDA;
    if (e != cudaSuccess) cudaGetLastError();
    const dm::SchedRequest& r = S->sched->requests()[sl.req];
    dm_server::Table& t = S->tables.at(r.table);
    uint64_t digest = 0;
    if (st == DM_OK && S->digest &&
        cudaMemcpy(&digest, sl.d_digest, sizeof(digest), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = DM_ECUDA;
    if (st == DM_OK && t.online) {
      // the merged main's |U'| and E'_C, for the commit
      if (cudaMemcpy(t.host_scalars.data(), t.scalars, t.host_scalars.size() * sizeof(uint64_t),
                     cudaMemcpyDeviceToHost) != cudaSuccess)
        st = DM_ECUDA;
    }
    if (st == DM_OK && t.online) {
      for (size_t c = 0; c < t.cols.size(); ++c) {
        t.cols[c].u = t.host_scalars[2 * c];
        t.cols[c].bits = (uint32_t)(t.host_scalars[2 * c + 1] & 0xFFFFFFFFu);
      }
      t.cur ^= 1u;
    }
    S->sched->requests_mut()[sl.req].digest = digest;
    S->sched->complete(sl.req, S->now(), st);
    sl.busy = false;
    progress = true;
  }
  for (const dm::SchedAdmit& a : S->sched->admit(S->now())) {
    auto& sl = S->slots[a.slot];
    const dm::SchedRequest& r = S->sched->requests()[a.request];
    auto& t = S->tables.at(r.table);
    progress = true;
    std::vector<dm_column_in> oin;
    std::vector<dm_column_out> oout;
    const std::vector<dm_column_in>* in = &t.in;
    const std::vector<dm_column_out>* out = &t.out;
    uint64_t tuples = t.tuples;
    uint32_t flags = S->merge_flags;
    if (t.online) {
      if (r.delta_rows == 0) {   // nothing inserted: nothing to merge or commit
        S->sched->complete(a.request, S->now(), DM_OK);
        continue;
      }
      online_args(S, r.table, t, r.delta, r.delta_rows, &oin, &oout);
      in = &oin;
      out = &oout;
      tuples = (S->sched->main_rows(r.table) + r.delta_rows) * t.cols.size();
      S->sched->requests_mut()[a.request].tuples = tuples;
      flags |= DM_FLAG_NO_GRAPH;   // sizes change with every version
    }
    dm_ctx_use_region(sl.ctx, static_cast<char*>(S->pool) + a.offset, a.bytes);
    sl.stream = sl.by_level[level_of(S, tuples)];
    dm_status st = DM_OK;
    // the merge reads the frozen delta after every insert into it has landed
    if (t.online && cudaStreamWaitEvent(sl.stream, t.inserted[r.delta], 0) != cudaSuccess) st = DM_ECUDA;
    if (st == DM_OK) st = dm_merge_table(sl.ctx, in->data(), (uint32_t)in->size(), out->data(), sl.stream, flags);
    if (st == DM_OK && S->digest && launch_digest(*in, *out, sl.d_digest, sl.stream) != cudaSuccess)
      st = DM_ECUDA;
    if (st == DM_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) st = DM_ECUDA;
    if (st != DM_OK) {
      S->sched->complete(a.request, S->now(), (int)st);
    } else {
      sl.busy = true;
      sl.req = a.request;
    }
  }
  return progress;
}

void worker_main(dm_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    const bool progress = round(S);
    if (progress) S->cv.notify_all();
    if (!progress) {
      // a slot still running: poll soon; nothing running: wait for a submit
      if (S->sched->running()) S->cv.wait_for(lk, std::chrono::microseconds(20));
      else S->cv.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

}  // namespace

extern "C" {

dm_status dm_column_digest(const dm_column_in* in, const dm_column_out* out, uint32_t col_index,
                           uint64_t* d_digest, void* stream) {
  if (!in || !out || !d_digest || (in->value_bytes != 4 && in->value_bytes != 8 && in->value_bytes != 16) ||
      !out->d_new_dict_len || !out->d_new_bits)
    return DM_EINVAL;
  if ((in->main_dict_len + in->delta_dict_len && !out->new_dict) ||
      (in->main_rows + in->delta_rows && dm_max_bits(in) && !out->new_packed))
    return DM_EINVAL;
  return launch_column_digest(*in, *out, col_index, reinterpret_cast<unsigned long long*>(d_digest),
                              static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? DM_OK
             : DM_ECUDA;
}

dm_status dm_server_create(dm_server** out, int device, const dm_server_config* cfg) {
  if (!out || !cfg || cfg->slots == 0 || cfg->slots > 16 || cfg->scratch_budget == 0) return DM_EINVAL;
  *out = nullptr;
  dm_server* S = new (std::nothrow) dm_server();
  if (!S) return DM_ENOMEM;
  S->device = device;
  S->cfg = *cfg;
  S->digest = (cfg->flags & DM_SERVER_DIGEST) != 0;
  S->merge_flags = cfg->flags & ~DM_SERVER_DIGEST;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete S;
    return DM_ECUDA;
  }
  if (cudaMalloc(&S->pool, cfg->scratch_budget) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return DM_ENOMEM;
  }
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->insert_stream, cudaStreamNonBlocking) != cudaSuccess) {
    if (S->insert_stream) cudaStreamDestroy(S->insert_stream);
    cudaFree(S->pool);
    delete S;
    return DM_ECUDA;
  }
  S->greatest = greatest;
  S->levels = std::min(dm_server::kLevels, least - greatest + 1);
  S->sched = new dm::Scheduler(cfg->scratch_budget, cfg->slots);
  S->slots.resize(cfg->slots);
  for (auto& sl : S->slots) {
    bool streams_ok = true;
    for (int l = 0; l < S->levels && streams_ok; ++l)
      streams_ok = cudaStreamCreateWithPriority(&sl.by_level[l], cudaStreamNonBlocking, S->greatest + l) == cudaSuccess;
    sl.stream = sl.by_level[0];
    if (!streams_ok || dm_create(&sl.ctx, device, 0) != DM_OK ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&sl.d_digest, sizeof(unsigned long long)) != cudaSuccess) {
      dm_server_destroy(S);
      return DM_ECUDA;
    }
    sl.ctx->coop_share = cfg->slots;
    sl.ctx->tuning.table_branches = kSlotBranches;
    dm_set_tune_cache(sl.ctx, &S->tune_cache);
  }
  S->worker = std::thread(worker_main, S);
  *out = S;
  return DM_OK;
}

dm_tune_cache* dm_server_tune_cache(dm_server* S) { return S ? &S->tune_cache : nullptr; }

void dm_server_destroy(dm_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  cudaSetDevice(S->device);
  for (auto& sl : S->slots) {
    for (cudaStream_t st : sl.by_level)
      if (st) cudaStreamSynchronize(st);
    if (sl.ctx) {
      sl.ctx->arena = nullptr;   // the pool region is not the context's to free
      dm_destroy(sl.ctx);
    }
    for (cudaStream_t st : sl.by_level)
      if (st) cudaStreamDestroy(st);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.d_digest) cudaFree(sl.d_digest);
  }
  if (S->insert_stream) {
    cudaStreamSynchronize(S->insert_stream);
    cudaStreamDestroy(S->insert_stream);
  }
  for (auto& kv : S->tables) free_online(kv.second);
  if (S->pool) cudaFree(S->pool);
  delete S->sched;
  delete S;
}

dm_status dm_server_add_table(dm_server* S, uint32_t id, const dm_column_in* in, uint32_t ncols,
                              const dm_column_out* out) {
  if (!S || !in || !out || ncols == 0) return DM_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  if (S->tables.count(id)) return DM_EINVAL;
  dm_server::Table t;
  t.in.assign(in, in + ncols);
  t.out.assign(out, out + ncols);
  for (uint32_t c = 0; c < ncols; ++c) t.tuples += in[c].main_rows + in[c].delta_rows;
  const uint64_t footprint = dm_table_scratch_bytes_for(in, ncols, S->merge_flags, kSlotBranches);
  if (!S->sched->add_table(id, footprint)) return DM_ENOMEM;
  S->tables.emplace(id, std::move(t));
  return DM_OK;
}

dm_status dm_server_add_online_table(dm_server* S, uint32_t id, uint32_t ncols, const dm_online_column* cols,
                                     const dm_online_config* cfg) {
  if (!S || !cols || !cfg || ncols == 0) return DM_EINVAL;
  if (cfg->rows_capacity < cfg->main_rows || cfg->delta_capacity == 0 || cfg->delta_capacity >= (1ull << 30) ||
      !(cfg->trigger >= 0))
    return DM_EINVAL;
  for (uint32_t c = 0; c < ncols; ++c) {
    const dm_online_column& oc = cols[c];
    if ((oc.value_bytes != 4 && oc.value_bytes != 8 && oc.value_bytes != 16) || oc.main_bits > 32 ||
        oc.main_bits < dm_bits_for(oc.main_dict_len) || (cfg->main_rows && !oc.main_dict_len) ||
        (oc.main_dict_len && !oc.main_dict) || (cfg->main_rows && oc.main_bits && !oc.main_packed) ||
        oc.main_dict_len + cfg->rows_capacity - cfg->main_rows > 0xFFFFFFFFull)
      return DM_EINVAL;
  }
  std::lock_guard<std::mutex> g(S->mu);
  if (S->tables.count(id)) return DM_EINVAL;
  if (cudaSetDevice(S->device) != cudaSuccess) return DM_ECUDA;
  dm_server::Table t;
  t.online = true;
  t.delta_cap = cfg->delta_capacity;
  auto dev_alloc = [&t](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    t.owned.push_back(p);
    return p;
  };
  bool ok = true;
  // the footprint at capacity: any merge of the table fits it
  std::vector<dm_column_in> cap(ncols);
  t.cols.resize(ncols);
  for (uint32_t c = 0; c < ncols && ok; ++c) {
    const dm_online_column& src = cols[c];
    OnlineColumn& oc = t.cols[c];
    oc.w = src.value_bytes;
    oc.dict_cap = src.main_dict_len + (cfg->rows_capacity - cfg->main_rows);
    oc.u = src.main_dict_len;
    oc.bits = src.main_bits;
    const uint32_t bits_cap = std::max<uint32_t>(dm_bits_for(oc.dict_cap), src.main_bits);
    const size_t packed_bytes = dm_packed_bytes(cfg->rows_capacity, bits_cap);
    for (int k = 0; k < 2 && ok; ++k) {
      oc.dict[k] = dev_alloc(oc.dict_cap * oc.w);
      oc.packed[k] = dev_alloc(packed_bytes);
      oc.delta[k] = dev_alloc(cfg->delta_capacity * oc.w);
      ok = oc.dict[k] && oc.packed[k] && oc.delta[k];
    }
    if (!ok) break;
    if (oc.u && cudaMemcpy(oc.dict[0], src.main_dict, oc.u * oc.w, cudaMemcpyDefault) != cudaSuccess) ok = false;
    const size_t main_bytes = dm_packed_bytes(cfg->main_rows, src.main_bits);
    if (ok && main_bytes && cudaMemcpy(oc.packed[0], src.main_packed, main_bytes, cudaMemcpyDefault) != cudaSuccess)
      ok = false;
    dm_column_in& ci = cap[c];
    ci.value_bytes = oc.w;
    ci.main_dict_len = oc.dict_cap;
    ci.main_bits = bits_cap;
    ci.main_rows = cfg->rows_capacity;
    ci.delta_dict_len = cfg->delta_capacity;
    ci.delta_rows = cfg->delta_capacity;
  }
  if (ok) {
    t.iota = static_cast<uint32_t*>(dev_alloc(cfg->delta_capacity * 4));
    t.scalars = static_cast<uint64_t*>(dev_alloc(2 * ncols * sizeof(uint64_t)));
    ok = t.iota && t.scalars;
  }
  if (ok) {
    // the codes of a delta whose dictionary is its rows' values in arrival order
    std::vector<uint32_t> h(cfg->delta_capacity);
    for (uint64_t i = 0; i < cfg->delta_capacity; ++i) h[i] = (uint32_t)i;
    ok = cudaMemcpy(t.iota, h.data(), h.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess;
  }
  for (auto& e : t.inserted)
    if (ok) ok = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    free_online(t);
    return DM_ENOMEM;
  }
  t.host_scalars.assign(2 * ncols, 0);
  // scratch grows with |U_M| except that dictionaries of up to
  // reencode_dir_max_codes() main codes may add a byte table: the footprint
  // is the larger of the two sizes at capacity
  std::vector<dm_column_in> cap_x8 = cap;
  for (auto& ci : cap_x8) ci.main_dict_len = std::min<uint64_t>(ci.main_dict_len, dm::reencode_dir_max_codes());
  const uint32_t fflags = S->merge_flags | DM_FLAG_NO_GRAPH;
  const uint64_t footprint = std::max(dm_table_scratch_bytes_for(cap.data(), ncols, fflags, kSlotBranches),
                                      dm_table_scratch_bytes_for(cap_x8.data(), ncols, fflags, kSlotBranches));
  if (!S->sched->add_online_table(id, footprint, cfg->main_rows, cfg->rows_capacity, cfg->delta_capacity,
                                  cfg->trigger)) {
    free_online(t);
    return DM_ENOMEM;
  }
  S->tables.emplace(id, std::move(t));
  return DM_OK;
}

dm_status dm_server_insert(dm_server* S, uint32_t id, uint64_t nrows, const void* const* values,
                           dm_insert_info* info) {
  if (!S || (nrows && !values)) return DM_EINVAL;
  dm::SchedInsert r;
  {
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->tables.find(id);
    if (it == S->tables.end() || !it->second.online) return DM_EINVAL;
    dm_server::Table& t = it->second;
    for (size_t c = 0; c < t.cols.size() && nrows; ++c)
      if (!values[c]) return DM_EINVAL;
    r = S->sched->insert(id, nrows, S->now());
    if (r.status == 2) return DM_EBUSY;
    if (r.status != 0) return DM_EINVAL;
    if (cudaSetDevice(S->device) != cudaSuccess) return DM_ECUDA;
    // the copies are queued under the lock, before the event a merge that
    // freezes this delta waits on
    cudaError_t e = cudaSuccess;
    for (size_t c = 0; c < t.cols.size() && nrows && e == cudaSuccess; ++c) {
      const OnlineColumn& oc = t.cols[c];
      e = cudaMemcpyAsync(static_cast<char*>(oc.delta[r.delta]) + r.first_row * oc.w, values[c], nrows * oc.w,
                          cudaMemcpyDefault, S->insert_stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(t.inserted[r.delta], S->insert_stream);
    if (e != cudaSuccess) return DM_ECUDA;
  }
  if (r.triggered) S->cv.notify_all();
  // the caller's buffers are free once the copies have landed
  if (cudaStreamSynchronize(S->insert_stream) != cudaSuccess) return DM_ECUDA;
  if (info) {
    info->delta = r.delta;
    info->first_row = r.first_row;
    info->lands_in = r.lands_in;
    info->triggered = r.triggered ? 1u : 0u;
    info->request = r.triggered ? r.request : 0;
  }
  return DM_OK;
}

dm_status dm_server_pause(dm_server* S, uint32_t id, int paused) {
  if (!S) return DM_EINVAL;
  {
    std::lock_guard<std::mutex> g(S->mu);
    if (!S->sched->set_paused(id, paused != 0)) return DM_EINVAL;
  }
  S->cv.notify_all();
  return DM_OK;
}

dm_status dm_server_online_view(dm_server* S, uint32_t id, uint32_t col, dm_online_view* v) {
  if (!S || !v) return DM_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->tables.find(id);
  if (it == S->tables.end() || !it->second.online || col >= it->second.cols.size()) return DM_EINVAL;
  const dm_server::Table& t = it->second;
  const OnlineColumn& oc = t.cols[col];
  v->version = S->sched->version(id);
  v->main_dict = oc.dict[t.cur];
  v->main_dict_len = oc.u;
  v->main_packed = oc.packed[t.cur];
  v->main_bits = oc.bits;
  v->main_rows = S->sched->main_rows(id);
  v->delta_rows = S->sched->delta_rows(id, 0) + S->sched->delta_rows(id, 1);
  return DM_OK;
}

dm_status dm_server_online_copy(dm_server* S, uint32_t id, uint32_t col, void* dict_dst, size_t dict_bytes,
                                void* packed_dst, size_t packed_bytes, dm_online_view* v) {
  if (!S || !v) return DM_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->tables.find(id);
  if (it == S->tables.end() || !it->second.online || col >= it->second.cols.size()) return DM_EINVAL;
  const dm_server::Table& t = it->second;
  const OnlineColumn& oc = t.cols[col];
  const uint64_t rows = S->sched->main_rows(id);
  const size_t db = oc.u * oc.w, pb = dm_packed_bytes(rows, oc.bits);
  if ((db && (!dict_dst || dict_bytes < db)) || (pb && (!packed_dst || packed_bytes < pb))) return DM_EINVAL;
  if (cudaSetDevice(S->device) != cudaSuccess) return DM_ECUDA;
  if (db && cudaMemcpy(dict_dst, oc.dict[t.cur], db, cudaMemcpyDefault) != cudaSuccess) return DM_ECUDA;
  if (pb && cudaMemcpy(packed_dst, oc.packed[t.cur], pb, cudaMemcpyDefault) != cudaSuccess) return DM_ECUDA;
  v->version = S->sched->version(id);
  v->main_dict = oc.dict[t.cur];
  v->main_dict_len = oc.u;
  v->main_packed = oc.packed[t.cur];
  v->main_bits = oc.bits;
  v->main_rows = rows;
  v->delta_rows = S->sched->delta_rows(id, 0) + S->sched->delta_rows(id, 1);
  return DM_OK;
}

dm_status dm_server_submit(dm_server* S, uint32_t table_id, uint64_t* request_id) {
  if (!S) return DM_EINVAL;
  {
    std::lock_guard<std::mutex> g(S->mu);
    if (!S->sched->has_table(table_id)) return DM_EINVAL;
    const uint64_t id = S->sched->submit(table_id, S->now());
    if (request_id) *request_id = id;
  }
  S->cv.notify_all();
  return DM_OK;
}

dm_status dm_server_drain(dm_server* S, uint64_t timeout_ms) {
  if (!S) return DM_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  const bool ok = S->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [S] { return S->sched->idle(); });
  return ok ? DM_OK : DM_EBUSY;
}

dm_status dm_server_request_info(dm_server* S, uint64_t id, dm_request_info* info) {
  if (!S || !info) return DM_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  const auto& rs = S->sched->requests();
  if (id >= rs.size()) return DM_EINVAL;
  const auto& r = rs[id];
  *info = dm_request_info{};
  info->table_id = r.table;
  info->status = r.done ? r.status : -1;
  info->submit_ns = r.submit_ns;
  info->admit_ns = r.admit_ns;
  info->done_ns = r.done_ns;
  info->footprint = r.footprint;
  info->slot = r.slot;
  info->automatic = r.automatic ? 1u : 0u;
  info->version = r.version;
  info->delta_rows = r.delta_rows;
  info->digest = r.digest;
  return DM_OK;
}

dm_status dm_server_stats_get(dm_server* S, dm_server_stats* st) {
  if (!S || !st) return DM_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  *st = dm_server_stats{};
  std::vector<double> lat;
  uint64_t first = ~0ull, last = 0;
  for (const auto& r : S->sched->requests()) {
    ++st->submitted;
    first = std::min(first, r.submit_ns);
    if (!r.done) continue;
    if (r.status != 0) {
      ++st->failed;
      continue;
    }
    ++st->completed;
    const auto& t = S->tables.at(r.table);
    st->tuples += t.online ? r.tuples : t.tuples;
    lat.push_back((r.done_ns - r.submit_ns) / 1e6);
    last = std::max(last, r.done_ns);
  }
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    double sum = 0;
    for (double v : lat) sum += v;
    st->mean_ms = sum / lat.size();
    st->p50_ms = lat[lat.size() / 2];
    st->p99_ms = lat[std::min(lat.size() - 1, (size_t)(0.99 * lat.size()))];
    st->max_ms = lat.back();
  }
  st->first_submit_ns = first == ~0ull ? 0 : first;
  st->last_done_ns = last;
  st->peak_scratch_bytes = S->sched->peak_bytes();
  st->peak_concurrency = S->sched->peak_running();
  st->scratch_budget = S->sched->pool_bytes();
  return DM_OK;
}

uint64_t dm_server_table_version(dm_server* S, uint32_t table_id) {
  if (!S) return 0;
  std::lock_guard<std::mutex> g(S->mu);
  return S->sched->has_table(table_id) ? S->sched->version(table_id) : 0;
}

// Event-driven run of the scheduler core with a fake clock: requests of
// req_table[i] arrive at arrival_ns[i] (non-decreasing) and each merge of
// table t takes service_ns[t].  Fills admit/done times and slots, the peak
// scratch bytes in use and the peak number of merges running at once.
dm_status dm_sched_simulate(uint64_t pool_bytes, uint32_t slots, uint32_t ntables, const uint64_t* footprint,
                            const uint64_t* service_ns, uint64_t nreq, const uint32_t* req_table,
                            const uint64_t* arrival_ns, uint64_t* admit_ns, uint64_t* done_ns, uint32_t* slot_out,
                            uint64_t* peak_bytes, uint32_t* peak_running) {
  if (!footprint || !service_ns || (nreq && (!req_table || !arrival_ns || !admit_ns || !done_ns || !slot_out)) ||
      slots == 0 || pool_bytes == 0)
    return DM_EINVAL;
  dm::Scheduler sch(pool_bytes, slots);
  for (uint32_t t = 0; t < ntables; ++t)
    if (!sch.add_table(t, footprint[t])) return DM_ENOMEM;
  for (uint64_t i = 0; i < nreq; ++i)
    if (req_table[i] >= ntables || (i && arrival_ns[i] < arrival_ns[i - 1])) return DM_EINVAL;
  std::multimap<uint64_t, uint64_t> running;   // done time -> request
  uint64_t next = 0, now = 0;
  while (next < nreq || !running.empty()) {
    const uint64_t ta = next < nreq ? arrival_ns[next] : ~0ull;
    const uint64_t tc = running.empty() ? ~0ull : running.begin()->first;
    now = std::min(ta, tc);
    while (!running.empty() && running.begin()->first == now) {
      sch.complete(running.begin()->second, now, 0);
      running.erase(running.begin());
    }
    while (next < nreq && arrival_ns[next] == now) sch.submit(req_table[next++], now);
    for (const auto& a : sch.admit(now)) {
      const uint32_t t = sch.requests()[a.request].table;
      running.emplace(now + service_ns[t], a.request);
    }
    if (next >= nreq && running.empty() && !sch.idle()) return DM_ENOMEM;   // cannot make progress
  }
  for (uint64_t i = 0; i < nreq; ++i) {
    const auto& r = sch.requests()[i];
    admit_ns[i] = r.admit_ns;
    done_ns[i] = r.done_ns;
    slot_out[i] = r.slot;
  }
  if (peak_bytes) *peak_bytes = sch.peak_bytes();
  if (peak_running) *peak_running = sch.peak_running();
  return DM_OK;
}

// The online rules on a fake clock: inserts, requests, pauses and resumes
// in time order against the same scheduler core the server runs.
dm_status dm_online_simulate(uint32_t slots, uint32_t ntables, const uint64_t* main_rows,
                             const uint64_t* delta_capacity, const double* trigger, const uint64_t* service_ns,
                             uint64_t nevents, const uint32_t* ev_kind, const uint32_t* ev_table,
                             const uint64_t* ev_rows, const uint64_t* ev_ns, uint64_t* ev_lands_in,
                             uint64_t* ev_version, uint64_t max_merges, uint32_t* merge_table,
                             uint64_t* merge_admit_ns, uint64_t* merge_done_ns, uint64_t* merge_rows,
                             uint64_t* merge_version, uint32_t* merge_automatic, uint64_t* nmerges) {
  if (slots == 0 || !main_rows || !delta_capacity || !trigger || !service_ns || !nmerges ||
      (nevents && (!ev_kind || !ev_table || !ev_rows || !ev_ns || !ev_lands_in || !ev_version)) ||
      (max_merges && (!merge_table || !merge_admit_ns || !merge_done_ns || !merge_rows || !merge_version ||
                      !merge_automatic)))
    return DM_EINVAL;
  for (uint64_t i = 0; i < nevents; ++i)
    if (ev_kind[i] > 3 || ev_table[i] >= ntables || (i && ev_ns[i] < ev_ns[i - 1])) return DM_EINVAL;
  dm::Scheduler sch(1ull << 62, slots);
  for (uint32_t t = 0; t < ntables; ++t)
    if (!sch.add_online_table(t, 1, main_rows[t], ~0ull >> 2, delta_capacity[t], trigger[t])) return DM_EINVAL;
  // the inserts waiting in each table's two deltas, to learn the version that takes them
  std::vector<std::vector<uint64_t>> pending(2 * (size_t)ntables);
  std::multimap<uint64_t, uint64_t> running;   // done time -> request
  std::vector<uint64_t> admitted;               // requests in admission order
  uint64_t next = 0;
  for (uint64_t i = 0; i < nevents; ++i) ev_lands_in[i] = ev_version[i] = 0;
  auto admit_now = [&](uint64_t now) {
    for (const auto& a : sch.admit(now)) {
      const auto& r = sch.requests()[a.request];
      admitted.push_back(a.request);
      running.emplace(now + (r.delta_rows ? service_ns[r.table] : 0), a.request);
    }
  };
  uint64_t guard = 0;
  while (next < nevents || !running.empty()) {
    if (++guard > 64 * (nevents + 16) + (1u << 20)) return DM_EINVAL;   // no progress
    const uint64_t te = next < nevents ? ev_ns[next] : ~0ull;
    const uint64_t tc = running.empty() ? ~0ull : running.begin()->first;
    const uint64_t now = std::min(te, tc);
    while (!running.empty() && running.begin()->first == now) {
      const uint64_t id = running.begin()->second;
      running.erase(running.begin());
      const auto& r = sch.requests()[id];
      const uint32_t tab = r.table, k = r.delta;
      const bool had_rows = r.delta_rows != 0;
      sch.complete(id, now, 0);
      if (had_rows) {
        for (uint64_t e : pending[2 * tab + k]) ev_version[e] = sch.requests()[id].version;
        pending[2 * tab + k].clear();
      }
    }
    while (next < nevents && ev_ns[next] == now) {
      const uint64_t i = next++;
      const uint32_t tab = ev_table[i];
      switch (ev_kind[i]) {
        case 0: {
          const dm::SchedInsert r = sch.insert(tab, ev_rows[i], now);
          if (r.status == 0) {
            ev_lands_in[i] = r.lands_in;
            pending[2 * tab + r.delta].push_back(i);
          }
          break;
        }
        case 1: sch.submit(tab, now); break;
        case 2: sch.set_paused(tab, true); break;
        default: sch.set_paused(tab, false); break;
      }
    }
    admit_now(now);
  }
  uint64_t n = 0;
  for (uint64_t id : admitted) {
    const auto& r = sch.requests()[id];
    if (n < max_merges) {
      merge_table[n] = r.table;
      merge_admit_ns[n] = r.admit_ns;
      merge_done_ns[n] = r.done_ns;
      merge_rows[n] = r.delta_rows;
      merge_version[n] = r.version;
      merge_automatic[n] = r.automatic ? 1u : 0u;
    }
    ++n;
  }
  *nmerges = n;
  return DM_OK;
}

}  // extern "C"
