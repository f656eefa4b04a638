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
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dm_ctx.h"
#include "dm_internal.h"
#include "dm_sched.h"

// Branches of each slot's batched table merges: slots already run side by
// side, so fewer than a table merged alone.
constexpr uint32_t kSlotBranches = 4;

struct dm_server {
  int device = 0;
  dm_server_config cfg{};
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
    uint64_t req = 0;
    bool busy = false;
  };
  std::vector<Slot> slots;
  dm_tune_cache tune_cache;   // shared by every slot's context
  struct Table {
    std::vector<dm_column_in> in;
    std::vector<dm_column_out> out;
    uint64_t tuples = 0;
  };
  std::unordered_map<uint32_t, Table> tables;
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
    S->sched->complete(sl.req, S->now(), st);
    sl.busy = false;
    progress = true;
  }
  for (const dm::SchedAdmit& a : S->sched->admit(S->now())) {
    auto& sl = S->slots[a.slot];
    const dm::SchedRequest& r = S->sched->requests()[a.request];
    auto& t = S->tables.at(r.table);
    dm_ctx_use_region(sl.ctx, static_cast<char*>(S->pool) + a.offset, a.bytes);
    sl.stream = sl.by_level[level_of(S, t.tuples)];
    dm_status st = dm_merge_table(sl.ctx, t.in.data(), (uint32_t)t.in.size(), t.out.data(), sl.stream, S->cfg.flags);
    if (st == DM_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) st = DM_ECUDA;
    if (st != DM_OK) {
      S->sched->complete(a.request, S->now(), (int)st);
    } else {
      sl.busy = true;
      sl.req = a.request;
    }
    progress = true;
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

dm_status dm_server_create(dm_server** out, int device, const dm_server_config* cfg) {
  if (!out || !cfg || cfg->slots == 0 || cfg->slots > 16 || cfg->scratch_budget == 0) return DM_EINVAL;
  *out = nullptr;
  dm_server* S = new (std::nothrow) dm_server();
  if (!S) return DM_ENOMEM;
  S->device = device;
  S->cfg = *cfg;
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
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
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
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
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
  }
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
  const uint64_t footprint = dm_table_scratch_bytes_for(in, ncols, S->cfg.flags, kSlotBranches);
  if (!S->sched->add_table(id, footprint)) return DM_ENOMEM;
  S->tables.emplace(id, std::move(t));
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
  info->table_id = r.table;
  info->status = r.done ? r.status : -1;
  info->submit_ns = r.submit_ns;
  info->admit_ns = r.admit_ns;
  info->done_ns = r.done_ns;
  info->footprint = r.footprint;
  info->slot = r.slot;
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
    st->tuples += S->tables.at(r.table).tuples;
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

}  // extern "C"
