// C ABI of libdmerge: context and scratch arena, argument checks, and the
// entry points declared in include/dmerge.h.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/dmerge.h"
#include "dm_common.cuh"
#include "dm_internal.h"

#include "dm_ctx.h"

namespace {

using dm::bits_for;

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

bool width_ok(uint32_t w) { return w == 4 || w == 8 || w == 16; }

// Bump allocator over the arena (or a dry run that only sums sizes).
struct Carver {
  char* base;
  size_t used = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  void* take(size_t bytes) {
    void* p = base ? base + used : nullptr;
    used += align_up(bytes ? bytes : 1);
    return p;
  }
};

struct ColumnScratch {
  uint32_t* zero = nullptr;   // one memset covers all Step 1 bookkeeping
  size_t zero_bytes = 0;
  dm::Step1Args s1{};
  uint32_t* xm = nullptr;
  uint32_t* xd = nullptr;
  uint32_t* xdir = nullptr;   // directory of X_M for Step 2(b)
  uint8_t* x8 = nullptr;      // its byte table
  uint2* gdir = nullptr;      // global directory (more main codes than the shared one covers)
  void** slots = nullptr;
};

// Lay out the scratch of one column merge; with base == nullptr only sizes.
size_t carve_column(void* base, const dm_column_in* in, const dm_column_out* out, ColumnScratch* cs) {
  Carver c(base);
  const uint32_t w = in->value_bytes;
  const uint64_t m = in->main_dict_len, d = in->delta_dict_len;
  const size_t zero_bytes = (size_t)dm::step1_zeroed_words(w, m + d, d) * 4;
  char* zero = static_cast<char*>(c.take(zero_bytes));
  void* k0 = c.take(d * w);
  void* k1 = c.take(d * w);
  void* v0 = c.take(d * 4);
  void* v1 = c.take(d * 4);
  void* slots = c.take(2 * sizeof(void*));
  void* xm = (out && out->x_main) ? nullptr : c.take(m * 4);
  void* xd = (out && out->x_delta) ? nullptr : c.take(d * 4);
  void* xdir = in->main_rows ? c.take((size_t)dm::reencode_dir_words(m) * 4) : nullptr;
  void* x8 = in->main_rows && dm::reencode_wants_x8(m) ? c.take(m) : nullptr;
  const uint64_t gdir_n = in->main_rows ? dm::reencode_gdir_entries(m, d) : 0;
  void* gdir = gdir_n ? c.take(gdir_n * sizeof(uint2)) : nullptr;
  void* cuts = c.take(((size_t)dm::merge_tiles(m + d, w) + 1) * 8);
  if (cs && base) {
    cs->zero = reinterpret_cast<uint32_t*>(zero);
    cs->zero_bytes = zero_bytes;
    cs->slots = static_cast<void**>(slots);
    cs->xdir = static_cast<uint32_t*>(xdir);
    cs->x8 = static_cast<uint8_t*>(x8);
    cs->gdir = static_cast<uint2*>(gdir);
    dm::Step1Args& a = cs->s1;
    dm::step1_layout(w, m + d, d, cs->zero, &a);
    a.in_keys = in->delta_dict;
    a.d = d;
    a.keys[0] = k0;
    a.keys[1] = k1;
    a.vals[0] = static_cast<uint32_t*>(v0);
    a.vals[1] = static_cast<uint32_t*>(v1);
    a.final_slot = cs->slots;
    a.a = in->main_dict;
    a.m = m;
    a.cuts = static_cast<uint64_t*>(cuts);
    cs->xm = (out && out->x_main) ? out->x_main : static_cast<uint32_t*>(xm);
    cs->xd = (out && out->x_delta) ? out->x_delta : static_cast<uint32_t*>(xd);
    a.xm = cs->xm;
    a.xd = cs->xd;
  }
  return c.used;
}

dm_status check_column(const dm_column_in* in, const dm_column_out* out, bool device_ptrs) {
  if (!in || !out) return DM_EINVAL;
  const uint32_t w = in->value_bytes;
  const uint64_t m = in->main_dict_len, d = in->delta_dict_len;
  if (!width_ok(w) || in->main_bits > 32) return DM_EINVAL;
  if (m + d > (1ull << 32) || m > 0xFFFFFFFFull || d >= (1ull << 30)) return DM_EINVAL;
  if (in->main_bits < bits_for(m)) return DM_EINVAL;
  if ((in->main_rows && !m) || (in->delta_rows && !d)) return DM_EINVAL;
  if (in->main_rows + in->delta_rows >= (1ull << 40)) return DM_EINVAL;
  const size_t ka = w == 16 ? 16 : w;
  if (m && (!in->main_dict || !aligned(in->main_dict, ka))) return DM_EINVAL;
  if (d && (!in->delta_dict || !aligned(in->delta_dict, ka))) return DM_EINVAL;
  if (in->main_rows && in->main_bits && (!in->main_packed || (device_ptrs && !aligned(in->main_packed, 16))))
    return DM_EINVAL;
  if (in->delta_rows && (!in->delta_codes || !aligned(in->delta_codes, 4))) return DM_EINVAL;
  const uint32_t maxb = bits_for(m + d);
  if (m + d && (!out->new_dict || !aligned(out->new_dict, ka))) return DM_EINVAL;
  if (in->main_rows + in->delta_rows && maxb &&
      (!out->new_packed || (device_ptrs && !aligned(out->new_packed, 16))))
    return DM_EINVAL;
  if (device_ptrs && (!out->d_new_dict_len || !out->d_new_bits)) return DM_EINVAL;
  if (out->x_main && !aligned(out->x_main, 4)) return DM_EINVAL;
  if (out->x_delta && !aligned(out->x_delta, 4)) return DM_EINVAL;
  return DM_OK;
}

dm_status cuda_status(cudaError_t e) { return e == cudaSuccess ? DM_OK : DM_ECUDA; }

// Launch choices in effect for one column.  A forced choice (the
// autotuner's candidates) is taken as it is; otherwise non-zero dm_tuning
// fields and the X_M staging flags come first, then the tune cache's entry
// for the column's class, then the library defaults (zeros).
struct Resolved {
  uint32_t warps, stages, obufs;
  uint32_t flags;          // the call's flags with the staging choice applied
  uint32_t step1_blocks;   // 0: every block that fits
  bool x8;
};

Resolved resolve(const dm_ctx* ctx, const dm_column_in* in, uint32_t flags, const dm_tune_choice* force) {
  dm_tune_choice c{};
  flags &= ~DM_FLAG_AUTOTUNE;
  if (force) {
    c = *force;
    flags &= ~(DM_FLAG_X_SMEM | DM_FLAG_X_GLOBAL);
  } else if (ctx->tune_cache->size.load(std::memory_order_relaxed)) {
    const dm_tune_key k = dm::tune_key_of(*in);
    if (dm_tune_cache_get(ctx->tune_cache, &k, &c) != DM_OK) c = dm_tune_choice{};
  }
  Resolved r;
  const bool expl = force == nullptr;
  r.warps = expl && ctx->tuning.reencode_warps ? ctx->tuning.reencode_warps : c.reencode_warps;
  r.stages = expl && ctx->tuning.reencode_stages ? ctx->tuning.reencode_stages : c.reencode_stages;
  r.obufs = expl && ctx->tuning.reencode_obufs ? ctx->tuning.reencode_obufs : c.reencode_obufs;
  r.flags = flags;
  if (!(flags & (DM_FLAG_X_SMEM | DM_FLAG_X_GLOBAL))) {
    if (c.x_staging == DM_STAGE_SMEM) r.flags |= DM_FLAG_X_SMEM;
    else if (c.x_staging == DM_STAGE_GLOBAL) r.flags |= DM_FLAG_X_GLOBAL;
  }
  r.step1_blocks = c.step1_blocks;
  r.x8 = c.x8 != DM_X8_OFF;
  return r;
}

// A column with rows whose class the context's tune cache lacks.
bool needs_tuning(const dm_ctx* ctx, const dm_column_in* in) {
  if (in->main_rows + in->delta_rows == 0) return false;
  const dm_tune_key k = dm::tune_key_of(*in);
  dm_tune_choice c;
  return dm_tune_cache_get(ctx->tune_cache, &k, &c) == DM_ENOENT;
}

// The autotuner's candidate choices for a column: X_M staging (shared
// memory or an L1/L2 gather, and the byte table where one is built) x
// Step 2(b) launch shape (warps, input stages, output buffers; the first is
// the default) x Step 1 grid (all blocks that fit, one per SM, a quarter).
std::vector<dm_tune_choice> tune_candidates(const dm_ctx* ctx, const dm_column_in* in) {
  static const uint32_t kShapes[][3] = {{0, 0, 0}, {16, 3, 1}, {16, 2, 2}, {8, 2, 1},
                                        {8, 3, 1}, {4, 2, 1}, {4, 4, 2}};
  std::vector<uint32_t> stagings = {DM_STAGE_AUTO};
  if (in->main_rows) stagings = {DM_STAGE_SMEM, DM_STAGE_GLOBAL};
  std::vector<uint32_t> x8s = {DM_X8_AUTO};
  if (in->main_rows && dm::reencode_wants_x8(in->main_dict_len)) x8s.push_back(DM_X8_OFF);
  const uint32_t grids[] = {0, ctx->sm_count, std::max<uint32_t>(1, ctx->sm_count / 4)};
  std::vector<dm_tune_choice> v;
  for (uint32_t st : stagings)
    for (uint32_t x8 : x8s)
      for (const auto& sh : kShapes)
        for (uint32_t g : grids) {
          dm_tune_choice c{};
          c.x_staging = st;
          c.x8 = x8;
          c.reencode_warps = sh[0];
          c.reencode_stages = sh[1];
          c.reencode_obufs = sh[2];
          c.step1_blocks = g;
          v.push_back(c);
        }
  return v;
}

// Step 2(b) arguments that only the launch plan reads (sizes, tuning).
dm::ReencodeArgs plan_args(const dm_column_in* in, const Resolved& r) {
  dm::ReencodeArgs ra{};
  ra.n_main = in->main_rows;
  ra.n_delta = in->delta_rows;
  ra.m = (uint32_t)std::min<uint64_t>(in->main_dict_len, 0xFFFFFFFFu);
  ra.d = (uint32_t)std::min<uint64_t>(in->delta_dict_len, 0xFFFFFFFFu);
  ra.max_bits = bits_for(in->main_dict_len + in->delta_dict_len);
  ra.tune_warps = r.warps;
  ra.tune_stages = r.stages;
  ra.tune_obufs = r.obufs;
  ra.xdir_words = dm::reencode_dir_words(in->main_dict_len);   // as carve_column lays out
  return ra;
}

// Steps 1(a)..2(b) of one column whose scratch is laid out at `base`.
// ev: five events recorded before Step 1, after the sort, after the merge
// and the X_M directory (one kernel: both at its end), before the Step 2(b)
// kernel and at the end (nullptr: no timing).
dm_status run_column(dm_ctx* ctx, const dm_column_in* in, const dm_column_out* out, void* base,
                     cudaStream_t s, uint32_t flags, cudaEvent_t* ev, const dm::ReencodePlan* pre_plan = nullptr,
                     uint32_t grid_cap = 0, dm::ReencodePlan* plan_out = nullptr,
                     dm::ReencodeArgs* args_out = nullptr, const dm_tune_choice* force = nullptr) {
  const bool timing = ev != nullptr;
  ColumnScratch cs;
  carve_column(base, in, out, &cs);
  const uint32_t w = in->value_bytes;
  const uint64_t m = in->main_dict_len, d = in->delta_dict_len;
  const uint64_t n_out = in->main_rows + in->delta_rows;
  const Resolved rs = resolve(ctx, in, flags, force);

  // Step 2(b) launch plan first: it says whether Step 1 builds a directory
  dm::ReencodeArgs ra = plan_args(in, rs);
  ra.main_words = static_cast<const uint32_t*>(in->main_packed);
  ra.main_words_n = dm_packed_bytes(in->main_rows, in->main_bits) / 4;
  ra.dcodes = in->delta_codes;
  ra.xm = cs.xm;
  ra.xd = cs.xd;
  ra.d = (uint32_t)d;
  ra.d_bits = out->d_new_bits;
  ra.out_words = static_cast<uint32_t*>(out->new_packed);
  ra.status = ctx->status;
  ra.xdir = cs.xdir;
  ra.x8 = rs.x8 ? cs.x8 : nullptr;
  ra.gdir = cs.gdir;
  dm::ReencodePlan plan{};
  if (pre_plan) plan = *pre_plan;
  else if (n_out && dm::plan_reencode(in->main_bits, ra, ctx->sm_count, rs.flags, &plan) != cudaSuccess)
    return DM_ECUDA;
  if (rs.step1_blocks && (!grid_cap || rs.step1_blocks < grid_cap)) grid_cap = rs.step1_blocks;

  cudaError_t e = cudaMemsetAsync(cs.zero, 0, cs.zero_bytes, s);
  if (e != cudaSuccess) return DM_ECUDA;
  if (timing) cudaEventRecord(ev[0], s);
  if (m + d) {
    dm::Step1Args& a = cs.s1;
    a.phases = dm::S1_MERGE | (d ? dm::S1_SORT : 0u) | (plan.needs_directory ? dm::S1_DIR : 0u);
    a.unew = out->new_dict;
    a.d_u = out->d_new_dict_len;
    a.d_bits = out->d_new_bits;
    a.xdir = cs.xdir;
    a.x8 = plan.needs_directory ? ra.x8 : nullptr;
    a.dir_shift = plan.dir_shift;
    a.dir_entries = plan.dir_entries;
    a.status = ctx->status;
    a.grid_cap = grid_cap;
    a.spin_limit = ctx->test_spin_limit;
    a.test_withhold = ctx->test_withhold;
    e = dm::launch_step1(w, a, s, ctx->sm_count, &ctx->launches);
    if (e != cudaSuccess) ctx->last_error = e;
  } else {
    e = cudaMemsetAsync(out->d_new_dict_len, 0, sizeof(uint64_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(out->d_new_bits, 0, sizeof(uint32_t), s);
  }
  if (e != cudaSuccess) return DM_ECUDA;
  // the global directory (columns past the shared-memory directory's reach)
  // from the finished X_M
  e = dm::launch_gdir(plan, ra, s, &ctx->launches);
  if (e != cudaSuccess) {
    ctx->last_error = e;
    return DM_ECUDA;
  }
  if (timing) {
    cudaEventRecord(ev[1], s);
    cudaEventRecord(ev[2], s);
    cudaEventRecord(ev[3], s);
  }
  if (plan_out) {
    // the caller launches Step 2(b) itself (in chunks)
    *plan_out = plan;
    if (args_out) *args_out = ra;
    return DM_OK;
  }
  if (n_out) {
    e = dm::launch_reencode_planned(plan, ra, s, &ctx->launches);
    if (e != cudaSuccess) {
      ctx->last_error = e;
      return DM_ECUDA;
    }
  }
  if (timing) cudaEventRecord(ev[4], s);
  return DM_OK;
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

}  // namespace

size_t dm_table_scratch_bytes_for(const dm_column_in* in, uint32_t ncols, uint32_t flags, uint32_t branches) {
  size_t mx = 0;
  for (uint32_t c = 0; c < ncols; ++c) mx = std::max(mx, align_up(dm_scratch_bytes(&in[c], flags)));
  if (flags & DM_FLAG_SERIAL) return mx;
  return mx * std::max<uint32_t>(1, std::min(ncols, branches));
}

extern "C" {

const char* dm_last_error(const dm_ctx* ctx) {
  return ctx ? cudaGetErrorString(ctx->last_error) : "no context";
}

const char* dm_status_str(dm_status s) {
  switch (s) {
    case DM_OK: return "DM_OK";
    case DM_EINVAL: return "DM_EINVAL";
    case DM_ENOMEM: return "DM_ENOMEM";
    case DM_EUNSORTED: return "DM_EUNSORTED";
    case DM_ECODE: return "DM_ECODE";
    case DM_ECUDA: return "DM_ECUDA";
    case DM_ETIMEOUT: return "DM_ETIMEOUT";
    case DM_EBUSY: return "DM_EBUSY";
    case DM_ENOENT: return "DM_ENOENT";
    case DM_EINTERNAL: return "DM_EINTERNAL";
  }
  return "DM_UNKNOWN";
}

size_t dm_packed_bytes(uint64_t rows, uint32_t bits) { return (size_t)((rows * bits + 127) / 128) * 16; }

uint32_t dm_bits_for(uint64_t n) { return bits_for(n); }

uint32_t dm_max_bits(const dm_column_in* in) {
  return in ? bits_for(in->main_dict_len + in->delta_dict_len) : 0;
}

size_t dm_scratch_bytes(const dm_column_in* in, uint32_t) {
  if (!in) return 0;
  return carve_column(nullptr, in, nullptr, nullptr);
}

size_t dm_table_scratch_bytes(const dm_column_in* in, uint32_t ncols, uint32_t flags) {
  return dm_table_scratch_bytes_for(in, ncols, flags, dm_ctx::kTableBranches);
}

dm_status dm_create(dm_ctx** out, int device, size_t arena_bytes) {
  if (!out) return DM_EINVAL;
  *out = nullptr;
  dm_ctx* ctx = new (std::nothrow) dm_ctx();
  if (!ctx) return DM_ENOMEM;
  ctx->device = device;
  int sms = 0;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete ctx;
    return DM_ECUDA;
  }
  ctx->sm_count = (uint32_t)sms;
  if (cudaMalloc(&ctx->status, 256) != cudaSuccess) {
    delete ctx;
    return DM_ENOMEM;
  }
  cudaMemset(ctx->status, 0, 256);
  if (cudaMallocHost(&ctx->host_status, sizeof(uint32_t)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->copy_done, cudaEventDisableTiming) != cudaSuccess) {
    dm_destroy(ctx);
    return DM_ECUDA;
  }
  for (auto& e : ctx->ev) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      dm_destroy(ctx);
      return DM_ECUDA;
    }
  }
  bool ok = cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&ctx->d2h_stream, cudaStreamNonBlocking) == cudaSuccess;
  for (uint32_t i = 0; ok && i < dm_ctx::kChunks; ++i)
    ok = cudaEventCreateWithFlags(&ctx->h2d_done[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&ctx->comp_done[i], cudaEventDisableTiming) == cudaSuccess;
  for (uint32_t i = 0; ok && i < dm_ctx::kTableStreams; ++i)
    ok = cudaStreamCreateWithFlags(&ctx->side[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&ctx->join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    dm_destroy(ctx);
    return DM_ECUDA;
  }
  if (arena_bytes) {
    dm_status st = dm_reserve(ctx, arena_bytes);
    if (st != DM_OK) {
      dm_destroy(ctx);
      return st;
    }
  }
  *out = ctx;
  return DM_OK;
}

void dm_destroy(dm_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->arena && ctx->owns_arena) cudaFree(ctx->arena);
  if (ctx->status) cudaFree(ctx->status);
  if (ctx->host_status) cudaFreeHost(ctx->host_status);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->copy_done) cudaEventDestroy(ctx->copy_done);
  for (auto e : ctx->ev)
    if (e) cudaEventDestroy(e);
  for (auto& g : ctx->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (uint32_t i = 0; i < dm_ctx::kTableStreams; ++i) {
    if (ctx->side[i]) cudaStreamDestroy(ctx->side[i]);
    if (ctx->join[i]) cudaEventDestroy(ctx->join[i]);
  }
  if (ctx->fork) cudaEventDestroy(ctx->fork);
  if (ctx->capture) cudaStreamDestroy(ctx->capture);
  if (ctx->d2h_stream) cudaStreamDestroy(ctx->d2h_stream);
  for (uint32_t i = 0; i < dm_ctx::kChunks; ++i) {
    if (ctx->h2d_done[i]) cudaEventDestroy(ctx->h2d_done[i]);
    if (ctx->comp_done[i]) cudaEventDestroy(ctx->comp_done[i]);
  }
  if (ctx->ring) {
    for (uint32_t i = 0; i < 5 * dm_ctx::kRing; ++i)
      if (ctx->ring[i]) cudaEventDestroy(ctx->ring[i]);
    delete[] ctx->ring;
  }
  delete ctx;
}

dm_status dm_reserve(dm_ctx* ctx, size_t bytes) {
  if (!ctx) return DM_EINVAL;
  if (bytes <= ctx->arena_bytes) return DM_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DM_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return DM_ECUDA;
  if (ctx->arena && ctx->owns_arena) cudaFree(ctx->arena);
  ctx->arena = nullptr;
  ctx->arena_bytes = 0;
  ctx->owns_arena = true;
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return DM_ENOMEM;
  }
  ctx->arena = p;
  ctx->arena_bytes = bytes;
  return DM_OK;
}

size_t dm_arena_bytes(const dm_ctx* ctx) { return ctx ? ctx->arena_bytes : 0; }

}  // extern "C"

void dm_ctx_use_region(dm_ctx* ctx, void* ptr, size_t bytes) {
  if (ctx->arena && ctx->owns_arena) cudaFree(ctx->arena);
  ctx->arena = ptr;
  ctx->arena_bytes = bytes;
  ctx->owns_arena = false;
}

extern "C" {

uint64_t dm_launch_count(const dm_ctx* ctx) { return ctx ? ctx->launches : 0; }

dm_status dm_merge_column(dm_ctx* ctx, const dm_column_in* in, const dm_column_out* out, void* stream,
                          uint32_t flags) {
  if (!ctx) return DM_EINVAL;
  dm_status st = check_column(in, out, true);
  if (st != DM_OK) return st;
  if (dm_scratch_bytes(in, flags) > ctx->arena_bytes) return DM_ENOMEM;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DM_ECUDA;
  if ((flags & DM_FLAG_AUTOTUNE) && needs_tuning(ctx, in)) {
    st = dm_autotune_column(ctx, in, out, stream, flags, 0, nullptr);
    if (st != DM_OK) return st;
  }
  flags &= ~DM_FLAG_AUTOTUNE;
  const bool timing = (flags & DM_FLAG_TIMING) != 0;
  if (timing && !ctx->ring) {
    ctx->ring = new (std::nothrow) cudaEvent_t[5 * dm_ctx::kRing]();
    if (!ctx->ring) return DM_ENOMEM;
    for (uint32_t i = 0; i < 5 * dm_ctx::kRing; ++i)
      if (cudaEventCreate(&ctx->ring[i]) != cudaSuccess) return DM_ECUDA;
  }
  cudaEvent_t* ev = nullptr;
  if (timing) ev = ctx->ring_n < dm_ctx::kRing ? ctx->ring + 5 * ctx->ring_n : ctx->ev;
  st = run_column(ctx, in, out, ctx->arena, as_stream(stream), flags, ev);
  ctx->timing_valid = timing && st == DM_OK;
  if (ctx->timing_valid) {
    ctx->last_ev = ev;
    if (ev != ctx->ev) ++ctx->ring_n;
  }
  return st;
}

namespace {

// Launch plans of a table's Step 2(b) kernels, made before any launch (their
// attribute and occupancy queries must stay out of a stream capture).
bool plan_table(dm_ctx* ctx, const dm_column_in* in, uint32_t ncols, uint32_t flags,
                std::vector<dm::ReencodePlan>* plans) {
  if (dm::step1_prepare() != cudaSuccess) return false;
  plans->assign(ncols, dm::ReencodePlan{});
  for (uint32_t c = 0; c < ncols; ++c) {
    if (in[c].main_rows + in[c].delta_rows == 0) continue;
    const Resolved rs = resolve(ctx, &in[c], flags, nullptr);
    dm::ReencodeArgs ra = plan_args(&in[c], rs);
    ra.xdir = reinterpret_cast<uint32_t*>(16);   // a directory will exist
    if (dm::reencode_gdir_entries(in[c].main_dict_len, in[c].delta_dict_len)) ra.gdir = reinterpret_cast<uint2*>(16);
    if (dm::plan_reencode(in[c].main_bits, ra, ctx->sm_count, rs.flags, &(*plans)[c]) != cudaSuccess) return false;
  }
  return true;
}

// Record the batched schedule of a table on `s` (capturing, or live): columns
// round-robin over the side streams, each stream with its own scratch.
dm_status record_table(dm_ctx* ctx, const dm_column_in* in, uint32_t ncols, const dm_column_out* out,
                       cudaStream_t s, uint32_t flags, const std::vector<dm::ReencodePlan>& plans, uint32_t S,
                       size_t region) {
  if (cudaEventRecord(ctx->fork, s) != cudaSuccess) return DM_ECUDA;
  for (uint32_t i = 0; i < S; ++i)
    if (cudaStreamWaitEvent(ctx->side[i], ctx->fork, 0) != cudaSuccess) return DM_ECUDA;
  for (uint32_t c = 0; c < ncols; ++c) {
    const uint32_t i = c % S;
    const uint32_t cap = dm::step1_capacity(in[c].value_bytes, ctx->sm_count) / (S * ctx->coop_share);
    void* base = static_cast<char*>(ctx->arena) + (size_t)i * region;
    dm_status st = run_column(ctx, &in[c], &out[c], base, ctx->side[i], flags, nullptr, &plans[c], cap ? cap : 1);
    if (st != DM_OK) return st;
  }
  for (uint32_t i = 0; i < S; ++i) {
    if (cudaEventRecord(ctx->join[i], ctx->side[i]) != cudaSuccess) return DM_ECUDA;
    if (cudaStreamWaitEvent(s, ctx->join[i], 0) != cudaSuccess) return DM_ECUDA;
  }
  return DM_OK;
}

}  // namespace

namespace {

// Median milliseconds of `reps` batched merges of a table (after one more
// that records its graph), from CUDA events on the stream.
dm_status time_table(dm_ctx* ctx, const dm_column_in* in, uint32_t ncols, const dm_column_out* out, void* stream,
                     uint32_t flags, uint32_t reps, float* ms) {
  cudaStream_t s = as_stream(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return DM_ECUDA;
  }
  std::vector<float> t;
  dm_status st = DM_OK;
  for (uint32_t r = 0; r <= reps && st == DM_OK; ++r) {
    if (cudaEventRecord(e0, s) != cudaSuccess) st = DM_ECUDA;
    if (st == DM_OK) st = dm_merge_table(ctx, in, ncols, out, stream, flags);
    if (st == DM_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
      st = DM_ECUDA;
    float x = 0;
    if (st == DM_OK && r && cudaEventElapsedTime(&x, e0, e1) != cudaSuccess) st = DM_ECUDA;
    if (st == DM_OK && r) t.push_back(x);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DM_OK) return st;
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return DM_OK;
}

// The classes just tuned were timed one column at a time; inside the
// table's graph columns run side by side, where another choice may win.
// Keep their tuned choices only if the whole table runs faster with them
// than with the library defaults; otherwise store the defaults for them
// (so they are not tuned again).
dm_status confirm_in_table(dm_ctx* ctx, const dm_column_in* in, uint32_t ncols, const dm_column_out* out,
                           void* stream, uint32_t flags, const std::vector<dm_tune_key>& tuned) {
  constexpr uint32_t kReps = 5;
  std::vector<dm_tune_choice> chosen(tuned.size());
  for (size_t i = 0; i < tuned.size(); ++i)
    if (dm_tune_cache_get(ctx->tune_cache, &tuned[i], &chosen[i]) != DM_OK) return DM_EINVAL;
  float with_tuned = 0, with_defaults = 0;
  dm_status st = time_table(ctx, in, ncols, out, stream, flags, kReps, &with_tuned);
  const dm_tune_choice defaults{};
  for (size_t i = 0; i < tuned.size() && st == DM_OK; ++i) st = dm_tune_cache_put(ctx->tune_cache, &tuned[i], &defaults);
  if (st == DM_OK) st = time_table(ctx, in, ncols, out, stream, flags, kReps, &with_defaults);
  if (st != DM_OK || with_tuned < with_defaults)
    for (size_t i = 0; i < tuned.size(); ++i) dm_tune_cache_put(ctx->tune_cache, &tuned[i], &chosen[i]);
  return st;
}

}  // namespace

dm_status dm_merge_table(dm_ctx* ctx, const dm_column_in* in, uint32_t ncols, const dm_column_out* out,
                         void* stream, uint32_t flags) {
  if (!ctx || (ncols && (!in || !out))) return DM_EINVAL;
  for (uint32_t c = 0; c < ncols; ++c) {
    dm_status st = check_column(&in[c], &out[c], true);
    if (st != DM_OK) return st;
  }
  // one column's scratch at least; the batched schedule runs as many
  // branches as the arena holds regions (up to the tuned or default count)
  if (dm_table_scratch_bytes_for(in, ncols, flags | DM_FLAG_SERIAL, 1) > ctx->arena_bytes) return DM_ENOMEM;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DM_ECUDA;
  cudaStream_t s = as_stream(stream);
  ctx->timing_valid = false;
  if (ncols == 0) return DM_OK;
  if (flags & DM_FLAG_AUTOTUNE) {
    // each class once, on its first column (the merges below overwrite the
    // outputs the tuning merges leave)
    const uint32_t tf = flags & ~(DM_FLAG_AUTOTUNE | DM_FLAG_SERIAL | DM_FLAG_TIMING);
    std::vector<dm_tune_key> tuned;
    for (uint32_t c = 0; c < ncols; ++c) {
      if (!needs_tuning(ctx, &in[c])) continue;
      dm_status st = dm_autotune_column(ctx, &in[c], &out[c], stream, tf, 0, nullptr);
      if (st != DM_OK) return st;
      tuned.push_back(dm::tune_key_of(in[c]));
    }
    flags &= ~DM_FLAG_AUTOTUNE;
    if (!tuned.empty() && !(flags & DM_FLAG_SERIAL)) {
      dm_status st = confirm_in_table(ctx, in, ncols, out, stream, flags, tuned);
      if (st != DM_OK) return st;
    }
  }
  if (flags & DM_FLAG_SERIAL) {
    // columns one after another on one stream, reusing one scratch region
    for (uint32_t c = 0; c < ncols; ++c) {
      dm_status st = run_column(ctx, &in[c], &out[c], ctx->arena, s, flags, nullptr);
      if (st != DM_OK) return st;
    }
    return DM_OK;
  }

  // batched: one CUDA graph holds every column's kernels on a few branches
  // (each with its own scratch region); it is recorded once per distinct
  // argument set and replayed
  size_t region = 0;
  for (uint32_t c = 0; c < ncols; ++c) region = std::max(region, align_up(dm_scratch_bytes(&in[c], flags)));
  uint32_t S = ctx->tuning.table_branches ? ctx->tuning.table_branches : dm_ctx::kTableBranches;
  if (region && ctx->arena_bytes / region < S) S = (uint32_t)(ctx->arena_bytes / region);
  S = std::max<uint32_t>(1, std::min<uint32_t>(S, ncols));
  if (flags & DM_FLAG_NO_GRAPH) {
    // the same schedule, issued on the branches' streams directly
    std::vector<dm::ReencodePlan> plans;
    if (!plan_table(ctx, in, ncols, flags, &plans)) return DM_ECUDA;
    return record_table(ctx, in, ncols, out, s, flags, plans, S, region);
  }
  std::string key;
  key.reserve(64 + ncols * (sizeof(dm_column_in) + sizeof(dm_column_out)));
  auto put = [&key](const void* p, size_t n) { key.append(static_cast<const char*>(p), n); };
  put(&ncols, sizeof(ncols));
  put(&flags, sizeof(flags));
  put(&ctx->arena, sizeof(ctx->arena));
  put(&ctx->tuning, sizeof(ctx->tuning));
  put(&ctx->coop_share, sizeof(ctx->coop_share));
  put(&ctx->test_spin_limit, sizeof(ctx->test_spin_limit));
  put(&ctx->test_withhold, sizeof(ctx->test_withhold));
  const uint64_t tune_gen = dm_tune_cache_generation(ctx->tune_cache);
  put(&ctx->tune_cache, sizeof(ctx->tune_cache));
  put(&tune_gen, sizeof(tune_gen));
  for (uint32_t c = 0; c < ncols; ++c) {
    put(&in[c], sizeof(dm_column_in));
    put(&out[c], sizeof(dm_column_out));
  }
  ++ctx->graph_clock;
  for (auto& g : ctx->graphs) {
    if (g.key == key) {
      g.last_use = ctx->graph_clock;
      ctx->launches += g.launches;
      const cudaError_t le = cudaGraphLaunch(g.exec, s);
      if (le != cudaSuccess) ctx->last_error = le;
      return le == cudaSuccess ? DM_OK : DM_ECUDA;
    }
  }
  // plan every launch before recording (attribute and occupancy queries
  // stay out of the capture)
  std::vector<dm::ReencodePlan> plans;
  if (!plan_table(ctx, in, ncols, flags, &plans)) return DM_ECUDA;
  const uint64_t launches0 = ctx->launches;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    ctx->last_error = e;
    return DM_ECUDA;
  }
  dm_status st = record_table(ctx, in, ncols, out, ctx->capture, flags, plans, S, region);
  e = cudaStreamEndCapture(ctx->capture, &graph);
  if (st != DM_OK || e != cudaSuccess) {
    if (e != cudaSuccess) ctx->last_error = e;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return st != DM_OK ? st : DM_ECUDA;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    ctx->last_error = e;
    return DM_ECUDA;
  }
  dm_ctx::GraphEntry ent;
  ent.key = std::move(key);
  ent.exec = exec;
  ent.launches = ctx->launches - launches0;
  ent.last_use = ctx->graph_clock;
  if (ctx->graphs.size() >= 8) {
    auto lru = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                [](const auto& a, const auto& b) { return a.last_use < b.last_use; });
    cudaGraphExecDestroy(lru->exec);
    ctx->graphs.erase(lru);
  }
  ctx->graphs.push_back(std::move(ent));
  e = cudaGraphLaunch(exec, s);
  if (e != cudaSuccess) ctx->last_error = e;
  return e == cudaSuccess ? DM_OK : DM_ECUDA;
}

size_t dm_host_scratch_bytes(const dm_column_in* in, uint32_t flags) {
  if (!in) return 0;
  const uint32_t w = in->value_bytes;
  const uint64_t m = in->main_dict_len, d = in->delta_dict_len;
  const uint64_t n_out = in->main_rows + in->delta_rows;
  size_t b = 0;
  b += align_up(m * w) + align_up(dm_packed_bytes(in->main_rows, in->main_bits));
  b += align_up(d * w) + align_up(in->delta_rows * 4);
  b += align_up((m + d) * w) + align_up(dm_packed_bytes(n_out, bits_for(m + d)));
  b += align_up(m * 4) + align_up(d * 4) + align_up(16);
  return b + dm_scratch_bytes(in, flags);
}

dm_status dm_merge_column_host(dm_ctx* ctx, const dm_column_in* in, const dm_column_out* out, void* stream,
                               uint32_t flags, uint64_t* new_dict_len, uint32_t* new_bits) {
  if (!ctx || !new_dict_len || !new_bits) return DM_EINVAL;
  dm_status st = check_column(in, out, false);
  if (st != DM_OK) return st;
  if (dm_host_scratch_bytes(in, flags) > ctx->arena_bytes) return DM_ENOMEM;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DM_ECUDA;
  cudaStream_t s = as_stream(stream);
  const uint32_t w = in->value_bytes;
  const uint64_t m = in->main_dict_len, d = in->delta_dict_len;
  const uint64_t n_out = in->main_rows + in->delta_rows;
  const size_t main_bytes = dm_packed_bytes(in->main_rows, in->main_bits);

  Carver c(ctx->arena);
  dm_column_in din = *in;
  dm_column_out dout{};
  void* p_main_dict = c.take(m * w);
  void* p_main = c.take(main_bytes);
  void* p_ddict = c.take(d * w);
  void* p_dcodes = c.take(in->delta_rows * 4);
  dout.new_dict = c.take((m + d) * w);
  dout.new_packed = c.take(dm_packed_bytes(n_out, bits_for(m + d)));
  dout.x_main = static_cast<uint32_t*>(c.take(m * 4));
  dout.x_delta = static_cast<uint32_t*>(c.take(d * 4));
  char* scal = static_cast<char*>(c.take(16));
  dout.d_new_dict_len = reinterpret_cast<uint64_t*>(scal);
  dout.d_new_bits = reinterpret_cast<uint32_t*>(scal + 8);
  void* scratch = c.take(0);
  din.main_dict = p_main_dict;
  din.main_packed = p_main;
  din.delta_dict = p_ddict;
  din.delta_codes = static_cast<const uint32_t*>(p_dcodes);

  cudaError_t e = cudaSuccess;
  // On any failure the side streams are drained first: the caller's host
  // buffers are free again once this call returns.
  auto fail = [&](cudaError_t err, dm_status code) {
    if (err != cudaSuccess) ctx->last_error = err;
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamSynchronize(ctx->d2h_stream);
    cudaStreamSynchronize(s);
    return code;
  };
  // The main vector goes up in chunks of whole 1024-row tiles on the copy
  // stream from the start (overlapping Steps 1(a), 1(b)); each chunk is
  // re-encoded as soon as it has landed and its output comes back on a
  // third stream while later chunks are still being uploaded or encoded.
  const uint64_t nm = in->main_rows;
  uint32_t K = ctx->tuning.host_chunks ? ctx->tuning.host_chunks : dm_ctx::kDefaultChunks;
  uint64_t per = ((nm + K - 1) / K + 1023) / 1024 * 1024;
  if (per == 0) per = 1024;
  K = (uint32_t)std::max<uint64_t>(1, (nm + per - 1) / per);
  auto chunk_lo = [&](uint32_t k) { return std::min<uint64_t>(nm, (uint64_t)k * per); };
  auto chunk_hi = [&](uint32_t k) { return k + 1 == K ? nm : std::min<uint64_t>(nm, (uint64_t)(k + 1) * per); };
  const uint32_t b = in->main_bits;

  if (m) e = cudaMemcpyAsync(p_main_dict, in->main_dict, m * w, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && d) e = cudaMemcpyAsync(p_ddict, in->delta_dict, d * w, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && in->delta_rows)
    e = cudaMemcpyAsync(p_dcodes, in->delta_codes, in->delta_rows * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->copy_done, s);   // later streams start after earlier work on s
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_done, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->d2h_stream, ctx->copy_done, 0);
  for (uint32_t k = 0; e == cudaSuccess && k < K; ++k) {
    const uint64_t w0 = chunk_lo(k) * b / 32;
    const uint64_t w1 = k + 1 == K ? main_bytes / 4 : chunk_hi(k) * b / 32;
    if (w1 > w0)
      e = cudaMemcpyAsync(static_cast<uint32_t*>(p_main) + w0, static_cast<const uint32_t*>(in->main_packed) + w0,
                          (w1 - w0) * 4, cudaMemcpyHostToDevice, ctx->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->h2d_done[k], ctx->copy_stream);
  }
  if (e != cudaSuccess) return fail(e, DM_ECUDA);

  // Steps 1(a), 1(b), 2(a) and the X_M directory (one kernel) on s
  dm::ReencodePlan plan{};
  dm::ReencodeArgs ra{};
  st = run_column(ctx, &din, &dout, scratch, s, flags, nullptr, nullptr, 0, &plan, &ra);
  if (st != DM_OK) return fail(cudaSuccess, st);
  // the new width fixes where each chunk's output starts: read it back
  uint64_t hs[2] = {0, 0};
  e = cudaMemcpyAsync(hs, scal, 16, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(e, DM_ECUDA);
  const uint64_t u = hs[0];
  const uint32_t bn = (uint32_t)(hs[1] & 0xFFFFFFFFu);
  if (u > m + d || bn > 32) return fail(cudaSuccess, DM_ETIMEOUT);
  *new_dict_len = u;
  *new_bits = bn;
  if (u) e = cudaMemcpyAsync(out->new_dict, dout.new_dict, u * w, cudaMemcpyDeviceToHost, ctx->d2h_stream);
  if (e == cudaSuccess && out->x_main && m)
    e = cudaMemcpyAsync(out->x_main, dout.x_main, m * 4, cudaMemcpyDeviceToHost, ctx->d2h_stream);
  if (e == cudaSuccess && out->x_delta && d)
    e = cudaMemcpyAsync(out->x_delta, dout.x_delta, d * 4, cudaMemcpyDeviceToHost, ctx->d2h_stream);

  const uint64_t out_words_total = dm_packed_bytes(n_out, bn) / 4;
  for (uint32_t k = 0; e == cudaSuccess && n_out && k < K; ++k) {
    const uint64_t r0 = chunk_lo(k), r1 = chunk_hi(k);
    const bool last = k + 1 == K;
    dm::ReencodeArgs rc = ra;
    rc.main_words = ra.main_words + r0 * b / 32;
    rc.main_words_n = (last ? main_bytes / 4 : r1 * b / 32) - r0 * b / 32;
    rc.n_main = r1 - r0;
    rc.n_delta = last ? in->delta_rows : 0;
    rc.out_words = ra.out_words + r0 * bn / 32;
    if (rc.n_main + rc.n_delta == 0) continue;
    e = cudaStreamWaitEvent(s, ctx->h2d_done[k], 0);
    if (e == cudaSuccess) e = dm::launch_reencode_planned(plan, rc, s, &ctx->launches);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->comp_done[k], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->d2h_stream, ctx->comp_done[k], 0);
    const uint64_t o0 = r0 * bn / 32, o1 = last ? out_words_total : r1 * bn / 32;
    if (e == cudaSuccess && bn && o1 > o0)
      e = cudaMemcpyAsync(static_cast<uint32_t*>(out->new_packed) + o0, ra.out_words + o0, (o1 - o0) * 4,
                          cudaMemcpyDeviceToHost, ctx->d2h_stream);
  }
  if (e != cudaSuccess) return fail(e, DM_ECUDA);
  e = cudaStreamSynchronize(ctx->d2h_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->copy_stream);
  if (e != cudaSuccess) return fail(e, DM_ECUDA);
  return DM_OK;
}

dm_status dm_sort_delta(dm_ctx* ctx, uint32_t w, const void* delta_dict, uint64_t d, void* ud_out,
                        uint32_t* perm_out, void* stream) {
  if (!ctx || !width_ok(w) || d >= (1ull << 30)) return DM_EINVAL;
  if (d == 0) return DM_OK;
  const size_t ka = w;
  if (!delta_dict || !ud_out || !perm_out || !aligned(delta_dict, ka) || !aligned(ud_out, ka)) return DM_EINVAL;
  dm_column_in in{};
  in.value_bytes = w;
  in.delta_dict = delta_dict;
  in.delta_dict_len = d;
  if (dm_scratch_bytes(&in, 0) > ctx->arena_bytes) return DM_ENOMEM;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DM_ECUDA;
  cudaStream_t s = as_stream(stream);
  ColumnScratch cs;
  carve_column(ctx->arena, &in, nullptr, &cs);
  if (cudaMemsetAsync(cs.zero, 0, cs.zero_bytes, s) != cudaSuccess) return DM_ECUDA;
  cs.s1.phases = dm::S1_SORT;
  cs.s1.status = ctx->status;
  cs.s1.spin_limit = ctx->test_spin_limit;
  if (dm::launch_step1(w, cs.s1, s, ctx->sm_count, &ctx->launches) != cudaSuccess) return DM_ECUDA;
  return cuda_status(dm::launch_sort_copy_out(w, cs.slots, d, ud_out, perm_out, s, &ctx->launches));
}

dm_status dm_merge_dicts(dm_ctx* ctx, uint32_t w, const void* main_dict, uint64_t m, const void* ud,
                         const uint32_t* perm, uint64_t d, void* new_dict, uint32_t* x_main, uint32_t* x_delta,
                         uint64_t* d_u, uint32_t* d_bits, void* stream) {
  if (!ctx || !width_ok(w) || m + d > (1ull << 32) || !d_u || !d_bits) return DM_EINVAL;
  if ((m && (!main_dict || !x_main)) || (d && (!ud || !perm || !x_delta)) || (m + d && !new_dict)) return DM_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DM_ECUDA;
  cudaStream_t s = as_stream(stream);
  if (m + d == 0) {
    if (cudaMemsetAsync(d_u, 0, 8, s) != cudaSuccess || cudaMemsetAsync(d_bits, 0, 4, s) != cudaSuccess)
      return DM_ECUDA;
    return DM_OK;
  }
  const size_t zb = (size_t)dm::step1_zeroed_words(w, m + d, 0) * 4;
  if (align_up(zb) > ctx->arena_bytes) return DM_ENOMEM;
  uint32_t* zero = static_cast<uint32_t*>(ctx->arena);
  if (cudaMemsetAsync(zero, 0, zb, s) != cudaSuccess) return DM_ECUDA;
  dm::Step1Args a{};
  dm::step1_layout(w, m + d, 0, zero, &a);
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
  a.status = ctx->status;
  a.spin_limit = ctx->test_spin_limit;
  a.test_withhold = ctx->test_withhold;
  return cuda_status(dm::launch_step1(w, a, s, ctx->sm_count, &ctx->launches));
}

dm_status dm_reencode(dm_ctx* ctx, const uint32_t* main_packed, uint32_t main_bits, uint64_t n_main,
                      const uint32_t* delta_codes, uint64_t n_delta, const uint32_t* x_main, uint64_t m,
                      const uint32_t* x_delta, uint64_t d, const uint32_t* d_bits, uint32_t max_bits,
                      uint32_t* out_packed, void* stream, uint32_t flags) {
  if (!ctx || main_bits > 32 || max_bits > 32 || !d_bits || m > 0xFFFFFFFFull || d > 0xFFFFFFFFull)
    return DM_EINVAL;
  if ((n_main && (!m || !x_main || (main_bits && (!main_packed || !aligned(main_packed, 16))))) ||
      (n_delta && (!d || !x_delta || !delta_codes)))
    return DM_EINVAL;
  if (n_main + n_delta && max_bits && (!out_packed || !aligned(out_packed, 16))) return DM_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DM_ECUDA;
  dm::ReencodeArgs ra{};
  ra.main_words = main_packed;
  ra.main_words_n = dm_packed_bytes(n_main, main_bits) / 4;
  ra.n_main = n_main;
  ra.dcodes = delta_codes;
  ra.n_delta = n_delta;
  ra.xm = x_main;
  ra.m = (uint32_t)m;
  ra.xd = x_delta;
  ra.d = (uint32_t)d;
  ra.d_bits = d_bits;
  ra.max_bits = max_bits;
  ra.out_words = out_packed;
  ra.status = ctx->status;
  // the X_M directory goes to the arena when it has room (else no
  // directory), its byte table after it when that fits too
  // (the refined directory's room when the arena has it, else the unrefined)
  size_t dir_bytes = (size_t)dm::reencode_dir_words(m) * 4;
  if (ctx->arena_bytes < dir_bytes) dir_bytes = (size_t)dm::reencode_dir_words(0) * 4;
  ra.xdir = ctx->arena_bytes >= dir_bytes ? static_cast<uint32_t*>(ctx->arena) : nullptr;
  ra.xdir_words = (uint32_t)(dir_bytes / 4);
  ra.x8 = ra.xdir && dm::reencode_wants_x8(m) && ctx->arena_bytes >= dir_bytes + m
              ? static_cast<uint8_t*>(ctx->arena) + dir_bytes
              : nullptr;
  // or, past the shared-memory directory's reach, the global directory
  const size_t gdir_bytes = (size_t)dm::reencode_gdir_entries(m, d) * sizeof(uint2);
  ra.gdir = gdir_bytes && n_main && ctx->arena_bytes >= dir_bytes + gdir_bytes
                ? reinterpret_cast<uint2*>(static_cast<char*>(ctx->arena) + dir_bytes)
                : nullptr;
  ra.tune_warps = ctx->tuning.reencode_warps;
  ra.tune_stages = ctx->tuning.reencode_stages;
  ra.tune_obufs = ctx->tuning.reencode_obufs;
  return cuda_status(dm::launch_reencode(main_bits, ra, as_stream(stream), ctx->sm_count, flags, &ctx->launches));
}

dm_status dm_set_wait_test(dm_ctx* ctx, uint32_t withhold_tile, uint32_t spin_limit) {
  if (!ctx) return DM_EINVAL;
  ctx->test_withhold = withhold_tile == DM_WAIT_TEST_OFF ? 0u : withhold_tile + 1;
  ctx->test_spin_limit = spin_limit;
  return DM_OK;
}

dm_status dm_set_tuning(dm_ctx* ctx, const dm_tuning* t) {
  if (!ctx || !t) return DM_EINVAL;
  if (t->reencode_warps > 16 || (t->reencode_stages && (t->reencode_stages < 2 || t->reencode_stages > 4)) ||
      t->reencode_obufs > 2 || t->host_chunks > dm_ctx::kChunks || t->table_branches > dm_ctx::kTableStreams)
    return DM_EINVAL;
  ctx->tuning = *t;
  return DM_OK;
}

dm_status dm_get_tuning(const dm_ctx* ctx, dm_tuning* t) {
  if (!ctx || !t) return DM_EINVAL;
  *t = ctx->tuning;
  return DM_OK;
}

dm_status dm_set_tune_cache(dm_ctx* ctx, dm_tune_cache* cache) {
  if (!ctx) return DM_EINVAL;
  ctx->tune_cache = cache ? cache : &ctx->own_cache;
  return DM_OK;
}

dm_tune_cache* dm_get_tune_cache(dm_ctx* ctx) { return ctx ? ctx->tune_cache : nullptr; }

uint32_t dm_tune_candidates(const dm_ctx* ctx, const dm_column_in* in, dm_tune_choice* out, uint32_t cap) {
  if (!ctx || !in) return 0;
  const std::vector<dm_tune_choice> v = tune_candidates(ctx, in);
  for (uint32_t i = 0; i < cap && i < v.size() && out; ++i) out[i] = v[i];
  return (uint32_t)v.size();
}

dm_status dm_autotune_column(dm_ctx* ctx, const dm_column_in* in, const dm_column_out* out, void* stream,
                             uint32_t flags, uint32_t reps, dm_tune_report* report) {
  if (!ctx) return DM_EINVAL;
  dm_status st = check_column(in, out, true);
  if (st != DM_OK) return st;
  if (dm_scratch_bytes(in, flags) > ctx->arena_bytes) return DM_ENOMEM;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DM_ECUDA;
  if (reps == 0) reps = 5;
  if (reps > 1000) return DM_EINVAL;
  flags &= ~(DM_FLAG_AUTOTUNE | DM_FLAG_SERIAL | DM_FLAG_TIMING | DM_FLAG_X_SMEM | DM_FLAG_X_GLOBAL);
  cudaStream_t s = as_stream(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return DM_ECUDA;
  }
  uint32_t timed = 0;
  // median of `reps` merges after one untimed merge
  auto measure = [&](const dm_tune_choice& c, float* ms) -> dm_status {
    std::vector<float> t;
    for (uint32_t r = 0; r <= reps; ++r) {
      if (cudaEventRecord(e0, s) != cudaSuccess) return DM_ECUDA;
      dm_status rs = run_column(ctx, in, out, ctx->arena, s, flags, nullptr, nullptr, 0, nullptr, nullptr, &c);
      if (rs != DM_OK) return rs;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return DM_ECUDA;
      float x = 0;
      if (r && cudaEventElapsedTime(&x, e0, e1) != cudaSuccess) return DM_ECUDA;
      if (r) t.push_back(x);
    }
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    ++timed;
    return DM_OK;
  };
  const std::vector<dm_tune_choice> all = tune_candidates(ctx, in);
  dm_tune_choice best{};
  float best_ms = 0, default_ms = 0;
  st = measure(best, &default_ms);
  best_ms = default_ms;
  std::vector<dm_tune_choice> tried = {best};   // each choice is timed once
  // one axis at a time, each over the values the candidate list holds,
  // the other fields held at the best so far
  auto axis = [&](auto field) -> dm_status {
    for (const dm_tune_choice& c : all) {
      dm_tune_choice t = best;
      field(t, c);
      bool seen = false;
      for (const auto& u : tried) seen = seen || memcmp(&u, &t, sizeof(t)) == 0;
      if (seen) continue;
      tried.push_back(t);
      float ms = 0;
      dm_status rs = measure(t, &ms);
      if (rs != DM_OK) return rs;
      if (ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
    return DM_OK;
  };
  if (st == DM_OK)
    st = axis([](dm_tune_choice& t, const dm_tune_choice& c) {
      t.x_staging = c.x_staging;
      t.x8 = c.x8;
    });
  if (st == DM_OK)
    st = axis([](dm_tune_choice& t, const dm_tune_choice& c) {
      t.reencode_warps = c.reencode_warps;
      t.reencode_stages = c.reencode_stages;
      t.reencode_obufs = c.reencode_obufs;
    });
  if (st == DM_OK) st = axis([](dm_tune_choice& t, const dm_tune_choice& c) { t.step1_blocks = c.step1_blocks; });
  // leave the result of the chosen launch in `out`
  if (st == DM_OK) st = run_column(ctx, in, out, ctx->arena, s, flags, nullptr, nullptr, 0, nullptr, nullptr, &best);
  if (st == DM_OK && cudaStreamSynchronize(s) != cudaSuccess) st = DM_ECUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DM_OK) return st;
  const dm_tune_key key = dm::tune_key_of(*in);
  st = dm_tune_cache_put(ctx->tune_cache, &key, &best);
  if (st != DM_OK) return st;
  if (report) {
    *report = dm_tune_report{};
    report->key = key;
    report->best = best;
    report->best_ms = best_ms;
    report->default_ms = default_ms;
    report->candidates = timed;
    report->reps = reps;
  }
  return DM_OK;
}

dm_status dm_sync_status(dm_ctx* ctx, void* stream) {
  if (!ctx) return DM_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DM_ECUDA;
  cudaStream_t s = as_stream(stream);
  if (cudaMemcpyAsync(ctx->host_status, ctx->status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return DM_ECUDA;
  const uint32_t v = *ctx->host_status;
  if (v) {
    if (cudaMemsetAsync(ctx->status, 0, 4, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
      return DM_ECUDA;
  }
  if (v & dm::ST_TIMEOUT) return DM_ETIMEOUT;
  if (v & dm::ST_INTERNAL) return DM_EINTERNAL;
  if (v & dm::ST_UNSORTED) return DM_EUNSORTED;
  if (v & dm::ST_CODE) return DM_ECODE;
  if (v & dm::ST_WIDTH) return DM_EINVAL;
  return DM_OK;
}

static dm_status elapsed5(cudaEvent_t* ev, float ms[5]) {
  if (cudaEventSynchronize(ev[4]) != cudaSuccess) return DM_ECUDA;
  if (cudaEventElapsedTime(&ms[0], ev[0], ev[1]) != cudaSuccess ||
      cudaEventElapsedTime(&ms[1], ev[1], ev[2]) != cudaSuccess ||
      cudaEventElapsedTime(&ms[2], ev[2], ev[3]) != cudaSuccess ||
      cudaEventElapsedTime(&ms[3], ev[3], ev[4]) != cudaSuccess ||
      cudaEventElapsedTime(&ms[4], ev[0], ev[4]) != cudaSuccess)
    return DM_ECUDA;
  return DM_OK;
}

dm_status dm_last_timing(dm_ctx* ctx, float ms[5]) {
  if (!ctx || !ms || !ctx->timing_valid || !ctx->last_ev) return DM_EINVAL;
  return elapsed5(ctx->last_ev, ms);
}

dm_status dm_timing_sum(dm_ctx* ctx, float ms[5], uint32_t* calls) {
  if (!ctx || !ms || !calls) return DM_EINVAL;
  for (int k = 0; k < 5; ++k) ms[k] = 0.f;
  *calls = 0;
  for (uint32_t i = 0; i < ctx->ring_n; ++i) {
    float one[5];
    dm_status st = elapsed5(ctx->ring + 5 * i, one);
    if (st != DM_OK) return st;
    for (int k = 0; k < 5; ++k) ms[k] += one[k];
  }
  *calls = ctx->ring_n;
  ctx->ring_n = 0;
  ctx->timing_valid = false;
  ctx->last_ev = nullptr;
  return DM_OK;
}

}  // extern "C"
