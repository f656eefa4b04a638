// The context object behind the opaque dm_ctx handle (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dmerge.h"
#include "dm_tune.h"

struct dm_ctx {
  int device = 0;
  uint32_t sm_count = 0;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  uint32_t* status = nullptr;      // device status word
  uint32_t* host_status = nullptr; // pinned readback
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_done = nullptr;
  // host-buffer merges: main upload and result download in chunks
  static constexpr uint32_t kChunks = 32, kDefaultChunks = 8;
  cudaStream_t d2h_stream = nullptr;
  cudaEvent_t h2d_done[kChunks] = {};
  cudaEvent_t comp_done[kChunks] = {};
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  bool timing_valid = false;
  // ring of per-call event quadruples for dm_timing_sum
  static constexpr uint32_t kRing = 1024;
  cudaEvent_t* ring = nullptr;
  uint32_t ring_n = 0;
  cudaEvent_t* last_ev = nullptr;   // quadruple of the last timed call
  dm_tuning tuning{};
  dm_tune_cache own_cache;                // launch choices per column class
  dm_tune_cache* tune_cache = &own_cache; // or a cache shared with other contexts
  // batched table merges: side streams, fork/join events, graph cache
  // branches of a batched table merge: kTableBranches by default (the
  // arena dm_table_scratch_bytes asks for), at most kTableStreams, and no
  // more than the arena holds scratch regions
  static constexpr uint32_t kTableStreams = 8, kTableBranches = 8;
  cudaStream_t side[kTableStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kTableStreams] = {};
  struct GraphEntry {
    std::string key;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches = 0;   // kernels in the graph
    uint64_t last_use = 0;
  };
  std::vector<GraphEntry> graphs;
  uint64_t graph_clock = 0;
  cudaStream_t capture = nullptr;   // graphs are recorded here, never on a caller's stream
  cudaError_t last_error = cudaSuccess;
  bool owns_arena = true;           // false: the arena is a region lent by a server
  uint32_t coop_share = 1;          // cooperative Step 1 grids get capacity / (branches * coop_share)
  uint64_t launches = 0;
  // dm_set_wait_test: polls before a Step 1 wait gives up (0: the library's
  // limit) and the merge tile (plus one; 0: none) that withholds its
  // look-back word
  uint32_t test_spin_limit = 0;
  uint32_t test_withhold = 0;
};


// Lend a region of device memory to a context as its arena (not owned).
void dm_ctx_use_region(dm_ctx* ctx, void* ptr, size_t bytes);

// dm_table_scratch_bytes for a batched schedule of `branches` branches.
size_t dm_table_scratch_bytes_for(const dm_column_in* in, uint32_t ncols, uint32_t flags, uint32_t branches);
