// Host-side interfaces between the translation units of libdmerge.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dm {

// ---------------------------------------------------------------- Step 1(a)
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

struct SortArgs {
  const void* in_keys;       // D_dict (insertion order)
  uint64_t d;
  void* keys[2];             // ping-pong key buffers, d keys each
  uint32_t* vals[2];         // ping-pong insertion codes
  uint32_t* hist;            // [W][256] digit counts (zeroed)
  uint32_t* counters;        // [W] dynamic tile counters (zeroed)
  uint32_t* lookback;        // [W][ntiles][256] look-back words (zeroed)
  uint32_t ntiles;
  void** final_slot;         // device slots: [0] = sorted keys, [1] = perm
  uint32_t* status;
};

// Scratch words the sort needs zeroed (hist + counters + look-back).
uint64_t sort_zeroed_words(uint32_t w, uint64_t d);
uint32_t sort_tiles(uint64_t d);
// Launches histogram + one kernel per digit pass on `stream`.
cudaError_t launch_sort(uint32_t w, const SortArgs& a, cudaStream_t stream, uint32_t sm_count,
                        uint64_t* launches);
// Copies the sorted result named by final_slot into caller buffers.
cudaError_t launch_sort_copy_out(uint32_t w, void** final_slot, uint64_t d, void* ud_out,
                                 uint32_t* perm_out, cudaStream_t stream, uint64_t* launches);

// ---------------------------------------------------------------- Step 1(b) + 2(a)
constexpr int MG_THREADS = 256;
constexpr int MG_ITEMS = 8;
constexpr int MG_TILE = MG_THREADS * MG_ITEMS;

struct MergeArgs {
  const void* a;             // U_M
  uint64_t m;
  const void* b;             // U_D (used when b_slot is NULL)
  const uint32_t* perm;      // insertion codes of U_D (used when b_slot is NULL)
  void* const* b_slot;       // device slots written by the sort: [0] U_D, [1] perm
  uint64_t d;
  void* unew;
  uint32_t* xm;
  uint32_t* xd;
  uint64_t* d_u;
  uint32_t* d_bits;
  uint64_t* lookback;        // [ntiles] (zeroed)
  uint32_t* counter;         // tile counter (zeroed)
  uint32_t ntiles;
  uint32_t* status;
};

uint32_t merge_tiles(uint64_t n);
cudaError_t launch_merge(uint32_t w, const MergeArgs& a, cudaStream_t stream, uint64_t* launches);

// ---------------------------------------------------------------- Step 2(b)
struct ReencodeArgs {
  const uint32_t* main_words;
  uint64_t main_words_n;     // words in the main stream buffer
  uint64_t n_main;
  const uint32_t* dcodes;
  uint64_t n_delta;
  const uint32_t* xm;
  uint32_t m;
  const uint32_t* xd;
  uint32_t d;
  const uint32_t* d_bits;    // E'_C (device scalar)
  uint32_t max_bits;         // host bound of E'_C; sizes the output buffer
  uint32_t* out_words;
  uint32_t* status;
};

cudaError_t launch_reencode(uint32_t b, const ReencodeArgs& a, cudaStream_t stream,
                            uint32_t sm_count, uint32_t flags, uint64_t* launches);

}  // namespace dm
