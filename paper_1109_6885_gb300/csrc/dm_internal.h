// Host-side interfaces between the translation units of libdmerge.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dm {

// ---------------------------------------------------------------- Step 1
constexpr int RS_ITEMS = 4;       // keys per thread of a sort tile
constexpr int RS_TILE = 256 * RS_ITEMS;   // keys per sort tile
// Merged positions per merge tile (a 100M-row column's merge fits one wave
// of tiles at two blocks per SM); MG_TILE_MIN bounds the tile count.
constexpr uint32_t mg_tile(uint32_t) { return 4096u; }
constexpr uint32_t MG_TILE_MIN = 2048;
constexpr uint32_t S1_SORT = 1, S1_MERGE = 2, S1_DIR = 4;   // phases
constexpr uint32_t S1_BARRIERS = 32;                        // barrier counters per launch

struct Step1Args {
  // Step 1(a): sort of the delta dictionary
  const void* in_keys;       // D_dict (insertion order)
  uint64_t d;
  void* keys[2];             // ping-pong key buffers, d keys each
  uint32_t* vals[2];         // ping-pong insertion codes
  uint32_t* hist;            // [W][256] digit counts (zeroed)
  uint32_t* sort_lb;         // [W][sort_tiles][256] look-back words (zeroed)
  uint32_t sort_tiles;
  uint32_t hist_blocks;      // set by the launcher
  // two-level partition of a large sort (bins of the two most significant
  // varying bytes), laid out with the zeroed bookkeeping when d can use it,
  // else nullptr: bin counts, bin cursors, then the bins' offsets
  // (JOINT_BINS + 1 words) followed by the decision word
  uint32_t* jhist;
  uint32_t* jcur;
  uint32_t* joff;
  uint32_t jgroup;           // bins per group of the in-place group sorts (set by the launcher)
  void** final_slot;         // optional: [0] sorted keys, [1] perm (for copy-out)
  // Step 1(b) + 2(a): merge with the main dictionary
  const void* a;             // U_M
  uint64_t m;
  const void* b;             // U_D when the sort phase is off
  const uint32_t* perm;      // its insertion codes
  void* unew;
  uint32_t* xm;
  uint32_t* xd;
  uint64_t* d_u;
  uint32_t* d_bits;
  uint64_t* merge_lb;        // [merge_tiles] look-back words (zeroed)
  uint32_t merge_tiles;
  uint64_t* cuts;            // optional [merge_tiles + 1]: U_M co-ranks of the tile boundaries,
                             // computed up front when the merge takes several waves of tiles
  // directory of X_M for Step 2(b)
  uint32_t* xdir;
  uint32_t dir_shift;
  uint32_t dir_entries;
  uint8_t* x8;               // optional [m]: byte table for the directory's crowded buckets
  // control
  uint32_t phases;           // S1_SORT | S1_MERGE | S1_DIR
  uint32_t* barriers;        // [S1_BARRIERS] (zeroed)
  uint32_t* status;
  uint32_t grid_cap;         // 0: whole device; else at most this many blocks
  // bounded waits: polls of a look-back word or barrier before the wait
  // gives up (0: kSpinLimit); testing: merge tile test_withhold - 1 never
  // publishes its look-back word, so the waits of the tiles after it run
  // out (0: none)
  uint32_t spin_limit;
  uint32_t test_withhold;
};

// Set the Step 1 kernels' launch attributes (outside any stream capture).
cudaError_t step1_prepare();
// Blocks of one Step 1 launch that can be resident on the device at once.
uint32_t step1_capacity(uint32_t w, uint32_t sm_count);

uint32_t sort_tiles(uint64_t d);
constexpr uint32_t JOINT_BINS = 1u << 16;
// Delta sizes past which a top-byte partition cannot leave every bucket
// within the shared-memory sort: the two-level partition's scratch exists.
constexpr uint64_t JOINT_MIN_KEYS = 256ull * 2048;
uint32_t merge_tiles(uint64_t n, uint32_t w);
// 32-bit words of bookkeeping to zero before a Step 1 launch that merges
// n_merge dictionary entries and sorts d_sort keys of w bytes.
uint64_t step1_zeroed_words(uint32_t w, uint64_t n_merge, uint64_t d_sort);
// Place that bookkeeping (look-back words, barriers, histograms) at `zero`.
void step1_layout(uint32_t w, uint64_t n_merge, uint64_t d_sort, uint32_t* zero, Step1Args* a);
// One cooperative launch running the phases in a.phases.
cudaError_t launch_step1(uint32_t w, const Step1Args& a, cudaStream_t stream, uint32_t sm_count,
                         uint64_t* launches);
// Copies the sorted result named by final_slot into caller buffers.
cudaError_t launch_sort_copy_out(uint32_t w, void** final_slot, uint64_t d, void* ud_out,
                                 uint32_t* perm_out, cudaStream_t stream, uint64_t* launches);

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
  uint32_t* xdir;            // scratch for the X_M directory or NULL
  uint32_t xdir_words;       // words at xdir (0: reencode_dir_words(0), the unrefined maximum)
  uint8_t* x8;               // scratch for its byte table ([m]) or NULL
  uint2* gdir;               // scratch for the global directory (reencode_gdir_entries(m, d)) or NULL
  uint32_t tune_warps;       // 0 = default; warps per block
  uint32_t tune_stages;      // 0 = default; input stages per warp
  uint32_t tune_obufs;       // 0 = default; output buffers per warp
};

// Words of directory scratch a column of m main codes is given: room for the
// refined directory above 2^22 main codes, else the unrefined maximum.
uint32_t reencode_dir_words(uint64_t m);
// Most main codes a directory can cover (m above it: no directory, no byte table).
uint64_t reencode_dir_max_codes();
// Whether a column of m main codes gets the directory's byte table.
bool reencode_wants_x8(uint64_t m);
// Entries of the global directory of X_M for m main codes and d delta
// dictionary entries (0: none; m is within the shared-memory directory's
// reach, which serves it instead, or too large for one).
uint64_t reencode_gdir_entries(uint64_t m, uint64_t d);

// Host-side launch plan of Step 2(b) (opaque storage).
struct ReencodePlan {
  alignas(8) unsigned char storage[96];
  bool needs_directory;
  uint32_t dir_shift;
  uint32_t dir_entries;
  uint64_t gdir_entries;     // global directory to build before Step 2(b) (0: none)
};
cudaError_t plan_reencode(uint32_t b, const ReencodeArgs& a, uint32_t sm_count, uint32_t flags, ReencodePlan* out);
cudaError_t launch_xdir(const ReencodePlan& plan, const ReencodeArgs& a, cudaStream_t s, uint64_t* launches);
// The global directory of the plan, if it has one, built from the finished X_M.
cudaError_t launch_gdir(const ReencodePlan& plan, const ReencodeArgs& a, cudaStream_t s, uint64_t* launches);
cudaError_t launch_reencode_planned(const ReencodePlan& plan, const ReencodeArgs& a, cudaStream_t s,
                                    uint64_t* launches);
cudaError_t launch_reencode(uint32_t b, const ReencodeArgs& a, cudaStream_t stream,
                            uint32_t sm_count, uint32_t flags, uint64_t* launches);

}  // namespace dm
