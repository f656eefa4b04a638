/*
 * dmerge.h — C ABI of the GB300 delta-to-main merge (libdmerge.so).
 *
 * One column merge (Krueger et al., "Fast Updates on Read-Optimized
 * Databases Using Multi-Core CPUs", Section 5) combines
 *   - the main partition: a sorted, duplicate-free dictionary U_M and the
 *     vector M of N_M codes into it, bit-packed at E_C bits, and
 *   - the delta partition: N_D rows, stored as an insertion-order
 *     dictionary D_dict of the distinct delta values plus one uint32 code
 *     per row into D_dict,
 * into a new dictionary U' = sorted(U_M ∪ D_dict) without duplicates (Eq. 3)
 * and a new packed vector of N'_M = N_M + N_D codes (Eq. 2): the main rows
 * in order, then the delta rows in order, each holding the position of its
 * value in U', at E'_C = ceil(log2 |U'|) bits (Eq. 4).  The translation
 * tables X_M (old main code -> new code) and X_D (delta code -> new code)
 * of Section 5.3 are outputs too.
 *
 * Steps, each a set of sm_103a kernels:
 *   1(a)  sort D_dict                 -> U_D, perm   (a radix partition on
 *         the most significant varying byte, then a shared-memory sort of
 *         each bucket; stable LSD radix passes when a bucket would exceed
 *         2048 keys)
 *   1(b)  merge U_M with U_D, dedup   -> U', X_M, X_D (merge path + scan)
 *   2(a)  E'_C = ceil(log2 |U'|)      -> device scalar
 *   2(b)  re-encode M and D           -> new packed vector (Eq. 11)
 *
 * Formats (the paper fixes none; these are this library's):
 *   keys      unsigned integers of value_bytes = 4 (uint32), 8 (uint64) or
 *             16 ({uint64 hi; uint64 lo;}, hi first in memory, compared
 *             hi first).  Arrays aligned to value_bytes.
 *   packed    code i occupies stream bits [i*b, (i+1)*b), least significant
 *             bit first; stream bit k is bit k%32 of little-endian 32-bit
 *             word k/32.  A stream of n codes at b bits occupies
 *             dm_packed_bytes(n, b) bytes (a whole number of 16-byte units,
 *             zero after the last code).  Packed buffers are 16-byte aligned.
 *   b = 0     legal when the dictionary has at most one entry: every code
 *             is 0 and the stream has zero bytes.
 *   duplicates inside D_dict are tolerated: every copy maps to the value's
 *             single code in U'.  Dictionary entries no row references are
 *             kept (U' is the union of the dictionaries, Eq. 3).
 *
 * Conventions:
 *   - Every call is asynchronous on the given CUDA stream (a cudaStream_t
 *     passed as void*; NULL = the legacy default stream) unless it says
 *     otherwise.  Argument errors are returned immediately, before any
 *     launch.  Data-dependent errors (U_M not increasing, a code out of
 *     range, a wait that timed out) are recorded in a per-context device
 *     status word and returned by dm_sync_status.  Kernels never fault on
 *     such data: out-of-range codes are clamped and flagged.
 *   - Inputs are never written.  All pointers in dm_column_in /
 *     dm_column_out are device pointers owned by the caller; the library
 *     never frees them.  Scratch memory comes from the context's arena,
 *     sized at dm_create / dm_reserve; too small an arena returns DM_ENOMEM
 *     before any launch.
 *   - A context serves one stream at a time: calls on different streams
 *     that may overlap need different contexts.
 */
#ifndef DMERGE_H_
#define DMERGE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DM_OK = 0,
  DM_EINVAL = 1,     /* bad argument: width, size, alignment, NULL */
  DM_ENOMEM = 2,     /* the context's arena is too small (or allocation failed) */
  DM_EUNSORTED = 3,  /* U_M is not strictly increasing */
  DM_ECODE = 4,      /* a main code >= |U_M| or a delta code >= |D_dict| */
  DM_ECUDA = 5,      /* a CUDA runtime call failed */
  DM_ETIMEOUT = 6,   /* a bounded device-side wait gave up */
  DM_EBUSY = 7,      /* the request cannot be admitted now */
  DM_ENOENT = 8,     /* no such entry (tune cache lookup, missing file) */
  DM_EINTERNAL = 9   /* an internal consistency check on the device failed (a
                        write index out of range, a hash slot missing); the
                        call's outputs are not valid.  Not caused by the data. */
} dm_status;

/* flags for dm_merge_column / dm_merge_table */
#define DM_FLAG_GENERIC_REENCODE 0x1u  /* force the runtime-width Step 2(b) path */
#define DM_FLAG_X_SMEM 0x2u            /* look X_M up in shared memory at any size (table or directory) */
#define DM_FLAG_X_GLOBAL 0x4u          /* gather X_M directly: no shared-memory table or directory, no
                                          global directory */
#define DM_FLAG_TIMING 0x8u            /* record per-step CUDA events (dm_last_timing) */
#define DM_FLAG_SERIAL 0x10u           /* dm_merge_table: one column after another, plain launches */
#define DM_FLAG_NO_GRAPH 0x40u         /* dm_merge_table: the batched schedule issued directly on the
                                          branches' streams, not recorded into a graph (for callers
                                          whose buffers or scratch move between calls) */
#define DM_FLAG_AUTOTUNE 0x20u         /* dm_merge_column / dm_merge_table: first tune every column
                                          class missing from the tune cache (dm_autotune_column;
                                          blocks the host while it runs) */

typedef struct dm_ctx dm_ctx;
/* Launch choices per column class (see "autotuning" below). */
typedef struct dm_tune_cache dm_tune_cache;

/* Create a context on `device` with a scratch arena of arena_bytes (may be
 * 0; grow it later with dm_reserve).  Synchronous. */
dm_status dm_create(dm_ctx** ctx, int device, size_t arena_bytes);
void dm_destroy(dm_ctx* ctx);
/* Grow the arena to at least arena_bytes.  Synchronises the device. */
dm_status dm_reserve(dm_ctx* ctx, size_t arena_bytes);
size_t dm_arena_bytes(const dm_ctx* ctx);

/* One column's inputs (device pointers, read only). */
typedef struct {
  uint32_t value_bytes;        /* E: 4, 8 or 16 */
  const void* main_dict;       /* U_M, main_dict_len keys, strictly increasing */
  uint64_t main_dict_len;      /* |U_M| */
  const void* main_packed;     /* M: main_rows codes at main_bits bits */
  uint32_t main_bits;          /* E_C, 0..32, >= dm_bits_for(main_dict_len) */
  uint64_t main_rows;          /* N_M */
  const void* delta_dict;      /* D_dict, delta_dict_len keys, insertion order */
  uint64_t delta_dict_len;     /* |D_dict| (< 2^30) */
  const uint32_t* delta_codes; /* delta_rows codes, each < delta_dict_len */
  uint64_t delta_rows;         /* N_D */
} dm_column_in;

/* One column's outputs (caller-allocated device buffers). */
typedef struct {
  void* new_dict;              /* U': capacity main_dict_len + delta_dict_len keys */
  void* new_packed;            /* dm_packed_bytes(main_rows + delta_rows, dm_max_bits(in)) bytes */
  uint32_t* x_main;            /* X_M: main_dict_len entries, or NULL (kept in scratch) */
  uint32_t* x_delta;           /* X_D by insertion code: delta_dict_len entries, or NULL */
  uint64_t* d_new_dict_len;    /* device scalar: |U'| */
  uint32_t* d_new_bits;        /* device scalar: E'_C */
} dm_column_out;

/* Bytes of a packed stream of `rows` codes at `bits` bits (16-byte units). */
size_t dm_packed_bytes(uint64_t rows, uint32_t bits);
/* Eq. 4 on the host: ceil(log2 n), 0 for n <= 1. */
uint32_t dm_bits_for(uint64_t n);
/* Upper bound of E'_C: dm_bits_for(main_dict_len + delta_dict_len). */
uint32_t dm_max_bits(const dm_column_in* in);
/* Arena bytes one dm_merge_column call on `in` needs. */
size_t dm_scratch_bytes(const dm_column_in* in, uint32_t flags);

/* The whole column merge, Steps 1(a) to 2(b) (Section 5 with the Section
 * 5.3 translation tables).  Writes out->new_dict[0..|U'|), x_main, x_delta,
 * the packed vector (dm_packed_bytes(N_M + N_D, E'_C) bytes of it; the
 * rest of the buffer is not touched), *d_new_dict_len and *d_new_bits.
 * Asynchronous; no host synchronisation inside. */
dm_status dm_merge_column(dm_ctx* ctx, const dm_column_in* in, const dm_column_out* out,
                          void* stream, uint32_t flags);

/* Merge ncols columns of one table (Section 6.2.1 scheme (i): columns are
 * independent tasks).  Same contract as dm_merge_column per column.  The
 * arena must hold one column's scratch (DM_ENOMEM otherwise); the full
 * batched schedule needs dm_table_scratch_bytes (flags as passed here), and
 * with less the schedule runs on fewer branches.
 *
 * By default the table runs as ONE CUDA-graph launch: the columns' kernels
 * are recorded once, round-robin over eight branches (dm_tuning.table_branches
 * sets another count), so that the latency-
 * bound Step 1 of some columns overlaps the bandwidth-bound Step 2(b) of
 * others, and replayed on later calls with the same argument bytes (the
 * same buffers; up to eight argument sets are kept per context).  With
 * DM_FLAG_SERIAL the columns run one after another with plain launches.
 * Not for use inside a caller's own stream capture. */
dm_status dm_merge_table(dm_ctx* ctx, const dm_column_in* in, uint32_t ncols,
                         const dm_column_out* out, void* stream, uint32_t flags);
size_t dm_table_scratch_bytes(const dm_column_in* in, uint32_t ncols, uint32_t flags);

/* The same merge with HOST buffers: every pointer in `in` and `out` is host
 * memory (page-locked for full copy speed), except that d_new_dict_len and
 * d_new_bits are ignored and the results go to *new_dict_len / *new_bits.
 * Inputs are copied to device scratch, merged, and the outputs copied back;
 * returns after the copies finish (synchronous).  The arena must hold
 * dm_host_scratch_bytes. */
dm_status dm_merge_column_host(dm_ctx* ctx, const dm_column_in* in, const dm_column_out* out,
                               void* stream, uint32_t flags, uint64_t* new_dict_len,
                               uint32_t* new_bits);
size_t dm_host_scratch_bytes(const dm_column_in* in, uint32_t flags);

/* ---- single steps (same formats; for step-level testing and reuse) ---- */

/* Step 1(a) (Section 5.1 with the Section 5.3 tuple-id map): sort the d
 * keys of delta_dict; ud_out receives them in increasing order (equal keys
 * in insertion order) and perm_out[j] the insertion code of ud_out[j]. */
dm_status dm_sort_delta(dm_ctx* ctx, uint32_t value_bytes, const void* delta_dict, uint64_t d,
                        void* ud_out, uint32_t* perm_out, void* stream);

/* Step 1(b) + 2(a) (Section 5.1 / 5.3, Eq. 4): merge the sorted U_M (m
 * keys) and U_D (d keys, perm from Step 1(a)) into U' without duplicates;
 * x_main[i] / x_delta[perm[j]] receive the U' position of U_M[i] / U_D[j];
 * *d_u and *d_bits (device scalars) receive |U'| and E'_C. */
dm_status dm_merge_dicts(dm_ctx* ctx, uint32_t value_bytes, const void* main_dict, uint64_t m,
                         const void* ud, const uint32_t* perm, uint64_t d, void* new_dict,
                         uint32_t* x_main, uint32_t* x_delta, uint64_t* d_u, uint32_t* d_bits,
                         void* stream);

/* Step 2(b) (Section 5.3, Eq. 11): out code i = x_main[M[i]] for i < n_main,
 * out code n_main + r = x_delta[delta_codes[r]], packed at the width read
 * from the device scalar *d_bits (which must be <= max_bits; the output
 * buffer holds dm_packed_bytes(n_main + n_delta, max_bits) bytes).  Table
 * entries must be < 2^(*d_bits).  The context's arena holds the lookup
 * structures built on the way when it has room for them: the directory of
 * X_M's steps (64 KiB; 256 KiB above 2^22 main codes, where its buckets are
 * refined when shared memory allows, if the arena holds that much), then its
 * byte table (m bytes, above 11 * 2^20
 * main codes; filled and read only when X_M's steps average two or more a
 * directory bucket) or, above 2^24 main codes, the global directory (8 bytes per 2^s
 * codes, s >= 6, at most 16 MiB); without room X_M is gathered directly. */
dm_status dm_reencode(dm_ctx* ctx, const uint32_t* main_packed, uint32_t main_bits,
                      uint64_t n_main, const uint32_t* delta_codes, uint64_t n_delta,
                      const uint32_t* x_main, uint64_t m, const uint32_t* x_delta, uint64_t d,
                      const uint32_t* d_bits, uint32_t max_bits, uint32_t* out_packed,
                      void* stream, uint32_t flags);

/* Step 2(b) by the paper's unoptimised route (Section 5.2, Eq. 5): each
 * tuple's value is decoded through U_M (main rows) or D_dict (delta rows)
 * and its new code found by binary search in U', with no translation
 * tables.  `in` is the column; `out` holds a finished merge of it (new_dict,
 * *d_new_dict_len and *d_new_bits as dm_merge_column left them); the packed
 * vector out->new_packed is rewritten, byte for byte the same as the
 * X_M / X_D route gives.  For measuring what the tables save and for
 * cross-checking.  Asynchronous; data errors go to the status word. */
dm_status dm_reencode_search(dm_ctx* ctx, const dm_column_in* in, const dm_column_out* out, void* stream);

/* ---- delta ingest ---- */

/* Delta ingest (Section 4, Figure 5): n values appended to a column's delta
 * partition, in arrival order (`values`, n keys of value_bytes each, device
 * memory), become the delta form the merge reads: dict_out receives D_dict,
 * each distinct value once in order of first arrival (capacity n keys), and
 * codes_out[i] the position of value i in it; the device scalar
 * *d_dict_len receives |D_dict|.  Scratch (dm_ingest_scratch_bytes) comes
 * from the context's arena.  n is at most 2^30.  Asynchronous.  No input is
 * a data error; dm_sync_status reports DM_EINTERNAL if a row was left
 * without a hash slot (impossible at the table's load of at most one half). */
size_t dm_ingest_scratch_bytes(uint32_t value_bytes, uint64_t n);
dm_status dm_ingest_delta(dm_ctx* ctx, uint32_t value_bytes, const void* values, uint64_t n, void* dict_out,
                          uint32_t* codes_out, uint64_t* d_dict_len, void* stream);

/* One column of a table ingest: its width, the n appended values (device)
 * and its outputs, as in dm_ingest_delta. */
typedef struct {
  uint32_t value_bytes;
  const void* values;
  void* dict_out;
  uint32_t* codes_out;
  uint64_t* d_dict_len;
} dm_ingest_column;

/* n rows appended to a table of ncols columns (Section 4: a row insert adds
 * one value to every column's delta; the update rate of Eq. 16 counts rows),
 * each column ingested exactly as dm_ingest_delta does.  The columns run
 * concurrently on the context's side streams, round-robin over as many
 * branches as a table merge uses, each branch with its own scratch region
 * of the arena (dm_ingest_table_scratch_bytes); the call's stream waits for
 * them all.  Every column is checked before anything is launched (DM_EINVAL
 * for the first bad one; DM_ENOMEM when the arena is too small).
 * Asynchronous. */
size_t dm_ingest_table_scratch_bytes(const dm_ingest_column* cols, uint32_t ncols, uint64_t n);
dm_status dm_ingest_table(dm_ctx* ctx, const dm_ingest_column* cols, uint32_t ncols, uint64_t n, void* stream);

/* ---- allocation-free variant ---- */

/* Largest |U_M| + |U_D| that dm_merge_dicts_noalloc accepts. */
#define DM_NOALLOC_MAX_ENTRIES (1u << 24)

/* Step 1(b) + 2(a) exactly as dm_merge_dicts, but without a context and
 * without allocating anything.  The paper has no counterpart: it exists for
 * callers that must not allocate device memory at merge time — an engine
 * that has already handed all of HBM to its own fixed pools, or a latency
 * path where cudaMalloc's implicit device-wide synchronisation (or its
 * failure when memory is fully reserved) is not acceptable.
 *
 * Its scratch (one look-back word per merge tile of 4096 entries plus the
 * barrier and tile counters; the array is sized for tiles of 2048, 64 KiB
 * and 128 bytes) is a fixed array in the library's static device memory,
 * so every GPU that loads libdmerge holds those 64 KiB until the process
 * exits.  The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Every call zeroes the part it uses on
 * `stream` before its kernel, and the array keeps the last call's contents
 * afterwards.  All calls on a device share the one array: calls whose work
 * may overlap on the GPU (different streams without ordering) race, so
 * serialise them.
 *
 * Arguments as dm_merge_dicts; m + d above DM_NOALLOC_MAX_ENTRIES returns
 * DM_EINVAL.  d_status, if not NULL, is a device word into which the kernel
 * ORs data errors (1: U_M not strictly increasing, 2: a bad insertion code,
 * 4: a wait timed out, 16: an internal check failed); the caller clears it.  With d_status NULL nothing
 * reports such errors: the outputs of a call on bad data (or one whose wait
 * timed out) are then unchecked.  Runs on the current device. */
dm_status dm_merge_dicts_noalloc(uint32_t value_bytes, const void* main_dict, uint64_t m,
                                 const void* ud, const uint32_t* perm, uint64_t d,
                                 void* new_dict, uint32_t* x_main, uint32_t* x_delta,
                                 uint64_t* d_u, uint32_t* d_bits, uint32_t* d_status,
                                 void* stream);

/* ---- result checksum ---- */

/* Add a 64-bit checksum of one merged column's outputs to the device word
 * *d_digest (zero it first; modulo 2^64): |U'| and E'_C as the device scalars
 * hold them, the |U'| keys of new_dict and the dm_packed_bytes(N_M + N_D,
 * E'_C) bytes of new_packed (X_M and X_D are not included).  Each 32-bit
 * word adds splitmix64's output function of its position (col_index, which
 * part, word index) and value, so equal results give equal sums in any
 * order and a changed word changes the sum unless two terms cancel.  For
 * comparing results of merges run in different forms (batched, plain,
 * served) without copying them.  `in` and `out` as given to the merge;
 * asynchronous on `stream`.  The paper has no counterpart. */
dm_status dm_column_digest(const dm_column_in* in, const dm_column_out* out, uint32_t col_index,
                           uint64_t* d_digest, void* stream);

/* ---- served merges (continuous batching) ---- */

/* A merge server: registered tables stay resident on the device; merge
 * requests arriving over time are admitted into `slots` concurrent table
 * merges whenever a slot is free, the table has no merge in flight, and a
 * contiguous region of the scratch pool of `scratch_budget` bytes holds the
 * request's footprint (dm_table_scratch_bytes of its columns).  A host
 * thread watches completions, commits each table's new version (the
 * registry's pointer swap of the paper's atomic commit, Section 3), frees
 * the region and admits the next requests, so work that arrives while
 * other merges run joins them on the device.  Each merge is launched on a
 * stream whose priority follows its size (fewer tuples, higher priority),
 * so a small merge that joins a large one is not held behind its kernels.
 * Results land in the output buffers given at registration; a table serves
 * one merge at a time. */
typedef struct dm_server dm_server;

typedef struct {
  uint32_t slots;            /* concurrent table merges, 1..16 */
  uint64_t scratch_budget;   /* bytes of the scratch pool: the admission budget */
  uint32_t flags;            /* passed to dm_merge_table (0: one graph launch per table),
                                plus the server's own DM_SERVER_* bits */
} dm_server_config;

/* dm_server_config.flags: after each merge, a kernel on the merge's stream
 * sums a 64-bit checksum of its outputs (every column's |U'|, E'_C, U' and
 * packed vector; X_M and X_D are not included) into the request's
 * dm_request_info.digest, so that a merge served among others can be
 * compared with the same merge run alone.  Costs one read of the outputs. */
#define DM_SERVER_DIGEST 0x1000u

typedef struct {
  uint32_t table_id;
  int32_t status;            /* dm_status of the merge; -1 while not finished */
  uint64_t submit_ns, admit_ns, done_ns;   /* server clock (steady, from creation) */
  uint64_t footprint;        /* scratch bytes it held */
  uint32_t slot;
  uint32_t automatic;        /* 1: requested by an online table's trigger */
  uint64_t version;          /* version of the table the merge committed (0: none) */
  uint64_t delta_rows;       /* online tables: delta rows the merge took */
  uint64_t digest;           /* DM_SERVER_DIGEST: checksum of the outputs (0 otherwise) */
} dm_request_info;

typedef struct {
  uint64_t submitted, completed, failed;
  uint64_t tuples;           /* N_M + N_D summed over the columns of completed merges */
  double p50_ms, p99_ms, max_ms, mean_ms;   /* submit -> completion latency */
  uint64_t first_submit_ns, last_done_ns;
  uint64_t peak_scratch_bytes;   /* most scratch ever held at once (<= scratch_budget) */
  uint64_t scratch_budget;
  uint32_t peak_concurrency;     /* most merges ever running at once */
} dm_server_stats;

dm_status dm_server_create(dm_server** server, int device, const dm_server_config* cfg);
/* The tune cache every slot of the server looks its choices up in (owned
 * by the server): load a saved cache into it before submitting, since
 * tuning inside a slot (DM_FLAG_AUTOTUNE in cfg.flags) times merges while
 * other slots run. */
dm_tune_cache* dm_server_tune_cache(dm_server* server);
/* Stops the scheduler thread (pending requests are dropped) and frees the pool. */
void dm_server_destroy(dm_server* server);
/* Register table `table_id`: ncols columns (device pointers, caller-owned,
 * valid until the server is destroyed).  DM_ENOMEM: its footprint exceeds
 * the pool. */
dm_status dm_server_add_table(dm_server* server, uint32_t table_id, const dm_column_in* in, uint32_t ncols,
                              const dm_column_out* out);
/* Queue a merge of the table; returns at once. */
dm_status dm_server_submit(dm_server* server, uint32_t table_id, uint64_t* request_id);
/* Wait until every submitted request has finished (DM_EBUSY on timeout). */
dm_status dm_server_drain(dm_server* server, uint64_t timeout_ms);
dm_status dm_server_request_info(dm_server* server, uint64_t request_id, dm_request_info* info);
dm_status dm_server_stats_get(dm_server* server, dm_server_stats* stats);
/* Committed merges of the table so far. */
uint64_t dm_server_table_version(dm_server* server, uint32_t table_id);

/* ---- online tables (the merge while inserts go on, Sections 3 and 4) ----
 *
 * An online table is owned by the server: its main partition (per column
 * the sorted dictionary U_M and the packed codes) lives in server memory in
 * two copies, and it has two delta partitions, each holding the raw values
 * of inserted rows in arrival order (the paper's uncompressed delta).
 * Inserts append to the active delta.  When a merge of the table is
 * admitted, the active delta is frozen and the other, empty delta becomes
 * active: rows inserted while the merge runs collect there (the paper's
 * temporary second delta).  The merge combines the committed main with the
 * frozen delta (D_dict = the frozen rows' values, row r coded r: repeated
 * values are tolerated, Eq. 3) into the other main copy; its commit at
 * completion makes that copy the table's main (version + 1) and empties the
 * frozen delta, so the second delta is what the next merge takes.  With a
 * trigger fraction k > 0, a merge is requested automatically as soon as the
 * active delta holds more than k * N_M rows (Section 4: merge when N_D
 * exceeds a fraction of N_M).  A paused table's merges are not admitted
 * (inserts and the trigger go on); resuming lets them start.  A merge that
 * has started runs to its end.  A merge that fails keeps its frozen delta,
 * and the table's next merge takes that delta again. */
typedef struct {
  uint32_t value_bytes;      /* 4, 8 or 16 */
  const void* main_dict;     /* initial U_M (device memory, copied at registration) */
  uint64_t main_dict_len;    /* its length */
  const void* main_packed;   /* initial packed codes (device memory, copied) */
  uint32_t main_bits;        /* their width, >= dm_bits_for(main_dict_len) */
} dm_online_column;

typedef struct {
  uint64_t main_rows;        /* N_M of the initial main */
  uint64_t rows_capacity;    /* most rows the main may reach (>= main_rows) */
  uint64_t delta_capacity;   /* most rows one delta holds */
  double trigger;            /* k of the merge trigger N_D > k N_M; 0: merges only on request */
} dm_online_config;

/* Register online table `table_id` with ncols columns.  The server
 * allocates its two main copies (per column main_dict_len + rows_capacity -
 * main_rows keys and dm_packed_bytes(rows_capacity, bits of that) bytes
 * each), its two deltas (delta_capacity keys per column each) and its
 * scratch footprint at those capacities.  DM_ENOMEM: device memory or the
 * pool is too small for it. */
dm_status dm_server_add_online_table(dm_server* server, uint32_t table_id, uint32_t ncols,
                                     const dm_online_column* cols, const dm_online_config* cfg);

/* Where dm_server_insert put the rows. */
typedef struct {
  uint32_t delta;            /* delta partition (0 or 1) they were appended to */
  uint64_t first_row;        /* their first row in it */
  uint64_t lands_in;         /* the table version that will contain them */
  uint32_t triggered;        /* 1: the insert requested a merge (request id below) */
  uint64_t request;
} dm_insert_info;

/* Append nrows rows to an online table: values[c] holds the rows' nrows
 * values of column c (value_bytes each; device or host memory).  Returns
 * once the rows are copied into the active delta (the caller's buffers are
 * free again).  DM_EBUSY: the active delta, or the main's row capacity,
 * cannot take them (nothing is appended); retry after the next commit.
 * info may be NULL. */
dm_status dm_server_insert(dm_server* server, uint32_t table_id, uint64_t nrows, const void* const* values,
                           dm_insert_info* info);

/* Pause (paused != 0) or resume the merges of a table. */
dm_status dm_server_pause(dm_server* server, uint32_t table_id, int paused);

/* The committed state of column `col` of an online table. */
typedef struct {
  uint64_t version;          /* committed merges */
  const void* main_dict;     /* U_M of that version (device memory, server-owned) */
  uint64_t main_dict_len;
  const void* main_packed;   /* its packed codes */
  uint32_t main_bits;
  uint64_t main_rows;
  uint64_t delta_rows;       /* rows inserted and not in this version yet */
} dm_online_view;

/* The buffers stay as they are until the merge that produces version +2
 * is admitted (merges alternate between the two main copies). */
dm_status dm_server_online_view(dm_server* server, uint32_t table_id, uint32_t col, dm_online_view* view);

/* Copy the committed version of column `col` out (host or device memory):
 * its main_dict_len keys to dict_dst (dict_bytes at least that many bytes)
 * and its dm_packed_bytes(main_rows, main_bits) bytes of codes to
 * packed_dst, taken while no commit can swap the version; *view describes
 * what was copied.  Synchronous.  DM_EINVAL: a buffer too small. */
dm_status dm_server_online_copy(dm_server* server, uint32_t table_id, uint32_t col, void* dict_dst,
                                size_t dict_bytes, void* packed_dst, size_t packed_bytes, dm_online_view* view);

/* The online rules on a fake clock (no GPU), for testing and planning:
 * ntables online tables (main_rows[t], delta_capacity[t], trigger[t]; rows
 * capacity unbounded), each merge of table t taking service_ns[t], `slots`
 * merges at once.  Events in time order (ev_ns non-decreasing): kind 0
 * inserts ev_rows rows, 1 requests a merge, 2 pauses the table, 3 resumes
 * it.  For every insert, ev_lands_in receives the version the insert said
 * its rows would land in and ev_version the version whose merge actually
 * took them (0 if rejected or never merged).  Merges, in admission order,
 * go to merge_table / merge_admit_ns / merge_done_ns / merge_rows /
 * merge_version / merge_automatic (at most max_merges; *nmerges receives
 * how many ran). */
dm_status dm_online_simulate(uint32_t slots, uint32_t ntables, const uint64_t* main_rows,
                             const uint64_t* delta_capacity, const double* trigger, const uint64_t* service_ns,
                             uint64_t nevents, const uint32_t* ev_kind, const uint32_t* ev_table,
                             const uint64_t* ev_rows, const uint64_t* ev_ns, uint64_t* ev_lands_in,
                             uint64_t* ev_version, uint64_t max_merges, uint32_t* merge_table,
                             uint64_t* merge_admit_ns, uint64_t* merge_done_ns, uint64_t* merge_rows,
                             uint64_t* merge_version, uint32_t* merge_automatic, uint64_t* nmerges);

/* The server's admission rules run on a fake clock (no GPU): requests of
 * table req_table[i] arrive at arrival_ns[i] (non-decreasing); a merge of
 * table t holds footprint[t] scratch bytes for service_ns[t].  Fills each
 * request's admission and completion times and slot, and the peaks of
 * scratch in use and of merges running at once.  For testing and
 * capacity planning. */
dm_status dm_sched_simulate(uint64_t pool_bytes, uint32_t slots, uint32_t ntables, const uint64_t* footprint,
                            const uint64_t* service_ns, uint64_t nreq, const uint32_t* req_table,
                            const uint64_t* arrival_ns, uint64_t* admit_ns, uint64_t* done_ns,
                            uint32_t* slot_out, uint64_t* peak_bytes, uint32_t* peak_running);

/* ---- status, timing, introspection ---- */

/* Wait for `stream`, read and clear the context's device status word:
 * DM_OK, or the most severe of DM_ETIMEOUT, DM_EINTERNAL, DM_EUNSORTED,
 * DM_ECODE, DM_EINVAL (a device width scalar above the call's bound). */
dm_status dm_sync_status(dm_ctx* ctx, void* stream);

/* Milliseconds of the last dm_merge_column issued with DM_FLAG_TIMING, from
 * CUDA events on the call's stream: [0] Step 1(a), [1] Step 1(b)+2(a),
 * [2] the X_M directory for Step 2(b) (0 when not built), [3] the Step 2(b)
 * kernel, [4] the whole merge.  Synchronises on those events. */
dm_status dm_last_timing(dm_ctx* ctx, float ms[5]);

/* Sum of the per-step milliseconds (as in dm_last_timing) over every
 * dm_merge_column call issued with DM_FLAG_TIMING since the previous
 * dm_timing_sum (at most 1024 calls are kept; *calls receives how many were
 * summed), then forget them.  Synchronises on those events. */
dm_status dm_timing_sum(dm_ctx* ctx, float ms[5], uint32_t* calls);

/* Launch parameters of the kernels, per context (0 = library default).
 * They change how the work is split, never the result. */
typedef struct {
  uint32_t reencode_warps;   /* Step 2(b): warps per block (1..16) */
  uint32_t reencode_stages;  /* Step 2(b): input bulk-copy stages per warp (2..4) */
  uint32_t reencode_obufs;   /* Step 2(b): output staging buffers per warp (1..2) */
  uint32_t host_chunks;      /* dm_merge_column_host: pieces the main vector is
                                uploaded, re-encoded and downloaded in (1..32) */
  uint32_t table_branches;   /* dm_merge_table: concurrent branches of the batched
                                schedule (1..8; default 8), each with its own scratch
                                region; fewer run when the arena holds fewer */
  uint32_t reserved[3];
} dm_tuning;

dm_status dm_set_tuning(dm_ctx* ctx, const dm_tuning* tuning);
dm_status dm_get_tuning(const dm_ctx* ctx, dm_tuning* tuning);

/* ---- autotuning ----
 *
 * The paper's table merge treats every column as an independent task
 * (Section 6.2.1, scheme (i)); which launch shape runs a column fastest
 * depends on the column's widths and sizes, not on the method.  The
 * autotuner times whole-column merges under candidate launch choices and
 * keeps the fastest per column class in a tune cache; later merges of a
 * class look its choice up.  Every choice gives byte-identical results.
 *
 * Precedence: non-zero dm_tuning fields and the DM_FLAG_X_SMEM /
 * DM_FLAG_X_GLOBAL flags override the cache's choice; a cache field of 0
 * means the library default. */


/* Class of a column: its widths and the bit lengths (floor(log2 v) + 1, 0
 * for v = 0) of its sizes. */
typedef struct {
  uint32_t value_bytes;        /* w */
  uint32_t main_bits;          /* E_C */
  uint32_t max_bits;           /* dm_max_bits: bound of E'_C */
  uint32_t log2_m;             /* bit length of |U_M| */
  uint32_t log2_d;             /* bit length of |D_dict| */
  uint32_t log2_main_rows;     /* bit length of N_M */
  uint32_t log2_delta_rows;    /* bit length of N_D */
  uint32_t reserved;
} dm_tune_key;

#define DM_STAGE_AUTO 0u     /* X_M lookup: library rule (shared memory from 2^20 main rows) */
#define DM_STAGE_SMEM 1u     /* X_M in shared memory (table or directory of its steps) when it fits */
#define DM_STAGE_GLOBAL 2u   /* X_M gathered through L1/L2 (no directory of its steps) */
#define DM_X8_AUTO 0u        /* byte table for crowded directory buckets above 11 * 2^20 main codes (dense steps) */
#define DM_X8_OFF 1u         /* no byte table: crowded buckets read X_M */

/* Launch choices for one column class (0 = library default). */
typedef struct {
  uint32_t reencode_warps;     /* Step 2(b): warps per block (1..16) */
  uint32_t reencode_stages;    /* Step 2(b): input bulk-copy stages per warp (2..4) */
  uint32_t reencode_obufs;     /* Step 2(b): output staging buffers per warp (1..2) */
  uint32_t x_staging;          /* DM_STAGE_* */
  uint32_t x8;                 /* DM_X8_* */
  uint32_t step1_blocks;       /* Step 1 grid: at most this many blocks (0: all that fit) */
  uint32_t reserved[2];
} dm_tune_choice;

/* What dm_autotune_column measured. */
typedef struct {
  dm_tune_key key;             /* the class tuned */
  dm_tune_choice best;         /* stored in the cache */
  float best_ms;               /* median whole-merge milliseconds of `best` */
  float default_ms;            /* the same for the library defaults */
  uint32_t candidates;         /* choices timed */
  uint32_t reps;               /* timed merges per choice */
} dm_tune_report;

/* The class of a column (host only; no device needed). */
dm_status dm_tune_key_of(const dm_column_in* in, dm_tune_key* key);

/* A tune cache is host memory only and thread-safe; contexts may share one.
 * Every context starts with a cache of its own. */
dm_status dm_tune_cache_create(dm_tune_cache** cache);
void dm_tune_cache_destroy(dm_tune_cache* cache);
/* Insert or replace the choice of a class (DM_EINVAL: a field out of range). */
dm_status dm_tune_cache_put(dm_tune_cache* cache, const dm_tune_key* key, const dm_tune_choice* choice);
/* The choice of a class, or DM_ENOENT. */
dm_status dm_tune_cache_get(const dm_tune_cache* cache, const dm_tune_key* key, dm_tune_choice* choice);
uint64_t dm_tune_cache_size(const dm_tune_cache* cache);
/* Changes with every put, clear and load. */
uint64_t dm_tune_cache_generation(const dm_tune_cache* cache);
dm_status dm_tune_cache_clear(dm_tune_cache* cache);
/* Write every entry to `path` as JSON; read such a file and merge its
 * entries in (file entries replace equal keys).  A malformed file returns
 * DM_EINVAL and changes nothing; a missing one DM_ENOENT. */
dm_status dm_tune_cache_save(const dm_tune_cache* cache, const char* path);
dm_status dm_tune_cache_load(dm_tune_cache* cache, const char* path);

/* Use `cache` (not owned; it must outlive its use) for this context's
 * lookups and tuning; NULL returns to the context's own cache. */
dm_status dm_set_tune_cache(dm_ctx* ctx, dm_tune_cache* cache);
dm_tune_cache* dm_get_tune_cache(dm_ctx* ctx);

/* Every candidate choice the autotuner considers for `in` on this context's
 * device: writes up to `cap` of them to `out` and returns how many exist. */
uint32_t dm_tune_candidates(const dm_ctx* ctx, const dm_column_in* in, dm_tune_choice* out, uint32_t cap);

/* Merge the column (as dm_merge_column) under candidate choices, timing
 * `reps` merges of each (0: 5; at most 1000, else DM_EINVAL) with CUDA
 * events on `stream`, and store the
 * fastest in the context's tune cache.  The search takes the X_M staging
 * and byte-table choices first, then the Step 2(b) launch shape, then the
 * Step 1 grid, each time keeping the fastest so far.  On return `out` holds
 * the merge result.  Synchronous (blocks the host); not inside a stream
 * capture. */
dm_status dm_autotune_column(dm_ctx* ctx, const dm_column_in* in, const dm_column_out* out, void* stream,
                             uint32_t flags, uint32_t reps, dm_tune_report* report);

/* ---- testing the bounded waits ----
 *
 * Every device-side wait of the merge (grid barriers, the look-back words
 * of the sort passes and of the merge tiles) polls a bounded number of
 * times, then ORs DM_ETIMEOUT's bit into the status word and lets the
 * kernel run to its end, so a wait that cannot be satisfied never hangs the
 * GPU.  This setting exercises that path: in Step 1 launches of this
 * context, merge tile `withhold_tile` (merged positions [4096 t, 4096 t +
 * 4096)) does not publish its look-back word, so the waits of the merge
 * tiles after it run out, and every Step 1 wait gives up after
 * `spin_limit` polls (0: the library's limit, about a second).  The merge
 * then finishes with wrong codes and dm_sync_status returns DM_ETIMEOUT;
 * every memory access stays in bounds.  DM_WAIT_TEST_OFF (with spin_limit
 * 0) restores normal merges.  Not for production use. */
#define DM_WAIT_TEST_OFF 0xFFFFFFFFu
dm_status dm_set_wait_test(dm_ctx* ctx, uint32_t withhold_tile, uint32_t spin_limit);

/* Kernels this context has launched so far. */
uint64_t dm_launch_count(const dm_ctx* ctx);

/* Name of a status code. */
const char* dm_status_str(dm_status s);

/* Text of the last CUDA runtime error a call on this context met (the
 * detail behind DM_ECUDA). */
const char* dm_last_error(const dm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DMERGE_H_ */
