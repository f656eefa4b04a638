// Directory of X_M for the Step 2(b) lookup (shared by the Step 1 kernel,
// which builds it after the merge, and by the standalone re-encode path).
//
// X_M[i] = i + c[i], where c[i] counts the delta-only values of U' that sort
// below U_M[i]: a step function of the main code with one step per new value
// (|U'| - |U_M| steps in all).  The directory cuts the main codes into
// buckets of 2^s (s <= 10) and keeps, per bucket, c at the bucket's start
// (base, 20 bits) and the offset thr of the bucket's single step, if it has
// exactly one, as
//   entry = (2048 - thr) << 20 | base.
// For a code i with offset lo = i mod 2^s in its bucket, entry + (lo << 20)
// carries into bit 31 exactly when lo >= thr, so
//   X_M[i] = i + (y & 0xFFFFF) + (y >> 31),  y = entry + (lo << 20).
// A bucket without steps stores thr = 1024 (above every offset, as s <= 10),
// so that every entry of a bucket read through the lookup is at least
// 1024 << 20 and the markers below are told apart by one compare.  A bucket with
// two or more steps (up to 255) and a 20-bit base, when a byte table X8 of
// c[i] - base exists, stores the marker thr = 2045 with its base, and its
// codes read X8: X_M[i] = i + base + X8[i] (X8 is a quarter of X_M's size,
// so it stays in L2 where X_M may not).  Other buckets store the marker
// thr = 2046 and their codes read X_M itself.
#pragma once

#include <stdint.h>

namespace dm {

constexpr uint32_t DIR_NONE = 1024, DIR_MANY = 2046, DIR_MANY8 = 2045;
constexpr uint32_t DIR_MANY_TOP = 2048 - DIR_MANY;     // top 12 bits of an entry read through X_M
constexpr uint32_t DIR_MANY8_TOP = 2048 - DIR_MANY8;   // top 12 bits of an entry read through X8
// Entries of both markers are below DIR_SLOW_BELOW; every other entry is at
// least 1024 << 20 (NONE has top 1024, a single step top 1025..2048).
constexpr uint32_t DIR_SLOW_BELOW = 4u << 20;
static_assert((DIR_MANY_TOP << 20) < DIR_SLOW_BELOW && (DIR_MANY8_TOP << 20) < DIR_SLOW_BELOW &&
                  ((2048u - DIR_NONE) << 20) >= DIR_SLOW_BELOW,
              "markers");
constexpr uint32_t RE_DIR_MAX = 16384;               // entries (64 KiB of shared memory)
constexpr uint32_t RE_DIR_SHIFT_MAX = 10;
// A refined directory (finer buckets than xdir_shape's, where shared memory
// allows) for more than RE_DIR_FINE_MIN_CODES main codes: at most this many
// entries of scratch.
constexpr uint32_t RE_DIR_FINE_MAX = 65536;
constexpr uint64_t RE_DIR_FINE_MIN_CODES = 1ull << 22;
static_assert((1u << RE_DIR_SHIFT_MAX) <= DIR_NONE, "a bucket without steps never carries");

// Entry of bucket b.  Coherent: X_M was written earlier in the same kernel,
// so it is read through L2 (ld.global.cg), never from a stale L1 line.
template <bool Coherent>
__device__ __forceinline__ uint32_t xdir_entry(const uint32_t* __restrict__ xm, uint32_t m, uint32_t s, uint32_t b,
                                               bool has_x8) {
  auto ld = [&](uint32_t i) { return Coherent ? __ldcg(xm + i) : __ldg(xm + i); };
  const uint32_t lo = b << s;
  const uint32_t hi = min(((b + 1) << s), m) - 1;
  const uint32_t base = lo == 0 ? 0u : ld(lo - 1) - (lo - 1);
  const uint32_t cnt = (ld(hi) - hi) - base;
  uint32_t thr;
  if (cnt == 0) {
    thr = DIR_NONE;
  } else if (cnt == 1) {
    // first code of the bucket past the step: c[i] > base
    uint32_t l = lo, h = hi;
    while (l < h) {
      uint32_t mid = (l + h) >> 1;
      if (ld(mid) - mid > base) h = mid;
      else l = mid + 1;
    }
    thr = l - lo;
  } else {
    thr = has_x8 && cnt <= 255 ? DIR_MANY8 : DIR_MANY;
  }
  if (base >= (1u << 20)) thr = DIR_MANY;
  return ((2048u - thr) << 20) | (thr == DIR_MANY ? 0u : base);
}

// Whether the crowded buckets should read the byte table: only when the
// steps are dense, at least two a bucket on average (their count is X_M's
// last entry less its code: the new values below the last main value).
// With fewer, a crowded code's X_M read is the cheaper path, so the buckets
// are marked DIR_MANY and the table is not written.
template <bool Coherent>
__device__ __forceinline__ bool xdir_x8_pays(const uint32_t* __restrict__ xm, uint32_t m, uint32_t entries) {
  if (m == 0) return false;
  const uint32_t last = Coherent ? __ldcg(xm + m - 1) : __ldg(xm + m - 1);
  return (uint64_t)(last - (m - 1)) >= 2ull * entries;
}

// X8[i] = c[i] - c[first code of i's bucket - 1] (mod 256); read only for
// codes in buckets marked DIR_MANY8, where it is exact.
template <bool Coherent>
__device__ __forceinline__ uint8_t xdir_x8(const uint32_t* __restrict__ xm, uint32_t s, uint32_t i) {
  auto ld = [&](uint32_t k) { return Coherent ? __ldcg(xm + k) : __ldg(xm + k); };
  const uint32_t lo = (i >> s) << s;
  const uint32_t base = lo == 0 ? 0u : ld(lo - 1) - (lo - 1);
  return (uint8_t)((ld(i) - i) - base);
}

// Fills X8 for codes t, t + nt, ... (a grid-stride loop over m codes).  With
// buckets of at least four codes and aligned tables, one thread takes four
// consecutive codes of one bucket: a 16-byte load of X_M, one load of the
// bucket's base and a 4-byte store.
template <bool Coherent>
__device__ __forceinline__ void xdir_x8_fill(const uint32_t* __restrict__ xm, uint32_t m, uint32_t s,
                                             uint8_t* __restrict__ x8, uint32_t t, uint32_t nt) {
  uint32_t done = 0;
  if (s >= 2 && (reinterpret_cast<uintptr_t>(xm) & 15u) == 0 && (reinterpret_cast<uintptr_t>(x8) & 3u) == 0) {
    const uint32_t q = m >> 2;
    const uint4* xm4 = reinterpret_cast<const uint4*>(xm);
    uint32_t* x84 = reinterpret_cast<uint32_t*>(x8);
    for (uint32_t k = t; k < q; k += nt) {
      const uint32_t i = k << 2, lo = (i >> s) << s;
      const uint4 v = Coherent ? __ldcg(xm4 + k) : __ldg(xm4 + k);
      const uint32_t prev = lo == 0 ? 0u : (Coherent ? __ldcg(xm + lo - 1) : __ldg(xm + lo - 1));
      const uint32_t b = lo == 0 ? i : i + (prev - (lo - 1));   // i + base
      x84[k] = ((v.x - b) & 0xFFu) | ((v.y - b - 1u) & 0xFFu) << 8 | ((v.z - b - 2u) & 0xFFu) << 16 |
               (v.w - b - 3u) << 24;
    }
    done = q << 2;
  }
  for (uint32_t i = done + t; i < m; i += nt) x8[i] = xdir_x8<Coherent>(xm, s, i);
}

// Bucket shift and entry count of the directory for m main codes.
__host__ __device__ inline void xdir_shape(uint64_t m, uint32_t* shift, uint32_t* entries) {
  uint32_t sh = 0;
  while (((m + (1ull << sh) - 1) >> sh) > RE_DIR_MAX) ++sh;
  *shift = sh;
  *entries = (uint32_t)((m + (1ull << sh) - 1) >> sh);
}

}  // namespace dm
