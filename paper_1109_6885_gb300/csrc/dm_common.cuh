// Shared device-side pieces of libdmerge: key types, status bits, PTX
// wrappers for mbarriers and bulk (TMA) copies, bounded waits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dmerge.h"

namespace dm {

// ---------------------------------------------------------------- status word
// Bits ORed into the per-context device status word by kernels.
enum : uint32_t {
  ST_UNSORTED = 1u,  // U_M not strictly increasing
  ST_CODE = 2u,      // a code outside its dictionary (clamped)
  ST_TIMEOUT = 4u,   // a bounded wait gave up
  ST_WIDTH = 8u,     // device width scalar above the host bound
  ST_INTERNAL = 16u, // an internal consistency check failed (a write index out
                     // of range, a hash slot missing): the outputs are invalid
};

// Spin limit of every device-side wait (about a second with the backoff).
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ void flag_status(uint32_t* status, uint32_t bit) {
  if (status) atomicOr(status, bit);
}

// ---------------------------------------------------------------- keys
struct u128 {
  uint64_t hi, lo;
};

template <int W>
struct KeyOf;
template <>
struct KeyOf<4> {
  using T = uint32_t;
};
template <>
struct KeyOf<8> {
  using T = uint64_t;
};
template <>
struct KeyOf<16> {
  using T = u128;
};

__device__ __forceinline__ bool key_lt(uint32_t a, uint32_t b) { return a < b; }
__device__ __forceinline__ bool key_lt(uint64_t a, uint64_t b) { return a < b; }
__device__ __forceinline__ bool key_lt(const u128& a, const u128& b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool key_eq(uint32_t a, uint32_t b) { return a == b; }
__device__ __forceinline__ bool key_eq(uint64_t a, uint64_t b) { return a == b; }
__device__ __forceinline__ bool key_eq(const u128& a, const u128& b) {
  return a.hi == b.hi && a.lo == b.lo;
}
template <class K>
__device__ __forceinline__ bool key_le(const K& a, const K& b) {
  return !key_lt(b, a);
}
template <class K>
__device__ __forceinline__ K key_max(const K& a, const K& b) {
  return key_lt(a, b) ? b : a;
}

// Byte `pass` of a key, pass 0 = least significant (16-byte keys: lo first).
__device__ __forceinline__ uint32_t key_digit(uint32_t k, int pass) { return (k >> (8 * pass)) & 0xFFu; }
__device__ __forceinline__ uint32_t key_digit(uint64_t k, int pass) {
  return (uint32_t)(k >> (8 * pass)) & 0xFFu;
}
__device__ __forceinline__ uint32_t key_digit(const u128& k, int pass) {
  return pass < 8 ? (uint32_t)(k.lo >> (8 * pass)) & 0xFFu : (uint32_t)(k.hi >> (8 * (pass - 8))) & 0xFFu;
}

template <class K>
__device__ __forceinline__ K key_max_value();
template <>
__device__ __forceinline__ uint32_t key_max_value<uint32_t>() { return 0xFFFFFFFFu; }
template <>
__device__ __forceinline__ uint64_t key_max_value<uint64_t>() { return ~0ull; }
template <>
__device__ __forceinline__ u128 key_max_value<u128>() { return u128{~0ull, ~0ull}; }

template <class K>
__device__ __forceinline__ K load_key(const K* p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ u128 load_key<u128>(const u128* p) {
  ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(p));
  return u128{v.x, v.y};
}

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ---------------------------------------------------------------- mbarrier / bulk copy
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on a phase of an mbarrier; false (and a status bit) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t* status) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 64) __nanosleep(128);
  }
  flag_status(status, ST_TIMEOUT);
  return false;
}

// Global -> shared bulk copy completing on an mbarrier (bytes % 16 == 0, both
// addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gmem_src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(smem_dst)),
      "l"(gmem_src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// L2 policy for data streamed once: its lines are evicted first, so that
// tables gathered from at random (X_M, X_D) keep their place in L2.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Global -> shared bulk copy with an L2 cache policy.
__device__ __forceinline__ void bulk_g2s_hint(void* smem_dst, const void* gmem_src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_addr(smem_dst)),
      "l"(gmem_src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

// Shared -> global bulk copy with an L2 cache policy, tracked by bulk groups.
__device__ __forceinline__ void bulk_s2g_hint(void* gmem_dst, const void* smem_src, uint32_t bytes, uint64_t policy) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(gmem_dst),
               "r"(smem_addr(smem_src)), "r"(bytes), "l"(policy)
               : "memory");
}

// Shared -> global bulk copy tracked by bulk groups.
__device__ __forceinline__ void bulk_s2g(void* gmem_dst, const void* smem_src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gmem_dst),
               "r"(smem_addr(smem_src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// ---------------------------------------------------------------- look-back words
// Decoupled look-back status: flag in the top bits, running count below.
constexpr uint32_t LB_AGG32 = 1u << 30, LB_INC32 = 2u << 30, LB_MASK32 = (1u << 30) - 1;
constexpr uint64_t LB_AGG64 = 1ull << 62, LB_INC64 = 2ull << 62, LB_MASK64 = (1ull << 62) - 1;

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_volatile(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_volatile(uint32_t* p, uint32_t v) {
  asm volatile("st.volatile.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_volatile(uint64_t* p, uint64_t v) {
  asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__host__ __device__ __forceinline__ uint32_t bits_for(uint64_t n) {
  uint32_t b = 0;
  while (b < 64 && (1ull << b) < n) ++b;
  return b;
}

}  // namespace dm
