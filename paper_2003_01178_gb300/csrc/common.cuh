// Device building blocks shared by the operator kernels: bulk asynchronous copies
// (TMA, cp.async.bulk) into shared memory with mbarrier completion, bounded waits,
// warp/block scans and reductions, and the hash function.  These are the sm_103a
// counterparts of the paper's block-wide functions (Section 3.3, Table "list-func"):
// BlockLoad = bulk copy of a tile into a shared-memory stage; BlockPred / BlockScan /
// BlockShuffle / BlockStore / BlockLookup / BlockAggregate are written out in each
// kernel on top of the helpers below.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "crystal.h"
#include "internal.h"

namespace crys {

constexpr int kWarp = 32;
// Upper bound of any spin-wait, in nanoseconds of %globaltimer.  Legitimate waits are
// microseconds; after this bound the waiting thread sets CRYS_DEV_TIMEOUT and its block
// abandons the work instead of hanging the GPU.
constexpr uint64_t kWaitBoundNs = 2000000000ull;
constexpr uint64_t kEmptySlot = 0xFFFFFFFFFFFFFFFFull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void set_error(int32_t* err, int32_t bits) {
  atomicOr(reinterpret_cast<int*>(err), bits);
}

__device__ __forceinline__ int32_t read_error(const int32_t* err) {
  return *reinterpret_cast<const volatile int32_t*>(err);
}

// ---------------------------------------------------------------- mbarrier + TMA

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

// Makes barrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's generic-proxy shared-memory accesses before later async-proxy
// accesses (a stage that was read by threads is about to be overwritten by TMA).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar_addr, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar_addr), "r"(parity)
      : "memory");
  return done != 0;
}

// Waits for phase `parity` of the barrier to complete, at most kWaitBoundNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int32_t* err) {
  const uint32_t addr = smem_u32(bar);
  if (mbar_try_wait(addr, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (true) {
    if (mbar_try_wait(addr, parity)) return true;
    if (global_timer_ns() - t0 > kWaitBoundNs) {
      set_error(err, CRYS_DEV_TIMEOUT);
      return false;
    }
  }
}

// L2 eviction policies for bulk copies and loads: streamed columns are read once
// (evict_first) so that hash tables probed at random stay resident (evict_last).
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// One-dimensional bulk copy global -> shared (TMA engine), completing `bytes` of
// transaction count on `bar`.  src and dst 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src, uint32_t bytes,
                                          uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst_smem)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// Bulk prefetch of a contiguous global range into L2 (copy engine; no registers, no
// completion to wait for).  Address 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------- global loads

// Streaming column loads: not allocated in L1, L2 policy from policy_evict_first().
__device__ __forceinline__ int4 ld_stream_v4(const int32_t* p, uint64_t pol) {
  int4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}

__device__ __forceinline__ int32_t ld_stream(const int32_t* p, uint64_t pol) {
  int32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;"
               : "=r"(v)
               : "l"(p), "l"(pol));
  return v;
}

// Hash-table slot read with the L2 policy from policy_evict_last() (tables are read-only
// while they are probed and should outlive the streamed columns in L2).
__device__ __forceinline__ uint64_t ld_slot(const uint64_t* p, uint64_t pol) {
  uint64_t v;
  asm volatile("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
  return v;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------- hashing

// Home slot of a key: (hi32(key * mult) >> shift) & mask, where hi32 is bits 32..63 of
// the 64-bit product (uint32)key * mult, formed as key * mult_hi + umulhi(key, mult_lo).
// Multiplicative (Fibonacci) hashing takes the top log2(capacity) bits of the product with
// mult = 0x9E3779B97F4A7C15 (the integer part of 2^64/phi, odd), shift = 32 - log2(capacity).
// With the 32-bit constant 2654435769 (2^32/phi) instead, dense keys 0..n-1 cluster at
// some sizes: a lookup examines 2.3 slots on average at n = 2^22 (1.7 at 2^21, 1.3 at
// 2^20) against 1.0 with the 64-bit product at every n from 2^10 to 2^27; random keys
// examine the 1.5 of linear probing at 50% fill either way.  Tables of at most
// kSmallHashSlots slots keep the 32-bit constant (mult_lo = 0: their dense keys do not
// cluster, 1.003 slots at most), so that a probe of a table held in shared memory needs
// one multiply.  Identity hashing (key mod capacity) uses mult = 2^32 (mult_hi = 1,
// mult_lo = 0), shift = 0.
constexpr int64_t kSmallHashSlots = 4096;
struct HashFn {
  uint32_t mult_hi, mult_lo;
  uint32_t shift, mask;
  uint32_t limit;  // keys >= limit (as unsigned) are absent without reading a slot
  uint32_t steps;  // further slots a lookup may examine after the home slot
};

// Hash function of a table kind and capacity (a power of two except for direct tables).
__host__ __device__ __forceinline__ HashFn make_hash(int32_t kind, int64_t capacity) {
  HashFn h;
  if (kind == CRYS_HASH_DIRECT) {
    // the slot of key k is k itself: a key is in its slot or absent
    h.mult_hi = 1u;
    h.mult_lo = 0u;
    h.shift = 0u;
    h.mask = 0xFFFFFFFFu;
    h.limit = static_cast<uint32_t>(capacity);
    h.steps = 0u;
    return h;
  }
  uint32_t log2cap = 0;
  while ((int64_t{1} << log2cap) < capacity) ++log2cap;
  h.mask = (log2cap >= 32) ? 0xFFFFFFFFu : ((1u << log2cap) - 1u);
  h.limit = 0xFFFFFFFFu;  // key -1 is the empty marker and never stored
  h.steps = h.mask;
  if (kind == CRYS_HASH_IDENT) {
    h.mult_hi = 1u;
    h.mult_lo = 0u;
    h.shift = 0u;
  } else if (capacity <= kSmallHashSlots) {
    h.mult_hi = 2654435769u;
    h.mult_lo = 0u;
    h.shift = 32u - log2cap;
  } else {
    h.mult_hi = 0x9E3779B9u;
    h.mult_lo = 0x7F4A7C15u;
    h.shift = 32u - log2cap;
  }
  return h;
}

__device__ __forceinline__ uint32_t hash_slot(int32_t key, const HashFn& f) {
  const uint32_t k = static_cast<uint32_t>(key);
  return ((k * f.mult_hi + __umulhi(k, f.mult_lo)) >> f.shift) & f.mask;
}
// The same for a table of at most kSmallHashSlots slots (mult_lo is 0 for every kind).
__device__ __forceinline__ uint32_t hash_slot_small(int32_t key, const HashFn& f) {
  return ((static_cast<uint32_t>(key) * f.mult_hi) >> f.shift) & f.mask;
}

// Whether a key can be in the table at all (direct tables: 0 <= key < capacity).
__device__ __forceinline__ bool hash_may_hold(int32_t key, const HashFn& f) {
  return static_cast<uint32_t>(key) < f.limit;
}

// Continues a lookup whose home slot `s` (at index h) was already loaded (kEmptySlot when
// the key cannot be in the table): linear probing until the key or an empty slot.
__device__ __forceinline__ bool hash_resolve(const uint64_t* slots, const HashFn& f, uint32_t h,
                                             uint64_t s, int32_t key, int32_t* value,
                                             uint64_t pol) {
  for (uint32_t probe = 0;; ++probe) {
    if (s == kEmptySlot) return false;
    if (static_cast<uint32_t>(s) == static_cast<uint32_t>(key)) {
      *value = static_cast<int32_t>(s >> 32);
      return true;
    }
    if (probe >= f.steps) return false;
    h = (h + 1) & f.mask;
    s = ld_slot(slots + h, pol);
  }
}

// Continues ITEMS lookups whose home slots were already loaded, all together (Section 4.3,
// linear probing): every round issues the next slot of each unresolved item before any
// of them is examined, so a warp waits one L2 round trip per probing step of its
// longest chain instead of one per item whose chain goes past the home slot.  Items
// outside `live` are never found.  Returns the bitmap of items whose key was found, with
// its value in `value`; `h` and `s` are consumed.
template <int ITEMS>
__device__ __forceinline__ uint32_t hash_resolve_all(const uint64_t* slots, const HashFn& f,
                                                     uint32_t (&h)[ITEMS], uint64_t (&s)[ITEMS],
                                                     const int32_t (&key)[ITEMS], uint32_t live,
                                                     int32_t (&value)[ITEMS], uint64_t pol) {
  uint32_t found = 0, pend = 0;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t bit = ((live >> i) & 1u) << i;
    if (s[i] == kEmptySlot || !bit) continue;
    if (static_cast<uint32_t>(s[i]) == static_cast<uint32_t>(key[i])) {
      value[i] = static_cast<int32_t>(s[i] >> 32);
      found |= bit;
    } else {
      pend |= bit;
    }
  }
  for (uint32_t probe = 0; pend != 0u && probe < f.steps; ++probe) {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
      if ((pend >> i) & 1u) {
        h[i] = (h[i] + 1) & f.mask;
        s[i] = ld_slot(slots + h[i], pol);
      }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
      if ((pend >> i) & 1u) {
        if (s[i] == kEmptySlot) {
          pend &= ~(1u << i);
        } else if (static_cast<uint32_t>(s[i]) == static_cast<uint32_t>(key[i])) {
          value[i] = static_cast<int32_t>(s[i] >> 32);
          found |= 1u << i;
          pend &= ~(1u << i);
        }
      }
  }
  return found;
}

// Looks `key` up; returns the value, or false when absent.
__device__ __forceinline__ bool hash_find(const uint64_t* slots, const HashFn& f, int32_t key,
                                          int32_t* value, uint64_t pol) {
  if (!hash_may_hold(key, f)) return false;
  const uint32_t h = hash_slot(key, f);
  return hash_resolve(slots, f, h, ld_slot(slots + h, pol), key, value, pol);
}

// Fire-and-forget 64-bit add to global memory (no value returned, so the issuing warp
// does not wait for it), with an L2 policy: accumulators that many rows update should
// stay resident while the fact stream passes through L2.
__device__ __forceinline__ void red_add_global(unsigned long long* p, unsigned long long v, uint64_t pol) {
  asm volatile("red.global.add.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}

// ---------------------------------------------------------------- scans / reductions

__device__ __forceinline__ int32_t warp_inclusive_scan(int32_t v, int lane) {
#pragma unroll
  for (int d = 1; d < kWarp; d <<= 1) {
    int32_t u = __shfl_up_sync(0xFFFFFFFFu, v, d);
    if (lane >= d) v += u;
  }
  return v;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, d);
  return v;
}

// Block-wide sum of one uint64 per thread; result valid in thread 0.
// `scratch` holds one uint64 per warp.
template <int THREADS>
__device__ __forceinline__ uint64_t block_sum_u64(uint64_t v, uint64_t* scratch) {
  constexpr int WARPS = THREADS / kWarp;
  const int lane = threadIdx.x % kWarp, warp = threadIdx.x / kWarp;
  v = warp_sum_u64(v);
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  uint64_t total = 0;
  if (warp == 0) {
    uint64_t w = lane < WARPS ? scratch[lane] : 0ull;
    total = warp_sum_u64(w);
  }
  __syncthreads();
  return total;
}

}  // namespace crys
