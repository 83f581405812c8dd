// Device-side building blocks for the gshoot kernels (sm_103a):
// bulk-copy (TMA) staging into shared memory guarded by mbarriers with
// bounded waits, the MUFU base-2 exponential, compensated FP32 arithmetic
// (Kahan updates and double-single pairs), programmatic dependent launch.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gs_internal.h"

namespace gs {

// Bound of every spin on an mbarrier phase.  An unanswered try_wait
// suspends the thread for a while before it returns false (measured on
// GB300: 4,194,304 of them took 15.7 s, 3.75 us each), so 2^18 polls bound a
// wait at about one second; the copies and releases waited for take
// microseconds.  A time check inside the poll loop measured 6-11% slower
// gradients (it weighs on the register allocation of the pair loops).
constexpr long kSpinLimit = 1L << 18;
// Bound of the global-memory poll of the wait check (diag.cu), in global
// time.
constexpr unsigned long long kWaitNs = 1000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
               ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Plain arrival (no transaction bytes) on an mbarrier.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bulk global -> shared copy (TMA, non-tensor); completes `bytes` of
// transaction count on `bar`.  dst, src 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// Bounded wait on phase `parity` of `bar`.  Returns false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const uint32_t addr = smem_u32(bar);
  for (long it = 0; it < kSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(addr), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}

// Programmatic dependent launch: wait for the preceding kernel's results.
// A no-op when launched without PDL.  No kernel triggers its dependents at
// its start: on GB300 that let the next step's clusters take SM slots while
// the current step ran, and made chains of 8-CTA-cluster steps up to 47%
// slower.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Let the next kernel in the stream launch once every CTA of this grid has
// issued this (or exited).  Its griddepcontrol.wait still waits for this
// grid to complete and flush, so the trigger moves only the next launch's
// set-up, never the data dependence.  The step kernels issue it late, after
// their pair sums, when the host asks for it (one-wave grids).
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// 2^x on the MUFU unit (flushes subnormal results to zero).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------- clusters
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

// Cluster-wide barrier: every thread of every CTA of the cluster arrives;
// shared-memory writes before it are visible to the cluster after it.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The two halves of a cluster barrier.  A CTA may touch a peer's shared
// memory only once the peer has started: arrive (relaxed, no ordering) at
// kernel start, and wait before the first remote access.
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;" ::: "memory"); }

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t dsmem_addr(uint32_t local, unsigned rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}

// Store to shared memory of a CTA of the cluster (address from dsmem_addr).
__device__ __forceinline__ void st_dsmem_f4(uint32_t addr, float4 v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}

__device__ __forceinline__ float2 ld_dsmem_f2(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}

// ---------------------------------------------------------------- FP64 reductions
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA in a fixed order; result valid in thread 0.  `sh` holds
// one double per warp.  Every thread of the CTA must call it.
__device__ __forceinline__ double block_sum_f64(double v, double* sh) {
  v = warp_sum_f64(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    r = warp_sum_f64(r);
  }
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------- compensated FP32
// The *_rn intrinsics are never contracted into FMAs, which keeps the error
// terms exact.

// Kahan step: (sum, c) absorbs x; the compensated value is sum - c.
__device__ __forceinline__ void kahan_add(float& sum, float& c, float x) {
  const float y = __fsub_rn(x, c);
  const float t = __fadd_rn(sum, y);
  c = __fsub_rn(__fsub_rn(t, sum), y);
  sum = t;
}

// Error-free a + b = s + e (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Error-free a + b = s + e when |a| >= |b| (Dekker's FastTwoSum).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// Double-single value hi + lo with |lo| <= ulp(hi)/2.
struct ds {
  float hi, lo;
};

__device__ __forceinline__ ds ds_from_kahan(float sum, float c) {
  ds r;
  fast_two_sum(sum, -c, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ ds ds_add(ds a, ds b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  ds r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

// (hi + lo) * f for an FP32 constant f, error-free product of hi.
__device__ __forceinline__ ds ds_mul_f(ds a, float f) {
  const float p = __fmul_rn(a.hi, f);
  float e = __fmaf_rn(a.hi, f, -p);
  e = __fmaf_rn(a.lo, f, e);
  ds r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ double ds_to_double(ds a) { return (double)a.hi + (double)a.lo; }

}  // namespace gs
