// Pieces shared by the kernels that run one problem's time steps on
// thread-block clusters (step_kernels.cu: one launch per step;
// sweep_kernels.cu: one persistent launch per sweep): the deterministic
// grid-wide sum, the push of split partials into the reducing CTA's shared
// memory, and the host side of cluster launches.
#pragma once

#include <mutex>
#include <set>

#include "pair_tile.cuh"

namespace gs {

// ---------------------------------------------------------------- device
// Grid-wide deterministic sum of per-CTA values: each CTA stores its value
// at red[cta]; the last CTA to take a ticket adds them with one warp in a
// fixed order.  Returns true in the threads of the finishing warp; their
// *out holds the total.
__device__ __forceinline__ bool grid_sum2(double vh, double vm, double* red_h, double* red_m, unsigned* ticket,
                                          double* sh, int* am_last, double* out_h, double* out_m) {
  const double bh = block_sum_f64(vh, sh);
  const double bm = block_sum_f64(vm, sh);
  const unsigned cta = blockIdx.y * gridDim.x + blockIdx.x;
  const unsigned ncta = gridDim.x * gridDim.y;
  if (threadIdx.x == 0) {
    red_h[cta] = bh;
    red_m[cta] = bm;
    __threadfence();
    const unsigned tk = atomicAdd(ticket, 1u);
    *am_last = (tk == ncta - 1);
  }
  __syncthreads();
  if (!*am_last || threadIdx.x >= 32) return false;
  __threadfence();
  double h = 0.0, m = 0.0;
  for (unsigned b = threadIdx.x; b < ncta; b += 32) {
    h += *((volatile double*)&red_h[b]);
    m += *((volatile double*)&red_m[b]);
  }
  *out_h = warp_sum_f64(h);
  *out_m = warp_sum_f64(m);
  return true;
}


// Send one target's 2D double-single partials (D float4) to the CTA of the
// cluster that reduces that target.  CTA `owner` reduces targets
// [owner*slice, (owner+1)*slice) of the tile; the partials of local target
// lt from source split `rank` land in the owner's
// recv[(rank*slice + lt - owner*slice)*D + 0..D-1].  The stores are remote
// (distributed shared memory) and need no reply; the cluster barrier that
// follows makes them visible to the owner.
template <int D>
__device__ __forceinline__ void push_partials(float4* recv, int lt, unsigned rank, int slice, const float4 (&x)[D]) {
  const int owner = lt / slice;
  const int lo = lt - owner * slice;
  const uint32_t addr = dsmem_addr(smem_u32(&recv[(static_cast<int>(rank) * slice + lo) * D]), owner);
#pragma unroll
  for (int f = 0; f < D; ++f) st_dsmem_f4(addr + 16u * f, x[f]);
}

// The 2D double-single values w[] of one target packed as D float4.
template <int D>
__device__ __forceinline__ void pack_ds(const ds (&w)[2 * D], float4 (&x)[D]) {
#pragma unroll
  for (int f = 0; f < D; ++f) x[f] = make_float4(w[2 * f].hi, w[2 * f].lo, w[2 * f + 1].hi, w[2 * f + 1].lo);
}

// ---------------------------------------------------------------- host
// Kernels already allowed clusters of up to 16 CTAs (one set per process).
inline std::mutex& attr_mutex() {
  static std::mutex m;
  return m;
}
inline std::set<const void*>& attr_done() {
  static std::set<const void*> s;
  return s;
}

// Launch attributes of a step kernel: cluster shape, the scheduling policy
// if one is set, and programmatic dependent launch.  Returns their count.
inline unsigned cluster_attrs(cudaLaunchAttribute* at, int cluster, bool pdl, int policy) {
  const int forced = forced_cluster_policy();
  if (forced >= 0) policy = forced;
  unsigned k = 0;
  at[k].id = cudaLaunchAttributeClusterDimension;
  at[k].val.clusterDim.x = cluster;
  at[k].val.clusterDim.y = 1;
  at[k].val.clusterDim.z = 1;
  ++k;
  if (policy == 1 || policy == 2) {
    at[k].id = cudaLaunchAttributeClusterSchedulingPolicyPreference;
    at[k].val.clusterSchedulingPolicyPreference =
        policy == 1 ? cudaClusterSchedulingPolicySpread : cudaClusterSchedulingPolicyLoadBalancing;
    ++k;
  }
  if (pdl) {
    at[k].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[k].val.programmaticStreamSerializationAllowed = 1;
    ++k;
  }
  return k;
}

template <typename K>
cudaError_t allow_large_clusters(K kern) {
  std::lock_guard<std::mutex> lk(attr_mutex());
  const void* key = reinterpret_cast<const void*>(kern);
  if (!attr_done().count(key)) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    attr_done().insert(key);
  }
  return cudaSuccess;
}

template <typename K>
cudaError_t occupancy_clusters(K kern, int threads, int cluster, int* out) {
  cudaError_t e = allow_large_clusters(kern);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster, 4096);
  cfg.blockDim = dim3(threads);
  cudaLaunchAttribute at[3];
  cfg.attrs = at;
  cfg.numAttrs = cluster_attrs(at, cluster, false, 0);
  return cudaOccupancyMaxActiveClusters(out, kern, &cfg);
}

template <typename K, typename A>
cudaError_t launch_cluster(K kern, const StepConfig& c, const A& args, cudaStream_t st, bool pdl) {
  const cudaError_t e = allow_large_clusters(kern);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c.cluster, c.tiles);
  cfg.blockDim = dim3(c.threads);
  cfg.stream = st;
  cudaLaunchAttribute at[3];
  cfg.attrs = at;
  cfg.numAttrs = cluster_attrs(at, c.cluster, pdl, c.policy);
  return cudaLaunchKernelEx(&cfg, kern, args);
}

}  // namespace gs
