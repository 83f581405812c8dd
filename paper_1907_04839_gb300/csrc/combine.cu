// O(N) kernels around the pair sums: packing the (N,3) caller arrays (or
// (N,2) for planar landmarks) into the FP64 master state and the prescaled
// FP32 pair records, unpacking
// results, and summing split partials straight to (N,3) outputs for the
// single-step entry points.
//
// Split partials are summed in double-single FP32 arithmetic (TwoSum).
// Eight lanes share a landmark: each sums a lane-strided subset of the
// splits, then a fixed xor-butterfly joins them.  The order is fixed, so the
// result is deterministic.
#include <cmath>

#include "gs_device.cuh"
#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kThreads = 128;
constexpr int kGroup = 8;  // lanes that share one landmark's split partials


// One thread per coordinate of the (N, D) caller arrays.
template <int D>
__global__ void __launch_bounds__(kThreads) k_pack(PackArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= D * a.n) return;
  const int i = t / D, k = t - D * i;
  const float q = a.q[t];
  const double p = a.p64_in ? a.p64_in[t] : (a.p ? (double)a.p[t] : 0.0);
  const float tg = a.tgt ? a.tgt[t] : 0.f;
  if (!isfinite(q) || !isfinite(p) || !isfinite(tg)) atomicOr(a.status, kErrNonFinite);
  a.q64[t] = q;
  a.p64[t] = p;
  if (a.t64) a.t64[t] = tg;
  float* r = reinterpret_cast<float*>(a.qp + (i >> 1) * D) + 2 * k + (i & 1);
  r[0] = -(float)(a.kq * (double)q);
  r[2 * D] = (float)p;
}

template <int D>
__global__ void __launch_bounds__(kThreads) k_restore(const double* ckq, const double* ckp, double* q64,
                                                      double* p64, float4* rec, int n, double kq) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= D * n) return;
  const int i = t / D, k = t - D * i;
  const double q = ckq[t], p = ckp[t];
  q64[t] = q;
  p64[t] = p;
  float* r = reinterpret_cast<float*>(rec + (i >> 1) * D) + 2 * k + (i & 1);
  r[0] = -(float)(kq * q);
  r[2 * D] = (float)p;
}

// Sum the split partials of landmark i over a group of kGroup lanes: lane l
// takes splits l, l + kGroup, ..., then a fixed xor-butterfly combines the
// lanes.  Every lane of the group ends with the same six sums (TwoSum is
// commutative), and the result does not depend on timing.
__device__ __forceinline__ void group_partials(const Partial* part, int splits, int npad, int i, bool valid,
                                               int lane, ds acc[6]) {
#pragma unroll
  for (int c = 0; c < 6; ++c) acc[c] = ds{0.f, 0.f};
  if (valid) {
    const Partial* pp = part + i;
#pragma unroll 4
    for (int s = lane; s < splits; s += kGroup) {
      const float4* v = reinterpret_cast<const float4*>(pp + static_cast<size_t>(s) * npad);
      const float4 x = v[0], y = v[1], z = v[2];
      acc[0] = ds_add(acc[0], ds{x.x, x.y});
      acc[1] = ds_add(acc[1], ds{x.z, x.w});
      acc[2] = ds_add(acc[2], ds{y.x, y.y});
      acc[3] = ds_add(acc[3], ds{y.z, y.w});
      acc[4] = ds_add(acc[4], ds{z.x, z.y});
      acc[5] = ds_add(acc[5], ds{z.z, z.w});
    }
  }
#pragma unroll
  for (int o = kGroup / 2; o > 0; o >>= 1) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const float hi = __shfl_xor_sync(0xffffffffu, acc[c].hi, o);
      const float lo = __shfl_xor_sync(0xffffffffu, acc[c].lo, o);
      acc[c] = ds_add(acc[c], ds{hi, lo});
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_unpack(UnpackArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < a.n3) a.out[t] = (float)a.x64[t];
}

__global__ void __launch_bounds__(kThreads) k_partials_to_out(const Partial* part, int splits, int n, int npad,
                                                              float* out_a, float* out_b) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gt / kGroup, lane = gt % kGroup;
  const bool valid = i < n;
  ds acc[6];
  group_partials(part, splits, npad, i, valid, lane, acc);
  if (!valid || lane >= 6) return;
  const int k = lane % 3;
  if (lane < 3) out_a[3 * i + k] = (float)ds_to_double(acc[k]);
  else out_b[3 * i + k] = (float)ds_to_double(acc[3 + k]);
}

// One thread per landmark slot i < npad (padding written as zeros).
__global__ void __launch_bounds__(kThreads) k_to_records(const float* x, const float* y, float4* rec, int n, int npad,
                                                         double sx, double sy, int ab_layout, unsigned* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  float* r = reinterpret_cast<float*>(rec + (i >> 1) * kRecF4) + (i & 1);
  const float fx = ab_layout ? 1.f : -1.f, fy = ab_layout ? -1.f : 1.f;
  for (int k = 0; k < 3; ++k) {
    float a = 0.f, b = 0.f;
    if (i < n) {
      a = x[3 * i + k];
      b = y[3 * i + k];
      if (!isfinite(a) || !isfinite(b)) atomicOr(status, kErrNonFinite);
    }
    r[2 * k] = fx * (float)(sx * a);
    r[6 + 2 * k] = fy * (float)(sy * b);
  }
}

inline int blocks_for(long long n) { return static_cast<int>((n + kThreads - 1) / kThreads); }

template <typename K, typename A>
cudaError_t launch_ex(K kern, int grid, const A& args, cudaStream_t st, bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args);
}

}  // namespace

KernelScales make_scales(double sigma) {
  KernelScales k;
  k.kq = std::sqrt(0.5 / std::log(2.0)) / sigma;  // kq^2 = log2(e) / (2 sigma^2)
  k.s = 1.0 / (sigma * sigma);
  k.kappa = k.s / k.kq;
  return k;
}

int combine_threads() { return kThreads; }
int combine_group() { return kGroup; }

cudaError_t launch_pack(const PackArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  if (a.dim == 2)
    k_pack<2><<<blocks_for(2LL * a.n), kThreads, 0, st>>>(a);
  else
    k_pack<3><<<blocks_for(3LL * a.n), kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_restore(const double* ckq, const double* ckp, double* q64, double* p64, float4* rec, int n,
                           double kq, cudaStream_t st, int dim) {
  if (dim == 2)
    k_restore<2><<<blocks_for(2LL * n), kThreads, 0, st>>>(ckq, ckp, q64, p64, rec, n, kq);
  else
    k_restore<3><<<blocks_for(3LL * n), kThreads, 0, st>>>(ckq, ckp, q64, p64, rec, n, kq);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const UnpackArgs& a, cudaStream_t st) {
  if (a.n3 <= 0) return cudaSuccess;
  k_unpack<<<blocks_for(a.n3), kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_partials_to_out(const Partial* part, int splits, int n, int npad,
                                   float* out_a, float* out_b, cudaStream_t st) {
  k_partials_to_out<<<blocks_for((long long)kGroup * n), kThreads, 0, st>>>(part, splits, n, npad, out_a, out_b);
  return cudaGetLastError();
}

cudaError_t launch_to_records(const float* a, const float* b, float4* rec, int n, int npad, double sa, double sb,
                              int ab_layout, unsigned* status, cudaStream_t st) {
  k_to_records<<<blocks_for(npad), kThreads, 0, st>>>(a, b, rec, n, npad, sa, sb, ab_layout, status);
  return cudaGetLastError();
}

}  // namespace gs
