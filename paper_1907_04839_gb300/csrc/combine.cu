// O(N) kernels around the pair sums.  This file holds:
//  * packing of the (N,3) inputs;
//  * the split combine followed by the Euler update (Algorithm 1,
//    lines 7-8 and 14-15);
//  * the loss of Eq. 3 with the adjoint initialisation;
//  * the gradient assembly.
//
// Numerics.  Per target, the source-split partials are summed in
// double-single FP32 arithmetic (TwoSum), in split order, so the result is
// deterministic.  The combined value is then converted to FP64, and the
// FP64 master state is updated.  The FP64 pipe of this part runs at about
// 1/80 of the FP32 rate, so FP64 is kept to a few operations per landmark
// coordinate and stays out of the S-way reduction.  The loss and H0 are
// reduced in FP64 in a fixed order: a warp tree per CTA, then one warp over
// the CTA partials, with the last CTA chosen by a ticket.
#include <cmath>

#include "gs_device.cuh"
#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kThreads = 128;

__device__ __forceinline__ bool finite64(double x) { return isfinite(x); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA in a fixed order; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

__device__ __forceinline__ ds load_ds(float2 v) { return ds{v.x, v.y}; }

__global__ void __launch_bounds__(kThreads) k_pack(PackArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * a.n) return;
  const int i = t / 3, k = t - 3 * i;
  const float q = a.q[t];
  const float p = a.p ? a.p[t] : 0.f;
  const float tg = a.tgt ? a.tgt[t] : 0.f;
  if (!isfinite(q) || !isfinite(p) || !isfinite(tg)) atomicOr(a.status, kErrNonFinite);
  a.q64[t] = q;
  a.p64[t] = p;
  if (a.t64) a.t64[t] = tg;
  reinterpret_cast<float*>(a.q4)[4 * i + k] = (float)(a.kq * (double)q);
  reinterpret_cast<float*>(a.p4)[4 * i + k] = p;
}

__global__ void __launch_bounds__(kThreads) k_combine_forward(CombineFwdArgs a) {
  __shared__ double sh[kThreads / 32];
  __shared__ int am_last;
  pdl_wait();  // the pair-sum partials of this step must be complete
  pdl_launch_dependents();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double hc = 0.0, mc = 0.0;
  if (t < 3 * a.n) {
    const int i = t / 3, k = t - 3 * i;
    ds hp{0.f, 0.f}, hq{0.f, 0.f};
    const Partial* pp = a.part + i;
    for (int s = 0; s < a.splits; ++s) {
      const float2* c = pp[static_cast<size_t>(s) * a.npad].c;
      hp = ds_add(hp, load_ds(c[k]));
      hq = ds_add(hq, load_ds(c[3 + k]));
    }
    const double Hp = ds_to_double(hp), Hq = ds_to_double(hq);
    const double p_old = a.p64[t];
    const double q = a.q64[t] + a.dt * Hp;
    const double p = p_old - a.dt * Hq;
    if (!finite64(q) || !finite64(p)) atomicOr(a.status, kErrNonFinite);
    if (a.first) {
      a.hp0[t] = Hp;
      a.hq0[t] = Hq;
      hc = 0.5 * p_old * Hp;
    }
    a.q64[t] = q;
    a.p64[t] = p;
    reinterpret_cast<float*>(a.q4_next)[4 * i + k] = (float)(a.kq * q);
    reinterpret_cast<float*>(a.p4_next)[4 * i + k] = (float)p;
    if (a.last && a.with_loss) {
      const double r = q - a.t64[t];
      mc = r * r;
      const double al = 2.0 * a.lambda * r;
      a.a64[t] = al;
      a.b64[t] = 0.0;
      reinterpret_cast<float*>(a.a4)[4 * i + k] = (float)al;
      reinterpret_cast<float*>(a.b4)[4 * i + k] = 0.f;
    }
  }
  const bool reduce_h = a.first != 0;
  const bool reduce_m = a.last && a.with_loss;
  if (!reduce_h && !reduce_m) return;  // uniform across the grid
  const double bh = block_sum(hc, sh);
  const double bm = block_sum(mc, sh);
  if (threadIdx.x == 0) {
    a.red_h[blockIdx.x] = bh;
    a.red_m[blockIdx.x] = bm;
    __threadfence();
    const unsigned tk = atomicAdd(a.ticket, 1u);
    am_last = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last || threadIdx.x >= 32) return;
  __threadfence();
  double h = 0.0, m = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += 32) {
    h += *((volatile double*)&a.red_h[b]);
    m += *((volatile double*)&a.red_m[b]);
  }
  h = warp_sum(h);
  m = warp_sum(m);
  if (threadIdx.x == 0) {
    if (reduce_h) a.scalars[0] = h;
    if (reduce_m) a.scalars[1] = (reduce_h ? h : a.scalars[0]) + a.lambda * m;
    *a.ticket = 0u;
  }
}

__global__ void __launch_bounds__(kThreads) k_combine_backward(CombineBwdArgs a) {
  pdl_wait();
  pdl_launch_dependents();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * a.n) return;
  const int i = t / 3, k = t - 3 * i;
  ds da{0.f, 0.f}, db{0.f, 0.f};
  const Partial* pp = a.part + i;
  for (int s = 0; s < a.splits; ++s) {
    const float2* c = pp[static_cast<size_t>(s) * a.npad].c;
    da = ds_add(da, load_ds(c[k]));
    db = ds_add(db, load_ds(c[3 + k]));
  }
  const double al = a.a64[t] + a.dt * ds_to_double(da);
  const double be = a.b64[t] + a.dt * ds_to_double(db);
  if (!finite64(al) || !finite64(be)) atomicOr(a.status, kErrNonFinite);
  a.a64[t] = al;
  a.b64[t] = be;
  reinterpret_cast<float*>(a.a4)[4 * i + k] = (float)al;
  reinterpret_cast<float*>(a.b4)[4 * i + k] = (float)(a.kappa * be);
  if (a.first) {
    if (a.grad_p0) a.grad_p0[t] = (float)(be + a.hp0[t]);
    if (a.grad_q0) a.grad_q0[t] = (float)(al + a.hq0[t]);
  }
}

__global__ void __launch_bounds__(kThreads) k_unpack(UnpackArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < a.n3) a.out[t] = (float)a.x64[t];
}

__global__ void __launch_bounds__(kThreads) k_partials_to_out(const Partial* part, int splits, int n, int npad,
                                                              float* out_a, float* out_b) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * n) return;
  const int i = t / 3, k = t - 3 * i;
  ds x{0.f, 0.f}, y{0.f, 0.f};
  for (int s = 0; s < splits; ++s) {
    const float2* c = part[static_cast<size_t>(s) * npad + i].c;
    x = ds_add(x, load_ds(c[k]));
    y = ds_add(y, load_ds(c[3 + k]));
  }
  out_a[t] = (float)ds_to_double(x);
  out_b[t] = (float)ds_to_double(y);
}

__global__ void __launch_bounds__(kThreads) k_to_float4(const float* x, float4* x4, int n, int npad,
                                                        double scale, unsigned* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (i < n) {
    const float a = x[3 * i], b = x[3 * i + 1], c = x[3 * i + 2];
    if (!isfinite(a) || !isfinite(b) || !isfinite(c)) atomicOr(status, kErrNonFinite);
    v = make_float4((float)(scale * a), (float)(scale * b), (float)(scale * c), 0.f);
  }
  x4[i] = v;
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

cudaError_t launch_pack(const PackArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  k_pack<<<blocks_for(3LL * a.n), kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_combine_forward(const CombineFwdArgs& a, cudaStream_t st, bool pdl, int* grid_out) {
  const int grid = blocks_for(3LL * a.n);
  if (grid_out) *grid_out = grid;
  return launch_ex(k_combine_forward, grid, a, st, pdl);
}

cudaError_t launch_combine_backward(const CombineBwdArgs& a, cudaStream_t st, bool pdl) {
  return launch_ex(k_combine_backward, blocks_for(3LL * a.n), a, st, pdl);
}

cudaError_t launch_unpack(const UnpackArgs& a, cudaStream_t st) {
  if (a.n3 <= 0) return cudaSuccess;
  k_unpack<<<blocks_for(a.n3), kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_partials_to_out(const Partial* part, int splits, int n, int npad,
                                   float* out_a, float* out_b, cudaStream_t st) {
  k_partials_to_out<<<blocks_for(3LL * n), kThreads, 0, st>>>(part, splits, n, npad, out_a, out_b);
  return cudaGetLastError();
}

cudaError_t launch_to_float4(const float* x, float4* x4, int n, int npad, double scale,
                             unsigned* status, cudaStream_t st) {
  k_to_float4<<<blocks_for(npad), kThreads, 0, st>>>(x, x4, n, npad, scale, status);
  return cudaGetLastError();
}

}  // namespace gs
