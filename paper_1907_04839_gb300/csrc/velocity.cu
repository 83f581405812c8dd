// The velocity field of Eq. 4 at arbitrary points, and points carried
// through the deformation by the flow.
//
// Eq. 4 extends the landmark motion to all of space:
//   v(x, t) = sum_l g(|q_l(t) - x|) p_l(t).
// Its pair sums are the Hp half of StepForward with query points as
// targets, so the kernel is built the same way: a cluster of C CTAs owns a
// tile of 256 query points (two per thread, so that each staged landmark
// record feeds two points), CTA r streams source split r of the landmark
// pair records through the shared-memory stage ring, and the C partial sums
// of each point meet in distributed shared memory in rank order.  One
// launch either writes v (velocity_field) or moves the points by one Euler
// step, x <- x + dt v (flow_points).  The points move with the landmark
// state of the same time step, exactly as the landmarks themselves do in
// the forward loop of Algorithm 1; a landmark used as a point therefore
// follows q(t).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <set>

#include "engine.h"
#include "pair_tile.cuh"

namespace gs {
namespace {

constexpr int kVT = 128;  // threads per CTA
constexpr int kVR = 2;    // query points per thread: a staged landmark record feeds kVR points

// Per query point x:  V = sum_j g(x, q_j) p_j  over the landmark pair
// records (negated prescaled positions, momenta).  A thread holds R points
// (base + r * stride).
template <int R>
struct VelTile {
  float2 q[R][3];  // prescaled points, duplicated for the paired lanes
  float sF[R][3], cF[R][3];

  __device__ __forceinline__ void load(const double* x64, int base, int stride, int m, double kq) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = base + r * stride;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float v = i < m ? static_cast<float>(kq * x64[3 * static_cast<size_t>(i) + k]) : 0.f;
        q[r][k] = dup(v);
        sF[r][k] = cF[r][k] = 0.f;
      }
    }
  }

  // Sources [lo, hi) of the staged chunk; lo is a multiple of 8.
  __device__ __forceinline__ void consume(const float4* const* bufs, int lo, int hi) {
    const float4* Q = bufs[0];
    for (int sb = lo; sb < hi; sb += kSub) {
      const int sl = min(kSub, hi - sb);
      float2 a[R][3];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) a[r][k] = make_float2(0.f, 0.f);
      for (int jj = 0; jj < sl; jj += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll / 2; ++u) {
          float2 v[6];  // v[k] = -q~_j, v[3 + k] = p_j
          rec_split<3>(Q + ((sb + jj) / 2 + u) * kRecF4, v);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float2 dx = __fadd2_rn(q[r][0], v[0]);
            const float2 dy = __fadd2_rn(q[r][1], v[1]);
            const float2 dz = __fadd2_rn(q[r][2], v[2]);
            float2 r2 = __fmul2_rn(dx, dx);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            const float2 g = gauss2(r2);
            a[r][0] = __ffma2_rn(g, v[3], a[r][0]);
            a[r][1] = __ffma2_rn(g, v[4], a[r][1]);
            a[r][2] = __ffma2_rn(g, v[5], a[r][2]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) kahan_add(sF[r][k], cF[r][k], __fadd_rn(a[r][k].x, a[r][k].y));
    }
  }
};

struct VelArgs {
  const float4* qp;  // QP pair records of the landmark state (npad landmarks)
  double* x64;       // points, FP64 (m x 3); moved in place when v_out is null
  float* v_out;      // velocity out (m x 3), or null for an Euler step
  int m, npad, split_len;
  double kq, dt;
  unsigned* status;
};

constexpr int kVM = kVT * kVR;  // query points per CTA

__global__ void __launch_bounds__(kVT) k_velocity(VelArgs a) {
  union Smem {
    StageBuf<1> st;
    float4 red[kVM][2];  // (V0 hi, lo, V1 hi, lo), (V2 hi, lo, -, -) per point
  };
  __shared__ __align__(128) Smem sm;
  __shared__ __align__(8) Pipe pp;

  const unsigned rank = cluster_rank(), C = cluster_size();
  // Same outcome in every CTA of a cluster: a bad launch leaves before any barrier.
  if (blockDim.x != kVT || kVM % static_cast<int>(C) != 0 || (a.split_len & 7) != 0 ||
      static_cast<long long>(a.split_len) * C < a.npad) {
    if (threadIdx.x == 0) atomicOr(a.status, kErrBadLaunch);
    return;
  }
  const int j0 = min(static_cast<int>(rank) * a.split_len, a.npad);
  const int j1 = min(j0 + a.split_len, a.npad);
  if (threadIdx.x == 0) pipe_init(pp, kVT / 32);
  __syncthreads();
  pdl_wait();  // the previous step's points must be complete

  const int tile0 = blockIdx.y * kVM;
  VelTile<kVR> t;
  t.load(a.x64, tile0 + static_cast<int>(threadIdx.x), kVT, a.m, a.kq);
  const float4* src[1] = {a.qp};
  stream_sources<1>(sm.st, pp, src, j0, j1, t, a.status);  // ends with a CTA barrier
#pragma unroll
  for (int r = 0; r < kVR; ++r) {
    const ds f0 = ds_from_kahan(t.sF[r][0], t.cF[r][0]);
    const ds f1 = ds_from_kahan(t.sF[r][1], t.cF[r][1]);
    const ds f2 = ds_from_kahan(t.sF[r][2], t.cF[r][2]);
    const int lt = static_cast<int>(threadIdx.x) + r * kVT;
    sm.red[lt][0] = make_float4(f0.hi, f0.lo, f1.hi, f1.lo);
    sm.red[lt][1] = make_float4(f2.hi, f2.lo, 0.f, 0.f);
  }
  cluster_sync();  // every CTA's partials are visible to the cluster

  const int slice = kVM / static_cast<int>(C);
  for (int item = threadIdx.x; item < slice * 3; item += kVT) {
    const int lt = static_cast<int>(rank) * slice + item / 3;
    const int k = item % 3;
    const int i = tile0 + lt;
    if (i >= a.m) continue;
    const uint32_t lp = smem_u32(&sm.red[lt][0]);
    ds acc{0.f, 0.f};
#pragma unroll 4
    for (unsigned rr = 0; rr < C; ++rr) {
      const float2 x = ld_dsmem_f2(dsmem_addr(lp, rr) + 8u * k);
      acc = ds_add(acc, ds{x.x, x.y});
    }
    const double vel = ds_to_double(acc);
    const size_t tt = 3 * static_cast<size_t>(i) + k;
    if (a.v_out) {
      if (!isfinite(vel)) atomicOr(a.status, kErrNonFinite);
      a.v_out[tt] = static_cast<float>(vel);
    } else {
      const double xn = a.x64[tt] + a.dt * vel;
      if (!isfinite(xn)) atomicOr(a.status, kErrNonFinite);
      a.x64[tt] = xn;
    }
  }
  cluster_sync();  // peers may still be reading this CTA's partials
}

__global__ void k_points_to64(const float* x, double* x64, size_t n3) {
  for (size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; t < n3;
       t += static_cast<size_t>(gridDim.x) * blockDim.x)
    x64[t] = x[t];
}

__global__ void k_points_to32(const double* x64, float* x, size_t n3) {
  for (size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; t < n3;
       t += static_cast<size_t>(gridDim.x) * blockDim.x)
    x[t] = static_cast<float>(x64[t]);
}

int conv_blocks(size_t n3) { return static_cast<int>(std::min<size_t>((n3 + 255) / 256, 4096)); }

// Launch shape: tiles of 128 points; the cluster size C (a power of two,
// at most 16) splits the landmarks so that the grid reaches about two
// waves when the points alone do not.
struct VelConfig {
  int tiles, cluster, split_len, policy;
};

VelConfig vel_config(int m, int npad, int num_sms) {
  VelConfig c{};
  c.tiles = (m + kVM - 1) / kVM;
  const int want = (2 * num_sms + c.tiles - 1) / c.tiles;
  const int cap = std::max(1, std::min(16, npad / 128));
  c.cluster = 1;
  while (c.cluster < want && c.cluster * 2 <= cap) c.cluster *= 2;
  const int len = (npad + c.cluster - 1) / c.cluster;
  c.split_len = (len + kUnroll - 1) / kUnroll * kUnroll;
  c.policy = policy_for_grid(static_cast<long long>(c.tiles) * c.cluster, num_sms);
  return c;
}

std::mutex g_vel_attr_mu;
bool g_vel_attr_done = false;

cudaError_t launch_velocity(const VelConfig& c, const VelArgs& a, cudaStream_t st, bool pdl) {
  {
    std::lock_guard<std::mutex> lk(g_vel_attr_mu);
    if (!g_vel_attr_done) {
      const cudaError_t e = cudaFuncSetAttribute(k_velocity, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
      g_vel_attr_done = true;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c.cluster, c.tiles);
  cfg.blockDim = dim3(kVT);
  cfg.stream = st;
  cudaLaunchAttribute at[3];
  unsigned k = 0;
  at[k].id = cudaLaunchAttributeClusterDimension;
  at[k].val.clusterDim.x = c.cluster;
  at[k].val.clusterDim.y = 1;
  at[k].val.clusterDim.z = 1;
  ++k;
  at[k].id = cudaLaunchAttributeClusterSchedulingPolicyPreference;
  at[k].val.clusterSchedulingPolicyPreference =
      c.policy == 2 ? cudaClusterSchedulingPolicyLoadBalancing : cudaClusterSchedulingPolicySpread;
  ++k;
  if (pdl) {
    at[k].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[k].val.programmaticStreamSerializationAllowed = 1;
    ++k;
  }
  cfg.attrs = at;
  cfg.numAttrs = k;
  return cudaLaunchKernelEx(&cfg, k_velocity, a);
}

// Room for m points (FP64 state and FP32 staging in and out).
gs_status reserve_points(Workspace& w, int m) {
  if (m <= w.cap_pts) return GS_OK;
  for (void* p : w.pt_allocs) cudaFree(p);
  w.pt_allocs.clear();
  w.cap_pts = 0;
  const size_t n3 = 3 * static_cast<size_t>(m);
  void* v = nullptr;
  GS_CUDA(cudaMalloc(&v, n3 * sizeof(double) + 256));
  w.pt_allocs.push_back(v);
  w.pts64 = static_cast<double*>(v);
  GS_CUDA(cudaMalloc(&v, n3 * sizeof(float) + 256));
  w.pt_allocs.push_back(v);
  w.pts_in = static_cast<float*>(v);
  GS_CUDA(cudaMalloc(&v, n3 * sizeof(float) + 256));
  w.pt_allocs.push_back(v);
  w.pts_out = static_cast<float*>(v);
  w.cap_pts = m;
  return GS_OK;
}

gs_status check_points(int64_t M, const float* x, const void* out) {
  if (M < 1 || M > (1LL << 26)) return fail(GS_EINVAL, "M must be in [1, 2^26]");
  if (!x || !out) return fail(GS_EINVAL, "point arrays must not be NULL");
  return GS_OK;
}

}  // namespace
}  // namespace gs

extern "C" gs_status velocity_field(int64_t N, int64_t M, double sigma, const float* q, const float* p,
                                    const float* x, float* v, void* stream) {
  using namespace gs;
  set_last_error("");
  if (N < 1 || N > (1LL << 26)) return fail(GS_EINVAL, "N must be in [1, 2^26]");
  if (!(sigma > 0.0) || !std::isfinite(sigma)) return fail(GS_EINVAL, "sigma must be finite and > 0");
  if (!q || !p) return fail(GS_EINVAL, "q and p must not be NULL");
  gs_status s = check_points(M, x, v);
  if (s != GS_OK) return s;
  std::lock_guard<std::mutex> lk(engine_mutex());
  Workspace* w = nullptr;
  if ((s = get_workspace(&w)) != GS_OK) return s;
  const int n = static_cast<int>(N), m = static_cast<int>(M), npad = round_up(n, kPad);
  if ((s = reserve(*w, npad, 1, 1)) != GS_OK) return s;
  if ((s = reserve_points(*w, m)) != GS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t n3 = 3 * static_cast<size_t>(n), m3 = 3 * static_cast<size_t>(m);
  bool host = false;
  const float *dq = nullptr, *dp = nullptr, *dx = nullptr;
  if ((s = stage_in(q, w->in_q, n3, st, &dq, &host)) != GS_OK) return s;
  if ((s = stage_in(p, w->in_p, n3, st, &dp, &host)) != GS_OK) return s;
  if ((s = stage_in(x, w->pts_in, m3, st, &dx, &host)) != GS_OK) return s;
  const KernelScales sc = make_scales(sigma);
  GS_CUDA(launch_to_records(dq, dp, w->traj, n, npad, sc.kq, 1.0, 0, w->status, st));
  w->clean_n = -1;  // record slot 0 was overwritten
  k_points_to64<<<conv_blocks(m3), 256, 0, st>>>(dx, w->pts64, m3);
  GS_CUDA(cudaGetLastError());
  const VelConfig c = vel_config(m, npad, w->num_sms);
  VelArgs a{w->traj, w->pts64, w->pts_out, m, npad, c.split_len, sc.kq, 0.0, w->status};
  GS_CUDA(launch_velocity(c, a, st, false));
  bool want_sync = host;
  if ((s = copy_out(v, w->pts_out, m3, st, &want_sync)) != GS_OK) return s;
  if (want_sync) return finish_sync(*w, st);
  return GS_OK;
}

extern "C" gs_status flow_points(const gs_params* prm, const float* q0, const float* p0, int64_t M,
                                 const float* x0, float* x1, void* stream) {
  using namespace gs;
  set_last_error("");
  gs_status s = check_params(prm);
  if (s != GS_OK) return s;
  if (!q0 || !p0) return fail(GS_EINVAL, "q0 and p0 must not be NULL");
  if (prm->integrator != GS_EULER) return fail(GS_EINVAL, "flow_points takes Euler steps only (integrator GS_EULER)");
  if (dim_of(*prm) != 3) return fail(GS_EINVAL, "flow_points is 3-D only (dim 3)");
  if ((s = check_points(M, x0, x1)) != GS_OK) return s;
  std::lock_guard<std::mutex> lk(engine_mutex());
  Workspace* w = nullptr;
  if ((s = get_workspace(&w)) != GS_OK) return s;
  const int n = static_cast<int>(prm->N), m = static_cast<int>(M), T = prm->T, npad = round_up(n, kPad);
  if ((s = reserve(*w, npad, record_slots(T, 0), 1, 0)) != GS_OK) return s;
  if ((s = reserve_points(*w, m)) != GS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((s = ensure_clean(*w, n, st)) != GS_OK) return s;
  const size_t n3 = 3 * static_cast<size_t>(n), m3 = 3 * static_cast<size_t>(m);
  bool host = false;
  const float *dq = nullptr, *dp = nullptr, *dx = nullptr;
  if ((s = stage_in(q0, w->in_q, n3, st, &dq, &host)) != GS_OK) return s;
  if ((s = stage_in(p0, w->in_p, n3, st, &dp, &host)) != GS_OK) return s;
  if ((s = stage_in(x0, w->pts_in, m3, st, &dx, &host)) != GS_OK) return s;
  // The forward flow: record slot k of the trajectory holds the landmark
  // state of step k.
  const KernelScales sc = make_scales(prm->sigma);
  PackArgs pk;
  pk.q = dq;
  pk.p = dp;
  pk.p64_in = nullptr;
  pk.tgt = nullptr;
  pk.q64 = w->q64;
  pk.p64 = w->p64;
  pk.t64 = nullptr;
  pk.qp = w->traj;
  pk.n = n;
  pk.kq = sc.kq;
  pk.status = w->status;
  pk.dim = 3;
  GS_CUDA(launch_pack(pk, st));
  cudaGraphExec_t ge = nullptr;
  if ((s = get_graph(*w, GraphKey{0, n, T, prm->sigma, 0.0, 0, w->phase_timing}, &ge)) != GS_OK) return s;
  GS_CUDA(cudaGraphLaunch(ge, st));
  // T Euler steps of the points, each with that step's landmark state.
  k_points_to64<<<conv_blocks(m3), 256, 0, st>>>(dx, w->pts64, m3);
  GS_CUDA(cudaGetLastError());
  const VelConfig c = vel_config(m, npad, w->num_sms);
  for (int k = 0; k < T; ++k) {
    VelArgs a{w->traj + static_cast<size_t>(k) * w->slot(), w->pts64, nullptr, m, npad, c.split_len, sc.kq,
              1.0 / T, w->status};
    GS_CUDA(launch_velocity(c, a, st, k > 0));
  }
  k_points_to32<<<conv_blocks(m3), 256, 0, st>>>(w->pts64, w->pts_out, m3);
  GS_CUDA(cudaGetLastError());
  bool want_sync = host;
  if ((s = copy_out(x1, w->pts_out, m3, st, &want_sync)) != GS_OK) return s;
  if (want_sync) return finish_sync(*w, st);
  return GS_OK;
}
