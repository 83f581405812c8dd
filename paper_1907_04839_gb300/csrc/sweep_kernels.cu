// Persistent sweeps: one launch runs every time step of the forward loop of
// Algorithm 1 (StepForward + Euler update, T times) or of its reverse loop
// (StepBackward + adjoint update, T times).
//
// The per-step kernels (step_kernels.cu) pay, at every step, for a grid
// launch and drain, the reload of the FP64 state their epilogue updates, and
// the start-up of their copy pipelines.  At a few thousand landmarks a step
// is a partial wave of about 30 us, and those fixed costs are a large share
// of it.  Here the clusters keep their roles (cluster = target tile, CTA
// rank = source split, slice of the tile reduced and updated per CTA) for
// all T steps:
//  * the FP64 state of a CTA's slice stays in registers, one (landmark,
//    coordinate) item per thread;
//  * the bulk-copy ring runs on across steps (its mbarrier phases continue);
//  * split partials meet in the reducing CTA's shared memory (remote
//    stores, one cluster barrier), in rank order, as in the per-step kernels,
//    so each step's result is bitwise that of the per-step kernel of the
//    same shape;
//  * between steps the grid meets at a barrier: the CTAs of a cluster
//    synchronise, the cluster's first CTA adds one arrival to a counter in
//    global memory and polls it, and hands the outcome to every CTA of its
//    cluster before a second cluster barrier.
// A grid barrier only works if every cluster is resident at once.  The host
// launches this form only when the occupancy calculator says they all fit
// (sweep_fits).  Every wait is still bounded: a barrier that has not
// completed after one second of global time records kErrTimeout, and the
// clusters leave together at that barrier (all CTAs of a cluster read the
// same outcome), so no CTA touches a peer that has exited.
#include <map>
#include <mutex>
#include <utility>

#include "step_common.cuh"

namespace gs {

namespace {

// Grid barrier number b of the launch: returns true when every cluster has
// arrived, false if the wait expired or a wait anywhere in the grid has
// (the kErrTimeout bit of the status word).  All threads of every CTA of the
// cluster call it.  `go` is a shared-memory word of each CTA.
__device__ __forceinline__ bool sweep_barrier(unsigned* count, unsigned target, unsigned* status, int* go,
                                              unsigned rank, unsigned C) {
  cluster_sync();  // the cluster's record stores happen before its arrival
  if (rank == 0 && threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    bool ok = false;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0;; ++it) {
      if (ld_acquire_gpu(count) >= target) {
        ok = true;
        break;
      }
      if ((it & 63u) == 63u && global_ns() - t0 > kWaitNs) break;
    }
    __threadfence();
    if (!ok) atomicOr(status, kErrTimeout);
    const unsigned g = ok && !(*reinterpret_cast<volatile unsigned*>(status) & kErrTimeout) ? 1u : 0u;
    for (unsigned r = 0; r < C; ++r) st_dsmem_u32(dsmem_addr(smem_u32(go), r), g);
  }
  cluster_sync();  // the outcome has reached every CTA of the cluster
  return *reinterpret_cast<volatile int*>(go) != 0;
}

// Add the C split partials (double-single, rank order) of slice item
// (ll, k): returns the two sums (Hp, Hq forward; dalpha, dbeta reverse).
template <int D>
__device__ __forceinline__ void combine_recv(const float4* recv, int ll, int k, unsigned C, int slice, ds& x0,
                                             ds& x1) {
  x0 = ds{0.f, 0.f};
  x1 = ds{0.f, 0.f};
#pragma unroll 4
  for (unsigned rr = 0; rr < C; ++rr) {
    const float2* rp = reinterpret_cast<const float2*>(&recv[(static_cast<int>(rr) * slice + ll) * D]);
    const float2 x = rp[k];
    const float2 y = rp[D + k];
    x0 = ds_add(x0, ds{x.x, x.y});
    x1 = ds_add(x1, ds{y.x, y.y});
  }
}

// The launch must match the kernel: NT threads, at most one CTA per target
// of the tile, at least 4 CTAs per cluster (so that a CTA's slice has at
// most one item per thread), splits (multiples of 8 sources) that cover the
// problem.  The outcome is the same in every CTA of the grid, so a bad
// launch leaves before any barrier.
template <int NT, int D>
__device__ __forceinline__ bool sweep_launch_ok(const SweepArgs& a, unsigned C) {
  const int slice = (NT + static_cast<int>(C) - 1) / static_cast<int>(C);
  return blockDim.x == NT && static_cast<int>(C) <= NT && slice * D <= NT && (a.split_len & 7) == 0 &&
         static_cast<long long>(a.split_len) * C >= a.npad;
}

// ---------------------------------------------------------------- forward sweep
template <int NT, int D = 3>
__global__ void __launch_bounds__(NT) k_sweep_forward(SweepArgs a) {
  constexpr int M = NT;  // one target per thread
  __shared__ __align__(128) StageBuf<1, D> st;
  __shared__ __align__(16) float4 recv[(M + 15) * D];
  __shared__ __align__(8) Pipe pp;
  __shared__ int go;
  __shared__ double shred[NT / 32];
  __shared__ int am_last;

  const unsigned rank = cluster_rank(), C = cluster_size();
  if (!sweep_launch_ok<NT, D>(a, C)) {
    if (threadIdx.x == 0) atomicOr(a.status, kErrBadLaunch);
    return;
  }
  cluster_arrive_relaxed();  // the first push waits for every peer's arrival
  const int lim = a.npad;
  const int j0 = min(static_cast<int>(rank) * a.split_len, lim);
  const int j1 = min(j0 + a.split_len, lim);
  const int nch = j1 > j0 ? (j1 - j0 + kChunk - 1) / kChunk : 0;
  if (threadIdx.x == 0) pipe_init(pp, NT / 32);
  __syncthreads();
  pdl_wait();

  const int tile = blockIdx.y, tile0 = tile * M;
  const int slice = (M + static_cast<int>(C) - 1) / static_cast<int>(C);
  const unsigned nclusters = gridDim.y;
  // This thread's item of the CTA's slice: landmark i, coordinate kc.
  const int ll = static_cast<int>(threadIdx.x) / D, kc = static_cast<int>(threadIdx.x) % D;
  const int lt = static_cast<int>(rank) * slice + ll;
  const bool mine = static_cast<int>(threadIdx.x) < slice * D && lt < M && tile0 + lt < a.n;
  const int i = tile0 + lt;
  const int tt = D * i + kc;
  double q = 0.0, p = 0.0;
  if (mine) {
    q = a.q64[tt];
    p = a.p64[tt];
  }
  double hc = 0.0, mc = 0.0;
  int base = 0;
  for (int k = 0; k < a.T; ++k) {
    const float4* qp = a.traj + static_cast<long long>(k) * a.slot;
    FwdTile<1, D> t;
    t.load(qp, tile0 + static_cast<int>(threadIdx.x), M, lim);
    if (threadIdx.x == 0) fence_proxy_async_global();  // the grid's record stores before these copies
    const float4* src[1] = {qp};
    stream_sources<1, 1, D>(st, pp, src, j0, j1, t, a.status, 0, base);  // ends with a CTA barrier
    base += nch;
    if (k == 0) cluster_wait();  // every peer's receive buffer exists
    {
      ds w[2 * D];
      t.result(0, a.kappa_f, w);
      float4 x[D];
      pack_ds<D>(w, x);
      push_partials<D>(recv, static_cast<int>(threadIdx.x), rank, slice, x);
    }
    cluster_sync();  // every split's partials have reached the CTA that reduces them
    if (mine) {
      ds hp, hq;
      combine_recv<D>(recv, ll, kc, C, slice, hp, hq);
      const double Hp = ds_to_double(hp), Hq = ds_to_double(hq);
      if (k == 0) {
        hc += 0.5 * p * Hp;  // H0 = 1/2 sum_i p0_i . Hp_i(q0, p0)
        a.hp0[tt] = Hp;
        a.hq0[tt] = Hq;
      }
      q = q + a.dt * Hp;
      p = p - a.dt * Hq;
      if (!isfinite(q) || !isfinite(p)) atomicOr(a.status, kErrNonFinite);
      float* qn = reinterpret_cast<float*>(a.traj + static_cast<long long>(k + 1) * a.slot + (i >> 1) * D) +
                  2 * kc + (i & 1);
      qn[0] = -(float)(a.kq * q);
      qn[2 * D] = (float)p;
      if (k + 1 == a.T) {
        a.q64[tt] = q;
        a.p64[tt] = p;
        if (a.with_loss) {
          const double r = q - a.t64[tt];
          mc += r * r;
          const double al = 2.0 * a.lambda * r;
          a.a64[tt] = al;
          a.b64[tt] = 0.0;
          float* an = reinterpret_cast<float*>(a.adj + (i >> 1) * D) + 2 * kc + (i & 1);
          an[0] = (float)al;
          an[2 * D] = 0.f;
        }
      }
      fence_proxy_async_global();  // these records are read by bulk copies next step
    }
    if (k + 1 < a.T && !sweep_barrier(a.bar, (k + 1) * nclusters, a.status, &go, rank, C)) return;
  }
  double h, m;
  if (grid_sum2(hc, mc, a.red_h, a.red_m, a.ticket, shred, &am_last, &h, &m) && threadIdx.x == 0) {
    a.scalars[0] = h;
    if (a.with_loss) a.scalars[1] = h + a.lambda * m;
    *a.ticket = 0u;
  }
}

// ---------------------------------------------------------------- reverse sweep
template <int NT, int D = 3>
__global__ void __launch_bounds__(NT) k_sweep_backward(SweepArgs a) {
  constexpr int M = NT;
  __shared__ __align__(128) StageBuf<2, D> st;
  __shared__ __align__(16) float4 recv[(M + 15) * D];
  __shared__ __align__(8) Pipe pp;
  __shared__ int go;

  const unsigned rank = cluster_rank(), C = cluster_size();
  if (!sweep_launch_ok<NT, D>(a, C)) {
    if (threadIdx.x == 0) atomicOr(a.status, kErrBadLaunch);
    return;
  }
  cluster_arrive_relaxed();
  const int lim = a.npad;
  const int j0 = min(static_cast<int>(rank) * a.split_len, lim);
  const int j1 = min(j0 + a.split_len, lim);
  const int nch = j1 > j0 ? (j1 - j0 + kChunk - 1) / kChunk : 0;
  if (threadIdx.x == 0) pipe_init(pp, NT / 32);
  __syncthreads();
  pdl_wait();

  const int tile = blockIdx.y, tile0 = tile * M;
  const int slice = (M + static_cast<int>(C) - 1) / static_cast<int>(C);
  const unsigned nclusters = gridDim.y;
  const int ll = static_cast<int>(threadIdx.x) / D, kc = static_cast<int>(threadIdx.x) % D;
  const int lt = static_cast<int>(rank) * slice + ll;
  const bool mine = static_cast<int>(threadIdx.x) < slice * D && lt < M && tile0 + lt < a.n;
  const int i = tile0 + lt;
  const int tt = D * i + kc;
  double al = 0.0, be = 0.0;  // the adjoint of the current step's end state
  if (mine) {
    al = a.a64[tt];
    be = a.b64[tt];
  }
  int base = 0;
  for (int s = 0; s < a.T; ++s) {
    const int k = a.T - 1 - s;
    const float4* qp = a.traj + static_cast<long long>(k) * a.slot;
    const float4* ab = a.adj + (s & 1) * a.slot;
    BwdTile<1, D> t;
    t.load(qp, ab, tile0 + static_cast<int>(threadIdx.x), M, lim);
    if (threadIdx.x == 0) fence_proxy_async_global();
    const float4* src[2] = {qp, ab};
    stream_sources<2, 1, D>(st, pp, src, j0, j1, t, a.status, 0, base);
    base += nch;
    if (s == 0) cluster_wait();
    {
      ds w[2 * D];
      t.result(0, a.kq_f, a.kappa_f, w);
      float4 x[D];
      pack_ds<D>(w, x);
      push_partials<D>(recv, static_cast<int>(threadIdx.x), rank, slice, x);
    }
    cluster_sync();
    if (mine) {
      ds da, db;
      combine_recv<D>(recv, ll, kc, C, slice, da, db);
      al = al + a.dt * ds_to_double(da);
      be = be + a.dt * ds_to_double(db);
      if (!isfinite(al) || !isfinite(be)) atomicOr(a.status, kErrNonFinite);
      if (k > 0) {
        float* an = reinterpret_cast<float*>(a.adj + ((s + 1) & 1) * a.slot + (i >> 1) * D) + 2 * kc + (i & 1);
        an[0] = (float)al;
        an[2 * D] = -(float)(a.kappa * be);
        fence_proxy_async_global();
      } else {
        a.a64[tt] = al;
        a.b64[tt] = be;
        const double gp = be + a.hp0[tt];
        if (a.grad_p0) a.grad_p0[tt] = (float)gp;
        if (a.grad_p0_64) a.grad_p0_64[tt] = gp;
        if (a.grad_q0) a.grad_q0[tt] = (float)(al + a.hq0[tt]);
      }
    }
    if (s + 1 < a.T && !sweep_barrier(a.bar, (s + 1) * nclusters, a.status, &go, rank, C)) return;
  }
}

// ---------------------------------------------------------------- host side
using SweepKernel = void (*)(SweepArgs);

SweepKernel sweep_kernel_for(int kind, int threads) {
  if (kind == 0) {
    if (threads == 64) return k_sweep_forward<64>;
    if (threads == 128) return k_sweep_forward<128>;
    return nullptr;
  }
  if (threads == 32) return k_sweep_backward<32>;
  if (threads == 64) return k_sweep_backward<64>;
  return nullptr;
}

int g_sweep_mode = -1;
std::mutex g_fit_mu;
// ((device, kernel), cluster size) -> clusters of that kernel resident at once
std::map<std::pair<std::pair<int, const void*>, int>, int> g_fit;

}  // namespace

void set_sweep_mode(int mode) { g_sweep_mode = mode; }
int sweep_mode() { return g_sweep_mode; }

bool sweep_fits(int kind, const StepConfig& c) {
  if (g_sweep_mode == 0) return false;
  if (c.R != 1 || c.groups != 1 || c.cluster < 4 || c.cluster > 16 || c.cluster > c.threads) return false;
  if ((c.threads + c.cluster - 1) / c.cluster * 3 > c.threads) return false;
  const SweepKernel kern = sweep_kernel_for(kind, c.threads);
  if (!kern) return false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const auto key = std::make_pair(std::make_pair(dev, reinterpret_cast<const void*>(kern)), c.cluster);
  int resident = -1;
  {
    std::lock_guard<std::mutex> lk(g_fit_mu);
    const auto it = g_fit.find(key);
    if (it != g_fit.end()) resident = it->second;
  }
  if (resident < 0) {
    int clusters = 0;
    if (occupancy_clusters(kern, c.threads, c.cluster, &clusters) != cudaSuccess) {
      cudaGetLastError();
      clusters = 0;
    }
    resident = clusters;
    std::lock_guard<std::mutex> lk(g_fit_mu);
    g_fit[key] = resident;
  }
  return c.tiles <= resident;
}

cudaError_t launch_sweep_forward(const StepConfig& c, const SweepArgs& a, cudaStream_t st, bool pdl) {
  const SweepKernel k = sweep_kernel_for(0, c.threads);
  if (!k) return cudaErrorNotSupported;
  return launch_cluster(k, c, a, st, pdl);
}

cudaError_t launch_sweep_backward(const StepConfig& c, const SweepArgs& a, cudaStream_t st, bool pdl) {
  const SweepKernel k = sweep_kernel_for(1, c.threads);
  if (!k) return cudaErrorNotSupported;
  return launch_cluster(k, c, a, st, pdl);
}

}  // namespace gs
