// Fused time-step kernels: StepForward plus the Euler update of the forward
// loop of Algorithm 1, and StepBackward plus the adjoint update of its
// reverse loop.  Each runs as one launch per time step.
//
// Work split.  A thread-block cluster of C CTAs owns a tile of M = NT*R
// targets.  CTA rank r sums the pair terms of every target in the tile
// against one contiguous split of the sources (pair_tile.cuh).  The C splits
// together cover all N sources.  The split sums then meet in distributed
// shared memory: with slice = ceil(M/C), CTA r reduces targets
// [r*slice, (r+1)*slice) of the tile (C need not divide M or be a power of
// two), adding the C partials of each of its targets in rank order, in
// double-single arithmetic, and applies the FP64 update to those targets.
// The forward kernel has every CTA store its partials straight into the
// reducing CTA's shared memory (remote stores: nothing waits on a remote
// load; one cluster barrier per step).  The reverse kernel does the same
// with one-warp CTAs; larger reverse CTAs have the reducing CTA load the
// partials from its peers after a barrier (which measured faster for them).
// The reduction
// order is fixed, so results are deterministic.  No split partials go
// through global memory, and no second kernel is needed.  This plays the
// role of the paper's shared-memory reduction (Section 2.5), spread over up
// to 16 SMs.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <set>
#include <utility>

#include "pair_tile.cuh"

namespace gs {

namespace {

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

}  // namespace

// ---------------------------------------------------------------- step bodies
// One problem as seen by a CTA: the problem's landmarks are [off, off+npad)
// of the packed arrays (off = 0 for a single problem), n of them real.  The
// CTA owns target tile `tile` of the problem and source split `rank` of its
// cluster.
struct StepView {
  int off, n, npad, split_len, tile;
  float kappa_f, kq_f;
  double kq, kappa, dt, lambda;
};

// Add the W warp groups' partials of every target into group 0's slot, in
// group order, in double-single arithmetic (each float4 holds two (hi, lo)
// values).  Each item is read and written by one thread only.
template <int W, int M, int D>
__device__ __forceinline__ void combine_groups(float4 (&red)[W][M][D]) {
  if constexpr (W > 1) {
    __syncthreads();
    for (int item = threadIdx.x; item < M * D; item += blockDim.x) {
      const int lt = item / D, k = item % D;
      float4 acc = red[0][lt][k];
#pragma unroll
      for (int g = 1; g < W; ++g) {
        const float4 x = red[g][lt][k];
        const ds s0 = ds_add(ds{acc.x, acc.y}, ds{x.x, x.y});
        const ds s1 = ds_add(ds{acc.z, acc.w}, ds{x.z, x.w});
        acc = make_float4(s0.hi, s0.lo, s1.hi, s1.lo);
      }
      red[0][lt][k] = acc;
    }
  }
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

// The sum over the cluster's C source splits of one target coordinate's two
// partials (get(rr, x, y) yields split rr's double-single x and y), added in
// rank order: in double-single arithmetic (TwoSum), or, when f64 is set,
// each partial converted to FP64 and added in FP64.
template <class Get>
__device__ __forceinline__ void combine_splits(unsigned C, bool f64, Get get, double& s0, double& s1) {
  if (f64) {
    double a = 0.0, b = 0.0;
#pragma unroll 4
    for (unsigned rr = 0; rr < C; ++rr) {
      float2 x, y;
      get(rr, x, y);
      a += static_cast<double>(x.x) + static_cast<double>(x.y);
      b += static_cast<double>(y.x) + static_cast<double>(y.y);
    }
    s0 = a;
    s1 = b;
    return;
  }
  ds a{0.f, 0.f}, b{0.f, 0.f};
#pragma unroll 4
  for (unsigned rr = 0; rr < C; ++rr) {
    float2 x, y;
    get(rr, x, y);
    a = ds_add(a, ds{x.x, x.y});
    b = ds_add(b, ds{y.x, y.y});
  }
  s0 = ds_to_double(a);
  s1 = ds_to_double(b);
}

// W > 1: the warp groups' partials of every target of the tile, added in
// shared memory in group order into red[0].  Ends with a CTA barrier.
template <int NT, int R, int W, int M, int D, class Tile, class Res>
__device__ __forceinline__ void combine_tile(float4 (&red)[W][M][D], const Tile& t, Res result, int lt0, int grp) {
  if constexpr (W > 1) {
    constexpr int TG = NT / W;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ds w[2 * D];
      result(t, r, w);
      pack_ds<D>(w, red[grp][lt0 + r * TG]);
    }
    combine_groups<W, M, D>(red);
    __syncthreads();
  }
}

// Push the tile's partials to their reducing CTAs: W = 1 straight from each
// thread's registers, W > 1 from red[0] (after combine_tile).  The caller
// makes sure every receiving CTA is ready (a cluster barrier wait first).
template <int NT, int R, int W, int M, int D, class Tile, class Res>
__device__ __forceinline__ void push_tile(const float4 (&red)[W][M][D], float4* recv, const Tile& t, Res result,
                                          int lt0, unsigned rank, int slice) {
  if constexpr (W == 1) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ds w[2 * D];
      result(t, r, w);
      float4 x[D];
      pack_ds<D>(w, x);
      push_partials<D>(recv, lt0 + r * NT, rank, slice, x);
    }
  } else {
    for (int lt = threadIdx.x; lt < M; lt += NT) push_partials<D>(recv, lt, rank, slice, red[0][lt]);
  }
}

// Forward step of one tile: pair sums, cluster reduction, Euler update.
// Accumulates this thread's H0 and mismatch contributions in hc, mc.
// V: the variants (RK4 stages, the terminal launch) are compiled in.  D: the
// dimension of the landmarks (3, or 2 for planar landmarks).
template <int NT, int R, int W, bool V, int D>
__device__ __forceinline__ void forward_body(const StepFwdArgs& a, const StepView& v, double& hc, double& mc) {
  constexpr int TG = NT / W;  // threads per warp group
  constexpr int M = TG * R;   // targets of the CTA
  static_assert(NT % W == 0 && TG % 32 == 0, "warp groups must be whole warps");
  union Smem {
    StageBuf<1, D> st;
    float4 red[W][M][D];  // per group: Hp (hi,lo) x D then Hq (hi,lo) x D per target
  };
  __shared__ __align__(128) Smem sm;
  // Partials of this CTA's slice of targets from every source split:
  // [C][slice][D] float4, the same 2D double-single values per target
  // (C * slice < M + C <= M + 16).
  __shared__ __align__(16) float4 recv[(M + 15) * D];
  __shared__ __align__(8) Pipe pp;

  const unsigned rank = cluster_rank(), C = cluster_size();
  // The launch must match the kernel: NT threads per CTA, at most one CTA of
  // the cluster per target of the tile, and splits (multiples of 8 sources)
  // that cover the problem.  The test has the same outcome in every CTA of a
  // cluster, so a bad launch leaves before any barrier.
  if (blockDim.x != NT || static_cast<int>(C) > M || (v.split_len & 7) != 0 ||
      static_cast<long long>(v.split_len) * C < v.npad) {
    if (threadIdx.x == 0) atomicOr(a.status, kErrBadLaunch);
    return;
  }
  cluster_arrive_relaxed();  // this CTA has started; the push waits for every peer's arrival
  const int lim = v.off + v.npad;
  const int j0 = min(v.off + static_cast<int>(rank) * v.split_len, lim);
  const int j1 = min(j0 + v.split_len, lim);
  if (threadIdx.x == 0) pipe_init(pp, NT / 32);
  __syncthreads();
  pdl_wait();  // the previous step's state must be complete

  const int tile0 = v.off + v.tile * M;
  const int grp = W == 1 ? 0 : static_cast<int>(threadIdx.x) / TG;
  const int lt0 = W == 1 ? static_cast<int>(threadIdx.x) : static_cast<int>(threadIdx.x) % TG;
  FwdTile<R, D> t;
  t.load(a.qp, tile0 + lt0, TG, lim);
  const float4* src[1] = {a.qp};
  stream_sources<1, W, D>(sm.st, pp, src, j0, j1, t, a.status, grp);  // ends with a CTA barrier
  const int slice = (M + static_cast<int>(C) - 1) / static_cast<int>(C);  // the last CTA may reduce fewer
  const auto res = [&](const FwdTile<R, D>& tt, int r, ds* w) { tt.result(r, v.kappa_f, w); };
  combine_tile<NT, R, W, M, D>(sm.red, t, res, lt0, grp);
  // recv is memory of its own, so a CTA may push as soon as every peer has
  // started (the arrival at kernel entry): one cluster barrier per step.
  cluster_wait();
  push_tile<NT, R, W, M, D>(sm.red, recv, t, res, lt0, rank, slice);
  cluster_sync();  // every split's partials have reached the CTA that reduces them
  if (a.late_trigger) pdl_trigger();  // only the epilogue is left

  for (int item = threadIdx.x; item < slice * D; item += NT) {
    const int ll = item / D;
    const int lt = static_cast<int>(rank) * slice + ll;
    const int k = item % D;
    if (lt >= M || v.tile * M + lt >= v.n) continue;
    const int i = tile0 + lt;  // packed landmark index
    double Hp, Hq;
    combine_splits(
        C, a.combine64 != 0,
        [&](unsigned rr, float2& x, float2& y) {
          const float2* rp = reinterpret_cast<const float2*>(&recv[(static_cast<int>(rr) * slice + ll) * D]);
          x = rp[k];
          y = rp[D + k];
        },
        Hp, Hq);
    if (a.dry) {  // timing only: keep the reduction, touch no state
      hc += Hp + Hq;
      continue;
    }
    const int tt = D * i + k;
    const double q_old = a.q64[tt], p_old = a.p64[tt];
    float* an = reinterpret_cast<float*>(a.ab + (i >> 1) * D) + 2 * k + (i & 1);
    if (V && a.terminal) {
      // The end state (q(1), p(1)): its kinetic term, the mismatch, and the
      // adjoint alpha = dL/dq(1) = 2 lambda r + Hq, beta = dL/dp(1) = Hp.
      hc += 0.5 * p_old * Hp;
      const double r = q_old - a.t64[tt];
      mc += r * r;
      const double al = 2.0 * v.lambda * r + Hq, be = Hp;
      if (!isfinite(al) || !isfinite(be)) atomicOr(a.status, kErrNonFinite);
      a.a64[tt] = al;
      a.b64[tt] = be;
      an[0] = (float)(a.adj_scale * al);
      an[2 * D] = -(float)(v.kappa * a.adj_scale * be);
      continue;
    }
    if (a.first) {
      hc += 0.5 * p_old * Hp;  // H0 = 1/2 sum_i p0_i . Hp_i(q0, p0)
      a.hp0[tt] = Hp;
      a.hq0[tt] = Hq;
    }
    double q, p;  // the state of the record this launch writes
    if (V && a.rk) {
      // Stage s of an RK4 step from y = (q_old, p_old) with f = (Hp, -Hq):
      // accumulate k1 + 2 k2 + 2 k3, write the next stage state
      // y + dt/2 f, y + dt/2 f, y + dt f, or at the last stage the new state
      // y + dt/6 (k1 + 2 k2 + 2 k3 + k4).
      const double fq = Hp, fp = -Hq;
      if (a.stage == 0) {
        a.qa64[tt] = fq;
        a.pa64[tt] = fp;
      } else if (a.stage < 3) {
        a.qa64[tt] += 2.0 * fq;
        a.pa64[tt] += 2.0 * fp;
      }
      if (a.stage < 3) {
        const double c = (a.stage == 2 ? 1.0 : 0.5) * v.dt;
        q = q_old + c * fq;
        p = p_old + c * fp;
      } else {
        q = q_old + v.dt / 6.0 * (a.qa64[tt] + fq);
        p = p_old + v.dt / 6.0 * (a.pa64[tt] + fp);
        a.q64[tt] = q;
        a.p64[tt] = p;
      }
    } else {
      q = q_old + v.dt * Hp;
      p = p_old - v.dt * Hq;
      a.q64[tt] = q;
      a.p64[tt] = p;
    }
    if (!isfinite(q) || !isfinite(p)) atomicOr(a.status, kErrNonFinite);
    float* qn = reinterpret_cast<float*>(a.qp_next + (i >> 1) * D) + 2 * k + (i & 1);
    qn[0] = -(float)(v.kq * q);
    qn[2 * D] = (float)p;
    if (a.last && a.with_loss) {
      const double r = q - a.t64[tt];
      mc += r * r;
      const double al = 2.0 * v.lambda * r;
      a.a64[tt] = al;
      a.b64[tt] = 0.0;
      an[0] = (float)((V && a.rk ? a.adj_scale : 1.0) * al);
      an[2 * D] = 0.f;
    }
  }
  // No trailing cluster barrier: every remote access of the step happened
  // before the one above.
}

// Reverse step of one tile: adjoint pair sums, cluster reduction, adjoint
// update, and at time step 0 the gradient.  V: the RK4 stages are compiled in.
// D: the dimension of the landmarks.  Ragged: the cluster size need not
// divide the tile (the last CTAs reduce fewer targets).  The plain form
// requires C | M; compiled that way the whole kernel ran 2% faster on GB300
// (N = 4096 and 16384, same cluster shape), so clusters that divide the tile
// use it and the others a separate instantiation.
template <int NT, int R, int W, bool V, int D, bool Ragged = false>
__device__ __forceinline__ void backward_body(const StepBwdArgs& a, const StepView& v) {
  constexpr int TG = NT / W;  // threads per warp group
  constexpr int M = TG * R;   // targets of the CTA
  static_assert(NT % W == 0 && TG % 32 == 0, "warp groups must be whole warps");
  union Smem {
    StageBuf<2, D> st;
    float4 red[W][M][D];  // per group: dalpha (hi,lo) x D then dbeta (hi,lo) x D per target
  };
  // CTAs of one warp push their partials into the reducing CTA's receive
  // buffer, as the forward kernel does; larger CTAs leave them in their own
  // idle stage ring for the reducing CTA to pull through distributed shared
  // memory.  Measured on GB300 (in-graph replay, 2048 to 16384 landmarks):
  // pushing is 1-4 % faster with 32-thread CTAs and 3-5 % slower with
  // 64-thread CTAs.
  constexpr bool kPush = NT == 32;
  __shared__ __align__(128) Smem sm;
  __shared__ __align__(16) float4 recv[kPush ? (Ragged ? M + 15 : M) * D : 1];
  __shared__ __align__(8) Pipe pp;

  const unsigned rank = cluster_rank(), C = cluster_size();
  // The launch must match the kernel: NT threads per CTA, a cluster size
  // that divides the tile (Ragged: at most one CTA per target of the tile),
  // and splits (multiples of 8 sources) that cover the problem.  The test has
  // the same outcome in every CTA of a cluster, so a bad launch leaves before
  // any barrier.
  if (blockDim.x != NT || (Ragged ? static_cast<int>(C) > M : M % static_cast<int>(C) != 0) ||
      (v.split_len & 7) != 0 || static_cast<long long>(v.split_len) * C < v.npad) {
    if (threadIdx.x == 0) atomicOr(a.status, kErrBadLaunch);
    return;
  }
  if constexpr (kPush) cluster_arrive_relaxed();  // waited on before the first remote store
  const int lim = v.off + v.npad;
  const int j0 = min(v.off + static_cast<int>(rank) * v.split_len, lim);
  const int j1 = min(j0 + v.split_len, lim);
  if (threadIdx.x == 0) pipe_init(pp, NT / 32);
  __syncthreads();
  pdl_wait();

  const int tile0 = v.off + v.tile * M;
  const int grp = W == 1 ? 0 : static_cast<int>(threadIdx.x) / TG;
  const int lt0 = W == 1 ? static_cast<int>(threadIdx.x) : static_cast<int>(threadIdx.x) % TG;
  BwdTile<R, D> t;
  t.load(a.qp, a.ab, tile0 + lt0, TG, lim);
  const float4* src[2] = {a.qp, a.ab};
  stream_sources<2, W, D>(sm.st, pp, src, j0, j1, t, a.status, grp);
  const int slice = Ragged ? (M + static_cast<int>(C) - 1) / static_cast<int>(C) : M / static_cast<int>(C);
  if constexpr (kPush) {
    const auto res = [&](const BwdTile<R, D>& tt, int r, ds* w) { tt.result(r, v.kq_f, v.kappa_f, w); };
    combine_tile<NT, R, W, M, D>(sm.red, t, res, lt0, grp);
    cluster_wait();  // every peer's receive buffer exists
    push_tile<NT, R, W, M, D>(sm.red, recv, t, res, lt0, rank, slice);
    cluster_sync();  // every push has landed
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ds w[2 * D];
      t.result(r, v.kq_f, v.kappa_f, w);
      pack_ds<D>(w, sm.red[grp][lt0 + r * TG]);
    }
    combine_groups<W, M, D>(sm.red);
    cluster_sync();  // every CTA's tile partials are visible to the cluster
  }
  if (a.late_trigger) pdl_trigger();  // only the reduction and the epilogue are left

  for (int item = threadIdx.x; item < slice * D; item += NT) {
    const int ll = item / D;
    const int lt = static_cast<int>(rank) * slice + ll;
    const int k = item % D;
    if ((Ragged && lt >= M) || v.tile * M + lt >= v.n) continue;
    const int i = tile0 + lt;
    double dA, dB;  // dalpha, dbeta of this coordinate
    if constexpr (kPush) {
      combine_splits(
          C, a.combine64 != 0,
          [&](unsigned rr, float2& x, float2& y) {
            const float2* rp = reinterpret_cast<const float2*>(&recv[(static_cast<int>(rr) * slice + ll) * D]);
            x = rp[k];
            y = rp[D + k];
          },
          dA, dB);
    } else {
      const uint32_t lp = smem_u32(&sm.red[0][lt][0]);
      combine_splits(
          C, a.combine64 != 0,
          [&](unsigned rr, float2& x, float2& y) {
            const uint32_t rp = dsmem_addr(lp, rr);
            x = ld_dsmem_f2(rp + 8u * k);
            y = ld_dsmem_f2(rp + 8u * D + 8u * k);
          },
          dA, dB);
    }
    if (a.dry) {
      if (!isfinite(dA + dB)) atomicOr(a.status, kErrNonFinite);
      continue;
    }
    const int tt = D * i + k;
    float* an = reinterpret_cast<float*>(a.ab_next + (i >> 1) * D) + 2 * k + (i & 1);
    double al, be;  // the adjoint of the step's start state, once complete
    if (V && a.rk) {
      // Reverse of RK4 stage s: v = J(Y_s)^T kbar_s came out of the pair sums.
      // The adjoint of the start state sums w (the adjoint of the end state)
      // and the four v; the next stage adjoint is
      //   kbar_{s-1} = dt b_{s-1} w + c_s dt v,  b = (1/6, 1/3, 1/3),
      //   c = (1/2, 1/2, 1) for s = 1, 2, 3.
      const double va = dA, vb = dB;
      const double wa = a.a64[tt], wb = a.b64[tt];
      const double ya = (a.stage == 3 ? wa : a.ya64[tt]) + va;
      const double yb = (a.stage == 3 ? wb : a.yb64[tt]) + vb;
      if (!isfinite(ya) || !isfinite(yb)) atomicOr(a.status, kErrNonFinite);
      if (a.stage > 0) {
        a.ya64[tt] = ya;
        a.yb64[tt] = yb;
        const double cw = (a.stage == 1 ? 1.0 / 6.0 : 1.0 / 3.0) * v.dt;
        const double cv = (a.stage == 3 ? 1.0 : 0.5) * v.dt;
        an[0] = (float)(cw * wa + cv * va);
        an[2 * D] = -(float)(v.kappa * (cw * wb + cv * vb));
        continue;
      }
      al = ya;
      be = yb;
      a.a64[tt] = al;
      a.b64[tt] = be;
      an[0] = (float)(v.dt / 6.0 * al);  // stage 4 adjoint of the previous step
      an[2 * D] = -(float)(v.kappa * (v.dt / 6.0 * be));
    } else {
      al = a.a64[tt] + v.dt * dA;
      be = a.b64[tt] + v.dt * dB;
      if (!isfinite(al) || !isfinite(be)) atomicOr(a.status, kErrNonFinite);
      a.a64[tt] = al;
      a.b64[tt] = be;
      an[0] = (float)al;
      an[2 * D] = -(float)(v.kappa * be);
    }
    if (a.first) {
      const double gp = be + (a.h_at_end ? 0.0 : a.hp0[tt]);
      if (a.grad_p0) a.grad_p0[tt] = (float)gp;
      if (a.grad_p0_64) a.grad_p0_64[tt] = gp;
      if (a.grad_q0) a.grad_q0[tt] = (float)(al + (a.h_at_end ? 0.0 : a.hq0[tt]));
    }
  }
  if constexpr (!kPush) cluster_sync();  // peers may still be reading this CTA's partials
}

// ---------------------------------------------------------------- single-problem kernels
// V selects the instantiation: false for the plain method (Euler steps, the
// kinetic term at t = 0), true with the variants compiled in (RK4 stages, the
// terminal launch).  Keeping them apart leaves the plain kernels' register
// allocation as the pair loop needs it.
template <int NT, int R, int W, bool V, int D = 3>
__global__ void __launch_bounds__(NT) k_step_forward(StepFwdArgs a) {
  __shared__ double shred[NT / 32];
  __shared__ int am_last;
  StepView v;
  v.off = 0;
  v.n = a.n;
  v.npad = a.npad;
  v.split_len = a.split_len;
  v.tile = blockIdx.y;
  v.kappa_f = a.kappa;
  v.kq_f = static_cast<float>(a.kq);
  v.kq = a.kq;
  v.kappa = a.kappa64;
  v.dt = a.dt;
  v.lambda = a.lambda;
  double hc = 0.0, mc = 0.0;
  forward_body<NT, R, W, V, D>(a, v, hc, mc);
  const bool reduce_h = a.first || a.terminal;
  const bool reduce_m = a.last && a.with_loss;
  if ((!reduce_h && !reduce_m) || a.dry) return;  // uniform across the grid
  double h, m;
  if (grid_sum2(hc, mc, a.red_h, a.red_m, a.ticket, shred, &am_last, &h, &m) && threadIdx.x == 0) {
    if (a.terminal) {
      a.scalars[2] = h;  // H(p(1), q(1))
      a.scalars[1] = h + a.lambda * m;
    } else {
      if (reduce_h) a.scalars[0] = h;
      if (reduce_m) a.scalars[1] = (reduce_h ? h : a.scalars[0]) + a.lambda * m;
    }
    *a.ticket = 0u;
  }
}

template <int NT, int R, int W, bool V, int D = 3, bool Ragged = false>
__global__ void __launch_bounds__(NT) k_step_backward(StepBwdArgs a) {
  StepView v;
  v.off = 0;
  v.n = a.n;
  v.npad = a.npad;
  v.split_len = a.split_len;
  v.tile = blockIdx.y;
  v.kappa_f = a.kappa;
  v.kq_f = a.kq;
  v.kq = 0.0;
  v.kappa = a.kappa64;
  v.dt = a.dt;
  v.lambda = 0.0;
  backward_body<NT, R, W, V, D, Ragged>(a, v);
}

// ---------------------------------------------------------------- packed batch kernels
// blockIdx.y indexes the item table; each item is one target tile of one
// problem.  The H0 and mismatch sums of each CTA go to red_h / red_m at
// index blockIdx.y * C + rank; a separate kernel adds them per problem.
__device__ __forceinline__ StepView batch_view(const BatchTables& bt, bool reverse) {
  const BatchItem it = bt.items[blockIdx.y];
  const BatchProb P = bt.probs[it.prob];
  StepView v;
  v.off = P.off;
  v.n = P.n;
  v.npad = P.npad;
  v.split_len = reverse ? P.split_len_b : P.split_len;
  v.tile = it.tile;
  v.kappa_f = static_cast<float>(P.kappa);
  v.kq_f = static_cast<float>(P.kq);
  v.kq = P.kq;
  v.kappa = P.kappa;
  v.dt = P.dt;
  v.lambda = P.lambda;
  return v;
}

template <int NT, int R, int W>
__global__ void __launch_bounds__(NT) k_bstep_forward(StepFwdArgs a, BatchTables bt) {
  __shared__ double shred[NT / 32];
  const StepView v = batch_view(bt, false);
  double hc = 0.0, mc = 0.0;
  forward_body<NT, R, W, false, 3>(a, v, hc, mc);
  const bool reduce_h = a.first != 0;
  const bool reduce_m = a.last && a.with_loss;
  if ((!reduce_h && !reduce_m) || a.dry) return;
  const double bh = block_sum_f64(hc, shred);
  const double bm = block_sum_f64(mc, shred);
  if (threadIdx.x == 0) {
    const unsigned cta = blockIdx.y * gridDim.x + cluster_rank();
    if (reduce_h) a.red_h[cta] = bh;
    if (reduce_m) a.red_m[cta] = bm;
  }
}

template <int NT, int R, int W>
__global__ void __launch_bounds__(NT) k_bstep_backward(StepBwdArgs a, BatchTables bt) {
  backward_body<NT, R, W, false, 3>(a, batch_view(bt, true));
}

// ---------------------------------------------------------------- host side

namespace {

// Compiled variants: (threads per CTA, targets per thread, warp groups).
#define GS_STEP_FWD_CASES(X)                                                                         \
  X(64, 1, 1) X(64, 2, 1) X(64, 4, 1) X(128, 1, 1) X(128, 2, 1) X(128, 4, 1) X(256, 1, 1) X(256, 2, 1) \
  X(64, 1, 2) X(128, 1, 2) X(128, 1, 4) X(256, 1, 4)
#define GS_STEP_BWD_CASES(X) \
  X(32, 1, 1) X(64, 1, 1) X(64, 2, 1) X(128, 1, 1) X(128, 2, 1) X(256, 1, 1) X(64, 1, 2) X(128, 1, 2) X(128, 1, 4) X(256, 1, 4)

std::mutex g_attr_mu;
std::set<const void*> g_attr_done;  // kernels allowed clusters of up to 16 CTAs

// Cluster scheduling preference forced on the step kernels (-1: each
// configuration's own; 0 the CUDA driver's default, 1 spread, 2 load balancing).
int g_cluster_policy = -1;

// Launch attributes of a step kernel: cluster shape, the scheduling policy
// if one is set, and programmatic dependent launch.  Returns their count.
unsigned cluster_attrs(cudaLaunchAttribute* at, int cluster, bool pdl, int policy) {
  if (g_cluster_policy >= 0) policy = g_cluster_policy;
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
  std::lock_guard<std::mutex> lk(g_attr_mu);
  const void* key = reinterpret_cast<const void*>(kern);
  if (!g_attr_done.count(key)) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    g_attr_done.insert(key);
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

bool valid_variant(int kind, int threads, int R, int groups) {
#define X(T_, R_, W_) \
  if (threads == T_ && R == R_ && groups == W_) return true;
  if (kind == 0) {
    GS_STEP_FWD_CASES(X)
  } else {
    GS_STEP_BWD_CASES(X)
  }
#undef X
  return false;
}

}  // namespace

StepConfig step_config_for(int kind, int npad, int threads, int R, int cluster, int groups) {
  StepConfig c{};
  if (groups < 1 || !valid_variant(kind, threads, R, groups)) return c;
  const int M = threads / groups * R;
  if (cluster < 1 || cluster > 16 || cluster > M) return c;
  // Reverse kernels for clusters that do not divide the tile exist for the
  // one-target, one-group CTAs of 32 and 64 threads only.
  if (kind == 1 && M % cluster != 0 && (R != 1 || groups != 1 || (threads != 32 && threads != kVarBwdThreads)))
    return c;
  c.threads = threads;
  c.R = R;
  c.groups = groups;
  c.cluster = cluster;
  c.tiles = (npad + M - 1) / M;
  int len = (npad + cluster - 1) / cluster;
  c.split_len = (len + kUnroll - 1) / kUnroll * kUnroll;
  return c;
}

namespace {
int g_override[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};  // threads, R, cluster, groups per kind
}

void set_cluster_policy(int policy) { g_cluster_policy = policy; }

namespace {
int g_late_trigger = -1;
std::mutex g_res_mu;
// ((device, kernel), cluster size) -> CTAs of that kernel resident at once
std::map<std::pair<std::pair<int, const void*>, int>, int> g_resident;
}  // namespace

void set_late_trigger(int mode) { g_late_trigger = mode; }

namespace {
bool g_combine64 = false;
}  // namespace

void set_combine_f64(bool on) { g_combine64 = on; }
bool combine_f64() { return g_combine64; }

bool late_trigger_for(int kind, const StepConfig& c, int dim, bool rk) {
  if (g_late_trigger >= 0) return g_late_trigger == 1;
  // The library's rule, from GB300 measurements of gradient graphs
  // (N = 2048..16384): reverse steps whose CTAs are all resident at once
  // trigger (-1.7% reverse-sweep time at N = 4096); forward steps never
  // (+13% forward-sweep time at N = 4096 with the trigger).  Residency is
  // that of the instantiation the launch runs (the uneven-cluster, RK4 and
  // planar kernels differ in registers and shared memory).
  if (kind != 1) return false;
  const BwdKernel kern = backward_kernel_for(c, dim, rk);
  if (!kern) return false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  const auto key = std::make_pair(std::make_pair(dev, reinterpret_cast<const void*>(kern)), c.cluster);
  int resident = -1;
  {
    std::lock_guard<std::mutex> lk(g_res_mu);
    const auto it = g_resident.find(key);
    if (it != g_resident.end()) resident = it->second;
  }
  if (resident < 0) {
    int clusters = 0;
    if (occupancy_clusters(kern, c.threads, c.cluster, &clusters) != cudaSuccess) {
      cudaGetLastError();
      clusters = 0;
    }
    resident = clusters * c.cluster;
    std::lock_guard<std::mutex> lk(g_res_mu);
    g_resident[key] = resident;
  }
  return static_cast<long long>(c.tiles) * c.cluster <= resident;
}

int policy_for_grid(long long ctas, int num_sms) { return 2 * ctas >= 3LL * 8 * num_sms ? 2 : 1; }

cudaError_t max_active_clusters(int kind, int threads, int R, int groups, int cluster, int* out) {
  *out = 0;
#define X(T_, R_, W_) \
  if (threads == T_ && R == R_ && groups == W_) return occupancy_clusters(k_step_forward<T_, R_, W_, false>, T_, cluster, out);
  if (kind == 0) {
    GS_STEP_FWD_CASES(X)
  }
#undef X
#define X(T_, R_, W_) \
  if (threads == T_ && R == R_ && groups == W_) return occupancy_clusters(k_step_backward<T_, R_, W_, false>, T_, cluster, out);
  if (kind == 1) {
    GS_STEP_BWD_CASES(X)
  }
#undef X
  return cudaErrorInvalidValue;
}

bool set_step_override(int kind, int threads, int R, int groups, int cluster) {
  if (threads == 0) {
    g_override[kind][0] = g_override[kind][1] = g_override[kind][2] = g_override[kind][3] = 0;
    return true;
  }
  if (step_config_for(kind, 1 << 16, threads, R, cluster, groups).threads == 0) return false;
  g_override[kind][0] = threads;
  g_override[kind][1] = R;
  g_override[kind][2] = cluster;
  g_override[kind][3] = groups;
  return true;
}

namespace {
// One row of the measured step-configuration table: the padded landmark
// count, then per kind (forward, reverse) the fastest CTA size and cluster
// size, and the fastest cluster size for the full-size CTAs.
struct StepRule {
  int npad;
  int fwd_threads, fwd_cluster, fwd_full_cluster;
  int bwd_threads, bwd_cluster, bwd_full_cluster;
};
#include "step_table.inc"
bool g_use_table = true;

// The table row for npad: the first row at or above it (rows are
// ascending), or null above the last row.
const StepRule* table_rule(int npad) {
  const StepRule* end = kStepTable + sizeof(kStepTable) / sizeof(kStepTable[0]);
  const StepRule* r = std::lower_bound(kStepTable, end, npad, [](const StepRule& e, int n) { return e.npad < n; });
  return r == end ? nullptr : r;
}
}  // namespace

void set_step_table(bool on) { g_use_table = on; }

namespace {
int g_batch_shape[2][2] = {{0, 0}, {0, 0}};  // threads, cluster per kind (0: built-in)
}  // namespace

void batch_shape(int kind, int* threads, int* cluster) {
  // Built-in: 128-thread CTAs forward, 64 reverse, one target per thread,
  // clusters of 8 for both.
  *threads = g_batch_shape[kind][0] ? g_batch_shape[kind][0] : (kind == 0 ? 128 : 64);
  *cluster = g_batch_shape[kind][1] ? g_batch_shape[kind][1] : 8;
}

bool set_batch_shape(int kind, int threads, int cluster) {
  if (kind != 0 && kind != 1) return false;
  if (threads == 0) {
    g_batch_shape[kind][0] = g_batch_shape[kind][1] = 0;
    return true;
  }
  // the packed kernels exist for the one-group shapes whose cluster divides the tile
  const StepConfig c = step_config_for(kind, 1 << 16, threads, 1, cluster);
  if (c.threads == 0 || threads % cluster != 0) return false;
  g_batch_shape[kind][0] = threads;
  g_batch_shape[kind][1] = cluster;
  return true;
}

// Default configuration per problem size, from sweeps on GB300 (152 SMs).
StepConfig choose_step_config(int kind, int npad, int num_sms, bool variants) {
  if (g_override[kind][0] && !variants) {
    StepConfig c = step_config_for(kind, npad, g_override[kind][0], g_override[kind][1],
                                   std::min(g_override[kind][2], std::max(1, npad / kUnroll)), g_override[kind][3]);
    c.policy = policy_for_grid(static_cast<long long>(c.tiles) * c.cluster, num_sms);
    if (c.threads) return c;
  }
  // One target per thread throughout.  On a device with the SM count it was
  // measured for, the table gives the CTA and cluster sizes per padded
  // landmark count up to 16384: the fastest shape swings by up to 20%
  // between neighbouring sizes as the clusters fill the SMs of each GPC
  // unevenly.  Above the table and on other devices, the size rule it
  // refines, measured on GB300 (in-graph replay, 1024..65536 landmarks):
  //  * from 4096 landmarks up, forward steps as 128-thread CTAs in clusters
  //    of 16 and reverse steps as 64-thread CTAs in clusters of 8;
  //  * below, CTAs of half the threads spread the few targets over more SMs:
  //    forward 64 threads, clusters of 16 (+13% at 1024 and 2048 landmarks);
  //    reverse 32 threads, clusters of 16 up to 1024 landmarks and of 8 up to
  //    2048.
  // The variant kernels (RK4 stages, the terminal launch, planar landmarks)
  // exist for the 128 / 64-thread CTAs only.  A grid of 1.5 waves or more
  // (8 CTAs per SM) is scheduled with load balancing, which keeps every SM
  // busy; a smaller grid is spread over the SMs.
  int threads = kind == 0 ? kVarFwdThreads : kVarBwdThreads;
  int c = 0;
  const StepRule* r = g_use_table && num_sms == kStepTableSms ? table_rule(npad) : nullptr;
  if (r) {
    if (kind == 0) {
      if (!variants) threads = r->fwd_threads;
      c = variants ? r->fwd_full_cluster : r->fwd_cluster;
    } else {
      if (!variants) threads = r->bwd_threads;
      c = variants ? r->bwd_full_cluster : r->bwd_cluster;
    }
    c = std::min(c, std::max(1, npad / kUnroll));  // every CTA keeps at least 8 sources
  } else {
    int cmax = kind == 0 ? 16 : 8;
    if (!variants && npad <= 2048) {
      threads /= 2;
      if (kind == 1 && npad <= 1024) cmax = 16;
    }
    const int cl = std::min(cmax, std::max(1, npad / kUnroll));
    c = 1;
    while (c * 2 <= cl) c *= 2;
  }
  StepConfig cfg = step_config_for(kind, npad, threads, 1, c);
  cfg.policy = policy_for_grid(static_cast<long long>(cfg.tiles) * c, num_sms);
  return cfg;
}

template <typename K, typename A>
cudaError_t launch_cluster2(K kern, int cluster, int threads, int policy, int items, const A& args,
                            const BatchTables& bt, cudaStream_t st, bool pdl) {
  const cudaError_t e = allow_large_clusters(kern);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster, items);
  cfg.blockDim = dim3(threads);
  cfg.stream = st;
  cudaLaunchAttribute at[3];
  cfg.attrs = at;
  cfg.numAttrs = cluster_attrs(at, cluster, pdl, policy);
  return cudaLaunchKernelEx(&cfg, kern, args, bt);
}

cudaError_t launch_bstep_forward(const StepConfig& c, int items, const StepFwdArgs& a, const BatchTables& bt,
                                 cudaStream_t st, bool pdl) {
#define X(T_, R_, W_) \
  if (c.threads == T_ && c.R == R_ && c.groups == W_) \
    return launch_cluster2(k_bstep_forward<T_, R_, W_>, c.cluster, T_, c.policy, items, a, bt, st, pdl);
  GS_STEP_FWD_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_bstep_backward(const StepConfig& c, int items, const StepBwdArgs& a, const BatchTables& bt,
                                  cudaStream_t st, bool pdl) {
#define X(T_, R_, W_) \
  if (c.threads == T_ && c.R == R_ && c.groups == W_) \
    return launch_cluster2(k_bstep_backward<T_, R_, W_>, c.cluster, T_, c.policy, items, a, bt, st, pdl);
  GS_STEP_BWD_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

// The instantiation that runs a launch of configuration c.  The variants
// (RK4 stages, the terminal launch) go to the V = true instantiation of the
// built-in configuration's kernel variant; planar landmarks (dim 2) to the
// D = 2 instantiations of that variant.  Null: no instantiation exists.
FwdKernel forward_kernel_for(const StepConfig& c, int dim, bool variants) {
  if (dim == 2) {  // planar landmarks: the built-in configuration only
    if (c.threads != kVarFwdThreads || c.R != 1 || c.groups != 1) return nullptr;
    return variants ? k_step_forward<kVarFwdThreads, 1, 1, true, 2> : k_step_forward<kVarFwdThreads, 1, 1, false, 2>;
  }
  if (variants) {
    if (c.threads == kVarFwdThreads && c.R == 1 && c.groups == 1) return k_step_forward<kVarFwdThreads, 1, 1, true>;
    return nullptr;
  }
#define X(T_, R_, W_) \
  if (c.threads == T_ && c.R == R_ && c.groups == W_) return k_step_forward<T_, R_, W_, false>;
  GS_STEP_FWD_CASES(X)
#undef X
  return nullptr;
}

BwdKernel backward_kernel_for(const StepConfig& c, int dim, bool rk) {
  if ((c.threads / c.groups * c.R) % c.cluster != 0) {  // the instantiations for clusters that do not divide the tile
    if (c.R != 1 || c.groups != 1 || (c.threads != 32 && c.threads != kVarBwdThreads)) return nullptr;
    if (dim == 2) {
      if (c.threads != kVarBwdThreads) return nullptr;
      return rk ? k_step_backward<kVarBwdThreads, 1, 1, true, 2, true> : k_step_backward<kVarBwdThreads, 1, 1, false, 2, true>;
    }
    if (rk) return c.threads == kVarBwdThreads ? k_step_backward<kVarBwdThreads, 1, 1, true, 3, true> : nullptr;
    if (c.threads == 32) return k_step_backward<32, 1, 1, false, 3, true>;
    return k_step_backward<kVarBwdThreads, 1, 1, false, 3, true>;
  }
  if (dim == 2) {
    if (c.threads != kVarBwdThreads || c.R != 1 || c.groups != 1) return nullptr;
    return rk ? k_step_backward<kVarBwdThreads, 1, 1, true, 2> : k_step_backward<kVarBwdThreads, 1, 1, false, 2>;
  }
  if (rk) {
    if (c.threads == kVarBwdThreads && c.R == 1 && c.groups == 1) return k_step_backward<kVarBwdThreads, 1, 1, true>;
    return nullptr;
  }
#define X(T_, R_, W_) \
  if (c.threads == T_ && c.R == R_ && c.groups == W_) return k_step_backward<T_, R_, W_, false>;
  GS_STEP_BWD_CASES(X)
#undef X
  return nullptr;
}

cudaError_t launch_step_forward(const StepConfig& c, const StepFwdArgs& a, cudaStream_t st, bool pdl) {
  const FwdKernel k = forward_kernel_for(c, a.dim, a.rk || a.terminal);
  if (!k) return cudaErrorNotSupported;
  return launch_cluster(k, c, a, st, pdl);
}

cudaError_t launch_step_backward(const StepConfig& c, const StepBwdArgs& a, cudaStream_t st, bool pdl) {
  const BwdKernel k = backward_kernel_for(c, a.dim, a.rk != 0);
  if (!k) return cudaErrorNotSupported;
  return launch_cluster(k, c, a, st, pdl);
}

}  // namespace gs
