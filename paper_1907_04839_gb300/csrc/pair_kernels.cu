// Pair-sum kernels: StepForward and StepBackward (Section 2.2, 2.5).
//
// These sums are the O(N^2) hot path of the method.  The paper's Algorithm 4
// has one block per target, a shared-memory tree reduction over 256 sources
// and atomicAdd into global memory.  This design differs:
//  * A CTA owns a tile of NT*R targets, held in registers (R per thread).
//  * A CTA streams one contiguous range of sources (a "split") through shared
//    memory.  The staging uses bulk TMA copies (cp.async.bulk) into a double
//    buffer, and each buffer is guarded by an mbarrier.
//  * Every warp reads the same source at the same time, so the shared-memory
//    read is a broadcast.
//  * Sources are stored as pair records of two landmarks, and paired FP32
//    instructions work on both at once (pair_tile.cuh).
//  * Each thread accumulates plain FP32 over a sub-block of at most 64
//    sources, then folds the sub-block sum into a Kahan (sum, compensation)
//    pair.  This is the compensated accumulation that the paper's accuracy
//    argument (Section 2.2) asks for.
//  * The split's result goes out as a double-single partial per target.  No
//    atomics are used, so the result is deterministic.  A separate kernel
//    combines the splits in a fixed order (combine.cu).
//  * The Gaussian is a single MUFU ex2 on prescaled coordinates.  With
//    q~ = kq q and kq^2 = log2(e) / (2 sigma^2),
//    g = exp(-|d|^2 / (2 sigma^2)) = 2^(-|q~_i - q~_j|^2).
//  * The kernels use no tensor cores.  The pair work is not a dense
//    contraction (d = 3), and it is bound by the FP32 pipe.
#include <cmath>
#include <cstdio>

#include "pair_tile.cuh"

namespace gs {

// ---------------------------------------------------------------- split-partial kernels
// Grid (tiles, splits).  CTA (x, y) owns targets x*NT*R + tid + r*NT and the
// sources of split y; it writes one double-single Partial per target.
template <int NT, int R>
__global__ void __launch_bounds__(NT) k_pair_forward(PairFwdArgs a) {
  __shared__ __align__(128) StageBuf<1> st;
  __shared__ __align__(8) Pipe pp;
  const int j0 = blockIdx.y * a.split_len;
  const int j1 = min(j0 + a.split_len, a.npad);
  if (threadIdx.x == 0) pipe_init(pp, NT / 32);
  __syncthreads();
  pdl_wait();  // the previous step's state must be complete
  const int base = blockIdx.x * (NT * R) + threadIdx.x;
  FwdTile<R> tile;
  tile.load(a.qp, base, NT, a.npad);
  const float4* src[1] = {a.qp};
  if (!stream_sources<1>(st, pp, src, j0, j1, tile, a.status)) return;
  Partial* out = a.part + static_cast<size_t>(blockIdx.y) * a.npad;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = base + r * NT;
    if (i >= a.npad) continue;
    ds v[6];
    tile.result(r, a.kappa, v);
    Partial pt;
#pragma unroll
    for (int c = 0; c < 6; ++c) pt.c[c] = make_float2(v[c].hi, v[c].lo);
    out[i] = pt;
  }
}

template <int NT, int R>
__global__ void __launch_bounds__(NT) k_pair_backward(PairBwdArgs a) {
  __shared__ __align__(128) StageBuf<2> st;
  __shared__ __align__(8) Pipe pp;
  const int j0 = blockIdx.y * a.split_len;
  const int j1 = min(j0 + a.split_len, a.npad);
  if (threadIdx.x == 0) pipe_init(pp, NT / 32);
  __syncthreads();
  pdl_wait();
  const int base = blockIdx.x * (NT * R) + threadIdx.x;
  BwdTile<R> tile;
  tile.load(a.qp, a.ab, base, NT, a.npad);
  const float4* src[2] = {a.qp, a.ab};
  if (!stream_sources<2>(st, pp, src, j0, j1, tile, a.status)) return;
  Partial* out = a.part + static_cast<size_t>(blockIdx.y) * a.npad;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = base + r * NT;
    if (i >= a.npad) continue;
    ds v[6];
    tile.result(r, a.kq, a.kappa, v);
    Partial pt;
#pragma unroll
    for (int c = 0; c < 6; ++c) pt.c[c] = make_float2(v[c].hi, v[c].lo);
    out[i] = pt;
  }
}

// ---------------------------------------------------------------- host side

namespace {

template <typename K, typename A>
cudaError_t launch(K kern, dim3 grid, dim3 block, const A& args, cudaStream_t st, bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args);
}

// Kernel variants: (threads per CTA, targets per thread).
struct Variant {
  int threads, R;
};
constexpr Variant kFwdVariants[] = {{64, 2}, {64, 4}, {128, 2}, {128, 4}, {256, 1}, {256, 2}};
constexpr Variant kBwdVariants[] = {{64, 1}, {64, 2}, {128, 1}, {128, 2}, {256, 1}};
constexpr int kNumFwd = sizeof(kFwdVariants) / sizeof(Variant);
constexpr int kNumBwd = sizeof(kBwdVariants) / sizeof(Variant);

#define GS_FWD_CASES(X) X(64, 2) X(64, 4) X(128, 2) X(128, 4) X(256, 1) X(256, 2)
#define GS_BWD_CASES(X) X(64, 1) X(64, 2) X(128, 1) X(128, 2) X(256, 1)

int fwd_index(int threads, int R) {
  for (int v = 0; v < kNumFwd; ++v)
    if (kFwdVariants[v].threads == threads && kFwdVariants[v].R == R) return v;
  return -1;
}
int bwd_index(int threads, int R) {
  for (int v = 0; v < kNumBwd; ++v)
    if (kBwdVariants[v].threads == threads && kBwdVariants[v].R == R) return v;
  return -1;
}

// Resident CTAs per SM of each variant (queried once; same for every GB300).
int g_fwd_occ[kNumFwd] = {};
int g_bwd_occ[kNumBwd] = {};

int fwd_occupancy(int v) {
  if (!g_fwd_occ[v]) {
    int occ = 1;
    const Variant& x = kFwdVariants[v];
#define X(T_, R_) \
    if (x.threads == T_ && x.R == R_) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair_forward<T_, R_>, T_, 0);
    GS_FWD_CASES(X)
#undef X
    g_fwd_occ[v] = occ > 0 ? occ : 1;
  }
  return g_fwd_occ[v];
}

int bwd_occupancy(int v) {
  if (!g_bwd_occ[v]) {
    int occ = 1;
    const Variant& x = kBwdVariants[v];
#define X(T_, R_) \
    if (x.threads == T_ && x.R == R_) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair_backward<T_, R_>, T_, 0);
    GS_BWD_CASES(X)
#undef X
    g_bwd_occ[v] = occ > 0 ? occ : 1;
  }
  return g_bwd_occ[v];
}

// Split lengths are multiples of kUnroll; the last split may be shorter.
void set_splits(PairConfig& c, int npad, int splits) {
  splits = max(1, min(splits, npad / kUnroll));
  int len = (npad + splits - 1) / splits;
  len = (len + kUnroll - 1) / kUnroll * kUnroll;
  c.split_len = len;
  c.splits = (npad + len - 1) / len;
}

// Choose the source-split count S for a tile grid.  The score favours
//  * whole CTAs per SM in one wave, so every SM carries the same load;
//  * at least 8 resident warps per SM to hide latency;
//  * few splits, since each split adds a partial per target.
PairConfig balanced_config(int npad, int num_sms, int threads, int R, int occ) {
  PairConfig c;
  c.threads = threads;
  c.R = R;
  const int tile = threads * R;
  c.tiles = (npad + tile - 1) / tile;
  const int slots = num_sms * occ;
  double best = -1.0;
  int best_s = 1;
  const int smax = max(1, npad / kUnroll);
  for (int s = 1; s <= smax; ++s) {
    PairConfig t = c;
    set_splits(t, npad, s);
    if (t.splits != s) continue;  // not reachable with this rounding
    const long long ctas = (long long)c.tiles * t.splits;
    if (ctas > 4LL * slots) break;
    const double per_sm = (double)ctas / num_sms;
    double balance;
    if (ctas <= slots) {
      balance = per_sm / std::ceil(per_sm);
    } else {
      const double waves = (double)ctas / slots;
      balance = waves / std::ceil(waves);
    }
    const double warps = std::min(per_sm, (double)occ) * threads / 32.0;
    const double lat = std::min(1.0, warps / 8.0);
    const double score = balance * lat - 0.001 * s;
    if (score > best + 1e-12) {
      best = score;
      best_s = s;
    }
  }
  set_splits(c, npad, best_s);
  return c;
}

constexpr int kFwdNT = 64, kFwdR = 4;
constexpr int kBwdNT = 64, kBwdR = 2;

}  // namespace

PairConfig forward_config_for(int npad, int num_sms, int threads, int R, int splits) {
  const int v = fwd_index(threads, R);
  if (v < 0) {
    PairConfig bad{};
    return bad;
  }
  PairConfig c = balanced_config(npad, num_sms, threads, R, fwd_occupancy(v));
  if (splits > 0) set_splits(c, npad, splits);
  return c;
}

PairConfig backward_config_for(int npad, int num_sms, int threads, int R, int splits) {
  const int v = bwd_index(threads, R);
  if (v < 0) {
    PairConfig bad{};
    return bad;
  }
  PairConfig c = balanced_config(npad, num_sms, threads, R, bwd_occupancy(v));
  if (splits > 0) set_splits(c, npad, splits);
  return c;
}

PairConfig choose_forward_config(int npad, int num_sms) {
  return forward_config_for(npad, num_sms, kFwdNT, kFwdR, 0);
}

PairConfig choose_forward_config_capped(int npad, int num_sms, int max_splits) {
  PairConfig c = choose_forward_config(npad, num_sms);
  if (c.splits > max_splits) set_splits(c, npad, max_splits);
  return c;
}

PairConfig choose_backward_config(int npad, int num_sms) {
  return backward_config_for(npad, num_sms, kBwdNT, kBwdR, 0);
}

cudaError_t launch_pair_forward(const PairConfig& cfg, const PairFwdArgs& a, cudaStream_t st, bool pdl) {
  const dim3 grid(cfg.tiles, cfg.splits);
#define X(T_, R_) \
  if (cfg.threads == T_ && cfg.R == R_) return launch(k_pair_forward<T_, R_>, grid, dim3(T_), a, st, pdl);
  GS_FWD_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_pair_backward(const PairConfig& cfg, const PairBwdArgs& a, cudaStream_t st, bool pdl) {
  const dim3 grid(cfg.tiles, cfg.splits);
#define X(T_, R_) \
  if (cfg.threads == T_ && cfg.R == R_) return launch(k_pair_backward<T_, R_>, grid, dim3(T_), a, st, pdl);
  GS_BWD_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace gs
