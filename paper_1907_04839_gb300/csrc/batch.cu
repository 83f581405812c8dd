// Packed batches of independent registrations and the serving loop built on
// them.
//
// Problems share packed device arrays: problem b owns landmarks
// [off_b, off_b + npad_b) of every array.  Segments are carved from a fixed
// capacity by a first-fit allocator, in units of kPad landmarks.  Each time
// step of a batched gradient is one launch of the fused step kernel over an
// item table of (problem, target tile) pairs.  Every problem has its own N,
// sigma and lambda; T is shared.
//
// L-BFGS runs per problem, as in lbfgs.cu, in rounds:
//  1. Problems that need a new direction get it from a two-loop kernel, one
//     CTA per problem.
//  2. Every active problem's current trial point is evaluated by one batched
//     gradient.
//  3. The host advances each problem's line-search state machine.
// Problems drop out as they finish.  For serving, new problems are admitted
// at round boundaries while memory is free: continuous batching.  All
// per-problem reductions are deterministic (fixed order), so a problem's
// iterates do not depend on which other problems share its rounds, as long
// as its tile configuration is the same.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "engine.h"
#include "gs_device.cuh"

namespace gs {
namespace {

constexpr int kBT = 256;     // threads of the per-problem kernels
constexpr int kMaxM = 64;

// ---------------------------------------------------------------- per-problem kernels
// One CTA per listed problem (blockIdx.x indexes `list`).

// q64 <- q0 (packed FP32 input), p64 <- x, record slot 0, for listed problems.
__global__ void __launch_bounds__(kBT) k_bpack(const int* list, const BatchProb* probs, const float* qin,
                                              const double* x, double* q64, double* p64, float4* rec,
                                              unsigned* status) {
  const BatchProb P = probs[list[blockIdx.x]];
  for (int t = threadIdx.x; t < 3 * P.n; t += kBT) {
    const int g = 3 * P.off + t;
    const int i = P.off + t / 3, k = t % 3;
    const double q = qin[g], p = x[g];
    if (!isfinite(q) || !isfinite(p)) atomicOr(status, kErrNonFinite);
    q64[g] = q;
    p64[g] = p;
    float* r = reinterpret_cast<float*>(rec + (i >> 1) * kRecF4) + 2 * k + (i & 1);
    r[0] = -(float)(P.kq * q);
    r[6] = (float)p;
  }
}

// loss_b = H0_b + lambda_b * sum |q1 - t|^2 from the per-CTA partials of the
// problem's items [item0, item0 + tiles) (cluster size C).
__global__ void __launch_bounds__(32) k_bloss(const int* list, const int* item0, const int* ntiles,
                                             const BatchProb* probs, const double* red_h, const double* red_m,
                                             int C, double* loss) {
  const int b = list[blockIdx.x];
  const int c0 = item0[b] * C, c1 = (item0[b] + ntiles[b]) * C;
  double h = 0.0, m = 0.0;
  for (int c = c0 + threadIdx.x; c < c1; c += 32) {
    h += red_h[c];
    m += red_m[c];
  }
  h = warp_sum_f64(h);
  m = warp_sum_f64(m);
  if (threadIdx.x == 0) loss[b] = h + probs[b].lambda * m;
}

struct DotSpec {
  // Up to 4 dot products per problem.  Each operand is a packed base array
  // plus an optional per-problem slot (slot * stride added; slot < 0 = none).
  const double* a[4];
  const double* b[4];
  const int* slot_a;  // per-problem slot for operands a (history), or null
  const int* slot_b;
  size_t stride;
  int count;
};

__global__ void __launch_bounds__(kBT) k_bdots(const int* list, const BatchProb* probs, DotSpec s, double* out) {
  __shared__ double sh[kBT / 32];
  const int b = list[blockIdx.x];
  const BatchProb P = probs[b];
  const size_t oa = s.slot_a ? static_cast<size_t>(s.slot_a[b]) * s.stride : 0;
  const size_t ob = s.slot_b ? static_cast<size_t>(s.slot_b[b]) * s.stride : 0;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int t = threadIdx.x; t < 3 * P.n; t += kBT) {
    const size_t g = 3 * static_cast<size_t>(P.off) + t;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < s.count) v[k] = fma(s.a[k][oa + g], s.b[k][ob + g], v[k]);
  }
  for (int k = 0; k < s.count; ++k) {
    const double r = block_sum_f64(v[k], sh);
    if (threadIdx.x == 0) out[4 * b + k] = r;
  }
}

// Per-problem L-BFGS state kept on the device for the two-loop kernel.
struct TwoLoopState {
  int head, stored;
  double gamma;
  double rho[kMaxM];
};

// d = -H g by the two-loop recursion, one CTA per listed problem.
__global__ void __launch_bounds__(kBT) k_btwoloop(const int* list, const BatchProb* probs,
                                                 const TwoLoopState* state, int m, size_t stride, const double* g,
                                                 const double* S, const double* Y, double* d, double* alpha_buf) {
  __shared__ double sh[kBT / 32];
  __shared__ double coef;
  const int b = list[blockIdx.x];
  const BatchProb P = probs[b];
  const TwoLoopState& st = state[b];
  const size_t base = 3 * static_cast<size_t>(P.off);
  const int n3 = 3 * P.n;
  double* alpha = alpha_buf + static_cast<size_t>(b) * kMaxM;
  for (int t = threadIdx.x; t < n3; t += kBT) d[base + t] = g[base + t];
  __syncthreads();
  for (int k = 0; k < st.stored; ++k) {
    const int j = (st.head - 1 - k + m) % m;
    const double* Sj = S + j * stride + base;
    const double* Yj = Y + j * stride + base;
    double v = 0.0;
    for (int t = threadIdx.x; t < n3; t += kBT) v = fma(Sj[t], d[base + t], v);
    v = block_sum_f64(v, sh);
    if (threadIdx.x == 0) {
      coef = st.rho[j] * v;
      alpha[j] = coef;
    }
    __syncthreads();
    const double a = coef;
    for (int t = threadIdx.x; t < n3; t += kBT) d[base + t] = fma(-a, Yj[t], d[base + t]);
    __syncthreads();
  }
  if (st.stored > 0)
    for (int t = threadIdx.x; t < n3; t += kBT) d[base + t] *= st.gamma;
  __syncthreads();
  for (int k = st.stored - 1; k >= 0; --k) {
    const int j = (st.head - 1 - k + m) % m;
    const double* Sj = S + j * stride + base;
    const double* Yj = Y + j * stride + base;
    double v = 0.0;
    for (int t = threadIdx.x; t < n3; t += kBT) v = fma(Yj[t], d[base + t], v);
    v = block_sum_f64(v, sh);
    if (threadIdx.x == 0) coef = alpha[j] - st.rho[j] * v;
    __syncthreads();
    const double c = coef;
    for (int t = threadIdx.x; t < n3; t += kBT) d[base + t] = fma(c, Sj[t], d[base + t]);
    __syncthreads();
  }
  for (int t = threadIdx.x; t < n3; t += kBT) d[base + t] = -d[base + t];
}

// Per-problem vector updates.  op 0: xt = x + a_b d;  op 1: d = -g;
// op 2: s_slot = xt - x, y_slot = gt - g;  op 3: x = xt, g = gt;  op 4: xt = x.
__global__ void __launch_bounds__(kBT) k_bvec(int op, const int* list, const BatchProb* probs, const double* a,
                                             const int* slot, size_t stride, double* x, double* g, double* d,
                                             double* xt, double* gt, double* S, double* Y) {
  const int b = list[blockIdx.x];
  const BatchProb P = probs[b];
  const size_t base = 3 * static_cast<size_t>(P.off);
  const int n3 = 3 * P.n;
  const size_t so = slot ? static_cast<size_t>(slot[b]) * stride : 0;
  for (int t = threadIdx.x; t < n3; t += kBT) {
    const size_t i = base + t;
    switch (op) {
      case 0: xt[i] = fma(a[b], d[i], x[i]); break;
      case 1: d[i] = -g[i]; break;
      case 2:
        S[so + i] = xt[i] - x[i];
        Y[so + i] = gt[i] - g[i];
        break;
      case 3:
        x[i] = xt[i];
        g[i] = gt[i];
        break;
      default: xt[i] = x[i]; break;
    }
  }
}

// Section 3.1 distances of a problem: out[2b] = mean |q1 - t|, out[2b+1] = max.
__global__ void __launch_bounds__(kBT) k_bdist(const int* list, const BatchProb* probs, const double* q1,
                                              const double* t, double* out) {
  __shared__ double sh[kBT / 32];
  __shared__ double shm[kBT / 32];
  const int b = list[blockIdx.x];
  const BatchProb P = probs[b];
  double s = 0.0, mx = 0.0;
  for (int i = threadIdx.x; i < P.n; i += kBT) {
    const size_t g = 3 * (static_cast<size_t>(P.off) + i);
    const double dx = q1[g] - t[g], dy = q1[g + 1] - t[g + 1], dz = q1[g + 2] - t[g + 2];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    s += r;
    mx = fmax(mx, r);
  }
  s = block_sum_f64(s, sh);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < kBT / 32; ++w) m = fmax(m, shm[w]);
    out[2 * b] = s / P.n;
    out[2 * b + 1] = m;
  }
}

template <typename K, typename... Args>
cudaError_t plaunch(int grid, int block, cudaStream_t st, K kern, Args... args) {
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, block, 0, st>>>(args...);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- host: problem records

enum Phase { kInit, kNeedDir, kSearch, kDone };

struct Problem {
  // identity and sizes
  int64_t id = 0;
  int n = 0, npad = 0, off = -1;
  double sigma = 0.0, lambda = 0.0;
  // caller buffers (register_batch) or owned result copies (server)
  float* p0_out = nullptr;
  gs_register_info* info_out = nullptr;
  // L-BFGS state
  Phase phase = kInit;
  int head = 0, stored = 0, iters = 0, evals = 0, status = 1;
  double rho[kMaxM] = {0.0};
  double gamma = 1.0, f = 0.0, g0 = 0.0, gnorm = 0.0;
  // line search state (mirrors Lbfgs::line_search in lbfgs.cu)
  double f0 = 0.0, dphi0 = 0.0, a = 0.0, a_prev = 0.0, f_prev = 0.0, d_prev = 0.0;
  double lo = 0.0, flo = 0.0, dlo = 0.0, hi = 0.0, fhi = 0.0, dhi = 0.0;
  bool zoom = false;
  int ls_it = 0, ls_used = 0;
  bool accepted = false;
  double f_acc = 0.0;
  // serving timestamps (seconds on the server clock)
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  // fair schedule: pair work charged so far (N^2 per evaluation)
  double vtime = 0.0;
  gs_register_info result{};
  std::vector<float> p0_result;
};

double cubic_min(double a, double fa, double da, double b, double fb, double db) {
  const double d1 = da + db - 3.0 * (fa - fb) / (a - b);
  const double disc = d1 * d1 - da * db;
  if (!(disc >= 0.0)) return NAN;
  const double d2 = (b > a ? 1.0 : -1.0) * std::sqrt(disc);
  const double den = db - da + 2.0 * d2;
  if (den == 0.0) return NAN;
  return b - (b - a) * (db + d2 - d1) / den;
}

// Advance a problem's strong-Wolfe line search with the value and slope at
// the last trial step.  Sets accepted / next trial / failure, like the
// sequential search in lbfgs.cu (c1 = 1e-4, c2 = 0.9, 20 evaluations).
void line_search_advance(Problem& p, double fa, double da) {
  const double c1 = 1e-4, c2 = 0.9;
  const int max_evals = 20;
  ++p.ls_used;
  const double a = p.a;
  if (!p.zoom) {
    if (!(fa <= p.f0 + c1 * a * p.dphi0) || (p.ls_it > 0 && fa >= p.f_prev)) {
      p.zoom = true;
      p.lo = p.a_prev; p.flo = p.f_prev; p.dlo = p.d_prev; p.hi = a; p.fhi = fa; p.dhi = da;
    } else if (std::fabs(da) <= -c2 * p.dphi0) {
      p.accepted = true;
      p.f_acc = fa;
      return;
    } else if (da >= 0.0) {
      p.zoom = true;
      p.lo = a; p.flo = fa; p.dlo = da; p.hi = p.a_prev; p.fhi = p.f_prev; p.dhi = p.d_prev;
    } else {
      p.a_prev = a; p.f_prev = fa; p.d_prev = da;
      p.a = 2.0 * a;
      ++p.ls_it;
      if (p.ls_used >= max_evals) p.a = 0.0;  // out of evaluations
      return;
    }
  } else {
    if (!(fa <= p.f0 + c1 * a * p.dphi0) || fa >= p.flo) {
      p.hi = a; p.fhi = fa; p.dhi = da;
    } else {
      if (std::fabs(da) <= -c2 * p.dphi0) {
        p.accepted = true;
        p.f_acc = fa;
        return;
      }
      if (da * (p.hi - p.lo) >= 0.0) {
        p.hi = p.lo; p.fhi = p.flo; p.dhi = p.dlo;
      }
      p.lo = a; p.flo = fa; p.dlo = da;
    }
  }
  if (p.ls_used >= max_evals) {
    p.a = 0.0;
    return;
  }
  // next zoom trial
  double aj = cubic_min(p.lo, p.flo, p.dlo, p.hi, p.fhi, p.dhi);
  const double w = p.hi - p.lo;
  const double b0 = w > 0 ? p.lo + 0.1 * w : p.hi - 0.1 * w;
  const double b1 = w > 0 ? p.hi - 0.1 * w : p.lo + 0.1 * w;
  if (!(aj >= std::min(b0, b1) && aj <= std::max(b0, b1))) aj = 0.5 * (p.lo + p.hi);
  p.a = aj;
}

// ---------------------------------------------------------------- host: the engine

struct BatchEngine {
  int device = 0, num_sms = 0;
  int T = 20, m = 10, max_iter = 100;
  double grad_tol = 1e-5;
  int schedule = GS_SCHED_ALL;
  StepConfig fcfg{}, bcfg{};
  int cap = 0;            // landmark capacity (multiple of kPad)
  int max_probs = 0;
  size_t bytes = 0;
  std::vector<void*> allocs;
  // packed arrays
  float4 *traj = nullptr, *adj = nullptr;
  double *q64 = nullptr, *p64 = nullptr, *a64 = nullptr, *b64 = nullptr, *t64 = nullptr, *hp0 = nullptr,
         *hq0 = nullptr, *gp64 = nullptr;
  float* qin = nullptr;
  double *x = nullptr, *g = nullptr, *d = nullptr, *xt = nullptr, *gt = nullptr, *S = nullptr, *Y = nullptr;
  double *red_h = nullptr, *red_m = nullptr;
  // per-problem device tables (indexed by problem slot)
  BatchProb* probs_d = nullptr;
  BatchItem* items_d = nullptr;
  int *list_d = nullptr, *item0_d = nullptr, *ntiles_d = nullptr, *slot_d = nullptr;
  double *loss_d = nullptr, *dots_d = nullptr, *a_d = nullptr, *alpha_d = nullptr, *dist_d = nullptr;
  TwoLoopState* state_d = nullptr;
  unsigned* status_d = nullptr;
  int max_items = 0;
  // host mirrors
  std::vector<BatchProb> probs_h;
  std::vector<Problem> slots;  // problem slots; slot index = row in probs_d
  std::vector<int> free_slots;
  std::vector<int> rejected;  // admitted with non-finite input, not yet reported
  std::vector<std::pair<int, int>> free_segs;  // (off, len) in landmarks
  cudaStream_t st = nullptr;
  std::chrono::steady_clock::time_point t0;
  // Pinned host mirrors of what every round uploads or reads back, so that
  // the copies are asynchronous and a round synchronises only where the
  // host needs a result: the item tables, the two-loop states, trial steps,
  // history slots, and a ring of problem lists (each upload takes the next
  // entry; the ring is longer than the uploads between two synchronisations).
  static constexpr int kListRing = 32;
  std::vector<void*> pinned;
  BatchItem* items_h = nullptr;  // forward items, then reverse items at + max_items
  int *item0_h = nullptr, *ntiles_h = nullptr, *slot_h = nullptr, *lists_h = nullptr;
  int list_next = 0;
  TwoLoopState* stv_h = nullptr;
  double *ah_h = nullptr, *loss_h = nullptr, *dots_h = nullptr;
  unsigned* status_h = nullptr;


  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  size_t stride() const { return 3 * static_cast<size_t>(cap); }

  gs_status init(int T_, int m_, int max_iter_, double tol, size_t budget, int max_probs_, cudaStream_t s) {
    T = T_;
    m = m_;
    max_iter = max_iter_;
    grad_tol = tol;
    st = s;
    t0 = std::chrono::steady_clock::now();
    GS_CUDA(cudaGetDevice(&device));
    GS_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
    // One kernel shape per kind for every problem of the engine (so that a
    // problem's sums split the same way alone and in any mix), fixed at
    // creation: batch_shape (the built-in shape, or a tuning override).
    int th = 0, cl = 0;
    batch_shape(0, &th, &cl);
    fcfg = step_config_for(0, 1 << 16, th, 1, cl);
    batch_shape(1, &th, &cl);
    bcfg = step_config_for(1, 1 << 16, th, 1, cl);
    if (fcfg.threads == 0 || bcfg.threads == 0) return fail(GS_EINVAL, "no packed kernel for the batch shape");
    max_probs = max_probs_;
    // bytes per landmark of capacity
    const size_t per = (T + 1) * kRecBytes / 2 + 2 * kRecBytes / 2 + 8 * 3 * sizeof(double) + 3 * sizeof(float) +
                       5 * 3 * sizeof(double) + 2 * static_cast<size_t>(m) * 3 * sizeof(double) +
                       2 * 16 * sizeof(double) / 64;
    const size_t fixed = 64u << 20;
    if (budget <= fixed + per * kPad) return fail(GS_EINVAL, "memory budget too small");
    cap = static_cast<int>(std::min<size_t>((budget - fixed) / per, size_t(1) << 28)) / kPad * kPad;
    // items: one per target tile of every problem, for the smaller of the
    // two kinds' tile sizes
    max_items = cap / std::min(fcfg.threads, bcfg.threads) + max_probs;
    auto get = [&](void** p, size_t b) -> cudaError_t {
      cudaError_t e = cudaMalloc(p, b + 256);
      if (e == cudaSuccess) {
        allocs.push_back(*p);
        bytes += b;
      }
      return e;
    };
    const size_t c3 = 3 * static_cast<size_t>(cap), slot = static_cast<size_t>(kRecF4) * (cap / 2);
    GS_CUDA(get((void**)&traj, sizeof(float4) * slot * (T + 1)));
    GS_CUDA(get((void**)&adj, sizeof(float4) * slot * 2));
    for (double** p : {&q64, &p64, &a64, &b64, &t64, &hp0, &hq0, &gp64, &x, &g, &d, &xt, &gt})
      GS_CUDA(get((void**)p, sizeof(double) * c3));
    GS_CUDA(get((void**)&S, sizeof(double) * c3 * m));
    GS_CUDA(get((void**)&Y, sizeof(double) * c3 * m));
    GS_CUDA(get((void**)&qin, sizeof(float) * c3));
    GS_CUDA(get((void**)&red_h, sizeof(double) * static_cast<size_t>(max_items) * 16));
    GS_CUDA(get((void**)&red_m, sizeof(double) * static_cast<size_t>(max_items) * 16));
    GS_CUDA(get((void**)&probs_d, sizeof(BatchProb) * max_probs));
    GS_CUDA(get((void**)&items_d, sizeof(BatchItem) * 2 * static_cast<size_t>(max_items)));
    for (int** p : {&list_d, &item0_d, &ntiles_d, &slot_d}) GS_CUDA(get((void**)p, sizeof(int) * max_probs));
    GS_CUDA(get((void**)&loss_d, sizeof(double) * max_probs));
    GS_CUDA(get((void**)&dots_d, sizeof(double) * 4 * max_probs));
    GS_CUDA(get((void**)&a_d, sizeof(double) * max_probs));
    GS_CUDA(get((void**)&alpha_d, sizeof(double) * kMaxM * max_probs));
    GS_CUDA(get((void**)&dist_d, sizeof(double) * 2 * max_probs));
    GS_CUDA(get((void**)&state_d, sizeof(TwoLoopState) * max_probs));
    GS_CUDA(get((void**)&status_d, sizeof(unsigned) * 8));
    GS_CUDA(cudaMemset(status_d, 0, sizeof(unsigned) * 8));
    auto host = [&](void** p, size_t b) -> cudaError_t {
      cudaError_t e = cudaMallocHost(p, b);
      if (e == cudaSuccess) pinned.push_back(*p);
      return e;
    };
    GS_CUDA(host((void**)&items_h, sizeof(BatchItem) * 2 * static_cast<size_t>(max_items)));
    for (int** p : {&item0_h, &ntiles_h, &slot_h}) GS_CUDA(host((void**)p, sizeof(int) * max_probs));
    GS_CUDA(host((void**)&lists_h, sizeof(int) * static_cast<size_t>(max_probs) * kListRing));
    GS_CUDA(host((void**)&stv_h, sizeof(TwoLoopState) * max_probs));
    GS_CUDA(host((void**)&ah_h, sizeof(double) * max_probs));
    GS_CUDA(host((void**)&loss_h, sizeof(double) * max_probs));
    GS_CUDA(host((void**)&dots_h, sizeof(double) * 4 * max_probs));
    GS_CUDA(host((void**)&status_h, sizeof(unsigned) * 8));
    // every optimiser vector starts at zero (never read before written, but
    // a stale NaN must not be able to leak through a zero coefficient)
    for (double* p : {x, g, d, xt, gt, q64, p64, a64, b64, t64, hp0, hq0, gp64})
      GS_CUDA(cudaMemset(p, 0, sizeof(double) * c3));
    GS_CUDA(cudaMemset(S, 0, sizeof(double) * c3 * m));
    GS_CUDA(cudaMemset(Y, 0, sizeof(double) * c3 * m));
    GS_CUDA(cudaMemset(traj, 0, sizeof(float4) * slot * (T + 1)));
    GS_CUDA(cudaMemset(adj, 0, sizeof(float4) * slot * 2));
    probs_h.assign(max_probs, BatchProb{});
    slots.assign(max_probs, Problem{});
    for (int i = max_probs - 1; i >= 0; --i) free_slots.push_back(i);
    free_segs.push_back({0, cap});
    return GS_OK;
  }

  void release() {
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    for (void* p : pinned) cudaFreeHost(p);
    pinned.clear();
  }

  int alloc_seg(int len) {
    for (size_t k = 0; k < free_segs.size(); ++k) {
      if (free_segs[k].second >= len) {
        const int off = free_segs[k].first;
        free_segs[k].first += len;
        free_segs[k].second -= len;
        if (free_segs[k].second == 0) free_segs.erase(free_segs.begin() + k);
        return off;
      }
    }
    return -1;
  }

  void free_seg(int off, int len) {
    free_segs.push_back({off, len});
    std::sort(free_segs.begin(), free_segs.end());
    std::vector<std::pair<int, int>> merged;
    for (auto& s : free_segs) {
      if (!merged.empty() && merged.back().first + merged.back().second == s.first)
        merged.back().second += s.second;
      else
        merged.push_back(s);
    }
    free_segs.swap(merged);
  }

  // Admit a problem: stage inputs into its segment.  Returns the slot, -1 if
  // there is no room now (capacity), or sets *err on a bad argument.
  int admit(const Problem& proto, const float* q0, const float* target, const float* p0, gs_status* err) {
    *err = GS_OK;
    if (free_slots.empty()) return -1;
    const int npad = round_up(proto.n, kPad);
    const int off = alloc_seg(npad);
    if (off < 0) return -1;
    const int sl = free_slots.back();
    free_slots.pop_back();
    // A newcomer starts at the smallest virtual time present (fair schedule).
    double vnow = -1.0;
    for (const Problem& o : slots)
      if (o.off >= 0 && o.phase != kDone && (vnow < 0.0 || o.vtime < vnow)) vnow = o.vtime;
    Problem& p = slots[sl];
    p = proto;
    p.vtime = vnow < 0.0 ? 0.0 : vnow;
    p.npad = npad;
    p.off = off;
    p.phase = kInit;
    p.t_admit = now();
    const KernelScales sc = make_scales(p.sigma);
    BatchProb bp;
    bp.off = off;
    bp.n = p.n;
    bp.npad = npad;
    int len = (npad + fcfg.cluster - 1) / fcfg.cluster;
    bp.split_len = (len + 7) / 8 * 8;
    len = (npad + bcfg.cluster - 1) / bcfg.cluster;
    bp.split_len_b = (len + 7) / 8 * 8;
    bp.pad_ = 0;
    bp.kq = sc.kq;
    bp.kappa = sc.kappa;
    bp.dt = 1.0 / T;
    bp.lambda = p.lambda;
    probs_h[sl] = bp;
    // The per-problem kernels of the next round read this row before any
    // gradient re-uploads the table, so it must be on the device now.
    {
      const cudaError_t eu = cudaMemcpyAsync(probs_d + sl, &probs_h[sl], sizeof(BatchProb), cudaMemcpyHostToDevice, st);
      if (eu != cudaSuccess) {
        *err = fail(GS_ECUDA, std::string("uploading a problem row: ") + cudaGetErrorString(eu));
        retire(sl);
        return -1;
      }
    }
    const size_t n3 = 3 * static_cast<size_t>(p.n), b3 = 3 * static_cast<size_t>(off);
    // A reused segment holds the previous problem's values.  Record padding
    // must be exactly zero, and the new problem starts from a clean state:
    // clear the segment in every record slot and every per-landmark array.
    {
      const size_t slot = static_cast<size_t>(kRecF4) * (cap / 2);
      const size_t r0 = static_cast<size_t>(kRecF4) * (off / 2), rl = static_cast<size_t>(kRecF4) * (npad / 2);
      cudaError_t e0 = cudaSuccess;
      for (int k = 0; k <= T && e0 == cudaSuccess; ++k)
        e0 = cudaMemsetAsync(traj + k * slot + r0, 0, rl * sizeof(float4), st);
      for (int k = 0; k < 2 && e0 == cudaSuccess; ++k) e0 = cudaMemsetAsync(adj + k * slot + r0, 0, rl * sizeof(float4), st);
      const size_t e3 = 3 * static_cast<size_t>(npad);
      for (double* arr : {q64, p64, a64, b64, t64, hp0, hq0, gp64, x, g, d, xt, gt})
        if (e0 == cudaSuccess) e0 = cudaMemsetAsync(arr + b3, 0, e3 * sizeof(double), st);
      for (int j = 0; j < m && e0 == cudaSuccess; ++j) {
        e0 = cudaMemsetAsync(S + j * stride() + b3, 0, e3 * sizeof(double), st);
        if (e0 == cudaSuccess) e0 = cudaMemsetAsync(Y + j * stride() + b3, 0, e3 * sizeof(double), st);
      }
      if (e0 == cudaSuccess) e0 = cudaMemsetAsync(qin + b3, 0, e3 * sizeof(float), st);
      if (e0 != cudaSuccess) {
        *err = fail(GS_ECUDA, std::string("clearing a segment: ") + cudaGetErrorString(e0));
        retire(sl);
        return -1;
      }
    }
    // Inputs: q0 -> qin (FP32), target -> t64, p0 -> x (FP64); padding zero.
    std::vector<double> tmp(3 * static_cast<size_t>(npad), 0.0);
    std::vector<float> tq(3 * static_cast<size_t>(npad), 0.f);
    auto fetch = [&](const float* src, float* dst) -> cudaError_t {
      if (!src) {
        std::fill(dst, dst + n3, 0.f);
        return cudaSuccess;
      }
      return cudaMemcpy(dst, src, n3 * sizeof(float), cudaMemcpyDefault);
    };
    cudaError_t e = fetch(q0, tq.data());
    if (e == cudaSuccess) e = cudaMemcpyAsync(qin + b3, tq.data(), tq.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    std::vector<float> tt(3 * static_cast<size_t>(npad), 0.f);
    if (e == cudaSuccess) e = fetch(target, tt.data());
    for (size_t i = 0; i < tt.size(); ++i) tmp[i] = tt[i];
    if (e == cudaSuccess) e = cudaMemcpyAsync(t64 + b3, tmp.data(), tmp.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    std::vector<float> tp(3 * static_cast<size_t>(npad), 0.f);
    if (e == cudaSuccess) e = fetch(p0, tp.data());
    for (size_t i = 0; i < tp.size(); ++i) tmp[i] = tp[i];
    if (e == cudaSuccess) e = cudaMemcpyAsync(x + b3, tmp.data(), tmp.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      *err = fail(GS_ECUDA, std::string("staging a problem: ") + cudaGetErrorString(e));
      retire(sl);
      return -1;
    }
    bool finite = true;
    for (size_t i = 0; i < n3; ++i)
      if (!std::isfinite(tq[i]) || !std::isfinite(tt[i]) || !std::isfinite(tp[i])) finite = false;
    if (!finite) {  // reported as failed by the next round, never evaluated
      p.phase = kDone;
      p.status = -1;
      rejected.push_back(sl);
    }
    return sl;
  }

  void retire(int sl) {
    Problem& p = slots[sl];
    if (p.off >= 0) free_seg(p.off, p.npad);
    p.off = -1;
    p.phase = kDone;
    free_slots.push_back(sl);
  }

  // Upload the problem table and the forward / reverse item tables of the
  // listed problems (items_d and items_d + max_items).  item0[b], ntiles[b]
  // describe each problem's forward items (for the loss reduction).
  //
  // The tables go through pinned mirrors: the previous round's copies out of
  // them finished at that round's last synchronisation, so no wait is needed
  // here.
  gs_status build_items(const std::vector<int>& list, int* n_fwd, int* n_bwd) {
    // largest problems first: their long CTAs start early
    std::vector<int> order(list);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return slots[a].n > slots[b].n; });
    const int Mf = fcfg.threads * fcfg.R, Mb = bcfg.threads * bcfg.R;
    int nf = 0, nb = 0;
    for (int b : order) {
      nf += (probs_h[b].npad + Mf - 1) / Mf;
      nb += (probs_h[b].npad + Mb - 1) / Mb;
    }
    if (std::max(nf, nb) > max_items) return fail(GS_ENOMEM, "batch item table full");
    BatchItem* fi = items_h;
    BatchItem* bi = items_h + max_items;
    std::fill(item0_h, item0_h + max_probs, 0);
    std::fill(ntiles_h, ntiles_h + max_probs, 0);
    nf = nb = 0;
    for (int b : order) {
      const int tf = (probs_h[b].npad + Mf - 1) / Mf, tb = (probs_h[b].npad + Mb - 1) / Mb;
      item0_h[b] = nf;
      ntiles_h[b] = tf;
      for (int t = 0; t < tf; ++t) fi[nf++] = BatchItem{b, t};
      for (int t = 0; t < tb; ++t) bi[nb++] = BatchItem{b, t};
    }
    GS_CUDA(cudaMemcpyAsync(probs_d, probs_h.data(), sizeof(BatchProb) * max_probs, cudaMemcpyHostToDevice, st));
    GS_CUDA(cudaMemcpyAsync(items_d, fi, sizeof(BatchItem) * nf, cudaMemcpyHostToDevice, st));
    GS_CUDA(cudaMemcpyAsync(items_d + max_items, bi, sizeof(BatchItem) * nb, cudaMemcpyHostToDevice, st));
    GS_CUDA(cudaMemcpyAsync(item0_d, item0_h, sizeof(int) * max_probs, cudaMemcpyHostToDevice, st));
    GS_CUDA(cudaMemcpyAsync(ntiles_d, ntiles_h, sizeof(int) * max_probs, cudaMemcpyHostToDevice, st));
    *n_fwd = nf;
    *n_bwd = nb;
    return GS_OK;
  }

  gs_status upload_list(const std::vector<int>& list) {
    int* h = lists_h + static_cast<size_t>(list_next) * max_probs;
    list_next = (list_next + 1) % kListRing;
    std::copy(list.begin(), list.end(), h);
    GS_CUDA(cudaMemcpyAsync(list_d, h, sizeof(int) * list.size(), cudaMemcpyHostToDevice, st));
    return GS_OK;
  }

  // The launches of one batched gradient of `count` listed problems (nf / nb
  // forward / reverse items) at p0 = xt, on stream cs: losses to loss_d,
  // FP64 gradients to gt; a forward flow only when grad is false.
  gs_status enqueue_gradient(cudaStream_t cs, int count, int nf, int nb, bool grad) {
    GS_CUDA(plaunch(count, kBT, cs, k_bpack, (const int*)list_d, (const BatchProb*)probs_d,
                    (const float*)qin, (const double*)xt, q64, p64, traj, status_d));
    const size_t slot = static_cast<size_t>(kRecF4) * (cap / 2);
    BatchTables bt{items_d, probs_d};
    StepConfig fc = fcfg, bc = bcfg;
    fc.policy = policy_for_grid(static_cast<long long>(nf) * fc.cluster, num_sms);
    bc.policy = policy_for_grid(static_cast<long long>(nb) * bc.cluster, num_sms);
    for (int k = 0; k < T; ++k) {
      StepFwdArgs a;
      std::memset(&a, 0, sizeof(a));
      a.qp = traj + k * slot;
      a.qp_next = traj + (k + 1) * slot;
      a.q64 = q64;
      a.p64 = p64;
      a.first = (k == 0);
      a.hp0 = hp0;
      a.hq0 = hq0;
      a.last = (k == T - 1);
      a.with_loss = grad ? 1 : 0;
      a.t64 = t64;
      a.a64 = a64;
      a.b64 = b64;
      a.ab = adj;
      a.red_h = red_h;
      a.red_m = red_m;
      a.status = status_d;
      a.combine64 = combine_f64() ? 1 : 0;
      GS_CUDA(launch_bstep_forward(fc, nf, a, bt, cs, k > 0));
    }
    if (!grad) return GS_OK;
    GS_CUDA(plaunch(count, 32, cs, k_bloss, (const int*)list_d, (const int*)item0_d,
                    (const int*)ntiles_d, (const BatchProb*)probs_d, (const double*)red_h, (const double*)red_m,
                    fcfg.cluster, loss_d));
    BatchTables btb{items_d + max_items, probs_d};
    for (int s2 = 0; s2 < T; ++s2) {
      const int k = T - 1 - s2;
      StepBwdArgs b;
      std::memset(&b, 0, sizeof(b));
      b.qp = traj + k * slot;
      b.ab = adj + (s2 & 1) * slot;
      b.ab_next = adj + ((s2 + 1) & 1) * slot;
      b.a64 = a64;
      b.b64 = b64;
      b.first = (k == 0);
      b.hp0 = hp0;
      b.hq0 = hq0;
      b.grad_p0_64 = gt;
      b.status = status_d;
      b.combine64 = combine_f64() ? 1 : 0;
      GS_CUDA(launch_bstep_backward(bc, nb, b, btb, cs, true));
    }
    return GS_OK;
  }

  // One batched gradient of the listed problems at p0 = xt: the tables are
  // uploaded, then the launch sequence is enqueued.  (Replaying that
  // sequence as a CUDA graph cached per shape measured no faster: a round of
  // small problems is bound by the latency of its chain of dependent
  // kernels, not by the launches.)
  gs_status gradient(const std::vector<int>& list, bool grad) {
    if (list.empty()) return GS_OK;
    int nf = 0, nb = 0;
    gs_status s = build_items(list, &nf, &nb);
    if (s != GS_OK) return s;
    if ((s = upload_list(list)) != GS_OK) return s;
    return enqueue_gradient(st, static_cast<int>(list.size()), nf, nb, grad);
  }

  // Dot products of the listed problems, read back with one
  // synchronisation; with_loss also reads the losses (loss_h) and the device
  // status word in the same wait, and reports an expired wait or a bad
  // launch.
  gs_status dots(const std::vector<int>& list, const DotSpec& spec, std::vector<double>* out,
                 bool with_loss = false) {
    if (list.empty()) return GS_OK;
    if ((upload_list(list)) != GS_OK) return GS_ECUDA;
    GS_CUDA(plaunch(static_cast<int>(list.size()), kBT, st, k_bdots, (const int*)list_d, (const BatchProb*)probs_d, spec,
                    dots_d));
    GS_CUDA(cudaMemcpyAsync(dots_h, dots_d, sizeof(double) * 4 * max_probs, cudaMemcpyDeviceToHost, st));
    if (with_loss) {
      GS_CUDA(cudaMemcpyAsync(loss_h, loss_d, sizeof(double) * max_probs, cudaMemcpyDeviceToHost, st));
      GS_CUDA(cudaMemcpyAsync(status_h, status_d, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    }
    GS_CUDA(cudaStreamSynchronize(st));
    out->assign(dots_h, dots_h + 4 * static_cast<size_t>(max_probs));
    if (with_loss) {
      if (*status_h & kErrTimeout) return fail(GS_ETIMEOUT, "a device-side wait expired");
      if (*status_h & kErrBadLaunch) return fail(GS_ECUDA, "device reported an inconsistent launch");
    }
    return GS_OK;
  }

  gs_status vec(int op, const std::vector<int>& list, const int* slot_host) {
    if (list.empty()) return GS_OK;
    if (upload_list(list) != GS_OK) return GS_ECUDA;
    if (slot_host) {
      std::copy(slot_host, slot_host + max_probs, slot_h);
      GS_CUDA(cudaMemcpyAsync(slot_d, slot_h, sizeof(int) * max_probs, cudaMemcpyHostToDevice, st));
    }
    GS_CUDA(plaunch(static_cast<int>(list.size()), kBT, st, k_bvec, op, (const int*)list_d, (const BatchProb*)probs_d,
                    (const double*)a_d, (const int*)(slot_host ? slot_d : nullptr), stride(), x, g, d, xt, gt, S, Y));
    return GS_OK;
  }


  // One round over the active problems the schedule selects (all of them,
  // or under the fair schedule those behind in charged pair work; see the
  // file comment).  Returns the slots that finished in this round in *done.
  gs_status round(std::vector<int>* done) {
    done->insert(done->end(), rejected.begin(), rejected.end());
    rejected.clear();
    std::vector<int> active, need_dir;
    double vmin = 0.0, cmin = 0.0;
    bool first = true;
    for (int sl = 0; sl < max_probs; ++sl) {
      const Problem& p = slots[sl];
      if (p.off < 0 || p.phase == kDone) continue;
      const double c = static_cast<double>(p.n) * p.n;
      if (first || p.vtime < vmin) vmin = p.vtime;
      if (first || c < cmin) cmin = c;
      first = false;
    }
    for (int sl = 0; sl < max_probs; ++sl) {
      Problem& p = slots[sl];
      if (p.off < 0 || p.phase == kDone) continue;
      // Fair schedule: the requests that are behind in charged pair work.
      if (schedule == GS_SCHED_FAIR && !(p.vtime < vmin + cmin)) continue;
      p.vtime += static_cast<double>(p.n) * p.n;
      active.push_back(sl);
      if (p.phase == kNeedDir) need_dir.push_back(sl);
    }
    if (active.empty()) return GS_OK;
    gs_status s;
    // 1. directions
    if (!need_dir.empty()) {
      TwoLoopState* stv = stv_h;
      for (int sl : need_dir) {
        Problem& p = slots[sl];
        stv[sl].head = p.head;
        stv[sl].stored = p.stored;
        stv[sl].gamma = p.gamma;
        std::memcpy(stv[sl].rho, p.rho, sizeof(p.rho));
      }
      GS_CUDA(cudaMemcpyAsync(state_d, stv, sizeof(TwoLoopState) * max_probs, cudaMemcpyHostToDevice, st));
      if ((s = upload_list(need_dir)) != GS_OK) return s;
      GS_CUDA(plaunch(static_cast<int>(need_dir.size()), kBT, st, k_btwoloop, (const int*)list_d,
                      (const BatchProb*)probs_d, (const TwoLoopState*)state_d, m, stride(), (const double*)g,
                      (const double*)S, (const double*)Y, d, alpha_d));
      DotSpec sp{};
      sp.a[0] = g; sp.b[0] = d; sp.a[1] = g; sp.b[1] = g;
      sp.count = 2;
      std::vector<double> r;
      if ((s = dots(need_dir, sp, &r)) != GS_OK) return s;  // synchronises
      std::vector<int> restart;
      for (int sl : need_dir) {
        Problem& p = slots[sl];
        p.dphi0 = r[4 * sl];
        if (!(p.dphi0 < 0.0)) {
          restart.push_back(sl);
          p.dphi0 = -r[4 * sl + 1];
          p.stored = 0;
        }
        p.f0 = p.f;
        p.a = (p.iters == 0) ? 1.0 / p.g0 : 1.0;
        p.a_prev = 0.0; p.f_prev = p.f0; p.d_prev = p.dphi0;
        p.zoom = false; p.ls_it = 0; p.ls_used = 0; p.accepted = false;
        p.phase = kSearch;
      }
      if ((s = vec(1, restart, nullptr)) != GS_OK) return s;
    }
    // 2. trial points and one batched gradient
    double* ah = ah_h;
    std::fill(ah, ah + max_probs, 0.0);
    std::vector<int> search;
    for (int sl : active) {
      Problem& p = slots[sl];
      if (p.phase == kSearch) {
        ah[sl] = p.a;
        search.push_back(sl);
      }
    }
    GS_CUDA(cudaMemcpyAsync(a_d, ah, sizeof(double) * max_probs, cudaMemcpyHostToDevice, st));
    if ((s = vec(0, search, nullptr)) != GS_OK) return s;   // xt = x + a d
    std::vector<int> init;
    for (int sl : active)
      if (slots[sl].phase == kInit) init.push_back(sl);
    if ((s = vec(4, init, nullptr)) != GS_OK) return s;  // xt = x for the first evaluation
    if ((s = gradient(active, true)) != GS_OK) return s;
    DotSpec sp{};
    sp.a[0] = gt; sp.b[0] = d; sp.a[1] = gt; sp.b[1] = gt;
    sp.count = 2;
    std::vector<double> r;
    if ((s = dots(active, sp, &r, true)) != GS_OK) return s;  // also the losses and the status word
    const std::vector<double> loss(loss_h, loss_h + max_probs);
    // 3. advance the state machines
    std::vector<int> accepted, to_copy;
    for (int sl : active) {
      Problem& p = slots[sl];
      ++p.evals;
      const double f = loss[sl];
      if (p.phase == kInit) {
        p.f = f;
        p.g0 = p.gnorm = std::sqrt(r[4 * sl + 1]);
        to_copy.push_back(sl);  // x = xt (unchanged), g = gt
        p.phase = (p.g0 == 0.0 || p.iters >= max_iter) ? kDone : kNeedDir;
        p.status = (p.g0 == 0.0) ? 0 : 1;
        if (!std::isfinite(f)) { p.phase = kDone; p.status = -1; }
        continue;
      }
      if (!std::isfinite(f) || !std::isfinite(r[4 * sl])) {
        p.phase = kDone;
        p.status = -1;
        continue;
      }
      line_search_advance(p, f, r[4 * sl]);
      if (p.accepted) {
        accepted.push_back(sl);
      } else if (p.a == 0.0) {
        p.phase = kDone;
        p.status = 2;
      }
    }
    if (!to_copy.empty() && (s = vec(3, to_copy, nullptr)) != GS_OK) return s;
    if (!accepted.empty()) {
      std::vector<int> slot_host(max_probs, 0);
      for (int sl : accepted) slot_host[sl] = slots[sl].head;
      if ((s = vec(2, accepted, slot_host.data())) != GS_OK) return s;  // s, y into the head slot (uploads slot_d)
      DotSpec u{};
      u.a[0] = S; u.b[0] = Y; u.a[1] = Y; u.b[1] = Y; u.a[2] = S; u.b[2] = S; u.a[3] = gt; u.b[3] = gt;
      u.slot_a = slot_d; u.slot_b = slot_d;
      u.stride = stride();
      u.count = 3;
      // the fourth product (gt.gt) does not use the history slot
      std::vector<double> r3;
      if ((s = dots(accepted, u, &r3)) != GS_OK) return s;
      if ((s = vec(3, accepted, nullptr)) != GS_OK) return s;  // x = xt, g = gt
      for (int sl : accepted) {
        Problem& p = slots[sl];
        const double sy = r3[4 * sl], yy = r3[4 * sl + 1], ss = r3[4 * sl + 2];
        if (sy > 1e-12 * std::sqrt(ss * yy)) {
          p.rho[p.head] = 1.0 / sy;
          p.gamma = sy / yy;
          p.head = (p.head + 1) % m;
          if (p.stored < m) ++p.stored;
        }
        p.f = p.f_acc;
        p.gnorm = std::sqrt(r[4 * sl + 1]);
        ++p.iters;
        if (p.gnorm <= grad_tol * p.g0) {
          p.phase = kDone;
          p.status = 0;
        } else if (p.iters >= max_iter) {
          p.phase = kDone;
          p.status = 1;
        } else {
          p.phase = kNeedDir;
        }
      }
    }
    for (int sl : active)
      if (slots[sl].phase == kDone) done->push_back(sl);
    return GS_OK;
  }

  // Final outputs of finished problems: p0 (FP32) and the distances at q(1).
  gs_status finish(const std::vector<int>& done) {
    if (done.empty()) return GS_OK;
    // q(1) at the final p0: one batched forward flow (not for requests
    // rejected at admission, which have no state to flow)
    std::vector<int> flow;
    for (int sl : done)
      if (slots[sl].evals > 0) flow.push_back(sl);
    gs_status s = vec(4, flow, nullptr);  // xt = x
    if (s != GS_OK) return s;
    if ((s = gradient(flow, false)) != GS_OK) return s;
    std::vector<double> dist(2 * static_cast<size_t>(max_probs), NAN);
    if (!flow.empty()) {
      if ((s = upload_list(flow)) != GS_OK) return s;
      GS_CUDA(plaunch(static_cast<int>(flow.size()), kBT, st, k_bdist, (const int*)list_d,
                      (const BatchProb*)probs_d, (const double*)q64, (const double*)t64, dist_d));
    }
    std::vector<double> dist_dev(2 * static_cast<size_t>(max_probs), 0.0);
    GS_CUDA(cudaMemcpyAsync(dist_dev.data(), dist_d, sizeof(double) * 2 * max_probs, cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    for (int sl : flow) {
      dist[2 * sl] = dist_dev[2 * sl];
      dist[2 * sl + 1] = dist_dev[2 * sl + 1];
    }
    const double tnow = now();
    for (int sl : done) {
      Problem& p = slots[sl];
      std::vector<double> xh(3 * static_cast<size_t>(p.n));
      // on this engine's stream: a second lane may be running on another
      GS_CUDA(cudaMemcpyAsync(xh.data(), x + 3 * static_cast<size_t>(p.off), xh.size() * sizeof(double),
                              cudaMemcpyDeviceToHost, st));
      GS_CUDA(cudaStreamSynchronize(st));
      p.p0_result.resize(xh.size());
      for (size_t i = 0; i < xh.size(); ++i) p.p0_result[i] = static_cast<float>(xh[i]);
      p.result.loss = p.f;
      p.result.grad_norm0 = p.g0;
      p.result.grad_norm = p.gnorm;
      p.result.avg_dist = dist[2 * sl];
      p.result.max_dist = dist[2 * sl + 1];
      p.result.iters = p.iters;
      p.result.evals = p.evals;
      p.result.status = p.status;
      p.t_done = tnow;
    }
    return GS_OK;
  }
};

}  // namespace
}  // namespace gs

// ---------------------------------------------------------------- C ABI

struct gs_server {
  gs::BatchEngine eng;    // every request; under GS_SCHED_LANES the large ones
  // GS_SCHED_LANES: requests of at most lane_split landmarks run in a second
  // engine on its own stream, under the fair schedule, concurrently with the
  // large lane's rounds.
  bool lanes = false;
  int lane_split = 0;
  gs::BatchEngine small;
  cudaStream_t small_st = nullptr;
  std::mutex mu;
  struct Pending {
    gs::Problem proto;
    std::vector<float> q0, target, p0;
  };
  std::deque<Pending> queue;            // submitted, not yet admitted
  std::map<int64_t, int> admitted;      // request id -> slot (lanes: slot + lane * kLaneTag)
  std::map<int64_t, gs::Problem> finished;
  int64_t next_id = 1;
};

namespace {

constexpr int kLaneTag = 1 << 24;  // admitted[] value offset of the small lane's slots

gs_status server_admit(gs_server* sv) {
  // admit in arrival order while a segment fits (in the request's lane)
  while (!sv->queue.empty()) {
    gs_server::Pending& pd = sv->queue.front();
    const bool small = sv->lanes && pd.proto.n <= sv->lane_split;
    gs::BatchEngine& e = small ? sv->small : sv->eng;
    gs_status err = GS_OK;
    const int sl = e.admit(pd.proto, pd.q0.data(), pd.target.data(), pd.p0.empty() ? nullptr : pd.p0.data(), &err);
    if (err != GS_OK) return err;
    if (sl < 0) break;  // no room until something finishes
    sv->admitted[pd.proto.id] = sl + (small ? kLaneTag : 0);
    sv->queue.pop_front();
  }
  return GS_OK;
}

bool has_active(const gs::BatchEngine& e) {
  for (const gs::Problem& p : e.slots)
    if (p.off >= 0 && p.phase != gs::kDone) return true;
  return false;
}

// Move an engine's finished problems to the server's results and free them.
void collect(gs_server* sv, gs::BatchEngine& e, const std::vector<int>& done) {
  for (int sl : done) {
    gs::Problem& p = e.slots[sl];
    sv->finished[p.id] = p;
    sv->admitted.erase(p.id);
    e.retire(sl);
  }
}

}  // namespace

extern "C" {

gs_status gs_server_create(const gs_server_config* cfg, gs_server** out) {
  gs::set_last_error("");
  if (!cfg || !out) {
    gs::set_last_error("cfg and out must not be NULL");
    return GS_EINVAL;
  }
  if (cfg->T < 1 || cfg->lbfgs_m < 1 || cfg->lbfgs_m > gs::kMaxM || cfg->max_iter < 0 || cfg->max_problems < 1) {
    gs::set_last_error("bad server configuration");
    return GS_EINVAL;
  }
  if (cfg->schedule != GS_SCHED_ALL && cfg->schedule != GS_SCHED_FAIR && cfg->schedule != GS_SCHED_LANES) {
    gs::set_last_error("schedule must be GS_SCHED_ALL, GS_SCHED_FAIR or GS_SCHED_LANES");
    return GS_EINVAL;
  }
  if (cfg->lane_split < 0 || (cfg->lane_split != 0 && cfg->schedule != GS_SCHED_LANES)) {
    gs::set_last_error("lane_split must be 0, or >= 1 with GS_SCHED_LANES");
    return GS_EINVAL;
  }
  gs_server* sv = new gs_server();
  gs_status s = GS_OK;
  if (cfg->schedule == GS_SCHED_LANES) {
    // a quarter of the budget for the small lane, the rest for the large one
    sv->lanes = true;
    sv->lane_split = cfg->lane_split > 0 ? cfg->lane_split : 8192;
    sv->eng.schedule = GS_SCHED_ALL;
    sv->small.schedule = GS_SCHED_FAIR;
    const uint64_t small_budget = cfg->memory_budget / 4;
    // The small lane's stream has the device's highest priority: its short
    // kernels take SM slots as the large lane's CTAs finish instead of
    // queueing behind every CTA of a large launch.
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sv->small_st, cudaStreamNonBlocking, greatest);
    if (e != cudaSuccess) {
      gs::set_last_error(cudaGetErrorString(e));
      delete sv;
      return GS_ECUDA;
    }
    s = sv->small.init(cfg->T, cfg->lbfgs_m, cfg->max_iter, cfg->grad_tol, small_budget, cfg->max_problems,
                       sv->small_st);
    if (s == GS_OK)
      s = sv->eng.init(cfg->T, cfg->lbfgs_m, cfg->max_iter, cfg->grad_tol, cfg->memory_budget - small_budget,
                       cfg->max_problems, static_cast<cudaStream_t>(cfg->stream));
    sv->small.t0 = sv->eng.t0;  // one clock for every request's timestamps
  } else {
    sv->eng.schedule = cfg->schedule;
    s = sv->eng.init(cfg->T, cfg->lbfgs_m, cfg->max_iter, cfg->grad_tol, cfg->memory_budget, cfg->max_problems,
                     static_cast<cudaStream_t>(cfg->stream));
  }
  if (s != GS_OK) {
    sv->eng.release();
    sv->small.release();
    if (sv->small_st) cudaStreamDestroy(sv->small_st);
    delete sv;
    return s;
  }
  *out = sv;
  return GS_OK;
}

gs_status gs_server_submit(gs_server* sv, int64_t N, double sigma, double lambda, const float* q0,
                           const float* target, const float* p0, int64_t* request_id) {
  gs::set_last_error("");
  if (!sv || !q0 || !target || N < 1 || N > (1LL << 26) || !(sigma > 0.0) || !std::isfinite(sigma) ||
      !(lambda >= 0.0) || !std::isfinite(lambda)) {
    gs::set_last_error("bad request");
    return GS_EINVAL;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  const gs::BatchEngine& lane = sv->lanes && N <= sv->lane_split ? sv->small : sv->eng;
  if (gs::round_up(N, gs::kPad) > lane.cap) {
    gs::set_last_error("request larger than the server's memory budget");
    return GS_ENOMEM;
  }
  gs_server::Pending pd;
  pd.proto.id = sv->next_id++;
  pd.proto.n = static_cast<int>(N);
  pd.proto.sigma = sigma;
  pd.proto.lambda = lambda;
  pd.proto.t_submit = sv->eng.now();
  const size_t n3 = 3 * static_cast<size_t>(N);
  pd.q0.resize(n3);
  pd.target.resize(n3);
  cudaError_t e = cudaMemcpy(pd.q0.data(), q0, n3 * sizeof(float), cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(pd.target.data(), target, n3 * sizeof(float), cudaMemcpyDefault);
  if (e == cudaSuccess && p0) {
    pd.p0.resize(n3);
    e = cudaMemcpy(pd.p0.data(), p0, n3 * sizeof(float), cudaMemcpyDefault);
  }
  if (e != cudaSuccess) {
    gs::set_last_error(cudaGetErrorString(e));
    return GS_ECUDA;
  }
  if (request_id) *request_id = pd.proto.id;
  sv->queue.push_back(std::move(pd));
  return GS_OK;
}

gs_status gs_server_step(gs_server* sv, int32_t* active, int32_t* queued, int32_t* completed) {
  gs::set_last_error("");
  if (!sv) return GS_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  gs_status s = server_admit(sv);
  if (s != GS_OK) return s;
  std::vector<int> done, done_small;
  const bool run_small = sv->lanes && has_active(sv->small);
  if (run_small && has_active(sv->eng)) {
    // One round of the large lane on this thread; meanwhile the small lane
    // runs rounds on a worker thread, on its own stream, until the large
    // round is over (at least one).
    std::atomic<bool> large_done{false};
    gs_status s_small = GS_OK;
    std::string why_small;  // the worker's error message (the message slot is per thread)
    const int device = sv->eng.device;
    std::thread worker([&] {
      const cudaError_t e = cudaSetDevice(device);
      if (e != cudaSuccess) {
        s_small = GS_ECUDA;
        why_small = cudaGetErrorString(e);
        return;
      }
      do {
        std::vector<int> d;
        if ((s_small = sv->small.round(&d)) == GS_OK) s_small = sv->small.finish(d);
        if (s_small != GS_OK) {
          why_small = gs_last_error();
          return;
        }
        done_small.insert(done_small.end(), d.begin(), d.end());
      } while (!large_done.load() && has_active(sv->small));
    });
    s = sv->eng.round(&done);
    if (s == GS_OK) s = sv->eng.finish(done);
    large_done.store(true);
    worker.join();
    if (s != GS_OK) return s;
    if (s_small != GS_OK) return gs::fail(s_small, "small lane: " + why_small);
  } else if (run_small) {
    if ((s = sv->small.round(&done_small)) != GS_OK) return s;
    if ((s = sv->small.finish(done_small)) != GS_OK) return s;
  } else {
    if ((s = sv->eng.round(&done)) != GS_OK) return s;
    if ((s = sv->eng.finish(done)) != GS_OK) return s;
  }
  collect(sv, sv->eng, done);
  collect(sv, sv->small, done_small);
  if ((s = server_admit(sv)) != GS_OK) return s;
  if (active) *active = static_cast<int32_t>(sv->admitted.size());
  if (queued) *queued = static_cast<int32_t>(sv->queue.size());
  if (completed) *completed = static_cast<int32_t>(done.size() + done_small.size());
  return GS_OK;
}

gs_status gs_server_poll(gs_server* sv, int64_t request_id, float* p0_out, gs_register_info* info,
                         double* latency, int32_t* done) {
  gs::set_last_error("");
  if (!sv || !done) return GS_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->finished.find(request_id);
  if (it == sv->finished.end()) {
    *done = 0;
    return GS_OK;
  }
  const gs::Problem& p = it->second;
  *done = 1;
  if (p0_out) {
    cudaError_t e = cudaMemcpy(p0_out, p.p0_result.data(), p.p0_result.size() * sizeof(float), cudaMemcpyDefault);
    if (e != cudaSuccess) {
      gs::set_last_error(cudaGetErrorString(e));
      return GS_ECUDA;
    }
  }
  if (info) *info = p.result;
  if (latency) {
    latency[0] = p.t_done - p.t_submit;  // submission to result
    latency[1] = p.t_done - p.t_admit;   // admission to result
  }
  if (p.status < 0) {
    gs::set_last_error("non-finite input or intermediate in this request");
    return GS_ENONFINITE;
  }
  return GS_OK;
}

gs_status gs_server_stats(gs_server* sv, int64_t* capacity_landmarks, int64_t* free_landmarks, int64_t* bytes) {
  if (!sv) return GS_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  int64_t fr = 0;
  for (auto& s : sv->eng.free_segs) fr += s.second;
  for (auto& s : sv->small.free_segs) fr += s.second;
  if (capacity_landmarks) *capacity_landmarks = static_cast<int64_t>(sv->eng.cap) + sv->small.cap;
  if (free_landmarks) *free_landmarks = fr;
  if (bytes) *bytes = static_cast<int64_t>(sv->eng.bytes + sv->small.bytes);
  return GS_OK;
}

void gs_server_destroy(gs_server* sv) {
  if (!sv) return;
  sv->eng.release();
  sv->small.release();
  if (sv->small_st) cudaStreamDestroy(sv->small_st);
  delete sv;
}

gs_status register_batch(int32_t B, gs_batch_problem* probs, int32_t T, int32_t lbfgs_m, int32_t max_iter,
                         double grad_tol, void* stream) {
  gs::set_last_error("");
  if (B < 1 || !probs) {
    gs::set_last_error("B must be >= 1 and probs non-NULL");
    return GS_EINVAL;
  }
  size_t need = 0;
  for (int b = 0; b < B; ++b) need += gs::round_up(probs[b].N, gs::kPad);
  gs_server_config cfg{};
  cfg.T = T;
  cfg.lbfgs_m = lbfgs_m;
  cfg.max_iter = max_iter;
  cfg.grad_tol = grad_tol;
  cfg.max_problems = B;
  // room for every problem at once (about 1.4 KB per landmark at T = 20, m = 10)
  cfg.memory_budget = (96u << 20) + need * (static_cast<size_t>(T + 3) * 24 + 13 * 24 + 12 + 48 * lbfgs_m + 64);
  cfg.stream = stream;
  gs_server* sv = nullptr;
  gs_status s = gs_server_create(&cfg, &sv);
  if (s != GS_OK) return s;
  std::vector<int64_t> ids(B);
  for (int b = 0; b < B; ++b) {
    s = gs_server_submit(sv, probs[b].N, probs[b].sigma, probs[b].lambda, probs[b].q0, probs[b].target,
                         probs[b].p0, &ids[b]);
    if (s != GS_OK) {
      gs_server_destroy(sv);
      return s;
    }
  }
  int32_t active = 1, queued = 1;
  while (active > 0 || queued > 0) {
    if ((s = gs_server_step(sv, &active, &queued, nullptr)) != GS_OK) {
      gs_server_destroy(sv);
      return s;
    }
  }
  gs_status worst = GS_OK;
  for (int b = 0; b < B; ++b) {
    int32_t done = 0;
    s = gs_server_poll(sv, ids[b], probs[b].p0, &probs[b].info, nullptr, &done);
    if (s < 0) worst = s;
    else if (probs[b].info.status != 0 && worst == GS_OK) worst = GS_NOT_CONVERGED;
  }
  gs_server_destroy(sv);
  return worst;
}

}  // extern "C"
