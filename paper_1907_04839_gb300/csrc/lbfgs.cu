// register_landmarks: minimise the loss of Eq. 3 over p0 by L-BFGS
// (Section 2.1; the outer optimisation of Algorithm 1).  The paper used
// VNL's L-BFGS without stating its settings; this one uses textbook choices:
//  * memory m, two-loop recursion with initial scaling gamma = s.y / y.y;
//  * first step -g scaled to 1/||g0||;
//  * strong-Wolfe line search (c1 = 1e-4, c2 = 0.9) by bracketing and zoom
//    with safeguarded cubic interpolation, at most 20 evaluations per search;
//  * a curvature pair is kept only if s.y > 1e-12 ||s|| ||y||;
//  * stop when ||g|| <= grad_tol ||g0||, or after max_iter iterations.
//
// The iterate, the gradient, the direction and the (s, y) history are FP64
// vectors on the device.  Dot products reduce deterministically: per-CTA
// partials, then the last CTA adds them in a fixed order.  The host runs the
// scalar control flow of the line search.  Each evaluation is one replay of
// the gradient graph at FP64 momenta, which returns the loss and
// phi'(a) = g.d to the host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "engine.h"
#include "gs_device.cuh"

namespace gs {
namespace {

constexpr int kLT = 256;     // threads per CTA of the vector kernels
constexpr int kMaxDots = 4;  // dot products computed in one pass
constexpr int kMaxM = 64;

// scal[] slots
constexpr int kAlpha = 0;             // alpha[m]
constexpr int kDots = kMaxM + 1;      // results of the last k_dots pass (kMaxM: spare)

int vec_grid(int n, int num_sms) { return std::max(1, std::min((n + kLT - 1) / kLT, 2 * num_sms)); }

struct DotArgs {
  const double* a[kMaxDots];
  const double* b[kMaxDots];
  int count;
  int n;
  double mult[kMaxDots];
  double* part;       // [count][gridDim.x]
  unsigned* ticket;
  double* out;        // out[k] = mult[k] * a[k].b[k]
};

// Up to four dot products in one pass, reduced deterministically.
__global__ void __launch_bounds__(kLT) k_dots(DotArgs d) {
  __shared__ double sh[kLT / 32];
  __shared__ int am_last;
  double v[kMaxDots] = {0.0, 0.0, 0.0, 0.0};
  for (int i = blockIdx.x * kLT + threadIdx.x; i < d.n; i += gridDim.x * kLT) {
#pragma unroll
    for (int k = 0; k < kMaxDots; ++k)
      if (k < d.count) v[k] = fma(d.a[k][i], d.b[k][i], v[k]);
  }
#pragma unroll
  for (int k = 0; k < kMaxDots; ++k) {
    if (k >= d.count) break;
    const double bs = block_sum_f64(v[k], sh);
    if (threadIdx.x == 0) d.part[k * gridDim.x + blockIdx.x] = bs;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    am_last = (atomicAdd(d.ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last || threadIdx.x >= 32) return;
  __threadfence();
  for (int k = 0; k < d.count; ++k) {
    double t = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += 32) t += *((volatile double*)&d.part[k * gridDim.x + b]);
    t = warp_sum_f64(t);
    if (threadIdx.x == 0) d.out[k] = d.mult[k] * t;
  }
  if (threadIdx.x == 0) *d.ticket = 0u;
}

// y <- y + (c0 + c1 * sa[0] + c2 * sb[0]) x   (sa, sb device scalars or null)
__global__ void __launch_bounds__(kLT) k_axpy(double* y, const double* x, int n, double c0, double c1,
                                             const double* sa, double c2, const double* sb) {
  const double coef = c0 + (sa ? c1 * sa[0] : 0.0) + (sb ? c2 * sb[0] : 0.0);
  for (int i = blockIdx.x * kLT + threadIdx.x; i < n; i += gridDim.x * kLT) y[i] = fma(coef, x[i], y[i]);
}

// y <- c x
__global__ void __launch_bounds__(kLT) k_scale(double* y, const double* x, int n, double c) {
  for (int i = blockIdx.x * kLT + threadIdx.x; i < n; i += gridDim.x * kLT) y[i] = c * x[i];
}

// xt <- x + a d
__global__ void __launch_bounds__(kLT) k_step(double* xt, const double* x, const double* d, int n, double a) {
  for (int i = blockIdx.x * kLT + threadIdx.x; i < n; i += gridDim.x * kLT) xt[i] = fma(a, d[i], x[i]);
}

// s <- xt - x, y <- gt - g
__global__ void __launch_bounds__(kLT) k_pair(double* s, double* y, const double* xt, const double* x,
                                             const double* gt, const double* g, int n) {
  for (int i = blockIdx.x * kLT + threadIdx.x; i < n; i += gridDim.x * kLT) {
    s[i] = xt[i] - x[i];
    y[i] = gt[i] - g[i];
  }
}

__global__ void __launch_bounds__(kLT) k_f32_to_f64(double* y, const float* x, int n) {
  for (int i = blockIdx.x * kLT + threadIdx.x; i < n; i += gridDim.x * kLT) y[i] = x ? (double)x[i] : 0.0;
}

__global__ void __launch_bounds__(kLT) k_f64_to_f32(float* y, const double* x, int n) {
  for (int i = blockIdx.x * kLT + threadIdx.x; i < n; i += gridDim.x * kLT) y[i] = (float)x[i];
}

// Landmark distances |q1_i - t_i| (Section 3.1): out[0] = sum, out[1] = max.
// Landmarks in dim = 2 or 3 dimensions.
__global__ void __launch_bounds__(kLT) k_dist(const double* q1, const double* t, int n, int dim, double* part,
                                             unsigned* ticket, double* out) {
  __shared__ double sh[kLT / 32];
  __shared__ double shm[kLT / 32];
  __shared__ int am_last;
  double sum = 0.0, mx = 0.0;
  for (int i = blockIdx.x * kLT + threadIdx.x; i < n; i += gridDim.x * kLT) {
    double r2 = 0.0;
    for (int k = 0; k < dim; ++k) {
      const double d = q1[dim * i + k] - t[dim * i + k];
      r2 += d * d;
    }
    const double r = sqrt(r2);
    sum += r;
    mx = fmax(mx, r);
  }
  const double bs = block_sum_f64(sum, sh);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < kLT / 32; ++w) m = fmax(m, shm[w]);
    part[blockIdx.x] = bs;
    part[gridDim.x + blockIdx.x] = m;
    __threadfence();
    am_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last || threadIdx.x != 0) return;
  __threadfence();
  double s = 0.0, m = 0.0;
  for (unsigned b = 0; b < gridDim.x; ++b) {
    s += *((volatile double*)&part[b]);
    m = fmax(m, *((volatile double*)&part[gridDim.x + b]));
  }
  out[0] = s;
  out[1] = m;
  *ticket = 0u;
}

template <typename K, typename... Args>
cudaError_t vlaunch(int grid, cudaStream_t st, K kern, Args... args) {
  kern<<<grid, kLT, 0, st>>>(args...);
  return cudaGetLastError();
}

gs_status alloc_lbfgs(Workspace& w, int n3, int m) {
  LbfgsBufs& b = w.lb;
  if (b.n3 >= n3 && b.m >= m) return GS_OK;
  b.free_all();
  auto get = [&](double** p, size_t count) -> cudaError_t {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, count * sizeof(double) + 256);
    if (e == cudaSuccess) {
      b.allocs.push_back(v);
      *p = static_cast<double*>(v);
    }
    return e;
  };
  const size_t n = static_cast<size_t>(n3);
  GS_CUDA(get(&b.x, n));
  GS_CUDA(get(&b.g, n));
  GS_CUDA(get(&b.d, n));
  GS_CUDA(get(&b.xt, n));
  GS_CUDA(get(&b.gt, n));
  GS_CUDA(get(&b.S, n * m));
  GS_CUDA(get(&b.Y, n * m));
  GS_CUDA(get(&b.scal, kMaxM + 16));
  GS_CUDA(get(&b.part, kMaxDots * 4 * 1024));
  double* t = nullptr;
  GS_CUDA(get(&t, 8));
  b.ticket = reinterpret_cast<unsigned*>(t);
  GS_CUDA(cudaMemset(b.ticket, 0, 8 * sizeof(double)));
  GS_CUDA(cudaMemset(b.S, 0, n * m * sizeof(double)));
  GS_CUDA(cudaMemset(b.Y, 0, n * m * sizeof(double)));
  b.n3 = n3;
  b.m = m;
  return GS_OK;
}

// One register_landmarks run on the current device (caller holds the lock).
struct Lbfgs {
  Workspace& w;
  const gs_params& prm;
  cudaStream_t st;
  const float* dq;
  const float* dt;
  int n3, m, grid;
  int evals = 0;

  Lbfgs(Workspace& w_, const gs_params& p, cudaStream_t s, const float* q, const float* t)
      : w(w_), prm(p), st(s), dq(q), dt(t), n3(static_cast<int>(dim_of(p) * p.N)), m(p.lbfgs_m),
        grid(vec_grid(n3, w_.num_sms)) {}

  gs_status dots(int count, const double* const* a, const double* const* b, const double* mult, double* host) {
    DotArgs d;
    std::memset(&d, 0, sizeof(d));
    for (int k = 0; k < count; ++k) {
      d.a[k] = a[k];
      d.b[k] = b[k];
      d.mult[k] = mult ? mult[k] : 1.0;
    }
    d.count = count;
    d.n = n3;
    d.part = w.lb.part;
    d.ticket = w.lb.ticket;
    d.out = w.lb.scal + kDots;
    GS_CUDA(vlaunch(grid, st, k_dots, d));
    if (host) {
      GS_CUDA(cudaMemcpyAsync(host, w.lb.scal + kDots, count * sizeof(double), cudaMemcpyDeviceToHost, st));
      GS_CUDA(cudaStreamSynchronize(st));
    }
    return GS_OK;
  }

  // f and g at p0 = xv (device FP64); g goes to gv.  Synchronises.
  gs_status evaluate(const double* xv, double* gv, double* f) {
    gs_status s = enqueue_gradient64(w, prm, dq, xv, dt, st);
    if (s != GS_OK) return s;
    GS_CUDA(cudaMemcpyAsync(gv, w.gp64, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    GS_CUDA(cudaMemcpyAsync(f, w.scalars + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    ++evals;
    return finish_sync(w, st);
  }

  // phi(a) = f(x + a d) and phi'(a) = g(x + a d).d; the point and its
  // gradient land in xt, gt.
  gs_status eval_step(double a, double* f, double* dphi) {
    GS_CUDA(vlaunch(grid, st, k_step, w.lb.xt, w.lb.x, w.lb.d, n3, a));
    gs_status s = evaluate(w.lb.xt, w.lb.gt, f);
    if (s != GS_OK) return s;
    const double* A[1] = {w.lb.gt};
    const double* B[1] = {w.lb.d};
    return dots(1, A, B, nullptr, dphi);
  }

  static double cubic_min(double a, double fa, double da, double b, double fb, double db) {
    const double d1 = da + db - 3.0 * (fa - fb) / (a - b);
    const double disc = d1 * d1 - da * db;
    if (!(disc >= 0.0)) return NAN;
    const double d2 = (b > a ? 1.0 : -1.0) * std::sqrt(disc);
    const double den = db - da + 2.0 * d2;
    if (den == 0.0) return NAN;
    return b - (b - a) * (db + d2 - d1) / den;
  }

  // Strong-Wolfe line search from f0 with slope dphi0 < 0 and first trial a1.
  // On success *step > 0 and xt, gt, *fnew hold the accepted point.
  gs_status line_search(double f0, double dphi0, double a1, double* step, double* fnew) {
    const double c1 = 1e-4, c2 = 0.9;
    const int max_evals = 20;
    *step = 0.0;
    int used = 0;
    double a_prev = 0.0, f_prev = f0, d_prev = dphi0, a = a1;
    for (int it = 0; used < max_evals; ++it) {
      double fa, da;
      gs_status s = eval_step(a, &fa, &da);
      if (s != GS_OK) return s;
      ++used;
      bool zoom = false;
      double lo = 0, flo = 0, dlo = 0, hi = 0, fhi = 0, dhi = 0;
      if (!(fa <= f0 + c1 * a * dphi0) || (it > 0 && fa >= f_prev)) {
        zoom = true;
        lo = a_prev; flo = f_prev; dlo = d_prev; hi = a; fhi = fa; dhi = da;
      } else if (std::fabs(da) <= -c2 * dphi0) {
        *step = a;
        *fnew = fa;
        return GS_OK;
      } else if (da >= 0.0) {
        zoom = true;
        lo = a; flo = fa; dlo = da; hi = a_prev; fhi = f_prev; dhi = d_prev;
      }
      if (zoom) {
        while (used < max_evals) {
          double aj = cubic_min(lo, flo, dlo, hi, fhi, dhi);
          const double wdt = hi - lo;
          const double b0 = wdt > 0 ? lo + 0.1 * wdt : hi - 0.1 * wdt;
          const double b1 = wdt > 0 ? hi - 0.1 * wdt : lo + 0.1 * wdt;
          if (!(aj >= std::min(b0, b1) && aj <= std::max(b0, b1))) aj = 0.5 * (lo + hi);
          double fj, dj;
          s = eval_step(aj, &fj, &dj);
          if (s != GS_OK) return s;
          ++used;
          if (!(fj <= f0 + c1 * aj * dphi0) || fj >= flo) {
            hi = aj; fhi = fj; dhi = dj;
          } else {
            if (std::fabs(dj) <= -c2 * dphi0) {
              *step = aj;
              *fnew = fj;
              return GS_OK;
            }
            if (dj * (hi - lo) >= 0.0) {
              hi = lo; fhi = flo; dhi = dlo;
            }
            lo = aj; flo = fj; dlo = dj;
          }
        }
        return GS_OK;  // no acceptable step: *step == 0
      }
      a_prev = a; f_prev = fa; d_prev = da;
      a = 2.0 * a;
    }
    return GS_OK;
  }

  // d = -H g by the two-loop recursion over the `stored` newest pairs.
  gs_status direction(int head, int stored, const double* rho, double gamma) {
    LbfgsBufs& b = w.lb;
    GS_CUDA(cudaMemcpyAsync(b.d, b.g, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    for (int k = 0; k < stored; ++k) {
      const int j = (head - 1 - k + m) % m;
      const double* A[1] = {b.S + static_cast<size_t>(j) * n3};
      const double* B[1] = {b.d};
      const double mult[1] = {rho[j]};
      gs_status s = dots(1, A, B, mult, nullptr);
      if (s != GS_OK) return s;
      GS_CUDA(cudaMemcpyAsync(b.scal + kAlpha + j, b.scal + kDots, sizeof(double), cudaMemcpyDeviceToDevice, st));
      GS_CUDA(vlaunch(grid, st, k_axpy, b.d, b.Y + static_cast<size_t>(j) * n3, n3, 0.0, -1.0,
                      (const double*)(b.scal + kAlpha + j), 0.0, (const double*)nullptr));
    }
    if (stored > 0) GS_CUDA(vlaunch(grid, st, k_scale, b.d, (const double*)b.d, n3, gamma));
    for (int k = stored - 1; k >= 0; --k) {
      const int j = (head - 1 - k + m) % m;
      const double* A[1] = {b.Y + static_cast<size_t>(j) * n3};
      const double* B[1] = {b.d};
      const double mult[1] = {rho[j]};
      gs_status s = dots(1, A, B, mult, nullptr);
      if (s != GS_OK) return s;
      GS_CUDA(vlaunch(grid, st, k_axpy, b.d, (const double*)(b.S + static_cast<size_t>(j) * n3), n3, 0.0, 1.0,
                      (const double*)(b.scal + kAlpha + j), -1.0, (const double*)(b.scal + kDots)));
    }
    GS_CUDA(vlaunch(grid, st, k_scale, b.d, (const double*)b.d, n3, -1.0));
    return GS_OK;
  }

  gs_status run(gs_register_info* info) {
    LbfgsBufs& b = w.lb;
    double rho[kMaxM] = {0.0};
    int head = 0, stored = 0, status = 1, it = 0;
    double gamma = 1.0, f = 0.0;
    gs_status s = evaluate(b.x, b.g, &f);
    if (s != GS_OK) return s;
    double gg = 0.0;
    {
      const double* A[1] = {b.g};
      const double* B[1] = {b.g};
      if ((s = dots(1, A, B, nullptr, &gg)) != GS_OK) return s;
    }
    const double g0 = std::sqrt(gg);
    double gnorm = g0;
    if (g0 == 0.0) status = 0;
    for (it = 0; status == 1 && it < prm.max_iter; ++it) {
      if ((s = direction(head, stored, rho, gamma)) != GS_OK) return s;
      double dphi0 = 0.0;
      {
        const double* A[1] = {b.g};
        const double* B[1] = {b.d};
        if ((s = dots(1, A, B, nullptr, &dphi0)) != GS_OK) return s;
      }
      if (!(dphi0 < 0.0)) {  // not a descent direction: restart from -g
        GS_CUDA(vlaunch(grid, st, k_scale, b.d, (const double*)b.g, n3, -1.0));
        dphi0 = -gnorm * gnorm;
        stored = 0;
      }
      const double a1 = (it == 0) ? 1.0 / g0 : 1.0;
      double a = 0.0, fn = 0.0;
      if ((s = line_search(f, dphi0, a1, &a, &fn)) != GS_OK) return s;
      if (a == 0.0) {
        status = 2;  // no step met the Wolfe conditions: noise floor reached
        break;
      }
      double* sv = b.S + static_cast<size_t>(head) * n3;
      double* yv = b.Y + static_cast<size_t>(head) * n3;
      GS_CUDA(vlaunch(grid, st, k_pair, sv, yv, (const double*)b.xt, (const double*)b.x, (const double*)b.gt,
                      (const double*)b.g, n3));
      double r4[4];
      {
        const double* A[4] = {sv, yv, sv, b.gt};
        const double* B[4] = {yv, yv, sv, b.gt};
        if ((s = dots(4, A, B, nullptr, r4)) != GS_OK) return s;
      }
      const double sy = r4[0], yy = r4[1], ss = r4[2];
      if (sy > 1e-12 * std::sqrt(ss * yy)) {
        rho[head] = 1.0 / sy;
        gamma = sy / yy;
        head = (head + 1) % m;
        if (stored < m) ++stored;
      }
      GS_CUDA(cudaMemcpyAsync(b.x, b.xt, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
      GS_CUDA(cudaMemcpyAsync(b.g, b.gt, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
      f = fn;
      gnorm = std::sqrt(r4[3]);
      if (gnorm <= prm.grad_tol * g0) {
        status = 0;
        ++it;
        break;
      }
    }
    if (info) {
      info->loss = f;
      info->grad_norm0 = g0;
      info->grad_norm = gnorm;
      info->iters = it;
      info->evals = evals;
      info->status = status;
    }
    return GS_OK;
  }
};

gs_status run_register(const gs_params* prm, const float* q0, const float* target, float* p0_inout,
                       gs_register_info* info, void* stream) {
  gs_status s = check_params(prm);
  if (s != GS_OK) return s;
  if (!q0 || !target || !p0_inout) return fail(GS_EINVAL, "q0, target and p0_inout must not be NULL");
  if (prm->lbfgs_m < 1 || prm->lbfgs_m > kMaxM) return fail(GS_EINVAL, "lbfgs_m must be in [1, 64]");
  if (prm->max_iter < 0) return fail(GS_EINVAL, "max_iter must be >= 0");
  if (!(prm->grad_tol >= 0.0)) return fail(GS_EINVAL, "grad_tol must be >= 0");
  std::lock_guard<std::mutex> lk(engine_mutex());
  Workspace* w = nullptr;
  if ((s = get_workspace(&w)) != GS_OK) return s;
  const int n = static_cast<int>(prm->N), npad = round_up(n, kPad), n3 = dim_of(*prm) * n;
  const int ckpt = effective_ckpt(prm->ckpt_every, prm->T);
  const int S = stages_of(prm->integrator);
  if ((s = reserve(*w, npad, std::max(S * prm->T, record_slots(prm->T, ckpt, S)), 1,
                   ckpt ? (prm->T + ckpt - 1) / ckpt : 0)) !=
      GS_OK)
    return s;
  if ((s = alloc_lbfgs(*w, n3, prm->lbfgs_m)) != GS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bool host = false;
  const float *dq = nullptr, *dt = nullptr, *dp = nullptr;
  if ((s = stage_in(q0, w->in_q, n3, st, &dq, &host)) != GS_OK) return s;
  if ((s = stage_in(target, w->in_t, n3, st, &dt, &host)) != GS_OK) return s;
  if ((s = stage_in(p0_inout, w->in_p, n3, st, &dp, &host)) != GS_OK) return s;
  const int grid = vec_grid(n3, w->num_sms);
  GS_CUDA(vlaunch(grid, st, k_f32_to_f64, w->lb.x, dp, n3));
  Lbfgs opt(*w, *prm, st, dq, dt);
  if ((s = opt.run(info)) != GS_OK) return s;
  // result: p0 back to float32, and the landmark distances at q(1)
  GS_CUDA(vlaunch(grid, st, k_f64_to_f32, w->out_a, (const double*)w->lb.x, n3));
  bool dummy = false;
  if ((s = copy_out(p0_inout, w->out_a, n3, st, &dummy)) != GS_OK) return s;
  if (info) {
    if ((s = enqueue_forward64(*w, *prm, dq, w->lb.x, st)) != GS_OK) return s;
    GS_CUDA(vlaunch(grid, st, k_dist, (const double*)w->q64, (const double*)w->t64, n, dim_of(*prm), w->lb.part,
                    w->lb.ticket,
                    w->lb.scal + kDots));
    double dist[2] = {0.0, 0.0};
    GS_CUDA(cudaMemcpyAsync(dist, w->lb.scal + kDots, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if ((s = finish_sync(*w, st)) != GS_OK) return s;
    info->avg_dist = dist[0] / n;
    info->max_dist = dist[1];
    return info->status == 0 ? GS_OK : GS_NOT_CONVERGED;
  }
  if ((s = finish_sync(*w, st)) != GS_OK) return s;
  return GS_OK;
}

}  // namespace
}  // namespace gs

extern "C" gs_status register_landmarks(const gs_params* prm, const float* q0, const float* target, float* p0_inout,
                                        gs_register_info* info, void* stream) {
  gs::set_last_error("");
  return gs::run_register(prm, q0, target, p0_inout, info, stream);
}
