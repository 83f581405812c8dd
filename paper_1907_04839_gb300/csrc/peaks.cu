// Measured throughput of the arithmetic units the pair kernels run on.
//
// The roofline of the pair-sum kernels is the FP32 pipe (they issue paired
// f32x2 FMA/ADD/MUL instructions), with the MUFU unit (one ex2 per pair)
// second; the FP64 unit serves the state updates.  Nominal unit counts times
// the clock give a derived peak, and this file measures the same rates on
// the device the library runs on, so that a fraction of peak rests on a
// measurement:
//   * FFMA:  scalar FP32 fused multiply-add, 2 flops each;
//   * FFMA2: the paired form (one instruction, two lanes), 2 flops per lane;
//   * EX2:   MUFU ex2.approx.ftz.f32, results per second;
//   * DFMA:  FP64 fused multiply-add, 2 flops each;
//   * FFMA2 with three distinct register operands per instruction (a
//     separate entry point): the paired rate when no operand is shared
//     between consecutive instructions.
// Each kernel runs CH independent dependency chains per thread on every SM
// (4 CTAs of 256 threads per SM: 8 warps per scheduler), long enough (about
// 50 ms) that launch overhead does not count, and is timed with CUDA events
// on the caller's stream.  The best of three timed launches is reported.
#include <cmath>

#include <algorithm>
#include <map>
#include <utility>
#include <vector>

#include "engine.h"
#include "gs_device.cuh"
#include "pair_tile.cuh"

namespace gs {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakCtasPerSm = 4;
constexpr int kChains = 8;
constexpr int kInner = 16;  // chain steps per loop iteration

// x <- x*a + b converges to b/(1-a) and never leaves the normal range, so
// every operation is a full-rate one.  The final test is never true for
// these constants, but the compiler cannot know it, so no chain is dead.
__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma(int iters, float a, float b, float* sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * threadIdx.x + c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kInner; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0f) sink[0] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma2(int iters, float a, float b, float* sink) {
  float2 x[kChains];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = make_float2(1e-3f * threadIdx.x + c, 2e-3f * threadIdx.x - c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kInner; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  if (s == -1.0f) sink[0] = s;
}

// The paired form with three distinct register operands per instruction:
// each chain has its own multiplier and addend, so no operand is shared
// between consecutive instructions (the pair loops' pattern, where most
// operands are per-record values).
__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma2_distinct(int iters, float a, float b, float* sink) {
  float2 x[kChains], y[kChains], z[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    x[c] = make_float2(1e-3f * threadIdx.x + c, 2e-3f * threadIdx.x - c);
    y[c] = make_float2(a - 1e-6f * c, a - 2e-6f * c - 1e-7f * threadIdx.x);
    z[c] = make_float2(b + 1e-6f * c, b + 3e-6f * c + 1e-7f * threadIdx.x);
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kInner; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], y[c], z[c]);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  if (s == -1.0f) sink[0] = s;
}

// y <- 2^-y stays in [0.5, 1] for y in [0, 1].
__global__ void __launch_bounds__(kPeakThreads) k_peak_ex2(int iters, float* sink) {
  float y[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) y[c] = 0.1f * c + 1e-4f * threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kInner; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) y[c] = ex2_approx(-y[c]);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += y[c];
  if (s == -1.0f) sink[0] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_dfma(int iters, double a, double b, float* sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * threadIdx.x + c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kInner; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = __fma_rn(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0) sink[0] = static_cast<float>(s);
}

// One launch of unit `which` with `iters` loop iterations; returns its
// device time in ms.
gs_status time_unit(int which, int iters, int blocks, float* sink, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                    float* ms) {
  GS_CUDA(cudaEventRecord(e0, st));
  switch (which) {
    case 0: k_peak_ffma<<<blocks, kPeakThreads, 0, st>>>(iters, 0.9999f, 1e-4f, sink); break;
    case 1: k_peak_ffma2<<<blocks, kPeakThreads, 0, st>>>(iters, 0.9999f, 1e-4f, sink); break;
    case 2: k_peak_ex2<<<blocks, kPeakThreads, 0, st>>>(iters, sink); break;
    case 3: k_peak_dfma<<<blocks, kPeakThreads, 0, st>>>(iters, 0.9999, 1e-4, sink); break;
    default: k_peak_ffma2_distinct<<<blocks, kPeakThreads, 0, st>>>(iters, 0.9999f, 1e-4f, sink); break;
  }
  GS_CUDA(cudaGetLastError());
  GS_CUDA(cudaEventRecord(e1, st));
  GS_CUDA(cudaEventSynchronize(e1));
  GS_CUDA(cudaEventElapsedTime(ms, e0, e1));
  return GS_OK;
}

// The inner loop of the pair tiles alone: one target per thread against
// kLoopRecords source records (two sources each) held in shared memory,
// `reps` times, with no copies, cluster barriers or epilogue.  The source
// count arrives as a kernel argument (nsrc = 2 * kLoopRecords), so the loop
// is compiled with run-time bounds, as in the step kernels.  Thread 0 of
// each CTA records its SM and the SM clock at the start and the end of the
// CTA's loop; the host takes, per SM, the span from the first start to the
// last end, which is what the SM needs for all of its CTAs' work (warps on
// one scheduler need not finish together).
constexpr int kLoopRecords = 64;

template <bool Bwd>
__global__ void k_loop_probe(const float4* qp, const float4* ab, int nsrc, int reps, long long* cycles, float* sink) {
  __shared__ __align__(16) float4 rq[kLoopRecords * 3], ra[kLoopRecords * 3];
  for (int i = threadIdx.x; i < kLoopRecords * 3; i += blockDim.x) {
    rq[i] = qp[i];
    ra[i] = ab[i];
  }
  __syncthreads();
  const int target = static_cast<int>(threadIdx.x) % kLoopRecords;  // 2 * kLoopRecords sources
  float s = 0.f;
  const long long t0 = clock64();
  if constexpr (Bwd) {
    BwdTile<1, 3> t;
    t.load(qp, ab, target, kLoopRecords, 2 * kLoopRecords);
    const float4* bufs[2] = {rq, ra};
    for (int r = 0; r < reps; ++r) t.consume(bufs, 0, nsrc);
    __syncthreads();
    ds w[6];
    t.result(0, 1.0f, 0.5f, w);
    for (int k = 0; k < 6; ++k) s += w[k].hi;
  } else {
    FwdTile<1, 3> t;
    t.load(qp, target, kLoopRecords, 2 * kLoopRecords);
    const float4* bufs[1] = {rq};
    for (int r = 0; r < reps; ++r) t.consume(bufs, 0, nsrc);
    __syncthreads();
    ds w[6];
    t.result(0, 1.0f, w);
    for (int k = 0; k < 6; ++k) s += w[k].hi;
  }
  const long long t1 = clock64();
  if (s == -1.0f) sink[0] = s;  // keeps the sums live; sink is a scratch word nobody reads
  if (threadIdx.x == 0) {
    unsigned sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    cycles[3 * blockIdx.x] = sm;
    cycles[3 * blockIdx.x + 1] = t0;
    cycles[3 * blockIdx.x + 2] = t1;
  }
}

// Calibrate the iteration count of unit `which` to about target_ms, then
// keep the best of three launches: TFLOP/s (ex2 results per second for
// unit 2) in *rate, the kernel time in *ms_best.
gs_status measure_unit(int which, int blocks, float* sink, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                       double target_ms, double* rate, double* ms_best) {
  int iters = which == 3 ? 64 : 2048;
  float ms = 0.f;
  gs_status s = GS_OK;
  for (int probe = 0; probe < 4 && s == GS_OK; ++probe) {
    s = time_unit(which, iters, blocks, sink, st, e0, e1, &ms);
    if (s != GS_OK || ms >= 0.5 * target_ms) break;
    const double scale = ms > 0.01 ? target_ms / ms : 64.0;
    iters = static_cast<int>(std::fmin(1e9, std::ceil(iters * std::fmin(scale, 64.0))));
  }
  float best = 1e30f;
  for (int r = 0; r < 3 && s == GS_OK; ++r) {
    s = time_unit(which, iters, blocks, sink, st, e0, e1, &ms);
    best = std::fmin(best, ms);
  }
  if (s != GS_OK) return s;
  const bool paired = which == 1 || which == 4;
  const double ops = static_cast<double>(blocks) * kPeakThreads * iters * kInner * kChains * (paired ? 2 : 1);
  const double per_s = ops / (best * 1e-3);
  *rate = which == 2 ? per_s : 2.0 * per_s * 1e-12;
  if (ms_best) *ms_best = best;
  return GS_OK;
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_measure_peaks(double* rates, double* ms_out, double target_ms, void* stream) {
  using namespace gs;
  set_last_error("");
  if (!rates) return fail(GS_EINVAL, "rates is NULL");
  if (!(target_ms >= 1.0 && target_ms <= 2000.0)) return fail(GS_EINVAL, "target_ms must be in [1, 2000]");
  std::lock_guard<std::mutex> lk(engine_mutex());
  Workspace* w = nullptr;
  gs_status s = get_workspace(&w);
  if (s != GS_OK) return s;
  if ((s = reserve(*w, kPad, 1, 1)) != GS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int blocks = w->num_sms * kPeakCtasPerSm;
  // The sink is a workspace word no kernel reads; the kernels never write it.
  float* sink = reinterpret_cast<float*>(w->status + 5);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  GS_CUDA(cudaEventCreate(&e0));
  GS_CUDA(cudaEventCreate(&e1));
  for (int which = 0; which < 4 && s == GS_OK; ++which)
    s = measure_unit(which, blocks, sink, st, e0, e1, target_ms, &rates[which], ms_out ? &ms_out[which] : nullptr);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}

extern "C" gs_status gs_measure_ffma2_distinct(double* tflops, double target_ms, void* stream) {
  using namespace gs;
  set_last_error("");
  if (!tflops) return fail(GS_EINVAL, "tflops is NULL");
  if (!(target_ms >= 1.0 && target_ms <= 2000.0)) return fail(GS_EINVAL, "target_ms must be in [1, 2000]");
  std::lock_guard<std::mutex> lk(engine_mutex());
  Workspace* w = nullptr;
  gs_status s = get_workspace(&w);
  if (s != GS_OK) return s;
  if ((s = reserve(*w, kPad, 1, 1)) != GS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* sink = reinterpret_cast<float*>(w->status + 5);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  GS_CUDA(cudaEventCreate(&e0));
  GS_CUDA(cudaEventCreate(&e1));
  s = measure_unit(4, w->num_sms * kPeakCtasPerSm, sink, st, e0, e1, target_ms, tflops, nullptr);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}

extern "C" gs_status gs_measure_pair_loop(int32_t kind, int32_t threads, int32_t ctas_per_sm, int32_t reps,
                                          double* cycles_per_record, void* stream) {
  using namespace gs;
  set_last_error("");
  if (!cycles_per_record) return fail(GS_EINVAL, "cycles_per_record is NULL");
  if (kind != 0 && kind != 1) return fail(GS_EINVAL, "kind must be 0 (StepForward) or 1 (StepBackward)");
  if (threads < 32 || threads > 256 || threads % 32 != 0) return fail(GS_EINVAL, "threads must be 32, 64, ..., 256");
  if (ctas_per_sm < 1 || ctas_per_sm > 16 || threads * ctas_per_sm > 1024)
    return fail(GS_EINVAL, "ctas_per_sm must be in [1, 16] with threads * ctas_per_sm <= 1024");
  if (reps < 1 || reps > 4096) return fail(GS_EINVAL, "reps must be in [1, 4096]");
  const auto kern = kind == 1 ? k_loop_probe<true> : k_loop_probe<false>;
  int dev = 0, sms = 0, fit = 0;
  GS_CUDA(cudaGetDevice(&dev));
  GS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  GS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kern, threads, 0));
  if (fit < ctas_per_sm) return fail(GS_EINVAL, "that many CTAs of the probe are not resident on an SM at once");
  const int blocks = sms * ctas_per_sm;
  // Source records of a smooth synthetic cloud: q~ in [-0.9, 0.9], p, alpha
  // and b~ in [-0.1, 0.1] (every exponent stays in the normal range).
  std::vector<float4> hq(kLoopRecords * 3), ha(kLoopRecords * 3);
  for (int i = 0; i < kLoopRecords * 3; ++i) {
    const float x = static_cast<float>(i);
    hq[i] = make_float4(0.9f * std::sin(1.7f * x), 0.9f * std::sin(2.3f * x + 1.f), 0.1f * std::cos(0.7f * x),
                        0.1f * std::cos(1.1f * x + 2.f));
    ha[i] = make_float4(0.1f * std::sin(0.3f * x), 0.1f * std::cos(0.9f * x), 0.1f * std::sin(1.3f * x + 0.5f),
                        0.1f * std::cos(0.5f * x + 1.5f));
  }
  float4 *dq = nullptr, *da = nullptr;
  long long* dc = nullptr;
  float* sink = nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMalloc(&dq, sizeof(float4) * hq.size());
  if (e == cudaSuccess) e = cudaMalloc(&da, sizeof(float4) * ha.size());
  if (e == cudaSuccess) e = cudaMalloc(&dc, 3 * sizeof(long long) * blocks);
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpyAsync(dq, hq.data(), sizeof(float4) * hq.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(da, ha.data(), sizeof(float4) * ha.size(), cudaMemcpyHostToDevice, st);
  std::vector<long long> hc(3 * static_cast<size_t>(blocks));
  for (int run = 0; run < 2 && e == cudaSuccess; ++run) {  // the first launch warms up
    kern<<<blocks, threads, 0, st>>>(dq, da, 2 * kLoopRecords, reps, dc, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), dc, 3 * sizeof(long long) * blocks, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dq);
  cudaFree(da);
  cudaFree(dc);
  cudaFree(sink);
  if (e != cudaSuccess) return fail(GS_ECUDA, cudaGetErrorString(e));
  // Per SM: first start to last end of its CTAs' loops (one SM clock).
  std::map<long long, std::pair<long long, long long>> span;
  for (int b = 0; b < blocks; ++b) {
    const long long sm = hc[3 * b], t0 = hc[3 * b + 1], t1 = hc[3 * b + 2];
    auto it = span.find(sm);
    if (it == span.end())
      span.emplace(sm, std::make_pair(t0, t1));
    else
      it->second = std::make_pair(std::min(it->second.first, t0), std::max(it->second.second, t1));
  }
  std::vector<long long> per_sm;
  for (const auto& kv : span) per_sm.push_back(kv.second.second - kv.second.first);
  std::sort(per_sm.begin(), per_sm.end());
  *cycles_per_record = static_cast<double>(per_sm[per_sm.size() / 2]) / (static_cast<double>(reps) * kLoopRecords);
  return GS_OK;
}
