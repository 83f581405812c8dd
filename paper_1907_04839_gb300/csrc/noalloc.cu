// step_forward_noalloc: StepForward for callers that cannot allocate device
// memory.
//
// The ordinary entry points draw their scratch from a workspace that the
// library grows with cudaMalloc on first use.  Two kinds of caller cannot
// take that:
//  * a host program whose device memory is already owned by another
//    allocator under a fixed budget, such as a framework's caching pool;
//  * code for which an allocation call is unacceptable, because cudaMalloc
//    can synchronise the whole device.
// This entry point instead runs the same StepForward kernels on scratch held
// in one file-scope __device__ array, sized below.  The array is created when
// the CUDA module that holds it is loaded, and every GPU that loads this
// library keeps it until the process exits.  Nothing here calls cudaMalloc,
// cudaFree, or any other routine that allocates.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "gs_internal.h"
#include "../../include/gshoot.h"

namespace gs {
namespace {

// Limits of the static scratch: at most kMaxN landmarks, and at most
// kMaxSplits source splits per call.
constexpr int kMaxN = 8192;
constexpr int kMaxSplits = 8;
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffQP = 0;
constexpr size_t kOffPart = align256(kOffQP + sizeof(float4) * kRecF4 * (kMaxN / 2));
constexpr size_t kOffStatus = align256(kOffPart + sizeof(Partial) * kMaxSplits * kMaxN);
constexpr size_t kScratchBytes = align256(kOffStatus + 4 * sizeof(unsigned));  // about 3.3 MB

// The scratch for every call on a device.  It holds the pair records of q
// and p, the split partials, and the device status word.  The pointer that
// host code passes to kernels comes from cudaGetSymbolAddress, because the
// array's name in host code does not give a device address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

// One-time set-up per device: look up the device address of the scratch
// array while that device is current.
gs_status scratch_for_current_device(unsigned char** out, int* num_sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_last_error("no CUDA device");
    return GS_ENOLIB;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_last_error("device ordinal beyond the no-allocation entry point's table");
    return GS_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_last_error(e != cudaSuccess ? cudaGetErrorString(e) : "scratch symbol has no device address");
      return GS_ECUDA;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
      set_last_error(cudaGetErrorString(e));
      return GS_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    g_num_sms[dev] = sms;
  }
  *out = g_scratch_ptr[dev];
  *num_sms = g_num_sms[dev];
  return GS_OK;
}

// Device memory of the current GPU, or managed memory (another GPU's
// memory and host memory are refused).
bool on_device(const void* p) { return pointer_kind(p) == kPtrDevice; }

gs_status cuda_fail(cudaError_t e) {
  set_last_error(cudaGetErrorString(e));
  return GS_ECUDA;
}

}  // namespace
}  // namespace gs

extern "C" gs_status step_forward_noalloc(int64_t N, double sigma, const float* q, const float* p,
                                          float* Hq, float* Hp, void* stream) {
  using namespace gs;
  set_last_error("");
  if (N < 1 || N > kMaxN) {
    set_last_error("step_forward_noalloc: N must be in [1, 8192], the size of its static scratch");
    return GS_EINVAL;
  }
  if (!(sigma > 0.0) || !std::isfinite(sigma)) {
    set_last_error("step_forward_noalloc: sigma must be finite and > 0");
    return GS_EINVAL;
  }
  if (!q || !p || !Hq || !Hp || !on_device(q) || !on_device(p) || !on_device(Hq) || !on_device(Hp)) {
    set_last_error("step_forward_noalloc: q, p, Hq and Hp must be device arrays of the current GPU");
    return GS_EINVAL;
  }
  unsigned char* base = nullptr;
  int num_sms = 0;
  gs_status s = scratch_for_current_device(&base, &num_sms);
  if (s != GS_OK) return s;
  float4* qp = reinterpret_cast<float4*>(base + kOffQP);
  Partial* part = reinterpret_cast<Partial*>(base + kOffPart);
  unsigned* status = reinterpret_cast<unsigned*>(base + kOffStatus);

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = static_cast<int>(N);
  const int npad = (n + kPad - 1) / kPad * kPad;
  const PairConfig cfg = choose_forward_config_capped(npad, num_sms, kMaxSplits);
  if (cfg.splits > kMaxSplits) {
    set_last_error("step_forward_noalloc: split count exceeds the static scratch");
    return GS_EINVAL;
  }
  const KernelScales sc = make_scales(sigma);
  // The status word keeps the previous call's value: clear it.  The pair
  // records (padding included) and the partials are fully rewritten below.
  cudaError_t e = cudaMemsetAsync(status, 0, 4 * sizeof(unsigned), st);
  if (e != cudaSuccess) return cuda_fail(e);
  if ((e = launch_to_records(q, p, qp, n, npad, sc.kq, 1.0, 0, status, st)) != cudaSuccess) return cuda_fail(e);
  PairFwdArgs a;
  a.qp = qp;
  a.part = part;
  a.npad = npad;
  a.split_len = cfg.split_len;
  a.kappa = static_cast<float>(sc.kappa);
  a.status = status;
  if ((e = launch_pair_forward(cfg, a, st, false)) != cudaSuccess) return cuda_fail(e);
  // Partials hold (Hp, Hq).
  if ((e = launch_partials_to_out(part, cfg.splits, n, npad, Hp, Hq, st)) != cudaSuccess) return cuda_fail(e);
  unsigned h = 0;
  if ((e = cudaMemcpyAsync(&h, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e);
  if (h & kErrTimeout) {
    set_last_error("step_forward_noalloc: a device-side wait expired");
    return GS_ETIMEOUT;
  }
  if (h & kErrNonFinite) {
    set_last_error("step_forward_noalloc: non-finite input");
    return GS_ENONFINITE;
  }
  return GS_OK;
}
