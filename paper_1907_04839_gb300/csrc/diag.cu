// Failure-detection check: a device wait that nothing completes must end
// at its iteration limit with the timeout bit in the status word, and leave
// the context usable.  The kernel waits, in one thread, on either
//   0: an mbarrier phase that no thread or copy completes (the wait of the
//      bulk-copy stage ring), or
//   1: a flag in global memory that nothing sets (a bounded poll loop),
// with the library's own limits (kSpinLimit polls of the mbarrier, about one
// second; one second of global time for the flag), and records the expiry.  No
// fault, trap or endless loop is involved.
#include <chrono>

#include "engine.h"
#include "gs_device.cuh"

namespace gs {
namespace {

__global__ void k_wait_timeout(int which, const unsigned* flag, unsigned* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  bool ok = false;
  if (which == 0) {
    mbar_init(&bar, 1);  // one arrival completes phase 0; none comes
    fence_mbar_init();
    ok = mbar_wait(&bar, 0);
  } else {
    // one second of global time
    const unsigned long long t0 = global_ns();
    for (long it = 0; !ok; ++it) {
      ok = *reinterpret_cast<const volatile unsigned*>(flag) != 0u;
      if ((it & 255) == 255 && global_ns() - t0 > kWaitNs) break;
    }
  }
  if (!ok) atomicOr(status, kErrTimeout);
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_check_wait_timeout(int32_t which, double* seconds, void* stream) {
  using namespace gs;
  set_last_error("");
  if (which != 0 && which != 1) return fail(GS_EINVAL, "which must be 0 (mbarrier) or 1 (global flag)");
  std::lock_guard<std::mutex> lk(engine_mutex());
  Workspace* w = nullptr;
  gs_status s = get_workspace(&w);
  if (s != GS_OK) return s;
  if ((s = reserve(*w, kPad, 1, 1)) != GS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // status[4] is a word nothing in the library writes: zero since allocation.
  const auto t0 = std::chrono::steady_clock::now();
  k_wait_timeout<<<1, 32, 0, st>>>(which, w->status + 4, w->status);
  GS_CUDA(cudaGetLastError());
  s = finish_sync(*w, st);
  if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return s;
}
