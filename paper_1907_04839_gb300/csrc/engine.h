// Host engine internals shared by engine.cu and lbfgs.cu: the per-device
// workspace, the CUDA-call error macro and the helpers that stage arrays,
// cache graphs and read the device status word.
#pragma once

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "gs_internal.h"
#include "../../include/gshoot.h"

namespace gs {

// Record the calling thread's error message and return `st`.
gs_status fail(gs_status st, const std::string& msg);

#define GS_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return ::gs::fail(e_ == cudaErrorMemoryAllocation ? GS_ENOMEM : GS_ECUDA,            \
                        std::string(#call) + ": " + cudaGetErrorString(e_));               \
  } while (0)

inline int round_up(long long x, int m) { return static_cast<int>((x + m - 1) / m * m); }

struct GraphKey {
  int kind;  // 0 forward only, 1 gradient
  int n, T;
  double sigma, lambda;
  int ckpt;       // checkpoint interval of the reverse sweep (0: whole trajectory)
  int timed = 0;  // records the workspace's phase events
  int integ = 0;  // GS_EULER or GS_RK4
  int h_end = 0;  // the loss takes the kinetic term at t = 1
  int dim = 3;    // 3-D or planar landmarks
  bool operator<(const GraphKey& o) const {
    return std::tie(kind, n, T, sigma, lambda, ckpt, timed, integ, h_end, dim) <
           std::tie(o.kind, o.n, o.T, o.sigma, o.lambda, o.ckpt, o.timed, o.integ, o.h_end, o.dim);
  }
};

// Dimension of the landmarks of a call (gs_params.dim: 2, or 3 / 0 for 3-D).
inline int dim_of(const gs_params& p) { return p.dim == 2 ? 2 : 3; }

// Pair-sum evaluations (stages) per time step of an integrator.
inline int stages_of(int integ) { return integ == GS_RK4 ? 4 : 1; }
// Effective checkpoint interval for T steps: 0 keeps the whole trajectory.
inline int effective_ckpt(int ckpt_every, int T) { return (ckpt_every > 0 && ckpt_every < T) ? ckpt_every : 0; }
// Trajectory record slots needed (slots 0..return value): one record per
// stage state and the end state; with checkpointing, the stage states of one
// segment.
inline int record_slots(int T, int ckpt, int stages = 1) {
  return ckpt ? (stages * ckpt > 2 ? stages * ckpt : 2) : stages * T;
}

// FP64 vectors of the device-resident L-BFGS (register_landmarks).
struct LbfgsBufs {
  int n3 = 0, m = 0;
  std::vector<void*> allocs;
  double *x = nullptr, *g = nullptr, *d = nullptr, *xt = nullptr, *gt = nullptr;
  double *S = nullptr, *Y = nullptr;  // m x n3 each
  double* scal = nullptr;             // alpha[m], beta, dots...
  double* part = nullptr;             // per-CTA partial sums of a dot product
  unsigned* ticket = nullptr;
  void free_all() {
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    n3 = m = 0;
  }
};

struct Workspace {
  int device = -1;
  int num_sms = 0;
  // capacities
  int cap_npad = 0, cap_T = 0, cap_splits = 0;
  int cap_red = 0, cap_ck = 0;
  std::vector<void*> allocs;
  float4* traj = nullptr;  // (cap_T + 1) slots of QP pair records
  float4* adj = nullptr;   // 2 slots of AB pair records: reverse steps alternate
  size_t slot() const { return static_cast<size_t>(kRecF4) * (cap_npad / 2); }  // float4 per slot
  double *q64 = nullptr, *p64 = nullptr, *a64 = nullptr, *b64 = nullptr, *t64 = nullptr;
  double *hp0 = nullptr, *hq0 = nullptr;
  double *qa64 = nullptr, *pa64 = nullptr;  // RK4 stage accumulators (forward)
  double *ya64 = nullptr, *yb64 = nullptr;  // RK4 start-state adjoint (reverse)
  double* gp64 = nullptr;  // FP64 dL/dp0 of the last gradient
  double* ck64 = nullptr;  // cap_ck checkpoints of the FP64 state: (q64, p64) pairs
  Partial* part = nullptr;   // cap_splits * cap_npad
  float *in_q = nullptr, *in_p = nullptr, *in_t = nullptr, *in_a = nullptr;
  float *out_a = nullptr, *out_b = nullptr;
  double *red_h = nullptr, *red_m = nullptr, *scalars = nullptr;
  unsigned *ticket = nullptr, *status = nullptr;
  // The trajectory and adjoint records hold zero padding for this N and
  // dimension (key 4 N + dim; -1: unknown).
  int clean_n = -1;
  cudaStream_t capture_stream = nullptr;
  std::map<GraphKey, cudaGraphExec_t> graphs;
  // Phase timing: when on, every graph records phase[0] before its first
  // time step, phase[1] between the forward and the reverse sweep and
  // phase[2] after its last step.
  bool phase_timing = false;
  cudaEvent_t phase[3] = {nullptr, nullptr, nullptr};
  LbfgsBufs lb;
  // Query points of velocity_field / flow_points (grown on demand).
  int cap_pts = 0;
  std::vector<void*> pt_allocs;
  double* pts64 = nullptr;
  float *pts_in = nullptr, *pts_out = nullptr;

  void drop_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
  }
  void free_all() {
    drop_graphs();
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    lb.free_all();
    for (void* p : pt_allocs) cudaFree(p);
    pt_allocs.clear();
    cap_pts = 0;
    cap_npad = cap_T = cap_splits = cap_red = cap_ck = 0;
    clean_n = -1;
  }
};

// The process-wide lock that serialises calls into the library.
std::mutex& engine_mutex();
gs_status get_workspace(Workspace** out);
// Room for npad landmarks, record slots 0..T, the split partials and nck
// FP64 state checkpoints.
gs_status reserve(Workspace& w, int npad, int T, int splits, int nck = 0);
gs_status ensure_clean(Workspace& w, int n, cudaStream_t st, int dim = 3);
// True for memory the current device can use in place: its own device
// memory or managed memory.
bool is_device_ptr(const void* p);
gs_status stage_in(const float* src, float* staging, size_t n3, cudaStream_t st, const float** dev, bool* host);
gs_status copy_out(float* dst, const float* src, size_t n3, cudaStream_t st, bool* host);
gs_status finish_sync(Workspace& w, cudaStream_t st);
gs_status check_params(const gs_params* prm);
gs_status get_graph(Workspace& w, const GraphKey& key, cudaGraphExec_t* out);
// Enqueue one gradient evaluation at FP64 momenta p64_in (device, N*3) with
// q0 and target already on the device: pack, then replay the gradient graph.
// Afterwards w.gp64 holds dL/dp0 and w.scalars[1] the loss (stream order).
gs_status enqueue_gradient64(Workspace& w, const gs_params& prm, const float* dq, const double* p64_in,
                             const float* dt, cudaStream_t st);
// Enqueue the forward flow only at FP64 momenta; w.q64 then holds q(1).
gs_status enqueue_forward64(Workspace& w, const gs_params& prm, const float* dq, const double* p64_in,
                            cudaStream_t st);

}  // namespace gs
