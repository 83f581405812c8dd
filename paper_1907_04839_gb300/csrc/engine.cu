// Host engine and C ABI of libgshoot.so.
//
// The engine owns one workspace per CUDA device:
//  * the FP32 trajectory that the pair kernels read;
//  * the FP64 master state;
//  * the split partials;
//  * staging buffers for host arrays;
//  * the reduction scratch and the device status word;
//  * a cache of instantiated CUDA graphs.
// Each graph holds the T forward steps, and for gradients also the T reverse
// steps: a pair-sum kernel followed by a combine kernel per step, linked by
// programmatic dependent launch.  A call packs the inputs, replays the
// graph, then copies the outputs out.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "engine.h"

namespace gs {

namespace {
thread_local std::string g_err;
std::mutex g_mu;
}  // namespace

gs_status fail(gs_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

std::mutex& engine_mutex() { return g_mu; }

std::map<int, Workspace*> g_ws;

template <typename T>
cudaError_t dalloc(Workspace& w, T** p, size_t count) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, count * sizeof(T) + 256);
  if (e != cudaSuccess) return e;
  w.allocs.push_back(v);
  *p = static_cast<T*>(v);
  return cudaSuccess;
}

gs_status get_workspace(Workspace** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(GS_ENOLIB, std::string("no CUDA device: ") + cudaGetErrorString(e));
  auto it = g_ws.find(dev);
  if (it == g_ws.end()) {
    Workspace* w = new Workspace();
    w->device = dev;
    GS_CUDA(cudaDeviceGetAttribute(&w->num_sms, cudaDevAttrMultiProcessorCount, dev));
    GS_CUDA(cudaStreamCreateWithFlags(&w->capture_stream, cudaStreamNonBlocking));
    it = g_ws.emplace(dev, w).first;
  }
  *out = it->second;
  return GS_OK;
}

// Make room for npad landmarks, T steps and the given split counts.
gs_status reserve(Workspace& w, int npad, int T, int splits, int nck) {
  // per-CTA reduction slots: at most Npad/4 fused-step CTAs (tiles of >= 64
  // targets, clusters of <= 16)
  const int red = npad + 64;
  if (npad <= w.cap_npad && T <= w.cap_T && splits <= w.cap_splits && red <= w.cap_red && nck <= w.cap_ck)
    return GS_OK;
  const int cn = std::max(npad, w.cap_npad), cT = std::max(T, w.cap_T);
  const int cs = std::max(splits, w.cap_splits), cr = std::max(red, w.cap_red);
  const int ck = std::max(nck, w.cap_ck);
  w.free_all();
  const size_t n3 = 3 * static_cast<size_t>(cn);
  const size_t slot = static_cast<size_t>(kRecF4) * (cn / 2);
  GS_CUDA(dalloc(w, &w.traj, static_cast<size_t>(cT + 1) * slot));
  GS_CUDA(dalloc(w, &w.adj, 2 * slot));
  GS_CUDA(dalloc(w, &w.q64, n3));
  GS_CUDA(dalloc(w, &w.p64, n3));
  GS_CUDA(dalloc(w, &w.a64, n3));
  GS_CUDA(dalloc(w, &w.b64, n3));
  GS_CUDA(dalloc(w, &w.t64, n3));
  GS_CUDA(dalloc(w, &w.hp0, n3));
  GS_CUDA(dalloc(w, &w.hq0, n3));
  GS_CUDA(dalloc(w, &w.gp64, n3));
  GS_CUDA(dalloc(w, &w.qa64, n3));
  GS_CUDA(dalloc(w, &w.pa64, n3));
  GS_CUDA(dalloc(w, &w.ya64, n3));
  GS_CUDA(dalloc(w, &w.yb64, n3));
  if (ck > 0) GS_CUDA(dalloc(w, &w.ck64, 2 * static_cast<size_t>(ck) * n3));
  GS_CUDA(dalloc(w, &w.part, static_cast<size_t>(cs) * cn));
  GS_CUDA(dalloc(w, &w.in_q, n3));
  GS_CUDA(dalloc(w, &w.in_p, n3));
  GS_CUDA(dalloc(w, &w.in_t, n3));
  GS_CUDA(dalloc(w, &w.in_a, n3));
  GS_CUDA(dalloc(w, &w.out_a, n3));
  GS_CUDA(dalloc(w, &w.out_b, n3));
  GS_CUDA(dalloc(w, &w.red_h, cr));
  GS_CUDA(dalloc(w, &w.red_m, cr));
  GS_CUDA(dalloc(w, &w.scalars, 8));
  GS_CUDA(dalloc(w, &w.ticket, 8));
  GS_CUDA(dalloc(w, &w.status, 8));
  GS_CUDA(cudaMemset(w.ticket, 0, 8 * sizeof(unsigned)));
  GS_CUDA(cudaMemset(w.status, 0, 8 * sizeof(unsigned)));
  GS_CUDA(cudaMemset(w.scalars, 0, 8 * sizeof(double)));
  w.cap_npad = cn;
  w.cap_T = cT;
  w.cap_splits = cs;
  w.cap_red = cr;
  w.cap_ck = ck;
  return GS_OK;
}

// Zero the float4 trajectory and adjoint arrays when the landmark count
// changes: padded entries must be exactly zero (they are never written).
gs_status ensure_clean(Workspace& w, int n, cudaStream_t st, int dim) {
  const int key = 4 * n + dim;
  if (w.clean_n == key) return GS_OK;
  GS_CUDA(cudaMemsetAsync(w.traj, 0, sizeof(float4) * (w.cap_T + 1) * w.slot(), st));
  GS_CUDA(cudaMemsetAsync(w.adj, 0, 2 * sizeof(float4) * w.slot(), st));
  w.clean_n = key;
  return GS_OK;
}

PtrKind classify_pointer(int type, int ptr_device, int current_device) {
  if (type == cudaMemoryTypeManaged) return kPtrDevice;  // migrates to whichever GPU touches it
  if (type != cudaMemoryTypeDevice) return kPtrHost;
  return ptr_device == current_device ? kPtrDevice : kPtrOtherDevice;
}

PtrKind pointer_kind(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return kPtrHost;
  }
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return kPtrOtherDevice;
  }
  return classify_pointer(static_cast<int>(at.type), at.device, cur);
}

bool is_device_ptr(const void* p) { return pointer_kind(p) == kPtrDevice; }

namespace {
gs_status other_device() {
  return fail(GS_EINVAL, "an array lives on another GPU than the current device: make its device current");
}
}  // namespace

// Device view of a caller input array: the pointer itself, or a staged copy.
gs_status stage_in(const float* src, float* staging, size_t n3, cudaStream_t st, const float** dev, bool* host) {
  if (!src) {
    *dev = nullptr;
    return GS_OK;
  }
  const PtrKind kind = pointer_kind(src);
  if (kind == kPtrOtherDevice) return other_device();
  if (kind == kPtrDevice) {
    *dev = src;
    return GS_OK;
  }
  GS_CUDA(cudaMemcpyAsync(staging, src, n3 * sizeof(float), cudaMemcpyHostToDevice, st));
  *dev = staging;
  *host = true;
  return GS_OK;
}

gs_status copy_out(float* dst, const float* src, size_t n3, cudaStream_t st, bool* host) {
  if (!dst) return GS_OK;
  const PtrKind kind = pointer_kind(dst);
  if (kind == kPtrOtherDevice) return other_device();
  const bool dev = kind == kPtrDevice;
  if (!dev) *host = true;
  GS_CUDA(cudaMemcpyAsync(dst, src, n3 * sizeof(float), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  return GS_OK;
}

// Read and clear the device status word (synchronises the stream).
gs_status finish_sync(Workspace& w, cudaStream_t st) {
  unsigned h = 0;
  GS_CUDA(cudaMemcpyAsync(&h, w.status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaStreamSynchronize(st));
  if (h) {
    cudaMemset(w.status, 0, sizeof(unsigned));
    if (h & kErrTimeout) return fail(GS_ETIMEOUT, "a device-side wait expired");
    if (h & kErrNonFinite) return fail(GS_ENONFINITE, "non-finite value in an input or intermediate");
    return fail(GS_ECUDA, "device reported an inconsistent launch");
  }
  return GS_OK;
}

gs_status check_params(const gs_params* prm) {
  if (!prm) return fail(GS_EINVAL, "params is NULL");
  if (prm->N < 1 || prm->N > (1LL << 26)) return fail(GS_EINVAL, "N must be in [1, 2^26]");
  if (prm->T < 1 || prm->T > 100000) return fail(GS_EINVAL, "T must be in [1, 100000]");
  if (!(prm->sigma > 0.0) || !std::isfinite(prm->sigma)) return fail(GS_EINVAL, "sigma must be finite and > 0");
  if (!(prm->lambda >= 0.0) || !std::isfinite(prm->lambda)) return fail(GS_EINVAL, "lambda must be finite and >= 0");
  if (prm->ckpt_every < 0) return fail(GS_EINVAL, "ckpt_every must be >= 0");
  if (prm->integrator != GS_EULER && prm->integrator != GS_RK4)
    return fail(GS_EINVAL, "integrator must be GS_EULER or GS_RK4");
  if (prm->kinetic_at != GS_KINETIC_START && prm->kinetic_at != GS_KINETIC_END)
    return fail(GS_EINVAL, "kinetic_at must be GS_KINETIC_START or GS_KINETIC_END");
  if (prm->dim != 0 && prm->dim != 2 && prm->dim != 3) return fail(GS_EINVAL, "dim must be 2 or 3 (0 means 3)");
  return GS_OK;
}

// Arguments of fused forward step k (kind 1: the last step also forms the
// loss and the adjoint initialisation).  For RK4 (integ), a launch is stage
// `stage` of step k; rd / wr default to the record slots of launch
// S*k + stage and the one after it.  h_end: the loss is formed by a separate
// terminal launch instead of the last step.
StepFwdArgs forward_step_args(Workspace& w, const StepConfig& c, int kind, int n, int T, int k, double sigma,
                              double lambda, int rd = -1, int wr = -1, bool recompute = false, int integ = GS_EULER,
                              int stage = 0, int h_end = 0, int dim = 3) {
  const int S = stages_of(integ);
  const int j = S * k + stage;  // launch index of the sweep
  const int npad = round_up(n, kPad);
  const KernelScales sc = make_scales(sigma);
  const size_t slot = w.slot();
  StepFwdArgs a;
  std::memset(&a, 0, sizeof(a));
  a.qp = w.traj + (rd < 0 ? j : rd) * slot;
  a.qp_next = w.traj + (wr < 0 ? j + 1 : wr) * slot;
  a.n = n;
  a.npad = npad;
  a.split_len = c.split_len;
  a.kappa = static_cast<float>(sc.kappa);
  a.dt = 1.0 / T;
  a.kq = sc.kq;
  a.q64 = w.q64;
  a.p64 = w.p64;
  // A recomputed step (checkpointed reverse sweep) only rebuilds the state.
  a.first = (j == 0) && !recompute;
  a.hp0 = w.hp0;
  a.hq0 = w.hq0;
  a.last = (j == S * T - 1) && !recompute;
  a.with_loss = (kind == 1) && !recompute && !h_end;
  a.rk = integ == GS_RK4;
  a.stage = stage;
  a.qa64 = w.qa64;
  a.pa64 = w.pa64;
  a.adj_scale = integ == GS_RK4 ? (1.0 / T) / 6.0 : 1.0;
  a.dim = dim;
  a.t64 = w.t64;
  a.lambda = lambda;
  a.a64 = w.a64;
  a.b64 = w.b64;
  a.ab = w.adj;  // buffer 0: read by the first reverse step
  a.kappa64 = sc.kappa;
  a.red_h = w.red_h;
  a.red_m = w.red_m;
  a.ticket = w.ticket;
  a.scalars = w.scalars;
  a.status = w.status;
  a.combine64 = combine_f64() ? 1 : 0;
  return a;
}

// Arguments of fused reverse launch number s = 0..S*T-1 (time step
// k = T-1-s/S, stage S-1-s%S; S = 1 for Euler, 4 for RK4).  rd defaults to
// the record slot of that stage state.
StepBwdArgs backward_step_args(Workspace& w, const StepConfig& c, int n, int T, int s, double sigma, int rd = -1,
                               int integ = GS_EULER, int h_end = 0, int dim = 3) {
  const int npad = round_up(n, kPad);
  const KernelScales sc = make_scales(sigma);
  const size_t slot = w.slot();
  const int S = stages_of(integ);
  const int k = T - 1 - s / S, stage = S - 1 - s % S;
  StepBwdArgs b;
  std::memset(&b, 0, sizeof(b));
  b.qp = w.traj + (rd < 0 ? S * k + stage : rd) * slot;
  b.ab = w.adj + (s & 1) * slot;
  b.ab_next = w.adj + ((s + 1) & 1) * slot;
  b.rk = integ == GS_RK4;
  b.stage = stage;
  b.ya64 = w.ya64;
  b.yb64 = w.yb64;
  b.h_at_end = h_end;
  b.dim = dim;
  b.n = n;
  b.npad = npad;
  b.split_len = c.split_len;
  b.kq = static_cast<float>(sc.kq);
  b.kappa = static_cast<float>(sc.kappa);
  b.dt = 1.0 / T;
  b.kappa64 = sc.kappa;
  b.a64 = w.a64;
  b.b64 = w.b64;
  b.first = (k == 0 && stage == 0);
  b.hp0 = w.hp0;
  b.hq0 = w.hq0;
  b.grad_p0 = w.out_a;
  b.grad_q0 = w.out_b;
  b.grad_p0_64 = w.gp64;
  b.status = w.status;
  b.combine64 = combine_f64() ? 1 : 0;
  return b;
}

// Enqueue the T forward steps (and, for kind 1, the loss and T reverse
// steps): one fused cluster kernel per time step, or per stage of an RK4
// step (S = 4 launches per step; record slot S*k + s holds the state of
// stage s of step k, slot S*T the end state).  With the kinetic term at
// t = 1 (h_end), a terminal launch at the end state forms the loss and the
// adjoint initialisation.
//
// With a checkpoint interval c (0 < c < T), the forward sweep keeps only the
// FP64 state at steps 0, c, 2c, ... (records go round two slots).  The
// reverse sweep handles the segments from the last to the first.  For each
// segment it restores the checkpoint, recomputes the segment's stage records
// into slots 0..S*len-1, then runs its reverse launches.  Each recomputed
// record is bitwise the one the forward sweep made, because it comes from
// the same FP64 state through the same kernels.
gs_status enqueue_steps(Workspace& w, int kind, int n, int T, double sigma, double lambda, int ckpt, int integ,
                        int h_end, int dim, cudaStream_t st, const cudaEvent_t* ev) {
  const int npad = round_up(n, kPad);
  if (kind == 0) {
    ckpt = 0;
    h_end = 0;
  }
  // Variant and planar launches run the built-in configuration's kernels.
  const bool variants = integ != GS_EULER || h_end || dim == 2;
  const StepConfig fc = choose_step_config(0, npad, w.num_sms, variants);
  const StepConfig bc = choose_step_config(1, npad, w.num_sms, variants);
  if (fc.threads == 0 || bc.threads == 0) return fail(GS_EINVAL, "no step kernel configuration");
  const int ftrig = late_trigger_for(0, fc, dim, integ == GS_RK4) ? 1 : 0;
  const int btrig = late_trigger_for(1, bc, dim, integ == GS_RK4) ? 1 : 0;
  const int S = stages_of(integ);
  const size_t n3 = static_cast<size_t>(dim) * n;  // FP64 state per checkpoint array
  if (ev) GS_CUDA(cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal));
  for (int k = 0; k < T; ++k) {
    if (ckpt && k % ckpt == 0) {
      double* ck = w.ck64 + 2 * static_cast<size_t>(k / ckpt) * n3;
      GS_CUDA(cudaMemcpyAsync(ck, w.q64, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
      GS_CUDA(cudaMemcpyAsync(ck + n3, w.p64, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    for (int s = 0; s < S; ++s) {
      const int j = S * k + s;
      const int rd = ckpt ? (j & 1) : -1, wr = ckpt ? ((j + 1) & 1) : -1;
      StepFwdArgs a = forward_step_args(w, fc, kind, n, T, k, sigma, lambda, rd, wr, false, integ, s, h_end, dim);
      a.late_trigger = ftrig;
      GS_CUDA(launch_step_forward(fc, a, st, j > 0));
    }
  }
  if (h_end) {
    const int rd = ckpt ? ((S * T) & 1) : S * T;
    StepFwdArgs a = forward_step_args(w, fc, kind, n, T, T - 1, sigma, lambda, rd, rd, true, integ, 0, 1, dim);
    a.terminal = 1;
    a.last = 1;
    a.with_loss = 1;
    a.late_trigger = ftrig;
    GS_CUDA(launch_step_forward(fc, a, st, true));
  }
  if (ev) GS_CUDA(cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal));
  if (kind == 0) {
    if (ev) GS_CUDA(cudaEventRecordWithFlags(ev[2], st, cudaEventRecordExternal));
    return GS_OK;
  }
  if (!ckpt) {
    for (int s = 0; s < S * T; ++s) {
      StepBwdArgs b = backward_step_args(w, bc, n, T, s, sigma, -1, integ, h_end, dim);
      b.late_trigger = s + 1 < S * T ? btrig : 0;
      GS_CUDA(launch_step_backward(bc, b, st, true));
    }
    if (ev) GS_CUDA(cudaEventRecordWithFlags(ev[2], st, cudaEventRecordExternal));
    return GS_OK;
  }
  const KernelScales sc = make_scales(sigma);
  const int nseg = (T + ckpt - 1) / ckpt;
  int s = 0;  // reverse-launch counter (picks the adjoint buffers)
  for (int m = nseg - 1; m >= 0; --m) {
    const int s0 = m * ckpt, len = std::min(ckpt, T - s0);
    const double* ck = w.ck64 + 2 * static_cast<size_t>(m) * n3;
    GS_CUDA(launch_restore(ck, ck + n3, w.q64, w.p64, w.traj, n, sc.kq, st, dim));
    // stage launches 0 .. S*len-2 of the segment write slots 1 .. S*len-1
    for (int r = 0; r + 1 < S * len; ++r) {
      StepFwdArgs a =
          forward_step_args(w, fc, kind, n, T, s0 + r / S, sigma, lambda, r, r + 1, true, integ, r % S, h_end, dim);
      a.late_trigger = ftrig;
      GS_CUDA(launch_step_forward(fc, a, st, r > 0));
    }
    for (int r = S * len - 1; r >= 0; --r, ++s) {
      StepBwdArgs b = backward_step_args(w, bc, n, T, s, sigma, r, integ, h_end, dim);
      b.late_trigger = btrig;
      GS_CUDA(launch_step_backward(bc, b, st, true));
    }
  }
  if (ev) GS_CUDA(cudaEventRecordWithFlags(ev[2], st, cudaEventRecordExternal));
  return GS_OK;
}

gs_status get_graph(Workspace& w, const GraphKey& key, cudaGraphExec_t* out) {
  auto it = w.graphs.find(key);
  if (it != w.graphs.end()) {
    *out = it->second;
    return GS_OK;
  }
  if (w.graphs.size() >= 16) w.drop_graphs();
  cudaStream_t cs = w.capture_stream;
  GS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  gs_status s = enqueue_steps(w, key.kind, key.n, key.T, key.sigma, key.lambda, key.ckpt, key.integ, key.h_end,
                              key.dim, cs, key.timed ? w.phase : nullptr);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  if (s != GS_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return fail(GS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  cudaGraphExec_t ge = nullptr;
  e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(GS_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  w.graphs[key] = ge;
  *out = ge;
  return GS_OK;
}

gs_status enqueue_gradient64(Workspace& w, const gs_params& prm, const float* dq, const double* p64_in,
                             const float* dt, cudaStream_t st) {
  const int n = static_cast<int>(prm.N), dim = dim_of(prm);
  gs_status s = ensure_clean(w, n, st, dim);
  if (s != GS_OK) return s;
  PackArgs pk;
  pk.q = dq;
  pk.p = nullptr;
  pk.p64_in = p64_in;
  pk.tgt = dt;
  pk.q64 = w.q64;
  pk.p64 = w.p64;
  pk.t64 = w.t64;
  pk.qp = w.traj;
  pk.n = n;
  pk.kq = make_scales(prm.sigma).kq;
  pk.status = w.status;
  pk.dim = dim;
  GS_CUDA(launch_pack(pk, st));
  cudaGraphExec_t ge = nullptr;
  const GraphKey key{1,           n, prm.T, prm.sigma, prm.lambda, effective_ckpt(prm.ckpt_every, prm.T), w.phase_timing,
                     prm.integrator, prm.kinetic_at, dim};
  if ((s = get_graph(w, key, &ge)) != GS_OK) return s;
  GS_CUDA(cudaGraphLaunch(ge, st));
  return GS_OK;
}

gs_status enqueue_forward64(Workspace& w, const gs_params& prm, const float* dq, const double* p64_in,
                            cudaStream_t st) {
  const int n = static_cast<int>(prm.N), dim = dim_of(prm);
  gs_status s = ensure_clean(w, n, st, dim);
  if (s != GS_OK) return s;
  PackArgs pk;
  pk.q = dq;
  pk.p = nullptr;
  pk.p64_in = p64_in;
  pk.tgt = nullptr;
  pk.q64 = w.q64;
  pk.p64 = w.p64;
  pk.t64 = nullptr;
  pk.qp = w.traj;
  pk.n = n;
  pk.kq = make_scales(prm.sigma).kq;
  pk.status = w.status;
  pk.dim = dim;
  GS_CUDA(launch_pack(pk, st));
  cudaGraphExec_t ge = nullptr;
  if ((s = get_graph(w, GraphKey{0, n, prm.T, prm.sigma, 0.0, 0, w.phase_timing, prm.integrator, 0, dim}, &ge)) !=
      GS_OK)
    return s;
  GS_CUDA(cudaGraphLaunch(ge, st));
  return GS_OK;
}

// Common driver of shoot_forward / shoot_gradient.
gs_status run_shoot(int kind, const gs_params* prm, const float* q0, const float* p0, const float* target,
                    float* q1, float* p1, double* H0, double* loss, float* gp, float* gq, void* stream) {
  gs_status s = check_params(prm);
  if (s != GS_OK) return s;
  if (!q0 || !p0 || (kind == 1 && !target)) return fail(GS_EINVAL, "q0, p0 (and target) must not be NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  Workspace* w = nullptr;
  if ((s = get_workspace(&w)) != GS_OK) return s;
  const int n = static_cast<int>(prm->N), T = prm->T;
  const int npad = round_up(n, kPad);
  const int ckpt = kind == 1 ? effective_ckpt(prm->ckpt_every, T) : 0;
  if ((s = reserve(*w, npad, record_slots(T, ckpt, stages_of(prm->integrator)), 1, ckpt ? (T + ckpt - 1) / ckpt : 0)) !=
      GS_OK)
    return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int dim = dim_of(*prm);
  if ((s = ensure_clean(*w, n, st, dim)) != GS_OK) return s;
  const size_t n3 = static_cast<size_t>(dim) * n;  // floats per (N, dim) array
  bool host = false;
  const float *dq = nullptr, *dp = nullptr, *dt = nullptr;
  if ((s = stage_in(q0, w->in_q, n3, st, &dq, &host)) != GS_OK) return s;
  if ((s = stage_in(p0, w->in_p, n3, st, &dp, &host)) != GS_OK) return s;
  if (kind == 1 && (s = stage_in(target, w->in_t, n3, st, &dt, &host)) != GS_OK) return s;
  PackArgs pk;
  pk.q = dq;
  pk.p = dp;
  pk.p64_in = nullptr;
  pk.tgt = dt;
  pk.q64 = w->q64;
  pk.p64 = w->p64;
  pk.t64 = kind == 1 ? w->t64 : nullptr;
  pk.qp = w->traj;
  pk.n = n;
  pk.kq = make_scales(prm->sigma).kq;
  pk.status = w->status;
  pk.dim = dim;
  GS_CUDA(launch_pack(pk, st));
  cudaGraphExec_t ge = nullptr;
  const GraphKey key{kind,           n, T, prm->sigma, kind == 1 ? prm->lambda : 0.0, ckpt, w->phase_timing,
                     prm->integrator, kind == 1 ? prm->kinetic_at : 0, dim};
  if ((s = get_graph(*w, key, &ge)) != GS_OK) return s;
  GS_CUDA(cudaGraphLaunch(ge, st));
  bool want_sync = host;
  if (kind == 0) {
    if (q1) {
      UnpackArgs u{w->q64, w->out_a, static_cast<int>(n3)};
      GS_CUDA(launch_unpack(u, st));
      if ((s = copy_out(q1, w->out_a, n3, st, &want_sync)) != GS_OK) return s;
    }
    if (p1) {
      UnpackArgs u{w->p64, w->out_b, static_cast<int>(n3)};
      GS_CUDA(launch_unpack(u, st));
      if ((s = copy_out(p1, w->out_b, n3, st, &want_sync)) != GS_OK) return s;
    }
    if (H0) {
      GS_CUDA(cudaMemcpyAsync(H0, w->scalars, sizeof(double), cudaMemcpyDeviceToHost, st));
      want_sync = true;
    }
  } else {
    if ((s = copy_out(gp, w->out_a, n3, st, &want_sync)) != GS_OK) return s;
    if ((s = copy_out(gq, w->out_b, n3, st, &want_sync)) != GS_OK) return s;
    if (loss) {
      GS_CUDA(cudaMemcpyAsync(loss, w->scalars + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
      want_sync = true;
    }
  }
  if (want_sync) return finish_sync(*w, st);
  return GS_OK;
}

gs_status run_step(int kind, int64_t N, double sigma, const float* q, const float* p, const float* alpha,
                   const float* beta, float* out0, float* out1, void* stream) {
  if (N < 1 || N > (1LL << 26)) return fail(GS_EINVAL, "N must be in [1, 2^26]");
  if (!(sigma > 0.0) || !std::isfinite(sigma)) return fail(GS_EINVAL, "sigma must be finite and > 0");
  if (!q || !p || !out0 || !out1 || (kind == 1 && (!alpha || !beta)))
    return fail(GS_EINVAL, "array arguments must not be NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  Workspace* w = nullptr;
  gs_status s = get_workspace(&w);
  if (s != GS_OK) return s;
  const int n = static_cast<int>(N), npad = round_up(n, kPad);
  const PairConfig c = kind == 0 ? choose_forward_config(npad, w->num_sms) : choose_backward_config(npad, w->num_sms);
  if ((s = reserve(*w, npad, 1, c.splits)) != GS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t n3 = 3 * static_cast<size_t>(n);
  bool host = false;
  const float *dq, *dp, *da = nullptr, *db = nullptr;
  if ((s = stage_in(q, w->in_q, n3, st, &dq, &host)) != GS_OK) return s;
  if ((s = stage_in(p, w->in_p, n3, st, &dp, &host)) != GS_OK) return s;
  if (kind == 1) {
    if ((s = stage_in(alpha, w->in_a, n3, st, &da, &host)) != GS_OK) return s;
    if ((s = stage_in(beta, w->in_t, n3, st, &db, &host)) != GS_OK) return s;
  }
  const KernelScales sc = make_scales(sigma);
  GS_CUDA(launch_to_records(dq, dp, w->traj, n, npad, sc.kq, 1.0, 0, w->status, st));
  if (kind == 0) {
    PairFwdArgs a;
    a.qp = w->traj;
    a.part = w->part;
    a.npad = npad;
    a.split_len = c.split_len;
    a.kappa = static_cast<float>(sc.kappa);
    a.status = w->status;
    GS_CUDA(launch_pair_forward(c, a, st, false));
  } else {
    GS_CUDA(launch_to_records(da, db, w->adj, n, npad, 1.0, sc.kappa, 1, w->status, st));
    PairBwdArgs a;
    a.qp = w->traj;
    a.ab = w->adj;
    a.part = w->part;
    a.npad = npad;
    a.split_len = c.split_len;
    a.kq = static_cast<float>(sc.kq);
    a.kappa = static_cast<float>(sc.kappa);
    a.status = w->status;
    GS_CUDA(launch_pair_backward(c, a, st, false));
  }
  // Partials hold (Hp, Hq) forward and (dalpha, dbeta) backward.
  GS_CUDA(launch_partials_to_out(w->part, c.splits, n, npad, w->out_a, w->out_b, st));
  w->clean_n = -1;  // traj slot 0 / adjoint arrays were overwritten
  bool want_sync = host;
  if (kind == 0) {
    if ((s = copy_out(out1, w->out_a, n3, st, &want_sync)) != GS_OK) return s;  // Hp
    if ((s = copy_out(out0, w->out_b, n3, st, &want_sync)) != GS_OK) return s;  // Hq
  } else {
    if ((s = copy_out(out0, w->out_a, n3, st, &want_sync)) != GS_OK) return s;  // dalpha
    if ((s = copy_out(out1, w->out_b, n3, st, &want_sync)) != GS_OK) return s;  // dbeta
  }
  if (want_sync) return finish_sync(*w, st);
  return GS_OK;
}

gs_status time_pair_kernels(const gs_params* prm, const float* q0, const float* p0, const float* target,
                            int reps, double* fwd_ms, double* bwd_ms, int* launches, void* stream) {
  if (reps < 1 || reps > 100000) return fail(GS_EINVAL, "reps must be in [1, 100000]");
  if (prm && dim_of(*prm) != 3) return fail(GS_EINVAL, "gs_time_pair_kernels times the 3-D kernels (dim 3)");
  double loss = 0.0;
  gs_status s = run_shoot(1, prm, q0, p0, target, nullptr, nullptr, nullptr, &loss, nullptr, nullptr, stream);
  if (s != GS_OK) return s;
  std::lock_guard<std::mutex> lk(g_mu);
  Workspace* w = nullptr;
  if ((s = get_workspace(&w)) != GS_OK) return s;
  const int n = static_cast<int>(prm->N), T = prm->T, npad = round_up(n, kPad);
  const StepConfig fc = choose_step_config(0, npad, w->num_sms);
  const StepConfig bc = choose_step_config(1, npad, w->num_sms);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // A middle time step on the state in record slot 0; dry runs change no state.
  StepFwdArgs fa = forward_step_args(*w, fc, 1, n, T, T / 2, prm->sigma, prm->lambda, 0, 1, true);
  fa.dry = 1;
  StepBwdArgs ba = backward_step_args(*w, bc, n, T, T - 1 - T / 2, prm->sigma, 0);
  ba.dry = 1;
  cudaEvent_t e0, e1, e2;
  GS_CUDA(cudaEventCreate(&e0));
  GS_CUDA(cudaEventCreate(&e1));
  GS_CUDA(cudaEventCreate(&e2));
  GS_CUDA(launch_step_forward(fc, fa, st, false));  // warm-up
  GS_CUDA(launch_step_backward(bc, ba, st, false));
  GS_CUDA(cudaEventRecord(e0, st));
  for (int r = 0; r < reps; ++r) GS_CUDA(launch_step_forward(fc, fa, st, false));
  GS_CUDA(cudaEventRecord(e1, st));
  for (int r = 0; r < reps; ++r) GS_CUDA(launch_step_backward(bc, ba, st, false));
  GS_CUDA(cudaEventRecord(e2, st));
  GS_CUDA(cudaEventSynchronize(e2));
  float m1 = 0.f, m2 = 0.f;
  GS_CUDA(cudaEventElapsedTime(&m1, e0, e1));
  GS_CUDA(cudaEventElapsedTime(&m2, e1, e2));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  if (fwd_ms) *fwd_ms = m1 / reps;
  if (bwd_ms) *bwd_ms = m2 / reps;
  // pack, S launches per forward step, the terminal launch, S per reverse step
  if (launches) *launches = 2 * stages_of(prm->integrator) * T + 1 + (prm->kinetic_at == GS_KINETIC_END ? 1 : 0);
  return finish_sync(*w, st);
}

gs_status time_pair_config(int kind_in, int64_t N, double sigma, const float* q, const float* p,
                           const float* alpha, const float* beta, int threads, int R, int groups, int splits, int reps,
                           double* ms, int* used, void* stream) {
  const bool graph = (kind_in & 16) != 0;
  const int kind = kind_in & ~16;
  if (kind < 0 || kind > 3) return fail(GS_EINVAL, "kind must be 0..3 (+16 for graph replay)");
  if (N < 1 || N > (1LL << 26)) return fail(GS_EINVAL, "N must be in [1, 2^26]");
  if (!(sigma > 0.0) || !std::isfinite(sigma)) return fail(GS_EINVAL, "sigma must be finite and > 0");
  if (reps < 1 || reps > 100000) return fail(GS_EINVAL, "reps must be in [1, 100000]");
  const bool bwd = (kind == 1 || kind == 3);
  if (!q || !p || (bwd && (!alpha || !beta))) return fail(GS_EINVAL, "array arguments must not be NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  Workspace* w = nullptr;
  gs_status s = get_workspace(&w);
  if (s != GS_OK) return s;
  const int n = static_cast<int>(N), npad = round_up(n, kPad);
  PairConfig c{};
  StepConfig sc{};
  if (kind < 2) {
    if (groups != 1) return fail(GS_EINVAL, "the split-partial kernels have one warp group");
    c = kind == 0 ? forward_config_for(npad, w->num_sms, threads, R, splits)
                  : backward_config_for(npad, w->num_sms, threads, R, splits);
    if (c.threads == 0) return fail(GS_EINVAL, "no such kernel variant");
  } else {
    sc = step_config_for(kind - 2, npad, threads, R, splits, groups);
    if (sc.threads == 0) return fail(GS_EINVAL, "no such step kernel variant / cluster size");
    sc.policy = policy_for_grid(static_cast<long long>(sc.tiles) * sc.cluster, w->num_sms);
  }
  if ((s = reserve(*w, npad, 1, kind < 2 ? c.splits : 1)) != GS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t n3 = 3 * static_cast<size_t>(n);
  bool host = false;
  const float *dq, *dp, *da = nullptr, *db = nullptr;
  if ((s = stage_in(q, w->in_q, n3, st, &dq, &host)) != GS_OK) return s;
  if ((s = stage_in(p, w->in_p, n3, st, &dp, &host)) != GS_OK) return s;
  if (bwd) {
    if ((s = stage_in(alpha, w->in_a, n3, st, &da, &host)) != GS_OK) return s;
    if ((s = stage_in(beta, w->in_t, n3, st, &db, &host)) != GS_OK) return s;
  }
  const KernelScales ks = make_scales(sigma);
  GS_CUDA(launch_to_records(dq, dp, w->traj, n, npad, ks.kq, 1.0, 0, w->status, st));
  if (bwd) GS_CUDA(launch_to_records(da, db, w->adj, n, npad, 1.0, ks.kappa, 1, w->status, st));
  w->clean_n = -1;
  PairFwdArgs fa;
  fa.qp = w->traj;
  fa.part = w->part;
  fa.npad = npad;
  fa.split_len = c.split_len;
  fa.kappa = static_cast<float>(ks.kappa);
  fa.status = w->status;
  PairBwdArgs ba;
  ba.qp = w->traj;
  ba.ab = w->adj;
  ba.part = w->part;
  ba.npad = npad;
  ba.split_len = c.split_len;
  ba.kq = static_cast<float>(ks.kq);
  ba.kappa = static_cast<float>(ks.kappa);
  ba.status = w->status;
  StepFwdArgs sfa = forward_step_args(*w, sc, 1, n, 1, 0, sigma, 1.0);
  sfa.dry = 1;
  StepBwdArgs sba = backward_step_args(*w, sc, n, 1, 0, sigma);
  sba.dry = 1;
  auto once = [&](cudaStream_t s, bool pdl) {
    switch (kind) {
      case 0: return launch_pair_forward(c, fa, s, pdl);
      case 1: return launch_pair_backward(c, ba, s, pdl);
      case 2: return launch_step_forward(sc, sfa, s, pdl);
      default: return launch_step_backward(sc, sba, s, pdl);
    }
  };
  GS_CUDA(once(st, false));  // warm-up
  cudaGraphExec_t ge = nullptr;
  if (graph) {  // the reps launches as one graph, linked by programmatic dependent launch
    cudaStream_t cs = w->capture_stream;
    GS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = once(cs, r > 0);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return fail(GS_ECUDA, std::string("capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(GS_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    GS_CUDA(cudaGraphLaunch(ge, st));  // warm-up replay
  }
  cudaEvent_t e0, e1;
  GS_CUDA(cudaEventCreate(&e0));
  GS_CUDA(cudaEventCreate(&e1));
  GS_CUDA(cudaEventRecord(e0, st));
  if (graph) {
    GS_CUDA(cudaGraphLaunch(ge, st));
  } else {
    for (int r = 0; r < reps; ++r) GS_CUDA(once(st, false));
  }
  GS_CUDA(cudaEventRecord(e1, st));
  GS_CUDA(cudaEventSynchronize(e1));
  float t = 0.f;
  GS_CUDA(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ge) cudaGraphExecDestroy(ge);
  if (ms) *ms = t / reps;
  if (used) *used = kind < 2 ? c.splits : sc.cluster;
  return finish_sync(*w, st);
}

void set_last_error(const char* msg) { g_err = msg ? msg : ""; }

}  // namespace gs

extern "C" {

gs_status step_forward(int64_t N, double sigma, const float* q, const float* p, float* Hq, float* Hp, void* stream) {
  gs::g_err.clear();
  return gs::run_step(0, N, sigma, q, p, nullptr, nullptr, Hq, Hp, stream);
}

gs_status step_backward(int64_t N, double sigma, const float* q, const float* p, const float* alpha,
                        const float* beta, float* dalpha, float* dbeta, void* stream) {
  gs::g_err.clear();
  return gs::run_step(1, N, sigma, q, p, alpha, beta, dalpha, dbeta, stream);
}

gs_status shoot_forward(const gs_params* prm, const float* q0, const float* p0, float* q1, float* p1, double* H0,
                        void* stream) {
  gs::g_err.clear();
  return gs::run_shoot(0, prm, q0, p0, nullptr, q1, p1, H0, nullptr, nullptr, nullptr, stream);
}

gs_status shoot_gradient(const gs_params* prm, const float* q0, const float* p0, const float* target, double* loss,
                         float* grad_p0, float* grad_q0, void* stream) {
  gs::g_err.clear();
  return gs::run_shoot(1, prm, q0, p0, target, nullptr, nullptr, nullptr, loss, grad_p0, grad_q0, stream);
}

gs_status gs_time_pair_kernels(const gs_params* prm, const float* q0, const float* p0, const float* target,
                               int32_t reps, double* fwd_ms, double* bwd_ms, int32_t* launches_per_eval,
                               void* stream) {
  gs::g_err.clear();
  int l = 0;
  gs_status s = gs::time_pair_kernels(prm, q0, p0, target, reps, fwd_ms, bwd_ms, &l, stream);
  if (launches_per_eval) *launches_per_eval = l;
  return s;
}

gs_status gs_time_pair_config(int32_t kind, int64_t N, double sigma, const float* q, const float* p,
                              const float* alpha, const float* beta, int32_t threads, int32_t R, int32_t groups,
                              int32_t splits, int32_t reps, double* ms, int32_t* splits_used, void* stream) {
  gs::g_err.clear();
  int used = 0;
  gs_status s =
      gs::time_pair_config(kind, N, sigma, q, p, alpha, beta, threads, R, groups, splits, reps, ms, &used, stream);
  if (splits_used) *splits_used = used;
  return s;
}

gs_status gs_set_step_config(int32_t kind, int32_t threads, int32_t R, int32_t groups, int32_t cluster) {
  gs::g_err.clear();
  if (kind != 0 && kind != 1) {
    gs::set_last_error("kind must be 0 (forward) or 1 (reverse)");
    return GS_EINVAL;
  }
  std::lock_guard<std::mutex> lk(gs::g_mu);
  if (!gs::set_step_override(kind, threads, R, groups, cluster)) {
    gs::set_last_error("no such step kernel variant / cluster size");
    return GS_EINVAL;
  }
  for (auto& kv : gs::g_ws) kv.second->drop_graphs();
  return GS_OK;
}

gs_status gs_set_cluster_policy(int32_t policy) {
  gs::g_err.clear();
  if (policy < -1 || policy > 2) return gs::fail(GS_EINVAL, "policy must be -1, 0, 1 or 2");
  std::lock_guard<std::mutex> lk(gs::g_mu);
  gs::set_cluster_policy(policy);
  for (auto& kv : gs::g_ws) kv.second->drop_graphs();
  return GS_OK;
}

gs_status gs_set_late_trigger(int32_t mode) {
  gs::g_err.clear();
  if (mode < -1 || mode > 1) return gs::fail(GS_EINVAL, "mode must be -1, 0 or 1");
  std::lock_guard<std::mutex> lk(gs::g_mu);
  gs::set_late_trigger(mode);
  for (auto& kv : gs::g_ws) kv.second->drop_graphs();
  return GS_OK;
}

gs_status gs_set_batch_config(int32_t kind, int32_t threads, int32_t cluster) {
  gs::g_err.clear();
  std::lock_guard<std::mutex> lk(gs::g_mu);
  if (!gs::set_batch_shape(kind, threads, cluster))
    return gs::fail(GS_EINVAL, "no packed kernel with that CTA size and cluster size");
  return GS_OK;
}

gs_status gs_set_combine_precision(int32_t f64) {
  gs::g_err.clear();
  if (f64 != 0 && f64 != 1) return gs::fail(GS_EINVAL, "f64 must be 0 (double-single) or 1 (FP64)");
  std::lock_guard<std::mutex> lk(gs::g_mu);
  gs::set_combine_f64(f64 == 1);
  for (auto& kv : gs::g_ws) kv.second->drop_graphs();
  return GS_OK;
}

gs_status gs_set_step_table(int32_t on) {
  gs::g_err.clear();
  if (on != 0 && on != 1) return gs::fail(GS_EINVAL, "on must be 0 or 1");
  std::lock_guard<std::mutex> lk(gs::g_mu);
  gs::set_step_table(on == 1);
  for (auto& kv : gs::g_ws) kv.second->drop_graphs();
  return GS_OK;
}

gs_status gs_step_config(int32_t kind, int64_t N, int32_t num_sms, int32_t variants, int32_t* threads,
                         int32_t* cluster) {
  gs::g_err.clear();
  if (kind != 0 && kind != 1) return gs::fail(GS_EINVAL, "kind must be 0 (forward) or 1 (reverse)");
  if (N < 1 || N > (1LL << 26)) return gs::fail(GS_EINVAL, "N must be in [1, 2^26]");
  if (!threads || !cluster) return gs::fail(GS_EINVAL, "output pointers must not be NULL");
  int sms = num_sms;
  if (sms <= 0) {
    int dev = 0;
    GS_CUDA(cudaGetDevice(&dev));
    GS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  std::lock_guard<std::mutex> lk(gs::g_mu);
  const gs::StepConfig c = gs::choose_step_config(kind, gs::round_up(N, gs::kPad), sms, variants != 0);
  if (c.threads == 0) return gs::fail(GS_EINVAL, "no step kernel configuration");
  *threads = c.threads;
  *cluster = c.cluster;
  return GS_OK;
}

gs_status gs_max_active_clusters(int32_t kind, int32_t threads, int32_t R, int32_t groups, int32_t cluster,
                                 int32_t* clusters) {
  gs::g_err.clear();
  if (!clusters || (kind != 0 && kind != 1) || cluster < 1 || cluster > 16)
    return gs::fail(GS_EINVAL, "bad kind, cluster size or NULL output");
  std::lock_guard<std::mutex> lk(gs::g_mu);
  int n = 0;
  const cudaError_t e = gs::max_active_clusters(kind, threads, R, groups, cluster, &n);
  if (e != cudaSuccess) return gs::fail(GS_EINVAL, std::string("occupancy query: ") + cudaGetErrorString(e));
  *clusters = n;
  return GS_OK;
}

gs_status gs_set_phase_timing(int32_t on) {
  gs::g_err.clear();
  std::lock_guard<std::mutex> lk(gs::g_mu);
  gs::Workspace* w = nullptr;
  gs_status s = gs::get_workspace(&w);
  if (s != GS_OK) return s;
  if (on && !w->phase[0]) {
    for (int k = 0; k < 3; ++k) {
      cudaError_t e = cudaEventCreate(&w->phase[k]);
      if (e != cudaSuccess) return gs::fail(GS_ECUDA, std::string("phase events: ") + cudaGetErrorString(e));
    }
  }
  w->phase_timing = on != 0;
  return GS_OK;
}

gs_status gs_phase_times(double* fwd_ms, double* bwd_ms) {
  gs::g_err.clear();
  if (!fwd_ms || !bwd_ms) return gs::fail(GS_EINVAL, "fwd_ms and bwd_ms must not be NULL");
  std::lock_guard<std::mutex> lk(gs::g_mu);
  gs::Workspace* w = nullptr;
  gs_status s = gs::get_workspace(&w);
  if (s != GS_OK) return s;
  if (!w->phase[0]) return gs::fail(GS_EINVAL, "phase timing was never switched on");
  float a = 0.f, b = 0.f;
  cudaError_t e = cudaEventElapsedTime(&a, w->phase[0], w->phase[1]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&b, w->phase[1], w->phase[2]);
  if (e != cudaSuccess) return gs::fail(GS_ECUDA, std::string("phase times: ") + cudaGetErrorString(e));
  *fwd_ms = a;
  *bwd_ms = b;
  return GS_OK;
}

const char* gs_last_error(void) { return gs::g_err.c_str(); }

void gs_release_workspace(void) {
  std::lock_guard<std::mutex> lk(gs::g_mu);
  for (auto& kv : gs::g_ws) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(kv.first);
    kv.second->free_all();
    for (cudaEvent_t& e : kv.second->phase)
      if (e) cudaEventDestroy(e);
    if (kv.second->capture_stream) cudaStreamDestroy(kv.second->capture_stream);
    delete kv.second;
    cudaSetDevice(cur);
  }
  gs::g_ws.clear();
}

int32_t gs_pointer_rule(int32_t type, int32_t ptr_device, int32_t current_device) {
  return static_cast<int32_t>(gs::classify_pointer(type, ptr_device, current_device));
}

int32_t gs_version(void) { return 107; }

}  // extern "C"
