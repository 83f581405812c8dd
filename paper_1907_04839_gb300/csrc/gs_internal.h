// Internal interfaces between the gshoot kernels and the host engine.
//
// Device data layout (one workspace per device; Npad = N rounded up to a
// multiple of kPad, padded landmarks stay exactly zero):
//   traj_q[k]  float4[Npad]  kq * q^k (xyz, w = 0), the prescaled positions
//   traj_p[k]  float4[Npad]  p^k (xyz, w = 0)
//   adj_a      float4[Npad]  alpha (adjoint of q) of the current reverse step
//   adj_b      float4[Npad]  kappa * beta (adjoint of p, prescaled)
//   q64, p64, a64, b64       double[N*3], FP64 master state, (N,3) row-major
//   part       Partial[S][Npad], per source split: six double-single sums
// with kq = sqrt(log2(e) / 2) / sigma (so g = 2^-(|kq d|^2)),
// s = 1/sigma^2 and kappa = s / kq.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gs {

// Bits of the device status word (workspace `status[0]`).
enum : unsigned {
  kErrTimeout = 1u,    // an mbarrier wait ran past its iteration limit
  kErrNonFinite = 2u,  // an input or intermediate value was NaN or Inf
  kErrBadLaunch = 4u,  // a kernel saw an inconsistent launch configuration
};

constexpr int kPad = 64;      // landmark padding granule = source sub-block
constexpr int kChunk = 256;   // sources staged in shared memory per bulk copy

// Six double-single sums for one target and one source split:
// forward  c[0..2] = Hp, c[3..5] = Hq
// backward c[0..2] = dalpha, c[3..5] = dbeta
struct __align__(16) Partial {
  float2 c[6];
};

struct KernelScales {
  double kq;     // position prescale, sqrt(log2 e / 2) / sigma
  double s;      // 1 / sigma^2
  double kappa;  // s / kq
};

KernelScales make_scales(double sigma);

struct PairFwdArgs {
  const float4* q4;   // traj_q slot, Npad
  const float4* p4;   // traj_p slot, Npad
  Partial* part;      // [S][Npad]
  int npad;
  int split_len;      // sources per split (multiple of kPad)
  float kappa;        // Hq = -kappa * sum c g (kq d)
  unsigned* status;
};

struct PairBwdArgs {
  const float4* q4;
  const float4* p4;
  const float4* a4;   // alpha
  const float4* b4;   // kappa * beta
  Partial* part;
  int npad;
  int split_len;
  float kq;           // dalpha = kq * A1 - kappa * A2
  float kappa;
  unsigned* status;
};

// Tile configuration chosen by the host for one problem size.
struct PairConfig {
  int threads;    // CTA size
  int R;          // targets per thread
  int tiles;      // target tiles = ceil(Npad / (threads * R))
  int splits;     // source splits S
  int split_len;  // sources per split
};

PairConfig choose_forward_config(int npad, int num_sms);
PairConfig choose_backward_config(int npad, int num_sms);
// Forward configuration with at most `max_splits` source splits.
PairConfig choose_forward_config_capped(int npad, int num_sms, int max_splits);

// Record the calling thread's error message (returned by gs_last_error).
void set_last_error(const char* msg);

cudaError_t launch_pair_forward(const PairConfig& cfg, const PairFwdArgs& a, cudaStream_t st, bool pdl);
cudaError_t launch_pair_backward(const PairConfig& cfg, const PairBwdArgs& a, cudaStream_t st, bool pdl);

// ---------------------------------------------------------------- combine kernels
struct PackArgs {
  const float* q;      // (N,3) float32 inputs (device)
  const float* p;      // may be null (zeros)
  const float* tgt;    // may be null
  double* q64;
  double* p64;
  double* t64;         // may be null
  float4* q4;          // traj_q[0]
  float4* p4;          // traj_p[0]
  int n;
  double kq;
  unsigned* status;
};

struct CombineFwdArgs {
  const Partial* part;
  int splits;
  int n, npad;
  double dt;
  double kq;
  double* q64;
  double* p64;
  float4* q4_next;     // traj_q[k+1]
  float4* p4_next;     // traj_p[k+1]
  // step 0: keep Hp(q0,p0), Hq(q0,p0) and reduce H0 = 1/2 sum p0 . Hp
  int first;
  double* hp0;
  double* hq0;
  // last step: loss = H0 + lambda |q - t|^2, alpha = 2 lambda (q - t), beta = 0
  int last;
  int with_loss;
  const double* t64;
  double lambda;
  double kappa;
  double* a64;
  double* b64;
  float4* a4;
  float4* b4;
  // deterministic grid reduction: per-CTA partials + ticket; scalars[0] = H0,
  // scalars[1] = loss
  double* red_h;
  double* red_m;
  unsigned* ticket;
  double* scalars;
  unsigned* status;
};

struct CombineBwdArgs {
  const Partial* part;
  int splits;
  int n, npad;
  double dt;
  double kappa;
  double* a64;
  double* b64;
  float4* a4;
  float4* b4;
  // step 0: gradient assembly
  int first;
  const double* hp0;
  const double* hq0;
  float* grad_p0;      // (N,3) float32, may be null
  float* grad_q0;
  unsigned* status;
};

struct UnpackArgs {
  const double* x64;
  float* out;
  int n3;
};

cudaError_t launch_pack(const PackArgs& a, cudaStream_t st);
cudaError_t launch_combine_forward(const CombineFwdArgs& a, cudaStream_t st, bool pdl, int* grid_out);
cudaError_t launch_combine_backward(const CombineBwdArgs& a, cudaStream_t st, bool pdl);
cudaError_t launch_unpack(const UnpackArgs& a, cudaStream_t st);
// Hq, Hp straight from one split-partial set (step_forward entry point).
cudaError_t launch_partials_to_out(const Partial* part, int splits, int n, int npad,
                                   float* out_a, float* out_b, cudaStream_t st);
// (N,3) float32 -> prescaled float4 (scale * x), zero-padded to npad.
cudaError_t launch_to_float4(const float* x, float4* x4, int n, int npad, double scale,
                             unsigned* status, cudaStream_t st);

int combine_threads();

}  // namespace gs
