// Internal interfaces between the gshoot kernels and the host engine.
//
// Device data layout (one workspace per device; Npad = N rounded up to a
// multiple of kPad; padded landmarks stay exactly zero):
//   traj[k]   QP pair records, Npad/2 x 3 float4: landmarks 2g and 2g+1
//             interleaved per coordinate, positions prescaled and negated:
//               {-q~x0, -q~x1, -q~y0, -q~y1} {-q~z0, -q~z1, px0, px1}
//               {py0, py1, pz0, pz1}
//   adj[2]    AB pair records, same shape, two buffers (a reverse step reads
//             one and writes the other):
//               {ax0, ax1, ay0, ay1} {az0, az1, -b~x0, -b~x1}
//               {-b~y0, -b~y1, -b~z0, -b~z1}
//   q64, p64, a64, b64   double[N*3], FP64 master state, (N,3) row-major
//   part      Partial[S][Npad], per source split: six double-single sums
// with q~ = kq q, b~ = kappa beta, kq = sqrt(log2(e) / 2) / sigma (so the
// Gaussian is 2^-|q~_i - q~_j|^2), s = 1/sigma^2 and kappa = s / kq.
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

constexpr int kPad = 64;      // landmark padding granule
constexpr int kChunk = 128;   // sources staged in shared memory per bulk copy
constexpr int kStages = 4;    // chunk buffers in flight per CTA
constexpr int kRecF4 = 3;     // float4 per pair record (two landmarks)
constexpr int kRecBytes = 48;

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
  const float4* qp;   // QP records of the state
  Partial* part;      // [S][Npad]
  int npad;
  int split_len;      // sources per split (multiple of kPad)
  float kappa;        // Hq = -kappa * sum c g (kq d)
  unsigned* status;
};

struct PairBwdArgs {
  const float4* qp;   // QP records of the state
  const float4* ab;   // AB records of the adjoint
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
// A given kernel variant (threads per CTA, targets per thread); splits <= 0
// picks the balanced split count.  threads == 0 in the result: no such variant.
PairConfig forward_config_for(int npad, int num_sms, int threads, int R, int splits);
PairConfig backward_config_for(int npad, int num_sms, int threads, int R, int splits);
PairConfig choose_backward_config(int npad, int num_sms);
// Forward configuration with at most `max_splits` source splits.
PairConfig choose_forward_config_capped(int npad, int num_sms, int max_splits);

// Record the calling thread's error message (returned by gs_last_error).
void set_last_error(const char* msg);

// Where a caller's array lives, as the current device sees it.  Host memory
// (pageable or pinned) is staged through a device buffer; device memory of
// the current GPU and managed memory are used in place; device memory of
// another GPU is rejected, because a kernel of this device reading it
// faults unless peer access happens to be enabled.
enum PtrKind { kPtrHost = 0, kPtrDevice = 1, kPtrOtherDevice = 2 };
// The rule itself, from cudaPointerAttributes::type and ::device and the
// current device's ordinal (no CUDA call).
PtrKind classify_pointer(int type, int ptr_device, int current_device);
PtrKind pointer_kind(const void* p);

cudaError_t launch_pair_forward(const PairConfig& cfg, const PairFwdArgs& a, cudaStream_t st, bool pdl);
cudaError_t launch_pair_backward(const PairConfig& cfg, const PairBwdArgs& a, cudaStream_t st, bool pdl);

// ---------------------------------------------------------------- fused step kernels
// One kernel per time step: a thread-block cluster of C CTAs owns a tile of
// targets; CTA rank r sums sources [r*split_len, (r+1)*split_len).  The C
// partial sums meet in distributed shared memory, and each CTA finishes the
// Euler (or adjoint) update for 1/C of the tile.
struct StepConfig {
  int threads;    // CTA size
  int R;          // targets per thread
  int cluster;    // C, CTAs per cluster = source splits
  int tiles;      // clusters = ceil(Npad / (threads / groups * R))
  int split_len;  // sources per CTA (multiple of 8)
  int policy;     // cluster scheduling: 0 driver default, 1 spread, 2 load balancing
  int groups;     // warp groups per CTA that split the CTA's sources (1: none)
};

struct StepFwdArgs {
  const float4* qp;    // traj[k]
  float4* qp_next;     // traj[k+1]
  int n, npad, split_len;
  float kappa;
  double dt, kq;
  double* q64;
  double* p64;
  int first;           // keep Hp, Hq of step 0 and reduce H0
  double* hp0;
  double* hq0;
  int last;            // last step of a gradient: loss terms and adjoint init
  int with_loss;
  const double* t64;
  double lambda;
  double* a64;
  double* b64;
  float4* ab;          // adjoint buffer the first reverse step reads
  double kappa64;
  double* red_h;       // per-CTA partial sums (grid-sized)
  double* red_m;
  unsigned* ticket;
  double* scalars;     // [0] = H0, [1] = loss, [2] = H at the end state (terminal launch)
  int dry;             // tuning: compute everything, write nothing
  unsigned* status;
  // Variants (all zero: an Euler step, the kinetic term at t = 0).
  int rk;              // 1: stage `stage` (0..3) of an RK4 step
  int stage;
  double* qa64;        // RK4: FP64 accumulators k1 + 2 k2 + 2 k3 (q and p parts)
  double* pa64;
  int terminal;        // evaluate at the end state: H(p(1), q(1)), the loss and
                       // the adjoint initialisation; no state update
  double adj_scale;    // factor of the adjoint record written at the loss
                       // (terminal launch, or the last RK4 stage): dt/6 for RK4, 1 for Euler
  int dim;             // 2: planar landmarks (records of 2 float4, (N,2) FP64
                       // arrays); 0 or 3: 3-D
  int late_trigger;    // trigger the next launch after the pair sums (pdl_trigger)
  int combine64;       // add the split partials in FP64 (0: double-single)
};

struct StepBwdArgs {
  const float4* qp;    // traj[k]
  const float4* ab;    // adjoint of step k+1
  float4* ab_next;     // adjoint of step k (the other buffer)
  int n, npad, split_len;
  float kq, kappa;
  double dt, kappa64;
  double* a64;
  double* b64;
  int first;           // k == 0: write the gradient
  const double* hp0;
  const double* hq0;
  float* grad_p0;
  float* grad_q0;
  double* grad_p0_64;  // FP64 copy of dL/dp0 (may be null)
  int dry;
  unsigned* status;
  // Variants (all zero: a reverse Euler step, gradient with the H(p0, q0) term).
  int rk;              // 1: stage `stage` (3..0) of the reverse of an RK4 step; the
                       // AB record then holds the stage adjoint, a64/b64 the
                       // adjoint of the step's end state
  int stage;
  double* ya64;        // RK4: FP64 adjoint of the step's start state, summed over the stages
  double* yb64;
  int h_at_end;        // the loss takes H at t = 1: no H(p0, q0) term in the gradient
  int dim;             // 2: planar landmarks; 0 or 3: 3-D
  int late_trigger;    // trigger the next launch after the pair sums (pdl_trigger)
  int combine64;       // add the split partials in FP64 (0: double-single)
};

// Packed batches of independent problems.  Problem b occupies landmarks
// [off, off+npad) of every packed array; items are (problem, target tile).
struct BatchProb {
  int off, n, npad;
  int split_len;    // sources per CTA of the forward kernel's clusters
  int split_len_b;  // and of the reverse kernel's
  int pad_;
  double kq, kappa, dt, lambda;
};
struct BatchItem {
  int prob, tile;
};
struct BatchTables {
  const BatchItem* items;
  const BatchProb* probs;
};

StepConfig step_config_for(int kind, int npad, int threads, int R, int cluster, int groups = 1);
// The built-in configuration for `kind` (0 forward, 1 reverse) and npad
// landmarks, or the tuning override when one is set.  variants: a sweep
// with RK4 stages or a terminal launch, whose kernels exist for the
// built-in CTA sizes only (so the override does not apply).
StepConfig choose_step_config(int kind, int npad, int num_sms, bool variants = false);
// CTA sizes of the built-in configurations (one target per thread, one warp
// group); the variant kernels are compiled for these.
constexpr int kVarFwdThreads = 128;
constexpr int kVarBwdThreads = 64;
// Override the fused step configuration of `kind` (threads == 0 restores the
// built-in choice).  Returns false for an unknown variant.
bool set_step_override(int kind, int threads, int R, int groups, int cluster);
// Cluster scheduling preference forced on every step-kernel launch (0
// driver default, 1 spread, 2 load balancing), or -1: each configuration's
// own policy.
void set_cluster_policy(int policy);
// When step kernels trigger the next launch after their pair sums: -1 the
// library's rule (reverse-step grids resident in one wave), 0 never, 1 always.
void set_late_trigger(int mode);
// Whether the step kernels add their split partials in FP64 (true) or in
// double-single arithmetic (false, the initial state).
void set_combine_f64(bool on);
bool combine_f64();
// Whether choose_step_config reads the measured step-configuration table.
void set_step_table(bool on);
// Whether a single-problem step launch of configuration c (kind 0 forward,
// 1 reverse; dim 3 or 2; rk: RK4 stages) triggers the next launch after its
// pair sums.
bool late_trigger_for(int kind, const StepConfig& c, int dim, bool rk);
// The policy for a launch of `ctas` CTAs on `num_sms` SMs: load balancing
// when the grid is at least 1.5 waves of 8 CTAs per SM, else spread.
int policy_for_grid(long long ctas, int num_sms);
// cudaOccupancyMaxActiveClusters of a single-problem step kernel variant.
cudaError_t max_active_clusters(int kind, int threads, int R, int groups, int cluster, int* out);
// The kernel instantiation a launch of configuration cfg runs (null: none
// compiled).  variants: RK4 stages or the terminal launch; rk: RK4 stages.
using FwdKernel = void (*)(StepFwdArgs);
using BwdKernel = void (*)(StepBwdArgs);
FwdKernel forward_kernel_for(const StepConfig& cfg, int dim, bool variants);
BwdKernel backward_kernel_for(const StepConfig& cfg, int dim, bool rk);
cudaError_t launch_step_forward(const StepConfig& cfg, const StepFwdArgs& a, cudaStream_t st, bool pdl);
cudaError_t launch_step_backward(const StepConfig& cfg, const StepBwdArgs& a, cudaStream_t st, bool pdl);
// The launch shape of the packed batch kernels of `kind` (0 forward, 1
// reverse) that a batch engine created now uses: CTA size and cluster size.
// set_batch_shape(kind, 0, 0) restores the built-in shape.
void batch_shape(int kind, int* threads, int* cluster);
bool set_batch_shape(int kind, int threads, int cluster);
// One launch over `items` (problem, tile) items; cfg gives the kernel variant
// and cluster size (its tiles / split_len fields are unused).
cudaError_t launch_bstep_forward(const StepConfig& cfg, int items, const StepFwdArgs& a, const BatchTables& bt,
                                 cudaStream_t st, bool pdl);
cudaError_t launch_bstep_backward(const StepConfig& cfg, int items, const StepBwdArgs& a, const BatchTables& bt,
                                  cudaStream_t st, bool pdl);

// ---------------------------------------------------------------- combine kernels
struct PackArgs {
  const float* q;      // (N,3) float32 inputs (device)
  const float* p;      // may be null (zeros)
  const double* p64_in;  // FP64 momenta (used instead of p when set)
  const float* tgt;    // may be null
  double* q64;
  double* p64;
  double* t64;         // may be null
  float4* qp;          // traj[0]
  int n;
  double kq;
  unsigned* status;
  int dim;             // 2: planar landmarks ((N,2) arrays); 0 or 3: 3-D
};

struct UnpackArgs {
  const double* x64;
  float* out;
  int n3;
};

cudaError_t launch_pack(const PackArgs& a, cudaStream_t st);
cudaError_t launch_unpack(const UnpackArgs& a, cudaStream_t st);
// Restore an FP64 state checkpoint into q64, p64 and record slot 0 of rec,
// with the same rounding as the step kernels' epilogue.
cudaError_t launch_restore(const double* ckq, const double* ckp, double* q64, double* p64, float4* rec, int n,
                           double kq, cudaStream_t st, int dim = 3);
// Hq, Hp straight from one split-partial set (step_forward entry point).
cudaError_t launch_partials_to_out(const Partial* part, int splits, int n, int npad,
                                   float* out_a, float* out_b, cudaStream_t st);
// Two (N,3) float32 arrays -> pair records {-sa * a, sb * b} (QP: a = q,
// b = p) or {sa * a, -sb * b} (AB: a = alpha, b = beta), zero-padded to npad.
cudaError_t launch_to_records(const float* a, const float* b, float4* rec, int n, int npad, double sa, double sb,
                              int ab_layout, unsigned* status, cudaStream_t st);

int combine_threads();
int combine_group();  // lanes per landmark in the combine kernels

}  // namespace gs
