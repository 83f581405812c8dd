/*
 * gshoot — landmark matching by geodesic shooting on one GB300 (sm_103a).
 *
 * C ABI of the library libgshoot.so.  It evaluates the method of
 * J. Wang, "Fast geodesic shooting for landmark matching using CUDA":
 * 3-D landmarks q_i, momenta p_i (i < N), Gaussian kernel
 * g_ij = exp(-||q_i - q_j||^2 / (2 sigma^2)), Hamiltonian
 * H = 1/2 sum_ij g_ij p_i . p_j (Eq. 1), Hamiltonian flow (Eq. 2) integrated by
 * T explicit Euler steps of dt = 1/T (Algorithm 1), loss
 * L(p0) = H(p0, q0) + lambda ||q(1) - target||^2 (Eq. 3), its gradient by the
 * exact reverse sweep of those Euler steps, and L-BFGS over p0 (Section 2.1).
 * Variants selected in gs_params: RK4 steps with their exact adjoint, the
 * kinetic term at t = 1 (Algorithm 1's pseudocode), and planar landmarks.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Arrays.  Every landmark array is (N, 3) row-major float32, contiguous
 *   (x0 y0 z0 x1 y1 z1 ...).  A pointer may be device memory (cudaMalloc,
 *   managed) or host memory (pageable or pinned); the library checks with
 *   cudaPointerGetAttributes and stages host arrays through its own device
 *   workspace.  Device memory must belong to the current device (the one
 *   cudaSetDevice selected in the calling thread): memory of another GPU is
 *   rejected with GS_EINVAL, because this device's kernels cannot safely
 *   read it.  The caller owns every array; the library never keeps a pointer
 *   past the call.
 * Scalars.  Scalar outputs (double*, int32_t*) are host pointers and may be
 *   NULL when not wanted.
 * Streams.  `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   Work is enqueued on it.  A call returns only after the stream has
 *   finished the call's work when any output is a host pointer or a scalar
 *   output is requested; otherwise the call is asynchronous and its outputs
 *   are ready in stream order.
 * Workspace.  The library owns one device workspace per CUDA device, grown on
 *   demand and freed by gs_release_workspace().  Calls into the library are
 *   serialised by a process-wide mutex.
 * Status.  GS_OK (0) on success; a negative gs_status on error, in which case
 *   the outputs are undefined and gs_last_error() describes the failure;
 *   a positive status is a warning with valid outputs.
 * Device errors.  Kernels record non-finite inputs and expired waits in a
 *   device status word instead of faulting; the synchronous path reads it and
 *   returns GS_ENONFINITE or GS_ETIMEOUT.  Every device-side wait gives up
 *   after one second (gs_check_wait_timeout exercises that path).
 */
#ifndef GSHOOT_H
#define GSHOOT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gs_status {
    GS_OK = 0,
    GS_NOT_CONVERGED = 1,   /* register_landmarks stopped at max_iter */
    GS_EINVAL = -1,         /* bad argument (N < 1, T < 1, sigma <= 0, NULL array, ...) */
    GS_ENOMEM = -2,         /* device allocation failed */
    GS_ECUDA = -3,          /* a CUDA runtime call failed (message in gs_last_error) */
    GS_ETIMEOUT = -4,       /* a bounded device-side wait expired */
    GS_ENONFINITE = -5,     /* an input or an intermediate was NaN or Inf */
    GS_ENOLIB = -6          /* no usable CUDA device */
} gs_status;

/* Time integrators of the flow (gs_params.integrator). */
enum {
    GS_EULER = 0,  /* explicit Euler, Algorithm 1: q <- q + dt Hp, p <- p - dt Hq */
    GS_RK4 = 1     /* classical fourth-order Runge-Kutta on y = (q, p), f = (Hp, -Hq):
                      k1 = f(y), k2 = f(y + dt/2 k1), k3 = f(y + dt/2 k2),
                      k4 = f(y + dt k3), y <- y + dt/6 (k1 + 2 k2 + 2 k3 + k4);
                      four pair-sum evaluations per step */
};

/* Where the kinetic term of the loss is evaluated (gs_params.kinetic_at). */
enum {
    GS_KINETIC_START = 0,  /* L = H(p0, q0) + lambda ||q(1) - target||^2 (Eq. 3) */
    GS_KINETIC_END = 1     /* L = H(p(1), q(1)) + lambda ||q(1) - target||^2, the form of
                              Algorithm 1's pseudocode (its loss line); the flow
                              conserves H, the discrete steps only approximately */
};

/* Parameters of one registration problem (Algorithm 1 inputs, Section 2.2). */
typedef struct gs_params {
    int64_t N;          /* number of landmarks, >= 1 */
    int32_t T;          /* number of time steps, >= 1; dt = 1/T */
    int32_t ckpt_every; /* 0: keep the whole trajectory; k > 0: keep the FP64
                           state every k steps and recompute the rest in the
                           reverse sweep */
    double sigma;       /* Gaussian kernel standard deviation, > 0 */
    double lambda;      /* weight of the landmark mismatch term of Eq. 3, >= 0 */
    int32_t lbfgs_m;    /* L-BFGS memory (pairs kept), 1..64 (register only) */
    int32_t max_iter;   /* L-BFGS iteration limit (register only) */
    double grad_tol;    /* stop when ||g_k|| <= grad_tol ||g_0|| (register only) */
    int32_t integrator; /* GS_EULER (0, the paper's) or GS_RK4; the gradient is
                           always the exact adjoint of the chosen steps */
    int32_t kinetic_at; /* GS_KINETIC_START (0) or GS_KINETIC_END */
    int32_t dim;        /* dimension of the landmarks: 3 (or 0) for 3-D, 2 for planar
                           landmarks (the paper codes both cases, Section 2.5).  With
                           dim = 2 every landmark array of shoot_forward,
                           shoot_gradient and register_landmarks is (N, 2) */
    int32_t reserved;   /* set to 0 */
} gs_params;

/*
 * step_forward — StepForward of Algorithm 2 / Algorithm 4 (Section 2.2, 2.5):
 * the two derivative terms of Eq. 2 at state (q, p),
 *   Hp_i = dH/dp_i =  sum_j g_ij p_j,
 *   Hq_i = dH/dq_i = -(1/sigma^2) sum_j (p_i . p_j) g_ij (q_i - q_j).
 * In: N, sigma, q, p.  Out: Hq, Hp (all (N,3) float32).
 */
gs_status step_forward(int64_t N, double sigma, const float* q, const float* p,
                       float* Hq, float* Hp, void* stream);

/*
 * step_backward — StepBackward (Section 2.2; formula not printed in the paper):
 * the transposed Jacobian of (Hp, -Hq) at (q, p) applied to the adjoint
 * (alpha, beta) = (dL/dq, dL/dp) of the state after the step.  With
 * e_ij = beta_i - beta_j, u_ij = alpha_i . p_j + alpha_j . p_i, s = 1/sigma^2:
 *   dalpha_i = s sum_j g_ij [ c_ij e_ij - (u_ij + s c_ij e_ij . d_ij) d_ij ]
 *   dbeta_i  =   sum_j g_ij [ alpha_j + s (e_ij . d_ij) p_j ]
 * One reverse Euler step is alpha <- alpha + dt dalpha, beta <- beta + dt dbeta.
 * In: N, sigma, q, p, alpha, beta.  Out: dalpha, dbeta.
 */
gs_status step_backward(int64_t N, double sigma, const float* q, const float* p,
                        const float* alpha, const float* beta,
                        float* dalpha, float* dbeta, void* stream);

/*
 * shoot_forward — the forward flow of Algorithm 1 (its forward loop): T explicit
 * Euler steps q <- q + dt Hp, p <- p - dt Hq from (q0, p0), or T RK4 steps
 * when prm->integrator is GS_RK4.
 * In: prm (N, T, sigma, integrator used), q0, p0.  Out: q1, p1 = state at
 * t = 1 (either may be NULL), *H0 = H(p0, q0) (Eq. 1) in FP64 (NULL to skip).
 */
gs_status shoot_forward(const gs_params* prm, const float* q0, const float* p0,
                        float* q1, float* p1, double* H0, void* stream);

/*
 * shoot_gradient — ComputeGradient of Algorithm 1: forward flow, the loss of
 * Eq. 3, and the reverse sweep.
 * In: prm (N, T, sigma, lambda, ckpt_every, integrator, kinetic_at used),
 *     q0, p0, target.
 * Out: *loss (FP64, NULL to skip), grad_p0 = dL/dp0 (NULL to skip),
 *      grad_q0 = dL/dq0 (NULL to skip), all (N,3) float32.
 * Variants: with GS_RK4 the reverse sweep is the exact adjoint of the RK4
 * steps (StepBackward at each of the four stage states of a step, applied to
 * stage adjoints built from the step's adjoint and the next stage's result).
 * With GS_KINETIC_END the adjoint starts from alpha(1) = 2 lambda (q(1) -
 * target) + Hq(q(1), p(1)), beta(1) = Hp(q(1), p(1)), and the gradient has no
 * H(p0, q0) term.
 */
gs_status shoot_gradient(const gs_params* prm, const float* q0, const float* p0,
                         const float* target, double* loss,
                         float* grad_p0, float* grad_q0, void* stream);

/* Result of register_landmarks (all fields written when the pointer is set). */
typedef struct gs_register_info {
    double loss;        /* loss of Eq. 3 at the returned p0 */
    double grad_norm0;  /* ||dL/dp0|| at the initial p0 */
    double grad_norm;   /* ||dL/dp0|| at the returned p0 */
    double avg_dist;    /* AverageDist(q(1), target) of Section 3.1 */
    double max_dist;    /* MaxDist(q(1), target) of Section 3.1 */
    int32_t iters;      /* L-BFGS iterations taken */
    int32_t evals;      /* gradient evaluations (ComputeGradient calls) */
    int32_t status;     /* 0: ||g|| <= grad_tol ||g0||; 1: max_iter reached;
                           2: the line search found no step meeting the
                              Wolfe conditions (rounding-noise floor) */
    int32_t reserved;
} gs_register_info;

/*
 * velocity_field — the velocity field of Eq. 4 at M query points:
 *   v(x_i) = sum_l g(|q_l - x_i|) p_l,   g(r) = exp(-r^2 / (2 sigma^2)),
 * for one landmark state (q, p).  At a landmark it equals Hp.
 * In: q, p (N, 3), x (M, 3).  Out: v (M, 3).  FP32 row-major arrays, host or
 * device; host outputs are written before the call returns.
 * GS_EINVAL: N or M outside [1, 2^26], sigma not finite and > 0, a NULL
 * array.  GS_ENONFINITE (synchronous calls): a non-finite velocity.
 */
gs_status velocity_field(int64_t N, int64_t M, double sigma, const float* q, const float* p,
                         const float* x, float* v, void* stream);

/*
 * flow_points — M points carried through the deformation that the initial
 * momentum p0 generates (Section 2.1, Eq. 4): the landmarks flow forward
 * from (q0, p0) as in shoot_forward, and every point takes the same T Euler
 * steps through the velocity field of the same time step,
 *   x <- x + dt v(x; q(t_k), p(t_k)),  k = 0..T-1,  dt = 1/T.
 * A landmark used as a point follows q(t).  Points are kept in FP64
 * between steps.
 * In: prm (N, T, sigma used), q0, p0 (N, 3), x0 (M, 3).  Out: x1 (M, 3).
 * Arrays as in velocity_field.  Errors as in shoot_forward; M outside
 * [1, 2^26] or a NULL point array is GS_EINVAL, and so is an integrator
 * other than GS_EULER (the points take Euler steps only) or dim = 2 (3-D
 * only).
 */
gs_status flow_points(const gs_params* prm, const float* q0, const float* p0, int64_t M,
                      const float* x0, float* x1, void* stream);

/*
 * register_landmarks — the outer optimisation of Algorithm 1: L-BFGS over the initial
 * momentum p0 of the loss L(p0) = H(p0, q0) + lambda ||q(1) - target||^2
 * (Eq. 3), each function evaluation being one ComputeGradient.  Settings
 * (the paper used VNL's L-BFGS without stating them): memory prm->lbfgs_m
 * (1..64), two-loop recursion with s.y / y.y scaling, first step -g scaled to
 * 1/||g0||, strong-Wolfe line search (c1 = 1e-4, c2 = 0.9, at most 20
 * evaluations), stop when ||g|| <= prm->grad_tol ||g0|| or after
 * prm->max_iter iterations.  Vectors are FP64 on the device.
 * In: prm (N, T, sigma, lambda, lbfgs_m, max_iter, grad_tol), q0, target,
 *     p0_inout = starting momenta (zeros for the default start).
 * Out: p0_inout = final momenta; *info (NULL to skip).
 * Returns GS_OK when the gradient tolerance was met (or info is NULL), and
 * GS_NOT_CONVERGED (> 0, outputs valid) when it stopped at max_iter or at the
 * noise floor (info->status).  Synchronises `stream`.
 */
gs_status register_landmarks(const gs_params* prm, const float* q0, const float* target,
                             float* p0_inout, gs_register_info* info, void* stream);

/* ---------------------------------------------------------------- batches and serving
 * Many independent registrations share packed device arrays.  Each time
 * step of their gradients is a single launch over all of them (one cluster
 * per target tile of any problem).  L-BFGS advances in rounds: each round
 * evaluates every active problem once.  The serving entry points add
 * continuous batching: requests that arrive while others run are admitted at
 * round boundaries as soon as device memory frees up.
 */

/* One problem of register_batch. */
typedef struct gs_batch_problem {
    int64_t N;                /* landmarks, >= 1 */
    double sigma, lambda;     /* kernel width and mismatch weight of this problem */
    const float* q0;          /* (N,3) template, host or device */
    const float* target;      /* (N,3) target, host or device */
    float* p0;                /* (N,3) starting momenta (NULL: zeros); receives the result */
    gs_register_info info;    /* output */
} gs_batch_problem;

/*
 * register_batch — B independent runs of register_landmarks, packed: every
 * time step of every gradient evaluation is one launch over all problems
 * still running.  Shared settings: T, lbfgs_m (1..64), max_iter, grad_tol.
 * Every problem is 3-D and uses the Euler integrator and the kinetic term
 * at t = 0 (GS_EULER, GS_KINETIC_START), as does the server.
 * Writes probs[b].p0 (when non-NULL) and probs[b].info.  Each problem
 * follows the same L-BFGS as register_landmarks.  Returns GS_OK,
 * GS_NOT_CONVERGED if any problem stopped short of grad_tol, or the first
 * error.  Synchronises `stream`.
 */
gs_status register_batch(int32_t B, gs_batch_problem* probs, int32_t T, int32_t lbfgs_m,
                         int32_t max_iter, double grad_tol, void* stream);

/* Settings of a registration server. */
typedef struct gs_server_config {
    int32_t T;              /* time steps of every request */
    int32_t lbfgs_m;        /* L-BFGS memory (1..64) */
    int32_t max_iter;       /* L-BFGS iteration limit */
    int32_t max_problems;   /* requests resident at once */
    double grad_tol;        /* stop at ||g|| <= grad_tol ||g0|| */
    uint64_t memory_budget; /* device bytes the server may allocate (admission limit) */
    void* stream;           /* cudaStream_t for all of the server's work */
    int32_t schedule;       /* GS_SCHED_ALL (0): every resident request is evaluated in
                               every round; GS_SCHED_FAIR (1): fair shares of pair work,
                               so small requests advance more rounds than large ones;
                               GS_SCHED_LANES (2): two lanes, see below */
    int32_t lane_split;     /* GS_SCHED_LANES: requests of at most this many landmarks go
                               to the small lane (0: 8192); must be 0 otherwise */
} gs_server_config;

/* Round schedules of the server (gs_server_config.schedule).  Under
 * GS_SCHED_FAIR each resident request carries a virtual time, the pair work
 * (N^2 per evaluation) it has been charged; a round evaluates the requests
 * whose virtual time is below the smallest one plus the smallest request's
 * cost, and a request starts at the smallest virtual time present when it is
 * admitted.  Every request then receives the same pair work per unit time,
 * and a small request finishes after its own work instead of the largest
 * request's.  Under GS_SCHED_LANES the server keeps two engines: requests of
 * at most lane_split landmarks go to a small lane (a quarter of the memory
 * budget, the fair schedule, a stream of its own at the device's highest
 * priority), the others to a large
 * lane (the rest of the budget, every resident request in every round, on
 * `stream`).  gs_server_step runs one round of the large lane and, on a
 * second host thread at the same time, as many rounds of the small lane as
 * fit in it (at least one), so small requests finish early without taking
 * rounds from the large ones.  A request's iterates do not depend on the
 * schedule or the lane. */
enum { GS_SCHED_ALL = 0, GS_SCHED_FAIR = 1, GS_SCHED_LANES = 2 };

typedef struct gs_server gs_server;

/* Create a server; allocates its whole memory budget up front. */
gs_status gs_server_create(const gs_server_config* cfg, gs_server** out);

/* Queue a request (arrays are copied; host or device).  *request_id names it.
 * GS_ENOMEM if the request alone exceeds the memory budget. */
gs_status gs_server_submit(gs_server* sv, int64_t N, double sigma, double lambda,
                           const float* q0, const float* target, const float* p0,
                           int64_t* request_id);

/* One round: admit queued requests while memory allows, evaluate the
 * resident requests the schedule selects once each (all of them under
 * GS_SCHED_ALL; under GS_SCHED_LANES one round of the large lane and the
 * small lane's rounds that run alongside it), advance their L-BFGS, retire
 * finished ones, admit again.
 * Out (each may be NULL): requests resident, requests queued, requests
 * finished in this round. */
gs_status gs_server_step(gs_server* sv, int32_t* active, int32_t* queued, int32_t* completed);

/* Result of a request.  *done = 0 while it is queued or running.  When done:
 * p0_out (N,3 float32, host or device, may be NULL), *info, and latency[0]
 * = seconds from submission to result, latency[1] = from admission to
 * result (latency may be NULL). */
gs_status gs_server_poll(gs_server* sv, int64_t request_id, float* p0_out,
                         gs_register_info* info, double* latency, int32_t* done);

/* Capacity and free space of the packed arrays (landmarks), bytes allocated. */
gs_status gs_server_stats(gs_server* sv, int64_t* capacity_landmarks, int64_t* free_landmarks,
                          int64_t* bytes);

/* Free the server and its device memory. */
void gs_server_destroy(gs_server* sv);

/*
 * gs_time_pair_kernels — diagnostics (no counterpart in the paper): the
 * average device time of one launch of each pair-sum kernel, StepForward and
 * StepBackward, in the tile configuration shoot_gradient uses for prm->N.
 * Runs shoot_gradient(prm, q0, p0, target) once to set up the trajectory and
 * adjoint state, then launches each pair kernel `reps` times back to back on
 * `stream` between two CUDA events (middle time step of the trajectory).
 * Out: *fwd_ms, *bwd_ms (host, per launch); *launches_per_eval = kernel
 * launches of one shoot_gradient call (NULL to skip any of them).
 * Synchronises `stream`.
 */
gs_status gs_time_pair_kernels(const gs_params* prm, const float* q0, const float* p0,
                               const float* target, int32_t reps, double* fwd_ms,
                               double* bwd_ms, int32_t* launches_per_eval, void* stream);

/*
 * step_forward_noalloc — StepForward for callers that cannot allocate device
 * memory.  The paper has no counterpart; it is a library-usage variant.
 *
 * The other entry points take their scratch from a workspace the library
 * grows with cudaMalloc.  Some callers cannot accept that: a host program
 * whose device memory is owned by another allocator under a fixed budget, or
 * code for which a cudaMalloc (which can synchronise the whole device) is not
 * acceptable.  This entry point computes the same Hq, Hp as step_forward, but
 * uses a file-scope static device array of about 3.3 MB as its scratch.  It
 * never calls cudaMalloc, cudaFree or any allocating routine.
 *
 * Limits: 1 <= N <= 8192.  Larger N is rejected with GS_EINVAL.  q, p, Hq
 *   and Hp must be device arrays: unlike step_forward, which stages host
 *   arrays through its own device workspace, this entry point rejects host
 *   memory with GS_EINVAL.  Device memory must belong to the current device (the one
 *   cudaSetDevice selected in the calling thread): memory of another GPU is
 *   rejected with GS_EINVAL, because this device's kernels cannot safely
 *   read it.  The caller owns every array; the library never keeps a pointer
 *   past the call.
 * Memory: every GPU that loads the library holds the static array until the
 *   process exits.
 * Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current).
 * Every call classifies its pointers with cudaPointerGetAttributes, and reads
 *   the device status word back into host memory.
 * Sharing: every call on a device uses the same array.  Each call clears the
 *   status word and rewrites the rest of the scratch it reads.  Calls whose
 *   work overlaps on the GPU (different streams or host threads) race on the
 *   array; serialise them.
 * Synchronises `stream` before returning, and reports GS_ENONFINITE or
 * GS_ETIMEOUT from the device status word.  The sum order differs from
 * step_forward (at most 8 source splits), so results agree to rounding,
 * not bitwise.
 */
gs_status step_forward_noalloc(int64_t N, double sigma, const float* q, const float* p,
                               float* Hq, float* Hp, void* stream);

/*
 * gs_time_pair_config — tuning diagnostics (no counterpart in the paper):
 * average device time of one launch of a pair-sum kernel variant.
 * kind 0 = StepForward split-partial kernel (alpha, beta ignored, may be
 *          NULL), 1 = StepBackward split-partial kernel;
 * kind 2 = fused forward time-step kernel, 3 = fused reverse time-step
 *          kernel, run in a mode that computes and reduces everything but
 *          writes no state.
 * threads, R, groups select the variant (CTA size, targets per thread,
 * warp groups that split each CTA's sources; groups must be 1 for kinds 0/1).
 * For kinds 0/1, splits > 0 forces the number of source splits and
 * splits <= 0 lets the library balance them; for kinds 2/3, splits is the
 * cluster size (1 to 16, at most the CTA's targets).  Adding 16 to kind
 * captures the `reps` launches into one CUDA graph (linked by programmatic
 * dependent launch) and times its replay.
 * The kernel runs `reps` times back to back on (q, p[, alpha,
 * beta]) between two CUDA events on `stream`.  Out: *ms per launch,
 * *splits_used (NULL to skip).  GS_EINVAL for an unknown variant.
 * Synchronises `stream`.
 */
gs_status gs_time_pair_config(int32_t kind, int64_t N, double sigma, const float* q,
                              const float* p, const float* alpha, const float* beta,
                              int32_t threads, int32_t R, int32_t groups, int32_t splits,
                              int32_t reps, double* ms, int32_t* splits_used, void* stream);

/*
 * gs_set_step_config — tuning (no counterpart in the paper): override the
 * fused time-step kernel configuration used by shoot_forward / shoot_gradient
 * for kind 0 (forward) or 1 (reverse): CTA size, targets per thread, warp
 * groups and cluster size, as in gs_time_pair_config.  threads = 0 restores
 * the built-in choice.  Clears the cached graphs.  GS_EINVAL for an unknown
 * variant.
 */
gs_status gs_set_step_config(int32_t kind, int32_t threads, int32_t R, int32_t groups,
                             int32_t cluster);

/*
 * gs_set_cluster_policy — tuning (no counterpart in the paper): force the
 * cluster scheduling preference of every fused time-step launch: 0 the CUDA
 * driver's default, 1 spread, 2 load balancing; -1 (the initial state)
 * restores the library's own choice, which is load balancing for grids of
 * 1.5 waves or more and spread below.  Clears the cached graphs.
 *
 * gs_max_active_clusters — diagnostics: how many clusters of `cluster` CTAs
 * of the fused time-step kernel variant (kind 0 forward, 1 reverse; threads,
 * R, groups as in gs_time_pair_config) can be resident on the current device at once
 * under the current policy.  GS_EINVAL for an unknown variant.
 */
gs_status gs_set_cluster_policy(int32_t policy);
gs_status gs_max_active_clusters(int32_t kind, int32_t threads, int32_t R, int32_t groups,
                                 int32_t cluster, int32_t* clusters);

/*
 * gs_set_late_trigger — tuning (no counterpart in the paper): when a fused
 * time-step kernel lets the next kernel of the graph launch (programmatic
 * dependent launch) before it finishes.  The trigger is issued after the
 * pair sums, so that the next step's launch overlaps only the reduction and
 * the epilogue; the next step still waits for this one's results.  mode -1
 * (the initial state): the library's rule, reverse-step grids whose CTAs are
 * all resident at once (forward steps measured slower with the trigger);
 * 0: never; 1: every step kernel.  Clears the cached graphs.  GS_EINVAL for
 * another mode.
 */
gs_status gs_set_late_trigger(int32_t mode);

/*
 * gs_set_batch_config — tuning (no counterpart in the paper): the launch
 * shape of the packed time-step kernels that register_batch and servers
 * created after this call use, for kind 0 (forward) or 1 (reverse): CTA
 * size (one target per thread) and cluster size, which must divide the CTA
 * size.  threads = 0 restores the built-in shape (128 threads forward, 64
 * reverse, clusters of 8).  An engine keeps the shape it was created with,
 * so a problem's sums split the same way alone and in any mix of that
 * engine.  GS_EINVAL for a shape with no packed kernel.
 */
gs_status gs_set_batch_config(int32_t kind, int32_t threads, int32_t cluster);

/*
 * gs_set_combine_precision — numerics (no counterpart in the paper): how the
 * time-step kernels add the per-split partial sums of each target (the
 * block-sum combine of every step).  f64 = 0 (the initial state):
 * double-single arithmetic (FP32 pairs with error-free TwoSum, about 48
 * significant bits); f64 = 1: each partial converted to FP64 and the
 * partials added in FP64.  Either way the order is fixed and the result
 * deterministic; the two differ in the last bits.  Applies to every entry
 * point that runs the step kernels, batched and served ones included.
 * Clears the cached graphs.  GS_EINVAL for another value.
 */
gs_status gs_set_combine_precision(int32_t f64);

/*
 * gs_set_step_table — tuning (no counterpart in the paper): whether the
 * fused time-step kernels take their CTA and cluster sizes from the table
 * measured offline on this GPU model (one entry per padded landmark count
 * up to 16384; used only on a device with the table's SM count; larger
 * counts take the size rule).  on = 1 (the initial state): the table; 0:
 * the size rule the table refines (forward 128-thread CTAs in clusters of 16 and reverse
 * 64-thread CTAs in clusters of 8, half-size CTAs up to 2048 landmarks).
 * The cluster size sets how each target's sum is split, so the two choices
 * can differ in the last bits of a result.  Clears the cached graphs.
 * GS_EINVAL for another value.
 */
gs_status gs_set_step_table(int32_t on);

/*
 * gs_step_config — diagnostics (no counterpart in the paper): the fused
 * time-step kernel configuration that shoot_forward / shoot_gradient launch
 * for N landmarks, kind 0 (forward) or 1 (reverse), on a device with
 * num_sms SMs (num_sms <= 0: the current device), under the current table
 * switch and overrides.  variants != 0 asks for the RK4 / terminal / planar
 * launches, which use the full-size CTAs.  Out: *threads per CTA and
 * *cluster (CTAs per cluster); one target per thread and one warp group
 * unless an override says otherwise.  With num_sms > 0 no CUDA call is
 * made.  GS_EINVAL for a bad kind, N outside [1, 2^26] or NULL outputs.
 */
gs_status gs_step_config(int32_t kind, int64_t N, int32_t num_sms, int32_t variants, int32_t* threads,
                         int32_t* cluster);

/*
 * gs_set_phase_timing — diagnostics (no counterpart in the paper): when `on`
 * is nonzero, the CUDA graphs of shoot_forward / shoot_gradient (and of the
 * L-BFGS evaluations) on the current device record three events: before the
 * first time step, between the forward and the reverse sweep, and after the
 * last step.  Graphs are cached separately with and without the events.
 * GS_ECUDA if the events cannot be created.
 *
 * gs_phase_times — the device time, in ms, of the forward sweep (T fused
 * forward step launches, pack excluded) and of the reverse sweep (T fused
 * reverse step launches, plus the checkpoint recomputation when
 * ckpt_every > 0) of the last graph replayed with phase timing on.  The
 * caller must have synchronised the stream of that replay; GS_ECUDA if it
 * has not finished, GS_EINVAL if phase timing was never switched on.
 */
gs_status gs_set_phase_timing(int32_t on);
gs_status gs_phase_times(double* fwd_ms, double* bwd_ms);

/*
 * gs_check_wait_timeout — failure detection (no counterpart in the paper):
 * runs one device wait that nothing completes, with the library's own
 * iteration limit, and reports how it ended.  which 0: an mbarrier phase
 * (the wait of the kernels' bulk-copy stage ring); 1: a flag in device
 * memory (a bounded poll loop).  The wait gives up, sets the timeout bit of
 * the device status word and returns; the call returns GS_ETIMEOUT, and the
 * context stays usable for the next call.  *seconds (may be NULL) receives
 * the wall time of the call.  Synchronises `stream`.  GS_EINVAL for another
 * `which`.
 */
gs_status gs_check_wait_timeout(int32_t which, double* seconds, void* stream);

/* Message for the last error of the calling thread ("" if none). */
const char* gs_last_error(void);

/* Free the device workspace and cached CUDA graphs of every device. */
void gs_release_workspace(void);


/*
 * gs_pointer_rule — diagnostics (no counterpart in the paper): the rule by
 * which every entry point treats a caller's array, given the
 * cudaPointerAttributes fields `type` (cudaMemoryType: 0 unregistered host,
 * 1 host, 2 device, 3 managed) and `device`, and the current device's
 * ordinal.  Returns 0 = host memory (staged through the workspace), 1 = used
 * in place (device memory of the current device, or managed memory),
 * 2 = rejected with GS_EINVAL (device memory of another GPU).  Makes no CUDA
 * call.
 */
int32_t gs_pointer_rule(int32_t type, int32_t ptr_device, int32_t current_device);

/*
 * gs_measure_peaks — diagnostics (no counterpart in the paper): measured
 * throughput of the arithmetic units that bound the pair kernels, on the
 * current device.  Each unit runs 8 independent dependency chains per
 * thread, 4 CTAs of 256 threads per SM, for about target_ms (1 to 2000) per
 * launch; the best of three launches timed with CUDA events on `stream`
 * counts.  rates (4 doubles, host):
 *   [0] scalar FP32 FFMA, TFLOP/s (2 flops per FMA);
 *   [1] paired FP32 FFMA2 (f32x2), TFLOP/s (2 flops per lane);
 *   [2] MUFU ex2.approx.ftz.f32 results per second;
 *   [3] FP64 DFMA, TFLOP/s.
 * ms_out (4 doubles, host, may be NULL): the kernel times behind them.
 * Synchronises `stream`.  GS_EINVAL for a NULL rates or target_ms outside
 * [1, 2000].
 */
gs_status gs_measure_peaks(double* rates, double* ms_out, double target_ms, void* stream);

/*
 * gs_measure_ffma2_distinct — diagnostics (no counterpart in the paper): the
 * paired FP32 FFMA2 rate, TFLOP/s (host double), measured as in
 * gs_measure_peaks but with three distinct register operands in every
 * instruction (each of the 8 chains has its own multiplier and addend).
 * gs_measure_peaks' rates[1] shares the multiplier and addend across all
 * instructions.  Synchronises `stream`.  GS_EINVAL for a NULL tflops or
 * target_ms outside [1, 2000].
 */
gs_status gs_measure_ffma2_distinct(double* tflops, double target_ms, void* stream);

/*
 * gs_measure_pair_loop — diagnostics (no counterpart in the paper): the
 * inner loop of the pair sums alone, at a chosen number of warps per SM.
 * kind 0 runs the StepForward loop (16 paired FP32 instructions per source
 * record of two landmarks), kind 1 the StepBackward loop (36).  Every SM
 * holds `ctas_per_sm` CTAs of `threads` threads (a multiple of 32, at most
 * 256; threads * ctas_per_sm <= 1024, and all of them resident at once, or
 * GS_EINVAL); each thread holds one target and runs the loop `reps` times
 * (1 to 4096) over 64 records (128 sources) in shared memory, with no
 * copies, barriers or epilogue.  *cycles_per_record (host): the median over
 * SMs of the SM clock cycles from the first CTA's loop start to the last
 * CTA's loop end on that SM, divided by reps * 64, i.e. the cycles per record
 * of one warp's share when the SM's warps share the schedulers (warps per
 * scheduler = threads * ctas_per_sm / 128).  The FP32
 * pipe's share of the time is then 2 * instructions * warps per scheduler /
 * cycles_per_record.  Synchronises `stream`; allocates and frees its own
 * small buffers.
 */
gs_status gs_measure_pair_loop(int32_t kind, int32_t threads, int32_t ctas_per_sm, int32_t reps,
                               double* cycles_per_record, void* stream);

/* Library ABI version: 100 * major + minor (101: gs_params gained
 * integrator and kinetic_at; 102: dim; 103: gs_server_config.schedule;
 * 104: gs_set_step_table; 105: gs_step_config; 106: gs_pointer_rule,
 * gs_measure_peaks, gs_set_combine_precision, gs_set_batch_config; 107:
 * gs_measure_pair_loop, gs_measure_ffma2_distinct). */
int32_t gs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GSHOOT_H */
