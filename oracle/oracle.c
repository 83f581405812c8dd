/*
 * FP64 CPU oracle for landmark matching by geodesic shooting
 * (J. Wang, "Fast geodesic shooting for landmark matching using CUDA").
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product (the CUDA
 * library under paper_1907_04839_gb300/) never calls it, shares no code,
 * header, table or constant with it, and fails loudly when its own CUDA
 * library is missing.
 *
 * Everything here is plain double-precision C: straightforward double loops
 * over landmark pairs i, j (the loop structure of Algorithm 2, with the
 * per-target local accumulator that Section 2.2 recommends), OpenMP over the
 * target index i only.  No blocking, fusion, reordering or approximation.
 *
 * Notation (Section 2.1): q_i, p_i in R^3 are landmark positions and momenta,
 * N landmarks, Gaussian kernel g_ij = exp(-||q_i - q_j||^2 / (2 sigma^2)),
 * s = 1/sigma^2, d_ij = q_i - q_j, c_ij = p_i . p_j.
 *
 * Readings of the paper where its text is garbled or silent:
 *   Eq. 1     H(p, q) = 1/2 <p, K(q) p> = 1/2 sum_ij g_ij p_i . p_j.
 *   Eq. 2     dq/dt = Hp = dH/dp,  dp/dt = -Hq = -dH/dq, so
 *             Hp_i = sum_j g_ij p_j,  Hq_i = -s sum_j c_ij g_ij d_ij.
 *   Alg. 2    the kernel is exp(-r^2 / (2 sigma^2)), sigma the Gaussian std.
 *   Alg. 1    dt = 1/T; T simultaneous explicit Euler steps from q0, p0:
 *             q <- q + dt Hp(q, p),  p <- p - dt Hq(q, p).
 *   Eq. 3     loss L(p0) = H(p0, q0) + lambda ||q(1) - target||^2, minimised.
 *   Alg. 1    the adjoint runs backwards through the same T Euler steps.  With
 *             alpha = dL/dq and beta = dL/dp (through the flow), one reverse
 *             step is alpha <- alpha + dt dalpha, beta <- beta + dt dbeta with
 *             (dalpha, dbeta) the transposed Jacobian of (Hp, -Hq) applied to
 *             (alpha, beta) -- StepBackward, whose formula the paper omits:
 *               e_ij = beta_i - beta_j,  u_ij = alpha_i . p_j + alpha_j . p_i,
 *               dalpha_i = s sum_j g_ij [ c_ij e_ij - (u_ij + s c_ij e_ij.d_ij) d_ij ]
 *               dbeta_i  =   sum_j g_ij [ alpha_j + s (e_ij . d_ij) p_j ]
 *             started from alpha(1) = 2 lambda (q(1) - target), beta(1) = 0.
 *             Gradient: dL/dp0 = beta(0) + Hp(q0, p0), dL/dq0 = alpha(0) + Hq(q0, p0).
 *   Eq. 4     v(x, t) = sum_l g(||q_l(t) - x||) p_l(t).
 *
 * Pins (tests/test_oracle_pins.py) tie these functions to the mathematics:
 * single landmark moves on a straight line; total momentum is conserved;
 * H drift falls at first order in dt; two-body head-on reduction to a scalar
 * recursion; rigid-motion invariance; the closed-form gradient at p0 = 0;
 * lambda = 0; a dense K matrix-vector product; brute-force central finite
 * differences of the loss; and an independent autograd of the Euler loop.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Gaussian kernel G_sigma of Section 2.1 on a squared distance. */
static double gauss(double r2, double sigma) { return exp(-r2 / (2.0 * sigma * sigma)); }

/* StepForward (Algorithm 2): Hq and Hp of Eq. 2 at state (q, p), for
 * landmarks in `dim` = 2 or 3 dimensions ((N, dim) arrays). */
void orc_step_forward_d(int dim, int64_t n, double sigma, const double* q, const double* p,
                        double* Hq, double* Hp) {
    const double s = 1.0 / (sigma * sigma);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double hq[3] = {0, 0, 0}, hp[3] = {0, 0, 0};
        for (int64_t j = 0; j < n; ++j) {
            double d[3], r2 = 0.0, c = 0.0;
            for (int k = 0; k < dim; ++k) {
                d[k] = q[dim * i + k] - q[dim * j + k];
                r2 += d[k] * d[k];
                c += p[dim * i + k] * p[dim * j + k];
            }
            const double g = gauss(r2, sigma);
            for (int k = 0; k < dim; ++k) {
                hp[k] += g * p[dim * j + k];
                hq[k] += -s * c * g * d[k];
            }
        }
        for (int k = 0; k < dim; ++k) {
            Hq[dim * i + k] = hq[k];
            Hp[dim * i + k] = hp[k];
        }
    }
}

void orc_step_forward(int64_t n, double sigma, const double* q, const double* p,
                      double* Hq, double* Hp) {
    orc_step_forward_d(3, n, sigma, q, p, Hq, Hp);
}

/* StepBackward: the transposed Jacobian of (Hp, -Hq) at (q, p) applied to the
 * adjoint (alpha, beta) of the state after the step.  See the header. */
void orc_step_backward_d(int dim, int64_t n, double sigma, const double* q, const double* p,
                         const double* alpha, const double* beta,
                         double* dalpha, double* dbeta) {
    const double s = 1.0 / (sigma * sigma);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double da[3] = {0, 0, 0}, db[3] = {0, 0, 0};
        for (int64_t j = 0; j < n; ++j) {
            double d[3], e[3], r2 = 0.0, c = 0.0, ed = 0.0, u = 0.0;
            for (int k = 0; k < dim; ++k) {
                d[k] = q[dim * i + k] - q[dim * j + k];
                e[k] = beta[dim * i + k] - beta[dim * j + k];
                r2 += d[k] * d[k];
                c += p[dim * i + k] * p[dim * j + k];
                ed += e[k] * d[k];
                u += alpha[dim * i + k] * p[dim * j + k] + alpha[dim * j + k] * p[dim * i + k];
            }
            const double g = gauss(r2, sigma);
            for (int k = 0; k < dim; ++k) {
                da[k] += s * g * (c * e[k] - (u + s * c * ed) * d[k]);
                db[k] += g * (alpha[dim * j + k] + s * ed * p[dim * j + k]);
            }
        }
        for (int k = 0; k < dim; ++k) {
            dalpha[dim * i + k] = da[k];
            dbeta[dim * i + k] = db[k];
        }
    }
}

void orc_step_backward(int64_t n, double sigma, const double* q, const double* p,
                       const double* alpha, const double* beta,
                       double* dalpha, double* dbeta) {
    orc_step_backward_d(3, n, sigma, q, p, alpha, beta, dalpha, dbeta);
}

/* StepForward restricted to the m target rows rows[0..m): (Hq, Hp) of those
 * landmarks only, each summed over all N sources.  Output (m, 3). */
void orc_step_forward_rows(int64_t n, double sigma, const double* q, const double* p,
                           int64_t m, const int64_t* rows, double* Hq, double* Hp) {
    const double s = 1.0 / (sigma * sigma);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m; ++r) {
        const int64_t i = rows[r];
        double hq[3] = {0, 0, 0}, hp[3] = {0, 0, 0};
        for (int64_t j = 0; j < n; ++j) {
            double d[3], r2 = 0.0, c = 0.0;
            for (int k = 0; k < 3; ++k) {
                d[k] = q[3 * i + k] - q[3 * j + k];
                r2 += d[k] * d[k];
                c += p[3 * i + k] * p[3 * j + k];
            }
            const double g = gauss(r2, sigma);
            for (int k = 0; k < 3; ++k) {
                hp[k] += g * p[3 * j + k];
                hq[k] += -s * c * g * d[k];
            }
        }
        for (int k = 0; k < 3; ++k) {
            Hq[3 * r + k] = hq[k];
            Hp[3 * r + k] = hp[k];
        }
    }
}

/* StepBackward restricted to the m target rows rows[0..m).  Output (m, 3). */
void orc_step_backward_rows(int64_t n, double sigma, const double* q, const double* p,
                            const double* alpha, const double* beta, int64_t m,
                            const int64_t* rows, double* dalpha, double* dbeta) {
    const double s = 1.0 / (sigma * sigma);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m; ++r) {
        const int64_t i = rows[r];
        double da[3] = {0, 0, 0}, db[3] = {0, 0, 0};
        for (int64_t j = 0; j < n; ++j) {
            double d[3], e[3], r2 = 0.0, c = 0.0, ed = 0.0, u = 0.0;
            for (int k = 0; k < 3; ++k) {
                d[k] = q[3 * i + k] - q[3 * j + k];
                e[k] = beta[3 * i + k] - beta[3 * j + k];
                r2 += d[k] * d[k];
                c += p[3 * i + k] * p[3 * j + k];
                ed += e[k] * d[k];
                u += alpha[3 * i + k] * p[3 * j + k] + alpha[3 * j + k] * p[3 * i + k];
            }
            const double g = gauss(r2, sigma);
            for (int k = 0; k < 3; ++k) {
                da[k] += s * g * (c * e[k] - (u + s * c * ed) * d[k]);
                db[k] += g * (alpha[3 * j + k] + s * ed * p[3 * j + k]);
            }
        }
        for (int k = 0; k < 3; ++k) {
            dalpha[3 * r + k] = da[k];
            dbeta[3 * r + k] = db[k];
        }
    }
}

/* Eq. 1: H(p, q) = 1/2 sum_i sum_j g_ij p_i . p_j (landmarks in dim dimensions). */
double orc_hamiltonian_d(int dim, int64_t n, double sigma, const double* q, const double* p) {
    double h = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : h)
    for (int64_t i = 0; i < n; ++i) {
        double hi = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double r2 = 0.0, c = 0.0;
            for (int k = 0; k < dim; ++k) {
                const double d = q[dim * i + k] - q[dim * j + k];
                r2 += d * d;
                c += p[dim * i + k] * p[dim * j + k];
            }
            hi += gauss(r2, sigma) * c;
        }
        h += hi;
    }
    return 0.5 * h;
}

double orc_hamiltonian(int64_t n, double sigma, const double* q, const double* p) {
    return orc_hamiltonian_d(3, n, sigma, q, p);
}

/* Forward flow of Algorithm 1 (its forward loop, started at q0): T explicit Euler
 * steps of Eq. 2.  traj_q / traj_p, when non-null, receive all T+1 states as
 * (T+1, N, 3) arrays. */
void orc_shoot_forward(int64_t n, int T, double sigma, const double* q0, const double* p0,
                       double* q1, double* p1, double* traj_q, double* traj_p) {
    const double dt = 1.0 / T;
    const size_t m = (size_t)n * 3;
    double* q = malloc(m * sizeof(double));
    double* p = malloc(m * sizeof(double));
    double* Hq = malloc(m * sizeof(double));
    double* Hp = malloc(m * sizeof(double));
    memcpy(q, q0, m * sizeof(double));
    memcpy(p, p0, m * sizeof(double));
    if (traj_q) memcpy(traj_q, q, m * sizeof(double));
    if (traj_p) memcpy(traj_p, p, m * sizeof(double));
    for (int t = 0; t < T; ++t) {
        orc_step_forward(n, sigma, q, p, Hq, Hp);
        for (size_t k = 0; k < m; ++k) {
            q[k] += Hp[k] * dt;
            p[k] -= Hq[k] * dt;
        }
        if (traj_q) memcpy(traj_q + (size_t)(t + 1) * m, q, m * sizeof(double));
        if (traj_p) memcpy(traj_p + (size_t)(t + 1) * m, p, m * sizeof(double));
    }
    memcpy(q1, q, m * sizeof(double));
    memcpy(p1, p, m * sizeof(double));
    free(q); free(p); free(Hq); free(Hp);
}

/* Eq. 3 objective: H(p0, q0) + lambda ||q(1) - target||^2. */
double orc_loss(int64_t n, int T, double sigma, double lambda, const double* q0,
                const double* p0, const double* target) {
    const size_t m = (size_t)n * 3;
    double* q1 = malloc(m * sizeof(double));
    double* p1 = malloc(m * sizeof(double));
    orc_shoot_forward(n, T, sigma, q0, p0, q1, p1, NULL, NULL);
    double mis = 0.0;
    for (size_t k = 0; k < m; ++k) mis += (q1[k] - target[k]) * (q1[k] - target[k]);
    const double L = orc_hamiltonian(n, sigma, q0, p0) + lambda * mis;
    free(q1); free(p1);
    return L;
}

/* ComputeGradient of Algorithm 1: forward flow, loss, reverse sweep.
 * Returns the loss; grad_p0 = dL/dp0 and grad_q0 = dL/dq0 (either may be
 * null).  q1, p1 and H0 receive the end state and H(p0, q0) when non-null. */
double orc_shoot_gradient(int64_t n, int T, double sigma, double lambda,
                          const double* q0, const double* p0, const double* target,
                          double* grad_p0, double* grad_q0,
                          double* q1_out, double* p1_out, double* H0_out) {
    const double dt = 1.0 / T;
    const size_t m = (size_t)n * 3;
    double* tq = malloc((size_t)(T + 1) * m * sizeof(double));
    double* tp = malloc((size_t)(T + 1) * m * sizeof(double));
    double* q1 = malloc(m * sizeof(double));
    double* p1 = malloc(m * sizeof(double));
    double* alpha = malloc(m * sizeof(double));
    double* beta = malloc(m * sizeof(double));
    double* da = malloc(m * sizeof(double));
    double* db = malloc(m * sizeof(double));
    double* Hq0 = malloc(m * sizeof(double));
    double* Hp0 = malloc(m * sizeof(double));

    orc_shoot_forward(n, T, sigma, q0, p0, q1, p1, tq, tp);
    const double H0 = orc_hamiltonian(n, sigma, q0, p0);
    double mis = 0.0;
    for (size_t k = 0; k < m; ++k) mis += (q1[k] - target[k]) * (q1[k] - target[k]);
    const double L = H0 + lambda * mis;

    for (size_t k = 0; k < m; ++k) {
        alpha[k] = 2.0 * lambda * (q1[k] - target[k]);
        beta[k] = 0.0;
    }
    for (int t = T - 1; t >= 0; --t) {
        orc_step_backward(n, sigma, tq + (size_t)t * m, tp + (size_t)t * m, alpha, beta, da, db);
        for (size_t k = 0; k < m; ++k) {
            alpha[k] += dt * da[k];
            beta[k] += dt * db[k];
        }
    }
    orc_step_forward(n, sigma, q0, p0, Hq0, Hp0);
    for (size_t k = 0; k < m; ++k) {
        if (grad_p0) grad_p0[k] = beta[k] + Hp0[k];
        if (grad_q0) grad_q0[k] = alpha[k] + Hq0[k];
    }
    if (q1_out) memcpy(q1_out, q1, m * sizeof(double));
    if (p1_out) memcpy(p1_out, p1, m * sizeof(double));
    if (H0_out) *H0_out = H0;
    free(tq); free(tp); free(q1); free(p1); free(alpha); free(beta);
    free(da); free(db); free(Hq0); free(Hp0);
    return L;
}

/* ------------------------------------------------------------------ variants
 * Two variants of the discretisation, both admitted by the paper's text:
 *
 * Integrator (integ = 0: explicit Euler as above; integ = 1: the classical
 * fourth-order Runge-Kutta method).  With y = (q, p) and f(y) = (Hp, -Hq) of
 * Eq. 2, one RK4 step of dt = 1/T is
 *   k1 = f(y), k2 = f(y + dt/2 k1), k3 = f(y + dt/2 k2), k4 = f(y + dt k3),
 *   y' = y + dt/6 (k1 + 2 k2 + 2 k3 + k4).
 * Its exact discrete adjoint, with J(Y)^T w = StepBackward at stage state Y
 * and w the adjoint of y':
 *   v4 = J(Y4)^T (dt/6 w),
 *   v3 = J(Y3)^T (dt/3 w + dt v4),
 *   v2 = J(Y2)^T (dt/3 w + dt/2 v3),
 *   v1 = J(y)^T  (dt/6 w + dt/2 v2),
 *   adjoint of y = w + v1 + v2 + v3 + v4.
 *
 * Dimension (dim = 3, or dim = 2 for planar landmarks: the paper codes the
 * two cases separately; every formula above holds with 2-vectors).
 *
 * Kinetic term (h_at_end = 0: H(p0, q0) as above; h_at_end = 1: H(p(1), q(1)),
 * the form Algorithm 1's pseudocode writes, evaluating the kinetic term at
 * the end state).  With it at the end, the adjoint starts from
 * alpha(1) = 2 lambda (q(1) - target) + Hq(q(1), p(1)), beta(1) = Hp(q(1), p(1)),
 * and the gradient is the adjoint at t = 0 with no extra term. */

/* One step of the chosen integrator from (q, p), in place.  When stage_q /
 * stage_p are non-null they receive the four RK4 stage states Y1..Y4 as
 * (4, N, 3) arrays (Y1 = y). */
static void integ_step(int dim, int64_t n, int integ, double dt, double sigma, double* q, double* p,
                       double* stage_q, double* stage_p) {
    const size_t m = (size_t)n * dim;
    if (integ == 0) {
        double* Hq = malloc(m * sizeof(double));
        double* Hp = malloc(m * sizeof(double));
        orc_step_forward_d(dim, n, sigma, q, p, Hq, Hp);
        for (size_t k = 0; k < m; ++k) {
            q[k] += Hp[k] * dt;
            p[k] -= Hq[k] * dt;
        }
        free(Hq); free(Hp);
        return;
    }
    /* RK4: kq_s, kp_s are the q and p parts of k_s = f(Y_s). */
    const double a[4] = {0.0, 0.5, 0.5, 1.0};      /* Y_s = y + a_s dt k_{s-1} */
    const double b[4] = {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6};
    double* Yq = malloc(m * sizeof(double));
    double* Yp = malloc(m * sizeof(double));
    double* Hq = malloc(m * sizeof(double));
    double* Hp = malloc(m * sizeof(double));
    double* sq = calloc(m, sizeof(double));
    double* sp = calloc(m, sizeof(double));
    memcpy(Yq, q, m * sizeof(double));
    memcpy(Yp, p, m * sizeof(double));
    for (int st = 0; st < 4; ++st) {
        if (st > 0) {
            for (size_t k = 0; k < m; ++k) {
                Yq[k] = q[k] + a[st] * dt * Hp[k];
                Yp[k] = p[k] - a[st] * dt * Hq[k];
            }
        }
        if (stage_q) memcpy(stage_q + (size_t)st * m, Yq, m * sizeof(double));
        if (stage_p) memcpy(stage_p + (size_t)st * m, Yp, m * sizeof(double));
        orc_step_forward_d(dim, n, sigma, Yq, Yp, Hq, Hp);
        for (size_t k = 0; k < m; ++k) {
            sq[k] += b[st] * Hp[k];
            sp[k] -= b[st] * Hq[k];
        }
    }
    for (size_t k = 0; k < m; ++k) {
        q[k] += dt * sq[k];
        p[k] += dt * sp[k];
    }
    free(Yq); free(Yp); free(Hq); free(Hp); free(sq); free(sp);
}

/* Forward flow with the chosen integrator: T steps from (q0, p0). */
void orc_shoot_forward_v(int dim, int64_t n, int T, double sigma, int integ, const double* q0, const double* p0,
                         double* q1, double* p1) {
    const double dt = 1.0 / T;
    const size_t m = (size_t)n * dim;
    memcpy(q1, q0, m * sizeof(double));
    memcpy(p1, p0, m * sizeof(double));
    for (int t = 0; t < T; ++t) integ_step(dim, n, integ, dt, sigma, q1, p1, NULL, NULL);
}

/* Eq. 3 objective of a variant: H at (p0, q0) or at (p(1), q(1)), plus
 * lambda ||q(1) - target||^2. */
double orc_loss_v(int dim, int64_t n, int T, double sigma, double lambda, int integ, int h_at_end,
                  const double* q0, const double* p0, const double* target) {
    const size_t m = (size_t)n * dim;
    double* q1 = malloc(m * sizeof(double));
    double* p1 = malloc(m * sizeof(double));
    orc_shoot_forward_v(dim, n, T, sigma, integ, q0, p0, q1, p1);
    double mis = 0.0;
    for (size_t k = 0; k < m; ++k) mis += (q1[k] - target[k]) * (q1[k] - target[k]);
    const double H = h_at_end ? orc_hamiltonian_d(dim, n, sigma, q1, p1) : orc_hamiltonian_d(dim, n, sigma, q0, p0);
    free(q1); free(p1);
    return H + lambda * mis;
}

/* ComputeGradient of a variant.  Returns the loss; grad_p0, grad_q0, q1, p1
 * (each may be null) as in orc_shoot_gradient; *H_out (may be null) is the
 * kinetic term of the loss. */
double orc_shoot_gradient_v(int dim, int64_t n, int T, double sigma, double lambda, int integ, int h_at_end,
                            const double* q0, const double* p0, const double* target,
                            double* grad_p0, double* grad_q0, double* q1_out, double* p1_out,
                            double* H_out) {
    const double dt = 1.0 / T;
    const size_t m = (size_t)n * dim;
    const int S = integ == 0 ? 1 : 4;   /* stage states kept per step */
    double* tq = malloc((size_t)T * S * m * sizeof(double));
    double* tp = malloc((size_t)T * S * m * sizeof(double));
    double* q = malloc(m * sizeof(double));
    double* p = malloc(m * sizeof(double));
    double* Hq = malloc(m * sizeof(double));
    double* Hp = malloc(m * sizeof(double));
    double* alpha = malloc(m * sizeof(double));
    double* beta = malloc(m * sizeof(double));
    double* ca = malloc(m * sizeof(double));
    double* cb = malloc(m * sizeof(double));
    double* va = malloc(m * sizeof(double));
    double* vb = malloc(m * sizeof(double));
    double* ya = malloc(m * sizeof(double));
    double* yb = malloc(m * sizeof(double));

    memcpy(q, q0, m * sizeof(double));
    memcpy(p, p0, m * sizeof(double));
    for (int t = 0; t < T; ++t) {
        double* sq = tq + (size_t)t * S * m;
        double* sp = tp + (size_t)t * S * m;
        if (integ == 0) {
            memcpy(sq, q, m * sizeof(double));
            memcpy(sp, p, m * sizeof(double));
            integ_step(dim, n, 0, dt, sigma, q, p, NULL, NULL);
        } else {
            integ_step(dim, n, 1, dt, sigma, q, p, sq, sp);
        }
    }
    double mis = 0.0;
    for (size_t k = 0; k < m; ++k) mis += (q[k] - target[k]) * (q[k] - target[k]);
    double H;
    if (h_at_end) {
        H = orc_hamiltonian_d(dim, n, sigma, q, p);
        orc_step_forward_d(dim, n, sigma, q, p, Hq, Hp);
        for (size_t k = 0; k < m; ++k) {
            alpha[k] = 2.0 * lambda * (q[k] - target[k]) + Hq[k];
            beta[k] = Hp[k];
        }
    } else {
        H = orc_hamiltonian_d(dim, n, sigma, q0, p0);
        for (size_t k = 0; k < m; ++k) {
            alpha[k] = 2.0 * lambda * (q[k] - target[k]);
            beta[k] = 0.0;
        }
    }
    const double L = H + lambda * mis;
    if (q1_out) memcpy(q1_out, q, m * sizeof(double));
    if (p1_out) memcpy(p1_out, p, m * sizeof(double));

    /* stage cotangent coefficients: cotangent of k_s = cw[s] dt w + cv[s] dt v_{s+1} */
    const double cw[4] = {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6};
    const double cv[4] = {0.5, 0.5, 1.0, 0.0};
    for (int t = T - 1; t >= 0; --t) {
        const double* sq = tq + (size_t)t * S * m;
        const double* sp = tp + (size_t)t * S * m;
        if (integ == 0) {
            orc_step_backward_d(dim, n, sigma, sq, sp, alpha, beta, va, vb);
            for (size_t k = 0; k < m; ++k) {
                alpha[k] += dt * va[k];
                beta[k] += dt * vb[k];
            }
            continue;
        }
        memcpy(ya, alpha, m * sizeof(double));
        memcpy(yb, beta, m * sizeof(double));
        for (int st = 3; st >= 0; --st) {
            for (size_t k = 0; k < m; ++k) {
                ca[k] = cw[st] * dt * alpha[k] + (st < 3 ? cv[st] * dt * va[k] : 0.0);
                cb[k] = cw[st] * dt * beta[k] + (st < 3 ? cv[st] * dt * vb[k] : 0.0);
            }
            orc_step_backward_d(dim, n, sigma, sq + (size_t)st * m, sp + (size_t)st * m, ca, cb, va, vb);
            for (size_t k = 0; k < m; ++k) {
                ya[k] += va[k];
                yb[k] += vb[k];
            }
        }
        memcpy(alpha, ya, m * sizeof(double));
        memcpy(beta, yb, m * sizeof(double));
    }
    if (!h_at_end) orc_step_forward_d(dim, n, sigma, q0, p0, Hq, Hp);
    for (size_t k = 0; k < m; ++k) {
        if (grad_p0) grad_p0[k] = beta[k] + (h_at_end ? 0.0 : Hp[k]);
        if (grad_q0) grad_q0[k] = alpha[k] + (h_at_end ? 0.0 : Hq[k]);
    }
    if (H_out) *H_out = H;
    free(tq); free(tp); free(q); free(p); free(Hq); free(Hp); free(alpha); free(beta);
    free(ca); free(cb); free(va); free(vb); free(ya); free(yb);
    return L;
}

/* Eq. 4: velocity v(x) = sum_l g(||q_l - x||) p_l at m query points x. */
void orc_velocity(int64_t m, const double* x, int64_t n, const double* q, const double* p,
                  double sigma, double* v) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double acc[3] = {0, 0, 0};
        for (int64_t l = 0; l < n; ++l) {
            double r2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double d = q[3 * l + k] - x[3 * i + k];
                r2 += d * d;
            }
            const double g = gauss(r2, sigma);
            for (int k = 0; k < 3; ++k) acc[k] += g * p[3 * l + k];
        }
        for (int k = 0; k < 3; ++k) v[3 * i + k] = acc[k];
    }
}

/* Points carried through the deformation by the flow of Algorithm 1's
 * forward loop (Section 2.1, Eq. 4): each of the T Euler steps moves a point x
 * by dt times the velocity field of Eq. 4 evaluated with the landmark state
 * of that step, x^{k+1} = x^k + dt v(x^k; q^k, p^k).  A landmark used as a
 * point moves exactly as the landmark does, since v(q_i) = Hp_i. */
void orc_flow_points(int64_t n, int T, double sigma, const double* q0, const double* p0,
                     int64_t m, const double* x0, double* x1) {
    const double dt = 1.0 / T;
    const size_t sn = (size_t)n * 3, sm = (size_t)m * 3;
    double* tq = malloc((size_t)(T + 1) * sn * sizeof(double));
    double* tp = malloc((size_t)(T + 1) * sn * sizeof(double));
    double* q1 = malloc(sn * sizeof(double));
    double* p1 = malloc(sn * sizeof(double));
    double* x = malloc(sm * sizeof(double));
    double* v = malloc(sm * sizeof(double));
    orc_shoot_forward(n, T, sigma, q0, p0, q1, p1, tq, tp);
    memcpy(x, x0, sm * sizeof(double));
    for (int t = 0; t < T; ++t) {
        orc_velocity(m, x, n, tq + (size_t)t * sn, tp + (size_t)t * sn, sigma, v);
        for (size_t k = 0; k < sm; ++k) x[k] += v[k] * dt;
    }
    memcpy(x1, x, sm * sizeof(double));
    free(tq); free(tp); free(q1); free(p1); free(x); free(v);
}

/* ------------------------------------------------------------------ L-BFGS
 * Limited-memory BFGS over x (Section 2.1 uses VNL's L-BFGS; its settings are
 * not stated, so this follows the reading written down for both paths):
 *   - memory m pairs (s_k, y_k), two-loop recursion, initial scaling
 *     gamma = s.y / y.y of the newest pair;
 *   - first direction -g with a first trial step 1/||g0||, later trials 1;
 *   - strong-Wolfe line search (c1 = 1e-4, c2 = 0.9) by bracketing and zoom
 *     with safeguarded cubic interpolation, at most 20 evaluations;
 *   - a pair is stored only if s.y > 1e-12 s.s^(1/2) y.y^(1/2);
 *   - stop when ||g|| <= grad_tol ||g0|| or after max_iter iterations.
 * fg(ctx, x, g) returns f(x) and writes its gradient. */
typedef double (*orc_fg_fn)(void* ctx, const double* x, double* g);

static double vdot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Minimiser of the cubic through (a, fa, da) and (b, fb, db); NAN if none. */
static double cubic_min(double a, double fa, double da, double b, double fb, double db) {
    const double d1 = da + db - 3.0 * (fa - fb) / (a - b);
    const double disc = d1 * d1 - da * db;
    if (!(disc >= 0.0)) return NAN;
    const double d2 = (b > a ? 1.0 : -1.0) * sqrt(disc);
    const double den = db - da + 2.0 * d2;
    if (den == 0.0) return NAN;
    return b - (b - a) * (db + d2 - d1) / den;
}

typedef struct {
    int64_t n;
    orc_fg_fn fg;
    void* ctx;
    const double* x;
    const double* d;
    double* xt;
    double* gt;
    int evals;
} ls_ctx;

static double ls_eval(ls_ctx* c, double a, double* dphi) {
    for (int64_t i = 0; i < c->n; ++i) c->xt[i] = c->x[i] + a * c->d[i];
    const double f = c->fg(c->ctx, c->xt, c->gt);
    c->evals++;
    *dphi = vdot(c->n, c->gt, c->d);
    return f;
}

/* Strong-Wolfe line search; returns the accepted step (xt, gt hold its point
 * and gradient, *f_out its value) or 0 on failure. */
static double line_search(ls_ctx* c, double f0, double dphi0, double a1, double* f_out) {
    const double c1 = 1e-4, c2 = 0.9;
    const int max_evals = 20;
    double a_prev = 0.0, f_prev = f0, d_prev = dphi0;
    double a = a1;
    const int start = c->evals;
    for (int it = 0; c->evals - start < max_evals; ++it) {
        double da;
        const double fa = ls_eval(c, a, &da);
        int zoom = 0;
        double lo = 0, flo = 0, dlo = 0, hi = 0, fhi = 0, dhi = 0;
        if (!(fa <= f0 + c1 * a * dphi0) || (it > 0 && fa >= f_prev)) {
            zoom = 1; lo = a_prev; flo = f_prev; dlo = d_prev; hi = a; fhi = fa; dhi = da;
        } else if (fabs(da) <= -c2 * dphi0) {
            *f_out = fa;
            return a;
        } else if (da >= 0.0) {
            zoom = 1; lo = a; flo = fa; dlo = da; hi = a_prev; fhi = f_prev; dhi = d_prev;
        }
        if (zoom) {
            while (c->evals - start < max_evals) {
                double aj = cubic_min(lo, flo, dlo, hi, fhi, dhi);
                const double w = hi - lo;
                const double lo_b = (w > 0 ? lo + 0.1 * w : hi - 0.1 * w);
                const double hi_b = (w > 0 ? hi - 0.1 * w : lo + 0.1 * w);
                const double mn = lo_b < hi_b ? lo_b : hi_b, mx = lo_b < hi_b ? hi_b : lo_b;
                if (!(aj >= mn && aj <= mx)) aj = 0.5 * (lo + hi);
                double dj;
                const double fj = ls_eval(c, aj, &dj);
                if (!(fj <= f0 + c1 * aj * dphi0) || fj >= flo) {
                    hi = aj; fhi = fj; dhi = dj;
                } else {
                    if (fabs(dj) <= -c2 * dphi0) {
                        *f_out = fj;
                        return aj;
                    }
                    if (dj * (hi - lo) >= 0.0) { hi = lo; fhi = flo; dhi = dlo; }
                    lo = aj; flo = fj; dlo = dj;
                }
            }
            return 0.0;
        }
        a_prev = a; f_prev = fa; d_prev = da;
        a = 2.0 * a;
    }
    return 0.0;
}

/* Returns 0 when the gradient tolerance was met, 1 at max_iter, -1 when a line
 * search failed.  trace (optional, max_iter+1 entries) receives f per iterate. */
int orc_lbfgs(int64_t n, double* x, orc_fg_fn fg, void* ctx, int m, int max_iter, double grad_tol,
              double* f_out, int* iters_out, int* evals_out, double* trace) {
    double* g = malloc(n * sizeof(double));
    double* d = malloc(n * sizeof(double));
    double* xt = malloc(n * sizeof(double));
    double* gt = malloc(n * sizeof(double));
    double* S = malloc((size_t)m * n * sizeof(double));
    double* Y = malloc((size_t)m * n * sizeof(double));
    double* rho = malloc(m * sizeof(double));
    double* alpha = malloc(m * sizeof(double));
    int stored = 0, head = 0, status = 1, it = 0;
    ls_ctx c = {n, fg, ctx, x, d, xt, gt, 0};
    double f = fg(ctx, x, g);
    c.evals = 1;
    const double g0 = sqrt(vdot(n, g, g));
    if (trace) trace[0] = f;
    if (g0 == 0.0) status = 0;
    for (it = 0; status == 1 && it < max_iter; ++it) {
        /* two-loop recursion: d = -H g */
        for (int64_t i = 0; i < n; ++i) d[i] = g[i];
        for (int k = 0; k < stored; ++k) {
            const int j = (head - 1 - k + m) % m;
            alpha[j] = rho[j] * vdot(n, S + (size_t)j * n, d);
            for (int64_t i = 0; i < n; ++i) d[i] -= alpha[j] * Y[(size_t)j * n + i];
        }
        if (stored > 0) {
            const int j = (head - 1 + m) % m;
            const double gamma = vdot(n, S + (size_t)j * n, Y + (size_t)j * n) /
                                 vdot(n, Y + (size_t)j * n, Y + (size_t)j * n);
            for (int64_t i = 0; i < n; ++i) d[i] *= gamma;
        }
        for (int k = stored - 1; k >= 0; --k) {
            const int j = (head - 1 - k + m) % m;
            const double b = rho[j] * vdot(n, Y + (size_t)j * n, d);
            for (int64_t i = 0; i < n; ++i) d[i] += (alpha[j] - b) * S[(size_t)j * n + i];
        }
        for (int64_t i = 0; i < n; ++i) d[i] = -d[i];
        double dphi0 = vdot(n, g, d);
        if (!(dphi0 < 0.0)) { /* not a descent direction: restart from -g */
            for (int64_t i = 0; i < n; ++i) d[i] = -g[i];
            dphi0 = -vdot(n, g, g);
            stored = 0;
        }
        const double a1 = (it == 0) ? 1.0 / g0 : 1.0;
        double fn = 0.0;
        const double a = line_search(&c, f, dphi0, a1, &fn);
        if (a == 0.0) { status = -1; break; }
        /* s = a d, y = gt - g */
        double* s = S + (size_t)head * n;
        double* y = Y + (size_t)head * n;
        for (int64_t i = 0; i < n; ++i) {
            s[i] = a * d[i];
            y[i] = gt[i] - g[i];
        }
        const double sy = vdot(n, s, y);
        if (sy > 1e-12 * sqrt(vdot(n, s, s) * vdot(n, y, y))) {
            rho[head] = 1.0 / sy;
            head = (head + 1) % m;
            if (stored < m) ++stored;
        }
        memcpy(x, xt, n * sizeof(double));
        memcpy(g, gt, n * sizeof(double));
        f = fn;
        if (trace) trace[it + 1] = f;
        if (sqrt(vdot(n, g, g)) <= grad_tol * g0) { status = 0; ++it; break; }
    }
    if (f_out) *f_out = f;
    if (iters_out) *iters_out = it;
    if (evals_out) *evals_out = c.evals;
    free(g); free(d); free(xt); free(gt); free(S); free(Y); free(rho); free(alpha);
    return status;
}

/* Pin helpers: a convex quadratic 1/2 x^T A x - b^T x (A dense, n x n) and the
 * extended Rosenbrock function. */
typedef struct { int64_t n; const double* A; const double* b; } quad_ctx;

static double quad_fg(void* p, const double* x, double* g) {
    const quad_ctx* q = p;
    double f = 0.0;
    for (int64_t i = 0; i < q->n; ++i) {
        double ax = 0.0;
        for (int64_t j = 0; j < q->n; ++j) ax += q->A[i * q->n + j] * x[j];
        g[i] = ax - q->b[i];
        f += 0.5 * x[i] * ax - q->b[i] * x[i];
    }
    return f;
}

int orc_lbfgs_quadratic(int64_t n, const double* A, const double* b, double* x, int m, int max_iter,
                        double grad_tol, double* f_out, int* iters, int* evals) {
    quad_ctx q = {n, A, b};
    return orc_lbfgs(n, x, quad_fg, &q, m, max_iter, grad_tol, f_out, iters, evals, NULL);
}

static double rosen_fg(void* p, const double* x, double* g) {
    const int64_t n = *(const int64_t*)p;
    double f = 0.0;
    for (int64_t i = 0; i < n; ++i) g[i] = 0.0;
    for (int64_t i = 0; i + 1 < n; ++i) {
        const double a = x[i + 1] - x[i] * x[i], b = 1.0 - x[i];
        f += 100.0 * a * a + b * b;
        g[i] += -400.0 * x[i] * a - 2.0 * b;
        g[i + 1] += 200.0 * a;
    }
    return f;
}

int orc_lbfgs_rosenbrock(int64_t n, double* x, int m, int max_iter, double grad_tol, double* f_out, int* iters,
                         int* evals) {
    return orc_lbfgs(n, x, rosen_fg, &n, m, max_iter, grad_tol, f_out, iters, evals, NULL);
}

/* register: minimise the Eq. 3 loss over p0 from p0_inout (the outer
 * optimisation of Algorithm 1).  Returns the orc_lbfgs status. */
typedef struct {
    int64_t n;
    int T;
    double sigma, lambda;
    const double* q0;
    const double* target;
    int integ, h_at_end, dim;
} reg_ctx;

static double reg_fg(void* p, const double* x, double* g) {
    const reg_ctx* r = p;
    if (r->integ == 0 && r->h_at_end == 0 && r->dim == 3)
        return orc_shoot_gradient(r->n, r->T, r->sigma, r->lambda, r->q0, x, r->target, g, NULL, NULL, NULL, NULL);
    return orc_shoot_gradient_v(r->dim, r->n, r->T, r->sigma, r->lambda, r->integ, r->h_at_end, r->q0, x, r->target,
                                g, NULL, NULL, NULL, NULL);
}

int orc_register(int64_t n, int T, double sigma, double lambda, int m, int max_iter, double grad_tol,
                 const double* q0, const double* target, double* p0, double* loss, int* iters, int* evals,
                 double* trace) {
    reg_ctx r = {n, T, sigma, lambda, q0, target, 0, 0, 3};
    return orc_lbfgs(3 * n, p0, reg_fg, &r, m, max_iter, grad_tol, loss, iters, evals, trace);
}

/* register with a variant of the discretisation (dim, integ, h_at_end as in
 * orc_shoot_gradient_v). */
int orc_register_v(int dim, int64_t n, int T, double sigma, double lambda, int integ, int h_at_end, int m,
                   int max_iter, double grad_tol, const double* q0, const double* target, double* p0, double* loss,
                   int* iters, int* evals, double* trace) {
    reg_ctx r = {n, T, sigma, lambda, q0, target, integ, h_at_end, dim};
    return orc_lbfgs(dim * n, p0, reg_fg, &r, m, max_iter, grad_tol, loss, iters, evals, trace);
}
