/*
 * FP64 CPU oracle for the 4D SlingBAG hot path (arXiv 2412.03898).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA library under
 * paper_2412_03898_gb300/csrc, and the product path never calls it.
 *
 * Every routine is a plain loop nest in double precision that follows the
 * definition it cites; there is no blocking, fusion or reordering beyond it.
 * Inputs arrive as double arrays (the callers promote fp32 inputs exactly).
 *
 * Channel order of a ball state: 0 = x, 1 = y, 2 = z (centre mu, Sec. 2.1),
 * 3 = a (standard deviation "size" a0), 4 = p (peak initial pressure p0).
 *
 * Radiator.  The paper cites SlingBAG's "differentiable rapid radiator"
 * (Sec. 2.2, last paragraph) without printing its formula.  The oracle uses
 * the exact solution of the 3D wave equation for a Gaussian initial pressure
 * p*exp(-|x-mu|^2/(2a^2)) with zero initial velocity (Poisson's spherical-mean
 * formula).  Observed at distance R from the centre it is
 *     P(R,t) = p/(2R) [ (R-ct) e^{-(R-ct)^2/(2a^2)} + (R+ct) e^{-(R+ct)^2/(2a^2)} ]
 * (oracle_pressure_full).  The forward projection keeps the first (outgoing)
 * term only; the second is below (R/a) e^{-R^2/(2a^2)} relative to the peak,
 * i.e. zero in double precision for R/a > 40 and far below any tolerance for
 * R/a >= 10.  Each ball contributes on the closed window |R - c t_k| <= kappa*a
 * with t_k = t0 + k/fs, k = 0..T-1.  A sensor with R <= kappa*a lies inside
 * the ball's support: that pair is skipped and counted as a domain error.
 * Balls with a <= 0 or p == 0 contribute nothing.
 *
 * Parity pins (tests/test_oracle_*.py): wave-equation residual, initial value
 * and zero initial velocity of oracle_pressure_full; brute-force voxelised
 * spherical-mean quadrature of the initial pressure; antisymmetry about R/c;
 * linearity in p; superposition; joint rigid-motion invariance; the
 * uniform-ball N-pulse; finite differences of every gradient group; the
 * adjoint dot-product identity; the special cases of Eq. 1-2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_DOMAIN 2

#define ORC_PROFILE_GAUSS 0
#define ORC_PROFILE_UNIFORM 1

static void set_threads(int32_t nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int32_t oracle_max_threads(void) {
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------
 * Eq. 2: one Gaussian basis of the deformation function,
 *   b_n(t) = exp(-(t - theta_n)^2 / (2 sigma_n^2)).
 * ------------------------------------------------------------------- */
static double gbasis(double t, double theta, double sigma) {
    double d = t - theta;
    return exp(-(d * d) / (2.0 * sigma * sigma));
}

/* Eq. 2: H_N(t) = sum_n omega_n b_n(t) for one ball and one channel.
 * omega/theta/sigma point at element (ch, 0, b) of a [5][nb][n] array;
 * consecutive basis functions are n elements apart. */
static double deform_h(double t, const double *omega, const double *theta,
                       const double *sigma, int32_t nb, int64_t n) {
    double h = 0.0;
    for (int32_t k = 0; k < nb; ++k)
        h += omega[(int64_t)k * n] * gbasis(t, theta[(int64_t)k * n], sigma[(int64_t)k * n]);
    return h;
}

/* Eq. 1: a0(t) = a0 (1 + H^a(t)), p0(t) = p0 (1 + H^p(t)),
 * mu(t) = mu (1 + H^mu(t)), with one independent H per channel (x, y, z, a, p).
 *   canon [5][n]; omega, theta, sigma [5][nb][n]; t [nf]; out [nf][5][n]. */
int32_t oracle_deform(int64_t n, int32_t nb, const double *canon,
                      const double *omega, const double *theta, const double *sigma,
                      int32_t nf, const double *t, double *out) {
    if (n < 0 || nb < 0 || nf < 0) return ORC_ERR_ARG;
    for (int64_t i = 0; i < 5LL * nb * n; ++i)
        if (!(sigma[i] > 0.0)) return ORC_ERR_DOMAIN;
    for (int32_t f = 0; f < nf; ++f)
        for (int ch = 0; ch < 5; ++ch)
            for (int64_t b = 0; b < n; ++b) {
                int64_t o = (int64_t)ch * nb * n + b;
                double h = deform_h(t[f], omega + o, theta + o, sigma + o, nb, n);
                out[((int64_t)f * 5 + ch) * n + b] = canon[(int64_t)ch * n + b] * (1.0 + h);
            }
    return ORC_OK;
}

/* Full Poisson solution for one Gaussian ball (both terms), at distance R and
 * travelled distance ct = c*t.  Used by the tests that pin the radiator to the
 * wave equation and to its initial condition. */
double oracle_pressure_full(double p, double a, double R, double ct) {
    double u = R - ct, v = R + ct, s2 = 2.0 * a * a;
    return p / (2.0 * R) * (u * exp(-u * u / s2) + v * exp(-v * v / s2));
}

/* Outgoing term of one ball at tau = R - c t (the radiated pulse). */
static double pulse(int32_t profile, double p, double a, double R, double tau) {
    if (profile == ORC_PROFILE_UNIFORM)
        return p * tau / (2.0 * R);  /* uniform ball: the textbook N-pulse */
    return p / (2.0 * R) * tau * exp(-tau * tau / (2.0 * a * a));
}

/* Closed sample window of one (ball, sensor) pair: every k in [0, T) with
 * |R - c (t0 + k/fs)| <= h.  Returns 0 when the window is empty. */
static int window(double R, double h, double c, double fs, double t0, int32_t T,
                  int64_t *klo, int64_t *khi) {
    double lo = ceil(((R - h) / c - t0) * fs);
    double hi = floor(((R + h) / c - t0) * fs);
    if (lo < 0.0) lo = 0.0;
    if (hi > (double)(T - 1)) hi = (double)(T - 1);
    if (hi < lo) return 0;
    *klo = (int64_t)lo;
    *khi = (int64_t)hi;
    return 1;
}

/* Forward projection (Sec. 2.2, last paragraph): for every frame f, sensor s
 * and sample k,
 *   y[f][s][k] = sum over balls b of the pulse of b at tau = R_bs - c t_k,
 * summed over b in index order.
 *   state [nf][5][n]; sens [3][ns]; traces [nf][ns][T] (overwritten).
 * n_contrib (optional): number of (f, s, b, k) terms summed.
 * n_domain (optional): number of pairs skipped because R <= h. */
int32_t oracle_forward(int32_t nf, int64_t n, const double *state, int32_t ns,
                       const double *sens, double c, double fs, double t0, int32_t T,
                       double kappa, int32_t profile, double *traces,
                       int64_t *n_contrib, int64_t *n_domain, int32_t nthreads) {
    if (nf < 0 || n < 0 || ns < 0 || T < 0 || !(c > 0.0) || !(fs > 0.0)) return ORC_ERR_ARG;
    set_threads(nthreads);
    int64_t total = 0, bad = 0;
    const int64_t rows = (int64_t)nf * ns;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total, bad)
    for (int64_t r = 0; r < rows; ++r) {
        int32_t f = (int32_t)(r / ns), s = (int32_t)(r % ns);
        const double *st = state + (int64_t)f * 5 * n;
        double *y = traces + r * T;
        for (int32_t k = 0; k < T; ++k) y[k] = 0.0;
        double sx = sens[s], sy = sens[ns + s], sz = sens[2 * ns + s];
        for (int64_t b = 0; b < n; ++b) {
            double x = st[b], yy = st[n + b], z = st[2 * n + b];
            double a = st[3 * n + b], p = st[4 * n + b];
            if (!(a > 0.0) || p == 0.0) continue;
            double dx = x - sx, dy = yy - sy, dz = z - sz;
            double R = sqrt(dx * dx + dy * dy + dz * dz);
            double h = (profile == ORC_PROFILE_UNIFORM) ? a : kappa * a;
            if (!(R > h)) { ++bad; continue; }
            int64_t klo, khi;
            if (!window(R, h, c, fs, t0, T, &klo, &khi)) continue;
            for (int64_t k = klo; k <= khi; ++k) {
                double tk = t0 + (double)k / fs;
                y[k] += pulse(profile, p, a, R, R - c * tk);
            }
            total += khi - klo + 1;
        }
    }
    if (n_contrib) *n_contrib = total;
    if (n_domain) *n_domain = bad;
    return bad ? ORC_ERR_DOMAIN : ORC_OK;
}

/* L2 data-fidelity loss per frame (Sec. 2.2, last paragraph):
 *   loss[f] = sum_{s,k} (pred - meas)^2, summed in index order. */
int32_t oracle_loss(int32_t nf, int64_t per_frame, const double *pred,
                    const double *meas, double *loss) {
    for (int32_t f = 0; f < nf; ++f) {
        double acc = 0.0;
        for (int64_t i = 0; i < per_frame; ++i) {
            double d = pred[(int64_t)f * per_frame + i] - meas[(int64_t)f * per_frame + i];
            acc += d * d;
        }
        loss[f] = acc;
    }
    return ORC_OK;
}

/* Adjoint of the forward projection with respect to the per-frame ball
 * states (Gaussian profile).  Given g = dL/dy [nf][ns][T], returns
 *   grad [nf][5][n] = dL/d(x, y, z, a, p)
 * from the analytic derivatives of v = A tau E, A = p/(2R),
 * E = exp(-tau^2/(2a^2)), tau = R - c t_k:
 *   dv/dp = tau E / (2R)
 *   dv/da = v tau^2 / a^3
 *   dv/dR = -v/R + A E (1 - tau^2/a^2),   dR/dmu = (mu - x_s)/R.
 * Window edges are held fixed (the truncated sum is piecewise smooth).
 * Balls with a <= 0 or p == 0 and pairs with R <= kappa*a get no gradient. */
int32_t oracle_adjoint_state(int32_t nf, int64_t n, const double *state, int32_t ns,
                             const double *sens, double c, double fs, double t0,
                             int32_t T, double kappa, const double *g, double *grad,
                             int32_t nthreads) {
    if (nf < 0 || n < 0 || ns < 0 || T < 0 || !(c > 0.0) || !(fs > 0.0)) return ORC_ERR_ARG;
    set_threads(nthreads);
    int64_t bad = 0;
    const int64_t items = (int64_t)nf * n;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : bad)
    for (int64_t it = 0; it < items; ++it) {
        int32_t f = (int32_t)(it / n);
        int64_t b = it % n;
        const double *st = state + (int64_t)f * 5 * n;
        double *gr = grad + (int64_t)f * 5 * n;
        double x = st[b], yy = st[n + b], z = st[2 * n + b];
        double a = st[3 * n + b], p = st[4 * n + b];
        double gx = 0, gy = 0, gz = 0, ga = 0, gp = 0;
        if (a > 0.0 && p != 0.0) {
            for (int32_t s = 0; s < ns; ++s) {
                double sx = sens[s], sy = sens[ns + s], sz = sens[2 * ns + s];
                double dx = x - sx, dy = yy - sy, dz = z - sz;
                double R = sqrt(dx * dx + dy * dy + dz * dz);
                double h = kappa * a;
                if (!(R > h)) { ++bad; continue; }
                int64_t klo, khi;
                if (!window(R, h, c, fs, t0, T, &klo, &khi)) continue;
                const double *gs = g + ((int64_t)f * ns + s) * T;
                double A = p / (2.0 * R);
                double dR = 0.0;
                for (int64_t k = klo; k <= khi; ++k) {
                    double tau = R - c * (t0 + (double)k / fs);
                    double E = exp(-tau * tau / (2.0 * a * a));
                    double v = A * tau * E;
                    gp += gs[k] * tau * E / (2.0 * R);
                    ga += gs[k] * v * tau * tau / (a * a * a);
                    dR += gs[k] * (-v / R + A * E * (1.0 - tau * tau / (a * a)));
                }
                gx += dR * dx / R;
                gy += dR * dy / R;
                gz += dR * dz / R;
            }
        }
        gr[b] = gx;
        gr[n + b] = gy;
        gr[2 * n + b] = gz;
        gr[3 * n + b] = ga;
        gr[4 * n + b] = gp;
    }
    return bad ? ORC_ERR_DOMAIN : ORC_OK;
}

/* Chain rule of Eq. 1-2 from per-frame state gradients to the canonical
 * attributes and the deformation parameters ("fully learnable", Sec. 2.2):
 * for channel value q(t) = q0 (1 + sum_n omega_n b_n(t)),
 *   dq/dq0      = 1 + H(t)
 *   dq/domega_n = q0 b_n(t)
 *   dq/dtheta_n = q0 omega_n b_n(t) (t - theta_n) / sigma_n^2
 *   dq/dsigma_n = q0 omega_n b_n(t) (t - theta_n)^2 / sigma_n^3
 * summed over frames.  gstate [nf][5][n]; outputs g_canon [5][n] and
 * g_omega, g_theta, g_sigma [5][nb][n] (overwritten). */
int32_t oracle_deform_backward(int64_t n, int32_t nb, const double *canon,
                               const double *omega, const double *theta,
                               const double *sigma, int32_t nf, const double *t,
                               const double *gstate, double *g_canon, double *g_omega,
                               double *g_theta, double *g_sigma) {
    for (int ch = 0; ch < 5; ++ch)
        for (int64_t b = 0; b < n; ++b) {
            int64_t o = (int64_t)ch * nb * n + b;
            double q0 = canon[(int64_t)ch * n + b];
            double gc = 0.0;
            for (int32_t k = 0; k < nb; ++k) {
                int64_t i = o + (int64_t)k * n;
                g_omega[i] = 0.0;
                g_theta[i] = 0.0;
                g_sigma[i] = 0.0;
            }
            for (int32_t f = 0; f < nf; ++f) {
                double gq = gstate[((int64_t)f * 5 + ch) * n + b];
                double h = deform_h(t[f], omega + o, theta + o, sigma + o, nb, n);
                gc += gq * (1.0 + h);
                for (int32_t k = 0; k < nb; ++k) {
                    int64_t i = o + (int64_t)k * n;
                    double bn = gbasis(t[f], theta[i], sigma[i]);
                    double d = t[f] - theta[i];
                    double sg = sigma[i];
                    g_omega[i] += gq * q0 * bn;
                    g_theta[i] += gq * q0 * omega[i] * bn * d / (sg * sg);
                    g_sigma[i] += gq * q0 * omega[i] * bn * d * d / (sg * sg * sg);
                }
            }
            g_canon[(int64_t)ch * n + b] = gc;
        }
    return ORC_OK;
}

/* 4D adjoint in the paper's order: deform every frame (Eq. 1-2), take the
 * state adjoint of the forward projection per frame, then apply the chain
 * rule of Eq. 1-2 back to the canonical cloud and deformation parameters.
 * Work buffers are allocated here (nf * 5 * n doubles, twice). */
int32_t oracle_adjoint_4d(int64_t n, int32_t nb, const double *canon,
                          const double *omega, const double *theta, const double *sigma,
                          int32_t nf, const double *t, int32_t ns, const double *sens,
                          double c, double fs, double t0, int32_t T, double kappa,
                          const double *g, double *g_canon, double *g_omega,
                          double *g_theta, double *g_sigma, int32_t nthreads) {
    size_t sz = (size_t)nf * 5 * (size_t)n;
    double *state = (double *)malloc(sz * sizeof(double) + 1);
    double *gstate = (double *)malloc(sz * sizeof(double) + 1);
    if (!state || !gstate) { free(state); free(gstate); return ORC_ERR_ARG; }
    int32_t rc = oracle_deform(n, nb, canon, omega, theta, sigma, nf, t, state);
    if (rc == ORC_OK) {
        rc = oracle_adjoint_state(nf, n, state, ns, sens, c, fs, t0, T, kappa, g, gstate, nthreads);
        oracle_deform_backward(n, nb, canon, omega, theta, sigma, nf, t, gstate,
                               g_canon, g_omega, g_theta, g_sigma);
    }
    free(state);
    free(gstate);
    return rc;
}
