/*
 * FP64 CPU oracle for the imaging side of 4D SlingBAG (arXiv 2412.03898):
 * the UBP comparison reconstruction, the point-cloud -> voxel conversion and
 * the SSIM of maximum amplitude projections (Sec. 3.1-3.2, Tab. 1).
 *
 * TEST INFRASTRUCTURE ONLY, like pa_oracle.c: only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg may
 * load it; it shares nothing with the CUDA library.
 *
 * The paper names these methods but prints none of them; each routine below
 * is the textbook definition, written as a plain double-precision loop nest.
 *
 * Voxel grids are [nz][ny][nx], voxel (ix, iy, iz) centred at
 * origin + h * (ix, iy, iz).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1

static void set_threads_img(int32_t nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* Universal back-projection, filtering step: for every sensor trace p(t_k),
 * t_k = t0 + k/fs, the back-projection term b(t) = 2 p(t) - 2 t dp/dt, with
 * dp/dt by central differences (one-sided at the first and last sample). */
int32_t oracle_ubp_filter(int32_t ns, int32_t T, double fs, double t0, const double *p, double *b) {
    if (ns < 0 || T < 2 || !(fs > 0.0)) return ORC_ERR_ARG;
    for (int32_t s = 0; s < ns; ++s) {
        const double *ps = p + (int64_t)s * T;
        double *bs = b + (int64_t)s * T;
        for (int32_t k = 0; k < T; ++k) {
            double dpdt;
            if (k == 0)
                dpdt = (ps[1] - ps[0]) * fs;
            else if (k == T - 1)
                dpdt = (ps[T - 1] - ps[T - 2]) * fs;
            else
                dpdt = (ps[k + 1] - ps[k - 1]) * fs / 2.0;
            double t = t0 + k / fs;
            bs[k] = 2.0 * ps[k] - 2.0 * t * dpdt;
        }
    }
    return ORC_OK;
}

/* Universal back-projection, summation step: for every voxel centre r,
 *     p0(r) = sum_s w_s b_s(|r - r_s| / c) / sum_s w_s,
 * w_s = cos(theta_s) / |r - r_s|^2 the solid angle of sensor s seen from r
 * (theta_s between the sensor's inward normal, pointing from r_s to the
 * array centre, and r - r_s); sensors with cos(theta_s) <= 0 are left out.
 * b_s(t) is linearly interpolated at the fractional sample (t - t0) fs and is
 * 0 outside [0, T - 1].  A voxel no sensor faces gets 0. */
int32_t oracle_ubp(int32_t ns, int32_t T, const double *sens, const double *center, double c, double fs,
                   double t0, const double *b, const double *origin, double h, int32_t nx, int32_t ny,
                   int32_t nz, double *vol, int32_t nthreads) {
    if (ns < 0 || T < 2 || !(c > 0.0) || !(fs > 0.0) || !(h > 0.0) || nx < 0 || ny < 0 || nz < 0)
        return ORC_ERR_ARG;
    set_threads_img(nthreads);
    const int64_t nvox = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < nvox; ++v) {
        const int64_t ix = v % nx, iy = (v / nx) % ny, iz = v / ((int64_t)nx * ny);
        const double rx = origin[0] + h * ix, ry = origin[1] + h * iy, rz = origin[2] + h * iz;
        double num = 0.0, den = 0.0;
        for (int32_t s = 0; s < ns; ++s) {
            const double sx = sens[s], sy = sens[ns + s], sz = sens[2 * ns + s];
            const double dx = rx - sx, dy = ry - sy, dz = rz - sz;
            const double d = sqrt(dx * dx + dy * dy + dz * dz);
            const double nxs = center[0] - sx, nys = center[1] - sy, nzs = center[2] - sz;
            const double nn = sqrt(nxs * nxs + nys * nys + nzs * nzs);
            if (!(d > 0.0) || !(nn > 0.0)) continue;
            const double cosv = (nxs * dx + nys * dy + nzs * dz) / (nn * d);
            if (!(cosv > 0.0)) continue;
            const double w = cosv / (d * d);
            const double f = (d / c - t0) * fs;
            const double fl = floor(f);
            double val = 0.0;
            if (fl >= 0.0 && fl + 1.0 <= (double)(T - 1)) {
                const int64_t i = (int64_t)fl;
                const double fr = f - fl;
                const double *bs = b + (int64_t)s * T;
                val = bs[i] + fr * (bs[i + 1] - bs[i]);
            }
            num += w * val;
            den += w;
        }
        vol[v] = den > 0.0 ? num / den : 0.0;
    }
    return ORC_OK;
}

/* Point cloud -> voxel grid (the conversion SlingBAG ends with, Sec. 2.1):
 *     v(r) = sum_b p_b exp(-|r - mu_b|^2 / (2 a_b^2))  over |r - mu_b| <= kappa a_b,
 * state [5][n] = (x, y, z, a, p); balls with a <= 0 or p == 0 add nothing. */
int32_t oracle_splat(int64_t n, const double *state, double kappa, const double *origin, double h,
                     int32_t nx, int32_t ny, int32_t nz, double *vol, int32_t nthreads) {
    if (n < 0 || !(h > 0.0) || !(kappa > 0.0) || nx < 0 || ny < 0 || nz < 0) return ORC_ERR_ARG;
    set_threads_img(nthreads);
    const int64_t nvox = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < nvox; ++v) {
        const int64_t ix = v % nx, iy = (v / nx) % ny, iz = v / ((int64_t)nx * ny);
        const double rx = origin[0] + h * ix, ry = origin[1] + h * iy, rz = origin[2] + h * iz;
        double acc = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            const double a = state[3 * n + i], p = state[4 * n + i];
            if (!(a > 0.0) || p == 0.0) continue;
            const double dx = rx - state[i], dy = ry - state[n + i], dz = rz - state[2 * n + i];
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > (kappa * a) * (kappa * a)) continue;
            acc += p * exp(-r2 / (2.0 * a * a));
        }
        vol[v] = acc;
    }
    return ORC_OK;
}

/* Structural similarity (Wang, Bovik, Sheikh, Simoncelli 2004) of two images
 * [H][W]: local statistics under an 11 x 11 Gaussian window (sigma 1.5,
 * weights normalised to sum 1) at every position where the window fits,
 *     SSIM = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2)),
 * C1 = (0.01 L)^2, C2 = (0.03 L)^2, L the dynamic range; returns the mean over
 * those positions in *out (and the map in `map` [(H-10)][(W-10)] if not NULL). */
int32_t oracle_ssim(int32_t H, int32_t W, const double *x, const double *y, double L, double *map, double *out) {
    if (H < 11 || W < 11 || !(L > 0.0)) return ORC_ERR_ARG;
    double g[11][11], gs = 0.0;
    for (int i = 0; i < 11; ++i)
        for (int j = 0; j < 11; ++j) {
            const double di = i - 5, dj = j - 5;
            g[i][j] = exp(-(di * di + dj * dj) / (2.0 * 1.5 * 1.5));
            gs += g[i][j];
        }
    for (int i = 0; i < 11; ++i)
        for (int j = 0; j < 11; ++j) g[i][j] /= gs;
    const double C1 = (0.01 * L) * (0.01 * L), C2 = (0.03 * L) * (0.03 * L);
    const int32_t oh = H - 10, ow = W - 10;
    double total = 0.0;
    for (int32_t r = 0; r < oh; ++r)
        for (int32_t q = 0; q < ow; ++q) {
            double mx = 0, my = 0, xx = 0, yy = 0, xy = 0;
            for (int i = 0; i < 11; ++i)
                for (int j = 0; j < 11; ++j) {
                    const double a = x[(int64_t)(r + i) * W + q + j], b = y[(int64_t)(r + i) * W + q + j];
                    mx += g[i][j] * a;
                    my += g[i][j] * b;
                    xx += g[i][j] * a * a;
                    yy += g[i][j] * b * b;
                    xy += g[i][j] * a * b;
                }
            const double sx = xx - mx * mx, sy = yy - my * my, sxy = xy - mx * my;
            const double s = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sx + sy + C2));
            if (map) map[(int64_t)r * ow + q] = s;
            total += s;
        }
    *out = total / ((double)oh * ow);
    return ORC_OK;
}
