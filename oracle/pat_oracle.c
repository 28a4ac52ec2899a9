/*
 * pat_oracle.c — plain FP64 CPU oracle (test infrastructure only; see
 * pat_oracle.h for the discretisation and for who may use this file).
 *
 * Everything here is written for a reader checking it against the model by
 * eye: plain loops, FP64 throughout, no blocking, no fusion, no reordering
 * beyond the definitions.  OpenMP (when the compiler offers it) only splits
 * the outer loop over detectors; results do not depend on the thread count
 * except through the order of the final FP64 sum in the adjoint.
 */
#include "pat_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int orc_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------------ */
/* Abel integral with the midpoint time derivative.                          */
/*                                                                           */
/* The 2D Poisson formula (solution of Eq. (1) with zero initial velocity)   */
/* reads p(t) = dQ/dt with Q(t) = int_0^t r M(r) / sqrt(t^2 - r^2) dr.       */
/* In units of Delta (r = rho Delta, t = tau Delta) and with M piecewise     */
/* linear on the integer nodes (hat functions), Q(t) = Delta sum_m M_m       */
/* w_m(tau) with w_m(tau) = int_0^tau hat_m(rho) rho / sqrt(tau^2-rho^2).    */
/* On a segment [a, b] inside [s, s+1] the two hats are (s+1-rho) and        */
/* (rho - s); with                                                           */
/*   I1 = int_a^b rho / S,   I2 = int_a^b rho^2 / S,   S = sqrt(tau^2-rho^2) */
/* the segment adds (s+1) I1 - I2 to w_s and I2 - s I1 to w_{s+1}.           */
/* ------------------------------------------------------------------------ */

/* x - sin(x), without cancellation for small x (Taylor series). */
static double x_minus_sin(double x)
{
    if (fabs(x) < 1.0) {
        const double x2 = x * x;
        double term = x * x2 / 6.0; /* x^3 / 3! */
        double sum = 0.0;
        double sign = 1.0;
        int n = 3;
        for (int i = 0; i < 40; ++i) {
            sum += sign * term;
            term *= x2 / (double)((n + 1) * (n + 2));
            n += 2;
            sign = -sign;
            if (fabs(term) < 1e-20 * fabs(sum)) break;
        }
        return sum;
    }
    return x - sin(x);
}

/* G(rho) = int_0^rho x^2 / sqrt(tau^2 - x^2) dx
 *        = (tau^2 / 2) (theta - sin(theta) cos(theta)),  theta = asin(rho/tau)
 *        = (tau^2 / 4) (2 theta - sin(2 theta)). */
static double abel_G(double rho, double tau)
{
    double x = rho / tau;
    if (x > 1.0) x = 1.0;
    return 0.25 * tau * tau * x_minus_sin(2.0 * asin(x));
}

void orc_abel_weights(double tau, int n_r, double* w)
{
    for (int m = 0; m < n_r; ++m) w[m] = 0.0;
    for (int s = 0; s + 1 < n_r && (double)s < tau; ++s) {
        const double a = (double)s;
        const double b = ((double)(s + 1) < tau) ? (double)(s + 1) : tau;
        /* sqrt((tau - r)(tau + r)) avoids the cancellation of tau^2 - r^2 */
        const double Sa = sqrt((tau - a) * (tau + a));
        const double Sb = (b < tau) ? sqrt((tau - b) * (tau + b)) : 0.0;
        /* I1 = Sa - Sb, rationalised to avoid cancellation */
        const double I1 = (b * b - a * a) / (Sa + Sb);
        const double I2 = abel_G(b, tau) - abel_G(a, tau);
        w[s] += (double)(s + 1) * I1 - I2;
        w[s + 1] += I2 - (double)s * I1;
    }
}

void orc_abel_matrix(int n_t, double* P)
{
    const int n_r = n_t + 2;
    double* wp = (double*)malloc(sizeof(double) * n_r);
    double* wm = (double*)malloc(sizeof(double) * n_r);
    for (int k = 1; k <= n_t; ++k) {
        /* p(t_k) ~ (Q(t_k + Delta/2) - Q(t_k - Delta/2)) / Delta; the Delta
         * factor of Q cancels the 1/Delta of the difference. */
        orc_abel_weights((double)k + 0.5, n_r, wp);
        orc_abel_weights((double)k - 0.5, n_r, wm);
        for (int m = 0; m < n_r; ++m) P[(size_t)(k - 1) * n_r + m] = wp[m] - wm[m];
    }
    free(wp);
    free(wm);
}

/* ------------------------------------------------------------------------ */
/* Circular means                                                            */
/* ------------------------------------------------------------------------ */

double orc_bilinear(const double* f, int n, double sx, double sy)
{
    const double h = 2.0 / (double)n;
    /* pixel-index coordinates: pixel ix has its centre at u = ix */
    const double u = (sx + 1.0) / h - 0.5;
    const double v = (sy + 1.0) / h - 0.5;
    if (!(u > -2.0 && u < (double)n + 1.0 && v > -2.0 && v < (double)n + 1.0)) return 0.0;
    const double fu = floor(u), fv = floor(v);
    const int i0 = (int)fu, j0 = (int)fv;
    const double a = u - fu, b = v - fv;
    const int ci[4] = {i0, i0 + 1, i0, i0 + 1};
    const int cj[4] = {j0, j0, j0 + 1, j0 + 1};
    const double cw[4] = {(1.0 - a) * (1.0 - b), a * (1.0 - b), (1.0 - a) * b, a * b};
    double val = 0.0;
    for (int c = 0; c < 4; ++c) {
        if (ci[c] < 0 || ci[c] >= n || cj[c] < 0 || cj[c] >= n) continue; /* zero outside */
        val += cw[c] * f[(size_t)cj[c] * n + ci[c]];
    }
    return val;
}

double orc_circle_mean(const double* f, int n, double cx, double cy, double r, int K)
{
    const double two_pi = 2.0 * acos(-1.0);
    double acc = 0.0;
    for (int q = 0; q < K; ++q) {
        const double phi = two_pi * (double)q / (double)K;
        acc += orc_bilinear(f, n, cx + r * cos(phi), cy + r * sin(phi));
    }
    return acc / (double)K;
}

void orc_detectors(const orc_geom* g, double* xy)
{
    for (int j = 0; j < g->n_det; ++j) {
        const double theta = g->arc_start + ((double)j + 0.5) * g->arc_span / (double)g->n_det;
        xy[2 * j] = cos(theta);
        xy[2 * j + 1] = sin(theta);
    }
}

void orc_circular_means(const orc_geom* g, const double* f, double* M)
{
    const int n_r = g->n_t + 2;
    const double dt = g->t_max / (double)g->n_t;
    double* xy = (double*)malloc(sizeof(double) * 2 * g->n_det);
    orc_detectors(g, xy);
#pragma omp parallel for num_threads(g_threads) schedule(dynamic)
    for (int j = 0; j < g->n_det; ++j)
        for (int m = 0; m < n_r; ++m)
            M[(size_t)j * n_r + m] =
                orc_circle_mean(f, g->n, xy[2 * j], xy[2 * j + 1], (double)m * dt, g->n_angles);
    free(xy);
}

void orc_forward(const orc_geom* g, const double* f, double* out)
{
    const int n_r = g->n_t + 2, n_t = g->n_t;
    double* M = (double*)malloc(sizeof(double) * (size_t)g->n_det * n_r);
    double* P = (double*)malloc(sizeof(double) * (size_t)n_t * n_r);
    orc_circular_means(g, f, M);
    orc_abel_matrix(n_t, P);
#pragma omp parallel for num_threads(g_threads)
    for (int j = 0; j < g->n_det; ++j)
        for (int k = 0; k < n_t; ++k) {
            double acc = 0.0;
            for (int m = 0; m < n_r; ++m) acc += P[(size_t)k * n_r + m] * M[(size_t)j * n_r + m];
            out[(size_t)j * n_t + k] = acc;
        }
    free(M);
    free(P);
}

/* ------------------------------------------------------------------------ */
/* Adjoint: the literal transpose of the two stages above.                   */
/* ------------------------------------------------------------------------ */

void orc_adjoint_time(const orc_geom* g, const double* gbar, double* Mbar)
{
    const int n_r = g->n_t + 2, n_t = g->n_t;
    double* P = (double*)malloc(sizeof(double) * (size_t)n_t * n_r);
    orc_abel_matrix(n_t, P);
    for (int j = 0; j < g->n_det; ++j)
        for (int m = 0; m < n_r; ++m) {
            double acc = 0.0;
            for (int k = 0; k < n_t; ++k) acc += P[(size_t)k * n_r + m] * gbar[(size_t)j * n_t + k];
            Mbar[(size_t)j * n_r + m] = acc;
        }
    free(P);
}

/* Scatter of one sample's bilinear weights times val into img (N x N). */
static void scatter_sample(double* img, int n, double sx, double sy, double val)
{
    const double h = 2.0 / (double)n;
    const double u = (sx + 1.0) / h - 0.5;
    const double v = (sy + 1.0) / h - 0.5;
    if (!(u > -2.0 && u < (double)n + 1.0 && v > -2.0 && v < (double)n + 1.0)) return;
    const double fu = floor(u), fv = floor(v);
    const int i0 = (int)fu, j0 = (int)fv;
    const double a = u - fu, b = v - fv;
    const int ci[4] = {i0, i0 + 1, i0, i0 + 1};
    const int cj[4] = {j0, j0, j0 + 1, j0 + 1};
    const double cw[4] = {(1.0 - a) * (1.0 - b), a * (1.0 - b), (1.0 - a) * b, a * b};
    for (int c = 0; c < 4; ++c) {
        if (ci[c] < 0 || ci[c] >= n || cj[c] < 0 || cj[c] >= n) continue;
        img[(size_t)cj[c] * n + ci[c]] += cw[c] * val;
    }
}

void orc_adjoint_means(const orc_geom* g, const double* Mbar, double* fbar)
{
    const int n = g->n, n_r = g->n_t + 2, K = g->n_angles;
    const double dt = g->t_max / (double)g->n_t;
    const double two_pi = 2.0 * acos(-1.0);
    const size_t npix = (size_t)n * n;
    double* xy = (double*)malloc(sizeof(double) * 2 * g->n_det);
    orc_detectors(g, xy);
    const int nt = g_threads;
    double* priv = (double*)calloc((size_t)nt * npix, sizeof(double));
#pragma omp parallel for num_threads(nt) schedule(dynamic)
    for (int j = 0; j < g->n_det; ++j) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* img = priv + (size_t)tid * npix;
        for (int m = 0; m < n_r; ++m) {
            const double val = Mbar[(size_t)j * n_r + m] / (double)K;
            const double r = (double)m * dt;
            for (int q = 0; q < K; ++q) {
                const double phi = two_pi * (double)q / (double)K;
                scatter_sample(img, n, xy[2 * j] + r * cos(phi), xy[2 * j + 1] + r * sin(phi), val);
            }
        }
    }
    for (size_t p = 0; p < npix; ++p) {
        double acc = 0.0;
        for (int t = 0; t < nt; ++t) acc += priv[(size_t)t * npix + p];
        fbar[p] = acc;
    }
    free(priv);
    free(xy);
}

void orc_adjoint(const orc_geom* g, const double* gbar, double* fbar)
{
    const int n_r = g->n_t + 2;
    double* Mbar = (double*)malloc(sizeof(double) * (size_t)g->n_det * n_r);
    orc_adjoint_time(g, gbar, Mbar);
    orc_adjoint_means(g, Mbar, fbar);
    free(Mbar);
}

long long orc_count_samples(const orc_geom* g)
{
    const int n = g->n, n_r = g->n_t + 2, K = g->n_angles;
    const double dt = g->t_max / (double)g->n_t;
    const double h = 2.0 / (double)n;
    const double two_pi = 2.0 * acos(-1.0);
    double* xy = (double*)malloc(sizeof(double) * 2 * g->n_det);
    orc_detectors(g, xy);
    long long count = 0;
    for (int j = 0; j < g->n_det; ++j)
        for (int m = 0; m < n_r; ++m)
            for (int q = 0; q < K; ++q) {
                const double phi = two_pi * (double)q / (double)K;
                const double u = (xy[2 * j] + (double)m * dt * cos(phi) + 1.0) / h - 0.5;
                const double v = (xy[2 * j + 1] + (double)m * dt * sin(phi) + 1.0) / h - 0.5;
                const double fu = floor(u), fv = floor(v);
                if (fu >= -1.0 && fu <= (double)(n - 1) && fv >= -1.0 && fv <= (double)(n - 1)) ++count;
            }
    free(xy);
    return count;
}

/* ------------------------------------------------------------------------ */
/* Smoothed isotropic total variation (the TV term of Eq. (4) and Eq. (5)).  */
/*   TV(f) = sum_{i,j} sqrt(dx^2 + dy^2 + eps^2),                            */
/*   dx = f[i][j+1] - f[i][j] (0 on the last column),                        */
/*   dy = f[i+1][j] - f[i][j] (0 on the last row).                           */
/* The gradient is accumulated term by term (chain rule, literally).         */
/* ------------------------------------------------------------------------ */

double orc_tv(int n, double eps, const double* f, double* grad)
{
    double value = 0.0;
    if (grad) memset(grad, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const double c = f[(size_t)i * n + j];
            const double dx = (j + 1 < n) ? f[(size_t)i * n + j + 1] - c : 0.0;
            const double dy = (i + 1 < n) ? f[(size_t)(i + 1) * n + j] - c : 0.0;
            const double s = sqrt(dx * dx + dy * dy + eps * eps);
            value += s;
            if (!grad) continue;
            if (j + 1 < n) {
                grad[(size_t)i * n + j + 1] += dx / s;
                grad[(size_t)i * n + j] -= dx / s;
            }
            if (i + 1 < n) {
                grad[(size_t)(i + 1) * n + j] += dy / s;
                grad[(size_t)i * n + j] -= dy / s;
            }
        }
    return value;
}
