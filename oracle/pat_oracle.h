/*
 * pat_oracle.h — plain FP64 CPU oracle for the discrete 2D circular-geometry
 * photoacoustic forward operator A and its adjoint A^T.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product
 * library never links, loads or calls it, and it shares no code, header or
 * table with the product.
 *
 * The continuous model is the wave initial-value problem of Eq. (1) with the
 * boundary trace of Eq. (2) (Sec. 2.1); the operator equation g = A f + delta
 * is Eq. (3).  With constant sound speed c = 1 the 2D Poisson formula gives
 *     p(y, t) = d/dt  int_0^t  r (M f)(y, r) / sqrt(t^2 - r^2)  dr,
 * where (M f)(y, r) is the mean of f over the circle of radius r about y.
 * The paper delegates the discretisation to its fast circular-geometry
 * operators (Sec. 2.1, last paragraph); this oracle implements the direct
 * discretisation of this library, step by step:
 *
 *   grid      N x N pixels on [-1,1]^2, h = 2/N, pixel (iy, ix) centred at
 *             (x, y) = (-1 + (ix + 1/2) h, -1 + (iy + 1/2) h); f[iy*N + ix].
 *   detectors on the unit circle, theta_j = theta0 + (j + 1/2) Phi / n_det
 *             (cell-centred on the arc: 256 detectors on 270 degrees, subsets
 *             of 170 and 112 give 179.30 and 118.125 degrees, Sec. 2.1/2.4.2).
 *   time      Delta = T / n_t, t_k = k Delta, k = 1..n_t; radii r_m = m Delta,
 *             m = 0..n_t+1 (n_r = n_t + 2 nodes).
 *   angles    phi_q = 2 pi q / K, q = 0..K-1 (periodic trapezoid rule).
 *   sample    bilinear interpolation of f, zero outside the N x N grid.
 *   means     M[j][m] = (1/K) sum_q f~(y_j + r_m (cos phi_q, sin phi_q)).
 *   time      M taken piecewise linear in r; the Abel integral is integrated
 *             exactly against hat functions (product integration) and the
 *             time derivative is the midpoint difference over +-Delta/2:
 *             g[j][k-1] = sum_m P[k-1][m] M[j][m].
 *   adjoint   the literal transpose: Mbar = P^T gbar, then a scatter of every
 *             sample's bilinear weights.
 *   TV        isotropic, forward differences, zero difference on the last
 *             row/column, smoothed by eps (Eq. (4), Eq. (5)).
 */
#ifndef PAT_ORACLE_H
#define PAT_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n;            /* image side N                                     */
    int n_det;        /* detectors on the arc                              */
    double arc_start; /* theta0 (radians)                                  */
    double arc_span;  /* Phi (radians), 0 < Phi <= 2 pi                    */
    int n_t;          /* time samples                                      */
    double t_max;     /* T                                                 */
    int n_angles;     /* K angular quadrature nodes per circular mean      */
} orc_geom;

/* Number of worker threads (OpenMP) the oracle may use; 1 = serial.       */
void orc_set_threads(int n);
int orc_get_threads(void);

/* Abel-plus-derivative matrix, dense row-major n_t x (n_t + 2).           */
void orc_abel_matrix(int n_t, double* P);

/* Dimensionless product-integration weights w_m(tau), m = 0..n_r-1.        */
void orc_abel_weights(double tau, int n_r, double* w);

/* Bilinear sample of f (N x N, zero outside) at the world point (sx, sy). */
double orc_bilinear(const double* f, int n, double sx, double sy);

/* Mean of f over K equispaced nodes on the circle of radius r about c.   */
double orc_circle_mean(const double* f, int n, double cx, double cy,
                       double r, int K);

/* Detector coordinates, xy[2j] = cos(theta_j), xy[2j+1] = sin(theta_j).   */
void orc_detectors(const orc_geom* g, double* xy);

/* M[j][m] (n_det x (n_t+2)).                                              */
void orc_circular_means(const orc_geom* g, const double* f, double* M);

/* g = A f, g is n_det x n_t (time fastest).                               */
void orc_forward(const orc_geom* g, const double* f, double* out);

/* Mbar = P^T gbar  (n_det x (n_t+2)).                                     */
void orc_adjoint_time(const orc_geom* g, const double* gbar, double* Mbar);

/* fbar = A^T gbar (N x N), by scattering every sample's weights.          */
void orc_adjoint(const orc_geom* g, const double* gbar, double* fbar);

/* Scatter part of A^T alone: fbar = C^T Mbar.                             */
void orc_adjoint_means(const orc_geom* g, const double* Mbar, double* fbar);

/* Number of (j, m, q) samples whose bilinear footprint touches the grid.  */
long long orc_count_samples(const orc_geom* g);

/* Smoothed isotropic TV value; grad (nullable) receives its gradient.     */
double orc_tv(int n, double eps, const double* f, double* grad);

#ifdef __cplusplus
}
#endif
#endif
