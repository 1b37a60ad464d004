/*
 * FP64 CPU oracle for the discrete Radon transform R_h and its adjoint R_h^*
 * (linear backprojection), Sec. 3.1 "Discretization" of the thesis.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load this file;
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Geometry (readings of the thesis, stated once here):
 *   pixel (i, j), 0 <= i, j < n, sits at x_i = h (i - (n-1)/2), y_j = h (j - (n-1)/2)
 *   (first array index i <-> x, second j <-> y; image stored u[i*n + j]);
 *   at angle theta_l it projects to the detector coordinate
 *       s = x_i cos(theta_l) + y_j sin(theta_l),
 *   bin k (0 <= k < M) is centred at s_k = (k - (M-1)/2) ds, so in bin units
 *       p = s / ds + (M-1)/2.
 *   Linear interpolation between the two nearest bins: bin floor(p) gets weight
 *   1 - frac(p) and bin floor(p)+1 gets frac(p) -- the hat function
 *   Lambda(p - k) = max(0, 1 - |p - k|).  Bins outside [0, M) are dropped
 *   (zero-padded detector).  Sinogram stored g[l*M + k].
 *
 * Three independent formulations are provided so they can check each other:
 *   oracle_rh_adjoint : pixel loop, gather with floor/frac   (definition of R_h^*)
 *   oracle_rh_forward : pixel loop, splat with floor/frac    (R_h = (R_h^*)^*, gamma weights)
 *   *_entries         : brute force with the hat function, one output at a time.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* detector coordinate p of pixel (i, j) at the angle with cosine ct, sine st */
static inline double det_p(int n, int M, double h, double ds, double ct, double st, int i, int j)
{
    double x = h * ((double)i - 0.5 * (double)(n - 1));
    double y = h * ((double)j - 0.5 * (double)(n - 1));
    return (x * ct + y * st) / ds + 0.5 * (double)(M - 1);
}

static void trig_tables(int N, const double *theta, double *ct, double *st)
{
    for (int l = 0; l < N; ++l) {
        ct[l] = cos(theta[l]);
        st[l] = sin(theta[l]);
    }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* u = R_h^* g : for each pixel, sum over angles of the linearly interpolated
 * sinogram value at the pixel's detector coordinate. */
int oracle_rh_adjoint(int n, int N, int M, double h, double ds, const double *theta,
                      const double *g, double *u)
{
    if (n < 0 || N < 0 || M < 0) return -1;
    double *ct = (double *)malloc(sizeof(double) * (N > 0 ? N : 1));
    double *st = (double *)malloc(sizeof(double) * (N > 0 ? N : 1));
    if (!ct || !st) { free(ct); free(st); return -2; }
    trig_tables(N, theta, ct, st);
#pragma omp parallel for schedule(static)
    for (long idx = 0; idx < (long)n * n; ++idx) {
        int i = (int)(idx / n), j = (int)(idx % n);
        double acc = 0.0;
        for (int l = 0; l < N; ++l) {
            double p = det_p(n, M, h, ds, ct[l], st[l], i, j);
            double fl = floor(p);
            long k = (long)fl;
            double a = p - fl;
            if (k >= 0 && k < M) acc += (1.0 - a) * g[(long)l * M + k];
            if (k + 1 >= 0 && k + 1 < M) acc += a * g[(long)l * M + k + 1];
        }
        u[idx] = acc;
    }
    free(ct);
    free(st);
    return 0;
}

/* g = R_h u : every pixel's value is split between bins floor(p) and
 * floor(p)+1 with the same weights the backprojection reads with. */
int oracle_rh_forward(int n, int N, int M, double h, double ds, const double *theta,
                      const double *u, double *g)
{
    if (n < 0 || N < 0 || M < 0) return -1;
    double *ct = (double *)malloc(sizeof(double) * (N > 0 ? N : 1));
    double *st = (double *)malloc(sizeof(double) * (N > 0 ? N : 1));
    if (!ct || !st) { free(ct); free(st); return -2; }
    trig_tables(N, theta, ct, st);
#pragma omp parallel for schedule(static)
    for (int l = 0; l < N; ++l) {
        double *row = g + (long)l * M;
        for (int k = 0; k < M; ++k) row[k] = 0.0;
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) {
                double p = det_p(n, M, h, ds, ct[l], st[l], i, j);
                double fl = floor(p);
                long k = (long)fl;
                double a = p - fl;
                double v = u[(long)i * n + j];
                if (k >= 0 && k < M) row[k] += (1.0 - a) * v;
                if (k + 1 >= 0 && k + 1 < M) row[k + 1] += a * v;
            }
        }
    }
    free(ct);
    free(st);
    return 0;
}

static inline double hat(double t)
{
    double a = 1.0 - fabs(t);
    return a > 0.0 ? a : 0.0;
}

/* (R_h u)_{l,k} for a list of (l, k) pairs, each by brute force over all
 * pixels with the hat weight Lambda(p - k). */
int oracle_rh_forward_entries(int n, int N, int M, double h, double ds, const double *theta,
                              const double *u, int count, const int *ls, const int *ks,
                              double *out)
{
    if (n < 0 || N < 0 || M < 0 || count < 0) return -1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int e = 0; e < count; ++e) {
        int l = ls[e], k = ks[e];
        double ct = cos(theta[l]), st = sin(theta[l]);
        double acc = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                acc += u[(long)i * n + j] * hat(det_p(n, M, h, ds, ct, st, i, j) - (double)k);
        out[e] = acc;
    }
    (void)N;
    return 0;
}

/* (R_h^* g)_{i,j} for a list of (i, j) pairs, each by brute force over all
 * sinogram entries with the hat weight. */
int oracle_rh_adjoint_entries(int n, int N, int M, double h, double ds, const double *theta,
                              const double *g, int count, const int *is, const int *js,
                              double *out)
{
    if (n < 0 || N < 0 || M < 0 || count < 0) return -1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int e = 0; e < count; ++e) {
        int i = is[e], j = js[e];
        double acc = 0.0;
        for (int l = 0; l < N; ++l) {
            double p = det_p(n, M, h, ds, cos(theta[l]), sin(theta[l]), i, j);
            for (int k = 0; k < M; ++k) acc += g[(long)l * M + k] * hat(p - (double)k);
        }
        out[e] = acc;
    }
    return 0;
}
