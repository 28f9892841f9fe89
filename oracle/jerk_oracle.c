/*
 * FP64 CPU oracle for the Fourier-domain jerk search -- TEST INFRASTRUCTURE.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may load this file's library.  It shares no code with the CUDA path.
 *
 * It computes, by the plain definitions and nothing cleverer:
 *   - the Fourier response of a signal with constant fddot (Sec. 2: one
 *     matched filter per (z, w), z = fdot T^2, w = fddot T^3) as the integral
 *       rho(q; z, w) = int_{-1/2}^{1/2} exp(2 pi i (-q u + z u^2/2 + w u^3/6)) du,
 *     evaluated by composite Gauss-Legendre quadrature (nodes supplied by the
 *     caller from a library routine);
 *   - the matched-filter correlation of a spectrum with a tap vector by
 *     direct summation (the quantity the paper's overlap-and-save FFT
 *     convolution evaluates, Sec. 2 and Fig. 1):
 *       O_p = sum_k F_k c_{b k - p},   |b k - p| <= D,  0 <= k < N.
 *
 * Build: gcc -O2 -fopenmp -fPIC -shared -ffp-contract=off (no fast-math).
 */
#include <math.h>
#include <stdint.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static const double TWO_PI = 6.283185307179586476925286766559;

/*
 * rho(q_j; z, w) for j < nq by composite Gauss-Legendre quadrature.
 * gl_x / gl_w: n_gl nodes and weights on [-1, 1]; the interval [-1/2, 1/2]
 * is cut into n_panels equal panels.  out: interleaved (re, im), 2*nq.
 */
void oracle_rho(const double *q, int64_t nq, double z, double w,
                const double *gl_x, const double *gl_w, int n_gl, int n_panels,
                double *out)
{
    const double h = 1.0 / (double)n_panels;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < nq; ++j) {
        double re = 0.0, im = 0.0;
        for (int p = 0; p < n_panels; ++p) {
            const double a = -0.5 + h * (double)p;
            double pre = 0.0, pim = 0.0;
            for (int i = 0; i < n_gl; ++i) {
                const double u = a + 0.5 * h * (gl_x[i] + 1.0);
                /* phase in cycles; reduce to [0,1) before scaling by 2 pi */
                double cyc = -q[j] * u + z * u * u / 2.0 + w * u * u * u / 6.0;
                cyc -= floor(cyc);
                const double ph = TWO_PI * cyc;
                pre += gl_w[i] * cos(ph);
                pim += gl_w[i] * sin(ph);
            }
            re += 0.5 * h * pre;
            im += 0.5 * h * pim;
        }
        out[2 * j] = re;
        out[2 * j + 1] = im;
    }
}

/*
 * Direct correlation of one tap vector with the spectrum.
 * F: interleaved complex[N]; taps: interleaved complex[2D+1] holding c_d for
 * d = -D..D at index d + D; outputs O_p for p = p0 .. p0+np-1 (interleaved).
 * Bins outside [0, N) are zero.
 */
void oracle_correlate(const double *F, int64_t N, int b,
                      const double *taps, int64_t D,
                      int64_t p0, int64_t np, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < np; ++j) {
        const int64_t p = p0 + j;
        /* k with |b k - p| <= D  ->  ceil((p - D)/b) <= k <= floor((p + D)/b) */
        int64_t klo = p - D;
        klo = (klo >= 0) ? (klo + b - 1) / b : -((-klo) / b);
        int64_t khi = p + D;
        khi = (khi >= 0) ? khi / b : -((-khi + b - 1) / b);
        if (klo < 0) klo = 0;
        if (khi > N - 1) khi = N - 1;
        double re = 0.0, im = 0.0;
        for (int64_t k = klo; k <= khi; ++k) {
            const int64_t d = b * k - p;
            const double fr = F[2 * k], fi = F[2 * k + 1];
            const double cr = taps[2 * (d + D)], ci = taps[2 * (d + D) + 1];
            re += fr * cr - fi * ci;
            im += fr * ci + fi * cr;
        }
        out[2 * j] = re;
        out[2 * j + 1] = im;
    }
}

/*
 * Power |O_p|^2 of many tap vectors at an explicit list of cells.
 * taps_all: interleaved complex, template t's taps start at tap_off[t]
 * (complex index) with half-width D[t].  cells: ncell pairs (t, p).
 * out: power per requested cell.
 */
void oracle_power_cells(const double *F, int64_t N, int b,
                        const double *taps_all, const int64_t *tap_off,
                        const int64_t *D, const int64_t *cell_t,
                        const int64_t *cell_p, int64_t ncell, double *out)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 0; c < ncell; ++c) {
        const int64_t t = cell_t[c], p = cell_p[c];
        const double *taps = taps_all + 2 * tap_off[t];
        const int64_t Dt = D[t];
        int64_t klo = p - Dt;
        klo = (klo >= 0) ? (klo + b - 1) / b : -((-klo) / b);
        int64_t khi = p + Dt;
        khi = (khi >= 0) ? khi / b : -((-khi + b - 1) / b);
        if (klo < 0) klo = 0;
        if (khi > N - 1) khi = N - 1;
        double re = 0.0, im = 0.0;
        for (int64_t k = klo; k <= khi; ++k) {
            const int64_t d = b * k - p;
            const double fr = F[2 * k], fi = F[2 * k + 1];
            const double cr = taps[2 * (d + Dt)], ci = taps[2 * (d + Dt) + 1];
            re += fr * cr - fi * ci;
            im += fr * ci + fi * cr;
        }
        out[c] = re * re + im * im;
    }
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
