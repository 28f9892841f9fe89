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
 *       O_p = sum_k F_k c_{b k - p},   |b k - p| <= D,  0 <= k < N;
 *   - the same correlation by overlap-and-save with a radix-2 FP64 DFT (the
 *     FFT route, oracle_fft_search below), for whole-bank searches of long
 *     spectra, with the harmonic sums, max-projections and statistics.
 *
 * Build: gcc -O2 -fopenmp -fPIC -shared -ffp-contract=off (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

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

/* ---------------------------------------------------------------------------
 * The FFT route (Sec. 2, Fig. 1: overlap-and-save), for searches too large
 * for direct summation.  Everything here is FP64 and follows the plain
 * definitions:
 *   - a radix-2 decimation-in-time DFT, X_k = sum_j x_j exp(s 2 pi i j k / n);
 *   - circular correlation by the DFT: y_n = sum_m g_m x_{(n+m) mod L} has
 *     DFT X_k G+_k with G+ the DFT of g of sign +1;
 *   - overlap-and-save: segment s of the spread spectrum (G_j = F_{j/b} for
 *     j = 0 mod b, 0 elsewhere and outside [0, bN)) starts at cell s V - Dmax,
 *     g_m = c_{m - Dmax} (zero beyond the template's own half-width), and the
 *     first V = L - 2 Dmax outputs of each segment are the cells s V + n;
 *   - harmonic sums S_H(p) = sum_{h=1..H} P(h p; h z, h w) (all integer h),
 *     accumulated in FP64 in h order;
 *   - per stage: the (z, w) max-projection of S_H rounded to FP32 (decisions
 *     in FP32), its argmax (lowest template on equal FP32 values, templates
 *     processed in ascending order), the runner-up FP32 value among the
 *     other fundamentals, and the sums of S_H and S_H^2 (FP64; per fixed
 *     block of cells, added in template and block order, so the result does
 *     not depend on the number of threads).
 * ------------------------------------------------------------------------- */
static void dft_radix2(double *x, int64_t n, int sign, const double *tw)
{
    /* bit-reversal permutation */
    for (int64_t i = 1, j = 0; i < n; ++i) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t0 = x[2 * i], t1 = x[2 * i + 1];
            x[2 * i] = x[2 * j];
            x[2 * i + 1] = x[2 * j + 1];
            x[2 * j] = t0;
            x[2 * j + 1] = t1;
        }
    }
    /* butterflies: sub-transforms of length len from two of length len/2 */
    for (int64_t len = 2; len <= n; len <<= 1) {
        const int64_t half = len >> 1, step = n / len;
        for (int64_t i = 0; i < n; i += len) {
            for (int64_t k = 0; k < half; ++k) {
                const double wr = tw[2 * k * step];
                const double wi = sign < 0 ? tw[2 * k * step + 1] : -tw[2 * k * step + 1];
                double *a = x + 2 * (i + k), *c = x + 2 * (i + k + half);
                const double vr = c[0] * wr - c[1] * wi, vi = c[0] * wi + c[1] * wr;
                c[0] = a[0] - vr;
                c[1] = a[1] - vi;
                a[0] += vr;
                a[1] += vi;
            }
        }
    }
}

/* exp(-2 pi i m / n) for m < n/2, interleaved */
static double *dft_twiddles(int64_t n)
{
    double *tw = (double *)malloc(sizeof(double) * (size_t)(n > 1 ? n : 2));
    if (!tw) return NULL;
    for (int64_t m = 0; m < n / 2; ++m) {
        const double a = TWO_PI * (double)m / (double)n;
        tw[2 * m] = cos(a);
        tw[2 * m + 1] = -sin(a);
    }
    return tw;
}

/* The DFT above on its own (pinned against a library FFT).  x: interleaved
 * complex[n], n a power of two; sign -1 or +1; unnormalised.  Returns 0, or
 * -1 if n is not a power of two or memory runs out. */
int oracle_dft(double *x, int64_t n, int sign)
{
    if (n < 1 || (n & (n - 1))) return -1;
    double *tw = dft_twiddles(n);
    if (!tw) return -1;
    dft_radix2(x, n, sign, tw);
    free(tw);
    return 0;
}

typedef struct {
    const double *F;
    int64_t N, bN;
    int b;
    const double *taps_all;
    const int64_t *tap_off, *D;
    int64_t L, V, Dmax, nseg;
    double *X;          /* [nseg][L] forward DFTs of the segments */
    const double *tw;
} ols_t;

/* forward DFTs of the segments of the spread spectrum into o->X */
static void ols_segments(ols_t *o)
{
    const int64_t L = o->L;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < o->nseg; ++s) {
        double *x = o->X + 2 * s * L;
        for (int64_t i = 0; i < L; ++i) {
            const int64_t j = s * o->V - o->Dmax + i;     /* spread cell */
            double re = 0.0, im = 0.0;
            if (j >= 0 && j < o->bN && j % o->b == 0) {
                re = o->F[2 * (j / o->b)];
                im = o->F[2 * (j / o->b) + 1];
            }
            x[2 * i] = re;
            x[2 * i + 1] = im;
        }
        dft_radix2(x, L, -1, o->tw);
    }
}

/* P(p) = |O_p|^2 of template u for every cell p < bN, into row */
static void ols_row(const ols_t *o, int64_t u, double *row, double *filt)
{
    const int64_t L = o->L, Du = o->D[u];
    const double *c = o->taps_all + 2 * o->tap_off[u];
    memset(filt, 0, sizeof(double) * 2 * (size_t)L);
    for (int64_t d = -Du; d <= Du; ++d) {          /* g_{d + Dmax} = c_d */
        filt[2 * (d + o->Dmax)] = c[2 * (d + Du)];
        filt[2 * (d + o->Dmax) + 1] = c[2 * (d + Du) + 1];
    }
    dft_radix2(filt, L, +1, o->tw);
    const double inv = 1.0 / (double)L;
#pragma omp parallel
    {
        double *y = (double *)malloc(sizeof(double) * 2 * (size_t)L);
#pragma omp for schedule(static)
        for (int64_t s = 0; s < o->nseg; ++s) {
            const double *X = o->X + 2 * s * L;
            for (int64_t k = 0; k < L; ++k) {
                const double xr = X[2 * k], xi = X[2 * k + 1], hr = filt[2 * k], hi = filt[2 * k + 1];
                y[2 * k] = xr * hr - xi * hi;
                y[2 * k + 1] = xr * hi + xi * hr;
            }
            dft_radix2(y, L, +1, o->tw);
            for (int64_t n = 0; n < o->V; ++n) {
                const int64_t p = s * o->V + n;
                if (p >= o->bN) break;
                const double re = y[2 * n] * inv, im = y[2 * n + 1] * inv;
                row[p] = re * re + im * im;
            }
        }
        free(y);
    }
}

enum { SUM_BLOCK = 65536 };

/* Fold the values S(p), p < n, of one fundamental t into stage s: FP32
 * max-projection, argmax, runner-up and the FP64 sums. */
static void stage_update(const double *S, int64_t stride, int64_t n, int32_t t,
                         float *Mv, int32_t *Mt, float *M2, double *sums)
{
    const int64_t nblk = (n + SUM_BLOCK - 1) / SUM_BLOCK;
    double *part = (double *)calloc((size_t)(2 * nblk), sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nblk; ++k) {
        const int64_t p1 = (k + 1) * SUM_BLOCK < n ? (k + 1) * SUM_BLOCK : n;
        double s1 = 0.0, s2 = 0.0;
        for (int64_t p = k * SUM_BLOCK; p < p1; ++p) {
            const double v = S[p * stride];
            s1 += v;
            s2 += v * v;
            const float f = (float)v;
            if (f > Mv[p]) {
                M2[p] = Mv[p];
                Mv[p] = f;
                Mt[p] = t;
            } else if (f > M2[p]) {
                M2[p] = f;
            }
        }
        part[2 * k] = s1;
        part[2 * k + 1] = s2;
    }
    for (int64_t k = 0; k < nblk; ++k) {
        sums[0] += part[2 * k];
        sums[1] += part[2 * k + 1];
    }
    free(part);
}

/*
 * The search by the FFT route over the fundamentals `fund` (ascending).
 *  F          normalised spectrum, interleaved complex[N]
 *  taps_all, tap_off, D   taps of every template (as for oracle_power_cells)
 *  L          DFT length (power of two, > 2 max D)
 *  stages     n_st stage numbers H, ascending, stages[0] == 1
 *  harm       [T][8]: template of (h z_t, h w_t), h = 1..8 (-1 off the grid)
 *  top        [T]: number of stages at which t is a fundamental (nested)
 *  moff       [n_st]: offset of stage s in Mv/Mt/M2 (n_valid(bN, H_s) cells)
 *  Mv, Mt, M2 max-projection, argmax, runner-up; Mv and M2 must be
 *             initialised to -inf and Mt to -1 by the caller
 *  sums       [n_st][2]: sum of S_H and of S_H^2 (added to)
 *  rows_done  (out) power rows computed
 * Returns 0, or -1 on bad sizes / memory.
 */
int oracle_fft_search(const double *F, int64_t N, int b,
                      const double *taps_all, const int64_t *tap_off, const int64_t *D, int64_t T,
                      int64_t L, int n_st, const int32_t *stages,
                      const int64_t *harm, const int32_t *top,
                      const int64_t *fund, int64_t n_fund,
                      const int64_t *moff, float *Mv, int32_t *Mt, float *M2, double *sums,
                      int64_t *rows_done)
{
    ols_t o;
    o.F = F;
    o.N = N;
    o.b = b;
    o.bN = (int64_t)b * N;
    o.taps_all = taps_all;
    o.tap_off = tap_off;
    o.D = D;
    o.L = L;
    o.Dmax = 0;
    for (int64_t t = 0; t < T; ++t)
        if (D[t] > o.Dmax) o.Dmax = D[t];
    o.V = L - 2 * o.Dmax;
    if (L < 2 || (L & (L - 1)) || o.V < 1 || n_st < 1 || stages[0] != 1) return -1;
    o.nseg = (o.bN + o.V - 1) / o.V;
    double *tw = dft_twiddles(L);
    o.X = (double *)malloc(sizeof(double) * 2 * (size_t)(o.nseg * L));
    double *row = (double *)malloc(sizeof(double) * (size_t)o.bN);
    double *acc = (double *)malloc(sizeof(double) * (size_t)o.bN);
    double *filt = (double *)malloc(sizeof(double) * 2 * (size_t)L);
    if (!tw || !o.X || !row || !acc || !filt) {
        free(tw); free(o.X); free(row); free(acc); free(filt);
        return -1;
    }
    o.tw = tw;
    ols_segments(&o);
    int64_t rows = 0;
    for (int64_t q = 0; q < n_fund; ++q) {
        const int64_t t = fund[q];
        const int ntop = top[t];
        const int hmax = stages[ntop - 1];
        for (int h = 1; h <= hmax; ++h) {
            const int64_t u = harm[t * 8 + (h - 1)];
            if (u < 0) { free(tw); free(o.X); free(row); free(acc); free(filt); return -1; }
            ols_row(&o, u, row, filt);
            ++rows;
            const int64_t nh = (o.bN - 1) / h + 1;          /* cells with h p < bN */
            if (hmax > 1) {
                if (h == 1) {
                    memcpy(acc, row, sizeof(double) * (size_t)nh);
                } else {
#pragma omp parallel for schedule(static)
                    for (int64_t p = 0; p < nh; ++p) acc[p] += row[h * p];
                }
            }
            for (int s = 0; s < ntop; ++s)
                if (stages[s] == h)
                    stage_update(h == 1 ? row : acc, 1, nh, (int32_t)t, Mv + moff[s], Mt + moff[s],
                                 M2 + moff[s], sums + 2 * s);
        }
    }
    if (rows_done) *rows_done = rows;
    free(tw); free(o.X); free(row); free(acc); free(filt);
    return 0;
}

/*
 * Power rows |O_p|^2 (p < bN) of the templates tlist[0..nt-1] by the FFT
 * route alone, FP64, into out[nt][bN] (to pin the route against direct
 * summation).  Arguments as for oracle_fft_search.  Returns 0 or -1.
 */
int oracle_fft_rows(const double *F, int64_t N, int b,
                    const double *taps_all, const int64_t *tap_off, const int64_t *D, int64_t T,
                    int64_t L, const int64_t *tlist, int64_t nt, double *out)
{
    ols_t o;
    o.F = F;
    o.N = N;
    o.b = b;
    o.bN = (int64_t)b * N;
    o.taps_all = taps_all;
    o.tap_off = tap_off;
    o.D = D;
    o.L = L;
    o.Dmax = 0;
    for (int64_t t = 0; t < T; ++t)
        if (D[t] > o.Dmax) o.Dmax = D[t];
    o.V = L - 2 * o.Dmax;
    if (L < 2 || (L & (L - 1)) || o.V < 1) return -1;
    o.nseg = (o.bN + o.V - 1) / o.V;
    double *tw = dft_twiddles(L);
    o.X = (double *)malloc(sizeof(double) * 2 * (size_t)(o.nseg * L));
    double *filt = (double *)malloc(sizeof(double) * 2 * (size_t)L);
    if (!tw || !o.X || !filt) {
        free(tw); free(o.X); free(filt);
        return -1;
    }
    o.tw = tw;
    ols_segments(&o);
    for (int64_t i = 0; i < nt; ++i) ols_row(&o, tlist[i], out + i * o.bN, filt);
    free(tw); free(o.X); free(filt);
    return 0;
}
