/*
 * jerk.h -- C ABI of the GB300 (sm_103a) Fourier-domain jerk search.
 *
 * The method (Adamek, Novotny, Dimoudi & Armour, "Searching for pulsars in
 * extreme orbits - GPU acceleration of the Fourier domain 'jerk' search"):
 * a power-normalised complex spectrum is correlated, by overlap-and-save
 * (Fig. 1), with one matched filter per (z, w), z = fdot T^2 and
 * w = fddot T^3 (Sec. 2); the |.|^2 power plane over (r, z, w) is harmonic-
 * summed and thresholded peaks are kept as candidates after computing the
 * mean and standard deviation (Sec. 3).
 *
 * Conventions used throughout:
 *   b        Fourier cells per bin ("numbetween"), must be 2.
 *   N        complex bins of the input spectrum; cells p = 0 .. bN-1, r = p/b.
 *   z_i      -zmax + i dz, i < nz = 2 zmax/dz + 1.
 *   w_j      -wmax + j dw, j < nw = 2 wmax/dw + 1.
 *   t        template index j*nz + i.
 *   m(z,w)   ceil(|z|/2 + |w|/8) + pad_bins: template half-width in bins.
 *   M        max over the bank of m(z, w); K = 2 b M + 1 taps.
 *   L        segment (FFT) length in cells; V = L - K + 1 outputs kept per segment.
 *   stage H  S_H(p, z, w) = sum_{h=1..H} P(h p, h z, h w), defined where
 *            H p < bN, |H z| <= zmax and |H w| <= wmax.
 *
 * Memory: every pointer argument named d_* is DEVICE memory on the plan's
 * device; h_* is host memory.  "complex64" is interleaved (re, im) float32.
 * The plan owns its device buffers (template bank, workspace, candidates);
 * the caller owns every buffer it passes in.  Calls taking a stream enqueue
 * work on that cudaStream_t (NULL = legacy default stream) and return
 * before it completes, unless stated otherwise.
 *
 * Errors: no call aborts or throws.  Invalid arguments return JERK_EINVAL
 * with nothing enqueued; a CUDA error (including a sticky one from earlier
 * work) returns JERK_ECUDA; allocation failures return JERK_ENOMEM.  A plan
 * is not thread-safe; distinct plans are independent.
 */
#ifndef JERK_H_
#define JERK_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct jerk_plan_s *jerk_plan;

typedef enum {
    JERK_OK = 0,
    JERK_EINVAL = 1,     /* invalid argument or parameter set */
    JERK_ENOMEM = 2,     /* device or host allocation failed / does not fit */
    JERK_ECUDA = 3,      /* a CUDA runtime error */
    JERK_ETIMEOUT = 4,   /* a bounded device-side wait expired */
    JERK_EOVERFLOW = 5,  /* more candidates than the buffer holds */
    JERK_ESTATE = 6      /* call out of order (e.g. search before templates) */
} jerk_status;

enum { JERK_THRESH_ABS = 0, JERK_THRESH_SIGMA = 1 };
enum { JERK_MAX_STAGES = 4, JERK_MAX_HARMONIC = 8 };
enum { JERK_BATCH_GRAPH = 1, JERK_BATCH_TRANSIENT = 2 };

/* Search parameters.  Sec. 2 defines the (z, w) filters; Sec. 3 the
 * user threshold, statistics and harmonic sum. */
typedef struct {
    int32_t zmax, dz;        /* zmax % dz == 0, dz > 0, zmax >= 0 */
    int32_t wmax, dw;        /* wmax % dw == 0, dw > 0, wmax >= 0 */
    int32_t numbetween;      /* b; must be 2 */
    int32_t pad_bins;        /* P >= 1; default 16 */
    int32_t seg_len;         /* L in cells: 1024, 2048, 4096 or 8192; 0 = choose */
    int32_t n_stages;        /* 1..4 */
    int32_t stages[4];       /* strictly ascending, stages[0] == 1, each <= 8 */
    int32_t thresh_mode;     /* JERK_THRESH_ABS or JERK_THRESH_SIGMA */
    float   thresh[4];       /* ABS: power; SIGMA: T in theta = mu + T sigma */
    int32_t norm_block;      /* B in bins (1..4096), 0 = input already normalised */
    int32_t precision;       /* filter arithmetic: 0 = FP32, 1 = BF16 and 2 = FP16 tensor-core
                                DFT blocks (FP32 accumulation; seg_len 0 or 4096) */
    int64_t max_bins;        /* capacity: largest N a search may use (total over a batch), <= 2^29 */
    int64_t max_candidates;  /* capacity of the plan's candidate buffer (total over a batch) */
    int32_t max_batch;       /* largest number of spectra in one jerk_search_batch; 0 = 1 */
    int32_t group_size;      /* templates per template group of the filter (a tile-shape choice:
                                each group is one work unit of the fused kernel, its bank slice
                                shared through L2); 0 = choose (32 MiB of bank per group, at
                                least 8 templates, about 6 waves of CTAs); 1 .. 65536 */
} jerk_params;

/* One candidate: a peak of the stage-H max-projection over (z, w). */
typedef struct {
    int64_t p;               /* cell index; Fourier frequency r = p / b */
    double  r;
    int32_t t;               /* template index of the maximum (lowest t on ties) */
    int32_t z_idx, w_idx;    /* t = w_idx * nz + z_idx */
    int32_t stage;           /* H */
    float   z, w;            /* z_i, w_j of the fundamental */
    float   power;           /* S_H at (p, t) in normalised power units (FP32) */
    int32_t item;            /* spectrum of the batch (0 for jerk_search) */
} jerk_candidate;

/* A candidate refined off the grid (jerk_refine). */
typedef struct {
    double  r;               /* Fourier frequency of the largest power evaluated */
    float   z, w;            /* its z, w */
    float   power;           /* that power (matched filter of the fundamental, h = 1) */
    float   power_in;        /* the power at the candidate's own (r, z, w) */
    int32_t is_peak;         /* 1 if power_in is not below any power evaluated */
    int32_t reserved;
} jerk_refined;

/* Read-only description of a plan (sizes derived from the parameters). */
typedef struct {
    int32_t nz, nw, n_templates;
    int32_t bank_halfwidth;  /* M in bins */
    int32_t taps;            /* K = 2 b M + 1 */
    int32_t seg_len;         /* L */
    int32_t seg_valid;       /* V = L - K + 1 */
    int32_t device;
    int64_t max_bins;
    int64_t slot_floats;     /* harmonic-row workspace at max_bins, in floats */
    int64_t workspace_bytes; /* device bytes of the plan's own workspace (bank excluded) */
    int64_t transforms;      /* length-L inverse transforms one search of max_bins bins performs */
    int32_t n_groups;        /* template groups (similar half-width, own segment length) */
    int32_t reserved;
    const void *d_bank;      /* complex64[n_templates][L] template spectra in processing order
                                (see jerk_template_row; valid after jerk_templates) */
    int64_t bank_bytes;      /* device bytes of the template bank and its tables, shared by
                                every plan made from it with jerk_plan_share */
} jerk_info;

/* Check a parameter set without touching any GPU: JERK_OK if
 * jerk_plan_create would accept it (device and memory aside), else
 * JERK_EINVAL.  The rules are those stated on the fields of jerk_params. */
jerk_status jerk_params_validate(const jerk_params *params);

/* Validate `params`, select device `device` (made current), size and
 * allocate the plan's device memory for spectra of up to max_bins bins.
 * The template bank is not built yet: call jerk_templates next.
 * On error *out is set to NULL. */
jerk_status jerk_plan_create(const jerk_params *params, int device, jerk_plan *out);

/* Build the template bank: for every (z, w), the taps
 *   c_d = conj(rho(d/b; z, w)),  |d| <= b m(z, w),
 *   rho(q; z, w) = int_{-1/2}^{1/2} exp(2 pi i (-q u + z u^2/2 + w u^3/6)) du
 * (the Fourier response of a signal with constant fddot, Sec. 2; u is time
 * from mid-observation) by FP64 Gauss-Legendre quadrature on the GPU, then
 * their length-L spectra (FP64 FFT, stored FP32, 1/L folded in).  Enqueued
 * on `stream`; the plan may be searched once it completes. */
jerk_status jerk_templates(jerk_plan plan, void *stream);

/* The whole hot path for one spectrum d_spec (complex64[n], device,
 * 1 <= n <= max_bins), enqueued on `stream`, no host synchronisation:
 * normalise (if norm_block > 0) -> segment FFT -> template multiply ->
 * inverse FFT -> |.|^2 (overlap-and-save, Fig. 1) -> statistics (SIGMA
 * mode) and stage-1 max-projection -> harmonic sums -> thresholded peaks
 * (Sec. 3) into the plan's candidate buffer.  d_spec must stay valid until
 * the stream reaches the end of this work.  Returns JERK_ESTATE before
 * jerk_templates. */
jerk_status jerk_search(jerk_plan plan, const void *d_spec, int64_t n, void *stream);

/* As jerk_search, with h_spec in host memory (pageable or pinned): the
 * spectrum is copied into a plan-owned device buffer on `stream` first. */
jerk_status jerk_search_host(jerk_plan plan, const void *h_spec, int64_t n, void *stream);

/* Search `count` independent spectra (e.g. DM trials) of uneven lengths at
 * once: d_specs[i] is complex64[n[i]] on the device, count <= max_batch and
 * sum(n) <= max_bins.  Every spectrum goes through the same path as
 * jerk_search and gives the same candidates it would give alone; the fused
 * filter stage runs as ONE launch over all (spectrum, template group,
 * segment) work items.  With flags & JERK_BATCH_GRAPH the sequence (copy-in,
 * normalisation, filtering, harmonic sums, statistics, peaks) is captured into
 * a CUDA graph the first time a set of lengths is seen and replayed after
 * that; the caller's buffers are copied into the plan first, so they may
 * differ between calls.  Candidates (jerk_candidates) carry the spectrum index
 * in `item` and are sorted by (item, stage, p).  A new set of lengths
 * rebuilds the launch tables (a host synchronisation). */
jerk_status jerk_search_batch(jerk_plan plan, const void *const *d_specs, const int64_t *n, int32_t count,
                              int32_t flags, void *stream);

/* As jerk_search_batch, with spectrum i searched over the sub-grid
 * |z| <= zmax[i], |w| <= wmax[i] of the plan's bank (host arrays; both NULL =
 * the whole bank for every spectrum).  Each zmax[i] must be a multiple of dz
 * in [0, plan zmax], each wmax[i] a multiple of dw in [0, plan wmax]; the
 * harmonic sum of spectrum i follows the definition of stage H with its own
 * zmax[i], wmax[i] (Sec. 3).  This is how one resident bank built for the
 * largest (zmax, wmax) serves requests of any smaller search range (Sec. 2
 * defines the filters per (z, w), so a sub-grid uses the same filters).
 * Results equal those of the same spectrum and sub-grid searched alone on
 * this bank; candidate t, z_idx, w_idx are indices of the bank's grid.
 * flags: JERK_BATCH_GRAPH as for jerk_search_batch; JERK_BATCH_TRANSIENT
 * builds the launch tables into buffers the plan allocates once, with one
 * asynchronous upload and no device synchronisation, so searches on several
 * plans sharing a bank overlap on the GPU (the host waits for this plan's
 * previous search only).  The two flags exclude each other. */
jerk_status jerk_search_batch_grid(jerk_plan plan, const void *const *d_specs, const int64_t *n, const int32_t *zmax,
                                   const int32_t *wmax, int32_t count, int32_t flags, void *stream);

/* ---- one search split over several GPUs by template range ----
 *
 * (No counterpart in the paper, which runs on one GPU.)  The max-projection
 * of stage H is a maximum over fundamentals and the statistics are sums over
 * them (Sec. 3), so one search divides exactly among ranks that each take a
 * range of templates, followed by one max-reduction of the max-projections
 * and one sum-reduction of the statistics:
 *   1. every rank: jerk_search_range over its range (ranges partition
 *      [0, n_templates)), then jerk_range_sums;
 *   2. the caller reduces, over the ranks, each stage's max-projection
 *      (jerk_maxproj; element-wise maximum of the packed uint64 entries, which
 *      keeps the largest power and, on equal powers, the lowest t) and the
 *      three sums (element-wise sum), writing the reduced arrays back in place;
 *   3. jerk_select with the reduced sums; jerk_candidates then returns the
 *      candidates of the whole search (all ranks may do this, or one).
 * Merged max-projections equal those of jerk_search bitwise; the statistics
 * differ from it only by the order of FP64 additions. */

/* Partial search of d_spec (complex64[n], device) over the templates
 * t_lo <= t < t_hi: the stage-1 max-projection over those templates, the
 * stage-H max-projections over the fundamentals among them (their harmonic
 * rows are made here even when the harmonic template lies outside the
 * range), and the statistics of both (SIGMA mode).  No candidates are
 * selected (jerk_candidates returns JERK_ESTATE until jerk_select).  Single
 * spectrum (item 0).  Enqueued on `stream`. */
jerk_status jerk_search_range(jerk_plan plan, const void *d_spec, int64_t n, int32_t t_lo, int32_t t_hi,
                              void *stream);

/* After jerk_search_range (synchronises it): per stage, the sum of S_H and
 * of S_H^2 over the range's cells (SIGMA mode; 0 in ABS mode) and the number
 * of cells counted.  Arrays of n_stages entries; any may be NULL.
 * JERK_ESTATE unless the plan's last search was a jerk_search_range. */
jerk_status jerk_range_sums(jerk_plan plan, double *h_sum, double *h_sumsq, double *h_count);

/* Thresholds from the given (reduced) sums -- mu = sum/count,
 * sd = (sumsq/count - mu^2)^(1/2), theta = mu + T sd in SIGMA mode, the
 * given power in ABS mode (the arrays may then be NULL) -- and the peaks of
 * the plan's current max-projections (Sec. 3), after the plan's previous
 * work; synchronises.  jerk_stats and jerk_candidates then report them.
 * Needs a single-spectrum search (jerk_search or jerk_search_range). */
jerk_status jerk_select(jerk_plan plan, const double *h_sum, const double *h_sumsq, const double *h_count,
                        void *stream);

/* (No counterpart in the paper, which searches one spectrum at a time.)
 * A new plan that uses `parent`'s template bank (not copied; jerk_templates
 * on either plan fills it for both) with its own workspace, candidate buffer
 * and thresholds, so several searches over one bank can be in flight at once
 * (one per plan, each on its own stream).  params must equal the parent's in
 * zmax, dz, wmax, dw, numbetween, pad_bins, n_stages, stages and precision,
 * and seg_len must be 0 or the parent's L; max_bins, max_candidates,
 * max_batch, thresh_mode, thresh and norm_block may differ.  The bank stays
 * allocated until the last plan using it is destroyed, in any order.  The
 * plans are independent for thread-safety purposes, but jerk_templates must
 * not run while another plan on the bank searches. */
jerk_status jerk_plan_share(jerk_plan parent, const jerk_params *params, jerk_plan *out);

/* Matched-filter power at arbitrary points of the continuous (r, z, w)
 * space (the response of Sec. 2 off the search grid):
 *   P(r, z, w) = |sum_k F~_k conj(rho(k - r; z, w))|^2 over |k - r| <= m(z, w),
 * with F~ the spectrum d_spec (complex64[n], device) normalised as in
 * jerk_search, bins outside [0, n) zero, m(z, w) = ceil(|z|/2 + |w|/8) +
 * pad_bins, and rho evaluated by the quadrature of the template bank.  On the
 * grid (r = p/b, integer z, w) it is the plane value P(p, z, w).  h_rzw is a
 * host array of `count` triples (r, z, w) (|z| <= 8192, |w| <= 65536); the
 * powers are written to the host array h_power (FP32, FP64 sums).  Enqueued
 * on `stream` after the plan's previous work, then synchronised.  Uses the
 * plan's normalised-spectrum buffer. */
jerk_status jerk_power_at(jerk_plan plan, const void *d_spec, int64_t n, const double *h_rzw, int64_t count,
                          float *h_power, void *stream);

/* Refine candidates off the grid (Sec. 2's response evaluated between the
 * grid points; the paper keeps candidates on its grid and defines no
 * refinement or 3-D peak rule): for candidate c, jerk_power_at over the
 * points (r_c + i h_step[0], z_c + j h_step[1], w_c + l h_step[2]),
 * |i| <= h_half[0], |j| <= h_half[1], |l| <= h_half[2] (each half <= 64,
 * steps >= 0), and h_out[c] receives the largest (first in (i, j, l) order on
 * ties), the power at the candidate's own point and whether that is the
 * largest.  With steps (1/b, dz, dw) and halves (1, 1, 1) this tests the
 * candidate against its 26 grid neighbours: a local maximum of the 3-D
 * power over (r, z, w).  The powers are those of the fundamental (h = 1),
 * also for candidates of stages H > 1.  count * (grid points) <= 2^26. */
jerk_status jerk_refine(jerk_plan plan, const void *d_spec, int64_t n, const jerk_candidate *h_cands, int32_t count,
                        const double *h_step, const int32_t *h_half, jerk_refined *h_out, void *stream);

/* (No counterpart in the paper.)  Measure, on `device`, two roofline
 * denominators of the filter kernels' rooflines: the FP32 FMA rate
 * (every SM busy with independent FMA chains; *fp32_tflops counts 2 flops per
 * FMA) and the L2 read bandwidth (a 64 MB buffer read 20 times with 16-byte
 * loads, *l2_gbs).  Takes about 100 ms; allocates and frees 64 MB. */
jerk_status jerk_measure_peaks(int device, double *fp32_tflops, double *l2_gbs);

/* (No counterpart in the paper.)  Measure, on `device`, the FP32 rate of
 * packed FMAs (fma.rn.f32x2: two lanes per instruction; every SM busy with
 * independent chains; *tflops counts 4 flops per packed FMA).  The filter
 * kernels use packed FP32 where their arithmetic pairs up: a packed FMA takes
 * one issue slot for two scalar FMAs, and this figure shows whether it also
 * raises the FP32 peak (on GB300 it does not: the roofline keeps the scalar
 * FMA peak).  Takes about 50 ms; allocates and frees a few MB.  JERK_EINVAL
 * for a null pointer or a device that does not exist, JERK_ECUDA on a CUDA
 * error. */
jerk_status jerk_measure_packed_fma(int device, double *tflops);

/* (No counterpart in the paper.)  Exercise the failure path of the device
 * waits: after the plan's previous work, one GPU thread waits, with the
 * bounded wait the filter kernels use on their bulk copies and tensor-core
 * products, on a barrier phase that nothing completes.  After limit_us
 * microseconds (1 .. 10^6) it gives up and sets the plan's device error flag,
 * as a filter CTA does.  Synchronises and returns what jerk_candidates would:
 * JERK_ETIMEOUT (the flag is then cleared, and the plan and its context stay
 * usable).  No other device state changes. */
jerk_status jerk_check_waits(jerk_plan plan, int32_t limit_us, void *stream);

/* (No counterpart in the paper.)  Bounds checks of the debug build.  A
 * library compiled with -DJERK_CHECKS (`python -m paper_1911_01353_gb300.build
 * --checks`, loaded by the Python binding when JERK_CHECKS=1) checks, before
 * each global store or copy whose index its kernels compute (harmonic-row
 * stores, plane rows, max-projection updates, the harmonic sum's row copies),
 * that the index lies inside the buffer; a failing check skips the access,
 * counts itself and records its site (the first one).  This call waits for the
 * plan's work so far and reports the count (*violations), the first site
 * (*first_site, 0 if none: 1-3 fused filter rows / plane / max-projection,
 * 4-5 harmonic copy / max-projection, 6-8 tensor-core filter rows / plane /
 * max-projection) and whether the checks are compiled in (*compiled_in; in the
 * release build every check is absent and the count stays 0).  Any output may
 * be NULL.  The counts cover every search of the plan since its creation. */
jerk_status jerk_check_counts(jerk_plan plan, int64_t *violations, int32_t *first_site, int32_t *compiled_in);

/* (No counterpart in the paper.)  Test hook of the debug build: make the
 * filter kernels' own bounded waits expire, with no fault.  From the next
 * search on, at template position `position` (>= 3) of every CTA's template
 * group, the kernel leaves out one event that its threads wait for: mode 1
 * the template copy (both filters: the wait on the copy expires), mode 2 the
 * completion signal of the tensor-core filter's first product, mode 3 that of
 * its second product (precision 1 and 2 only).  Each waiting CTA gives up after
 * about one second, drains its copies in flight, frees its tensor memory and
 * leaves; jerk_candidates then returns JERK_ETIMEOUT and clears the flag.
 * Mode 0 turns the hook off.  JERK_EINVAL for a mode outside 0..3 or a
 * position below 3 (the first templates are copied before the loop);
 * JERK_ESTATE in the release build, which does not contain the hook. */
jerk_status jerk_check_inject(jerk_plan plan, int32_t mode, int32_t position);

/* Wait for the last search to finish and copy its candidates to h_out
 * (capacity cap records), sorted by (stage position, p).  *n_out receives
 * the number found.  If it exceeds cap (JERK_EOVERFLOW, first cap records
 * copied) or the plan's max_candidates (JERK_EOVERFLOW, the kept ones are
 * not guaranteed to be the first), the call says so. */
jerk_status jerk_candidates(jerk_plan plan, jerk_candidate *h_out, int64_t cap, int64_t *n_out);

/* Release everything the plan owns.  NULL is accepted. */
jerk_status jerk_plan_destroy(jerk_plan plan);

/* Static, human-readable name of a status code. */
const char *jerk_status_str(jerk_status status);

/* Fill *info.  Never fails on a valid plan. */
jerk_status jerk_plan_info(jerk_plan plan, jerk_info *info);

/* Where template t (0 <= t < n_templates) sits in the bank: *row is its row
 * of d_bank, *tap_offset the offset bM_g of its group (the spectrum of row
 * `row` is G[f] = (1/L) sum_m c_{m - bM_g} exp(+2 pi i f m / L), m < 2 bM_g + 1,
 * stored as such for precision 1 and 2; for precision 0 the row holds, for
 * f < L/2, G[f] + G[f + L/2] at index 2f and (G[f] - G[f + L/2]) exp(+2 pi i k / R0)
 * at index 2f + 1, with R0 = 2^(log2 L mod 4) (16 if that is 1) and
 * k = floor(floor(f / (L/16)) / (16/R0)): the FP32 filter's folded form,
 * because the spectra of the spread spectrum's segments have period L/2) and
 * *seg_valid its group's segment length V_g = L - 2 bM_g.  Any output may be
 * NULL.  Templates are grouped by half-width m(z, w) so that a group of short
 * filters uses a short overlap. */
jerk_status jerk_template_row(jerk_plan plan, int32_t t, int32_t *row, int32_t *tap_offset, int32_t *seg_valid);

/* ---- single steps of the path (for parity checks and composition) ---- */

/* Power normalisation only: for each block of norm_block bins (the last may
 * be short), med = the element of rank floor((n-1)/2) of |F_k|^2 (FP64),
 * F_k <- F_k (med / ln 2)^(-1/2); a block with med == 0 is copied.  The paper
 * is silent on normalisation; this is the reading the library uses.
 * d_in, d_out: complex64[n] device; may alias. */
jerk_status jerk_normalise(jerk_plan plan, const void *d_in, int64_t n, void *d_out, void *stream);

/* The FP64 taps of templates t0 .. t0+nt-1 (0 <= t0, t0+nt <= n_templates)
 * into d_out: complex128 (interleaved double) [nt][K], tap d at index d + bM,
 * zero outside the template's own half-width. */
jerk_status jerk_taps(jerk_plan plan, int32_t t0, int32_t nt, void *d_out, void *stream);

/* Power plane rows P[t][p] = |O_p(z_t, w_t)|^2 for templates t0 .. t0+nt-1
 * and every cell p < b n, computed by the same fused overlap-and-save
 * kernel as jerk_search, written to d_out: float32[nt][b n] (device).
 * The spectrum is normalised first when norm_block > 0. */
jerk_status jerk_plane(jerk_plan plan, const void *d_spec, int64_t n, int32_t t0, int32_t nt,
                       float *d_out, void *stream);

/* After a search: device pointer to the stage-`stage_idx` max-projection of
 * spectrum `item` (0 for jerk_search), uint64[n_cells] with
 * n_cells = floor((b n - 1)/H) + 1, each entry
 * (float bits of M_H(p)) << 32 | (0xFFFFFFFF - t).  Valid until the next
 * search on the plan. */
jerk_status jerk_maxproj(jerk_plan plan, int32_t item, int32_t stage_idx, const uint64_t **d_out, int64_t *n_cells);

/* After a search (synchronises it): for spectrum `item`, per stage mean and
 * standard deviation of S_H over its defined cells (computed only in SIGMA
 * mode, else 0) and the FP32 threshold applied.  Arrays of n_stages entries;
 * any may be NULL. */
jerk_status jerk_stats(jerk_plan plan, int32_t item, double *h_mean, double *h_std, float *h_theta);

/* ---- per-stage timing (the paper's run-time breakdown, Sec. 3 / Fig. 3) ---- */

enum { JERK_N_PHASES = 5 };   /* normalise, conv (fused filter + stage-1), harmonic, stats, peaks */

/* Enable (1) or disable (0) CUDA-event timing of the phases of each
 * jerk_search.  Off by default; costs five event records per search. */
jerk_status jerk_profile(jerk_plan plan, int32_t enable);

/* After a profiled search (synchronises it): milliseconds of each phase, in
 * the order of the enum above, into h_ms[0 .. min(n, JERK_N_PHASES)-1].
 * JERK_ESTATE if the last search was not profiled. */
jerk_status jerk_phase_times(jerk_plan plan, float *h_ms, int32_t n);

/* ---- the harmonic sum indexed by the highest harmonic ----
 *
 * Sec. 3 names the harmonic sum without defining it; the main path sums
 * over fundamentals (S_H above).  This is the other common form: for a top
 * harmonic at cell q of template t = (z, w),
 *   S'_H(q, t) = sum_{h=1..H} P(round(h q / H), z_h, w_h),
 * (z_h, w_h) = the grid point nearest to (h z / H, h w / H), halves rounded
 * away from zero in q, z and w; every template and every cell is a top
 * harmonic.  It needs the whole power plane, so it serves banks whose plane
 * fits on the device.  d_plane: float32[n_templates][b n] (device), the
 * planes of jerk_plane for t0 = 0, nt = n_templates.  Writes, for stage H
 * (1..8), d_maxproj (uint64[b n], device): the max over t of S'_H(q, t) in the
 * packed form of jerk_maxproj (FP32 sums in h order, lowest t on equal
 * values), and d_sums (double[2], device): the sum of S'_H and of S'_H^2 over
 * all templates and cells (for mu = d_sums[0] / (n_templates b n) etc.).
 * Thresholds and peaks: jerk_peaks_noalloc on d_maxproj.  Enqueued on
 * `stream` after the plan's previous work; uses the plan's statistics
 * workspace, so it must not overlap another call on the same plan. */
jerk_status jerk_subharmonic(jerk_plan plan, const float *d_plane, int64_t n, int32_t H, uint64_t *d_maxproj,
                             double *d_sums, void *stream);

/* ---- candidate extraction without allocation (no counterpart in the paper) ----
 *
 * For callers that cannot allocate device memory at the point where they
 * extract candidates: a real-time stage that reserved all its memory before
 * observing started (an allocation there can synchronise the device), or a
 * program whose device memory belongs to another allocator.  It applies the
 * library's peak rule to one stage-H max-projection (the array jerk_maxproj
 * returns: n_cells packed entries (float bits << 32) | (0xFFFFFFFF - t)):
 * a cell p is kept when M(p) > theta, M(p) > M(p-1) and M(p) >= M(p+1), a
 * missing neighbour counting as -inf.  Kept cells are written in increasing
 * p to d_out (device, capacity cap records; r = p/2, z/w from the grid given
 * by zmax, dz, wmax, dw; stage = H) and their number to *d_count (device
 * int64; it may exceed cap, and then only the first cap are written).
 *
 * Nothing is allocated: the scratch (per-block counts and offsets) is a
 * fixed 512 KiB array inside the library that each GPU using the library
 * holds until the process exits.  n_cells above 2^27 is rejected with
 * JERK_EINVAL.  All calls share that array: calls that may overlap on a GPU
 * (other streams or host threads) race and must be serialised by the caller.
 * The first call on a device looks up the array's device address with that
 * device current; make it before starting any CUDA stream capture.  The
 * address is kept for the life of the process, so after cudaDeviceReset on a
 * device this call must not be used on that device again.  A cell whose
 * packed template index lies outside the grid (no template reached it) gets
 * z_idx = w_idx = -1 and z = w = 0, as in jerk_candidates.
 * Enqueued on `stream` on the current device; no host synchronisation. */
jerk_status jerk_peaks_noalloc(const uint64_t *d_maxproj, int64_t n_cells, float theta, int32_t stage,
                               int32_t zmax, int32_t dz, int32_t wmax, int32_t dw,
                               jerk_candidate *d_out, int64_t cap, int64_t *d_count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* JERK_H_ */
