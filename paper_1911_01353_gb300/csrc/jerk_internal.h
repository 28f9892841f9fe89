// Internal declarations shared by the translation units of libjerk.so.
#pragma once

#include <cstddef>

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <memory>
#include <vector>

#include "../../include/jerk.h"

namespace jerk {

// Device-side candidate record written by the peak kernel.
struct DevCand {
    int64_t p;
    int32_t t;
    int32_t stage_idx;
    float power;
    int32_t item;            // spectrum of the batch
};

// A fundamental template with its harmonic-row slots (h = 1 .. h_top).
struct FundEntry {
    int32_t t;
    int32_t top_stage;       // index of the highest stage at which t is a valid fundamental
    int64_t off[JERK_MAX_HARMONIC];   // slot offset (floats) of harmonic h = i + 1
};

// A group of templates processed together: templates with similar half-width
// share a tap offset bM and segment length V (processing indices tb..te-1 of
// the bank).  In a launch table, cta0 is the entry's first CTA and item the
// spectrum it works on.
struct ConvGroup {
    int32_t tb, te, V, bM, cta0, item;
};

// One spectrum of a launch (a batch of independent spectra, or just one).
struct ItemDesc {
    const float2 *spec;      // normalised spectrum, N bins
    int64_t N, bN;
    unsigned long long *M1;  // stage-1 max-projection of this spectrum
    const int64_t *slot_off; // [n_entries] harmonic-row offsets of this spectrum (floats)
    const int64_t *slot_len; // [n_entries] harmonic-row lengths
};

// Arguments of the fused overlap-and-save kernel.
struct ConvArgs {
    const ItemDesc *items;   // spectra of the launch
    const float2 *bank;      // [T][L] template spectra in processing order
    const int32_t *order;    // position -> template index t
    const int32_t *rows;     // position -> bank row; null: the identity.  A work entry's
                             // tb..te-1 are positions; when items search sub-grids of the
                             // bank, positions list the templates inside each sub-grid
    const ConvGroup *grp;    // [n_work + 1] (item, group) entries; grp[n_work].cta0 = total CTAs
    int32_t T, n_work;
    int32_t t0, nt;          // template range written in plane mode
    // search mode
    const int32_t *slot_beg; // [T + 1] CSR into the slot entries
    const int32_t *slot_h;
    float *slots;
    double *stat_part;       // [gridDim.y][gridDim.x][2]
    int *err;                // set to 1 when a bounded device wait expires
    int64_t slot_cap;        // floats of `slots` (bounds checks of the debug build)
    long long *chk;          // violation counter and first site (bounds checks of the debug build)
    // test hook of the debug build (jerk_check_inject): at template position
    // inject_pos of every CTA's group, 1 skips the template copy, 2 skips the
    // completion signal of the tensor-core step 1, 3 that of step 3, so that a
    // bounded wait expires; 0 (and the release build) does nothing
    int32_t inject, inject_pos;
    // plane mode
    float *plane;            // [nt][bN]
    int64_t plane_len;       // floats of `plane` (bounds checks of the debug build)
    // reduced-precision (tensor-core) filter
    const void *tc_const;    // 16-bit B operand (32 KB) then the twiddle table (float2 [64][64])
    const float *tc_cmax;    // max over the bank of max(|Re C|, |Im C|)
};

// The test hook: true when the debug build is asked to leave out event `mode`
// at template position `pos` of the CTA's group (always false in the release
// build, where the hook is compiled out).
#ifdef JERK_CHECKS
__device__ __forceinline__ bool inject_at(const ConvArgs &a, int mode, int pos) {
    return a.inject == mode && a.inject_pos == pos;
}
#else
__device__ __forceinline__ bool inject_at(const ConvArgs &, int, int) { return false; }
#endif

// Sites of the debug build's bounds checks (the first failing one is recorded).
enum CheckSite {
    kChkRowStore = 1,     // fused filter: harmonic-row store
    kChkPlaneStore = 2,   // fused filter: plane row store (plane mode)
    kChkMaxProj = 3,      // fused filter: stage-1 max-projection update
    kChkHarmCopy = 4,     // harmonic sum: bulk copy of a row chunk
    kChkHarmStore = 5,    // harmonic sum: max-projection store
    kChkTcRowStore = 6,   // tensor-core filter: harmonic-row store
    kChkTcPlaneStore = 7, // tensor-core filter: plane row store
    kChkTcMaxProj = 8,    // tensor-core filter: stage-1 max-projection update
};

// A template's harmonic-row slot entries (at most one per h), prefetched into
// shared memory: harmonic number, row offset (floats) and row length (cells).
struct RowEntries {
    int h[JERK_MAX_HARMONIC];
    int64_t off[JERK_MAX_HARMONIC], len[JERK_MAX_HARMONIC];
};

// Per-template metadata of the template pipeline, prefetched ahead by cp.async.
struct TplMeta {
    int t, e0, e1, pad;
};
// cp.async copies 4- and 8-byte fields straight into these structs: each field
// must sit at a multiple of its own size
static_assert(offsetof(RowEntries, off) % 8 == 0 && offsetof(RowEntries, len) % 8 == 0,
              "RowEntries: 8-byte fields must be 8-byte aligned");
static_assert(sizeof(TplMeta) == 16 && offsetof(TplMeta, e0) % 4 == 0, "TplMeta layout");

struct HarmArgs {
    const float *slots;
    const FundEntry *fund;
    int32_t n_fund;
    int32_t n_stages;
    int32_t stages[JERK_MAX_STAGES];
    int64_t n_cells[JERK_MAX_STAGES];     // floor((bN-1)/H) + 1
    unsigned long long *M[JERK_MAX_STAGES];
    double *stat_part;                     // [gridDim.x][n_stages][2]
    int32_t f_chunk;                       // fundamentals per block (y split)
    int *err;                              // set on an expired wait (JERK_ETIMEOUT)
    int64_t slot_cap;                      // floats of `slots` (bounds checks of the debug build)
    long long *chk;                        // violation counter and first site (debug build)
};

struct PeakArgs {
    const unsigned long long *M[JERK_MAX_STAGES];
    int64_t n_cells[JERK_MAX_STAGES];
    const float *theta;                    // device, per stage
    int32_t n_stages;
    int32_t item;
    DevCand *out;
    int64_t cap;
    unsigned long long *count;
};

// launchers (return cudaGetLastError())
cudaError_t launch_normalise(const float2 *in, float2 *out, int64_t n, int block, cudaStream_t st);
cudaError_t launch_taps(const int32_t *zt, const int32_t *wt, const int32_t *tlist, int32_t t0, int32_t nt, int b,
                        int pad, int bM, const double2 *gl, int n_gl, double2 *out, cudaStream_t st);
cudaError_t launch_template_fft(const double2 *taps, const int32_t *shift, const int32_t *klen, int32_t nt, int K,
                                int L, const double2 *tw, int fold_r0, float2 *bank, cudaStream_t st);
int conv_fold_radix(int log2L);      // radix of the FP32 filter's first inverse pass (the bank's folded form)
// the tensor-core filter's bank pairs spectrum values f and f + kTcBankPair
// (the two rows of a DFT block one thread multiplies together)
constexpr int kTcBankPair = 64;
cudaError_t launch_twiddles64(double2 *tw, int L, cudaStream_t st);
cudaError_t launch_conv(int log2L, int mode, bool stats, const ConvArgs &a, int n_ctas, cudaStream_t st);
cudaError_t launch_conv_tc(int precision, int mode, bool stats, const ConvArgs &a, int n_ctas, cudaStream_t st);
cudaError_t launch_bank_maxabs(const float2 *bank, int64_t n, float *out, int sms, cudaStream_t st);
int conv_segs_per_cta(int log2L);
cudaError_t launch_harmonic(const HarmArgs &a, int nblk_y, bool stats, cudaStream_t st);
int harmonic_cells_per_block();
cudaError_t launch_finalise_stats(const double *part1, int64_t n1, const double *partH, int64_t nH,
                                  int n_stages, const double *counts, const float *thresh, int mode,
                                  double *stats_out, float *theta_out, cudaStream_t st);
cudaError_t launch_peaks(const PeakArgs &a, int sms, cudaStream_t st);
cudaError_t launch_wait_check(int *err, uint64_t limit_ns, cudaStream_t st);
cudaError_t measure_peaks(int sms, double *fp32_tflops, double *l2_gbs);
cudaError_t measure_packed_fma(int sms, double *tflops);

// host helpers
int device_sms(int device);         // multiprocessor count of `device` (1 if the query fails)
int current_device_sms();           // the same for the current device
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w);

}  // namespace jerk

// Launch tables of one set of spectrum lengths (a batch, or one spectrum).
struct BatchLayout {
    std::vector<int64_t> n;                        // lengths: the cache key
    std::vector<int32_t> zmax, wmax;               // per-item sub-grids (empty: whole bank); part of the key
    int32_t t_lo = 0, t_hi = -1;                   // template range of a partial search (t_hi < 0: none); key
    int64_t stat_ctas = -1;                        // range search: conv CTAs whose statistics count (>= 0)
    std::vector<double> counts_host;               // [count][JERK_MAX_STAGES] cells counted by the statistics
    std::vector<int32_t> n_fund;                   // [count] fundamentals of each item (stages > 1)
    int64_t total_ctas = 0;
    int n_work = 0;
    std::vector<int64_t> item_cta0;                // [count + 1] conv CTAs of each item
    std::vector<int64_t> harm0;                    // [count + 1] harmonic partial blocks of each item
    std::vector<int64_t> spec_off;                 // [count] offset in the normalised-spectrum buffer
    std::vector<int64_t> m_off[JERK_MAX_STAGES];   // [count] offset in each max-projection buffer
    std::vector<int64_t> slot_base;                // [count + 1] harmonic-row floats of each item
    jerk::ItemDesc *d_items = nullptr;
    jerk::ConvGroup *d_work = nullptr;
    int64_t *d_soff = nullptr, *d_slen = nullptr;  // [count][n_entries]
    jerk::FundEntry *d_fund = nullptr;             // [count][n_fund]
    double *d_counts = nullptr;                    // [count][JERK_MAX_STAGES]
    int32_t *d_rows = nullptr;                     // position -> bank row (sub-grid layouts)
    int32_t *d_tl = nullptr;                       // position -> template index (sub-grid layouts)
    cudaGraphExec_t graph = nullptr;               // captured batch sequence
    uint64_t last_use = 0;                         // LRU stamp
};

// Bank-level device state that plans created by jerk_plan_share use
// together: the template spectra and the per-template tables.  Freed when the
// last plan holding it is destroyed.
struct BankShare {
    int device = 0;
    float2 *d_bank = nullptr;
    int32_t *d_zt = nullptr, *d_wt = nullptr, *d_order = nullptr;
    int32_t *d_slot_beg = nullptr, *d_slot_h = nullptr;
    double2 *d_gl = nullptr;
    float *d_cmax = nullptr;          // max(|Re|, |Im|) over the bank (set by jerk_templates)
    int64_t bytes = 0;
    std::atomic<bool> ready{false};   // jerk_templates has filled d_bank
    ~BankShare();
};

// Preallocated launch tables for JERK_BATCH_TRANSIENT searches: filled from
// pinned host staging by asynchronous copies, so a search allocates and frees
// nothing and never synchronises the device.
struct TransientTables {
    int64_t cap_work = 0, cap_ent = 0, cap_fund = 0, cap_rows = 0;
    void *h_stage = nullptr;          // pinned: items | work | soff | slen | fund | counts | rows
    void *d_buf = nullptr;            // device copy of the same layout
    size_t bytes = 0;
};

struct jerk_plan_s {
    jerk_params prm;
    int device;
    int sms = 1;                       // streaming multiprocessors of the device (grid sizing)
    int b, nz, nw, T, M, K, L, log2L, V;
    std::vector<int32_t> zt, wt, mt;   // grid values and per-template half-width
    // device memory; the bank-level arrays belong to `share`
    std::shared_ptr<BankShare> share;
    float2 *d_bank = nullptr;
    float2 *d_spec_in = nullptr;
    float2 *d_spec_norm = nullptr;
    unsigned long long *d_M[JERK_MAX_STAGES] = {nullptr, nullptr, nullptr, nullptr};
    float *d_slots = nullptr;
    int64_t slot_cap = 0;              // floats
    int32_t *d_zt = nullptr, *d_wt = nullptr;
    // template groups (fixed at plan creation) and their CTA prefix for the current n
    std::vector<int32_t> order;        // processing index -> t
    std::vector<int32_t> row_of;       // t -> processing index
    std::vector<jerk::ConvGroup> groups;
    int32_t *d_order = nullptr;
    void *d_tc = nullptr;              // tensor-core filter constants (precision 1, 2)
    float *d_cmax = nullptr;

    int32_t *d_slot_beg = nullptr, *d_slot_h = nullptr;
    int n_entries = 0, n_fund = 0;
    // harmonic-row structure (independent of n): entry e of the CSR (by
    // producing template) is harmonic ent_h[e] of fundamental ent_f[e]
    std::vector<int32_t> ent_f, ent_h, fund_t, fund_top;
    std::vector<int32_t> fh_entry;     // [n_fund][JERK_MAX_HARMONIC] -> entry (or -1)
    int32_t max_batch = 1;
    std::vector<BatchLayout *> layouts;   // tables of recently used sets of lengths (LRU)
    BatchLayout *cur = nullptr;           // tables of the last search
    BatchLayout transient_layout;         // host side of the transient tables
    TransientTables tt;
    uint64_t use_clock = 0;
    cudaStream_t cap_stream = nullptr; // private stream graphs are captured on
    double *d_stat_part = nullptr;     // conv partials then harmonic partials
    int64_t stat_part_cap = 0;         // doubles
    double *d_stats = nullptr;         // [n_stages][2]
    double *d_counts = nullptr;        // [n_stages]
    float *d_thresh = nullptr;         // [n_stages] user thresholds
    float *d_theta = nullptr;          // [n_stages] applied thresholds
    jerk::DevCand *d_cand = nullptr;
    unsigned long long *d_count = nullptr;
    int *d_err = nullptr;              // device error flag (bounded waits)
    long long *d_chk = nullptr;        // bounds-check violations and first site (debug build)
    int32_t inject = 0, inject_pos = 0;   // test hook of the debug build (jerk_check_inject)
    double2 *d_gl = nullptr;
    int n_gl = 0;
    int64_t bytes = 0;
    std::vector<int32_t> h_slot_beg, h_slot_h;
    // state
    int32_t last_count = 0;            // spectra of the last search
    bool searched = false;
    bool partial = false;              // the last search was a jerk_search_range (no candidates yet)
    cudaEvent_t done = nullptr;
    bool profile = false, profiled = false;
    cudaEvent_t ev[JERK_N_PHASES + 1] = {};
    jerk::DevCand *h_cand = nullptr;   // pinned staging for candidates
};
