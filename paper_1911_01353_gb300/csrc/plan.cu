// Host side of libjerk.so: parameter validation, plan sizing, the template
// bank, the launch sequence of a search (one spectrum or a batch of
// independent spectra, optionally replayed from a CUDA graph) and the
// candidate read-back.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "jerk_internal.h"

using namespace jerk;

BankShare::~BankShare() {
    int cur = -1;
    const bool had = cudaGetDevice(&cur) == cudaSuccess;
    cudaSetDevice(device);
    cudaFree(d_bank);
    cudaFree(d_zt);
    cudaFree(d_wt);
    cudaFree(d_order);
    cudaFree(d_slot_beg);
    cudaFree(d_slot_h);
    cudaFree(d_gl);
    cudaFree(d_cmax);
    if (had) cudaSetDevice(cur);
}

namespace {

constexpr size_t kGroupBytes = 32u << 20;   // bank slice a template group keeps in L2

jerk_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return JERK_OK;
    if (e == cudaErrorMemoryAllocation) return JERK_ENOMEM;
    return JERK_ECUDA;
}

#define JCHECK(x)                                    \
    do {                                             \
        cudaError_t e_ = (x);                        \
        if (e_ != cudaSuccess) return from_cuda(e_); \
    } while (0)

int halfwidth(int z, int w, int pad) { return (4 * std::abs(z) + std::abs(w) + 7) / 8 + pad; }

int64_t n_cells(int64_t bN, int H) { return (bN - 1) / H + 1; }

// passes of the transform (pass 0 + radix-16 passes) as a cost proxy
int fft_passes(int log2L) { return (log2L % 4) ? log2L / 4 + 1 : log2L / 4; }

bool valid_at(const jerk_plan_s *pl, int t, int H) {
    return (int64_t)H * std::abs(pl->zt[t]) <= pl->prm.zmax && (int64_t)H * std::abs(pl->wt[t]) <= pl->prm.wmax;
}

int index_of(const jerk_plan_s *pl, int z, int w) {
    const int i = (z + pl->prm.zmax) / pl->prm.dz;
    const int j = (w + pl->prm.wmax) / pl->prm.dw;
    return j * pl->nz + i;
}

int64_t round32(int64_t x) { return (x + 31) / 32 * 32; }

// Harmonic-row structure (independent of the spectrum length): for every
// harmonic h of every fundamental valid at the smallest stage >= max(h, 2),
// one row written by template (h z, h w); entries in CSR order by that template.
void build_row_structure(jerk_plan_s *pl) {
    const int ns = pl->prm.n_stages;
    struct Ent { int32_t t, f, h; };
    std::vector<Ent> ents;
    pl->fund_t.clear();
    pl->fund_top.clear();
    if (ns > 1) {
        for (int t = 0; t < pl->T; ++t) {
            int top = 0;
            for (int si = 1; si < ns; ++si)
                if (valid_at(pl, t, pl->prm.stages[si])) top = si;
            if (top == 0) continue;
            const int f = (int)pl->fund_t.size();
            pl->fund_t.push_back(t);
            pl->fund_top.push_back(top);
            for (int h = 1; h <= pl->prm.stages[top]; ++h)
                ents.push_back({index_of(pl, h * pl->zt[t], h * pl->wt[t]), f, h});
        }
    }
    std::stable_sort(ents.begin(), ents.end(), [](const Ent &x, const Ent &y) { return x.t < y.t; });
    pl->n_entries = (int)ents.size();
    pl->n_fund = (int)pl->fund_t.size();
    pl->h_slot_beg.assign(pl->T + 1, 0);
    pl->h_slot_h.resize(ents.size());
    pl->ent_f.resize(ents.size());
    pl->ent_h.resize(ents.size());
    pl->fh_entry.assign((size_t)pl->n_fund * JERK_MAX_HARMONIC, -1);
    for (size_t e = 0; e < ents.size(); ++e) {
        pl->h_slot_beg[ents[e].t + 1]++;
        pl->h_slot_h[e] = ents[e].h;
        pl->ent_f[e] = ents[e].f;
        pl->ent_h[e] = ents[e].h;
        pl->fh_entry[(size_t)ents[e].f * JERK_MAX_HARMONIC + ents[e].h - 1] = (int32_t)e;
    }
    for (int t = 0; t < pl->T; ++t) pl->h_slot_beg[t + 1] += pl->h_slot_beg[t];
}

bool valid_in(const jerk_plan_s *pl, int t, int H, int zs, int ws) {
    return (int64_t)H * std::abs(pl->zt[t]) <= zs && (int64_t)H * std::abs(pl->wt[t]) <= ws;
}

// Row offsets and lengths of one spectrum of n bins searched over the
// sub-grid |z| <= zs, |w| <= ws, whose rows start at `base` (floats); returns
// the floats used.  Rows are 128-byte aligned.  An entry whose fundamental is
// not a fundamental of the sub-grid at any stage > 1, or whose harmonic lies
// above the fundamental's top stage there, gets length 0 (the filter kernel
// skips it).  *nf receives the fundamentals written to `fund`, nf_stage[si]
// those valid at stage si.
int64_t item_rows(const jerk_plan_s *pl, int64_t n, int zs, int ws, int64_t base, int64_t *soff, int64_t *slen,
                  FundEntry *fund, int *nf, int64_t *nf_stage, int32_t t_lo = 0, int32_t t_hi = INT32_MAX) {
    const int64_t bN = (int64_t)pl->b * n;
    int64_t off = base;
    int k = 0;
    for (int f = 0; f < pl->n_fund; ++f) {
        const int t = pl->fund_t[f];
        int top = 0;
        for (int si = 1; si <= pl->fund_top[f]; ++si)
            if (valid_in(pl, t, pl->prm.stages[si], zs, ws)) top = si;
        if (t < t_lo || t >= t_hi) top = 0;           // a partial search's fundamentals: its range
        const int Hmaster = pl->prm.stages[pl->fund_top[f]];
        const int Htop = top ? pl->prm.stages[top] : 0;
        FundEntry fe;
        std::memset(&fe, 0, sizeof(fe));
        fe.t = t;
        fe.top_stage = top;
        for (int h = 1; h <= Hmaster; ++h) {
            const int e = pl->fh_entry[(size_t)f * JERK_MAX_HARMONIC + h - 1];
            int64_t len = 0;
            if (h <= Htop) {
                int sn = 1;
                while (pl->prm.stages[sn] < std::max(h, 2)) ++sn;
                len = n_cells(bN, pl->prm.stages[sn]);
            }
            fe.off[h - 1] = off;
            if (soff) soff[e] = off;
            if (slen) slen[e] = len;
            off += round32(len);
        }
        if (top == 0) continue;
        if (nf_stage)
            for (int si = 1; si <= top; ++si) ++nf_stage[si];
        if (fund) fund[k] = fe;
        ++k;
    }
    if (nf) *nf = k;
    return off - base;
}

int nseg_for(const jerk_plan_s *pl, int64_t n) {
    const int64_t bN = (int64_t)pl->b * n;
    return (int)((bN + pl->V - 1) / pl->V);
}

int tpg_for(const jerk_plan_s *pl, int nseg, int nt) {
    if (pl->prm.group_size > 0) return std::max(1, std::min(pl->prm.group_size, nt));
    const int64_t target = (int64_t)pl->sms * 6;
    int64_t tpg = ((int64_t)nt * nseg + target - 1) / target;
    const int64_t cap = std::max<int64_t>(1, (int64_t)(kGroupBytes / ((size_t)pl->L * sizeof(float2))));
    tpg = std::min<int64_t>(std::max<int64_t>(tpg, 8), cap);
    tpg = std::min<int64_t>(tpg, nt);
    return (int)std::max<int64_t>(tpg, 1);
}

// Group templates by filter half-width: sort by (m_t, t), cut into runs of
// `tpg`, process each run in ascending t (so ties keep the lowest t).  A
// group's tap offset is b * max(m_t) and its segment length L - 2 b max(m_t).
void build_groups(jerk_plan_s *pl, int tpg) {
    std::vector<int32_t> idx(pl->T);
    for (int t = 0; t < pl->T; ++t) idx[t] = t;
    std::stable_sort(idx.begin(), idx.end(), [pl](int x, int y) { return pl->mt[x] < pl->mt[y]; });
    pl->order.clear();
    pl->groups.clear();
    for (int k0 = 0; k0 < pl->T; k0 += tpg) {
        const int k1 = std::min(pl->T, k0 + tpg);
        std::sort(idx.begin() + k0, idx.begin() + k1);
        int mg = 0;
        for (int k = k0; k < k1; ++k) mg = std::max(mg, pl->mt[idx[k]]);
        ConvGroup g;
        g.tb = k0;
        g.te = k1;
        g.bM = pl->b * mg;
        g.V = pl->L - 2 * g.bM;
        g.cta0 = 0;
        g.item = 0;
        pl->groups.push_back(g);
    }
    pl->order = idx;
    pl->row_of.assign(pl->T, 0);
    for (int k = 0; k < pl->T; ++k) pl->row_of[pl->order[k]] = k;
}

// conv CTAs one spectrum of n bins needs
int64_t ctas_for(const jerk_plan_s *pl, int64_t n) {
    const int64_t bN = (int64_t)pl->b * n;
    const int segs = conv_segs_per_cta(pl->log2L);
    int64_t c = 0;
    for (const auto &x : pl->groups) c += ((bN + x.V - 1) / x.V + segs - 1) / segs;
    return c;
}

// inverse transforms one search of n bins performs
int64_t transforms_for(const jerk_plan_s *pl, int64_t n) {
    const int64_t bN = (int64_t)pl->b * n;
    int64_t s = 0;
    for (const auto &x : pl->groups) s += (int64_t)(x.te - x.tb) * ((bN + x.V - 1) / x.V);
    return s;
}

int64_t harm_blocks_for(const jerk_plan_s *pl, int64_t n) {
    if (pl->prm.n_stages < 2) return 0;
    const int64_t cpb = harmonic_cells_per_block();
    return (n_cells((int64_t)pl->b * n, pl->prm.stages[1]) + cpb - 1) / cpb;
}

jerk_status validate(const jerk_params *p) {
    if (!p) return JERK_EINVAL;
    if (p->dz <= 0 || p->dw <= 0 || p->zmax < 0 || p->wmax < 0) return JERK_EINVAL;
    if (p->zmax % p->dz || p->wmax % p->dw) return JERK_EINVAL;
    if (p->zmax > 4096 || p->wmax > 32768) return JERK_EINVAL;
    if (p->numbetween != 2) return JERK_EINVAL;
    if (p->pad_bins < 1 || p->pad_bins > 1024) return JERK_EINVAL;
    if (p->n_stages < 1 || p->n_stages > JERK_MAX_STAGES) return JERK_EINVAL;
    if (p->stages[0] != 1) return JERK_EINVAL;
    for (int i = 1; i < p->n_stages; ++i)
        if (p->stages[i] <= p->stages[i - 1] || p->stages[i] > JERK_MAX_HARMONIC) return JERK_EINVAL;
    if (p->thresh_mode != JERK_THRESH_ABS && p->thresh_mode != JERK_THRESH_SIGMA) return JERK_EINVAL;
    for (int i = 0; i < p->n_stages; ++i)
        if (!std::isfinite(p->thresh[i])) return JERK_EINVAL;
    if (p->norm_block < 0 || p->norm_block > 4096) return JERK_EINVAL;
    if (p->precision < 0 || p->precision > 2) return JERK_EINVAL;
    if (p->precision != 0 && p->seg_len != 0 && p->seg_len != 4096) return JERK_EINVAL;   // 64 x 64 DFT blocks
    if (p->max_bins < 1 || p->max_bins > ((int64_t)1 << 29)) return JERK_EINVAL;
    if (p->max_candidates < 1 || p->max_candidates > ((int64_t)1 << 26)) return JERK_EINVAL;
    if (p->max_batch < 0 || p->max_batch > 4096) return JERK_EINVAL;
    if (p->group_size < 0 || p->group_size > 65536) return JERK_EINVAL;
    if (p->seg_len != 0 && (p->seg_len < 1024 || p->seg_len > 8192 || (p->seg_len & (p->seg_len - 1))))
        return JERK_EINVAL;
    return JERK_OK;
}

template <typename T>
cudaError_t dalloc(int64_t *bytes, T **ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)ptr, count * sizeof(T));
    if (e == cudaSuccess) *bytes += (int64_t)(count * sizeof(T));
    return e;
}

bool bank_ready(const jerk_plan_s *pl) { return pl->share && pl->share->ready.load(); }

constexpr size_t kMaxLayouts = 128;

void free_layout(BatchLayout &L) {
    if (L.graph) cudaGraphExecDestroy(L.graph);
    cudaFree(L.d_items);
    cudaFree(L.d_work);
    cudaFree(L.d_soff);
    cudaFree(L.d_slen);
    cudaFree(L.d_fund);
    cudaFree(L.d_counts);
    cudaFree(L.d_rows);
    cudaFree(L.d_tl);
    L = BatchLayout();
}

void release(jerk_plan_s *pl) {
    for (BatchLayout *L : pl->layouts) {
        free_layout(*L);
        delete L;
    }
    pl->layouts.clear();
    pl->cur = nullptr;
    if (pl->tt.d_buf) cudaFree(pl->tt.d_buf);
    if (pl->tt.h_stage) cudaFreeHost(pl->tt.h_stage);
    pl->tt = TransientTables();
    pl->share.reset();                 // the bank goes with the last plan using it
    pl->d_bank = nullptr;
    cudaFree(pl->d_spec_in);
    cudaFree(pl->d_spec_norm);
    for (auto &m : pl->d_M) cudaFree(m);
    cudaFree(pl->d_slots);
    cudaFree(pl->d_stat_part);
    cudaFree(pl->d_stats);
    cudaFree(pl->d_thresh);
    cudaFree(pl->d_theta);
    cudaFree(pl->d_cand);
    cudaFree(pl->d_count);
    cudaFree(pl->d_err);
    cudaFree(pl->d_chk);
    cudaFree(pl->d_tc);
    if (pl->h_cand) cudaFreeHost(pl->h_cand);
    if (pl->done) cudaEventDestroy(pl->done);
    for (auto &e : pl->ev)
        if (e) cudaEventDestroy(e);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
}

// phase marker i of a profiled search
cudaError_t mark(jerk_plan_s *pl, int i, cudaStream_t st, bool capturing) {
    return (pl->profile && !capturing) ? cudaEventRecord(pl->ev[i], st) : cudaSuccess;
}

// Host side of a batch's launch tables.  Items' device pointers are filled in
// once the tables' device addresses are known.
struct HostTables {
    std::vector<ItemDesc> items;
    std::vector<ConvGroup> work;
    std::vector<int64_t> soff, slen;
    std::vector<FundEntry> fund;
    std::vector<double> counts;
    std::vector<int32_t> rows, tl;   // sub-grid layouts: position -> bank row, template index
};

// Launch tables for spectra of lengths n, item i searched over |z| <= zm[i],
// |w| <= wm[i] (zm, wm empty: the whole bank).  Fills L's host fields and h.
//
// With t_hi >= 0 (one spectrum only) the tables are those of a partial search
// over the templates t_lo <= t < t_hi: its stage-1 templates are those of the
// range and its fundamentals (stages > 1) those of the range, whose harmonic
// rows are made by templates inside or outside it.  The conv work lists the
// range's templates of every group first, then the other templates that make
// one of those rows; only the first part's CTAs count in the statistics.
jerk_status plan_tables(jerk_plan_s *pl, BatchLayout &L, const std::vector<int64_t> &n,
                        const std::vector<int32_t> &zm, const std::vector<int32_t> &wm, HostTables &h,
                        int32_t t_lo = 0, int32_t t_hi = -1) {
    const int count = (int)n.size();
    const int ns = pl->prm.n_stages;
    const bool range = t_hi >= 0;
    const bool sub = !zm.empty() || range;
    if (range && (count != 1 || !zm.empty() || t_lo < 0 || t_hi > pl->T || t_lo >= t_hi)) return JERK_EINVAL;
    L.n = n;
    L.zmax = zm;
    L.wmax = wm;
    L.t_lo = t_lo;
    L.t_hi = t_hi;
    L.stat_ctas = -1;
    L.total_ctas = 0;
    L.item_cta0.assign(count + 1, 0);
    L.harm0.assign(count + 1, 0);
    L.spec_off.assign(count, 0);
    L.slot_base.assign(count + 1, 0);
    L.n_fund.assign(count, 0);
    for (int si = 0; si < ns; ++si) L.m_off[si].assign(count, 0);
    h.items.assign(count, ItemDesc());
    h.soff.assign((size_t)count * std::max(pl->n_entries, 1), 0);
    h.slen.assign(h.soff.size(), 0);
    h.fund.assign((size_t)count * std::max(pl->n_fund, 1), FundEntry());
    h.counts.assign((size_t)count * JERK_MAX_STAGES, 0.0);
    h.work.clear();
    h.rows.clear();
    h.tl.clear();
    int64_t spec = 0, m[JERK_MAX_STAGES] = {0, 0, 0, 0};
    const int segs = conv_segs_per_cta(pl->log2L);
    for (int i = 0; i < count; ++i) {
        const int zs = !zm.empty() ? zm[i] : pl->prm.zmax, ws = !zm.empty() ? wm[i] : pl->prm.wmax;
        const int64_t bN = (int64_t)pl->b * n[i];
        L.spec_off[i] = spec;
        spec += n[i];
        for (int si = 0; si < ns; ++si) {
            L.m_off[si][i] = m[si];
            m[si] += n_cells(bN, pl->prm.stages[si]);
        }
        int64_t nf_stage[JERK_MAX_STAGES] = {0, 0, 0, 0};
        int nf = 0;
        const int64_t used = item_rows(pl, n[i], zs, ws, L.slot_base[i], h.soff.data() + (size_t)i * pl->n_entries,
                                       h.slen.data() + (size_t)i * pl->n_entries,
                                       h.fund.data() + (size_t)i * pl->n_fund, &nf, nf_stage,
                                       range ? t_lo : 0, range ? t_hi : INT32_MAX);
        L.slot_base[i + 1] = L.slot_base[i] + used;
        L.n_fund[i] = nf;
        // conv work: this spectrum's (group, segment range) entries, item-major;
        // a sub-grid keeps, per group, the templates inside it (positions into `rows`)
        int64_t nt_item = 0;
        // a partial search: templates outside the range that make a row of a range fundamental
        std::vector<char> extra;
        if (range) {
            extra.assign(pl->T, 0);
            const int64_t *sl = h.slen.data() + (size_t)i * pl->n_entries;
            for (int t = 0; t < pl->T; ++t)
                if (t < t_lo || t >= t_hi)
                    for (int e = pl->h_slot_beg[t]; e < pl->h_slot_beg[t + 1]; ++e)
                        if (sl[e] > 0) extra[t] = 1;
        }
        for (int part = 0; part < (range ? 2 : 1); ++part) {
            if (part == 1) L.stat_ctas = L.total_ctas - L.item_cta0[i];
            for (const auto &g : pl->groups) {
                ConvGroup w = g;
                if (sub) {
                    w.tb = (int32_t)h.rows.size();
                    for (int k = g.tb; k < g.te; ++k) {
                        const int t = pl->order[k];
                        const bool in = range ? (part == 0 ? (t >= t_lo && t < t_hi) : extra[t] != 0)
                                              : (std::abs(pl->zt[t]) <= zs && std::abs(pl->wt[t]) <= ws);
                        if (in) {
                            h.rows.push_back(k);
                            h.tl.push_back(t);
                        }
                    }
                    w.te = (int32_t)h.rows.size();
                    if (w.te == w.tb) continue;
                }
                if (part == 0) nt_item += w.te - w.tb;
                w.cta0 = (int32_t)L.total_ctas;
                w.item = i;
                h.work.push_back(w);
                L.total_ctas += ((bN + g.V - 1) / g.V + segs - 1) / segs;
            }
        }
        L.item_cta0[i + 1] = L.total_ctas;
        L.harm0[i + 1] = L.harm0[i] + harm_blocks_for(pl, n[i]);
        h.counts[(size_t)i * JERK_MAX_STAGES] = (double)bN * nt_item;
        for (int si = 1; si < ns; ++si)
            h.counts[(size_t)i * JERK_MAX_STAGES + si] = (double)nf_stage[si] * n_cells(bN, pl->prm.stages[si]);
    }
    L.counts_host = h.counts;
    ConvGroup end;
    std::memset(&end, 0, sizeof(end));
    end.cta0 = (int32_t)L.total_ctas;
    h.work.push_back(end);
    L.n_work = (int)h.work.size() - 1;
    // capacity checks (the plan was sized for max_bins bins in total)
    if (spec > pl->prm.max_bins || L.slot_base[count] > pl->slot_cap ||
        2 * (L.total_ctas + (int64_t)ns * L.harm0[count]) > pl->stat_part_cap || L.total_ctas >= INT32_MAX)
        return JERK_ENOMEM;
    for (int si = 0; si < ns; ++si)
        if (m[si] > n_cells((int64_t)pl->b * pl->prm.max_bins, pl->prm.stages[si]) + pl->max_batch)
            return JERK_ENOMEM;
    return JERK_OK;
}

void fill_items(const jerk_plan_s *pl, const BatchLayout &L, HostTables &h) {
    for (size_t i = 0; i < L.n.size(); ++i) {
        ItemDesc &it = h.items[i];
        it.spec = pl->d_spec_norm + L.spec_off[i];
        it.N = L.n[i];
        it.bN = (int64_t)pl->b * L.n[i];
        it.M1 = pl->d_M[0] + L.m_off[0][i];
        it.slot_off = L.d_soff + i * pl->n_entries;
        it.slot_len = L.d_slen + i * pl->n_entries;
    }
}

// Cached tables: own device buffers, synchronous upload.
jerk_status build_layout(jerk_plan_s *pl, BatchLayout &L, const std::vector<int64_t> &n,
                         const std::vector<int32_t> &zm, const std::vector<int32_t> &wm, int32_t t_lo = 0,
                         int32_t t_hi = -1) {
    HostTables h;
    const jerk_status s = plan_tables(pl, L, n, zm, wm, h, t_lo, t_hi);
    if (s != JERK_OK) return s;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&L.d_items, sizeof(ItemDesc) * h.items.size());
    if (e == cudaSuccess) e = cudaMalloc(&L.d_work, sizeof(ConvGroup) * h.work.size());
    if (e == cudaSuccess) e = cudaMalloc(&L.d_soff, sizeof(int64_t) * h.soff.size());
    if (e == cudaSuccess) e = cudaMalloc(&L.d_slen, sizeof(int64_t) * h.slen.size());
    if (e == cudaSuccess) e = cudaMalloc(&L.d_fund, sizeof(FundEntry) * h.fund.size());
    if (e == cudaSuccess) e = cudaMalloc(&L.d_counts, sizeof(double) * h.counts.size());
    if (e == cudaSuccess && !h.rows.empty()) e = cudaMalloc(&L.d_rows, sizeof(int32_t) * h.rows.size());
    if (e == cudaSuccess && !h.tl.empty()) e = cudaMalloc(&L.d_tl, sizeof(int32_t) * h.tl.size());
    if (e != cudaSuccess) return from_cuda(e);
    fill_items(pl, L, h);
    auto up = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up(L.d_items, h.items.data(), sizeof(ItemDesc) * h.items.size());
    up(L.d_work, h.work.data(), sizeof(ConvGroup) * h.work.size());
    up(L.d_soff, h.soff.data(), sizeof(int64_t) * h.soff.size());
    up(L.d_slen, h.slen.data(), sizeof(int64_t) * h.slen.size());
    up(L.d_fund, h.fund.data(), sizeof(FundEntry) * h.fund.size());
    up(L.d_counts, h.counts.data(), sizeof(double) * h.counts.size());
    up(L.d_rows, h.rows.data(), sizeof(int32_t) * h.rows.size());
    up(L.d_tl, h.tl.data(), sizeof(int32_t) * h.tl.size());
    return from_cuda(e);
}

// Launch tables for a set of spectrum lengths (and sub-grids): reused from a
// small LRU cache, built on first use (a host synchronisation).
jerk_status ensure_layout(jerk_plan_s *pl, const std::vector<int64_t> &n, const std::vector<int32_t> &zm,
                          const std::vector<int32_t> &wm, cudaStream_t st, int32_t t_lo = 0, int32_t t_hi = -1) {
    for (BatchLayout *L : pl->layouts)
        if (L->n == n && L->zmax == zm && L->wmax == wm && L->t_lo == t_lo && L->t_hi == t_hi) {
            L->last_use = ++pl->use_clock;
            pl->cur = L;
            return JERK_OK;
        }
    JCHECK(cudaStreamSynchronize(st));
    BatchLayout *L = nullptr;
    if (pl->layouts.size() >= kMaxLayouts) {
        L = *std::min_element(pl->layouts.begin(), pl->layouts.end(),
                              [](const BatchLayout *x, const BatchLayout *y) { return x->last_use < y->last_use; });
        if (pl->cur == L) pl->cur = nullptr;
        free_layout(*L);
    } else {
        L = new (std::nothrow) BatchLayout();
        if (!L) return JERK_ENOMEM;
        pl->layouts.push_back(L);
    }
    const jerk_status s = build_layout(pl, *L, n, zm, wm, t_lo, t_hi);
    if (s != JERK_OK) {
        free_layout(*L);
        pl->layouts.erase(std::find(pl->layouts.begin(), pl->layouts.end(), L));
        if (pl->cur == L) pl->cur = nullptr;
        delete L;
        return s;
    }
    L->last_use = ++pl->use_clock;
    pl->cur = L;
    return JERK_OK;
}

jerk_status ensure_layout(jerk_plan_s *pl, const std::vector<int64_t> &n, cudaStream_t st) {
    static const std::vector<int32_t> none;
    return ensure_layout(pl, n, none, none, st);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Transient tables: built into the plan's preallocated buffers and uploaded by
// one asynchronous copy from pinned staging on `st`.  Waits (on the host) only
// for this plan's previous search, whose upload used the same staging.
jerk_status transient_layout(jerk_plan_s *pl, const std::vector<int64_t> &n, const std::vector<int32_t> &zm,
                             const std::vector<int32_t> &wm, cudaStream_t st) {
    TransientTables &tt = pl->tt;
    if (!tt.d_buf) {
        // capacity: max_batch items, each with every group, entry, fundamental and template
        const size_t mb = (size_t)pl->max_batch;
        tt.cap_work = (int64_t)(mb * pl->groups.size() + 1);
        tt.cap_ent = (int64_t)(mb * std::max(pl->n_entries, 1));
        tt.cap_fund = (int64_t)(mb * std::max(pl->n_fund, 1));
        tt.cap_rows = (int64_t)(mb * pl->T);
        tt.bytes = align256(sizeof(ItemDesc) * mb) + align256(sizeof(ConvGroup) * tt.cap_work) +
                   2 * align256(sizeof(int64_t) * tt.cap_ent) + align256(sizeof(FundEntry) * tt.cap_fund) +
                   align256(sizeof(double) * mb * JERK_MAX_STAGES) + 2 * align256(sizeof(int32_t) * tt.cap_rows);
        cudaError_t e = cudaMalloc(&tt.d_buf, tt.bytes);
        if (e == cudaSuccess) e = cudaMallocHost(&tt.h_stage, tt.bytes);
        if (e != cudaSuccess) {
            if (tt.d_buf) cudaFree(tt.d_buf);
            tt = TransientTables();
            return from_cuda(e);
        }
        pl->bytes += (int64_t)tt.bytes;
    }
    BatchLayout &L = pl->transient_layout;
    HostTables h;
    const jerk_status s = plan_tables(pl, L, n, zm, wm, h);
    if (s != JERK_OK) return s;
    if ((int64_t)h.work.size() > tt.cap_work || (int64_t)h.rows.size() > tt.cap_rows) return JERK_ENOMEM;
    // section offsets (capacity-sized, so the device pointers never move)
    const size_t mb = (size_t)pl->max_batch;
    char *d0 = (char *)tt.d_buf;
    size_t o = 0;
    const size_t o_items = o;  o += align256(sizeof(ItemDesc) * mb);
    const size_t o_work = o;   o += align256(sizeof(ConvGroup) * tt.cap_work);
    const size_t o_soff = o;   o += align256(sizeof(int64_t) * tt.cap_ent);
    const size_t o_slen = o;   o += align256(sizeof(int64_t) * tt.cap_ent);
    const size_t o_fund = o;   o += align256(sizeof(FundEntry) * tt.cap_fund);
    const size_t o_counts = o; o += align256(sizeof(double) * mb * JERK_MAX_STAGES);
    const size_t o_rows = o;   o += align256(sizeof(int32_t) * tt.cap_rows);
    const size_t o_tl = o;
    L.d_items = (ItemDesc *)(d0 + o_items);
    L.d_work = (ConvGroup *)(d0 + o_work);
    L.d_soff = (int64_t *)(d0 + o_soff);
    L.d_slen = (int64_t *)(d0 + o_slen);
    L.d_fund = (FundEntry *)(d0 + o_fund);
    L.d_counts = (double *)(d0 + o_counts);
    L.d_rows = h.rows.empty() ? nullptr : (int32_t *)(d0 + o_rows);
    L.d_tl = h.tl.empty() ? nullptr : (int32_t *)(d0 + o_tl);
    L.graph = nullptr;
    fill_items(pl, L, h);
    JCHECK(cudaEventSynchronize(pl->done));   // the previous upload has left the staging buffer
    char *h0 = (char *)tt.h_stage;
    std::memcpy(h0 + o_items, h.items.data(), sizeof(ItemDesc) * h.items.size());
    std::memcpy(h0 + o_work, h.work.data(), sizeof(ConvGroup) * h.work.size());
    std::memcpy(h0 + o_soff, h.soff.data(), sizeof(int64_t) * h.soff.size());
    std::memcpy(h0 + o_slen, h.slen.data(), sizeof(int64_t) * h.slen.size());
    std::memcpy(h0 + o_fund, h.fund.data(), sizeof(FundEntry) * h.fund.size());
    std::memcpy(h0 + o_counts, h.counts.data(), sizeof(double) * h.counts.size());
    if (!h.rows.empty()) {
        std::memcpy(h0 + o_rows, h.rows.data(), sizeof(int32_t) * h.rows.size());
        std::memcpy(h0 + o_tl, h.tl.data(), sizeof(int32_t) * h.tl.size());
    }
    const size_t used = h.rows.empty() ? o_rows : o_tl + sizeof(int32_t) * h.tl.size();
    JCHECK(cudaMemcpyAsync(tt.d_buf, tt.h_stage, used, cudaMemcpyHostToDevice, st));
    pl->cur = &L;
    return JERK_OK;
}

// Enqueue the whole path for the spectra of the current layout.  in[i] is
// spectrum i (device).  Capturable into a CUDA graph (no host copies, no
// host synchronisation, no event waits).
jerk_status enqueue_peaks(jerk_plan_s *pl, cudaStream_t st);

jerk_status enqueue_search(jerk_plan_s *pl, const float2 *const *in, cudaStream_t st, bool capturing,
                           bool peaks = true) {
    const BatchLayout &L = *pl->cur;
    const int count = (int)L.n.size();
    const int ns = pl->prm.n_stages;
    const bool sigma = pl->prm.thresh_mode == JERK_THRESH_SIGMA;

    JCHECK(mark(pl, 0, st, capturing));
    for (int i = 0; i < count; ++i) {
        float2 *dst = pl->d_spec_norm + L.spec_off[i];
        if (pl->prm.norm_block > 0)
            JCHECK(launch_normalise(in[i], dst, L.n[i], pl->prm.norm_block, st));
        else if (in[i] != dst)
            JCHECK(cudaMemcpyAsync(dst, in[i], sizeof(float2) * L.n[i], cudaMemcpyDeviceToDevice, st));
    }
    for (int si = 0; si < ns; ++si) {
        const int64_t used = L.m_off[si][count - 1] + n_cells((int64_t)pl->b * L.n[count - 1], pl->prm.stages[si]);
        JCHECK(cudaMemsetAsync(pl->d_M[si], 0, sizeof(unsigned long long) * used, st));
    }
    JCHECK(mark(pl, 1, st, capturing));

    // fused overlap-and-save + stage-1 max-projection + harmonic rows, all spectra in one launch
    ConvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.items = L.d_items;
    a.bank = pl->d_bank;
    a.order = L.d_tl ? L.d_tl : pl->d_order;
    a.rows = L.d_rows;
    a.grp = L.d_work;
    a.n_work = L.n_work;
    a.T = pl->T;
    a.t0 = 0;
    a.nt = pl->T;
    a.slot_beg = pl->d_slot_beg;
    a.slot_h = pl->d_slot_h;
    a.slots = pl->d_slots;
    a.stat_part = pl->d_stat_part;
    a.err = pl->d_err;
    a.chk = pl->d_chk;
    a.inject = pl->inject;
    a.inject_pos = pl->inject_pos;
    a.slot_cap = pl->slot_cap;
    a.tc_const = pl->d_tc;
    a.tc_cmax = pl->d_cmax;
    JCHECK(pl->prm.precision ? launch_conv_tc(pl->prm.precision, 0, sigma, a, (int)L.total_ctas, st)
                             : launch_conv(pl->log2L, 0, sigma, a, (int)L.total_ctas, st));
    JCHECK(mark(pl, 2, st, capturing));

    // harmonic sums for stages > 1, per spectrum
    double *partH = pl->d_stat_part + 2 * L.total_ctas;
    if (ns > 1) {
        for (int i = 0; i < count; ++i) {
            const int64_t bN = (int64_t)pl->b * L.n[i];
            HarmArgs h;
            std::memset(&h, 0, sizeof(h));
            h.slots = pl->d_slots;
            h.fund = L.d_fund + (size_t)i * pl->n_fund;
            h.n_fund = L.n_fund[i];
            h.n_stages = ns;
            for (int si = 0; si < ns; ++si) {
                h.stages[si] = pl->prm.stages[si];
                h.n_cells[si] = n_cells(bN, pl->prm.stages[si]);
                h.M[si] = pl->d_M[si] + L.m_off[si][i];
            }
            h.stat_part = partH + 2 * ns * L.harm0[i];
            h.f_chunk = L.n_fund[i];
            h.err = pl->d_err;
            h.chk = pl->d_chk;
            h.slot_cap = pl->slot_cap;
            JCHECK(launch_harmonic(h, 1, sigma, st));
        }
    }
    JCHECK(mark(pl, 3, st, capturing));
    for (int i = 0; i < count; ++i)
        JCHECK(launch_finalise_stats(pl->d_stat_part + 2 * L.item_cta0[i],
                                     L.stat_ctas >= 0 ? L.stat_ctas : L.item_cta0[i + 1] - L.item_cta0[i],
                                     partH + 2 * ns * L.harm0[i], L.harm0[i + 1] - L.harm0[i], ns,
                                     L.d_counts + (size_t)i * JERK_MAX_STAGES, pl->d_thresh, pl->prm.thresh_mode,
                                     pl->d_stats + (size_t)i * 2 * JERK_MAX_STAGES,
                                     pl->d_theta + (size_t)i * JERK_MAX_STAGES, st));

    // peaks
    JCHECK(mark(pl, 4, st, capturing));
    if (peaks) {
        const jerk_status ps = enqueue_peaks(pl, st);
        if (ps != JERK_OK) return ps;
    }
    JCHECK(mark(pl, 5, st, capturing));
    return JERK_OK;
}

// thresholded peaks of every spectrum of the current layout (Sec. 3)
jerk_status enqueue_peaks(jerk_plan_s *pl, cudaStream_t st) {
    const BatchLayout &L = *pl->cur;
    const int count = (int)L.n.size();
    const int ns = pl->prm.n_stages;
    JCHECK(cudaMemsetAsync(pl->d_count, 0, sizeof(unsigned long long), st));
    for (int i = 0; i < count; ++i) {
        const int64_t bN = (int64_t)pl->b * L.n[i];
        PeakArgs pk;
        std::memset(&pk, 0, sizeof(pk));
        for (int si = 0; si < ns; ++si) {
            pk.M[si] = pl->d_M[si] + L.m_off[si][i];
            pk.n_cells[si] = n_cells(bN, pl->prm.stages[si]);
        }
        pk.theta = pl->d_theta + (size_t)i * JERK_MAX_STAGES;
        pk.n_stages = ns;
        pk.item = i;
        pk.out = pl->d_cand;
        pk.cap = pl->prm.max_candidates;
        pk.count = pl->d_count;
        JCHECK(launch_peaks(pk, pl->sms, st));
    }
    return JERK_OK;
}

// after a synchronisation point: did a bounded device wait expire?
jerk_status device_error(jerk_plan_s *pl) {
    int err = 0;
    JCHECK(cudaMemcpy(&err, pl->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        cudaMemset(pl->d_err, 0, sizeof(int));
        return JERK_ETIMEOUT;
    }
    return JERK_OK;
}

jerk_status finish_search(jerk_plan_s *pl, cudaStream_t st, int count, bool profiled) {
    JCHECK(cudaEventRecord(pl->done, st));
    pl->last_count = count;
    pl->searched = true;
    pl->profiled = profiled;
    pl->partial = false;
    return JERK_OK;
}

// ---- plan construction ------------------------------------------------------

// Constants of the tensor-core filter (L = 4096 = 64 x 64): the real block
// form of F[a][b] = exp(+2 pi i a b / 64),
//   B[kk][c] = [[Re F, Im F], [-Im F, Re F]]  (kk: re | im of the input index,
//                                               c: re | im of the output index),
// as a 16-bit (BF16 for precision 1, FP16 for 2) K-major 128 x 128 operand in
// 8 x 8 core matrices (128 B apart along K, 2048 B along N), followed by the
// twiddle table tw[n2][k1] = exp(+2 pi i k1 n2 / 4096), stored for two rows
// n2 = 2p, 2p + 1 at a time as float4 [p][k1] = (Re tw[2p][k1], Re tw[2p+1][k1],
// Im tw[2p][k1], Im tw[2p+1][k1]) so that one 16-byte load feeds a packed
// complex product of two cells.  FP64 arithmetic, rounded once.
std::vector<unsigned char> tc_constants(int precision) {
    const double two_pi = 6.283185307179586476925286766559;
    std::vector<unsigned char> out(128 * 128 * 2 + 64 * 64 * 8, 0);
    for (int kk = 0; kk < 128; ++kk)
        for (int c = 0; c < 128; ++c) {
            const int a = kk & 63, bcol = c & 63;
            const double ang = two_pi * (double)((a * bcol) % 64) / 64.0;
            const double re = std::cos(ang), im = std::sin(ang);
            double v;
            if (kk < 64) v = c < 64 ? re : im;
            else v = c < 64 ? -im : re;
            uint16_t bits;
            if (precision == 1) {
                const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
                std::memcpy(&bits, &h, 2);
            } else {
                const __half h = __float2half_rn((float)v);
                std::memcpy(&bits, &h, 2);
            }
            const size_t off = (size_t)(c >> 3) * 2048 + (size_t)(kk >> 3) * 128 + (size_t)(c & 7) * 16 + (size_t)(kk & 7) * 2;
            std::memcpy(out.data() + off, &bits, 2);
        }
    float *tw = reinterpret_cast<float *>(out.data() + 128 * 128 * 2);
    for (int n2 = 0; n2 < 64; ++n2)
        for (int k1 = 0; k1 < 64; ++k1) {
            const double ang = two_pi * (double)(k1 * n2) / 4096.0;
            float *e = tw + 4 * ((n2 >> 1) * 64 + k1) + (n2 & 1);
            e[0] = (float)std::cos(ang);
            e[2] = (float)std::sin(ang);
        }
    return out;
}

// Grid values, segment length, template groups and harmonic-row structure of
// pl->prm (host only).
jerk_status plan_structure(jerk_plan_s *pl) {
    const jerk_params *params = &pl->prm;
    pl->b = params->numbetween;
    pl->nz = 2 * params->zmax / params->dz + 1;
    pl->nw = 2 * params->wmax / params->dw + 1;
    pl->T = pl->nz * pl->nw;
    pl->zt.resize(pl->T);
    pl->wt.resize(pl->T);
    pl->mt.resize(pl->T);
    pl->M = 0;
    for (int j = 0; j < pl->nw; ++j)
        for (int i = 0; i < pl->nz; ++i) {
            const int t = j * pl->nz + i;
            pl->zt[t] = -params->zmax + i * params->dz;
            pl->wt[t] = -params->wmax + j * params->dw;
            pl->mt[t] = halfwidth(pl->zt[t], pl->wt[t], params->pad_bins);
            pl->M = std::max(pl->M, pl->mt[t]);
        }
    pl->K = 2 * pl->b * pl->M + 1;
    if (params->precision != 0) {
        pl->L = 4096;                          // the tensor-core filter is built for 64 x 64 DFT blocks
    } else if (params->seg_len) {
        pl->L = params->seg_len;
    } else {
        double best = 1e300;
        for (int lg = 10; lg <= 13; ++lg) {
            const int L = 1 << lg, V = L - pl->K + 1;
            if (V < L / 4) continue;
            const double cost = (fft_passes(lg) + 1.0) * L / V;
            if (cost < best - 1e-9) {
                best = cost;
                pl->L = L;
            }
        }
        if (best >= 1e300) return JERK_EINVAL;
    }
    pl->log2L = 0;
    while ((1 << pl->log2L) < pl->L) ++pl->log2L;
    pl->V = pl->L - pl->K + 1;
    if (pl->V < 64) return JERK_EINVAL;
    build_row_structure(pl);
    build_groups(pl, tpg_for(pl, nseg_for(pl, params->max_bins), pl->T));
    return JERK_OK;
}

// Device memory of a plan: with own_bank, the template bank and per-template
// tables (a new BankShare); always the workspace a search writes, sized for
// any set of at most max_batch spectra totalling at most max_bins bins.
jerk_status plan_memory(jerk_plan_s *pl, bool own_bank) {
    const jerk_params *params = &pl->prm;
    const int64_t N = params->max_bins, bN = (int64_t)pl->b * N;
    const int ns = params->n_stages;
    // (rows, CTAs and harmonic blocks grow with n; each extra spectrum adds rounding)
    pl->slot_cap = item_rows(pl, N, params->zmax, params->wmax, 0, nullptr, nullptr, nullptr, nullptr, nullptr) +
                   (int64_t)pl->max_batch * 32 * std::max(1, pl->n_fund * JERK_MAX_HARMONIC);
    const int64_t conv_blocks = ctas_for(pl, N) + (int64_t)pl->max_batch * (int64_t)pl->groups.size();
    const int64_t harm_blocks = harm_blocks_for(pl, N) + pl->max_batch;
    // (a partial search by template range runs each group's templates of the range
    // and, separately, the other templates its fundamentals need: up to twice the CTAs)
    pl->stat_part_cap = 2 * 2 * conv_blocks + 2 * (int64_t)ns * harm_blocks;

    // does it fit?
    size_t free_b = 0, total_b = 0;
    JCHECK(cudaMemGetInfo(&free_b, &total_b));
    int64_t need = 2 * N * 8 + pl->slot_cap * 4 + pl->stat_part_cap * 8 +
                   params->max_candidates * (int64_t)sizeof(DevCand);
    if (own_bank) need += (int64_t)pl->T * pl->L * 8 + (int64_t)pl->T * 40;
    for (int si = 0; si < ns; ++si) need += (n_cells(bN, params->stages[si]) + pl->max_batch) * 8;
    if ((double)need > 0.97 * (double)free_b) return JERK_ENOMEM;

    cudaError_t e = cudaSuccess;
#define TRY(x) \
    if (e == cudaSuccess) e = (x)
    if (own_bank) {
        BankShare *sh = new (std::nothrow) BankShare();
        if (!sh) return JERK_ENOMEM;
        sh->device = pl->device;
        pl->share.reset(sh);
        TRY(dalloc(&sh->bytes, &sh->d_bank, (size_t)pl->T * pl->L));
        TRY(dalloc(&sh->bytes, &sh->d_zt, (size_t)pl->T));
        TRY(dalloc(&sh->bytes, &sh->d_order, (size_t)pl->T));
        TRY(dalloc(&sh->bytes, &sh->d_wt, (size_t)pl->T));
        TRY(dalloc(&sh->bytes, &sh->d_slot_beg, (size_t)pl->T + 1));
        TRY(dalloc(&sh->bytes, &sh->d_slot_h, (size_t)pl->n_entries));
        TRY(dalloc(&sh->bytes, &sh->d_gl, 64));
        TRY(dalloc(&sh->bytes, &sh->d_cmax, 1));
        TRY(cudaMemcpy(sh->d_zt, pl->zt.data(), sizeof(int32_t) * pl->T, cudaMemcpyHostToDevice));
        TRY(cudaMemcpy(sh->d_order, pl->order.data(), sizeof(int32_t) * pl->T, cudaMemcpyHostToDevice));
        TRY(cudaMemcpy(sh->d_wt, pl->wt.data(), sizeof(int32_t) * pl->T, cudaMemcpyHostToDevice));
        TRY(cudaMemcpy(sh->d_slot_beg, pl->h_slot_beg.data(), sizeof(int32_t) * (pl->T + 1),
                       cudaMemcpyHostToDevice));
        if (pl->n_entries)
            TRY(cudaMemcpy(sh->d_slot_h, pl->h_slot_h.data(), sizeof(int32_t) * pl->n_entries,
                           cudaMemcpyHostToDevice));
        if (e == cudaSuccess) {
            std::vector<double> x, w;
            gauss_legendre(64, x, w);
            std::vector<double2> gl(64);
            for (int i = 0; i < 64; ++i) gl[i] = make_double2(x[i], w[i]);
            e = cudaMemcpy(sh->d_gl, gl.data(), sizeof(double2) * 64, cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess) {
        const BankShare *sh = pl->share.get();
        pl->d_bank = sh->d_bank;
        pl->d_zt = sh->d_zt;
        pl->d_wt = sh->d_wt;
        pl->d_order = sh->d_order;
        pl->d_slot_beg = sh->d_slot_beg;
        pl->d_slot_h = sh->d_slot_h;
        pl->d_gl = sh->d_gl;
        pl->d_cmax = sh->d_cmax;
        pl->n_gl = 64;
    }
    if (params->precision != 0 && e == cudaSuccess) {
        const std::vector<unsigned char> c = tc_constants(params->precision);
        TRY(cudaMalloc(&pl->d_tc, c.size()));
        if (e == cudaSuccess) pl->bytes += (int64_t)c.size();
        TRY(cudaMemcpy(pl->d_tc, c.data(), c.size(), cudaMemcpyHostToDevice));
    }
    TRY(dalloc(&pl->bytes, &pl->d_spec_in, (size_t)N));
    TRY(dalloc(&pl->bytes, &pl->d_spec_norm, (size_t)N));
    for (int si = 0; si < ns; ++si)
        TRY(dalloc(&pl->bytes, &pl->d_M[si], (size_t)(n_cells(bN, params->stages[si]) + pl->max_batch)));
    TRY(dalloc(&pl->bytes, &pl->d_slots, (size_t)pl->slot_cap));
    TRY(dalloc(&pl->bytes, &pl->d_stat_part, (size_t)pl->stat_part_cap));
    TRY(dalloc(&pl->bytes, &pl->d_stats, (size_t)2 * JERK_MAX_STAGES * pl->max_batch));
    TRY(dalloc(&pl->bytes, &pl->d_thresh, (size_t)JERK_MAX_STAGES));
    TRY(dalloc(&pl->bytes, &pl->d_theta, (size_t)JERK_MAX_STAGES * pl->max_batch));
    TRY(dalloc(&pl->bytes, &pl->d_cand, (size_t)params->max_candidates));
    TRY(dalloc(&pl->bytes, &pl->d_count, 1));
    TRY(dalloc(&pl->bytes, &pl->d_err, 1));
    TRY(cudaMemset(pl->d_err, 0, sizeof(int)));
    TRY(dalloc(&pl->bytes, &pl->d_chk, 2));
    TRY(cudaMemset(pl->d_chk, 0, 2 * sizeof(long long)));
    TRY(cudaMallocHost((void **)&pl->h_cand, sizeof(DevCand) * (size_t)params->max_candidates));
    TRY(cudaEventCreateWithFlags(&pl->done, cudaEventDisableTiming));
    TRY(cudaMemcpy(pl->d_thresh, params->thresh, sizeof(float) * JERK_MAX_STAGES, cudaMemcpyHostToDevice));
#undef TRY
    return from_cuda(e);
}

}  // namespace

extern "C" {

const char *jerk_status_str(jerk_status s) {
    switch (s) {
        case JERK_OK: return "JERK_OK";
        case JERK_EINVAL: return "JERK_EINVAL: invalid argument";
        case JERK_ENOMEM: return "JERK_ENOMEM: out of memory";
        case JERK_ECUDA: return "JERK_ECUDA: CUDA error";
        case JERK_ETIMEOUT: return "JERK_ETIMEOUT: device wait expired";
        case JERK_EOVERFLOW: return "JERK_EOVERFLOW: candidate buffer too small";
        case JERK_ESTATE: return "JERK_ESTATE: call out of order";
    }
    return "unknown jerk_status";
}

jerk_status jerk_params_validate(const jerk_params *params) { return validate(params); }

jerk_status jerk_plan_create(const jerk_params *params, int device, jerk_plan *out) {
    if (!out) return JERK_EINVAL;
    *out = nullptr;
    jerk_status v = validate(params);
    if (v != JERK_OK) return v;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return JERK_EINVAL;
    JCHECK(cudaSetDevice(device));

    jerk_plan_s *pl = new (std::nothrow) jerk_plan_s();
    if (!pl) return JERK_ENOMEM;
    pl->prm = *params;
    pl->device = device;
    pl->sms = device_sms(device);
    pl->max_batch = std::max(1, params->max_batch);
    v = plan_structure(pl);
    if (v == JERK_OK) v = plan_memory(pl, true);
    if (v != JERK_OK) {
        release(pl);
        delete pl;
        return v;
    }
    *out = pl;
    return JERK_OK;
}

jerk_status jerk_plan_share(jerk_plan parent, const jerk_params *params, jerk_plan *out) {
    if (!out) return JERK_EINVAL;
    *out = nullptr;
    if (!parent) return JERK_EINVAL;
    jerk_status v = validate(params);
    if (v != JERK_OK) return v;
    const jerk_params &q = parent->prm;
    // the bank-defining parameters must be the parent's
    if (params->zmax != q.zmax || params->dz != q.dz || params->wmax != q.wmax || params->dw != q.dw ||
        params->numbetween != q.numbetween || params->pad_bins != q.pad_bins || params->n_stages != q.n_stages ||
        params->precision != q.precision || (params->seg_len != 0 && params->seg_len != parent->L))
        return JERK_EINVAL;
    for (int i = 0; i < q.n_stages; ++i)
        if (params->stages[i] != q.stages[i]) return JERK_EINVAL;
    JCHECK(cudaSetDevice(parent->device));

    jerk_plan_s *pl = new (std::nothrow) jerk_plan_s();
    if (!pl) return JERK_ENOMEM;
    pl->prm = *params;
    pl->prm.seg_len = parent->L;
    pl->device = parent->device;
    pl->sms = parent->sms;
    pl->max_batch = std::max(1, params->max_batch);
    // the parent's structure: its groups fix the tap offset baked into every bank row
    pl->b = parent->b;
    pl->nz = parent->nz;
    pl->nw = parent->nw;
    pl->T = parent->T;
    pl->M = parent->M;
    pl->K = parent->K;
    pl->L = parent->L;
    pl->log2L = parent->log2L;
    pl->V = parent->V;
    pl->zt = parent->zt;
    pl->wt = parent->wt;
    pl->mt = parent->mt;
    pl->order = parent->order;
    pl->row_of = parent->row_of;
    pl->groups = parent->groups;
    pl->n_entries = parent->n_entries;
    pl->n_fund = parent->n_fund;
    pl->ent_f = parent->ent_f;
    pl->ent_h = parent->ent_h;
    pl->fund_t = parent->fund_t;
    pl->fund_top = parent->fund_top;
    pl->fh_entry = parent->fh_entry;
    pl->h_slot_beg = parent->h_slot_beg;
    pl->h_slot_h = parent->h_slot_h;
    pl->share = parent->share;
    v = plan_memory(pl, false);
    if (v != JERK_OK) {
        release(pl);
        delete pl;
        return v;
    }
    *out = pl;
    return JERK_OK;
}

jerk_status jerk_plan_destroy(jerk_plan pl) {
    if (!pl) return JERK_OK;
    cudaSetDevice(pl->device);
    if (pl->done) cudaEventSynchronize(pl->done);
    release(pl);
    delete pl;
    return JERK_OK;
}

jerk_status jerk_plan_info(jerk_plan pl, jerk_info *info) {
    if (!pl || !info) return JERK_EINVAL;
    info->nz = pl->nz;
    info->nw = pl->nw;
    info->n_templates = pl->T;
    info->bank_halfwidth = pl->M;
    info->taps = pl->K;
    info->seg_len = pl->L;
    info->seg_valid = pl->V;
    info->device = pl->device;
    info->max_bins = pl->prm.max_bins;
    info->slot_floats = pl->slot_cap;
    info->workspace_bytes = pl->bytes;
    info->bank_bytes = pl->share ? pl->share->bytes : 0;
    info->transforms = transforms_for(pl, pl->prm.max_bins);
    info->n_groups = (int32_t)pl->groups.size();
    info->reserved = 0;
    info->d_bank = pl->d_bank;
    return JERK_OK;
}

jerk_status jerk_template_row(jerk_plan pl, int32_t t, int32_t *row, int32_t *tap_offset, int32_t *seg_valid) {
    if (!pl || t < 0 || t >= pl->T) return JERK_EINVAL;
    const int k = pl->row_of[t];
    const ConvGroup *g = nullptr;
    for (const auto &x : pl->groups)
        if (k >= x.tb && k < x.te) g = &x;
    if (!g) return JERK_EINVAL;
    if (row) *row = k;
    if (tap_offset) *tap_offset = g->bM;
    if (seg_valid) *seg_valid = g->V;
    return JERK_OK;
}

jerk_status jerk_taps(jerk_plan pl, int32_t t0, int32_t nt, void *d_out, void *stream) {
    if (!pl || !d_out || t0 < 0 || nt < 1 || (int64_t)t0 + nt > pl->T) return JERK_EINVAL;
    JCHECK(cudaSetDevice(pl->device));
    cudaStream_t st = (cudaStream_t)stream;
    JCHECK(launch_taps(pl->d_zt, pl->d_wt, nullptr, t0, nt, pl->b, pl->prm.pad_bins, pl->b * pl->M, pl->d_gl,
                       pl->n_gl, (double2 *)d_out, st));
    return JERK_OK;
}

jerk_status jerk_templates(jerk_plan pl, void *stream) {
    if (!pl) return JERK_EINVAL;
    JCHECK(cudaSetDevice(pl->device));
    cudaStream_t st = (cudaStream_t)stream;
    // per bank row (processing order): tap offset shift and filter length of its group
    std::vector<int32_t> shift(pl->T), klen(pl->T);
    for (const auto &g : pl->groups)
        for (int k = g.tb; k < g.te; ++k) {
            shift[k] = pl->b * pl->M - g.bM;
            klen[k] = 2 * g.bM + 1;
        }
    // process the bank in chunks so the FP64 tap buffer stays small
    const int chunk = std::max(1, std::min(pl->T, (int)((256u << 20) / ((size_t)pl->K * sizeof(double2)))));
    double2 *taps = nullptr, *tw = nullptr;
    int32_t *d_shift = nullptr, *d_klen = nullptr;
    JCHECK(cudaMallocAsync((void **)&taps, (size_t)chunk * pl->K * sizeof(double2), st));
    cudaError_t e = cudaMallocAsync((void **)&tw, (size_t)(pl->L / 2) * sizeof(double2), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_shift, sizeof(int32_t) * pl->T, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_klen, sizeof(int32_t) * pl->T, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_shift, shift.data(), sizeof(int32_t) * pl->T, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_klen, klen.data(), sizeof(int32_t) * pl->T, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_twiddles64(tw, pl->L, st);
    for (int k0 = 0; k0 < pl->T && e == cudaSuccess; k0 += chunk) {
        const int nt = std::min(chunk, pl->T - k0);
        e = launch_taps(pl->d_zt, pl->d_wt, pl->d_order + k0, 0, nt, pl->b, pl->prm.pad_bins, pl->b * pl->M,
                        pl->d_gl, pl->n_gl, taps, st);
        if (e == cudaSuccess)
            e = launch_template_fft(taps, d_shift + k0, d_klen + k0, nt, pl->K, pl->L, tw,
                                    pl->prm.precision ? -kTcBankPair : conv_fold_radix(pl->log2L),
                                    pl->d_bank + (size_t)k0 * pl->L, st);
    }
    if (e == cudaSuccess) e = launch_bank_maxabs(pl->d_bank, (int64_t)pl->T * pl->L, pl->d_cmax, pl->sms, st);
    cudaFreeAsync(taps, st);
    if (tw) cudaFreeAsync(tw, st);
    if (d_shift) cudaFreeAsync(d_shift, st);
    if (d_klen) cudaFreeAsync(d_klen, st);
    // the host vectors above must outlive the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
    JCHECK(cudaEventRecord(pl->done, st));
    pl->share->ready = true;
    return JERK_OK;
}

jerk_status jerk_normalise(jerk_plan pl, const void *d_in, int64_t n, void *d_out, void *stream) {
    if (!pl || !d_in || !d_out || n < 1) return JERK_EINVAL;
    if (pl->prm.norm_block < 1) return JERK_EINVAL;
    JCHECK(cudaSetDevice(pl->device));
    JCHECK(launch_normalise((const float2 *)d_in, (float2 *)d_out, n, pl->prm.norm_block, (cudaStream_t)stream));
    return JERK_OK;
}

jerk_status jerk_plane(jerk_plan pl, const void *d_spec, int64_t n, int32_t t0, int32_t nt, float *d_out,
                       void *stream) {
    if (!pl || !d_spec || !d_out || n < 1 || n > pl->prm.max_bins) return JERK_EINVAL;
    if (t0 < 0 || nt < 1 || (int64_t)t0 + nt > pl->T) return JERK_EINVAL;
    if (!bank_ready(pl)) return JERK_ESTATE;
    JCHECK(cudaSetDevice(pl->device));
    cudaStream_t st = (cudaStream_t)stream;
    JCHECK(cudaStreamWaitEvent(st, pl->done, 0));
    {
        const jerk_status ls = ensure_layout(pl, std::vector<int64_t>{n}, st);
        if (ls != JERK_OK) return ls;
    }
    if (pl->prm.norm_block > 0)
        JCHECK(launch_normalise((const float2 *)d_spec, pl->d_spec_norm, n, pl->prm.norm_block, st));
    else
        JCHECK(cudaMemcpyAsync(pl->d_spec_norm, d_spec, sizeof(float2) * n, cudaMemcpyDeviceToDevice, st));
    ConvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.items = pl->cur->d_items;
    a.bank = pl->d_bank;
    a.order = pl->d_order;
    a.grp = pl->cur->d_work;
    a.n_work = pl->cur->n_work;
    a.T = pl->T;
    a.t0 = t0;
    a.nt = nt;
    a.plane = d_out;
    a.err = pl->d_err;
    a.chk = pl->d_chk;
    a.inject = pl->inject;
    a.inject_pos = pl->inject_pos;
    a.plane_len = (int64_t)nt * 2 * n;
    a.slot_beg = pl->d_slot_beg;
    a.tc_const = pl->d_tc;
    a.tc_cmax = pl->d_cmax;
    JCHECK(pl->prm.precision ? launch_conv_tc(pl->prm.precision, 1, false, a, (int)pl->cur->total_ctas, st)
                             : launch_conv(pl->log2L, 1, false, a, (int)pl->cur->total_ctas, st));
    JCHECK(cudaEventRecord(pl->done, st));
    return JERK_OK;
}

jerk_status jerk_search(jerk_plan pl, const void *d_spec, int64_t n, void *stream) {
    if (!pl || !d_spec || n < 1 || n > pl->prm.max_bins) return JERK_EINVAL;
    if (!bank_ready(pl)) return JERK_ESTATE;
    JCHECK(cudaSetDevice(pl->device));
    cudaStream_t st = (cudaStream_t)stream;
    JCHECK(cudaStreamWaitEvent(st, pl->done, 0));
    jerk_status s = ensure_layout(pl, std::vector<int64_t>{n}, st);
    if (s != JERK_OK) return s;
    const float2 *in[1] = {(const float2 *)d_spec};
    s = enqueue_search(pl, in, st, false);
    if (s != JERK_OK) return s;
    return finish_search(pl, st, 1, pl->profile);
}

jerk_status jerk_search_range(jerk_plan pl, const void *d_spec, int64_t n, int32_t t_lo, int32_t t_hi,
                              void *stream) {
    if (!pl || !d_spec || n < 1 || n > pl->prm.max_bins) return JERK_EINVAL;
    if (t_lo < 0 || t_hi > pl->T || t_lo >= t_hi) return JERK_EINVAL;
    if (!bank_ready(pl)) return JERK_ESTATE;
    JCHECK(cudaSetDevice(pl->device));
    cudaStream_t st = (cudaStream_t)stream;
    JCHECK(cudaStreamWaitEvent(st, pl->done, 0));
    static const std::vector<int32_t> none;
    jerk_status s = ensure_layout(pl, std::vector<int64_t>{n}, none, none, st, t_lo, t_hi);
    if (s != JERK_OK) return s;
    const float2 *in[1] = {(const float2 *)d_spec};
    s = enqueue_search(pl, in, st, false, false);
    if (s != JERK_OK) return s;
    JCHECK(cudaMemsetAsync(pl->d_count, 0, sizeof(unsigned long long), st));   // no candidates yet
    s = finish_search(pl, st, 1, false);
    pl->partial = true;
    return s;
}

jerk_status jerk_range_sums(jerk_plan pl, double *h_sum, double *h_sumsq, double *h_count) {
    if (!pl) return JERK_EINVAL;
    if (!pl->searched || !pl->partial || !pl->cur) return JERK_ESTATE;
    JCHECK(cudaSetDevice(pl->device));
    JCHECK(cudaEventSynchronize(pl->done));
    const jerk_status de = device_error(pl);
    if (de != JERK_OK) return de;
    const int ns = pl->prm.n_stages;
    double st[2 * JERK_MAX_STAGES];
    JCHECK(cudaMemcpy(st, pl->d_stats, sizeof(double) * 2 * ns, cudaMemcpyDeviceToHost));
    for (int si = 0; si < ns; ++si) {
        // the sums behind (mu, sd) = (S1 / n, sqrt(S2 / n - mu^2)) as computed on the device
        const double cnt = pl->cur->counts_host[si], mu = st[2 * si], sd = st[2 * si + 1];
        if (h_sum) h_sum[si] = mu * cnt;
        if (h_sumsq) h_sumsq[si] = (sd * sd + mu * mu) * cnt;
        if (h_count) h_count[si] = cnt;
    }
    return JERK_OK;
}

jerk_status jerk_select(jerk_plan pl, const double *h_sum, const double *h_sumsq, const double *h_count,
                        void *stream) {
    if (!pl) return JERK_EINVAL;
    if (!pl->searched || !pl->cur || pl->cur->n.size() != 1) return JERK_ESTATE;
    const bool sigma = pl->prm.thresh_mode == JERK_THRESH_SIGMA;
    if (sigma && (!h_sum || !h_sumsq || !h_count)) return JERK_EINVAL;
    JCHECK(cudaSetDevice(pl->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int ns = pl->prm.n_stages;
    double stats[2 * JERK_MAX_STAGES] = {0};
    float theta[JERK_MAX_STAGES];
    for (int si = 0; si < ns; ++si) {
        // the same arithmetic as the device's finalisation of the statistics
        double mu = 0.0, sd = 0.0;
        theta[si] = pl->prm.thresh[si];
        if (sigma && h_count[si] > 0.0) {
            mu = h_sum[si] / h_count[si];
            const double var = h_sumsq[si] / h_count[si] - mu * mu;
            sd = std::sqrt(var > 0.0 ? var : 0.0);
            theta[si] = (float)(mu + (double)pl->prm.thresh[si] * sd);
        }
        stats[2 * si] = mu;
        stats[2 * si + 1] = sd;
    }
    JCHECK(cudaStreamWaitEvent(st, pl->done, 0));
    JCHECK(cudaMemcpyAsync(pl->d_stats, stats, sizeof(double) * 2 * ns, cudaMemcpyHostToDevice, st));
    JCHECK(cudaMemcpyAsync(pl->d_theta, theta, sizeof(float) * ns, cudaMemcpyHostToDevice, st));
    const jerk_status s = enqueue_peaks(pl, st);
    if (s != JERK_OK) return s;
    JCHECK(cudaStreamSynchronize(st));             // the host arrays above are on the stack
    JCHECK(cudaEventRecord(pl->done, st));
    pl->partial = false;
    return JERK_OK;
}

jerk_status jerk_search_batch_grid(jerk_plan pl, const void *const *d_specs, const int64_t *n, const int32_t *zmax,
                                   const int32_t *wmax, int32_t count, int32_t flags, void *stream) {
    if (!pl || !d_specs || !n || count < 1 || count > pl->max_batch) return JERK_EINVAL;
    if (flags & ~(JERK_BATCH_GRAPH | JERK_BATCH_TRANSIENT)) return JERK_EINVAL;
    if ((flags & JERK_BATCH_GRAPH) && (flags & JERK_BATCH_TRANSIENT)) return JERK_EINVAL;
    if ((zmax == nullptr) != (wmax == nullptr)) return JERK_EINVAL;
    int64_t total = 0;
    for (int i = 0; i < count; ++i) {
        if (!d_specs[i] || n[i] < 1) return JERK_EINVAL;
        total += n[i];
    }
    if (total > pl->prm.max_bins) return JERK_EINVAL;
    // sub-grids: on the bank's grid and inside it; all-whole-bank batches use the plain tables
    std::vector<int32_t> zm, wm;
    if (zmax) {
        bool whole = true;
        for (int i = 0; i < count; ++i) {
            if (zmax[i] < 0 || zmax[i] > pl->prm.zmax || zmax[i] % pl->prm.dz) return JERK_EINVAL;
            if (wmax[i] < 0 || wmax[i] > pl->prm.wmax || wmax[i] % pl->prm.dw) return JERK_EINVAL;
            whole = whole && zmax[i] == pl->prm.zmax && wmax[i] == pl->prm.wmax;
        }
        if (!whole) {
            zm.assign(zmax, zmax + count);
            wm.assign(wmax, wmax + count);
        }
    }
    if (!bank_ready(pl)) return JERK_ESTATE;
    JCHECK(cudaSetDevice(pl->device));
    cudaStream_t st = (cudaStream_t)stream;
    JCHECK(cudaStreamWaitEvent(st, pl->done, 0));
    const std::vector<int64_t> nv(n, n + count);
    jerk_status s = (flags & JERK_BATCH_TRANSIENT) ? transient_layout(pl, nv, zm, wm, st)
                                                   : ensure_layout(pl, nv, zm, wm, st);
    if (s != JERK_OK) return s;
    if (!(flags & JERK_BATCH_GRAPH)) {
        std::vector<const float2 *> in(count);
        for (int i = 0; i < count; ++i) in[i] = (const float2 *)d_specs[i];
        s = enqueue_search(pl, in.data(), st, false);
        if (s != JERK_OK) return s;
        return finish_search(pl, st, count, pl->profile);
    }
    // graph mode: the graph reads the spectra from the plan's input buffer,
    // so the caller's buffers may change from call to call
    BatchLayout &L = *pl->cur;
    std::vector<const float2 *> in(count);
    for (int i = 0; i < count; ++i) {
        float2 *dst = pl->d_spec_in + L.spec_off[i];
        JCHECK(cudaMemcpyAsync(dst, d_specs[i], sizeof(float2) * n[i], cudaMemcpyDeviceToDevice, st));
        in[i] = dst;
    }
    if (!L.graph) {
        // capture on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured); the graph is launched on `st`
        if (!pl->cap_stream) JCHECK(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        JCHECK(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal));
        s = enqueue_search(pl, in.data(), pl->cap_stream, true);
        cudaError_t ce = cudaStreamEndCapture(pl->cap_stream, &g);
        if (s != JERK_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (ce != cudaSuccess) return from_cuda(ce);
        ce = cudaGraphInstantiate(&L.graph, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) {
            L.graph = nullptr;
            return from_cuda(ce);
        }
    }
    JCHECK(cudaGraphLaunch(L.graph, st));
    return finish_search(pl, st, count, false);
}

jerk_status jerk_search_batch(jerk_plan pl, const void *const *d_specs, const int64_t *n, int32_t count,
                              int32_t flags, void *stream) {
    return jerk_search_batch_grid(pl, d_specs, n, nullptr, nullptr, count, flags, stream);
}

jerk_status jerk_search_host(jerk_plan pl, const void *h_spec, int64_t n, void *stream) {
    if (!pl || !h_spec || n < 1 || n > pl->prm.max_bins) return JERK_EINVAL;
    if (!bank_ready(pl)) return JERK_ESTATE;
    JCHECK(cudaSetDevice(pl->device));
    cudaStream_t st = (cudaStream_t)stream;
    JCHECK(cudaStreamWaitEvent(st, pl->done, 0));
    JCHECK(cudaMemcpyAsync(pl->d_spec_in, h_spec, (size_t)n * sizeof(float2), cudaMemcpyHostToDevice, st));
    return jerk_search(pl, pl->d_spec_in, n, stream);
}

jerk_status jerk_candidates(jerk_plan pl, jerk_candidate *h_out, int64_t cap, int64_t *n_out) {
    if (!pl || !n_out || cap < 0 || (cap > 0 && !h_out)) return JERK_EINVAL;
    if (!pl->searched || pl->partial) return JERK_ESTATE;
    JCHECK(cudaSetDevice(pl->device));
    JCHECK(cudaEventSynchronize(pl->done));
    {
        const jerk_status de = device_error(pl);
        if (de != JERK_OK) return de;
    }
    unsigned long long cnt = 0;
    JCHECK(cudaMemcpy(&cnt, pl->d_count, sizeof(cnt), cudaMemcpyDeviceToHost));
    const int64_t kept = std::min<int64_t>((int64_t)cnt, pl->prm.max_candidates);
    if (kept > 0)
        JCHECK(cudaMemcpy(pl->h_cand, pl->d_cand, sizeof(DevCand) * (size_t)kept, cudaMemcpyDeviceToHost));
    std::vector<DevCand> v(pl->h_cand, pl->h_cand + kept);
    std::sort(v.begin(), v.end(), [](const DevCand &x, const DevCand &y) {
        if (x.item != y.item) return x.item < y.item;
        return x.stage_idx != y.stage_idx ? x.stage_idx < y.stage_idx : x.p < y.p;
    });
    const int64_t ncopy = std::min<int64_t>(kept, cap);
    for (int64_t i = 0; i < ncopy; ++i) {
        jerk_candidate &c = h_out[i];
        const DevCand &d = v[i];
        const int t = d.t;
        c.p = d.p;
        c.r = (double)d.p / pl->b;
        c.t = t;
        c.z_idx = (t >= 0 && t < pl->T) ? t % pl->nz : -1;
        c.w_idx = (t >= 0 && t < pl->T) ? t / pl->nz : -1;
        c.stage = pl->prm.stages[d.stage_idx];
        c.z = (t >= 0 && t < pl->T) ? (float)pl->zt[t] : 0.f;
        c.w = (t >= 0 && t < pl->T) ? (float)pl->wt[t] : 0.f;
        c.power = d.power;
        c.item = d.item;
    }
    *n_out = (int64_t)cnt;
    if ((int64_t)cnt > pl->prm.max_candidates || (int64_t)cnt > cap) return JERK_EOVERFLOW;
    return JERK_OK;
}

jerk_status jerk_maxproj(jerk_plan pl, int32_t item, int32_t stage_idx, const uint64_t **d_out,
                         int64_t *n_cells_out) {
    if (!pl || !d_out || !n_cells_out || stage_idx < 0 || stage_idx >= pl->prm.n_stages) return JERK_EINVAL;
    if (!pl->searched) return JERK_ESTATE;
    if (!pl->cur || item < 0 || item >= pl->last_count || item >= (int)pl->cur->n.size()) return JERK_EINVAL;
    *d_out = (const uint64_t *)(pl->d_M[stage_idx] + pl->cur->m_off[stage_idx][item]);
    *n_cells_out = n_cells((int64_t)pl->b * pl->cur->n[item], pl->prm.stages[stage_idx]);
    return JERK_OK;
}

jerk_status jerk_profile(jerk_plan pl, int32_t enable) {
    if (!pl) return JERK_EINVAL;
    JCHECK(cudaSetDevice(pl->device));
    if (enable && !pl->ev[0])
        for (auto &e : pl->ev) JCHECK(cudaEventCreate(&e));
    pl->profile = enable != 0;
    return JERK_OK;
}

jerk_status jerk_phase_times(jerk_plan pl, float *h_ms, int32_t n) {
    if (!pl || !h_ms || n < 0) return JERK_EINVAL;
    if (!pl->searched || !pl->profiled) return JERK_ESTATE;
    JCHECK(cudaSetDevice(pl->device));
    JCHECK(cudaEventSynchronize(pl->done));
    for (int i = 0; i < n && i < JERK_N_PHASES; ++i) JCHECK(cudaEventElapsedTime(h_ms + i, pl->ev[i], pl->ev[i + 1]));
    return JERK_OK;
}

jerk_status jerk_measure_peaks(int device, double *fp32_tflops, double *l2_gbs) {
    if (!fp32_tflops || !l2_gbs) return JERK_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return JERK_EINVAL;
    JCHECK(cudaSetDevice(device));
    int sms = 0;
    JCHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    JCHECK(measure_peaks(sms, fp32_tflops, l2_gbs));
    return JERK_OK;
}

jerk_status jerk_measure_packed_fma(int device, double *tflops) {
    if (!tflops) return JERK_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return JERK_EINVAL;
    JCHECK(cudaSetDevice(device));
    int sms = 0;
    JCHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    JCHECK(measure_packed_fma(sms, tflops));
    return JERK_OK;
}

jerk_status jerk_check_waits(jerk_plan pl, int32_t limit_us, void *stream) {
    if (!pl || limit_us < 1 || limit_us > 1000000) return JERK_EINVAL;
    JCHECK(cudaSetDevice(pl->device));
    cudaStream_t st = (cudaStream_t)stream;
    JCHECK(cudaStreamWaitEvent(st, pl->done, 0));
    JCHECK(launch_wait_check(pl->d_err, (uint64_t)limit_us * 1000ull, st));
    JCHECK(cudaEventRecord(pl->done, st));
    JCHECK(cudaEventSynchronize(pl->done));
    return device_error(pl);          // JERK_ETIMEOUT, and the flag is cleared for the next search
}

jerk_status jerk_check_inject(jerk_plan pl, int32_t mode, int32_t position) {
    if (!pl || mode < 0 || mode > 3 || (mode > 0 && position < 3)) return JERK_EINVAL;
#ifdef JERK_CHECKS
    pl->inject = mode;
    pl->inject_pos = mode ? position : 0;
    return JERK_OK;
#else
    return JERK_ESTATE;
#endif
}

jerk_status jerk_check_counts(jerk_plan pl, int64_t *violations, int32_t *first_site, int32_t *compiled_in) {
    if (!pl) return JERK_EINVAL;
#ifdef JERK_CHECKS
    if (compiled_in) *compiled_in = 1;
#else
    if (compiled_in) *compiled_in = 0;
#endif
    JCHECK(cudaSetDevice(pl->device));
    JCHECK(cudaEventSynchronize(pl->done));
    long long c[2] = {0, 0};
    JCHECK(cudaMemcpy(c, pl->d_chk, sizeof(c), cudaMemcpyDeviceToHost));
    if (violations) *violations = (int64_t)c[0];
    if (first_site) *first_site = (int32_t)c[1];
    return JERK_OK;
}

jerk_status jerk_stats(jerk_plan pl, int32_t item, double *h_mean, double *h_std, float *h_theta) {
    if (!pl) return JERK_EINVAL;
    if (!pl->searched) return JERK_ESTATE;
    if (item < 0 || item >= pl->last_count) return JERK_EINVAL;
    JCHECK(cudaSetDevice(pl->device));
    JCHECK(cudaEventSynchronize(pl->done));
    {
        const jerk_status de = device_error(pl);
        if (de != JERK_OK) return de;
    }
    double st[2 * JERK_MAX_STAGES];
    float th[JERK_MAX_STAGES];
    JCHECK(cudaMemcpy(st, pl->d_stats + (size_t)item * 2 * JERK_MAX_STAGES, sizeof(st), cudaMemcpyDeviceToHost));
    JCHECK(cudaMemcpy(th, pl->d_theta + (size_t)item * JERK_MAX_STAGES, sizeof(th), cudaMemcpyDeviceToHost));
    for (int si = 0; si < pl->prm.n_stages; ++si) {
        if (h_mean) h_mean[si] = st[2 * si];
        if (h_std) h_std[si] = st[2 * si + 1];
        if (h_theta) h_theta[si] = th[si];
    }
    return JERK_OK;
}

}  // extern "C"
