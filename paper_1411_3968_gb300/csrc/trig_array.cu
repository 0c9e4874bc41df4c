// trig_array.cu -- multi-tower selection on sm_103a (arXiv 1411.3968,
// "Results and perspectives": every tower's trigger seeds go to a central
// selection, whose candidates' times bring back each tower's window of data).
//
// After trig_batch_run has left each tower's time-ordered trigger list on
// the device, the selection runs without the host:
//   k_acount    triggers per tower (clamped to the list capacity), offsets
//   k_aselect   per trigger, the towers holding a causally related trigger
//               (binary search into each other tower's list, then a scan of
//               the +-W range against the cross-tower dt table)
//   scan        positions of the selected triggers; k_apack packs them,
//               k_aseloff finds each tower's range
//   k_amerge    each selected trigger's rank in the (t, tower) merge of the
//               towers' lists, by binary search in the other lists
//   k_ahead     window heads among the merged triggers (gap > 2h + 1)
//   scan        window index of every head; k_awin_a / k_awin_b write the
//               windows (and a compact copy of their bounds)
//   k_abkt      per 4 us time bucket, the first window that can hold it
//   k_amark     every tower hit finds its window (bucket table, then a
//               search among the bucket's few windows), counts itself into
//               its (window, PMT) cell
//               and, at the start of a run, records the run's first index
//   scan        cell offsets in (window, tower, PMT) order
//   k_afrag     fragment offsets, window hit counts, status
//   k_acopy     every hit inside a window copies itself to its place
// The scans are one multi-block exclusive scan (partial sums, a scan of the
// partials, a final pass) over counts whose length the device knows.
#include <algorithm>
#include <cstring>
#include <memory>
#include <vector>

#include "trig_array.h"
#include "trig_internal.h"

namespace trig {
namespace {

constexpr uint32_t kMaxTowers = 64;
constexpr uint32_t kMaxArrayPmt = 4096;
constexpr uint32_t kScanPer = 4;                    // values per thread of the scan
constexpr uint32_t kScanBlock = 1024 * kScanPer;    // values per scan block
constexpr uint32_t kNone = 0xffffffffu;

struct ATower {
    const trig_trigger *trig;
    const trig_slice_stats *stats;
    uint64_t trig_cap;
    const trig_hit *hits;
    const uint64_t *pmt_off;
    uint64_t hit0;              // first index of the tower's hits in the all-tower hit numbering
    uint32_t n_pmt;
    uint32_t base;              // first array-wide PMT index of the tower
};

struct AHeader {
    uint32_t nt, pt;            // towers, PMTs of the array
    uint32_t K, W;
    int64_t h;
    uint64_t seed_cap, win_cap, hit_cap;
    uint64_t n_hits;            // hits of all towers
    trig_array_seed *seeds;
    trig_window *windows;
    uint64_t *frag_off;
    trig_hit *hits;
    trig_array_stats *stats;
    const uint16_t *dt;         // [pt * pt] min(dt_max, W)
    uint32_t *sel_flag;         // [cap] tower count of a selected trigger, else 0
    uint32_t *sel_pos;          // [cap + 1] exclusive scan of (sel_flag != 0)
    trig_array_seed *sel;       // [cap] selected triggers, tower by tower
    int64_t *merged_t;          // [cap] selected times in merge order
    uint32_t *head;             // [cap] window head flags of the merged triggers
    uint32_t *head_pos;         // [cap + 1] exclusive scan of head
    uint32_t *win_first;        // [cap] first merged trigger of each window
    int64_t *wlo, *whi;         // [win_cap] bounds of the stored windows
    uint32_t *cell_cnt;         // [win_cap * pt] hits per (window, PMT)
    uint32_t *cell_off;         // [win_cap * pt + 1] exclusive scan of cell_cnt
    uint32_t *cell_first;       // [win_cap * pt] first hit index of each (window, PMT) run
    uint32_t *win_id;           // [n_hits] window of each tower hit, or kNone
    uint32_t *part;             // scan partial sums
    uint32_t *bkt_win;          // [n_bkt + 1] first stored window ending at or after each time bucket
    int64_t bkt_org;            // time of bucket 0 (t0 - h): no window starts earlier
    uint32_t bkt_shift;         // bucket width 2^bkt_shift ns
    uint32_t n_bkt;
    // written on the device
    uint32_t n[kMaxTowers];     // triggers per tower
    uint32_t off[kMaxTowers + 1];
    uint32_t soff[kMaxTowers + 1];  // selected triggers per tower: [soff[b], soff[b + 1])
    uint32_t n_trig;            // triggers of all towers
    uint32_t n_sel;             // selected
    uint32_t n_win, n_win_stored, n_cells;
    uint32_t flags;
    uint32_t scan_total;
};

__device__ __forceinline__ uint32_t tower_of(const uint32_t *off, uint32_t nt, uint32_t i)
{
    uint32_t a = 0;
    while (a + 1 < nt && off[a + 1] <= i) ++a;
    return a;
}

__device__ __forceinline__ uint32_t tower_of_hit(const ATower *tw, uint32_t nt, uint64_t gi)
{
    uint32_t lo = 0, hi = nt;              // last b with hit0 <= gi
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (tw[mid].hit0 <= gi) lo = mid; else hi = mid;
    }
    return lo;
}

// first index j in [0, n) with L[j].t_ns >= v (or > v when upper)
__device__ __forceinline__ uint32_t trig_bound(const trig_trigger *L, uint32_t n, int64_t v, bool upper)
{
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const int64_t t = L[mid].t_ns;
        if (t < v || (upper && t == v)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t seed_bound(const trig_array_seed *L, uint32_t n, int64_t v, bool upper)
{
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const int64_t t = L[mid].t_ns;
        if (t < v || (upper && t == v)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Block-wide exclusive scan of one value per thread (blockDim.x = 1024);
// returns the exclusive prefix and writes the block total to *total.
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t *red, uint32_t *total)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (uint32_t)o) x += u;
    }
    if (lane == 31) red[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const uint32_t y = red[lane];
        uint32_t z = y;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= (uint32_t)o) z += u;
        }
        red[lane] = z - y;
        if (lane == 31) red[32] = z;
    }
    __syncthreads();
    const uint32_t r = red[warp] + x - v;
    *total = red[32];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------- the scan
// Exclusive scan of in[0 .. *n) (values, or 1 for every non-zero value when
// ones) into out[0 .. *n], out[*n] = total, also written to *total.  Blocks
// of 1024 threads, kScanBlock values each; the grid covers the largest n.

template <bool ONES>
__device__ __forceinline__ uint32_t scan_val(const uint32_t *in, uint32_t i, uint32_t n)
{
    if (i >= n) return 0u;
    const uint32_t v = in[i];
    return ONES ? (v != 0u) : v;
}

template <bool ONES>
__global__ void __launch_bounds__(1024) k_scan_part(const uint32_t *in, const uint32_t *n_ptr, uint32_t *part)
{
    __shared__ uint32_t red[33];
    const uint32_t n = *n_ptr, base = blockIdx.x * kScanBlock;
    if (base >= n && blockIdx.x > 0) return;
    uint32_t sum = 0;
#pragma unroll
    for (uint32_t r = 0; r < kScanPer; ++r) sum += scan_val<ONES>(in, base + threadIdx.x * kScanPer + r, n);
    uint32_t tot;
    block_excl_scan(sum, red, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(const uint32_t *n_ptr, uint32_t *part, uint32_t *total)
{
    __shared__ uint32_t red[33];
    const uint32_t nb = (*n_ptr + kScanBlock - 1) / kScanBlock;
    uint32_t carry = 0;
    for (uint32_t b0 = 0; b0 < nb; b0 += 1024) {
        const uint32_t b = b0 + threadIdx.x;
        const uint32_t v = b < nb ? part[b] : 0u;
        uint32_t tot;
        const uint32_t ex = block_excl_scan(v, red, &tot);
        if (b < nb) part[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

template <bool ONES>
__global__ void __launch_bounds__(1024) k_scan_final(const uint32_t *in, const uint32_t *n_ptr, const uint32_t *part,
                                                    const uint32_t *total, uint32_t *out)
{
    __shared__ uint32_t red[33];
    const uint32_t n = *n_ptr, base = blockIdx.x * kScanBlock;
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = *total;
    if (base >= n) return;
    uint32_t v[kScanPer], sum = 0;
#pragma unroll
    for (uint32_t r = 0; r < kScanPer; ++r) {
        v[r] = scan_val<ONES>(in, base + threadIdx.x * kScanPer + r, n);
        sum += v[r];
    }
    uint32_t tot;
    uint32_t run = part[blockIdx.x] + block_excl_scan(sum, red, &tot);
#pragma unroll
    for (uint32_t r = 0; r < kScanPer; ++r) {
        const uint32_t i = base + threadIdx.x * kScanPer + r;
        if (i < n) out[i] = run;
        run += v[r];
    }
}

template <bool ONES>
void launch_scan(const uint32_t *in, const uint32_t *n_ptr, uint64_t n_max, uint32_t *part, uint32_t *total,
                 uint32_t *out, cudaStream_t st, uint64_t &launches)
{
    const uint32_t nb = (uint32_t)std::max<uint64_t>(1, (n_max + kScanBlock - 1) / kScanBlock);
    k_scan_part<ONES><<<nb, 1024, 0, st>>>(in, n_ptr, part);
    k_scan_top<<<1, 1024, 0, st>>>(n_ptr, part, total);
    k_scan_final<ONES><<<nb, 1024, 0, st>>>(in, n_ptr, part, total, out);
    launches += 3;
}

// ------------------------------------------------------------ selection

// one thread per tower (blockDim.x = kMaxTowers)
__global__ void k_acount(AHeader *h, const ATower *tw)
{
    __shared__ uint32_t n_s[kMaxTowers];
    __shared__ uint32_t fl;
    const uint32_t b = threadIdx.x;
    if (b == 0) fl = 0;
    __syncthreads();
    if (b < h->nt) {
        const trig_slice_stats *s = tw[b].stats;
        const uint64_t n = s->n_triggers < tw[b].trig_cap ? s->n_triggers : tw[b].trig_cap;
        n_s[b] = (uint32_t)n;
        h->n[b] = (uint32_t)n;
        if (s->status != 0) atomicOr(&fl, TRIG_AFLAG_TOWER_INCOMPLETE);
    }
    __syncthreads();
    if (b == 0) {
        uint32_t o = 0;
        for (uint32_t a = 0; a < h->nt; ++a) {
            h->off[a] = o;
            o += n_s[a];
        }
        h->off[h->nt] = o;
        h->n_trig = o;
        h->flags = fl;
        h->n_sel = h->n_win = h->n_win_stored = h->n_cells = 0;
        h->stats->n_tower_triggers = o;
        h->stats->n_selected = h->stats->n_windows = h->stats->n_hits = 0;
        h->stats->flags = 0;
        h->stats->status = 0;
    }
}

__global__ void k_aselect(AHeader *h, const ATower *tw)
{
    const uint32_t nt = h->nt, total = h->n_trig, K = h->K;
    const int64_t W = h->W;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const uint32_t a = tower_of(h->off, nt, i);
        const trig_trigger s = tw[a].trig[i - h->off[a]];
        uint32_t cnt = 0;
        if (s.pmt < tw[a].n_pmt) {
            const uint16_t *row = h->dt + (size_t)(tw[a].base + s.pmt) * h->pt;
            for (uint32_t b = 0; b < nt; ++b) {
                if (b == a) {
                    ++cnt;                  // s itself: |0| <= dt_max[p][p]
                    continue;
                }
                const trig_trigger *L = tw[b].trig;
                const uint32_t nb = h->n[b];
                for (uint32_t j = trig_bound(L, nb, s.t_ns - W, false); j < nb; ++j) {
                    const trig_trigger u = L[j];
                    if (u.t_ns > s.t_ns + W) break;
                    if (u.pmt >= tw[b].n_pmt) continue;
                    const int64_t d = u.t_ns > s.t_ns ? u.t_ns - s.t_ns : s.t_ns - u.t_ns;
                    if (d <= (int64_t)__ldg(row + tw[b].base + u.pmt)) {
                        ++cnt;
                        break;
                    }
                }
            }
        }
        h->sel_flag[i] = cnt >= K ? cnt : 0u;
    }
}

__global__ void k_apack(AHeader *h, const ATower *tw)
{
    const uint32_t nt = h->nt, total = h->n_trig;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const uint32_t f = h->sel_flag[i];
        if (!f) continue;
        const uint32_t a = tower_of(h->off, nt, i);
        const trig_trigger s = tw[a].trig[i - h->off[a]];
        trig_array_seed e;
        e.t_ns = s.t_ns;
        e.pmt = s.pmt;
        e.tower = (uint16_t)a;
        e.n_towers = f;
        h->sel[h->sel_pos[i]] = e;
    }
}

__global__ void k_aseloff(AHeader *h)
{
    const uint32_t b = threadIdx.x, nt = h->nt;
    if (b <= nt) h->soff[b] = h->sel_pos[h->off[b]];        // sel_pos[n_trig] is the total
    if (b == 0) h->n_sel = h->sel_pos[h->n_trig];
}

__global__ void k_amerge(AHeader *h)
{
    const uint32_t nt = h->nt, M = h->n_sel;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
        const uint32_t a = tower_of(h->soff, nt, i), k = i - h->soff[a];
        const trig_array_seed s = h->sel[i];
        uint64_t g = k;
        for (uint32_t b = 0; b < nt; ++b)
            if (b != a) g += seed_bound(h->sel + h->soff[b], h->soff[b + 1] - h->soff[b], s.t_ns, b < a);
        h->merged_t[g] = s.t_ns;
        if (g < h->seed_cap) h->seeds[g] = s;
    }
}

// ------------------------------------------------------------- windows

__global__ void k_ahead(AHeader *h)
{
    const uint32_t M = h->n_sel;
    const int64_t gap = 2 * h->h + 1;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < M; g += gridDim.x * blockDim.x)
        h->head[g] = (g == 0 || h->merged_t[g] - h->merged_t[g - 1] > gap) ? 1u : 0u;
}

__global__ void k_awin_a(AHeader *h)
{
    const uint32_t M = h->n_sel;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < M; g += gridDim.x * blockDim.x)
        if (h->head[g]) h->win_first[h->head_pos[g]] = g;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint32_t nw = h->head_pos[M];
        const uint32_t ns = (uint32_t)(nw < h->win_cap ? nw : h->win_cap);
        h->n_win = nw;
        h->n_win_stored = ns;
        h->n_cells = ns * h->pt;
        uint32_t f = 0;
        if (M > h->seed_cap) f |= TRIG_AFLAG_SEED_FULL;
        if (nw > h->win_cap) f |= TRIG_AFLAG_WIN_FULL;
        atomicOr(&h->flags, f);
        h->stats->n_selected = M;
        h->stats->n_windows = nw;
    }
}

__global__ void k_awin_b(AHeader *h)
{
    const uint32_t M = h->n_sel, nw = h->n_win, ns = h->n_win_stored;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < ns; w += gridDim.x * blockDim.x) {
        const uint32_t first = h->win_first[w], next = w + 1 < nw ? h->win_first[w + 1] : M;
        const int64_t lo = h->merged_t[first] - h->h, hi = h->merged_t[next - 1] + h->h;
        h->wlo[w] = lo;
        h->whi[w] = hi;
        h->windows[w].lo_ns = lo;
        h->windows[w].hi_ns = hi;
        h->windows[w].n_triggers = next - first;
    }
}

// -------------------------------------------------------------- readback

__global__ void k_azero(AHeader *h)
{
    const uint32_t n = h->n_cells;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) h->cell_cnt[i] = 0;
}

// first stored window w in [lo, hi) with whi[w] >= t (hi if none)
__device__ __forceinline__ uint32_t first_ending_at(const int64_t *whi, uint32_t lo, uint32_t hi, int64_t t)
{
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (whi[mid] < t) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Bucket table of the window search: bkt_win[j] = the first stored window
// ending at or after the start of time bucket j.  The windows are disjoint
// and ordered, so a time in bucket j can only lie in windows
// bkt_win[j] .. bkt_win[j + 1].
__global__ void k_abkt(AHeader *h)
{
    const uint32_t ns = h->n_win_stored, nb = h->n_bkt;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= nb; j += gridDim.x * blockDim.x)
        h->bkt_win[j] = first_ending_at(h->whi, 0, ns, h->bkt_org + ((int64_t)j << h->bkt_shift));
}

// window of time t among the stored ones, or kNone
__device__ __forceinline__ uint32_t window_of(const AHeader *h, uint32_t ns, int64_t t)
{
    if (t < h->bkt_org) return kNone;
    const uint64_t j = (uint64_t)(t - h->bkt_org) >> h->bkt_shift;
    if (j >= h->n_bkt) return kNone;
    const uint32_t lo = h->bkt_win[j], hi = min(h->bkt_win[j + 1] + 1u, ns);
    const uint32_t w = first_ending_at(h->whi, lo, hi, t);
    return (w < ns && h->wlo[w] <= t) ? w : kNone;
}

__global__ void k_amark(AHeader *h, const ATower *tw)
{
    const uint32_t nt = h->nt, ns = h->n_win_stored, pt = h->pt;
    const uint64_t n = h->n_hits;
    for (uint64_t gi = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < n;
         gi += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t b = tower_of_hit(tw, nt, gi);
        const uint64_t i = gi - tw[b].hit0;
        const trig_hit *hs = tw[b].hits;
        const int64_t t = hs[i].t_ns;
        const uint32_t q = hs[i].pmt;
        uint32_t w = ns ? window_of(h, ns, t) : kNone;
        if (q >= tw[b].n_pmt) w = kNone;
        h->win_id[gi] = w;
        if (w == kNone) continue;
        const size_t cell = (size_t)w * pt + tw[b].base + q;
        atomicAdd(&h->cell_cnt[cell], 1u);
        // the first hit of its PMT inside this window starts the run
        if (i == tw[b].pmt_off[q] || hs[i - 1].t_ns < h->wlo[w]) h->cell_first[cell] = (uint32_t)i;
    }
}

__global__ void k_afrag(AHeader *h, const ATower *tw)
{
    const uint32_t nt = h->nt, ns = h->n_win_stored, pt = h->pt;
    const uint32_t total = h->cell_off[h->n_cells];
    const uint32_t stride = gridDim.x * blockDim.x, t0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t k = t0; k < ns * nt; k += stride)
        h->frag_off[k] = h->cell_off[(size_t)(k / nt) * pt + tw[k % nt].base];
    for (uint32_t w = t0; w < ns; w += stride)
        h->windows[w].n_hits = h->cell_off[(size_t)(w + 1) * pt] - h->cell_off[(size_t)w * pt];
    if (t0 == 0) {
        h->frag_off[(size_t)ns * nt] = total;
        uint32_t f = h->flags;
        if (total > h->hit_cap) f |= TRIG_AFLAG_HIT_FULL;
        h->stats->n_hits = total;
        h->stats->flags = f;
        h->stats->status = f ? TRIG_ECAPACITY : TRIG_OK;
    }
}

__global__ void k_acopy(AHeader *h, const ATower *tw)
{
    const uint32_t nt = h->nt, pt = h->pt;
    const uint64_t n = h->n_hits;
    for (uint64_t gi = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < n;
         gi += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t w = h->win_id[gi];
        if (w == kNone) continue;
        const uint32_t b = tower_of_hit(tw, nt, gi);
        const uint64_t i = gi - tw[b].hit0;
        const trig_hit x = tw[b].hits[i];
        const size_t cell = (size_t)w * pt + tw[b].base + x.pmt;
        const uint64_t dst = (uint64_t)h->cell_off[cell] + (i - (uint64_t)h->cell_first[cell]);
        if (dst < h->hit_cap) h->hits[dst] = x;
    }
}

}  // namespace
}  // namespace trig

using namespace trig;

struct trig_array {
    uint32_t nt = 0, pt = 0;
    std::vector<trig_detector *> towers;
    std::vector<uint32_t> base, n_pmt;
    trig_array_params par{};
    uint16_t *dt = nullptr;     // [pt * pt] min(dt_max, W)
    int device = 0;
};

extern "C" int trig_array_create(trig_detector *const *towers, uint32_t n_towers, const trig_array_params *params,
                                 trig_array **out)
{
    if (!out) return report_error(TRIG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!towers || !params) return report_error(TRIG_EINVAL, "towers or params is NULL");
    if (n_towers < 1 || n_towers > kMaxTowers) return report_error(TRIG_EINVAL, "n_towers must be in [1, 64]");
    if (params->min_towers < 1 || params->corr_window_ns > 60000 || params->win_half_ns > 60000 ||
        params->reserved != 0)
        return report_error(TRIG_EINVAL, "min_towers >= 1, corr_window_ns and win_half_ns <= 60000, reserved 0");
    std::unique_ptr<trig_array> a(new trig_array());
    a->nt = n_towers;
    a->par = *params;
    std::vector<int32_t> xyz;
    DetInfo first{};
    for (uint32_t b = 0; b < n_towers; ++b) {
        DetInfo di{};
        if (!detector_info(towers[b], &di)) return report_error(TRIG_EINVAL, "a tower is NULL");
        if (b == 0) first = di;
        if (di.par.tol_ns != first.par.tol_ns || di.par.n_num != first.par.n_num || di.par.n_den != first.par.n_den)
            return report_error(TRIG_EINVAL, "towers must share tol_ns, n_num and n_den");
        if ((int64_t)params->win_half_ns > di.in_halo)
            return report_error(TRIG_EINVAL, "win_half_ns exceeds a tower's accepted halo");
        a->towers.push_back(towers[b]);
        a->base.push_back(a->pt);
        a->n_pmt.push_back(di.n_pmt);
        a->pt += di.n_pmt;
        if (a->pt > kMaxArrayPmt) return report_error(TRIG_EINVAL, "the towers hold more than 4096 PMTs");
        xyz.insert(xyz.end(), di.xyz, di.xyz + 3 * (size_t)di.n_pmt);
    }
    cudaGetDevice(&a->device);
    const size_t PP = (size_t)a->pt * a->pt;
    int32_t *d_xyz = nullptr, *dt_exact = nullptr;
    uint16_t *dmax = nullptr;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaMalloc(&a->dt, PP * 2);
    if (!e) e = cudaMalloc(&dt_exact, PP * 4);
    if (!e) e = cudaMalloc(&dmax, (size_t)a->pt * 2);
    if (!e) e = cudaMalloc(&d_xyz, xyz.size() * 4);
    if (!e) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (!e) e = cudaMemcpyAsync(d_xyz, xyz.data(), xyz.size() * 4, cudaMemcpyHostToDevice, st);
    if (!e)
        e = launch_dtmax(d_xyz, a->pt, first.par.tol_ns, first.par.n_num, first.par.n_den, params->corr_window_ns,
                         dt_exact, a->dt, dmax, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (st) cudaStreamDestroy(st);
    cudaFree(d_xyz);
    cudaFree(dt_exact);
    cudaFree(dmax);
    if (e) {
        cudaFree(a->dt);
        return report_cuda_error(e, "trig_array_create: cross-tower dt_max");
    }
    count_launches(2);
    *out = a.release();
    return TRIG_OK;
}

extern "C" int trig_array_destroy(trig_array *a)
{
    if (!a) return TRIG_EINVAL;
    cudaFree(a->dt);
    delete a;
    return TRIG_OK;
}

namespace {

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct ALayout {
    size_t hdr, towers, sel_flag, sel_pos, sel, merged_t, head, head_pos, win_first, wlo, whi, cell_cnt, cell_off,
        cell_first, win_id, part, bkt_win, bytes;
    uint64_t cap, n_hits, cells, part_n;
    uint32_t bkt_shift, n_bkt;
};

int array_layout(const trig_array *a, const trig_slice_dev *slices, const trig_array_out *out, ALayout &L)
{
    if (!a || !slices || !out) return report_error(TRIG_EINVAL, "array, slices or out is NULL");
    uint64_t cap = 0, n_hits = 0;
    for (uint32_t b = 0; b < a->nt; ++b) {
        if (slices[b].det != a->towers[b]) return report_error(TRIG_EINVAL, "slices[b] is not tower b's slice");
        if (slices[b].t0_ns != slices[0].t0_ns) return report_error(TRIG_EINVAL, "tower slices differ in t0_ns");
        if (!slices[b].triggers || !slices[b].stats || (slices[b].n_hits && !slices[b].hits) || !slices[b].pmt_off)
            return report_error(TRIG_EINVAL, "a tower slice lacks triggers, stats or hits");
        cap += slices[b].trig_cap;
        n_hits += slices[b].n_hits;
    }
    if (cap >= 0xfffffff0ull) return report_error(TRIG_EINVAL, "the towers' trigger capacities exceed 2^32");
    if (n_hits >= 0xfffffff0ull) return report_error(TRIG_EINVAL, "the towers hold 2^32 hits or more");
    if ((out->seed_cap && !out->seeds) || (out->win_cap && !out->windows) || !out->frag_off || !out->stats ||
        (out->hit_cap && !out->hits))
        return report_error(TRIG_EINVAL, "an output with capacity has no buffer");
    const uint64_t cells = out->win_cap * a->pt;
    if (out->win_cap > 0xffffffffull / a->nt || cells >= 0xfffffff0ull)
        return report_error(TRIG_EINVAL, "win_cap too large for this array");
    const uint64_t part_n = std::max(cap, cells) / kScanBlock + 2;
    // buckets of the window search over [t0 - h, t0 + S + h], at most 2^20
    int64_t span = 1;
    for (uint32_t b = 0; b < a->nt; ++b) {
        DetInfo di{};
        detector_info(a->towers[b], &di);
        span = std::max<int64_t>(span, di.par.slice_ns + 2 * (int64_t)a->par.win_half_ns + 1);
    }
    uint32_t shift = 12;
    while (((span >> shift) + 1) > ((int64_t)1 << 20)) ++shift;
    L.bkt_shift = shift;
    L.n_bkt = (uint32_t)((span >> shift) + 1);
    size_t o = 0;
    auto take = [&](size_t &field, size_t bytes) {
        field = o;
        o += al256(bytes);
    };
    take(L.hdr, sizeof(AHeader));
    take(L.towers, sizeof(ATower) * a->nt);
    take(L.sel_flag, 4 * (size_t)(cap + 1));
    take(L.sel_pos, 4 * (size_t)(cap + 1));
    take(L.sel, sizeof(trig_array_seed) * (size_t)(cap + 1));
    take(L.merged_t, 8 * (size_t)(cap + 1));
    take(L.head, 4 * (size_t)(cap + 1));
    take(L.head_pos, 4 * (size_t)(cap + 1));
    take(L.win_first, 4 * (size_t)(cap + 1));
    take(L.wlo, 8 * (size_t)(out->win_cap + 1));
    take(L.whi, 8 * (size_t)(out->win_cap + 1));
    take(L.cell_cnt, 4 * (size_t)(cells + 1));
    take(L.cell_off, 4 * (size_t)(cells + 1));
    take(L.cell_first, 4 * (size_t)(cells + 1));
    take(L.win_id, 4 * (size_t)(n_hits + 1));
    take(L.part, 4 * (size_t)part_n);
    take(L.bkt_win, 4 * ((size_t)L.n_bkt + 2));
    L.bytes = o;
    L.cap = cap;
    L.n_hits = n_hits;
    L.cells = cells;
    L.part_n = part_n;
    return TRIG_OK;
}

}  // namespace

extern "C" size_t trig_array_scratch_bytes(const trig_array *a, const trig_slice_dev *slices, const trig_array_out *out)
{
    ALayout L{};
    return array_layout(a, slices, out, L) == TRIG_OK ? L.bytes : 0;
}

extern "C" int trig_array_select(trig_array *a, const trig_slice_dev *slices, const trig_array_out *out,
                                 void *scratch, size_t scratch_bytes, void *stream)
{
    ALayout L{};
    int rc = array_layout(a, slices, out, L);
    if (rc) return rc;
    if (!scratch || ((uintptr_t)scratch & 255u))
        return report_error(TRIG_EINVAL, "trig_array_select: scratch must be 256-byte aligned device memory");
    if (scratch_bytes < L.bytes) return report_error(TRIG_ECAPACITY, "trig_array_select: scratch too small");
    char *sp = static_cast<char *>(scratch);
    AHeader hd{};
    hd.nt = a->nt;
    hd.pt = a->pt;
    hd.K = a->par.min_towers;
    hd.W = a->par.corr_window_ns;
    hd.h = a->par.win_half_ns;
    hd.seed_cap = out->seed_cap;
    hd.win_cap = out->win_cap;
    hd.hit_cap = out->hit_cap;
    hd.seeds = out->seeds;
    hd.windows = out->windows;
    hd.frag_off = out->frag_off;
    hd.hits = out->hits;
    hd.stats = out->stats;
    hd.dt = a->dt;
    hd.n_hits = L.n_hits;
    hd.sel_flag = reinterpret_cast<uint32_t *>(sp + L.sel_flag);
    hd.sel_pos = reinterpret_cast<uint32_t *>(sp + L.sel_pos);
    hd.sel = reinterpret_cast<trig_array_seed *>(sp + L.sel);
    hd.merged_t = reinterpret_cast<int64_t *>(sp + L.merged_t);
    hd.head = reinterpret_cast<uint32_t *>(sp + L.head);
    hd.head_pos = reinterpret_cast<uint32_t *>(sp + L.head_pos);
    hd.win_first = reinterpret_cast<uint32_t *>(sp + L.win_first);
    hd.wlo = reinterpret_cast<int64_t *>(sp + L.wlo);
    hd.whi = reinterpret_cast<int64_t *>(sp + L.whi);
    hd.cell_cnt = reinterpret_cast<uint32_t *>(sp + L.cell_cnt);
    hd.cell_off = reinterpret_cast<uint32_t *>(sp + L.cell_off);
    hd.cell_first = reinterpret_cast<uint32_t *>(sp + L.cell_first);
    hd.win_id = reinterpret_cast<uint32_t *>(sp + L.win_id);
    hd.part = reinterpret_cast<uint32_t *>(sp + L.part);
    hd.bkt_win = reinterpret_cast<uint32_t *>(sp + L.bkt_win);
    hd.bkt_org = slices[0].t0_ns - (int64_t)a->par.win_half_ns;
    hd.bkt_shift = L.bkt_shift;
    hd.n_bkt = L.n_bkt;
    ATower tw[kMaxTowers];
    uint64_t hit0 = 0;
    for (uint32_t b = 0; b < a->nt; ++b) {
        tw[b].trig = slices[b].triggers;
        tw[b].stats = slices[b].stats;
        tw[b].trig_cap = slices[b].trig_cap;
        tw[b].hits = slices[b].hits;
        tw[b].pmt_off = slices[b].pmt_off;
        tw[b].hit0 = hit0;
        tw[b].n_pmt = a->n_pmt[b];
        tw[b].base = a->base[b];
        hit0 += slices[b].n_hits;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    AHeader *d_h = reinterpret_cast<AHeader *>(sp + L.hdr);
    ATower *d_t = reinterpret_cast<ATower *>(sp + L.towers);
    // pageable sources: both copies are staged before the calls return
    cudaError_t e = cudaMemcpyAsync(d_h, &hd, sizeof hd, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(d_t, tw, sizeof(ATower) * a->nt, cudaMemcpyHostToDevice, st);
    if (e) return report_cuda_error(e, "trig_array_select: copy descriptors");
    const int sms = device_sm_count();
    const unsigned grid = (unsigned)sms * 4;
    uint64_t nl = 0;
    uint32_t *scan_total = &d_h->scan_total;
    k_acount<<<1, kMaxTowers, 0, st>>>(d_h, d_t);
    k_aselect<<<grid, 256, 0, st>>>(d_h, d_t);
    launch_scan<true>(hd.sel_flag, &d_h->n_trig, L.cap, hd.part, scan_total, hd.sel_pos, st, nl);
    k_apack<<<grid, 256, 0, st>>>(d_h, d_t);
    k_aseloff<<<1, kMaxTowers + 32, 0, st>>>(d_h);
    k_amerge<<<grid, 256, 0, st>>>(d_h);
    k_ahead<<<grid, 256, 0, st>>>(d_h);
    launch_scan<false>(hd.head, &d_h->n_sel, L.cap, hd.part, scan_total, hd.head_pos, st, nl);
    k_awin_a<<<grid, 256, 0, st>>>(d_h);
    k_awin_b<<<grid, 256, 0, st>>>(d_h);
    k_abkt<<<grid, 256, 0, st>>>(d_h);
    k_azero<<<grid * 2, 256, 0, st>>>(d_h);
    k_amark<<<grid * 2, 256, 0, st>>>(d_h, d_t);
    launch_scan<false>(hd.cell_cnt, &d_h->n_cells, L.cells, hd.part, scan_total, hd.cell_off, st, nl);
    k_afrag<<<grid, 256, 0, st>>>(d_h, d_t);
    k_acopy<<<grid * 2, 256, 0, st>>>(d_h, d_t);
    count_launches(nl + 13);
    e = cudaGetLastError();
    return e ? report_cuda_error(e, "trig_array_select: launch") : TRIG_OK;
}
