// trig_array.cu -- multi-tower selection on sm_103a (arXiv 1411.3968,
// "Results and perspectives": every tower's trigger seeds go to a central
// selection, whose candidates' times bring back each tower's window of data).
//
// After trig_batch_run has left each tower's time-ordered trigger list on
// the device, eight small kernels finish the job without the host:
//   k_acount   triggers per tower (clamped to the list capacity), offsets
//   k_aselect  per trigger, the towers holding a causally related trigger
//              (binary search into each other tower's list, then a scan of
//              the +-W range against the cross-tower dt table)
//   k_acompact per tower, the selected triggers in list order
//   k_amerge   each selected trigger's rank in the (t, tower) merge of the
//              towers' lists, by binary search in the other lists
//   k_awindows windows of +-h around the merged times, merged when touching
//   k_afcount  hits of each (window, tower) fragment: per-PMT binary search
//   k_afscan   fragment offsets, window hit counts, status
//   k_acopy    the fragments, PMT run by PMT run
// The work is a few per cent of the tower triggers' (one pass over the
// triggers and one over the hits inside windows).
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

struct ATower {
    const trig_trigger *trig;
    const trig_slice_stats *stats;
    uint64_t trig_cap;
    const trig_hit *hits;
    const uint64_t *pmt_off;
    uint32_t n_pmt;
    uint32_t base;              // first array-wide PMT index of the tower
};

struct AHeader {
    uint32_t nt, pt;            // towers, PMTs of the array
    uint32_t K, W;
    int64_t h;
    uint64_t seed_cap, win_cap, hit_cap;
    trig_array_seed *seeds;
    trig_window *windows;
    uint64_t *frag_off;
    trig_hit *hits;
    trig_array_stats *stats;
    const uint16_t *dt;         // [pt * pt] min(dt_max, W)
    uint32_t *sel_flag;         // [cap] tower count of a selected trigger, else 0
    trig_array_seed *sel;       // [cap] per tower, its selected triggers from off[b]
    int64_t *merged_t;          // [cap] selected times in merge order
    uint32_t *win_of;           // [cap] window of each merged trigger
    uint32_t *win_first;        // [cap] first merged trigger of each window
    uint64_t *frag_cnt;         // [win_cap * nt]
    // written on the device
    uint32_t n[kMaxTowers];     // triggers per tower
    uint32_t off[kMaxTowers + 1];
    uint32_t nsel[kMaxTowers];  // selected per tower
    uint32_t n_sel, n_win, n_win_stored, flags;
};

__device__ __forceinline__ uint32_t tower_of(const AHeader *h, uint32_t i)
{
    uint32_t a = 0;
    while (a + 1 < h->nt && h->off[a + 1] <= i) ++a;
    return a;
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

// first index in [lo, hi) of a time-ordered hit run with t >= v
__device__ __forceinline__ uint64_t hit_bound(const trig_hit *hs, uint64_t lo, uint64_t hi, int64_t v)
{
    while (lo < hi) {
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if (hs[mid].t_ns < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint64_t warp_sum64(uint64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

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
        h->flags = fl;
        h->n_sel = h->n_win = h->n_win_stored = 0;
        h->stats->n_tower_triggers = o;
        h->stats->n_selected = h->stats->n_windows = h->stats->n_hits = 0;
        h->stats->flags = 0;
        h->stats->status = 0;
    }
}

__global__ void k_aselect(AHeader *h, const ATower *tw)
{
    const uint32_t nt = h->nt, total = h->off[nt], K = h->K;
    const int64_t W = h->W;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const uint32_t a = tower_of(h, i);
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
        uint32_t y = lane < (blockDim.x >> 5) ? red[lane] : 0u, z = y;
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

__global__ void __launch_bounds__(1024) k_acompact(AHeader *h, const ATower *tw)
{
    __shared__ uint32_t red[33];
    const uint32_t b = blockIdx.x;
    if (b >= h->nt) return;
    const uint32_t o = h->off[b], n = h->n[b];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < n; base += 1024) {
        const uint32_t k = base + threadIdx.x;
        const uint32_t f = k < n ? h->sel_flag[o + k] : 0u;
        uint32_t tot;
        const uint32_t pos = carry + block_excl_scan(f ? 1u : 0u, red, &tot);
        if (f) {
            const trig_trigger s = tw[b].trig[k];
            trig_array_seed e;
            e.t_ns = s.t_ns;
            e.pmt = s.pmt;
            e.tower = (uint16_t)b;
            e.n_towers = f;
            h->sel[o + pos] = e;
        }
        carry += tot;
    }
    if (threadIdx.x == 0) h->nsel[b] = carry;
}

__global__ void k_amerge(AHeader *h)
{
    const uint32_t nt = h->nt, total = h->off[nt];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const uint32_t a = tower_of(h, i), k = i - h->off[a];
        if (k >= h->nsel[a]) continue;
        const trig_array_seed s = h->sel[i];
        uint64_t g = k;
        for (uint32_t b = 0; b < nt; ++b)
            if (b != a) g += seed_bound(h->sel + h->off[b], h->nsel[b], s.t_ns, b < a);
        h->merged_t[g] = s.t_ns;
        if (g < h->seed_cap) h->seeds[g] = s;
    }
}

__global__ void __launch_bounds__(1024) k_awindows(AHeader *h)
{
    __shared__ uint32_t red[33];
    uint32_t M = 0;
    for (uint32_t b = 0; b < h->nt; ++b) M += h->nsel[b];
    const int64_t hw = h->h;
    // pass 1: window index of each merged trigger, first trigger of each window
    uint32_t carry = 0;
    for (uint32_t base = 0; base < M; base += 1024) {
        const uint32_t g = base + threadIdx.x;
        bool head = false;
        if (g < M) head = g == 0 || h->merged_t[g] - hw > h->merged_t[g - 1] + hw + 1;
        uint32_t tot;
        const uint32_t ex = block_excl_scan(head ? 1u : 0u, red, &tot);
        if (g < M) {
            const uint32_t w = carry + ex + (head ? 1u : 0u) - 1u;
            h->win_of[g] = w;
            if (head) {
                h->win_first[w] = g;
                if (w < h->win_cap) h->windows[w].lo_ns = h->merged_t[g] - hw;
            }
        }
        carry += tot;
    }
    __syncthreads();
    // pass 2: the last trigger of a window closes it
    for (uint32_t g = threadIdx.x; g < M; g += 1024) {
        const uint32_t w = h->win_of[g];
        if ((g + 1 == M || h->win_of[g + 1] != w) && w < h->win_cap) {
            h->windows[w].hi_ns = h->merged_t[g] + hw;
            h->windows[w].n_triggers = g - h->win_first[w] + 1;
        }
    }
    if (threadIdx.x == 0) {
        const uint32_t nw = carry;
        h->n_sel = M;
        h->n_win = nw;
        h->n_win_stored = (uint32_t)(nw < h->win_cap ? nw : h->win_cap);
        uint32_t f = 0;
        if (M > h->seed_cap) f |= TRIG_AFLAG_SEED_FULL;
        if (nw > h->win_cap) f |= TRIG_AFLAG_WIN_FULL;
        h->flags |= f;
        h->stats->n_selected = M;
        h->stats->n_windows = nw;
    }
}

// one warp per (window, tower) fragment
__global__ void k_afcount(AHeader *h, const ATower *tw)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nt = h->nt, npairs = h->n_win_stored * nt;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < npairs; p += warps) {
        const uint32_t w = p / nt, b = p % nt;
        const int64_t lo = h->windows[w].lo_ns, hi = h->windows[w].hi_ns;
        uint64_t c = 0;
        for (uint32_t q = lane; q < tw[b].n_pmt; q += 32) {
            const uint64_t s0 = tw[b].pmt_off[q], s1 = tw[b].pmt_off[q + 1];
            const uint64_t a = hit_bound(tw[b].hits, s0, s1, lo);
            c += hit_bound(tw[b].hits, a, s1, hi + 1) - a;
        }
        c = warp_sum64(c);
        if (lane == 0) h->frag_cnt[p] = c;
    }
}

__global__ void __launch_bounds__(1024) k_afscan(AHeader *h)
{
    __shared__ unsigned long long red[33];
    const uint32_t nt = h->nt, npairs = h->n_win_stored * nt;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    unsigned long long carry = 0;
    for (uint32_t base = 0; base < npairs; base += 1024) {
        const uint32_t p = base + threadIdx.x;
        const unsigned long long v = p < npairs ? h->frag_cnt[p] : 0ull;
        unsigned long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (uint32_t)o) x += u;
        }
        if (lane == 31) red[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const unsigned long long y = red[lane];
            unsigned long long z = y;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long u = __shfl_up_sync(0xffffffffu, z, o);
                if (lane >= (uint32_t)o) z += u;
            }
            red[lane] = z - y;
            if (lane == 31) red[32] = z;
        }
        __syncthreads();
        if (p < npairs) h->frag_off[p] = carry + red[warp] + x - v;
        carry += red[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) h->frag_off[npairs] = carry;
    __syncthreads();
    for (uint32_t w = threadIdx.x; w < h->n_win_stored; w += 1024)
        h->windows[w].n_hits = h->frag_off[(w + 1) * nt] - h->frag_off[w * nt];
    if (threadIdx.x == 0) {
        uint32_t f = h->flags;
        if (carry > h->hit_cap) f |= TRIG_AFLAG_HIT_FULL;
        h->stats->n_hits = carry;
        h->stats->flags = f;
        h->stats->status = f ? TRIG_ECAPACITY : TRIG_OK;
    }
}

// one warp per fragment: PMT runs in order, 32 PMTs at a time
__global__ void k_acopy(AHeader *h, const ATower *tw)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nt = h->nt, npairs = h->n_win_stored * nt;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < npairs; p += warps) {
        const uint32_t w = p / nt, b = p % nt;
        const int64_t lo = h->windows[w].lo_ns, hi = h->windows[w].hi_ns;
        uint64_t dst = h->frag_off[p];
        const trig_hit *src = tw[b].hits;
        for (uint32_t q0 = 0; q0 < tw[b].n_pmt; q0 += 32) {
            const uint32_t q = q0 + lane;
            uint64_t a = 0, len = 0;
            if (q < tw[b].n_pmt) {
                const uint64_t s0 = tw[b].pmt_off[q], s1 = tw[b].pmt_off[q + 1];
                a = hit_bound(src, s0, s1, lo);
                len = hit_bound(src, a, s1, hi + 1) - a;
            }
            uint64_t incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (uint32_t)o) incl += u;
            }
            const uint64_t mine = dst + incl - len;
            for (uint32_t r = 0; r < 32; ++r) {
                const uint64_t ra = __shfl_sync(0xffffffffu, a, r);
                const uint64_t rl = __shfl_sync(0xffffffffu, len, r);
                const uint64_t rd = __shfl_sync(0xffffffffu, mine, r);
                for (uint64_t e = lane; e < rl; e += 32)
                    if (rd + e < h->hit_cap) h->hits[rd + e] = src[ra + e];
            }
            dst += __shfl_sync(0xffffffffu, incl, 31);
        }
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
    size_t hdr, towers, sel_flag, sel, merged_t, win_of, win_first, frag_cnt, bytes;
    uint64_t cap;
};

int array_layout(const trig_array *a, const trig_slice_dev *slices, const trig_array_out *out, ALayout &L)
{
    if (!a || !slices || !out) return report_error(TRIG_EINVAL, "array, slices or out is NULL");
    uint64_t cap = 0;
    for (uint32_t b = 0; b < a->nt; ++b) {
        if (slices[b].det != a->towers[b]) return report_error(TRIG_EINVAL, "slices[b] is not tower b's slice");
        if (slices[b].t0_ns != slices[0].t0_ns) return report_error(TRIG_EINVAL, "tower slices differ in t0_ns");
        if (!slices[b].triggers || !slices[b].stats || !slices[b].hits || !slices[b].pmt_off)
            return report_error(TRIG_EINVAL, "a tower slice lacks triggers, stats or hits");
        cap += slices[b].trig_cap;
    }
    if (cap >= 0xffffffffull) return report_error(TRIG_EINVAL, "the towers' trigger capacities exceed 2^32");
    if ((out->seed_cap && !out->seeds) || (out->win_cap && (!out->windows)) || !out->frag_off || !out->stats ||
        (out->hit_cap && !out->hits))
        return report_error(TRIG_EINVAL, "an output with capacity has no buffer");
    if (out->win_cap > 0xffffffffull / a->nt) return report_error(TRIG_EINVAL, "win_cap too large");
    size_t o = 0;
    L.hdr = o;
    o += al256(sizeof(AHeader));
    L.towers = o;
    o += al256(sizeof(ATower) * a->nt);
    L.sel_flag = o;
    o += al256(4 * (size_t)(cap + 1));
    L.sel = o;
    o += al256(sizeof(trig_array_seed) * (size_t)(cap + 1));
    L.merged_t = o;
    o += al256(8 * (size_t)(cap + 1));
    L.win_of = o;
    o += al256(4 * (size_t)(cap + 1));
    L.win_first = o;
    o += al256(4 * (size_t)(cap + 1));
    L.frag_cnt = o;
    o += al256(8 * (size_t)(out->win_cap * a->nt + 1));
    L.bytes = o;
    L.cap = cap;
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
    if (!scratch || scratch_bytes < L.bytes) return report_error(TRIG_ECAPACITY, "trig_array_select: scratch too small");
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
    hd.sel_flag = reinterpret_cast<uint32_t *>(sp + L.sel_flag);
    hd.sel = reinterpret_cast<trig_array_seed *>(sp + L.sel);
    hd.merged_t = reinterpret_cast<int64_t *>(sp + L.merged_t);
    hd.win_of = reinterpret_cast<uint32_t *>(sp + L.win_of);
    hd.win_first = reinterpret_cast<uint32_t *>(sp + L.win_first);
    hd.frag_cnt = reinterpret_cast<uint64_t *>(sp + L.frag_cnt);
    ATower tw[kMaxTowers];
    for (uint32_t b = 0; b < a->nt; ++b) {
        tw[b].trig = slices[b].triggers;
        tw[b].stats = slices[b].stats;
        tw[b].trig_cap = slices[b].trig_cap;
        tw[b].hits = slices[b].hits;
        tw[b].pmt_off = slices[b].pmt_off;
        tw[b].n_pmt = a->n_pmt[b];
        tw[b].base = a->base[b];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    AHeader *d_h = reinterpret_cast<AHeader *>(sp + L.hdr);
    ATower *d_t = reinterpret_cast<ATower *>(sp + L.towers);
    // pageable sources: both copies are staged before the calls return
    cudaError_t e = cudaMemcpyAsync(d_h, &hd, sizeof hd, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(d_t, tw, sizeof(ATower) * a->nt, cudaMemcpyHostToDevice, st);
    if (e) return report_cuda_error(e, "trig_array_select: copy descriptors");
    const int sms = device_sm_count();
    k_acount<<<1, kMaxTowers, 0, st>>>(d_h, d_t);
    k_aselect<<<sms * 4, 256, 0, st>>>(d_h, d_t);
    k_acompact<<<a->nt, 1024, 0, st>>>(d_h, d_t);
    k_amerge<<<sms * 4, 256, 0, st>>>(d_h);
    k_awindows<<<1, 1024, 0, st>>>(d_h);
    k_afcount<<<sms * 4, 256, 0, st>>>(d_h, d_t);
    k_afscan<<<1, 1024, 0, st>>>(d_h);
    k_acopy<<<sms * 4, 256, 0, st>>>(d_h, d_t);
    count_launches(8);
    e = cudaGetLastError();
    return e ? report_cuda_error(e, "trig_array_select: launch") : TRIG_OK;
}
