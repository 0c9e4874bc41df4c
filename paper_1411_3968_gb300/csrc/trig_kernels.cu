// trig_kernels.cu -- sm_103a kernels of the online muon trigger (arXiv 1411.3968).
//
// Pipeline per batch of slices (all launches on one stream):
//   k_prep     zero the batch's counters and per-slice statistics.
//   k_bounds   structure pass of the k-way merge ("DAQ system": the Hit
//              Manager merges the PMT streams into time slices).  One read
//              of every hit: validates the CSR layout and ordering, and for
//              every time tile g and PMT p records where p's stream crosses
//              the tile's halo edges B_g - H and B_{g+1} + H.
//   k_tile     persistent, warp-specialised: a producer warp dequeues tiles
//              and stages each tile's hits (one contiguous run per PMT) into
//              shared memory with bulk TMA copies (cp.async.bulk + mbarrier,
//              double-buffered); 16 consumer warps merge the runs into time
//              order (bucket sort on the time key), select seeds (charge
//              threshold or floor coincidence, "Sorting and triggering in
//              GPU"), count causally related hits per seed with warp
//              ballot/popc against the integer dt_max table ("Muon trigger
//              strategy"), and emit the fired seeds at their merged rank.
//   k_scan / k_copy   stream compaction of the fired seeds (tile prefix sum,
//              then a copy into the dense trigger list).
//   k_wscan / k_wwrite / k_wcount   the +-3 us windows around the
//              triggers, merged while lo_next <= hi_cur + 1, with the hit
//              count inside each: the difference of two merged ranks the
//              tile pass records beside each fired seed.
//
// Every wait on an mbarrier is bounded; a wait that gives up sets
// TRIG_FLAG_TIMEOUT on the batch and the kernel returns.
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "trig_internal.h"

namespace trig {

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait with a suspend-time hint: a thread whose phase is not complete
// is suspended until it completes or about `ns` nanoseconds pass, instead
// of spinning and issuing instructions.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t *bar, uint32_t parity, uint32_t ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Built with -DTRIG_PHASE_STATS, the tile kernel adds its per-phase clock
// cycles and its waits (cycles, try_wait rounds) into device counters that
// trig_phase_stats reads; without it the counters compile to nothing.
#ifdef TRIG_PHASE_STATS
__device__ unsigned long long g_phase[24];
#define PHASE_ADD(i, v) atomicAdd(&g_phase[(i)], (unsigned long long)(v))
#else
#define PHASE_ADD(i, v) ((void)0)
#endif
enum PhaseCounter {
    kPhTiles, kPhConsWait, kPhConsWaitRounds, kPhProdWait, kPhProdWaitRounds, kPhA, kPhB, kPhC, kPhD, kPhE,
    kPhF, kPhG, kPhSeeds, kPhProdItem, kPhConsTotal, kPhProdTotal, kPhKeys
};

// Bounded wait: gives up after limit_ns of the GPU's global timer and
// reports failure.  *rounds (optional) counts the try_wait rounds.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns,
                                          uint32_t *rounds = nullptr)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t_start = global_ns();
    for (uint32_t r = 1;; ++r) {
        if (rounds) *rounds = r;
        if (mbar_try_wait_hint(bar, parity, 20000u)) return true;
        if (global_ns() - t_start > limit_ns) return false;
    }
}

// Bulk (non-tensor) TMA copy global -> shared, completing on an mbarrier.
// Source and destination 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void named_sync(uint32_t id, uint32_t n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Named barrier over n threads that also ANDs a predicate across them: every
// thread leaves with the same answer.
__device__ __forceinline__ bool named_sync_and(uint32_t id, uint32_t n, bool p)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred q, o;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred o, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, o;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
    const uint32_t lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= (uint32_t)o) v += u;
    }
    return v;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ trig_hit load_hit(const trig_hit *p)
{
    int4 v = __ldg(reinterpret_cast<const int4 *>(p));
    trig_hit h;
    h.t_ns = (int64_t)(((uint64_t)(uint32_t)v.y << 32) | (uint32_t)v.x);
    h.pmt = (uint16_t)((uint32_t)v.z & 0xffffu);
    h.charge = (uint16_t)((uint32_t)v.z >> 16);
    h.reserved = (uint32_t)v.w;
    return h;
}

// first index i in [lo, hi) of a time-ordered hit run with t >= v
__device__ __forceinline__ uint64_t lb_time(const trig_hit *h, uint64_t lo, uint64_t hi, int64_t v)
{
    while (lo < hi) {
        uint64_t mid = lo + ((hi - lo) >> 1);
        if (h[mid].t_ns < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// --------------------------------------------------------------- self-check

// Built with -DTRIG_CHECK, every computed index into global or shared
// memory is checked first; a violation is recorded (the first one: site
// number, index, limit) and the access is skipped.  Without TRIG_CHECK the
// checks compile to nothing.
#ifdef TRIG_CHECK
struct CheckRecord {
    unsigned int site;
    unsigned int count;
    unsigned long long index, limit;
};
__device__ CheckRecord g_check;
__device__ __noinline__ bool check_fail(unsigned site, unsigned long long index, unsigned long long limit)
{
    if (atomicAdd(&g_check.count, 1u) == 0) {
        g_check.site = site;
        g_check.index = index;
        g_check.limit = limit;
    }
    return false;
}
#define CHECK(site, idx, lim) \
    (((unsigned long long)(idx) < (unsigned long long)(lim)) ? true : check_fail((site), (idx), (lim)))
#else
#define CHECK(site, idx, lim) true
#endif

// ------------------------------------------------------------------- dt_max

// Exact integer causality table.  For PMTs d mm apart the light needs
// d * n_num / (n_den * 1000) ns; dt_max = tol + ceil of that.  With
// X = n_num^2 * d^2 and r = floor(sqrt(X)): the ceiling is ceil(r / M) when
// X is a perfect square and floor(r / M) + 1 otherwise (M = n_den * 1000).
__global__ void k_dtmax(const int32_t *__restrict__ xyz, uint32_t P, uint32_t tol, uint32_t n_num,
                        uint32_t n_den, uint32_t corr, int32_t *__restrict__ dt_exact, uint16_t *__restrict__ dt)
{
    uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (uint64_t)P * P) return;
    uint32_t i = (uint32_t)(idx / P), j = (uint32_t)(idx % P);
    int64_t d2 = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        int64_t dx = (int64_t)xyz[3 * i + c] - (int64_t)xyz[3 * j + c];
        d2 += dx * dx;
    }
    unsigned __int128 X = (unsigned __int128)((uint64_t)n_num * n_num) * (uint64_t)d2;
    uint64_t r = (uint64_t)sqrt((double)X);
    while ((unsigned __int128)r * r > X) --r;
    while ((unsigned __int128)(r + 1) * (r + 1) <= X) ++r;
    const uint64_t M = (uint64_t)n_den * 1000u;
    uint64_t k = ((unsigned __int128)r * r == X) ? (r + M - 1) / M : r / M + 1;
    uint64_t v = (uint64_t)tol + k;
    dt_exact[idx] = v > 0x7fffffffull ? 0x7fffffff : (int32_t)v;
    dt[idx] = (uint16_t)(v < corr ? v : corr);
}

__global__ void k_row_max(const uint16_t *__restrict__ dt, uint32_t P, uint16_t *__restrict__ dmax_row)
{
    uint32_t p = blockIdx.x;
    uint32_t m = 0;
    for (uint32_t q = threadIdx.x; q < P; q += blockDim.x) m = max(m, (uint32_t)dt[(size_t)p * P + q]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ uint32_t wm[32];
    if (lane_id() == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t r = 0;
        for (uint32_t w = 0; w < (blockDim.x + 31) / 32; ++w) r = max(r, wm[w]);
        dmax_row[p] = (uint16_t)r;
    }
}

cudaError_t launch_dtmax(const int32_t *xyz, uint32_t n_pmt, uint32_t tol, uint32_t n_num, uint32_t n_den,
                         uint32_t corr, int32_t *dt_exact, uint16_t *dt, uint16_t *dmax_row, cudaStream_t st)
{
    uint64_t n = (uint64_t)n_pmt * n_pmt;
    k_dtmax<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(xyz, n_pmt, tol, n_num, n_den, corr, dt_exact, dt);
    k_row_max<<<n_pmt, 256, 0, st>>>(dt, n_pmt, dmax_row);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ uint32_t find_slice_by_item(const SliceDesc *desc, uint32_t n, uint32_t item)
{
    // largest s with desc[s].item0 <= item
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (desc[mid].item0 <= item) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t find_slice_by_chunk(const SliceDesc *desc, uint32_t n, uint32_t c)
{
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (desc[mid].chunk0 <= c) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void report(const SliceDesc &d, uint32_t flags)
{
    atomicOr(&d.stats->flags, flags);
}

// Time bucket of a wide slice: floor((t - O) / Wb) clamped to [0, NB).
// For offsets below 2^31 the high half of rel * ceil(2^32 / Wb) is the
// quotient or one more; one multiply corrects it.
__device__ __forceinline__ uint32_t bkt_index(const SliceDesc &d, int64_t t)
{
    const int64_t rel = t - d.bkt_origin;
    if (rel <= 0) return 0u;
    uint32_t q;
    if (d.bkt32 && rel < ((int64_t)1 << 31)) {
        const uint32_t r = (uint32_t)rel;
        q = __umulhi(r, d.bkt_magic);
        if (q * d.bkt_w > r) --q;
    } else {
        const int64_t q64 = rel / (int64_t)d.bkt_w;
        q = q64 >= (int64_t)d.n_bkt ? d.n_bkt : (uint32_t)q64;
    }
    return q < d.n_bkt ? q : d.n_bkt - 1;
}

// ---------------------------------------------------------------- k_prep

__global__ void k_prep(BatchHeader *hdr, const SliceDesc *desc)
{
    uint32_t n = hdr->n_slices;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        hdr->queue = 0;
        hdr->err = 0;
    }
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        trig_slice_stats *st = desc[s].stats;
        st->status = 0;
        st->flags = 0;
        st->n_hits = desc[s].n_hits;
        st->n_seeds = 0;
        st->n_triggers = 0;
        st->n_windows = 0;
        st->n_events = 0;
    }
    // bucket counts of the wide slices start at zero
    for (uint32_t s = 0; hdr->any_wide && s < n; ++s) {
        if (!desc[s].wide) continue;
        uint32_t *cnt = desc[s].bkt_cnt;
        const uint32_t nb = desc[s].n_bkt;
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) cnt[i] = 0;
    }
}

// ---------------------------------------------------------------- k_bounds

// Number of tile edges v_g = base + g * W (g in [0, NG)) with v_g <= t,
// i.e. floor((t - base) / W) + 1 clamped to [0, NG].  (Slices longer than
// about 2 s; kept out of line.)
__device__ __noinline__ uint32_t edges_le64(int64_t t, int64_t base, int64_t W, uint32_t ng)
{
    const int64_t rel = t - base;
    if (rel < 0) return 0u;
    const int64_t q = rel / W;
    return q + 1 >= (int64_t)ng ? ng : (uint32_t)(q + 1);
}

// Same for 0 <= rel < 2^31 and W < 2^31: the high half of rel * ceil(2^32 / W)
// is the quotient or one more; one multiply corrects it.
__device__ __forceinline__ uint32_t edges_le32(int64_t rel64, uint32_t W, uint32_t magic, uint32_t ng)
{
    if (rel64 < 0) return 0u;
    const uint32_t rel = (uint32_t)rel64;
    uint32_t q = __umulhi(rel, magic);
    if (q * W > rel) --q;
    return q + 1 >= ng ? ng : q + 1;
}

__device__ __forceinline__ void fill_edges(uint32_t *e, uint32_t P, uint32_t p, uint32_t g0, uint32_t g1,
                                           uint32_t v)
{
    for (uint32_t g = g0; g < g1; ++g)
        if (CHECK(1, (size_t)g * P + p, (size_t)g1 * P)) e[(size_t)g * P + p] = v;
}

// Edges after a PMT's last hit, and all edges of the empty PMTs that follow.
__device__ __noinline__ void fill_run_end(uint32_t *e_lo, uint32_t *e_hi, const uint64_t *poff, uint32_t P,
                                          uint32_t NG, uint32_t p, uint32_t lo_to, uint32_t hi_to, uint32_t ep)
{
    fill_edges(e_lo, P, p, lo_to, NG, ep);
    fill_edges(e_hi, P, p, hi_to, NG, ep);
    for (uint32_t q = p + 1; q < P && poff[q] == poff[q + 1]; ++q) {
        fill_edges(e_lo, P, q, 0, NG, ep);
        fill_edges(e_hi, P, q, 0, NG, ep);
    }
}

// All edges of the empty PMTs before the slice's first hit.
__device__ __noinline__ void fill_leading_empty(uint32_t *e_lo, uint32_t *e_hi, uint32_t P, uint32_t NG, uint32_t p)
{
    for (uint32_t q = 0; q < p; ++q) {
        fill_edges(e_lo, P, q, 0, NG, 0u);
        fill_edges(e_hi, P, q, 0, NG, 0u);
    }
}

constexpr int kBoundsThreads = 256;
constexpr int kBoundsUnroll = 4;
constexpr uint32_t kBoundsPerWarp = kChunkHits / (kBoundsThreads / 32);    // consecutive hits per warp

// Structure pass over one chunk of a wide slice: the same checks of the CSR
// layout and time order, then each valid hit counted in its time bucket.
__device__ __noinline__ void bounds_wide_chunk(const SliceDesc &d, uint64_t first)
{
    const uint32_t lane = lane_id(), P = d.n_pmt;
    const uint64_t n_hits = d.n_hits;
    const trig_hit *__restrict__ hits = d.hits;
    const uint64_t *__restrict__ poff = d.pmt_off;
    for (uint32_t k0 = 0; k0 < kChunkHits; k0 += kBoundsThreads) {
        const uint64_t li = first + k0 + threadIdx.x;
        const bool valid = li < n_hits;
        trig_hit h;
        if (valid) h = load_hit(hits + li);
        else h.t_ns = 0, h.pmt = 0xffff;
        const uint32_t p = h.pmt;
        const int64_t t = h.t_ns;
        uint32_t pp = __shfl_up_sync(0xffffffffu, p, 1);
        int64_t tp = __shfl_up_sync(0xffffffffu, t, 1);
        uint32_t pn = __shfl_down_sync(0xffffffffu, p, 1);
        if (!valid) continue;
        if (lane == 0 && li > 0) {
            const trig_hit q = load_hit(hits + li - 1);
            pp = q.pmt;
            tp = q.t_ns;
        }
        if (lane == 31 && li + 1 < n_hits) pn = hits[li + 1].pmt;
        const bool is_first = li == 0 || pp != p;
        const bool is_last = li + 1 == n_hits || pn != p;
        uint32_t bad = 0;
        if (p >= P) bad |= TRIG_FLAG_BAD_PMT;
        else {
            if (is_first && poff[p] != li) bad |= TRIG_FLAG_BAD_PMT;
            if (is_last && poff[p + 1] != li + 1) bad |= TRIG_FLAG_BAD_PMT;
            if (li + 1 == n_hits && poff[P] != n_hits) bad |= TRIG_FLAG_BAD_PMT;
        }
        if (t < d.in_lo || t >= d.in_hi) bad |= TRIG_FLAG_OUT_OF_RANGE;
        if (!is_first && tp > t) bad |= TRIG_FLAG_UNSORTED;
        if (bad) {
            report(d, bad);
            continue;
        }
        atomicAdd(&d.bkt_cnt[bkt_index(d, t)], 1u);
    }
}

// One read of every hit.  Per hit: CSR layout and time order are checked
// (run starts and ends against pmt_off, neighbours from adjacent lanes), and
// the tile edges passed between the previous hit of the PMT and this one
// get this hit's index.
__global__ void __launch_bounds__(kBoundsThreads, 4) k_bounds(const BatchHeader *__restrict__ hdr,
                                                           const SliceDesc *__restrict__ desc)
{
    const uint32_t n_slices = hdr->n_slices, n_chunks = hdr->n_chunks;
    const uint32_t lane = lane_id();
    for (uint32_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        const uint32_t s = find_slice_by_chunk(desc, n_slices, c);
        const SliceDesc &d = desc[s];
        const uint32_t P = d.n_pmt, NG = d.n_tiles;
        const int64_t W = d.tile_w;
        const uint32_t W32 = (uint32_t)W, magic = d.w_magic;
        const bool span32 = d.span32 != 0;
        const int64_t base_lo = d.t0 - (int64_t)d.halo;             // lo edge g: t0 - H + g W
        const int64_t base_hi = d.t0 + (int64_t)d.halo + W;         // hi edge g: t0 + H + (g + 1) W
        const uint64_t first = (uint64_t)(c - d.chunk0) * kChunkHits;
        const uint64_t n_hits = d.n_hits;
        const trig_hit *__restrict__ hits = d.hits;
        const uint64_t *__restrict__ poff = d.pmt_off;
        uint32_t *__restrict__ e_lo = d.e_lo;
        uint32_t *__restrict__ e_hi = d.e_hi;
        const int64_t in_lo = d.in_lo, in_hi = d.in_hi;
        if (d.wide) {
            bounds_wide_chunk(d, first);
            continue;
        }
        // tile edges at or below t: lo edge g at base_lo + g W, hi edge g at
        // base_lo + D + g W with D = 2H + W = a W + b; with t - base_lo =
        // q W + r the hi count is q - a + 1 - (r < b), so one division
        // serves both
        const uint32_t D32 = 2u * d.halo + W32, a32 = span32 ? D32 / W32 : 0u, b32 = D32 - a32 * W32;
        auto edges = [&](int64_t t, uint32_t &lo, uint32_t &hi) {
            if (span32) {
                const int64_t x64 = t - base_lo;
                if (x64 < 0) {
                    lo = hi = 0u;
                    return;
                }
                const uint32_t x = (uint32_t)x64;
                uint32_t q = __umulhi(x, magic);
                if (q * W32 > x) --q;
                const uint32_t r = x - q * W32;
                lo = q + 1 >= NG ? NG : q + 1;
                const int32_t qh = (int32_t)q - (int32_t)a32 + 1 - (r < b32 ? 1 : 0);
                hi = qh <= 0 ? 0u : ((uint32_t)qh >= NG ? NG : (uint32_t)qh);
            } else {
                lo = edges_le64(t, base_lo, W, NG);
                hi = edges_le64(t, base_hi, W, NG);
            }
        };
        // each warp walks kBoundsPerWarp consecutive hits, 32 at a time: a
        // hit's predecessor is the previous lane's (lane 0: the previous
        // step's lane 31; the first step loads it).  The first hit of a run
        // closes the previous PMT's run.
        const uint32_t warp = threadIdx.x >> 5;
        const uint64_t wbase = first + (uint64_t)warp * kBoundsPerWarp;
        uint32_t c_p = 0xffffu, c_lo = 0u, c_hi = 0u;
        int64_t c_t = 0;
        if (wbase > 0 && wbase <= n_hits) {
            const trig_hit q = load_hit(hits + wbase - 1);
            c_p = q.pmt;
            c_t = q.t_ns;
            edges(c_t, c_lo, c_hi);
        }
        for (uint32_t k0 = 0; k0 < kBoundsPerWarp; k0 += 32 * kBoundsUnroll) {
            trig_hit h[kBoundsUnroll];
#pragma unroll
            for (int u = 0; u < kBoundsUnroll; ++u) {
                const uint64_t li = wbase + k0 + u * 32 + lane;
                if (li < n_hits) h[u] = load_hit(hits + li);
                else h[u].t_ns = 0, h[u].pmt = 0xffff;
            }
#pragma unroll
            for (int u = 0; u < kBoundsUnroll; ++u) {
                const uint64_t li = wbase + k0 + u * 32 + lane;
                const bool valid = li < n_hits;
                const uint32_t p = h[u].pmt;
                const int64_t t = h[u].t_ns;
                uint32_t lo_to = 0u, hi_to = 0u;
                if (valid) edges(t, lo_to, hi_to);
                uint32_t pp = __shfl_up_sync(0xffffffffu, p, 1);
                int64_t tp = __shfl_up_sync(0xffffffffu, t, 1);
                uint32_t lo_p = __shfl_up_sync(0xffffffffu, lo_to, 1);
                uint32_t hi_p = __shfl_up_sync(0xffffffffu, hi_to, 1);
                if (lane == 0) {
                    pp = c_p;
                    tp = c_t;
                    lo_p = c_lo;
                    hi_p = c_hi;
                }
                c_p = __shfl_sync(0xffffffffu, p, 31);
                c_t = __shfl_sync(0xffffffffu, t, 31);
                c_lo = __shfl_sync(0xffffffffu, lo_to, 31);
                c_hi = __shfl_sync(0xffffffffu, hi_to, 31);
                if (!valid) continue;
                const bool is_first = li == 0 || pp != p;
                uint32_t bad = 0;
                if (is_first && li > 0 && pp < P) {
                    // hit li - 1 was the last of PMT pp's run
                    if (poff[pp + 1] != li) bad |= TRIG_FLAG_BAD_PMT;
                    fill_run_end(e_lo, e_hi, poff, P, NG, pp, lo_p, hi_p, (uint32_t)li);
                }
                if (p >= P) bad |= TRIG_FLAG_BAD_PMT;
                else {
                    if (is_first && poff[p] != li) bad |= TRIG_FLAG_BAD_PMT;
                    if (li + 1 == n_hits && (poff[p + 1] != n_hits || poff[P] != n_hits)) bad |= TRIG_FLAG_BAD_PMT;
                }
                if (t < in_lo || t >= in_hi) bad |= TRIG_FLAG_OUT_OF_RANGE;
                if (!is_first && tp > t) bad |= TRIG_FLAG_UNSORTED;
                if (bad) { report(d, bad); continue; }
                fill_edges(e_lo, P, p, is_first ? 0u : lo_p, lo_to, (uint32_t)li);
                fill_edges(e_hi, P, p, is_first ? 0u : hi_p, hi_to, (uint32_t)li);
                if (li + 1 == n_hits) fill_run_end(e_lo, e_hi, poff, P, NG, p, lo_to, hi_to, (uint32_t)(li + 1));
                if (li == 0 && p > 0) fill_leading_empty(e_lo, e_hi, P, NG, p);
            }
        }
    }
}

// ----------------------------------------------------------- k_bsum, k_bscan

// Wide slices: bucket offsets = exclusive prefix of the bucket counts, in
// two grid-wide passes over chunks of kBktChunk buckets (a block per chunk):
// the chunk sums, then each chunk's scan from the sums of the chunks before
// it.  The counts are reset to serve as fill cursors of the scatter.
__global__ void __launch_bounds__(kBktChunk) k_bsum(const BatchHeader *__restrict__ hdr,
                                                    const SliceDesc *__restrict__ desc)
{
    __shared__ uint32_t wsum[32];
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    for (uint32_t s = 0; s < hdr->n_slices; ++s) {
        const SliceDesc &d = desc[s];
        if (!d.wide) continue;
        const uint32_t nb = d.n_bkt, nch = (nb + kBktChunk - 1) / kBktChunk;
        for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
            const uint32_t i = c * kBktChunk + tid;
            uint32_t v = i < nb ? d.bkt_cnt[i] : 0u;
            v = __reduce_add_sync(0xffffffffu, v);
            if (lane == 0) wsum[warp] = v;
            __syncthreads();
            if (warp == 0) {
                uint32_t t = lane < kBktChunk / 32 ? wsum[lane] : 0u;
                t = __reduce_add_sync(0xffffffffu, t);
                if (lane == 0) d.bkt_part[c] = t;
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kBktChunk) k_bscan(const BatchHeader *__restrict__ hdr,
                                                     const SliceDesc *__restrict__ desc)
{
    __shared__ uint32_t wsum[33];
    __shared__ uint32_t base;
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    constexpr uint32_t NW = kBktChunk / 32;
    for (uint32_t s = 0; s < hdr->n_slices; ++s) {
        const SliceDesc &d = desc[s];
        if (!d.wide) continue;
        const uint32_t nb = d.n_bkt, nch = (nb + kBktChunk - 1) / kBktChunk;
        for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
            // sum of the chunks before c
            uint32_t pre = 0;
            for (uint32_t q = tid; q < c; q += kBktChunk) pre += d.bkt_part[q];
            pre = __reduce_add_sync(0xffffffffu, pre);
            if (lane == 0) wsum[warp] = pre;
            __syncthreads();
            if (warp == 0) {
                uint32_t t = lane < NW ? wsum[lane] : 0u;
                t = __reduce_add_sync(0xffffffffu, t);
                if (lane == 0) base = t;
            }
            __syncthreads();
            // the chunk's own exclusive scan
            const uint32_t i = c * kBktChunk + tid;
            const uint32_t v = i < nb ? d.bkt_cnt[i] : 0u;
            const uint32_t incl = warp_incl_scan(v);
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();
            if (warp == 0) {
                const uint32_t w = lane < NW ? wsum[lane] : 0u;
                const uint32_t wi = warp_incl_scan(w);
                if (lane < NW) wsum[lane] = wi - w;
                if (lane == NW - 1) wsum[32] = wi;
            }
            __syncthreads();
            if (i < nb) {
                d.bkt_off[i] = base + wsum[warp] + incl - v;
                d.bkt_cnt[i] = 0;
            }
            if (c == nch - 1 && tid == 0) d.bkt_off[nb] = base + wsum[32];
            __syncthreads();
        }
    }
}

// --------------------------------------------------------------- k_scatter

// Wide slices: every hit copied to its time bucket's range of tbuf (the
// order inside a bucket is arbitrary; the tile pass sorts).  Slices with
// malformed input (flagged by the structure pass) are skipped.
__global__ void __launch_bounds__(256) k_scatter(const BatchHeader *__restrict__ hdr, const SliceDesc *__restrict__ desc)
{
    const uint32_t n_slices = hdr->n_slices, n_chunks = hdr->n_chunks;
    for (uint32_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        const SliceDesc &d = desc[find_slice_by_chunk(desc, n_slices, c)];
        if (!d.wide) continue;
        if (d.stats->flags & (TRIG_FLAG_BAD_PMT | TRIG_FLAG_UNSORTED | TRIG_FLAG_OUT_OF_RANGE)) continue;
        const uint64_t first = (uint64_t)(c - d.chunk0) * kChunkHits;
        for (uint32_t k = threadIdx.x; k < kChunkHits; k += blockDim.x) {
            const uint64_t li = first + k;
            if (li >= d.n_hits) break;
            const int4 v = *reinterpret_cast<const int4 *>(d.hits + li);
            const int64_t t = (int64_t)(((uint64_t)(uint32_t)v.y << 32) | (uint32_t)v.x);
            const uint32_t b = bkt_index(d, t);
            const uint32_t pos = d.bkt_off[b] + atomicAdd(&d.bkt_cnt[b], 1u);
            if (CHECK(17, pos, d.n_hits)) *reinterpret_cast<int4 *>(d.tbuf + pos) = v;
        }
    }
}

// ------------------------------------------------------------------ k_tile

struct ItemInfo {
    int32_t item;       // -1: no more work
    uint32_t slice;
    uint32_t g;
    uint32_t n;         // staged hits
    uint32_t rank_lo;   // merged rank of the first staged hit
    uint32_t mode;      // 0 staged, 1 overflow (split path), 2 skip (bad slice or empty)
    uint32_t lo_t;      // B_g minus the time of the staged range's start
    uint32_t span;      // length of the staged time range (ns)
};

// Shared memory of the tile kernel, in this order: the staging buffers of
// CAP 16-byte records (two, or one for the 2048-hit tile: its tile pass
// hands the buffer back once it has read it, so the next tile's copy
// overlaps the rest of the pass, and two blocks of it then fit on an SM);
// the tile's packed keys in merged order (+16 bytes: four end keys that the
// causal count's 16-byte loads may read past the last key); the keys in
// bucket order (reused for the seed rounds' lists, then the seed list and
// seed counts); the charges in bucket order and in merged order; the floor
// of each merged key; the bucket offsets; the seed mask; the PMT tables
// (floor, row maximum of dt, and dt itself when the detector's table fits).
template <int CAP>
struct TileLayout {
    // time buckets of the in-tile merge, at most: two per hit slot up to
    // 2048 hits (shorter chains in the floor-coincidence rounds), one at 4096
    static constexpr int NBK = CAP <= 2048 ? 2 * CAP : CAP;
    static constexpr uint32_t NS = CAP == 2048 ? 1u : 2u;  // staging buffers
    static constexpr size_t kStage = (size_t)CAP * 16;     // one staging buffer
    static constexpr size_t kPkS = (size_t)CAP * 4 + 16;
    static constexpr size_t kPkB = (size_t)CAP * 4;
    static constexpr size_t kChg = (size_t)CAP * 2;
    static constexpr size_t kFlk = (size_t)CAP * 2;
    static constexpr size_t kCnt = (size_t)(NBK + 1) * 4;
    static constexpr size_t kMask = (size_t)(CAP / 32) * 4;
    static constexpr size_t oPkS = NS * kStage;
    static constexpr size_t oPkB = oPkS + kPkS;
    static constexpr size_t oChgB = oPkB + kPkB;
    static constexpr size_t oChgS = oChgB + kChg;
    static constexpr size_t oFlk = oChgS + kChg;
    static constexpr size_t oCnt = oFlk + kFlk;
    static constexpr size_t oMask = oCnt + kCnt;
    static constexpr size_t oTab = (oMask + kMask + 15) & ~(size_t)15;
    static_assert(oCnt % 16 == 0, "the bucket counts are read as 16-byte vectors");
    static size_t bytes(uint32_t P, bool smem_dt)
    {
        size_t b = oTab;
        b += 2 * (size_t)((P + 7) & ~7u) * 2;              // floor + dmax_row
        if (smem_dt) b += (size_t)P * P * 2;
        return (b + 127) & ~(size_t)127;
    }
};

// Dynamic shared memory of the tile kernel (layout TileLayout<CAP>).
extern __shared__ __align__(128) unsigned char g_tile_smem[];

// The tile kernel's shared-memory regions sit at fixed offsets, so their
// addresses are recomputed where used instead of living in registers
// through every phase; only the PMT-table stride depends on the launch.
template <int CAP>
struct TileCtx {
    using L = TileLayout<CAP>;
    uint32_t P;             // PMTs of the loaded slice
    uint32_t pp;            // PMT table stride: the launch's max_pmt rounded up to 8
    const uint16_t *dt_g;   // the loaded slice's dt table in global memory
    __device__ __forceinline__ uint64_t *stage(uint32_t b) const
    {
        return reinterpret_cast<uint64_t *>(g_tile_smem + (size_t)b * L::kStage);
    }
    __device__ __forceinline__ uint32_t *pk_s() const { return reinterpret_cast<uint32_t *>(g_tile_smem + L::oPkS); }
    __device__ __forceinline__ uint32_t *pk_b() const { return reinterpret_cast<uint32_t *>(g_tile_smem + L::oPkB); }
    __device__ __forceinline__ uint16_t *seed_idx() const { return reinterpret_cast<uint16_t *>(g_tile_smem + L::oPkB); }
    __device__ __forceinline__ uint16_t *seed_cnt() const
    {
        return reinterpret_cast<uint16_t *>(g_tile_smem + L::oPkB) + CAP;
    }
    __device__ __forceinline__ uint16_t *chg_b() const { return reinterpret_cast<uint16_t *>(g_tile_smem + L::oChgB); }
    __device__ __forceinline__ uint16_t *chg_s() const { return reinterpret_cast<uint16_t *>(g_tile_smem + L::oChgS); }
    __device__ __forceinline__ uint16_t *flk() const { return reinterpret_cast<uint16_t *>(g_tile_smem + L::oFlk); }
    // per-warp lists of the seed rounds (the bucket-order key region, free then)
    __device__ __forceinline__ uint16_t *live() const { return reinterpret_cast<uint16_t *>(g_tile_smem + L::oPkB); }
    __device__ __forceinline__ uint32_t *cnt() const { return reinterpret_cast<uint32_t *>(g_tile_smem + L::oCnt); }
    __device__ __forceinline__ uint32_t *mask() const { return reinterpret_cast<uint32_t *>(g_tile_smem + L::oMask); }
    // warp w's 4096-bit PMT set of the distinct count above 128 PMTs (extended
    // builds: the bucket-order charges and the floor keys are no longer read
    // by then; each region holds CAP / 256 sets)
    __device__ __forceinline__ uint32_t *pmt_set(uint32_t w) const
    {
        constexpr uint32_t per = (uint32_t)CAP / 256;
        return w < per ? reinterpret_cast<uint32_t *>(g_tile_smem + L::oChgB) + 128 * w
                       : reinterpret_cast<uint32_t *>(g_tile_smem + L::oFlk) + 128 * (w - per);
    }
    __device__ __forceinline__ uint16_t *floor_s() const { return reinterpret_cast<uint16_t *>(g_tile_smem + L::oTab); }
    __device__ __forceinline__ uint16_t *dmax_s() const { return floor_s() + pp; }
    __device__ __forceinline__ uint16_t *dt_s() const { return floor_s() + 2 * (size_t)pp; }
};

constexpr uint32_t kBarCons = 1;        // named barrier of the consumers

// Floor coincidences in bucket order: candidates of a key checked in the
// first pass before the rounds take over.
constexpr uint32_t kFloorPairs = 3;

template <int NC>
__device__ __forceinline__ void cons_sync() { named_sync(kBarCons, NC); }

__device__ __forceinline__ uint32_t key_t(uint64_t k) { return (uint32_t)(k >> 32); }
__device__ __forceinline__ uint32_t key_p(uint64_t k) { return (uint32_t)(k >> 16) & 0xffffu; }
__device__ __forceinline__ uint32_t key_q(uint64_t k) { return (uint32_t)k & 0xffffu; }

// Packed key of the trigger phases: time within the staged range (below
// 2^20 ns) and PMT (below 2^12).  0xffffffff marks "no hit".
constexpr uint32_t kPkNone = 0xffffffffu;
__device__ __forceinline__ uint32_t pk_t(uint32_t k) { return k >> 12; }
__device__ __forceinline__ uint32_t pk_p(uint32_t k) { return k & 0xfffu; }

// Consumer-wide exclusive scan of cnt[0..nb), nb a multiple of NC; writes
// the total to cnt[nb].  Scratch words red[0..NC/32].
template <int NC, uint32_t NB>
__device__ void cons_exclusive_scan(uint32_t *cnt, uint32_t *red)
{
    constexpr uint32_t NW = NC / 32, PER = NB / NC, V = PER / 4;
    static_assert(NB % NC == 0 && PER % 4 == 0, "each thread scans whole 16-byte vectors");
    const uint32_t tid = threadIdx.x;
    uint4 *c4 = reinterpret_cast<uint4 *>(cnt) + tid * V;
    uint4 v[V];
    uint32_t local = 0;
#pragma unroll
    for (uint32_t i = 0; i < V; ++i) {
        v[i] = c4[i];
        local += v[i].x + v[i].y + v[i].z + v[i].w;
    }
    uint32_t incl = warp_incl_scan(local);
    if (lane_id() == 31) red[tid >> 5] = incl;
    cons_sync<NC>();
    if (tid < 32) {
        uint32_t w = tid < NW ? red[tid] : 0u;
        uint32_t wi = warp_incl_scan(w);
        if (tid < NW) red[tid] = wi - w;
        if (tid == NW - 1) red[NW] = wi;
    }
    cons_sync<NC>();
    uint32_t run = red[tid >> 5] + incl - local;
#pragma unroll
    for (uint32_t i = 0; i < V; ++i) {
        uint4 o;
        o.x = run;
        o.y = o.x + v[i].x;
        o.z = o.y + v[i].y;
        o.w = o.z + v[i].z;
        run = o.w + v[i].w;
        c4[i] = o;
    }
    if (tid == 0) cnt[NB] = red[NW];
    cons_sync<NC>();
}

// Bucket of a time relative to the tile base: t_rel >> bsh, the last of
// the NB buckets taking everything beyond.
template <uint32_t NB>
__device__ __forceinline__ uint32_t bucket_of(uint32_t t_rel, uint32_t bsh)
{
    const uint32_t b = t_rel >> bsh;
    return b < NB ? b : NB - 1;
}

struct CoreOut {
    uint32_t n_fired;
    uint32_t n_seeds;
    uint32_t c0;
};

// Seeds, causal counts and emission over the sorted tile keys[0..n).  The
// core is t_rel in [H, H + core_w).  Fired seeds go to out[0..n_fired).
struct TrigParams {
    uint32_t H, tau, q_seed, threshold, win_half;
    uint32_t l0_hits, l0_window, l0_distinct;
    uint32_t seed_rule, sc_w, fc_w, afc_w, count_distinct;
    const uint8_t *rel;
    trig_hit *dbg_merged;
    uint32_t *dbg_seedcnt;
};

// Seed rule 1 at sorted index i: [SC and AFC] or [FC and AFC].  Walks the
// keys within the widest of the three windows on both sides (all staged:
// the tile halo covers it) and looks each pair up in the PMT relation row
// of p_i.
__device__ __noinline__ bool coincidence_seed(const uint32_t *pk, uint32_t n, uint32_t i, const uint8_t *rel,
                                              uint32_t P, uint32_t sc, uint32_t fc, uint32_t afc)
{
    const uint32_t ki = pk[i], ti = pk_t(ki), pi = pk_p(ki);
    if (!CHECK(14, pi, P)) return false;
    const uint8_t *row = rel + (size_t)pi * P;
    const uint32_t wmax = max(sc, max(fc, afc));
    bool c = false, a = false;
    for (uint32_t j = i + 1; j < n; ++j) {
        const uint32_t kj = pk[j], d = pk_t(kj) - ti;
        if (d > wmax) break;
        if (!CHECK(15, pk_p(kj), P)) continue;
        const uint32_t r = __ldg(row + pk_p(kj));
        c = c || ((r & kRelAdjacent) && d <= sc) || ((r & kRelFloor) && d <= fc);
        a = a || ((r & kRelNextFloor) && d <= afc);
        if (a && c) return true;
    }
    for (uint32_t j = i; j-- > 0;) {
        const uint32_t kj = pk[j], d = ti - pk_t(kj);
        if (d > wmax) break;
        if (!CHECK(15, pk_p(kj), P)) continue;
        const uint32_t r = __ldg(row + pk_p(kj));
        c = c || ((r & kRelAdjacent) && d <= sc) || ((r & kRelFloor) && d <= fc);
        a = a || ((r & kRelNextFloor) && d <= afc);
        if (a && c) return true;
    }
    return false;
}

// A seed's scan range: the keys [j0, j1) of the buckets covering
// [t_s - d, t_s + d], d its row's maximum (keys beyond fail the causal
// test), from the sorted tile's bucket offsets.
template <int CAP, uint32_t NB>
__device__ __forceinline__ void seed_range(const TileCtx<CAP> &cx, uint32_t ts, uint32_t ps, uint32_t bsh,
                                           uint32_t &j0, uint32_t &j1)
{
    const uint32_t dm = ps < cx.P ? (uint32_t)cx.dmax_s()[ps] : 0u;
    const uint32_t *boff = cx.cnt();
    j0 = boff[bucket_of<NB>(ts >= dm ? ts - dm : 0u, bsh)];
    j1 = boff[bucket_of<NB>(ts + dm, bsh) + 1];
}

// Distinct-PMT causal count: c(s) = the number of different PMTs among the
// keys j with |t_j - t_s| <= min(dt_max[p_s][p_j], W).  Up to 128 PMTs,
// eight lanes per seed each collect a 128-bit PMT set in registers over
// every eighth key of the seed's scan range, and the sets are OR-ed and
// counted; above, a warp per seed marks the PMTs in a shared-memory set.
template <int CAP, int NC, bool SMEM_DT, uint32_t NB>
__device__ __noinline__ void count_distinct_pmts(const TileCtx<CAP> &cx, const uint32_t *pk, uint32_t n, uint32_t ns,
                                                 const uint16_t *seed_idx, uint32_t bsh, uint16_t *seed_cnt)
{
    constexpr uint32_t G = 8, NG = NC / G;
    static_assert(NC / 32 <= CAP / 128, "a PMT set per consumer warp");
    const uint32_t tid = threadIdx.x, gl = tid & (G - 1u), gid = tid / G, P = cx.P;
    if (P > 128) {
        const uint32_t warp = tid >> 5, lane = tid & 31u, nwords = (P + 31u) >> 5;
        uint32_t *set = cx.pmt_set(warp);
        for (uint32_t k = warp; k < ns; k += NC / 32) {
            for (uint32_t w = lane; w < nwords; w += 32) set[w] = 0u;
            __syncwarp();
            const uint32_t ks = pk[seed_idx[k]];
            const uint32_t ts = pk_t(ks), ps = pk_p(ks);
            uint32_t j0, j1;
            seed_range<CAP, NB>(cx, ts, ps, bsh, j0, j1);
            if (CHECK(12, j1, n + 1) && CHECK(13, ps, P) && CHECK(16, nwords, 129)) {
                const uint16_t *row_s = cx.dt_s() + (size_t)ps * P;
                const uint16_t *row_g = cx.dt_g + (size_t)ps * P;
                for (uint32_t q = j0 + lane; q < j1; q += 32) {
                    const uint32_t kj = pk[q], tj = pk_t(kj), pj = pk_p(kj);
                    if (!CHECK(11, pj, P)) continue;
                    const uint32_t lim = SMEM_DT ? (uint32_t)row_s[pj] : (uint32_t)__ldg(row_g + pj);
                    if ((tj > ts ? tj - ts : ts - tj) <= lim) atomicOr(&set[pj >> 5], 1u << (pj & 31u));
                }
            }
            __syncwarp();
            uint32_t c = 0;
            for (uint32_t w = lane; w < nwords; w += 32) c += __popc(set[w]);
            c = __reduce_add_sync(0xffffffffu, c);
            if (lane == 0) seed_cnt[k] = (uint16_t)c;
            __syncwarp();                       // the set is read before the next seed clears it
        }
        return;
    }
    const uint32_t rounds = (ns + NG - 1) / NG;
    for (uint32_t r = 0; r < rounds; ++r) {
        const uint32_t k = r * NG + gid;
        uint32_t m0 = 0, m1 = 0, m2 = 0, m3 = 0;
        if (k < ns) {
            const uint32_t ks = pk[seed_idx[k]];
            const uint32_t ts = pk_t(ks), ps = pk_p(ks);
            uint32_t j0, j1;
            seed_range<CAP, NB>(cx, ts, ps, bsh, j0, j1);
            if (CHECK(12, j1, n + 1) && CHECK(13, ps, P)) {
                const uint16_t *row_s = cx.dt_s() + (size_t)ps * P;
                const uint16_t *row_g = cx.dt_g + (size_t)ps * P;
                for (uint32_t q = j0 + gl; q < j1; q += G) {
                    const uint32_t kj = pk[q], tj = pk_t(kj), pj = pk_p(kj);
                    if (!CHECK(11, pj, P)) continue;
                    const uint32_t lim = SMEM_DT ? (uint32_t)row_s[pj] : (uint32_t)__ldg(row_g + pj);
                    if ((tj > ts ? tj - ts : ts - tj) > lim) continue;
                    const uint32_t b = 1u << (pj & 31u), h = pj >> 5;
                    m0 |= h == 0 ? b : 0u;
                    m1 |= h == 1 ? b : 0u;
                    m2 |= h == 2 ? b : 0u;
                    m3 |= h == 3 ? b : 0u;
                }
            }
        }
        for (uint32_t off = G >> 1; off; off >>= 1) {
            m0 |= __shfl_xor_sync(0xffffffffu, m0, off);
            m1 |= __shfl_xor_sync(0xffffffffu, m1, off);
            m2 |= __shfl_xor_sync(0xffffffffu, m2, off);
            m3 |= __shfl_xor_sync(0xffffffffu, m3, off);
        }
        if (k < ns && gl == 0) seed_cnt[k] = (uint16_t)(__popc(m0) + __popc(m1) + __popc(m2) + __popc(m3));
    }
}

// Level 0 at sorted index i: some window [t_j, t_j + TW) with
// t_i - TW < t_j <= t_i holds at least N hits, or hits of N different PMTs
// (P <= 128 here; above, level0_distinct_warp).  Only the first index of each time starts a window; every
// hit within TW of a core hit is staged (the tile halo covers TW).  The
// distinct count slides the window back start by start, keeping per-PMT
// counts, so it reads each hit within 2 TW once.
__device__ __noinline__ bool level0_pass(const uint32_t *pk, uint32_t n, uint32_t i, uint32_t N, uint32_t TW,
                                         bool distinct)
{
    const uint32_t ts = pk_t(pk[i]);
    uint32_t j = i;
    while (j > 0 && pk_t(pk[j - 1]) == ts) --j;             // first index of t_i
    if (!distinct) {
        for (;;) {
            const uint32_t tj = pk_t(pk[j]);
            if (j + N - 1 < n && pk_t(pk[j + N - 1]) - tj < TW) return true;
            if (j == 0) return false;
            const uint32_t tp = pk_t(pk[j - 1]);
            if (ts - tp >= TW) return false;
            for (--j; j > 0 && pk_t(pk[j - 1]) == tp; --j) {
            }
        }
    }
    uint16_t cnt[128];
    for (uint32_t p = 0; p < 128; ++p) cnt[p] = 0;
    uint32_t distinct_n = 0, e = j;
    for (;;) {
        const uint32_t tj = pk_t(pk[j]);
        while (e < n && pk_t(pk[e]) - tj < TW) {                // extend the end
            if (cnt[pk_p(pk[e]) & 127u]++ == 0) ++distinct_n;
            ++e;
        }
        if (distinct_n >= N) return true;
        if (j == 0) return false;
        const uint32_t tp = pk_t(pk[j - 1]);
        if (ts - tp >= TW) return false;
        // the previous start: add its hits, drop hits at or past tp + TW
        uint32_t nj = j - 1;
        while (nj > 0 && pk_t(pk[nj - 1]) == tp) --nj;
        for (uint32_t q = nj; q < j; ++q)
            if (cnt[pk_p(pk[q]) & 127u]++ == 0) ++distinct_n;
        while (e > j && pk_t(pk[e - 1]) - tp >= TW) {
            --e;
            if (--cnt[pk_p(pk[e]) & 127u] == 0) --distinct_n;
        }
        j = nj;
    }
}

// Level 0 with distinct PMTs above 128 PMTs, by a warp: the same window
// starts as level0_pass (each first index of a time within TW before t_i),
// each window's PMTs marked in the warp's 4096-bit set in shared memory and
// counted; the first window with N different PMTs ends the search.
__device__ __noinline__ bool level0_distinct_warp(const uint32_t *pk, uint32_t n, uint32_t i, uint32_t N, uint32_t TW,
                                                  uint32_t P, uint32_t *set)
{
    const uint32_t lane = lane_id(), nwords = (P + 31u) >> 5;
    const uint32_t ts = pk_t(pk[i]);
    uint32_t j = i;
    while (j > 0 && pk_t(pk[j - 1]) == ts) --j;             // first index of t_i
    for (;;) {
        const uint32_t tj = pk_t(pk[j]);
        for (uint32_t w = lane; w < nwords; w += 32) set[w] = 0u;
        __syncwarp();
        // the window [t_j, t_j + TW): keys from j on, in time order
        for (uint32_t k0 = j; k0 < n; k0 += 32) {
            const uint32_t k = k0 + lane;
            bool in = false;
            if (k < n) {
                const uint32_t kk = pk[k], pj = pk_p(kk);
                in = pk_t(kk) - tj < TW;
                if (in && CHECK(27, pj, P)) atomicOr(&set[pj >> 5], 1u << (pj & 31u));
            }
            if (!__any_sync(0xffffffffu, in)) break;
        }
        __syncwarp();
        uint32_t c = 0;
        for (uint32_t w = lane; w < nwords; w += 32) c += __popc(set[w]);
        c = __reduce_add_sync(0xffffffffu, c);
        __syncwarp();                                       // the set is read before it is cleared again
        if (c >= N) return true;
        if (j == 0) return false;
        const uint32_t tp = pk_t(pk[j - 1]);
        if (ts - tp >= TW) return false;
        for (--j; j > 0 && pk_t(pk[j - 1]) == tp; --j) {
        }
    }
}

// Causal count c(s) = #{ j : |t_j - t_s| <= min(dt_max[p_s][p_j], W) }
// over each seed's scan range keys [j0, j1) (seed_range): a group of 2^LG
// lanes per seed,
// seeds dealt round-robin to the groups, four independent tests per lane in
// flight.
template <int CAP, int NC, bool SMEM_DT, uint32_t LG, uint32_t NB>
__device__ __forceinline__ void count_causal(const TileCtx<CAP> &cx, const uint32_t *pk, uint32_t n, uint32_t ns,
                                             const uint16_t *seed_idx, uint32_t bsh, uint16_t *seed_cnt)
{
    constexpr uint32_t G = 1u << LG, NG = NC >> LG;
    const uint32_t tid = threadIdx.x, gl = tid & (G - 1u), gid = tid >> LG, P = cx.P;
    const uint32_t rounds = (ns + NG - 1) / NG;
#ifdef TRIG_PHASE_STATS
    uint32_t keys_seen = 0;
    struct Flush {
        uint32_t &k;
        __device__ ~Flush()
        {
            const uint32_t w = __reduce_add_sync(0xffffffffu, k);
            if ((threadIdx.x & 31u) == 0 && w) PHASE_ADD(kPhKeys, w);
        }
    } flush{keys_seen};
#endif
    for (uint32_t r = 0; r < rounds; ++r) {
        const uint32_t k = r * NG + gid;
        uint32_t c = 0;
        if (k < ns) {
            const uint32_t ks = pk[seed_idx[k]];
            const uint32_t ts = pk_t(ks), ps = pk_p(ks);
            uint32_t j0, j1;
            seed_range<CAP, NB>(cx, ts, ps, bsh, j0, j1);
#ifdef TRIG_PHASE_STATS
            keys_seen += gl == 0 ? j1 - j0 : 0u;
#endif
            if (CHECK(12, j1, n + 1) && CHECK(13, ps, P)) {
                const uint16_t *row_s = cx.dt_s() + (size_t)ps * P;
                const uint16_t *row_g = cx.dt_g + (size_t)ps * P;
                // key kj counts when |t_j - t_s| <= dt[p_s][p_j]
                auto causal = [&](uint32_t kj) -> uint32_t {
                    const uint32_t tj = pk_t(kj), pj = pk_p(kj);
                    if (!CHECK(11, pj, P)) return 0u;
                    const uint32_t lim = SMEM_DT ? (uint32_t)row_s[pj] : (uint32_t)__ldg(row_g + pj);
                    return (tj > ts ? tj - ts : ts - tj) <= lim;
                };
                // each lane takes four consecutive keys per 16-byte load, from
                // j0 rounded down to a multiple of 4.  No key outside
                // [j0, j1) can pass: those before j0 lie in earlier buckets,
                // more than dmax_row(p_s) >= dt before t_s, those from j1 on
                // in later buckets, and the four end keys past the last key
                // (time 2^20 - 1, PMT 0) are beyond any dt as well
                uint32_t ca = 0, cb = 0, cc = 0, cd = 0;
                for (uint32_t q = (j0 & ~3u) + 4 * gl; q < j1; q += 4 * G) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(pk + q);
                    ca += causal(v.x);
                    cb += causal(v.y);
                    cc += causal(v.z);
                    cd += causal(v.w);
                }
                c = ca + cb + cc + cd;
            }
        }
        if (LG == 5) {
            c = __reduce_add_sync(0xffffffffu, c);
        } else {
#pragma unroll
            for (uint32_t off = G >> 1; off; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
        }
        if (k < ns && gl == 0) seed_cnt[k] = (uint16_t)c;
    }
}

// A window-edge rank the tile pass could not read off its staged keys.
constexpr uint32_t kRankUnknown = 0xffffffffu;

// Staged keys with time below x (relative to the staged range's start, x
// in [0, span]): the buckets before x's bucket, plus the keys of that bucket
// below x.  The keys of a bucket are contiguous in bucket order and in
// sorted order alike.
template <uint32_t NB>
__device__ __forceinline__ uint32_t keys_before(const uint32_t *pk, const uint32_t *cnt, uint32_t n, uint32_t x,
                                                uint32_t bsh, uint32_t span)
{
    if (x >= span) return n;
    const uint32_t b = bucket_of<NB>(x, bsh);
    uint32_t c = cnt[b];
    const uint32_t e = cnt[b + 1];
    for (uint32_t m = c; m < e; ++m) c += pk_t(pk[m]) < x;
    return c;
}

// Bucket shift of a staged range of `span` ns: buckets of 2^bsh ns, NBK of
// them cover the range.
template <uint32_t NB>
__device__ __forceinline__ uint32_t bucket_shift(uint32_t span)
{
    const uint32_t top = span > 1 ? 32u - __clz(span - 1u) : 0u;      // bits of span - 1
    const uint32_t nb_bits = 31u - __clz(NB);
    return top > nb_bits ? top - nb_bits : 0u;
}

// One staged tile through the whole trigger: the n records of `stage` (16
// bytes each, time t_ns, PMT and charge; any order) span [tb, tb + span);
// the core is t - tb in [lo_t, hi_t).
//
//  A. every record becomes a packed key (t - tb) << 12 | pmt and is counted
//     in its time bucket (t - tb) >> bsh; the stage buffer is then handed
//     back to the producer (release_bar), the rest works on the keys;
//  B. bucket offsets (exclusive scan of the counts);
//  C. the k-way merge of the PMT runs ("DAQ system of NEMO Phase II"):
//     keys, charges and floors scattered to their bucket, about one key per
//     bucket.  For the default rule that bucket order is the final order;
//     the builds with the extended rules, row outputs and event extraction
//     (SORT) also rank each key inside its bucket by (t, pmt, charge);
//  D. floor coincidences ("Sorting and triggering in GPU": another PMT of
//     the same floor within tau), in rounds: round r checks the pair
//     (i, i + r) of every key i still live.  Sorted, a key stays live while
//     its next keys lie within tau; in bucket order, while i + r + 1 is
//     before the end of the bucket holding t_i + tau (every key within tau
//     after it in that order).  Every pair is checked once, both hits are
//     marked, and each warp keeps its own list of live keys.  Seed rule 1
//     and level 0 (SORT builds) test each core key instead;
//  E. the ordered seed list; F. the causal count of every seed over whole
//     buckets of its scan range, each key tested exactly ("Muon trigger
//     strategy"); G. the fired seeds, in (t, pmt, charge) order, to out.
//
// Returns the counts and c0 = the number of staged keys before the core.
// cnt and mask are zero on entry and on return.
template <int CAP, int NC, bool SMEM_DT, bool EXT, bool DENSE>
__device__ CoreOut tile_pass(TileCtx<CAP> &cx, const uint64_t *stage, uint32_t n, int64_t tb, uint32_t span,
                             uint32_t lo_t, uint32_t hi_t, const TrigParams &tp, trig_trigger *out, uint32_t *wr,
                             bool out_at_c0, uint32_t rank_base, int64_t dbg_rank_lo, uint64_t *release_bar)
{
    constexpr bool SORT = EXT;
    constexpr uint32_t NW = NC / 32;
    constexpr int PER = CAP / NC;
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    // buckets of the in-tile merge: the finer grid where it pays (the dense
    // builds, whose long causal scans dominate, keep one bucket per slot)
    constexpr uint32_t NB = DENSE ? (uint32_t)CAP : (uint32_t)TileLayout<CAP>::NBK;
    const uint32_t bsh = bucket_shift<NB>(span);
    const uint32_t tau = tp.tau;
    __shared__ uint32_t s_red[NW + 1];
    __shared__ uint32_t s_below[3];
    __shared__ uint32_t s_tot[2 * NW];
    uint32_t *cnt = cx.cnt();
    uint32_t *mask = cx.mask();
#ifdef TRIG_PHASE_STATS
    long long t_ph = clock64();
#define PHASE_MARK(i)                                   \
    do {                                                \
        if (tid == 0) {                                 \
            const long long now_ = clock64();           \
            PHASE_ADD((i), now_ - t_ph);                \
            t_ph = now_;                                \
        }                                               \
    } while (0)
#else
#define PHASE_MARK(i) ((void)0)
#endif

    // A. keys and bucket counts; keys before the core, before its end, and
    //    too early to pair with a core key (t + tau < lo_t)
    uint32_t key[PER], cs[PER];           // packed key; charge << 16 | slot in the bucket
    uint32_t below_lo = 0, below_hi = 0, below_w = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const uint32_t i = tid + r * NC;
        key[r] = kPkNone;
        cs[r] = 0;
        if (i < n) {
            const uint4 v = *reinterpret_cast<const uint4 *>(stage + 2 * i);
            // t - tb in 32 bits (the staged range spans less than 2^20 ns)
            const uint32_t tr = min(v.x - (uint32_t)tb, span - 1u);
            key[r] = (tr << 12) | (v.z & 0xfffu);
            const uint32_t slot = atomicAdd(&cnt[bucket_of<NB>(tr, bsh)], 1u);
            cs[r] = (v.z & 0xffff0000u) | slot;
            below_lo += tr < lo_t;
            below_hi += tr < hi_t;
            below_w += tr + tau < lo_t;
        }
    }
    below_lo = __reduce_add_sync(0xffffffffu, below_lo);
    below_hi = __reduce_add_sync(0xffffffffu, below_hi);
    below_w = __reduce_add_sync(0xffffffffu, below_w);
    if (tid == 0) s_below[0] = s_below[1] = s_below[2] = 0;
    cons_sync<NC>();
    if (lane == 0) {
        if (below_lo) atomicAdd(&s_below[0], below_lo);
        if (below_hi) atomicAdd(&s_below[1], below_hi);
        if (below_w) atomicAdd(&s_below[2], below_w);
    }
    // the stage buffer has been read: order those reads before the
    // producer's next bulk copy into it, then hand it back
    if (release_bar) fence_proxy_async_smem();

    // B. bucket offsets (the scan's barriers also publish s_below and end
    //    every read of the stage buffer)
    cons_exclusive_scan<NC, NB>(cnt, s_red);
    if (release_bar && tid == 0) mbar_arrive(release_bar);
    const uint32_t c0 = s_below[0], c1 = s_below[1], d_lo = s_below[2];
    PHASE_MARK(kPhA);

    // C. bucket order (with each key's floor); SORT: then the rank inside
    //    the bucket
    uint32_t *pk = cx.pk_s();
    uint16_t *chg = cx.chg_s(), *flk = cx.flk();
    uint32_t *pk_c = SORT ? cx.pk_b() : pk;
    uint16_t *chg_c = SORT ? cx.chg_b() : chg;
    const uint16_t *fl = cx.floor_s();
    const bool charge_rule = !(EXT && tp.seed_rule == 1);
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        if (key[r] != kPkNone) {
            const uint32_t tr = key[r] >> 12;
            const uint32_t pos = cnt[bucket_of<NB>(tr, bsh)] + (cs[r] & 0xffffu);
            if (CHECK(22, pos, CAP)) {
                pk_c[pos] = key[r];
                chg_c[pos] = (uint16_t)(cs[r] >> 16);
                if (!SORT) {
                    flk[pos] = fl[key[r] & 0xfffu];
                    if (charge_rule && (cs[r] >> 16) >= tp.q_seed && tr >= lo_t && tr < hi_t)
                        atomicOr(&mask[pos >> 5], 1u << (pos & 31u));
                }
            }
        }
    }
    if (tid < 4) pk[n + tid] = 0xfffff000u;           // end keys (time 2^20 - 1, PMT 0)
    cons_sync<NC>();
    PHASE_MARK(kPhB);
    if (SORT) {
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const uint32_t k = key[r];
            if (k == kPkNone) continue;
            const uint32_t b = bucket_of<NB>(k >> 12, bsh);
            const uint32_t s0 = cnt[b], s1 = cnt[b + 1], q = cs[r] >> 16, pos = s0 + (cs[r] & 0xffffu);
            uint32_t rk = s0;
            for (uint32_t m = s0; m < s1; ++m) {
                const uint32_t o = pk_c[m];
                rk += o < k;
                if (o == k) {                      // equal time and PMT: charge, then position
                    const uint32_t oq = chg_c[m];
                    rk += oq < q || (oq == q && m < pos);
                }
            }
            if (CHECK(23, rk, CAP)) {
                pk[rk] = k;
                chg[rk] = (uint16_t)q;
                flk[rk] = fl[k & 0xfffu];
                const uint32_t tr = k >> 12;
                if (charge_rule && q >= tp.q_seed && tr >= lo_t && tr < hi_t)
                    atomicOr(&mask[rk >> 5], 1u << (rk & 31u));
            }
        }
        cons_sync<NC>();
    }
    PHASE_MARK(kPhC);

    // D. seed flags of the core keys
    const uint32_t P = cx.P;
    if (EXT && tp.seed_rule == 1) {
        for (uint32_t base = c0 & ~31u; base < c1; base += NC) {
            const uint32_t i = base + tid;
            const bool seed = i >= c0 && i < c1 && coincidence_seed(pk, n, i, tp.rel, P, tp.sc_w, tp.fc_w, tp.afc_w);
            const uint32_t m = __ballot_sync(0xffffffffu, seed);
            if (lane == 0 && m) atomicOr(&mask[(base >> 5) + warp], m);
        }
    } else {
        // the keys that can pair with a core key -- sorted: [d_lo, c1); in
        // bucket order: the buckets from t = lo_t - tau to hi_t + tau - 1 --
        // in contiguous shares per warp; a live entry is (end << 16) | i
        // with end the first position past i's candidates
        const uint32_t lt = (1u << lane) - 1u;
        const uint32_t r_lo = SORT ? d_lo : cnt[bucket_of<NB>(lo_t > tau ? lo_t - tau : 0u, bsh)];
        const uint32_t r_hi = SORT ? c1 : cnt[bucket_of<NB>(hi_t + tau - 1u, bsh) + 1];
        const uint32_t d_n = r_hi > r_lo ? r_hi - r_lo : 0u;
        const uint32_t share = ((d_n + NW - 1) / NW + 31u) & ~31u;
        const uint32_t w_begin = min(r_lo + warp * share, r_hi), w_end = min(w_begin + share, r_hi);
        uint32_t *live = cx.pk_b() + warp * (CAP / NW);
        auto core = [&](uint32_t i, uint32_t ti) { return SORT ? (i >= c0 && i < c1) : (ti >= lo_t && ti < hi_t); };
        auto pair = [&](uint32_t i, uint32_t j, uint32_t ki, uint32_t kj) {
            const uint32_t ti = ki >> 12, tj = kj >> 12;
            if ((SORT || (tj > ti ? tj - ti : ti - tj) <= tau) && (ki & 0xfffu) != (kj & 0xfffu) && flk[i] == flk[j]) {
                if (core(i, ti)) atomicOr(&mask[i >> 5], 1u << (i & 31u));
                if (core(j, tj)) atomicOr(&mask[j >> 5], 1u << (j & 31u));
            }
        };
        uint32_t nlive = 0;
        for (uint32_t x = w_begin; x < w_end; x += 32) {
            const uint32_t i = x + lane;
            bool alive = false;
            uint32_t end = 0;
            if (i < w_end) {
                const uint32_t ki = pk[i], ti = ki >> 12;
                if (SORT) {
                    // i + 1 <= c1 <= n: an end key at worst
                    const uint32_t kj = pk[i + 1];
                    if ((kj >> 12) - ti <= tau && i + 1 < n) {
                        alive = true;
                        pair(i, i + 1, ki, kj);
                    }
                } else if (ti + tau >= lo_t && ti < hi_t + tau) {
                    // the first kFloorPairs candidates inline (most keys
                    // have no more), the rest in the rounds below
                    end = cnt[bucket_of<NB>(ti + tau, bsh) + 1];
#pragma unroll
                    for (uint32_t r = 1; r <= kFloorPairs; ++r)
                        if (i + r < end) pair(i, i + r, ki, pk[i + r]);
                    alive = i + kFloorPairs + 1 < end;
                }
            }
            const uint32_t m = __ballot_sync(0xffffffffu, alive);
            if (alive) live[nlive + __popc(m & lt)] = (end << 16) | i;
            nlive += __popc(m);
        }
        for (uint32_t d = SORT ? 2u : kFloorPairs + 1; nlive; ++d) {
            uint32_t next = 0;
            for (uint32_t x = 0; x < nlive; x += 32) {
                bool alive = false;
                uint32_t e = 0;
                if (x + lane < nlive) {
                    e = live[x + lane];
                    const uint32_t i = e & 0xffffu, j = i + d;
                    if (SORT) {
                        if (j < n) {
                            const uint32_t ki = pk[i], kj = pk[j];
                            if ((kj >> 12) - (ki >> 12) <= tau) {
                                alive = true;
                                pair(i, j, ki, kj);
                            }
                        }
                    } else {
                        pair(i, j, pk[i], pk[j]);           // j < end by the list
                        alive = j + 1 < (e >> 16);
                    }
                }
                // the ballot orders this batch's reads of the list before
                // the writes below (which land at or before x + 31)
                const uint32_t m = __ballot_sync(0xffffffffu, alive);
                if (alive) live[next + __popc(m & lt)] = e;
                next += __popc(m);
            }
            nlive = next;
        }
    }
    cons_sync<NC>();
    if (EXT && tp.l0_hits) {
        // level 0 (N hits within TW) before the seed triggers count
        if (tp.l0_distinct && P > 128) {
            // a warp per seed, its PMT set in the bucket-order key region
            // (free between the floor coincidences and the seed list)
            static_assert(NC / 32 * 128 <= CAP, "a 4096-bit PMT set per consumer warp");
            uint32_t *set = cx.pk_b() + warp * 128;
            for (uint32_t base = (c0 & ~31u) + warp * 32; base < c1; base += NC) {
                const uint32_t i = base + lane;
                const uint32_t w = (i >= c0 && i < c1) ? mask[i >> 5] : 0u;
                uint32_t cand = __ballot_sync(0xffffffffu, (w >> (i & 31u)) & 1u);
                uint32_t drop = 0;
                while (cand) {
                    const uint32_t b = __ffs(cand) - 1;
                    cand &= cand - 1;
                    if (!level0_distinct_warp(pk, n, base + b, tp.l0_hits, tp.l0_window, P, set)) drop |= 1u << b;
                }
                if (lane == 0 && drop) atomicAnd(&mask[base >> 5], ~drop);
            }
        } else {
            for (uint32_t base = c0 & ~31u; base < c1; base += NC) {
                const uint32_t i = base + tid;
                const uint32_t w = (i >= c0 && i < c1) ? mask[i >> 5] : 0u;
                const bool drop = ((w >> (i & 31u)) & 1u) &&
                                  !level0_pass(pk, n, i, tp.l0_hits, tp.l0_window, tp.l0_distinct != 0);
                const uint32_t m = __ballot_sync(0xffffffffu, drop);
                if (lane == 0 && m) atomicAnd(&mask[(base >> 5) + warp], ~m);
            }
        }
        cons_sync<NC>();
    }
    PHASE_MARK(kPhD);

    // E. ordered seed list: thread x takes mask word w_lo + x (at most
    //    CAP / 32 <= NC words); each word's offset adds the totals of the
    //    warps before it.  Marks lie in the core: sorted, positions
    //    [c0, c1); in bucket order, the buckets of [lo_t, hi_t)
    uint16_t *seed_idx = SORT ? cx.seed_idx() : cx.flk();
    const uint32_t p_lo = SORT ? c0 : cnt[bucket_of<NB>(lo_t, bsh)];
    const uint32_t p_hi = SORT ? c1 : cnt[bucket_of<NB>(hi_t > 0 ? hi_t - 1 : 0, bsh) + 1];
    const uint32_t w_lo = p_lo >> 5, w_hi = (p_hi + 31) >> 5;
    const uint32_t nwords = w_hi - w_lo;
    const uint32_t nw_used = (nwords + 31) >> 5;
    uint32_t *wtot = s_tot;                               // [NW]
    uint32_t ns = 0;
    {
        const uint32_t m = tid < nwords ? mask[w_lo + tid] : 0u;
        const uint32_t c = __popc(m);
        const uint32_t incl = warp < nw_used ? warp_incl_scan(c) : 0u;
        if (warp < nw_used && lane == 31) wtot[warp] = incl;
        cons_sync<NC>();
        uint32_t before = 0;
        for (uint32_t w2 = 0; w2 < nw_used; ++w2) {
            const uint32_t v = wtot[w2];
            before += w2 < warp ? v : 0u;
            ns += v;
        }
        uint32_t at = before + incl - c;
        uint32_t mm = m;
        while (mm) {
            const uint32_t bit = __ffs(mm) - 1;
            mm &= mm - 1;
            if (CHECK(2, at, CAP)) seed_idx[at] = (uint16_t)((w_lo + tid) * 32 + bit);
            ++at;
        }
    }
    cons_sync<NC>();
    PHASE_MARK(kPhE);
    if (tid == 0) PHASE_ADD(kPhSeeds, ns);

    // F. causal count c(s) over each seed's scan range (sparse batches give
    //    each seed 4 lanes, dense ones a warp), or its distinct-PMT form
    // (in bucket order the seed list sits in the floor array, so the
    // counts take the second half of the bucket-order key region)
    uint16_t *seed_cnt = cx.seed_cnt();
    if (EXT && tp.count_distinct) {
        count_distinct_pmts<CAP, NC, SMEM_DT, NB>(cx, pk, n, ns, seed_idx, bsh, seed_cnt);
    } else {
        count_causal<CAP, NC, SMEM_DT, DENSE ? 5u : 2u, NB>(cx, pk, n, ns, seed_idx, bsh, seed_cnt);
    }
    cons_sync<NC>();
    PHASE_MARK(kPhF);
    auto count_of = [&](uint32_t k) -> uint32_t { return seed_cnt[k]; };

    // G. emit the fired seeds in order: warp w takes a contiguous range of
    //    the seed list and adds up the fired totals of the warps before it.
    //    In bucket order a fired seed's rank also counts the fired seeds of
    //    its bucket (adjacent in the list) with a smaller (t, pmt, charge).
    const uint32_t threshold = tp.threshold;
    const uint32_t per_w = (ns + NW - 1) / NW;
    const uint32_t k_begin = min(ns, warp * per_w), k_end = min(ns, k_begin + per_w);
    uint32_t my_f = 0;
    for (uint32_t k0 = k_begin; k0 < k_end; k0 += 32) {
        const uint32_t k = k0 + lane;
        my_f += __popc(__ballot_sync(0xffffffffu, k < k_end && count_of(k) >= threshold));
    }
    uint32_t *ftot = s_tot + NW;                          // [NW]: fired per warp, then their prefix
    if (lane == 0) ftot[warp] = my_f;
    cons_sync<NC>();
    if (warp == 0) {
        const uint32_t v = lane < NW ? ftot[lane] : 0u;
        const uint32_t vi = warp_incl_scan(v);
        if (lane < NW) ftot[lane] = vi - v;
        if (lane == NW - 1) s_red[0] = vi;
    }
    cons_sync<NC>();
    const uint32_t n_fired = s_red[0];
    uint32_t F = ftot[warp];
    trig_trigger *dst = out + (out_at_c0 ? c0 : 0u);
    for (uint32_t k0 = k_begin; k0 < k_end; k0 += 32) {
        const uint32_t k = k0 + lane;
        const uint32_t cnt_k = k < k_end ? count_of(k) : 0u;
        const bool fired = k < k_end && cnt_k >= threshold;
        const uint32_t m = __ballot_sync(0xffffffffu, fired);
        if (fired) {
            const uint32_t i = seed_idx[k];
            const uint32_t ks = pk[i];
            const uint32_t q = chg[i];
            uint32_t o_ = F + __popc(m & ((1u << lane) - 1u));
            if (!SORT) {
                // fired seeds of the same bucket before k that order after
                // it, and after k that order before it
                const uint32_t bk = bucket_of<NB>(ks >> 12, bsh);
                const uint64_t key_k = ((uint64_t)ks << 16) | q;
                for (uint32_t k2 = k; k2-- > 0;) {
                    const uint32_t i2 = seed_idx[k2];
                    if (bucket_of<NB>(pk[i2] >> 12, bsh) != bk) break;
                    if (count_of(k2) >= threshold && (((uint64_t)pk[i2] << 16) | chg[i2]) > key_k) --o_;
                }
                for (uint32_t k2 = k + 1; k2 < ns; ++k2) {
                    const uint32_t i2 = seed_idx[k2];
                    if (bucket_of<NB>(pk[i2] >> 12, bsh) != bk) break;
                    if (count_of(k2) >= threshold && (((uint64_t)pk[i2] << 16) | chg[i2]) < key_k) ++o_;
                }
            }
            trig_trigger tr;
            tr.t_ns = tb + (int64_t)(ks >> 12);
            tr.pmt = (uint16_t)(ks & 0xfffu);
            tr.charge = (uint16_t)q;
            tr.count = cnt_k;
            if (CHECK(3, o_, c1 - c0)) {
                dst[o_] = tr;
                // the merged ranks of the first hit of the seed's event
                // window [t - h, t + h] and of the first hit past it, where
                // that bound lies in the staged range (else kRankUnknown:
                // the window pass searches for it)
                const uint32_t ts = ks >> 12, wh = tp.win_half;
                const uint32_t r_lo = ts >= wh ? rank_base + keys_before<NB>(pk, cnt, n, ts - wh, bsh, span)
                                               : kRankUnknown;
                const uint32_t r_hi = ts + wh + 1u <= span
                                          ? rank_base + keys_before<NB>(pk, cnt, n, ts + wh + 1u, bsh, span)
                                          : kRankUnknown;
                *reinterpret_cast<uint2 *>(wr + 2 * ((out_at_c0 ? c0 : 0u) + o_)) = make_uint2(r_lo, r_hi);
            }
        }
        F += __popc(m);
    }
    // optional row outputs (SORT builds): the merged core rows
    // (verification, and the merged stream of event extraction) and each
    // row's causal count (verification only); rows are indexed by merged
    // rank minus the rank of the slice's first owned hit
    if (SORT && tp.dbg_merged) {
        const uint64_t dbg_base = (uint64_t)(dbg_rank_lo + (int64_t)c0);
        for (uint32_t i = tid; i < c1 - c0; i += NC) {
            const uint32_t k = pk[c0 + i];
            trig_hit h;
            h.t_ns = tb + (int64_t)(k >> 12);
            h.pmt = (uint16_t)(k & 0xfffu);
            h.charge = chg[c0 + i];
            h.reserved = 0;
            tp.dbg_merged[dbg_base + i] = h;
            if (tp.dbg_seedcnt) tp.dbg_seedcnt[dbg_base + i] = 0xffffffffu;
        }
        if (tp.dbg_seedcnt) {
            cons_sync<NC>();
            for (uint32_t k = tid; k < ns; k += NC) tp.dbg_seedcnt[dbg_base + (seed_idx[k] - c0)] = seed_cnt[k];
        }
    }
    // leave the bucket counts and the seed mask zero for the next tile
    // (after every warp's last read of the offsets: the window ranks above)
    cons_sync<NC>();
    for (uint32_t i = tid; i < NB; i += NC) cnt[i] = 0;
    for (uint32_t w = w_lo + tid; w < w_hi; w += NC) mask[w] = 0;
    cons_sync<NC>();
    PHASE_MARK(kPhG);
#undef PHASE_MARK
    CoreOut co;
    co.n_fired = n_fired;
    co.n_seeds = ns;
    co.c0 = c0;
    return co;
}

// Overflow path: the tile holds more than CAP hits with its halo.  Split
// Overflow path: the tile holds more than CAP hits with its halo.  Split
// its core in halves until each piece fits; pieces are staged with plain
// loads after per-PMT binary searches.  A 1 ns core that still does not
// fit is reported (TRIG_FLAG_TILE_FULL) and skipped.
template <int CAP, int NC, bool SMEM_DT, bool EXT, bool DENSE>
__device__ void tile_overflow(TileCtx<CAP> &cx, uint64_t *buf, const SliceDesc &d, const TrigParams &tp, uint32_t g,
                              uint32_t *red, int64_t *stk)
{
    constexpr uint32_t NW = NC / 32;
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const uint32_t P = d.n_pmt, H = d.halo;
    const int64_t W = d.tile_w;
    const int64_t Bg = d.t0 + (int64_t)g * W;
    const int64_t core_end = min(Bg + W, d.t0 + d.slice_ns);
    uint64_t *part = reinterpret_cast<uint64_t *>(red + 8);          // [NW]
    uint64_t *part2 = reinterpret_cast<uint64_t *>(red + 8 + 2 * NW);  // [NW]
    // merged rank of the tile's first core hit
    uint64_t rk = 0;
    for (uint32_t p = tid; p < P; p += NC) {
        uint64_t sp = d.pmt_off[p], ep = d.pmt_off[p + 1];
        rk += lb_time(d.hits, sp, ep, Bg) - sp;
    }
    rk = warp_sum_u64(rk);
    if (lane == 0) part[warp] = rk;
    cons_sync<NC>();
    if (tid == 0) {
        uint64_t tot = 0;
        for (uint32_t w = 0; w < NW; ++w) tot += part[w];
        red[4] = (uint32_t)tot;     // tile rank
        red[5] = 0;                 // fired so far
        red[6] = 0;                 // seeds so far
        stk[0] = Bg;
        stk[1] = core_end;
        red[7] = 1;                 // stack depth
    }
    cons_sync<NC>();
    const uint32_t tile_rank = red[4];
    for (int guard = 0; guard < 1 << 20; ++guard) {
        uint32_t depth = red[7];
        if (depth == 0) break;
        const int64_t lo = stk[2 * (depth - 1)], hi = stk[2 * (depth - 1) + 1];
        cons_sync<NC>();
        // extended count and rank of the piece
        uint64_t tot = 0, rlo = 0;
        for (uint32_t p = tid; p < P; p += NC) {
            uint64_t sp = d.pmt_off[p], ep = d.pmt_off[p + 1];
            uint64_t a = lb_time(d.hits, sp, ep, lo - (int64_t)H);
            uint64_t b = lb_time(d.hits, a, ep, hi + (int64_t)H);
            tot += b - a;
            rlo += a - sp;
        }
        tot = warp_sum_u64(tot);
        rlo = warp_sum_u64(rlo);
        if (lane == 0) {
            part[warp] = tot;
            part2[warp] = rlo;
        }
        cons_sync<NC>();
        if (tid == 0) {
            uint64_t T = 0, R = 0;
            for (uint32_t w = 0; w < NW; ++w) {
                T += part[w];
                R += part2[w];
            }
            red[2] = T > 0xffffffffull ? 0xffffffffu : (uint32_t)T;
            red[3] = (uint32_t)R;
            red[7] = depth - 1;                      // pop
            if (T > (uint64_t)CAP) {
                if (hi - lo > 1 && depth + 1 < 64) {
                    int64_t mid = lo + (hi - lo) / 2;
                    stk[2 * (depth - 1)] = mid;          // right half below ...
                    stk[2 * (depth - 1) + 1] = hi;
                    stk[2 * depth] = lo;                 // ... left half on top
                    stk[2 * depth + 1] = mid;
                    red[7] = depth + 1;
                } else {
                    report(d, TRIG_FLAG_TILE_FULL);
                }
            }
        }
        cons_sync<NC>();
        const uint32_t total = red[2];
        if (total > (uint32_t)CAP) continue;         // split (or skipped)
        const uint32_t rank_lo = red[3];
        // stage the piece: PMTs in order, warps take groups of 32 PMTs
        uint32_t dst = 0;
        for (uint32_t p0 = 0; p0 < P; p0 += 32) {
            uint32_t p = p0 + lane;
            uint64_t a = 0, len = 0;
            if (p < P) {
                uint64_t sp = d.pmt_off[p], ep = d.pmt_off[p + 1];
                a = lb_time(d.hits, sp, ep, lo - (int64_t)H);
                len = lb_time(d.hits, a, ep, hi + (int64_t)H) - a;
            }
            uint32_t incl = warp_incl_scan((uint32_t)len);
            uint32_t my = dst + incl - (uint32_t)len;
            if (((p0 >> 5) % NW) == warp) {
                for (uint32_t q = 0; q < 32; ++q) {
                    uint64_t qa = __shfl_sync(0xffffffffu, a, q);
                    uint32_t ql = __shfl_sync(0xffffffffu, (uint32_t)len, q);
                    uint32_t qd = __shfl_sync(0xffffffffu, my, q);
                    for (uint32_t e = lane; e < ql; e += 32) {
                        trig_hit h = load_hit(d.hits + qa + e);
                        if (!CHECK(4, qd + e, CAP) || !CHECK(5, qa + e, d.n_hits)) continue;
                        buf[2 * (qd + e)] = (uint64_t)h.t_ns;
                        buf[2 * (qd + e) + 1] = (uint64_t)h.pmt | ((uint64_t)h.charge << 16);
                    }
                }
            }
            dst += __shfl_sync(0xffffffffu, incl, 31);
        }
        cons_sync<NC>();
        const int64_t tb = lo - (int64_t)H;
        const uint32_t span = (uint32_t)(hi - lo) + 2 * H;
        const uint32_t fired0 = red[5];
        CoreOut co = tile_pass<CAP, NC, SMEM_DT, EXT, DENSE>(cx, buf, total, tb, span, H, H + (uint32_t)(hi - lo), tp,
                                                             d.stage + tile_rank + fired0,
                                                             d.wrank + 2 * (size_t)(tile_rank + fired0), false,
                                                             rank_lo, (int64_t)rank_lo - (int64_t)d.dbg_rank0,
                                                             nullptr);
        if (tid == 0) {
            red[5] = fired0 + co.n_fired;
            red[6] += co.n_seeds;
        }
        cons_sync<NC>();
    }
    if (tid == 0) {
        d.tile_nfired[g] = red[5];
        d.tile_rank[g] = tile_rank;
        atomicAdd(reinterpret_cast<unsigned long long *>(&d.stats->n_seeds), (unsigned long long)red[6]);
    }
    cons_sync<NC>();
}

template <int CAP, int NC, bool SMEM_DT, bool EXT, bool DENSE>
__global__ void __launch_bounds__(NC + 32, (CAP <= 1024 ? 4 : CAP <= 2048 ? 2 : 1)) k_tile(BatchHeader *__restrict__ hdr,
                                                                          const SliceDesc *__restrict__ desc,
                                                                          uint32_t max_pmt)
{
    constexpr uint32_t NW = NC / 32;
    constexpr uint32_t NSTG = TileLayout<CAP>::NS;
    __shared__ uint64_t full_bar[2], empty_bar[2];
    __shared__ ItemInfo info[2];
    __shared__ __align__(16) uint32_t red[64 + 64];
    __shared__ int64_t stk[128];

    TileCtx<CAP> cx;
    cx.pp = (max_pmt + 7) & ~7u;
    cx.dt_g = nullptr;
    cx.P = 0;

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    if (tid == 0) {
        mbar_init(&full_bar[0], 1);
        mbar_init(&full_bar[1], 1);
        mbar_init(&empty_bar[0], 1);
        mbar_init(&empty_bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const uint32_t n_slices = hdr->n_slices, n_items = hdr->n_items;
    const uint64_t wait_ns = hdr->wait_ns;

    if (warp == NW) {
        // test control: stage nothing, so that the consumers' first wait
        // runs out (no copy is ever in flight)
        if (hdr->stall) return;
        // ------------------------------------------------ producer warp
        // The next item is dequeued and its per-PMT runs looked up before
        // waiting for a free buffer, so those global loads overlap the wait.
        uint32_t s = 0;
        bool bad = false;
        const SliceDesc *d = nullptr;
        constexpr int R = 4;                       // PMTs per lane kept in registers
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(&hdr->queue, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        for (uint32_t it = 0;; ++it) {
            const uint32_t b = it % NSTG, use = it / NSTG;
#ifdef TRIG_PHASE_STATS
            const long long tp0 = clock64();
#endif
            uint32_t g = 0, P = 0, mode = 2, lo_t = 0, span = 0;
            uint64_t ra[R];
            uint32_t rl[R];
            uint64_t tot = 0, rlo = 0;
            bool wide = false;
            if (item < n_items) {
                // items arrive in increasing order: walk the slice index forward
                if (d == nullptr || item < d->item0) s = find_slice_by_item(desc, n_slices, item), d = nullptr;
                while (s + 1 < n_slices && desc[s + 1].item0 <= item) ++s, d = nullptr;
                if (d == nullptr) {
                    d = &desc[s];
                    bad = (d->stats->flags & (TRIG_FLAG_BAD_PMT | TRIG_FLAG_UNSORTED | TRIG_FLAG_OUT_OF_RANGE)) != 0;
                }
                g = item - d->item0;
                P = d->n_pmt;
                wide = d->wide != 0;
                if (wide) {
                    // one contiguous range of the bucketed copy: the core
                    // buckets and hh buckets of halo on each side
                    const uint32_t hh = d->bkt_halo, m = d->bkt_per_tile;
                    const uint32_t c_lo = d->bkt_lead + g * m;
                    const uint32_t b_lo = c_lo > hh ? c_lo - hh : 0u;
                    const uint32_t b_hi = min(c_lo + m + hh, d->n_bkt);
                    lo_t = (c_lo - b_lo) * d->bkt_w;
                    span = (b_hi - b_lo) * d->bkt_w;
                    if (!bad) {
                        rlo = __ldg(d->bkt_off + b_lo);
                        tot = __ldg(d->bkt_off + b_hi) - rlo;
                    }
                } else {
                    // the PMTs' runs [lb(B_g - H), lb(B_{g+1} + H)), P <= 32 R
                    const uint32_t *elo = d->e_lo + (size_t)g * P;
                    const uint32_t *ehi = d->e_hi + (size_t)g * P;
                    const uint64_t *poff = d->pmt_off;
                    lo_t = d->halo;
                    span = (uint32_t)d->tile_w + 2u * d->halo;
                    if (!bad) {
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            const uint32_t p = r * 32 + lane;
                            uint64_t a = 0, e = 0, sp_ = 0, ep_ = 0;
                            if (p < P) {
                                a = __ldg(elo + p);
                                e = __ldg(ehi + p);
                                sp_ = __ldg(poff + p);
                                ep_ = __ldg(poff + p + 1);
                                a = min(max(a, sp_), ep_);
                                e = min(max(e, a), ep_);
                            }
                            ra[r] = a;
                            rl[r] = (uint32_t)(e - a);
                            tot += e - a;
                            rlo += a - sp_;
                        }
                    }
                    tot = warp_sum_u64(tot);
                    rlo = warp_sum_u64(rlo);
                }
                mode = bad ? 2u : (tot > (uint64_t)CAP ? 1u : (tot == 0 ? 2u : 0u));
            }
            uint32_t next = 0;
            if (item < n_items) {
                if (lane == 0) next = atomicAdd(&hdr->queue, 1u);
                next = __shfl_sync(0xffffffffu, next, 0);
            }
            // lane 0 waits (bounded) for the buffer and decides for the warp
#ifdef TRIG_PHASE_STATS
            const long long tw0 = clock64();
            if (lane == 0) PHASE_ADD(kPhProdItem, tw0 - tp0);
#endif
            uint32_t free_ok = 1;
            if (it >= NSTG && lane == 0) {
#ifdef TRIG_PHASE_STATS
                uint32_t pr = 0;
                free_ok = mbar_wait(&empty_bar[b], (use - 1) & 1u, wait_ns, &pr) ? 1u : 0u;
                PHASE_ADD(kPhProdWait, clock64() - tw0);
                PHASE_ADD(kPhProdWaitRounds, pr);
#else
                free_ok = mbar_wait(&empty_bar[b], (use - 1) & 1u, wait_ns) ? 1u : 0u;
#endif
            }
            free_ok = __shfl_sync(0xffffffffu, free_ok, 0);
            __syncwarp();
            if (!free_ok) {
                if (lane == 0) atomicOr(&hdr->err, TRIG_FLAG_TIMEOUT);
                break;
            }
            if (item >= n_items) {
                if (lane == 0) {
                    info[b].item = -1;
                    mbar_arrive(&full_bar[b]);
                }
                break;
            }
            if (lane == 0) {
                info[b].item = (int32_t)item;
                info[b].slice = s;
                info[b].g = g;
                info[b].n = (uint32_t)min(tot, (uint64_t)CAP);
                info[b].rank_lo = (uint32_t)rlo;
                info[b].mode = mode;
                info[b].lo_t = lo_t;
                info[b].span = span;
                if (mode == 0) mbar_arrive_expect_tx(&full_bar[b], (uint32_t)tot * 16u);
                else mbar_arrive(&full_bar[b]);
            }
            __syncwarp();
            if (mode == 0 && wide) {
                if (lane == 0 && CHECK(7, rlo + tot, d->n_hits + 1))
                    bulk_g2s(cx.stage(b), d->tbuf + rlo, (uint32_t)tot * 16u, &full_bar[b]);
            } else if (mode == 0) {
                uint32_t dst = 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t len = rl[r];
                    const uint64_t a = ra[r];
                    const uint32_t incl = warp_incl_scan(len);
                    if (len && CHECK(6, dst + incl, CAP + 1) && CHECK(7, a + len, d->n_hits + 1))
                        bulk_g2s(cx.stage(b) + 2 * (size_t)(dst + incl - len), d->hits + a, len * 16u, &full_bar[b]);
                    dst += __shfl_sync(0xffffffffu, incl, 31);
                }
            }
#ifdef TRIG_PHASE_STATS
            if (lane == 0) PHASE_ADD(kPhProdTotal, clock64() - tp0);
#endif
            item = next;
        }
        return;
    }

    // ---------------------------------------------------- consumer warps
    // the tile pass expects zero bucket counts and seed mask (and leaves them so)
    for (uint32_t i = tid; i < (uint32_t)TileLayout<CAP>::NBK; i += NC) cx.cnt()[i] = 0;
    for (uint32_t i = tid; i < (uint32_t)CAP / 32; i += NC) cx.mask()[i] = 0;
    cons_sync<NC>();
    const SliceDesc *loaded = nullptr;
    // the slice's trigger parameters live in shared memory (written by one
    // thread when the slice changes), keeping registers for the tile phases
    __shared__ TrigParams tp;
    // the loaded slice's tile width, t0, length and merged rank of its first
    // owned hit, also kept in shared memory
    __shared__ int64_t sl[4];
    for (uint32_t it = 0;; ++it) {
        const uint32_t b = it % NSTG, use = it / NSTG;
        // every thread waits (bounded) for the staged tile; the barrier
        // ANDs their results, so the block never splits on a timeout
#ifdef TRIG_PHASE_STATS
        const long long tw0 = clock64();
        uint32_t cr = 0;
        const bool cwait_ok = mbar_wait(&full_bar[b], use & 1u, wait_ns, &cr);
        if (tid == 0) {
            PHASE_ADD(kPhConsWait, clock64() - tw0);
            PHASE_ADD(kPhConsWaitRounds, cr);
            PHASE_ADD(kPhTiles, 1);
        }
#else
        const bool cwait_ok = mbar_wait(&full_bar[b], use & 1u, wait_ns);
#endif
        if (!named_sync_and(kBarCons, NC, cwait_ok)) {
            if (tid == 0) atomicOr(&hdr->err, TRIG_FLAG_TIMEOUT);
            break;
        }
        const ItemInfo &inf = info[b];      // stable until this buffer is released
        if (inf.item < 0) break;
        const SliceDesc &d = desc[inf.slice];
        if (&d != loaded) {
            // (re)load the detector tables of this slice
            cons_sync<NC>();
            const uint32_t P = d.n_pmt;
            for (uint32_t p = tid; p < P; p += NC) {
                cx.floor_s()[p] = d.floor[p];
                cx.dmax_s()[p] = d.dmax_row[p];
            }
            if (SMEM_DT && P <= kSmemDtMaxPmt)
                for (uint32_t i = tid; i < P * P; i += NC) cx.dt_s()[i] = d.dt[i];
            cx.dt_g = d.dt;
            cx.P = P;
            loaded = &d;
            if (tid == 0) {
                tp.H = d.halo;
                tp.win_half = d.win_half;
                tp.tau = d.tau;
                tp.q_seed = d.q_seed;
                tp.threshold = d.threshold;
                tp.l0_hits = d.l0_hits;
                tp.l0_window = d.l0_window;
                tp.l0_distinct = d.l0_distinct;
                tp.seed_rule = d.seed_rule;
                tp.sc_w = d.sc_w;
                tp.fc_w = d.fc_w;
                tp.afc_w = d.afc_w;
                tp.count_distinct = d.count_distinct;
                tp.rel = d.rel;
                tp.dbg_merged = d.dbg_merged;
                tp.dbg_seedcnt = d.dbg_seedcnt;
            }
            if (tid == 0) {
                sl[0] = d.tile_w;
                sl[1] = d.t0;
                sl[2] = d.slice_ns;
                sl[3] = (int64_t)d.dbg_rank0;
            }
            cons_sync<NC>();
        }
        if (inf.mode == 2) {
            if (tid == 0) {
                d.tile_nfired[inf.g] = 0;
                d.tile_rank[inf.g] = 0;
            }
        } else if (inf.mode == 1) {
            tile_overflow<CAP, NC, SMEM_DT, EXT, DENSE>(cx, cx.stage(b), d, tp, inf.g, red, stk);
        } else {
            const int64_t W = sl[0];
            const uint32_t g = inf.g, n_st = inf.n, rank_lo = inf.rank_lo, span = inf.span;
            const int64_t Bg = sl[1] + (int64_t)g * W;
            const int64_t core_end = min(Bg + W, sl[1] + sl[2]);
            // the staged range starts lo_t (>= H) before the core
            const uint32_t lo_t = inf.lo_t;
            const int64_t tb = Bg - (int64_t)lo_t;
            const uint32_t hi_t = lo_t + (uint32_t)(core_end - Bg);
            // the pass hands the buffer back as soon as it has read it (inf
            // is not read after that); the core's first hit has merged rank
            // rank_lo + c0
            CoreOut co = tile_pass<CAP, NC, SMEM_DT, EXT, DENSE>(cx, cx.stage(b), n_st, tb, span, lo_t, hi_t, tp,
                                                                 d.stage + rank_lo, d.wrank + 2 * (size_t)rank_lo,
                                                                 true, rank_lo, (int64_t)rank_lo - sl[3],
                                                                 &empty_bar[b]);
            const uint32_t tile_rank = rank_lo + co.c0;
            if (tid == 0 && CHECK(14, (uint64_t)tile_rank + co.n_fired, d.n_hits + 1) && CHECK(15, g, d.n_tiles)) {
                d.tile_nfired[g] = co.n_fired;
                d.tile_rank[g] = tile_rank;
                atomicAdd(reinterpret_cast<unsigned long long *>(&d.stats->n_seeds), (unsigned long long)co.n_seeds);
            }
            continue;
        }
        // release the buffer to the producer: order our generic-proxy
        // accesses before its next bulk copy into the same buffer
        fence_proxy_async_smem();
        cons_sync<NC>();
        if (tid == 0) mbar_arrive(&empty_bar[b]);
    }
}

// ------------------------------------------------------------------ k_scan

// Block-wide exclusive scan of vals[0..n) into out[0..n); returns the total.
__device__ unsigned long long block_scan_u32(const uint32_t *vals, uint32_t *out, uint32_t n, uint32_t *wsum,
                                             unsigned long long *carry)
{
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) *carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < n; base += blockDim.x) {
        uint32_t g = base + tid;
        uint32_t v = g < n ? vals[g] : 0u;
        uint32_t incl = warp_incl_scan(v);
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = lane < nw ? wsum[lane] : 0u;
            uint32_t wi = warp_incl_scan(w);
            wsum[lane] = wi - w;
        }
        __syncthreads();
        unsigned long long c = *carry;
        if (g < n) out[g] = (uint32_t)(c + wsum[warp] + incl - v);
        __syncthreads();
        if (tid == blockDim.x - 1) *carry = c + wsum[warp] + incl;
        __syncthreads();
    }
    return *carry;
}

__global__ void __launch_bounds__(1024) k_scan(const BatchHeader *__restrict__ hdr, const SliceDesc *__restrict__ desc)
{
    if (hdr->err) return;           // the tile pass gave up: its per-tile outputs are not valid
    __shared__ uint32_t wsum[32];
    __shared__ unsigned long long carry;
    for (uint32_t s = blockIdx.x; s < hdr->n_slices; s += gridDim.x) {
        const SliceDesc &d = desc[s];
        unsigned long long F = block_scan_u32(d.tile_nfired, d.tile_out, d.n_tiles, wsum, &carry);
        if (threadIdx.x == 0) {
            d.stats->n_triggers = F;
            if (F > d.trig_cap) atomicOr(&d.stats->flags, TRIG_FLAG_TRIG_FULL);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ k_copy

// One warp per tile: copy its fired seeds into the dense trigger list and
// count the window heads among them.  A trigger starts a new window unless
// it lies within 2h + 1 ns of the previous trigger of the slice (windows
// [t - h, t + h] merge while lo_next <= hi_cur + 1).
__device__ __forceinline__ uint32_t find_tile_of_pos(const uint32_t *tile_out, uint32_t ng, uint32_t pos)
{
    // last tile g with tile_out[g] <= pos
    uint32_t lo = 0, hi = ng;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (tile_out[mid] <= pos) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_copy(const BatchHeader *__restrict__ hdr, const SliceDesc *__restrict__ desc)
{
    if (hdr->err) return;           // the tile pass gave up: its per-tile outputs are not valid
    const uint32_t n_items = hdr->n_items, n_slices = hdr->n_slices;
    const uint32_t lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t item = gw; item < n_items; item += nw) {
        const uint32_t s = find_slice_by_item(desc, n_slices, item);
        const SliceDesc &d = desc[s];
        const uint32_t g = item - d.item0;
        const uint32_t F = d.tile_nfired[g];
        if (!F) {
            if (lane == 0) d.tile_nwin[g] = 0;
            continue;
        }
        if (!CHECK(8, (uint64_t)d.tile_rank[g] + F, d.n_hits + 1)) continue;
        const trig_trigger *src = d.stage + d.tile_rank[g];
        const uint64_t o = d.tile_out[g];
        const int64_t gap = 2 * (int64_t)d.win_half + 1;
        // the slice's trigger before this tile's first: last of the previous non-empty tile
        int64_t t_before = 0;
        const bool has_before = o > 0;
        if (has_before) {
            uint32_t gp = find_tile_of_pos(d.tile_out, d.n_tiles, (uint32_t)(o - 1));
            t_before = d.stage[d.tile_rank[gp] + (uint32_t)(o - 1 - d.tile_out[gp])].t_ns;
        }
        uint32_t heads = 0;
        for (uint32_t f0 = 0; f0 < F; f0 += 32) {
            const uint32_t f = f0 + lane;
            int64_t t = 0;
            bool head = false;
            if (f < F) {
                int4 v = *reinterpret_cast<const int4 *>(src + f);
                if (o + f < d.trig_cap) *reinterpret_cast<int4 *>(d.triggers + o + f) = v;
                t = (int64_t)(((uint64_t)(uint32_t)v.y << 32) | (uint32_t)v.x);
                int64_t tp = f ? src[f - 1].t_ns : t_before;
                head = (f == 0 && !has_before) || (t - tp > gap);
            }
            heads += __popc(__ballot_sync(0xffffffffu, head));
        }
        if (lane == 0) d.tile_nwin[g] = heads;
    }
}

// ----------------------------------------------------------------- k_wscan

__global__ void __launch_bounds__(1024) k_wscan(const BatchHeader *__restrict__ hdr, const SliceDesc *__restrict__ desc)
{
    if (hdr->err) return;           // the tile pass gave up: its per-tile outputs are not valid
    __shared__ uint32_t wsum[32];
    __shared__ unsigned long long carry;
    for (uint32_t s = blockIdx.x; s < hdr->n_slices; s += gridDim.x) {
        const SliceDesc &d = desc[s];
        unsigned long long nw = block_scan_u32(d.tile_nwin, d.tile_wout, d.n_tiles, wsum, &carry);
        if (threadIdx.x == 0) {
            d.stats->n_windows = nw;
            if (nw > d.win_cap) atomicOr(&d.stats->flags, TRIG_FLAG_WIN_FULL);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- k_wwrite

// One warp per tile: window w of a head trigger is tile_wout[g] plus the
// heads before it in the tile; heads write lo, the first trigger index and
// the rank of the window's first hit, tails (the next trigger is a head, or
// none follows) write hi, the last trigger index and the rank one past the
// window's last hit (both ranks recorded by the tile pass beside the
// fired seed).
__global__ void __launch_bounds__(256) k_wwrite(const BatchHeader *__restrict__ hdr, const SliceDesc *__restrict__ desc)
{
    if (hdr->err) return;           // the tile pass gave up: its per-tile outputs are not valid
    const uint32_t n_items = hdr->n_items, n_slices = hdr->n_slices;
    const uint32_t lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t item = gw; item < n_items; item += nw) {
        const uint32_t s = find_slice_by_item(desc, n_slices, item);
        const SliceDesc &d = desc[s];
        if (d.stats->flags & TRIG_FLAG_TRIG_FULL) continue;      // triggers incomplete
        const uint32_t g = item - d.item0;
        const uint32_t F = d.tile_nfired[g];
        if (!F) continue;
        const uint64_t o = d.tile_out[g];
        const uint64_t nt = d.stats->n_triggers;
        const trig_trigger *T = d.triggers;
        const int64_t gap = 2 * (int64_t)d.win_half + 1;
        const int64_t h = d.win_half;
        uint64_t w_run = d.tile_wout[g];     // windows started before this tile
        for (uint32_t f0 = 0; f0 < F; f0 += 32) {
            const uint32_t f = f0 + lane;
            const uint64_t k = o + f;
            bool head = false, tail = false;
            int64_t t = 0;
            if (f < F) {
                t = T[k].t_ns;
                head = (k == 0) || (t - T[k - 1].t_ns > gap);
                tail = (k + 1 == nt) || (T[k + 1].t_ns - t > gap);
            }
            const uint32_t m = __ballot_sync(0xffffffffu, head);
            const uint64_t w = w_run + __popc(m & ((2u << lane) - 1u)) - 1;   // window of trigger k
            const uint64_t at = 2 * ((uint64_t)d.tile_rank[g] + f);            // the seed's staged ranks
            if (head && w < d.win_cap) {
                d.windows[w].lo_ns = t - h;
                d.windows[w].n_triggers = k;        // first trigger, turned into a count by k_wcount
                if (CHECK(9, at, 2 * d.n_hits)) d.win_r[2 * w] = d.wrank[at];
            }
            if (tail && w < d.win_cap) {
                d.windows[w].hi_ns = t + h;
                d.windows[w].n_hits = k;            // last trigger, turned into the hit count by k_wcount
                if (CHECK(9, at + 1, 2 * d.n_hits)) d.win_r[2 * w + 1] = d.wrank[at + 1];
            }
            w_run += __popc(m);
        }
    }
}

// ---------------------------------------------------------------- k_wcount

// Hit rank of time x in PMT p's stream, narrowed by the tile edges the
// structure pass recorded: x in tile g's core lies between the PMT's
// offsets at B_g - H and B_{g+1} + H, so the binary search covers a handful
// of hits.  Outside the slice the first or last tile's outer edge bounds it.
__device__ __forceinline__ uint64_t rank_in_pmt(const SliceDesc &d, uint32_t p, int64_t x, uint64_t sp, uint64_t ep)
{
    const int64_t W = d.tile_w;
    const int64_t rel = x - d.t0;
    int64_t g = rel < 0 ? 0 : rel / W;
    if (g >= (int64_t)d.n_tiles) g = (int64_t)d.n_tiles - 1;
    const int64_t Bg = d.t0 + g * W;
    const size_t at = (size_t)g * d.n_pmt + p;
    uint64_t lo = sp, hi = ep;
    const uint64_t a = d.e_lo[at], b = d.e_hi[at];
    if (x >= Bg - (int64_t)d.halo) lo = max(lo, min(a, ep));
    if (x <= Bg + W + (int64_t)d.halo) hi = min(hi, max(b, lo));
    return lb_time(d.hits, lo, hi, x);
}

// Merged rank of time x (the hits of the submission with t < x), by the
// warp: per-PMT searches, or for a wide slice the bucket offsets plus the
// edge bucket's hits below x.
__device__ uint64_t warp_rank_of(const SliceDesc &d, int64_t x)
{
    const uint32_t lane = lane_id();
    uint64_t r = 0;
    if (d.wide) {
        const uint32_t bx = bkt_index(d, x);
        const uint32_t e0 = d.bkt_off[bx], e1 = d.bkt_off[bx + 1];
        if (lane == 0) r = e0;
        for (uint32_t j = e0 + lane; j < e1; j += 32) r += d.tbuf[j].t_ns < x;
    } else {
        for (uint32_t p = lane; p < d.n_pmt; p += 32) {
            const uint64_t sp = d.pmt_off[p], ep = d.pmt_off[p + 1];
            r += rank_in_pmt(d, p, x, sp, ep) - sp;
        }
    }
    return warp_sum_u64(r);
}

// Each window's counts from what k_wwrite left: triggers = last - first + 1,
// hits = (rank one past its last hit) - (rank of its first hit); event
// slices also keep the first-hit rank.  The tile pass records both ranks
// beside every fired seed whose window edge lies in its staged range; the
// few others (seeds near a tile edge) are searched for here.  A warp per
// window over the whole batch; the window's slice comes from a prefix over
// slices.
__global__ void __launch_bounds__(256) k_wcount(const BatchHeader *__restrict__ hdr, const SliceDesc *__restrict__ desc)
{
    if (hdr->err) return;           // the tile pass gave up: its per-tile outputs are not valid
    __shared__ unsigned long long pre[1025];
    const uint32_t lane = lane_id();
    const uint32_t n_slices = hdr->n_slices;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint32_t s0 = 0; s0 < n_slices; s0 += 1024) {
        const uint32_t ns = min(1024u, n_slices - s0);
        if (threadIdx.x == 0) {
            unsigned long long run = 0;
            for (uint32_t i = 0; i < ns; ++i) {
                pre[i] = run;
                const SliceDesc &d = desc[s0 + i];
                if (!(d.stats->flags & (TRIG_FLAG_TRIG_FULL | TRIG_FLAG_BAD_PMT | TRIG_FLAG_UNSORTED |
                                        TRIG_FLAG_OUT_OF_RANGE)))
                    run += min((unsigned long long)d.stats->n_windows, (unsigned long long)d.win_cap);
            }
            pre[ns] = run;
        }
        __syncthreads();
        const unsigned long long total = pre[ns];
        for (uint64_t wi = gw; wi < total; wi += nw) {
            uint32_t lo = 0, hi = ns;                     // slice: last i with pre[i] <= wi
            while (hi - lo > 1) {
                uint32_t mid = (lo + hi) >> 1;
                if (pre[mid] <= wi) lo = mid; else hi = mid;
            }
            const SliceDesc &d = desc[s0 + lo];
            const uint64_t i = wi - pre[lo];
            if (!CHECK(10, i, d.win_cap)) continue;
            const uint2 r = *reinterpret_cast<const uint2 *>(d.win_r + 2 * i);
            const trig_window win = d.windows[i];
            const uint64_t r_lo = r.x != kRankUnknown ? (uint64_t)r.x : warp_rank_of(d, win.lo_ns);
            const uint64_t r_hi = r.y != kRankUnknown ? (uint64_t)r.y : warp_rank_of(d, win.hi_ns + 1);
            __syncwarp();
            if (lane == 0) {
                d.windows[i].n_triggers = win.n_hits - win.n_triggers + 1;
                d.windows[i].n_hits = r_hi - r_lo;
                if (d.ev && d.ev_cap) d.win_rlo[i] = (uint32_t)r_lo;
            }
        }
        __syncthreads();
    }
}

// ----------------------------------------------------- event extraction

// The slice's leading halo (t < t0) and trailing halo (t >= t0 + S) in
// merged order at the two ends of its merged stream (the tile pass writes
// the owned hits between them, at their merged ranks).  One block per
// slice; each halo is gathered into shared memory as keys relative to its
// start and ranked by counting.  More than TRIG_EV_HALO_MAX hits in a halo
// sets TRIG_FLAG_EV_FULL.
constexpr uint32_t kEvHaloThreads = 1024;

__device__ void ev_halo_side(const SliceDesc &d, bool lead, uint64_t *keys, uint32_t *psum, int64_t base, int64_t t_cut)
{
    const uint32_t tid = threadIdx.x, P = d.n_pmt;
    const trig_hit *hits = d.hits;
    const uint64_t *poff = d.pmt_off;
    // per-PMT counts of the halo hits (each thread a contiguous run of PMTs)
    const uint32_t per = (P + kEvHaloThreads - 1) / kEvHaloThreads;
    const uint32_t p0 = min(P, tid * per), p1 = min(P, p0 + per);
    uint32_t local = 0;
    for (uint32_t p = p0; p < p1; ++p) {
        const uint64_t a = lb_time(hits, poff[p], poff[p + 1], t_cut);
        local += (uint32_t)(lead ? a - poff[p] : poff[p + 1] - a);
    }
    // exclusive block scan of the per-thread counts
    psum[tid] = local;
    __syncthreads();
    for (uint32_t off = 1; off < kEvHaloThreads; off <<= 1) {
        const uint32_t v = tid >= off ? psum[tid - off] : 0u;
        __syncthreads();
        psum[tid] += v;
        __syncthreads();
    }
    const uint32_t total = psum[kEvHaloThreads - 1];
    uint32_t at = psum[tid] - local;
    __syncthreads();
    if (total > TRIG_EV_HALO_MAX) {
        if (tid == 0) report(d, TRIG_FLAG_EV_FULL);
        return;
    }
    for (uint32_t p = p0; p < p1; ++p) {
        const uint64_t a = lb_time(hits, poff[p], poff[p + 1], t_cut);
        const uint64_t b = lead ? poff[p] : a, e = lead ? a : poff[p + 1];
        for (uint64_t j = b; j < e; ++j, ++at) {
            const trig_hit h = load_hit(hits + j);
            keys[at] = ((uint64_t)(uint32_t)(h.t_ns - base) << 32) | ((uint64_t)h.pmt << 16) | h.charge;
        }
    }
    __syncthreads();
    const uint64_t dst0 = lead ? 0 : d.n_hits - total;
    for (uint32_t i = tid; i < total; i += kEvHaloThreads) {
        const uint64_t k = keys[i];
        uint32_t r = 0;
        for (uint32_t j = 0; j < total; ++j) {
            const uint64_t o = keys[j];
            r += (o < k) || (o == k && j < i);
        }
        trig_hit h;
        h.t_ns = base + (int64_t)(k >> 32);
        h.pmt = (uint16_t)(k >> 16);
        h.charge = (uint16_t)k;
        h.reserved = 0;
        d.dbg_merged[dst0 + r] = h;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kEvHaloThreads) k_evhalo(const BatchHeader *__restrict__ hdr,
                                                           const SliceDesc *__restrict__ desc)
{
    if (hdr->err) return;           // the tile pass gave up: its per-tile outputs are not valid
    extern __shared__ __align__(16) unsigned char ev_smem[];
    uint64_t *keys = reinterpret_cast<uint64_t *>(ev_smem);
    uint32_t *psum = reinterpret_cast<uint32_t *>(keys + TRIG_EV_HALO_MAX);
    for (uint32_t s = blockIdx.x; s < hdr->n_slices; s += gridDim.x) {
        const SliceDesc &d = desc[s];
        if (!d.ev || d.ev_cap == 0) continue;
        if (d.stats->flags & (TRIG_FLAG_BAD_PMT | TRIG_FLAG_UNSORTED | TRIG_FLAG_OUT_OF_RANGE)) continue;
        ev_halo_side(d, true, keys, psum, d.in_lo, d.t0);
        ev_halo_side(d, false, keys, psum, d.t0 + d.slice_ns, d.t0 + d.slice_ns);
    }
}

// Offsets of the windows in the event output: exclusive prefix of their hit
// counts (one block per slice); the total is n_events.
__global__ void __launch_bounds__(1024) k_escan(const BatchHeader *__restrict__ hdr, const SliceDesc *__restrict__ desc)
{
    if (hdr->err) return;           // the tile pass gave up: its per-tile outputs are not valid
    __shared__ uint32_t wsum[33];
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5, nwp = blockDim.x >> 5;
    for (uint32_t s = blockIdx.x; s < hdr->n_slices; s += gridDim.x) {
        const SliceDesc &d = desc[s];
        if (!d.ev || d.ev_cap == 0) continue;
        if (d.stats->flags & (TRIG_FLAG_BAD_PMT | TRIG_FLAG_UNSORTED | TRIG_FLAG_OUT_OF_RANGE | TRIG_FLAG_TRIG_FULL |
                              TRIG_FLAG_WIN_FULL)) {
            if (tid == 0) d.stats->n_events = 0;
            continue;
        }
        const uint32_t nw = (uint32_t)min((unsigned long long)d.stats->n_windows, (unsigned long long)d.win_cap);
        uint32_t carry = 0;
        for (uint32_t base = 0; base < nw; base += blockDim.x) {
            const uint32_t i = base + tid;
            const uint32_t v = i < nw ? (uint32_t)d.windows[i].n_hits : 0u;
            const uint32_t incl = warp_incl_scan(v);
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();
            if (warp == 0) {
                const uint32_t w = lane < nwp ? wsum[lane] : 0u;
                const uint32_t wi = warp_incl_scan(w);
                if (lane < nwp) wsum[lane] = wi - w;
                if (lane == nwp - 1) wsum[32] = wi;
            }
            __syncthreads();
            if (i < nw) d.ev_off[i] = carry + wsum[warp] + incl - v;
            carry += wsum[32];
            __syncthreads();
        }
        if (tid == 0) {
            d.ev_off[nw] = carry;
            d.stats->n_events = carry;
            if (carry > d.ev_cap) atomicOr(&d.stats->flags, TRIG_FLAG_EV_FULL);
        }
        __syncthreads();
    }
}

// The event output: event e of window w is merged hit win_rlo[w] + e -
// ev_off[w].  Slices with any capacity flag (including a skipped 1 ns tile
// piece, whose rows the merged stream lacks) copy nothing.
__global__ void __launch_bounds__(256) k_events(const BatchHeader *__restrict__ hdr, const SliceDesc *__restrict__ desc)
{
    if (hdr->err) return;           // the tile pass gave up: its per-tile outputs are not valid
    const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    for (uint32_t s = 0; s < hdr->n_slices; ++s) {
        const SliceDesc &d = desc[s];
        if (!d.ev || d.ev_cap == 0) continue;
        if (d.stats->flags & (TRIG_FLAG_BAD_PMT | TRIG_FLAG_UNSORTED | TRIG_FLAG_OUT_OF_RANGE | TRIG_FLAG_TRIG_FULL |
                              TRIG_FLAG_WIN_FULL | TRIG_FLAG_EV_FULL | TRIG_FLAG_TILE_FULL))
            continue;
        const uint32_t nw = (uint32_t)min((unsigned long long)d.stats->n_windows, (unsigned long long)d.win_cap);
        const uint64_t ne = d.stats->n_events;
        for (uint64_t e = gt; e < ne; e += nt) {
            // window of event e: last w with ev_off[w] <= e
            uint32_t lo = 0, hi = nw;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (d.ev_off[mid] <= e) lo = mid; else hi = mid;
            }
            const uint64_t src = (uint64_t)d.win_rlo[lo] + (e - d.ev_off[lo]);
            if (CHECK(18, src, d.n_hits) && CHECK(19, e, d.ev_cap))
                *reinterpret_cast<int4 *>(d.ev + e) = *reinterpret_cast<const int4 *>(d.dbg_merged + src);
        }
    }
}

// ----------------------------------------------------------------- k_rank0

// Merged rank of each slice's first owned hit (hits before t0 are the
// leading halo); row outputs are indexed from it.
__global__ void k_rank0(const BatchHeader *__restrict__ hdr, SliceDesc *__restrict__ desc)
{
    const uint32_t s = blockIdx.x;
    if (s >= hdr->n_slices) return;
    SliceDesc &d = desc[s];
    uint64_t r = 0, r1 = 0;
    for (uint32_t p = threadIdx.x; p < d.n_pmt; p += blockDim.x) {
        uint64_t sp = d.pmt_off[p], ep = d.pmt_off[p + 1];
        uint64_t a = lb_time(d.hits, sp, ep, d.t0);
        r += a - sp;
        r1 += lb_time(d.hits, a, ep, d.t0 + d.slice_ns) - sp;
    }
    r = warp_sum_u64(r);
    r1 = warp_sum_u64(r1);
    __shared__ unsigned long long acc, acc1;
    if (threadIdx.x == 0) acc = acc1 = 0;
    __syncthreads();
    if (lane_id() == 0) {
        atomicAdd(&acc, (unsigned long long)r);
        atomicAdd(&acc1, (unsigned long long)r1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        d.dbg_rank0 = acc;
        d.dbg_rank1 = acc1;
    }
}

// -------------------------------------------------------------- k_prepend

// Largest p in [0, P) with off[p] <= x, for non-decreasing offsets with
// off[0] = 0 <= x < off[P].
__device__ __forceinline__ uint32_t run_of(const uint64_t *off, uint32_t P, uint64_t x)
{
    uint32_t lo = 0, hi = P;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (off[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// A continuation submission ("Preparation in CPU": at the end of a slice the
// trigger proceeds on the first hits of the next one; here the next slice
// starts on the last hits of the previous one): PMT p's stream of the
// combined slice is the detector's resident tail of p followed by the
// submission's hits of p.  Tail hit j of PMT p lands at j + fresh_off[p],
// fresh hit i at i + tail_off[p + 1]; the combined offsets are the sums.
__global__ void k_prepend(const trig_hit *__restrict__ tail, const uint64_t *__restrict__ tail_off, uint64_t n_tail,
                          const trig_hit *__restrict__ fresh, const uint64_t *__restrict__ fresh_off,
                          uint64_t n_fresh, uint32_t P, trig_hit *__restrict__ out, uint64_t *__restrict__ out_off)
{
    const uint64_t n = n_tail + n_fresh, total = n + P + 1;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (uint64_t)gridDim.x * blockDim.x) {
        if (x >= n) {
            const uint64_t q = x - n;
            out_off[q] = tail_off[q] + fresh_off[q];
            continue;
        }
        const trig_hit *src;
        uint64_t dst;
        if (x < n_tail) {
            const uint32_t p = run_of(tail_off, P, x);
            src = tail + x;
            dst = x + fresh_off[p];
        } else {
            const uint64_t i = x - n_tail;
            const uint32_t p = run_of(fresh_off, P, i);
            src = fresh + i;
            dst = i + tail_off[p + 1];
        }
        if (CHECK(21, dst, n)) *reinterpret_cast<int4 *>(out + dst) = *reinterpret_cast<const int4 *>(src);
    }
}

cudaError_t launch_prepend(const trig_hit *tail, const uint64_t *tail_off, uint64_t n_tail, const trig_hit *fresh,
                           const uint64_t *fresh_off, uint64_t n_fresh, uint32_t P, trig_hit *out, uint64_t *out_off,
                           cudaStream_t st)
{
    const uint64_t total = n_tail + n_fresh + P + 1;
    const uint64_t blocks = std::min<uint64_t>((total + 255) / 256, (uint64_t)device_sm_count() * 16);
    k_prepend<<<(unsigned)blocks, 256, 0, st>>>(tail, tail_off, n_tail, fresh, fresh_off, n_fresh, P, out, out_off);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- k_status

__global__ void k_status(const BatchHeader *__restrict__ hdr, const SliceDesc *__restrict__ desc)
{
    const uint32_t n = hdr->n_slices;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        trig_slice_stats *st = desc[s].stats;
        uint32_t f = st->flags | hdr->err;
        st->flags = f;
        int32_t status = TRIG_OK;
        if (f & (TRIG_FLAG_BAD_PMT | TRIG_FLAG_UNSORTED | TRIG_FLAG_OUT_OF_RANGE)) status = TRIG_EINVAL;
        else if (f & TRIG_FLAG_TIMEOUT) status = TRIG_ETIMEOUT;
        else if (f & (TRIG_FLAG_TILE_FULL | TRIG_FLAG_TRIG_FULL | TRIG_FLAG_WIN_FULL | TRIG_FLAG_EV_FULL))
            status = TRIG_ECAPACITY;
        st->status = status;
    }
}

#ifdef TRIG_PHASE_STATS
// Tile-kernel counters of the phase-statistics build (summed over blocks
// since the last reset): read n of them into out, then optionally reset.
extern "C" int trig_phase_stats(unsigned long long *out, int n, int reset)
{
    unsigned long long v[24] = {};
    if (n > 24) n = 24;
    if (cudaMemcpyFromSymbol(v, g_phase, sizeof v) != cudaSuccess) return -1;
    for (int i = 0; i < n; ++i) out[i] = v[i];
    if (reset) {
        const unsigned long long z[24] = {};
        if (cudaMemcpyToSymbol(g_phase, z, sizeof z) != cudaSuccess) return -1;
    }
    return 0;
}
#endif

#ifdef TRIG_CHECK
// First recorded check failure of the process (checked builds only).
extern "C" int trig_check_record(unsigned *site, unsigned *count, unsigned long long *index,
                                 unsigned long long *limit)
{
    CheckRecord r{};
    if (cudaMemcpyFromSymbol(&r, g_check, sizeof r) != cudaSuccess) return -1;
    *site = r.site;
    *count = r.count;
    *index = r.index;
    *limit = r.limit;
    return 0;
}
#endif

// ------------------------------------------------- static scratch array

// Scratch of trig_batch_run_noalloc: a fixed device array, present on every
// device that loads the library until the process exits.  Calls share it
// and it keeps the previous call's contents; k_prep clears the counters
// that must start at zero, and everything else is written before it is
// read.  Calls that overlap on the GPU race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TRIG_NOALLOC_SCRATCH_BYTES];

// Device address of the array for the current device, looked up once per
// device (host code may not use the symbol's name as an address).
cudaError_t static_scratch(void **ptr, size_t *bytes)
{
    static std::mutex mu;
    static void *addr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e) return e;
        addr[dev] = p;
    }
    *ptr = addr[dev];
    *bytes = sizeof(g_noalloc_scratch);
    return cudaSuccess;
}

// ------------------------------------------------- no-allocation upload

// The batch header and descriptors of trig_batch_run_noalloc travel as the
// kernel's parameter (copied at launch), so nothing is read from host memory
// after the call returns and no copy waits on the caller's stream.
__global__ void k_put_plan(const NoallocPlan plan, BatchHeader *hdr, SliceDesc *desc)
{
    const uint32_t nw_hdr = sizeof(BatchHeader) / 4;
    const uint32_t nw_desc = plan.n * (uint32_t)(sizeof(SliceDesc) / 4);
    const uint32_t *src_h = reinterpret_cast<const uint32_t *>(&plan.hdr);
    const uint32_t *src_d = reinterpret_cast<const uint32_t *>(plan.desc);
    for (uint32_t i = threadIdx.x; i < nw_hdr; i += blockDim.x) reinterpret_cast<uint32_t *>(hdr)[i] = src_h[i];
    for (uint32_t i = threadIdx.x; i < nw_desc; i += blockDim.x) reinterpret_cast<uint32_t *>(desc)[i] = src_d[i];
}

cudaError_t launch_put_plan(const NoallocPlan &plan, BatchHeader *hdr, SliceDesc *desc, cudaStream_t st)
{
    k_put_plan<<<1, 256, 0, st>>>(plan, hdr, desc);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ launch

int device_sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// The dynamic shared memory limit of a kernel is per-function state that
// CUDA graphs do not capture: a graph replayed after the limit was lowered
// for a smaller launch would exceed it.  So each tile kernel's limit is set
// once per device, to the device's opt-in maximum, and never lowered.
template <typename K>
static cudaError_t raise_smem_limit(K kern, bool *done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (done[dev]) return cudaSuccess;
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kern))) return e;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  optin - (int)fa.sharedSizeBytes)))
        return e;
    done[dev] = true;
    return cudaSuccess;
}

template <int CAP, int NC, bool SMEM_DT, bool EXT = false, bool DENSE = false>
static cudaError_t launch_tile(BatchHeader *hdr, SliceDesc *desc, uint32_t max_pmt, cudaStream_t st)
{
    static bool limit_set[64] = {};
    size_t smem = TileLayout<CAP>::bytes(max_pmt, SMEM_DT);
    auto kern = k_tile<CAP, NC, SMEM_DT, EXT, DENSE>;
    cudaError_t e = raise_smem_limit(kern, limit_set);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NC + 32, smem);
    if (per_sm < 1) per_sm = 1;
    kern<<<device_sm_count() * per_sm, NC + 32, smem, st>>>(hdr, desc, max_pmt);
    return cudaGetLastError();
}

const char *const kKernelNames[kPipelineKernels] = {"k_prep",   "k_bounds", "k_bsum",  "k_bscan",  "k_scatter",
                                                     "k_tile",   "k_evhalo", "k_scan",  "k_copy",   "k_wscan",
                                                     "k_wwrite", "k_wcount", "k_escan", "k_events", "k_status"};

cudaError_t launch_batch(BatchHeader *d_hdr, SliceDesc *d_desc, uint32_t n_slices, uint32_t max_pmt,
                         bool any_smem_dt, bool any_wide, bool any_events, bool any_ext, bool dense,
                         const TileConfig &cfg, cudaStream_t st, uint64_t *launches, bool rows, cudaEvent_t *ev)
{
    const int sms = device_sm_count();
    auto mark = [&](int i) {
        if (ev) cudaEventRecord(ev[i], st);
    };
    const uint32_t sb = n_slices < (uint32_t)sms * 4 ? n_slices : (uint32_t)sms * 4;
    uint64_t nl = 0;
    mark(0);
    k_prep<<<any_wide ? sms : 1, 256, 0, st>>>(d_hdr, d_desc);
    mark(1);
    k_bounds<<<sms * 8, kBoundsThreads, 0, st>>>(d_hdr, d_desc);
    nl += 2;
    if (rows) {
        k_rank0<<<n_slices, 256, 0, st>>>(d_hdr, d_desc);
        nl += 1;
    }
    mark(2);
    if (any_wide) {
        k_bsum<<<sms * 2, kBktChunk, 0, st>>>(d_hdr, d_desc);
        mark(3);
        k_bscan<<<sms * 2, kBktChunk, 0, st>>>(d_hdr, d_desc);
        mark(4);
        k_scatter<<<sms * 8, 256, 0, st>>>(d_hdr, d_desc);
        nl += 3;
    } else {
        mark(3);
        mark(4);
    }
    mark(5);
    cudaError_t e;
    const bool smem_dt = any_smem_dt && max_pmt <= kSmemDtMaxPmt;
    if (any_ext || any_events || rows) {
        // level 0, seed rule 1, distinct count, and every batch that needs
        // the merged rows (event extraction, row outputs): the build that
        // puts each tile in full (t, pmt, charge) order, one per shape, dt
        // rows read through the cache
        if (cfg.cap == 1024)
            e = launch_tile<1024, 128, false, true>(d_hdr, d_desc, max_pmt, st);
        else if (cfg.cap == 2048)
            e = cfg.warps == 16 ? launch_tile<2048, 512, false, true>(d_hdr, d_desc, max_pmt, st)
                                : launch_tile<2048, 256, false, true>(d_hdr, d_desc, max_pmt, st);
        else
            e = cfg.warps == 8 ? launch_tile<4096, 256, false, true>(d_hdr, d_desc, max_pmt, st)
                               : launch_tile<4096, 512, false, true>(d_hdr, d_desc, max_pmt, st);
    } else if (dense) {
        // a warp per seed in the causal count; dt rows read through the cache
        if (cfg.cap == 1024)
            e = launch_tile<1024, 128, false, false, true>(d_hdr, d_desc, max_pmt, st);
        else if (cfg.cap == 2048)
            e = cfg.warps == 16 ? launch_tile<2048, 512, false, false, true>(d_hdr, d_desc, max_pmt, st)
                                : launch_tile<2048, 256, false, false, true>(d_hdr, d_desc, max_pmt, st);
        else
            e = cfg.warps == 8 ? launch_tile<4096, 256, false, false, true>(d_hdr, d_desc, max_pmt, st)
                               : launch_tile<4096, 512, false, false, true>(d_hdr, d_desc, max_pmt, st);
    } else if (cfg.cap == 1024)
        e = smem_dt ? launch_tile<1024, 128, true>(d_hdr, d_desc, max_pmt, st)
                    : launch_tile<1024, 128, false>(d_hdr, d_desc, max_pmt, st);
    else if (cfg.cap == 2048 && cfg.warps == 16)
        e = smem_dt ? launch_tile<2048, 512, true>(d_hdr, d_desc, max_pmt, st)
                    : launch_tile<2048, 512, false>(d_hdr, d_desc, max_pmt, st);
    else if (cfg.cap == 2048)
        e = smem_dt ? launch_tile<2048, 256, true>(d_hdr, d_desc, max_pmt, st)
                    : launch_tile<2048, 256, false>(d_hdr, d_desc, max_pmt, st);
    else if (cfg.warps == 8)
        e = smem_dt ? launch_tile<4096, 256, true>(d_hdr, d_desc, max_pmt, st)
                    : launch_tile<4096, 256, false>(d_hdr, d_desc, max_pmt, st);
    else
        e = smem_dt ? launch_tile<4096, 512, true>(d_hdr, d_desc, max_pmt, st)
                    : launch_tile<4096, 512, false>(d_hdr, d_desc, max_pmt, st);
    if (e != cudaSuccess) return e;
    mark(6);
    if (any_events) {
        static bool ev_limit_set[64] = {};
        int dev = 0;
        if ((e = cudaGetDevice(&dev))) return e;
        const int ev_smem = (int)(TRIG_EV_HALO_MAX * 8 + kEvHaloThreads * 4);
        if (dev >= 0 && dev < 64 && !ev_limit_set[dev]) {
            if ((e = cudaFuncSetAttribute(k_evhalo, cudaFuncAttributeMaxDynamicSharedMemorySize, ev_smem))) return e;
            ev_limit_set[dev] = true;
        }
        k_evhalo<<<sb, kEvHaloThreads, ev_smem, st>>>(d_hdr, d_desc);
        nl += 1;
    }
    mark(7);
    k_scan<<<sb, 1024, 0, st>>>(d_hdr, d_desc);
    mark(8);
    k_copy<<<sms * 4, 256, 0, st>>>(d_hdr, d_desc);
    mark(9);
    k_wscan<<<sb, 1024, 0, st>>>(d_hdr, d_desc);
    mark(10);
    k_wwrite<<<sms * 4, 256, 0, st>>>(d_hdr, d_desc);
    mark(11);
    k_wcount<<<sms * 4, 256, 0, st>>>(d_hdr, d_desc);
    mark(12);
    if (any_events) {
        k_escan<<<sb, 1024, 0, st>>>(d_hdr, d_desc);
        mark(13);
        k_events<<<sms * 8, 256, 0, st>>>(d_hdr, d_desc);
        nl += 2;
    } else {
        mark(13);
    }
    mark(14);
    k_status<<<1, 256, 0, st>>>(d_hdr, d_desc);
    mark(15);
    nl += 7;
    if (launches) *launches += nl;
    return cudaGetLastError();
}

}  // namespace trig
