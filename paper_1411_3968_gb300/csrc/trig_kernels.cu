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
//   k_windows  the +-3 us windows around the triggers, merged while
//              lo_next <= hi_cur + 1, with the hit count inside each.
//
// Every wait on an mbarrier is bounded; a wait that gives up sets
// TRIG_FLAG_TIMEOUT on the batch and the kernel returns.
#include <cstdint>
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

// Bounded wait: about a second at most, then report failure.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (uint32_t i = 0; i < (1u << 22); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i >= 8) __nanosleep(i < 4096 ? 32 : 256);
    }
    return false;
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
    }
}

// ---------------------------------------------------------------- k_bounds

// Number of tile boundaries v_g (g in [0, NG)) with v_g <= t, for
// v_g = base + g * W (lo edges: base = t0 - H) written as
// floor((t - base) / W) + 1, clamped to [0, NG].
__device__ __forceinline__ uint32_t edges_le(int64_t t, int64_t base, uint32_t ws, uint32_t ng)
{
    int64_t q = ((t - base) >> ws) + 1;
    return q <= 0 ? 0u : (q >= (int64_t)ng ? ng : (uint32_t)q);
}

__device__ __forceinline__ void fill_edges(uint32_t *e, uint32_t P, uint32_t p, uint32_t g0, uint32_t g1,
                                           uint32_t v)
{
    for (uint32_t g = g0; g < g1; ++g) e[(size_t)g * P + p] = v;
}

__global__ void __launch_bounds__(256) k_bounds(const BatchHeader *__restrict__ hdr,
                                                const SliceDesc *__restrict__ desc)
{
    const uint32_t n_slices = hdr->n_slices, n_chunks = hdr->n_chunks;
    for (uint32_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        const uint32_t s = find_slice_by_chunk(desc, n_slices, c);
        const SliceDesc &d = desc[s];
        const uint32_t P = d.n_pmt, NG = d.n_tiles, ws = d.wshift;
        const int64_t base_lo = d.t0 - (int64_t)d.halo;             // lo edge g: t0 - H + g W
        const int64_t base_hi = d.t0 + (int64_t)d.halo;             // hi edge g: t0 + H + (g + 1) W
        const uint64_t first = (uint64_t)(c - d.chunk0) * kChunkHits;
        for (uint32_t k = threadIdx.x; k < kChunkHits; k += blockDim.x) {
            const uint64_t li = first + k;
            if (li >= d.n_hits) break;
            const trig_hit h = load_hit(d.hits + li);
            const uint32_t p = h.pmt;
            if (p >= P) { report(d, TRIG_FLAG_BAD_PMT); continue; }
            const uint64_t sp = d.pmt_off[p], ep = d.pmt_off[p + 1];
            if (li < sp || li >= ep) { report(d, TRIG_FLAG_BAD_PMT); continue; }
            const int64_t t = h.t_ns;
            uint32_t bad = 0;
            if (t < d.in_lo || t >= d.in_hi) bad |= TRIG_FLAG_OUT_OF_RANGE;
            const bool is_first = (li == sp);
            int64_t tprev = 0;
            if (!is_first) {
                tprev = d.hits[li - 1].t_ns;
                if (tprev > t) bad |= TRIG_FLAG_UNSORTED;
            }
            if (bad) { report(d, bad); continue; }
            const uint32_t lo_to = edges_le(t, base_lo, ws, NG);
            const uint32_t hi_to = edges_le(t, base_hi + ((int64_t)1 << ws), ws, NG);
            const uint32_t lo_from = is_first ? 0u : edges_le(tprev, base_lo, ws, NG);
            const uint32_t hi_from = is_first ? 0u : edges_le(tprev, base_hi + ((int64_t)1 << ws), ws, NG);
            fill_edges(d.e_lo, P, p, lo_from, lo_to, (uint32_t)li);
            fill_edges(d.e_hi, P, p, hi_from, hi_to, (uint32_t)li);
            if (li == ep - 1) {
                // edges after the last hit point past the stream; so do all edges
                // of the empty PMTs that follow
                fill_edges(d.e_lo, P, p, lo_to, NG, (uint32_t)ep);
                fill_edges(d.e_hi, P, p, hi_to, NG, (uint32_t)ep);
                for (uint32_t q = p + 1; q < P && d.pmt_off[q] == d.pmt_off[q + 1]; ++q) {
                    fill_edges(d.e_lo, P, q, 0, NG, (uint32_t)ep);
                    fill_edges(d.e_hi, P, q, 0, NG, (uint32_t)ep);
                }
            }
            if (li == 0) {
                for (uint32_t q = 0; q < p; ++q) {
                    fill_edges(d.e_lo, P, q, 0, NG, 0u);
                    fill_edges(d.e_hi, P, q, 0, NG, 0u);
                }
            }
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
};

template <int CAP>
struct TileLayout {
    static constexpr int NBK = CAP / 2;                    // time buckets of the in-tile sort
    static constexpr size_t kStage = (size_t)CAP * 16;     // one staging buffer
    static constexpr size_t kTemp = (size_t)CAP * 8;
    static constexpr size_t kCnt = (size_t)(NBK + 1) * 4;
    static constexpr size_t kMask = (size_t)(CAP / 32) * 4;
    static size_t bytes(uint32_t P, bool smem_dt)
    {
        size_t b = 2 * kStage + kTemp + kCnt + kMask;
        b += 2 * (size_t)((P + 7) & ~7u) * 2;              // floor + dmax_row
        if (smem_dt) b += (size_t)P * P * 2;
        return (b + 127) & ~(size_t)127;
    }
};

struct TileCtx {
    // shared memory
    uint64_t *stage[2];
    uint64_t *temp;
    uint32_t *cnt;
    uint32_t *mask;
    uint16_t *floor_s;
    uint16_t *dmax_s;
    uint16_t *dt_s;
    // current tables
    const uint16_t *dt_g;
    uint32_t P;
    bool dt_in_smem;
};

constexpr uint32_t kNC = 512;           // consumer threads
constexpr uint32_t kNW = kNC / 32;      // consumer warps
constexpr uint32_t kBarCons = 1;        // named barrier of the consumers

__device__ __forceinline__ void cons_sync() { named_sync(kBarCons, kNC); }

__device__ __forceinline__ uint32_t key_t(uint64_t k) { return (uint32_t)(k >> 32); }
__device__ __forceinline__ uint32_t key_p(uint64_t k) { return (uint32_t)(k >> 16) & 0xffffu; }
__device__ __forceinline__ uint32_t key_q(uint64_t k) { return (uint32_t)k & 0xffffu; }

__device__ __forceinline__ uint32_t lb_key(const uint64_t *a, uint32_t n, uint64_t v)
{
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Block-wide (consumer) exclusive scan of cnt[0..nb), nb a multiple of kNC;
// writes the total to cnt[nb].  Uses scratch words red[kNW].
__device__ void cons_exclusive_scan(uint32_t *cnt, uint32_t nb, uint32_t *red)
{
    const uint32_t tid = threadIdx.x, per = nb / kNC;
    uint32_t local = 0;
    for (uint32_t i = 0; i < per; ++i) local += cnt[tid * per + i];
    uint32_t incl = warp_incl_scan(local);
    if (lane_id() == 31) red[tid >> 5] = incl;
    cons_sync();
    if (tid < 32) {
        uint32_t v = tid < kNW ? red[tid] : 0u;
        uint32_t vi = warp_incl_scan(v);
        if (tid < kNW) red[tid] = vi - v;
        if (tid == kNW - 1) red[kNW] = vi;
    }
    cons_sync();
    uint32_t run = red[tid >> 5] + incl - local;
    for (uint32_t i = 0; i < per; ++i) {
        uint32_t c = cnt[tid * per + i];
        cnt[tid * per + i] = run;
        run += c;
    }
    if (tid == 0) cnt[nb] = red[kNW];
    cons_sync();
}

// Merge (sort) the n staged records of `buf` by (t - tb, pmt, charge); the
// keys land, in order, in the first 8 * n bytes of `buf`.
template <int CAP>
__device__ void tile_sort(TileCtx &cx, uint64_t *buf, uint32_t n, int64_t tb, uint32_t span, uint32_t *red)
{
    constexpr int NBK = TileLayout<CAP>::NBK;
    constexpr int PER = CAP / kNC;
    const uint32_t tid = threadIdx.x;
    uint32_t bsh = 0;
    {
        uint32_t top = span > 1 ? 32u - __clz(span - 1u) : 0u;    // bits of span - 1
        uint32_t nb_bits = 31u - __clz((uint32_t)NBK);
        bsh = top > nb_bits ? top - nb_bits : 0u;
    }
    for (uint32_t i = tid; i < (uint32_t)NBK; i += kNC) cx.cnt[i] = 0;
    cons_sync();
    uint64_t kreg[PER];
    uint32_t slot[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        uint32_t i = tid + r * kNC;
        kreg[r] = 0;
        slot[r] = 0;
        if (i < n) {
            const uint64_t *rec = buf + 2 * i;
            int64_t t = (int64_t)rec[0];
            uint32_t w1 = (uint32_t)rec[1];
            int64_t rel = t - tb;
            uint32_t tr = rel < 0 ? 0u : (rel > 0xffffffffll ? 0xffffffffu : (uint32_t)rel);
            kreg[r] = ((uint64_t)tr << 32) | ((uint64_t)(w1 & 0xffffu) << 16) | (uint64_t)(w1 >> 16);
            uint32_t bk = tr >> bsh;
            if (bk >= (uint32_t)NBK) bk = NBK - 1;
            slot[r] = atomicAdd(&cx.cnt[bk], 1u);
        }
    }
    cons_sync();
    cons_exclusive_scan(cx.cnt, NBK, red);
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        uint32_t i = tid + r * kNC;
        if (i < n) {
            uint32_t bk = key_t(kreg[r]) >> bsh;
            if (bk >= (uint32_t)NBK) bk = NBK - 1;
            cx.temp[cx.cnt[bk] + slot[r]] = kreg[r];
        }
    }
    cons_sync();
    // rank inside each bucket; identical keys are interchangeable
    for (uint32_t j = tid; j < n; j += kNC) {
        uint64_t k = cx.temp[j];
        uint32_t bk = key_t(k) >> bsh;
        if (bk >= (uint32_t)NBK) bk = NBK - 1;
        uint32_t s0 = cx.cnt[bk], s1 = cx.cnt[bk + 1];
        uint32_t r = s0;
        for (uint32_t m = s0; m < s1; ++m) {
            uint64_t o = cx.temp[m];
            r += (o < k) || (o == k && m < j);
        }
        buf[r] = k;
    }
    cons_sync();
}

struct CoreOut {
    uint32_t n_fired;
    uint32_t n_seeds;
    uint32_t c0;
};

// Seeds, causal counts and emission over the sorted tile keys[0..n).  The
// core is t_rel in [H, H + core_w).  Fired seeds go to out[0..n_fired).
template <int CAP, bool SMEM_DT>
__device__ CoreOut tile_trigger(TileCtx &cx, const uint64_t *keys, uint32_t n, uint32_t H, uint32_t core_w,
                                int64_t tb, const SliceDesc &d, trig_trigger *out, int64_t dbg_rank_lo,
                                uint32_t *red)
{
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const uint32_t c0 = lb_key(keys, n, (uint64_t)H << 32);
    const uint32_t c1 = lb_key(keys, n, (uint64_t)(H + core_w) << 32);
    const uint32_t ncore = c1 - c0;
    const uint32_t tau = d.tau, qseed = d.q_seed, P = cx.P;
    uint16_t *seed_idx = reinterpret_cast<uint16_t *>(cx.temp);
    uint32_t *seed_cnt = reinterpret_cast<uint32_t *>(cx.temp) + CAP / 2;

    // 1. seed flags (one bit per core hit)
    const uint32_t nwords = (ncore + 31) / 32;
    for (uint32_t base = 0; base < ncore; base += kNC) {
        uint32_t i = c0 + base + tid;
        bool seed = false;
        if (i < c1) {
            uint64_t ki = keys[i];
            seed = key_q(ki) >= qseed;
            if (!seed) {
                const uint32_t ti = key_t(ki), pi = key_p(ki), fi = cx.floor_s[pi];
                for (uint32_t j = i + 1; j < n; ++j) {
                    uint64_t kj = keys[j];
                    if (key_t(kj) - ti > tau) break;
                    uint32_t pj = key_p(kj);
                    if (pj != pi && cx.floor_s[pj] == fi) { seed = true; break; }
                }
                if (!seed) {
                    for (uint32_t j = i; j-- > 0;) {
                        uint64_t kj = keys[j];
                        if (ti - key_t(kj) > tau) break;
                        uint32_t pj = key_p(kj);
                        if (pj != pi && cx.floor_s[pj] == fi) { seed = true; break; }
                    }
                }
            }
        }
        uint32_t m = __ballot_sync(0xffffffffu, seed);
        if (lane == 0 && (base + warp * 32) < ncore) cx.mask[(base + warp * 32) >> 5] = m;
    }
    cons_sync();

    // 2. ordered seed list (warp 0)
    if (warp == 0) {
        const uint32_t per = (nwords + 31) / 32;
        uint32_t w0 = lane * per, w1 = min(w0 + per, nwords);
        uint32_t loc = 0;
        for (uint32_t w = w0; w < w1; ++w) loc += __popc(cx.mask[w]);
        uint32_t incl = warp_incl_scan(loc);
        uint32_t pos = incl - loc;
        for (uint32_t w = w0; w < w1; ++w) {
            uint32_t m = cx.mask[w];
            while (m) {
                uint32_t b = __ffs(m) - 1;
                m &= m - 1;
                seed_idx[pos++] = (uint16_t)(c0 + w * 32 + b);
            }
        }
        if (lane == 31) red[0] = incl;
    }
    cons_sync();
    const uint32_t ns = red[0];

    // 3. causal count, one warp per seed: c(s) = #{ j : |t_j - t_s| <= min(dt_max, W) }
    for (uint32_t k = warp; k < ns; k += kNW) {
        const uint64_t ks = keys[seed_idx[k]];
        const uint32_t ts = key_t(ks), ps = key_p(ks);
        const uint32_t dm = cx.dmax_s[ps];
        const uint32_t hi_t = ts + dm;
        uint32_t j = lb_key(keys, n, (uint64_t)(ts - dm) << 32) + lane;
        const uint16_t *row_s = cx.dt_s + (size_t)ps * P;
        const uint16_t *row_g = cx.dt_g + (size_t)ps * P;
        uint32_t c = 0;
        for (;; j += 32) {
            bool in = j < n;
            uint64_t kj = in ? keys[j] : ~0ull;
            uint32_t tj = key_t(kj);
            in = in && tj <= hi_t;
            bool ok = false;
            if (in) {
                uint32_t pj = key_p(kj);
                uint32_t lim = SMEM_DT ? (uint32_t)row_s[pj] : (uint32_t)__ldg(row_g + pj);
                uint32_t ad = tj > ts ? tj - ts : ts - tj;
                ok = ad <= lim;
            }
            c += __popc(__ballot_sync(0xffffffffu, ok));
            if (__ballot_sync(0xffffffffu, in) != 0xffffffffu) break;
        }
        if (lane == 0) seed_cnt[k] = c;
    }
    cons_sync();

    // 4. emit fired seeds in order (warp 0)
    if (warp == 0) {
        uint32_t F = 0;
        for (uint32_t k0 = 0; k0 < ns; k0 += 32) {
            uint32_t k = k0 + lane;
            bool fired = k < ns && seed_cnt[k] >= d.threshold;
            uint32_t m = __ballot_sync(0xffffffffu, fired);
            if (fired) {
                uint64_t ks = keys[seed_idx[k]];
                trig_trigger tr;
                tr.t_ns = tb + (int64_t)key_t(ks);
                tr.pmt = (uint16_t)key_p(ks);
                tr.charge = (uint16_t)key_q(ks);
                tr.count = seed_cnt[k];
                out[F + __popc(m & ((1u << lane) - 1u))] = tr;
            }
            F += __popc(m);
        }
        if (lane == 0) red[1] = F;
    }
    // 5. optional row outputs (verification)
    if (d.dbg_merged) {
        // rows are indexed by merged rank minus the rank of the slice's first owned hit
        const uint64_t dbg_base = (uint64_t)(dbg_rank_lo + (int64_t)c0);
        for (uint32_t i = tid; i < ncore; i += kNC) {
            uint64_t k = keys[c0 + i];
            trig_hit h;
            h.t_ns = tb + (int64_t)key_t(k);
            h.pmt = (uint16_t)key_p(k);
            h.charge = (uint16_t)key_q(k);
            h.reserved = 0;
            d.dbg_merged[dbg_base + i] = h;
            d.dbg_seedcnt[dbg_base + i] = 0xffffffffu;
        }
        cons_sync();
        for (uint32_t k = tid; k < ns; k += kNC) d.dbg_seedcnt[dbg_base + (seed_idx[k] - c0)] = seed_cnt[k];
    }
    cons_sync();
    CoreOut r;
    r.n_fired = red[1];
    r.n_seeds = ns;
    r.c0 = c0;
    cons_sync();
    return r;
}

// Overflow path: the tile holds more than CAP hits with its halo.  Split
// its core in halves until each piece fits; pieces are staged with plain
// loads after per-PMT binary searches.  A 1 ns core that still does not
// fit is reported (TRIG_FLAG_TILE_FULL) and skipped.
template <int CAP, bool SMEM_DT>
__device__ void tile_overflow(TileCtx &cx, uint64_t *buf, const SliceDesc &d, uint32_t g, uint32_t *red,
                              int64_t *stk)
{
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const uint32_t P = d.n_pmt, H = d.halo;
    const int64_t W = (int64_t)1 << d.wshift;
    const int64_t Bg = d.t0 + (int64_t)g * W;
    const int64_t core_end = min(Bg + W, d.t0 + d.slice_ns);
    // merged rank of the tile's first core hit
    uint64_t rk = 0;
    for (uint32_t p = tid; p < P; p += kNC) {
        uint64_t sp = d.pmt_off[p], ep = d.pmt_off[p + 1];
        rk += lb_time(d.hits, sp, ep, Bg) - sp;
    }
    rk = warp_sum_u64(rk);
    if (lane == 0) reinterpret_cast<uint64_t *>(red + 8)[warp] = rk;
    cons_sync();
    if (tid == 0) {
        uint64_t tot = 0;
        for (uint32_t w = 0; w < kNW; ++w) tot += reinterpret_cast<uint64_t *>(red + 8)[w];
        red[4] = (uint32_t)tot;     // tile rank
        red[5] = 0;                 // fired so far
        red[6] = 0;                 // seeds so far
        stk[0] = Bg;
        stk[1] = core_end;
        red[7] = 1;                 // stack depth
    }
    cons_sync();
    const uint32_t tile_rank = red[4];
    for (int guard = 0; guard < 1 << 20; ++guard) {
        uint32_t depth = red[7];
        if (depth == 0) break;
        const int64_t lo = stk[2 * (depth - 1)], hi = stk[2 * (depth - 1) + 1];
        cons_sync();
        // extended count and rank of the piece
        uint64_t tot = 0, rlo = 0;
        for (uint32_t p = tid; p < P; p += kNC) {
            uint64_t sp = d.pmt_off[p], ep = d.pmt_off[p + 1];
            uint64_t a = lb_time(d.hits, sp, ep, lo - (int64_t)H);
            uint64_t b = lb_time(d.hits, a, ep, hi + (int64_t)H);
            tot += b - a;
            rlo += a - sp;
        }
        tot = warp_sum_u64(tot);
        rlo = warp_sum_u64(rlo);
        if (lane == 0) {
            reinterpret_cast<uint64_t *>(red + 8)[warp] = tot;
            reinterpret_cast<uint64_t *>(red + 8 + 2 * kNW)[warp] = rlo;
        }
        cons_sync();
        if (tid == 0) {
            uint64_t T = 0, R = 0;
            for (uint32_t w = 0; w < kNW; ++w) {
                T += reinterpret_cast<uint64_t *>(red + 8)[w];
                R += reinterpret_cast<uint64_t *>(red + 8 + 2 * kNW)[w];
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
        cons_sync();
        const uint32_t total = red[2];
        if (total > (uint32_t)CAP) continue;         // split (or skipped)
        const uint32_t rank_lo = red[3];
        // stage the piece: PMTs in order, one warp per PMT
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
            // warp w copies the PMTs with (p0 / 32) % kNW == w
            if (((p0 >> 5) % kNW) == warp) {
                for (uint32_t q = 0; q < 32; ++q) {
                    uint64_t qa = __shfl_sync(0xffffffffu, a, q);
                    uint32_t ql = __shfl_sync(0xffffffffu, (uint32_t)len, q);
                    uint32_t qd = __shfl_sync(0xffffffffu, my, q);
                    for (uint32_t e = lane; e < ql; e += 32) {
                        trig_hit h = load_hit(d.hits + qa + e);
                        buf[2 * (qd + e)] = (uint64_t)h.t_ns;
                        buf[2 * (qd + e) + 1] = (uint64_t)h.pmt | ((uint64_t)h.charge << 16);
                    }
                }
            }
            dst += __shfl_sync(0xffffffffu, incl, 31);
        }
        cons_sync();
        const int64_t tb = lo - (int64_t)H;
        const uint32_t span = (uint32_t)(hi - lo) + 2 * H;
        tile_sort<CAP>(cx, buf, total, tb, span, red + 64);
        const uint32_t fired0 = red[5];
        CoreOut co = tile_trigger<CAP, SMEM_DT>(cx, buf, total, H, (uint32_t)(hi - lo), tb, d,
                                                 d.stage + tile_rank + fired0,
                                                 (int64_t)rank_lo - (int64_t)d.dbg_rank0, red + 64);
        if (tid == 0) {
            red[5] = fired0 + co.n_fired;
            red[6] += co.n_seeds;
        }
        cons_sync();
    }
    if (tid == 0) {
        d.tile_nfired[g] = red[5];
        d.tile_rank[g] = tile_rank;
        atomicAdd(reinterpret_cast<unsigned long long *>(&d.stats->n_seeds), (unsigned long long)red[6]);
    }
    cons_sync();
}

template <int CAP, bool SMEM_DT>
__global__ void __launch_bounds__(kNC + 32, 1) k_tile(BatchHeader *__restrict__ hdr,
                                                      const SliceDesc *__restrict__ desc, uint32_t max_pmt)
{
    using L = TileLayout<CAP>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t full_bar[2], empty_bar[2];
    __shared__ ItemInfo info[2];
    __shared__ __align__(16) uint32_t red[64 + 64];
    __shared__ int64_t stk[128];

    TileCtx cx;
    unsigned char *sp = smem_raw;
    cx.stage[0] = reinterpret_cast<uint64_t *>(sp);
    sp += L::kStage;
    cx.stage[1] = reinterpret_cast<uint64_t *>(sp);
    sp += L::kStage;
    cx.temp = reinterpret_cast<uint64_t *>(sp);
    sp += L::kTemp;
    cx.cnt = reinterpret_cast<uint32_t *>(sp);
    sp += L::kCnt;
    cx.mask = reinterpret_cast<uint32_t *>(sp);
    sp += L::kMask;
    const uint32_t pp = (max_pmt + 7) & ~7u;
    cx.floor_s = reinterpret_cast<uint16_t *>(sp);
    sp += (size_t)pp * 2;
    cx.dmax_s = reinterpret_cast<uint16_t *>(sp);
    sp += (size_t)pp * 2;
    cx.dt_s = reinterpret_cast<uint16_t *>(sp);
    cx.dt_g = nullptr;
    cx.P = 0;
    cx.dt_in_smem = SMEM_DT;

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

    if (warp == kNW) {
        // ------------------------------------------------ producer warp
        for (uint32_t it = 0;; ++it) {
            const uint32_t b = it & 1u, use = it >> 1;
            if (it >= 2 && !mbar_wait(&empty_bar[b], (use - 1) & 1u)) {
                if (lane == 0) atomicOr(&hdr->err, TRIG_FLAG_TIMEOUT);
                break;
            }
            uint32_t item = 0;
            if (lane == 0) item = atomicAdd(&hdr->queue, 1u);
            item = __shfl_sync(0xffffffffu, item, 0);
            if (item >= n_items) {
                if (lane == 0) {
                    info[b].item = -1;
                    mbar_arrive(&full_bar[b]);
                }
                break;
            }
            const uint32_t s = find_slice_by_item(desc, n_slices, item);
            const SliceDesc &d = desc[s];
            const uint32_t g = item - d.item0, P = d.n_pmt;
            const bool bad = (d.stats->flags & (TRIG_FLAG_BAD_PMT | TRIG_FLAG_UNSORTED | TRIG_FLAG_OUT_OF_RANGE)) != 0;
            uint64_t tot = 0, rlo = 0;
            if (!bad) {
                for (uint32_t p0 = 0; p0 < P; p0 += 32) {
                    uint32_t p = p0 + lane;
                    if (p < P) {
                        uint64_t sp_ = d.pmt_off[p], ep_ = d.pmt_off[p + 1];
                        uint64_t a = d.e_lo[(size_t)g * P + p], e = d.e_hi[(size_t)g * P + p];
                        a = min(max(a, sp_), ep_);
                        e = min(max(e, a), ep_);
                        tot += e - a;
                        rlo += a - sp_;
                    }
                }
            }
            tot = warp_sum_u64(tot);
            rlo = warp_sum_u64(rlo);
            const uint32_t mode = bad ? 2u : (tot > (uint64_t)CAP ? 1u : (tot == 0 ? 2u : 0u));
            if (lane == 0) {
                info[b].item = (int32_t)item;
                info[b].slice = s;
                info[b].g = g;
                info[b].n = (uint32_t)min(tot, (uint64_t)CAP);
                info[b].rank_lo = (uint32_t)rlo;
                info[b].mode = mode;
                if (mode == 0) mbar_arrive_expect_tx(&full_bar[b], (uint32_t)tot * 16u);
                else mbar_arrive(&full_bar[b]);
            }
            __syncwarp();
            if (mode == 0) {
                uint32_t dst = 0;
                for (uint32_t p0 = 0; p0 < P; p0 += 32) {
                    uint32_t p = p0 + lane;
                    uint32_t len = 0;
                    uint64_t a = 0;
                    if (p < P) {
                        uint64_t sp_ = d.pmt_off[p], ep_ = d.pmt_off[p + 1];
                        a = d.e_lo[(size_t)g * P + p];
                        uint64_t e = d.e_hi[(size_t)g * P + p];
                        a = min(max(a, sp_), ep_);
                        e = min(max(e, a), ep_);
                        len = (uint32_t)(e - a);
                    }
                    uint32_t incl = warp_incl_scan(len);
                    if (len) bulk_g2s(cx.stage[b] + 2 * (size_t)(dst + incl - len), d.hits + a, len * 16u,
                                      &full_bar[b]);
                    dst += __shfl_sync(0xffffffffu, incl, 31);
                }
            }
        }
        return;
    }

    // ---------------------------------------------------- consumer warps
    const SliceDesc *loaded = nullptr;
    for (uint32_t it = 0;; ++it) {
        const uint32_t b = it & 1u, use = it >> 1;
        if (!mbar_wait(&full_bar[b], use & 1u)) {
            if (tid == 0) atomicOr(&hdr->err, TRIG_FLAG_TIMEOUT);
            break;
        }
        const ItemInfo inf = info[b];
        if (inf.item < 0) break;
        const SliceDesc &d = desc[inf.slice];
        if (&d != loaded) {
            // (re)load the detector tables of this slice
            cons_sync();
            const uint32_t P = d.n_pmt;
            for (uint32_t p = tid; p < P; p += kNC) {
                cx.floor_s[p] = d.floor[p];
                cx.dmax_s[p] = d.dmax_row[p];
            }
            if (SMEM_DT && P <= kSmemDtMaxPmt)
                for (uint32_t i = tid; i < P * P; i += kNC) cx.dt_s[i] = d.dt[i];
            cx.dt_g = d.dt;
            cx.P = P;
            loaded = &d;
            cons_sync();
        }
        if (inf.mode == 2) {
            if (tid == 0) {
                d.tile_nfired[inf.g] = 0;
                d.tile_rank[inf.g] = 0;
            }
        } else if (inf.mode == 1) {
            tile_overflow<CAP, SMEM_DT>(cx, cx.stage[b], d, inf.g, red, stk);
        } else {
            const int64_t W = (int64_t)1 << d.wshift;
            const int64_t Bg = d.t0 + (int64_t)inf.g * W;
            const int64_t core_end = min(Bg + W, d.t0 + d.slice_ns);
            const uint32_t H = d.halo;
            const int64_t tb = Bg - (int64_t)H;
            const uint32_t span = (uint32_t)W + 2 * H;
            tile_sort<CAP>(cx, cx.stage[b], inf.n, tb, span, red);
            // rank of the core's first hit = rank_lo + c0, known after the sort
            const uint32_t c0 = lb_key(cx.stage[b], inf.n, (uint64_t)H << 32);
            const uint32_t tile_rank = inf.rank_lo + c0;
            CoreOut co = tile_trigger<CAP, SMEM_DT>(cx, cx.stage[b], inf.n, H, (uint32_t)(core_end - Bg), tb, d,
                                                     d.stage + tile_rank,
                                                     (int64_t)inf.rank_lo - (int64_t)d.dbg_rank0, red);
            if (tid == 0) {
                d.tile_nfired[inf.g] = co.n_fired;
                d.tile_rank[inf.g] = tile_rank;
                atomicAdd(reinterpret_cast<unsigned long long *>(&d.stats->n_seeds), (unsigned long long)co.n_seeds);
            }
        }
        // release the buffer to the producer: order our generic-proxy
        // accesses before its next bulk copy into the same buffer
        fence_proxy_async_smem();
        cons_sync();
        if (tid == 0) mbar_arrive(&empty_bar[b]);
    }
}

// ------------------------------------------------------------------ k_scan

__global__ void __launch_bounds__(1024) k_scan(const BatchHeader *__restrict__ hdr, const SliceDesc *__restrict__ desc)
{
    const uint32_t s = blockIdx.x;
    if (s >= hdr->n_slices) return;
    const SliceDesc &d = desc[s];
    const uint32_t NG = d.n_tiles, tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    __shared__ uint32_t wsum[32];
    __shared__ unsigned long long carry;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < NG; base += blockDim.x) {
        uint32_t g = base + tid;
        uint32_t v = g < NG ? d.tile_nfired[g] : 0u;
        uint32_t incl = warp_incl_scan(v);
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = lane < (blockDim.x >> 5) ? wsum[lane] : 0u;
            uint32_t wi = warp_incl_scan(w);
            wsum[lane] = wi - w;
        }
        __syncthreads();
        unsigned long long c = carry;
        if (g < NG) d.tile_out[g] = (uint32_t)(c + wsum[warp] + incl - v);
        __syncthreads();
        if (tid == blockDim.x - 1) carry = c + wsum[warp] + incl;
        __syncthreads();
    }
    if (tid == 0) {
        d.stats->n_triggers = carry;
        if (carry > d.trig_cap) atomicOr(&d.stats->flags, TRIG_FLAG_TRIG_FULL);
    }
}

// ------------------------------------------------------------------ k_copy

__global__ void __launch_bounds__(256) k_copy(const BatchHeader *__restrict__ hdr, const SliceDesc *__restrict__ desc)
{
    const uint32_t n_items = hdr->n_items, n_slices = hdr->n_slices;
    const uint32_t lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t item = gw; item < n_items; item += nw) {
        const uint32_t s = find_slice_by_item(desc, n_slices, item);
        const SliceDesc &d = desc[s];
        const uint32_t g = item - d.item0;
        const uint32_t F = d.tile_nfired[g];
        if (!F) continue;
        const trig_trigger *src = d.stage + d.tile_rank[g];
        const uint64_t o = d.tile_out[g];
        for (uint32_t f = lane; f < F; f += 32) {
            if (o + f < d.trig_cap) {
                int4 v = *reinterpret_cast<const int4 *>(src + f);
                *reinterpret_cast<int4 *>(d.triggers + o + f) = v;
            }
        }
    }
}

// --------------------------------------------------------------- k_windows

// Windows [t - h, t + h] of consecutive triggers (already in time order)
// belong to one merged window unless t_k - t_{k-1} > 2h + 1.  Each thread
// takes a contiguous run of triggers; a block scan gives the window index.
__global__ void __launch_bounds__(512) k_windows(const BatchHeader *__restrict__ hdr, const SliceDesc *__restrict__ desc)
{
    const uint32_t s = blockIdx.x;
    if (s >= hdr->n_slices) return;
    const SliceDesc &d = desc[s];
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5, nt = blockDim.x;
    __shared__ uint32_t wsum[32];
    __shared__ unsigned long long total_w;
    const uint64_t F = min((unsigned long long)d.stats->n_triggers, (unsigned long long)d.trig_cap);
    const int64_t h = d.win_half;
    const int64_t gap = 2 * h + 1;
    const trig_trigger *T = d.triggers;
    const uint64_t per = (F + nt - 1) / nt;
    const uint64_t k0 = min(F, (uint64_t)tid * per), k1 = min(F, k0 + per);
    auto is_head = [&](uint64_t k) -> bool { return k == 0 || T[k].t_ns - T[k - 1].t_ns > gap; };
    uint32_t heads = 0;
    for (uint64_t k = k0; k < k1; ++k) heads += is_head(k);
    uint32_t incl = warp_incl_scan(heads);
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (nt >> 5) ? wsum[lane] : 0u;
        uint32_t wi = warp_incl_scan(w);
        wsum[lane] = wi - w;
        if (lane == (nt >> 5) - 1) total_w = wi;
    }
    __syncthreads();
    const uint64_t W = total_w;
    const uint64_t cap = d.win_cap;
    // window index of trigger k = (#heads in [0, k]) - 1
    uint64_t w = (uint64_t)wsum[warp] + incl - heads;   // heads before k0
    for (uint64_t k = k0; k < k1; ++k) {
        if (is_head(k)) {
            if (w < cap) {
                d.windows[w].lo_ns = T[k].t_ns - h;
                d.windows[w].n_triggers = k;          // first trigger, fixed below
            }
            ++w;
        }
        bool tail = (k + 1 == F) || is_head(k + 1);
        if (tail && w - 1 < cap) {
            d.windows[w - 1].hi_ns = T[k].t_ns + h;
            d.windows[w - 1].n_hits = k;              // last trigger, fixed below
        }
    }
    __syncthreads();
    const uint64_t Wn = min(W, cap);
    if (tid == 0) {
        d.stats->n_windows = W;
        if (W > cap) atomicOr(&d.stats->flags, TRIG_FLAG_WIN_FULL);
    }
    const uint32_t P = d.n_pmt;
    for (uint64_t i = warp; i < Wn; i += nt >> 5) {
        trig_window win = d.windows[i];
        uint64_t cnt = 0;
        for (uint32_t p = lane; p < P; p += 32) {
            uint64_t sp = d.pmt_off[p], ep = d.pmt_off[p + 1];
            uint64_t a = lb_time(d.hits, sp, ep, win.lo_ns);
            uint64_t b = lb_time(d.hits, a, ep, win.hi_ns + 1);
            cnt += b - a;
        }
        cnt = warp_sum_u64(cnt);
        __syncwarp();
        if (lane == 0) {
            d.windows[i].n_triggers = win.n_hits - win.n_triggers + 1;
            d.windows[i].n_hits = cnt;
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
        else if (f & (TRIG_FLAG_TILE_FULL | TRIG_FLAG_TRIG_FULL | TRIG_FLAG_WIN_FULL)) status = TRIG_ECAPACITY;
        st->status = status;
    }
}

// ------------------------------------------------------------------ launch

int device_sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

template <int CAP, bool SMEM_DT>
static cudaError_t launch_tile(BatchHeader *hdr, SliceDesc *desc, uint32_t max_pmt, cudaStream_t st)
{
    size_t smem = TileLayout<CAP>::bytes(max_pmt, SMEM_DT);
    auto kern = k_tile<CAP, SMEM_DT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNC + 32, smem);
    if (per_sm < 1) per_sm = 1;
    kern<<<device_sm_count() * per_sm, kNC + 32, smem, st>>>(hdr, desc, max_pmt);
    return cudaGetLastError();
}

cudaError_t launch_batch(BatchHeader *d_hdr, SliceDesc *d_desc, uint32_t n_slices, uint32_t max_pmt,
                         bool any_smem_dt, const TileConfig &cfg, cudaStream_t st, uint64_t *launches, bool rows)
{
    const int sms = device_sm_count();
    k_prep<<<1, 256, 0, st>>>(d_hdr, d_desc);
    k_bounds<<<sms * 8, 256, 0, st>>>(d_hdr, d_desc);
    if (rows) {
        k_rank0<<<n_slices, 256, 0, st>>>(d_hdr, d_desc);
        if (launches) *launches += 1;
    }
    cudaError_t e;
    const bool smem_dt = any_smem_dt && max_pmt <= kSmemDtMaxPmt;
    if (cfg.cap == 2048)
        e = smem_dt ? launch_tile<2048, true>(d_hdr, d_desc, max_pmt, st)
                    : launch_tile<2048, false>(d_hdr, d_desc, max_pmt, st);
    else
        e = smem_dt ? launch_tile<4096, true>(d_hdr, d_desc, max_pmt, st)
                    : launch_tile<4096, false>(d_hdr, d_desc, max_pmt, st);
    if (e != cudaSuccess) return e;
    k_scan<<<n_slices, 1024, 0, st>>>(d_hdr, d_desc);
    k_copy<<<sms * 4, 256, 0, st>>>(d_hdr, d_desc);
    k_windows<<<n_slices, 512, 0, st>>>(d_hdr, d_desc);
    k_status<<<1, 256, 0, st>>>(d_hdr, d_desc);
    if (launches) *launches += 7;
    return cudaGetLastError();
}

}  // namespace trig
