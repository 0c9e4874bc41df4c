// trig_engine.cpp -- host runtime behind trig.h: detectors, batch planning,
// CUDA-graph replay and the continuously batching slice engine.
//
// Serving model (the paper's TGPU, "CPU-GPU"): slices of several detectors
// arrive on the host; each submission is copied straight from the caller's
// (pageable) memory into a device block before trig_submit_slice returns,
// and queued; a worker thread forms batches from whatever is pending,
// admits a batch when a slot (stream + device arena for outputs and
// scratch) is free and the device has the memory, runs the whole trigger
// for all its slices in one launch sequence, and hands results back per
// detector in submission order.  Up to kSlots batches are in flight, so the
// submissions' copies and the result read-back overlap other batches'
// kernels.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "trig_internal.h"

using namespace trig;

// ---------------------------------------------------------------- errors

// Per-thread message of the last failure; a fixed buffer, so reporting an
// error never allocates.
static thread_local char g_last_error[256];

static int fail(int code, const char *msg)
{
    std::snprintf(g_last_error, sizeof g_last_error, "%s", msg);
    return code;
}

static int fail(int code, const std::string &msg) { return fail(code, msg.c_str()); }

static int cuda_fail(cudaError_t e, const char *what)
{
    std::snprintf(g_last_error, sizeof g_last_error, "%s: %s", what, cudaGetErrorString(e));
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? TRIG_ENOMEM : TRIG_EDEVICE;
}

extern "C" const char *trig_last_error(void) { return g_last_error; }

extern "C" int trig_host_alloc(size_t bytes, void **out)
{
    if (!out || bytes == 0) return fail(TRIG_EINVAL, "trig_host_alloc: out is NULL or bytes is 0");
    *out = nullptr;
    cudaError_t e = cudaHostAlloc(out, bytes, cudaHostAllocPortable);
    if (e) {
        *out = nullptr;
        (void)cudaGetLastError();
        return fail(TRIG_ENOMEM, "trig_host_alloc: cudaHostAlloc failed");
    }
    return TRIG_OK;
}

extern "C" int trig_host_free(void *ptr)
{
    if (!ptr) return fail(TRIG_EINVAL, "trig_host_free: NULL");
    cudaError_t e = cudaFreeHost(ptr);
    return e ? cuda_fail(e, "trig_host_free") : TRIG_OK;
}

static std::atomic<uint64_t> g_launches{0};
extern "C" uint64_t trig_kernel_launch_count(void) { return g_launches.load(); }

static std::mutex g_cfg_mu;
static TileConfig g_cfg{4096, 16, 60};

extern "C" int trig_set_tile_config(uint32_t cap, uint32_t warps, uint32_t fill_pct)
{
    if (!valid_tile_shape(cap, warps) || fill_pct < 10 || fill_pct > 95)
        return fail(TRIG_EINVAL, "trig_set_tile_config: (cap, warps) in {(4096,16), (4096,8), (2048,16), (2048,8), "
                                 "(1024,4)}, fill_pct in [10, 95]");
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    g_cfg = TileConfig{cap, warps, fill_pct};
    return TRIG_OK;
}

extern "C" int trig_get_tile_config(uint32_t *cap, uint32_t *warps, uint32_t *fill_pct)
{
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    if (cap) *cap = g_cfg.cap;
    if (warps) *warps = g_cfg.warps;
    if (fill_pct) *fill_pct = g_cfg.fill_pct;
    return TRIG_OK;
}

// Limit of the tile pass's device waits and the stall test control.
static std::atomic<uint64_t> g_wait_ns{kDefaultWaitNs};
static std::atomic<uint32_t> g_stall{0};

extern "C" int trig_set_device_wait(uint64_t limit_ns, int stall)
{
    if (stall != 0 && stall != 1) return fail(TRIG_EINVAL, "stall must be 0 or 1");
    if (limit_ns > (uint64_t)600 * kDefaultWaitNs) return fail(TRIG_EINVAL, "limit_ns must be at most 600 s");
    g_wait_ns = limit_ns ? limit_ns : kDefaultWaitNs;
    g_stall = (uint32_t)stall;
    return TRIG_OK;
}

static TileConfig current_cfg()
{
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    return g_cfg;
}

static bool tune_cache_lookup(uint32_t n_pmt, TileConfig &out);

// ------------------------------------------------------------- detectors

struct DetQueue {
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> order;                    // submitted ids, oldest first
    std::map<uint64_t, trig_result *> done;
    uint64_t in_flight = 0;
};

// The detector's resident slice tail: the hits of its last submission in
// [t0 + S - halo, t0 + S) (halo = the accepted input halo), grouped by PMT,
// kept on the device as the leading halo of a continuation submission.
struct TailState {
    std::mutex mu;                  // serialises the detector's submissions
    bool have = false;
    int64_t next_t0 = 0;            // t0 of the slice that may continue it
    // two device copies: a submission reads the current one (cur) while it
    // writes the next slice's into the other, so one stream sync suffices
    trig_hit *d_hits[2] = {nullptr, nullptr};   // device, cap[i] entries
    uint64_t *d_off[2] = {nullptr, nullptr};    // device, n_pmt + 1 offsets
    size_t cap[2] = {0, 0};
    int cur = 0;
    trig_hit *h_hits = nullptr;     // page-locked staging of the next tail, h_cap entries
    uint64_t *h_off = nullptr;      // page-locked, n_pmt + 1 offsets
    size_t h_cap = 0;
    std::vector<uint64_t> off;      // host copy of the current offsets
};

struct trig_detector {
    uint32_t n_pmt = 0;
    trig_params par{};
    int device = 0;
    uint32_t tile_halo = 0;       // max(max_q min(dt_max, W), tau)
    int64_t in_halo = 0;          // accepted halo around a slice
    std::vector<int32_t> xyz;
    std::vector<uint32_t> floor_id;
    DetDev dev{};
    int32_t *d_xyz = nullptr;
    std::shared_ptr<DetQueue> q;
    bool tuned = false;           // tile shape chosen by trig_autotune (or its cache)
    TileConfig tile{};
    bool events = false;          // engine results carry the event payload
    TailState tail;
};

namespace trig {
bool detector_info(const trig_detector *d, DetInfo *out)
{
    if (!d || !out) return false;
    out->n_pmt = d->n_pmt;
    out->xyz = d->xyz.data();
    out->par = d->par;
    out->in_halo = d->in_halo;
    out->device = d->device;
    return true;
}
int report_error(int code, const char *msg) { return fail(code, msg); }
int report_cuda_error(cudaError_t e, const char *what) { return cuda_fail(e, what); }
void count_launches(uint64_t n) { g_launches += n; }
}  // namespace trig

static void free_det_dev(trig_detector *d)
{
    for (int i = 0; i < 2; ++i) {
        cudaFree(d->tail.d_hits[i]);
        cudaFree(d->tail.d_off[i]);
        d->tail.d_hits[i] = nullptr;
        d->tail.d_off[i] = nullptr;
        d->tail.cap[i] = 0;
    }
    cudaFreeHost(d->tail.h_hits);
    cudaFreeHost(d->tail.h_off);
    d->tail.h_hits = nullptr;
    d->tail.h_off = nullptr;
    d->tail.h_cap = 0;
    cudaFree(d->dev.dt);
    cudaFree(d->dev.dt_exact);
    cudaFree(d->dev.floor);
    cudaFree(d->dev.dmax_row);
    cudaFree(d->dev.rel);
    cudaFree(d->d_xyz);
    d->dev = DetDev{};
    d->d_xyz = nullptr;
}

static int check_params(const trig_params *p)
{
    if (!p) return fail(TRIG_EINVAL, "params is NULL");
    if (p->n_den == 0 || p->n_num == 0) return fail(TRIG_EINVAL, "n_num and n_den must be positive");
    if (p->slice_ns <= 0 || p->slice_ns > ((int64_t)1 << 40)) return fail(TRIG_EINVAL, "slice_ns out of range");
    if (p->corr_window_ns > 60000 || p->win_half_ns > 60000 || p->floor_tau_ns > 60000)
        return fail(TRIG_EINVAL, "corr_window_ns, win_half_ns and floor_tau_ns must be <= 60000");
    if (p->q_seed_adc > 65536) return fail(TRIG_EINVAL, "q_seed_adc > 65536");
    if (p->l0_hits > 0 && (p->l0_window_ns == 0 || p->l0_window_ns > 60000))
        return fail(TRIG_EINVAL, "l0_window_ns must be in [1, 60000] when l0_hits > 0");
    if (p->l0_hits > 4096) return fail(TRIG_EINVAL, "l0_hits > 4096");
    if (p->l0_distinct_pmts > 1) return fail(TRIG_EINVAL, "l0_distinct_pmts is 0 or 1");
    if (p->seed_rule > 1) return fail(TRIG_EINVAL, "seed_rule is 0 or 1");
    if (p->sc_window_ns > 60000 || p->fc_window_ns > 60000 || p->afc_window_ns > 60000)
        return fail(TRIG_EINVAL, "sc_window_ns, fc_window_ns and afc_window_ns must be <= 60000");
    if (p->count_distinct_pmts > 1 || p->reserved != 0)
        return fail(TRIG_EINVAL, "count_distinct_pmts is 0 or 1, reserved 0");
    return TRIG_OK;
}

// Relations of the coincidence seed rule, rel[p * P + q] (kRel* bits):
// another PMT of the same floor; adjacent (same floor, at most sc_dist_mm
// apart); on a consecutive floor of the same tower.  A tower's floors are
// ordered by the z of their lowest PMT, then by floor id.
static std::vector<uint8_t> pmt_relations(const trig_geometry *g, uint32_t sc_dist_mm)
{
    const uint32_t P = g->n_pmt;
    auto tower = [&](uint32_t p) { return g->tower_id ? g->tower_id[p] : 0u; };
    std::map<uint32_t, int32_t> low;                    // floor id -> z of its lowest PMT
    for (uint32_t p = 0; p < P; ++p) {
        auto it = low.find(g->floor_id[p]);
        const int32_t z = g->xyz_mm[3 * p + 2];
        if (it == low.end()) low.emplace(g->floor_id[p], z);
        else it->second = std::min(it->second, z);
    }
    // per tower: its floors in height order -> position in that order
    std::map<uint32_t, std::vector<std::pair<int32_t, uint32_t>>> floors;
    for (uint32_t p = 0; p < P; ++p) floors[tower(p)].push_back({low[g->floor_id[p]], g->floor_id[p]});
    std::map<std::pair<uint32_t, uint32_t>, int64_t> level;    // (tower, floor id) -> position
    for (auto &tf : floors) {
        auto &v = tf.second;
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        for (size_t i = 0; i < v.size(); ++i) level[{tf.first, v[i].second}] = (int64_t)i;
    }
    std::vector<int64_t> lv(P);
    for (uint32_t p = 0; p < P; ++p) lv[p] = level[{tower(p), g->floor_id[p]}];
    const int64_t r2 = (int64_t)sc_dist_mm * sc_dist_mm;
    std::vector<uint8_t> rel((size_t)P * P, 0);
    for (uint32_t p = 0; p < P; ++p)
        for (uint32_t q = 0; q < P; ++q) {
            uint8_t r = 0;
            if (p != q && g->floor_id[p] == g->floor_id[q]) {
                r |= kRelFloor;
                int64_t d2 = 0;
                for (int c = 0; c < 3; ++c) {
                    const int64_t dc = (int64_t)g->xyz_mm[3 * p + c] - g->xyz_mm[3 * q + c];
                    d2 += dc * dc;
                }
                if (d2 <= r2) r |= kRelAdjacent;
            }
            if (tower(p) == tower(q) && (lv[p] - lv[q] == 1 || lv[q] - lv[p] == 1)) r |= kRelNextFloor;
            rel[(size_t)p * P + q] = r;
        }
    return rel;
}

extern "C" int trig_create(const trig_geometry *g, const trig_params *params, trig_detector **out)
{
    if (!out) return fail(TRIG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!g || !g->xyz_mm || !g->floor_id) return fail(TRIG_EINVAL, "geometry or its arrays are NULL");
    if (g->n_pmt < 1 || g->n_pmt > kMaxPmt) return fail(TRIG_EINVAL, "n_pmt must be in [1, 4096]");
    int rc = check_params(params);
    if (rc) return rc;
    const uint32_t P = g->n_pmt;
    for (uint32_t i = 0; i < 3 * P; ++i)
        if (g->xyz_mm[i] > 100000000 || g->xyz_mm[i] < -100000000)
            return fail(TRIG_EINVAL, "coordinates must lie within +-1e8 mm");

    std::unique_ptr<trig_detector> d(new trig_detector());
    d->n_pmt = P;
    d->par = *params;
    cudaGetDevice(&d->device);
    d->xyz.assign(g->xyz_mm, g->xyz_mm + 3 * P);
    d->floor_id.assign(g->floor_id, g->floor_id + P);
    // dense floor indices
    std::vector<uint16_t> floor_dense(P);
    {
        std::map<uint32_t, uint16_t> ids;
        for (uint32_t p = 0; p < P; ++p) {
            auto it = ids.find(g->floor_id[p]);
            if (it == ids.end()) it = ids.emplace(g->floor_id[p], (uint16_t)ids.size()).first;
            floor_dense[p] = it->second;
        }
    }
    const size_t PP = (size_t)P * P;
    cudaError_t e;
    if ((e = cudaMalloc(&d->dev.dt, PP * 2)) || (e = cudaMalloc(&d->dev.dt_exact, PP * 4)) ||
        (e = cudaMalloc(&d->dev.floor, (size_t)P * 2)) || (e = cudaMalloc(&d->dev.dmax_row, (size_t)P * 2)) ||
        (e = cudaMalloc(&d->d_xyz, (size_t)3 * P * 4)) ||
        (params->seed_rule == 1 && (e = cudaMalloc(&d->dev.rel, PP)))) {
        free_det_dev(d.get());
        return cuda_fail(e, "trig_create: cudaMalloc");
    }
    cudaStream_t st;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking))) {
        free_det_dev(d.get());
        return cuda_fail(e, "trig_create: stream");
    }
    std::vector<uint16_t> dmax(P);
    std::vector<uint8_t> rel;
    if (params->seed_rule == 1) rel = pmt_relations(g, params->sc_dist_mm);
    e = cudaMemcpyAsync(d->d_xyz, g->xyz_mm, (size_t)3 * P * 4, cudaMemcpyHostToDevice, st);
    if (!e && !rel.empty()) e = cudaMemcpyAsync(d->dev.rel, rel.data(), PP, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(d->dev.floor, floor_dense.data(), (size_t)P * 2, cudaMemcpyHostToDevice, st);
    if (!e)
        e = launch_dtmax(d->d_xyz, P, params->tol_ns, params->n_num, params->n_den, params->corr_window_ns,
                         d->dev.dt_exact, d->dev.dt, d->dev.dmax_row, st);
    if (!e) e = cudaMemcpyAsync(dmax.data(), d->dev.dmax_row, (size_t)P * 2, cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (e) {
        free_det_dev(d.get());
        return cuda_fail(e, "trig_create: building dt_max");
    }
    // the tile halo covers every hit a core hit's seed test, level 0 and
    // causal count look at; the accepted input halo as well
    const uint32_t l0w = params->l0_hits > 0 ? params->l0_window_ns : 0u;
    const uint32_t cw = params->seed_rule == 1
                            ? std::max({params->sc_window_ns, params->fc_window_ns, params->afc_window_ns})
                            : params->floor_tau_ns;
    uint32_t H = std::max(cw, l0w);
    for (uint16_t v : dmax) H = std::max<uint32_t>(H, v);
    d->tile_halo = H;
    d->in_halo = std::max<int64_t>({(int64_t)params->corr_window_ns, (int64_t)params->win_half_ns,
                                    (int64_t)cw, (int64_t)l0w});
    d->q = std::make_shared<DetQueue>();
    TileConfig cached{};
    if (tune_cache_lookup(P, cached)) {
        d->tuned = true;
        d->tile = cached;
    }
    *out = d.release();
    return TRIG_OK;
}

extern "C" int64_t trig_detector_halo_ns(const trig_detector *d) { return d ? d->in_halo : -1; }

extern "C" int trig_set_events(trig_detector *det, int on)
{
    if (!det) return fail(TRIG_EINVAL, "NULL detector");
    det->events = on != 0;
    return TRIG_OK;
}

extern "C" int trig_detector_dtmax(const trig_detector *d, int32_t *dt_out)
{
    if (!d || !dt_out) return fail(TRIG_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpy(dt_out, d->dev.dt_exact, (size_t)d->n_pmt * d->n_pmt * 4, cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(e, "trig_detector_dtmax");
    return TRIG_OK;
}

// ------------------------------------------------------------ batch plan

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Plan {
    BatchHeader hdr{};
    std::vector<SliceDesc> desc;
    size_t bytes = 0;
    uint32_t max_pmt = 0;
    bool smem_dt = true;
    bool any_wide = false;
    bool any_events = false;
    TileConfig shape{};         // launch shape of this batch
};

// Tile width W (ns): a tile plus its two halos is expected to hold fill% of
// the tile capacity at the slice's mean rate; W >= 256 ns and at most 2^20
// tiles per slice.
static int64_t choose_tile_w(const trig_detector *det, uint64_t n_hits, const TileConfig &cfg)
{
    const double span = (double)det->par.slice_ns + 2.0 * (double)det->in_halo;
    const double rate = n_hits > 0 ? (double)n_hits / span : 1e-9;       // hits per ns
    const uint32_t fill = det->tuned ? det->tile.fill_pct : cfg.fill_pct;
    const double target = (double)cfg.cap * fill / 100.0;
    double w = target / rate - 2.0 * det->tile_halo;
    const double w_min = std::max(256.0, (double)det->par.slice_ns / (double)kMaxTilesPerSlice + 1.0);
    if (w < w_min) w = w_min;
    if (w > (double)det->par.slice_ns) w = (double)det->par.slice_ns;
    // a tile plus its halos spans less than kMaxTileSpan ns
    const double w_max = std::max(1.0, (double)(kMaxTileSpan - 1) - 2.0 * det->tile_halo);
    if (w > w_max) w = w_max;
    return (int64_t)w;
}

// Bucket grid of a wide slice: buckets of Wb ns from O = t0 - lead * Wb,
// tiles of m buckets, hh buckets of halo on each side (hh * Wb >= H).  Wb
// is about H / 2, smaller when a bucket would hold more than an eighth of a
// tile at the slice's mean rate; m fills a tile with its halos to the
// target fill.
struct WideGrid {
    uint32_t wb, hh, m, lead, nb;
};

static WideGrid wide_grid(const trig_detector *det, uint64_t n_hits, const TileConfig &cfg)
{
    const double S = (double)det->par.slice_ns;
    const double span = S + 2.0 * (double)det->in_halo;
    const double rate = n_hits > 0 ? (double)n_hits / span : 1e-9;        // hits per ns
    const uint32_t fill = det->tuned ? det->tile.fill_pct : cfg.fill_pct;
    const double target = (double)cfg.cap * fill / 100.0;
    const uint32_t H = det->tile_halo;
    double wb = std::max(64.0, std::ceil(H / 2.0));
    wb = std::min(wb, std::max(64.0, std::floor(target / 8.0 / rate)));
    wb = std::max(wb, std::ceil(span / (double)(1u << 22)));                 // at most ~4M buckets
    WideGrid g{};
    g.wb = (uint32_t)std::min(wb, 1e9);
    g.hh = H ? (H + g.wb - 1) / g.wb : 0;
    double m = std::floor(target / ((double)g.wb * rate)) - 2.0 * g.hh;
    m = std::min(m, std::ceil(S / g.wb));
    m = std::min(m, std::floor((double)(kMaxTileSpan - 1) / g.wb) - 2.0 * g.hh);   // staged span below 2^20 ns
    m = std::max(1.0, m);
    g.m = (uint32_t)m;
    g.lead = (uint32_t)(((uint64_t)det->in_halo + g.wb - 1) / g.wb);
    g.nb = g.lead + (uint32_t)(((uint64_t)det->par.slice_ns + (uint64_t)det->in_halo + g.wb - 1) / g.wb) + 1;
    return g;
}

// Plans a batch into caller-provided storage (no allocation): descriptors
// desc[0..n), the header, the scratch size and the launch shape.
// The launch shape of a batch: the tuned shape of the detector with the
// most hits in it, else the global configuration.
static TileConfig batch_shape(const trig_slice_dev *sl, uint32_t n, const TileConfig &cfg)
{
    TileConfig out = cfg;
    uint64_t best = 0;
    for (uint32_t s = 0; s < n; ++s) {
        const trig_detector *det = sl[s].det;
        if (det && det->tuned && sl[s].n_hits >= best) {
            best = sl[s].n_hits;
            out.cap = det->tile.cap;
            out.warps = det->tile.warps;
        }
    }
    return out;
}

static int plan_into(const trig_slice_dev *sl, uint32_t n, uintptr_t base, const TileConfig &cfg_in,
                     BatchHeader &hdr, SliceDesc *desc, size_t &bytes, uint32_t &max_pmt, bool &smem_dt,
                     bool &any_wide, TileConfig *shape_out = nullptr, const trig_slice_events *ev = nullptr,
                     bool *any_events_out = nullptr)
{
    bool any_events = false, any_ext = false, dense = false;
    if (!sl || n == 0) return fail(TRIG_EINVAL, "no slices");
    const TileConfig cfg = batch_shape(sl, n, cfg_in);
    if (shape_out) *shape_out = cfg;
    size_t off = align256(sizeof(BatchHeader));
    off += align256(sizeof(SliceDesc) * n);
    uint32_t items = 0, chunks = 0;
    max_pmt = 0;
    smem_dt = true;
    any_wide = false;
    for (uint32_t s = 0; s < n; ++s) {
        const trig_slice_dev &x = sl[s];
        const trig_detector *det = x.det;
        if (!det) return fail(TRIG_EINVAL, "slice without detector");
        if (!x.pmt_off || !x.stats || (x.n_hits && !x.hits)) return fail(TRIG_EINVAL, "slice buffers are NULL");
        if (x.n_hits > kMaxSliceHits) return fail(TRIG_EINVAL, "slice has too many hits (limit 2^32 - 16)");
        if (((uintptr_t)x.hits & 15u) != 0) return fail(TRIG_EINVAL, "hits must be 16-byte aligned");
        if ((x.trig_cap && !x.triggers) || (x.win_cap && !x.windows)) return fail(TRIG_EINVAL, "outputs are NULL");
        if (x.t0_ns < -((int64_t)1 << 61) || x.t0_ns > ((int64_t)1 << 61)) return fail(TRIG_EINVAL, "t0 out of range");
        SliceDesc &d = desc[s];
        d = SliceDesc{};
        const uint32_t P = det->n_pmt;
        max_pmt = std::max(max_pmt, P);
        if (P > kSmemDtMaxPmt) smem_dt = false;
        d.hits = x.hits;
        d.pmt_off = x.pmt_off;
        d.dt = det->dev.dt;
        d.floor = det->dev.floor;
        d.dmax_row = det->dev.dmax_row;
        d.n_pmt = P;
        d.halo = det->tile_halo;
        d.q_seed = det->par.q_seed_adc;
        d.tau = det->par.floor_tau_ns;
        d.threshold = det->par.threshold;
        d.l0_hits = det->par.l0_hits;
        d.l0_window = det->par.l0_window_ns;
        d.l0_distinct = det->par.l0_distinct_pmts;
        d.seed_rule = det->par.seed_rule;
        d.sc_w = det->par.sc_window_ns;
        d.fc_w = det->par.fc_window_ns;
        d.afc_w = det->par.afc_window_ns;
        d.count_distinct = det->par.count_distinct_pmts;
        d.rel = det->dev.rel;
        d.win_half = det->par.win_half_ns;
        d.t0 = x.t0_ns;
        d.slice_ns = det->par.slice_ns;
        d.in_lo = x.t0_ns - det->in_halo;
        d.in_hi = x.t0_ns + det->par.slice_ns + det->in_halo;
        d.n_hits = x.n_hits;
        const bool wide = P >= kWideMinPmt;
        any_wide |= wide;
        any_ext |= det->par.l0_hits > 0 || det->par.seed_rule != 0 || det->par.count_distinct_pmts != 0;
        {
            const double span = (double)det->par.slice_ns + 2.0 * (double)det->in_halo;
            dense |= (double)x.n_hits / span * (2.0 * det->tile_halo + 1.0) >= kDenseKeys;
        }
        int64_t W = 0;
        if (wide) {
            const WideGrid wg = wide_grid(det, x.n_hits, cfg);
            if ((uint64_t)(wg.m + 2 * wg.hh) * wg.wb >= (uint64_t)kMaxTileSpan)
                return fail(TRIG_EINVAL, "slice too long for this detector's tiles");
            W = (int64_t)wg.m * wg.wb;
            d.wide = 1;
            d.bkt_w = wg.wb;
            d.bkt_magic = (uint32_t)((((uint64_t)1 << 32) + wg.wb - 1) / wg.wb);
            d.bkt_lead = wg.lead;
            d.bkt_per_tile = wg.m;
            d.bkt_halo = wg.hh;
            d.n_bkt = wg.nb;
            d.bkt32 = (uint64_t)wg.nb * wg.wb < ((uint64_t)1 << 31);
            d.bkt_origin = x.t0_ns - (int64_t)wg.lead * wg.wb;
        } else {
            W = choose_tile_w(det, x.n_hits, cfg);
        }
        d.tile_w = W;
        d.w_magic = (uint32_t)((((uint64_t)1 << 32) + (uint64_t)W - 1) / (uint64_t)W);
        d.span32 = (det->par.slice_ns + 2 * det->in_halo + 2 * (int64_t)det->tile_halo + 2 * W) < ((int64_t)1 << 31);
        const uint64_t ng = x.n_hits ? (uint64_t)((det->par.slice_ns + W - 1) / W) : 0;
        if (ng > kMaxTilesPerSlice) return fail(TRIG_EINVAL, "too many tiles");
        d.n_tiles = (uint32_t)ng;
        d.item0 = items;
        d.chunk0 = chunks;
        items += d.n_tiles;
        chunks += (uint32_t)((x.n_hits + kChunkHits - 1) / kChunkHits);
        if (wide) {
            d.bkt_cnt = reinterpret_cast<uint32_t *>(base + off);
            off += align256((size_t)d.n_bkt * 4);
            d.bkt_off = reinterpret_cast<uint32_t *>(base + off);
            off += align256(((size_t)d.n_bkt + 1) * 4);
            d.bkt_part = reinterpret_cast<uint32_t *>(base + off);
            off += align256(((size_t)d.n_bkt + kBktChunk - 1) / kBktChunk * 4);
            d.tbuf = reinterpret_cast<trig_hit *>(base + off);
            off += align256((size_t)x.n_hits * sizeof(trig_hit));
        } else {
            const size_t eb = (size_t)d.n_tiles * P * 4;
            d.e_lo = reinterpret_cast<uint32_t *>(base + off);
            off += align256(eb);
            d.e_hi = reinterpret_cast<uint32_t *>(base + off);
            off += align256(eb);
        }
        d.tile_nfired = reinterpret_cast<uint32_t *>(base + off);
        off += align256((size_t)d.n_tiles * 4);
        d.tile_rank = reinterpret_cast<uint32_t *>(base + off);
        off += align256((size_t)d.n_tiles * 4);
        d.tile_out = reinterpret_cast<uint32_t *>(base + off);
        off += align256((size_t)d.n_tiles * 4);
        d.tile_nwin = reinterpret_cast<uint32_t *>(base + off);
        off += align256((size_t)d.n_tiles * 4);
        d.tile_wout = reinterpret_cast<uint32_t *>(base + off);
        off += align256((size_t)d.n_tiles * 4);
        d.stage = reinterpret_cast<trig_trigger *>(base + off);
        off += align256((size_t)x.n_hits * sizeof(trig_trigger));
        d.wrank = reinterpret_cast<uint32_t *>(base + off);
        off += align256((size_t)x.n_hits * 8);
        d.win_r = reinterpret_cast<uint32_t *>(base + off);
        off += align256((size_t)x.win_cap * 8);
        d.triggers = x.triggers;
        d.trig_cap = x.trig_cap;
        d.windows = x.windows;
        d.win_cap = x.win_cap;
        d.stats = x.stats;
        d.dbg_merged = nullptr;
        d.dbg_seedcnt = nullptr;
        d.dbg_rank0 = 0;
        d.ev = nullptr;
        d.ev_cap = 0;
        if (ev && ev[s].ev_cap > 0) {
            // event extraction: the tile pass writes the merged stream (row
            // outputs from merged rank 0, no seed counts)
            if (!ev[s].events || ((uintptr_t)ev[s].events & 15u)) return fail(TRIG_EINVAL, "events must be 16-byte aligned device memory");
            if (x.n_hits > 0xFFFFFFFFull) return fail(TRIG_EINVAL, "event extraction takes slices below 2^32 hits");
            any_events = true;
            d.ev = ev[s].events;
            d.ev_cap = ev[s].ev_cap;
            d.dbg_merged = reinterpret_cast<trig_hit *>(base + off);
            off += align256((size_t)x.n_hits * sizeof(trig_hit));
            d.win_rlo = reinterpret_cast<uint32_t *>(base + off);
            off += align256((size_t)x.win_cap * 4);
            d.ev_off = reinterpret_cast<uint32_t *>(base + off);
            off += align256(((size_t)x.win_cap + 1) * 4);
        }
    }
    if (any_events_out) *any_events_out = any_events;
    hdr = BatchHeader{};
    hdr.n_slices = n;
    hdr.any_wide = any_wide ? 1u : 0u;
    hdr.any_events = any_events ? 1u : 0u;
    hdr.any_ext = any_ext ? 1u : 0u;
    hdr.dense = dense ? 1u : 0u;
    hdr.n_items = items;
    hdr.n_chunks = chunks;
    hdr.wait_ns = g_wait_ns.load();
    hdr.stall = g_stall.load();
    bytes = off;
    return TRIG_OK;
}

static int make_plan(const trig_slice_dev *sl, uint32_t n, uintptr_t base, const TileConfig &cfg, Plan &pl,
                     bool rows, const trig_slice_events *ev = nullptr)
{
    (void)rows;
    if (!sl || n == 0) return fail(TRIG_EINVAL, "no slices");
    pl.desc.assign(n, SliceDesc{});
    return plan_into(sl, n, base, cfg, pl.hdr, pl.desc.data(), pl.bytes, pl.max_pmt, pl.smem_dt, pl.any_wide,
                     &pl.shape, ev, &pl.any_events);
}

extern "C" size_t trig_batch_scratch_bytes(const trig_slice_dev *slices, uint32_t n_slices)
{
    Plan pl;
    if (make_plan(slices, n_slices, 0, current_cfg(), pl, false)) return 0;
    return pl.bytes;
}

extern "C" size_t trig_batch_events_scratch_bytes(const trig_slice_dev *slices, const trig_slice_events *events,
                                                  uint32_t n_slices)
{
    Plan pl;
    if (make_plan(slices, n_slices, 0, current_cfg(), pl, false, events)) return 0;
    return pl.bytes;
}

static void pack_plan(const Plan &pl, std::vector<unsigned char> &buf)
{
    const size_t desc_off = align256(sizeof(BatchHeader));
    buf.assign(desc_off + sizeof(SliceDesc) * pl.desc.size(), 0);
    std::memcpy(buf.data(), &pl.hdr, sizeof(BatchHeader));
    std::memcpy(buf.data() + desc_off, pl.desc.data(), sizeof(SliceDesc) * pl.desc.size());
}

// ------------------------------------------------------------ graph cache

// A graph is replayed only for the plan it was captured with: the same
// stream, scratch and descriptor bytes (so the same slices, buffers and
// tile shape).  A repeated batch (a fixed set of resident slices run again
// and again) replays its graph; a new batch captures a new one.  At most
// kMaxGraphs are kept, the least recently used is dropped.
struct GraphKey {
    cudaStream_t stream;
    uintptr_t scratch;
    uint64_t plan_hash;
    size_t plan_bytes;
    bool operator<(const GraphKey &o) const
    {
        return std::tie(stream, scratch, plan_hash, plan_bytes) < std::tie(o.stream, o.scratch, o.plan_hash, o.plan_bytes);
    }
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    unsigned char *pinned = nullptr;     // header + descriptors, copied by the graph's first node
    std::vector<unsigned char> plan;     // the plan bytes (hash collisions are checked against it)
    cudaEvent_t done = nullptr;          // last replay finished
    bool launched = false;
    uint64_t last_use = 0;
    uint64_t launches = 0;               // kernels per replay
};

constexpr size_t kMaxGraphs = 64;
static std::mutex g_graph_mu;
static std::map<GraphKey, GraphEntry> g_graphs;
static uint64_t g_graph_clock = 0;

static uint64_t fnv1a(const unsigned char *p, size_t n)
{
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) h = (h ^ p[i]) * 1099511628211ull;
    return h;
}

static void drop_graph(GraphEntry &ge)
{
    if (ge.launched) cudaEventSynchronize(ge.done);
    if (ge.exec) cudaGraphExecDestroy(ge.exec);
    if (ge.done) cudaEventDestroy(ge.done);
    if (ge.pinned) cudaFreeHost(ge.pinned);
    ge = GraphEntry{};
}

static int run_graph(const Plan &pl, void *scratch, cudaStream_t st)
{
    const TileConfig &cfg = pl.shape;
    std::vector<unsigned char> host;
    pack_plan(pl, host);
    GraphKey key{st, (uintptr_t)scratch, fnv1a(host.data(), host.size()), host.size()};
    std::lock_guard<std::mutex> lk(g_graph_mu);
    auto found = g_graphs.find(key);
    if (found != g_graphs.end() && found->second.plan != host) {
        drop_graph(found->second);          // hash collision: recapture
        g_graphs.erase(found);
        found = g_graphs.end();
    }
    if (found == g_graphs.end() && g_graphs.size() >= kMaxGraphs) {
        auto lru = g_graphs.begin();
        for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it)
            if (it->second.last_use < lru->second.last_use) lru = it;
        drop_graph(lru->second);
        g_graphs.erase(lru);
    }
    GraphEntry &ge = g_graphs[key];
    ge.last_use = ++g_graph_clock;
    cudaError_t e;
    if (!ge.exec) {
        auto forget = [&](int rc) {
            drop_graph(ge);
            g_graphs.erase(key);
            return rc;
        };
        if ((e = cudaMallocHost(&ge.pinned, host.size()))) return forget(cuda_fail(e, "graph: pinned descriptors"));
        if ((e = cudaEventCreateWithFlags(&ge.done, cudaEventDisableTiming))) return forget(cuda_fail(e, "graph: event"));
        std::memcpy(ge.pinned, host.data(), host.size());
        ge.plan = host;
        // capture on a private stream (the caller's may be the legacy default
        // stream, which cannot capture); replays go to the caller's stream
        cudaGraph_t graph;
        cudaStream_t cap;
        if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking))) return forget(cuda_fail(e, "graph: stream"));
        if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal))) {
            cudaStreamDestroy(cap);
            return forget(cuda_fail(e, "graph: capture"));
        }
        uint64_t nl = 0;
        cudaError_t ce = cudaMemcpyAsync(scratch, ge.pinned, host.size(), cudaMemcpyHostToDevice, cap);
        if (!ce)
            ce = launch_batch(reinterpret_cast<BatchHeader *>(scratch),
                              reinterpret_cast<SliceDesc *>((char *)scratch + align256(sizeof(BatchHeader))),
                              pl.hdr.n_slices, pl.max_pmt, pl.smem_dt, pl.any_wide, pl.any_events,
                              pl.hdr.any_ext != 0, pl.hdr.dense != 0, cfg, cap, &nl,
                              false);
        ge.launches = nl;
        e = cudaStreamEndCapture(cap, &graph);
        cudaStreamDestroy(cap);
        if (ce) {
            if (!e) cudaGraphDestroy(graph);
            return forget(cuda_fail(ce, "graph: capture launch"));
        }
        if (e) return forget(cuda_fail(e, "graph: end capture"));
        e = cudaGraphInstantiate(&ge.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e) {
            ge.exec = nullptr;
            return forget(cuda_fail(e, "graph: instantiate"));
        }
    }
    // a replay reads the same descriptor bytes as the previous one, so it
    // need not wait for it: stream order serialises the two
    if ((e = cudaGraphLaunch(ge.exec, st))) return cuda_fail(e, "graph: launch");
    if ((e = cudaEventRecord(ge.done, st))) return cuda_fail(e, "graph: record");
    ge.launched = true;
    g_launches += ge.launches;
    return TRIG_OK;
}

// ------------------------------------------------------- kernel timing

struct TimedRun {
    cudaEvent_t ev[kPipelineKernels + 1];
};

static std::mutex g_time_mu;
static std::vector<TimedRun> g_time_pending, g_time_free;

static int timed_events(TimedRun &tr)
{
    std::lock_guard<std::mutex> lk(g_time_mu);
    if (!g_time_free.empty()) {
        tr = g_time_free.back();
        g_time_free.pop_back();
        return TRIG_OK;
    }
    for (auto &e : tr.ev) {
        cudaError_t c = cudaEventCreate(&e);
        if (c) return cuda_fail(c, "timing events");
    }
    return TRIG_OK;
}

extern "C" int trig_kernel_times(double *avg_ms, const char **names, uint32_t max_kernels, uint32_t *n_runs)
{
    std::vector<TimedRun> runs;
    {
        std::lock_guard<std::mutex> lk(g_time_mu);
        runs.swap(g_time_pending);
    }
    double acc[kPipelineKernels] = {};
    for (auto &r : runs) {
        cudaError_t e = cudaEventSynchronize(r.ev[kPipelineKernels]);
        if (e) return cuda_fail(e, "trig_kernel_times");
        for (int i = 0; i < kPipelineKernels; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, r.ev[i], r.ev[i + 1]);
            acc[i] += ms;
        }
    }
    for (uint32_t i = 0; i < (uint32_t)kPipelineKernels && i < max_kernels; ++i) {
        if (avg_ms) avg_ms[i] = runs.empty() ? 0.0 : acc[i] / (double)runs.size();
        if (names) names[i] = kKernelNames[i];
    }
    if (n_runs) *n_runs = (uint32_t)runs.size();
    std::lock_guard<std::mutex> lk(g_time_mu);
    for (auto &r : runs) g_time_free.push_back(r);
    return kPipelineKernels;
}

static int run_plan(const Plan &pl, void *scratch, size_t scratch_bytes, cudaStream_t st, uint32_t flags, bool rows)
{
    const TileConfig &cfg = pl.shape;
    if (!scratch || ((uintptr_t)scratch & 255u)) return fail(TRIG_EINVAL, "scratch must be 256-byte aligned device memory");
    if (scratch_bytes < pl.bytes) return fail(TRIG_EINVAL, "scratch too small (see trig_batch_scratch_bytes)");
    if ((flags & TRIG_RUN_GRAPH) && (flags & TRIG_RUN_TIMED)) return fail(TRIG_EINVAL, "TIMED runs cannot use GRAPH");
    if ((flags & TRIG_RUN_GRAPH) && !rows) return run_graph(pl, scratch, st);
    std::vector<unsigned char> host;
    pack_plan(pl, host);
    cudaError_t e = cudaMemcpyAsync(scratch, host.data(), host.size(), cudaMemcpyHostToDevice, st);
    if (e) return cuda_fail(e, "copy descriptors");
    TimedRun tr{};
    const bool timed = (flags & TRIG_RUN_TIMED) && !rows;
    if (timed) {
        int rc = timed_events(tr);
        if (rc) return rc;
    }
    uint64_t nl = 0;
    e = launch_batch(reinterpret_cast<BatchHeader *>(scratch),
                     reinterpret_cast<SliceDesc *>((char *)scratch + align256(sizeof(BatchHeader))), pl.hdr.n_slices,
                     pl.max_pmt, pl.smem_dt, pl.any_wide, pl.any_events, pl.hdr.any_ext != 0, pl.hdr.dense != 0, cfg,
                     st, &nl, rows,
                     timed ? tr.ev : nullptr);
    g_launches += nl;
    if (timed) {
        std::lock_guard<std::mutex> lk(g_time_mu);
        g_time_pending.push_back(tr);
    }
    if (e) return cuda_fail(e, "launch");
    return TRIG_OK;
}

extern "C" int trig_batch_run_events(const trig_slice_dev *slices, const trig_slice_events *events,
                                     uint32_t n_slices, void *scratch, size_t scratch_bytes, void *stream,
                                     uint32_t flags)
{
    if (!events) return fail(TRIG_EINVAL, "events is NULL");
    const TileConfig cfg = current_cfg();
    Plan pl;
    int rc = make_plan(slices, n_slices, (uintptr_t)scratch, cfg, pl, false, events);
    if (rc) return rc;
    return run_plan(pl, scratch, scratch_bytes, (cudaStream_t)stream, flags, false);
}

extern "C" int trig_batch_run(const trig_slice_dev *slices, uint32_t n_slices, void *scratch, size_t scratch_bytes,
                              void *stream, uint32_t flags)
{
    const TileConfig cfg = current_cfg();
    Plan pl;
    int rc = make_plan(slices, n_slices, (uintptr_t)scratch, cfg, pl, false);
    if (rc) return rc;
    return run_plan(pl, scratch, scratch_bytes, (cudaStream_t)stream, flags, false);
}

extern "C" int trig_slice_rows(const trig_slice_dev *slice, trig_hit *merged_out, uint32_t *seedcnt_out,
                               uint64_t *n_owned_out, void *scratch, size_t scratch_bytes, void *stream)
{
    if (!slice || !merged_out || !seedcnt_out || !n_owned_out) return fail(TRIG_EINVAL, "NULL argument");
    const TileConfig cfg = current_cfg();
    Plan pl;
    int rc = make_plan(slice, 1, (uintptr_t)scratch, cfg, pl, true);
    if (rc) return rc;
    pl.desc[0].dbg_merged = merged_out;
    pl.desc[0].dbg_seedcnt = seedcnt_out;
    cudaStream_t st = (cudaStream_t)stream;
    rc = run_plan(pl, scratch, scratch_bytes, st, 0, true);
    if (rc) return rc;
    SliceDesc back;
    cudaError_t e = cudaMemcpyAsync(&back, (char *)scratch + align256(sizeof(BatchHeader)), sizeof(SliceDesc),
                                    cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return cuda_fail(e, "trig_slice_rows");
    // k_rank0 stored the merged ranks of t0 and t0 + S
    *n_owned_out = back.dbg_rank1 - back.dbg_rank0;
    return TRIG_OK;
}

// ------------------------------------------------------------- autotuner

static std::string gpu_name()
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string n = prop.name;
    for (auto &c : n)
        if (c == ' ' || c == '\t') c = '_';
    return n;
}

// Cache file (path in TRIG_TUNE_CACHE): one line per (GPU, PMT count):
// "<gpu> <n_pmt> <cap> <warps> <fill_pct> <ms>".
static bool tune_cache_lookup(uint32_t n_pmt, TileConfig &out)
{
    const char *path = std::getenv("TRIG_TUNE_CACHE");
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    const std::string gpu = gpu_name();
    char g[256];
    unsigned p, c, w, fl;
    double ms;
    bool found = false;
    while (std::fscanf(f, "%255s %u %u %u %u %lf", g, &p, &c, &w, &fl, &ms) == 6)
        if (gpu == g && p == n_pmt && valid_tile_shape(c, w)) {
            out = TileConfig{c, w, fl};
            found = true;
        }
    std::fclose(f);
    return found;
}

static void tune_cache_store(uint32_t n_pmt, const TileConfig &cfg, double ms)
{
    const char *path = std::getenv("TRIG_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %u %u %u %u %.6f\n", gpu_name().c_str(), n_pmt, cfg.cap, cfg.warps, cfg.fill_pct, ms);
    std::fclose(f);
}

// Times every candidate launch shape on the given slices of one detector
// and keeps the fastest for that detector: the tile capacity, consumer
// warps per block and tile fill that suit its PMT count and rate.
extern "C" int trig_autotune(trig_detector *det, const trig_slice_dev *slices, uint32_t n_slices, void *stream,
                             trig_tune_result *out)
{
    if (!det || !slices || n_slices == 0) return fail(TRIG_EINVAL, "trig_autotune: NULL argument");
    for (uint32_t s = 0; s < n_slices; ++s)
        if (slices[s].det != det) return fail(TRIG_EINVAL, "trig_autotune: all slices must belong to det");
    static const uint32_t shapes[][2] = {{4096, 16}, {4096, 8}, {2048, 16}, {2048, 8}, {1024, 4}};
    static const uint32_t fills[] = {55, 75, 90, 95};
    cudaStream_t st = (cudaStream_t)stream;
    // scratch for the largest candidate
    const bool was_tuned = det->tuned;
    const TileConfig was = det->tile;
    size_t need = 0;
    for (auto &sh : shapes)
        for (uint32_t f : fills) {
            det->tuned = true;
            det->tile = TileConfig{sh[0], sh[1], f};
            need = std::max(need, trig_batch_scratch_bytes(slices, n_slices));
        }
    det->tuned = was_tuned;
    det->tile = was;
    if (!need) return fail(TRIG_EINVAL, "trig_autotune: cannot plan these slices");
    void *scratch = nullptr;
    cudaError_t e = cudaMalloc(&scratch, need);
    if (e) return cuda_fail(e, "trig_autotune: scratch");
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    TileConfig best{};
    double best_ms = 1e30;
    uint32_t tried = 0;
    int rc = TRIG_OK;
    for (auto &sh : shapes) {
        for (uint32_t f : fills) {
            det->tuned = true;
            det->tile = TileConfig{sh[0], sh[1], f};
            rc = trig_batch_run(slices, n_slices, scratch, need, stream, 0);       // warm-up
            if (rc) break;
            cudaEventRecord(a, st);
            for (int r = 0; r < 3 && !rc; ++r) rc = trig_batch_run(slices, n_slices, scratch, need, stream, 0);
            cudaEventRecord(b, st);
            if (rc) break;
            e = cudaEventSynchronize(b);
            if (e) {
                rc = cuda_fail(e, "trig_autotune: timing");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            ms /= 3.f;
            ++tried;
            if (ms < best_ms) {
                best_ms = ms;
                best = det->tile;
            }
        }
        if (rc) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(scratch);
    if (rc || !tried) {
        det->tuned = was_tuned;
        det->tile = was;
        return rc ? rc : fail(TRIG_EDEVICE, "trig_autotune: nothing timed");
    }
    det->tuned = true;
    det->tile = best;
    tune_cache_store(det->n_pmt, best, best_ms);
    if (out) {
        out->cap = best.cap;
        out->warps = best.warps;
        out->fill_pct = best.fill_pct;
        out->n_tried = tried;
        out->ms = best_ms;
    }
    return TRIG_OK;
}

extern "C" int trig_detector_tile_config(const trig_detector *det, uint32_t *cap, uint32_t *warps, uint32_t *fill_pct)
{
    if (!det) return fail(TRIG_EINVAL, "NULL detector");
    const TileConfig c = det->tuned ? det->tile : current_cfg();
    if (cap) *cap = c.cap;
    if (warps) *warps = c.warps;
    if (fill_pct) *fill_pct = c.fill_pct;
    return det->tuned ? 1 : 0;
}

// ------------------------------------------------- no-allocation batch

// Callers on a DAQ node's real-time path, or threads running while another
// thread captures a CUDA graph in global mode, must not call cudaMalloc (it
// can synchronise the device and stall the other streams, and it is
// refused during global capture).  This entry point runs a batch in a
// static device array compiled into the library instead of caller scratch.
extern "C" int trig_batch_run_noalloc(const trig_slice_dev *slices, uint32_t n_slices, void *stream)
{
    if (!slices || n_slices == 0 || n_slices > TRIG_NOALLOC_MAX_SLICES)
        return fail(TRIG_EINVAL, "trig_batch_run_noalloc: 1 to TRIG_NOALLOC_MAX_SLICES slices");
    cudaStream_t st = (cudaStream_t)stream;
    // the legacy default stream synchronises with every blocking stream,
    // and another thread's global-mode capture forbids its use
    if (st == nullptr || st == cudaStreamLegacy)
        return fail(TRIG_EINVAL, "trig_batch_run_noalloc: pass a stream created with cudaStreamNonBlocking");
    // the shared static array would be baked into a graph and raced by
    // every replay: the call is not for capture
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap_status);
    if (e) return cuda_fail(e, "trig_batch_run_noalloc: stream capture status");
    if (cap_status != cudaStreamCaptureStatusNone)
        return fail(TRIG_EINVAL, "trig_batch_run_noalloc: the stream is capturing; this call must not be captured");
    void *scratch = nullptr;
    size_t cap = 0;
    e = static_scratch(&scratch, &cap);
    if (e) return cuda_fail(e, "trig_batch_run_noalloc: static scratch address");
    const TileConfig cfg = current_cfg();
    NoallocPlan plan;
    size_t bytes = 0;
    uint32_t max_pmt = 0;
    bool smem_dt = true, any_wide = false;
    TileConfig shape{};
    int rc = plan_into(slices, n_slices, (uintptr_t)scratch, cfg, plan.hdr, plan.desc, bytes, max_pmt, smem_dt,
                       any_wide, &shape);
    if (rc) return rc;
    if (bytes > cap) return fail(TRIG_ECAPACITY, "trig_batch_run_noalloc: batch needs more than TRIG_NOALLOC_SCRATCH_BYTES of scratch");
    plan.n = n_slices;
    BatchHeader *d_hdr = reinterpret_cast<BatchHeader *>(scratch);
    SliceDesc *d_desc = reinterpret_cast<SliceDesc *>((char *)scratch + align256(sizeof(BatchHeader)));
    e = launch_put_plan(plan, d_hdr, d_desc, st);
    if (e) return cuda_fail(e, "trig_batch_run_noalloc: descriptors");
    uint64_t nl = 1;
    e = launch_batch(d_hdr, d_desc, n_slices, max_pmt, smem_dt, any_wide, false, plan.hdr.any_ext != 0,
                     plan.hdr.dense != 0, shape, st, &nl, false);
    g_launches += nl;
    if (e) return cuda_fail(e, "trig_batch_run_noalloc: launch");
    return TRIG_OK;
}

// ================================================================ engine

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
    trig_detector *det = nullptr;
    std::shared_ptr<DetQueue> q;
    uint64_t id = 0;
    int64_t t0 = 0;
    unsigned char *dblk = nullptr;       // device copy: hits, then pmt_off at pmt_at
    size_t dbytes = 0;
    size_t pmt_at = 0;
    uint64_t n_hits = 0;
    Clock::time_point t_submit;
    Clock::time_point t_queued;         // copied to the device and queued
    uint32_t copy_wait_us = 0;          // of that, waiting for the copies after the host work
    bool continuation = false;
};

// Device blocks for submitted slices, in power-of-two size classes and
// reused once their batch completes.  Growth keeps a reserve of free
// device memory (2 % of the total) for the slot arenas; idle blocks of
// other classes are released first when the limit is reached.
struct DevicePool {
    std::mutex mu;
    std::multimap<size_t, unsigned char *> free_blocks;
    size_t used = 0;
    size_t in_use = 0;              // bytes of blocks handed out and not yet returned
    size_t limit = 0;               // 0: no limit beyond free device memory
    unsigned char *get(size_t bytes, size_t *got)
    {
        size_t cls = (size_t)1 << 16;
        while (cls < bytes) cls <<= 1;
        std::lock_guard<std::mutex> lk(mu);
        if (limit && in_use + cls > limit) return nullptr;
        // the smallest free block that fits, up to four classes larger
        auto it = free_blocks.lower_bound(cls);
        if (it != free_blocks.end() && it->first <= 4 * cls) {
            unsigned char *p = it->second;
            *got = it->first;
            in_use += it->first;
            free_blocks.erase(it);
            return p;
        }
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        const size_t reserve = total_b / 50;
        for (auto f = free_blocks.begin(); f != free_blocks.end() && free_b < cls + reserve;) {
            cudaFree(f->second);
            used -= f->first;
            free_b += f->first;
            f = free_blocks.erase(f);
        }
        if (free_b < cls + reserve) return nullptr;
        void *p = nullptr;
        if (cudaMalloc(&p, cls) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        used += cls;
        in_use += cls;
        *got = cls;
        return static_cast<unsigned char *>(p);
    }
    void put(unsigned char *p, size_t cls)
    {
        std::lock_guard<std::mutex> lk(mu);
        in_use -= cls;
        free_blocks.emplace(cls, p);
    }
};

// Pinned host blocks that results are read back into (the device-to-host
// copy lands where the caller reads it), in power-of-two size classes,
// returned by trig_result_free; at most 24 GB.
struct HostPool {
    std::mutex mu;
    std::multimap<size_t, unsigned char *> free_blocks;
    size_t used = 0, limit = (size_t)24 << 30;
    uint32_t fail_next = 0;         // failure injection: the next n requests fail
    unsigned char *get(size_t bytes, size_t *got)
    {
        size_t cls = 4096;
        while (cls < bytes) cls <<= 1;
        std::lock_guard<std::mutex> lk(mu);
        if (fail_next) {
            --fail_next;
            return nullptr;
        }
        // the smallest free block that fits, up to four classes larger: a
        // new page-locked allocation stalls the engine thread for
        // milliseconds
        auto it = free_blocks.lower_bound(cls);
        if (it != free_blocks.end() && it->first <= 4 * cls) {
            unsigned char *p = it->second;
            *got = it->first;
            free_blocks.erase(it);
            return p;
        }
        for (auto f = free_blocks.begin(); f != free_blocks.end() && used + cls > limit;) {
            cudaFreeHost(f->second);
            used -= f->first;
            f = free_blocks.erase(f);
        }
        if (used + cls > limit) return nullptr;
        void *p = nullptr;
        if (cudaMallocHost(&p, cls) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        used += cls;
        *got = cls;
        return static_cast<unsigned char *>(p);
    }
    void put(unsigned char *p, size_t cls)
    {
        std::lock_guard<std::mutex> lk(mu);
        free_blocks.emplace(cls, p);
    }
};

// A result and the pinned block its arrays live in (NULL for results
// without arrays); trig_result_free returns the block to its pool.
struct ResultBox {
    trig_result pub;
    HostPool *pool;
    unsigned char *blk;
    size_t cls;
};

trig_result *new_result(uint64_t id, int64_t t0, int32_t status)
{
    ResultBox *b = static_cast<ResultBox *>(std::calloc(1, sizeof(ResultBox)));
    if (!b) return nullptr;
    b->pub.slice_id = id;
    b->pub.t0_ns = t0;
    b->pub.status = status;
    return &b->pub;
}


}  // namespace



namespace {

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_stats = nullptr, ev_done = nullptr;
    cudaEvent_t ev_launch = nullptr;                // timing events around the batch's kernels
    uint64_t batch_id = 0;
    Clock::time_point t_launch, t_stats;
    void *arena = nullptr;
    size_t arena_bytes = 0;
    unsigned char *bounce = nullptr;                // pinned: stats + outputs
    size_t bounce_bytes = 0;
    int state = 0;                                  // 0 idle, 1 computing, 2 copying back
    std::vector<Pending> slices;
    std::vector<size_t> out_off;                    // per slice offset of its triggers in its block
    std::vector<trig_slice_dev> dev;
    std::vector<uint64_t> trig_n, win_n;
    std::vector<size_t> win_off;                    // per slice offset of its windows in its block
    std::vector<size_t> ev_off;                     // per slice offset of its events in its block
    std::vector<unsigned char *> rblk;              // per slice pinned result block (NULL: none)
    std::vector<size_t> rcls;
    std::vector<trig_slice_events> evs;             // per slice event output (ev_cap 0: none)
    std::vector<uint64_t> ev_n;
    std::vector<uint8_t> lost;                      // per slice: no result block, outputs dropped
};

constexpr int kSlots = 3;
constexpr uint32_t kMaxBatchSlices = 256;

struct Engine {
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Pending> pending;
    Slot slots[kSlots];
    DevicePool pool;
    HostPool rpool;
    std::thread worker;
    bool stop = false;
    bool hold = false;              // admit no new batch while set
    int mode = 1;
    std::atomic<uint64_t> next_id{1};
    std::atomic<uint64_t> batches{0}, completed{0};
    // per-slice trace (trig_engine_trace): records of completed slices
    std::mutex trace_mu;
    std::vector<trig_trace_rec> trace;
    size_t trace_cap = 0;
    Clock::time_point trace_t0;
    bool started = false;
    std::string fatal;

    int start()
    {
        cudaGetDevice(&device);
        for (auto &s : slots) {
            cudaError_t e;
            if ((e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking)) ||
                (e = cudaEventCreate(&s.ev_stats)) || (e = cudaEventCreate(&s.ev_launch)) ||
                (e = cudaEventCreateWithFlags(&s.ev_done, cudaEventDisableTiming)))
                return cuda_fail(e, "engine start");
        }
        worker = std::thread([this] { run(); });
        started = true;
        return TRIG_OK;
    }

    void shutdown()
    {
        {
            std::lock_guard<std::mutex> lk(mu);
            stop = true;
        }
        cv.notify_all();
        if (worker.joinable()) worker.join();
    }

    void run();
    void fail_slot(Slot &s, cudaError_t err);
    bool launch_batch_on(Slot &s, std::vector<Pending> &batch);
    void collect_stats(Slot &s);
    void finish(Slot &s);
};

Engine *g_engine = nullptr;
std::mutex g_engine_mu;

void engine_atexit()
{
    std::lock_guard<std::mutex> lk(g_engine_mu);
    if (g_engine) g_engine->shutdown();
}

Engine *engine()
{
    std::lock_guard<std::mutex> lk(g_engine_mu);
    if (!g_engine) {
        Engine *e = new Engine();
        if (e->start()) {
            delete e;
            return nullptr;
        }
        g_engine = e;
        std::atexit(engine_atexit);
    }
    return g_engine;
}

uint64_t win_cap_for(const trig_detector *det)
{
    const int64_t h = det->par.win_half_ns;
    return (uint64_t)((det->par.slice_ns + 2 * h) / (2 * h + 2)) + 2;
}

// Device footprint of a batch in one arena: outputs, stats, events, scratch
// (the inputs stay in the submissions' device blocks).
struct ArenaLayout {
    size_t bytes = 0;
    std::vector<size_t> trig, win, stats, ev;
    size_t scratch = 0, scratch_bytes = 0;
};

}  // namespace

bool Engine::launch_batch_on(Slot &s, std::vector<Pending> &batch)
{
    // layout of the arena: the outputs of every slice, then the batch
    // scratch
    const uint32_t n = (uint32_t)batch.size();
    std::vector<trig_slice_dev> dev(n);
    ArenaLayout L;
    size_t off = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const Pending &p = batch[i];
        const uint32_t P = p.det->n_pmt;
        dev[i].det = p.det;
        dev[i].n_hits = p.n_hits;
        dev[i].t0_ns = p.t0;
        dev[i].trig_cap = std::max<uint64_t>(p.n_hits, 1);
        dev[i].win_cap = win_cap_for(p.det);
        // placeholder pointers for sizing (the real ones are set below)
        // the inputs are the submission's device copy
        dev[i].hits = reinterpret_cast<const trig_hit *>(p.dblk);
        dev[i].pmt_off = reinterpret_cast<const uint64_t *>(p.dblk + p.pmt_at);
        dev[i].triggers = reinterpret_cast<trig_trigger *>(256);
        dev[i].windows = reinterpret_cast<trig_window *>(256);
        dev[i].stats = reinterpret_cast<trig_slice_stats *>(256);
        (void)P;
        L.trig.push_back(off);
        off += align256(dev[i].trig_cap * sizeof(trig_trigger));
        L.win.push_back(off);
        off += align256(dev[i].win_cap * sizeof(trig_window));
        L.stats.push_back(off);
        off += align256(sizeof(trig_slice_stats));
        L.ev.push_back(off);
        if (p.det->events) off += align256(std::max<uint64_t>(p.n_hits, 1) * sizeof(trig_hit));
    }
    // event outputs (placeholders for sizing; the real pointers are set below)
    std::vector<trig_slice_events> evs(n);
    bool any_ev = false;
    for (uint32_t i = 0; i < n; ++i) {
        if (!batch[i].det->events) continue;
        any_ev = true;
        evs[i].events = reinterpret_cast<trig_hit *>(256);
        evs[i].ev_cap = std::max<uint64_t>(batch[i].n_hits, 1);
    }
    L.scratch = off;
    L.scratch_bytes = any_ev ? trig_batch_events_scratch_bytes(dev.data(), evs.data(), n)
                             : trig_batch_scratch_bytes(dev.data(), n);
    if (!L.scratch_bytes) {
        fatal = g_last_error;
        return false;
    }
    off += align256(L.scratch_bytes);
    L.bytes = off;
    // grow the arena when needed (geometrically, so a serving mix settles
    // after a few batches); admission: the device must have the memory,
    // keeping a reserve, else the batch waits for other slots to finish
    if (s.arena_bytes < L.bytes) {
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        const size_t reserve = total_b / 50;
        size_t want = std::max(L.bytes, s.arena_bytes + s.arena_bytes / 2);
        if (want > free_b + s.arena_bytes - std::min(free_b + s.arena_bytes, reserve)) want = L.bytes;
        if (L.bytes + reserve > free_b + s.arena_bytes) return false;
        if (s.arena) cudaFree(s.arena);
        s.arena = nullptr;
        s.arena_bytes = 0;
        if (cudaMalloc(&s.arena, want) != cudaSuccess) {
            (void)cudaGetLastError();
            if (cudaMalloc(&s.arena, L.bytes) != cudaSuccess) {
                (void)cudaGetLastError();
                return false;
            }
            want = L.bytes;
        }
        s.arena_bytes = want;
    }
    char *A = static_cast<char *>(s.arena);
    s.out_off.assign(n, 0);
    for (uint32_t i = 0; i < n; ++i) {
        dev[i].triggers = reinterpret_cast<trig_trigger *>(A + L.trig[i]);
        dev[i].windows = reinterpret_cast<trig_window *>(A + L.win[i]);
        dev[i].stats = reinterpret_cast<trig_slice_stats *>(A + L.stats[i]);
        if (evs[i].ev_cap) evs[i].events = reinterpret_cast<trig_hit *>(A + L.ev[i]);
    }
    // the pinned bounce buffer takes the per-slice counters now, and the
    // triggers and windows (by their actual counts) once those are known
    const size_t stats_off = 0;
    const size_t bounce_need = align256(n * sizeof(trig_slice_stats));
    if (s.bounce_bytes < bounce_need) {
        if (s.bounce) cudaFreeHost(s.bounce);
        s.bounce = nullptr;
        s.bounce_bytes = 0;
        void *p = nullptr;
        const size_t want = std::max(bounce_need, s.bounce_bytes + s.bounce_bytes / 2);
        if (cudaMallocHost(&p, want) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        s.bounce = static_cast<unsigned char *>(p);
        s.bounce_bytes = want;
    }
    // run, stats back
    cudaError_t e = cudaSuccess;
    // batches of the engine vary in size and composition from one launch
    // to the next, so they are launched directly rather than from graphs
    s.t_launch = Clock::now();
    cudaEventRecord(s.ev_launch, s.stream);
    int rc = any_ev ? trig_batch_run_events(dev.data(), evs.data(), n, A + L.scratch, L.scratch_bytes, s.stream, 0)
                    : trig_batch_run(dev.data(), n, A + L.scratch, L.scratch_bytes, s.stream, 0);
    if (rc) {
        fatal = g_last_error;
        return false;
    }
    for (uint32_t i = 0; i < n && !e; ++i)
        e = cudaMemcpyAsync(s.bounce + stats_off + i * sizeof(trig_slice_stats), dev[i].stats,
                            sizeof(trig_slice_stats), cudaMemcpyDeviceToHost, s.stream);
    if (!e) e = cudaEventRecord(s.ev_stats, s.stream);
    if (e) {
        fatal = cudaGetErrorString(e);
        (void)cudaGetLastError();
        return false;
    }
    s.slices = std::move(batch);
    s.dev = std::move(dev);
    s.evs = std::move(evs);
    s.state = 1;
    s.trig_n.assign(n, 0);
    s.win_n.assign(n, 0);
    s.batch_id = ++batches;
    return true;
}

// A device error: deliver EDEVICE results for the slot's slices (their
// staging memory is not reused, the device may still reference it) and
// leave the slot idle.
void Engine::fail_slot(Slot &s, cudaError_t err)
{
    std::fprintf(stderr, "trig engine: batch failed: %s\n", cudaGetErrorString(err));
    (void)cudaGetLastError();
    for (auto &p : s.slices) {
        trig_result *r = new_result(p.id, p.t0, TRIG_EDEVICE);
        std::lock_guard<std::mutex> lk(p.q->mu);
        p.q->done[p.id] = r;
        p.q->in_flight--;
        p.q->cv.notify_all();
    }
    s.slices.clear();
    s.state = 0;
}

void Engine::collect_stats(Slot &s)
{
    s.t_stats = Clock::now();
    const uint32_t n = (uint32_t)s.slices.size();
    const trig_slice_stats *st = reinterpret_cast<const trig_slice_stats *>(s.bounce);
    // per slice one pinned block sized by the actual counts: triggers,
    // windows, events
    s.out_off.assign(n, 0);
    s.win_off.assign(n, 0);
    s.ev_off.assign(n, 0);
    s.rblk.assign(n, nullptr);
    s.rcls.assign(n, 0);
    s.lost.assign(n, 0);
    s.ev_n.assign(n, 0);
    cudaError_t e = cudaSuccess;
    for (uint32_t i = 0; i < n && !e; ++i) {
        s.trig_n[i] = std::min<uint64_t>(st[i].n_triggers, s.dev[i].trig_cap);
        s.win_n[i] = std::min<uint64_t>(st[i].n_windows, s.dev[i].win_cap);
        if (s.evs[i].ev_cap && !(st[i].flags & TRIG_FLAG_EV_FULL))
            s.ev_n[i] = std::min<uint64_t>(st[i].n_events, s.evs[i].ev_cap);
        const size_t tb = align256(s.trig_n[i] * sizeof(trig_trigger));
        const size_t wb = align256(s.win_n[i] * sizeof(trig_window));
        const size_t eb = s.ev_n[i] * sizeof(trig_hit);
        s.win_off[i] = tb;
        s.ev_off[i] = tb + wb;
        if (tb + wb + eb == 0) continue;
        s.rblk[i] = rpool.get(tb + wb + eb, &s.rcls[i]);
        if (!s.rblk[i]) {
            s.lost[i] = 1;
            s.trig_n[i] = s.win_n[i] = s.ev_n[i] = 0;
            continue;
        }
        if (s.trig_n[i])
            e = cudaMemcpyAsync(s.rblk[i], s.dev[i].triggers, s.trig_n[i] * sizeof(trig_trigger),
                                cudaMemcpyDeviceToHost, s.stream);
        if (!e && s.win_n[i])
            e = cudaMemcpyAsync(s.rblk[i] + tb, s.dev[i].windows, s.win_n[i] * sizeof(trig_window),
                                cudaMemcpyDeviceToHost, s.stream);
        if (!e && s.ev_n[i])
            e = cudaMemcpyAsync(s.rblk[i] + tb + wb, s.evs[i].events, eb, cudaMemcpyDeviceToHost, s.stream);
    }
    if (!e) e = cudaEventRecord(s.ev_done, s.stream);
    if (e) {
        fatal = cudaGetErrorString(e);
        (void)cudaGetLastError();
    }
    s.state = 2;
}

void Engine::finish(Slot &s)
{
    const uint32_t n = (uint32_t)s.slices.size();
    const trig_slice_stats *st = reinterpret_cast<const trig_slice_stats *>(s.bounce);
    const auto now = Clock::now();
    {
        std::lock_guard<std::mutex> tk(trace_mu);
        if (trace.size() < trace_cap) {
            float dev_ms = -1.f;
            if (cudaEventElapsedTime(&dev_ms, s.ev_launch, s.ev_stats) != cudaSuccess) {
                (void)cudaGetLastError();
                dev_ms = -1.f;
            }
            auto ns = [&](Clock::time_point t) {
                return (int64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(t - trace_t0).count();
            };
            for (uint32_t i = 0; i < n && trace.size() < trace_cap; ++i) {
                const Pending &p = s.slices[i];
                trig_trace_rec t{};
                t.slice_id = p.id;
                t.batch = s.batch_id;
                t.batch_slices = n;
                t.n_pmt = p.det->n_pmt;
                t.n_hits = p.n_hits;
                t.status = s.lost[i] ? TRIG_ENOMEM : st[i].status;
                t.continuation = p.continuation ? 1u : 0u;
                t.t_submit_ns = ns(p.t_submit);
                t.t_queued_ns = ns(p.t_queued);
                t.t_launch_ns = ns(s.t_launch);
                t.t_stats_ns = ns(s.t_stats);
                t.t_done_ns = ns(now);
                t.device_ms = dev_ms;
                t.copy_wait_us = p.copy_wait_us;
                trace.push_back(t);
            }
        }
    }
    for (uint32_t i = 0; i < n; ++i) {
        Pending &p = s.slices[i];
        trig_result *r = new_result(p.id, p.t0, s.lost[i] ? TRIG_ENOMEM : st[i].status);
        if (r) {
            ResultBox *box = reinterpret_cast<ResultBox *>(r);
            r->flags = st[i].flags;
            r->n_hits = st[i].n_hits;
            r->n_seeds = st[i].n_seeds;
            r->n_triggers = s.trig_n[i];
            r->n_windows = s.win_n[i];
            if (s.rblk[i]) {
                box->pool = &rpool;
                box->blk = s.rblk[i];
                box->cls = s.rcls[i];
                if (r->n_triggers) r->triggers = reinterpret_cast<trig_trigger *>(s.rblk[i]);
                if (r->n_windows) r->windows = reinterpret_cast<trig_window *>(s.rblk[i] + s.win_off[i]);
                if (s.ev_n[i]) r->events = reinterpret_cast<trig_hit *>(s.rblk[i] + s.ev_off[i]);
            }
            if (s.evs[i].ev_cap) r->n_events = s.lost[i] ? 0 : st[i].n_events;
            r->latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(now - p.t_submit).count();
        } else if (s.rblk[i]) {
            rpool.put(s.rblk[i], s.rcls[i]);
        }
        pool.put(p.dblk, p.dbytes);
        {
            std::lock_guard<std::mutex> lk(p.q->mu);
            p.q->done[p.id] = r;
            p.q->in_flight--;
        }
        p.q->cv.notify_all();
        completed++;
    }
    s.slices.clear();
    s.state = 0;
}

void Engine::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        bool busy = false;
        for (auto &s : slots) busy |= s.state != 0;
        if (stop && !busy && pending.empty()) break;
        if (!busy && (pending.empty() || hold)) {
            cv.wait(lk);
            continue;
        }
        // progress in-flight slots; a CUDA error fails the slot's slices
        lk.unlock();
        for (auto &s : slots) {
            if (s.state == 1) {
                cudaError_t q = cudaEventQuery(s.ev_stats);
                if (q == cudaSuccess) collect_stats(s);
                else if (q != cudaErrorNotReady) fail_slot(s, q);
            }
            if (s.state == 2) {
                cudaError_t q = cudaEventQuery(s.ev_done);
                if (q == cudaSuccess) finish(s);
                else if (q != cudaErrorNotReady) fail_slot(s, q);
            }
        }
        lk.lock();
        // admit a new batch into an idle slot
        bool launched = false;
        if (!pending.empty() && !hold) {
            for (auto &s : slots) {
                if (s.state != 0) continue;
                std::vector<Pending> batch;
                const uint32_t take = (mode == 1) ? kMaxBatchSlices : 1u;
                while (!pending.empty() && batch.size() < take) {
                    batch.push_back(std::move(pending.front()));
                    pending.pop_front();
                }
                lk.unlock();
                bool ok = launch_batch_on(s, batch);
                lk.lock();
                if (!ok) {
                    bool others = false;
                    for (auto &o : slots) others |= o.state != 0;
                    if (others && fatal.empty()) {
                        // admission refused for now (memory): put back, retry later
                        for (auto it = batch.rbegin(); it != batch.rend(); ++it) pending.push_front(std::move(*it));
                    } else {
                        // cannot run at all: fail these slices
                        for (auto &p : batch) {
                            trig_result *r = new_result(p.id, p.t0, fatal.empty() ? TRIG_ENOMEM : TRIG_EDEVICE);
                            // after a launch error kernels may still read the block: keep it
                            if (fatal.empty()) pool.put(p.dblk, p.dbytes);
                            std::lock_guard<std::mutex> ql(p.q->mu);
                            p.q->done[p.id] = r;
                            p.q->in_flight--;
                            p.q->cv.notify_all();
                        }
                        fatal.clear();
                    }
                    break;
                }
                launched = true;
                break;
            }
        }
        if (!launched) cv.wait_for(lk, std::chrono::microseconds(20));
    }
}

extern "C" int trig_engine_set_mode(int mode)
{
    if (mode != 0 && mode != 1) return fail(TRIG_EINVAL, "mode must be 0 (plain) or 1 (batched)");
    Engine *e = engine();
    if (!e) return TRIG_EDEVICE;
    std::lock_guard<std::mutex> lk(e->mu);
    e->mode = mode;
    return TRIG_OK;
}

extern "C" int trig_engine_hold(int on)
{
    if (on != 0 && on != 1) return fail(TRIG_EINVAL, "on must be 0 or 1");
    Engine *e = engine();
    if (!e) return TRIG_EDEVICE;
    {
        std::lock_guard<std::mutex> lk(e->mu);
        e->hold = on != 0;
    }
    e->cv.notify_all();
    return TRIG_OK;
}

extern "C" int trig_engine_set_staging_limit(uint64_t bytes)
{
    Engine *e = engine();
    if (!e) return TRIG_EDEVICE;
    std::lock_guard<std::mutex> lk(e->pool.mu);
    e->pool.limit = (size_t)bytes;
    return TRIG_OK;
}

extern "C" int trig_engine_fail_result_allocs(uint32_t n)
{
    Engine *e = engine();
    if (!e) return TRIG_EDEVICE;
    std::lock_guard<std::mutex> lk(e->rpool.mu);
    e->rpool.fail_next = n;
    return TRIG_OK;
}

extern "C" int trig_engine_trace(uint32_t capacity)
{
    Engine *e = engine();
    if (!e) return TRIG_EDEVICE;
    std::lock_guard<std::mutex> lk(e->trace_mu);
    e->trace.clear();
    e->trace.shrink_to_fit();
    e->trace_cap = capacity;
    if (capacity) e->trace.reserve(std::min<size_t>(capacity, (size_t)1 << 20));
    e->trace_t0 = Clock::now();
    return TRIG_OK;
}

extern "C" int trig_engine_trace_read(trig_trace_rec *out, uint32_t max, uint32_t *n_out)
{
    if (!n_out || (max && !out)) return fail(TRIG_EINVAL, "NULL argument");
    Engine *e = engine();
    if (!e) return TRIG_EDEVICE;
    std::lock_guard<std::mutex> lk(e->trace_mu);
    const uint32_t n = (uint32_t)std::min<size_t>(max, e->trace.size());
    std::copy(e->trace.begin(), e->trace.begin() + n, out);
    e->trace.erase(e->trace.begin(), e->trace.begin() + n);
    *n_out = n;
    return TRIG_OK;
}

extern "C" int trig_engine_stats(uint64_t *batches, uint64_t *slices)
{
    Engine *e = engine();
    if (!e) return TRIG_EDEVICE;
    if (batches) *batches = e->batches.load();
    if (slices) *slices = e->completed.load();
    return TRIG_OK;
}

// First index i in [lo, hi) of a time-ordered host run with hits[i].t_ns >= v
// (for a run that is not ordered: some index in [lo, hi]).
// A large host-to-device copy in chunks with at most two queued on the
// stream: copies from other submitting threads queue behind two chunks, not
// behind a whole large slice.
static cudaError_t copy_paced(void *dst, const void *src, size_t bytes, cudaStream_t st)
{
    constexpr size_t kChunk = (size_t)64 << 20;
    if (bytes <= 2 * kChunk) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    thread_local cudaEvent_t ev[2] = {nullptr, nullptr};
    thread_local int ev_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    if (ev_dev != dev) {
        for (int i = 0; i < 2; ++i) {
            if ((e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming))) return e;
        }
        ev_dev = dev;
    }
    size_t k = 0;
    for (size_t off = 0; off < bytes; off += kChunk, ++k) {
        const size_t len = std::min(kChunk, bytes - off);
        if ((e = cudaMemcpyAsync(static_cast<unsigned char *>(dst) + off, static_cast<const unsigned char *>(src) + off,
                                 len, cudaMemcpyHostToDevice, st)))
            return e;
        if ((e = cudaEventRecord(ev[k & 1], st))) return e;
        if (k >= 1 && (e = cudaEventSynchronize(ev[(k - 1) & 1]))) return e;
    }
    return cudaSuccess;
}

static uint64_t host_lb(const trig_hit *h, uint64_t lo, uint64_t hi, int64_t v)
{
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (h[mid].t_ns < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// The same for a v near the end of the run: steps of 1, 2, 4, ... back from
// hi, then a bisection of the last step, so a tail of k hits costs about
// 2 log2(k) reads near the run's end instead of log2(run) scattered ones.
static uint64_t host_lb_back(const trig_hit *h, uint64_t lo, uint64_t hi, int64_t v)
{
    uint64_t right = hi, step = 1;
    while (right > lo) {
        const uint64_t left = right - std::min<uint64_t>(step, right - lo);
        if (h[left].t_ns < v) return host_lb(h, left + 1, right, v);
        right = left;
        step <<= 1;
    }
    return lo;
}

extern "C" int trig_submit_slice(trig_detector *det, int64_t t0, const trig_hit *hits, const uint64_t *pmt_off,
                                 int is_continuation, uint64_t *slice_id_out)
{
    const auto t_entry = Clock::now();
    if (!det || !pmt_off) return fail(TRIG_EINVAL, "NULL argument");
    if (is_continuation != 0 && is_continuation != 1) return fail(TRIG_EINVAL, "is_continuation must be 0 or 1");
    const uint32_t P = det->n_pmt;
    if (pmt_off[0] != 0) return fail(TRIG_EINVAL, "pmt_off[0] must be 0");
    for (uint32_t p = 0; p < P; ++p)
        if (pmt_off[p + 1] < pmt_off[p]) return fail(TRIG_EINVAL, "pmt_off must be non-decreasing");
    const uint64_t n = pmt_off[P];
    if (n && !hits) return fail(TRIG_EINVAL, "hits is NULL");
    const int64_t S = det->par.slice_ns, halo = det->in_halo;
    if (halo > S) return fail(TRIG_EINVAL, "the detector's halo is longer than its slice");
    if (t0 < -((int64_t)1 << 61) || t0 > ((int64_t)1 << 61)) return fail(TRIG_EINVAL, "t0 out of range");
    Engine *e = engine();
    if (!e) return fail(TRIG_EDEVICE, std::string("engine failed to start: ") + g_last_error);
    // one submission of a detector at a time: its resident tail changes here
    TailState &tl = det->tail;
    std::lock_guard<std::mutex> tail_lock(tl.mu);
    uint64_t T = 0;                                   // resident tail hits prepended
    if (is_continuation) {
        if (!tl.have) return fail(TRIG_EINVAL, "is_continuation: the detector has no previous submission");
        if (t0 != tl.next_t0) return fail(TRIG_EINVAL, "is_continuation: t0 must be the previous slice's t0 + slice_ns");
        T = tl.off[P];
        // the resident tail is the leading halo: the submission starts at t0
        for (uint32_t q = 0; q < P; ++q)
            if (pmt_off[q + 1] > pmt_off[q] && hits[pmt_off[q]].t_ns < t0)
                return fail(TRIG_EINVAL, "is_continuation: the submission holds hits before t0");
    }
    if (n + T > kMaxSliceHits) return fail(TRIG_EINVAL, "too many hits in one slice");
    Pending p;
    p.det = det;
    p.q = det->q;
    p.t0 = t0;
    p.n_hits = n + T;
    // copy the slice to a device block now (the caller may reuse its
    // buffers on return), on a stream of this thread's own; a continuation
    // goes to a second block first and is combined with the resident tail
    p.pmt_at = align256(p.n_hits * sizeof(trig_hit));
    const size_t bytes = p.pmt_at + (size_t)(P + 1) * 8;
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    struct DeviceGuard {
        int prev, dev;
        ~DeviceGuard() { if (prev != dev) cudaSetDevice(prev); }
    } guard{prev_dev, e->device};
    if (prev_dev != e->device) cudaSetDevice(e->device);
    p.dblk = e->pool.get(bytes, &p.dbytes);
    if (!p.dblk) return fail(TRIG_EAGAIN, "device staging memory full; poll results and retry");
    unsigned char *raw = nullptr;
    size_t raw_bytes = 0, raw_pmt_at = 0;
    if (T) {
        raw_pmt_at = align256(n * sizeof(trig_hit));
        raw = e->pool.get(raw_pmt_at + (size_t)(P + 1) * 8, &raw_bytes);
        if (!raw) {
            e->pool.put(p.dblk, p.dbytes);
            return fail(TRIG_EAGAIN, "device staging memory full; poll results and retry");
        }
    }
    thread_local cudaStream_t copy_stream = nullptr;
    thread_local int copy_dev = -1;
    cudaError_t ce = cudaSuccess;
    if (!copy_stream || copy_dev != e->device) {
        ce = cudaStreamCreateWithFlags(&copy_stream, cudaStreamNonBlocking);
        copy_dev = e->device;
    }
    unsigned char *dst = T ? raw : p.dblk;
    const size_t dst_pmt_at = T ? raw_pmt_at : p.pmt_at;
    if (!ce && n) ce = copy_paced(dst, hits, n * sizeof(trig_hit), copy_stream);
    if (!ce) ce = cudaMemcpyAsync(dst + dst_pmt_at, pmt_off, (size_t)(P + 1) * 8, cudaMemcpyHostToDevice, copy_stream);
    if (!ce && T)
        ce = launch_prepend(tl.d_hits[tl.cur], tl.d_off[tl.cur], T, reinterpret_cast<const trig_hit *>(raw),
                            reinterpret_cast<const uint64_t *>(raw + raw_pmt_at), n, P,
                            reinterpret_cast<trig_hit *>(p.dblk), reinterpret_cast<uint64_t *>(p.dblk + p.pmt_at),
                            copy_stream);
    // while the copy finishes, the next slice's leading halo: this
    // submission's hits in [t0 + S - halo, t0 + S), PMT by PMT (a producer's
    // unordered stream gives some sub-range; the device flags such a slice),
    // staged in page-locked memory so that its copy is asynchronous like the
    // slice's, and sent to the device copy the prepend above does not read
    std::vector<uint64_t> toff(P + 1, 0), tfrom(P, 0);
    for (uint32_t q = 0; q < P; ++q) {
        const uint64_t a = host_lb_back(hits, pmt_off[q], pmt_off[q + 1], t0 + S - halo);
        const uint64_t b = host_lb_back(hits, a, pmt_off[q + 1], t0 + S);
        tfrom[q] = a;
        toff[q + 1] = toff[q] + (b - a);
    }
    const size_t tn = (size_t)toff[P];
    if (!ce && tn > tl.h_cap) {
        cudaFreeHost(tl.h_hits);
        tl.h_hits = nullptr;
        tl.h_cap = 0;
        const size_t want = std::max<size_t>(tn + tn / 2, 1024);
        ce = cudaHostAlloc(reinterpret_cast<void **>(&tl.h_hits), want * sizeof(trig_hit), cudaHostAllocPortable);
        if (!ce) tl.h_cap = want;
    }
    if (!ce && !tl.h_off) ce = cudaHostAlloc(reinterpret_cast<void **>(&tl.h_off), (size_t)(P + 1) * 8,
                                             cudaHostAllocPortable);
    if (!ce) {
        for (uint32_t q = 0; q < P; ++q)
            std::memcpy(tl.h_hits + toff[q], hits + tfrom[q], (size_t)(toff[q + 1] - toff[q]) * sizeof(trig_hit));
        std::memcpy(tl.h_off, toff.data(), (size_t)(P + 1) * 8);
    }
    const int nx = tl.cur ^ 1;
    if (!ce && tn > tl.cap[nx]) {
        cudaFree(tl.d_hits[nx]);
        tl.d_hits[nx] = nullptr;
        tl.cap[nx] = 0;
        const size_t want = std::max<size_t>(tn + tn / 2, 1024);
        ce = cudaMalloc(&tl.d_hits[nx], want * sizeof(trig_hit));
        if (!ce) tl.cap[nx] = want;
    }
    if (!ce && !tl.d_off[nx]) ce = cudaMalloc(&tl.d_off[nx], (size_t)(P + 1) * 8);
    if (!ce && tn)
        ce = cudaMemcpyAsync(tl.d_hits[nx], tl.h_hits, tn * sizeof(trig_hit), cudaMemcpyHostToDevice, copy_stream);
    if (!ce) ce = cudaMemcpyAsync(tl.d_off[nx], tl.h_off, (size_t)(P + 1) * 8, cudaMemcpyHostToDevice, copy_stream);
    const auto t_wait = Clock::now();
    if (!ce) ce = cudaStreamSynchronize(copy_stream);
    p.copy_wait_us = (uint32_t)std::min<int64_t>(
        std::chrono::duration_cast<std::chrono::microseconds>(Clock::now() - t_wait).count(), 0xffffffffLL);
    if (raw) e->pool.put(raw, raw_bytes);
    if (ce) {
        (void)cudaGetLastError();
        tl.have = false;                              // the resident tail is not valid now
        e->pool.put(p.dblk, p.dbytes);
        return fail(TRIG_EDEVICE, std::string("copying the slice to the device: ") + cudaGetErrorString(ce));
    }
    tl.off = std::move(toff);
    tl.cur = nx;
    tl.have = true;
    tl.next_t0 = t0 + S;
    p.t_submit = t_entry;
    p.t_queued = Clock::now();
    p.continuation = is_continuation != 0;
    p.id = e->next_id++;
    {
        std::lock_guard<std::mutex> lk(p.q->mu);
        p.q->order.push_back(p.id);
        p.q->in_flight++;
    }
    if (slice_id_out) *slice_id_out = p.id;
    {
        std::lock_guard<std::mutex> lk(e->mu);
        e->pending.push_back(std::move(p));
    }
    e->cv.notify_all();
    return TRIG_OK;
}

extern "C" int trig_poll(trig_detector *det, int timeout_ms, trig_result **out)
{
    if (!det || !out) return fail(TRIG_EINVAL, "NULL argument");
    *out = nullptr;
    if (!det->q) return fail(TRIG_EAGAIN, "nothing submitted");
    DetQueue &q = *det->q;
    std::unique_lock<std::mutex> lk(q.mu);
    auto ready = [&] { return !q.order.empty() && q.done.count(q.order.front()); };
    if (!ready()) {
        if (timeout_ms == 0) return fail(TRIG_EAGAIN, "no result ready");
        if (timeout_ms < 0) q.cv.wait(lk, ready);
        else if (!q.cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
            return fail(TRIG_EAGAIN, "no result ready");
    }
    uint64_t id = q.order.front();
    q.order.pop_front();
    *out = q.done[id];
    q.done.erase(id);
    if (!*out) return fail(TRIG_ENOMEM, "result allocation failed");
    return TRIG_OK;
}

extern "C" void trig_result_free(trig_result *r)
{
    if (!r) return;
    ResultBox *box = reinterpret_cast<ResultBox *>(r);
    if (box->blk && box->pool) box->pool->put(box->blk, box->cls);
    std::free(box);
}

extern "C" int trig_destroy(trig_detector *det)
{
    if (!det) return TRIG_OK;
    if (det->q) {
        std::unique_lock<std::mutex> lk(det->q->mu);
        det->q->cv.wait(lk, [&] { return det->q->in_flight == 0; });
        for (auto &kv : det->q->done) trig_result_free(kv.second);
        det->q->done.clear();
    }
    cudaDeviceSynchronize();
    free_det_dev(det);
    delete det;
    return TRIG_OK;
}
