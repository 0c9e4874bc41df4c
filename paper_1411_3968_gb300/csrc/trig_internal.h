// trig_internal.h -- structures shared by the sm_103a kernels (trig_kernels.cu)
// and the host runtime (trig_engine.cpp).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "trig.h"

namespace trig {

// Limits of this implementation.
constexpr uint32_t kMaxPmt = 4096;          // PMTs per detector
constexpr uint32_t kSmemDtMaxPmt = 96;      // dt table lives in shared memory up to this P
constexpr uint32_t kWideMinPmt = 129;       // from this P on, slices are staged from a bucketed copy
constexpr uint32_t kBktChunk = 1024;        // buckets per block of the bucket scan
// A tile plus its halos spans less than 2^20 ns, so a hit's time within the
// staged range and its PMT (< 2^12) pack into 32 bits.  The limit keeps
// 65536 ns (more than any dt, <= 60000 ns) between the last staged time and
// 2^20 - 1, the time of the end keys that the causal count may read past
// the last key.
constexpr uint32_t kTileSpanBits = 20;
constexpr int64_t kMaxTileSpan = ((int64_t)1 << kTileSpanBits) - 65536;
constexpr uint64_t kMaxSliceHits = 0xFFFFFFF0ull;

// Detector tables resident on the device (owned by trig_detector).
struct DetDev {
    uint16_t *dt;         // [P*P] min(dt_max, W), row p_s
    int32_t *dt_exact;    // [P*P] exact dt_max
    uint16_t *floor;      // [P] dense floor index
    uint16_t *dmax_row;   // [P] max_q min(dt_max[p][q], W)
    uint8_t *rel;         // [P*P] relation of PMTs p, q (seed rule 1 only), kRel* bits
};

// PMT relations of the coincidence seed rule.
constexpr uint8_t kRelFloor = 1;        // another PMT of the same floor (FC)
constexpr uint8_t kRelAdjacent = 2;     // adjacent PMT: same floor, within sc_dist (SC)
constexpr uint8_t kRelNextFloor = 4;    // PMT on a consecutive floor of the same tower (AFC)

// Per-slice descriptor in device scratch, written by the host each run.
struct SliceDesc {
    const trig_hit *hits;
    const uint64_t *pmt_off;
    const uint16_t *dt;
    const uint16_t *floor;
    const uint16_t *dmax_row;
    uint32_t n_pmt;
    uint32_t halo;          // tile halo H = max(max dmax_row, floor_tau)
    uint32_t q_seed;
    uint32_t tau;
    uint32_t threshold;
    uint32_t win_half;
    uint32_t l0_hits;       // level 0: N hits (0 = off) within l0_window ns,
    uint32_t l0_window;     //   of different PMTs if l0_distinct
    uint32_t l0_distinct;
    uint32_t seed_rule;     // 0: charge or floor coincidence; 1: [SC and AFC] or [FC and AFC]
    uint32_t sc_w, fc_w, afc_w;     // coincidence windows of seed rule 1 (ns)
    uint32_t count_distinct;        // c(s) counts different PMTs (P <= 128)
    const uint8_t *rel;     // [P*P] kRel* bits (seed rule 1)
    int64_t t0;
    int64_t slice_ns;
    int64_t in_lo, in_hi;   // accepted hit times [in_lo, in_hi)
    uint64_t n_hits;
    int64_t tile_w;         // tile width W (ns); tile g owns [t0 + g W, t0 + (g+1) W)
    uint32_t w_magic;       // ceil(2^32 / W): 32-bit quotient estimate when span32
    uint32_t span32;        // all in-range times are < 2^31 ns past t0 - H
    uint32_t n_tiles;       // NG (<= 2^20)
    uint32_t item0;         // first work item (tile) of this slice
    uint32_t chunk0;        // first structure-pass chunk of this slice
    uint32_t *e_lo;         // [NG][P] first hit index with t >= B_g - H (narrow slices)
    uint32_t *e_hi;         // [NG][P] first hit index with t >= B_{g+1} + H (narrow slices)
    // Wide slices (P >= kWideMinPmt): the hits are also copied, grouped by
    // time bucket [O + b Wb, O + (b+1) Wb), into tbuf; tile g's core is the
    // buckets [lead + g m, lead + (g+1) m) and it stages those plus `hh`
    // buckets on each side, one contiguous range of tbuf.
    uint32_t wide;
    uint32_t bkt_w;         // Wb (ns)
    uint32_t bkt_magic;     // ceil(2^32 / Wb)
    uint32_t bkt_lead;      // buckets before t0
    uint32_t bkt_per_tile;  // m
    uint32_t bkt_halo;      // hh = ceil(H / Wb)
    uint32_t n_bkt;         // NB
    uint32_t bkt32;         // every in-range time is < 2^31 ns past O
    int64_t bkt_origin;     // O = t0 - lead * Wb
    uint32_t *bkt_cnt;      // [NB] hits per bucket, then fill cursors
    uint32_t *bkt_off;      // [NB + 1] exclusive prefix of the counts
    uint32_t *bkt_part;     // [ceil(NB / kBktChunk)] sums of the counts per chunk
    trig_hit *tbuf;         // [n_hits] hits in bucket order
    trig_trigger *stage;    // [n_hits] fired seeds at their merged rank
    uint32_t *wrank;        // [n_hits][2] beside each staged fired seed: the merged ranks of the
                            //   first hit at or after t - win_half and of the first after t + win_half
    uint32_t *win_r;        // [win_cap][2] a window's first-hit rank (from its first trigger)
                            //   and its one-past-last rank (from its last trigger)
    uint32_t *tile_nfired;  // [NG]
    uint32_t *tile_rank;    // [NG] merged rank of the tile's first core hit
    uint32_t *tile_out;     // [NG] exclusive prefix of tile_nfired
    uint32_t *tile_nwin;    // [NG] window heads among the tile's triggers
    uint32_t *tile_wout;    // [NG] exclusive prefix of tile_nwin
    trig_trigger *triggers;
    uint64_t trig_cap;
    trig_window *windows;
    uint64_t win_cap;
    trig_slice_stats *stats;
    // event extraction (ev != nullptr): the slice's hits in merged order,
    // each window's first merged rank and its offset in the event output
    trig_hit *ev;
    uint64_t ev_cap;
    uint32_t *win_rlo;      // [win_cap]
    uint32_t *ev_off;       // [win_cap + 1]
    trig_hit *dbg_merged;   // merged rows, indexed by merged rank - dbg_rank0 (row outputs,
                            // or the slice's merged stream for event extraction)
    uint32_t *dbg_seedcnt;
    uint64_t dbg_rank0;     // merged rank of the first owned hit (row outputs only)
    uint64_t dbg_rank1;     // merged rank of the first hit after the owned range
};

struct BatchHeader {
    uint32_t n_slices;
    uint32_t n_items;       // total tiles
    uint32_t n_chunks;      // total structure-pass chunks
    uint32_t err;
    uint32_t queue;         // tile work queue head
    uint32_t any_wide;      // a slice of the batch is wide
    uint32_t any_events;    // a slice of the batch extracts events
    uint32_t any_ext;       // a slice uses level 0, seed rule 1 or the distinct count
    uint32_t dense;         // a slice expects kDenseKeys or more keys per causal scan range
    uint32_t stall;         // test control: the tile pass's stagers fill nothing, so its waits run out
    uint64_t wait_ns;       // limit of every device wait (ns); a wait that runs out sets TRIG_FLAG_TIMEOUT
};

constexpr uint64_t kDefaultWaitNs = 1000000000ull;     // one second

// Expected keys in a seed's scan range (2H + 1 ns at the slice's mean rate)
// from which the causal count gives each seed a warp instead of 4 lanes.
constexpr double kDenseKeys = 600.0;

constexpr uint32_t kChunkHits = 4096;       // structure-pass chunk

// Kernel launch helpers implemented in trig_kernels.cu.
cudaError_t launch_dtmax(const int32_t *xyz, uint32_t n_pmt, uint32_t tol, uint32_t n_num, uint32_t n_den,
                         uint32_t corr, int32_t *dt_exact, uint16_t *dt, uint16_t *dmax_row, cudaStream_t st);

// Launch shape of the tile kernel: hits per shared-memory tile, consumer
// warps per block, and the target fill of a tile (percent of cap) that sets
// the tile width.  Valid (cap, warps): (4096, 16), (4096, 8), (2048, 16),
// (2048, 8), (1024, 4); smaller tiles run more blocks per SM (up to 2 for
// 2048 hits, 4 or more for 1024).
struct TileConfig {
    uint32_t cap;
    uint32_t warps;
    uint32_t fill_pct;
};
inline bool valid_tile_shape(uint32_t cap, uint32_t warps)
{
    return ((cap == 4096 || cap == 2048) && (warps == 16 || warps == 8)) || (cap == 1024 && warps == 4);
}
constexpr uint32_t kMaxTilesPerSlice = 1u << 20;

// Enqueues the batch pipeline; header/desc already copied to device scratch.
constexpr int kPipelineKernels = 15;
extern const char *const kKernelNames[kPipelineKernels];

// any_wide: the batch holds a wide slice (the bucket sums, scan and
// scatter kernels run only then); any_events: a slice extracts events (the
// halo, event-offset and event-copy kernels run only then); any_ext: a slice
// uses level 0, seed rule 1 or the distinct count (the tile kernel built
// with those rules runs, else the one without them); dense: the tile kernel
// built with a warp per seed in the causal count runs.  ev (optional, kPipelineKernels + 1 events): ev[i]
// is recorded before pipeline kernel i and ev[kPipelineKernels] after the
// last one (a kernel that does not run gets an empty interval).
// *launches is increased by the number of kernels launched.
cudaError_t launch_batch(BatchHeader *d_hdr, SliceDesc *d_desc, uint32_t n_slices, uint32_t max_pmt,
                         bool any_smem_dt, bool any_wide, bool any_events, bool any_ext, bool dense,
                         const TileConfig &cfg,
                         cudaStream_t st,
                         uint64_t *launches, bool rows, cudaEvent_t *ev = nullptr);

int device_sm_count();

// Continuation submissions: the combined slice (resident tail of each PMT,
// then the submission's hits of that PMT) into out / out_off.
cudaError_t launch_prepend(const trig_hit *tail, const uint64_t *tail_off, uint64_t n_tail, const trig_hit *fresh,
                           const uint64_t *fresh_off, uint64_t n_fresh, uint32_t P, trig_hit *out, uint64_t *out_off,
                           cudaStream_t st);

// What other translation units of the library read of a detector.
struct DetInfo {
    uint32_t n_pmt;
    const int32_t *xyz;     // host, 3 * n_pmt (the detector's copy)
    trig_params par;
    int64_t in_halo;        // accepted halo around a slice
    int device;
};
bool detector_info(const trig_detector *d, DetInfo *out);

// The library's error reporting (trig_last_error) and launch counter.
int report_error(int code, const char *msg);
int report_cuda_error(cudaError_t e, const char *what);
void count_launches(uint64_t n);

// Address and size of the library's static scratch array on the current device.
cudaError_t static_scratch(void **ptr, size_t *bytes);

// A no-allocation batch's header and descriptors, passed by value to the
// kernel that writes them into the static scratch array.
struct NoallocPlan {
    BatchHeader hdr;
    SliceDesc desc[TRIG_NOALLOC_MAX_SLICES];
    uint32_t n;
};
static_assert(sizeof(BatchHeader) % 4 == 0 && sizeof(SliceDesc) % 4 == 0, "copied as 32-bit words");
static_assert(sizeof(NoallocPlan) <= 32000, "kernel parameter space");
cudaError_t launch_put_plan(const NoallocPlan &plan, BatchHeader *hdr, SliceDesc *desc, cudaStream_t st);

}  // namespace trig
