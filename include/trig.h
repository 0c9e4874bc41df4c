/*
 * trig.h -- C ABI of the GB300 online muon trigger (arXiv 1411.3968).
 *
 * The method ("Muon trigger strategy" and "Sorting and triggering in GPU"):
 * every 200 ms time slice of merged PMT hits of a detector is scanned for
 * seed hits (charge over threshold, or two hits on one floor within a few
 * ns); each seed counts the hits causally related to it,
 *     c(s) = #{ j : |t_j - t_s| <= min(dt_max[p_s][p_j], W) },
 * with dt_max the light travel time between the two PMTs plus a tolerance
 * and W the 3 us correlation interval; the seed fires when c(s) reaches the
 * threshold, and the 6 us windows centred on the fired seeds (+-3 us, the
 * data sent to the Event Manager, "DAQ system of NEMO Phase II") are merged
 * and returned.
 *
 * The paper's other rules are parameters of the same path: the level-0
 * trigger (N hits within TW, optionally on different PMTs), its combination
 * of simple, floor and adjacent-floor coincidences, and a causal count over
 * different PMTs (trig_params).
 *
 * Two faces:
 *   - the engine (trig_create / trig_submit_slice / trig_poll / trig_destroy):
 *     host buffers in, host results out; slices from all detectors are
 *     batched continuously on one GPU;
 *   - the device batch call (trig_batch_run): device buffers in and out, the
 *     caller owns all memory, one launch sequence for many slices; its
 *     events form also copies every hit inside the windows, and
 *     trig_array.h selects across the towers of an array and reads their
 *     windows back.
 *
 * All functions return TRIG_OK (0) or a negative TRIG_E* code and never
 * throw.  trig_last_error() gives a message for the calling thread's last
 * failure.  Pointers marked "device" must be CUDA device (or managed)
 * memory of the current device; "host" pointers are ordinary host memory.
 */
#ifndef TRIG_H
#define TRIG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- codes */
#define TRIG_OK          0
#define TRIG_EINVAL     (-1)  /* bad argument or malformed input slice          */
#define TRIG_ENOMEM     (-2)  /* host or device allocation failed               */
#define TRIG_EAGAIN     (-3)  /* admission full (submit) / nothing ready (poll) */
#define TRIG_ETIMEOUT   (-4)  /* a bounded wait ran out                         */
#define TRIG_EDEVICE    (-5)  /* CUDA error                                     */
#define TRIG_ECAPACITY  (-6)  /* output capacity or tile capacity exceeded      */

/* Slice status bits reported by the device (trig_slice_stats.flags). */
#define TRIG_FLAG_BAD_PMT      0x01u  /* hit.pmt >= n_pmt or outside its CSR row  */
#define TRIG_FLAG_UNSORTED     0x02u  /* a PMT stream is not time-ordered         */
#define TRIG_FLAG_OUT_OF_RANGE 0x04u  /* hit outside [t0 - halo, t0 + S + halo)   */
#define TRIG_FLAG_TILE_FULL    0x08u  /* > tile capacity hits inside one 1 ns core
                                         plus its halo; results incomplete       */
#define TRIG_FLAG_TRIG_FULL    0x10u  /* more triggers than trig_cap             */
#define TRIG_FLAG_WIN_FULL     0x20u  /* more windows than win_cap               */
#define TRIG_FLAG_TIMEOUT      0x40u  /* a bounded device wait gave up            */
#define TRIG_FLAG_EV_FULL      0x80u  /* more event hits than ev_cap, or a halo of
                                         more than TRIG_EV_HALO_MAX hits              */

/* ----------------------------------------------------------------- types */

/* One PMT hit, 16 bytes: the fixed-size GPU hit record of "CPU-GPU" (charge,
 * time, DU identification).  `reserved` is carried but never read. */
typedef struct {
    int64_t t_ns;       /* hit time, integer ns                       */
    uint16_t pmt;       /* PMT (detection unit) index, < n_pmt         */
    uint16_t charge;    /* ADC counts (1 pe = 100 in the workloads)    */
    uint32_t reserved;
} trig_hit;

/* Detector description, copied by trig_create.  Two PMTs are on the same
 * floor iff their floor_id values are equal (ids need not be dense).
 * Coordinates must lie within +-1e8 mm; 1 <= n_pmt <= 4096. */
typedef struct {
    uint32_t n_pmt;
    const int32_t *xyz_mm;      /* host, 3 * n_pmt: x, y, z of PMT p       */
    const uint32_t *floor_id;   /* host, n_pmt                              */
    const uint32_t *tower_id;   /* host, n_pmt, or NULL (one tower): groups
                                   floors for the consecutive-floor test */
} trig_geometry;

/* Trigger constants.  The paper names the primitives (QTRIG charge
 * threshold, floor coincidence, 3 us correlation interval, +-3 us tagging)
 * but leaves their values open; the workloads use
 * {300, 20, 20, 6900, 1499, 3000, 4, 3000, 200000000}. */
typedef struct {
    uint32_t q_seed_adc;        /* charge seed: charge >= q_seed_adc                */
    uint32_t floor_tau_ns;      /* floor coincidence: |t_i - t_j| <= tau            */
    uint32_t tol_ns;            /* dt_max = tol + ceil(d * n_num / (n_den * 1000))  */
    uint32_t n_num, n_den;      /*   for d in mm: n_num/n_den ns per metre          */
    uint32_t corr_window_ns;    /* W: the causal test uses min(dt_max, W)           */
    uint32_t threshold;         /* fire when c(s) >= threshold                      */
    uint32_t win_half_ns;       /* event window [t - h, t + h], merged when touching */
    int64_t slice_ns;           /* a slice owns [t0, t0 + slice_ns)                 */
    /* Level-0 trigger ("Muon trigger strategy", "Sorting and triggering in
     * GPU": N7TW1000 / DN7TW1000, N hits within TW, applied before the
     * seed triggers).  With l0_hits = N > 0 a seed counts only if some
     * window [a, a + TW) containing it holds at least N hits, or, with
     * l0_distinct_pmts, hits of at least N different PMTs (any n_pmt).
     * l0_hits = 0 turns it off; TW <= 60000 ns. */
    uint32_t l0_hits;
    uint32_t l0_window_ns;
    uint32_t l0_distinct_pmts;
    /* Seed rule.  0: charge >= q_seed_adc, or a hit on another PMT of the
     * same floor within floor_tau_ns.  1: the paper's combination of
     * coincidences ("Sorting and triggering in GPU", "Results and
     * perspectives": [SC and AFC] or [FC and AFC]): a hit is a seed iff a
     * hit on a consecutive floor of its tower lies within afc_window_ns
     * (AFC), and a hit on an adjacent PMT within sc_window_ns (SC) or on
     * another PMT of its floor within fc_window_ns (FC).  Adjacent PMTs:
     * different PMTs of one floor at most sc_dist_mm apart.  Consecutive
     * floors: neighbours when a tower's floors (trig_geometry.tower_id,
     * NULL = one tower) are ordered by the z of their lowest PMT, ties by
     * floor_id.  Level 0 applies after either rule; with threshold = 1
     * every seed fires (c(s) >= 1 always), which is the paper's trigger
     * ladder N7TW, then [SC and AFC] or [FC and AFC]. */
    uint32_t seed_rule;
    uint32_t sc_window_ns;      /* <= 60000 */
    uint32_t fc_window_ns;      /* <= 60000 */
    uint32_t afc_window_ns;     /* <= 60000 */
    uint32_t sc_dist_mm;
    /* 1: c(s) counts the different PMTs among the causally related hits
     * (the distinct-PMT variant, robust to a single PMT's bursts; any
     * n_pmt); 0: c(s) counts hits. */
    uint32_t count_distinct_pmts;
    uint32_t reserved;          /* 0 */
} trig_params;

/* A fired seed: its hit and causal count c(s). 16 bytes. */
typedef struct {
    int64_t t_ns;
    uint16_t pmt;
    uint16_t charge;
    uint32_t count;
} trig_trigger;

/* A merged event window [lo_ns, hi_ns] (inclusive), the number of hits of
 * the slice submission inside it and the number of triggers it merged. */
typedef struct {
    int64_t lo_ns, hi_ns;
    uint64_t n_hits;
    uint64_t n_triggers;
} trig_window;

/* Per-slice counters written by the device. status is TRIG_OK,
 * TRIG_EINVAL (input flags), TRIG_ECAPACITY or TRIG_ETIMEOUT. */
typedef struct {
    int32_t status;
    uint32_t flags;             /* TRIG_FLAG_* bits                          */
    uint64_t n_hits;            /* hits submitted (owned range and halos)    */
    uint64_t n_seeds;
    uint64_t n_triggers;        /* may exceed trig_cap (then TRIG_FLAG_TRIG_FULL) */
    uint64_t n_windows;         /* may exceed win_cap  (then TRIG_FLAG_WIN_FULL)  */
    uint64_t n_events;          /* hits inside the merged windows (event runs
                                   only; may exceed ev_cap, then TRIG_FLAG_EV_FULL) */
} trig_slice_stats;

typedef struct trig_detector trig_detector;

/* Engine result of one slice; owned by the library until trig_result_free. */
typedef struct {
    uint64_t slice_id;
    int64_t t0_ns;
    int32_t status;             /* TRIG_OK or a TRIG_E* code      */
    uint32_t flags;             /* TRIG_FLAG_* bits               */
    uint64_t n_hits, n_seeds, n_triggers, n_windows;
    trig_trigger *triggers;     /* n_triggers entries, (t, pmt, charge) order */
    trig_window *windows;       /* n_windows entries, time order              */
    int64_t latency_ns;         /* submit -> result ready (host clock)        */
    trig_hit *events;           /* n_events hits inside the windows, in (t,
                                   pmt, charge) order, when the detector
                                   extracts events (trig_set_events); else NULL */
    uint64_t n_events;
} trig_result;

/* ------------------------------------------------------------- detectors */

/* Creates a detector: copies the geometry and parameters, builds the exact
 * integer causality table dt_max on the device ("Muon trigger strategy":
 * the time-space correlation) and keeps it resident until trig_destroy.
 * EINVAL on n_pmt outside [1, 4096], NULL pointers, n_den == 0,
 * slice_ns <= 0 or coordinates beyond +-1e8 mm; ENOMEM / EDEVICE on CUDA
 * failures.  The detector is bound to the CUDA device current at creation. */
int trig_create(const trig_geometry *geometry, const trig_params *params, trig_detector **out);

/* Drains the detector's in-flight slices, then frees it and its device
 * tables (the end of a run of the paper's per-tower TGPU, "Results and
 * perspectives").  Results not yet polled are discarded; the detector's
 * resident slice tail is freed.  NULL is accepted. */
int trig_destroy(trig_detector *det);

/* Copies the exact (unclamped) dt_max table into host memory dt_out
 * (n_pmt * n_pmt int32, row p_s, column p_j). */
int trig_detector_dtmax(const trig_detector *det, int32_t *dt_out);

/* Halo the detector needs around each slice: hits in
 * [t0 - halo, t0 + slice_ns + halo) are accepted and used; halo is the
 * largest of corr_window_ns, win_half_ns, the seed rule's coincidence window
 * (floor_tau_ns, or the largest of sc/fc/afc_window_ns under seed rule 1)
 * and l0_window_ns when level 0 is on. */
int64_t trig_detector_halo_ns(const trig_detector *det);

/* ---------------------------------------------------------------- engine */

/* Submits one slice (host memory).  hits are grouped by PMT (CSR):
 * hits[pmt_off[p] .. pmt_off[p+1]) are PMT p's hits in non-decreasing time;
 * pmt_off has n_pmt + 1 entries, pmt_off[0] == 0, and pmt_off[n_pmt] is the
 * hit count (< 2^32).  Seeds are only those in [t0, t0 + slice_ns).  The
 * hits are copied before the call returns.
 *
 * Halos ("Preparation in CPU": at the end of a slice the trigger proceeds
 * on the first hits of the next one).  The producer always includes the
 * trailing halo, the hits of [t0 + slice_ns, t0 + slice_ns + halo).  The
 * leading halo [t0 - halo, t0) comes from one of two places:
 *   - is_continuation = 0: from the submission itself (every hit of
 *     [t0 - halo, t0 + slice_ns + halo) the detector recorded; none for the
 *     first slice of a run);
 *   - is_continuation = 1: from the device.  The library keeps the last
 *     `halo` ns of every submission of the detector, [t0' + slice_ns - halo,
 *     t0' + slice_ns), resident on the device and prepends them PMT by PMT;
 *     t0 must then be the previous submission's t0' + slice_ns, and the
 *     submission holds no hit before t0.
 * Submissions of one detector are serialised.  EINVAL on malformed offsets
 * or a continuation that does not follow the previous submission; EAGAIN
 * when the engine's staging memory is full (poll, then retry).  Malformed
 * hit records (bad pmt, unsorted streams, out-of-range times) are detected
 * on the device and reported through the result's status (EINVAL) and
 * flags. */
int trig_submit_slice(trig_detector *det, int64_t slice_t0_ns, const trig_hit *hits, const uint64_t *pmt_off,
                      int is_continuation, uint64_t *slice_id_out);

/* Returns the detector's oldest unreturned result: the triggered windows
 * handed to the Event Manager ("DAQ system of NEMO Phase II": the 6 us
 * window around each trigger seed is kept).  Slices complete in submission
 * order per detector.  Waits up to timeout_ms (0: do not wait, < 0: wait
 * without limit); EAGAIN if nothing is ready in time.  *out is owned by the
 * library until trig_result_free. */
int trig_poll(trig_detector *det, int timeout_ms, trig_result **out);

/* Returns a result's memory (its trigger, window and event arrays) to the
 * library.  NULL is accepted. */
void trig_result_free(trig_result *res);

/* Engine policy: 0 = plain (every slice is its own launch sequence),
 * 1 = batched (pending slices of all detectors share one launch, replayed
 * from a CUDA graph).  Default 1. */
int trig_engine_set_mode(int mode);

/* Engine counters since start: batches launched, slices completed. */
int trig_engine_stats(uint64_t *batches, uint64_t *slices);

/* Message of the calling thread's last failure ("" if none): the library's
 * own error report (the paper has no error interface).  The string is
 * thread-local and valid until the thread's next failing call. */
const char *trig_last_error(void);

/* Engine controls for operations and tests (the engine's own policy; the
 * paper has no counterpart).
 *   trig_engine_hold(1): admit no new batch (submissions still queue) until
 *     trig_engine_hold(0); the queued slices then share batches.
 *   trig_engine_set_staging_limit(bytes): device staging memory that queued
 *     and running submissions may hold at once (0: no limit beyond free
 *     device memory, the default); a submission beyond it gets TRIG_EAGAIN.
 *   trig_engine_fail_result_allocs(n): failure injection on the host: the
 *     next n requests for result memory fail as if page-locked memory were
 *     exhausted; those slices complete with status TRIG_ENOMEM and no
 *     arrays. */
int trig_engine_hold(int on);
int trig_engine_set_staging_limit(uint64_t bytes);
int trig_engine_fail_result_allocs(uint32_t n);

/* Engine trace: one record per completed slice, for latency studies (the
 * engine's own instrumentation; the paper has no counterpart).  Times are
 * steady-clock ns since trig_engine_trace was called. */
typedef struct {
    uint64_t slice_id;
    uint64_t batch;             /* engine batch number, from 1             */
    uint32_t batch_slices;      /* slices in that batch                     */
    uint32_t n_pmt;
    uint64_t n_hits;            /* hits of the submission (with the tail)   */
    int32_t status;
    uint32_t continuation;      /* submitted with is_continuation = 1       */
    int64_t t_submit_ns;        /* trig_submit_slice entered                */
    int64_t t_queued_ns;        /* copied to the device and queued          */
    int64_t t_launch_ns;        /* its batch launched                       */
    int64_t t_stats_ns;         /* its batch's counters reached the host    */
    int64_t t_done_ns;          /* result delivered to trig_poll            */
    float device_ms;            /* its batch's device time (CUDA events from
                                   launch to counters), -1 if unknown       */
    uint32_t copy_wait_us;      /* of t_queued - t_submit: the time the
                                   submission waited for its copies to the
                                   device after its host work (microseconds) */
} trig_trace_rec;

/* Starts recording (clearing earlier records) up to `capacity` slices;
 * 0 stops.  trig_engine_trace_read moves up to `max` records, oldest first,
 * into host memory `out` and sets *n_out. */
int trig_engine_trace(uint32_t capacity);
int trig_engine_trace_read(trig_trace_rec *out, uint32_t max, uint32_t *n_out);

/* Bounded device waits.  Every wait of the tile pass (the stager waiting
 * for a free buffer, the consumers waiting for a staged tile) gives up after
 * limit_ns of the GPU's global timer (default 1 s; 0 restores it, at most
 * 600 s), sets TRIG_FLAG_TIMEOUT and ends the pass; the batch's slices then
 * report TRIG_ETIMEOUT with no output, and the device stays usable.
 * stall = 1 is a test control: later batches stage no tile, so the first
 * wait of every block runs out with no copy in flight; stall = 0 ends it;
 * any other value is TRIG_EINVAL.  Applies to batches planned after the
 * call. */
int trig_set_device_wait(uint64_t limit_ns, int stall);

/* Page-locked host memory for a producer's slice buffers (the Hit
 * Manager's output, "DAQ system of NEMO Phase II"): trig_submit_slice
 * copies such buffers to the device by DMA, without the CUDA driver's staging
 * of pageable memory, whose speed depends on how the host's pages are
 * laid out.  *out receives `bytes` bytes (16-byte aligned) owned by the
 * caller until trig_host_free.  Errors: TRIG_EINVAL, TRIG_ENOMEM. */
int trig_host_alloc(size_t bytes, void **out);
int trig_host_free(void *ptr);

/* ------------------------------------------------------- device batches */

/* One slice for trig_batch_run.  All buffers are device memory owned by the
 * caller.  hits must be 16-byte aligned.  Layout and halo rules as for
 * trig_submit_slice.  Outputs: up to trig_cap triggers and win_cap windows;
 * a window bound that can never overflow is
 *   win_cap >= (slice_ns + 2 * win_half_ns) / (2 * win_half_ns + 2) + 1. */
typedef struct {
    const trig_detector *det;
    const trig_hit *hits;          /* device */
    const uint64_t *pmt_off;       /* device, n_pmt + 1 */
    uint64_t n_hits;               /* == pmt_off[n_pmt]  */
    int64_t t0_ns;
    trig_trigger *triggers;        /* device, trig_cap entries */
    uint64_t trig_cap;
    trig_window *windows;          /* device, win_cap entries  */
    uint64_t win_cap;
    trig_slice_stats *stats;       /* device, one entry        */
} trig_slice_dev;

/* Scratch bytes trig_batch_run needs for these slices (0 on bad input). */
size_t trig_batch_scratch_bytes(const trig_slice_dev *slices, uint32_t n_slices);

/* Runs the whole hot path for n_slices slices on `stream` (a cudaStream_t,
 * NULL for the legacy default stream): the k-way merge of the PMT streams,
 * seed selection, causal counting, stream compaction of the fired seeds and
 * the window merge.  Asynchronous: results are valid once the stream
 * reaches this point.  `scratch` is device memory of at least
 * trig_batch_scratch_bytes(), 256-byte aligned; it must not be used by
 * anything else until the work completes.  flags: TRIG_RUN_GRAPH replays
 * the launch sequence from a cached CUDA graph (one per stream, scratch
 * pointer and batch plan; a new batch captures a new graph).  EINVAL on bad
 * arguments (nothing is launched). */
#define TRIG_RUN_GRAPH 0x1u
#define TRIG_RUN_TIMED 0x2u   /* record CUDA events around each kernel (not with GRAPH) */
int trig_batch_run(const trig_slice_dev *slices, uint32_t n_slices, void *scratch, size_t scratch_bytes,
                   void *stream, uint32_t flags);

/* Event extraction: the Event Manager's payload ("DAQ system of NEMO
 * Phase II": a 6 us window around each trigger seed is stored; "Sorting and
 * triggering in GPU": all hits within +-3 us of a seed are tagged and sent
 * back).  For each slice, every hit of the submission (owned range and
 * halos) inside one of its merged windows, in (t, pmt, charge) order; the
 * windows are disjoint and time-ordered, so window w's hits start at the
 * sum of n_hits of the windows before it.  events is device memory of
 * ev_cap entries (ev_cap 0 skips the slice); stats.n_events gets the count.
 * When the status is not TRIG_OK the events buffer is not written.
 * The leading and trailing halos of a slice may hold at most
 * TRIG_EV_HALO_MAX hits each for extraction (else TRIG_FLAG_EV_FULL). */
#define TRIG_EV_HALO_MAX 8192u
typedef struct {
    trig_hit *events;           /* device, ev_cap entries */
    uint64_t ev_cap;
} trig_slice_events;

/* Scratch for trig_batch_run_events (more than trig_batch_scratch_bytes:
 * the merged stream of each slice with events). */
size_t trig_batch_events_scratch_bytes(const trig_slice_dev *slices, const trig_slice_events *events,
                                       uint32_t n_slices);

/* trig_batch_run plus event extraction for the slices whose events entry
 * has ev_cap > 0.  Same stream, scratch, flags and error rules. */
int trig_batch_run_events(const trig_slice_dev *slices, const trig_slice_events *events, uint32_t n_slices,
                          void *scratch, size_t scratch_bytes, void *stream, uint32_t flags);

/* Engine: extract events for det's later submissions (on = 1) or not
 * (on = 0, the default); results then carry events/n_events. */
int trig_set_events(trig_detector *det, int on);

/* The same hot path as trig_batch_run for callers that cannot allocate
 * device memory: a trigger node's real-time acquisition thread (cudaMalloc
 * can synchronise the whole device and stall it for milliseconds) or code
 * that runs while another thread captures a CUDA graph in global mode
 * (where cudaMalloc is refused).  The scratch is a static device array of
 * TRIG_NOALLOC_SCRATCH_BYTES inside the library, held by every device that
 * loads it until the process exits; the caller still passes inputs and
 * outputs as for trig_batch_run.  Nothing is allocated: no cudaMalloc,
 * cudaFree or allocating library call.  The paper has no counterpart; this
 * is a deployment interface.
 *   - stream must be a stream the caller created, best with
 *     cudaStreamNonBlocking: NULL (the legacy default stream) is refused
 *     with TRIG_EINVAL, since it synchronises with other streams and is
 *     forbidden while another thread captures in global mode.  The batch's
 *     descriptors travel as a kernel parameter, so the call does not wait
 *     for earlier work on the stream.
 *   - A stream that is capturing is refused with TRIG_EINVAL: the call must
 *     not be captured into a CUDA graph.
 *   - At most TRIG_NOALLOC_MAX_SLICES slices; a batch whose scratch would
 *     exceed the array (about 3.9 M hits at 16 B of staging per hit) is
 *     rejected with TRIG_ECAPACITY before anything is launched.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream
 *     capture.
 *   - All calls share the array and it keeps the last call's contents; the
 *     library clears what must start at zero.  Calls whose work overlaps on
 *     the GPU (different streams, or different host threads) race on it:
 *     serialise them. */
#define TRIG_NOALLOC_SCRATCH_BYTES (64u << 20)
#define TRIG_NOALLOC_MAX_SLICES 16u
int trig_batch_run_noalloc(const trig_slice_dev *slices, uint32_t n_slices, void *stream);

/* Row-level view of one slice for verification: writes the owned hits in
 * merged (t, pmt, charge) order to merged_out (device, n_hits entries; the
 * owned hits start at index 0) and, for each of them, its causal count if
 * it is a seed or 0xFFFFFFFF if not, to seedcnt_out (device, n_hits
 * entries).  *n_owned_out (host) receives the number of owned hits.  Runs
 * the same kernels as trig_batch_run and synchronises the stream. */
int trig_slice_rows(const trig_slice_dev *slice, trig_hit *merged_out, uint32_t *seedcnt_out,
                    uint64_t *n_owned_out, void *scratch, size_t scratch_bytes, void *stream);

/* Default launch shape of the tile kernel for detectors that have not been
 * tuned: tile capacity (hits per shared-memory tile including halos),
 * consumer warps per block and target fill (percent of the capacity a tile
 * plus its halos should hold at the slice's mean rate; it sets the tile
 * width).  (cap, warps) must be (4096, 16), (4096, 8), (2048, 16), (2048, 8)
 * or (1024, 4);
 * fill_pct in [10, 95].  Applies to later runs in this process. */
int trig_set_tile_config(uint32_t cap, uint32_t warps, uint32_t fill_pct);
int trig_get_tile_config(uint32_t *cap, uint32_t *warps, uint32_t *fill_pct);

/* Autotuner: times every launch shape (5 (cap, warps) pairs x 4 fills) on
 * the given device-resident slices, which must all belong to det, keeps the
 * fastest on det (later runs use it for det's slices; a batch mixing
 * detectors takes the shape of the one with the most hits) and, when the
 * environment variable TRIG_TUNE_CACHE names a file, appends
 * "<gpu> <n_pmt> <cap> <warps> <fill> <ms>" to it; trig_create applies a
 * cached entry for the same GPU and PMT count.  Allocates its own scratch
 * and synchronises the stream. */
typedef struct {
    uint32_t cap, warps, fill_pct, n_tried;
    double ms;                  /* mean time of the chosen shape per batch */
} trig_tune_result;
int trig_autotune(trig_detector *det, const trig_slice_dev *slices, uint32_t n_slices, void *stream,
                  trig_tune_result *out);

/* det's launch shape (tuned or default); returns 1 if tuned, 0 if not. */
int trig_detector_tile_config(const trig_detector *det, uint32_t *cap, uint32_t *warps, uint32_t *fill_pct);

/* Kernel launches issued by trig_batch_run so far (graph replays count
 * their kernels). */
uint64_t trig_kernel_launch_count(void);

/* Average device time per kernel of the pipeline over the runs made with
 * TRIG_RUN_TIMED since the previous call (waits for their events), in the
 * launch order k_prep, k_bounds, k_bsum, k_bscan, k_scatter, k_tile,
 * k_evhalo, k_scan, k_copy, k_wscan, k_wwrite, k_wcount, k_escan,
 * k_events, k_status.  k_bsum, k_bscan and k_scatter run only for batches
 * with a detector of 129 or more PMTs, k_evhalo, k_escan and k_events only
 * for event extraction; the others read about 0.
 * avg_ms[i] and names[i] (static strings) for i < max_kernels; returns the
 * number of kernels (15) and the number of runs in *n_runs. */
int trig_kernel_times(double *avg_ms, const char **names, uint32_t max_kernels, uint32_t *n_runs);

#ifdef __cplusplus
}
#endif
#endif /* TRIG_H */
