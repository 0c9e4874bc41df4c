/*
 * trig_array.h -- multi-tower selection of the online muon trigger
 * (arXiv 1411.3968, "Results and perspectives": for the eight KM3Net-It
 * towers, each tower's GPU looks for all trigger seeds of its tower and
 * sends them to a central CPU; that CPU selects the muon-track candidates
 * and sends their times back, and every tower ships its window of data
 * around them to the Event Manager).
 *
 * Here the towers are trig_detectors whose slices for one time range were
 * run by trig_batch_run (their triggers and stats are on the device).  One
 * call then selects the candidates across towers and reads every tower's
 * hits around them back into one device buffer, all on the device.
 *
 * The paper names these steps but not the selection rule.  The rule here
 * is the paper's time-space correlation applied across towers: a tower's
 * trigger s (PMT p_s, time t_s) is selected iff at least min_towers towers,
 * its own included, hold a trigger j of the same slice period with
 *   |t_j - t_s| <= min(dt_max(p_s, p_j), corr_window_ns),
 * dt_max computed from the two PMTs' positions in the common frame of the
 * towers' geometries with the towers' (equal) tol_ns, n_num and n_den.
 * Windows [t - win_half_ns, t + win_half_ns] around the selected triggers
 * of all towers, in time order, merge while lo_next <= hi_cur + 1.  The
 * readback lists, window by window and tower by tower, the tower's hits
 * inside the window in the order of the tower's slice (PMT by PMT, time
 * order within a PMT).
 */
#ifndef TRIG_ARRAY_H
#define TRIG_ARRAY_H

#include "trig.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct trig_array trig_array;

typedef struct {
    uint32_t min_towers;        /* K >= 1                                          */
    uint32_t corr_window_ns;    /* W <= 60000: the cross-tower test uses min(dt_max, W) */
    uint32_t win_half_ns;       /* h: readback window [t - h, t + h]; at most every
                                   tower's accepted halo (trig_detector_halo_ns)  */
    uint32_t reserved;          /* 0 */
} trig_array_params;

/* A selected trigger, 16 bytes. */
typedef struct {
    int64_t t_ns;
    uint16_t pmt;               /* PMT index within its tower */
    uint16_t tower;             /* tower index in the array   */
    uint32_t n_towers;          /* towers with a causally related trigger, its own included */
} trig_array_seed;

/* Status bits (trig_array_stats.flags). */
#define TRIG_AFLAG_SEED_FULL   0x01u  /* more selected triggers than seed_cap     */
#define TRIG_AFLAG_WIN_FULL    0x02u  /* more windows than win_cap; the readback
                                         covers the first win_cap windows        */
#define TRIG_AFLAG_HIT_FULL    0x04u  /* more readback hits than hit_cap          */
#define TRIG_AFLAG_TOWER_INCOMPLETE 0x08u /* a tower slice's status was not 0: its
                                         trigger list may be incomplete         */

/* Device counters of one selection, 40 bytes. */
typedef struct {
    uint64_t n_tower_triggers;  /* triggers of all towers read                 */
    uint64_t n_selected;        /* selected triggers (may exceed seed_cap)     */
    uint64_t n_windows;         /* windows (may exceed win_cap)                */
    uint64_t n_hits;            /* readback hits of the stored windows (may exceed hit_cap) */
    uint32_t flags;             /* TRIG_AFLAG_*                                 */
    int32_t status;             /* TRIG_OK when complete, else TRIG_ECAPACITY   */
} trig_array_stats;

/* Outputs, device memory owned by the caller.  Fragment (w, b) -- tower b's
 * hits inside window w -- is hits[frag_off[w * n_towers + b] ..
 * frag_off[w * n_towers + b + 1]); frag_off has win_cap * n_towers + 1
 * entries, of which the first min(n_windows, win_cap) * n_towers + 1 are
 * written.  windows[w].n_hits counts the hits of all towers inside window w;
 * n_triggers the selected triggers inside it. */
typedef struct {
    trig_array_seed *seeds;     /* seed_cap entries, (t, tower, rank in tower) order */
    uint64_t seed_cap;
    trig_window *windows;       /* win_cap entries */
    uint64_t win_cap;
    uint64_t *frag_off;         /* win_cap * n_towers + 1 entries */
    trig_hit *hits;             /* hit_cap entries */
    uint64_t hit_cap;
    trig_array_stats *stats;    /* one entry */
} trig_array_out;

/* Group n_towers detectors (1..64, 4096 PMTs in all) into an array; tower
 * b is towers[b].  The detectors must share tol_ns, n_num and n_den, stay
 * alive as long as the array, and have their coordinates in one frame.
 * Builds the cross-tower dt_max table on the current device.  Errors:
 * TRIG_EINVAL (bad counts, mismatched constants, h above a tower's halo),
 * TRIG_ENOMEM, TRIG_EDEVICE. */
int trig_array_create(trig_detector *const *towers, uint32_t n_towers, const trig_array_params *params,
                      trig_array **out);
int trig_array_destroy(trig_array *array);

/* Device scratch bytes trig_array_select needs for these tower slices and
 * outputs (0 on bad input). */
size_t trig_array_scratch_bytes(const trig_array *array, const trig_slice_dev *slices, const trig_array_out *out);

/* Select across towers and read the windows back.  slices[b] is tower b's
 * slice (slices[b].det == towers[b]), all with the same t0_ns, already run
 * by trig_batch_run (or its no-alloc or events form) on `stream` or before
 * it.  Enqueues the selection kernels on `stream` (a cudaStream_t) and
 * returns; stats and outputs are valid once the stream reaches this point.
 * scratch is device memory, 256-byte aligned, of trig_array_scratch_bytes.
 * Errors: TRIG_EINVAL (mismatched slices, unaligned scratch),
 * TRIG_ECAPACITY (scratch too small), TRIG_EDEVICE. */
int trig_array_select(trig_array *array, const trig_slice_dev *slices, const trig_array_out *out, void *scratch,
                      size_t scratch_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TRIG_ARRAY_H */
