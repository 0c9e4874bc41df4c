/*
 * oracle.h -- CPU reference of the online muon trigger (test infrastructure).
 * Only tests, the package smoke check and the benchmark's CPU-baseline leg
 * use it.  See oracle.c for the definitions it follows.
 */
#ifndef TRIG_ORACLE_H
#define TRIG_ORACLE_H
#include <stdint.h>

typedef struct {
    int64_t t_ns;
    uint16_t pmt;
    uint16_t charge;
    uint32_t reserved;
} oracle_hit;

typedef struct {
    uint32_t q_seed_adc;      /* charge seed: charge >= q_seed_adc          */
    uint32_t floor_tau_ns;    /* floor coincidence: |dt| <= tau             */
    uint32_t tol_ns;          /* dt_max tolerance                           */
    uint32_t n_num, n_den;    /* light travel: n_num / n_den ns per metre   */
    uint32_t corr_window_ns;  /* correlation interval W (clamps dt_max)     */
    uint32_t threshold;       /* fire when c(s) >= threshold                */
    uint32_t win_half_ns;     /* event window [t - h, t + h]                */
    int64_t slice_ns;         /* owned range of a slice: [t0, t0 + S)       */
    uint32_t l0_hits;         /* level 0: N hits (0 = off) ...              */
    uint32_t l0_window_ns;    /* ... within TW ns ...                       */
    uint32_t l0_distinct_pmts;/* ... counting different PMTs only if 1      */
    uint32_t seed_rule;       /* 0: QTRIG or floor coincidence within tau;
                                 1: [SC and AFC] or [FC and AFC]            */
    uint32_t sc_window_ns;    /* SC: adjacent PMTs, |dt| <= this            */
    uint32_t fc_window_ns;    /* FC: same floor, |dt| <= this               */
    uint32_t afc_window_ns;   /* AFC: consecutive floors, |dt| <= this      */
    uint32_t sc_dist_mm;      /* adjacent: same floor, at most this apart   */
    uint32_t count_distinct_pmts; /* c(s) counts different PMTs if 1        */
    uint32_t reserved;
} oracle_params;

typedef struct {
    int64_t t_ns;
    uint16_t pmt;
    uint16_t charge;
    uint32_t count;
} oracle_seed;

typedef struct {
    int64_t lo_ns, hi_ns;     /* inclusive */
    uint64_t n_hits;
    uint64_t n_triggers;
} oracle_window;

typedef struct {
    uint64_t n_seeds, n_triggers, n_windows;
    oracle_seed *seeds;       /* every seed of the slice, with its count */
    oracle_seed *triggers;    /* seeds with count >= threshold            */
    oracle_window *windows;
} oracle_slice_result;

int64_t oracle_dtmax_pair(int64_t d2_mm2, uint32_t tol_ns, uint32_t n_num, uint32_t n_den);
int oracle_dtmax(uint32_t n_pmt, const int32_t *xyz_mm, uint32_t tol_ns, uint32_t n_num, uint32_t n_den,
                 int32_t *dt_out);
int oracle_merge(const oracle_hit *hits, uint64_t n, oracle_hit *sorted_out);
/* Largest detector the oracle takes (oracle_run returns -1 above it or at 0). */
#define ORACLE_MAX_PMT 4096u

int oracle_run(uint32_t n_pmt, const int32_t *xyz_mm, const uint32_t *floor_id, const uint32_t *tower_id,
               const oracle_params *par,
               const oracle_hit *hits, uint64_t n_hits, const int64_t *slice_t0, uint32_t n_slices,
               int n_threads, oracle_slice_result *out);
void oracle_free(oracle_slice_result *r, uint32_t n_slices);
int oracle_threads_used(int n_threads);

#endif
