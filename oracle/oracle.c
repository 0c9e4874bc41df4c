/*
 * oracle.c -- plain, slow CPU reference of the online muon trigger.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code with the CUDA
 * library: it is written from the method's definition, in the plainest form
 * that can be checked against the paper by eye.
 *
 * What it computes (arXiv 1411.3968, "Muon trigger strategy" and "Sorting
 * and triggering in GPU"; the constants the paper leaves open are inputs):
 *
 *   H       all hits of a detector run (the merged PMT streams).
 *   merge   H ordered by time -- the Hit Manager's merge of the PMT streams
 *           into time slices ("DAQ system of NEMO Phase II").  Here a plain
 *           library sort by (t, pmt, charge); ties keep input order.
 *   dt_max  dt_max[i][j] = tol + ceil(d_ij * n_num / (n_den * 1000)) ns for
 *           PMTs d_ij millimetres apart (the light's travel time in water
 *           plus a tolerance).  Computed exactly in integers: the smallest
 *           k >= 0 with (k * n_den * 1000)^2 >= (n_num * d)^2, so no
 *           floating-point rounding reaches the table.
 *   seed    hit s in the slice's owned range [T0, T0 + S) with
 *           charge >= q_seed (charge over threshold, QTRIG) or another hit
 *           j on a different PMT of the same floor with |t_j - t_s| <= tau
 *           (the floor coincidence).
 *   count   c(s) = #{ j in H : |t_j - t_s| <= min(dt_max[p_s][p_j], W) },
 *           W the 3 us correlation interval; s itself and hits on its own
 *           PMT are included.  Obtained by testing every hit in
 *           [t_s - W, t_s + W] -- the brute force over the window.
 *   level 0 (optional, "Muon trigger strategy": N hits in a fixed time
 *           window TW, N7TW1000, applied before the other triggers; its
 *           DN variant counts different PMTs): a seed is kept only if some
 *           window [a, a + TW) that contains it holds at least N hits (N
 *           different PMTs).  Only windows starting at a hit need testing:
 *           moving a window's start up to its first hit loses nothing.
 *   ladder  (seed_rule 1, the combination of "Sorting and triggering in
 *           GPU" and "Results and perspectives": N7TW1000, then [SC and
 *           AFC] or [FC and AFC]) replaces the seed rule above: hit s is a
 *           seed iff some hit on a consecutive floor of its tower lies within
 *           the AFC window (AFC), and some hit on an adjacent PMT lies within
 *           the SC window (SC) or some hit on another PMT of its floor within
 *           the FC window (FC).  Adjacent PMTs: different PMTs of one floor
 *           at most sc_dist apart.  Consecutive floors: floors of one tower
 *           next to each other when the tower's floors are ordered by
 *           height (the z of a floor's lowest PMT), ties by floor id.
 *           Level 0 then applies as above.
 *   distinct (count_distinct_pmts, the distinct-PMT variant of the count):
 *           c(s) = the number of different PMTs among the hits j above.
 *   trigger seeds with c(s) >= threshold, in (t, pmt, charge) order.
 *   windows [t_s - h, t_s + h] around every trigger (the 6 us window centred
 *           on the seed), merged while lo_next <= hi_cur + 1; n_hits counts
 *           the hits of H inside each merged window.
 *
 * Slices are independent; a pool of POSIX threads takes them one at a time.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <unistd.h>

#include "oracle.h"

/* ------------------------------------------------------------ dt_max */

/* (k * n_den * 1000)^2 >= (n_num * d)^2, with d^2 = d2 given in mm^2 */
static int covers(uint64_t k, uint64_t n_num, uint64_t n_den, uint64_t d2)
{
    unsigned __int128 lhs = (unsigned __int128)(k * n_den * 1000u) * (k * n_den * 1000u);
    unsigned __int128 rhs = (unsigned __int128)(n_num * n_num) * d2;
    return lhs >= rhs;
}

int64_t oracle_dtmax_pair(int64_t d2_mm2, uint32_t tol_ns, uint32_t n_num, uint32_t n_den)
{
    if (d2_mm2 < 0 || n_den == 0) return -1;
    /* start near the answer, then walk to the smallest k that covers d */
    double est = (double)n_num * sqrt((double)d2_mm2) / ((double)n_den * 1000.0);
    uint64_t k = est > 2.0 ? (uint64_t)est - 2u : 0u;
    while (k > 0 && covers(k - 1, n_num, n_den, (uint64_t)d2_mm2)) --k;
    while (!covers(k, n_num, n_den, (uint64_t)d2_mm2)) ++k;
    return (int64_t)tol_ns + (int64_t)k;
}

int oracle_dtmax(uint32_t n_pmt, const int32_t *xyz_mm, uint32_t tol_ns, uint32_t n_num, uint32_t n_den,
                 int32_t *dt_out)
{
    if (!xyz_mm || !dt_out || n_den == 0) return -1;
    for (uint32_t i = 0; i < n_pmt; ++i) {
        for (uint32_t j = 0; j < n_pmt; ++j) {
            int64_t d2 = 0;
            for (int c = 0; c < 3; ++c) {
                int64_t dx = (int64_t)xyz_mm[3 * i + c] - (int64_t)xyz_mm[3 * j + c];
                d2 += dx * dx;
            }
            int64_t v = oracle_dtmax_pair(d2, tol_ns, n_num, n_den);
            dt_out[(size_t)i * n_pmt + j] = v > INT32_MAX ? INT32_MAX : (int32_t)v;
        }
    }
    return 0;
}

/* -------------------------------------------------------------- merge */

typedef struct {
    oracle_hit h;
    uint64_t idx;
} keyed_hit;

static int cmp_keyed(const void *a, const void *b)
{
    const keyed_hit *x = (const keyed_hit *)a, *y = (const keyed_hit *)b;
    if (x->h.t_ns != y->h.t_ns) return x->h.t_ns < y->h.t_ns ? -1 : 1;
    if (x->h.pmt != y->h.pmt) return x->h.pmt < y->h.pmt ? -1 : 1;
    if (x->h.charge != y->h.charge) return x->h.charge < y->h.charge ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

int oracle_merge(const oracle_hit *hits, uint64_t n, oracle_hit *sorted_out)
{
    if (n && (!hits || !sorted_out)) return -1;
    keyed_hit *k = (keyed_hit *)malloc((n ? n : 1) * sizeof(keyed_hit));
    if (!k) return -2;
    for (uint64_t i = 0; i < n; ++i) { k[i].h = hits[i]; k[i].idx = i; }
    qsort(k, n, sizeof(keyed_hit), cmp_keyed);
    for (uint64_t i = 0; i < n; ++i) sorted_out[i] = k[i].h;
    free(k);
    return 0;
}

/* first index i with sorted[i].t_ns >= t */
static uint64_t lower_bound_t(const oracle_hit *s, uint64_t n, int64_t t)
{
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (s[mid].t_ns < t) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* ------------------------------------------------------------ trigger */

typedef struct {
    uint32_t n_pmt;
    const uint32_t *floor_id;
    const uint32_t *tower_id;   /* n_pmt, or NULL: a single tower */
    const int32_t *xyz_mm;
    const uint32_t *floor_rank; /* n_pmt: rank of p's floor among its tower's floors */
    const int32_t *dt;          /* n_pmt * n_pmt, exact dt_max */
    const oracle_params *par;
    const oracle_hit *sorted;
    uint64_t n;
    const int64_t *slice_t0;
    uint32_t n_slices;
    oracle_slice_result *out;
    uint32_t next;
    int error;
    pthread_mutex_t mu;
} run_job;

static int push_seed(oracle_seed **v, uint64_t *n, uint64_t *cap, oracle_seed s)
{
    if (*n == *cap) {
        uint64_t nc = *cap ? *cap * 2 : 64;
        oracle_seed *nv = (oracle_seed *)realloc(*v, nc * sizeof(oracle_seed));
        if (!nv) return -1;
        *v = nv;
        *cap = nc;
    }
    (*v)[(*n)++] = s;
    return 0;
}

/* Level 0 at the seed H[s]: some window [t_j, t_j + TW) with
 * t_s - TW < t_j <= t_s holds at least N hits (N different PMTs). */
static int level0_pass(const run_job *job, uint64_t s)
{
    const oracle_params *par = job->par;
    const oracle_hit *H = job->sorted;
    const uint64_t n = job->n;
    const int64_t ts = H[s].t_ns, TW = par->l0_window_ns;
    for (uint64_t j = lower_bound_t(H, n, ts - TW + 1); j < n && H[j].t_ns <= ts; ++j) {
        const int64_t a = H[j].t_ns;
        const uint64_t b = lower_bound_t(H, n, a);        /* every hit of the window */
        uint32_t count = 0;
        if (!par->l0_distinct_pmts) {
            for (uint64_t q = b; q < n && H[q].t_ns < a + TW; ++q) ++count;
        } else {
            unsigned char seen[ORACLE_MAX_PMT];
            memset(seen, 0, job->n_pmt);
            for (uint64_t q = b; q < n && H[q].t_ns < a + TW; ++q)
                if (!seen[H[q].pmt]) { seen[H[q].pmt] = 1; ++count; }
        }
        if (count >= par->l0_hits) return 1;
    }
    return 0;
}

static uint32_t tower_of(const run_job *job, uint32_t p)
{
    return job->tower_id ? job->tower_id[p] : 0u;
}

/* Different PMTs of one floor at most sc_dist_mm apart. */
static int adjacent_pmts(const run_job *job, uint32_t p, uint32_t q)
{
    if (p == q || job->floor_id[p] != job->floor_id[q]) return 0;
    const int64_t dx = (int64_t)job->xyz_mm[3 * p] - job->xyz_mm[3 * q];
    const int64_t dy = (int64_t)job->xyz_mm[3 * p + 1] - job->xyz_mm[3 * q + 1];
    const int64_t dz = (int64_t)job->xyz_mm[3 * p + 2] - job->xyz_mm[3 * q + 2];
    const int64_t r = job->par->sc_dist_mm;
    return dx * dx + dy * dy + dz * dz <= r * r;
}

/* PMTs on two floors of one tower that are next to each other in height. */
static int consecutive_floors(const run_job *job, uint32_t p, uint32_t q)
{
    if (tower_of(job, p) != tower_of(job, q)) return 0;
    const int64_t a = job->floor_rank[p], b = job->floor_rank[q];
    return a - b == 1 || b - a == 1;
}

/* The paper's combination at H[s]: [SC and AFC] or [FC and AFC]. */
static int ladder_seed(const run_job *job, uint64_t s)
{
    const oracle_params *par = job->par;
    const oracle_hit *H = job->sorted;
    const uint64_t n = job->n;
    const int64_t ts = H[s].t_ns;
    int64_t wmax = par->sc_window_ns;
    if (par->fc_window_ns > wmax) wmax = par->fc_window_ns;
    if (par->afc_window_ns > wmax) wmax = par->afc_window_ns;
    int sc = 0, fc = 0, afc = 0;
    for (uint64_t j = lower_bound_t(H, n, ts - wmax); j < n && H[j].t_ns <= ts + wmax; ++j) {
        if (j == s) continue;
        int64_t d = H[j].t_ns - ts;
        if (d < 0) d = -d;
        const uint32_t p = H[s].pmt, q = H[j].pmt;
        if (d <= par->sc_window_ns && adjacent_pmts(job, p, q)) sc = 1;
        if (d <= par->fc_window_ns && p != q && job->floor_id[p] == job->floor_id[q]) fc = 1;
        if (d <= par->afc_window_ns && consecutive_floors(job, p, q)) afc = 1;
    }
    return (sc && afc) || (fc && afc);
}

static int run_slice(run_job *job, uint32_t k)
{
    const oracle_params *par = job->par;
    const oracle_hit *H = job->sorted;
    const uint64_t n = job->n;
    const int64_t T0 = job->slice_t0[k];
    const int64_t T1 = T0 + par->slice_ns;
    const int64_t tau = par->floor_tau_ns;
    const int64_t W = par->corr_window_ns;
    oracle_slice_result *res = &job->out[k];
    memset(res, 0, sizeof(*res));

    uint64_t cap_s = 0, cap_t = 0;
    uint64_t first = lower_bound_t(H, n, T0);
    uint64_t last = lower_bound_t(H, n, T1);
    for (uint64_t s = first; s < last; ++s) {
        const oracle_hit *hs = &H[s];
        int is_seed = par->seed_rule == 1 ? ladder_seed(job, s) : hs->charge >= par->q_seed_adc;
        if (!is_seed && par->seed_rule != 1) {
            for (uint64_t j = lower_bound_t(H, n, hs->t_ns - tau); j < n && H[j].t_ns <= hs->t_ns + tau; ++j) {
                if (j == s) continue;
                if (H[j].pmt != hs->pmt && job->floor_id[H[j].pmt] == job->floor_id[hs->pmt]) {
                    is_seed = 1;
                    break;
                }
            }
        }
        if (is_seed && par->l0_hits > 0) is_seed = level0_pass(job, s);
        if (!is_seed) continue;
        uint32_t c = 0;
        unsigned char seen[ORACLE_MAX_PMT];
        if (par->count_distinct_pmts) memset(seen, 0, job->n_pmt);
        for (uint64_t j = lower_bound_t(H, n, hs->t_ns - W); j < n && H[j].t_ns <= hs->t_ns + W; ++j) {
            int64_t lim = job->dt[(size_t)hs->pmt * job->n_pmt + H[j].pmt];
            if (lim > W) lim = W;
            int64_t dtj = H[j].t_ns - hs->t_ns;
            if (dtj < 0) dtj = -dtj;
            if (dtj > lim) continue;
            if (!par->count_distinct_pmts) ++c;
            else if (!seen[H[j].pmt]) { seen[H[j].pmt] = 1; ++c; }
        }
        oracle_seed sd = {hs->t_ns, hs->pmt, hs->charge, c};
        if (push_seed(&res->seeds, &res->n_seeds, &cap_s, sd)) return -2;
        if (c >= par->threshold && push_seed(&res->triggers, &res->n_triggers, &cap_t, sd)) return -2;
    }

    /* windows around the triggers, which are already in time order */
    const int64_t h = par->win_half_ns;
    res->windows = (oracle_window *)malloc((res->n_triggers ? res->n_triggers : 1) * sizeof(oracle_window));
    if (!res->windows) return -2;
    for (uint64_t i = 0; i < res->n_triggers; ++i) {
        int64_t lo = res->triggers[i].t_ns - h, hi = res->triggers[i].t_ns + h;
        if (res->n_windows > 0 && lo <= res->windows[res->n_windows - 1].hi_ns + 1) {
            oracle_window *w = &res->windows[res->n_windows - 1];
            if (hi > w->hi_ns) w->hi_ns = hi;
            w->n_triggers += 1;
        } else {
            oracle_window w = {lo, hi, 0, 1};
            res->windows[res->n_windows++] = w;
        }
    }
    for (uint64_t i = 0; i < res->n_windows; ++i) {
        oracle_window *w = &res->windows[i];
        w->n_hits = lower_bound_t(H, n, w->hi_ns + 1) - lower_bound_t(H, n, w->lo_ns);
    }
    return 0;
}

static void *run_worker(void *arg)
{
    run_job *job = (run_job *)arg;
    for (;;) {
        pthread_mutex_lock(&job->mu);
        uint32_t k = job->next++;
        pthread_mutex_unlock(&job->mu);
        if (k >= job->n_slices) break;
        int rc = run_slice(job, k);
        if (rc) {
            pthread_mutex_lock(&job->mu);
            job->error = rc;
            pthread_mutex_unlock(&job->mu);
        }
    }
    return NULL;
}

/* Floor order of the towers: rank[p] = how many different floors of p's
 * tower lie below p's floor, floors compared by (height, floor id), the
 * height of a floor being the z of its lowest PMT. */
static void floor_ranks(uint32_t n_pmt, const int32_t *xyz_mm, const uint32_t *floor_id, const uint32_t *tower_id,
                        uint32_t *rank)
{
    int64_t *height = (int64_t *)malloc(n_pmt * sizeof(int64_t));
    unsigned char *counted = (unsigned char *)malloc(n_pmt);
    if (!height || !counted) { free(height); free(counted); memset(rank, 0, n_pmt * sizeof(uint32_t)); return; }
    for (uint32_t p = 0; p < n_pmt; ++p) {
        height[p] = xyz_mm[3 * p + 2];
        for (uint32_t q = 0; q < n_pmt; ++q)
            if (floor_id[q] == floor_id[p] && xyz_mm[3 * q + 2] < height[p]) height[p] = xyz_mm[3 * q + 2];
    }
    for (uint32_t p = 0; p < n_pmt; ++p) {
        const uint32_t tp = tower_id ? tower_id[p] : 0u;
        memset(counted, 0, n_pmt);
        rank[p] = 0;
        for (uint32_t q = 0; q < n_pmt; ++q) {
            if ((tower_id ? tower_id[q] : 0u) != tp) continue;
            const int below = height[q] < height[p] || (height[q] == height[p] && floor_id[q] < floor_id[p]);
            if (!below) continue;
            /* count each floor once: its first PMT of this tower */
            uint32_t first = q;
            for (uint32_t r = 0; r < q; ++r)
                if (floor_id[r] == floor_id[q] && (tower_id ? tower_id[r] : 0u) == tp) { first = r; break; }
            if (!counted[first]) { counted[first] = 1; ++rank[p]; }
        }
    }
    free(height);
    free(counted);
}

int oracle_run(uint32_t n_pmt, const int32_t *xyz_mm, const uint32_t *floor_id, const uint32_t *tower_id,
               const oracle_params *par, const oracle_hit *hits, uint64_t n_hits, const int64_t *slice_t0,
               uint32_t n_slices, int n_threads, oracle_slice_result *out)
{
    if (!xyz_mm || !floor_id || !par || (n_hits && !hits) || (n_slices && (!slice_t0 || !out)))
        return -1;
    /* the distinct-PMT forms mark PMTs in a 4096-entry array per seed */
    if (n_pmt == 0 || n_pmt > ORACLE_MAX_PMT) return -1;
    for (uint64_t i = 0; i < n_hits; ++i)
        if (hits[i].pmt >= n_pmt) return -1;
    memset(out, 0, n_slices * sizeof(oracle_slice_result));

    int32_t *dt = (int32_t *)malloc(((size_t)n_pmt * n_pmt ? (size_t)n_pmt * n_pmt : 1) * sizeof(int32_t));
    oracle_hit *sorted = (oracle_hit *)malloc((n_hits ? n_hits : 1) * sizeof(oracle_hit));
    if (!dt || !sorted) { free(dt); free(sorted); return -2; }
    oracle_dtmax(n_pmt, xyz_mm, par->tol_ns, par->n_num, par->n_den, dt);
    uint32_t *rank = (uint32_t *)malloc((n_pmt ? n_pmt : 1) * sizeof(uint32_t));
    if (!rank) { free(dt); free(sorted); return -2; }
    if (par->seed_rule == 1) floor_ranks(n_pmt, xyz_mm, floor_id, tower_id, rank);
    int rc = oracle_merge(hits, n_hits, sorted);
    if (rc) { free(dt); free(sorted); free(rank); return rc; }

    run_job job;
    job.n_pmt = n_pmt;
    job.floor_id = floor_id;
    job.tower_id = tower_id;
    job.xyz_mm = xyz_mm;
    job.floor_rank = rank;
    job.dt = dt;
    job.par = par;
    job.sorted = sorted;
    job.n = n_hits;
    job.slice_t0 = slice_t0;
    job.n_slices = n_slices;
    job.out = out;
    job.next = 0;
    job.error = 0;
    pthread_mutex_init(&job.mu, NULL);
    int nt = n_threads > 0 ? n_threads : (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nt < 1) nt = 1;
    if (nt > 512) nt = 512;
    if ((uint32_t)nt > n_slices) nt = n_slices ? (int)n_slices : 1;
    pthread_t th[512];
    int started = 0;
    for (int i = 1; i < nt; ++i)
        if (pthread_create(&th[i], NULL, run_worker, &job) == 0) ++started; else break;
    run_worker(&job);
    for (int i = 1; i <= started; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&job.mu);
    free(dt);
    free(sorted);
    free(rank);
    if (job.error) { oracle_free(out, n_slices); return job.error; }
    return 0;
}

void oracle_free(oracle_slice_result *r, uint32_t n_slices)
{
    if (!r) return;
    for (uint32_t k = 0; k < n_slices; ++k) {
        free(r[k].seeds);
        free(r[k].triggers);
        free(r[k].windows);
        memset(&r[k], 0, sizeof(r[k]));
    }
}

int oracle_threads_used(int n_threads)
{
    int nt = n_threads > 0 ? n_threads : (int)sysconf(_SC_NPROCESSORS_ONLN);
    return nt < 1 ? 1 : nt;
}
