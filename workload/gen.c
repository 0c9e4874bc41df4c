/*
 * gen.c -- seeded synthetic PMT hit streams for the muon-trigger workloads.
 *
 * This module only draws inputs: Poisson background per PMT, straight
 * downgoing muon tracks seen through the Cherenkov cone, and
 * bioluminescence bursts.  It contains none of the trigger's arithmetic
 * (no causality table, no seed rule, no counting, no windows); both the
 * CPU oracle and the GPU library consume what it writes.
 *
 * Random numbers: SplitMix64 seeds one xoshiro256** state per
 * (seed, stream, sub-stream) triple, so a PMT's hits do not depend on the
 * thread count.  Gaussians use Box-Muller, small Poisson counts use Knuth's
 * product method, and background hits come from exponential gaps, which
 * yields each PMT's stream already in time order.
 *
 * Hit record (16 B): int64 t_ns, uint16 pmt, uint16 charge (ADC counts,
 * 1 pe = 100), uint32 reserved.  The generator writes ground truth into
 * `reserved`: 0 for background and bursts, 1 + track index for muon hits.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t t_ns;
    uint16_t pmt;
    uint16_t charge;
    uint32_t reserved;
} gen_hit;

typedef struct {
    uint32_t n_pmt;
    const int32_t *xyz_mm;   /* 3 * n_pmt, integer millimetres            */
    int64_t t_begin_ns;      /* hits are drawn in [t_begin, t_end)        */
    int64_t t_end_ns;
    const double *rate_hz;   /* per-PMT background rate                   */
    uint32_t n_muons;
    int64_t muon_margin_ns;  /* track reference times keep this margin    */
    double muon_pe_scale;    /* mean pe at d = 0 (3.0)                     */
    double muon_att_m;       /* attenuation length (40 m)                  */
    double muon_max_d_m;     /* PMTs farther than this see nothing (100 m) */
    double muon_jitter_ns;   /* Gaussian time jitter sigma (3 ns)          */
    double cherenkov_deg;    /* cone half-angle (41 deg)                   */
    double refr_index;       /* light index in water (1.38)                */
    double box_grow_m;       /* track points lie in the PMT box grown by this (100 m) */
    uint32_t n_bursts;
    int64_t burst_len_ns;
    double burst_rate_hz;
    uint32_t burst_pmts;
    double pe_adc;           /* ADC counts per pe (100)                    */
    double pe_sigma_adc;     /* charge sigma per sqrt(pe) (40)             */
    uint64_t seed;
    uint64_t stream;
    int n_threads;
} gen_spec;

/* ---------------------------------------------------------------- PRNG */

static uint64_t splitmix64(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } rng_t;

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_u64(rng_t *r)
{
    uint64_t *s = r->s;
    uint64_t out = rotl64(s[1] * 5u, 7) * 9u;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

static void rng_init(rng_t *r, uint64_t seed, uint64_t stream, uint64_t sub)
{
    uint64_t x = seed ^ (stream * 0xD1B54A32D192ED03ull) ^ (sub * 0x8CB92BA72F3D8DD7ull);
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

/* uniform in [0, 1) with 53 random bits */
static double rng_uniform(rng_t *r) { return (double)(rng_u64(r) >> 11) * 0x1.0p-53; }
/* uniform in (0, 1) */
static double rng_uniform_open(rng_t *r) { return ((double)(rng_u64(r) >> 11) + 0.5) * 0x1.0p-53; }

static double rng_normal(rng_t *r)
{
    double u1 = rng_uniform_open(r), u2 = rng_uniform(r);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* Knuth's product method; used only for small means (muon pe <= a few). */
static uint32_t rng_poisson_small(rng_t *r, double lambda)
{
    double limit = exp(-lambda), p = 1.0;
    uint32_t k = 0;
    do {
        ++k;
        p *= rng_uniform(r);
    } while (p > limit);
    return k - 1;
}

static uint16_t charge_for_pe(rng_t *r, double npe, const gen_spec *sp)
{
    double q = sp->pe_adc * npe + sp->pe_sigma_adc * sqrt(npe) * rng_normal(r);
    double rq = (q >= 0.0) ? floor(q + 0.5) : -floor(-q + 0.5); /* half away from zero */
    if (rq < 1.0) rq = 1.0;
    if (rq > 65535.0) rq = 65535.0;
    return (uint16_t)rq;
}

/* ------------------------------------------------------- per-PMT lists */

typedef struct {
    gen_hit *v;
    uint64_t n, cap;
    int failed;
} hit_list;

static void list_push(hit_list *l, gen_hit h)
{
    if (l->failed) return;
    if (l->n == l->cap) {
        uint64_t nc = l->cap ? l->cap * 2 : 256;
        gen_hit *nv = (gen_hit *)realloc(l->v, nc * sizeof(gen_hit));
        if (!nv) { l->failed = 1; return; }
        l->v = nv;
        l->cap = nc;
    }
    l->v[l->n++] = h;
}

/* Poisson process with exponential gaps on [a, b); times floor()ed to ns. */
static void draw_poisson_process(hit_list *l, rng_t *r, uint16_t pmt, double a, double b,
                                 double rate_hz, const gen_spec *sp)
{
    if (rate_hz <= 0.0 || b <= a) return;
    double per_ns = rate_hz * 1e-9;
    double t = a;
    for (;;) {
        t += -log(rng_uniform_open(r)) / per_ns;
        if (t >= b) break;
        gen_hit h;
        h.t_ns = (int64_t)floor(t);
        if ((double)h.t_ns < a) h.t_ns = (int64_t)ceil(a);
        h.pmt = pmt;
        h.charge = charge_for_pe(r, 1.0, sp);
        h.reserved = 0;
        list_push(l, h);
    }
}

typedef struct {
    const gen_spec *sp;
    hit_list *lists;
    uint32_t next;
    pthread_mutex_t mu;
} bg_job;

static void *bg_worker(void *arg)
{
    bg_job *job = (bg_job *)arg;
    const gen_spec *sp = job->sp;
    for (;;) {
        pthread_mutex_lock(&job->mu);
        uint32_t p = job->next++;
        pthread_mutex_unlock(&job->mu);
        if (p >= sp->n_pmt) break;
        rng_t r;
        rng_init(&r, sp->seed, sp->stream, (uint64_t)p);
        draw_poisson_process(&job->lists[p], &r, (uint16_t)p, (double)sp->t_begin_ns,
                             (double)sp->t_end_ns, sp->rate_hz[p], sp);
    }
    return NULL;
}

static int cmp_hit_time(const void *a, const void *b)
{
    const gen_hit *x = (const gen_hit *)a, *y = (const gen_hit *)b;
    if (x->t_ns != y->t_ns) return x->t_ns < y->t_ns ? -1 : 1;
    if (x->reserved != y->reserved) return x->reserved < y->reserved ? -1 : 1;
    if (x->charge != y->charge) return x->charge < y->charge ? -1 : 1;
    return 0;
}

/* ------------------------------------------------------------- muons */

static void draw_muons(hit_list *lists, const gen_spec *sp)
{
    const double c_m_per_ns = 0.2998;
    const double th = sp->cherenkov_deg * 3.141592653589793 / 180.0;
    const double tan_c = tan(th), sin_c = sin(th);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (uint32_t p = 0; p < sp->n_pmt; ++p)
        for (int k = 0; k < 3; ++k) {
            double v = sp->xyz_mm[3 * p + k] * 1e-3;
            if (v < lo[k]) lo[k] = v;
            if (v > hi[k]) hi[k] = v;
        }
    for (int k = 0; k < 3; ++k) { lo[k] -= sp->box_grow_m; hi[k] += sp->box_grow_m; }

    for (uint32_t m = 0; m < sp->n_muons; ++m) {
        rng_t r;
        rng_init(&r, sp->seed, sp->stream, 0x100000000ull + m);
        double cos_t = rng_uniform(&r);               /* downgoing, isotropic */
        double sin_t = sqrt(fmax(0.0, 1.0 - cos_t * cos_t));
        double phi = 6.283185307179586 * rng_uniform(&r);
        double u[3] = {sin_t * cos(phi), sin_t * sin(phi), -cos_t};
        double p0[3];
        for (int k = 0; k < 3; ++k) p0[k] = lo[k] + (hi[k] - lo[k]) * rng_uniform(&r);
        double ta = (double)(sp->t_begin_ns + sp->muon_margin_ns);
        double tb = (double)(sp->t_end_ns - sp->muon_margin_ns);
        double t_ref = ta + (tb - ta) * rng_uniform(&r);
        for (uint32_t p = 0; p < sp->n_pmt; ++p) {
            double v[3];
            for (int k = 0; k < 3; ++k) v[k] = sp->xyz_mm[3 * p + k] * 1e-3 - p0[k];
            double l = v[0] * u[0] + v[1] * u[1] + v[2] * u[2];
            double w[3] = {v[0] - l * u[0], v[1] - l * u[1], v[2] - l * u[2]};
            double d = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
            if (d > sp->muon_max_d_m) continue;
            double att = exp(-d / sp->muon_att_m);
            if (rng_uniform(&r) >= att) continue;
            uint32_t npe = rng_poisson_small(&r, sp->muon_pe_scale * att) + 1;
            double t = t_ref + (l - d / tan_c) / c_m_per_ns + (d / sin_c) * sp->refr_index / c_m_per_ns +
                       sp->muon_jitter_ns * rng_normal(&r);
            int64_t ti = (int64_t)floor(t + 0.5);
            if (ti < sp->t_begin_ns || ti >= sp->t_end_ns) continue;
            gen_hit h;
            h.t_ns = ti;
            h.pmt = (uint16_t)p;
            h.charge = charge_for_pe(&r, (double)npe, sp);
            h.reserved = 1u + m;
            list_push(&lists[p], h);
        }
    }
}

static void draw_bursts(hit_list *lists, const gen_spec *sp)
{
    for (uint32_t b = 0; b < sp->n_bursts; ++b) {
        rng_t r;
        rng_init(&r, sp->seed, sp->stream, 0x200000000ull + b);
        double span = (double)(sp->t_end_ns - sp->t_begin_ns - sp->burst_len_ns);
        if (span < 0) span = 0;
        double a = (double)sp->t_begin_ns + span * rng_uniform(&r);
        uint32_t k = sp->burst_pmts < sp->n_pmt ? sp->burst_pmts : sp->n_pmt;
        uint32_t chosen[64];
        if (k > 64) k = 64;
        for (uint32_t i = 0; i < k; ++i) {
            for (;;) {
                uint32_t c = (uint32_t)(rng_u64(&r) % sp->n_pmt);
                int dup = 0;
                for (uint32_t j = 0; j < i; ++j) dup |= chosen[j] == c;
                if (!dup) { chosen[i] = c; break; }
            }
            rng_t rp;
            rng_init(&rp, sp->seed, sp->stream, 0x300000000ull + ((uint64_t)b << 16) + i);
            draw_poisson_process(&lists[chosen[i]], &rp, (uint16_t)chosen[i], a,
                                 a + (double)sp->burst_len_ns, sp->burst_rate_hz, sp);
        }
    }
}

/* ----------------------------------------------------------- public API */

typedef struct {
    uint32_t n_pmt;
    hit_list *lists;
} gen_result;

void gen_stream_free(void *handle)
{
    gen_result *res = (gen_result *)handle;
    if (!res) return;
    for (uint32_t p = 0; p < res->n_pmt; ++p) free(res->lists[p].v);
    free(res->lists);
    free(res);
}

/* Draws one stream; returns an opaque handle (NULL on failure) and the hit count. */
void *gen_stream(const gen_spec *sp, uint64_t *n_hits_out)
{
    if (!sp || !n_hits_out || sp->n_pmt == 0 || sp->n_pmt > 65536 || sp->t_end_ns < sp->t_begin_ns)
        return NULL;
    gen_result *res = (gen_result *)calloc(1, sizeof(gen_result));
    if (!res) return NULL;
    res->n_pmt = sp->n_pmt;
    res->lists = (hit_list *)calloc(sp->n_pmt, sizeof(hit_list));
    if (!res->lists) { free(res); return NULL; }

    bg_job job;
    job.sp = sp;
    job.lists = res->lists;
    job.next = 0;
    pthread_mutex_init(&job.mu, NULL);
    int nt = sp->n_threads > 0 ? sp->n_threads : 1;
    if (nt > 256) nt = 256;
    pthread_t th[256];
    int started = 0;
    for (int i = 1; i < nt; ++i)
        if (pthread_create(&th[i], NULL, bg_worker, &job) == 0) ++started; else break;
    bg_worker(&job);
    for (int i = 1; i <= started; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&job.mu);

    draw_muons(res->lists, sp);
    draw_bursts(res->lists, sp);

    uint64_t total = 0;
    for (uint32_t p = 0; p < sp->n_pmt; ++p) {
        hit_list *l = &res->lists[p];
        if (l->failed) { gen_stream_free(res); return NULL; }
        /* background arrives sorted; muon and burst hits were appended */
        qsort(l->v, l->n, sizeof(gen_hit), cmp_hit_time);
        total += l->n;
    }
    *n_hits_out = total;
    return res;
}

/* Copies the stream out as CSR grouped by PMT: hits[pmt_off[p] .. pmt_off[p+1]). */
void gen_stream_copy(void *handle, gen_hit *hits, uint64_t *pmt_off)
{
    gen_result *res = (gen_result *)handle;
    uint64_t o = 0;
    for (uint32_t p = 0; p < res->n_pmt; ++p) {
        pmt_off[p] = o;
        if (res->lists[p].n) memcpy(hits + o, res->lists[p].v, res->lists[p].n * sizeof(gen_hit));
        o += res->lists[p].n;
    }
    pmt_off[res->n_pmt] = o;
}
