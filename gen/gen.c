/*
 * Seeded synthetic string generators shared by the CPU oracle tests, the GPU
 * tests and the benchmark.  This file holds no sorting arithmetic: it only
 * produces zero-terminated byte strings.
 *
 * Every string i draws from its own xoshiro256** stream seeded from
 * (seed, i) through splitmix64, so the output does not depend on the number
 * of threads used to produce it.  Two passes are made with the same streams:
 * gen_lengths() reports each string's size (terminator included) and
 * gen_fill() writes the bytes at caller-chosen offsets.
 *
 * Kinds (workload shapes):
 *   1  uniform:  length uniform in [8,20] characters, bytes uniform 'a'..'z'
 *                (shaped after the paper's "Random" instance, Sec. 4).
 *   2  url-like: host from a pool of 2,000 host strings drawn Zipf(s=1.1),
 *                then 1..6 "/"-separated segments of 3..12 chars [a-z0-9]
 *                drawn Zipf(s=1.1) from a pool of 50,000 segments
 *                (shaped after the paper's URL instances, Table 1).
 *   3  dna:      64 characters over {A,C,G,T} from an order-3 Markov chain
 *                with seeded random transition rows; the last tenth of the
 *                strings are exact copies of uniformly chosen originals and
 *                all strings are shuffled into random positions
 *                (shaped after the paper's Sinha DNA instance, Table 1).
 *
 * Compiled with -ffp-contract=off so that the few floating point steps
 * (Zipf tables, Markov thresholds) round the same way on x86-64 and Arm.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ RNG */

static inline uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } rng_t;

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t result = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

static void rng_seed(rng_t *r, uint64_t seed, uint64_t stream) {
    uint64_t x = seed * 0xD1B54A32D192ED03ull ^ (stream + 0x8CB92BA72F3D8DD7ull) * 0x9E3779B97F4A7C15ull;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64_next(&x);
}

/* uniform integer in [0, n) */
static inline uint64_t rng_below(rng_t *r, uint64_t n) {
    return (uint64_t)(((__uint128_t)rng_next(r) * n) >> 64);
}

/* uniform double in [0, 1) */
static inline double rng_unit(rng_t *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

/* stream ids for the pools, far away from per-string stream ids */
#define STREAM_HOSTS 0x7000000000000000ull
#define STREAM_SEGS 0x7100000000000000ull
#define STREAM_TRANS 0x7200000000000000ull
#define STREAM_DUPS 0x7300000000000000ull
#define STREAM_SHUF 0x7400000000000000ull

/* ---------------------------------------------------------------- Zipf */

typedef struct { double *cdf; uint32_t n; } zipf_t;

static int zipf_init(zipf_t *z, uint32_t n, double s) {
    z->n = n;
    z->cdf = (double *)malloc(sizeof(double) * n);
    if (!z->cdf) return -1;
    double acc = 0.0;
    for (uint32_t k = 0; k < n; k++) {
        acc += pow((double)(k + 1), -s);
        z->cdf[k] = acc;
    }
    for (uint32_t k = 0; k < n; k++) z->cdf[k] /= acc;
    z->cdf[n - 1] = 1.0;
    return 0;
}

static inline uint32_t zipf_draw(const zipf_t *z, rng_t *r) {
    double u = rng_unit(r);
    uint32_t lo = 0, hi = z->n - 1;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (z->cdf[mid] > u) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* ------------------------------------------------------------ url pools */

#define URL_HOSTS 2000u
#define URL_SEGS 50000u
#define URL_MAX_SEGS 6

static const char *const kTlds[] = {".com", ".org", ".net", ".de", ".edu", ".gov",
                                    ".io", ".info", ".co.uk", ".fr", ".jp", ".ru"};
static const char kAlnum[] = "abcdefghijklmnopqrstuvwxyz0123456789";

typedef struct {
    char *host_bytes; uint32_t *host_off; uint32_t *host_len;
    char *seg_bytes; uint32_t *seg_off; uint32_t *seg_len;
    zipf_t zh, zs;
} url_pools_t;

static void url_pools_free(url_pools_t *p) {
    free(p->host_bytes); free(p->host_off); free(p->host_len);
    free(p->seg_bytes); free(p->seg_off); free(p->seg_len);
    free(p->zh.cdf); free(p->zs.cdf);
    memset(p, 0, sizeof(*p));
}

static int url_pools_init(url_pools_t *p, uint64_t seed) {
    memset(p, 0, sizeof(*p));
    p->host_bytes = (char *)malloc(URL_HOSTS * 64);
    p->host_off = (uint32_t *)malloc(sizeof(uint32_t) * URL_HOSTS);
    p->host_len = (uint32_t *)malloc(sizeof(uint32_t) * URL_HOSTS);
    p->seg_bytes = (char *)malloc(URL_SEGS * 16);
    p->seg_off = (uint32_t *)malloc(sizeof(uint32_t) * URL_SEGS);
    p->seg_len = (uint32_t *)malloc(sizeof(uint32_t) * URL_SEGS);
    if (!p->host_bytes || !p->host_off || !p->host_len || !p->seg_bytes || !p->seg_off || !p->seg_len) {
        url_pools_free(p);
        return -1;
    }
    uint32_t pos = 0;
    for (uint32_t h = 0; h < URL_HOSTS; h++) {
        rng_t r;
        rng_seed(&r, seed, STREAM_HOSTS + h);
        char *o = p->host_bytes + pos;
        uint32_t len = 0;
        const char *scheme = rng_below(&r, 10) < 7 ? "http://" : "https://";
        for (const char *c = scheme; *c; c++) o[len++] = *c;
        if (rng_below(&r, 10) < 6) { o[len++] = 'w'; o[len++] = 'w'; o[len++] = 'w'; o[len++] = '.'; }
        uint32_t name = 8 + (uint32_t)rng_below(&r, 17);
        o[len++] = (char)('a' + rng_below(&r, 26));
        for (uint32_t i = 1; i < name; i++) o[len++] = kAlnum[rng_below(&r, 36)];
        const char *tld = kTlds[rng_below(&r, sizeof(kTlds) / sizeof(kTlds[0]))];
        for (const char *c = tld; *c; c++) o[len++] = *c;
        p->host_off[h] = pos;
        p->host_len[h] = len;
        pos += 64;
    }
    pos = 0;
    for (uint32_t s = 0; s < URL_SEGS; s++) {
        rng_t r;
        rng_seed(&r, seed, STREAM_SEGS + s);
        uint32_t len = 3 + (uint32_t)rng_below(&r, 10);
        for (uint32_t i = 0; i < len; i++) p->seg_bytes[pos + i] = kAlnum[rng_below(&r, 36)];
        p->seg_off[s] = pos;
        p->seg_len[s] = len;
        pos += 16;
    }
    if (zipf_init(&p->zh, URL_HOSTS, 1.1) || zipf_init(&p->zs, URL_SEGS, 1.1)) {
        url_pools_free(p);
        return -1;
    }
    return 0;
}

typedef struct { uint32_t host; uint32_t nseg; uint32_t seg[URL_MAX_SEGS]; } url_spec_t;

static inline uint32_t url_spec(const url_pools_t *p, uint64_t seed, uint64_t i, url_spec_t *sp) {
    rng_t r;
    rng_seed(&r, seed, i);
    sp->host = zipf_draw(&p->zh, &r);
    sp->nseg = 1 + (uint32_t)rng_below(&r, URL_MAX_SEGS);
    uint32_t len = p->host_len[sp->host];
    for (uint32_t k = 0; k < sp->nseg; k++) {
        sp->seg[k] = zipf_draw(&p->zs, &r);
        len += 1 + p->seg_len[sp->seg[k]];
    }
    return len + 1; /* terminator */
}

/* ------------------------------------------------------------- dna model */

typedef struct { double cum[64][4]; } dna_model_t;

static void dna_model_init(dna_model_t *m, uint64_t seed) {
    rng_t r;
    rng_seed(&r, seed, STREAM_TRANS);
    for (int c = 0; c < 64; c++) {
        double w[4], s = 0.0;
        for (int a = 0; a < 4; a++) { w[a] = 1.0 + (double)rng_below(&r, 1000); s += w[a]; }
        double acc = 0.0;
        for (int a = 0; a < 4; a++) { acc += w[a] / s; m->cum[c][a] = acc; }
        m->cum[c][3] = 1.0;
    }
}

static const char kDna[4] = {'A', 'C', 'G', 'T'};

static void dna_write(const dna_model_t *m, uint64_t seed, uint64_t orig, uint8_t *o) {
    rng_t r;
    rng_seed(&r, seed, orig);
    uint32_t ctx = 0;
    for (int i = 0; i < 64; i++) {
        uint32_t a;
        if (i < 3) {
            a = (uint32_t)rng_below(&r, 4);
        } else {
            double u = rng_unit(&r);
            a = 0;
            while (a < 3 && m->cum[ctx][a] <= u) a++;
        }
        o[i] = (uint8_t)kDna[a];
        ctx = ((ctx << 2) | a) & 63u;
    }
    o[64] = 0;
}

/* the position -> original map of the dna workload: the first n - n/10
 * positions hold originals, the rest copies of uniformly chosen originals,
 * then everything is Fisher-Yates shuffled */
static uint32_t *dna_sources(uint64_t n, uint64_t seed) {
    uint32_t *src = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    if (!src) return NULL;
    uint64_t n_orig = n - n / 10;
    if (n_orig == 0) n_orig = n;
    rng_t r;
    rng_seed(&r, seed, STREAM_DUPS);
    for (uint64_t p = 0; p < n; p++) src[p] = (uint32_t)(p < n_orig ? p : rng_below(&r, n_orig));
    rng_seed(&r, seed, STREAM_SHUF);
    for (uint64_t p = n; p > 1; p--) {
        uint64_t q = rng_below(&r, p);
        uint32_t t = src[p - 1]; src[p - 1] = src[q]; src[q] = t;
    }
    return src;
}

/* ------------------------------------------------------------- threading */

typedef struct {
    int kind; uint64_t seed; uint64_t lo, hi;
    uint32_t *lens; const uint64_t *offsets; uint8_t *chars;
    const url_pools_t *pools; const dna_model_t *dna; const uint32_t *src;
} job_t;

static void *job_run(void *arg) {
    job_t *j = (job_t *)arg;
    for (uint64_t i = j->lo; i < j->hi; i++) {
        if (j->kind == 1) {
            rng_t r;
            rng_seed(&r, j->seed, i);
            uint32_t len = 8 + (uint32_t)rng_below(&r, 13);
            if (j->lens) { j->lens[i] = len + 1; continue; }
            uint8_t *o = j->chars + j->offsets[i];
            for (uint32_t k = 0; k < len; k++) o[k] = (uint8_t)('a' + rng_below(&r, 26));
            o[len] = 0;
        } else if (j->kind == 2) {
            url_spec_t sp;
            uint32_t len = url_spec(j->pools, j->seed, i, &sp);
            if (j->lens) { j->lens[i] = len; continue; }
            uint8_t *o = j->chars + j->offsets[i];
            const url_pools_t *p = j->pools;
            memcpy(o, p->host_bytes + p->host_off[sp.host], p->host_len[sp.host]);
            o += p->host_len[sp.host];
            for (uint32_t k = 0; k < sp.nseg; k++) {
                *o++ = '/';
                memcpy(o, p->seg_bytes + p->seg_off[sp.seg[k]], p->seg_len[sp.seg[k]]);
                o += p->seg_len[sp.seg[k]];
            }
            *o = 0;
        } else {
            if (j->lens) { j->lens[i] = 65; continue; }
            dna_write(j->dna, j->seed, j->src[i], j->chars + j->offsets[i]);
        }
    }
    return NULL;
}

static int run_jobs(job_t proto, uint64_t n, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 64) nthreads = 64;
    if ((uint64_t)nthreads > n) nthreads = n ? (int)n : 1;
    pthread_t th[64];
    int spawned[64];
    job_t jobs[64];
    for (int t = 0; t < nthreads; t++) {
        jobs[t] = proto;
        jobs[t].lo = n * (uint64_t)t / (uint64_t)nthreads;
        jobs[t].hi = n * (uint64_t)(t + 1) / (uint64_t)nthreads;
        spawned[t] = 0;
        if (t == nthreads - 1) {
            job_run(&jobs[t]);
        } else if (pthread_create(&th[t], NULL, job_run, &jobs[t]) == 0) {
            spawned[t] = 1;
        } else {
            job_run(&jobs[t]); /* no thread available: run inline */
        }
    }
    for (int t = 0; t < nthreads - 1; t++)
        if (spawned[t]) pthread_join(th[t], NULL);
    return 0;
}

/* ------------------------------------------------------------- exported */

/* lens[i] = bytes of string i including its terminator */
int gen_lengths(int kind, uint64_t n, uint64_t seed, uint32_t *lens, int nthreads) {
    if (kind < 1 || kind > 3 || (n && !lens)) return -1;
    job_t j;
    memset(&j, 0, sizeof(j));
    j.kind = kind; j.seed = seed; j.lens = lens;
    url_pools_t pools;
    if (kind == 2) {
        if (url_pools_init(&pools, seed)) return -2;
        j.pools = &pools;
    }
    int rc = run_jobs(j, n, nthreads);
    if (kind == 2) url_pools_free(&pools);
    return rc;
}

/* writes string i at chars + offsets[i]; offsets must leave room for lens[i] */
int gen_fill(int kind, uint64_t n, uint64_t seed, const uint64_t *offsets, uint8_t *chars, int nthreads) {
    if (kind < 1 || kind > 3 || (n && (!offsets || !chars))) return -1;
    job_t j;
    memset(&j, 0, sizeof(j));
    j.kind = kind; j.seed = seed; j.offsets = offsets; j.chars = chars;
    url_pools_t pools;
    dna_model_t dna;
    uint32_t *src = NULL;
    if (kind == 2) {
        if (url_pools_init(&pools, seed)) return -2;
        j.pools = &pools;
    } else if (kind == 3) {
        dna_model_init(&dna, seed);
        src = dna_sources(n, seed);
        if (!src) return -2;
        j.dna = &dna; j.src = src;
    }
    int rc = run_jobs(j, n, nthreads);
    if (kind == 2) url_pools_free(&pools);
    free(src);
    return rc;
}

/* ------------------------------------------------------------- batches
 *
 * Many independent sets in one call: set j has kind kinds[j], sizes[j]
 * strings and its own per-string streams (seed seeds[j]); the url pools and
 * the dna Markov model are built once from pool_seed and shared by all sets
 * of that kind.  Sets are laid out back to back; lens / offsets are indexed
 * globally.  Parallel over sets. */

typedef struct {
    uint32_t lo, hi; /* sets */
    const int *kinds; const uint64_t *sizes, *seeds, *first;
    uint32_t *lens; const uint64_t *offsets; uint8_t *chars;
    const url_pools_t *pools; const dna_model_t *dna;
} batch_job_t;

static void *batch_run(void *arg) {
    batch_job_t *b = (batch_job_t *)arg;
    for (uint32_t j = b->lo; j < b->hi; j++) {
        job_t jj;
        memset(&jj, 0, sizeof(jj));
        jj.kind = b->kinds[j];
        jj.seed = b->seeds[j];
        jj.pools = b->pools;
        jj.dna = b->dna;
        jj.lo = 0;
        jj.hi = b->sizes[j];
        uint32_t *src = NULL;
        if (b->lens) {
            jj.lens = b->lens + b->first[j];
        } else {
            jj.offsets = b->offsets + b->first[j];
            jj.chars = b->chars;
            if (jj.kind == 3) {
                src = dna_sources(b->sizes[j], jj.seed);
                if (!src) continue;
                jj.src = src;
            }
        }
        job_run(&jj);
        free(src);
    }
    return NULL;
}

static int batch_common(uint32_t num_sets, const int *kinds, const uint64_t *sizes, const uint64_t *seeds,
                        uint64_t pool_seed, uint32_t *lens, const uint64_t *offsets, uint8_t *chars, int nthreads) {
    for (uint32_t j = 0; j < num_sets; j++)
        if (kinds[j] < 1 || kinds[j] > 3) return -1;
    uint64_t *first = (uint64_t *)malloc(sizeof(uint64_t) * (num_sets + 1));
    if (!first) return -2;
    first[0] = 0;
    for (uint32_t j = 0; j < num_sets; j++) first[j + 1] = first[j] + sizes[j];
    url_pools_t pools;
    dna_model_t dna;
    if (url_pools_init(&pools, pool_seed)) { free(first); return -2; }
    dna_model_init(&dna, pool_seed);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 64) nthreads = 64;
    pthread_t th[64];
    int spawned[64];
    batch_job_t jobs[64];
    for (int t = 0; t < nthreads; t++) {
        batch_job_t bj = {0};
        bj.lo = (uint32_t)((uint64_t)num_sets * t / nthreads);
        bj.hi = (uint32_t)((uint64_t)num_sets * (t + 1) / nthreads);
        bj.kinds = kinds; bj.sizes = sizes; bj.seeds = seeds; bj.first = first;
        bj.lens = lens; bj.offsets = offsets; bj.chars = chars; bj.pools = &pools; bj.dna = &dna;
        jobs[t] = bj;
        spawned[t] = 0;
        if (t == nthreads - 1) batch_run(&jobs[t]);
        else if (pthread_create(&th[t], NULL, batch_run, &jobs[t]) == 0) spawned[t] = 1;
        else batch_run(&jobs[t]);
    }
    for (int t = 0; t < nthreads - 1; t++)
        if (spawned[t]) pthread_join(th[t], NULL);
    url_pools_free(&pools);
    free(first);
    return 0;
}

int gen_batch_lengths(uint32_t num_sets, const int *kinds, const uint64_t *sizes, const uint64_t *seeds,
                      uint64_t pool_seed, uint32_t *lens, int nthreads) {
    return batch_common(num_sets, kinds, sizes, seeds, pool_seed, lens, NULL, NULL, nthreads);
}

int gen_batch_fill(uint32_t num_sets, const int *kinds, const uint64_t *sizes, const uint64_t *seeds,
                   uint64_t pool_seed, const uint64_t *offsets, uint8_t *chars, int nthreads) {
    return batch_common(num_sets, kinds, sizes, seeds, pool_seed, NULL, offsets, chars, nthreads);
}

/* uniform integers in [0, bound) from stream (seed, stream): used for set
 * sizes and kind choices of the batched workload */
int gen_uniform_u64(uint64_t seed, uint64_t stream, uint64_t count, uint64_t bound, uint64_t *out) {
    if (!out || bound == 0) return -1;
    rng_t r;
    rng_seed(&r, seed, stream);
    for (uint64_t i = 0; i < count; i++) out[i] = rng_below(&r, bound);
    return 0;
}

/* uniform doubles in [0, 1) from stream (seed, stream) */
int gen_uniform_f64(uint64_t seed, uint64_t stream, uint64_t count, double *out) {
    if (!out) return -1;
    rng_t r;
    rng_seed(&r, seed, stream);
    for (uint64_t i = 0; i < count; i++) out[i] = rng_unit(&r);
    return 0;
}
