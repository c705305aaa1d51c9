/*
 * CPU ORACLE for string sorting with LCP output -- test infrastructure only.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  The GPU library never links, loads or calls it, and
 * this file shares no code with it.
 *
 * Everything here is the plain definition of what the GPU path must produce,
 * written for obviousness, not speed:
 *
 *   oracle_sort         multikey quicksort (Bentley-Sedgewick, Sec. 2.1 of
 *                       the paper) on unsigned bytes; a group whose pivot
 *                       character is the terminator holds equal strings and
 *                       is put in ascending original index.
 *   oracle_lcp_scan     lcp_x(i) = lcp(x_{i-1}, x_i) by a direct byte scan
 *                       (definition in Sec. 2); lcp_x(0) = 0.
 *   oracle_verify       the paper's output check (App. B.1: permutation, then
 *                       non-descending order) tightened to the unique answer:
 *                       equal strings in ascending index, LCP exact.
 *   oracle_dist_prefix  D, the distinguishing prefix size (Sec. 2), with
 *                       terminators counted.
 *   oracle_key_word     the next w = 8 characters at depth l packed into one
 *                       64-bit word, first character most significant
 *                       (Sec. 3.1, "as many characters as fit into a machine
 *                       word"); bytes after the terminator read as 0.
 *   oracle_classify     bucket of a key among sorted splitters x_0..x_{v-1}
 *                       with equality buckets (Sec. 3.1, Fig. 1):
 *                       b = 2 * #{i : x_i < key} + [key equals that x].
 *   oracle_select_splitters  the recursive duplicate-skipping splitter
 *                       choice of Sec. 3.1 "Implementation Details", laid
 *                       out as a perfect tree in level order plus in order.
 *   oracle_sort_parallel  the same answer on several host threads: P - 1
 *                       splitter strings from a regular sample cut the
 *                       order into P independent ranges (a sample sort's
 *                       top level, Sec. 2.3), each range is sorted by
 *                       oracle_sort on its own thread, then the LCP scan.
 *                       Only a timing baseline; its output is pinned to
 *                       oracle_sort's.
 *   oracle_cdf_*        the monotone piecewise-linear CDF used to propose
 *                       buckets (an addition to the paper): forward, MSE
 *                       loss and its analytic gradient, in double.
 *
 * Strings: string i starts at chars[offsets[i]] and ends at its first 0 byte.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

/* ------------------------------------------------------ helpers */

static inline uint8_t char_at(const uint8_t *chars, const uint64_t *offsets, uint32_t s, uint64_t d) {
    return chars[offsets[s] + d];
}

/* full comparison of strings a and b starting at depth d (the first d
 * characters are known to be equal); equal strings order by index */
static int less_from(const uint8_t *chars, const uint64_t *offsets, uint32_t a, uint32_t b, uint64_t d) {
    const uint8_t *p = chars + offsets[a] + d;
    const uint8_t *q = chars + offsets[b] + d;
    for (;;) {
        if (*p != *q) return *p < *q;
        if (*p == 0) return a < b;
        p++;
        q++;
    }
}

static void insertion_sort(const uint8_t *chars, const uint64_t *offsets, uint32_t *a, uint32_t m, uint64_t d) {
    for (uint32_t i = 1; i < m; i++) {
        uint32_t t = a[i];
        uint32_t j = i;
        while (j > 0 && less_from(chars, offsets, t, a[j - 1], d)) {
            a[j] = a[j - 1];
            j--;
        }
        a[j] = t;
    }
}

static int cmp_u32(const void *x, const void *y) {
    uint32_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
    return (a > b) - (a < b);
}

typedef struct { uint32_t lo, hi; uint64_t d; } frame_t;

/* ------------------------------------------------------ sort */

/* perm[r] = original index of the r-th smallest string (ties by index).
 * Returns 0, or -2 when memory runs out. */
int oracle_sort(const uint8_t *chars, const uint64_t *offsets, uint32_t n, uint32_t *perm) {
    for (uint32_t i = 0; i < n; i++) perm[i] = i;
    if (n < 2) return 0;
    size_t cap = 1024, top = 0;
    frame_t *st = (frame_t *)malloc(cap * sizeof(frame_t));
    if (!st) return -2;
    st[top++] = (frame_t){0, n, 0};
    while (top) {
        frame_t f = st[--top];
        uint32_t m = f.hi - f.lo;
        if (m < 2) continue;
        if (m < 16) {
            insertion_sort(chars, offsets, perm + f.lo, m, f.d);
            continue;
        }
        /* pivot character: median of three characters at depth d */
        uint8_t c0 = char_at(chars, offsets, perm[f.lo], f.d);
        uint8_t c1 = char_at(chars, offsets, perm[f.lo + m / 2], f.d);
        uint8_t c2 = char_at(chars, offsets, perm[f.hi - 1], f.d);
        uint8_t p = c0 < c1 ? (c1 < c2 ? c1 : (c0 < c2 ? c2 : c0))
                            : (c0 < c2 ? c0 : (c1 < c2 ? c2 : c1));
        /* ternary partition: [lo,lt) <, [lt,gt) =, [gt,hi) > */
        uint32_t lt = f.lo, i = f.lo, gt = f.hi;
        while (i < gt) {
            uint8_t c = char_at(chars, offsets, perm[i], f.d);
            if (c < p) {
                uint32_t t = perm[lt]; perm[lt] = perm[i]; perm[i] = t;
                lt++; i++;
            } else if (c > p) {
                gt--;
                uint32_t t = perm[gt]; perm[gt] = perm[i]; perm[i] = t;
            } else {
                i++;
            }
        }
        if (top + 3 > cap) {
            cap *= 2;
            frame_t *ns = (frame_t *)realloc(st, cap * sizeof(frame_t));
            if (!ns) { free(st); return -2; }
            st = ns;
        }
        st[top++] = (frame_t){f.lo, lt, f.d};
        st[top++] = (frame_t){gt, f.hi, f.d};
        if (p != 0) {
            st[top++] = (frame_t){lt, gt, f.d + 1};
        } else {
            /* every string of the '=' group ended here: they are equal */
            qsort(perm + lt, gt - lt, sizeof(uint32_t), cmp_u32);
        }
    }
    free(st);
    return 0;
}

/* ------------------------------------------------------ parallel sort */

void oracle_lcp_scan(const uint8_t *chars, const uint64_t *offsets, uint32_t n, const uint32_t *perm, uint32_t *lcp);
static uint32_t lcp_pair(const uint8_t *chars, const uint64_t *offsets, uint32_t a, uint32_t b);

/* unsigned-byte comparison of whole strings: <0, 0, >0 */
static int str_cmp(const uint8_t *p, const uint8_t *q) {
    for (;; p++, q++) {
        if (*p != *q) return *p < *q ? -1 : 1;
        if (*p == 0) return 0;
    }
}

typedef struct {
    const uint8_t *chars;
    const uint64_t *offsets;
    const uint32_t *members;  /* original indices, ascending, range by range */
    const uint64_t *start;    /* [P + 1] first member of each range */
    uint32_t *perm;           /* output: sorted original indices */
    uint32_t P;
    volatile int next;        /* next range to take (under mu) */
    int err;
    pthread_mutex_t mu;
} par_job;

static void *par_worker(void *arg) {
    par_job *J = (par_job *)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int r = J->next < (int)J->P ? J->next++ : -1;
        pthread_mutex_unlock(&J->mu);
        if (r < 0) break;
        uint64_t lo = J->start[r], m = J->start[r + 1] - lo;
        if (m == 0) continue;
        /* the range's strings as a set of their own: local index k is the
         * k-th smallest original index, so oracle_sort's tie-break by local
         * index is the tie-break by original index */
        uint64_t *off = (uint64_t *)malloc(m * sizeof(uint64_t));
        uint32_t *lp = (uint32_t *)malloc(m * sizeof(uint32_t));
        if (!off || !lp) { free(off); free(lp); J->err = -2; continue; }
        for (uint64_t k = 0; k < m; k++) off[k] = J->offsets[J->members[lo + k]];
        if (oracle_sort(J->chars, off, (uint32_t)m, lp) != 0) J->err = -2;
        for (uint64_t k = 0; k < m; k++) J->perm[lo + k] = J->members[lo + lp[k]];
        free(off);
        free(lp);
    }
    return NULL;
}

/* f(arg, t) for t = 0..threads-1, each on a thread of its own */
typedef struct { void *(*f)(void *); void *arg; uint32_t t; } slice_t;
static void *slice_main(void *p) {
    slice_t *s = (slice_t *)p;
    void *(*f)(void *) = s->f;
    return f(s);
}
static int run_threads(int threads, void *(*f)(void *), void *arg) {
    pthread_t *th = (pthread_t *)malloc((size_t)threads * sizeof(pthread_t));
    slice_t *sl = (slice_t *)malloc((size_t)threads * sizeof(slice_t));
    char *ok = (char *)calloc((size_t)threads, 1);
    if (!th || !sl || !ok) { free(th); free(sl); free(ok); return -2; }
    for (int t = 0; t < threads; t++) {
        sl[t] = (slice_t){f, arg, (uint32_t)t};
        ok[t] = pthread_create(&th[t], NULL, slice_main, &sl[t]) == 0;
        if (!ok[t]) slice_main(&sl[t]);
    }
    for (int t = 0; t < threads; t++)
        if (ok[t]) pthread_join(th[t], NULL);
    free(th); free(sl); free(ok);
    return 0;
}

/* contiguous slice t of [0, n) for `parts` slices */
static void slice_bounds(uint32_t n, uint32_t parts, uint32_t t, uint32_t *lo, uint32_t *hi) {
    *lo = (uint32_t)((uint64_t)n * t / parts);
    *hi = (uint32_t)((uint64_t)n * (t + 1) / parts);
}

typedef struct {
    const uint8_t *chars; const uint64_t *offsets; const uint8_t **x; uint32_t P;
    uint32_t *part; uint32_t n, parts;
} range_job;
static void *range_worker(void *p) {
    slice_t *s = (slice_t *)p;
    range_job *R = (range_job *)s->arg;
    uint32_t lo, hi;
    slice_bounds(R->n, R->parts, s->t, &lo, &hi);
    for (uint32_t i = lo; i < hi; i++) {
        const uint8_t *sp = R->chars + R->offsets[i];
        uint32_t a = 0, b = R->P - 1;
        while (a < b) {
            uint32_t mid = (a + b) / 2;
            if (str_cmp(R->x[mid], sp) < 0) a = mid + 1; else b = mid;
        }
        R->part[i] = a;
    }
    return NULL;
}

typedef struct {
    const uint8_t *chars; const uint64_t *offsets; const uint32_t *perm; uint32_t *lcp;
    uint32_t n, parts;
} lcp_job;
static void *lcp_worker(void *p) {
    slice_t *s = (slice_t *)p;
    lcp_job *L = (lcp_job *)s->arg;
    uint32_t lo, hi;
    slice_bounds(L->n, L->parts, s->t, &lo, &hi);
    for (uint32_t i = lo; i < hi; i++)
        L->lcp[i] = i == 0 ? 0u : lcp_pair(L->chars, L->offsets, L->perm[i - 1], L->perm[i]);
    return NULL;
}

/* perm and lcp as oracle_sort + oracle_lcp_scan give them, computed on
 * `threads` host threads.  Range r holds the strings s with
 * x_{r-1} < s <= x_r for sample strings x_0 <= ... <= x_{P-2}, so equal
 * strings share a range and the ranges follow one another in the sorted
 * order.  Returns 0, or -2 when memory runs out. */
int oracle_sort_parallel(const uint8_t *chars, const uint64_t *offsets, uint32_t n, uint32_t *perm,
                         uint32_t *lcp, int threads) {
    if (threads < 1) threads = 1;
    uint32_t P = (uint32_t)threads * 8u;
    if (n < 4096u || threads == 1) {
        if (oracle_sort(chars, offsets, n, perm) != 0) return -2;
        oracle_lcp_scan(chars, offsets, n, perm, lcp);
        return 0;
    }
    /* splitters: every (m/P)-th string of a sorted regular sample of m strings */
    uint32_t m = P * 32u;
    uint64_t *soff = (uint64_t *)malloc(m * sizeof(uint64_t));
    uint32_t *sperm = (uint32_t *)malloc(m * sizeof(uint32_t));
    const uint8_t **x = (const uint8_t **)malloc(P * sizeof(uint8_t *));
    uint32_t *part = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint64_t *start = (uint64_t *)calloc(P + 1, sizeof(uint64_t));
    uint32_t *members = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    int rc = -2;
    if (!soff || !sperm || !x || !part || !start || !members) goto out;
    for (uint32_t j = 0; j < m; j++) soff[j] = offsets[(uint64_t)j * n / m];
    if (oracle_sort(chars, soff, m, sperm) != 0) goto out;
    for (uint32_t r = 1; r < P; r++) x[r - 1] = chars + soff[sperm[(uint64_t)r * m / P]];
    /* range of each string: the number of splitters below it */
    {
        range_job R = {chars, offsets, x, P, part, n, (uint32_t)threads};
        if (run_threads(threads, range_worker, &R) != 0) goto out;
    }
    for (uint32_t i = 0; i < n; i++) start[part[i] + 1]++;
    for (uint32_t r = 0; r < P; r++) start[r + 1] += start[r];
    {
        uint64_t *fill = (uint64_t *)malloc(P * sizeof(uint64_t));
        if (!fill) goto out;
        memcpy(fill, start, P * sizeof(uint64_t));
        for (uint32_t i = 0; i < n; i++) members[fill[part[i]]++] = i;  /* ascending index per range */
        free(fill);
    }
    {
        par_job J;
        J.chars = chars; J.offsets = offsets; J.members = members; J.start = start; J.perm = perm;
        J.P = P; J.next = 0; J.err = 0;
        pthread_mutex_init(&J.mu, NULL);
        pthread_t *th = (pthread_t *)malloc((size_t)threads * sizeof(pthread_t));
        if (!th) { pthread_mutex_destroy(&J.mu); goto out; }
        int started = 0;
        for (int t = 0; t < threads; t++)
            if (pthread_create(&th[t], NULL, par_worker, &J) == 0) started++;
        if (started == 0) par_worker(&J);
        for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
        free(th);
        pthread_mutex_destroy(&J.mu);
        if (J.err) goto out;
    }
    {
        lcp_job Lj = {chars, offsets, perm, lcp, n, (uint32_t)threads};
        if (run_threads(threads, lcp_worker, &Lj) != 0) goto out;
    }
    rc = 0;
out:
    free(soff); free(sperm); free(x); free(part); free(start); free(members);
    return rc;
}

/* ------------------------------------------------------ lcp */

static uint32_t lcp_pair(const uint8_t *chars, const uint64_t *offsets, uint32_t a, uint32_t b) {
    const uint8_t *p = chars + offsets[a];
    const uint8_t *q = chars + offsets[b];
    uint32_t k = 0;
    while (p[k] == q[k] && p[k] != 0) k++;
    return k;
}

void oracle_lcp_scan(const uint8_t *chars, const uint64_t *offsets, uint32_t n, const uint32_t *perm, uint32_t *lcp) {
    if (n == 0) return;
    lcp[0] = 0;
    for (uint32_t i = 1; i < n; i++) lcp[i] = lcp_pair(chars, offsets, perm[i - 1], perm[i]);
}

/* ------------------------------------------------------ verify */

/* Returns 0 when (perm, lcp) is the unique correct answer.  Otherwise a code
 * and *bad = the first offending rank:
 *   1 perm is not a permutation, 2 order violated, 3 equal strings not in
 *   index order, 4 lcp wrong.  -2: out of memory. */
int oracle_verify(const uint8_t *chars, const uint64_t *offsets, uint32_t n, const uint32_t *perm,
                  const uint32_t *lcp, uint64_t *bad) {
    *bad = 0;
    if (n == 0) return 0;
    uint8_t *seen = (uint8_t *)calloc(n, 1);
    if (!seen) return -2;
    for (uint32_t i = 0; i < n; i++) {
        if (perm[i] >= n || seen[perm[i]]) { free(seen); *bad = i; return 1; }
        seen[perm[i]] = 1;
    }
    free(seen);
    if (lcp && lcp[0] != 0) { *bad = 0; return 4; }
    for (uint32_t i = 1; i < n; i++) {
        uint32_t a = perm[i - 1], b = perm[i];
        uint32_t k = lcp_pair(chars, offsets, a, b);
        uint8_t ca = chars[offsets[a] + k], cb = chars[offsets[b] + k];
        if (ca > cb) { *bad = i; return 2; }
        if (ca == cb && a > b) { *bad = i; return 3; }
        if (lcp && lcp[i] != k) { *bad = i; return 4; }
    }
    return 0;
}

/* ------------------------------------------------------ D */

/* D = sum over strings of min(|s|, 1 + max(lcp with left, lcp with right)),
 * |s| counting the terminator; lcp beyond the ends is 0. */
uint64_t oracle_dist_prefix(const uint8_t *chars, const uint64_t *offsets, uint32_t n, const uint32_t *perm,
                            const uint32_t *lcp) {
    uint64_t D = 0;
    for (uint32_t i = 0; i < n; i++) {
        uint64_t len = strlen((const char *)(chars + offsets[perm[i]])) + 1;
        uint64_t left = i > 0 ? lcp[i] : 0;
        uint64_t right = i + 1 < n ? lcp[i + 1] : 0;
        uint64_t need = 1 + (left > right ? left : right);
        D += need < len ? need : len;
    }
    return D;
}

/* ------------------------------------------------------ per-step definitions */

uint64_t oracle_key_word(const uint8_t *chars, uint64_t offset, uint64_t depth) {
    const uint8_t *s = chars + offset;
    for (uint64_t p = 0; p < depth; p++)
        if (s[p] == 0) return 0; /* the string ended before depth */
    uint64_t k = 0;
    int ended = 0;
    for (int j = 0; j < 8; j++) {
        uint8_t c = ended ? 0 : s[depth + j];
        if (c == 0) ended = 1;
        k = (k << 8) | c;
    }
    return k;
}

uint32_t oracle_classify(uint64_t key, const uint64_t *x, uint32_t v) {
    uint32_t j = 0;
    while (j < v && x[j] < key) j++;
    return 2 * j + (j < v && x[j] == key ? 1 : 0);
}

static void pick(const uint64_t *s, int64_t a, int64_t b, uint64_t parent, uint32_t node, uint32_t v,
                 uint64_t *level) {
    if (node > v) return;
    uint64_t x;
    int64_t bl, ar;
    if (a > b) {
        x = parent; /* nothing left in this range: repeat the parent */
        bl = a - 1; /* both children stay empty */
        ar = b + 1;
    } else {
        int64_t m = a + (b - a) / 2;
        x = s[m];
        bl = m - 1;
        while (bl >= a && s[bl] == x) bl--;
        ar = m + 1;
        while (ar <= b && s[ar] == x) ar++;
    }
    level[node - 1] = x;
    pick(s, a, bl, x, 2 * node, v, level);
    pick(s, ar, b, x, 2 * node + 1, v, level);
}

static void inorder_walk(const uint64_t *level, uint32_t node, uint32_t v, uint64_t *out, uint32_t *pos) {
    if (node > v) return;
    inorder_walk(level, 2 * node, v, out, pos);
    out[(*pos)++] = level[node - 1];
    inorder_walk(level, 2 * node + 1, v, out, pos);
}

/* sample: count >= 1 keys sorted ascending.  Fills v = 2^k - 1 splitters:
 * level[0] is the root, level[i-1] has children level[2i-1], level[2i]. */
int oracle_select_splitters(const uint64_t *sample, int64_t count, int k, uint64_t *level, uint64_t *inorder) {
    if (count < 1 || k < 1 || k > 20) return -1;
    uint32_t v = (1u << k) - 1;
    pick(sample, 0, count - 1, sample[0], 1, v, level);
    uint32_t pos = 0;
    inorder_walk(level, 1, v, inorder, &pos);
    return 0;
}

/* ------------------------------------------------------ learned CDF */

static double softplus(double t) { return t > 30 ? t : log1p(exp(t)); }
static double sigmoid(double t) { return 1.0 / (1.0 + exp(-t)); }

/* F(u) for the monotone piecewise-linear CDF with M equal-width segments on
 * [0,1]: increments softplus(theta_m), normalised to total 1. */
void oracle_cdf_forward(const double *theta, int M, const double *u, int S, double *F) {
    double *delta = (double *)malloc(sizeof(double) * M);
    double T = 0.0;
    for (int m = 0; m < M; m++) { delta[m] = softplus(theta[m]); T += delta[m]; }
    for (int s = 0; s < S; s++) {
        double t = u[s] * M;
        int m = (int)floor(t);
        if (m < 0) m = 0;
        if (m > M - 1) m = M - 1;
        double f = t - m;
        if (f < 0) f = 0;
        if (f > 1) f = 1;
        double P = 0.0;
        for (int j = 0; j < m; j++) P += delta[j];
        F[s] = (P + f * delta[m]) / T;
    }
    free(delta);
}

/* L = mean over s of (F(u_s) - y_s)^2 */
double oracle_cdf_loss(const double *theta, int M, const double *u, const double *y, int S) {
    double *F = (double *)malloc(sizeof(double) * (S > 0 ? S : 1));
    oracle_cdf_forward(theta, M, u, S, F);
    double L = 0.0;
    for (int s = 0; s < S; s++) L += (F[s] - y[s]) * (F[s] - y[s]);
    free(F);
    return S > 0 ? L / S : 0.0;
}

/* dL/dtheta by the chain rule written out term by term:
 * dF_s/ddelta_j = ([j < m_s] + f_s [j == m_s]) / T - F_s / T,
 * ddelta_j/dtheta_j = sigmoid(theta_j). */
void oracle_cdf_grad(const double *theta, int M, const double *u, const double *y, int S, double *grad) {
    double *delta = (double *)malloc(sizeof(double) * M);
    double *F = (double *)malloc(sizeof(double) * (S > 0 ? S : 1));
    double T = 0.0;
    for (int m = 0; m < M; m++) { delta[m] = softplus(theta[m]); T += delta[m]; }
    oracle_cdf_forward(theta, M, u, S, F);
    for (int j = 0; j < M; j++) {
        double g = 0.0;
        for (int s = 0; s < S; s++) {
            double t = u[s] * M;
            int m = (int)floor(t);
            if (m < 0) m = 0;
            if (m > M - 1) m = M - 1;
            double f = t - m;
            if (f < 0) f = 0;
            if (f > 1) f = 1;
            double dF = ((j < m ? 1.0 : 0.0) + (j == m ? f : 0.0)) / T - F[s] / T;
            g += 2.0 * (F[s] - y[s]) / S * dF;
        }
        grad[j] = g * sigmoid(theta[j]);
    }
    free(delta);
    free(F);
}
