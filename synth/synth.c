/*
 * Seeded synthetic input generators for the RR-set influence-maximization path.
 *
 * The paper evaluates on real social/web graphs (Table 4: DBLP ... twitter7) that
 * are not available here, so every workload is a directed R-MAT graph of the same
 * vertex count, edge count and degree skew, given as a *transposed* CSR: row v
 * lists the in-edges (u -> v) of v as col[e] = u for e in [row_ptr[v], row_ptr[v+1]).
 *
 * This file holds no arithmetic of the influence-maximization method itself: it
 * draws graphs and edge parameters only.  Its random stream is SplitMix64 (Steele,
 * Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), used
 * as a keyed hash so that every value is a pure function of (seed, stream, index)
 * and the output does not depend on the thread count.
 *
 * Conventions shared with the callers:
 *  - R-MAT quadrant probabilities (a, b, c, d) are turned into integer thresholds
 *    floor(a*2^32), floor((a+b)*2^32), floor((a+b+c)*2^32); levels = ceil(log2 n);
 *    a pair with an endpoint >= n is redrawn (attempt counter in the key).
 *  - duplicates and self-loops are kept, so m is exact.
 *  - a seeded Fisher-Yates permutation relabels the vertices so that ids do not
 *    encode degree.
 *  - each CSR row is ordered by (source id, draw index).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

static inline uint64_t sm64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

/* value `i` of stream `stream` under `seed` */
static inline uint64_t hkey(uint64_t seed, uint64_t stream, uint64_t i) {
    return sm64(sm64(seed ^ (stream * 0xD1B54A32D192ED03ull)) ^ (i * 0xA24BAED4963EE407ull));
}

enum { ST_RMAT = 0x100, ST_PERM = 2, ST_PROB = 3, ST_LT = 4 };

static int n_threads(void) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    if (c < 1) c = 1;
    if (c > 64) c = 64;
    return (int)c;
}

typedef struct {
    uint64_t seed, lo, hi;
    uint32_t n;
    int levels;
    uint32_t A, AB, ABC;
    uint32_t *src, *dst;
} rmat_job;

static void *rmat_worker(void *arg) {
    rmat_job *J = (rmat_job *)arg;
    for (uint64_t i = J->lo; i < J->hi; i++) {
        for (uint64_t att = 0;; att++) {
            uint64_t base = hkey(J->seed, ST_RMAT + att, i);
            uint32_t u = 0, v = 0;
            uint64_t r64 = 0;
            for (int l = 0; l < J->levels; l++) {
                if ((l & 1) == 0) r64 = sm64(base + (uint64_t)l);
                uint32_t r = (l & 1) ? (uint32_t)(r64 >> 32) : (uint32_t)r64;
                uint32_t bu = (r >= J->AB), bv = (r >= J->A && r < J->AB) || (r >= J->ABC);
                u = (u << 1) | bu;
                v = (v << 1) | bv;
            }
            if (u < J->n && v < J->n) {
                J->src[i] = u;
                J->dst[i] = v;
                break;
            }
        }
    }
    return NULL;
}

typedef struct {
    const uint32_t *row_ptr;
    uint32_t *col;
    uint32_t lo, hi;
} sort_job;

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Each row arrives in draw order; sort it by (source, position-in-row) so that
 * equal sources keep draw order. */
static void *sort_worker(void *arg) {
    sort_job *J = (sort_job *)arg;
    uint64_t cap = 0;
    uint64_t *tmp = NULL;
    for (uint32_t v = J->lo; v < J->hi; v++) {
        uint32_t b = J->row_ptr[v], e = J->row_ptr[v + 1], d = e - b;
        if (d < 2) continue;
        if (d > cap) {
            free(tmp);
            cap = d;
            tmp = (uint64_t *)malloc(cap * sizeof(uint64_t));
        }
        for (uint32_t t = 0; t < d; t++) tmp[t] = ((uint64_t)J->col[b + t] << 32) | t;
        qsort(tmp, d, sizeof(uint64_t), cmp_u64);
        for (uint32_t t = 0; t < d; t++) J->col[b + t] = (uint32_t)(tmp[t] >> 32);
    }
    free(tmp);
    return NULL;
}

/*
 * Directed R-MAT graph with n vertices and exactly m edges, returned as a
 * transposed CSR.  row_ptr: n+1 entries (caller-allocated), col: m entries.
 * Requires m < 2^32.  Returns 0 on success, -1 on bad arguments or no memory.
 */
int synth_rmat(uint32_t n, uint64_t m, uint64_t seed, double a, double b, double c,
               uint32_t *row_ptr, uint32_t *col) {
    if (n == 0 || m >= (1ull << 32) || a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return -1;
    int levels = 0;
    while (((uint64_t)1 << levels) < n) levels++;
    uint32_t *src = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
    uint32_t *dst = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
    uint32_t *perm = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!src || !dst || !perm) {
        free(src); free(dst); free(perm);
        return -1;
    }
    const double two32 = 4294967296.0;
    double fa = floor(a * two32), fab = floor((a + b) * two32), fabc = floor((a + b + c) * two32);
    uint32_t A = fa >= two32 ? 0xFFFFFFFFu : (uint32_t)fa;
    uint32_t AB = fab >= two32 ? 0xFFFFFFFFu : (uint32_t)fab;
    uint32_t ABC = fabc >= two32 ? 0xFFFFFFFFu : (uint32_t)fabc;

    int T = n_threads();
    pthread_t th[64];
    rmat_job jobs[64];
    for (int t = 0; t < T; t++) {
        jobs[t] = (rmat_job){seed, m * t / T, m * (t + 1) / T, n, levels, A, AB, ABC, src, dst};
        pthread_create(&th[t], NULL, rmat_worker, &jobs[t]);
    }
    for (int t = 0; t < T; t++) pthread_join(th[t], NULL);

    /* seeded Fisher-Yates relabelling */
    for (uint32_t i = 0; i < n; i++) perm[i] = i;
    for (uint32_t i = n - 1; i >= 1; i--) {
        uint32_t j = (uint32_t)(((hkey(seed, ST_PERM, i) >> 32) * ((uint64_t)i + 1)) >> 32);
        uint32_t tmp = perm[i];
        perm[i] = perm[j];
        perm[j] = tmp;
    }

    /* counting sort by target, scatter in draw order */
    memset(row_ptr, 0, ((size_t)n + 1) * sizeof(uint32_t));
    for (uint64_t i = 0; i < m; i++) row_ptr[perm[dst[i]] + 1]++;
    for (uint32_t v = 0; v < n; v++) row_ptr[v + 1] += row_ptr[v];
    uint32_t *fill = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!fill) {
        free(src); free(dst); free(perm);
        return -1;
    }
    memcpy(fill, row_ptr, (size_t)n * sizeof(uint32_t));
    for (uint64_t i = 0; i < m; i++) col[fill[perm[dst[i]]]++] = perm[src[i]];
    free(fill);
    free(src);
    free(dst);
    free(perm);

    sort_job sj[64];
    for (int t = 0; t < T; t++) {
        sj[t] = (sort_job){row_ptr, col, (uint32_t)((uint64_t)n * t / T), (uint32_t)((uint64_t)n * (t + 1) / T)};
        pthread_create(&th[t], NULL, sort_worker, &sj[t]);
    }
    for (int t = 0; t < T; t++) pthread_join(th[t], NULL);
    return 0;
}

/* IC edge probabilities, uniform on [0, pmax): p[e] = fp32(u24) * pmax with
 * u24 = (h >> 40) * 2^-24, all in fp32. */
void synth_ic_uniform(uint64_t m, uint64_t seed, float pmax, float *p) {
    for (uint64_t e = 0; e < m; e++) {
        float u = (float)(uint32_t)(hkey(seed, ST_PROB, e) >> 40) * 0x1p-24f;
        p[e] = u * pmax;
    }
}

/* Weighted cascade: every in-edge of v carries 1/indeg(v) in fp32. */
void synth_weighted_cascade(uint32_t n, const uint32_t *row_ptr, float *p) {
    for (uint32_t v = 0; v < n; v++) {
        uint32_t b = row_ptr[v], e = row_ptr[v + 1];
        if (e == b) continue;
        float w = 1.0f / (float)(e - b);
        for (uint32_t i = b; i < e; i++) p[i] = w;
    }
}

/*
 * LT in-weights: raw r_e ~ U(0,1], normalised per target so that they sum to at
 * most 1.  Each fp32 weight is rounded toward zero from the exact quotient, so
 * sum_e floor(w_e * 2^32) <= 2^32 holds for every vertex.
 */
void synth_lt_weights(uint32_t n, const uint32_t *row_ptr, uint64_t seed, float *w) {
    for (uint32_t v = 0; v < n; v++) {
        uint32_t b = row_ptr[v], e = row_ptr[v + 1];
        if (e == b) continue;
        double s = 0.0;
        for (uint32_t i = b; i < e; i++) s += (double)((hkey(seed, ST_LT, i) >> 11) + 1) * 0x1p-53;
        for (uint32_t i = b; i < e; i++) {
            double r = (double)((hkey(seed, ST_LT, i) >> 11) + 1) * 0x1p-53;
            double q = r / s;
            float f = (float)q;
            if ((double)f > q) f = nextafterf(f, 0.0f);
            w[i] = f;
        }
    }
}

/* 64-bit keyed draws for the query-stream generator of the serving workload. */
void synth_draws(uint64_t seed, uint64_t stream, uint64_t count, uint64_t *out) {
    for (uint64_t i = 0; i < count; i++) out[i] = hkey(seed, 0x1000 + stream, i);
}
