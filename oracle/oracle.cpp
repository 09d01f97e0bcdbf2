/*
 * ORACLE -- test infrastructure only.
 *
 * A plain, slow, obviously-correct CPU statement of what the GPU path computes:
 * IMM (two-phase martingale sampling, then greedy max coverage) over RR sets that
 * are kept uncompressed and sorted, plus a separate Huffman/bitmap encoder and
 * decoder for the compressed form.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library; the product never does.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Paper: HBMax, "Compress-to-compute" influence maximization (arXiv 2208.00613).
 *   - IC / LT diffusion: Section 2.1.
 *   - RR and random RR sets: Section 2.2, Definitions 1 and 2.
 *   - IMM sampling effort theta_i: Section 2.2, Eq. (1) (see imm_params below).
 *   - greedy max-coverage seed selection: Section 2.2; Algorithms 2 and 3.
 *   - skewness S and density D of set sizes: Section 3.2, Eq. (2).
 *   - 1/32 density cut between id lists and bitmaps: Section 3.2.
 *   - Huffman codebook from the warm-up block, copy array for uncoded vertices:
 *     Section 4.2.2, Algorithm 1.
 *   - bitmap encoding with zero padding: Section 4.2.3.
 *
 * Where the paper is silent the reading taken is stated at the function.  The
 * random stream is Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC 2011), written here from that paper; it is
 * checked against an independent library implementation in the tests.
 *
 * Compile with -ffp-contract=off: the FP64 IMM bounds must round exactly as
 * written.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al. 2011, Section 4: the Philox S-box with N=4,   */
/* W=32; multipliers and Weyl key increments as published there).             */
/* ------------------------------------------------------------------------- */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox_batch(uint64_t count, const uint32_t *ctr, const uint32_t key[2], uint32_t *out) {
    for (uint64_t i = 0; i < count; i++) orc_philox(ctr + 4 * i, key, out + 4 * i);
}

/* ------------------------------------------------------------------------- */
/* Graph: transposed CSR.  In-edges (u -> v) of v are col[e] = u for          */
/* e in [row_ptr[v], row_ptr[v+1]); e is the edge id.                         */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint32_t n;
    uint64_t m;
    const uint32_t *row_ptr;
    const uint32_t *col;
    const float *prob;       /* IC: activation probability of each edge, or NULL */
    const float *lt_weight;  /* LT: in-weight of each edge, or NULL */
} orc_graph;

enum { ORC_IC = 0, ORC_LT = 1 };
enum { STREAM_IC = 1, STREAM_LT = 2, STREAM_ROOT = 3 };

static void draw(uint64_t seed, uint32_t c0, uint64_t j, uint32_t epoch, uint32_t stream, uint32_t out[4]) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {c0, (uint32_t)j, epoch, stream};
    orc_philox(ctr, key, out);
}

/* Root of RR set j: a uniform vertex, floor(x * n / 2^32) of one 32-bit draw. */
static uint32_t root_of(uint32_t n, uint64_t seed, uint32_t epoch, uint64_t j) {
    uint32_t r[4];
    draw(seed, 0, j, epoch, STREAM_ROOT, r);
    return (uint32_t)(((uint64_t)r[0] * (uint64_t)n) >> 32);
}

/* LT fixed-point in-weight: q = floor(w * 2^32), kept below 2^32 so that it fits
 * 32 bits (a weight of exactly 1 becomes (2^32-1)/2^32).  Reading: the paper
 * states the LT model as a threshold compare (Section 2.1); the live-edge form
 * with one uniform 32-bit draw per vertex is the standard equivalent. */
static uint64_t lt_fixed(float w) {
    double q = std::floor((double)w * 4294967296.0);
    if (q > 4294967295.0) q = 4294967295.0;
    return (uint64_t)q;
}

/*
 * One random RR set (Definition 2): the vertices that reach `root` in a random
 * live-edge subgraph, found by a reverse search from the root.
 *   IC: in-edge e of a reached vertex is live iff u24(x) < p[e], where x is word
 *       (e mod 4) of Philox(ctr = (e/4, j, epoch, 1)) and u24(x) = (x >> 8) * 2^-24
 *       (an exact fp32 value).  The edge's coin does not depend on which vertex
 *       reached it first, so the set does not depend on search order.
 *   LT: at reached vertex v draw x = word 0 of Philox((v, j, epoch, 2)) and take
 *       the first in-edge e whose inclusive prefix sum Q of fixed-point weights
 *       exceeds x; stop when there is none or its source is already in the set.
 * `mark` is an all-zero scratch array of n bytes, returned all-zero.
 * The set is returned sorted ascending.
 */
static void rr_set(const orc_graph *g, int model, uint64_t seed, uint32_t epoch, uint64_t j,
                   std::vector<uint8_t> &mark, std::vector<uint32_t> &out,
                   uint64_t *edges_scanned, uint64_t *edges_live) {
    out.clear();
    uint64_t scanned = 0, live = 0;
    uint32_t root = root_of(g->n, seed, epoch, j);
    out.push_back(root);
    mark[root] = 1;
    if (model == ORC_IC) {
        size_t head = 0;
        while (head < out.size()) {
            uint32_t v = out[head++];
            for (uint64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++) {
                uint32_t x[4];
                draw(seed, (uint32_t)(e >> 2), j, epoch, STREAM_IC, x);
                float u24 = (float)(x[e & 3] >> 8) * 0x1p-24f;
                scanned++;
                if (u24 < g->prob[e]) {
                    live++;
                    uint32_t u = g->col[e];
                    if (!mark[u]) {
                        mark[u] = 1;
                        out.push_back(u);
                    }
                }
            }
        }
    } else {
        uint32_t v = root;
        for (;;) {
            uint64_t b = g->row_ptr[v], end = g->row_ptr[v + 1];
            if (b == end) break;
            uint32_t x[4];
            draw(seed, v, j, epoch, STREAM_LT, x);
            uint64_t Q = 0;
            uint64_t chosen = end;
            for (uint64_t e = b; e < end; e++) {
                scanned++;
                Q += lt_fixed(g->lt_weight[e]);
                if ((uint64_t)x[0] < Q) {
                    chosen = e;
                    break;
                }
            }
            if (chosen == end) break;
            live++;
            uint32_t u = g->col[chosen];
            if (mark[u]) break;
            mark[u] = 1;
            out.push_back(u);
            v = u;
        }
    }
    for (uint32_t u : out) mark[u] = 0;
    std::sort(out.begin(), out.end());
    if (edges_scanned) *edges_scanned += scanned;
    if (edges_live) *edges_live += live;
}

/* Validation of the diffusion parameters; 0 = ok, -1 = bad value, -2 = an LT
 * vertex whose fixed-point in-weights sum above 2^32 (weights sum > 1). */
int orc_validate(const orc_graph *g, int model) {
    if (g->n == 0) return -1;
    if (g->row_ptr[0] != 0 || g->row_ptr[g->n] != g->m) return -1;
    for (uint32_t v = 0; v < g->n; v++)
        if (g->row_ptr[v + 1] < g->row_ptr[v]) return -1;
    for (uint64_t e = 0; e < g->m; e++)
        if (g->col[e] >= g->n) return -1;
    if (model == ORC_IC) {
        if (!g->prob) return -1;
        for (uint64_t e = 0; e < g->m; e++)
            if (!(g->prob[e] >= 0.0f && g->prob[e] <= 1.0f)) return -1;
    } else {
        if (!g->lt_weight) return -1;
        for (uint64_t e = 0; e < g->m; e++)
            if (!(g->lt_weight[e] >= 0.0f && g->lt_weight[e] <= 1.0f)) return -1;
        for (uint32_t v = 0; v < g->n; v++) {
            uint64_t s = 0;
            for (uint64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++)
                s += (uint64_t)std::floor((double)g->lt_weight[e] * 4294967296.0);
            if (s > 4294967296ull) return -2;
        }
    }
    return 0;
}

/* One RR set j into out (capacity cap); returns its size (or the needed size
 * if it does not fit). */
uint64_t orc_rr_set(const orc_graph *g, int model, uint64_t seed, uint32_t epoch, uint64_t j,
                    uint32_t *out, uint64_t cap) {
    std::vector<uint8_t> mark(g->n, 0);
    std::vector<uint32_t> s;
    rr_set(g, model, seed, epoch, j, mark, s, nullptr, nullptr);
    if (s.size() <= cap) std::copy(s.begin(), s.end(), out);
    return s.size();
}

/* ------------------------------------------------------------------------- */
/* A pool of RR sets [0, T), uncompressed and sorted.                         */
/* ------------------------------------------------------------------------- */
struct orc_pool {
    orc_graph g;
    int model;
    uint64_t seed;
    uint32_t epoch;
    std::vector<std::vector<uint32_t>> sets;
    uint64_t edges_scanned = 0, edges_live = 0;
};

void *orc_pool_new(const orc_graph *g, int model, uint64_t seed, uint32_t epoch) {
    orc_pool *p = new orc_pool();
    p->g = *g;
    p->model = model;
    p->seed = seed;
    p->epoch = epoch;
    return p;
}

void orc_pool_free(void *h) { delete (orc_pool *)h; }

/* Sample sets [size, T).  Sets are independent, so threads split the ids. */
int orc_pool_extend(void *h, uint64_t T, int nthreads) {
    orc_pool *p = (orc_pool *)h;
    uint64_t T0 = p->sets.size();
    if (T <= T0) return 0;
    p->sets.resize(T);
    uint64_t scanned = 0, live = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads) reduction(+ : scanned, live)
#endif
    {
        std::vector<uint8_t> mark(p->g.n, 0);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int64_t j = (int64_t)T0; j < (int64_t)T; j++)
            rr_set(&p->g, p->model, p->seed, p->epoch, (uint64_t)j, mark, p->sets[j], &scanned, &live);
    }
    p->edges_scanned += scanned;
    p->edges_live += live;
    return 0;
}

uint64_t orc_pool_count(void *h) { return ((orc_pool *)h)->sets.size(); }
uint64_t orc_pool_set_size(void *h, uint64_t j) { return ((orc_pool *)h)->sets[j].size(); }
void orc_pool_get_set(void *h, uint64_t j, uint32_t *out) {
    const auto &s = ((orc_pool *)h)->sets[j];
    std::copy(s.begin(), s.end(), out);
}
void orc_pool_sizes(void *h, uint64_t j0, uint64_t j1, uint64_t *out) {
    orc_pool *p = (orc_pool *)h;
    for (uint64_t j = j0; j < j1; j++) out[j - j0] = p->sets[j].size();
}
/* Concatenate sets [j0, j1) into out (sizes from orc_pool_sizes). */
void orc_pool_concat(void *h, uint64_t j0, uint64_t j1, uint32_t *out) {
    orc_pool *p = (orc_pool *)h;
    uint64_t o = 0;
    for (uint64_t j = j0; j < j1; j++) {
        std::copy(p->sets[j].begin(), p->sets[j].end(), out + o);
        o += p->sets[j].size();
    }
}
void orc_pool_edge_counts(void *h, uint64_t *scanned, uint64_t *live) {
    *scanned = ((orc_pool *)h)->edges_scanned;
    *live = ((orc_pool *)h)->edges_live;
}

/* ------------------------------------------------------------------------- */
/* Greedy max coverage (Section 2.2; Algorithms 2 and 3).                     */
/* Readings: exactly k seeds are chosen (the "while |seeds| <= k" loops of    */
/* Algorithms 2 and 3 would pick k+1); the argmax is exact, with the lowest   */
/* vertex id winning ties, and once every count is 0 the lowest-id vertex not */
/* yet chosen is taken.  cnt[v] = number of not-yet-covered sets holding v;   */
/* after u* is chosen every set holding it is covered and its vertices'       */
/* counts drop by one, which is what the per-iteration recount of the paper   */
/* reconstructs.                                                              */
/* ------------------------------------------------------------------------- */
static void greedy_from(uint32_t n, const std::vector<std::vector<uint32_t>> &sets, uint64_t j_lo, uint64_t T,
                        uint32_t k, uint32_t *seeds, uint64_t *marginal, uint64_t *covered_out) {
    std::vector<uint64_t> cnt(n, 0);
    std::vector<uint8_t> alive(T, 1), chosen(n, 0);
    for (uint64_t j = 0; j < j_lo; j++) alive[j] = 0;
    for (uint64_t j = j_lo; j < T; j++)
        for (uint32_t v : sets[j]) cnt[v]++;
    uint64_t covered = 0;
    for (uint32_t it = 0; it < k; it++) {
        uint32_t best = n;
        for (uint32_t v = 0; v < n; v++) {
            if (chosen[v]) continue;
            if (best == n || cnt[v] > cnt[best]) best = v;
        }
        chosen[best] = 1;
        seeds[it] = best;
        uint64_t gain = 0;
        for (uint64_t j = 0; j < T; j++) {
            if (!alive[j]) continue;
            if (!std::binary_search(sets[j].begin(), sets[j].end(), best)) continue;
            alive[j] = 0;
            gain++;
            for (uint32_t v : sets[j]) cnt[v]--;
        }
        covered += gain;
        if (marginal) marginal[it] = gain;
    }
    if (covered_out) *covered_out = covered;
}

/* Greedy over the sets [0, T). */
static void greedy(uint32_t n, const std::vector<std::vector<uint32_t>> &sets, uint64_t T, uint32_t k,
                   uint32_t *seeds, uint64_t *marginal, uint64_t *covered_out) {
    greedy_from(n, sets, 0, T, k, seeds, marginal, covered_out);
}

int orc_pool_greedy(void *h, uint64_t T, uint32_t k, uint32_t *seeds, uint64_t *marginal, uint64_t *covered) {
    orc_pool *p = (orc_pool *)h;
    if (T > p->sets.size() || k > p->g.n) return -1;
    greedy(p->g.n, p->sets, T, k, seeds, marginal, covered);
    return 0;
}

/* Greedy over sets given as concatenated sorted lists (tests). */
int orc_greedy_lists(uint32_t n, uint64_t T, const uint64_t *offsets /*T+1*/, const uint32_t *verts,
                     uint32_t k, uint32_t *seeds, uint64_t *marginal, uint64_t *covered) {
    if (k > n) return -1;
    std::vector<std::vector<uint32_t>> sets(T);
    for (uint64_t j = 0; j < T; j++) {
        sets[j].assign(verts + offsets[j], verts + offsets[j + 1]);
        std::sort(sets[j].begin(), sets[j].end());
        sets[j].erase(std::unique(sets[j].begin(), sets[j].end()), sets[j].end());
    }
    greedy(n, sets, T, k, seeds, marginal, covered);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* IMM (Tang, Shi, Xiao 2015), as summarised in Section 2.2 and Eq. (1).      */
/* Eq. (1) is printed garbled; the reading taken is IMM's own bound with      */
/* eps' = sqrt(2) eps, under which the printed factors match term by term     */
/* ((2 + 2 sqrt(2)/3 eps) = 2 + 2/3 eps', 2 eps^2 = eps'^2, and the product   */
/* "log C(n,k) . log n" read as the sum "log C(n,k) + l . log n"):            */
/*   l'      = l (1 + ln 2 / ln n)                                            */
/*   lambda' = (2 + 2 eps'/3)(ln C(n,k) + l' ln n + ln log2 n) n / eps'^2     */
/*   theta_i = lambda' / x_i,  x_i = n / 2^i   (= lambda' 2^i / n, Eq. (1))   */
/*   alpha   = sqrt(l' ln n + ln 2)                                           */
/*   beta    = sqrt((1 - 1/e)(ln C(n,k) + l' ln n + ln 2))                    */
/*   lambda* = 2 n ((1 - 1/e) alpha + beta)^2 / eps^2                         */
/* ln C(n,k) is summed as sum_{i=1..k} ln((n-k+i)/i) in that order.           */
/* out: [eps', l', lnC, lambda', lambda*, alpha, beta]                        */
/* ------------------------------------------------------------------------- */
int orc_imm_params(uint32_t n, uint32_t k, double eps, double ell, double *out) {
    if (n < 2 || k == 0 || k > n || !(eps > 0.0 && eps < 1.0) || !(ell > 0.0)) return -1;
    double dn = (double)n;
    double epsp = std::sqrt(2.0) * eps;
    double ellp = ell * (1.0 + std::log(2.0) / std::log(dn));
    double lnc = 0.0;
    for (uint32_t i = 1; i <= k; i++) lnc += std::log(((double)(n - k) + (double)i) / (double)i);
    double lambda_p = (2.0 + 2.0 * epsp / 3.0) * (lnc + ellp * std::log(dn) + std::log(std::log2(dn))) * dn /
                      (epsp * epsp);
    double one_m_inv_e = 1.0 - std::exp(-1.0);
    double alpha = std::sqrt(ellp * std::log(dn) + std::log(2.0));
    double beta = std::sqrt(one_m_inv_e * (lnc + ellp * std::log(dn) + std::log(2.0)));
    double s = one_m_inv_e * alpha + beta;
    double lambda_star = 2.0 * dn * s * s / (eps * eps);
    out[0] = epsp; out[1] = ellp; out[2] = lnc; out[3] = lambda_p; out[4] = lambda_star;
    out[5] = alpha; out[6] = beta;
    return 0;
}

/* Number of estimation rounds: i = 1 .. floor(log2 n) - 1 (integer log). */
static uint32_t floor_log2(uint32_t n) {
    uint32_t r = 0;
    while ((n >> (r + 1)) != 0) r++;
    return r;
}

/*
 * IMM driver.  Estimation rounds i = 1 .. floor(log2 n) - 1:
 *   x = n / 2^i;  T_i = max(T_{i-1}, ceil(lambda' / x));  sample up to T_i;
 *   greedy(k) on [0, T_i) covering `cov` sets;
 *   if n cov / T_i >= (1 + eps') x:  LB = (n cov / T_i) / (1 + eps'), stop.
 * LB = 1 if no round stops.  Final theta = max(T_i, ceil(lambda* / LB)); the
 * estimation sets are reused; greedy(k) on [0, theta) gives the seeds, and the
 * influence estimate is n cov / theta.
 * round_T (up to 64 entries) records T_1, T_2, ... and then theta.
 */
int orc_imm_pool_fresh(void *h, uint32_t k, double eps, double ell, int nthreads, int fresh_final,
                       uint32_t *seeds, uint64_t *marginal, double *influence, uint64_t *theta,
                       uint64_t *covered_out, double *lb_out, uint32_t *rounds_out, uint64_t *round_T);

int orc_imm_pool(void *h, uint32_t k, double eps, double ell, int nthreads, uint32_t *seeds,
                 uint64_t *marginal, double *influence, uint64_t *theta, uint64_t *covered_out, double *lb_out,
                 uint32_t *rounds_out, uint64_t *round_T) {
    return orc_imm_pool_fresh(h, k, eps, ell, nthreads, 0, seeds, marginal, influence, theta, covered_out, lb_out,
                              rounds_out, round_T);
}

/*
 * fresh_final = 1: the final phase draws theta = ceil(lambda* / LB) new sets,
 * [T_i, T_i + theta), instead of reusing the estimation sets (the reading of
 * Section 2.2 that keeps the two phases independent); greedy runs on those
 * sets only and the estimate is n cov / theta.  round_T's last entry is then
 * T_i + theta.
 */
int orc_imm_pool_fresh(void *h, uint32_t k, double eps, double ell, int nthreads, int fresh_final,
                       uint32_t *seeds, uint64_t *marginal, double *influence, uint64_t *theta,
                       uint64_t *covered_out, double *lb_out, uint32_t *rounds_out, uint64_t *round_T) {
    orc_pool *p = (orc_pool *)h;
    uint32_t n = p->g.n;
    double prm[7];
    if (orc_imm_params(n, k, eps, ell, prm) != 0) return -1;
    double epsp = prm[0], lambda_p = prm[3], lambda_star = prm[4];
    double dn = (double)n;
    std::vector<uint32_t> s(k);
    uint64_t Ti = 0;
    double LB = 1.0;
    uint32_t rounds = 0;
    uint32_t imax = floor_log2(n) - 1;
    for (uint32_t i = 1; i <= imax; i++) {
        double x = dn / std::ldexp(1.0, (int)i);
        uint64_t t = (uint64_t)std::ceil(lambda_p / x);
        if (t > Ti) Ti = t;
        orc_pool_extend(h, Ti, nthreads);
        uint64_t cov = 0;
        greedy(n, p->sets, Ti, k, s.data(), nullptr, &cov);
        if (round_T && rounds < 63) round_T[rounds] = Ti;
        rounds++;
        double est = dn * (double)cov / (double)Ti;
        if (est >= (1.0 + epsp) * x) {
            LB = est / (1.0 + epsp);
            break;
        }
    }
    uint64_t T = (uint64_t)std::ceil(lambda_star / LB);
    uint64_t j_lo = 0;
    if (fresh_final) {
        j_lo = Ti;
    } else if (T < Ti) {
        T = Ti;
    }
    orc_pool_extend(h, j_lo + T, nthreads);
    uint64_t cov = 0;
    greedy_from(n, p->sets, j_lo, j_lo + T, k, seeds, marginal, &cov);
    if (round_T) round_T[rounds < 63 ? rounds : 63] = j_lo + T;
    *influence = dn * (double)cov / (double)T;
    *theta = T;
    *covered_out = cov;
    *lb_out = LB;
    *rounds_out = rounds;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Skewness S and density D of the set sizes, Section 3.2, Eq. (2).           */
/* Reading: s is the population standard deviation (1/theta).                 */
/* ------------------------------------------------------------------------- */
void orc_size_stats(const uint64_t *sizes, uint64_t T, uint32_t n, double *skew, double *density) {
    double sum = 0.0;
    for (uint64_t i = 0; i < T; i++) sum += (double)sizes[i];
    double mean = sum / (double)T;
    double m2 = 0.0, m3 = 0.0;
    for (uint64_t i = 0; i < T; i++) {
        double d = (double)sizes[i] - mean;
        m2 += d * d;
        m3 += d * d * d;
    }
    m2 /= (double)T;
    m3 /= (double)T;
    *skew = m2 > 0.0 ? m3 / (m2 * std::sqrt(m2)) : 0.0;
    *density = sum / ((double)T * (double)n);
}

/* ------------------------------------------------------------------------- */
/* Warm-up vertex frequencies (Section 4.2.2; Algorithm 1, first block).      */
/* Reading: the warm-up block is sets [0, W); only sets that will be Huffman- */
/* coded (cut * |R| <= n) count, and a vertex counts once per set.            */
/* ------------------------------------------------------------------------- */
int orc_pool_warmup_freq(void *h, uint64_t W, uint32_t cut, uint32_t *freq) {
    orc_pool *p = (orc_pool *)h;
    if (W > p->sets.size()) return -1;
    std::fill(freq, freq + p->g.n, 0u);
    for (uint64_t j = 0; j < W; j++) {
        const auto &s = p->sets[j];
        if ((uint64_t)cut * s.size() > (uint64_t)p->g.n) continue;
        for (uint32_t v : s) freq[v]++;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Huffman code lengths (Huffman 1952), built with the two-queue method.      */
/* Readings (the paper names BuildHuffmanCode without details):               */
/*  - symbols are the vertices with f > 0, ordered by (f, id) ascending;      */
/*  - each merge takes the two lightest fronts of the leaf queue and the      */
/*    internal-node queue, taking the leaf on equal weight;                   */
/*  - one symbol alone gets length 1;                                         */
/*  - if some length exceeds 32, every f becomes ceil(f/2) (at least 1) and   */
/*    the code is rebuilt.                                                    */
/* ------------------------------------------------------------------------- */
static void huffman_once(const std::vector<uint64_t> &f, std::vector<uint32_t> &len) {
    size_t ns = f.size();
    len.assign(ns, 0);
    if (ns == 0) return;
    if (ns == 1) {
        len[0] = 1;
        return;
    }
    std::vector<uint32_t> order(ns);
    for (size_t i = 0; i < ns; i++) order[i] = (uint32_t)i;
    /* symbols are given in vertex-id order, so a stable sort by f gives (f, id) */
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return f[a] < f[b]; });
    /* nodes: 0..ns-1 leaves, ns.. internal */
    std::vector<uint64_t> w(2 * ns - 1);
    std::vector<int64_t> parent(2 * ns - 1, -1);
    for (size_t i = 0; i < ns; i++) w[i] = f[i];
    size_t lq = 0;              /* next leaf in `order` */
    size_t iq = ns, iend = ns;  /* internal queue [iq, iend) */
    auto take = [&]() -> size_t {
        bool have_leaf = lq < ns, have_int = iq < iend;
        if (have_leaf && (!have_int || w[order[lq]] <= w[iq])) return order[lq++];
        return iq++;
    };
    while (iend < 2 * ns - 1) {
        size_t a = take();
        size_t b = take();
        w[iend] = w[a] + w[b];
        parent[a] = (int64_t)iend;
        parent[b] = (int64_t)iend;
        iend++;
    }
    /* depth, top-down: internal nodes were created in increasing order, the root last */
    std::vector<uint32_t> depth(2 * ns - 1, 0);
    for (int64_t v = (int64_t)(2 * ns - 3); v >= 0; v--) depth[v] = depth[parent[v]] + 1;
    for (size_t i = 0; i < ns; i++) len[i] = depth[i];
}

/* Lengths for `ns` symbols with weights f (in the caller's symbol order). */
int orc_huffman_lengths(uint64_t ns, const uint64_t *f_in, uint32_t *len_out) {
    std::vector<uint64_t> f(f_in, f_in + ns);
    std::vector<uint32_t> len;
    for (;;) {
        huffman_once(f, len);
        uint32_t mx = 0;
        for (uint32_t l : len) mx = std::max(mx, l);
        if (mx <= 32) break;
        for (auto &x : f) x = std::max<uint64_t>(1, (x + 1) / 2);
    }
    std::copy(len.begin(), len.end(), len_out);
    return 0;
}

/*
 * Canonical code assignment (RFC 1951 Section 3.2.2 style) for `ns` symbols
 * with lengths len[] (0 = no code), symbols given in id order.  Coded symbols
 * are ranked by (length, id) ascending; codes of one length are consecutive
 * integers, and the first code of length L is (first code of L-1 + count of
 * L-1) << 1.  Outputs: code (right-aligned) and rank (0xFFFFFFFF = no code).
 * Returns the number of coded symbols.
 */
uint32_t orc_canonical(uint64_t ns, const uint32_t *len, uint32_t *code_out, uint32_t *rank_out) {
    std::vector<uint32_t> order;
    for (uint64_t i = 0; i < ns; i++) {
        code_out[i] = 0;
        rank_out[i] = 0xFFFFFFFFu;
        if (len[i]) order.push_back((uint32_t)i);
    }
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return len[a] < len[b]; });
    uint64_t code = 0;
    uint32_t cur_len = 0;
    for (size_t r = 0; r < order.size(); r++) {
        uint32_t i = order[r];
        if (r == 0) {
            code = 0;
        } else {
            code += 1;
        }
        if (len[i] > cur_len) {
            code <<= (len[i] - cur_len);
            cur_len = len[i];
        }
        code_out[i] = (uint32_t)code;
        rank_out[i] = (uint32_t)r;
    }
    return (uint32_t)order.size();
}

/*
 * Codebook over vertices from warm-up frequencies (Section 4.2.2): vertices with
 * freq > 0 get Huffman lengths (orc_huffman_lengths) and canonical codes
 * (orc_canonical).  Outputs per vertex: len (0 = no code), code, rank.
 * Returns the number of coded vertices.
 */
uint32_t orc_codebook(uint32_t n, const uint32_t *freq, uint32_t *len_of_v, uint32_t *code_of_v,
                      uint32_t *rank_of_v) {
    std::vector<uint32_t> sym;
    std::vector<uint64_t> f;
    for (uint32_t v = 0; v < n; v++)
        if (freq[v] > 0) {
            sym.push_back(v);
            f.push_back(freq[v]);
        }
    std::vector<uint32_t> len(sym.size());
    orc_huffman_lengths(sym.size(), f.data(), len.data());
    for (uint32_t v = 0; v < n; v++) len_of_v[v] = 0;
    for (size_t i = 0; i < sym.size(); i++) len_of_v[sym[i]] = len[i];
    return orc_canonical(n, len_of_v, code_of_v, rank_of_v);
}

/* ------------------------------------------------------------------------- */
/* Per-set encoding (Sections 3.2, 4.2.2, 4.2.3).                             */
/*  - bitmap iff cut * |R| > n (integer compare; equality stays Huffman):     */
/*    n bits, bit v in little-endian 32-bit word v/32 at bit v%32, padding 0. */
/*  - Huffman otherwise: coded vertices in ascending rank (reading: the paper */
/*    moves the current top vertex to the front of each byte-string; rank     */
/*    order puts every frequent vertex first), codes written MSB-first: bit b */
/*    of the stream is bit 7 - b%8 of byte b/8, the last byte zero-padded;    */
/*    uncoded vertices go to the copy array, ascending by id.                 */
/* kind: 0 = Huffman, 1 = bitmap.  bytes: ceil(bits/8) bytes; bitmap:         */
/* ceil(n/32) words.  Returns 0, or -1 if a buffer is too small.              */
/* ------------------------------------------------------------------------- */
int orc_encode_set(uint32_t n, uint32_t cut, const uint32_t *len_of_v, const uint32_t *code_of_v,
                   const uint32_t *rank_of_v, const uint32_t *set, uint64_t size, uint32_t *kind,
                   uint32_t *n_coded, uint64_t *code_bits, uint8_t *bytes, uint64_t cap_bytes, uint32_t *raw,
                   uint32_t *n_raw, uint32_t *bitmap, uint64_t cap_words) {
    if ((uint64_t)cut * size > (uint64_t)n) {
        uint64_t words = ((uint64_t)n + 31) / 32;
        if (words > cap_words) return -1;
        for (uint64_t w = 0; w < words; w++) bitmap[w] = 0;
        for (uint64_t i = 0; i < size; i++) bitmap[set[i] / 32] |= 1u << (set[i] % 32);
        *kind = 1;
        *n_coded = 0;
        *n_raw = 0;
        *code_bits = 0;
        return 0;
    }
    std::vector<std::pair<uint32_t, uint32_t>> coded;  /* (rank, vertex) */
    std::vector<uint32_t> uncoded;
    for (uint64_t i = 0; i < size; i++) {
        uint32_t v = set[i];
        if (rank_of_v[v] != 0xFFFFFFFFu) coded.push_back({rank_of_v[v], v});
        else uncoded.push_back(v);
    }
    std::sort(coded.begin(), coded.end());
    std::sort(uncoded.begin(), uncoded.end());
    uint64_t bits = 0;
    for (auto &c : coded) bits += len_of_v[c.second];
    uint64_t nbytes = (bits + 7) / 8;
    if (nbytes > cap_bytes) return -1;
    for (uint64_t b = 0; b < nbytes; b++) bytes[b] = 0;
    uint64_t pos = 0;
    for (auto &c : coded) {
        uint32_t L = len_of_v[c.second], code = code_of_v[c.second];
        for (uint32_t t = 0; t < L; t++) {
            uint32_t bit = (code >> (L - 1 - t)) & 1u;
            if (bit) bytes[pos / 8] |= (uint8_t)(0x80u >> (pos % 8));
            pos++;
        }
    }
    for (size_t i = 0; i < uncoded.size(); i++) raw[i] = uncoded[i];
    *kind = 0;
    *n_coded = (uint32_t)coded.size();
    *n_raw = (uint32_t)uncoded.size();
    *code_bits = bits;
    return 0;
}

/*
 * Inverse of orc_encode_set: rebuild the sorted vertex list.  Huffman streams
 * are decoded bit by bit, matching the prefix against the codebook of each
 * length in turn.  Returns the set size, or -1 on a malformed stream.
 */
int64_t orc_decode_set(uint32_t n, const uint32_t *len_of_v, const uint32_t *code_of_v, uint32_t kind,
                       uint32_t n_coded, uint64_t code_bits, const uint8_t *bytes, const uint32_t *raw,
                       uint32_t n_raw, const uint32_t *bitmap, uint32_t *out) {
    std::vector<uint32_t> s;
    if (kind == 1) {
        for (uint32_t v = 0; v < n; v++)
            if (bitmap[v / 32] >> (v % 32) & 1u) s.push_back(v);
    } else {
        /* (length, code) -> vertex */
        std::vector<std::vector<std::pair<uint32_t, uint32_t>>> by_len(33);
        for (uint32_t v = 0; v < n; v++)
            if (len_of_v[v]) by_len[len_of_v[v]].push_back({code_of_v[v], v});
        for (auto &b : by_len) std::sort(b.begin(), b.end());
        uint64_t pos = 0;
        for (uint32_t i = 0; i < n_coded; i++) {
            uint64_t acc = 0;
            bool found = false;
            for (uint32_t L = 1; L <= 32 && !found; L++) {
                if (pos >= code_bits) return -1;
                acc = (acc << 1) | ((bytes[pos / 8] >> (7 - pos % 8)) & 1u);
                pos++;
                auto &b = by_len[L];
                auto it = std::lower_bound(b.begin(), b.end(), std::make_pair((uint32_t)acc, 0u));
                if (it != b.end() && it->first == (uint32_t)acc) {
                    s.push_back(it->second);
                    found = true;
                }
            }
            if (!found) return -1;
        }
        if (pos != code_bits) return -1;
        for (uint32_t i = 0; i < n_raw; i++) s.push_back(raw[i]);
        std::sort(s.begin(), s.end());
    }
    std::copy(s.begin(), s.end(), out);
    return (int64_t)s.size();
}

/* ------------------------------------------------------------------------- */
/* Paper-literal modes (the results must equal the plain greedy's).           */
/* ------------------------------------------------------------------------- */

/* Exact argmax of a frequency table: the largest count, the lowest vertex id  */
/* on ties, chosen vertices excluded (with every count 0 the lowest-id vertex  */
/* not yet chosen).                                                            */
static uint32_t argmax_unchosen(const std::vector<uint64_t> &h, const std::vector<uint8_t> &chosen) {
    uint32_t n = (uint32_t)h.size(), best = n;
    for (uint32_t v = 0; v < n; v++) {
        if (chosen[v]) continue;
        if (best == n || h[v] > h[best]) best = v;
    }
    return best;
}

/*
 * Greedy with the frequency table rebuilt from scratch every iteration, as
 * Algorithms 2 and 3 print it: h <- counts over the sets not yet covered;
 * u* <- argmax h; every live set holding u* is deleted.  Exactly k seeds.
 */
int orc_pool_greedy_recount(void *hp, uint64_t T, uint32_t k, uint32_t *seeds, uint64_t *marginal,
                            uint64_t *covered_out) {
    orc_pool *p = (orc_pool *)hp;
    uint32_t n = p->g.n;
    if (T > p->sets.size() || k > n) return -1;
    std::vector<uint8_t> alive(T, 1), chosen(n, 0);
    uint64_t covered = 0;
    for (uint32_t it = 0; it < k; it++) {
        std::vector<uint64_t> h(n, 0);
        for (uint64_t j = 0; j < T; j++)
            if (alive[j])
                for (uint32_t v : p->sets[j]) h[v]++;
        uint32_t u = argmax_unchosen(h, chosen);
        chosen[u] = 1;
        seeds[it] = u;
        uint64_t gain = 0;
        for (uint64_t j = 0; j < T; j++) {
            if (alive[j] && std::binary_search(p->sets[j].begin(), p->sets[j].end(), u)) {
                alive[j] = 0;
                gain++;
            }
        }
        covered += gain;
        if (marginal) marginal[it] = gain;
    }
    if (covered_out) *covered_out = covered;
    return 0;
}

/*
 * Characterize (Algorithm 1, first block): the skewness S (Eq. (2)) of the
 * sizes of the warm-up sets [0, W) picks the scheme for the whole graph:
 * Bitmax (every set a bitmap) when S < 0, else Huffmax (every set Huffman-
 * coded, uncoded vertices in copy arrays).  Returns 1 for Bitmax, 0 for
 * Huffmax, -1 on bad arguments; *skew_out gets S.
 */
int orc_pool_scheme(void *hp, uint64_t W, double *skew_out) {
    orc_pool *p = (orc_pool *)hp;
    if (W == 0 || W > p->sets.size()) return -1;
    std::vector<uint64_t> sizes(W);
    for (uint64_t j = 0; j < W; j++) sizes[j] = p->sets[j].size();
    double skew = 0.0, density = 0.0;
    orc_size_stats(sizes.data(), W, p->g.n, &skew, &density);
    if (skew_out) *skew_out = skew;
    return skew < 0.0 ? 1 : 0;
}

/*
 * Bitmax block (Section 4.2.3) in the vertex-major form of Eq. (3): rows are
 * vertices, columns are sets.  Tile t holds columns [32t, 32t + 32): word v of
 * tile t (tiles[t * n + v]) has bit s set iff v is in set 32t + s; columns past
 * T are zero.
 */
int orc_pool_bitmax_tiles(void *hp, uint64_t T, uint32_t *tiles) {
    orc_pool *p = (orc_pool *)hp;
    uint32_t n = p->g.n;
    if (T > p->sets.size()) return -1;
    uint64_t nt = (T + 31) / 32;
    std::fill(tiles, tiles + nt * n, 0u);
    for (uint64_t j = 0; j < T; j++)
        for (uint32_t v : p->sets[j]) tiles[(j / 32) * n + v] |= 1u << (j % 32);
    return 0;
}

/*
 * BitmaxQuery (Algorithm 3; Eq. (3)) over vertex-major tiles: every iteration
 * POPCOUNT gives each row's frequency, u* is the argmax over rows not yet
 * chosen (deleteVTXflag), its popcount is the marginal gain, and every row v is
 * replaced by SUBTRACT(v, u*) = v AND (v XOR u*), which clears the columns of
 * the sets u* covers.  The tiles are modified in place.
 */
int orc_bitmax_query(uint32_t n, uint64_t T, uint32_t *tiles, uint32_t k, uint32_t *seeds, uint64_t *marginal,
                     uint64_t *covered_out) {
    if (k > n) return -1;
    uint64_t nt = (T + 31) / 32;
    std::vector<uint8_t> chosen(n, 0);
    std::vector<uint32_t> urow(nt);
    uint64_t covered = 0;
    for (uint32_t it = 0; it < k; it++) {
        std::vector<uint64_t> h(n, 0);
        for (uint32_t v = 0; v < n; v++)
            for (uint64_t t = 0; t < nt; t++) h[v] += (uint64_t)__builtin_popcount(tiles[t * n + v]);
        uint32_t u = argmax_unchosen(h, chosen);
        chosen[u] = 1;
        seeds[it] = u;
        for (uint64_t t = 0; t < nt; t++) urow[t] = tiles[t * n + u];
        for (uint32_t v = 0; v < n; v++)
            for (uint64_t t = 0; t < nt; t++) {
                uint32_t x = tiles[t * n + v];
                tiles[t * n + v] = x & (x ^ urow[t]);
            }
        covered += h[u];
        if (marginal) marginal[it] = h[u];
    }
    if (covered_out) *covered_out = covered;
    return 0;
}

/*
 * HuffmaxDecodeQuery (Algorithm 2) over the encoded pool: each set j is given
 * as its encoding (kind 0: n_coded codes in code_bits MSB-first bits of
 * bytes[byte_off[j] ..], then n_raw copy-array ids at raw[raw_off[j] ..]; kind
 * 1: a bitmap of ceil(n/32) words at bm[bm_off[j] ..]).  Every iteration the
 * frequency table is rebuilt from the live sets: a live set is decoded; if it
 * holds u* it is deleted, else its vertices are added to the table for the
 * next iteration.  The first table counts every set.
 */
int orc_huffmax_query(uint32_t n, const uint32_t *len_of_v, const uint32_t *code_of_v, uint64_t T,
                      const uint32_t *kind, const uint32_t *n_coded, const uint64_t *code_bits,
                      const uint64_t *byte_off, const uint8_t *bytes, const uint32_t *n_raw,
                      const uint64_t *raw_off, const uint32_t *raw, const uint64_t *bm_off, const uint32_t *bm,
                      uint32_t k, uint32_t *seeds, uint64_t *marginal, uint64_t *covered_out) {
    if (k > n) return -1;
    std::vector<uint32_t> buf(n);
    auto decode = [&](uint64_t j, std::vector<uint32_t> &out) -> bool {
        int64_t sz = orc_decode_set(n, len_of_v, code_of_v, kind[j], n_coded[j], code_bits[j], bytes + byte_off[j],
                                    raw + raw_off[j], n_raw[j], bm + bm_off[j], buf.data());
        if (sz < 0) return false;
        out.assign(buf.begin(), buf.begin() + sz);
        return true;
    };
    std::vector<uint8_t> alive(T, 1), chosen(n, 0);
    std::vector<uint64_t> h(n, 0);
    std::vector<uint32_t> s;
    for (uint64_t j = 0; j < T; j++) {
        if (!decode(j, s)) return -2;
        for (uint32_t v : s) h[v]++;
    }
    uint64_t covered = 0;
    for (uint32_t it = 0; it < k; it++) {
        uint32_t u = argmax_unchosen(h, chosen);
        chosen[u] = 1;
        seeds[it] = u;
        std::vector<uint64_t> next(n, 0);
        uint64_t gain = 0;
        for (uint64_t j = 0; j < T; j++) {
            if (!alive[j]) continue;
            if (!decode(j, s)) return -2;
            if (std::binary_search(s.begin(), s.end(), u)) {
                alive[j] = 0;
                gain++;
            } else {
                for (uint32_t v : s) next[v]++;
            }
        }
        h.swap(next);
        covered += gain;
        if (marginal) marginal[it] = gain;
    }
    if (covered_out) *covered_out = covered;
    return 0;
}

}  /* extern "C" */
