/*
 * hbx.h -- C ABI of the GB300 library for influence maximization over
 * compressed reverse-reachable (RR) sets.
 *
 * Method: HBMax (arXiv 2208.00613).  The library runs the data-parallel hot path
 * of IMM on one GPU:
 *   (a) random RR sets under IC or LT (Section 2.1; Section 2.2, Definitions 1-2),
 *   (b) each set encoded as it is sampled, with canonical Huffman codes learned
 *       from a warm-up block or as a bitmap when dense (Section 3.2; Section 4.2,
 *       Algorithm 1),
 *   (c) greedy max-coverage seed selection on the encoded sets (Section 4.3,
 *       Algorithms 2 and 3),
 * driven by IMM's sampling bound (Section 2.2, Eq. (1)).
 *
 * Conventions for every call:
 *  - Return 0 (HBX_OK) on success, a negative HBX_ERR_* code on failure.  The
 *    context keeps a message for the last failure (hbx_last_error).
 *  - Handles (hbx_ctx, hbx_graph, hbx_pool, hbx_server, hbx_ticket) are owned by
 *    the library and freed by the matching *_destroy call.  Every array passed
 *    in is owned by the caller; the library copies what it keeps.  Host arrays
 *    are plain host pointers; no call takes device pointers unless it says so.
 *  - Vertex ids are 0..n-1 (uint32).  The graph is a *transposed* CSR: the
 *    in-edges (u -> v) of v are col[e] = u for e in [row_ptr[v], row_ptr[v+1]);
 *    e is the edge id used by the random stream.
 *  - Results are bit-identical for any launch shape, batching, encoding or
 *    serving mix: RR set j is a pure function of (graph, model, seed, epoch, j).
 *  - A context is not thread-safe; the serving calls synchronise internally.
 */
#ifndef HBX_H
#define HBX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hbx_ctx hbx_ctx;
typedef struct hbx_graph hbx_graph;
typedef struct hbx_pool hbx_pool;
typedef struct hbx_server hbx_server;
typedef struct hbx_ticket hbx_ticket;

/* Diffusion models of Section 2.1. */
typedef enum { HBX_IC = 0, HBX_LT = 1 } hbx_model;

enum {
    HBX_OK = 0,
    HBX_ERR_INVALID_ARG = -1,  /* bad size, id, probability, option or handle */
    HBX_ERR_OOM = -2,          /* device allocation failed or over max_device_bytes */
    HBX_ERR_CUDA = -3,         /* a CUDA call failed; message in hbx_last_error */
    HBX_ERR_TIMEOUT = -4,      /* a bounded wait ran out (hbx_wait, or a device-side wait) */
    HBX_ERR_WEIGHTS_GT_1 = -5, /* an LT vertex's in-weights sum above 1 */
    HBX_ERR_ADMISSION = -6,    /* a served query can never fit the memory budget */
    HBX_ERR_CANCELLED = -7,    /* a served query was cancelled */
    HBX_ERR_INTERNAL = -8      /* a kernel reported an inconsistent state */
};

/* Set kinds in an RR pool. */
enum { HBX_KIND_HUFFMAN = 0, HBX_KIND_BITMAP = 1, HBX_KIND_RAW = 2 };

typedef struct {
    /* c: set R is a bitmap iff c * |R| > n (Section 3.2 derives c = 32 from
     * 32-bit ids).  0 selects 32. */
    uint32_t density_cut;
    /* W: sets [0, W) form the warm-up block whose vertex frequencies build the
     * Huffman codebook (Section 4.2.2, Algorithm 1).  0 selects ceil(T_1 / 8),
     * T_1 being IMM's first sampling target. */
    uint32_t warmup_sets;
    /* 0: sets stored uncompressed as 32-bit ids; 1: Huffman + bitmap. */
    uint32_t encode;
    /* 0: plain form, one launch per step: every set of a batch sampled by one
     * thread block with HBM scratch, sets assigned to blocks statically, and
     * the k selection rounds launched one by one with a host read-back after
     * each; 1: persistent work-stealing warp kernel with shared-memory and
     * HBM block tiers for the sets that outgrow it, fused with encoding, and
     * the k selection rounds in one persistent cooperative launch. */
    uint32_t form;
    /* Philox counter word 2 of every draw; pools with different epochs are
     * independent.  Default 0. */
    uint32_t pool_epoch;
    /* Largest set one warp samples in shared memory (power of two, 64..2048);
     * bigger sets go to a block per set.  0 lets the autotuner choose. */
    uint32_t warp_capacity;
    /* Edge groups (4 consecutive in-edges) a warp may scan for one set before
     * the set moves to a block; 0 = 2048 when warp_capacity is given, else
     * autotuned; 0xFFFFFFFF = no limit. */
    uint32_t warp_group_budget;
    /* Blocks of a thread-block cluster that search one heavy set together
     * (1, 2, 4 or 8); 0 = 1 when warp_capacity is given, else autotuned. */
    uint32_t block_cluster;
    /* Upper bound on the device bytes of one pool; 0 = no bound. */
    uint64_t max_device_bytes;
    /* Longest a device-side wait may last, in SM clock cycles (the grid
     * barriers of the batched form's selection); a wait that runs out ends the
     * call with TIMEOUT and leaves the context usable.  0 = 4e9 (about 2 s). */
    uint64_t wait_cycles;
    /* Encoding scheme of an encoded pool.  0: per set, by density_cut (a set
     * is a bitmap iff c * |R| > n).  1: per graph, as Algorithm 1's
     * Characterize does: the skewness S (Eq. (2)) of the warm-up block's set
     * sizes picks Bitmax (every set a bitmap) when S < 0, else Huffmax (every
     * set Huffman-coded, density_cut ignored).  A Bitmax IC pool stores its
     * sets as the vertex-major bit matrix of Section 4.2.3 / Eq. (3): tiles of
     * 32 consecutive sets, word v of a tile holding bit s for set 32t + s; it
     * samples every set with the bit-parallel search. */
    uint32_t scheme;
    /* Greedy counting of the batched form.  0: count once, then decrement the
     * covered sets' vertices each iteration.  1: rebuild the counts from the
     * sets not yet covered every iteration, as Algorithms 2 and 3 print it
     * (Bitmax tiles: POPCOUNT of each row under the live-set mask, i.e. after
     * Eq. (3)'s SUBTRACT).  2: choose per iteration, as Ripples' update-or-
     * recount counting does (Section 2.2): recount when the chosen vertex
     * covers more than half of the sets still live (the rest are then fewer
     * to read than the covered ones), decrement otherwise.  The seeds are the
     * same in every mode; the plain form always decrements. */
    uint32_t select_mode;
    /* IMM's final phase: 0 reuses the estimation rounds' sets (theta =
     * max(T_i, ceil(lambda* / LB)) sets [0, theta)); 1 draws theta =
     * ceil(lambda* / LB) new sets [T_i, T_i + theta) and selects on those only,
     * keeping the two phases independent. */
    uint32_t fresh_final;
    uint32_t reserved_opt;
} hbx_options;

typedef struct {
    uint64_t theta;            /* RR sets used for the final selection */
    uint64_t covered;          /* sets covered by the k seeds */
    uint64_t sets_huffman, sets_bitmap, sets_raw;
    uint64_t sets_big;         /* sets sampled by a whole block (> warp capacity) */
    uint64_t rr_vertices;      /* sum of |R_j| over the pool */
    uint64_t edges_scanned;    /* in-edges of the sets' members (IC) or weights read (LT) */
    uint64_t edges_live;       /* live in-edges found; for IC sets searched bit-parallel (those
                                  that outgrow shared memory) only the live edges into sources
                                  not yet in the set at the edge's BFS level */
    uint64_t pool_bytes;       /* index + code + copy + bitmap heaps in use */
    uint64_t raw_int32_bytes;  /* 4 * rr_vertices + 8 * theta: the uncompressed pool */
    uint64_t code_bits;        /* Huffman payload bits */
    uint64_t warmup_sets;      /* W used */
    uint32_t rounds;           /* IMM estimation rounds run */
    uint32_t warp_capacity;    /* launch shape used */
    uint32_t warp_group_budget;
    uint32_t block_cluster;
    double lb;                 /* IMM lower bound on OPT */
    double sample_s, select_s, total_s;
    double skewness, density;  /* Eq. (2) over the pool's set sizes */
    /* device time (CUDA events on the library's stream) of the sampling kernels
     * that produced the pool's sets (warm-up and calibration passes excluded),
     * and the number of those launches */
    double sample_kernel_s;
    uint64_t sample_kernel_launches;
    /* every kernel the library launched for this pool or query (graph nodes
     * included) */
    uint64_t kernel_launches;
    /* device time (CUDA events) of the selections' count passes -- the initial
     * per-vertex occurrence counts over the sets each selection counted -- and
     * the bytes those passes read: 4 per heap word of the counted sets, 16 per
     * set record, 8 per chunk item and 4 per bitmap-list entry */
    double count_kernel_s;
    uint64_t count_bytes;
    /* the bit-parallel search of the IC sets that outgrow shared memory:
     * device time of its batches (levels, tally, emit), sets searched, and
     * Philox blocks drawn (one per edge group and set that needed coins) */
    double ms_kernel_s;
    uint64_t ms_sets;
    uint64_t ms_philox_blocks;
    /* greedy iterations of the selections: device time (CUDA events around
     * them, the initial count excluded), iterations run, and for the batched
     * form the time of their cover-and-decrement phases (the persistent
     * kernel decrements a covered set where it finds it) and the bytes the
     * decrements read (code bytes and items of the covered Huffman sets'
     * chunks, copy-array ids, covered bitmap rows or tiles) */
    double select_kernel_s;
    uint64_t select_iterations;
    double dec_s;
    uint64_t dec_bytes;
    /* vertex occurrences of Huffman sets stored in copy arrays (no code) */
    uint64_t uncoded_vertices;
    /* encoding scheme in effect: 0 per-set density cut, 1 Huffmax, 2 Bitmax
     * (the per-graph scheme), 3 Bitmax in vertex-major tiles; and the warm-up
     * sizes' skewness that the per-graph scheme decided on */
    uint32_t scheme;
    /* launch shape: capacity of the second warp tier that takes the sets
     * outgrowing warp_capacity before the block tiers (0: none) */
    uint32_t second_warp_capacity;
    double scheme_skewness;
    /* batched form: time of the selections' argmax phases (barrier to
     * barrier, as dec_s) */
    double argmax_s;
    /* the bit-parallel search: edge groups staged (one per in-edge group of a
     * frontier vertex per level, for all the sets that expand it then), and
     * vertex expansions deferred by a level so that more sets share one */
    uint64_t ms_group_visits;
    uint64_t ms_deferrals;
} hbx_stats;

/* Human-readable name of an HBX_ERR_* code. */
const char *hbx_strerror(int code);

/* Message of the last failure on ctx ("" if none). */
const char *hbx_last_error(const hbx_ctx *ctx);

/* Defaults: density_cut 32, warmup_sets 0 (auto), encode 1, form 1, epoch 0,
 * warp_capacity 0 and warp_group_budget 0 (autotune), max_device_bytes 0. */
void hbx_default_options(hbx_options *opts);

/* Create a context on CUDA device `cuda_device`.  `cuda_stream` is a
 * cudaStream_t to run on (NULL: the library creates its own).  Errors:
 * INVALID_ARG (no such device), CUDA. */
int hbx_create(hbx_ctx **out, int cuda_device, void *cuda_stream);

/* Route every later device allocation of ctx through alloc/free (for example a
 * framework's caching allocator).  alloc(bytes, user) returns a device pointer
 * or NULL; free(ptr, user) releases it.  Allocations must be 256-byte aligned.
 * Passing NULL for both restores cudaMalloc/cudaFree. */
int hbx_set_allocator(hbx_ctx *ctx, void *(*alloc_fn)(size_t bytes, void *user),
                      void (*free_fn)(void *ptr, void *user), void *user);

/* Destroy ctx and everything created from it that is still alive. */
void hbx_destroy(hbx_ctx *ctx);

/*
 * Copy a graph G = (V, E, w) (Section 2.1) to the device.
 *   n, m        vertex and edge counts; 2 <= n, m < 2^32.
 *   row_ptr     host, n+1 entries, row_ptr[0] = 0, row_ptr[n] = m, non-decreasing.
 *   col         host, m entries < n: col[e] is the source of in-edge e.
 *   ic_prob     host, m entries in [0, 1], or NULL: IC activation probability
 *               p(u, v) of edge e (Section 2.1).  Needed for HBX_IC.
 *   lt_weight   host, m entries in [0, 1], or NULL: LT in-weight of edge e
 *               (Section 2.1).  Stored as floor(w * 2^32) (at most 2^32 - 1);
 *               a vertex whose stored weights sum above 2^32 fails with
 *               WEIGHTS_GT_1.  Needed for HBX_LT.
 * Errors: INVALID_ARG, WEIGHTS_GT_1, OOM, CUDA.
 */
int hbx_graph_create(hbx_ctx *ctx, uint32_t n, uint64_t m, const uint32_t *row_ptr, const uint32_t *col,
                     const float *ic_prob, const float *lt_weight, hbx_graph **out);
void hbx_graph_destroy(hbx_graph *g);

/*
 * Influence maximization (Section 2.1) by IMM (Section 2.2): choose k seeds
 * maximising the expected spread under `model`, with error eps and failure
 * probability n^-ell.  Sampling follows Eq. (1) with eps' = sqrt(2) eps and
 * l' = l (1 + ln 2 / ln n); the rounds, the final theta = ceil(lambda* / LB) and
 * the estimate n * covered / theta are computed in FP64.  A fresh pool is built
 * and released inside the call.
 *   seeds_out      host, k entries (caller-owned): the seeds in selection order.
 *   influence_out  host: n * covered / theta.
 *   marginal_out   host, k entries or NULL: sets newly covered by each seed.
 *   stats_out      host or NULL.
 * Errors: INVALID_ARG (k == 0 or k > n, eps not in (0,1), ell <= 0, model
 * without its parameters), OOM, CUDA, INTERNAL.
 */
int hbx_imm(hbx_ctx *ctx, hbx_graph *g, hbx_model model, uint32_t k, double eps, double ell, uint64_t seed,
            const hbx_options *opts, uint32_t *seeds_out, double *influence_out, uint64_t *marginal_out,
            hbx_stats *stats_out);

/*
 * An RR pool: the sets R_0, R_1, ... of one (graph, model, seed, epoch), kept on
 * the device in the form chosen by opts (Algorithm 1's encoded blocks).  With
 * encode = 1 the codebook is built, on the first hbx_pool_extend, from the
 * warm-up sets [0, W), W = opts->warmup_sets (must be > 0 here).
 * Errors: INVALID_ARG, OOM, CUDA.
 */
int hbx_pool_create(hbx_ctx *ctx, hbx_graph *g, hbx_model model, uint64_t seed, const hbx_options *opts,
                    hbx_pool **out);
void hbx_pool_destroy(hbx_pool *p);

/* Sample (and encode) sets [size, T).  T < 2^32.  Errors: INVALID_ARG, OOM, CUDA. */
int hbx_pool_extend(hbx_pool *p, uint64_t T);

/* Number of sets in the pool. */
uint64_t hbx_pool_size(const hbx_pool *p);

/*
 * Greedy max coverage (Section 2.2; Algorithms 2-3) over sets [0, T) of the
 * pool, T <= size: k times take the vertex in the most uncovered sets (lowest
 * id on ties; once all counts are 0, the lowest-id vertex not chosen), cover
 * its sets.  seeds: k entries; marginal: k entries or NULL; covered: or NULL.
 * All host pointers.  Errors: INVALID_ARG, CUDA.
 */
int hbx_pool_select(hbx_pool *p, uint64_t T, uint32_t k, uint32_t *seeds, uint64_t *marginal,
                    uint64_t *covered);

/* IMM (as hbx_imm) reusing and extending an existing pool. */
int hbx_imm_pool(hbx_pool *p, uint32_t k, double eps, double ell, uint32_t *seeds_out, double *influence_out,
                 uint64_t *marginal_out, hbx_stats *stats_out);

/*
 * Export set j as stored (for inspection and tests).  Identity of a set is
 * (kind, size, n_coded, code bits, copy array, bitmap bits); heap placement is
 * not part of it.
 *   kind      HBX_KIND_*.
 *   payload   host buffer of cap bytes:
 *             HUFFMAN: ceil(code_bits/8) code bytes (MSB-first within a byte,
 *                      codes in ascending codebook rank, zero-padded), then the
 *                      copy array (uncoded vertex ids, ascending) as n_raw
 *                      little-endian uint32 starting at the next multiple of 4;
 *             BITMAP:  ceil(n/32) little-endian uint32 words, bit v of the set
 *                      at word v/32, bit v%32 (Section 4.2.3; padding bits 0);
 *             RAW:     size uint32 ids in sampling order.
 *   nbytes    bytes written (or needed, if cap is too small: then INVALID_ARG).
 */
int hbx_pool_export_set(hbx_pool *p, uint64_t j, uint32_t *kind, uint32_t *size, uint32_t *n_coded,
                        uint32_t *n_raw, uint64_t *code_bits, uint8_t *payload, uint64_t cap,
                        uint64_t *nbytes);

/*
 * Decode sets [j0, j1) on the device with the same decoder the selection uses
 * and return them sorted: offsets (j1-j0+1 entries) and verts (cap entries),
 * both host.  Errors: INVALID_ARG (cap too small; *needed holds the total).
 */
int hbx_pool_decode_sets(hbx_pool *p, uint64_t j0, uint64_t j1, uint64_t *offsets, uint32_t *verts,
                         uint64_t cap, uint64_t *needed);

/*
 * Export the pool's codebook (Section 4.2.2): per vertex its code length (0 =
 * no code: the vertex goes to copy arrays), its canonical code (right-aligned)
 * and its rank (0xFFFFFFFF = none), plus the warm-up frequency table used.
 * Each array: n host entries.  Errors: INVALID_ARG (no codebook).
 */
int hbx_pool_export_codebook(hbx_pool *p, uint32_t *len_of_v, uint32_t *code_of_v, uint32_t *rank_of_v,
                             uint32_t *freq);

/* Pool statistics (theta = pool size here; selection fields zero). */
int hbx_pool_stats(hbx_pool *p, hbx_stats *stats);

/*
 * Serving (continuous batching): queries arrive at any time; a worker thread
 * admits each as device memory allows (by the projected compressed footprint of
 * its pool), keeps graphs and pools resident across queries keyed by (graph,
 * model, seed, epoch), and overlaps the work of admitted queries on separate
 * streams.  Results equal those of hbx_imm for the same arguments.
 *   hbx_server_create  max_inflight concurrent queries, memory budget in bytes
 *                      (0 = 90% of free device memory).
 *   hbx_submit         non-blocking; returns a ticket.  ADMISSION if the
 *                      query's projected footprint exceeds the whole budget.
 *   hbx_wait           blocks up to timeout_us (< 0: forever); TIMEOUT if not
 *                      done (the ticket stays valid).  Fills the outputs and the
 *                      query's latency (seconds from submit to completion).
 *   hbx_cancel         cancel a query that has not started: its wait returns
 *                      CANCELLED.
 *   hbx_ticket_destroy release a completed or cancelled ticket.
 */
int hbx_server_create(hbx_ctx *ctx, uint32_t max_inflight, uint64_t memory_budget, hbx_server **out);
void hbx_server_destroy(hbx_server *s);
int hbx_submit(hbx_server *s, hbx_graph *g, hbx_model model, uint32_t k, double eps, double ell, uint64_t seed,
               const hbx_options *opts, hbx_ticket **out);
int hbx_wait(hbx_ticket *t, uint32_t *seeds_out, double *influence_out, hbx_stats *stats_out,
             double *latency_s, int64_t timeout_us);
int hbx_cancel(hbx_ticket *t);
void hbx_ticket_destroy(hbx_ticket *t);

/*
 * Measurement aid (the paper has no counterpart): the device's rate of IC coin
 * blocks as the bit-parallel search of the sets that outgrow shared memory
 * computes them -- the part of Philox4x32-10 that depends on both the edge
 * group and the set (15 of its 20 wide multiplies; the other 5 are shared by
 * every set of a group or every group of a set) -- with every thread finishing
 * blocks back to back and touching no memory but one output word.  Best of
 * three timed launches on the context's stream after one warm-up launch.
 *   blocks_per_s  out: coin blocks per second.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
int hbx_philox_ceiling(hbx_ctx *ctx, double *blocks_per_s);

/*
 * Allocation-free argmax over a device array of counts.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device
 * memory where they need it -- a service that reserves all of its GPU memory up
 * front and must stay within that fixed budget, or code running inside a
 * memory allocator's own hook, where allocating again would re-enter the
 * allocator.  It runs the selection's argmax (largest count, lowest id on
 * ties; any int32 values) but keeps its scratch (per-block partial maxima and a
 * finish counter, 32 KB) in a static device array that every device loading
 * the library holds until the process exits.  It calls no allocation routine
 * (see the set-up below).
 *   d_counts  device pointer, n int32 counts, on the current device.
 *   n         1 .. HBX_ARGMAX_NOALLOC_MAX; larger n fails with INVALID_ARG.
 *   d_out     device pointer to one uint32: the winning index, written when the
 *             stream reaches the launch (the call does not synchronise).
 *   stream    cudaStream_t of the current device (NULL = legacy default stream).
 * The first call on a device does a one-time set-up with that device current:
 * it loads the library's device code on that device (CUDA loads modules lazily,
 * and loading reserves device memory for the code and the 32 KB array) and
 * looks up the scratch array's device address.  Only the calls after it are
 * allocation-free, so make the first call before the memory budget is
 * reserved and before any stream capture.  A call with d_counts == NULL,
 * n == 0 and d_out == NULL does only that set-up and launches nothing.  All
 * calls on a device share the array: calls whose launches overlap on the GPU
 * race and must be ordered by the caller (one stream, or events).
 * Errors: INVALID_ARG, CUDA.
 */
#define HBX_ARGMAX_NOALLOC_MAX 16777216u
int hbx_argmax_noalloc(const int32_t *d_counts, uint32_t n, uint32_t *d_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HBX_H */
