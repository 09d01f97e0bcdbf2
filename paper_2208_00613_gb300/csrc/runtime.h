// Host-side objects behind the opaque handles of include/hbx.h.
#pragma once
#include <cuda_runtime.h>

#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "hbx.h"
#include "internal.h"

namespace hbx {
// launch shape of the sampler: warp capacity and warp edge-group budget
struct Shape {
    uint32_t qw;
    uint32_t gb;
    uint32_t bc;  // blocks per cluster working on one heavy set
    uint32_t q2;  // capacity of a second warp tier for the sets that outgrow qw (0: none)
};
struct Heap {
    uint32_t* d = nullptr;
    uint64_t cap = 0;  // words usable (the allocation has slack words beyond)
};
}  // namespace hbx

struct hbx_ctx {
    int device = 0;
    int sms = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* (*alloc_fn)(size_t, void*) = nullptr;
    void (*free_fn)(void*, void*) = nullptr;
    void* alloc_user = nullptr;
    std::string last_error;
    std::map<void*, size_t> sizes;  // live device allocations
    size_t live_bytes = 0;
    std::set<hbx_graph*> graphs;
    std::set<hbx_pool*> pools;
    std::set<hbx_server*> servers;
    // autotuned launch shapes, keyed by (graph fingerprint, model)
    std::map<std::pair<uint64_t, int>, hbx::Shape> tuned;
    std::mutex mu;  // guards allocation bookkeeping when a server worker runs
};

struct hbx_graph {
    hbx_ctx* ctx = nullptr;
    uint32_t n = 0, m = 0;
    uint32_t max_indeg = 0;
    uint64_t fingerprint = 0;  // hash of sizes and sampled CSR entries
    uint32_t* row_ptr = nullptr;
    uint32_t* col = nullptr;
    uint32_t* thr = nullptr;  // IC live thresholds ceil(p * 2^24), 4*ceil(m/4) entries
    uint32_t* q = nullptr;  // LT fixed-point weights
};


struct hbx_pool {
    hbx_ctx* ctx = nullptr;
    hbx_graph* g = nullptr;
    hbx_model model = HBX_IC;
    uint64_t seed = 0;
    hbx_options o{};
    uint64_t T = 0;
    hbx::Shape shape{0, 0};
    size_t device_bytes = 0;
    hbx::SetRec* recs = nullptr;
    uint64_t rec_cap = 0;
    hbx::Heap raw, code, bm;
    hbx::Counters* ctr = nullptr;
    hbx::Counters hc{};
    double* moments = nullptr;
    unsigned long long aux_scanned = 0, aux_live = 0;  // edges of warm-up/calibration passes
    uint64_t hist_sets = 0, hist_dense = 0, hist_verts = 0;  // warm-up pass: sets, dense sets, other vertices
    // effective density cut: the option, or from the per-graph scheme 0
    // (Huffmax) or n + 1 (Bitmax)
    uint32_t cut = 32;
    bool bitmax = false;   // per-graph scheme chose Bitmax
    bool tiles = false;    // bitmap sets are columns of vertex-major 32-set tiles
    double scheme_skew = 0.0;
    uint32_t* wsizes = nullptr;  // warm-up set sizes, during the warm-up pass of the per-graph scheme
    uint32_t wsizes_cap = 0;
    // codebook
    bool has_cb = false;
    uint64_t W = 0;
    uint32_t nsym = 0, max_len = 0;
    uint32_t *rank_of = nullptr, *vertex_of_rank = nullptr, *code_of_rank = nullptr, *lut = nullptr, *dec = nullptr;
    uint8_t* len_of_rank = nullptr;
    std::vector<uint32_t> h_freq, h_len, h_code, h_rank;
    // selection index
    unsigned long long* items = nullptr;
    uint64_t items_cap = 0;
    uint32_t* bm_sets = nullptr;
    uint64_t bm_list_cap = 0;
    // sampling lists
    uint32_t *big_list = nullptr, *retry_list = nullptr, *list_in = nullptr, *giant_list = nullptr;
    uint64_t list_cap = 0;
    // block-path scratch
    uint32_t *bp_visited = nullptr, *bp_rbits = nullptr, *bp_aux = nullptr, *bp_queue = nullptr;
    uint32_t bp_slots = 0;
    uint64_t bp_words = 0;
    // bit-parallel search scratch (masks and lists of n entries each)
    uint32_t *ms_vis = nullptr, *ms_nxt = nullptr, *ms_F = nullptr, *ms_N = nullptr;  // ms_N: frontier masks
    uint32_t *ms_pend = nullptr, *ms_ndef = nullptr;  // deferred expansions: masks, per-vertex level counts
    uint4* ms_heavy = nullptr;
    uint32_t ms_heavy_cap = 0;
    hbx::MsCounters* ms_c = nullptr;
    uint32_t* ms_sets = nullptr;
    unsigned long long* ms_rowoff = nullptr;
    uint32_t* ms_sparse = nullptr;  // mask bits and ids of a batch's sets under the density cut
    cudaGraphExec_t ms_first = nullptr, ms_more = nullptr;  // the level loop's graphs
    // selection state
    int32_t* cnt = nullptr;
    // counts of sets [0, base_T) before any decrement, kept for the next
    // selection on a longer prefix; bounds: pool size at each batch end ->
    // (chunk items, bitmap list entries) of the sets below it
    int32_t* cnt_base = nullptr;
    uint64_t base_T = 0;
    struct Bound {
        uint64_t items, bm, words;  // chunk items, bitmap-list entries, heap words of the sets below
    };
    std::map<uint64_t, Bound> bounds;
    double count_kernel_s = 0;
    uint64_t count_bytes = 0;
    cudaEvent_t evc0 = nullptr, evc1 = nullptr, evs0 = nullptr, evs1 = nullptr;
    double select_kernel_s = 0, dec_s = 0, argmax_s = 0;
    uint64_t select_iterations = 0, dec_bytes = 0;
    double ms_kernel_s = 0;
    uint64_t ms_nsets = 0, ms_blocks = 0, ms_visits = 0, ms_deferred = 0;
    bool count_pending = false;
    uint8_t* alive = nullptr;
    uint64_t alive_cap = 0;
    uint32_t *cov_huff = nullptr, *cov_bm = nullptr, *cov_raw = nullptr;
    uint32_t* tile_live = nullptr;  // tile pools: live-set mask per tile (recount)
    unsigned long long* dec_items = nullptr;  // chunk items of the sets covered in one iteration
    uint64_t dec_cap = 0;
    void* st = nullptr;
    unsigned long long* partials = nullptr;
    unsigned int* ticket = nullptr;
    uint32_t* d_seeds = nullptr;
    unsigned long long* d_marg = nullptr;
    uint32_t kcap = 0;
    double sample_s = 0, select_s = 0;
    double sample_kernel_s = 0;
    uint64_t sample_kernel_launches = 0;
    uint64_t launches = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // stream of every launch and copy of this pool: the context's stream, or
    // the pool's own one when a server runs pools side by side
    cudaStream_t stream = nullptr;
    bool own_stream = false;
};

namespace hbx {
int fail(hbx_ctx* c, int code, const std::string& msg);
int cuda_fail(hbx_ctx* c, cudaError_t e, const char* what);
int dalloc(hbx_ctx* c, void** p, size_t bytes);
void dfree(hbx_ctx* c, void* p);
int pool_extend(hbx_pool* p, uint64_t T);
// greedy on sets [j_lo, T) (j_lo = 0 or a batch end of the pool)
int pool_select(hbx_pool* p, uint64_t T, uint32_t k, uint32_t* seeds, uint64_t* marginal, uint64_t* covered,
                uint64_t j_lo = 0);
int imm_on_pool(hbx_pool* p, uint32_t k, double eps, double ell, uint32_t* seeds, double* influence,
                uint64_t* marginal, hbx_stats* stats);
void fill_stats(hbx_pool* p, hbx_stats* s);
// lambda' and lambda* of the IMM bounds (false on bad arguments)
bool imm_lambda(uint32_t n, uint32_t k, double eps, double ell, double* lambda_p, double* lambda_star);
}  // namespace hbx

void hbx_server_destroy_all(hbx_ctx* c);
