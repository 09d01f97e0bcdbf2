// Host runtime of the library: contexts, graphs, RR pools, the IMM driver and
// the C ABI (include/hbx.h).
//
// Compiled with -ffp-contract=off: the IMM bounds of Section 2.2 / Eq. (1) are
// FP64 expressions whose rounding must not depend on contraction.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "hbx.h"
#include "internal.h"
#include "runtime.h"

using namespace hbx;

// ===========================================================================
// errors and device memory
// ===========================================================================
namespace hbx {

int fail(hbx_ctx* c, int code, const std::string& msg) {
    if (c) {
        std::lock_guard<std::mutex> lock(c->mu);
        c->last_error = msg;
    }
    return code;
}

int cuda_fail(hbx_ctx* c, cudaError_t e, const char* what) {
    return fail(c, HBX_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int dalloc(hbx_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~(size_t)255;
    if (c->alloc_fn) {
        *p = c->alloc_fn(bytes, c->alloc_user);
        if (!*p) return fail(c, HBX_ERR_OOM, "allocator returned NULL for " + std::to_string(bytes) + " bytes");
        if (((uintptr_t)*p) & 255) {
            c->free_fn(*p, c->alloc_user);
            *p = nullptr;
            return fail(c, HBX_ERR_INVALID_ARG, "allocator returned memory not 256-byte aligned");
        }
    } else {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return fail(c, HBX_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
        }
    }
    {
        std::lock_guard<std::mutex> lock(c->mu);
        c->live_bytes += bytes;
        c->sizes[*p] = bytes;
    }
    return HBX_OK;
}

void dfree(hbx_ctx* c, void* p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lock(c->mu);
        auto it = c->sizes.find(p);
        if (it != c->sizes.end()) {
            c->live_bytes -= it->second;
            c->sizes.erase(it);
        }
    }
    if (c->free_fn) c->free_fn(p, c->alloc_user);
    else cudaFree(p);
}

}  // namespace hbx

#define CK(call)                                                 \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)
#define RC(call)                  \
    do {                          \
        int r_ = (call);          \
        if (r_ != HBX_OK) return r_; \
    } while (0)

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ===========================================================================
// context
// ===========================================================================
extern "C" const char* hbx_strerror(int code) {
    switch (code) {
        case HBX_OK: return "ok";
        case HBX_ERR_INVALID_ARG: return "invalid argument";
        case HBX_ERR_OOM: return "out of device memory";
        case HBX_ERR_CUDA: return "CUDA error";
        case HBX_ERR_TIMEOUT: return "timed out";
        case HBX_ERR_WEIGHTS_GT_1: return "LT in-weights of a vertex sum above 1";
        case HBX_ERR_ADMISSION: return "query can never fit the memory budget";
        case HBX_ERR_CANCELLED: return "cancelled";
        case HBX_ERR_INTERNAL: return "internal error";
        default: return "unknown error";
    }
}

extern "C" const char* hbx_last_error(const hbx_ctx* c) { return c ? c->last_error.c_str() : "no context"; }

extern "C" void hbx_default_options(hbx_options* o) {
    if (!o) return;
    o->density_cut = 32;
    o->warmup_sets = 0;
    o->encode = 1;
    o->form = 1;
    o->pool_epoch = 0;
    o->warp_capacity = 0;
    o->warp_group_budget = 0;
    o->block_cluster = 0;
    o->max_device_bytes = 0;
    o->wait_cycles = 0;
    o->scheme = 0;
    o->select_mode = 0;
    o->fresh_final = 0;
    o->reserved_opt = 0;
}

extern "C" int hbx_create(hbx_ctx** out, int dev, void* stream) {
    if (!out) return HBX_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || dev < 0 || dev >= ndev) {
        cudaGetLastError();
        return HBX_ERR_INVALID_ARG;
    }
    hbx_ctx* ctx = new hbx_ctx();
    ctx->device = dev;
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess) {
        delete ctx;
        return HBX_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev);
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
        ctx->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return HBX_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    *out = ctx;
    return HBX_OK;
}

extern "C" int hbx_set_allocator(hbx_ctx* c, void* (*a)(size_t, void*), void (*f)(void*, void*), void* user) {
    if (!c) return HBX_ERR_INVALID_ARG;
    if ((a == nullptr) != (f == nullptr)) return fail(c, HBX_ERR_INVALID_ARG, "alloc and free must both be set");
    if (!c->sizes.empty()) return fail(c, HBX_ERR_INVALID_ARG, "allocator must be set before any allocation");
    c->alloc_fn = a;
    c->free_fn = f;
    c->alloc_user = user;
    return HBX_OK;
}

void pool_free_all(hbx_pool* p);

extern "C" void hbx_destroy(hbx_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    hbx_server_destroy_all(c);
    for (hbx_pool* p : std::vector<hbx_pool*>(c->pools.begin(), c->pools.end())) hbx_pool_destroy(p);
    for (hbx_graph* g : std::vector<hbx_graph*>(c->graphs.begin(), c->graphs.end())) hbx_graph_destroy(g);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

// ===========================================================================
// graphs
// ===========================================================================
extern "C" int hbx_graph_create(hbx_ctx* ctx, uint32_t n, uint64_t m, const uint32_t* row_ptr, const uint32_t* col,
                                const float* ic_prob, const float* lt_weight, hbx_graph** out) {
    if (!ctx || !out) return HBX_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 2 || n == 0xFFFFFFFFu) return fail(ctx, HBX_ERR_INVALID_ARG, "n must be in [2, 2^32-1)");
    if (m >= (1ull << 32)) return fail(ctx, HBX_ERR_INVALID_ARG, "m must be below 2^32");
    if (!row_ptr || (m && !col)) return fail(ctx, HBX_ERR_INVALID_ARG, "row_ptr/col missing");
    if (!ic_prob && !lt_weight) return fail(ctx, HBX_ERR_INVALID_ARG, "no diffusion parameters");
    if (row_ptr[0] != 0 || row_ptr[n] != m) return fail(ctx, HBX_ERR_INVALID_ARG, "row_ptr must run from 0 to m");
    uint32_t max_deg = 0;
    for (uint32_t v = 0; v < n; v++) {
        if (row_ptr[v + 1] < row_ptr[v]) return fail(ctx, HBX_ERR_INVALID_ARG, "row_ptr decreases");
        max_deg = std::max(max_deg, row_ptr[v + 1] - row_ptr[v]);
    }
    // Edge checks and the IC live thresholds, over the host's cores.  The IC coin
    // a * 2^-24 < p (a = top 24 bits of a Philox word) is the integer compare
    // a < ceil(p * 2^24); p * 2^24 is exact in double.
    std::vector<uint32_t> thr(ic_prob ? m : 0);
    {
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const unsigned T = m < (1u << 20) ? 1u : std::min(hw, 32u);
        std::vector<int> bad(T, 0);  // 1: col out of range, 2: probability outside [0,1]
        auto check = [&](unsigned t) {
            const uint64_t e0 = m * t / T, e1 = m * (t + 1) / T;
            for (uint64_t e = e0; e < e1; e++) {
                if (col[e] >= n) {
                    bad[t] = 1;
                    return;
                }
                if (ic_prob) {
                    const float p = ic_prob[e];
                    if (!(p >= 0.0f && p <= 1.0f)) {
                        bad[t] = 2;
                        return;
                    }
                    thr[e] = (uint32_t)std::ceil((double)p * 16777216.0);
                }
            }
        };
        std::vector<std::thread> pool;
        for (unsigned t = 1; t < T; t++) pool.emplace_back(check, t);
        check(0);
        for (auto& th : pool) th.join();
        for (unsigned t = 0; t < T; t++) {
            if (bad[t] == 1) return fail(ctx, HBX_ERR_INVALID_ARG, "col id out of range");
            if (bad[t] == 2) return fail(ctx, HBX_ERR_INVALID_ARG, "IC probability outside [0,1]");
        }
    }
    std::vector<uint32_t> q;
    if (lt_weight) {
        q.resize(m ? m : 1);
        for (uint32_t v = 0; v < n; v++) {
            uint64_t sum = 0;
            for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) {
                const float w = lt_weight[e];
                if (!(w >= 0.0f && w <= 1.0f)) return fail(ctx, HBX_ERR_INVALID_ARG, "LT weight outside [0,1]");
                const uint64_t fx = (uint64_t)std::floor((double)w * 4294967296.0);
                sum += fx;
                q[e] = (uint32_t)std::min<uint64_t>(fx, 0xFFFFFFFFull);
            }
            if (sum > 4294967296ull)
                return fail(ctx, HBX_ERR_WEIGHTS_GT_1, "LT in-weights of vertex " + std::to_string(v) + " sum above 1");
        }
    }
    cudaSetDevice(ctx->device);
    hbx_graph* g = new hbx_graph();
    g->ctx = ctx;
    g->n = n;
    g->m = (uint32_t)m;
    g->max_indeg = max_deg;
    {
        // content fingerprint (FNV-1a over sizes and 64 sampled CSR entries)
        uint64_t h = 1469598103934665603ull;
        auto mix = [&](uint64_t x) {
            for (int b = 0; b < 8; b++) {
                h ^= (x >> (8 * b)) & 0xFF;
                h *= 1099511628211ull;
            }
        };
        mix(n);
        mix(m);
        for (uint32_t i = 0; i < 64; i++) {
            const uint64_t v = (uint64_t)n * i / 64, e = m ? m * i / 64 : 0;
            mix(row_ptr[v]);
            if (m) mix(col[e]);
            if (m && ic_prob) mix((uint64_t)(ic_prob[e] * 1e9f));
            if (m && lt_weight) mix((uint64_t)(lt_weight[e] * 1e9f));
        }
        g->fingerprint = h;
    }
    auto up = [&](void** dst, const void* src, size_t bytes, size_t alloc_bytes) -> int {
        int r = dalloc(ctx, dst, alloc_bytes);
        if (r) return r;
        if (alloc_bytes > bytes) CK(cudaMemsetAsync((char*)*dst + bytes, 0, alloc_bytes - bytes, ctx->stream));
        if (bytes) CK(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
        return HBX_OK;
    };
    int r = up((void**)&g->row_ptr, row_ptr, ((size_t)n + 1) * 4, ((size_t)n + 1) * 4);
    if (!r) r = up((void**)&g->col, col, m * 4, m * 4 + 16);
    const size_t m4 = ((m + 3) / 4) * 4;
    if (!r && ic_prob) r = up((void**)&g->thr, thr.data(), m * 4, m4 * 4 + 16);
    if (!r && lt_weight) r = up((void**)&g->q, q.data(), m * 4, m * 4 + 16);
    if (!r) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) r = cuda_fail(ctx, e, "graph upload");
    }
    if (r) {
        dfree(ctx, g->row_ptr);
        dfree(ctx, g->col);
        dfree(ctx, g->thr);
        dfree(ctx, g->q);
        delete g;
        return r;
    }
    ctx->graphs.insert(g);
    *out = g;
    return HBX_OK;
}

extern "C" void hbx_graph_destroy(hbx_graph* g) {
    if (!g) return;
    hbx_ctx* c = g->ctx;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (hbx_pool* p : std::vector<hbx_pool*>(c->pools.begin(), c->pools.end()))
        if (p->g == g) hbx_pool_destroy(p);
    dfree(c, g->row_ptr);
    dfree(c, g->col);
    dfree(c, g->thr);
    dfree(c, g->q);
    c->graphs.erase(g);
    delete g;
}

// ===========================================================================
// pools
// ===========================================================================
namespace hbx {

static DevGraph dev_graph(const hbx_graph* g) {
    DevGraph d;
    d.n = g->n;
    d.m = g->m;
    d.row_ptr = g->row_ptr;
    d.col = g->col;
    d.thr = g->thr;
    d.q = g->q;
    return d;
}

static DevCodebook dev_codebook(const hbx_pool* p) {
    DevCodebook c;
    memset(&c, 0, sizeof(c));
    if (!p->has_cb) return c;
    c.rank_of = p->rank_of;
    c.vertex_of_rank = p->vertex_of_rank;
    c.len_of_rank = p->len_of_rank;
    c.code_of_rank = p->code_of_rank;
    c.lut = p->lut;
    c.dec = p->dec;
    c.nsym = p->nsym;
    c.max_len = p->max_len;
    return c;
}

static int pool_bytes_check(hbx_pool* p, size_t add) {
    if (p->o.max_device_bytes && p->device_bytes + add > p->o.max_device_bytes)
        return fail(p->ctx, HBX_ERR_OOM, "pool would exceed max_device_bytes");
    return HBX_OK;
}

// (Re)allocate a zero-filled device array of `bytes`, keeping the first `keep` bytes.
int grow_buffer(hbx_pool* p, void** buf, size_t old_bytes, size_t new_bytes, size_t keep) {
    hbx_ctx* ctx = p->ctx;
    RC(pool_bytes_check(p, new_bytes > old_bytes ? new_bytes - old_bytes : 0));
    void* nb = nullptr;
    RC(dalloc(ctx, &nb, new_bytes));
    CK(cudaMemsetAsync(nb, 0, new_bytes, p->stream));
    if (*buf && keep) CK(cudaMemcpyAsync(nb, *buf, keep, cudaMemcpyDeviceToDevice, p->stream));
    if (*buf) {
        CK(cudaStreamSynchronize(p->stream));
        dfree(ctx, *buf);
    }
    *buf = nb;
    p->device_bytes += new_bytes;
    p->device_bytes -= old_bytes;
    return HBX_OK;
}

static const uint64_t HEAP_SLACK = 64;  // words past the end, for the decoder's look-ahead

static int grow_heap(hbx_pool* p, Heap& h, uint64_t need_words, bool exact = false) {
    if (need_words <= h.cap) return HBX_OK;
    // doubling, or growth by a quarter once the heap passes 8 GB
    const uint64_t step = h.cap * 4 > (8ull << 30) ? h.cap / 4 : h.cap;
    uint64_t nc = exact ? need_words : std::max<uint64_t>(need_words + need_words / 8, h.cap + step);
    nc = std::max<uint64_t>(nc, 1u << 16);
    nc = (nc + 3) & ~3ull;
    RC(grow_buffer(p, (void**)&h.d, h.d ? (h.cap + HEAP_SLACK) * 4 : 0, (nc + HEAP_SLACK) * 4, h.cap * 4));
    h.cap = nc;
    return HBX_OK;
}

static int ensure_recs(hbx_pool* p, uint64_t T) {
    if (T <= p->rec_cap) return HBX_OK;
    uint64_t nc = std::max<uint64_t>(T, p->rec_cap * 2);
    nc = std::max<uint64_t>(nc, 4096);
    void* b = p->recs;
    // new records are KIND_PENDING (all-ones bytes: kind bits 3) until written
    hbx_ctx* ctx = p->ctx;
    RC(pool_bytes_check(p, (nc - p->rec_cap) * sizeof(SetRec)));
    void* nb = nullptr;
    RC(dalloc(ctx, &nb, nc * sizeof(SetRec)));
    CK(cudaMemsetAsync(nb, 0xFF, nc * sizeof(SetRec), p->stream));
    if (b) {
        CK(cudaMemcpyAsync(nb, b, p->rec_cap * sizeof(SetRec), cudaMemcpyDeviceToDevice, p->stream));
        CK(cudaStreamSynchronize(p->stream));
        dfree(ctx, b);
    }
    p->device_bytes += (nc - p->rec_cap) * sizeof(SetRec);
    p->recs = (SetRec*)nb;
    p->rec_cap = nc;
    return HBX_OK;
}

static int ensure_lists(hbx_pool* p, uint64_t count) {
    if (count <= p->list_cap) return HBX_OK;
    uint64_t nc = std::max<uint64_t>(count, p->list_cap * 2);
    RC(grow_buffer(p, (void**)&p->big_list, p->list_cap * 4, nc * 4, 0));
    RC(grow_buffer(p, (void**)&p->retry_list, p->list_cap * 4, nc * 4, 0));
    RC(grow_buffer(p, (void**)&p->list_in, p->list_cap * 4, nc * 4, 0));
    RC(grow_buffer(p, (void**)&p->giant_list, p->list_cap * 4, nc * 4, 0));
    p->list_cap = nc;
    return HBX_OK;
}

static int ensure_block_scratch(hbx_pool* p, uint32_t slots) {
    if (slots <= p->bp_slots) return HBX_OK;
    const uint64_t words = p->bp_words;
    const uint64_t n = p->g->n;
    RC(grow_buffer(p, (void**)&p->bp_visited, p->bp_slots * words * 4, slots * words * 4, 0));
    RC(grow_buffer(p, (void**)&p->bp_rbits, p->bp_slots * words * 4, slots * words * 4, 0));
    RC(grow_buffer(p, (void**)&p->bp_aux, p->bp_slots * words * 4, slots * words * 4, 0));
    RC(grow_buffer(p, (void**)&p->bp_queue, p->bp_slots * n * 4, slots * n * 4, 0));
    p->bp_slots = slots;
    return HBX_OK;
}

static int read_counters(hbx_pool* p) {
    hbx_ctx* ctx = p->ctx;
    CK(cudaMemcpyAsync(&p->hc, p->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    if (p->hc.error) return fail(ctx, HBX_ERR_INTERNAL, "kernel error code " + std::to_string(p->hc.error));
    return HBX_OK;
}

// zero the per-launch fields of the device counters
static int reset_launch_counters(hbx_pool* p) {
    hbx_ctx* ctx = p->ctx;
    CK(cudaMemsetAsync(p->ctr, 0, 2 * sizeof(unsigned long long), p->stream));  // work, big_work
    CK(cudaMemsetAsync(&p->ctr->big_count, 0, 2 * sizeof(unsigned long long), p->stream));
    CK(cudaMemsetAsync(&p->ctr->mid_work, 0, 2 * sizeof(unsigned long long), p->stream));  // + giant_count
    CK(cudaMemsetAsync(&p->ctr->raw_fail, 0xFF, 3 * sizeof(unsigned long long), p->stream));
    return HBX_OK;
}

static SampleArgs sample_args(hbx_pool* p, uint32_t mode, uint32_t j0, uint32_t count, const uint32_t* list,
                              uint32_t* freq, uint32_t cut, const Shape& sh) {
    SampleArgs a;
    memset(&a, 0, sizeof(a));
    a.g = dev_graph(p->g);
    a.key0 = (uint32_t)p->seed;
    a.key1 = (uint32_t)(p->seed >> 32);
    a.rk = philox_round_keys(a.key0, a.key1);
    a.epoch = p->o.pool_epoch;
    a.model = (uint32_t)p->model;
    a.mode = mode;
    a.cut = cut;
    a.j0 = j0;
    a.count = count;
    a.list = list;
    a.persistent = p->o.form ? 1u : 0u;
    a.group_budget = sh.gb;
    a.freq = freq;
    a.recs = p->recs;
    a.raw_heap = p->raw.d;
    a.raw_cap = p->raw.cap;
    a.code_heap = p->code.d;
    a.code_cap = p->code.cap;
    a.bm_heap = p->bm.d;
    a.bm_cap = p->bm.cap;
    a.cb = dev_codebook(p);
    a.big_list = p->big_list;
    a.retry_list = p->retry_list;
    a.giant_list = p->giant_list;
    a.ctr = p->ctr;
    a.bp_visited = p->bp_visited;
    a.bp_rbits = p->bp_rbits;
    a.bp_queue = p->bp_queue;
    a.bp_aux = p->bp_aux;
    a.bp_words = p->bp_words;
    a.sizes = p->wsizes;
    a.sizes_cap = p->wsizes_cap;
    return a;
}

// Time one sampler launch (unless it is a histogram pass) and read the counters.
template <class F>
static int timed_launch(hbx_pool* p, bool timed, F&& launch) {
    hbx_ctx* ctx = p->ctx;
    if (timed) CK(cudaEventRecord(p->ev0, p->stream));
    CK(launch());
    if (timed) CK(cudaEventRecord(p->ev1, p->stream));
    p->launches++;
    RC(read_counters(p));
    if (timed) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
        p->sample_kernel_s += ms * 1e-3;
        p->sample_kernel_launches++;
    }
    return HBX_OK;
}

// Run the block kernel over `nitems` sets: the giant list, or with a.direct the
// batch itself.  Each resident cluster holds one scratch slot (an n-bit visited
// bitmap and an n-entry queue in HBM); the slots take at most 32 GB, or an
// eighth of the pool's device-memory limit.
static int run_block_path(hbx_pool* p, SampleArgs a, uint32_t nitems, uint32_t csize, bool timed) {
    const uint64_t slot_bytes = p->bp_words * 12 + (uint64_t)p->g->n * 4;
    uint64_t budget = 32ull << 30;
    if (p->o.max_device_bytes) budget = std::min<uint64_t>(budget, p->o.max_device_bytes / 8);
    const uint64_t mem_slots = std::max<uint64_t>(1, budget / slot_bytes);
    uint32_t slots = std::min<uint32_t>(nitems, (uint32_t)block_path_max_clusters(csize));
    slots = (uint32_t)std::min<uint64_t>(slots, std::max<uint64_t>(mem_slots, p->bp_slots));
    RC(ensure_block_scratch(p, slots));
    a.bp_visited = p->bp_visited;
    a.bp_rbits = p->bp_rbits;
    a.bp_queue = p->bp_queue;
    a.bp_aux = p->bp_aux;
    return timed_launch(p, timed, [&] { return launch_sample_block(a, nitems, slots, csize, p->stream); });
}

static int ensure_ms_scratch(hbx_pool* p) {
    if (p->ms_vis) return HBX_OK;
    const uint64_t n4 = (((uint64_t)p->g->n + 3) & ~3ull) * 4;  // 16-byte padded mask arrays
    RC(grow_buffer(p, (void**)&p->ms_vis, 0, n4, 0));
    RC(grow_buffer(p, (void**)&p->ms_nxt, 0, n4, 0));
    RC(grow_buffer(p, (void**)&p->ms_F, 0, n4, 0));
    RC(grow_buffer(p, (void**)&p->ms_N, 0, n4, 0));
    RC(grow_buffer(p, (void**)&p->ms_pend, 0, n4, 0));
    RC(grow_buffer(p, (void**)&p->ms_ndef, 0, n4 / 4, 0));  // zero: nothing deferred
    // a heavy vertex has more than 32 edge groups, so at most m/128 of them,
    // each cut into chunks of 256 groups
    const uint64_t m = p->g->m;
    p->ms_heavy_cap = (uint32_t)std::min<uint64_t>(m / 128 + m / 1024 + 1024, 0xFFFFFFFFull);
    RC(grow_buffer(p, (void**)&p->ms_heavy, 0, (size_t)p->ms_heavy_cap * sizeof(uint4), 0));
    RC(grow_buffer(p, (void**)&p->ms_c, 0, sizeof(MsCounters), 0));
    RC(grow_buffer(p, (void**)&p->ms_sets, 0, MS_SETS * 4, 0));
    RC(grow_buffer(p, (void**)&p->ms_rowoff, 0, MS_SETS * 8, 0));
    RC(grow_buffer(p, (void**)&p->ms_sparse, 0, 2 * MS_SETS * 4, 0));
    return HBX_OK;
}

static MsArgs ms_args(hbx_pool* p) {
    MsArgs a;
    memset(&a, 0, sizeof(a));
    a.g = dev_graph(p->g);
    a.col4 = p->g->col;  // allocated with 16 zero bytes past m entries
    a.key0 = (uint32_t)p->seed;
    a.key1 = (uint32_t)(p->seed >> 32);
    a.rk = philox_round_keys(a.key0, a.key1);
    a.epoch = p->o.pool_epoch;
    a.sets = p->ms_sets;
    a.vis = p->ms_vis;
    a.nxt = p->ms_nxt;
    a.F = p->ms_F;
    a.Ff = p->ms_N;
    a.pend = p->ms_pend;
    a.ndef = p->ms_ndef;
    a.defer_groups = MS_DEFER_GROUPS;
    a.defer_max = MS_DEFER_MAX;
    a.heavy = p->ms_heavy;
    a.heavy_cap = p->ms_heavy_cap;
    a.mc = p->ms_c;
    a.ctr = p->ctr;
    a.recs = p->recs;
    a.rowoff = p->ms_rowoff;
    a.sizes = p->wsizes;
    a.sizes_cap = p->wsizes_cap;
    return a;
}

// The level loop's CUDA graphs (every argument is a fixed pool buffer; the
// batch's set ids and count are read from device memory).
static int ensure_ms_graphs(hbx_pool* p, const MsArgs& a) {
    if (p->ms_first) return HBX_OK;
    hbx_ctx* ctx = p->ctx;
    for (int which = 0; which < 2; which++) {
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t le = which == 0 ? launch_ms_start(a, ctx->sms, p->stream) : cudaSuccess;
        for (int l = 0; l < MS_GRAPH_LEVELS && le == cudaSuccess; l++) le = launch_ms_level(a, ctx->sms, p->stream);
        const cudaError_t ce = cudaStreamEndCapture(p->stream, &graph);
        if (le != cudaSuccess) return cuda_fail(ctx, le, "level graph capture");
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaStreamEndCapture");
        cudaGraphExec_t exec;
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return cuda_fail(ctx, ie, "cudaGraphInstantiate");
        (which == 0 ? p->ms_first : p->ms_more) = exec;
    }
    return HBX_OK;
}

// One batch of the bit-parallel search: the listed sets (NONE = an unused
// slot) searched to the end; their sizes and edge counts come back in *mc.
// With `timed`, an event pair opens around the batch (closed by the caller).
static int ms_search_batch(hbx_pool* p, const uint32_t* ids, uint32_t nb, bool timed, MsCounters* mc) {
    hbx_ctx* ctx = p->ctx;
    const uint32_t n = p->g->n;
    CK(cudaMemcpyAsync(p->ms_sets, ids, (size_t)nb * 4, cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemsetAsync(p->ms_c, 0, sizeof(MsCounters), p->stream));
    CK(cudaMemcpyAsync(&p->ms_c->nsets, &nb, 4, cudaMemcpyHostToDevice, p->stream));
    const MsArgs a = ms_args(p);
    RC(ensure_ms_graphs(p, a));
    if (timed) CK(cudaEventRecord(p->ev0, p->stream));
    // the levels run from CUDA graphs of MS_GRAPH_LEVELS levels each, the
    // first one preceded by the roots; the host looks at the frontier after
    // each graph
    for (uint64_t level = 0;; level += MS_GRAPH_LEVELS) {
        if (level > (uint64_t)n) return fail(ctx, HBX_ERR_INTERNAL, "bit-parallel search did not end");
        CK(cudaGraphLaunch(level ? p->ms_more : p->ms_first, p->stream));
        p->launches += (level ? 0 : 3) + 4 * MS_GRAPH_LEVELS;
        // the first six words: frontier sizes, set count, deferred vertices, force
        uint32_t head[6] = {0};
        CK(cudaMemcpyAsync(head, p->ms_c, sizeof(head), cudaMemcpyDeviceToHost, p->stream));
        CK(cudaStreamSynchronize(p->stream));
        if (head[0] == 0 && head[5] == 0) break;  // empty frontier, nothing deferred
    }
    CK(launch_ms_finish(a, ctx->sms, p->stream));
    p->launches++;
    CK(cudaMemcpyAsync(mc, p->ms_c, sizeof(*mc), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    if (timed) {
        p->ms_nsets += nb;
        p->ms_blocks += mc->blocks;
        p->ms_visits += mc->visits;
        p->ms_deferred += mc->deferred;
    }
    return HBX_OK;
}

// Sample the listed IC sets (ids on the host) MS_SETS at a time with the
// bit-parallel search.  Dense sets are stored as bitmap rows (MODE_ENCODE) or
// counted (MODE_HIST); each of the others is encoded (or histogrammed) by one
// block from its membership row, as the per-set block kernel would.
static int run_multi_source(hbx_pool* p, uint32_t mode, uint32_t cut, const std::vector<uint32_t>& ids,
                            uint32_t* freq, const Shape& sh, bool timed) {
    hbx_ctx* ctx = p->ctx;
    RC(ensure_ms_scratch(p));
    const uint64_t row = p->bp_words;
    const uint32_t n = p->g->n;
    for (size_t b0 = 0; b0 < ids.size(); b0 += MS_SETS) {
        const uint32_t nb = (uint32_t)std::min<size_t>(MS_SETS, ids.size() - b0);
        MsCounters mc;
        RC(ms_search_batch(p, ids.data() + b0, nb, timed, &mc));
        const MsArgs a = ms_args(p);
        uint32_t dense = 0, nd = 0, nsp = 0;
        unsigned long long rowoff[MS_SETS] = {0};
        uint32_t sparse[2 * MS_SETS];  // mask bits, then set ids, of the sets under the cut
        for (uint32_t s = 0; s < nb; s++) {
            if ((unsigned long long)cut * mc.size[s] > n) {
                dense |= 1u << s;
                rowoff[s] = p->hc.bm_cursor + (unsigned long long)nd * row;
                nd++;
            } else {
                sparse[nsp] = s;
                sparse[MS_SETS + nsp] = ids[b0 + s];
                nsp++;
            }
        }
        if (nsp) {
            RC(ensure_block_scratch(p, nsp));
            CK(cudaMemcpyAsync(p->ms_sparse, sparse, sizeof(sparse), cudaMemcpyHostToDevice, p->stream));
            const SampleArgs sa = sample_args(p, mode, 0, 0, nullptr, freq, cut, sh);
            CK(launch_ms_sparse(sa, p->ms_vis, p->ms_sparse, p->ms_sparse + MS_SETS, p->ms_c, nsp, p->stream));
            p->launches++;
        }
        if (mode == MODE_ENCODE && nd) {
            // the rows are placed by the host: no set of the batch can overflow
            const unsigned long long cursor = p->hc.bm_cursor + (unsigned long long)nd * row;
            RC(grow_heap(p, p->bm, cursor));
            CK(cudaMemcpyAsync(p->ms_rowoff, rowoff, sizeof(rowoff), cudaMemcpyHostToDevice, p->stream));
            CK(cudaMemcpyAsync(&p->ctr->bm_cursor, &cursor, 8, cudaMemcpyHostToDevice, p->stream));
            p->hc.bm_cursor = cursor;
        }
        CK(launch_ms_emit(a, dense, mode, row, p->bm.d, ctx->sms, p->stream));
        p->launches += 2;
        if (timed) {
            CK(cudaEventRecord(p->ev1, p->stream));
            CK(cudaEventSynchronize(p->ev1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
            p->sample_kernel_s += ms * 1e-3;
            p->ms_kernel_s += ms * 1e-3;
            p->sample_kernel_launches++;
        }
    }
    return read_counters(p);
}

// Sample sets (range [j0, j0+count) or list) in `mode`, handling sets too large
// for a warp and heaps that run out.  The list, if any, is a device array.
// The batched form runs the persistent warp kernel, then the shared-memory
// block kernel on the sets that outgrew a warp, then the HBM-scratch block
// kernel on those that outgrew shared memory.  The plain form runs every set
// of the batch through the HBM-scratch block kernel, one block per set.
static int run_sample(hbx_pool* p, uint32_t mode, uint32_t j0, uint32_t count, const uint32_t* list,
                      uint32_t* freq, uint32_t cut, const Shape& sh) {
    hbx_ctx* ctx = p->ctx;
    for (int attempt = 0; count > 0; attempt++) {
        if (attempt > 40) return fail(ctx, HBX_ERR_INTERNAL, "sampling retries did not converge");
        RC(ensure_lists(p, count));
        RC(reset_launch_counters(p));
        const bool timed = mode != MODE_HIST;
        SampleArgs a = sample_args(p, mode, j0, count, list, freq, cut, sh);
        if (!a.persistent) {
            a.direct = 1;
            RC(run_block_path(p, a, count, 1u, timed));
        } else {
            RC(timed_launch(p, timed, [&] { return launch_sample_warp(a, sh.qw, ctx->sms, p->stream); }));
            uint32_t nmid = (uint32_t)p->hc.big_count;
            if (nmid && sh.q2) {
                // the sets that outgrew the warp go through warps of capacity q2
                // first (many more of them in flight than shared-memory blocks;
                // thin deep sets gain most), then on to the block tiers
                CK(cudaMemcpyAsync(p->list_in, p->big_list, (size_t)nmid * 4, cudaMemcpyDeviceToDevice, p->stream));
                CK(cudaMemsetAsync(p->ctr, 0, sizeof(unsigned long long), p->stream));  // work
                CK(cudaMemsetAsync(&p->ctr->big_count, 0, sizeof(unsigned long long), p->stream));
                SampleArgs a2 = sample_args(p, mode, 0, nmid, p->list_in, freq, cut, sh);
                a2.group_budget = 0xFFFFFFFFu;
                RC(timed_launch(p, timed, [&] { return launch_sample_warp(a2, sh.q2, ctx->sms, p->stream); }));
                nmid = (uint32_t)p->hc.big_count;
            }
            if (nmid) RC(timed_launch(p, timed, [&] { return launch_sample_mid(a, nmid, ctx->sms, p->stream); }));
            uint32_t nbig = (uint32_t)p->hc.giant_count;
            if (nbig && p->model == HBX_IC && mode != MODE_RAW) {
                // IC sets that outgrew shared memory: bit-parallel search, 32 at a time
                std::vector<uint32_t> ids(nbig);
                CK(cudaMemcpyAsync(ids.data(), p->giant_list, (size_t)nbig * 4, cudaMemcpyDeviceToHost, p->stream));
                CK(cudaStreamSynchronize(p->stream));
                RC(run_multi_source(p, mode, cut, ids, freq, sh, timed));
                nbig = 0;
            }
            if (nbig) {
                SampleArgs b = sample_args(p, mode, j0, count, list, freq, cut, sh);  // heaps may have moved
                b.big_list = p->giant_list;
                RC(run_block_path(p, b, nbig, sh.bc ? sh.bc : 1u, timed));
            }
        }
        const uint32_t nretry = (uint32_t)p->hc.retry_count;
        if (nretry == 0) break;
        // Every allocation that fitted a heap lies below the lowest failed
        // offset, and every one at or past it failed: the listed sets need
        // exactly the words past it.  Roll each cursor back there, grow the
        // heaps to the old cursor, and redo the listed sets.
        const unsigned long long fails[3] = {p->hc.raw_fail, p->hc.code_fail, p->hc.bm_fail};
        unsigned long long rolled[3] = {p->hc.raw_cursor, p->hc.code_cursor, p->hc.bm_cursor};
        for (int h = 0; h < 3; h++)
            if (fails[h] != ~0ull) rolled[h] = fails[h];
        CK(cudaMemcpyAsync(&p->ctr->raw_cursor, rolled, sizeof(rolled), cudaMemcpyHostToDevice, p->stream));
        RC(grow_heap(p, p->raw, p->hc.raw_cursor + 1024));
        RC(grow_heap(p, p->code, p->hc.code_cursor + 1024));
        const uint64_t row = (((uint64_t)p->g->n + 31) / 32 + 3) & ~3ull;
        RC(grow_heap(p, p->bm, p->hc.bm_cursor + (p->hc.bm_cursor > p->bm.cap ? 8 * row : 0)));
        CK(cudaMemcpyAsync(p->list_in, p->retry_list, (size_t)nretry * 4, cudaMemcpyDeviceToDevice, p->stream));
        list = p->list_in;
        count = nretry;
        j0 = 0;
    }
    return HBX_OK;
}

// ---------------------------------------------------------------------------
// Codebook (Section 4.2.2): Huffman code lengths from the warm-up frequencies,
// then canonical codes.  Rules (the paper names BuildHuffmanCode only):
// symbols = vertices with f > 0 taken in (f, id) order; each merge takes the
// two lightest queue fronts, preferring a leaf over an internal node of equal
// weight; a lone symbol gets length 1; lengths over 32 trigger f = ceil(f/2)
// (at least 1) and a rebuild.  Canonical codes: ranks in (length, id) order,
// code(first of length L) = (code(first of L-1) + count(L-1)) << 1.
// ---------------------------------------------------------------------------
static void huffman_code_lengths(const std::vector<uint32_t>& sym, std::vector<uint64_t> w,
                                 std::vector<uint8_t>& len_out) {
    const size_t S = sym.size();
    len_out.assign(S, 0);
    if (S == 0) return;
    if (S == 1) {
        len_out[0] = 1;
        return;
    }
    for (;;) {
        // order leaves by (weight, id): ids are increasing in `sym`, so a stable
        // bucket pass on weight keeps id order among equal weights
        std::vector<uint32_t> leaf(S);
        {
            std::vector<std::pair<uint64_t, uint32_t>> kv(S);
            for (size_t i = 0; i < S; i++) kv[i] = {w[i], (uint32_t)i};
            std::stable_sort(kv.begin(), kv.end(),
                             [](const std::pair<uint64_t, uint32_t>& x, const std::pair<uint64_t, uint32_t>& y) {
                                 return x.first < y.first;
                             });
            for (size_t i = 0; i < S; i++) leaf[i] = kv[i].second;
        }
        // node ids: leaves 0..S-1, internal S..2S-2
        std::vector<uint64_t> nw(2 * S - 1);
        std::vector<uint32_t> up(2 * S - 1, 0);
        for (size_t i = 0; i < S; i++) nw[i] = w[i];
        size_t li = 0, qi = S, qe = S;
        auto pick = [&]() -> uint32_t {
            if (li < S && (qi == qe || nw[leaf[li]] <= nw[qi])) return leaf[li++];
            return (uint32_t)qi++;
        };
        while (qe < 2 * S - 1) {
            const uint32_t x = pick(), y = pick();
            nw[qe] = nw[x] + nw[y];
            up[x] = up[y] = (uint32_t)qe;
            qe++;
        }
        std::vector<uint32_t> depth(2 * S - 1, 0);
        uint32_t maxd = 0;
        for (size_t v = 2 * S - 1; v-- > 0;) {
            if (v == 2 * S - 2) continue;
            depth[v] = depth[up[v]] + 1;
            if (v < S) maxd = std::max(maxd, depth[v]);
        }
        if (maxd <= 32) {
            for (size_t i = 0; i < S; i++) len_out[i] = (uint8_t)depth[i];
            return;
        }
        for (auto& x : w) x = std::max<uint64_t>(1, (x + 1) / 2);
    }
}

static int build_codebook(hbx_pool* p, const std::vector<uint32_t>& freq) {
    hbx_ctx* ctx = p->ctx;
    const uint32_t n = p->g->n;
    std::vector<uint32_t> sym;
    std::vector<uint64_t> w;
    for (uint32_t v = 0; v < n; v++)
        if (freq[v]) {
            sym.push_back(v);
            w.push_back(freq[v]);
        }
    std::vector<uint8_t> L;
    huffman_code_lengths(sym, w, L);
    uint32_t bl_count[34] = {0};
    for (uint8_t x : L) bl_count[x]++;
    bl_count[0] = 0;
    // first code and first rank of each length (RFC 1951 Section 3.2.2 recurrence)
    uint32_t first_code[33] = {0}, first_rank[33] = {0};
    for (int b = 2; b <= 32; b++) {
        first_code[b] = (first_code[b - 1] + bl_count[b - 1]) << 1;
        first_rank[b] = first_rank[b - 1] + bl_count[b - 1];
    }
    const uint32_t S = (uint32_t)sym.size();
    std::vector<uint32_t> rank_of(n, NONE), vor(std::max<uint32_t>(S, 1)), cor(std::max<uint32_t>(S, 1));
    std::vector<uint8_t> lor(std::max<uint32_t>(S, 1));
    std::vector<uint32_t> next_rank(first_rank, first_rank + 33);
    p->h_len.assign(n, 0);
    p->h_code.assign(n, 0);
    uint32_t maxL = 0;
    for (uint32_t i = 0; i < S; i++) {  // ids ascending
        const uint32_t l = L[i];
        const uint32_t r = next_rank[l]++;
        const uint32_t c = first_code[l] + (r - first_rank[l]);
        rank_of[sym[i]] = r;
        vor[r] = sym[i];
        cor[r] = c;
        lor[r] = (uint8_t)l;
        p->h_len[sym[i]] = l;
        p->h_code[sym[i]] = c;
        maxL = std::max(maxL, l);
    }
    std::vector<uint32_t> lut(1u << LUT_BITS, 0);
    for (uint32_t r = 0; r < S; r++) {
        const uint32_t l = lor[r];
        if (l > (uint32_t)LUT_BITS) continue;
        const uint32_t lo = cor[r] << (LUT_BITS - l), hi = (cor[r] + 1) << (LUT_BITS - l);
        for (uint32_t x = lo; x < hi; x++) lut[x] = (r << 6) | l;
    }
    std::vector<uint32_t> dec(99, 0);
    for (int b = 0; b <= 32; b++) {
        dec[b] = first_code[b];
        dec[33 + b] = b ? bl_count[b] : 0;
        dec[66 + b] = first_rank[b];
    }
    p->h_rank = rank_of;
    p->h_freq = freq;
    p->nsym = S;
    p->max_len = maxL;
    auto up = [&](void** dst, const void* src, size_t bytes) -> int {
        RC(grow_buffer(p, dst, 0, bytes + 16, 0));
        CK(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, p->stream));
        return HBX_OK;
    };
    RC(up((void**)&p->rank_of, rank_of.data(), (size_t)n * 4));
    RC(up((void**)&p->vertex_of_rank, vor.data(), vor.size() * 4));
    RC(up((void**)&p->code_of_rank, cor.data(), cor.size() * 4));
    RC(up((void**)&p->len_of_rank, lor.data(), lor.size()));
    RC(up((void**)&p->lut, lut.data(), lut.size() * 4));
    RC(up((void**)&p->dec, dec.data(), dec.size() * 4));
    CK(cudaStreamSynchronize(p->stream));
    p->has_cb = true;
    return HBX_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: pick the launch shape of the sampler -- the warp capacity QW (the
// set size above which a set moves from a warp to a whole block) and the
// warp's edge-group budget (the scan work above which it does the same) -- by
// timing a calibration batch per graph and model; cached in the context.
// ---------------------------------------------------------------------------
static int choose_shape(hbx_pool* p, Shape* out) {
    hbx_ctx* ctx = p->ctx;
    if (!p->o.form) {  // the plain form runs the block kernel only
        *out = {256, 2048, 1, 0};
        return HBX_OK;
    }
    if (p->o.warp_capacity) {
        out->qw = p->o.warp_capacity;
        out->gb = p->o.warp_group_budget ? p->o.warp_group_budget : 2048u;
        out->bc = p->o.block_cluster ? p->o.block_cluster : 1u;
        out->q2 = 0;
        return HBX_OK;
    }
    auto key = std::make_pair(p->g->fingerprint, (int)p->model);
    {
        std::lock_guard<std::mutex> lock(ctx->mu);
        auto it = ctx->tuned.find(key);
        if (it != ctx->tuned.end()) {
            *out = it->second;
            return HBX_OK;
        }
    }
    // (warp capacity, warp group budget, cluster size, second warp tier)
    const Shape cands[] = {{64, 0, 1, 0},       {128, 256, 1, 0},    {128, 1024, 1, 0},  {256, 4096, 1, 0},
                           {128, 1024, 2, 0},   {256, 1024, 2, 0},   {256, 4096, 4, 0},  {512, 4096, 1, 0},
                           {128, 1024, 1, 1024}, {128, 256, 1, 2048}, {256, 4096, 1, 1024}};
    uint32_t* freq = nullptr;
    RC(grow_buffer(p, (void**)&freq, 0, (size_t)p->g->n * 4, 0));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    Shape best = {256, 2048, 1, 0};
    const uint32_t base = 0x40000000u;  // calibration ids, never part of a pool prefix
    const unsigned long long sc0 = p->hc.edges_scanned, lv0 = p->hc.edges_live;
    // Calibration batch: 8192 sets timed twice per shape, or, where a probe of
    // 256 sets shows heavy sets, as many as scan about 2^31 edges, timed once.
    uint32_t ncal = 8192;
    int reps = 2;
    {
        const uint32_t nprobe = 256;
        int r = run_sample(p, MODE_HIST, base + 0x20000000u, nprobe, nullptr, freq, 0u, cands[0]);
        if (r) {
            dfree(ctx, freq);
            return r;
        }
        const double per_set = (double)(p->hc.edges_scanned - sc0) / nprobe;
        const double budget = 2147483648.0;
        if (per_set * ncal > budget) {
            ncal = std::max<uint32_t>(64, (uint32_t)(budget / per_set) & ~63u);
            reps = 1;
        }
    }
    for (int rep = 2 - reps; rep < 2; rep++) {
        for (const Shape& sh : cands) {
            CK(cudaEventRecord(e0, p->stream));
            int r = run_sample(p, MODE_HIST, base, ncal, nullptr, freq, 0u, sh);
            if (r) {
                dfree(ctx, freq);
                return r;
            }
            CK(cudaEventRecord(e1, p->stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (rep == 1 && ms < best_ms) {
                best_ms = ms;
                best = sh;
            }
        }
    }
    p->aux_scanned += p->hc.edges_scanned - sc0;
    p->aux_live += p->hc.edges_live - lv0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(ctx, freq);
    p->device_bytes -= (size_t)p->g->n * 4;
    {
        std::lock_guard<std::mutex> lock(ctx->mu);
        ctx->tuned[key] = best;
    }
    *out = best;
    return HBX_OK;
}

// Characterize (Algorithm 1, first block): the skewness S of the warm-up sets'
// sizes (Eq. (2), population standard deviation, the sizes summed in set
// order) picks Bitmax (every set a bitmap: cut n + 1) when S < 0, else Huffmax
// (every set coded: cut 0).  A Bitmax IC pool keeps its sets as vertex-major
// tiles of 32 sets.
static int characterize(hbx_pool* p) {
    hbx_ctx* ctx = p->ctx;
    const uint64_t W = p->wsizes_cap;
    std::vector<uint32_t> sz(W);
    CK(cudaMemcpyAsync(sz.data(), p->wsizes, W * 4, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    double sum = 0.0;
    for (uint64_t i = 0; i < W; i++) sum += (double)sz[i];
    const double mean = sum / (double)W;
    double m2 = 0.0, m3 = 0.0;
    for (uint64_t i = 0; i < W; i++) {
        const double d = (double)sz[i] - mean;
        m2 += d * d;
        m3 += d * d * d;
    }
    m2 /= (double)W;
    m3 /= (double)W;
    p->scheme_skew = m2 > 0.0 ? m3 / (m2 * std::sqrt(m2)) : 0.0;
    p->bitmax = p->scheme_skew < 0.0;
    const uint32_t n = p->g->n;
    if (p->bitmax) {
        p->cut = n + 1;
        p->tiles = p->model == HBX_IC && p->o.form == 1;
        p->hist_dense = W;
        p->hist_verts = 0;
    } else {
        p->cut = 0;
        p->hist_dense = 0;
        p->hist_verts = (uint64_t)sum;
    }
    return HBX_OK;
}

static int ensure_codebook(hbx_pool* p) {
    hbx_ctx* ctx = p->ctx;
    if (!p->o.encode || p->has_cb) return HBX_OK;
    if (p->W == 0) return fail(ctx, HBX_ERR_INVALID_ARG, "encoded pool needs warmup_sets > 0");
    if (p->W >= (1ull << 32)) return fail(ctx, HBX_ERR_INVALID_ARG, "warm-up block too large");
    uint32_t* freq = nullptr;
    const uint32_t n = p->g->n;
    RC(grow_buffer(p, (void**)&freq, 0, (size_t)n * 4, 0));
    const unsigned long long sc0 = p->hc.edges_scanned, lv0 = p->hc.edges_live;
    const unsigned long long hd0 = p->hc.hist_dense, hv0 = p->hc.hist_verts;
    // the per-graph scheme (Algorithm 1) counts every warm-up set (Huffmax
    // codes all of them) and records the sizes for Characterize
    if (p->o.scheme) {
        p->cut = 0;
        RC(grow_buffer(p, (void**)&p->wsizes, 0, (size_t)p->W * 4, 0));
        p->wsizes_cap = (uint32_t)p->W;
    }
    int r = run_sample(p, MODE_HIST, 0, (uint32_t)p->W, nullptr, freq, p->cut, p->shape);
    p->aux_scanned += p->hc.edges_scanned - sc0;
    p->aux_live += p->hc.edges_live - lv0;
    p->hist_sets = p->W;
    p->hist_dense = p->hc.hist_dense - hd0;
    p->hist_verts = p->hc.hist_verts - hv0;
    std::vector<uint32_t> hf(n);
    if (!r) {
        cudaError_t e = cudaMemcpyAsync(hf.data(), freq, (size_t)n * 4, cudaMemcpyDeviceToHost, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) r = cuda_fail(ctx, e, "warm-up histogram");
    }
    dfree(ctx, freq);
    p->device_bytes -= (size_t)n * 4;
    if (!r && p->o.scheme) r = characterize(p);
    if (p->wsizes) {
        dfree(ctx, p->wsizes);
        p->device_bytes -= (size_t)p->wsizes_cap * 4;
        p->wsizes = nullptr;
        p->wsizes_cap = 0;
    }
    if (r) return r;
    return build_codebook(p, hf);
}

// Grow the heaps ahead of a batch of `count` sets by projecting each heap's
// words per set from the sets stored so far or, before the first batch of an
// encoded pool, from the warm-up pass (sizes of the same first sets, with the
// frequency-weighted mean code length).  Heavy sets then seldom overflow a
// heap, which would make them be sampled twice.
static int reserve_heaps(hbx_pool* p, uint64_t count) {
    const uint64_t row = (((uint64_t)p->g->n + 31) / 32 + 3) & ~3ull;
    double per[3] = {0, 0, 0}, dense = 0;  // raw, code, bitmap words per set; dense fraction
    if (p->T) {
        per[0] = (double)p->hc.raw_cursor / (double)p->T;
        per[1] = (double)p->hc.code_cursor / (double)p->T;
        dense = (double)p->hc.sets_bm / (double)p->T;
    } else if (p->hist_sets && p->has_cb) {
        double fl = 0, f = 0;
        for (uint32_t v = 0; v < p->g->n; v++) {
            fl += (double)p->h_freq[v] * p->h_len[v];
            f += (double)p->h_freq[v];
        }
        const double bits = f > 0 ? fl / f : 32.0;
        per[1] = (double)p->hist_verts / (double)p->hist_sets * (bits + 2.0) / 32.0 + 2.0;
        dense = (double)p->hist_dense / (double)p->hist_sets;
    } else {
        return HBX_OK;
    }
    // the dense count of a batch varies like a binomial: three deviations of room
    const double c = (double)count;
    const double nd = c * dense + 3.0 * std::sqrt(c * dense * (1.0 - dense)) + 1.0;
    RC(grow_heap(p, p->raw, p->hc.raw_cursor + (uint64_t)(per[0] * c * 1.1) + 1024, true));
    RC(grow_heap(p, p->code, p->hc.code_cursor + (uint64_t)(per[1] * c * 1.1) + 1024, true));
    if (dense > 0) RC(grow_heap(p, p->bm, p->hc.bm_cursor + (uint64_t)nd * row, true));
    return HBX_OK;
}

// Sets [j0, j0 + count) of a Bitmax IC pool, as the vertex-major bit matrix
// of Section 4.2.3 / Eq. (3): tile t (at word t * n4 of the bitmap heap, n4 =
// n rounded up to 4) holds sets [32t, 32t + 32), word v bit s for set 32t + s.
// Every set is found by the bit-parallel search, one tile's sets per batch, so
// the search's visited masks are the tile's words.
static int run_tiles(hbx_pool* p, uint32_t j0, uint32_t count) {
    hbx_ctx* ctx = p->ctx;
    RC(ensure_ms_scratch(p));
    const uint64_t n4 = ((uint64_t)p->g->n + 3) & ~3ull;
    const uint64_t jend = (uint64_t)j0 + count;
    for (uint64_t j = j0; j < jend;) {
        const uint64_t t = j / 32;
        const uint32_t s0 = (uint32_t)(j % 32), s1 = (uint32_t)std::min<uint64_t>(32, s0 + (jend - j));
        uint32_t ids[MS_SETS];
        uint32_t slots = 0;
        for (uint32_t s = 0; s < MS_SETS; s++) {
            const bool on = s >= s0 && s < s1;
            ids[s] = on ? (uint32_t)(32 * t + s) : NONE;
            if (on) slots |= 1u << s;
        }
        MsCounters mc;
        RC(ms_search_batch(p, ids, MS_SETS, true, &mc));
        const uint64_t off = t * n4;
        const bool fresh = off + n4 > p->hc.bm_cursor;  // the tile's first batch
        if (fresh) {
            RC(grow_heap(p, p->bm, off + n4));
            const unsigned long long cursor = off + n4;
            CK(cudaMemcpyAsync(&p->ctr->bm_cursor, &cursor, 8, cudaMemcpyHostToDevice, p->stream));
            p->hc.bm_cursor = cursor;
        }
        const MsArgs a = ms_args(p);
        CK(launch_ms_tile(a, slots, p->bm.d, off, fresh ? n4 : 0, ctx->sms, p->stream));
        p->launches += 2;
        CK(cudaEventRecord(p->ev1, p->stream));
        CK(cudaEventSynchronize(p->ev1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
        p->sample_kernel_s += ms * 1e-3;
        p->ms_kernel_s += ms * 1e-3;
        p->sample_kernel_launches++;
        j += s1 - s0;
    }
    return read_counters(p);
}

int pool_extend(hbx_pool* p, uint64_t T) {
    hbx_ctx* ctx = p->ctx;
    if (T <= p->T) return HBX_OK;
    if (T >= (1ull << 32)) return fail(ctx, HBX_ERR_INVALID_ARG, "pools hold fewer than 2^32 sets");
    cudaSetDevice(ctx->device);
    const double t0 = now_s();
    if (!p->shape.qw) RC(choose_shape(p, &p->shape));
    RC(ensure_codebook(p));
    RC(ensure_recs(p, T));
    const uint32_t mode = p->o.encode ? MODE_ENCODE : MODE_RAW;
    const uint64_t batch_max = 1ull << 22;
    while (p->T < T) {
        const uint64_t j0 = p->T;
        const uint32_t count = (uint32_t)std::min<uint64_t>(T - j0, batch_max);
        const unsigned long long verts_before = p->hc.rr_vertices;
        RC(reserve_heaps(p, count));
        if (p->tiles) RC(run_tiles(p, (uint32_t)j0, count));
        else RC(run_sample(p, mode, (uint32_t)j0, count, nullptr, nullptr, p->cut, p->shape));
        // selection index of the new sets
        const uint64_t added = p->hc.rr_vertices - verts_before;
        const uint64_t items_need = p->hc.chunk_items + added / 32 + 2ull * count + 16;
        if (items_need > p->items_cap) {
            const uint64_t nc = std::max<uint64_t>(items_need + items_need / 4, p->items_cap * 2);
            RC(grow_buffer(p, (void**)&p->items, p->items_cap * 8, nc * 8, p->hc.chunk_items * 8));
            p->items_cap = nc;
        }
        const uint64_t bm_need = p->hc.bm_list + count;
        if (bm_need > p->bm_list_cap) {
            const uint64_t nc = std::max<uint64_t>(bm_need + bm_need / 4, p->bm_list_cap * 2);
            RC(grow_buffer(p, (void**)&p->bm_sets, p->bm_list_cap * 4, nc * 4, p->hc.bm_list * 4));
            p->bm_list_cap = nc;
        }
        IndexArgs ia;
        ia.recs = p->recs;
        ia.j0 = (uint32_t)j0;
        ia.j1 = (uint32_t)(j0 + count);
        ia.chunk_items = p->items;
        ia.items_cap = p->items_cap;
        ia.bm_sets = p->bm_sets;
        ia.bm_cap = (uint32_t)std::min<uint64_t>(p->bm_list_cap, 0xFFFFFFFFull);
        ia.ctr = p->ctr;
        ia.moments = p->moments;
        CK(launch_index(ia, p->stream));
        p->launches++;
        RC(read_counters(p));
        p->T = j0 + count;
        p->bounds[p->T] = {p->hc.chunk_items, p->hc.bm_list, p->hc.words_used};
    }
    p->sample_s += now_s() - t0;
    return HBX_OK;
}

// ---------------------------------------------------------------------------
// selection
// ---------------------------------------------------------------------------
static int ensure_sel(hbx_pool* p, uint64_t T, uint32_t k) {
    const uint32_t n4 = (p->g->n + 3) & ~3u;
    if (!p->cnt) {
        RC(grow_buffer(p, (void**)&p->cnt, 0, (size_t)n4 * 4, 0));
        RC(grow_buffer(p, (void**)&p->st, 0, sizeof(SelState), 0));
        RC(grow_buffer(p, (void**)&p->partials, 0, (size_t)p->ctx->sms * 8 * 8, 0));
        RC(grow_buffer(p, (void**)&p->ticket, 0, 256, 0));
    }
    if (T > p->alive_cap) {
        // a multiple of 32: a tile's 32 live flags are read as two 16-byte words
        const uint64_t nc = (std::max<uint64_t>(T, p->alive_cap * 2) + 31) & ~31ull;
        RC(grow_buffer(p, (void**)&p->alive, p->alive_cap, nc, 0));
        RC(grow_buffer(p, (void**)&p->cov_huff, p->alive_cap * 4, nc * 4, 0));
        RC(grow_buffer(p, (void**)&p->cov_bm, p->alive_cap * 4, nc * 4, 0));
        RC(grow_buffer(p, (void**)&p->cov_raw, p->alive_cap * 4, nc * 4, 0));
        if (p->tiles) RC(grow_buffer(p, (void**)&p->tile_live, p->alive_cap / 8, nc / 8, 0));
        p->alive_cap = nc;
    }
    if (p->tiles && (T + 31) / 32 > p->dec_cap) {
        // one decrement entry per covered tile
        const uint64_t nc = std::max<uint64_t>((T + 31) / 32, p->dec_cap * 2);
        RC(grow_buffer(p, (void**)&p->dec_items, p->dec_cap * 8, nc * 8, 0));
        p->dec_cap = nc;
    }
    if (p->hc.chunk_items > p->dec_cap) {
        // the sets covered in one iteration hold at most every chunk of the pool
        const uint64_t nc = std::max<uint64_t>(p->hc.chunk_items, p->dec_cap * 2);
        RC(grow_buffer(p, (void**)&p->dec_items, p->dec_cap * 8, nc * 8, 0));
        p->dec_cap = nc;
    }
    if (k > p->kcap) {
        RC(grow_buffer(p, (void**)&p->d_seeds, p->kcap * 4, (size_t)k * 4, 0));
        RC(grow_buffer(p, (void**)&p->d_marg, p->kcap * 8, (size_t)k * 8, 0));
        p->kcap = k;
    }
    return HBX_OK;
}

static SelArgs sel_args(hbx_pool* p, uint64_t T) {
    SelArgs a;
    memset(&a, 0, sizeof(a));
    a.n = p->g->n;
    a.n4 = (p->g->n + 3) & ~3u;
    a.T = (uint32_t)T;
    a.recs = p->recs;
    a.raw_heap = p->raw.d;
    a.code_heap = p->code.d;
    a.bm_heap = p->bm.d;
    a.cb = dev_codebook(p);
    a.has_cb = p->has_cb ? 1u : 0u;
    a.hot = p->has_cb ? std::min<uint32_t>(p->nsym, 12288u) : 0u;
    a.cnt = p->cnt;
    a.alive = p->alive;
    a.chunk_items = p->items;
    a.n_items = p->hc.chunk_items;
    a.bm_sets = p->bm_sets;
    a.n_bm = (uint32_t)p->hc.bm_list;
    a.st = (SelState*)p->st;
    a.cov_huff = p->cov_huff;
    a.cov_bm = p->cov_bm;
    a.cov_raw = p->cov_raw;
    a.dec_items = p->dec_items;
    a.dec_cap = p->dec_cap;
    a.partials = p->partials;
    a.ticket = p->ticket;
    a.seeds = p->d_seeds;
    a.marginal = p->d_marg;
    a.sms = p->ctx->sms;
    a.wait_cycles = p->o.wait_cycles ? (long long)std::min<uint64_t>(p->o.wait_cycles, 1ull << 62) : 4000000000ll;
    a.select_mode = p->o.select_mode;
    a.tiles = p->tiles ? 1u : 0u;
    a.n4w = ((uint64_t)p->g->n + 3) & ~3ull;
    a.tile_live = p->tile_live;
    return a;
}

// The persistent selection's grid barrier lives in the pool's small counter
// allocation, after the argmax finish counter.
static SelBarrier* sel_barrier(hbx_pool* p) {
    return reinterpret_cast<SelBarrier*>(reinterpret_cast<char*>(p->ticket) + 64);
}

// Launch greedy selection on sets [0, T) on stream `st` without waiting.  The
// batched form runs the k iterations in one persistent cooperative launch; the
// plain form launches them one by one and reads u* back after each.
static int pool_select_launch(hbx_pool* p, uint64_t T, uint32_t k, cudaStream_t st, uint64_t j_lo = 0) {
    hbx_ctx* ctx = p->ctx;
    if (T == 0 || T > p->T) return fail(ctx, HBX_ERR_INVALID_ARG, "T must be in [1, pool size]");
    if (k == 0 || k > p->g->n) return fail(ctx, HBX_ERR_INVALID_ARG, "k must be in [1, n]");
    if (j_lo >= T) return fail(ctx, HBX_ERR_INVALID_ARG, "a selection range must start below T");
    // the last batch end at or below j_lo (the count passes skip sets below j_lo)
    auto lo_bd = p->bounds.upper_bound(j_lo);
    const bool lo_known = lo_bd != p->bounds.begin();
    if (lo_known) --lo_bd;
    cudaSetDevice(ctx->device);
    RC(ensure_sel(p, T, k));
    SelArgs a = sel_args(p, T);
    a.j_lo = (uint32_t)j_lo;  // sets below j_lo start covered
    const uint32_t enc = p->o.encode;
    CK(launch_sel_init(a, st));
    // The batched form counts incrementally: the undecremented counts of the
    // last selection's prefix [0, base_T) are restored and only the sets
    // [base_T, T) are counted (their chunk items and bitmap entries follow the
    // prefix's, base_T being a batch end).
    SelArgs c = a;
    const size_t cbytes = (size_t)a.n4 * 4;
    const auto bd = p->bounds.find(p->base_T);
    uint64_t words_lo = 0;
    if (j_lo) {
        // a range [j_lo, T): counted from scratch
        if (lo_known) {
            c.chunk_items = p->items + lo_bd->second.items;
            c.n_items = a.n_items - lo_bd->second.items;
            c.bm_sets = p->bm_sets + lo_bd->second.bm;
            c.n_bm = a.n_bm - (uint32_t)lo_bd->second.bm;
            words_lo = lo_bd->second.words;
        }
    } else if (p->o.form && p->base_T && p->base_T <= T && bd != p->bounds.end()) {
        CK(cudaMemcpyAsync(p->cnt, p->cnt_base, cbytes, cudaMemcpyDeviceToDevice, st));
        c.chunk_items = p->items + bd->second.items;
        c.n_items = a.n_items - bd->second.items;
        c.bm_sets = p->bm_sets + bd->second.bm;
        c.n_bm = a.n_bm - (uint32_t)bd->second.bm;
        c.j_lo = (uint32_t)p->base_T;
        words_lo = bd->second.words;
    }
    if (!p->evc0) {
        CK(cudaEventCreate(&p->evc0));
        CK(cudaEventCreate(&p->evc1));
        CK(cudaEventCreate(&p->evs0));
        CK(cudaEventCreate(&p->evs1));
    }
    CK(cudaEventRecord(p->evc0, st));
    CK(launch_count(c, enc, st));
    CK(cudaEventRecord(p->evc1, st));
    p->count_pending = true;
    {
        const auto hi = p->bounds.find(T);
        const uint64_t words_hi = hi != p->bounds.end() ? hi->second.words : p->hc.words_used;
        p->count_bytes += 4 * (words_hi - std::min(words_hi, words_lo)) + 16 * (T - c.j_lo) + 8 * c.n_items +
                          4ull * c.n_bm;
    }
    if (p->o.form && p->bounds.count(T) && !j_lo) {
        if (!p->cnt_base) RC(grow_buffer(p, (void**)&p->cnt_base, 0, cbytes, 0));
        CK(cudaMemcpyAsync(p->cnt_base, p->cnt, cbytes, cudaMemcpyDeviceToDevice, st));
        p->base_T = T;
    }
    const uint64_t per_it = 3 + (enc ? (uint64_t)(a.has_cb ? 1 : 0) + (a.n_bm ? 1 : 0) : 1);
    p->launches += 1 + (enc ? (uint64_t)((a.n_items && a.has_cb) ? 1 : 0) + (a.n_bm ? 1 : 0) : 1);
    CK(cudaEventRecord(p->evs0, st));
    if (p->o.form) {
        // all k iterations in one cooperative launch with bounded grid barriers
        SelBarrier* bar = sel_barrier(p);
        CK(cudaMemsetAsync(bar, 0, sizeof(SelBarrier), st));
        CK(launch_select_persistent(a, k, bar, st));
        p->launches += 1;
        CK(cudaEventRecord(p->evs1, st));
    } else {
        p->launches += per_it * k;
        SelState hs;
        for (uint32_t it = 0; it < k; it++) {
            CK(launch_iteration(a, enc, st));
            CK(cudaMemcpyAsync(&hs, a.st, sizeof(SelState), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        }
        CK(cudaEventRecord(p->evs1, st));
    }
    return HBX_OK;
}

// Wait for the selection launched on `st` and read its results.
static int pool_select_finish(hbx_pool* p, uint32_t k, uint32_t* seeds, uint64_t* marginal, uint64_t* covered,
                              cudaStream_t st) {
    hbx_ctx* ctx = p->ctx;
    SelState hs;
    std::vector<unsigned long long> hm(k);
    CK(cudaMemcpyAsync(&hs, p->st, sizeof(SelState), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(seeds, p->d_seeds, (size_t)k * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hm.data(), p->d_marg, (size_t)k * 8, cudaMemcpyDeviceToHost, st));
    SelBarrier hb = {0, 0, 0, 0};
    if (p->o.form) CK(cudaMemcpyAsync(&hb, sel_barrier(p), sizeof(hb), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hb.err) return fail(ctx, HBX_ERR_TIMEOUT, "selection: a grid barrier wait ran out");
    if (p->count_pending) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, p->evc0, p->evc1));
        p->count_kernel_s += ms * 1e-3;
        CK(cudaEventElapsedTime(&ms, p->evs0, p->evs1));
        p->select_kernel_s += ms * 1e-3;
        p->count_pending = false;
    }
    p->select_iterations += hs.it;
    p->dec_bytes += hs.dec_bytes;
    p->dec_s += 1e-9 * (double)(hs.t_cover_ns + hs.t_dec_ns);
    p->argmax_s += 1e-9 * (double)hs.t_argmax_ns;
    if (hs.pad == 1) return fail(ctx, HBX_ERR_INTERNAL, "undecodable Huffman stream during selection");
    if (hs.pad) return fail(ctx, HBX_ERR_INTERNAL, "decrement item list overflow during selection");
    if (hs.it != k) return fail(ctx, HBX_ERR_INTERNAL, "selection ran " + std::to_string(hs.it) + " iterations");
    if (marginal)
        for (uint32_t i = 0; i < k; i++) marginal[i] = hm[i];
    if (covered) *covered = hs.covered;
    return HBX_OK;
}

int pool_select(hbx_pool* p, uint64_t T, uint32_t k, uint32_t* seeds, uint64_t* marginal, uint64_t* covered,
                uint64_t j_lo) {
    const double t0 = now_s();
    RC(pool_select_launch(p, T, k, p->stream, j_lo));
    RC(pool_select_finish(p, k, seeds, marginal, covered, p->stream));
    p->select_s += now_s() - t0;
    return HBX_OK;
}

}  // namespace hbx

extern "C" int hbx_pool_create(hbx_ctx* ctx, hbx_graph* g, hbx_model model, uint64_t seed, const hbx_options* opts,
                               hbx_pool** out) {
    if (!ctx || !g || !out) return HBX_ERR_INVALID_ARG;
    *out = nullptr;
    if (model != HBX_IC && model != HBX_LT) return fail(ctx, HBX_ERR_INVALID_ARG, "unknown model");
    if (model == HBX_IC && !g->thr) return fail(ctx, HBX_ERR_INVALID_ARG, "graph has no IC probabilities");
    if (model == HBX_LT && !g->q) return fail(ctx, HBX_ERR_INVALID_ARG, "graph has no LT weights");
    hbx_options o;
    hbx_default_options(&o);
    if (opts) o = *opts;
    if (o.density_cut == 0) o.density_cut = 32;
    if (o.encode > 1 || o.form > 1) return fail(ctx, HBX_ERR_INVALID_ARG, "encode and form are 0 or 1");
    if (o.warp_capacity && (o.warp_capacity < 64 || o.warp_capacity > 2048 ||
                            (o.warp_capacity & (o.warp_capacity - 1))))
        return fail(ctx, HBX_ERR_INVALID_ARG, "warp_capacity must be a power of two in [64, 2048]");
    if (o.block_cluster > 8 || (o.block_cluster & (o.block_cluster - 1)))
        return fail(ctx, HBX_ERR_INVALID_ARG, "block_cluster must be 0, 1, 2, 4 or 8");
    if (o.scheme > 1 || o.select_mode > 2 || o.fresh_final > 1)
        return fail(ctx, HBX_ERR_INVALID_ARG, "scheme and fresh_final are 0 or 1, select_mode 0, 1 or 2");
    if (o.scheme && !o.encode) return fail(ctx, HBX_ERR_INVALID_ARG, "the per-graph scheme needs encode = 1");
    if (g->n >= 0xFFFFFFFFu && o.scheme) return fail(ctx, HBX_ERR_INVALID_ARG, "graph too large for the Bitmax cut");
    cudaSetDevice(ctx->device);
    hbx_pool* p = new hbx_pool();
    p->ctx = ctx;
    p->g = g;
    p->model = model;
    p->seed = seed;
    p->o = o;
    p->W = o.warmup_sets;
    p->cut = o.density_cut;
    p->stream = ctx->stream;
    p->bp_words = (((uint64_t)g->n + 31) / 32 + 3) & ~3ull;
    int r = grow_buffer(p, (void**)&p->ctr, 0, sizeof(Counters), 0);
    if (!r) r = grow_buffer(p, (void**)&p->moments, 0, 3 * sizeof(double), 0);
    if (!r && (cudaEventCreate(&p->ev0) != cudaSuccess || cudaEventCreate(&p->ev1) != cudaSuccess))
        r = fail(ctx, HBX_ERR_CUDA, "cudaEventCreate");
    if (!r) {
        memset(&p->hc, 0, sizeof(p->hc));
        std::lock_guard<std::mutex> lock(ctx->mu);
        ctx->pools.insert(p);
        *out = p;
        return HBX_OK;
    }
    dfree(ctx, p->ctr);
    dfree(ctx, p->moments);
    delete p;
    return r;
}

extern "C" void hbx_pool_destroy(hbx_pool* p) {
    if (!p) return;
    hbx_ctx* c = p->ctx;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(p->stream);
    void* bufs[] = {p->recs, p->raw.d, p->code.d, p->bm.d, p->ctr, p->moments, p->rank_of, p->vertex_of_rank,
                    p->code_of_rank, p->len_of_rank, p->lut, p->dec, p->items, p->bm_sets, p->big_list,
                    p->retry_list, p->list_in, p->giant_list, p->bp_visited, p->bp_rbits, p->bp_aux, p->bp_queue, p->cnt,
                    p->alive, p->cov_huff, p->cov_bm, p->cov_raw, p->st, p->partials, p->ticket, p->d_seeds,
                    p->d_marg, p->dec_items, p->cnt_base, p->ms_vis, p->ms_nxt, p->ms_F, p->ms_N, p->ms_pend, p->ms_ndef,
                    p->ms_heavy, p->ms_c, p->ms_sets, p->ms_rowoff, p->ms_sparse, p->tile_live};
    for (void* b : bufs) dfree(c, b);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    if (p->ms_first) cudaGraphExecDestroy(p->ms_first);
    if (p->ms_more) cudaGraphExecDestroy(p->ms_more);
    if (p->evc0) cudaEventDestroy(p->evc0);
    if (p->evs0) cudaEventDestroy(p->evs0);
    if (p->evs1) cudaEventDestroy(p->evs1);
    if (p->evc1) cudaEventDestroy(p->evc1);
    if (p->own_stream) cudaStreamDestroy(p->stream);
    {
        std::lock_guard<std::mutex> lock(c->mu);
        c->pools.erase(p);
    }
    delete p;
}

extern "C" int hbx_pool_extend(hbx_pool* p, uint64_t T) {
    if (!p) return HBX_ERR_INVALID_ARG;
    return pool_extend(p, T);
}

extern "C" uint64_t hbx_pool_size(const hbx_pool* p) { return p ? p->T : 0; }

extern "C" int hbx_pool_select(hbx_pool* p, uint64_t T, uint32_t k, uint32_t* seeds, uint64_t* marginal,
                               uint64_t* covered) {
    if (!p || !seeds) return HBX_ERR_INVALID_ARG;
    return pool_select(p, T, k, seeds, marginal, covered);
}

// ===========================================================================
// IMM (Section 2.2, Eq. (1)), read as IMM's own bounds with eps' = sqrt(2) eps:
//   l'      = l (1 + ln 2 / ln n)
//   lambda' = (2 + 2 eps'/3)(ln C(n,k) + l' ln n + ln log2 n) n / eps'^2
//   lambda* = 2 n ((1 - 1/e) alpha + beta)^2 / eps^2,
//   alpha = sqrt(l' ln n + ln 2), beta = sqrt((1 - 1/e)(ln C(n,k) + l' ln n + ln 2))
// Round i = 1 .. floor(log2 n) - 1: x = n / 2^i, T_i = max(T_{i-1}, ceil(lambda'/x)),
// greedy on [0, T_i); stop when n cov / T_i >= (1 + eps') x with
// LB = (n cov / T_i) / (1 + eps').  Final theta = max(T_i, ceil(lambda*/LB)).
// ===========================================================================
namespace hbx {

struct ImmBounds {
    double epsp, ellp, lnc, lambda_p, lambda_star;
};

static bool imm_bounds(uint32_t n, uint32_t k, double eps, double ell, ImmBounds* b);

bool imm_lambda(uint32_t n, uint32_t k, double eps, double ell, double* lambda_p, double* lambda_star) {
    ImmBounds b;
    if (!imm_bounds(n, k, eps, ell, &b)) return false;
    *lambda_p = b.lambda_p;
    *lambda_star = b.lambda_star;
    return true;
}

static bool imm_bounds(uint32_t n, uint32_t k, double eps, double ell, ImmBounds* b) {
    if (n < 2 || k == 0 || k > n || !(eps > 0.0 && eps < 1.0) || !(ell > 0.0)) return false;
    const double dn = (double)n;
    const double epsp = std::sqrt(2.0) * eps;
    const double ellp = ell * (1.0 + std::log(2.0) / std::log(dn));
    double lnc = 0.0;
    for (uint32_t i = 1; i <= k; i++) lnc += std::log(((double)(n - k) + (double)i) / (double)i);
    const double lambda_p =
        (2.0 + 2.0 * epsp / 3.0) * (lnc + ellp * std::log(dn) + std::log(std::log2(dn))) * dn / (epsp * epsp);
    const double e1 = 1.0 - std::exp(-1.0);
    const double alpha = std::sqrt(ellp * std::log(dn) + std::log(2.0));
    const double beta = std::sqrt(e1 * (lnc + ellp * std::log(dn) + std::log(2.0)));
    const double s = e1 * alpha + beta;
    b->epsp = epsp;
    b->ellp = ellp;
    b->lnc = lnc;
    b->lambda_p = lambda_p;
    b->lambda_star = 2.0 * dn * s * s / (eps * eps);
    return true;
}

static uint32_t ilog2_floor(uint32_t n) { return 31u - (uint32_t)__builtin_clz(n); }

void fill_stats(hbx_pool* p, hbx_stats* s) {
    memset(s, 0, sizeof(*s));
    s->theta = p->T;
    s->sets_huffman = p->hc.sets_huff;
    s->sets_bitmap = p->hc.sets_bm;
    s->sets_raw = p->hc.sets_raw;
    s->sets_big = p->hc.sets_big;
    s->rr_vertices = p->hc.rr_vertices;
    s->edges_scanned = p->hc.edges_scanned - p->aux_scanned;
    s->edges_live = p->hc.edges_live - p->aux_live;
    s->code_bits = p->hc.code_bits;
    s->warmup_sets = p->o.encode ? p->W : 0;
    s->warp_capacity = p->shape.qw;
    s->warp_group_budget = p->shape.gb;
    s->block_cluster = p->shape.bc;
    s->second_warp_capacity = p->shape.q2;
    double mom[3] = {0, 0, 0};
    cudaMemcpyAsync(mom, p->moments, 3 * sizeof(double), cudaMemcpyDeviceToHost, p->stream);
    cudaStreamSynchronize(p->stream);
    // bytes held by the sets (heap words written) plus the 16-byte index per set
    s->pool_bytes = 4ull * p->hc.words_used + sizeof(SetRec) * p->T;
    s->raw_int32_bytes = 4ull * p->hc.rr_vertices + 8ull * p->T;
    if (p->T) {
        const double T = (double)p->T, mean = mom[0] / T;
        const double m2 = mom[1] / T - mean * mean;
        const double m3 = mom[2] / T - 3 * mean * mom[1] / T + 2 * mean * mean * mean;
        s->skewness = m2 > 0 ? m3 / (m2 * std::sqrt(m2)) : 0.0;
        s->density = mom[0] / (T * (double)p->g->n);
    }
    s->sample_s = p->sample_s;
    s->select_s = p->select_s;
    s->sample_kernel_s = p->sample_kernel_s;
    s->sample_kernel_launches = p->sample_kernel_launches;
    s->kernel_launches = p->launches;
    s->count_kernel_s = p->count_kernel_s;
    s->count_bytes = p->count_bytes;
    s->ms_kernel_s = p->ms_kernel_s;
    s->ms_sets = p->ms_nsets;
    s->ms_philox_blocks = p->ms_blocks;
    s->ms_group_visits = p->ms_visits;
    s->ms_deferrals = p->ms_deferred;
    s->select_kernel_s = p->select_kernel_s;
    s->select_iterations = p->select_iterations;
    s->dec_s = p->dec_s;
    s->dec_bytes = p->dec_bytes;
    s->uncoded_vertices = p->hc.uncoded;
    s->scheme = !p->o.scheme ? 0u : (!p->bitmax ? 1u : (p->tiles ? 3u : 2u));
    s->scheme_skewness = p->scheme_skew;
    s->argmax_s = p->argmax_s;
}

int imm_on_pool(hbx_pool* p, uint32_t k, double eps, double ell, uint32_t* seeds, double* influence,
                uint64_t* marginal, hbx_stats* stats) {
    hbx_ctx* ctx = p->ctx;
    const double t0 = now_s();
    const uint32_t n = p->g->n;
    ImmBounds b;
    if (!imm_bounds(n, k, eps, ell, &b)) return fail(ctx, HBX_ERR_INVALID_ARG, "bad k, eps, ell or n");
    const double dn = (double)n;
    if (p->o.encode && !p->has_cb && p->W == 0) {
        const uint64_t T1 = (uint64_t)std::ceil(b.lambda_p / (dn / std::ldexp(1.0, 1)));
        p->W = (T1 + 7) / 8;
    }
    std::vector<uint32_t> last_seeds(k);
    std::vector<uint64_t> last_marg(k);
    uint64_t Ti = 0, last_T = 0, last_cov = 0;
    double LB = 1.0;
    uint32_t rounds = 0;
    const uint32_t imax = ilog2_floor(n) - 1;
    for (uint32_t i = 1; i <= imax; i++) {
        const double x = dn / std::ldexp(1.0, (int)i);
        const uint64_t t = (uint64_t)std::ceil(b.lambda_p / x);
        if (t > Ti) Ti = t;
        RC(pool_extend(p, Ti));
        uint64_t cov = 0;
        if (Ti != last_T) {
            RC(pool_select(p, Ti, k, last_seeds.data(), last_marg.data(), &cov));
            last_T = Ti;
            last_cov = cov;
        }
        cov = last_cov;
        rounds++;
        const double est = dn * (double)cov / (double)Ti;
        if (est >= (1.0 + b.epsp) * x) {
            LB = est / (1.0 + b.epsp);
            break;
        }
    }
    uint64_t T = (uint64_t)std::ceil(b.lambda_star / LB);
    uint64_t cov = 0;
    if (p->o.fresh_final) {
        // the final phase on theta new sets [T_i, T_i + theta)
        RC(pool_extend(p, Ti + T));
        RC(pool_select(p, Ti + T, k, seeds, marginal, &cov, Ti));
    } else if ((T = std::max(T, Ti)) == last_T) {
        // greedy selection is a function of the sets [0, T): the last round's
        // result is the final one
        for (uint32_t i = 0; i < k; i++) seeds[i] = last_seeds[i];
        if (marginal)
            for (uint32_t i = 0; i < k; i++) marginal[i] = last_marg[i];
        cov = last_cov;
    } else {
        RC(pool_extend(p, T));
        RC(pool_select(p, T, k, seeds, marginal, &cov));
    }
    *influence = dn * (double)cov / (double)T;
    if (stats) {
        fill_stats(p, stats);
        stats->theta = T;
        stats->covered = cov;
        stats->rounds = rounds;
        stats->lb = LB;
        stats->total_s = now_s() - t0;
    }
    return HBX_OK;
}

}  // namespace hbx

extern "C" int hbx_imm_pool(hbx_pool* p, uint32_t k, double eps, double ell, uint32_t* seeds, double* influence,
                            uint64_t* marginal, hbx_stats* stats) {
    if (!p || !seeds || !influence) return HBX_ERR_INVALID_ARG;
    return imm_on_pool(p, k, eps, ell, seeds, influence, marginal, stats);
}

extern "C" int hbx_imm(hbx_ctx* ctx, hbx_graph* g, hbx_model model, uint32_t k, double eps, double ell,
                       uint64_t seed, const hbx_options* opts, uint32_t* seeds, double* influence,
                       uint64_t* marginal, hbx_stats* stats) {
    if (!ctx || !g || !seeds || !influence) return HBX_ERR_INVALID_ARG;
    hbx_pool* p = nullptr;
    RC(hbx_pool_create(ctx, g, model, seed, opts, &p));
    const int r = imm_on_pool(p, k, eps, ell, seeds, influence, marginal, stats);
    hbx_pool_destroy(p);
    return r;
}

// ===========================================================================
// inspection
// ===========================================================================
namespace hbx {
// Decode sets [j0, j1) on the device (offsets: host, j1-j0+1 entries already
// filled; verts: host) and optionally return each Huffman stream's end bit.
static int decode_range(hbx_pool* p, uint64_t j0, uint64_t j1, const uint64_t* offsets, uint32_t* verts,
                        uint64_t* ends) {
    hbx_ctx* ctx = p->ctx;
    const uint64_t cnt = j1 - j0;
    unsigned long long* d_off = nullptr;
    unsigned long long* d_end = nullptr;
    uint32_t* d_out = nullptr;
    RC(dalloc(ctx, (void**)&d_off, (cnt + 1) * 8));
    int r = dalloc(ctx, (void**)&d_out, std::max<uint64_t>(offsets[cnt], 1) * 4);
    if (!r) r = dalloc(ctx, (void**)&d_end, cnt * 8);
    if (r) {
        dfree(ctx, d_off);
        dfree(ctx, d_out);
        return r;
    }
    DecodeArgs a;
    a.recs = p->recs;
    a.raw_heap = p->raw.d;
    a.code_heap = p->code.d;
    a.bm_heap = p->bm.d;
    a.cb = dev_codebook(p);
    a.has_cb = p->has_cb;
    a.n = p->g->n;
    a.j0 = (uint32_t)j0;
    a.j1 = (uint32_t)j1;
    a.offsets = d_off;
    a.out = d_out;
    a.ends = d_end;
    a.ctr = p->ctr;
    a.tiles = p->tiles ? 1u : 0u;
    cudaError_t e = cudaMemcpyAsync(d_off, offsets, (cnt + 1) * 8, cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_end, 0, cnt * 8, p->stream);
    if (e == cudaSuccess) e = launch_decode(a, p->stream);
    p->launches++;
    if (e == cudaSuccess && offsets[cnt])
        e = cudaMemcpyAsync(verts, d_out, offsets[cnt] * 4, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess && ends) e = cudaMemcpyAsync(ends, d_end, cnt * 8, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    dfree(ctx, d_off);
    dfree(ctx, d_out);
    dfree(ctx, d_end);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "decode");
    return read_counters(p);
}
}  // namespace hbx

extern "C" int hbx_pool_export_set(hbx_pool* p, uint64_t j, uint32_t* kind, uint32_t* size, uint32_t* n_coded,
                                   uint32_t* n_raw, uint64_t* code_bits, uint8_t* payload, uint64_t cap,
                                   uint64_t* nbytes) {
    if (!p) return HBX_ERR_INVALID_ARG;
    hbx_ctx* ctx = p->ctx;
    if (j >= p->T) return fail(ctx, HBX_ERR_INVALID_ARG, "set id beyond the pool");
    cudaSetDevice(ctx->device);
    SetRec r;
    CK(cudaMemcpyAsync(&r, p->recs + j, sizeof(r), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    const uint32_t k = rec_kind(r);
    const uint64_t off = rec_off(r);
    if (k == KIND_PENDING) return fail(ctx, HBX_ERR_INTERNAL, "set not written");
    uint64_t bits = 0;
    if (k == KIND_HUFF) {
        // the stream length is where the decoder stops after n_coded codes
        std::vector<uint64_t> offs = {0, r.size};
        std::vector<uint32_t> tmp(std::max<uint32_t>(r.size, 1));
        RC(decode_range(p, j, j + 1, offs.data(), tmp.data(), &bits));
    }
    if (kind) *kind = k;
    if (size) *size = r.size;
    if (n_coded) *n_coded = k == KIND_HUFF ? r.n_coded : 0;
    if (n_raw) *n_raw = k == KIND_HUFF ? r.size - r.n_coded : 0;
    if (code_bits) *code_bits = bits;
    std::vector<uint8_t> buf;
    if (k == KIND_HUFF) {
        const uint32_t nside = side_words(r.n_coded);
        const uint32_t nr = r.size - r.n_coded;
        const uint64_t cb = (bits + 7) / 8, cw = (bits + 31) / 32;
        const uint64_t raw_at = (cb + 3) & ~3ull;
        buf.assign(raw_at + 4ull * nr, 0);
        std::vector<uint32_t> words(cw + 1);
        if (cw)
            CK(cudaMemcpyAsync(words.data(), p->code.d + off + nside + nr, cw * 4, cudaMemcpyDeviceToHost,
                               p->stream));
        if (nr)
            CK(cudaMemcpyAsync(buf.data() + raw_at, p->code.d + off + nside, 4ull * nr, cudaMemcpyDeviceToHost,
                               p->stream));
        CK(cudaStreamSynchronize(p->stream));
        memcpy(buf.data(), words.data(), cb);
    } else if (k == KIND_BITMAP) {
        const uint32_t n = p->g->n;
        const uint64_t nw = ((uint64_t)n + 31) / 32;
        buf.assign(nw * 4, 0);
        if (p->tiles) {
            // column j % 32 of a vertex-major tile
            std::vector<uint32_t> tile(n);
            CK(cudaMemcpyAsync(tile.data(), p->bm.d + off, (size_t)n * 4, cudaMemcpyDeviceToHost, p->stream));
            CK(cudaStreamSynchronize(p->stream));
            uint32_t* row = reinterpret_cast<uint32_t*>(buf.data());
            for (uint32_t v = 0; v < n; v++)
                if ((tile[v] >> (j & 31)) & 1u) row[v >> 5] |= 1u << (v & 31);
        } else {
            CK(cudaMemcpyAsync(buf.data(), p->bm.d + off, nw * 4, cudaMemcpyDeviceToHost, p->stream));
            CK(cudaStreamSynchronize(p->stream));
        }
    } else {
        buf.resize(4ull * r.size);
        CK(cudaMemcpyAsync(buf.data(), p->raw.d + off, 4ull * r.size, cudaMemcpyDeviceToHost, p->stream));
        CK(cudaStreamSynchronize(p->stream));
    }
    if (nbytes) *nbytes = buf.size();
    if (buf.size() > cap || (!payload && buf.size()))
        return fail(ctx, HBX_ERR_INVALID_ARG, "payload buffer too small");
    if (buf.size()) memcpy(payload, buf.data(), buf.size());
    return HBX_OK;
}

extern "C" int hbx_pool_decode_sets(hbx_pool* p, uint64_t j0, uint64_t j1, uint64_t* offsets, uint32_t* verts,
                                    uint64_t cap, uint64_t* needed) {
    if (!p || !offsets) return HBX_ERR_INVALID_ARG;
    hbx_ctx* ctx = p->ctx;
    if (j0 > j1 || j1 > p->T) return fail(ctx, HBX_ERR_INVALID_ARG, "range beyond the pool");
    cudaSetDevice(ctx->device);
    const uint64_t cnt = j1 - j0;
    std::vector<SetRec> recs(cnt);
    if (cnt)
        CK(cudaMemcpyAsync(recs.data(), p->recs + j0, cnt * sizeof(SetRec), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    offsets[0] = 0;
    for (uint64_t i = 0; i < cnt; i++) offsets[i + 1] = offsets[i] + recs[i].size;
    if (needed) *needed = offsets[cnt];
    if (offsets[cnt] > cap || (!verts && offsets[cnt]))
        return fail(ctx, HBX_ERR_INVALID_ARG, "verts buffer too small");
    if (!cnt) return HBX_OK;
    RC(decode_range(p, j0, j1, offsets, verts, nullptr));
    for (uint64_t i = 0; i < cnt; i++) std::sort(verts + offsets[i], verts + offsets[i + 1]);
    return HBX_OK;
}

extern "C" int hbx_pool_export_codebook(hbx_pool* p, uint32_t* len_of_v, uint32_t* code_of_v, uint32_t* rank_of_v,
                                        uint32_t* freq) {
    if (!p) return HBX_ERR_INVALID_ARG;
    if (!p->has_cb) return fail(p->ctx, HBX_ERR_INVALID_ARG, "pool has no codebook");
    const uint32_t n = p->g->n;
    if (len_of_v) memcpy(len_of_v, p->h_len.data(), (size_t)n * 4);
    if (code_of_v) memcpy(code_of_v, p->h_code.data(), (size_t)n * 4);
    if (rank_of_v) memcpy(rank_of_v, p->h_rank.data(), (size_t)n * 4);
    if (freq) memcpy(freq, p->h_freq.data(), (size_t)n * 4);
    return HBX_OK;
}

extern "C" int hbx_pool_stats(hbx_pool* p, hbx_stats* s) {
    if (!p || !s) return HBX_ERR_INVALID_ARG;
    cudaSetDevice(p->ctx->device);
    fill_stats(p, s);
    return HBX_OK;
}

extern "C" int hbx_philox_ceiling(hbx_ctx* ctx, double* blocks_per_s) {
    using namespace hbx;
    if (!ctx || !blocks_per_s) return HBX_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    const uint32_t blocks = (uint32_t)ctx->sms * 8, per_thread = 4096;
    void* out = nullptr;
    RC(dalloc(ctx, &out, (size_t)blocks * 256 * 4));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HBX_OK;
    float best = 0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = cuda_fail(ctx, cudaGetLastError(), "cudaEventCreate");
    } else {
        for (int r = 0; r < 4 && rc == HBX_OK; r++) {
            cudaEventRecord(e0, ctx->stream);
            cudaError_t le = launch_philox_ceiling(blocks, per_thread, (uint32_t*)out, ctx->stream);
            cudaEventRecord(e1, ctx->stream);
            if (le == cudaSuccess) le = cudaEventSynchronize(e1);
            float ms = 0;
            if (le == cudaSuccess) le = cudaEventElapsedTime(&ms, e0, e1);
            if (le != cudaSuccess) rc = cuda_fail(ctx, le, "Philox ceiling");
            else if (r > 0 && (best == 0 || ms < best)) best = ms;  // launch 0 warms up
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dfree(ctx, out);
    if (rc == HBX_OK) *blocks_per_s = (double)blocks * 256.0 * per_thread / (best * 1e-3);
    return rc;
}
