// Host-side declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace hbx {

// ---- sampling (sample.cu) ----
cudaError_t launch_sample_warp(const SampleArgs& a, uint32_t qw, int sms, cudaStream_t s);
cudaError_t launch_sample_mid(const SampleArgs& a, uint32_t nbig, int sms, cudaStream_t s);
cudaError_t launch_sample_block(const SampleArgs& a, uint32_t nbig, uint32_t slots, uint32_t csize, cudaStream_t s);
int block_path_max_clusters(uint32_t csize);

// ---- bit-parallel search of heavy IC sets (msbfs.cu) ----
constexpr uint32_t MS_SETS = 32;  // sets searched together, one mask bit each

struct MsCounters {
    uint32_t nF, nN, nH, nsets;       // frontier, next frontier being compacted, heavy chunks of this level;
                                      // sets of the batch
    uint32_t npend;                   // vertices whose expansion the compaction being run deferred
    uint32_t force;                   // this level's compaction expands every deferred vertex
    uint32_t lwork, hwork;            // work-stealing cursors of this level's light and heavy kernels
    unsigned long long size[MS_SETS];     // per set of the batch
    unsigned long long scanned[MS_SETS];
    unsigned long long live[MS_SETS];
    unsigned long long blocks;  // Philox blocks drawn for the batch
    unsigned long long visits;  // edge groups staged (one per group of a frontier vertex per level)
    unsigned long long deferred;  // vertex expansions deferred by a level
};

struct MsArgs {
    DevGraph g;
    PhiloxKeys rk;         // round keys of (key0, key1)
    const uint32_t* col4;  // g.col padded to 4*ceil(m/4) entries, 16-byte aligned
    uint32_t key0, key1, epoch;
    const uint32_t* sets;  // [MS_SETS] set ids of the batch (mc->nsets of them)
    uint32_t* vis;         // [n] masks: visited
    uint32_t* nxt;         // [n] masks: reached during this level
    uint32_t* F;           // [n] frontier vertices
    uint32_t* Ff;          // [n] their masks: the sets whose frontier holds them
    uint32_t* pend;        // [n] sets whose expansion of the vertex is deferred (valid where ndef != 0)
    uint32_t* ndef;        // [n/4] one byte per vertex: levels its expansion has been deferred (0: none pending)
    uint32_t defer_groups; // vertices of more edge groups than this may have their expansion deferred
    uint32_t defer_max;    // by at most this many levels (0: never)
    uint4* heavy;          // (vertex, first group, end group, mask) chunks of this level's heavy vertices
    uint32_t heavy_cap;
    MsCounters* mc;
    Counters* ctr;
    SetRec* recs;
    const unsigned long long* rowoff;  // [MS_SETS] bitmap-heap word offset of each dense set's row
    uint32_t* sizes;                   // histogram passes: sizes[j] = |R_j| for j < sizes_cap (or null)
    uint32_t sizes_cap;
};

// roots of the batch, compacted into the first frontier
cudaError_t launch_ms_start(const MsArgs& a, int sms, cudaStream_t s);
// one level: light and heavy expansion, then compaction into the next frontier
// (every kernel returns at once when the frontier is empty, so a fixed run of
// levels can be captured in a CUDA graph)
cudaError_t launch_ms_level(const MsArgs& a, int sms, cudaStream_t s);
constexpr int MS_GRAPH_LEVELS = 8;  // levels per graph launch
// Expansion of a vertex of more than MS_DEFER_GROUPS edge groups (512 in-edges)
// may wait up to MS_DEFER_MAX levels for more sets to reach it.
constexpr uint32_t MS_DEFER_GROUPS = 128;
constexpr uint32_t MS_DEFER_MAX = 2;
// per-set sizes and scanned edges into a.mc
cudaError_t launch_ms_finish(const MsArgs& a, int sms, cudaStream_t s);
// bitmap rows and records of the dense sets; masks cleared
cudaError_t launch_ms_emit(const MsArgs& a, uint32_t dense, uint32_t mode, uint64_t row_words, uint32_t* bm_heap,
                           int sms, cudaStream_t s);

// Philox4x32-10 blocks drawn back to back by `blocks` x 256 threads,
// `per_thread` each (the ALU ceiling of the bit-parallel search); out: one
// word per thread.
cudaError_t launch_philox_ceiling(uint32_t blocks, uint32_t per_thread, uint32_t* out, cudaStream_t s);

// a tile batch (slot s = set 32t + s for the slots in `slots`): the visited
// masks ORed into the tile at word offset tile_off of the bitmap heap, the
// slots' records written; masks cleared
cudaError_t launch_ms_tile(const MsArgs& a, uint32_t slots, uint32_t* bm_heap, uint64_t tile_off,
                           uint64_t new_words, int sms, cudaStream_t s);

// sets of a bit-parallel batch under the density cut, encoded one block each
// (scratch slot b for the b-th listed set)
cudaError_t launch_ms_sparse(const SampleArgs& a, const uint32_t* vis, const uint32_t* sbits, const uint32_t* ids,
                             const MsCounters* mc, uint32_t count, cudaStream_t s);

// ---- selection (select.cu) ----
struct SelState {
    uint32_t u;            // current u*
    uint32_t it;           // iteration
    uint32_t n_cov_huff, n_cov_bm, n_cov_raw, pad;
    unsigned long long gain;     // sets covered by u* this iteration
    unsigned long long covered;  // total covered
    unsigned long long n_dec;    // chunk items of the Huffman sets covered this iteration
    unsigned long long dec_bytes;  // bytes read by the decrement passes (code bytes, copy ids, items, rows)
    unsigned long long t_argmax_ns, t_cover_ns, t_dec_ns;  // persistent selection: phase times (globaltimer)
};

struct SelArgs {
    uint32_t n, n4, T;
    uint32_t j_lo;                         // count passes over uncompressed sets: [j_lo, T)
    const SetRec* recs;
    const uint32_t* raw_heap;
    const uint32_t* code_heap;
    const uint32_t* bm_heap;
    DevCodebook cb;
    uint32_t has_cb;
    uint32_t hot;                          // ranks counted in shared memory
    int32_t* cnt;                          // [n4]; -1 = chosen or padding
    uint8_t* alive;                        // [T]
    const unsigned long long* chunk_items; // (j << 32) | chunk
    unsigned long long n_items;
    const uint32_t* bm_sets;               // bitmap set ids
    uint32_t n_bm;
    SelState* st;
    uint32_t* cov_huff;                    // sets covered this iteration, by kind
    uint32_t* cov_bm;
    uint32_t* cov_raw;
    unsigned long long* dec_items;         // (j << 32) | chunk of covered Huffman sets
    unsigned long long dec_cap;
    unsigned long long* partials;          // argmax per-block results
    unsigned int* ticket;
    uint32_t* seeds;                       // [k]
    unsigned long long* marginal;          // [k]
    int sms;
    long long wait_cycles;                 // bound of every grid-barrier wait
    uint32_t select_mode;                  // 0: decrement; 1: recount every iteration; 2: recount when
                                           // u* covers over half of the live sets (persistent form)
    // Bitmax pools in vertex-major tiles: every set is a column of a tile
    // (tile t at word t * n4w of bm_heap, word v bit s = set 32t + s)
    uint32_t tiles;
    uint64_t n4w;
    uint32_t* tile_live;                   // [ceil(T/32)] live-set masks after the cover (recount)
};

constexpr uint32_t HOT_RANKS = 12288;  // ranks privatised in shared memory by the count kernel

// Launch shapes used by the selection kernels (grids are fixed so that the k
// iterations can be captured in one CUDA graph).
struct SelShape {
    uint32_t count_blocks, argmax_blocks, cover_blocks, dec_blocks;
};
SelShape sel_shape(int sms);

cudaError_t launch_sel_init(const SelArgs& a, cudaStream_t s);
cudaError_t launch_count(const SelArgs& a, uint32_t encode, cudaStream_t s);
// one greedy iteration: argmax, cover test, decrements, finalize
cudaError_t launch_iteration(const SelArgs& a, uint32_t encode, cudaStream_t s);
cudaError_t launch_argmax(const SelArgs& a, cudaStream_t s);

// Grid barrier of the persistent selection (zeroed before each launch).
struct SelBarrier {
    unsigned int count, gen, err, pad;
};
// All k greedy iterations in one cooperative launch (argmax, cover, decrement
// separated by bounded grid barriers); bar->err != 0 afterwards means a
// barrier wait ran out.  select_persistent_blocks: its grid (0: cannot run).
cudaError_t launch_select_persistent(const SelArgs& a, uint32_t k, SelBarrier* bar, cudaStream_t s);
int select_persistent_blocks(int sms);

// ---- pool indexing and inspection (select.cu) ----
struct IndexArgs {
    const SetRec* recs;
    uint32_t j0, j1;
    unsigned long long* chunk_items;
    unsigned long long items_cap;
    uint32_t* bm_sets;
    uint32_t bm_cap;
    Counters* ctr;
    double* moments;  // [3]: sums of |R|, |R|^2, |R|^3
};
cudaError_t launch_index(const IndexArgs& a, cudaStream_t s);

struct DecodeArgs {
    const SetRec* recs;
    const uint32_t* raw_heap;
    const uint32_t* code_heap;
    const uint32_t* bm_heap;
    DevCodebook cb;
    uint32_t has_cb;
    uint32_t n;
    uint32_t j0, j1;
    const unsigned long long* offsets;  // j1-j0+1, into out
    uint32_t* out;
    unsigned long long* ends;           // j1-j0 bit positions after the last code, or null
    Counters* ctr;
    uint32_t tiles;                     // bitmap sets are columns of vertex-major tiles
};
cudaError_t launch_decode(const DecodeArgs& a, cudaStream_t s);

}  // namespace hbx
