// Greedy max-coverage seed selection on the encoded RR pool (Section 2.2;
// Section 4.3, Algorithms 2 and 3), without materialising decoded sets.
//
// State: cnt[v] = number of uncovered sets holding v (int32; -1 marks a chosen
// vertex and the padding up to a multiple of 4), alive[j] = set j not yet
// covered.  One iteration:
//   argmax     u* = the vertex with the largest cnt, lowest id on ties (an exact
//              reduction; the paper's per-thread "parallel merge" of Section
//              4.3.4 can miss the true maximum and is not used);
//   cover      every alive set holding u* is marked covered: Huffman sets decode
//              only until a rank >= rank(u*) (codes are in ascending rank, and a
//              side index of chunk offsets allows a binary search), or search
//              their sorted copy array; bitmaps test one bit (Algorithm 3's
//              row of u*);
//   decrement  the covered sets' vertices lose one count: Huffman sets are
//              decoded in 32-code chunks, bitmaps are summed per vertex with
//              bit-plane counters (the SUBTRACT + POPCOUNT of Eq. (3));
//   finalize   record u*, its marginal gain, and mark it chosen.
// Counts are exact integers (the paper's float table is not needed).
#include "common.cuh"
#include "internal.h"

namespace hbx {

constexpr int SEL_THREADS = 256;
constexpr int COUNT_THREADS = 512;
constexpr uint32_t BM_BATCH = 255;  // bitmap sets per bit-plane flush

SelShape sel_shape(int sms) {
    SelShape s;
    s.count_blocks = (uint32_t)sms * 2;
    s.argmax_blocks = (uint32_t)sms * 2;
    s.cover_blocks = (uint32_t)sms * 4;
    s.dec_blocks = (uint32_t)sms * 4;
    return s;
}

// Pointers into a Huffman set's region: side index, copy array, code stream.
struct HuffView {
    const uint32_t* side;
    const uint32_t* raw;
    const uint32_t* words;
    uint32_t n_coded, n_raw;
};

__device__ __forceinline__ HuffView huff_view(const uint32_t* code_heap, const SetRec& rec) {
    HuffView h;
    const uint64_t off = rec_off(rec);
    const uint32_t nside = side_words(rec.n_coded);
    h.n_coded = rec.n_coded;
    h.n_raw = rec.size - rec.n_coded;
    h.side = code_heap + off;
    h.raw = code_heap + off + nside;
    h.words = code_heap + off + nside + h.n_raw;
    return h;
}

__global__ void sel_init_kernel(SelArgs a) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < a.n4; v += stride) a.cnt[v] = v < a.n ? 0 : -1;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < a.T; j += stride) a.alive[j] = j >= a.j_lo;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        SelState z;
        z.u = NONE; z.it = 0; z.n_cov_huff = 0; z.n_cov_bm = 0; z.n_cov_raw = 0; z.pad = 0; z.gain = 0; z.covered = 0;
        z.n_dec = 0; z.dec_bytes = 0; z.t_argmax_ns = 0; z.t_cover_ns = 0; z.t_dec_ns = 0;
        *a.st = z;
        *a.ticket = 0;
    }
}

// ---------------------------------------------------------------------------
// Count (sign +1, over every chunk of the pool) or decrement (sign -1, over the
// chunks of the sets covered this iteration): one thread decodes one 32-code
// chunk (or reads 32 copy-array ids).  Hot ranks go to a shared-memory
// histogram, the rest to cnt, with one atomic per group of lanes hitting the
// same counter.  The item count comes from the device (n_dev) or the host.
// ---------------------------------------------------------------------------

// Chunk c of Huffman set j, one per lane of the calling warp (all lanes call
// it; valid = false: no chunk): its 32 codes (or 32 copy-array ids) are
// decoded and each vertex's count moves by `sign` -- hot ranks in the block's
// shared histogram, the rest in cnt, one atomic per group of lanes that hit
// the same counter.  alive_only (recount) skips sets not alive; sets outside
// [j_lo, T) are skipped.
__device__ __forceinline__ void count_chunk_warp(const SelArgs& a, const DecodeSmem& ds, uint32_t* hist, uint32_t hot,
                                                 bool valid, uint32_t j, uint32_t c, int sign,
                                                 const uint8_t* alive_only = nullptr) {
    const uint32_t lane = threadIdx.x & 31;
    uint32_t ncodes = 0, is_code = 0;
    uint64_t pos = 0, pos0 = 0;
    const uint32_t* words = nullptr;
    const uint32_t* raw = nullptr;
    if (valid && j < a.T && j >= a.j_lo && (!alive_only || __ldcg(alive_only + j))) {
        const HuffView h = huff_view(a.code_heap, a.recs[j]);
        const uint32_t nch = (h.n_coded + 31) / 32;
        if (c < nch) {
            words = h.words;
            pos = c ? h.side[c - 1] : 0u;
            pos0 = pos;
            ncodes = min(32u, h.n_coded - 32 * c);
            is_code = 1;
        } else {
            const uint32_t rc = c - nch;
            raw = h.raw + 32ull * rc;
            ncodes = min(32u, h.n_raw - 32 * rc);
        }
    }
    for (uint32_t i = 0; i < 32; i++) {
        const bool have = i < ncodes;
        uint32_t target = NONE;
        if (have) {
            if (is_code) {
                const uint32_t r = decode_one(ds, words, pos);
                if (r == NONE) atomicMax(&a.st->pad, 1u);
                else target = r < hot ? r : (RAW_FLAG | __ldg(a.cb.vertex_of_rank + r));
            } else {
                target = RAW_FLAG | __ldg(raw + i);
            }
        }
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, target);
        if (have && target != NONE && lane == (uint32_t)(__ffs(peers) - 1)) {
            const uint32_t n = __popc(peers);
            if (target & RAW_FLAG) atomicAdd(&a.cnt[target & ~RAW_FLAG], sign * (int)n);
            else atomicAdd(&hist[target], n);
        }
        if (__all_sync(0xFFFFFFFFu, i + 1 >= ncodes)) break;
    }
    if (sign < 0) {
        // bytes this decrement read: the chunk item, its code bits (with the
        // side entry) or copy-array ids
        uint32_t by = 0;
        if (ncodes) by = 8u + (is_code ? (uint32_t)((pos - pos0 + 7) / 8) + 4u : 4u * ncodes);
        by = warp_sum(by);
        if (lane == 0 && by) atomicAdd(&a.st->dec_bytes, (unsigned long long)by);
    }
}

// Items [wb, wb + 32) of `items` ((j << 32) | chunk), one per lane of the
// calling warp (all lanes call it).  Items are read through L2: decrement
// lists are written by other blocks of the same persistent launch.
__device__ __forceinline__ void count_items_warp(const SelArgs& a, const DecodeSmem& ds, uint32_t* hist, uint32_t hot,
                                                 const unsigned long long* items, unsigned long long n_items,
                                                 unsigned long long wb, int sign,
                                                 const uint8_t* alive_only = nullptr) {
    const unsigned long long t = wb + (threadIdx.x & 31);
    unsigned long long item = 0;
    if (t < n_items) item = __ldcg(items + t);
    count_chunk_warp(a, ds, hist, hot, t < n_items, (uint32_t)(item >> 32), (uint32_t)item, sign, alive_only);
}

__global__ void __launch_bounds__(COUNT_THREADS) count_items_kernel(SelArgs a, const unsigned long long* items,
                                                                   const unsigned long long* n_dev,
                                                                   unsigned long long n_host, int sign) {
    extern __shared__ __align__(16) uint32_t smem[];
    const unsigned long long n_items = n_dev ? *n_dev : n_host;
    if ((unsigned long long)blockIdx.x * blockDim.x >= n_items) return;  // no item for this block
    DecodeSmem& ds = *reinterpret_cast<DecodeSmem*>(smem);
    uint32_t* hist = smem + sizeof(DecodeSmem) / 4;
    load_decode_smem(ds, a.cb);
    for (uint32_t i = threadIdx.x; i < a.hot; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long wb = (unsigned long long)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
         wb < n_items; wb += nwarps * 32)
        count_items_warp(a, ds, hist, a.hot, items, n_items, wb, sign);
    __syncthreads();
    for (uint32_t r = threadIdx.x; r < a.hot; r += blockDim.x) {
        const uint32_t h = hist[r];
        if (h) atomicAdd(&a.cnt[__ldg(a.cb.vertex_of_rank + r)], sign * (int)h);
    }
}

// Carry-save adder: the bitwise sum of a, b, c is sum + 2 * carry.
__device__ __forceinline__ void csa(uint32_t& carry, uint32_t& sum, uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t u = a ^ b;
    carry = (a & b) | (u & c);
    sum = u ^ c;
}

// Bit-sliced counter of up to 255 rows for the 32 bits of one word: planes of
// weight 1, 2, 4 and 8, 16, 32, 64, 128 (Harley-Seal: eight rows pass through a
// tree of seven carry-save adders, and only the weight-8 carry ripples on).
struct Planes {
    uint32_t ones = 0, twos = 0, fours = 0, h[5] = {0, 0, 0, 0, 0};
    __device__ __forceinline__ void add8(const uint32_t* w) {
        uint32_t twosA, twosB, foursA, foursB, eights;
        csa(twosA, ones, ones, w[0], w[1]);
        csa(twosB, ones, ones, w[2], w[3]);
        csa(foursA, twos, twos, twosA, twosB);
        csa(twosA, ones, ones, w[4], w[5]);
        csa(twosB, ones, ones, w[6], w[7]);
        csa(foursB, twos, twos, twosA, twosB);
        csa(eights, fours, fours, foursA, foursB);
        uint32_t c = eights;
#pragma unroll
        for (int i = 0; i < 5; i++) {
            const uint32_t t = h[i] & c;
            h[i] ^= c;
            c = t;
        }
    }
    __device__ __forceinline__ uint32_t any() const { return ones | twos | fours | h[0] | h[1] | h[2] | h[3] | h[4]; }
    __device__ __forceinline__ uint32_t count(uint32_t bit) const {
        uint32_t hi = 0;
#pragma unroll
        for (int i = 4; i >= 0; i--) hi = (hi << 1) | ((h[i] >> bit) & 1u);
        return ((ones >> bit) & 1u) + 2u * ((twos >> bit) & 1u) + 4u * ((fours >> bit) & 1u) + 8u * hi;
    }
};

// Per-vertex sums over bitmap rows.  A tile is (batch of up to 255 listed sets,
// blockDim.x x 4 consecutive words): the block stages the batch's row offsets
// in shared memory, each thread streams its 16 bytes of every row (eight rows
// in flight) into bit-sliced counters, then adds sign * count to cnt[32w + bit]
// for every bit with a nonzero count.  Rows are padded to a multiple of 4 words
// and 16-byte aligned.  All threads of the block call it with the same tile.
__device__ __forceinline__ void bitmap_tile(const SelArgs& a, const uint32_t* list, uint32_t len, uint64_t tile,
                                            int sign, unsigned long long* s_off, uint32_t* s_n,
                                            const uint8_t* alive_only = nullptr) {
    const uint32_t nw = (a.n + 31) / 32;
    const uint32_t nq = (nw + 3) / 4;  // 16-byte quads per row
    const uint32_t nchunk = (nq + blockDim.x - 1) / blockDim.x;
    const uint32_t b = (uint32_t)(tile / nchunk), ch = (uint32_t)(tile % nchunk);
    __syncthreads();  // the previous tile is done with s_off
    if (threadIdx.x == 0) *s_n = 0;
    __syncthreads();
    const uint32_t s0 = b * BM_BATCH, s1 = min(len, s0 + BM_BATCH);
    for (uint32_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
        const uint32_t j = __ldcg(list + i);
        if (j < a.T && j >= a.j_lo && (!alive_only || __ldcg(alive_only + j))) s_off[atomicAdd(s_n, 1u)] = rec_off(a.recs[j]);
    }
    __syncthreads();
    const uint32_t rows = *s_n;
    const uint32_t q = ch * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    Planes pl[4];
    for (uint32_t r0 = 0; r0 < rows; r0 += 8) {
        uint32_t w[4][8];
#pragma unroll
        for (int r = 0; r < 8; r++) {
            uint4 x = make_uint4(0, 0, 0, 0);
            if (r0 + r < rows) x = __ldg(reinterpret_cast<const uint4*>(a.bm_heap + s_off[r0 + r]) + q);
            w[0][r] = x.x;
            w[1][r] = x.y;
            w[2][r] = x.z;
            w[3][r] = x.w;
        }
#pragma unroll
        for (int c = 0; c < 4; c++) pl[c].add8(w[c]);
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
        uint32_t any = pl[c].any();
        const uint32_t wbase = (q * 4 + c) * 32;
        while (any) {
            const uint32_t bit = __ffs(any) - 1;
            any &= any - 1;
            const uint32_t v = wbase + bit;
            if (v < a.n) atomicAdd(&a.cnt[v], sign * (int)pl[c].count(bit));
        }
    }
}

__device__ __forceinline__ uint64_t bitmap_tiles(const SelArgs& a, uint32_t len) {
    const uint32_t nq = ((a.n + 31) / 32 + 3) / 4;
    const uint32_t nchunk = (nq + blockDim.x - 1) / blockDim.x;
    return (uint64_t)((len + BM_BATCH - 1) / BM_BATCH) * nchunk;
}

__global__ void __launch_bounds__(SEL_THREADS) bitmap_count_kernel(SelArgs a, const uint32_t* list,
                                                                  const uint32_t* list_len_dev,
                                                                  uint32_t list_len_host, int sign) {
    __shared__ unsigned long long s_off[BM_BATCH];
    __shared__ uint32_t s_n;
    const uint32_t len = list_len_dev ? *list_len_dev : list_len_host;
    const uint64_t tiles = bitmap_tiles(a, len);
    for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) bitmap_tile(a, list, len, tile, sign, s_off, &s_n);
}

// Vertex-major tiles (Bitmax pools): cnt[v] += sum over the tiles of sets
// [j_lo, T) of POPCOUNT(word v under the mask of those sets' columns).  One
// thread owns four consecutive vertices, so no atomics are needed.
__global__ void __launch_bounds__(SEL_THREADS) tile_count_kernel(SelArgs a, uint32_t j_lo) {
    const uint32_t nq = (a.n + 3) / 4;
    const uint32_t t0 = j_lo / 32, t1 = (a.T + 31) / 32;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
        for (uint32_t t = t0; t < t1; t++) {
            const uint32_t lo = max(j_lo, 32 * t), hi = min(a.T, 32 * t + 32);
            const uint32_t cm = (hi - lo == 32) ? 0xFFFFFFFFu : (((1u << (hi - lo)) - 1u) << (lo - 32 * t));
            const uint4 w = __ldg(reinterpret_cast<const uint4*>(a.bm_heap + (uint64_t)t * a.n4w) + q);
            c0 += __popc(w.x & cm);
            c1 += __popc(w.y & cm);
            c2 += __popc(w.z & cm);
            c3 += __popc(w.w & cm);
        }
        int4* c4 = reinterpret_cast<int4*>(a.cnt) + q;
        int4 c = *c4;
        c.x += (int)c0;
        c.y += (int)c1;
        c.z += (int)c2;
        c.w += (int)c3;
        *c4 = c;
    }
}

// Uncompressed pools: one warp per set.
__global__ void count_raw_kernel(SelArgs a) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t j = a.j_lo + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < a.T; j += nwarps) {
        const SetRec rec = a.recs[j];
        const uint32_t* x = a.raw_heap + rec_off(rec);
        for (uint32_t i = lane; i < rec.size; i += 32) atomicAdd(&a.cnt[x[i]], 1);
    }
}

// ---------------------------------------------------------------------------
// argmax: key = (cnt + 1) << 32 | (2^32 - 1 - v); the largest key is the
// largest count with the lowest id.  Chosen vertices (cnt = -1) get key high
// word 0 and never win while an unchosen vertex exists.  The last block to
// finish reduces the per-block results.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SEL_THREADS) argmax_kernel(SelArgs a) {
    __shared__ unsigned long long s_w[SEL_THREADS / 32];
    __shared__ bool s_last;
    unsigned long long best = 0;
    const uint32_t n4q = a.n4 / 4;
    const int4* c4 = reinterpret_cast<const int4*>(a.cnt);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n4q; i += gridDim.x * blockDim.x) {
        const int4 c = c4[i];
        const uint32_t v = i * 4;
        unsigned long long k0 = ((unsigned long long)(uint32_t)(c.x + 1) << 32) | (0xFFFFFFFFu - v);
        unsigned long long k1 = ((unsigned long long)(uint32_t)(c.y + 1) << 32) | (0xFFFFFFFFu - (v + 1));
        unsigned long long k2 = ((unsigned long long)(uint32_t)(c.z + 1) << 32) | (0xFFFFFFFFu - (v + 2));
        unsigned long long k3 = ((unsigned long long)(uint32_t)(c.w + 1) << 32) | (0xFFFFFFFFu - (v + 3));
        k0 = k0 > k1 ? k0 : k1;
        k2 = k2 > k3 ? k2 : k3;
        k0 = k0 > k2 ? k0 : k2;
        best = best > k0 ? best : k0;
    }
    best = warp_max_u64(best);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned long long x = threadIdx.x < SEL_THREADS / 32 ? s_w[threadIdx.x] : 0ull;
        x = warp_max_u64(x);
        if (threadIdx.x == 0) {
            a.partials[blockIdx.x] = x;
            __threadfence();
            const unsigned int t = atomicAdd(a.ticket, 1u);
            s_last = (t == gridDim.x - 1);
        }
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    unsigned long long x = 0;
    for (uint32_t i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
        const unsigned long long y = __ldcg(a.partials + i);
        x = x > y ? x : y;
    }
    x = warp_max_u64(x);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = 0;
        for (int i = 0; i < SEL_THREADS / 32; i++) m = m > s_w[i] ? m : s_w[i];
        const uint32_t u = 0xFFFFFFFFu - (uint32_t)m;
        a.st->u = u;
        a.seeds[a.st->it] = u;
        *a.ticket = 0;
    }
}

// Membership of rank ru in a Huffman set: binary search on the first code of
// each 32-code chunk, then a scan of one chunk, stopping at the first rank >= ru.
__device__ bool huff_contains(const DevCodebook& cb, const HuffView& h, uint32_t ru) {
    const uint32_t n = h.n_coded;
    if (n == 0) return false;
    const uint32_t nside = side_words(n);
    uint32_t lo = 0, hi = nside;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        uint64_t pos = __ldg(h.side + mid - 1);
        const uint32_t r = decode_one_g(cb, h.words, pos);
        if (r <= ru) lo = mid;
        else hi = mid - 1;
    }
    uint64_t pos = lo ? __ldg(h.side + lo - 1) : 0u;
    const uint32_t cnt = min(32u, n - 32 * lo);
    for (uint32_t i = 0; i < cnt; i++) {
        const uint32_t r = decode_one_g(cb, h.words, pos);
        if (r >= ru) return r == ru;
    }
    return false;
}

__device__ bool sorted_contains(const uint32_t* __restrict__ x, uint32_t len, uint32_t u) {
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint32_t y = __ldg(x + mid);
        if (y < u) lo = mid + 1;
        else hi = mid;
    }
    return lo < len && __ldg(x + lo) == u;
}

// Cover test of sets [jb, jb + 32), one per lane of the calling warp (all lanes
// call it): every alive set holding u is marked covered and appended to the
// covered list of its kind; covered Huffman sets also list their chunk items
// for the decrement pass.  Returns the lane's gain (0 or 1).
__device__ __forceinline__ uint32_t cover_warp(const SelArgs& a, uint32_t u, uint32_t ru, uint32_t jb) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t j = jb + lane;
    bool member = false;
    uint32_t kind = KIND_PENDING, nit = 0;
    if (j < a.T && __ldcg(a.alive + j)) {
        const SetRec rec = a.recs[j];
        kind = rec_kind(rec);
        nit = (rec.n_coded + 31) / 32 + (rec.size - rec.n_coded + 31) / 32;
        if (kind == KIND_HUFF) {
            const HuffView h = huff_view(a.code_heap, rec);
            if (ru != NONE) member = huff_contains(a.cb, h, ru);
            else member = sorted_contains(h.raw, h.n_raw, u);
        } else if (kind == KIND_BITMAP) {
            member = (__ldg(a.bm_heap + rec_off(rec) + (u >> 5)) >> (u & 31)) & 1u;
        } else {
            const uint32_t* x = a.raw_heap + rec_off(rec);
            for (uint32_t i = 0; i < rec.size && !member; i++) member = __ldg(x + i) == u;
        }
        if (member) a.alive[j] = 0;
    }
    // one list append per warp and kind
#pragma unroll
    for (uint32_t k = 0; k < 3; k++) {
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, member && kind == k);
        if (!bal) continue;
        uint32_t* list = k == KIND_HUFF ? a.cov_huff : (k == KIND_BITMAP ? a.cov_bm : a.cov_raw);
        uint32_t* len = k == KIND_HUFF ? &a.st->n_cov_huff : (k == KIND_BITMAP ? &a.st->n_cov_bm : &a.st->n_cov_raw);
        const uint32_t leader = __ffs(bal) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(len, (uint32_t)__popc(bal));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        if (member && kind == k) list[base + __popc(bal & lanemask_lt())] = j;
    }
    // chunk items of the covered Huffman sets, for the decrement pass
    if (!(member && kind == KIND_HUFF)) nit = 0;
    const uint32_t incl = warp_incl_scan(nit);
    const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (tot) {
        unsigned long long base = 0;
        if (lane == 31) base = atomicAdd(&a.st->n_dec, (unsigned long long)tot);
        base = __shfl_sync(0xFFFFFFFFu, base, 31);
        const unsigned long long my = base + incl - nit;
        if (my + nit <= a.dec_cap) {
            for (uint32_t c = 0; c < nit; c++) a.dec_items[my + c] = ((unsigned long long)j << 32) | c;
        } else if (nit) {
            atomicMax(&a.st->pad, 2u);
        }
    }
    return member ? 1u : 0u;
}

// The persistent form's cover of sets [jb, jb + 32), one per lane (all lanes
// call it): every alive set holding u is marked covered and its vertices lose
// one count right away -- a covered Huffman set's chunks are spread over the
// warp's lanes, a covered uncompressed set is walked by the whole warp --
// while covered bitmap rows are listed for the bit-plane pass.  Returns the
// lane's gain (0 or 1).
__device__ __forceinline__ uint32_t cover_dec_warp(const SelArgs& a, const DecodeSmem& ds, uint32_t* hist,
                                                   uint32_t hot, uint32_t u, uint32_t ru, uint32_t jb) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t j = jb + lane;
    bool member = false;
    uint32_t kind = KIND_PENDING, nit = 0, size = 0;
    uint64_t off = 0;
    if (j < a.T && __ldcg(a.alive + j)) {
        const SetRec rec = a.recs[j];
        kind = rec_kind(rec);
        size = rec.size;
        off = rec_off(rec);
        nit = (rec.n_coded + 31) / 32 + (rec.size - rec.n_coded + 31) / 32;
        if (kind == KIND_HUFF) {
            const HuffView h = huff_view(a.code_heap, rec);
            if (ru != NONE) member = huff_contains(a.cb, h, ru);
            else member = sorted_contains(h.raw, h.n_raw, u);
        } else if (kind == KIND_BITMAP) {
            member = (__ldg(a.bm_heap + off + (u >> 5)) >> (u & 31)) & 1u;
        } else {
            const uint32_t* x = a.raw_heap + off;
            for (uint32_t i = 0; i < rec.size && !member; i++) member = __ldg(x + i) == u;
        }
        if (member) a.alive[j] = 0;
    }
    // covered bitmap rows: one list append per warp
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, member && kind == KIND_BITMAP);
    if (bal) {
        const uint32_t leader = __ffs(bal) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&a.st->n_cov_bm, (uint32_t)__popc(bal));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        if (member && kind == KIND_BITMAP) a.cov_bm[base + __popc(bal & lanemask_lt())] = j;
    }
    // covered Huffman sets: their chunks over the lanes
    const uint32_t mine = (member && kind == KIND_HUFF) ? nit : 0u;
    const uint32_t incl = warp_incl_scan(mine);
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t t = base + lane;
        // owner lane of task t: the first lane whose inclusive count exceeds t
        uint32_t lo = 0;
#pragma unroll
        for (uint32_t step = 16; step; step >>= 1) {
            const uint32_t s = __shfl_sync(0xFFFFFFFFu, incl, lo + step - 1);
            if (s <= t) lo += step;
        }
        const uint32_t oj = __shfl_sync(0xFFFFFFFFu, j, lo);
        const uint32_t oex = __shfl_sync(0xFFFFFFFFu, incl - mine, lo);
        count_chunk_warp(a, ds, hist, hot, t < total, oj, t - oex, -1);
    }
    // covered uncompressed sets: the warp walks each one
    uint32_t rb = __ballot_sync(0xFFFFFFFFu, member && kind == KIND_RAW);
    while (rb) {
        const uint32_t l = __ffs(rb) - 1;
        rb &= rb - 1;
        const uint64_t o = __shfl_sync(0xFFFFFFFFu, off, l);
        const uint32_t sz = __shfl_sync(0xFFFFFFFFu, size, l);
        for (uint32_t q = lane; q < sz; q += 32) atomicAdd(&a.cnt[__ldg(a.raw_heap + o + q)], -1);
    }
    return member ? 1u : 0u;
}

__global__ void __launch_bounds__(SEL_THREADS) cover_kernel(SelArgs a) {
    const uint32_t u = a.st->u;
    const uint32_t ru = a.has_cb ? __ldg(a.cb.rank_of + u) : NONE;
    uint32_t gain = 0;
    // warp-uniform loop: every lane reaches the ballots in cover_warp
    for (uint32_t jb = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); jb < a.T; jb += gridDim.x * blockDim.x)
        gain += cover_warp(a, u, ru, jb);
    gain = warp_sum(gain);
    if ((threadIdx.x & 31) == 0 && gain) atomicAdd(&a.st->gain, (unsigned long long)gain);
}

__global__ void __launch_bounds__(SEL_THREADS) dec_raw_kernel(SelArgs a) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    const uint32_t len = a.st->n_cov_raw;
    for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < len; i += nwarps) {
        const SetRec rec = a.recs[a.cov_raw[i]];
        const uint32_t* x = a.raw_heap + rec_off(rec);
        for (uint32_t k = lane; k < rec.size; k += 32) atomicAdd(&a.cnt[__ldg(x + k)], -1);
    }
}

__global__ void finalize_kernel(SelArgs a) {
    SelState s = *a.st;
    s.dec_bytes += 4ull * s.n_cov_bm * (((a.n + 31) / 32 + 3) & ~3u);
    a.cnt[s.u] = -1;
    a.marginal[s.it] = s.gain;
    s.covered += s.gain;
    s.gain = 0;
    s.it++;
    s.n_cov_huff = 0;
    s.n_cov_bm = 0;
    s.n_cov_raw = 0;
    s.n_dec = 0;
    *a.st = s;
}

// ---------------------------------------------------------------------------
// Persistent selection: all k greedy iterations in one cooperative launch
// whose blocks are all resident.  An iteration is three phases separated by
// grid barriers:
//   A  argmax: per-block maxima of the count keys, then every block reduces
//      the per-block results itself, so all blocks know u* without another
//      barrier (the previous u*, whose count is zero by now, is excluded and
//      marked chosen with -1 here);
//   B  cover: every alive set holding u* is covered and listed (cover_warp);
//   C  decrement: the covered sets' Huffman chunks (hot ranks through a small
//      shared-memory histogram), bitmap rows (bit-plane sums) and raw sets
//      lose one count per vertex; block 0 records u* and its gain.
// Data written by other blocks of the launch (counts, alive flags, lists,
// per-iteration counters) is read through L2 (__ldcg / atomics).  Every
// barrier wait is bounded by a clock64 budget: a block that runs out sets the
// error word, and every block leaves at its next barrier, so the launch ends
// and the host reports a timeout.
// ---------------------------------------------------------------------------
constexpr int PS_THREADS = 512;
constexpr uint32_t PS_HOT = 2048;                    // ranks counted in shared memory by phase C
__device__ __forceinline__ bool grid_barrier(SelBarrier* b, uint32_t nblocks, long long budget, bool* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = true;
        volatile unsigned int* gen = &b->gen;
        volatile unsigned int* err = &b->err;
        const unsigned int g = *gen;
        __threadfence();
        if (atomicAdd(&b->count, 1u) == nblocks - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (*err) {
                    ok = false;
                    break;
                }
                if (clock64() - t0 > budget) {
                    atomicExch(&b->err, 1u);
                    ok = false;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        *s_ok = ok && *err == 0;
    }
    __syncthreads();
    return *s_ok;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(PS_THREADS) select_persistent_kernel(SelArgs a, uint32_t k, SelBarrier* bar) {
    __shared__ DecodeSmem ds;
    __shared__ uint32_t hist[PS_HOT];
    __shared__ unsigned long long s_off[BM_BATCH];
    __shared__ unsigned long long s_w[PS_THREADS / 32];
    __shared__ uint32_t s_n, s_u;
    __shared__ int s_cu;  // count of u* (the live sets it covers)
    __shared__ bool s_ok;
    const uint32_t nb = gridDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t hot = min(a.hot, PS_HOT);
    if (a.has_cb) load_decode_smem(ds, a.cb);
    __syncthreads();
    uint32_t u_prev = NONE;
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;  // block 0 times the phases, barrier to barrier
    unsigned long long t_a = 0, t_b = 0, t_c = 0, t_prev = timer ? globaltimer_ns() : 0ull;
    for (uint32_t it = 0; it < k; it++) {
        // ---- A: argmax (key = (cnt + 1) << 32 | (2^32 - 1 - v), u_prev excluded)
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (u_prev != NONE) a.cnt[u_prev] = -1;
            a.st->gain = 0;
            a.st->n_cov_huff = 0;
            a.st->n_cov_bm = 0;
            a.st->n_cov_raw = 0;
            a.st->n_dec = 0;
        }
        unsigned long long best = 0;
        const uint32_t n4q = a.n4 / 4;
        for (uint32_t i = blockIdx.x * PS_THREADS + threadIdx.x; i < n4q; i += nb * PS_THREADS) {
            const int4 c = __ldcg(reinterpret_cast<const int4*>(a.cnt) + i);
            const int cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint32_t v = i * 4 + q;
                const unsigned long long key =
                    v == u_prev ? 0ull : (((unsigned long long)(uint32_t)(cv[q] + 1) << 32) | (0xFFFFFFFFu - v));
                best = key > best ? key : best;
            }
        }
        best = warp_max_u64(best);
        if (lane == 0) s_w[warp] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long m = 0;
            for (int w = 0; w < PS_THREADS / 32; w++) m = s_w[w] > m ? s_w[w] : m;
            a.partials[blockIdx.x] = m;
        }
        if (!grid_barrier(bar, nb, a.wait_cycles, &s_ok)) return;
        {
            unsigned long long m = 0;
            for (uint32_t i = threadIdx.x; i < nb; i += PS_THREADS) {
                const unsigned long long y = __ldcg(a.partials + i);
                m = y > m ? y : m;
            }
            m = warp_max_u64(m);
            __syncthreads();  // s_w is reused
            if (lane == 0) s_w[warp] = m;
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned long long r = 0;
                for (int w = 0; w < PS_THREADS / 32; w++) r = s_w[w] > r ? s_w[w] : r;
                s_u = 0xFFFFFFFFu - (uint32_t)r;
                s_cu = (int)(uint32_t)(r >> 32) - 1;
                if (blockIdx.x == 0) {
                    a.seeds[it] = s_u;
                    a.st->u = s_u;
                }
            }
            __syncthreads();
        }
        const uint32_t u = s_u;
        // recount or decrement this iteration: mode 1 always recounts; mode 2
        // (adaptive) recounts when u* covers more than half of the live sets,
        // so that counting the rest from scratch reads less than decrementing
        // the covered ones.  Every block decides alike (same counters, read
        // after the barrier); both forms leave the same counts.
        const unsigned long long live = (unsigned long long)(a.T - a.j_lo) - __ldcg(&a.st->covered);
        const bool recount = a.select_mode == 1 || (a.select_mode == 2 && s_cu > 0 && 2ull * (unsigned)s_cu > live);
        if (timer) {
            const unsigned long long t = globaltimer_ns();
            t_a += t - t_prev;
            t_prev = t;
        }
        // ---- B: cover (the persistent update form also decrements here)
        {
            uint32_t gain = 0;
            if (a.tiles) {
                // a tile's live columns holding u*: bits of word u* under the
                // live mask; the tile and those columns go to the decrement list
                const uint32_t ntiles = (a.T + 31) / 32;
                for (uint32_t t = blockIdx.x * PS_THREADS + threadIdx.x; t < ntiles; t += nb * PS_THREADS) {
                    const uint4* al = reinterpret_cast<const uint4*>(a.alive + 32ull * t);
                    uint32_t am = 0;
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const uint4 x = __ldcg(al + h);
                        const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                        for (int q = 0; q < 4; q++)
#pragma unroll
                            for (int b = 0; b < 4; b++)
                                if ((xs[q] >> (8 * b)) & 0xFFu) am |= 1u << (16 * h + 4 * q + b);
                    }
                    const uint32_t hi = min(32u, a.T - 32 * t);
                    if (hi < 32) am &= (1u << hi) - 1u;
                    const uint32_t m = am & __ldg(a.bm_heap + (uint64_t)t * a.n4w + u);
                    if (m) {
                        for (uint32_t mm = m; mm; mm &= mm - 1) a.alive[32 * t + __ffs(mm) - 1] = 0;
                        gain += __popc(m);
                        const unsigned long long slot = atomicAdd(&a.st->n_dec, 1ull);
                        if (slot < a.dec_cap) a.dec_items[slot] = ((unsigned long long)t << 32) | m;
                        else atomicMax(&a.st->pad, 2u);
                    }
                    if (recount) a.tile_live[t] = am & ~m;
                }
            } else if (recount) {
                const uint32_t ru = a.has_cb ? __ldg(a.cb.rank_of + u) : NONE;
                for (uint32_t jb = (blockIdx.x * PS_THREADS + (threadIdx.x & ~31u)); jb < a.T; jb += nb * PS_THREADS)
                    gain += cover_warp(a, u, ru, jb);
                // recount: this iteration's counts are spent (u* is known)
                for (uint32_t v = blockIdx.x * PS_THREADS + threadIdx.x; v < a.n; v += nb * PS_THREADS)
                    if (__ldcg(a.cnt + v) > 0) a.cnt[v] = 0;
            } else {
                const uint32_t ru = a.has_cb ? __ldg(a.cb.rank_of + u) : NONE;
                for (uint32_t i = threadIdx.x; i < hot; i += PS_THREADS) hist[i] = 0;
                __syncthreads();
                for (uint32_t jb = (blockIdx.x * PS_THREADS + (threadIdx.x & ~31u)); jb < a.T; jb += nb * PS_THREADS)
                    gain += cover_dec_warp(a, ds, hist, hot, u, ru, jb);
                __syncthreads();
                for (uint32_t r = threadIdx.x; r < hot; r += PS_THREADS) {
                    const uint32_t h = hist[r];
                    if (h) atomicAdd(&a.cnt[__ldg(a.cb.vertex_of_rank + r)], -(int)h);
                }
            }
            gain = warp_sum(gain);
            if (lane == 0 && gain) atomicAdd(&a.st->gain, (unsigned long long)gain);
        }
        if (!grid_barrier(bar, nb, a.wait_cycles, &s_ok)) return;
        if (timer) {
            const unsigned long long t = globaltimer_ns();
            t_b += t - t_prev;
            t_prev = t;
            // the iteration's gain is complete
            const unsigned long long g = __ldcg(&a.st->gain);
            a.marginal[it] = g;
            a.st->covered += g;
            a.st->it = it + 1;
        }
        // ---- C: tiles (decrement or recount), recount, or the covered bitmap
        // rows of the update form; skipped when none of these has work (every
        // block reads the same counters after the barrier)
        const uint32_t n_cov_bm = __ldcg(&a.st->n_cov_bm);
        bool phase_c = true;
        if (a.tiles) {
            // one thread owns a vertex: cnt[v] -= POPCOUNT(word v & covered
            // columns) over the covered tiles or, recounting, cnt[v] =
            // POPCOUNT(word v & live columns) over every tile (Eq. (3))
            const unsigned long long n_cov = min(__ldcg(&a.st->n_dec), a.dec_cap);
            const uint32_t ntiles = (a.T + 31) / 32;
            for (uint32_t v = blockIdx.x * PS_THREADS + threadIdx.x; v < a.n; v += nb * PS_THREADS) {
                const int c = __ldcg(a.cnt + v);
                if (c < 0) continue;
                uint32_t acc = 0;
                if (recount) {
                    for (uint32_t t = 0; t < ntiles; t++)
                        acc += __popc(__ldg(a.bm_heap + (uint64_t)t * a.n4w + v) & __ldcg(a.tile_live + t));
                    a.cnt[v] = (int)acc;
                } else {
                    for (unsigned long long i = 0; i < n_cov; i++) {
                        const unsigned long long item = __ldcg(a.dec_items + i);
                        acc += __popc(__ldg(a.bm_heap + (item >> 32) * a.n4w + v) & (uint32_t)item);
                    }
                    if (acc) a.cnt[v] = c - (int)acc;
                }
            }
            if (timer)
                atomicAdd(&a.st->dec_bytes, 4ull * (recount ? (unsigned long long)ntiles : n_cov) * a.n4w);
        } else if (recount) {
            for (uint32_t i = threadIdx.x; i < hot; i += PS_THREADS) hist[i] = 0;
            __syncthreads();
            // every chunk of the sets still live
            if (a.has_cb) {
                const unsigned long long nwarps = (unsigned long long)nb * (PS_THREADS / 32);
                for (unsigned long long wb = (unsigned long long)(blockIdx.x * (PS_THREADS / 32) + warp) * 32;
                     wb < a.n_items; wb += nwarps * 32)
                    count_items_warp(a, ds, hist, hot, a.chunk_items, a.n_items, wb, 1, a.alive);
            }
            __syncthreads();
            for (uint32_t r = threadIdx.x; r < hot; r += PS_THREADS) {
                const uint32_t h = hist[r];
                if (h) atomicAdd(&a.cnt[__ldg(a.cb.vertex_of_rank + r)], (int)h);
            }
            if (a.n_bm) {
                const uint64_t tiles = bitmap_tiles(a, a.n_bm);
                for (uint64_t tile = blockIdx.x; tile < tiles; tile += nb)
                    bitmap_tile(a, a.bm_sets, a.n_bm, tile, 1, s_off, &s_n, a.alive);
            }
            for (uint32_t j = blockIdx.x * (PS_THREADS / 32) + warp; j < a.T; j += nb * (PS_THREADS / 32)) {
                const SetRec rec = a.recs[j];
                if (rec_kind(rec) != KIND_RAW || !__ldcg(a.alive + j)) continue;
                const uint32_t* x = a.raw_heap + rec_off(rec);
                for (uint32_t q = lane; q < rec.size; q += 32) atomicAdd(&a.cnt[__ldg(x + q)], 1);
            }
        } else if (n_cov_bm) {
            const uint64_t tiles = bitmap_tiles(a, n_cov_bm);
            for (uint64_t tile = blockIdx.x; tile < tiles; tile += nb)
                bitmap_tile(a, a.cov_bm, n_cov_bm, tile, -1, s_off, &s_n);
            if (timer) atomicAdd(&a.st->dec_bytes, 4ull * n_cov_bm * (((a.n + 31) / 32 + 3) & ~3u));
        } else {
            phase_c = false;
        }
        if (phase_c) {
            if (!grid_barrier(bar, nb, a.wait_cycles, &s_ok)) return;
            if (timer) {
                const unsigned long long t = globaltimer_ns();
                t_c += t - t_prev;
                t_prev = t;
            }
        }
        u_prev = u;
    }
    if (timer) {
        if (u_prev != NONE) a.cnt[u_prev] = -1;
        a.st->t_argmax_ns += t_a;
        a.st->t_cover_ns += t_b;
        a.st->t_dec_ns += t_c;
    }
}

int select_persistent_blocks(int sms) {
    static int per_sm = -1;
    if (per_sm < 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, select_persistent_kernel, PS_THREADS, 0) !=
            cudaSuccess) {
            cudaGetLastError();
            b = 0;
        }
        per_sm = b > 2 ? 2 : b;
    }
    return per_sm * sms;
}

cudaError_t launch_select_persistent(const SelArgs& a, uint32_t k, SelBarrier* bar, cudaStream_t s) {
    const int blocks = select_persistent_blocks(a.sms);
    if (blocks <= 0) return cudaErrorInvalidConfiguration;
    SelArgs aa = a;
    uint32_t kk = k;
    SelBarrier* bb = bar;
    void* args[] = {&aa, &kk, &bb};
    return cudaLaunchCooperativeKernel((const void*)select_persistent_kernel, dim3((unsigned)blocks),
                                       dim3(PS_THREADS), args, 0, s);
}

cudaError_t launch_sel_init(const SelArgs& a, cudaStream_t s) {
    const uint32_t work = a.n4 > a.T ? a.n4 : a.T;
    uint32_t blocks = (work + SEL_THREADS - 1) / SEL_THREADS;
    const uint32_t cap = (uint32_t)a.sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    sel_init_kernel<<<blocks, SEL_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_count(const SelArgs& a, uint32_t encode, cudaStream_t s) {
    const SelShape sh = sel_shape(a.sms);
    if (!encode) {
        count_raw_kernel<<<sh.count_blocks * 2, SEL_THREADS, 0, s>>>(a);
        return cudaGetLastError();
    }
    if (a.has_cb) {
        // the kernel's largest shared-memory footprint, the same value from every
        // pool and thread (a per-pool value could race with another pool's
        // launch); also covers the decrement launches captured after this
        const size_t smem_max = sizeof(DecodeSmem) + (size_t)HOT_RANKS * 4;
        cudaError_t e =
            cudaFuncSetAttribute(count_items_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
        if (e != cudaSuccess) return e;
    }
    if (a.n_items && a.has_cb) {
        const size_t smem = sizeof(DecodeSmem) + (size_t)a.hot * 4;
        count_items_kernel<<<sh.count_blocks, COUNT_THREADS, smem, s>>>(a, a.chunk_items, nullptr, a.n_items, 1);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (a.tiles) {
        tile_count_kernel<<<sh.count_blocks * 2, SEL_THREADS, 0, s>>>(a, a.j_lo);
        return cudaGetLastError();
    }
    if (a.n_bm) {
        bitmap_count_kernel<<<sh.count_blocks * 2, SEL_THREADS, 0, s>>>(a, a.bm_sets, nullptr, a.n_bm, 1);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

cudaError_t launch_argmax(const SelArgs& a, cudaStream_t s) {
    const SelShape sh = sel_shape(a.sms);
    argmax_kernel<<<sh.argmax_blocks, SEL_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_iteration(const SelArgs& a, uint32_t encode, cudaStream_t s) {
    const SelShape sh = sel_shape(a.sms);
    const uint32_t cover_blocks = min(sh.cover_blocks, (a.T + SEL_THREADS - 1) / SEL_THREADS);
    argmax_kernel<<<sh.argmax_blocks, SEL_THREADS, 0, s>>>(a);
    cover_kernel<<<cover_blocks ? cover_blocks : 1u, SEL_THREADS, 0, s>>>(a);
    if (encode) {
        if (a.has_cb)
            count_items_kernel<<<sh.count_blocks, COUNT_THREADS, sizeof(DecodeSmem) + (size_t)a.hot * 4, s>>>(
                a, a.dec_items, &a.st->n_dec, 0, -1);
        if (a.n_bm) bitmap_count_kernel<<<sh.dec_blocks, SEL_THREADS, 0, s>>>(a, a.cov_bm, &a.st->n_cov_bm, 0, -1);
    } else {
        dec_raw_kernel<<<sh.dec_blocks, SEL_THREADS, 0, s>>>(a);
    }
    finalize_kernel<<<1, 1, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pool indexing after sampling: Huffman sets contribute one work item per 32
// codes or 32 copy-array ids; bitmap sets are listed.  Also the size moments of
// Eq. (2).
// ---------------------------------------------------------------------------
__global__ void index_kernel(IndexArgs a) {
    __shared__ double s_m[3][SEL_THREADS / 32];
    double m1 = 0, m2 = 0, m3 = 0;
    uint32_t uncoded = 0;
    for (uint32_t j = a.j0 + blockIdx.x * blockDim.x + threadIdx.x; j < a.j1; j += gridDim.x * blockDim.x) {
        const SetRec rec = a.recs[j];
        const uint32_t kind = rec_kind(rec);
        if (kind == KIND_PENDING) {
            atomicMax(&a.ctr->error, 3ull);
            continue;
        }
        const double x = (double)rec.size;
        m1 += x;
        m2 += x * x;
        m3 += x * x * x;
        if (kind == KIND_HUFF) {
            uncoded += rec.size - rec.n_coded;
            const uint32_t nch = (rec.n_coded + 31) / 32 + (rec.size - rec.n_coded + 31) / 32;
            const unsigned long long base = atomicAdd(&a.ctr->chunk_items, (unsigned long long)nch);
            if (base + nch > a.items_cap) {
                atomicMax(&a.ctr->error, 4ull);
                continue;
            }
            for (uint32_t c = 0; c < nch; c++) a.chunk_items[base + c] = ((unsigned long long)j << 32) | c;
        } else if (kind == KIND_BITMAP) {
            const unsigned long long b = atomicAdd(&a.ctr->bm_list, 1ull);
            if (b >= a.bm_cap) {
                atomicMax(&a.ctr->error, 4ull);
                continue;
            }
            a.bm_sets[b] = j;
        }
    }
    uncoded = warp_sum(uncoded);
    if ((threadIdx.x & 31) == 0 && uncoded) atomicAdd(&a.ctr->uncoded, (unsigned long long)uncoded);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        m1 += __shfl_xor_sync(0xFFFFFFFFu, m1, d);
        m2 += __shfl_xor_sync(0xFFFFFFFFu, m2, d);
        m3 += __shfl_xor_sync(0xFFFFFFFFu, m3, d);
    }
    if ((threadIdx.x & 31) == 0) {
        s_m[0][threadIdx.x >> 5] = m1;
        s_m[1][threadIdx.x >> 5] = m2;
        s_m[2][threadIdx.x >> 5] = m3;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0;
        for (int i = 0; i < SEL_THREADS / 32; i++) t += s_m[threadIdx.x][i];
        if (t != 0) atomicAdd(&a.moments[threadIdx.x], t);
    }
}

cudaError_t launch_index(const IndexArgs& a, cudaStream_t s) {
    if (a.j1 <= a.j0) return cudaSuccess;
    uint32_t blocks = (a.j1 - a.j0 + SEL_THREADS - 1) / SEL_THREADS;
    if (blocks > 1024) blocks = 1024;
    index_kernel<<<blocks, SEL_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Decode sets [j0, j1) to vertex lists (one warp per set), for inspection.
// Huffman: vertices in rank order then the copy array; bitmap: ascending;
// raw: as stored.  ends[j - j0] receives the bit position after the last code.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SEL_THREADS) decode_kernel(DecodeArgs a) {
    __shared__ DecodeSmem ds;
    if (a.has_cb) load_decode_smem(ds, a.cb);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t j = a.j0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < a.j1; j += nwarps) {
        const SetRec rec = a.recs[j];
        const uint32_t kind = rec_kind(rec);
        uint32_t* out = a.out + a.offsets[j - a.j0];
        if (kind == KIND_HUFF) {
            const HuffView h = huff_view(a.code_heap, rec);
            const uint32_t nch = (h.n_coded + 31) / 32;
            for (uint32_t c = lane; c < nch; c += 32) {
                uint64_t pos = c ? h.side[c - 1] : 0u;
                const uint32_t cnt = min(32u, h.n_coded - 32 * c);
                for (uint32_t k = 0; k < cnt; k++) {
                    const uint32_t r = decode_one(ds, h.words, pos);
                    if (r == NONE) {
                        atomicMax(&a.ctr->error, 5ull);
                        out[32 * c + k] = NONE;
                    } else {
                        out[32 * c + k] = a.cb.vertex_of_rank[r];
                    }
                }
                if (c == nch - 1 && a.ends) a.ends[j - a.j0] = pos;
            }
            if (nch == 0 && lane == 0 && a.ends) a.ends[j - a.j0] = 0;
            for (uint32_t k = lane; k < h.n_raw; k += 32) out[h.n_coded + k] = h.raw[k];
        } else if (kind == KIND_BITMAP) {
            const uint32_t nw = (a.n + 31) / 32;
            const uint32_t* row = a.bm_heap + rec_off(rec);
            uint32_t base = 0;
            for (uint32_t w0 = 0; w0 < nw; w0 += 32) {
                const uint32_t w = w0 + lane;
                uint32_t x = 0;
                if (a.tiles) {
                    // column j % 32 of a vertex-major tile: vertex v is bit j % 32 of word v
                    for (uint32_t b = 0; b < 32; b++) {
                        const uint32_t v = w * 32 + b;
                        if (v < a.n) x |= ((row[v] >> (j & 31)) & 1u) << b;
                    }
                } else if (w < nw) {
                    x = row[w];
                }
                const uint32_t c = __popc(x);
                const uint32_t incl = warp_incl_scan(c);
                uint32_t p = base + incl - c;
                while (x) {
                    const uint32_t b = __ffs(x) - 1;
                    out[p++] = w * 32 + b;
                    x &= x - 1;
                }
                base += __shfl_sync(0xFFFFFFFFu, incl, 31);
            }
        } else if (kind == KIND_RAW) {
            const uint32_t* x = a.raw_heap + rec_off(rec);
            for (uint32_t k = lane; k < rec.size; k += 32) out[k] = x[k];
        } else if (lane == 0) {
            atomicMax(&a.ctr->error, 3ull);
        }
    }
}

cudaError_t launch_decode(const DecodeArgs& a, cudaStream_t s) {
    if (a.j1 <= a.j0) return cudaSuccess;
    uint32_t blocks = (a.j1 - a.j0 + 7) / 8;
    if (blocks > 2048) blocks = 2048;
    decode_kernel<<<blocks, SEL_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace hbx
