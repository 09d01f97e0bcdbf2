// Device-side definitions shared by the sampling and selection kernels.
//
// Layout of an RR pool in HBM (one pool = the sets R_0, R_1, ... of one graph,
// model, seed and epoch; Section 4.2, Algorithm 1 keeps the same per-block
// structures C_i, CP_i, B_i):
//   recs[j]     16-byte record of set j: kind and word offset into the heap of
//               its kind, size, number of coded vertices.
//   code heap   32-bit words.  A Huffman set owns one region of
//               nside + n_raw + ceil(code_bits/32) words: first the side index
//               (nside = (n_coded-1)/32 entries, the bit offset where code 32*c
//               starts, c = 1..), then its copy array CP_j (ids of vertices
//               without a code, ascending), then its code stream.  Stream word i
//               holds stream bits [32i, 32i+32) most-significant first, stored
//               byte-swapped so that memory bytes read as the MSB-first
//               byte-string of Section 4.2.2.
//   bitmap heap 32-bit words: a bitmap set owns ceil(n/32) words rounded up to a
//               multiple of 4 (16-byte aligned rows); bit v = word v/32, bit v%32
//               (Section 4.2.3).
//   raw heap    32-bit vertex ids of the sets of an uncompressed pool, in
//               sampling order.
// Every heap is zero-filled when allocated and written once.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hbx {

constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr uint32_t RAW_FLAG = 0x80000000u;  // sort key of a vertex without a code
constexpr int LUT_BITS = 11;                // first-level Huffman decode table

enum : uint32_t { KIND_HUFF = 0, KIND_BITMAP = 1, KIND_RAW = 2, KIND_PENDING = 3 };
enum : uint32_t { MODE_HIST = 0, MODE_RAW = 1, MODE_ENCODE = 2 };
enum : uint32_t { MODEL_IC = 0, MODEL_LT = 1 };
enum : uint32_t { STREAM_IC = 1, STREAM_LT = 2, STREAM_ROOT = 3 };

struct SetRec {
    uint64_t off_kind;  // kind << 62 | word offset into the heap of that kind
    uint32_t size;
    uint32_t n_coded;
};
static_assert(sizeof(SetRec) == 16, "SetRec is 16 bytes");
constexpr uint64_t OFF_MASK = (1ull << 62) - 1;

__host__ __device__ __forceinline__ uint32_t rec_kind(const SetRec& r) { return (uint32_t)(r.off_kind >> 62); }
__host__ __device__ __forceinline__ uint64_t rec_off(const SetRec& r) { return r.off_kind & OFF_MASK; }
__host__ __device__ __forceinline__ SetRec make_rec(uint32_t kind, uint64_t off, uint32_t size, uint32_t n_coded) {
    SetRec r;
    r.off_kind = ((uint64_t)kind << 62) | off;
    r.size = size;
    r.n_coded = n_coded;
    return r;
}
// side-index entries of a Huffman set with n_coded codes
__host__ __device__ __forceinline__ uint32_t side_words(uint32_t n_coded) { return n_coded ? (n_coded - 1) / 32 : 0; }

struct DevGraph {
    uint32_t n;
    uint32_t m;
    const uint32_t* row_ptr;  // n+1
    const uint32_t* col;      // m
    const uint32_t* thr;      // IC: live threshold ceil(p * 2^24) per edge, 4*ceil(m/4) entries,
                              // 16-byte aligned, zero padded
    const uint32_t* q;        // LT: floor(w * 2^32), capped at 2^32-1
};

struct DevCodebook {
    const uint32_t* rank_of;         // [n], NONE = no code
    const uint32_t* vertex_of_rank;  // [nsym]
    const uint8_t* len_of_rank;      // [nsym]
    const uint32_t* code_of_rank;    // [nsym], right-aligned
    const uint32_t* lut;             // [1 << LUT_BITS]: (rank << 6) | len, len 0 = longer code
    const uint32_t* dec;             // [3 * 33]: first_code[L], count[L], first_rank[L]
    uint32_t nsym;
    uint32_t max_len;
};

// The ten round keys of one Philox key, (k0 + r * 0x9E3779B9, k1 + r *
// 0xBB67AE85) for round r, computed once on the host and passed in the kernel
// arguments: the rounds then read their keys from the constant bank instead
// of adding the Weyl increments in every call.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

__host__ __device__ inline PhiloxKeys philox_round_keys(uint32_t k0, uint32_t k1) {
    PhiloxKeys rk;
    for (int r = 0; r < 10; r++) {
        rk.k0[r] = k0 + (uint32_t)r * 0x9E3779B9u;
        rk.k1[r] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
    return rk;
}

// Device counters of one pool (kept in one allocation).
struct Counters {
    unsigned long long work;         // work-stealing cursor of the warp kernel
    unsigned long long big_work;     // work-stealing cursor of the block kernel
    unsigned long long raw_cursor, code_cursor, bm_cursor;  // heap bump pointers (words)
    unsigned long long big_count, retry_count;
    unsigned long long edges_scanned, edges_live, rr_vertices, code_bits;
    unsigned long long sets_huff, sets_bm, sets_raw, sets_big;
    unsigned long long error;
    unsigned long long chunk_items, bm_list;  // selection indexes
    unsigned long long words_used;            // heap words held by emitted sets
    unsigned long long mid_work;              // work-stealing cursor of the shared-memory block kernel
    unsigned long long giant_count;           // sets too large for shared memory
    // lowest offset of a heap allocation that did not fit (all ones: none); every
    // allocation that fitted ends at or below it, so the host rolls the cursor back
    unsigned long long raw_fail, code_fail, bm_fail;
    // histogram passes: sets at or above the density cut, vertices of the others
    unsigned long long hist_dense, hist_verts;
    unsigned long long uncoded;  // vertices of Huffman sets stored in copy arrays
    unsigned long long pad[4];
};

struct SampleArgs {
    DevGraph g;
    PhiloxKeys rk;            // round keys of (key0, key1)
    uint32_t key0, key1, epoch, model;
    uint32_t mode, cut;
    uint32_t j0, count;       // sets j0 .. j0+count-1, or list[0..count)
    const uint32_t* list;
    uint32_t persistent;      // 1: work stealing over a fixed grid; 0: the plain form
    uint32_t direct;          // block kernel: sample the batch itself, statically assigned
    uint32_t group_budget;    // 4-edge groups a warp may scan for one set before handing it to a block
    uint32_t* freq;           // MODE_HIST: warm-up vertex frequencies [n]
    SetRec* recs;
    uint32_t* raw_heap;
    uint64_t raw_cap;
    uint32_t* code_heap;
    uint64_t code_cap;
    uint32_t* bm_heap;
    uint64_t bm_cap;
    DevCodebook cb;
    uint32_t* big_list;       // sets larger than a warp's capacity
    uint32_t* retry_list;     // sets whose heap space ran out
    uint32_t* giant_list;     // sets larger than a block's shared memory holds
    Counters* ctr;
    // block-per-set scratch, one slot per resident block
    uint32_t* bp_visited;     // slots x bp_words
    uint32_t* bp_rbits;       // slots x bp_words (rank bitmap)
    uint32_t* bp_queue;       // slots x n
    uint32_t* bp_aux;         // slots x bp_words
    uint64_t bp_words;        // ceil(n/32) rounded up to 4
    uint32_t* sizes;          // MODE_HIST: sizes[j] = |R_j| for j < sizes_cap (or null)
    uint32_t sizes_cap;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of the
// 4x32 S-box with the published multipliers and Weyl key increments.
// ---------------------------------------------------------------------------
// Philox4x32 round multipliers
constexpr uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        // one 32 x 32 -> 64-bit product per multiplier gives both halves
        const uint64_t p0 = (uint64_t)PHILOX_M0 * c.x, p1 = (uint64_t)PHILOX_M1 * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Philox4x32-10 with precomputed round keys (the same function as above).
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const PhiloxKeys& rk) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint64_t p0 = (uint64_t)PHILOX_M0 * c.x, p1 = (uint64_t)PHILOX_M1 * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c = make_uint4(hi1 ^ c.y ^ rk.k0[r], lo1, hi0 ^ c.w ^ rk.k1[r], lo0);
    }
    return c;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ void set_error(Counters* c, unsigned long long code) { atomicMax(&c->error, code); }

// IC coin of Section 2.1: edge e is live in sample j when the top 24 bits of
// its Philox word, as a fraction of 2^24 (exact in fp32), fall below p(e).
// With a = x >> 8 an integer and p * 2^24 exact, a * 2^-24 < p holds exactly
// when a < ceil(p * 2^24), the threshold stored per edge at graph upload.
__device__ __forceinline__ bool ic_live(uint32_t x, uint32_t thr) { return (x >> 8) < thr; }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const uint32_t lane = lane_id();
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, d);
        if (lane >= (uint32_t)d) v += t;
    }
    return v;
}

__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long v) {
    const uint32_t lane = lane_id();
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        unsigned long long t = __shfl_up_sync(0xFFFFFFFFu, v, d);
        if (lane >= (uint32_t)d) v += t;
    }
    return v;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, d);
    return v;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xFFFFFFFFu, v, d);
        v = t > v ? t : v;
    }
    return v;
}

__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0, 0x0123); }

// 32 stream bits starting at bit `pos` of a byte-swapped code stream.  May read
// one word past the last code word; every code heap keeps slack words at its end.
__device__ __forceinline__ uint32_t peek32(const uint32_t* __restrict__ words, uint64_t pos) {
    const uint64_t wi = pos >> 5;
    const uint32_t sh = (uint32_t)pos & 31u;
    const uint32_t a = bswap32(__ldg(words + wi));
    if (sh == 0) return a;
    const uint32_t b = bswap32(__ldg(words + wi + 1));
    return (a << sh) | (b >> (32 - sh));
}

// Shared-memory copy of the decode tables.
struct DecodeSmem {
    uint32_t lut[1 << LUT_BITS];
    uint32_t first_code[33];
    uint32_t count[33];
    uint32_t first_rank[33];
};

__device__ __forceinline__ void load_decode_smem(DecodeSmem& s, const DevCodebook& cb) {
    for (uint32_t i = threadIdx.x; i < (1u << LUT_BITS); i += blockDim.x) s.lut[i] = cb.lut[i];
    for (uint32_t i = threadIdx.x; i < 33; i += blockDim.x) {
        s.first_code[i] = cb.dec[i];
        s.count[i] = cb.dec[33 + i];
        s.first_rank[i] = cb.dec[66 + i];
    }
}

// Decode one canonical Huffman code at bit `pos` (advanced past it); returns
// its rank, or NONE for a bit pattern that is no code.
__device__ __forceinline__ uint32_t decode_one(const DecodeSmem& s, const uint32_t* __restrict__ words,
                                               uint64_t& pos) {
    const uint32_t win = peek32(words, pos);
    const uint32_t e = s.lut[win >> (32 - LUT_BITS)];
    uint32_t L = e & 63u;
    if (L) {
        pos += L;
        return e >> 6;
    }
    for (L = LUT_BITS + 1; L <= 32; L++) {
        const uint32_t c = L == 32 ? win : (win >> (32 - L));
        const uint32_t d = c - s.first_code[L];
        if (d < s.count[L]) {
            pos += L;
            return s.first_rank[L] + d;
        }
    }
    return NONE;
}

// The same decoder reading the tables straight from global memory through the
// read-only cache (for kernels that decode only a few codes per block).
__device__ __forceinline__ uint32_t decode_one_g(const DevCodebook& cb, const uint32_t* __restrict__ words,
                                                 uint64_t& pos) {
    const uint32_t win = peek32(words, pos);
    const uint32_t e = __ldg(cb.lut + (win >> (32 - LUT_BITS)));
    uint32_t L = e & 63u;
    if (L) {
        pos += L;
        return e >> 6;
    }
    for (L = LUT_BITS + 1; L <= 32; L++) {
        const uint32_t c = L == 32 ? win : (win >> (32 - L));
        const uint32_t d = c - __ldg(cb.dec + L);
        if (d < __ldg(cb.dec + 33 + L)) {
            pos += L;
            return __ldg(cb.dec + 66 + L) + d;
        }
    }
    return NONE;
}

}  // namespace hbx
