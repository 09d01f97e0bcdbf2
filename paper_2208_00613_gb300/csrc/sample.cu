// RR-set sampling fused with encoding (Section 2.2; Section 4.2, Algorithm 1).
//
// One random RR set (Definition 2) is the set of vertices that reach a random
// root through live edges.  Every coin is a Philox draw keyed by (edge or
// vertex id, set id j, epoch, stream), so the set does not depend on the order
// in which the search meets its edges:
//   root   = floor(x * n / 2^32),  x = word 0 of Philox(0, j, epoch, 3)
//   IC     in-edge e is live iff (x >> 8) * 2^-24 < p[e] (exact fp32), i.e.
//          (x >> 8) < ceil(p[e] * 2^24), x = word e%4 of Philox(e/4, j, epoch,
//          1): one draw serves the 4 edges of an aligned group, and a thread
//          handles one group (one uint4 of thresholds)
//   LT     at vertex v, x = word 0 of Philox(v, j, epoch, 2); the walk moves to
//          the source of the first in-edge whose inclusive prefix sum of fixed-
//          point weights exceeds x, and stops when there is none or that source
//          is already in the set.
//
// Kernels:
//   sample_warp_kernel   one warp per set, persistent over the batch (work
//                        stealing).  The set's vertex list (the BFS queue) and a
//                        hash set of visited ids live in shared memory.  A set
//                        that outgrows the warp's capacity QW, or whose frontier
//                        would exceed the warp's edge-group budget, is handed on.
//                        The finished set is encoded by the same warp: a bitmap if
//                        cut*|R| > n, else its vertices are mapped to codebook
//                        ranks, sorted (bitonic), and the codes bit-packed over a
//                        prefix sum of lengths.
//   sample_mid_kernel    one 512-thread block per set handed on by a warp, up to
//                        4096 vertices, everything in shared memory; a single warp
//                        runs ahead while the frontier is thin.  IC sets that
//                        outgrow it go to the bit-parallel search (msbfs.cu) in
//                        encoded pools and histogram passes, the others to the
//                        block kernel.
//   sample_block_kernel  one thread-block cluster (1 to 8 blocks of 512 threads)
//                        per set: level-synchronous BFS whose edge groups are
//                        spread over all blocks of the cluster (a block-wide scan
//                        of group counts per 512 frontier vertices), level barriers
//                        on the cluster barrier, the queue tail in block 0's shared
//                        memory (reached by the others through distributed shared
//                        memory), the visited set as an n-bit bitmap and the queue
//                        in HBM.  The visited bitmap is the bitmap encoding; small
//                        Huffman sets are sorted in shared memory, large ones
//                        through a rank bitmap.  The plain form samples every set
//                        with this kernel.
//   sample_ms_sparse_kernel  encodes a bit-parallel search's sets that fall under
//                        the density cut, one block each, as the block kernel does.
#include <cstdio>

#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace hbx {

constexpr int WP_WARPS = 8;
constexpr int BP_THREADS = 512;
constexpr int BP_WARPS = BP_THREADS / 32;
constexpr int BP_ILP = 4;  // edge groups per thread per step of the block path
constexpr uint32_t WORK_CHUNK = 4;  // sets taken per work-stealing step

struct WarpLocal {
    uint32_t scan[32];
    uint32_t g0[32];
    uint32_t eb[32];
    uint32_t ee[32];
    uint32_t stage[40];
};


// Open-addressing insert into a warp's shared hash set (key v+1, 0 = empty).
// The table holds at most QW + 31 keys in 2*QW slots, so a probe always ends.
__device__ __forceinline__ bool hash_insert(uint32_t* h, uint32_t mask, uint32_t shift, uint32_t v,
                                            Counters* ctr) {
    const uint32_t key = v + 1u;
    uint32_t s = (v * 0x9E3779B1u) >> shift;
    for (uint32_t probe = 0; probe <= mask; probe++) {
        const uint32_t old = atomicCAS(&h[s], 0u, key);
        if (old == 0u) return true;
        if (old == key) return false;
        s = (s + 1u) & mask;
    }
    set_error(ctr, 1);
    return false;
}


// Coins of one aligned 4-edge group gg of set j, restricted to [eb, ee).
// Returns the live mask; adds the in-range edge count to *scanned.
__device__ __forceinline__ uint32_t group_coins(const SampleArgs& a, uint32_t j, uint32_t gg, uint32_t eb,
                                                uint32_t ee, unsigned long long* scanned) {
    const uint4 t4 = __ldg(reinterpret_cast<const uint4*>(a.g.thr) + gg);
    const uint4 x = philox4x32_10_rk(make_uint4(gg, j, a.epoch, STREAM_IC), a.rk);
    const uint32_t e0 = gg * 4u;
    const bool v0 = e0 >= eb && e0 < ee, v1 = e0 + 1 >= eb && e0 + 1 < ee;
    const bool v2 = e0 + 2 >= eb && e0 + 2 < ee, v3 = e0 + 3 >= eb && e0 + 3 < ee;
    *scanned += (uint32_t)v0 + (uint32_t)v1 + (uint32_t)v2 + (uint32_t)v3;
    return (uint32_t)(v0 && ic_live(x.x, t4.x)) | ((uint32_t)(v1 && ic_live(x.y, t4.y)) << 1) |
           ((uint32_t)(v2 && ic_live(x.z, t4.z)) << 2) | ((uint32_t)(v3 && ic_live(x.w, t4.w)) << 3);
}

// Bitonic sort of 32 keys held one per lane (ascending by lane).
__device__ __forceinline__ uint32_t warp_sort32(uint32_t key) {
    const uint32_t lane = lane_id();
#pragma unroll
    for (uint32_t k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (uint32_t jj = k >> 1; jj > 0; jj >>= 1) {
            const uint32_t other = __shfl_xor_sync(0xFFFFFFFFu, key, jj);
            const bool up = (lane & k) == 0;
            const bool lower = (lane & jj) == 0;
            key = (lower == up) ? min(key, other) : max(key, other);
        }
    }
    return key;
}

// Bitonic sort of s[0..P) (P a power of two) by one warp.
__device__ void warp_sort_smem(uint32_t* s, uint32_t P) {
    const uint32_t lane = lane_id();
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t jj = k >> 1; jj > 0; jj >>= 1) {
            for (uint32_t i = lane; i < P; i += 32) {
                const uint32_t ixj = i ^ jj;
                if (ixj > i) {
                    const uint32_t x = s[i], y = s[ixj];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) {
                        s[i] = y;
                        s[ixj] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// Warp path
// ---------------------------------------------------------------------------
struct WarpStats {
    unsigned long long scanned = 0, live = 0, verts = 0, bits = 0, huff = 0, bm = 0, raw = 0, words = 0;
};

// Samples set j into queue[0..tail).  Returns false if it outgrew QW or the
// group budget (then the block kernel takes it).
template <uint32_t QW>
__device__ bool warp_sample(const SampleArgs& a, uint32_t j, uint32_t* queue, uint32_t* hash, WarpLocal& wl,
                            uint32_t& tail_out, WarpStats& st) {
    constexpr uint32_t HMASK = 2 * QW - 1;
    constexpr uint32_t HSHIFT = 32 - __builtin_ctz(2 * QW);
    const uint32_t lane = lane_id();
    const uint4 rr = philox4x32_10(make_uint4(0u, j, a.epoch, STREAM_ROOT), a.key0, a.key1);
    const uint32_t root = __umulhi(rr.x, a.g.n);
    if (lane == 0) {
        hash_insert(hash, HMASK, HSHIFT, root, a.ctr);
        queue[0] = root;
    }
    __syncwarp();
    uint32_t tail = 1;
    bool overflow = false;

    if (a.model == MODEL_IC) {
        uint32_t head = 0, groups_done = 0;
        while (head < tail && !overflow) {
            const uint32_t cnt = min(32u, tail - head);
            uint32_t b = 0, e = 0, ng = 0, gfirst = 0;
            if (lane < cnt) {
                const uint32_t v = queue[head + lane];
                b = __ldg(a.g.row_ptr + v);
                e = __ldg(a.g.row_ptr + v + 1);
                if (e > b) {
                    gfirst = b >> 2;
                    ng = ((e - 1) >> 2) - gfirst + 1;
                }
            }
            const uint32_t incl = warp_incl_scan(ng);
            const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
            groups_done += total;
            if (groups_done > a.group_budget) {
                overflow = true;
                break;
            }
            wl.scan[lane] = incl;
            wl.g0[lane] = gfirst;
            wl.eb[lane] = b;
            wl.ee[lane] = e;
            __syncwarp();
            head += cnt;
            for (uint32_t base = 0; base < total && !overflow; base += 32) {
                const uint32_t t = base + lane;
                uint32_t live_mask = 0, gg = 0;
                if (t < total) {
                    uint32_t lo = 0, hi = cnt - 1;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (wl.scan[mid] > t) hi = mid;
                        else lo = mid + 1;
                    }
                    const uint32_t prev = lo ? wl.scan[lo - 1] : 0u;
                    gg = wl.g0[lo] + (t - prev);
                    live_mask = group_coins(a, j, gg, wl.eb[lo], wl.ee[lo], &st.scanned);
                    st.live += __popc(live_mask);
                }
                uint32_t u[4];
#pragma unroll
                for (int k = 0; k < 4; k++) u[k] = (live_mask >> k & 1u) ? __ldg(a.g.col + gg * 4u + k) : 0u;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    bool isnew = false;
                    if (live_mask >> k & 1u) isnew = hash_insert(hash, HMASK, HSHIFT, u[k], a.ctr);
                    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, isnew);
                    if (bal) {
                        const uint32_t pos = tail + __popc(bal & lanemask_lt());
                        if (isnew && pos < QW) queue[pos] = u[k];
                        tail += __popc(bal);
                        if (tail > QW) {
                            overflow = true;
                            break;
                        }
                    }
                }
                __syncwarp();
            }
        }
    } else {
        uint32_t v = root;
        for (;;) {
            const uint32_t b = __ldg(a.g.row_ptr + v), e = __ldg(a.g.row_ptr + v + 1);
            if (b == e) break;
            const uint32_t x = philox4x32_10(make_uint4(v, j, a.epoch, STREAM_LT), a.key0, a.key1).x;
            unsigned long long Q = 0;
            uint32_t chosen = NONE;
            for (uint32_t base = b; base < e; base += 32) {
                const uint32_t idx = base + lane;
                const uint32_t qi = idx < e ? __ldg(a.g.q + idx) : 0u;
                const unsigned long long incl = warp_incl_scan_u64(qi) + Q;
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, idx < e && (unsigned long long)x < incl);
                if (bal) {
                    chosen = base + __ffs(bal) - 1;
                    break;
                }
                Q = __shfl_sync(0xFFFFFFFFu, incl, 31);
            }
            st.scanned += (chosen == NONE ? e - b : chosen - b + 1) * (lane == 0);
            if (chosen == NONE) break;
            st.live += (lane == 0);
            const uint32_t u = __ldg(a.g.col + chosen);
            uint32_t isnew = 0;
            if (lane == 0) isnew = hash_insert(hash, HMASK, HSHIFT, u, a.ctr);
            isnew = __shfl_sync(0xFFFFFFFFu, isnew, 0);
            if (!isnew) break;
            if (tail >= QW) {
                overflow = true;
                break;
            }
            if (lane == 0) queue[tail] = u;
            tail++;
            v = u;
        }
    }
    __syncwarp();
    tail_out = tail;
    return !overflow;
}

// Store a Huffman set whose keys (rank, or RAW_FLAG|id for the copy array) are
// sorted ascending in keys[0..size): allocate its region, pack the codes 32 at a
// time through `stage` (40 words of shared memory), write the copy array and
// the record.  Called by one whole warp.  Returns false if the code heap is
// full (nothing of the set is written).
__device__ bool warp_huff_store(const SampleArgs& a, uint32_t j, const uint32_t* keys, uint32_t size, uint32_t* stage,
                                WarpStats& st) {
    const uint32_t lane = lane_id();
    uint32_t n_coded = 0, bits = 0;
    for (uint32_t base = 0; base < size; base += 32) {
        const uint32_t i = base + lane;
        const uint32_t key = i < size ? keys[i] : 0xFFFFFFFFu;
        const bool coded = key < RAW_FLAG;
        n_coded += __popc(__ballot_sync(0xFFFFFFFFu, coded));
        bits += warp_sum(coded ? (uint32_t)__ldg(a.cb.len_of_rank + key) : 0u);
    }
    const uint32_t n_raw = size - n_coded;
    const uint32_t nside = side_words(n_coded);
    const unsigned long long words = (unsigned long long)nside + n_raw + (bits + 31) / 32;
    unsigned long long off = 0;
    if (lane == 0) off = words ? atomicAdd(&a.ctr->code_cursor, words) : 0ull;
    off = __shfl_sync(0xFFFFFFFFu, off, 0);
    if (off + words > a.code_cap) {
        if (lane == 0) atomicMin(&a.ctr->code_fail, off);
        return false;
    }

    // pack 32 codes at a time into the stage, write completed words
    uint32_t* out = a.code_heap + off + nside + n_raw;
    uint32_t carry = 0;  // bit offset of the current chunk's first code
    for (uint32_t i = lane; i < 40; i += 32) stage[i] = 0;
    __syncwarp();
    for (uint32_t c = 0; c * 32 < n_coded; c++) {
        const uint32_t i = c * 32 + lane;
        uint32_t L = 0, code = 0;
        if (i < n_coded) {
            const uint32_t r = keys[i];
            L = __ldg(a.cb.len_of_rank + r);
            code = __ldg(a.cb.code_of_rank + r);
        }
        const uint32_t incl = warp_incl_scan(L);
        const uint32_t chunk_bits = __shfl_sync(0xFFFFFFFFu, incl, 31);
        if (c > 0 && lane == 0) a.code_heap[off + c - 1] = carry;
        const uint32_t wbase = carry >> 5;
        const uint32_t lo = (carry & 31u) + incl - L;  // offset within the stage
        if (L) {
            const uint32_t w = lo >> 5, sh = lo & 31u;
            if (sh + L <= 32) {
                atomicOr(&stage[w], code << (32 - sh - L));
            } else {
                atomicOr(&stage[w], code >> (sh + L - 32));
                atomicOr(&stage[w + 1], code << (64 - sh - L));
            }
        }
        __syncwarp();
        const uint32_t end = carry + chunk_bits;
        const uint32_t done = (end >> 5) - wbase;  // complete words in the stage
        for (uint32_t w = lane; w < done; w += 32) out[wbase + w] = bswap32(stage[w]);
        __syncwarp();
        const uint32_t partial = stage[done];
        __syncwarp();
        for (uint32_t w = lane; w < 40; w += 32) stage[w] = 0;
        __syncwarp();
        if (lane == 0) stage[0] = partial;
        __syncwarp();
        carry = end;
    }
    if ((carry & 31u) && lane == 0) out[carry >> 5] = bswap32(stage[0]);
    for (uint32_t i = lane; i < n_raw; i += 32) a.code_heap[off + nside + i] = keys[n_coded + i] & ~RAW_FLAG;
    if (lane == 0) {
        a.recs[j] = make_rec(KIND_HUFF, off, size, n_coded);
        st.verts += size;
        st.bits += bits;
        st.huff += 1;
        st.words += words;
    }
    __syncwarp();
    return true;
}


// Encode a finished set held in queue[0..size) and write its record.
// Returns false if a heap ran out of space (nothing of the set is written).
template <uint32_t QW>
__device__ bool warp_emit(const SampleArgs& a, uint32_t j, uint32_t* queue, uint32_t size, WarpLocal& wl,
                          WarpStats& st) {
    const uint32_t lane = lane_id();
    const uint32_t n = a.g.n;
    if (a.mode == MODE_HIST) {
        const bool dense = (unsigned long long)a.cut * size > n;
        if (!dense)
            for (uint32_t i = lane; i < size; i += 32) atomicAdd(&a.freq[queue[i]], 1u);
        if (lane == 0) {  // sizes of the sampled sets, kept apart from the pool's statistics
            st.bm += dense;
            st.verts += dense ? 0u : size;
            if (a.sizes && j < a.sizes_cap) a.sizes[j] = size;
        }
        return true;
    }
    if (a.mode == MODE_RAW) {
        unsigned long long off = 0;
        if (lane == 0) off = atomicAdd(&a.ctr->raw_cursor, (unsigned long long)size);
        off = __shfl_sync(0xFFFFFFFFu, off, 0);
        if (off + size > a.raw_cap) {
            if (lane == 0) atomicMin(&a.ctr->raw_fail, off);
            return false;
        }
        for (uint32_t i = lane; i < size; i += 32) a.raw_heap[off + i] = queue[i];
        if (lane == 0) {
            a.recs[j] = make_rec(KIND_RAW, off, size, 0);
            st.verts += size;
            st.raw += 1;
            st.words += size;
        }
        return true;
    }
    // MODE_ENCODE
    if ((unsigned long long)a.cut * size > n) {
        const unsigned long long row = (((unsigned long long)n + 31) / 32 + 3) & ~3ull;
        unsigned long long off = 0;
        if (lane == 0) off = atomicAdd(&a.ctr->bm_cursor, row);
        off = __shfl_sync(0xFFFFFFFFu, off, 0);
        if (off + row > a.bm_cap) {
            if (lane == 0) atomicMin(&a.ctr->bm_fail, off);
            return false;
        }
        for (uint32_t i = lane; i < size; i += 32) {
            const uint32_t v = queue[i];
            atomicOr(&a.bm_heap[off + (v >> 5)], 1u << (v & 31));
        }
        if (lane == 0) {
            a.recs[j] = make_rec(KIND_BITMAP, off, size, 0);
            st.verts += size;
            st.bm += 1;
            st.words += row;
        }
        return true;
    }
    // Huffman: keys = rank (coded) or RAW_FLAG|id (copy array), sorted ascending
    for (uint32_t i = lane; i < size; i += 32) {
        const uint32_t v = queue[i];
        const uint32_t r = __ldg(a.cb.rank_of + v);
        queue[i] = (r != NONE) ? r : (RAW_FLAG | v);
    }
    __syncwarp();
    if (size <= 32) {
        uint32_t key = lane < size ? queue[lane] : 0xFFFFFFFFu;
        key = warp_sort32(key);
        if (lane < size) queue[lane] = key;
    } else {
        uint32_t P = 64;
        while (P < size) P <<= 1;
        for (uint32_t i = size + lane; i < P; i += 32) queue[i] = 0xFFFFFFFFu;
        __syncwarp();
        warp_sort_smem(queue, P);
    }
    __syncwarp();
    return warp_huff_store(a, j, queue, size, wl.stage, st);
}

template <uint32_t QW>
__global__ void __launch_bounds__(WP_WARPS * 32) sample_warp_kernel(SampleArgs a) {
    extern __shared__ __align__(16) uint32_t dyn[];
    __shared__ WarpLocal wl_all[WP_WARPS];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* queue = dyn + warp * (3 * QW);
    uint32_t* hash = queue + QW;
    WarpLocal& wl = wl_all[warp];
    for (uint32_t i = lane; i < (2 * QW) / 4; i += 32) reinterpret_cast<uint4*>(hash)[i] = make_uint4(0, 0, 0, 0);
    __syncwarp();
    WarpStats st;

    uint32_t item = 0, item_end = 0;
    for (;;) {
        if (item >= item_end) {
            unsigned long long b = 0;
            if (lane == 0) b = atomicAdd(&a.ctr->work, (unsigned long long)WORK_CHUNK);
            b = __shfl_sync(0xFFFFFFFFu, b, 0);
            if (b >= a.count) break;
            item = (uint32_t)b;
            item_end = (uint32_t)min(b + WORK_CHUNK, (unsigned long long)a.count);
        }
        const uint32_t j = a.list ? a.list[item] : a.j0 + item;
        item++;
        uint32_t size = 0;
        WarpStats local;  // edges of this set, counted once the set is emitted
        const bool fits = warp_sample<QW>(a, j, queue, hash, wl, size, local);
        if (!fits) {
            if (lane == 0) a.big_list[atomicAdd(&a.ctr->big_count, 1ull)] = j;
        } else if (!warp_emit<QW>(a, j, queue, size, wl, st)) {
            if (lane == 0) a.retry_list[atomicAdd(&a.ctr->retry_count, 1ull)] = j;
        } else {
            st.scanned += local.scanned;
            st.live += local.live;
        }
        __syncwarp();
        for (uint32_t i = lane; i < (2 * QW) / 4; i += 32)
            reinterpret_cast<uint4*>(hash)[i] = make_uint4(0, 0, 0, 0);
        __syncwarp();
    }
    unsigned long long sc = st.scanned, lv = st.live;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        sc += __shfl_xor_sync(0xFFFFFFFFu, sc, d);
        lv += __shfl_xor_sync(0xFFFFFFFFu, lv, d);
    }
    if (lane == 0) {
        if (sc) atomicAdd(&a.ctr->edges_scanned, sc);
        if (lv) atomicAdd(&a.ctr->edges_live, lv);
        if (st.verts) atomicAdd(a.mode == MODE_HIST ? &a.ctr->hist_verts : &a.ctr->rr_vertices, st.verts);
        if (st.bits) atomicAdd(&a.ctr->code_bits, st.bits);
        if (st.huff) atomicAdd(&a.ctr->sets_huff, st.huff);
        if (st.bm) atomicAdd(a.mode == MODE_HIST ? &a.ctr->hist_dense : &a.ctr->sets_bm, st.bm);
        if (st.raw) atomicAdd(&a.ctr->sets_raw, st.raw);
        if (st.words) atomicAdd(&a.ctr->words_used, st.words);
    }
}

// ---------------------------------------------------------------------------
// Block path
// ---------------------------------------------------------------------------
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_warp, uint32_t& total) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nw = blockDim.x >> 5;
    const uint32_t incl = warp_incl_scan(v);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t x = lane < nw ? s_warp[lane] : 0u;
        const uint32_t xi = warp_incl_scan(x);
        if (lane < nw) s_warp[lane] = xi - x;
        if (lane == 31) s_warp[32] = xi;
    }
    __syncthreads();
    total = s_warp[32];
    const uint32_t r = s_warp[warp] + incl - v;
    __syncthreads();
    return r;
}

__device__ uint32_t block_sum(uint32_t v, uint32_t* s_warp) {
    uint32_t total;
    block_excl_scan(v, s_warp, total);
    return total;
}

// Write the set bits of words [0, nwords) in ascending order to out[0..),
// zeroing the words; returns the count.  Each thread takes a contiguous range.
__device__ uint32_t compact_bits(uint32_t* words, uint64_t nwords, uint32_t* out, uint32_t* s_warp) {
    const uint64_t per = (nwords + blockDim.x - 1) / blockDim.x;
    const uint64_t w0 = min((uint64_t)threadIdx.x * per, nwords), w1 = min(w0 + per, nwords);
    uint32_t c = 0;
    for (uint64_t w = w0; w < w1; w++) c += __popc(words[w]);
    uint32_t total;
    uint32_t pos = block_excl_scan(c, s_warp, total);
    for (uint64_t w = w0; w < w1; w++) {
        uint32_t x = words[w];
        if (!x) continue;
        words[w] = 0;
        while (x) {
            const uint32_t b = __ffs(x) - 1;
            out[pos++] = (uint32_t)(w * 32) + b;
            x &= x - 1;
        }
    }
    __syncthreads();
    return total;
}

constexpr uint32_t BP_SORT_MAX = 4096;  // sets up to this size are sorted in shared memory
constexpr uint32_t BP_LIVE = 4096;      // live edges staged per pass (in the sort buffer)
static_assert(BP_LIVE <= BP_SORT_MAX && BP_LIVE % BP_THREADS == 0, "live stage");

struct BlockShared {
    uint32_t keys[BP_SORT_MAX];
    uint32_t stage[40];
    uint32_t scan[BP_THREADS];
    uint32_t g0[BP_THREADS];
    uint32_t eb[BP_THREADS];
    uint32_t ee[BP_THREADS];
    uint32_t warp[33];
    uint32_t tail, item;
    unsigned long long off;
    int fail;
};

// Level-synchronous BFS of set j whose root is queue[0]; returns the size.
// Level-synchronous BFS of set j whose root is queue[0], by a cluster of
// csize blocks: every block scans the same frontier chunk and takes every
// csize-th slice of its edge groups; new vertices are appended through the
// tail counter in block 0's shared memory.  Returns the set size.
__device__ uint32_t block_bfs_ic(const SampleArgs& a, uint32_t j, uint32_t* visited, uint32_t* queue, BlockShared& s,
                                 uint32_t* tail0, uint32_t crank, uint32_t csize, unsigned long long* scanned,
                                 unsigned long long* live) {
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t tid = threadIdx.x, lane = tid & 31;
    uint32_t head = 0;
    for (;;) {
        cl.sync();  // the previous level's appends are complete and visible
        const uint32_t tail = *tail0;
        cl.sync();  // every block has read the level's end before anyone appends
        if (head >= tail) break;
        for (uint32_t c0 = head; c0 < tail; c0 += BP_THREADS) {
            const uint32_t cnt = min((uint32_t)BP_THREADS, tail - c0);
            uint32_t b = 0, e = 0, ng = 0, gfirst = 0;
            if (tid < cnt) {
                const uint32_t v = queue[c0 + tid];
                b = __ldg(a.g.row_ptr + v);
                e = __ldg(a.g.row_ptr + v + 1);
                if (e > b) {
                    gfirst = b >> 2;
                    ng = ((e - 1) >> 2) - gfirst + 1;
                }
            }
            uint32_t total;
            const uint32_t ex = block_excl_scan(ng, s.warp, total);
            s.scan[tid] = ex + ng;
            s.g0[tid] = gfirst;
            s.eb[tid] = b;
            s.ee[tid] = e;
            __syncthreads();
            // BP_ILP groups per thread per step: their loads and Philox chains
            // are independent, so they overlap
            for (uint32_t base = crank * BP_THREADS * BP_ILP; base < total; base += csize * BP_THREADS * BP_ILP) {
                uint32_t gg[BP_ILP], eb[BP_ILP], ee[BP_ILP];
                bool ok[BP_ILP];
#pragma unroll
                for (int q = 0; q < BP_ILP; q++) {
                    const uint32_t t = base + q * BP_THREADS + tid;
                    ok[q] = t < total;
                    gg[q] = 0;
                    eb[q] = 0;
                    ee[q] = 0;
                    if (ok[q]) {
                        uint32_t lo = 0, hi = cnt - 1;
                        while (lo < hi) {
                            const uint32_t mid = (lo + hi) >> 1;
                            if (s.scan[mid] > t) hi = mid;
                            else lo = mid + 1;
                        }
                        const uint32_t prev = lo ? s.scan[lo - 1] : 0u;
                        gg[q] = s.g0[lo] + (t - prev);
                        eb[q] = s.eb[lo];
                        ee[q] = s.ee[lo];
                    }
                }
                uint32_t m = 0;  // bit 4q+k: edge 4*gg[q]+k is live
#pragma unroll
                for (int q = 0; q < BP_ILP; q++)
                    if (ok[q]) m |= group_coins(a, j, gg[q], eb[q], ee[q], scanned) << (4 * q);
                *live += __popc(m);
                // Stage the step's live edges in shared memory, then take them one
                // per thread, so that the col loads and visited updates of the
                // whole block are in flight together.
                uint32_t nlive;
                const uint32_t first = block_excl_scan((uint32_t)__popc(m), s.warp, nlive);
                for (uint32_t p0 = 0; p0 < nlive; p0 += BP_LIVE) {
                    uint32_t idx = first, mm = m;
                    while (mm) {
                        const uint32_t b = __ffs(mm) - 1;
                        mm &= mm - 1;
                        if (idx >= p0 && idx < p0 + BP_LIVE) {
                            uint32_t g = gg[0];
#pragma unroll
                            for (int q = 1; q < BP_ILP; q++)
                                if ((b >> 2) == (uint32_t)q) g = gg[q];
                            s.keys[idx - p0] = g * 4u + (b & 3u);
                        }
                        idx++;
                    }
                    __syncthreads();
                    const uint32_t nstage = min((uint32_t)BP_LIVE, nlive - p0);
                    constexpr int PER = BP_LIVE / BP_THREADS;
                    uint32_t u[PER];
#pragma unroll
                    for (int r = 0; r < PER; r++) {
                        const uint32_t i = tid + r * BP_THREADS;
                        u[r] = i < nstage ? __ldg(a.g.col + s.keys[i]) : NONE;
                    }
                    uint32_t fresh = 0;  // bit r: u[r] was not yet visited
#pragma unroll
                    for (int r = 0; r < PER; r++) {
                        if (u[r] != NONE) {
                            const uint32_t bit = 1u << (u[r] & 31);
                            if (!(atomicOr(&visited[u[r] >> 5], bit) & bit)) fresh |= 1u << r;
                        }
                    }
                    const uint32_t c = __popc(fresh);
                    const uint32_t incl = warp_incl_scan(c);
                    uint32_t pos = 0;
                    if (lane == 31 && incl) pos = atomicAdd(tail0, incl);
                    pos = __shfl_sync(0xFFFFFFFFu, pos, 31) + incl - c;
#pragma unroll
                    for (int r = 0; r < PER; r++)
                        if (fresh >> r & 1u) queue[pos++] = u[r];
                    __syncthreads();  // the stage is free again
                }
            }
            __syncthreads();
        }
        head = tail;
    }
    return head;
}

// LT walk of set j by warp 0 of block 0 (the walk is sequential); the size is
// left in block 0's tail counter.
__device__ void block_walk_lt(const SampleArgs& a, uint32_t j, uint32_t* visited, uint32_t* queue, BlockShared& s,
                              unsigned long long* scanned, unsigned long long* live) {
    const uint32_t tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
        uint32_t v = queue[0], tail = 1;
        for (;;) {
            const uint32_t b = __ldg(a.g.row_ptr + v), e = __ldg(a.g.row_ptr + v + 1);
            if (b == e) break;
            const uint32_t x = philox4x32_10(make_uint4(v, j, a.epoch, STREAM_LT), a.key0, a.key1).x;
            unsigned long long Q = 0;
            uint32_t chosen = NONE;
            for (uint32_t base = b; base < e; base += 32) {
                const uint32_t idx = base + lane;
                const uint32_t qi = idx < e ? __ldg(a.g.q + idx) : 0u;
                const unsigned long long incl = warp_incl_scan_u64(qi) + Q;
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, idx < e && (unsigned long long)x < incl);
                if (bal) {
                    chosen = base + __ffs(bal) - 1;
                    break;
                }
                Q = __shfl_sync(0xFFFFFFFFu, incl, 31);
            }
            *scanned += (chosen == NONE ? e - b : chosen - b + 1) * (lane == 0);
            if (chosen == NONE) break;
            *live += (lane == 0);
            const uint32_t u = __ldg(a.g.col + chosen);
            uint32_t isnew = 0;
            if (lane == 0) {
                const uint32_t bit = 1u << (u & 31);
                isnew = !(atomicOr(&visited[u >> 5], bit) & bit);
            }
            isnew = __shfl_sync(0xFFFFFFFFu, isnew, 0);
            if (!isnew) break;
            if (lane == 0) queue[tail] = u;
            tail++;
            v = u;
        }
        if (lane == 0) s.tail = tail;
    }
    __syncthreads();
}

// Encode the finished set j, whose vertices are queue[0..size) and bits in
// visited, with the whole block: warm-up frequencies, raw ids, a bitmap row or
// Huffman codes by the density cut.  Leaves visited and rbits clear; sets
// s.fail when a heap ran out (nothing of the set is then recorded).
__device__ void block_emit(const SampleArgs& a, uint32_t j, uint32_t size, uint32_t* visited, uint32_t* rbits,
                           uint32_t* aux, uint32_t* queue, BlockShared& s) {
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t n = a.g.n;
    bool clear_by_list = true;
    if (a.mode == MODE_HIST) {
        if ((unsigned long long)a.cut * size <= n) {
            for (uint32_t i = tid; i < size; i += BP_THREADS) atomicAdd(&a.freq[queue[i]], 1u);
            if (tid == 0) atomicAdd(&a.ctr->hist_verts, (unsigned long long)size);
        } else if (tid == 0) {
            atomicAdd(&a.ctr->hist_dense, 1ull);
        }
        if (tid == 0 && a.sizes && j < a.sizes_cap) a.sizes[j] = size;
    } else if (a.mode == MODE_RAW) {
        if (tid == 0) {
            s.off = atomicAdd(&a.ctr->raw_cursor, (unsigned long long)size);
            s.fail = s.off + size > a.raw_cap;
            if (s.fail) atomicMin(&a.ctr->raw_fail, s.off);
        }
        __syncthreads();
        if (!s.fail) {
            for (uint32_t i = tid; i < size; i += BP_THREADS) a.raw_heap[s.off + i] = queue[i];
            if (tid == 0) {
                a.recs[j] = make_rec(KIND_RAW, s.off, size, 0);
                atomicAdd(&a.ctr->sets_raw, 1ull);
                atomicAdd(&a.ctr->rr_vertices, (unsigned long long)size);
                atomicAdd(&a.ctr->words_used, (unsigned long long)size);
            }
        }
    } else if ((unsigned long long)a.cut * size > n) {
        const uint64_t row = a.bp_words;  // ceil(n/32) rounded up to 4
        if (tid == 0) {
            s.off = atomicAdd(&a.ctr->bm_cursor, (unsigned long long)row);
            s.fail = s.off + row > a.bm_cap;
            if (s.fail) atomicMin(&a.ctr->bm_fail, s.off);
        }
        __syncthreads();
        uint4* vis4 = reinterpret_cast<uint4*>(visited);
        if (!s.fail) {
            uint4* dst = reinterpret_cast<uint4*>(a.bm_heap + s.off);
            for (uint64_t w = tid; w < row / 4; w += BP_THREADS) {
                dst[w] = vis4[w];
                vis4[w] = make_uint4(0, 0, 0, 0);
            }
            if (tid == 0) {
                a.recs[j] = make_rec(KIND_BITMAP, s.off, size, 0);
                atomicAdd(&a.ctr->sets_bm, 1ull);
                atomicAdd(&a.ctr->rr_vertices, (unsigned long long)size);
                atomicAdd(&a.ctr->words_used, (unsigned long long)row);
            }
        } else {
            for (uint64_t w = tid; w < row / 4; w += BP_THREADS) vis4[w] = make_uint4(0, 0, 0, 0);
        }
        clear_by_list = false;
    } else if (size <= BP_SORT_MAX) {
        // Huffman, small set: keys sorted in shared memory, visited cleared by list
        uint32_t P = 2;
        while (P < size) P <<= 1;
        for (uint32_t i = tid; i < P; i += BP_THREADS) {
            uint32_t key = 0xFFFFFFFFu;
            if (i < size) {
                const uint32_t v = queue[i];
                const uint32_t r = __ldg(a.cb.rank_of + v);
                key = (r != NONE) ? r : (RAW_FLAG | v);
                visited[v >> 5] = 0u;
            }
            s.keys[i] = key;
        }
        __syncthreads();
        for (uint32_t k = 2; k <= P; k <<= 1) {
            for (uint32_t jj = k >> 1; jj > 0; jj >>= 1) {
                for (uint32_t i = tid; i < P; i += BP_THREADS) {
                    const uint32_t ixj = i ^ jj;
                    if (ixj > i) {
                        const uint32_t x = s.keys[i], y = s.keys[ixj];
                        if ((x > y) == ((i & k) == 0)) {
                            s.keys[i] = y;
                            s.keys[ixj] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        if (warp == 0) {
            WarpStats ws;
            const bool ok = warp_huff_store(a, j, s.keys, size, s.stage, ws);
            if (lane == 0) {
                s.fail = !ok;
                if (ok) {
                    atomicAdd(&a.ctr->sets_huff, 1ull);
                    atomicAdd(&a.ctr->rr_vertices, (unsigned long long)size);
                    atomicAdd(&a.ctr->code_bits, ws.bits);
                    atomicAdd(&a.ctr->words_used, ws.words);
                }
            }
        }
        __syncthreads();
        clear_by_list = false;
    } else {
        // Huffman, large set: ranks into the rank bitmap, coded ids out of the
        // visited bitmap, both read back in order
        uint32_t mine = 0;
        for (uint32_t i = tid; i < size; i += BP_THREADS) {
            const uint32_t v = queue[i];
            const uint32_t r = __ldg(a.cb.rank_of + v);
            if (r != NONE) {
                atomicOr(&rbits[r >> 5], 1u << (r & 31));
                atomicAnd(&visited[v >> 5], ~(1u << (v & 31)));
                mine++;
            }
        }
        const uint32_t n_coded = block_sum(mine, s.warp);  // includes barriers
        const uint32_t got_c = compact_bits(rbits, ((uint64_t)a.cb.nsym + 31) / 32, queue, s.warp);
        const uint32_t got_r = compact_bits(visited, ((uint64_t)n + 31) / 32, queue + n_coded, s.warp);
        if (got_c != n_coded || got_r != size - n_coded) set_error(a.ctr, 2);
        const uint32_t n_raw = size - n_coded;
        const uint32_t nch = (n_coded + 31) / 32;
        for (uint32_t c = warp; c < nch; c += BP_WARPS) {
            const uint32_t i = c * 32 + lane;
            const uint32_t L = i < n_coded ? (uint32_t)__ldg(a.cb.len_of_rank + queue[i]) : 0u;
            const uint32_t sum = warp_sum(L);
            if (lane == 0) aux[c] = sum;
        }
        __syncthreads();
        // exclusive scan of chunk bit counts, in place
        uint32_t carry = 0;
        for (uint32_t t0 = 0; t0 < nch; t0 += BP_THREADS) {
            const uint32_t c = t0 + tid;
            const uint32_t x = c < nch ? aux[c] : 0u;
            uint32_t tot;
            const uint32_t ex = block_excl_scan(x, s.warp, tot);
            if (c < nch) aux[c] = carry + ex;
            carry += tot;
        }
        __syncthreads();
        const uint32_t bits = carry;
        const uint32_t nside = side_words(n_coded);
        const unsigned long long words = (unsigned long long)nside + n_raw + (bits + 31) / 32;
        if (tid == 0) {
            s.off = words ? atomicAdd(&a.ctr->code_cursor, words) : 0ull;
            s.fail = s.off + words > a.code_cap;
            if (s.fail) atomicMin(&a.ctr->code_fail, s.off);
        }
        __syncthreads();
        if (!s.fail) {
            uint32_t* out = a.code_heap + s.off + nside + n_raw;
            for (uint32_t c = warp; c < nch; c += BP_WARPS) {
                const uint32_t i = c * 32 + lane;
                uint32_t L = 0, code = 0;
                if (i < n_coded) {
                    const uint32_t r = queue[i];
                    L = __ldg(a.cb.len_of_rank + r);
                    code = __ldg(a.cb.code_of_rank + r);
                }
                const uint32_t incl = warp_incl_scan(L);
                const uint32_t o = aux[c] + incl - L;
                if (c > 0 && lane == 0) a.code_heap[s.off + c - 1] = aux[c];
                if (L) {
                    const uint32_t w = o >> 5, sh = o & 31u;
                    if (sh + L <= 32) {
                        atomicOr(&out[w], bswap32(code << (32 - sh - L)));
                    } else {
                        atomicOr(&out[w], bswap32(code >> (sh + L - 32)));
                        atomicOr(&out[w + 1], bswap32(code << (64 - sh - L)));
                    }
                }
            }
            for (uint32_t i = tid; i < n_raw; i += BP_THREADS) a.code_heap[s.off + nside + i] = queue[n_coded + i];
            if (tid == 0) {
                a.recs[j] = make_rec(KIND_HUFF, s.off, size, n_coded);
                atomicAdd(&a.ctr->sets_huff, 1ull);
                atomicAdd(&a.ctr->rr_vertices, (unsigned long long)size);
                atomicAdd(&a.ctr->code_bits, (unsigned long long)bits);
                atomicAdd(&a.ctr->words_used, words);
            }
        }
        clear_by_list = false;
    }
    if (clear_by_list) {
        __syncthreads();
        for (uint32_t i = tid; i < size; i += BP_THREADS) visited[queue[i] >> 5] = 0u;
    }
    __syncthreads();
}

// One heavy set per thread-block cluster (a cluster of 1 is a plain block).
// Block 0 of the cluster owns the set's bookkeeping in its shared memory, and
// encodes the set once the cluster has finished the search.
__global__ void __launch_bounds__(BP_THREADS, 2) sample_block_kernel(SampleArgs a, uint32_t nbig) {
    __shared__ BlockShared s;
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t crank = cl.block_rank(), csize = cl.num_blocks();
    const uint32_t slot = blockIdx.x / csize;
    uint32_t* tail0 = cl.map_shared_rank(&s.tail, 0);
    uint32_t* item0 = cl.map_shared_rank(&s.item, 0);
    int* fail0 = cl.map_shared_rank(&s.fail, 0);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t n = a.g.n;
    uint32_t* visited = a.bp_visited + (uint64_t)slot * a.bp_words;
    uint32_t* rbits = a.bp_rbits + (uint64_t)slot * a.bp_words;
    uint32_t* aux = a.bp_aux + (uint64_t)slot * a.bp_words;
    uint32_t* queue = a.bp_queue + (uint64_t)slot * n;
    unsigned long long scanned = 0, live = 0;  // emitted sets only

    const uint64_t nslots = gridDim.x / csize;
    for (uint64_t round = 0;; round++) {
        unsigned long long set_scanned = 0, set_live = 0;
        if (crank == 0 && tid == 0) {
            // plain form: item i of the batch goes to slot i mod slots; otherwise
            // the listed heavy sets are taken by work stealing
            const unsigned long long next = a.direct ? slot + round * nslots : atomicAdd(&a.ctr->big_work, 1ull);
            s.item = (uint32_t)min(next, (unsigned long long)nbig);
        }
        cl.sync();
        const uint32_t item = *item0;
        if (item >= nbig) break;
        const uint32_t j = !a.direct ? a.big_list[item] : (a.list ? a.list[item] : a.j0 + item);
        if (crank == 0 && tid == 0) {
            const uint4 rr = philox4x32_10(make_uint4(0u, j, a.epoch, STREAM_ROOT), a.key0, a.key1);
            const uint32_t root = __umulhi(rr.x, n);
            visited[root >> 5] |= 1u << (root & 31);
            queue[0] = root;
            s.tail = 1;
            s.fail = 0;
        }
        uint32_t size;
        if (a.model == MODEL_IC) {
            size = block_bfs_ic(a, j, visited, queue, s, tail0, crank, csize, &set_scanned, &set_live);
        } else {
            cl.sync();
            if (crank == 0) block_walk_lt(a, j, visited, queue, s, &set_scanned, &set_live);
            cl.sync();
            size = *tail0;
        }
        if (crank == 0) {
            __syncthreads();
            block_emit(a, j, size, visited, rbits, aux, queue, s);
        }
        cl.sync();  // the set is encoded and the slot is clean
        const int failed = *fail0;
        if (crank == 0 && tid == 0) {
            if (failed) a.retry_list[atomicAdd(&a.ctr->retry_count, 1ull)] = j;
            else if (a.mode != MODE_HIST) atomicAdd(&a.ctr->sets_big, 1ull);
        }
        if (!failed) {
            scanned += set_scanned;
            live += set_live;
        }
    }
    cl.sync();  // no block leaves while another may still read block 0's shared memory
    unsigned long long sc = scanned, lv = live;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        sc += __shfl_xor_sync(0xFFFFFFFFu, sc, d);
        lv += __shfl_xor_sync(0xFFFFFFFFu, lv, d);
    }
    if (lane == 0) {
        if (sc) atomicAdd(&a.ctr->edges_scanned, sc);
        if (lv) atomicAdd(&a.ctr->edges_live, lv);
    }
}

// Sets found by the bit-parallel search (msbfs.cu) that fall under the density
// cut: block b takes mask bit sbits[b] (set ids[b]), gathers the set's
// membership row from the masks into its scratch slot with one ballot per
// word, lists the ids in ascending order, and encodes the set as the block
// kernel does.  The set's size and edge counts come from the search.
__global__ void __launch_bounds__(BP_THREADS, 2) sample_ms_sparse_kernel(SampleArgs a, const uint32_t* vis,
                                                                        const uint32_t* sbits, const uint32_t* ids,
                                                                        const MsCounters* mc) {
    __shared__ BlockShared s;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t n = a.g.n, nw = (n + 31) / 32;
    const uint32_t slot = blockIdx.x;
    uint32_t* visited = a.bp_visited + (uint64_t)slot * a.bp_words;
    uint32_t* rbits = a.bp_rbits + (uint64_t)slot * a.bp_words;
    uint32_t* aux = a.bp_aux + (uint64_t)slot * a.bp_words;
    uint32_t* queue = a.bp_queue + (uint64_t)slot * n;
    const uint32_t sb = sbits[blockIdx.x], j = ids[blockIdx.x];
    for (uint32_t w = warp; w < nw; w += BP_WARPS) {
        const uint32_t v = w * 32 + lane;
        const uint32_t m = v < n ? vis[v] : 0u;
        const uint32_t r = __ballot_sync(0xFFFFFFFFu, (m >> sb) & 1u);
        if (lane == 0) visited[w] = r;
    }
    __syncthreads();
    const uint32_t size = compact_bits(visited, nw, queue, s.warp);  // clears visited
    if (size != (uint32_t)mc->size[sb]) set_error(a.ctr, 6);
    for (uint32_t i = tid; i < size; i += BP_THREADS) atomicOr(&visited[queue[i] >> 5], 1u << (queue[i] & 31));
    if (tid == 0) s.fail = 0;
    __syncthreads();
    block_emit(a, j, size, visited, rbits, aux, queue, s);
    if (tid == 0) {
        if (s.fail) {
            a.retry_list[atomicAdd(&a.ctr->retry_count, 1ull)] = j;
        } else {
            if (a.mode != MODE_HIST) atomicAdd(&a.ctr->sets_big, 1ull);
            atomicAdd(&a.ctr->edges_scanned, mc->scanned[sb]);
            atomicAdd(&a.ctr->edges_live, mc->live[sb]);
        }
    }
}

// ---------------------------------------------------------------------------
// Shared-memory block path: one 512-thread block per set that outgrew a warp,
// for sets of up to BQ vertices.  The vertex list, each vertex's CSR bounds
// (loaded when the vertex is discovered, so the next level does not wait for
// them) and the visited hash set all live in shared memory; a BFS level costs
// one block-wide scan of group counts and one barrier per 512 frontier
// vertices.  A set that outgrows BQ goes to the global-bitmap block kernel.
// ---------------------------------------------------------------------------
constexpr uint32_t BQ = 4096;
constexpr uint32_t BQ_HASH = 2 * BQ;

struct MidShared {
    uint32_t scan[BP_THREADS];
    uint32_t g0[BP_THREADS];
    uint32_t eb[BP_THREADS];
    uint32_t ee[BP_THREADS];
    uint32_t warp[33];
    uint32_t stage[40];
    uint32_t tail, item, head;
    int overflow, fail;
};

constexpr size_t MID_DYN_SMEM = (size_t)(3 * BQ + BQ_HASH) * sizeof(uint32_t);

__device__ __forceinline__ void mid_append(const SampleArgs& a, MidShared& s, uint32_t* Q, uint32_t* QB,
                                           uint32_t* QE, bool isnew, uint32_t u) {
    const uint32_t lane = lane_id();
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, isnew);
    if (!bal) return;
    const uint32_t leader = __ffs(bal) - 1;
    uint32_t pos = 0;
    if (lane == leader) pos = atomicAdd(&s.tail, (uint32_t)__popc(bal));
    pos = __shfl_sync(0xFFFFFFFFu, pos, leader) + __popc(bal & lanemask_lt());
    if (isnew) {
        if (pos < BQ) {
            Q[pos] = u;
            QB[pos] = __ldg(a.g.row_ptr + u);
            QE[pos] = __ldg(a.g.row_ptr + u + 1);
        } else {
            s.overflow = 1;
        }
    }
}

constexpr uint32_t MID_WARP_GROUPS = 512;  // a chunk with more edge groups goes to the whole block

// Warp 0 of the block expands the queue alone, 32 vertices at a time in FIFO
// order, while the unexpanded vertices fit one warp and their edge groups stay
// under MID_WARP_GROUPS; the rest of the block waits at a barrier.  Deep sets
// with thin frontiers then advance without block barriers.  Each lane takes
// BP_ILP edge groups per pass, and the live edges' col loads are issued four
// at a time before their inserts.  Returns the new head; s.tail is updated.
__device__ uint32_t mid_warp_run(const SampleArgs& a, MidShared& s, uint32_t* Q, uint32_t* QB, uint32_t* QE,
                                 uint32_t* H, uint32_t j, uint32_t head, unsigned long long* scanned,
                                 unsigned long long* live) {
    constexpr uint32_t HMASK = BQ_HASH - 1;
    constexpr uint32_t HSHIFT = 32 - __builtin_ctz(BQ_HASH);
    const uint32_t lane = lane_id();
    uint32_t tail = s.tail;
    bool overflow = false;
    while (head < tail && tail - head <= 32 && !overflow) {
        const uint32_t cnt = tail - head;
        uint32_t b = 0, e = 0, ng = 0, gfirst = 0;
        if (lane < cnt) {
            b = QB[head + lane];
            e = QE[head + lane];
            if (e > b) {
                gfirst = b >> 2;
                ng = ((e - 1) >> 2) - gfirst + 1;
            }
        }
        const uint32_t incl = warp_incl_scan(ng);
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        if (total > MID_WARP_GROUPS) break;
        s.scan[lane] = incl;
        s.g0[lane] = gfirst;
        s.eb[lane] = b;
        s.ee[lane] = e;
        __syncwarp();
        for (uint32_t base = 0; base < total && !overflow; base += 32 * BP_ILP) {
            uint32_t gg[BP_ILP], eb[BP_ILP], ee[BP_ILP];
#pragma unroll
            for (int q = 0; q < BP_ILP; q++) {
                const uint32_t t = base + q * 32 + lane;
                gg[q] = 0;
                eb[q] = 0;
                ee[q] = 0;
                if (t < total) {
                    uint32_t lo = 0, hi = cnt - 1;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (s.scan[mid] > t) hi = mid;
                        else lo = mid + 1;
                    }
                    gg[q] = s.g0[lo] + (t - (lo ? s.scan[lo - 1] : 0u));
                    eb[q] = s.eb[lo];
                    ee[q] = s.ee[lo];
                }
            }
            uint32_t m = 0;
#pragma unroll
            for (int q = 0; q < BP_ILP; q++)
                if (ee[q] > eb[q]) m |= group_coins(a, j, gg[q], eb[q], ee[q], scanned) << (4 * q);
            *live += __popc(m);
            while (__any_sync(0xFFFFFFFFu, m != 0) && !overflow) {
                uint32_t u[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    u[k] = NONE;
                    if (m) {
                        const uint32_t bit = __ffs(m) - 1;
                        m &= m - 1;
                        uint32_t g = gg[0];
#pragma unroll
                        for (int q = 1; q < BP_ILP; q++)
                            if ((bit >> 2) == (uint32_t)q) g = gg[q];
                        u[k] = __ldg(a.g.col + g * 4u + (bit & 3u));
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const bool isnew = u[k] != NONE && hash_insert(H, HMASK, HSHIFT, u[k], a.ctr);
                    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, isnew);
                    if (!bal) continue;
                    const uint32_t pos = tail + __popc(bal & lanemask_lt());
                    if (isnew && pos < BQ) {
                        Q[pos] = u[k];
                        QB[pos] = __ldg(a.g.row_ptr + u[k]);
                        QE[pos] = __ldg(a.g.row_ptr + u[k] + 1);
                    }
                    tail += __popc(bal);
                    if (tail > BQ) {
                        overflow = true;
                        break;
                    }
                }
            }
        }
        head += cnt;
        __syncwarp();
    }
    if (lane == 0) {
        s.tail = tail;
        if (overflow) s.overflow = 1;
    }
    return head;
}

__global__ void __launch_bounds__(BP_THREADS) sample_mid_kernel(SampleArgs a, uint32_t nbig) {
    extern __shared__ __align__(16) uint32_t mdyn[];
    __shared__ MidShared s;
    uint32_t* Q = mdyn;
    uint32_t* QB = Q + BQ;
    uint32_t* QE = QB + BQ;
    uint32_t* H = QE + BQ;
    constexpr uint32_t HMASK = BQ_HASH - 1;
    constexpr uint32_t HSHIFT = 32 - __builtin_ctz(BQ_HASH);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t n = a.g.n;
    unsigned long long scanned = 0, live = 0;  // emitted sets only
    for (uint32_t i = tid; i < BQ_HASH / 4; i += BP_THREADS) reinterpret_cast<uint4*>(H)[i] = make_uint4(0, 0, 0, 0);

    for (;;) {
        unsigned long long set_scanned = 0, set_live = 0;
        if (tid == 0) s.item = (uint32_t)min(atomicAdd(&a.ctr->mid_work, 1ull), (unsigned long long)nbig);
        __syncthreads();
        const uint32_t item = s.item;
        if (item >= nbig) break;
        const uint32_t j = a.big_list[item];
        if (tid == 0) {
            const uint4 rr = philox4x32_10(make_uint4(0u, j, a.epoch, STREAM_ROOT), a.key0, a.key1);
            const uint32_t root = __umulhi(rr.x, n);
            hash_insert(H, HMASK, HSHIFT, root, a.ctr);
            Q[0] = root;
            QB[0] = __ldg(a.g.row_ptr + root);
            QE[0] = __ldg(a.g.row_ptr + root + 1);
            s.tail = 1;
            s.overflow = 0;
            s.fail = 0;
        }
        __syncthreads();

        if (a.model == MODEL_IC) {
            uint32_t head = 0;
            for (;;) {
                const uint32_t tail = s.tail;  // the previous step ended with a barrier
                if (head >= tail || s.overflow) break;
                if (tail - head <= 32) {
                    // thin frontier: warp 0 runs ahead alone
                    const uint32_t h0 = head;
                    if (warp == 0) {
                        const uint32_t nh = mid_warp_run(a, s, Q, QB, QE, H, j, head, &set_scanned, &set_live);
                        if (lane == 0) s.head = nh;
                    }
                    __syncthreads();
                    head = s.head;
                    if (head != h0) {
                        __syncthreads();  // everyone has read s.head before it changes
                        continue;
                    }
                    // no progress: the chunk's edge groups are too many for one warp
                }
                const uint32_t ltail = s.tail;
                for (uint32_t c0 = head; c0 < ltail; c0 += BP_THREADS) {
                    const uint32_t cnt = min((uint32_t)BP_THREADS, ltail - c0);
                    uint32_t b = 0, e = 0, ng = 0, gfirst = 0;
                    if (tid < cnt) {
                        b = QB[c0 + tid];
                        e = QE[c0 + tid];
                        if (e > b) {
                            gfirst = b >> 2;
                            ng = ((e - 1) >> 2) - gfirst + 1;
                        }
                    }
                    uint32_t total;
                    const uint32_t ex = block_excl_scan(ng, s.warp, total);
                    s.scan[tid] = ex + ng;
                    s.g0[tid] = gfirst;
                    s.eb[tid] = b;
                    s.ee[tid] = e;
                    __syncthreads();
                    for (uint32_t base = 0; base < total; base += BP_THREADS * BP_ILP) {
                        // a set past BQ stops growing here: each warp inserts at most one
                        // more round after it sees the flag, so the table stays under 2*BQ
                        if (*(volatile int*)&s.overflow) break;
                        uint32_t gg[BP_ILP], eb[BP_ILP], ee[BP_ILP];
#pragma unroll
                        for (int q = 0; q < BP_ILP; q++) {
                            const uint32_t t = base + q * BP_THREADS + tid;
                            gg[q] = 0;
                            eb[q] = 0;
                            ee[q] = 0;
                            if (t < total) {
                                uint32_t lo = 0, hi = cnt - 1;
                                while (lo < hi) {
                                    const uint32_t mid = (lo + hi) >> 1;
                                    if (s.scan[mid] > t) hi = mid;
                                    else lo = mid + 1;
                                }
                                gg[q] = s.g0[lo] + (t - (lo ? s.scan[lo - 1] : 0u));
                                eb[q] = s.eb[lo];
                                ee[q] = s.ee[lo];
                            }
                        }
                        uint32_t m = 0;
#pragma unroll
                        for (int q = 0; q < BP_ILP; q++)
                            if (ee[q] > eb[q]) m |= group_coins(a, j, gg[q], eb[q], ee[q], &set_scanned) << (4 * q);
                        set_live += __popc(m);
                        const uint32_t rounds = __reduce_max_sync(0xFFFFFFFFu, (uint32_t)__popc(m));
                        for (uint32_t r = 0; r < rounds; r++) {
                            if (*(volatile int*)&s.overflow) break;
                            bool isnew = false;
                            uint32_t u = 0;
                            if (m) {
                                const uint32_t bit = __ffs(m) - 1;
                                m &= m - 1;
                                uint32_t g = gg[0];
#pragma unroll
                                for (int q = 1; q < BP_ILP; q++)
                                    if ((bit >> 2) == (uint32_t)q) g = gg[q];
                                u = __ldg(a.g.col + g * 4u + (bit & 3u));
                                isnew = hash_insert(H, HMASK, HSHIFT, u, a.ctr);
                            }
                            mid_append(a, s, Q, QB, QE, isnew, u);
                        }
                    }
                    __syncthreads();
                }
                head = ltail;
            }
        } else if (warp == 0) {
            uint32_t v = Q[0], tail = 1;
            for (;;) {
                const uint32_t b = __ldg(a.g.row_ptr + v), e = __ldg(a.g.row_ptr + v + 1);
                if (b == e) break;
                const uint32_t x = philox4x32_10(make_uint4(v, j, a.epoch, STREAM_LT), a.key0, a.key1).x;
                unsigned long long Qs = 0;
                uint32_t chosen = NONE;
                for (uint32_t base = b; base < e; base += 32) {
                    const uint32_t idx = base + lane;
                    const uint32_t qi = idx < e ? __ldg(a.g.q + idx) : 0u;
                    const unsigned long long incl = warp_incl_scan_u64(qi) + Qs;
                    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, idx < e && (unsigned long long)x < incl);
                    if (bal) {
                        chosen = base + __ffs(bal) - 1;
                        break;
                    }
                    Qs = __shfl_sync(0xFFFFFFFFu, incl, 31);
                }
                set_scanned += (chosen == NONE ? e - b : chosen - b + 1) * (lane == 0);
                if (chosen == NONE) break;
                set_live += (lane == 0);
                const uint32_t u = __ldg(a.g.col + chosen);
                uint32_t isnew = 0;
                if (lane == 0) isnew = hash_insert(H, HMASK, HSHIFT, u, a.ctr);
                isnew = __shfl_sync(0xFFFFFFFFu, isnew, 0);
                if (!isnew) break;
                if (tail >= BQ) {
                    if (lane == 0) s.overflow = 1;
                    break;
                }
                if (lane == 0) Q[tail] = u;
                tail++;
                v = u;
            }
            if (lane == 0) s.tail = tail;
        }
        __syncthreads();
        const uint32_t size = min(s.tail, BQ);
        const bool overflow = s.overflow != 0;

        if (overflow) {
            if (tid == 0) a.giant_list[atomicAdd(&a.ctr->giant_count, 1ull)] = j;
        } else if (a.mode == MODE_HIST) {
            if ((unsigned long long)a.cut * size <= n) {
                for (uint32_t i = tid; i < size; i += BP_THREADS) atomicAdd(&a.freq[Q[i]], 1u);
                if (tid == 0) atomicAdd(&a.ctr->hist_verts, (unsigned long long)size);
            } else if (tid == 0) {
                atomicAdd(&a.ctr->hist_dense, 1ull);
            }
            if (tid == 0 && a.sizes && j < a.sizes_cap) a.sizes[j] = size;
        } else if (a.mode == MODE_RAW) {
            if (tid == 0) {
                s.item = 0;
                const unsigned long long off = atomicAdd(&a.ctr->raw_cursor, (unsigned long long)size);
                s.fail = off + size > a.raw_cap;
                if (s.fail) atomicMin(&a.ctr->raw_fail, off);
                s.warp[0] = (uint32_t)off;
                s.warp[1] = (uint32_t)(off >> 32);
            }
            __syncthreads();
            const unsigned long long off = ((unsigned long long)s.warp[1] << 32) | s.warp[0];
            if (!s.fail) {
                for (uint32_t i = tid; i < size; i += BP_THREADS) a.raw_heap[off + i] = Q[i];
                if (tid == 0) {
                    a.recs[j] = make_rec(KIND_RAW, off, size, 0);
                    atomicAdd(&a.ctr->sets_raw, 1ull);
                    atomicAdd(&a.ctr->rr_vertices, (unsigned long long)size);
                    atomicAdd(&a.ctr->words_used, (unsigned long long)size);
                }
            }
        } else if ((unsigned long long)a.cut * size > n) {
            const unsigned long long row = (((unsigned long long)n + 31) / 32 + 3) & ~3ull;
            if (tid == 0) {
                const unsigned long long off = atomicAdd(&a.ctr->bm_cursor, row);
                s.fail = off + row > a.bm_cap;
                if (s.fail) atomicMin(&a.ctr->bm_fail, off);
                s.warp[0] = (uint32_t)off;
                s.warp[1] = (uint32_t)(off >> 32);
            }
            __syncthreads();
            const unsigned long long off = ((unsigned long long)s.warp[1] << 32) | s.warp[0];
            if (!s.fail) {
                for (uint32_t i = tid; i < size; i += BP_THREADS) {
                    const uint32_t v = Q[i];
                    atomicOr(&a.bm_heap[off + (v >> 5)], 1u << (v & 31));
                }
                if (tid == 0) {
                    a.recs[j] = make_rec(KIND_BITMAP, off, size, 0);
                    atomicAdd(&a.ctr->sets_bm, 1ull);
                    atomicAdd(&a.ctr->rr_vertices, (unsigned long long)size);
                    atomicAdd(&a.ctr->words_used, row);
                }
            }
        } else {
            // keys (rank, or RAW_FLAG|id) sorted in shared memory, reusing QB
            uint32_t P = 2;
            while (P < size) P <<= 1;
            for (uint32_t i = tid; i < P; i += BP_THREADS) {
                uint32_t key = 0xFFFFFFFFu;
                if (i < size) {
                    const uint32_t v = Q[i];
                    const uint32_t r = __ldg(a.cb.rank_of + v);
                    key = (r != NONE) ? r : (RAW_FLAG | v);
                }
                QB[i] = key;
            }
            __syncthreads();
            for (uint32_t k = 2; k <= P; k <<= 1) {
                for (uint32_t jj = k >> 1; jj > 0; jj >>= 1) {
                    for (uint32_t i = tid; i < P; i += BP_THREADS) {
                        const uint32_t ixj = i ^ jj;
                        if (ixj > i) {
                            const uint32_t x = QB[i], y = QB[ixj];
                            if ((x > y) == ((i & k) == 0)) {
                                QB[i] = y;
                                QB[ixj] = x;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            if (warp == 0) {
                WarpStats ws;
                const bool ok = warp_huff_store(a, j, QB, size, s.stage, ws);
                if (lane == 0) {
                    s.fail = !ok;
                    if (ok) {
                        atomicAdd(&a.ctr->sets_huff, 1ull);
                        atomicAdd(&a.ctr->rr_vertices, (unsigned long long)size);
                        atomicAdd(&a.ctr->code_bits, ws.bits);
                        atomicAdd(&a.ctr->words_used, ws.words);
                    }
                }
            }
        }
        __syncthreads();
        const bool failed = s.fail != 0;
        if (tid == 0 && !overflow) {
            if (failed) a.retry_list[atomicAdd(&a.ctr->retry_count, 1ull)] = j;
            else if (a.mode != MODE_HIST) atomicAdd(&a.ctr->sets_big, 1ull);
        }
        if (!overflow && !failed) {
            scanned += set_scanned;
            live += set_live;
        }
        for (uint32_t i = tid; i < BQ_HASH / 4; i += BP_THREADS) reinterpret_cast<uint4*>(H)[i] = make_uint4(0, 0, 0, 0);
        __syncthreads();
    }
    unsigned long long sc = scanned, lv = live;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        sc += __shfl_xor_sync(0xFFFFFFFFu, sc, d);
        lv += __shfl_xor_sync(0xFFFFFFFFu, lv, d);
    }
    if (lane == 0) {
        if (sc) atomicAdd(&a.ctr->edges_scanned, sc);
        if (lv) atomicAdd(&a.ctr->edges_live, lv);
    }
}

cudaError_t launch_sample_mid(const SampleArgs& a, uint32_t nbig, int sms, cudaStream_t s) {
    if (nbig == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(sample_mid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)MID_DYN_SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sample_mid_kernel, BP_THREADS, MID_DYN_SMEM);
    if (e != cudaSuccess) return e;
    uint32_t grid = (uint32_t)(sms * (per_sm > 0 ? per_sm : 1));
    if (grid > nbig) grid = nbig;
    sample_mid_kernel<<<grid, BP_THREADS, MID_DYN_SMEM, s>>>(a, nbig);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <uint32_t QW>
static cudaError_t launch_warp_t(const SampleArgs& a, int sms, cudaStream_t s) {
    const size_t smem = (size_t)WP_WARPS * 3 * QW * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(sample_warp_kernel<QW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sample_warp_kernel<QW>, WP_WARPS * 32, smem);
    if (e != cudaSuccess) return e;
    const uint32_t grid = (uint32_t)(sms * (per_sm > 0 ? per_sm : 1));
    sample_warp_kernel<QW><<<grid, WP_WARPS * 32, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sample_warp(const SampleArgs& a, uint32_t qw, int sms, cudaStream_t s) {
    switch (qw) {
        case 64: return launch_warp_t<64>(a, sms, s);
        case 128: return launch_warp_t<128>(a, sms, s);
        case 256: return launch_warp_t<256>(a, sms, s);
        case 512: return launch_warp_t<512>(a, sms, s);
        case 1024: return launch_warp_t<1024>(a, sms, s);
        case 2048: return launch_warp_t<2048>(a, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

// `slots` clusters of `csize` blocks each
cudaError_t launch_ms_sparse(const SampleArgs& a, const uint32_t* vis, const uint32_t* sbits, const uint32_t* ids,
                             const MsCounters* mc, uint32_t count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    sample_ms_sparse_kernel<<<count, BP_THREADS, 0, s>>>(a, vis, sbits, ids, mc);
    return cudaGetLastError();
}

cudaError_t launch_sample_block(const SampleArgs& a, uint32_t nbig, uint32_t slots, uint32_t csize, cudaStream_t s) {
    if (nbig == 0 || slots == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(slots * csize, 1, 1);
    cfg.blockDim = dim3(BP_THREADS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, sample_block_kernel, a, nbig);
}

// Clusters of `csize` blocks of the block kernel that fit on the GPU at once.
int block_path_max_clusters(uint32_t csize) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize, 1, 1);
    cfg.blockDim = dim3(BP_THREADS, 1, 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (void*)sample_block_kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

}  // namespace hbx
