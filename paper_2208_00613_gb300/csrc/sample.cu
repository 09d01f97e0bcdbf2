// RR-set sampling fused with encoding (Section 2.2; Section 4.2, Algorithm 1).
//
// One random RR set (Definition 2) is the set of vertices that reach a random
// root through live edges.  Every coin is a Philox draw keyed by (edge or
// vertex id, set id j, epoch, stream), so the set does not depend on the order
// in which the search meets its edges:
//   root   = floor(x * n / 2^32),  x = word 0 of Philox(0, j, epoch, 3)
//   IC     in-edge e is live iff (x >> 8) * 2^-24 < p[e] (exact fp32), x = word
//          e%4 of Philox(e/4, j, epoch, 1): one draw serves 4 consecutive edges
//   LT     at vertex v, x = word 0 of Philox(v, j, epoch, 2); the walk moves to
//          the source of the first in-edge whose inclusive prefix sum of fixed-
//          point weights exceeds x, and stops when there is none or that source
//          is already in the set.
//
// Two kernels:
//   sample_warp_kernel   one warp per set.  The set's vertex list (the BFS queue)
//                        and a hash set of visited ids live in shared memory; a
//                        set that outgrows the warp's capacity QW is handed to
//                        the block kernel.  The finished set is encoded by the
//                        same warp: a bitmap if cut*|R| > n, else its vertices
//                        are mapped to codebook ranks, sorted (bitonic), and the
//                        codes bit-packed over a prefix sum of code lengths.
//   sample_block_kernel  one 512-thread block per large set, level-synchronous
//                        BFS with the visited set as an n-bit bitmap and the
//                        queue in HBM; the visited bitmap is the bitmap
//                        encoding, and a rank bitmap gives the sorted code order.
#include <cstdio>

#include "common.cuh"
#include "internal.h"

namespace hbx {

constexpr int WP_WARPS = 8;
constexpr int BP_THREADS = 512;
constexpr int BP_WARPS = BP_THREADS / 32;
constexpr uint32_t WORK_CHUNK = 4;  // sets taken per work-stealing step

struct WarpLocal {
    uint32_t scan[32];
    uint32_t g0[32];
    uint32_t eb[32];
    uint32_t ee[32];
    uint32_t stage[40];
};

__device__ __forceinline__ void set_error(Counters* c, unsigned long long code) {
    atomicMax(&c->error, code);
}

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

__device__ __forceinline__ bool ic_live(uint32_t x, float p) {
    return (float)(x >> 8) * 0x1p-24f < p;
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
            // lower partner keeps min when sorting up, max when sorting down
            const bool keep_min = (lower == up);
            key = keep_min ? min(key, other) : max(key, other);
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
    unsigned long long scanned = 0, live = 0, verts = 0, bits = 0, huff = 0, bm = 0, raw = 0;
};

// Samples set j into queue[0..tail).  Returns false if it outgrew QW.
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
        uint32_t head = 0;
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
                    const uint32_t eb = wl.eb[lo], ee = wl.ee[lo];
                    const float4 p4 = __ldg(reinterpret_cast<const float4*>(a.g.prob) + gg);
                    const uint4 x = philox4x32_10(make_uint4(gg, j, a.epoch, STREAM_IC), a.key0, a.key1);
                    const uint32_t e0 = gg * 4u;
                    const bool v0 = e0 >= eb && e0 < ee, v1 = e0 + 1 >= eb && e0 + 1 < ee;
                    const bool v2 = e0 + 2 >= eb && e0 + 2 < ee, v3 = e0 + 3 >= eb && e0 + 3 < ee;
                    st.scanned += (uint32_t)v0 + (uint32_t)v1 + (uint32_t)v2 + (uint32_t)v3;
                    live_mask = (uint32_t)(v0 && ic_live(x.x, p4.x)) | ((uint32_t)(v1 && ic_live(x.y, p4.y)) << 1) |
                                ((uint32_t)(v2 && ic_live(x.z, p4.z)) << 2) |
                                ((uint32_t)(v3 && ic_live(x.w, p4.w)) << 3);
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

// Encode a finished set held in queue[0..size) and write its record.
// Returns false if a heap ran out of space (nothing of the set is written).
template <uint32_t QW>
__device__ bool warp_emit(const SampleArgs& a, uint32_t j, uint32_t* queue, uint32_t size, WarpLocal& wl,
                          WarpStats& st) {
    const uint32_t lane = lane_id();
    const uint32_t n = a.g.n;
    if (a.mode == MODE_HIST) {
        if ((unsigned long long)a.cut * size <= n)
            for (uint32_t i = lane; i < size; i += 32) atomicAdd(&a.freq[queue[i]], 1u);
        return true;
    }
    if (a.mode == MODE_RAW) {
        unsigned long long off = 0;
        if (lane == 0) off = atomicAdd(&a.ctr->raw_cursor, (unsigned long long)size);
        off = __shfl_sync(0xFFFFFFFFu, off, 0);
        if (off + size > a.raw_cap) return false;
        for (uint32_t i = lane; i < size; i += 32) a.raw_heap[off + i] = queue[i];
        if (lane == 0) {
            SetRec r;
            r.size = size; r.n_coded = 0; r.code_bits = 0; r.kind = KIND_RAW; r.off = off; r.raw_off = 0;
            a.recs[j] = r;
        }
        st.verts += size * (lane == 0);
        st.raw += (lane == 0);
        return true;
    }
    // MODE_ENCODE
    if ((unsigned long long)a.cut * size > n) {
        const unsigned long long row = (((unsigned long long)n + 31) / 32 + 3) & ~3ull;
        unsigned long long off = 0;
        if (lane == 0) off = atomicAdd(&a.ctr->bm_cursor, row);
        off = __shfl_sync(0xFFFFFFFFu, off, 0);
        if (off + row > a.bm_cap) return false;
        for (uint32_t i = lane; i < size; i += 32) {
            const uint32_t v = queue[i];
            atomicOr(&a.bm_heap[off + (v >> 5)], 1u << (v & 31));
        }
        if (lane == 0) {
            SetRec r;
            r.size = size; r.n_coded = 0; r.code_bits = 0; r.kind = KIND_BITMAP; r.off = off; r.raw_off = 0;
            a.recs[j] = r;
        }
        st.verts += size * (lane == 0);
        st.bm += (lane == 0);
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
    uint32_t n_coded = 0, bits = 0;
    for (uint32_t base = 0; base < size; base += 32) {
        const uint32_t i = base + lane;
        const uint32_t key = i < size ? queue[i] : 0xFFFFFFFFu;
        const bool coded = key < RAW_FLAG;
        n_coded += __popc(__ballot_sync(0xFFFFFFFFu, coded));
        bits += warp_sum(coded ? (uint32_t)__ldg(a.cb.len_of_rank + key) : 0u);
    }
    const uint32_t n_raw = size - n_coded;
    const uint32_t nside = n_coded ? (n_coded - 1) / 32 : 0;
    const unsigned long long words = nside + (bits + 31) / 32;
    unsigned long long off = 0, roff = 0;
    if (lane == 0) {
        off = words ? atomicAdd(&a.ctr->code_cursor, words) : 0ull;
        roff = n_raw ? atomicAdd(&a.ctr->raw_cursor, (unsigned long long)n_raw) : 0ull;
    }
    off = __shfl_sync(0xFFFFFFFFu, off, 0);
    roff = __shfl_sync(0xFFFFFFFFu, roff, 0);
    if (off + words > a.code_cap || roff + n_raw > a.raw_cap) return false;

    // pack 32 codes at a time into the stage, write completed words
    uint32_t* out = a.code_heap + off + nside;
    uint32_t carry = 0;  // bit offset of the current chunk's first code
    for (uint32_t i = lane; i < 40; i += 32) wl.stage[i] = 0;
    __syncwarp();
    for (uint32_t c = 0; c * 32 < n_coded; c++) {
        const uint32_t i = c * 32 + lane;
        uint32_t L = 0, code = 0;
        if (i < n_coded) {
            const uint32_t r = queue[i];
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
                atomicOr(&wl.stage[w], code << (32 - sh - L));
            } else {
                atomicOr(&wl.stage[w], code >> (sh + L - 32));
                atomicOr(&wl.stage[w + 1], code << (64 - sh - L));
            }
        }
        __syncwarp();
        const uint32_t end = carry + chunk_bits;
        const uint32_t done = (end >> 5) - wbase;  // complete words in the stage
        for (uint32_t w = lane; w < done; w += 32) out[wbase + w] = bswap32(wl.stage[w]);
        __syncwarp();
        const uint32_t partial = wl.stage[done];
        __syncwarp();
        for (uint32_t w = lane; w < 40; w += 32) wl.stage[w] = 0;
        __syncwarp();
        if (lane == 0) wl.stage[0] = partial;
        __syncwarp();
        carry = end;
    }
    if ((carry & 31u) && lane == 0) out[carry >> 5] = bswap32(wl.stage[0]);
    for (uint32_t i = lane; i < n_raw; i += 32) a.raw_heap[roff + i] = queue[n_coded + i] & ~RAW_FLAG;
    if (lane == 0) {
        SetRec r;
        r.size = size; r.n_coded = n_coded; r.code_bits = bits; r.kind = KIND_HUFF; r.off = off; r.raw_off = roff;
        a.recs[j] = r;
    }
    __syncwarp();
    st.verts += size * (lane == 0);
    st.bits += bits * (lane == 0);
    st.huff += (lane == 0);
    return true;
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
    if (!a.persistent) {
        item = blockIdx.x * WP_WARPS + warp;
        item_end = min(item + 1, a.count);
    }
    for (;;) {
        if (item >= item_end) {
            if (!a.persistent) break;
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
    // per-warp statistics
    const unsigned long long s0 = st.scanned, s1 = st.live;
    unsigned long long sc = s0, lv = s1;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        sc += __shfl_xor_sync(0xFFFFFFFFu, sc, d);
        lv += __shfl_xor_sync(0xFFFFFFFFu, lv, d);
    }
    if (lane == 0) {
        if (sc) atomicAdd(&a.ctr->edges_scanned, sc);
        if (lv) atomicAdd(&a.ctr->edges_live, lv);
        if (st.verts) atomicAdd(&a.ctr->rr_vertices, st.verts);
        if (st.bits) atomicAdd(&a.ctr->code_bits, st.bits);
        if (st.huff) atomicAdd(&a.ctr->sets_huff, st.huff);
        if (st.bm) atomicAdd(&a.ctr->sets_bm, st.bm);
        if (st.raw) atomicAdd(&a.ctr->sets_raw, st.raw);
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

// Write the set bits of words [0, nwords) in ascending order to out[base..),
// zeroing the words; returns the count.  Each thread takes a contiguous range.
__device__ uint32_t compact_bits(uint32_t* words, uint64_t nwords, uint32_t* out, uint32_t xor_flag,
                                 uint32_t* s_warp) {
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
            out[pos++] = ((uint32_t)(w * 32) + b) | xor_flag;
            x &= x - 1;
        }
    }
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(BP_THREADS) sample_block_kernel(SampleArgs a, uint32_t nbig) {
    __shared__ WarpLocal wl_all[BP_WARPS];
    __shared__ uint32_t s_warp[33];
    __shared__ uint32_t s_tail, s_item;
    __shared__ unsigned long long s_off, s_roff;
    __shared__ int s_fail;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t n = a.g.n;
    uint32_t* visited = a.bp_visited + (uint64_t)blockIdx.x * a.bp_words;
    uint32_t* rbits = a.bp_rbits + (uint64_t)blockIdx.x * a.bp_words;
    uint32_t* aux = a.bp_aux + (uint64_t)blockIdx.x * a.bp_words;
    uint32_t* queue = a.bp_queue + (uint64_t)blockIdx.x * n;
    WarpLocal& wl = wl_all[warp];
    unsigned long long scanned = 0, live = 0;  // emitted sets only

    for (;;) {
        unsigned long long set_scanned = 0, set_live = 0;
        if (tid == 0) s_item = (uint32_t)min(atomicAdd(&a.ctr->big_work, 1ull), (unsigned long long)nbig);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= nbig) break;
        const uint32_t j = a.big_list[item];
        if (tid == 0) {
            const uint4 rr = philox4x32_10(make_uint4(0u, j, a.epoch, STREAM_ROOT), a.key0, a.key1);
            const uint32_t root = __umulhi(rr.x, n);
            visited[root >> 5] |= 1u << (root & 31);
            queue[0] = root;
            s_tail = 1;
        }
        __syncthreads();
        if (a.model == MODEL_IC) {
            uint32_t head = 0;
            for (;;) {
                const uint32_t tail = s_tail;
                __syncthreads();
                if (head >= tail) break;
                for (uint32_t c0 = head + warp * 32; c0 < tail; c0 += BP_WARPS * 32) {
                    const uint32_t cnt = min(32u, tail - c0);
                    uint32_t b = 0, e = 0, ng = 0, gfirst = 0;
                    if (lane < cnt) {
                        const uint32_t v = queue[c0 + lane];
                        b = __ldg(a.g.row_ptr + v);
                        e = __ldg(a.g.row_ptr + v + 1);
                        if (e > b) {
                            gfirst = b >> 2;
                            ng = ((e - 1) >> 2) - gfirst + 1;
                        }
                    }
                    const uint32_t incl = warp_incl_scan(ng);
                    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
                    wl.scan[lane] = incl;
                    wl.g0[lane] = gfirst;
                    wl.eb[lane] = b;
                    wl.ee[lane] = e;
                    __syncwarp();
                    for (uint32_t base = 0; base < total; base += 32) {
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
                            const uint32_t eb = wl.eb[lo], ee = wl.ee[lo];
                            const float4 p4 = __ldg(reinterpret_cast<const float4*>(a.g.prob) + gg);
                            const uint4 x = philox4x32_10(make_uint4(gg, j, a.epoch, STREAM_IC), a.key0, a.key1);
                            const uint32_t e0 = gg * 4u;
                            const bool v0 = e0 >= eb && e0 < ee, v1 = e0 + 1 >= eb && e0 + 1 < ee;
                            const bool v2 = e0 + 2 >= eb && e0 + 2 < ee, v3 = e0 + 3 >= eb && e0 + 3 < ee;
                            set_scanned += (uint32_t)v0 + (uint32_t)v1 + (uint32_t)v2 + (uint32_t)v3;
                            live_mask = (uint32_t)(v0 && ic_live(x.x, p4.x)) |
                                        ((uint32_t)(v1 && ic_live(x.y, p4.y)) << 1) |
                                        ((uint32_t)(v2 && ic_live(x.z, p4.z)) << 2) |
                                        ((uint32_t)(v3 && ic_live(x.w, p4.w)) << 3);
                            set_live += __popc(live_mask);
                        }
                        uint32_t u[4];
#pragma unroll
                        for (int k = 0; k < 4; k++)
                            u[k] = (live_mask >> k & 1u) ? __ldg(a.g.col + gg * 4u + k) : 0u;
#pragma unroll
                        for (int k = 0; k < 4; k++) {
                            bool isnew = false;
                            if (live_mask >> k & 1u) {
                                const uint32_t bit = 1u << (u[k] & 31);
                                isnew = !(atomicOr(&visited[u[k] >> 5], bit) & bit);
                            }
                            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, isnew);
                            if (bal) {
                                uint32_t pos = 0;
                                if (lane == (uint32_t)(__ffs(bal) - 1)) pos = atomicAdd(&s_tail, (uint32_t)__popc(bal));
                                pos = __shfl_sync(0xFFFFFFFFu, pos, __ffs(bal) - 1);
                                if (isnew) queue[pos + __popc(bal & lanemask_lt())] = u[k];
                            }
                        }
                    }
                    __syncwarp();
                }
                __syncthreads();
                head = tail;
            }
        } else {
            if (warp == 0) {
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
                    set_scanned += (chosen == NONE ? e - b : chosen - b + 1) * (lane == 0);
                    if (chosen == NONE) break;
                    set_live += (lane == 0);
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
                if (lane == 0) s_tail = tail;
            }
            __syncthreads();
        }
        const uint32_t size = s_tail;
        __syncthreads();

        // ---- emit ----
        bool clear_by_list = true;
        if (tid == 0) s_fail = 0;
        __syncthreads();
        if (a.mode == MODE_HIST) {
            if ((unsigned long long)a.cut * size <= n)
                for (uint32_t i = tid; i < size; i += BP_THREADS) atomicAdd(&a.freq[queue[i]], 1u);
        } else if (a.mode == MODE_RAW) {
            if (tid == 0) {
                s_off = atomicAdd(&a.ctr->raw_cursor, (unsigned long long)size);
                s_fail = s_off + size > a.raw_cap;
            }
            __syncthreads();
            if (!s_fail) {
                for (uint32_t i = tid; i < size; i += BP_THREADS) a.raw_heap[s_off + i] = queue[i];
                if (tid == 0) {
                    SetRec r;
                    r.size = size; r.n_coded = 0; r.code_bits = 0; r.kind = KIND_RAW; r.off = s_off; r.raw_off = 0;
                    a.recs[j] = r;
                    atomicAdd(&a.ctr->sets_raw, 1ull);
                    atomicAdd(&a.ctr->rr_vertices, (unsigned long long)size);
                }
            } else if (tid == 0) {
                a.retry_list[atomicAdd(&a.ctr->retry_count, 1ull)] = j;
            }
        } else if ((unsigned long long)a.cut * size > n) {
            const uint64_t row = a.bp_words;  // ceil(n/32) rounded up to 4
            if (tid == 0) {
                s_off = atomicAdd(&a.ctr->bm_cursor, (unsigned long long)row);
                s_fail = s_off + row > a.bm_cap;
            }
            __syncthreads();
            uint4* vis4 = reinterpret_cast<uint4*>(visited);
            if (!s_fail) {
                uint4* dst = reinterpret_cast<uint4*>(a.bm_heap + s_off);
                for (uint64_t w = tid; w < row / 4; w += BP_THREADS) {
                    dst[w] = vis4[w];
                    vis4[w] = make_uint4(0, 0, 0, 0);
                }
                if (tid == 0) {
                    SetRec r;
                    r.size = size; r.n_coded = 0; r.code_bits = 0; r.kind = KIND_BITMAP; r.off = s_off; r.raw_off = 0;
                    a.recs[j] = r;
                    atomicAdd(&a.ctr->sets_bm, 1ull);
                    atomicAdd(&a.ctr->rr_vertices, (unsigned long long)size);
                }
            } else {
                for (uint64_t w = tid; w < row / 4; w += BP_THREADS) vis4[w] = make_uint4(0, 0, 0, 0);
                if (tid == 0) a.retry_list[atomicAdd(&a.ctr->retry_count, 1ull)] = j;
            }
            clear_by_list = false;
        } else {
            // Huffman: ranks into the rank bitmap, coded ids out of the visited bitmap
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
            const uint32_t n_coded = block_sum(mine, s_warp);  // includes a barrier
            const uint32_t got_c = compact_bits(rbits, ((uint64_t)a.cb.nsym + 31) / 32, queue, 0u, s_warp);
            const uint32_t got_r = compact_bits(visited, ((uint64_t)n + 31) / 32, queue + n_coded, 0u, s_warp);
            if (got_c != n_coded || got_r != size - n_coded) set_error(a.ctr, 2);
            const uint32_t n_raw = size - n_coded;
            const uint32_t nch = (n_coded + 31) / 32;
            for (uint32_t c = warp; c < nch; c += BP_WARPS) {
                const uint32_t i = c * 32 + lane;
                const uint32_t L = i < n_coded ? (uint32_t)__ldg(a.cb.len_of_rank + queue[i]) : 0u;
                const uint32_t s = warp_sum(L);
                if (lane == 0) aux[c] = s;
            }
            __syncthreads();
            // exclusive scan of chunk bit counts, in place
            uint32_t carry = 0;
            for (uint32_t t0 = 0; t0 < nch; t0 += BP_THREADS) {
                const uint32_t c = t0 + tid;
                const uint32_t x = c < nch ? aux[c] : 0u;
                uint32_t tot;
                const uint32_t ex = block_excl_scan(x, s_warp, tot);
                if (c < nch) aux[c] = carry + ex;
                carry += tot;
            }
            __syncthreads();
            const uint32_t bits = carry;
            const uint32_t nside = n_coded ? (n_coded - 1) / 32 : 0;
            const unsigned long long words = nside + (bits + 31) / 32;
            if (tid == 0) {
                s_off = words ? atomicAdd(&a.ctr->code_cursor, words) : 0ull;
                s_roff = n_raw ? atomicAdd(&a.ctr->raw_cursor, (unsigned long long)n_raw) : 0ull;
                s_fail = (s_off + words > a.code_cap) || (s_roff + n_raw > a.raw_cap);
            }
            __syncthreads();
            if (!s_fail) {
                uint32_t* out = a.code_heap + s_off + nside;
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
                    if (c > 0 && lane == 0) a.code_heap[s_off + c - 1] = aux[c];
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
                for (uint32_t i = tid; i < n_raw; i += BP_THREADS) a.raw_heap[s_roff + i] = queue[n_coded + i];
                if (tid == 0) {
                    SetRec r;
                    r.size = size; r.n_coded = n_coded; r.code_bits = bits; r.kind = KIND_HUFF;
                    r.off = s_off; r.raw_off = s_roff;
                    a.recs[j] = r;
                    atomicAdd(&a.ctr->sets_huff, 1ull);
                    atomicAdd(&a.ctr->rr_vertices, (unsigned long long)size);
                    atomicAdd(&a.ctr->code_bits, (unsigned long long)bits);
                }
            } else if (tid == 0) {
                a.retry_list[atomicAdd(&a.ctr->retry_count, 1ull)] = j;
            }
            clear_by_list = false;
        }
        if (clear_by_list) {
            __syncthreads();
            for (uint32_t i = tid; i < size; i += BP_THREADS) visited[queue[i] >> 5] = 0u;
        }
        if (tid == 0 && !s_fail) atomicAdd(&a.ctr->sets_big, 1ull);
        if (!s_fail) {
            scanned += set_scanned;
            live += set_live;
        }
        __syncthreads();
    }
    // statistics
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

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <uint32_t QW>
static cudaError_t launch_warp_t(const SampleArgs& a, int sms, cudaStream_t s) {
    const size_t smem = (size_t)WP_WARPS * 3 * QW * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(sample_warp_kernel<QW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    uint32_t grid;
    if (a.persistent) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sample_warp_kernel<QW>, WP_WARPS * 32, smem);
        if (e != cudaSuccess) return e;
        grid = (uint32_t)(sms * (per_sm > 0 ? per_sm : 1));
    } else {
        grid = (a.count + WP_WARPS - 1) / WP_WARPS;
    }
    if (grid == 0) return cudaSuccess;
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

cudaError_t launch_sample_block(const SampleArgs& a, uint32_t nbig, uint32_t slots, cudaStream_t s) {
    if (nbig == 0 || slots == 0) return cudaSuccess;
    sample_block_kernel<<<slots, BP_THREADS, 0, s>>>(a, nbig);
    return cudaGetLastError();
}

int block_path_threads() { return BP_THREADS; }

}  // namespace hbx
