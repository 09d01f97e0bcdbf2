// Bit-parallel reverse BFS for the IC sets that outgrow shared memory.
//
// Under IC (Section 2.1) the RR set of sample j is the set of vertices that
// reach its root through edges whose coin, drawn from Philox at (edge group,
// j, epoch, 1), is live.  The set does not depend on the order in which the
// search visits vertices, so up to 32 such sets are searched together, one
// bit per set: vis[v] and nxt[v] are 32-bit masks (visited; reached during
// this level), and the frontier lists each vertex once per level with the
// mask of the sets whose frontier holds it.  A vertex's in-edge probabilities
// and sources are then read once for all of those sets.  A set draws its coins
// for a group of 4 in-edges only while one of their sources is still unvisited
// in that set (a visited source cannot join it again), so the sets equal those
// of one full search per set; their scanned-edge counts are those of the full
// search (every in-edge of every member), while their live-edge counts cover
// only the live edges into sources not yet visited at the edge's level.
//
// A level is: the light kernel takes the frontier 32 vertices per warp (edge
// groups spread over the lanes by a warp prefix sum; vertices with more than
// MS_HEAVY groups are cut into chunks of MS_CHUNK groups for the heavy
// kernel); in both, a warp stages 32 groups at a time, finds the sets that
// still need each group's coins, and spreads those (group, set) pairs evenly
// over its lanes, one Philox block each.  Every live edge ORs its sets into
// nxt[source] with a reduction that returns nothing, so no thread waits on it;
// then the compaction pass turns nxt into the next frontier, keeping for each
// vertex only the sets that had not visited it yet (marking them in vis), and
// clears nxt.  The host advances levels until the frontier is empty, then a
// tally pass gives each set's size and scanned edges, and the emit pass writes
// the dense sets' bitmap rows (a 32 x 32 bit transpose per warp through shared
// memory) and clears vis for the next batch.
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace hbx {

constexpr int MS_THREADS = 256;
constexpr int MS_WARPS = MS_THREADS / 32;
// A warp takes 32 frontier vertices of at most MS_HEAVY edge groups each, so
// no warp holds more than 1024 groups; bigger vertices are cut into chunks of
// MS_CHUNK groups, one warp per chunk.
constexpr uint32_t MS_HEAVY = 32;
constexpr uint32_t MS_CHUNK = 256;
// A group's sources' visited masks are read only when at least this many sets
// hold its vertex in their frontier: for fewer, the gathers (which mostly miss
// L2 on the largest graphs) cost more than the Philox blocks they save.
constexpr uint32_t MS_VIS_MIN = 4;

// The IC coin block of (edge group g, set j) is Philox4x32-10 of the counter
// (g, j, epoch, STREAM_IC).  Following its words through the first rounds:
// round 0 multiplies g and epoch, round 1 multiplies a word that depends on j
// alone and one that depends on g alone, and round 2 multiplies one word that
// depends on g alone.  Those five of the twenty 32 x 32 -> 64-bit products are
// computed once per group (three) or once per set (two), and each (group, set)
// pair finishes with the other fifteen.  The result is the same function,
// bit for bit.
//
// Group words: (w1 ^ K1[1], y2 ^ K0[2], hi(M0 x2) ^ K1[2], lo(M0 x2)), where
// round 0 gives z1 = hi(M0 g) ^ STREAM_IC ^ K1[0], w1 = lo(M0 g), and round 1
// gives x2 = hi(M1 z1) ^ lo(M1 epoch) ^ K0[1], y2 = lo(M1 z1).
__device__ __forceinline__ uint4 ic_group_words(uint32_t g, uint32_t epoch, const PhiloxKeys& rk) {
    const uint64_t p0 = (uint64_t)PHILOX_M0 * g;
    const uint32_t z1 = (uint32_t)(p0 >> 32) ^ STREAM_IC ^ rk.k1[0], w1 = (uint32_t)p0;
    const uint32_t le = (uint32_t)((uint64_t)PHILOX_M1 * epoch);
    const uint64_t pz = (uint64_t)PHILOX_M1 * z1;
    const uint32_t x2 = (uint32_t)(pz >> 32) ^ le ^ rk.k0[1], y2 = (uint32_t)pz;
    const uint64_t px = (uint64_t)PHILOX_M0 * x2;
    return make_uint4(w1 ^ rk.k1[1], y2 ^ rk.k0[2], (uint32_t)(px >> 32) ^ rk.k1[2], (uint32_t)px);
}

// Set words: M0 a1 (high, low) with a1 = hi(M1 epoch) ^ j ^ K0[0], the
// round-0 output word that carries the set id.
__device__ __forceinline__ uint2 ic_set_words(uint32_t j, uint32_t epoch, const PhiloxKeys& rk) {
    const uint32_t a1 = (uint32_t)(((uint64_t)PHILOX_M1 * epoch) >> 32) ^ j ^ rk.k0[0];
    const uint64_t pa = (uint64_t)PHILOX_M0 * a1;
    return make_uint2((uint32_t)(pa >> 32), (uint32_t)pa);
}

// The pair's coin block: round 2's remaining product, then rounds 3-9.
__device__ __forceinline__ uint4 ic_coins(uint4 G, uint2 S, const PhiloxKeys& rk) {
    const uint64_t pm = (uint64_t)PHILOX_M1 * (S.x ^ G.x);
    uint4 c = make_uint4((uint32_t)(pm >> 32) ^ G.y, (uint32_t)pm, G.z ^ S.y, G.w);
#pragma unroll
    for (int r = 3; r < 10; r++) {
        const uint64_t p0 = (uint64_t)PHILOX_M0 * c.x, p1 = (uint64_t)PHILOX_M1 * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk.k0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk.k1[r],
                       (uint32_t)p0);
    }
    return c;
}

// Per-warp live-edge counts of the batch's sets in shared memory, added to the
// batch totals when the warp is done.
__device__ __forceinline__ void ms_init_shared(const MsArgs& a, uint2* s_sw, uint32_t (*s_live)[MS_SETS]) {
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // set words of the batch's sets (unused slots never get a bit)
    if (threadIdx.x < MS_SETS) s_sw[threadIdx.x] = ic_set_words(a.sets[threadIdx.x], a.epoch, a.rk);
    s_live[warp][lane] = 0;
    __syncthreads();
}

__device__ __forceinline__ void ms_flush_live(const MsArgs& a, uint32_t (*s_live)[MS_SETS], uint32_t nblk,
                                              uint32_t nvis) {
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncwarp();
    const uint32_t c = s_live[warp][lane];
    if (c) atomicAdd(&a.mc->live[lane], (unsigned long long)c);
    if (lane == 0 && nblk) atomicAdd(&a.mc->blocks, (unsigned long long)nblk);
    if (lane == 0 && nvis) atomicAdd(&a.mc->visits, (unsigned long long)nvis);
}

// One warp's staging of a round: up to MS_ROUND aligned groups of 4 in-edges,
// two per lane (slot 2l + k holds lane l's k-th group), and for each the sets
// that still need its coins.  The round's (slot, set) pairs are listed and
// drawn MS_ITEMS at a time.
constexpr uint32_t MS_ROUND = 64;
constexpr uint32_t MS_ITEMS = 512;
constexpr int MS_ILP = 2;  // pairs a lane draws at once
struct MsRound {
    uint16_t items[MS_ITEMS];  // slot << 5 | set of the window's pairs
    uint4 thr[MS_ROUND];      // live thresholds of the group's edges
    uint4 um[MS_ROUND];       // per edge: sets of the frontier mask whose source is not yet visited
    uint4 em[MS_ROUND];       // per edge: sets for which it is live (filled by the items)
    uint4 gw[MS_ROUND];       // group words of the coin blocks (ic_group_words)
};

// One group of a round: its sources and thresholds (loaded together, so
// both are in flight at once), then the visited masks of its sources.
struct MsGroup {
    uint4 c, thr, um;
    uint32_t need;
};

__device__ __forceinline__ MsGroup ms_stage(const MsArgs& a, bool valid, uint32_t gg, uint32_t eb, uint32_t ee,
                                            uint32_t f) {
    MsGroup G;
    G.c = make_uint4(0, 0, 0, 0);
    G.thr = make_uint4(0, 0, 0, 0);
    G.um = make_uint4(0, 0, 0, 0);
    if (valid && f) {
        G.c = __ldg(reinterpret_cast<const uint4*>(a.col4) + gg);
        G.thr = __ldg(reinterpret_cast<const uint4*>(a.g.thr) + gg);
    }
    return G;
}

__device__ __forceinline__ void ms_visited(const MsArgs& a, MsGroup& G, bool valid, uint32_t gg, uint32_t eb,
                                           uint32_t ee, uint32_t f) {
    if (valid && f && (uint32_t)__popc(f) < MS_VIS_MIN) {
        const uint32_t e0 = gg * 4u;
        if (e0 >= eb && e0 < ee) G.um.x = f;
        if (e0 + 1 >= eb && e0 + 1 < ee) G.um.y = f;
        if (e0 + 2 >= eb && e0 + 2 < ee) G.um.z = f;
        if (e0 + 3 >= eb && e0 + 3 < ee) G.um.w = f;
    } else if (valid && f) {
        const uint32_t e0 = gg * 4u;
        if (e0 >= eb && e0 < ee) G.um.x = f & ~__ldg(a.vis + G.c.x);
        if (e0 + 1 >= eb && e0 + 1 < ee) G.um.y = f & ~__ldg(a.vis + G.c.y);
        if (e0 + 2 >= eb && e0 + 2 < ee) G.um.z = f & ~__ldg(a.vis + G.c.z);
        if (e0 + 3 >= eb && e0 + 3 < ee) G.um.w = f & ~__ldg(a.vis + G.c.w);
    }
    G.need = G.um.x | G.um.y | G.um.z | G.um.w;
}

// One round of a warp.  Lane l brings groups gg[k] (k = 0, 1) of frontier
// vertices whose in-edges are [eb[k], ee[k]), for the sets of masks f[k]
// (valid[k] = false: no group).  A set needs a group's Philox block only if
// the source of one of the vertex's edges in the group has not been visited
// by that set: a visited source cannot join the set again, so its coin
// decides nothing.  The (group, set) pairs that remain are listed in slot
// order, MS_ITEMS at a time, and spread evenly over the lanes, one Philox
// block each; live edges into unvisited sources are collected per edge in
// shared memory and then ORed into nxt[source] with one reduction per edge.
__device__ __forceinline__ void ms_round(const MsArgs& a, MsRound& R, const uint2* s_sw, uint32_t* s_live_w,
                                         uint32_t& nblk, uint32_t& nvis, const bool* valid, const uint32_t* gg,
                                         const uint32_t* eb, const uint32_t* ee, const uint32_t* f) {
    const uint32_t lane = threadIdx.x & 31;
    MsGroup G0 = ms_stage(a, valid[0], gg[0], eb[0], ee[0], f[0]);
    MsGroup G1 = ms_stage(a, valid[1], gg[1], eb[1], ee[1], f[1]);
    ms_visited(a, G0, valid[0], gg[0], eb[0], ee[0], f[0]);
    ms_visited(a, G1, valid[1], gg[1], eb[1], ee[1], f[1]);
    nvis += __popc(__ballot_sync(0xFFFFFFFFu, valid[0] && f[0])) + __popc(__ballot_sync(0xFFFFFFFFu, valid[1] && f[1]));
    const uint32_t n0 = __popc(G0.need), n1 = __popc(G1.need);
    const uint32_t incl = warp_incl_scan(n0 + n1);
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (total == 0) return;  // warp-uniform
    nblk += total;  // one Philox block per (group, set) pair
    R.thr[2 * lane] = G0.thr;
    R.thr[2 * lane + 1] = G1.thr;
    R.um[2 * lane] = G0.um;
    R.um[2 * lane + 1] = G1.um;
    R.em[2 * lane] = make_uint4(0, 0, 0, 0);
    R.em[2 * lane + 1] = make_uint4(0, 0, 0, 0);
    if (n0) R.gw[2 * lane] = ic_group_words(gg[0], a.epoch, a.rk);
    if (n1) R.gw[2 * lane + 1] = ic_group_words(gg[1], a.epoch, a.rk);
    uint32_t m0 = G0.need, m1 = G1.need, o = incl - n0 - n1;  // the lane's pairs: positions [o, incl)
    for (uint32_t w0 = 0; w0 < total; w0 += MS_ITEMS) {
        const uint32_t wend = min(w0 + MS_ITEMS, total);
        // list the lane's pairs that fall in this window
        while (o < wend && o < incl) {
            uint32_t it;
            if (m0) {
                it = ((2 * lane) << 5) | (uint32_t)(__ffs(m0) - 1);
                m0 &= m0 - 1;
            } else {
                it = ((2 * lane + 1) << 5) | (uint32_t)(__ffs(m1) - 1);
                m1 &= m1 - 1;
            }
            R.items[o - w0] = (uint16_t)it;
            o++;
        }
        __syncwarp();
        // MS_ILP pairs per lane per step: their Philox blocks are independent,
        // so the rounds of one fill the others' multiply latency
        for (uint32_t t0 = w0 + lane; t0 < wend; t0 += 32 * MS_ILP) {
            uint32_t slot[MS_ILP], s[MS_ILP];
            bool have[MS_ILP];
            uint4 x[MS_ILP];
#pragma unroll
            for (int q = 0; q < MS_ILP; q++) {
                const uint32_t t = t0 + 32 * q;
                have[q] = t < wend;
                const uint32_t it = have[q] ? (uint32_t)R.items[t - w0] : 0u;
                slot[q] = it >> 5;
                s[q] = it & 31u;
            }
#pragma unroll
            for (int q = 0; q < MS_ILP; q++) x[q] = ic_coins(R.gw[slot[q]], s_sw[s[q]], a.rk);
#pragma unroll
            for (int q = 0; q < MS_ILP; q++) {
                if (!have[q]) continue;
                const uint4 th = R.thr[slot[q]], u = R.um[slot[q]];
                const uint32_t bit = 1u << s[q];
                const bool l0 = (u.x & bit) && ic_live(x[q].x, th.x);
                const bool l1 = (u.y & bit) && ic_live(x[q].y, th.y);
                const bool l2 = (u.z & bit) && ic_live(x[q].z, th.z);
                const bool l3 = (u.w & bit) && ic_live(x[q].w, th.w);
                if (l0 | l1 | l2 | l3) {
                    uint32_t* em = reinterpret_cast<uint32_t*>(&R.em[slot[q]]);
                    if (l0) atomicOr(em + 0, bit);
                    if (l1) atomicOr(em + 1, bit);
                    if (l2) atomicOr(em + 2, bit);
                    if (l3) atomicOr(em + 3, bit);
                    atomicAdd(&s_live_w[s[q]], (uint32_t)l0 + (uint32_t)l1 + (uint32_t)l2 + (uint32_t)l3);
                }
            }
        }
        __syncwarp();  // the window's list is rewritten by the next one
    }
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const uint4 em = R.em[2 * lane + k];
        const uint4 c = k ? G1.c : G0.c;
        if (em.x) atomicOr(&a.nxt[c.x], em.x);
        if (em.y) atomicOr(&a.nxt[c.y], em.y);
        if (em.z) atomicOr(&a.nxt[c.z], em.z);
        if (em.w) atomicOr(&a.nxt[c.w], em.w);
    }
    __syncwarp();  // the staging is reused by the next round
}

// Roots of the batch's sets, reached at level 0.  <<<1, 32>>>
__global__ void ms_start_kernel(MsArgs a) {
    const uint32_t s = threadIdx.x;
    if (s < a.mc->nsets && a.sets[s] != NONE) {  // NONE: an unused slot of a tile batch
        const uint4 rr = philox4x32_10(make_uint4(0u, a.sets[s], a.epoch, STREAM_ROOT), a.key0, a.key1);
        atomicOr(&a.nxt[__umulhi(rr.x, a.g.n)], 1u << s);
    }
}

__global__ void __launch_bounds__(MS_THREADS, 4) ms_light_kernel(MsArgs a) {
    __shared__ uint2 s_sw[MS_SETS];
    __shared__ uint32_t s_live[MS_WARPS][MS_SETS];
    __shared__ uint32_t w_scan[MS_WARPS][32], w_g0[MS_WARPS][32], w_eb[MS_WARPS][32], w_ee[MS_WARPS][32],
        w_f[MS_WARPS][32];
    __shared__ MsRound s_round[MS_WARPS];
    const uint32_t nF = a.mc->nF;
    if (blockIdx.x * MS_WARPS * 32 >= nF) return;  // thin level: this block has no chunk
    ms_init_shared(a, s_sw, s_live);
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t nblk = 0, nvis = 0;
    for (;;) {
        // the next 32 frontier vertices (work stealing: the cost of a chunk
        // varies with its vertices' degrees and masks)
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(&a.mc->lwork, 32u);
        c = __shfl_sync(0xFFFFFFFFu, c, 0);
        if (c >= nF) break;
        const uint32_t i = c + lane;
        uint32_t v = 0, f = 0, b = 0, e = 0, gfirst = 0, ng = 0;
        if (i < nF) {
            v = a.F[i];
            f = a.Ff[i];
            b = __ldg(a.g.row_ptr + v);
            e = __ldg(a.g.row_ptr + v + 1);
            if (e > b) {
                gfirst = b >> 2;
                ng = ((e - 1) >> 2) - gfirst + 1;
            }
            if (ng > MS_HEAVY) {
                // heavy vertex: its groups go to whole warps in chunks
                for (uint32_t g = gfirst; g < gfirst + ng; g += MS_CHUNK) {
                    const uint32_t h = atomicAdd(&a.mc->nH, 1u);
                    if (h < a.heavy_cap) a.heavy[h] = make_uint4(v, g, min(g + MS_CHUNK, gfirst + ng), f);
                    else set_error(a.ctr, 5);
                }
                ng = 0;
            }
        }
        const uint32_t incl = warp_incl_scan(ng);
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        w_scan[warp][lane] = incl;
        w_g0[warp][lane] = gfirst;
        w_eb[warp][lane] = b;
        w_ee[warp][lane] = e;
        w_f[warp][lane] = f;
        __syncwarp();
        for (uint32_t base = 0; base < total; base += MS_ROUND) {
            bool ok[2];
            uint32_t gg[2], eb[2], ee[2], ff[2];
#pragma unroll
            for (int k = 0; k < 2; k++) {
                // consecutive lanes take consecutive groups (coalesced loads)
                const uint32_t t = base + 32 * k + lane;
                ok[k] = t < total;
                gg[k] = eb[k] = ee[k] = ff[k] = 0;
                if (ok[k]) {
                    uint32_t lo = 0, hi = 31;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (w_scan[warp][mid] > t) hi = mid;
                        else lo = mid + 1;
                    }
                    gg[k] = w_g0[warp][lo] + (t - (lo ? w_scan[warp][lo - 1] : 0u));
                    eb[k] = w_eb[warp][lo];
                    ee[k] = w_ee[warp][lo];
                    ff[k] = w_f[warp][lo];
                }
            }
            ms_round(a, s_round[warp], s_sw, s_live[warp], nblk, nvis, ok, gg, eb, ee, ff);
        }
        __syncwarp();
    }
    ms_flush_live(a, s_live, nblk, nvis);
}

__global__ void __launch_bounds__(MS_THREADS, 4) ms_heavy_kernel(MsArgs a) {
    __shared__ uint2 s_sw[MS_SETS];
    __shared__ uint32_t s_live[MS_WARPS][MS_SETS];
    __shared__ MsRound s_round[MS_WARPS];
    const uint32_t nH = min(a.mc->nH, a.heavy_cap);
    if (blockIdx.x * MS_WARPS >= nH) return;
    ms_init_shared(a, s_sw, s_live);
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t nblk = 0, nvis = 0;
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(&a.mc->hwork, 1u);
        it = __shfl_sync(0xFFFFFFFFu, it, 0);
        if (it >= nH) break;
        const uint4 item = a.heavy[it];  // one chunk per warp (work stealing)
        const uint32_t eb = __ldg(a.g.row_ptr + item.x), ee = __ldg(a.g.row_ptr + item.x + 1);
        for (uint32_t g = item.y; g < item.z; g += MS_ROUND) {
            const bool ok[2] = {g + lane < item.z, g + 32 + lane < item.z};
            const uint32_t gg[2] = {g + lane, g + 32 + lane}, ebs[2] = {eb, eb}, ees[2] = {ee, ee};
            const uint32_t ff[2] = {item.w, item.w};
            ms_round(a, s_round[warp], s_sw, s_live[warp], nblk, nvis, ok, gg, ebs, ees, ff);
        }
    }
    ms_flush_live(a, s_live, nblk, nvis);
}

// The vertices reached during the level, with the sets that had not visited
// them yet, join the next frontier (warp-aggregated appends); vis gains those
// sets and nxt is cleared.  A vertex of more than defer_groups edge groups may
// instead wait: its sets are kept in pend and it is reconsidered at the next
// compaction, at most defer_max times in a row, so that sets reaching it at
// nearby levels share one pass over its in-edges (and by then more of its
// sources are visited, so fewer coins are drawn).  The sets do not depend on
// when a member's in-edges are expanded.  When a level's frontier would be
// empty with vertices still waiting, the next compaction (force) takes them
// all.  A thread takes 4 vertices with 16-byte loads (the mask arrays are
// padded to a multiple of 4 entries; ndef holds one byte per vertex).
__global__ void __launch_bounds__(MS_THREADS) ms_compact_kernel(MsArgs a, bool after_level) {
    const bool force = a.mc->force != 0;
    if (after_level && a.mc->nF == 0 && !force) return;  // the search has ended: nxt is clear
    const uint32_t lane = threadIdx.x & 31, n4 = (a.g.n + 3) / 4;
    const uint32_t stride = gridDim.x * MS_THREADS;
    uint4* nxt4 = reinterpret_cast<uint4*>(a.nxt);
    uint4* vis4 = reinterpret_cast<uint4*>(a.vis);
    const uint4* pend4 = reinterpret_cast<const uint4*>(a.pend);
    uint32_t npend = 0;
    for (uint32_t q0 = blockIdx.x * MS_THREADS + (threadIdx.x & ~31u); q0 < n4; q0 += stride) {
        const uint32_t q = q0 + lane;
        uint32_t fw[4] = {0, 0, 0, 0};
        if (q < n4) {
            const uint4 x = nxt4[q];
            const uint32_t nd = a.ndef[q];
            if (x.x | x.y | x.z | x.w) {
                nxt4[q] = make_uint4(0, 0, 0, 0);
                const uint4 old = vis4[q];
                const uint4 f = make_uint4(x.x & ~old.x, x.y & ~old.y, x.z & ~old.z, x.w & ~old.w);
                if (f.x | f.y | f.z | f.w) vis4[q] = make_uint4(old.x | f.x, old.y | f.y, old.z | f.z, old.w | f.w);
                fw[0] = f.x;
                fw[1] = f.y;
                fw[2] = f.z;
                fw[3] = f.w;
            }
            if (nd) {
                const uint4 pd = pend4[q];
                const uint32_t pw[4] = {pd.x, pd.y, pd.z, pd.w};
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if ((nd >> (8 * k)) & 0xFFu) fw[k] |= pw[k];
            }
            if ((fw[0] | fw[1] | fw[2] | fw[3]) && a.defer_max && !force) {
                uint32_t nd2 = 0;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    if (!fw[k]) continue;
                    const uint32_t v = q * 4 + k;
                    const uint32_t b = __ldg(a.g.row_ptr + v), e = __ldg(a.g.row_ptr + v + 1);
                    const uint32_t ng = e > b ? ((e - 1) >> 2) - (b >> 2) + 1 : 0u;
                    const uint32_t d = (nd >> (8 * k)) & 0xFFu;
                    if (ng > a.defer_groups && d < a.defer_max) {
                        a.pend[v] = fw[k];
                        nd2 |= (d + 1) << (8 * k);
                        fw[k] = 0;
                        npend++;
                    }
                }
                if (nd2 != nd) a.ndef[q] = nd2;
            } else if (nd) {
                a.ndef[q] = 0;
            }
        }
        const uint32_t c = (fw[0] != 0) + (fw[1] != 0) + (fw[2] != 0) + (fw[3] != 0);
        const uint32_t incl = warp_incl_scan(c);
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        if (!total) continue;
        uint32_t pos = 0;
        if (lane == 31) pos = atomicAdd(&a.mc->nN, total);
        pos = __shfl_sync(0xFFFFFFFFu, pos, 31) + incl - c;
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (fw[k]) {
                a.F[pos] = q * 4 + k;
                a.Ff[pos] = fw[k];
                pos++;
            }
    }
    npend = __reduce_add_sync(0xFFFFFFFFu, npend);
    if (lane == 0 && npend) {
        atomicAdd(&a.mc->npend, npend);
        atomicAdd(&a.mc->deferred, (unsigned long long)npend);
    }
}

// Next level: the compacted list becomes the frontier; if it is empty while
// vertices wait, the next compaction takes them all.  <<<1, 1>>>
__global__ void ms_advance_kernel(MsArgs a) {
    MsCounters* c = a.mc;
    if (c->nF == 0 && c->nN == 0 && c->npend == 0 && !c->force) return;
    c->force = (c->nN == 0 && c->npend > 0) ? 1u : 0u;
    c->nF = c->nN;
    c->nN = 0;
    c->nH = 0;
    c->npend = 0;
    c->lwork = 0;
    c->hwork = 0;
}

// Size and scanned in-edges of each set of the batch, from the visited masks:
// lane s of every warp keeps set s's totals.
__global__ void __launch_bounds__(MS_THREADS) ms_tally_kernel(MsArgs a) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t n = a.g.n;
    unsigned long long size = 0, scanned = 0;
    const uint32_t stride = gridDim.x * MS_THREADS;
    for (uint32_t v0 = blockIdx.x * MS_THREADS + (threadIdx.x & ~31u); v0 < n; v0 += stride) {
        const uint32_t v = v0 + lane;
        uint32_t m = 0, d = 0;
        if (v < n) {
            m = a.vis[v];
            if (m) d = __ldg(a.g.row_ptr + v + 1) - __ldg(a.g.row_ptr + v);
        }
        uint32_t any = __reduce_or_sync(0xFFFFFFFFu, m);
        while (any) {
            const uint32_t s = __ffs(any) - 1;
            any &= any - 1;
            const bool in = (m >> s) & 1u;
            const uint32_t cnt = __popc(__ballot_sync(0xFFFFFFFFu, in));
            const uint32_t sd = __reduce_add_sync(0xFFFFFFFFu, in ? d : 0u);
            if (lane == s) {
                size += cnt;
                scanned += sd;
            }
        }
    }
    if (size) atomicAdd(&a.mc->size[lane], size);
    if (scanned) atomicAdd(&a.mc->scanned[lane], scanned);
}

// Bitmap rows of the dense sets (bit s of mask `dense`; row of set s at word
// offset rowoff[s] of the bitmap heap), and the masks cleared for the next
// batch.  A warp takes 32 words (1024 vertices) at a time.
__global__ void __launch_bounds__(MS_THREADS) ms_emit_kernel(MsArgs a, uint32_t dense, uint32_t* bm_heap) {
    __shared__ uint32_t tile[MS_WARPS][32][33];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t n = a.g.n, nw = (n + 31) / 32;
    const uint32_t nchunks = (nw + 31) / 32;
    for (uint32_t c = blockIdx.x * MS_WARPS + warp; c < nchunks; c += gridDim.x * MS_WARPS) {
        for (uint32_t wi = 0; wi < 32; wi++) {
            const uint32_t v = (c * 32 + wi) * 32 + lane;
            uint32_t m = 0;
            if (v < n) {
                m = a.vis[v];
                if (m) a.vis[v] = 0u;
            }
            uint32_t ds = dense;
            while (ds) {
                const uint32_t s = __ffs(ds) - 1;
                ds &= ds - 1;
                const uint32_t r = __ballot_sync(0xFFFFFFFFu, (m >> s) & 1u);
                if (lane == 0) tile[warp][s][wi] = r;
            }
        }
        __syncwarp();
        const uint32_t w = c * 32 + lane;
        uint32_t ds = dense;
        while (ds) {
            const uint32_t s = __ffs(ds) - 1;
            ds &= ds - 1;
            if (w < nw) bm_heap[a.rowoff[s] + w] = tile[warp][s][lane];
        }
        __syncwarp();
    }
}

// Records and pool counters of the batch's dense sets (MODE_ENCODE), or the
// dense-set count of a histogram pass.  <<<1, 32>>>
__global__ void ms_commit_kernel(MsArgs a, uint32_t dense, uint32_t mode, uint64_t row_words) {
    const uint32_t s = threadIdx.x;
    const bool d = (dense >> s) & 1u;
    unsigned long long verts = 0, sc = 0, lv = 0;
    if (mode == MODE_HIST && s < a.mc->nsets && a.sizes && a.sets[s] < a.sizes_cap)
        a.sizes[a.sets[s]] = (uint32_t)a.mc->size[s];
    if (d && mode == MODE_ENCODE) {
        a.recs[a.sets[s]] = make_rec(KIND_BITMAP, a.rowoff[s], (uint32_t)a.mc->size[s], 0);
        verts = a.mc->size[s];
    }
    // edges of the stored sets; a histogram pass counts those of its dense sets
    // too (the autotuner measures the work per set by them)
    if (d) {
        sc = a.mc->scanned[s];
        lv = a.mc->live[s];
    }
    for (int o = 16; o > 0; o >>= 1) {
        verts += __shfl_xor_sync(0xFFFFFFFFu, verts, o);
        sc += __shfl_xor_sync(0xFFFFFFFFu, sc, o);
        lv += __shfl_xor_sync(0xFFFFFFFFu, lv, o);
    }
    if (s == 0) {
        const unsigned long long nd = (unsigned long long)__popc(dense);
        if (mode == MODE_HIST) {
            atomicAdd(&a.ctr->hist_dense, nd);
        } else if (nd) {
            atomicAdd(&a.ctr->sets_bm, nd);
            atomicAdd(&a.ctr->sets_big, nd);
            atomicAdd(&a.ctr->rr_vertices, verts);
            atomicAdd(&a.ctr->words_used, nd * row_words);
        }
        if (sc) atomicAdd(&a.ctr->edges_scanned, sc);
        if (lv) atomicAdd(&a.ctr->edges_live, lv);
    }
}

// Vertex-major tile of a Bitmax pool (Section 4.2.3, Eq. (3)): the batch's
// slots are the tile's columns, so the visited masks are the tile's words;
// they are ORed into it (a tile may be filled over several batches) and
// cleared.
__global__ void __launch_bounds__(MS_THREADS) ms_tile_emit_kernel(MsArgs a, uint32_t* tile) {
    const uint32_t n4 = (a.g.n + 3) / 4;
    uint4* vis4 = reinterpret_cast<uint4*>(a.vis);
    uint4* t4 = reinterpret_cast<uint4*>(tile);
    for (uint32_t q = blockIdx.x * MS_THREADS + threadIdx.x; q < n4; q += gridDim.x * MS_THREADS) {
        const uint4 m = vis4[q];
        if (m.x | m.y | m.z | m.w) {
            const uint4 o = t4[q];
            t4[q] = make_uint4(o.x | m.x, o.y | m.y, o.z | m.z, o.w | m.w);
            vis4[q] = make_uint4(0, 0, 0, 0);
        }
    }
}

// Records and pool counters of a tile batch's sets (slot s = set 32t + s for
// the slots in `slots`); new_words: heap words the batch's tile adds (its
// first batch).  <<<1, 32>>>
__global__ void ms_tile_commit_kernel(MsArgs a, uint32_t slots, uint64_t tile_off, uint64_t new_words) {
    const uint32_t s = threadIdx.x;
    const bool on = (slots >> s) & 1u;
    unsigned long long verts = 0, sc = 0, lv = 0;
    if (on) {
        a.recs[a.sets[s]] = make_rec(KIND_BITMAP, tile_off, (uint32_t)a.mc->size[s], 0);
        verts = a.mc->size[s];
        sc = a.mc->scanned[s];
        lv = a.mc->live[s];
    }
    for (int o = 16; o > 0; o >>= 1) {
        verts += __shfl_xor_sync(0xFFFFFFFFu, verts, o);
        sc += __shfl_xor_sync(0xFFFFFFFFu, sc, o);
        lv += __shfl_xor_sync(0xFFFFFFFFu, lv, o);
    }
    if (s == 0) {
        const unsigned long long nd = (unsigned long long)__popc(slots);
        atomicAdd(&a.ctr->sets_bm, nd);
        atomicAdd(&a.ctr->sets_big, nd);
        atomicAdd(&a.ctr->rr_vertices, verts);
        if (new_words) atomicAdd(&a.ctr->words_used, (unsigned long long)new_words);
        if (sc) atomicAdd(&a.ctr->edges_scanned, sc);
        if (lv) atomicAdd(&a.ctr->edges_live, lv);
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static uint32_t ms_grid(const void* kernel, int sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, MS_THREADS, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    return (uint32_t)(sms * (per_sm > 0 ? per_sm : 1));
}

cudaError_t launch_ms_start(const MsArgs& a, int sms, cudaStream_t s) {
    ms_start_kernel<<<1, 32, 0, s>>>(a);
    ms_compact_kernel<<<(uint32_t)sms * 8, MS_THREADS, 0, s>>>(a, false);
    ms_advance_kernel<<<1, 1, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ms_level(const MsArgs& a, int sms, cudaStream_t s) {
    static const uint32_t gl = ms_grid((const void*)ms_light_kernel, sms);
    static const uint32_t gh = ms_grid((const void*)ms_heavy_kernel, sms);
    ms_light_kernel<<<gl, MS_THREADS, 0, s>>>(a);
    ms_heavy_kernel<<<gh, MS_THREADS, 0, s>>>(a);
    ms_compact_kernel<<<(uint32_t)sms * 8, MS_THREADS, 0, s>>>(a, true);
    ms_advance_kernel<<<1, 1, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ms_finish(const MsArgs& a, int sms, cudaStream_t s) {
    ms_tally_kernel<<<(uint32_t)sms * 4, MS_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ms_tile(const MsArgs& a, uint32_t slots, uint32_t* bm_heap, uint64_t tile_off,
                           uint64_t new_words, int sms, cudaStream_t s) {
    ms_tile_emit_kernel<<<(uint32_t)sms * 4, MS_THREADS, 0, s>>>(a, bm_heap + tile_off);
    ms_tile_commit_kernel<<<1, 32, 0, s>>>(a, slots, tile_off, new_words);
    return cudaGetLastError();
}

cudaError_t launch_ms_emit(const MsArgs& a, uint32_t dense, uint32_t mode, uint64_t row_words, uint32_t* bm_heap,
                           int sms, cudaStream_t s) {
    ms_emit_kernel<<<(uint32_t)sms * 2, MS_THREADS, 0, s>>>(a, mode == MODE_ENCODE ? dense : 0u, bm_heap);
    ms_commit_kernel<<<1, 32, 0, s>>>(a, dense, mode, row_words);
    return cudaGetLastError();
}

}  // namespace hbx

// ---------------------------------------------------------------------------
// Coin-block throughput ceiling: every thread finishes `per_thread` coin
// blocks back to back (the per-pair remainder of Philox4x32-10 that the search
// computes for each (edge group, set) pair, from distinct group words) and
// folds them into one word, so the kernel does nothing but the search's
// per-pair arithmetic.  Its rate is the ALU roofline of that search.
// ---------------------------------------------------------------------------
namespace hbx {

__global__ void __launch_bounds__(256) philox_ceiling_kernel(uint32_t per_thread, PhiloxKeys rk, uint32_t* out) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint2 S = ic_set_words(tid, 0u, rk);
    uint32_t acc = 0;
    for (uint32_t i = 0; i < per_thread; i++) {
        const uint4 x = ic_coins(make_uint4(i, tid ^ i, i * 0x9E3779B9u, tid + i), S, rk);
        acc ^= x.x ^ x.y ^ x.z ^ x.w;
    }
    out[tid] = acc;
}

cudaError_t launch_philox_ceiling(uint32_t blocks, uint32_t per_thread, uint32_t* out, cudaStream_t s) {
    philox_ceiling_kernel<<<blocks, 256, 0, s>>>(per_thread, philox_round_keys(0x243F6A88u, 0x85A308D3u), out);
    return cudaGetLastError();
}

}  // namespace hbx
