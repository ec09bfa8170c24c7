// reach_cta.cuh -- one CTA per world: reach-only worlds and upper-bound (LRR) worlds.
//
// A CTA traverses one live-edge world (Sec. 2.1: coins by Philox on (world, edge),
// blocked nodes pre-marked as visited) breadth first, level by level.  Per level:
//   phase 1  warps claim 32-node slices of the frontier from a shared counter.  A
//            warp scans its slice's work-item counts with shuffles, and each pass gives
//            one item to each lane.  A lane finds its node by a five-step shuffle
//            search over the warp's running counts, so there is no block-wide scan and
//            no barrier inside the level.  A node with more than BIG items (a hub)
//            goes to a shared list instead.
//   phase 2  the hubs' items are cut into pieces of PIECE items; warps claim pieces,
//            so a hub's edges spread over the whole CTA.
// Forward, an item is a 4-edge group (one 32-byte record: 4 targets, 4 coin
// thresholds; one Philox call draws its four coins).  In reverse, an item is one
// in-edge.  A pass keeps each lane's live in-range edges; the warp stages them in
// shared memory, and each lane then claims one target in the visited bitmap (shared
// or global) with an atomic OR.  Newly visited nodes are appended to the queue with
// one shared atomic per warp ballot.
//
// Upper-bound worlds (Sec. 5.2, the Global Sampling bound) then draw the target t
// uniformly from V'_s.  If the forward pass reached t, they run the reverse BFS from
// t over live in-edges whose source the forward pass reached and which is not a seed
// (nor blocked).  That set is the world's LRR set; it is credited and stored.  Every
// count equals that of the warp-per-world kernel: a world's results are sets.
#pragma once

#include "common.cuh"

namespace reach_cta {

struct CArgs {
    const WTask *tasks;
    int ntasks;
    uint32_t *task_claim;
    uint32_t *task_done;
    char *slot_base;
    size_t slot_bytes;
    size_t bm_words;
    size_t off_queue, off_bm2, off_q2;
    // lower bound: node -> queue position, per position BFS level, dominator
    // estimate, subtree size, preorder rank, child cursor; level starts; edge pairs
    size_t off_loc, off_lvl, off_idom, off_sz, off_pre, off_cur, off_lstart, off_pu, off_pv;
    int ecap;
    uint32_t flags;
    int l2_keep;   // group records loaded with the evict-last L2 policy
};

constexpr int BIG = 32;       // nodes with more items are expanded in phase 2
constexpr int PIECE = 128;    // items per phase-2 claim
constexpr int BIGCAP = 256;   // hubs staged per level (further hubs stay in phase 1)
constexpr int CAND = 128;     // per-warp staging: 32 lanes x 4 edges

template <int BD, bool SRC = false>
struct Shared {
    int pp[BIGCAP + 1];   // running piece counts of the staged hubs
    int bb[BIGCAP], be[BIGCAP], bi[BIGCAP];   // hub edge range and queue position
    int cand[BD / 32][CAND];
    int cand2[SRC ? BD / 32 : 1][SRC ? CAND : 1];   // queue position of each candidate's source
    int slice[2], nbig[2], piece[2], app[2];   // per level parity
    int task;
    uint32_t rel;
    int target;
    int npairs;           // lower bound: live edges recorded
    int root;             // lower bound: preorder ranges handed to dominator-tree roots
    int nlev;
    unsigned long long edges;
    unsigned long long sbase;
};

// What a traversal records besides the queue.  NoRec: nothing (reach-only and the
// upper bound).  DomRec (lower bound): for each new node its queue position (loc), BFS
// level and BFS parent (the first estimate of its immediate dominator), and every live
// edge into a non-seed node as a (source position, target) pair.
struct NoRec {
    static constexpr bool kOn = false;
    __device__ __forceinline__ uint32_t filter(uint32_t live, const int4 &) const { return live; }
    __device__ __forceinline__ void on_new(int, int, int, int) const {}
    __device__ __forceinline__ bool want_pair(int) const { return false; }
    __device__ __forceinline__ void put_pair(int, int, int) const {}
    __device__ __forceinline__ void level_start(int, int) const {}
};

struct DomRec {
    static constexpr bool kOn = true;
    int32_t *loc, *lvl, *idom, *pu, *pv, *lstart;
    const uint32_t *seed_bm, *blocked_bm;
    int ecap;
    __device__ __forceinline__ static bool bit(const uint32_t *bm, int v)
    {
        return (__ldg(bm + (v >> 5)) >> (v & 31)) & 1u;
    }
    // blocked nodes are never entered: their in-edges are neither followed nor recorded
    __device__ __forceinline__ uint32_t filter(uint32_t live, const int4 &c4) const
    {
        if (!blocked_bm || !live) return live;
        if ((live & 1u) && bit(blocked_bm, c4.x)) live &= ~1u;
        if ((live & 2u) && bit(blocked_bm, c4.y)) live &= ~2u;
        if ((live & 4u) && bit(blocked_bm, c4.z)) live &= ~4u;
        if ((live & 8u) && bit(blocked_bm, c4.w)) live &= ~8u;
        return live;
    }
    __device__ __forceinline__ void on_new(int v, int pos, int src, int level) const
    {
        loc[v] = pos;
        lvl[pos] = level;
        idom[pos] = src;
    }
    __device__ __forceinline__ bool want_pair(int v) const { return !bit(seed_bm, v); }
    __device__ __forceinline__ void put_pair(int idx, int src, int v) const
    {
        if (idx < ecap) {
            pu[idx] = src;
            pv[idx] = v;
        }
    }
    __device__ __forceinline__ void level_start(int level, int head) const { lstart[level] = head; }
};

__device__ __forceinline__ uint4 philox10_w(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1,
                       (uint32_t)p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

struct Coins {
    uint32_t j, tag, inst, klo, khi;
};

// Forward items: the 4-edge groups of a node's out-edges [b, e).
// L2 cache policy for the graph's group records: with `keep`, evict-last (the records
// are re-read by every world in flight, the visited bitmaps and queues are not), else
// the normal policy.
__device__ __forceinline__ uint64_t graph_l2_policy(bool keep)
{
    uint64_t pol;
    if (keep)
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    else
        asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ uint4 ld_group_half(const void *p, uint64_t pol)
{
    uint4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}

struct Fwd {
    static constexpr bool kCountEdges = true;   // the scanned edges are reported
    const int32_t *row_ptr;
    const uint4 *ce;
    uint64_t pol;                    // L2 policy of the group loads
    const int2 *rng = nullptr;       // relabelled index (HotView): label -> [b, e)
    const uint32_t *gid = nullptr;   // relabelled index: group -> original group index
    __device__ __forceinline__ void range(int u, int &b, int &e) const
    {
        if (rng) {
            const int2 r = __ldg(rng + u);
            b = r.x;
            e = r.y;
        } else {
            b = row_ptr[u];
            e = row_ptr[u + 1];
        }
    }
    __device__ __forceinline__ static int first(int b) { return b >> 2; }
    __device__ __forceinline__ static int count(int b, int e) { return e > b ? ((e + 3) >> 2) - (b >> 2) : 0; }
    // live in-range edges of group g as a 4-bit mask, their targets in c4
    __device__ __forceinline__ uint32_t live(int g, int ob, int oe, const Coins &K, int4 &c4) const
    {
        const uint4 *p = ce + 2 * (size_t)g;
        const uint4 cu = ld_group_half(p, pol);
        c4 = make_int4((int)cu.x, (int)cu.y, (int)cu.z, (int)cu.w);
        const uint4 t4 = ld_group_half(p + 1, pol);
        const uint32_t gc = gid ? __ldg(gid + g) : (uint32_t)g;   // the coin counter
        const uint4 w = philox10_w(make_uint4(gc, K.j, K.tag, K.inst), K.klo, K.khi);
        uint32_t m = (uint32_t)((w.x >> 8) < t4.x) | ((uint32_t)((w.y >> 8) < t4.y) << 1) |
                     ((uint32_t)((w.z >> 8) < t4.z) << 2) | ((uint32_t)((w.w >> 8) < t4.w) << 3);
        // edges of the group outside [ob, oe) belong to neighbouring nodes
        const int e0 = g << 2;
        if (e0 < ob) m &= 0xFu << (ob - e0);
        if (e0 + 4 > oe) m &= (1u << (oe - e0)) - 1u;
        return m;
    }
};

// Reverse items: the in-edges [b, e) of a node; an in-edge (u, v) is followed when u
// was reached by the forward pass, u is neither a seed nor blocked, and its coin (the
// forward edge's) is live.
template <bool SMEM_BM>
struct Rev {
    static constexpr bool kCountEdges = false;
    const int32_t *in_ptr, *in_src, *in_eid;
    const uint32_t *in_thr;
    const uint32_t *fwd_bm, *seed_bm, *blocked_bm;
    __device__ __forceinline__ void range(int v, int &b, int &e) const
    {
        b = in_ptr[v];
        e = in_ptr[v + 1];
    }
    __device__ __forceinline__ static int first(int b) { return b; }
    __device__ __forceinline__ static int count(int b, int e) { return e - b; }
    __device__ __forceinline__ uint32_t live(int idx, int, int, const Coins &K, int4 &c4) const
    {
        const int u = __ldg(in_src + idx);
        const uint32_t fw = SMEM_BM ? fwd_bm[u >> 5] : __ldcg(fwd_bm + (u >> 5));
        if (!((fw >> (u & 31)) & 1u)) return 0;
        if ((__ldg(seed_bm + (u >> 5)) >> (u & 31)) & 1u) return 0;
        if (blocked_bm && ((__ldg(blocked_bm + (u >> 5)) >> (u & 31)) & 1u)) return 0;
        const int eid = __ldg(in_eid + idx);
        const uint32_t th = __ldg(in_thr + idx);
        const uint4 w = philox10_w(make_uint4((uint32_t)eid >> 2, K.j, K.tag, K.inst), K.klo, K.khi);
        const int c = eid & 3;
        const uint32_t word = c == 0 ? w.x : (c == 1 ? w.y : (c == 2 ? w.z : w.w));
        c4.x = u;
        return (word >> 8) < th ? 1u : 0u;
    }
};

// One pass over one item per lane (act): stage the live targets of the warp, claim
// them in bm and append the new ones to Q[tail + ...].  All 32 lanes must call it.
template <class Op, class Rec>
__device__ __forceinline__ void pass(const Op &op, const Rec &rec, bool act, int it, int ob, int oe, int src,
                                     int level, const Coins &K, uint32_t *bm, int32_t *Q, int *cand,
                                     int *cand2, int *app, int *npairs, int tail, int lane, uint32_t lt_mask)
{
    uint32_t live = 0;
    int4 c4 = make_int4(0, 0, 0, 0);
    if (act) live = rec.filter(op.live(it, ob, oe, K, c4), c4);
    const int nl = __popc(live);
    int incl = nl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(IMIN_FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const int tot = __shfl_sync(IMIN_FULL, incl, 31);
    if (tot == 0) return;
    int off = incl - nl;
    if (Rec::kOn)
        for (int c = 0; c < nl; ++c) cand2[off + c] = src;
    if (live & 1u) cand[off++] = c4.x;
    if (live & 2u) cand[off++] = c4.y;
    if (live & 4u) cand[off++] = c4.z;
    if (live & 8u) cand[off] = c4.w;
    __syncwarp();
    for (int k0 = 0; k0 < tot; k0 += 32) {
        const int k = k0 + lane;
        bool fresh = false, pair = false;
        int v = 0, sv = 0;
        if (k < tot) {
            v = cand[k];
            if (Rec::kOn) {
                sv = cand2[k];
                pair = rec.want_pair(v);
            }
            const uint32_t bit = 1u << (v & 31);
            const uint32_t old = atomicOr(&bm[v >> 5], bit);
            fresh = !(old & bit);
        }
        const uint32_t bal = __ballot_sync(IMIN_FULL, fresh);
        if (bal) {
            int base = 0;
            if (lane == 0) base = atomicAdd(app, __popc(bal));
            base = __shfl_sync(IMIN_FULL, base, 0);
            if (fresh) {
                const int pos = tail + base + __popc(bal & lt_mask);
                Q[pos] = v;
                rec.on_new(v, pos, sv, level + 1);
            }
        }
        if (Rec::kOn) {
            const uint32_t pb = __ballot_sync(IMIN_FULL, pair);
            if (pb) {
                int pbase = 0;
                if (lane == 0) pbase = atomicAdd(npairs, __popc(pb));
                pbase = __shfl_sync(IMIN_FULL, pbase, 0);
                if (pair) rec.put_pair(pbase + __popc(pb & lt_mask), sv, v);
            }
        }
    }
    __syncwarp();
}

// The same pass for traversals that record nothing besides the queue (reach-only and
// LRR worlds): each lane claims its own live targets directly, up to four independent
// atomics in flight per lane (no staging, one round trip to the bitmap), and the new
// nodes are appended at offsets taken from four ballots.  The queue order differs from
// the staged pass; a world's results are sets and do not depend on it.
template <class Op>
__device__ __forceinline__ void pass_direct(const Op &op, bool act, int it, int ob, int oe, const Coins &K,
                                            uint32_t *bm, int32_t *Q, int *app, int tail, int lane,
                                            uint32_t lt_mask)
{
    uint32_t live = 0;
    int4 c4 = make_int4(0, 0, 0, 0);
    if (act) live = op.live(it, ob, oe, K, c4);
    uint32_t o0 = ~0u, o1 = ~0u, o2 = ~0u, o3 = ~0u;
    const uint32_t m0 = 1u << (c4.x & 31), m1 = 1u << (c4.y & 31), m2 = 1u << (c4.z & 31),
                   m3 = 1u << (c4.w & 31);
    if (live & 1u) o0 = atomicOr(&bm[c4.x >> 5], m0);
    if (live & 2u) o1 = atomicOr(&bm[c4.y >> 5], m1);
    if (live & 4u) o2 = atomicOr(&bm[c4.z >> 5], m2);
    if (live & 8u) o3 = atomicOr(&bm[c4.w >> 5], m3);
    const bool f0 = !(o0 & m0), f1 = !(o1 & m1), f2 = !(o2 & m2), f3 = !(o3 & m3);
    const uint32_t b0 = __ballot_sync(IMIN_FULL, f0), b1 = __ballot_sync(IMIN_FULL, f1),
                   b2 = __ballot_sync(IMIN_FULL, f2), b3 = __ballot_sync(IMIN_FULL, f3);
    const int tot = __popc(b0) + __popc(b1) + __popc(b2) + __popc(b3);
    if (tot == 0) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(app, tot);
    base = __shfl_sync(IMIN_FULL, base, 0);
    int pos = tail + base + __popc(b0 & lt_mask) + __popc(b1 & lt_mask) + __popc(b2 & lt_mask) +
              __popc(b3 & lt_mask);
    if (f0) Q[pos++] = c4.x;
    if (f1) Q[pos++] = c4.y;
    if (f2) Q[pos++] = c4.z;
    if (f3) Q[pos] = c4.w;
}

template <class Op, class Rec>
__device__ __forceinline__ void pass_any(const Op &op, const Rec &rec, bool act, int it, int ob, int oe, int src,
                                         int level, const Coins &K, uint32_t *bm, int32_t *Q, int *cand,
                                         int *cand2, int *app, int *npairs, int tail, int lane,
                                         uint32_t lt_mask)
{
    if constexpr (Rec::kOn)
        pass(op, rec, act, it, ob, oe, src, level, K, bm, Q, cand, cand2, app, npairs, tail, lane, lt_mask);
    else
        pass_direct(op, act, it, ob, oe, K, bm, Q, app, tail, lane, lt_mask);
}

// Breadth-first expansion of Q[0, tail0) until no level adds a node; returns the
// final tail.  The caller zeroes the counters of both parities and passes a CTA
// barrier before the call; the call ends with a CTA barrier.
template <int BD, bool SRC, class Op, class Rec>
__device__ __forceinline__ int bfs(const Op &op, const Rec &rec, const Coins &K, uint32_t *bm, int32_t *Q,
                                   int tail0, Shared<BD, SRC> &sh, unsigned long long &wedges)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    int *const cand = sh.cand[warp];
    int *const cand2 = sh.cand2[SRC ? warp : 0];
    int head = 0, tail = tail0, lvl = 0;
    while (head < tail) {
        const int p = lvl & 1;
        if (tid == 0) {
            sh.slice[p ^ 1] = sh.nbig[p ^ 1] = sh.piece[p ^ 1] = 0;
            rec.level_start(lvl, head);
        }
        // ---- phase 1: 32-node slices, one warp each; the queue entries of the next
        // slice are read while the current one is expanded ----
        int sl = 0;
        if (lane == 0) sl = atomicAdd(&sh.slice[p], 1);
        sl = __shfl_sync(IMIN_FULL, sl, 0);
        int nbase = head + sl * 32;
        int nu = nbase + lane < tail ? Q[nbase + lane] : 0;
        for (;;) {
            const int base = nbase;
            if (base >= tail) break;
            const int i = base + lane;
            const int u = nu;
            if (lane == 0) sl = atomicAdd(&sh.slice[p], 1);
            sl = __shfl_sync(IMIN_FULL, sl, 0);
            nbase = head + sl * 32;
            nu = nbase + lane < tail ? Q[nbase + lane] : 0;
            int b = 0, e = 0, cnt = 0;
            if (i < tail) {
                op.range(u, b, e);
                cnt = Op::count(b, e);
                if (Op::kCountEdges) wedges += (unsigned long long)(e - b);
            }
            const bool hub = cnt > BIG;
            const uint32_t hm = __ballot_sync(IMIN_FULL, hub);
            if (hm) {
                int hb = 0;
                if (lane == 0) hb = atomicAdd(&sh.nbig[p], __popc(hm));
                hb = __shfl_sync(IMIN_FULL, hb, 0);
                const int my = hb + __popc(hm & lt_mask);
                if (hub && my < BIGCAP) {
                    sh.bb[my] = b;
                    sh.be[my] = e;
                    sh.bi[my] = i;
                    cnt = 0;
                }
            }
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(IMIN_FULL, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(IMIN_FULL, incl, 31);
            const int excl = incl - cnt;
            for (int t0 = 0; t0 < total; t0 += 32) {
                const int t = t0 + lane;
                // owner lane: the number of lanes whose running count is <= t
                int pos = 0;
#pragma unroll
                for (int s = 16; s >= 1; s >>= 1) {
                    const int c = __shfl_sync(IMIN_FULL, incl, pos + s - 1);
                    if (c <= t) pos += s;
                }
                const int ob = __shfl_sync(IMIN_FULL, b, pos);
                const int oe = __shfl_sync(IMIN_FULL, e, pos);
                const int ox = __shfl_sync(IMIN_FULL, excl, pos);
                pass_any(op, rec, t < total, Op::first(ob) + (t - ox), ob, oe, base + pos, lvl, K, bm, Q, cand,
                     cand2, &sh.app[p], &sh.npairs, tail, lane, lt_mask);
            }
        }
        __syncthreads();
        if (tid == 0) sh.app[p ^ 1] = 0;
        // ---- phase 2: hubs, in pieces of PIECE items ----
        const int nb = min(sh.nbig[p], BIGCAP);
        if (nb > 0) {
            if (warp == 0) {
                int carry = 0;
                for (int c0 = 0; c0 < nb; c0 += 32) {
                    const int i = c0 + lane;
                    int np = 0;
                    if (i < nb) np = (Op::count(sh.bb[i], sh.be[i]) + PIECE - 1) / PIECE;
                    int incl = np;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(IMIN_FULL, incl, o);
                        if (lane >= o) incl += y;
                    }
                    if (i < nb) sh.pp[i + 1] = carry + incl;
                    carry += __shfl_sync(IMIN_FULL, incl, 31);
                }
                if (lane == 0) sh.pp[0] = 0;
            }
            __syncthreads();
            const int npieces = sh.pp[nb];
            for (;;) {
                int pc = 0;
                if (lane == 0) pc = atomicAdd(&sh.piece[p], 1);
                pc = __shfl_sync(IMIN_FULL, pc, 0);
                if (pc >= npieces) break;
                int lo = 0, hi = nb;   // pp[lo] <= pc < pp[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (sh.pp[mid] <= pc) lo = mid; else hi = mid;
                }
                const int ob = sh.bb[lo], oe = sh.be[lo], oi = sh.bi[lo];
                const int i0 = Op::first(ob) + (pc - sh.pp[lo]) * PIECE;
                const int iend = min(i0 + PIECE, Op::first(ob) + Op::count(ob, oe));
                for (int is = i0; is < iend; is += 32)
                    pass_any(op, rec, is + lane < iend, is + lane, ob, oe, oi, lvl, K, bm, Q, cand, cand2, &sh.app[p],
                         &sh.npairs, tail, lane, lt_mask);
            }
        }
        __syncthreads();
        const int ntail = tail + sh.app[p];
        head = tail;
        tail = ntail;
        ++lvl;
    }
    if (tid == 0) {
        rec.level_start(lvl, tail);
        sh.nlev = lvl;
    }
    return tail;
}

// bump allocation that never overshoots `cap`; returns ~0ull on failure
__device__ __forceinline__ unsigned long long reserve_store(unsigned long long *cursor,
                                                            unsigned long long cnt,
                                                            unsigned long long cap)
{
    unsigned long long old = *(volatile unsigned long long *)cursor;
    for (int tries = 0; tries < (1 << 20); ++tries) {
        if (old + cnt > cap) return ~0ull;
        const unsigned long long prev = atomicCAS(cursor, old, old + cnt);
        if (prev == old) return old;
        old = prev;
    }
    return ~0ull;
}

template <int BD, int MINB, bool SMEM_BM, bool STOP, bool UPPER>
__global__ void __launch_bounds__(BD, MINB) cta_world_kernel(const CArgs a)
{
    extern __shared__ uint32_t s_bm[];   // n bits when SMEM_BM
    __shared__ Shared<BD> sh;

    const int tid = threadIdx.x, lane = tid & 31;
    char *slot = a.slot_base + (size_t)blockIdx.x * a.slot_bytes;
    uint32_t *const bm = SMEM_BM ? s_bm : reinterpret_cast<uint32_t *>(slot);
    int32_t *const Q = reinterpret_cast<int32_t *>(slot + a.off_queue);
    uint32_t *const bm2 = UPPER ? reinterpret_cast<uint32_t *>(slot + a.off_bm2) : nullptr;
    int32_t *const Q2 = UPPER ? reinterpret_cast<int32_t *>(slot + a.off_q2) : nullptr;
    const bool store = (a.flags & WF_STORE) != 0;
    if (SMEM_BM) {
        for (size_t w = tid; w < a.bm_words; w += BD) s_bm[w] = 0;
    }
    int ti = (int)(blockIdx.x % (unsigned)a.ntasks);
    for (;;) {
        // ---- claim a world (thread 0) ----
        if (tid == 0) {
            int got = -1;
            uint32_t rel = 0;
            for (int scan = 0; scan < a.ntasks; ++scan) {
                const int t = (ti + scan) % a.ntasks;
                if (*(volatile uint32_t *)(a.task_done + t)) continue;
                const WTask *tp = a.tasks + t;
                if (STOP && *(volatile unsigned long long *)(tp->out.acc + 3) >= tp->out.stop_T) {
                    a.task_done[t] = 1u;
                    continue;
                }
                const uint32_t r = atomicAdd(a.task_claim + t, 1u);
                if (r >= tp->count) {
                    a.task_done[t] = 1u;
                    continue;
                }
                got = t;
                rel = r;
                break;
            }
            sh.task = got;
            sh.rel = rel;
            sh.edges = 0;
            sh.slice[0] = sh.nbig[0] = sh.piece[0] = sh.app[0] = 0;
            sh.slice[1] = sh.nbig[1] = sh.piece[1] = sh.app[1] = 0;
        }
        __syncthreads();
        const int got = sh.task;
        if (got < 0) break;
        ti = got;
        const uint32_t rel = sh.rel;
        const WTask &T = a.tasks[ti];
        Coins K;
        K.klo = (uint32_t)T.q.key;
        K.khi = (uint32_t)(T.q.key >> 32);
        K.tag = T.q.tag;
        K.inst = T.q.inst;
        const uint32_t wrel = T.list ? (T.list[rel] & 0x7fffffffu) : rel;
        K.j = (uint32_t)(T.first + (uint64_t)wrel);
        const int nS = T.q.nS;

        // ---- seeds, blocked nodes pre-marked as visited ----
        for (int i = tid; i < T.q.nB; i += BD) {
            const int v = T.q.B[i];
            atomicOr(&bm[v >> 5], 1u << (v & 31));
        }
        for (int i = tid; i < nS; i += BD) {
            const int s = T.q.S[i];
            atomicOr(&bm[s >> 5], 1u << (s & 31));
            Q[i] = s;
        }
        __syncthreads();
        unsigned long long wedges = 0;
        const Fwd fwd{T.row_ptr, T.ce, graph_l2_policy(a.l2_keep != 0)};
        const int tail = bfs<BD, false>(fwd, NoRec{}, K, bm, Q, nS, sh, wedges);

        // ---- upper bound: target from V'_s, reverse BFS inside the reached set ----
        int tail2 = 0;
        bool defer = false;
        if (UPPER) {
            if (tid == 0) {
                int tn = -1;
                if (T.q.nVs > 0) {
                    const uint4 w = philox10_w(make_uint4(0xFFFFFFFFu, K.j, K.tag, K.inst), K.klo, K.khi);
                    const unsigned long long r64 = ((unsigned long long)w.y << 32) | w.x;
                    const unsigned long long idx = __umul64hi(r64, (unsigned long long)T.q.nVs);
                    const int t = T.q.Vs[idx];
                    const uint32_t fw = SMEM_BM ? bm[t >> 5] : __ldcg(bm + (t >> 5));
                    const bool blk = T.q.blocked_bm && ((T.q.blocked_bm[t >> 5] >> (t & 31)) & 1u);
                    if (((fw >> (t & 31)) & 1u) && !blk) tn = t;
                }
                if (tn >= 0) {
                    atomicOr(&bm2[tn >> 5], 1u << (tn & 31));
                    Q2[0] = tn;
                }
                sh.target = tn;
                sh.slice[0] = sh.nbig[0] = sh.piece[0] = sh.app[0] = 0;
                sh.slice[1] = sh.nbig[1] = sh.piece[1] = sh.app[1] = 0;
            }
            __syncthreads();
            if (sh.target >= 0) {
                const Rev<SMEM_BM> rev{T.in_ptr, T.in_src, T.in_eid, T.in_thr, bm, T.q.seed_bm,
                                       T.q.blocked_bm};
                tail2 = bfs<BD, false>(rev, NoRec{}, K, bm2, Q2, 1, sh, wedges);
            }
            if (store) {
                if (tid == 0)
                    sh.sbase = tail2 > 0 ? reserve_store(T.out.set_cursor, (unsigned long long)tail2,
                                                         T.out.set_cap)
                                         : 0ull;
                __syncthreads();
                defer = sh.sbase == ~0ull;
            }
        }

        if (defer) {
            // no store room: the world contributes nothing and is re-run after the host
            // grows the store
            if (tid == 0) {
                const uint32_t d = atomicAdd(T.out.n_deferred, 1u);
                if (d < T.out.deferred_cap)
                    T.out.deferred[d] = wrel;
                else
                    atomicOr(T.out.err, DERR_INTERNAL);
            }
        } else {
            // ---- outputs ----
            if (T.out.reach)
                for (int i = tid; i < tail; i += BD) atomicAdd(T.out.reach + Q[i], 1ull);
            if (UPPER) {
                if (T.out.credit_U)
                    for (int i = tid; i < tail2; i += BD) atomicAdd(T.out.credit_U + Q2[i], 1ull);
                if (store) {
                    const unsigned long long sb = sh.sbase;
                    for (int i = tid; i < tail2; i += BD) T.out.set_elem[sb + i] = Q2[i];
                    if (tid == 0) {
                        T.out.set_off[wrel] = sb;
                        T.out.set_len[wrel] = (uint32_t)tail2;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wedges += __shfl_xor_sync(IMIN_FULL, wedges, o);
            if (lane == 0 && wedges) atomicAdd(&sh.edges, wedges);
            __syncthreads();
            if (tid == 0) {
                atomicAdd(T.out.acc + 0, (unsigned long long)tail);
                atomicAdd(T.out.acc + 1, sh.edges);
                if (UPPER && tail2 > 0) atomicAdd(T.out.acc + 2, 1ull);
                if (STOP) atomicAdd(T.out.acc + 3, (unsigned long long)tail);
                atomicAdd(T.out.acc + 4, 1ull);
                if (T.out.world_spread) T.out.world_spread[wrel] = (uint32_t)tail;
            }
        }
        // ---- clear the visited marks ----
        if (UPPER)
            for (int i = tid; i < tail2; i += BD) bm2[Q2[i] >> 5] = 0;
        if (SMEM_BM) {
            __syncthreads();
            for (size_t w = tid; w < a.bm_words; w += BD) s_bm[w] = 0;
        } else {
            for (int i = tid; i < tail; i += BD) bm[Q[i] >> 5] = 0;
            for (int i = tid; i < T.q.nB; i += BD) bm[T.q.B[i] >> 5] = 0;
        }
        __syncthreads();
    }
}

// LCA of queue positions a and b in the current dominator-estimate tree (-1 = the
// virtual root s): the deeper one (by BFS level) steps to its estimate until they meet.
__device__ __forceinline__ int dt_lca(int a, int b, const int32_t *lvl, const int32_t *idom, int nS)
{
    for (int guard = 0; guard < (1 << 22) && a != b; ++guard) {
        const int la = a < 0 ? -1 : lvl[a];
        const int lb = b < 0 ? -1 : lvl[b];
        if (la >= lb)
            a = (a < nS) ? -1 : __ldcg(idom + a);
        else
            b = (b < nS) ? -1 : __ldcg(idom + b);
    }
    return a;
}

// Lower-bound worlds (Algorithm 2, Local Sampling; Sec. 4): one CTA per world.
//   1. forward BFS recording positions, levels, BFS parents and live edge pairs;
//   2. immediate dominators by repeated relaxation idom(v) <- LCA(idom(v), u) over the
//      live edges (u, v) until a pass changes nothing (a dominator is an ancestor in
//      every BFS tree, so the BFS parents are a valid first estimate);
//   3. subtree sizes bottom-up by level, credit_L[v] += subtree size (the number of
//      CP sets containing v);
//   4. CP records in dominator-tree preorder: node, distance back to the parent record
//      (0 for a root), subtree size.
// A world whose edge pairs overflow the slot is deferred to a large slot (top bit),
// one that finds no store room is deferred until the host grows the store.
template <int BD, int MINB, bool SMEM_BM>
__global__ void __launch_bounds__(BD, MINB) cta_lower_kernel(const CArgs a)
{
    extern __shared__ uint32_t s_bm[];
    __shared__ Shared<BD, true> sh;

    const int tid = threadIdx.x, lane = tid & 31;
    char *slot = a.slot_base + (size_t)blockIdx.x * a.slot_bytes;
    uint32_t *const bm = SMEM_BM ? s_bm : reinterpret_cast<uint32_t *>(slot);
    int32_t *const Q = reinterpret_cast<int32_t *>(slot + a.off_queue);
    int32_t *const loc = reinterpret_cast<int32_t *>(slot + a.off_loc);
    int32_t *const lvl = reinterpret_cast<int32_t *>(slot + a.off_lvl);
    int32_t *const idom = reinterpret_cast<int32_t *>(slot + a.off_idom);
    int32_t *const sz = reinterpret_cast<int32_t *>(slot + a.off_sz);
    int32_t *const pre = reinterpret_cast<int32_t *>(slot + a.off_pre);
    int32_t *const cur = reinterpret_cast<int32_t *>(slot + a.off_cur);
    int32_t *const lstart = reinterpret_cast<int32_t *>(slot + a.off_lstart);
    int32_t *const pu = reinterpret_cast<int32_t *>(slot + a.off_pu);
    int32_t *const pv = reinterpret_cast<int32_t *>(slot + a.off_pv);
    const bool store = (a.flags & WF_STORE) != 0;
    if (SMEM_BM) {
        for (size_t w = tid; w < a.bm_words; w += BD) s_bm[w] = 0;
    }
    int ti = (int)(blockIdx.x % (unsigned)a.ntasks);
    for (;;) {
        if (tid == 0) {
            int got = -1;
            uint32_t rel = 0;
            for (int scan = 0; scan < a.ntasks; ++scan) {
                const int t = (ti + scan) % a.ntasks;
                if (*(volatile uint32_t *)(a.task_done + t)) continue;
                const uint32_t r = atomicAdd(a.task_claim + t, 1u);
                if (r >= a.tasks[t].count) {
                    a.task_done[t] = 1u;
                    continue;
                }
                got = t;
                rel = r;
                break;
            }
            sh.task = got;
            sh.rel = rel;
            sh.edges = 0;
            sh.npairs = 0;
            sh.root = 0;
            sh.slice[0] = sh.nbig[0] = sh.piece[0] = sh.app[0] = 0;
            sh.slice[1] = sh.nbig[1] = sh.piece[1] = sh.app[1] = 0;
        }
        __syncthreads();
        const int got = sh.task;
        if (got < 0) break;
        ti = got;
        const uint32_t rel = sh.rel;
        const WTask &T = a.tasks[ti];
        Coins K;
        K.klo = (uint32_t)T.q.key;
        K.khi = (uint32_t)(T.q.key >> 32);
        K.tag = T.q.tag;
        K.inst = T.q.inst;
        const uint32_t wrel = T.list ? (T.list[rel] & 0x7fffffffu) : rel;
        K.j = (uint32_t)(T.first + (uint64_t)wrel);
        const int nS = T.q.nS;

        // ---- 1. forward BFS from the seeds (blocked nodes are filtered, not marked) ----
        for (int i = tid; i < nS; i += BD) {
            const int s = T.q.S[i];
            atomicOr(&bm[s >> 5], 1u << (s & 31));
            Q[i] = s;
            loc[s] = i;
            lvl[i] = 0;
            idom[i] = -1;
        }
        __syncthreads();
        unsigned long long wedges = 0;
        const Fwd fwd{T.row_ptr, T.ce, graph_l2_policy(a.l2_keep != 0)};
        const DomRec rec{loc, lvl, idom, pu, pv, lstart, T.q.seed_bm, T.q.blocked_bm, a.ecap};
        const int tail = bfs<BD, true>(fwd, rec, K, bm, Q, nS, sh, wedges);
        __syncthreads();
        const int L = sh.nlev;
        const int npairs = sh.npairs;
        const bool big = npairs > a.ecap;
        bool defer = big;

        if (!big) {
            // ---- 2. immediate dominators ----
            for (int k = tid; k < npairs; k += BD) pv[k] = loc[pv[k]];
            for (int i = tid; i < tail; i += BD) {
                sz[i] = i < nS ? 0 : 1;
                cur[i] = 0;
            }
            __syncthreads();
            for (int it = 0;; ++it) {
                int changed = 0;
                for (int k = tid; k < npairs; k += BD) {
                    const int i = pv[k];
                    if (i < nS) continue;
                    const int p = pu[k];
                    int c0 = __ldcg(idom + i);
                    for (int guard = 0; guard < (1 << 22); ++guard) {
                        const int c = dt_lca(c0, p, lvl, idom, nS);
                        if (c == c0) break;
                        const int old = atomicCAS(idom + i, c0, c);
                        if (old == c0) {
                            changed = 1;
                            break;
                        }
                        c0 = old;
                    }
                }
                if (!__syncthreads_or(changed)) break;
                if (it > (1 << 20)) {
                    if (tid == 0) atomicOr(T.out.err, DERR_TIMEOUT);
                    break;
                }
            }
            // ---- 3. subtree sizes, deepest level first ----
            for (int lv = L - 1; lv >= 1; --lv) {
                const int s0 = lstart[lv], s1 = lstart[lv + 1];
                for (int i = s0 + tid; i < s1; i += BD) {
                    const int d = __ldcg(idom + i);
                    if (d >= nS) atomicAdd(sz + d, __ldcg(sz + i));
                }
                __syncthreads();
            }
            if (store) {
                if (tid == 0)
                    sh.sbase = reserve_store(T.out.rec_cursor, (unsigned long long)(tail - nS), T.out.rec_cap);
                __syncthreads();
                defer = sh.sbase == ~0ull;
            }
        }

        if (defer) {
            if (tid == 0) {
                const uint32_t d = atomicAdd(T.out.n_deferred, 1u);
                if (d < T.out.deferred_cap)
                    T.out.deferred[d] = wrel | (big ? 0x80000000u : 0u);
                else
                    atomicOr(T.out.err, DERR_INTERNAL);
            }
        } else {
            // ---- 4. outputs ----
            if (T.out.credit_L)
                for (int i = nS + tid; i < tail; i += BD)
                    atomicAdd(T.out.credit_L + Q[i], (unsigned long long)__ldcg(sz + i));
            if (store) {
                const unsigned long long sb = sh.sbase;
                for (int lv = 1; lv < L; ++lv) {
                    const int s0 = lstart[lv], s1 = lstart[lv + 1];
                    for (int i = s0 + tid; i < s1; i += BD) {
                        const int d = __ldcg(idom + i);
                        const int size_i = __ldcg(sz + i);
                        int pr, poff;
                        if (d < nS) {
                            pr = atomicAdd(&sh.root, size_i);
                            poff = 0;
                        } else {
                            const int pd = __ldcg(pre + d);
                            pr = pd + 1 + atomicAdd(cur + d, size_i);
                            poff = pr - pd;
                        }
                        pre[i] = pr;
                        const unsigned long long r = sb + (unsigned long long)pr;
                        T.out.rec_node[r] = Q[i];
                        T.out.rec_par[r] = poff;
                        T.out.rec_size[r] = size_i;
                    }
                    __syncthreads();
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wedges += __shfl_xor_sync(IMIN_FULL, wedges, o);
            if (lane == 0 && wedges) atomicAdd(&sh.edges, wedges);
            __syncthreads();
            if (tid == 0) {
                atomicAdd(T.out.acc + 0, (unsigned long long)tail);
                atomicAdd(T.out.acc + 1, sh.edges);
                atomicAdd(T.out.acc + 4, 1ull);
                if (T.out.world_spread) T.out.world_spread[wrel] = (uint32_t)tail;
            }
            if (T.out.reach)
                for (int i = tid; i < tail; i += BD) atomicAdd(T.out.reach + Q[i], 1ull);
        }
        // ---- clear the visited marks ----
        if (SMEM_BM) {
            __syncthreads();
            for (size_t w = tid; w < a.bm_words; w += BD) s_bm[w] = 0;
        } else {
            for (int i = tid; i < tail; i += BD) bm[Q[i] >> 5] = 0;
        }
        __syncthreads();
    }
}

inline size_t static_smem(int bd, bool lower = false)
{
    return (size_t)(4 * BIGCAP + 1 + (lower ? 2 : 1) * (bd / 32) * CAND + 8 + 6 + (lower ? 0 : 1)) * 4 + 16 + 16;
}

template <int BD, int MINB, bool SMEM, bool STOP, bool UPPER>
void launch_one(cudaStream_t st, const CArgs &a, int blocks, size_t smem)
{
    auto kern = cta_world_kernel<BD, MINB, SMEM, STOP, UPPER>;
    if (smem > 0)
        IM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<blocks, BD, smem, st>>>(a);
    IM_CHECK_LAUNCH();
}

template <int BD, int MINB, bool SMEM>
void launch_lower(cudaStream_t st, const CArgs &a, int blocks, size_t smem)
{
    auto kern = cta_lower_kernel<BD, MINB, SMEM>;
    if (smem > 0)
        IM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<blocks, BD, smem, st>>>(a);
    IM_CHECK_LAUNCH();
}

// kind: 0 reach-only, 1 reach-only with the stopping rule, 2 upper bound, 3 lower bound
template <int BD, int MINB>
void launch(cudaStream_t st, const CArgs &a, int blocks, bool smem_bm, int kind, size_t smem)
{
    if (kind == 3) {
        if (smem_bm) launch_lower<BD, MINB, true>(st, a, blocks, smem);
        else launch_lower<BD, MINB, false>(st, a, blocks, smem);
        return;
    }
    if (smem_bm) {
        if (kind == 2) launch_one<BD, MINB, true, false, true>(st, a, blocks, smem);
        else if (kind == 1) launch_one<BD, MINB, true, true, false>(st, a, blocks, smem);
        else launch_one<BD, MINB, true, false, false>(st, a, blocks, smem);
    } else {
        if (kind == 2) launch_one<BD, MINB, false, false, true>(st, a, blocks, smem);
        else if (kind == 1) launch_one<BD, MINB, false, true, false>(st, a, blocks, smem);
        else launch_one<BD, MINB, false, false, false>(st, a, blocks, smem);
    }
}

// resident CTAs per SM (0 if the configuration cannot launch)
template <int BD, int MINB>
int occupancy(bool smem_bm, bool upper, bool lower, size_t smem)
{
    int nb = 0;
    cudaError_t e;
    if (lower) {
        auto kern = smem_bm ? cta_lower_kernel<BD, MINB, true> : cta_lower_kernel<BD, MINB, false>;
        if (smem > 0) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BD, smem);
    } else if (smem_bm) {
        auto kern = upper ? cta_world_kernel<BD, MINB, true, false, true>
                          : cta_world_kernel<BD, MINB, true, true, false>;
        if (smem > 0) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BD, smem);
    } else {
        auto kern = upper ? cta_world_kernel<BD, MINB, false, false, true>
                          : cta_world_kernel<BD, MINB, false, true, false>;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BD, 0);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

// explicit instantiations live in reach_cta_<BD>.cu
#define IMIN_REACH_CTA_INSTANTIATE(BD_, MINB_)                                                          \
    template void launch<BD_, MINB_>(cudaStream_t, const CArgs &, int, bool, int, size_t);             \
    template int occupancy<BD_, MINB_>(bool, bool, bool, size_t);

#define IMIN_REACH_CTA_EXTERN(BD_, MINB_)                                                               \
    extern template void launch<BD_, MINB_>(cudaStream_t, const CArgs &, int, bool, int, size_t);      \
    extern template int occupancy<BD_, MINB_>(bool, bool, bool, size_t);

}  // namespace reach_cta
