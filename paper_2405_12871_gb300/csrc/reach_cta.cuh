// reach_cta.cuh -- reach-only worlds with one CTA per world (kernel template).
//
// A CTA traverses one live-edge world (Sec. 2.1: coins by Philox on (world, edge),
// blocked nodes pre-marked as visited) level by level.  Per level:
//   phase 1  warps claim 32-node slices of the frontier from a shared counter.  A
//            warp scans its slice's 4-edge group counts with shuffles, and each
//            pass gives one group to each lane.  A lane finds its node by a
//            five-step shuffle search over the warp's running counts, so there is
//            no block-wide scan and no barrier inside the level.  A node with more
//            than BIG_GROUPS groups (a hub) goes to a shared list instead.
//   phase 2  the hubs' groups are cut into pieces of PIECE groups; warps claim
//            pieces, so a hub's edges spread over the whole CTA.
// A pass loads each lane's group (one 32-byte record: 4 targets, 4 coin thresholds),
// draws its four coins with one Philox call, and keeps the in-range live edges.  The
// warp stages them in shared memory, and each lane then claims one target in the
// visited bitmap (shared or global) with an atomic OR.  Newly visited nodes are
// appended to the queue with one shared atomic per warp ballot.  Every count equals
// that of the warp-per-world kernel, because the result of a world is a set.
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
    size_t off_queue;
};

constexpr int BIG_GROUPS = 32;   // nodes with more groups are expanded in phase 2
constexpr int PIECE = 128;       // groups per phase-2 claim
constexpr int BIGCAP = 256;      // hubs staged per level (further hubs stay in phase 1)
constexpr int CAND = 128;        // per-warp staging: 32 lanes x 4 edges

template <int BD>
struct Shared {
    int pp[BIGCAP + 1];   // running piece counts of the staged hubs
    int bb[BIGCAP], be[BIGCAP];
    int cand[BD / 32][CAND];
    int slice[2], nbig[2], piece[2], app[2];   // per level parity
    int task;
    uint32_t rel;
    unsigned long long edges;
};

struct World {
    const uint4 *ce;
    uint32_t *bm;
    int32_t *Q;
    uint32_t j, tag, inst, klo, khi;
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

// One pass: each active lane expands group g of a node whose edges are [ob, oe).
// Must be called by all 32 lanes of the warp.  Appends go to Q[tail + ...] through
// the level's append counter.
template <bool SMEM_BM>
__device__ __forceinline__ void expand_groups(bool act, int g, int ob, int oe, const World &W,
                                              int *cand, int *app, int tail, int lane,
                                              uint32_t lt_mask)
{
    uint32_t live = 0;
    int4 c4 = make_int4(0, 0, 0, 0);
    if (act) {
        const int4 *p = reinterpret_cast<const int4 *>(W.ce + 2 * (size_t)g);
        c4 = __ldg(p);
        const uint4 t4 = __ldg(reinterpret_cast<const uint4 *>(p + 1));
        const uint4 w = philox10_w(make_uint4((uint32_t)g, W.j, W.tag, W.inst), W.klo, W.khi);
        live = (uint32_t)((w.x >> 8) < t4.x) | ((uint32_t)((w.y >> 8) < t4.y) << 1) |
               ((uint32_t)((w.z >> 8) < t4.z) << 2) | ((uint32_t)((w.w >> 8) < t4.w) << 3);
        // edges of the group outside [ob, oe) belong to neighbouring nodes
        const int e0 = g << 2;
        if (e0 < ob) live &= 0xFu << (ob - e0);
        if (e0 + 4 > oe) live &= (1u << (oe - e0)) - 1u;
    }
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
    if (live & 1u) cand[off++] = c4.x;
    if (live & 2u) cand[off++] = c4.y;
    if (live & 4u) cand[off++] = c4.z;
    if (live & 8u) cand[off] = c4.w;
    __syncwarp();
    for (int k0 = 0; k0 < tot; k0 += 32) {
        const int k = k0 + lane;
        bool fresh = false;
        int v = 0;
        if (k < tot) {
            v = cand[k];
            const uint32_t bit = 1u << (v & 31);
            const uint32_t old = atomicOr(&W.bm[v >> 5], bit);
            fresh = !(old & bit);
        }
        const uint32_t bal = __ballot_sync(IMIN_FULL, fresh);
        if (bal) {
            int base = 0;
            if (lane == 0) base = atomicAdd(app, __popc(bal));
            base = __shfl_sync(IMIN_FULL, base, 0);
            if (fresh) W.Q[tail + base + __popc(bal & lt_mask)] = v;
        }
    }
    __syncwarp();
}

template <int BD, int MINB, bool SMEM_BM, bool STOP>
__global__ void __launch_bounds__(BD, MINB) cta_reach_kernel(const CArgs a)
{
    extern __shared__ uint32_t s_bm[];   // n bits when SMEM_BM
    __shared__ Shared<BD> sh;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    char *slot = a.slot_base + (size_t)blockIdx.x * a.slot_bytes;
    World W;
    W.bm = SMEM_BM ? s_bm : reinterpret_cast<uint32_t *>(slot);
    W.Q = reinterpret_cast<int32_t *>(slot + a.off_queue);
    int *const cand = sh.cand[warp];
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
            sh.app[1] = 0;
        }
        __syncthreads();
        const int got = sh.task;
        if (got < 0) break;
        ti = got;
        const uint32_t rel = sh.rel;
        const WTask &T = a.tasks[ti];
        const int32_t *const row_ptr = T.row_ptr;
        W.ce = T.ce;
        W.klo = (uint32_t)T.q.key;
        W.khi = (uint32_t)(T.q.key >> 32);
        W.tag = T.q.tag;
        W.inst = T.q.inst;
        const uint32_t wrel = T.list ? (T.list[rel] & 0x7fffffffu) : rel;
        W.j = (uint32_t)(T.first + (uint64_t)wrel);
        const int nS = T.q.nS;

        // ---- seeds, blocked nodes pre-marked as visited ----
        for (int i = tid; i < T.q.nB; i += BD) {
            const int v = T.q.B[i];
            atomicOr(&W.bm[v >> 5], 1u << (v & 31));
        }
        for (int i = tid; i < nS; i += BD) {
            const int s = T.q.S[i];
            atomicOr(&W.bm[s >> 5], 1u << (s & 31));
            W.Q[i] = s;
        }
        __syncthreads();
        int head = 0, tail = nS, lvl = 0;
        unsigned long long wedges = 0;
        while (head < tail) {
            const int p = lvl & 1;
            if (tid == 0) sh.slice[p ^ 1] = sh.nbig[p ^ 1] = sh.piece[p ^ 1] = 0;
            // ---- phase 1: 32-node slices, one warp each ----
            for (;;) {
                int sl = 0;
                if (lane == 0) sl = atomicAdd(&sh.slice[p], 1);
                sl = __shfl_sync(IMIN_FULL, sl, 0);
                const int base = head + sl * 32;
                if (base >= tail) break;
                const int i = base + lane;
                int b = 0, e = 0, cnt = 0;
                if (i < tail) {
                    const int u = W.Q[i];
                    b = row_ptr[u];
                    e = row_ptr[u + 1];
                    wedges += (unsigned long long)(e - b);
                    if (e > b) cnt = ((e + 3) >> 2) - (b >> 2);
                }
                const bool hub = cnt > BIG_GROUPS;
                const uint32_t hm = __ballot_sync(IMIN_FULL, hub);
                if (hm) {
                    int hb = 0;
                    if (lane == 0) hb = atomicAdd(&sh.nbig[p], __popc(hm));
                    hb = __shfl_sync(IMIN_FULL, hb, 0);
                    const int my = hb + __popc(hm & lt_mask);
                    if (hub && my < BIGCAP) {
                        sh.bb[my] = b;
                        sh.be[my] = e;
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
                    expand_groups<SMEM_BM>(t < total, (ob >> 2) + (t - ox), ob, oe, W, cand,
                                           &sh.app[p], tail, lane, lt_mask);
                }
            }
            __syncthreads();
            if (tid == 0) sh.app[p ^ 1] = 0;
            // ---- phase 2: hubs, in pieces of PIECE groups ----
            const int nb = min(sh.nbig[p], BIGCAP);
            if (nb > 0) {
                if (warp == 0) {
                    int carry = 0;
                    for (int c0 = 0; c0 < nb; c0 += 32) {
                        const int i = c0 + lane;
                        int np = 0;
                        if (i < nb) {
                            const int g = ((sh.be[i] + 3) >> 2) - (sh.bb[i] >> 2);
                            np = (g + PIECE - 1) / PIECE;
                        }
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
                    const int ob = sh.bb[lo], oe = sh.be[lo];
                    const int g0 = (ob >> 2) + (pc - sh.pp[lo]) * PIECE;
                    const int gend = min(g0 + PIECE, (oe + 3) >> 2);
                    for (int gs = g0; gs < gend; gs += 32)
                        expand_groups<SMEM_BM>(gs + lane < gend, gs + lane, ob, oe, W, cand, &sh.app[p],
                                               tail, lane, lt_mask);
                }
            }
            __syncthreads();
            const int ntail = tail + sh.app[p];
            head = tail;
            tail = ntail;
            ++lvl;
        }
        // ---- outputs ----
        if (T.out.reach)
            for (int i = tid; i < tail; i += BD) atomicAdd(T.out.reach + W.Q[i], 1ull);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wedges += __shfl_xor_sync(IMIN_FULL, wedges, o);
        if (lane == 0 && wedges) atomicAdd(&sh.edges, wedges);
        __syncthreads();
        if (tid == 0) {
            atomicAdd(T.out.acc + 0, (unsigned long long)tail);
            atomicAdd(T.out.acc + 1, sh.edges);
            if (STOP) atomicAdd(T.out.acc + 3, (unsigned long long)tail);
            atomicAdd(T.out.acc + 4, 1ull);
            if (T.out.world_spread) T.out.world_spread[wrel] = (uint32_t)tail;
        }
        // ---- clear the visited marks ----
        if (SMEM_BM) {
            for (size_t w = tid; w < a.bm_words; w += BD) s_bm[w] = 0;
        } else {
            for (int i = tid; i < tail; i += BD) W.bm[W.Q[i] >> 5] = 0;
            for (int i = tid; i < T.q.nB; i += BD) W.bm[T.q.B[i] >> 5] = 0;
        }
        __syncthreads();
    }
}

inline size_t static_smem(int bd)
{
    return (size_t)(3 * BIGCAP + 1 + (bd / 32) * CAND + 8 + 2) * 4 + 8 + 16;
}

template <int BD, int MINB, bool SMEM, bool STOP>
void launch_one(cudaStream_t st, const CArgs &a, int blocks, size_t smem)
{
    auto kern = cta_reach_kernel<BD, MINB, SMEM, STOP>;
    if (smem > 48 * 1024)
        IM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<blocks, BD, smem, st>>>(a);
    IM_CHECK_LAUNCH();
}

template <int BD, int MINB>
void launch(cudaStream_t st, const CArgs &a, int blocks, bool smem_bm, bool stop, size_t smem)
{
    if (smem_bm) {
        if (stop) launch_one<BD, MINB, true, true>(st, a, blocks, smem);
        else launch_one<BD, MINB, true, false>(st, a, blocks, smem);
    } else {
        if (stop) launch_one<BD, MINB, false, true>(st, a, blocks, smem);
        else launch_one<BD, MINB, false, false>(st, a, blocks, smem);
    }
}

// resident CTAs per SM (0 if the configuration cannot launch)
template <int BD, int MINB>
int occupancy(bool smem_bm, size_t smem)
{
    int nb = 0;
    cudaError_t e;
    if (smem_bm) {
        auto kern = cta_reach_kernel<BD, MINB, true, true>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BD, smem);
    } else {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cta_reach_kernel<BD, MINB, false, true>, BD, 0);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

// explicit instantiations live in reach_cta_<BD>.cu
#define IMIN_REACH_CTA_INSTANTIATE(BD_, MINB_)                                                          \
    template void launch<BD_, MINB_>(cudaStream_t, const CArgs &, int, bool, bool, size_t);            \
    template int occupancy<BD_, MINB_>(bool, size_t);

#define IMIN_REACH_CTA_EXTERN(BD_, MINB_)                                                               \
    extern template void launch<BD_, MINB_>(cudaStream_t, const CArgs &, int, bool, bool, size_t);     \
    extern template int occupancy<BD_, MINB_>(bool, size_t);

}  // namespace reach_cta
