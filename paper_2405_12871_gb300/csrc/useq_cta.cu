// useq_cta.cu -- LRR sequences (Sec. 4.2, "Discussion" after Algorithm 3): in every
// world, the LRR set of EVERY node of phi^s = R_phi(s) \ S, i.e. one reverse closure
// per reached node.  The paper rejects this estimator of D^U on a CPU because it
// needs |R \ S| traversals per world (Table 2); here one CTA handles a world and its
// warps run the closures side by side.
//
// Per world (one CTA):
//   1. forward breadth-first traversal from the seeds (blocked nodes never entered),
//      recording each node's queue position and every live edge into a non-seed node
//      as a (source position, target) pair;
//   2. the reverse adjacency of phi^s over queue positions: the recorded edges whose
//      source is not a seed, bucketed by target (count, block scan, fill);
//   3. each warp takes target positions t in turn and traverses the reverse adjacency
//      from t (its visited set is a per-warp bitmap over positions): the closure is
//      L_phi(v_t).  Every member's counter is raised by one, and the closure meets the
//      query set when one of its nodes is in it;
//   4. credit_useq[u] += counter of u (= |M_phi({u})|), the world's coverage of the
//      query set |M_phi(Q)| and the element count sum |L_phi(v)| are written out.
#include "reach_cta.cuh"

#include <cstdlib>

namespace useq_cta {

using reach_cta::Coins;
using reach_cta::Fwd;
using reach_cta::Shared;

constexpr int BD = 256;
constexpr int WARPS = BD / 32;

// the forward pass records positions and live edge pairs (compare DomRec)
struct PairRec {
    static constexpr bool kOn = true;
    int32_t *loc, *pu, *pv;
    const uint32_t *seed_bm, *blocked_bm;
    int ecap;
    __device__ __forceinline__ static bool bit(const uint32_t *bm, int v)
    {
        return (__ldg(bm + (v >> 5)) >> (v & 31)) & 1u;
    }
    __device__ __forceinline__ uint32_t filter(uint32_t live, const int4 &c4) const
    {
        if (!blocked_bm || !live) return live;
        if ((live & 1u) && bit(blocked_bm, c4.x)) live &= ~1u;
        if ((live & 2u) && bit(blocked_bm, c4.y)) live &= ~2u;
        if ((live & 4u) && bit(blocked_bm, c4.z)) live &= ~4u;
        if ((live & 8u) && bit(blocked_bm, c4.w)) live &= ~8u;
        return live;
    }
    __device__ __forceinline__ void on_new(int v, int pos, int, int) const { loc[v] = pos; }
    __device__ __forceinline__ bool want_pair(int v) const { return !bit(seed_bm, v); }
    __device__ __forceinline__ void put_pair(int idx, int src, int v) const
    {
        if (idx < ecap) {
            pu[idx] = src;
            pv[idx] = v;
        }
    }
    __device__ __forceinline__ void level_start(int, int) const {}
};

struct UArgs {
    const int32_t *row_ptr;
    const uint4 *ce;
    const int32_t *S;
    int32_t nS;
    const uint32_t *seed_bm, *blocked_bm, *query_bm;
    Coins K0;                 // key, tag, inst (j set per world)
    uint64_t first;
    uint32_t count;
    uint32_t *claim;
    char *slot_base;
    size_t slot_bytes;
    size_t off_q, off_loc, off_pu, off_pv, off_rptr, off_rcur, off_radj, off_cnt, off_wq, off_wb;
    int32_t qcap;             // n + 1
    size_t words;             // bitmap words of qcap bits
    int32_t ecap;
    int l2_keep;
    unsigned long long *credit;      // [n] or null
    unsigned long long *cov_world;   // [count] or null
    unsigned long long *acc;         // [0] elements [1] coverage [2] nodes [3] edges [4] worlds
    uint32_t *err;
};

__global__ void __launch_bounds__(BD, 2) useq_kernel(const UArgs a)
{
    __shared__ Shared<BD, true> sh;
    __shared__ int s_target;
    __shared__ int s_wtail[WARPS];
    __shared__ unsigned long long s_elems, s_cov;
    __shared__ int s_carry;
    __shared__ int s_wsum[WARPS];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    char *slot = a.slot_base + (size_t)blockIdx.x * a.slot_bytes;
    uint32_t *const bm = reinterpret_cast<uint32_t *>(slot);
    int32_t *const Q = reinterpret_cast<int32_t *>(slot + a.off_q);
    int32_t *const loc = reinterpret_cast<int32_t *>(slot + a.off_loc);
    int32_t *const pu = reinterpret_cast<int32_t *>(slot + a.off_pu);
    int32_t *const pv = reinterpret_cast<int32_t *>(slot + a.off_pv);
    int32_t *const rptr = reinterpret_cast<int32_t *>(slot + a.off_rptr);
    int32_t *const rcur = reinterpret_cast<int32_t *>(slot + a.off_rcur);
    int32_t *const radj = reinterpret_cast<int32_t *>(slot + a.off_radj);
    int32_t *const cnt = reinterpret_cast<int32_t *>(slot + a.off_cnt);
    int32_t *const wq = reinterpret_cast<int32_t *>(slot + a.off_wq) + (size_t)warp * a.qcap;
    uint32_t *const wb = reinterpret_cast<uint32_t *>(slot + a.off_wb) + (size_t)warp * a.words;
    const int nS = a.nS;
    for (;;) {
        if (tid == 0) {
            const uint32_t r = atomicAdd(a.claim, 1u);
            sh.rel = r;
            sh.task = r < a.count ? 0 : -1;
            sh.edges = 0;
            sh.npairs = 0;
            s_elems = 0;
            s_cov = 0;
            sh.slice[0] = sh.nbig[0] = sh.piece[0] = sh.app[0] = 0;
            sh.slice[1] = sh.nbig[1] = sh.piece[1] = sh.app[1] = 0;
        }
        __syncthreads();
        if (sh.task < 0) break;
        const uint32_t rel = sh.rel;
        Coins K = a.K0;
        K.j = (uint32_t)(a.first + (uint64_t)rel);

        // ---- 1. forward traversal recording positions and live pairs ----
        for (int i = tid; i < nS; i += BD) {
            const int s = a.S[i];
            atomicOr(&bm[s >> 5], 1u << (s & 31));
            Q[i] = s;
            loc[s] = i;
        }
        __syncthreads();
        unsigned long long wedges = 0;
        const Fwd fwd{a.row_ptr, a.ce, reach_cta::graph_l2_policy(a.l2_keep != 0)};
        const PairRec rec{loc, pu, pv, a.seed_bm, a.blocked_bm, a.ecap};
        const int tail = reach_cta::bfs<BD, true>(fwd, rec, K, bm, Q, nS, sh, wedges);
        __syncthreads();
        const int npairs = sh.npairs;
        const bool fits = npairs <= a.ecap;
        if (!fits && tid == 0) atomicOr(a.err, 4u);   // pairs overflow: the call fails

        if (fits) {
            // ---- 2. reverse adjacency of phi^s over positions ----
            for (int i = tid; i <= tail; i += BD) rptr[i] = 0;
            __syncthreads();
            for (int k = tid; k < npairs; k += BD) {
                const int s = pu[k];
                if (s >= nS) atomicAdd(&rptr[loc[pv[k]] + 1], 1);
            }
            __syncthreads();
            // inclusive scan of rptr[1..tail] in chunks of BD (rptr[0] = 0)
            if (tid == 0) s_carry = 0;
            __syncthreads();
            for (int c0 = 1; c0 <= tail; c0 += BD) {
                const int i = c0 + tid;
                int x = i <= tail ? rptr[i] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(IMIN_FULL, x, o);
                    if (lane >= o) x += y;
                }
                if (lane == 31) s_wsum[warp] = x;
                __syncthreads();
                int add = s_carry;
                for (int w2 = 0; w2 < warp; ++w2) add += s_wsum[w2];
                if (i <= tail) rptr[i] = x + add;
                __syncthreads();
                if (tid == BD - 1) s_carry = x + add;
                __syncthreads();
            }
            for (int i = tid; i < tail; i += BD) rcur[i] = rptr[i];
            __syncthreads();
            for (int k = tid; k < npairs; k += BD) {
                const int s = pu[k];
                if (s >= nS) {
                    const int t = loc[pv[k]];
                    radj[atomicAdd(&rcur[t], 1)] = s;
                }
            }
            if (tid == 0) s_target = nS;
            __syncthreads();

            // ---- 3. one reverse closure per node of phi^s, a warp at a time ----
            unsigned long long my_elems = 0, my_cov = 0;
            for (;;) {
                int t = 0;
                if (lane == 0) t = atomicAdd(&s_target, 1);
                t = __shfl_sync(IMIN_FULL, t, 0);
                if (t >= tail) break;
                if (lane == 0) {
                    wq[0] = t;
                    wb[t >> 5] |= 1u << (t & 31);
                    s_wtail[warp] = 1;
                }
                __syncwarp();
                int qh = 0, qt = 1;
                while (qh < qt) {
                    for (int base = qh; base < qt; base += 32) {
                        const int i = base + lane;
                        if (i < qt) {
                            const int x = wq[i];
                            for (int q = rptr[x]; q < rptr[x + 1]; ++q) {
                                const int y = radj[q];
                                const uint32_t mk = 1u << (y & 31);
                                if (!(atomicOr(&wb[y >> 5], mk) & mk)) wq[atomicAdd(&s_wtail[warp], 1)] = y;
                            }
                        }
                    }
                    __syncwarp();
                    qh = qt;
                    qt = s_wtail[warp];
                    __syncwarp();
                }
                bool meets = false;
                for (int i = lane; i < qt; i += 32) {
                    const int y = wq[i];
                    atomicAdd(&cnt[y], 1);
                    if (a.query_bm) {
                        const int v = Q[y];
                        meets |= (__ldg(a.query_bm + (v >> 5)) >> (v & 31)) & 1u;
                    }
                }
                __syncwarp();
                for (int i = lane; i < qt; i += 32) wb[wq[i] >> 5] = 0u;
                const bool any = __any_sync(IMIN_FULL, meets);
                __syncwarp();
                if (lane == 0) {
                    my_elems += (unsigned long long)qt;
                    if (any) my_cov += 1ull;
                }
            }
            if (lane == 0) {
                atomicAdd(&s_elems, my_elems);
                atomicAdd(&s_cov, my_cov);
            }
            __syncthreads();

            // ---- 4. outputs ----
            for (int i = nS + tid; i < tail; i += BD) {
                const int c = cnt[i];
                if (c) {
                    if (a.credit) atomicAdd(a.credit + Q[i], (unsigned long long)c);
                    cnt[i] = 0;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wedges += __shfl_xor_sync(IMIN_FULL, wedges, o);
        if (lane == 0 && wedges) atomicAdd(&sh.edges, wedges);
        __syncthreads();
        if (tid == 0) {
            if (a.cov_world) a.cov_world[rel] = s_cov;
            atomicAdd(a.acc + 0, s_elems);
            atomicAdd(a.acc + 1, s_cov);
            atomicAdd(a.acc + 2, (unsigned long long)tail);
            atomicAdd(a.acc + 3, sh.edges);
            atomicAdd(a.acc + 4, 1ull);
        }
        // ---- clear the visited marks ----
        for (int i = tid; i < tail; i += BD) bm[Q[i] >> 5] = 0;
        __syncthreads();
    }
}

}  // namespace useq_cta

namespace {
inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

// slot: [bitmap][queue][loc][pu][pv][rptr][rcur][radj][cnt][per-warp queues][per-warp bitmaps]
size_t useq_slot_bytes(int32_t n, int32_t ecap, size_t off[10])
{
    const size_t qcap = (size_t)n + 1;
    const size_t words = (qcap + 31) / 32;
    size_t o = al256(((size_t)n + 31) / 32 * 4);
    const size_t sz[10] = {qcap * 4, (size_t)n * 4, (size_t)ecap * 4, (size_t)ecap * 4, (qcap + 1) * 4,
                           qcap * 4, (size_t)ecap * 4, qcap * 4, useq_cta::WARPS * qcap * 4,
                           useq_cta::WARPS * words * 4};
    for (int i = 0; i < 10; ++i) {
        if (off) off[i] = o;
        o += al256(sz[i]);
    }
    return o;
}

int useq_blocks_per_sm()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, useq_cta::useq_kernel, useq_cta::BD, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

void launch_useq(imin_ctx *ctx, const UseqLaunch &L)
{
    useq_cta::UArgs a{};
    a.row_ptr = L.row_ptr;
    a.ce = L.ce;
    a.S = L.S;
    a.nS = L.nS;
    a.seed_bm = L.seed_bm;
    a.blocked_bm = L.blocked_bm;
    a.query_bm = L.query_bm;
    a.K0.klo = (uint32_t)L.key;
    a.K0.khi = (uint32_t)(L.key >> 32);
    a.K0.tag = L.tag;
    a.K0.inst = L.inst;
    a.K0.j = 0;
    a.first = L.first;
    a.count = L.count;
    a.claim = L.claim;
    a.slot_base = reinterpret_cast<char *>(L.slot_base);
    size_t off[10];
    a.slot_bytes = useq_slot_bytes(L.n, L.ecap, off);
    a.off_q = off[0];
    a.off_loc = off[1];
    a.off_pu = off[2];
    a.off_pv = off[3];
    a.off_rptr = off[4];
    a.off_rcur = off[5];
    a.off_radj = off[6];
    a.off_cnt = off[7];
    a.off_wq = off[8];
    a.off_wb = off[9];
    a.qcap = L.n + 1;
    a.words = ((size_t)L.n + 1 + 31) / 32;
    a.ecap = L.ecap;
    const char *env = std::getenv("IMIN_L2_KEEP");
    a.l2_keep = (env && env[0] == '0') ? 0 : 1;
    a.credit = L.credit;
    a.cov_world = L.cov_world;
    a.acc = L.acc;
    a.err = L.err;
    useq_cta::useq_kernel<<<L.ctas, useq_cta::BD, 0, ctx->stream>>>(a);
    IM_CHECK_LAUNCH();
}
