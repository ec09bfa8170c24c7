// gs_rev.cu -- Global Sampling worlds (Algorithm 3) traversed backwards from the target.
//
// The LRR set of world phi for target t is L_phi(t) = the nodes of R_phi(s) \ S that
// reach t inside phi^s (Def. 4.2).  The forward pass of the CTA kernel computes all of
// R_phi(s) (tens of thousands of nodes on a power-law graph) to test membership.  The
// same set follows from the nodes near t alone:
//   X = the non-seed, unblocked nodes that reach t by live edges avoiding the seeds
//       (and blocked nodes), found by a reverse traversal from t over live in-edges;
//   L_phi(t) = the nodes of X reachable from a seed by a live path whose non-seed nodes
//       all lie in X, if t is one of them, and the empty set otherwise.
// (A node of X reachable from S has a path whose part after the last seed lies in X,
// since every node on it reaches t through the node; and every node on a path inside
// phi^s from u to t is reachable from S through u.)  Under weighted-cascade
// probabilities a node has one live in-edge on average, so X has a handful of nodes
// where R_phi(s) has thousands.
//
// One warp per world.  X lives in a per-warp open-addressing table in shared memory
// (node -> local id), with the live in-edges found between nodes of X and the nodes
// entered directly from a seed.  A world whose X or edge list outgrows the table is
// deferred with the top bit (the host retries it with the wide tables, then with the
// forward kernel), as is a world without store room (without the top bit).  The coins are the forward edges' (edge id eid, Philox counter eid >> 2), so
// the sets are those of the forward kernel and of the oracle.
#include "reach_cta.cuh"

namespace gs_rev {

// Two table sizes: the narrow one (8 warps per CTA, 3.7 KB per warp) takes every world;
// the few worlds it cannot hold go to the wide one (one warp per CTA with 116 KB), and
// only those that outgrow that to the forward kernel.
template <int WARPS_, int XCAP_, int HT_, int HBITS_, int ECAP_>
struct Cfg {
    static constexpr int WARPS = WARPS_;   // warps per CTA
    static constexpr int XCAP = XCAP_;     // nodes of X per world
    static constexpr int HT = HT_;         // hash slots (power of two, >= 2 XCAP)
    static constexpr int HBITS = HBITS_;   // log2(HT)
    static constexpr int ECAP = ECAP_;     // live edges inside X per world
};
using Narrow = Cfg<8, 128, 256, 8, 256>;
using Wide = Cfg<1, 4096, 8192, 13, 8192>;

template <class C>
struct WarpSmem {
    int key[C::HT];
    int val[C::HT];
    int x[C::XCAP];               // local id -> node
    short eu[C::ECAP], ev[C::ECAP];   // live edge (local source, local target)
    unsigned char flag[C::XCAP];  // bit 0: entered from a seed / reached from one
    int nx, ne, ovf;
};

template <class C>
__device__ __forceinline__ uint32_t hslot(int v)
{
    return ((uint32_t)v * 2654435761u) >> (32 - C::HBITS);
}

__device__ __forceinline__ bool bit_of(const uint32_t *bm, int v)
{
    return bm && ((__ldg(bm + (v >> 5)) >> (v & 31)) & 1u);
}

// local id of node v in the table; -1 if absent
template <class C>
__device__ __forceinline__ int lookup(WarpSmem<C> &w, int v)
{
    uint32_t h = hslot<C>(v);
    for (int probe = 0; probe < C::HT; ++probe) {
        const int k = w.key[h];
        if (k == v) return w.val[h];
        if (k < 0) return -1;
        h = (h + 1) & (C::HT - 1);
    }
    return -1;
}

struct RArgs {
    const WTask *tasks;
    int ntasks;
    uint32_t *claim, *done;
};

template <class C>
__global__ void __launch_bounds__(C::WARPS * 32, C::WARPS == 1 ? 1 : 4) gs_rev_kernel(const RArgs a)
{
    constexpr int WARPS = C::WARPS, XCAP = C::XCAP, HT = C::HT, ECAP = C::ECAP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpSmem<C> &w = reinterpret_cast<WarpSmem<C> *>(smem_raw)[wid];
    for (int i = lane; i < HT; i += 32) w.key[i] = -1;
    __syncwarp();
    int ti = (int)((blockIdx.x * WARPS + wid) % (unsigned)a.ntasks);
    for (;;) {
        // ---- claim a world ----
        int got = -1;
        uint32_t rel = 0;
        if (lane == 0) {
            for (int scan = 0; scan < a.ntasks; ++scan) {
                const int t = (ti + scan) % a.ntasks;
                if (*(volatile uint32_t *)(a.done + t)) continue;
                const uint32_t r = atomicAdd(a.claim + t, 1u);
                if (r >= a.tasks[t].count) {
                    a.done[t] = 1u;
                    continue;
                }
                got = t;
                rel = r;
                break;
            }
        }
        got = __shfl_sync(IMIN_FULL, got, 0);
        rel = __shfl_sync(IMIN_FULL, rel, 0);
        if (got < 0) break;
        ti = got;
        const WTask &T = a.tasks[ti];
        const uint32_t wrel = T.list ? (T.list[rel] & 0x7fffffffu) : rel;
        reach_cta::Coins K;
        K.klo = (uint32_t)T.q.key;
        K.khi = (uint32_t)(T.q.key >> 32);
        K.tag = T.q.tag;
        K.inst = T.q.inst;
        K.j = (uint32_t)(T.first + (uint64_t)wrel);

        // ---- target t uniform in V'_s ----
        int tn = -1;
        if (T.q.nVs > 0) {
            const uint4 r4 = reach_cta::philox10_w(make_uint4(0xFFFFFFFFu, K.j, K.tag, K.inst), K.klo, K.khi);
            const unsigned long long r64 = ((unsigned long long)r4.y << 32) | r4.x;
            const int t = T.q.Vs[__umul64hi(r64, (unsigned long long)T.q.nVs)];
            if (!bit_of(T.q.blocked_bm, t)) tn = t;
        }
        unsigned long long scanned = 0;
        int L = 0;
        bool overflow = false;
        if (tn >= 0) {
            if (lane == 0) {
                const uint32_t h = hslot<C>(tn);
                w.key[h] = tn;
                w.val[h] = 0;
                w.x[0] = tn;
                w.flag[0] = 0;
                w.nx = 1;
                w.ne = 0;
                w.ovf = 0;
            }
            __syncwarp();
            // ---- reverse traversal: X and the live edges inside it ----
            for (int head = 0;; ++head) {
                const int nx = *(volatile int *)&w.nx;
                if (head >= nx || *(volatile int *)&w.ovf) break;
                const int x = w.x[head];
                const int b = __ldg(T.in_ptr + x), e = __ldg(T.in_ptr + x + 1);
                scanned += (unsigned long long)(e - b);
                for (int q0 = b; q0 < e; q0 += 32) {
                    const int q = q0 + lane;
                    int u = -1;
                    bool live = false;
                    if (q < e) {
                        u = __ldg(T.in_src + q);
                        if (!bit_of(T.q.blocked_bm, u)) {
                            const int eid = __ldg(T.in_eid + q);
                            const uint4 c =
                                reach_cta::philox10_w(make_uint4((uint32_t)eid >> 2, K.j, K.tag, K.inst), K.klo, K.khi);
                            live = (pick_word(c, eid & 3) >> 8) < __ldg(T.in_thr + q);
                        }
                    }
                    const bool seed = live && bit_of(T.q.seed_bm, u);
                    if (__any_sync(IMIN_FULL, seed) && lane == 0) w.flag[head] |= 1u;   // entered from a seed
                    const bool inner = live && !seed;
                    // insert new sources: claim a slot by CAS, then number the new ones
                    bool fresh = false;
                    int slot = -1;
                    if (inner) {
                        uint32_t h = hslot<C>(u);
                        for (int probe = 0; probe < HT; ++probe) {
                            const int old = atomicCAS(&w.key[h], -1, u);
                            if (old == -1) {
                                fresh = true;
                                slot = (int)h;
                                break;
                            }
                            if (old == u) break;
                            h = (h + 1) & (HT - 1);
                        }
                    }
                    const uint32_t fb = __ballot_sync(IMIN_FULL, fresh);
                    int base = 0;
                    if (lane == 0) {
                        base = w.nx;
                        w.nx = base + __popc(fb);
                    }
                    base = __shfl_sync(IMIN_FULL, base, 0);
                    if (fresh) {
                        const int id = base + __popc(fb & ((1u << lane) - 1u));
                        if (id < XCAP) {
                            w.val[slot] = id;
                            w.x[id] = u;
                            w.flag[id] = 0;
                        } else {
                            w.val[slot] = -1;
                            w.ovf = 1;
                        }
                    }
                    __syncwarp();
                    // record the live edge (u -> x) between nodes of X
                    int iu = -1;
                    if (inner) {
                        iu = lookup(w, u);
                        if (iu < 0) w.ovf = 1;
                    }
                    const bool rec = inner && iu >= 0;
                    const uint32_t rb = __ballot_sync(IMIN_FULL, rec);
                    int eb = 0;
                    if (lane == 0) {
                        eb = w.ne;
                        w.ne = eb + __popc(rb);
                    }
                    eb = __shfl_sync(IMIN_FULL, eb, 0);
                    if (rec) {
                        const int ei = eb + __popc(rb & ((1u << lane) - 1u));
                        if (ei < ECAP) {
                            w.eu[ei] = (short)iu;
                            w.ev[ei] = (short)head;
                        } else {
                            w.ovf = 1;
                        }
                    }
                    __syncwarp();
                }
            }
            __syncwarp();
            overflow = *(volatile int *)&w.ovf != 0 || w.nx > XCAP;
            if (!overflow) {
                // ---- forward closure inside X from the nodes entered from a seed ----
                const int nx = w.nx, ne = w.ne;
                for (;;) {
                    bool changed = false;
                    for (int i = lane; i < ne; i += 32) {
                        const int su = w.eu[i], sv = w.ev[i];
                        if ((w.flag[su] & 1u) && !(w.flag[sv] & 1u)) {
                            w.flag[sv] |= 1u;
                            changed = true;
                        }
                    }
                    __syncwarp();
                    if (!__any_sync(IMIN_FULL, changed)) break;
                }
                if (w.flag[0] & 1u)   // t is reached: L(t) = the reached nodes of X
                    for (int i = lane; i < nx; i += 32) L += (w.flag[i] & 1u) ? 1 : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) L += __shfl_xor_sync(IMIN_FULL, L, o);
            }
        }
        bool defer = overflow;
        unsigned long long sb = 0;
        if (!defer && (T.out.set_cursor != nullptr)) {
            if (lane == 0)
                sb = L > 0 ? reach_cta::reserve_store(T.out.set_cursor, (unsigned long long)L, T.out.set_cap) : 0ull;
            sb = __shfl_sync(IMIN_FULL, sb, 0);
            defer = sb == ~0ull;
        }
        if (defer) {
            if (lane == 0) {
                const uint32_t d = atomicAdd(T.out.n_deferred, 1u);
                if (d < T.out.deferred_cap)
                    T.out.deferred[d] = wrel | (overflow ? 0x80000000u : 0u);
                else
                    atomicOr(T.out.err, DERR_INTERNAL);
            }
        } else {
            if (L > 0) {
                int at = 0;
                for (int i0 = 0; i0 < w.nx; i0 += 32) {
                    const int i = i0 + lane;
                    const bool in = i < w.nx && (w.flag[i] & 1u);
                    const uint32_t bl = __ballot_sync(IMIN_FULL, in);
                    if (in) {
                        const int v = w.x[i];
                        if (T.out.credit_U) atomicAdd(T.out.credit_U + v, 1ull);
                        if (T.out.set_cursor) T.out.set_elem[sb + at + __popc(bl & ((1u << lane) - 1u))] = v;
                    }
                    at += __popc(bl);
                }
            }
            if (lane == 0) {
                if (T.out.set_cursor) {
                    T.out.set_off[wrel] = sb;
                    T.out.set_len[wrel] = (uint32_t)L;
                }
                if (L > 0) atomicAdd(T.out.acc + 2, 1ull);
                atomicAdd(T.out.acc + 4, 1ull);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) scanned += __shfl_xor_sync(IMIN_FULL, scanned, o);
        if (lane == 0 && tn >= 0 && !defer) {
            atomicAdd(T.out.acc + 0, (unsigned long long)min(w.nx, XCAP));
            atomicAdd(T.out.acc + 1, scanned);
        }
        // ---- clear the table ----
        __syncwarp();
        if (tn >= 0) {
            for (int i = lane; i < HT; i += 32) w.key[i] = -1;
        }
        __syncwarp();
    }
}

}  // namespace gs_rev

namespace {
template <class C>
void launch_cfg(imin_ctx *ctx, const gs_rev::RArgs &a, int max_ctas)
{
    const size_t smem = sizeof(gs_rev::WarpSmem<C>) * C::WARPS;
    auto kern = gs_rev::gs_rev_kernel<C>;
    IM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, C::WARPS * 32, smem) != cudaSuccess) {
        cudaGetLastError();
        nb = 1;
    }
    int ctas = ctx->num_sms * std::max(nb, 1);
    if (max_ctas > 0) ctas = std::min(ctas, max_ctas);
    kern<<<std::max(ctas, 1), C::WARPS * 32, smem, ctx->stream>>>(a);
    IM_CHECK_LAUNCH();
}
}  // namespace

void launch_gs_rev(imin_ctx *ctx, const WTask *d_tasks, int ntasks, uint32_t *d_claim, uint32_t *d_done, bool wide,
                   int max_ctas)
{
    gs_rev::RArgs a;
    a.tasks = d_tasks;
    a.ntasks = ntasks;
    a.claim = d_claim;
    a.done = d_done;
    if (wide)
        launch_cfg<gs_rev::Wide>(ctx, a, max_ctas);
    else
        launch_cfg<gs_rev::Narrow>(ctx, a, max_ctas);
}
