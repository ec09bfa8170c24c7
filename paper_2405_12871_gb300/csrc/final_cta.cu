// final_cta.cu -- the final estimates of Algorithm 1 (line 4) for up to three candidate
// blocker sets in one traversal per world.
//
// The three (gamma, delta)-estimates of E[I_{G[V \ B]}(s)] for B_L, B_U and B_R draw
// the same worlds (stream tag 5).  A world's coins are then shared, and only the
// blocked sets differ, so one breadth-first traversal carries, for every node, the
// set of candidates under which it has been reached: a 4-bit field per node (bits
// 0..2 = L, U, R) in a nibble map, claimed with one atomic OR per live edge.  A queue
// entry packs a node with the candidate bits it newly gained, (v << 3) | bits; its
// out-edges then propagate exactly those bits.  A candidate's blocked nodes are
// pre-marked with its bit, so they are never entered under it.  Each candidate's
// reach set is therefore the one a separate traversal under its own blocked set would
// find, and |R_j(B_c)| is the number of queue entries carrying bit c.  A node enters
// the queue at most once per bit, so 3(n + 1) entries always suffice; the host sizes
// the queue from the expected spread instead, and a world that would overflow it is
// abandoned (its slot's map wiped) and listed for the host, which runs it again one
// candidate at a time.
//
// Stopping rule: worlds are claimed in index order.  A candidate whose running sum of
// sizes has reached its threshold is dropped from the worlds claimed after that (its
// stopping index N is then no larger than theirs, so no size it needs is skipped),
// and a task ends once all its candidates are dropped.  The host finds each N exactly
// from the per-world sizes.
#include "reach_cta.cuh"

#include <cstdlib>

namespace final_cta {

using reach_cta::BIG;
using reach_cta::BIGCAP;
using reach_cta::Coins;
using reach_cta::Fwd;
using reach_cta::PIECE;
using reach_cta::Shared;

struct FArgs {
    const FTask *tasks;
    int ntasks;
    uint32_t *claim, *done;
    char *slot_base;
    size_t slot_bytes;
    size_t off_queue;
    int32_t qcap;        // queue entries per slot
    size_t nib_words;    // words of a slot's nibble map
    int l2_keep;
};

// One pass over one 4-edge group per lane: claim the live targets for the source's
// candidate bits `om` and append the entries whose bits are new.  All lanes call it.
__device__ __forceinline__ void pass_multi(const Fwd &op, bool act, int it, int ob, int oe, uint32_t om,
                                           const Coins &K, uint32_t *nib, int32_t *Q, int *app, int tail,
                                           int lane, uint32_t lt_mask, int qcap, int *ovf)
{
    uint32_t live = 0;
    int4 c4 = make_int4(0, 0, 0, 0);
    if (act) live = op.live(it, ob, oe, K, c4);
    uint32_t n0 = 0, n1 = 0, n2 = 0, n3 = 0;
    const int s0 = (c4.x & 7) * 4, s1 = (c4.y & 7) * 4, s2 = (c4.z & 7) * 4, s3 = (c4.w & 7) * 4;
    if (live & 1u) n0 = om & ~(atomicOr(&nib[c4.x >> 3], om << s0) >> s0);
    if (live & 2u) n1 = om & ~(atomicOr(&nib[c4.y >> 3], om << s1) >> s1);
    if (live & 4u) n2 = om & ~(atomicOr(&nib[c4.z >> 3], om << s2) >> s2);
    if (live & 8u) n3 = om & ~(atomicOr(&nib[c4.w >> 3], om << s3) >> s3);
    const uint32_t b0 = __ballot_sync(IMIN_FULL, n0 != 0), b1 = __ballot_sync(IMIN_FULL, n1 != 0),
                   b2 = __ballot_sync(IMIN_FULL, n2 != 0), b3 = __ballot_sync(IMIN_FULL, n3 != 0);
    const int tot = __popc(b0) + __popc(b1) + __popc(b2) + __popc(b3);
    if (tot == 0) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(app, tot);
    base = __shfl_sync(IMIN_FULL, base, 0);
    int pos = tail + base + __popc(b0 & lt_mask) + __popc(b1 & lt_mask) + __popc(b2 & lt_mask) +
              __popc(b3 & lt_mask);
    if (tail + base + tot > qcap) {   // the queue is full: the world is abandoned
        if (lane == 0) *ovf = 1;
        return;
    }
    if (n0) Q[pos++] = (c4.x << 3) | (int)n0;
    if (n1) Q[pos++] = (c4.y << 3) | (int)n1;
    if (n2) Q[pos++] = (c4.z << 3) | (int)n2;
    if (n3) Q[pos] = (c4.w << 3) | (int)n3;
}

// Level-synchronous expansion of the packed queue Q[0, tail0), with the slice / hub
// structure of the reach kernel (reach_cta.cuh, bfs): 32-entry slices per warp, hub
// entries cut into pieces shared by the CTA.  Returns the final tail.
template <int BD>
__device__ __forceinline__ int bfs_multi(const Fwd &op, const Coins &K, uint32_t *nib, int32_t *Q, int tail0,
                                         Shared<BD> &sh, unsigned long long &wedges, int qcap, int *ovf)
{
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    int head = 0, tail = tail0, lvl = 0;
    while (head < tail) {
        const int p = lvl & 1;
        if (tid == 0) sh.slice[p ^ 1] = sh.nbig[p ^ 1] = sh.piece[p ^ 1] = 0;
        int sl = 0;
        if (lane == 0) sl = atomicAdd(&sh.slice[p], 1);
        sl = __shfl_sync(IMIN_FULL, sl, 0);
        int nbase = head + sl * 32;
        int nx = nbase + lane < tail ? Q[nbase + lane] : 0;
        for (;;) {
            const int base = nbase;
            if (base >= tail) break;
            const int i = base + lane;
            const int x = nx;
            if (lane == 0) sl = atomicAdd(&sh.slice[p], 1);
            sl = __shfl_sync(IMIN_FULL, sl, 0);
            nbase = head + sl * 32;
            nx = nbase + lane < tail ? Q[nbase + lane] : 0;
            int b = 0, e = 0, cnt = 0;
            if (i < tail) {
                op.range(x >> 3, b, e);
                cnt = Fwd::count(b, e);
                wedges += (unsigned long long)(e - b);
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
                    sh.bi[my] = x;   // the packed entry: its candidate bits
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
                int pos = 0;
#pragma unroll
                for (int s = 16; s >= 1; s >>= 1) {
                    const int c = __shfl_sync(IMIN_FULL, incl, pos + s - 1);
                    if (c <= t) pos += s;
                }
                const int ob = __shfl_sync(IMIN_FULL, b, pos);
                const int oe = __shfl_sync(IMIN_FULL, e, pos);
                const int ox = __shfl_sync(IMIN_FULL, excl, pos);
                const uint32_t om = (uint32_t)__shfl_sync(IMIN_FULL, x, pos) & 7u;
                pass_multi(op, t < total, Fwd::first(ob) + (t - ox), ob, oe, om, K, nib, Q, &sh.app[p], tail,
                           lane, lt_mask, qcap, ovf);
            }
        }
        __syncthreads();
        if (tid == 0) sh.app[p ^ 1] = 0;
        const int nb = min(sh.nbig[p], BIGCAP);
        if (nb > 0) {
            if ((tid >> 5) == 0) {
                int carry = 0;
                for (int c0 = 0; c0 < nb; c0 += 32) {
                    const int i = c0 + lane;
                    int np = 0;
                    if (i < nb) np = (Fwd::count(sh.bb[i], sh.be[i]) + PIECE - 1) / PIECE;
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
                int lo = 0, hi = nb;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (sh.pp[mid] <= pc) lo = mid; else hi = mid;
                }
                const int ob = sh.bb[lo], oe = sh.be[lo];
                const uint32_t om = (uint32_t)sh.bi[lo] & 7u;
                const int i0 = Fwd::first(ob) + (pc - sh.pp[lo]) * PIECE;
                const int iend = min(i0 + PIECE, Fwd::first(ob) + Fwd::count(ob, oe));
                for (int is = i0; is < iend; is += 32)
                    pass_multi(op, is + lane < iend, is + lane, ob, oe, om, K, nib, Q, &sh.app[p], tail, lane,
                               lt_mask, qcap, ovf);
            }
        }
        __syncthreads();
        if (*(volatile int *)ovf) return -1;   // entries were dropped: the world is abandoned
        const int ntail = tail + sh.app[p];
        head = tail;
        tail = ntail;
        ++lvl;
    }
    return tail;
}

template <int BD, int MINB>
__global__ void __launch_bounds__(BD, MINB) cta_final_kernel(const FArgs a)
{
    __shared__ Shared<BD> sh;
    __shared__ unsigned int cnt3[3];
    __shared__ uint32_t smask;
    __shared__ int s_ovf;

    const int tid = threadIdx.x, lane = tid & 31;
    char *slot = a.slot_base + (size_t)blockIdx.x * a.slot_bytes;
    uint32_t *const nib = reinterpret_cast<uint32_t *>(slot);
    int32_t *const Q = reinterpret_cast<int32_t *>(slot + a.off_queue);
    int ti = (int)(blockIdx.x % (unsigned)a.ntasks);
    for (;;) {
        // ---- claim a world and the candidates it still has to serve (thread 0) ----
        if (tid == 0) {
            int got = -1;
            uint32_t rel = 0, mask = 0;
            for (int scan = 0; scan < a.ntasks; ++scan) {
                const int t = (ti + scan) % a.ntasks;
                if (*(volatile uint32_t *)(a.done + t)) continue;
                const FTask *tp = a.tasks + t;
                uint32_t m = 0;
                for (int c = 0; c < 3; ++c)
                    if (((tp->cands >> c) & 1u) &&
                        *(volatile unsigned long long *)(tp->acc + c) < tp->stop_T[c])
                        m |= 1u << c;
                if (!m) {
                    a.done[t] = 1u;
                    continue;
                }
                const uint32_t r = atomicAdd(a.claim + t, 1u);
                if (r >= tp->count) {
                    a.done[t] = 1u;
                    continue;
                }
                got = t;
                rel = r;
                mask = m;
                break;
            }
            sh.task = got;
            sh.rel = rel;
            smask = mask;
            s_ovf = 0;
            sh.edges = 0;
            cnt3[0] = cnt3[1] = cnt3[2] = 0;
            sh.slice[0] = sh.nbig[0] = sh.piece[0] = sh.app[0] = 0;
            sh.slice[1] = sh.nbig[1] = sh.piece[1] = sh.app[1] = 0;
        }
        __syncthreads();
        const int got = sh.task;
        if (got < 0) break;
        ti = got;
        const uint32_t rel = sh.rel, mask = smask;
        const FTask &T = a.tasks[ti];
        Coins K;
        K.klo = (uint32_t)T.key;
        K.khi = (uint32_t)(T.key >> 32);
        K.tag = T.tag;
        K.inst = T.inst;
        K.j = (uint32_t)(T.first + (uint64_t)rel);
        const int nS = T.nS;

        // ---- blocked nodes pre-marked with their candidate's bit; seeds with all ----
        for (int c = 0; c < 3; ++c)
            if ((mask >> c) & 1u)
                for (int i = tid; i < T.nB[c]; i += BD) {
                    const int v = T.B[c][i];
                    atomicOr(&nib[v >> 3], (1u << c) << ((v & 7) * 4));
                }
        for (int i = tid; i < nS; i += BD) {
            const int s = T.S[i];
            atomicOr(&nib[s >> 3], mask << ((s & 7) * 4));
            Q[i] = (s << 3) | (int)mask;
        }
        __syncthreads();
        unsigned long long wedges = 0;
        const Fwd fwd{T.row_ptr, T.ce, reach_cta::graph_l2_policy(a.l2_keep != 0), T.rng, T.gid};
        const int tail = bfs_multi<BD>(fwd, K, nib, Q, nS, sh, wedges, a.qcap, &s_ovf);
        if (tail < 0) {
            // overflow: wipe the map (dropped entries left bits that the queue cannot
            // find) and list the world for the host
            for (size_t w = tid; w < a.nib_words; w += BD) nib[w] = 0u;
            if (tid == 0) {
                const uint32_t d = atomicAdd(T.n_deferred, 1u);
                if (d < T.deferred_cap) T.deferred[d] = rel;
            }
            __syncthreads();
            continue;
        }

        // ---- per-candidate sizes; the nibble map is cleared through the queue ----
        unsigned int c0 = 0, c1 = 0, c2 = 0;
        for (int i = tid; i < tail; i += BD) {
            const int x = Q[i];
            c0 += x & 1;
            c1 += (x >> 1) & 1;
            c2 += (x >> 2) & 1;
            nib[(x >> 3) >> 3] = 0u;
        }
        for (int c = 0; c < 3; ++c)
            if ((mask >> c) & 1u)
                for (int i = tid; i < T.nB[c]; i += BD) nib[T.B[c][i] >> 3] = 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c0 += __shfl_xor_sync(IMIN_FULL, c0, o);
            c1 += __shfl_xor_sync(IMIN_FULL, c1, o);
            c2 += __shfl_xor_sync(IMIN_FULL, c2, o);
            wedges += __shfl_xor_sync(IMIN_FULL, wedges, o);
        }
        if (lane == 0) {
            if (c0) atomicAdd(&cnt3[0], c0);
            if (c1) atomicAdd(&cnt3[1], c1);
            if (c2) atomicAdd(&cnt3[2], c2);
            if (wedges) atomicAdd(&sh.edges, wedges);
        }
        __syncthreads();
        if (tid == 0) {
            uint32_t *sz = T.sizes + (size_t)rel * 4;
            for (int c = 0; c < 3; ++c) {
                sz[c] = cnt3[c];
                if ((mask >> c) & 1u) atomicAdd(T.acc + c, (unsigned long long)cnt3[c]);
            }
            atomicAdd(T.acc + 3, (unsigned long long)tail);
            atomicAdd(T.acc + 4, sh.edges);
            atomicAdd(T.acc + 5, 1ull);
        }
        __syncthreads();
    }
}

template <int BD, int MINB>
void launch(cudaStream_t st, const FArgs &a, int blocks)
{
    cta_final_kernel<BD, MINB><<<blocks, BD, 0, st>>>(a);
    IM_CHECK_LAUNCH();
}

}  // namespace final_cta

namespace {
inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

// slot: [nibble map: 4 bits per node] [queue: qcap packed entries]
size_t final_slot_bytes(int32_t n, int32_t qcap, size_t *off_queue)
{
    const size_t nib = al256((((size_t)n + 7) / 8) * 4);
    if (off_queue) *off_queue = nib;
    return nib + al256((size_t)qcap * 4);
}

void launch_final_tasks(imin_ctx *ctx, const FTask *d_tasks, int ntasks, int32_t nmax, int32_t qcap, int bd,
                        int ctas, void *slot_base, uint32_t *d_claim, uint32_t *d_done)
{
    final_cta::FArgs a;
    a.tasks = d_tasks;
    a.ntasks = ntasks;
    a.claim = d_claim;
    a.done = d_done;
    a.slot_base = reinterpret_cast<char *>(slot_base);
    a.slot_bytes = final_slot_bytes(nmax, qcap, &a.off_queue);
    a.qcap = qcap;
    a.nib_words = ((size_t)nmax + 7) / 8;
    const char *env = std::getenv("IMIN_L2_KEEP");
    a.l2_keep = (env && env[0] == '0') ? 0 : 1;
    if (bd == 256)
        final_cta::launch<256, 8>(ctx->stream, a, ctas);
    else
        final_cta::launch<512, 4>(ctx->stream, a, ctas);
}

int final_blocks_per_sm(int bd)
{
    int nb = 0;
    cudaError_t e = bd == 256
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, final_cta::cta_final_kernel<256, 8>, 256, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, final_cta::cta_final_kernel<512, 4>, 512, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}
