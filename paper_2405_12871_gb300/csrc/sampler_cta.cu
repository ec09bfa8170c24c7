// sampler_cta.cu -- reach-only worlds with one CTA per world.
//
// The warp-per-world kernel keeps thousands of worlds in flight, and their visited
// bitmaps (n bits each) do not fit in L2: they evict the graph's edge groups and
// every claim costs a DRAM round trip.  Here a whole CTA (up to 1024 threads)
// traverses one world, so only one or two worlds per SM are in flight:
//   * the visited bitmap lives in shared memory when n bits fit (claims are shared
//     memory atomics; the graph stays resident in L2), or in a per-CTA global slot;
//   * each frontier chunk (one node per thread) is flattened by a block-wide scan of
//     its 4-edge group counts, and every thread then takes groups t, t + blockDim, ...
//     (owner found by binary search in shared memory), so a hub's edges spread over
//     the whole CTA;
//   * the BFS advances level by level with a CTA barrier; new nodes are appended to
//     the queue with one shared-memory atomic per warp ballot.
// Coins, claims and outputs are those of the warp kernel (Sec. 2.1 live-edge worlds,
// blocked nodes pre-marked as visited), so every count is identical.
#include "common.cuh"

#include <algorithm>

namespace {

struct CArgs {
    const WTask *tasks;
    int ntasks;
    uint32_t *task_claim;
    uint32_t *task_done;
    char *slot_base;
    size_t slot_bytes;
    size_t bm_words;
    size_t off_queue;
    uint32_t flags;
};

template <int BD>
__device__ __forceinline__ int block_excl_scan(int x, int *s_w, int &total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(IMIN_FULL, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) s_w[w] = v;
    __syncthreads();
    if (w == 0) {
        int s = lane < BD / 32 ? s_w[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(IMIN_FULL, s, o);
            if (lane >= o) s += y;
        }
        if (lane < BD / 32) s_w[lane] = s;
    }
    __syncthreads();
    total = s_w[BD / 32 - 1];
    return (w > 0 ? s_w[w - 1] : 0) + v - x;
}

template <int BD, bool SMEM_BM, bool STOP>
__global__ void __launch_bounds__(BD, 2048 / BD >= 4 ? 4 : 2048 / BD) cta_reach_kernel(const CArgs a)
{
    extern __shared__ uint32_t s_bm[];          // n bits when SMEM_BM
    __shared__ int s_excl[BD + 1];
    __shared__ int s_b[BD];
    __shared__ int s_e[BD];
    __shared__ int s_w[32];
    __shared__ int s_tail;
    __shared__ int s_task;
    __shared__ uint32_t s_rel;
    __shared__ unsigned long long s_edges;

    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    char *slot = a.slot_base + (size_t)blockIdx.x * a.slot_bytes;
    uint32_t *bm = SMEM_BM ? s_bm : reinterpret_cast<uint32_t *>(slot);
    int32_t *Q = reinterpret_cast<int32_t *>(slot + a.off_queue);
    if (SMEM_BM) {
        for (size_t w = tid; w < a.bm_words; w += BD) s_bm[w] = 0;
    }
    int ti = (int)(blockIdx.x % (unsigned)a.ntasks);
    for (;;) {
        // ---- claim a world (thread 0), as in the warp kernel ----
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
            s_task = got;
            s_rel = rel;
            s_edges = 0;
        }
        __syncthreads();
        const int got = s_task;
        if (got < 0) break;
        ti = got;
        const uint32_t rel = s_rel;
        const WTask &T = a.tasks[ti];
        const int32_t *const row_ptr = T.row_ptr;
        const uint4 *const ce = T.ce;
        const int nS = T.q.nS;
        const uint32_t klo = (uint32_t)T.q.key, khi = (uint32_t)(T.q.key >> 32);
        const uint32_t tag = T.q.tag, inst = T.q.inst;
        const uint32_t wrel = T.list ? (T.list[rel] & 0x7fffffffu) : rel;
        const uint32_t j = (uint32_t)(T.first + (uint64_t)wrel);

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
        if (tid == 0) s_tail = nS;
        __syncthreads();
        int head = 0, tail = nS;
        unsigned long long wedges = 0;
        while (head < tail) {
            const int fend = tail;
            for (int base = head; base < fend; base += BD) {
                const int i = base + tid;
                int b = 0, e = 0, cnt = 0;
                if (i < fend) {
                    const int u = Q[i];
                    b = row_ptr[u];
                    e = row_ptr[u + 1];
                    if (e > b) cnt = ((e + 3) >> 2) - (b >> 2);
                    wedges += (unsigned long long)(e - b);
                }
                int total;
                const int excl = block_excl_scan<BD>(cnt, s_w, total);
                s_excl[tid] = excl;
                s_b[tid] = b;
                s_e[tid] = e;
                if (tid == 0) s_excl[BD] = total;
                __syncthreads();
                for (int t0 = 0; t0 < total; t0 += 2 * BD) {
                    int gq[2], obq[2], oeq[2];
                    bool act[2];
#pragma unroll
                    for (int uu = 0; uu < 2; ++uu) {
                        const int t = t0 + uu * BD + tid;
                        act[uu] = t < total;
                        // owner: the last chunk node whose range starts at or before t
                        int lo = 0, hi = BD;   // s_excl[lo] <= t < s_excl[hi]
                        if (act[uu]) {
                            while (hi - lo > 1) {
                                const int mid = (lo + hi) >> 1;
                                if (s_excl[mid] <= t) lo = mid; else hi = mid;
                            }
                        }
                        obq[uu] = s_b[lo];
                        oeq[uu] = s_e[lo];
                        gq[uu] = (obq[uu] >> 2) + (t - s_excl[lo]);
                    }
                    int4 c4[2];
                    uint4 t4[2];
#pragma unroll
                    for (int uu = 0; uu < 2; ++uu) {
                        if (act[uu]) {
                            const int4 *p = reinterpret_cast<const int4 *>(ce + 2 * (size_t)gq[uu]);
                            c4[uu] = __ldg(p);
                            t4[uu] = __ldg(reinterpret_cast<const uint4 *>(p + 1));
                        } else {
                            c4[uu] = make_int4(0, 0, 0, 0);
                            t4[uu] = make_uint4(0, 0, 0, 0);
                        }
                    }
#pragma unroll
                    for (int uu = 0; uu < 2; ++uu) {
                        int nv[4] = {-1, -1, -1, -1};
                        if (act[uu]) {
                            const int g = gq[uu];
                            const uint4 w = philox10(make_uint4((uint32_t)g, j, tag, inst), klo, khi);
                            const int cv[4] = {c4[uu].x, c4[uu].y, c4[uu].z, c4[uu].w};
                            const uint32_t tv[4] = {t4[uu].x, t4[uu].y, t4[uu].z, t4[uu].w};
                            const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
                            uint32_t old[4];
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const int ec = (g << 2) + c;
                                const bool ok = ec >= obq[uu] && ec < oeq[uu] && (wv[c] >> 8) < tv[c];
                                old[c] = ok ? atomicOr(&bm[cv[c] >> 5], 1u << (cv[c] & 31)) : 0xffffffffu;
                            }
#pragma unroll
                            for (int c = 0; c < 4; ++c)
                                if (!((old[c] >> (cv[c] & 31)) & 1u)) nv[c] = cv[c];
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const uint32_t bal = __ballot_sync(IMIN_FULL, nv[c] >= 0);
                            if (bal) {
                                int wbase = 0;
                                if (lane == 0) wbase = atomicAdd(&s_tail, __popc(bal));
                                wbase = __shfl_sync(IMIN_FULL, wbase, 0);
                                if (nv[c] >= 0) Q[wbase + __popc(bal & lt_mask)] = nv[c];
                            }
                        }
                    }
                }
                __syncthreads();
            }
            tail = s_tail;
            head = fend;
            __syncthreads();
        }
        // ---- outputs ----
        if (T.out.reach)
            for (int i = tid; i < tail; i += BD) atomicAdd(T.out.reach + Q[i], 1ull);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wedges += __shfl_xor_sync(IMIN_FULL, wedges, o);
        if (lane == 0 && wedges) atomicAdd(&s_edges, wedges);
        __syncthreads();
        if (tid == 0) {
            atomicAdd(T.out.acc + 0, (unsigned long long)tail);
            atomicAdd(T.out.acc + 1, s_edges);
            if (STOP) atomicAdd(T.out.acc + 3, (unsigned long long)tail);
            atomicAdd(T.out.acc + 4, 1ull);
            if (T.out.world_spread) T.out.world_spread[wrel] = (uint32_t)tail;
        }
        // ---- clear the visited marks ----
        if (SMEM_BM) {
            for (size_t w = tid; w < a.bm_words; w += BD) s_bm[w] = 0;
        } else {
            for (int i = tid; i < tail; i += BD) bm[Q[i] >> 5] = 0;
            for (int i = tid; i < T.q.nB; i += BD) bm[T.q.B[i] >> 5] = 0;
        }
        __syncthreads();
    }
}

inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

template <int BD, bool SMEM, bool STOP>
void launch_one(imin_ctx *ctx, const CArgs &a, int blocks, size_t smem)
{
    auto kern = cta_reach_kernel<BD, SMEM, STOP>;
    if (smem > 48 * 1024)
        IM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<blocks, BD, smem, ctx->stream>>>(a);
    IM_CHECK_LAUNCH();
}

}  // namespace

// static shared memory of the CTA kernel besides the bitmap
size_t cta_static_smem(int bd) { return (size_t)(3 * bd + 1 + 32 + 4) * 4 + 16; }

size_t cta_slot_bytes(const SlotCfg &cfg)
{
    return (cfg.smem_bm ? 0 : al16(cfg.bm_words * 4)) + al16((size_t)cfg.qcap * 4);
}

template <int BD>
static void launch_bd(imin_ctx *ctx, const CArgs &a, int blocks, bool smem_bm, bool stop, size_t smem)
{
    if (smem_bm) {
        if (stop) launch_one<BD, true, true>(ctx, a, blocks, smem);
        else launch_one<BD, true, false>(ctx, a, blocks, smem);
    } else {
        if (stop) launch_one<BD, false, true>(ctx, a, blocks, smem);
        else launch_one<BD, false, false>(ctx, a, blocks, smem);
    }
}

// resident CTAs per SM of a CTA-mode configuration (registers, threads, shared memory)
int cta_blocks_per_sm(int bd, bool smem_bm, size_t bm_words)
{
    const size_t smem = smem_bm ? bm_words * 4 : 0;
    int nb = 0;
    cudaError_t e = cudaSuccess;
#define IM_OCC(BD_, SM_)                                                                                     \
    do {                                                                                                     \
        auto kern = cta_reach_kernel<BD_, SM_, true>;                                                        \
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BD_, smem);                             \
    } while (0)
    if (bd == 256) {
        if (smem_bm) IM_OCC(256, true); else IM_OCC(256, false);
    } else if (bd == 512) {
        if (smem_bm) IM_OCC(512, true); else IM_OCC(512, false);
    } else {
        if (smem_bm) IM_OCC(1024, true); else IM_OCC(1024, false);
    }
#undef IM_OCC
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

void launch_cta_tasks(imin_ctx *ctx, const WTask *d_tasks, int ntasks, uint32_t flags,
                      const SlotCfg &cfg, void *slot_base, uint32_t *d_claim, uint32_t *d_done)
{
    CArgs a;
    a.tasks = d_tasks;
    a.ntasks = ntasks;
    a.task_claim = d_claim;
    a.task_done = d_done;
    a.slot_base = reinterpret_cast<char *>(slot_base);
    a.slot_bytes = cta_slot_bytes(cfg);
    a.bm_words = cfg.bm_words;
    a.off_queue = cfg.smem_bm ? 0 : al16(cfg.bm_words * 4);
    a.flags = flags;
    const bool stop = (flags & WF_STOP) != 0;
    const size_t smem = cfg.smem_bm ? cfg.bm_words * 4 : 0;
    if (cfg.cta_threads == 256)
        launch_bd<256>(ctx, a, cfg.ctas, cfg.smem_bm, stop, smem);
    else if (cfg.cta_threads == 512)
        launch_bd<512>(ctx, a, cfg.ctas, cfg.smem_bm, stop, smem);
    else
        launch_bd<1024>(ctx, a, cfg.ctas, cfg.smem_bm, stop, smem);
}
