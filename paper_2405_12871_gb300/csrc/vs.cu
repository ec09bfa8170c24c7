// vs.cu -- V'_s on the device: the nodes reachable from S over edges of nonzero
// probability while avoiding the blocked nodes, S itself excluded (the node set over
// which Global Sampling draws its target, Sec. 5.2, and whose size normalises the
// stopping rule's estimates, Sec. 6).
//
// A level-synchronous breadth-first search over the whole graph:
//   * warps claim 32-node slices of the frontier from a global counter, scan the
//     slice's out-degrees with shuffles and give one edge to each lane per pass; a
//     node of more than HUB edges is deferred to a hub list instead;
//   * a second kernel spreads each hub's edges over a whole block;
//   * a visited bitmap (pre-marked with S and the blocked nodes) is claimed with
//     atomic OR and new nodes are appended with one atomic per warp ballot.
// All levels run in one cooperative launch with grid barriers between the expansion,
// the hub step and the next level (the per-level form with a host round trip per
// level is the fallback where cooperative launches are not available).  The list is
// then read off the bitmap in ascending order (a per-word population count, a scan, a
// scatter).  The work buffers are cached in the context.
#include "common.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace {

constexpr int HUB = 1024;

struct VsCtl {
    unsigned int slice;   // next 32-node slice of the frontier
    unsigned int nout;    // nodes appended to the next frontier
    unsigned int nhub;    // hubs deferred to the hub kernel
    unsigned int pad;
};

__global__ void k_vs_mark(uint32_t *vis, const uint32_t *seed_bm, const uint32_t *blk_bm, size_t words)
{
    for (size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (size_t)gridDim.x * blockDim.x)
        vis[w] = seed_bm[w] | (blk_bm ? blk_bm[w] : 0u);
}

__device__ __forceinline__ void vs_claim_append(bool want, int v, uint32_t *vis, int32_t *qout, VsCtl *ctl,
                                                int lane, uint32_t lt_mask)
{
    bool fresh = false;
    if (want) {
        const uint32_t bit = 1u << (v & 31);
        fresh = !(atomicOr(&vis[v >> 5], bit) & bit);
    }
    const uint32_t bal = __ballot_sync(IMIN_FULL, fresh);
    if (bal) {
        unsigned int base = 0;
        if (lane == 0) base = atomicAdd(&ctl->nout, (unsigned)__popc(bal));
        base = __shfl_sync(IMIN_FULL, base, 0);
        if (fresh) qout[base + __popc(bal & lt_mask)] = v;
    }
}

__global__ void __launch_bounds__(256) k_vs_expand(const int32_t *row_ptr, const int32_t *col,
                                                   const uint32_t *thr, uint32_t *vis, const int32_t *qin,
                                                   int nin, int32_t *qout, int32_t *hubs, VsCtl *ctl)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (;;) {
        unsigned int sl = 0;
        if (lane == 0) sl = atomicAdd(&ctl->slice, 1u);
        sl = __shfl_sync(IMIN_FULL, sl, 0);
        const long long base = (long long)sl * 32;
        if (base >= nin) break;
        const long long i = base + lane;
        int b = 0, cnt = 0;
        if (i < nin) {
            const int u = qin[i];
            b = row_ptr[u];
            cnt = row_ptr[u + 1] - b;
            if (cnt > HUB) {
                hubs[atomicAdd(&ctl->nhub, 1u)] = u;
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
            const int ox = __shfl_sync(IMIN_FULL, excl, pos);
            bool want = false;
            int v = 0;
            if (t < total) {
                const int e = ob + (t - ox);
                v = col[e];
                want = thr[e] != 0u;
            }
            vs_claim_append(want, v, vis, qout, ctl, lane, lt_mask);
        }
    }
}

// one block per hub at a time (grid-stride over the hub list)
__global__ void __launch_bounds__(256) k_vs_hubs(const int32_t *row_ptr, const int32_t *col, const uint32_t *thr,
                                                 uint32_t *vis, int32_t *qout, const int32_t *hubs,
                                                 VsCtl *ctl)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const unsigned int nh = *(volatile unsigned int *)&ctl->nhub;
    for (unsigned int h = blockIdx.x; h < nh; h += gridDim.x) {
        const int u = hubs[h];
        const int b = row_ptr[u], e = row_ptr[u + 1];
        // whole warps step together so that the ballot sees every lane
        for (int base = b + (int)(threadIdx.x & ~31u); base < e; base += (int)blockDim.x) {
            const int x = base + lane;
            bool want = false;
            int v = 0;
            if (x < e) {
                v = col[x];
                want = thr[x] != 0u;
            }
            vs_claim_append(want, v, vis, qout, ctl, lane, lt_mask);
        }
    }
}

// The warp-slice expansion of one frontier (the body of k_vs_expand), for the
// persistent kernel: slices are claimed from c->slice by warps of the whole grid.
__device__ __forceinline__ void vs_expand_level(const int32_t *row_ptr, const int32_t *col, const uint32_t *thr,
                                                uint32_t *vis, const int32_t *qin, long long nin, int32_t *qout,
                                                int32_t *hubs, VsCtl *c, int lane, uint32_t lt_mask)
{
    for (;;) {
        unsigned int sl = 0;
        if (lane == 0) sl = atomicAdd(&c->slice, 1u);
        sl = __shfl_sync(IMIN_FULL, sl, 0);
        const long long base = (long long)sl * 32;
        if (base >= nin) break;
        const long long i = base + lane;
        int b = 0, cnt = 0;
        if (i < nin) {
            const int u = __ldcg(qin + i);
            b = row_ptr[u];
            cnt = row_ptr[u + 1] - b;
            if (cnt > HUB) {
                hubs[atomicAdd(&c->nhub, 1u)] = u;
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
                const int cc = __shfl_sync(IMIN_FULL, incl, pos + s - 1);
                if (cc <= t) pos += s;
            }
            const int ob = __shfl_sync(IMIN_FULL, b, pos);
            const int ox = __shfl_sync(IMIN_FULL, excl, pos);
            bool want = false;
            int v = 0;
            if (t < total) {
                const int e = ob + (t - ox);
                v = col[e];
                want = thr[e] != 0u;
            }
            vs_claim_append(want, v, vis, qout, c, lane, lt_mask);
        }
    }
}

// Every level of the search in one cooperative launch.  ctl[3] rotate: the counters
// of level L are ctl[L % 3]; those of level L - 1 are cleared after the first barrier
// of level L (every thread has read them by then) for use again at level L + 2.
__global__ void __launch_bounds__(256) k_vs_all(const int32_t *row_ptr, const int32_t *col, const uint32_t *thr,
                                                uint32_t *vis, int32_t *qa, int32_t *qb, long long nS,
                                                int32_t *hubs, VsCtl *ctl)
{
    cg::grid_group grid = cg::this_grid();
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    int32_t *qin = qa, *qout = qb;
    long long nin = nS;
    for (int level = 0; nin > 0; ++level) {   // every node enters a frontier at most once
        VsCtl *c = ctl + (level % 3);
        vs_expand_level(row_ptr, col, thr, vis, qin, nin, qout, hubs, c, lane, lt_mask);
        grid.sync();
        if (blockIdx.x == 0 && threadIdx.x == 0 && level > 0) {
            VsCtl *prev = ctl + ((level + 2) % 3);
            prev->slice = prev->nout = prev->nhub = 0u;
        }
        const unsigned int nh = *(volatile unsigned int *)&c->nhub;
        for (unsigned int h = blockIdx.x; h < nh; h += gridDim.x) {
            const int u = __ldcg(hubs + h);
            const int b = row_ptr[u], e = row_ptr[u + 1];
            for (int base = b + (int)(threadIdx.x & ~31u); base < e; base += (int)blockDim.x) {
                const int x = base + lane;
                bool want = false;
                int v = 0;
                if (x < e) {
                    v = col[x];
                    want = thr[x] != 0u;
                }
                vs_claim_append(want, v, vis, qout, c, lane, lt_mask);
            }
        }
        grid.sync();
        nin = *(volatile unsigned int *)&c->nout;
        int32_t *t = qin;
        qin = qout;
        qout = t;
    }
}

// per word: visited nodes that are neither seeds nor blocked
__global__ void k_vs_count(const uint32_t *vis, const uint32_t *seed_bm, const uint32_t *blk_bm, size_t words,
                           int32_t n, long long *cnt)
{
    for (size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x; w <= words; w += (size_t)gridDim.x * blockDim.x) {
        if (w == words) {
            cnt[w] = 0;
            continue;
        }
        uint32_t m = vis[w] & ~seed_bm[w] & ~(blk_bm ? blk_bm[w] : 0u);
        if ((w + 1) * 32 > (size_t)n) m &= (1u << (n - w * 32)) - 1u;
        cnt[w] = __popc(m);
    }
}

__global__ void k_vs_scatter(const uint32_t *vis, const uint32_t *seed_bm, const uint32_t *blk_bm, size_t words,
                             int32_t n, const long long *pos, int32_t *out)
{
    for (size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (size_t)gridDim.x * blockDim.x) {
        uint32_t m = vis[w] & ~seed_bm[w] & ~(blk_bm ? blk_bm[w] : 0u);
        if ((w + 1) * 32 > (size_t)n) m &= (1u << (n - w * 32)) - 1u;
        long long p = pos[w];
        while (m) {
            const int b = __ffs(m) - 1;
            out[p++] = (int32_t)(w * 32 + b);
            m &= m - 1u;
        }
    }
}

int grid_for(imin_ctx *ctx, long long work)
{
    long long b = (work + 255) / 256;
    const long long cap = (long long)ctx->num_sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

int32_t device_reach_set(imin_ctx *ctx, const imin_graph *g, const int32_t *dS, int32_t nS,
                         const uint32_t *seed_bm, const uint32_t *blk_bm, DBuf &out)
{
    cudaStream_t st = ctx->stream;
    const int32_t n = g->n;
    const size_t words = ((size_t)n + 31) / 32;
    // work buffers, cached in the context (grow-only)
    DBuf &vis = ctx->vs_vis, &qa = ctx->vs_qa, &qb = ctx->vs_qb, &hubs = ctx->vs_hubs, &ctl = ctx->vs_ctl;
    DBuf &cnt = ctx->vs_cnt, &tmp = ctx->vs_tmp;
    vis.ensure(ctx, words * 4 + 16);
    qa.ensure(ctx, (size_t)n * 4 + 16);
    qb.ensure(ctx, (size_t)n * 4 + 16);
    hubs.ensure(ctx, (size_t)n * 4 + 16);
    ctl.ensure(ctx, 3 * sizeof(VsCtl));
    k_vs_mark<<<grid_for(ctx, (long long)words), 256, 0, st>>>(vis.as<uint32_t>(), seed_bm, blk_bm, words);
    IM_CHECK_LAUNCH();
    IM_CUDA(cudaMemcpyAsync(qa.p, dS, (size_t)nS * 4, cudaMemcpyDeviceToDevice, st));
    int32_t *qin = qa.as<int32_t>(), *qout = qb.as<int32_t>();
    long long nin = nS;
    VsCtl h;
    // all levels in one cooperative launch when the device supports it
    // (IMIN_VS_PERSISTENT=0: one launch pair per level)
    int coop = 0, per_sm = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_vs_all, 256, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
    }
    const char *penv = std::getenv("IMIN_VS_PERSISTENT");
    if (coop && per_sm > 0 && !(penv && penv[0] == '0')) {
        IM_CUDA(cudaMemsetAsync(ctl.p, 0, 3 * sizeof(VsCtl), st));
        const int32_t *rp = g->row_ptr.as<int32_t>(), *cl = g->col.as<int32_t>();
        const uint32_t *th = g->thr.as<uint32_t>();
        uint32_t *vp = vis.as<uint32_t>();
        int32_t *pa = qa.as<int32_t>(), *pb = qb.as<int32_t>(), *ph = hubs.as<int32_t>();
        long long ns = nS;
        VsCtl *pc = ctl.as<VsCtl>();
        void *args[] = {(void *)&rp, (void *)&cl, (void *)&th, (void *)&vp, (void *)&pa, (void *)&pb,
                        (void *)&ns, (void *)&ph, (void *)&pc};
        IM_CUDA(cudaLaunchCooperativeKernel((const void *)k_vs_all, dim3(ctx->num_sms * std::min(per_sm, 4)),
                                            dim3(256), args, 0, st));
        IM_CHECK_LAUNCH();
        nin = 0;
    }
    while (nin > 0) {   // every node enters a frontier at most once
        IM_CUDA(cudaMemsetAsync(ctl.p, 0, sizeof(VsCtl), st));
        const int slices = (int)((nin + 31) / 32);
        const int blocks = std::max(1, std::min(ctx->num_sms * 8, (slices + 7) / 8));
        k_vs_expand<<<blocks, 256, 0, st>>>(g->row_ptr.as<int32_t>(), g->col.as<int32_t>(), g->thr.as<uint32_t>(),
                                            vis.as<uint32_t>(), qin, (int)nin, qout, hubs.as<int32_t>(),
                                            ctl.as<VsCtl>());
        IM_CHECK_LAUNCH();
        k_vs_hubs<<<ctx->num_sms * 2, 256, 0, st>>>(g->row_ptr.as<int32_t>(), g->col.as<int32_t>(),
                                                    g->thr.as<uint32_t>(), vis.as<uint32_t>(), qout,
                                                    hubs.as<int32_t>(), ctl.as<VsCtl>());
        IM_CHECK_LAUNCH();
        IM_CUDA(cudaMemcpyAsync(&h, ctl.p, sizeof(VsCtl), cudaMemcpyDeviceToHost, st));
        IM_CUDA(cudaStreamSynchronize(st));
        nin = h.nout;
        std::swap(qin, qout);
    }
    cnt.ensure(ctx, (words + 1) * 8);
    tmp.ensure(ctx, scan_tmp_bytes((int64_t)words + 1));
    k_vs_count<<<grid_for(ctx, (long long)words + 1), 256, 0, st>>>(vis.as<uint32_t>(), seed_bm, blk_bm, words, n,
                                                                    cnt.as<long long>());
    IM_CHECK_LAUNCH();
    exclusive_scan_i64(ctx, cnt.as<long long>(), (int64_t)words + 1, tmp.p);
    long long total = 0;
    IM_CUDA(cudaMemcpyAsync(&total, cnt.as<long long>() + words, 8, cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaStreamSynchronize(st));
    out.ensure(ctx, (size_t)total * 4 + 16);
    if (total > 0) {
        k_vs_scatter<<<grid_for(ctx, (long long)words), 256, 0, st>>>(vis.as<uint32_t>(), seed_bm, blk_bm, words, n,
                                                                      cnt.as<long long>(), out.as<int32_t>());
        IM_CHECK_LAUNCH();
    }
    return (int32_t)total;
}
