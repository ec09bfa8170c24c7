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
// The host reads two counters per level.  The list is then read off the bitmap in
// ascending order (a per-word population count, a scan, a scatter).
#include "common.cuh"

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
    DBuf vis, qa, qb, hubs, ctl, cnt, tmp;
    vis.ensure(ctx, words * 4 + 16);
    qa.ensure(ctx, (size_t)n * 4 + 16);
    qb.ensure(ctx, (size_t)n * 4 + 16);
    hubs.ensure(ctx, (size_t)n * 4 + 16);
    ctl.ensure(ctx, sizeof(VsCtl));
    k_vs_mark<<<grid_for(ctx, (long long)words), 256, 0, st>>>(vis.as<uint32_t>(), seed_bm, blk_bm, words);
    IM_CHECK_LAUNCH();
    IM_CUDA(cudaMemcpyAsync(qa.p, dS, (size_t)nS * 4, cudaMemcpyDeviceToDevice, st));
    int32_t *qin = qa.as<int32_t>(), *qout = qb.as<int32_t>();
    long long nin = nS;
    VsCtl h;
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
