// hot_view.cu -- the relabelled forward index of one query (HotView, common.cuh).
//
// Labels: nodes in decreasing order of their reach count over a short run of the
// query's worlds (a counting sort over the count values; nodes with equal counts in an
// arbitrary order, which changes no result: the traversals that use the view only count
// nodes).  Edges: label r's out-edges [b, e) are the original groups b/4 .. (e-1)/4
// copied, whole, to consecutive new groups starting at base(r) (a scan of the group
// counts in label order), so an edge keeps its lane in its group; its new position is
// 4 base(r) + (b mod 4) + (its offset in the row).  Every new group records its
// original index, which is the coin counter of its four edges (Eq. of the coin rule:
// Philox over the group index, the world, the stream tag and the instance).
#include "common.cuh"

#include <vector>

namespace {

constexpr int HV_BD = 256;
constexpr int HV_ITEMS = 8;   // nodes per thread in the placement kernel

__global__ void k_count_hist(const unsigned long long *counts, int32_t n, uint32_t maxc, uint32_t *hist)
{
    extern __shared__ uint32_t s_hist[];   // maxc + 1 bins
    for (uint32_t b = threadIdx.x; b <= maxc; b += blockDim.x) s_hist[b] = 0;
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long c = counts[v];
        atomicAdd(&s_hist[c < maxc ? (uint32_t)c : maxc], 1u);
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b <= maxc; b += blockDim.x)
        if (s_hist[b]) atomicAdd(hist + b, s_hist[b]);
}

// Each block places HV_BD * HV_ITEMS consecutive nodes: a rank inside the block per
// count value (shared-memory atomics), one reservation per count value and block in
// the global cursor, then label = off[count] + reservation + rank.
__global__ void k_place(const unsigned long long *counts, int32_t n, uint32_t maxc, const uint32_t *off,
                        uint32_t *cursor, int32_t *perm, int32_t *inv)
{
    extern __shared__ uint32_t s_mem[];
    uint32_t *lc = s_mem;              // maxc + 1: nodes of the block per count value
    uint32_t *base = s_mem + maxc + 1; // maxc + 1: the block's reservation per count value
    for (uint32_t b = threadIdx.x; b <= maxc; b += blockDim.x) lc[b] = 0;
    __syncthreads();
    const int64_t v0 = (int64_t)blockIdx.x * HV_BD * HV_ITEMS;
    uint32_t bin[HV_ITEMS], rank[HV_ITEMS];
#pragma unroll
    for (int i = 0; i < HV_ITEMS; ++i) {
        const int64_t v = v0 + (int64_t)i * HV_BD + threadIdx.x;
        bin[i] = 0;
        rank[i] = 0;
        if (v < n) {
            const unsigned long long c = counts[v];
            bin[i] = c < maxc ? (uint32_t)c : maxc;
            rank[i] = atomicAdd(&lc[bin[i]], 1u);
        }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b <= maxc; b += blockDim.x)
        if (lc[b]) base[b] = atomicAdd(cursor + b, lc[b]);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < HV_ITEMS; ++i) {
        const int64_t v = v0 + (int64_t)i * HV_BD + threadIdx.x;
        if (v < n) {
            const int32_t r = (int32_t)(off[bin[i]] + base[bin[i]] + rank[i]);
            perm[v] = r;
            inv[r] = (int32_t)v;
        }
    }
}

// groups[r] = the number of original groups label r's out-edges touch
__global__ void k_row_groups(const int32_t *row_ptr, const int32_t *inv, int32_t n, long long *groups)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n) return;
    if (r == n) {
        groups[r] = 0;
        return;
    }
    const int32_t v = inv[r];
    const int32_t b = row_ptr[v], e = row_ptr[v + 1];
    groups[r] = e > b ? (long long)(((e + 3) >> 2) - (b >> 2)) : 0ll;
}

// one warp per label: its range in the new positions and its groups, copied with the
// targets relabelled (lanes outside the row keep a relabelled in-range target or 0:
// they are masked by the range and never followed)
__global__ void k_fill(const int32_t *row_ptr, const uint4 *ce, const int32_t *perm, const int32_t *inv,
                       const long long *gbase, int32_t n, int2 *rng, uint4 *nce, uint32_t *gid)
{
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w; r < n; r += nw) {
        const int32_t v = inv[r];
        const int32_t b = row_ptr[v], e = row_ptr[v + 1];
        const long long nb = gbase[r];
        if (lane == 0) {
            const int32_t nbeg = (int32_t)(nb * 4 + (b & 3));
            rng[r] = make_int2(nbeg, nbeg + (e - b));
        }
        if (e <= b) continue;
        const int32_t g0 = b >> 2, cnt = ((e + 3) >> 2) - g0;
        for (int32_t i = lane; i < cnt; i += 32) {
            const uint4 t = ce[2 * (size_t)(g0 + i)];
            const uint4 th = ce[2 * (size_t)(g0 + i) + 1];
            auto lab = [&](uint32_t x) -> uint32_t { return x < (uint32_t)n ? (uint32_t)perm[x] : 0u; };
            const size_t ng = (size_t)(nb + i);
            nce[2 * ng] = make_uint4(lab(t.x), lab(t.y), lab(t.z), lab(t.w));
            nce[2 * ng + 1] = th;
            gid[ng] = (uint32_t)(g0 + i);
        }
    }
}

__global__ void k_map(const int32_t *perm, const int32_t *src, int32_t cnt, int32_t *dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) dst[i] = perm[src[i]];
}

}  // namespace

int hot_view_build(imin_ctx *ctx, const imin_graph *g, const unsigned long long *d_counts, uint32_t max_count,
                   const int32_t *d_S, int32_t nS, HotView &hv)
{
    hv.on = false;
    const int32_t n = g->n;
    if (n <= 0) return 0;
    cudaStream_t st = ctx->stream;
    const uint32_t maxc = std::max<uint32_t>(max_count, 1u);
    const size_t nbins = (size_t)maxc + 1;
    // count histogram, then label offsets per count value, most often reached first
    DBuf tmp;
    tmp.ensure(ctx, nbins * 8 + 64);
    uint32_t *hist = tmp.as<uint32_t>(), *cursor = hist + nbins;
    IM_CUDA(cudaMemsetAsync(tmp.p, 0, nbins * 8, st));
    const size_t smem1 = nbins * 4, smem2 = nbins * 8;
    if (smem2 > 48 * 1024) throw ImError{IMIN_EINVAL, "hot view: more than 6,143 count values"};
    const int hblocks = std::max(1, std::min(ctx->num_sms * 4, (int)((n + HV_BD - 1) / HV_BD)));
    k_count_hist<<<hblocks, HV_BD, smem1, st>>>(d_counts, n, maxc, hist);
    IM_CHECK_LAUNCH();
    std::vector<uint32_t> h(nbins), off(nbins);
    IM_CUDA(cudaMemcpyAsync(h.data(), hist, nbins * 4, cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaStreamSynchronize(st));
    uint64_t acc = 0;
    for (size_t b = nbins; b-- > 0;) {
        off[b] = (uint32_t)acc;
        acc += h[b];
    }
    IM_CUDA(cudaMemcpyAsync(hist, off.data(), nbins * 4, cudaMemcpyHostToDevice, st));
    hv.perm.ensure(ctx, (size_t)n * 4);
    DBuf inv;
    inv.ensure(ctx, (size_t)n * 4);
    const int64_t per_block = (int64_t)HV_BD * HV_ITEMS;
    k_place<<<(unsigned)((n + per_block - 1) / per_block), HV_BD, smem2, st>>>(
        d_counts, n, maxc, hist, cursor, hv.perm.as<int32_t>(), inv.as<int32_t>());
    IM_CHECK_LAUNCH();
    // new group positions: an exclusive scan of the label order's group counts
    DBuf gb;
    const size_t sb = scan_tmp_bytes((int64_t)n + 1);
    gb.ensure(ctx, ((size_t)n + 1) * 8 + sb);
    long long *gbase = gb.as<long long>();
    k_row_groups<<<(unsigned)((n + 1 + 255) / 256), 256, 0, st>>>(g->row_ptr.as<int32_t>(), inv.as<int32_t>(), n,
                                                                  gbase);
    IM_CHECK_LAUNCH();
    exclusive_scan_i64(ctx, gbase, (int64_t)n + 1, reinterpret_cast<char *>(gb.p) + ((size_t)n + 1) * 8);
    long long total = 0;
    IM_CUDA(cudaMemcpyAsync(&total, gbase + n, 8, cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaStreamSynchronize(st));
    // edge positions are int32 in the traversals: 4 x groups + 4 must stay below 2^31
    const int launches = 3 + scan_launches((int64_t)n + 1);
    if (total < 0 || 4 * (total + 1) >= ((long long)1 << 31)) {
        hv.release();
        return launches;
    }
    const size_t groups = (size_t)std::max<long long>(total, 1);
    hv.rng.ensure(ctx, (size_t)n * 8);
    hv.ce.ensure(ctx, groups * 32);
    hv.gid.ensure(ctx, groups * 4);
    const int fblocks = std::max(1, std::min(ctx->num_sms * 8, (int)(((int64_t)n * 32 + 255) / 256)));
    k_fill<<<fblocks, 256, 0, st>>>(g->row_ptr.as<int32_t>(), g->ce.as<uint4>(), hv.perm.as<int32_t>(),
                                    inv.as<int32_t>(), gbase, n, hv.rng.as<int2>(), hv.ce.as<uint4>(),
                                    hv.gid.as<uint32_t>());
    IM_CHECK_LAUNCH();
    hv.S.ensure(ctx, (size_t)std::max(nS, 1) * 4);
    if (nS > 0) {
        k_map<<<(nS + 255) / 256, 256, 0, st>>>(hv.perm.as<int32_t>(), d_S, nS, hv.S.as<int32_t>());
        IM_CHECK_LAUNCH();
    }
    IM_CUDA(cudaStreamSynchronize(st));
    hv.n = n;
    hv.on = true;
    return launches + 1 + (nS > 0 ? 1 : 0);
}

void hot_view_map(imin_ctx *ctx, const HotView &hv, const int32_t *d_src, int32_t cnt, int32_t *d_dst)
{
    if (cnt <= 0) return;
    k_map<<<(cnt + 255) / 256, 256, 0, ctx->stream>>>(hv.perm.as<int32_t>(), d_src, cnt, d_dst);
    IM_CHECK_LAUNCH();
}
