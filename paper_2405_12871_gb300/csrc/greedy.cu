// greedy.cu -- Procedure Max-Coverage (Algorithm 4) on the device.
//
// Lower bound (CP sets): the sets of one world are the DT ancestor chains of its
// reached non-seed nodes.  They are stored implicitly as records in DT preorder:
// rec_node, rec_par (distance back to the parent record, 0 for a chain root) and
// rec_size (subtree size).  The set of record r is {node of r and of its
// ancestors}; the records whose sets contain the node of r are exactly r's
// subtree [r, r + size).  Gains: gain[v] = sum over records x of v of
// contrib[x] = number of still-uncovered records in x's subtree.  Picking u
// covers the subtrees of u's uncovered records: their own contrib is removed
// from their nodes' gains, and every ancestor loses the newly covered count.
//
// Upper bound (LRR sets): classic max coverage with an inverted index.
//
// Every round is decided on the device (no host round trip): the argmax with
// ties to the smaller id, the exact sum of the k largest gains (a radix select
// over the 64-bit gains: 11-bit digits from the top bit of the maximum), the
// commit of the pick, and the decrement.  The host launches k + 1 rounds.
#include "greedy.cuh"

#include <algorithm>

namespace {

constexpr int RS_BITS = 11;
constexpr int RS_BINS = 1 << RS_BITS;

__device__ __forceinline__ bool better(unsigned long long g1, int v1, unsigned long long g2, int v2)
{
    return g1 > g2 || (g1 == g2 && v1 < v2);
}

// per-block argmax -> partials; the last block reduces, commits the pick, and
// initialises the top-k selection for this round.
__global__ void __launch_bounds__(256) k_argmax(GState *st, const unsigned long long *gain, int32_t n,
                                                unsigned long long *part_g, int32_t *part_v,
                                                unsigned int *done_ctr, int32_t round, int32_t k,
                                                int32_t *B, unsigned long long *cov)
{
    if (st->stopped) return;
    unsigned long long bg = 0;
    int bv = 0x7fffffff;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long gv = gain[v];
        if (better(gv, (int)v, bg, bv)) {
            bg = gv;
            bv = (int)v;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long og = __shfl_xor_sync(IMIN_FULL, bg, o);
        const int ov = __shfl_xor_sync(IMIN_FULL, bv, o);
        if (better(og, ov, bg, bv)) {
            bg = og;
            bv = ov;
        }
    }
    __shared__ unsigned long long sg[8];
    __shared__ int sv[8];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sg[w] = bg;
        sv[w] = bv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i)
            if (better(sg[i], sv[i], bg, bv)) {
                bg = sg[i];
                bv = sv[i];
            }
        part_g[blockIdx.x] = bg;
        part_v[blockIdx.x] = bv;
        __threadfence();
        const unsigned int t = atomicAdd(done_ctr, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    bg = 0;
    bv = 0x7fffffff;
    for (unsigned b = 0; b < gridDim.x; ++b) {
        const unsigned long long g = *(volatile unsigned long long *)(part_g + b);
        const int v = *(volatile int *)(part_v + b);
        if (better(g, v, bg, bv)) {
            bg = g;
            bv = v;
        }
    }
    *done_ctr = 0;
    st->gmax = bg;
    st->u = bv;
    st->pick = 0;
    // top-k selection state for this round
    st->tsum = 0;
    st->krem = k < n ? k : n;
    st->prefix = 0;
    if (bg == 0) {
        st->hi = 0;
        st->tdone = 1;
    } else {
        st->hi = 64 - __clzll((long long)bg);
        st->tdone = 0;
    }
    if (round < k) {
        if (bg == 0) {
            st->stopped = 1;          // nothing left to cover: |B| = round
            st->nb = round;
        } else {
            B[round] = bv;
            cov[round + 1] = cov[round] + bg;
            st->pick = 1;
            st->nb = round + 1;
        }
    }
}

// histogram of the next digit of the gains that match the selected prefix
__global__ void __launch_bounds__(256) k_topk_hist(const GState *st, const unsigned long long *gain,
                                                   int32_t n, unsigned int *hcnt,
                                                   unsigned long long *hsum)
{
    if (st->tdone) return;
    const int hi = st->hi;
    const int lo = hi > RS_BITS ? hi - RS_BITS : 0;
    const unsigned long long prefix = st->prefix;
    const unsigned long long dmask = (1ull << (hi - lo)) - 1ull;
    __shared__ unsigned int sc[RS_BINS];
    __shared__ unsigned long long ss[RS_BINS];
    for (int i = threadIdx.x; i < RS_BINS; i += blockDim.x) {
        sc[i] = 0;
        ss[i] = 0;
    }
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long g = gain[v];
        if (hi < 64 && (g >> hi) != (prefix >> hi)) continue;
        const int d = (int)((g >> lo) & dmask);
        atomicAdd(&sc[d], 1u);
        atomicAdd(&ss[d], g);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < RS_BINS; i += blockDim.x)
        if (sc[i]) {
            atomicAdd(hcnt + i, sc[i]);
            atomicAdd(hsum + i, ss[i]);
        }
}

// pick the digit that holds the k-th largest value; resolve when all bits are fixed
__global__ void __launch_bounds__(1024) k_topk_select(GState *st, unsigned int *hcnt,
                                                      unsigned long long *hsum,
                                                      unsigned long long *topk, int32_t round)
{
    if (st->tdone) return;
    __shared__ unsigned int c[RS_BINS];
    __shared__ unsigned long long s[RS_BINS];
    for (int i = threadIdx.x; i < RS_BINS; i += blockDim.x) {
        c[i] = hcnt[i];
        s[i] = hsum[i];
        hcnt[i] = 0;
        hsum[i] = 0;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int hi = st->hi;
    const int lo = hi > RS_BITS ? hi - RS_BITS : 0;
    const int nb = 1 << (hi - lo);
    long long krem = st->krem;
    unsigned long long tsum = st->tsum;
    int dstar = -1;
    for (int d = nb - 1; d >= 0; --d) {
        if ((long long)c[d] >= krem) {
            dstar = d;
            break;
        }
        krem -= c[d];
        tsum += s[d];
    }
    if (dstar < 0) {             // fewer candidates than k: the sum of all of them
        st->tsum = tsum;
        st->tdone = 1;
        topk[round] = tsum;
        return;
    }
    const unsigned long long prefix = st->prefix | ((unsigned long long)dstar << lo);
    if (lo == 0) {               // the k-th largest value is `prefix` itself
        tsum += (unsigned long long)krem * prefix;
        st->tsum = tsum;
        st->tdone = 1;
        topk[round] = tsum;
        return;
    }
    st->prefix = prefix;
    st->hi = lo;
    st->krem = (int32_t)krem;
    st->tsum = tsum;
}

__global__ void k_topk_zero(const GState *st, unsigned long long *topk, int32_t round)
{
    // gmax == 0: the top-k sum is 0
    if (st->tdone && st->tsum == 0 && st->gmax == 0) topk[round] = 0;
}

// Decrement for a pick on CP records: one warp per record of u.
__global__ void __launch_bounds__(256) k_cp_update(const GState *st, const long long *inv_off,
                                                   const long long *inv_rec,
                                                   const int32_t *rnode, const int32_t *rpar,
                                                   const int32_t *rsize, int32_t *contrib,
                                                   uint8_t *covered, unsigned long long *gain)
{
    if (!st->pick) return;
    const int u = st->u;
    const long long beg = inv_off[u], end = inv_off[u + 1];
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long idx = beg + gw; idx < end; idx += nw) {
        const long long r = inv_rec[idx];
        if (covered[r]) continue;
        const int newcov = contrib[r];
        if (lane == 0) {
            long long x = r;
            int po = rpar[x];
            while (po != 0) {
                x -= po;
                contrib[x] -= newcov;
                atomicAdd(gain + rnode[x], (unsigned long long)(-(long long)newcov));
                po = rpar[x];
            }
        }
        const long long e = r + rsize[r];
        for (long long x = r + lane; x < e; x += 32) {
            if (covered[x]) continue;
            const int c = contrib[x];
            if (c) atomicAdd(gain + rnode[x], (unsigned long long)(-(long long)c));
            contrib[x] = 0;
            covered[x] = 1;
        }
        __syncwarp();
    }
}

// Decrement for a pick on LRR sets: one warp per set of u.
__global__ void __launch_bounds__(256) k_lrr_update(const GState *st, const long long *inv_off,
                                                    const uint32_t *inv_set,
                                                    const unsigned long long *set_off,
                                                    const uint32_t *set_len,
                                                    const int32_t *set_elem, uint8_t *covered,
                                                    unsigned long long *gain)
{
    if (!st->pick) return;
    const int u = st->u;
    const long long beg = inv_off[u], end = inv_off[u + 1];
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long idx = beg + gw; idx < end; idx += nw) {
        const uint32_t s = inv_set[idx];
        if (covered[s]) continue;
        const unsigned long long o = set_off[s];
        const uint32_t L = set_len[s];
        for (uint32_t t = lane; t < L; t += 32) atomicAdd(gain + set_elem[o + t], ~0ull);
        __syncwarp();
        if (lane == 0) covered[s] = 1;
    }
}

// ---- inverted indices ----------------------------------------------------------
__global__ void k_count_nodes(const int32_t *nodes, long long cnt, long long *counts)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x)
        atomicAdd((unsigned long long *)(counts + nodes[i]), 1ull);
}

__global__ void k_fill_cp_inv(const int32_t *rnode, long long cnt, const long long *inv_off,
                              unsigned int *fill, long long *inv_rec)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x) {
        const int v = rnode[i];
        inv_rec[inv_off[v] + atomicAdd(fill + v, 1u)] = i;
    }
}

__global__ void k_fill_lrr_inv(const unsigned long long *set_off, const uint32_t *set_len,
                               uint32_t nsets, const int32_t *set_elem, const long long *inv_off,
                               unsigned int *fill, uint32_t *inv_set)
{
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long s = gw; s < nsets; s += nw) {
        const unsigned long long o = set_off[s];
        const uint32_t L = set_len[s];
        for (uint32_t t = lane; t < L; t += 32) {
            const int v = set_elem[o + t];
            inv_set[inv_off[v] + atomicAdd(fill + v, 1u)] = (uint32_t)s;
        }
    }
}

__global__ void k_init_cp(const int32_t *rsize, long long cnt, int32_t *contrib, uint8_t *covered)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x) {
        contrib[i] = rsize[i];
        covered[i] = 0;
    }
}

// ---- coverage of a fixed set B ----------------------------------------------------
__device__ __forceinline__ bool in_bm(const uint32_t *bm, int v) { return (bm[v >> 5] >> (v & 31)) & 1u; }

__global__ void __launch_bounds__(256) k_cov_cp(const int32_t *rnode, const int32_t *rpar,
                                                const int32_t *rsize, long long cnt,
                                                const uint32_t *inB, unsigned long long *out)
{
    unsigned long long acc = 0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < cnt;
         r += (long long)gridDim.x * blockDim.x) {
        if (!in_bm(inB, rnode[r])) continue;
        // count r's subtree unless an ancestor is also in B (then it is counted there)
        long long x = r;
        int po = rpar[x];
        bool top = true;
        while (po != 0) {
            x -= po;
            if (in_bm(inB, rnode[x])) {
                top = false;
                break;
            }
            po = rpar[x];
        }
        if (top) acc += (unsigned long long)rsize[r];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(IMIN_FULL, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

__global__ void __launch_bounds__(256) k_cov_lrr(const unsigned long long *set_off,
                                                 const uint32_t *set_len, uint32_t nsets,
                                                 const int32_t *set_elem, const uint32_t *inB,
                                                 unsigned long long *out)
{
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long acc = 0;
    for (long long s = gw; s < nsets; s += nw) {
        const unsigned long long o = set_off[s];
        const uint32_t L = set_len[s];
        bool hit = false;
        for (uint32_t t = lane; t < L && !hit; t += 32) hit = in_bm(inB, set_elem[o + t]);
        if (__any_sync(IMIN_FULL, hit)) acc += 1;
    }
    if (lane == 0 && acc) atomicAdd(out, acc);
}

}  // namespace

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
static int grid_for(imin_ctx *ctx, long long work, int per_block = 256)
{
    long long b = (work + per_block - 1) / per_block;
    long long cap = (long long)ctx->num_sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

void greedy_scratch(imin_ctx *ctx, GreedyBufs &gb, int32_t n, int32_t k)
{
    const int parts = ctx->num_sms * 8;
    gb.state.ensure(ctx, sizeof(GState));
    gb.part_g.ensure(ctx, (size_t)parts * 8);
    gb.part_v.ensure(ctx, (size_t)parts * 4);
    gb.done.ensure(ctx, 64);
    gb.hcnt.ensure(ctx, RS_BINS * 4);
    gb.hsum.ensure(ctx, RS_BINS * 8);
    gb.B.ensure(ctx, (size_t)(k + 1) * 4);
    gb.cov.ensure(ctx, (size_t)(k + 2) * 8);
    gb.topk.ensure(ctx, (size_t)(k + 2) * 8);
    gb.gain.ensure(ctx, (size_t)n * 8);
    IM_CUDA(cudaMemsetAsync(gb.done.p, 0, 64, ctx->stream));
    IM_CUDA(cudaMemsetAsync(gb.hcnt.p, 0, RS_BINS * 4, ctx->stream));
    IM_CUDA(cudaMemsetAsync(gb.hsum.p, 0, RS_BINS * 8, ctx->stream));
    IM_CUDA(cudaMemsetAsync(gb.state.p, 0, sizeof(GState), ctx->stream));
    IM_CUDA(cudaMemsetAsync(gb.cov.p, 0, (size_t)(k + 2) * 8, ctx->stream));
    IM_CUDA(cudaMemsetAsync(gb.topk.p, 0, (size_t)(k + 2) * 8, ctx->stream));
}

// k + 1 rounds of argmax / top-k / decrement.  `update` launches the decrement.
template <class F>
static void greedy_rounds(imin_ctx *ctx, GreedyBufs &gb, int32_t n, int32_t k, F update)
{
    const int grid = grid_for(ctx, n);
    GState *st = gb.state.as<GState>();
    for (int32_t round = 0; round <= k; ++round) {
        k_argmax<<<grid, 256, 0, ctx->stream>>>(st, gb.gain.as<unsigned long long>(), n,
                                                gb.part_g.as<unsigned long long>(),
                                                gb.part_v.as<int32_t>(), gb.done.as<unsigned int>(),
                                                round, k, gb.B.as<int32_t>(),
                                                gb.cov.as<unsigned long long>());
        IM_CHECK_LAUNCH();
        for (int pass = 0; pass < 6; ++pass) {
            k_topk_hist<<<grid, 256, 0, ctx->stream>>>(st, gb.gain.as<unsigned long long>(), n,
                                                       gb.hcnt.as<unsigned int>(),
                                                       gb.hsum.as<unsigned long long>());
            IM_CHECK_LAUNCH();
            k_topk_select<<<1, 1024, 0, ctx->stream>>>(st, gb.hcnt.as<unsigned int>(),
                                                       gb.hsum.as<unsigned long long>(),
                                                       gb.topk.as<unsigned long long>(), round);
            IM_CHECK_LAUNCH();
        }
        k_topk_zero<<<1, 1, 0, ctx->stream>>>(st, gb.topk.as<unsigned long long>(), round);
        IM_CHECK_LAUNCH();
        if (round < k) update();
    }
}

void greedy_cp(imin_ctx *ctx, GreedyBufs &gb, CpStore &c, int32_t n, int32_t k,
               const unsigned long long *credit)
{
    cudaStream_t s = ctx->stream;
    const long long R = c.count;
    // inverted index node -> records
    c.inv_off.ensure(ctx, (size_t)(n + 1) * 8);
    c.inv_rec.ensure(ctx, (size_t)std::max<long long>(R, 1) * 8);
    c.fill.ensure(ctx, (size_t)(n + 1) * 4);
    c.contrib.ensure(ctx, (size_t)std::max<long long>(R, 1) * 4);
    c.covered.ensure(ctx, (size_t)std::max<long long>(R, 1));
    c.scan_tmp.ensure(ctx, scan_tmp_bytes(n + 1));
    IM_CUDA(cudaMemsetAsync(c.inv_off.p, 0, (size_t)(n + 1) * 8, s));
    IM_CUDA(cudaMemsetAsync(c.fill.p, 0, (size_t)(n + 1) * 4, s));
    if (R > 0) {
        k_count_nodes<<<grid_for(ctx, R), 256, 0, s>>>(c.node.as<int32_t>(), R, c.inv_off.as<long long>());
        IM_CHECK_LAUNCH();
    }
    exclusive_scan_i64(ctx, c.inv_off.as<long long>(), n + 1, c.scan_tmp.p);
    if (R > 0) {
        k_fill_cp_inv<<<grid_for(ctx, R), 256, 0, s>>>(c.node.as<int32_t>(), R, c.inv_off.as<long long>(),
                                                      c.fill.as<unsigned int>(), c.inv_rec.as<long long>());
        k_init_cp<<<grid_for(ctx, R), 256, 0, s>>>(c.size.as<int32_t>(), R, c.contrib.as<int32_t>(),
                                                  c.covered.as<uint8_t>());
        IM_CHECK_LAUNCH();
    }
    greedy_scratch(ctx, gb, n, k);
    IM_CUDA(cudaMemcpyAsync(gb.gain.p, credit, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    const int ugrid = ctx->num_sms * 8;
    greedy_rounds(ctx, gb, n, k, [&]() {
        k_cp_update<<<ugrid, 256, 0, s>>>(gb.state.as<GState>(), c.inv_off.as<long long>(),
                                          c.inv_rec.as<long long>(), c.node.as<int32_t>(),
                                          c.par.as<int32_t>(), c.size.as<int32_t>(),
                                          c.contrib.as<int32_t>(), c.covered.as<uint8_t>(),
                                          gb.gain.as<unsigned long long>());
        IM_CHECK_LAUNCH();
    });
}

void greedy_lrr(imin_ctx *ctx, GreedyBufs &gb, LrrStore &L, int32_t n, int32_t k,
                const unsigned long long *credit)
{
    cudaStream_t s = ctx->stream;
    const long long E = (long long)L.elems;
    const uint32_t ns = L.nsets;
    L.inv_off.ensure(ctx, (size_t)(n + 1) * 8);
    L.inv_set.ensure(ctx, (size_t)std::max<long long>(E, 1) * 4);
    L.fill.ensure(ctx, (size_t)(n + 1) * 4);
    L.covered.ensure(ctx, (size_t)std::max<uint32_t>(ns, 1));
    L.scan_tmp.ensure(ctx, scan_tmp_bytes(n + 1));
    IM_CUDA(cudaMemsetAsync(L.inv_off.p, 0, (size_t)(n + 1) * 8, s));
    IM_CUDA(cudaMemsetAsync(L.fill.p, 0, (size_t)(n + 1) * 4, s));
    IM_CUDA(cudaMemsetAsync(L.covered.p, 0, (size_t)std::max<uint32_t>(ns, 1), s));
    if (E > 0) {
        k_count_nodes<<<grid_for(ctx, E), 256, 0, s>>>(L.elem.as<int32_t>(), E, L.inv_off.as<long long>());
        IM_CHECK_LAUNCH();
    }
    exclusive_scan_i64(ctx, L.inv_off.as<long long>(), n + 1, L.scan_tmp.p);
    if (ns > 0) {
        k_fill_lrr_inv<<<grid_for(ctx, (long long)ns * 32), 256, 0, s>>>(
            L.off.as<unsigned long long>(), L.len.as<uint32_t>(), ns, L.elem.as<int32_t>(),
            L.inv_off.as<long long>(), L.fill.as<unsigned int>(), L.inv_set.as<uint32_t>());
        IM_CHECK_LAUNCH();
    }
    greedy_scratch(ctx, gb, n, k);
    IM_CUDA(cudaMemcpyAsync(gb.gain.p, credit, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    const int ugrid = ctx->num_sms * 8;
    greedy_rounds(ctx, gb, n, k, [&]() {
        k_lrr_update<<<ugrid, 256, 0, s>>>(gb.state.as<GState>(), L.inv_off.as<long long>(),
                                           L.inv_set.as<uint32_t>(), L.off.as<unsigned long long>(),
                                           L.len.as<uint32_t>(), L.elem.as<int32_t>(),
                                           L.covered.as<uint8_t>(), gb.gain.as<unsigned long long>());
        IM_CHECK_LAUNCH();
    });
}

unsigned long long cov_cp(imin_ctx *ctx, CpStore &c, const uint32_t *inB, unsigned long long *d_out,
                          unsigned long long *h_out)
{
    IM_CUDA(cudaMemsetAsync(d_out, 0, 8, ctx->stream));
    if (c.count > 0) {
        k_cov_cp<<<grid_for(ctx, c.count), 256, 0, ctx->stream>>>(
            c.node.as<int32_t>(), c.par.as<int32_t>(), c.size.as<int32_t>(), c.count, inB, d_out);
        IM_CHECK_LAUNCH();
    }
    IM_CUDA(cudaMemcpyAsync(h_out, d_out, 8, cudaMemcpyDeviceToHost, ctx->stream));
    IM_CUDA(cudaStreamSynchronize(ctx->stream));
    return *h_out;
}

unsigned long long cov_lrr(imin_ctx *ctx, LrrStore &L, const uint32_t *inB, unsigned long long *d_out,
                           unsigned long long *h_out)
{
    IM_CUDA(cudaMemsetAsync(d_out, 0, 8, ctx->stream));
    if (L.nsets > 0) {
        k_cov_lrr<<<grid_for(ctx, (long long)L.nsets * 32), 256, 0, ctx->stream>>>(
            L.off.as<unsigned long long>(), L.len.as<uint32_t>(), L.nsets, L.elem.as<int32_t>(), inB,
            d_out);
        IM_CHECK_LAUNCH();
    }
    IM_CUDA(cudaMemcpyAsync(h_out, d_out, 8, cudaMemcpyDeviceToHost, ctx->stream));
    IM_CUDA(cudaStreamSynchronize(ctx->stream));
    return *h_out;
}
