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

#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>

namespace cg = cooperative_groups;

namespace {

constexpr int RS_BITS = 11;
constexpr int RS_BINS = 1 << RS_BITS;
constexpr long long CHUNK = 256;   // subtree entries per update work item (CP)

__device__ __forceinline__ bool better(unsigned long long g1, int v1, unsigned long long g2, int v2)
{
    return g1 > g2 || (g1 == g2 && v1 < v2);
}

// Every step below serves all instances of a batch: a table maps each (virtual) block
// to its instance, so one pass over the blocks covers every Max-Coverage run at once.
// The steps run either as one launch each per round, or all k + 1 rounds inside one
// cooperative persistent kernel with a grid barrier between steps.  Inside the
// persistent kernel, data that other blocks change (gains, record state, round
// state, histograms) is read through L2 (__ldcg / volatile), never from L1.

struct RoundSmem {
    unsigned int c[RS_BINS];
    unsigned long long s[RS_BINS];
    unsigned long long wg[8];
    int wv[8];
    int last;
};

// per-block argmax -> partials; the instance's last block reduces, commits the pick
// and initialises the top-k selection of this round
__device__ __forceinline__ void step_argmax(const GInst *gi, const int32_t *blk2inst, int vb,
                                            int32_t round, RoundSmem &sm)
{
    const GInst &I = gi[blk2inst[vb]];
    if (round > I.k) return;
    volatile GState *st = I.st;
    if (st->stopped) return;
    const int lb = vb - I.blk0;
    const int32_t n = I.n;
    unsigned long long bg = 0;
    int bv = 0x7fffffff;
    // only candidates can have a nonzero gain; a zero maximum stops the run either way
    for (int64_t i = (int64_t)lb * blockDim.x + threadIdx.x; i < I.ncand; i += (int64_t)I.nblk * blockDim.x) {
        const int v = I.cand[i];
        const unsigned long long gv = __ldcg(I.gain + v);
        if (better(gv, v, bg, bv)) {
            bg = gv;
            bv = v;
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
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sm.wg[w] = bg;
        sm.wv[w] = bv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i)
            if (better(sm.wg[i], sm.wv[i], bg, bv)) {
                bg = sm.wg[i];
                bv = sm.wv[i];
            }
        I.part_g[lb] = bg;
        I.part_v[lb] = bv;
        __threadfence();
        const unsigned int t = atomicAdd(I.done_ctr, 1u);
        sm.last = (t == (unsigned)I.nblk - 1);
    }
    __syncthreads();
    const bool last = sm.last;
    __syncthreads();   // sm is reused by the next step
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    bg = 0;
    bv = 0x7fffffff;
    for (int b = 0; b < I.nblk; ++b) {
        const unsigned long long g = *(volatile unsigned long long *)(I.part_g + b);
        const int v = *(volatile int *)(I.part_v + b);
        if (better(g, v, bg, bv)) {
            bg = g;
            bv = v;
        }
    }
    *(volatile unsigned int *)I.done_ctr = 0;
    st->gmax = bg;
    st->u = bv;
    st->pick = 0;
    st->tsum = 0;
    st->krem = I.k < n ? I.k : n;
    st->prefix = 0;
    if (bg == 0) {
        st->hi = 0;
        st->tdone = 1;
        st->npass = 0;
        I.topk[round] = 0;            // every gain is 0
    } else {
        st->hi = 64 - __clzll((long long)bg);
        st->tdone = 0;
        st->npass = (st->hi + RS_BITS - 1) / RS_BITS;
    }
    if (round < I.k) {
        if (bg == 0) {
            st->stopped = 1;          // nothing left to cover: |B| = round
            st->nb = round;
        } else {
            I.B[round] = bv;
            I.cov[round + 1] = *(volatile unsigned long long *)(I.cov + round) + bg;
            st->pick = 1;
            st->nb = round + 1;
        }
    }
    __threadfence();
}

// one block: pick the digit that holds the k-th largest value from the histogram in
// sm; resolve when all bits are fixed
__device__ __forceinline__ void select_digit(const GInst &I, int32_t round, RoundSmem &sm)
{
    volatile GState *st = I.st;
    const int hi = st->hi;
    const int lo = hi > RS_BITS ? hi - RS_BITS : 0;
    const int nb = 1 << (hi - lo);
    long long krem = st->krem;
    unsigned long long tsum = st->tsum;
    int dstar = -1;
    for (int d = nb - 1; d >= 0; --d) {
        if ((long long)sm.c[d] >= krem) {
            dstar = d;
            break;
        }
        krem -= sm.c[d];
        tsum += sm.s[d];
    }
    if (dstar < 0) {             // fewer candidates than k: the sum of all of them
        st->tsum = tsum;
        st->tdone = 1;
        I.topk[round] = tsum;
        return;
    }
    const unsigned long long prefix = st->prefix | ((unsigned long long)dstar << lo);
    if (lo == 0) {               // the k-th largest value is `prefix` itself
        tsum += (unsigned long long)krem * prefix;
        st->tsum = tsum;
        st->tdone = 1;
        I.topk[round] = tsum;
        return;
    }
    st->prefix = prefix;
    st->hi = lo;
    st->krem = (int32_t)krem;
    st->tsum = tsum;
}

// histogram of the next digit of the gains that match the selected prefix; with
// `fused`, the instance's last block then selects the digit (otherwise a separate
// one-block-per-instance step does)
__device__ __forceinline__ void step_hist(const GInst *gi, const int32_t *blk2inst, int vb,
                                          int32_t round, RoundSmem &sm, bool fused)
{
    const GInst &I = gi[blk2inst[vb]];
    if (round > I.k) return;
    volatile GState *st = I.st;
    if (st->tdone) return;
    const int lb = vb - I.blk0;
    const int hi = st->hi;
    const int lo = hi > RS_BITS ? hi - RS_BITS : 0;
    const unsigned long long prefix = st->prefix;
    const unsigned long long dmask = (1ull << (hi - lo)) - 1ull;
    for (int i = threadIdx.x; i < RS_BINS; i += blockDim.x) {
        sm.c[i] = 0;
        sm.s[i] = 0;
    }
    __syncthreads();
    // gains of non-candidates are 0 and never reach the k largest sum
    for (int64_t i = (int64_t)lb * blockDim.x + threadIdx.x; i < I.ncand; i += (int64_t)I.nblk * blockDim.x) {
        const unsigned long long g = __ldcg(I.gain + I.cand[i]);
        if (hi < 64 && (g >> hi) != (prefix >> hi)) continue;
        const int d = (int)((g >> lo) & dmask);
        atomicAdd(&sm.c[d], 1u);
        atomicAdd(&sm.s[d], g);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < RS_BINS; i += blockDim.x)
        if (sm.c[i]) {
            atomicAdd(I.hcnt + i, sm.c[i]);
            atomicAdd(I.hsum + i, sm.s[i]);
        }
    if (!fused) {
        __syncthreads();
        return;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sm.last = atomicAdd(I.done_ctr2, 1u) == (unsigned)I.nblk - 1;
    __syncthreads();
    if (sm.last) {
        __threadfence();
        for (int i = threadIdx.x; i < RS_BINS; i += blockDim.x) {
            sm.c[i] = __ldcg(I.hcnt + i);
            sm.s[i] = __ldcg(I.hsum + i);
            I.hcnt[i] = 0;
            I.hsum[i] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            *(volatile unsigned int *)I.done_ctr2 = 0;
            select_digit(I, round, sm);
            __threadfence();
        }
    }
    __syncthreads();
}

// one block per instance (the non-fused form)
__device__ __forceinline__ void step_select(const GInst *gi, int inst, int32_t round, RoundSmem &sm)
{
    const GInst &I = gi[inst];
    if (round > I.k) return;
    if (I.st->tdone) return;
    for (int i = threadIdx.x; i < RS_BINS; i += blockDim.x) {
        sm.c[i] = I.hcnt[i];
        sm.s[i] = I.hsum[i];
        I.hcnt[i] = 0;
        I.hsum[i] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) select_digit(I, round, sm);
    __syncthreads();
}

// Decrement after a pick: one warp per record (CP) or set (LRR) of u.
__device__ __forceinline__ void step_update(const GInst *gi, const int32_t *ublk2inst, int vb,
                                            int32_t round, int lrr)
{
    const GInst &I = gi[ublk2inst[vb]];
    if (round >= I.k) return;
    volatile GState *st = I.st;
    if (!st->pick) return;
    const int u = st->u;
    const long long beg = I.inv_off[u], end = I.inv_off[u + 1];
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)(vb - I.ublk0) * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)I.unblk * blockDim.x) >> 5;
    unsigned long long *gain = I.gain;
    if (!lrr) {
        // u's records are cut into chunks of CHUNK subtree entries so that one large
        // subtree spreads over many warps.  Chunk 0 of a record also takes the record
        // itself: if it was still uncovered, its ancestors lose its remaining count.
        // A record covered earlier has its whole subtree covered (covering is closed
        // under subtrees), so the other chunks of such a record find nothing to do.
        const long long cb = I.inv_cpre[beg], cend = I.inv_cpre[end];
        for (long long ch = cb + gw; ch < cend; ch += nw) {
            long long lo = beg, hi = end;   // inv_cpre[lo] <= ch < inv_cpre[hi]
            while (hi - lo > 1) {
                const long long mid = (lo + hi) >> 1;
                if (I.inv_cpre[mid] <= ch) lo = mid; else hi = mid;
            }
            const long long r = I.inv_rec[lo];
            const long long c = ch - I.inv_cpre[lo];
            const long long x0 = r + c * CHUNK;
            const long long x1 = min(r + (long long)I.rsize[r], x0 + CHUNK);
            if (c == 0) {
                if (__ldcg(I.covered + r)) continue;
                const int newcov = __ldcg(I.contrib + r);
                if (lane == 0) {
                    long long x = r;
                    int po = I.rpar[x];
                    while (po != 0) {
                        x -= po;
                        atomicSub(I.contrib + x, newcov);
                        atomicAdd(gain + I.rnode[x], (unsigned long long)(-(long long)newcov));
                        po = I.rpar[x];
                    }
                }
            }
            for (long long x = x0 + lane; x < x1; x += 32) {
                const uint8_t cv = __ldcg(I.covered + x);
                const int cx = __ldcg(I.contrib + x);
                if (cv) continue;
                if (cx) atomicAdd(gain + I.rnode[x], (unsigned long long)(-(long long)cx));
                __stcg(I.contrib + x, 0);
                __stcg(I.covered + x, (uint8_t)1);
            }
            __syncwarp();
        }
    } else {
        for (long long idx = beg + gw; idx < end; idx += nw) {
            const uint32_t s = I.inv_set[idx];
            if (__ldcg(I.covered + s)) continue;
            const unsigned long long o = I.set_off[s];
            const uint32_t L = I.set_len[s];
            for (uint32_t t = lane; t < L; t += 32) atomicAdd(gain + I.set_elem[o + t], ~0ull);
            __syncwarp();
            if (lane == 0) __stcg(I.covered + s, (uint8_t)1);
        }
    }
}

__global__ void __launch_bounds__(256) k_argmax(const GInst *gi, const int32_t *blk2inst, int32_t round)
{
    __shared__ RoundSmem sm;
    step_argmax(gi, blk2inst, blockIdx.x, round, sm);
}

__global__ void __launch_bounds__(256) k_topk_hist(const GInst *gi, const int32_t *blk2inst, int32_t round)
{
    __shared__ RoundSmem sm;
    step_hist(gi, blk2inst, blockIdx.x, round, sm, false);
}

__global__ void __launch_bounds__(256) k_topk_select(const GInst *gi, int32_t round)
{
    __shared__ RoundSmem sm;
    step_select(gi, blockIdx.x, round, sm);
}

__global__ void __launch_bounds__(256) k_update(const GInst *gi, const int32_t *ublk2inst, int32_t round,
                                                int lrr)
{
    step_update(gi, ublk2inst, blockIdx.x, round, lrr);
}

// All rounds of a batch in one cooperative launch.  Every block runs the same steps
// and the same number of grid barriers.  The digit passes of a round are the most any
// instance needs (st->npass, set by the argmax commit before the barrier that
// precedes this read and not written again until after the round's last barrier), so
// every block computes the same count; a step with nothing to do returns at once.
constexpr int RS_PASSES = (64 + RS_BITS - 1) / RS_BITS;

__global__ void __launch_bounds__(256) k_greedy_rounds(const GInst *gi, int nj, const int32_t *blk2inst,
                                                       int nb, const int32_t *ublk2inst, int nub,
                                                       int32_t kmax, int lrr)
{
    __shared__ RoundSmem sm;
    cg::grid_group grid = cg::this_grid();
    for (int32_t round = 0; round <= kmax; ++round) {
        for (int vb = blockIdx.x; vb < nb; vb += gridDim.x) step_argmax(gi, blk2inst, vb, round, sm);
        grid.sync();
        int npass = 0;
        for (int i = 0; i < nj; ++i) npass = max(npass, (int)((volatile GState *)gi[i].st)->npass);
        npass = min(npass, RS_PASSES);
        for (int pass = 0; pass < npass; ++pass) {
            for (int vb = blockIdx.x; vb < nb; vb += gridDim.x) step_hist(gi, blk2inst, vb, round, sm, true);
            grid.sync();
        }
        if (round < kmax) {
            for (int vb = blockIdx.x; vb < nub; vb += gridDim.x) step_update(gi, ublk2inst, vb, round, lrr);
            grid.sync();
        }
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

// update chunks of each inverted-list entry (a record of size s has ceil(s / CHUNK))
__global__ void k_chunks(const long long *inv_rec, const int32_t *rsize, long long cnt, long long *cpre)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= cnt;
         i += (long long)gridDim.x * blockDim.x)
        cpre[i] = i < cnt ? ((long long)rsize[inv_rec[i]] + CHUNK - 1) / CHUNK : 0;
}

// candidates: nodes with a nonzero initial gain, ascending
__global__ void k_flag_nonzero(const unsigned long long *credit, int32_t n, long long *flags)
{
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v <= n;
         v += (long long)gridDim.x * blockDim.x)
        flags[v] = v < n && credit[v] != 0ull ? 1 : 0;
}

__global__ void k_scatter_cand(const unsigned long long *credit, int32_t n, const long long *pos, int32_t *cand)
{
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x)
        if (credit[v] != 0ull) cand[pos[v]] = (int32_t)v;
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

// inverted index node -> records (CP) or sets (LRR), and the per-run greedy state
static void prepare_index(imin_ctx *ctx, GreedyJob &j)
{
    cudaStream_t s = ctx->stream;
    const int32_t n = j.n;
    if (j.c) {
        CpStore &c = *j.c;
        const long long R = c.count;
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
            IM_CHECK_LAUNCH();
            k_init_cp<<<grid_for(ctx, R), 256, 0, s>>>(c.size.as<int32_t>(), R, c.contrib.as<int32_t>(),
                                                      c.covered.as<uint8_t>());
            IM_CHECK_LAUNCH();
        }
        c.inv_cpre.ensure(ctx, (size_t)(R + 1) * 8);
        c.scan_tmp.ensure(ctx, scan_tmp_bytes(std::max<long long>(R + 1, n + 1)));
        k_chunks<<<grid_for(ctx, R + 1), 256, 0, s>>>(c.inv_rec.as<long long>(), c.size.as<int32_t>(), R,
                                                      c.inv_cpre.as<long long>());
        IM_CHECK_LAUNCH();
        exclusive_scan_i64(ctx, c.inv_cpre.as<long long>(), R + 1, c.scan_tmp.p);
    } else {
        LrrStore &L = *j.L;
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
    }
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// blocks of the persistent round kernel: every block must be resident at once (a
// cooperative launch); 0 if the device cannot launch it cooperatively
static int persistent_grid(imin_ctx *ctx)
{
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_greedy_rounds, 256, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (!coop || per_sm < 1) return 0;
    return ctx->num_sms * std::min(per_sm, 4);
}

double greedy_batch(imin_ctx *ctx, GreedyBufs &gb, std::vector<GreedyJob *> &jobs)
{
    cudaStream_t s = ctx->stream;
    const int nj = (int)jobs.size();
    if (nj == 0) return 0.0;
    const char *trenv = std::getenv("IMIN_TRACE");
    const bool trace_idx = trenv && trenv[0] == '1';
    cudaEvent_t i0 = nullptr, i1 = nullptr;
    if (trace_idx) {
        IM_CUDA(cudaEventCreate(&i0));
        IM_CUDA(cudaEventCreate(&i1));
        IM_CUDA(cudaEventRecord(i0, s));
    }
    for (GreedyJob *j : jobs) prepare_index(ctx, *j);
    // candidate lists (nodes with a nonzero initial gain), one readback for all jobs
    size_t cand_total = 0;
    int32_t nmax = 1;
    for (GreedyJob *j : jobs) {
        cand_total += (size_t)j->n;
        nmax = std::max(nmax, j->n);
    }
    gb.cand.ensure(ctx, std::max<size_t>(cand_total, 1) * 4);
    gb.flags.ensure(ctx, (size_t)(nmax + 1) * 8);
    gb.scan_tmp.ensure(ctx, scan_tmp_bytes(nmax + 1));
    gb.ncand.ensure(ctx, (size_t)nj * 8);
    std::vector<size_t> cand_off(nj);
    {
        size_t o = 0;
        for (int i = 0; i < nj; ++i) {
            GreedyJob &j = *jobs[i];
            cand_off[i] = o;
            k_flag_nonzero<<<grid_for(ctx, (long long)j.n + 1), 256, 0, s>>>(j.credit, j.n,
                                                                             gb.flags.as<long long>());
            IM_CHECK_LAUNCH();
            exclusive_scan_i64(ctx, gb.flags.as<long long>(), (int64_t)j.n + 1, gb.scan_tmp.p);
            k_scatter_cand<<<grid_for(ctx, j.n), 256, 0, s>>>(j.credit, j.n, gb.flags.as<long long>(),
                                                             gb.cand.as<int32_t>() + o);
            IM_CHECK_LAUNCH();
            IM_CUDA(cudaMemcpyAsync(gb.ncand.as<long long>() + i, gb.flags.as<long long>() + j.n, 8,
                                    cudaMemcpyDeviceToDevice, s));
            o += (size_t)j.n;
        }
    }
    std::vector<long long> ncand(nj);
    IM_CUDA(cudaMemcpyAsync(ncand.data(), gb.ncand.p, (size_t)nj * 8, cudaMemcpyDeviceToHost, s));
    IM_CUDA(cudaStreamSynchronize(s));
    if (trace_idx) {
        IM_CUDA(cudaEventRecord(i1, s));
        IM_CUDA(cudaEventSynchronize(i1));
        float x = 0.0f;
        IM_CUDA(cudaEventElapsedTime(&x, i0, i1));
        long long items = 0;
        for (GreedyJob *j : jobs) items += j->c ? j->c->count : (long long)j->L->elems;
        std::fprintf(stderr, "[imin] greedy index %s jobs=%d items=%lld %.2fms\n", jobs[0]->c ? "cp" : "lrr",
                     nj, items, x);
        cudaEventDestroy(i0);
        cudaEventDestroy(i1);
    }
    // candidates per argmax / histogram block (tuning hook IMIN_GREEDY_CAND_PER_BLOCK):
    // every block of an instance adds its 2,048-bin histogram to the instance's with
    // global atomics, so fewer, fuller blocks cost less per digit pass
    long long per_blk = 512;
    if (const char *env = std::getenv("IMIN_GREEDY_CAND_PER_BLOCK")) {
        const long long v = std::strtoll(env, nullptr, 10);
        if (v >= 256) per_blk = v;
    }
    // per-instance state in one arena
    std::vector<GInst> gi(nj);
    std::vector<size_t> off(nj);
    std::vector<int32_t> blk2inst, ublk2inst;
    size_t total = 0;
    int32_t kmax = 0;
    for (int i = 0; i < nj; ++i) {
        const GreedyJob &j = *jobs[i];
        const int32_t n = j.n, k = j.k;
        kmax = std::max(kmax, k);
        const int nblk = (int)std::min<long long>((long long)ctx->num_sms * 4,
                                                   std::max<long long>(1, (ncand[i] + per_blk - 1) / per_blk));
        // decrement grid: sized by the stored items (records or set elements)
        const long long items = j.c ? j.c->count : (long long)j.L->elems;
        const int unblk = (int)std::min<long long>((long long)ctx->num_sms * 8,
                                                    std::max<long long>(1, (items + 4095) / 4096));
        GInst &I = gi[i];
        I.n = n;
        I.k = k;
        I.cand = gb.cand.as<int32_t>() + cand_off[i];
        I.ncand = (int32_t)ncand[i];
        I.blk0 = (int32_t)blk2inst.size();
        I.nblk = nblk;
        for (int b = 0; b < nblk; ++b) blk2inst.push_back(i);
        I.ublk0 = (int32_t)ublk2inst.size();
        I.unblk = unblk;
        for (int b = 0; b < unblk; ++b) ublk2inst.push_back(i);
        off[i] = total;
        total += al256((size_t)n * 8) + al256(sizeof(GState)) + al256((size_t)(k + 1) * 4) +
                 2 * al256((size_t)(k + 2) * 8) + al256(RS_BINS * 4) + al256(RS_BINS * 8) +
                 al256((size_t)nblk * 8) + al256((size_t)nblk * 4) + 2 * 256;
    }
    gb.arena.ensure(ctx, total);
    IM_CUDA(cudaMemsetAsync(gb.arena.p, 0, total, s));
    char *base = reinterpret_cast<char *>(gb.arena.p);
    for (int i = 0; i < nj; ++i) {
        const GreedyJob &j = *jobs[i];
        GInst &I = gi[i];
        char *p = base + off[i];
        auto take = [&](size_t bytes) {
            char *q = p;
            p += al256(bytes);
            return q;
        };
        I.gain = reinterpret_cast<unsigned long long *>(take((size_t)j.n * 8));
        I.st = reinterpret_cast<GState *>(take(sizeof(GState)));
        I.B = reinterpret_cast<int32_t *>(take((size_t)(j.k + 1) * 4));
        I.cov = reinterpret_cast<unsigned long long *>(take((size_t)(j.k + 2) * 8));
        I.topk = reinterpret_cast<unsigned long long *>(take((size_t)(j.k + 2) * 8));
        I.hcnt = reinterpret_cast<unsigned int *>(take(RS_BINS * 4));
        I.hsum = reinterpret_cast<unsigned long long *>(take(RS_BINS * 8));
        I.part_g = reinterpret_cast<unsigned long long *>(take((size_t)I.nblk * 8));
        I.part_v = reinterpret_cast<int32_t *>(take((size_t)I.nblk * 4));
        I.done_ctr = reinterpret_cast<unsigned int *>(take(4));
        I.done_ctr2 = reinterpret_cast<unsigned int *>(take(4));
        IM_CUDA(cudaMemcpyAsync(I.gain, j.credit, (size_t)j.n * 8, cudaMemcpyDeviceToDevice, s));
        I.inv_rec = nullptr;
        I.inv_cpre = nullptr;
        I.rnode = I.rpar = I.rsize = nullptr;
        I.contrib = nullptr;
        I.covered = nullptr;
        I.inv_set = nullptr;
        I.set_off = nullptr;
        I.set_len = nullptr;
        I.set_elem = nullptr;
        if (j.c) {
            I.inv_off = j.c->inv_off.as<long long>();
            I.inv_rec = j.c->inv_rec.as<long long>();
            I.inv_cpre = j.c->inv_cpre.as<long long>();
            I.rnode = j.c->node.as<int32_t>();
            I.rpar = j.c->par.as<int32_t>();
            I.rsize = j.c->size.as<int32_t>();
            I.contrib = j.c->contrib.as<int32_t>();
            I.covered = j.c->covered.as<uint8_t>();
        } else {
            I.inv_off = j.L->inv_off.as<long long>();
            I.inv_set = j.L->inv_set.as<uint32_t>();
            I.set_off = j.L->off.as<unsigned long long>();
            I.set_len = j.L->len.as<uint32_t>();
            I.set_elem = j.L->elem.as<int32_t>();
            I.covered = j.L->covered.as<uint8_t>();
        }
    }
    gb.ginst.ensure(ctx, (size_t)nj * sizeof(GInst));
    gb.blkmap.ensure(ctx, (blk2inst.size() + ublk2inst.size()) * 4);
    IM_CUDA(cudaMemcpyAsync(gb.ginst.p, gi.data(), (size_t)nj * sizeof(GInst), cudaMemcpyHostToDevice, s));
    IM_CUDA(cudaMemcpyAsync(gb.blkmap.p, blk2inst.data(), blk2inst.size() * 4, cudaMemcpyHostToDevice, s));
    IM_CUDA(cudaMemcpyAsync(gb.blkmap.as<int32_t>() + blk2inst.size(), ublk2inst.data(),
                            ublk2inst.size() * 4, cudaMemcpyHostToDevice, s));
    const GInst *dgi = gb.ginst.as<GInst>();
    const int32_t *dblk = gb.blkmap.as<int32_t>();
    const int32_t *dublk = dblk + blk2inst.size();
    const int nb = (int)blk2inst.size(), nub = (int)ublk2inst.size();
    // every job is either CP or LRR; both kinds may not share a batch
    const int lrr = jobs[0]->L ? 1 : 0;
    cudaEvent_t e0, e1;
    IM_CUDA(cudaEventCreate(&e0));
    IM_CUDA(cudaEventCreate(&e1));
    IM_CUDA(cudaEventRecord(e0, s));
    // all rounds in one cooperative persistent launch (IMIN_GREEDY_PERSISTENT=0: one
    // launch per round step)
    const int coop = std::min(persistent_grid(ctx), std::max(nb, nub));
    const char *env = std::getenv("IMIN_GREEDY_PERSISTENT");
    if (coop > 0 && !(env && env[0] == '0')) {
        int nj_ = nj, nb_ = nb, nub_ = nub, lrr_ = lrr;
        int32_t kmax_ = kmax;
        void *args[] = {(void *)&dgi, (void *)&nj_, (void *)&dblk, (void *)&nb_, (void *)&dublk,
                        (void *)&nub_, (void *)&kmax_, (void *)&lrr_};
        IM_CUDA(cudaLaunchCooperativeKernel((const void *)k_greedy_rounds, dim3(coop), dim3(256), args, 0, s));
        IM_CHECK_LAUNCH();
    } else {
        // IMIN_TRACE=1: time the three kinds of step apart (events between them)
        const char *tr = std::getenv("IMIN_TRACE");
        const bool trace = tr && tr[0] == '1';
        cudaEvent_t ev[4];
        double tms[3] = {0, 0, 0};
        if (trace)
            for (cudaEvent_t &e : ev) IM_CUDA(cudaEventCreate(&e));
        auto lap = [&](int a, int b, int slot) {
            if (!trace) return;
            float x = 0.0f;
            IM_CUDA(cudaEventSynchronize(ev[b]));
            IM_CUDA(cudaEventElapsedTime(&x, ev[a], ev[b]));
            tms[slot] += x;
        };
        for (int32_t round = 0; round <= kmax; ++round) {
            if (trace) IM_CUDA(cudaEventRecord(ev[0], s));
            k_argmax<<<nb, 256, 0, s>>>(dgi, dblk, round);
            IM_CHECK_LAUNCH();
            if (trace) IM_CUDA(cudaEventRecord(ev[1], s));
            for (int pass = 0; pass < RS_PASSES; ++pass) {
                k_topk_hist<<<nb, 256, 0, s>>>(dgi, dblk, round);
                IM_CHECK_LAUNCH();
                k_topk_select<<<nj, 256, 0, s>>>(dgi, round);
                IM_CHECK_LAUNCH();
            }
            if (trace) IM_CUDA(cudaEventRecord(ev[2], s));
            if (round < kmax) {
                k_update<<<nub, 256, 0, s>>>(dgi, dublk, round, lrr);
                IM_CHECK_LAUNCH();
            }
            if (trace) {
                IM_CUDA(cudaEventRecord(ev[3], s));
                lap(0, 1, 0);
                lap(1, 2, 1);
                lap(2, 3, 2);
            }
        }
        if (trace) {
            std::fprintf(stderr, "[imin] greedy %s jobs=%d kmax=%d argmax=%.2fms topk=%.2fms update=%.2fms\n",
                         lrr ? "lrr" : "cp", nj, kmax, tms[0], tms[1], tms[2]);
            for (cudaEvent_t &e : ev) cudaEventDestroy(e);
        }
    }
    IM_CUDA(cudaEventRecord(e1, s));
    IM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    IM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // read back B, Cov(B_i), top-k sums
    for (int i = 0; i < nj; ++i) {
        GreedyJob &j = *jobs[i];
        const GInst &I = gi[i];
        GState st;
        IM_CUDA(cudaMemcpy(&st, I.st, sizeof(GState), cudaMemcpyDeviceToHost));
        GreedyOut &o = j.out;
        const int nbk = st.nb;
        o.B.resize(nbk);
        o.cov.resize(nbk + 1);
        o.topk.resize(nbk + 1);
        if (nbk > 0) IM_CUDA(cudaMemcpy(o.B.data(), I.B, (size_t)nbk * 4, cudaMemcpyDeviceToHost));
        IM_CUDA(cudaMemcpy(o.cov.data(), I.cov, (size_t)(nbk + 1) * 8, cudaMemcpyDeviceToHost));
        IM_CUDA(cudaMemcpy(o.topk.data(), I.topk, (size_t)(nbk + 1) * 8, cudaMemcpyDeviceToHost));
        o.covu = o.cov[0] + o.topk[0];
        for (int t = 1; t <= nbk; ++t) o.covu = std::min(o.covu, o.cov[t] + o.topk[t]);
    }
    return ms;
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
