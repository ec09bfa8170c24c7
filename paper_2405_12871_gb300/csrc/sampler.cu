// sampler.cu -- the warp-per-world kernel: one warp traverses one live-edge world at a
// time.  The CTA-per-world kernels (reach_cta.cuh) compute the same counts and are the
// default; this kernel remains an autotuner candidate (small worlds), serves worlds that
// carry both bounds at once, and runs the large-slot pass for worlds that overflow.
//
// Per world j (Sec. 2.1, Algorithms 2 and 3):
//   1. masked reach BFS from the seed set (the unified seed s of Sec. 3.1 is the
//      multi-source start); blocked nodes are never entered;
//   2. (lower bound) immediate dominators of the live subgraph on R_j with root s,
//      DT subtree sizes = |N_phi(v)| credits, and optionally the CP records
//      (node, parent distance, subtree size) in DT preorder;
//   3. (upper bound) the Global Sampling target t_j and its LRR set inside
//      phi^s = live edges between nodes of R_j \ S, by reverse BFS.
//
// Warp-cooperative frontier expansion: the 32 lanes take 32 frontier nodes, an
// inclusive warp scan over their counts of 4-edge groups flattens the work, and
// every lane then processes one group per step: one 16-byte load of col, one of
// the coin thresholds, one Philox call (its 4 words are the 4 coins of the group:
// counter word 0 is e >> 2).  New nodes are appended with ballot/popc compaction;
// no atomics are needed for the queue because the warp owns the world.
//
// Dominators: initialise idom(v) to v's BFS parent and relax idom(v) <- LCA(idom(v),
// p) over every live in-edge (p, v) until nothing changes.  Every estimate is an
// ancestor of v in the BFS tree, so a dominator chain always descends in BFS level
// and LCA walks by level; the relaxation only moves estimates up, never past the
// true immediate dominator (dominators of v are ancestors of v in every spanning
// tree rooted at s), so the fixed point is the dominator tree -- which is unique,
// so the result equals Lengauer-Tarjan's.
#include "common.cuh"

#include <algorithm>
#include <cstdlib>

namespace {

struct KArgs {
    const WTask *tasks;        // device array of task descriptors
    int ntasks;
    uint32_t *task_claim;      // per task: next world to claim
    uint32_t *task_done;       // per task: 1 once exhausted (or stopped)
    char *slot_base;
    size_t slot_bytes;
    size_t bm_words;
    int32_t qcap, ecap;
    size_t off_queue, off_loc, off_lvl, off_par, off_idom, off_size, off_pre, off_cur, off_lstart,
        off_pu, off_pv, off_bm2, off_q2;
    uint32_t flags;
};

__device__ __forceinline__ int warp_incl_scan(int x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(IMIN_FULL, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ __forceinline__ bool bit_test(const uint32_t *bm, int v)
{
    return (bm[v >> 5] >> (v & 31)) & 1u;
}

__device__ __forceinline__ bool bit_test_cg(const uint32_t *bm, int v)
{
    return (__ldcg(bm + (v >> 5)) >> (v & 31)) & 1u;
}

// index of the lane whose [incl - cnt, incl) range holds t (incl non-decreasing)
__device__ __forceinline__ int owner_lane(int incl, int t)
{
    int lo = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const int v = __shfl_sync(IMIN_FULL, incl, lo + s - 1);
        if (v <= t) lo += s;
    }
    return lo;
}

// LCA of local nodes a and b in the current dominator-estimate tree (-1 = root s).
__device__ __forceinline__ int tree_lca(int a, int b, const int32_t *lvl, int32_t *idom, int nS)
{
    while (a != b) {
        const int la = a < 0 ? -1 : lvl[a];
        const int lb = b < 0 ? -1 : lvl[b];
        if (la >= lb)
            a = (a < nS) ? -1 : __ldcg(idom + a);
        else
            b = (b < nS) ? -1 : __ldcg(idom + b);
    }
    return a;
}

// bump allocation that never overshoots `cap`; returns ~0ull on failure
__device__ unsigned long long reserve(unsigned long long *cursor, unsigned long long cnt,
                                      unsigned long long cap)
{
    unsigned long long old = *(volatile unsigned long long *)cursor;
    for (int tries = 0; tries < (1 << 20); ++tries) {
        if (old + cnt > cap) return ~0ull;
        const unsigned long long prev = atomicCAS(cursor, old, old + cnt);
        if (prev == old) return old;
        old = prev;
    }
    return ~0ull;
}

// reach-only and upper-bound worlds run 32 warps per SM (<= 64 registers); the lower bound
// keeps more state per world and runs fewer, larger warps
template <int U, bool LOWER, bool UPPER, bool STOP>
__global__ void __launch_bounds__(256, LOWER ? 1 : 4) world_kernel(const KArgs a)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const size_t wid = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    char *slot = a.slot_base + wid * a.slot_bytes;
    uint32_t *bm = reinterpret_cast<uint32_t *>(slot);
    int32_t *Q = reinterpret_cast<int32_t *>(slot + a.off_queue);
    int32_t *loc = nullptr, *lvl = nullptr, *par = nullptr, *idom = nullptr, *sz = nullptr,
            *pre = nullptr, *cur = nullptr, *lstart = nullptr, *pu = nullptr, *pv = nullptr;
    if (LOWER) {
        loc = reinterpret_cast<int32_t *>(slot + a.off_loc);
        lvl = reinterpret_cast<int32_t *>(slot + a.off_lvl);
        par = reinterpret_cast<int32_t *>(slot + a.off_par);
        idom = reinterpret_cast<int32_t *>(slot + a.off_idom);
        sz = reinterpret_cast<int32_t *>(slot + a.off_size);
        pre = reinterpret_cast<int32_t *>(slot + a.off_pre);
        cur = reinterpret_cast<int32_t *>(slot + a.off_cur);
        lstart = reinterpret_cast<int32_t *>(slot + a.off_lstart);
        pu = reinterpret_cast<int32_t *>(slot + a.off_pu);
        pv = reinterpret_cast<int32_t *>(slot + a.off_pv);
    }
    uint32_t *bm2 = nullptr;
    int32_t *Q2 = nullptr;
    if (UPPER) {
        bm2 = reinterpret_cast<uint32_t *>(slot + a.off_bm2);
        Q2 = reinterpret_cast<int32_t *>(slot + a.off_q2);
    }
    const int qcap = a.qcap;
    const bool store = (a.flags & WF_STORE) != 0;
    int ti = (int)(wid % (size_t)a.ntasks);

    for (;;) {
        // lane 0 claims the next world of an unfinished task, starting with the task the
        // warp worked on last; a task is finished when its range is used up or (stopping
        // rule) its running spread has reached its threshold
        int got = -1;
        uint32_t rel = 0xffffffffu;
        if (lane == 0) {
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
        }
        got = __shfl_sync(IMIN_FULL, got, 0);
        rel = __shfl_sync(IMIN_FULL, rel, 0);
        if (got < 0) break;
        ti = got;
        const WTask &T = a.tasks[ti];
        // the fields the traversal touches, read once per world
        const int32_t *const row_ptr = T.row_ptr;
        const uint4 *const ce = T.ce;
        const uint32_t *const seed_bm = T.q.seed_bm;
        const uint32_t *const blocked_bm = T.q.blocked_bm;
        const int nS = T.q.nS;
        const uint32_t klo = (uint32_t)T.q.key, khi = (uint32_t)(T.q.key >> 32);
        const uint32_t tag = T.q.tag, inst = T.q.inst;
        // wrel: index of the world relative to `first` (outputs are indexed by it)
        const uint32_t wrel = T.list ? (T.list[rel] & 0x7fffffffu) : rel;
        const uint32_t j = (uint32_t)(T.first + (uint64_t)wrel);

        // ---- 1. masked reach BFS -------------------------------------------------
        if (!LOWER && !UPPER)
            for (int i = lane; i < T.q.nB; i += 32) {
                const int v = T.q.B[i];
                atomicOr(&bm[v >> 5], 1u << (v & 31));
            }
        for (int i = lane; i < nS; i += 32) {
            const int s = T.q.S[i];
            atomicOr(&bm[s >> 5], 1u << (s & 31));
            Q[i] = s;
            if (LOWER) {
                loc[s] = i;
                lvl[i] = 0;
                par[i] = -1;
            }
        }
        int tail = nS, head = 0, L = 0, npairs = 0;
        bool ovf = false;
        unsigned long long wedges = 0;
        if (LOWER && lane == 0) lstart[0] = 0;
        __syncwarp();
        while (head < tail) {
            const int fend = tail;
            for (int base = head; base < fend; base += 32) {
                const int i = base + lane;
                int b = 0, e = 0, cnt = 0;
                if (i < fend) {
                    const int u = Q[i];
                    b = row_ptr[u];
                    e = row_ptr[u + 1];
                    if (e > b) cnt = ((e + 3) >> 2) - (b >> 2);
                    wedges += (unsigned long long)(e - b);
                }
                const int incl = warp_incl_scan(cnt, lane);
                const int total = __shfl_sync(IMIN_FULL, incl, 31);
                // U groups per lane per step: every lane issues the loads of all its
                // groups before any coin or atomic, so U loads are in flight per lane.
                for (int t0 = 0; t0 < total; t0 += 32 * U) {
                    int gq[U], obq[U], oeq[U], oiq[U];
                    bool act[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int t = t0 + u * 32 + lane;
                        const int lo = owner_lane(incl, t);
                        obq[u] = __shfl_sync(IMIN_FULL, b, lo);
                        oeq[u] = __shfl_sync(IMIN_FULL, e, lo);
                        const int ostart = __shfl_sync(IMIN_FULL, incl - cnt, lo);
                        oiq[u] = base + lo;
                        act[u] = t < total;
                        gq[u] = (obq[u] >> 2) + (t - ostart);
                    }
                    int4 c4[U];
                    uint4 t4[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (act[u]) {
                            const int4 *p = reinterpret_cast<const int4 *>(ce + 2 * (size_t)gq[u]);
                            c4[u] = __ldg(p);
                            t4[u] = __ldg(reinterpret_cast<const uint4 *>(p + 1));
                        } else {
                            c4[u] = make_int4(0, 0, 0, 0);
                            t4[u] = make_uint4(0, 0, 0, 0);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        int nv[4] = {-1, -1, -1, -1};
                        int pvv[4] = {-1, -1, -1, -1};
                        if (act[u]) {
                            const int g = gq[u];
                            const uint4 w = philox10(make_uint4((uint32_t)g, j, tag, inst), klo, khi);
                            const int cv[4] = {c4[u].x, c4[u].y, c4[u].z, c4[u].w};
                            const uint32_t tv[4] = {t4[u].x, t4[u].y, t4[u].z, t4[u].w};
                            const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
                            bool ok[4];
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const int ec = (g << 2) + c;
                                ok[c] = ec >= obq[u] && ec < oeq[u] && (wv[c] >> 8) < tv[c];
                                // reach-only worlds pre-mark blocked nodes as visited
                                if ((LOWER || UPPER) && ok[c] && blocked_bm)
                                    ok[c] = !bit_test(blocked_bm, cv[c]);
                                if (LOWER && ok[c] && !bit_test(seed_bm, cv[c])) pvv[c] = cv[c];
                            }
                            // the (rare) claims are independent: issue them back to back
                            uint32_t old[4];
#pragma unroll
                            for (int c = 0; c < 4; ++c)
                                old[c] = ok[c] ? atomicOr(&bm[cv[c] >> 5], 1u << (cv[c] & 31))
                                               : 0xffffffffu;
#pragma unroll
                            for (int c = 0; c < 4; ++c)
                                if (!((old[c] >> (cv[c] & 31)) & 1u)) nv[c] = cv[c];
                        }
                        const int oi = oiq[u];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const uint32_t bal = __ballot_sync(IMIN_FULL, nv[c] >= 0);
                            if (bal) {
                                const int pos = tail + __popc(bal & lt_mask);
                                if (nv[c] >= 0 && pos < qcap) {
                                    Q[pos] = nv[c];
                                    if (LOWER) {
                                        loc[nv[c]] = pos;
                                        lvl[pos] = L + 1;
                                        par[pos] = oi;
                                    }
                                }
                                tail += __popc(bal);
                            }
                            if (LOWER) {
                                const uint32_t pb = __ballot_sync(IMIN_FULL, pvv[c] >= 0);
                                if (pb) {
                                    const int pp = npairs + __popc(pb & lt_mask);
                                    if (pvv[c] >= 0 && pp < a.ecap) {
                                        pu[pp] = oi;
                                        pv[pp] = pvv[c];
                                    }
                                    npairs += __popc(pb);
                                }
                            }
                        }
                    }
                }
            }
            if (tail > qcap || (LOWER && npairs > a.ecap)) {
                ovf = true;
                break;
            }
            head = fend;
            ++L;
            if (LOWER && lane == 0) lstart[L] = fend;
            __syncwarp();
        }

        // ---- 2. dominator tree, subtree sizes -----------------------------------
        if (LOWER && !ovf) {
            __syncwarp();
            for (int k = lane; k < npairs; k += 32) pv[k] = loc[pv[k]];
            for (int i = lane; i < tail; i += 32) {
                idom[i] = (i < nS) ? -1 : par[i];
                sz[i] = (i < nS) ? 0 : 1;
                cur[i] = 0;
            }
            __syncwarp();
            for (int pass = 0;; ++pass) {
                bool changed = false;
                for (int k = lane; k < npairs; k += 32) {
                    const int i = pv[k];
                    if (i < nS) continue;
                    const int p = pu[k];
                    int c0 = __ldcg(idom + i);
                    for (int guard = 0; guard < (1 << 22); ++guard) {
                        const int c = tree_lca(c0, p, lvl, idom, nS);
                        if (c == c0) break;
                        const int old = atomicCAS(idom + i, c0, c);
                        if (old == c0) {
                            changed = true;
                            break;
                        }
                        c0 = old;
                    }
                }
                __syncwarp();
                if (!__any_sync(IMIN_FULL, changed)) break;
                if (pass > (1 << 20)) {
                    if (lane == 0) atomicOr(T.out.err, DERR_TIMEOUT);
                    break;
                }
            }
            __syncwarp();
            for (int lv = L - 1; lv >= 1; --lv) {
                const int s0 = lstart[lv], s1 = lstart[lv + 1];
                for (int i = s0 + lane; i < s1; i += 32) {
                    const int d = __ldcg(idom + i);
                    if (d >= nS) atomicAdd(sz + d, __ldcg(sz + i));
                }
                __syncwarp();
            }
        }

        // ---- 3. Global Sampling target and LRR set --------------------------------
        int tail2 = 0;
        if (UPPER && !ovf && T.q.nVs > 0) {
            int tnode = -1;
            if (lane == 0) {
                const uint4 w = philox10(make_uint4(0xFFFFFFFFu, j, tag, inst), klo, khi);
                const unsigned long long r64 = ((unsigned long long)w.y << 32) | w.x;
                const unsigned long long idx = __umul64hi(r64, (unsigned long long)T.q.nVs);
                const int t = T.q.Vs[idx];
                if (bit_test_cg(bm, t)) tnode = t;
            }
            tnode = __shfl_sync(IMIN_FULL, tnode, 0);
            if (tnode >= 0) {
                if (lane == 0) {
                    atomicOr(&bm2[tnode >> 5], 1u << (tnode & 31));
                    Q2[0] = tnode;
                }
                tail2 = 1;
                int head2 = 0;
                __syncwarp();
                while (head2 < tail2) {
                    const int fend = tail2;
                    for (int base = head2; base < fend; base += 32) {
                        const int i = base + lane;
                        int b = 0, cnt = 0;
                        if (i < fend) {
                            const int v = Q2[i];
                            b = T.in_ptr[v];
                            cnt = T.in_ptr[v + 1] - b;
                        }
                        const int incl = warp_incl_scan(cnt, lane);
                        const int total = __shfl_sync(IMIN_FULL, incl, 31);
                        for (int t0 = 0; t0 < total; t0 += 32) {
                            const int t = t0 + lane;
                            const int lo = owner_lane(incl, t);
                            const int ob = __shfl_sync(IMIN_FULL, b, lo);
                            const int ostart = __shfl_sync(IMIN_FULL, incl - cnt, lo);
                            int nu = -1;
                            if (t < total) {
                                const int idx = ob + (t - ostart);
                                const int u = __ldg(T.in_src + idx);
                                if (bit_test_cg(bm, u) && !bit_test(seed_bm, u)) {
                                    const int eid = __ldg(T.in_eid + idx);
                                    const uint32_t th = __ldg(T.in_thr + idx);
                                    const uint4 w = philox10(
                                        make_uint4((uint32_t)eid >> 2, j, tag, inst), klo, khi);
                                    if ((pick_word(w, eid & 3) >> 8) < th) {
                                        const uint32_t bit = 1u << (u & 31);
                                        const uint32_t old = atomicOr(&bm2[u >> 5], bit);
                                        if (!(old & bit)) nu = u;
                                    }
                                }
                            }
                            const uint32_t bal = __ballot_sync(IMIN_FULL, nu >= 0);
                            if (bal) {
                                const int pos = tail2 + __popc(bal & lt_mask);
                                if (nu >= 0 && pos < qcap) Q2[pos] = nu;
                                tail2 += __popc(bal);
                            }
                        }
                    }
                    if (tail2 > qcap) {
                        ovf = true;
                        break;
                    }
                    head2 = fend;
                    __syncwarp();
                }
            }
        }

        // ---- 4. reserve store space -----------------------------------------------
        const bool slot_ovf = ovf;
        unsigned long long sbase = 0;
        if (!ovf && store && (LOWER || UPPER)) {
            if (lane == 0) {
                if (LOWER)
                    sbase = reserve(T.out.rec_cursor, (unsigned long long)(tail - nS), T.out.rec_cap);
                else
                    sbase = tail2 > 0 ? reserve(T.out.set_cursor, (unsigned long long)tail2,
                                                T.out.set_cap)
                                      : 0ull;
            }
            sbase = __shfl_sync(IMIN_FULL, sbase, 0);
            if (sbase == ~0ull) ovf = true;
        }

        if (ovf) {
            // defer the world: clear every visited mark, contribute nothing
            __syncwarp();
            for (size_t w = lane; w < a.bm_words; w += 32) bm[w] = 0;
            if (UPPER)
                for (size_t w = lane; w < a.bm_words; w += 32) bm2[w] = 0;
            if (lane == 0) {
                const uint32_t d = atomicAdd(T.out.n_deferred, 1u);
                // the top bit marks worlds that need a large slot (not just store room)
                if (d < T.out.deferred_cap)
                    T.out.deferred[d] = wrel | (slot_ovf ? 0x80000000u : 0u);
                else
                    atomicOr(T.out.err, DERR_INTERNAL);
            }
            __syncwarp();
            continue;
        }

        // ---- 5. outputs ---------------------------------------------------------------
        if (LOWER) {
            if (T.out.credit_L)
                for (int i = nS + lane; i < tail; i += 32)
                    atomicAdd(T.out.credit_L + Q[i], (unsigned long long)__ldcg(sz + i));
            if (store) {
                // DT preorder, level by level: roots (idom = s or a seed) get consecutive
                // ranges; a child starts after its parent and the earlier siblings' subtrees.
                int rootbase = 0;
                for (int lv = 1; lv < L; ++lv) {
                    const int s0 = lstart[lv], s1 = lstart[lv + 1];
                    for (int ib = s0; ib < s1; ib += 32) {
                        const int i = ib + lane;
                        const bool valid = i < s1;
                        const int d = valid ? __ldcg(idom + i) : 0;
                        const int size_i = valid ? __ldcg(sz + i) : 0;
                        const bool isroot = valid && d < nS;
                        const int rs = isroot ? size_i : 0;
                        const int rincl = warp_incl_scan(rs, lane);
                        const int rtot = __shfl_sync(IMIN_FULL, rincl, 31);
                        if (valid) {
                            int pr, poff;
                            if (isroot) {
                                pr = rootbase + rincl - rs;
                                poff = 0;
                            } else {
                                const int pd = pre[d];
                                pr = pd + 1 + atomicAdd(cur + d, size_i);
                                poff = pr - pd;
                            }
                            pre[i] = pr;
                            const unsigned long long r = sbase + (unsigned long long)pr;
                            T.out.rec_node[r] = Q[i];
                            T.out.rec_par[r] = poff;
                            T.out.rec_size[r] = size_i;
                        }
                        rootbase += rtot;
                    }
                    __syncwarp();
                }
            }
        }
        if (UPPER) {
            if (T.out.credit_U)
                for (int i = lane; i < tail2; i += 32) atomicAdd(T.out.credit_U + Q2[i], 1ull);
            if (store) {
                for (int i = lane; i < tail2; i += 32) T.out.set_elem[sbase + i] = Q2[i];
                if (lane == 0) {
                    T.out.set_off[wrel] = sbase;
                    T.out.set_len[wrel] = (uint32_t)tail2;
                }
            }
            for (int i = lane; i < tail2; i += 32) bm2[Q2[i] >> 5] = 0;
        }
        if (a.flags & WF_REACH)
            for (int i = lane; i < tail; i += 32) atomicAdd(T.out.reach + Q[i], 1ull);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wedges += __shfl_xor_sync(IMIN_FULL, wedges, o);
        if (lane == 0) {
            atomicAdd(T.out.acc + 0, (unsigned long long)tail);
            atomicAdd(T.out.acc + 1, wedges);
            if (UPPER && tail2 > 0) atomicAdd(T.out.acc + 2, 1ull);
            if (STOP) atomicAdd(T.out.acc + 3, (unsigned long long)tail);
            atomicAdd(T.out.acc + 4, 1ull);
            if (T.out.world_spread) T.out.world_spread[wrel] = (uint32_t)tail;
        }
        __syncwarp();
        for (int i = lane; i < tail; i += 32) bm[Q[i] >> 5] = 0;
        if (!LOWER && !UPPER)
            for (int i = lane; i < T.q.nB; i += 32) bm[T.q.B[i] >> 5] = 0;
        __syncwarp();
    }
}

inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

}  // namespace

size_t SlotCfg::bytes_per_slot() const
{
    if (ctas > 0) return cta_slot_bytes(*this);
    size_t b = al16(bm_words * 4) + al16((size_t)qcap * 4);
    if (lower) {
        // loc is indexed by node id: n entries = 32 * bm_words upper bound
        b += al16(bm_words * 32 * 4) + 6 * al16((size_t)qcap * 4) + al16(((size_t)qcap + 2) * 4) +
             2 * al16((size_t)ecap * 4);
    }
    if (upper) b += al16(bm_words * 4) + al16((size_t)qcap * 4);
    return b;
}

// resident 256-thread blocks per SM of the instantiation a launch would use
int world_kernel_blocks_per_sm(uint32_t flags, int U)
{
    const bool lower = (flags & WF_LOWER) != 0, upper = (flags & WF_UPPER) != 0,
               stop = (flags & WF_STOP) != 0;
    int nb = 0;
    cudaError_t e = cudaSuccess;
#define IM_OCC(UU)                                                                               \
    do {                                                                                         \
        if (lower && upper)                                                                      \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, world_kernel<UU, true, true, false>, 256, 0);   \
        else if (lower)                                                                          \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, world_kernel<UU, true, false, false>, 256, 0);  \
        else if (upper)                                                                          \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, world_kernel<UU, false, true, false>, 256, 0);  \
        else if (stop)                                                                           \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, world_kernel<UU, false, false, true>, 256, 0);  \
        else                                                                                     \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, world_kernel<UU, false, false, false>, 256, 0); \
    } while (0)
    if (U >= 4)
        IM_OCC(4);
    else if (U == 2)
        IM_OCC(2);
    else
        IM_OCC(1);
#undef IM_OCC
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb < 1 ? 1 : nb;
}

WTask make_task(const imin_graph *g, const QueryDev &q, uint64_t first, uint32_t count,
                const uint32_t *list, const WorldOut &out)
{
    WTask t;
    t.row_ptr = g->row_ptr.as<int32_t>();
    t.ce = g->ce.as<uint4>();
    t.in_ptr = g->in_ptr.as<int32_t>();
    t.in_src = g->in_src.as<int32_t>();
    t.in_eid = g->in_eid.as<int32_t>();
    t.in_thr = g->in_thr.as<uint32_t>();
    t.n = g->n;
    t.q = q;
    t.first = first;
    t.count = count;
    t.list = list;
    t.out = out;
    return t;
}

void launch_tasks(imin_ctx *ctx, const WTask *d_tasks, int ntasks, const imin_graph *g,
                  uint32_t flags, const SlotCfg &cfg, void *slot_base, uint32_t *d_claim,
                  uint32_t *d_done)
{
    if (ntasks <= 0) return;
    if (cfg.ctas > 0) {
        launch_cta_tasks(ctx, d_tasks, ntasks, flags, cfg, slot_base, d_claim, d_done);
        return;
    }
    KArgs a;
    a.tasks = d_tasks;
    a.ntasks = ntasks;
    a.task_claim = d_claim;
    a.task_done = d_done;
    a.slot_base = reinterpret_cast<char *>(slot_base);
    a.slot_bytes = cfg.bytes_per_slot();
    a.bm_words = cfg.bm_words;
    a.qcap = cfg.qcap;
    a.ecap = cfg.ecap;
    size_t off = al16(cfg.bm_words * 4);
    a.off_queue = off;
    off += al16((size_t)cfg.qcap * 4);
    a.off_loc = a.off_lvl = a.off_par = a.off_idom = a.off_size = a.off_pre = a.off_cur =
        a.off_lstart = a.off_pu = a.off_pv = a.off_bm2 = a.off_q2 = 0;
    if (cfg.lower) {
        a.off_loc = off;    off += al16(cfg.bm_words * 32 * 4);
        a.off_lvl = off;    off += al16((size_t)cfg.qcap * 4);
        a.off_par = off;    off += al16((size_t)cfg.qcap * 4);
        a.off_idom = off;   off += al16((size_t)cfg.qcap * 4);
        a.off_size = off;   off += al16((size_t)cfg.qcap * 4);
        a.off_pre = off;    off += al16((size_t)cfg.qcap * 4);
        a.off_cur = off;    off += al16((size_t)cfg.qcap * 4);
        a.off_lstart = off; off += al16(((size_t)cfg.qcap + 2) * 4);
        a.off_pu = off;     off += al16((size_t)cfg.ecap * 4);
        a.off_pv = off;     off += al16((size_t)cfg.ecap * 4);
    }
    if (cfg.upper) {
        a.off_bm2 = off;    off += al16(cfg.bm_words * 4);
        a.off_q2 = off;     off += al16((size_t)cfg.qcap * 4);
    }
    a.flags = flags;

    const int threads = 256;
    const int blocks = cfg.warps / (threads / 32);
    const bool lower = (flags & WF_LOWER) != 0, upper = (flags & WF_UPPER) != 0,
               stop = (flags & WF_STOP) != 0;
    const int U = cfg.groups_per_lane;
    // keep the interleaved edge array resident in L2 while worlds are traversed
    cudaLaunchAttribute attr[1];
    int nattr = 0;
    // tuning hook: IMIN_L2_PERSIST=<hit ratio in percent> enables the window (off by default:
    // on the 1M-node Chung-Lu workload the carve-out left too little L2 for the bitmaps)
    double hit_pct = 0.0;
    if (const char *env = std::getenv("IMIN_L2_PERSIST")) hit_pct = std::strtod(env, nullptr);
    if (hit_pct > 0.0 && ctx->l2_window_bytes > 0 && g && g->ce.p) {
        attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[0].val.accessPolicyWindow.base_ptr = g->ce.p;
        attr[0].val.accessPolicyWindow.num_bytes = std::min(ctx->l2_window_bytes, g->ce_bytes);
        attr[0].val.accessPolicyWindow.hitRatio =
            (float)std::min(hit_pct / 100.0, (double)ctx->l2_persist_bytes /
                                                 (double)attr[0].val.accessPolicyWindow.num_bytes);
        attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        nattr = 1;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(blocks);
    lc.blockDim = dim3(threads);
    lc.dynamicSmemBytes = 0;
    lc.stream = ctx->stream;
    lc.attrs = nattr ? attr : nullptr;
    lc.numAttrs = nattr;
#define IM_WKX(UU, L_, U_, S_) IM_CUDA(cudaLaunchKernelEx(&lc, world_kernel<UU, L_, U_, S_>, a))
#undef IM_WK
#define IM_WK(UU)                                        \
    do {                                                 \
        if (lower && upper)                              \
            IM_WKX(UU, true, true, false);               \
        else if (lower)                                  \
            IM_WKX(UU, true, false, false);              \
        else if (upper)                                  \
            IM_WKX(UU, false, true, false);              \
        else if (stop)                                   \
            IM_WKX(UU, false, false, true);              \
        else                                             \
            IM_WKX(UU, false, false, false);             \
    } while (0)
    if (U >= 4)
        IM_WK(4);
    else if (U == 2)
        IM_WK(2);
    else
        IM_WK(1);
#undef IM_WKX
#undef IM_WK
    IM_CHECK_LAUNCH();
}
