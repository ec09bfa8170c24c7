// sampler.cu -- the world kernel: one warp traverses one live-edge world at a time.
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

namespace {

struct KArgs {
    const int32_t *row_ptr;
    const int4 *col4;
    const uint4 *thr4;
    const int32_t *in_ptr, *in_src, *in_eid;
    const uint32_t *in_thr;
    int32_t n;
    QueryDev q;
    uint64_t first;
    uint32_t count;
    const uint32_t *list;
    uint32_t *claim;
    char *slot_base;
    size_t slot_bytes;
    size_t bm_words;
    int32_t qcap, ecap;
    size_t off_queue, off_loc, off_lvl, off_par, off_idom, off_size, off_pre, off_cur, off_lstart,
        off_pu, off_pv, off_bm2, off_q2;
    uint32_t flags;
    WorldOut out;
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

template <bool LOWER, bool UPPER, bool STOP>
__global__ void __launch_bounds__(256) world_kernel(const KArgs a)
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
    const int nS = a.q.nS;
    const int qcap = a.qcap;
    const uint32_t klo = (uint32_t)a.q.key, khi = (uint32_t)(a.q.key >> 32);
    const uint32_t tag = a.q.tag, inst = a.q.inst;
    const bool store = (a.flags & WF_STORE) != 0;

    for (;;) {
        uint32_t rel = 0xffffffffu;
        if (lane == 0) {
            bool stop = false;
            if (STOP) stop = *(volatile unsigned long long *)(a.out.acc + 3) >= a.out.stop_T;
            if (!stop) rel = atomicAdd(a.claim, 1u);
        }
        rel = __shfl_sync(IMIN_FULL, rel, 0);
        if (rel >= a.count) break;
        // wrel: index of the world relative to `first` (outputs are indexed by it)
        const uint32_t wrel = a.list ? a.list[rel] : rel;
        const uint32_t j = (uint32_t)(a.first + (uint64_t)wrel);

        // ---- 1. masked reach BFS -------------------------------------------------
        for (int i = lane; i < nS; i += 32) {
            const int s = a.q.S[i];
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
                    b = a.row_ptr[u];
                    e = a.row_ptr[u + 1];
                    if (e > b) cnt = ((e + 3) >> 2) - (b >> 2);
                    wedges += (unsigned long long)(e - b);
                }
                const int incl = warp_incl_scan(cnt, lane);
                const int total = __shfl_sync(IMIN_FULL, incl, 31);
                for (int t0 = 0; t0 < total; t0 += 32) {
                    const int t = t0 + lane;
                    const int lo = owner_lane(incl, t);
                    const int ob = __shfl_sync(IMIN_FULL, b, lo);
                    const int oe = __shfl_sync(IMIN_FULL, e, lo);
                    const int ostart = __shfl_sync(IMIN_FULL, incl - cnt, lo);
                    const int oi = base + lo;
                    int nv[4] = {-1, -1, -1, -1};
                    int pvv[4] = {-1, -1, -1, -1};
                    if (t < total) {
                        const int g = (ob >> 2) + (t - ostart);
                        const int4 c4 = __ldg(a.col4 + g);
                        const uint4 t4 = __ldg(a.thr4 + g);
                        const uint4 w = philox10(make_uint4((uint32_t)g, j, tag, inst), klo, khi);
                        const int cv[4] = {c4.x, c4.y, c4.z, c4.w};
                        const uint32_t tv[4] = {t4.x, t4.y, t4.z, t4.w};
                        const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int ec = (g << 2) + c;
                            if (ec < ob || ec >= oe) continue;
                            if ((wv[c] >> 8) >= tv[c]) continue;
                            const int v = cv[c];
                            if (a.q.blocked_bm && bit_test(a.q.blocked_bm, v)) continue;
                            if (LOWER && !bit_test(a.q.seed_bm, v)) pvv[c] = v;
                            const uint32_t bit = 1u << (v & 31);
                            const uint32_t old = atomicOr(&bm[v >> 5], bit);
                            if (!(old & bit)) nv[c] = v;
                        }
                    }
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
                    if (lane == 0) atomicOr(a.out.err, DERR_TIMEOUT);
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
        if (UPPER && !ovf && a.q.nVs > 0) {
            int tnode = -1;
            if (lane == 0) {
                const uint4 w = philox10(make_uint4(0xFFFFFFFFu, j, tag, inst), klo, khi);
                const unsigned long long r64 = ((unsigned long long)w.y << 32) | w.x;
                const unsigned long long idx = __umul64hi(r64, (unsigned long long)a.q.nVs);
                const int t = a.q.Vs[idx];
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
                            b = a.in_ptr[v];
                            cnt = a.in_ptr[v + 1] - b;
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
                                const int u = __ldg(a.in_src + idx);
                                if (bit_test_cg(bm, u) && !bit_test(a.q.seed_bm, u)) {
                                    const int eid = __ldg(a.in_eid + idx);
                                    const uint32_t th = __ldg(a.in_thr + idx);
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
        unsigned long long sbase = 0;
        if (!ovf && store && (LOWER || UPPER)) {
            if (lane == 0) {
                if (LOWER)
                    sbase = reserve(a.out.rec_cursor, (unsigned long long)(tail - nS), a.out.rec_cap);
                else
                    sbase = tail2 > 0 ? reserve(a.out.set_cursor, (unsigned long long)tail2,
                                                a.out.set_cap)
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
                const uint32_t d = atomicAdd(a.out.n_deferred, 1u);
                if (d < a.out.deferred_cap)
                    a.out.deferred[d] = wrel;
                else
                    atomicOr(a.out.err, DERR_INTERNAL);
            }
            __syncwarp();
            continue;
        }

        // ---- 5. outputs ---------------------------------------------------------------
        if (LOWER) {
            if (a.out.credit_L)
                for (int i = nS + lane; i < tail; i += 32)
                    atomicAdd(a.out.credit_L + Q[i], (unsigned long long)__ldcg(sz + i));
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
                            a.out.rec_node[r] = Q[i];
                            a.out.rec_par[r] = poff;
                            a.out.rec_size[r] = size_i;
                        }
                        rootbase += rtot;
                    }
                    __syncwarp();
                }
            }
        }
        if (UPPER) {
            if (a.out.credit_U)
                for (int i = lane; i < tail2; i += 32) atomicAdd(a.out.credit_U + Q2[i], 1ull);
            if (store) {
                for (int i = lane; i < tail2; i += 32) a.out.set_elem[sbase + i] = Q2[i];
                if (lane == 0) {
                    a.out.set_off[wrel] = sbase;
                    a.out.set_len[wrel] = (uint32_t)tail2;
                }
            }
            for (int i = lane; i < tail2; i += 32) bm2[Q2[i] >> 5] = 0;
        }
        if (a.flags & WF_REACH)
            for (int i = lane; i < tail; i += 32) atomicAdd(a.out.reach + Q[i], 1ull);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wedges += __shfl_xor_sync(IMIN_FULL, wedges, o);
        if (lane == 0) {
            atomicAdd(a.out.acc + 0, (unsigned long long)tail);
            atomicAdd(a.out.acc + 1, wedges);
            if (UPPER && tail2 > 0) atomicAdd(a.out.acc + 2, 1ull);
            if (STOP) atomicAdd(a.out.acc + 3, (unsigned long long)tail);
            atomicAdd(a.out.acc + 4, 1ull);
            if (a.out.world_spread) a.out.world_spread[wrel] = (uint32_t)tail;
        }
        __syncwarp();
        for (int i = lane; i < tail; i += 32) bm[Q[i] >> 5] = 0;
        __syncwarp();
    }
}

inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

}  // namespace

size_t SlotCfg::bytes_per_slot() const
{
    size_t b = al16(bm_words * 4) + al16((size_t)qcap * 4);
    if (lower) {
        // loc is indexed by node id: n entries = 32 * bm_words upper bound
        b += al16(bm_words * 32 * 4) + 6 * al16((size_t)qcap * 4) + al16(((size_t)qcap + 2) * 4) +
             2 * al16((size_t)ecap * 4);
    }
    if (upper) b += al16(bm_words * 4) + al16((size_t)qcap * 4);
    return b;
}

void launch_worlds(imin_ctx *ctx, const imin_graph *g, const QueryDev &q, uint32_t flags,
                   uint64_t first, uint32_t count, const uint32_t *list, const SlotCfg &cfg,
                   void *slot_base, const WorldOut &out, uint32_t *claim_counter)
{
    if (count == 0) return;
    KArgs a;
    a.row_ptr = g->row_ptr.as<int32_t>();
    a.col4 = g->col.as<int4>();
    a.thr4 = g->thr.as<uint4>();
    a.in_ptr = g->in_ptr.as<int32_t>();
    a.in_src = g->in_src.as<int32_t>();
    a.in_eid = g->in_eid.as<int32_t>();
    a.in_thr = g->in_thr.as<uint32_t>();
    a.n = g->n;
    a.q = q;
    a.first = first;
    a.count = count;
    a.list = list;
    a.claim = claim_counter;
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
    a.out = out;

    const int threads = 256;
    const int blocks = cfg.warps / (threads / 32);
    IM_CUDA(cudaMemsetAsync(claim_counter, 0, sizeof(uint32_t), ctx->stream));
    const bool lower = (flags & WF_LOWER) != 0, upper = (flags & WF_UPPER) != 0,
               stop = (flags & WF_STOP) != 0;
    if (lower && upper) {
        world_kernel<true, true, false><<<blocks, threads, 0, ctx->stream>>>(a);
    } else if (lower) {
        world_kernel<true, false, false><<<blocks, threads, 0, ctx->stream>>>(a);
    } else if (upper) {
        world_kernel<false, true, false><<<blocks, threads, 0, ctx->stream>>>(a);
    } else if (stop) {
        world_kernel<false, false, true><<<blocks, threads, 0, ctx->stream>>>(a);
    } else {
        world_kernel<false, false, false><<<blocks, threads, 0, ctx->stream>>>(a);
    }
    IM_CHECK_LAUNCH();
}
