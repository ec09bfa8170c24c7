/*
 * oracle.c -- plain, single-threaded CPU oracle for the SandIMIN hot path
 * ("Efficient Influence Minimization via Node Blocking", arXiv 2405.12871).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  It may be used only by tests/, by the smoke check of the
 * package entry point and by the CPU-baseline leg of bench.py.  It shares no
 * code, header, table or constant generator with the CUDA path: every step is
 * re-derived here from the paper's text, in the paper's order, as slowly and
 * plainly as is practical.
 *
 * What it computes (paper passages in brackets):
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the edge coin
 *     that realises a live-edge world phi [Sec. 2.1, Eq. 1].
 *   - The reach set R_phi(s) of the unified seed s (virtual node, p=1 edges to
 *     every seed) with blocked nodes never entered [Sec. 2.1 blocking; Sec. 3.1].
 *   - Local Sampling [Algorithm 2]: DFS from s, Lengauer-Tarjan immediate
 *     dominators, CP sets built by inheriting idom's CP set in DFS order.
 *   - Global Sampling [Algorithm 3, Def. 4.2]: a uniform target in V'_s and
 *     its LRR set in phi^s [Sec. 3.3].
 *   - Procedure Max-Coverage [Algorithm 4] with Cov(B_i) and the top-k
 *     marginal sum needed by Cov^u [Algorithm 4, sigma^U; Lemma 5.3 proof].
 *   - The stopping-rule spread estimate (Dagum-Karp-Luby-Ross), LSBM
 *     [Algorithm 4], GSBM [Sec. 5.2], LHGA [Sec. 5.3] and the Sandwich
 *     combiner [Algorithm 1, Eq. 3].
 *
 * Readings where the paper is silent are listed at the top of each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define O_E 2.718281828459045235360287

/* ====================================================================== */
/* Philox4x32-10 (SC'11, "Parallel Random Numbers: As Easy as 1, 2, 3").   */
/* One round: two 32x32->64 products of the multipliers with words 0 and 2, */
/* the high halves xored with the other words and the round key.  The key  */
/* is bumped by the two Weyl constants between rounds.                     */
/* ====================================================================== */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Coin threshold: an edge with probability p is live in world j iff the
 * 24-bit uniform u = word >> 8 satisfies u * 2^-24 < p.  For an integer u this
 * is u < ceil(p * 2^24); the product is exact in double (p has a 24-bit
 * significand).  p = 0 gives 0 (never live), p = 1 gives 2^24 (always live). */
uint32_t oracle_coin_threshold(float p)
{
    double t = ceil((double)p * 16777216.0);
    if (t < 0.0) t = 0.0;
    if (t > 16777216.0) t = 16777216.0;
    return (uint32_t)t;
}

/* ====================================================================== */
/* Graph                                                                   */
/* ====================================================================== */
typedef struct OGraph {
    int32_t n;
    int64_t m;
    int64_t *row_ptr;   /* n+1 */
    int32_t *col;       /* m */
    float *prob;        /* m */
    uint32_t *thr;      /* m: coin thresholds */
    int64_t *in_ptr;    /* n+1: in-edges grouped by target */
    int32_t *in_src;    /* m */
    int64_t *in_eid;    /* m: id of the forward edge */
} OGraph;

void oracle_graph_free(OGraph *g)
{
    if (!g) return;
    free(g->row_ptr); free(g->col); free(g->prob); free(g->thr);
    free(g->in_ptr); free(g->in_src); free(g->in_eid);
    free(g);
}

OGraph *oracle_graph_new(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                         const float *prob)
{
    OGraph *g = (OGraph *)calloc(1, sizeof(OGraph));
    if (!g) return NULL;
    g->n = n; g->m = m;
    g->row_ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    g->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    g->prob = (float *)malloc(sizeof(float) * (size_t)(m > 0 ? m : 1));
    g->thr = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
    g->in_ptr = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    g->in_src = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    g->in_eid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    if (!g->row_ptr || !g->col || !g->prob || !g->thr || !g->in_ptr || !g->in_src || !g->in_eid) {
        oracle_graph_free(g);
        return NULL;
    }
    for (int32_t i = 0; i <= n; ++i) g->row_ptr[i] = row_ptr[i];
    for (int64_t e = 0; e < m; ++e) {
        g->col[e] = col[e];
        g->prob[e] = prob[e];
        g->thr[e] = oracle_coin_threshold(prob[e]);
    }
    /* in-edges by counting sort on the target, forward-edge order kept */
    for (int64_t e = 0; e < m; ++e) g->in_ptr[col[e] + 1]++;
    for (int32_t v = 0; v < n; ++v) g->in_ptr[v + 1] += g->in_ptr[v];
    int64_t *fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int32_t u = 0; u < n; ++u)
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col[e];
            int64_t at = g->in_ptr[v] + fill[v]++;
            g->in_src[at] = u;
            g->in_eid[at] = e;
        }
    free(fill);
    return g;
}

/* ====================================================================== */
/* Live-edge world phi [Sec. 2.1]: edge e is live in world j of stream     */
/* (tag, inst) under key iff (w >> 8) < thr[e], with w = word (e & 3) of   */
/* Philox(ctr = {e >> 2, j, tag, inst}, key = {key_lo, key_hi}).  A world  */
/* may instead be given explicitly as a 0/1 mask over the edges.           */
/* ====================================================================== */
typedef struct World {
    const uint8_t *mask;   /* explicit world, or NULL for Philox coins */
    uint64_t key;
    uint64_t j;
    uint32_t tag, inst;
} World;

static int live(const OGraph *g, const World *w, int64_t e)
{
    if (w->mask) return w->mask[e] != 0;
    uint32_t ctr[4] = {(uint32_t)(e >> 2), (uint32_t)w->j, w->tag, w->inst};
    uint32_t key[2] = {(uint32_t)w->key, (uint32_t)(w->key >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return (out[e & 3] >> 8) < g->thr[e];
}

int oracle_edge_live(const OGraph *g, int64_t e, uint64_t key, uint64_t j, uint32_t tag,
                     uint32_t inst)
{
    World w = {NULL, key, j, tag, inst};
    return live(g, &w, e);
}

/* Uniform index in [0, count) for the Global Sampling target of world j:
 * r64 = (out[1] << 32) | out[0] of Philox(ctr = {0xFFFFFFFF, j, tag, inst}),
 * index = floor(r64 * count / 2^64).  (The counter word 0 never equals an edge
 * group index because edge ids stay below 2^31.) */
uint64_t oracle_target_index(uint64_t key, uint64_t j, uint32_t tag, uint32_t inst, uint64_t count)
{
    uint32_t ctr[4] = {0xFFFFFFFFu, (uint32_t)j, tag, inst};
    uint32_t k[2] = {(uint32_t)key, (uint32_t)(key >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, k, out);
    uint64_t r64 = ((uint64_t)out[1] << 32) | (uint64_t)out[0];
    unsigned __int128 prod = (unsigned __int128)r64 * (unsigned __int128)count;
    return (uint64_t)(prod >> 64);
}

/* ====================================================================== */
/* Per-call workspace                                                      */
/* ====================================================================== */
typedef struct Work {
    int32_t n;
    uint8_t *is_seed;      /* n */
    uint8_t *is_blocked;   /* n */
    int32_t *mark;         /* n: world stamp of the last visit */
    int32_t stamp;
    int32_t *queue;        /* n */
    /* DFS / Lengauer-Tarjan over the reached nodes plus the virtual root s,
     * which gets local number 0; node v gets local id lid[v]. */
    int32_t *lid;          /* n */
    int32_t *node_of;      /* n+1: local id -> node (s -> -1) */
    int32_t *dfn;          /* n+1 (local) */
    int32_t *vertex;       /* n+1: dfs number -> local id */
    int32_t *parent;       /* n+1 */
    int32_t *semi, *idom, *label, *ancestor;
    int64_t *pred_off;     /* n+2 */
    int32_t *pred;         /* live in-edges (local ids), grown on demand */
    int64_t pred_cap;
    int32_t *bucket_head, *bucket_next;
    int32_t *stk_node;     /* DFS stack */
    int64_t *stk_edge;
    int32_t *cstk;         /* compress path */
    /* CP sets of the current world, flattened */
    int64_t *cp_off;       /* n+1 */
    int64_t *cp_len;       /* n+1 */
    int32_t *idom_node;    /* n: idom by node id of the last local-sampled world (-1 = s) */
    int32_t *cp_elem;
    int64_t cp_cap;
    /* reverse BFS for LRR */
    int32_t *mark2;
    int32_t stamp2;
    int32_t *queue2;
    /* pairs scratch for pred collection */
    int32_t *pair_u, *pair_v;
    int64_t pair_cap;
} Work;

static void work_free(Work *w)
{
    if (!w) return;
    free(w->is_seed); free(w->is_blocked); free(w->mark); free(w->queue); free(w->lid);
    free(w->node_of); free(w->dfn); free(w->vertex); free(w->parent); free(w->semi);
    free(w->idom); free(w->label); free(w->ancestor); free(w->pred_off); free(w->pred);
    free(w->bucket_head); free(w->bucket_next); free(w->stk_node); free(w->stk_edge);
    free(w->cstk); free(w->cp_off); free(w->cp_len); free(w->idom_node); free(w->cp_elem); free(w->mark2); free(w->queue2);
    free(w->pair_u); free(w->pair_v);
    free(w);
}

static Work *work_new(const OGraph *g, const int32_t *S, int32_t nS, const int32_t *B, int32_t nB)
{
    int32_t n = g->n;
    Work *w = (Work *)calloc(1, sizeof(Work));
    w->n = n;
    w->is_seed = (uint8_t *)calloc((size_t)n + 1, 1);
    w->is_blocked = (uint8_t *)calloc((size_t)n + 1, 1);
    w->mark = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    w->queue = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    w->lid = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    size_t L = (size_t)n + 2;
    w->node_of = (int32_t *)malloc(sizeof(int32_t) * L);
    w->dfn = (int32_t *)malloc(sizeof(int32_t) * L);
    w->vertex = (int32_t *)malloc(sizeof(int32_t) * L);
    w->parent = (int32_t *)malloc(sizeof(int32_t) * L);
    w->semi = (int32_t *)malloc(sizeof(int32_t) * L);
    w->idom = (int32_t *)malloc(sizeof(int32_t) * L);
    w->label = (int32_t *)malloc(sizeof(int32_t) * L);
    w->ancestor = (int32_t *)malloc(sizeof(int32_t) * L);
    w->pred_off = (int64_t *)malloc(sizeof(int64_t) * (L + 1));
    w->pred_cap = 1024;
    w->pred = (int32_t *)malloc(sizeof(int32_t) * (size_t)w->pred_cap);
    w->bucket_head = (int32_t *)malloc(sizeof(int32_t) * L);
    w->bucket_next = (int32_t *)malloc(sizeof(int32_t) * L);
    w->stk_node = (int32_t *)malloc(sizeof(int32_t) * L);
    w->stk_edge = (int64_t *)malloc(sizeof(int64_t) * L);
    w->cstk = (int32_t *)malloc(sizeof(int32_t) * L);
    w->cp_off = (int64_t *)malloc(sizeof(int64_t) * L);
    w->cp_len = (int64_t *)malloc(sizeof(int64_t) * L);
    w->idom_node = (int32_t *)malloc(sizeof(int32_t) * L);
    w->cp_cap = 1024;
    w->cp_elem = (int32_t *)malloc(sizeof(int32_t) * (size_t)w->cp_cap);
    w->mark2 = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    w->queue2 = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    w->pair_cap = 1024;
    w->pair_u = (int32_t *)malloc(sizeof(int32_t) * (size_t)w->pair_cap);
    w->pair_v = (int32_t *)malloc(sizeof(int32_t) * (size_t)w->pair_cap);
    for (int32_t i = 0; i < nS; ++i) w->is_seed[S[i]] = 1;
    for (int32_t i = 0; i < nB; ++i) w->is_blocked[B[i]] = 1;
    return w;
}

/* ====================================================================== */
/* Reach set R_phi(s) by BFS from the seeds [Sec. 2.1]; blocked nodes are   */
/* never entered (their in-edges have p = 0).  Seeds count in I_phi.       */
/* Returns |R|; the nodes are left in w->queue[0..|R|).                     */
/* ====================================================================== */
static int32_t world_reach(const OGraph *g, Work *w, const World *wd, const int32_t *S, int32_t nS)
{
    w->stamp++;
    int32_t head = 0, tail = 0;
    for (int32_t i = 0; i < nS; ++i) {
        int32_t s = S[i];
        if (w->mark[s] == w->stamp) continue;
        w->mark[s] = w->stamp;
        w->queue[tail++] = s;
    }
    while (head < tail) {
        int32_t u = w->queue[head++];
        for (int64_t e = g->row_ptr[u]; e < g->row_ptr[u + 1]; ++e) {
            int32_t v = g->col[e];
            if (w->is_blocked[v] || w->mark[v] == w->stamp) continue;
            if (!live(g, wd, e)) continue;
            w->mark[v] = w->stamp;
            w->queue[tail++] = v;
        }
    }
    return tail;
}

/* ====================================================================== */
/* Lengauer-Tarjan immediate dominators (TOPLAS 1979, the "simple" version  */
/* with path compression) over the live subgraph reached from s.  Local id  */
/* 0 is s; preds[] are live in-edges between reached nodes (plus s->seed).  */
/* ====================================================================== */
static int32_t lt_eval(Work *w, int32_t v)
{
    if (w->ancestor[v] < 0) return v;
    /* compress the ancestor path of v (iteratively) */
    int32_t top = 0;
    int32_t x = v;
    while (w->ancestor[w->ancestor[x]] >= 0) {
        w->cstk[top++] = x;
        x = w->ancestor[x];
    }
    while (top > 0) {
        int32_t y = w->cstk[--top];
        int32_t a = w->ancestor[y];
        if (w->semi[w->label[a]] < w->semi[w->label[y]]) w->label[y] = w->label[a];
        w->ancestor[y] = w->ancestor[a];
    }
    return w->label[v];
}

/* ====================================================================== */
/* Collections of sets (CP sets of several worlds, or LRR sets)            */
/* ====================================================================== */
typedef struct SetColl {
    int64_t nworlds;   /* |C| (CP sequences) or |L| (LRR sets incl. empty ones) */
    int64_t nsets;
    int64_t *off;      /* nsets + 1 */
    int32_t *elem;
    int64_t cap_sets, cap_elem;
} SetColl;

static void coll_init(SetColl *c)
{
    memset(c, 0, sizeof(*c));
    c->cap_sets = 1024;
    c->cap_elem = 4096;
    c->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(c->cap_sets + 1));
    c->elem = (int32_t *)malloc(sizeof(int32_t) * (size_t)c->cap_elem);
    c->off[0] = 0;
}

static void coll_free(SetColl *c)
{
    free(c->off);
    free(c->elem);
    memset(c, 0, sizeof(*c));
}

static void coll_add(SetColl *c, const int32_t *items, int64_t cnt)
{
    if (c->nsets + 1 > c->cap_sets) {
        c->cap_sets *= 2;
        c->off = (int64_t *)realloc(c->off, sizeof(int64_t) * (size_t)(c->cap_sets + 1));
    }
    int64_t base = c->off[c->nsets];
    if (base + cnt > c->cap_elem) {
        while (base + cnt > c->cap_elem) c->cap_elem *= 2;
        c->elem = (int32_t *)realloc(c->elem, sizeof(int32_t) * (size_t)c->cap_elem);
    }
    memcpy(c->elem + base, items, sizeof(int32_t) * (size_t)cnt);
    c->nsets++;
    c->off[c->nsets] = base + cnt;
}

/* Local Sampling [Algorithm 2] for one world.
 *   Line 2: DFS from s (s -> seeds in the given order, then live out-edges in
 *           CSR order) collecting R_phi(s) and every live in-edge between
 *           reached nodes (the predecessor lists Lengauer-Tarjan needs).
 *   Line 3: Lengauer-Tarjan immediate dominators with root s.
 *   Lines 4-12: for u in DFS order, u not a seed (M[u] = 0):
 *           C(u) = C(idom u) + {u}  if idom u is neither s nor a seed,
 *           C(u) = {u}               otherwise (the reading for idom u = s).
 * The CP sets are appended to *cp (when non-NULL).  Returns |R| (seeds
 * included); the reached nodes are left in w->queue[0..|R|) and marked with
 * the current w->stamp. */
static int32_t world_local_sampling(const OGraph *g, Work *w, const World *wd, const int32_t *S,
                                    int32_t nS, SetColl *cp)
{
    w->stamp++;
    int32_t nloc = 1;                 /* local 0 = s */
    w->node_of[0] = -1;
    int64_t npair = 0;
    int32_t ndfs = 0;
    w->dfn[0] = ndfs; w->vertex[ndfs++] = 0; w->parent[0] = -1;
    int32_t sp = 0;
    w->stk_node[sp] = 0; w->stk_edge[sp] = 0; sp++;
    while (sp > 0) {
        int32_t x = w->stk_node[sp - 1];
        int32_t child = -1;
        for (;;) {
            int32_t v;
            int32_t vl;
            if (x == 0) {
                if (w->stk_edge[sp - 1] >= nS) break;
                v = S[w->stk_edge[sp - 1]++];          /* edge s -> seed, p = 1 */
            } else {
                int32_t u = w->node_of[x];
                if (w->stk_edge[sp - 1] >= g->row_ptr[u + 1]) break;
                int64_t e = w->stk_edge[sp - 1]++;
                v = g->col[e];
                if (w->is_blocked[v]) continue;
                if (!live(g, wd, e)) continue;
            }
            int fresh = (w->mark[v] != w->stamp);
            if (fresh) {
                w->mark[v] = w->stamp;
                w->lid[v] = nloc;
                w->node_of[nloc] = v;
                nloc++;
            }
            vl = w->lid[v];
            if (npair == w->pair_cap) {
                w->pair_cap *= 2;
                w->pair_u = (int32_t *)realloc(w->pair_u, sizeof(int32_t) * (size_t)w->pair_cap);
                w->pair_v = (int32_t *)realloc(w->pair_v, sizeof(int32_t) * (size_t)w->pair_cap);
            }
            w->pair_u[npair] = x;
            w->pair_v[npair] = vl;
            npair++;
            if (fresh) { child = vl; break; }
        }
        if (child >= 0) {
            w->dfn[child] = ndfs; w->vertex[ndfs++] = child; w->parent[child] = x;
            w->stk_node[sp] = child;
            w->stk_edge[sp] = g->row_ptr[w->node_of[child]];
            sp++;
        } else {
            sp--;
        }
    }
    int32_t N = nloc;   /* reached nodes + s */
    for (int32_t i = 1; i < N; ++i) w->queue[i - 1] = w->node_of[i];

    /* predecessor lists (CSR over local ids) */
    for (int32_t i = 0; i <= N; ++i) w->pred_off[i] = 0;
    for (int64_t p = 0; p < npair; ++p) w->pred_off[w->pair_v[p] + 1]++;
    for (int32_t i = 0; i < N; ++i) w->pred_off[i + 1] += w->pred_off[i];
    if (npair > w->pred_cap) {
        w->pred_cap = npair;
        w->pred = (int32_t *)realloc(w->pred, sizeof(int32_t) * (size_t)w->pred_cap);
    }
    {
        int64_t *fill = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
        for (int64_t p = 0; p < npair; ++p) {
            int32_t v = w->pair_v[p];
            w->pred[w->pred_off[v] + fill[v]++] = w->pair_u[p];
        }
        free(fill);
    }

    /* Line 3: Lengauer-Tarjan; semi[] holds DFS numbers. */
    for (int32_t i = 0; i < N; ++i) {
        w->semi[i] = w->dfn[i];
        w->label[i] = i;
        w->ancestor[i] = -1;
        w->idom[i] = -1;
        w->bucket_head[i] = -1;
    }
    for (int32_t k = N - 1; k >= 1; --k) {
        int32_t x = w->vertex[k];
        for (int64_t p = w->pred_off[x]; p < w->pred_off[x + 1]; ++p) {
            int32_t u = lt_eval(w, w->pred[p]);
            if (w->semi[u] < w->semi[x]) w->semi[x] = w->semi[u];
        }
        int32_t sv = w->vertex[w->semi[x]];
        w->bucket_next[x] = w->bucket_head[sv];
        w->bucket_head[sv] = x;
        int32_t px = w->parent[x];
        w->ancestor[x] = px;                         /* LINK(parent(x), x) */
        for (int32_t v = w->bucket_head[px]; v >= 0;) {
            int32_t nxt = w->bucket_next[v];
            int32_t u = lt_eval(w, v);
            w->idom[v] = (w->semi[u] < w->semi[v]) ? u : px;
            v = nxt;
        }
        w->bucket_head[px] = -1;
    }
    for (int32_t k = 1; k < N; ++k) {
        int32_t x = w->vertex[k];
        if (w->idom[x] != w->vertex[w->semi[x]]) w->idom[x] = w->idom[w->idom[x]];
    }
    w->idom[0] = -1;
    /* export idom by node for inspection: idom_node[v] (s -> -1) */
    for (int32_t k = 1; k < N; ++k) {
        int32_t x = w->vertex[k];
        w->idom_node[w->node_of[x]] = (w->idom[x] == 0) ? -1 : w->node_of[w->idom[x]];
    }

    /* Lines 4-12: CP sets in DFS order. */
    if (cp) {
        int64_t ne = 0;
        for (int32_t k = 0; k < N; ++k) { w->cp_off[k] = -1; w->cp_len[k] = 0; }
        for (int32_t k = 1; k < N; ++k) {
            int32_t x = w->vertex[k];
            int32_t u = w->node_of[x];
            if (w->is_seed[u]) continue;                          /* M[u] = 1 */
            int32_t d = w->idom[x];
            int dom_marked = (d == 0) || w->is_seed[w->node_of[d]];  /* M[idom u] */
            int64_t need = 1 + (dom_marked ? 0 : w->cp_len[d]);
            if (ne + need > w->cp_cap) {
                while (ne + need > w->cp_cap) w->cp_cap *= 2;
                w->cp_elem = (int32_t *)realloc(w->cp_elem, sizeof(int32_t) * (size_t)w->cp_cap);
            }
            w->cp_off[x] = ne;
            if (!dom_marked) {
                memcpy(w->cp_elem + ne, w->cp_elem + w->cp_off[d],
                       sizeof(int32_t) * (size_t)w->cp_len[d]);
            }
            w->cp_elem[ne + need - 1] = u;
            w->cp_len[x] = need;
            coll_add(cp, w->cp_elem + ne, need);
            ne += need;
        }
    }
    return N - 1;
}

/* ====================================================================== */
/* V'_s: nodes reachable from S in G (edges with p > 0, blocked nodes never */
/* entered), excluding S [Sec. 4.2, before Lemma 4.2].  Sorted ascending.   */
/* ====================================================================== */
static int32_t compute_Vs(const OGraph *g, Work *w, const int32_t *S, int32_t nS, int32_t *out)
{
    w->stamp++;
    int32_t head = 0, tail = 0;
    for (int32_t i = 0; i < nS; ++i) {
        if (w->mark[S[i]] == w->stamp) continue;
        w->mark[S[i]] = w->stamp;
        w->queue[tail++] = S[i];
    }
    while (head < tail) {
        int32_t u = w->queue[head++];
        for (int64_t e = g->row_ptr[u]; e < g->row_ptr[u + 1]; ++e) {
            int32_t v = g->col[e];
            if (g->thr[e] == 0 || w->is_blocked[v] || w->mark[v] == w->stamp) continue;
            w->mark[v] = w->stamp;
            w->queue[tail++] = v;
        }
    }
    int32_t cnt = 0;
    for (int32_t v = 0; v < g->n; ++v)
        if (w->mark[v] == w->stamp && !w->is_seed[v]) out[cnt++] = v;
    return cnt;
}

/* Global Sampling [Algorithm 3] for world j: the LRR set of the target t
 * (nodes of R\S that reach t by live edges whose two endpoints lie in R\S),
 * or the empty set when t is not reached.  Requires that w->mark still holds
 * the reach set of this world (stamp == w->stamp).  Returns |L| (0 if empty),
 * the set left in w->queue2. */
static int32_t world_lrr(const OGraph *g, Work *w, const World *wd, const int32_t *Vs, int32_t nVs)
{
    if (nVs <= 0) return 0;
    uint64_t idx = oracle_target_index(wd->key, wd->j, wd->tag, wd->inst, (uint64_t)nVs);
    int32_t t = Vs[idx];
    if (w->mark[t] != w->stamp) return 0;      /* t not in R_phi(s) */
    w->stamp2++;
    int32_t head = 0, tail = 0;
    w->mark2[t] = w->stamp2;
    w->queue2[tail++] = t;
    while (head < tail) {
        int32_t v = w->queue2[head++];
        for (int64_t q = g->in_ptr[v]; q < g->in_ptr[v + 1]; ++q) {
            int32_t u = g->in_src[q];
            if (w->mark[u] != w->stamp || w->is_seed[u]) continue;   /* u must be in R \ S */
            if (w->mark2[u] == w->stamp2) continue;
            if (!live(g, wd, g->in_eid[q])) continue;
            w->mark2[u] = w->stamp2;
            w->queue2[tail++] = u;
        }
    }
    return tail;
}


/* ====================================================================== */
/* One explicit world (for pins): live[e] in {0,1}.  By node id:           */
/*   reached[v] in {0,1}; idom[v] = -2 unreached, -1 the unified seed s,    */
/*   else a node id; credit_lower[v] += number of CP sets containing v;     */
/*   lrr[v] = 1 for v in L(target) when target >= 0 (and target reached).   */
/* Returns |R| (seeds included).                                            */
/* ====================================================================== */
static int32_t lrr_from_target(const OGraph *g, Work *w, const World *wd, int32_t t);

int32_t oracle_world_explicit(const OGraph *g, const uint8_t *live_mask, const int32_t *S,
                              int32_t nS, const int32_t *B, int32_t nB, int32_t target,
                              uint8_t *reached, int32_t *idom, uint64_t *credit_lower,
                              uint8_t *lrr)
{
    Work *w = work_new(g, S, nS, B, nB);
    World wd = {live_mask, 0, 0, 0, 0};
    SetColl cp;
    coll_init(&cp);
    int32_t R = world_local_sampling(g, w, &wd, S, nS, &cp);
    for (int32_t v = 0; v < g->n; ++v) {
        if (reached) reached[v] = 0;
        if (idom) idom[v] = -2;
        if (lrr) lrr[v] = 0;
    }
    for (int32_t i = 0; i < R; ++i) {
        int32_t v = w->queue[i];
        if (reached) reached[v] = 1;
        if (idom) idom[v] = w->idom_node[v];
    }
    if (credit_lower)
        for (int64_t p = 0; p < cp.off[cp.nsets]; ++p) credit_lower[cp.elem[p]] += 1;
    if (lrr && target >= 0 && w->mark[target] == w->stamp && !w->is_seed[target]) {
        int32_t L = lrr_from_target(g, w, &wd, target);
        for (int32_t i = 0; i < L; ++i) lrr[w->queue2[i]] = 1;
    }
    coll_free(&cp);
    work_free(w);
    return R;
}

/* Reverse BFS of Definition 4.2: nodes of R \ S reaching t in phi^s. */
static int32_t lrr_from_target(const OGraph *g, Work *w, const World *wd, int32_t t)
{
    w->stamp2++;
    int32_t head = 0, tail = 0;
    w->mark2[t] = w->stamp2;
    w->queue2[tail++] = t;
    while (head < tail) {
        int32_t v = w->queue2[head++];
        for (int64_t q = g->in_ptr[v]; q < g->in_ptr[v + 1]; ++q) {
            int32_t u = g->in_src[q];
            if (w->mark[u] != w->stamp || w->is_seed[u]) continue;   /* u in R \ S */
            if (w->mark2[u] == w->stamp2) continue;
            if (!live(g, wd, g->in_eid[q])) continue;
            w->mark2[u] = w->stamp2;
            w->queue2[tail++] = u;
        }
    }
    return tail;
}

/* ====================================================================== */
/* imin_sample counterpart: worlds [first, first + theta) of stream         */
/* (key, tag, inst).  mode bits: 1 = reach counts, 2 = lower credit (CP     */
/* sets), 4 = upper credit (LRR sets).  Counts are ADDED into the arrays.   */
/* scal[0] = sum |R_j| (seeds included), scal[1] = edges scanned (sum of    */
/* out-degrees of reached nodes), scal[2] = worlds with a non-empty LRR set.*/
/* ====================================================================== */
int oracle_sample(const OGraph *g, const int32_t *S, int32_t nS, const int32_t *B, int32_t nB,
                  uint64_t theta, uint64_t key, uint32_t tag, uint32_t inst, uint64_t first,
                  uint32_t mode, uint64_t *reach, uint64_t *credit_lower, uint64_t *credit_upper,
                  uint32_t *world_spread, uint64_t *scal)
{
    Work *w = work_new(g, S, nS, B, nB);
    int32_t *Vs = NULL;
    int32_t nVs = 0;
    if (mode & 4) {
        Vs = (int32_t *)malloc(sizeof(int32_t) * ((size_t)g->n + 1));
        nVs = compute_Vs(g, w, S, nS, Vs);
    }
    SetColl cp;
    coll_init(&cp);
    scal[0] = scal[1] = scal[2] = 0;
    for (uint64_t t = 0; t < theta; ++t) {
        World wd = {NULL, key, first + t, tag, inst};
        int32_t R;
        if (mode & 2) {
            cp.nsets = 0;
            cp.off[0] = 0;
            R = world_local_sampling(g, w, &wd, S, nS, &cp);
            if (credit_lower)
                for (int64_t p = 0; p < cp.off[cp.nsets]; ++p) credit_lower[cp.elem[p]] += 1;
        } else {
            R = world_reach(g, w, &wd, S, nS);
        }
        for (int32_t i = 0; i < R; ++i) {
            int32_t u = w->queue[i];
            if ((mode & 1) && reach) reach[u] += 1;
            scal[1] += (uint64_t)(g->row_ptr[u + 1] - g->row_ptr[u]);
        }
        scal[0] += (uint64_t)R;
        if (world_spread) world_spread[t] = (uint32_t)R;
        if (mode & 4) {
            int32_t L = world_lrr(g, w, &wd, Vs, nVs);
            if (L > 0) {
                scal[2] += 1;
                if (credit_upper)
                    for (int32_t i = 0; i < L; ++i) credit_upper[w->queue2[i]] += 1;
            }
        }
    }
    coll_free(&cp);
    free(Vs);
    work_free(w);
    return 0;
}

/* ====================================================================== */
/* LRR sequences (Sec. 4.2, "Discussion" after Algorithm 3): in world phi,  */
/* the LRR set L_phi(v) of EVERY node v of R_phi(s) \ S, each by its own   */
/* reverse traversal of phi^s (the one-per-reached-node cost the paper's    */
/* Table 2 measures).  Per world:                                            */
/*   credit_useq[u] += |{v : u in L_phi(v)}| (= |M_phi({u})|),              */
/*   elements += sum over v of |L_phi(v)|,                                   */
/*   cov = |{v : L_phi(v) meets Q}| (= |M_phi(Q)|, the world's term of       */
/*   Cov_{L^s}(Q), whose mean over worlds is D^U(Q)).                        */
/* ====================================================================== */
static uint64_t world_lrr_sequence(const OGraph *g, Work *w, const World *wd, const int32_t *S,
                                   int32_t nS, const uint8_t *inQ, uint64_t *credit_useq,
                                   uint64_t *elements, int32_t *R_out)
{
    int32_t R = world_reach(g, w, wd, S, nS);
    uint64_t cov = 0;
    for (int32_t i = 0; i < R; ++i) {
        int32_t v = w->queue[i];
        if (w->is_seed[v]) continue;
        int32_t L = lrr_from_target(g, w, wd, v);
        int meets = 0;
        for (int32_t q = 0; q < L; ++q) {
            int32_t u = w->queue2[q];
            if (credit_useq) credit_useq[u] += 1;
            if (inQ && inQ[u]) meets = 1;
        }
        *elements += (uint64_t)L;
        cov += (uint64_t)meets;
    }
    if (R_out) *R_out = R;
    return cov;
}

/* worlds [first, first + theta) of (key, tag, inst), blocked set B, query set Q;
 * counts are ADDED into credit_useq; cov_world[t] = |M_phi(Q)| of world first + t;
 * scal[0] = sum of |L(v)|, scal[1] = sum of cov_world, scal[2] = sum |R_j|. */
int oracle_sample_useq(const OGraph *g, const int32_t *S, int32_t nS, const int32_t *B, int32_t nB,
                       const int32_t *Q, int32_t nQ, uint64_t theta, uint64_t key, uint32_t tag,
                       uint32_t inst, uint64_t first, uint64_t *credit_useq, uint64_t *cov_world,
                       uint64_t *scal)
{
    Work *w = work_new(g, S, nS, B, nB);
    uint8_t *inQ = (uint8_t *)calloc((size_t)g->n + 1, 1);
    for (int32_t i = 0; i < nQ; ++i) inQ[Q[i]] = 1;
    scal[0] = scal[1] = scal[2] = 0;
    for (uint64_t t = 0; t < theta; ++t) {
        World wd = {NULL, key, first + t, tag, inst};
        int32_t R = 0;
        uint64_t c = world_lrr_sequence(g, w, &wd, S, nS, inQ, credit_useq, &scal[0], &R);
        if (cov_world) cov_world[t] = c;
        scal[1] += c;
        scal[2] += (uint64_t)R;
    }
    free(inQ);
    work_free(w);
    return 0;
}

/* the same for one explicit world (live_mask[e] = 1 if edge e is live) */
int oracle_useq_explicit(const OGraph *g, const uint8_t *live_mask, const int32_t *S, int32_t nS,
                         const int32_t *Q, int32_t nQ, uint64_t *credit_useq, uint64_t *scal)
{
    Work *w = work_new(g, S, nS, NULL, 0);
    uint8_t *inQ = (uint8_t *)calloc((size_t)g->n + 1, 1);
    for (int32_t i = 0; i < nQ; ++i) inQ[Q[i]] = 1;
    World wd = {live_mask, 0, 0, 0, 0};
    int32_t R = 0;
    scal[0] = 0;
    scal[1] = world_lrr_sequence(g, w, &wd, S, nS, inQ, credit_useq, &scal[0], &R);
    scal[2] = (uint64_t)R;
    free(inQ);
    work_free(w);
    return 0;
}

/* V'_s as an API (count returned; nodes written to out[] ascending). */
int32_t oracle_vs(const OGraph *g, const int32_t *S, int32_t nS, const int32_t *B, int32_t nB,
                  int32_t *out)
{
    Work *w = work_new(g, S, nS, B, nB);
    int32_t c = compute_Vs(g, w, S, nS, out);
    work_free(w);
    return c;
}

/* ====================================================================== */
/* Procedure Max-Coverage [Algorithm 4] over a collection of sets.          */
/* Round i (i = 0, 1, ...) sees B_i (the first i picks):                    */
/*   cov[i]  = Cov(B_i) = number of sets meeting B_i,                       */
/*   topk[i] = sum of the k largest marginal coverages w.r.t. B_i           */
/*             (maxMC(B_i, k) of the Cov^u line and Lemma 5.3's proof);     */
/* then u = argmax marginal coverage (reading: ties to the smaller node id; */
/* a zero maximum ends the procedure early, |B| <= k is allowed).           */
/* Returns |B|; cov[] and topk[] get |B| + 1 entries.                       */
/* ====================================================================== */
static int cmp_u64_desc(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x < y) - (x > y);
}

static uint64_t sum_top_k(const uint64_t *gain, int32_t n, int32_t k, uint64_t *scratch)
{
    /* plain: copy, sort descending, add the first k */
    memcpy(scratch, gain, sizeof(uint64_t) * (size_t)n);
    qsort(scratch, (size_t)n, sizeof(uint64_t), cmp_u64_desc);
    uint64_t s = 0;
    for (int32_t i = 0; i < k && i < n; ++i) s += scratch[i];
    return s;
}

static int32_t max_coverage(const SetColl *c, int32_t n, int32_t k, int32_t *B, uint64_t *cov,
                            uint64_t *topk)
{
    int64_t ns = c->nsets;
    /* inverted index node -> sets */
    int64_t *ioff = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t p = 0; p < c->off[ns]; ++p) ioff[c->elem[p] + 1]++;
    for (int32_t v = 0; v < n; ++v) ioff[v + 1] += ioff[v];
    int64_t *iset = (int64_t *)malloc(sizeof(int64_t) * (size_t)(c->off[ns] > 0 ? c->off[ns] : 1));
    int64_t *fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t s = 0; s < ns; ++s)
        for (int64_t p = c->off[s]; p < c->off[s + 1]; ++p) {
            int32_t v = c->elem[p];
            iset[ioff[v] + fill[v]++] = s;
        }
    free(fill);
    uint64_t *gain = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    uint64_t *scratch = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    uint8_t *covered = (uint8_t *)calloc((size_t)(ns > 0 ? ns : 1), 1);
    for (int64_t p = 0; p < c->off[ns]; ++p) gain[c->elem[p]] += 1;
    int32_t nb = 0;
    cov[0] = 0;
    for (int32_t i = 0;; ++i) {
        topk[i] = sum_top_k(gain, n, k, scratch);
        if (i == k) break;
        int32_t u = -1;
        uint64_t best = 0;
        for (int32_t v = 0; v < n; ++v)
            if (gain[v] > best) { best = gain[v]; u = v; }
        if (u < 0) break;                              /* max marginal coverage is 0 */
        B[nb++] = u;
        cov[i + 1] = cov[i] + best;
        for (int64_t q = ioff[u]; q < ioff[u + 1]; ++q) {
            int64_t s = iset[q];
            if (covered[s]) continue;
            covered[s] = 1;
            for (int64_t p = c->off[s]; p < c->off[s + 1]; ++p) gain[c->elem[p]] -= 1;
        }
    }
    free(ioff); free(iset); free(gain); free(scratch); free(covered);
    return nb;
}

/* Cov of a fixed set B: number of sets that meet B. */
static uint64_t coll_cov(const SetColl *c, const uint8_t *inB)
{
    uint64_t cnt = 0;
    for (int64_t s = 0; s < c->nsets; ++s)
        for (int64_t p = c->off[s]; p < c->off[s + 1]; ++p)
            if (inB[c->elem[p]]) { cnt++; break; }
    return cnt;
}

/* Max-Coverage over caller-given sets (pins). */
int32_t oracle_max_coverage_sets(int64_t nsets, const int64_t *off, const int32_t *elem, int32_t n,
                                 int32_t k, int32_t *B, uint64_t *cov, uint64_t *topk)
{
    SetColl c;
    coll_init(&c);
    for (int64_t s = 0; s < nsets; ++s) coll_add(&c, elem + off[s], off[s + 1] - off[s]);
    int32_t nb = max_coverage(&c, n, k, B, cov, topk);
    coll_free(&c);
    return nb;
}

/* ====================================================================== */
/* Spread estimate by the stopping rule (reading of the cited "generalized  */
/* stopping rule"): Dagum-Karp-Luby-Ross with Z_j = |R_j| / W, where        */
/* W = |V'_s| + |S| bounds I_phi.  Upsilon = 4(e-2) ln(2/delta') / beta^2,  */
/* Upsilon1 = 1 + (1+beta) Upsilon.  Worlds j = 0, 1, ... are drawn until   */
/* sum |R_j| >= T = ceil(Upsilon1 * W); then N = j + 1 and                  */
/* I = W * Upsilon1 / N.                                                    */
/* ====================================================================== */
static uint64_t stop_rule(const OGraph *g, const int32_t *S, int32_t nS, const int32_t *B,
                          int32_t nB, double beta, double dprime, uint64_t key, uint32_t tag,
                          uint32_t inst, double *I_out, uint64_t *edges_out, int32_t *nVs_out)
{
    Work *w = work_new(g, S, nS, B, nB);
    int32_t *Vs = (int32_t *)malloc(sizeof(int32_t) * ((size_t)g->n + 1));
    int32_t nVs = compute_Vs(g, w, S, nS, Vs);
    free(Vs);
    double W = (double)nVs + (double)nS;
    double ups = 4.0 * (O_E - 2.0) * log(2.0 / dprime) / (beta * beta);
    double ups1 = 1.0 + (1.0 + beta) * ups;
    uint64_t T = (uint64_t)ceil(ups1 * W);
    uint64_t sum = 0, N = 0, edges = 0;
    for (uint64_t j = 0;; ++j) {
        World wd = {NULL, key, j, tag, inst};
        int32_t R = world_reach(g, w, &wd, S, nS);
        for (int32_t i = 0; i < R; ++i) {
            int32_t u = w->queue[i];
            edges += (uint64_t)(g->row_ptr[u + 1] - g->row_ptr[u]);
        }
        sum += (uint64_t)R;
        if (sum >= T) { N = j + 1; break; }
    }
    *I_out = W * ups1 / (double)N;
    if (edges_out) *edges_out = edges;
    if (nVs_out) *nVs_out = nVs;
    work_free(w);
    return N;
}

uint64_t oracle_stop_rule(const OGraph *g, const int32_t *S, int32_t nS, const int32_t *B,
                          int32_t nB, double beta, double dprime, uint64_t key, uint32_t tag,
                          uint32_t inst, double *I_out)
{
    return stop_rule(g, S, nS, B, nB, beta, dprime, key, tag, inst, I_out, NULL, NULL);
}

/* ====================================================================== */
/* Host math of LSBM / GSBM (Algorithm 4, Lemma 5.2, Sec. 5.2)              */
/* ====================================================================== */
static double ln_binom(double a, double b)
{
    return lgamma(a + 1.0) - lgamma(b + 1.0) - lgamma(a - b + 1.0);
}

/* sigma^L branch value ((sqrt(x + 2a/9) - sqrt(a/2))^2 - a/18) / theta */
static double sigma_low(double x, double a, double theta)
{
    double r = sqrt(x + 2.0 * a / 9.0) - sqrt(a / 2.0);
    return (r * r - a / 18.0) / theta;
}

/* (sqrt(y + a/2) + sqrt(a/2))^2 / theta */
static double sigma_up(double y, double a, double theta)
{
    double r = sqrt(y + a / 2.0) + sqrt(a / 2.0);
    return r * r / theta;
}

double oracle_sigma_low(double x, double a, double theta) { return sigma_low(x, a, theta); }
double oracle_sigma_up(double y, double a, double theta) { return sigma_up(y, a, theta); }

/* theta_max of Lemma 5.2 (LSBM) */
double oracle_lsbm_theta_max(double I_hat, int32_t n, int32_t nS, int32_t k, double eps,
                             double delta, double beta, double OPT)
{
    double a = 1.0 - 1.0 / O_E;
    double l12 = log(12.0 / delta);
    double c = a * sqrt(l12) + sqrt(a * (ln_binom((double)(n - nS), (double)k) + l12));
    return 2.0 * I_hat * c * c / ((1.0 - beta) * eps * eps * OPT);
}

/* theta_max of Sec. 5.2 (GSBM); reading: ln C(max(|V'_s| - |S|, k), k). */
double oracle_gsbm_theta_max(int32_t nVs, int32_t nS, int32_t k, double eps, double delta,
                             double OPT)
{
    double a = 1.0 - 1.0 / O_E;
    double l6 = log(6.0 / delta);
    int32_t top = nVs - nS;
    if (top < k) top = k;
    double c = a * sqrt(l6) + sqrt(a * (ln_binom((double)top, (double)k) + l6));
    return 2.0 * (double)nVs * c * c / (eps * eps * OPT);
}

/* ====================================================================== */
/* Solve (Algorithm 1 with LSBM, GSBM, LHGA)                                */
/* ====================================================================== */
typedef struct OResult {
    int32_t n_blockers, chosen, iters_L, iters_U;
    int32_t nBL, nBU, nBR, nVs;
    double I_hat, I_after[3], sigmaL_L, sigmaU_L, sigmaL_U, sigmaU_U, DL_hat, DU_hat, ratio_lb,
        OPT_L, theta_max_L, theta_max_U;
    uint64_t n_spread, theta_C1, theta_C2, theta_L1, theta_L2, n_final[3], covC2, covL2;
} OResult;

enum { OV_SANDIMIN = 0, OV_SANDIMIN_MINUS = 1, OV_LSBM = 2, OV_GSBM = 3, OV_LHGA = 4 };

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

typedef struct { double score; int32_t v; } ScoreItem;

static int cmp_score_desc(const void *a, const void *b)
{
    const ScoreItem *x = (const ScoreItem *)a, *y = (const ScoreItem *)b;
    if (x->score > y->score) return -1;
    if (x->score < y->score) return 1;
    return (x->v > y->v) - (x->v < y->v);
}

static void append_cp_worlds(const OGraph *g, Work *w, const int32_t *S, int32_t nS, SetColl *c,
                             uint64_t from, uint64_t to, uint64_t key, uint32_t tag, uint32_t inst)
{
    for (uint64_t j = from; j < to; ++j) {
        World wd = {NULL, key, j, tag, inst};
        world_local_sampling(g, w, &wd, S, nS, c);
        c->nworlds++;
    }
}

static void append_lrr_worlds(const OGraph *g, Work *w, const int32_t *S, int32_t nS,
                              const int32_t *Vs, int32_t nVs, SetColl *c, uint64_t from,
                              uint64_t to, uint64_t key, uint32_t tag, uint32_t inst)
{
    for (uint64_t j = from; j < to; ++j) {
        World wd = {NULL, key, j, tag, inst};
        world_reach(g, w, &wd, S, nS);
        int32_t L = world_lrr(g, w, &wd, Vs, nVs);
        if (L > 0) coll_add(c, w->queue2, L);
        c->nworlds++;
    }
}

int oracle_solve(const OGraph *g, const int32_t *S_in, int32_t nS, int32_t k, double eps,
                 double delta, double beta, double gamma, uint64_t key, uint32_t inst,
                 int32_t variant, uint64_t fixed_theta, uint64_t pr_worlds, int32_t *blockers,
                 int32_t *BL, int32_t *BU, int32_t *BR, OResult *res)
{
    memset(res, 0, sizeof(*res));
    int32_t n = g->n;
    int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nS > 0 ? nS : 1));
    memcpy(S, S_in, sizeof(int32_t) * (size_t)nS);
    qsort(S, (size_t)nS, sizeof(int32_t), cmp_i32);
    Work *w = work_new(g, S, nS, NULL, 0);

    /* ON: nodes directly activated by S (out-neighbours with p > 0, not in S) */
    uint8_t *inON = (uint8_t *)calloc((size_t)n + 1, 1);
    for (int32_t i = 0; i < nS; ++i)
        for (int64_t e = g->row_ptr[S[i]]; e < g->row_ptr[S[i] + 1]; ++e)
            if (g->thr[e] > 0 && !w->is_seed[g->col[e]]) inON[g->col[e]] = 1;
    int32_t nON = 0;
    for (int32_t v = 0; v < n; ++v) nON += inON[v];
    int32_t *ON = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nON > 0 ? nON : 1));
    nON = 0;
    for (int32_t v = 0; v < n; ++v) if (inON[v]) ON[nON++] = v;

    if (nON <= k) {                        /* Algorithm 4, lines 2-3 (and Sec. 5.3) */
        for (int32_t i = 0; i < nON; ++i) blockers[i] = BL[i] = BU[i] = BR[i] = ON[i];
        res->n_blockers = res->nBL = res->nBU = res->nBR = nON;
        res->chosen = 0;
        free(ON); free(inON); free(S); work_free(w);
        return 0;
    }

    /* q(v) = 1 - prod over seed edges (u, v) of (1 - p_q(u, v)), p_q = thr / 2^24:
     * the probability that v is activated directly by S (reading of Pr[s -> v]). */
    double *prod = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    for (int32_t v = 0; v < n; ++v) prod[v] = 1.0;
    for (int32_t i = 0; i < nS; ++i)
        for (int64_t e = g->row_ptr[S[i]]; e < g->row_ptr[S[i] + 1]; ++e) {
            int32_t v = g->col[e];
            if (!inON[v]) continue;
            double pq = (double)g->thr[e] / 16777216.0;
            prod[v] = prod[v] * (1.0 - pq);
        }
    double *pr = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    for (int32_t v = 0; v < n; ++v) pr[v] = 1.0 - prod[v];
    /* The alternative reading: Pr[s -> v] as the fraction of the worlds
     * 0 .. pr_worlds - 1 of stream tag 6 in which S reaches v. */
    if (pr_worlds > 0) {
        uint64_t *cnt = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
        for (uint64_t t = 0; t < pr_worlds; ++t) {
            World wd = {NULL, key, t, 6u, inst};
            int32_t R = world_reach(g, w, &wd, S, nS);
            for (int32_t i = 0; i < R; ++i) cnt[w->queue[i]] += 1;
        }
        for (int32_t v = 0; v < n; ++v) pr[v] = (double)cnt[v] / (double)pr_worlds;
        free(cnt);
    }
    ScoreItem *byq = (ScoreItem *)malloc(sizeof(ScoreItem) * (size_t)nON);
    ScoreItem *bys = (ScoreItem *)malloc(sizeof(ScoreItem) * (size_t)nON);
    for (int32_t i = 0; i < nON; ++i) {
        int32_t v = ON[i];
        double q = pr[v];
        byq[i].score = q; byq[i].v = v;
        bys[i].score = q * (double)(g->row_ptr[v + 1] - g->row_ptr[v]); bys[i].v = v;
    }
    qsort(byq, (size_t)nON, sizeof(ScoreItem), cmp_score_desc);
    qsort(bys, (size_t)nON, sizeof(ScoreItem), cmp_score_desc);
    double OPT = 0.0;
    for (int32_t i = 0; i < k; ++i) OPT += byq[i].score;
    res->OPT_L = OPT;
    free(pr);
    if (!(OPT > 0.0)) {                    /* no top-k node reached in any world */
        free(byq); free(bys); free(prod); free(ON); free(inON); free(S); work_free(w);
        return 2;
    }

    /* LHGA (Sec. 5.3): top-k of ON by q(v) * outdeg(v) */
    for (int32_t i = 0; i < k; ++i) BR[i] = bys[i].v;
    res->nBR = k;

    int32_t *Vs = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t nVs = compute_Vs(g, w, S, nS, Vs);
    res->nVs = nVs;
    double one_m_inv_e_m_eps = 1.0 - 1.0 / O_E - eps;

    int32_t *Btmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    uint64_t *cov = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)k + 1));
    uint64_t *topk = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)k + 1));
    uint8_t *inB = (uint8_t *)calloc((size_t)n + 1, 1);

    int do_L = (variant == OV_SANDIMIN || variant == OV_SANDIMIN_MINUS || variant == OV_LSBM);
    int do_U = (variant == OV_SANDIMIN || variant == OV_GSBM);
    int do_R = (variant == OV_SANDIMIN || variant == OV_SANDIMIN_MINUS || variant == OV_LHGA);

    /* ---------------- LSBM (Algorithm 4) ---------------- */
    double I_hat = 0.0;
    {
        uint64_t edges = 0;
        res->n_spread = stop_rule(g, S, nS, NULL, 0, beta, delta / 6.0, key, 0, inst, &I_hat,
                                  &edges, NULL);
        res->I_hat = I_hat;
    }
    if (do_L) {
        double th_max = oracle_lsbm_theta_max(I_hat, n, nS, k, eps, delta, beta, OPT);
        double th0d = floor(th_max * (1.0 - beta) * eps * eps * OPT / I_hat);
        if (th0d < 1.0) th0d = 1.0;
        int32_t imax = (int32_t)ceil(log2(th_max / th0d));
        if (imax < 1) imax = 1;
        uint64_t th = (uint64_t)th0d;
        if (fixed_theta) { th = fixed_theta; imax = 1; }
        res->theta_max_L = th_max;
        double a1 = log(3.0 * (double)imax / delta), a2 = a1;
        SetColl C1, C2;
        coll_init(&C1); coll_init(&C2);
        append_cp_worlds(g, w, S, nS, &C1, 0, th, key, 1, inst);
        append_cp_worlds(g, w, S, nS, &C2, 0, th, key, 2, inst);
        int32_t nb = 0;
        double sL = 0.0, sU = 0.0;
        uint64_t cov2 = 0;
        for (int32_t i = 1; i <= imax; ++i) {
            nb = max_coverage(&C1, n, k, Btmp, cov, topk);
            uint64_t covu = cov[0] + topk[0];
            for (int32_t t = 1; t <= nb; ++t)
                if (cov[t] + topk[t] < covu) covu = cov[t] + topk[t];
            memset(inB, 0, (size_t)n);
            for (int32_t t = 0; t < nb; ++t) inB[Btmp[t]] = 1;
            cov2 = coll_cov(&C2, inB);
            double xlo = (double)cov2 * (1.0 - beta) / I_hat;
            double xhi = (double)cov2 * (1.0 + beta) / I_hat;
            sL = 0.0;
            if (xlo >= 5.0 * a1 / 18.0) sL = sigma_low(xlo, a1, (double)C2.nworlds);
            else if (xhi <= 5.0 * a1 / 18.0) sL = sigma_low(xhi, a1, (double)C2.nworlds);
            sU = sigma_up((double)covu * (1.0 + beta) / I_hat, a2, (double)C1.nworlds);
            res->iters_L = i;
            if (sL / sU >= one_m_inv_e_m_eps || i == imax) break;
            append_cp_worlds(g, w, S, nS, &C1, th, 2 * th, key, 1, inst);
            append_cp_worlds(g, w, S, nS, &C2, th, 2 * th, key, 2, inst);
            th *= 2;
        }
        for (int32_t t = 0; t < nb; ++t) BL[t] = Btmp[t];
        res->nBL = nb;
        res->sigmaL_L = sL; res->sigmaU_L = sU;
        res->theta_C1 = (uint64_t)C1.nworlds; res->theta_C2 = (uint64_t)C2.nworlds;
        res->covC2 = cov2;
        res->DL_hat = (double)cov2 / (double)C2.nworlds;
        coll_free(&C1); coll_free(&C2);
    }

    /* ---------------- GSBM (Sec. 5.2) ---------------- */
    if (do_U) {
        double th_max = oracle_gsbm_theta_max(nVs, nS, k, eps, delta, OPT);
        double th0d = floor(th_max * eps * eps * OPT / (double)nVs);
        if (th0d < 1.0) th0d = 1.0;
        int32_t imax = (int32_t)ceil(log2(th_max / th0d));
        if (imax < 1) imax = 1;
        uint64_t th = (uint64_t)th0d;
        if (fixed_theta) { th = fixed_theta; imax = 1; }
        res->theta_max_U = th_max;
        double a1 = log(3.0 * (double)imax / delta), a2 = a1;
        SetColl L1, L2;
        coll_init(&L1); coll_init(&L2);
        append_lrr_worlds(g, w, S, nS, Vs, nVs, &L1, 0, th, key, 3, inst);
        append_lrr_worlds(g, w, S, nS, Vs, nVs, &L2, 0, th, key, 4, inst);
        int32_t nb = 0;
        double sL = 0.0, sU = 0.0;
        uint64_t cov2 = 0;
        for (int32_t i = 1; i <= imax; ++i) {
            nb = max_coverage(&L1, n, k, Btmp, cov, topk);
            uint64_t covu = cov[0] + topk[0];
            for (int32_t t = 1; t <= nb; ++t)
                if (cov[t] + topk[t] < covu) covu = cov[t] + topk[t];
            memset(inB, 0, (size_t)n);
            for (int32_t t = 0; t < nb; ++t) inB[Btmp[t]] = 1;
            cov2 = coll_cov(&L2, inB);
            sL = sigma_low((double)cov2, a1, (double)L2.nworlds) * (double)nVs;
            sU = sigma_up((double)covu, a2, (double)L1.nworlds) * (double)nVs;
            res->iters_U = i;
            if (sL / sU >= one_m_inv_e_m_eps || i == imax) break;
            append_lrr_worlds(g, w, S, nS, Vs, nVs, &L1, th, 2 * th, key, 3, inst);
            append_lrr_worlds(g, w, S, nS, Vs, nVs, &L2, th, 2 * th, key, 4, inst);
            th *= 2;
        }
        for (int32_t t = 0; t < nb; ++t) BU[t] = Btmp[t];
        res->nBU = nb;
        res->sigmaL_U = sL; res->sigmaU_U = sU;
        res->theta_L1 = (uint64_t)L1.nworlds; res->theta_L2 = (uint64_t)L2.nworlds;
        res->covL2 = cov2;
        res->DU_hat = (double)nVs * (double)cov2 / (double)L2.nworlds;
        coll_free(&L1); coll_free(&L2);
    }

    /* ---------------- Sandwich (Algorithm 1, lines 4-5) ----------------
     * Reading: the paper does not say which worlds the three (gamma, delta)-
     * estimates draw.  They draw the same ones (stream tag 5, common random
     * numbers): each candidate's estimate is still the stopping rule over an
     * i.i.d. sequence of worlds, so each keeps its guarantee, and the argmin
     * compares the candidates on paired worlds. */
    const int32_t *cand[3] = {BL, BU, BR};
    int32_t ncand[3] = {res->nBL, res->nBU, res->nBR};
    int use[3] = {do_L, do_U, do_R};
    int32_t best = -1;
    for (int32_t c = 0; c < 3; ++c) {
        res->I_after[c] = 0.0;
        if (!use[c]) continue;
        double Ia = 0.0;
        res->n_final[c] = stop_rule(g, S, nS, cand[c], ncand[c], gamma, delta, key,
                                    5u, inst, &Ia, NULL, NULL);
        res->I_after[c] = Ia;
        if (best < 0 || Ia < res->I_after[best]) best = c;
    }
    res->chosen = best;
    res->n_blockers = ncand[best];
    for (int32_t t = 0; t < ncand[best]; ++t) blockers[t] = cand[best][t];
    if (do_U && variant == OV_SANDIMIN && res->DU_hat > 0.0) {
        double gr = (1.0 - gamma) * (1.0 - gamma) / ((1.0 + gamma) * (1.0 + gamma));
        res->ratio_lb = gr * one_m_inv_e_m_eps * (I_hat - res->I_after[1]) / res->DU_hat;
    }

    free(Btmp); free(cov); free(topk); free(inB); free(Vs);
    free(byq); free(bys); free(prod); free(ON); free(inON); free(S);
    work_free(w);
    return 0;
}

/* ====================================================================== */
/* The dominator-tree baselines of Xie et al. as the paper describes them   */
/* (Sec. 2.3): the estimate of D_s(v | B) is the average size of v's        */
/* subtree in the dominator tree of a live-edge world of G[V \ B] (Example */
/* 2.1).  AdvancedGreedy adds the best node k times.  GreedyReplace first   */
/* fills B from the seeds' out-neighbours (up to min(d_out, k) nodes), then */
/* takes the blockers out in reverse insertion order, each time putting     */
/* back the best node of V \ S, and returns as soon as the node put back is */
/* the one taken out.                                                       */
/* Readings: every estimate draws theta new worlds, estimate number c using */
/* worlds [c theta, (c+1) theta) of stream tag 8 (which no solve uses);     */
/* ties go to the smaller node id; no node is added when every estimate is  */
/* zero.  The second stage walks the blockers of the first stage, newest    */
/* first.                                                                   */
/* ====================================================================== */
#define BASELINE_TAG 8u

/* summed subtree sizes of every node over theta worlds of G[V \ B] */
static void dt_estimate(const OGraph *g, const int32_t *S, int32_t nS, const int32_t *B, int32_t nB,
                        uint64_t theta, uint64_t key, uint64_t call, uint64_t *est)
{
    Work *w = work_new(g, S, nS, B, nB);
    SetColl cp;
    coll_init(&cp);
    memset(est, 0, sizeof(uint64_t) * (size_t)g->n);
    for (uint64_t t = 0; t < theta; ++t) {
        World wd = {NULL, key, call * theta + t, BASELINE_TAG, 0};
        cp.nsets = 0;
        cp.off[0] = 0;
        world_local_sampling(g, w, &wd, S, nS, &cp);
        /* the CP sets containing v are the worlds' nodes in v's subtree */
        for (int64_t p = 0; p < cp.off[cp.nsets]; ++p) est[cp.elem[p]] += 1;
    }
    coll_free(&cp);
    work_free(w);
}

/* the allowed node of largest estimate (smaller id on ties), -1 if all are 0 */
static int32_t best_node(const OGraph *g, const uint64_t *est, const uint8_t *allowed)
{
    int32_t u = -1;
    uint64_t best = 0;
    for (int32_t v = 0; v < g->n; ++v)
        if (allowed[v] && est[v] > best) { best = est[v]; u = v; }
    return u;
}

int32_t oracle_advanced_greedy(const OGraph *g, const int32_t *S, int32_t nS, int32_t k, uint64_t theta,
                               uint64_t key, int32_t *B, int32_t *calls)
{
    uint64_t *est = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)g->n + 1));
    uint8_t *allowed = (uint8_t *)malloc((size_t)g->n + 1);
    int32_t nb = 0, c = 0;
    for (int32_t r = 0; r < k; ++r) {
        dt_estimate(g, S, nS, B, nb, theta, key, (uint64_t)c++, est);
        memset(allowed, 1, (size_t)g->n);
        for (int32_t i = 0; i < nS; ++i) allowed[S[i]] = 0;
        for (int32_t i = 0; i < nb; ++i) allowed[B[i]] = 0;
        int32_t u = best_node(g, est, allowed);
        if (u < 0) break;
        B[nb++] = u;
    }
    *calls = c;
    free(est); free(allowed);
    return nb;
}

int32_t oracle_greedy_replace(const OGraph *g, const int32_t *S, int32_t nS, int32_t k, uint64_t theta,
                              uint64_t key, int32_t *B, int32_t *calls)
{
    int32_t n = g->n;
    uint64_t *est = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    uint8_t *allowed = (uint8_t *)malloc((size_t)n + 1);
    uint8_t *is_seed = (uint8_t *)calloc((size_t)n + 1, 1);
    uint8_t *on = (uint8_t *)calloc((size_t)n + 1, 1);
    int32_t *rest = (int32_t *)malloc(sizeof(int32_t) * ((size_t)k + 1));
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * ((size_t)k + 1));
    for (int32_t i = 0; i < nS; ++i) is_seed[S[i]] = 1;
    int32_t d_out = 0;
    for (int32_t i = 0; i < nS; ++i)
        for (int64_t e = g->row_ptr[S[i]]; e < g->row_ptr[S[i] + 1]; ++e) {
            int32_t v = g->col[e];
            if (g->thr[e] > 0 && !is_seed[v] && !on[v]) { on[v] = 1; d_out++; }
        }
    int32_t c = 0, nb = 0;
    int32_t target = d_out < k ? d_out : k;
    /* stage 1: candidates = out-neighbours of the seeds */
    while (nb < target) {
        dt_estimate(g, S, nS, B, nb, theta, key, (uint64_t)c++, est);
        for (int32_t v = 0; v < n; ++v) allowed[v] = on[v];
        for (int32_t i = 0; i < nb; ++i) allowed[B[i]] = 0;
        int32_t u = best_node(g, est, allowed);
        if (u < 0) break;
        B[nb++] = u;
    }
    /* stage 2: replacement in reverse insertion order */
    for (int32_t i = 0; i < nb; ++i) order[i] = B[nb - 1 - i];
    int32_t nstage1 = nb;
    for (int32_t r = 0; r < nstage1; ++r) {
        int32_t out = order[r];
        int32_t nr = 0;
        for (int32_t i = 0; i < nb; ++i)
            if (B[i] != out) rest[nr++] = B[i];
        dt_estimate(g, S, nS, rest, nr, theta, key, (uint64_t)c++, est);
        for (int32_t v = 0; v < n; ++v) allowed[v] = !is_seed[v];
        for (int32_t i = 0; i < nr; ++i) allowed[rest[i]] = 0;
        int32_t u = best_node(g, est, allowed);
        if (u < 0 || u == out) break;
        for (int32_t i = 0; i < nr; ++i) B[i] = rest[i];
        B[nr] = u;
        nb = nr + 1;
    }
    *calls = c;
    free(est); free(allowed); free(is_seed); free(on); free(rest); free(order);
    return nb;
}

/* size of the result struct, for the binding's layout check */
int32_t oracle_result_size(void) { return (int32_t)sizeof(OResult); }
