// api.cu -- the C ABI (include/imin.h) and the host controller of the solve.
//
// The controller follows Algorithm 1 with LSBM (Algorithm 4), GSBM (Sec. 5.2)
// and LHGA (Sec. 5.3).  Every sampled quantity is an integer produced on the
// device; the host turns integers into the scalars of the stopping rules (the
// same IEEE double operations, in the same order, on every platform).
//
// Readings of the paper that the controller implements:
//   * The spread estimate of Algorithm 4 line 4 (the cited "generalized stopping
//     rule") is the Dagum-Karp-Luby-Ross stopping rule on Z_j = |R_j| / W with
//     W = |V'_s| + |S| (an upper bound of I_phi): Upsilon = 4(e-2) ln(2/delta')/beta^2,
//     Upsilon1 = 1 + (1+beta) Upsilon; worlds are drawn until sum |R_j| >= ceil(Upsilon1 W);
//     the estimate is W Upsilon1 / N.
//   * Pr[s -> v] for v in ON (OPT^L and LHGA) is the direct activation probability
//     q(v) = 1 - prod over seed edges (u, v) of (1 - p_q(u, v)), p_q = thr / 2^24.
//   * deg[v] in LHGA is the out-degree.
//   * theta_0 is rounded down; i_max = max(1, ceil(log2(theta_max / theta_0))).
//   * sigma^L = 0 when neither branch of Algorithm 4 (lines 14-17) applies.
//   * GSBM uses ln C(max(|V'_s| - |S|, k), k).
//   * Max-Coverage breaks ties toward the smaller node id and stops at zero gain.
#include "common.cuh"
#include "greedy.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <numeric>

void build_device_graph(imin_graph *g, const float *h_prob);

namespace {

constexpr double IM_E = 2.718281828459045235360287;

struct EventTimer {
    imin_ctx *ctx;
    cudaEvent_t a = nullptr, b = nullptr;
    explicit EventTimer(imin_ctx *c) : ctx(c)
    {
        IM_CUDA(cudaEventCreate(&a));
        IM_CUDA(cudaEventCreate(&b));
        IM_CUDA(cudaEventRecord(a, ctx->stream));
    }
    double stop()
    {
        IM_CUDA(cudaEventRecord(b, ctx->stream));
        IM_CUDA(cudaEventSynchronize(b));
        float ms = 0.0f;
        IM_CUDA(cudaEventElapsedTime(&ms, a, b));
        return ms;
    }
    ~EventTimer()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

struct Timer {
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double ms() const
    {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

void fail(int code, const std::string &msg) { throw ImError{code, msg}; }

// ---------------------------------------------------------------------------
// Query preparation
// ---------------------------------------------------------------------------
struct Query {
    std::vector<int32_t> S;       // sorted, distinct
    std::vector<int32_t> blocked; // sorted, distinct
    std::vector<uint8_t> is_seed, is_blocked;
    DBuf dS, dseed_bm, dblk_bm, dB, dVs;
    std::vector<int32_t> Vs;      // sorted ascending
    size_t words = 0;
};

void check_nodes(const imin_graph *g, const int32_t *a, int32_t cnt, const char *what,
                 std::vector<int32_t> &out)
{
    if (cnt < 0) fail(IMIN_EINVAL, std::string(what) + ": negative count");
    if (cnt > 0 && !a) fail(IMIN_EINVAL, std::string(what) + ": NULL array");
    out.assign(a, a + cnt);
    for (int32_t v : out)
        if (v < 0 || v >= g->n) fail(IMIN_EINVAL, std::string(what) + ": node id out of range");
    std::sort(out.begin(), out.end());
    if (std::adjacent_find(out.begin(), out.end()) != out.end())
        fail(IMIN_EINVAL, std::string(what) + ": duplicate node ids");
}

// V'_s: nodes reachable from S in G[V \ blocked] over edges with p > 0, minus S.
void compute_Vs(const imin_graph *g, Query &q)
{
    const int32_t n = g->n;
    std::vector<uint8_t> mark(n, 0);
    std::vector<int32_t> queue;
    queue.reserve(1024);
    for (int32_t s : q.S) {
        mark[s] = 1;
        queue.push_back(s);
    }
    for (size_t h = 0; h < queue.size(); ++h) {
        const int32_t u = queue[h];
        for (int32_t e = g->h_row_ptr[u]; e < g->h_row_ptr[u + 1]; ++e) {
            const int32_t v = g->h_col[e];
            if (g->h_thr[e] == 0 || mark[v] || q.is_blocked[v]) continue;
            mark[v] = 1;
            queue.push_back(v);
        }
    }
    q.Vs.clear();
    for (int32_t v = 0; v < n; ++v)
        if (mark[v] && !q.is_seed[v]) q.Vs.push_back(v);
}

void prepare_query(imin_ctx *ctx, const imin_graph *g, Query &q, const int32_t *S, int32_t nS,
                   const int32_t *B, int32_t nB, bool need_vs)
{
    if (nS < 1) fail(IMIN_EINVAL, "empty seed set");
    check_nodes(g, S, nS, "seed set", q.S);
    check_nodes(g, B, nB, "blocked set", q.blocked);
    q.is_seed.assign(g->n, 0);
    q.is_blocked.assign(g->n, 0);
    for (int32_t s : q.S) q.is_seed[s] = 1;
    for (int32_t b : q.blocked) {
        if (q.is_seed[b]) fail(IMIN_EINVAL, "a blocked node is a seed");
        q.is_blocked[b] = 1;
    }
    q.words = ((size_t)g->n + 31) / 32;
    cudaStream_t st = ctx->stream;
    q.dS.ensure(ctx, q.S.size() * 4 + 16);
    IM_CUDA(cudaMemcpyAsync(q.dS.p, q.S.data(), q.S.size() * 4, cudaMemcpyHostToDevice, st));
    q.dseed_bm.ensure(ctx, q.words * 4);
    fill_bitmap(ctx, q.dseed_bm.as<uint32_t>(), q.words, q.dS.as<int32_t>(), (int32_t)q.S.size());
    if (!q.blocked.empty()) {
        q.dB.ensure(ctx, q.blocked.size() * 4);
        IM_CUDA(cudaMemcpyAsync(q.dB.p, q.blocked.data(), q.blocked.size() * 4,
                                cudaMemcpyHostToDevice, st));
        q.dblk_bm.ensure(ctx, q.words * 4);
        fill_bitmap(ctx, q.dblk_bm.as<uint32_t>(), q.words, q.dB.as<int32_t>(),
                    (int32_t)q.blocked.size());
    }
    if (need_vs) {
        compute_Vs(g, q);
        q.dVs.ensure(ctx, q.Vs.size() * 4 + 16);
        if (!q.Vs.empty())
            IM_CUDA(cudaMemcpyAsync(q.dVs.p, q.Vs.data(), q.Vs.size() * 4, cudaMemcpyHostToDevice, st));
    }
    IM_CUDA(cudaStreamSynchronize(st));
}

QueryDev qdev(const Query &q, uint64_t key, uint32_t tag, uint32_t inst)
{
    QueryDev d;
    d.S = q.dS.as<int32_t>();
    d.nS = (int32_t)q.S.size();
    d.seed_bm = q.dseed_bm.as<uint32_t>();
    d.blocked_bm = q.blocked.empty() ? nullptr : q.dblk_bm.as<uint32_t>();
    d.B = q.blocked.empty() ? nullptr : q.dB.as<int32_t>();
    d.nB = (int32_t)q.blocked.size();
    d.Vs = q.Vs.empty() ? nullptr : q.dVs.as<int32_t>();
    d.nVs = (int32_t)q.Vs.size();
    d.key = key;
    d.tag = tag;
    d.inst = inst;
    return d;
}

// ---------------------------------------------------------------------------
// Task runner: one persistent launch over several tasks, then the deferred
// worlds (store room after growth on normal slots, oversized worlds on large
// slots) until none is left.
// ---------------------------------------------------------------------------
struct TaskRun {
    const imin_graph *g = nullptr;
    QueryDev q;
    uint64_t first = 0;
    uint32_t count = 0;
    WorldOut out;
    std::function<void(uint32_t)> grow;   // enlarge the task's store for nd worlds; updates out
    unsigned long long acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t claimed_main = 0;
};

constexpr size_t CTL = 128;   // per-task control block: acc[8] | n_deferred | err

struct Runner {
    imin_ctx *ctx;
    double kernel_ms = 0.0;   // device time of the world-kernel launches (CUDA events)
    int launches = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    DBuf ctl, cd, dtasks, defer, lists;

    explicit Runner(imin_ctx *c) : ctx(c)
    {
        IM_CUDA(cudaEventCreate(&ev0));
        IM_CUDA(cudaEventCreate(&ev1));
    }
    ~Runner()
    {
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }

    SlotCfg cfg_for(uint32_t flags, int32_t n, int64_t m, int32_t nS, bool big) const
    {
        SlotCfg c;
        c.lower = (flags & WF_LOWER) != 0;
        c.upper = (flags & WF_UPPER) != 0;
        c.bm_words = ((size_t)n + 31) / 32;
        c.groups_per_lane = 2;
        if (const char *env = std::getenv("IMIN_GROUPS_PER_LANE")) {
            const long v = std::strtol(env, nullptr, 10);
            if (v == 1 || v == 2 || v == 4) c.groups_per_lane = (int)v;
        }
        if (big) {
            c.qcap = n + 1;
            c.ecap = (int32_t)std::min<int64_t>(std::max<int64_t>(m, 1), 4 * ((int64_t)n + 1));
            c.warps = 256;
        } else {
            int32_t q = c.lower ? (1 << 19) : (1 << 18);
            // test hook: IMIN_SLOT_QCAP shrinks the per-warp queue so that the
            // deferred-world path (large slots) is exercised on small graphs
            if (const char *env = std::getenv("IMIN_SLOT_QCAP")) {
                const long v = std::strtol(env, nullptr, 10);
                if (v > 0 && v < q) q = (int32_t)v;
            }
            c.qcap = std::min<int32_t>(n + 1, std::max<int32_t>(q, nS + 1));
            c.ecap = c.lower ? (int32_t)std::min<int64_t>(std::max<int64_t>(m, 1), 2 * (int64_t)c.qcap) : 0;
            int per_sm = c.lower ? 8 : 32;
            // tuning hook: IMIN_SLOT_WARPS_PER_SM overrides the resident warps per SM
            if (const char *env = std::getenv("IMIN_SLOT_WARPS_PER_SM")) {
                const long v = std::strtol(env, nullptr, 10);
                if (v >= 1 && v <= 64) per_sm = (int)v;
            }
            // never more warps than can be resident at once (the kernel is persistent)
            per_sm = std::min(per_sm, 8 * world_kernel_blocks_per_sm(flags, c.groups_per_lane));
            c.warps = ctx->num_sms * per_sm;
        }
        // never use more than half of the free device memory for slots
        size_t freeb = 0, totalb = 0;
        cudaMemGetInfo(&freeb, &totalb);
        size_t avail = freeb / 2;
        if (ctx->budget)
            avail = std::min(avail, ctx->budget > ctx->in_use ? (ctx->budget - ctx->in_use) / 2 : 0);
        const size_t per = c.bytes_per_slot();
        size_t maxw = per ? avail / per : 0;
        maxw = maxw / 8 * 8;
        if ((size_t)c.warps > maxw) c.warps = (int)maxw;
        if (c.warps < 8) {
            if (per * 8 > freeb) fail(IMIN_ENOMEM, "not enough device memory for sampling slots");
            c.warps = 8;
        }
        return c;
    }

    // Slot bitmaps must start clear; the kernel leaves them clear after every world,
    // so the arena is only wiped when its layout changes.
    void prepare_slots(DBuf &arena, const SlotCfg &cfg, size_t &layout)
    {
        const size_t bytes = cfg.bytes_per_slot() * (size_t)cfg.warps;
        const size_t key = cfg.bytes_per_slot() * 1315423911u + (size_t)cfg.warps;
        const void *before = arena.p;
        if (arena.p && arena.bytes < bytes) arena.release();   // never hold two arenas at once
        arena.ensure(ctx, bytes, false, true);
        if (arena.p != before || layout != key) {
            IM_CUDA(cudaMemsetAsync(arena.p, 0, arena.bytes, ctx->stream));
            layout = key;
        }
    }

    void launch(const std::vector<WTask> &ht, const imin_graph *g0, uint32_t flags,
                const SlotCfg &cfg, DBuf &arena)
    {
        const int n = (int)ht.size();
        dtasks.ensure(ctx, ht.size() * sizeof(WTask));
        cd.ensure(ctx, (size_t)n * 8 + 16);
        IM_CUDA(cudaMemcpyAsync(dtasks.p, ht.data(), ht.size() * sizeof(WTask), cudaMemcpyHostToDevice,
                                ctx->stream));
        IM_CUDA(cudaMemsetAsync(cd.p, 0, (size_t)n * 8, ctx->stream));
        IM_CUDA(cudaEventRecord(ev0, ctx->stream));
        launch_tasks(ctx, dtasks.as<WTask>(), n, g0, flags, cfg, arena.p, cd.as<uint32_t>(),
                     cd.as<uint32_t>() + n);
        IM_CUDA(cudaEventRecord(ev1, ctx->stream));
        IM_CUDA(cudaEventSynchronize(ev1));
        float ms = 0.0f;
        IM_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
        kernel_ms += ms;
        ++launches;
    }

    void run(std::vector<TaskRun *> &T, uint32_t flags)
    {
        const int n = (int)T.size();
        if (n == 0) return;
        ctl.ensure(ctx, (size_t)n * CTL);
        IM_CUDA(cudaMemsetAsync(ctl.p, 0, (size_t)n * CTL, ctx->stream));
        std::vector<size_t> doff(n + 1, 0);
        int32_t nmax = 1, nSmax = 1;
        int64_t mmax = 1;
        for (int i = 0; i < n; ++i) {
            doff[i + 1] = doff[i] + T[i]->count;
            nmax = std::max(nmax, T[i]->g->n);
            mmax = std::max(mmax, T[i]->g->m);
            nSmax = std::max(nSmax, T[i]->q.nS);
        }
        defer.ensure(ctx, doff[n] * 4 + 16);
        char *c0 = reinterpret_cast<char *>(ctl.p);
        for (int i = 0; i < n; ++i) {
            WorldOut &o = T[i]->out;
            o.acc = reinterpret_cast<unsigned long long *>(c0 + (size_t)i * CTL);
            o.n_deferred = reinterpret_cast<uint32_t *>(c0 + (size_t)i * CTL + 64);
            o.err = reinterpret_cast<uint32_t *>(c0 + (size_t)i * CTL + 68);
            o.deferred = defer.as<uint32_t>() + doff[i];
            o.deferred_cap = T[i]->count;
        }
        SlotCfg cfg = cfg_for(flags, nmax, mmax, nSmax, false);
        DBuf &arena = cfg.lower ? ctx->slots_lower : ctx->slots;
        size_t &layout = cfg.lower ? ctx->slots_lower_layout : ctx->slots_layout;
        prepare_slots(arena, cfg, layout);
        std::vector<WTask> ht;
        for (int i = 0; i < n; ++i)
            ht.push_back(make_task(T[i]->g, T[i]->q, T[i]->first, T[i]->count, nullptr, T[i]->out));
        launch(ht, T[0]->g, flags, cfg, arena);
        std::vector<unsigned char> hc((size_t)n * CTL);
        std::vector<uint32_t> claims(n);
        IM_CUDA(cudaMemcpy(claims.data(), cd.p, (size_t)n * 4, cudaMemcpyDeviceToHost));
        IM_CUDA(cudaMemcpy(hc.data(), ctl.p, hc.size(), cudaMemcpyDeviceToHost));
        for (int i = 0; i < n; ++i) T[i]->claimed_main = std::min(claims[i], T[i]->count);
        check_err(hc, n);
        std::vector<uint32_t> h_def;
        for (int rounds = 0;; ++rounds) {
            std::vector<uint32_t> nd(n);
            bool any = false;
            for (int i = 0; i < n; ++i) {
                std::memcpy(&nd[i], hc.data() + (size_t)i * CTL + 64, 4);
                any |= nd[i] > 0;
            }
            if (!any) break;
            if (rounds > 40) fail(IMIN_ERANGE, "worlds could not be stored after repeated growth");
            // worlds flagged in the top bit overflowed their slot and need a large slot;
            // the others only lacked store room and re-run on normal slots
            std::vector<std::vector<uint32_t>> small(n), big(n);
            for (int i = 0; i < n; ++i) {
                if (!nd[i]) continue;
                if (T[i]->grow) T[i]->grow(nd[i]);
                h_def.resize(nd[i]);
                IM_CUDA(cudaMemcpy(h_def.data(), defer.as<uint32_t>() + doff[i], (size_t)nd[i] * 4,
                                   cudaMemcpyDeviceToHost));
                for (uint32_t x : h_def)
                    ((x & 0x80000000u) ? big[i] : small[i]).push_back(x & 0x7fffffffu);
                IM_CUDA(cudaMemsetAsync(c0 + (size_t)i * CTL + 64, 0, 4, ctx->stream));
            }
            for (int pass = 0; pass < 2; ++pass) {
                std::vector<std::vector<uint32_t>> &L = pass == 0 ? small : big;
                size_t tot = 0;
                for (int i = 0; i < n; ++i) tot += L[i].size();
                if (!tot) continue;
                lists.ensure(ctx, tot * 4);
                std::vector<WTask> lt;
                size_t at = 0;
                for (int i = 0; i < n; ++i) {
                    if (L[i].empty()) continue;
                    IM_CUDA(cudaMemcpy(lists.as<uint32_t>() + at, L[i].data(), L[i].size() * 4,
                                       cudaMemcpyHostToDevice));
                    lt.push_back(make_task(T[i]->g, T[i]->q, T[i]->first, (uint32_t)L[i].size(),
                                           lists.as<uint32_t>() + at, T[i]->out));
                    at += L[i].size();
                }
                if (pass == 0) {
                    launch(lt, T[0]->g, flags, cfg, arena);
                } else {
                    SlotCfg bc = cfg_for(flags, nmax, mmax, nSmax, true);
                    prepare_slots(ctx->big_slots, bc, ctx->big_slots_layout);
                    launch(lt, T[0]->g, flags, bc, ctx->big_slots);
                }
            }
            IM_CUDA(cudaMemcpy(hc.data(), ctl.p, hc.size(), cudaMemcpyDeviceToHost));
            check_err(hc, n);
        }
        for (int i = 0; i < n; ++i) std::memcpy(T[i]->acc, hc.data() + (size_t)i * CTL, 64);
    }

    void check_err(const std::vector<unsigned char> &hc, int n)
    {
        uint32_t e = 0;
        for (int i = 0; i < n; ++i) {
            uint32_t x;
            std::memcpy(&x, hc.data() + (size_t)i * CTL + 68, 4);
            e |= x;
        }
        if (e & DERR_TIMEOUT) fail(IMIN_ETIMEOUT, "a bounded device loop gave up");
        if (e & DERR_INTERNAL) fail(IMIN_EDEVICE, "device invariant failed");
    }
};

// ---------------------------------------------------------------------------
// Stopping-rule spread estimates (reach-only worlds with early exit), several
// queries in one launch
// ---------------------------------------------------------------------------
struct SpreadEst {
    double I = 0.0;
    uint64_t N = 0;
    uint64_t worlds = 0, edges = 0, nodes = 0, launches = 0;
    double kernel_ms = 0.0;
};

struct StopSpec {
    const imin_graph *g;
    const Query *q;
    double beta, dprime;
    uint64_t key;
    uint32_t tag, inst;
    SpreadEst est;
};

void stop_rules(imin_ctx *ctx, std::vector<StopSpec> &specs)
{
    const size_t ns = specs.size();
    std::vector<TaskRun> tr(ns);
    std::vector<TaskRun *> tp;
    std::vector<DBuf> spread(ns);
    std::vector<double> W(ns), ups1(ns);
    std::vector<unsigned long long> T(ns);
    for (size_t i = 0; i < ns; ++i) {
        StopSpec &sp = specs[i];
        W[i] = (double)sp.q->Vs.size() + (double)sp.q->S.size();
        const double ups = 4.0 * (IM_E - 2.0) * std::log(2.0 / sp.dprime) / (sp.beta * sp.beta);
        ups1[i] = 1.0 + (1.0 + sp.beta) * ups;
        const double Td = std::ceil(ups1[i] * W[i]);
        if (!(Td < 1.8e19)) fail(IMIN_ERANGE, "stopping threshold too large");
        T[i] = (unsigned long long)Td;
        // every world reaches at least |S| nodes, so N <= ceil(T / |S|)
        const uint64_t nmax = (T[i] + sp.q->S.size() - 1) / sp.q->S.size();
        if (nmax >= ((uint64_t)1 << 31)) fail(IMIN_ERANGE, "the stopping rule may need >= 2^31 worlds");
        spread[i].ensure(ctx, (size_t)nmax * 4 + 16);
        tr[i].g = sp.g;
        tr[i].q = qdev(*sp.q, sp.key, sp.tag, sp.inst);
        tr[i].first = 0;
        tr[i].count = (uint32_t)nmax;
        tr[i].out.world_spread = spread[i].as<uint32_t>();
        tr[i].out.stop_T = T[i];
        tp.push_back(&tr[i]);
    }
    Runner run(ctx);
    run.run(tp, WF_STOP | WF_SPREAD);
    for (size_t i = 0; i < ns; ++i) {
        // every claimed world is complete (deferred ones were re-run), and the worlds
        // below the last claimed index hold at least T reached nodes in total
        const uint64_t want = tr[i].claimed_main;
        std::vector<uint32_t> sizes(want);
        if (want) IM_CUDA(cudaMemcpy(sizes.data(), spread[i].p, want * 4, cudaMemcpyDeviceToHost));
        unsigned long long sum = 0;
        uint64_t N = 0;
        for (uint64_t j = 0; j < want; ++j) {
            sum += sizes[j];
            if (sum >= T[i]) {
                N = j + 1;
                break;
            }
        }
        if (N == 0) fail(IMIN_EDEVICE, "stopping rule: threshold not reached by the traversed worlds");
        SpreadEst &r = specs[i].est;
        r.N = N;
        r.I = W[i] * ups1[i] / (double)N;
        r.worlds = tr[i].acc[4];
        r.edges = tr[i].acc[1];
        r.nodes = tr[i].acc[0];
    }
    // device time is shared by the tasks of the launch: report it on the first
    specs[0].est.kernel_ms = run.kernel_ms;
    specs[0].est.launches = (uint64_t)run.launches;
}

SpreadEst stop_rule(imin_ctx *ctx, const imin_graph *g, const Query &q, double beta, double dprime,
                    uint64_t key, uint32_t tag, uint32_t inst)
{
    std::vector<StopSpec> v{StopSpec{g, &q, beta, dprime, key, tag, inst, SpreadEst{}}};
    stop_rules(ctx, v);
    return v[0].est;
}

// ---------------------------------------------------------------------------
// Collections: CP records (C1, C2) and LRR sets (L1, L2), appended together
// ---------------------------------------------------------------------------
void cp_reserve(imin_ctx *ctx, CpStore &c, unsigned long long need)
{
    if (need <= c.cap && c.node.p) return;
    unsigned long long cap = std::max<unsigned long long>(need, c.cap + c.cap / 2);
    cap = std::max<unsigned long long>(cap, 1024);
    c.node.ensure(ctx, cap * 4, true);
    c.par.ensure(ctx, cap * 4, true);
    c.size.ensure(ctx, cap * 4, true);
    c.cap = cap;
}

struct CpJob {
    CpStore *c;
    uint32_t tag;
    unsigned long long *credit;   // may be null
};

// append worlds [from, to) of each job's tag to its CP collection, one launch for all jobs
void sample_cp(imin_ctx *ctx, const imin_graph *g, const Query &q, std::vector<CpJob> &jobs,
               uint64_t from, uint64_t to, uint64_t key, uint32_t inst, double est_per_world,
               SpreadEst *stats)
{
    if (to <= from) return;
    if (to > ((uint64_t)1 << 31)) fail(IMIN_ERANGE, "world index >= 2^31");
    const size_t nj = jobs.size();
    std::vector<TaskRun> tr(nj);
    std::vector<TaskRun *> tp;
    std::vector<unsigned long long> before(nj);
    for (size_t i = 0; i < nj; ++i) {
        CpStore &c = *jobs[i].c;
        c.cursor.ensure(ctx, 16);
        if (c.worlds == 0) {
            IM_CUDA(cudaMemsetAsync(c.cursor.p, 0, 8, ctx->stream));
            c.count = 0;
        }
        const unsigned long long est =
            (unsigned long long)((double)(to - from) * std::max(est_per_world, 1.0) * 1.25) + 4096;
        cp_reserve(ctx, c, (unsigned long long)c.count + est);
        before[i] = (unsigned long long)c.count;
        TaskRun &t = tr[i];
        t.g = g;
        t.q = qdev(q, key, jobs[i].tag, inst);
        t.first = from;
        t.count = (uint32_t)(to - from);
        t.out.credit_L = jobs[i].credit;
        t.out.rec_node = c.node.as<int32_t>();
        t.out.rec_par = c.par.as<int32_t>();
        t.out.rec_size = c.size.as<int32_t>();
        t.out.rec_cursor = c.cursor.as<unsigned long long>();
        t.out.rec_cap = c.cap;
        CpStore *cp = &c;
        TaskRun *self = &t;
        const unsigned long long b0 = before[i];
        t.grow = [ctx, cp, self, b0, from, to, g](uint32_t nd) {
            unsigned long long used = 0;
            IM_CUDA(cudaMemcpy(&used, cp->cursor.p, 8, cudaMemcpyDeviceToHost));
            const uint64_t worlds = (to - from) > nd ? (to - from) - nd : 1;
            const unsigned long long avg = (used - b0) / worlds + 1;
            cp_reserve(ctx, *cp, std::max<unsigned long long>(
                                     2 * cp->cap, used + (unsigned long long)nd * 2 * avg + (unsigned long long)g->n));
            self->out.rec_node = cp->node.as<int32_t>();
            self->out.rec_par = cp->par.as<int32_t>();
            self->out.rec_size = cp->size.as<int32_t>();
            self->out.rec_cap = cp->cap;
        };
        tp.push_back(&t);
    }
    Runner run(ctx);
    run.run(tp, WF_LOWER | WF_STORE);
    for (size_t i = 0; i < nj; ++i) {
        CpStore &c = *jobs[i].c;
        unsigned long long used = 0;
        IM_CUDA(cudaMemcpy(&used, c.cursor.p, 8, cudaMemcpyDeviceToHost));
        c.count = (long long)used;
        c.worlds += to - from;
        if (stats) {
            stats->worlds += tr[i].acc[4];
            stats->edges += tr[i].acc[1];
            stats->nodes += tr[i].acc[0];
        }
    }
    if (stats) {
        stats->kernel_ms += run.kernel_ms;
        stats->launches += (uint64_t)run.launches;
    }
}

void lrr_reserve(imin_ctx *ctx, LrrStore &L, unsigned long long need_elems, uint64_t need_worlds)
{
    if (!(need_elems <= L.cap && L.elem.p)) {
        unsigned long long cap = std::max<unsigned long long>(need_elems, L.cap + L.cap / 2);
        cap = std::max<unsigned long long>(cap, 1024);
        L.elem.ensure(ctx, cap * 4, true);
        L.cap = cap;
    }
    if (need_worlds > L.worlds_cap || !L.off.p) {
        uint64_t wc = std::max<uint64_t>(need_worlds, L.worlds_cap * 2);
        wc = std::max<uint64_t>(wc, 1024);
        L.off.ensure(ctx, wc * 8, true);
        L.len.ensure(ctx, wc * 4, true);
        L.worlds_cap = wc;
    }
}

struct LrrJob {
    LrrStore *L;
    uint32_t tag;
    unsigned long long *credit;   // may be null
};

void sample_lrr(imin_ctx *ctx, const imin_graph *g, const Query &q, std::vector<LrrJob> &jobs,
                uint64_t from, uint64_t to, uint64_t key, uint32_t inst, SpreadEst *stats)
{
    if (to <= from) return;
    if (to > ((uint64_t)1 << 31)) fail(IMIN_ERANGE, "world index >= 2^31");
    const size_t nj = jobs.size();
    std::vector<TaskRun> tr(nj);
    std::vector<TaskRun *> tp;
    for (size_t i = 0; i < nj; ++i) {
        LrrStore &L = *jobs[i].L;
        L.cursor.ensure(ctx, 16);
        if (L.nsets == 0) {
            IM_CUDA(cudaMemsetAsync(L.cursor.p, 0, 8, ctx->stream));
            L.elems = 0;
        }
        // start from the average set size seen so far (64 per world before any is known)
        const unsigned long long per = L.nsets ? L.elems / L.nsets + 1 : 64;
        lrr_reserve(ctx, L, L.elems + (to - from) * per * 2 + 65536, to);
        TaskRun &t = tr[i];
        t.g = g;
        t.q = qdev(q, key, jobs[i].tag, inst);
        t.first = from;
        t.count = (uint32_t)(to - from);
        t.out.credit_U = jobs[i].credit;
        t.out.set_elem = L.elem.as<int32_t>();
        t.out.set_off = L.off.as<unsigned long long>() + from;
        t.out.set_len = L.len.as<uint32_t>() + from;
        t.out.set_cursor = L.cursor.as<unsigned long long>();
        t.out.set_cap = L.cap;
        LrrStore *lp = &L;
        TaskRun *self = &t;
        t.grow = [ctx, lp, self, from, to, g](uint32_t nd) {
            unsigned long long used = 0;
            IM_CUDA(cudaMemcpy(&used, lp->cursor.p, 8, cudaMemcpyDeviceToHost));
            lrr_reserve(ctx, *lp, std::max<unsigned long long>(
                                      2 * lp->cap, used + (unsigned long long)nd * (unsigned long long)g->n), to);
            self->out.set_elem = lp->elem.as<int32_t>();
            self->out.set_off = lp->off.as<unsigned long long>() + from;
            self->out.set_len = lp->len.as<uint32_t>() + from;
            self->out.set_cap = lp->cap;
        };
        tp.push_back(&t);
    }
    Runner run(ctx);
    run.run(tp, WF_UPPER | WF_STORE);
    for (size_t i = 0; i < nj; ++i) {
        LrrStore &L = *jobs[i].L;
        unsigned long long used = 0;
        IM_CUDA(cudaMemcpy(&used, L.cursor.p, 8, cudaMemcpyDeviceToHost));
        L.elems = used;
        L.nsets = (uint32_t)to;
        if (stats) {
            stats->worlds += tr[i].acc[4];
            stats->edges += tr[i].acc[1];
            stats->nodes += tr[i].acc[0];
        }
    }
    if (stats) {
        stats->kernel_ms += run.kernel_ms;
        stats->launches += (uint64_t)run.launches;
    }
}

double ln_binom(double a, double b) { return std::lgamma(a + 1.0) - std::lgamma(b + 1.0) - std::lgamma(a - b + 1.0); }

double sigma_low(double x, double a, double theta)
{
    const double r = std::sqrt(x + 2.0 * a / 9.0) - std::sqrt(a / 2.0);
    return (r * r - a / 18.0) / theta;
}

double sigma_up(double y, double a, double theta)
{
    const double r = std::sqrt(y + a / 2.0) + std::sqrt(a / 2.0);
    return r * r / theta;
}

struct ScoreItem {
    double score;
    int32_t v;
};

bool score_desc(const ScoreItem &x, const ScoreItem &y)
{
    if (x.score != y.score) return x.score > y.score;
    return x.v < y.v;
}

void set_bitmap_host(imin_ctx *ctx, DBuf &bm, size_t words, const std::vector<int32_t> &nodes)
{
    std::vector<uint32_t> h(words, 0);
    for (int32_t v : nodes) h[v >> 5] |= 1u << (v & 31);
    bm.ensure(ctx, words * 4);
    IM_CUDA(cudaMemcpy(bm.p, h.data(), words * 4, cudaMemcpyHostToDevice));
}

struct GreedyOut {
    std::vector<int32_t> B;
    std::vector<unsigned long long> cov, topk;
    unsigned long long covu = 0;
};

GreedyOut read_greedy(imin_ctx *ctx, GreedyBufs &gb, int32_t k)
{
    GState st;
    IM_CUDA(cudaMemcpyAsync(&st, gb.state.p, sizeof(GState), cudaMemcpyDeviceToHost, ctx->stream));
    IM_CUDA(cudaStreamSynchronize(ctx->stream));
    GreedyOut o;
    const int nb = st.nb;
    o.B.resize(nb);
    o.cov.resize(nb + 1);
    o.topk.resize(nb + 1);
    if (nb > 0) IM_CUDA(cudaMemcpy(o.B.data(), gb.B.p, (size_t)nb * 4, cudaMemcpyDeviceToHost));
    IM_CUDA(cudaMemcpy(o.cov.data(), gb.cov.p, (size_t)(nb + 1) * 8, cudaMemcpyDeviceToHost));
    IM_CUDA(cudaMemcpy(o.topk.data(), gb.topk.p, (size_t)(nb + 1) * 8, cudaMemcpyDeviceToHost));
    o.covu = o.cov[0] + o.topk[0];
    for (int t = 1; t <= nb; ++t) o.covu = std::min(o.covu, o.cov[t] + o.topk[t]);
    (void)k;
    return o;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

namespace {
int run_guarded(imin_ctx *ctx, const std::function<void()> &f)
{
    try {
        f();
        return IMIN_OK;
    } catch (const ImError &e) {
        if (ctx) ctx->last_error = e.msg;
        if (e.code == IMIN_EDEVICE && ctx) cudaGetLastError();
        return e.code;
    } catch (const std::bad_alloc &) {
        if (ctx) ctx->last_error = "host allocation failed";
        return IMIN_ENOMEM;
    } catch (...) {
        if (ctx) ctx->last_error = "unknown error";
        return IMIN_EDEVICE;
    }
}
}  // namespace

extern "C" {

const char *imin_strerror(int status)
{
    switch (status) {
    case IMIN_OK: return "ok";
    case IMIN_EINVAL: return "invalid argument";
    case IMIN_ERANGE: return "size out of supported range";
    case IMIN_ENOMEM: return "out of device memory or over budget";
    case IMIN_EDEVICE: return "CUDA device error";
    case IMIN_ETIMEOUT: return "bounded device wait expired";
    default: return "unknown status";
    }
}

void imin_last_error(imin_ctx *ctx, char *buf, size_t len)
{
    if (!buf || len == 0) return;
    const std::string &m = ctx ? ctx->last_error : std::string();
    const size_t c = std::min(len - 1, m.size());
    std::memcpy(buf, m.data(), c);
    buf[c] = 0;
}

int imin_create(imin_ctx **out, int device, size_t device_mem_budget, void *stream)
{
    if (!out) return IMIN_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return IMIN_EDEVICE;
    }
    if (device < 0 || device >= ndev) return IMIN_EINVAL;
    imin_ctx *ctx = new (std::nothrow) imin_ctx();
    if (!ctx) return IMIN_ENOMEM;
    ctx->device = device;
    ctx->budget = device_mem_budget;
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
    int rc = run_guarded(ctx, [&] {
        IM_CUDA(cudaSetDevice(device));
        IM_CUDA(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
    });
    if (rc != IMIN_OK) {
        delete ctx;
        return rc;
    }
    *out = ctx;
    return IMIN_OK;
}

void imin_destroy(imin_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->persist_set) {
        cudaCtxResetPersistingL2Cache();
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, ctx->prev_persist_limit);
        cudaGetLastError();
    }
    ctx->slots.release();
    ctx->slots_lower.release();
    ctx->big_slots.release();
    ctx->misc.release();
    delete ctx;
}

int imin_load_graph(imin_ctx *ctx, int32_t n, int64_t m, const int32_t *row_ptr,
                    const int32_t *col, const float *prob, imin_graph **out)
{
    if (!ctx || !out) return IMIN_EINVAL;
    *out = nullptr;
    imin_graph *g = nullptr;
    int rc = run_guarded(ctx, [&] {
        IM_CUDA(cudaSetDevice(ctx->device));
        if (n < 1 || n >= 0x7fffffff - 1) fail(n < 1 ? IMIN_EINVAL : IMIN_ERANGE, "n out of range");
        if (m < 0) fail(IMIN_EINVAL, "negative m");
        if (m >= (int64_t)0x7fffffff - 4) fail(IMIN_ERANGE, "m >= 2^31 - 4");
        if (!row_ptr || (m > 0 && (!col || !prob))) fail(IMIN_EINVAL, "NULL array");
        if (row_ptr[0] != 0 || (int64_t)row_ptr[n] != m) fail(IMIN_EINVAL, "row_ptr must run from 0 to m");
        for (int32_t i = 0; i < n; ++i)
            if (row_ptr[i + 1] < row_ptr[i]) fail(IMIN_EINVAL, "row_ptr not monotone");
        for (int64_t e = 0; e < m; ++e)
            if (col[e] < 0 || col[e] >= n) fail(IMIN_EINVAL, "col out of range");
        for (int64_t e = 0; e < m; ++e) {
            const float p = prob[e];
            if (!(p >= 0.0f && p <= 1.0f)) fail(IMIN_EINVAL, "probability NaN or outside [0, 1]");
        }
        g = new imin_graph();
        g->ctx = ctx;
        g->n = n;
        g->m = m;
        g->m4 = (m + 3) / 4 * 4;
        g->h_row_ptr.assign(row_ptr, row_ptr + n + 1);
        g->h_col.assign(col, col + m);
        g->h_thr.resize(m);
        for (int64_t e = 0; e < m; ++e) {
            double t = std::ceil((double)prob[e] * 16777216.0);
            g->h_thr[e] = (uint32_t)std::min(std::max(t, 0.0), 16777216.0);
        }
        build_device_graph(g, prob);
    });
    if (rc != IMIN_OK) {
        delete g;
        return rc;
    }
    *out = g;
    return IMIN_OK;
}

void imin_free_graph(imin_graph *g)
{
    if (!g) return;
    cudaSetDevice(g->ctx->device);
    delete g;
}

int imin_sample(imin_graph *g, const int32_t *S, int32_t nS, const int32_t *blocked, int32_t nB,
                uint64_t theta, const imin_sample_opts *opts, imin_sample_out *out)
{
    if (!g || !opts || !out) return IMIN_EINVAL;
    imin_ctx *ctx = g->ctx;
    return run_guarded(ctx, [&] {
        IM_CUDA(cudaSetDevice(ctx->device));
        const uint32_t mode = opts->mode;
        if (opts->reserved != 0 || (mode & ~(uint32_t)(IMIN_REACH | IMIN_CREDIT_LOWER |
                                                       IMIN_CREDIT_UPPER | IMIN_OUT_DEVICE)))
            fail(IMIN_EINVAL, "unknown mode bits");
        if (opts->first_sample + theta > ((uint64_t)1 << 32) || theta >= ((uint64_t)1 << 31))
            fail(IMIN_ERANGE, "world index >= 2^32 or theta >= 2^31");
        Query q;
        const bool upper = (mode & IMIN_CREDIT_UPPER) != 0, lower = (mode & IMIN_CREDIT_LOWER) != 0;
        prepare_query(ctx, g, q, S, nS, blocked, nB, upper);
        const int32_t n = g->n;
        const bool dev_out = (mode & IMIN_OUT_DEVICE) != 0;
        cudaStream_t st = ctx->stream;
        DBuf dreach, dcl, dcu, dws;
        unsigned long long *preach = nullptr, *pcl = nullptr, *pcu = nullptr;
        auto dest = [&](uint64_t *user, DBuf &tmp) -> unsigned long long * {
            if (!user) return nullptr;
            unsigned long long *p;
            if (dev_out) {
                p = reinterpret_cast<unsigned long long *>(user);
            } else {
                tmp.ensure(ctx, (size_t)n * 8);
                p = tmp.as<unsigned long long>();
            }
            IM_CUDA(cudaMemsetAsync(p, 0, (size_t)n * 8, st));
            return p;
        };
        if (mode & IMIN_REACH) preach = dest(out->reach, dreach);
        if (lower) pcl = dest(out->credit_lower, dcl);
        if (upper) pcu = dest(out->credit_upper, dcu);
        uint32_t *pws = nullptr;
        if (out->world_spread && theta > 0) {
            if (dev_out) {
                pws = out->world_spread;
            } else {
                dws.ensure(ctx, (size_t)theta * 4);
                pws = dws.as<uint32_t>();
            }
        }
        TaskRun t;
        t.g = g;
        t.q = qdev(q, opts->key, opts->tag, opts->inst);
        t.first = opts->first_sample;
        t.count = (uint32_t)theta;
        t.out.reach = preach;
        t.out.credit_L = pcl;
        t.out.credit_U = pcu;
        t.out.world_spread = pws;
        uint32_t flags = (preach ? WF_REACH : 0u) | (lower ? WF_LOWER : 0u) | (upper ? WF_UPPER : 0u) |
                         (pws ? WF_SPREAD : 0u);
        if (theta > 0) {
            std::vector<TaskRun *> tp{&t};
            Runner run(ctx);
            run.run(tp, flags);
        }
        out->total_spread = t.acc[0];
        out->edges_scanned = t.acc[1];
        out->nonempty_lrr = t.acc[2];
        if (!dev_out) {
            if (preach) IM_CUDA(cudaMemcpyAsync(out->reach, preach, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
            if (pcl) IM_CUDA(cudaMemcpyAsync(out->credit_lower, pcl, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
            if (pcu) IM_CUDA(cudaMemcpyAsync(out->credit_upper, pcu, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
            if (pws) IM_CUDA(cudaMemcpyAsync(out->world_spread, pws, (size_t)theta * 4, cudaMemcpyDeviceToHost, st));
        }
        IM_CUDA(cudaStreamSynchronize(st));
    });
}

int imin_solve(imin_graph *g, const int32_t *S_in, int32_t nS, int32_t k, double eps, double delta,
               const imin_solve_opts *opts, imin_result *res)
{
    if (!g || !opts || !res || !res->blockers) return IMIN_EINVAL;
    imin_ctx *ctx = g->ctx;
    return run_guarded(ctx, [&] {
        Timer total;
        const unsigned long long launches0 = g_kernel_launches;
        IM_CUDA(cudaSetDevice(ctx->device));
        const double beta = opts->beta, gamma = opts->gamma;
        if (!(eps > 0.0 && eps < 1.0) || !(delta > 0.0 && delta < 1.0) || !(beta > 0.0 && beta < 1.0) ||
            !(gamma > 0.0 && gamma < 1.0))
            fail(IMIN_EINVAL, "eps, delta, beta and gamma must lie in (0, 1)");
        if (opts->variant < IMIN_SANDIMIN || opts->variant > IMIN_LHGA) fail(IMIN_EINVAL, "unknown variant");
        const int32_t n = g->n;
        if (k < 1 || (int64_t)k >= (int64_t)n - nS) fail(IMIN_EINVAL, "k must satisfy 1 <= k < n - |S|");
        const uint64_t key = opts->key;
        const uint32_t inst = opts->inst;
        const int variant = opts->variant;
        int32_t *B_L = res->B_L, *B_U = res->B_U, *B_R = res->B_R, *blockers = res->blockers;
        std::memset(res, 0, sizeof(*res));
        res->blockers = blockers;
        res->B_L = B_L;
        res->B_U = B_U;
        res->B_R = B_R;

        Query q;
        prepare_query(ctx, g, q, S_in, nS, nullptr, 0, true);
        const std::vector<int32_t> &S = q.S;
        Timer host_t;
        double host_ms = 0.0;

        // ON: out-neighbours of S with p > 0, not in S (Algorithm 4, line 1)
        std::vector<uint8_t> inON(n, 0);
        for (int32_t s : S)
            for (int32_t e = g->h_row_ptr[s]; e < g->h_row_ptr[s + 1]; ++e)
                if (g->h_thr[e] > 0 && !q.is_seed[g->h_col[e]]) inON[g->h_col[e]] = 1;
        std::vector<int32_t> ON;
        for (int32_t v = 0; v < n; ++v)
            if (inON[v]) ON.push_back(v);
        auto put = [&](int32_t *dst, const std::vector<int32_t> &src) {
            if (dst) std::copy(src.begin(), src.end(), dst);
        };
        if ((int32_t)ON.size() <= k) {   // Algorithm 4, lines 2-3; Sec. 5.3
            put(blockers, ON);
            put(B_L, ON);
            put(B_U, ON);
            put(B_R, ON);
            res->n_blockers = res->nBL = res->nBU = res->nBR = (int32_t)ON.size();
            res->chosen = 0;
            res->nVs = (int32_t)q.Vs.size();
            res->ms_stage[7] = total.ms();
            return;
        }
        // q(v) and OPT^L (Sec. 5.1), LHGA scores (Sec. 5.3)
        std::vector<double> prod(n, 1.0);
        for (int32_t s : S)
            for (int32_t e = g->h_row_ptr[s]; e < g->h_row_ptr[s + 1]; ++e) {
                const int32_t v = g->h_col[e];
                if (!inON[v]) continue;
                const double pq = (double)g->h_thr[e] / 16777216.0;
                prod[v] = prod[v] * (1.0 - pq);
            }
        std::vector<ScoreItem> byq(ON.size()), bys(ON.size());
        for (size_t i = 0; i < ON.size(); ++i) {
            const int32_t v = ON[i];
            const double qv = 1.0 - prod[v];
            byq[i] = {qv, v};
            bys[i] = {qv * (double)(g->h_row_ptr[v + 1] - g->h_row_ptr[v]), v};
        }
        std::sort(byq.begin(), byq.end(), score_desc);
        std::sort(bys.begin(), bys.end(), score_desc);
        double OPT = 0.0;
        for (int32_t i = 0; i < k; ++i) OPT += byq[i].score;
        res->OPT_L = OPT;
        std::vector<int32_t> BRv(k);
        for (int32_t i = 0; i < k; ++i) BRv[i] = bys[i].v;
        const int32_t nVs = (int32_t)q.Vs.size();
        res->nVs = nVs;
        const double one_m_inv_e_m_eps = 1.0 - 1.0 / IM_E - eps;
        host_ms += host_t.ms();

        const bool do_L = variant == IMIN_SANDIMIN || variant == IMIN_SANDIMIN_MINUS || variant == IMIN_LSBM;
        const bool do_U = variant == IMIN_SANDIMIN || variant == IMIN_GSBM;
        const bool do_R = variant == IMIN_SANDIMIN || variant == IMIN_SANDIMIN_MINUS || variant == IMIN_LHGA;
        const size_t words = q.words;
        DBuf d_inB, d_cov;
        d_cov.ensure(ctx, 16);
        unsigned long long h_cov = 0;
        GreedyBufs gb;
        std::vector<int32_t> BLv, BUv;

        // ---- spread estimate (beta, delta/6): Algorithm 4, line 4 ----
        Timer t0;
        SpreadEst I0 = stop_rule(ctx, g, q, beta, delta / 6.0, key, 0, inst);
        const double I_hat = I0.I;
        res->I_hat = I_hat;
        res->n_spread = I0.N;
        res->worlds_sampled += I0.worlds;
        res->edges_scanned += I0.edges;
        res->kernel_ms[0] += I0.kernel_ms;
        res->reach_nodes += I0.nodes;
        res->reach_edges += I0.edges;
        res->reach_launches += I0.launches;
        res->ms_stage[0] = t0.ms();

        // ---- LSBM (Algorithm 4) ----
        if (do_L) {
            Timer ts;
            const double a = 1.0 - 1.0 / IM_E;
            const double l12 = std::log(12.0 / delta);
            const double c1 = a * std::sqrt(l12) + std::sqrt(a * (ln_binom((double)(n - nS), (double)k) + l12));
            const double th_max = 2.0 * I_hat * c1 * c1 / ((1.0 - beta) * eps * eps * OPT);
            double th0d = std::floor(th_max * (1.0 - beta) * eps * eps * OPT / I_hat);
            if (th0d < 1.0) th0d = 1.0;
            int32_t imax = (int32_t)std::ceil(std::log2(th_max / th0d));
            if (imax < 1) imax = 1;
            uint64_t th = (uint64_t)th0d;
            if (opts->fixed_theta) {
                th = opts->fixed_theta;
                imax = 1;
            }
            res->theta_max_L = th_max;
            const double a1 = std::log(3.0 * (double)imax / delta), a2 = a1;
            CpStore C1, C2;
            DBuf credC1;
            credC1.ensure(ctx, (size_t)n * 8);
            IM_CUDA(cudaMemsetAsync(credC1.p, 0, (size_t)n * 8, ctx->stream));
            const double per_world = std::max(I_hat - (double)nS, 1.0);
            SpreadEst st;
            std::vector<CpJob> cj{CpJob{&C1, 1u, credC1.as<unsigned long long>()},
                                  CpJob{&C2, 2u, nullptr}};
            sample_cp(ctx, g, q, cj, 0, th, key, inst, per_world, &st);
            double samp_ms = ts.ms(), greedy_ms = 0.0;
            GreedyOut go;
            double sL = 0.0, sU = 0.0;
            unsigned long long cov2 = 0;
            for (int32_t i = 1; i <= imax; ++i) {
                Timer tg;
                {
                    EventTimer et(ctx);
                    greedy_cp(ctx, gb, C1, n, k, credC1.as<unsigned long long>());
                    res->kernel_ms[3] += et.stop();
                }
                go = read_greedy(ctx, gb, k);
                set_bitmap_host(ctx, d_inB, words, go.B);
                cov2 = cov_cp(ctx, C2, d_inB.as<uint32_t>(), d_cov.as<unsigned long long>(), &h_cov);
                greedy_ms += tg.ms();
                const double xlo = (double)cov2 * (1.0 - beta) / I_hat;
                const double xhi = (double)cov2 * (1.0 + beta) / I_hat;
                sL = 0.0;
                if (xlo >= 5.0 * a1 / 18.0)
                    sL = sigma_low(xlo, a1, (double)C2.worlds);
                else if (xhi <= 5.0 * a1 / 18.0)
                    sL = sigma_low(xhi, a1, (double)C2.worlds);
                sU = sigma_up((double)go.covu * (1.0 + beta) / I_hat, a2, (double)C1.worlds);
                res->iters_L = i;
                if (sL / sU >= one_m_inv_e_m_eps || i == imax) break;
                Timer ts2;
                sample_cp(ctx, g, q, cj, th, 2 * th, key, inst, per_world, &st);
                samp_ms += ts2.ms();
                th *= 2;
            }
            BLv = go.B;
            res->nBL = (int32_t)BLv.size();
            put(B_L, BLv);
            res->sigmaL_L = sL;
            res->sigmaU_L = sU;
            res->theta_C1 = C1.worlds;
            res->theta_C2 = C2.worlds;
            res->covC2 = cov2;
            res->DL_hat = (double)cov2 / (double)C2.worlds;
            res->ms_stage[1] = samp_ms;
            res->ms_stage[2] = greedy_ms;
            res->worlds_sampled += st.worlds;
            res->edges_scanned += st.edges;
            res->kernel_ms[1] += st.kernel_ms;
        }

        // ---- GSBM (Sec. 5.2) ----
        if (do_U) {
            Timer ts;
            const double a = 1.0 - 1.0 / IM_E;
            const double l6 = std::log(6.0 / delta);
            int32_t top = nVs - nS;
            if (top < k) top = k;
            const double c2 = a * std::sqrt(l6) + std::sqrt(a * (ln_binom((double)top, (double)k) + l6));
            const double th_max = 2.0 * (double)nVs * c2 * c2 / (eps * eps * OPT);
            double th0d = std::floor(th_max * eps * eps * OPT / (double)nVs);
            if (th0d < 1.0) th0d = 1.0;
            int32_t imax = (int32_t)std::ceil(std::log2(th_max / th0d));
            if (imax < 1) imax = 1;
            uint64_t th = (uint64_t)th0d;
            if (opts->fixed_theta) {
                th = opts->fixed_theta;
                imax = 1;
            }
            res->theta_max_U = th_max;
            const double a1 = std::log(3.0 * (double)imax / delta), a2 = a1;
            LrrStore L1, L2;
            DBuf credL1;
            credL1.ensure(ctx, (size_t)n * 8);
            IM_CUDA(cudaMemsetAsync(credL1.p, 0, (size_t)n * 8, ctx->stream));
            SpreadEst st;
            std::vector<LrrJob> lj{LrrJob{&L1, 3u, credL1.as<unsigned long long>()},
                                   LrrJob{&L2, 4u, nullptr}};
            sample_lrr(ctx, g, q, lj, 0, th, key, inst, &st);
            double samp_ms = ts.ms(), greedy_ms = 0.0;
            GreedyOut go;
            double sL = 0.0, sU = 0.0;
            unsigned long long cov2 = 0;
            for (int32_t i = 1; i <= imax; ++i) {
                Timer tg;
                {
                    EventTimer et(ctx);
                    greedy_lrr(ctx, gb, L1, n, k, credL1.as<unsigned long long>());
                    res->kernel_ms[3] += et.stop();
                }
                go = read_greedy(ctx, gb, k);
                set_bitmap_host(ctx, d_inB, words, go.B);
                cov2 = cov_lrr(ctx, L2, d_inB.as<uint32_t>(), d_cov.as<unsigned long long>(), &h_cov);
                greedy_ms += tg.ms();
                sL = sigma_low((double)cov2, a1, (double)L2.nsets) * (double)nVs;
                sU = sigma_up((double)go.covu, a2, (double)L1.nsets) * (double)nVs;
                res->iters_U = i;
                if (sL / sU >= one_m_inv_e_m_eps || i == imax) break;
                Timer ts2;
                sample_lrr(ctx, g, q, lj, th, 2 * th, key, inst, &st);
                samp_ms += ts2.ms();
                th *= 2;
            }
            BUv = go.B;
            res->nBU = (int32_t)BUv.size();
            put(B_U, BUv);
            res->sigmaL_U = sL;
            res->sigmaU_U = sU;
            res->theta_L1 = L1.nsets;
            res->theta_L2 = L2.nsets;
            res->covL2 = cov2;
            res->DU_hat = (double)nVs * (double)cov2 / (double)L2.nsets;
            res->ms_stage[3] = samp_ms;
            res->ms_stage[4] = greedy_ms;
            res->worlds_sampled += st.worlds;
            res->edges_scanned += st.edges;
            res->kernel_ms[2] += st.kernel_ms;
        }
        res->nBR = k;
        put(B_R, BRv);

        // ---- Sandwich: Algorithm 1, lines 4-5 ----
        Timer tf;
        const std::vector<int32_t> *cand[3] = {&BLv, &BUv, &BRv};
        const bool use[3] = {do_L, do_U, do_R};
        Query qb[3];
        std::vector<StopSpec> fin;
        std::vector<int> fin_c;
        for (int c = 0; c < 3; ++c) {
            res->I_after[c] = 0.0;
            if (!use[c]) continue;
            prepare_query(ctx, g, qb[c], S.data(), (int32_t)S.size(), cand[c]->data(),
                          (int32_t)cand[c]->size(), true);
            fin.push_back(StopSpec{g, &qb[c], gamma, delta, key, (uint32_t)(5 + c), inst, SpreadEst{}});
            fin_c.push_back(c);
        }
        stop_rules(ctx, fin);
        int best = -1;
        for (size_t i = 0; i < fin.size(); ++i) {
            const int c = fin_c[i];
            const SpreadEst &e = fin[i].est;
            res->I_after[c] = e.I;
            res->n_final[c] = e.N;
            res->worlds_sampled += e.worlds;
            res->edges_scanned += e.edges;
            res->kernel_ms[0] += e.kernel_ms;
            res->reach_nodes += e.nodes;
            res->reach_edges += e.edges;
            res->reach_launches += e.launches;
        }
        for (int c = 0; c < 3; ++c)
            if (use[c] && (best < 0 || res->I_after[c] < res->I_after[best])) best = c;
        res->ms_stage[5] = tf.ms();
        res->chosen = best;
        res->n_blockers = (int32_t)cand[best]->size();
        put(blockers, *cand[best]);
        if (do_U && variant == IMIN_SANDIMIN && res->DU_hat > 0.0) {
            const double gr = (1.0 - gamma) * (1.0 - gamma) / ((1.0 + gamma) * (1.0 + gamma));
            res->ratio_lb = gr * one_m_inv_e_m_eps * (I_hat - res->I_after[1]) / res->DU_hat;
        }
        res->ms_stage[6] = host_ms;
        res->ms_stage[7] = total.ms();
        res->kernel_launches = g_kernel_launches - launches0;
    });
}

}  // extern "C"
