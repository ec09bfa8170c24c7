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
#include <array>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
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
    DBuf dS, dseed_bm, dblk_bm, dB, dVs;   // dVs: V'_s sorted ascending (nVs entries)
    int32_t nVs = 0;
    size_t words = 0;
    void release()
    {
        for (DBuf *b : {&dS, &dseed_bm, &dblk_bm, &dB, &dVs}) b->release();
        nVs = 0;
        std::vector<uint8_t>().swap(is_seed);
        std::vector<uint8_t>().swap(is_blocked);
    }
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
    q.nVs = 0;
    if (need_vs)
        q.nVs = device_reach_set(ctx, g, q.dS.as<int32_t>(), (int32_t)q.S.size(), q.dseed_bm.as<uint32_t>(),
                                 q.blocked.empty() ? nullptr : q.dblk_bm.as<uint32_t>(), q.dVs);
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
    d.Vs = q.nVs > 0 ? q.dVs.as<int32_t>() : nullptr;
    d.nVs = q.nVs;
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
    const uint32_t *list = nullptr;   // device: the worlds are first + list[0 .. count) (else consecutive)
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

    const SlotCfg *force = nullptr;     // autotuner: launch configuration to time
    const imin_graph *gref = nullptr;   // graph whose tuned configuration applies

    // slot memory of at most half the free device memory (and half the budget left)
    size_t slot_avail(size_t *freeb_out = nullptr) const
    {
        size_t freeb = 0, totalb = 0;
        cudaMemGetInfo(&freeb, &totalb);
        size_t avail = freeb / 2;
        if (ctx->budget)
            avail = std::min(avail, ctx->budget > ctx->in_use ? (ctx->budget - ctx->in_use) / 2 : 0);
        if (freeb_out) *freeb_out = freeb;
        return avail;
    }

    SlotCfg cap_ctas(SlotCfg c) const
    {
        size_t freeb = 0;
        const size_t avail = slot_avail(&freeb);
        const size_t per = c.bytes_per_slot();
        const size_t maxc = per ? avail / per : (size_t)c.ctas;
        if ((size_t)c.ctas > maxc) c.ctas = (int)std::max<size_t>(maxc, 1);
        if (per > freeb) fail(IMIN_ENOMEM, "not enough device memory for sampling slots");
        c.warps = c.ctas * (c.cta_threads / 32);
        return c;
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
        // reach-only worlds: one world per CTA, as many CTAs as fit on an SM, the visited
        // bitmap in shared memory when n bits fit; the autotuner's choice for the graph
        // wins when there is one (IMIN_REACH_CTA=0 selects the warp-per-world kernel)
        const char *cta_env = std::getenv("IMIN_REACH_CTA");
        const char *upper_env = std::getenv("IMIN_UPPER_CTA");
        const bool upper_cta = c.upper && !(upper_env && upper_env[0] == '0');
        // lower-bound worlds (without the upper bound in the same pass) also run one per
        // CTA (IMIN_LOWER_CTA=0: warp per world); their edge pairs get a fixed budget and
        // a world that needs more is deferred to the large-slot pass
        const char *lower_env = std::getenv("IMIN_LOWER_CTA");
        const bool lower_cta = c.lower && !c.upper && !(lower_env && lower_env[0] == '0');
        if ((lower_cta || (!c.lower && (!c.upper || upper_cta))) && !big) {
            if (c.lower) {
                c.ecap = (int32_t)std::min<int64_t>(std::max<int64_t>(m, 1),
                                                    std::max<int64_t>(1 << 20, 2 * ((int64_t)n + 1)));
                if (const char *env = std::getenv("IMIN_SLOT_QCAP")) {   // test hook, as below
                    const long v = std::strtol(env, nullptr, 10);
                    if (v > 0 && v < c.ecap) c.ecap = (int32_t)v;
                }
            }
            if (force) {   // autotuner probe
                SlotCfg f = *force;
                f.upper = c.upper;
                return cap_ctas(f);
            }
            const bool env_warp = cta_env && cta_env[0] == '0';
            if (gref && gref->tuned_ctas > 0 && !env_warp) {
                c.smem_bm = gref->tuned_smem;
                c.cta_threads = gref->tuned_bd;
                c.cta_minb = gref->tuned_minb;
                c.qcap = n + 1;
                c.ctas = gref->tuned_ctas;
                if (c.lower) {
                    // lower-bound worlds (dominators: many barriers per world) run on
                    // 512-thread CTAs, 4 per SM, whatever the reach-only tuning chose
                    // (IMIN_LOWER_BD=256/512/1024 selects another CTA size)
                    int lbd = 512;
                    if (const char *env = std::getenv("IMIN_LOWER_BD")) {
                        const long v = std::strtol(env, nullptr, 10);
                        if (v == 256 || v == 512 || v == 1024) lbd = (int)v;
                    }
                    c.cta_threads = lbd;
                    c.cta_minb = lbd == 256 ? 8 : (lbd == 512 ? 4 : 2);
                    c.ctas = ctx->num_sms * c.cta_minb;
                }
                if (c.lower || c.upper) {
                    // the same shape, at most as many CTAs per SM as the bound's kernel fits
                    if (c.smem_bm) {
                        int optin = 0;
                        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
                        cudaGetLastError();
                        if (c.bm_words * 4 + cta_static_smem(c.cta_threads, c.lower) + 1024 > (size_t)optin)
                            c.smem_bm = false;
                    }
                    const int occ = cta_blocks_per_sm(c.cta_threads, c.cta_minb, c.smem_bm, c.upper, c.lower,
                                                      c.bm_words);
                    c.ctas = ctx->num_sms * std::max(1, std::min(gref->tuned_ctas / ctx->num_sms, occ));
                }
                c.warps = c.ctas * (c.cta_threads / 32);
                return cap_ctas(c);
            }
            if (!env_warp && !(gref && gref->tuned_ctas < 0)) {
                int optin = 0;
                cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
                cudaGetLastError();
                // test hooks: IMIN_REACH_BD picks the CTA size (and IMIN_REACH_MINB the
                // CTAs per SM it is compiled for), IMIN_REACH_SMEM=0 keeps the visited
                // bitmap in global memory
                int bd = 512, minb = 4;
                if (const char *env = std::getenv("IMIN_REACH_BD")) {
                    const long v = std::strtol(env, nullptr, 10);
                    if (v == 256 || v == 512 || v == 1024) bd = (int)v;
                    minb = bd == 256 ? 8 : (bd == 512 ? 4 : 2);
                }
                if (const char *env = std::getenv("IMIN_REACH_MINB")) {
                    const long v = std::strtol(env, nullptr, 10);
                    for (int i = 0; i < kNumCtaShapes; ++i)
                        if (kCtaShapes[i][0] == bd && kCtaShapes[i][1] == v) minb = (int)v;
                }
                c.smem_bm = c.bm_words * 4 + cta_static_smem(bd, c.lower) + 1024 <= (size_t)optin;
                if (const char *env = std::getenv("IMIN_REACH_SMEM"))
                    if (env[0] == '0') c.smem_bm = false;
                c.cta_threads = bd;
                c.cta_minb = minb;
                c.qcap = n + 1;
                c.ctas = ctx->num_sms *
                         std::max(1, cta_blocks_per_sm(bd, minb, c.smem_bm, c.upper, c.lower, c.bm_words));
                c.warps = c.ctas * (bd / 32);
                return cap_ctas(c);
            }
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
            if (!c.lower && !c.upper && gref && gref->tuned_ctas < 0) per_sm = -gref->tuned_ctas;
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
        size_t freeb = 0;
        const size_t avail = slot_avail(&freeb);
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
        const size_t bytes = cfg.bytes_per_slot() * (size_t)cfg.slots();
        const size_t key = cfg.bytes_per_slot() * 1315423911u + (size_t)cfg.slots();
        const void *before = arena.p;
        if (arena.p && arena.bytes < bytes) arena.release();   // never hold two arenas at once
        arena.ensure(ctx, bytes, false, true);
        if (arena.p != before || layout != key) {
            IM_CUDA(cudaMemsetAsync(arena.p, 0, arena.bytes, ctx->stream));
            layout = key;
        }
    }

    // The slot arena is prepared last, after every other allocation of the launch: an
    // allocation that does not fit drops the (cached) arenas, see dev_alloc.
    void launch(const std::vector<WTask> &ht, const imin_graph *g0, uint32_t flags,
                const SlotCfg &cfg, DBuf &arena, size_t &layout)
    {
        const int n = (int)ht.size();
        dtasks.ensure(ctx, ht.size() * sizeof(WTask));
        cd.ensure(ctx, (size_t)n * 8 + 16);
        prepare_slots(arena, cfg, layout);
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
        for (int i = 0; i < n; ++i)
            if (!gref || T[i]->g->n > gref->n) gref = T[i]->g;
        SlotCfg cfg = cfg_for(flags, nmax, mmax, nSmax, false);
        DBuf &arena = cfg.lower ? ctx->slots_lower : ctx->slots;
        size_t &layout = cfg.lower ? ctx->slots_lower_layout : ctx->slots_layout;
        std::vector<WTask> ht;
        for (int i = 0; i < n; ++i)
            ht.push_back(make_task(T[i]->g, T[i]->q, T[i]->first, T[i]->count, T[i]->list, T[i]->out));
        launch(ht, T[0]->g, flags, cfg, arena, layout);
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
                // a deferred world was claimed before the early exit, so it must complete:
                // the re-runs never apply the stopping rule
                const uint32_t rflags = flags & ~(uint32_t)WF_STOP;
                if (pass == 0) {
                    launch(lt, T[0]->g, rflags, cfg, arena, layout);
                } else {
                    SlotCfg bc = cfg_for(rflags, nmax, mmax, nSmax, true);
                    launch(lt, T[0]->g, rflags, bc, ctx->big_slots, ctx->big_slots_layout);
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
// Autotuner: the launch configuration of reach-only worlds (the frontier tile = CTA
// size, worlds per SM, where the visited bitmap lives, or the warp-per-world kernel)
// is chosen per graph by timing a short probe of each candidate on the first query
// that reaches the graph.  The probe draws worlds of a tag no solve uses and its
// outputs are discarded, so it changes no result.  IMIN_AUTOTUNE=0 keeps the
// default (one 1024-thread CTA per world).
// ---------------------------------------------------------------------------
// graphs of the same shape (n, m and 64 sampled row offsets) share a tuning
uint64_t graph_signature(const imin_graph *g)
{
    uint64_t h = 1469598103934665603ull ^ (uint64_t)g->n ^ ((uint64_t)g->m << 20);
    const size_t len = g->h_row_ptr.size();
    for (int i = 0; i < 64 && len; ++i) {
        h ^= (uint64_t)(uint32_t)g->h_row_ptr[(size_t)i * (len - 1) / 63];
        h *= 1099511628211ull;
    }
    return h;
}

void autotune_reach(imin_ctx *ctx, imin_graph *g, const Query &q)
{
    if (g->tuned_ctas != 0) return;
    if (const char *env = std::getenv("IMIN_AUTOTUNE"))
        if (env[0] == '0') return;
    const uint64_t sig = graph_signature(g);
    for (const imin_ctx::TuneEntry &te : ctx->tune_cache)
        if (te.sig == sig && te.n == g->n && te.m == g->m) {
            g->tuned_ctas = te.ctas;
            g->tuned_bd = te.bd;
            g->tuned_minb = te.minb;
            g->tuned_smem = te.smem;
            return;
        }
    const size_t words = ((size_t)g->n + 31) / 32;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    cudaGetLastError();
    struct Cand {
        int bd, minb, ctas;
        bool smem;
        int warp_per_sm;   // > 0: warp-per-world kernel
    };
    std::vector<Cand> cands;
    for (int i = 0; i < kNumCtaShapes; ++i)
        for (int sm = 1; sm >= 0; --sm) {
            const int bd = kCtaShapes[i][0], minb = kCtaShapes[i][1];
            const bool smem = sm == 1;
            if (smem && words * 4 + cta_static_smem(bd) + 1024 > (size_t)optin) continue;
            const int nb = std::min(minb, cta_blocks_per_sm(bd, minb, smem, false, false, words));
            if (nb <= 0) continue;
            // a shape compiled for more CTAs per SM than fit is the same launch as a
            // smaller one with fewer registers: skip it
            if (nb < minb && minb > 1) {
                bool dup = false;
                for (int k = 0; k < kNumCtaShapes; ++k)
                    dup |= kCtaShapes[k][0] == bd && kCtaShapes[k][1] < minb && kCtaShapes[k][1] >= nb;
                if (dup) continue;
            }
            cands.push_back(Cand{bd, minb, ctx->num_sms * nb, smem, 0});
        }
    cands.push_back(Cand{0, 0, 0, false, 32});
    // Each candidate is timed on W and on 2W worlds; the difference over W is its cost
    // per world in a long launch, free of the launch's fill and drain (the solve's
    // launches hold thousands of worlds per CTA).  W is two waves of the candidate.
    uint32_t widest = 0;
    for (const Cand &cd : cands) widest = std::max<uint32_t>(widest, (uint32_t)cd.ctas);
    Runner probe_runner(ctx);
    double best = 1e30;
    Cand pick = cands.front();
    for (const Cand &cd : cands) {
        SlotCfg c;
        c.bm_words = words;
        if (cd.warp_per_sm) {
            g->tuned_ctas = -cd.warp_per_sm;
            probe_runner.force = nullptr;
        } else {
            c.ctas = cd.ctas;
            c.cta_threads = cd.bd;
            c.cta_minb = cd.minb;
            c.smem_bm = cd.smem;
            c.qcap = g->n + 1;
            c.warps = cd.ctas * (cd.bd / 32);
            probe_runner.force = &c;
        }
        const uint32_t concurrent = cd.warp_per_sm ? (uint32_t)(ctx->num_sms * cd.warp_per_sm)
                                                   : (uint32_t)cd.ctas;
        auto timed = [&](uint32_t count, uint32_t inst) {
            TaskRun t;
            t.g = g;
            t.q = qdev(q, 0x5eedull, 0xFFFFFFF0u, inst);
            t.first = 0;
            t.count = count;
            std::vector<TaskRun *> tp{&t};
            const double before = probe_runner.kernel_ms;
            probe_runner.gref = g;
            probe_runner.run(tp, 0u);
            return probe_runner.kernel_ms - before;
        };
        // an untimed wave loads the kernel; then W and 2W worlds, with W at least two
        // waves and large enough that W worlds take a few milliseconds (small worlds
        // would otherwise be timed at the resolution of the events)
        timed(std::min<uint32_t>(concurrent, 1024), 0);
        uint64_t W = std::min<uint32_t>(std::max<uint32_t>(2 * std::max(concurrent, widest), 2048), 16384);
        double ms[3] = {0.0, timed((uint32_t)W, 1), 0.0};
        if (ms[1] < 3.0) {
            W = std::min<uint64_t>(W * (uint64_t)std::ceil(3.0 / std::max(ms[1], 0.01)), (uint64_t)1 << 20);
            ms[1] = timed((uint32_t)W, 1);
        }
        ms[2] = timed((uint32_t)(2 * W), 2);
        const double per_world = ms[2] > ms[1] ? (ms[2] - ms[1]) / W : ms[2] / (2.0 * W);
        if (per_world < best) {
            best = per_world;
            pick = cd;
        }
        g->tuned_ctas = 0;
    }
    if (pick.warp_per_sm) {
        g->tuned_ctas = -pick.warp_per_sm;
    } else {
        g->tuned_ctas = pick.ctas;
        g->tuned_bd = pick.bd;
        g->tuned_minb = pick.minb;
        g->tuned_smem = pick.smem;
    }
    ctx->tune_cache.push_back(imin_ctx::TuneEntry{sig, g->n, g->m, g->tuned_ctas, g->tuned_bd, g->tuned_minb,
                                                  g->tuned_smem});
}

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
    // Worlds are drawn in index order in chunks: each launch serves every unfinished
    // estimate over its next range of worlds, with the threshold still missing as its
    // early-exit bound; the host scans the sizes in order to find N exactly.
    const size_t ns = specs.size();
    for (size_t i = 0; i < ns; ++i)
        autotune_reach(ctx, const_cast<imin_graph *>(specs[i].g), *specs[i].q);
    std::vector<double> W(ns), ups1(ns);
    std::vector<unsigned long long> T(ns), sum(ns, 0);
    std::vector<uint64_t> first(ns, 0), N(ns, 0), chunk(ns);
    std::vector<size_t> soff(ns, 0);   // per estimate: offset of its sizes in ctx->stop_spread
    for (size_t i = 0; i < ns; ++i) {
        StopSpec &sp = specs[i];
        W[i] = (double)sp.q->nVs + (double)sp.q->S.size();
        const double ups = 4.0 * (IM_E - 2.0) * std::log(2.0 / sp.dprime) / (sp.beta * sp.beta);
        ups1[i] = 1.0 + (1.0 + sp.beta) * ups;
        const double Td = std::ceil(ups1[i] * W[i]);
        if (!(Td < 1.8e19)) fail(IMIN_ERANGE, "stopping threshold too large");
        T[i] = (unsigned long long)Td;
        // every world reaches at least |S| nodes, so N <= ceil(T / |S|)
        const uint64_t nmax = (T[i] + sp.q->S.size() - 1) / sp.q->S.size();
        if (nmax >= ((uint64_t)1 << 32) - 1) fail(IMIN_ERANGE, "the stopping rule may need >= 2^32 worlds");
        uint64_t c0 = (uint64_t)1 << 21;
        // test hook: IMIN_STOP_CHUNK sets the first chunk (to exercise several chunks)
        if (const char *env = std::getenv("IMIN_STOP_CHUNK")) {
            const long long v = std::strtoll(env, nullptr, 10);
            if (v > 0) c0 = (uint64_t)v;
        }
        chunk[i] = std::min<uint64_t>(nmax, c0);
    }
    double kms = 0.0;
    uint64_t launches = 0;
    for (;;) {
        std::vector<TaskRun> tr(ns);
        std::vector<TaskRun *> tp;
        std::vector<size_t> idx;
        // the per-world sizes of every estimate of this launch, in one cached buffer
        size_t total = 0;
        for (size_t i = 0; i < ns; ++i) {
            if (N[i]) continue;
            const uint64_t cnt = std::min<uint64_t>(chunk[i], ((uint64_t)1 << 32) - 1 - first[i]);
            soff[i] = total;
            total += ((size_t)cnt + 4) & ~(size_t)3;
        }
        ctx->stop_spread.ensure(ctx, total * 4 + 16);
        for (size_t i = 0; i < ns; ++i) {
            if (N[i]) continue;
            const uint64_t cnt = std::min<uint64_t>(chunk[i], ((uint64_t)1 << 32) - 1 - first[i]);
            TaskRun &t = tr[i];
            t.g = specs[i].g;
            t.q = qdev(*specs[i].q, specs[i].key, specs[i].tag, specs[i].inst);
            t.first = first[i];
            t.count = (uint32_t)cnt;
            t.out.world_spread = ctx->stop_spread.as<uint32_t>() + soff[i];
            t.out.stop_T = T[i] - sum[i];
            tp.push_back(&t);
            idx.push_back(i);
        }
        if (tp.empty()) break;
        // estimates on graphs that the autotuner gave different launch shapes run in
        // separate launches, each in its graph's shape (one launch when they agree)
        std::vector<std::vector<TaskRun *>> groups;
        std::vector<std::array<int, 4>> keys;
        for (TaskRun *t : tp) {
            const std::array<int, 4> key{t->g->tuned_ctas, t->g->tuned_bd, t->g->tuned_minb,
                                         t->g->tuned_smem ? 1 : 0};
            size_t gi = 0;
            while (gi < keys.size() && keys[gi] != key) ++gi;
            if (gi == keys.size()) {
                keys.push_back(key);
                groups.emplace_back();
            }
            groups[gi].push_back(t);
        }
        for (std::vector<TaskRun *> &grp : groups) {
            Runner run(ctx);
            run.run(grp, WF_STOP | WF_SPREAD);
            kms += run.kernel_ms;
            launches += (uint64_t)run.launches;
        }
        for (size_t i : idx) {
            // every claimed world is complete (deferred ones were re-run)
            const uint64_t want = tr[i].claimed_main;
            std::vector<uint32_t> sizes(want);
            if (want)
                IM_CUDA(cudaMemcpy(sizes.data(), ctx->stop_spread.as<uint32_t>() + soff[i], want * 4,
                                   cudaMemcpyDeviceToHost));
            for (uint64_t j = 0; j < want; ++j) {
                sum[i] += sizes[j];
                if (sum[i] >= T[i]) {
                    N[i] = first[i] + j + 1;
                    break;
                }
            }
            SpreadEst &r = specs[i].est;
            r.worlds += tr[i].acc[4];
            r.edges += tr[i].acc[1];
            r.nodes += tr[i].acc[0];
            if (!N[i]) {
                if (want < tr[i].count) fail(IMIN_EDEVICE, "stopping rule: threshold not reached");
                first[i] += want;
                chunk[i] = std::min<uint64_t>(chunk[i] * 2, (uint64_t)1 << 30);
            }
        }
    }
    for (size_t i = 0; i < ns; ++i) {
        SpreadEst &r = specs[i].est;
        r.N = N[i];
        r.I = W[i] * ups1[i] / (double)N[i];
    }
    // device time is shared by the tasks of the launches: report it on the first
    specs[0].est.kernel_ms = kms;
    specs[0].est.launches = launches;
}

SpreadEst stop_rule(imin_ctx *ctx, const imin_graph *g, const Query &q, double beta, double dprime,
                    uint64_t key, uint32_t tag, uint32_t inst)
{
    std::vector<StopSpec> v{StopSpec{g, &q, beta, dprime, key, tag, inst, SpreadEst{}}};
    stop_rules(ctx, v);
    return v[0].est;
}

// ---------------------------------------------------------------------------
// Relabelled forward index of a query (hot_view.cu) for its fused final estimates.
// It changes no result (the estimates count nodes, and every edge keeps its coin); it
// pays where the worlds' candidate maps live in global memory and miss L2 (on the 1M-node
// Chung-Lu workload the final estimates take 14% less time; the spread estimate's 1-bit
// visited bitmaps gained nothing measurable and keep the original index).  IMIN_HOT_VIEW=0 turns it
// off, =2 builds it on every graph (test hook); IMIN_HOT_WORLDS sets the worlds of the
// reach counts that order the labels (default 2,048, of a stream tag no estimate draws).
// ---------------------------------------------------------------------------
constexpr uint32_t TAG_HOT = 0xFFFFFFF1u;

struct HotStats {
    double kernel_ms = 0.0;
    uint64_t launches = 0;
};

HotStats maybe_hot_view(imin_ctx *ctx, const imin_graph *g, const Query &q, uint64_t key, uint32_t inst,
                        HotView &hv)
{
    HotStats hs;
    hv.release();
    const char *env = std::getenv("IMIN_HOT_VIEW");
    const bool force = env && env[0] == '2';
    if (env && env[0] == '0') return hs;
    if (!force && !(g->tuned_ctas > 0 && !g->tuned_smem && g->n >= (1 << 18))) return hs;
    if (!q.blocked.empty()) return hs;
    uint32_t W0 = 2048;
    if (const char *we = std::getenv("IMIN_HOT_WORLDS")) {
        const long v = std::strtol(we, nullptr, 10);
        if (v >= 1 && v <= 6000) W0 = (uint32_t)v;
    }
    // the view is an optimisation: without the memory for it the estimates run on the
    // original index
    try {
        DBuf counts;
        counts.ensure(ctx, (size_t)g->n * 8);
        IM_CUDA(cudaMemsetAsync(counts.p, 0, (size_t)g->n * 8, ctx->stream));
        TaskRun t;
        t.g = g;
        t.q = qdev(q, key, TAG_HOT, inst);
        t.first = 0;
        t.count = W0;
        t.out.reach = counts.as<unsigned long long>();
        std::vector<TaskRun *> tp{&t};
        Runner run(ctx);
        run.run(tp, WF_REACH);
        hs.kernel_ms = run.kernel_ms;
        hs.launches = (uint64_t)run.launches;
        hs.launches += (uint64_t)hot_view_build(ctx, g, counts.as<unsigned long long>(), W0, q.dS.as<int32_t>(),
                                                (int32_t)q.S.size(), hv);
    } catch (const ImError &e) {
        if (e.code != IMIN_ENOMEM) throw;
        hv.release();
    }
    return hs;
}

// the candidates' blocked lists in the view's labels
int hot_view_blocked(imin_ctx *ctx, HotView &hv, const Query *const qb[3], const bool use[3])
{
    if (!hv.on) return 0;
    int launches = 0;
    int64_t tot = 0;
    for (int c = 0; c < 3; ++c) {
        hv.boff[c] = tot;
        if (use[c]) tot += (int64_t)qb[c]->blocked.size();
    }
    try {
        hv.B.ensure(ctx, (size_t)std::max<int64_t>(tot, 1) * 4);
    } catch (const ImError &e) {
        if (e.code != IMIN_ENOMEM) throw;
        hv.release();
        return 0;
    }
    for (int c = 0; c < 3; ++c)
        if (use[c] && !qb[c]->blocked.empty())
        {
            hot_view_map(ctx, hv, qb[c]->dB.as<int32_t>(), (int32_t)qb[c]->blocked.size(),
                         hv.B.as<int32_t>() + hv.boff[c]);
            ++launches;
        }
    IM_CUDA(cudaStreamSynchronize(ctx->stream));
    return launches;
}

// ---------------------------------------------------------------------------
// Final estimates (Algorithm 1, line 4): the (gamma, delta)-estimates of the residual
// spread of up to three candidate blocker sets, all on the worlds of stream tag 5.
// One traversal per world serves every candidate (final_cta.cu); each candidate
// stops at its own N, found exactly on the host from the per-world sizes.
// ---------------------------------------------------------------------------
constexpr uint32_t TAG_FINAL = 5u;
constexpr uint32_t TAG_PR = 6u;   // worlds of the reach-frequency reading of Pr[s -> v]

struct FinalSpec {
    const imin_graph *g;
    const Query *q;        // the query (seeds)
    const Query *qb[3];    // per candidate: S with the candidate's blockers (V'_s in G[V \ B])
    bool use[3];
    double gamma, delta;
    uint64_t key;
    uint32_t inst;
    double spread_hint;   // expected spread without blockers (sizes the fused queue; 0 = unknown)
    SpreadEst est[3];
    const HotView *hv;    // relabelled forward index with the candidates' blocked lists (or null)
};

struct FinalStats {
    double kernel_ms = 0.0;
    uint64_t launches = 0;
};

FinalStats final_estimates(imin_ctx *ctx, std::vector<FinalSpec> &specs)
{
    FinalStats fs;
    const size_t ns = specs.size();
    if (!ns) return fs;
    int32_t nmax = 1;
    for (const FinalSpec &f : specs) nmax = std::max(nmax, f.g->n);
    const char *env = std::getenv("IMIN_FINAL_FUSED");
    const bool fused = !(env && env[0] == '0') && nmax < (1 << 28);
    if (!fused) {
        // one reach-only stopping rule per candidate, each on the same worlds (tag 5):
        // the same sizes as the fused traversal, so the same estimates
        std::vector<StopSpec> sp;
        std::vector<std::pair<size_t, int>> ref;
        for (size_t i = 0; i < ns; ++i)
            for (int c = 0; c < 3; ++c)
                if (specs[i].use[c]) {
                    sp.push_back(StopSpec{specs[i].g, specs[i].qb[c], specs[i].gamma, specs[i].delta,
                                          specs[i].key, TAG_FINAL, specs[i].inst, SpreadEst{}});
                    ref.emplace_back(i, c);
                }
        if (sp.empty()) return fs;
        stop_rules(ctx, sp);
        for (size_t k = 0; k < sp.size(); ++k) specs[ref[k].first].est[ref[k].second] = sp[k].est;
        fs.kernel_ms = sp[0].est.kernel_ms;
        fs.launches = sp[0].est.launches;
        for (size_t k = 0; k < sp.size(); ++k) specs[ref[k].first].est[ref[k].second].kernel_ms = 0.0;
        return fs;
    }
    for (size_t i = 0; i < ns; ++i)
        autotune_reach(ctx, const_cast<imin_graph *>(specs[i].g), *specs[i].q);
    // thresholds T_c = ceil(Upsilon1 W_c), W_c = |V'_s in G[V \ B_c]| + |S|
    std::vector<std::array<double, 3>> W(ns), ups1(ns);
    std::vector<std::array<unsigned long long, 3>> T(ns), sum(ns);
    std::vector<std::array<uint64_t, 3>> N(ns);
    std::vector<uint64_t> first(ns, 0), chunk(ns, 1);
    for (size_t i = 0; i < ns; ++i) {
        FinalSpec &f = specs[i];
        uint64_t cmax = 1;
        for (int c = 0; c < 3; ++c) {
            sum[i][c] = 0;
            N[i][c] = 0;
            T[i][c] = 0;
            if (!f.use[c]) continue;
            W[i][c] = (double)f.qb[c]->nVs + (double)f.q->S.size();
            const double ups = 4.0 * (IM_E - 2.0) * std::log(2.0 / f.delta) / (f.gamma * f.gamma);
            ups1[i][c] = 1.0 + (1.0 + f.gamma) * ups;
            const double Td = std::ceil(ups1[i][c] * W[i][c]);
            if (!(Td < 1.8e19)) fail(IMIN_ERANGE, "stopping threshold too large");
            T[i][c] = (unsigned long long)Td;
            const uint64_t nm = (T[i][c] + f.q->S.size() - 1) / f.q->S.size();
            if (nm >= ((uint64_t)1 << 32) - 1) fail(IMIN_ERANGE, "the stopping rule may need >= 2^32 worlds");
            cmax = std::max(cmax, nm);
        }
        uint64_t c0 = (uint64_t)1 << 21;
        if (const char *ce = std::getenv("IMIN_STOP_CHUNK")) {   // test hook: several chunks
            const long long v = std::strtoll(ce, nullptr, 10);
            if (v > 0) c0 = (uint64_t)v;
        }
        chunk[i] = std::min<uint64_t>(cmax, c0);
    }
    // launch shape: the graph's tuned CTA size (256 or 512 threads), as many CTAs as are
    // resident, within half of the free memory
    // 256 threads x 8 CTAs per SM (the fastest shape of this kernel on the power-law
    // workloads measured; the reach-only tuning does not carry over: the candidate map
    // is four times the visited bitmap)
    int bd = 256;
    int minb = 8;
    // tuning hook: IMIN_FINAL_SHAPE=<threads>:<CTAs per SM> (256 or 512 threads)
    if (const char *fe = std::getenv("IMIN_FINAL_SHAPE")) {
        int b = 0, m = 0;
        if (std::sscanf(fe, "%d:%d", &b, &m) == 2 && (b == 256 || b == 512) && m >= 1) {
            bd = b;
            minb = std::min(m, b == 256 ? 8 : 4);
        }
    }
    const int occ = std::max(1, std::min(minb, final_blocks_per_sm(bd)));
    // queue entries per slot: a world needs at most the three reach sets' sizes; the
    // queue holds 32 times the expected spread (all 3 (n + 1) when it is not known), and
    // a world that overflows it (the reach distribution has a long tail) is re-run one
    // candidate at a time below
    double hint = 0.0;
    int32_t nSmax = 1;
    for (const FinalSpec &f : specs) {
        hint = std::max(hint, f.spread_hint > 0.0 ? f.spread_hint : 1e30);
        nSmax = std::max<int32_t>(nSmax, (int32_t)f.q->S.size());
    }
    const double full = 3.0 * ((double)nmax + 1.0);
    int32_t qcap = (int32_t)std::min(full, std::max(262144.0, 32.0 * hint + 3.0 * nSmax));
    if (const char *qe = std::getenv("IMIN_FINAL_QCAP")) {   // test hook: tiny queues, many re-runs
        const long v = std::strtol(qe, nullptr, 10);
        if (v > nSmax && v < qcap) qcap = (int32_t)v;
    }
    size_t off_q = 0;
    const size_t per = final_slot_bytes(nmax, qcap, &off_q);
    size_t freeb = 0, totalb = 0;
    cudaMemGetInfo(&freeb, &totalb);
    size_t avail = freeb / 2;
    if (ctx->budget)
        avail = std::min(avail, ctx->budget > ctx->in_use ? (ctx->budget - ctx->in_use) / 2 : 0);
    size_t ctas = (size_t)ctx->num_sms * occ;
    if (per * ctas > avail) ctas = std::max<size_t>(avail / per, 1);
    if (per > freeb) fail(IMIN_ENOMEM, "not enough device memory for the final estimates");
    DBuf ctl, cd, dtasks, rerun_ws;
    // per spec and launch: sizes [count][4] and the overflow list, in one cached buffer
    std::vector<size_t> zoff(ns, 0), doff(ns, 0);

    std::vector<std::vector<uint32_t>> hsz(ns);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    IM_CUDA(cudaEventCreate(&e0));
    IM_CUDA(cudaEventCreate(&e1));
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard()
        {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } evg{e0, e1};
    for (;;) {
        std::vector<FTask> ht;
        std::vector<size_t> idx;
        size_t total = 0;
        for (size_t i = 0; i < ns; ++i) {
            bool any = false;
            for (int c = 0; c < 3; ++c) any |= specs[i].use[c] && !N[i][c];
            if (!any) continue;
            const uint64_t cnt = std::min<uint64_t>(chunk[i], ((uint64_t)1 << 32) - 1 - first[i]);
            zoff[i] = total;
            total += (size_t)cnt * 4 + 4;
            doff[i] = total;
            total += ((size_t)cnt + 4) & ~(size_t)3;
        }
        ctx->final_scratch.ensure(ctx, total * 4 + 16);
        auto sizes_of = [&](size_t i) { return ctx->final_scratch.as<uint32_t>() + zoff[i]; };
        auto defl_of = [&](size_t i) { return ctx->final_scratch.as<uint32_t>() + doff[i]; };
        for (size_t i = 0; i < ns; ++i) {
            FinalSpec &f = specs[i];
            uint32_t cands = 0;
            for (int c = 0; c < 3; ++c)
                if (f.use[c] && !N[i][c]) cands |= 1u << c;
            if (!cands) continue;
            const uint64_t cnt = std::min<uint64_t>(chunk[i], ((uint64_t)1 << 32) - 1 - first[i]);
            FTask t{};
            t.row_ptr = f.g->row_ptr.as<int32_t>();
            t.ce = f.g->ce.as<uint4>();
            t.S = f.q->dS.as<int32_t>();
            t.nS = (int32_t)f.q->S.size();
            t.cands = cands;
            const bool view = f.hv && f.hv->on;
            if (view) {
                t.rng = f.hv->rng.as<int2>();
                t.gid = f.hv->gid.as<uint32_t>();
                t.ce = f.hv->ce.as<uint4>();
                t.S = f.hv->S.as<int32_t>();
            }
            for (int c = 0; c < 3; ++c) {
                t.B[c] = f.use[c] ? (view ? f.hv->B.as<int32_t>() + f.hv->boff[c] : f.qb[c]->dB.as<int32_t>())
                                  : nullptr;
                t.nB[c] = f.use[c] ? (int32_t)f.qb[c]->blocked.size() : 0;
                t.stop_T[c] = ((cands >> c) & 1u) ? T[i][c] - sum[i][c] : 0ull;
            }
            t.key = f.key;
            t.tag = TAG_FINAL;
            t.inst = f.inst;
            t.first = first[i];
            t.count = (uint32_t)cnt;
            t.sizes = sizes_of(i);
            t.deferred = defl_of(i);
            t.deferred_cap = (uint32_t)cnt;
            ht.push_back(t);
            idx.push_back(i);
        }
        if (ht.empty()) break;
        const int nt = (int)ht.size();
        ctl.ensure(ctx, (size_t)nt * 64);
        cd.ensure(ctx, (size_t)nt * 8 + 16);
        dtasks.ensure(ctx, (size_t)nt * sizeof(FTask));
        for (int k = 0; k < nt; ++k) {
            ht[k].acc = ctl.as<unsigned long long>() + (size_t)k * 8;
            ht[k].n_deferred = reinterpret_cast<uint32_t *>(ht[k].acc + 6);
        }
        // the arena is prepared last (an allocation that does not fit drops the cached
        // arenas); nibble maps must start clear, and every world leaves them clear
        {
            const size_t bytes = per * ctas;
            const size_t key = per * 2654435761u + ctas;
            const void *before = ctx->slots_final.p;
            if (ctx->slots_final.p && ctx->slots_final.bytes < bytes) ctx->slots_final.release();
            ctx->slots_final.ensure(ctx, bytes, false, true);
            if (ctx->slots_final.p != before || ctx->slots_final_layout != key) {
                IM_CUDA(cudaMemsetAsync(ctx->slots_final.p, 0, ctx->slots_final.bytes, ctx->stream));
                ctx->slots_final_layout = key;
            }
        }
        IM_CUDA(cudaMemsetAsync(ctl.p, 0, (size_t)nt * 64, ctx->stream));
        IM_CUDA(cudaMemsetAsync(cd.p, 0, (size_t)nt * 8, ctx->stream));
        IM_CUDA(cudaMemcpyAsync(dtasks.p, ht.data(), ht.size() * sizeof(FTask), cudaMemcpyHostToDevice,
                                ctx->stream));
        IM_CUDA(cudaEventRecord(e0, ctx->stream));
        launch_final_tasks(ctx, dtasks.as<FTask>(), nt, nmax, qcap, bd, (int)ctas, ctx->slots_final.p,
                           cd.as<uint32_t>(), cd.as<uint32_t>() + nt);
        IM_CUDA(cudaEventRecord(e1, ctx->stream));
        IM_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        IM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        fs.kernel_ms += ms;
        fs.launches += 1;
        std::vector<unsigned long long> acc((size_t)nt * 8);
        std::vector<uint32_t> claims(nt);
        IM_CUDA(cudaMemcpy(acc.data(), ctl.p, acc.size() * 8, cudaMemcpyDeviceToHost));
        IM_CUDA(cudaMemcpy(claims.data(), cd.p, (size_t)nt * 4, cudaMemcpyDeviceToHost));
        if (const char *tr = std::getenv("IMIN_TRACE"))
            if (tr[0] == '1') {
                unsigned long long w = 0, en = 0, ed = 0, nd = 0;
                for (int k = 0; k < nt; ++k) {
                    en += acc[(size_t)k * 8 + 3];
                    ed += acc[(size_t)k * 8 + 4];
                    w += acc[(size_t)k * 8 + 5];
                    nd += (uint32_t)acc[(size_t)k * 8 + 6];
                }
                std::fprintf(stderr,
                             "[imin] fused final launch: %d task(s), %llu worlds, %llu queue entries, %llu edges, "
                             "%llu overflowed, %.3f ms, %zu CTAs x %d threads, queue %d\n",
                             nt, w, en, ed, nd, ms, ctas, bd, qcap);
            }
        // worlds that overflowed the fused queue: each candidate's size by its own
        // reach-only traversal of the same world (tag 5), all in one launch
        {
            std::vector<uint32_t> nd(nt);
            for (int k = 0; k < nt; ++k) std::memcpy(&nd[k], &acc[(size_t)k * 8 + 6], 4);
            std::vector<TaskRun> rr;
            std::vector<std::pair<int, int>> rref;
            size_t wsz = 0;
            for (int k = 0; k < nt; ++k)
                if (nd[k])
                    for (int c = 0; c < 3; ++c)
                        if ((ht[k].cands >> c) & 1u) wsz += ht[k].count;
            if (wsz) {
                rerun_ws.ensure(ctx, wsz * 4 + 16);
                size_t at = 0;
                rr.reserve((size_t)nt * 3);
                for (int k = 0; k < nt; ++k) {
                    if (!nd[k]) continue;
                    const size_t i = idx[k];
                    for (int c = 0; c < 3; ++c) {
                        if (!((ht[k].cands >> c) & 1u)) continue;
                        TaskRun t;
                        t.g = specs[i].g;
                        t.q = qdev(*specs[i].qb[c], specs[i].key, TAG_FINAL, specs[i].inst);
                        t.first = ht[k].first;
                        t.count = nd[k];
                        t.list = defl_of(i);
                        t.out.world_spread = rerun_ws.as<uint32_t>() + at;
                        at += ht[k].count;
                        rr.push_back(t);
                        rref.emplace_back(k, c);
                    }
                }
                std::vector<TaskRun *> rp;
                for (TaskRun &t : rr) rp.push_back(&t);
                Runner run(ctx);
                run.run(rp, WF_SPREAD);
                fs.kernel_ms += run.kernel_ms;
                fs.launches += (uint64_t)run.launches;
                std::vector<uint32_t> hws(wsz), hdef;
                IM_CUDA(cudaMemcpy(hws.data(), rerun_ws.p, wsz * 4, cudaMemcpyDeviceToHost));
                at = 0;
                for (size_t r = 0; r < rr.size(); ++r) {
                    const int k = rref[r].first, c = rref[r].second;
                    const size_t i = idx[k];
                    hdef.resize(nd[k]);
                    IM_CUDA(cudaMemcpy(hdef.data(), defl_of(i), (size_t)nd[k] * 4, cudaMemcpyDeviceToHost));
                    // the re-run's sizes sit at the worlds' relative indices
                    std::vector<uint32_t> szk((size_t)ht[k].count * 4);
                    IM_CUDA(cudaMemcpy(szk.data(), sizes_of(i), szk.size() * 4, cudaMemcpyDeviceToHost));
                    for (uint32_t rel : hdef) szk[(size_t)rel * 4 + c] = hws[at + rel];
                    IM_CUDA(cudaMemcpy(sizes_of(i), szk.data(), szk.size() * 4, cudaMemcpyHostToDevice));
                    SpreadEst &r0 = specs[i].est[c];
                    r0.nodes += rr[r].acc[0];
                    r0.edges += rr[r].acc[1];
                    r0.worlds += rr[r].acc[4];
                    at += ht[k].count;
                }
            }
        }
        for (int k = 0; k < nt; ++k) {
            const size_t i = idx[k];
            FinalSpec &f = specs[i];
            const uint64_t got = std::min<uint64_t>(claims[k], ht[k].count);
            hsz[i].resize(got * 4);
            if (got) IM_CUDA(cudaMemcpy(hsz[i].data(), sizes_of(i), got * 16, cudaMemcpyDeviceToHost));
            // launch totals are shared by the candidates: the first served one gets them
            int first_c = -1;
            for (int c = 0; c < 3; ++c) {
                if (!((ht[k].cands >> c) & 1u)) continue;
                if (first_c < 0) first_c = c;
                for (uint64_t j = 0; j < got; ++j) {
                    sum[i][c] += hsz[i][j * 4 + c];
                    if (sum[i][c] >= T[i][c]) {
                        N[i][c] = first[i] + j + 1;
                        break;
                    }
                }
                if (!N[i][c] && got < ht[k].count) fail(IMIN_EDEVICE, "final estimate: threshold not reached");
            }
            SpreadEst &r = f.est[first_c];
            r.nodes += acc[(size_t)k * 8 + 3];
            r.edges += acc[(size_t)k * 8 + 4];
            r.worlds += acc[(size_t)k * 8 + 5];
            first[i] += got;
            chunk[i] = std::min<uint64_t>(chunk[i] * 2, (uint64_t)1 << 30);
        }
    }
    for (size_t i = 0; i < ns; ++i)
        for (int c = 0; c < 3; ++c)
            if (specs[i].use[c]) {
                specs[i].est[c].N = N[i][c];
                specs[i].est[c].I = W[i][c] * ups1[i][c] / (double)N[i][c];
            }
    return fs;
}

// ---------------------------------------------------------------------------
// Collections: CP records (C1, C2) and LRR sets (L1, L2), appended together
// ---------------------------------------------------------------------------
bool store_tight()
{
    const char *env = std::getenv("IMIN_STORE_TIGHT");
    return env && env[0] == '1';
}

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
    const imin_graph *g;
    const Query *q;
    CpStore *c;
    uint32_t tag;
    unsigned long long *credit;   // may be null
    uint64_t from, to;
    uint64_t key;
    uint32_t inst;
    double per_world;             // expected records per world (sizes the store)
    SpreadEst *stats;             // may be null
};

// append worlds [from, to) of each job's tag to its CP collection, one launch for all jobs
void sample_cp(imin_ctx *ctx, std::vector<CpJob> &jobs)
{
    const size_t nj = jobs.size();
    std::vector<TaskRun> tr(nj);
    std::vector<TaskRun *> tp;
    for (size_t i = 0; i < nj; ++i) {
        CpJob &J = jobs[i];
        if (J.to <= J.from) continue;
        if (J.to > ((uint64_t)1 << 31)) fail(IMIN_ERANGE, "world index >= 2^31");
        CpStore &c = *J.c;
        c.cursor.ensure(ctx, 16);
        if (c.worlds == 0) {
            IM_CUDA(cudaMemsetAsync(c.cursor.p, 0, 8, ctx->stream));
            c.count = 0;
        }
        const unsigned long long est =
            (unsigned long long)((double)(J.to - J.from) * std::max(J.per_world, 1.0) * 1.25) + 4096;
        cp_reserve(ctx, c, (unsigned long long)c.count + (store_tight() ? 1 : est));
        TaskRun &t = tr[i];
        t.g = J.g;
        t.q = qdev(*J.q, J.key, J.tag, J.inst);
        t.first = J.from;
        t.count = (uint32_t)(J.to - J.from);
        t.out.credit_L = J.credit;
        t.out.rec_node = c.node.as<int32_t>();
        t.out.rec_par = c.par.as<int32_t>();
        t.out.rec_size = c.size.as<int32_t>();
        t.out.rec_cursor = c.cursor.as<unsigned long long>();
        t.out.rec_cap = c.cap;
        CpStore *cp = &c;
        TaskRun *self = &t;
        const unsigned long long b0 = (unsigned long long)c.count;
        const uint64_t span = J.to - J.from;
        const int32_t n = J.g->n;
        t.grow = [ctx, cp, self, b0, span, n](uint32_t nd) {
            unsigned long long used = 0;
            IM_CUDA(cudaMemcpy(&used, cp->cursor.p, 8, cudaMemcpyDeviceToHost));
            const uint64_t worlds = span > nd ? span - nd : 1;
            const unsigned long long avg = (used - b0) / worlds + 1;
            cp_reserve(ctx, *cp, std::max<unsigned long long>(
                                     2 * cp->cap, used + (unsigned long long)nd * 2 * avg + (unsigned long long)n));
            self->out.rec_node = cp->node.as<int32_t>();
            self->out.rec_par = cp->par.as<int32_t>();
            self->out.rec_size = cp->size.as<int32_t>();
            self->out.rec_cap = cp->cap;
        };
        tp.push_back(&t);
    }
    if (tp.empty()) return;
    Runner run(ctx);
    run.run(tp, WF_LOWER | WF_STORE);
    for (size_t i = 0; i < nj; ++i) {
        CpJob &J = jobs[i];
        if (J.to <= J.from) continue;
        CpStore &c = *J.c;
        unsigned long long used = 0;
        IM_CUDA(cudaMemcpy(&used, c.cursor.p, 8, cudaMemcpyDeviceToHost));
        c.count = (long long)used;
        c.worlds += J.to - J.from;
        if (J.stats) {
            J.stats->worlds += tr[i].acc[4];
            J.stats->edges += tr[i].acc[1];
            J.stats->nodes += tr[i].acc[0];
            J.stats->kernel_ms += run.kernel_ms / (double)tp.size();
            J.stats->launches += (uint64_t)run.launches;
        }
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
    const imin_graph *g;
    const Query *q;
    LrrStore *L;
    uint32_t tag;
    unsigned long long *credit;   // may be null
    uint64_t from, to;
    uint64_t key;
    uint32_t inst;
    SpreadEst *stats;             // may be null
};

void sample_lrr(imin_ctx *ctx, std::vector<LrrJob> &jobs)
{
    const size_t nj = jobs.size();
    std::vector<TaskRun> tr(nj);
    std::vector<TaskRun *> tp;
    for (size_t i = 0; i < nj; ++i) {
        LrrJob &J = jobs[i];
        if (J.to <= J.from) continue;
        if (J.to > ((uint64_t)1 << 31)) fail(IMIN_ERANGE, "world index >= 2^31");
        LrrStore &L = *J.L;
        L.cursor.ensure(ctx, 16);
        if (L.nsets == 0) {
            IM_CUDA(cudaMemsetAsync(L.cursor.p, 0, 8, ctx->stream));
            L.elems = 0;
        }
        // start from the average set size seen so far (64 per world before any is known);
        // test hook: IMIN_STORE_TIGHT=1 starts from almost nothing, so that most worlds
        // take the store-growth (deferred world) path
        const unsigned long long per = L.nsets ? L.elems / L.nsets + 1 : 64;
        if (store_tight())
            lrr_reserve(ctx, L, L.elems + 1, J.to);
        else
            lrr_reserve(ctx, L, L.elems + (J.to - J.from) * per * 2 + 65536, J.to);
        TaskRun &t = tr[i];
        t.g = J.g;
        t.q = qdev(*J.q, J.key, J.tag, J.inst);
        t.first = J.from;
        t.count = (uint32_t)(J.to - J.from);
        t.out.credit_U = J.credit;
        t.out.set_elem = L.elem.as<int32_t>();
        t.out.set_off = L.off.as<unsigned long long>() + J.from;
        t.out.set_len = L.len.as<uint32_t>() + J.from;
        t.out.set_cursor = L.cursor.as<unsigned long long>();
        t.out.set_cap = L.cap;
        LrrStore *lp = &L;
        TaskRun *self = &t;
        const uint64_t from = J.from, to = J.to;
        const int32_t n = J.g->n;
        t.grow = [ctx, lp, self, from, to, n](uint32_t nd) {
            unsigned long long used = 0;
            IM_CUDA(cudaMemcpy(&used, lp->cursor.p, 8, cudaMemcpyDeviceToHost));
            lrr_reserve(ctx, *lp, std::max<unsigned long long>(
                                      2 * lp->cap, used + (unsigned long long)nd * (unsigned long long)n), to);
            self->out.set_elem = lp->elem.as<int32_t>();
            self->out.set_off = lp->off.as<unsigned long long>() + from;
            self->out.set_len = lp->len.as<uint32_t>() + from;
            self->out.set_cap = lp->cap;
        };
        tp.push_back(&t);
    }
    if (tp.empty()) return;
    const char *rev_env = std::getenv("IMIN_GS_REVERSE");
    double rev_ms = 0.0;
    uint64_t rev_launches = 0;
    if (!(rev_env && rev_env[0] == '0')) {
        // Global Sampling worlds backwards from the target (gs_rev.cu): every world with
        // the narrow per-warp tables, the few it cannot hold with the wide ones, and
        // what is left (reverse set still too large, or no store room) forwards below
        const int nt = (int)tp.size();
        // one reverse pass over the worlds lists[i] of task i (all of them when
        // `all`); adds its counters to acc[i] and returns the worlds it leaves, split
        // into too-large (big) and no-store-room (small)
        std::vector<std::array<unsigned long long, 8>> acc_rev(nt);
        for (auto &a8 : acc_rev) a8.fill(0ull);
        auto rev_pass = [&](bool wide, const std::vector<std::vector<uint32_t>> *lists,
                            std::vector<std::vector<uint32_t>> &big, std::vector<std::vector<uint32_t>> &small) {
            DBuf ctl, cd, dt, defl, dl;
            ctl.ensure(ctx, (size_t)nt * CTL);
            IM_CUDA(cudaMemsetAsync(ctl.p, 0, (size_t)nt * CTL, ctx->stream));
            size_t tot = 0, ltot = 0;
            for (int i = 0; i < nt; ++i) {
                tot += tp[i]->count;
                if (lists) ltot += (*lists)[i].size();
            }
            defl.ensure(ctx, tot * 4 + 16);
            if (lists) dl.ensure(ctx, ltot * 4 + 16);
            std::vector<WTask> ht;
            std::vector<int> owner;
            size_t at = 0, lat = 0;
            char *c0 = reinterpret_cast<char *>(ctl.p);
            int maxw = 0;
            for (int i = 0; i < nt; ++i) {
                const uint32_t cnt = lists ? (uint32_t)(*lists)[i].size() : tp[i]->count;
                WorldOut o = tp[i]->out;
                o.acc = reinterpret_cast<unsigned long long *>(c0 + (size_t)i * CTL);
                o.n_deferred = reinterpret_cast<uint32_t *>(c0 + (size_t)i * CTL + 64);
                o.err = reinterpret_cast<uint32_t *>(c0 + (size_t)i * CTL + 68);
                o.deferred = defl.as<uint32_t>() + at;
                o.deferred_cap = tp[i]->count;
                at += tp[i]->count;
                if (cnt == 0) continue;
                const uint32_t *list = nullptr;
                if (lists) {
                    IM_CUDA(cudaMemcpy(dl.as<uint32_t>() + lat, (*lists)[i].data(), (size_t)cnt * 4,
                                       cudaMemcpyHostToDevice));
                    list = dl.as<uint32_t>() + lat;
                    lat += cnt;
                }
                ht.push_back(make_task(tp[i]->g, tp[i]->q, tp[i]->first, cnt, list, o));
                owner.push_back(i);
                maxw += (int)std::min<uint32_t>(cnt, 1u << 20);
            }
            big.assign(nt, {});
            small.assign(nt, {});
            if (ht.empty()) return;
            const int nh = (int)ht.size();
            dt.ensure(ctx, ht.size() * sizeof(WTask));
            cd.ensure(ctx, (size_t)nh * 8 + 16);
            IM_CUDA(cudaMemcpyAsync(dt.p, ht.data(), ht.size() * sizeof(WTask), cudaMemcpyHostToDevice, ctx->stream));
            IM_CUDA(cudaMemsetAsync(cd.p, 0, (size_t)nh * 8, ctx->stream));
            EventTimer et(ctx);
            launch_gs_rev(ctx, dt.as<WTask>(), nh, cd.as<uint32_t>(), cd.as<uint32_t>() + nh, wide,
                          wide ? maxw : 0);
            rev_ms += et.stop();
            rev_launches += 1;
            std::vector<unsigned char> hc((size_t)nt * CTL);
            IM_CUDA(cudaMemcpy(hc.data(), ctl.p, hc.size(), cudaMemcpyDeviceToHost));
            at = 0;
            for (int i = 0; i < nt; ++i) {
                uint32_t e = 0, nd = 0;
                std::memcpy(&e, hc.data() + (size_t)i * CTL + 68, 4);
                if (e) fail(IMIN_EDEVICE, "device invariant failed (reverse Global Sampling)");
                std::memcpy(&nd, hc.data() + (size_t)i * CTL + 64, 4);
                unsigned long long a8[8];
                std::memcpy(a8, hc.data() + (size_t)i * CTL, 64);
                for (int k = 0; k < 8; ++k) acc_rev[i][k] += a8[k];
                if (nd) {
                    std::vector<uint32_t> raw(nd);
                    IM_CUDA(cudaMemcpy(raw.data(), defl.as<uint32_t>() + at, (size_t)nd * 4, cudaMemcpyDeviceToHost));
                    for (uint32_t x : raw) ((x & 0x80000000u) ? big[i] : small[i]).push_back(x & 0x7fffffffu);
                }
                at += tp[i]->count;
            }
        };
        std::vector<std::vector<uint32_t>> big1, small1, big2, small2;
        rev_pass(false, nullptr, big1, small1);
        size_t nbig1 = 0;
        for (auto &v : big1) nbig1 += v.size();
        if (nbig1) rev_pass(true, &big1, big2, small2);
        else {
            big2.assign(nt, {});
            small2.assign(nt, {});
        }
        std::vector<std::vector<uint32_t>> left(nt);
        size_t nleft = 0;
        for (int i = 0; i < nt; ++i) {
            for (auto *v : {&small1[i], &big2[i], &small2[i]}) left[i].insert(left[i].end(), v->begin(), v->end());
            std::sort(left[i].begin(), left[i].end());
            nleft += left[i].size();
        }
        if (const char *trc = std::getenv("IMIN_TRACE"))
            if (trc[0] == '1') {
                size_t w = 0, s1 = 0, b2 = 0, s2 = 0;
                for (int i = 0; i < nt; ++i) {
                    w += tp[i]->count;
                    s1 += small1[i].size();
                    b2 += big2[i].size();
                    s2 += small2[i].size();
                }
                std::fprintf(stderr,
                             "[imin] reverse GS: %zu worlds; %zu too large for the narrow tables, %zu for the wide "
                             "ones; %zu + %zu without store room; %.3f ms\n",
                             w, nbig1, b2, s1, s2, rev_ms);
            }
        std::vector<TaskRun *> keep;
        DBuf dleft;
        if (nleft) {
            dleft.ensure(ctx, nleft * 4 + 16);
            size_t o = 0;
            for (int i = 0; i < nt; ++i) {
                if (left[i].empty()) continue;
                IM_CUDA(cudaMemcpy(dleft.as<uint32_t>() + o, left[i].data(), left[i].size() * 4, cudaMemcpyHostToDevice));
                tp[i]->list = dleft.as<uint32_t>() + o;
                tp[i]->count = (uint32_t)left[i].size();
                o += left[i].size();
                keep.push_back(tp[i]);
            }
        }
        if (!keep.empty()) {
            Runner run(ctx);
            run.run(keep, WF_UPPER | WF_STORE);
            rev_ms += run.kernel_ms;
            rev_launches += (uint64_t)run.launches;
        }
        for (int i = 0; i < nt; ++i) {
            const bool rerun = !left[i].empty();
            for (int k = 0; k < 8; ++k) tp[i]->acc[k] = acc_rev[i][k] + (rerun ? tp[i]->acc[k] : 0ull);
        }
        for (size_t i = 0; i < nj; ++i) {
            LrrJob &J = jobs[i];
            if (J.to <= J.from) continue;
            LrrStore &L = *J.L;
            unsigned long long used = 0;
            IM_CUDA(cudaMemcpy(&used, L.cursor.p, 8, cudaMemcpyDeviceToHost));
            L.elems = used;
            L.nsets = (uint32_t)J.to;
            if (J.stats) {
                J.stats->worlds += tr[i].acc[4];
                J.stats->edges += tr[i].acc[1];
                J.stats->nodes += tr[i].acc[0];
                J.stats->kernel_ms += rev_ms / (double)tp.size();
                J.stats->launches += rev_launches;
            }
        }
        return;
    }
    Runner run(ctx);
    run.run(tp, WF_UPPER | WF_STORE);
    for (size_t i = 0; i < nj; ++i) {
        LrrJob &J = jobs[i];
        if (J.to <= J.from) continue;
        LrrStore &L = *J.L;
        unsigned long long used = 0;
        IM_CUDA(cudaMemcpy(&used, L.cursor.p, 8, cudaMemcpyDeviceToHost));
        L.elems = used;
        L.nsets = (uint32_t)J.to;
        if (J.stats) {
            J.stats->worlds += tr[i].acc[4];
            J.stats->edges += tr[i].acc[1];
            J.stats->nodes += tr[i].acc[0];
            J.stats->kernel_ms += run.kernel_ms / (double)tp.size();
            J.stats->launches += (uint64_t)run.launches;
        }
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

// ---------------------------------------------------------------------------
// Solve (Algorithm 1) as a state machine per instance.  solve_all() advances every
// instance of a batch stage by stage, so each sampling stage is one launch for all
// instances and each Max-Coverage round is one launch per round step; imin_solve is
// a batch of one.  Every instance's result depends on its own query only (worlds are
// addressed by index), so a query gives the same answer alone and in any batch.
// ---------------------------------------------------------------------------
struct Bound {
    bool active = false;
    uint64_t th = 0, from = 0, to = 0;
    int32_t imax = 0, it = 0;
    double a1 = 0.0, a2 = 0.0, th_max = 0.0;
    double sL = 0.0, sU = 0.0;
    unsigned long long cov2 = 0;
    GreedyOut go;
    SpreadEst st;
};

struct Inst {
    imin_graph *g = nullptr;
    int32_t k = 0;
    double eps = 0.0, delta = 0.0, beta = 0.0, gamma = 0.0;
    uint64_t key = 0, fixed_theta = 0;
    uint64_t pr_worlds = 0;   // Pr[s -> v] reading: 0 = q(v), else reach frequency over that many worlds
    uint32_t inst = 0;
    int variant = 0;
    imin_result *res = nullptr;
    int32_t *B_L = nullptr, *B_U = nullptr, *B_R = nullptr, *blockers = nullptr;
    Query q;
    std::vector<int32_t> ON, BLv, BUv, BRv;
    double OPT = 0.0, I_hat = 0.0;
    int32_t nVs = 0;
    bool done = false, do_L = false, do_U = false, do_R = false;
    Bound L, U;
    CpStore C1, C2;
    LrrStore L1, L2;
    DBuf credC1, credL1, inB;
    int stage = 0;            // Stage of the scheduler
    Query qb[3];              // final-estimate queries (S with B_L / B_U / B_R blocked)
    HotView hv;               // relabelled forward index for the final estimates
    bool hv_built = false;
};

void put(int32_t *dst, const std::vector<int32_t> &src)
{
    if (dst) std::copy(src.begin(), src.end(), dst);
}

// validation, ON, q(v), OPT^L and LHGA (host); returns false when ON answers at once
void inst_prepare(imin_ctx *ctx, Inst &I, const int32_t *S_in, int32_t nS)
{
    imin_result *res = I.res;
    if (!(I.eps > 0.0 && I.eps < 1.0) || !(I.delta > 0.0 && I.delta < 1.0) ||
        !(I.beta > 0.0 && I.beta < 1.0) || !(I.gamma > 0.0 && I.gamma < 1.0))
        fail(IMIN_EINVAL, "eps, delta, beta and gamma must lie in (0, 1)");
    if (I.variant < IMIN_SANDIMIN || I.variant > IMIN_LHGA) fail(IMIN_EINVAL, "unknown variant");
    if (I.pr_worlds >= ((uint64_t)1 << 31)) fail(IMIN_EINVAL, "pr_worlds must be below 2^31");
    const int32_t n = I.g->n, k = I.k;
    if (k < 1 || (int64_t)k >= (int64_t)n - nS) fail(IMIN_EINVAL, "k must satisfy 1 <= k < n - |S|");
    std::memset(res, 0, sizeof(*res));
    res->blockers = I.blockers;
    res->B_L = I.B_L;
    res->B_U = I.B_U;
    res->B_R = I.B_R;
    prepare_query(ctx, I.g, I.q, S_in, nS, nullptr, 0, true);
    const imin_graph *g = I.g;
    const std::vector<int32_t> &S = I.q.S;
    // ON: out-neighbours of S with p > 0, not in S (Algorithm 4, line 1)
    std::vector<uint8_t> inON(n, 0);
    for (int32_t s : S)
        for (int32_t e = g->h_row_ptr[s]; e < g->h_row_ptr[s + 1]; ++e)
            if (g->h_thr[e] > 0 && !I.q.is_seed[g->h_col[e]]) inON[g->h_col[e]] = 1;
    for (int32_t v = 0; v < n; ++v)
        if (inON[v]) I.ON.push_back(v);
    I.nVs = I.q.nVs;
    if ((int32_t)I.ON.size() <= k) {   // Algorithm 4, lines 2-3; Sec. 5.3 (nothing sampled)
        put(I.blockers, I.ON);
        put(I.B_L, I.ON);
        put(I.B_U, I.ON);
        put(I.B_R, I.ON);
        res->n_blockers = res->nBL = res->nBU = res->nBR = (int32_t)I.ON.size();
        res->chosen = 0;
        I.done = true;
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
    std::vector<double> pr(n);
    for (int32_t v = 0; v < n; ++v) pr[v] = 1.0 - prod[v];
    // the alternative reading: Pr[s -> v] as the fraction of the worlds
    // 0 .. pr_worlds - 1 of stream tag 6 in which S reaches v
    if (I.pr_worlds > 0) {
        DBuf cnt;
        cnt.ensure(ctx, (size_t)n * 8);
        IM_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)n * 8, ctx->stream));
        TaskRun t;
        t.g = g;
        t.q = qdev(I.q, I.key, TAG_PR, I.inst);
        t.first = 0;
        t.count = (uint32_t)I.pr_worlds;
        t.out.reach = cnt.as<unsigned long long>();
        std::vector<TaskRun *> tp{&t};
        Runner run(ctx);
        run.run(tp, WF_REACH);
        std::vector<unsigned long long> h((size_t)n);
        IM_CUDA(cudaMemcpy(h.data(), cnt.p, (size_t)n * 8, cudaMemcpyDeviceToHost));
        for (int32_t v = 0; v < n; ++v) pr[v] = (double)h[v] / (double)I.pr_worlds;
        res->worlds_sampled += t.acc[4];
        res->edges_scanned += t.acc[1];
    }
    std::vector<ScoreItem> byq(I.ON.size()), bys(I.ON.size());
    for (size_t i = 0; i < I.ON.size(); ++i) {
        const int32_t v = I.ON[i];
        const double qv = pr[v];
        byq[i] = {qv, v};
        bys[i] = {qv * (double)(g->h_row_ptr[v + 1] - g->h_row_ptr[v]), v};
    }
    std::sort(byq.begin(), byq.end(), score_desc);
    std::sort(bys.begin(), bys.end(), score_desc);
    res->nVs = I.nVs;
    double OPT = 0.0;
    for (int32_t i = 0; i < k; ++i) OPT += byq[i].score;
    I.OPT = OPT;
    res->OPT_L = OPT;
    if (!(OPT > 0.0)) fail(IMIN_ERANGE, "OPT^L = 0: no top-k node of ON was reached in the pr_worlds worlds");
    I.BRv.resize(k);
    for (int32_t i = 0; i < k; ++i) I.BRv[i] = bys[i].v;
    I.do_L = I.variant == IMIN_SANDIMIN || I.variant == IMIN_SANDIMIN_MINUS || I.variant == IMIN_LSBM;
    I.do_U = I.variant == IMIN_SANDIMIN || I.variant == IMIN_GSBM;
    I.do_R = I.variant == IMIN_SANDIMIN || I.variant == IMIN_SANDIMIN_MINUS || I.variant == IMIN_LHGA;
}

// theta_max, theta_0, i_max, a1, a2 of LSBM (Algorithm 4 lines 6-10) or GSBM (Sec. 5.2)
void bound_init(Inst &I, Bound &B, bool upper)
{
    const double a = 1.0 - 1.0 / IM_E;
    const int32_t n = I.g->n, nS = (int32_t)I.q.S.size(), k = I.k;
    double th0d;
    if (!upper) {
        const double l12 = std::log(12.0 / I.delta);
        const double c1 = a * std::sqrt(l12) + std::sqrt(a * (ln_binom((double)(n - nS), (double)k) + l12));
        B.th_max = 2.0 * I.I_hat * c1 * c1 / ((1.0 - I.beta) * I.eps * I.eps * I.OPT);
        th0d = std::floor(B.th_max * (1.0 - I.beta) * I.eps * I.eps * I.OPT / I.I_hat);
    } else {
        const double l6 = std::log(6.0 / I.delta);
        int32_t top = I.nVs - nS;
        if (top < k) top = k;
        const double c2 = a * std::sqrt(l6) + std::sqrt(a * (ln_binom((double)top, (double)k) + l6));
        B.th_max = 2.0 * (double)I.nVs * c2 * c2 / (I.eps * I.eps * I.OPT);
        th0d = std::floor(B.th_max * I.eps * I.eps * I.OPT / (double)I.nVs);
    }
    if (th0d < 1.0) th0d = 1.0;
    int32_t imax = (int32_t)std::ceil(std::log2(B.th_max / th0d));
    if (imax < 1) imax = 1;
    uint64_t th = (uint64_t)th0d;
    if (I.fixed_theta) {
        th = I.fixed_theta;
        imax = 1;
    }
    B.th = th;
    B.imax = imax;
    B.a1 = std::log(3.0 * (double)imax / I.delta);
    B.a2 = B.a1;
    B.from = 0;
    B.to = th;
    B.it = 0;
    B.active = true;
}

// sigma^L / sigma^U of one iteration (Algorithm 4 lines 13-19; Sec. 5.2); true = stop
bool bound_check(Inst &I, Bound &B, bool upper, uint64_t n1, uint64_t n2)
{
    const double one_m_inv_e_m_eps = 1.0 - 1.0 / IM_E - I.eps;
    const unsigned long long cov2 = B.cov2;
    if (!upper) {
        const double xlo = (double)cov2 * (1.0 - I.beta) / I.I_hat;
        const double xhi = (double)cov2 * (1.0 + I.beta) / I.I_hat;
        B.sL = 0.0;
        if (xlo >= 5.0 * B.a1 / 18.0)
            B.sL = sigma_low(xlo, B.a1, (double)n2);
        else if (xhi <= 5.0 * B.a1 / 18.0)
            B.sL = sigma_low(xhi, B.a1, (double)n2);
        B.sU = sigma_up((double)B.go.covu * (1.0 + I.beta) / I.I_hat, B.a2, (double)n1);
    } else {
        B.sL = sigma_low((double)cov2, B.a1, (double)n2) * (double)I.nVs;
        B.sU = sigma_up((double)B.go.covu, B.a2, (double)n1) * (double)I.nVs;
    }
    return B.sL / B.sU >= one_m_inv_e_m_eps || B.it == B.imax;
}

// ---------------------------------------------------------------------------
// Scheduler: advances any number of solves (Algorithm 1), each at its own stage.
// Every step runs, for all instances at once: one stop-rule launch (spread
// estimates and final estimates), one lower-bound sampling launch with its batched
// Max-Coverage, and one upper-bound sampling launch with its batched Max-Coverage.
// Instances may be added between steps (continuous batching); a result depends on
// its own query only, because worlds are addressed by index.
// ---------------------------------------------------------------------------
enum Stage { ST_IHAT, ST_LSAMPLE, ST_UGATE, ST_USAMPLE, ST_FINAL, ST_DONE };

struct Scheduler {
    imin_ctx *ctx;
    GreedyBufs gb;
    DBuf d_cov;
    unsigned long long h_cov = 0;
    std::vector<Inst *> active;
    double ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double kms[4] = {0, 0, 0, 0};
    uint64_t reach_launches = 0;
    double final_kms = 0.0;
    uint64_t final_launches = 0;

    explicit Scheduler(imin_ctx *c) : ctx(c) { d_cov.ensure(ctx, 16); }

    void add(Inst *I)
    {
        if (I->done) return;
        I->stage = ST_IHAT;
        active.push_back(I);
    }

    // move an instance to the next bound (or the final estimates) after `from`
    void next_after(Inst &I, int finished)   // finished: -1 none (after I_hat), 0 lower, 1 upper
    {
        if (finished < 0 && I.do_L) {
            start_bound(I, false);
            return;
        }
        if (finished < 1 && I.do_U) {
            start_bound(I, true);
            return;
        }
        start_final(I);
    }

    void start_bound(Inst &I, bool upper)
    {
        bound_init(I, upper ? I.U : I.L, upper);
        DBuf &cred = upper ? I.credL1 : I.credC1;
        const int32_t n = I.g->n;
        cred.ensure(ctx, (size_t)n * 8);
        IM_CUDA(cudaMemsetAsync(cred.p, 0, (size_t)n * 8, ctx->stream));
        I.stage = upper ? ST_USAMPLE : ST_LSAMPLE;
    }

    void start_final(Inst &I)
    {
        I.res->nBR = I.k;
        put(I.B_R, I.BRv);
        const std::vector<int32_t> *cand[3] = {&I.BLv, &I.BUv, &I.BRv};
        const bool use[3] = {I.do_L, I.do_U, I.do_R};
        for (int c = 0; c < 3; ++c) {
            I.res->I_after[c] = 0.0;
            if (!use[c]) continue;
            prepare_query(ctx, I.g, I.qb[c], I.q.S.data(), (int32_t)I.q.S.size(), cand[c]->data(),
                          (int32_t)cand[c]->size(), true);
        }
        I.stage = ST_FINAL;
    }

    void finish(Inst &I)
    {
        imin_result *res = I.res;
        const std::vector<int32_t> *cand[3] = {&I.BLv, &I.BUv, &I.BRv};
        const bool use[3] = {I.do_L, I.do_U, I.do_R};
        int best = -1;
        for (int c = 0; c < 3; ++c)
            if (use[c] && (best < 0 || res->I_after[c] < res->I_after[best])) best = c;
        res->chosen = best;
        res->n_blockers = (int32_t)cand[best]->size();
        put(I.blockers, *cand[best]);
        if (I.do_U && I.variant == IMIN_SANDIMIN && res->DU_hat > 0.0) {
            const double one_m_inv_e_m_eps = 1.0 - 1.0 / IM_E - I.eps;
            const double gr = (1.0 - I.gamma) * (1.0 - I.gamma) / ((1.0 + I.gamma) * (1.0 + I.gamma));
            res->ratio_lb = gr * one_m_inv_e_m_eps * (I.I_hat - res->I_after[1]) / res->DU_hat;
        }
        for (int c = 0; c < 3; ++c) I.qb[c].release();
        I.hv.release();
        I.stage = ST_DONE;
        I.done = true;
    }

    void bound_done(Inst &I, bool upper)
    {
        Bound &B = upper ? I.U : I.L;
        imin_result *res = I.res;
        res->worlds_sampled += B.st.worlds;
        res->edges_scanned += B.st.edges;
        if (!upper) {
            I.BLv = B.go.B;
            res->nBL = (int32_t)I.BLv.size();
            put(I.B_L, I.BLv);
            res->sigmaL_L = B.sL;
            res->sigmaU_L = B.sU;
            res->iters_L = B.it;
            res->theta_C1 = I.C1.worlds;
            res->theta_C2 = I.C2.worlds;
            res->covC2 = B.cov2;
            res->DL_hat = (double)B.cov2 / (double)I.C2.worlds;
            res->theta_max_L = B.th_max;
            I.C1.release();
            I.C2.release();
            I.credC1.release();
        } else {
            I.BUv = B.go.B;
            res->nBU = (int32_t)I.BUv.size();
            put(I.B_U, I.BUv);
            res->sigmaL_U = B.sL;
            res->sigmaU_U = B.sU;
            res->iters_U = B.it;
            res->theta_L1 = I.L1.nsets;
            res->theta_L2 = I.L2.nsets;
            res->covL2 = B.cov2;
            res->DU_hat = (double)I.nVs * (double)B.cov2 / (double)I.L2.nsets;
            res->theta_max_U = B.th_max;
            I.L1.release();
            I.L2.release();
            I.credL1.release();
        }
        next_after(I, upper ? 1 : 0);
    }

    // spread estimates (Algorithm 4, line 4) and final estimates (Algorithm 1, line 4)
    void phase_stop()
    {
        Timer t;
        std::vector<StopSpec> sp;
        std::vector<Inst *> ihat;
        std::vector<FinalSpec> fsp;
        std::vector<Inst *> fin;
        for (Inst *I : active) {
            if (I->stage == ST_IHAT) {
                sp.push_back(StopSpec{I->g, &I->q, I->beta, I->delta / 6.0, I->key, 0u, I->inst, SpreadEst{}});
                ihat.push_back(I);
            } else if (I->stage == ST_FINAL) {
                if (!I->hv_built) {
                    // the relabelled index, built once before the instance's final estimates
                    autotune_reach(ctx, I->g, I->q);
                    const HotStats hs = maybe_hot_view(ctx, I->g, I->q, I->key, I->inst, I->hv);
                    const Query *qb[3] = {&I->qb[0], &I->qb[1], &I->qb[2]};
                    const bool use[3] = {I->do_L, I->do_U, I->do_R};
                    kms[0] += hs.kernel_ms;
                    reach_launches += hs.launches + (uint64_t)hot_view_blocked(ctx, I->hv, qb, use);
                    I->hv_built = true;
                }
                FinalSpec f{};
                f.g = I->g;
                f.q = &I->q;
                for (int c = 0; c < 3; ++c) f.qb[c] = &I->qb[c];
                f.use[0] = I->do_L;
                f.use[1] = I->do_U;
                f.use[2] = I->do_R;
                f.gamma = I->gamma;
                f.delta = I->delta;
                f.key = I->key;
                f.inst = I->inst;
                f.spread_hint = I->I_hat;
                f.hv = &I->hv;
                fsp.push_back(f);
                fin.push_back(I);
            }
        }
        if (sp.empty() && fsp.empty()) return;
        Timer t_ihat;
        if (!sp.empty()) {
            stop_rules(ctx, sp);
            kms[0] += sp[0].est.kernel_ms;
            reach_launches += sp[0].est.launches;
        }
        const double dt_ihat = t_ihat.ms();
        Timer t_fin;
        if (!fsp.empty()) {
            const FinalStats st = final_estimates(ctx, fsp);
            kms[0] += st.kernel_ms;
            reach_launches += st.launches;
            final_kms += st.kernel_ms;
            final_launches += st.launches;
        }
        const double dt_fin = t_fin.ms();
        for (size_t i = 0; i < sp.size(); ++i) {
            Inst &I = *ihat[i];
            const SpreadEst &e = sp[i].est;
            imin_result *res = I.res;
            res->worlds_sampled += e.worlds;
            res->edges_scanned += e.edges;
            res->reach_nodes += e.nodes;
            res->reach_edges += e.edges;
            I.I_hat = e.I;
            res->I_hat = e.I;
            res->n_spread = e.N;
        }
        for (size_t i = 0; i < fsp.size(); ++i) {
            Inst &I = *fin[i];
            imin_result *res = I.res;
            for (int c = 0; c < 3; ++c) {
                if (!fsp[i].use[c]) continue;
                const SpreadEst &e = fsp[i].est[c];
                res->worlds_sampled += e.worlds;
                res->edges_scanned += e.edges;
                res->reach_nodes += e.nodes;
                res->reach_edges += e.edges;
                res->final_entries += e.nodes;
                res->final_edges += e.edges;
                res->I_after[c] = e.I;
                res->n_final[c] = e.N;
            }
        }
        for (Inst *I : ihat) next_after(*I, -1);
        for (Inst *I : fin) finish(*I);
        const double rest = t.ms() - dt_ihat - dt_fin;
        ms[0] += dt_ihat + (fsp.empty() ? rest : 0.0);
        ms[5] += dt_fin + (fsp.empty() ? 0.0 : rest);
    }

    // one doubling round of LSBM (upper = false) or GSBM (upper = true)
    void phase_bound(bool upper)
    {
        const Stage want = upper ? ST_USAMPLE : ST_LSAMPLE;
        std::vector<Inst *> bl;
        for (Inst *I : active)
            if (I->stage == want) bl.push_back(I);
        if (bl.empty()) return;
        Timer ts;
        double kms_before = 0.0;
        for (Inst *I : bl) kms_before += (upper ? I->U : I->L).st.kernel_ms;
        if (!upper) {
            std::vector<CpJob> jobs;
            for (Inst *I : bl) {
                Bound &B = I->L;
                const double per_world = std::max(I->I_hat - (double)I->q.S.size(), 1.0);
                jobs.push_back(CpJob{I->g, &I->q, &I->C1, 1u, I->credC1.as<unsigned long long>(),
                                     B.from, B.to, I->key, I->inst, per_world, &B.st});
                jobs.push_back(CpJob{I->g, &I->q, &I->C2, 2u, nullptr, B.from, B.to, I->key, I->inst,
                                     per_world, &B.st});
            }
            sample_cp(ctx, jobs);
        } else {
            std::vector<LrrJob> jobs;
            for (Inst *I : bl) {
                Bound &B = I->U;
                jobs.push_back(LrrJob{I->g, &I->q, &I->L1, 3u, I->credL1.as<unsigned long long>(),
                                      B.from, B.to, I->key, I->inst, &B.st});
                jobs.push_back(LrrJob{I->g, &I->q, &I->L2, 4u, nullptr, B.from, B.to, I->key, I->inst,
                                      &B.st});
            }
            sample_lrr(ctx, jobs);
        }
        double kms_after = 0.0;
        for (Inst *I : bl) kms_after += (upper ? I->U : I->L).st.kernel_ms;
        kms[upper ? 2 : 1] += kms_after - kms_before;
        ms[upper ? 3 : 1] += ts.ms();
        // Max-Coverage on C1 / L1 of every instance of this round (one batch)
        Timer tg;
        std::vector<GreedyJob> gj(bl.size());
        std::vector<GreedyJob *> gjp;
        for (size_t i = 0; i < bl.size(); ++i) {
            Inst *I = bl[i];
            gj[i].n = I->g->n;
            gj[i].k = I->k;
            if (!upper) {
                gj[i].c = &I->C1;
                gj[i].credit = I->credC1.as<unsigned long long>();
            } else {
                gj[i].L = &I->L1;
                gj[i].credit = I->credL1.as<unsigned long long>();
            }
            gjp.push_back(&gj[i]);
        }
        kms[3] += greedy_batch(ctx, gb, gjp);
        const double t_greedy = tg.ms();
        for (size_t i = 0; i < bl.size(); ++i) {
            Inst &I = *bl[i];
            Bound &B = upper ? I.U : I.L;
            B.go = std::move(gj[i].out);
            B.it += 1;
            set_bitmap_host(ctx, I.inB, I.q.words, B.go.B);
            bool stop;
            if (!upper) {
                B.cov2 = cov_cp(ctx, I.C2, I.inB.as<uint32_t>(), d_cov.as<unsigned long long>(), &h_cov);
                stop = bound_check(I, B, false, I.C1.worlds, I.C2.worlds);
            } else {
                B.cov2 = cov_lrr(ctx, I.L2, I.inB.as<uint32_t>(), d_cov.as<unsigned long long>(), &h_cov);
                stop = bound_check(I, B, true, I.L1.nsets, I.L2.nsets);
            }
            if (stop) {
                bound_done(I, upper);
            } else {
                // double both collections: worlds [th, 2 th)
                B.from = B.th;
                B.to = 2 * B.th;
                B.th *= 2;
            }
        }
        ms[upper ? 4 : 2] += tg.ms();
        if (const char *tr = std::getenv("IMIN_TRACE"))
            if (tr[0] == '1')
                std::fprintf(stderr, "[imin] %s bound step: %zu instance(s), greedy %.2f ms, coverage and check %.2f ms\n",
                             upper ? "upper" : "lower", bl.size(), t_greedy, tg.ms() - t_greedy);
    }

    // one step; returns the instances finished in it
    std::vector<Inst *> step()
    {
        phase_stop();
        phase_bound(false);
        phase_bound(true);
        std::vector<Inst *> fin, keep;
        for (Inst *I : active) (I->done ? fin : keep).push_back(I);
        active.swap(keep);
        return fin;
    }
};

void solve_all(imin_ctx *ctx, std::vector<Inst *> &all)
{
    Timer total;
    const unsigned long long launches0 = g_kernel_launches;
    Scheduler sch(ctx);
    // Instances are admitted as a rolling window: at most `cap` in flight (each holds
    // its sample stores until it finishes), and a new one only while at least a quarter
    // of the device memory is free (the slot arenas count as free: they are caches).
    // The window starts at 64 and widens by 64 after every step that ends with more
    // than half of the device memory free, up to 512: instances grow their stores over
    // several steps, so the window only widens once the ones in flight have shown what
    // they hold.  IMIN_BATCH_ACTIVE="c" fixes the window at c; "c:m" starts it at c and
    // widens it by c up to m.
    int cap = 64, cap_max = 512;
    if (const char *env = std::getenv("IMIN_BATCH_ACTIVE")) {
        char *end = nullptr;
        const long v = std::strtol(env, &end, 10);
        if (v >= 1) {
            cap = cap_max = (int)v;
            if (end && *end == ':') {
                const long m = std::strtol(end + 1, nullptr, 10);
                if (m >= v) cap_max = (int)m;
            }
        }
    }
    const int cap_step = cap;
    auto free_frac = [&]() {
        size_t freeb = 0, totalb = 0;
        cudaMemGetInfo(&freeb, &totalb);
        cudaGetLastError();
        freeb += ctx->slots.bytes + ctx->slots_lower.bytes + ctx->big_slots.bytes + ctx->slots_final.bytes;
        return totalb ? (double)freeb / (double)totalb : 0.0;
    };
    size_t next = 0;
    auto admit = [&]() {
        while (next < all.size() && (int)sch.active.size() < cap) {
            if (!sch.active.empty() && free_frac() < 0.25) break;
            sch.add(all[next++]);
        }
    };
    admit();
    while (!sch.active.empty()) {
        sch.step();
        if (cap < cap_max && next < all.size() && free_frac() > 0.5) cap = std::min(cap_max, cap + cap_step);
        admit();
    }
    sch.ms[7] = total.ms();
    sch.ms[6] = sch.ms[7] - sch.ms[0] - sch.ms[1] - sch.ms[2] - sch.ms[3] - sch.ms[4] - sch.ms[5];
    // stage times and device times belong to the whole batch: every result reports them
    bool any = false;
    for (Inst *I : all) any |= I->stage == ST_DONE;
    for (Inst *I : all) {
        for (int i = 0; i < 8; ++i) I->res->ms_stage[i] = any ? sch.ms[i] : 0.0;
        if (!any) I->res->ms_stage[7] = total.ms();
        for (int i = 0; i < 4; ++i) I->res->kernel_ms[i] = sch.kms[i];
        I->res->reach_launches = sch.reach_launches;
        I->res->final_kernel_ms = sch.final_kms;
        I->res->final_launches = sch.final_launches;
        I->res->kernel_launches = g_kernel_launches - launches0;
    }
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
    case IMIN_EAGAIN: return "not finished yet";
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
    ctx->slots_final.release();
    ctx->stop_spread.release();
    ctx->final_scratch.release();
    for (DBuf *b : {&ctx->vs_vis, &ctx->vs_qa, &ctx->vs_qb, &ctx->vs_hubs, &ctx->vs_ctl, &ctx->vs_cnt, &ctx->vs_tmp})
        b->release();
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

int imin_graph_autotune(imin_graph *g, const int32_t *S, int32_t nS)
{
    if (!g) return IMIN_EINVAL;
    imin_ctx *ctx = g->ctx;
    return run_guarded(ctx, [&] {
        IM_CUDA(cudaSetDevice(ctx->device));
        Query q;
        prepare_query(ctx, g, q, S, nS, nullptr, 0, false);
        autotune_reach(ctx, g, q);
    });
}

int imin_graph_tuning(const imin_graph *g, int32_t out[4])
{
    if (!g || !out) return IMIN_EINVAL;
    out[0] = g->tuned_ctas;
    out[1] = g->tuned_bd;
    out[2] = g->tuned_minb;
    out[3] = g->tuned_smem ? 1 : 0;
    return IMIN_OK;
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

int imin_final_estimates(imin_graph *g, const int32_t *S, int32_t nS, int32_t n_cand, const int32_t *const *B,
                         const int32_t *nB, double gamma, double delta, uint64_t key, uint32_t inst,
                         double spread_hint, double *I_after, uint64_t *n_worlds)
{
    if (!g || !B || !nB || !I_after || !n_worlds || n_cand < 1 || n_cand > 3) return IMIN_EINVAL;
    imin_ctx *ctx = g->ctx;
    return run_guarded(ctx, [&] {
        IM_CUDA(cudaSetDevice(ctx->device));
        if (!(gamma > 0.0 && gamma < 1.0) || !(delta > 0.0 && delta < 1.0))
            fail(IMIN_EINVAL, "gamma and delta must lie in (0, 1)");
        Query q, qb[3];
        prepare_query(ctx, g, q, S, nS, nullptr, 0, false);
        FinalSpec f{};
        f.g = g;
        f.q = &q;
        for (int c = 0; c < 3; ++c) {
            f.qb[c] = &qb[c];
            f.use[c] = c < n_cand;
            if (f.use[c]) prepare_query(ctx, g, qb[c], q.S.data(), (int32_t)q.S.size(), B[c], nB[c], true);
        }
        f.gamma = gamma;
        f.delta = delta;
        f.key = key;
        f.inst = inst;
        f.spread_hint = spread_hint > 0.0 ? spread_hint : 0.0;
        autotune_reach(ctx, g, q);
        HotView hv;
        maybe_hot_view(ctx, g, q, key, inst, hv);
        hot_view_blocked(ctx, hv, f.qb, f.use);
        f.hv = &hv;
        std::vector<FinalSpec> v{f};
        final_estimates(ctx, v);
        for (int c = 0; c < n_cand; ++c) {
            I_after[c] = v[0].est[c].I;
            n_worlds[c] = v[0].est[c].N;
        }
    });
}

int imin_sample_lrr_sequences(imin_graph *g, const int32_t *S, int32_t nS, const int32_t *blocked, int32_t nB,
                              const int32_t *query, int32_t nQ, uint64_t theta, const imin_sample_opts *opts,
                              uint64_t *credit_useq, uint64_t *cov_world, uint64_t totals[5])
{
    if (!g || !opts || !totals || (nQ > 0 && !query)) return IMIN_EINVAL;
    imin_ctx *ctx = g->ctx;
    return run_guarded(ctx, [&] {
        IM_CUDA(cudaSetDevice(ctx->device));
        if (opts->reserved != 0) fail(IMIN_EINVAL, "reserved field must be 0");
        if (opts->first_sample + theta > ((uint64_t)1 << 32) || theta >= ((uint64_t)1 << 31))
            fail(IMIN_ERANGE, "world index >= 2^32 or theta >= 2^31");
        Query q, qq;
        prepare_query(ctx, g, q, S, nS, blocked, nB, false);
        std::vector<int32_t> Qv;
        check_nodes(g, query, nQ, "query set", Qv);
        const int32_t n = g->n;
        cudaStream_t st = ctx->stream;
        DBuf dq, dqbm, dcredit, dcov, dctl, arena;
        const uint32_t *qbm = nullptr;
        if (!Qv.empty()) {
            dq.ensure(ctx, Qv.size() * 4);
            IM_CUDA(cudaMemcpyAsync(dq.p, Qv.data(), Qv.size() * 4, cudaMemcpyHostToDevice, st));
            dqbm.ensure(ctx, q.words * 4);
            fill_bitmap(ctx, dqbm.as<uint32_t>(), q.words, dq.as<int32_t>(), (int32_t)Qv.size());
            qbm = dqbm.as<uint32_t>();
        }
        unsigned long long *pcredit = nullptr, *pcov = nullptr;
        if (credit_useq) {
            dcredit.ensure(ctx, (size_t)n * 8);
            IM_CUDA(cudaMemsetAsync(dcredit.p, 0, (size_t)n * 8, st));
            pcredit = dcredit.as<unsigned long long>();
        }
        if (cov_world && theta > 0) {
            dcov.ensure(ctx, (size_t)theta * 8);
            pcov = dcov.as<unsigned long long>();
        }
        dctl.ensure(ctx, 128);
        IM_CUDA(cudaMemsetAsync(dctl.p, 0, 128, st));
        unsigned long long h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (theta > 0) {
            // every live pair of a world is an edge of the graph, so m pairs always fit;
            // the slot holds min(m, max(2^20, 4 (n + 1))) and a world with more fails the call
            const int32_t ecap = (int32_t)std::min<int64_t>(std::max<int64_t>(g->m, 1),
                                                            std::max<int64_t>(1 << 20, 4 * ((int64_t)n + 1)));
            const size_t per = useq_slot_bytes(n, ecap, nullptr);
            size_t freeb = 0, totalb = 0;
            cudaMemGetInfo(&freeb, &totalb);
            size_t avail = freeb / 2;
            if (ctx->budget)
                avail = std::min(avail, ctx->budget > ctx->in_use ? (ctx->budget - ctx->in_use) / 2 : 0);
            size_t ctas = (size_t)ctx->num_sms * (size_t)std::max(1, std::min(2, useq_blocks_per_sm()));
            ctas = std::min<size_t>(ctas, theta);
            if (per * ctas > avail) ctas = std::max<size_t>(avail / per, 1);
            if (per > freeb) fail(IMIN_ENOMEM, "not enough device memory for an LRR-sequence slot");
            arena.ensure(ctx, per * ctas, false, true);
            IM_CUDA(cudaMemsetAsync(arena.p, 0, arena.bytes, st));
            UseqLaunch L{};
            L.row_ptr = g->row_ptr.as<int32_t>();
            L.ce = g->ce.as<uint4>();
            L.n = n;
            L.S = q.dS.as<int32_t>();
            L.nS = (int32_t)q.S.size();
            L.seed_bm = q.dseed_bm.as<uint32_t>();
            L.blocked_bm = q.blocked.empty() ? nullptr : q.dblk_bm.as<uint32_t>();
            L.query_bm = qbm;
            L.key = opts->key;
            L.tag = opts->tag;
            L.inst = opts->inst;
            L.first = opts->first_sample;
            L.count = (uint32_t)theta;
            L.claim = reinterpret_cast<uint32_t *>(dctl.as<char>() + 64);
            L.slot_base = arena.p;
            L.ecap = ecap;
            L.ctas = (int)ctas;
            L.credit = pcredit;
            L.cov_world = pcov;
            L.acc = dctl.as<unsigned long long>();
            L.err = reinterpret_cast<uint32_t *>(dctl.as<char>() + 68);
            launch_useq(ctx, L);
            IM_CUDA(cudaMemcpyAsync(h, dctl.p, 64, cudaMemcpyDeviceToHost, st));
            uint32_t err = 0;
            IM_CUDA(cudaMemcpyAsync(&err, dctl.as<char>() + 68, 4, cudaMemcpyDeviceToHost, st));
            IM_CUDA(cudaStreamSynchronize(st));
            if (err) fail(IMIN_ERANGE, "a world has more live edges inside its reach set than a slot holds");
        }
        if (credit_useq)
            IM_CUDA(cudaMemcpyAsync(credit_useq, pcredit, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
        if (pcov) IM_CUDA(cudaMemcpyAsync(cov_world, pcov, (size_t)theta * 8, cudaMemcpyDeviceToHost, st));
        IM_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < 5; ++i) totals[i] = h[i];
    });
}

int imin_solve(imin_graph *g, const int32_t *S_in, int32_t nS, int32_t k, double eps, double delta,
               const imin_solve_opts *opts, imin_result *res)
{
    if (!g || !opts || !res || !res->blockers) return IMIN_EINVAL;
    imin_query q;
    q.g = g;
    q.S = S_in;
    q.nS = nS;
    q.k = k;
    q.eps = eps;
    q.delta = delta;
    q.opts = *opts;
    return imin_solve_batch(g->ctx, 1, &q, res);
}

int imin_solve_batch(imin_ctx *ctx, int32_t n_inst, const imin_query *queries, imin_result *results)
{
    if (!ctx || n_inst < 0 || (n_inst > 0 && (!queries || !results))) return IMIN_EINVAL;
    for (int32_t i = 0; i < n_inst; ++i)
        if (!queries[i].g || queries[i].g->ctx != ctx || !results[i].blockers) return IMIN_EINVAL;
    return run_guarded(ctx, [&] {
        IM_CUDA(cudaSetDevice(ctx->device));
        std::vector<std::unique_ptr<Inst>> owned;
        std::vector<Inst *> all;
        for (int32_t i = 0; i < n_inst; ++i) {
            const imin_query &qq = queries[i];
            owned.emplace_back(new Inst());
            Inst &I = *owned.back();
            I.g = qq.g;
            I.k = qq.k;
            I.eps = qq.eps;
            I.delta = qq.delta;
            I.beta = qq.opts.beta;
            I.gamma = qq.opts.gamma;
            I.key = qq.opts.key;
            I.inst = qq.opts.inst;
            I.variant = qq.opts.variant;
            I.fixed_theta = qq.opts.fixed_theta;
            I.pr_worlds = qq.opts.pr_worlds;
            I.res = &results[i];
            I.blockers = results[i].blockers;
            I.B_L = results[i].B_L;
            I.B_U = results[i].B_U;
            I.B_R = results[i].B_R;
            inst_prepare(ctx, I, qq.S, qq.nS);
            all.push_back(&I);
        }
        solve_all(ctx, all);
    });
}

}  // extern "C"

namespace {

// ---------------------------------------------------------------------------
// Server: continuous batching over resident graphs.  A worker thread owns the
// scheduler; queries are admitted between steps while the concurrency limit and the
// device-memory estimate allow, so new queries join launches already serving others.
// ---------------------------------------------------------------------------
struct SrvJob {
    uint64_t ticket = 0;
    imin_query q;
    std::vector<int32_t> S, blockers, BL, BU, BR;
    imin_result res;
    std::unique_ptr<Inst> inst;
    int status = 0;           // 0 queued, 1 running, 2 done, 3 failed
    int err = IMIN_OK;
    size_t mem = 0;
    std::chrono::steady_clock::time_point t_submit, t_done;
};

}  // namespace

struct imin_server {
    imin_ctx *ctx = nullptr;
    int32_t max_active = 64;
    size_t mem_budget = 0;
    size_t mem_in_use = 0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    bool stopping = false;
    std::deque<SrvJob *> pending;
    std::vector<SrvJob *> running;
    std::map<uint64_t, std::unique_ptr<SrvJob>> jobs;
    uint64_t next_ticket = 1;
    uint64_t completed = 0;
    std::string fatal;
};

namespace {

// device bytes a query may need beyond its resident graph (bitmaps, credit and gain
// arrays, V'_s, and collections of a few thousand worlds), used for admission only
size_t query_mem_estimate(const imin_graph *g)
{
    return ((size_t)16 << 20) + (size_t)g->n * 96u;
}

void server_loop(imin_server *srv)
{
    imin_ctx *ctx = srv->ctx;
    cudaSetDevice(ctx->device);
    Scheduler sch(ctx);
    for (;;) {
        std::vector<SrvJob *> admit;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv.wait(lk, [&] { return srv->stopping || !srv->pending.empty() || !srv->running.empty(); });
            if (srv->stopping && srv->pending.empty() && srv->running.empty()) break;
            while (!srv->pending.empty() && (int32_t)srv->running.size() + (int32_t)admit.size() < srv->max_active) {
                SrvJob *j = srv->pending.front();
                if (srv->mem_in_use + j->mem > srv->mem_budget && !(srv->running.empty() && admit.empty()))
                    break;   // wait until memory frees up (a lone query is always admitted)
                srv->pending.pop_front();
                srv->mem_in_use += j->mem;
                j->status = 1;
                admit.push_back(j);
            }
        }
        // prepare the admitted queries (host work and small uploads)
        for (SrvJob *j : admit) {
            const int rc = run_guarded(ctx, [&] { inst_prepare(ctx, *j->inst, j->S.data(), (int32_t)j->S.size()); });
            std::lock_guard<std::mutex> lk(srv->mu);
            if (rc != IMIN_OK) {
                j->status = 3;
                j->err = rc;
                j->t_done = std::chrono::steady_clock::now();
                srv->mem_in_use -= j->mem;
                srv->done_cv.notify_all();
                continue;
            }
            if (j->inst->done) {   // answered by ON at once
                j->status = 2;
                j->t_done = std::chrono::steady_clock::now();
                srv->mem_in_use -= j->mem;
                srv->completed++;
                srv->done_cv.notify_all();
                continue;
            }
            sch.add(j->inst.get());
            srv->running.push_back(j);
        }
        if (sch.active.empty()) continue;
        std::vector<Inst *> fin;
        const int rc = run_guarded(ctx, [&] { fin = sch.step(); });
        std::lock_guard<std::mutex> lk(srv->mu);
        const auto now = std::chrono::steady_clock::now();
        if (rc != IMIN_OK) {
            // a failed step fails every query it was serving
            for (SrvJob *j : srv->running) {
                j->status = 3;
                j->err = rc;
                j->t_done = now;
                srv->mem_in_use -= j->mem;
            }
            srv->running.clear();
            sch.active.clear();
            srv->done_cv.notify_all();
            continue;
        }
        std::vector<SrvJob *> still;
        for (SrvJob *j : srv->running) {
            if (j->inst->done) {
                j->status = 2;
                j->t_done = now;
                j->res.ms_stage[7] =
                    std::chrono::duration<double, std::milli>(now - j->t_submit).count();
                srv->mem_in_use -= j->mem;
                srv->completed++;
            } else {
                still.push_back(j);
            }
        }
        srv->running.swap(still);
        if (!fin.empty()) srv->done_cv.notify_all();
    }
}

}  // namespace

extern "C" {

int imin_server_start(imin_ctx *ctx, const imin_server_opts *opts, imin_server **out)
{
    if (!ctx || !out) return IMIN_EINVAL;
    *out = nullptr;
    imin_server *srv = new (std::nothrow) imin_server();
    if (!srv) return IMIN_ENOMEM;
    srv->ctx = ctx;
    if (opts && opts->max_active > 0) srv->max_active = opts->max_active;
    size_t freeb = 0, totalb = 0;
    cudaSetDevice(ctx->device);
    cudaMemGetInfo(&freeb, &totalb);
    cudaGetLastError();
    srv->mem_budget = (opts && opts->mem_budget) ? (size_t)opts->mem_budget : freeb / 2;
    try {
        srv->worker = std::thread(server_loop, srv);
    } catch (...) {
        delete srv;
        return IMIN_EDEVICE;
    }
    *out = srv;
    return IMIN_OK;
}

int imin_server_submit(imin_server *srv, const imin_query *q, uint64_t *ticket)
{
    if (!srv || !q || !ticket || !q->g || q->g->ctx != srv->ctx || q->nS < 1 || !q->S || q->k < 1)
        return IMIN_EINVAL;
    std::unique_ptr<SrvJob> j(new (std::nothrow) SrvJob());
    if (!j) return IMIN_ENOMEM;
    j->q = *q;
    j->S.assign(q->S, q->S + q->nS);
    j->blockers.resize(q->k);
    j->BL.resize(q->k);
    j->BU.resize(q->k);
    j->BR.resize(q->k);
    std::memset(&j->res, 0, sizeof(j->res));
    j->res.blockers = j->blockers.data();
    j->res.B_L = j->BL.data();
    j->res.B_U = j->BU.data();
    j->res.B_R = j->BR.data();
    j->inst.reset(new Inst());
    Inst &I = *j->inst;
    I.g = q->g;
    I.k = q->k;
    I.eps = q->eps;
    I.delta = q->delta;
    I.beta = q->opts.beta;
    I.gamma = q->opts.gamma;
    I.key = q->opts.key;
    I.inst = q->opts.inst;
    I.variant = q->opts.variant;
    I.fixed_theta = q->opts.fixed_theta;
    I.pr_worlds = q->opts.pr_worlds;
    I.res = &j->res;
    I.blockers = j->res.blockers;
    I.B_L = j->res.B_L;
    I.B_U = j->res.B_U;
    I.B_R = j->res.B_R;
    j->mem = query_mem_estimate(q->g);
    j->t_submit = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stopping) return IMIN_EINVAL;
    j->ticket = srv->next_ticket++;
    *ticket = j->ticket;
    srv->pending.push_back(j.get());
    srv->jobs[j->ticket] = std::move(j);
    srv->cv.notify_all();
    return IMIN_OK;
}

int imin_server_poll(imin_server *srv, uint64_t ticket, int32_t wait_ms, imin_result *res,
                     double *latency_ms)
{
    if (!srv || !res || !res->blockers) return IMIN_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(ticket);
    if (it == srv->jobs.end()) return IMIN_EINVAL;
    SrvJob *j = it->second.get();
    auto ready = [&] { return j->status >= 2; };
    if (!ready()) {
        if (wait_ms > 0)
            srv->done_cv.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
        else if (wait_ms < 0)
            srv->done_cv.wait(lk, ready);
    }
    if (!ready()) return IMIN_EAGAIN;
    if (j->status == 3) {
        const int e = j->err;
        srv->jobs.erase(it);
        return e;
    }
    int32_t *bl = res->blockers, *bL = res->B_L, *bU = res->B_U, *bR = res->B_R;
    *res = j->res;
    res->blockers = bl;
    res->B_L = bL;
    res->B_U = bU;
    res->B_R = bR;
    std::copy(j->blockers.begin(), j->blockers.begin() + j->res.n_blockers, bl);
    if (bL) std::copy(j->BL.begin(), j->BL.begin() + j->res.nBL, bL);
    if (bU) std::copy(j->BU.begin(), j->BU.begin() + j->res.nBU, bU);
    if (bR) std::copy(j->BR.begin(), j->BR.begin() + j->res.nBR, bR);
    if (latency_ms)
        *latency_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count();
    srv->jobs.erase(it);
    return IMIN_OK;
}

int imin_server_stop(imin_server *srv)
{
    if (!srv) return IMIN_EINVAL;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
        srv->cv.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    delete srv;
    return IMIN_OK;
}

}  // extern "C"
