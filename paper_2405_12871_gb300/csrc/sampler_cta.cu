// sampler_cta.cu -- host side of the CTA-per-world kernel (reach_cta.cuh): slot
// layout, occupancy and the dispatch over CTA size and CTAs per SM.
#include "reach_cta.cuh"

#include <cstdlib>

namespace reach_cta {
IMIN_REACH_CTA_EXTERN(256, 4)
IMIN_REACH_CTA_EXTERN(256, 8)
IMIN_REACH_CTA_EXTERN(512, 2)
IMIN_REACH_CTA_EXTERN(512, 4)
IMIN_REACH_CTA_EXTERN(1024, 1)
IMIN_REACH_CTA_EXTERN(1024, 2)
}  // namespace reach_cta

namespace {
inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }
}  // namespace

const int kCtaShapes[][2] = {{256, 4}, {256, 8}, {512, 2}, {512, 4}, {1024, 1}, {1024, 2}};
const int kNumCtaShapes = 6;

size_t cta_static_smem(int bd, bool lower) { return reach_cta::static_smem(bd, lower); }

// slot: [visited bitmap unless in shared memory] [queue]; upper-bound worlds add the
// reverse pass's bitmap and queue; lower-bound worlds add node -> position (n), five
// per-position arrays, the level starts and the live edge pairs (ecap each)
static void cta_layout(const SlotCfg &cfg, reach_cta::CArgs *a, size_t *bytes)
{
    const size_t q4 = al16((size_t)cfg.qcap * 4);
    size_t o = cfg.smem_bm ? 0 : al16(cfg.bm_words * 4);
    reach_cta::CArgs t{};
    t.off_queue = o;
    o += q4;
    if (cfg.upper) {
        t.off_bm2 = o;
        o += al16(cfg.bm_words * 4);
        t.off_q2 = o;
        o += q4;
    }
    if (cfg.lower) {
        t.off_loc = o;
        o += al16(cfg.bm_words * 32 * 4);
        size_t *arr[5] = {&t.off_lvl, &t.off_idom, &t.off_sz, &t.off_pre, &t.off_cur};
        for (size_t *x : arr) {
            *x = o;
            o += q4;
        }
        t.off_lstart = o;
        o += al16(((size_t)cfg.qcap + 2) * 4);
        t.off_pu = o;
        o += al16((size_t)cfg.ecap * 4);
        t.off_pv = o;
        o += al16((size_t)cfg.ecap * 4);
    }
    t.ecap = cfg.ecap;
    if (a) {
        a->off_queue = t.off_queue;
        a->off_bm2 = t.off_bm2;
        a->off_q2 = t.off_q2;
        a->off_loc = t.off_loc;
        a->off_lvl = t.off_lvl;
        a->off_idom = t.off_idom;
        a->off_sz = t.off_sz;
        a->off_pre = t.off_pre;
        a->off_cur = t.off_cur;
        a->off_lstart = t.off_lstart;
        a->off_pu = t.off_pu;
        a->off_pv = t.off_pv;
        a->ecap = t.ecap;
    }
    if (bytes) *bytes = o;
}

size_t cta_slot_bytes(const SlotCfg &cfg)
{
    size_t b = 0;
    cta_layout(cfg, nullptr, &b);
    return b;
}

int cta_blocks_per_sm(int bd, int minb, bool smem_bm, bool upper, bool lower, size_t bm_words)
{
    const size_t smem = smem_bm ? bm_words * 4 : 0;
    using namespace reach_cta;
    if (bd == 256)
        return minb == 4 ? occupancy<256, 4>(smem_bm, upper, lower, smem)
                         : occupancy<256, 8>(smem_bm, upper, lower, smem);
    if (bd == 512)
        return minb == 2 ? occupancy<512, 2>(smem_bm, upper, lower, smem)
                         : occupancy<512, 4>(smem_bm, upper, lower, smem);
    return minb == 1 ? occupancy<1024, 1>(smem_bm, upper, lower, smem)
                     : occupancy<1024, 2>(smem_bm, upper, lower, smem);
}

void launch_cta_tasks(imin_ctx *ctx, const WTask *d_tasks, int ntasks, uint32_t flags,
                      const SlotCfg &cfg, void *slot_base, uint32_t *d_claim, uint32_t *d_done)
{
    reach_cta::CArgs a;
    a.tasks = d_tasks;
    a.ntasks = ntasks;
    a.task_claim = d_claim;
    a.task_done = d_done;
    a.slot_base = reinterpret_cast<char *>(slot_base);
    a.slot_bytes = cta_slot_bytes(cfg);
    a.bm_words = cfg.bm_words;
    cta_layout(cfg, &a, nullptr);
    a.flags = flags;
    // tuning knob: IMIN_L2_KEEP=0 loads the graph's group records with the normal L2
    // policy instead of evict-last
    {
        const char *env = std::getenv("IMIN_L2_KEEP");
        a.l2_keep = (env && env[0] == '0') ? 0 : 1;
    }
    const int kind = (flags & WF_LOWER) ? 3 : ((flags & WF_UPPER) ? 2 : ((flags & WF_STOP) ? 1 : 0));
    const size_t smem = cfg.smem_bm ? cfg.bm_words * 4 : 0;
    const int bd = cfg.cta_threads, mb = cfg.cta_minb;
    cudaStream_t st = ctx->stream;
    using namespace reach_cta;
    if (bd == 256) {
        if (mb == 8) launch<256, 8>(st, a, cfg.ctas, cfg.smem_bm, kind, smem);
        else launch<256, 4>(st, a, cfg.ctas, cfg.smem_bm, kind, smem);
    } else if (bd == 512) {
        if (mb == 4) launch<512, 4>(st, a, cfg.ctas, cfg.smem_bm, kind, smem);
        else launch<512, 2>(st, a, cfg.ctas, cfg.smem_bm, kind, smem);
    } else {
        if (mb == 2) launch<1024, 2>(st, a, cfg.ctas, cfg.smem_bm, kind, smem);
        else launch<1024, 1>(st, a, cfg.ctas, cfg.smem_bm, kind, smem);
    }
}
