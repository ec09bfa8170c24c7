// sampler_cta.cu -- host side of the CTA-per-world kernel (reach_cta.cuh): slot
// layout, occupancy and the dispatch over CTA size and CTAs per SM.
#include "reach_cta.cuh"

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

size_t cta_static_smem(int bd) { return reach_cta::static_smem(bd); }

// slot: [visited bitmap unless in shared memory] [queue]; upper-bound worlds add the
// reverse pass's bitmap and queue
size_t cta_slot_bytes(const SlotCfg &cfg)
{
    size_t b = (cfg.smem_bm ? 0 : al16(cfg.bm_words * 4)) + al16((size_t)cfg.qcap * 4);
    if (cfg.upper) b += al16(cfg.bm_words * 4) + al16((size_t)cfg.qcap * 4);
    return b;
}

int cta_blocks_per_sm(int bd, int minb, bool smem_bm, bool upper, size_t bm_words)
{
    const size_t smem = smem_bm ? bm_words * 4 : 0;
    using namespace reach_cta;
    if (bd == 256)
        return minb == 4 ? occupancy<256, 4>(smem_bm, upper, smem) : occupancy<256, 8>(smem_bm, upper, smem);
    if (bd == 512)
        return minb == 2 ? occupancy<512, 2>(smem_bm, upper, smem) : occupancy<512, 4>(smem_bm, upper, smem);
    return minb == 1 ? occupancy<1024, 1>(smem_bm, upper, smem) : occupancy<1024, 2>(smem_bm, upper, smem);
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
    a.off_queue = cfg.smem_bm ? 0 : al16(cfg.bm_words * 4);
    a.off_bm2 = a.off_queue + al16((size_t)cfg.qcap * 4);
    a.off_q2 = a.off_bm2 + al16(cfg.bm_words * 4);
    a.flags = flags;
    const int kind = (flags & WF_UPPER) ? 2 : ((flags & WF_STOP) ? 1 : 0);
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
