// common.cuh -- internal declarations shared by the library's translation units.
//
// Device-side layout (all resident in HBM):
//   graph:  row_ptr int32[n+1]; ce: one 32-byte record per 4-edge Philox counter group
//           (4 targets, 4 coin thresholds; m rounded up to a multiple of 4, padding
//           threshold 0); col int32[m4] and thr uint32[m4] flat copies; reverse index
//           in_ptr int32[n+1], in_src int32[m], in_eid int32[m], in_thr uint32[m] (thr of
//           the forward edge, for coalescing).
//   slots:  one per world in flight.  CTA-per-world kernels (reach_cta.cuh): one slot
//           per resident CTA (visited bitmap unless it is in shared memory, queue of n + 1,
//           and the bound's arrays).  Warp-per-world kernel (sampler.cu): one slot per
//           resident warp (bitmap, queue of qcap, lower-bound arrays of qcap and ecap);
//           worlds that overflow are re-run on large slots.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/imin.h"

#define IMIN_FULL 0xffffffffu

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32 -> 64-bit
// products on words 0 and 2, high halves mixed with words 1, 3 and the round
// key; the key advances by the two Weyl constants after each round.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t pick_word(const uint4 &w, int i)
{
    return i == 0 ? w.x : (i == 1 ? w.y : (i == 2 ? w.z : w.w));
}

// ---------------------------------------------------------------------------
// Error handling
// ---------------------------------------------------------------------------
struct ImError {
    int code;
    std::string msg;
};

#define IM_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t _e = (call);                                                           \
        if (_e != cudaSuccess)                                                             \
            throw ImError{IMIN_EDEVICE, std::string(#call) + ": " + cudaGetErrorString(_e)}; \
    } while (0)

// process-wide count of kernels the library launched (reported per call)
extern unsigned long long g_kernel_launches;
#define IM_CHECK_LAUNCH()                 \
    do {                                  \
        ++g_kernel_launches;              \
        IM_CUDA(cudaGetLastError());      \
    } while (0)

// Device-side error flags (bit set by kernels, read by the host after a launch).
enum : uint32_t {
    DERR_TIMEOUT = 1u,    // a bounded iteration gave up
    DERR_INTERNAL = 2u,   // an invariant failed (index out of range)
};

// ---------------------------------------------------------------------------
// Device memory: grow-only buffers charged against the context's budget.
// ---------------------------------------------------------------------------
struct imin_ctx;

struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    imin_ctx *ctx = nullptr;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    void release();
    // ensure capacity (contents are NOT preserved unless keep = true); `exact` allocates
    // exactly `need` bytes instead of growing geometrically
    void ensure(imin_ctx *c, size_t need, bool keep = false, bool exact = false);
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

struct imin_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0;      // 0 = none
    size_t in_use = 0;
    int num_sms = 0;
    std::string last_error;
    // scratch shared by calls (grow-only)
    DBuf slots;             // world-kernel slot arena (reach-only and upper-bound worlds)
    DBuf slots_lower;       // slot arena of lower-bound worlds (larger slots, fewer of them)
    DBuf big_slots;         // slots for deferred (oversized) worlds
    DBuf slots_final;       // slots of the fused final estimates
    size_t slots_layout = 0, slots_lower_layout = 0, big_slots_layout = 0, slots_final_layout = 0;
    // L2 persistence for the graph's edge array (0 = not available)
    size_t l2_window_bytes = 0, l2_persist_bytes = 0;
    size_t prev_persist_limit = 0;
    bool persist_set = false;
    // reach-only launch configurations chosen by the autotuner, by graph shape
    struct TuneEntry {
        uint64_t sig;
        int32_t n;
        int64_t m;
        int ctas, bd, minb;
        bool smem;
    };
    std::vector<TuneEntry> tune_cache;
    DBuf misc;              // small per-call device scalars
    DBuf vs_vis, vs_qa, vs_qb, vs_hubs, vs_ctl, vs_cnt, vs_tmp;   // V'_s search work buffers
    DBuf stop_spread;       // per-world sizes of the stopping-rule launches
    DBuf final_scratch;     // per-world candidate sizes and overflow lists of the fused finals
    DBuf hostpin_dummy;
    unsigned long long *h_misc = nullptr;  // pinned host mirror of `misc` scalars
};

void *dev_alloc(imin_ctx *ctx, size_t bytes);
void dev_free(imin_ctx *ctx, void *p, size_t bytes);

// ---------------------------------------------------------------------------
// Graph
// ---------------------------------------------------------------------------
struct imin_graph {
    imin_ctx *ctx = nullptr;
    int32_t n = 0;
    int64_t m = 0, m4 = 0;
    // device
    DBuf row_ptr, col, thr, in_ptr, in_src, in_eid, in_thr;
    DBuf ce;                // per 4-edge group {col x4, thr x4}: one 32-byte sector per group
    size_t ce_bytes = 0;
    // reach-only launch configuration chosen by the autotuner (0 = not tuned yet):
    // tuned_ctas > 0 -> CTA kernel with tuned_bd threads (compiled for tuned_minb CTAs
    // per SM), tuned_smem bitmap in shared memory; tuned_ctas < 0 -> warp-per-world
    // kernel with -tuned_ctas warps per SM
    int tuned_ctas = 0, tuned_bd = 0, tuned_minb = 0;
    bool tuned_smem = false;
    // host copies used by the controller (ON, q(v), out-degrees, V'_s)
    std::vector<int32_t> h_row_ptr, h_col;
    std::vector<uint32_t> h_thr;
};

// ---------------------------------------------------------------------------
// World kernel interface (sampler.cu)
// ---------------------------------------------------------------------------
enum : uint32_t {
    WF_REACH = 1u,       // reach[v] += 1
    WF_LOWER = 2u,       // dominator tree + credit_L
    WF_UPPER = 4u,       // LRR set + credit_U
    WF_STORE = 8u,       // store CP records / LRR sets
    WF_SPREAD = 16u,     // world_spread[rel] = |R_j|
    WF_STOP = 32u,       // stop claiming worlds once the running spread reaches stop_T
};

struct SlotCfg {
    int warps = 0;          // number of slots (= resident warps of the launch)
    int32_t qcap = 0;       // queue / local-array capacity per slot
    int32_t ecap = 0;       // live-edge pair capacity per slot (lower bound only)
    size_t bm_words = 0;    // 32-bit words of one visited bitmap
    bool lower = false, upper = false;
    int groups_per_lane = 2;  // U: 4-edge groups each lane has in flight per step
    int ctas = 0;             // > 0: reach-only worlds run one per CTA (this many CTAs)
    int cta_threads = 1024;   // CTA mode: threads per CTA (the frontier tile)
    int cta_minb = 1;         // CTA mode: CTAs per SM the kernel is compiled for
    bool smem_bm = false;     // CTA mode: visited bitmap in shared memory
    size_t bytes_per_slot() const;
    int slots() const { return ctas > 0 ? ctas : warps; }   // one slot per world in flight
};

// Outputs / stores written by the world kernel.
struct WorldOut {
    unsigned long long *reach = nullptr, *credit_L = nullptr, *credit_U = nullptr;
    uint32_t *world_spread = nullptr;        // indexed by relative world index
    unsigned long long *acc = nullptr;       // [0] spread, [1] edges, [2] nonempty LRR,
                                             // [3] running spread (stop rule), [4] worlds done
    unsigned long long stop_T = 0;
    uint32_t *deferred = nullptr;            // relative indices of worlds to redo
    uint32_t *n_deferred = nullptr;
    uint32_t deferred_cap = 0;
    uint32_t *err = nullptr;
    // CP record store (lower bound)
    int32_t *rec_node = nullptr, *rec_par = nullptr, *rec_size = nullptr;
    unsigned long long *rec_cursor = nullptr;
    unsigned long long rec_cap = 0;
    // LRR set store (upper bound)
    int32_t *set_elem = nullptr;
    unsigned long long *set_off = nullptr;   // [rel world]
    uint32_t *set_len = nullptr;             // [rel world]
    unsigned long long *set_cursor = nullptr;
    unsigned long long set_cap = 0;
};

struct QueryDev {
    const int32_t *S = nullptr;      // device, nS entries (distinct)
    int32_t nS = 0;
    const uint32_t *seed_bm = nullptr;
    const uint32_t *blocked_bm = nullptr;   // may be null
    const int32_t *B = nullptr;      // device, nB blocked nodes (pre-marked in reach-only worlds)
    int32_t nB = 0;
    const int32_t *Vs = nullptr;     // device, sorted ascending
    int32_t nVs = 0;
    uint64_t key = 0;
    uint32_t tag = 0, inst = 0;
};

int world_kernel_blocks_per_sm(uint32_t flags, int U);

// One stream of worlds of one query on one graph: worlds [first, first + count)
// (or first + list[i]) of (key, tag, inst), with its own outputs and stopping rule.
struct WTask {
    const int32_t *row_ptr;
    const uint4 *ce;
    const int32_t *in_ptr, *in_src, *in_eid;
    const uint32_t *in_thr;
    int32_t n;
    QueryDev q;
    uint64_t first;
    uint32_t count;
    const uint32_t *list;
    WorldOut out;
};

WTask make_task(const imin_graph *g, const QueryDev &q, uint64_t first, uint32_t count,
                const uint32_t *list, const WorldOut &out);

// Final estimates of up to three candidate blocker sets on shared worlds (final_cta.cu):
// one traversal per world, a 4-bit field of candidate bits per node.
struct FTask {
    const int32_t *row_ptr;
    const uint4 *ce;
    const int2 *rng;                 // relabelled forward index (HotView), else null: label -> [b, e)
    const uint32_t *gid;             // relabelled forward index: group -> original group index
    const int32_t *S;                // device, nS seeds
    int32_t nS;
    uint32_t cands;                  // candidates served (bits 0..2)
    const int32_t *B[3];             // device blocked lists per candidate
    int32_t nB[3];
    uint64_t key;
    uint32_t tag, inst;
    uint64_t first;
    uint32_t count;
    unsigned long long stop_T[3];    // per candidate: sizes still missing to its threshold
    unsigned long long *acc;         // [0..2] running sizes, [3] queue entries, [4] edges, [5] worlds
    uint32_t *sizes;                 // [count][4]: |R_j| per candidate (0 where not served)
    uint32_t *deferred;              // relative indices of worlds that overflowed the queue
    uint32_t *n_deferred;
    uint32_t deferred_cap;
};
size_t final_slot_bytes(int32_t n, int32_t qcap, size_t *off_queue);
int final_blocks_per_sm(int bd);
void launch_final_tasks(imin_ctx *ctx, const FTask *d_tasks, int ntasks, int32_t nmax, int32_t qcap, int bd,
                        int ctas, void *slot_base, uint32_t *d_claim, uint32_t *d_done);

// Global Sampling worlds traversed backwards from the target (gs_rev.cu): one warp per
// world; worlds whose reverse set outgrows the warp's table are deferred (top bit).
void launch_gs_rev(imin_ctx *ctx, const WTask *d_tasks, int ntasks, uint32_t *d_claim, uint32_t *d_done, bool wide,
                   int max_ctas);

// LRR sequences (useq_cta.cu): the LRR set of every reached node of every world.
struct UseqLaunch {
    const int32_t *row_ptr;
    const uint4 *ce;
    int32_t n;
    const int32_t *S;
    int32_t nS;
    const uint32_t *seed_bm, *blocked_bm, *query_bm;   // blocked / query may be null
    uint64_t key;
    uint32_t tag, inst;
    uint64_t first;
    uint32_t count;
    uint32_t *claim;              // zeroed world counter
    void *slot_base;
    int32_t ecap;                 // live-pair capacity of a slot
    int ctas;
    unsigned long long *credit;   // [n] or null
    unsigned long long *cov_world;// [count] or null
    unsigned long long *acc;      // [0] elements [1] coverage [2] nodes [3] edges [4] worlds
    uint32_t *err;                // bit 4: a world's live pairs exceeded ecap
};
size_t useq_slot_bytes(int32_t n, int32_t ecap, size_t off[10]);
int useq_blocks_per_sm();
void launch_useq(imin_ctx *ctx, const UseqLaunch &L);

// CTA-per-world reach kernel (reach_cta.cuh, sampler_cta.cu): the compiled shapes
// {threads per CTA, CTAs per SM}
extern const int kCtaShapes[][2];
extern const int kNumCtaShapes;
size_t cta_static_smem(int bd, bool lower = false);
size_t cta_slot_bytes(const SlotCfg &cfg);
int cta_blocks_per_sm(int bd, int minb, bool smem_bm, bool upper, bool lower, size_t bm_words);
void launch_cta_tasks(imin_ctx *ctx, const WTask *d_tasks, int ntasks, uint32_t flags,
                      const SlotCfg &cfg, void *slot_base, uint32_t *d_claim, uint32_t *d_done);

// One persistent launch over several tasks (all of the mode given by `flags`).
// d_tasks holds the descriptors; d_claim / d_done are zeroed per-task counters.
void launch_tasks(imin_ctx *ctx, const WTask *d_tasks, int ntasks, const imin_graph *g0,
                  uint32_t flags, const SlotCfg &cfg, void *slot_base, uint32_t *d_claim,
                  uint32_t *d_done);

// ---------------------------------------------------------------------------
// Utilities (graph.cu)
// ---------------------------------------------------------------------------
// V'_s (vs.cu): nodes reachable from S over edges of nonzero probability, avoiding the
// blocked nodes (blk_bm may be null), S excluded; written to `out` in ascending order.
// Returns |V'_s|.
int32_t device_reach_set(imin_ctx *ctx, const imin_graph *g, const int32_t *dS, int32_t nS,
                         const uint32_t *seed_bm, const uint32_t *blk_bm, DBuf &out);

// Relabelled forward index of one query (hot_view.cu).  The final estimates (Algorithm
// 1, line 4) count the nodes each world reaches, and a count does not depend on the nodes' labels as long as
// every edge keeps its coin.  Nodes are relabelled by how often a short run of the
// query's worlds reaches them (most often first); each node's out-edges are copied with
// their whole 4-edge groups into a new group array in label order, each new group
// keeping its original index, from which its coins are drawn.  The worlds' visited
// bitmaps and candidate maps then touch fewer 32-byte sectors, and the group records of
// the nodes most often reached lie together.
struct HotView {
    bool on = false;
    int32_t n = 0;
    DBuf perm;   // int32[n]: node -> label
    DBuf rng;    // int2[n]: label -> [b, e) in the new edge positions
    DBuf ce;     // group records in label order: targets relabelled, thresholds kept
    DBuf gid;    // uint32 per new group: its original group index
    DBuf S;      // the seeds' labels
    DBuf B;      // blocked nodes' labels (the final candidates' lists, concatenated)
    int64_t boff[3] = {0, 0, 0};
    void release()
    {
        for (DBuf *b : {&perm, &rng, &ce, &gid, &S, &B}) b->release();
        on = false;
    }
};
// Builds `hv` from per-node reach counts (each <= max_count) of the query's worlds on
// g; S: device, nS seeds.  Leaves hv.on false when the relabelled edge positions would
// not fit in int32.  Returns the kernel launches it made.
int hot_view_build(imin_ctx *ctx, const imin_graph *g, const unsigned long long *d_counts, uint32_t max_count,
                    const int32_t *d_S, int32_t nS, HotView &hv);
// dst[i] = label of src[i] (device arrays, cnt entries)
void hot_view_map(imin_ctx *ctx, const HotView &hv, const int32_t *d_src, int32_t cnt, int32_t *d_dst);

// exclusive scan of n int64 values in place (d_tmp: >= scan_tmp_bytes(n) bytes)
size_t scan_tmp_bytes(int64_t n);
int scan_launches(int64_t n);   // kernel launches of one scan of n values
void exclusive_scan_i64(imin_ctx *ctx, long long *d, int64_t n, void *d_tmp);
void exclusive_scan_i32(imin_ctx *ctx, int32_t *d, int64_t n, void *d_tmp);
void fill_bitmap(imin_ctx *ctx, uint32_t *bm, size_t words, const int32_t *d_nodes, int32_t cnt);
