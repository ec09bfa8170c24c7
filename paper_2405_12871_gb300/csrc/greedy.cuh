// greedy.cuh -- device state of Procedure Max-Coverage and the sample stores.
#pragma once

#include "common.cuh"

// Per-round state, read and written by the round kernels only.
struct GState {
    unsigned long long gmax;    // largest gain this round
    unsigned long long prefix;  // top-k radix select: value bits fixed so far
    unsigned long long tsum;    // top-k radix select: sum of values above the prefix range
    int32_t u;                  // argmax node
    int32_t pick;               // 1 if this round committed a pick
    int32_t stopped;            // 1 once the maximum gain was 0
    int32_t nb;                 // number of picks so far
    int32_t hi;                 // top-k radix select: bits >= hi are fixed
    int32_t krem;               // top-k radix select: values still to take
    int32_t tdone;              // top-k radix select finished
    int32_t npass;              // top-k radix select: digit passes this round needs
};

struct CpStore;
struct LrrStore;

// One Max-Coverage instance as the batched round kernels see it.
struct GInst {
    int32_t n, k;
    const int32_t *cand;     // nodes with a nonzero initial gain, ascending (ncand)
    int32_t ncand;
    unsigned long long *gain;
    GState *st;
    int32_t *B;
    unsigned long long *cov, *topk;
    unsigned int *hcnt;
    unsigned long long *hsum;
    unsigned long long *part_g;
    int32_t *part_v;
    unsigned int *done_ctr;    // argmax blocks finished this round
    unsigned int *done_ctr2;   // histogram blocks finished this pass (persistent kernel)
    int32_t blk0, nblk;      // blocks of the argmax / histogram grids
    int32_t ublk0, unblk;    // blocks of the decrement grid
    const long long *inv_off;
    // CP records
    const long long *inv_rec;
    const long long *inv_cpre;   // running count of update chunks over inv_rec (R + 1)
    const int32_t *rnode, *rpar, *rsize;
    int32_t *contrib;
    uint8_t *covered;
    // LRR sets
    const uint32_t *inv_set;
    const unsigned long long *set_off;
    const uint32_t *set_len;
    const int32_t *set_elem;
};

// Result of one Max-Coverage run: B_i, Cov(B_i), top-k marginal sums, Cov^u.
struct GreedyOut {
    std::vector<int32_t> B;
    std::vector<unsigned long long> cov, topk;
    unsigned long long covu = 0;
};

// A Max-Coverage job: CP records (c) or LRR sets (L), gains initialised from credit.
struct GreedyJob {
    CpStore *c = nullptr;
    LrrStore *L = nullptr;
    int32_t n = 0, k = 0;
    const unsigned long long *credit = nullptr;
    GreedyOut out;
};

struct GreedyBufs {
    DBuf arena, ginst, blkmap, cand, flags, scan_tmp, ncand;
};

// CP records of one collection (C1 or C2), in DT preorder per world.
struct CpStore {
    DBuf node, par, size;          // int32 each, `cap` entries
    DBuf cursor;                   // unsigned long long
    long long count = 0;           // records stored
    unsigned long long cap = 0;
    uint64_t worlds = 0;           // |C|
    DBuf inv_off, inv_rec, inv_cpre, fill, contrib, covered, scan_tmp;
    void release()
    {
        for (DBuf *b : {&node, &par, &size, &cursor, &inv_off, &inv_rec, &inv_cpre, &fill, &contrib, &covered,
                        &scan_tmp})
            b->release();
        count = 0;
        cap = 0;
        worlds = 0;
    }
};

// LRR sets of one collection (L1 or L2), one slot per world (empty sets have len 0).
struct LrrStore {
    DBuf elem;                     // int32, `cap` entries
    DBuf off, len;                 // per world
    DBuf cursor;
    unsigned long long elems = 0;
    unsigned long long cap = 0;
    uint32_t nsets = 0;            // worlds (|L|, empty sets included)
    uint64_t worlds_cap = 0;
    DBuf inv_off, inv_set, fill, covered, scan_tmp;
    void release()
    {
        for (DBuf *b : {&elem, &off, &len, &cursor, &inv_off, &inv_set, &fill, &covered, &scan_tmp})
            b->release();
        elems = 0;
        cap = 0;
        nsets = 0;
        worlds_cap = 0;
    }
};

// Run every job's Max-Coverage together: one launch per round step for all jobs.
// Returns the device time of the round kernels (CUDA events).
double greedy_batch(imin_ctx *ctx, GreedyBufs &gb, std::vector<GreedyJob *> &jobs);
unsigned long long cov_cp(imin_ctx *ctx, CpStore &c, const uint32_t *inB, unsigned long long *d_out,
                          unsigned long long *h_out);
unsigned long long cov_lrr(imin_ctx *ctx, LrrStore &L, const uint32_t *inB,
                           unsigned long long *d_out, unsigned long long *h_out);
