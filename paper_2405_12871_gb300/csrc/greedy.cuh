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
    int32_t pad;
};

struct GreedyBufs {
    DBuf state, part_g, part_v, done, hcnt, hsum, B, cov, topk, gain;
};

// CP records of one collection (C1 or C2), in DT preorder per world.
struct CpStore {
    DBuf node, par, size;          // int32 each, `cap` entries
    DBuf cursor;                   // unsigned long long
    long long count = 0;           // records stored
    unsigned long long cap = 0;
    uint64_t worlds = 0;           // |C|
    DBuf inv_off, inv_rec, fill, contrib, covered, scan_tmp;
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
};

void greedy_scratch(imin_ctx *ctx, GreedyBufs &gb, int32_t n, int32_t k);
void greedy_cp(imin_ctx *ctx, GreedyBufs &gb, CpStore &c, int32_t n, int32_t k,
               const unsigned long long *credit);
void greedy_lrr(imin_ctx *ctx, GreedyBufs &gb, LrrStore &L, int32_t n, int32_t k,
                const unsigned long long *credit);
unsigned long long cov_cp(imin_ctx *ctx, CpStore &c, const uint32_t *inB, unsigned long long *d_out,
                          unsigned long long *h_out);
unsigned long long cov_lrr(imin_ctx *ctx, LrrStore &L, const uint32_t *inB,
                           unsigned long long *d_out, unsigned long long *h_out);
