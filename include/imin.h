/*
 * imin.h -- C ABI of the GB300 influence-minimisation library.
 *
 * The library computes the data-parallel hot path of the Sandwich method for
 * Influence Minimization by node blocking (arXiv 2405.12871): Monte Carlo
 * live-edge worlds of the Independent Cascade model traversed from the seed
 * set S with blocked nodes masked out, the per-world credit of candidate
 * blockers under the lower bound D^L (dominator-tree subtree sizes, i.e. CP
 * sets) and the upper bound D^U (LRR sets), and the greedy selection of k
 * blockers under the LSBM / GSBM stopping rules, combined by Algorithm 1.
 *
 * Conventions for every call:
 *   - Status: every int-returning call returns IMIN_OK (0) or one of the
 *     imin_status codes below.  On error no output is written, except that
 *     imin_solve may have overwritten the blocker arrays' contents.
 *   - Ownership: input arrays are read during the call only and never kept;
 *     the library copies what it needs.  Output arrays are allocated by the
 *     caller.  Graphs stay resident on the device until imin_free_graph.
 *   - Memory: host pointers unless a flag says "device" (then the pointer is a
 *     CUDA device address on the context's device).
 *   - Streams: all device work of a context runs on the stream given to
 *     imin_create (NULL = the legacy default stream); every call returns after
 *     its work has completed.  A context must not be used from two host
 *     threads at once.
 *   - Determinism: results are a pure function of (graph, S, blocked or k,
 *     eps, delta, options).  They do not depend on launch configuration,
 *     batching or co-scheduled work, because world j of stream (key, tag,
 *     inst) is addressed by index: edge e is live in world j iff
 *         (w >> 8) < ceil(p_e * 2^24),  w = word (e & 3) of
 *         Philox4x32-10(ctr = {e >> 2, j, tag, inst}, key = {lo32(key), hi32(key)})
 *     (Sec. 2.1: a realization keeps edge e with probability p(e)).
 */
#ifndef IMIN_H
#define IMIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum imin_status {
    IMIN_OK = 0,
    IMIN_EINVAL = 1,    /* malformed input: row_ptr not monotone, col out of range, p NaN or
                           outside [0,1], duplicate or out-of-range seeds, blocked node in S,
                           k < 1, eps or delta outside (0,1), beta or gamma outside (0,1) */
    IMIN_ERANGE = 2,    /* size limit: n >= 2^31 - 1, m >= 2^31 - 4, a world index >= 2^32,
                           or a per-world structure larger than the library supports */
    IMIN_ENOMEM = 3,    /* device memory budget exceeded, or an allocation failed */
    IMIN_EDEVICE = 4,   /* CUDA error (message available through imin_last_error) */
    IMIN_ETIMEOUT = 5,  /* a bounded device-side wait expired */
    IMIN_EAGAIN = 6     /* imin_server_poll: the query has not finished yet */
};

/* Sampling mode bits for imin_sample_opts.mode. */
enum imin_mode {
    IMIN_REACH = 1,           /* reach[v] = number of worlds whose reach set contains v      */
    IMIN_CREDIT_LOWER = 2,    /* credit_lower[v] = sum over worlds of |N_phi(v)| (Sec. 3.2),
                                 the dominator-tree subtree size of v (Algorithm 2)         */
    IMIN_CREDIT_UPPER = 4,    /* credit_upper[v] = number of worlds whose LRR set holds v
                                 (Algorithm 3, Definition 4.2)                              */
    IMIN_OUT_DEVICE = 0x100   /* output arrays are device pointers                         */
};

/* Solve variants (Algorithm 1 and Sec. 6's SandIMIN-). */
enum imin_variant {
    IMIN_SANDIMIN = 0,        /* B_L (LSBM), B_U (GSBM), B_R (LHGA), argmin of the final estimate */
    IMIN_SANDIMIN_MINUS = 1,  /* without GSBM (alpha_2 = 0)                                  */
    IMIN_LSBM = 2,            /* lower-bound maximisation only                                */
    IMIN_GSBM = 3,            /* upper-bound maximisation only                                */
    IMIN_LHGA = 4             /* heuristic only                                              */
};

typedef struct imin_ctx imin_ctx;       /* opaque, library-owned */
typedef struct imin_graph imin_graph;   /* opaque, library-owned, device-resident */

/* Create a context on CUDA device `device`.  device_mem_budget caps the bytes
 * the context allocates on the device (0 = no cap beyond the device's free
 * memory).  stream is a cudaStream_t (NULL = legacy default stream).
 * Errors: IMIN_EINVAL (bad device), IMIN_EDEVICE. */
int imin_create(imin_ctx **out, int device, size_t device_mem_budget, void *stream);

/* Destroy a context and every buffer it owns.  Graphs loaded through it must
 * have been freed first.  NULL is ignored. */
void imin_destroy(imin_ctx *ctx);

/* Load a directed graph G = (V, E, p) (Sec. 2.1) in CSR-by-source form and keep
 * it resident on the device.
 *   n        number of nodes, 1 <= n < 2^31 - 1
 *   m        number of edges, 0 <= m < 2^31 - 4
 *   row_ptr  host int32[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = m
 *   col      host int32[m], targets in [0, n); self-loops and multi-edges allowed
 *            (each edge is an independent coin)
 *   prob     host float[m], p(u, v) in [0, 1]
 * The library derives the coin thresholds ceil(p * 2^24) and the in-edge
 * (reverse) index on the device.  Errors: IMIN_EINVAL, IMIN_ERANGE,
 * IMIN_ENOMEM, IMIN_EDEVICE. */
int imin_load_graph(imin_ctx *ctx, int32_t n, int64_t m, const int32_t *row_ptr,
                    const int32_t *col, const float *prob, imin_graph **out);

/* Release a graph.  NULL is ignored. */
void imin_free_graph(imin_graph *g);

/* Choose the reach-only launch shape of graph g now (the autotuner otherwise runs on
 * the first stopping-rule estimate that reaches the graph): every compiled CTA shape
 * and the warp-per-world kernel are timed on worlds from the seeds S (a stream no
 * solve draws; no result changes), and the fastest is kept for g and for every graph
 * of the same shape in the context.  A graph that is already tuned is left as it is.
 * Errors: IMIN_EINVAL, IMIN_ENOMEM, IMIN_EDEVICE. */
int imin_graph_autotune(imin_graph *g, const int32_t *S, int32_t nS);

/* The launch configuration the library's autotuner chose for reach-only worlds on
 * this graph (performance only: every configuration gives the same counts).  The
 * first stopping-rule estimate on a graph times a short probe of each configuration
 * and keeps the fastest; graphs of the same shape reuse the choice.
 *   out[0]  > 0: CTAs of the CTA-per-world kernel; < 0: minus the warps per SM of
 *           the warp-per-world kernel; 0: not tuned yet (defaults apply)
 *   out[1]  threads per CTA, out[2] CTAs per SM the kernel was compiled for,
 *   out[3]  1 if the visited bitmap lives in shared memory.
 * Errors: IMIN_EINVAL (NULL argument). */
int imin_graph_tuning(const imin_graph *g, int32_t out[4]);

/* Options of imin_sample.  Worlds [first_sample, first_sample + theta) of the
 * stream (key, tag, inst) are drawn. */
typedef struct imin_sample_opts {
    uint64_t key;           /* Philox key */
    uint32_t tag;           /* stream tag (the solve uses 0..7; see imin_solve) */
    uint32_t inst;          /* instance id (lets independent queries use disjoint streams) */
    uint64_t first_sample;  /* index of the first world */
    uint32_t mode;          /* IMIN_REACH | IMIN_CREDIT_LOWER | IMIN_CREDIT_UPPER [| IMIN_OUT_DEVICE] */
    uint32_t reserved;      /* must be 0 */
} imin_sample_opts;

/* Outputs of imin_sample.  Arrays are caller-allocated (host, or device with
 * IMIN_OUT_DEVICE), NULL = not requested; requested arrays are OVERWRITTEN. */
typedef struct imin_sample_out {
    uint64_t *reach;          /* [n], needs IMIN_REACH */
    uint64_t *credit_lower;   /* [n], needs IMIN_CREDIT_LOWER; 0 for seeds */
    uint64_t *credit_upper;   /* [n], needs IMIN_CREDIT_UPPER; 0 for seeds */
    uint32_t *world_spread;   /* [theta]: |R_j| of each world, seeds included */
    uint64_t total_spread;    /* sum over worlds of |R_j| (seeds count: I_phi(S), Sec. 2.1) */
    uint64_t edges_scanned;   /* sum over worlds of the out-degrees of reached nodes */
    uint64_t nonempty_lrr;    /* worlds whose Global Sampling target was reached (Algorithm 3) */
} imin_sample_out;

/* Monte Carlo sampling of theta live-edge worlds from the seed set S with the
 * blocked set B masked out (Sec. 2.1: a blocker's in-edges get p = 0).
 * Reach counts, lower credit (Algorithm 2 / Lemma 4.1: the credit of v in
 * world j is the number of CP sets of world j that contain v) and upper credit
 * (Algorithm 3 / Lemma 4.2: the target t_j is uniform over V'_s -- the nodes
 * reachable from S in G[V \ B] over edges with p > 0, minus S -- drawn as
 * floor(r64 * |V'_s| / 2^64) with r64 = (out[1] << 32) | out[0] of
 * Philox(ctr = {0xFFFFFFFF, j, tag, inst}) over V'_s sorted ascending; the LRR
 * set holds the nodes of R_j \ S that reach t_j by live edges inside R_j \ S).
 *   S, nS        host int32[nS], 1 <= nS, distinct, in [0, n)
 *   blocked, nB  host int32[nB] (NULL if nB = 0), distinct, in [0, n), disjoint from S
 *   theta        number of worlds, first_sample + theta <= 2^32
 * Errors: IMIN_EINVAL, IMIN_ERANGE, IMIN_ENOMEM, IMIN_EDEVICE. */
int imin_sample(imin_graph *g, const int32_t *S, int32_t nS, const int32_t *blocked, int32_t nB,
                uint64_t theta, const imin_sample_opts *opts, imin_sample_out *out);

/* Final estimates (Algorithm 1, line 4) of given blocker sets: for each of n_cand
 * (1..3) candidate sets B[c] (host int32[nB[c]], distinct, disjoint from S), the
 * (gamma, delta)-estimate of E[I_{G[V \ B[c]}](s)] by the stopping rule (the reading
 * imin_solve uses), all on the worlds of stream tag 5 of (key, inst): the same values
 * imin_solve reports in I_after / n_final for its candidates.  One traversal per world
 * serves every candidate.  On graphs of at least 2^18 nodes whose worlds keep their
 * visited structures in global memory, the traversal runs on a relabelled copy of the
 * forward index (nodes ordered by how often 2,048 worlds of a stream tag no estimate
 * draws reach them; each edge keeps its coin), which changes no value and takes at most
 * 48 B per node + 9 B per edge of device memory while the call runs (imin_solve holds
 * it from its final estimates to its return; 125 MB on a 1M-node, 8.5M-edge graph).  spread_hint: the expected spread without
 * blockers if known (sizes the traversal queue; 0 = unknown).  Outputs: I_after[n_cand], n_worlds[n_cand]
 * (the N each stopping rule chose).  Errors: IMIN_EINVAL, IMIN_ERANGE, IMIN_ENOMEM,
 * IMIN_EDEVICE. */
int imin_final_estimates(imin_graph *g, const int32_t *S, int32_t nS, int32_t n_cand, const int32_t *const *B,
                         const int32_t *nB, double gamma, double delta, uint64_t key, uint32_t inst,
                         double spread_hint, double *I_after, uint64_t *n_worlds);

/* LRR sequences (Sec. 4.2, "Discussion" after Algorithm 3): for each world j of
 * [first_sample, first_sample + theta) of the stream (opts->key, tag, inst), the LRR
 * set L_phi(v) of EVERY node v of phi^s = R_phi(s) \ S (the nodes of phi^s that
 * reach v inside phi^s), one reverse traversal per node -- the estimator of D^U the
 * paper finds too slow on a CPU (Table 2) and replaces by Global Sampling.
 *   S, nS          seeds (as imin_sample); blocked, nB: nodes never entered
 *   query, nQ      host int32[nQ] (NULL if nQ = 0), distinct node ids: the set Q whose
 *                  coverage Cov_{L^s}(Q) is counted
 *   opts           key, tag, inst, first_sample as imin_sample (mode is ignored)
 *   credit_useq    HOST uint64[n] or NULL: sum over worlds of |{v : u in L_phi(v)}|
 *                  (= |M_phi({u})|, the nodes of phi^s that u reaches)
 *   cov_world      HOST uint64[theta] or NULL: per world, |{v : L_phi(v) meets Q}|
 *                  (= |M_phi(Q)|; its mean over worlds estimates D^U(Q) without bias)
 *   totals         HOST uint64[5]: sum of |L_phi(v)|, sum of cov_world, nodes reached
 *                  (seeds included), edges scanned, worlds
 * Outputs are written only on success.  Errors: IMIN_EINVAL, IMIN_ERANGE (world
 * index >= 2^32, or a world with more live edges inside its reach set than a
 * slot holds), IMIN_ENOMEM, IMIN_EDEVICE. */
int imin_sample_lrr_sequences(imin_graph *g, const int32_t *S, int32_t nS, const int32_t *blocked, int32_t nB,
                              const int32_t *query, int32_t nQ, uint64_t theta, const imin_sample_opts *opts,
                              uint64_t *credit_useq, uint64_t *cov_world, uint64_t totals[5]);

/* Options of imin_solve.  Defaults used by the paper (Sec. 6): beta = gamma = 0.1. */
typedef struct imin_solve_opts {
    double beta;            /* relative error of the spread estimate used by LSBM, in (0,1) */
    double gamma;           /* relative error of the final estimates of Algorithm 1, in (0,1) */
    uint64_t key;           /* Philox key */
    uint32_t inst;          /* instance id (stream separation between queries) */
    int32_t variant;        /* imin_variant */
    uint64_t fixed_theta;   /* 0 = the paper's stopping rules; otherwise LSBM and GSBM
                               use theta_0 = fixed_theta and a single iteration */
    uint64_t pr_worlds;     /* Pr[s -> v] in OPT^L (Sec. 5.1) and LHGA (Sec. 5.3): 0 = the
                               direct activation probability q(v) = 1 - prod over seed
                               edges (u, v) of (1 - p_q(u, v)); > 0 = the reach frequency
                               count(v) / pr_worlds over worlds [0, pr_worlds) of stream
                               tag 6 (seeds S, nothing blocked); at most 2^31 - 1.  With
                               it, OPT^L = 0 (no top-k node reached) is IMIN_ERANGE */
} imin_solve_opts;

/* Result of imin_solve.  The four arrays are caller-allocated with room for
 * k entries each (B_L, B_U, B_R may be NULL). */
typedef struct imin_result {
    int32_t *blockers;      /* chosen blocker set (ascending by the order picked) */
    int32_t *B_L, *B_U, *B_R;
    int32_t n_blockers, nBL, nBU, nBR;
    int32_t chosen;         /* 0 = B_L, 1 = B_U, 2 = B_R */
    int32_t iters_L, iters_U;
    int32_t nVs;            /* |V'_s| */
    double I_hat;           /* (beta, delta/6)-estimate of E[I_G(s)] (Algorithm 4, line 4) */
    double I_after[3];      /* (gamma, delta)-estimates of E[I_{G[V\B]}(s)] for B_L, B_U, B_R */
    double sigmaL_L, sigmaU_L, sigmaL_U, sigmaU_U;   /* last sigma^L, sigma^U of LSBM / GSBM */
    double DL_hat;          /* Cov_{C2}(B_L) / |C2| */
    double DU_hat;          /* |V'_s| Cov_{L2}(B_U) / |L2| */
    double ratio_lb;        /* computable approximation-ratio lower bound (Sec. 6.4) */
    double OPT_L;           /* lower bound of D^L(B^o_L) (Sec. 5.1) */
    double theta_max_L, theta_max_U;
    uint64_t n_spread;      /* worlds drawn for I_hat */
    uint64_t theta_C1, theta_C2, theta_L1, theta_L2;  /* final collection sizes */
    uint64_t n_final[3];    /* worlds drawn for each final estimate */
    uint64_t covC2, covL2;  /* Cov_{C2}(B_L), Cov_{L2}(B_U) */
    uint64_t edges_scanned; /* forward edges scanned over the whole solve */
    uint64_t worlds_sampled;/* worlds traversed over the whole solve (incl. speculative ones) */
    double ms_stage[8];     /* wall time per stage: 0 I_hat, 1 LSBM sampling, 2 LSBM greedy,
                               3 GSBM sampling, 4 GSBM greedy, 5 final estimates, 6 host, 7 total */
    double kernel_ms[4];    /* device time (CUDA events on the context's stream) of the world
                               kernel launches: 0 reach-only (the stopping-rule estimates of
                               I_hat and of the three final candidates), 1 lower-bound sampling,
                               2 upper-bound sampling; 3 the greedy rounds */
    uint64_t reach_nodes;   /* nodes reached by the reach-only launches (seeds included) */
    uint64_t reach_edges;   /* edges scanned by the reach-only launches */
    uint64_t reach_launches;/* reach-only world-kernel launches */
    uint64_t kernel_launches; /* kernels the library launched during the call */
    double final_kernel_ms; /* device time of the fused final-estimate launches (part of kernel_ms[0]) */
    uint64_t final_entries; /* queue entries of those launches: nodes reached, one entry per new
                               candidate set (part of reach_nodes) */
    uint64_t final_edges;   /* edges they scanned (part of reach_edges) */
    uint64_t final_launches;/* fused final-estimate launches (part of reach_launches) */
} imin_result;

/* Influence Minimization (problem statement, Sec. 2.1): choose at most k
 * blockers from V \ S by Algorithm 1 (LSBM Algorithm 4, GSBM Sec. 5.2, LHGA
 * Sec. 5.3).  Stream tags: 0 spread estimate, 1/2 CP collections C1/C2,
 * 3/4 LRR collections L1/L2, 5 the final estimates of B_L, B_U and B_R (all
 * three on the same worlds: Algorithm 1, line 4, with common random numbers),
 * 6 the reach frequencies of opts->pr_worlds.
 * Worlds of two more tags are drawn and change no result: 0xFFFFFFF0 times the
 * launch shapes of a graph's first query (the autotuner), 0xFFFFFFF1 orders the
 * labels of the relabelled index the final estimates traverse.
 *   S, nS   host int32[nS], distinct, in [0, n), nS >= 1
 *   k       1 <= k < n - nS
 *   eps     in (0, 1); delta in (0, 1) (the paper uses delta = 1/n)
 * When the out-neighbours ON of S number at most k, ON is returned for every
 * candidate without sampling (Algorithm 4, lines 2-3).
 * Errors: IMIN_EINVAL, IMIN_ERANGE, IMIN_ENOMEM, IMIN_EDEVICE, IMIN_ETIMEOUT. */
int imin_solve(imin_graph *g, const int32_t *S, int32_t nS, int32_t k, double eps, double delta,
               const imin_solve_opts *opts, imin_result *res);

/* One query of a batch: the arguments of imin_solve.  The blocker arrays of the
 * matching imin_result are caller-allocated as for imin_solve. */
typedef struct imin_query {
    imin_graph *g;          /* a graph loaded through the same context */
    const int32_t *S;       /* host int32[nS] */
    int32_t nS;
    int32_t k;
    double eps, delta;
    imin_solve_opts opts;
} imin_query;

/* Batch engine: solve n_inst independent queries (possibly on different graphs of
 * the same context) together.  Each stage of Algorithm 1 -- the spread estimates,
 * every doubling round of LSBM and GSBM, the final estimates -- runs as one
 * persistent launch over all instances still in that stage, and every Max-Coverage
 * round step is one launch for all instances.  results[i] is exactly what
 * imin_solve returns for queries[i] alone (worlds are addressed by index; the
 * batch only changes how they are scheduled); ms_stage and kernel_ms report the
 * whole batch.  Errors: as imin_solve; on error no result is complete. */
int imin_solve_batch(imin_ctx *ctx, int32_t n_inst, const imin_query *queries,
                     imin_result *results);

/* ---------------------------------------------------------------------------
 * Server: continuous batching over graphs resident in one context.  A worker
 * thread owns the context while the server runs (the caller must not use the
 * context from another thread meanwhile).  Submitted queries wait until the
 * concurrency limit and the device-memory estimate admit them; admitted queries
 * join the running scheduler between steps, so their sampling shares launches
 * with the queries already in flight.  Each result is the same as imin_solve
 * returns for that query alone; ms_stage[7] is its latency from submit to done.
 */
typedef struct imin_server imin_server;

typedef struct imin_server_opts {
    int32_t max_active;     /* queries in flight at once (<= 0: 64) */
    int32_t reserved;
    uint64_t mem_budget;    /* device bytes admitted queries may use (0: half the free memory) */
} imin_server_opts;

/* Start a server on ctx.  Errors: IMIN_EINVAL, IMIN_ENOMEM, IMIN_EDEVICE. */
int imin_server_start(imin_ctx *ctx, const imin_server_opts *opts, imin_server **out);

/* Queue a query (its arrays are copied); *ticket identifies it.
 * Errors: IMIN_EINVAL (bad query, graph of another context, server stopping). */
int imin_server_submit(imin_server *srv, const imin_query *q, uint64_t *ticket);

/* Collect a query's result.  wait_ms: 0 = do not wait, > 0 = wait up to that long,
 * < 0 = wait until done.  Returns IMIN_EAGAIN while the query runs, IMIN_OK with the
 * result copied into res (blocker arrays caller-allocated with room for k), or the
 * query's error; a ticket can be collected once.  latency_ms (may be NULL) receives
 * the time from submit to completion. */
int imin_server_poll(imin_server *srv, uint64_t ticket, int32_t wait_ms, imin_result *res,
                     double *latency_ms);

/* Finish every submitted query, stop the worker and free the server. */
int imin_server_stop(imin_server *srv);

/* Static description of a status code. */
const char *imin_strerror(int status);

/* Copy the context's last error message (NUL-terminated, truncated to len). */
void imin_last_error(imin_ctx *ctx, char *buf, size_t len);

/* ---------------------------------------------------------------------------
 * No-allocation variant.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory -- an application whose device
 * memory is reserved in full by its own pooling allocator (for example a
 * framework's caching allocator or a serving process under a hard quota), or a
 * plug-in whose host program does not let it call cudaMalloc.
 *
 * imin_sample_reach_noalloc draws worlds [first_sample, first_sample + theta)
 * of the stream (key, tag, inst) exactly as imin_sample with mode IMIN_REACH
 * does (same coins, same masked BFS from S, no blocked set) and gives the same
 * counts.  It calls no cudaMalloc, cudaFree or allocating library routine: its
 * scratch is one file-scope __device__ array of IMIN_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits.
 *   d_row_ptr, d_col, d_prob  the graph in CSR form (as imin_load_graph), in
 *                             DEVICE memory owned by the caller, n <= IMIN_NOALLOC_MAX_NODES
 *   S, nS                     HOST int32[nS], distinct, in [0, n), 1 <= nS <= 1024
 *   d_reach                   DEVICE uint64[n] or NULL; overwritten with reach counts
 *   d_world_spread            DEVICE uint32[theta] or NULL; |R_j| per world
 *   totals                    HOST uint64[2]: total spread, edges scanned
 *   stream                    cudaStream_t of the caller's device (NULL = legacy default)
 * The device arrays cannot be checked before the launch; the kernel checks each
 * value it uses (row_ptr pairs within [0, m] and non-decreasing, targets in
 * [0, n), probabilities in [0, 1] and not NaN), skips a bad one without reading
 * or writing through it, and the call then returns IMIN_EINVAL with d_reach,
 * d_world_spread and totals unspecified.  Seeds are checked on the host.
 * Throughput: one 8-warp CTA of scratch slots holds n bits plus n + 1 int32 per
 * warp, so the number of worlds in flight falls with n: 8 per SM for small
 * graphs, but at n = 2,000,000 only 8 warps (one CTA) run on the whole GPU,
 * roughly two orders of magnitude below imin_sample on the same graph.
 * The first call made with a given device current looks up the array's device
 * address (cudaGetSymbolAddress) and keeps it; make that first call before any
 * stream capture.  Every call reuses the same array and clears what must start
 * at zero; calls whose GPU work overlaps (other streams, other host threads)
 * race on the array and must be serialised by the caller.  The call returns
 * after its work has completed.
 * Errors: IMIN_EINVAL (NULL pointer, bad seeds, invalid device arrays found by
 * the kernel), IMIN_ERANGE (n above the maximum, more than 1024 seeds, world
 * index >= 2^32), IMIN_EDEVICE. */
#define IMIN_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
#define IMIN_NOALLOC_MAX_NODES 2000000
int imin_sample_reach_noalloc(const int32_t *d_row_ptr, const int32_t *d_col, const float *d_prob,
                              int32_t n, int64_t m, const int32_t *S, int32_t nS, uint64_t theta,
                              uint64_t key, uint32_t tag, uint32_t inst, uint64_t first_sample,
                              uint64_t *d_reach, uint32_t *d_world_spread, uint64_t *totals,
                              void *stream);

#ifdef __cplusplus
}
#endif

#endif /* IMIN_H */
