// graph.cu -- device memory, graph residency and small device utilities.
//
// Graph load (Sec. 2.1: G = (V, E, p)): the CSR arrays are copied to the device;
// the coin thresholds thr[e] = ceil(p_e * 2^24) and the reverse (in-edge) index
// are derived on the device.  col and thr are padded to a multiple of 4 edges so
// that the sampler can read one Philox counter group (4 edges) with one 16-byte
// load from each array.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstdlib>

unsigned long long g_kernel_launches = 0;

// ---------------------------------------------------------------------------
// device memory accounting
// ---------------------------------------------------------------------------
// The world-kernel slot arenas are caches sized from the free memory at the time of a
// launch; when an allocation does not fit they are dropped (cudaFree waits for the
// device) and re-sized by the next launch.  Returns whether anything was freed.
static bool trim_slot_arenas(imin_ctx *ctx)
{
    bool any = false;
    for (DBuf *b : {&ctx->slots, &ctx->slots_lower, &ctx->big_slots, &ctx->slots_final})
        if (b->p) {
            b->release();
            any = true;
        }
    ctx->slots_layout = ctx->slots_lower_layout = ctx->big_slots_layout = ctx->slots_final_layout = 0;
    return any;
}

void *dev_alloc(imin_ctx *ctx, size_t bytes)
{
    if (bytes == 0) return nullptr;
    if (ctx->budget && ctx->in_use + bytes > ctx->budget) trim_slot_arenas(ctx);
    if (ctx->budget && ctx->in_use + bytes > ctx->budget)
        throw ImError{IMIN_ENOMEM, "device memory budget exceeded (" + std::to_string(ctx->in_use) +
                                       " + " + std::to_string(bytes) + " > " +
                                       std::to_string(ctx->budget) + " bytes)"};
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        if (trim_slot_arenas(ctx)) e = cudaMalloc(&p, bytes);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw ImError{IMIN_ENOMEM, std::string("cudaMalloc(") + std::to_string(bytes) +
                                       "): " + cudaGetErrorString(e)};
    }
    ctx->in_use += bytes;
    return p;
}

void dev_free(imin_ctx *ctx, void *p, size_t bytes)
{
    if (!p) return;
    cudaFree(p);
    if (ctx) ctx->in_use -= bytes;
}

void DBuf::release()
{
    if (p) dev_free(ctx, p, bytes);
    p = nullptr;
    bytes = 0;
}

void DBuf::ensure(imin_ctx *c, size_t need, bool keep, bool exact)
{
    if (need <= bytes && p) return;
    size_t nb = exact ? need : std::max(need, bytes + bytes / 2);
    nb = (nb + 255) & ~(size_t)255;
    void *np = dev_alloc(c, nb);
    if (keep && p && bytes) {
        IM_CUDA(cudaMemcpyAsync(np, p, bytes, cudaMemcpyDeviceToDevice, c->stream));
        IM_CUDA(cudaStreamSynchronize(c->stream));
    }
    release();
    ctx = c;
    p = np;
    bytes = nb;
}

// ---------------------------------------------------------------------------
// scans (three phases: block sums, one-block scan of the sums, add back)
// ---------------------------------------------------------------------------
namespace {

constexpr int SCAN_T = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

template <class T>
__device__ T block_excl_scan(T x, T *sh, T *total)
{
    // sh: SCAN_T / 32 entries
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(IMIN_FULL, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        T s = lane < SCAN_T / 32 ? sh[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(IMIN_FULL, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_T / 32) sh[lane] = s;
    }
    __syncthreads();
    T before = (w > 0 ? sh[w - 1] : T(0)) + v - x;
    if (total) *total = sh[SCAN_T / 32 - 1];
    __syncthreads();
    return before;
}

template <class T>
__global__ void __launch_bounds__(SCAN_T) scan_tiles(T *d, int64_t n, T *tile_sums)
{
    __shared__ T sh[SCAN_T / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < n) ? d[base + k] : T(0);
        s += v[k];
    }
    T tot;
    T before = block_excl_scan<T>(s, sh, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) d[base + k] = before;
        before += v[k];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

template <class T>
__global__ void __launch_bounds__(SCAN_T) scan_add(T *d, int64_t n, const T *tile_off)
{
    const T add = tile_off[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int k = threadIdx.x; k < SCAN_TILE; k += SCAN_T)
        if (base + k < n) d[base + k] += add;
}

template <class T>
void excl_scan(imin_ctx *ctx, T *d, int64_t n, void *tmp)
{
    if (n <= 0) return;
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    T *sums = reinterpret_cast<T *>(tmp);
    scan_tiles<T><<<(unsigned)tiles, SCAN_T, 0, ctx->stream>>>(d, n, sums);
    IM_CHECK_LAUNCH();
    if (tiles > 1) {
        excl_scan<T>(ctx, sums, tiles, sums + ((tiles + 255) & ~255));
        scan_add<T><<<(unsigned)tiles, SCAN_T, 0, ctx->stream>>>(d, n, sums);
        IM_CHECK_LAUNCH();
    }
}

}  // namespace

int scan_launches(int64_t n)
{
    if (n <= 0) return 0;
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    return tiles > 1 ? 2 + scan_launches(tiles) : 1;
}

size_t scan_tmp_bytes(int64_t n)
{
    size_t total = 0;
    int64_t t = n;
    do {
        t = (t + SCAN_TILE - 1) / SCAN_TILE;
        total += (size_t)((t + 255) & ~255) * 8;
    } while (t > 1);
    return total + 256;
}

void exclusive_scan_i64(imin_ctx *ctx, long long *d, int64_t n, void *tmp)
{
    excl_scan<long long>(ctx, d, n, tmp);
}

void exclusive_scan_i32(imin_ctx *ctx, int32_t *d, int64_t n, void *tmp)
{
    excl_scan<int32_t>(ctx, d, n, tmp);
}

// ---------------------------------------------------------------------------
// bitmaps
// ---------------------------------------------------------------------------
namespace {
__global__ void set_bits(uint32_t *bm, const int32_t *nodes, int32_t cnt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) atomicOr(&bm[nodes[i] >> 5], 1u << (nodes[i] & 31));
}
}  // namespace

void fill_bitmap(imin_ctx *ctx, uint32_t *bm, size_t words, const int32_t *d_nodes, int32_t cnt)
{
    IM_CUDA(cudaMemsetAsync(bm, 0, words * 4, ctx->stream));
    if (cnt > 0) {
        set_bits<<<(cnt + 255) / 256, 256, 0, ctx->stream>>>(bm, d_nodes, cnt);
        IM_CHECK_LAUNCH();
    }
}

// ---------------------------------------------------------------------------
// graph construction kernels
// ---------------------------------------------------------------------------
namespace {

// thr[e] = ceil(p * 2^24): the product is exact in fp32 (a power-of-two scale).
__global__ void make_thr(const float *prob, uint32_t *thr, int64_t m, int64_t m4)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m4) return;
    uint32_t t = 0;
    if (e < m) {
        const float x = ceilf(prob[e] * 16777216.0f);
        t = x <= 0.0f ? 0u : (x >= 16777216.0f ? 16777216u : (uint32_t)x);
    }
    thr[e] = t;
}

// interleave: group g -> {col[4g..4g+3], thr[4g..4g+3]} (32 bytes)
__global__ void make_ce(const int32_t *col, const uint32_t *thr, int64_t groups, uint32_t *ce)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // one edge slot
    if (i >= groups * 4) return;
    const int64_t g = i >> 2, c = i & 3;
    ce[8 * g + c] = (uint32_t)col[i];
    ce[8 * g + 4 + c] = thr[i];
}

__global__ void pad_col(int32_t *col, int64_t m, int64_t m4)
{
    const int64_t e = m + threadIdx.x;
    if (e < m4) col[e] = 0;
}

__global__ void count_in(const int32_t *col, int64_t m, int32_t *indeg)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) atomicAdd(indeg + col[e], 1);
}

// one warp per source node: scatter its out-edges into the in-edge lists
__global__ void fill_in(const int32_t *row_ptr, const int32_t *col, const uint32_t *thr, int32_t n,
                        const int32_t *in_ptr, int32_t *fill, int32_t *in_src, int32_t *in_eid,
                        uint32_t *in_thr)
{
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = gw; u < n; u += nw) {
        const int b = row_ptr[u], e = row_ptr[u + 1];
        for (int k = b + lane; k < e; k += 32) {
            const int v = col[k];
            const int pos = in_ptr[v] + atomicAdd(fill + v, 1);
            in_src[pos] = (int32_t)u;
            in_eid[pos] = k;
            in_thr[pos] = thr[k];
        }
    }
}

}  // namespace

void build_device_graph(imin_graph *g, const float *h_prob)
{
    imin_ctx *ctx = g->ctx;
    const int32_t n = g->n;
    const int64_t m = g->m, m4 = g->m4;
    cudaStream_t st = ctx->stream;
    g->row_ptr.ensure(ctx, (size_t)(n + 1) * 4);
    g->col.ensure(ctx, (size_t)std::max<int64_t>(m4, 4) * 4);
    g->thr.ensure(ctx, (size_t)std::max<int64_t>(m4, 4) * 4);
    g->in_ptr.ensure(ctx, (size_t)(n + 1) * 4);
    g->in_src.ensure(ctx, (size_t)std::max<int64_t>(m, 1) * 4);
    g->in_eid.ensure(ctx, (size_t)std::max<int64_t>(m, 1) * 4);
    g->in_thr.ensure(ctx, (size_t)std::max<int64_t>(m, 1) * 4);
    IM_CUDA(cudaMemcpyAsync(g->row_ptr.p, g->h_row_ptr.data(), (size_t)(n + 1) * 4,
                            cudaMemcpyHostToDevice, st));
    if (m > 0)
        IM_CUDA(cudaMemcpyAsync(g->col.p, g->h_col.data(), (size_t)m * 4, cudaMemcpyHostToDevice, st));
    pad_col<<<1, 32, 0, st>>>(g->col.as<int32_t>(), m, m4);
    IM_CHECK_LAUNCH();
    // probabilities: staged through the in_thr buffer (same size), then converted
    if (m > 0)
        IM_CUDA(cudaMemcpyAsync(g->in_thr.p, h_prob, (size_t)m * 4, cudaMemcpyHostToDevice, st));
    if (m4 > 0) {
        make_thr<<<(unsigned)((m4 + 255) / 256), 256, 0, st>>>(g->in_thr.as<float>(),
                                                               g->thr.as<uint32_t>(), m, m4);
        IM_CHECK_LAUNCH();
    } else {
        IM_CUDA(cudaMemsetAsync(g->thr.p, 0, 16, st));
    }
    // interleaved edge groups for the sampler
    {
        const int64_t groups = std::max<int64_t>(m4, 4) / 4;
        g->ce_bytes = (size_t)groups * 32;
        g->ce.ensure(ctx, g->ce_bytes);
        make_ce<<<(unsigned)((groups * 4 + 255) / 256), 256, 0, st>>>(
            g->col.as<int32_t>(), g->thr.as<uint32_t>(), groups, g->ce.as<uint32_t>());
        IM_CHECK_LAUNCH();
    }
    // L2 persistence (context-wide limit, restored by imin_destroy); only when asked for
    if (!ctx->persist_set && std::getenv("IMIN_L2_PERSIST")) {
        int maxp = 0, maxw = 0;
        if (cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, ctx->device) == cudaSuccess &&
            cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, ctx->device) == cudaSuccess &&
            maxp > 0 && maxw > 0) {
            size_t prev = 0;
            if (cudaDeviceGetLimit(&prev, cudaLimitPersistingL2CacheSize) == cudaSuccess &&
                cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, (size_t)maxp) == cudaSuccess) {
                ctx->prev_persist_limit = prev;
                ctx->persist_set = true;
                ctx->l2_persist_bytes = (size_t)maxp;
                ctx->l2_window_bytes = (size_t)maxw;
            }
        }
        cudaGetLastError();
    }
    // reverse index
    DBuf tmp;
    const size_t scan_bytes = scan_tmp_bytes(n + 1);
    tmp.ensure(ctx, (size_t)(n + 1) * 4 + scan_bytes);
    int32_t *fill = tmp.as<int32_t>();
    IM_CUDA(cudaMemsetAsync(g->in_ptr.p, 0, (size_t)(n + 1) * 4, st));
    if (m > 0) {
        count_in<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(g->col.as<int32_t>(), m,
                                                             g->in_ptr.as<int32_t>());
        IM_CHECK_LAUNCH();
    }
    exclusive_scan_i32(ctx, g->in_ptr.as<int32_t>(), n + 1,
                       reinterpret_cast<char *>(tmp.p) + (size_t)(n + 1) * 4);
    IM_CUDA(cudaMemsetAsync(fill, 0, (size_t)(n + 1) * 4, st));
    if (m > 0) {
        const int blocks = std::max(1, std::min<int>(ctx->num_sms * 8, (n + 7) / 8));
        fill_in<<<blocks, 256, 0, st>>>(g->row_ptr.as<int32_t>(), g->col.as<int32_t>(),
                                        g->thr.as<uint32_t>(), n, g->in_ptr.as<int32_t>(), fill,
                                        g->in_src.as<int32_t>(), g->in_eid.as<int32_t>(),
                                        g->in_thr.as<uint32_t>());
        IM_CHECK_LAUNCH();
    }
    IM_CUDA(cudaStreamSynchronize(st));
}
