// noalloc.cu -- reach-only Monte Carlo sampling that allocates no device memory.
//
// Some callers cannot call cudaMalloc: an application whose device memory is
// entirely reserved up front by its own pooling allocator (a framework's caching
// allocator, a serving process with a hard quota), or a plug-in that its host
// program does not allow to allocate device memory behind its back.  For them,
// imin_sample_reach_noalloc runs the reach-only world traversal (the same coins,
// the same masked BFS from the seed set as imin_sample with IMIN_REACH) on graph
// and output arrays the caller already owns, with all of its scratch in one
// file-scope __device__ array of fixed size.
//
// The array is part of the library image: every GPU that loads the library holds
// IMIN_NOALLOC_SCRATCH_BYTES of it until the process exits.  Host code must not
// use its name as an address (it is a host-side shadow); the device address is
// taken once per device with cudaGetSymbolAddress, on the first call made with
// that device current.  Every call reuses the array and it keeps the last call's
// contents, so each call clears the part that must start at zero; two calls whose
// work overlaps on the GPU (on different streams, or from two host threads) race
// on it and must be serialised by the caller.
//
// The graph arrays live in the caller's device memory, so the host cannot check them
// before the launch.  The kernel checks every value it uses instead: a row_ptr pair
// outside [0, m] or decreasing, a target outside [0, n), or a probability that is NaN
// or outside [0, 1] is skipped (nothing is read or written through it) and sets an
// error word that the host turns into IMIN_EINVAL.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>

namespace {

constexpr size_t NOALLOC_BYTES = (size_t)IMIN_NOALLOC_SCRATCH_BYTES;
constexpr int NOALLOC_MAX_SEEDS = 1024;
constexpr size_t HDR = 256;                                  // counters
constexpr size_t SEEDS_OFF = HDR;                            // int32[NOALLOC_MAX_SEEDS]
constexpr size_t SLOTS_OFF = SEEDS_OFF + 4 * NOALLOC_MAX_SEEDS;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_mu;
void *g_base[256] = {nullptr};   // device address of g_noalloc_scratch, per device

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

constexpr size_t ERR_OFF = 128;                              // uint32 error word

struct NArgs {
    const int32_t *row_ptr, *col;
    const float *prob;
    int64_t m;
    int32_t n;
    int32_t nS;
    uint64_t first;
    uint32_t count;
    uint32_t klo, khi, tag, inst;
    unsigned char *base;       // device address of the scratch array
    size_t slot_bytes, bm_words;
    int32_t qcap;
    unsigned long long *reach; // [n] or null
    uint32_t *world_spread;    // [count] or null
};

__device__ __forceinline__ int n_scan(int x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(IMIN_FULL, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// coin threshold ceil(p * 2^24) (an exact power-of-two scaling in fp32)
__device__ __forceinline__ uint32_t n_thr(float p)
{
    const float x = ceilf(p * 16777216.0f);
    return x <= 0.0f ? 0u : (x >= 16777216.0f ? 16777216u : (uint32_t)x);
}

// One warp per world, as in the main sampler; the graph arrays are read one edge at
// a time because the caller's arrays carry no alignment or padding guarantee, and
// every world's queue holds up to n nodes (there is no second, larger pass).
__global__ void __launch_bounds__(256) noalloc_reach_kernel(const NArgs a)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const size_t wid = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(a.base);   // [0] nodes [1] edges
    uint32_t *claim = reinterpret_cast<uint32_t *>(a.base + 64);
    uint32_t *err = reinterpret_cast<uint32_t *>(a.base + ERR_OFF);
    const int32_t *S = reinterpret_cast<const int32_t *>(a.base + SEEDS_OFF);
    unsigned char *slot = a.base + SLOTS_OFF + wid * a.slot_bytes;
    uint32_t *bm = reinterpret_cast<uint32_t *>(slot);
    int32_t *Q = reinterpret_cast<int32_t *>(slot + al16(a.bm_words * 4));
    for (;;) {
        uint32_t rel = 0xffffffffu;
        if (lane == 0) rel = atomicAdd(claim, 1u);
        rel = __shfl_sync(IMIN_FULL, rel, 0);
        if (rel >= a.count) break;
        const uint32_t j = (uint32_t)(a.first + rel);
        for (int i = lane; i < a.nS; i += 32) {
            const int s = S[i];
            atomicOr(&bm[s >> 5], 1u << (s & 31));
            Q[i] = s;
        }
        int tail = a.nS, head = 0;
        unsigned long long wedges = 0;
        __syncwarp();
        while (head < tail) {
            const int fend = tail;
            for (int base = head; base < fend; base += 32) {
                const int i = base + lane;
                int b = 0, e = 0, cnt = 0;
                if (i < fend) {
                    const int u = Q[i];
                    b = a.row_ptr[u];
                    e = a.row_ptr[u + 1];
                    if (b < 0 || e < b || (int64_t)e > a.m) {   // invalid row: skip it
                        atomicOr(err, 1u);
                        b = e = 0;
                    }
                    if (e > b) cnt = ((e + 3) >> 2) - (b >> 2);
                    wedges += (unsigned long long)(e - b);
                }
                const int incl = n_scan(cnt, lane);
                const int total = __shfl_sync(IMIN_FULL, incl, 31);
                for (int t0 = 0; t0 < total; t0 += 32) {
                    const int t = t0 + lane;
                    int lo = 0;
#pragma unroll
                    for (int s = 16; s > 0; s >>= 1) {
                        const int v = __shfl_sync(IMIN_FULL, incl, lo + s - 1);
                        if (v <= t) lo += s;
                    }
                    const int ob = __shfl_sync(IMIN_FULL, b, lo);
                    const int oe = __shfl_sync(IMIN_FULL, e, lo);
                    const int ostart = __shfl_sync(IMIN_FULL, incl - cnt, lo);
                    int nv[4] = {-1, -1, -1, -1};
                    if (t < total) {
                        const int g = (ob >> 2) + (t - ostart);
                        const uint4 w = philox10(make_uint4((uint32_t)g, j, a.tag, a.inst), a.klo, a.khi);
                        const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int ec = (g << 2) + c;
                            if (ec < ob || ec >= oe) continue;
                            const float pe = a.prob[ec];
                            if (!(pe >= 0.0f && pe <= 1.0f)) {   // NaN or outside [0, 1]
                                atomicOr(err, 2u);
                                continue;
                            }
                            if ((wv[c] >> 8) >= n_thr(pe)) continue;
                            const int v = a.col[ec];
                            if (v < 0 || v >= a.n) {
                                atomicOr(err, 4u);
                                continue;
                            }
                            const uint32_t bit = 1u << (v & 31);
                            if (!(atomicOr(&bm[v >> 5], bit) & bit)) nv[c] = v;
                        }
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint32_t bal = __ballot_sync(IMIN_FULL, nv[c] >= 0);
                        if (bal) {
                            const int pos = tail + __popc(bal & lt);
                            if (nv[c] >= 0) Q[pos] = nv[c];    // pos < n: every node enters once
                            tail += __popc(bal);
                        }
                    }
                }
            }
            head = fend;
            __syncwarp();
        }
        if (a.reach)
            for (int i = lane; i < tail; i += 32) atomicAdd(a.reach + Q[i], 1ull);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wedges += __shfl_xor_sync(IMIN_FULL, wedges, o);
        if (lane == 0) {
            atomicAdd(acc + 0, (unsigned long long)tail);
            atomicAdd(acc + 1, wedges);
            if (a.world_spread) a.world_spread[rel] = (uint32_t)tail;
        }
        __syncwarp();
        for (int i = lane; i < tail; i += 32) bm[Q[i] >> 5] = 0;
        __syncwarp();
    }
}

}  // namespace

extern "C" int imin_sample_reach_noalloc(const int32_t *d_row_ptr, const int32_t *d_col,
                                         const float *d_prob, int32_t n, int64_t m,
                                         const int32_t *S, int32_t nS, uint64_t theta,
                                         uint64_t key, uint32_t tag, uint32_t inst,
                                         uint64_t first_sample, uint64_t *d_reach,
                                         uint32_t *d_world_spread, uint64_t *totals,
                                         void *stream)
{
    if (!d_row_ptr || !S || !totals || (m > 0 && (!d_col || !d_prob))) return IMIN_EINVAL;
    if (n < 1 || m < 0 || nS < 1) return IMIN_EINVAL;
    if (n > IMIN_NOALLOC_MAX_NODES || m >= (int64_t)0x7fffffff - 4 || nS > NOALLOC_MAX_SEEDS)
        return IMIN_ERANGE;
    // world indices must stay below 2^32 (written so that the sum cannot wrap)
    if (theta >= ((uint64_t)1 << 32) || first_sample > ((uint64_t)1 << 32) - theta) return IMIN_ERANGE;
    for (int32_t i = 0; i < nS; ++i) {
        if (S[i] < 0 || S[i] >= n) return IMIN_EINVAL;
        for (int32_t k = 0; k < i; ++k)
            if (S[k] == S[i]) return IMIN_EINVAL;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return IMIN_EDEVICE;
    }
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_base[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return IMIN_EDEVICE;
            }
            g_base[dev] = p;
        }
        base = reinterpret_cast<unsigned char *>(g_base[dev]);
    }
    const size_t words = ((size_t)n + 31) / 32;
    const int32_t qcap = n + 1;
    const size_t slot_bytes = al16(words * 4) + al16((size_t)qcap * 4);
    int dev_sms = 0;
    if (cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return IMIN_EDEVICE;
    }
    size_t slots = (NOALLOC_BYTES - SLOTS_OFF) / slot_bytes;
    slots = std::min<size_t>(slots, (size_t)dev_sms * 8);
    slots = slots / 8 * 8;
    if (slots < 8) return IMIN_ERANGE;
    // clear what must start at zero: counters and the visited bitmaps of the slots used
    cudaError_t e = cudaMemsetAsync(base, 0, HDR, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + SLOTS_OFF, 0, slots * slot_bytes, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + SEEDS_OFF, S, (size_t)nS * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && d_reach) e = cudaMemsetAsync(d_reach, 0, (size_t)n * 8, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return IMIN_EDEVICE;
    }
    if (theta > 0) {
        NArgs a;
        a.row_ptr = d_row_ptr;
        a.col = d_col;
        a.prob = d_prob;
        a.m = m;
        a.n = n;
        a.nS = nS;
        a.first = first_sample;
        a.count = (uint32_t)theta;
        a.klo = (uint32_t)key;
        a.khi = (uint32_t)(key >> 32);
        a.tag = tag;
        a.inst = inst;
        a.base = base;
        a.slot_bytes = slot_bytes;
        a.bm_words = words;
        a.qcap = qcap;
        a.reach = reinterpret_cast<unsigned long long *>(d_reach);
        a.world_spread = d_world_spread;
        noalloc_reach_kernel<<<(unsigned)(slots / 8), 256, 0, st>>>(a);
        if (cudaGetLastError() != cudaSuccess) return IMIN_EDEVICE;
    }
    unsigned long long h[2] = {0, 0};
    uint32_t herr = 0;
    e = cudaMemcpyAsync(h, base, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, base + ERR_OFF, sizeof(herr), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return IMIN_EDEVICE;
    }
    if (herr) return IMIN_EINVAL;
    totals[0] = h[0];
    totals[1] = h[1];
    return IMIN_OK;
}
