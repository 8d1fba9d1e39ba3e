// k_reorder_l2.cu -- reorder by a large random index sequence with L2-resident
// passes (dst[i] = src[idx[i]], arXiv:1011.3583 Sec. III.A indexed access).
//
// A direct gather from a source far larger than the L2 pays a whole DRAM
// access (32-64 B) for every element it reads.  Here the source and the
// destination are cut into chunks of about 32 MB (CS elements); element i
// belongs to bucket (c, d) with c = idx[i] / CS and d = i / CS.  The passes:
//   K1 sample    : index locality on 4096 short runs of idx; if most
//                  neighbours are close (|idx[j+1] - idx[j]| <= 16), the
//                  direct gather is already streaming and K2..K6 do nothing,
//                  otherwise K7 does nothing.
//   K2 histogram : bucket sizes.
//   K3 scan      : bucket starts in c-major order, and the d-major work units
//                  of the scatter pass.
//   K4 partition : each 4096-element tile is counting-sorted by c in shared
//                  memory and written as contiguous segments: s-array (source
//                  index) and i-array (destination index), c-major.
//   K5 gather    : v[k] = src[s[k]] walking k in order, so the CTAs in flight
//                  read one ~32 MB source chunk at a time from L2.
//   K6 scatter   : dst[i[k]] = v[k] walking the buckets d-major, so the CTAs
//                  in flight complete one ~32 MB destination chunk in L2.
//   K7 direct    : the plain gather (when K1 found locality).
// Traffic: 2 (idx) + 2 (s, i written) + 2 (s, i read) + 1 (src) + 2 (v) + 1
// (dst) = 10 n-word passes of streaming access instead of n random accesses.
// Scratch ((8 + E) n bytes) comes from a stream-ordered pool owned by the
// library; the kernels are ordered on the caller's stream and none waits on
// another.
#include <cuda_runtime.h>

#include <mutex>

#include "bodies.cuh"
#include "launch.h"

namespace rearr {

namespace {

constexpr int kTile = 4096;        // elements per partition tile / scatter unit
constexpr int kMaxChunks = 512;    // C, D <= 512
constexpr int kSampleRuns = 4096;
constexpr int kSampleLen = 64;
constexpr uint32_t kNear = 16;

struct L2Reorder {
    const char *src;
    char *dst;
    const uint32_t *idx;
    uint32_t n;
    uint32_t cs_shift;             // chunk = 2^cs_shift elements
    uint32_t C, D;                 // source / destination chunks
    unsigned long long *near;      // K1: close neighbour pairs in the sample
    uint32_t *hist;                // [C*D] bucket sizes, c-major (b = c*D + d)
    uint32_t *base;                // [C*D] bucket starts, c-major
    uint32_t *cursor;              // [C*D] partition write cursors
    uint32_t *uprefix;             // [C*D + 1] d-major prefix of scatter units
    uint32_t *sarr, *iarr;         // [n] source / destination indices, c-major
    char *varr;                    // [n] gathered values, c-major
    unsigned long long near_threshold;
};

// Source chunk of an index; clamped so that an index >= n (undefined
// behaviour for the caller) cannot address shared memory out of bounds.
__device__ __forceinline__ uint32_t chunk_of(const L2Reorder &p, uint32_t v)
{
    return min(v >> p.cs_shift, p.C - 1);
}

__device__ __forceinline__ bool bucketed(const L2Reorder &p)
{
    return *reinterpret_cast<volatile unsigned long long *>(p.near) < p.near_threshold;
}

__global__ void __launch_bounds__(kThreads) k_l2_sample(const L2Reorder p)
{
    const uint32_t r = blockIdx.x * kThreads + threadIdx.x;  // one run per thread
    uint32_t cnt = 0;
    if (r < kSampleRuns && p.n > kSampleLen) {
        const uint64_t start = uint64_t(r) * (p.n - kSampleLen) / kSampleRuns;
        uint32_t prev = __ldg(p.idx + start);
        for (int j = 1; j < kSampleLen; ++j) {
            const uint32_t v = __ldg(p.idx + start + j);
            const uint32_t dlt = v > prev ? v - prev : prev - v;
            cnt += dlt <= kNear;
            prev = v;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(p.near, (unsigned long long)cnt);
}

__global__ void __launch_bounds__(kThreads) k_l2_hist(const L2Reorder p)
{
    if (!bucketed(p)) return;
    __shared__ uint32_t sh[kMaxChunks];
    const uint32_t tiles = (p.n + kTile - 1) / kTile;
    for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        for (uint32_t c = threadIdx.x; c < p.C; c += kThreads) sh[c] = 0;
        __syncthreads();
        const uint32_t i0 = t * kTile;
        const uint32_t cnt = min(uint32_t(kTile), p.n - i0);
        for (uint32_t k = threadIdx.x; k < cnt; k += kThreads)
            atomicAdd(&sh[chunk_of(p, __ldg(p.idx + i0 + k))], 1u);
        __syncthreads();
        const uint32_t d = i0 >> p.cs_shift;
        for (uint32_t c = threadIdx.x; c < p.C; c += kThreads)
            if (sh[c]) atomicAdd(&p.hist[c * p.D + d], sh[c]);
        __syncthreads();
    }
}

// Exclusive block-wide scan of one value per thread (1024 threads); returns
// the prefix and the block total in *total.
__device__ __forceinline__ uint32_t block_scan(uint32_t v, uint32_t *warp_sums, uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = warp_sums[lane];
        uint32_t s = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s - w;  // exclusive prefix of the warps
        if (lane == 31) *total = s;
    }
    __syncthreads();
    const uint32_t r = warp_sums[warp] + x - v;
    __syncthreads();
    return r;
}

// One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_l2_scan(const L2Reorder p)
{
    if (!bucketed(p)) return;
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t total;
    const uint32_t nb = p.C * p.D;
    uint32_t carry = 0;
    for (uint32_t b0 = 0; b0 < nb; b0 += 1024) {  // bucket starts, c-major
        const uint32_t b = b0 + threadIdx.x;
        const uint32_t v = b < nb ? p.hist[b] : 0;
        const uint32_t e = block_scan(v, warp_sums, &total);
        if (b < nb) {
            p.base[b] = carry + e;
            p.cursor[b] = carry + e;
        }
        carry += total;
    }
    carry = 0;
    for (uint32_t s0 = 0; s0 < nb; s0 += 1024) {  // scatter units, d-major (s = d*C + c)
        const uint32_t s = s0 + threadIdx.x;
        uint32_t v = 0;
        if (s < nb) {
            const uint32_t d = s / p.C, c = s - d * p.C;
            v = (p.hist[c * p.D + d] + kTile - 1) / kTile;
        }
        const uint32_t e = block_scan(v, warp_sums, &total);
        if (s < nb) p.uprefix[s] = carry + e;
        carry += total;
    }
    if (threadIdx.x == 0) p.uprefix[nb] = carry;
}

__global__ void __launch_bounds__(kThreads) k_l2_partition(const L2Reorder p)
{
    if (!bucketed(p)) return;
    constexpr int PER = kTile / kThreads;  // 16 elements per thread
    __shared__ uint32_t s_st[kTile], i_st[kTile];
    __shared__ uint16_t c_of[kTile];
    __shared__ uint32_t cnt[kMaxChunks], off[kMaxChunks], gb[kMaxChunks];
    __shared__ uint32_t warp_sums[32];
    const uint32_t tiles = (p.n + kTile - 1) / kTile;
    for (uint32_t c = threadIdx.x; c < p.C; c += kThreads) cnt[c] = 0;
    __syncthreads();
    for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint32_t i0 = t * kTile;
        const uint32_t m = min(uint32_t(kTile), p.n - i0);
        const uint32_t d = i0 >> p.cs_shift;
        uint32_t v[PER], rk[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t k = j * kThreads + threadIdx.x;
            v[j] = k < m ? __ldg(p.idx + i0 + k) : 0;
        }
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t k = j * kThreads + threadIdx.x;
            rk[j] = k < m ? atomicAdd(&cnt[chunk_of(p, v[j])], 1u) : 0;
        }
        __syncthreads();
        // segment offsets in the staging buffer (C <= 512: two entries per thread)
        {
            const uint32_t c0 = 2 * threadIdx.x;
            const uint32_t a = c0 < p.C ? cnt[c0] : 0, b = c0 + 1 < p.C ? cnt[c0 + 1] : 0;
            // 256 threads: scan pairs with one warp-level pass per warp + warp sums
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            uint32_t x = a + b;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) warp_sums[warp] = x;
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t s = 0;
                for (int w = 0; w < kThreads / 32; ++w) {
                    const uint32_t q = warp_sums[w];
                    warp_sums[w] = s;
                    s += q;
                }
            }
            __syncthreads();
            const uint32_t e = warp_sums[warp] + x - (a + b);
            if (c0 < p.C) off[c0] = e;
            if (c0 + 1 < p.C) off[c0 + 1] = e + a;
            if (c0 < p.C && a) gb[c0] = atomicAdd(&p.cursor[c0 * p.D + d], a);
            if (c0 + 1 < p.C && b) gb[c0 + 1] = atomicAdd(&p.cursor[(c0 + 1) * p.D + d], b);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t k = j * kThreads + threadIdx.x;
            if (k < m) {
                const uint32_t c = chunk_of(p, v[j]);
                const uint32_t pos = off[c] + rk[j];
                s_st[pos] = v[j];
                i_st[pos] = i0 + k;
                c_of[pos] = uint16_t(c);
            }
        }
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < m; q += kThreads) {
            const uint32_t c = c_of[q];
            const uint32_t g = gb[c] + (q - off[c]);
            p.sarr[g] = s_st[q];
            p.iarr[g] = i_st[q];
        }
        for (uint32_t c = threadIdx.x; c < p.C; c += kThreads) cnt[c] = 0;
        __syncthreads();
    }
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_l2_gather(const L2Reorder p, const GatherDesc g, uint64_t units,
                                                        int want_bucketed)
{
    if (bucketed(p) != bool(want_bucketed)) return;
    for (uint64_t u = blockIdx.x; u < units; u += gridDim.x) gather_body<W>(g, u);
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_l2_scatter(const L2Reorder p, uint32_t max_units)
{
    if (!bucketed(p)) return;
    using T = typename Word<W>::T;
    const uint32_t nb = p.C * p.D;
    const uint32_t total = p.uprefix[nb];
    for (uint32_t u = blockIdx.x; u < total && u < max_units; u += gridDim.x) {
        // d-major segment s with uprefix[s] <= u < uprefix[s + 1]
        uint32_t lo = 0, hi = nb - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (p.uprefix[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        const uint32_t d = lo / p.C, c = lo - d * p.C;
        const uint32_t b = c * p.D + d;
        const uint32_t piece = u - p.uprefix[lo];
        const uint32_t k0 = p.base[b] + piece * kTile;
        const uint32_t k1 = p.base[b] + min(p.hist[b], (piece + 1) * uint32_t(kTile));
        constexpr int U = 4;
        for (uint32_t kb = k0; kb < k1; kb += kThreads * U) {
            uint32_t di[U];
            T val[U];
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const uint32_t k = kb + j * kThreads + threadIdx.x;
                if (k < k1) {
                    di[j] = __ldg(p.iarr + k);
                    val[j] = ldg_stream<W>(p.varr + uint64_t(k) * W);
                }
            }
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const uint32_t k = kb + j * kThreads + threadIdx.x;
                if (k < k1) stg<W>(p.dst + uint64_t(di[j]) * W, val[j]);
            }
        }
    }
}

std::mutex g_pool_mu;
cudaMemPool_t g_pool[64];
bool g_pool_ready[64];

cudaError_t get_pool(cudaMemPool_t &pool)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool_ready[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&g_pool[dev], &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;  // keep freed scratch in the pool for the next call
        cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool_ready[dev] = true;
    }
    pool = g_pool[dev];
    return cudaSuccess;
}

template <int W>
cudaError_t run_l2(const GatherDesc &g, cudaStream_t s)
{
    L2Reorder p = {};
    p.src = g.src;
    p.dst = g.dst;
    p.idx = g.idx;
    p.n = uint32_t(g.n);
    // ~32 MB chunks, at most kMaxChunks of them
    uint32_t shift = 0;
    while ((uint64_t(1) << shift) * W < (uint64_t(32) << 20)) ++shift;
    while (((uint64_t(g.n) + (uint64_t(1) << shift) - 1) >> shift) > kMaxChunks) ++shift;
    p.cs_shift = shift;
    p.C = p.D = uint32_t((uint64_t(g.n) + (uint64_t(1) << shift) - 1) >> shift);
    const uint32_t nb = p.C * p.D;
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t off_hist = 256, off_base = off_hist + al(nb * 4), off_cur = off_base + al(nb * 4),
                 off_up = off_cur + al(nb * 4), off_s = off_up + al((nb + 1) * 4), off_i = off_s + al(size_t(g.n) * 4),
                 off_v = off_i + al(size_t(g.n) * 4), bytes = off_v + al(size_t(g.n) * W);
    cudaMemPool_t pool;
    cudaError_t e = get_pool(pool);
    if (e != cudaSuccess) return e;
    char *scratch = nullptr;
    e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&scratch), bytes, pool, s);
    if (e != cudaSuccess) return e;
    p.near = reinterpret_cast<unsigned long long *>(scratch);
    p.hist = reinterpret_cast<uint32_t *>(scratch + off_hist);
    p.base = reinterpret_cast<uint32_t *>(scratch + off_base);
    p.cursor = reinterpret_cast<uint32_t *>(scratch + off_cur);
    p.uprefix = reinterpret_cast<uint32_t *>(scratch + off_up);
    p.sarr = reinterpret_cast<uint32_t *>(scratch + off_s);
    p.iarr = reinterpret_cast<uint32_t *>(scratch + off_i);
    p.varr = scratch + off_v;
    const uint64_t pairs = uint64_t(kSampleRuns) * (kSampleLen - 1);
    p.near_threshold = pairs / 2;
    e = cudaMemsetAsync(scratch, 0, off_base, s);  // near counter and histogram

    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t tiles = (p.n + kTile - 1) / kTile;
    const unsigned pgrid = unsigned(std::min<uint32_t>(tiles, uint32_t(sms) * 4));
    GatherDesc gb = g;  // K5: v[k] = src[s[k]]
    gb.dst = p.varr;
    gb.idx = p.sarr;
    gb.vec = 1;
    gb.c = 1;
    gb.unit_elems = uint32_t(kThreads) * 32;
    const uint64_t gunits = (g.n + gb.unit_elems - 1) / gb.unit_elems;
    const uint64_t dunits = (g.n + g.unit_elems - 1) / g.unit_elems;
    const uint32_t max_units = tiles + nb;
    if (e == cudaSuccess) { k_l2_sample<<<kSampleRuns / kThreads, kThreads, 0, s>>>(p); e = cudaGetLastError(); }
    if (e == cudaSuccess) { k_l2_hist<<<pgrid, kThreads, 0, s>>>(p); e = cudaGetLastError(); }
    if (e == cudaSuccess) { k_l2_scan<<<1, 1024, 0, s>>>(p); e = cudaGetLastError(); }
    if (e == cudaSuccess) { k_l2_partition<<<pgrid, kThreads, 0, s>>>(p); e = cudaGetLastError(); }
    if (e == cudaSuccess) {
        k_l2_gather<W><<<unsigned(std::min<uint64_t>(gunits, 0x7FFFFFFFull)), kThreads, 0, s>>>(p, gb, gunits, 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_l2_scatter<W><<<unsigned(std::min<uint32_t>(max_units, 0x7FFFFFFFu)), kThreads, 0, s>>>(p, max_units);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_l2_gather<W><<<unsigned(std::min<uint64_t>(dunits, 0x7FFFFFFFull)), kThreads, 0, s>>>(p, g, dunits, 0);
        e = cudaGetLastError();
    }
    g_launches.fetch_add(7, std::memory_order_relaxed);
    cudaError_t e2 = cudaFreeAsync(scratch, s);
    return e != cudaSuccess ? e : e2;
}

}  // namespace

cudaError_t launch_reorder_l2(const OpDesc &op, cudaStream_t s)
{
    switch (op.word) {
        case 4: return run_l2<4>(op.gather, s);
        case 8: return run_l2<8>(op.gather, s);
        case 16: return run_l2<16>(op.gather, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rearr
