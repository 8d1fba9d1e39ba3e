// k_reorder_l2.cu -- reorder by a large random index sequence with L2-resident
// passes (dst[i] = src[idx[i]], arXiv:1011.3583 Sec. III.A indexed access),
// 32- or 64-bit indices, n < 2^32.
//
// A direct gather from a source far larger than the L2 pays a whole DRAM
// access (32-64 B) for every element it reads.  Here the source is cut into
// chunks of about 16 MB (CS elements, C chunks), and the passes make the
// gather read one chunk at a time, L2-resident.  K1 first samples the index
// locality on 4096 short runs of idx: if most neighbours are close
// (|idx[j+1] - idx[j]| <= 16), the direct gather (K7) is already streaming
// and every other pass returns at once; otherwise K7 returns at once.
//
// Tile-local form (gathers whose destination splits into CTA-sized chunks of
// DS = 64 KB of elements, the usual case):
//   partition : each 4096-index tile is counting-sorted by source chunk in
//               shared memory and written back in place -- s-array (source
//               index) and i-array (16-bit offset of the destination in its
//               DS chunk) at the tile's own positions -- with the tile's
//               C + 1 segment starts in a small table.  No pass over the
//               whole sequence comes first.
//   gather    : for each source chunk c in turn, v = src[s] over the
//               c-segment of every tile, written at the same positions, so
//               the CTAs in flight read one ~16 MB chunk at a time from L2.
//   scatter   : one CTA per destination chunk reads the chunk's tiles in
//               order, places each value at its offset in shared memory and
//               writes the chunk out with coalesced stores.
// L2 form (more than reorder_smem_max_buckets() (C, DS-chunk) buckets, or
// forced by the tuning table): destination chunks of CS elements, element i
// in bucket (c, d), d = i / CS; a histogram of the buckets and a scan give
// c-major bucket starts; the partition writes each tile's c-segments at the
// buckets' cursors (s-array, 32-bit i-array); the gather walks the s-array in
// order; the scatter writes dst[i] = v walking the buckets d-major, so the
// CTAs in flight complete one ~16 MB destination chunk in L2.
// A scatter (dst[idx[i]] = src[i]) uses one bucket dimension only (D = 1,
// buckets by the destination chunk of idx[i]): the partition writes
// (destination index, element) pairs, and a linear pass writes
// dst[s[k]] = v[k] with the destination chunk L2-resident.
// Random global accesses cost one L1 request each (about one per clock per
// SM, whatever the working set); random shared-memory accesses run about
// twelve times as fast, so in the tile-local form the gather is the one pass
// bound by random requests.  Its streaming traffic in index-sized words per
// element: idx 1, s 2, i 1 (two 16-bit offsets), src 1, v 2, dst 1 = 8
// passes instead of n random DRAM accesses.
// Scratch ((8 + E) n bytes, plus 12 bytes per bucket and 2 (C + 1) bytes per
// 4096-index tile) comes from a
// stream-ordered pool owned by the library; the kernels are ordered on the
// caller's stream and none waits on another.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "bodies.cuh"
#include "launch.h"
#include "reorder_geometry.h"
#include "tuning.h"

namespace rearr {

namespace {

constexpr int kTile = 4096;        // elements per partition tile / scatter unit
constexpr int kMaxChunks = int(kReorderMaxChunks);  // C <= 512; D <= 512 for the L2 scatter
constexpr int kScatterThreads = 512;
constexpr uint32_t kScatterChunkBytes = kReorderScatterChunkBytes;  // destination chunk of the shared-memory scatter
constexpr int kSampleRuns = 4096;
constexpr int kSampleLen = 64;
constexpr uint32_t kNear = 16;

struct L2Reorder {
    const char *src;
    char *dst;
    const uint32_t *idx;
    uint32_t idx64;                // 1: idx holds uint64 indices (every valid one < n < 2^32)
    uint32_t n;
    uint32_t cs_shift;             // source chunk = 2^cs_shift elements
    uint32_t ds_shift;             // destination chunk = 2^ds_shift elements (>= log2 kTile)
    uint32_t C, D;                 // source / destination chunks
    unsigned long long *near;      // K1: close neighbour pairs in the sample
    unsigned int *ctr_gather;      // K5 / K6 work counters (units handed out in order)
    unsigned int *ctr_scatter;
    uint32_t *hist;                // [C*D] bucket sizes, c-major (b = c*D + d)
    uint32_t *rowtot;              // [C] elements per source chunk
    uint32_t *base;                // [C*D] bucket starts, c-major
    uint32_t *cursor;              // [C*D] partition write cursors
    uint32_t *uprefix;             // [C*D + 1] d-major prefix of scatter units
    uint32_t *sarr, *iarr;         // [n] source / destination indices, c-major; with CTA-sized
                                   // destination chunks the i-array holds uint16 offsets in the chunk
    char *varr;                    // [n] gathered values, c-major
    uint16_t *st;                  // tile-local form: [tiles][C + 1] segment starts per tile
    uint32_t tiles;                // 4096-index tiles of the sequence
    unsigned long long near_threshold;
};

// Source chunk of an index; clamped so that an index >= n (undefined
// behaviour for the caller) cannot address shared memory out of bounds.
__device__ __forceinline__ uint32_t chunk_of(const L2Reorder &p, uint32_t v)
{
    return min(v >> p.cs_shift, p.C - 1);
}

// Second bucket coordinate of element i: its destination chunk for a gather;
// a scatter has one (D = 1).
__device__ __forceinline__ uint32_t dest_chunk(const L2Reorder &p, uint32_t i)
{
    return p.D == 1 ? 0u : i >> p.ds_shift;
}

// Index i of the sequence, narrowed to 32 bits (an index >= n is undefined
// behaviour for the caller either way).
__device__ __forceinline__ uint32_t index_at(const L2Reorder &p, uint64_t i)
{
    return p.idx64 ? uint32_t(__ldg(reinterpret_cast<const unsigned long long *>(p.idx) + i)) : __ldg(p.idx + i);
}

// The same with the index width fixed at compile time (I64: 64-bit indices).
template <bool I64>
__device__ __forceinline__ uint32_t index_at_t(const L2Reorder &p, uint64_t i)
{
    if constexpr (I64) return uint32_t(__ldg(reinterpret_cast<const unsigned long long *>(p.idx) + i));
    else return __ldg(p.idx + i);
}

__device__ __forceinline__ bool bucketed(const L2Reorder &p)
{
    return *reinterpret_cast<volatile unsigned long long *>(p.near) < p.near_threshold;
}

// One warp per sampled run of 64 consecutive indices: each lane loads two
// neighbouring entries and compares them with the next lane's.
__global__ void __launch_bounds__(kThreads) k_l2_sample(const L2Reorder p)
{
    const uint32_t r = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    const uint32_t lane = threadIdx.x & 31;
    uint32_t cnt = 0;
    if (r < kSampleRuns && p.n > kSampleLen) {
        const uint64_t start = uint64_t(r) * (p.n - kSampleLen) / kSampleRuns;
        const uint32_t a = index_at(p, start + 2 * lane), b = index_at(p, start + 2 * lane + 1);
        const uint32_t next_a = __shfl_down_sync(0xffffffffu, a, 1);
        const uint32_t d1 = b > a ? b - a : a - b;
        const uint32_t d2 = next_a > b ? next_a - b : b - next_a;
        cnt = (d1 <= kNear) + (lane < 31 && d2 <= kNear);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(p.near, (unsigned long long)cnt);
}

// Elements of a tile: warp w owns the contiguous slice [w*512, (w+1)*512);
// lane l holds its elements j*32 + l, j < 16 (every load instruction of a warp
// reads 128 contiguous bytes, all 16 are in flight together).
constexpr int kWarps = kThreads / 32;
constexpr int kPer = kTile / kThreads;  // 16

// Tile index k of this thread's element j.
__device__ __forceinline__ uint32_t tile_k(int j)
{
    return (threadIdx.x >> 5) * (kTile / kWarps) + uint32_t(j) * 32 + (threadIdx.x & 31);
}

template <bool I64>
__device__ __forceinline__ void load_tile(const L2Reorder &p, uint32_t i0, uint32_t m, uint32_t (&v)[kPer])
{
    if (m == kTile) {  // a full tile: no bounds test per element
#pragma unroll
        for (int j = 0; j < kPer; ++j) v[j] = index_at_t<I64>(p, i0 + tile_k(j));
    } else {
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const uint32_t k = tile_k(j);
            v[j] = k < m ? index_at_t<I64>(p, i0 + k) : 0xFFFFFFFFu;
        }
    }
}

// Each CTA walks a contiguous range of tiles with per-warp shared counters
// (the only contention is among the lanes of one warp) and flushes them to
// the global histogram whenever the destination chunk changes.
template <bool I64>
__global__ void __launch_bounds__(kThreads) k_l2_hist(const L2Reorder p, uint32_t tiles_per_cta)
{
    if (!bucketed(p)) return;
    __shared__ uint32_t sh[kWarps][kMaxChunks];
    const uint32_t w = threadIdx.x >> 5;
    const uint32_t tiles = (p.n + kTile - 1) / kTile;
    const uint32_t t0 = blockIdx.x * tiles_per_cta, t1 = min(tiles, t0 + tiles_per_cta);
    for (uint32_t c = threadIdx.x; c < kWarps * kMaxChunks; c += kThreads) (&sh[0][0])[c] = 0;
    __syncthreads();
    uint32_t cur_d = t0 < t1 ? dest_chunk(p, t0 * kTile) : 0;
    uint32_t row[kMaxChunks / kThreads] = {};  // this CTA's count of chunks c = threadIdx.x + j * kThreads
    uint32_t v[kPer];
    if (t0 < t1) load_tile<I64>(p, t0 * kTile, min(uint32_t(kTile), p.n - t0 * kTile), v);
    for (uint32_t t = t0; t < t1; ++t) {
        uint32_t nxt[kPer];
        if (t + 1 < t1) load_tile<I64>(p, (t + 1) * kTile, min(uint32_t(kTile), p.n - (t + 1) * kTile), nxt);
        const uint32_t m = min(uint32_t(kTile), p.n - t * kTile);
        if (m == kTile) {
#pragma unroll
            for (int j = 0; j < kPer; ++j) atomicAdd(&sh[w][chunk_of(p, v[j])], 1u);
        } else {
#pragma unroll
            for (int j = 0; j < kPer; ++j)
                if (tile_k(j) < m) atomicAdd(&sh[w][chunk_of(p, v[j])], 1u);
        }
        const uint32_t next_d = t + 1 < t1 ? dest_chunk(p, (t + 1) * kTile) : 0xFFFFFFFFu;
        if (next_d != cur_d) {
            __syncthreads();
#pragma unroll
            for (int j = 0; j < kMaxChunks / kThreads; ++j) {
                const uint32_t c = threadIdx.x + j * kThreads;
                if (c >= p.C) break;
                uint32_t tot = 0;
#pragma unroll
                for (int x = 0; x < kWarps; ++x) {
                    tot += sh[x][c];
                    sh[x][c] = 0;
                }
                row[j] += tot;
                if (tot) atomicAdd(&p.hist[c * p.D + cur_d], tot);
            }
            __syncthreads();
            cur_d = next_d;
        }
        if (t + 1 < t1) {
#pragma unroll
            for (int j = 0; j < kPer; ++j) v[j] = nxt[j];
        }
    }
#pragma unroll
    for (int j = 0; j < kMaxChunks / kThreads; ++j) {
        const uint32_t c = threadIdx.x + j * kThreads;
        if (c < p.C && row[j]) atomicAdd(&p.rowtot[c], row[j]);
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

// Partition: per tile, every warp ranks its 512 elements by source chunk in
// its own counters; thread t then owns chunks 2t and 2t + 1: it sums their
// counts over the warps, and a block scan of those sums gives each chunk's
// segment start in the tile.  The same thread turns its chunks' per-warp
// counts into absolute slots and takes the segment's global position with
// one global atomic per chunk on the bucket's cursor.  The tile is staged in
// shared memory grouped by chunk (the bucketed index and the tile index
// packed in one 64-bit word; the chunk is recomputed from the index) and
// written out as contiguous segments.  The next tile's indices load while this
// one is sorted.
struct PartitionSmem {
    unsigned long long sk[kTile];       // bucketed index (gather: source, scatter: destination) | tile index << 32
    uint32_t cnt[kWarps][kMaxChunks];   // per-warp counts, then per-warp slots
    uint32_t delta[kMaxChunks];         // global position of tile slot 0 of the chunk's segment
    uint32_t warp_sums[kWarps];
};
static_assert(sizeof(PartitionSmem) % 16 == 0, "the scatter form's element buffer follows, 16-byte aligned");

// SW = 0: gather form with ~16 MB destination chunks (s-array: source index,
// i-array: destination index).
// SW = W: scatter form (s-array: destination index, v-array: the element
// itself): the tile's source elements are copied into shared memory with
// cp.async behind the index loads and written out beside their indices, so
// the scatter needs no separate pass that reads the source by position.
template <int SW, bool I64>
__global__ void __launch_bounds__(kThreads, 4) k_l2_partition(const L2Reorder p, uint32_t tiles_per_cta)
{
    if (!bucketed(p)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PartitionSmem &S = *reinterpret_cast<PartitionSmem *>(smem_raw);
    unsigned char *vals = smem_raw + sizeof(PartitionSmem);  // scatter form: kTile * SW bytes
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tiles = (p.n + kTile - 1) / kTile;
    const uint32_t t0 = blockIdx.x * tiles_per_cta, t1 = min(tiles, t0 + tiles_per_cta);
    const uint32_t c0 = 2 * threadIdx.x;  // this thread's chunks: c0, c0 + 1
    for (uint32_t c = threadIdx.x; c < kWarps * kMaxChunks; c += kThreads) (&S.cnt[0][0])[c] = 0;
    uint32_t v[kPer];
    if (t0 < t1) load_tile<I64>(p, t0 * kTile, min(uint32_t(kTile), p.n - t0 * kTile), v);
    __syncthreads();
    for (uint32_t t = t0; t < t1; ++t) {
        const uint32_t i0 = t * kTile;
        const uint32_t m = min(uint32_t(kTile), p.n - i0);
        const uint32_t d = dest_chunk(p, i0);
        if constexpr (SW > 0) {
            // the tile's source elements -> shared memory (waited for before the write-out)
            const char *g = p.src + uint64_t(i0) * SW;
            if ((reinterpret_cast<uintptr_t>(p.src) & 15) == 0) {
                for (uint32_t x = threadIdx.x; x < m * SW / 16; x += kThreads)
                    cp_async<16>(vals + 16 * x, g + 16 * x);
                for (uint32_t k = m * SW / 16 * 16 / SW + threadIdx.x; k < m; k += kThreads)
                    cp_async<SW>(vals + k * SW, g + uint64_t(k) * SW);
            } else {
                for (uint32_t k = threadIdx.x; k < m; k += kThreads) cp_async<SW>(vals + k * SW, g + uint64_t(k) * SW);
            }
            cp_async_commit();
        }
        uint32_t nxt[kPer];
        if (t + 1 < t1) load_tile<I64>(p, (t + 1) * kTile, min(uint32_t(kTile), p.n - (t + 1) * kTile), nxt);
        uint32_t rk[kPer];
        if (m == kTile) {
#pragma unroll
            for (int j = 0; j < kPer; ++j) rk[j] = atomicAdd(&S.cnt[w][chunk_of(p, v[j])], 1u);
        } else {
#pragma unroll
            for (int j = 0; j < kPer; ++j) rk[j] = tile_k(j) < m ? atomicAdd(&S.cnt[w][chunk_of(p, v[j])], 1u) : 0u;
        }
        __syncthreads();
        uint32_t a = 0, b = 0;
        if (c0 < p.C) {
#pragma unroll
            for (int x = 0; x < kWarps; ++x) a += S.cnt[x][c0];
        }
        if (c0 + 1 < p.C) {
#pragma unroll
            for (int x = 0; x < kWarps; ++x) b += S.cnt[x][c0 + 1];
        }
        uint32_t xs = a + b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, xs, o);
            if (lane >= o) xs += y;
        }
        if (lane == 31) S.warp_sums[w] = xs;
        __syncthreads();
        uint32_t before = 0;
#pragma unroll
        for (int x = 0; x < kWarps; ++x) before += x < int(w) ? S.warp_sums[x] : 0u;
        const uint32_t e0 = before + xs - (a + b), e1 = e0 + a;  // segment starts of c0, c0 + 1
        if (c0 < p.C) {
            uint32_t run = e0;
#pragma unroll
            for (int x = 0; x < kWarps; ++x) {
                const uint32_t q = S.cnt[x][c0];
                S.cnt[x][c0] = run;
                run += q;
            }
            const uint32_t g = a ? atomicAdd(&p.cursor[c0 * p.D + d], a) : 0u;
            S.delta[c0] = g - e0;
        }
        if (c0 + 1 < p.C) {
            uint32_t run = e1;
#pragma unroll
            for (int x = 0; x < kWarps; ++x) {
                const uint32_t q = S.cnt[x][c0 + 1];
                S.cnt[x][c0 + 1] = run;
                run += q;
            }
            const uint32_t g = b ? atomicAdd(&p.cursor[(c0 + 1) * p.D + d], b) : 0u;
            S.delta[c0 + 1] = g - e1;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const uint32_t k = tile_k(j);
            if (m == kTile || k < m) {
                const uint32_t pos = S.cnt[w][chunk_of(p, v[j])] + rk[j];
                S.sk[pos] = (unsigned long long)v[j] | ((unsigned long long)k << 32);
            }
        }
        if constexpr (SW > 0) cp_async_wait<0>();
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < m; q += kThreads) {
            const unsigned long long x = S.sk[q];
            const uint32_t sv = uint32_t(x), k = uint32_t(x >> 32);
            const uint32_t g = S.delta[chunk_of(p, sv)] + q;
            p.sarr[g] = sv;
            if constexpr (SW > 0) {
                using T = typename Word<SW>::T;
                reinterpret_cast<T *>(p.varr)[g] = reinterpret_cast<const T *>(vals)[k];
            } else {
                p.iarr[g] = i0 + k;
            }
        }
        // only the C chunks in use need zeroing (not all kMaxChunks)
        for (uint32_t x = threadIdx.x; x < kWarps * p.C; x += kThreads) S.cnt[x / p.C][x % p.C] = 0;
        __syncthreads();
        if (t + 1 < t1) {
#pragma unroll
            for (int j = 0; j < kPer; ++j) v[j] = nxt[j];
        }
    }
}

// Tile-local form (a gather with CTA-sized destination chunks): no pass over
// the whole index sequence has to come before the partition.  Each 4096-index
// tile is counting-sorted by source chunk as above and written back IN PLACE
// (s-array: source index, i-array: 16-bit offset of the destination in its
// chunk, both at the tile's own positions), with the tile's C + 1 segment
// starts in st.  The gather then walks, for each source chunk c in turn, the
// c-segment of every tile, and writes each value at its element's position;
// the scatter reads one destination chunk's tiles in order.
template <bool I64>
__global__ void __launch_bounds__(kThreads, 4) k_l2_partition_local(const L2Reorder p, uint32_t tiles_per_cta)
{
    if (!bucketed(p)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PartitionSmem &S = *reinterpret_cast<PartitionSmem *>(smem_raw);
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t t0 = blockIdx.x * tiles_per_cta, t1 = min(p.tiles, t0 + tiles_per_cta);
    const uint32_t c0 = 2 * threadIdx.x;  // this thread's chunks: c0, c0 + 1
    const uint32_t dmask = (1u << p.ds_shift) - 1;
    for (uint32_t c = threadIdx.x; c < kWarps * kMaxChunks; c += kThreads) (&S.cnt[0][0])[c] = 0;
    uint32_t v[kPer];
    if (t0 < t1) load_tile<I64>(p, t0 * kTile, min(uint32_t(kTile), p.n - t0 * kTile), v);
    __syncthreads();
    for (uint32_t t = t0; t < t1; ++t) {
        const uint32_t i0 = t * kTile;
        const uint32_t m = min(uint32_t(kTile), p.n - i0);
        uint32_t nxt[kPer];
        if (t + 1 < t1) load_tile<I64>(p, (t + 1) * kTile, min(uint32_t(kTile), p.n - (t + 1) * kTile), nxt);
        uint32_t rk[kPer];
        if (m == kTile) {
#pragma unroll
            for (int j = 0; j < kPer; ++j) rk[j] = atomicAdd(&S.cnt[w][chunk_of(p, v[j])], 1u);
        } else {
#pragma unroll
            for (int j = 0; j < kPer; ++j) rk[j] = tile_k(j) < m ? atomicAdd(&S.cnt[w][chunk_of(p, v[j])], 1u) : 0u;
        }
        __syncthreads();
        uint32_t a = 0, b = 0;
        if (c0 < p.C) {
#pragma unroll
            for (int x = 0; x < kWarps; ++x) a += S.cnt[x][c0];
        }
        if (c0 + 1 < p.C) {
#pragma unroll
            for (int x = 0; x < kWarps; ++x) b += S.cnt[x][c0 + 1];
        }
        uint32_t xs = a + b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, xs, o);
            if (lane >= o) xs += y;
        }
        if (lane == 31) S.warp_sums[w] = xs;
        __syncthreads();
        uint32_t before = 0;
#pragma unroll
        for (int x = 0; x < kWarps; ++x) before += x < int(w) ? S.warp_sums[x] : 0u;
        const uint32_t e0 = before + xs - (a + b), e1 = e0 + a;  // segment starts of c0, c0 + 1
        uint16_t *row = p.st + size_t(t) * (p.C + 1);
        if (c0 < p.C) {
            uint32_t run = e0;
#pragma unroll
            for (int x = 0; x < kWarps; ++x) {
                const uint32_t q = S.cnt[x][c0];
                S.cnt[x][c0] = run;
                run += q;
            }
            row[c0] = uint16_t(e0);
        }
        if (c0 + 1 < p.C) {
            uint32_t run = e1;
#pragma unroll
            for (int x = 0; x < kWarps; ++x) {
                const uint32_t q = S.cnt[x][c0 + 1];
                S.cnt[x][c0 + 1] = run;
                run += q;
            }
            row[c0 + 1] = uint16_t(e1);
        }
        if (threadIdx.x == 0) row[p.C] = uint16_t(m);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const uint32_t k = tile_k(j);
            if (m == kTile || k < m) {
                const uint32_t pos = S.cnt[w][chunk_of(p, v[j])] + rk[j];
                S.sk[pos] = (unsigned long long)v[j] | ((unsigned long long)k << 32);
            }
        }
        __syncthreads();
        uint16_t *ioff = reinterpret_cast<uint16_t *>(p.iarr) + i0;
        for (uint32_t q = threadIdx.x; q < m; q += kThreads) {
            const unsigned long long x = S.sk[q];
            p.sarr[i0 + q] = uint32_t(x);
            ioff[q] = uint16_t((i0 + uint32_t(x >> 32)) & dmask);
        }
        for (uint32_t x = threadIdx.x; x < kWarps * p.C; x += kThreads) S.cnt[x / p.C][x % p.C] = 0;
        __syncthreads();
        if (t + 1 < t1) {
#pragma unroll
            for (int j = 0; j < kPer; ++j) v[j] = nxt[j];
        }
    }
}

// The streamed arrays (s, i, v) are marked to leave the L2 first
// (l2_evict_first) so that the resident source / destination chunk
// (l2_evict_last) stays.

// Next work unit for the whole CTA, handed out in increasing order so that the
// units in flight stay a narrow window of the c-major (d-major) order.
__device__ __forceinline__ uint32_t next_unit(unsigned int *ctr, uint32_t *slot)
{
    __syncthreads();
    if (threadIdx.x == 0) *slot = atomicAdd(ctr, 1u);
    __syncthreads();
    return *slot;
}

constexpr int kGatherUnit = 2048;  // elements per gather / scatter unit (8 per thread)

// K5: v[k] = src[s[k]] in k order; the source chunk being read is L2-resident.
template <int W>
__global__ void __launch_bounds__(kThreads, W == 4 ? 8 : W == 8 ? 6 : 4) k_l2_gather(const L2Reorder p)
{
    if (!bucketed(p)) return;
    __shared__ uint32_t slot;
    using T = typename Word<W>::T;
    const uint64_t first = l2_evict_first(), last = l2_evict_last();
    const uint32_t units = (p.n + kGatherUnit - 1) / kGatherUnit;
    for (;;) {
        const uint32_t u = next_unit(p.ctr_gather, &slot);
        if (u >= units) break;
        const uint32_t k0 = u * kGatherUnit;
        constexpr int PER = kGatherUnit / kThreads;
        uint32_t sv[PER];
        T val[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t k = k0 + j * kThreads + threadIdx.x;
            sv[j] = k < p.n ? ldg_hint<4>(p.sarr + k, first) : 0u;
        }
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t k = k0 + j * kThreads + threadIdx.x;
            if (k < p.n) val[j] = ldg_hint<W>(p.src + uint64_t(sv[j]) * W, last);
        }
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t k = k0 + j * kThreads + threadIdx.x;
            if (k < p.n) stg_hint<W>(p.varr + uint64_t(k) * W, val[j], first);
        }
    }
}

// Gather over the tile-local form: unit (c, g) takes source chunk c's
// segment in each of the kWarps * S tiles of group g; a warp walks the
// segments of S tiles together, J elements of each per lane in flight,
// reading s and writing v at the same positions.  S grows with C (segments
// shrink as 4096 / C), so that a unit stays about 2048 elements, and 32 J
// covers a segment's mean length plus three standard deviations, so that
// one round usually finishes it.  Units go out in c-major order, so the CTAs
// in flight read about one ~16 MB source chunk at a time from the L2.
template <int W, int S, int J>
__global__ void __launch_bounds__(kThreads, W == 4 ? 6 : W == 8 ? 5 : 4) k_l2_gather_local(const L2Reorder p)
{
    if (!bucketed(p)) return;
    constexpr uint32_t kUnitTiles = kWarps * S;
    __shared__ uint32_t slot;
    using T = typename Word<W>::T;
    const uint64_t first = l2_evict_first(), last = l2_evict_last();
    const uint32_t groups = (p.tiles + kUnitTiles - 1) / kUnitTiles;
    const uint32_t units = p.C * groups;
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        const uint32_t u = next_unit(p.ctr_gather, &slot);
        if (u >= units) break;
        const uint32_t c = u / groups, g = u - c * groups;
        uint32_t beg[S], end[S], len = 0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const uint32_t t = g * kUnitTiles + w * S + s;
            beg[s] = end[s] = 0;
            if (t < p.tiles) {
                const uint16_t *row = p.st + size_t(t) * (p.C + 1);
                beg[s] = t * kTile + row[c];
                end[s] = t * kTile + row[c + 1];
                len = max(len, end[s] - beg[s]);
            }
        }
        for (uint32_t off = 0; off < len; off += 32 * J) {
            uint32_t sv[S][J];
            T val[S][J];
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const uint32_t k = beg[s] + off + uint32_t(j) * 32 + lane;
                    sv[s][j] = k < end[s] ? ldg_hint<4>(p.sarr + k, first) : 0u;
                }
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const uint32_t k = beg[s] + off + uint32_t(j) * 32 + lane;
                    if (k < end[s]) val[s][j] = ldg_hint<W>(p.src + uint64_t(sv[s][j]) * W, last);
                }
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const uint32_t k = beg[s] + off + uint32_t(j) * 32 + lane;
                    if (k < end[s]) stg_hint<W>(p.varr + uint64_t(k) * W, val[s][j], first);
                }
        }
    }
}

// Scatter over the tile-local form: one CTA per destination chunk d reads the
// chunk's i- and v-arrays in order (its own tiles), places each value at its
// offset of the chunk in shared memory and writes the chunk out with
// coalesced stores, 16 bytes per lane when dst allows.
template <int W>
__global__ void __launch_bounds__(kScatterThreads) k_l2_scatter_local(const L2Reorder p)
{
    if (!bucketed(p)) return;
    using T = typename Word<W>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *chunk = reinterpret_cast<T *>(smem_raw);
    const uint64_t first = l2_evict_first();
    constexpr int U = 4;
    const uint32_t dmask = (1u << p.ds_shift) - 1;
    const bool vec = (reinterpret_cast<uintptr_t>(p.dst) & 15) == 0;
    const uint16_t *off = reinterpret_cast<const uint16_t *>(p.iarr);
    for (uint32_t d = blockIdx.x; d < p.D; d += gridDim.x) {
        const uint64_t i0 = uint64_t(d) << p.ds_shift;
        const uint32_t m = uint32_t(min(uint64_t(dmask) + 1, uint64_t(p.n) - i0));
        uint32_t q = threadIdx.x;
        for (; q + (U - 1) * kScatterThreads < m; q += U * kScatterThreads) {
            uint32_t di[U];
            T val[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                di[u] = ldg_hint<2>(off + i0 + q + u * kScatterThreads, first);
                val[u] = ldg_hint<W>(p.varr + (i0 + q + u * kScatterThreads) * W, first);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) chunk[di[u] & dmask] = val[u];
        }
        for (; q < m; q += kScatterThreads)
            chunk[ldg_hint<2>(off + i0 + q, first) & dmask] = ldg_hint<W>(p.varr + (i0 + q) * W, first);
        __syncthreads();
        char *out = p.dst + i0 * W;
        uint32_t done = 0;
        if (vec) {
            const uint32_t nv = m * W / 16;
            const uint4 *c16 = reinterpret_cast<const uint4 *>(smem_raw);
            for (uint32_t x = threadIdx.x; x < nv; x += kScatterThreads) reinterpret_cast<uint4 *>(out)[x] = c16[x];
            done = nv * 16 / W;
        }
        for (uint32_t x = done + threadIdx.x; x < m; x += kScatterThreads) reinterpret_cast<T *>(out)[x] = chunk[x];
        __syncthreads();
    }
}

// K6: dst[i[k]] = v[k] walking the buckets d-major; the destination chunk
// being written is L2-resident, so its sectors are completed there.
template <int W>
__global__ void __launch_bounds__(kThreads) k_l2_scatter(const L2Reorder p)
{
    if (!bucketed(p)) return;
    __shared__ uint32_t slot, sk0, sk1;
    using T = typename Word<W>::T;
    const uint64_t first = l2_evict_first(), last = l2_evict_last();
    const uint32_t nb = p.C * p.D;
    const uint32_t total = p.uprefix[nb];
    for (;;) {
        const uint32_t u = next_unit(p.ctr_scatter, &slot);
        if (u >= total) break;
        if (threadIdx.x == 0) {
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
            sk0 = p.base[b] + piece * kTile;
            sk1 = p.base[b] + min(p.hist[b], (piece + 1) * uint32_t(kTile));
        }
        __syncthreads();
        const uint32_t k0 = sk0, k1 = sk1;
        constexpr int PER = kTile / kThreads;
        uint32_t di[PER];
        T val[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t k = k0 + j * kThreads + threadIdx.x;
            if (k < k1) {
                di[j] = ldg_hint<4>(p.iarr + k, first);
                val[j] = ldg_hint<W>(p.varr + uint64_t(k) * W, first);
            }
        }
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t k = k0 + j * kThreads + threadIdx.x;
            if (k < k1) stg_hint<W>(p.dst + uint64_t(di[j]) * W, val[j], last);
        }
    }
}

// Scatter form, last pass: dst[s[k]] = v[k] in k order (c-major: one
// destination chunk at a time, L2-resident while its sectors are completed).
template <int W>
__global__ void __launch_bounds__(kThreads) k_l2_scatter_linear(const L2Reorder p)
{
    if (!bucketed(p)) return;
    __shared__ uint32_t slot;
    using T = typename Word<W>::T;
    const uint64_t first = l2_evict_first(), last = l2_evict_last();
    const uint32_t units = (p.n + kGatherUnit - 1) / kGatherUnit;
    for (;;) {
        const uint32_t u = next_unit(p.ctr_scatter, &slot);
        if (u >= units) break;
        const uint32_t k0 = u * kGatherUnit;
        constexpr int PER = kGatherUnit / kThreads;
        uint32_t di[PER];
        T val[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t k = k0 + j * kThreads + threadIdx.x;
            if (k < p.n) {
                di[j] = ldg_hint<4>(p.sarr + k, first);
                val[j] = ldg_hint<W>(p.varr + uint64_t(k) * W, first);
            }
        }
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t k = k0 + j * kThreads + threadIdx.x;
            if (k < p.n) stg_hint<W>(p.dst + uint64_t(di[j]) * W, val[j], last);
        }
    }
}

// K7: the direct gather, when K1 found the indices local.
template <int W>
__global__ void __launch_bounds__(kThreads) k_l2_direct(const L2Reorder p, const GatherDesc g, uint64_t units)
{
    if (bucketed(p)) return;
    for (uint64_t u = blockIdx.x; u < units; u += gridDim.x) gather_body<W>(g, u);
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
    p.idx64 = g.idx64;
    p.n = uint32_t(g.n);
    // ~16 MB source chunks; CTA-sized destination chunks (shared-memory
    // scatter) while the bucket count stays within the tuned bound
    const ReorderGeometry gm = reorder_geometry(g.n, W, g.scatter != 0, reorder_smem_max_buckets());
    p.cs_shift = gm.cs_shift;
    p.C = gm.C;
    const bool smem_scatter = gm.smem_scatter;
    p.ds_shift = gm.ds_shift;
    p.D = gm.D;
    const size_t off_hist = gm.off_hist, off_row = gm.off_row, off_base = gm.off_base, off_cur = gm.off_cur,
                 off_up = gm.off_up, off_s = gm.off_s, off_i = gm.off_i, off_v = gm.off_v, off_st = gm.off_st,
                 bytes = gm.bytes;
    cudaMemPool_t pool;
    cudaError_t e = get_pool(pool);
    if (e != cudaSuccess) return e;
    char *scratch = nullptr;
    e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&scratch), bytes, pool, s);
    if (e != cudaSuccess) return e;
    p.near = reinterpret_cast<unsigned long long *>(scratch);
    p.ctr_gather = reinterpret_cast<unsigned int *>(scratch + 8);
    p.ctr_scatter = reinterpret_cast<unsigned int *>(scratch + 16);
    p.hist = reinterpret_cast<uint32_t *>(scratch + off_hist);
    p.rowtot = reinterpret_cast<uint32_t *>(scratch + off_row);
    p.base = reinterpret_cast<uint32_t *>(scratch + off_base);
    p.cursor = reinterpret_cast<uint32_t *>(scratch + off_cur);
    p.uprefix = reinterpret_cast<uint32_t *>(scratch + off_up);
    p.sarr = reinterpret_cast<uint32_t *>(scratch + off_s);
    p.iarr = reinterpret_cast<uint32_t *>(scratch + off_i);
    p.varr = scratch + off_v;
    p.st = reinterpret_cast<uint16_t *>(scratch + off_st);
    p.tiles = uint32_t((g.n + kTile - 1) / kTile);
    const uint64_t pairs = uint64_t(kSampleRuns) * (kSampleLen - 1);
    p.near_threshold = pairs / 2;
    e = cudaMemsetAsync(scratch, 0, off_base, s);  // near counter, histogram, row totals

    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t tiles = (p.n + kTile - 1) / kTile;
    const uint32_t resident = uint32_t(sms) * 4;
    const uint32_t tpc = (tiles + resident - 1) / resident;  // contiguous tiles per CTA
    const unsigned pgrid = unsigned((tiles + tpc - 1) / tpc);
    // Per device, once: the partition's shared-memory opt-in and occupancy.
    static std::mutex setup_mu;
    static bool smem_set[64] = {false};
    static int part_per_sm[64] = {0}, spart_per_sm[64] = {0}, scat_per_sm[64] = {0};
    int per_sm_part = 1, per_sm_scat = 1;
    if (dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> lock(setup_mu);
        if (!smem_set[dev]) {
            e = cudaFuncSetAttribute(k_l2_partition<0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(sizeof(PartitionSmem)));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_l2_partition<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(sizeof(PartitionSmem)));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_l2_partition<W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(sizeof(PartitionSmem) + kTile * W));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_l2_partition_local<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(sizeof(PartitionSmem)));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_l2_partition_local<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(sizeof(PartitionSmem)));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_l2_scatter_local<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(kScatterChunkBytes));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_l2_partition<W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(sizeof(PartitionSmem) + kTile * W));
            smem_set[dev] = e == cudaSuccess;
            int per_sm = 0;
            if (e == cudaSuccess && cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                        &per_sm, k_l2_partition<0, false>, kThreads, sizeof(PartitionSmem)) == cudaSuccess)
                part_per_sm[dev] = per_sm;
            per_sm = 0;
            if (e == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_l2_partition<W, false>, kThreads,
                                                              sizeof(PartitionSmem) + kTile * W) == cudaSuccess)
                spart_per_sm[dev] = per_sm;
            per_sm = 0;
            if (e == cudaSuccess && cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                        &per_sm, k_l2_scatter_local<W>, kScatterThreads, kScatterChunkBytes) ==
                                        cudaSuccess)
                scat_per_sm[dev] = per_sm;
        }
        per_sm_part = std::max(1, g.scatter ? spart_per_sm[dev] : part_per_sm[dev]);
        per_sm_scat = std::max(1, scat_per_sm[dev]);
    }
    // The partition runs one wave: every resident CTA takes a contiguous
    // range of tiles (a second, partial wave would leave SMs idle).
    const uint32_t part_resident = uint32_t(sms) * uint32_t(per_sm_part);
    const uint32_t part_tpc = (tiles + part_resident - 1) / part_resident;
    const unsigned part_grid = unsigned((tiles + part_tpc - 1) / part_tpc);
    const unsigned pers = unsigned(sms) * 8;  // persistent grids of the gated passes
    const uint64_t dunits = (g.n + g.unit_elems - 1) / g.unit_elems;
    if (e == cudaSuccess) { k_l2_sample<<<kSampleRuns / (kThreads / 32), kThreads, 0, s>>>(p); e = cudaGetLastError(); }
    // A gather with CTA-sized destination chunks runs the tile-local form:
    // partition in place, gather over the tiles' segments, scatter per chunk.
    const bool local = smem_scatter && !g.scatter;
    if (local) {
        if (e == cudaSuccess) {
            if (p.idx64) k_l2_partition_local<true><<<part_grid, kThreads, sizeof(PartitionSmem), s>>>(p, part_tpc);
            else k_l2_partition_local<false><<<part_grid, kThreads, sizeof(PartitionSmem), s>>>(p, part_tpc);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            // segments of 4096 / C elements: tiles per warp so that a unit is ~2048 elements
            // (wider elements take fewer per lane, within the register budget)
            constexpr int J1 = W == 16 ? 8 : 10, J2 = W == 16 ? 4 : 6, J4 = W == 4 ? 3 : 2;
            if (p.C <= 16) k_l2_gather_local<W, 1, J1><<<pers, kThreads, 0, s>>>(p);
            else if (p.C <= 32) k_l2_gather_local<W, 2, J2><<<pers, kThreads, 0, s>>>(p);
            else if (p.C <= 64) k_l2_gather_local<W, 4, J4><<<pers, kThreads, 0, s>>>(p);
            else k_l2_gather_local<W, 4, 2><<<pers, kThreads, 0, s>>>(p);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            const unsigned sgrid = unsigned(std::min<uint64_t>(p.D, uint64_t(sms) * per_sm_scat));
            k_l2_scatter_local<W><<<sgrid, kScatterThreads, kScatterChunkBytes, s>>>(p);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess && !local) {
        if (p.idx64) k_l2_hist<true><<<pgrid, kThreads, 0, s>>>(p, tpc);
        else k_l2_hist<false><<<pgrid, kThreads, 0, s>>>(p, tpc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !local) { k_l2_scan<<<1, 1024, 0, s>>>(p); e = cudaGetLastError(); }
    if (e == cudaSuccess && !local) {
        const size_t sm_part = sizeof(PartitionSmem) + (g.scatter ? size_t(kTile) * W : 0);
        if (g.scatter && p.idx64) k_l2_partition<W, true><<<part_grid, kThreads, sm_part, s>>>(p, part_tpc);
        else if (g.scatter) k_l2_partition<W, false><<<part_grid, kThreads, sm_part, s>>>(p, part_tpc);
        else if (p.idx64) k_l2_partition<0, true><<<part_grid, kThreads, sm_part, s>>>(p, part_tpc);
        else k_l2_partition<0, false><<<part_grid, kThreads, sm_part, s>>>(p, part_tpc);
        e = cudaGetLastError();
    }
    if (local) {
        // done above
    } else if (!g.scatter) {
        if (e == cudaSuccess) { k_l2_gather<W><<<pers, kThreads, 0, s>>>(p); e = cudaGetLastError(); }
        if (e == cudaSuccess) { k_l2_scatter<W><<<pers, kThreads, 0, s>>>(p); e = cudaGetLastError(); }
    } else {
        // the partition wrote (destination index, element) pairs
        if (e == cudaSuccess) { k_l2_scatter_linear<W><<<pers, kThreads, 0, s>>>(p); e = cudaGetLastError(); }
    }
    if (e == cudaSuccess) {
        // two resident waves: when the bucketed passes ran, the grid exits at
        // once; when it gathers, that is as fast as one CTA per unit
        const uint64_t cap = uint64_t(sms) * 16;
        k_l2_direct<W><<<unsigned(std::min<uint64_t>(dunits, cap)), kThreads, 0, s>>>(p, g, dunits);
        e = cudaGetLastError();
    }
    g_launches.fetch_add(local ? 5 : g.scatter ? 6 : 7, std::memory_order_relaxed);
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
