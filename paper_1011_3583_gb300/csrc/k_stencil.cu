// k_stencil.cu -- generic 2-D stencil kernels (Sec. III.D) for sm_103a.
//
// Every CTA of 256 threads computes 128 x 64 tiles of outputs from an input
// box in shared memory (Sec. III.D uses shared memory as a cache the program
// manages): the tile, r halo rows above and below and 8 staged columns left
// and right.
//
// Staging.  When the grid's rows are 16-byte aligned the box arrives by ONE
// TMA tensor copy (cp.async.bulk.tensor.2d) whose out-of-grid cells the copy
// engine fills with zeros, so the halo needs neither designated halo threads
// nor uncoalesced apron loads (the costs Sec. III.D names).  Other grids are
// staged by plain coalesced loads.  With the clamped boundary, edge tiles then
// overwrite their out-of-grid cells with the nearest in-grid cell.  One tile
// per CTA and four CTAs per SM: while some CTAs compute, the others' copies
// are in flight.  (A persistent variant with two boxes per CTA, copying tile
// i + 1 while computing tile i, fits only two CTAs per SM and measured
// slower: 5.4 against 7.0 TB/s on a 16384^2 grid.)
//
// Compute bodies reading a box:
//   cross<r> / box<r>: each thread owns 8 rows x 4 columns of outputs and
//     streams the input rows it needs through registers (16-byte shared
//     loads); every staged value is read once per thread and feeds all the
//     taps that touch it.  Weights are compile-time-indexed kernel parameters.
//   generic, long tap lists (more than 24 taps): each thread owns 32 rows of
//     one column, computed as two halves of 16.  Per distinct dx of the tap
//     list it loads that input column (16 + 2r values) into registers and
//     applies the column's taps from there (a switch on dy selects the
//     compile-time register offset).
//   generic, short tap lists: each thread owns 32 rows of one column and
//     reads one staged value per tap and output (fewer instructions per tap;
//     measured faster up to about two dozen taps).
// The paper's diagonal block order (partition camping) has no counterpart on
// this memory system: tiles run in row-major order, so neighbouring CTAs
// share halo cells in L2.
#include <cuda.h>

#include <atomic>
#include <mutex>

#include "launch.h"
#include "stencil.h"

namespace rearr {

__device__ unsigned long long g_stencil_wait_timeouts = 0;

namespace {

constexpr int TY = kStencilTileY;
constexpr int PITCH = kStencilPitch;
constexpr int MAXR = kStencilMaxRadius;
constexpr int WARPS = kStencilThreads / 32;
static_assert(kStencilPitch * 4 % 16 == 0, "staged rows must stay 16-byte aligned");
static_assert(PITCH <= 3 * 32, "a warp stages a row in three passes");

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for phase `parity` of the mbarrier at shared address bar; gives up
// after 2^22 polls or 2 s, whichever comes first.
__device__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0; it < (1u << 22); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63) == 63 && globaltimer_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}

__device__ __forceinline__ int64_t clamp64(int64_t v, int64_t n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

// One thread: copy the box whose cell (0, 0) is grid point (by, bx) into box,
// completing on the mbarrier at bar.  bx is a multiple of 4 floats (tile
// columns start at multiples of 64, the halo is 8 columns), the TMA rule for
// the innermost coordinate.
__device__ __forceinline__ void tma_issue(const CUtensorMap *tmap, float *box, uint32_t bar, int64_t by, int64_t bx,
                                          uint32_t bytes)
{
    // Order this CTA's earlier generic-proxy accesses of the buffer (reads of
    // the previous tile, clamp rewrites) before the copy's async-proxy writes.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(box)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(int(bx)), "r"(int(by)), "r"(bar)
        : "memory");
}

// Clamped boundary: every out-of-grid cell of the box takes the nearest
// in-grid cell, which the box also holds (it overlaps the grid).  In-grid
// cells are only read, so the rewrite has no read/write conflict.  A warp
// per box row.
__device__ void clamp_fixup(const StencilArgs &a, float *box, int64_t by, int64_t bx, int rows)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = int(bx < 0 ? -bx : 0), c1 = int(a.nx - bx < PITCH ? a.nx - bx : PITCH);
    const int r0 = int(by < 0 ? -by : 0), r1 = int(a.ny - by < rows ? a.ny - by : rows);
    for (int rr = warp; rr < rows; rr += WARPS) {
        const int sr = rr < r0 ? r0 : (rr >= r1 ? r1 - 1 : rr);
        for (int cc = lane; cc < PITCH; cc += 32) {
            const int sc = cc < c0 ? c0 : (cc >= c1 ? c1 - 1 : cc);
            if (sr != rr || sc != cc) box[rr * PITCH + cc] = box[sr * PITCH + sc];
        }
    }
}

// Plain staging of the box (any alignment), boundary applied: a warp per
// box row, 32 consecutive columns per instruction, as 4-byte cp.async copies
// (all of a thread's copies in flight at once; a copy of 0 source bytes
// zero-fills its cell).  The caller waits with cp.async.wait_all.
__device__ void plain_stage(const StencilArgs &a, float *box, int64_t by, int64_t bx, int rows)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool clamp = a.boundary == REARR_STENCIL_CLAMP;
    for (int rr = warp; rr < rows; rr += WARPS) {
        const int64_t gy = by + rr;
        const bool row_in = gy >= 0 && gy < a.ny;
        const float *src_row = a.src + clamp64(gy, a.ny) * a.nx;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int cc = lane + 32 * q;
            if (cc >= PITCH) break;
            const int64_t gx = bx + cc;
            const uint32_t n = (clamp || (row_in && gx >= 0 && gx < a.nx)) ? 4 : 0;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(box + rr * PITCH + cc)),
                         "l"(src_row + clamp64(gx, a.nx)), "r"(n)
                         : "memory");
        }
    }
}

// Cross / box bodies: thread (cx, cy) owns tile rows cy*8 .. cy*8+7 and
// columns 4cx .. 4cx+3.
template <int R, int BODY>
__device__ __forceinline__ void compute_blocked(const StencilArgs &a, const float *box, int64_t y0, int64_t x0)
{
    constexpr int BY = 8;
    constexpr int R4 = (R + 3) & ~3;  // side columns loaded as whole float4s
    constexpr int NW = 2 * R + 1;
    static_assert(16 * BY == TY && 16 * 4 == kStencilTileX, "thread grid must cover the tile");
    static_assert(R4 <= kStencilHaloX, "side loads must stay inside the staged columns");
    const int cx = threadIdx.x & 15, cy = threadIdx.x >> 4;

    float acc[BY][4];
#pragma unroll
    for (int v = 0; v < BY; ++v)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[v][c] = 0.f;

    // Box row cy*BY + j holds tile row cy*BY + j - R.
    const float *base = box + cy * BY * PITCH + kStencilHaloX + 4 * cx;
#pragma unroll
    for (int j = 0; j < BY + 2 * R; ++j) {
        const float *row = base + j * PITCH;
        // Only taps with dy == 0 reach sideways in a cross: input row j feeds
        // them for output row v = j - R.
        const bool side = BODY == kBodyBox || (j >= R && j < R + BY);
        float seg[4 + 2 * R4];
        {
            const float4 m = *reinterpret_cast<const float4 *>(row);
            seg[R4] = m.x, seg[R4 + 1] = m.y, seg[R4 + 2] = m.z, seg[R4 + 3] = m.w;
        }
        if (side) {
#pragma unroll
            for (int q = 0; q < R4 / 4; ++q) {
                const float4 l = *reinterpret_cast<const float4 *>(row - R4 + 4 * q);
                const float4 h = *reinterpret_cast<const float4 *>(row + 4 + 4 * q);
                seg[4 * q] = l.x, seg[4 * q + 1] = l.y, seg[4 * q + 2] = l.z, seg[4 * q + 3] = l.w;
                seg[R4 + 4 + 4 * q] = h.x, seg[R4 + 5 + 4 * q] = h.y, seg[R4 + 6 + 4 * q] = h.z,
                                 seg[R4 + 7 + 4 * q] = h.w;
            }
        }
#pragma unroll
        for (int v = 0; v < BY; ++v) {
            const int dy = j - R - v;
            if (dy < -R || dy > R) continue;
#pragma unroll
            for (int dx = -R; dx <= R; ++dx) {
                if (BODY == kBodyCross && dy != 0 && dx != 0) continue;
                const float wt = a.w[(dy + R) * NW + dx + R];
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[v][c] = fmaf(wt, seg[R4 + c + dx], acc[v][c]);
            }
        }
    }

    const int64_t gx = x0 + 4 * cx;
#pragma unroll
    for (int v = 0; v < BY; ++v) {
        const int64_t gy = y0 + cy * BY + v;
        if (gy >= a.ny) break;
        float *out = a.dst + gy * a.nx + gx;
        if (a.tma) {
            // nx is a multiple of 4: a float4 is wholly inside or outside.
            if (gx < a.nx) *reinterpret_cast<float4 *>(out) = make_float4(acc[v][0], acc[v][1], acc[v][2], acc[v][3]);
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (gx + c < a.nx) out[c] = acc[v][c];
        }
    }
}

constexpr int RPT = TY / (kStencilThreads / kStencilTileX);  // generic body: rows per thread
constexpr int HALF = RPT / 2;                                 // rows per pass
constexpr int NCOL = HALF + 2 * MAXR;                         // registers of one input column

// acc[v] += w * col[v + DY + MAXR]: one tap of the generic body.
template <int DY>
__device__ __forceinline__ void tap_column(float (&acc)[HALF], const float (&col)[NCOL], float w)
{
#pragma unroll
    for (int v = 0; v < HALF; ++v) acc[v] = fmaf(w, col[v + DY + MAXR], acc[v]);
}

// Generic body: thread (tx, ty) owns tile column tx, rows ty*RPT .. +RPT-1,
// in two passes of HALF rows.
__device__ __forceinline__ void compute_generic(const StencilArgs &a, const float *box, int64_t y0, int64_t x0)
{
    static_assert(kStencilThreads % kStencilTileX == 0 && RPT * (kStencilThreads / kStencilTileX) == TY,
                  "thread grid must cover the tile");
    const int tx = threadIdx.x % kStencilTileX, ty = threadIdx.x / kStencilTileX;
    const int64_t gx = x0 + tx;
    const int ilo = MAXR - a.r, ihi = HALF + MAXR + a.r;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        float acc[HALF];
#pragma unroll
        for (int v = 0; v < HALF; ++v) acc[v] = 0.f;
        // col[i] holds tile row ty*RPT + h*HALF + i - MAXR, i.e. box row
        // row0 + i; only i in [MAXR - r, HALF + MAXR + r) is read (|dy| <= r).
        const int row0 = ty * RPT + h * HALF + a.r - MAXR;
        int k = 0;
        for (int g = 0; g < a.ngroups; ++g) {
            const int c = kStencilHaloX + tx + a.gdx[g];
            float col[NCOL];
#pragma unroll
            for (int i = 0; i < NCOL; ++i)
                if (i >= ilo && i < ihi) col[i] = box[(row0 + i) * PITCH + c];
            for (const int kend = a.gend[g]; k < kend; ++k) {
                const float w = a.tw[k];
                switch (a.tdy[k]) {
                    case -8: tap_column<-8>(acc, col, w); break;
                    case -7: tap_column<-7>(acc, col, w); break;
                    case -6: tap_column<-6>(acc, col, w); break;
                    case -5: tap_column<-5>(acc, col, w); break;
                    case -4: tap_column<-4>(acc, col, w); break;
                    case -3: tap_column<-3>(acc, col, w); break;
                    case -2: tap_column<-2>(acc, col, w); break;
                    case -1: tap_column<-1>(acc, col, w); break;
                    case 0: tap_column<0>(acc, col, w); break;
                    case 1: tap_column<1>(acc, col, w); break;
                    case 2: tap_column<2>(acc, col, w); break;
                    case 3: tap_column<3>(acc, col, w); break;
                    case 4: tap_column<4>(acc, col, w); break;
                    case 5: tap_column<5>(acc, col, w); break;
                    case 6: tap_column<6>(acc, col, w); break;
                    case 7: tap_column<7>(acc, col, w); break;
                    default: tap_column<8>(acc, col, w); break;  // |dy| <= 8 is checked on the host
                }
            }
        }
        if (gx < a.nx) {
#pragma unroll
            for (int v = 0; v < HALF; ++v) {
                const int64_t gy = y0 + ty * RPT + h * HALF + v;
                if (gy >= a.ny) break;
                a.dst[gy * a.nx + gx] = acc[v];
            }
        }
    }
}

// Generic body for short tap lists: thread (tx, ty) owns tile column tx,
// rows ty*RPT .. +RPT-1, and reads one staged value per tap and output.
__device__ __forceinline__ void compute_generic_taps(const StencilArgs &a, const float *box, int64_t y0, int64_t x0)
{
    const int tx = threadIdx.x % kStencilTileX, ty = threadIdx.x / kStencilTileX;
    float acc[RPT];
#pragma unroll
    for (int v = 0; v < RPT; ++v) acc[v] = 0.f;
    const float *base = box + (ty * RPT + a.r) * PITCH + kStencilHaloX + tx;
    for (int k = 0; k < a.ntaps; ++k) {
        const float w = a.tw[k];
        const float *p = base + a.tdy[k] * PITCH + a.tdx[k];
#pragma unroll
        for (int v = 0; v < RPT; ++v) acc[v] = fmaf(w, p[v * PITCH], acc[v]);
    }
    const int64_t gx = x0 + tx;
    if (gx >= a.nx) return;
#pragma unroll
    for (int v = 0; v < RPT; ++v) {
        const int64_t gy = y0 + ty * RPT + v;
        if (gy >= a.ny) break;
        a.dst[gy * a.nx + gx] = acc[v];
    }
}

template <int R, int BODY>
__device__ __forceinline__ void compute(const StencilArgs &a, const float *box, int64_t y0, int64_t x0)
{
    if constexpr (BODY == kBodyGenericColumns) compute_generic(a, box, y0, x0);
    else if constexpr (BODY == kBodyGenericTaps) compute_generic_taps(a, box, y0, x0);
    else compute_blocked<R, BODY>(a, box, y0, x0);
}

// Tile of CTA blockIdx.x: row-major, rotated by one row of tiles so that the
// bottom edge (whose clamped boundary costs a rewrite) runs first instead of
// forming the kernel's tail.
__device__ __forceinline__ void tile_origin(const StencilArgs &a, int64_t &y0, int64_t &x0)
{
    const int64_t n = gridDim.x;
    int64_t t = int64_t(blockIdx.x) + (n - a.tiles_x);
    if (t >= n) t -= n;
    const int64_t ty = t / a.tiles_x;
    y0 = ty * TY;
    x0 = (t - ty * a.tiles_x) * kStencilTileX;
}

__device__ __forceinline__ bool edge_box(const StencilArgs &a, int64_t by, int64_t bx, int rows)
{
    return by < 0 || bx < 0 || by + rows > a.ny || bx + PITCH > a.nx;
}

// One tile per CTA, staged by a TMA tensor copy.
template <int R, int BODY>
__global__ void __launch_bounds__(kStencilThreads, 4)
    k_stencil_tma(const __grid_constant__ StencilArgs a, const __grid_constant__ CUtensorMap tmap)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar_storage;
    const int rows = TY + 2 * a.r;
    int64_t y0, x0;
    tile_origin(a, y0, x0);
    const int64_t by = y0 - a.r, bx = x0 - kStencilHaloX;
    const uint32_t bar = smem_u32(&bar_storage);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tma_issue(&tmap, smem, bar, by, bx, uint32_t(rows) * PITCH * 4 + a.extra_tx);
    }
    __syncthreads();  // the barrier is initialised before anyone polls it
    const bool ok = mbar_wait_bounded(bar, 0);
    if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) atomicAdd(&g_stencil_wait_timeouts, 1ull);
        mbar_wait_bounded(bar, 0);  // let a late copy land before the CTA exits
        return;
    }
    if (a.boundary == REARR_STENCIL_CLAMP && edge_box(a, by, bx, rows)) {
        clamp_fixup(a, smem, by, bx, rows);
        __syncthreads();
    }
    compute<R, BODY>(a, smem, y0, x0);
}

// One tile per CTA, plain staging (rows not 16-byte aligned).
template <int R, int BODY>
__global__ void __launch_bounds__(kStencilThreads, 4) k_stencil_plain(const __grid_constant__ StencilArgs a)
{
    extern __shared__ __align__(128) float smem[];
    const int rows = TY + 2 * a.r;
    int64_t y0, x0;
    tile_origin(a, y0, x0);
    plain_stage(a, smem, y0 - a.r, x0 - kStencilHaloX, rows);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    compute<R, BODY>(a, smem, y0, x0);
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
EncodeTiled encode_tiled()
{
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

template <int R, int BODY>
cudaError_t launch_one(const StencilPlan &pl, const CUtensorMap &m, cudaStream_t s)
{
    if (pl.a.tma) k_stencil_tma<R, BODY><<<unsigned(pl.n_tiles), kStencilThreads, pl.smem_bytes, s>>>(pl.a, m);
    else k_stencil_plain<R, BODY><<<unsigned(pl.n_tiles), kStencilThreads, pl.smem_bytes, s>>>(pl.a);
    return cudaGetLastError();
}

std::atomic<int> g_inject_timeouts{0};

}  // namespace

void inject_wait_timeout(int n) { g_inject_timeouts.store(n); }

cudaError_t launch_stencil2d(const StencilPlan &plan, cudaStream_t s)
{
    if (plan.n_tiles == 0) return cudaSuccess;
    StencilPlan pl = plan;
    if (pl.a.tma) {
        int n = g_inject_timeouts.load();
        while (n > 0 && !g_inject_timeouts.compare_exchange_weak(n, n - 1)) {
        }
        if (n > 0) pl.a.extra_tx = 16;
    }
    CUtensorMap m;
    memset(&m, 0, sizeof(m));
    if (pl.a.tma) {
        EncodeTiled enc = encode_tiled();
        if (!enc) return cudaErrorNotSupported;
        const cuuint64_t dims[2] = {cuuint64_t(pl.a.nx), cuuint64_t(pl.a.ny)};
        const cuuint64_t strides[1] = {cuuint64_t(pl.a.nx) * sizeof(float)};
        const cuuint32_t boxdim[2] = {cuuint32_t(PITCH), cuuint32_t(TY + 2 * pl.a.r)};
        const cuuint32_t estr[2] = {1, 1};
        if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(pl.a.src), dims, strides, boxdim, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaErrorInvalidValue;
    const int r = pl.a.r;
    if (pl.body == kBodyCross) {
        switch (r) {
            case 1: e = launch_one<1, kBodyCross>(pl, m, s); break;
            case 2: e = launch_one<2, kBodyCross>(pl, m, s); break;
            case 3: e = launch_one<3, kBodyCross>(pl, m, s); break;
            case 4: e = launch_one<4, kBodyCross>(pl, m, s); break;
            case 5: e = launch_one<5, kBodyCross>(pl, m, s); break;
            case 6: e = launch_one<6, kBodyCross>(pl, m, s); break;
            case 7: e = launch_one<7, kBodyCross>(pl, m, s); break;
            case 8: e = launch_one<8, kBodyCross>(pl, m, s); break;
            default: break;
        }
    } else if (pl.body == kBodyBox) {
        if (r == 1) e = launch_one<1, kBodyBox>(pl, m, s);
        else if (r == 2) e = launch_one<2, kBodyBox>(pl, m, s);
    } else if (pl.body == kBodyGenericTaps) {
        e = launch_one<0, kBodyGenericTaps>(pl, m, s);
    } else {
        e = launch_one<0, kBodyGenericColumns>(pl, m, s);
    }
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

cudaError_t read_wait_timeouts(uint64_t *count)
{
    unsigned long long v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_stencil_wait_timeouts, sizeof(v));
    *count = v;
    return e;
}

}  // namespace rearr
