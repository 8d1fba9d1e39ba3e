// k_stencil.cu -- generic 2-D stencil kernels (Sec. III.D) for sm_103a.
//
// A CTA of 256 threads computes a 128 x 64 tile of outputs.  Its input box --
// the tile, r halo rows above and below and 8 staged columns left and right --
// is copied to shared memory (the "user managed cache" of Sec. III.D) by ONE
// TMA tensor copy when the grid's rows are 16-byte aligned: the copy engine
// zero-fills cells outside the grid, so the halo needs no per-thread
// boundary logic and no uncoalesced apron loads (the cost Sec. III.D
// attributes to designated halo threads).  Other grids are staged by plain
// coalesced loads.  With the clamped boundary, edge tiles then overwrite their
// out-of-grid cells with the nearest in-grid cell.
//
// Compute bodies reading that box:
//   cross<r> / box<r>: each thread owns 8 rows x 4 columns of outputs and
//     streams the input rows it needs through registers (16-byte shared
//     loads); every staged value is read once per thread and used by all the
//     taps that touch it.  Weights are compile-time-indexed kernel parameters.
//   generic: each thread owns 32 rows of one column and loops over the tap
//     list: one shared-memory read and one FMA per tap and output.
// The paper's diagonal block order (partition camping) has no counterpart on
// this memory system: tiles run in row-major order, so horizontally adjacent
// CTAs share halo columns in L2.
#include <cuda.h>

#include <mutex>

#include "launch.h"
#include "stencil.h"

namespace rearr {

__device__ unsigned long long g_stencil_wait_timeouts = 0;

namespace {

constexpr int TY = kStencilTileY;
constexpr int PITCH = kStencilPitch;
static_assert(kStencilPitch * 4 % 16 == 0, "staged rows must stay 16-byte aligned");
static_assert((kStencilTileY + 2 * kStencilMaxRadius) * kStencilPitch * 4 <= 48 * 1024,
              "box must fit the default dynamic shared memory limit");

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

// Stages rows y0 - r .. y0 + TY + r - 1 and columns x0 - 8 .. x0 + 71 of the
// source into box (row pitch PITCH floats).  Returns false when the TMA copy
// did not complete in time (the CTA then computes nothing).
__device__ bool stage_box(const StencilArgs &a, const CUtensorMap *tmap, float *box, uint64_t *bar, int64_t y0,
                          int64_t x0)
{
    const int rows = TY + 2 * a.r;
    const int tid = threadIdx.x;
    const int64_t by = y0 - a.r, bx = x0 - kStencilHaloX;  // grid position of box cell (0, 0)
    if (a.tma) {
        const uint32_t b = smem_u32(bar);
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
                         "r"(rows * PITCH * 4)
                         : "memory");
            // x = bx is a multiple of 4 floats (16 bytes): x0 is a multiple of
            // 64 and the halo is 8 columns.  Cells outside the grid read 0.
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(box)),
                "l"(reinterpret_cast<uint64_t>(tmap)), "r"(int(bx)), "r"(int(by)), "r"(b)
                : "memory");
        }
        __syncthreads();  // the barrier is initialised before anyone polls it
        const bool ok = mbar_wait_bounded(b, 0);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicAdd(&g_stencil_wait_timeouts, 1ull);
            mbar_wait_bounded(b, 0);  // let a late copy land before the CTA exits
            return false;
        }
        const bool edge = by < 0 || bx < 0 || by + rows > a.ny || bx + PITCH > a.nx;
        if (a.boundary == REARR_STENCIL_CLAMP && edge) {
            // Out-of-grid cells take the nearest in-grid cell, which lies in
            // the box too (the box overlaps the grid); in-grid cells are only
            // read here, so the rewrite has no read/write conflict.
            for (int i = tid; i < rows * PITCH; i += kStencilThreads) {
                const int rr = i / PITCH, cc = i - rr * PITCH;
                const int64_t gy = by + rr, gx = bx + cc;
                if (gy >= 0 && gy < a.ny && gx >= 0 && gx < a.nx) continue;
                box[i] = box[(clamp64(gy, a.ny) - by) * PITCH + (clamp64(gx, a.nx) - bx)];
            }
            __syncthreads();
        }
        return true;
    }
    for (int i = tid; i < rows * PITCH; i += kStencilThreads) {
        const int rr = i / PITCH, cc = i - rr * PITCH;
        int64_t gy = by + rr, gx = bx + cc;
        float v = 0.f;
        const bool in = gy >= 0 && gy < a.ny && gx >= 0 && gx < a.nx;
        if (in || a.boundary == REARR_STENCIL_CLAMP) {
            gy = clamp64(gy, a.ny);
            gx = clamp64(gx, a.nx);
            v = __ldg(a.src + gy * a.nx + gx);
        }
        box[i] = v;
    }
    __syncthreads();
    return true;
}

// Cross / box bodies: thread (cx, cy) owns tile rows cy*8 .. cy*8+7 and
// columns 4cx .. 4cx+3.
template <int R, int SHAPE>
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
        const bool side = SHAPE == REARR_STENCIL_BOX || (j >= R && j < R + BY);
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
                if (SHAPE == REARR_STENCIL_CROSS && dy != 0 && dx != 0) continue;
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

// Generic body: thread (tx, ty) owns tile column tx, rows ty*32 .. ty*32+31.
__device__ __forceinline__ void compute_generic(const StencilArgs &a, const float *box, int64_t y0, int64_t x0)
{
    constexpr int RPT = TY / 4;
    static_assert(kStencilThreads == 4 * kStencilTileX, "thread grid must cover the tile");
    const int tx = threadIdx.x & (kStencilTileX - 1), ty = threadIdx.x / kStencilTileX;
    float acc[RPT];
#pragma unroll
    for (int v = 0; v < RPT; ++v) acc[v] = 0.f;
    const float *base = box + (ty * RPT + a.r) * PITCH + kStencilHaloX + tx;
    for (int k = 0; k < a.ntaps; ++k) {
        const float wt = a.tw[k];
        const float *p = base + a.tdy[k] * PITCH + a.tdx[k];
#pragma unroll
        for (int v = 0; v < RPT; ++v) acc[v] = fmaf(wt, p[v * PITCH], acc[v]);
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

template <int R, int SHAPE>
__global__ void __launch_bounds__(kStencilThreads, 4)
    k_stencil(const __grid_constant__ StencilArgs a, const __grid_constant__ CUtensorMap tmap)
{
    extern __shared__ __align__(128) float box[];
    __shared__ __align__(8) uint64_t bar;
    const int64_t t = blockIdx.x;
    const int64_t ty = t / a.tiles_x, tx = t - ty * a.tiles_x;
    const int64_t y0 = ty * TY, x0 = tx * kStencilTileX;
    if (!stage_box(a, &tmap, box, &bar, y0, x0)) return;
    if constexpr (SHAPE == REARR_STENCIL_GENERIC) compute_generic(a, box, y0, x0);
    else compute_blocked<R, SHAPE>(a, box, y0, x0);
}

template <int R, int SHAPE>
cudaError_t launch_one(const StencilPlan &pl, const CUtensorMap &m, cudaStream_t s)
{
    k_stencil<R, SHAPE><<<unsigned(pl.n_tiles), kStencilThreads, pl.smem_bytes, s>>>(pl.a, m);
    return cudaGetLastError();
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

}  // namespace

cudaError_t launch_stencil2d(const StencilPlan &pl, cudaStream_t s)
{
    if (pl.n_tiles == 0) return cudaSuccess;
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
    if (pl.shape == REARR_STENCIL_CROSS) {
        switch (r) {
            case 1: e = launch_one<1, REARR_STENCIL_CROSS>(pl, m, s); break;
            case 2: e = launch_one<2, REARR_STENCIL_CROSS>(pl, m, s); break;
            case 3: e = launch_one<3, REARR_STENCIL_CROSS>(pl, m, s); break;
            case 4: e = launch_one<4, REARR_STENCIL_CROSS>(pl, m, s); break;
            case 5: e = launch_one<5, REARR_STENCIL_CROSS>(pl, m, s); break;
            case 6: e = launch_one<6, REARR_STENCIL_CROSS>(pl, m, s); break;
            case 7: e = launch_one<7, REARR_STENCIL_CROSS>(pl, m, s); break;
            case 8: e = launch_one<8, REARR_STENCIL_CROSS>(pl, m, s); break;
            default: break;
        }
    } else if (pl.shape == REARR_STENCIL_BOX) {
        if (r == 1) e = launch_one<1, REARR_STENCIL_BOX>(pl, m, s);
        else if (r == 2) e = launch_one<2, REARR_STENCIL_BOX>(pl, m, s);
    } else {
        e = launch_one<0, REARR_STENCIL_GENERIC>(pl, m, s);
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
