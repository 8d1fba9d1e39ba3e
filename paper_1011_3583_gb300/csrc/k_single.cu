// k_single.cu -- one-launch-per-call kernels of librearr and their launcher.
//
// Each kernel runs one op: CTA i handles work units i, i + gridDim.x, ...
// with the body of the op's class (bodies.cuh).
#include <atomic>

#include "bodies.cuh"
#include "launch.h"
#include "variants.h"

namespace rearr {

std::atomic<uint64_t> g_launches{0};

// Programmatic dependent launch.  Every single-op kernel is launched with
// programmatic stream serialisation: when the kernel before it on the stream
// is also one of these, it may be launched while that one drains, its CTAs
// taking SM slots as they free up.  Each kernel therefore first waits for
// the grid it depends on to complete and its writes to be visible
// (griddepcontrol.wait; a no-op when nothing is pending), and then allows
// the next kernel to launch (griddepcontrol.launch_dependents; that launch
// happens once every CTA of this grid has started or exited).  No memory is
// touched before the wait, so ordering on the stream is as without it.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <int E, int VIN, int VOUT, int ROWB, int TBYTES = kTileBytes>
__global__ void __launch_bounds__(kThreads) k_tile_fast(const __grid_constant__ TileDesc d, uint32_t n)
{
    pdl_enter();
    __shared__ __align__(16) unsigned char smem[TBYTES];
    for (uint32_t t = blockIdx.x; t < n; t += gridDim.x) tile_fast_body<E, VIN, VOUT, ROWB, TBYTES>(d, t, smem);
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_tile_cells(const __grid_constant__ TileDesc d, uint32_t n)
{
    pdl_enter();
    __shared__ __align__(16) unsigned char smem[kSmemBytes];
    for (uint32_t t = blockIdx.x; t < n; t += gridDim.x) tile_cells_body<W>(d, t, smem);
}

// Blocked runs (a cells tile with pitch 0) in a kernel of their own: no shared
// memory and their own register allocation (the staged cells body needs
// about twice the registers, which would halve the CTAs per SM).
template <int W>
__global__ void __launch_bounds__(kThreads) k_tile_runs(const __grid_constant__ TileDesc d, uint32_t n)
{
    pdl_enter();
    for (uint32_t t = blockIdx.x; t < n; t += gridDim.x) tile_runs_body<W>(d, t);
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_runs(const __grid_constant__ RunsDesc d, uint64_t n)
{
    pdl_enter();
    __shared__ __align__(16) unsigned char smem[kMaxRunsPerUnit * 8];
    for (uint64_t u = blockIdx.x; u < n; u += gridDim.x) runs_body<W>(d, u, smem);
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_copy(const __grid_constant__ CopyDesc d, uint64_t n)
{
    pdl_enter();
    for (uint64_t u = blockIdx.x; u < n; u += gridDim.x) copy_body<W>(d, u);
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_gather(const __grid_constant__ GatherDesc d, uint64_t n)
{
    pdl_enter();
    for (uint64_t u = blockIdx.x; u < n; u += gridDim.x) gather_body<W>(d, u);
}

template <int W, int ND>
__global__ void __launch_bounds__(kThreads) k_strided(const __grid_constant__ StridedDesc d, uint64_t n)
{
    pdl_enter();
    for (uint64_t u = blockIdx.x; u < n; u += gridDim.x) strided_body<W, ND>(d, u);
}

template <int W, int NU>
__global__ void __launch_bounds__(kThreads, 3) k_box(const __grid_constant__ BoxDesc d, uint32_t n)
{
    pdl_enter();
    __shared__ __align__(16) unsigned char smem[kBoxBytes];
    for (uint32_t u = blockIdx.x; u < n; u += gridDim.x) box_body<W, NU>(d, u, smem);
}

// Interlace kernels take every plane pointer by value.
struct InterlaceParams {
    InterlaceDesc d;
    char *planes[kMaxK];
};

template <int E, int K, bool INTER>
__global__ void __launch_bounds__(kThreads) k_inter_fast(const __grid_constant__ InterlaceParams p, uint64_t n)
{
    pdl_enter();
    __shared__ __align__(16) unsigned char smem[kThreads / 32 * K * 32 * 16];
    for (uint64_t u = blockIdx.x; u < n; u += gridDim.x) {
        if constexpr (INTER) interlace_fast_body<E, K>(p.d, p.planes, u, n, smem);
        else deinterlace_fast_body<E, K>(p.d, p.planes, u, n, smem);
    }
}

template <int W, bool INTER>
__global__ void __launch_bounds__(kThreads) k_inter_generic(const __grid_constant__ InterlaceParams p, uint64_t n)
{
    pdl_enter();
    for (uint64_t u = blockIdx.x; u < n; u += gridDim.x) interlace_generic_body<W>(p.d, p.planes, u, INTER);
}

namespace {

inline unsigned grid_for(uint64_t units)
{
    return unsigned(units < 0x7FFFFFFFull ? units : 0x7FFFFFFFull);
}

template <typename P, typename N>
cudaError_t go(void (*kernel)(P, N), uint64_t units, const P &param, N n, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid_for(units));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, param, n);
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

#define RT_CASE(E, VI, VO, RB)                                                                \
    case tile_variant(E, VI, VO, RB):                                                             \
        return go(k_tile_fast<E, VI, VO, RB>, op.units, op.tile, uint32_t(op.units), s);

#define RT_HALF(E, VI, VO, RB)                                                                \
    case tile_variant(E, VI, VO, RB, 8192):                                                       \
        return go(k_tile_fast<E, VI, VO, RB, 8192>, op.units, op.tile, uint32_t(op.units), s);

#define RT_DOUBLE(E, VI, VO, RB)                                                              \
    case tile_variant(E, VI, VO, RB, 32768):                                                      \
        return go(k_tile_fast<E, VI, VO, RB, 32768>, op.units, op.tile, uint32_t(op.units), s);

cudaError_t launch_tile_fast(const OpDesc &op, cudaStream_t s)
{
    switch (op.tile.variant) {
        REARR_TILE_VARIANTS(RT_CASE)
        REARR_TILE_HALF_VARIANTS(RT_HALF)
        REARR_TILE_DOUBLE_VARIANTS(RT_DOUBLE)
        default: return cudaErrorInvalidValue;
    }
}
#undef RT_CASE
#undef RT_HALF
#undef RT_DOUBLE

template <template <int> class Fn, typename... A>
cudaError_t by_word(int W, A &&...a)
{
    switch (W) {
        case 1: return Fn<1>::run(a...);
        case 2: return Fn<2>::run(a...);
        case 4: return Fn<4>::run(a...);
        case 8: return Fn<8>::run(a...);
        case 16: return Fn<16>::run(a...);
        default: return cudaErrorInvalidValue;
    }
}

template <int W> struct RunCells {
    static cudaError_t run(const OpDesc &op, cudaStream_t s)
    {
        if (op.tile.pitch == 0) return go(k_tile_runs<W>, op.units, op.tile, uint32_t(op.units), s);
        return go(k_tile_cells<W>, op.units, op.tile, uint32_t(op.units), s);
    }
};
template <int W> struct RunRuns {
    static cudaError_t run(const OpDesc &op, cudaStream_t s) { return go(k_runs<W>, op.units, op.runs, op.units, s); }
};
template <int W> struct RunCopy {
    static cudaError_t run(const OpDesc &op, cudaStream_t s) { return go(k_copy<W>, op.units, op.copy, op.units, s); }
};
template <int W> struct RunStrided {
    static cudaError_t run(const OpDesc &op, cudaStream_t s)
    {
        switch (op.strided.nd) {  // the usual ranks after collapsing, then any
            case 2: return go(k_strided<W, 2>, op.units, op.strided, op.units, s);
            case 3: return go(k_strided<W, 3>, op.units, op.strided, op.units, s);
            case 4: return go(k_strided<W, 4>, op.units, op.strided, op.units, s);
            case 5: return go(k_strided<W, 5>, op.units, op.strided, op.units, s);
            default: return go(k_strided<W, 0>, op.units, op.strided, op.units, s);
        }
    }
};
template <int W> struct RunBox {
    static cudaError_t run(const OpDesc &op, cudaStream_t s)
    {
        switch (op.box.nu) {
            case 1: return go(k_box<W, 1>, op.units, op.box, uint32_t(op.units), s);
            case 2: return go(k_box<W, 2>, op.units, op.box, uint32_t(op.units), s);
            case 3: return go(k_box<W, 3>, op.units, op.box, uint32_t(op.units), s);
            case 4: return go(k_box<W, 4>, op.units, op.box, uint32_t(op.units), s);
            default: return cudaErrorInvalidValue;
        }
    }
};
template <int W> struct RunGather {
    static cudaError_t run(const OpDesc &op, cudaStream_t s)
    {
        return go(k_gather<W>, op.units, op.gather, op.units, s);
    }
};

template <int E, bool INTER>
cudaError_t launch_inter_fast_k(const InterlaceParams &p, uint64_t units, cudaStream_t s)
{
    switch (p.d.k) {
        case 1: return go(k_inter_fast<E, 1, INTER>, units, p, units, s);
        case 2: return go(k_inter_fast<E, 2, INTER>, units, p, units, s);
        case 3: return go(k_inter_fast<E, 3, INTER>, units, p, units, s);
        case 4: return go(k_inter_fast<E, 4, INTER>, units, p, units, s);
        case 5: return go(k_inter_fast<E, 5, INTER>, units, p, units, s);
        case 6: return go(k_inter_fast<E, 6, INTER>, units, p, units, s);
        case 7: return go(k_inter_fast<E, 7, INTER>, units, p, units, s);
        case 8: return go(k_inter_fast<E, 8, INTER>, units, p, units, s);
        default: return cudaErrorInvalidValue;
    }
}

template <bool INTER>
cudaError_t launch_inter(const InterlaceParams &p, const OpDesc &op, cudaStream_t s)
{
    if (p.d.fast) {
        switch (p.d.elem_bytes) {
            case 1: return launch_inter_fast_k<1, INTER>(p, op.units, s);
            case 2: return launch_inter_fast_k<2, INTER>(p, op.units, s);
            case 4: return launch_inter_fast_k<4, INTER>(p, op.units, s);
            case 8: return launch_inter_fast_k<8, INTER>(p, op.units, s);
            case 16: return launch_inter_fast_k<16, INTER>(p, op.units, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (op.word) {
        case 1: return go(k_inter_generic<1, INTER>, op.units, p, op.units, s);
        case 2: return go(k_inter_generic<2, INTER>, op.units, p, op.units, s);
        case 4: return go(k_inter_generic<4, INTER>, op.units, p, op.units, s);
        case 8: return go(k_inter_generic<8, INTER>, op.units, p, op.units, s);
        case 16: return go(k_inter_generic<16, INTER>, op.units, p, op.units, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_single(const OpDesc &op, char *const *planes_all, cudaStream_t s)
{
    if (op.units == 0) return cudaSuccess;
    switch (op.cls) {
        case OC_TILE: return launch_tile_fast(op, s);
        case OC_TILE_CELLS: return by_word<RunCells>(int(op.word), op, s);
        case OC_RUNS: return by_word<RunRuns>(int(op.word), op, s);
        case OC_COPY: return by_word<RunCopy>(int(op.word), op, s);
        case OC_STRIDED: return by_word<RunStrided>(int(op.word), op, s);
        case OC_BOX: return by_word<RunBox>(int(op.word), op, s);
        case OC_GATHER:
            if (op.gather.l2) return launch_reorder_l2(op, s);
            return by_word<RunGather>(int(op.word), op, s);
        case OC_INTERLACE:
        case OC_DEINTERLACE: {
            InterlaceParams p;
            p.d = op.inter;
            for (uint32_t j = 0; j < kMaxK; ++j) p.planes[j] = j < op.inter.k ? planes_all[j] : nullptr;
            return op.cls == OC_INTERLACE ? launch_inter<true>(p, op, s) : launch_inter<false>(p, op, s);
        }
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rearr
