// batch.cu -- batched execution: one persistent kernel runs the tiles of many
// independent ops from a device-side work list, captured once in a CUDA graph.
//
// Work list: the ops' descriptors and the prefix sum of their tile counts.
// Every CTA repeatedly takes the next `grab` tiles with one atomicAdd on a
// device counter, finds the op of the first by binary search over the prefix
// array and runs the matching body (bodies.cuh) for each tile.  No CTA ever
// waits for another: the only shared state is the counter.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/librearr.h"
#include "tuning.h"
#include "bodies.cuh"
#include "launch.h"
#include "plan.h"
#include "variants.h"
#include "worklist.h"

namespace rearr {

rearr_status fail(rearr_status st, const std::string &msg);
rearr_status cuda_fail(cudaError_t e, const char *what);

namespace {

__device__ __forceinline__ char *const *planes_of(const InterlaceDesc &d)
{
    return d.k <= uint32_t(kInlineK) ? d.planes : d.planes_dev;
}

// One non-inlined function per body variant, each running a range [u0, u1)
// of one op's units.  Separate functions get separate register allocations
// (a single function holding every inlined variant overflows the register
// file), and the call overhead is paid once per range, not once per tile.
// Fast tiles are pipelined over the range: tile u+1 is copied (cp.async)
// into the second half of the shared buffer while tile u is stored from the
// first, so a CTA's next load latency hides behind its current stores (tiles
// of the uneven mix are often partly filled and latency-bound).
template <int E, int VI, int VO, int RB, int TBYTES = kTileBytes>
__device__ __noinline__ void tile_range(const TileDesc &d, uint32_t u0, uint32_t u1, unsigned char *smem)
{
    static_assert(2 * TBYTES <= kBatchSmemBytes, "two tile buffers must fit the batched kernel's shared memory");
    if constexpr (VI < 4) {  // 1- and 2-byte loads: cp.async copies 4 bytes or more
        for (uint32_t u = u0; u < u1; ++u) tile_fast_body<E, VI, VO, RB, TBYTES>(d, u, smem);
    } else {
        if (u0 >= u1) return;
        tile_fast_issue<E, VI, VO, RB, TBYTES>(d, u0, smem);
        for (uint32_t u = u0; u < u1; ++u) {
            unsigned char *cur = smem + ((u - u0) & 1u) * TBYTES;
            if (u + 1 < u1) {
                // the other buffer's last reader was tile u-1, finished at the
                // barrier that ended the previous iteration
                tile_fast_issue<E, VI, VO, RB, TBYTES>(d, u + 1, smem + ((u + 1 - u0) & 1u) * TBYTES);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            tile_fast_store<E, VI, VO, RB, TBYTES>(d, u, cur);
            __syncthreads();
        }
    }
}

template <int W>
__device__ __noinline__ void cells_range(const TileDesc &d, uint32_t u0, uint32_t u1, unsigned char *smem)
{
    for (uint32_t u = u0; u < u1; ++u) tile_cells_any<W>(d, u, smem);
}

template <int W>
__device__ __noinline__ void runs_range(const RunsDesc &d, uint64_t u0, uint64_t u1, unsigned char *smem)
{
    for (uint64_t u = u0; u < u1; ++u) runs_body<W>(d, u, smem);
}

template <int W>
__device__ __noinline__ void copy_range(const CopyDesc &d, uint64_t u0, uint64_t u1)
{
    for (uint64_t u = u0; u < u1; ++u) copy_body<W>(d, u);
}

template <int W, int ND>
__device__ __noinline__ void strided_range_nd(const StridedDesc &d, uint64_t u0, uint64_t u1)
{
    for (uint64_t u = u0; u < u1; ++u) strided_body<W, ND>(d, u);
}

template <int W>
__device__ __forceinline__ void strided_range(const StridedDesc &d, uint64_t u0, uint64_t u1)
{
    switch (d.nd) {  // the usual ranks after collapsing, then any
        case 2: strided_range_nd<W, 2>(d, u0, u1); return;
        case 3: strided_range_nd<W, 3>(d, u0, u1); return;
        case 4: strided_range_nd<W, 4>(d, u0, u1); return;
        case 5: strided_range_nd<W, 5>(d, u0, u1); return;
        default: strided_range_nd<W, 0>(d, u0, u1); return;
    }
}

template <int W, int NU>
__device__ __noinline__ void box_range_nu(const BoxDesc &d, uint64_t u0, uint64_t u1, unsigned char *smem)
{
    for (uint64_t u = u0; u < u1; ++u) box_body<W, NU>(d, u, smem);
}

template <int W>
__device__ __forceinline__ void box_range(const BoxDesc &d, uint64_t u0, uint64_t u1, unsigned char *smem)
{
    switch (d.nu) {
        case 1: box_range_nu<W, 1>(d, u0, u1, smem); return;
        case 2: box_range_nu<W, 2>(d, u0, u1, smem); return;
        case 3: box_range_nu<W, 3>(d, u0, u1, smem); return;
        default: box_range_nu<W, 4>(d, u0, u1, smem); return;
    }
}

template <int W>
__device__ __noinline__ void gather_range(const GatherDesc &d, uint64_t u0, uint64_t u1)
{
    for (uint64_t u = u0; u < u1; ++u) gather_body<W>(d, u);
}

template <int W>
__device__ __noinline__ void igen_range(const InterlaceDesc &d, uint64_t u0, uint64_t u1, bool inter)
{
    for (uint64_t u = u0; u < u1; ++u) interlace_generic_body<W>(d, planes_of(d), u, inter);
}

template <int E, int K>
__device__ __noinline__ void ifast_range(const InterlaceDesc &d, uint64_t u0, uint64_t u1, uint64_t n, bool inter,
                                         unsigned char *smem)
{
    for (uint64_t u = u0; u < u1; ++u) {
        if (inter) interlace_fast_body<E, K>(d, planes_of(d), u, n, smem);
        else deinterlace_fast_body<E, K>(d, planes_of(d), u, n, smem);
    }
}

#define BT_CASE(E, VI, VO, RB) \
    case tile_variant(E, VI, VO, RB): tile_range<E, VI, VO, RB>(d.tile, uint32_t(u0), uint32_t(u1), smem); return;

#define BT_HALF(E, VI, VO, RB) \
    case tile_variant(E, VI, VO, RB, 8192): tile_range<E, VI, VO, RB, 8192>(d.tile, uint32_t(u0), uint32_t(u1), smem); return;

__device__ __forceinline__ void run_tile_fast(const OpDesc &d, uint64_t u0, uint64_t u1, unsigned char *smem)
{
    switch (d.tile.variant) {
        REARR_TILE_VARIANTS(BT_CASE)
        REARR_TILE_HALF_VARIANTS(BT_HALF)
        default: return;
    }
}
#undef BT_CASE
#undef BT_HALF

template <int W>
__device__ __forceinline__ void run_word_class(const OpDesc &d, uint64_t u0, uint64_t u1, unsigned char *smem)
{
    switch (d.cls) {
        case OC_TILE_CELLS: cells_range<W>(d.tile, uint32_t(u0), uint32_t(u1), smem); return;
        case OC_RUNS: runs_range<W>(d.runs, u0, u1, smem); return;
        case OC_COPY: copy_range<W>(d.copy, u0, u1); return;
        case OC_STRIDED: strided_range<W>(d.strided, u0, u1); return;
        case OC_BOX: box_range<W>(d.box, u0, u1, smem); return;
        case OC_GATHER: gather_range<W>(d.gather, u0, u1); return;
        case OC_INTERLACE: igen_range<W>(d.inter, u0, u1, true); return;
        case OC_DEINTERLACE: igen_range<W>(d.inter, u0, u1, false); return;
        default: return;
    }
}

template <int E>
__device__ __forceinline__ void run_inter_fast(const OpDesc &d, uint64_t u0, uint64_t u1, unsigned char *smem)
{
    const bool inter = d.cls == OC_INTERLACE;
    switch (d.inter.k) {
        case 1: ifast_range<E, 1>(d.inter, u0, u1, d.units, inter, smem); return;
        case 2: ifast_range<E, 2>(d.inter, u0, u1, d.units, inter, smem); return;
        case 3: ifast_range<E, 3>(d.inter, u0, u1, d.units, inter, smem); return;
        case 4: ifast_range<E, 4>(d.inter, u0, u1, d.units, inter, smem); return;
        default: return;
    }
}

// Units [u0, u1) of one op.
__device__ __forceinline__ void run_range(const OpDesc &d, uint64_t u0, uint64_t u1, unsigned char *smem)
{
    if (d.cls == OC_TILE) { run_tile_fast(d, u0, u1, smem); return; }
    if ((d.cls == OC_INTERLACE || d.cls == OC_DEINTERLACE) && d.inter.fast) {
        switch (d.inter.elem_bytes) {
            case 1: run_inter_fast<1>(d, u0, u1, smem); return;
            case 2: run_inter_fast<2>(d, u0, u1, smem); return;
            case 4: run_inter_fast<4>(d, u0, u1, smem); return;
            case 8: run_inter_fast<8>(d, u0, u1, smem); return;
            case 16: run_inter_fast<16>(d, u0, u1, smem); return;
            default: return;
        }
    }
    switch (d.word) {
        case 1: run_word_class<1>(d, u0, u1, smem); return;
        case 2: run_word_class<2>(d, u0, u1, smem); return;
        case 4: run_word_class<4>(d, u0, u1, smem); return;
        case 8: run_word_class<8>(d, u0, u1, smem); return;
        case 16: run_word_class<16>(d, u0, u1, smem); return;
        default: return;
    }
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 4) k_batch(const OpDesc *__restrict__ ops,
                                                       const uint64_t *__restrict__ prefix, int n_ops,
                                                       unsigned long long *counter, uint32_t grab)
{
    __shared__ __align__(16) unsigned char smem[kBatchSmemBytes];
    __shared__ unsigned long long s_start;
    const uint64_t total = prefix[n_ops];
    for (;;) {
        if (threadIdx.x == 0) s_start = atomicAdd(counter, (unsigned long long)grab);
        __syncthreads();
        const uint64_t start = s_start;
        __syncthreads();
        if (start >= total) break;
        const uint64_t end = min(total, start + grab);
        // op containing `start`: last index with prefix[op] <= start
        int lo = 0, hi = n_ops - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= start) lo = mid;
            else hi = mid - 1;
        }
        // the grabbed range, split at op boundaries
        for (uint64_t t = start; t < end; ++lo) {
            const uint64_t seg_end = min(end, prefix[lo + 1]);
            run_range(ops[lo], t - prefix[lo], seg_end - prefix[lo], smem);
            t = seg_end;
        }
    }
}

}  // namespace rearr

// ---------------------------------------------------------------------------
// Host side of the batched plan.

using namespace rearr;

struct rearr_plan {
    std::vector<OpDesc> ops;
    std::vector<std::vector<char *>> plane_lists;  // per op (empty unless k > kInlineK)
    bool finalized = false;
    void *dev = nullptr;               // one allocation: ops | prefix | plane arrays | counter
    OpDesc *d_ops = nullptr;
    uint64_t *d_prefix = nullptr;
    unsigned long long *d_counter = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t total_units = 0;
    int n_launch_ops = 0;              // ops with at least one unit
    uint32_t grab = 1;
    int grid = 0;
};

static rearr_status add_op(rearr_plan *p, const OpDesc &op_in, std::vector<char *> planes = {})
{
    if (op_in.units == 0) return REARR_OK;
    OpDesc op = op_in;
    batch_form(op);
    p->ops.push_back(op);
    p->plane_lists.push_back(std::move(planes));
    return REARR_OK;
}

extern "C" {

rearr_status rearr_plan_create(rearr_plan **plan)
{
    if (!plan) return fail(REARR_EINVAL, "rearr_plan_create: plan is NULL");
    *plan = new (std::nothrow) rearr_plan();
    if (!*plan) return fail(REARR_ENOMEM, "rearr_plan_create: out of host memory");
    return REARR_OK;
}

rearr_status rearr_plan_add_permute(rearr_plan *plan, void *dst, const void *src, size_t elem_bytes, int rank,
                                    const int64_t *dims, const int *perm)
{
    if (!plan) return fail(REARR_EINVAL, "rearr_plan_add_permute: plan is NULL");
    if (plan->finalized) return fail(REARR_EBUSY, "rearr_plan_add_permute: plan is finalized");
    PermPlan pl;
    std::string err;
    rearr_status st = plan_permute(dst, src, elem_bytes, rank, dims, perm, pl, err);
    if (st != REARR_OK) return fail(st, "rearr_plan_add_permute: " + err);
    return add_op(plan, pl.op);
}

rearr_status rearr_plan_add_scatter(rearr_plan *plan, void *dst, const void *src, const uint32_t *idx, size_t n,
                                    size_t elem_bytes)
{
    if (!plan) return fail(REARR_EINVAL, "rearr_plan_add_scatter: plan is NULL");
    if (plan->finalized) return fail(REARR_EBUSY, "rearr_plan_add_scatter: plan is finalized");
    OpDesc op;
    std::string err;
    rearr_status st = plan_reorder(dst, src, idx, n, elem_bytes, op, err, 4, true);
    if (st != REARR_OK) return fail(st, "rearr_plan_add_scatter: " + err);
    return add_op(plan, op);
}

rearr_status rearr_plan_add_reorder_nm(rearr_plan *plan, void *dst, const void *src, size_t elem_bytes,
                                       int rank_in, const int64_t *dims, int rank_out, const int *order,
                                       const int64_t *base, const int64_t *range)
{
    if (!plan) return fail(REARR_EINVAL, "rearr_plan_add_reorder_nm: plan is NULL");
    if (plan->finalized) return fail(REARR_EBUSY, "rearr_plan_add_reorder_nm: plan is finalized");
    PermPlan pl;
    std::string err;
    rearr_status st = plan_reorder_nm(dst, src, elem_bytes, rank_in, dims, rank_out, order, base, range, pl, err);
    if (st != REARR_OK) return fail(st, "rearr_plan_add_reorder_nm: " + err);
    return add_op(plan, pl.op);
}

rearr_status rearr_plan_add_reorder(rearr_plan *plan, void *dst, const void *src, const uint32_t *idx, size_t n,
                                    size_t elem_bytes)
{
    if (!plan) return fail(REARR_EINVAL, "rearr_plan_add_reorder: plan is NULL");
    if (plan->finalized) return fail(REARR_EBUSY, "rearr_plan_add_reorder: plan is finalized");
    OpDesc op;
    std::string err;
    rearr_status st = plan_reorder(dst, src, idx, n, elem_bytes, op, err);
    if (st != REARR_OK) return fail(st, "rearr_plan_add_reorder: " + err);
    return add_op(plan, op);
}

static rearr_status plan_add_inter(rearr_plan *plan, bool inter, char *iv, char *const *planes, int k, size_t n,
                                   size_t elem_bytes, const char *who)
{
    if (!plan) return fail(REARR_EINVAL, std::string(who) + ": plan is NULL");
    if (plan->finalized) return fail(REARR_EBUSY, std::string(who) + ": plan is finalized");
    InterlacePlan pl;
    std::string err;
    rearr_status st = plan_interlace(inter, iv, planes, k, n, elem_bytes, pl, err);
    if (st != REARR_OK) return fail(st, std::string(who) + ": " + err);
    if (pl.op.units == 0) return REARR_OK;
    std::vector<char *> lst;
    if (k > kInlineK) lst = pl.planes;
    return add_op(plan, pl.op, std::move(lst));
}

rearr_status rearr_plan_add_interlace(rearr_plan *plan, void *dst, const void *const *srcs, int k, size_t n,
                                      size_t elem_bytes)
{
    return plan_add_inter(plan, true, static_cast<char *>(dst),
                          const_cast<char *const *>(reinterpret_cast<const char *const *>(srcs)), k, n, elem_bytes,
                          "rearr_plan_add_interlace");
}

rearr_status rearr_plan_add_deinterlace(rearr_plan *plan, void *const *dsts, const void *src, int k, size_t n,
                                        size_t elem_bytes)
{
    return plan_add_inter(plan, false, static_cast<char *>(const_cast<void *>(src)),
                          reinterpret_cast<char *const *>(dsts), k, n, elem_bytes, "rearr_plan_add_deinterlace");
}

rearr_status rearr_plan_finalize(rearr_plan *plan, rearr_stream_t stream)
{
    if (!plan) return fail(REARR_EINVAL, "rearr_plan_finalize: plan is NULL");
    if (plan->finalized) return fail(REARR_EBUSY, "rearr_plan_finalize: plan is already finalized");
    const size_t n = plan->ops.size();
    plan->finalized = true;
    if (n == 0) return REARR_OK;
    order_for_batch(plan->ops, plan->plane_lists);
    // Host image of the device block.
    size_t n_ptrs = 0;
    for (auto &l : plan->plane_lists) n_ptrs += l.size();
    const size_t off_ops = 0;
    const size_t off_prefix = (n * sizeof(OpDesc) + 255) / 256 * 256;
    const size_t off_planes = off_prefix + ((n + 1) * sizeof(uint64_t) + 255) / 256 * 256;
    const size_t off_counter = off_planes + (n_ptrs * sizeof(char *) + 255) / 256 * 256;
    const size_t total_bytes = off_counter + 256;
    std::vector<unsigned char> host(total_bytes, 0);
    std::vector<uint64_t> prefix(n + 1, 0);
    for (size_t i = 0; i < n; ++i) prefix[i + 1] = prefix[i] + plan->ops[i].units;
    plan->total_units = prefix[n];

    cudaError_t e = cudaMalloc(&plan->dev, total_bytes);
    if (e != cudaSuccess) {
        plan->dev = nullptr;
        return fail(REARR_ENOMEM, std::string("rearr_plan_finalize: cudaMalloc: ") + cudaGetErrorString(e));
    }
    char *base = static_cast<char *>(plan->dev);
    plan->d_ops = reinterpret_cast<OpDesc *>(base + off_ops);
    plan->d_prefix = reinterpret_cast<uint64_t *>(base + off_prefix);
    plan->d_counter = reinterpret_cast<unsigned long long *>(base + off_counter);
    size_t pi = 0;
    for (size_t i = 0; i < n; ++i) {
        OpDesc &op = plan->ops[i];
        auto &l = plan->plane_lists[i];
        if (!l.empty()) {
            char **dst = reinterpret_cast<char **>(host.data() + off_planes) + pi;
            std::memcpy(dst, l.data(), l.size() * sizeof(char *));
            op.inter.planes_dev = reinterpret_cast<char *const *>(base + off_planes + pi * sizeof(char *));
            pi += l.size();
        }
    }
    std::memcpy(host.data() + off_ops, plan->ops.data(), n * sizeof(OpDesc));
    std::memcpy(host.data() + off_prefix, prefix.data(), (n + 1) * sizeof(uint64_t));
    cudaStream_t us = reinterpret_cast<cudaStream_t>(stream);
    e = cudaMemcpyAsync(plan->dev, host.data(), total_bytes, cudaMemcpyHostToDevice, us);
    if (e == cudaSuccess) e = cudaStreamSynchronize(us);
    if (e != cudaSuccess) return cuda_fail(e, "rearr_plan_finalize: upload");

    // Persistent grid: every SM filled to the kernel's occupancy.
    int dev_id = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev_id);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, kThreads, 0);
    if (e != cudaSuccess) return cuda_fail(e, "rearr_plan_finalize: occupancy");
    const BatchTuning &tun = batch_tuning();
    plan->grab = tun.grab_for(plan->total_units, uint64_t(sms) * uint64_t(std::max(per_sm, 1)));
    uint64_t grid = uint64_t(sms) * uint64_t(std::max(per_sm, 1));
    const uint64_t grabs = (plan->total_units + plan->grab - 1) / plan->grab;
    if (grid > grabs) grid = grabs;
    plan->grid = int(std::max<uint64_t>(grid, 1));
    plan->n_launch_ops = int(n);

    // Capture the counter reset and the launch in a graph on a private stream.
    cudaStream_t cap;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "rearr_plan_finalize: stream");
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(plan->d_counter, 0, sizeof(unsigned long long), cap);
        k_batch<<<plan->grid, kThreads, 0, cap>>>(plan->d_ops, plan->d_prefix, int(n), plan->d_counter, plan->grab);
        cudaError_t le = cudaGetLastError();
        e = cudaStreamEndCapture(cap, &plan->graph);
        if (e == cudaSuccess && le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return cuda_fail(e, "rearr_plan_finalize: graph capture");
    return REARR_OK;
}

rearr_status rearr_batch(rearr_plan *plan, rearr_stream_t stream)
{
    if (!plan) return fail(REARR_EINVAL, "rearr_batch: plan is NULL");
    if (!plan->finalized) return fail(REARR_EINVAL, "rearr_batch: plan is not finalized");
    if (!plan->exec) return REARR_OK;  // empty plan
    cudaError_t e = cudaGraphLaunch(plan->exec, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rearr_batch: graph launch");
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return REARR_OK;
}

void rearr_plan_destroy(rearr_plan *plan)
{
    if (!plan) return;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->dev) cudaFree(plan->dev);
    delete plan;
}

rearr_status rearr_plan_stats(const rearr_plan *plan, int64_t *n_ops, int64_t *n_tiles)
{
    if (!plan) return fail(REARR_EINVAL, "rearr_plan_stats: plan is NULL");
    if (n_ops) *n_ops = int64_t(plan->ops.size());
    if (n_tiles) {
        uint64_t t = 0;
        for (auto &op : plan->ops) t += op.units;
        *n_tiles = int64_t(t);
    }
    return REARR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// rearr_batch_noalloc: the batched kernel run from a fixed, statically sized
// work-list buffer instead of a buffer that rearr_plan_finalize allocates.
//
// Some callers cannot call cudaMalloc: a serving process that has reserved
// the GPU's memory for its own pool up front must not have a library grow
// device memory behind its back, and a latency-critical path cannot afford
// the device-wide synchronisation cudaMalloc / cudaFree may imply.  For them
// the work list (op descriptors, tile prefix sums, plane pointer arrays and
// the work counter) lives in g_noalloc_worklist below, a file-scope device
// array of kNoallocBytes that every GPU loading this library holds until the
// process exits.  Every call shares it and leaves its contents behind; calls
// whose kernels overlap on the GPU (different streams, or several host
// threads) race on it, so callers must order them, e.g. on one stream.

namespace {

constexpr size_t kNoallocBytes = 512 * 1024;
constexpr int kNoallocMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_worklist[kNoallocBytes];

struct NoallocDevice {
    bool ready = false;
    unsigned char *addr = nullptr;  // device address of g_noalloc_worklist
    int resident = 0;               // SMs x resident k_batch CTAs per SM
};

std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[kNoallocMaxDevices];
unsigned char g_noalloc_image[kNoallocBytes];  // host image, built under the mutex

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" rearr_status rearr_batch_noalloc(const rearr_plan *plan, rearr_stream_t stream)
{
    if (!plan) return fail(REARR_EINVAL, "rearr_batch_noalloc: plan is NULL");
    const size_t n = plan->ops.size();
    if (n == 0) return REARR_OK;
    size_t n_ptrs = 0;
    for (auto &l : plan->plane_lists) n_ptrs += l.size();
    const size_t off_prefix = round256(n * sizeof(OpDesc));
    const size_t off_planes = off_prefix + round256((n + 1) * sizeof(uint64_t));
    const size_t off_counter = off_planes + round256(n_ptrs * sizeof(char *));
    const size_t need = off_counter + 256;
    if (need > kNoallocBytes) {
        return fail(REARR_EINVAL, "rearr_batch_noalloc: the plan's work list needs " + std::to_string(need) +
                                      " bytes, more than the fixed " + std::to_string(kNoallocBytes) +
                                      "-byte buffer (about 1280 ops); use rearr_plan_finalize + rearr_batch");
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "rearr_batch_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(REARR_EINVAL, "rearr_batch_noalloc: device id out of range");

    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocDevice &nd = g_noalloc_dev[dev];
    if (!nd.ready) {
        // One-time set-up on this device, with the device current.
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_worklist);
        if (e != cudaSuccess) return cuda_fail(e, "rearr_batch_noalloc: cudaGetSymbolAddress");
        int sms = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, kThreads, 0);
        if (e != cudaSuccess) return cuda_fail(e, "rearr_batch_noalloc: device query");
        nd.addr = static_cast<unsigned char *>(p);
        nd.resident = std::max(1, sms * std::max(per_sm, 1));
        nd.ready = true;
    }

    // Host image: descriptors (plane arrays re-pointed into the buffer),
    // prefix sums of the tile counts, plane pointers, and a zero work counter.
    unsigned char *img = g_noalloc_image;
    std::memset(img, 0, need);
    OpDesc *ops = reinterpret_cast<OpDesc *>(img);
    uint64_t *prefix = reinterpret_cast<uint64_t *>(img + off_prefix);
    char **planes = reinterpret_cast<char **>(img + off_planes);
    size_t pi = 0;
    for (size_t i = 0; i < n; ++i) {
        ops[i] = plan->ops[i];
        prefix[i + 1] = prefix[i] + plan->ops[i].units;
        const auto &l = plan->plane_lists[i];
        if (!l.empty()) {
            std::memcpy(planes + pi, l.data(), l.size() * sizeof(char *));
            ops[i].inter.planes_dev = reinterpret_cast<char *const *>(nd.addr + off_planes + pi * sizeof(char *));
            pi += l.size();
        }
    }
    const uint64_t total = prefix[n];
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // From pageable host memory: the call returns once the image is staged,
    // so the static host image may be rebuilt by the next call.
    e = cudaMemcpyAsync(nd.addr, img, need, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "rearr_batch_noalloc: work-list upload");
    const uint32_t grab = batch_tuning().grab_for(total, uint64_t(nd.resident));
    uint64_t grid = uint64_t(nd.resident);
    const uint64_t grabs = (total + grab - 1) / grab;
    if (grid > grabs) grid = grabs;
    k_batch<<<unsigned(std::max<uint64_t>(grid, 1)), kThreads, 0, s>>>(
        reinterpret_cast<const OpDesc *>(nd.addr), reinterpret_cast<const uint64_t *>(nd.addr + off_prefix), int(n),
        reinterpret_cast<unsigned long long *>(nd.addr + off_counter), grab);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rearr_batch_noalloc: launch");
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return REARR_OK;
}

// ---------------------------------------------------------------------------
// Work lists built and launched from host code (serving loop).

namespace rearr {

// Ops of a batch are independent, so their order in the work list is free.
// The batched kernel holds every body, and a mix that interleaves dozens of
// variants stalls on instruction fetch; a mix grouped by class runs its
// memory-bound and issue-bound classes one after the other instead of
// overlapping them.  So each class's ops are sorted by body variant and the
// classes are merged in proportion to their work units: the CTAs in flight
// run a few bodies, one current variant per class.
void order_for_batch(std::vector<OpDesc> &all_ops, std::vector<std::vector<char *>> &plane_lists)
{
    const size_t n = all_ops.size();
    auto sub = [&](const OpDesc &o) -> uint64_t {
        if (o.cls == OC_TILE) return o.tile.variant;
        if (o.cls == OC_INTERLACE || o.cls == OC_DEINTERLACE)
            return uint64_t(o.inter.fast) << 40 | uint64_t(o.inter.k) << 8 | o.inter.elem_bytes;
        return o.word;
    };
    std::vector<std::vector<size_t>> groups(OC_COUNT);
    std::vector<uint64_t> group_units(OC_COUNT, 0);
    for (size_t i = 0; i < n; ++i) {
        groups[all_ops[i].cls].push_back(i);
        group_units[all_ops[i].cls] += std::max<uint64_t>(all_ops[i].units, 1);
    }
    for (auto &g : groups)
        std::stable_sort(g.begin(), g.end(), [&](size_t a, size_t b) { return sub(all_ops[a]) < sub(all_ops[b]); });
    std::vector<size_t> order;
    order.reserve(n);
    std::vector<size_t> next(OC_COUNT, 0);
    std::vector<uint64_t> done(OC_COUNT, 0);
    while (order.size() < n) {
        // the class furthest behind in its share of units goes next
        int best = -1;
        for (int c = 0; c < int(OC_COUNT); ++c) {
            if (next[c] >= groups[c].size()) continue;
            if (best < 0 ||
                double(done[c]) / double(group_units[c]) < double(done[best]) / double(group_units[best]))
                best = c;
        }
        const size_t i = groups[best][next[best]++];
        done[best] += std::max<uint64_t>(all_ops[i].units, 1);
        order.push_back(i);
    }
    std::vector<OpDesc> ops(n);
    std::vector<std::vector<char *>> lists(n);
    for (size_t i = 0; i < n; ++i) {
        ops[i] = all_ops[order[i]];
        lists[i] = std::move(plane_lists[order[i]]);
    }
    all_ops.swap(ops);
    plane_lists.swap(lists);
}

void batch_form(OpDesc &op)
{
    tile_to_single_width(op);
    if ((op.cls == OC_INTERLACE || op.cls == OC_DEINTERLACE) && op.inter.fast && op.inter.k > 4) {
        // The batched kernel instantiates the 16-byte group bodies for k <= 4
        // only: larger k runs the generic body (the fast path implies a
        // power-of-two element of at most 16 bytes on 16-byte aligned planes).
        InterlaceDesc &d = op.inter;
        const int W = pow2_align(16, d.elem_bytes);
        d.fast = 0;
        op.word = uint32_t(W);
        d.c = d.elem_bytes / uint32_t(W);
        const uint64_t kc = uint64_t(d.k) * d.c;
        d.unit_groups = std::max<uint64_t>(1, 8192 / kc);
        d.kc_div = make_fastdiv(uint32_t(kc));
        d.c_div = make_fastdiv(d.c);
        op.units = (d.n + d.unit_groups - 1) / d.unit_groups;
    }
    if (op.cls == OC_GATHER && op.units > 0) {
        // one iteration of gather_body per unit: 4 elements x 2 groups per
        // thread (vector path) or 4 elements per thread
        op.gather.unit_elems = op.gather.vec ? uint32_t(kThreads) * 8 : uint32_t(kThreads) * 4;
        op.units = (op.gather.n + op.gather.unit_elems - 1) / op.gather.unit_elems;
    }
}

WorklistLayout worklist_layout(size_t n_ops, size_t n_ptrs)
{
    WorklistLayout l;
    l.off_prefix = round256(n_ops * sizeof(OpDesc));
    l.off_planes = l.off_prefix + round256((n_ops + 1) * sizeof(uint64_t));
    l.off_counter = l.off_planes + round256(n_ptrs * sizeof(char *));
    l.bytes = l.off_counter + 256;
    return l;
}

uint64_t build_worklist(const OpDesc *ops, const std::vector<char *> *plane_lists, size_t n, unsigned char *img,
                        uintptr_t dev_base, const WorklistLayout &layout)
{
    OpDesc *dops = reinterpret_cast<OpDesc *>(img);
    uint64_t *prefix = reinterpret_cast<uint64_t *>(img + layout.off_prefix);
    char **planes = reinterpret_cast<char **>(img + layout.off_planes);
    prefix[0] = 0;
    size_t pi = 0;
    for (size_t i = 0; i < n; ++i) {
        dops[i] = ops[i];
        prefix[i + 1] = prefix[i] + ops[i].units;
        const std::vector<char *> &l = plane_lists[i];
        if (!l.empty()) {
            std::memcpy(planes + pi, l.data(), l.size() * sizeof(char *));
            dops[i].inter.planes_dev = reinterpret_cast<char *const *>(dev_base + layout.off_planes + pi * sizeof(char *));
            pi += l.size();
        }
    }
    std::memset(img + layout.off_counter, 0, 256);
    return prefix[n];
}

static int resident_ctas_current_device()
{
    static std::mutex mu;
    static int cached[kNoallocMaxDevices] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return 0;
    std::lock_guard<std::mutex> lock(mu);
    if (!cached[dev]) {
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, kThreads, 0) != cudaSuccess) return 0;
        cached[dev] = std::max(1, sms * std::max(per_sm, 1));
    }
    return cached[dev];
}

cudaError_t launch_worklist(uintptr_t dev_base, const WorklistLayout &layout, size_t n, uint64_t total_units,
                            cudaStream_t s)
{
    if (n == 0 || total_units == 0) return cudaSuccess;
    const int resident = resident_ctas_current_device();
    if (resident == 0) return cudaErrorInvalidDevice;
    const uint32_t grab = batch_tuning().grab_for(total_units, uint64_t(resident));
    uint64_t grid = uint64_t(resident);
    const uint64_t grabs = (total_units + grab - 1) / grab;
    if (grid > grabs) grid = grabs;
    const char *base = reinterpret_cast<const char *>(dev_base);
    k_batch<<<unsigned(std::max<uint64_t>(grid, 1)), kThreads, 0, s>>>(
        reinterpret_cast<const OpDesc *>(base), reinterpret_cast<const uint64_t *>(base + layout.off_prefix), int(n),
        reinterpret_cast<unsigned long long *>(const_cast<char *>(base) + layout.off_counter), grab);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

}  // namespace rearr
