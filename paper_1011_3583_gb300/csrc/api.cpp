// api.cpp -- the C ABI of librearr for single operations (include/librearr.h).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/librearr.h"
#include "launch.h"
#include "plan.h"
#include "reorder_geometry.h"
#include "tuning.h"
#include "stencil.h"

namespace rearr {

thread_local std::string t_last_error;

rearr_status fail(rearr_status st, const std::string &msg)
{
    t_last_error = msg;
    return st;
}

rearr_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(REARR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace rearr

using namespace rearr;

extern "C" {

const char *rearr_status_str(rearr_status status)
{
    switch (status) {
        case REARR_OK: return "REARR_OK";
        case REARR_EINVAL: return "REARR_EINVAL";
        case REARR_ENOMEM: return "REARR_ENOMEM";
        case REARR_ECUDA: return "REARR_ECUDA";
        case REARR_ERANGE: return "REARR_ERANGE";
        case REARR_ETIMEDOUT: return "REARR_ETIMEDOUT";
        case REARR_EBUSY: return "REARR_EBUSY";
        default: return "REARR_UNKNOWN";
    }
}

const char *rearr_last_error(void) { return t_last_error.c_str(); }

rearr_status rearr_permute(void *dst, const void *src, size_t elem_bytes, int rank, const int64_t *dims,
                           const int *perm, rearr_stream_t stream)
{
    PermPlan pl;
    std::string err;
    rearr_status st = plan_permute(dst, src, elem_bytes, rank, dims, perm, pl, err);
    if (st != REARR_OK) return fail(st, "rearr_permute: " + err);
    cudaError_t e = launch_single(pl.op, nullptr, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rearr_permute launch");
    return REARR_OK;
}

rearr_status rearr_reorder_nm(void *dst, const void *src, size_t elem_bytes, int rank_in, const int64_t *dims,
                              int rank_out, const int *order, const int64_t *base, const int64_t *range,
                              rearr_stream_t stream)
{
    PermPlan pl;
    std::string err;
    rearr_status st = plan_reorder_nm(dst, src, elem_bytes, rank_in, dims, rank_out, order, base, range, pl, err);
    if (st != REARR_OK) return fail(st, "rearr_reorder_nm: " + err);
    cudaError_t e = launch_single(pl.op, nullptr, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rearr_reorder_nm launch");
    return REARR_OK;
}

rearr_status rearr_reorder(void *dst, const void *src, const uint32_t *idx, size_t n, size_t elem_bytes,
                           rearr_stream_t stream)
{
    OpDesc op;
    std::string err;
    rearr_status st = plan_reorder(dst, src, idx, n, elem_bytes, op, err);
    if (st != REARR_OK) return fail(st, "rearr_reorder: " + err);
    cudaError_t e = launch_single(op, nullptr, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rearr_reorder launch");
    return REARR_OK;
}

static rearr_status indexed_call(const char *who, void *dst, const void *src, const void *idx, size_t n,
                                 size_t elem_bytes, int idx_bytes, bool scatter, rearr_stream_t stream)
{
    OpDesc op;
    std::string err;
    rearr_status st = plan_reorder(dst, src, static_cast<const uint32_t *>(idx), n, elem_bytes, op, err, idx_bytes,
                                   scatter);
    if (st != REARR_OK) return fail(st, std::string(who) + ": " + err);
    cudaError_t e = launch_single(op, nullptr, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, who);
    return REARR_OK;
}

rearr_status rearr_scatter(void *dst, const void *src, const uint32_t *idx, size_t n, size_t elem_bytes,
                           rearr_stream_t stream)
{
    return indexed_call("rearr_scatter", dst, src, idx, n, elem_bytes, 4, true, stream);
}

rearr_status rearr_reorder64(void *dst, const void *src, const uint64_t *idx, size_t n, size_t elem_bytes,
                             rearr_stream_t stream)
{
    return indexed_call("rearr_reorder64", dst, src, idx, n, elem_bytes, 8, false, stream);
}

rearr_status rearr_scatter64(void *dst, const void *src, const uint64_t *idx, size_t n, size_t elem_bytes,
                             rearr_stream_t stream)
{
    return indexed_call("rearr_scatter64", dst, src, idx, n, elem_bytes, 8, true, stream);
}

rearr_status rearr_check_indices(const void *idx, size_t n, int idx_bytes, uint64_t bound, uint64_t *n_bad,
                                 rearr_stream_t stream)
{
    if (!n_bad) return fail(REARR_EINVAL, "rearr_check_indices: n_bad is NULL");
    *n_bad = 0;
    if (idx_bytes != 4 && idx_bytes != 8) return fail(REARR_EINVAL, "rearr_check_indices: idx_bytes must be 4 or 8");
    if (n == 0) return REARR_OK;
    if (!idx) return fail(REARR_EINVAL, "rearr_check_indices: idx is NULL");
    if (reinterpret_cast<uintptr_t>(idx) % uintptr_t(idx_bytes) != 0)
        return fail(REARR_EINVAL, "rearr_check_indices: idx not aligned to its index size");
    cudaError_t e = count_bad_indices(idx, n, idx_bytes, bound, n_bad, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rearr_check_indices");
    return REARR_OK;
}

rearr_status rearr_reorder_checked(void *dst, const void *src, const uint32_t *idx, size_t n, size_t elem_bytes,
                                   rearr_stream_t stream)
{
    OpDesc op;
    std::string err;
    rearr_status st = plan_reorder(dst, src, idx, n, elem_bytes, op, err);
    if (st != REARR_OK) return fail(st, "rearr_reorder_checked: " + err);
    if (op.units == 0) return REARR_OK;
    uint64_t bad = 0;
    cudaError_t e = count_bad_indices(idx, n, 4, n, &bad, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rearr_reorder_checked: index check");
    if (bad) return fail(REARR_ERANGE, "rearr_reorder_checked: " + std::to_string(bad) + " of " + std::to_string(n) +
                                           " indices are >= n");
    e = launch_single(op, nullptr, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rearr_reorder_checked launch");
    return REARR_OK;
}

rearr_status rearr_interlace(void *dst, const void *const *srcs, int k, size_t n, size_t elem_bytes,
                             rearr_stream_t stream)
{
    InterlacePlan pl;
    std::string err;
    rearr_status st = plan_interlace(true, static_cast<char *>(dst), const_cast<char *const *>(
                                         reinterpret_cast<const char *const *>(srcs)), k, n, elem_bytes, pl, err);
    if (st != REARR_OK) return fail(st, "rearr_interlace: " + err);
    cudaError_t e = launch_single(pl.op, pl.planes.data(), reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rearr_interlace launch");
    return REARR_OK;
}

rearr_status rearr_deinterlace(void *const *dsts, const void *src, int k, size_t n, size_t elem_bytes,
                               rearr_stream_t stream)
{
    InterlacePlan pl;
    std::string err;
    rearr_status st = plan_interlace(false, static_cast<char *>(const_cast<void *>(src)),
                                     reinterpret_cast<char *const *>(dsts), k, n, elem_bytes, pl, err);
    if (st != REARR_OK) return fail(st, "rearr_deinterlace: " + err);
    cudaError_t e = launch_single(pl.op, pl.planes.data(), reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rearr_deinterlace launch");
    return REARR_OK;
}

rearr_status rearr_stencil2d_f32(float *dst, const float *src, int64_t ny, int64_t nx, int ntaps, const int *dy,
                                 const int *dx, const float *w, int boundary, rearr_stream_t stream)
{
    StencilPlan pl;
    std::string err;
    rearr_status st = plan_stencil2d(dst, src, ny, nx, ntaps, dy, dx, w, boundary, pl, err);
    if (st != REARR_OK) return fail(st, "rearr_stencil2d_f32: " + err);
    cudaError_t e = launch_stencil2d(pl, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rearr_stencil2d_f32 launch");
    return REARR_OK;
}

rearr_status rearr_stencil2d_describe(int64_t ny, int64_t nx, int ntaps, const int *dy, const int *dx, const float *w,
                                      int boundary, uintptr_t dst_addr, uintptr_t src_addr, rearr_stencil_info *info)
{
    if (!info) return fail(REARR_EINVAL, "rearr_stencil2d_describe: info is NULL");
    if (dst_addr == 0) dst_addr = uintptr_t(1) << 47;
    if (src_addr == 0) src_addr = uintptr_t(1) << 46;
    StencilPlan pl;
    std::string err;
    rearr_status st = plan_stencil2d(reinterpret_cast<float *>(dst_addr), reinterpret_cast<const float *>(src_addr),
                                     ny, nx, ntaps, dy, dx, w, boundary, pl, err);
    if (st != REARR_OK) return fail(st, "rearr_stencil2d_describe: " + err);
    info->shape = pl.shape;
    info->body = pl.body;
    info->radius = pl.a.r;
    info->n_unique = pl.n_unique;
    info->tma = pl.a.tma;
    info->tile_y = kStencilTileY;
    info->tile_x = kStencilTileX;
    info->n_tiles = pl.n_tiles;
    info->smem_bytes = int64_t(pl.smem_bytes);
    return REARR_OK;
}

rearr_status rearr_wait_timeouts(uint64_t *count)
{
    if (!count) return fail(REARR_EINVAL, "rearr_wait_timeouts: count is NULL");
    cudaError_t e = read_wait_timeouts(count);
    if (e != cudaSuccess) return cuda_fail(e, "rearr_wait_timeouts");
    return REARR_OK;
}

rearr_status rearr_inject_wait_timeout(int n_launches)
{
    if (n_launches < 0) return fail(REARR_EINVAL, "rearr_inject_wait_timeout: negative count");
    inject_wait_timeout(n_launches);
    return REARR_OK;
}

rearr_status rearr_permute_describe(size_t elem_bytes, int rank, const int64_t *dims, const int *perm,
                                    uintptr_t dst_addr, uintptr_t src_addr, rearr_permute_info *info)
{
    if (!info) return fail(REARR_EINVAL, "rearr_permute_describe: info is NULL");
    // Addresses only steer the alignment decisions; 0 stands for a 256-byte
    // aligned buffer (two far-apart fake addresses, so no overlap is seen).
    if (dst_addr == 0) dst_addr = uintptr_t(1) << 47;
    if (src_addr == 0) src_addr = uintptr_t(1) << 46;
    PermPlan pl;
    std::string err;
    rearr_status st = plan_permute(reinterpret_cast<void *>(dst_addr), reinterpret_cast<const void *>(src_addr),
                                   elem_bytes, rank, dims, perm, pl, err);
    if (st != REARR_OK) return fail(st, "rearr_permute_describe: " + err);
    *info = pl.info;
    return REARR_OK;
}

rearr_status rearr_reorder_nm_describe(size_t elem_bytes, int rank_in, const int64_t *dims, int rank_out,
                                      const int *order, const int64_t *base, const int64_t *range,
                                      uintptr_t dst_addr, uintptr_t src_addr, rearr_permute_info *info)
{
    if (!info) return fail(REARR_EINVAL, "rearr_reorder_nm_describe: info is NULL");
    if (dst_addr == 0) dst_addr = uintptr_t(1) << 47;
    if (src_addr == 0) src_addr = uintptr_t(1) << 46;
    PermPlan pl;
    std::string err;
    rearr_status st = plan_reorder_nm(reinterpret_cast<void *>(dst_addr), reinterpret_cast<const void *>(src_addr),
                                      elem_bytes, rank_in, dims, rank_out, order, base, range, pl, err);
    if (st != REARR_OK) return fail(st, "rearr_reorder_nm_describe: " + err);
    *info = pl.info;
    return REARR_OK;
}

rearr_status rearr_reorder_describe(size_t n, size_t elem_bytes, int idx_bytes, int scatter, uintptr_t dst_addr,
                                    uintptr_t src_addr, uintptr_t idx_addr, rearr_reorder_info *info)
{
    if (!info) return fail(REARR_EINVAL, "rearr_reorder_describe: info is NULL");
    if (idx_bytes != 4 && idx_bytes != 8) return fail(REARR_EINVAL, "rearr_reorder_describe: idx_bytes must be 4 or 8");
    if (dst_addr == 0) dst_addr = uintptr_t(1) << 47;
    if (src_addr == 0) src_addr = uintptr_t(1) << 46;
    if (idx_addr == 0) idx_addr = uintptr_t(1) << 45;
    OpDesc op;
    std::memset(&op, 0, sizeof(op));
    std::string err;
    rearr_status st = plan_reorder(reinterpret_cast<void *>(dst_addr), reinterpret_cast<const void *>(src_addr),
                                   reinterpret_cast<const uint32_t *>(idx_addr), n, elem_bytes, op, err, idx_bytes,
                                   scatter != 0);
    if (st != REARR_OK) return fail(st, "rearr_reorder_describe: " + err);
    rearr_reorder_info r;
    std::memset(&r, 0, sizeof(r));
    r.word_bytes = int(op.word);
    if (op.cls == OC_GATHER && op.gather.l2) {
        const ReorderGeometry gm = reorder_geometry(n, op.word, scatter != 0, reorder_smem_max_buckets());
        r.form = scatter ? REARR_REORDER_LINEAR_SCATTER
                         : gm.smem_scatter ? REARR_REORDER_SMEM_SCATTER : REARR_REORDER_L2_SCATTER;
        r.bucket_chunks = gm.C;
        r.bucket_chunk_elems = uint64_t(1) << gm.cs_shift;
        r.dest_chunks = gm.D;
        r.dest_chunk_elems = scatter ? 0 : uint64_t(1) << gm.ds_shift;
        r.scratch_bytes = gm.bytes;
    }
    *info = r;
    return REARR_OK;
}

rearr_status rearr_memcpy_d2d(void *dst, const void *src, size_t bytes, rearr_stream_t stream)
{
    if (bytes == 0) return REARR_OK;
    if (!dst || !src) return fail(REARR_EINVAL, "rearr_memcpy_d2d: NULL pointer");
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rearr_memcpy_d2d");
    return REARR_OK;
}

uint64_t rearr_launch_count(void) { return g_launches.load(); }

rearr_status rearr_selftest_host(void)
{
    std::string err;
    if (!selftest_host(err)) return fail(REARR_EINVAL, "selftest: " + err);
    return REARR_OK;
}

}  // extern "C"
