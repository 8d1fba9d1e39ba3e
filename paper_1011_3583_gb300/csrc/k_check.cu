// k_check.cu -- device check of index sequences (checked reorder).
//
// Counts the indices >= bound with one read of the sequence: grid-stride
// 16-byte loads, a warp reduction and one atomic per warp that saw any.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/librearr.h"
#include "device_common.cuh"
#include "launch.h"

namespace rearr {
rearr_status fail(rearr_status st, const std::string &msg);
rearr_status cuda_fail(cudaError_t e, const char *what);
}  // namespace rearr

namespace rearr {
namespace {

template <typename T>
__device__ __forceinline__ uint64_t count_vec(const uint4 &v, uint64_t bound)
{
    if constexpr (sizeof(T) == 4) {
        return uint64_t(v.x >= bound) + uint64_t(v.y >= bound) + uint64_t(v.z >= bound) + uint64_t(v.w >= bound);
    } else {
        const uint64_t a = (uint64_t(v.y) << 32) | v.x, b = (uint64_t(v.w) << 32) | v.z;
        return uint64_t(a >= bound) + uint64_t(b >= bound);
    }
}

// idx 16-byte aligned: n_vec whole 16-byte vectors, then a scalar tail.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_check_indices(const T *idx, uint64_t n, uint64_t bound,
                                                            unsigned long long *bad)
{
    constexpr uint64_t PER = 16 / sizeof(T);
    const uint64_t n_vec = n / PER;
    const uint64_t stride = uint64_t(gridDim.x) * kThreads;
    uint64_t c = 0;
    const uint4 *v = reinterpret_cast<const uint4 *>(idx);
    for (uint64_t i = uint64_t(blockIdx.x) * kThreads + threadIdx.x; i < n_vec; i += stride)
        c += count_vec<T>(ldg_stream<16>(v + i), bound);
    for (uint64_t i = n_vec * PER + uint64_t(blockIdx.x) * kThreads + threadIdx.x; i < n; i += stride)
        c += uint64_t(uint64_t(idx[i]) >= bound);
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(bad, static_cast<unsigned long long>(c));
}

// Scalar form for sequences that are not 16-byte aligned.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_check_indices_scalar(const T *idx, uint64_t n, uint64_t bound,
                                                                   unsigned long long *bad)
{
    const uint64_t stride = uint64_t(gridDim.x) * kThreads;
    uint64_t c = 0;
    for (uint64_t i = uint64_t(blockIdx.x) * kThreads + threadIdx.x; i < n; i += stride)
        c += uint64_t(uint64_t(idx[i]) >= bound);
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(bad, static_cast<unsigned long long>(c));
}

}  // namespace

cudaError_t count_bad_indices(const void *idx, size_t n, int idx_bytes, uint64_t bound, uint64_t *n_bad,
                              cudaStream_t s)
{
    *n_bad = 0;
    if (n == 0) return cudaSuccess;
    unsigned long long *d = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d), sizeof(*d), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(d, 0, sizeof(*d), s);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        const uint64_t blocks_needed = (n + kThreads * 4 - 1) / (kThreads * 4);
        const unsigned grid = unsigned(std::min<uint64_t>(blocks_needed, uint64_t(sms) * 8));
        const bool vec = reinterpret_cast<uintptr_t>(idx) % 16 == 0;
        if (idx_bytes == 4) {
            if (vec) k_check_indices<uint32_t><<<grid, kThreads, 0, s>>>(static_cast<const uint32_t *>(idx), n, bound, d);
            else k_check_indices_scalar<uint32_t><<<grid, kThreads, 0, s>>>(static_cast<const uint32_t *>(idx), n, bound, d);
        } else {
            if (vec) k_check_indices<uint64_t><<<grid, kThreads, 0, s>>>(static_cast<const uint64_t *>(idx), n, bound, d);
            else k_check_indices_scalar<uint64_t><<<grid, kThreads, 0, s>>>(static_cast<const uint64_t *>(idx), n, bound, d);
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaError_t ef = cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = ef;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *n_bad = h;
    return e;
}

}  // namespace rearr
