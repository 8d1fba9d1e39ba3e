// device_common.cuh -- typed global / shared memory access helpers for the
// librearr kernels (sm_103a).  Payloads are moved as unsigned integer words,
// never as floating point, so every bit pattern is preserved.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rearr_internal.h"

namespace rearr {

// Word of N bytes.
template <int N> struct Word;
template <> struct Word<1> { using T = uint8_t; };
template <> struct Word<2> { using T = uint16_t; };
template <> struct Word<4> { using T = uint32_t; };
template <> struct Word<8> { using T = uint2; };
template <> struct Word<16> { using T = uint4; };

// Global loads of data read once: non-coherent path, no L1 allocation.
template <int N> __device__ __forceinline__ typename Word<N>::T ldg_stream(const void *p);

template <> __device__ __forceinline__ uint8_t ldg_stream<1>(const void *p)
{
    unsigned short v;
    asm volatile("ld.global.nc.L1::no_allocate.u8 %0, [%1];" : "=h"(v) : "l"(p));
    return uint8_t(v);
}
template <> __device__ __forceinline__ uint16_t ldg_stream<2>(const void *p)
{
    unsigned short v;
    asm volatile("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}
template <> __device__ __forceinline__ uint32_t ldg_stream<4>(const void *p)
{
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
template <> __device__ __forceinline__ uint2 ldg_stream<8>(const void *p)
{
    uint2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];"
                 : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}
template <> __device__ __forceinline__ uint4 ldg_stream<16>(const void *p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

// Global loads that may hit lines other threads also touch (gather sources).
template <int N> __device__ __forceinline__ typename Word<N>::T ldg_any(const void *p)
{
    return __ldg(reinterpret_cast<const typename Word<N>::T *>(p));
}
template <> __device__ __forceinline__ uint8_t ldg_any<1>(const void *p)
{
    return __ldg(reinterpret_cast<const unsigned char *>(p));
}

template <int N> __device__ __forceinline__ void stg(void *p, typename Word<N>::T v)
{
    *reinterpret_cast<typename Word<N>::T *>(p) = v;
}

template <int N> __device__ __forceinline__ void sts(void *p, typename Word<N>::T v)
{
    *reinterpret_cast<typename Word<N>::T *>(p) = v;
}

template <int N> __device__ __forceinline__ typename Word<N>::T lds(const void *p)
{
    return *reinterpret_cast<const typename Word<N>::T *>(p);
}

// L2 eviction priorities (createpolicy): data read or written once is marked
// to leave the L2 first, data that is reused to stay.
__device__ __forceinline__ uint64_t l2_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Loads (non-coherent, no L1 allocation) and stores with an L2 policy.
template <int N> __device__ __forceinline__ typename Word<N>::T ldg_hint(const void *p, uint64_t pol);
template <> __device__ __forceinline__ uint16_t ldg_hint<2>(const void *p, uint64_t pol)
{
    uint16_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
    return v;
}
template <> __device__ __forceinline__ uint32_t ldg_hint<4>(const void *p, uint64_t pol)
{
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
template <> __device__ __forceinline__ uint2 ldg_hint<8>(const void *p, uint64_t pol)
{
    uint2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
                 : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
    return v;
}
template <> __device__ __forceinline__ uint4 ldg_hint<16>(const void *p, uint64_t pol)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p), "l"(pol));
    return v;
}

template <int N> __device__ __forceinline__ void stg_hint(void *p, typename Word<N>::T v, uint64_t pol);
template <> __device__ __forceinline__ void stg_hint<4>(void *p, uint32_t v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}
template <> __device__ __forceinline__ void stg_hint<8>(void *p, uint2 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(p), "r"(v.x), "r"(v.y), "l"(pol)
                 : "memory");
}
template <> __device__ __forceinline__ void stg_hint<16>(void *p, uint4 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w), "l"(pol)
                 : "memory");
}

// Thread index read through a volatile move.  The persistent batched kernel
// runs many inlined tile bodies inside one loop; with a plain threadIdx.x the
// compiler hoists every body's thread-dependent offsets out of that loop and
// keeps them all live, which overflows the register file.
__device__ __forceinline__ int tid_x()
{
    int t;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(t));
    return t;
}

// Byte select of two words (PRMT): result byte i = byte sel_i of {b:a}.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    return __byte_perm(a, b, sel);
}

__device__ __forceinline__ uint32_t word_of(const uint4 &v, int i)
{
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

__device__ __forceinline__ void set_word(uint4 &v, int i, uint32_t w)
{
    if (i == 0) v.x = w;
    else if (i == 1) v.y = w;
    else if (i == 2) v.z = w;
    else v.w = w;
}

}  // namespace rearr
