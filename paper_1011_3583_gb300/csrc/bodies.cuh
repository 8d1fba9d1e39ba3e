// bodies.cuh -- per-work-unit device bodies of every librearr op class.
//
// Each body moves one work unit (a tile, a block of runs, a copy block, ...)
// with the whole CTA of kThreads threads.  The single-op kernels call a body
// once per CTA; the batched persistent kernel calls the body that matches the
// op of every tile it takes from the work list.  Bodies that use shared
// memory end with a barrier so that the caller may reuse the buffer.
#pragma once

#include "device_common.cuh"

namespace rearr {

// ---------------------------------------------------------------------------
// Tiled transpose (arXiv:1011.3583 Sec. III.B): the 2-D plane spanned by the
// input's fastest axis (A) and the output's fastest axis (B) is cut into
// tiles; a tile is read along A (contiguous in the input), staged in shared
// memory, and written along B (contiguous in the output), so both global
// sides are coalesced.  The remaining axes batch the plane.

// Fast tiles hold TBYTES of payload (16 KB, or 8 KB for small planes); the
// staged rows (along A) are ROWB = 128, 256 or 512 bytes, so TB = TBYTES / ROWB
// rows along B.
template <int E, int ROWB, int TBYTES = kTileBytes> struct FastTile {
    static constexpr int TA = ROWB / E;
    static constexpr int TB = TBYTES / ROWB;
};

// Origin of tile t: (a0, b0) in the plane and the byte offsets of its batch.
__device__ __forceinline__ void tile_origin(const TileDesc &d, uint32_t t, uint32_t &a0,
                                            uint32_t &b0, int64_t &in_off, int64_t &out_off)
{
    uint32_t q, ta, tb;
    fdivmod(t, d.ta_div, q, ta);
    fdivmod(q, d.tb_div, q, tb);
    a0 = ta * d.TA;
    b0 = tb * d.TB;
    in_off = 0;
    out_off = 0;
#pragma unroll
    for (int i = kMaxBatch - 1; i >= 0; --i) {
        if (i < d.nb) {
            uint32_t r;
            fdivmod(q, d.bdiv[i], q, r);
            in_off += int64_t(r) * d.bin[i];
            out_off += int64_t(r) * d.bout[i];
        }
    }
}

// Input offset of row b of the (possibly widened) B axis, and output offset
// of element a of the (possibly widened) A axis (TileDesc).
__device__ __forceinline__ int64_t b_row_in(const TileDesc &d, uint32_t b)
{
    uint32_t hi, lo;
    fdivmod(b, d.db_split, hi, lo);
    return int64_t(lo) * d.sb_in + int64_t(hi) * d.sb1_in;
}

__device__ __forceinline__ int64_t a_col_out(const TileDesc &d, uint32_t a)
{
    uint32_t hi, lo;
    fdivmod(a, d.da_split, hi, lo);
    return int64_t(lo) * d.sa_out + int64_t(hi) * d.sa1_out;
}

// Output piece m of a register block: rows r[0..VB) of the staged tile, each
// a 16-byte chunk of 16/E elements along A, give for element m of the chunk
// the VB consecutive B-elements as one word of VB*E bytes.
template <int E, int VB>
__device__ __forceinline__ typename Word<E * VB>::T piece(const uint4 (&r)[VB], int m)
{
    if constexpr (E >= 4) {
        constexpr int EW = E / 4;  // words per element
        uint32_t w[VB * EW];
#pragma unroll
        for (int i = 0; i < VB; ++i)
#pragma unroll
            for (int x = 0; x < EW; ++x) w[i * EW + x] = word_of(r[i], m * EW + x);
        if constexpr (VB * EW == 4) return make_uint4(w[0], w[1], w[2], w[3]);
        else if constexpr (VB * EW == 2) return make_uint2(w[0], w[1]);
        else return w[0];
    } else if constexpr (E == 2) {
        const uint32_t sel = (m & 1) ? 0x7632u : 0x5410u;
        if constexpr (VB == 4) {
            return make_uint2(prmt(word_of(r[0], m >> 1), word_of(r[1], m >> 1), sel),
                              prmt(word_of(r[2], m >> 1), word_of(r[3], m >> 1), sel));
        } else if constexpr (VB == 2) {
            return prmt(word_of(r[0], m >> 1), word_of(r[1], m >> 1), sel);
        } else {
            const uint32_t w = word_of(r[0], m >> 1);
            return uint16_t((m & 1) ? (w >> 16) : (w & 0xFFFFu));
        }
    } else {  // E == 1
        const uint32_t bp = uint32_t(m & 3);
        const uint32_t sel = bp | ((4u + bp) << 4);
        if constexpr (VB == 4) {
            const uint32_t lo = prmt(word_of(r[0], m >> 2), word_of(r[1], m >> 2), sel);
            const uint32_t hi = prmt(word_of(r[2], m >> 2), word_of(r[3], m >> 2), sel);
            return prmt(lo, hi, 0x5410u);
        } else if constexpr (VB == 2) {
            return uint16_t(prmt(word_of(r[0], m >> 2), word_of(r[1], m >> 2), sel) & 0xFFFFu);
        } else {
            return uint8_t((word_of(r[0], m >> 2) >> (8 * bp)) & 0xFFu);
        }
    }
}

// Fast tile: cells are single E-byte elements (E a power of two <= 16).
// VIN: width of the global loads along A; VOUT: width of the global stores
// along B (VOUT/E = VB consecutive B-elements per store).  Shared memory holds
// the tile row-major by B with 16-byte chunks XOR-swizzled by (row/VB)&7, so
// the 16-byte row stores of the load phase and the 16-byte column-block loads
// of the store phase are both free of bank conflicts.
template <int E, int VIN, int VOUT, int ROWB, int TBYTES = kTileBytes>
__device__ __forceinline__ void tile_fast_body(const TileDesc &d, uint32_t t, unsigned char *smem)
{
    constexpr int TA = FastTile<E, ROWB, TBYTES>::TA, TB = FastTile<E, ROWB, TBYTES>::TB;
    constexpr int V = 16 / E;        // elements per 16-byte chunk
    constexpr int VB = VOUT / E;     // B-elements per output store
    constexpr int PPR = ROWB / VIN;  // load pieces per row
    constexpr int NP = TB * PPR;
    constexpr int PT = NP / kThreads;
    static_assert(NP % kThreads == 0, "tile must split evenly over the CTA");
    static_assert(ROWB % 128 == 0, "swizzle works on groups of 8 chunks");
    static_assert(VB >= 1 && VB <= 4, "output block of 1..4 rows");
    static_assert(TB / VB >= 8, "eight row groups per swizzle period");

    uint32_t a0, b0;
    int64_t ioff, ooff;
    tile_origin(d, t, a0, b0, ioff, ooff);
    const uint32_t na = min(uint32_t(TA), d.DA - a0);
    const uint32_t nbv = min(uint32_t(TB), d.DB - b0);
    const char *in = d.src + ioff + int64_t(a0) * E;
    char *out = d.dst + ooff + int64_t(b0) * E;
    const int tid = tid_x();
    const uint32_t row_valid_bytes = na * E;
    // a widened A whose planes end inside 16-byte chunks
    const bool fine_split = d.sa1_out != 0 && (d.da_split.d & uint32_t(V - 1)) != 0;

    // Loads are issued in batches of up to 8 per thread before their shared
    // stores, which keeps narrow-width variants within the register budget.
    constexpr int PB = PT < 8 ? PT : 8;
    static_assert(PT % PB == 0, "load batches must divide the per-thread pieces");
#pragma unroll
    for (int k0 = 0; k0 < PT; k0 += PB) {
        typename Word<VIN>::T buf[PB];
#pragma unroll
        for (int k = 0; k < PB; ++k) {
            const int f = (k0 + k) * kThreads + tid;
            const int row = f / PPR, x = (f % PPR) * VIN;
            if (uint32_t(row) < nbv && uint32_t(x) < row_valid_bytes)
                buf[k] = ldg_stream<VIN>(in + b_row_in(d, b0 + uint32_t(row)) + x);
        }
#pragma unroll
        for (int k = 0; k < PB; ++k) {
            const int f = (k0 + k) * kThreads + tid;
            const int row = f / PPR, x = (f % PPR) * VIN;
            if (uint32_t(row) < nbv && uint32_t(x) < row_valid_bytes) {
                const int sw = (row / VB) & 7;
                sts<VIN>(smem + row * ROWB + (((x >> 4) ^ sw) << 4) + (x & 15), buf[k]);
            }
        }
    }
    __syncthreads();

    constexpr int UB = TB / VB, UQ = TA / V, NU = UB * UQ;
    static_assert(NU % kThreads == 0, "store units must split evenly");
#pragma unroll
    for (int u0 = 0; u0 < NU; u0 += kThreads) {
        const int u = u0 + tid;
        const int bq = u % UB, q = u / UB;
        const int b = bq * VB;
        if (uint32_t(b) < nbv) {
            uint4 r[VB];
#pragma unroll
            for (int i = 0; i < VB; ++i)
                r[i] = lds<16>(smem + (b + i) * ROWB + ((q ^ (bq & 7)) << 4));
            if (fine_split) {
                // a widened A that splits inside a chunk: each element's own
                // output row
#pragma unroll
                for (int m = 0; m < V; ++m) {
                    const uint32_t a = uint32_t(q * V + m);
                    if (a < na) stg<VOUT>(out + a_col_out(d, a0 + a) + int64_t(b) * E, piece<E, VB>(r, m));
                }
            } else {
                // the V elements of chunk q share their absorbed index
                char *col = out + a_col_out(d, a0 + uint32_t(q * V)) + int64_t(b) * E;
#pragma unroll
                for (int m = 0; m < V; ++m) {
                    const uint32_t a = uint32_t(q * V + m);
                    if (a < na) stg<VOUT>(col + int64_t(m) * d.sa_out, piece<E, VB>(r, m));
                }
            }
        }
    }
    __syncthreads();
}

// The fast tile in two phases for pipelined ranges of tiles: tile_fast_issue
// starts the tile's global -> shared copies as cp.async (no registers held,
// 16-byte copies bypass the L1) into the same swizzled layout as
// tile_fast_body, and commits them as one group; tile_fast_store runs the
// store phase from shared memory once the group has landed (the caller waits
// with cp.async.wait_group and a block barrier).  A CTA can so copy tile t+1
// into a second buffer while it stores tile t.
template <int N>
__device__ __forceinline__ void cp_async(void *smem_dst, const void *gsrc)
{
    const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    if constexpr (N == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gsrc), "n"(N) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int PENDING>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory"); }

template <int E, int VIN, int VOUT, int ROWB, int TBYTES = kTileBytes>
__device__ __forceinline__ void tile_fast_issue(const TileDesc &d, uint32_t t, unsigned char *smem)
{
    constexpr int TA = FastTile<E, ROWB, TBYTES>::TA, TB = FastTile<E, ROWB, TBYTES>::TB;
    constexpr int VB = VOUT / E;
    constexpr int PPR = ROWB / VIN;
    constexpr int NP = TB * PPR;
    constexpr int PT = NP / kThreads;
    static_assert(NP % kThreads == 0, "tile must split evenly over the CTA");
    static_assert(VIN == 4 || VIN == 8 || VIN == 16, "cp.async copies 4, 8 or 16 bytes");
    uint32_t a0, b0;
    int64_t ioff, ooff;
    tile_origin(d, t, a0, b0, ioff, ooff);
    const uint32_t na = min(uint32_t(TA), d.DA - a0);
    const uint32_t nbv = min(uint32_t(TB), d.DB - b0);
    const char *in = d.src + ioff + int64_t(a0) * E;
    const uint32_t row_valid_bytes = na * E;
    const int tid = tid_x();
#pragma unroll
    for (int k = 0; k < PT; ++k) {
        const int f = k * kThreads + tid;
        const int row = f / PPR, x = (f % PPR) * VIN;
        if (uint32_t(row) < nbv && uint32_t(x) < row_valid_bytes) {
            const int sw = (row / VB) & 7;
            cp_async<VIN>(smem + row * ROWB + (((x >> 4) ^ sw) << 4) + (x & 15),
                          in + b_row_in(d, b0 + uint32_t(row)) + x);
        }
    }
    cp_async_commit();
}

template <int E, int VIN, int VOUT, int ROWB, int TBYTES = kTileBytes>
__device__ __forceinline__ void tile_fast_store(const TileDesc &d, uint32_t t, const unsigned char *smem)
{
    constexpr int TA = FastTile<E, ROWB, TBYTES>::TA, TB = FastTile<E, ROWB, TBYTES>::TB;
    constexpr int V = 16 / E;
    constexpr int VB = VOUT / E;
    uint32_t a0, b0;
    int64_t ioff, ooff;
    tile_origin(d, t, a0, b0, ioff, ooff);
    const uint32_t na = min(uint32_t(TA), d.DA - a0);
    const uint32_t nbv = min(uint32_t(TB), d.DB - b0);
    char *out = d.dst + ooff + int64_t(b0) * E;
    const int tid = tid_x();
    // a widened A whose planes end inside 16-byte chunks
    const bool fine_split = d.sa1_out != 0 && (d.da_split.d & uint32_t(V - 1)) != 0;
    constexpr int UB = TB / VB, UQ = TA / V, NU = UB * UQ;
    static_assert(NU % kThreads == 0, "store units must split evenly");
#pragma unroll
    for (int u0 = 0; u0 < NU; u0 += kThreads) {
        const int u = u0 + tid;
        const int bq = u % UB, q = u / UB;
        const int b = bq * VB;
        if (uint32_t(b) < nbv) {
            uint4 r[VB];
#pragma unroll
            for (int i = 0; i < VB; ++i) r[i] = lds<16>(smem + (b + i) * ROWB + ((q ^ (bq & 7)) << 4));
            if (fine_split) {
#pragma unroll
                for (int m = 0; m < V; ++m) {
                    const uint32_t a = uint32_t(q * V + m);
                    if (a < na) stg<VOUT>(out + a_col_out(d, a0 + a) + int64_t(b) * E, piece<E, VB>(r, m));
                }
            } else {
                char *col = out + a_col_out(d, a0 + uint32_t(q * V)) + int64_t(b) * E;
#pragma unroll
                for (int m = 0; m < V; ++m) {
                    const uint32_t a = uint32_t(q * V + m);
                    if (a < na) stg<VOUT>(col + int64_t(m) * d.sa_out, piece<E, VB>(r, m));
                }
            }
        }
    }
}

// Cells tile: each cell is c words of W bytes (any cell size; used for
// element sizes that are not a power of two, unaligned element addresses and
// permutes whose innermost axis is unmoved but short).  Rows are padded to a
// pitch P = c (mod 32) words, which makes the column walk of the store phase
// touch consecutive banks.
template <int W>
__device__ __forceinline__ void tile_cells_body(const TileDesc &d, uint32_t t, unsigned char *smem_raw)
{
    using T = typename Word<W>::T;
    T *smem = reinterpret_cast<T *>(smem_raw);
    uint32_t a0, b0;
    int64_t ioff, ooff;
    tile_origin(d, t, a0, b0, ioff, ooff);
    const uint32_t c = d.c, P = d.pitch;
    const uint32_t na = min(d.TA, d.DA - a0);
    const uint32_t nbv = min(d.TB, d.DB - b0);
    const char *in = d.src + ioff + int64_t(a0) * c * W + int64_t(b0) * d.sb_in;
    char *out = d.dst + ooff + int64_t(a0) * d.sa_out + int64_t(b0) * c * W;
    const int tid = tid_x();
    constexpr int U = 8;

    const uint32_t RW = d.rowwords_div.d;  // TA*c
    const uint32_t total_in = d.TB * RW;
    const uint32_t rw_valid = na * c;
    for (uint32_t base = 0; base < total_in; base += kThreads * U) {
        T v[U];
        uint32_t row[U], w[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t f = base + k * kThreads + tid;
            fdivmod(f, d.rowwords_div, row[k], w[k]);
            if (f < total_in && row[k] < nbv && w[k] < rw_valid)
                v[k] = ldg_stream<W>(in + int64_t(row[k]) * d.sb_in + int64_t(w[k]) * W);
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t f = base + k * kThreads + tid;
            if (f < total_in && row[k] < nbv && w[k] < rw_valid) smem[row[k] * P + w[k]] = v[k];
        }
    }
    __syncthreads();

    const uint32_t OW = d.outwords_div.d;  // TB*c
    const uint32_t total_out = d.TA * OW;
    const uint32_t ow_valid = nbv * c;
    for (uint32_t base = 0; base < total_out; base += kThreads * U) {
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t f = base + k * kThreads + tid;
            uint32_t arow, w, b, kk;
            fdivmod(f, d.outwords_div, arow, w);
            if (f < total_out && arow < na && w < ow_valid) {
                fdivmod(w, d.c_div, b, kk);
                stg<W>(out + int64_t(arow) * d.sa_out + int64_t(w) * W, smem[b * P + arow * c + kk]);
            }
        }
    }
    __syncthreads();
}

// Blocked runs (a cells tile with pitch 0): cells of 128 bytes or more -- an
// unmoved inner run of the permute -- on the transpose plane, TA x TB cells
// per tile, copied word for word without staging (a cell is at least one
// whole 128-byte line, so each side is coalesced as it is).  Consecutive
// words walk the tile's input rows, so a tile reads TB runs of TA * cell
// contiguous bytes and writes TA runs of TB * cell contiguous bytes, where a
// walk in output (or input) order reads (or writes) one cell per DRAM burst
// run.  No shared memory is used.
template <int W>
__device__ __forceinline__ void tile_runs_body(const TileDesc &d, uint32_t t)
{
    uint32_t a0, b0;
    int64_t ioff, ooff;
    tile_origin(d, t, a0, b0, ioff, ooff);
    const uint32_t c = d.c;
    const uint32_t na = min(d.TA, d.DA - a0);
    const uint32_t nbv = min(d.TB, d.DB - b0);
    const char *in = d.src + ioff + int64_t(a0) * c * W + int64_t(b0) * d.sb_in;
    char *out = d.dst + ooff + int64_t(a0) * d.sa_out + int64_t(b0) * c * W;
    const uint32_t total = d.TB * d.rowwords_div.d;  // TB rows of TA * c words
    const uint32_t rw_valid = na * c;
    constexpr int U = W >= 16 ? 4 : 8;
    for (uint32_t base = 0; base < total; base += kThreads * U) {
        typename Word<W>::T v[U];
        uint32_t row[U], w[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t f = base + k * kThreads + tid_x();
            fdivmod(f, d.rowwords_div, row[k], w[k]);
            if (f < total && row[k] < nbv && w[k] < rw_valid)
                v[k] = ldg_stream<W>(in + int64_t(row[k]) * d.sb_in + int64_t(w[k]) * W);
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t f = base + k * kThreads + tid_x();
            if (f < total && row[k] < nbv && w[k] < rw_valid) {
                uint32_t a, ww;
                fdivmod(w[k], d.c_div, a, ww);
                stg<W>(out + int64_t(a) * d.sa_out + (int64_t(row[k]) * c + ww) * W, v[k]);
            }
        }
    }
}

// A cells tile: staged in shared memory, or (pitch 0) blocked runs.
template <int W>
__device__ __forceinline__ void tile_cells_any(const TileDesc &d, uint32_t t, unsigned char *smem)
{
    if (d.pitch == 0) tile_runs_body<W>(d, t);
    else tile_cells_body<W>(d, t, smem);
}

// ---------------------------------------------------------------------------
// Runs: permutes whose output is a sequence of contiguous input runs of at
// least 128 bytes (an unmoved innermost axis, or large elements).  A unit is
// runs_per_unit consecutive output runs: their input offsets are decoded
// once into shared memory, then the CTA walks the unit's words with U loads
// in flight per thread; consecutive threads take consecutive words, so both
// sides are coalesced however short the runs are.
__device__ __forceinline__ int64_t run_offset(const RunsDesc &d, uint32_t q)
{
    int64_t off = 0;
#pragma unroll
    for (int a = kMaxRank - 1; a >= 0; --a) {
        if (a < d.nd) {
            uint32_t dig;
            fdivmod(q, d.div[a], q, dig);
            off += int64_t(dig) * d.in_stride[a];
        }
    }
    return off;
}

template <int W>
__device__ __forceinline__ void copy_words(const char *src, char *dst, uint32_t w0, uint32_t w1)
{
    constexpr int U = W >= 16 ? 4 : 8;  // 64 bytes in flight per thread for 16-byte words (80 registers at U = 8)
    for (uint32_t b = w0; b < w1; b += kThreads * U) {
        typename Word<W>::T v[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t w = b + k * kThreads + tid_x();
            if (w < w1) v[k] = ldg_stream<W>(src + int64_t(w) * W);
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t w = b + k * kThreads + tid_x();
            if (w < w1) stg<W>(dst + int64_t(w) * W, v[k]);
        }
    }
}

template <int W>
__device__ __forceinline__ void runs_body(const RunsDesc &d, uint64_t unit, unsigned char *smem)
{
    if (d.cpr_div.d > 1) {
        // Long runs: a unit is one chunk of chunk_words words of one run.
        uint32_t run, ch;
        fdivmod(uint32_t(unit), d.cpr_div, run, ch);
        const uint32_t wpr = d.wpr_div.d;
        const uint32_t w0 = ch * d.chunk_words;
        const uint32_t w1 = min(wpr, w0 + d.chunk_words);
        copy_words<W>(d.src + run_offset(d, run), d.dst + int64_t(run) * d.run_bytes, w0, w1);
        return;
    }
    int64_t *base = reinterpret_cast<int64_t *>(smem);
    const uint64_t r0 = unit * d.runs_per_unit;
    const uint32_t nr = uint32_t(min(d.n_runs - r0, uint64_t(d.runs_per_unit)));
    for (uint32_t i = tid_x(); i < nr; i += kThreads) base[i] = run_offset(d, uint32_t(r0 + i));
    __syncthreads();
    const uint32_t wpr = d.wpr_div.d;  // words per run
    const uint32_t total = nr * wpr;
    char *out = d.dst + int64_t(r0) * d.run_bytes;
    constexpr int U = W >= 16 ? 4 : 8;  // 64 bytes in flight per thread for 16-byte words (80 registers at U = 8)
    if (d.mirror) {
        // Runs walked in input order: the input is read contiguously and
        // base[] holds each run's output offset (short runs: sequential reads
        // keep DRAM rows open, the scattered writes are whole runs).
        const char *in = d.src + int64_t(r0) * d.run_bytes;
        for (uint32_t f0 = 0; f0 < total; f0 += kThreads * U) {
            typename Word<W>::T v[U];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const uint32_t f = f0 + k * kThreads + tid_x();
                if (f < total) v[k] = ldg_stream<W>(in + int64_t(f) * W);
            }
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const uint32_t f = f0 + k * kThreads + tid_x();
                if (f < total) {
                    uint32_t r, w;
                    fdivmod(f, d.wpr_div, r, w);
                    stg<W>(d.dst + base[r] + int64_t(w) * W, v[k]);
                }
            }
        }
        __syncthreads();
        return;
    }
    for (uint32_t f0 = 0; f0 < total; f0 += kThreads * U) {
        typename Word<W>::T v[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t f = f0 + k * kThreads + tid_x();
            if (f < total) {
                uint32_t r, w;
                fdivmod(f, d.wpr_div, r, w);
                v[k] = ldg_stream<W>(d.src + base[r] + int64_t(w) * W);
            }
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t f = f0 + k * kThreads + tid_x();
            if (f < total) stg<W>(out + int64_t(f) * W, v[k]);
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Contiguous copy (Sec. III.A, the sequential read/write kernel): each thread
// moves U words of W bytes per unit, all loads issued before the stores.
template <int W>
__device__ __forceinline__ void copy_body(const CopyDesc &d, uint64_t unit)
{
    constexpr int U = 4;
    const uint64_t base = unit * d.unit_bytes;
    typename Word<W>::T v[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
        const uint64_t off = base + uint64_t(k * kThreads + tid_x()) * W;
        if (off < d.bytes) v[k] = ldg_stream<W>(d.src + off);
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
        const uint64_t off = base + uint64_t(k * kThreads + tid_x()) * W;
        if (off < d.bytes) stg<W>(d.dst + off, v[k]);
    }
}

// ---------------------------------------------------------------------------
// Reorder by an index sequence (Sec. III.A, indexed access): dst[i] = src[idx[i]].

template <int W>
__device__ __forceinline__ void store4(char *p, const typename Word<W>::T (&v)[4])
{
    if constexpr (W == 1) {
        stg<4>(p, uint32_t(v[0]) | (uint32_t(v[1]) << 8) | (uint32_t(v[2]) << 16) | (uint32_t(v[3]) << 24));
    } else if constexpr (W == 2) {
        stg<8>(p, make_uint2(uint32_t(v[0]) | (uint32_t(v[1]) << 16), uint32_t(v[2]) | (uint32_t(v[3]) << 16)));
    } else if constexpr (W == 4) {
        stg<16>(p, make_uint4(v[0], v[1], v[2], v[3]));
    } else if constexpr (W == 8) {
        stg<16>(p, make_uint4(v[0].x, v[0].y, v[1].x, v[1].y));
        stg<16>(p + 16, make_uint4(v[2].x, v[2].y, v[3].x, v[3].y));
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) stg<16>(p + 16 * k, v[k]);
    }
}

// store4 with an L2 policy on every store.
template <int W>
__device__ __forceinline__ void store4_hint(char *p, const typename Word<W>::T (&v)[4], uint64_t pol)
{
    if constexpr (W == 1) {
        stg_hint<4>(p, uint32_t(v[0]) | (uint32_t(v[1]) << 8) | (uint32_t(v[2]) << 16) | (uint32_t(v[3]) << 24), pol);
    } else if constexpr (W == 2) {
        stg_hint<8>(p, make_uint2(uint32_t(v[0]) | (uint32_t(v[1]) << 16), uint32_t(v[2]) | (uint32_t(v[3]) << 16)),
                    pol);
    } else if constexpr (W == 4) {
        stg_hint<16>(p, make_uint4(v[0], v[1], v[2], v[3]), pol);
    } else if constexpr (W == 8) {
        stg_hint<16>(p, make_uint4(v[0].x, v[0].y, v[1].x, v[1].y), pol);
        stg_hint<16>(p + 16, make_uint4(v[2].x, v[2].y, v[3].x, v[3].y), pol);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) stg_hint<16>(p + 16 * k, v[k], pol);
    }
}

// Four consecutive W-byte words from an address aligned to min(16, 4W).
template <int W>
__device__ __forceinline__ void load4(const char *p, typename Word<W>::T (&v)[4])
{
    if constexpr (W == 1) {
        const uint32_t x = ldg_stream<4>(p);
        v[0] = uint8_t(x); v[1] = uint8_t(x >> 8); v[2] = uint8_t(x >> 16); v[3] = uint8_t(x >> 24);
    } else if constexpr (W == 2) {
        const uint2 x = ldg_stream<8>(p);
        v[0] = uint16_t(x.x); v[1] = uint16_t(x.x >> 16); v[2] = uint16_t(x.y); v[3] = uint16_t(x.y >> 16);
    } else if constexpr (W == 4) {
        const uint4 x = ldg_stream<16>(p);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else if constexpr (W == 8) {
        const uint4 a = ldg_stream<16>(p), b = ldg_stream<16>(p + 16);
        v[0] = make_uint2(a.x, a.y); v[1] = make_uint2(a.z, a.w); v[2] = make_uint2(b.x, b.y); v[3] = make_uint2(b.z, b.w);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = ldg_stream<16>(p + 16 * k);
    }
}

template <int W>
__device__ __forceinline__ void gather_body(const GatherDesc &d, uint64_t unit)
{
    using T = typename Word<W>::T;
    const uint64_t e0 = unit * d.unit_elems;
    const uint64_t e1 = min(d.n, e0 + d.unit_elems);
    if (d.vec && d.scatter) {
        // Scatter, groups of 4 consecutive elements per thread: one 16-byte
        // index load, one 4*W-byte source load, four independent stores.
        constexpr int G = 2;
        for (uint64_t g0 = e0; g0 < e1; g0 += uint64_t(kThreads) * 4 * G) {
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const uint64_t i = g0 + (uint64_t(k) * kThreads + tid_x()) * 4;
                if (i + 3 < e1) {
                    const uint4 ix = ldg_stream<16>(d.idx + i);
                    T v[4];
                    load4<W>(d.src + i * W, v);
                    stg<W>(d.dst + uint64_t(ix.x) * W, v[0]);
                    stg<W>(d.dst + uint64_t(ix.y) * W, v[1]);
                    stg<W>(d.dst + uint64_t(ix.z) * W, v[2]);
                    stg<W>(d.dst + uint64_t(ix.w) * W, v[3]);
                } else {
                    for (uint64_t q = i; q < e1 && q < i + 4; ++q)
                        stg<W>(d.dst + uint64_t(d.idx[q]) * W, ldg_any<W>(d.src + q * W));
                }
            }
        }
    } else if (d.vec) {
        // Groups of 4 consecutive elements per thread: one 16-byte index load,
        // four independent source loads, one store of 4*W bytes.  The index
        // and destination streams are marked to leave the L2 first, so that
        // the randomly read source stays resident (many ops are in flight in
        // the batched kernel).
        constexpr int G = 2;  // groups per thread in flight
        const uint64_t stream_pol = l2_evict_first();
        for (uint64_t g0 = e0; g0 < e1; g0 += uint64_t(kThreads) * 4 * G) {
            T v[G][4];
            bool full[G];
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const uint64_t i = g0 + (uint64_t(k) * kThreads + tid_x()) * 4;
                full[k] = i + 3 < e1;
                if (full[k]) {
                    const uint4 ix = ldg_hint<16>(d.idx + i, stream_pol);
                    v[k][0] = ldg_any<W>(d.src + uint64_t(ix.x) * W);
                    v[k][1] = ldg_any<W>(d.src + uint64_t(ix.y) * W);
                    v[k][2] = ldg_any<W>(d.src + uint64_t(ix.z) * W);
                    v[k][3] = ldg_any<W>(d.src + uint64_t(ix.w) * W);
                } else {
                    for (uint64_t j = i; j < e1 && j < i + 4; ++j)
                        stg<W>(d.dst + j * W, ldg_any<W>(d.src + uint64_t(d.idx[j]) * W));
                }
            }
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const uint64_t i = g0 + (uint64_t(k) * kThreads + tid_x()) * 4;
                if (full[k]) store4_hint<W>(d.dst + i * W, v[k], stream_pol);
            }
        }
    } else {
        // Any element size, 32- or 64-bit indices, gather or scatter: c words
        // per element, U elements per thread in flight.
        constexpr int U = 4;
        const uint32_t c = d.c;
        const uint64_t *idx64 = reinterpret_cast<const uint64_t *>(d.idx);
        for (uint64_t b0 = e0; b0 < e1; b0 += uint64_t(kThreads) * U) {
            uint64_t j[U];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const uint64_t i = b0 + uint64_t(k) * kThreads + tid_x();
                j[k] = i < e1 ? (d.idx64 ? __ldg(idx64 + i) : uint64_t(ldg_stream<4>(d.idx + i))) : 0u;
            }
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const uint64_t i = b0 + uint64_t(k) * kThreads + tid_x();
                if (i < e1) {
                    const uint64_t from = d.scatter ? i : j[k], to = d.scatter ? j[k] : i;
                    const char *s = d.src + from * c * W;
                    char *o = d.dst + to * c * W;
                    for (uint32_t w = 0; w < c; ++w) stg<W>(o + w * W, ldg_any<W>(s + w * W));
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Interlace / de-interlace (Sec. III.C).  The fast form works on 16-byte
// groups: a thread reads one 16-byte group from each of the K planes
// (V = 16/E records) and writes the K*16 interleaved bytes of those records
// contiguously, re-interleaving in registers; de-interlace is the inverse.
// Every byte move is fixed at compile time (word moves for E >= 4, PRMT byte
// selects below that), so no shared memory is needed.

template <int E, int K>
__device__ __forceinline__ void interleave_regs(const uint32_t (&in)[K][4], uint32_t (&out)[K * 4])
{
#pragma unroll
    for (int ow = 0; ow < K * 4; ++ow) {
        if constexpr (E >= 4) {
            const int ob = ow * 4, oe = ob / E, bb = ob % E;
            const int i = oe / K, j = oe % K;
            out[ow] = in[j][(i * E + bb) / 4];
        } else {
            uint32_t w = 0;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int ob = ow * 4 + p, oe = ob / E, bb = ob % E;
                const int i = oe / K, j = oe % K, sb = i * E + bb;
                // insert byte (sb & 3) of the source word at byte p of w
                const uint32_t sel = (0x3210u & ~(0xFu << (4 * p))) | (uint32_t(4 + (sb & 3)) << (4 * p));
                w = prmt(w, in[j][sb / 4], sel);
            }
            out[ow] = w;
        }
    }
}

template <int E, int K>
__device__ __forceinline__ void deinterleave_regs(const uint32_t (&in)[K * 4], uint32_t (&out)[K][4])
{
#pragma unroll
    for (int j = 0; j < K; ++j) {
#pragma unroll
        for (int pw = 0; pw < 4; ++pw) {
            if constexpr (E >= 4) {
                const int sb = pw * 4, i = sb / E, bb = sb % E;
                const int ob = (i * K + j) * E + bb;
                out[j][pw] = in[ob / 4];
            } else {
                uint32_t w = 0;
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const int sb = pw * 4 + p, i = sb / E, bb = sb % E;
                    const int ob = (i * K + j) * E + bb;
                    const uint32_t sel = (0x3210u & ~(0xFu << (4 * p))) | (uint32_t(4 + (ob & 3)) << (4 * p));
                    w = prmt(w, in[ob / 4], sel);
                }
                out[j][pw] = w;
            }
        }
    }
}

// Element-wise tail of an interlace / de-interlace: records [r0, n).
template <int E>
__device__ __forceinline__ void interlace_tail(const InterlaceDesc &d, char *const *planes, uint64_t r0,
                                               bool inter)
{
    const uint64_t cnt = (d.n - r0) * d.k;
    for (uint64_t f = tid_x(); f < cnt; f += kThreads) {
        const uint64_t i = r0 + f / d.k;
        const uint32_t j = uint32_t(f % d.k);
        char *iv = d.inter + (i * d.k + j) * E;
        char *pl = planes[j] + i * E;
        if (inter) stg<E>(iv, lds<E>(pl));  // plain (coherent) loads: tail is tiny
        else stg<E>(pl, lds<E>(iv));
    }
}

// Element-wise strided copy (OC_STRIDED): permutes whose transpose plane is
// too small to fill a tile (a tile per tiny plane would move a few dozen
// bytes per pass).  Each output cell's input offset is decomposed directly
// from its index; the writes are coalesced (consecutive cells per thread,
// 16-byte stores when aligned) and the reads hit the L1 / L2 wherever
// neighbouring cells share sectors.
// ND > 0: the number of output axes fixed at compile time (no per-axis test);
// ND = 0: read from the descriptor.
template <int ND>
__device__ __forceinline__ int64_t strided_offset(const StridedDesc &d, uint32_t q)
{
    constexpr int R = ND > 0 ? ND : kMaxRank;
    int64_t off = 0;
#pragma unroll
    for (int i = R - 1; i >= 0; --i) {
        if (ND > 0 || i < d.nd) {
            uint32_t r;
            fdivmod(q, d.div[i], q, r);
            off += int64_t(r) * d.in_stride[i];
        }
    }
    return off;
}

template <int W, int ND = 0>
__device__ __forceinline__ void strided_body(const StridedDesc &d, uint64_t unit)
{
    constexpr int V = 16 / W;  // cells per 16-byte store
    constexpr int R = ND > 0 ? ND : kMaxRank;
    using T = typename Word<W>::T;
    const uint64_t per_unit = uint64_t(kThreads) * V * kStridedSteps;
    const uint64_t c0 = unit * per_unit;
    const uint64_t c1 = min(d.n_cells, c0 + per_unit);
    const int tid = tid_x();
    if (d.vec) {
        for (uint64_t base = c0 + uint64_t(tid) * V; base < c1; base += uint64_t(kThreads) * V) {
            union {
                uint4 u;
                T e[V];
            } v;
            v.u = make_uint4(0, 0, 0, 0);
            // The thread's V consecutive cells: the first one's input offset
            // from its multi-index (one division per axis), the next ones by
            // stepping the multi-index like an odometer (an add per cell, a
            // carry into the next axis when an extent is reached).
            uint32_t digit[R];
            int64_t off = 0;
            {
                uint32_t q = uint32_t(base);
#pragma unroll
                for (int i = R - 1; i >= 0; --i) {
                    digit[i] = 0;
                    if (ND > 0 || i < d.nd) {
                        fdivmod(q, d.div[i], q, digit[i]);
                        off += int64_t(digit[i]) * d.in_stride[i];
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < V; ++k) {
                if (base + k < c1) v.e[k] = ldg_any<W>(d.src + off);
#pragma unroll
                for (int i = R - 1; i >= 0; --i) {
                    if (ND > 0 || i < d.nd) {
                        off += d.in_stride[i];
                        if (++digit[i] < d.div[i].d) break;
                        off -= int64_t(d.div[i].d) * d.in_stride[i];
                        digit[i] = 0;
                    }
                }
            }
            if (base + V <= c1) {
                stg<16>(d.dst + base * W, v.u);
            } else {
#pragma unroll
                for (int k = 0; k < V; ++k)
                    if (base + k < c1) stg<W>(d.dst + (base + k) * W, v.e[k]);
            }
        }
    } else {
        for (uint64_t q = c0 + tid; q < c1; q += kThreads)
            stg<W>(d.dst + q * W, ldg_any<W>(d.src + strided_offset<ND>(d, uint32_t(q))));
    }
}

// Box permute (OC_BOX): one unit is the sub-box U of its unit index (see
// BoxDesc).  Every full unit has the same shape, so a thread visits the same
// cells of each: its first cell's digits (U in input order for the loads, in
// output order for the stores) come from one decomposition, and each next
// cell of the thread (kThreads loads or stores further on) from adding the
// digits of that stride with carries -- no division per cell.
// Load phase: VL bytes per load (a load never spans two runs of the input
// chain), stored densely in input order in shared memory.  Store phase:
// V = VO / E consecutive cells of an output run per thread, each read from its
// shared-memory slot (stepping the output digits like an odometer), written
// with one VO-byte store.  Cells whose partial-axis index is past the axis'
// end (its last range) are neither read nor written; that unit moves single
// cells on both sides.

// Digits of n over the first NU extents (fastest first).
template <int NU>
__device__ __forceinline__ void box_digits(uint32_t n, const FastDiv *ext, uint32_t (&dig)[NU])
{
#pragma unroll
    for (int i = 0; i < NU; ++i) fdivmod(n, ext[i], n, dig[i]);
}

// dig += step in the mixed radix of the extents (every step digit is below
// its extent, so each digit wraps at most once).
template <int NU>
__device__ __forceinline__ void box_advance(uint32_t (&dig)[NU], const uint32_t (&step)[NU], const uint32_t (&ext)[NU])
{
    uint32_t carry = 0;
#pragma unroll
    for (int i = 0; i < NU; ++i) {
        const uint32_t v = dig[i] + step[i] + carry;
        carry = v >= ext[i];
        dig[i] = carry ? v - ext[i] : v;
    }
}

template <int E, int VL, int NU>
__device__ __forceinline__ void box_load(const BoxDesc &d, const char *in, uint32_t keff, unsigned char *smem)
{
    constexpr int B = VL >= 8 ? 4 : 8;  // loads in flight per thread (a unit is at most 4 16-byte loads per thread)
    constexpr uint32_t CV = VL / E;     // cells per load
    const uint32_t cells = d.cells;
    const uint32_t c0 = uint32_t(tid_x()) * CV;
    uint32_t dig[NU], step[NU], ext[NU];
    box_digits<NU>(c0, d.iext, dig);
    box_digits<NU>(uint32_t(kThreads) * CV, d.iext, step);
#pragma unroll
    for (int i = 0; i < NU; ++i) ext[i] = d.iext[i].d;
    for (uint32_t c = c0; c < cells; c += uint32_t(kThreads) * CV * B) {
        typename Word<VL>::T r[B];
        bool ok[B];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const uint32_t cj = c + uint32_t(j) * kThreads * CV;
            ok[j] = false;
            if (cj < cells) {
                int64_t off = 0;
                uint32_t kd = 0;
#pragma unroll
                for (int i = 0; i < NU; ++i) {
                    off += int64_t(dig[i]) * d.iin[i];
                    if (i == d.kin) kd = dig[i];
                }
                if (kd < keff) {
                    r[j] = ldg_stream<VL>(in + off);
                    ok[j] = true;
                }
                box_advance<NU>(dig, step, ext);
            }
        }
#pragma unroll
        for (int j = 0; j < B; ++j)
            if (ok[j]) sts<VL>(smem + (c + uint32_t(j) * kThreads * CV) * E, r[j]);
    }
}

template <int E, int VO, int NU>
__device__ __forceinline__ void box_store(const BoxDesc &d, char *out, uint32_t keff, const unsigned char *smem)
{
    constexpr int V = VO / E;
    const uint32_t cells = d.cells;
    const uint32_t y0 = uint32_t(tid_x()) * V;
    uint32_t dig[NU], step[NU], ext[NU], sms[NU];
    box_digits<NU>(y0, d.oext, dig);
    box_digits<NU>(uint32_t(kThreads) * V, d.oext, step);
#pragma unroll
    for (int i = 0; i < NU; ++i) {
        ext[i] = d.oext[i].d;
        sms[i] = d.osm[i];
    }
    for (uint32_t y = y0; y < cells; y += uint32_t(kThreads) * V) {
        uint32_t sm = 0, kd = 0;
        int64_t off = 0;
#pragma unroll
        for (int i = 0; i < NU; ++i) {
            sm += dig[i] * sms[i];
            off += int64_t(dig[i]) * d.oout[i];
            if (i == d.kout) kd = dig[i];
        }
        if (kd < keff) {
            union {
                typename Word<VO>::T v;
                typename Word<E>::T e[V];
            } u;
            uint32_t dd[NU];
#pragma unroll
            for (int i = 0; i < NU; ++i) dd[i] = dig[i];
#pragma unroll
            for (int k = 0; k < V; ++k) {
                u.e[k] = lds<E>(smem + sm);
                if (k + 1 < V) {
#pragma unroll
                    for (int i = 0; i < NU; ++i) {
                        sm += sms[i];
                        if (++dd[i] < ext[i]) break;
                        sm -= ext[i] * sms[i];
                        dd[i] = 0;
                    }
                }
            }
            stg<VO>(out + off, u.v);
        }
        box_advance<NU>(dig, step, ext);
    }
}

template <int E, int NU>
__device__ __forceinline__ void box_phases(const BoxDesc &d, const char *in, char *out, uint32_t keff,
                                           unsigned char *smem)
{
    // the partial axis' last range: single cells (a wider access could cross its end)
    const uint32_t vin = keff < d.K ? uint32_t(E) : d.vin, vout = keff < d.K ? uint32_t(E) : d.vout;
    switch (vin) {
        case 16: box_load<E, 16, NU>(d, in, keff, smem); break;
        case 8: if constexpr (E <= 8) box_load<E, 8, NU>(d, in, keff, smem); break;
        case 4: if constexpr (E <= 4) box_load<E, 4, NU>(d, in, keff, smem); break;
        case 2: if constexpr (E <= 2) box_load<E, 2, NU>(d, in, keff, smem); break;
        default: if constexpr (E == 1) box_load<E, 1, NU>(d, in, keff, smem); break;
    }
    __syncthreads();
    switch (vout) {
        case 16: box_store<E, 16, NU>(d, out, keff, smem); break;
        case 8: if constexpr (E <= 8) box_store<E, 8, NU>(d, out, keff, smem); break;
        case 4: if constexpr (E <= 4) box_store<E, 4, NU>(d, out, keff, smem); break;
        case 2: if constexpr (E <= 2) box_store<E, 2, NU>(d, out, keff, smem); break;
        default: if constexpr (E == 1) box_store<E, 1, NU>(d, out, keff, smem); break;
    }
    __syncthreads();
}

// Input / output offsets of a unit and its partial-axis extent.  Not inlined:
// inlined into a kernel's unit loop, the descriptor fields it reads would be
// hoisted out of that loop and held in registers across both phases.
struct BoxUnit {
    int64_t in, out;
    uint32_t keff;
};

static __device__ __noinline__ BoxUnit box_unit(const BoxDesc &d, uint32_t q)
{
    BoxUnit b{0, 0, d.K};
#pragma unroll
    for (int i = kMaxBoxOuter - 1; i >= 0; --i) {
        if (i < d.no) {
            uint32_t dig;
            fdivmod(q, d.udiv[i], q, dig);
            b.in += int64_t(dig) * d.uin[i];
            b.out += int64_t(dig) * d.uout[i];
            if (i == d.kunit) b.keff = min(d.K, d.kfull - dig * d.K);
        }
    }
    return b;
}

// One unit of a box permute with NU axes in the box (one kernel per (E, NU):
// the phases' register needs grow with NU).
template <int E, int NU>
__device__ __forceinline__ void box_body(const BoxDesc &d, uint64_t unit, unsigned char *smem)
{
    const BoxUnit b = box_unit(d, uint32_t(unit));
    box_phases<E, NU>(d, d.src + b.in, d.dst + b.out, b.keff, smem);
}

// Fast interlace / de-interlace.  A warp handles 32 consecutive 16-byte groups
// per step, one per lane, reading (interlace) or writing (de-interlace) one
// 16-byte vector per plane per lane -- 512 contiguous bytes per instruction on
// every plane.  The interlaced side of those 32 groups is K * 512 contiguous
// bytes; it goes through a per-warp staging area in shared memory, so that it
// too is moved 512 contiguous bytes per instruction (a lane's own K chunks
// are K * 16 bytes apart from its neighbours', which would touch 32 lines per
// instruction).  Chunk x of lane l sits at stage_pos<K>(l, x): a bijection on
// the K * 32 chunks, skewed so that neither the lane-major nor the
// chunk-major access has a shared-memory bank conflict (K = 6: the
// chunk-major side keeps a few two-way conflicts).
template <int K>
__device__ __forceinline__ int stage_pos(int l, int x)
{
    if constexpr (K > 1 && (K & (K - 1)) == 0) return l * K + (x ^ ((l / (8 / K)) & (K - 1)));
    else if constexpr (K == 6) return l * K + (x + ((l >> 2) & 1)) % K;
    else return l * K + x;
}

template <int E, int K>
__device__ __forceinline__ void interlace_fast_body(const InterlaceDesc &d, char *const *planes, uint64_t unit,
                                                    uint64_t n_units, unsigned char *smem)
{
    const uint64_t groups = d.n * E / 16;
    const uint64_t g0 = unit * d.unit_groups;
    const uint64_t g1 = min(groups, g0 + d.unit_groups);
    const int tid = tid_x(), lane = tid & 31, warp = tid >> 5;
    uint4 *stage = reinterpret_cast<uint4 *>(smem) + warp * K * 32;
    for (uint64_t gw = g0 + uint64_t(warp) * 32; gw < g1; gw += kThreads) {
        const uint64_t g = gw + lane;
        if (g < g1) {
            uint32_t in[K][4], out[K * 4];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const uint4 v = ldg_stream<16>(planes[j] + g * 16);
                in[j][0] = v.x; in[j][1] = v.y; in[j][2] = v.z; in[j][3] = v.w;
            }
            interleave_regs<E, K>(in, out);
#pragma unroll
            for (int x = 0; x < K; ++x)
                stage[stage_pos<K>(lane, x)] = make_uint4(out[4 * x], out[4 * x + 1], out[4 * x + 2], out[4 * x + 3]);
        }
        __syncwarp();
        const uint32_t nq = uint32_t(min(uint64_t(32), g1 - gw)) * K;  // chunks of this warp's groups
        char *o = d.inter + gw * 16 * K;
#pragma unroll
        for (int sidx = 0; sidx < K; ++sidx) {
            const uint32_t q = uint32_t(sidx) * 32 + lane;
            const uint32_t t = q / K, x = q - t * K;
            if (q < nq) stg<16>(o + uint64_t(q) * 16, stage[stage_pos<K>(int(t), int(x))]);
        }
        __syncwarp();
    }
    // Every warp is done with its staging before the CTA's next body (in the
    // batched kernel another op's body) writes shared memory.
    __syncthreads();
    if (unit == n_units - 1 && groups * 16 / E < d.n) interlace_tail<E>(d, planes, groups * 16 / E, true);
}

template <int E, int K>
__device__ __forceinline__ void deinterlace_fast_body(const InterlaceDesc &d, char *const *planes, uint64_t unit,
                                                      uint64_t n_units, unsigned char *smem)
{
    const uint64_t groups = d.n * E / 16;
    const uint64_t g0 = unit * d.unit_groups;
    const uint64_t g1 = min(groups, g0 + d.unit_groups);
    const int tid = tid_x(), lane = tid & 31, warp = tid >> 5;
    uint4 *stage = reinterpret_cast<uint4 *>(smem) + warp * K * 32;
    for (uint64_t gw = g0 + uint64_t(warp) * 32; gw < g1; gw += kThreads) {
        const uint32_t nq = uint32_t(min(uint64_t(32), g1 - gw)) * K;
        const char *src = d.inter + gw * 16 * K;
        uint4 v[K];
#pragma unroll
        for (int sidx = 0; sidx < K; ++sidx) {
            const uint32_t q = uint32_t(sidx) * 32 + lane;
            if (q < nq) v[sidx] = ldg_stream<16>(src + uint64_t(q) * 16);
        }
#pragma unroll
        for (int sidx = 0; sidx < K; ++sidx) {
            const uint32_t q = uint32_t(sidx) * 32 + lane;
            const uint32_t t = q / K, x = q - t * K;
            if (q < nq) stage[stage_pos<K>(int(t), int(x))] = v[sidx];
        }
        __syncwarp();
        const uint64_t g = gw + lane;
        if (g < g1) {
            uint32_t in[K * 4], out[K][4];
#pragma unroll
            for (int x = 0; x < K; ++x) {
                const uint4 w = stage[stage_pos<K>(lane, x)];
                in[4 * x] = w.x; in[4 * x + 1] = w.y; in[4 * x + 2] = w.z; in[4 * x + 3] = w.w;
            }
            deinterleave_regs<E, K>(in, out);
#pragma unroll
            for (int j = 0; j < K; ++j)
                stg<16>(planes[j] + g * 16, make_uint4(out[j][0], out[j][1], out[j][2], out[j][3]));
        }
        __syncwarp();
    }
    __syncthreads();  // staging free for the CTA's next body
    if (unit == n_units - 1 && groups * 16 / E < d.n) interlace_tail<E>(d, planes, groups * 16 / E, false);
}

// Generic interlace / de-interlace: any k, any element size (c words of W
// bytes).  A unit covers unit_groups records; within it the interlaced words
// are walked in order (coalesced on the interlaced side).
template <int W>
__device__ __forceinline__ void interlace_generic_body(const InterlaceDesc &d, char *const *planes, uint64_t unit,
                                                       bool inter)
{
    const uint64_t r0 = unit * d.unit_groups;
    const uint64_t r1 = min(d.n, r0 + d.unit_groups);
    if (r0 >= r1) return;
    const uint32_t kc = d.kc_div.d, c = d.c;
    const uint32_t total = uint32_t(r1 - r0) * kc;
    char *ibase = d.inter + r0 * kc * W;
    constexpr int U = 4;
    for (uint32_t base = 0; base < total; base += kThreads * U) {
        typename Word<W>::T v[U];
        char *dstp[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t f = base + k * kThreads + tid_x();
            dstp[k] = nullptr;
            if (f < total) {
                uint32_t i, rem, j, w;
                fdivmod(f, d.kc_div, i, rem);
                fdivmod(rem, d.c_div, j, w);
                char *pl = planes[j] + ((r0 + i) * c + w) * W;
                char *iv = ibase + uint64_t(f) * W;
                if (inter) { v[k] = ldg_stream<W>(pl); dstp[k] = iv; }
                else { v[k] = ldg_stream<W>(iv); dstp[k] = pl; }
            }
        }
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (dstp[k]) stg<W>(dstp[k], v[k]);
    }
}

}  // namespace rearr
