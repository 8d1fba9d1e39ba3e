/*
 * rearr_oracle.c -- plain, single-threaded CPU oracle for the data-rearrangement
 * operations of "Fast GPGPU Data Rearrangement Kernels using CUDA"
 * (Bader, Bungartz, Mudigere, Narasimhan, Narayanan, arXiv:1011.3583).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this code.  The CUDA library shares no
 * code, header, table or helper with it, and nothing in the product path may
 * call it.
 *
 * What it computes is the plain definition of each operation; the method is
 * exact data movement, so no blocking, tiling, axis merging or reordering of
 * work is done here.  Every element is moved with memcpy(elem_bytes) and is
 * never loaded as a number, so any bit pattern (NaN payloads, -0) survives.
 *
 * Conventions (readings of the paper, Sec. III.B):
 *   - Storage is row-major: dims[0] is the slowest axis, dims[rank-1] the
 *     fastest (the paper's default linearisation is row-major).
 *   - perm follows numpy's transpose: output axis i is input axis perm[i].
 *     The paper lists an order vector fastest-dimension-first; a paper order
 *     vector o converts to perm[i] = rank-1-o[rank-1-i].
 *   - Reorder by an index sequence is a gather, dst[i] = src[idx[i]], the
 *     access of a given set of indices of Sec. III.A.
 *   - Interlace joins k arrays of n elements each into one array of k*n
 *     elements, dst[i*k + j] = src_j[i]; de-interlace splits it back
 *     (Sec. III.C).
 *
 * Return value of every entry point: 0 on success, -1 on invalid arguments.
 */
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include "rearr_oracle.h"

/* Validation shared by the permute entry points: rank in [1, 8], dims >= 0,
 * perm a permutation of 0..rank-1, elem_bytes >= 1. */
static int check_permute_args(size_t elem_bytes, int rank, const int64_t *dims,
                              const int *perm)
{
    if (elem_bytes == 0 || rank < 1 || rank > ORACLE_MAX_RANK || !dims || !perm)
        return -1;
    int seen[ORACLE_MAX_RANK] = {0};
    for (int i = 0; i < rank; ++i) {
        if (dims[i] < 0) return -1;
        if (perm[i] < 0 || perm[i] >= rank) return -1;
        if (seen[perm[i]]) return -1;
        seen[perm[i]] = 1;
    }
    return 0;
}

static int64_t element_count(int rank, const int64_t *dims)
{
    int64_t n = 1;
    for (int i = 0; i < rank; ++i) n *= dims[i];
    return n;
}

/* Row-major strides of the input, in elements: s[rank-1] = 1 and
 * s[i] = s[i+1] * dims[i+1]  (the "offset/striding approach", Sec. III.B). */
static void row_major_strides(int rank, const int64_t *dims, int64_t *s)
{
    s[rank - 1] = 1;
    for (int i = rank - 2; i >= 0; --i) s[i] = s[i + 1] * dims[i + 1];
}

/* Input linear offset (elements) of the output element with multi-index j:
 * output axis i is input axis perm[i], so its index advances the input by
 * s[perm[i]] per step. */
static int64_t input_offset(int rank, const int *perm, const int64_t *s,
                            const int64_t *j)
{
    int64_t off = 0;
    for (int i = 0; i < rank; ++i) off += j[i] * s[perm[i]];
    return off;
}

int oracle_permute(void *dst, const void *src, size_t elem_bytes, int rank,
                   const int64_t *dims, const int *perm)
{
    if (check_permute_args(elem_bytes, rank, dims, perm)) return -1;
    int64_t total = element_count(rank, dims);
    if (total == 0) return 0;
    if (!dst || !src) return -1;

    int64_t s[ORACLE_MAX_RANK], od[ORACLE_MAX_RANK], j[ORACLE_MAX_RANK];
    row_major_strides(rank, dims, s);
    for (int i = 0; i < rank; ++i) {
        od[i] = dims[perm[i]];
        j[i] = 0;
    }

    unsigned char *out = (unsigned char *)dst;
    const unsigned char *in = (const unsigned char *)src;
    /* Walk the output in its own row-major order (last index fastest): an
     * odometer over od.  The output is written sequentially. */
    for (int64_t lin = 0; lin < total; ++lin) {
        int64_t off = input_offset(rank, perm, s, j);
        memcpy(out + (size_t)lin * elem_bytes, in + (size_t)off * elem_bytes,
               elem_bytes);
        for (int i = rank - 1; i >= 0; --i) {
            if (++j[i] < od[i]) break;
            j[i] = 0;
        }
    }
    return 0;
}

int oracle_permute_sample(void *vals, const void *src, size_t elem_bytes,
                          int rank, const int64_t *dims, const int *perm,
                          const int64_t *out_lin, int64_t count)
{
    if (check_permute_args(elem_bytes, rank, dims, perm)) return -1;
    if (count < 0) return -1;
    if (count == 0) return 0;
    if (!vals || !src || !out_lin) return -1;
    int64_t total = element_count(rank, dims);

    int64_t s[ORACLE_MAX_RANK], od[ORACLE_MAX_RANK], j[ORACLE_MAX_RANK];
    row_major_strides(rank, dims, s);
    for (int i = 0; i < rank; ++i) od[i] = dims[perm[i]];

    unsigned char *out = (unsigned char *)vals;
    const unsigned char *in = (const unsigned char *)src;
    for (int64_t t = 0; t < count; ++t) {
        int64_t lin = out_lin[t];
        if (lin < 0 || lin >= total) return -1;
        /* Output multi-index of lin, last axis fastest. */
        for (int i = rank - 1; i >= 0; --i) {
            j[i] = lin % od[i];
            lin /= od[i];
        }
        int64_t off = input_offset(rank, perm, s, j);
        memcpy(out + (size_t)t * elem_bytes, in + (size_t)off * elem_bytes,
               elem_bytes);
    }
    return 0;
}

int oracle_reorder_nm(void *dst, const void *src, size_t elem_bytes,
                      int rank_in, const int64_t *dims, int rank_out,
                      const int *order, const int64_t *base,
                      const int64_t *range)
{
    if (elem_bytes == 0 || rank_in < 1 || rank_in > ORACLE_MAX_RANK || !dims ||
        rank_out < 1 || rank_out > rank_in || !order || !base || !range)
        return -1;
    int kept[ORACLE_MAX_RANK] = {0};
    for (int a = 0; a < rank_in; ++a)
        if (dims[a] < 0) return -1;
    for (int i = 0; i < rank_out; ++i) {
        const int a = order[i];
        if (a < 0 || a >= rank_in || kept[a]) return -1;
        kept[a] = 1;
    }
    /* kept axes span [base, base + range); dropped axes sit at base */
    int64_t total = 1;
    for (int a = 0; a < rank_in; ++a) {
        if (base[a] < 0) return -1;
        if (kept[a]) {
            if (range[a] < 0 || base[a] + range[a] > dims[a]) return -1;
            total *= range[a];
        } else if (base[a] >= dims[a]) {
            return -1;
        }
    }
    if (total == 0) return 0;
    if (!dst || !src) return -1;

    int64_t s[ORACLE_MAX_RANK], j[ORACLE_MAX_RANK], x[ORACLE_MAX_RANK];
    row_major_strides(rank_in, dims, s);
    for (int i = 0; i < rank_out; ++i) j[i] = 0;
    unsigned char *out = (unsigned char *)dst;
    const unsigned char *in = (const unsigned char *)src;
    for (int64_t lin = 0; lin < total; ++lin) {
        /* input multi-index of output multi-index j */
        for (int a = 0; a < rank_in; ++a) x[a] = base[a];
        for (int i = 0; i < rank_out; ++i) x[order[i]] += j[i];
        int64_t off = 0;
        for (int a = 0; a < rank_in; ++a) off += x[a] * s[a];
        memcpy(out + (size_t)lin * elem_bytes, in + (size_t)off * elem_bytes,
               elem_bytes);
        for (int i = rank_out - 1; i >= 0; --i) {
            if (++j[i] < range[order[i]]) break;
            j[i] = 0;
        }
    }
    return 0;
}

int oracle_reorder(void *dst, const void *src, const uint32_t *idx, size_t n,
                   size_t elem_bytes)
{
    if (elem_bytes == 0) return -1;
    if (n == 0) return 0;
    if (!dst || !src || !idx) return -1;
    unsigned char *out = (unsigned char *)dst;
    const unsigned char *in = (const unsigned char *)src;
    for (size_t i = 0; i < n; ++i) {
        if ((size_t)idx[i] >= n) return -1;
        memcpy(out + i * elem_bytes, in + (size_t)idx[i] * elem_bytes, elem_bytes);
    }
    return 0;
}

int oracle_reorder_sample(void *vals, const void *src, const uint32_t *idx,
                          size_t n, size_t elem_bytes, const int64_t *pos,
                          int64_t count)
{
    if (elem_bytes == 0 || count < 0) return -1;
    if (count == 0) return 0;
    if (!vals || !src || !idx || !pos) return -1;
    unsigned char *out = (unsigned char *)vals;
    const unsigned char *in = (const unsigned char *)src;
    for (int64_t t = 0; t < count; ++t) {
        if (pos[t] < 0 || (size_t)pos[t] >= n) return -1;
        const uint32_t j = idx[pos[t]];
        if ((size_t)j >= n) return -1;
        memcpy(out + (size_t)t * elem_bytes, in + (size_t)j * elem_bytes, elem_bytes);
    }
    return 0;
}

int oracle_indexed(void *dst, const void *src, const void *idx, int idx_bytes,
                   int scatter, size_t n, size_t elem_bytes)
{
    if (elem_bytes == 0 || (idx_bytes != 4 && idx_bytes != 8)) return -1;
    if (n == 0) return 0;
    if (!dst || !src || !idx) return -1;
    unsigned char *out = (unsigned char *)dst;
    const unsigned char *in = (const unsigned char *)src;
    for (size_t i = 0; i < n; ++i) {
        const uint64_t j = idx_bytes == 4 ? (uint64_t)((const uint32_t *)idx)[i]
                                          : ((const uint64_t *)idx)[i];
        if (j >= (uint64_t)n) return -1;
        if (scatter) /* dst[idx[i]] = src[i]; a repeated index keeps the last write */
            memcpy(out + (size_t)j * elem_bytes, in + i * elem_bytes, elem_bytes);
        else         /* dst[i] = src[idx[i]] */
            memcpy(out + i * elem_bytes, in + (size_t)j * elem_bytes, elem_bytes);
    }
    return 0;
}

int oracle_interlace(void *dst, const void *const *srcs, int k, size_t n,
                     size_t elem_bytes)
{
    if (elem_bytes == 0 || k < 1 || !srcs) return -1;
    if (n == 0) return 0;
    if (!dst) return -1;
    for (int j = 0; j < k; ++j)
        if (!srcs[j]) return -1;
    unsigned char *out = (unsigned char *)dst;
    for (size_t i = 0; i < n; ++i)
        for (int j = 0; j < k; ++j)
            memcpy(out + (i * (size_t)k + (size_t)j) * elem_bytes,
                   (const unsigned char *)srcs[j] + i * elem_bytes, elem_bytes);
    return 0;
}

int oracle_deinterlace(void *const *dsts, const void *src, int k, size_t n,
                       size_t elem_bytes)
{
    if (elem_bytes == 0 || k < 1 || !dsts) return -1;
    if (n == 0) return 0;
    if (!src) return -1;
    for (int j = 0; j < k; ++j)
        if (!dsts[j]) return -1;
    const unsigned char *in = (const unsigned char *)src;
    for (size_t i = 0; i < n; ++i)
        for (int j = 0; j < k; ++j)
            memcpy((unsigned char *)dsts[j] + i * elem_bytes,
                   in + (i * (size_t)k + (size_t)j) * elem_bytes, elem_bytes);
    return 0;
}

/* 2-D stencil (Sec. III.D): out[y][x] = sum_k w[k] * in[y + dy[k]][x + dx[k]],
 * accumulated in double in tap order.  Points outside the grid read 0
 * (boundary 0) or the nearest grid point (boundary 1).  The result is
 * returned in double, one value per grid point. */
int oracle_stencil2d(double *dst, const float *src, int64_t ny, int64_t nx,
                     int ntaps, const int *dy, const int *dx, const double *w,
                     int boundary)
{
    if (ny < 0 || nx < 0 || ntaps < 1 || !dy || !dx || !w) return -1;
    if (boundary != 0 && boundary != 1) return -1;
    if (ny == 0 || nx == 0) return 0;
    if (!dst || !src) return -1;
    for (int64_t y = 0; y < ny; ++y) {
        for (int64_t x = 0; x < nx; ++x) {
            double acc = 0.0;
            for (int k = 0; k < ntaps; ++k) {
                int64_t yy = y + dy[k], xx = x + dx[k];
                double v;
                if (yy >= 0 && yy < ny && xx >= 0 && xx < nx) {
                    v = (double)src[yy * nx + xx];
                } else if (boundary == 0) {
                    v = 0.0;
                } else {
                    yy = yy < 0 ? 0 : (yy >= ny ? ny - 1 : yy);
                    xx = xx < 0 ? 0 : (xx >= nx ? nx - 1 : xx);
                    v = (double)src[yy * nx + xx];
                }
                acc += w[k] * v;
            }
            dst[y * nx + x] = acc;
        }
    }
    return 0;
}
