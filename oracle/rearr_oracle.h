/*
 * rearr_oracle.h -- declarations of the CPU oracle (test infrastructure only).
 *
 * This header belongs to the oracle alone; the CUDA library does not include it.
 * See rearr_oracle.c for the conventions (row-major storage, numpy-style perm,
 * gather reorder, element-granular interlace) and the paper passages each
 * function follows.
 */
#ifndef REARR_ORACLE_H
#define REARR_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#define ORACLE_MAX_RANK 8

#ifdef __cplusplus
extern "C" {
#endif

/* N-D permute (Sec. III.B "3D Permute Kernel" / "Reorder Kernel"):
 * out[lin(j)] = in[sum_i j_i * s[perm[i]]], s the row-major input strides. */
int oracle_permute(void *dst, const void *src, size_t elem_bytes, int rank,
                   const int64_t *dims, const int *perm);

/* The same definition evaluated only at the output linear indices out_lin[0..count):
 * vals[t] = out[out_lin[t]].  Used to check full-size results at sampled points. */
int oracle_permute_sample(void *vals, const void *src, size_t elem_bytes,
                          int rank, const int64_t *dims, const int *perm,
                          const int64_t *out_lin, int64_t count);

/* N-to-M reorder (Sec. III.B): the output has rank_out <= rank_in axes; output
 * axis i is input axis order[i] and spans [base[a], base[a] + range[a]) of it
 * (a = order[i]); every input axis not in order sits at index base[a]:
 *   out[j] = in[x],  x[a] = base[a] + (j_i if a == order[i] else 0). */
int oracle_reorder_nm(void *dst, const void *src, size_t elem_bytes,
                      int rank_in, const int64_t *dims, int rank_out,
                      const int *order, const int64_t *base,
                      const int64_t *range);

/* Reorder by an index sequence (Sec. III.A indexed access): dst[i] = src[idx[i]],
 * src holding n elements; an index >= n is rejected with -1. */
int oracle_reorder(void *dst, const void *src, const uint32_t *idx, size_t n,
                   size_t elem_bytes);

/* The reorder definition evaluated only at the output positions pos[0..count):
 * vals[t] = src[idx[pos[t]]], with src and idx of n entries each. */
int oracle_reorder_sample(void *vals, const void *src, const uint32_t *idx,
                          size_t n, size_t elem_bytes, const int64_t *pos,
                          int64_t count);

/* Reorder by an index sequence with 4- or 8-byte indices, as a gather
 * (scatter == 0: dst[i] = src[idx[i]]) or a scatter (scatter != 0:
 * dst[idx[i]] = src[i], a repeated index keeping the last write); src, dst and
 * idx hold n entries and every index must be < n. */
int oracle_indexed(void *dst, const void *src, const void *idx, int idx_bytes,
                   int scatter, size_t n, size_t elem_bytes);

/* Interlace (Sec. III.C): dst[i*k + j] = srcs[j][i], i < n, j < k. */
int oracle_interlace(void *dst, const void *const *srcs, int k, size_t n,
                     size_t elem_bytes);

/* De-interlace (Sec. III.C): dsts[j][i] = src[i*k + j], i < n, j < k. */
int oracle_deinterlace(void *const *dsts, const void *src, int k, size_t n,
                       size_t elem_bytes);

/* 2-D stencil (Sec. III.D): out[y][x] = sum_k w[k] * in[y + dy[k]][x + dx[k]]
 * in double, taps in order; boundary 0 reads zeros outside the grid, 1 the
 * nearest grid point. */
int oracle_stencil2d(double *dst, const float *src, int64_t ny, int64_t nx,
                     int ntaps, const int *dy, const int *dx, const double *w,
                     int boundary);

#ifdef __cplusplus
}
#endif

#endif
