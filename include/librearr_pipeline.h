/*
 * librearr_pipeline.h -- host-buffer form of librearr: the operations of
 * librearr.h on inputs and outputs that live in HOST memory.  The paper
 * (arXiv:1011.3583) times its kernels on device-resident data and has no
 * counterpart; this is the end-to-end path a caller holding host arrays uses.
 *
 * A pipeline owns `slots` device staging slots of `slot_bytes` each and three
 * CUDA streams: host-to-device copies, kernels, device-to-host copies.  Each
 * submitted op takes the next slot in turn; its inputs are copied into the
 * slot, its kernel runs there and its outputs are copied back, so with three
 * or more slots the upload of op i+1, the kernel of op i and the download of
 * op i-1 overlap.  A slot is reused only after its previous op's download
 * finished (ordered on the GPU with events; submitting never blocks the host
 * except inside the CUDA runtime for pageable host memory).
 *
 * Direct ops: where the GPU reaches host memory through the host's own page
 * tables (a coherent link such as NVLink-C2C; the pipeline's default there),
 * a permute, interlace or de-interlace whose host buffers are page-locked and
 * whose plan streams through them (copy, tiles, runs, boxes, interlace
 * kernels) runs its kernel on the host buffers directly, with no staging:
 * every byte still crosses the host link once, but reads and writes share it
 * in both directions inside one kernel.  Other ops, and every op on pageable
 * memory, are staged as above.  A direct op starts after everything
 * submitted before it and everything submitted after it waits for it, so the
 * ops act on host memory in submission order whichever way each one runs.
 * rearr_pipeline_set_direct turns direct ops on or off.
 *
 * Conventions are those of librearr.h, except that every data pointer here is
 * a HOST pointer.  Page-locked (pinned) host memory gives full copy speed;
 * pageable memory works but its uploads are staged by the driver.  The caller
 * must not modify an op's inputs or read its outputs until rearr_pipeline_sync
 * returns.  Ops of one pipeline may feed each other through host memory: an
 * op whose input overlaps an earlier op's output reads that output.  Each op's inputs and outputs, each rounded up to 256 bytes, must
 * fit in one slot (REARR_EINVAL otherwise; nothing is enqueued).  A pipeline
 * is used by one host thread at a time.
 */
#ifndef LIBREARR_PIPELINE_H
#define LIBREARR_PIPELINE_H

#include <stddef.h>
#include <stdint.h>

#include "librearr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rearr_pipeline rearr_pipeline;

/* slots: 1..8 (3 or more for full overlap).  Allocates slots * slot_bytes of
 * device memory on the current device (REARR_ENOMEM if that fails). */
rearr_status rearr_pipeline_create(size_t slot_bytes, int slots, rearr_pipeline **pipe);

/* The ops: same arguments, layouts and validation as the librearr.h calls of
 * the same name, with host pointers.  The whole source array of an N-to-M
 * reorder (every element of dims) is uploaded; its output is the box.  A
 * scatter does not upload dst: with a permutation every element is written,
 * otherwise the elements no index names come back undefined.
 * Asynchronous: a call returns once the op's copies and kernel are enqueued.  A CUDA failure is returned by the
 * call that sees it and by every later call (the pipeline is then broken). */
rearr_status rearr_pipeline_permute(rearr_pipeline *pipe, void *dst, const void *src, size_t elem_bytes,
                                    int rank, const int64_t *dims, const int *perm);
rearr_status rearr_pipeline_reorder(rearr_pipeline *pipe, void *dst, const void *src, const uint32_t *idx,
                                    size_t n, size_t elem_bytes);
rearr_status rearr_pipeline_reorder_nm(rearr_pipeline *pipe, void *dst, const void *src, size_t elem_bytes,
                                       int rank_in, const int64_t *dims, int rank_out, const int *order,
                                       const int64_t *base, const int64_t *range);
rearr_status rearr_pipeline_scatter(rearr_pipeline *pipe, void *dst, const void *src, const uint32_t *idx,
                                    size_t n, size_t elem_bytes);
rearr_status rearr_pipeline_reorder64(rearr_pipeline *pipe, void *dst, const void *src, const uint64_t *idx,
                                      size_t n, size_t elem_bytes);
rearr_status rearr_pipeline_scatter64(rearr_pipeline *pipe, void *dst, const void *src, const uint64_t *idx,
                                      size_t n, size_t elem_bytes);
rearr_status rearr_pipeline_interlace(rearr_pipeline *pipe, void *dst, const void *const *srcs, int k,
                                      size_t n, size_t elem_bytes);
rearr_status rearr_pipeline_deinterlace(rearr_pipeline *pipe, void *const *dsts, const void *src, int k,
                                        size_t n, size_t elem_bytes);
rearr_status rearr_pipeline_stencil2d_f32(rearr_pipeline *pipe, float *dst, const float *src, int64_t ny,
                                          int64_t nx, int ntaps, const int *dy, const int *dx, const float *w,
                                          int boundary);

/* Waits until every submitted op's outputs are in host memory. */
rearr_status rearr_pipeline_sync(rearr_pipeline *pipe);

/* mode 1: run eligible ops directly on page-locked host buffers (see above);
 * 0: stage every op.  Applies to ops submitted afterwards. */
rearr_status rearr_pipeline_set_direct(rearr_pipeline *pipe, int mode);

/* Ops that ran directly on host buffers so far, and the current mode. */
rearr_status rearr_pipeline_direct_ops(const rearr_pipeline *pipe, uint64_t *direct_ops, int *mode);

/* Ops submitted and bytes moved host-to-device / device-to-host so far (by
 * copies, or across the host link by the kernels of direct ops). */
rearr_status rearr_pipeline_stats(const rearr_pipeline *pipe, uint64_t *ops, uint64_t *h2d_bytes,
                                  uint64_t *d2h_bytes);

/* Waits for the pipeline's work, then frees its slots, streams and events. */
void rearr_pipeline_destroy(rearr_pipeline *pipe);

#ifdef __cplusplus
}
#endif

#endif /* LIBREARR_PIPELINE_H */
