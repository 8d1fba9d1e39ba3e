/*
 * librearr_dist.h -- the N-D permute of librearr.h (arXiv:1011.3583 Sec. III.B)
 * over an array sharded across nranks processes, one GPU each: a local pack
 * permute, an all-to-all exchange of equal pieces, and a local unpack
 * permute.  The paper's kernels run on one device and are meant to be built
 * into larger applications (Sec. IV); a distributed transpose (the data
 * exchange step of distributed FFTs and PDE solvers) is that use on several
 * GPUs.  The library plans the two local permutes and runs them; the exchange
 * is the caller's collective (an all-to-all with nranks equal splits of
 * piece_bytes, e.g. ncclAllToAll or torch.distributed.all_to_all_single).
 *
 * Layout.  The global array has `rank` axes, dims[0] the slowest (row-major,
 * as in librearr.h); the output is dims permuted by perm (output axis i is
 * input axis perm[i]).  Input and output are each sharded along their slowest
 * axis in equal contiguous slabs: rank r holds input rows
 * [r * dims[0] / nranks, (r + 1) * dims[0] / nranks) of axis 0, and output
 * rows [r * dims[perm[0]] / nranks, ...) of output axis 0, each slab dense
 * row-major.  Both extents must be multiples of nranks (REARR_EINVAL
 * otherwise).
 *
 * Steps on every rank (same plan everywhere):
 *   exchange == 0 (perm[0] == 0: the sharded axis stays slowest):
 *     rearr_dist_permute_pack(out_slab, in_slab, ...) is the whole operation.
 *   exchange == 1:
 *     rearr_dist_permute_pack(send, in_slab, ...)      send: nranks pieces,
 *                                                      piece j for rank j
 *     all-to-all(recv <- send), piece_bytes per peer   recv: piece j from rank j
 *     rearr_dist_permute_unpack(out_slab, recv, ...)
 * Buffers are device memory of slab_bytes each (send, recv, slabs); none may
 * overlap another.  Pack and unpack are one rearr_permute each (pack: the
 * input slab with axis perm[0] split into (destination rank, rows), rank + 1
 * axes; unpack: the received pieces with the source rank moved next to the
 * output axis that carries input axis 0), enqueued on `stream` with the
 * alignment rules and errors of rearr_permute.
 */
#ifndef LIBREARR_DIST_H
#define LIBREARR_DIST_H

#include <stddef.h>
#include <stdint.h>

#include "librearr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rearr_dist_plan {
    int nranks;
    int exchange;          /* 1: pack, all-to-all, unpack; 0: pack alone */
    uint64_t slab_bytes;   /* bytes of each rank's input slab (= its output slab) */
    uint64_t piece_bytes;  /* bytes sent to and received from each rank (exchange == 1) */
    int pack_rank;         /* the pack permute: rank, input dims, perm */
    int64_t pack_dims[REARR_MAX_RANK];
    int pack_perm[REARR_MAX_RANK];
    int unpack_rank;       /* the unpack permute (exchange == 1; else 0) */
    int64_t unpack_dims[REARR_MAX_RANK];
    int unpack_perm[REARR_MAX_RANK];
} rearr_dist_plan;

/* Host only.  rank 1..REARR_MAX_RANK - 1, dims >= 1, perm a permutation of
 * 0..rank-1, nranks >= 1, elem_bytes >= 1 (REARR_EINVAL otherwise). */
rearr_status rearr_dist_permute_plan(size_t elem_bytes, int rank, const int64_t *dims, const int *perm,
                                     int nranks, rearr_dist_plan *plan);

/* send (or out_slab when plan->exchange == 0) <- in_slab. */
rearr_status rearr_dist_permute_pack(void *send, const void *in_slab, const rearr_dist_plan *plan,
                                     size_t elem_bytes, rearr_stream_t stream);

/* out_slab <- recv (plan->exchange == 1; REARR_EINVAL otherwise). */
rearr_status rearr_dist_permute_unpack(void *out_slab, const void *recv, const rearr_dist_plan *plan,
                                       size_t elem_bytes, rearr_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* LIBREARR_DIST_H */
