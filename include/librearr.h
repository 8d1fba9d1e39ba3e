/*
 * librearr.h -- C ABI of librearr, GB300 (sm_103a) kernels for the data
 * rearrangement operations of "Fast GPGPU Data Rearrangement Kernels using
 * CUDA" (Bader, Bungartz, Mudigere, Narasimhan, Narayanan; arXiv:1011.3583).
 *
 * Common conventions
 * ------------------
 *  - Every data pointer (dst, src, idx, plane pointers) is a DEVICE pointer to
 *    memory of the current CUDA device, owned by the caller.  Arrays of plane
 *    pointers (srcs, dsts) and the dims / perm arrays are HOST arrays, read
 *    during the call only.
 *  - Elements are opaque: elem_bytes bytes are moved bit for bit, never
 *    interpreted as numbers (NaN payloads and -0 survive).
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *    default stream).  A call returns once its kernel is launched; completion
 *    is observed with the usual stream / event synchronisation.
 *  - Errors that can be detected on the host are returned synchronously and
 *    launch nothing: invalid rank, dims, perm, k or elem_bytes, NULL pointers
 *    with a nonzero size, destination overlapping a source (REARR_EINVAL).
 *    A failed launch returns REARR_ECUDA.  Operations of zero elements return
 *    REARR_OK and launch nothing.  In-place operation is not supported.
 *  - rearr_last_error() gives a human-readable message for the most recent
 *    failure on the calling thread.
 */
#ifndef LIBREARR_H
#define LIBREARR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The stream type: identical to cudaStream_t (struct CUstream_st *), declared
 * here so that this header needs no CUDA header. */
typedef struct CUstream_st *rearr_stream_t;

typedef enum {
    REARR_OK = 0,
    REARR_EINVAL = 1,     /* invalid argument                                  */
    REARR_ENOMEM = 2,     /* device or host allocation failed / over budget    */
    REARR_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed       */
    REARR_ERANGE = 4,     /* an index was out of range (checked reorder)       */
    REARR_ETIMEDOUT = 5,  /* a wait ran past its deadline                      */
    REARR_EBUSY = 6       /* the object is in use (e.g. plan already final)    */
} rearr_status;

#define REARR_MAX_RANK 8
#define REARR_MAX_K 256

/* Name of a status code ("REARR_OK", ...).  Never NULL. */
const char *rearr_status_str(rearr_status status);

/* Message describing the last failure on the calling thread ("" if none). */
const char *rearr_last_error(void);

/* ---------------------------------------------------------------------------
 * rearr_permute -- N-D axis permute (arXiv:1011.3583 Sec. III.B, "3D Permute
 * Kernel" and the generic N-to-N "Reorder Kernel"; Tables 1 and 2).
 *
 *   src   : rank-dimensional array, row-major (dims[0] slowest), contiguous.
 *   dst   : the permuted array, row-major over output extents dims[perm[i]].
 *   Output axis i is input axis perm[i] (numpy transpose semantics):
 *       dst[lin(j)] = src[sum_i j_i * s[perm[i]]],  s = row-major strides of src.
 *   The paper's order vector o (fastest dimension first) corresponds to
 *   perm[i] = rank-1-o[rank-1-i].
 *   elem_bytes : any value >= 1.
 *   rank       : 1..8; dims[i] >= 0; perm a permutation of 0..rank-1.
 *   Every collapsed axis of a transposing permute must be < 2^31 elements.
 * ------------------------------------------------------------------------- */
rearr_status rearr_permute(void *dst, const void *src, size_t elem_bytes, int rank,
                           const int64_t *dims, const int *perm, rearr_stream_t stream);

/* ---------------------------------------------------------------------------
 * rearr_reorder_nm -- N-to-M reorder (arXiv:1011.3583 Sec. III.B: "N-to-M"
 * reorder with a base index and a range per dimension): a sub-box of the
 * input, with some axes dropped, in a chosen axis order.
 *
 *   src      : rank_in-dimensional row-major array of extents dims.
 *   order    : rank_out distinct input axes; output axis i is input axis
 *              order[i] (1 <= rank_out <= rank_in).
 *   base     : per input axis, the start index (dropped axes sit there).
 *   range    : per input axis, the extent taken from base (kept axes only;
 *              base + range <= dims); ignored for dropped axes.
 *   dst      : row-major over extents range[order[i]]:
 *       dst[j] = src[x],  x[a] = base[a] + (j_i if a == order[i] else 0).
 *   With rank_out == rank_in, base 0 and range dims it is rearr_permute; a
 *   rank-1 box is the access of a specified range of Sec. III.A.  When the box
 *   keeps no input-contiguous axis, reads cannot be coalesced (the paper notes
 *   the same) and the op runs as a gather of short runs.
 * ------------------------------------------------------------------------- */
rearr_status rearr_reorder_nm(void *dst, const void *src, size_t elem_bytes, int rank_in,
                              const int64_t *dims, int rank_out, const int *order,
                              const int64_t *base, const int64_t *range, rearr_stream_t stream);

/* ---------------------------------------------------------------------------
 * rearr_reorder -- reorder by an index sequence, the "accessing specified set
 * of indices" pattern of arXiv:1011.3583 Sec. III.A:
 *       dst[i] = src[idx[i]],  0 <= i < n.
 *   src holds n elements of elem_bytes; idx holds n uint32 indices, each < n
 *   (repeats allowed).  An index >= n is undefined behaviour (the call would
 *   read outside src).
 *   When src is 128 MiB or more and elem_bytes is 4, 8 or 16, the call first
 *   samples the locality of idx on the device; random indices then go through
 *   L2-resident bucketed passes (partition by source and destination chunk,
 *   gather, scatter) with (8 + elem_bytes) * n bytes of scratch from a
 *   stream-ordered memory pool the library owns (kept for later calls), and
 *   local indices through the direct gather.  Results are identical.
 * ------------------------------------------------------------------------- */
rearr_status rearr_reorder(void *dst, const void *src, const uint32_t *idx, size_t n,
                           size_t elem_bytes, rearr_stream_t stream);

/* ---------------------------------------------------------------------------
 * Other index-sequence forms (the scatter direction and 64-bit indices of the
 * reorder; Sec. III.A reads the elements at a given set of indices):
 *   rearr_scatter   : dst[idx[i]] = src[i], uint32 indices.
 *   rearr_reorder64 : dst[i] = src[idx[i]], uint64 indices (n may exceed 2^32).
 *   rearr_scatter64 : dst[idx[i]] = src[i], uint64 indices.
 *   src, dst and idx hold n entries; every index must be < n (an index >= n
 *   is undefined behaviour).  For a scatter whose indices repeat, a
 *   destination element receives one of the colliding source elements, which
 *   one is unspecified; with a permutation the result is unique.  idx must be
 *   aligned to its index size.  Large gathers and scatters with 4/8/16-byte
 *   elements (either index size, n < 2^32) use the L2-resident passes of
 *   rearr_reorder (a scatter's buckets by destination chunk), with the same
 *   locality check and scratch pool.
 * ------------------------------------------------------------------------- */
rearr_status rearr_scatter(void *dst, const void *src, const uint32_t *idx, size_t n,
                           size_t elem_bytes, rearr_stream_t stream);
rearr_status rearr_reorder64(void *dst, const void *src, const uint64_t *idx, size_t n,
                             size_t elem_bytes, rearr_stream_t stream);
rearr_status rearr_scatter64(void *dst, const void *src, const uint64_t *idx, size_t n,
                             size_t elem_bytes, rearr_stream_t stream);

/* ---------------------------------------------------------------------------
 * Checked index sequences.  The reorders above leave an out-of-range index
 * undefined (the fast path does not test it).  The checked forms test every
 * index on the device first:
 *   rearr_check_indices   : *n_bad = number of the n entries of idx (idx_bytes
 *                           4 or 8, aligned to it) that are >= bound.  Waits for
 *                           its kernel on `stream` (synchronous).
 *   rearr_reorder_checked : rearr_reorder after that check; REARR_ERANGE, with
 *                           dst untouched and nothing launched after the check,
 *                           if any idx[i] >= n.  Waits for the check only; the
 *                           reorder itself is asynchronous as usual.
 * ------------------------------------------------------------------------- */
rearr_status rearr_check_indices(const void *idx, size_t n, int idx_bytes, uint64_t bound, uint64_t *n_bad,
                                 rearr_stream_t stream);
rearr_status rearr_reorder_checked(void *dst, const void *src, const uint32_t *idx, size_t n,
                                   size_t elem_bytes, rearr_stream_t stream);

/* ---------------------------------------------------------------------------
 * rearr_reorder_describe: host-only view of how an index-sequence op runs
 * (scatter 0: rearr_reorder / rearr_reorder64, 1: rearr_scatter /
 * rearr_scatter64; idx_bytes 4 or 8; the addresses only steer the alignment
 * decisions, 0 standing for a 256-byte-aligned buffer).  Validation as the
 * op itself.  A form other than REARR_REORDER_DIRECT means the op is eligible
 * for the L2-resident bucketed passes.  At run time the device still takes
 * the direct path when its locality sample finds the indices local.  Then:
 *   bucket_chunks, bucket_chunk_elems : chunks of the bucketed side (the
 *                                       source of a gather, the destination
 *                                       of a scatter), ~16 MB each;
 *   dest_chunks, dest_chunk_elems     : the gather's destination chunks (64 KB
 *                                       for the shared-memory scatter);
 *                                       1 and 0 for a scatter;
 *   scratch_bytes                     : scratch the call takes from the
 *                                       library's pool while it runs.
 * ------------------------------------------------------------------------- */
typedef enum {
    REARR_REORDER_DIRECT = 0,          /* one direct gather / scatter kernel         */
    REARR_REORDER_SMEM_SCATTER = 1,    /* gather, tile-local passes: partition in
                                          place, gather per source chunk, scatter
                                          through shared memory per 64 KB chunk  */
    REARR_REORDER_L2_SCATTER = 2,      /* gather, last pass through ~16 MB L2 chunks */
    REARR_REORDER_LINEAR_SCATTER = 3   /* scatter: (destination, element) pairs      */
} rearr_reorder_form;

typedef struct {
    int form;                     /* rearr_reorder_form               */
    int word_bytes;               /* access word (element size here) */
    uint32_t bucket_chunks, dest_chunks;
    uint64_t bucket_chunk_elems, dest_chunk_elems;
    uint64_t scratch_bytes;
} rearr_reorder_info;

rearr_status rearr_reorder_describe(size_t n, size_t elem_bytes, int idx_bytes, int scatter, uintptr_t dst_addr,
                                    uintptr_t src_addr, uintptr_t idx_addr, rearr_reorder_info *info);

/* ---------------------------------------------------------------------------
 * rearr_interlace -- join k arrays into one interlaced array
 * (arXiv:1011.3583 Sec. III.C, Table 3):
 *       dst[i*k + j] = srcs[j][i],  0 <= i < n, 0 <= j < k.
 *   srcs : host array of k device pointers, each to n elements.
 *   dst  : n*k elements.  1 <= k <= REARR_MAX_K.
 * ------------------------------------------------------------------------- */
rearr_status rearr_interlace(void *dst, const void *const *srcs, int k, size_t n,
                             size_t elem_bytes, rearr_stream_t stream);

/* ---------------------------------------------------------------------------
 * rearr_deinterlace -- split one interlaced array into k arrays
 * (arXiv:1011.3583 Sec. III.C, Table 3):
 *       dsts[j][i] = src[i*k + j],  0 <= i < n, 0 <= j < k.
 *   dsts : host array of k device pointers, each to room for n elements.
 *   src  : n*k elements.  1 <= k <= REARR_MAX_K.
 * ------------------------------------------------------------------------- */
rearr_status rearr_deinterlace(void *const *dsts, const void *src, int k, size_t n,
                               size_t elem_bytes, rearr_stream_t stream);

/* ---------------------------------------------------------------------------
 * rearr_stencil2d_f32 -- generic 2-D stencil on a float grid (arXiv:1011.3583
 * Sec. III.D, "Generic 2D Stencil Calculation Kernel"; Fig. 2, Table 4):
 *       dst[y][x] = sum_k w[k] * src[y + dy[k]][x + dx[k]],
 *   0 <= y < ny, 0 <= x < nx.
 *   src, dst : ny x nx row-major float32 grids (device, caller-owned); they
 *              must not overlap.
 *   dy, dx, w: ntaps host entries (1 <= ntaps <= REARR_STENCIL_MAX_TAPS),
 *              |dy[k]|, |dx[k]| <= REARR_STENCIL_MAX_RADIUS.  The paper's
 *              functor holding a single-threaded stencil function becomes this
 *              weighted tap list (a C caller cannot pass a template functor).
 *              Offsets may repeat; each tap is one term of the sum.
 *   boundary : REARR_STENCIL_ZERO -- points outside the grid read 0;
 *              REARR_STENCIL_CLAMP -- they read the nearest grid point.
 *   Arithmetic is fp32 fused multiply-add in the kernel's order, so each
 *   result is within (ntaps + 1) * 2^-24 * sum_k |w[k]| |src[y+dy[k]][x+dx[k]]|
 *   of the exact sum (NaN and infinities propagate as in that sum).
 *   The tap set selects the kernel: a full cross of radius r (the order-r
 *   finite-difference Laplacian of the paper's experiments) or a full box of
 *   radius 1 or 2 (smoothing filters), with distinct offsets, run
 *   register-blocked bodies; any other set runs the generic body (one
 *   shared-memory read per tap and point).
 *   Grids whose rows are 16-byte aligned (src and dst 16-byte aligned, nx a
 *   multiple of 4) are staged by TMA tensor copies, others by plain loads;
 *   the results are the same.
 * ------------------------------------------------------------------------- */
#define REARR_STENCIL_MAX_RADIUS 8
#define REARR_STENCIL_MAX_TAPS 64

typedef enum { REARR_STENCIL_ZERO = 0, REARR_STENCIL_CLAMP = 1 } rearr_stencil_boundary;

rearr_status rearr_stencil2d_f32(float *dst, const float *src, int64_t ny, int64_t nx, int ntaps,
                                 const int *dy, const int *dx, const float *w, int boundary,
                                 rearr_stream_t stream);

typedef enum {
    REARR_STENCIL_GENERIC = 0,  /* any tap set                               */
    REARR_STENCIL_CROSS = 1,    /* every offset with dy == 0 or dx == 0, |.| <= r */
    REARR_STENCIL_BOX = 2       /* every offset with |dy|, |dx| <= r (r <= 2)  */
} rearr_stencil_shape;

typedef struct {
    int shape;           /* rearr_stencil_shape of the tap set                */
    int body;            /* kernel body: 1 cross, 2 box; generic lists run 3
                            (one shared read per tap, <= 24 taps) or 0
                            (input columns held in registers)                */
    int radius;          /* largest |dy| or |dx| of the taps                  */
    int n_unique;        /* distinct tap offsets                              */
    int tma;             /* 1: staged by TMA tensor copies; 0: plain loads    */
    int tile_y, tile_x;  /* outputs per CTA                                   */
    int64_t n_tiles;     /* CTAs launched                                     */
    int64_t smem_bytes;  /* shared memory per CTA                             */
} rearr_stencil_info;

/* The kernel choice of rearr_stencil2d_f32 for these arguments (host only;
 * nothing is read or written; dst_addr / src_addr steer the alignment test,
 * 0 meaning 256-byte aligned).  Same validation as the call. */
rearr_status rearr_stencil2d_describe(int64_t ny, int64_t nx, int ntaps, const int *dy, const int *dx,
                                      const float *w, int boundary, uintptr_t dst_addr,
                                      uintptr_t src_addr, rearr_stencil_info *info);

/* Number of bounded device-side waits (a TMA copy's completion barrier) that
 * ran out of time since the library was loaded, on the current device; such
 * a CTA skips its outputs.  0 in normal operation.  Synchronises the device. */
rearr_status rearr_wait_timeouts(uint64_t *count);

/* Fault injection for tests of those waits: the next n_launches TMA-staged
 * stencil launches of this process expect 16 bytes more than their copy
 * delivers, so each CTA's barrier never completes, its bounded waits run out
 * (about 2 s each, twice), it counts a timeout and skips its outputs.  No
 * copy is left in flight and the context stays usable.  n_launches < 0 is
 * REARR_EINVAL; 0 cancels. */
rearr_status rearr_inject_wait_timeout(int n_launches);

/* ---------------------------------------------------------------------------
 * Batched execution.  The paper has no batching; these calls run many of the
 * operations above in one persistent kernel launch driven by a device-side
 * tile work list, captured once in a CUDA graph and replayed.
 *
 *   rearr_plan_create    : new empty plan (host object).
 *   rearr_plan_add_*     : record one operation; same arguments and validation
 *                          as the single calls, minus the stream.  Pointers are
 *                          recorded, not data: the buffers must stay allocated
 *                          and unchanged until the batch's stream work is done.
 *   rearr_plan_finalize  : builds the work list, uploads it (one device
 *                          allocation owned by the plan), picks tile shapes from
 *                          the tuning table and captures the launch in a CUDA
 *                          graph on `stream`.  No op can be added afterwards
 *                          (REARR_EBUSY).
 *   rearr_batch          : replays the captured graph on `stream`; every op of
 *                          the plan is computed exactly as its single call
 *                          would compute it.  Replays on one stream are ordered;
 *                          overlapping replays of ONE plan on different streams
 *                          race on the plan's work counter and are not allowed.
 *   rearr_plan_destroy   : frees the plan (waits for nothing; the caller must
 *                          make sure no replay is still running).
 * ------------------------------------------------------------------------- */
typedef struct rearr_plan rearr_plan;

rearr_status rearr_plan_create(rearr_plan **plan);
rearr_status rearr_plan_add_permute(rearr_plan *plan, void *dst, const void *src,
                                    size_t elem_bytes, int rank, const int64_t *dims,
                                    const int *perm);
rearr_status rearr_plan_add_reorder(rearr_plan *plan, void *dst, const void *src,
                                    const uint32_t *idx, size_t n, size_t elem_bytes);
rearr_status rearr_plan_add_scatter(rearr_plan *plan, void *dst, const void *src,
                                    const uint32_t *idx, size_t n, size_t elem_bytes);
rearr_status rearr_plan_add_reorder_nm(rearr_plan *plan, void *dst, const void *src, size_t elem_bytes,
                                       int rank_in, const int64_t *dims, int rank_out, const int *order,
                                       const int64_t *base, const int64_t *range);
rearr_status rearr_plan_add_interlace(rearr_plan *plan, void *dst, const void *const *srcs,
                                      int k, size_t n, size_t elem_bytes);
rearr_status rearr_plan_add_deinterlace(rearr_plan *plan, void *const *dsts, const void *src,
                                        int k, size_t n, size_t elem_bytes);
rearr_status rearr_plan_finalize(rearr_plan *plan, rearr_stream_t stream);
rearr_status rearr_batch(rearr_plan *plan, rearr_stream_t stream);
void rearr_plan_destroy(rearr_plan *plan);

/* ---------------------------------------------------------------------------
 * rearr_batch_noalloc -- run a plan's ops with the batched kernel without any
 * device allocation.  The paper has no counterpart; this is a service for
 * callers that cannot call cudaMalloc, such as a serving process that has
 * reserved the GPU's memory for its own pool and must not see a library grow
 * device memory, or a latency-critical path that cannot take the device-wide
 * synchronisation cudaMalloc / cudaFree may cause.
 *
 *   plan   : a plan built with rearr_plan_add_* (finalized or not; only its
 *            host-side op list is read).  The caller still owns every input
 *            and output buffer the ops name.  A finalized plan runs in the
 *            work-list order rearr_plan_finalize chose (ops grouped by body);
 *            a plan that was not finalized runs its ops in the order they were
 *            added, with the same results.
 *   stream : the work list is copied and the kernel launched on this stream.
 *
 * The work list goes to a fixed 512 KiB device buffer compiled into the
 * library (about 1280 ops; fewer when interlaces have more than 8 planes);
 * every GPU that loads the library holds that buffer until the process exits.
 * A plan that does not fit returns REARR_EINVAL and launches nothing.  The
 * first call on a device looks up the buffer's address and the kernel's
 * occupancy (cudaGetSymbolAddress and device queries) with that device
 * current; make that first call before any stream capture.  All calls share
 * the buffer and leave their contents in it: calls whose work overlaps on the
 * GPU (several streams or host threads) race on it and must be ordered by the
 * caller, e.g. by issuing them on one stream.  Results are the same as
 * rearr_batch's.  Calls no cudaMalloc, cudaFree or other allocating routine.
 * ------------------------------------------------------------------------- */
rearr_status rearr_batch_noalloc(const rearr_plan *plan, rearr_stream_t stream);

/* Number of ops and of work-list tiles in a plan (after finalize), host only. */
rearr_status rearr_plan_stats(const rearr_plan *plan, int64_t *n_ops, int64_t *n_tiles);

/* ---------------------------------------------------------------------------
 * Introspection of the permute plan compiler (host only; needs no GPU).
 *
 * The plan compiler drops extent-1 axes, merges output axes that are adjacent
 * and in order in the input, folds an unmoved innermost run into a wider
 * element, and classifies the op (the offset and stride computation and the 2-D
 * plane of Sec. III.B: the plane of the input's fastest and the output's
 * fastest dimension).
 * ------------------------------------------------------------------------- */
typedef enum {
    REARR_KIND_NOOP = 0,        /* zero elements                                */
    REARR_KIND_COPY = 1,        /* contiguous copy (identity after collapsing)  */
    REARR_KIND_TILE = 2,        /* shared-memory tiled transpose, 1 word/cell   */
    REARR_KIND_TILE_CELLS = 3,  /* tiled transpose of multi-word cells          */
    REARR_KIND_RUNS = 4,        /* copy of long contiguous runs                 */
    REARR_KIND_STRIDED = 5,     /* element-wise strided copy: a transpose plane
                                   too small to fill tiles (by the tuning
                                   table's thin-plane rule) whose box (below)
                                   would have short runs, or a box with no
                                   input-contiguous axis and one-word cells  */
    REARR_KIND_BOX = 6          /* a thin transpose plane staged as boxes of
                                   several whole axes (Sec. III.B, generic
                                   reorder): runs of tile_a cells read, runs of
                                   tile_b cells written, one-word cells       */
} rearr_kind;

typedef struct {
    int kind;                 /* rearr_kind                                      */
    int rank;                 /* collapsed rank (after folding)                  */
    int64_t dims[8];          /* collapsed output extents, slowest first         */
    int64_t in_strides[8];    /* input stride of each output axis, in cells      */
    int64_t cell_bytes;       /* bytes per cell after folding                    */
    int word_bytes;           /* access word size (power of two, <= 16)          */
    int plane_a;              /* output axis that is input-innermost (-1: none)  */
    int vec_in, vec_out;      /* global access widths in bytes (TILE, BOX)       */
    int tile_a, tile_b;       /* tile extents in cells (TILE, TILE_CELLS); BOX:
                                 cells of an input run and of an output run     */
    int64_t n_tiles;          /* work units (tiles, runs or copy blocks)         */
    int wide_a, wide_b;       /* TILE on a short plane: the output axis whose
                                 planes the tile's A side (input rows) or B side
                                 (output runs) also spans, -1: none; tile_a and
                                 tile_b then count cells of the widened sides  */
} rearr_permute_info;

/* dst_addr / src_addr only steer the alignment decisions (0: 256-byte aligned);
 * nothing is read or written. */
rearr_status rearr_permute_describe(size_t elem_bytes, int rank, const int64_t *dims,
                                    const int *perm, uintptr_t dst_addr, uintptr_t src_addr,
                                    rearr_permute_info *info);

/* The same view of an N-to-M reorder (arguments and validation as
 * rearr_reorder_nm; the box's base offset is added to src_addr). */
rearr_status rearr_reorder_nm_describe(size_t elem_bytes, int rank_in, const int64_t *dims, int rank_out,
                                      const int *order, const int64_t *base, const int64_t *range,
                                      uintptr_t dst_addr, uintptr_t src_addr, rearr_permute_info *info);

/* ---------------------------------------------------------------------------
 * Tuning table.  The paper chooses block and thread shapes per kernel by hand
 * (Sec. III); here the fast tile's staged row length per (element size,
 * plane-extent class), the batched kernel's work grab and the thin-plane
 * thresholds of the strided copy come from a text table written by the
 * project's autotuner.  rearr_tuning_load reads such a
 * table (path NULL or "": built-in defaults) for plans compiled afterwards;
 * REARR_EINVAL if the file cannot be read (the previous table stays).  The
 * REARR_TUNE_TABLE environment variable names a table read on first use.
 * ------------------------------------------------------------------------- */
rearr_status rearr_tuning_load(const char *path);

/* ---------------------------------------------------------------------------
 * Measurement helpers (not rearrangement operations).
 *   rearr_memcpy_d2d   : cudaMemcpyAsync(dst, src, bytes, DeviceToDevice, stream),
 *                        the roofline reference the paper measures against
 *                        (Sec. I, Sec. III.A).
 *   rearr_launch_count : number of kernels this library has launched in this
 *                        process (graph replays count the kernels they run).
 *   rearr_selftest_host: host-only checks of the plan compiler's integer
 *                        helpers, and box plans of pseudo-random permutes run
 *                        on the host against the permute written out;
 *                        returns REARR_OK when they all pass.
 * ------------------------------------------------------------------------- */
rearr_status rearr_memcpy_d2d(void *dst, const void *src, size_t bytes, rearr_stream_t stream);
uint64_t rearr_launch_count(void);
rearr_status rearr_selftest_host(void);

#ifdef __cplusplus
}
#endif

#endif /* LIBREARR_H */
