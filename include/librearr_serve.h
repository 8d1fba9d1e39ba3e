/*
 * librearr_serve.h -- serving form of librearr: a request loop that admits
 * rearrangement requests against a device-memory budget, keeps their buffers
 * resident in one device slab, groups the requests that are ready into
 * batched launches of the persistent kernel (continuous batching over several
 * streams) and reports per-request latency.  The paper (arXiv:1011.3583) has
 * no serving layer; every op a request runs is one of librearr.h's.
 *
 * Conventions are those of librearr.h.  Times are seconds on the host's
 * steady clock; timeouts are microseconds (negative: wait forever).
 */
#ifndef LIBREARR_SERVE_H
#define LIBREARR_SERVE_H

#include <stddef.h>
#include <stdint.h>

#include "librearr.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------------------
 * Arena: first-fit allocator with coalescing over a caller-given address range
 * [base, base + bytes).  It touches no memory and makes no CUDA call (the
 * server places it over its device slab), so it can run anywhere.
 *   rearr_arena_alloc : 256-byte aligned block, REARR_ENOMEM if no free block
 *                       is large enough (the arena state is unchanged).
 *   rearr_arena_free  : returns a block; REARR_EINVAL for an unknown address.
 * ------------------------------------------------------------------------- */
typedef struct rearr_arena rearr_arena;

rearr_status rearr_arena_create(uintptr_t base, size_t bytes, rearr_arena **arena);
rearr_status rearr_arena_alloc(rearr_arena *arena, size_t bytes, uintptr_t *addr);
rearr_status rearr_arena_free(rearr_arena *arena, uintptr_t addr);
rearr_status rearr_arena_stats(const rearr_arena *arena, size_t *used, size_t *free_bytes,
                               size_t *largest_free, size_t *n_blocks);
void rearr_arena_destroy(rearr_arena *arena);

/* ---------------------------------------------------------------------------
 * Request specification.
 * Buffers of a request, in order:
 *   PERMUTE     : in[0] src (N*e)                      out[0] dst (N*e)
 *   REORDER     : in[0] src (n*e), in[1] idx (n*4)      out[0] dst (n*e)
 *   INTERLACE   : in[0..k) planes (n*e each)            out[0] interlaced (n*k*e)
 *   DEINTERLACE : in[0] interlaced (n*k*e)              out[0..k) planes (n*e each)
 * ------------------------------------------------------------------------- */
typedef enum {
    REARR_OP_PERMUTE = 0,
    REARR_OP_REORDER = 1,
    REARR_OP_INTERLACE = 2,
    REARR_OP_DEINTERLACE = 3
} rearr_op_kind;

typedef struct {
    int kind;             /* rearr_op_kind                                  */
    int rank;             /* PERMUTE: 1..8                                  */
    int k;                /* INTERLACE / DEINTERLACE: planes, 1..256        */
    int reserved;
    size_t elem_bytes;
    size_t n;             /* REORDER / (DE)INTERLACE: elements per plane    */
    int64_t dims[8];      /* PERMUTE                                        */
    int perm[8];          /* PERMUTE                                        */
} rearr_op_spec;

/* ---------------------------------------------------------------------------
 * Server.
 * In batching mode, requests moving at least large_bytes (read + write) run as
 * their own single-op launch, and so does a request that is alone in the
 * ready queue; those go out in arrival order on one stream of their own (at
 * light load the server then behaves as the plain path), the others are
 * grouped into batches on the stream slots.
 *   budget_bytes     : size of the device slab holding every request buffer
 *                      (one cudaMalloc at create).
 *   n_streams        : batches in flight at once (1..8); each has its stream
 *                      and its own device work-list buffer.
 *   max_batch_ops    : most requests grouped into one launch (1..4096).
 *   batching         : 1: group ready requests into one persistent-kernel
 *                      launch per stream slot (continuous batching);
 *                      0: the plain per-call path, one single-op launch per
 *                      request, in arrival order.
 *   poll_interval_us : completion polling period of the server thread.
 * ------------------------------------------------------------------------- */
typedef struct {
    size_t budget_bytes;
    int n_streams;
    int max_batch_ops;
    int batching;
    int poll_interval_us;
    size_t large_bytes;     /* 0: default 64 MiB */
} rearr_server_config;

typedef struct rearr_server rearr_server;

rearr_status rearr_server_create(const rearr_server_config *config, rearr_server **server);

/* Admission: reserve the request's buffers in the slab.  Requests are admitted
 * in FIFO order as memory frees up; the call waits up to timeout_us for its
 * turn and its memory (REARR_ETIMEDOUT, nothing reserved), and fails at once
 * with REARR_ENOMEM if the request alone exceeds the budget.  The arrival time
 * of the request is the time of this call. */
rearr_status rearr_server_reserve(rearr_server *server, const rearr_op_spec *spec, int64_t timeout_us,
                                  uint64_t *ticket);

/* Device addresses of a reserved request's input and output buffers (the
 * caller fills the inputs before submitting).  ins / outs may be NULL. */
rearr_status rearr_server_buffers(rearr_server *server, uint64_t ticket, void **ins, int *n_in,
                                  void **outs, int *n_out);

/* Queue a reserved request for execution. */
rearr_status rearr_server_submit(rearr_server *server, uint64_t ticket);

/* Queue a reserved request whose inputs are first copied, on the server's own
 * stream and in order before its kernel, from device sources: input j is
 * filled from srcs[j] (NULL: left as the caller wrote it), j < n_srcs.  The
 * sources must stay valid until the request completes. */
rearr_status rearr_server_submit_from(rearr_server *server, uint64_t ticket, const void *const *srcs, int n_srcs);

/* Completion: poll, or wait up to timeout_us (REARR_ETIMEDOUT when it runs
 * out; the request stays in flight and can be waited for again). */
rearr_status rearr_server_poll(rearr_server *server, uint64_t ticket, int *done);
rearr_status rearr_server_wait(rearr_server *server, uint64_t ticket, int64_t timeout_us);

/* Seconds from arrival (reserve) to the detection of completion. */
rearr_status rearr_server_latency(rearr_server *server, uint64_t ticket, double *seconds);

/* Free a completed request's buffers (admits waiting requests).  Releasing a
 * request that is not complete returns REARR_EBUSY. */
rearr_status rearr_server_release(rearr_server *server, uint64_t ticket);

typedef struct {
    uint64_t admitted, completed, released, launches;
    size_t slab_bytes, slab_used, slab_peak;
    double busy_seconds;      /* wall time with at least one launch in flight */
} rearr_server_stats;

rearr_status rearr_server_stats_get(rearr_server *server, rearr_server_stats *stats);

/* Host-side fault injection for tests: completions are hidden from the
 * server thread until delay_us after their launch (no GPU involvement). */
rearr_status rearr_server_inject_completion_delay(rearr_server *server, int64_t delay_us);

/* Stops the server thread after all submitted work is complete (waiting at
 * most timeout_us; REARR_ETIMEDOUT leaves the server running) and frees it. */
rearr_status rearr_server_destroy(rearr_server *server, int64_t timeout_us);

/* ---------------------------------------------------------------------------
 * Trace driver: replays an arrival trace against a server from native
 * threads.  Request i arrives at arrival_s[i] seconds after the call starts:
 * it is reserved (waiting for admission) and submitted; inputs with a
 * template pointer templates[i*4 + j] (device, NULL: left as is; templates
 * may be NULL) are filled from it on the server's stream before the request's
 * kernel (rearr_server_submit_from).  A second thread waits for completions
 * in order, records latency_s[i] from the scheduled arrival time and releases
 * the request.  Returns when every request has completed (or REARR_ETIMEDOUT
 * after timeout_us), with the wall time from the first arrival to the last
 * completion in *wall_s.
 * ------------------------------------------------------------------------- */
rearr_status rearr_server_run_trace(rearr_server *server, const rearr_op_spec *specs, const double *arrival_s,
                                    const void *const *templates, size_t n, double *latency_s, double *wall_s,
                                    int64_t timeout_us);

#ifdef __cplusplus
}
#endif

#endif /* LIBREARR_SERVE_H */
