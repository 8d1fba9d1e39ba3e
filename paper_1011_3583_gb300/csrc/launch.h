// launch.h -- kernel launchers of librearr (host side).
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "rearr_internal.h"

namespace rearr {

// Kernels launched by this library so far (graph replays add their kernels).
extern std::atomic<uint64_t> g_launches;

// Launch the one-op kernel of `op` on stream s.  planes_all holds the k plane
// pointers of an interlace / de-interlace (ignored otherwise).
cudaError_t launch_single(const OpDesc &op, char *const *planes_all, cudaStream_t s);

// The L2-resident bucketed reorder (k_reorder_l2.cu) of a gather op with l2 set.
cudaError_t launch_reorder_l2(const OpDesc &op, cudaStream_t s);

// Number of the n indices (idx_bytes 4 or 8) that are >= bound, counted on the
// device; waits for the count on stream s (k_check.cu).
cudaError_t count_bad_indices(const void *idx, size_t n, int idx_bytes, uint64_t bound, uint64_t *n_bad,
                              cudaStream_t s);

}  // namespace rearr
