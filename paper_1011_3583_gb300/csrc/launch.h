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

}  // namespace rearr
