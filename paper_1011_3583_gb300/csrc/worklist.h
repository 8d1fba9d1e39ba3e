// worklist.h -- building and launching a batched work list from host code
// (used by the serving loop, which keeps one device work-list buffer per
// stream slot).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "rearr_internal.h"

namespace rearr {

struct WorklistLayout {
    size_t off_prefix = 0, off_planes = 0, off_counter = 0, bytes = 0;
};

// Adapts a single-call op descriptor to the batched kernel: gathers get small
// work units (2048 elements), so that the window of units in flight -- the
// resident CTAs times the work grab -- keeps only a few random-read sources
// in the L2 at a time instead of thrashing it.
void batch_form(OpDesc &op);

// Reorders a batch's ops (and their plane lists) for the batched kernel: each
// op class sorted by body variant, the classes merged in proportion to their
// work units.  Ops of a batch are independent, so any order is correct.
void order_for_batch(std::vector<OpDesc> &ops, std::vector<std::vector<char *>> &plane_lists);

// Byte layout of a work list of n_ops descriptors and n_ptrs plane pointers:
// descriptors | prefix sums (n_ops + 1) | plane pointers | work counter.
WorklistLayout worklist_layout(size_t n_ops, size_t n_ptrs);

// Writes the work-list image into img (host memory of layout.bytes bytes) for
// a device copy at dev_base; plane lists of interlaces with k > kInlineK are
// re-pointed into the image.  The counter slot is zeroed.  Returns the total
// number of work units.
uint64_t build_worklist(const OpDesc *ops, const std::vector<char *> *plane_lists, size_t n, unsigned char *img,
                        uintptr_t dev_base, const WorklistLayout &layout);

// Launches the persistent batched kernel over a work list already resident at
// dev_base (on stream s, after its upload on the same stream).
cudaError_t launch_worklist(uintptr_t dev_base, const WorklistLayout &layout, size_t n, uint64_t total_units,
                            cudaStream_t s);

}  // namespace rearr
