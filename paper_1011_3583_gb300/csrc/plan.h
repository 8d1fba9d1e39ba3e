// plan.h -- host plan compiler of librearr: validates an operation, reduces
// it to canonical form and fills the work-list descriptor of its kernel.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/librearr.h"
#include "rearr_internal.h"

namespace rearr {

struct PermPlan {
    rearr_permute_info info;  // what rearr_permute_describe reports
    OpDesc op;                // descriptor of the kernel that runs it
};

struct InterlacePlan {
    OpDesc op;
    std::vector<char *> planes;  // all k plane pointers
};

// Each returns REARR_OK or REARR_EINVAL (with a message in err).  A plan with
// op.units == 0 is a no-op.
rearr_status plan_permute(void *dst, const void *src, size_t elem_bytes, int rank,
                          const int64_t *dims, const int *perm, PermPlan &pl, std::string &err);
rearr_status plan_reorder_nm(void *dst, const void *src, size_t elem_bytes, int rank_in, const int64_t *dims,
                             int rank_out, const int *order, const int64_t *base, const int64_t *range,
                             PermPlan &pl, std::string &err);
// Gather dst[i] = src[idx[i]] (or, with scatter, dst[idx[i]] = src[i]) with
// idx_bytes-byte (4 or 8) indices.
rearr_status plan_reorder(void *dst, const void *src, const uint32_t *idx, size_t n,
                          size_t elem_bytes, OpDesc &op, std::string &err, int idx_bytes = 4,
                          bool scatter = false);
rearr_status plan_interlace(bool inter, char *interlaced, char *const *planes, int k, size_t n,
                            size_t elem_bytes, InterlacePlan &pl, std::string &err);

// A fast tile planned with the 32 KB payload re-planned with the 16 KB tile of
// the same row length (the batched kernel holds two 16 KB tiles per CTA).
void tile_to_single_width(OpDesc &op);

// Largest power of two <= 16 dividing every argument.
int pow2_align(uint64_t a, uint64_t b = 0, uint64_t c = 0, uint64_t d = 0);

// Host self-checks of the integer helpers (fast division, alignment).
bool selftest_host(std::string &err);

}  // namespace rearr
