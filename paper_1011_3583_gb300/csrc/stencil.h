// stencil.h -- the generic 2-D stencil of librearr (Sec. III.D): plan shared
// by the host plan compiler (stencil_plan.cpp) and the kernels (k_stencil.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/librearr.h"

namespace rearr {

constexpr int kStencilMaxRadius = REARR_STENCIL_MAX_RADIUS;
constexpr int kStencilMaxTaps = REARR_STENCIL_MAX_TAPS;
constexpr int kStencilThreads = 256;
constexpr int kStencilTileX = 64;    // output columns per CTA
constexpr int kStencilTileY = 128;   // output rows per CTA
// Staged columns left and right of a tile: 8 floats keep the box's first
// column 16-byte aligned (the TMA start rule) and cover any radius <= 8.
constexpr int kStencilHaloX = 8;
constexpr int kStencilPitch = kStencilTileX + 2 * kStencilHaloX;  // floats per staged row
constexpr int kStencilDense = 2 * kStencilMaxRadius + 1;

// Compute bodies (kernel template argument).  Cross and box equal their
// rearr_stencil_shape values.
constexpr int kBodyGenericColumns = 0;  // generic, input columns held in registers
constexpr int kBodyCross = REARR_STENCIL_CROSS;
constexpr int kBodyBox = REARR_STENCIL_BOX;
constexpr int kBodyGenericTaps = 3;     // generic, one shared read per tap and output
constexpr int kGenericTapsMax = 24;     // longest list for kBodyGenericTaps

// Kernel parameters (passed by value; about 1.6 KB).
struct StencilArgs {
    const float *src;
    float *dst;
    int64_t ny, nx;
    int64_t tiles_x;  // tiles along x
    int r;            // halo rows above and below a tile: largest |dy|, |dx|
    int boundary;     // REARR_STENCIL_ZERO / REARR_STENCIL_CLAMP
    int tma;          // 1: box staged by a TMA tensor copy, 16-byte stores
    uint32_t extra_tx;  // bytes expected beyond the copy (0; > 0 only to inject a timeout)
    int ntaps;        // taps (generic body), grouped by dx in ascending dx,
                      // each group in the caller's order
    int ngroups;      // distinct dx values
    int8_t tdy[kStencilMaxTaps], tdx[kStencilMaxTaps];
    float tw[kStencilMaxTaps];
    int8_t gdx[kStencilDense];   // dx of group g
    uint8_t gend[kStencilDense]; // one past the last tap of group g
    // Dense weights of the cross / box bodies: w[(dy + r) * (2r + 1) + dx + r].
    float w[kStencilDense * kStencilDense];
};

struct StencilPlan {
    StencilArgs a;
    int shape;           // rearr_stencil_shape
    int body;            // kBody*
    int n_unique;        // distinct tap offsets
    int64_t n_tiles;     // 0: nothing to launch
    size_t smem_bytes;   // dynamic shared memory per CTA
};

// Validates the call, classifies the tap set and fills the kernel arguments.  Pointers may be fake addresses (describe).
rearr_status plan_stencil2d(float *dst, const float *src, int64_t ny, int64_t nx, int ntaps, const int *dy,
                            const int *dx, const float *w, int boundary, StencilPlan &pl, std::string &err);

cudaError_t launch_stencil2d(const StencilPlan &pl, cudaStream_t s);

// Reads the device's count of timed-out waits (synchronous).
cudaError_t read_wait_timeouts(uint64_t *count);

// Makes the next n TMA-staged launches wait for bytes that never arrive.
void inject_wait_timeout(int n);

}  // namespace rearr
