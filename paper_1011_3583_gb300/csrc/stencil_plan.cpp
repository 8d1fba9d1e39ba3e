// stencil_plan.cpp -- host plan compiler of the 2-D stencil (Sec. III.D).
//
// The paper writes the stencil as a functor with a single-threaded stencil
// function and instantiates the kernel template with it.  A C caller passes a
// weighted tap list instead; this file recognises the two families the
// register-blocked bodies are compiled for -- the full cross of radius r (the
// order-r finite-difference Laplacian of the paper's experiments) and the
// full (2r+1)^2 box for r <= 2 (smoothing filters), each with distinct
// offsets.  Everything else runs the generic body over the taps as given.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "stencil.h"

namespace rearr {

rearr_status plan_stencil2d(float *dst, const float *src, int64_t ny, int64_t nx, int ntaps, const int *dy,
                            const int *dx, const float *w, int boundary, StencilPlan &pl, std::string &err)
{
    std::memset(&pl, 0, sizeof(pl));
    if (ny < 0 || nx < 0) return err = "negative grid extent", REARR_EINVAL;
    if (ntaps < 1 || ntaps > kStencilMaxTaps) return err = "ntaps must be 1..64", REARR_EINVAL;
    if (!dy || !dx || !w) return err = "NULL tap array", REARR_EINVAL;
    if (boundary != REARR_STENCIL_ZERO && boundary != REARR_STENCIL_CLAMP)
        return err = "boundary must be REARR_STENCIL_ZERO or REARR_STENCIL_CLAMP", REARR_EINVAL;

    // Taps are kept as given: two taps at one offset are two terms of the sum
    // (merging them would change the sum's NaN / infinity behaviour, e.g.
    // 0 * inf + 1 * inf is NaN while (0 + 1) * inf is not).
    int r = 0, n_unique = 0;
    bool repeats = false;
    for (int k = 0; k < ntaps; ++k) {
        if (dy[k] < -kStencilMaxRadius || dy[k] > kStencilMaxRadius || dx[k] < -kStencilMaxRadius ||
            dx[k] > kStencilMaxRadius)
            return err = "tap offset beyond radius 8", REARR_EINVAL;
        bool seen = false;
        for (int q = 0; q < k && !seen; ++q) seen = dy[q] == dy[k] && dx[q] == dx[k];
        repeats |= seen;
        n_unique += seen ? 0 : 1;
        r = std::max(r, std::max(std::abs(dy[k]), std::abs(dx[k])));
    }

    StencilArgs &a = pl.a;
    a.src = src;
    a.dst = dst;
    a.ny = ny;
    a.nx = nx;
    a.r = r;
    a.boundary = boundary;
    a.ntaps = ntaps;
    bool on_axes = true;
    for (int k = 0; k < ntaps; ++k) {
        a.w[(dy[k] + r) * (2 * r + 1) + dx[k] + r] = w[k];
        on_axes &= dy[k] == 0 || dx[k] == 0;
    }
    // The generic body loads one input column per distinct dx and applies
    // every tap of that column from registers: group the taps by dx.
    int k_out = 0;
    for (int gx = -kStencilMaxRadius; gx <= kStencilMaxRadius; ++gx) {
        const int k0 = k_out;
        for (int k = 0; k < ntaps; ++k) {
            if (dx[k] != gx) continue;
            a.tdy[k_out] = int8_t(dy[k]);
            a.tdx[k_out] = int8_t(dx[k]);
            a.tw[k_out] = w[k];
            ++k_out;
        }
        if (k_out > k0) {
            a.gdx[a.ngroups] = int8_t(gx);
            a.gend[a.ngroups] = uint8_t(k_out);
            ++a.ngroups;
        }
    }
    // With distinct offsets, a count of 4r + 1 on the axes is the full cross
    // and (2r + 1)^2 the full box.
    pl.shape = REARR_STENCIL_GENERIC;
    if (!repeats && r >= 1 && on_axes && ntaps == 4 * r + 1) pl.shape = REARR_STENCIL_CROSS;
    if (!repeats && r >= 1 && r <= 2 && ntaps == (2 * r + 1) * (2 * r + 1)) pl.shape = REARR_STENCIL_BOX;
    pl.body = pl.shape != REARR_STENCIL_GENERIC ? pl.shape
              : ntaps <= kGenericTapsMax        ? kBodyGenericTaps
                                                : kBodyGenericColumns;
    pl.n_unique = n_unique;
    pl.smem_bytes = size_t(kStencilTileY + 2 * r) * kStencilPitch * sizeof(float);

    const uintptr_t s = reinterpret_cast<uintptr_t>(src), d = reinterpret_cast<uintptr_t>(dst);
    // TMA coordinates are signed 32-bit: keep every box inside that range.
    a.tma = (s % 16 == 0 && d % 16 == 0 && nx % 4 == 0 && nx < (int64_t(1) << 31) - 256 &&
             ny < (int64_t(1) << 31) - 256) ? 1 : 0;
    a.tiles_x = (nx + kStencilTileX - 1) / kStencilTileX;
    const int64_t tiles_y = (ny + kStencilTileY - 1) / kStencilTileY;
    if (ny == 0 || nx == 0) return REARR_OK;  // nothing to compute

    if (!dst || !src) return err = "NULL grid pointer", REARR_EINVAL;
    if (nx > (int64_t(1) << 40) || ny > (int64_t(1) << 40) || ny > (int64_t(1) << 60) / nx)
        return err = "grid too large", REARR_EINVAL;
    const uint64_t bytes = uint64_t(ny) * uint64_t(nx) * sizeof(float);
    if (s < d + bytes && d < s + bytes) return err = "dst overlaps src", REARR_EINVAL;
    if (a.tiles_x * tiles_y > int64_t(0x7fffffff)) return err = "grid too large", REARR_EINVAL;
    pl.n_tiles = a.tiles_x * tiles_y;
    return REARR_OK;
}

}  // namespace rearr
