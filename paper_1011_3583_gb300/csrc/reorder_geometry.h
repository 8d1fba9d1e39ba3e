// reorder_geometry.h -- bucket geometry and scratch layout of the
// L2-resident reorder passes (k_reorder_l2.cu), shared with the host-only
// rearr_reorder_describe.  Source chunks of ~16 MB (at most 512 of them);
// destination chunks of 64 KB (one CTA's shared memory) while the bucket
// count stays within the bound, else the source chunks' size.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <algorithm>

namespace rearr {

constexpr uint32_t kReorderMaxChunks = 512;
constexpr uint64_t kReorderSourceChunkBytes = uint64_t(16) << 20;
constexpr uint32_t kReorderScatterChunkBytes = 64u << 10;
constexpr uint64_t kReorderMaxSmemBuckets = uint64_t(1) << 24;

struct ReorderGeometry {
    uint32_t cs_shift;   // source chunk = 2^cs_shift elements
    uint32_t ds_shift;   // destination chunk = 2^ds_shift elements
    uint32_t C, D;       // source / destination chunks (D = 1 for a scatter)
    bool smem_scatter;   // the gather's last pass through shared memory
    // scratch layout: byte offsets of the arrays and the total
    size_t off_hist, off_row, off_base, off_cur, off_up, off_s, off_i, off_v, off_st, bytes;
};

// n elements of W bytes; scatter: buckets by destination chunk only;
// smem_bucket_limit: the tuned bound on C * D for the shared-memory scatter.
inline ReorderGeometry reorder_geometry(uint64_t n, uint32_t W, bool scatter, uint64_t smem_bucket_limit)
{
    ReorderGeometry g{};
    uint32_t shift = 0;
    while ((uint64_t(1) << shift) * W < kReorderSourceChunkBytes) ++shift;
    while (((n + (uint64_t(1) << shift) - 1) >> shift) > kReorderMaxChunks) ++shift;
    g.cs_shift = shift;
    g.C = uint32_t((n + (uint64_t(1) << shift) - 1) >> shift);
    uint32_t dshift = 0;
    while ((uint64_t(2) << dshift) * W <= kReorderScatterChunkBytes) ++dshift;
    const uint64_t d_small = (n + (uint64_t(1) << dshift) - 1) >> dshift;
    g.smem_scatter = !scatter && uint64_t(g.C) * d_small <= std::min(smem_bucket_limit, kReorderMaxSmemBuckets);
    g.ds_shift = g.smem_scatter ? dshift : shift;
    g.D = scatter ? 1u : g.smem_scatter ? uint32_t(d_small) : g.C;
    const size_t nb = size_t(g.C) * g.D;
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    g.off_hist = 256;
    g.off_row = g.off_hist + al(nb * 4);
    g.off_base = g.off_row + al(size_t(g.C) * 4);
    g.off_cur = g.off_base + al(nb * 4);
    g.off_up = g.off_cur + al(nb * 4);
    g.off_s = g.off_up + al((nb + 1) * 4);
    g.off_i = g.off_s + al(size_t(n) * 4);
    g.off_v = g.off_i + al(size_t(n) * 4);
    g.off_st = g.off_v + al(size_t(n) * W);
    // tile-local form: C + 1 segment starts (uint16) per 4096-index tile
    const size_t tiles = size_t((n + 4095) / 4096);
    g.bytes = g.off_st + al(tiles * (size_t(g.C) + 1) * 2);
    return g;
}

}  // namespace rearr
