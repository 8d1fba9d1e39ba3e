// tuning.h -- tuning knobs of librearr: the batched kernel's work grab and
// the fast tile's staged row length per (element size, plane extents) class.
#pragma once

#include <stdint.h>

namespace rearr {

struct BatchTuning {
    // Tiles a CTA takes per atomicAdd on the work counter: enough work per
    // grab to hide the atomic, few enough that the tail balances.
    uint32_t min_grab = 1;
    uint32_t max_grab = 8;
    uint32_t grabs_per_cta = 8;  // target number of grabs per resident CTA

    uint32_t grab_for(uint64_t total_units, uint64_t resident_ctas) const
    {
        if (resident_ctas == 0) resident_ctas = 1;
        uint64_t g = total_units / (resident_ctas * grabs_per_cta);
        if (g < min_grab) g = min_grab;
        if (g > max_grab) g = max_grab;
        return uint32_t(g);
    }
};

BatchTuning batch_tuning();

// When a tiled permute runs as an element-wise strided copy instead (thin
// transpose planes): when its tiles would average fewer than tile_bytes of
// payload, or, for ops of at most l2_bytes (whose scattered reads stay in the
// L2), fewer than tile_cells cells (capped at the cells a full tile holds, so
// an op whose tiles are all full stays tiled).
struct ThinTuning {
    uint64_t tile_bytes = 1024;
    uint64_t tile_cells = 1024;
    uint64_t l2_bytes = uint64_t(32) << 20;
};

// Runs of at most this many bytes are walked in input order (sequential
// reads, whole runs written scattered) when the input is a dense array;
// 0 keeps output order for every run length.
uint64_t runs_mirror_max_bytes();

// Runs (cells of 128 bytes or more) shorter than runs_tile_max_bytes() on a
// transpose plane are copied in square blocks of cells (tile_runs_body); 1
// never.  A block side holds runs_tile_side_bytes() / cell cells, at least
// runs_tile_cells().
uint64_t runs_tile_max_bytes();
uint64_t runs_tile_cells();
uint64_t runs_tile_side_bytes();

// Widest global access of a fast tile: 16 (the widest the alignment allows)
// or 4 (loads and stores of at most 4 bytes; for measuring the choice).
int tile_vector_bytes();

ThinTuning thin_tuning();

// A fast tile's plane side (input rows of DA * E bytes, output runs of
// DB * E bytes) shorter than this is widened over the axis that continues it
// (plan.cpp, choose_widening); 1 never widens.
uint64_t wide_min_bytes();

// Ops smaller than this run 32 KB fast tiles as 16 KB tiles of the same row
// length (enough CTAs to fill the GPU).
uint64_t double_tile_min_bytes();

// A large random reorder scatters through CTA-sized destination chunks in
// shared memory when its (source chunk, destination chunk) bucket count is at
// most this; above it (or at 1) it scatters through ~16 MB chunks in the L2.
uint64_t reorder_smem_max_buckets();

// Thin planes of cells of at most box_max_cell_bytes() (0, the default: none)
// run as staged boxes (OC_BOX) when the box's input and output runs both reach
// box_min_run_bytes(), else as strided copies.  A box grows until both runs
// reach box_run_bytes() and it holds half a tile.
uint64_t box_min_run_bytes();
uint64_t box_run_bytes();
uint64_t box_max_cell_bytes();

// Shape of a fast tile: staged row bytes (128, 256 or 512) and payload bytes
// (16384; 8192 for the half tile; 32768 for the double tile of a widened
// plane, where double_tile_ok).
struct TileShape {
    int rowb;
    int tbytes;
};

// The 32 KB tile shapes that exist (variants.h).
constexpr bool double_tile_ok(int E, int rowb)
{
    return E <= 2 ? (rowb == 128 || rowb == 256) : (E <= 16 && (rowb == 256 || rowb == 512));
}

// The shape the tuning table assigns to a fully vectorised fast tile of
// element size E on a DA x DB plane (extents before widening; `wide`: the
// plane is widened); false if the table has no entry.
bool tuned_shape(int E, int64_t DA, int64_t DB, bool wide, TileShape &shape);

}  // namespace rearr
