// plan.cpp -- host plan compiler of librearr.
//
// A permute is brought to canonical form in the spirit of the paper's
// "offset/striding approach" (arXiv:1011.3583 Sec. III.B):
//   1. extent-1 axes are dropped;
//   2. output axes that are adjacent and in order in the input are merged
//      (stride[i] == stride[i+1] * extent[i+1]);
//   3. an unmoved innermost axis (input stride 1 on the output's last axis)
//      is folded into a wider cell; after that the output's fastest axis
//      always differs from the input's fastest axis;
//   4. the op is classified: a plain copy, long contiguous runs, or a tiled
//      transpose on the plane of the input's fastest and the output's fastest
//      axes with the other axes as batch (Sec. III.B: the 2-D plane of the
//      fastest dimensions of the original and the desired order).
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "tuning.h"
#include "variants.h"

namespace rearr {

namespace {

constexpr int64_t kMaxExtent = (int64_t(1) << 31) - 1;
constexpr int64_t kRunMinBytes = 128;     // cells this large are copied as runs
constexpr int64_t kRunUnitBytes = 32768;  // payload of one runs work unit
constexpr uint64_t kReorderL2MinBytes = uint64_t(128) << 20;  // reorder sources this large use L2 passes
constexpr uint64_t kMaxUnits = 0xFFFFFFFFull;

bool mul_overflows(uint64_t a, uint64_t b, uint64_t &out)
{
    if (a != 0 && b > UINT64_MAX / a) return true;
    out = a * b;
    return false;
}

bool ranges_overlap(uintptr_t a, uint64_t na, uintptr_t b, uint64_t nb)
{
    if (na == 0 || nb == 0) return false;
    return a < b + nb && b < a + na;
}

struct Axis {
    int64_t extent;
    int64_t stride;  // input stride in bytes
};

}  // namespace

int pow2_align(uint64_t a, uint64_t b, uint64_t c, uint64_t d)
{
    const uint64_t v = a | b | c | d | 16;
    return int(v & (~v + 1));  // lowest set bit, at most 16
}

// Shape of a fully vectorised fast tile: staged row bytes (128/256/512) and
// payload (16 KB, or the 8 KB half tile where an element size has one).  The
// shape that fills the DA x DB plane best is chosen (ragged last tiles waste
// bandwidth), ties broken toward full tiles and then toward equal input-row
// and output-row bytes.  An autotuned table may override the choice per
// (E, DA, DB) class.
static TileShape choose_shape(int E, int64_t DA, int64_t DB)
{
    std::vector<TileShape> cands = {{128, kTileBytes}, {256, kTileBytes}};
    if (E != 1) cands.push_back({512, kTileBytes});
    if (half_tile_vout(E)) cands.push_back({128, kTileBytes / 2});
    TileShape best{default_rowb(E), kTileBytes};
    double best_util = -1.0, best_bal = 1e9;
    for (const TileShape &c : cands) {
        const int64_t TA = c.rowb / E, TB = c.tbytes / c.rowb;
        const double ua = double(DA) / double(((DA + TA - 1) / TA) * TA);
        const double ub = double(DB) / double(((DB + TB - 1) / TB) * TB);
        const double util = ua * ub;
        // a half tile must fill clearly better to be chosen
        const double bal = std::fabs(std::log2(double(c.rowb)) - std::log2(double(TB * E))) +
                           (c.tbytes < kTileBytes ? 8.0 : 0.0);
        if (util > best_util + 0.01 || (util > best_util - 0.01 && bal < best_bal)) {
            best = c;
            best_util = std::max(best_util, util);
            best_bal = bal;
        }
    }
    TileShape tuned;
    if (tuned_shape(E, DA, DB, false, tuned) && (tuned.tbytes != kTileBytes / 2 || half_tile_vout(E))) return tuned;
    return best;
}

// The tile descriptor of plane (A = axis p, B = axis R-1) with the other
// axes as batch.  qa / qb (-1: none) are the batch axes that A / B absorb
// (a widened plane): A then spans DA * extent(qa) cells, B DB * extent(qb).
// Tile shape of a widened plane (see choose_widening): the candidate that
// fills the DA x DB plane (extents after widening) best, then the one whose
// shorter side -- input rows of ROWB bytes or output runs of TB * E bytes,
// each at most what the plane offers -- is longest (up to 512 bytes), then
// the smaller tile.  32 KB tiles exist for the shapes of double_tile_ok().
static TileShape choose_wide_shape(int E, int64_t DA0, int64_t DB0, int64_t DA, int64_t DB)
{
    TileShape tuned;
    if (tuned_shape(E, DA0, DB0, true, tuned)) return tuned;
    TileShape best{default_rowb(E), kTileBytes};
    double best_util = -1.0;
    int64_t best_run = -1;
    for (int rowb : {128, 256, 512}) {
        if (E == 1 && rowb == 512) continue;
        for (int tbytes : {kTileBytes, 2 * kTileBytes}) {
            if (tbytes > kTileBytes && !double_tile_ok(E, rowb)) continue;
            const int64_t TA = rowb / E, TB = tbytes / rowb;
            const double ua = double(DA) / double(((DA + TA - 1) / TA) * TA);
            const double ub = double(DB) / double(((DB + TB - 1) / TB) * TB);
            const double util = ua * ub;
            const int64_t run = std::min<int64_t>({int64_t(rowb), DA * E, TB * E, DB * E, 512});
            if (util > best_util + 0.01 || (util > best_util - 0.01 && run > best_run)) {
                best = {rowb, tbytes};
                best_util = std::max(best_util, util);
                best_run = run;
            }
        }
    }
    return best;
}

// A transpose plane whose input rows (DA cells of A) or output runs (DB cells
// of B) are short leaves DRAM with short bursts scattered far apart: every
// tile reads DB rows of DA*E bytes at the stride of B and writes DA runs of
// DB*E bytes at the stride of A.  Such a side is widened over the axis that
// continues it -- A over the batch axis of input stride DA cells (the input
// stays contiguous across the planes), B over the output axis just before it
// (the output stays contiguous) -- so one tile spans several planes and both
// its reads and its writes come in runs of up to 512 bytes.  Sides of at
// least wide_min_bytes() are left alone; an axis that continues both sides
// widens the shorter one.  Fast tiles only (one element per cell).  When DA
// is not a multiple of a 16-byte chunk's elements, the store phase splits
// every element's coordinate on its own (tile_fast_body).
static void choose_widening(const std::vector<Axis> &ax, int p, int64_t cell, int &qa, int &qb)
{
    const int R = int(ax.size());
    const uint64_t lim = wide_min_bytes();
    qa = qb = -1;
    if (R < 3) return;
    const int64_t DA = ax[p].extent, DB = ax[R - 1].extent;
    if (uint64_t(DA * cell) < lim)
        for (int i = 0; i < R - 1; ++i)
            if (i != p && ax[i].stride == DA * cell && DA * ax[i].extent <= kMaxExtent) qa = i;
    if (uint64_t(DB * cell) < lim && R - 2 != p && DB * ax[R - 2].extent <= kMaxExtent) qb = R - 2;
    if (qa >= 0 && qa == qb) {
        if (DA <= DB) qb = -1;
        else qa = -1;
    }
}

static void fill_tile_common(TileDesc &t, const std::vector<Axis> &ax, int p, int64_t cell, int qa, int qb,
                             char *dst, const char *src)
{
    const int R = int(ax.size());
    // Output strides (cells) of the canonical output axes, row-major.
    std::vector<int64_t> os(R);
    os[R - 1] = 1;
    for (int i = R - 2; i >= 0; --i) os[i] = os[i + 1] * ax[i + 1].extent;
    const int64_t DA = ax[p].extent, DB = ax[R - 1].extent;
    t.dst = dst;
    t.src = src;
    t.sb_in = ax[R - 1].stride;
    t.sa_out = os[p] * cell;
    t.DA = uint32_t(qa >= 0 ? DA * ax[qa].extent : DA);
    t.DB = uint32_t(qb >= 0 ? DB * ax[qb].extent : DB);
    t.da_split = make_fastdiv(uint32_t(DA));
    t.db_split = make_fastdiv(uint32_t(DB));
    t.sa1_out = qa >= 0 ? os[qa] * cell : 0;
    t.sb1_in = qb >= 0 ? ax[qb].stride : 0;
    int nb = 0;
    for (int i = 0; i < R; ++i) {
        if (i == p || i == R - 1 || i == qa || i == qb) continue;
        t.bin[nb] = ax[i].stride;
        t.bout[nb] = os[i] * cell;
        t.bdiv[nb] = make_fastdiv(uint32_t(ax[i].extent));
        ++nb;
    }
    for (int i = nb; i < kMaxBatch; ++i) {
        t.bin[i] = 0;
        t.bout[i] = 0;
        t.bdiv[i] = make_fastdiv(1);
    }
    t.nb = nb;
}

// Box plan of a thin-plane permute with cells of one aligned E-byte word (see
// BoxDesc).  The unit's sub-box U grows from the input-innermost and the
// output-innermost axes: each step takes the axis that continues the shorter
// of the two runs (the input chain's next axis has an input stride equal to
// the chain's length, the output chain's an output stride equal to its),
// else the other side's, whole while the unit fits kBoxBytes.  When neither
// fits whole, the first becomes the partial axis over K indices (the last
// step).  Growth stops once both runs reach box_run_bytes() and the unit holds
// half a tile.  False when the box needs more axes than the descriptor holds,
// a run stays shorter than box_min_run_bytes(), or its stores would be
// narrower than 4 bytes.
static bool plan_box(const std::vector<Axis> &ax, int64_t E, uintptr_t da, uintptr_t sa, char *dst,
                     const char *src, OpDesc &op, rearr_permute_info &info)
{
    const int R = int(ax.size());
    std::vector<int64_t> os(R);  // output strides in bytes
    os[R - 1] = E;
    for (int i = R - 2; i >= 0; --i) os[i] = os[i + 1] * ax[i + 1].extent;
    const int64_t cap = kBoxBytes / E;
    std::vector<int> U;
    int kax = -1;
    int64_t K = 1, prod = 1;
    auto in_u = [&](int i) { return std::find(U.begin(), U.end(), i) != U.end(); };
    // One side's chain: its run in bytes, the axes on it and the next axis (-1: none).
    auto chain = [&](bool input, int64_t &run, std::vector<int> &on, int &next) {
        run = E;
        on.clear();
        next = -1;
        for (;;) {
            int hit = -1;
            for (int i = 0; i < R; ++i)
                if ((input ? ax[i].stride : os[i]) == run) hit = i;
            if (hit < 0) return;
            if (!in_u(hit)) {
                next = hit;
                return;
            }
            on.push_back(hit);
            if (hit == kax) {
                run *= K;
                return;
            }
            run *= ax[hit].extent;
        }
    };
    int64_t rin = E, rout = E;
    std::vector<int> on_in, on_out;
    const int64_t target = int64_t(box_run_bytes());
    for (;;) {
        int nin, nout;
        chain(true, rin, on_in, nin);
        chain(false, rout, on_out, nout);
        if (kax >= 0 || int(U.size()) == kMaxBoxAxes) break;
        if (rin >= target && rout >= target && 2 * prod * E >= kBoxBytes) break;
        const int first = rin <= rout ? (nin >= 0 ? nin : nout) : (nout >= 0 ? nout : nin);
        const int second = first == nin ? nout : nin;
        if (first < 0) break;
        if (prod * ax[first].extent <= cap) {
            U.push_back(first);
            prod *= ax[first].extent;
            continue;
        }
        if (second >= 0 && prod * ax[second].extent <= cap) {
            U.push_back(second);
            prod *= ax[second].extent;
            continue;
        }
        int64_t k = cap / prod;
        // range starts stay 16-byte aligned on both sides where K allows
        const int64_t m = std::max(16 / std::min<int64_t>(16, ax[first].stride & -ax[first].stride),
                                   16 / std::min<int64_t>(16, os[first] & -os[first]));
        if (k >= 2 * m) k -= k % m;
        if (k < 2) break;
        U.push_back(first);
        kax = first;
        K = k;
        prod *= k;
    }
    if (rin < int64_t(box_min_run_bytes()) || rout < int64_t(box_min_run_bytes())) return false;
    // unit-index axes: the others in output order, the partial axis as its range index
    struct Slot {
        int64_t ext, in, out;
    };
    std::vector<Slot> outer;
    int kunit = -1;
    for (int i = 0; i < R; ++i) {
        if (i == kax) {
            kunit = int(outer.size());
            outer.push_back({(ax[i].extent + K - 1) / K, K * ax[i].stride, K * os[i]});
        } else if (!in_u(i)) {
            outer.push_back({ax[i].extent, ax[i].stride, os[i]});
        }
    }
    if (int(outer.size()) > kMaxBoxOuter) return false;
    uint64_t units = 1;
    for (const Slot &o : outer) units *= uint64_t(o.ext);
    if (units >= kMaxUnits) return false;
    // widest loads / stores: within a run, and every run start aligned
    auto width = [&](bool input) {
        const std::vector<int> &on = input ? on_in : on_out;
        uint64_t bits = uint64_t(input ? rin : rout) | uint64_t(input ? sa : da) | 16;
        for (int i : U)
            if (std::find(on.begin(), on.end(), i) == on.end()) bits |= uint64_t(input ? ax[i].stride : os[i]);
        for (const Slot &o : outer) bits |= uint64_t(input ? o.in : o.out);
        const uint64_t v = bits & (~bits + 1);
        return uint32_t(std::max<uint64_t>(v, uint64_t(E)));
    };
    BoxDesc b;
    std::memset(&b, 0, sizeof(b));
    b.dst = dst;
    b.src = src;
    std::vector<int> by_in = U, by_out = U;
    std::sort(by_in.begin(), by_in.end(), [&](int x, int y) { return ax[x].stride < ax[y].stride; });
    std::sort(by_out.begin(), by_out.end(), [&](int x, int y) { return os[x] < os[y]; });
    const int nu = int(U.size());
    std::vector<int64_t> sm(R, 0);  // shared-memory strides, dense in input order
    int64_t acc = E;
    for (int j = 0; j < nu; ++j) {
        const int i = by_in[j];
        const int64_t ext = i == kax ? K : ax[i].extent;
        b.iext[j] = make_fastdiv(uint32_t(ext));
        b.iin[j] = ax[i].stride;
        sm[i] = acc;
        acc *= ext;
    }
    for (int j = 0; j < nu; ++j) {
        const int i = by_out[j];
        b.oext[j] = make_fastdiv(uint32_t(i == kax ? K : ax[i].extent));
        b.oout[j] = os[i];
        b.osm[j] = uint32_t(sm[i]);
    }
    for (int j = nu; j < kMaxBoxAxes; ++j) b.iext[j] = b.oext[j] = make_fastdiv(1);
    const int no = int(outer.size());
    for (int j = 0; j < kMaxBoxOuter; ++j) {
        b.udiv[j] = make_fastdiv(j < no ? uint32_t(outer[j].ext) : 1u);
        b.uin[j] = j < no ? outer[j].in : 0;
        b.uout[j] = j < no ? outer[j].out : 0;
    }
    b.nu = int8_t(nu);
    b.no = int8_t(no);
    b.kin = b.kout = -1;
    for (int j = 0; j < nu; ++j) {
        if (by_in[j] == kax) b.kin = int8_t(j);
        if (by_out[j] == kax) b.kout = int8_t(j);
    }
    b.kunit = int8_t(kunit);
    b.K = uint32_t(K);
    b.kfull = uint32_t(kax >= 0 ? ax[kax].extent : 1);
    b.vin = width(true);
    b.vout = width(false);
    // byte or 2-byte stores of short cells: the strided copy writes its
    // contiguous output 16 bytes at a time instead
    if (b.vout < 4) return false;
    b.cells = uint32_t(prod);
    op.cls = OC_BOX;
    op.word = uint32_t(E);
    op.box = b;
    op.units = units;
    info.kind = REARR_KIND_BOX;
    info.word_bytes = int(E);
    info.tile_a = int(rin / E);
    info.tile_b = int(rout / E);
    info.vec_in = int(b.vin);
    info.vec_out = int(b.vout);
    info.wide_a = info.wide_b = -1;
    info.n_tiles = int64_t(units);
    return true;
}

// Plans a gather of `total` elements of elem_bytes whose output axes are
// given in order (slowest first) with their input byte strides; src already
// points at the element of output index 0.  The output is contiguous.
static rearr_status plan_axes(void *dst, const char *src, size_t elem_bytes, const std::vector<Axis> &in_axes,
                              uint64_t total, PermPlan &pl, std::string &err)
{
    rearr_permute_info &info = pl.info;
    const uint64_t bytes = total * elem_bytes;
    // Axes with extent > 1, merged where adjacent and in order.
    std::vector<Axis> ax;
    for (const Axis &cur : in_axes) {
        if (cur.extent == 1) continue;
        if (!ax.empty() && ax.back().stride == cur.stride * cur.extent) {
            ax.back().extent *= cur.extent;
            ax.back().stride = cur.stride;
        } else {
            ax.push_back(cur);
        }
    }
    int64_t cell = int64_t(elem_bytes);
    const uintptr_t da = uintptr_t(dst), sa = uintptr_t(src);

    auto set_copy = [&]() {
        info.kind = REARR_KIND_COPY;
        info.rank = 1;
        info.dims[0] = int64_t(total);
        info.in_strides[0] = 1;
        info.cell_bytes = int64_t(elem_bytes);
        const int W = pow2_align(da, sa, bytes);
        info.word_bytes = W;
        OpDesc &op = pl.op;
        op.cls = OC_COPY;
        op.word = uint32_t(W);
        op.copy.dst = static_cast<char *>(dst);
        op.copy.src = src;
        op.copy.bytes = bytes;
        op.copy.unit_bytes = uint64_t(kThreads) * 4 * W;
        op.units = (bytes + op.copy.unit_bytes - 1) / op.copy.unit_bytes;
        info.n_tiles = int64_t(op.units);
    };

    if (ax.empty() || (ax.size() == 1 && ax[0].stride == cell)) {  // one contiguous range
        set_copy();
        return REARR_OK;
    }
    // Fold an unmoved (input-contiguous) innermost axis into the cell.
    if (ax.back().stride == cell) {
        cell *= ax.back().extent;
        ax.pop_back();
        if (ax.empty() || (ax.size() == 1 && ax[0].stride == cell)) {
            set_copy();
            return REARR_OK;
        }
    }
    const int R = int(ax.size());
    uint64_t strides_or = 0;
    info.rank = R;
    for (int i = 0; i < R; ++i) {
        info.dims[i] = ax[i].extent;
        info.in_strides[i] = ax[i].stride / cell;
        strides_or |= uint64_t(ax[i].stride);
    }
    info.cell_bytes = cell;
    int p = -1;  // output axis along which input cells are contiguous
    for (int i = 0; i < R; ++i)
        if (ax[i].stride == cell) p = i;

    // Every output cell copied on its own (one cell is one W-byte word), 16/W
    // consecutive cells per thread written with one 16-byte store.
    auto set_strided = [&](int W, uint64_t n_cells) {
        StridedDesc sd;
        std::memset(&sd, 0, sizeof(sd));
        sd.dst = static_cast<char *>(dst);
        sd.src = src;
        sd.nd = R;
        for (int i = 0; i < kMaxRank; ++i) {
            sd.in_stride[i] = i < R ? ax[i].stride : 0;
            sd.div[i] = make_fastdiv(i < R ? uint32_t(ax[i].extent) : 1u);
        }
        sd.n_cells = n_cells;
        sd.vec = (da % 16 == 0) ? 1u : 0u;
        const uint64_t per_unit = uint64_t(kThreads) * (16 / W) * kStridedSteps;
        OpDesc &op = pl.op;
        op.cls = OC_STRIDED;
        op.word = uint32_t(W);
        op.strided = sd;
        op.units = (n_cells + per_unit - 1) / per_unit;
        info.kind = REARR_KIND_STRIDED;
        info.tile_a = info.tile_b = 0;
        info.wide_a = info.wide_b = -1;
        info.word_bytes = W;
        info.vec_in = W;
        info.vec_out = sd.vec ? 16 : W;
        info.n_tiles = int64_t(op.units);
    };

    // A box with no input-contiguous axis and cells of one aligned word (the
    // input's fastest axis dropped): every read is a scattered word, so each
    // cell is gathered on its own and the output written 16 bytes at a time.
    if (p < 0 && cell <= 16) {
        const int W = pow2_align(da, sa, uint64_t(cell), strides_or);
        const uint64_t n_cells = bytes / uint64_t(cell);
        bool fits = n_cells < kMaxUnits;
        for (int i = 0; i < R; ++i) fits &= ax[i].extent < int64_t(kMaxUnits);
        if (W == cell && fits) {
            set_strided(W, n_cells);
            return REARR_OK;
        }
    }

    // Cells of 128 bytes or more are copied as runs, and so are boxes with no
    // input-contiguous axis (there both sides cannot be coalesced).  Runs
    // shorter than runs_tile_max_bytes() on a transpose plane are copied in
    // blocks of cells instead (tile_runs_body), for long runs on both sides.
    const bool blocked_runs = p >= 0 && cell >= kRunMinBytes && uint64_t(cell) < runs_tile_max_bytes();
    if ((cell >= kRunMinBytes && !blocked_runs) || p < 0) {
        const int W = pow2_align(da, sa, uint64_t(cell), strides_or);
        uint64_t n_runs = 1;
        for (int i = 0; i < R; ++i) n_runs *= uint64_t(ax[i].extent);
        if (n_runs > kMaxUnits) { err = "too many runs"; return REARR_EINVAL; }
        for (int i = 0; i < R; ++i)
            if (ax[i].extent > int64_t(kMaxUnits)) { err = "a collapsed axis has 2^32 or more elements"; return REARR_EINVAL; }
        info.kind = REARR_KIND_RUNS;
        info.word_bytes = W;
        OpDesc &op = pl.op;
        op.cls = OC_RUNS;
        op.word = uint32_t(W);
        RunsDesc &r = op.runs;
        r.dst = static_cast<char *>(dst);
        r.src = src;
        r.run_bytes = cell;
        r.nd = R;
        for (int i = 0; i < kMaxRank; ++i) {
            r.in_stride[i] = i < R ? ax[i].stride : 0;
            r.div[i] = make_fastdiv(i < R ? uint32_t(ax[i].extent) : 1u);
        }
        r.n_runs = n_runs;
        const uint64_t wpr = uint64_t(cell) / W;
        if (wpr > 0xFFFFFFFFull) { err = "a run has 2^32 or more words"; return REARR_EINVAL; }
        r.wpr_div = make_fastdiv(uint32_t(wpr));
        if (cell > kRunUnitBytes) {
            // long runs: units are chunks of kRunUnitBytes
            const uint64_t cw = kRunUnitBytes / W;
            const uint64_t cpr = (wpr + cw - 1) / cw;
            if (n_runs * cpr > kMaxUnits) { err = "too many run chunks"; return REARR_EINVAL; }
            r.chunk_words = uint32_t(cw);
            r.cpr_div = make_fastdiv(uint32_t(cpr));
            r.runs_per_unit = 1;
            op.units = n_runs * cpr;
        } else {
            r.chunk_words = uint32_t(wpr);
            r.cpr_div = make_fastdiv(1);
            r.runs_per_unit = uint32_t(std::min<int64_t>(kMaxRunsPerUnit, std::max<int64_t>(1, kRunUnitBytes / cell)));
            op.units = (n_runs + r.runs_per_unit - 1) / r.runs_per_unit;
            // Short runs of a dense input may be walked in input order: the
            // reads become sequential and each run is written whole.
            if (uint64_t(cell) <= runs_mirror_max_bytes()) {
                std::vector<int> by_in(R);
                for (int i = 0; i < R; ++i) by_in[i] = i;
                std::sort(by_in.begin(), by_in.end(), [&](int a, int b) { return ax[a].stride > ax[b].stride; });
                bool dense = true;
                int64_t expect = cell;
                for (int k = R - 1; k >= 0; --k) {
                    dense &= ax[by_in[k]].stride == expect;
                    expect *= ax[by_in[k]].extent;
                }
                if (dense) {
                    std::vector<int64_t> out_stride(R);
                    int64_t os = cell;
                    for (int i = R - 1; i >= 0; --i) {
                        out_stride[i] = os;
                        os *= ax[i].extent;
                    }
                    r.mirror = 1;
                    for (int k = 0; k < kMaxRank; ++k) {
                        r.in_stride[k] = k < R ? out_stride[by_in[k]] : 0;
                        r.div[k] = make_fastdiv(k < R ? uint32_t(ax[by_in[k]].extent) : 1u);
                    }
                }
            }
        }
        info.n_tiles = int64_t(op.units);
        return REARR_OK;
    }

    info.plane_a = p;
    const int64_t DA = ax[p].extent, DB = ax[R - 1].extent;
    for (int i = 0; i < R; ++i)
        if (ax[i].extent > kMaxExtent) { err = "a collapsed axis has 2^31 or more elements"; return REARR_EINVAL; }

    OpDesc &op = pl.op;
    TileDesc &t = op.tile;
    const int W = pow2_align(da, sa, uint64_t(cell), strides_or);
    info.word_bytes = W;
    int vin = 0, vout = 0, qa = -1, qb = -1;
    if (W == cell) {
        const int E = int(cell);
        // Widest legal global access on each side.  Input rows start at src
        // plus sums of the input strides of the axes other than A (and other
        // than the axis a widened A absorbs: the widened row is contiguous
        // over DA * extent(qa) cells, so the load width follows that row
        // length); output rows start at multiples of DB*E bytes from dst.
        choose_widening(ax, p, cell, qa, qb);
        uint64_t in_or = 0;
        for (int i = 0; i < R; ++i)
            if (i != p && i != qa) in_or |= uint64_t(ax[i].stride);
        const int64_t DAw = qa >= 0 ? DA * ax[qa].extent : DA;
        const int vcap = tile_vector_bytes();
        vin = E;
        for (int v : {16, 4}) {
            if (v > E && v <= vcap && (uint64_t(DAw) * E) % v == 0 && sa % v == 0 && in_or % v == 0) { vin = v; break; }
        }
        vout = E;
        const int vmax = std::min(std::min(16, 4 * E), vcap);
        for (int v : {vmax, 4}) {
            if (v > E && (uint64_t(DB) * E) % v == 0 && da % v == 0) { vout = v; break; }
        }
    }
    fill_tile_common(t, ax, p, cell, qa, qb, static_cast<char *>(dst), src);
    info.wide_a = qa;
    info.wide_b = qb;
    uint64_t batch = 1;
    for (int i = 0; i < t.nb; ++i) batch *= t.bdiv[i].d;

    if (W == cell) {
        // Fast tile: one power-of-two element per cell.
        const int E = int(cell);
        // Tile shape: the default for the element size, or for the fully
        // vectorised widths the shape that fills the plane best (a widened
        // plane: the shape with the longest runs on both sides).
        TileShape shape{default_rowb(E), kTileBytes};
        if (vin == 16 && vout == std::min(16, 4 * E)) {
            shape = (qa >= 0 || qb >= 0) ? choose_wide_shape(E, DA, DB, t.DA, t.DB) : choose_shape(E, DA, DB);
            if (shape.tbytes < kTileBytes) vout = half_tile_vout(E);
        }
        t.TA = uint32_t(shape.rowb / E);
        t.TB = uint32_t(shape.tbytes / shape.rowb);
        info.kind = REARR_KIND_TILE;
        info.vec_in = vin;
        info.vec_out = vout;
        t.variant = tile_variant(E, vin, vout, shape.rowb, shape.tbytes);
        t.c = 1;
        t.pitch = 0;
        op.cls = OC_TILE;
    } else if (blocked_runs) {
        const int64_t c = cell / W;
        const int64_t side = std::max<int64_t>(int64_t(runs_tile_cells()), int64_t(runs_tile_side_bytes()) / cell);
        const int64_t nbk = std::max<int64_t>(1, std::min<int64_t>(side, 64));
        const int64_t TA = std::min<int64_t>(DA, nbk), TB = std::min<int64_t>(DB, nbk);
        if (TB * TA * c > int64_t(kMaxUnits)) { err = "a runs block has 2^32 or more words"; return REARR_EINVAL; }
        info.kind = REARR_KIND_TILE_CELLS;
        t.TA = uint32_t(TA);
        t.TB = uint32_t(TB);
        t.c = uint32_t(c);
        t.pitch = 0;  // no staging: blocked runs
        t.rowwords_div = make_fastdiv(uint32_t(TA * c));
        t.outwords_div = make_fastdiv(uint32_t(TB * c));
        t.c_div = make_fastdiv(uint32_t(c));
        t.variant = uint32_t(W);
        op.cls = OC_TILE_CELLS;
    } else {
        const int64_t c = cell / W;
        int64_t TA = std::max<int64_t>(1, std::min<int64_t>(DA, 256 / cell));
        int64_t TB = std::max<int64_t>(1, std::min<int64_t>(DB, 16384 / (TA * cell)));
        if (TB == DB) TA = std::max<int64_t>(1, std::min<int64_t>(DA, 16384 / (TB * cell)));
        auto pitch_of = [&](int64_t ta) {
            const int64_t rw = ta * c;
            const int64_t pad = ((c - rw) % 32 + 32) % 32;
            return rw + pad;
        };
        while (TB > 1 && TB * pitch_of(TA) * W > kSmemBytes) --TB;
        while (TA > 1 && TB * pitch_of(TA) * W > kSmemBytes) --TA;
        info.kind = REARR_KIND_TILE_CELLS;
        t.TA = uint32_t(TA);
        t.TB = uint32_t(TB);
        t.c = uint32_t(c);
        t.pitch = uint32_t(pitch_of(TA));
        t.rowwords_div = make_fastdiv(uint32_t(TA * c));
        t.outwords_div = make_fastdiv(uint32_t(TB * c));
        t.c_div = make_fastdiv(uint32_t(c));
        t.variant = uint32_t(W);
        op.cls = OC_TILE_CELLS;
    }
    info.tile_a = int(t.TA);
    info.tile_b = int(t.TB);
    const uint64_t ta_tiles = (uint64_t(t.DA) + t.TA - 1) / t.TA;
    const uint64_t tb_tiles = (uint64_t(t.DB) + t.TB - 1) / t.TB;
    const uint64_t units = ta_tiles * tb_tiles * batch;
    if (units > kMaxUnits || ta_tiles > kMaxUnits || tb_tiles > kMaxUnits) {
        err = "too many tiles";
        return REARR_EINVAL;
    }
    t.ta_div = make_fastdiv(uint32_t(ta_tiles));
    t.tb_div = make_fastdiv(uint32_t(tb_tiles));
    op.word = uint32_t(W);
    op.units = units;
    info.n_tiles = int64_t(units);

    // Thin planes (DA x DB far below a tile): every output cell copied on its
    // own (one cell is one W-byte word) when the tiles would carry little
    // payload on average -- a tile costs a whole load / store round trip
    // whatever its fill.  Decided after the tile plan so that the tile count
    // is the one the tile kernel would run; the thresholds are tuning knobs.
    // A 32 KB tile halves the CTA count: small ops keep the 16 KB tile of the
    // same row length so that they still fill the GPU.
    if (op.cls == OC_TILE && bytes < double_tile_min_bytes()) {
        tile_to_single_width(op);
        info.tile_b = int(t.TB);
        info.n_tiles = int64_t(op.units);
    }
    const uint64_t n_cells = bytes / uint64_t(cell);
    const ThinTuning thin = thin_tuning();
    // (a threshold above what a tile holds means: every under-filled tile;
    // ops whose tiles are all full stay tiles)
    const uint64_t cells_rule = std::min<uint64_t>(thin.tile_cells, uint64_t(t.TA) * t.TB);
    const bool thin_plane = bytes < op.units * thin.tile_bytes ||
                            (bytes <= thin.l2_bytes && n_cells < op.units * cells_rule);
    if (W == cell && thin_plane && n_cells < kMaxUnits &&
        !(uint64_t(cell) <= box_max_cell_bytes() && plan_box(ax, cell, da, sa, static_cast<char *>(dst), src, op, info)))
        set_strided(W, n_cells);
    return REARR_OK;
}

rearr_status plan_permute(void *dst, const void *src, size_t elem_bytes, int rank, const int64_t *dims,
                          const int *perm, PermPlan &pl, std::string &err)
{
    std::memset(&pl, 0, sizeof(pl));
    rearr_permute_info &info = pl.info;
    info.plane_a = -1;
    info.wide_a = info.wide_b = -1;
    if (elem_bytes == 0) { err = "elem_bytes must be >= 1"; return REARR_EINVAL; }
    if (rank < 1 || rank > kMaxRank) { err = "rank must be in [1, 8]"; return REARR_EINVAL; }
    if (!dims || !perm) { err = "dims and perm must not be NULL"; return REARR_EINVAL; }
    bool seen[kMaxRank] = {false};
    for (int i = 0; i < rank; ++i) {
        if (dims[i] < 0) { err = "dims must be >= 0"; return REARR_EINVAL; }
        if (perm[i] < 0 || perm[i] >= rank || seen[perm[i]]) {
            err = "perm is not a permutation of 0..rank-1";
            return REARR_EINVAL;
        }
        seen[perm[i]] = true;
    }
    uint64_t total = 1;
    for (int i = 0; i < rank; ++i)
        if (mul_overflows(total, uint64_t(dims[i]), total)) { err = "element count overflows"; return REARR_EINVAL; }
    uint64_t bytes;
    if (mul_overflows(total, elem_bytes, bytes) || bytes > (uint64_t(1) << 62)) {
        err = "byte count overflows";
        return REARR_EINVAL;
    }
    if (total == 0) {
        info.kind = REARR_KIND_NOOP;
        pl.op.units = 0;
        return REARR_OK;
    }
    if (!dst || !src) { err = "dst and src must not be NULL"; return REARR_EINVAL; }
    if (ranges_overlap(uintptr_t(dst), bytes, uintptr_t(src), bytes)) {
        err = "dst overlaps src (in-place permute is not supported)";
        return REARR_EINVAL;
    }
    // Row-major input strides in bytes; output axis i is input axis perm[i].
    int64_t s[kMaxRank];
    s[rank - 1] = int64_t(elem_bytes);
    for (int i = rank - 2; i >= 0; --i) s[i] = s[i + 1] * dims[i + 1];
    std::vector<Axis> ax;
    for (int i = 0; i < rank; ++i) ax.push_back(Axis{dims[perm[i]], s[perm[i]]});
    return plan_axes(dst, static_cast<const char *>(src), elem_bytes, ax, total, pl, err);
}

rearr_status plan_reorder_nm(void *dst, const void *src, size_t elem_bytes, int rank_in, const int64_t *dims,
                             int rank_out, const int *order, const int64_t *base, const int64_t *range,
                             PermPlan &pl, std::string &err)
{
    std::memset(&pl, 0, sizeof(pl));
    pl.info.plane_a = -1;
    pl.info.wide_a = pl.info.wide_b = -1;
    if (elem_bytes == 0) { err = "elem_bytes must be >= 1"; return REARR_EINVAL; }
    if (rank_in < 1 || rank_in > kMaxRank) { err = "rank_in must be in [1, 8]"; return REARR_EINVAL; }
    if (rank_out < 1 || rank_out > rank_in) { err = "rank_out must be in [1, rank_in]"; return REARR_EINVAL; }
    if (!dims || !order || !base || !range) { err = "dims, order, base and range must not be NULL"; return REARR_EINVAL; }
    bool kept[kMaxRank] = {false};
    for (int i = 0; i < rank_out; ++i) {
        const int a = order[i];
        if (a < 0 || a >= rank_in || kept[a]) { err = "order must list distinct input axes"; return REARR_EINVAL; }
        kept[a] = true;
    }
    uint64_t total = 1, in_total = 1;
    for (int a = 0; a < rank_in; ++a) {
        if (dims[a] < 0 || base[a] < 0) { err = "dims and base must be >= 0"; return REARR_EINVAL; }
        if (kept[a]) {
            if (range[a] < 0 || base[a] + range[a] > dims[a]) { err = "a kept axis range leaves the input"; return REARR_EINVAL; }
            if (mul_overflows(total, uint64_t(range[a]), total)) { err = "element count overflows"; return REARR_EINVAL; }
        } else if (base[a] >= dims[a]) {
            err = "a dropped axis base index is out of range";
            return REARR_EINVAL;
        }
        if (mul_overflows(in_total, uint64_t(dims[a]), in_total)) { err = "element count overflows"; return REARR_EINVAL; }
    }
    uint64_t bytes, in_bytes;
    if (mul_overflows(total, elem_bytes, bytes) || mul_overflows(in_total, elem_bytes, in_bytes) ||
        in_bytes > (uint64_t(1) << 62)) {
        err = "byte count overflows";
        return REARR_EINVAL;
    }
    if (total == 0) {
        pl.info.kind = REARR_KIND_NOOP;
        pl.op.units = 0;
        return REARR_OK;
    }
    if (!dst || !src) { err = "dst and src must not be NULL"; return REARR_EINVAL; }
    if (ranges_overlap(uintptr_t(dst), bytes, uintptr_t(src), in_bytes)) {
        err = "dst overlaps src";
        return REARR_EINVAL;
    }
    int64_t s[kMaxRank];
    s[rank_in - 1] = int64_t(elem_bytes);
    for (int a = rank_in - 2; a >= 0; --a) s[a] = s[a + 1] * dims[a + 1];
    int64_t off = 0;
    for (int a = 0; a < rank_in; ++a) off += base[a] * s[a];
    std::vector<Axis> ax;
    for (int i = 0; i < rank_out; ++i) ax.push_back(Axis{range[order[i]], s[order[i]]});
    return plan_axes(dst, static_cast<const char *>(src) + off, elem_bytes, ax, total, pl, err);
}

rearr_status plan_reorder(void *dst, const void *src, const uint32_t *idx, size_t n, size_t elem_bytes,
                          OpDesc &op, std::string &err, int idx_bytes, bool scatter)
{
    std::memset(&op, 0, sizeof(op));
    if (elem_bytes == 0) { err = "elem_bytes must be >= 1"; return REARR_EINVAL; }
    uint64_t bytes;
    if (mul_overflows(n, elem_bytes, bytes) || bytes > (uint64_t(1) << 62)) {
        err = "byte count overflows";
        return REARR_EINVAL;
    }
    if (idx_bytes == 4 && n > 0xFFFFFFFFull + 1) { err = "n exceeds the uint32 index range"; return REARR_EINVAL; }
    if (n == 0) { op.units = 0; return REARR_OK; }
    if (!dst || !src || !idx) { err = "dst, src and idx must not be NULL"; return REARR_EINVAL; }
    const uintptr_t da = uintptr_t(dst), sa = uintptr_t(src), ia = uintptr_t(idx);
    if (ranges_overlap(da, bytes, sa, bytes) || ranges_overlap(da, bytes, ia, uint64_t(n) * idx_bytes)) {
        err = "dst overlaps src or idx";
        return REARR_EINVAL;
    }
    if (ia % uintptr_t(idx_bytes) != 0) { err = "idx must be aligned to its index size"; return REARR_EINVAL; }
    const int W = pow2_align(da, sa, elem_bytes);
    op.cls = OC_GATHER;
    op.word = uint32_t(W);
    GatherDesc &g = op.gather;
    g.dst = static_cast<char *>(dst);
    g.src = static_cast<const char *>(src);
    g.idx = idx;
    g.n = n;
    g.c = uint32_t(elem_bytes / W);
    g.idx64 = idx_bytes == 8 ? 1u : 0u;
    g.scatter = scatter ? 1u : 0u;
    // the contiguous side (dst of a gather, src of a scatter) in groups of 4
    const uintptr_t contiguous = scatter ? sa : da;
    g.vec = (g.c == 1 && idx_bytes == 4 && ia % 16 == 0 && contiguous % uint64_t(std::min(16, 4 * W)) == 0) ? 1u : 0u;
    g.unit_elems = g.vec ? uint32_t(kThreads) * 32 : uint32_t(kThreads) * 16;
    op.units = (uint64_t(n) + g.unit_elems - 1) / g.unit_elems;
    // Sources much larger than the L2 go through the bucketed passes (which
    // fall back to this direct gather on the device if the indices turn out
    // to be local).
    // (64-bit indices too: every valid one is < n < 2^32)
    const bool l2_ok = g.vec || (g.c == 1 && idx_bytes == 8 && contiguous % uint64_t(std::min(16, 4 * W)) == 0);
    g.l2 = (l2_ok && (W == 4 || W == 8 || W == 16) && bytes >= kReorderL2MinBytes && n <= 0xFFFFFFFFull) ? 1u : 0u;
    return REARR_OK;
}

rearr_status plan_interlace(bool inter, char *interlaced, char *const *planes, int k, size_t n,
                            size_t elem_bytes, InterlacePlan &pl, std::string &err)
{
    std::memset(&pl.op, 0, sizeof(pl.op));
    pl.planes.clear();
    if (elem_bytes == 0) { err = "elem_bytes must be >= 1"; return REARR_EINVAL; }
    if (k < 1 || k > kMaxK) { err = "k must be in [1, 256]"; return REARR_EINVAL; }
    if (!planes) { err = "the plane pointer array must not be NULL"; return REARR_EINVAL; }
    uint64_t pbytes, ibytes;
    if (mul_overflows(n, elem_bytes, pbytes) || mul_overflows(pbytes, uint64_t(k), ibytes) ||
        ibytes > (uint64_t(1) << 62)) {
        err = "byte count overflows";
        return REARR_EINVAL;
    }
    if (n == 0) { pl.op.units = 0; return REARR_OK; }
    if (!interlaced) { err = "the interlaced array pointer must not be NULL"; return REARR_EINVAL; }
    uint64_t align_or = uintptr_t(interlaced);
    for (int j = 0; j < k; ++j) {
        if (!planes[j]) { err = "a plane pointer is NULL"; return REARR_EINVAL; }
        if (ranges_overlap(uintptr_t(planes[j]), pbytes, uintptr_t(interlaced), ibytes)) {
            err = "a plane overlaps the interlaced array";
            return REARR_EINVAL;
        }
        align_or |= uintptr_t(planes[j]);
        pl.planes.push_back(planes[j]);
    }
    if (!inter) {  // de-interlace writes the planes: they must not overlap each other
        std::vector<std::pair<uintptr_t, int>> order;
        for (int j = 0; j < k; ++j) order.push_back({uintptr_t(planes[j]), j});
        std::sort(order.begin(), order.end());
        for (int j = 1; j < k; ++j)
            if (order[j - 1].first + pbytes > order[j].first) {
                err = "destination planes overlap";
                return REARR_EINVAL;
            }
    }
    OpDesc &op = pl.op;
    InterlaceDesc &d = op.inter;
    op.cls = inter ? OC_INTERLACE : OC_DEINTERLACE;
    d.inter = interlaced;
    for (int j = 0; j < kInlineK; ++j) d.planes[j] = j < k ? planes[j] : nullptr;
    d.planes_dev = nullptr;
    d.n = n;
    d.k = uint32_t(k);
    d.elem_bytes = uint32_t(elem_bytes);
    const bool pow2e = elem_bytes == 1 || elem_bytes == 2 || elem_bytes == 4 || elem_bytes == 8 ||
                       elem_bytes == 16;
    d.fast = (pow2e && k <= 8 && align_or % 16 == 0) ? 1u : 0u;
    if (d.fast) {
        const uint64_t groups = uint64_t(n) * elem_bytes / 16;
        op.word = uint32_t(elem_bytes);
        d.c = 1;
        d.unit_groups = uint64_t(kThreads) * 4;
        op.units = std::max<uint64_t>(1, (groups + d.unit_groups - 1) / d.unit_groups);
    } else {
        const int W = pow2_align(align_or, elem_bytes);
        op.word = uint32_t(W);
        d.c = uint32_t(elem_bytes / W);
        const uint64_t kc = uint64_t(k) * d.c;
        if (kc > 0xFFFFFFFFull) { err = "k * elem_bytes too large"; return REARR_EINVAL; }
        d.unit_groups = std::max<uint64_t>(1, 8192 / kc);
        d.kc_div = make_fastdiv(uint32_t(kc));
        d.c_div = make_fastdiv(d.c);
        op.units = (uint64_t(n) + d.unit_groups - 1) / d.unit_groups;
    }
    return REARR_OK;
}

void tile_to_single_width(OpDesc &op)
{
    if (op.cls != OC_TILE) return;
    TileDesc &t = op.tile;
    const uint32_t v = t.variant;
    const int tbytes = int((v >> 22) & 0xFu) * 8192;
    if (tbytes <= kTileBytes) return;
    const int E = int(v & 0x3Fu), vin = int((v >> 6) & 0x3Fu), vout = int((v >> 12) & 0x3Fu);
    const int rowb = int((v >> 18) & 0xFu) * 128;
    t.TB = uint32_t(kTileBytes / rowb);
    t.variant = tile_variant(E, vin, vout, rowb, kTileBytes);
    uint64_t batch = 1;
    for (int i = 0; i < t.nb; ++i) batch *= t.bdiv[i].d;
    const uint64_t ta_tiles = t.ta_div.d;
    const uint64_t tb_tiles = (uint64_t(t.DB) + t.TB - 1) / t.TB;
    t.tb_div = make_fastdiv(uint32_t(tb_tiles));
    op.units = ta_tiles * tb_tiles * batch;
}

// Host run of a box descriptor over the cells the device body visits
// (box_body), checking what the body relies on: every load and store inside
// its buffer and aligned to its width, the cells of one load (store)
// consecutive in the input (output) and inside the partial axis' range, every
// shared-memory access inside the unit, and the odometer's slot equal to the
// one decomposed from the cell's index.  Shared memory is poisoned before
// each unit.
static bool box_emulate(const OpDesc &op, const char *src0, size_t src_bytes, char *dst0, size_t dst_bytes, int E,
                        std::string &err)
{
    const BoxDesc &d = op.box;
    std::vector<unsigned char> smem(kBoxBytes);
    auto in_cell = [&](uint32_t c, int64_t &off, uint32_t &kd) {
        off = 0;
        kd = 0;
        for (int i = 0; i < d.nu; ++i) {
            uint32_t dig;
            fdivmod(c, d.iext[i], c, dig);
            off += int64_t(dig) * d.iin[i];
            if (i == d.kin) kd = dig;
        }
    };
    auto out_cell = [&](uint32_t c, uint32_t *dig, uint32_t &sm, int64_t &off, uint32_t &kd) {
        sm = 0;
        off = 0;
        kd = 0;
        for (int i = 0; i < d.nu; ++i) {
            fdivmod(c, d.oext[i], c, dig[i]);
            sm += dig[i] * d.osm[i];
            off += int64_t(dig[i]) * d.oout[i];
            if (i == d.kout) kd = dig[i];
        }
    };
    if (uint64_t(d.cells) * E > uint64_t(kBoxBytes)) { err = "box unit larger than its shared memory"; return false; }
    for (uint64_t unit = 0; unit < op.units; ++unit) {
        std::memset(smem.data(), 0xCD, smem.size());
        uint32_t q = uint32_t(unit), keff = d.K;
        int64_t bin = 0, bout = 0;
        for (int i = d.no - 1; i >= 0; --i) {
            uint32_t dig;
            fdivmod(q, d.udiv[i], q, dig);
            bin += int64_t(dig) * d.uin[i];
            bout += int64_t(dig) * d.uout[i];
            if (i == d.kunit) keff = std::min(d.K, d.kfull - dig * d.K);
        }
        const uint32_t vin = keff < d.K ? uint32_t(E) : d.vin, vout = keff < d.K ? uint32_t(E) : d.vout;
        for (uint32_t x = 0; x < d.cells * uint32_t(E); x += vin) {
            int64_t off;
            uint32_t kd;
            in_cell(x / E, off, kd);
            if (kd >= keff) continue;
            const char *g = d.src + bin + off;
            if (uintptr_t(g) % vin) { err = "box load misaligned"; return false; }
            if (g < src0 || g + vin > src0 + src_bytes) { err = "box load outside the source"; return false; }
            for (uint32_t k = 1; k < vin / uint32_t(E); ++k) {
                int64_t o2;
                uint32_t k2;
                in_cell(x / E + k, o2, k2);
                if (o2 != off + int64_t(k) * E || k2 >= keff) { err = "box load spans two runs"; return false; }
            }
            std::memcpy(&smem[x], g, vin);
        }
        const uint32_t V = vout / uint32_t(E);
        for (uint32_t y = 0; y < d.cells; y += V) {
            uint32_t dig[kMaxBoxAxes], sm, kd;
            int64_t off;
            out_cell(y, dig, sm, off, kd);
            if (kd >= keff) continue;
            char *g = d.dst + bout + off;
            if (uintptr_t(g) % vout) { err = "box store misaligned"; return false; }
            if (g < dst0 || g + vout > dst0 + dst_bytes) { err = "box store outside the destination"; return false; }
            for (uint32_t k = 0; k < V; ++k) {
                uint32_t dig2[kMaxBoxAxes], sm2, kd2;
                int64_t off2;
                out_cell(y + k, dig2, sm2, off2, kd2);
                if (sm2 != sm || off2 != off + int64_t(k) * E || kd2 >= keff) { err = "box store spans two runs"; return false; }
                if (uint64_t(sm) + E > uint64_t(d.cells) * E) { err = "box slot outside the unit"; return false; }
                std::memcpy(g + k * E, &smem[sm], E);
                for (int i = 0; i < d.nu; ++i) {  // the device body's odometer step
                    sm += d.osm[i];
                    if (++dig[i] < d.oext[i].d) break;
                    sm -= d.oext[i].d * d.osm[i];
                    dig[i] = 0;
                }
            }
        }
    }
    return true;
}

// Box plans of pseudo-random permutes (ranks 2-6, extents up to a few
// thousand, cells of 1-16 bytes, aligned and unaligned pointers) run on the
// host by box_emulate and compared with the permute written out directly.
static bool selftest_box(std::string &err)
{
    uint64_t x = 0x2545F4914F6CDD1Dull;
    auto rnd = [&](uint64_t n) {
        x ^= x << 13; x ^= x >> 7; x ^= x << 17;
        return x % n;
    };
    int boxes = 0, partial = 0;
    for (int t = 0; t < 2000 && boxes < 300; ++t) {
        const int rank = 2 + int(rnd(5));
        const int E = 1 << rnd(5);
        int64_t dims[kMaxRank];
        uint64_t total = 1;
        for (int i = 0; i < rank; ++i) {
            dims[i] = rnd(4) == 0 ? 1 + int64_t(rnd(3000)) : 1 + int64_t(rnd(rnd(2) ? 12 : 60));
            total *= uint64_t(dims[i]);
        }
        if (total > (uint64_t(1) << 17) || total < 2) continue;
        int perm[kMaxRank];
        for (int i = 0; i < rank; ++i) perm[i] = i;
        for (int i = rank - 1; i > 0; --i) std::swap(perm[i], perm[rnd(uint64_t(i) + 1)]);
        const size_t bytes = size_t(total) * E;
        const int so = rnd(3) == 0 ? E : 0, dof = rnd(3) == 0 ? E : 0;
        std::vector<char> sbuf(bytes + 64), dbuf(bytes + 64), want(bytes);
        char *src = sbuf.data() + ((16 - uintptr_t(sbuf.data()) % 16) % 16) + so;
        char *dst = dbuf.data() + ((16 - uintptr_t(dbuf.data()) % 16) % 16) + dof;
        for (size_t i = 0; i < bytes; ++i) src[i] = char(rnd(256));
        // the permute written out: output cell o (row-major over dims[perm])
        int64_t s[kMaxRank];
        s[rank - 1] = E;
        for (int i = rank - 2; i >= 0; --i) s[i] = s[i + 1] * dims[i + 1];
        for (uint64_t o = 0; o < total; ++o) {
            uint64_t r = o;
            int64_t in = 0;
            for (int i = rank - 1; i >= 0; --i) {
                const int64_t ext = dims[perm[i]];
                in += int64_t(r % uint64_t(ext)) * s[perm[i]];
                r /= uint64_t(ext);
            }
            std::memcpy(&want[o * E], src + in, E);
        }
        // canonical axes as plan_axes forms them
        std::vector<Axis> ax;
        for (int i = 0; i < rank; ++i) {
            const Axis cur{dims[perm[i]], s[perm[i]]};
            if (cur.extent == 1) continue;
            if (!ax.empty() && ax.back().stride == cur.stride * cur.extent) {
                ax.back().extent *= cur.extent;
                ax.back().stride = cur.stride;
            } else {
                ax.push_back(cur);
            }
        }
        if (ax.size() < 2 || ax.back().stride == E) continue;  // a copy or an unmoved inner axis
        bool has_a = false;
        for (const Axis &a : ax) has_a |= a.stride == E;
        if (!has_a) continue;
        OpDesc op;
        std::memset(&op, 0, sizeof(op));
        rearr_permute_info info;
        std::memset(&info, 0, sizeof(info));
        if (!plan_box(ax, E, uintptr_t(dst), uintptr_t(src), dst, src, op, info)) continue;
        ++boxes;
        partial += op.box.kunit >= 0;
        std::memset(dst, 0, bytes);
        if (!box_emulate(op, src, bytes, dst, bytes, E, err)) return false;
        if (std::memcmp(dst, want.data(), bytes) != 0) {
            char buf[160];
            std::snprintf(buf, sizeof buf, "box plan of a rank-%d permute of %d-byte cells differs from the permute",
                          rank, E);
            err = buf;
            return false;
        }
    }
    if (boxes < 100 || partial < 10) {
        char buf[96];
        std::snprintf(buf, sizeof buf, "box self-test planned only %d boxes (%d partial)", boxes, partial);
        err = buf;
        return false;
    }
    return true;
}

bool selftest_host(std::string &err)
{
    // Fast division against the hardware divide on divisors and dividends
    // near powers of two, small values and pseudo-random values.
    std::vector<uint32_t> ds, ns;
    for (uint32_t v = 1; v < 300; ++v) ds.push_back(v);
    for (int b = 1; b < 32; ++b) {
        const uint32_t p = uint32_t(1) << b;
        ds.push_back(p - 1); ds.push_back(p); ds.push_back(p + 1);
    }
    ds.push_back(0xFFFFFFFFu); ds.push_back(0xFFFFFFFEu); ds.push_back(0x80000001u);
    uint64_t x = 0x9E3779B97F4A7C15ull;
    for (int i = 0; i < 200; ++i) {
        x ^= x << 13; x ^= x >> 7; x ^= x << 17;
        ds.push_back(uint32_t(x) | 1u);
        ds.push_back(uint32_t(x >> 40) + 1u);
        ns.push_back(uint32_t(x >> 3));
    }
    for (uint32_t v = 0; v < 1000; ++v) ns.push_back(v);
    for (int b = 1; b < 32; ++b) {
        const uint32_t p = uint32_t(1) << b;
        ns.push_back(p - 1); ns.push_back(p); ns.push_back(p + 1);
    }
    ns.push_back(0xFFFFFFFFu); ns.push_back(0xFFFFFFFEu);
    for (uint32_t d : ds) {
        const FastDiv f = make_fastdiv(d);
        for (uint32_t n : ns) {
            uint32_t q, r;
            fdivmod(n, f, q, r);
            if (q != n / d || r != n % d) {
                char buf[128];
                std::snprintf(buf, sizeof buf, "fastdiv %u / %u gave %u r %u", n, d, q, r);
                err = buf;
                return false;
            }
        }
        // every multiple boundary of small quotients
        for (uint64_t m = 1; m < 5; ++m) {
            const uint64_t n = m * d;
            if (n > 0xFFFFFFFFull) break;
            for (int off = -1; off <= 1; ++off) {
                const uint64_t nn = n + off;
                if (nn > 0xFFFFFFFFull) continue;
                uint32_t q, r;
                fdivmod(uint32_t(nn), f, q, r);
                if (q != uint32_t(nn / d) || r != uint32_t(nn % d)) { err = "fastdiv boundary"; return false; }
            }
        }
    }
    if (pow2_align(0) != 16 || pow2_align(12) != 4 || pow2_align(1024, 6) != 2 || pow2_align(3) != 1) {
        err = "pow2_align";
        return false;
    }
    return selftest_box(err);
}

}  // namespace rearr
