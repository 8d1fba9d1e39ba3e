// tuning.cpp -- tuning table of librearr.  The defaults can be replaced by a
// table written by the project's autotuner (paper_1011_3583_gb300/autotune.py):
// the file named by the REARR_TUNE_TABLE environment variable is read on first
// use, and rearr_tuning_load swaps in another file at run time.  Lines:
//   min_grab <v> | max_grab <v> | grabs_per_cta <v>
//   thin_tile_bytes <v> | thin_tile_cells <v> | thin_l2_bytes <v>
//   runs_mirror_bytes <v>   (1: never; runs of at most v bytes in input order)
//   runs_tile_max_bytes <v> (runs shorter than v bytes on a transpose plane
//                            are copied in blocks of cells; 1: never)
//   runs_tile_side_bytes <v> | runs_tile_cells <v>  (a block side holds
//                            v / cell cells, at least runs_tile_cells)
//   tile_vector_bytes <v>   (4: fast tiles load and store at most 4 bytes per
//                            access; 16: the widest the alignment allows)
//   double_tile_min_bytes <v> (32 KB tiles only for ops of at least v bytes)
//   wide_bytes <v>          (fast-tile plane sides shorter than v bytes are
//                            widened over the axis that continues them; 1: never)
//   reorder_smem_buckets <v> (bucket bound of the shared-memory scatter; 1: never)
//   box_min_run_bytes <v>   (thin planes run as staged boxes when both runs of
//                            the box reach v bytes, else as strided copies;
//                            a v above 16 KB: never)
//   box_run_bytes <v>       (a box stops growing once both runs reach v bytes
//                            and it holds half a tile)
//   box_max_cell_bytes <v>  (boxes only for cells of at most v bytes; 0: never)
//   rowb <E> <da_lo> <da_hi> <db_lo> <db_hi> <rowb> [<tile bytes> [<wide>]]
//                           (wide 1: the rule applies to widened planes, keyed
//                            by their extents before widening; 0: to the others)
// ("#" starts a comment line).  Plans compiled after a load use the new table.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/librearr.h"
#include "tuning.h"

namespace rearr {

rearr_status fail(rearr_status st, const std::string &msg);

namespace {

struct RowbRule {
    int E;
    int64_t da_lo, da_hi, db_lo, db_hi;
    int rowb;
    int tbytes;
    int wide;
};

struct Table {
    BatchTuning batch;
    ThinTuning thin;
    uint64_t runs_mirror_bytes = 0;
    uint64_t wide_bytes = 512;
    uint64_t double_tile_min_bytes = uint64_t(64) << 20;
    uint64_t runs_tile_max_bytes = 1024;
    uint64_t runs_tile_cells = 8;
    uint64_t runs_tile_side_bytes = 2048;
    uint64_t tile_vector_bytes = 16;
    uint64_t reorder_smem_buckets = uint64_t(1) << 22;
    uint64_t box_min_run_bytes = 16;
    uint64_t box_run_bytes = 512;
    uint64_t box_max_cell_bytes = 0;
    std::vector<RowbRule> rowb;
};

std::shared_ptr<const Table> parse(const char *path)
{
    FILE *f = std::fopen(path, "r");
    if (!f) return nullptr;
    auto t = std::make_shared<Table>();
    char line[256];
    while (std::fgets(line, sizeof line, f)) {
        char key[32];
        unsigned long v;
        RowbRule r;
        long long a, b, c, d;
        if (line[0] == '#') continue;
        int tb = 16384, wide = 0;
        const int got = std::sscanf(line, "rowb %d %lld %lld %lld %lld %d %d %d", &r.E, &a, &b, &c, &d, &r.rowb, &tb,
                                    &wide);
        if (got >= 6) {
            r.da_lo = a; r.da_hi = b; r.db_lo = c; r.db_hi = d;
            r.tbytes = got >= 7 ? tb : 16384;
            r.wide = got >= 8 ? wide : 0;
            const bool ok_rowb = r.rowb == 128 || r.rowb == 256 || (r.rowb == 512 && r.E != 1);
            const bool ok_tb = r.tbytes == 16384 || (r.tbytes == 8192 && r.rowb == 128) ||
                               (r.tbytes == 32768 && double_tile_ok(r.E, r.rowb));
            if (ok_rowb && ok_tb && (r.wide == 0 || r.wide == 1)) t->rowb.push_back(r);
        } else if (std::sscanf(line, "%31s %lu", key, &v) == 2 && !std::strcmp(key, "box_max_cell_bytes")) {
            t->box_max_cell_bytes = v;
        } else if (std::sscanf(line, "%31s %lu", key, &v) == 2 && v >= 1) {
            if (!std::strcmp(key, "min_grab")) t->batch.min_grab = uint32_t(v);
            else if (!std::strcmp(key, "max_grab")) t->batch.max_grab = uint32_t(v);
            else if (!std::strcmp(key, "grabs_per_cta")) t->batch.grabs_per_cta = uint32_t(v);
            else if (!std::strcmp(key, "thin_tile_bytes")) t->thin.tile_bytes = v;
            else if (!std::strcmp(key, "thin_tile_cells")) t->thin.tile_cells = v;
            else if (!std::strcmp(key, "thin_l2_bytes")) t->thin.l2_bytes = v;
            else if (!std::strcmp(key, "runs_mirror_bytes")) t->runs_mirror_bytes = v;
            else if (!std::strcmp(key, "wide_bytes")) t->wide_bytes = v;
            else if (!std::strcmp(key, "double_tile_min_bytes")) t->double_tile_min_bytes = v;
            else if (!std::strcmp(key, "runs_tile_max_bytes")) t->runs_tile_max_bytes = v;
            else if (!std::strcmp(key, "runs_tile_cells")) t->runs_tile_cells = v;
            else if (!std::strcmp(key, "runs_tile_side_bytes")) t->runs_tile_side_bytes = v;
            else if (!std::strcmp(key, "tile_vector_bytes")) t->tile_vector_bytes = v < 16 ? 4 : 16;
            else if (!std::strcmp(key, "reorder_smem_buckets")) t->reorder_smem_buckets = v;
            else if (!std::strcmp(key, "box_min_run_bytes")) t->box_min_run_bytes = v;
            else if (!std::strcmp(key, "box_run_bytes")) t->box_run_bytes = v;
        }
    }
    std::fclose(f);
    if (t->batch.max_grab < t->batch.min_grab) t->batch.max_grab = t->batch.min_grab;
    return t;
}

std::mutex g_mu;
std::shared_ptr<const Table> g_table;

std::shared_ptr<const Table> current()
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_table) {
        const char *path = std::getenv("REARR_TUNE_TABLE");
        if (path && *path) g_table = parse(path);
        if (!g_table) g_table = std::make_shared<Table>();
    }
    return g_table;
}

}  // namespace

BatchTuning batch_tuning() { return current()->batch; }

ThinTuning thin_tuning() { return current()->thin; }

uint64_t runs_mirror_max_bytes() { return current()->runs_mirror_bytes; }

uint64_t wide_min_bytes() { return current()->wide_bytes; }

uint64_t double_tile_min_bytes() { return current()->double_tile_min_bytes; }

uint64_t runs_tile_max_bytes() { return current()->runs_tile_max_bytes; }

uint64_t runs_tile_cells() { return current()->runs_tile_cells; }

uint64_t runs_tile_side_bytes() { return current()->runs_tile_side_bytes; }

int tile_vector_bytes() { return int(current()->tile_vector_bytes); }

uint64_t reorder_smem_max_buckets() { return current()->reorder_smem_buckets; }

uint64_t box_min_run_bytes() { return current()->box_min_run_bytes; }

uint64_t box_run_bytes() { return current()->box_run_bytes; }

uint64_t box_max_cell_bytes() { return current()->box_max_cell_bytes; }

bool tuned_shape(int E, int64_t DA, int64_t DB, bool wide, TileShape &shape)
{
    const std::shared_ptr<const Table> t = current();
    for (const RowbRule &r : t->rowb)
        if (r.E == E && r.wide == int(wide) && DA >= r.da_lo && DA <= r.da_hi && DB >= r.db_lo && DB <= r.db_hi) {
            shape = {r.rowb, r.tbytes};
            return true;
        }
    return false;
}

}  // namespace rearr

extern "C" rearr_status rearr_tuning_load(const char *path)
{
    std::shared_ptr<const rearr::Table> t;
    if (path && *path) {
        t = rearr::parse(path);
        if (!t) return rearr::fail(REARR_EINVAL, std::string("rearr_tuning_load: cannot read ") + path);
    } else {
        t = std::make_shared<rearr::Table>();
    }
    std::lock_guard<std::mutex> lock(rearr::g_mu);
    rearr::g_table = t;
    return REARR_OK;
}
