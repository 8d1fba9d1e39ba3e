// tuning.cpp -- tuning table of librearr.  The defaults can be replaced at
// run time by a table written by the project's autotuner, named by the
// REARR_TUNE_TABLE environment variable.  The file holds lines of
//   min_grab <v> | max_grab <v> | grabs_per_cta <v>
//   rowb <E> <da_lo> <da_hi> <db_lo> <db_hi> <rowb>
// ("#" starts a comment line).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "tuning.h"

namespace rearr {

namespace {

struct RowbRule {
    int E;
    int64_t da_lo, da_hi, db_lo, db_hi;
    int rowb;
};

struct Table {
    BatchTuning batch;
    std::vector<RowbRule> rowb;
};

const Table &table()
{
    static Table t;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *path = std::getenv("REARR_TUNE_TABLE");
        if (!path || !*path) return;
        FILE *f = std::fopen(path, "r");
        if (!f) return;
        char line[256];
        while (std::fgets(line, sizeof line, f)) {
            char key[32];
            unsigned long v;
            RowbRule r;
            long long a, b, c, d;
            if (line[0] == '#') continue;
            if (std::sscanf(line, "rowb %d %lld %lld %lld %lld %d", &r.E, &a, &b, &c, &d, &r.rowb) == 6) {
                r.da_lo = a; r.da_hi = b; r.db_lo = c; r.db_hi = d;
                const bool ok_rowb = r.rowb == 128 || r.rowb == 256 || (r.rowb == 512 && r.E != 1);
                if (ok_rowb) t.rowb.push_back(r);
            } else if (std::sscanf(line, "%31s %lu", key, &v) == 2 && v >= 1) {
                if (!std::strcmp(key, "min_grab")) t.batch.min_grab = uint32_t(v);
                else if (!std::strcmp(key, "max_grab")) t.batch.max_grab = uint32_t(v);
                else if (!std::strcmp(key, "grabs_per_cta")) t.batch.grabs_per_cta = uint32_t(v);
            }
        }
        std::fclose(f);
        if (t.batch.max_grab < t.batch.min_grab) t.batch.max_grab = t.batch.min_grab;
    });
    return t;
}

}  // namespace

const BatchTuning &batch_tuning() { return table().batch; }

int tuned_rowb(int E, int64_t DA, int64_t DB)
{
    for (const RowbRule &r : table().rowb)
        if (r.E == E && DA >= r.da_lo && DA <= r.da_hi && DB >= r.db_lo && DB <= r.db_hi) return r.rowb;
    return 0;
}

}  // namespace rearr
