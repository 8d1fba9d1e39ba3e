// tuning.cpp -- tuning table of the batched kernel.  The defaults can be
// replaced at run time by a table written by the project's autotuner, named by
// the REARR_TUNE_TABLE environment variable: a text file of "key value" lines
// (min_grab, max_grab, grabs_per_cta).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "batch.h"

namespace rearr {

const BatchTuning &batch_tuning()
{
    static BatchTuning t;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *path = std::getenv("REARR_TUNE_TABLE");
        if (!path || !*path) return;
        FILE *f = std::fopen(path, "r");
        if (!f) return;
        char key[64];
        unsigned long v;
        while (std::fscanf(f, "%63s %lu", key, &v) == 2) {
            if (!std::strcmp(key, "min_grab") && v >= 1) t.min_grab = uint32_t(v);
            else if (!std::strcmp(key, "max_grab") && v >= 1) t.max_grab = uint32_t(v);
            else if (!std::strcmp(key, "grabs_per_cta") && v >= 1) t.grabs_per_cta = uint32_t(v);
        }
        std::fclose(f);
        if (t.max_grab < t.min_grab) t.max_grab = t.min_grab;
    });
    return t;
}

}  // namespace rearr
