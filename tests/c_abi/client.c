/* A plain C client of the librearr C ABI: only the headers under include/ and
 * the shared library.  It makes the host-only calls (plan descriptions, the
 * distributed plan, argument validation, the host self-test) and prints one
 * line per call for tests/test_c_abi.py; nothing here touches a GPU. */
#include <stdint.h>
#include <stdio.h>

#include "librearr.h"
#include "librearr_dist.h"
#include "librearr_pipeline.h"

int main(void)
{
    /* the 512^3 fp32 reversal: one fast-tile plan over the (0, 2) plane */
    const int64_t dims[3] = {512, 512, 512};
    const int perm[3] = {2, 1, 0};
    rearr_permute_info info;
    rearr_status st = rearr_permute_describe(4, 3, dims, perm, 0, 0, &info);
    printf("describe %s kind %d rank %d cell %lld word %d tiles %lld\n", rearr_status_str(st), info.kind, info.rank,
           (long long)info.cell_bytes, info.word_bytes, (long long)info.n_tiles);

    /* a repeated axis is rejected before any CUDA call */
    const int bad[3] = {0, 0, 1};
    st = rearr_permute((void *)0, (const void *)0, 4, 3, dims, bad, (rearr_stream_t)0);
    printf("bad_perm %s\n", rearr_status_str(st));

    /* the permute of an 8 x 6 x 4 array sharded over 2 ranks */
    const int64_t gd[3] = {8, 6, 4};
    const int gp[3] = {2, 0, 1};
    rearr_dist_plan plan;
    st = rearr_dist_permute_plan(4, 3, gd, gp, 2, &plan);
    printf("dist %s exchange %d slab %llu piece %llu pack", rearr_status_str(st), plan.exchange,
           (unsigned long long)plan.slab_bytes, (unsigned long long)plan.piece_bytes);
    for (int i = 0; i < plan.pack_rank; ++i) printf(" %lld/%d", (long long)plan.pack_dims[i], plan.pack_perm[i]);
    printf(" unpack");
    for (int i = 0; i < plan.unpack_rank; ++i) printf(" %lld/%d", (long long)plan.unpack_dims[i], plan.unpack_perm[i]);
    printf("\n");

    /* the order-1 finite-difference Laplacian on a 4096^2 grid */
    const int dy[5] = {0, -1, 1, 0, 0}, dx[5] = {0, 0, 0, -1, 1};
    const float w[5] = {-4.0f, 1.0f, 1.0f, 1.0f, 1.0f};
    rearr_stencil_info si;
    st = rearr_stencil2d_describe(4096, 4096, 5, dy, dx, w, REARR_STENCIL_ZERO, 0, 0, &si);
    printf("stencil %s shape %d radius %d\n", rearr_status_str(st), si.shape, si.radius);

    /* a random reorder of 2^28 fp32: the bucketed passes, shared-memory scatter */
    rearr_reorder_info ri;
    st = rearr_reorder_describe((size_t)1 << 28, 4, 4, 0, 0, 0, 0, &ri);
    printf("reorder %s form %d chunks %u %u\n", rearr_status_str(st), ri.form, ri.bucket_chunks, ri.dest_chunks);

    /* a box that drops the input's fastest axis: one strided gather per cell */
    const int64_t bd[3] = {40, 50, 60}, bb[3] = {3, 7, 11}, br[3] = {30, 40, 1};
    const int bo[2] = {1, 0};
    rearr_permute_info ni;
    st = rearr_reorder_nm_describe(4, 3, bd, 2, bo, bb, br, 0, 0, &ni);
    printf("nm %s kind %d\n", rearr_status_str(st), ni.kind);

    /* a pipeline of zero slots is rejected before any CUDA call */
    rearr_pipeline *pipe = (rearr_pipeline *)0;
    st = rearr_pipeline_create(1 << 20, 0, &pipe);
    printf("pipeline %s\n", rearr_status_str(st));

    st = rearr_selftest_host();
    printf("selftest %s\n", rearr_status_str(st));
    return 0;
}
