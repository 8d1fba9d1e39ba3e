// dist.cpp -- the distributed N-D permute of include/librearr_dist.h: host
// planning of the pack and unpack permutes (arXiv:1011.3583 Sec. III.B
// permute, on an array sharded along its slowest axis).
//
// With P ranks, input dims D (D[0] slowest) and q = perm[0]: rank r holds
// input rows [r D[0]/P, (r+1) D[0]/P) and must produce output rows
// [r D[q]/P, (r+1) D[q]/P) of output axis 0, i.e. input axis q restricted to
// that range.  Pack splits the local slab's axis q into (P, D[q]/P) and moves
// the P part to the front, followed by the output order: piece j (contiguous)
// is the part of rank j's output slab that this rank's input rows cover, in
// output order, with output axis a = perm^-1(0) cut to D[0]/P rows.  After
// the all-to-all, piece j on rank r comes from rank j; unpack moves the
// source-rank axis next to (slower than) output axis a, which makes it the
// high part of that axis: output row a = j * D[0]/P + local row.
#include <cstring>
#include <string>

#include "../../include/librearr.h"
#include "../../include/librearr_dist.h"

namespace rearr {
rearr_status fail(rearr_status st, const std::string &msg);
}

using namespace rearr;

extern "C" {

rearr_status rearr_dist_permute_plan(size_t elem_bytes, int rank, const int64_t *dims, const int *perm,
                                     int nranks, rearr_dist_plan *plan)
{
    const char *who = "rearr_dist_permute_plan: ";
    if (!plan || !dims || !perm) return fail(REARR_EINVAL, std::string(who) + "null argument");
    if (elem_bytes == 0) return fail(REARR_EINVAL, std::string(who) + "elem_bytes must be >= 1");
    if (rank < 1 || rank > REARR_MAX_RANK - 1) return fail(REARR_EINVAL, std::string(who) + "rank out of range");
    if (nranks < 1) return fail(REARR_EINVAL, std::string(who) + "nranks must be >= 1");
    bool seen[REARR_MAX_RANK] = {};
    for (int i = 0; i < rank; ++i) {
        if (dims[i] < 1) return fail(REARR_EINVAL, std::string(who) + "dims must be >= 1");
        if (perm[i] < 0 || perm[i] >= rank || seen[perm[i]])
            return fail(REARR_EINVAL, std::string(who) + "perm is not a permutation");
        seen[perm[i]] = true;
    }
    const int q = perm[0];
    const int64_t P = nranks;
    if (dims[0] % P || dims[q] % P)
        return fail(REARR_EINVAL, std::string(who) + "the sharded extents must be multiples of nranks");
    uint64_t total = 1;
    for (int i = 0; i < rank; ++i) {
        if (total > UINT64_MAX / uint64_t(dims[i])) return fail(REARR_EINVAL, std::string(who) + "array too large");
        total *= uint64_t(dims[i]);
    }
    if (total > UINT64_MAX / elem_bytes) return fail(REARR_EINVAL, std::string(who) + "array too large");
    rearr_dist_plan pl;
    std::memset(&pl, 0, sizeof pl);
    pl.nranks = nranks;
    pl.slab_bytes = total / uint64_t(P) * elem_bytes;
    int64_t L[REARR_MAX_RANK];  // local input slab
    for (int i = 0; i < rank; ++i) L[i] = dims[i];
    L[0] = dims[0] / P;
    if (q == 0) {
        // output axis 0 is input axis 0: the local slab permutes on its own
        pl.exchange = 0;
        pl.pack_rank = rank;
        for (int i = 0; i < rank; ++i) {
            pl.pack_dims[i] = L[i];
            pl.pack_perm[i] = perm[i];
        }
        *plan = pl;
        return REARR_OK;
    }
    pl.exchange = 1;
    pl.piece_bytes = pl.slab_bytes / uint64_t(P);
    // pack: local slab with axis q split into (P, D[q]/P): axes a < q keep
    // their index, q -> (q, q + 1), a > q -> a + 1
    auto split = [q](int a) { return a < q ? a : a + 1; };
    pl.pack_rank = rank + 1;
    for (int i = 0, k = 0; i < rank; ++i) {
        if (i == q) {
            pl.pack_dims[k++] = P;
            pl.pack_dims[k++] = L[q] / P;
        } else {
            pl.pack_dims[k++] = L[i];
        }
    }
    pl.pack_perm[0] = q;  // destination rank, slowest
    pl.pack_perm[1] = q + 1;
    for (int i = 1; i < rank; ++i) pl.pack_perm[i + 1] = split(perm[i]);
    // unpack: received pieces [source rank][output slab rows, output axis a
    // cut to D[0]/P]; the source rank moves to just before axis a
    int a = 0;
    while (perm[a] != 0) ++a;  // a >= 1 since perm[0] = q != 0
    pl.unpack_rank = rank + 1;
    pl.unpack_dims[0] = P;
    for (int i = 0; i < rank; ++i) pl.unpack_dims[i + 1] = i == 0 ? L[q] / P : i == a ? L[0] : dims[perm[i]];
    for (int i = 0, k = 0; i < rank; ++i) {
        if (i == a) pl.unpack_perm[k++] = 0;
        pl.unpack_perm[k++] = i + 1;
    }
    *plan = pl;
    return REARR_OK;
}

rearr_status rearr_dist_permute_pack(void *send, const void *in_slab, const rearr_dist_plan *plan,
                                     size_t elem_bytes, rearr_stream_t stream)
{
    if (!plan) return fail(REARR_EINVAL, "rearr_dist_permute_pack: null plan");
    return rearr_permute(send, in_slab, elem_bytes, plan->pack_rank, plan->pack_dims, plan->pack_perm, stream);
}

rearr_status rearr_dist_permute_unpack(void *out_slab, const void *recv, const rearr_dist_plan *plan,
                                       size_t elem_bytes, rearr_stream_t stream)
{
    if (!plan || !plan->exchange)
        return fail(REARR_EINVAL, "rearr_dist_permute_unpack: no plan, or a plan without an exchange");
    return rearr_permute(out_slab, recv, elem_bytes, plan->unpack_rank, plan->unpack_dims, plan->unpack_perm,
                         stream);
}

}  // extern "C"
