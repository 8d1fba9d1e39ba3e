// pipeline.cpp -- host-buffer pipeline of librearr (include/librearr_pipeline.h).
//
// Three streams per pipeline (uploads, kernels, downloads) and a ring of
// device staging slots.  For the op in slot s:
//   upload stream   : wait for slot s's previous download; copy inputs in;
//                     record in_ready[s]
//   kernel stream   : wait in_ready[s]; launch the op's kernel on the slot;
//                     record computed[s]
//   download stream : wait computed[s]; copy outputs out; record out_done[s]
// so consecutive ops overlap their uploads, kernels and downloads, and a slot
// is never overwritten while its previous op is still being read.  An upload
// that reads host memory an op still in flight writes also waits for that
// op's download, so an op may consume an earlier op's output.
//
// Direct ops.  With direct access on (the default where the GPU reaches host
// memory through the system's page tables, as over NVLink-C2C), a permute or
// (de-)interlace whose host buffers are page-locked and whose plan streams
// (copy, tiles, runs, boxes, interlace kernels) runs its kernel on the host
// buffers themselves: each byte crosses the host link once, as with the
// copies, but reads and writes share the link in both directions within one
// kernel instead of relying on the overlap of separate copies.  A direct op
// runs on the kernel stream after everything enqueued before it on the three
// streams, and everything enqueued after it waits for it, so host memory sees
// the ops in submission order whichever way each runs.
#include <cuda_runtime.h>

#include <cstring>
#include <functional>
#include <memory>
#include <string>
#include <vector>

#include "../../include/librearr_pipeline.h"
#include "launch.h"
#include "plan.h"
#include "stencil.h"

namespace rearr {
rearr_status fail(rearr_status st, const std::string &msg);
rearr_status cuda_fail(cudaError_t e, const char *what);
}  // namespace rearr

using namespace rearr;

struct rearr_pipeline {
    char *dev = nullptr;
    size_t slot_bytes = 0;
    int slots = 0;
    int next = 0;
    cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
    std::vector<cudaEvent_t> in_ready, computed, out_done;
    std::vector<bool> used;
    std::vector<std::vector<std::pair<uintptr_t, size_t>>> wrote;  // host ranges the slot's last op writes
    cudaEvent_t up_tail = nullptr, down_tail = nullptr, direct_done = nullptr;
    int direct = 0;
    cudaError_t broken = cudaSuccess;
    uint64_t ops = 0, h2d = 0, d2h = 0, direct_ops = 0;
};

namespace {

constexpr size_t kAlign = 256;

size_t round_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

struct HostRange {
    const void *host;
    size_t bytes;
};
struct HostOut {
    void *host;
    size_t bytes;
};

// Device addresses of an op's inputs and outputs inside one slot.
struct SlotLayout {
    std::vector<char *> in, out;
};

rearr_status layout(rearr_pipeline *p, int slot, const std::vector<HostRange> &ins,
                    const std::vector<HostOut> &outs, SlotLayout &lay, const char *who)
{
    size_t need = 0;
    for (const HostRange &r : ins) need += round_up(r.bytes);
    for (const HostOut &r : outs) need += round_up(r.bytes);
    if (need > p->slot_bytes)
        return fail(REARR_EINVAL, std::string(who) + ": op needs " + std::to_string(need) +
                                      " bytes of staging, a slot holds " + std::to_string(p->slot_bytes));
    char *at = p->dev + size_t(slot) * p->slot_bytes;
    for (const HostRange &r : ins) {
        lay.in.push_back(at);
        at += round_up(r.bytes);
    }
    for (const HostOut &r : outs) {
        lay.out.push_back(at);
        at += round_up(r.bytes);
    }
    return REARR_OK;
}

// Device-visible addresses of the ranges when every non-empty one starts and
// ends in page-locked host memory the device can address.
bool device_views(const std::vector<HostRange> &ins, const std::vector<HostOut> &outs, SlotLayout &lay)
{
    auto view = [](const void *h, size_t bytes, char *&d) {
        if (bytes == 0) {
            d = nullptr;
            return true;
        }
        cudaPointerAttributes a, b;
        if (cudaPointerGetAttributes(&a, h) != cudaSuccess ||
            cudaPointerGetAttributes(&b, static_cast<const char *>(h) + bytes - 1) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
            return false;
        d = static_cast<char *>(a.devicePointer);
        return static_cast<char *>(b.devicePointer) == d + bytes - 1;
    };
    for (const HostRange &r : ins) {
        char *d;
        if (!view(r.host, r.bytes, d)) return false;
        lay.in.push_back(d);
    }
    for (const HostOut &r : outs) {
        char *d;
        if (!view(r.host, r.bytes, d)) return false;
        lay.out.push_back(d);
    }
    return true;
}

// Plans whose kernels stream through their buffers (every byte read and
// written about once, in runs): the ones a direct op may run on host memory.
bool streams(uint32_t cls)
{
    return cls == OC_COPY || cls == OC_TILE || cls == OC_TILE_CELLS || cls == OC_RUNS || cls == OC_BOX ||
           cls == OC_INTERLACE || cls == OC_DEINTERLACE;
}

template <class Launch>
rearr_status run_op(rearr_pipeline *p, const char *who, const std::vector<HostRange> &ins,
                    const std::vector<HostOut> &outs, Launch &&launch)
{
    if (!p) return fail(REARR_EINVAL, std::string(who) + ": pipeline is NULL");
    if (p->broken != cudaSuccess) return cuda_fail(p->broken, who);
    for (const HostRange &r : ins)
        if (r.bytes && !r.host) return fail(REARR_EINVAL, std::string(who) + ": NULL host input");
    for (const HostOut &r : outs)
        if (r.bytes && !r.host) return fail(REARR_EINVAL, std::string(who) + ": NULL host output");
    if (p->direct) {
        SlotLayout dl;
        if (device_views(ins, outs, dl)) {
            std::string err;
            std::function<cudaError_t(cudaStream_t)> go;
            uint32_t cls = OC_COUNT;
            rearr_status st = launch(dl, go, err, cls);
            if (st != REARR_OK) return fail(st, std::string(who) + ": " + err);
            if (streams(cls)) {
                cudaError_t e = cudaEventRecord(p->up_tail, p->up);
                if (e == cudaSuccess) e = cudaEventRecord(p->down_tail, p->down);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(p->comp, p->up_tail, 0);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(p->comp, p->down_tail, 0);
                if (e == cudaSuccess) e = go(p->comp);
                if (e == cudaSuccess) e = cudaEventRecord(p->direct_done, p->comp);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(p->up, p->direct_done, 0);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(p->down, p->direct_done, 0);
                if (e != cudaSuccess) {
                    p->broken = e;
                    return cuda_fail(e, who);
                }
                p->ops += 1;
                p->direct_ops += 1;
                for (const HostRange &r : ins) p->h2d += r.bytes;
                for (const HostOut &r : outs) p->d2h += r.bytes;
                return REARR_OK;
            }
        }
    }
    const int s = p->next;
    SlotLayout lay;
    rearr_status st = layout(p, s, ins, outs, lay, who);
    if (st != REARR_OK) return st;
    // The op is planned (and validated) on the slot's device addresses before
    // anything is enqueued.
    std::string err;
    std::function<cudaError_t(cudaStream_t)> go;
    uint32_t cls = OC_COUNT;
    st = launch(lay, go, err, cls);
    if (st != REARR_OK) return fail(st, std::string(who) + ": " + err);

    cudaError_t e = cudaSuccess;
    if (p->used[s]) e = cudaStreamWaitEvent(p->up, p->out_done[s], 0);
    // an input that an earlier op still in flight writes: upload after that
    // op's download (ops older than the slot ring were waited for above)
    for (int o = 0; o < p->slots && e == cudaSuccess; ++o) {
        if (o == s || !p->used[o]) continue;
        bool hit = false;
        for (const HostRange &r : ins)
            for (const auto &w : p->wrote[o])
                hit |= r.bytes && uintptr_t(r.host) < w.first + w.second && w.first < uintptr_t(r.host) + r.bytes;
        if (hit) e = cudaStreamWaitEvent(p->up, p->out_done[o], 0);
    }
    for (size_t i = 0; i < ins.size() && e == cudaSuccess; ++i)
        if (ins[i].bytes) e = cudaMemcpyAsync(lay.in[i], ins[i].host, ins[i].bytes, cudaMemcpyHostToDevice, p->up);
    if (e == cudaSuccess) e = cudaEventRecord(p->in_ready[s], p->up);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->comp, p->in_ready[s], 0);
    if (e == cudaSuccess) e = go(p->comp);
    if (e == cudaSuccess) e = cudaEventRecord(p->computed[s], p->comp);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->down, p->computed[s], 0);
    for (size_t i = 0; i < outs.size() && e == cudaSuccess; ++i)
        if (outs[i].bytes)
            e = cudaMemcpyAsync(outs[i].host, lay.out[i], outs[i].bytes, cudaMemcpyDeviceToHost, p->down);
    if (e == cudaSuccess) e = cudaEventRecord(p->out_done[s], p->down);
    if (e != cudaSuccess) {
        p->broken = e;
        return cuda_fail(e, who);
    }
    p->used[s] = true;
    p->wrote[s].clear();
    for (const HostOut &r : outs)
        if (r.bytes) p->wrote[s].push_back({uintptr_t(r.host), r.bytes});
    p->next = (s + 1) % p->slots;
    p->ops += 1;
    for (const HostRange &r : ins) p->h2d += r.bytes;
    for (const HostOut &r : outs) p->d2h += r.bytes;
    return REARR_OK;
}

size_t product(int rank, const int64_t *dims)
{
    size_t n = 1;
    for (int i = 0; i < rank; ++i) n *= dims[i] < 0 ? 0 : size_t(dims[i]);
    return n;
}

// Gather / scatter with 4- or 8-byte indices.
rearr_status pipeline_indexed(rearr_pipeline *pipe, const char *who, void *dst, const void *src,
                              const void *idx, size_t n, size_t elem_bytes, int idx_bytes, bool scatter)
{
    return run_op(pipe, who, {{src, n * elem_bytes}, {idx, n * size_t(idx_bytes)}}, {{dst, n * elem_bytes}},
                  [&](const SlotLayout &l, std::function<cudaError_t(cudaStream_t)> &go, std::string &err, uint32_t &cls) {
                      auto op = std::make_shared<OpDesc>();
                      rearr_status st = plan_reorder(l.out[0], l.in[0], reinterpret_cast<const uint32_t *>(l.in[1]),
                                                     n, elem_bytes, *op, err, idx_bytes, scatter);
                      go = [op](cudaStream_t s) { return launch_single(*op, nullptr, s); };
                      return st;
                  });
}

}  // namespace

extern "C" {

rearr_status rearr_pipeline_create(size_t slot_bytes, int slots, rearr_pipeline **pipe)
{
    if (!pipe) return fail(REARR_EINVAL, "rearr_pipeline_create: pipe is NULL");
    *pipe = nullptr;
    if (slots < 1 || slots > 8) return fail(REARR_EINVAL, "rearr_pipeline_create: slots must be 1..8");
    if (slot_bytes == 0) return fail(REARR_EINVAL, "rearr_pipeline_create: slot_bytes is 0");
    auto *p = new rearr_pipeline;
    p->slot_bytes = round_up(slot_bytes);
    p->slots = slots;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&p->dev), p->slot_bytes * size_t(slots));
    if (e != cudaSuccess) {
        delete p;
        cudaGetLastError();
        return fail(REARR_ENOMEM, std::string("rearr_pipeline_create: cudaMalloc: ") + cudaGetErrorString(e));
    }
    for (cudaStream_t *s : {&p->up, &p->comp, &p->down})
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
    p->in_ready.assign(slots, nullptr);
    p->computed.assign(slots, nullptr);
    p->out_done.assign(slots, nullptr);
    p->used.assign(slots, false);
    p->wrote.assign(slots, {});
    for (int i = 0; i < slots && e == cudaSuccess; ++i)
        for (cudaEvent_t *ev : {&p->in_ready[i], &p->computed[i], &p->out_done[i]})
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    for (cudaEvent_t *ev : {&p->up_tail, &p->down_tail, &p->direct_done})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    // direct ops by default where the device uses the host's page tables
    // (coherent host access, as over NVLink-C2C)
    int dev = 0, ats = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ats, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev);
    p->direct = ats ? 1 : 0;
    if (e != cudaSuccess) {
        rearr_pipeline_destroy(p);
        return cuda_fail(e, "rearr_pipeline_create");
    }
    *pipe = p;
    return REARR_OK;
}

rearr_status rearr_pipeline_permute(rearr_pipeline *pipe, void *dst, const void *src, size_t elem_bytes, int rank,
                                    const int64_t *dims, const int *perm)
{
    const size_t bytes = (rank >= 1 && rank <= REARR_MAX_RANK && dims) ? product(rank, dims) * elem_bytes : 0;
    return run_op(pipe, "rearr_pipeline_permute", {{src, bytes}}, {{dst, bytes}},
                  [&](const SlotLayout &l, std::function<cudaError_t(cudaStream_t)> &go, std::string &err, uint32_t &cls) {
                      auto pl = std::make_shared<PermPlan>();
                      rearr_status st = plan_permute(l.out[0], l.in[0], elem_bytes, rank, dims, perm, *pl, err);
                      cls = pl->info.kind == REARR_KIND_NOOP ? uint32_t(OC_COPY) : pl->op.cls;
                      go = [pl](cudaStream_t s) { return launch_single(pl->op, nullptr, s); };
                      return st;
                  });
}

rearr_status rearr_pipeline_reorder(rearr_pipeline *pipe, void *dst, const void *src, const uint32_t *idx, size_t n,
                                    size_t elem_bytes)
{
    return run_op(pipe, "rearr_pipeline_reorder", {{src, n * elem_bytes}, {idx, n * sizeof(uint32_t)}},
                  {{dst, n * elem_bytes}},
                  [&](const SlotLayout &l, std::function<cudaError_t(cudaStream_t)> &go, std::string &err, uint32_t &cls) {
                      auto op = std::make_shared<OpDesc>();
                      rearr_status st = plan_reorder(l.out[0], l.in[0], reinterpret_cast<const uint32_t *>(l.in[1]),
                                                     n, elem_bytes, *op, err);
                      go = [op](cudaStream_t s) { return launch_single(*op, nullptr, s); };
                      return st;
                  });
}

rearr_status rearr_pipeline_reorder_nm(rearr_pipeline *pipe, void *dst, const void *src, size_t elem_bytes,
                                       int rank_in, const int64_t *dims, int rank_out, const int *order,
                                       const int64_t *base, const int64_t *range)
{
    const bool shape_ok = rank_in >= 1 && rank_in <= REARR_MAX_RANK && dims && rank_out >= 1 &&
                          rank_out <= rank_in && order && range;
    size_t in_bytes = shape_ok ? product(rank_in, dims) * elem_bytes : 0, out_bytes = 0;
    if (shape_ok) {
        out_bytes = elem_bytes;
        for (int i = 0; i < rank_out; ++i)
            out_bytes *= (order[i] >= 0 && order[i] < rank_in && range[order[i]] > 0) ? size_t(range[order[i]]) : 0;
    }
    return run_op(pipe, "rearr_pipeline_reorder_nm", {{src, in_bytes}}, {{dst, out_bytes}},
                  [&](const SlotLayout &l, std::function<cudaError_t(cudaStream_t)> &go, std::string &err, uint32_t &cls) {
                      auto pl = std::make_shared<PermPlan>();
                      rearr_status st = plan_reorder_nm(l.out[0], l.in[0], elem_bytes, rank_in, dims, rank_out,
                                                        order, base, range, *pl, err);
                      go = [pl](cudaStream_t s) { return launch_single(pl->op, nullptr, s); };
                      return st;
                  });
}

rearr_status rearr_pipeline_scatter(rearr_pipeline *pipe, void *dst, const void *src, const uint32_t *idx, size_t n,
                                    size_t elem_bytes)
{
    return pipeline_indexed(pipe, "rearr_pipeline_scatter", dst, src, idx, n, elem_bytes, 4, true);
}

rearr_status rearr_pipeline_reorder64(rearr_pipeline *pipe, void *dst, const void *src, const uint64_t *idx, size_t n,
                                      size_t elem_bytes)
{
    return pipeline_indexed(pipe, "rearr_pipeline_reorder64", dst, src, idx, n, elem_bytes, 8, false);
}

rearr_status rearr_pipeline_scatter64(rearr_pipeline *pipe, void *dst, const void *src, const uint64_t *idx, size_t n,
                                      size_t elem_bytes)
{
    return pipeline_indexed(pipe, "rearr_pipeline_scatter64", dst, src, idx, n, elem_bytes, 8, true);
}

rearr_status rearr_pipeline_interlace(rearr_pipeline *pipe, void *dst, const void *const *srcs, int k, size_t n,
                                      size_t elem_bytes)
{
    std::vector<HostRange> ins;
    if (srcs && k >= 1 && k <= REARR_MAX_K)
        for (int j = 0; j < k; ++j) ins.push_back({srcs[j], n * elem_bytes});
    const size_t out = ins.empty() ? 0 : n * elem_bytes * size_t(k);
    return run_op(pipe, "rearr_pipeline_interlace", ins, {{dst, out}},
                  [&](const SlotLayout &l, std::function<cudaError_t(cudaStream_t)> &go, std::string &err, uint32_t &cls) {
                      auto pl = std::make_shared<InterlacePlan>();
                      std::vector<char *> planes(l.in.begin(), l.in.end());
                      rearr_status st = plan_interlace(true, l.out.empty() ? nullptr : l.out[0],
                                                       planes.empty() ? nullptr : planes.data(), k, n, elem_bytes,
                                                       *pl, err);
                      cls = pl->op.cls;
                      go = [pl](cudaStream_t s) { return launch_single(pl->op, pl->planes.data(), s); };
                      return st;
                  });
}

rearr_status rearr_pipeline_deinterlace(rearr_pipeline *pipe, void *const *dsts, const void *src, int k, size_t n,
                                        size_t elem_bytes)
{
    std::vector<HostOut> outs;
    if (dsts && k >= 1 && k <= REARR_MAX_K)
        for (int j = 0; j < k; ++j) outs.push_back({dsts[j], n * elem_bytes});
    const size_t in = outs.empty() ? 0 : n * elem_bytes * size_t(k);
    return run_op(pipe, "rearr_pipeline_deinterlace", {{src, in}}, outs,
                  [&](const SlotLayout &l, std::function<cudaError_t(cudaStream_t)> &go, std::string &err, uint32_t &cls) {
                      auto pl = std::make_shared<InterlacePlan>();
                      std::vector<char *> planes(l.out.begin(), l.out.end());
                      rearr_status st = plan_interlace(false, l.in[0], planes.empty() ? nullptr : planes.data(), k,
                                                       n, elem_bytes, *pl, err);
                      cls = pl->op.cls;
                      go = [pl](cudaStream_t s) { return launch_single(pl->op, pl->planes.data(), s); };
                      return st;
                  });
}

rearr_status rearr_pipeline_stencil2d_f32(rearr_pipeline *pipe, float *dst, const float *src, int64_t ny, int64_t nx,
                                          int ntaps, const int *dy, const int *dx, const float *w, int boundary)
{
    const size_t bytes = (ny > 0 && nx > 0) ? size_t(ny) * size_t(nx) * sizeof(float) : 0;
    return run_op(pipe, "rearr_pipeline_stencil2d_f32", {{src, bytes}}, {{dst, bytes}},
                  [&](const SlotLayout &l, std::function<cudaError_t(cudaStream_t)> &go, std::string &err, uint32_t &cls) {
                      auto pl = std::make_shared<StencilPlan>();
                      rearr_status st = plan_stencil2d(reinterpret_cast<float *>(l.out[0]),
                                                       reinterpret_cast<const float *>(l.in[0]), ny, nx, ntaps, dy,
                                                       dx, w, boundary, *pl, err);
                      go = [pl](cudaStream_t s) { return launch_stencil2d(*pl, s); };
                      return st;
                  });
}

rearr_status rearr_pipeline_sync(rearr_pipeline *pipe)
{
    if (!pipe) return fail(REARR_EINVAL, "rearr_pipeline_sync: pipeline is NULL");
    cudaError_t e = cudaSuccess;
    for (cudaStream_t s : {pipe->up, pipe->comp, pipe->down}) {
        cudaError_t es = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = es;
    }
    if (e != cudaSuccess) {
        pipe->broken = e;
        return cuda_fail(e, "rearr_pipeline_sync");
    }
    if (pipe->broken != cudaSuccess) return cuda_fail(pipe->broken, "rearr_pipeline_sync");
    return REARR_OK;
}

rearr_status rearr_pipeline_set_direct(rearr_pipeline *pipe, int mode)
{
    if (!pipe) return fail(REARR_EINVAL, "rearr_pipeline_set_direct: pipeline is NULL");
    if (mode != 0 && mode != 1) return fail(REARR_EINVAL, "rearr_pipeline_set_direct: mode must be 0 or 1");
    pipe->direct = mode;
    return REARR_OK;
}

rearr_status rearr_pipeline_direct_ops(const rearr_pipeline *pipe, uint64_t *direct_ops, int *mode)
{
    if (!pipe) return fail(REARR_EINVAL, "rearr_pipeline_direct_ops: pipeline is NULL");
    if (direct_ops) *direct_ops = pipe->direct_ops;
    if (mode) *mode = pipe->direct;
    return REARR_OK;
}

rearr_status rearr_pipeline_stats(const rearr_pipeline *pipe, uint64_t *ops, uint64_t *h2d_bytes, uint64_t *d2h_bytes)
{
    if (!pipe) return fail(REARR_EINVAL, "rearr_pipeline_stats: pipeline is NULL");
    if (ops) *ops = pipe->ops;
    if (h2d_bytes) *h2d_bytes = pipe->h2d;
    if (d2h_bytes) *d2h_bytes = pipe->d2h;
    return REARR_OK;
}

void rearr_pipeline_destroy(rearr_pipeline *pipe)
{
    if (!pipe) return;
    for (cudaStream_t s : {pipe->up, pipe->comp, pipe->down})
        if (s) cudaStreamSynchronize(s);
    for (auto *v : {&pipe->in_ready, &pipe->computed, &pipe->out_done})
        for (cudaEvent_t ev : *v)
            if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : {pipe->up_tail, pipe->down_tail, pipe->direct_done})
        if (ev) cudaEventDestroy(ev);
    for (cudaStream_t s : {pipe->up, pipe->comp, pipe->down})
        if (s) cudaStreamDestroy(s);
    if (pipe->dev) cudaFree(pipe->dev);
    delete pipe;
}

}  // extern "C"
