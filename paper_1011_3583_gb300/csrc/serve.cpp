// serve.cpp -- serving loop of librearr (include/librearr_serve.h).
//
// Requests are admitted in FIFO order against a device slab managed by the
// first-fit Arena; a submitted request joins the ready queue.  One server
// thread launches the ready requests and watches completions:
//   batching mode: every free stream slot takes up to max_batch_ops ready
//     requests, uploads their descriptors into the slot's own work-list
//     buffer and launches the persistent batched kernel (continuous batching:
//     requests that arrive while other batches run go out as soon as a slot
//     frees up, so their work overlaps on the device); a large request, or a
//     request that is alone in the ready queue, runs as its single-op kernel
//     on the single-op lane, one stream in arrival order;
//   plain mode: every ready request is launched at once as its own single-op
//     kernel on one stream, in arrival order (the one-launch-per-call path).
// Completion is found by polling CUDA events; the server never waits on the
// GPU while holding its lock, and no kernel waits on another.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/librearr_serve.h"
#include "arena.h"
#include "launch.h"
#include "plan.h"
#include "worklist.h"

namespace rearr {

rearr_status fail(rearr_status st, const std::string &msg);
rearr_status cuda_fail(cudaError_t e, const char *what);

namespace {

using Clock = std::chrono::steady_clock;

double now_s()
{
    return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

enum State { RESERVED, QUEUED, RUNNING, DONE };

struct Req {
    uint64_t ticket = 0;
    rearr_op_spec spec{};
    std::vector<uintptr_t> ins, outs;
    std::vector<uintptr_t> blocks;
    double t_arrival = 0, t_done = 0;
    State state = RESERVED;
    cudaEvent_t ev = nullptr;  // plain mode: completion event of this request
    std::vector<const void *> in_src;  // device sources copied into the inputs first
    size_t bytes = 0;                  // read + write bytes of the op
};

// Copies a request's input sources into its inputs on stream s.
cudaError_t copy_inputs(const Req &r, const std::vector<size_t> &in_sizes, cudaStream_t s)
{
    for (size_t j = 0; j < r.in_src.size() && j < r.ins.size(); ++j) {
        if (!r.in_src[j]) continue;
        cudaError_t e = cudaMemcpyAsync(reinterpret_cast<void *>(r.ins[j]), r.in_src[j], in_sizes[j],
                                        cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Byte sizes of a request's buffers (inputs, outputs), or false if invalid.
bool buffer_sizes(const rearr_op_spec &s, std::vector<size_t> &in, std::vector<size_t> &out, std::string &err)
{
    in.clear();
    out.clear();
    const size_t e = s.elem_bytes;
    switch (s.kind) {
        case REARR_OP_PERMUTE: {
            if (s.rank < 1 || s.rank > 8) { err = "rank must be in [1, 8]"; return false; }
            size_t t = 1;
            for (int i = 0; i < s.rank; ++i) {
                if (s.dims[i] < 0) { err = "dims must be >= 0"; return false; }
                t *= size_t(s.dims[i]);
            }
            in = {t * e};
            out = {t * e};
            return true;
        }
        case REARR_OP_REORDER:
            in = {s.n * e, s.n * 4};
            out = {s.n * e};
            return true;
        case REARR_OP_INTERLACE:
        case REARR_OP_DEINTERLACE: {
            if (s.k < 1 || s.k > kMaxK) { err = "k must be in [1, 256]"; return false; }
            std::vector<size_t> planes(size_t(s.k), s.n * e);
            std::vector<size_t> one = {s.n * e * size_t(s.k)};
            if (s.kind == REARR_OP_INTERLACE) { in = planes; out = one; }
            else { in = one; out = planes; }
            return true;
        }
        default:
            err = "unknown op kind";
            return false;
    }
}

// Plan one request on its (arena) buffers.
rearr_status plan_request(const Req &r, OpDesc &op, std::vector<char *> &planes, std::string &err)
{
    const rearr_op_spec &s = r.spec;
    planes.clear();
    switch (s.kind) {
        case REARR_OP_PERMUTE: {
            PermPlan pl;
            rearr_status st = plan_permute(reinterpret_cast<void *>(r.outs[0]), reinterpret_cast<const void *>(r.ins[0]),
                                           s.elem_bytes, s.rank, s.dims, s.perm, pl, err);
            op = pl.op;
            return st;
        }
        case REARR_OP_REORDER:
            return plan_reorder(reinterpret_cast<void *>(r.outs[0]), reinterpret_cast<const void *>(r.ins[0]),
                                reinterpret_cast<const uint32_t *>(r.ins[1]), s.n, s.elem_bytes, op, err);
        case REARR_OP_INTERLACE:
        case REARR_OP_DEINTERLACE: {
            const bool inter = s.kind == REARR_OP_INTERLACE;
            std::vector<char *> pl;
            const std::vector<uintptr_t> &pv = inter ? r.ins : r.outs;
            for (uintptr_t p : pv) pl.push_back(reinterpret_cast<char *>(p));
            char *iv = reinterpret_cast<char *>(inter ? r.outs[0] : r.ins[0]);
            InterlacePlan ip;
            rearr_status st = plan_interlace(inter, iv, pl.data(), s.k, s.n, s.elem_bytes, ip, err);
            op = ip.op;
            if (st == REARR_OK) planes = ip.planes;
            return st;
        }
        default:
            err = "unknown op kind";
            return REARR_EINVAL;
    }
}

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    void *dev_wl = nullptr;          // device work-list buffer
    unsigned char *host_wl = nullptr;  // pinned staging of the same size
    size_t wl_bytes = 0;
    bool busy = false;
    double t_launch = 0;
    std::vector<Req *> reqs;
};

constexpr size_t kMaxPlanePtrsPerBatch = 65536;

}  // namespace

struct Server {
    rearr_server_config cfg{};
    void *slab = nullptr;
    std::unique_ptr<Arena> arena;
    int device = 0;

    std::mutex mu;
    std::condition_variable cv;
    uint64_t next_ticket = 1;
    std::deque<uint64_t> admit_q;      // reservations waiting for their turn / memory
    std::deque<Req *> ready;           // submitted, not launched
    std::deque<Req *> ready_large;     // batching mode: submitted large requests, not launched
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    std::vector<Slot> slots;
    std::deque<Req *> plain_inflight;  // single-op launches in stream order, not yet complete
    cudaStream_t lane = nullptr;       // batching mode: the stream of single-op launches
    std::vector<cudaEvent_t> event_pool;
    bool stop = false;
    std::thread worker;
    int64_t inject_delay_us = 0;
    std::string worker_error;

    rearr_server_stats st{};
    double busy_since = -1;

    ~Server();
    void run();
    void launch_batches(std::unique_lock<std::mutex> &lk);
    void launch_plain(std::unique_lock<std::mutex> &lk);
    void launch_on_lane(Req *r, cudaStream_t stream);
    // Queues a submitted request (large ones apart in batching mode).
    void enqueue(Req *r)
    {
        if (cfg.batching && r->bytes >= cfg.large_bytes) ready_large.push_back(r);
        else ready.push_back(r);
    }
    bool pending() const { return !ready.empty() || !ready_large.empty(); }
    bool poll_completions();
    bool inflight() const;
};

bool Server::inflight() const
{
    if (!plain_inflight.empty()) return true;
    for (const Slot &s : slots)
        if (s.busy) return true;
    return false;
}

Server::~Server()
{
    for (Slot &s : slots) {
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.dev_wl) cudaFree(s.dev_wl);
        if (s.host_wl) cudaFreeHost(s.host_wl);
    }
    if (lane) cudaStreamDestroy(lane);
    for (cudaEvent_t e : event_pool) cudaEventDestroy(e);
    for (auto &kv : reqs)
        if (kv.second->ev) cudaEventDestroy(kv.second->ev);
    if (slab) cudaFree(slab);
}

// Marks finished work; true if anything completed.
bool Server::poll_completions()
{
    bool any = false;
    const double t = now_s();
    const double delay = double(inject_delay_us) * 1e-6;
    for (Slot &s : slots) {
        if (!s.busy) continue;
        if (t < s.t_launch + delay) continue;
        if (cudaEventQuery(s.done) != cudaSuccess) continue;
        for (Req *r : s.reqs) {
            r->state = DONE;
            r->t_done = t;
            ++st.completed;
        }
        s.reqs.clear();
        s.busy = false;
        any = true;
    }
    while (!plain_inflight.empty()) {  // plain launches complete in stream order
        Req *r = plain_inflight.front();
        if (t < r->t_arrival + delay) break;
        if (cudaEventQuery(r->ev) != cudaSuccess) break;
        r->state = DONE;
        r->t_done = t;
        ++st.completed;
        event_pool.push_back(r->ev);
        r->ev = nullptr;
        plain_inflight.pop_front();
        any = true;
    }
    const bool busy = inflight();
    if (busy && busy_since < 0) busy_since = t;
    if (!busy && busy_since >= 0) {
        st.busy_seconds += t - busy_since;
        busy_since = -1;
    }
    return any;
}

void Server::launch_batches(std::unique_lock<std::mutex> &)
{
    // A large request runs as its own single-op kernel on the single-op lane
    // as soon as it is ready: large requests never wait for a slot, and run
    // back to back in arrival order.
    while (!ready_large.empty()) {
        Req *r = ready_large.front();
        ready_large.pop_front();
        launch_on_lane(r, lane);
    }
    for (Slot &s : slots) {
        // A lone ready request also runs as its single-op kernel on the lane
        // (one op gains nothing from a work list): at light load the server
        // then behaves as the plain path does; batches take over as soon as
        // requests queue up.
        if (ready.size() == 1) {
            Req *r = ready.front();
            ready.pop_front();
            launch_on_lane(r, lane);
        }
        if (ready.empty()) return;
        if (s.busy) continue;
        // Take ready requests in FIFO order while the slot's work list has room.
        std::vector<OpDesc> ops;
        std::vector<std::vector<char *>> planes;
        std::vector<Req *> taken;
        size_t n_ptrs = 0;
        while (!ready.empty() && int(taken.size()) < cfg.max_batch_ops) {
            Req *r = ready.front();
            if (r->bytes >= cfg.large_bytes) break;  // goes to the single-op lane
            OpDesc op;
            std::vector<char *> pl;
            std::string err;
            if (plan_request(*r, op, pl, err) != REARR_OK) {  // validated at reserve: should not happen
                worker_error = "plan failed in the server: " + err;
                ready.pop_front();
                r->state = DONE;
                r->t_done = now_s();
                ++st.completed;
                continue;
            }
            const size_t extra = (op.cls == OC_INTERLACE || op.cls == OC_DEINTERLACE) && op.inter.k > kInlineK
                                     ? pl.size() : 0;
            if (n_ptrs + extra > kMaxPlanePtrsPerBatch && !taken.empty()) break;
            ready.pop_front();
            taken.push_back(r);
            if (op.units == 0) continue;  // zero-size op: done with the batch, no work
            batch_form(op);
            ops.push_back(op);
            planes.push_back(extra ? pl : std::vector<char *>{});
            n_ptrs += extra;
        }
        if (taken.empty()) return;
        const WorklistLayout lay = worklist_layout(ops.size(), n_ptrs);
        cudaError_t e = cudaSuccess;
        for (Req *r : taken) {
            if (r->in_src.empty() || e != cudaSuccess) continue;
            std::vector<size_t> in_sz, out_sz;
            std::string err;
            buffer_sizes(r->spec, in_sz, out_sz, err);
            e = copy_inputs(*r, in_sz, s.stream);
        }
        if (!ops.empty() && e == cudaSuccess) {
            order_for_batch(ops, planes);
            const uint64_t total = build_worklist(ops.data(), planes.data(), ops.size(), s.host_wl,
                                                  reinterpret_cast<uintptr_t>(s.dev_wl), lay);
            e = cudaMemcpyAsync(s.dev_wl, s.host_wl, lay.bytes, cudaMemcpyHostToDevice, s.stream);
            if (e == cudaSuccess) e = launch_worklist(reinterpret_cast<uintptr_t>(s.dev_wl), lay, ops.size(), total, s.stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(s.done, s.stream);
        if (e != cudaSuccess) worker_error = std::string("batch launch failed: ") + cudaGetErrorString(e);
        for (Req *r : taken) r->state = RUNNING;
        s.reqs = std::move(taken);
        s.busy = true;
        s.t_launch = now_s();
        ++st.launches;
    }
}

// One request as its single-op kernel on `stream`; its completion event
// joins plain_inflight (requests on one stream complete in order).
void Server::launch_on_lane(Req *r, cudaStream_t stream)
{
    OpDesc op;
    std::vector<char *> pl;
    std::string err;
    std::vector<size_t> in_sz, out_sz;
    buffer_sizes(r->spec, in_sz, out_sz, err);
    cudaError_t e = copy_inputs(*r, in_sz, stream);
    if (e != cudaSuccess) {
        worker_error = std::string("input copy failed: ") + cudaGetErrorString(e);
    } else if (plan_request(*r, op, pl, err) == REARR_OK) {
        e = launch_single(op, pl.data(), stream);
    } else {
        worker_error = "plan failed in the server: " + err;
    }
    if (event_pool.empty()) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) event_pool.push_back(ev);
    }
    if (!event_pool.empty()) {
        r->ev = event_pool.back();
        event_pool.pop_back();
        if (e == cudaSuccess) e = cudaEventRecord(r->ev, stream);
    }
    if (e != cudaSuccess) worker_error = std::string("single-op launch failed: ") + cudaGetErrorString(e);
    r->state = RUNNING;
    if (r->ev) plain_inflight.push_back(r);
    else { r->state = DONE; r->t_done = now_s(); ++st.completed; }
    ++st.launches;
}

void Server::launch_plain(std::unique_lock<std::mutex> &)
{
    while (!ready.empty()) {
        Req *r = ready.front();
        ready.pop_front();
        launch_on_lane(r, slots[0].stream);
    }
}

void Server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        const bool completed = poll_completions();
        if (cfg.batching) launch_batches(lk);
        else launch_plain(lk);
        if (completed) cv.notify_all();
        if (stop && !pending() && !inflight()) break;
        if (inflight()) {
            cv.wait_for(lk, std::chrono::microseconds(cfg.poll_interval_us));
        } else {
            cv.wait(lk, [&] { return stop || pending(); });
        }
    }
    cv.notify_all();
}

}  // namespace rearr

struct rearr_server {
    rearr::Server s;
};

using namespace rearr;

extern "C" {

rearr_status rearr_server_create(const rearr_server_config *config, rearr_server **server)
{
    if (!config || !server) return fail(REARR_EINVAL, "rearr_server_create: NULL argument");
    rearr_server_config c = *config;
    if (c.budget_bytes < Arena::kAlign) return fail(REARR_EINVAL, "rearr_server_create: budget too small");
    if (c.n_streams < 1 || c.n_streams > 8) return fail(REARR_EINVAL, "rearr_server_create: n_streams must be 1..8");
    if (c.max_batch_ops < 1 || c.max_batch_ops > 4096)
        return fail(REARR_EINVAL, "rearr_server_create: max_batch_ops must be 1..4096");
    if (c.poll_interval_us < 1) c.poll_interval_us = 1;
    if (c.large_bytes == 0) c.large_bytes = size_t(64) << 20;
    if (!c.batching) c.n_streams = 1;
    auto *out = new (std::nothrow) rearr_server();
    if (!out) return fail(REARR_ENOMEM, "rearr_server_create: out of host memory");
    Server &S = out->s;
    S.cfg = c;
    cudaGetDevice(&S.device);
    cudaError_t e = cudaMalloc(&S.slab, c.budget_bytes);
    if (e != cudaSuccess) {
        S.slab = nullptr;
        delete out;
        return fail(REARR_ENOMEM, std::string("rearr_server_create: slab cudaMalloc: ") + cudaGetErrorString(e));
    }
    S.arena.reset(new Arena(reinterpret_cast<uintptr_t>(S.slab), c.budget_bytes));
    S.st.slab_bytes = S.arena->capacity();
    const WorklistLayout lay = worklist_layout(size_t(c.max_batch_ops), kMaxPlanePtrsPerBatch);
    S.slots.resize(size_t(c.n_streams));
    for (Slot &s : S.slots) {
        e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e == cudaSuccess && c.batching) {
            s.wl_bytes = lay.bytes;
            e = cudaMalloc(&s.dev_wl, lay.bytes);
            if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&s.host_wl), lay.bytes, cudaHostAllocDefault);
        }
        if (e != cudaSuccess) {
            delete out;
            return cuda_fail(e, "rearr_server_create: stream slot");
        }
    }
    if (c.batching) {
        e = cudaStreamCreateWithFlags(&S.lane, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete out;
            return cuda_fail(e, "rearr_server_create: single-op lane");
        }
    }
    S.worker = std::thread([&S] { S.run(); });
    *server = out;
    return REARR_OK;
}

rearr_status rearr_server_reserve(rearr_server *server, const rearr_op_spec *spec, int64_t timeout_us, uint64_t *ticket)
{
    if (!server || !spec || !ticket) return fail(REARR_EINVAL, "rearr_server_reserve: NULL argument");
    Server &S = server->s;
    const double t_arrival = now_s();
    std::vector<size_t> in, out;
    std::string err;
    if (!buffer_sizes(*spec, in, out, err)) return fail(REARR_EINVAL, "rearr_server_reserve: " + err);
    size_t total = 0;
    for (size_t b : in) total += Arena::round(b);
    for (size_t b : out) total += Arena::round(b);
    if (total > S.arena->capacity()) return fail(REARR_ENOMEM, "rearr_server_reserve: request exceeds the budget");
    {  // validate the op itself on placeholder addresses before it may wait
        Req probe;
        probe.spec = *spec;
        uintptr_t fake = uintptr_t(1) << 46;
        for (size_t b : in) { probe.ins.push_back(fake); fake += Arena::round(b) + 256; }
        for (size_t b : out) { probe.outs.push_back(fake); fake += Arena::round(b) + 256; }
        OpDesc op;
        std::vector<char *> pl;
        if (plan_request(probe, op, pl, err) != REARR_OK) return fail(REARR_EINVAL, "rearr_server_reserve: " + err);
    }
    std::unique_lock<std::mutex> lk(S.mu);
    const uint64_t t = S.next_ticket++;
    S.admit_q.push_back(t);
    auto r = std::make_unique<Req>();
    r->ticket = t;
    r->spec = *spec;
    r->t_arrival = t_arrival;
    for (size_t b : in) r->bytes += b;
    for (size_t b : out) r->bytes += b;
    auto try_admit = [&]() -> bool {
        if (S.admit_q.front() != t) return false;
        std::vector<uintptr_t> got;
        for (size_t b : in) {
            uintptr_t a;
            if (!S.arena->alloc(b, a)) break;
            got.push_back(a);
        }
        if (got.size() == in.size()) {
            for (size_t b : out) {
                uintptr_t a;
                if (!S.arena->alloc(b, a)) break;
                got.push_back(a);
            }
        }
        if (got.size() != in.size() + out.size()) {
            for (uintptr_t a : got) S.arena->free(a);
            return false;
        }
        r->blocks = got;
        r->ins.assign(got.begin(), got.begin() + in.size());
        r->outs.assign(got.begin() + in.size(), got.end());
        return true;
    };
    const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
    bool ok = try_admit();
    while (!ok) {
        if (timeout_us < 0) S.cv.wait(lk);
        else if (S.cv.wait_until(lk, deadline) == std::cv_status::timeout) {
            ok = try_admit();
            break;
        }
        ok = try_admit();
    }
    if (!ok) {
        S.admit_q.erase(std::find(S.admit_q.begin(), S.admit_q.end(), t));
        S.cv.notify_all();
        return fail(REARR_ETIMEDOUT, "rearr_server_reserve: no room in the budget before the deadline");
    }
    S.admit_q.pop_front();
    ++S.st.admitted;
    S.st.slab_used = S.arena->used();
    S.st.slab_peak = std::max(S.st.slab_peak, S.st.slab_used);
    S.reqs[t] = std::move(r);
    *ticket = t;
    S.cv.notify_all();  // the next reservation in line may fit too
    return REARR_OK;
}

static Req *find_req(Server &S, uint64_t ticket)
{
    auto it = S.reqs.find(ticket);
    return it == S.reqs.end() ? nullptr : it->second.get();
}

rearr_status rearr_server_buffers(rearr_server *server, uint64_t ticket, void **ins, int *n_in, void **outs, int *n_out)
{
    if (!server) return fail(REARR_EINVAL, "rearr_server_buffers: server is NULL");
    Server &S = server->s;
    std::lock_guard<std::mutex> lk(S.mu);
    Req *r = find_req(S, ticket);
    if (!r) return fail(REARR_EINVAL, "rearr_server_buffers: unknown ticket");
    if (n_in) *n_in = int(r->ins.size());
    if (n_out) *n_out = int(r->outs.size());
    if (ins)
        for (size_t i = 0; i < r->ins.size(); ++i) ins[i] = reinterpret_cast<void *>(r->ins[i]);
    if (outs)
        for (size_t i = 0; i < r->outs.size(); ++i) outs[i] = reinterpret_cast<void *>(r->outs[i]);
    return REARR_OK;
}

rearr_status rearr_server_submit(rearr_server *server, uint64_t ticket)
{
    if (!server) return fail(REARR_EINVAL, "rearr_server_submit: server is NULL");
    Server &S = server->s;
    std::lock_guard<std::mutex> lk(S.mu);
    Req *r = find_req(S, ticket);
    if (!r) return fail(REARR_EINVAL, "rearr_server_submit: unknown ticket");
    if (r->state != RESERVED) return fail(REARR_EBUSY, "rearr_server_submit: request already submitted");
    r->state = QUEUED;
    S.enqueue(r);
    S.cv.notify_all();
    return REARR_OK;
}

rearr_status rearr_server_submit_from(rearr_server *server, uint64_t ticket, const void *const *srcs, int n_srcs)
{
    if (!server || (n_srcs > 0 && !srcs) || n_srcs < 0) return fail(REARR_EINVAL, "rearr_server_submit_from: bad argument");
    Server &S = server->s;
    std::lock_guard<std::mutex> lk(S.mu);
    Req *r = find_req(S, ticket);
    if (!r) return fail(REARR_EINVAL, "rearr_server_submit_from: unknown ticket");
    if (r->state != RESERVED) return fail(REARR_EBUSY, "rearr_server_submit_from: request already submitted");
    if (size_t(n_srcs) > r->ins.size()) return fail(REARR_EINVAL, "rearr_server_submit_from: more sources than inputs");
    r->in_src.assign(srcs, srcs + n_srcs);
    r->state = QUEUED;
    S.enqueue(r);
    S.cv.notify_all();
    return REARR_OK;
}

rearr_status rearr_server_poll(rearr_server *server, uint64_t ticket, int *done)
{
    if (!server || !done) return fail(REARR_EINVAL, "rearr_server_poll: NULL argument");
    Server &S = server->s;
    std::lock_guard<std::mutex> lk(S.mu);
    Req *r = find_req(S, ticket);
    if (!r) return fail(REARR_EINVAL, "rearr_server_poll: unknown ticket");
    *done = r->state == DONE ? 1 : 0;
    return REARR_OK;
}

rearr_status rearr_server_wait(rearr_server *server, uint64_t ticket, int64_t timeout_us)
{
    if (!server) return fail(REARR_EINVAL, "rearr_server_wait: server is NULL");
    Server &S = server->s;
    std::unique_lock<std::mutex> lk(S.mu);
    Req *r = find_req(S, ticket);
    if (!r) return fail(REARR_EINVAL, "rearr_server_wait: unknown ticket");
    if (r->state == RESERVED) return fail(REARR_EINVAL, "rearr_server_wait: request was never submitted");
    auto pred = [&] { return r->state == DONE; };
    if (timeout_us < 0) S.cv.wait(lk, pred);
    else if (!S.cv.wait_for(lk, std::chrono::microseconds(timeout_us), pred))
        return fail(REARR_ETIMEDOUT, "rearr_server_wait: not complete before the deadline");
    if (!S.worker_error.empty()) return fail(REARR_ECUDA, "rearr_server_wait: " + S.worker_error);
    return REARR_OK;
}

rearr_status rearr_server_latency(rearr_server *server, uint64_t ticket, double *seconds)
{
    if (!server || !seconds) return fail(REARR_EINVAL, "rearr_server_latency: NULL argument");
    Server &S = server->s;
    std::lock_guard<std::mutex> lk(S.mu);
    Req *r = find_req(S, ticket);
    if (!r) return fail(REARR_EINVAL, "rearr_server_latency: unknown ticket");
    if (r->state != DONE) return fail(REARR_EBUSY, "rearr_server_latency: request not complete");
    *seconds = r->t_done - r->t_arrival;
    return REARR_OK;
}

rearr_status rearr_server_release(rearr_server *server, uint64_t ticket)
{
    if (!server) return fail(REARR_EINVAL, "rearr_server_release: server is NULL");
    Server &S = server->s;
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.reqs.find(ticket);
    if (it == S.reqs.end()) return fail(REARR_EINVAL, "rearr_server_release: unknown ticket");
    Req *r = it->second.get();
    if (r->state == QUEUED || r->state == RUNNING)
        return fail(REARR_EBUSY, "rearr_server_release: request still in flight");
    for (uintptr_t a : r->blocks) S.arena->free(a);
    if (r->ev) S.event_pool.push_back(r->ev);
    S.reqs.erase(it);
    ++S.st.released;
    S.st.slab_used = S.arena->used();
    S.cv.notify_all();  // memory freed: waiting reservations may fit now
    return REARR_OK;
}

rearr_status rearr_server_stats_get(rearr_server *server, rearr_server_stats *stats)
{
    if (!server || !stats) return fail(REARR_EINVAL, "rearr_server_stats_get: NULL argument");
    Server &S = server->s;
    std::lock_guard<std::mutex> lk(S.mu);
    *stats = S.st;
    if (S.busy_since >= 0) stats->busy_seconds += now_s() - S.busy_since;
    return REARR_OK;
}

rearr_status rearr_server_inject_completion_delay(rearr_server *server, int64_t delay_us)
{
    if (!server || delay_us < 0) return fail(REARR_EINVAL, "rearr_server_inject_completion_delay: bad argument");
    std::lock_guard<std::mutex> lk(server->s.mu);
    server->s.inject_delay_us = delay_us;
    return REARR_OK;
}

rearr_status rearr_server_destroy(rearr_server *server, int64_t timeout_us)
{
    if (!server) return REARR_OK;
    Server &S = server->s;
    {
        std::unique_lock<std::mutex> lk(S.mu);
        auto idle = [&] { return !S.pending() && !S.inflight(); };
        if (timeout_us < 0) S.cv.wait(lk, idle);
        else if (!S.cv.wait_for(lk, std::chrono::microseconds(timeout_us), idle))
            return fail(REARR_ETIMEDOUT, "rearr_server_destroy: work still in flight");
        S.stop = true;
        S.cv.notify_all();
    }
    if (S.worker.joinable()) S.worker.join();
    delete server;
    return REARR_OK;
}

// ---------------------------------------------------------------------------
// Trace driver.

rearr_status rearr_server_run_trace(rearr_server *server, const rearr_op_spec *specs, const double *arrival_s,
                                    const void *const *templates, size_t n, double *latency_s, double *wall_s,
                                    int64_t timeout_us)
{
    if (!server || (n && (!specs || !arrival_s || !latency_s))) return fail(REARR_EINVAL, "rearr_server_run_trace: NULL argument");
    if (n == 0) {
        if (wall_s) *wall_s = 0;
        return REARR_OK;
    }
    Server &S = server->s;
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<uint64_t> tickets(n, 0);
    std::vector<char> submitted(n, 0);
    std::mutex tmu;
    std::condition_variable tcv;
    rearr_status sub_status = REARR_OK, done_status = REARR_OK;
    std::string sub_err, done_err;
    const double t0 = now_s() + 1e-3;
    const double deadline = timeout_us < 0 ? 1e300 : t0 + double(timeout_us) * 1e-6;
    double t_last = t0;

    std::thread submitter([&] {
        cudaSetDevice(dev);
        for (size_t i = 0; i < n; ++i) {
            const double ta = t0 + arrival_s[i];
            for (;;) {  // sleep until the arrival time, spin for the last 50 us
                const double d = ta - now_s();
                if (d <= 0) break;
                if (d > 60e-6) std::this_thread::sleep_for(std::chrono::duration<double>(d - 50e-6));
            }
            uint64_t tk = 0;
            const int64_t left = int64_t((deadline - now_s()) * 1e6);
            rearr_status st = rearr_server_reserve(server, &specs[i], left > 0 ? left : 0, &tk);
            if (st != REARR_OK) { sub_status = st; sub_err = rearr_last_error(); break; }
            bool any = false;
            if (templates)
                for (int j = 0; j < 4; ++j) any = any || templates[i * 4 + size_t(j)] != nullptr;
            if (any) {
                std::vector<size_t> in, out;
                std::string err;
                buffer_sizes(specs[i], in, out, err);
                const int n_src = int(std::min<size_t>(4, in.size()));
                rearr_server_submit_from(server, tk, templates + i * 4, n_src);
            } else {
                rearr_server_submit(server, tk);
            }
            {
                std::lock_guard<std::mutex> g(tmu);
                tickets[i] = tk;
                submitted[i] = 1;
            }
            tcv.notify_all();
        }
        tcv.notify_all();
    });

    std::thread completer([&] {
        for (size_t i = 0; i < n; ++i) {
            uint64_t tk;
            {
                std::unique_lock<std::mutex> g(tmu);
                tcv.wait(g, [&] { return submitted[i] || sub_status != REARR_OK; });
                if (!submitted[i]) return;
                tk = tickets[i];
            }
            const int64_t left = int64_t((deadline - now_s()) * 1e6);
            rearr_status st = rearr_server_wait(server, tk, left > 0 ? left : 0);
            if (st != REARR_OK) { done_status = st; done_err = rearr_last_error(); return; }
            double lat_from_reserve = 0;
            rearr_server_latency(server, tk, &lat_from_reserve);
            {
                std::lock_guard<std::mutex> lk(S.mu);
                Req *r = find_req(S, tk);
                const double td = r ? r->t_done : now_s();
                latency_s[i] = td - (t0 + arrival_s[i]);  // from the scheduled arrival
                t_last = std::max(t_last, td);
            }
            rearr_server_release(server, tk);
        }
    });
    submitter.join();
    completer.join();
    if (wall_s) *wall_s = t_last - (t0 + arrival_s[0]);
    if (sub_status != REARR_OK) return fail(sub_status, "rearr_server_run_trace: submit: " + sub_err);
    if (done_status != REARR_OK) return fail(done_status, "rearr_server_run_trace: wait: " + done_err);
    return REARR_OK;
}

}  // extern "C"
