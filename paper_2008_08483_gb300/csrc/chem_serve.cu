// chem_serve.cu -- persistent serving loop: many host producers (simulated CFD ranks, the
// paper's offload pattern) submit source-term and integration requests of uneven sizes;
// one worker thread batches them onto device slots and replays captured CUDA graphs.
//
// Life of a request: submit() validates it and appends it to the queue.  The worker takes
// the oldest queued request, adds every later queued request with the same batch key
// (mechanism, kind, precision, dt, tolerances) while the slot capacity allows, packs their
// inputs into the slot's page-locked staging, and enqueues on the slot's stream: the
// host->device copies, the graph of the batch's power-of-two size bucket (captured on first
// use: the source-term kernel, or the workspace clear and the reactor kernel, which reads
// the real cell count from device memory), the device->host copies and a host callback
// that wakes the worker.  Other slots run their batches meanwhile, so requests that arrive
// while the GPU is busy are admitted as soon as a slot frees: continuous batching over a
// fixed device footprint set by the HBM budget.  Slot 0 takes source-term batches only, so
// cheap source-term requests never wait behind long integrations, and integration batches
// stop at 65536 cells.  When a slot completes, the worker copies
// each request's rows to the caller's arrays and releases its waiters.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "chem_internal.h"

namespace chem {

using Clock = std::chrono::steady_clock;

constexpr int kSlots = 4;
constexpr int64_t kMinBucket = 64;
constexpr int64_t kIntegBatch = 65536;     // cells per integration batch (largest request)

struct Req {
    uint64_t id = 0;
    chem_request r;
    int ns = 0;
    Clock::time_point t_submit, t_launch;
    bool done = false;
    chem_result res;
};

struct BatchKey {
    int mech = 0, kind = 0, prec = 0, fixed = 0;
    double dt = 0, rtol = 0, atol = 0;
    bool operator==(const BatchKey &o) const
    {
        return mech == o.mech && kind == o.kind && prec == o.prec && fixed == o.fixed &&
               dt == o.dt && rtol == o.rtol && atol == o.atol;
    }
    bool operator<(const BatchKey &o) const
    {
        return std::tie(mech, kind, prec, fixed, dt, rtol, atol) <
               std::tie(o.mech, o.kind, o.prec, o.fixed, o.dt, o.rtol, o.atol);
    }
};

static BatchKey key_of(const chem_request &r)
{
    BatchKey k;
    k.mech = r.mech_index;
    k.kind = r.kind;
    k.prec = (int)r.precision;
    if (r.kind == CHEM_REQ_INTEGRATE) {
        k.fixed = r.fixed_steps;
        k.dt = r.dt;
        k.rtol = r.rtol;
        k.atol = r.atol;
    }
    return k;
}

struct Server;

struct Slot {
    Server *srv = nullptr;
    int index = 0;
    cudaStream_t stream = nullptr;
    // device buffers (element type per request: double, or float for FP32 / split-BF16)
    void *dT = nullptr, *dP = nullptr, *dY = nullptr, *dO = nullptr;
    int32_t *dStatus = nullptr;
    int64_t *dN = nullptr;
    void *dWs = nullptr;
    size_t ws_bytes = 0;
    // page-locked staging
    void *hT = nullptr, *hP = nullptr, *hY = nullptr, *hO = nullptr;
    int32_t *hStatus = nullptr;
    int64_t *hN = nullptr;
    // the batch in flight
    bool busy = false, ready = false;
    chem_status launch_status = CHEM_OK;
    BatchKey key;
    std::vector<std::shared_ptr<Req>> members;
    std::vector<int64_t> offsets;
    int64_t cells = 0;
    std::map<std::pair<BatchKey, int64_t>, cudaGraphExec_t> graphs;
};

struct Server {
    std::vector<const chem_mech *> mechs;
    int device = 0, ns_max = 0;
    int64_t cap = 0;
    size_t device_bytes = 0;
    Slot slots[kSlots];
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Req>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Req>> tickets;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    chem_serve_info info;

    void run();
    void launch(Slot &s);
    void retire(Slot &s);
};

static size_t elt_of(int prec) { return prec == CHEM_FP64 ? sizeof(double) : sizeof(float); }

static void CUDART_CB on_slot_done(void *arg)
{
    Slot *s = (Slot *)arg;
    {
        std::lock_guard<std::mutex> g(s->srv->mu);
        s->ready = true;
    }
    s->srv->cv_work.notify_all();
}

static int64_t bucket_for(int64_t n, int64_t cap)
{
    int64_t b = kMinBucket;
    while (b < n) b <<= 1;
    return b < cap ? b : cap;
}

// Enqueue the slot's batch (members and key already set).  Called without the lock.
void Server::launch(Slot &s)
{
    const BatchKey &k = s.key;
    const chem_mech *m = mechs[k.mech];
    const int ns = m->ns;
    const size_t elt = elt_of(k.prec);
    int64_t o = 0;
    s.offsets.clear();
    for (auto &q : s.members) {
        const int64_t n = q->r.n_cells;
        s.offsets.push_back(o);
        memcpy((char *)s.hT + o * elt, q->r.T, n * elt);
        memcpy((char *)s.hP + o * elt, q->r.P, n * elt);
        memcpy((char *)s.hY + o * ns * elt, q->r.Y, n * ns * elt);
        o += n;
    }
    s.cells = o;
    const int64_t bucket = bucket_for(o, cap);
    cudaError_t e = cudaSuccess;
    chem_status st = CHEM_OK;
    auto ck = [&](cudaError_t x) {
        if (e == cudaSuccess && x != cudaSuccess) e = x;
    };
    ck(cudaMemcpyAsync(s.dT, s.hT, o * elt, cudaMemcpyHostToDevice, s.stream));
    ck(cudaMemcpyAsync(s.dP, s.hP, o * elt, cudaMemcpyHostToDevice, s.stream));
    ck(cudaMemcpyAsync(s.dY, s.hY, o * ns * elt, cudaMemcpyHostToDevice, s.stream));
    if (k.kind == CHEM_REQ_INTEGRATE) {
        *s.hN = o;
        ck(cudaMemcpyAsync(s.dN, s.hN, sizeof(int64_t), cudaMemcpyHostToDevice, s.stream));
    }
    if (e == cudaSuccess) {
        auto gk = std::make_pair(k, bucket);
        auto it = s.graphs.find(gk);
        cudaGraphExec_t exec = nullptr;
        if (it != s.graphs.end()) {
            exec = it->second;
        } else {
            cudaGraph_t g = nullptr;
            ck(cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal));
            if (e == cudaSuccess) {
                if (k.kind == CHEM_REQ_SOURCE)
                    st = chem_source_term(m, bucket, s.dT, s.dP, s.dY, ns, s.dO, ns,
                                          (chem_precision)k.prec, s.stream);
                else {
                    chem_integrate_opts o;
                    memset(&o, 0, sizeof o);
                    o.fixed_steps = k.fixed;
                    st = integrate_launch(m, bucket, s.dN, (double *)s.dT, (const double *)s.dP,
                                          (double *)s.dY, ns, k.dt, k.rtol, k.atol, &o, s.dStatus,
                                          s.dWs, s.ws_bytes, s.stream);
                }
                cudaError_t ec = cudaStreamEndCapture(s.stream, &g);
                if (st == CHEM_OK) ck(ec);
            }
            if (e == cudaSuccess && st == CHEM_OK) {
                ck(cudaGraphInstantiate(&exec, g, 0));
                if (e == cudaSuccess) {
                    s.graphs[gk] = exec;
                    std::lock_guard<std::mutex> lg(mu);
                    ++info.graphs_captured;
                }
            }
            if (g) cudaGraphDestroy(g);
        }
        if (e == cudaSuccess && st == CHEM_OK) {
            ck(cudaGraphLaunch(exec, s.stream));
            std::lock_guard<std::mutex> lg(mu);
            ++info.graph_launches;
        }
    }
    if (e == cudaSuccess && st == CHEM_OK) {
        if (k.kind == CHEM_REQ_SOURCE) {
            ck(cudaMemcpyAsync(s.hO, s.dO, o * ns * elt, cudaMemcpyDeviceToHost, s.stream));
        } else {
            ck(cudaMemcpyAsync(s.hT, s.dT, o * elt, cudaMemcpyDeviceToHost, s.stream));
            ck(cudaMemcpyAsync(s.hY, s.dY, o * ns * elt, cudaMemcpyDeviceToHost, s.stream));
            ck(cudaMemcpyAsync(s.hStatus, s.dStatus, o * sizeof(int32_t), cudaMemcpyDeviceToHost,
                               s.stream));
        }
        ck(cudaLaunchHostFunc(s.stream, on_slot_done, &s));
    }
    if (e != cudaSuccess && st == CHEM_OK) st = set_error(CHEM_ECUDA, "serve: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lg(mu);
    s.launch_status = st;
    if (st != CHEM_OK) s.ready = true;      // nothing in flight: retire at once
}

// Copy results out and complete the members.  Called without the lock.
void Server::retire(Slot &s)
{
    const BatchKey &k = s.key;
    const int ns = mechs[k.mech]->ns;
    const size_t elt = elt_of(k.prec);
    chem_status st = s.launch_status;
    if (st == CHEM_OK) {
        cudaError_t e = cudaStreamSynchronize(s.stream);     // already complete: cheap
        if (e != cudaSuccess) st = set_error(CHEM_ECUDA, "serve: %s", cudaGetErrorString(e));
    }
    const auto now = Clock::now();
    for (size_t i = 0; i < s.members.size(); ++i) {
        Req &q = *s.members[i];
        const int64_t o = s.offsets.size() > i ? s.offsets[i] : 0, n = q.r.n_cells;
        int32_t failed = 0;
        if (st == CHEM_OK) {
            if (k.kind == CHEM_REQ_SOURCE) {
                memcpy(q.r.omega, (char *)s.hO + o * ns * elt, n * ns * elt);
            } else {
                memcpy(q.r.T_out, (double *)s.hT + o, n * sizeof(double));
                memcpy(q.r.Y_out, (double *)s.hY + o * ns, n * ns * sizeof(double));
                for (int64_t c = 0; c < n; ++c) failed += s.hStatus[o + c] != CHEM_CELL_OK;
                if (q.r.cell_status) memcpy(q.r.cell_status, s.hStatus + o, n * sizeof(int32_t));
            }
        }
        q.res.status = st != CHEM_OK ? st : (failed ? CHEM_ENONCONV : CHEM_OK);
        q.res.n_failed = failed;
        q.res.n_cells = n;
        q.res.batch_cells = s.cells;
        q.res.batch_requests = (int32_t)s.members.size();
        q.res.slot = s.index;
        q.res.queue_us = std::chrono::duration<double, std::micro>(q.t_launch - q.t_submit).count();
        q.res.latency_us = std::chrono::duration<double, std::micro>(now - q.t_submit).count();
    }
    std::lock_guard<std::mutex> lg(mu);
    for (auto &q : s.members) q->done = true;
    info.completed += s.members.size();
    s.members.clear();
    s.busy = false;
    s.ready = false;
    cv_done.notify_all();
}

void Server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        // retire completed slots
        for (Slot &s : slots) {
            if (s.busy && s.ready) {
                lk.unlock();
                retire(s);
                lk.lock();
            }
        }
        bool any_busy = false;
        for (Slot &s : slots) any_busy |= s.busy;
        if (stop && !any_busy) break;
        // admit queued requests into free slots
        bool launched = false;
        if (!stop) {
            for (Slot &s : slots) {
                if (s.busy || queue.empty()) continue;
                // slot 0 is the source-term lane: long integrations never block it
                auto head = queue.begin();
                if (s.index == 0)
                    while (head != queue.end() && (*head)->r.kind != CHEM_REQ_SOURCE) ++head;
                if (head == queue.end()) continue;
                const BatchKey key = key_of((*head)->r);
                // integrations are batched up to the largest request, so that one long
                // batch does not hold every queued integration until it ends
                const int64_t limit = key.kind == CHEM_REQ_INTEGRATE ? std::min(cap, kIntegBatch) : cap;
                s.members.clear();
                int64_t cells = 0;
                for (auto it = head; it != queue.end();) {
                    const Req &q = **it;
                    if (key_of(q.r) == key && (cells == 0 || cells + q.r.n_cells <= limit)) {
                        cells += q.r.n_cells;
                        s.members.push_back(*it);
                        it = queue.erase(it);
                    } else {
                        ++it;
                    }
                }
                const auto now = Clock::now();
                for (auto &q : s.members) q->t_launch = now;
                s.key = key;
                s.busy = true;
                s.ready = false;
                ++info.batches;
                if ((int32_t)s.members.size() > info.max_batch_requests)
                    info.max_batch_requests = (int32_t)s.members.size();
                lk.unlock();
                launch(s);
                lk.lock();
                launched = true;
            }
        }
        if (launched) continue;
        bool pending_ready = false;
        for (Slot &s : slots) pending_ready |= s.busy && s.ready;
        if (pending_ready) continue;
        // nothing could be launched (queue empty, no free slot, or only integrations queued
        // while the source-term lane is the free slot): sleep until a submission or a slot
        // completion (bounded, as a safety net)
        cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
}

static void free_server(Server *S)
{
    for (Slot &s : S->slots) {
        for (auto &kv : s.graphs) cudaGraphExecDestroy(kv.second);
        s.graphs.clear();
        if (s.stream) cudaStreamDestroy(s.stream);
        cudaFree(s.dT);
        cudaFree(s.dP);
        cudaFree(s.dY);
        cudaFree(s.dO);
        cudaFree(s.dStatus);
        cudaFree(s.dN);
        cudaFree(s.dWs);
        cudaFreeHost(s.hT);
        cudaFreeHost(s.hP);
        cudaFreeHost(s.hY);
        cudaFreeHost(s.hO);
        cudaFreeHost(s.hStatus);
        cudaFreeHost(s.hN);
    }
    delete S;
}

}  // namespace chem

using namespace chem;

extern "C" chem_status chem_serve_create(const chem_mech *const *mechs, int32_t n_mechs,
                                         size_t hbm_budget, void **server)
{
    clear_error();
    if (!server) return set_error(CHEM_EINVAL, "server is NULL");
    *server = nullptr;
    if (!mechs || n_mechs < 1) return set_error(CHEM_EINVAL, "need at least one mechanism");
    int dev = -1;
    cudaGetDevice(&dev);
    Server *S = new (std::nothrow) Server();
    if (!S) return set_error(CHEM_ENOMEM, "host allocation failed");
    memset(&S->info, 0, sizeof S->info);
    S->device = dev;
    size_t ws_max = 0;
    for (int i = 0; i < n_mechs; ++i) {
        if (!mechs[i] || mechs[i]->device != dev) {
            delete S;
            return set_error(CHEM_EINVAL, "mechanism %d is NULL or on another device", i);
        }
        S->mechs.push_back(mechs[i]);
        if (mechs[i]->ns > S->ns_max) S->ns_max = mechs[i]->ns;
        const size_t w = integrate_workspace_bytes(mechs[i], (int64_t)1 << 30);
        if (w > ws_max) ws_max = w;
    }
    clear_error();
    // per slot: T, P, Y, omega (double-sized), status, count, integrator workspace
    const size_t per_cell = 2 * sizeof(double) + 2 * sizeof(double) * S->ns_max + sizeof(int32_t);
    const size_t per_slot = hbm_budget / kSlots;
    if (per_slot <= ws_max + 4096 || (per_slot - ws_max - 4096) / per_cell < (size_t)kMinBucket) {
        delete S;
        return set_error(CHEM_ENOMEM, "serve: budget %zu below %d slots of %lld cells", hbm_budget,
                         kSlots, (long long)kMinBucket);
    }
    int64_t cap = kMinBucket;
    while ((size_t)(cap * 2) <= (per_slot - ws_max - 4096) / per_cell) cap *= 2;
    S->cap = cap;
    cudaError_t e = cudaSuccess;
    auto ck = [&](cudaError_t x) {
        if (e == cudaSuccess && x != cudaSuccess) e = x;
    };
    const size_t nsm = (size_t)S->ns_max;
    for (int i = 0; i < kSlots && e == cudaSuccess; ++i) {
        Slot &s = S->slots[i];
        s.srv = S;
        s.index = i;
        ck(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
        ck(cudaMalloc(&s.dT, cap * sizeof(double)));
        ck(cudaMalloc(&s.dP, cap * sizeof(double)));
        ck(cudaMalloc(&s.dY, cap * nsm * sizeof(double)));
        ck(cudaMalloc(&s.dO, cap * nsm * sizeof(double)));
        ck(cudaMalloc((void **)&s.dStatus, cap * sizeof(int32_t)));
        ck(cudaMalloc((void **)&s.dN, sizeof(int64_t)));
        s.ws_bytes = ws_max;
        ck(cudaMalloc(&s.dWs, ws_max));
        ck(cudaMallocHost(&s.hT, cap * sizeof(double)));
        ck(cudaMallocHost(&s.hP, cap * sizeof(double)));
        ck(cudaMallocHost(&s.hY, cap * nsm * sizeof(double)));
        ck(cudaMallocHost(&s.hO, cap * nsm * sizeof(double)));
        ck(cudaMallocHost((void **)&s.hStatus, cap * sizeof(int32_t)));
        ck(cudaMallocHost((void **)&s.hN, sizeof(int64_t)));
        if (e != cudaSuccess) break;
        // rows past a batch's end are evaluated as padding of its size bucket: give them a
        // finite state (1000 K, 1 bar, all mass fractions zero) in both element types
        for (int64_t c = 0; c < cap; ++c) {
            ((double *)s.hT)[c] = 1000.0;
            ((double *)s.hP)[c] = 1e6;
        }
        ck(cudaMemcpy(s.dT, s.hT, cap * sizeof(double), cudaMemcpyHostToDevice));
        ck(cudaMemcpy(s.dP, s.hP, cap * sizeof(double), cudaMemcpyHostToDevice));
        ck(cudaMemset(s.dY, 0, cap * nsm * sizeof(double)));
        ck(cudaMemset(s.dN, 0, sizeof(int64_t)));
        S->device_bytes += 2 * cap * sizeof(double) + 2 * cap * nsm * sizeof(double) +
                           cap * sizeof(int32_t) + sizeof(int64_t) + ws_max;
    }
    if (e != cudaSuccess) {
        free_server(S);
        return set_error(CHEM_ENOMEM, "serve: allocation failed: %s", cudaGetErrorString(e));
    }
    // first (eager) launch of every kernel a graph may hold: sets kernel attributes outside
    // stream capture; the integrator reads a cell count of zero and returns at once
    Slot &s0 = S->slots[0];
    for (size_t i = 0; i < S->mechs.size(); ++i) {
        const chem_mech *m = S->mechs[i];
        for (int p = 0; p < 3; ++p) {
            if (p == CHEM_SPLIT_BF16 && !m->have_bf16) continue;
            chem_source_term(m, kMinBucket, s0.dT, s0.dP, s0.dY, m->ns, s0.dO, m->ns,
                             (chem_precision)p, s0.stream);
        }
        if (integrate_workspace_bytes(m, 1) > 0)
            integrate_launch(m, kMinBucket, s0.dN, (double *)s0.dT, (const double *)s0.dP,
                             (double *)s0.dY, m->ns, 1e-9, 1e-6, 1e-12, nullptr, s0.dStatus, s0.dWs,
                             s0.ws_bytes, s0.stream);
    }
    e = cudaStreamSynchronize(s0.stream);
    clear_error();
    if (e != cudaSuccess) {
        free_server(S);
        return set_error(CHEM_ECUDA, "serve: warm-up: %s", cudaGetErrorString(e));
    }
    S->info.n_slots = kSlots;
    S->info.slot_cells = cap;
    S->info.device_bytes = S->device_bytes;
    S->worker = std::thread([S] { S->run(); });
    *server = S;
    return CHEM_OK;
}

extern "C" chem_status chem_serve_submit(void *server, const chem_request *req, uint64_t *ticket)
{
    clear_error();
    Server *S = (Server *)server;
    if (!S || !req || !ticket) return set_error(CHEM_EINVAL, "NULL server, request or ticket");
    const chem_request &r = *req;
    if (r.mech_index < 0 || r.mech_index >= (int)S->mechs.size())
        return set_error(CHEM_EINVAL, "mech_index %d out of range", r.mech_index);
    const chem_mech *m = S->mechs[r.mech_index];
    if (r.n_cells < 1) return set_error(CHEM_EINVAL, "n_cells must be >= 1");
    if (!r.T || !r.P || !r.Y) return set_error(CHEM_EINVAL, "NULL T, P or Y");
    if (r.kind == CHEM_REQ_SOURCE) {
        if (r.precision != CHEM_FP64 && r.precision != CHEM_FP32 && r.precision != CHEM_SPLIT_BF16)
            return set_error(CHEM_EINVAL, "unknown precision %d", (int)r.precision);
        if (!r.omega) return set_error(CHEM_EINVAL, "NULL omega");
        if (r.precision == CHEM_SPLIT_BF16 && !m->have_bf16)
            return set_error(CHEM_EUNSUPPORTED, "split-BF16 path not available for this mechanism");
    } else if (r.kind == CHEM_REQ_INTEGRATE) {
        if (r.precision != CHEM_FP64) return set_error(CHEM_EINVAL, "integration requests are FP64");
        if (!r.T_out || !r.Y_out) return set_error(CHEM_EINVAL, "NULL T_out or Y_out");
        if (!(r.dt >= 0.0) || !(r.dt < 1e300) || !(r.rtol > 0.0) || !(r.atol >= 0.0))
            return set_error(CHEM_EINVAL, "need finite dt >= 0, rtol > 0, atol >= 0");
        if (r.fixed_steps < 0) return set_error(CHEM_EINVAL, "fixed_steps must be >= 0");
        if (integrate_workspace_bytes(m, 1) == 0)
            return set_error(CHEM_EUNSUPPORTED, "reactor kernels not available for this mechanism");
    } else {
        return set_error(CHEM_EINVAL, "unknown request kind %d", r.kind);
    }
    if (r.n_cells > S->cap)
        return set_error(CHEM_ENOMEM, "request of %lld cells exceeds the slot capacity %lld",
                         (long long)r.n_cells, (long long)S->cap);
    auto q = std::make_shared<Req>();
    q->r = r;
    q->ns = m->ns;
    q->t_submit = Clock::now();
    memset(&q->res, 0, sizeof q->res);
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stop) return set_error(CHEM_EBUSY, "server is stopping");
        q->id = S->next_id++;
        S->tickets[q->id] = q;
        S->queue.push_back(q);
        ++S->info.submitted;
        *ticket = q->id;
    }
    S->cv_work.notify_all();
    return CHEM_OK;
}

extern "C" chem_status chem_serve_poll(void *server, uint64_t ticket, chem_result *result,
                                       int64_t timeout_us)
{
    clear_error();
    Server *S = (Server *)server;
    if (!S) return set_error(CHEM_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return set_error(CHEM_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    std::shared_ptr<Req> q = it->second;
    if (!q->done) {
        if (timeout_us == 0) return CHEM_ENOTREADY;
        if (timeout_us < 0) {
            S->cv_done.wait(lk, [&] { return q->done || S->stop; });
        } else {
            S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us),
                                [&] { return q->done || S->stop; });
        }
        if (!q->done) {
            if (S->stop) return set_error(CHEM_EBUSY, "server is stopping");
            return set_error(CHEM_ETIMEOUT, "ticket %llu not done after %lld us",
                             (unsigned long long)ticket, (long long)timeout_us);
        }
    }
    if (result) *result = q->res;
    S->tickets.erase(ticket);
    return CHEM_OK;
}

extern "C" chem_status chem_serve_info_get(void *server, chem_serve_info *out)
{
    clear_error();
    Server *S = (Server *)server;
    if (!S || !out) return set_error(CHEM_EINVAL, "NULL server or info");
    std::lock_guard<std::mutex> g(S->mu);
    *out = S->info;
    return CHEM_OK;
}

extern "C" chem_status chem_serve_destroy(void *server)
{
    clear_error();
    Server *S = (Server *)server;
    if (!S) return CHEM_OK;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        S->queue.clear();
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (Slot &s : S->slots)
        if (s.stream) cudaStreamSynchronize(s.stream);
    free_server(S);
    return CHEM_OK;
}
