// chem_serve.cu -- persistent serving loop: many host producers (simulated CFD ranks, the
// paper's offload pattern, Secs. 1 and 3.2) submit source-term and integration requests of
// uneven sizes; one worker thread batches them onto streams ("lanes") and replays captured
// CUDA graphs.
//
// Memory: the HBM budget is one device allocation, carved per batch by a first-fit arena
// (256-byte aligned blocks, freed blocks coalesced), with a page-locked host mirror of the
// same size whose block at the same offset is the batch's staging.  A batch holds exactly
// the bytes its cells need (inputs, outputs, per-cell status and step counts, and the
// integrator workspace for its cell count) from launch to retirement.
//
// SMs: two partitions, 16 SMs for lanes 0 and 1 (source-term batches only) and the rest for
// lanes 2 and 3 (integrations; source-term batches while no integration is queued or
// running there), as green contexts when the driver provides them, else only through the
// grids of the persistent kernels (bounded by tl_sm_limit while a batch is recorded).  The
// reactor and split-precision kernels hold their SMs for a whole batch, so without the split
// a source-term request would wait for a running integration to end.
//
// Life of a request: submit() validates it (a request whose bytes exceed the whole budget
// is refused) and appends it to the queue.  When a lane is free the worker takes the oldest
// queued request that lane may run,
// adds later queued requests with the same batch key (mechanism, kind, precision, dt,
// tolerances) while the batch stays within its cell limit and the arena's largest free
// block, and takes the batch's block.  If even the oldest request does not fit in the free
// memory now, it waits (in order) until a batch retires and frees its block.  The batch is
// packed into its staging, copied to the device, run by the lane's graph for its key (the
// first batch of a key captures it; later batches capture the launch with their own
// pointers and cell count and update the executable graph in place, re-instantiating only
// if the update is refused), copied back, and a host callback wakes the worker, which
// copies each request's rows to the caller's arrays and releases its waiters.  Batches on
// different lanes overlap on the device: requests that arrive while the GPU is busy are
// admitted as soon as a lane and memory free up (continuous batching).
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

#include <cuda.h>

#include "chem_arena.h"
#include "chem_internal.h"

namespace chem {

using Clock = std::chrono::steady_clock;

constexpr int kLanes = 4;            // lanes 0, 1: source-term partition; 2, 3: integration
constexpr int kSourceSMs = 16;       // SMs of the source-term partition (a multiple of 8)
constexpr int64_t kSourceBatch = (int64_t)1 << 20;   // cells per source-term batch, at most
constexpr int64_t kIntegBatch = 65536;               // cells per integration batch, at most
constexpr size_t kAlign = 256;

static size_t align_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

struct Req {
    uint64_t id = 0;
    chem_request r;
    int ns = 0;
    Clock::time_point t_submit, t_launch;
    bool done = false;
    bool mem_wait = false;            // counted once in info.memory_waits
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

static size_t elt_of(int prec) { return prec == CHEM_FP64 ? sizeof(double) : sizeof(float); }

// Byte offsets of one batch's buffers inside its arena block.
struct BatchLayout {
    size_t T = 0, P = 0, Y = 0, O = 0, status = 0, nacc = 0, nrej = 0, n = 0, ws = 0;
    size_t ws_bytes = 0, total = 0;
};

static BatchLayout layout_of(const chem_mech *m, const BatchKey &k, int64_t cells)
{
    BatchLayout L;
    const size_t c = (size_t)cells, ns = (size_t)m->ns;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align_up(bytes);
        return at;
    };
    if (k.kind == CHEM_REQ_SOURCE) {
        const size_t e = elt_of(k.prec);
        L.T = take(c * e);
        L.P = take(c * e);
        L.Y = take(c * ns * e);
        L.O = take(c * ns * e);
    } else {
        L.T = take(c * sizeof(double));
        L.P = take(c * sizeof(double));
        L.Y = take(c * ns * sizeof(double));
        L.status = take(c * sizeof(int32_t));
        L.nacc = take(c * sizeof(int32_t));
        L.nrej = take(c * sizeof(int32_t));
        L.n = take(sizeof(int64_t));
        L.ws_bytes = integrate_workspace_bytes(m, cells);
        L.ws = take(L.ws_bytes);
    }
    L.total = o;
    return L;
}

struct Server;

struct Lane {
    Server *srv = nullptr;
    int index = 0;
    int part = 0;                     // SM partition: 0 source term, 1 integration
    cudaStream_t stream = nullptr;
    // the batch in flight
    bool busy = false, ready = false;
    chem_status launch_status = CHEM_OK;
    BatchKey key;
    std::vector<std::shared_ptr<Req>> members;
    std::vector<int64_t> offsets;
    int64_t cells = 0;
    size_t off = 0;                   // its arena block
    BatchLayout lay;
    std::map<BatchKey, cudaGraphExec_t> graphs;
};

struct Server {
    std::vector<const chem_mech *> mechs;
    int device = 0;
    size_t budget = 0;
    unsigned char *dbase = nullptr;   // device block of the budget
    unsigned char *hbase = nullptr;   // its page-locked host mirror
    Arena arena;
    Lane lanes[kLanes];
    // SM partitions: green contexts when the driver provides them, else grid limits only
    bool green = false;
    CUgreenCtx gctx[2] = {nullptr, nullptr};
    int part_sms[2] = {0, 0};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Req>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Req>> tickets;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    chem_serve_info info;

    void run();
    bool admit(Lane &l);
    void launch(Lane &l);
    void retire(Lane &l);
};

// ---- SM partitions (driver entry points looked up at run time: nothing links libcuda)

template <typename F>
static bool drv_fn(const char *name, F &f)
{
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion(name, &ptr, 12080, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !ptr) {
        (void)cudaGetLastError();
        return false;
    }
    f = (F)ptr;
    return true;
}

struct GreenApi {
    CUresult (*dev_get)(CUdevice *, int) = nullptr;
    CUresult (*get_res)(CUdevice, CUdevResource *, CUdevResourceType) = nullptr;
    CUresult (*split)(CUdevResource *, unsigned int *, const CUdevResource *, CUdevResource *,
                      unsigned int, unsigned int) = nullptr;
    CUresult (*gen_desc)(CUdevResourceDesc *, CUdevResource *, unsigned int) = nullptr;
    CUresult (*create)(CUgreenCtx *, CUdevResourceDesc, CUdevice, unsigned int) = nullptr;
    CUresult (*destroy)(CUgreenCtx) = nullptr;
    CUresult (*stream)(CUstream *, CUgreenCtx, unsigned int, int) = nullptr;
    bool load()
    {
        return drv_fn("cuDeviceGet", dev_get) && drv_fn("cuDeviceGetDevResource", get_res) &&
               drv_fn("cuDevSmResourceSplitByCount", split) &&
               drv_fn("cuDevResourceGenerateDesc", gen_desc) && drv_fn("cuGreenCtxCreate", create) &&
               drv_fn("cuGreenCtxDestroy", destroy) && drv_fn("cuGreenCtxStreamCreate", stream);
    }
};

static GreenApi &green_api()
{
    static GreenApi g;
    static bool ok = g.load();
    if (!ok) g = GreenApi();
    return g;
}

// Two green contexts on the server's device: kSourceSMs SMs for source-term batches and the
// rest for integrations.  false, with nothing left created, when the driver cannot.
static bool make_partitions(Server *S)
{
    GreenApi &g = green_api();
    if (!g.create) return false;
    CUdevice cd;
    CUdevResource all, src, rest;
    memset(&all, 0, sizeof all);
    memset(&src, 0, sizeof src);
    memset(&rest, 0, sizeof rest);
    unsigned int ng = 1;
    CUdevResourceDesc d0 = nullptr, d1 = nullptr;
    if (g.dev_get(&cd, S->device) != CUDA_SUCCESS ||
        g.get_res(cd, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS ||
        all.sm.smCount < 2u * kSourceSMs ||
        g.split(&src, &ng, &all, &rest, 0, kSourceSMs) != CUDA_SUCCESS || ng != 1 ||
        rest.sm.smCount == 0 || g.gen_desc(&d0, &src, 1) != CUDA_SUCCESS ||
        g.gen_desc(&d1, &rest, 1) != CUDA_SUCCESS)
        return false;
    if (g.create(&S->gctx[0], d0, cd, CU_GREEN_CTX_DEFAULT_STREAM) != CUDA_SUCCESS) {
        S->gctx[0] = nullptr;
        return false;
    }
    if (g.create(&S->gctx[1], d1, cd, CU_GREEN_CTX_DEFAULT_STREAM) != CUDA_SUCCESS) {
        g.destroy(S->gctx[0]);
        S->gctx[0] = S->gctx[1] = nullptr;
        return false;
    }
    S->part_sms[0] = (int)src.sm.smCount;
    S->part_sms[1] = (int)rest.sm.smCount;
    return true;
}

static void drop_partitions(Server *S)
{
    for (CUgreenCtx &c : S->gctx)
        if (c) {
            green_api().destroy(c);
            c = nullptr;
        }
}

static void CUDART_CB on_lane_done(void *arg)
{
    Lane *l = (Lane *)arg;
    {
        std::lock_guard<std::mutex> g(l->srv->mu);
        l->ready = true;
    }
    l->srv->cv_work.notify_all();
}

// Record the batch's work on the lane's stream (kernels only: the graph's contents).
static chem_status record_batch(const chem_mech *m, const BatchKey &k, int64_t cells,
                                unsigned char *d, const BatchLayout &L, cudaStream_t s)
{
    const int ns = m->ns;
    if (k.kind == CHEM_REQ_SOURCE)
        return chem_source_term(m, cells, d + L.T, d + L.P, d + L.Y, ns, d + L.O, ns,
                                (chem_precision)k.prec, s);
    chem_integrate_opts o;
    memset(&o, 0, sizeof o);
    o.fixed_steps = k.fixed;
    o.n_accepted = (int32_t *)(d + L.nacc);
    o.n_rejected = (int32_t *)(d + L.nrej);
    return integrate_launch(m, cells, (const int64_t *)(d + L.n), (double *)(d + L.T),
                            (const double *)(d + L.P), (double *)(d + L.Y), ns, k.dt, k.rtol,
                            k.atol, &o, (int32_t *)(d + L.status), d + L.ws, L.ws_bytes, s);
}

// Enqueue the lane's batch (members, key and block already set).  Called without the lock.
void Server::launch(Lane &l)
{
    const BatchKey &k = l.key;
    const chem_mech *m = mechs[k.mech];
    const int ns = m->ns;
    const size_t elt = k.kind == CHEM_REQ_SOURCE ? elt_of(k.prec) : sizeof(double);
    const BatchLayout &L = l.lay;
    unsigned char *d = dbase + l.off, *h = hbase + l.off;
    int64_t o = 0;
    l.offsets.clear();
    for (auto &q : l.members) {
        const int64_t n = q->r.n_cells;
        l.offsets.push_back(o);
        memcpy(h + L.T + o * elt, q->r.T, n * elt);
        memcpy(h + L.P + o * elt, q->r.P, n * elt);
        memcpy(h + L.Y + o * ns * elt, q->r.Y, n * ns * elt);
        o += n;
    }
    l.cells = o;
    cudaError_t e = cudaSuccess;
    chem_status st = CHEM_OK;
    auto ck = [&](cudaError_t x) {
        if (e == cudaSuccess && x != cudaSuccess) e = x;
    };
    cudaStream_t s = l.stream;
    ck(cudaMemcpyAsync(d + L.T, h + L.T, o * elt, cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(d + L.P, h + L.P, o * elt, cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(d + L.Y, h + L.Y, o * ns * elt, cudaMemcpyHostToDevice, s));
    if (k.kind == CHEM_REQ_INTEGRATE) {
        memcpy(h + L.n, &o, sizeof o);
        ck(cudaMemcpyAsync(d + L.n, h + L.n, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    }
    bool captured = false, updated = false;
    if (e == cudaSuccess) {
        // the batch's kernels as a graph with this batch's pointers and cell count
        cudaGraph_t g = nullptr;
        ck(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        if (e == cudaSuccess) {
            tl_sm_limit = part_sms[l.part];
            st = record_batch(m, k, o, d, L, s);
            tl_sm_limit = 0;
            cudaError_t ec = cudaStreamEndCapture(s, &g);
            if (st == CHEM_OK) ck(ec);
        }
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess && st == CHEM_OK) {
            auto it = l.graphs.find(k);
            if (it != l.graphs.end()) {
                cudaGraphExecUpdateResultInfo ui;
                if (cudaGraphExecUpdate(it->second, g, &ui) == cudaSuccess) {
                    exec = it->second;
                    updated = true;
                } else {
                    (void)cudaGetLastError();
                    cudaGraphExecDestroy(it->second);
                    l.graphs.erase(it);
                }
            }
            if (!exec) {
                ck(cudaGraphInstantiate(&exec, g, 0));
                if (e == cudaSuccess) {
                    l.graphs[k] = exec;
                    captured = true;
                }
            }
        }
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess && st == CHEM_OK) ck(cudaGraphLaunch(exec, s));
    }
    if (e == cudaSuccess && st == CHEM_OK) {
        if (k.kind == CHEM_REQ_SOURCE) {
            ck(cudaMemcpyAsync(h + L.O, d + L.O, o * ns * elt, cudaMemcpyDeviceToHost, s));
        } else {
            ck(cudaMemcpyAsync(h + L.T, d + L.T, o * elt, cudaMemcpyDeviceToHost, s));
            ck(cudaMemcpyAsync(h + L.Y, d + L.Y, o * ns * elt, cudaMemcpyDeviceToHost, s));
            // status, accepted and rejected step counts: three adjacent int32 arrays
            ck(cudaMemcpyAsync(h + L.status, d + L.status, L.n - L.status, cudaMemcpyDeviceToHost, s));
        }
        ck(cudaLaunchHostFunc(s, on_lane_done, &l));
    }
    if (e != cudaSuccess && st == CHEM_OK) st = set_error(CHEM_ECUDA, "serve: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lg(mu);
    if (captured) ++info.graphs_captured;
    if (updated) ++info.graph_updates;
    if (st == CHEM_OK) ++info.graph_launches;
    l.launch_status = st;
    if (st != CHEM_OK) l.ready = true;      // nothing in flight: retire at once
}

// Copy results out, complete the members and free the batch's block.  Called without the
// lock.
void Server::retire(Lane &l)
{
    const BatchKey &k = l.key;
    const int ns = mechs[k.mech]->ns;
    const size_t elt = k.kind == CHEM_REQ_SOURCE ? elt_of(k.prec) : sizeof(double);
    const BatchLayout &L = l.lay;
    const unsigned char *h = hbase + l.off;
    chem_status st = l.launch_status;
    if (st == CHEM_OK) {
        cudaError_t e = cudaStreamSynchronize(l.stream);     // already complete: cheap
        if (e != cudaSuccess) st = set_error(CHEM_ECUDA, "serve: %s", cudaGetErrorString(e));
    }
    const auto now = Clock::now();
    const int32_t *hst = (const int32_t *)(h + L.status), *hacc = (const int32_t *)(h + L.nacc),
                  *hrej = (const int32_t *)(h + L.nrej);
    for (size_t i = 0; i < l.members.size(); ++i) {
        Req &q = *l.members[i];
        const int64_t o = l.offsets.size() > i ? l.offsets[i] : 0, n = q.r.n_cells;
        int32_t failed = 0;
        int64_t acc = 0, rej = 0;
        if (st == CHEM_OK) {
            if (k.kind == CHEM_REQ_SOURCE) {
                memcpy(q.r.omega, h + L.O + o * ns * elt, n * ns * elt);
            } else {
                memcpy(q.r.T_out, h + L.T + o * elt, n * sizeof(double));
                memcpy(q.r.Y_out, h + L.Y + o * ns * elt, n * ns * sizeof(double));
                for (int64_t c = 0; c < n; ++c) {
                    failed += hst[o + c] != CHEM_CELL_OK;
                    acc += hacc[o + c];
                    rej += hrej[o + c];
                }
                if (q.r.cell_status) memcpy(q.r.cell_status, hst + o, n * sizeof(int32_t));
            }
        }
        q.res.status = st != CHEM_OK ? st : (failed ? CHEM_ENONCONV : CHEM_OK);
        q.res.n_failed = failed;
        q.res.n_cells = n;
        q.res.batch_cells = l.cells;
        q.res.batch_requests = (int32_t)l.members.size();
        q.res.slot = l.index;
        q.res.queue_us = std::chrono::duration<double, std::micro>(q.t_launch - q.t_submit).count();
        q.res.latency_us = std::chrono::duration<double, std::micro>(now - q.t_submit).count();
        q.res.steps_accepted = acc;
        q.res.steps_rejected = rej;
    }
    std::lock_guard<std::mutex> lg(mu);
    for (auto &q : l.members) q->done = true;
    info.completed += l.members.size();
    arena.release(l.off, l.lay.total);
    info.bytes_in_use = arena.in_use;
    l.members.clear();
    l.busy = false;
    l.ready = false;
    cv_done.notify_all();
}

// Form a batch for a free lane from the queue (lock held).  false: nothing this lane may
// run, or the oldest request it may run does not fit in the free memory yet.
bool Server::admit(Lane &l)
{
    // source-term lanes take source-term requests; integration lanes take integrations, and
    // source-term requests only while no integration is queued or running on them
    auto head = queue.begin();
    if (l.part == 0) {
        while (head != queue.end() && (*head)->r.kind != CHEM_REQ_SOURCE) ++head;
    } else {
        bool integ = false;
        for (const Lane &o : lanes) integ |= o.part == 1 && o.busy && o.key.kind == CHEM_REQ_INTEGRATE;
        for (auto it = queue.begin(); !integ && it != queue.end(); ++it)
            integ = (*it)->r.kind == CHEM_REQ_INTEGRATE;
        if (integ)
            while (head != queue.end() && (*head)->r.kind != CHEM_REQ_INTEGRATE) ++head;
    }
    if (head == queue.end()) return false;
    const BatchKey key = key_of((*head)->r);
    const chem_mech *m = mechs[key.mech];
    const int64_t limit = key.kind == CHEM_REQ_INTEGRATE ? kIntegBatch : kSourceBatch;
    // the oldest request already waiting for memory keeps its bytes reserved: other batches
    // only use what the largest free block holds beyond them, so that a steady stream of
    // small batches on other lanes cannot hold it off
    size_t room = arena.largest_free();
    for (const auto &q : queue) {
        if (!q->mem_wait) continue;
        if (q.get() != head->get()) {
            const size_t need = layout_of(mechs[q->r.mech_index], key_of(q->r), q->r.n_cells).total;
            room = room > need ? room - need : 0;
        }
        break;
    }
    if (layout_of(m, key, (*head)->r.n_cells).total > room) {
        if (!(*head)->mem_wait) {
            (*head)->mem_wait = true;
            ++info.memory_waits;
        }
        return false;
    }
    l.members.clear();
    int64_t cells = 0;
    for (auto it = head; it != queue.end();) {
        const Req &q = **it;
        const int64_t c2 = cells + q.r.n_cells;
        if (key_of(q.r) == key && (cells == 0 || (c2 <= limit && layout_of(m, key, c2).total <= room))) {
            cells = c2;
            l.members.push_back(*it);
            it = queue.erase(it);
        } else {
            ++it;
        }
    }
    l.lay = layout_of(m, key, cells);
    if (!arena.alloc(l.lay.total, l.off)) {    // cannot happen: the block fits in `room`
        for (auto rit = l.members.rbegin(); rit != l.members.rend(); ++rit) queue.push_front(*rit);
        l.members.clear();
        return false;
    }
    if (arena.in_use > info.bytes_in_use_max) info.bytes_in_use_max = arena.in_use;
    info.bytes_in_use = arena.in_use;
    const auto now = Clock::now();
    for (auto &q : l.members) q->t_launch = now;
    l.key = key;
    l.busy = true;
    l.ready = false;
    ++info.batches;
    if ((int32_t)l.members.size() > info.max_batch_requests)
        info.max_batch_requests = (int32_t)l.members.size();
    return true;
}

void Server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        // retire completed lanes (frees their memory before admission)
        for (Lane &l : lanes) {
            if (l.busy && l.ready) {
                lk.unlock();
                retire(l);
                lk.lock();
            }
        }
        bool any_busy = false;
        for (Lane &l : lanes) any_busy |= l.busy;
        if (stop && !any_busy) break;
        // admit queued requests into free lanes
        bool launched = false;
        if (!stop) {
            for (Lane &l : lanes) {
                if (l.busy || queue.empty() || !admit(l)) continue;
                lk.unlock();
                launch(l);
                lk.lock();
                launched = true;
            }
        }
        if (launched) continue;
        bool pending_ready = false;
        for (Lane &l : lanes) pending_ready |= l.busy && l.ready;
        if (pending_ready) continue;
        // nothing could be launched (queue empty, no free lane, the oldest request waiting
        // for memory, or only integrations queued while the source-term lane is the free
        // one): sleep until a submission or a completion (bounded, as a safety net)
        cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
}

static void free_server(Server *S)
{
    for (Lane &l : S->lanes) {
        for (auto &kv : l.graphs) cudaGraphExecDestroy(kv.second);
        l.graphs.clear();
        if (l.stream) cudaStreamDestroy(l.stream);
    }
    drop_partitions(S);
    cudaFree(S->dbase);
    cudaFreeHost(S->hbase);
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
    // warm-up block: 64 cells of the largest layout any mechanism and kind needs
    size_t warm = 0;
    for (int i = 0; i < n_mechs; ++i) {
        if (!mechs[i] || mechs[i]->device != dev) {
            delete S;
            return set_error(CHEM_EINVAL, "mechanism %d is NULL or on another device", i);
        }
        S->mechs.push_back(mechs[i]);
        BatchKey k;
        k.kind = CHEM_REQ_SOURCE;
        k.prec = CHEM_FP64;
        warm = std::max(warm, layout_of(mechs[i], k, 64).total);
        k.kind = CHEM_REQ_INTEGRATE;
        if (integrate_workspace_bytes(mechs[i], 1) > 0) warm = std::max(warm, layout_of(mechs[i], k, 64).total);
    }
    clear_error();
    const size_t budget = hbm_budget / kAlign * kAlign;
    if (budget < warm) {
        delete S;
        return set_error(CHEM_ENOMEM, "serve: budget %zu below one batch of 64 cells (%zu bytes)",
                         hbm_budget, warm);
    }
    cudaError_t e = cudaSuccess;
    auto ck = [&](cudaError_t x) {
        if (e == cudaSuccess && x != cudaSuccess) e = x;
    };
    ck(cudaMalloc((void **)&S->dbase, budget));
    ck(cudaMallocHost((void **)&S->hbase, budget));
    // SM partitions: green contexts whose streams run only on their SMs, checked with one
    // device-to-device copy between buffers of this context on each partition's stream;
    // otherwise plain streams, and the partition is kept by the persistent kernels' grids
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && make_partitions(S)) {
        bool good = true;
        for (int i = 0; i < kLanes && good; ++i) {
            Lane &l = S->lanes[i];
            l.part = i < kLanes / 2 ? 0 : 1;
            CUstream cs = nullptr;
            good = green_api().stream(&cs, S->gctx[l.part], CU_STREAM_NON_BLOCKING, 0) == CUDA_SUCCESS;
            l.stream = (cudaStream_t)cs;
            if (good) {
                const uint32_t pat = 0x5EED0000u + (uint32_t)i;
                uint32_t back = 0;
                good = cudaMemcpy(S->dbase, &pat, sizeof pat, cudaMemcpyHostToDevice) == cudaSuccess &&
                       cudaMemcpyAsync(S->dbase + kAlign, S->dbase, sizeof pat, cudaMemcpyDeviceToDevice,
                                       l.stream) == cudaSuccess &&
                       cudaStreamSynchronize(l.stream) == cudaSuccess &&
                       cudaMemcpy(&back, S->dbase + kAlign, sizeof back, cudaMemcpyDeviceToHost) == cudaSuccess &&
                       back == pat;
            }
        }
        if (!good) {
            (void)cudaGetLastError();
            for (Lane &l : S->lanes)
                if (l.stream) {
                    cudaStreamDestroy(l.stream);
                    l.stream = nullptr;
                }
            drop_partitions(S);
        } else {
            S->green = true;
        }
    }
    if (!S->green) {
        S->part_sms[0] = kSourceSMs < nsm ? kSourceSMs : nsm;
        S->part_sms[1] = nsm > 2 * kSourceSMs ? nsm - kSourceSMs : nsm;
    }
    for (int i = 0; i < kLanes && e == cudaSuccess; ++i) {
        Lane &l = S->lanes[i];
        l.srv = S;
        l.index = i;
        l.part = i < kLanes / 2 ? 0 : 1;
        if (!l.stream) ck(cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking));
    }
    if (e != cudaSuccess) {
        free_server(S);
        return set_error(CHEM_ENOMEM, "serve: allocation failed: %s", cudaGetErrorString(e));
    }
    S->budget = budget;
    S->arena.init(budget);
    // first (eager) launch of every kernel a graph may hold, outside stream capture (sets
    // kernel attributes); 64 finite cells (1000 K, 1 bar, all mass fractions zero)
    {
        Lane &l0 = S->lanes[0];
        for (size_t i = 0; i < S->mechs.size() && e == cudaSuccess; ++i) {
            const chem_mech *m = S->mechs[i];
            for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
                BatchKey k;
                k.kind = kind;
                k.dt = 1e-9;
                k.rtol = 1e-6;
                k.atol = 1e-12;
                if (kind == CHEM_REQ_INTEGRATE && integrate_workspace_bytes(m, 1) == 0) continue;
                for (int p = 0; p < (kind == CHEM_REQ_SOURCE ? 3 : 1); ++p) {
                    if (p == CHEM_SPLIT_BF16 && !m->have_bf16) continue;
                    k.prec = p;
                    const BatchLayout L = layout_of(m, k, 64);
                    const size_t el = kind == CHEM_REQ_SOURCE ? elt_of(p) : sizeof(double);
                    for (int c = 0; c < 64; ++c) {
                        if (el == sizeof(double)) {
                            ((double *)(S->hbase + L.T))[c] = 1000.0;
                            ((double *)(S->hbase + L.P))[c] = 1e6;
                        } else {
                            ((float *)(S->hbase + L.T))[c] = 1000.0f;
                            ((float *)(S->hbase + L.P))[c] = 1e6f;
                        }
                    }
                    memset(S->hbase + L.Y, 0, 64 * m->ns * el);
                    const int64_t zero = 0;
                    memcpy(S->hbase + L.n, &zero, sizeof zero);   // integrator: no cells
                    ck(cudaMemcpyAsync(S->dbase, S->hbase, L.total, cudaMemcpyHostToDevice, l0.stream));
                    Lane &lw = S->lanes[kind == CHEM_REQ_SOURCE ? 0 : kLanes / 2];
                    ck(cudaStreamSynchronize(l0.stream));
                    tl_sm_limit = S->part_sms[lw.part];
                    if (e == cudaSuccess) record_batch(m, k, 64, S->dbase, L, lw.stream);
                    tl_sm_limit = 0;
                    ck(cudaStreamSynchronize(lw.stream));
                }
            }
        }
    }
    clear_error();
    if (e != cudaSuccess) {
        free_server(S);
        return set_error(CHEM_ECUDA, "serve: warm-up: %s", cudaGetErrorString(e));
    }
    S->info.n_slots = kLanes;
    S->info.source_sms = S->part_sms[0];
    S->info.integrate_sms = S->part_sms[1];
    S->info.green_contexts = S->green ? 1 : 0;
    S->info.slot_cells = kSourceBatch;
    S->info.device_bytes = budget;
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
    const size_t need = layout_of(m, key_of(r), r.n_cells).total;
    if (need > S->budget)
        return set_error(CHEM_ENOMEM, "request of %lld cells needs %zu bytes, above the budget %zu",
                         (long long)r.n_cells, need, S->budget);
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
    for (Lane &l : S->lanes)
        if (l.stream) cudaStreamSynchronize(l.stream);
    free_server(S);
    return CHEM_OK;
}
