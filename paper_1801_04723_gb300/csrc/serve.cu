// Serving: inversion requests admitted continuously by device-memory
// footprint, batched as they arrive, and run concurrently on a pool of CUDA
// streams.
//
// A request (A, n, precision, tol) waits in a FIFO queue until a slot is
// free and its footprint (device copy of A when A is in host memory, the
// result X, and the inversion workspace) fits the server's HBM budget; it
// then runs on that slot's stream while other requests run on theirs, so
// requests that arrive while others are on the GPU overlap with them.
//
// Continuous batching: a request of order n <= batch_max_order is padded
// with the identity to np, the next multiple of 32 ([[A, 0], [0, I]] has
// inverse [[A^-1, 0], [0, I]], and the recursion keeps the cross blocks
// exactly zero).  When a slot takes such a request it also takes every
// queued request with the same padded order, precision and tolerance (up to
// max_batch, as long as the budget holds) and runs them as one lockstep
// batched recursion (the many-block parallelism of Alg. 2, Sec. 3.3): one
// launch per product and per leaf for the whole group.  A batchable request
// always takes this path, even alone, and every decision in it is per
// matrix, so its result does not depend on which requests it was batched
// with.  Results stay in device memory (counted against the budget) until
// the client polls them.  Memory comes from a stream-ordered pool
// (cudaMallocAsync), so admission does not synchronise the device.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace spin {
namespace {

using Clock = std::chrono::steady_clock;

constexpr int kPadMultiple = 32;
constexpr int kDefaultMaxBatch = 64;
constexpr int64_t kDefaultBatchMaxOrder = 1024;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
    uint64_t ticket;
    const double* A;
    int64_t lda, n;
    int64_t np;             // padded order when batchable, else 0
    bool a_on_device;
    int precision;
    double tol;
    size_t footprint_run;   // released when the run ends (staged A + workspace)
    size_t footprint_keep;  // released when the client polls (X)
    size_t share;           // batchable: staged A and padded copies (the group workspace is counted apart)
    Clock::time_point t_submit, t_start, t_end;
    double* X = nullptr;    // device, n x n, owned by the server until polled
    spin_info info{};
    int status = SPIN_ERR_BUSY;
    bool done = false;
    int deferrals = 0;      // times put back in the queue for lack of device memory
    int batch = 0;          // requests in the launch group it ran in
};

}  // namespace
}  // namespace spin

struct spin_server {
    spin_serve_cfg cfg;
    int max_batch = 1;
    int64_t batch_max_order = 0;
    int device = 0;
    cudaMemPool_t pool = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<spin::Request>> queue;
    std::map<uint64_t, std::shared_ptr<spin::Request>> table;
    size_t in_use = 0;
    size_t queued_a_bytes = 0;  // n*n*8 of every queued (not yet admitted) request
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;       // per slot, default priority
    std::vector<cudaStream_t> hi_streams;    // per slot, high priority (small requests)
    cudaStream_t copy_stream = nullptr;
    // counters
    uint64_t submitted = 0, completed = 0, rejected = 0, shed = 0, deferred = 0;
    uint64_t groups = 0, grouped = 0;  // batched launch groups run, requests they held
    int max_group = 0;
    // test hook (SPIN_SERVE_INJECT_OOM="ticket:count", read at creation): the
    // first count allocation attempts of that ticket fail as if the device
    // were out of memory
    uint64_t inject_ticket = 0;
    int inject_left = 0;
    int running = 0, peak_running = 0;
    // a request whose memory could not be allocated waits at the head of the
    // queue until another request completes (completed > retry_after)
    uint64_t retry_after = 0;
    bool retry_wait = false;
};

namespace spin {
namespace {

bool verbose() {
    static const bool v = getenv("SPIN_VERBOSE") != nullptr;
    return v;
}

spin_opts request_opts(int precision, double tol) {
    spin_opts o = spin_opts_default();
    o.precision = precision;
    o.tol = tol;
    return o;
}

size_t request_workspace(int64_t n, int precision, double tol) {
    spin_opts o = request_opts(precision, tol);
    return spin_workspace_bytes(n, &o);
}

int64_t padded_order(int64_t n) { return (n + kPadMultiple - 1) / kPadMultiple * kPadMultiple; }

bool same_group(const Request& a, const Request& b) {
    return a.np > 0 && a.np == b.np && a.precision == b.precision && a.tol == b.tol;
}

// Device bytes of a launch group held until it ends: every member's share
// plus the group's batched workspace.
size_t group_run_bytes(const std::vector<std::shared_ptr<Request>>& g) {
    size_t b = 0;
    for (auto& r : g) b += r->share;
    const spin_opts o = request_opts(g[0]->precision, g[0]->tol);
    return b + bucket_bytes(g[0]->np, (int)g.size(), o);
}

// Device memory of one launch group, from the server's pool on stream s.
struct GroupMem {
    std::vector<double*> staged, apad, xpad;  // per member (nullptr when not needed)
    void* ws = nullptr;
    size_t ws_bytes = 0;
};

void release_group(std::vector<std::shared_ptr<Request>>& g, GroupMem& m, cudaStream_t s, bool drop_x) {
    cudaGetLastError();
    for (size_t i = 0; i < g.size(); i++) {
        if (i < m.staged.size() && m.staged[i]) cudaFreeAsync(m.staged[i], s);
        if (i < m.apad.size() && m.apad[i]) cudaFreeAsync(m.apad[i], s);
        if (i < m.xpad.size() && m.xpad[i]) cudaFreeAsync(m.xpad[i], s);
        if (drop_x && g[i]->X) {
            cudaFreeAsync(g[i]->X, s);
            g[i]->X = nullptr;
        }
    }
    if (m.ws) cudaFreeAsync(m.ws, s);
    m = GroupMem();
}

// One allocation attempt for the whole group (false: something failed).
bool alloc_group(spin_server* sv, std::vector<std::shared_ptr<Request>>& g, GroupMem& m, bool batched,
                 cudaStream_t s) {
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (auto& r : g)
            if (r->ticket == sv->inject_ticket && sv->inject_left > 0) {
                sv->inject_left--;
                return false;
            }
    }
    const size_t k = g.size();
    m.staged.assign(k, nullptr);
    m.apad.assign(k, nullptr);
    m.xpad.assign(k, nullptr);
    for (size_t i = 0; i < k; i++) {
        Request& r = *g[i];
        const size_t nn = (size_t)r.n * (size_t)r.n * sizeof(double);
        if (cudaMallocFromPoolAsync((void**)&r.X, nn, sv->pool, s) != cudaSuccess) return false;
        if (!r.a_on_device && cudaMallocFromPoolAsync((void**)&m.staged[i], nn, sv->pool, s) != cudaSuccess)
            return false;
        if (batched && r.np > r.n) {
            const size_t pp = (size_t)r.np * (size_t)r.np * sizeof(double);
            if (cudaMallocFromPoolAsync((void**)&m.apad[i], pp, sv->pool, s) != cudaSuccess) return false;
            if (cudaMallocFromPoolAsync((void**)&m.xpad[i], pp, sv->pool, s) != cudaSuccess) return false;
        }
    }
    const spin_opts o = request_opts(g[0]->precision, g[0]->tol);
    m.ws_bytes = batched ? bucket_bytes(g[0]->np, (int)k, o) : request_workspace(g[0]->n, o.precision, o.tol);
    if (m.ws_bytes && cudaMallocFromPoolAsync(&m.ws, m.ws_bytes, sv->pool, s) != cudaSuccess) return false;
    return true;
}

// Run one request alone on the single-matrix path (orders above
// batch_max_order, or batching off).  Returns the status.
int run_single(Request& r, GroupMem& m, cudaStream_t s) {
    const int64_t n = r.n;
    const double* Ause = r.A;
    int64_t lda = r.lda;
    if (!r.a_on_device) {
        if (cudaMemcpy2DAsync(m.staged[0], n * sizeof(double), r.A, r.lda * sizeof(double), n * sizeof(double), n,
                              cudaMemcpyHostToDevice, s) != cudaSuccess)
            return SPIN_ERR_CUDA;
        Ause = m.staged[0];
        lda = n;
    }
    spin_opts o = request_opts(r.precision, r.tol);
    o.blocking = 1;
    o.workspace = m.ws;
    o.workspace_bytes = m.ws_bytes;
    int rc = spin_invert_ex(Ause, lda, r.X, n, n, &o, &r.info, (spin_stream_t)s);
    if (rc == SPIN_OK || rc == SPIN_ERR_SINGULAR || rc == SPIN_ERR_NOT_CONVERGED) rc = r.info.status;
    return rc;
}

// Run a launch group (same padded order, precision and tolerance) as one
// batched recursion.  Enqueues everything, the copies of the results into
// each request's X included; the caller synchronises and then reads the
// statuses with bucket_result.
int run_group(std::vector<std::shared_ptr<Request>>& g, GroupMem& m, void* host_stage, cudaStream_t s) {
    const size_t k = g.size();
    const int64_t np = g[0]->np;
    std::vector<const double*> in(k);
    std::vector<int64_t> ld(k);
    std::vector<double*> out(k);
    std::vector<int> nv(k);
    for (size_t i = 0; i < k; i++) {
        Request& r = *g[i];
        const double* Ause = r.A;
        int64_t lda = r.lda;
        if (!r.a_on_device) {
            SPIN_CUDA_TRY(cudaMemcpy2DAsync(m.staged[i], r.n * sizeof(double), r.A, r.lda * sizeof(double),
                                            r.n * sizeof(double), r.n, cudaMemcpyHostToDevice, s));
            Ause = m.staged[i];
            lda = r.n;
        }
        if (np > r.n) {
            const int rc = launch_pad_identity(Ause, lda, r.n, m.apad[i], np, s);
            if (rc != SPIN_OK) return rc;
            in[i] = m.apad[i];
            ld[i] = np;
            out[i] = m.xpad[i];
        } else {
            in[i] = Ause;
            ld[i] = lda;
            out[i] = r.X;
        }
        nv[i] = (int)r.n;
    }
    const spin_opts o = request_opts(g[0]->precision, g[0]->tol);
    int rc = run_bucket(in.data(), ld.data(), out.data(), nv.data(), np, (int)k, o, m.ws, m.ws_bytes, host_stage, s);
    if (rc != SPIN_OK) return rc;
    for (size_t i = 0; i < k; i++) {
        Request& r = *g[i];
        if (np > r.n)
            SPIN_CUDA_TRY(cudaMemcpy2DAsync(r.X, r.n * sizeof(double), m.xpad[i], np * sizeof(double),
                                            r.n * sizeof(double), r.n, cudaMemcpyDeviceToDevice, s));
    }
    return SPIN_OK;
}

void worker_loop(spin_server* sv, int slot) {
    cudaSetDevice(sv->device);
    void* host_stage = nullptr;  // pinned: pointer upload and results of a launch group
    if (sv->max_batch > 1 && cudaMallocHost(&host_stage, bucket_host_bytes(sv->max_batch)) != cudaSuccess) {
        cudaGetLastError();
        host_stage = nullptr;  // every group then fails with SPIN_ERR_CUDA, loudly
    }
    while (true) {
        std::vector<std::shared_ptr<Request>> g;
        size_t keep = 0, run_bytes = 0;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait(lk, [&] {
                if (sv->stop) return true;
                if (sv->queue.empty()) return false;
                if (sv->retry_wait && sv->completed <= sv->retry_after && sv->running > 0) return false;
                const auto& h = sv->queue.front();
                return sv->in_use + h->footprint_run + h->footprint_keep <= sv->cfg.hbm_budget_bytes;
            });
            if (sv->stop) break;
            g.push_back(sv->queue.front());
            sv->queue.pop_front();
            sv->retry_wait = false;
            keep = g[0]->footprint_keep;
            run_bytes = g[0]->footprint_run;
            if (g[0]->np > 0) {
                // continuous batching: every queued request of the same group
                // key joins, while the budget holds
                for (auto it = sv->queue.begin(); it != sv->queue.end() && (int)g.size() < sv->max_batch;) {
                    if (!same_group(*g[0], **it)) {
                        ++it;
                        continue;
                    }
                    g.push_back(*it);
                    const size_t rb = group_run_bytes(g);
                    if (sv->in_use + keep + (*it)->footprint_keep + rb > sv->cfg.hbm_budget_bytes) {
                        g.pop_back();
                        break;
                    }
                    keep += (*it)->footprint_keep;
                    run_bytes = rb;
                    it = sv->queue.erase(it);
                }
            }
            for (auto& r : g) sv->queued_a_bytes -= (size_t)r->n * (size_t)r->n * sizeof(double);
            sv->in_use += keep + run_bytes;
            sv->running += (int)g.size();
            if (sv->running > sv->peak_running) sv->peak_running = sv->running;
        }
        const size_t k = g.size();
        const Clock::time_point t_start = Clock::now();
        const bool batched = g[0]->np > 0;
        for (auto& r : g) {
            r->t_start = t_start;
            r->batch = batched ? (int)k : 0;
        }
        const bool mixed = g[0]->precision != SPIN_FP64;
        const int64_t order = batched ? g[0]->np : g[0]->n;
        cudaStream_t s = (sv->cfg.priority_order > 0 && order <= sv->cfg.priority_order) ? sv->hi_streams[slot]
                                                                                           : sv->streams[slot];
        // The budget bounds what the server holds, but the device is shared
        // (the client's own tensors, other processes, and blocks the pool
        // keeps for reuse), so an allocation can still fail: release the
        // group's blocks, return the pool's unused memory to the device and
        // try once more; failing that, put the group back at the head of the
        // queue until another request completes, and fail it only when
        // nothing else is running.
        GroupMem m;
        int rc = SPIN_OK;
        if (!alloc_group(sv, g, m, batched, s)) {
            release_group(g, m, s, true);
            cudaStreamSynchronize(s);
            cudaMemPoolTrimTo(sv->pool, 0);
            if (!alloc_group(sv, g, m, batched, s)) {
                release_group(g, m, s, true);
                cudaStreamSynchronize(s);
                bool deferred = false;
                {
                    std::lock_guard<std::mutex> lk(sv->mu);
                    if (sv->running > (int)k && g[0]->deferrals < 1000) {
                        for (auto it = g.rbegin(); it != g.rend(); ++it) {
                            (*it)->deferrals++;
                            sv->queued_a_bytes += (size_t)(*it)->n * (size_t)(*it)->n * sizeof(double);
                            sv->queue.push_front(*it);
                        }
                        sv->deferred += k;
                        sv->in_use -= keep + run_bytes;
                        sv->running -= (int)k;
                        sv->retry_wait = true;
                        sv->retry_after = sv->completed;
                        deferred = true;
                    }
                }
                if (deferred) {
                    sv->cv.notify_all();
                    continue;
                }
                rc = SPIN_ERR_OOM;
            }
        }
        if (rc == SPIN_OK) {
            if (!batched)
                rc = run_single(*g[0], m, s);
            else if (host_stage == nullptr)
                rc = SPIN_ERR_CUDA;
            else
                rc = run_group(g, m, host_stage, s);
        }
        if ((rc == SPIN_ERR_CUDA || rc == SPIN_ERR_OOM) && verbose())
            fprintf(stderr, "spin serve: group of %zu (order %lld) failed with status %d: %s\n", k, (long long)order,
                    rc, spin_last_error());
        release_group(g, m, s, false);  // staged, padded and workspace blocks; X stays until polled
        cudaStreamSynchronize(s);
        const Clock::time_point t_end = Clock::now();
        std::vector<int> status(k, rc);
        if (batched && rc == SPIN_OK) {
            for (size_t i = 0; i < k; i++) {
                int32_t st = 0;
                bucket_result(host_stage, (int)k, (int)i, mixed, &st, &g[i]->info.rel_residual,
                              &g[i]->info.refine_iters);
                g[i]->info.status = st;
                status[i] = st;
            }
        }
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (size_t i = 0; i < k; i++) {
                g[i]->t_end = t_end;
                g[i]->status = status[i];
                g[i]->done = true;
            }
            sv->in_use -= run_bytes;
            sv->running -= (int)k;
            sv->completed += k;
            if (batched) {
                sv->groups++;
                sv->grouped += k;
                sv->max_group = std::max(sv->max_group, (int)k);
            }
        }
        sv->cv.notify_all();
    }
    if (host_stage) cudaFreeHost(host_stage);
}

}  // namespace
}  // namespace spin

using namespace spin;
extern "C" int spin_serve_create(const spin_serve_cfg* cfg, spin_server** out) {
    if (cfg == nullptr || out == nullptr || cfg->max_slots < 1 || cfg->max_slots > 64 || cfg->hbm_budget_bytes == 0 ||
        cfg->priority_order < 0 || cfg->max_batch < 0 || cfg->max_batch > 4096 || cfg->batch_max_order < 0 ||
        cfg->batch_max_order > 4096)
        return SPIN_ERR_INVALID_ARG;
    auto* sv = new spin_server();
    sv->cfg = *cfg;
    sv->max_batch = cfg->max_batch == 0 ? kDefaultMaxBatch : cfg->max_batch;
    sv->batch_max_order = cfg->batch_max_order == 0 ? kDefaultBatchMaxOrder : cfg->batch_max_order;
    if (cudaGetDevice(&sv->device) != cudaSuccess) {
        delete sv;
        return SPIN_ERR_CUDA;
    }
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = sv->device;
    if (cudaMemPoolCreate(&sv->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        delete sv;
        return SPIN_ERR_CUDA;
    }
    if (const char* e = getenv("SPIN_SERVE_INJECT_OOM")) {
        unsigned long long t = 0;
        int c = 0;
        if (sscanf(e, "%llu:%d", &t, &c) == 2) {
            sv->inject_ticket = t;
            sv->inject_left = c;
        }
    }
    uint64_t keep = cfg->hbm_budget_bytes;  // keep freed blocks for reuse up to the budget
    cudaMemPoolSetAttribute(sv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    int prio_lo = 0, prio_hi = 0;  // numerically: least and greatest priority
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    sv->streams.resize(cfg->max_slots);
    sv->hi_streams.resize(cfg->max_slots);
    for (auto& st : sv->streams) cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio_lo);
    for (auto& st : sv->hi_streams) cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio_hi);
    cudaStreamCreateWithFlags(&sv->copy_stream, cudaStreamNonBlocking);
    for (int i = 0; i < cfg->max_slots; i++) sv->workers.emplace_back(worker_loop, sv, i);
    *out = sv;
    return SPIN_OK;
}

extern "C" int spin_serve_submit(spin_server* sv, const double* A, int64_t lda, int64_t n, int precision, double tol,
                                 uint64_t* ticket) {
    if (sv == nullptr || A == nullptr || ticket == nullptr || n < 1 || lda < n) return SPIN_ERR_INVALID_ARG;
    if (!valid_precision(precision) || !(tol > 0.0))
        return SPIN_ERR_INVALID_ARG;
    cudaPointerAttributes at;
    bool on_dev = false;
    if (cudaPointerGetAttributes(&at, A) == cudaSuccess)
        on_dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    else
        cudaGetLastError();
    auto rq = std::make_shared<Request>();
    rq->A = A;
    rq->lda = lda;
    rq->n = n;
    rq->a_on_device = on_dev;
    rq->precision = precision;
    rq->tol = tol;
    const size_t nn = (size_t)n * (size_t)n * sizeof(double);
    rq->footprint_keep = nn;
    const bool batchable = sv->max_batch > 1 && n <= sv->batch_max_order &&
                           (precision == SPIN_FP64 || precision == SPIN_MIXED_BF16X3);
    if (batchable) {
        rq->np = padded_order(n);
        const size_t pp = (size_t)rq->np * (size_t)rq->np * sizeof(double);
        rq->share = (on_dev ? 0 : nn) + (rq->np > n ? 2 * pp : 0);
        const spin_opts o = request_opts(precision, tol);
        rq->footprint_run = rq->share + bucket_bytes(rq->np, 1, o);
    } else {
        rq->np = 0;
        rq->share = 0;
        rq->footprint_run = request_workspace(n, precision, tol) + (on_dev ? 0 : nn);
    }
    rq->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (rq->footprint_run + rq->footprint_keep > sv->cfg.hbm_budget_bytes) {
            sv->rejected++;
            return SPIN_ERR_OOM;  // can never fit the budget
        }
        // an empty queue takes any request, so that none is refused for ever
        if (sv->cfg.max_queued_bytes != 0 && sv->queued_a_bytes > 0 &&
            sv->queued_a_bytes + nn > sv->cfg.max_queued_bytes) {
            sv->shed++;
            return SPIN_ERR_BUSY;  // load shedding: the queue is full
        }
        sv->queued_a_bytes += nn;
        rq->ticket = sv->next_ticket++;
        sv->table[rq->ticket] = rq;
        sv->queue.push_back(rq);
        sv->submitted++;
    }
    sv->cv.notify_all();
    *ticket = rq->ticket;
    return SPIN_OK;
}

extern "C" int spin_serve_poll(spin_server* sv, uint64_t ticket, double* X, int64_t ldx, spin_result* r) {
    if (sv == nullptr) return SPIN_ERR_INVALID_ARG;
    std::shared_ptr<Request> rq;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->table.find(ticket);
        if (it == sv->table.end()) return SPIN_ERR_INVALID_ARG;
        rq = it->second;
        if (!rq->done) return SPIN_ERR_BUSY;
        sv->table.erase(it);
    }
    const int64_t n = rq->n;
    int rc = SPIN_OK;
    if (X != nullptr && rq->X != nullptr) {
        if (ldx < n) {
            rc = SPIN_ERR_INVALID_ARG;
        } else if (cudaMemcpy2DAsync(X, ldx * sizeof(double), rq->X, n * sizeof(double), n * sizeof(double), n,
                                     cudaMemcpyDefault, sv->copy_stream) != cudaSuccess ||
                   cudaStreamSynchronize(sv->copy_stream) != cudaSuccess) {
            rc = SPIN_ERR_CUDA;
        }
    }
    if (rq->X) {
        cudaFreeAsync(rq->X, sv->copy_stream);
        cudaStreamSynchronize(sv->copy_stream);
        rq->X = nullptr;
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->in_use -= rq->footprint_keep;
    }
    sv->cv.notify_all();
    if (r) {
        r->status = rq->status;
        r->refine_iters = rq->info.refine_iters;
        r->precision = rq->precision;
        r->rel_residual = rq->info.rel_residual;
        r->queue_ms = ms_between(rq->t_submit, rq->t_start);
        r->run_ms = ms_between(rq->t_start, rq->t_end);
        r->latency_ms = ms_between(rq->t_submit, rq->t_end);
        r->batch = rq->batch;
    }
    return rc;
}

extern "C" int spin_serve_stats(spin_server* sv, spin_serve_stats_t* st) {
    if (sv == nullptr || st == nullptr) return SPIN_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    st->submitted = sv->submitted;
    st->completed = sv->completed;
    st->rejected = sv->rejected;
    st->queued = sv->queue.size();
    st->running = sv->running;
    st->peak_running = sv->peak_running;
    st->bytes_in_use = sv->in_use;
    st->shed = sv->shed;
    st->deferred = sv->deferred;
    st->groups = sv->groups;
    st->grouped = sv->grouped;
    st->max_group = sv->max_group;
    return SPIN_OK;
}

extern "C" int spin_serve_destroy(spin_server* sv) {
    if (sv == nullptr) return SPIN_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    for (auto& t : sv->workers) t.join();
    for (auto& kv : sv->table)
        if (kv.second->X) cudaFreeAsync(kv.second->X, sv->copy_stream);
    cudaStreamSynchronize(sv->copy_stream);
    for (auto& st : sv->streams) cudaStreamDestroy(st);
    for (auto& st : sv->hi_streams) cudaStreamDestroy(st);
    cudaStreamDestroy(sv->copy_stream);
    cudaMemPoolDestroy(sv->pool);
    delete sv;
    return SPIN_OK;
}
