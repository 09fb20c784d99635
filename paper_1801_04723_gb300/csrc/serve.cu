// Serving: inversion requests admitted continuously by device-memory
// footprint and run concurrently on a pool of CUDA streams.
//
// A request (A, n, precision, tol) waits in a FIFO queue until a slot is
// free and its footprint (device copy of A when A is in host memory, the
// result X, and the inversion workspace) fits the server's HBM budget; it
// then runs on that slot's stream while other requests run on theirs, so
// requests that arrive while others are on the GPU overlap with them.  Its
// result stays in device memory (counted against the budget) until the
// client polls it.  Memory comes from a stream-ordered pool
// (cudaMallocAsync), so admission does not synchronise the device.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

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

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
    uint64_t ticket;
    const double* A;
    int64_t lda, n;
    bool a_on_device;
    int precision;
    double tol;
    size_t footprint_run;   // released when the run ends (staged A + workspace)
    size_t footprint_keep;  // released when the client polls (X)
    Clock::time_point t_submit, t_start, t_end;
    double* X = nullptr;    // device, n x n, owned by the server until polled
    spin_info info{};
    int status = SPIN_ERR_BUSY;
    bool done = false;
    int deferrals = 0;      // times put back in the queue for lack of device memory
};

}  // namespace
}  // namespace spin

struct spin_server {
    spin_serve_cfg cfg;
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

size_t request_workspace(int64_t n, int precision, double tol) {
    spin_opts o = spin_opts_default();
    o.precision = precision;
    o.tol = tol;
    return spin_workspace_bytes(n, &o);
}

void worker_loop(spin_server* sv, int slot) {
    cudaSetDevice(sv->device);
    while (true) {
        std::shared_ptr<Request> rq;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait(lk, [&] {
                if (sv->stop) return true;
                if (sv->queue.empty()) return false;
                if (sv->retry_wait && sv->completed <= sv->retry_after && sv->running > 0) return false;
                const auto& h = sv->queue.front();
                return sv->in_use + h->footprint_run + h->footprint_keep <= sv->cfg.hbm_budget_bytes;
            });
            if (sv->stop) return;
            rq = sv->queue.front();
            sv->queue.pop_front();
            sv->retry_wait = false;
            sv->queued_a_bytes -= (size_t)rq->n * (size_t)rq->n * sizeof(double);
            sv->in_use += rq->footprint_run + rq->footprint_keep;
            sv->running++;
            if (sv->running > sv->peak_running) sv->peak_running = sv->running;
        }
        rq->t_start = Clock::now();
        const int64_t n = rq->n;
        cudaStream_t s = (sv->cfg.priority_order > 0 && n <= sv->cfg.priority_order) ? sv->hi_streams[slot]
                                                                                       : sv->streams[slot];
        const size_t nn = (size_t)n * (size_t)n * sizeof(double);
        const size_t ws_bytes = request_workspace(n, rq->precision, rq->tol);
        double* Ad = nullptr;
        void* ws = nullptr;
        // The budget bounds what the server holds, but the device is shared
        // (the client's own tensors, other processes, and blocks the pool
        // keeps for reuse), so an allocation can still fail: release this
        // request's blocks, return the pool's unused memory to the device and
        // try once more; failing that, put the request back at the head of
        // the queue until another request completes, and fail it only when
        // nothing else is running.
        auto alloc_all = [&]() -> bool {
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                if (rq->ticket == sv->inject_ticket && sv->inject_left > 0) {
                    sv->inject_left--;
                    return false;
                }
            }
            if (cudaMallocFromPoolAsync((void**)&rq->X, nn, sv->pool, s) != cudaSuccess) return false;
            if (ws_bytes && cudaMallocFromPoolAsync(&ws, ws_bytes, sv->pool, s) != cudaSuccess) return false;
            if (!rq->a_on_device && cudaMallocFromPoolAsync((void**)&Ad, nn, sv->pool, s) != cudaSuccess) return false;
            return true;
        };
        auto release_all = [&]() {
            cudaGetLastError();
            if (rq->X) cudaFreeAsync(rq->X, s);
            if (ws) cudaFreeAsync(ws, s);
            if (Ad) cudaFreeAsync(Ad, s);
            rq->X = nullptr;
            ws = nullptr;
            Ad = nullptr;
            cudaStreamSynchronize(s);
        };
        int rc = SPIN_OK;
        if (!alloc_all()) {
            release_all();
            cudaMemPoolTrimTo(sv->pool, 0);
            if (!alloc_all()) {
                release_all();
                bool deferred = false;
                {
                    std::lock_guard<std::mutex> lk(sv->mu);
                    if (sv->running > 1 && rq->deferrals < 1000) {
                        rq->deferrals++;
                        sv->deferred++;
                        sv->in_use -= rq->footprint_run + rq->footprint_keep;
                        sv->running--;
                        sv->queued_a_bytes += nn;
                        sv->queue.push_front(rq);
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
        const double* Ause = rq->A;
        int64_t lda = rq->lda;
        if (rc == SPIN_OK && !rq->a_on_device) {
            if (cudaMemcpy2DAsync(Ad, n * sizeof(double), rq->A, rq->lda * sizeof(double), n * sizeof(double), n,
                                  cudaMemcpyHostToDevice, s) != cudaSuccess)
                rc = SPIN_ERR_CUDA;
            Ause = Ad;
            lda = n;
        }
        if (rc == SPIN_OK) {
            spin_opts o = spin_opts_default();
            o.precision = rq->precision;
            o.tol = rq->tol;
            o.blocking = 1;
            o.workspace = ws;
            o.workspace_bytes = ws_bytes;
            rc = spin_invert_ex(Ause, lda, rq->X, n, n, &o, &rq->info, (spin_stream_t)s);
            if (rc == SPIN_OK || rc == SPIN_ERR_SINGULAR || rc == SPIN_ERR_NOT_CONVERGED) rc = rq->info.status;
        }
        if ((rc == SPIN_ERR_CUDA || rc == SPIN_ERR_OOM) && verbose())
            fprintf(stderr, "spin serve: request %llu (n = %lld) failed with status %d: %s\n",
                    (unsigned long long)rq->ticket, (long long)n, rc, spin_last_error());
        if (Ad) cudaFreeAsync(Ad, s);
        if (ws) cudaFreeAsync(ws, s);
        cudaStreamSynchronize(s);
        rq->t_end = Clock::now();
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            rq->status = rc;
            rq->done = true;
            sv->in_use -= rq->footprint_run;
            sv->running--;
            sv->completed++;
        }
        sv->cv.notify_all();
    }
}

}  // namespace
}  // namespace spin

using namespace spin;

extern "C" int spin_serve_create(const spin_serve_cfg* cfg, spin_server** out) {
    if (cfg == nullptr || out == nullptr || cfg->max_slots < 1 || cfg->max_slots > 64 || cfg->hbm_budget_bytes == 0 ||
        cfg->priority_order < 0)
        return SPIN_ERR_INVALID_ARG;
    auto* sv = new spin_server();
    sv->cfg = *cfg;
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
    rq->footprint_run = request_workspace(n, precision, tol) + (on_dev ? 0 : nn);
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
        r->reserved = 0;
        r->rel_residual = rq->info.rel_residual;
        r->queue_ms = ms_between(rq->t_submit, rq->t_start);
        r->run_ms = ms_between(rq->t_start, rq->t_end);
        r->latency_ms = ms_between(rq->t_submit, rq->t_end);
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
