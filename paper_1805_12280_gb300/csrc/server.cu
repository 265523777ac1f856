// Served form: a continuous-batching request loop over one plan (see include/fdas.h).
//
// Requests carry a device input array.  A scheduler thread admits them in arrival
// order as soon as the plane memory they need (4*M*n bytes, from a pool reserved once at
// creation) is free, packs admitted requests into batches and replays the persistent
// batch kernel on whichever lane (stream + work counter + graph) is idle, so batches on
// different lanes overlap on the GPU.  A host function on the lane's stream marks the
// batch complete.  The templates and their transforms stay resident in the plan.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fdas_internal.cuh"

struct fdas_server_s;

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, size) with 256-byte granules and coalescing frees.
class PoolAllocator {
  public:
    void reset(int64_t size)
    {
        free_.clear();
        free_[0] = size;
        used_ = 0;
    }
    int64_t alloc(int64_t bytes)
    {
        bytes = (bytes + 255) & ~int64_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const int64_t off = it->first, rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                used_ += bytes;
                return off;
            }
        }
        return -1;
    }
    void release(int64_t off, int64_t bytes)
    {
        bytes = (bytes + 255) & ~int64_t(255);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    int64_t used() const { return used_; }

  private:
    std::map<int64_t, int64_t> free_;
    int64_t used_ = 0;
};

enum class State { Queued, Admitted, Running, Done, Failed };

struct Request {
    const void *in = nullptr;
    int64_t n = 0, bytes = 0, offset = -1;
    State state = State::Queued;
    int rc = FDAS_OK;
    Clock::time_point t_submit, t_done;
};

struct LaneState {
    fdas_server_s *srv = nullptr;
    fdas::Lane lane;
    cudaStream_t stream = nullptr;
    bool busy = false;
    std::vector<int64_t> tickets;
};

}  // namespace

struct fdas_server_s {
    fdas_plan plan = nullptr;
    int device = -1, M = 0, max_batch = 32;
    char *pool = nullptr;
    int64_t budget = 0;
    PoolAllocator alloc;
    std::vector<LaneState *> lanes;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<int64_t> queue, admitted;
    std::unordered_map<int64_t, Request> reqs;
    int64_t next_ticket = 1;
    bool stop = false;
    std::thread sched;
    // statistics
    std::vector<double> lat_ms;
    int64_t submitted = 0, completed = 0, rejected = 0, admission_waits = 0, launches = 0, peak = 0;
    bool have_first = false;
    Clock::time_point first_submit, last_done;
};

namespace {

void CUDART_CB on_lane_done(void *arg)
{
    // Runs on a CUDA driver thread: no CUDA calls here, only host bookkeeping.
    LaneState *ls = static_cast<LaneState *>(arg);
    fdas_server_s *s = ls->srv;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const Clock::time_point now = Clock::now();
        for (int64_t t : ls->tickets) {
            auto it = s->reqs.find(t);
            if (it == s->reqs.end()) continue;
            Request &r = it->second;
            if (r.state == State::Running) {
                r.state = State::Done;
                r.t_done = now;
                s->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r.t_submit).count());
                s->completed++;
                s->last_done = now;
            }
        }
        ls->tickets.clear();
        ls->busy = false;
    }
    s->cv_sched.notify_all();
    s->cv_done.notify_all();
}

void admit_locked(fdas_server_s *s)
{
    while (!s->queue.empty()) {
        Request &r = s->reqs[s->queue.front()];
        const int64_t off = s->alloc.alloc(r.bytes);
        if (off < 0) break;                      // arrival order: the head waits for memory
        r.offset = off;
        r.state = State::Admitted;
        s->admitted.push_back(s->queue.front());
        s->queue.pop_front();
        s->peak = std::max(s->peak, s->alloc.used());
    }
}

void scheduler(fdas_server_s *s)
{
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    std::vector<const void *> ins;
    std::vector<int64_t> ns;
    std::vector<float *> outs;
    while (!s->stop) {
        admit_locked(s);
        bool launched = false;
        for (LaneState *ls : s->lanes) {
            if (ls->busy || s->admitted.empty()) continue;
            ins.clear();
            ns.clear();
            outs.clear();
            ls->tickets.clear();
            while (!s->admitted.empty() && (int)ls->tickets.size() < s->max_batch) {
                const int64_t t = s->admitted.front();
                s->admitted.pop_front();
                Request &r = s->reqs[t];
                r.state = State::Running;
                ls->tickets.push_back(t);
                ins.push_back(r.in);
                ns.push_back(r.n);
                outs.push_back(reinterpret_cast<float *>(s->pool + r.offset));
            }
            ls->busy = true;
            s->launches++;
            lk.unlock();   // CUDA calls outside the lock; only this thread launches
            int rc = fdas::lane_launch(s->plan, &ls->lane, (int)ins.size(), ins.data(), ns.data(), outs.data(),
                                       ls->stream);
            if (rc == FDAS_OK && cudaLaunchHostFunc(ls->stream, on_lane_done, ls) != cudaSuccess) rc = FDAS_ERR_CUDA;
            lk.lock();
            if (rc != FDAS_OK) {
                for (int64_t t : ls->tickets) {
                    Request &r = s->reqs[t];
                    r.state = State::Failed;
                    r.rc = rc;
                }
                ls->tickets.clear();
                ls->busy = false;
                s->cv_done.notify_all();
            }
            launched = true;
        }
        if (!launched) s->cv_sched.wait(lk);
    }
    lk.unlock();
    if (prev >= 0) cudaSetDevice(prev);
}

}  // namespace

extern "C" {

int fdas_server_create(fdas_server *out, fdas_plan plan, const fdas_server_opts *opts)
{
    if (!out || !plan || !opts) return fdas::set_error(FDAS_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (opts->budget_bytes < 256) return fdas::set_error(FDAS_ERR_INVALID_ARG, "budget_bytes must be positive");
    const int lanes = opts->lanes ? opts->lanes : 2;
    const int max_batch = opts->max_batch ? opts->max_batch : 32;
    if (lanes < 1 || lanes > 16) return fdas::set_error(FDAS_ERR_INVALID_ARG, "lanes outside [1, 16]");
    if (max_batch < 1 || max_batch > fdas::kBatchMax)
        return fdas::set_error(FDAS_ERR_INVALID_ARG, "max_batch outside [1, 120]");
    if (fdas::plan_grouped(plan)) return fdas::set_error(FDAS_ERR_UNSUPPORTED, "the server is built for ungrouped plans");
    if (fdas::plan_precision(plan) == FDAS_PREC_TC_FP16)
        return fdas::set_error(FDAS_ERR_UNSUPPORTED, "the server is not built for the single-pass tensor-core form");
    fdas_server_s *s = new (std::nothrow) fdas_server_s;
    if (!s) return fdas::set_error(FDAS_ERR_OOM, "host allocation");
    s->plan = plan;
    s->device = fdas::plan_device(plan);
    s->M = fdas::plan_templates(plan);
    s->max_batch = max_batch;
    s->budget = opts->budget_bytes;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    int rc = FDAS_OK;
    if (cudaMalloc(&s->pool, (size_t)s->budget) != cudaSuccess) {
        cudaGetLastError();
        rc = fdas::set_error(FDAS_ERR_OOM, "cannot reserve the plane budget on the device");
    }
    for (int i = 0; rc == FDAS_OK && i < lanes; ++i) {
        LaneState *ls = new LaneState;
        ls->srv = s;
        s->lanes.push_back(ls);
        if (cudaStreamCreateWithFlags(&ls->stream, cudaStreamNonBlocking) != cudaSuccess)
            rc = fdas::set_error(FDAS_ERR_CUDA, "lane stream");
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (rc != FDAS_OK) {
        fdas_server_destroy(s);
        return rc;
    }
    s->alloc.reset(s->budget);
    s->sched = std::thread(scheduler, s);
    *out = s;
    return FDAS_OK;
}

int fdas_server_submit(fdas_server s, const void *in, int64_t n, int64_t *ticket)
{
    if (!s || !ticket) return fdas::set_error(FDAS_ERR_INVALID_ARG, "null argument");
    *ticket = 0;
    if (!in) return fdas::set_error(FDAS_ERR_INVALID_ARG, "null input pointer");
    if (reinterpret_cast<uintptr_t>(in) % 16) return fdas::set_error(FDAS_ERR_INVALID_ARG, "input pointer must be 16-byte aligned");
    if (n < 1 || n > fdas::plan_n_max(s->plan)) return fdas::set_error(FDAS_ERR_INVALID_ARG, "n outside [1, n_max]");
    const int64_t bytes = (int64_t)sizeof(float) * s->M * n;
    std::lock_guard<std::mutex> lk(s->mu);
    if (((bytes + 255) & ~int64_t(255)) > s->budget) {
        s->rejected++;
        return fdas::set_error(FDAS_ERR_REJECTED, "the plane of this array exceeds the whole memory budget");
    }
    const int64_t t = s->next_ticket++;
    Request &r = s->reqs[t];
    r.in = in;
    r.n = n;
    r.bytes = bytes;
    r.t_submit = Clock::now();
    if (!s->have_first) {
        s->have_first = true;
        s->first_submit = r.t_submit;
    }
    s->submitted++;
    const bool waits = !s->queue.empty() || s->alloc.used() + ((bytes + 255) & ~int64_t(255)) > s->budget;
    if (waits) s->admission_waits++;
    s->queue.push_back(t);
    *ticket = t;
    s->cv_sched.notify_all();
    return FDAS_OK;
}

int fdas_server_wait(fdas_server s, int64_t ticket, int64_t timeout_ms, float **plane)
{
    if (!s) return fdas::set_error(FDAS_ERR_INVALID_ARG, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fdas::set_error(FDAS_ERR_INVALID_ARG, "unknown ticket");
    auto done = [&] {
        const State st = s->reqs[ticket].state;
        return st == State::Done || st == State::Failed;
    };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, done);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
        return fdas::set_error(FDAS_ERR_TIMEOUT, "request not complete within the deadline");
    }
    Request &r = s->reqs[ticket];
    if (r.state == State::Failed) return fdas::set_error(r.rc ? r.rc : FDAS_ERR_CUDA, "request failed at launch");
    if (plane) *plane = reinterpret_cast<float *>(s->pool + r.offset);
    return FDAS_OK;
}

int fdas_server_release(fdas_server s, int64_t ticket)
{
    if (!s) return fdas::set_error(FDAS_ERR_INVALID_ARG, "null server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return fdas::set_error(FDAS_ERR_INVALID_ARG, "unknown ticket");
        Request &r = it->second;
        if (r.state != State::Done && r.state != State::Failed)
            return fdas::set_error(FDAS_ERR_BUSY, "request still queued or running");
        if (r.offset >= 0) s->alloc.release(r.offset, r.bytes);
        s->reqs.erase(it);
    }
    s->cv_sched.notify_all();
    return FDAS_OK;
}

int fdas_server_stats(fdas_server s, fdas_server_report *st)
{
    if (!s || !st) return fdas::set_error(FDAS_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(st, 0, sizeof *st);
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->rejected = s->rejected;
    st->queued = (int64_t)s->queue.size();
    st->in_flight = (int64_t)s->reqs.size() - st->queued;
    st->bytes_in_use = s->alloc.used();
    st->peak_bytes_in_use = s->peak;
    st->admission_waits = s->admission_waits;
    st->launches = s->launches;
    if (!s->lat_ms.empty()) {
        std::vector<double> v = s->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))]; };
        st->p50_ms = pct(0.50);
        st->p99_ms = pct(0.99);
        st->max_ms = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        st->mean_ms = sum / v.size();
        const double span = std::chrono::duration<double>(s->last_done - s->first_submit).count();
        st->arrays_per_s = span > 0 ? s->completed / span : 0.0;
    }
    return FDAS_OK;
}

int fdas_server_reset_stats(fdas_server s)
{
    if (!s) return fdas::set_error(FDAS_ERR_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    s->lat_ms.clear();
    s->submitted = s->completed = s->rejected = s->admission_waits = s->launches = 0;
    s->peak = s->alloc.used();
    s->have_first = false;
    return FDAS_OK;
}

int fdas_server_destroy(fdas_server s)
{
    if (!s) return fdas::set_error(FDAS_ERR_INVALID_ARG, "null server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_sched.notify_all();
    if (s->sched.joinable()) s->sched.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (LaneState *ls : s->lanes) {
        if (ls->stream) {
            cudaStreamSynchronize(ls->stream);   // in-flight batches finish (their callbacks run)
            cudaStreamDestroy(ls->stream);
        }
        fdas::lane_free(&ls->lane);
        delete ls;
    }
    cudaFree(s->pool);
    if (prev >= 0) cudaSetDevice(prev);
    delete s;
    return FDAS_OK;
}

}  // extern "C"
