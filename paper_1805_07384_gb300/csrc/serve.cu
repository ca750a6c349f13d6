// serve.cu -- request server: continuous batching of compress / decompress
// requests over cached plans (no counterpart in the paper, which compresses
// one field per call).
//
// One worker thread owns every CUDA call the server makes.  Each turn it
//   1. completes the batches whose event has fired (results were copied to
//      pinned host memory behind the batch on its stream),
//   2. while a stream has no batch in flight, admits arrived requests in
//      arrival order: the oldest one fixes the kind (compress or decompress)
//      of the next batch, and later arrived requests of that kind join it
//      while a plan for their (shape, options) is idle or can be created
//      inside the HBM budget (evicting idle plans, least recently used first);
//      the batch launches at once on that stream,
//   3. sleeps until the next arrival, a new submission, or a short poll tick
//      while batches are in flight.
// Plans are busy from launch to completion, so a plan never serves two
// requests at once; requests whose plan is busy simply wait their turn.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "plan.cuh"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxSlots = 16;  // batch records (one per stream is in flight)

struct CachedPlan {
    fpsnr_plan_t p = nullptr;
    std::string key;
    size_t bytes = 0;
    bool busy = false;
    uint64_t last_use = 0;
};

struct Req {
    uint64_t ticket;
    fpsnr_request r;
    std::string key;
    double arrival;  // when it may start: max(requested arrival, submission)
    double origin;   // latency is measured from here: the requested arrival, else submission
};

struct Slot {
    bool used = false;
    int kind = 0;
    cudaEvent_t ev = nullptr;
    cudaStream_t st = nullptr;
    fpsnr_stats* d_stats = nullptr;
    uint64_t* d_nbytes = nullptr;
    int* d_status = nullptr;
    fpsnr_stats* h_stats = nullptr;
    uint64_t* h_nbytes = nullptr;
    int* h_status = nullptr;
    std::vector<Req> reqs;
    std::vector<CachedPlan*> plans;
    double start = 0.0;
};

std::string key_of(const fpsnr_request& r) {
    char b[160];
    snprintf(b, sizeof(b), "%d|%llu,%llu,%llu|%d,%d,%d,%d,%d,%d", r.ndim, (unsigned long long)r.dims[0],
             (unsigned long long)r.dims[1], (unsigned long long)r.dims[2], r.opts.radius,
             r.opts.chunk, r.opts.lmax, r.opts.lorenzo_dims, r.opts.psnr_mode, r.opts.lossless);
    return b;
}

}  // namespace

struct fpsnr_server_s {
    int device = 0;
    fpsnr_server_opts o{};
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;       // worker: new work or stop
    std::condition_variable done_cv;  // waiters: a request completed
    bool stop = false;
    std::thread worker;
    std::deque<Req> pending;  // ordered by arrival
    std::list<CachedPlan> plans;
    size_t plan_bytes = 0;
    uint64_t plans_created = 0;
    uint64_t use_clock = 0;
    std::vector<Slot> slots;
    std::vector<cudaStream_t> streams;
    int next_stream = 0;
    std::unordered_map<uint64_t, fpsnr_result> results;
    std::deque<uint64_t> done_order;  // completion order (tickets taken by poll are skipped)
    uint64_t next_ticket = 1;
    uint64_t outstanding = 0;  // submitted and not yet completed
    std::vector<double> lat;
    uint64_t completed = 0, failed = 0, batches = 0, bytes_in = 0;

    double now() const {
        return std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
    }
    void run();
    void harvest();
    bool launch_next(double now_us);
    CachedPlan* acquire(const Req& q, int* err);
    void finish(const Req& q, const fpsnr_result& res);
};

void fpsnr_server_s::finish(const Req& q, const fpsnr_result& res) {
    results[q.ticket] = res;
    done_order.push_back(q.ticket);
    completed++;
    if (res.status) failed++;
    else lat.push_back(res.done_us - res.arrival_us);
    uint64_t n = 1;
    for (int i = 0; i < q.r.ndim; i++) n *= q.r.dims[i];
    bytes_in += 4 * n;
    outstanding--;
}

// A plan for the request's key: an idle cached one, else a new one inside the
// budget (evicting idle plans of any key, least recently used first).  Returns
// nullptr with *err = 0 when the request must wait for a busy plan, or with
// *err set when it can never be served.  A new plan is sized on the host
// first: while the request has to wait, nothing is allocated or evicted
// (both synchronise the device).
CachedPlan* fpsnr_server_s::acquire(const Req& q, int* err) {
    *err = 0;
    for (auto& c : plans)
        if (!c.busy && c.key == q.key) {
            c.busy = true;
            c.last_use = ++use_clock;
            return &c;
        }
    fpsnr_plan_s* p = nullptr;
    int rc = fp::plan_layout(&p, q.r.ndim, q.r.dims,
                             q.r.kind == FPSNR_REQ_COMPRESS ? q.r.target_psnr_db : 60.0, &q.r.opts);
    if (rc) {
        *err = rc;
        return nullptr;
    }
    const size_t need = p->slab_bytes;
    if (need > o.hbm_budget) {
        delete p;
        *err = FPSNR_ENOMEM;
        return nullptr;
    }
    size_t idle = 0;
    for (auto& c : plans)
        if (!c.busy) idle += c.bytes;
    if (plan_bytes - idle + need > o.hbm_budget) {
        // it cannot fit until a batch finishes: wait
        delete p;
        return nullptr;
    }
    while (plan_bytes + need > o.hbm_budget) {
        auto victim = plans.end();
        for (auto it = plans.begin(); it != plans.end(); ++it)
            if (!it->busy && (victim == plans.end() || it->last_use < victim->last_use)) victim = it;
        if (victim == plans.end()) {  // not reached: the idle plans cover the shortfall
            delete p;
            return nullptr;
        }
        plan_bytes -= victim->bytes;
        fpsnr_plan_destroy(victim->p);
        plans.erase(victim);
    }
    rc = fp::plan_allocate(p);
    if (rc) {
        *err = rc;
        return nullptr;
    }
    plans_created++;
    plans.push_back(CachedPlan{p, q.key, need, true, ++use_clock});
    plan_bytes += need;
    return &plans.back();
}

void fpsnr_server_s::harvest() {
    for (auto& s : slots) {
        if (!s.used) continue;
        const cudaError_t e = cudaEventQuery(s.ev);
        if (e == cudaErrorNotReady) continue;
        const double t = now();
        for (size_t i = 0; i < s.reqs.size(); i++) {
            fpsnr_result res;
            memset(&res, 0, sizeof(res));
            if (e != cudaSuccess) {
                cudaGetLastError();
                res.status = FPSNR_ECUDA;
            } else if (s.kind == FPSNR_REQ_COMPRESS) {
                res.stats = s.h_stats[i];
                res.out_bytes = s.h_nbytes[i];
                res.status = res.stats.status;
            } else {
                res.status = s.h_status[i];
            }
            res.arrival_us = s.reqs[i].origin;
            res.start_us = s.start;
            res.done_us = t;
            finish(s.reqs[i], res);
            s.plans[i]->busy = false;
        }
        s.reqs.clear();
        s.plans.clear();
        s.used = false;
        done_cv.notify_all();
    }
}

// Forms and launches one batch from the arrived requests; false if none could go.
bool fpsnr_server_s::launch_next(double now_us) {
    // one batch in flight per stream: while every stream is busy, arriving
    // requests queue up and leave together in the next batch
    Slot* slot = nullptr;
    int inflight = 0;
    for (auto& s : slots) {
        if (s.used) inflight++;
        else if (!slot) slot = &s;
    }
    if (!slot || inflight >= (int)streams.size() || pending.empty() || pending.front().arrival > now_us)
        return false;
    const int kind = pending.front().r.kind;
    std::vector<Req> take;
    std::vector<CachedPlan*> got;
    for (auto it = pending.begin(); it != pending.end() && (int)take.size() < o.max_batch;) {
        if (it->arrival > now_us) break;
        if (it->r.kind != kind) {
            ++it;
            continue;
        }
        int err = 0;
        CachedPlan* c = acquire(*it, &err);
        if (err) {
            fpsnr_result res;
            memset(&res, 0, sizeof(res));
            res.status = err;
            res.arrival_us = it->origin;
            res.start_us = res.done_us = now();
            finish(*it, res);
            it = pending.erase(it);
            done_cv.notify_all();
            continue;
        }
        if (!c) {
            // its plan is busy or memory is full: the oldest request keeps its
            // place; later ones of this kind may still go
            ++it;
            continue;
        }
        take.push_back(*it);
        got.push_back(c);
        it = pending.erase(it);
    }
    if (take.empty()) return false;
    const int n = (int)take.size();
    std::vector<fpsnr_plan_t> ps(n);
    for (int i = 0; i < n; i++) {
        ps[i] = got[i]->p;
        if (kind == FPSNR_REQ_COMPRESS) fpsnr_plan_set_psnr(ps[i], take[i].r.target_psnr_db);
    }
    // a stream with no batch in flight (one exists: fewer batches than streams)
    for (size_t k = 0; k < streams.size(); k++) {
        cudaStream_t cand = streams[(next_stream + k) % streams.size()];
        bool busy = false;
        for (auto& o2 : slots) busy |= o2.used && o2.st == cand;
        if (!busy) {
            slot->st = cand;
            next_stream = (int)((next_stream + k + 1) % streams.size());
            break;
        }
    }
    int rc;
    if (kind == FPSNR_REQ_COMPRESS) {
        std::vector<const float*> in(n);
        std::vector<void*> out(n);
        std::vector<uint64_t> cap(n);
        for (int i = 0; i < n; i++) {
            in[i] = static_cast<const float*>(take[i].r.d_in);
            out[i] = take[i].r.d_out;
            cap[i] = take[i].r.out_cap;
        }
        rc = fpsnr_compress_batch(ps.data(), in.data(), out.data(), cap.data(), slot->d_nbytes,
                                  slot->d_stats, n, slot->st);
        if (rc == FPSNR_OK &&
            (cudaMemcpyAsync(slot->h_stats, slot->d_stats, n * sizeof(fpsnr_stats),
                             cudaMemcpyDeviceToHost, slot->st) != cudaSuccess ||
             cudaMemcpyAsync(slot->h_nbytes, slot->d_nbytes, n * sizeof(uint64_t),
                             cudaMemcpyDeviceToHost, slot->st) != cudaSuccess))
            rc = FPSNR_ECUDA;
    } else {
        std::vector<const void*> in(n);
        std::vector<uint64_t> nb(n);
        std::vector<float*> out(n);
        for (int i = 0; i < n; i++) {
            in[i] = take[i].r.d_in;
            nb[i] = take[i].r.in_bytes;
            out[i] = static_cast<float*>(take[i].r.d_out);
        }
        rc = fpsnr_decompress_batch(ps.data(), in.data(), nb.data(), out.data(), slot->d_status, n,
                                    slot->st);
        if (rc == FPSNR_OK && cudaMemcpyAsync(slot->h_status, slot->d_status, n * sizeof(int),
                                              cudaMemcpyDeviceToHost, slot->st) != cudaSuccess)
            rc = FPSNR_ECUDA;
    }
    if (rc == FPSNR_OK && cudaEventRecord(slot->ev, slot->st) != cudaSuccess) rc = FPSNR_ECUDA;
    batches++;
    if (rc != FPSNR_OK) {
        cudaGetLastError();
        const double t = now();
        for (int i = 0; i < n; i++) {
            fpsnr_result res;
            memset(&res, 0, sizeof(res));
            res.status = rc;
            res.arrival_us = take[i].origin;
            res.start_us = res.done_us = t;
            finish(take[i], res);
            got[i]->busy = false;
        }
        done_cv.notify_all();
        return true;
    }
    slot->used = true;
    slot->kind = kind;
    slot->start = now();
    slot->reqs = std::move(take);
    slot->plans = std::move(got);
    return true;
}

void fpsnr_server_s::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        harvest();
        while (launch_next(now())) {
        }
        bool inflight = false;
        for (auto& s : slots) inflight |= s.used;
        if (stop && pending.empty() && !inflight) break;
        if (inflight) {
            // completions are found by polling events: a short tick, woken early
            // by a new submission
            cv.wait_for(lk, std::chrono::microseconds(20));
        } else if (!pending.empty()) {
            const double wait = pending.front().arrival - now();
            if (wait > 0) cv.wait_for(lk, std::chrono::microseconds((int64_t)wait + 1));
        } else {
            cv.wait(lk, [&] { return stop || !pending.empty(); });
        }
    }
}

extern "C" {

int fpsnr_server_create(const fpsnr_server_opts* opts, fpsnr_server_t* out) {
    if (!opts || !out) return FPSNR_EINVAL;
    *out = nullptr;
    if (opts->max_batch < 1 || opts->max_batch > fp::kMaxBatch || opts->streams < 1 ||
        opts->streams > 16 || opts->hbm_budget == 0)
        return FPSNR_EINVAL;
    auto* s = new (std::nothrow) fpsnr_server_s();
    if (!s) return FPSNR_ENOMEM;
    s->o = *opts;
    s->t0 = Clock::now();
    bool ok = cudaGetDevice(&s->device) == cudaSuccess;
    for (int i = 0; ok && i < opts->streams; i++) {
        cudaStream_t st = nullptr;
        ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
        if (ok) s->streams.push_back(st);
    }
    s->slots.resize(kMaxSlots);
    const int B = fp::kMaxBatch;
    for (auto& sl : s->slots) {
        if (!ok) break;
        ok = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) == cudaSuccess &&
             cudaMalloc(&sl.d_stats, B * sizeof(fpsnr_stats)) == cudaSuccess &&
             cudaMalloc(&sl.d_nbytes, B * sizeof(uint64_t)) == cudaSuccess &&
             cudaMalloc(&sl.d_status, B * sizeof(int)) == cudaSuccess &&
             cudaMallocHost(&sl.h_stats, B * sizeof(fpsnr_stats)) == cudaSuccess &&
             cudaMallocHost(&sl.h_nbytes, B * sizeof(uint64_t)) == cudaSuccess &&
             cudaMallocHost(&sl.h_status, B * sizeof(int)) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        fpsnr_server_destroy(s);
        return FPSNR_ENOMEM;
    }
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return FPSNR_OK;
}

int fpsnr_server_submit(fpsnr_server_t s, const fpsnr_request* r, uint64_t* ticket) {
    if (!s || !r || !ticket) return FPSNR_EINVAL;
    if (r->kind != FPSNR_REQ_COMPRESS && r->kind != FPSNR_REQ_DECOMPRESS) return FPSNR_EINVAL;
    if (r->ndim < 1 || r->ndim > 3 || !r->d_in || !r->d_out) return FPSNR_EINVAL;
    if (r->kind == FPSNR_REQ_COMPRESS &&
        (((uintptr_t)r->d_in & 3u) || ((uintptr_t)r->d_out & 15u) || !(r->target_psnr_db > 0.0) ||
         !(r->target_psnr_db <= FPSNR_MAX_PSNR)))
        return FPSNR_EINVAL;
    if (r->kind == FPSNR_REQ_DECOMPRESS && (((uintptr_t)r->d_in & 15u) || ((uintptr_t)r->d_out & 15u)))
        return FPSNR_EINVAL;
    Req q;
    q.r = *r;
    for (int i = r->ndim; i < 3; i++) q.r.dims[i] = 1;
    if (q.r.opts.radius == 0) fpsnr_default_opts(&q.r.opts);
    q.key = key_of(q.r);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        q.ticket = s->next_ticket++;
        const double t = s->now();
        q.arrival = std::max(r->arrival_us, t);
        q.origin = r->arrival_us > 0.0 ? r->arrival_us : t;
        // keep arrival order (submissions are usually already in order)
        auto it = s->pending.end();
        while (it != s->pending.begin() && std::prev(it)->arrival > q.arrival) --it;
        s->pending.insert(it, q);
        s->outstanding++;
        *ticket = q.ticket;
    }
    s->cv.notify_one();
    return FPSNR_OK;
}

int fpsnr_server_poll(fpsnr_server_t s, uint64_t ticket, fpsnr_result* res) {
    if (!s || !res) return FPSNR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it != s->results.end()) {
        *res = it->second;
        s->results.erase(it);
        return FPSNR_OK;
    }
    if (ticket == 0 || ticket >= s->next_ticket) return FPSNR_EINVAL;
    for (auto& q : s->pending)
        if (q.ticket == ticket) return FPSNR_EAGAIN;
    for (auto& sl : s->slots)
        for (auto& q : sl.reqs)
            if (sl.used && q.ticket == ticket) return FPSNR_EAGAIN;
    return FPSNR_EINVAL;  // already taken
}

int fpsnr_server_take_any(fpsnr_server_t s, uint64_t* ticket, fpsnr_result* res) {
    if (!s || !ticket || !res) return FPSNR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    while (!s->done_order.empty()) {
        const uint64_t t = s->done_order.front();
        s->done_order.pop_front();
        auto it = s->results.find(t);
        if (it == s->results.end()) continue;  // taken by ticket already
        *ticket = t;
        *res = it->second;
        s->results.erase(it);
        return FPSNR_OK;
    }
    return FPSNR_EAGAIN;
}

int fpsnr_server_wait(fpsnr_server_t s, uint64_t ticket, fpsnr_result* res, double timeout_s) {
    if (!s || !res) return FPSNR_EINVAL;
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        const int rc = fpsnr_server_poll(s, ticket, res);
        if (rc != FPSNR_EAGAIN) return rc;
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->results.count(ticket)) continue;
        if (s->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && !s->results.count(ticket))
            return FPSNR_ETIMEOUT;
    }
}

int fpsnr_server_drain(fpsnr_server_t s, double timeout_s) {
    if (!s) return FPSNR_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                        [&] { return s->outstanding == 0; });
    return ok ? FPSNR_OK : FPSNR_ETIMEOUT;
}

int fpsnr_server_get_stats(fpsnr_server_t s, fpsnr_server_stats* st) {
    if (!s || !st) return FPSNR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(st, 0, sizeof(*st));
    st->completed = s->completed;
    st->failed = s->failed;
    st->batches = s->batches;
    st->plans = s->plans.size();
    st->plan_bytes = s->plan_bytes;
    st->plans_created = s->plans_created;
    st->bytes_in = s->bytes_in;
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        std::sort(v.begin(), v.end());
        auto q = [&](double f) { return v[std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5))]; };
        st->p50_us = q(0.50);
        st->p99_us = q(0.99);
        st->max_us = v.back();
    }
    return FPSNR_OK;
}

double fpsnr_server_now(fpsnr_server_t s) { return s ? s->now() : 0.0; }

void fpsnr_server_destroy(fpsnr_server_t s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != s->device) cudaSetDevice(s->device);
    for (auto& st : s->streams) cudaStreamSynchronize(st);
    for (auto& c : s->plans) fpsnr_plan_destroy(c.p);
    for (auto& sl : s->slots) {
        if (sl.ev) cudaEventDestroy(sl.ev);
        cudaFree(sl.d_stats);
        cudaFree(sl.d_nbytes);
        cudaFree(sl.d_status);
        cudaFreeHost(sl.h_stats);
        cudaFreeHost(sl.h_nbytes);
        cudaFreeHost(sl.h_status);
    }
    for (auto& st : s->streams) cudaStreamDestroy(st);
    if (cur >= 0 && cur != s->device) cudaSetDevice(cur);
    delete s;
}

}  // extern "C"
