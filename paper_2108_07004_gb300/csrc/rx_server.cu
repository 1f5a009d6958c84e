// Serving loop with continuous batching over receiver handles.
//
// A request is one stream (any built-in or custom format, its own link and
// receiver parameters).  Requests wait in a FIFO queue until a slot is free
// and their device-memory estimate fits the budget; an admitted request gets
// its own handle and CUDA stream and is processed a few blocks at a time
// ("blocks_per_step"), interleaved with every other admitted request, so the work of requests
// that arrived at different times overlaps on the device.  A finished
// request frees its slot and its memory estimate; its handle (with its CUDA
// stream and buffers) is kept idle for the next request with the same
// creation key, so that no cudaFree stalls the running requests, and the
// queue's head is admitted at the next step.  Each request's computation is that of a
// handle processing the stream alone (the library's kernels are
// deterministic), so its results do not depend on the mix.
//
// A request's handle issues in one-stream mode by default (rx_set_param
// "issue" 1: every launch on the request's stream, no event operations): the
// other requests fill the device, and the host issues about a third of the
// operations of the multi-stream mode.
//
// The steps come from the caller (rx_server_step / rx_server_run) or from the
// server's own host thread (rx_server_start), which steps while requests run
// or wait; every entry point takes the server's lock, which a step releases
// while it issues blocks.
//
// Host code only; everything on the device goes through the public entry
// points (rx_create, rx_process_blocks, rx_get_stats, ...).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <exception>
#include <mutex>
#include <memory>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "rx.h"

namespace {

enum { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2, Q_FAILED = 3 };

struct Req {
    uint64_t id = 0;
    int state = Q_QUEUED;
    rx_request r{};
    std::vector<float> points;          // copies of a custom table
    std::vector<uint32_t> labels;
    rx_handle *h = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    long N = 0, nblk = 0, next = 0;
    size_t mem = 0;
    rx_stats stats{};
    std::string err;
    std::string key;                    // handle_key of the request
    long cap_n = 0;                     // symbols the handle's buffers hold (reused handles: >= N)
    double t_submit = 0, t_admit = 0, t_done = 0;   // server step counters
    std::vector<cudaEvent_t> lat_ev;    // "block_latency": start / end event of each issue call
};

size_t estimate_bytes_n(size_t N) {
    // per symbol: CDC output 32 B, FIR output 16 B, phase index 1 B, phase
    // code 2 B, reference labels 2 B; plus tables, taps ring and partials
    return 53 * N + (1u << 20);
}

size_t estimate_bytes(const rx_request &r) { return estimate_bytes_n(r.n_samples / 2); }

// What rx_create fixes: requests with equal keys can share a handle (the
// dispersion and the FFT / block settings are parameters set per request).
std::string handle_key(const rx_request &r, const std::vector<float> &pts, const std::vector<uint32_t> &labs) {
    std::string k;
    auto put = [&k](const void *p, size_t n) { k.append(static_cast<const char *>(p), n); };
    put(&r.format.kind, sizeof r.format.kind);
    put(&r.format.dims, sizeof r.format.dims);
    put(&r.format.m_bits, sizeof r.format.m_bits);
    put(&r.format.sym_order, sizeof r.format.sym_order);
    put(&r.symbol_rate, sizeof r.symbol_rate);
    put(&r.sps, sizeof r.sps);
    put(&r.taps, sizeof r.taps);
    put(&r.bps_phases, sizeof r.bps_phases);
    if (r.format.kind == RX_FMT_CUSTOM) {
        put(pts.data(), sizeof(float) * pts.size());
        put(labs.data(), sizeof(uint32_t) * labs.size());
    }
    return k;
}

// A finished request's handle, kept with its stream and buffers for the
// next compatible request: destroying a handle frees device memory, which
// synchronises the whole device and would stall every running request.
struct Pooled {
    std::string key;
    rx_handle *h = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    long cap_n = 0;      // symbols its buffers hold
    size_t mem = 0;
};

}  // namespace

struct rx_server {
    size_t budget = 0, used = 0;
    int max_slots = 1;
    uint64_t next_id = 1;
    long steps = 0;
    std::deque<Req *> queue;
    std::vector<Req *> active;
    std::unordered_map<uint64_t, std::unique_ptr<Req>> all;
    std::vector<Pooled> pool;           // idle handles, oldest first
    size_t issue_threads = 1;           // host threads that issue a step's blocks
    size_t pooled = 0;                  // their memory estimates
    int max_active_seen = 0;
    int issue = 1;                      // the handles' issue mode (rx_set_param "issue")
    long blocks_per_step = 1;           // blocks of a running request issued per step
    long n_created = 0, n_destroyed = 0, n_regrown = 0;   // handles made, freed, reused with too small buffers
    bool block_latency = false;         // time each issue call of a request (events on its stream)
    std::vector<double> blk_ms;         // those times of retired requests, in retirement order
    // the server's own loop (rx_server_start): the host thread that steps,
    // the lock every entry point takes around the server's state, and the
    // condition it waits on while idle
    mutable std::mutex mu;
    std::condition_variable cv;
    std::thread loop;
    std::atomic<bool> running{false};
};

namespace {

thread_local std::string g_srv_err;

int srv_fail(int code, const std::string &msg) {
    g_srv_err = msg;
    return code;
}

void destroy_handle(rx_server *s, rx_handle *h, cudaStream_t st, cudaEvent_t done) {
    if (h) {
        rx_destroy(h);
        ++s->n_destroyed;
    }
    if (done) cudaEventDestroy(done);
    if (st) cudaStreamDestroy(st);
}

// elapsed times of q's issue calls (from the start of the call's first
// launch on q's stream to the end of its last), then the events are freed
void collect_latency(rx_server *s, Req *q) {
    for (size_t i = 0; i + 1 < q->lat_ev.size(); i += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, q->lat_ev[i], q->lat_ev[i + 1]) == cudaSuccess) s->blk_ms.push_back(ms);
    }
    for (cudaEvent_t e : q->lat_ev) cudaEventDestroy(e);
    q->lat_ev.clear();
}

void release(rx_server *s, Req *q) {
    if (q->h && q->state == Q_DONE) {
        // keep the handle for a later request with the same key
        Pooled p;
        p.key = q->key;
        p.h = q->h;
        p.st = q->st;
        p.done = q->done;
        p.cap_n = std::max(q->cap_n, q->N);
        p.mem = estimate_bytes_n((size_t)p.cap_n);
        s->pool.push_back(p);
        s->pooled += p.mem;
    } else {
        destroy_handle(s, q->h, q->st, q->done);
    }
    q->h = nullptr;
    q->st = nullptr;
    q->done = nullptr;
    s->used -= q->mem;
}

// index of the pooled handle for q (same key; the smallest that holds q's
// symbols, else the largest), -1 if none
int find_pooled(const rx_server *s, const Req *q) {
    int best = -1;
    for (int i = 0; i < (int)s->pool.size(); ++i) {
        const Pooled &p = s->pool[i];
        if (p.key != q->key) continue;
        if (best < 0) { best = i; continue; }
        const Pooled &b = s->pool[best];
        const bool fits = p.cap_n >= q->N, bfits = b.cap_n >= q->N;
        if ((fits && (!bfits || p.cap_n < b.cap_n)) || (!fits && !bfits && p.cap_n > b.cap_n)) best = i;
    }
    return best;
}

// true if q can be admitted within the budget, destroying idle handles
// (oldest first, never the one q will reuse) while that is what is missing
bool make_room(rx_server *s, const Req *q) {
    const int reuse = find_pooled(s, q);
    const size_t reuse_mem = reuse >= 0 ? s->pool[reuse].mem : 0;
    auto fits = [&] { return s->used + (s->pooled - reuse_mem) + q->mem <= s->budget; };
    for (size_t i = 0; !fits() && i < s->pool.size();) {
        if ((int)i == find_pooled(s, q)) { ++i; continue; }
        Pooled p = s->pool[i];
        s->pool.erase(s->pool.begin() + (long)i);
        s->pooled -= p.mem;
        destroy_handle(s, p.h, p.st, p.done);
    }
    return fits();
}

// create the handle of an admitted request; false (and FAILED) on error
bool admit(rx_server *s, Req *q) {
    int rc = RX_OK;
    const int reuse = find_pooled(s, q);
    if (reuse >= 0) {
        // a finished request's handle: every per-request setting is set
        // again (the defaults where the request leaves one at 0), which also
        // resets its stream state
        Pooled p = s->pool[reuse];
        s->pool.erase(s->pool.begin() + reuse);
        s->pooled -= p.mem;
        q->h = p.h;
        q->st = p.st;
        q->done = p.done;
        q->cap_n = p.cap_n;
        if (p.cap_n < q->N) ++s->n_regrown;
        rc |= rx_set_param(q->h, "cd_ps_per_nm", q->r.cd_ps_per_nm);
        rc |= rx_set_param(q->h, "fft", q->r.fft ? q->r.fft : 1024);
        rc |= rx_set_param(q->h, "overlap", q->r.overlap ? q->r.overlap : 256);
        rc |= rx_set_param(q->h, "block", q->r.block ? q->r.block : 4096);
        rc |= rx_set_param(q->h, "n_pre", q->r.n_pre ? q->r.n_pre : 2048);
    } else {
        rx_format f = q->r.format;
        if (f.kind == RX_FMT_CUSTOM) {
            f.points = q->points.data();
            f.labels = q->labels.data();
        }
        q->h = rx_create(&f, q->r.symbol_rate, q->r.sps, q->r.cd_ps_per_nm, q->r.taps, q->r.bps_phases);
        if (!q->h) {
            q->err = rx_last_error();
            q->state = Q_FAILED;
            return false;
        }
        ++s->n_created;
        if (q->r.fft) rc |= rx_set_param(q->h, "fft", q->r.fft);
        if (q->r.overlap) rc |= rx_set_param(q->h, "overlap", q->r.overlap);
        if (q->r.block) rc |= rx_set_param(q->h, "block", q->r.block);
        if (q->r.n_pre) rc |= rx_set_param(q->h, "n_pre", q->r.n_pre);
        if (rc == RX_OK && cudaStreamCreateWithFlags(&q->st, cudaStreamNonBlocking) != cudaSuccess) rc = RX_ECUDA;
        if (rc == RX_OK && cudaEventCreateWithFlags(&q->done, cudaEventDisableTiming) != cudaSuccess) rc = RX_ECUDA;
    }
    if (rc == RX_OK) rc = rx_set_stream(q->h, q->st);
    double issue = -1;
    if (rc == RX_OK) rc = rx_get_param(q->h, "issue", &issue);
    if (rc == RX_OK && issue != s->issue) rc = rx_set_param(q->h, "issue", s->issue);
    // a request without reference bits clears what a reused handle still
    // holds from its previous request (no training stage, no counting)
    if (rc == RX_OK) rc = q->r.ref_bits ? rx_set_reference(q->h, q->r.ref_bits, q->N)
                                        : rx_set_reference(q->h, nullptr, 0);
    if (rc != RX_OK) {
        q->err = rx_last_error();
        q->state = Q_FAILED;
        s->used += q->mem;
        release(s, q);
        return false;
    }
    double blk = 0;
    rx_get_param(q->h, "block", &blk);
    q->nblk = (q->N + (long)blk - 1) / (long)blk;
    q->state = Q_RUNNING;
    q->t_admit = (double)s->steps;
    s->used += q->mem;
    return true;
}

}  // namespace

namespace {

// One step: retire finished requests, admit from the queue, then issue the
// next blocks_per_step blocks of every running request.  The server's lock
// is held around the bookkeeping and released while blocks are issued (the
// requests being issued are touched by this step alone; submit and poll may
// run meanwhile).  Returns how many requests had blocks issued.
size_t step_impl(rx_server *s, int *n_active) {
    std::vector<Req *> todo;
    long per_step = 1;
    size_t threads = 1;
    bool timed = false;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        ++s->steps;
        // retire requests whose last block has finished
        for (size_t i = 0; i < s->active.size();) {
            Req *q = s->active[i];
            if (q->next >= q->nblk && cudaEventQuery(q->done) == cudaSuccess) {
                if (rx_get_stats(q->h, &q->stats) != RX_OK) q->err = rx_last_error();
                collect_latency(s, q);
                q->state = q->err.empty() ? Q_DONE : Q_FAILED;
                q->t_done = (double)s->steps;
                release(s, q);
                s->active.erase(s->active.begin() + (long)i);
            } else {
                ++i;
            }
        }
        // admit from the head of the queue while a slot and memory are free
        while (!s->queue.empty() && (int)s->active.size() < s->max_slots && make_room(s, s->queue.front())) {
            Req *q = s->queue.front();
            s->queue.pop_front();
            if (admit(s, q)) s->active.push_back(q);
        }
        if ((int)s->active.size() > s->max_active_seen) s->max_active_seen = (int)s->active.size();
        for (Req *q : s->active)
            if (q->next < q->nblk) todo.push_back(q);
        per_step = s->blocks_per_step;
        threads = s->issue_threads;
        timed = s->block_latency;
    }
    // the next blocks_per_step blocks of every running request, each request
    // on its own stream.  Issuing a block costs the host a few launches (and,
    // in issue mode 0, event operations) plus the call's own set-up, so the
    // requests are split over a few host threads (each touches only its own
    // requests' handles; the results are those of one thread)
    std::vector<int> rcs(todo.size(), RX_OK);
    std::vector<std::string> errs(todo.size());
    int dev = 0;
    cudaGetDevice(&dev);
    auto issue = [&](size_t i0, size_t i1) {
        cudaSetDevice(dev);                 // a new host thread starts on device 0
        for (size_t i = i0; i < i1; ++i) {
            Req *q = todo[i];
            const long b1 = std::min(q->nblk, q->next + per_step);
            cudaEvent_t ev[2] = {nullptr, nullptr};
            if (timed && cudaEventCreate(&ev[0]) == cudaSuccess && cudaEventCreate(&ev[1]) == cudaSuccess &&
                cudaEventRecord(ev[0], q->st) == cudaSuccess) {
                q->lat_ev.push_back(ev[0]);
                q->lat_ev.push_back(ev[1]);
            } else if (timed) {
                if (ev[0]) cudaEventDestroy(ev[0]);
                if (ev[1]) cudaEventDestroy(ev[1]);
                ev[1] = nullptr;
            }
            rcs[i] = rx_process_blocks(q->h, q->r.samples, q->r.n_samples, (size_t)q->next, (size_t)b1,
                                       q->r.llr_out, nullptr);
            if (rcs[i] != RX_OK) errs[i] = rx_last_error();
            if (ev[1]) cudaEventRecord(ev[1], q->st);
        }
    };
    const size_t nt = std::min<size_t>(threads, todo.size() / 4 + 1);
    if (nt <= 1) {
        issue(0, todo.size());
    } else {
        std::vector<std::thread> pool;
        const size_t per = (todo.size() + nt - 1) / nt;
        for (size_t t = 1; t < nt; ++t)
            pool.emplace_back(issue, std::min(todo.size(), t * per), std::min(todo.size(), (t + 1) * per));
        issue(0, std::min(todo.size(), per));
        for (auto &th : pool) th.join();
    }
    std::lock_guard<std::mutex> lock(s->mu);
    for (size_t i = 0; i < todo.size(); ++i) {
        Req *q = todo[i];
        if (rcs[i] != RX_OK) {
            q->err = errs[i];
            q->next = q->nblk;
        } else {
            q->next = std::min(q->nblk, q->next + per_step);
        }
        if (q->next >= q->nblk) cudaEventRecord(q->done, q->st);
    }
    if (n_active) *n_active = (int)(s->active.size() + s->queue.size());
    return todo.size();
}

// The server's own loop (rx_server_start): steps while requests run or wait;
// when a step issued nothing (every running request's blocks are in flight,
// or nothing can be admitted yet) it waits up to 100 us for a submission or
// for the device to finish some; with nothing submitted it sleeps until a
// submission or rx_server_stop.
void loop_main(rx_server *s, int dev) {
    cudaSetDevice(dev);
    while (s->running) {
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv.wait(lock, [s] { return !s->running || !s->queue.empty() || !s->active.empty(); });
            if (!s->running) break;
        }
        const size_t issued = step_impl(s, nullptr);
        if (issued == 0) {
            std::unique_lock<std::mutex> lock(s->mu);
            const size_t queued = s->queue.size();
            s->cv.wait_for(lock, std::chrono::microseconds(100),
                           [s, queued] { return !s->running || s->queue.size() != queued; });
        }
    }
}

}  // namespace

extern "C" {

const char *rx_server_last_error(void) { return g_srv_err.c_str(); }

rx_server *rx_server_create(size_t mem_budget_bytes, int max_slots) {
    if (max_slots < 1 || max_slots > 1024 || mem_budget_bytes == 0) {
        srv_fail(RX_EINVAL, "rx_server_create: budget must be > 0 and slots 1..1024");
        return nullptr;
    }
    rx_server *s = new rx_server();
    const unsigned hc = std::thread::hardware_concurrency();
    // Defaults by the hardware work queues the CUDA context has
    // (CUDA_DEVICE_MAX_CONNECTIONS, 8 unless set before the context is made).
    // The requests' streams share those queues, so with few queues a
    // request's consecutive blocks hold up the requests queued behind them:
    // one block per step interleaves best, and more issue threads do not
    // help.  Measured serving capacity, 64 mixed requests (Gbit/s):
    //   blocks per step 1 / 2 / 4 / all (2 threads): 8 queues 6.64 / 6.14 /
    //   5.80 / 4.47, 16 queues 7.55 / 7.95 / 7.74 / 6.90, 32 queues 7.36 /
    //   7.99 / 8.33 / 8.38;
    //   issue threads 1 / 2 / 4 / 8: 8 queues, 1 block per step 6.81 / 6.61 /
    //   6.55 / 6.46; 32 queues, 4 blocks per step 7.64 / 8.23 / 8.90 / 8.65.
    const char *conn = std::getenv("CUDA_DEVICE_MAX_CONNECTIONS");
    const long nconn = conn ? std::strtol(conn, nullptr, 10) : 8;
    s->blocks_per_step = nconn >= 32 ? 4 : nconn >= 16 ? 2 : 1;
    s->issue_threads = std::max(1u, std::min(nconn >= 32 ? 4u : 2u, hc ? hc : 1u));
    s->budget = mem_budget_bytes;
    s->max_slots = max_slots;
    return s;
}

void rx_server_destroy(rx_server *s) {
    if (!s) return;
    if (s->running) rx_server_stop(s);
    for (Req *q : s->active) {
        if (q->st) cudaStreamSynchronize(q->st);
        for (cudaEvent_t e : q->lat_ev) cudaEventDestroy(e);
        destroy_handle(s, q->h, q->st, q->done);
        q->h = nullptr;
    }
    for (Pooled &p : s->pool) destroy_handle(s, p.h, p.st, p.done);
    delete s;
}

int rx_server_submit(rx_server *s, const rx_request *r, uint64_t *id) {
    if (!s || !r || !id) return srv_fail(RX_EINVAL, "NULL argument");
    if (!r->samples || !r->llr_out || r->n_samples < 2 || (r->n_samples & 1))
        return srv_fail(RX_EINVAL, "request needs device samples, an even n_samples and an LLR buffer");
    auto q = std::make_unique<Req>();
    q->r = *r;
    if (r->format.kind == RX_FMT_CUSTOM) {
        const int M = 1 << r->format.m_bits;
        if (!r->format.points || !r->format.labels || r->format.dims < 2 || r->format.dims > 4 || M > 256)
            return srv_fail(RX_EINVAL, "custom format needs its table");
        q->points.assign(r->format.points, r->format.points + (size_t)M * r->format.dims);
        q->labels.assign(r->format.labels, r->format.labels + M);
    }
    q->N = (long)(r->n_samples / 2);
    q->mem = estimate_bytes(*r);
    q->key = handle_key(*r, q->points, q->labels);
    if (q->mem > s->budget)
        return srv_fail(RX_EINVAL, "request needs about " + std::to_string(q->mem) +
                                       " bytes, more than the whole budget");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        q->id = s->next_id++;
        q->t_submit = (double)s->steps;
        *id = q->id;
        s->queue.push_back(q.get());
        s->all[q->id] = std::move(q);
    }
    s->cv.notify_one();
    return RX_OK;
}

int rx_server_step(rx_server *s, int *n_active) {
    if (!s) return srv_fail(RX_EINVAL, "NULL server");
    if (s->running) return srv_fail(RX_ESTATE, "the server's own loop is running (rx_server_stop first)");
    step_impl(s, n_active);
    return RX_OK;
}

int rx_server_run(rx_server *s) {
    if (!s) return srv_fail(RX_EINVAL, "NULL server");
    if (s->running) return srv_fail(RX_ESTATE, "the server's own loop is running (rx_server_stop first)");
    int left = 1;
    while (left > 0) {
        step_impl(s, &left);
        cudaEvent_t oldest = nullptr;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            if (left > 0 && !s->active.empty()) {
                // all blocks issued: wait for the oldest running request
                bool issued = true;
                for (Req *q : s->active) issued &= q->next >= q->nblk;
                if (issued) oldest = s->active.front()->done;
            }
        }
        if (oldest) cudaEventSynchronize(oldest);
    }
    return RX_OK;
}

int rx_server_start(rx_server *s) {
    if (!s) return srv_fail(RX_EINVAL, "NULL server");
    if (s->running) return srv_fail(RX_ESTATE, "the server's loop is already running");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return srv_fail(RX_ECUDA, "no CUDA device");
    s->running = true;
    try {
        s->loop = std::thread(loop_main, s, dev);
    } catch (const std::exception &e) {
        s->running = false;
        return srv_fail(RX_ENOMEM, std::string("cannot start the server's thread: ") + e.what());
    }
    return RX_OK;
}

int rx_server_stop(rx_server *s) {
    if (!s) return srv_fail(RX_EINVAL, "NULL server");
    if (!s->running) return srv_fail(RX_ESTATE, "the server's loop is not running");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->running = false;
    }
    s->cv.notify_all();
    s->loop.join();
    return RX_OK;
}

int rx_server_poll(rx_server *s, uint64_t id, int *state, rx_stats *stats) {
    if (!s || !state) return srv_fail(RX_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return srv_fail(RX_EINVAL, "unknown request id");
    Req *q = it->second.get();
    *state = q->state;
    if (stats && q->state == Q_DONE) *stats = q->stats;
    if (q->state == Q_FAILED) g_srv_err = q->err;
    return RX_OK;
}

int rx_server_set_param(rx_server *s, const char *key, double value) {
    if (!s || !key) return srv_fail(RX_EINVAL, "NULL argument");
    const std::string k(key);
    std::lock_guard<std::mutex> lock(s->mu);
    if (k == "issue") {
        if (value != 0 && value != 1 && value != 2) return srv_fail(RX_EINVAL, "issue must be 0, 1 or 2");
        s->issue = (int)value;
    } else if (k == "issue_threads") {
        if (!(value >= 1 && value <= 64) || value != (double)(long)value)
            return srv_fail(RX_EINVAL, "issue_threads must be 1 .. 64");
        s->issue_threads = (size_t)value;
    } else if (k == "block_latency") {
        if (value != 0 && value != 1) return srv_fail(RX_EINVAL, "block_latency must be 0 or 1");
        s->block_latency = value != 0;
        if (s->block_latency) s->blk_ms.clear();
    } else if (k == "blocks_per_step") {
        if (!(value >= 1 && value <= 1 << 20) || value != (double)(long)value)
            return srv_fail(RX_EINVAL, "blocks_per_step must be 1 .. 2^20");
        s->blocks_per_step = (long)value;
    } else {
        return srv_fail(RX_EINVAL, "unknown server parameter '" + k + "'");
    }
    return RX_OK;
}

int rx_server_get_param(const rx_server *s, const char *key, double *value) {
    if (!s || !key || !value) return srv_fail(RX_EINVAL, "NULL argument");
    const std::string k(key);
    std::lock_guard<std::mutex> lock(s->mu);
    if (k == "issue") *value = s->issue;
    else if (k == "running") *value = s->running ? 1 : 0;
    else if (k == "issue_threads") *value = (double)s->issue_threads;
    else if (k == "blocks_per_step") *value = (double)s->blocks_per_step;
    else if (k == "block_latency") *value = s->block_latency ? 1 : 0;
    else if (k == "handles_created") *value = (double)s->n_created;
    else if (k == "handles_destroyed") *value = (double)s->n_destroyed;
    else if (k == "handle_regrows") *value = (double)s->n_regrown;
    else return srv_fail(RX_EINVAL, "unknown server parameter '" + k + "'");
    return RX_OK;
}

int rx_server_get_block_latency(const rx_server *s, double *ms, size_t cap, size_t *n) {
    if (!s || !n || (cap && !ms)) return srv_fail(RX_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    *n = s->blk_ms.size();
    std::copy(s->blk_ms.begin(), s->blk_ms.begin() + (long)std::min(cap, s->blk_ms.size()), ms);
    return RX_OK;
}

int rx_server_info(rx_server *s, size_t *mem_used, int *max_active, long *steps) {
    if (!s) return srv_fail(RX_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lock(s->mu);
    if (mem_used) *mem_used = s->used;
    if (max_active) *max_active = s->max_active_seen;
    if (steps) *steps = s->steps;
    return RX_OK;
}

}  // extern "C"
