// Serving loop with continuous batching over receiver handles.
//
// A request is one stream (any built-in or custom format, its own link and
// receiver parameters).  Requests wait in a FIFO queue until a slot is free
// and their device-memory estimate fits the budget; an admitted request gets
// its own handle and CUDA stream and is processed one block at a time,
// interleaved with every other admitted request, so the work of requests
// that arrived at different times overlaps on the device.  A finished
// request frees its handle (memory and slot) and the queue's head is
// admitted at the next step.  Each request's computation is that of a
// handle processing the stream alone (the library's kernels are
// deterministic), so its results do not depend on the mix.
//
// Host code only; everything on the device goes through the public entry
// points (rx_create, rx_process_blocks, rx_get_stats, ...).
#include <cstring>
#include <deque>
#include <memory>
#include <string>
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
    double t_submit = 0, t_admit = 0, t_done = 0;   // server step counters
};

size_t estimate_bytes(const rx_request &r) {
    // per symbol: CDC output 32 B, FIR output 16 B, phase index 1 B, phase
    // code 2 B, reference labels 2 B; plus tables, taps ring and partials
    const size_t N = r.n_samples / 2;
    return 53 * N + (1u << 20);
}

}  // namespace

struct rx_server {
    size_t budget = 0, used = 0;
    int max_slots = 1;
    uint64_t next_id = 1;
    long steps = 0;
    std::deque<Req *> queue;
    std::vector<Req *> active;
    std::unordered_map<uint64_t, std::unique_ptr<Req>> all;
    int max_active_seen = 0;
};

namespace {

thread_local std::string g_srv_err;

int srv_fail(int code, const std::string &msg) {
    g_srv_err = msg;
    return code;
}

void release(rx_server *s, Req *q) {
    if (q->h) { rx_destroy(q->h); q->h = nullptr; }
    if (q->done) { cudaEventDestroy(q->done); q->done = nullptr; }
    if (q->st) { cudaStreamDestroy(q->st); q->st = nullptr; }
    s->used -= q->mem;
}

// create the handle of an admitted request; false (and FAILED) on error
bool admit(rx_server *s, Req *q) {
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
    int rc = RX_OK;
    if (q->r.fft) rc |= rx_set_param(q->h, "fft", q->r.fft);
    if (q->r.overlap) rc |= rx_set_param(q->h, "overlap", q->r.overlap);
    if (q->r.block) rc |= rx_set_param(q->h, "block", q->r.block);
    if (q->r.n_pre) rc |= rx_set_param(q->h, "n_pre", q->r.n_pre);
    if (rc == RX_OK && cudaStreamCreateWithFlags(&q->st, cudaStreamNonBlocking) != cudaSuccess) rc = RX_ECUDA;
    if (rc == RX_OK && cudaEventCreateWithFlags(&q->done, cudaEventDisableTiming) != cudaSuccess) rc = RX_ECUDA;
    if (rc == RX_OK) rc = rx_set_stream(q->h, q->st);
    if (rc == RX_OK && q->r.ref_bits) rc = rx_set_reference(q->h, q->r.ref_bits, q->N);
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

extern "C" {

const char *rx_server_last_error(void) { return g_srv_err.c_str(); }

rx_server *rx_server_create(size_t mem_budget_bytes, int max_slots) {
    if (max_slots < 1 || max_slots > 1024 || mem_budget_bytes == 0) {
        srv_fail(RX_EINVAL, "rx_server_create: budget must be > 0 and slots 1..1024");
        return nullptr;
    }
    rx_server *s = new rx_server();
    s->budget = mem_budget_bytes;
    s->max_slots = max_slots;
    return s;
}

void rx_server_destroy(rx_server *s) {
    if (!s) return;
    for (Req *q : s->active) {
        if (q->st) cudaStreamSynchronize(q->st);
        release(s, q);
    }
    delete s;
}

int rx_server_submit(rx_server *s, const rx_request *r, uint64_t *id) {
    if (!s || !r || !id) return srv_fail(RX_EINVAL, "NULL argument");
    if (!r->samples || !r->llr_out || r->n_samples < 2 || (r->n_samples & 1))
        return srv_fail(RX_EINVAL, "request needs device samples, an even n_samples and an LLR buffer");
    auto q = std::make_unique<Req>();
    q->id = s->next_id++;
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
    if (q->mem > s->budget)
        return srv_fail(RX_EINVAL, "request needs about " + std::to_string(q->mem) +
                                       " bytes, more than the whole budget");
    q->t_submit = (double)s->steps;
    *id = q->id;
    s->queue.push_back(q.get());
    s->all[q->id] = std::move(q);
    return RX_OK;
}

int rx_server_step(rx_server *s, int *n_active) {
    if (!s) return srv_fail(RX_EINVAL, "NULL server");
    ++s->steps;
    // retire requests whose last block has finished
    for (size_t i = 0; i < s->active.size();) {
        Req *q = s->active[i];
        if (q->next >= q->nblk && cudaEventQuery(q->done) == cudaSuccess) {
            if (rx_get_stats(q->h, &q->stats) != RX_OK) q->err = rx_last_error();
            q->state = q->err.empty() ? Q_DONE : Q_FAILED;
            q->t_done = (double)s->steps;
            release(s, q);
            s->active.erase(s->active.begin() + (long)i);
        } else {
            ++i;
        }
    }
    // admit from the head of the queue while a slot and memory are free
    while (!s->queue.empty() && (int)s->active.size() < s->max_slots &&
           s->used + s->queue.front()->mem <= s->budget) {
        Req *q = s->queue.front();
        s->queue.pop_front();
        if (admit(s, q)) s->active.push_back(q);
    }
    if ((int)s->active.size() > s->max_active_seen) s->max_active_seen = (int)s->active.size();
    // one block of every running request, each on its own stream
    for (Req *q : s->active) {
        if (q->next >= q->nblk) continue;
        const int rc = rx_process_blocks(q->h, q->r.samples, q->r.n_samples, (size_t)q->next,
                                         (size_t)q->next + 1, q->r.llr_out, nullptr);
        if (rc != RX_OK) {
            q->err = rx_last_error();
            q->next = q->nblk;
        } else {
            ++q->next;
        }
        if (q->next >= q->nblk) cudaEventRecord(q->done, q->st);
    }
    if (n_active) *n_active = (int)(s->active.size() + s->queue.size());
    return RX_OK;
}

int rx_server_run(rx_server *s) {
    if (!s) return srv_fail(RX_EINVAL, "NULL server");
    int left = 1;
    while (left > 0) {
        const int rc = rx_server_step(s, &left);
        if (rc != RX_OK) return rc;
        if (left > 0 && !s->active.empty()) {
            // all blocks issued: wait for the oldest running request
            bool issued = true;
            for (Req *q : s->active) issued &= q->next >= q->nblk;
            if (issued) cudaEventSynchronize(s->active.front()->done);
        }
    }
    return RX_OK;
}

int rx_server_poll(rx_server *s, uint64_t id, int *state, rx_stats *stats) {
    if (!s || !state) return srv_fail(RX_EINVAL, "NULL argument");
    auto it = s->all.find(id);
    if (it == s->all.end()) return srv_fail(RX_EINVAL, "unknown request id");
    Req *q = it->second.get();
    *state = q->state;
    if (stats && q->state == Q_DONE) *stats = q->stats;
    if (q->state == Q_FAILED) g_srv_err = q->err;
    return RX_OK;
}

int rx_server_info(rx_server *s, size_t *mem_used, int *max_active, long *steps) {
    if (!s) return srv_fail(RX_EINVAL, "NULL server");
    if (mem_used) *mem_used = s->used;
    if (max_active) *max_active = s->max_active_seen;
    if (steps) *steps = s->steps;
    return RX_OK;
}

}  // extern "C"
