// server.cu -- the influence oracle as a serving loop with continuous
// batching (queries of Section 5.1, Eq. unionest, over resident sketches).
//
// Requests are seed sets submitted from any host thread.  A server thread
// admits pending requests into a launch group while in-flight slots and
// scratch memory allow (each query needs a hash table of about 2|S|(k-1)
// slots), copies the group's seeds to the device and launches the batched
// query kernel on one of several streams.  Groups on different streams run
// concurrently; when a group finishes, its slots and scratch return to the
// pool and requests that arrived meanwhile are admitted into the next group.
// Every query's estimate is an exact fixed-point sum rounded once, so a
// result is bitwise the same alone, in any group and on any stream.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"
#include "skim.h"

using namespace skim;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    std::vector<uint32_t> seeds;
    uint64_t slots;  // hash-table slots it needs
};

struct Lane {  // one stream and its buffers
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    uint64_t arena_slots = 0;
    uint64_t *hk = nullptr, *hv = nullptr;
    uint32_t *d_seeds = nullptr, *h_seeds = nullptr;
    uint64_t seed_cap = 0;
    uint64_t *d_meta = nullptr, *h_meta = nullptr;  // seed | table | chunk offsets, 3 x (group_cap + 1)
    double *d_out = nullptr, *h_out = nullptr;
    unsigned *d_err = nullptr;
    uint64_t *d_top = nullptr;
    unsigned *d_topu = nullptr;
    void *d_part = nullptr;
    uint64_t part_cap = 0;
    uint32_t group_cap = 0;
    std::vector<uint64_t> tickets;
};

uint64_t table_slots(uint64_t s, uint32_t k) {
    uint64_t need = std::max<uint64_t>(64, 2 * s * (k - 1) + 2), p = 1;
    while (p < need) p <<= 1;
    return p;
}

}  // namespace

struct skim_server {
    const uint64_t *X = nullptr;
    const uint32_t *xlen = nullptr;
    uint32_t n = 0, k = 0, l = 0;
    QueryTerms terms{0, 0.0, 1.0};
    uint32_t max_inflight = 0;
    std::vector<Lane> lanes;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;
    std::unordered_map<uint64_t, double> results;
    std::unordered_map<uint64_t, Clock::time_point> finished_at;
    uint64_t next_ticket = 1;
    uint32_t inflight = 0;
    bool stopping = false;
    int error = SKIM_OK;
    uint64_t groups = 0, grouped = 0;
    std::thread worker;
    bool record_times = false;
};

namespace {

void free_lane(Lane &ln) {
    if (ln.st) cudaStreamSynchronize(ln.st);
    if (ln.hk) cudaFree(ln.hk);
    if (ln.hv) cudaFree(ln.hv);
    if (ln.d_seeds) cudaFree(ln.d_seeds);
    if (ln.d_meta) cudaFree(ln.d_meta);
    if (ln.d_out) cudaFree(ln.d_out);
    if (ln.d_err) cudaFree(ln.d_err);
    if (ln.d_top) cudaFree(ln.d_top);
    if (ln.d_topu) cudaFree(ln.d_topu);
    if (ln.d_part) cudaFree(ln.d_part);
    if (ln.h_seeds) cudaFreeHost(ln.h_seeds);
    if (ln.h_meta) cudaFreeHost(ln.h_meta);
    if (ln.h_out) cudaFreeHost(ln.h_out);
    if (ln.done) cudaEventDestroy(ln.done);
    if (ln.st) cudaStreamDestroy(ln.st);
    ln = Lane{};
}

// Retire finished groups (lock held).
void retire(skim_server *s) {
    for (auto &ln : s->lanes) {
        if (!ln.busy) continue;
        cudaError_t q = cudaEventQuery(ln.done);
        if (q == cudaErrorNotReady) continue;
        const Clock::time_point now = Clock::now();
        if (q != cudaSuccess) s->error = SKIM_ECUDA;
        for (size_t i = 0; i < ln.tickets.size(); i++) {
            s->results[ln.tickets[i]] = ln.h_out[i];
            if (s->record_times) s->finished_at[ln.tickets[i]] = now;
        }
        s->inflight -= static_cast<uint32_t>(ln.tickets.size());
        ln.tickets.clear();
        ln.busy = false;
        s->cv_done.notify_all();
    }
}

// Admit pending requests into one group on a free lane and launch it (lock
// held; the launch itself is asynchronous).
bool admit(skim_server *s) {
    if (s->pending.empty()) return false;
    Lane *ln = nullptr;
    for (auto &c : s->lanes)
        if (!c.busy) {
            ln = &c;
            break;
        }
    if (!ln) return false;
    uint64_t used = 0, nseeds = 0, chunks = 0;
    uint32_t cnt = 0;
    const size_t g1 = static_cast<size_t>(ln->group_cap) + 1;
    uint64_t *h_off = ln->h_meta, *h_toff = ln->h_meta + g1, *h_coff = ln->h_meta + 2 * g1;
    h_off[0] = h_toff[0] = h_coff[0] = 0;
    while (!s->pending.empty() && cnt < ln->group_cap && s->inflight + cnt < s->max_inflight) {
        Request &r = s->pending.front();
        if (used + r.slots > ln->arena_slots || nseeds + r.seeds.size() > ln->seed_cap) break;  // memory admission
        if (!r.seeds.empty()) std::memcpy(ln->h_seeds + nseeds, r.seeds.data(), r.seeds.size() * sizeof(uint32_t));
        nseeds += r.seeds.size();
        used += r.slots;
        chunks += query_chunks(r.slots);
        h_off[cnt + 1] = nseeds;
        h_toff[cnt + 1] = used;
        h_coff[cnt + 1] = chunks;
        ln->tickets.push_back(r.ticket);
        cnt++;
        s->pending.pop_front();
    }
    if (cnt == 0) return false;
    s->inflight += cnt;
    s->groups++;
    s->grouped += cnt;
    ln->busy = true;
    bool ok = true;
    if (nseeds)
        ok &= cudaMemcpyAsync(ln->d_seeds, ln->h_seeds, nseeds * sizeof(uint32_t), cudaMemcpyHostToDevice, ln->st) ==
              cudaSuccess;
    ok &= cudaMemcpyAsync(ln->d_meta, ln->h_meta, 3 * g1 * sizeof(uint64_t), cudaMemcpyHostToDevice, ln->st) ==
          cudaSuccess;
    QueryScratch qs{ln->hk, ln->hv, ln->d_top, ln->d_topu, ln->d_part, ln->d_err};
    ok &= launch_query_multi(s->X, s->xlen, s->n, s->k, s->terms, ln->d_seeds, ln->d_meta, ln->d_meta + g1,
                             ln->d_meta + 2 * g1, cnt, used, nseeds, static_cast<uint32_t>(chunks), qs, ln->d_out,
                             ln->st) == cudaSuccess;
    ok &= cudaMemcpyAsync(ln->h_out, ln->d_out, cnt * sizeof(double), cudaMemcpyDeviceToHost, ln->st) == cudaSuccess;
    ok &= cudaEventRecord(ln->done, ln->st) == cudaSuccess;
    if (!ok) s->error = SKIM_ECUDA;
    return true;
}

void serve(skim_server *s, int device) {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        retire(s);
        while (admit(s)) {
        }
        bool busy = false;
        for (auto &ln : s->lanes) busy |= ln.busy;
        if (s->stopping && !busy && s->pending.empty()) break;
        if (busy) {
            // groups in flight: poll their events at a short interval
            lock.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(5));
            lock.lock();
        } else {
            s->cv_work.wait(lock, [&] { return s->stopping || !s->pending.empty(); });
        }
    }
}

}  // namespace

extern "C" {

int skim_server_start(skim_ctx *ctx, uint32_t max_inflight, uint64_t scratch_slots, uint32_t streams,
                      skim_server **out) {
    if (!ctx || !out || max_inflight == 0 || streams == 0 || streams > 16) return SKIM_EINVAL;
    *out = nullptr;
    const uint64_t *X = nullptr;
    const uint32_t *xlen = nullptr;
    int rc = skim_sketch_pointers(ctx, &X, &xlen);
    if (rc) return rc;
    uint32_t n = 0, k = 0, l = 0;
    rc = skim_context_shape(ctx, &n, &k, &l);
    if (rc) return rc;
    skim_server *s = new skim_server();
    s->X = X;
    s->xlen = xlen;
    s->n = n;
    s->k = k;
    s->l = l;
    s->terms = query_terms_of(ctx);
    s->max_inflight = max_inflight;
    s->lanes.resize(streams);
    const uint64_t arena = std::max<uint64_t>(scratch_slots / streams, 64);
    const uint32_t gcap = std::max<uint32_t>(1, max_inflight);
    bool ok = true;
    for (auto &ln : s->lanes) {
        ln.arena_slots = arena;
        ln.group_cap = gcap;
        ln.seed_cap = arena / 2 + gcap;  // a query of |S| seeds takes at least 2|S| slots
        ok &= cudaStreamCreateWithFlags(&ln.st, cudaStreamNonBlocking) == cudaSuccess;
        ok &= cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming) == cudaSuccess;
        ok &= cudaMalloc(&ln.hk, arena * sizeof(uint64_t)) == cudaSuccess;
        ok &= cudaMalloc(&ln.hv, arena * sizeof(uint64_t)) == cudaSuccess;
        ok &= cudaMalloc(&ln.d_seeds, ln.seed_cap * sizeof(uint32_t)) == cudaSuccess;
        ln.part_cap = arena / 64 + gcap;  // chunks: at most one per 64 slots (smallest table) per query
        ok &= cudaMalloc(&ln.d_meta, 3 * (gcap + 1) * sizeof(uint64_t)) == cudaSuccess;
        ok &= cudaMalloc(&ln.d_out, gcap * sizeof(double)) == cudaSuccess;
        ok &= cudaMalloc(&ln.d_err, sizeof(unsigned)) == cudaSuccess;
        ok &= cudaMalloc(&ln.d_top, gcap * sizeof(uint64_t)) == cudaSuccess;
        ok &= cudaMalloc(&ln.d_topu, gcap * sizeof(unsigned)) == cudaSuccess;
        ok &= cudaMalloc(&ln.d_part, ln.part_cap * query_partial_bytes()) == cudaSuccess;
        ok &= cudaMallocHost(&ln.h_seeds, ln.seed_cap * sizeof(uint32_t)) == cudaSuccess;
        ok &= cudaMallocHost(&ln.h_meta, 3 * (gcap + 1) * sizeof(uint64_t)) == cudaSuccess;
        ok &= cudaMallocHost(&ln.h_out, gcap * sizeof(double)) == cudaSuccess;
        if (!ok) break;
    }
    if (!ok) {
        cudaGetLastError();
        for (auto &ln : s->lanes) free_lane(ln);
        delete s;
        return SKIM_ENOMEM;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    s->worker = std::thread(serve, s, dev);
    *out = s;
    return SKIM_OK;
}

int skim_server_submit(skim_server *s, const uint32_t *seeds, uint32_t n_seeds, uint64_t *ticket) {
    if (!s || !ticket || (n_seeds && !seeds)) return SKIM_EINVAL;
    for (uint32_t i = 0; i < n_seeds; i++)
        if (seeds[i] >= s->n) return SKIM_EINVAL;
    const uint64_t slots = table_slots(n_seeds, s->k);
    if (slots > s->lanes[0].arena_slots || n_seeds + 1 > s->lanes[0].seed_cap) return SKIM_ERANGE;
    Request r;
    r.seeds.assign(seeds, seeds + n_seeds);
    r.slots = slots;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stopping) return SKIM_EINVAL;
        if (s->error) return s->error;
        r.ticket = s->next_ticket++;
        *ticket = r.ticket;
        s->pending.push_back(std::move(r));
    }
    s->cv_work.notify_one();
    return SKIM_OK;
}

int skim_server_poll(skim_server *s, uint64_t ticket, int *done, double *est) {
    if (!s || !done || !est) return SKIM_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) {
        *done = 0;
        return s->error;
    }
    *done = 1;
    *est = it->second;
    s->results.erase(it);
    return SKIM_OK;
}

int skim_server_wait(skim_server *s, uint64_t ticket, double *est, uint32_t timeout_ms) {
    if (!s || !est) return SKIM_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    const bool got = s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), [&] {
        return s->results.count(ticket) != 0 || s->error != SKIM_OK;
    });
    if (!got) return SKIM_ETIMEOUT;
    if (s->error) return s->error;
    *est = s->results[ticket];
    s->results.erase(ticket);
    return SKIM_OK;
}

int skim_server_replay(skim_server *s, const double *arrival_s, const uint64_t *offsets, const uint32_t *seeds,
                       uint32_t q, double *latency_s, double *est_out) {
    if (!s || !offsets || (q && (!arrival_s || !latency_s || !est_out))) return SKIM_EINVAL;
    std::vector<uint64_t> tickets(q);
    std::vector<Clock::time_point> sent(q);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->record_times = true;
        s->finished_at.clear();
    }
    const Clock::time_point t0 = Clock::now();
    for (uint32_t i = 0; i < q; i++) {
        const Clock::time_point at = t0 + std::chrono::duration_cast<Clock::duration>(
                                              std::chrono::duration<double>(arrival_s[i]));
        while (Clock::now() < at) {
        }
        sent[i] = Clock::now();
        int rc = skim_server_submit(s, seeds + offsets[i], static_cast<uint32_t>(offsets[i + 1] - offsets[i]),
                                    &tickets[i]);
        if (rc) return rc;
    }
    for (uint32_t i = 0; i < q; i++) {
        int rc = skim_server_wait(s, tickets[i], &est_out[i], 60000);
        if (rc) return rc;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    for (uint32_t i = 0; i < q; i++)
        latency_s[i] = std::chrono::duration<double>(s->finished_at[tickets[i]] - sent[i]).count();
    s->record_times = false;
    s->finished_at.clear();
    return SKIM_OK;
}

int skim_server_stats(skim_server *s, uint64_t *groups, uint64_t *queries) {
    if (!s || !groups || !queries) return SKIM_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    *groups = s->groups;
    *queries = s->grouped;
    return SKIM_OK;
}

int skim_server_stop(skim_server *s) {
    if (!s) return SKIM_EINVAL;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    const int err = s->error;
    for (auto &ln : s->lanes) free_lane(ln);
    delete s;
    return err;
}

}  // extern "C"
