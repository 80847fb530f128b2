// Serving loop: a device-resident index answers threshold queries that
// arrive one at a time, with continuous batching.
//
// Requests wait in one queue.  Each of the server's worker threads owns a
// CUDA stream; when it is free it takes the oldest waiting requests as one
// micro-batch -- as many as fit both max_batch and the memory budget still
// unclaimed by the batches in flight (scratch of a query slot plus the
// worst-case size of its result) -- runs it through the batched executor
// (thr_batch.cu, graph replay included) and hands each result back.  So
// requests that arrive while others are on the GPU join the next
// micro-batch as soon as a worker and memory are free, and the micro-batches
// of different workers overlap on the device.  A batch with no other batch
// in flight always admits its first request, so an oversized request still
// runs (alone).  Results do not depend on the batch a request lands in.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/thr.h"
#include "thr_batch.h"
#include "thr_index.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    std::vector<uint32_t> ids;
    uint32_t T = 0;
    std::vector<uint64_t> result;
    thr_status status = THR_OK;
    std::string error;
    Clock::time_point t_submit, t_start, t_done;
    uint64_t cost = 0;  // bytes claimed from the budget while in flight
    bool done = false;
    bool waited = false;  // a thr_server_wait call has claimed it
};

}  // namespace

struct thr_server {
    const thr_index* idx = nullptr;
    uint32_t max_batch = 1;
    uint64_t budget = 0;
    uint32_t flags = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, Request*> live;
    uint64_t next_ticket = 1;
    uint64_t claimed = 0;  // budget bytes held by batches in flight
    uint32_t in_flight = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    // statistics
    uint64_t n_done = 0, n_batches = 0, batch_queries = 0;
    uint32_t max_in_flight = 0, max_batch_seen = 0;
    uint64_t max_claimed = 0;
};

namespace {

uint64_t request_cost(const thr_index* idx) {
    return thr::scratch_per_slot(idx->W, idx->NG) + 8 * (uint64_t(idx->W) + 1);
}

void run_micro_batch(thr_server* s, std::vector<Request*>& batch, cudaStream_t st,
                     uint64_t*& dpool, uint64_t& dpool_cap, std::vector<uint64_t>& host) {
    const uint32_t nq = uint32_t(batch.size());
    std::vector<uint32_t> id_off(nq + 1, 0), ids, T(nq);
    for (uint32_t q = 0; q < nq; ++q) {
        id_off[q + 1] = id_off[q] + uint32_t(batch[q]->ids.size());
        ids.insert(ids.end(), batch[q]->ids.begin(), batch[q]->ids.end());
        T[q] = batch[q]->T;
    }
    const uint64_t cap = uint64_t(nq) * (uint64_t(s->idx->W) + 1);
    // counting variant of each query under the server's policy (one model
    // evaluation for the whole micro-batch)
    std::vector<uint8_t> var;
    thr_status rs = thr::choose_variants(s->idx, nq, id_off.data(), ids.data(), T.data(),
                                         s->flags & THR_POLICY_MASK, s->flags & THR_VARIANT_MASK,
                                         &var);
    if (rs == THR_OK && dpool_cap < cap) {
        cudaFree(dpool);
        dpool = nullptr;
        dpool_cap = 0;
        if (cudaMalloc(&dpool, sizeof(uint64_t) * cap) != cudaSuccess) {
            cudaGetLastError();
            rs = thr::report_error(THR_E_NOMEM, "server: result pool");
        } else {
            dpool_cap = cap;
        }
    }
    std::vector<uint64_t> off(nq), len(nq);
    uint64_t total = 0;
    if (rs == THR_OK) {
        thr::BatchInput in{nq, id_off.data(), ids.data(), T.data(), var.data()};
        thr::BatchOptions opt;
        opt.graph = true;
        rs = thr::run_batch(s->idx, in, dpool, dpool_cap, off.data(), len.data(), &total, st,
                            opt, nullptr);
    }
    if (rs == THR_OK && total) {
        host.resize(total);
        if (cudaMemcpyAsync(host.data(), dpool, sizeof(uint64_t) * total,
                            cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            rs = thr::report_error(THR_E_CUDA, "server: copy results");
        }
    }
    for (uint32_t q = 0; q < nq; ++q) {
        Request* r = batch[q];
        r->status = rs;
        if (rs == THR_OK)
            r->result.assign(host.begin() + off[q], host.begin() + off[q] + len[q]);
        else
            r->error = thr_last_error();
    }
}

void worker_main(thr_server* s) {
    cudaSetDevice(s->idx->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    uint64_t* dpool = nullptr;
    uint64_t dpool_cap = 0;
    std::vector<uint64_t> host;
    const uint64_t cost = request_cost(s->idx);
    for (;;) {
        std::vector<Request*> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] {
                if (s->pending.empty()) return s->stop;
                return s->in_flight == 0 || s->claimed + cost <= s->budget;
            });
            if (s->pending.empty()) break;  // stopping, nothing left
            uint64_t claim = 0;
            while (!s->pending.empty() && batch.size() < s->max_batch &&
                   (batch.empty() && s->in_flight == 0
                        ? true
                        : s->claimed + claim + cost <= s->budget)) {
                Request* r = s->pending.front();
                s->pending.pop_front();
                r->cost = cost;
                r->t_start = Clock::now();
                claim += cost;
                batch.push_back(r);
            }
            if (batch.empty()) continue;
            s->claimed += claim;
            s->max_claimed = std::max(s->max_claimed, s->claimed);
            ++s->in_flight;
            s->max_in_flight = std::max(s->max_in_flight, s->in_flight);
            ++s->n_batches;
            s->batch_queries += batch.size();
            s->max_batch_seen = std::max<uint32_t>(s->max_batch_seen, uint32_t(batch.size()));
        }
        run_micro_batch(s, batch, st, dpool, dpool_cap, host);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            const auto now = Clock::now();
            for (Request* r : batch) {
                r->t_done = now;
                r->done = true;
                s->claimed -= r->cost;
                ++s->n_done;
            }
            --s->in_flight;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
    cudaFree(dpool);
    cudaStreamDestroy(st);
}

}  // namespace

using thr::report_error;

extern "C" {

thr_status thr_server_create(const thr_index* idx, uint32_t workers, uint32_t max_batch,
                             uint64_t mem_budget, uint32_t flags, thr_server** out) {
    if (!idx || !out) return report_error(THR_E_INVAL, "null argument");
    if (workers == 0 || workers > 64) return report_error(THR_E_INVAL, "workers must be 1..64");
    if (max_batch == 0) return report_error(THR_E_INVAL, "max_batch must be at least 1");
    if (flags & ~(THR_POLICY_MASK | THR_VARIANT_MASK))
        return report_error(THR_E_INVAL, "unknown flags");
    const uint32_t policy = flags & THR_POLICY_MASK;
    if (policy != THR_POLICY_PLAIN && policy != THR_POLICY_RULE && policy != THR_POLICY_LEARNED)
        return report_error(THR_E_INVAL, "unknown policy");
    if (thr::variant_of_flag(flags & THR_VARIANT_MASK) < 0)
        return report_error(THR_E_INVAL, "unknown variant");
    thr_server* s = new (std::nothrow) thr_server;
    if (!s) return report_error(THR_E_NOMEM, "server");
    s->idx = idx;
    s->max_batch = max_batch;
    s->budget = mem_budget;
    s->flags = flags;
    try {
        for (uint32_t i = 0; i < workers; ++i) s->workers.emplace_back(worker_main, s);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        for (auto& t : s->workers) t.join();
        delete s;
        return report_error(THR_E_NOMEM, "server threads");
    }
    *out = s;
    return THR_OK;
}

thr_status thr_server_submit(thr_server* s, const uint32_t* ids, uint32_t n, uint32_t T,
                             uint64_t* ticket) {
    if (!s || !ids || !ticket) return report_error(THR_E_INVAL, "null argument");
    if (n == 0 || n > THR_MAX_IDS)
        return report_error(THR_E_INVAL, "n must be in 1..THR_MAX_IDS (2^20 - 1)");
    for (uint32_t i = 0; i < n; ++i)
        if (ids[i] >= s->idx->nbitmaps) return report_error(THR_E_INVAL, "id out of range");
    Request* r = new (std::nothrow) Request;
    if (!r) return report_error(THR_E_NOMEM, "request");
    r->ids.assign(ids, ids + n);
    r->T = T;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return report_error(THR_E_INVAL, "server is stopping");
        }
        r->ticket = s->next_ticket++;
        s->live[r->ticket] = r;
        s->pending.push_back(r);
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return THR_OK;
}

thr_status thr_server_wait(thr_server* s, uint64_t ticket, uint64_t* out, uint64_t cap,
                           uint64_t* out_len, double* latency_ms) {
    if (!s || !out_len || (cap > 0 && !out)) return report_error(THR_E_INVAL, "null argument");
    Request* r = nullptr;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->live.find(ticket);
        if (it == s->live.end()) return report_error(THR_E_INVAL, "unknown ticket");
        r = it->second;
        if (r->waited)
            return report_error(THR_E_INVAL, "another thr_server_wait call has this ticket");
        r->waited = true;
        s->cv_done.wait(lk, [&] { return r->done; });
        // by key, not by the iterator found before the wait: submissions made
        // while this thread waited (the lock is released then) may have
        // rehashed the map and invalidated every iterator into it
        s->live.erase(ticket);
    }
    const thr_status st = r->status;
    const std::string err = r->error;
    *out_len = r->result.size();
    if (latency_ms)
        *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    if (st == THR_OK && r->result.size() <= cap && !r->result.empty())
        std::memcpy(out, r->result.data(), sizeof(uint64_t) * r->result.size());
    const bool fits = r->result.size() <= cap;
    delete r;
    if (st != THR_OK) return report_error(st, err.c_str());
    if (!fits) return report_error(THR_E_NOSPACE, "output buffer too small");
    return THR_OK;
}

thr_status thr_server_stats(thr_server* s, uint64_t* stats) {
    if (!s || !stats) return report_error(THR_E_INVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    stats[0] = s->n_done;
    stats[1] = s->n_batches;
    stats[2] = s->batch_queries;
    stats[3] = s->max_in_flight;
    stats[4] = s->max_batch_seen;
    stats[5] = s->max_claimed;
    stats[6] = s->pending.size();
    stats[7] = s->in_flight;
    return THR_OK;
}

void thr_server_free(thr_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->live) delete kv.second;
    delete s;
}

}  // extern "C"
