// Serving: continuous batching of events that arrive one by one (host side only).
//
// The paper's filter unit processes one event after another and overlaps the transfer of
// the next event with the processing of the current one (Sec. 8).  Here a request loop
// runs on `n_lanes` worker threads, each owning a complete trk handle (its own device
// pools, stream and captured graphs) sized for a micro-batch.  Submitted events wait in a
// host queue; whenever a lane is free it admits every waiting event that fits its
// capacities (events and hits), copies them in, reconstructs them in one call and hands
// each event's candidates back.  While one lane's batch is on the GPU the other lanes
// admit and launch what arrives meanwhile, so batches overlap on the device.  Geometry,
// binning and every pool stay resident for the server's lifetime.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "trk.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
    uint64_t ticket;
    std::vector<trk_hit> hits;
    Clock::time_point t_submit;
};

struct Done {
    int status = 0;
    int rc = 0;
    std::vector<trk_candidate> cand;   // hit_off relative to `hits`
    std::vector<int32_t> hits;         // event-local hit indices
    double latency_s = 0.0;
    int batch_events = 0;
};

}  // namespace

struct trk_server {
    std::vector<trk_ctx *> ctx;
    std::vector<std::thread> threads;
    std::vector<cudaStream_t> streams;
    std::vector<trk_hit *> stage_hits;       // pinned per lane
    std::vector<int64_t *> stage_offs;
    int32_t max_events = 1;
    int64_t max_hits = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Pending> queue;
    std::unordered_map<uint64_t, Done> done;
    uint64_t next_ticket = 1;
    bool stop = false;
    int64_t n_batches = 0, n_events_done = 0, n_failed = 0;
    std::string err;
};

static void lane_loop(trk_server *S, int lane)
{
    cudaSetDevice(S->device);
    trk_ctx *h = S->ctx[lane];
    std::vector<Pending> batch;
    for (;;) {
        batch.clear();
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
            if (S->stop && S->queue.empty())
                return;
            // admission: as many waiting events as the lane's capacities allow
            int64_t hits = 0;
            while (!S->queue.empty() && (int32_t)batch.size() < S->max_events &&
                   hits + (int64_t)S->queue.front().hits.size() <= S->max_hits) {
                hits += (int64_t)S->queue.front().hits.size();
                batch.push_back(std::move(S->queue.front()));
                S->queue.pop_front();
            }
        }
        if (batch.empty())
            continue;
        // pack into the lane's pinned staging buffers
        trk_hit *sh = S->stage_hits[lane];
        int64_t *so = S->stage_offs[lane];
        so[0] = 0;
        for (size_t e = 0; e < batch.size(); ++e) {
            const size_t n = batch[e].hits.size();
            if (n)
                std::memcpy(sh + so[e], batch[e].hits.data(), n * sizeof(trk_hit));
            so[e + 1] = so[e] + (int64_t)n;
        }
        trk_candidates out;
        std::memset(&out, 0, sizeof(out));
        const int rc = trk_reconstruct_host(h, sh, so[batch.size()], so, (int32_t)batch.size(),
                                            &out, S->streams[lane]);
        const auto t_done = Clock::now();
        std::vector<Done> results(batch.size());
        for (size_t e = 0; e < batch.size(); ++e) {
            Done &d = results[e];
            d.rc = rc;
            d.batch_events = (int)batch.size();
            d.latency_s = std::chrono::duration<double>(t_done - batch[e].t_submit).count();
            if (rc != TRK_OK && rc != TRK_ERR_CAPACITY) {
                d.status = -1;
                continue;
            }
            d.status = out.status[e];
            const int64_t c0 = out.cand_off[e], c1 = out.cand_off[e + 1];
            for (int64_t c = c0; c < c1 && out.h_cand; ++c) {
                trk_candidate r = out.h_cand[c];
                const int64_t src = r.hit_off;
                r.hit_off = (int64_t)d.hits.size();
                for (int q = 0; q < r.n_hits; ++q)
                    d.hits.push_back(out.h_hit_ids[src + q] - (int32_t)so[e]);
                r.event = 0;
                d.cand.push_back(r);
            }
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (size_t e = 0; e < batch.size(); ++e) {
                if (results[e].status != 0)
                    S->n_failed++;
                S->done.emplace(batch[e].ticket, std::move(results[e]));
            }
            S->n_batches++;
            S->n_events_done += (int64_t)batch.size();
        }
        S->cv_done.notify_all();
    }
}

static void server_free(trk_server *S)
{
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->threads)
        if (t.joinable())
            t.join();
    for (trk_ctx *h : S->ctx)
        trk_destroy(h);
    for (cudaStream_t s : S->streams)
        if (s)
            cudaStreamDestroy(s);
    for (trk_hit *p : S->stage_hits)
        if (p)
            cudaFreeHost(p);
    for (int64_t *p : S->stage_offs)
        if (p)
            cudaFreeHost(p);
    delete S;
}

extern "C" int trk_server_create(trk_server **out, const trk_geometry *geometry,
                                 const trk_binning *binning, const trk_options *lane_options,
                                 int32_t n_lanes)
{
    if (!out || !geometry || !binning || !lane_options || n_lanes < 1 || n_lanes > 16)
        return TRK_ERR_INVALID;
    *out = nullptr;
    trk_server *S = new trk_server();
    S->max_events = lane_options->max_events;
    S->max_hits = lane_options->max_hits;
    S->device = lane_options->device;
    trk_options lane = *lane_options;
    lane.fit_candidates = 0;            // served events return candidates and hits only
    lane.use_graph = 0;                 // no capture in lane threads: it would make device-
                                        // wide synchronisation elsewhere in the process invalid
    for (int l = 0; l < n_lanes; ++l) {
        trk_ctx *h = nullptr;
        const int rc = trk_create(&h, geometry, binning, &lane);
        if (rc != TRK_OK) {
            server_free(S);
            return rc;
        }
        S->ctx.push_back(h);
        cudaStream_t s = nullptr;
        trk_hit *ph = nullptr;
        int64_t *po = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMallocHost((void **)&ph, sizeof(trk_hit) * (size_t)S->max_hits) != cudaSuccess ||
            cudaMallocHost((void **)&po, sizeof(int64_t) * ((size_t)S->max_events + 1)) !=
                cudaSuccess) {
            if (s)
                cudaStreamDestroy(s);
            if (ph)
                cudaFreeHost(ph);
            server_free(S);
            return TRK_ERR_NOMEM;
        }
        S->streams.push_back(s);
        S->stage_hits.push_back(ph);
        S->stage_offs.push_back(po);
    }
    for (int l = 0; l < n_lanes; ++l)
        S->threads.emplace_back(lane_loop, S, l);
    *out = S;
    return TRK_OK;
}

extern "C" int trk_server_submit(trk_server *S, const trk_hit *hits, int64_t n_hits,
                                 uint64_t *ticket)
{
    if (!S || !ticket || n_hits < 0 || (n_hits > 0 && !hits))
        return TRK_ERR_INVALID;
    if (n_hits > S->max_hits)
        return TRK_ERR_CAPACITY;
    Pending p;
    p.hits.assign(hits, hits + n_hits);
    p.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        p.ticket = S->next_ticket++;
        *ticket = p.ticket;
        S->queue.push_back(std::move(p));
    }
    S->cv_work.notify_one();
    return TRK_OK;
}

extern "C" int trk_server_wait(trk_server *S, uint64_t ticket, double timeout_s,
                               trk_served_event *out)
{
    if (!S || !out)
        return TRK_ERR_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    const auto until = Clock::now() + std::chrono::duration<double>(timeout_s);
    while (S->done.find(ticket) == S->done.end()) {
        if (timeout_s <= 0.0 || S->cv_done.wait_until(lk, until) == std::cv_status::timeout) {
            if (S->done.find(ticket) == S->done.end())
                return TRK_PENDING;
        }
    }
    Done &d = S->done[ticket];
    out->status = d.status;
    out->rc = d.rc;
    out->latency_s = d.latency_s;
    out->batch_events = d.batch_events;
    out->n_candidates = (int64_t)d.cand.size();
    out->n_hit_ids = (int64_t)d.hits.size();
    return TRK_OK;
}

extern "C" int trk_server_take(trk_server *S, uint64_t ticket, trk_candidate *cand,
                               int64_t cand_cap, int32_t *hit_ids, int64_t hit_cap)
{
    if (!S)
        return TRK_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->done.find(ticket);
    if (it == S->done.end())
        return TRK_PENDING;
    const Done &d = it->second;
    if ((int64_t)d.cand.size() > cand_cap || (int64_t)d.hits.size() > hit_cap)
        return TRK_ERR_CAPACITY;
    if (!d.cand.empty() && cand)
        std::memcpy(cand, d.cand.data(), d.cand.size() * sizeof(trk_candidate));
    if (!d.hits.empty() && hit_ids)
        std::memcpy(hit_ids, d.hits.data(), d.hits.size() * sizeof(int32_t));
    S->done.erase(it);
    return TRK_OK;
}

extern "C" int trk_server_counts(trk_server *S, int64_t *n_batches, int64_t *n_events,
                                 int64_t *n_failed, int64_t *n_queued)
{
    if (!S)
        return TRK_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    if (n_batches)
        *n_batches = S->n_batches;
    if (n_events)
        *n_events = S->n_events_done;
    if (n_failed)
        *n_failed = S->n_failed;
    if (n_queued)
        *n_queued = (int64_t)S->queue.size();
    return TRK_OK;
}

extern "C" int trk_server_destroy(trk_server *S)
{
    if (S)
        server_free(S);
    return TRK_OK;
}
