// Serving: continuous batching of events that arrive one by one (host side only).
//
// The paper's filter unit processes one event after another and overlaps the transfer of
// the next event with the processing of the current one (Sec. 8).  Here a request loop
// runs on `n_lanes` worker threads, each owning a complete trk handle (its own device
// pools, stream and captured graphs) sized for a micro-batch.  Submitted events wait in a
// host queue; whenever a lane is free it admits the waiting events, in arrival order, that
// fit its capacities -- events, hits, and device memory for their votes -- copies them in,
// reconstructs them in one call and hands each event's candidates back.  The lanes take
// the GPU in turn: a free lane forms its batch from the events waiting then, packs it and
// queues its copy to the device while another lane's batch computes, then holds the GPU
// from launching its kernels until they have finished, releases it, and copies the
// results back and files them while the next lane's batch computes.  So the transfers and
// the host work of one batch overlap the computation of another, and batches do not slow
// each other down by sharing the GPU.
//
// Batch size follows the backlog.  Batching k events saves a few per cent of each event's
// device time (fewer launches and tails; about 4 % at four events of the 256-event mix on
// GB300), but every event of the batch gets its results only when the last one is done,
// up to k - 1 event times later.  Taking k events pays only when the saving, summed over
// the events still waiting behind them, exceeds that delay, i.e. when about 25 (k - 1)
// events wait; so a lane takes one event more per kBacklogPerExtra waiting ones, and a
// lightly loaded server runs one event per call while a backed-up one runs full batches.
// Geometry, binning and every pool stay resident for the server's lifetime.
//
// Memory-sized admission: an event's votes are bounded by its hit triplets
// (sum over layer triples of |La||Lb||Lc|, counted from its hits at submission) times the
// largest acceptance fraction seen so far (starting from 1/2); a lane admits events while
// that bound fits the vote list it was given.  When the lanes are created with
// vote_capacity 0, the vote list is sized from the device memory free at creation
// (cudaMemGetInfo), shared equally by the lanes.  A batch whose votes still overflow is
// reconstructed again one event at a time.
#include <algorithm>
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
    int64_t triplets = 0;             // sum over layer triples of |La||Lb||Lc|
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

namespace trk {
int capture_call_graphs(trk_ctx *h, int max_events);
int64_t event_device_bytes(const trk_ctx *h, int64_t votes);
}  // namespace trk

struct trk_server {
    std::vector<trk_ctx *> ctx;
    std::vector<std::thread> threads;
    std::vector<cudaStream_t> streams;
    std::vector<trk_hit *> stage_hits;       // pinned per lane
    std::vector<int64_t *> stage_offs;
    std::vector<trk_hit *> d_hits;           // device inputs per lane
    std::vector<int64_t *> d_offs;
    std::vector<trk_candidate *> res_cand;   // pinned results per lane
    std::vector<int32_t *> res_hits;
    int64_t cand_cap = 0, hit_cap = 0;
    std::mutex gpu_mu;                       // held by the lane whose batch computes
    int32_t max_events = 1;
    int64_t max_hits = 0;
    int64_t vote_budget = 0;                 // votes a lane's vote list holds
    double accept_max = 0.5;                 // largest votes / triplets seen (admission bound)
    int device = 0;
    int n_layers = 0, n_triples = 0;
    std::vector<int32_t> triples;            // 3 per layer triple
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Pending> queue;
    std::unordered_map<uint64_t, Done> done;
    uint64_t next_ticket = 1;
    bool stop = false;
    int64_t n_batches = 0, n_events_done = 0, n_failed = 0;
    std::string err;
};

// Waiting events per event added to a batch beyond the first (see above).
constexpr size_t kBacklogPerExtra = 24;

// Admission, in arrival order: events, hits and the vote-list bound must fit; the first
// event always fits a lane (submission checks its hits).  Called with S->mu held.
static void admit(trk_server *S, std::vector<Pending> &batch)
{
    int64_t hits = 0;
    double votes = 0.0;
    const size_t by_backlog = 1 + S->queue.size() / kBacklogPerExtra;
    const size_t limit = std::min(by_backlog, (size_t)S->max_events);
    while (!S->queue.empty() && batch.size() < limit) {
        const Pending &p = S->queue.front();
        const double v = S->accept_max * (double)p.triplets;
        if (!batch.empty() &&
            (hits + (int64_t)p.hits.size() > S->max_hits || votes + v > (double)S->vote_budget))
            break;
        hits += (int64_t)p.hits.size();
        votes += v;
        batch.push_back(std::move(S->queue.front()));
        S->queue.pop_front();
    }
}

// Packs the events `which` of `batch` into the lane's pinned staging buffers and queues
// their copy to the device on the lane's stream.  Needs no GPU lock: the copy overlaps the
// kernels of the lane that holds the GPU.
static int stage(trk_server *S, int lane, std::vector<Pending> &batch,
                 const std::vector<size_t> &which)
{
    trk_hit *sh = S->stage_hits[lane];
    int64_t *so = S->stage_offs[lane];
    cudaStream_t st = S->streams[lane];
    so[0] = 0;
    for (size_t e = 0; e < which.size(); ++e) {
        const size_t n = batch[which[e]].hits.size();
        if (n)
            std::memcpy(sh + so[e], batch[which[e]].hits.data(), n * sizeof(trk_hit));
        so[e + 1] = so[e] + (int64_t)n;
    }
    const int n_ev = (int32_t)which.size();
    if (cudaMemcpyAsync(S->d_hits[lane], sh, sizeof(trk_hit) * (size_t)so[n_ev],
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(S->d_offs[lane], so, sizeof(int64_t) * (size_t)(n_ev + 1),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
        return TRK_ERR_CUDA;
    return TRK_OK;
}

// Reconstructs the staged events (the caller holds the GPU); returns the call's code and
// outputs once the kernels are done; the results stay on the device.
static int compute(trk_server *S, int lane, int n_ev, trk_candidates &out)
{
    std::memset(&out, 0, sizeof(out));
    return trk_reconstruct(S->ctx[lane], S->d_hits[lane], S->stage_offs[lane][n_ev],
                           S->d_offs[lane], n_ev, &out, S->streams[lane]);
}

// Copies the results back, files every event and returns the events to run again alone
// (their vote list overflowed in a multi-event call).
static std::vector<size_t> deliver(trk_server *S, int lane, std::vector<Pending> &batch,
                                   const std::vector<size_t> &which, int rc,
                                   const trk_candidates &out)
{
    cudaStream_t st = S->streams[lane];
    const int64_t *so = S->stage_offs[lane];
    const int n_ev = (int32_t)which.size();
    const bool have = (rc == TRK_OK || rc == TRK_ERR_CAPACITY) && out.n_candidates > 0;
    if (have) {
        cudaMemcpyAsync(S->res_cand[lane], out.d_cand, sizeof(trk_candidate) * out.n_candidates,
                        cudaMemcpyDeviceToHost, st);
        if (out.n_hit_ids > 0)
            cudaMemcpyAsync(S->res_hits[lane], out.d_hit_ids, sizeof(int32_t) * out.n_hit_ids,
                            cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess)
            rc = TRK_ERR_CUDA;
    }
    const auto t_done = Clock::now();
    trk_stats stats;
    trk_get_stats(S->ctx[lane], &stats);
    std::vector<size_t> again;
    std::vector<Done> results(which.size());
    int64_t trip = 0;
    for (size_t e = 0; e < which.size(); ++e)
        trip += batch[which[e]].triplets;
    for (size_t e = 0; e < which.size(); ++e) {
        Done &d = results[e];
        const Pending &p = batch[which[e]];
        d.rc = rc;
        d.batch_events = n_ev;
        d.latency_s = std::chrono::duration<double>(t_done - p.t_submit).count();
        if (rc != TRK_OK && rc != TRK_ERR_CAPACITY) {
            d.status = -1;
            continue;
        }
        d.status = out.status[e];
        if ((d.status & TRK_EV_VOTE_OVERFLOW) && n_ev > 1) {
            again.push_back(which[e]);
            continue;
        }
        // the event's candidates and hit ids are contiguous (sorted by event)
        const int64_t c0 = out.cand_off[e], c1 = out.cand_off[e + 1];
        if (c1 > c0 && have) {
            const trk_candidate *cs = S->res_cand[lane];
            d.cand.assign(cs + c0, cs + c1);
            const int64_t h0 = d.cand.front().hit_off;
            const int64_t h1 = d.cand.back().hit_off + d.cand.back().n_hits;
            d.hits.assign(S->res_hits[lane] + h0, S->res_hits[lane] + h1);
            const int32_t base = (int32_t)so[e];
            for (int32_t &x : d.hits)
                x -= base;
            for (trk_candidate &r : d.cand) {
                r.hit_off -= h0;
                r.event = 0;
            }
        }
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (trip > 0 && stats.n_votes > 0 && rc == TRK_OK) {
            const double f = (double)stats.n_votes / (double)trip;
            if (f > S->accept_max)
                S->accept_max = f;
        }
        for (size_t e = 0; e < which.size(); ++e) {
            if (std::find(again.begin(), again.end(), which[e]) != again.end())
                continue;
            if (results[e].status != 0)
                S->n_failed++;
            S->done.emplace(batch[which[e]].ticket, std::move(results[e]));
            S->n_events_done++;
        }
        S->n_batches++;
    }
    S->cv_done.notify_all();
    return again;
}

static void lane_loop(trk_server *S, int lane)
{
    cudaSetDevice(S->device);
    std::vector<Pending> batch;
    for (;;) {
        batch.clear();
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
            if (S->stop && S->queue.empty())
                return;
        }
        std::vector<size_t> all;
        trk_candidates out;
        int rc;
        // a free lane forms its batch from what waits now and stages it while another
        // lane's batch computes; it then waits for the GPU and holds it until its kernels
        // are done
        {
            std::lock_guard<std::mutex> lk(S->mu);
            admit(S, batch);
        }
        if (batch.empty())
            continue;
        all.resize(batch.size());
        for (size_t e = 0; e < batch.size(); ++e)
            all[e] = e;
        rc = stage(S, lane, batch, all);
        if (rc == TRK_OK) {
            std::lock_guard<std::mutex> g(S->gpu_mu);
            rc = compute(S, lane, (int)all.size(), out);
        } else {
            std::memset(&out, 0, sizeof(out));
        }
        for (size_t e : deliver(S, lane, batch, all, rc, out)) {
            const std::vector<size_t> one{e};
            int rc1 = stage(S, lane, batch, one);
            if (rc1 == TRK_OK) {
                std::lock_guard<std::mutex> g(S->gpu_mu);
                rc1 = compute(S, lane, 1, out);
            }
            deliver(S, lane, batch, one, rc1, out);
        }
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
    for (trk_candidate *p : S->res_cand)
        if (p)
            cudaFreeHost(p);
    for (int32_t *p : S->res_hits)
        if (p)
            cudaFreeHost(p);
    for (trk_hit *p : S->d_hits)
        if (p)
            cudaFree(p);
    for (int64_t *p : S->d_offs)
        if (p)
            cudaFree(p);
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
    S->n_layers = geometry->n_layers;
    S->n_triples = geometry->n_triples;
    for (int t = 0; t < geometry->n_triples; ++t)
        for (int k = 0; k < 3; ++k)
            S->triples.push_back(geometry->triples[t][k]);
    trk_options lane = *lane_options;
    lane.fit_candidates = 0;            // served events return candidates and hits only
    if (lane.vote_capacity == 0) {
        // size each lane's vote list from the device memory free now: a lane without votes
        // (a probe handle) tells the fixed footprint, the rest is shared by the lanes' votes
        if (cudaSetDevice(lane.device) != cudaSuccess) {
            delete S;
            return TRK_ERR_CUDA;
        }
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            delete S;
            return TRK_ERR_CUDA;
        }
        trk_options probe = lane;
        probe.vote_capacity = 32;
        trk_ctx *ph = nullptr;
        int rc = trk_create(&ph, geometry, binning, &probe);
        if (rc != TRK_OK) {
            delete S;
            return rc;
        }
        size_t free_after = 0;
        cudaMemGetInfo(&free_after, &total_b);
        trk_destroy(ph);
        const double fixed = (double)(free_b > free_after ? free_b - free_after : 0);
        const double per_lane = 0.9 * (double)free_b / n_lanes - fixed;
        const int64_t votes = (int64_t)(per_lane / 8.75);   // 8 B per vote + 24 B per 32
        if (votes < 32) {
            delete S;
            return TRK_ERR_NOMEM;
        }
        lane.vote_capacity = votes;
    }
    S->vote_budget = lane.vote_capacity;
    for (int l = 0; l < n_lanes; ++l) {
        trk_ctx *h = nullptr;
        int rc = trk_create(&h, geometry, binning, &lane);
        if (rc != TRK_OK) {
            server_free(S);
            return rc;
        }
        S->ctx.push_back(h);
        // every batch size's graph, captured here, before any lane thread runs
        rc = trk::capture_call_graphs(h, S->max_events);
        if (rc != TRK_OK) {
            server_free(S);
            return rc;
        }
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
        trk_hit *dh = nullptr;
        int64_t *dof = nullptr;
        trk_candidate *rcand = nullptr;
        int32_t *rhits = nullptr;
        const bool ok =
            cudaMalloc((void **)&dh, sizeof(trk_hit) * (size_t)(S->max_hits > 0 ? S->max_hits : 1)) ==
                cudaSuccess &&
            cudaMalloc((void **)&dof, sizeof(int64_t) * ((size_t)S->max_events + 1)) == cudaSuccess &&
            cudaMallocHost((void **)&rcand, sizeof(trk_candidate) * (size_t)lane.cand_capacity) ==
                cudaSuccess &&
            cudaMallocHost((void **)&rhits, sizeof(int32_t) * (size_t)lane.assign_capacity) ==
                cudaSuccess;
        S->d_hits.push_back(dh);
        S->d_offs.push_back(dof);
        S->res_cand.push_back(rcand);
        S->res_hits.push_back(rhits);
        if (!ok) {
            server_free(S);
            return TRK_ERR_NOMEM;
        }
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
        // hit triplets of the event, for the admission bound on its votes
        std::vector<int64_t> per_layer((size_t)S->n_layers, 0);
        for (int64_t i = 0; i < n_hits; ++i)
            if (hits[i].layer >= 0 && hits[i].layer < S->n_layers)
                per_layer[(size_t)hits[i].layer]++;
        for (int t = 0; t < S->n_triples; ++t)
            p.triplets += per_layer[(size_t)S->triples[3 * t]] *
                          per_layer[(size_t)S->triples[3 * t + 1]] *
                          per_layer[(size_t)S->triples[3 * t + 2]];
    }
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
