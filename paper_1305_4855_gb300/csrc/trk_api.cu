// Host side of the C ABI declared in include/trk.h: validation, device pools (allocated
// once per handle), the launch sequence of one call, its CUDA-graph capture and the
// debug helpers.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "trk_common.cuh"

namespace trk {
cudaError_t launch_vote(const VoteArgs &A, int ti, int tj, int level, int grid, cudaStream_t s);
cudaError_t vote_occupancy(int ti, int tj, int level, int *blocks);
bool vote_tile_supported(int ti, int tj);
bool vote_level_supported(int level);
cudaError_t prepare_vote_kernel(int ti, int tj, int level);
cudaError_t prepare_pipeline_kernels();
cudaError_t launch_fit_triplets(const trk_hit *hits, int64_t n_hits, const int32_t *ijk,
                                int64_t n, const FitConst &C, float *params, uint32_t *bins,
                                int32_t *flags, cudaStream_t s);
cudaError_t launch_pack(const CallArgs *args, int n_events, int L, int max_per_event,
                        float4 *packed, int32_t *lay_off, int64_t *ev_begin, int32_t *status,
                        cudaStream_t s);
cudaError_t launch_schedule(const CallArgs *args, const DevGeo *geo, const int32_t *lay_off,
                            const int32_t *status, int ti, int tj, int64_t *item_off,
                            Counters *ctr, cudaStream_t s);
size_t peak_pass1_smem(const FitConst &C, int td);
cudaError_t launch_peaks(const int32_t *hist, int32_t *m3, const FitConst &C, int g0, int G,
                         int td, int threshold, const int32_t *status, uint32_t *cbits, int64_t W,
                         uint32_t *filter, unsigned long long *ties, unsigned long long *n_ties,
                         int64_t tie_cap, int n_sm, cudaStream_t s, bool vec_ok);
cudaError_t launch_peak_ties(const int32_t *hist, const FitConst &C,
                             const unsigned long long *ties, const unsigned long long *n_ties,
                             int64_t tie_cap, uint32_t *cbits, int64_t W, uint32_t *filter,
                             unsigned long long *overflow, int n_sm, cudaStream_t s);
cudaError_t launch_word_scan(const uint32_t *cbits, int64_t n_words, uint32_t *wprefix,
                             int64_t *bsum, unsigned long long *total, cudaStream_t s);
cudaError_t launch_cand_emit(const uint32_t *cbits, const uint32_t *wprefix, int64_t n_words,
                             int64_t W, const int32_t *hist, const FitConst &C,
                             trk_candidate *cand, int32_t *fill, int64_t cand_cap, Counters *ctr,
                             int n_sm, cudaStream_t s);
cudaError_t launch_vote_offsets(const trk_candidate *cand, const unsigned long long *n_cand,
                                int64_t cand_cap, int64_t *vote_off, int64_t *bsum,
                                unsigned long long *total, cudaStream_t s);
cudaError_t launch_assign(const AssignArgs &A, int n_events, int n_sm, cudaStream_t s);
cudaError_t launch_cand_fit(const trk_candidate *cand, const unsigned long long *n_cand,
                            int64_t cand_cap, const int32_t *hit_ids, int64_t hit_cap,
                            const CallArgs *args, double kB, int n_layers, trk_track *out,
                            uint8_t *hit_used, int32_t *order, int32_t *buckets, int n_sm,
                            cudaStream_t s);
cudaError_t prepare_fit_kernel();
cudaError_t launch_cand_hits(const trk_candidate *cand, const unsigned long long *n_cand,
                             int64_t cand_cap, const int64_t *vote_off, int32_t *assign,
                             int64_t assign_cap, const CallArgs *args, int32_t *nhits,
                             int max_words, int n_sm, cudaStream_t s);
cudaError_t launch_hit_offsets(const int32_t *nhits, const unsigned long long *n_cand,
                               int64_t cand_cap, int64_t *hit_off, int64_t *bsum,
                               unsigned long long *total, cudaStream_t s);
cudaError_t launch_compact(trk_candidate *cand, const unsigned long long *n_cand, int64_t cand_cap,
                           const int64_t *vote_off, const int32_t *assign, const int32_t *nhits,
                           const int64_t *hit_off, const int64_t *ev_begin, int32_t *hit_ids,
                           int n_sm, cudaStream_t s);
cudaError_t launch_finalize(const uint32_t *wprefix, int64_t W, const CallArgs *args,
                            Counters *ctr, int64_t cand_cap, int64_t *cand_off, int32_t *status,
                            cudaStream_t s);
cudaError_t launch_chunk_positions(const int32_t *chunk_count, int64_t n_chunks, int64_t *pos,
                                   int64_t *bsum, unsigned long long *total, cudaStream_t s);
cudaError_t launch_decode_votes(const AssignArgs &A, const int64_t *chunk_pos, int64_t n_chunks,
                                int32_t *dst, uint32_t *bins, int64_t cap, int n_sm,
                                cudaStream_t s);

}  // namespace trk

using namespace trk;

static std::string g_create_error;

namespace trk {
// Message for trk_last_error(NULL), from handle-free entry points.
void set_global_error(const std::string &msg) { g_create_error = msg; }
}  // namespace trk

struct trk_ctx {
    int device = 0;
    int n_sm = 0;
    trk_geometry geo;
    trk_binning bin;
    trk_options opt;
    FitConst C;
    int64_t nbins = 0, W = 0;
    int td = 0, group = 1, vote_grid = 0, max_words = 0, level = 3;
    int64_t chunk_cap = 0, bsum_cap = 0, tie_cap = 0;

    DevGeo *d_geo = nullptr;
    CallArgs *d_args = nullptr;
    Counters *d_ctr = nullptr;
    float4 *d_packed = nullptr;
    int32_t *d_lay_off = nullptr;
    int64_t *d_ev_begin = nullptr;
    int32_t *d_status = nullptr;
    int64_t *d_item_off = nullptr;
    int32_t *d_hist = nullptr;
    uint32_t *d_vote_bin = nullptr;    // vote list: bins and codes of the same slots
    uint32_t *d_vote_code = nullptr;
    int32_t *d_chunk_item = nullptr;
    int32_t *d_chunk_count = nullptr;
    int32_t *d_chunk_event = nullptr;
    int4 *d_chunk_loc = nullptr;
    int32_t *d_m3 = nullptr;
    unsigned long long *d_ties = nullptr;
    uint32_t *d_cbits = nullptr;
    uint32_t *d_filter = nullptr;        // candidate filters (kFilterWords per event)
    uint32_t *d_wprefix = nullptr;
    int64_t *d_bsum = nullptr;
    trk_candidate *d_cand = nullptr;
    int32_t *d_fill = nullptr;
    int64_t *d_vote_off = nullptr;
    int32_t *d_assign = nullptr;
    int32_t *d_nhits = nullptr;
    int64_t *d_hit_off = nullptr;
    int32_t *d_hit_ids = nullptr;
    trk_track *d_tracks = nullptr;       // candidate fits (fit_candidates)
    uint8_t *d_hit_used = nullptr;       // per hit id: kept by the fit
    int32_t *d_fit_order = nullptr;      // candidates grouped by hit count
    int32_t *d_fit_buckets = nullptr;
    int64_t *d_cand_off = nullptr;
    trk_hit *d_in_hits = nullptr;
    int64_t *d_in_offsets = nullptr;
    int64_t *d_chunk_pos = nullptr;

    CallArgs *h_args = nullptr;
    Counters *h_ctr = nullptr;
    int64_t *h_cand_off = nullptr;
    int32_t *h_status = nullptr;
    trk_candidate *h_cand = nullptr;
    int32_t *h_hit_ids = nullptr;
    trk_track *h_tracks = nullptr;
    uint8_t *h_hit_used = nullptr;

    std::map<int, cudaGraphExec_t> graphs;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t ev_st[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // stage boundaries
    cudaStream_t own_stream = nullptr;   // used when the caller passes the legacy stream
    std::vector<cudaEvent_t> pending;    // recorded after asynchronous work on caller streams
    trk_stats stats;
    int last_n_events = 0;
    std::string err;
};

// Persistent vote blocks: blocks_per_sm if given, else what the occupancy calculator
// allows for the instantiation (at least one per SM).
static int vote_grid_for(int n_sm, int ti, int tj, int level, int blocks_per_sm)
{
    int bps = blocks_per_sm;
    if (bps <= 0) {
        int occ = 0;
        if (vote_occupancy(ti, tj, level, &occ) != cudaSuccess || occ < 1)
            occ = 1;
        bps = occ;
    }
    return n_sm * bps;
}

static int fail(trk_ctx *h, int code, const std::string &msg)
{
    if (h)
        h->err = msg;
    else
        g_create_error = msg;
    return code;
}

#define TRK_CUDA(h, call)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(h, TRK_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)

extern "C" void trk_options_default(trk_options *o, int32_t max_events, int64_t max_hits)
{
    std::memset(o, 0, sizeof(*o));
    o->device = 0;
    o->max_events = max_events > 0 ? max_events : 1;
    o->max_hits = max_hits > 0 ? max_hits : 1;
    o->max_hits_per_event = 1 << 16;
    o->vote_capacity = (int64_t)1 << 27;
    o->cand_capacity = (int64_t)1 << 22;
    o->assign_capacity = (int64_t)1 << 26;
    o->peak_scratch_bytes = (int64_t)1 << 30;
    o->tile_i = 16;
    o->tile_j = 16;
    o->k_chunk = 2048;
    o->blocks_per_sm = 0;
    o->use_graph = 1;
    o->vote_level = 0;
}

extern "C" const char *trk_version(void) { return "trk 0.1 (sm_103a)"; }

extern "C" const char *trk_last_error(const trk_ctx *h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

static int validate(const trk_geometry *g, const trk_binning *b, const trk_options *o,
                    std::string &why)
{
    char buf[256];
    if (g->n_layers < 3 || g->n_layers > TRK_MAX_LAYERS) {
        why = "n_layers out of [3, TRK_MAX_LAYERS]";
        return 0;
    }
    if (g->n_triples < 1 || g->n_triples > TRK_MAX_TRIPLES) {
        why = "n_triples out of [1, TRK_MAX_TRIPLES]";
        return 0;
    }
    if (!(g->b_tesla > 0.0) || !std::isfinite(g->b_tesla)) {
        why = "b_tesla must be positive";
        return 0;
    }
    for (int t = 0; t < g->n_triples; ++t) {
        const int *x = g->triples[t];
        for (int k = 0; k < 3; ++k)
            if (x[k] < 0 || x[k] >= g->n_layers) {
                snprintf(buf, sizeof buf, "triple %d: layer id out of range", t);
                why = buf;
                return 0;
            }
        if (x[0] == x[1] || x[1] == x[2] || x[0] == x[2]) {
            snprintf(buf, sizeof buf, "triple %d: layers must be distinct", t);
            why = buf;
            return 0;
        }
    }
    double nb = 1.0;
    for (int k = 0; k < 5; ++k) {
        if (!(b->lo[k] < b->hi[k]) || !std::isfinite(b->lo[k]) || !std::isfinite(b->hi[k]) ||
            b->n[k] < 1) {
            snprintf(buf, sizeof buf, "binning dimension %d invalid", k);
            why = buf;
            return 0;
        }
        nb *= b->n[k];
    }
    if (nb >= 4294967295.0) {
        why = "number of bins must be below 2^32";
        return 0;
    }
    if (b->periodic & ~1) {
        why = "only dimension 0 (phi0) may be periodic";
        return 0;
    }
    if ((b->periodic & 1) && std::fabs((b->hi[0] - b->lo[0]) - 2.0 * M_PI) > 1e-6) {
        why = "a periodic phi0 range must span 2 pi";
        return 0;
    }
    if (b->threshold < 1) {
        why = "threshold must be >= 1";
        return 0;
    }
    if (!(b->sagitta_fp64_cm >= 0.0f)) {
        why = "sagitta_fp64_cm must be >= 0";
        return 0;
    }
    if ((double)b->n[3] * (b->n[4] + 1) * 8.0 * 3.0 > 200.0 * 1024.0) {
        why = "n[3] * (n[4] + 1) too large for the peak filter tile (must be <= 8533)";
        return 0;
    }
    if (o->max_events < 1 || o->max_hits < 1 || o->max_hits > ((int64_t)1 << 31) - 1) {
        why = "max_events / max_hits out of range";
        return 0;
    }
    if (o->max_hits_per_event < 1 || o->max_hits_per_event > (1 << 20)) {
        why = "max_hits_per_event out of [1, 2^20]";
        return 0;
    }
    if (o->vote_capacity < 32 || o->cand_capacity < 1 || o->assign_capacity < 3) {
        why = "capacities too small";
        return 0;
    }
    if (!vote_tile_supported(o->tile_i, o->tile_j)) {
        why = "unsupported tile_i x tile_j";
        return 0;
    }
    if (o->vote_level != 0 && !vote_level_supported(o->vote_level)) {
        why = "vote_level must be 0 (default), 2, 3 or 4";
        return 0;
    }
    return 1;
}

static void free_all(trk_ctx *h)
{
    void *dev[] = {h->d_geo,       h->d_args,       h->d_ctr,         h->d_packed,   h->d_lay_off,
                   h->d_ev_begin,  h->d_status,     h->d_item_off,    h->d_hist,     h->d_vote_bin, h->d_vote_code,
                   h->d_chunk_item, h->d_chunk_count, h->d_chunk_event, h->d_chunk_loc,
                   h->d_m3,        h->d_ties,
                   h->d_cbits,     h->d_filter,     h->d_wprefix,
                   h->d_bsum,      h->d_cand,       h->d_fill,        h->d_vote_off, h->d_assign,
                   h->d_nhits,     h->d_hit_off,    h->d_hit_ids,     h->d_cand_off, h->d_in_hits,
                   h->d_tracks,    h->d_hit_used,   h->d_fit_order,   h->d_fit_buckets,
                   h->d_in_offsets, h->d_chunk_pos};
    for (void *p : dev)
        if (p)
            cudaFree(p);
    void *host[] = {h->h_args,  h->h_ctr,     h->h_cand_off, h->h_status,
                    h->h_cand,  h->h_hit_ids, h->h_tracks,   h->h_hit_used};
    for (void *p : host)
        if (p)
            cudaFreeHost(p);
    for (auto &kv : h->graphs)
        cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    if (h->ev0)
        cudaEventDestroy(h->ev0);
    if (h->ev1)
        cudaEventDestroy(h->ev1);
    if (h->own_stream)
        cudaStreamDestroy(h->own_stream);
    for (cudaEvent_t &e : h->ev_st)
        if (e)
            cudaEventDestroy(e);
    for (cudaEvent_t e : h->pending)
        cudaEventDestroy(e);
    h->pending.clear();
}

// Marks the end of asynchronous work the handle enqueued on a caller's stream, so that
// trk_destroy can wait for exactly that work (events of finished work are reused).
static cudaError_t note_async(trk_ctx *h, cudaStream_t s)
{
    cudaEvent_t ev = nullptr;
    for (size_t i = 0; i < h->pending.size(); ++i)
        if (cudaEventQuery(h->pending[i]) == cudaSuccess) {
            ev = h->pending[i];
            h->pending.erase(h->pending.begin() + (long)i);
            break;
        }
    if (!ev) {
        const cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess)
            return e;
    }
    h->pending.push_back(ev);
    return cudaEventRecord(ev, s);
}

template <class T>
static cudaError_t dalloc(T **p, size_t count)
{
    return cudaMalloc((void **)p, sizeof(T) * (count > 0 ? count : 1));
}

extern "C" int trk_create(trk_ctx **out, const trk_geometry *geometry, const trk_binning *binning,
                          const trk_options *options)
{
    if (!out || !geometry || !binning)
        return fail(nullptr, TRK_ERR_INVALID, "null argument");
    *out = nullptr;
    trk_options o;
    if (options)
        o = *options;
    else
        trk_options_default(&o, 1, 1 << 20);
    std::string why;
    if (!validate(geometry, binning, &o, why))
        return fail(nullptr, TRK_ERR_INVALID, why);
    trk_ctx *h = new trk_ctx();
    h->geo = *geometry;
    h->bin = *binning;
    h->opt = o;
    h->device = o.device;
    std::memset(&h->stats, 0, sizeof(h->stats));
    cudaError_t e = cudaSetDevice(o.device);
    if (e != cudaSuccess) {
        delete h;
        return fail(nullptr, TRK_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    }
    cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, o.device);

    // fit and binning constants
    FitConst &C = h->C;
    std::memset(&C, 0, sizeof(C));
    const double kB = kGeVPerTeslaCm * geometry->b_tesla;
    C.kB = (float)kB;
    C.inv_kB = (float)(1.0 / kB);
    C.kB_d = kB;
    const double qmax = std::fmax(std::fabs(binning->lo[1]), std::fabs(binning->hi[1]));
    // 4 D^2 <= (kB qmax)^2 |u|^2|v|^2|w|^2, with a 1e-3 relative margin so that the
    // prefilter is a superset of the FP32 range test made later on the same inputs
    C.pre_k2 = (float)(0.25 * (kB * qmax) * (kB * qmax) * (1.0 + 1e-3));
    C.sag2 = binning->sagitta_fp64_cm * binning->sagitta_fp64_cm;
    C.periodic = binning->periodic;
    uint32_t stride = 1;
    for (int k = 4; k >= 0; --k) {
        C.stride[k] = stride;
        stride *= (uint32_t)binning->n[k];
    }
    h->nbins = (int64_t)C.stride[0] * binning->n[0];
    C.nbins = (uint32_t)h->nbins;
    for (int k = 0; k < 5; ++k) {
        C.lo[k] = (float)binning->lo[k];
        C.hi[k] = (float)binning->hi[k];
        C.inv_w[k] = (float)(binning->n[k] / (binning->hi[k] - binning->lo[k]));
        C.n[k] = binning->n[k];
        C.lo_d[k] = binning->lo[k];
        C.hi_d[k] = binning->hi[k];
        C.w_d[k] = (binning->hi[k] - binning->lo[k]) / binning->n[k];
    }
    C.period0 = C.hi[0] - C.lo[0];
    h->W = (h->nbins + 31) / 32;
    // peak filter: rows per slab and events per group
    // rows of a peak-filter slab: small enough for 4 resident blocks per SM (halo rows cost
    // 2/td extra loads)
    int td = binning->n[2];
    while (td > 1 && peak_pass1_smem(C, td) > 48 * 1024)
        --td;
    if (peak_pass1_smem(C, td) > 100 * 1024) {
        delete h;
        return fail(nullptr, TRK_ERR_INVALID, "n[3] * (n[4] + 1) too large for the filter tile");
    }
    h->td = td;
    int64_t g = o.peak_scratch_bytes / (h->nbins * 4);
    g = g < 1 ? 1 : (g > o.max_events ? o.max_events : g);
    h->group = (int)g;
    h->max_words = (o.max_hits_per_event + 31) / 32;
    // bins listed for the tie test: at least the candidates; a flat region above threshold
    // lists every bin of it
    h->tie_cap = 2 * o.cand_capacity > ((int64_t)1 << 20) ? 2 * o.cand_capacity : ((int64_t)1 << 20);
    h->chunk_cap = (o.vote_capacity + 31) / 32;
    int64_t caps[] = {o.cand_capacity, (int64_t)o.max_events * h->W, h->chunk_cap};
    int64_t mc = 0;
    for (int64_t c : caps)
        mc = c > mc ? c : mc;
    h->bsum_cap = (mc + 4095) / 4096 + 1;

    h->level = o.vote_level ? o.vote_level : 3;
    if (prepare_vote_kernel(o.tile_i, o.tile_j, h->level) != cudaSuccess) {
        delete h;
        return fail(nullptr, TRK_ERR_CUDA, "vote kernel attributes");
    }
    h->vote_grid = vote_grid_for(h->n_sm, o.tile_i, o.tile_j, h->level, o.blocks_per_sm);

    DevGeo dg;
    std::memset(&dg, 0, sizeof(dg));
    dg.n_layers = geometry->n_layers;
    dg.n_triples = geometry->n_triples;
    std::memcpy(dg.triples, geometry->triples, sizeof(dg.triples));

    const int L1 = geometry->n_layers + 1;
    const int64_t E = o.max_events;
#define ALLOC(ptr, n)                                                                          \
    do {                                                                                       \
        cudaError_t a_ = dalloc(&h->ptr, (size_t)(n));                                         \
        if (a_ != cudaSuccess) {                                                               \
            free_all(h);                                                                       \
            delete h;                                                                          \
            return fail(nullptr, TRK_ERR_NOMEM, std::string("cudaMalloc " #ptr ": ") +         \
                                                    cudaGetErrorString(a_));                   \
        }                                                                                      \
    } while (0)
    ALLOC(d_geo, 1);
    ALLOC(d_args, 1);
    ALLOC(d_ctr, 1);
    ALLOC(d_packed, o.max_hits);
    ALLOC(d_lay_off, E * L1);
    ALLOC(d_ev_begin, E + 1);
    ALLOC(d_status, E);
    ALLOC(d_item_off, E * geometry->n_triples + 1);
    ALLOC(d_hist, E * h->nbins);
    ALLOC(d_vote_bin, h->chunk_cap * 32);
    ALLOC(d_vote_code, h->chunk_cap * 32);
    ALLOC(d_chunk_item, h->chunk_cap);
    ALLOC(d_chunk_count, h->chunk_cap);
    ALLOC(d_chunk_event, h->chunk_cap);
    ALLOC(d_chunk_loc, h->chunk_cap);
    ALLOC(d_m3, (int64_t)h->group * h->nbins);
    ALLOC(d_ties, h->tie_cap);
    ALLOC(d_cbits, E * h->W);
    ALLOC(d_filter, (int64_t)kFilterWords * o.max_events);
    ALLOC(d_wprefix, E * h->W);
    ALLOC(d_bsum, h->bsum_cap);
    ALLOC(d_cand, o.cand_capacity);
    ALLOC(d_fill, o.cand_capacity);
    ALLOC(d_vote_off, o.cand_capacity);
    ALLOC(d_assign, o.assign_capacity);
    ALLOC(d_nhits, o.cand_capacity);
    ALLOC(d_hit_off, o.cand_capacity);
    ALLOC(d_hit_ids, o.assign_capacity);
    if (o.fit_candidates) {
        ALLOC(d_tracks, o.cand_capacity);
        ALLOC(d_hit_used, o.assign_capacity);
        ALLOC(d_fit_order, o.cand_capacity);
        ALLOC(d_fit_buckets, 1024);
    }
    ALLOC(d_cand_off, E + 1);
#undef ALLOC
    if (cudaMallocHost((void **)&h->h_args, sizeof(CallArgs)) != cudaSuccess ||
        cudaMallocHost((void **)&h->h_ctr, sizeof(Counters)) != cudaSuccess ||
        cudaMallocHost((void **)&h->h_cand_off, sizeof(int64_t) * (E + 1)) != cudaSuccess ||
        cudaMallocHost((void **)&h->h_status, sizeof(int32_t) * E) != cudaSuccess) {
        free_all(h);
        delete h;
        return fail(nullptr, TRK_ERR_NOMEM, "cudaMallocHost failed");
    }
    std::memset(h->h_ctr, 0, sizeof(Counters));
    // initialisation on the handle's own non-blocking stream, synchronised on that stream
    // only: a device-wide synchronisation would be invalid while another thread captures
    cudaError_t ie = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
    cudaStream_t is = h->own_stream;
    const cudaError_t init[] = {
        ie,
        cudaMemcpyAsync(h->d_geo, &dg, sizeof(dg), cudaMemcpyHostToDevice, is),
        cudaEventCreate(&h->ev0), cudaEventCreate(&h->ev1),
        cudaEventCreate(&h->ev_st[0]), cudaEventCreate(&h->ev_st[1]),
        cudaEventCreate(&h->ev_st[2]), cudaEventCreate(&h->ev_st[3]),
        cudaEventCreate(&h->ev_st[4]),
        prepare_pipeline_kernels(), prepare_fit_kernel(),
        cudaMemsetAsync(h->d_hist, 0, sizeof(int32_t) * (size_t)(E * h->nbins), is),
        cudaMemsetAsync(h->d_chunk_item, 0xff, sizeof(int32_t) * (size_t)h->chunk_cap, is),
        cudaMemsetAsync(h->d_chunk_count, 0, sizeof(int32_t) * (size_t)h->chunk_cap, is),
        cudaStreamSynchronize(is)};
    for (cudaError_t r : init) {
        if (r != cudaSuccess) {
            free_all(h);
            delete h;
            return fail(nullptr, TRK_ERR_CUDA,
                        std::string("initialisation failed: ") + cudaGetErrorString(r));
        }
    }
    *out = h;
    return TRK_OK;
}

extern "C" int trk_destroy(trk_ctx *h)
{
    if (!h)
        return TRK_OK;
    cudaSetDevice(h->device);
    // wait for the handle's own work only: its stream, and what its asynchronous entry
    // points left on callers' streams (a device-wide synchronisation would be invalid while
    // another thread of the process captures a graph, e.g. a server lane)
    if (h->own_stream)
        cudaStreamSynchronize(h->own_stream);
    for (cudaEvent_t e : h->pending)
        cudaEventSynchronize(e);
    free_all(h);
    delete h;
    return TRK_OK;
}

// Everything of one call after the argument copy, on stream s.
static int enqueue(trk_ctx *h, int n_events, cudaStream_t s, bool capturing)
{
    // inside a capture the stage events must become event-record nodes
    auto mark = [&](cudaEvent_t ev) {
        return capturing ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                         : cudaEventRecord(ev, s);
    };
    const trk_options &o = h->opt;
    const int L = h->geo.n_layers;
    const int64_t n_words = (int64_t)n_events * h->W;
    Counters *ctr = h->d_ctr;
    TRK_CUDA(h, cudaMemsetAsync(ctr, 0, sizeof(Counters), s));
    TRK_CUDA(h, cudaMemsetAsync(h->d_hist, 0, sizeof(int32_t) * (size_t)n_events * h->nbins, s));
    TRK_CUDA(h, launch_pack(h->d_args, n_events, L, o.max_hits_per_event, h->d_packed,
                            h->d_lay_off, h->d_ev_begin, h->d_status, s));
    TRK_CUDA(h, launch_schedule(h->d_args, h->d_geo, h->d_lay_off, h->d_status, o.tile_i,
                                o.tile_j, h->d_item_off, ctr, s));
    VoteArgs va;
    va.packed = h->d_packed;
    va.lay_off = h->d_lay_off;
    va.item_off = h->d_item_off;
    va.geo = h->d_geo;
    va.args = h->d_args;
    va.status = h->d_status;
    va.hist = h->d_hist;
    va.vote_bin = h->d_vote_bin;
    va.vote_code = h->d_vote_code;
    va.chunk_item = h->d_chunk_item;
    va.chunk_count = h->d_chunk_count;
    va.chunk_event = h->d_chunk_event;
    va.chunk_loc = h->d_chunk_loc;
    va.chunk_cap = h->chunk_cap;
    va.ctr = ctr;
    va.C = h->C;
    TRK_CUDA(h, mark(h->ev_st[0]));
    TRK_CUDA(h, launch_vote(va, o.tile_i, o.tile_j, h->level, h->vote_grid, s));
    TRK_CUDA(h, mark(h->ev_st[1]));
    TRK_CUDA(h, cudaMemsetAsync(h->d_cbits, 0, sizeof(uint32_t) * (size_t)n_words, s));
    TRK_CUDA(h, cudaMemsetAsync(h->d_filter, 0, sizeof(uint32_t) * kFilterWords * n_events, s));
    for (int g0 = 0; g0 < n_events; g0 += h->group) {
        const int G = (n_events - g0) < h->group ? (n_events - g0) : h->group;
        TRK_CUDA(h, launch_peaks(h->d_hist, h->d_m3, h->C, g0, G, h->td, h->bin.threshold,
                                 h->d_status, h->d_cbits, h->W, h->d_filter, h->d_ties,
                                 &ctr->n_ties, h->tie_cap, h->n_sm, s, true));
    }
    // the plateau maxima the passes listed
    TRK_CUDA(h, launch_peak_ties(h->d_hist, h->C, h->d_ties, &ctr->n_ties, h->tie_cap, h->d_cbits,
                                 h->W, h->d_filter, &ctr->overflow, h->n_sm, s));
    TRK_CUDA(h, mark(h->ev_st[2]));
    TRK_CUDA(h, launch_word_scan(h->d_cbits, n_words, h->d_wprefix, h->d_bsum, &ctr->n_cand, s));
    TRK_CUDA(h, launch_cand_emit(h->d_cbits, h->d_wprefix, n_words, h->W, h->d_hist, h->C,
                                 h->d_cand, h->d_fill, o.cand_capacity, ctr, h->n_sm, s));
    TRK_CUDA(h, launch_vote_offsets(h->d_cand, &ctr->n_cand, o.cand_capacity, h->d_vote_off,
                                    h->d_bsum, &ctr->n_assign, s));
    TRK_CUDA(h, mark(h->ev_st[3]));
    AssignArgs aa;
    aa.vote_bin = h->d_vote_bin;
    aa.vote_code = h->d_vote_code;
    aa.chunk_item = h->d_chunk_item;
    aa.chunk_count = h->d_chunk_count;
    aa.chunk_event = h->d_chunk_event;
    aa.chunk_loc = h->d_chunk_loc;
    aa.chunk_cap = h->chunk_cap;
    aa.item_off = h->d_item_off;
    aa.geo = h->d_geo;
    aa.lay_off = h->d_lay_off;
    aa.args = h->d_args;
    aa.packed = h->d_packed;
    aa.ev_begin = h->d_ev_begin;
    aa.cbits = h->d_cbits;
    aa.filter = h->d_filter;
    aa.wprefix = h->d_wprefix;
    aa.W = h->W;
    aa.vote_off = h->d_vote_off;
    aa.fill = h->d_fill;
    aa.assign = h->d_assign;
    aa.assign_cap = o.assign_capacity;
    // the queue of candidate-vote slots borrows the hit-id buffer, written only later by the
    // compaction (a candidate vote fills three assignment entries, so the queue needs at most
    // assign_capacity / 3 slots of the assign_capacity / 2 that fit)
    aa.cqueue = reinterpret_cast<unsigned long long *>(h->d_hit_ids);
    aa.cqueue_cap = o.assign_capacity / 2;
    aa.cand_cap = o.cand_capacity;
    aa.ctr = ctr;
    aa.ti = o.tile_i;
    aa.tj = o.tile_j;
    TRK_CUDA(h, launch_assign(aa, n_events, h->n_sm, s));
    TRK_CUDA(h, launch_cand_hits(h->d_cand, &ctr->n_cand, o.cand_capacity, h->d_vote_off,
                                 h->d_assign, o.assign_capacity, h->d_args, h->d_nhits,
                                 h->max_words, h->n_sm, s));
    TRK_CUDA(h, launch_hit_offsets(h->d_nhits, &ctr->n_cand, o.cand_capacity, h->d_hit_off,
                                   h->d_bsum, &ctr->n_hit_ids, s));
    TRK_CUDA(h, launch_compact(h->d_cand, &ctr->n_cand, o.cand_capacity, h->d_vote_off,
                               h->d_assign, h->d_nhits, h->d_hit_off, h->d_ev_begin,
                               h->d_hit_ids, h->n_sm, s));
    TRK_CUDA(h, mark(h->ev_st[4]));
    if (o.fit_candidates)
        TRK_CUDA(h, launch_cand_fit(h->d_cand, &ctr->n_cand, o.cand_capacity, h->d_hit_ids,
                                    o.assign_capacity, h->d_args, h->C.kB_d, h->geo.n_layers,
                                    h->d_tracks, h->d_hit_used, h->d_fit_order,
                                    h->d_fit_buckets, h->n_sm, s));
    TRK_CUDA(h, launch_finalize(h->d_wprefix, h->W, h->d_args, ctr, o.cand_capacity,
                                h->d_cand_off, h->d_status, s));
    TRK_CUDA(h, cudaMemcpyAsync(h->h_ctr, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    TRK_CUDA(h, cudaMemcpyAsync(h->h_cand_off, h->d_cand_off, sizeof(int64_t) * (n_events + 1),
                                cudaMemcpyDeviceToHost, s));
    TRK_CUDA(h, cudaMemcpyAsync(h->h_status, h->d_status, sizeof(int32_t) * n_events,
                                cudaMemcpyDeviceToHost, s));
    return TRK_OK;
}

// The captured graph of one call shape (n_events), captured on stream s if not cached.
// Nothing runs during a capture: the graph reads its inputs through the device copy of
// CallArgs, so it serves every later call of that shape.
static int graph_for(trk_ctx *h, int n_events, cudaStream_t s, cudaGraphExec_t *out)
{
    auto it = h->graphs.find(n_events);
    if (it == h->graphs.end()) {
        cudaGraph_t graph;
        TRK_CUDA(h, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const int rc = enqueue(h, n_events, s, true);
        cudaError_t ec = cudaStreamEndCapture(s, &graph);
        if (rc != TRK_OK) {
            if (ec == cudaSuccess)
                cudaGraphDestroy(graph);
            return rc;
        }
        TRK_CUDA(h, ec);
        cudaGraphExec_t exec;
        cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        TRK_CUDA(h, ei);
        it = h->graphs.emplace(n_events, exec).first;
    }
    *out = it->second;
    return TRK_OK;
}

static int run_call(trk_ctx *h, int n_events, cudaStream_t s)
{
    TRK_CUDA(h, cudaMemcpyAsync(h->d_args, h->h_args, sizeof(CallArgs), cudaMemcpyHostToDevice, s));
    if (h->opt.use_graph) {
        cudaGraphExec_t exec = nullptr;
        const int rc = graph_for(h, n_events, s, &exec);
        if (rc != TRK_OK)
            return rc;
        TRK_CUDA(h, cudaGraphLaunch(exec, s));
        return TRK_OK;
    }
    return enqueue(h, n_events, s, false);
}

namespace trk {
// Captures the graphs of call shapes 1 .. max_events on the handle's own stream, so that
// later calls only launch them (the server does this before its lane threads start).
int capture_call_graphs(trk_ctx *h, int max_events)
{
    if (!h->opt.use_graph)
        return TRK_OK;
    TRK_CUDA(h, cudaSetDevice(h->device));
    for (int n = 1; n <= max_events && n <= h->opt.max_events; ++n) {
        cudaGraphExec_t exec = nullptr;
        const int rc = graph_for(h, n, h->own_stream, &exec);
        if (rc != TRK_OK)
            return rc;
    }
    return TRK_OK;
}

// Device bytes one event needs at most for a given vote count: its histogram, candidate
// bitmap and prefix, and the vote list (bin, code and chunk record per 32 votes).
int64_t event_device_bytes(const trk_ctx *h, int64_t votes)
{
    return 4 * h->nbins + 8 * h->W + votes * 8 + (votes / 32 + 1) * 24;
}
}  // namespace trk

static int finish_call(trk_ctx *h, int n_events, trk_candidates *out, cudaStream_t s)
{
    TRK_CUDA(h, cudaEventRecord(h->ev1, s));
    TRK_CUDA(h, cudaStreamSynchronize(s));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    const Counters &c = *h->h_ctr;
    const bool over = c.overflow != 0 || c.n_cand > (unsigned long long)h->opt.cand_capacity;
    trk_stats &st = h->stats;
    st.n_triplets = (int64_t)c.n_triplets;
    st.n_fit = (int64_t)c.n_fit;
    st.n_exact = (int64_t)c.n_exact;
    st.n_votes = (int64_t)c.n_votes;
    st.n_fp64 = (int64_t)c.n_fp64;
    st.n_candidates = over ? 0 : (int64_t)c.n_cand;
    st.n_hit_ids = over ? 0 : (int64_t)c.n_hit_ids;
    st.n_work_items = (int64_t)c.n_items;
    st.ms_total = ms;
    st.n_plateau = (int64_t)c.n_ties;
    st.n_cand_votes = (int64_t)c.n_cvotes;
    h->last_n_events = n_events;
    int any = 0;
    for (int e = 0; e < n_events; ++e)
        any |= h->h_status[e];
    if (out) {
        out->n_events = n_events;
        out->n_candidates = st.n_candidates;
        out->n_hit_ids = st.n_hit_ids;
        out->cand_off = h->h_cand_off;
        out->status = h->h_status;
        out->d_cand = h->d_cand;
        out->d_hit_ids = h->d_hit_ids;
        out->h_cand = nullptr;
        out->h_hit_ids = nullptr;
        out->d_tracks = h->d_tracks;
        out->d_hit_used = h->d_hit_used;
        out->h_tracks = nullptr;
        out->h_hit_used = nullptr;
    }
    if (over)
        return fail(h, TRK_ERR_CAPACITY, "candidate or assignment capacity exceeded");
    if (any & (TRK_EV_TOO_MANY_HITS | TRK_EV_VOTE_OVERFLOW | TRK_EV_CAND_OVERFLOW))
        return fail(h, TRK_ERR_CAPACITY, "some event exceeded a capacity (see status)");
    return TRK_OK;
}

static int check_call(trk_ctx *h, const void *hits, int64_t n_hits, const void *offsets,
                      int32_t n_events)
{
    if (!h)
        return TRK_ERR_INVALID;
    if (n_events < 1 || n_events > h->opt.max_events)
        return fail(h, TRK_ERR_INVALID, "n_events out of [1, max_events]");
    if (n_hits < 0 || n_hits > h->opt.max_hits)
        return fail(h, TRK_ERR_INVALID, "n_hits out of [0, max_hits]");
    if (!offsets || (n_hits > 0 && !hits))
        return fail(h, TRK_ERR_INVALID, "null hits or offsets");
    return TRK_OK;
}

extern "C" int trk_reconstruct(trk_ctx *h, const trk_hit *hits, int64_t n_hits,
                               const int64_t *event_offsets, int32_t n_events,
                               trk_candidates *out, void *stream)
{
    int rc = check_call(h, hits, n_hits, event_offsets, n_events);
    if (rc != TRK_OK)
        return rc;
    cudaStream_t s = stream ? (cudaStream_t)stream : h->own_stream;
    TRK_CUDA(h, cudaSetDevice(h->device));
    h->h_args->hits = hits;
    h->h_args->offsets = event_offsets;
    h->h_args->n_hits = n_hits;
    h->h_args->n_events = n_events;
    TRK_CUDA(h, cudaEventRecord(h->ev0, s));
    rc = run_call(h, n_events, s);
    if (rc != TRK_OK)
        return rc;
    return finish_call(h, n_events, out, s);
}

extern "C" int trk_reconstruct_host(trk_ctx *h, const trk_hit *hits, int64_t n_hits,
                                    const int64_t *event_offsets, int32_t n_events,
                                    trk_candidates *out, void *stream)
{
    int rc = check_call(h, hits, n_hits, event_offsets, n_events);
    if (rc != TRK_OK)
        return rc;
    cudaStream_t s = stream ? (cudaStream_t)stream : h->own_stream;
    TRK_CUDA(h, cudaSetDevice(h->device));
    if (!h->d_in_hits) {
        if (dalloc(&h->d_in_hits, (size_t)h->opt.max_hits) != cudaSuccess ||
            dalloc(&h->d_in_offsets, (size_t)h->opt.max_events + 1) != cudaSuccess)
            return fail(h, TRK_ERR_NOMEM, "input staging allocation failed");
    }
    if (!h->h_cand) {
        if (cudaMallocHost((void **)&h->h_cand, sizeof(trk_candidate) * h->opt.cand_capacity) !=
                cudaSuccess ||
            cudaMallocHost((void **)&h->h_hit_ids, sizeof(int32_t) * h->opt.assign_capacity) !=
                cudaSuccess)
            return fail(h, TRK_ERR_NOMEM, "pinned result allocation failed");
        if (h->opt.fit_candidates &&
            (cudaMallocHost((void **)&h->h_tracks, sizeof(trk_track) * h->opt.cand_capacity) !=
                 cudaSuccess ||
             cudaMallocHost((void **)&h->h_hit_used, (size_t)h->opt.assign_capacity) != cudaSuccess))
            return fail(h, TRK_ERR_NOMEM, "pinned result allocation failed");
    }
    TRK_CUDA(h, cudaEventRecord(h->ev0, s));
    if (n_hits > 0)
        TRK_CUDA(h, cudaMemcpyAsync(h->d_in_hits, hits, sizeof(trk_hit) * n_hits,
                                    cudaMemcpyHostToDevice, s));
    TRK_CUDA(h, cudaMemcpyAsync(h->d_in_offsets, event_offsets, sizeof(int64_t) * (n_events + 1),
                                cudaMemcpyHostToDevice, s));
    h->h_args->hits = h->d_in_hits;
    h->h_args->offsets = h->d_in_offsets;
    h->h_args->n_hits = n_hits;
    h->h_args->n_events = n_events;
    rc = run_call(h, n_events, s);
    if (rc != TRK_OK)
        return rc;
    // the counts decide the sizes of the result copies: wait for them, then copy
    TRK_CUDA(h, cudaStreamSynchronize(s));
    const Counters &c = *h->h_ctr;
    const bool over = c.overflow != 0 || c.n_cand > (unsigned long long)h->opt.cand_capacity;
    if (!over) {
        if (c.n_cand > 0)
            TRK_CUDA(h, cudaMemcpyAsync(h->h_cand, h->d_cand, sizeof(trk_candidate) * c.n_cand,
                                        cudaMemcpyDeviceToHost, s));
        if (c.n_hit_ids > 0)
            TRK_CUDA(h, cudaMemcpyAsync(h->h_hit_ids, h->d_hit_ids, sizeof(int32_t) * c.n_hit_ids,
                                        cudaMemcpyDeviceToHost, s));
        if (h->opt.fit_candidates && c.n_cand > 0)
            TRK_CUDA(h, cudaMemcpyAsync(h->h_tracks, h->d_tracks, sizeof(trk_track) * c.n_cand,
                                        cudaMemcpyDeviceToHost, s));
        if (h->opt.fit_candidates && c.n_hit_ids > 0)
            TRK_CUDA(h, cudaMemcpyAsync(h->h_hit_used, h->d_hit_used, (size_t)c.n_hit_ids,
                                        cudaMemcpyDeviceToHost, s));
    }
    rc = finish_call(h, n_events, out, s);
    if (out) {
        out->h_cand = h->h_cand;
        out->h_hit_ids = h->h_hit_ids;
        out->h_tracks = h->h_tracks;
        out->h_hit_used = h->h_hit_used;
    }
    return rc;
}

extern "C" int trk_get_stats(trk_ctx *h, trk_stats *out)
{
    if (!h || !out)
        return TRK_ERR_INVALID;
    *out = h->stats;
    return TRK_OK;
}

extern "C" int64_t trk_histogram_size(const trk_ctx *h) { return h ? h->nbins : 0; }

extern "C" int trk_get_histogram(trk_ctx *h, int32_t event, int32_t *dst, void *stream)
{
    if (!h || !dst)
        return TRK_ERR_INVALID;
    if (event < 0 || event >= h->last_n_events)
        return fail(h, TRK_ERR_INVALID, "event out of range of the last call");
    TRK_CUDA(h, cudaSetDevice(h->device));
    TRK_CUDA(h, cudaMemcpyAsync(dst, h->d_hist + (size_t)event * h->nbins,
                                sizeof(int32_t) * (size_t)h->nbins, cudaMemcpyDeviceToDevice,
                                (cudaStream_t)stream));
    TRK_CUDA(h, note_async(h, (cudaStream_t)stream));
    return TRK_OK;
}

extern "C" int trk_get_votes(trk_ctx *h, int32_t *dst, uint32_t *bins, int64_t cap,
                             int64_t *n_out, void *stream)
{
    if (!h || !n_out || (cap > 0 && (!dst || !bins)))
        return TRK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    TRK_CUDA(h, cudaSetDevice(h->device));
    int64_t n_chunks = (int64_t)h->h_ctr->n_chunks;
    n_chunks = n_chunks < h->chunk_cap ? n_chunks : h->chunk_cap;
    if (!h->d_chunk_pos && dalloc(&h->d_chunk_pos, (size_t)h->chunk_cap) != cudaSuccess)
        return fail(h, TRK_ERR_NOMEM, "chunk position allocation failed");
    if (n_chunks == 0) {
        *n_out = 0;
        return TRK_OK;
    }
    TRK_CUDA(h, launch_chunk_positions(h->d_chunk_count, n_chunks, h->d_chunk_pos, h->d_bsum,
                                       &h->d_ctr->pad[0], s));
    AssignArgs aa;
    std::memset(&aa, 0, sizeof(aa));
    aa.vote_bin = h->d_vote_bin;
    aa.vote_code = h->d_vote_code;
    aa.chunk_item = h->d_chunk_item;
    aa.chunk_count = h->d_chunk_count;
    aa.chunk_cap = h->chunk_cap;
    aa.item_off = h->d_item_off;
    aa.geo = h->d_geo;
    aa.lay_off = h->d_lay_off;
    aa.args = h->d_args;
    aa.packed = h->d_packed;
    aa.ti = h->opt.tile_i;
    aa.tj = h->opt.tile_j;
    if (cap > 0)
        TRK_CUDA(h, launch_decode_votes(aa, h->d_chunk_pos, n_chunks, dst, bins, cap, h->n_sm, s));
    unsigned long long total = 0;
    TRK_CUDA(h, cudaMemcpyAsync(&total, &h->d_ctr->pad[0], sizeof(total), cudaMemcpyDeviceToHost, s));
    TRK_CUDA(h, cudaStreamSynchronize(s));
    *n_out = (int64_t)total;
    return TRK_OK;
}

extern "C" int trk_fit_triplets(trk_ctx *h, const trk_hit *hits, int64_t n_hits,
                                const int32_t *ijk, int64_t n, float *params, uint32_t *bins,
                                int32_t *flags, void *stream)
{
    if (!h || n < 0 || n_hits < 0 || (n > 0 && (!hits || !ijk || !params || !bins || !flags)))
        return TRK_ERR_INVALID;
    TRK_CUDA(h, cudaSetDevice(h->device));
    TRK_CUDA(h, launch_fit_triplets(hits, n_hits, ijk, n, h->C, params, bins, flags,
                                    (cudaStream_t)stream));
    TRK_CUDA(h, note_async(h, (cudaStream_t)stream));
    return TRK_OK;
}

extern "C" int trk_profile_stages(trk_ctx *h, float ms[8], void *stream)
{
    if (!h || !ms)
        return TRK_ERR_INVALID;
    TRK_CUDA(h, cudaSetDevice(h->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : h->own_stream;
    TRK_CUDA(h, cudaStreamSynchronize(s));
    for (int i = 0; i < 8; ++i)
        ms[i] = 0.0f;
    TRK_CUDA(h, cudaEventElapsedTime(&ms[0], h->ev_st[0], h->ev_st[1]));
    TRK_CUDA(h, cudaEventElapsedTime(&ms[1], h->ev0, h->ev_st[0]));
    TRK_CUDA(h, cudaEventElapsedTime(&ms[2], h->ev_st[1], h->ev_st[2]));
    TRK_CUDA(h, cudaEventElapsedTime(&ms[3], h->ev_st[2], h->ev_st[3]));
    TRK_CUDA(h, cudaEventElapsedTime(&ms[4], h->ev_st[3], h->ev_st[4]));
    TRK_CUDA(h, cudaEventElapsedTime(&ms[5], h->ev_st[4], h->ev1));
    return TRK_OK;
}

extern "C" int trk_autotune(trk_ctx *h, const trk_hit *hits, int64_t n_hits,
                            const int64_t *event_offsets, int32_t n_events, int32_t reps,
                            trk_tuning *best, void *stream)
{
    if (!h || !best || reps < 1)
        return TRK_ERR_INVALID;
    static const int tiles[][2] = {{16, 16}, {8, 16}, {16, 8}, {8, 8}, {4, 16}, {8, 4}, {4, 8}};
    const int levels[] = {2, 3, 4};
    trk_tuning cur;
    std::memset(&cur, 0, sizeof(cur));
    float best_ms = 1e30f;
    const trk_options saved = h->opt;
    const int saved_level = h->level, saved_grid = h->vote_grid;
    int bti = saved.tile_i, btj = saved.tile_j, blv = saved_level;
    for (const auto &t : tiles) {
        for (int lv : levels) {
            if (prepare_vote_kernel(t[0], t[1], lv) != cudaSuccess)
                continue;
            h->opt.tile_i = t[0];
            h->opt.tile_j = t[1];
            h->level = lv;
            h->vote_grid = vote_grid_for(h->n_sm, t[0], t[1], lv, saved.blocks_per_sm);
            for (auto &kv : h->graphs)
                cudaGraphExecDestroy(kv.second);
            h->graphs.clear();
            float tot = 0.0f;
            int ok = 1;
            for (int r = 0; r <= reps && ok; ++r) {
                const int rc = trk_reconstruct(h, hits, n_hits, event_offsets, n_events, nullptr,
                                               stream);
                if (rc != TRK_OK && rc != TRK_ERR_CAPACITY) {
                    ok = 0;
                    break;
                }
                float ms[8];
                if (trk_profile_stages(h, ms, stream) != TRK_OK) {
                    ok = 0;
                    break;
                }
                if (r > 0)
                    tot += ms[0];
            }
            if (ok && tot / reps < best_ms) {
                best_ms = tot / reps;
                bti = t[0];
                btj = t[1];
                blv = lv;
            }
        }
    }
    if (best_ms >= 1e29f) {
        h->opt = saved;
        h->level = saved_level;
        h->vote_grid = saved_grid;
        prepare_vote_kernel(saved.tile_i, saved.tile_j, saved_level);
        return fail(h, TRK_ERR_CUDA, "autotune: no configuration ran");
    }
    h->opt.tile_i = bti;
    h->opt.tile_j = btj;
    h->level = blv;
    h->vote_grid = vote_grid_for(h->n_sm, bti, btj, blv, saved.blocks_per_sm);
    TRK_CUDA(h, prepare_vote_kernel(bti, btj, blv));
    for (auto &kv : h->graphs)
        cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    best->tile_i = bti;
    best->tile_j = btj;
    best->vote_level = blv;
    best->vote_ms = best_ms;
    return TRK_OK;
}
