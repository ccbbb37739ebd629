/*
 * trk -- GB300-native displaced-track Hough transform (C ABI).
 *
 * The method (paper: "GPU Enhancement of the Trigger to Extend Physics Reach at the LHC",
 * Sec. 7 and Fig. 3, Sec. 8): every combination of hits maps to a point of a binned
 * track-parameter space, votes accumulate there, local maxima are track candidates and
 * their hits are handed on (Sec. 8, the fit after candidate finding).  Here the
 * combinations are hit triplets, one hit from each layer of a listed layer triple, and
 * the parameter space is the 5-parameter helix (phi0, q/pT, d0, cot(theta), z0) about
 * the coordinate origin with no beam-spot constraint, so that displaced tracks survive
 * (Sec. 8: curved displaced tracks need a parameter space beyond the two-parameter
 * interaction-point-constrained one; circles are fixed by centre and radius).
 *
 * Conventions (readings of the paper, which fixes none of them): units cm, GeV, T; field
 * along +z; pT = K B R with K = 0.299792458e-2 GeV/(T cm); positive charges turn
 * clockwise seen from +z, so q = -sign(D) with D = (p2 - p1) x (p3 - p1) in the
 * transverse plane (hits in layer order a, b, c); perigee P = closest point of the
 * circle to the origin, phi0 = direction of motion at P in [-pi, pi),
 * d0 = -P_x sin(phi0) + P_y cos(phi0); s_k = +-2R asin(|p_k - P| / 2R), the signed path
 * length from P: + for a hit after P in the direction of motion ((p_k - P) . (cos phi0,
 * sin phi0) >= 0), - for one before it, so that z = z0 + s cot(theta) holds on both sides
 * of the perigee (a hit at the point opposite P, where the sign is undefined, makes the
 * triplet edge-ambiguous); on a straight line (D == 0) s_k = +-|p_k - P|;
 * (cot(theta), z0) = unweighted least-squares line z = z0 + s cot(theta) over the three
 * hits; bin index floor((p - lo) / ((hi - lo)/n)), a triplet votes iff all five
 * parameters are in range, periodic dimensions are wrapped first; bins are numbered
 * row-major with phi0 slowest.  A bin is a candidate iff its count is >= threshold and
 * it beats every one of its 3^5 - 1 neighbours: >= all of them, and > those with a
 * smaller bin number.  A candidate's hits are the sorted union of the hits of the
 * triplets that voted for it; its parameters are its bin centre.
 *
 * Everything on the device runs in the library's own sm_103a kernels.  All functions
 * return 0 (TRK_OK) or a negative TRK_ERR_* code; none throws; none frees caller memory.
 * A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef TRK_H
#define TRK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TRK_MAX_LAYERS 64
#define TRK_MAX_TRIPLES 512

/* return codes */
#define TRK_OK 0
#define TRK_ERR_INVALID (-1)  /* bad argument: null pointer, bad size, bad geometry/binning */
#define TRK_ERR_CAPACITY (-2) /* some event exceeded a capacity; see the per-event status */
#define TRK_ERR_CUDA (-3)     /* a CUDA call failed; trk_last_error() has the text */
#define TRK_ERR_NOMEM (-4)    /* device or pinned-host allocation failed */
#define TRK_PENDING (-5)      /* served event not finished yet (trk_server_wait / _take) */

/* per-event status bits (an event with a non-zero status has no candidates: like a
 * problematic event in the filter farm, it is passed on unprocessed) */
#define TRK_EV_BAD_HIT 1        /* layer id out of range or non-finite coordinate */
#define TRK_EV_TOO_MANY_HITS 2  /* more hits than trk_options.max_hits_per_event */
#define TRK_EV_VOTE_OVERFLOW 4  /* the call's vote list overflowed */
#define TRK_EV_CAND_OVERFLOW 8  /* the call's candidate or assignment capacity overflowed */
#define TRK_EV_BAD_OFFSETS 16   /* event_offsets not non-decreasing within [0, n_hits] */

/* One hit: 16 bytes, float32 position in cm and the layer index (0 .. n_layers-1). */
typedef struct trk_hit {
    float x, y, z;
    int32_t layer;
} trk_hit;

/* Barrel geometry.  Only b_tesla, n_layers and the layer triples enter the arithmetic;
 * radius/z_half describe the detector for bookkeeping. */
typedef struct trk_geometry {
    int32_t n_layers;                       /* 3 .. TRK_MAX_LAYERS */
    int32_t n_triples;                      /* 1 .. TRK_MAX_TRIPLES */
    double b_tesla;                         /* > 0 */
    double radius[TRK_MAX_LAYERS];
    double z_half[TRK_MAX_LAYERS];
    int32_t triples[TRK_MAX_TRIPLES][3];    /* layer ids (a, b, c), pairwise distinct */
} trk_geometry;

/* Binning of (phi0, q/pT, d0, cot(theta), z0) in that order. */
typedef struct trk_binning {
    double lo[5], hi[5];                    /* lo < hi */
    int32_t n[5];                           /* >= 1; product < 2^32; n[3]*n[4] <= 8192 */
    int32_t periodic;                       /* bit k set: dimension k wraps (phi0: bit 0) */
    int32_t threshold;                      /* minimum votes of a candidate, >= 1 */
    float sagitta_fp64_cm;                  /* FP32 fits with |D| / |p3 - p1| at or below
                                               this are recomputed in FP64 (0: only D == 0) */
} trk_binning;

/* Capacities and tuning; trk_options_default() fills sensible values.  All device memory
 * is allocated once in trk_create. */
typedef struct trk_options {
    int32_t device;                         /* CUDA device ordinal */
    int32_t max_events;                     /* events per call (histogram slots) */
    int64_t max_hits;                       /* hits per call */
    int32_t max_hits_per_event;             /* <= 1 << 20 */
    int64_t vote_capacity;                  /* accepted triplets per call */
    int64_t cand_capacity;                  /* candidates per call */
    int64_t assign_capacity;                /* sum over candidates of 3 x votes per call */
    int64_t peak_scratch_bytes;             /* scratch of the peak filter (4 B x bins per
                                               event of a pass) */
    int32_t tile_i, tile_j;                 /* pair tile of the vote kernel (one block):
                                               16x16, 8x16, 16x8, 8x8, 4x16, or the one-warp
                                               tiles 8x4 and 4x8 */
    int32_t k_chunk;                        /* outer-layer hits staged per shared chunk */
    int32_t blocks_per_sm;                  /* persistent vote blocks per SM (0: auto) */
    int32_t use_graph;                      /* capture each call shape in a CUDA graph (the
                                               capture runs in the calling thread) */
    int32_t vote_level;                     /* vote kernel occupancy: 2, 3 or 4 blocks of 256
                                               threads per SM (0: 3) */
    int32_t fit_candidates;                 /* 1: fit a helix to every candidate's hits in
                                               the same call (trk_track, below); 0: skip */
} trk_options;

/* One candidate (48 bytes). */
typedef struct trk_candidate {
    uint32_t bin;                           /* row-major bin inside its event's histogram */
    int32_t event;                          /* event index within the call */
    int32_t votes;                          /* the bin's count */
    int32_t n_hits;                         /* number of assigned hits */
    int64_t hit_off;                        /* offset of its hits in hit_ids */
    float params[5];                        /* bin centre (phi0, q/pT, d0, cot, z0) */
    int32_t reserved;
} trk_candidate;

/* Fitted helix of one candidate (48 bytes), parallel to the candidates.
 *
 * Paper Sec. 8 (with Fig. 6): the candidates found in the parameter space are then fitted
 * to their hits; the paper times such a fit but does not define it.  The fit here, in
 * FP64 on the device, one thread per candidate, hits in the candidate's (sorted) order:
 *   1. algebraic circle fit of all the candidate's hits: (a, b, c) minimising
 *      sum (u^2 + v^2 + a u + b v + c)^2, (u, v) = (x, y) - centroid, through the 3 x 3
 *      normal equations; centre = centroid - (a, b)/2, R^2 = a^2/4 + b^2/4 - c;
 *   2. on each layer only the hit with the smallest | |p - centre| - R | is kept (ties: the
 *      earlier hit), and the circle is fitted again on the kept hits;
 *   3. the sense of rotation is the sign of the signed area of the kept hits' polygon in
 *      layer order (for three hits, D of the triplet); q/pT, phi0, d0 follow as for a
 *      triplet (perigee about the origin);
 *   4. signed arc lengths from the perigee as for a triplet, and the least-squares line
 *      z = z0 + s cot(theta) over the kept hits.
 * status: TRK_FIT_OK, TRK_FIT_FEW_LAYERS (kept hits on fewer than 3 layers) or
 * TRK_FIT_DEGENERATE (singular normal equations, centre on the origin, equal arc lengths);
 * the parameters are zero unless TRK_FIT_OK. */
#define TRK_FIT_OK 0
#define TRK_FIT_FEW_LAYERS 1
#define TRK_FIT_DEGENERATE 2

typedef struct trk_track {
    float params[5];                        /* phi0, q/pT [1/GeV], d0 [cm], cot(theta), z0 [cm] */
    float chi2_rphi;                        /* sum over kept hits of (|p - centre| - R)^2 [cm^2] */
    float chi2_rz;                          /* sum over kept hits of (z - z0 - s cot)^2 [cm^2] */
    int32_t n_used;                         /* kept hits */
    int32_t status;                         /* TRK_FIT_* */
    int32_t event;                          /* event index within the call */
    uint64_t layers;                        /* bit l set: a hit of layer l was kept */
} trk_track;

/* Results of one call.  Device arrays and host arrays are owned by the library and
 * stay valid until the next trk_reconstruct* on the same handle or trk_destroy. */
typedef struct trk_candidates {
    int32_t n_events;
    int64_t n_candidates;                   /* total over the call */
    int64_t n_hit_ids;                      /* total over the call */
    const int64_t *cand_off;                /* host [n_events + 1]: candidates of event e are
                                               cand[cand_off[e] .. cand_off[e+1]) */
    const int32_t *status;                  /* host [n_events]: TRK_EV_* bits */
    const trk_candidate *d_cand;            /* device [n_candidates], sorted by (event, bin) */
    const int32_t *d_hit_ids;               /* device [n_hit_ids]: input hit indices (global,
                                               i.e. into the call's hit array), sorted per
                                               candidate */
    const trk_candidate *h_cand;            /* host copies, filled only by
                                               trk_reconstruct_host (else NULL) */
    const int32_t *h_hit_ids;
    const trk_track *d_tracks;              /* device [n_candidates] fits when the handle was
                                               created with fit_candidates, else NULL */
    const uint8_t *d_hit_used;              /* device [n_hit_ids]: 1 if the fit kept the hit */
    const trk_track *h_tracks;              /* host copies (trk_reconstruct_host), else NULL */
    const uint8_t *h_hit_used;
} trk_candidates;

/* Counters of the last call. */
typedef struct trk_stats {
    int64_t n_triplets;                     /* sum over events and triples of |La||Lb||Lc| */
    int64_t n_fit;                          /* triplets through the FP32 fit (survivors of
                                               the curvature prefilter) */
    int64_t n_exact;                        /* of those, triplets whose q/pT and d0 are in
                                               range (through the longitudinal part) */
    int64_t n_votes;                        /* accepted triplets */
    int64_t n_fp64;                         /* fits redone in FP64 */
    int64_t n_candidates;
    int64_t n_hit_ids;
    int64_t n_work_items;
    double ms_total;                        /* device time of the call (events on the stream) */
    int64_t n_plateau;                      /* bins at their box maximum that share it with a
                                               neighbour (checked by the tie pass) */
    int64_t n_cand_votes;                   /* votes in candidate bins */
} trk_stats;

typedef struct trk_ctx trk_ctx;

/* Defaults for a workload of at most max_events events and max_hits hits per call. */
void trk_options_default(trk_options *opt, int32_t max_events, int64_t max_hits);

/* Create a handle: validates geometry and binning, copies them to the device and
 * allocates every pool.  *out receives the handle (NULL on failure).
 * Paper Sec. 8: the event, the parameter space and the peak detection are resident on the
 * GPU; the handle holds the geometry, the binned parameter space (Sec. 7, Fig. 3) and
 * every buffer of the steps below, so that no call allocates. */
int trk_create(trk_ctx **out, const trk_geometry *geometry, const trk_binning *binning,
               const trk_options *options /* nullable: defaults for 1 event */);

/* Reconstruct n_events events: paper Sec. 7 and Fig. 3 (every hit combination votes into
 * the binned parameter space; local maxima are track candidates) with Sec. 8's curved
 * displaced tracks (circle by centre and radius, no beam-spot constraint) and Sec. 8's
 * hand-over of each candidate's hits to a fit.  Steps: pack the hits per layer, fit and
 * bin every triplet of every listed layer triple, vote, find the candidate bins, collect
 * each candidate's hits.
 * hits: DEVICE pointer to n_hits trk_hit; event_offsets:
 * DEVICE pointer to n_events + 1 int64, event e owning hits [off[e], off[e+1]).  Runs on
 * `stream` (a cudaStream_t, NULL = the legacy default stream) and returns after the
 * per-event counts reached the host (the call's only synchronisation).  Returns TRK_OK,
 * TRK_ERR_CAPACITY (some event flagged, the others are complete), or an error. */
int trk_reconstruct(trk_ctx *h, const trk_hit *hits, int64_t n_hits,
                    const int64_t *event_offsets, int32_t n_events, trk_candidates *out,
                    void *stream);

/* Same, from HOST buffers (any host memory): copies the hits in, reconstructs and copies
 * the candidates and hit ids back to library-owned pinned host memory (out->h_cand,
 * out->h_hit_ids).  The end-to-end path of a caller whose events live in host memory
 * (paper Sec. 8: the event is transferred to the GPU, processed there, and the candidates
 * come back to the host for the fit). */
int trk_reconstruct_host(trk_ctx *h, const trk_hit *hits, int64_t n_hits,
                         const int64_t *event_offsets, int32_t n_events,
                         trk_candidates *out, void *stream);

/* Destroy a handle and free everything it owns (the paper has no counterpart).  Waits for
 * the handle's own work (its streams), not for the whole device.  NULL is accepted. */
int trk_destroy(trk_ctx *h);

/* Counters of the last call. */
int trk_get_stats(trk_ctx *h, trk_stats *out);

/* Vote-kernel configuration chosen by trk_autotune. */
typedef struct trk_tuning {
    int32_t tile_i, tile_j;                 /* pair tile of a block */
    int32_t vote_level;                     /* occupancy level (blocks of 256 threads / SM) */
    float vote_ms;                          /* mean vote-kernel time of the winner */
} trk_tuning;

/* Autotuner: reconstructs the given events (DEVICE buffers, as trk_reconstruct) reps + 1
 * times with every supported vote-kernel tile and occupancy level, keeps the one whose
 * vote kernel is fastest (the results do not depend on the choice) and reports it.
 * Later calls use it; cached graphs are dropped.  Synchronises. */
int trk_autotune(trk_ctx *h, const trk_hit *hits, int64_t n_hits, const int64_t *event_offsets,
                 int32_t n_events, int32_t reps, trk_tuning *best, void *stream);

/* Copy event e's dense vote histogram of the last call (n bins int32, row-major) to the
 * DEVICE buffer dst, on `stream`. */
int trk_get_histogram(trk_ctx *h, int32_t event, int32_t *dst, void *stream);

/* Number of bins of one event's histogram. */
int64_t trk_histogram_size(const trk_ctx *h);

/* The last call's accepted triplets, decoded: for vote v, dst[4v..4v+3] = (event, i, j, k)
 * with i, j, k input hit indices (global) from layers a, b, c, and bins[v] its bin.  DEVICE
 * buffers of capacity `cap` votes; *n_out receives the number of votes (all are written
 * only if n_out <= cap).  Synchronises the stream. */
int trk_get_votes(trk_ctx *h, int32_t *dst, uint32_t *bins, int64_t cap, int64_t *n_out,
                  void *stream);

/* Fit explicit triplets with exactly the arithmetic of the vote kernel: for t < n,
 * ijk[3t..3t+2] are indices into hits[0 .. n_hits) (DEVICE).  Writes params[5t..5t+4]
 * (FP32, NaN when degenerate), bins[t] (valid when accepted) and flags[t]: bit 0
 * accepted, bit 1 computed in FP64, bit 2 degenerate, bit 3 index out of range (nothing
 * else written for that triplet).  All DEVICE buffers.  Asynchronous. */
int trk_fit_triplets(trk_ctx *h, const trk_hit *hits, int64_t n_hits, const int32_t *ijk,
                     int64_t n, float *params, uint32_t *bins, int32_t *flags, void *stream);

/* Device time (ms) of the stages of the last call, from CUDA events the library records on
 * the call's stream: ms[0] the vote kernel (triplet fit + vote), ms[1] argument copy,
 * histogram clear, packing and scheduling, ms[2] the peak finder, ms[3] candidate emission,
 * ms[4] hit assignment and compaction, ms[5] the candidate fit (when enabled) and the
 * result copies; ms[6..7] = 0.  Synchronises. */
int trk_profile_stages(trk_ctx *h, float ms[8], void *stream);

/* ---- serving: continuous batching of events that arrive one at a time ------------------
 * The paper's filter unit takes one event after another and overlaps the next event's
 * transfer with the current one's processing (Sec. 8).  A server keeps n_lanes complete
 * handles resident (each with its own pools, stream and graphs, created with
 * lane_options) and a host queue of submitted events.  Each lane runs on its own host
 * thread.  A free lane admits waiting events, in arrival order, while they fit its
 * capacities (lane_options.max_events events, max_hits hits, and the device memory of its
 * vote list) and the backlog (one event more than the first per 24 waiting: batching
 * delays every event of a batch to its end and pays only when many wait), and copies them
 * to the device while another lane computes.  The lanes take the GPU in turn: a lane
 * holds it from launching its call until the kernels are done, then copies the
 * candidates back and files each event's results while the next batch computes.  An
 * event's results are identical whether it is reconstructed alone, in a batch or by the
 * server. */
typedef struct trk_server trk_server;

typedef struct trk_served_event {
    int32_t status;                         /* TRK_EV_* bits of the event (-1: call failed) */
    int32_t rc;                             /* return code of the lane's reconstruction */
    double latency_s;                       /* submit -> results on the host */
    int32_t batch_events;                   /* events reconstructed in the same call */
    int64_t n_candidates;
    int64_t n_hit_ids;
} trk_served_event;

/* Paper Sec. 8 for every call below: the filter unit processes a stream of events, and
 * the next event's transfer and processing overlap the current one's.
 * Create a server of n_lanes (1..16) lanes; each lane allocates one trk handle with
 * lane_options: a batch holds at most lane_options.max_events events and max_hits hits.
 * fit_candidates is ignored (served events return candidates and hits).  With use_graph,
 * the graph of every batch size is captured here, in the calling thread, so that lanes
 * only launch graphs.  Device memory decides admission: an event's votes are bounded by
 * its hit triplets times the largest acceptance fraction seen so far (starting from 1/2),
 * and a lane admits waiting events, in arrival order, while their bounds fit its vote list
 * (a batch that overflows anyway is run again one event at a time).  With
 * lane_options.vote_capacity 0 the vote lists are sized from the device memory free at
 * creation (cudaMemGetInfo), 90 % of it shared by the lanes. */
int trk_server_create(trk_server **out, const trk_geometry *geometry, const trk_binning *binning,
                      const trk_options *lane_options, int32_t n_lanes);

/* Queue one event (HOST hits, copied before returning); *ticket identifies it.
 * TRK_ERR_CAPACITY if it has more hits than a lane accepts. */
int trk_server_submit(trk_server *s, const trk_hit *hits, int64_t n_hits, uint64_t *ticket);

/* Wait up to timeout_s seconds (0: do not wait) for an event; TRK_PENDING if not done. */
int trk_server_wait(trk_server *s, uint64_t ticket, double timeout_s, trk_served_event *out);

/* Copy a finished event's candidates (hit_off into hit_ids, event 0) and its hit ids
 * (event-local indices, sorted per candidate) to HOST buffers and forget the event. */
int trk_server_take(trk_server *s, uint64_t ticket, trk_candidate *cand, int64_t cand_cap,
                    int32_t *hit_ids, int64_t hit_cap);

/* Batches run, events finished, events whose call or status failed, events waiting. */
int trk_server_counts(trk_server *s, int64_t *n_batches, int64_t *n_events, int64_t *n_failed,
                      int64_t *n_queued);

/* Stop the lanes (finishing queued events) and free everything.  NULL is accepted. */
int trk_server_destroy(trk_server *s);

/* Largest histogram, in bins per event, that trk_find_peaks_noalloc accepts. */
#define TRK_NOALLOC_MAX_BINS (1 << 21)

/* Candidate bins of dense vote histograms, for callers that may not allocate device memory.
 * The paper has no counterpart: this is a deployment variant of the peak step.
 *
 * Who needs it: code that must never call cudaMalloc (or any allocating library routine)
 * while it runs -- a trigger path with a fixed latency budget where an allocation could
 * stall, a process whose device memory is all handed out up front by its own pool, a
 * plug-in that is given device buffers by a host framework and may not own any.  Such a
 * caller cannot create a trk handle (trk_create allocates its pools) but may hold vote
 * histograms.  This function applies the candidate rule of trk_reconstruct to them and
 * allocates nothing: the peak filter's scratch (up to 12 bytes per bin) is in static device
 * arrays of the library, 24 MiB, present on every GPU that loads the library until the
 * process exits.
 *
 * hist: DEVICE int32, n_events dense histograms of the binning's size, row-major (as
 * trk_get_histogram writes them), 4-byte aligned (any int32 pointer; 16-byte alignment
 * lets the kernels use wider loads); cand_bits: DEVICE uint32, n_events x ceil(bins / 32)
 * words, 4-byte aligned, bit b of event e set iff bin b is a candidate; both owned by the
 * caller.  Runs on
 * `stream` (a cudaStream_t; NULL = legacy default stream), asynchronously.
 * Returns TRK_ERR_INVALID (nothing launched) for null or misaligned pointers,
 * n_events < 1, an invalid binning, or more than TRK_NOALLOC_MAX_BINS bins; TRK_ERR_CUDA on
 * a launch failure.
 * trk_last_error(NULL) gives the reason.
 *
 * The first call on a device sets that device up (looks up the static array's device
 * addresses with cudaGetSymbolAddress and sets kernel attributes): make that first call
 * outside any stream capture.  Every call on a device uses the same arrays, which keep
 * the last call's contents (each call clears what it needs cleared -- its list counter
 * and the caller's cand_bits -- and writes every other entry before reading it); calls
 * whose work overlaps on the GPU (other streams, other threads) race on them and must be
 * serialized by the caller.  The device addresses are kept for the life of the process:
 * do not call this function after cudaDeviceReset. */
int trk_find_peaks_noalloc(const int32_t *hist, int32_t n_events, const trk_binning *binning,
                           uint32_t *cand_bits, void *stream);

/* ---------------------------------------------------------------------------------------
 * Per-hit 2-D Hough transforms (the paper's own demonstrations)
 *
 * TRK2D_STRAIGHT -- Sec. 7 and Fig. 3: each hit of a straight track maps to a sinusoid in
 *   the (theta, rho) space of lines x cos(theta) + y sin(theta) = rho; peaks are tracks.
 *   Column c: theta_c = (c + 1/2) pi / n_cols; a hit votes in each column for the row of
 *   rho = x cos(theta_c) + y sin(theta_c).  Columns wrap with the row mirrored (theta and
 *   theta + pi are the same line with rho negated), so the rho range must be symmetric.
 * TRK2D_CURVED_IP -- Sec. 8 and Fig. 5: curved tracks constrained to the interaction point,
 *   a 2-D space like the straight case.  Column c: phi0_c = -pi + (c + 1/2) 2 pi / n_cols;
 *   a hit votes for the q/pT of the circle through the origin and the hit that leaves the
 *   origin in direction phi0_c: q/pT = 2 (x sin(phi0_c) - y cos(phi0_c)) / (K B (x^2 + y^2)),
 *   K = 0.299792458e-2 GeV/(T cm) (positive charges turn clockwise).  Columns wrap.
 * Both: row j = floor((v - lo) / ((hi - lo) / n_rows)), a vote iff lo <= v < hi; one
 * histogram of n_cols x n_rows int32 per event, bin = c * n_rows + j.  A bin is a candidate
 * iff h >= threshold, h >= each of its 8 neighbours and h > each neighbour with a smaller
 * bin number (rows outside the range have no neighbour; columns wrap as above).  A
 * candidate's hits are the hits that voted in its bin.  Hits use only x and y; layer and z
 * are ignored.  FP32 on the device.
 *
 * Vertices (TRK2D_STRAIGHT only, vertex_bins > 0) -- Sec. 9 and Figs. 7-8, displaced jets:
 * the track peaks of a jet lie on one sinusoid of (theta, rho), the sinusoid of the jet's
 * vertex, and a second Hough transform over the peaks finds it.  Each candidate
 * with votes >= vertex_min_votes draws its line x cos(theta) + y sin(theta) = rho (bin
 * centres, FP64) into a vertex_bins x vertex_bins grid over [-vertex_range, vertex_range)^2
 * (cell centres g_a = -range + (a + 1/2) w): once per x column in the row of
 * y = (rho - g_a cos(theta)) / sin(theta) when |sin(theta)| >= |cos(theta)|, else once per y
 * row in the column of x = (rho - g_b sin(theta)) / cos(theta).  Cell (a, b) has index
 * a * vertex_bins + b; vertices are the cells passing the 2-D peak rule (8 neighbours, no
 * wrap) with vertex_threshold; a vertex's tracks are the candidates that voted in its cell.
 * --------------------------------------------------------------------------------------- */
#define TRK2D_STRAIGHT 0
#define TRK2D_CURVED_IP 1

typedef struct trk2d_config {
    int32_t kind;                           /* TRK2D_* */
    int32_t n_cols;                         /* theta / phi0 bins, 3 .. 65536 */
    int32_t n_rows;                         /* rho / q/pT bins, 2 .. 16384 */
    int32_t threshold;                      /* >= 1 */
    double lo, hi;                          /* row range (cm, or 1/GeV) */
    double b_tesla;                         /* field (TRK2D_CURVED_IP) */
    int32_t max_events;                     /* events per call */
    int32_t reserved;
    int64_t max_hits;                       /* hits per call */
    int64_t cand_capacity;                  /* candidates per call */
    int64_t hit_capacity;                   /* sum over candidates of their hits per call */
    int32_t vertex_bins;                    /* 0: no vertex transform; else 3 .. 128 */
    int32_t vertex_threshold;               /* >= 1 */
    int32_t vertex_min_votes;               /* candidates below it draw no line */
    int32_t max_vertices;                   /* per event, <= 1024 */
    double vertex_range;                    /* cm */
} trk2d_config;

#define TRK2D_VERTEX_MAX_TRACKS 64          /* tracks listed per vertex */

typedef struct trk2d_vertex {               /* 32 bytes */
    uint32_t cell;                          /* a * vertex_bins + b */
    int32_t event;
    int32_t votes;                          /* candidate lines through the cell */
    int32_t n_tracks;                       /* listed: min(votes, TRK2D_VERTEX_MAX_TRACKS),
                                               the candidates with the smallest indices */
    float xy[2];                            /* cell centre (cm) */
    int64_t track_off;                      /* its tracks: vertex_tracks[track_off ..
                                               track_off + n_tracks), candidate indices into
                                               d_cand, ascending */
} trk2d_vertex;

typedef struct trk2d_candidate {            /* 32 bytes */
    uint32_t bin;                           /* c * n_rows + j */
    int32_t event;
    int32_t votes;                          /* = number of hits */
    int32_t reserved;
    int64_t hit_off;                        /* offset of its hits in hit_ids */
    float params[2];                        /* column centre (theta or phi0), row centre */
} trk2d_candidate;

typedef struct trk2d_result {
    int32_t n_events;
    int64_t n_candidates;
    int64_t n_hit_ids;
    const int64_t *cand_off;                /* host [n_events + 1] */
    const trk2d_candidate *d_cand;          /* device, sorted by (event, bin) */
    const int32_t *d_hit_ids;               /* device: input hit indices (global), sorted per
                                               candidate */
    int64_t n_vertices;                     /* total over the call (0 without vertex_bins) */
    const int64_t *vertex_off;              /* host [n_events + 1] */
    const trk2d_vertex *d_vertices;         /* device, sorted by (event, cell) */
    const int32_t *d_vertex_tracks;         /* device */
    int32_t vertex_overflow;                /* 1: some event had more than max_vertices (its
                                               list holds the first max_vertices by cell) */
} trk2d_result;

typedef struct trk2d_ctx trk2d_ctx;

/* Validates the configuration and allocates every buffer on `device`.  TRK_ERR_INVALID on a
 * bad configuration (trk_last_error(NULL) says which), TRK_ERR_NOMEM, TRK_ERR_CUDA. */
int trk2d_create(trk2d_ctx **out, const trk2d_config *config, int32_t device);

/* Histogram, peaks and hit lists for a batch of events: hits and event_offsets are DEVICE
 * buffers as for trk_reconstruct; outputs are library-owned and valid until the next call
 * on the handle.  TRK_ERR_INVALID on bad arguments (more events or hits than configured),
 * TRK_ERR_CAPACITY when the candidates or their hits overflowed (the outputs are then
 * empty).  Runs on `stream` (NULL: the handle's own), then synchronises it. */
int trk2d_reconstruct(trk2d_ctx *h, const trk_hit *hits, int64_t n_hits,
                      const int64_t *event_offsets, int32_t n_events, trk2d_result *out,
                      void *stream);

/* The vertex transform alone, over candidates the caller supplies (DEVICE arrays: cand
 * sorted by event, cand_off [n_events + 1] the per-event ranges; only bin, event and votes
 * are read): for peaks found elsewhere.  Needs a handle created with vertex_bins.  Fills
 * the vertex fields of out (the candidate fields are zero); vertex track indices point
 * into the caller's cand.  Synchronous. */
int trk2d_find_vertices(trk2d_ctx *h, const trk2d_candidate *cand, const int64_t *cand_off,
                        int32_t n_events, trk2d_result *out, void *stream);

/* Copy event e's histogram of the last call (n_cols x n_rows int32, DEVICE dst).
 * Synchronous. */
int trk2d_get_histogram(trk2d_ctx *h, int32_t event, int32_t *dst, void *stream);

/* Device time (ms) of the last call's vote-and-peak kernel and of the whole call. */
int trk2d_last_ms(trk2d_ctx *h, float *vote_peak_ms, float *total_ms);

/* Text of the last error on a 2-D handle (NULL: of the calling thread's last failed
 * trk2d_create). */
const char *trk2d_last_error(const trk2d_ctx *h);

int trk2d_destroy(trk2d_ctx *h);

/* Text of the last error on this handle (h NULL: of the last failed trk_create or
 * trk_find_peaks_noalloc). */
const char *trk_last_error(const trk_ctx *h);

/* Library version string. */
const char *trk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TRK_H */
