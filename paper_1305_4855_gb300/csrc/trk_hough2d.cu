// Per-hit 2-D Hough transforms: straight lines (paper Sec. 7, Fig. 3: every hit traces a
// sinusoid in (theta, rho), peaks are tracks) and curved tracks constrained to the
// interaction point (Sec. 8, Fig. 5: a 2-D space like the straight case).  The definitions
// are given with trk2d_config in trk.h.
//
// GB300 layout: one block per (event, slab of columns).  The block's slab of the
// histogram, with one halo column on each side, sits in shared memory; every hit of the
// event votes in every column of the slab (a warp per column, lanes over hits, shared-
// memory atomics).  The peak rule then reads only shared memory, and the slab is written
// out once (coalesced) for the candidate emission and the histogram copy.  Candidate bits
// go to a bitmap; a scan of its popcounts orders the candidates by (event, bin), a scan of
// their votes places their hit lists, and a warp per candidate re-evaluates the event's
// hits in the candidate's column with the same arithmetic as the vote.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include <cuda_runtime.h>

#include "trk_common.cuh"
#include "trk_scan.cuh"

namespace trk {

struct H2Const {
    int kind, n_cols, n_rows, threshold;
    float lo, hi, inv_w, kB;
    float col_w, col_lo;          // column centre = col_lo + (c + 1/2) col_w
    double lo_d, w_d, col_lo_d, col_w_d;   // the same in FP64, for the bin centres
    uint32_t nbins;
    int64_t W;                    // bitmap words per event
    // vertex transform
    int vb, v_threshold, v_min_votes, max_vertices;
    double v_range, v_w;
};

struct H2Counters {
    unsigned long long n_cand, n_hit;
};

constexpr int kH2Threads = 256;
constexpr int kH2Stage = 1024;    // hits staged per chunk

// Row of a hit in a column: v = scale (x a + y b), the same expression in every kernel.
__device__ __forceinline__ float h2_scale(const H2Const &K, float x, float y)
{
    return K.kind == TRK2D_CURVED_IP ? 2.0f / (K.kB * fmaf(x, x, y * y)) : 1.0f;
}

__device__ __forceinline__ bool h2_row(const H2Const &K, float x, float y, float scale,
                                       float2 ab, int &j)
{
    const float v = scale * fmaf(x, ab.x, y * ab.y);
    if (!(v >= K.lo && v < K.hi))
        return false;
    const int jj = (int)floorf((v - K.lo) * K.inv_w);
    j = jj < 0 ? 0 : (jj >= K.n_rows ? K.n_rows - 1 : jj);
    return true;
}

// Global column of local column lc of a slab starting at c0, and whether its rows are
// stored mirrored (a straight-line column reached across the theta wrap).
__device__ __forceinline__ int h2_map_col(const H2Const &K, int gc, bool &mirror)
{
    mirror = false;
    if (gc < 0) {
        gc += K.n_cols;
        mirror = K.kind == TRK2D_STRAIGHT;
    } else if (gc >= K.n_cols) {
        gc -= K.n_cols;
        mirror = K.kind == TRK2D_STRAIGHT;
    }
    return gc;
}

__global__ void __launch_bounds__(kH2Threads) k_h2_vote_peak(H2Const K, const trk_hit *hits,
                                                             const int64_t *offsets,
                                                             const float2 *coef, int S,
                                                             int32_t *hist, uint32_t *cbits)
{
    extern __shared__ int32_t sh[];                 // (S + 2) x n_rows counts
    __shared__ float3 s_hit[kH2Stage];
    const int e = blockIdx.y;
    const int c0 = blockIdx.x * S;
    const int nint = min(S, K.n_cols - c0);          // interior columns of this slab
    const int ncl = nint + 2;
    const int R = K.n_rows;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < ncl * R; q += kH2Threads)
        sh[q] = 0;
    const int64_t h0 = offsets[e], h1 = offsets[e + 1];
    __syncthreads();
    for (int64_t b0 = h0; b0 < h1; b0 += kH2Stage) {
        const int nh = (int)min((int64_t)kH2Stage, h1 - b0);
        for (int q = threadIdx.x; q < nh; q += kH2Threads) {
            const trk_hit hh = hits[b0 + q];
            s_hit[q] = make_float3(hh.x, hh.y, h2_scale(K, hh.x, hh.y));
        }
        __syncthreads();
        for (int lc = w; lc < ncl; lc += kH2Threads / 32) {
            bool mirror;
            const int gc = h2_map_col(K, c0 - 1 + lc, mirror);
            const float2 ab = coef[gc];
            int32_t *col = sh + lc * R;
            for (int q = lane; q < nh; q += 32) {
                const float3 p = s_hit[q];
                int j;
                if (h2_row(K, p.x, p.y, p.z, ab, j))
                    atomicAdd(col + (mirror ? R - 1 - j : j), 1);
            }
        }
        __syncthreads();
    }
    // peak rule on the interior columns; the slab goes out to the event's histogram
    int32_t *he = hist + (size_t)e * K.nbins;
    for (int q = threadIdx.x; q < nint * R; q += kH2Threads) {
        const int lc = 1 + q / R, j = q - (q / R) * R;
        const int h = sh[lc * R + j];
        const int gc = c0 + lc - 1;
        const uint32_t bin = (uint32_t)gc * R + j;
        he[bin] = h;
        if (h < K.threshold)
            continue;
        bool cand = true;
        for (int dc = -1; dc <= 1 && cand; ++dc) {
            bool mirror;
            const int nc = h2_map_col(K, gc + dc, mirror);
            for (int dj = -1; dj <= 1; ++dj) {
                if (dc == 0 && dj == 0)
                    continue;
                const int r = j + dj;                  // stored row in the slab
                if (r < 0 || r >= R)
                    continue;
                const int hn = sh[(lc + dc) * R + r];
                const uint32_t nbin = (uint32_t)nc * R + (mirror ? R - 1 - r : r);
                if (nbin == bin)
                    continue;
                if (hn > h || (hn == h && nbin < bin)) {
                    cand = false;
                    break;
                }
            }
        }
        if (cand)
            atomicOr(&cbits[(size_t)e * K.W + (bin >> 5)], 1u << (bin & 31));
    }
}

__global__ void k_h2_emit(H2Const K, const uint32_t *cbits, const uint32_t *wprefix,
                          int64_t n_words, const int32_t *hist, trk2d_candidate *cand,
                          int64_t cand_cap)
{
    for (int64_t gw = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gw < n_words;
         gw += (int64_t)gridDim.x * blockDim.x) {
        uint32_t word = cbits[gw];
        int64_t idx = wprefix[gw];
        const int e = (int)(gw / K.W);
        const int64_t wl = gw - (int64_t)e * K.W;
        while (word) {
            const int bit = __ffs(word) - 1;
            word &= word - 1;
            if (idx < cand_cap) {
                const uint32_t bin = (uint32_t)(wl * 32 + bit);
                trk2d_candidate c;
                c.bin = bin;
                c.event = e;
                c.votes = hist[(size_t)e * K.nbins + bin];
                c.reserved = 0;
                c.hit_off = 0;
                const int col = (int)(bin / (uint32_t)K.n_rows), row = (int)(bin % (uint32_t)K.n_rows);
                c.params[0] = (float)(K.col_lo_d + (col + 0.5) * K.col_w_d);
                c.params[1] = (float)(K.lo_d + (row + 0.5) * K.w_d);
                cand[idx] = c;
            }
            ++idx;
        }
    }
}

struct H2CandVotes {
    const trk2d_candidate *c;
    __device__ int64_t operator()(int64_t i) const { return c[i].votes; }
};

__global__ void k_h2_set_off(trk2d_candidate *cand, const int64_t *off,
                             const unsigned long long *n_cand, int64_t cand_cap)
{
    int64_t n = (int64_t)*n_cand;
    n = n < cand_cap ? n : cand_cap;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        cand[i].hit_off = off[i];
}

// A warp per candidate: the event's hits in input order whose row in the candidate's
// column is the candidate's row (exactly the hits that voted there).
__global__ void k_h2_assign(H2Const K, const trk_hit *hits, const int64_t *offsets,
                            const float2 *coef, const trk2d_candidate *cand,
                            const unsigned long long *n_cand, int64_t cand_cap, int32_t *hit_ids,
                            int64_t hit_cap)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t n = (int64_t)*n_cand;
    n = n < cand_cap ? n : cand_cap;
    for (int64_t ci = warp0; ci < n; ci += nwarps) {
        const trk2d_candidate c = cand[ci];
        const int col = (int)(c.bin / (uint32_t)K.n_rows), row = (int)(c.bin % (uint32_t)K.n_rows);
        const float2 ab = coef[col];
        const int64_t h0 = offsets[c.event], h1 = offsets[c.event + 1];
        int64_t pos = c.hit_off;
        const int64_t end = c.hit_off + c.votes;
        for (int64_t b0 = h0; b0 < h1; b0 += 32) {
            const int64_t k = b0 + lane;
            bool match = false;
            if (k < h1) {
                const trk_hit hh = hits[k];
                int j;
                match = h2_row(K, hh.x, hh.y, h2_scale(K, hh.x, hh.y), ab, j) && j == row;
            }
            const unsigned m = __ballot_sync(kFull, match);
            const int64_t at = pos + __popc(m & lanemask_lt());
            if (match && at < end && at < hit_cap)
                hit_ids[at] = (int32_t)k;
            pos += __popc(m);
        }
    }
}

__global__ void k_h2_cand_off(const uint32_t *wprefix, int64_t W, int n_events,
                              const unsigned long long *n_cand, int64_t *cand_off)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n_events)
        cand_off[e] = wprefix[(size_t)e * W];
    else if (e == n_events)
        cand_off[e] = (int64_t)*n_cand;
}

// ---------------------------------------------------------------------------------------
// vertices: a block per event; the (x, y) grid in shared memory
// ---------------------------------------------------------------------------------------

constexpr int kVtxThreads = 256;

// Line geometry of a candidate, computed once (FP64): cos and sin of its theta and rho.
struct VtxLine {
    double c, s, rho;
    int by_col;      // sweep x columns (|sin| >= |cos|) or y rows
    int pad;
};

__global__ void k_h2_cand_geom(H2Const K, const trk2d_candidate *cand,
                               const unsigned long long *n_dev, int64_t n_host, int64_t cap,
                               VtxLine *geom)
{
    int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    n = n < cap ? n : cap;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t bin = cand[i].bin;
        const int col = (int)(bin / (uint32_t)K.n_rows), row = (int)(bin % (uint32_t)K.n_rows);
        const double theta = K.col_lo_d + (col + 0.5) * K.col_w_d;
        VtxLine L;
        sincos(theta, &L.s, &L.c);
        L.rho = K.lo_d + (row + 0.5) * K.w_d;
        L.by_col = fabs(L.s) >= fabs(L.c);
        L.pad = 0;
        geom[i] = L;
    }
}

// Cell of a line at step a (its swept column or row), or -1.
__device__ __forceinline__ int vtx_cell(const H2Const &K, const VtxLine &L, int a)
{
    const double g = -K.v_range + (a + 0.5) * K.v_w;
    const double other = L.by_col ? (L.rho - g * L.c) / L.s : (L.rho - g * L.s) / L.c;
    if (!(other >= -K.v_range && other < K.v_range))
        return -1;
    int k = (int)floor((other + K.v_range) / K.v_w);
    k = k >= K.vb ? K.vb - 1 : k;
    return L.by_col ? a * K.vb + k : k * K.vb + a;
}

// Does the raster of candidate bin `bin` contain `cell`?  (It visits one cell per swept
// column or row, so only the step through the cell's column or row is evaluated.)
__device__ __forceinline__ bool vtx_raster_has(const H2Const &K, const VtxLine &L, int cell)
{
    const int a = cell / K.vb, b = cell - (cell / K.vb) * K.vb;
    return vtx_cell(K, L, L.by_col ? a : b) == cell;
}

// The 2-D peak rule on the (x, y) grid (8 neighbours, no wrap) for cell with count h.
__device__ __forceinline__ bool vtx_is_peak(const int32_t *vh, int nb, int cell, int h)
{
    const int a = cell / nb, b = cell - (cell / nb) * nb;
    for (int da = -1; da <= 1; ++da)
        for (int db = -1; db <= 1; ++db) {
            if (da == 0 && db == 0)
                continue;
            const int aa = a + da, bb = b + db;
            if (aa < 0 || aa >= nb || bb < 0 || bb >= nb)
                continue;
            const int nbc = aa * nb + bb, hn = vh[nbc];
            if (hn > h || (hn == h && nbc < cell))
                return false;
        }
    return true;
}

__global__ void __launch_bounds__(kVtxThreads) k_h2_vertex(H2Const K, const trk2d_candidate *cand,
                                                           const VtxLine *geom,
                                                           const int64_t *cand_off,
                                                           int64_t cand_cap,
                                                           trk2d_vertex *slots,
                                                           int32_t *slot_tracks, int32_t *count,
                                                           int32_t *overflow)
{
    extern __shared__ int32_t vh[];              // vb * vb cells
    __shared__ int32_t s_warp[kVtxThreads / 32];
    __shared__ int32_t s_ntr[1024];
    const int e = blockIdx.x;
    const int nb = K.vb, ncell = nb * nb;
    int64_t c0 = cand_off[e], c1 = cand_off[e + 1];
    c0 = c0 < cand_cap ? c0 : cand_cap;
    c1 = c1 < cand_cap ? c1 : cand_cap;
    const int64_t nc = c1 - c0;
    for (int q = threadIdx.x; q < ncell; q += kVtxThreads)
        vh[q] = 0;
    for (int q = threadIdx.x; q < K.max_vertices; q += kVtxThreads)
        s_ntr[q] = 0;
    __syncthreads();
    for (int64_t q = threadIdx.x; q < nc * nb; q += kVtxThreads) {
        const int64_t i = c0 + q / nb;
        if (cand[i].votes < K.v_min_votes)
            continue;
        const int cell = vtx_cell(K, geom[i], (int)(q % nb));
        if (cell >= 0)
            atomicAdd(&vh[cell], 1);
    }
    __syncthreads();
    // peaks in cell order: each thread a contiguous run of cells, then a block scan
    const int per = (ncell + kVtxThreads - 1) / kVtxThreads;
    const int p0 = threadIdx.x * per, p1 = min(p0 + per, ncell);
    int mine = 0;
    for (int cell = p0; cell < p1; ++cell) {
        const int h = vh[cell];
        if (h < K.v_threshold)
            continue;
        mine += vtx_is_peak(vh, nb, cell, h);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(kFull, incl, o);
        if (lane >= o)
            incl += u;
    }
    if (lane == 31)
        s_warp[w] = incl;
    __syncthreads();
    int base = 0;
    for (int k = 0; k < w; ++k)
        base += s_warp[k];
    int total = 0;
    for (int k = 0; k < kVtxThreads / 32; ++k)
        total += s_warp[k];
    int idx = base + incl - mine;
    __syncthreads();                             // every peak test has read the counts
    for (int cell = p0; cell < p1 && mine > 0; ++cell) {
        const int h = vh[cell];
        if (h < K.v_threshold)
            continue;
        if (!vtx_is_peak(vh, nb, cell, h))
            continue;
        const int a = cell / nb, b = cell - (cell / nb) * nb;
        if (idx < K.max_vertices) {
            trk2d_vertex v;
            v.cell = (uint32_t)cell;
            v.event = e;
            v.votes = h;
            v.n_tracks = 0;
            v.xy[0] = (float)(-K.v_range + (a + 0.5) * K.v_w);
            v.xy[1] = (float)(-K.v_range + (b + 0.5) * K.v_w);
            v.track_off = ((int64_t)e * K.max_vertices + idx) * TRK2D_VERTEX_MAX_TRACKS;
            slots[(size_t)e * K.max_vertices + idx] = v;
        }
        ++idx;
    }
    __syncthreads();
    // mark the vertex cells with their slot (the counts are no longer needed)
    const int nv = total < K.max_vertices ? total : K.max_vertices;
    for (int k = threadIdx.x; k < nv; k += kVtxThreads)
        vh[slots[(size_t)e * K.max_vertices + k].cell] = -(k + 1);
    __syncthreads();
    for (int64_t q = threadIdx.x; q < nc * nb; q += kVtxThreads) {
        const int64_t i = c0 + q / nb;
        if (cand[i].votes < K.v_min_votes)
            continue;
        const int cell = vtx_cell(K, geom[i], (int)(q % nb));
        if (cell < 0 || vh[cell] >= 0)
            continue;
        const int slot = -vh[cell] - 1;
        if (slots[(size_t)e * K.max_vertices + slot].votes > TRK2D_VERTEX_MAX_TRACKS)
            continue;                            // listed below, in candidate order
        const int k = atomicAdd(&s_ntr[slot], 1);
        if (k < TRK2D_VERTEX_MAX_TRACKS)
            slot_tracks[((int64_t)e * K.max_vertices + slot) * TRK2D_VERTEX_MAX_TRACKS + k] =
                (int32_t)(c0 + q / nb);
    }
    __syncthreads();
    // vertices with more lines than list entries: a warp walks the candidates in order and
    // keeps the first TRK2D_VERTEX_MAX_TRACKS whose raster contains the cell
    for (int k = w; k < nv; k += kVtxThreads / 32) {
        const trk2d_vertex &v = slots[(size_t)e * K.max_vertices + k];
        if (v.votes <= TRK2D_VERTEX_MAX_TRACKS)
            continue;
        int32_t *t = slot_tracks + ((int64_t)e * K.max_vertices + k) * TRK2D_VERTEX_MAX_TRACKS;
        int n = 0;
        for (int64_t i0 = 0; i0 < nc && n < TRK2D_VERTEX_MAX_TRACKS; i0 += 32) {
            const int64_t i = i0 + lane;
            bool has = false;
            if (i < nc) {
                has = cand[c0 + i].votes >= K.v_min_votes &&
                      vtx_raster_has(K, geom[c0 + i], (int)v.cell);
            }
            const unsigned m = __ballot_sync(kFull, has);
            const int at = n + __popc(m & lanemask_lt());
            if (has && at < TRK2D_VERTEX_MAX_TRACKS)
                t[at] = (int32_t)(c0 + i);
            n += __popc(m);
        }
        if (lane == 0)
            s_ntr[k] = n < TRK2D_VERTEX_MAX_TRACKS ? n : TRK2D_VERTEX_MAX_TRACKS;
    }
    __syncthreads();
    // ascending track lists (one thread per vertex: at most 64 entries)
    for (int k = threadIdx.x; k < nv; k += kVtxThreads) {
        const int n = min(s_ntr[k], TRK2D_VERTEX_MAX_TRACKS);
        int32_t *t = slot_tracks + ((int64_t)e * K.max_vertices + k) * TRK2D_VERTEX_MAX_TRACKS;
        for (int i = 1; i < n; ++i) {
            const int32_t x = t[i];
            int j = i - 1;
            while (j >= 0 && t[j] > x) {
                t[j + 1] = t[j];
                --j;
            }
            t[j + 1] = x;
        }
        slots[(size_t)e * K.max_vertices + k].n_tracks = n;
    }
    if (threadIdx.x == 0) {
        count[e] = nv;
        if (total > K.max_vertices)
            atomicOr(overflow, 1);
    }
}

struct CountVal {
    const int32_t *c;
    __device__ int64_t operator()(int64_t i) const { return c[i]; }
};

__global__ void k_h2_vertex_pack(const trk2d_vertex *slots, const int32_t *count,
                                 const int64_t *voff, int n_events, int max_vertices,
                                 trk2d_vertex *out)
{
    const int64_t total = (int64_t)n_events * max_vertices;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(q / max_vertices), k = (int)(q - (int64_t)e * max_vertices);
        if (k < count[e])
            out[voff[e] + k] = slots[q];
    }
}

__global__ void k_h2_vertex_total(const int64_t *voff, const int32_t *count, int n_events,
                                  int64_t *voff_out)
{
    if (blockIdx.x == 0 && threadIdx.x == 0)
        voff_out[n_events] = voff[n_events - 1] + count[n_events - 1];
}

}  // namespace trk

using namespace trk;

struct trk2d_ctx {
    trk2d_config cfg;
    H2Const K;
    int device = 0, n_sm = 0, S = 0;
    size_t smem = 0;
    float2 *d_coef = nullptr;
    int32_t *d_hist = nullptr;
    uint32_t *d_cbits = nullptr, *d_wprefix = nullptr;
    int64_t *d_bsum = nullptr, *d_hit_off = nullptr, *d_cand_off = nullptr;
    int64_t bsum_cap = 0;
    trk2d_candidate *d_cand = nullptr;
    int32_t *d_hit_ids = nullptr;
    H2Counters *d_ctr = nullptr, *h_ctr = nullptr;
    int64_t *h_cand_off = nullptr;
    trk2d_vertex *d_vslots = nullptr, *d_vertices = nullptr;
    VtxLine *d_geom = nullptr;
    int64_t geom_cap = 0;
    int32_t *d_vtracks = nullptr, *d_vcount = nullptr, *d_voverflow = nullptr;
    int64_t *d_voff = nullptr, *h_voff = nullptr;
    int32_t h_voverflow = 0;
    cudaStream_t own = nullptr;
    cudaEvent_t ev0 = nullptr, ev_v0 = nullptr, ev_v1 = nullptr, ev1 = nullptr;
    int last_n_events = 0;
    std::string err;
};

namespace {
thread_local std::string g_err;      // the calling thread's last trk2d_create failure

void set_create_error(const std::string &m) { g_err = m; }

int fail2(trk2d_ctx *h, int code, const std::string &m)
{
    if (h)
        h->err = m;
    return code;
}

void free2(trk2d_ctx *h)
{
    void *dev[] = {h->d_coef,    h->d_hist,     h->d_cbits,    h->d_wprefix,  h->d_bsum,
                   h->d_hit_off, h->d_cand_off, h->d_cand,     h->d_hit_ids,  h->d_ctr,
                   h->d_vslots,  h->d_vertices, h->d_vtracks,  h->d_vcount,   h->d_voverflow,
                   h->d_voff,    h->d_geom};
    for (void *p : dev)
        if (p)
            cudaFree(p);
    if (h->h_ctr)
        cudaFreeHost(h->h_ctr);
    if (h->h_cand_off)
        cudaFreeHost(h->h_cand_off);
    if (h->h_voff)
        cudaFreeHost(h->h_voff);
    cudaEvent_t evs[] = {h->ev0, h->ev_v0, h->ev_v1, h->ev1};
    for (cudaEvent_t e : evs)
        if (e)
            cudaEventDestroy(e);
    if (h->own)
        cudaStreamDestroy(h->own);
    delete h;
}

template <class T>
cudaError_t dalloc2(T **p, size_t n)
{
    return cudaMalloc((void **)p, sizeof(T) * (n > 0 ? n : 1));
}
}  // namespace

#define H2_CUDA(h, call)                                                                       \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail2(h, TRK_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// The vertex stage over candidates cand (cand_off[e] .. cand_off[e + 1] per event): the
// kernel, the per-event counts' scan, the dense copy, and the copies of the offsets and the
// overflow flag to the host.
static int enqueue_vertices(trk2d_ctx *h, const trk2d_candidate *cand, const int64_t *cand_off,
                            const unsigned long long *n_cand_dev, int64_t cand_cap, int n_events,
                            cudaStream_t s)
{
    const H2Const &K = h->K;
    if (cand_cap > h->geom_cap) {           // only the standalone entry can need more
        if (h->d_geom)
            cudaFree(h->d_geom);
        h->d_geom = nullptr;
        h->geom_cap = 0;
        H2_CUDA(h, dalloc2(&h->d_geom, (size_t)cand_cap));
        h->geom_cap = cand_cap;
    }
    H2_CUDA(h, cudaMemsetAsync(h->d_voverflow, 0, sizeof(int32_t), s));
    k_h2_cand_geom<<<h->n_sm * 4, 256, 0, s>>>(K, cand, n_cand_dev, cand_cap, cand_cap, h->d_geom);
    H2_CUDA(h, cudaGetLastError());
    k_h2_vertex<<<n_events, kVtxThreads, sizeof(int32_t) * K.vb * K.vb, s>>>(
        K, cand, h->d_geom, cand_off, cand_cap, h->d_vslots, h->d_vtracks, h->d_vcount,
        h->d_voverflow);
    H2_CUDA(h, cudaGetLastError());
    H2_CUDA(h, scan_exclusive(CountVal{h->d_vcount}, nullptr, n_events, n_events, h->d_voff,
                              h->d_bsum, nullptr, s));
    k_h2_vertex_total<<<1, 32, 0, s>>>(h->d_voff, h->d_vcount, n_events, h->d_voff);
    k_h2_vertex_pack<<<h->n_sm * 2, 256, 0, s>>>(h->d_vslots, h->d_vcount, h->d_voff, n_events,
                                                 K.max_vertices, h->d_vertices);
    H2_CUDA(h, cudaGetLastError());
    H2_CUDA(h, cudaMemcpyAsync(h->h_voff, h->d_voff, sizeof(int64_t) * (n_events + 1),
                               cudaMemcpyDeviceToHost, s));
    H2_CUDA(h, cudaMemcpyAsync(&h->h_voverflow, h->d_voverflow, sizeof(int32_t),
                               cudaMemcpyDeviceToHost, s));
    return TRK_OK;
}

extern "C" int trk2d_create(trk2d_ctx **out, const trk2d_config *c, int32_t device)
{
    if (!out || !c) {
        set_create_error("null argument");
        return TRK_ERR_INVALID;
    }
    *out = nullptr;
    std::string why;
    if (c->kind != TRK2D_STRAIGHT && c->kind != TRK2D_CURVED_IP)
        why = "kind must be TRK2D_STRAIGHT or TRK2D_CURVED_IP";
    else if (c->n_cols < 3 || c->n_cols > 65536 || c->n_rows < 2 || c->n_rows > 16384)
        why = "n_cols must be in 3..65536 and n_rows in 2..16384";
    else if (!(c->hi > c->lo) || !std::isfinite(c->lo) || !std::isfinite(c->hi))
        why = "row range must be finite with hi > lo";
    else if (c->kind == TRK2D_STRAIGHT && c->lo != -c->hi)
        why = "the rho range of TRK2D_STRAIGHT must be symmetric (lo = -hi)";
    else if (c->kind == TRK2D_CURVED_IP && !(c->b_tesla > 0.0))
        why = "TRK2D_CURVED_IP needs b_tesla > 0";
    else if (c->threshold < 1 || c->max_events < 1 || c->max_hits < 1 || c->cand_capacity < 1 ||
             c->hit_capacity < 1)
        why = "threshold, max_events, max_hits and the capacities must be >= 1";
    else if (c->vertex_bins != 0 &&
             (c->kind != TRK2D_STRAIGHT || c->vertex_bins < 3 || c->vertex_bins > 128 ||
              c->vertex_threshold < 1 || c->max_vertices < 1 || c->max_vertices > 1024 ||
              !(c->vertex_range > 0.0)))
        why = "vertices need TRK2D_STRAIGHT, vertex_bins in 3..128, vertex_threshold >= 1, "
              "max_vertices in 1..1024 and vertex_range > 0";
    if (!why.empty()) {
        set_create_error(why);
        return TRK_ERR_INVALID;
    }
    trk2d_ctx *h = new trk2d_ctx();
    h->cfg = *c;
    h->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        set_create_error("cudaSetDevice failed");
        free2(h);
        return TRK_ERR_CUDA;
    }
    H2Const &K = h->K;
    K.kind = c->kind;
    K.n_cols = c->n_cols;
    K.n_rows = c->n_rows;
    K.threshold = c->threshold;
    K.lo = (float)c->lo;
    K.hi = (float)c->hi;
    K.inv_w = (float)(c->n_rows / (c->hi - c->lo));
    K.kB = (float)(0.299792458e-2 * c->b_tesla);
    const double col_lo = c->kind == TRK2D_STRAIGHT ? 0.0 : -M_PI;
    const double col_w = (c->kind == TRK2D_STRAIGHT ? M_PI : 2.0 * M_PI) / c->n_cols;
    K.col_lo = (float)col_lo;
    K.col_w = (float)col_w;
    K.col_lo_d = col_lo;
    K.col_w_d = col_w;
    K.lo_d = c->lo;
    K.w_d = (c->hi - c->lo) / c->n_rows;
    K.vb = c->vertex_bins;
    K.v_threshold = c->vertex_threshold;
    K.v_min_votes = c->vertex_min_votes;
    K.max_vertices = c->max_vertices > 0 ? c->max_vertices : 1;
    K.v_range = c->vertex_range;
    K.v_w = c->vertex_bins > 0 ? 2.0 * c->vertex_range / c->vertex_bins : 1.0;
    K.nbins = (uint32_t)c->n_cols * (uint32_t)c->n_rows;
    K.W = (K.nbins + 31) / 32;
    if ((uint64_t)c->n_cols * (uint64_t)c->n_rows > (1ull << 31)) {
        set_create_error("n_cols x n_rows too large");
        free2(h);
        return TRK_ERR_INVALID;
    }
    // slab width: the shared histogram (S + 2 columns) within 96 KB
    const int per_col = (int)sizeof(int32_t) * c->n_rows;
    h->S = (96 * 1024) / per_col - 2;
    if (h->S < 1) {
        set_create_error("n_rows too large for the shared-memory slab");
        free2(h);
        return TRK_ERR_INVALID;
    }
    h->S = h->S < c->n_cols ? h->S : c->n_cols;
    h->smem = (size_t)(h->S + 2) * per_col;
    // column coefficients in FP64, rounded once to FP32
    float2 *coef = new float2[c->n_cols];
    for (int i = 0; i < c->n_cols; ++i) {
        const double a = col_lo + (i + 0.5) * col_w;
        coef[i] = c->kind == TRK2D_STRAIGHT ? make_float2((float)std::cos(a), (float)std::sin(a))
                                            : make_float2((float)std::sin(a), (float)-std::cos(a));
    }
    const int64_t E = c->max_events;
    const int64_t n_words = E * K.W;
    h->bsum_cap = (std::max<int64_t>(n_words, c->cand_capacity) + kScanBlock - 1) / kScanBlock + 1;
    bool ok = dalloc2(&h->d_coef, (size_t)c->n_cols) == cudaSuccess &&
              dalloc2(&h->d_hist, (size_t)(E * K.nbins)) == cudaSuccess &&
              dalloc2(&h->d_cbits, (size_t)n_words) == cudaSuccess &&
              dalloc2(&h->d_wprefix, (size_t)n_words) == cudaSuccess &&
              dalloc2(&h->d_bsum, (size_t)h->bsum_cap) == cudaSuccess &&
              dalloc2(&h->d_hit_off, (size_t)c->cand_capacity) == cudaSuccess &&
              dalloc2(&h->d_cand_off, (size_t)(E + 1)) == cudaSuccess &&
              dalloc2(&h->d_cand, (size_t)c->cand_capacity) == cudaSuccess &&
              dalloc2(&h->d_hit_ids, (size_t)c->hit_capacity) == cudaSuccess &&
              dalloc2(&h->d_ctr, 1) == cudaSuccess &&
              cudaMallocHost((void **)&h->h_ctr, sizeof(H2Counters)) == cudaSuccess &&
              cudaMallocHost((void **)&h->h_cand_off, sizeof(int64_t) * (size_t)(E + 1)) ==
                  cudaSuccess;
    ok = ok && cudaMemcpy(h->d_coef, coef, sizeof(float2) * c->n_cols, cudaMemcpyHostToDevice) ==
                   cudaSuccess;
    delete[] coef;
    if (ok && c->vertex_bins > 0) {
        const size_t slots = (size_t)E * K.max_vertices;
        ok = dalloc2(&h->d_vslots, slots) == cudaSuccess &&
             dalloc2(&h->d_vertices, slots) == cudaSuccess &&
             dalloc2(&h->d_vtracks, slots * TRK2D_VERTEX_MAX_TRACKS) == cudaSuccess &&
             dalloc2(&h->d_vcount, (size_t)E) == cudaSuccess &&
             dalloc2(&h->d_voverflow, 1) == cudaSuccess &&
             dalloc2(&h->d_voff, (size_t)E + 1) == cudaSuccess &&
             dalloc2(&h->d_geom, (size_t)c->cand_capacity) == cudaSuccess &&
             cudaMallocHost((void **)&h->h_voff, sizeof(int64_t) * (size_t)(E + 1)) == cudaSuccess &&
             (h->geom_cap = c->cand_capacity) > 0 &&
             cudaFuncSetAttribute(k_h2_vertex, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(int32_t) * c->vertex_bins * c->vertex_bins)) ==
                 cudaSuccess;
    }
    ok = ok && cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreate(&h->ev0) == cudaSuccess && cudaEventCreate(&h->ev_v0) == cudaSuccess &&
         cudaEventCreate(&h->ev_v1) == cudaSuccess && cudaEventCreate(&h->ev1) == cudaSuccess &&
         cudaFuncSetAttribute(k_h2_vote_peak, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)h->smem) == cudaSuccess;
    if (!ok) {
        set_create_error("device allocation or set-up failed");
        free2(h);
        return TRK_ERR_NOMEM;
    }
    *out = h;
    return TRK_OK;
}

extern "C" int trk2d_reconstruct(trk2d_ctx *h, const trk_hit *hits, int64_t n_hits,
                                 const int64_t *event_offsets, int32_t n_events,
                                 trk2d_result *out, void *stream)
{
    if (!h)
        return TRK_ERR_INVALID;
    if (!event_offsets || (n_hits > 0 && !hits) || n_hits < 0 || n_hits > h->cfg.max_hits ||
        n_events < 1 || n_events > h->cfg.max_events)
        return fail2(h, TRK_ERR_INVALID, "bad arguments (null pointer, or more hits or events "
                                         "than configured)");
    H2_CUDA(h, cudaSetDevice(h->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : h->own;
    const H2Const &K = h->K;
    const int64_t n_words = (int64_t)n_events * K.W;
    H2Counters *ctr = h->d_ctr;
    H2_CUDA(h, cudaEventRecord(h->ev0, s));
    H2_CUDA(h, cudaMemsetAsync(ctr, 0, sizeof(H2Counters), s));
    H2_CUDA(h, cudaMemsetAsync(h->d_cbits, 0, sizeof(uint32_t) * (size_t)n_words, s));
    const dim3 grid((unsigned)((K.n_cols + h->S - 1) / h->S), (unsigned)n_events);
    H2_CUDA(h, cudaEventRecord(h->ev_v0, s));
    k_h2_vote_peak<<<grid, kH2Threads, h->smem, s>>>(K, hits, event_offsets, h->d_coef, h->S,
                                                     h->d_hist, h->d_cbits);
    H2_CUDA(h, cudaGetLastError());
    H2_CUDA(h, cudaEventRecord(h->ev_v1, s));
    H2_CUDA(h, scan_exclusive(PopcVal{h->d_cbits}, nullptr, n_words, n_words, h->d_wprefix,
                              h->d_bsum, &ctr->n_cand, s));
    k_h2_emit<<<h->n_sm * 4, 256, 0, s>>>(K, h->d_cbits, h->d_wprefix, n_words, h->d_hist,
                                          h->d_cand, h->cfg.cand_capacity);
    H2_CUDA(h, cudaGetLastError());
    H2_CUDA(h, scan_exclusive(H2CandVotes{h->d_cand}, &ctr->n_cand, 0, h->cfg.cand_capacity,
                              h->d_hit_off, h->d_bsum, &ctr->n_hit, s));
    k_h2_set_off<<<h->n_sm * 2, 256, 0, s>>>(h->d_cand, h->d_hit_off, &ctr->n_cand,
                                             h->cfg.cand_capacity);
    H2_CUDA(h, cudaGetLastError());
    k_h2_assign<<<h->n_sm * 8, 256, 0, s>>>(K, hits, event_offsets, h->d_coef, h->d_cand,
                                            &ctr->n_cand, h->cfg.cand_capacity, h->d_hit_ids,
                                            h->cfg.hit_capacity);
    H2_CUDA(h, cudaGetLastError());
    k_h2_cand_off<<<(n_events + 1 + 255) / 256, 256, 0, s>>>(h->d_wprefix, K.W, n_events,
                                                             &ctr->n_cand, h->d_cand_off);
    H2_CUDA(h, cudaGetLastError());
    if (K.vb > 0) {
        const int rc = enqueue_vertices(h, h->d_cand, h->d_cand_off, &h->d_ctr->n_cand,
                                        h->cfg.cand_capacity, n_events, s);
        if (rc != TRK_OK)
            return rc;
    }
    H2_CUDA(h, cudaMemcpyAsync(h->h_ctr, ctr, sizeof(H2Counters), cudaMemcpyDeviceToHost, s));
    H2_CUDA(h, cudaMemcpyAsync(h->h_cand_off, h->d_cand_off, sizeof(int64_t) * (n_events + 1),
                               cudaMemcpyDeviceToHost, s));
    H2_CUDA(h, cudaEventRecord(h->ev1, s));
    H2_CUDA(h, cudaStreamSynchronize(s));
    h->last_n_events = n_events;
    const bool over = h->h_ctr->n_cand > (unsigned long long)h->cfg.cand_capacity ||
                      h->h_ctr->n_hit > (unsigned long long)h->cfg.hit_capacity;
    if (out) {
        out->n_events = n_events;
        out->n_candidates = over ? 0 : (int64_t)h->h_ctr->n_cand;
        out->n_hit_ids = over ? 0 : (int64_t)h->h_ctr->n_hit;
        out->cand_off = h->h_cand_off;
        out->d_cand = h->d_cand;
        out->d_hit_ids = h->d_hit_ids;
        out->n_vertices = (K.vb > 0 && !over) ? h->h_voff[n_events] : 0;
        out->vertex_off = K.vb > 0 ? h->h_voff : nullptr;
        out->d_vertices = h->d_vertices;
        out->d_vertex_tracks = h->d_vtracks;
        out->vertex_overflow = K.vb > 0 ? h->h_voverflow : 0;
    }
    if (over)
        return fail2(h, TRK_ERR_CAPACITY, "candidate or hit capacity exceeded");
    return TRK_OK;
}

extern "C" int trk2d_find_vertices(trk2d_ctx *h, const trk2d_candidate *cand,
                                   const int64_t *cand_off, int32_t n_events, trk2d_result *out,
                                   void *stream)
{
    if (!h)
        return TRK_ERR_INVALID;
    if (h->K.vb <= 0)
        return fail2(h, TRK_ERR_INVALID, "the handle was created without vertex_bins");
    if (!cand || !cand_off || n_events < 1 || n_events > h->cfg.max_events)
        return fail2(h, TRK_ERR_INVALID, "bad arguments (null pointer or event count)");
    H2_CUDA(h, cudaSetDevice(h->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : h->own;
    int64_t last = 0;
    H2_CUDA(h, cudaMemcpyAsync(&last, cand_off + n_events, sizeof(int64_t),
                               cudaMemcpyDeviceToHost, s));
    H2_CUDA(h, cudaStreamSynchronize(s));
    if (last < 0)
        return fail2(h, TRK_ERR_INVALID, "bad candidate offsets");
    const int rc = enqueue_vertices(h, cand, cand_off, nullptr, last, n_events, s);
    if (rc != TRK_OK)
        return rc;
    H2_CUDA(h, cudaStreamSynchronize(s));
    if (out) {
        std::memset(out, 0, sizeof(*out));
        out->n_events = n_events;
        out->n_vertices = h->h_voff[n_events];
        out->vertex_off = h->h_voff;
        out->d_vertices = h->d_vertices;
        out->d_vertex_tracks = h->d_vtracks;
        out->vertex_overflow = h->h_voverflow;
    }
    return TRK_OK;
}

extern "C" int trk2d_get_histogram(trk2d_ctx *h, int32_t event, int32_t *dst, void *stream)
{
    if (!h || !dst)
        return TRK_ERR_INVALID;
    if (event < 0 || event >= h->last_n_events)
        return fail2(h, TRK_ERR_INVALID, "event out of range of the last call");
    cudaStream_t s = stream ? (cudaStream_t)stream : h->own;
    H2_CUDA(h, cudaMemcpyAsync(dst, h->d_hist + (size_t)event * h->K.nbins,
                               sizeof(int32_t) * h->K.nbins, cudaMemcpyDeviceToDevice, s));
    H2_CUDA(h, cudaStreamSynchronize(s));
    return TRK_OK;
}

extern "C" int trk2d_last_ms(trk2d_ctx *h, float *vote_peak_ms, float *total_ms)
{
    if (!h)
        return TRK_ERR_INVALID;
    if (vote_peak_ms)
        H2_CUDA(h, cudaEventElapsedTime(vote_peak_ms, h->ev_v0, h->ev_v1));
    if (total_ms)
        H2_CUDA(h, cudaEventElapsedTime(total_ms, h->ev0, h->ev1));
    return TRK_OK;
}

extern "C" const char *trk2d_last_error(const trk2d_ctx *h)
{
    return h ? h->err.c_str() : g_err.c_str();
}

extern "C" int trk2d_destroy(trk2d_ctx *h)
{
    if (h)
        free2(h);
    return TRK_OK;
}
