// Triplet enumeration + helix fit + vote: the hot loop (paper Sec. 7 and Fig. 3: every
// hit combination votes into the parameter space; Sec. 8: concurrent votes race, so the
// accumulation is done with atomics).
//
// Persistent blocks pull work items (event, layer triple, tile of inner x middle hits)
// from a device counter.  Each thread owns one (inner, middle) hit pair and walks the
// outer-layer hits, staged in shared memory, through three stages:
//   A  curvature prefilter (14 FP32 ops): a superset test of the q/pT range;
//   B  the FP32 fit: the transverse part (q/pT, d0, with their exact range tests), then
//      for the triplets in range the longitudinal part (cot, z0);
//   C  phi0, the five bin indices, the histogram atomic and the vote-list record.
// Between stages the surviving items are compacted into per-warp ring queues in shared
// memory (stage B's accepted fits with their parameters) so that every stage runs with
// all 32 lanes busy.  Fits that the FP32 path cannot resolve (near-collinear, degenerate)
// are recomputed in FP64.
#pragma once

#include "trk_common.cuh"

namespace trk {



struct Q1 {                       // a (pair, outer hit) item
    float x, y, z;
    uint32_t code;                // vote_code(i in tile, j in tile, k in layer c)
};

struct __align__(16) Q2 {         // an accepted FP32 fit: everything but phi0
    float cx, cy, sgn, qopt;
    float d0, cot, z0;
    uint32_t code;
};

constexpr int kRing = 64;

template <int NW>
struct WarpQueues {
    Q1 q1[NW][kRing];             // survivors of the curvature prefilter
    Q2 q2[NW][kRing];             // triplets whose FP32 fit is in range
    uint64_t stg[NW][kRing];      // votes waiting for a 32-slot chunk
    int4 loc;                     // chunk_loc of the current work item
};

// Per-warp queue state, identical in every lane.
struct WarpState {
    int h1, n1, h2, n2, hs, ns;
    int64_t res_chunk;            // next reserved chunk index
    int res_left;                 // reserved chunks left
    uint32_t n_fit, n_exact, n_fp64, n_votes;   // per lane; below 2^32 for any call
                                                 // under 6e14 triplets
};

template <int NW>
__device__ __forceinline__ void flush_votes(const VoteArgs &A, WarpQueues<NW> &Q, WarpState &ws,
                                            int w, int lane, int count, int item, int event)
{
    if (ws.res_left == 0) {
        long long base = 0;
        if (lane == 0)
            base = (long long)atomicAdd(&A.ctr->n_chunks, 4ull);
        ws.res_chunk = __shfl_sync(kFull, base, 0);
        ws.res_left = 4;
    }
    const int64_t cid = ws.res_chunk;
    ws.res_chunk++;
    ws.res_left--;
    if (cid < A.chunk_cap) {
        if (lane < count) {
            const uint64_t v = Q.stg[w][(ws.hs + lane) & (kRing - 1)];
            A.vote_bin[cid * kWarp + lane] = (uint32_t)v;
            A.vote_code[cid * kWarp + lane] = (uint32_t)(v >> 32);
        }
        if (lane == 0) {
            A.chunk_item[cid] = item;
            A.chunk_count[cid] = count;
            A.chunk_event[cid] = event;
            A.chunk_loc[cid] = Q.loc;
        }
    } else if (lane == 0) {
        atomicOr(&A.status[event], TRK_EV_VOTE_OVERFLOW);
    }
    ws.hs = (ws.hs + count) & (kRing - 1);
    ws.ns -= count;
    ws.n_votes += count;
}

// Warp-uniform: lanes with `has` vote for `bin` with `code`.
template <int NW>
__device__ __forceinline__ void push_votes(const VoteArgs &A, WarpQueues<NW> &Q, WarpState &ws,
                                           int w, int lane, bool has, uint32_t bin, uint32_t code,
                                           int32_t *hist_e, int item, int event)
{
    const unsigned m = __ballot_sync(kFull, has);
    if (has) {
        atomicAdd(hist_e + bin, 1);
        const int pos = (ws.hs + ws.ns + __popc(m & lanemask_lt())) & (kRing - 1);
        Q.stg[w][pos] = (uint64_t)bin | ((uint64_t)code << 32);
    }
    ws.ns += __popc(m);
    if (ws.ns >= kWarp) {
        __syncwarp();
        flush_votes(A, Q, ws, w, lane, kWarp, item, event);
        __syncwarp();
    }
}

// phi0, bins and vote on up to 32 queued accepted fits.
template <int NW, int TJ>
__device__ __forceinline__ void drain2(const VoteArgs &A, WarpQueues<NW> &Q, WarpState &ws, int w,
                                       int lane, int count, int32_t *hist_e, int item, int event)
{
    __syncwarp();
    bool has = false;
    uint32_t bin = 0, code = 0;
    if (lane < count) {
        const Q2 e = Q.q2[w][(ws.h2 + lane) & (kRing - 1)];
        FitB r;
        r.cx = e.cx;
        r.cy = e.cy;
        r.sgn = e.sgn;
        r.qopt = e.qopt;
        r.d0 = e.d0;
        r.cot = e.cot;
        r.z0 = e.z0;
        code = e.code;
        float phi0;
        has = fit_stage_c(r, A.C, phi0, bin);
    }
    ws.h2 = (ws.h2 + count) & (kRing - 1);
    ws.n2 -= count;
    __syncwarp();
    push_votes(A, Q, ws, w, lane, has, bin, code, hist_e, item, event);
}

// The FP32 fit on up to 32 queued prefilter survivors: the transverse part, then the
// longitudinal part for those whose q/pT and d0 are in range.  Accepted fits go to the
// second queue; FP64 recomputations (rare) vote here.
template <int NW, int TJ>
__device__ __forceinline__ void drain1(const VoteArgs &A, WarpQueues<NW> &Q, WarpState &ws, int w,
                                       int lane, int count, const float4 *s_i, const float4 *s_j,
                                       int32_t *hist_e, int item, int event)
{
    __syncwarp();
    bool keep = false, f64 = false;
    Q2 out;
    // the item's slot keeps it until the queue refills after this drain, so the FP64 path
    // reads it again instead of holding the hits in registers through the fit
    const int slot = (ws.h1 + lane) & (kRing - 1);
    if (lane < count) {
        const Q1 e = Q.q1[w][slot];
        out.code = e.code;
        const float4 p1 = s_i[code_i(e.code)];
        const float4 p2 = s_j[code_j(e.code)];
        const float4 p3 = make_float4(e.x, e.y, e.z, 0.0f);
        // both parts run on every lane (85 % of the transverse fits pass, so a warp would
        // run the longitudinal part anyway); the statuses decide what is kept
        Trans t;
        const int st = fit_transverse(p1, p2, p3, A.C, t);
        const int sl = fit_longitudinal(p1, p2, p3, t, A.C, out.cot, out.z0);
        ws.n_fit++;
        ws.n_exact += (st == kPass);
        keep = st == kPass && sl == kPass;
        f64 = st == kNeedFp64 || (st == kPass && sl == kNeedFp64);
        out.cx = t.cx;
        out.cy = t.cy;
        out.sgn = t.sgn;
        out.qopt = t.qopt;
        out.d0 = t.d0;
    }
    ws.h1 = (ws.h1 + count) & (kRing - 1);
    ws.n1 -= count;
    // FP64 recomputation of the near-collinear / degenerate ones (rare)
    if (__any_sync(kFull, f64)) {
        bool has = false;
        uint32_t bin = 0;
        if (f64) {
            const Q1 e = Q.q1[w][slot];
            const float4 p1 = s_i[code_i(e.code)];
            const float4 p2 = s_j[code_j(e.code)];
            const float4 p3 = make_float4(e.x, e.y, e.z, 0.0f);
            double par[5];
            has = (fit_f64(p1, p2, p3, A.C, par, bin) == kFit64Accepted);
            ws.n_fp64++;
        }
        __syncwarp();
        push_votes(A, Q, ws, w, lane, has, bin, out.code, hist_e, item, event);
    }
    __syncwarp();
    const unsigned m = __ballot_sync(kFull, keep);
    if (keep) {
        const int pos = (ws.h2 + ws.n2 + __popc(m & lanemask_lt())) & (kRing - 1);
        Q.q2[w][pos] = out;
    }
    ws.n2 += __popc(m);
    if (ws.n2 >= kWarp)
        drain2<NW, TJ>(A, Q, ws, w, lane, kWarp, hist_e, item, event);
}

template <int TI, int TJ, int KC, int MINB>
__global__ void __launch_bounds__(TI *TJ, MINB) k_vote(VoteArgs A)
{
    constexpr int NT = TI * TJ;
    constexpr int NW = NT / kWarp;
    static_assert(TI <= 16 && TJ <= 16, "the vote code holds 4-bit tile positions");
    extern __shared__ __align__(16) unsigned char smem[];
    float4 *s_k = reinterpret_cast<float4 *>(smem);
    float4 *s_i = s_k + KC;
    float4 *s_j = s_i + TI;
    WarpQueues<NW> &Q = *reinterpret_cast<WarpQueues<NW> *>(s_j + TJ);
    __shared__ int64_t s_item;

    const int tid = threadIdx.x;
    const int w = tid >> 5, lane = tid & 31;
    const int n_events = A.args->n_events;
    const int T = A.geo->n_triples;
    const int L1 = A.geo->n_layers + 1;
    const int F = n_events * T;
    const int64_t n_items = A.item_off[F];

    WarpState ws;
    ws.h1 = ws.n1 = ws.h2 = ws.n2 = ws.hs = ws.ns = 0;
    ws.res_chunk = 0;
    ws.res_left = 0;
    ws.n_fit = ws.n_exact = ws.n_fp64 = ws.n_votes = 0;

    for (;;) {
        if (tid == 0)
            s_item = (int64_t)atomicAdd(&A.ctr->work_next, 1ull);
        __syncthreads();
        const int64_t item = s_item;
        __syncthreads();
        if (item >= n_items)
            break;
        const int f = upper_index(A.item_off, F, item);
        const int e = f / T, t = f - e * T;
        const int la = A.geo->triples[t][0], lb = A.geo->triples[t][1], lc = A.geo->triples[t][2];
        const int32_t *lo = A.lay_off + (size_t)e * L1;
        const int a0 = lo[la], na = lo[la + 1] - a0;
        const int b0 = lo[lb], nb = lo[lb + 1] - b0;
        const int c0 = lo[lc], nc = lo[lc + 1] - c0;
        const int64_t local = item - A.item_off[f];
        const int ntj = (nb + TJ - 1) / TJ;
        const int ti = (int)(local / ntj), tj = (int)(local - (int64_t)ti * ntj);
        const int i0 = ti * TI, j0 = tj * TJ;
        if (tid < TI)
            s_i[tid] = (i0 + tid < na) ? __ldg(A.packed + a0 + i0 + tid) : make_float4(0, 0, 0, 0);
        else if (tid < TI + TJ)
            s_j[tid - TI] = (j0 + tid - TI < nb) ? __ldg(A.packed + b0 + j0 + tid - TI)
                                                 : make_float4(0, 0, 0, 0);
        int32_t *hist_e = A.hist + (size_t)e * A.C.nbins;
        if (tid == 0)      // every warp is past the previous item's flushes (barriers above)
            Q.loc = make_int4(a0 + i0, b0 + j0, c0, (int)item);
        __syncthreads();

        const int pi = tid / TJ, pj = tid - (tid / TJ) * TJ;
        const bool valid = (i0 + pi < na) && (j0 + pj < nb);
        const float4 p1 = s_i[pi], p2 = s_j[pj];
        const float ux = p2.x - p1.x, uy = p2.y - p1.y;
        const float uu = fmaf(ux, ux, uy * uy);
        const float pre = A.C.pre_k2 * uu;
        const uint32_t pair_code = vote_code((uint32_t)pi, (uint32_t)pj, 0u);

        for (int kc = 0; kc < nc; kc += KC) {
            const int cnt = min(KC, nc - kc);
            for (int x = tid; x < cnt; x += NT)
                s_k[x] = __ldg(A.packed + c0 + kc + x);
            __syncthreads();
            for (int kk = 0; kk < cnt; ++kk) {
                const float4 p3 = s_k[kk];
                const float vx = p3.x - p1.x, vy = p3.y - p1.y;
                const float wx = p3.x - p2.x, wy = p3.y - p2.y;
                const float D = fmaf(ux, vy, -(uy * vx));
                const float vv = fmaf(vx, vx, vy * vy);
                const float ww = fmaf(wx, wx, wy * wy);
                const bool pass = valid && (D * D <= pre * (vv * ww));
                const unsigned m = __ballot_sync(kFull, pass);
                if (pass) {
                    const int pos = (ws.h1 + ws.n1 + __popc(m & lanemask_lt())) & (kRing - 1);
                    Q1 q;
                    q.x = p3.x;
                    q.y = p3.y;
                    q.z = p3.z;
                    q.code = pair_code | (uint32_t)(kc + kk);
                    Q.q1[w][pos] = q;
                }
                ws.n1 += __popc(m);
                if (ws.n1 >= kWarp)
                    drain1<NW, TJ>(A, Q, ws, w, lane, kWarp, s_i, s_j, hist_e, (int)item, e);
            }
            __syncthreads();
        }
        // end of the work item: drain everything (partial rounds)
        if (ws.n1 > 0)
            drain1<NW, TJ>(A, Q, ws, w, lane, ws.n1, s_i, s_j, hist_e, (int)item, e);
        while (ws.n2 > 0)
            drain2<NW, TJ>(A, Q, ws, w, lane, min(ws.n2, kWarp), hist_e, (int)item, e);
        if (ws.ns > 0) {
            __syncwarp();
            flush_votes(A, Q, ws, w, lane, ws.ns, (int)item, e);
        }
        __syncwarp();
    }
    // release reserved chunks that stayed empty
    for (int r = 0; r < ws.res_left; ++r) {
        const int64_t cid = ws.res_chunk + r;
        if (lane == 0 && cid < A.chunk_cap) {
            A.chunk_item[cid] = -1;
            A.chunk_count[cid] = 0;
        }
    }
    // statistics
    unsigned long long nf = ws.n_fit, nx = ws.n_exact, n64 = ws.n_fp64, nv = ws.n_votes;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nf += __shfl_xor_sync(kFull, nf, o);
        nx += __shfl_xor_sync(kFull, nx, o);
        n64 += __shfl_xor_sync(kFull, n64, o);
    }
    if (lane == 0) {
        atomicAdd(&A.ctr->n_fit, nf);
        atomicAdd(&A.ctr->n_exact, nx);
        if (n64)
            atomicAdd(&A.ctr->n_fp64, n64);
        atomicAdd(&A.ctr->n_votes, nv);
    }
}

// ---------------------------------------------------------------------------------------
// launch helpers for one instantiation (TI x TJ pairs per block, MINB blocks per SM)
// ---------------------------------------------------------------------------------------

template <int TI, int TJ, int KC, int MINB>
size_t vote_smem()
{
    return sizeof(float4) * (KC + TI + TJ) + sizeof(WarpQueues<TI * TJ / kWarp>);
}

template <int TI, int TJ, int KC, int MINB>
cudaError_t vote_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(k_vote<TI, TJ, KC, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)vote_smem<TI, TJ, KC, MINB>());
    if (e != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_vote<TI, TJ, KC, MINB>,
                                cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

template <int TI, int TJ, int KC, int MINB>
cudaError_t vote_launch(const VoteArgs &A, int grid, cudaStream_t s)
{
    k_vote<TI, TJ, KC, MINB><<<grid, TI * TJ, vote_smem<TI, TJ, KC, MINB>(), s>>>(A);
    return cudaGetLastError();
}

template <int TI, int TJ, int KC, int MINB>
cudaError_t vote_occ(int *blocks)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks, k_vote<TI, TJ, KC, MINB>, TI * TJ, vote_smem<TI, TJ, KC, MINB>());
}

// Dispatch of one occupancy level (blocks of 256 threads per SM) over the tiles.
#define TRK_VOTE_LEVEL_DISPATCH(LEVEL)                                                         \
    cudaError_t vote_dispatch_level##LEVEL(int op, int ti, int tj, const VoteArgs *A,          \
                                           int grid, cudaStream_t s, int *blocks)              \
    {                                                                                          \
        constexpr int KC = 768;                                                                \
        if (ti == 16 && tj == 16)                                                              \
            return op == 0 ? vote_prepare<16, 16, KC, LEVEL>()                                 \
                   : op == 1 ? vote_launch<16, 16, KC, LEVEL>(*A, grid, s)                     \
                             : vote_occ<16, 16, KC, LEVEL>(blocks);                            \
        if (ti == 8 && tj == 16)                                                               \
            return op == 0 ? vote_prepare<8, 16, KC, 2 * LEVEL>()                              \
                   : op == 1 ? vote_launch<8, 16, KC, 2 * LEVEL>(*A, grid, s)                  \
                             : vote_occ<8, 16, KC, 2 * LEVEL>(blocks);                         \
        if (ti == 16 && tj == 8)                                                               \
            return op == 0 ? vote_prepare<16, 8, KC, 2 * LEVEL>()                              \
                   : op == 1 ? vote_launch<16, 8, KC, 2 * LEVEL>(*A, grid, s)                  \
                             : vote_occ<16, 8, KC, 2 * LEVEL>(blocks);                         \
        if (ti == 8 && tj == 8)                                                                \
            return op == 0 ? vote_prepare<8, 8, KC, 4 * LEVEL>()                               \
                   : op == 1 ? vote_launch<8, 8, KC, 4 * LEVEL>(*A, grid, s)                   \
                             : vote_occ<8, 8, KC, 4 * LEVEL>(blocks);                          \
        if (ti == 4 && tj == 16)                                                               \
            return op == 0 ? vote_prepare<4, 16, KC, 4 * LEVEL>()                              \
                   : op == 1 ? vote_launch<4, 16, KC, 4 * LEVEL>(*A, grid, s)                  \
                             : vote_occ<4, 16, KC, 4 * LEVEL>(blocks);                         \
        /* one-warp blocks: no block-wide barrier waits on other warps; 8 LEVEL blocks of */ \
        /* 32 threads per SM, outer hits staged 128 at a time to fit the shared memory    */ \
        if (ti == 8 && tj == 4)                                                                \
            return op == 0 ? vote_prepare<8, 4, 128, 8 * LEVEL>()                              \
                   : op == 1 ? vote_launch<8, 4, 128, 8 * LEVEL>(*A, grid, s)                  \
                             : vote_occ<8, 4, 128, 8 * LEVEL>(blocks);                         \
        if (ti == 4 && tj == 8)                                                                \
            return op == 0 ? vote_prepare<4, 8, 128, 8 * LEVEL>()                              \
                   : op == 1 ? vote_launch<4, 8, 128, 8 * LEVEL>(*A, grid, s)                  \
                             : vote_occ<4, 8, 128, 8 * LEVEL>(blocks);                         \
        return cudaErrorInvalidValue;                                                          \
    }

}  // namespace trk
