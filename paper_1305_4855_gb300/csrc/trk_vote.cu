// Triplet fit kernel for explicit triplets, and dispatch of the vote kernel over its
// occupancy levels (each level is instantiated in its own translation unit so that the
// big kernel compiles in parallel).
#include "trk_vote_kernel.cuh"

namespace trk {

cudaError_t vote_dispatch_level2(int op, int ti, int tj, const VoteArgs *A, int grid,
                                 cudaStream_t s, int *blocks);
cudaError_t vote_dispatch_level3(int op, int ti, int tj, const VoteArgs *A, int grid,
                                 cudaStream_t s, int *blocks);
cudaError_t vote_dispatch_level4(int op, int ti, int tj, const VoteArgs *A, int grid,
                                 cudaStream_t s, int *blocks);

// One-shot fit of explicit triplets with the vote kernel's arithmetic.
__global__ void k_fit_triplets(const trk_hit *hits, int64_t n_hits, const int32_t *ijk, int64_t n,
                               FitConst C, float *params, uint32_t *bins, int32_t *flags)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t ia = ijk[3 * t], ib = ijk[3 * t + 1], ic = ijk[3 * t + 2];
        if (ia < 0 || ib < 0 || ic < 0 || ia >= n_hits || ib >= n_hits || ic >= n_hits) {
            flags[t] = 8;
            continue;
        }
        const trk_hit a = hits[ia], b = hits[ib], c = hits[ic];
        const float4 p1 = make_float4(a.x, a.y, a.z, 0), p2 = make_float4(b.x, b.y, b.z, 0),
                     p3 = make_float4(c.x, c.y, c.z, 0);
        float par[5];
        uint32_t bin = 0;
        int fl = 0;
        // parameters always evaluated fully (the range checks only gate the vote)
        FitConst Cw = C;
        for (int k = 0; k < 5; ++k) {
            Cw.lo[k] = -INFINITY;
            Cw.hi[k] = INFINITY;
        }
        FitB r;
        const int st = fit_stage_b(p1, p2, p3, Cw, r);
        if (st == kPass) {
            float phi0 = atan2_poly(-r.sgn * r.cx, r.sgn * r.cy);
            par[0] = phi0;
            par[1] = r.qopt;
            par[2] = r.d0;
            par[3] = r.cot;
            par[4] = r.z0;
            FitB rr = r;
            float ph;
            if (fit_stage_b(p1, p2, p3, C, rr) == kPass && fit_stage_c(rr, C, ph, bin))
                fl |= 1;
        } else {
            double pd[5];
            const int r64 = fit_f64(p1, p2, p3, C, pd, bin);
            fl |= 2;
            if (r64 == kFit64Degenerate) {
                fl |= 4;
                for (int k = 0; k < 5; ++k)
                    par[k] = NAN;
            } else {
                for (int k = 0; k < 5; ++k)
                    par[k] = (float)pd[k];
                if (r64 == kFit64Accepted)
                    fl |= 1;
            }
        }
        for (int k = 0; k < 5; ++k)
            params[5 * t + k] = par[k];
        bins[t] = bin;
        flags[t] = fl;
    }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------

static cudaError_t vote_dispatch(int op, int ti, int tj, int level, const VoteArgs *A, int grid,
                                 cudaStream_t s, int *blocks)
{
    switch (level) {
    case 2:
        return vote_dispatch_level2(op, ti, tj, A, grid, s, blocks);
    case 3:
        return vote_dispatch_level3(op, ti, tj, A, grid, s, blocks);
    case 4:
        return vote_dispatch_level4(op, ti, tj, A, grid, s, blocks);
    default:
        return cudaErrorInvalidValue;
    }
}

bool vote_tile_supported(int ti, int tj)
{
    return (ti == 16 && tj == 16) || (ti == 8 && tj == 16) || (ti == 16 && tj == 8) ||
           (ti == 8 && tj == 8) || (ti == 4 && tj == 16) || (ti == 8 && tj == 4) ||
           (ti == 4 && tj == 8);
}

bool vote_level_supported(int level) { return level >= 2 && level <= 4; }

cudaError_t prepare_vote_kernel(int ti, int tj, int level)
{
    return vote_dispatch(0, ti, tj, level, nullptr, 0, nullptr, nullptr);
}

cudaError_t launch_vote(const VoteArgs &A, int ti, int tj, int level, int grid, cudaStream_t s)
{
    return vote_dispatch(1, ti, tj, level, &A, grid, s, nullptr);
}

cudaError_t vote_occupancy(int ti, int tj, int level, int *blocks)
{
    return vote_dispatch(2, ti, tj, level, nullptr, 0, nullptr, blocks);
}

cudaError_t launch_fit_triplets(const trk_hit *hits, int64_t n_hits, const int32_t *ijk,
                                int64_t n, const FitConst &C, float *params, uint32_t *bins,
                                int32_t *flags, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    const int64_t blocks64 = (n + 255) / 256;
    const int grid = (int)(blocks64 < 4096 ? blocks64 : 4096);
    k_fit_triplets<<<grid, 256, 0, s>>>(hits, n_hits, ijk, n, C, params, bins, flags);
    return cudaGetLastError();
}

}  // namespace trk
