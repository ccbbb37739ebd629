// Candidate fit: a helix through each candidate's hits (paper Sec. 8 and Fig. 6: the
// candidates found in the parameter space are then fitted to their hits; the paper times
// such a fit on CPU cores without defining it).  The definition implemented here is given
// with trk_track in trk.h: algebraic circle fit, one hit per layer, signed arcs from the
// perigee and a least-squares line in (s, z).
//
// One thread per candidate, in FP64: the algebraic circle fit squares the coordinates, and
// for the stiff tracks (R up to ~1e5 cm) its normal equations lose about ten digits, which
// FP32 does not have.  GB300's FP64 pipe is narrow, so nothing is computed redundantly:
// a candidate's few hits (about 20) are walked serially by its thread, in list order, so
// the sums are formed in the same order as the definition's.  The per-layer choice lives
// in a small shared-memory table per thread.
#include <climits>

#include "trk_common.cuh"

namespace trk {

struct FitTrackArgs {
    const trk_candidate *cand;
    const unsigned long long *n_cand;
    int64_t cand_cap;
    const int32_t *hit_ids;      // global input hit indices, per candidate at hit_off
    int64_t hit_cap;
    const CallArgs *args;        // the call's input hits
    double kB;                   // K * B [GeV / cm]
    trk_track *out;
    uint8_t *hit_used;
    const int32_t *order;        // candidates in processing order (by hit count)
};

// Candidates are fitted in an order grouped by hit count (a counting sort on
// min(n_hits, kFitBuckets - 1), largest first), so that the threads of a warp walk hit lists
// of similar length; the results go to each candidate's own slot, so the order does not
// change them.
constexpr int kFitBuckets = 1024;

__device__ __forceinline__ int fit_bucket(int n_hits)
{
    const int m = n_hits < 0 ? 0 : (n_hits >= kFitBuckets ? kFitBuckets - 1 : n_hits);
    return kFitBuckets - 1 - m;
}

__global__ void k_fit_count(const trk_candidate *cand, const unsigned long long *n_cand,
                            int64_t cand_cap, int32_t *counts)
{
    int64_t n = (int64_t)*n_cand;
    n = n < cand_cap ? n : cand_cap;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&counts[fit_bucket(cand[c].n_hits)], 1);
}

// Exclusive scan of the bucket counts in place (one block of kFitBuckets threads).
__global__ void __launch_bounds__(kFitBuckets) k_fit_scan(int32_t *counts)
{
    __shared__ int32_t warp_tot[kFitBuckets / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int v = counts[t];
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(kFull, incl, o);
        if (lane >= o)
            incl += u;
    }
    if (lane == 31)
        warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int x = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(kFull, x, o);
            if (lane >= o)
                x += u;
        }
        warp_tot[lane] = x;
    }
    __syncthreads();
    counts[t] = (w > 0 ? warp_tot[w - 1] : 0) + incl - v;
}

__global__ void k_fit_scatter(const trk_candidate *cand, const unsigned long long *n_cand,
                              int64_t cand_cap, int32_t *next, int32_t *order)
{
    int64_t n = (int64_t)*n_cand;
    n = n < cand_cap ? n : cand_cap;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x)
        order[atomicAdd(&next[fit_bucket(cand[c].n_hits)], 1)] = (int32_t)c;
}

constexpr int kFitThreads = 128;

// Solution of the 3 x 3 normal equations of the algebraic circle fit by Cramer's rule.
// Returns false when the determinant is zero or R^2 <= 0.
__device__ __forceinline__ bool circle_solve(double suu, double suv, double svv, double su,
                                             double sv, double sw, double suw, double svw,
                                             double m, double mx, double my, double &cx,
                                             double &cy, double &R)
{
    const double M[3][3] = {{suu, suv, su}, {suv, svv, sv}, {su, sv, m}};
    const double r[3] = {-suw, -svw, -sw};
    auto det3 = [](const double A[3][3]) {
        return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
               A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
               A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    };
    const double det = det3(M);
    if (det == 0.0)
        return false;
    double sol[3];
#pragma unroll
    for (int col = 0; col < 3; ++col) {
        double A[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                A[i][j] = (j == col) ? r[i] : M[i][j];
        sol[col] = det3(A) / det;
    }
    const double r2 = sol[0] * sol[0] / 4.0 + sol[1] * sol[1] / 4.0 - sol[2];
    if (!(r2 > 0.0))
        return false;
    cx = mx - sol[0] / 2.0;
    cy = my - sol[1] / 2.0;
    R = sqrt(r2);
    return true;
}

struct LayerPick {
    double res;     // smallest residual so far (then: the kept hit's arc length)
    int q;          // its position in the candidate's list (-1: none)
    int pad;
};

// Circle through the listed hits with `keep(q)` (all when keep is null).
template <class Keep>
__device__ __forceinline__ int circle_of(const int32_t *ids, int m, const trk_hit *H,
                                         int64_t n_hits, Keep keep, double &cx, double &cy,
                                         double &R)
{
    double mx = 0.0, my = 0.0;
    int n = 0;
    for (int q = 0; q < m; ++q) {
        if (!keep(q))
            continue;
        const int32_t id = ids[q];
        const trk_hit h = (id >= 0 && id < n_hits) ? H[id] : trk_hit{0.0f, 0.0f, 0.0f, -1};
        mx += h.x;
        my += h.y;
        ++n;
    }
    if (n < 3)
        return 1;
    mx /= n;
    my /= n;
    double suu = 0, suv = 0, svv = 0, su = 0, sv = 0, sw = 0, suw = 0, svw = 0;
    for (int q = 0; q < m; ++q) {
        if (!keep(q))
            continue;
        const int32_t id = ids[q];
        const trk_hit h = (id >= 0 && id < n_hits) ? H[id] : trk_hit{0.0f, 0.0f, 0.0f, -1};
        const double u = h.x - mx, v = h.y - my, w = u * u + v * v;
        suu += u * u;
        suv += u * v;
        svv += v * v;
        su += u;
        sv += v;
        sw += w;
        suw += u * w;
        svw += v * w;
    }
    return circle_solve(suu, suv, svv, su, sv, sw, suw, svw, (double)n, mx, my, cx, cy, R) ? 0 : 2;
}

__global__ void __launch_bounds__(kFitThreads) k_cand_fit(FitTrackArgs A, int n_layers)
{
    extern __shared__ LayerPick s_pick[];       // [kFitThreads][n_layers]
    LayerPick *pick = s_pick + (size_t)threadIdx.x * n_layers;
    int64_t n = (int64_t)*A.n_cand;
    n = n < A.cand_cap ? n : A.cand_cap;
    const trk_hit *H = A.args->hits;
    const int64_t n_hits = A.args->n_hits;
    for (int64_t ci = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ci < n;
         ci += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = A.order[ci];
        const trk_candidate cd = A.cand[c];
        const int m = cd.n_hits;
        const int64_t off = cd.hit_off;
        trk_track t;
        for (int k = 0; k < 5; ++k)
            t.params[k] = 0.0f;
        t.chi2_rphi = t.chi2_rz = 0.0f;
        t.n_used = 0;
        t.status = TRK_FIT_FEW_LAYERS;
        t.event = cd.event;
        t.layers = 0ull;
        if (off < 0 || m < 0 || off + m > A.hit_cap) {
            A.out[c] = t;
            continue;
        }
        const int32_t *ids = A.hit_ids + off;
        uint8_t *used = A.hit_used + off;
        auto hit = [&](int q) {
            const int32_t id = ids[q];
            return (id >= 0 && id < n_hits) ? H[id] : trk_hit{0.0f, 0.0f, 0.0f, -1};
        };
        auto all = [](int) { return true; };
        for (int q = 0; q < m; ++q)
            used[q] = 0;
        // 1. circle of all hits
        double cx, cy, R;
        int st = circle_of(ids, m, H, n_hits, all, cx, cy, R);
        if (st) {
            t.status = st == 1 ? TRK_FIT_FEW_LAYERS : TRK_FIT_DEGENERATE;
            A.out[c] = t;
            continue;
        }
        // 2. one hit per layer: the smallest | |p - c| - R |, the earlier hit on a tie
        for (int L = 0; L < n_layers; ++L) {
            pick[L].res = 0.0;
            pick[L].q = -1;
        }
        for (int q = 0; q < m; ++q) {
            const trk_hit h = hit(q);
            if (h.layer < 0 || h.layer >= n_layers)
                continue;
            const double dx = h.x - cx, dy = h.y - cy;
            const double res = fabs(sqrt(dx * dx + dy * dy) - R);
            LayerPick &p = pick[h.layer];
            if (p.q < 0 || res < p.res) {
                p.res = res;
                p.q = q;
            }
        }
        int n_used = 0;
        uint64_t layers = 0ull;
        for (int L = 0; L < n_layers; ++L)
            if (pick[L].q >= 0) {
                ++n_used;
                layers |= 1ull << L;
                used[pick[L].q] = 1;
            }
        t.n_used = n_used;
        t.layers = layers;
        if (n_used < 3) {
            A.out[c] = t;
            continue;
        }
        auto kept = [&](int q) { return used[q] != 0; };
        st = circle_of(ids, m, H, n_hits, kept, cx, cy, R);
        const double cn = sqrt(cx * cx + cy * cy);
        if (st || cn == 0.0) {
            t.status = TRK_FIT_DEGENERATE;
            A.out[c] = t;
            continue;
        }
        // 3. sense: signed area of the kept hits' polygon in layer order
        double area2 = 0.0;
        int first = -1, prev = -1;
        for (int L = 0; L < n_layers; ++L) {
            const int q = pick[L].q;
            if (q < 0)
                continue;
            if (first < 0) {
                first = q;
            } else {
                const trk_hit a = hit(prev), b = hit(q);
                area2 += (double)a.x * b.y - (double)a.y * b.x;
            }
            prev = q;
        }
        {
            const trk_hit a = hit(prev), b = hit(first);
            area2 += (double)a.x * b.y - (double)a.y * b.x;
        }
        const double sgn = area2 >= 0.0 ? 1.0 : -1.0;
        const double power = cx * cx + cy * cy - R * R;
        const double cmr = power / (cn + R);
        const double px = cx * (cmr / cn), py = cy * (cmr / cn);
        const double phi0 = atan2(-sgn * cx, sgn * cy);
        double sphi, cphi;
        sincos(phi0, &sphi, &cphi);
        const double d0 = -px * sphi + py * cphi;
        const double qopt = -sgn / (A.kB * R);
        // 4. signed arcs from the perigee (kept in the layer table), least-squares line
        double sbar = 0.0, zbar = 0.0;
        for (int q = 0; q < m; ++q) {
            if (!used[q])
                continue;
            const trk_hit h = hit(q);
            const double dx = h.x - px, dy = h.y - py;
            double a = sqrt(dx * dx + dy * dy) / (2.0 * R);
            a = a > 1.0 ? 1.0 : a;
            const double sk = ((dx * cphi + dy * sphi) >= 0.0 ? 1.0 : -1.0) * 2.0 * R * asin(a);
            pick[h.layer].res = sk;
            sbar += sk;
            zbar += h.z;
        }
        sbar /= n_used;
        zbar /= n_used;
        double sss = 0.0, ssz = 0.0;
        for (int q = 0; q < m; ++q) {
            if (!used[q])
                continue;
            const trk_hit h = hit(q);
            const double sk = pick[h.layer].res;
            sss += (sk - sbar) * (sk - sbar);
            ssz += (sk - sbar) * (h.z - zbar);
        }
        if (sss == 0.0) {
            t.status = TRK_FIT_DEGENERATE;
            A.out[c] = t;
            continue;
        }
        const double cot = ssz / sss, z0 = zbar - cot * sbar;
        double c2r = 0.0, c2z = 0.0;
        for (int q = 0; q < m; ++q) {
            if (!used[q])
                continue;
            const trk_hit h = hit(q);
            const double dx = h.x - cx, dy = h.y - cy;
            const double rr = sqrt(dx * dx + dy * dy) - R;
            const double rz = h.z - z0 - cot * pick[h.layer].res;
            c2r += rr * rr;
            c2z += rz * rz;
        }
        t.status = TRK_FIT_OK;
        t.params[0] = (float)phi0;
        t.params[1] = (float)qopt;
        t.params[2] = (float)d0;
        t.params[3] = (float)cot;
        t.params[4] = (float)z0;
        t.chi2_rphi = (float)c2r;
        t.chi2_rz = (float)c2z;
        A.out[c] = t;
    }
}

cudaError_t launch_cand_fit(const trk_candidate *cand, const unsigned long long *n_cand,
                            int64_t cand_cap, const int32_t *hit_ids, int64_t hit_cap,
                            const CallArgs *args, double kB, int n_layers, trk_track *out,
                            uint8_t *hit_used, int32_t *order, int32_t *buckets, int n_sm,
                            cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(buckets, 0, sizeof(int32_t) * kFitBuckets, s);
    if (e != cudaSuccess)
        return e;
    k_fit_count<<<n_sm * 4, 256, 0, s>>>(cand, n_cand, cand_cap, buckets);
    k_fit_scan<<<1, kFitBuckets, 0, s>>>(buckets);
    k_fit_scatter<<<n_sm * 4, 256, 0, s>>>(cand, n_cand, cand_cap, buckets, order);
    FitTrackArgs A;
    A.cand = cand;
    A.n_cand = n_cand;
    A.cand_cap = cand_cap;
    A.hit_ids = hit_ids;
    A.hit_cap = hit_cap;
    A.args = args;
    A.kB = kB;
    A.out = out;
    A.hit_used = hit_used;
    A.order = order;
    const size_t smem = sizeof(LayerPick) * kFitThreads * (size_t)n_layers;
    k_cand_fit<<<n_sm * 8, kFitThreads, smem, s>>>(A, n_layers);
    return cudaGetLastError();
}

cudaError_t prepare_fit_kernel()
{
    return cudaFuncSetAttribute(k_cand_fit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(LayerPick) * kFitThreads * TRK_MAX_LAYERS));
}

}  // namespace trk
