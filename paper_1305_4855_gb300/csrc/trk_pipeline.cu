// The steps around the vote kernel: packing hits per layer, scheduling work items, the
// local-maximum peak finder, candidate emission and hit assignment (paper Sec. 7 and
// Fig. 3: candidates are local maxima of the accumulated parameter space; Sec. 8: the
// whole event, the parameter space and the peak detection stay resident on the GPU, and
// the hits of each candidate go on to a fit).
#include "trk_common.cuh"
#include "trk_scan.cuh"

namespace trk {

// ---------------------------------------------------------------------------------------
// a1: pack -- validate, then a stable counting sort of each event's hits by layer into
// float4 (x, y, z, input index bits); the event keeps its input index range.
// ---------------------------------------------------------------------------------------

constexpr int kPackThreads = 256;

__global__ void __launch_bounds__(kPackThreads) k_pack(const CallArgs *args, int L, int max_per_event,
                                                       float4 *packed, int32_t *lay_off,
                                                       int64_t *ev_begin, int32_t *status)
{
    constexpr int NW = kPackThreads / kWarp;
    __shared__ int cnt[TRK_MAX_LAYERS];
    __shared__ int base[TRK_MAX_LAYERS];
    __shared__ int wcnt[NW][TRK_MAX_LAYERS];
    __shared__ int woff[NW][TRK_MAX_LAYERS];
    __shared__ int bad;
    const int e = blockIdx.x;
    if (e >= args->n_events)
        return;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int64_t n = args->n_hits;
    const int64_t a = args->offsets[e], b = args->offsets[e + 1];
    int32_t *lo = lay_off + (size_t)e * (L + 1);
    int st = 0;
    if (!(a >= 0 && a <= b && b <= n))
        st = TRK_EV_BAD_OFFSETS;
    else if (b - a > max_per_event)
        st = TRK_EV_TOO_MANY_HITS;
    if (st) {
        for (int l = tid; l <= L; l += kPackThreads)
            lo[l] = 0;
        if (tid == 0) {
            status[e] = st;
            ev_begin[e] = 0;
        }
        return;
    }
    for (int l = tid; l < TRK_MAX_LAYERS; l += kPackThreads) {
        cnt[l] = 0;
        for (int q = 0; q < NW; ++q)
            wcnt[q][l] = 0;
    }
    if (tid == 0)
        bad = 0;
    __syncthreads();
    const trk_hit *hits = args->hits;
    for (int64_t h = a + tid; h < b; h += kPackThreads) {
        const trk_hit x = hits[h];
        if (x.layer < 0 || x.layer >= L || !isfinite(x.x) || !isfinite(x.y) || !isfinite(x.z))
            bad = 1;
        else
            atomicAdd(&cnt[x.layer], 1);
    }
    __syncthreads();
    if (bad) {
        for (int l = tid; l <= L; l += kPackThreads)
            lo[l] = 0;
        if (tid == 0) {
            status[e] = TRK_EV_BAD_HIT;
            ev_begin[e] = 0;
        }
        return;
    }
    if (tid == 0) {
        int run = (int)a;
        for (int l = 0; l < L; ++l) {
            lo[l] = run;
            base[l] = run;
            run += cnt[l];
        }
        lo[L] = run;
        status[e] = 0;
        ev_begin[e] = a;
    }
    __syncthreads();
    for (int64_t c0 = a; c0 < b; c0 += kPackThreads) {
        const int64_t h = c0 + tid;
        trk_hit x;
        int layer = -1;
        if (h < b) {
            x = hits[h];
            layer = x.layer;
        }
        const unsigned peers = __match_any_sync(kFull, layer);
        const int rank = __popc(peers & lanemask_lt());
        if (layer >= 0 && lane == __ffs(peers) - 1)
            wcnt[w][layer] = __popc(peers);
        __syncthreads();
        if (tid < L) {
            int run = base[tid];
            for (int q = 0; q < NW; ++q) {
                woff[q][tid] = run;
                run += wcnt[q][tid];
                wcnt[q][tid] = 0;
            }
            base[tid] = run;
        }
        __syncthreads();
        if (layer >= 0)
            packed[woff[w][layer] + rank] = make_float4(x.x, x.y, x.z, __int_as_float((int)h));
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// a2: schedule -- work items per (event, layer triple) and their prefix sum
// ---------------------------------------------------------------------------------------

constexpr int kSchedThreads = 1024;

__global__ void __launch_bounds__(kSchedThreads) k_schedule(const CallArgs *args, const DevGeo *geo,
                                                            const int32_t *lay_off,
                                                            const int32_t *status, int ti, int tj,
                                                            int64_t *item_off, Counters *ctr)
{
    __shared__ int64_t warp_sum[kSchedThreads / kWarp];
    __shared__ int64_t carry;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int T = geo->n_triples, L1 = geo->n_layers + 1;
    const int F = args->n_events * T;
    if (tid == 0)
        carry = 0;
    unsigned long long trip = 0;
    __syncthreads();
    for (int f0 = 0; f0 < F; f0 += kSchedThreads) {
        const int f = f0 + tid;
        int64_t items = 0;
        if (f < F) {
            const int e = f / T, t = f - (f / T) * T;
            if (status[e] == 0) {
                const int32_t *lo = lay_off + (size_t)e * L1;
                const int la = geo->triples[t][0], lb = geo->triples[t][1], lc = geo->triples[t][2];
                const int64_t na = lo[la + 1] - lo[la], nb = lo[lb + 1] - lo[lb],
                              nc = lo[lc + 1] - lo[lc];
                if (na > 0 && nb > 0 && nc > 0) {
                    items = ((na + ti - 1) / ti) * ((nb + tj - 1) / tj);
                    trip += (unsigned long long)(na * nb * nc);
                }
            }
        }
        // block exclusive scan of items
        int64_t v = items;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(kFull, v, o);
            if (lane >= o)
                v += u;
        }
        if (lane == 31)
            warp_sum[w] = v;
        __syncthreads();
        if (w == 0) {
            int64_t s = warp_sum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(kFull, s, o);
                if (lane >= o)
                    s += u;
            }
            warp_sum[lane] = s;
        }
        __syncthreads();
        const int64_t before = carry + (w > 0 ? warp_sum[w - 1] : 0) + v - items;
        if (f < F)
            item_off[f] = before;
        __syncthreads();
        if (tid == kSchedThreads - 1)
            carry = before + items;
        __syncthreads();
    }
    if (tid == 0) {
        item_off[F] = carry;
        ctr->n_items = (unsigned long long)carry;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        trip += __shfl_xor_sync(kFull, trip, o);
    if (lane == 0 && trip)
        atomicAdd(&ctr->n_triplets, trip);
}

// ---------------------------------------------------------------------------------------
// a5: peaks.  Bin b is a candidate iff h[b] >= T, h[b] >= h[m] for every neighbour m of its
// 3^5 box, and h[b] > h[m] for the neighbours with a smaller bin number.  The first two
// conditions say h[b] equals the maximum count over the box, which is separable: pass 1
// takes it over (d0, cot, z0) in shared memory, pass 2 over (phi0, q/pT) with a sliding
// window along phi0.
//
// Every maximum carries, in bit 0, whether it is attained more than once in its part of the
// box: key = count << 1, and two keys combine to their maximum, with bit 0 set when their
// counts are equal (kcomb).  The parts combined at each stage are disjoint, so the final bit
// says whether the box maximum occurs twice in the 3^5 box.  A bin that reaches the
// threshold and its box maximum is then a candidate outright when that maximum occurs once
// (it beats every neighbour), and pass 2 sets its bit; when it occurs again (a plateau) the
// bin is listed, and the tie pass keeps it unless a neighbour with a smaller bin number has
// the same count.
// ---------------------------------------------------------------------------------------

__device__ __forceinline__ int kcomb(int a, int b)
{
    return max(a, b) | (int)((a >> 1) == (b >> 1));
}
__device__ __forceinline__ int kcomb3(int a, int b, int c) { return kcomb(kcomb(a, b), c); }

// In-place combination over {i-1, i, i+1} along a line of n keys with the given stride.
__device__ __forceinline__ void line_comb3(int32_t *p, int n, int stride)
{
    int prev = 0, cur = p[0];
    for (int i = 0; i < n; ++i) {
        const int next = (i + 1 < n) ? p[(i + 1) * stride] : 0;
        p[i * stride] = kcomb3(prev, cur, next);
        prev = cur;
        cur = next;
    }
}

__device__ __forceinline__ void set_candidate(uint32_t *cbits, int64_t W, uint32_t *filter, int e,
                                              uint32_t bin)
{
    atomicOr(&cbits[(size_t)e * W + (bin >> 5)], 1u << (bin & 31));
    if (filter) {
        const uint32_t fb = cand_filter_bit(e, bin);
        atomicOr(&filter[(size_t)e * kFilterWords + (fb >> 5)], 1u << (fb & 31));
    }
}

constexpr int kPeakThreads = 256;

// Division by a fixed divisor d >= 1 through a multiply-high.  With m = ceil(2^32 / d) and
// e = m d - 2^32 < d, x m / 2^32 = x / d + x e / (d 2^32); when x d < 2^32 the added term
// is below 1 / d, less than the gap from x / d to the next integer, so the floor is exact.
struct DivBy {
    uint32_t m;
    bool one;
};
__device__ __forceinline__ DivBy make_div(uint32_t d)
{
    DivBy r;
    r.one = d <= 1u;
    r.m = r.one ? 0u : 0xFFFFFFFFu / d + 1u;
    return r;
}
__device__ __forceinline__ uint32_t div_by(uint32_t x, DivBy D)
{
    return D.one ? x : __umulhi(x, D.m);
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_pass1(const int32_t *hist, int32_t *m3,
                                                             FitConst C, int g0, int td,
                                                             const int32_t *status)
{
    extern __shared__ int32_t sk[];
    const int n0 = C.n[0], n1 = C.n[1], n2 = C.n[2], n3 = C.n[3], n4 = C.n[4];
    const int P4 = n4 + 1;
    const int nslab = (n2 + td - 1) / td;
    int b = blockIdx.x;
    const int slab = b % nslab;
    b /= nslab;
    const int i1 = b % n1;
    b /= n1;
    const int i0 = b % n0;
    const int ge = b / n0;
    const int e = g0 + ge;
    if (status[e] != 0)
        return;
    const int tid = threadIdx.x;
    const int d_start = slab * td;
    const int rows = min(td, n2 - d_start);
    const int plane = n3 * n4;
    const int32_t *h_e = hist + (size_t)e * C.nbins;
    const uint32_t base = (uint32_t)i0 * C.stride[0] + (uint32_t)i1 * C.stride[1];
    // The slab and its two halo rows are one contiguous run of the histogram (d0 is the
    // third-slowest axis): element x of the run is global offset (d_start - 1) * plane + x,
    // and zero outside [0, n2 * plane).  Eight loads per thread are issued before the
    // shared-memory stores so that the pass streams instead of waiting on each load.
    const int total = (rows + 2) * plane;        // < 2^16 (shared-memory sized)
    const DivBy by4 = make_div((uint32_t)n4);
    const int64_t g_first = (int64_t)(d_start - 1) * plane;
    const int64_t g_end = (int64_t)n2 * plane;
    constexpr int kL = 8;
    for (int x0 = tid; x0 < total; x0 += kL * kPeakThreads) {
        int v[kL];
#pragma unroll
        for (int u = 0; u < kL; ++u) {
            const int x = x0 + u * kPeakThreads;
            const int64_t g = g_first + x;
            v[u] = (x < total && g >= 0 && g < g_end) ? __ldg(h_e + base + g) : 0;
        }
#pragma unroll
        for (int u = 0; u < kL; ++u) {
            const int x = x0 + u * kPeakThreads;
            if (x < total)                   // row-padded: line x / n4, column x % n4
                sk[x + (int)div_by((uint32_t)x, by4)] = v[u] << 1;
        }
    }
    __syncthreads();
    for (int line = tid; line < (rows + 2) * n3; line += kPeakThreads)
        line_comb3(sk + line * P4, n4, 1);
    __syncthreads();
    for (int line = tid; line < (rows + 2) * n4; line += kPeakThreads) {
        const int lr = (int)div_by((uint32_t)line, by4), i4 = line - lr * n4;
        line_comb3(sk + lr * n3 * P4 + i4, n3, P4);
    }
    __syncthreads();
    int32_t *out = m3 + (size_t)ge * C.nbins + base + (uint32_t)d_start * C.stride[2];
    const int rs = n3 * P4;
    for (int line = tid; line < plane; line += kPeakThreads) {
        const int i3 = (int)div_by((uint32_t)line, by4), i4 = line - i3 * n4;
        const int32_t *q = sk + i3 * P4 + i4;
        int prev = q[0], cur = q[rs];
        for (int r = 0; r < rows; ++r) {
            const int next = q[(r + 2) * rs];
            out[(size_t)r * plane + line] = kcomb3(prev, cur, next);
            prev = cur;
            cur = next;
        }
    }
}

// Pass 1 in registers, for row blocks of at most 32 cot lines of 4, 8, 12 or 16 z0 bins
// (16-byte aligned histogram): a warp per (event, phi0, q/pT, run of kRun1 d0 rows), a
// lane per cot line holding the line's z0 bins.  Per d0 row the lane loads its line (16-byte
// loads; the warp reads the row's contiguous n3 n4 counts), combines over z0 within its
// registers and over cot with the neighbouring lanes (shuffles), and slides a window of
// three rows along d0, storing the middle row.  No shared memory and no barriers; every
// count is read once plus two halo rows per run.
constexpr int kRun1 = 8;
constexpr int kPass1WarpsPerBlock = 4;

template <int N4>
__global__ void __launch_bounds__(32 * kPass1WarpsPerBlock)
    k_peak_pass1r(const int32_t *hist, int32_t *m3, FitConst C, int g0, int G,
                  const int32_t *status)
{
    const int lane = threadIdx.x & 31;
    const int n0 = C.n[0], n1 = C.n[1], n2 = C.n[2], n3 = C.n[3];
    const int runs = (n2 + kRun1 - 1) / kRun1;
    int64_t w = (int64_t)blockIdx.x * kPass1WarpsPerBlock + (threadIdx.x >> 5);
    if (w >= (int64_t)G * n0 * n1 * runs)
        return;
    const int run = (int)(w % runs);
    w /= runs;
    const int i1 = (int)(w % n1);
    w /= n1;
    const int i0 = (int)(w % n0);
    const int ge = (int)(w / n0);
    const int e = g0 + ge;
    if (status[e] != 0)
        return;
    const bool line = lane < n3;
    const uint32_t plane = C.stride[2];
    const uint32_t base = (uint32_t)i0 * C.stride[0] + (uint32_t)i1 * C.stride[1] +
                          (uint32_t)lane * N4;
    const int32_t *h_e = hist + (size_t)e * C.nbins + base;
    int32_t *out = m3 + (size_t)ge * C.nbins + base;
    constexpr int NV = N4 / 4;
    // keys of row d combined over z0 and cot (0 outside the histogram)
    auto row_keys = [&](int d, int (&b)[N4]) {
        int k[N4];
        if (line && d >= 0 && d < n2) {
            const int4 *q = reinterpret_cast<const int4 *>(h_e + (size_t)d * plane);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const int4 x = __ldg(q + v);
                k[4 * v] = x.x << 1;
                k[4 * v + 1] = x.y << 1;
                k[4 * v + 2] = x.z << 1;
                k[4 * v + 3] = x.w << 1;
            }
        } else {
#pragma unroll
            for (int j = 0; j < N4; ++j)
                k[j] = 0;
        }
        int a[N4];
#pragma unroll
        for (int j = 0; j < N4; ++j)
            a[j] = kcomb3(j > 0 ? k[j - 1] : 0, k[j], j + 1 < N4 ? k[j + 1] : 0);
#pragma unroll
        for (int j = 0; j < N4; ++j) {
            int up = __shfl_up_sync(kFull, a[j], 1);
            int dn = __shfl_down_sync(kFull, a[j], 1);
            up = lane > 0 ? up : 0;
            dn = lane + 1 < n3 ? dn : 0;
            b[j] = kcomb3(up, a[j], dn);
        }
    };
    const int d_start = run * kRun1;
    const int d_end = min(n2, d_start + kRun1);
    int prev[N4], cur[N4];
    row_keys(d_start - 1, prev);
    row_keys(d_start, cur);
    for (int d = d_start; d < d_end; ++d) {
        int nx[N4];
        row_keys(d + 1, nx);
        if (line) {
            int4 *o = reinterpret_cast<int4 *>(out + (size_t)d * plane);
#pragma unroll
            for (int v = 0; v < NV; ++v)
                o[v] = make_int4(kcomb3(prev[4 * v], cur[4 * v], nx[4 * v]),
                                 kcomb3(prev[4 * v + 1], cur[4 * v + 1], nx[4 * v + 1]),
                                 kcomb3(prev[4 * v + 2], cur[4 * v + 2], nx[4 * v + 2]),
                                 kcomb3(prev[4 * v + 3], cur[4 * v + 3], nx[4 * v + 3]));
        }
#pragma unroll
        for (int j = 0; j < N4; ++j) {
            prev[j] = cur[j];
            cur[j] = nx[j];
        }
    }
}

// Pass 2: thread per (event, q/pT row, V consecutive inner positions, segment of kSeg
// phi0 rows); walks its segment keeping the maxima over q/pT +-1 of the three phi0 rows
// around the current one.  Segments (two extra rows of loads per kSeg) give the grid
// enough threads to fill every SM in even waves.  With V = 4 (inner size a multiple of 4)
// every load is a 16-byte vector, so a warp reads 512 contiguous bytes per row.  The
// plateau bins are collected per block in shared memory and appended to the global list
// with one atomic per block tile.
constexpr int kTieBuf = 2048;
constexpr int kSeg = 16;

template <int V>
struct IntV;
template <>
struct IntV<1> {
    int v[1];
    __device__ __forceinline__ static IntV load(const int32_t *p)
    {
        IntV r;
        r.v[0] = __ldg(p);
        return r;
    }
};
template <>
struct IntV<4> {
    int v[4];
    __device__ __forceinline__ static IntV load(const int32_t *p)
    {
        const int4 q = __ldg(reinterpret_cast<const int4 *>(p));
        IntV r;
        r.v[0] = q.x;
        r.v[1] = q.y;
        r.v[2] = q.z;
        r.v[3] = q.w;
        return r;
    }
};

template <int V>
__device__ __forceinline__ IntV<V> vcomb(IntV<V> a, const IntV<V> &b)
{
#pragma unroll
    for (int c = 0; c < V; ++c)
        a.v[c] = kcomb(a.v[c], b.v[c]);
    return a;
}

template <int V>
__global__ void __launch_bounds__(kPeakThreads, 4) k_peak_pass2(const int32_t *hist, const int32_t *m3,
                                                             FitConst C, int g0, int G,
                                                             int threshold, const int32_t *status,
                                                             uint32_t *cbits, int64_t W,
                                                             uint32_t *filter,
                                                             unsigned long long *ties,
                                                             unsigned long long *n_ties,
                                                             int64_t tie_cap)
{
    __shared__ unsigned long long s_buf[kTieBuf];
    __shared__ int s_n;
    __shared__ unsigned long long s_base;
    const int n0 = C.n[0], n1 = C.n[1];
    const uint32_t inner = C.stride[1];
    const uint32_t innerV = inner / V;
    const bool per0 = (C.periodic & 1) != 0;
    const int nseg = (n0 + kSeg - 1) / kSeg;
    const int64_t total = (int64_t)G * n1 * innerV * nseg;
    if (threadIdx.x == 0)
        s_n = 0;
    __syncthreads();
    // block-uniform trip count, so that every thread reaches the flush barriers
    for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x; t0 < total;
         t0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = t0 + threadIdx.x;
        const uint32_t rest = (uint32_t)(t % innerV) * V;
        const int64_t q = t / innerV;
        const int i1 = (int)(q % n1);
        const int64_t q2 = q / n1;
        const int seg = (int)(q2 % nseg);
        const int ge = (int)(q2 / nseg);
        const int e = g0 + ge;
        if (t < total && status[e] == 0) {
            const int32_t *m = m3 + (size_t)ge * C.nbins + rest;
            const int32_t *h_e = hist + (size_t)e * C.nbins + rest;
            auto colmax = [&](int j0) {
                const int32_t *r = m + (size_t)j0 * C.stride[0];
                IntV<V> x = IntV<V>::load(r + (size_t)i1 * inner);
                if (i1 > 0)
                    x = vcomb(x, IntV<V>::load(r + (size_t)(i1 - 1) * inner));
                if (i1 + 1 < n1)
                    x = vcomb(x, IntV<V>::load(r + (size_t)(i1 + 1) * inner));
                return x;
            };
            // phi0 rows in groups of kR: the column maxima of rows i0+1 .. i0+kR and the
            // counts of rows i0 .. i0+kR-1 are loaded together, then the window slides.
            constexpr int kR = V == 1 ? 8 : 2;
            IntV<V> zero;
#pragma unroll
            for (int c = 0; c < V; ++c)
                zero.v[c] = 0;
            const int r_begin = seg * kSeg;
            const int r_end = min(n0, r_begin + kSeg);
            IntV<V> prev = r_begin > 0 ? colmax(r_begin - 1) : (per0 ? colmax(n0 - 1) : zero);
            IntV<V> cur = colmax(r_begin);
            for (int c0 = r_begin; c0 < r_end; c0 += kR) {
                IntV<V> nx[kR], hh[kR];
#pragma unroll
                for (int u = 0; u < kR; ++u) {
                    const int r = c0 + u;
                    const int rn = r + 1;
                    // rows past the segment's end are loaded only as the last row's next
                    nx[u] = rn < n0 ? (r < r_end ? colmax(rn) : zero)
                                    : (rn == n0 && per0 ? colmax(0) : zero);
                    hh[u] = r < r_end ? IntV<V>::load(h_e + (size_t)r * C.stride[0] +
                                                      (size_t)i1 * inner)
                                      : zero;
                }
#pragma unroll
                for (int u = 0; u < kR; ++u) {
                    const int r = c0 + u;
#pragma unroll
                    for (int c = 0; c < V; ++c) {
                        const int h = hh[u].v[c];
                        const int box = kcomb3(prev.v[c], cur.v[c], nx[u].v[c]);
                        if (r < r_end && h >= threshold && h == (box >> 1)) {
                            const uint32_t bin = (uint32_t)r * C.stride[0] + (uint32_t)i1 * inner +
                                                 rest + (uint32_t)c;
                            if (!(box & 1)) {        // the only maximum of its box
                                set_candidate(cbits, W, filter, e, bin);
                                continue;
                            }
                            const unsigned long long key =
                                ((unsigned long long)(unsigned)e << 32) | bin;
                            const int k = atomicAdd(&s_n, 1);
                            if (k < kTieBuf) {
                                s_buf[k] = key;
                            } else {      // buffer full: append directly
                                const unsigned long long slot = atomicAdd(n_ties, 1ull);
                                if ((int64_t)slot < tie_cap)
                                    ties[slot] = key;
                            }
                        }
                    }
                    prev = cur;
                    cur = nx[u];
                }
            }
        }
        __syncthreads();
        const int nb = min(s_n, kTieBuf);
        if (nb > 0) {
            if (threadIdx.x == 0)
                s_base = atomicAdd(n_ties, (unsigned long long)nb);
            __syncthreads();
            for (int k = threadIdx.x; k < nb; k += blockDim.x) {
                const unsigned long long slot = s_base + (unsigned long long)k;
                if ((int64_t)slot < tie_cap)
                    ties[slot] = s_buf[k];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0)
            s_n = 0;
        __syncthreads();
    }
}

// Warp-cooperative tie test of one bin whose count h reaches its box maximum: true iff a
// neighbour with a smaller bin number has the same count (that neighbour, or a lower one,
// keeps the plateau's candidate).  Every lane returns the answer.
__device__ __forceinline__ bool lower_equal_neighbour(const int32_t *h_e, const FitConst &C,
                                                      uint32_t bin, int h, int lane)
{
    const int n0 = C.n[0];
    const bool per0 = (C.periodic & 1) != 0;
    int idx[5];
    uint32_t rem = bin;
    for (int k = 0; k < 5; ++k) {
        idx[k] = (int)(rem / C.stride[k]);
        rem -= (uint32_t)idx[k] * C.stride[k];
    }
    bool beaten = false;
    for (int o = lane; o < 243; o += 32) {
        int off = o;
        uint32_t nb = 0;
        bool ok = true;
#pragma unroll
        for (int k = 4; k >= 0; --k) {
            const int dk = off % 3 - 1;
            off /= 3;
            int j = idx[k] + dk;
            if (j < 0 || j >= C.n[k]) {
                if (k == 0 && per0)
                    j = (j + n0) % n0;
                else
                    ok = false;
            }
            nb += (uint32_t)j * C.stride[k];
        }
        if (ok && nb < bin && h_e[nb] == h)
            beaten = true;
    }
    return __any_sync(kFull, beaten);
}

// Tie pass: warp per listed bin; candidate unless a neighbour with a smaller bin number
// has the same count.
__global__ void k_peak_ties(const int32_t *hist, FitConst C, const unsigned long long *ties,
                            const unsigned long long *n_ties, int64_t tie_cap, uint32_t *cbits,
                            int64_t W, uint32_t *filter, unsigned long long *overflow)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t n = (int64_t)*n_ties;
    if (n > tie_cap) {
        if (warp0 == 0 && lane == 0)
            atomicOr(overflow, 1ull);
        n = tie_cap;
    }
    for (int64_t i = warp0; i < n; i += nwarps) {
        const unsigned long long key = ties[i];
        const int e = (int)(key >> 32);
        const uint32_t bin = (uint32_t)key;
        const int32_t *h_e = hist + (size_t)e * C.nbins;
        const bool beaten = lower_equal_neighbour(h_e, C, bin, h_e[bin], lane);
        if (!beaten && lane == 0)
            set_candidate(cbits, W, filter, e, bin);
    }
}

struct CandVotes3 {
    const trk_candidate *c;
    __device__ int64_t operator()(int64_t i) const { return 3 * (int64_t)c[i].votes; }
};
struct CandHits {
    const int32_t *nh;
    __device__ int64_t operator()(int64_t i) const { return nh[i]; }
};
struct ChunkCount {
    const int32_t *cnt;
    __device__ int64_t operator()(int64_t i) const { return cnt[i] > 0 ? cnt[i] : 0; }
};

// ---------------------------------------------------------------------------------------
// candidates, assignment, compaction
// ---------------------------------------------------------------------------------------

__global__ void k_cand_emit(const uint32_t *cbits, const uint32_t *wprefix, int64_t n_words,
                            int64_t W, const int32_t *hist, FitConst C, trk_candidate *cand,
                            int32_t *fill, int64_t cand_cap, Counters *ctr)
{
    // a thread per bitmap word; the few set bits are expanded serially
    for (int64_t gw = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gw < n_words;
         gw += (int64_t)gridDim.x * blockDim.x) {
        uint32_t word = cbits[gw];
        if (word == 0)
            continue;
        const int e = (int)(gw / W);
        int64_t c = (int64_t)wprefix[gw];
        const uint32_t base = (uint32_t)((gw - (int64_t)e * W) * 32);
        while (word) {
            const int bit = __ffs(word) - 1;
            word &= word - 1;
            const uint32_t bin = base + (uint32_t)bit;
            if (c < cand_cap) {
                trk_candidate r;
                r.bin = bin;
                r.event = e;
                r.votes = hist[(size_t)e * C.nbins + bin];
                r.n_hits = 0;
                r.hit_off = 0;
                r.reserved = 0;
                uint32_t rem = bin;
                for (int k = 0; k < 5; ++k) {
                    const uint32_t idx = rem / C.stride[k];
                    rem -= idx * C.stride[k];
                    const double centre =
                        __dadd_rn(C.lo_d[k], __dmul_rn((double)idx + 0.5, C.w_d[k]));
                    r.params[k] = __double2float_rn(centre);
                }
                cand[c] = r;
                fill[c] = 0;
            } else {
                atomicOr(&ctr->overflow, 1ull);
            }
            ++c;
        }
    }
}

// Locates a work item: event, layer triple and the first packed hit of each tile.
struct ItemLoc {
    int e, a_first, b_first, c_first;
};

__device__ __forceinline__ ItemLoc locate_item(int64_t item, const int64_t *item_off, int F, int T,
                                               const DevGeo *geo, const int32_t *lay_off, int ti,
                                               int tj)
{
    const int f = upper_index(item_off, F, item);
    const int e = f / T, t = f - e * T;
    const int L1 = geo->n_layers + 1;
    const int32_t *lo = lay_off + (size_t)e * L1;
    const int la = geo->triples[t][0], lb = geo->triples[t][1], lc = geo->triples[t][2];
    const int nb = lo[lb + 1] - lo[lb];
    const int64_t local = item - item_off[f];
    const int ntj = (nb + tj - 1) / tj;
    const int ti_ = (int)(local / ntj), tj_ = (int)(local - (int64_t)ti_ * ntj);
    ItemLoc r;
    r.e = e;
    r.a_first = lo[la] + ti_ * ti;
    r.b_first = lo[lb] + tj_ * tj;
    r.c_first = lo[lc];
    return r;
}



constexpr int kAssignThreads = 1024;

// Assignment, part 1: a stream over the bins of the vote list that finds the candidate
// votes and queues their slots.  Only ~1 % of the votes land in candidate bins.  A warp
// takes kU whole 32-slot chunks at a time, a lane per slot: every lane issues its kU bin
// loads (each warp load is one chunk's 128 contiguous bytes, streamed with the evict-first
// hint) while the chunks' counts and events arrive as warp-wide broadcasts; slots past a
// chunk's count hold stale data and are discarded.  The shared-memory candidate filter
// leaves the bitmap lookup to the few votes whose filter bit is set, and those lookups are
// issued together.  A candidate vote's slot goes to the queue with one atomic per warp, so
// the stream never waits on the dependent loads of the hit decoding (part 2).
template <bool kOneEvent>
__global__ void __launch_bounds__(kAssignThreads, 1) k_assign_scan(AssignArgs A)
{
    extern __shared__ uint32_t s_filter[];
    if (kOneEvent) {
        for (uint32_t q = threadIdx.x; q < kFilterWords / 4; q += kAssignThreads)
            reinterpret_cast<uint4 *>(s_filter)[q] =
                __ldg(reinterpret_cast<const uint4 *>(A.filter) + q);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    int64_t n_chunks = (int64_t)A.ctr->n_chunks;
    n_chunks = n_chunks < A.chunk_cap ? n_chunks : A.chunk_cap;
    constexpr int kU = 16;
    const int64_t warps = (int64_t)gridDim.x * (kAssignThreads / 32);
    const int64_t warp = blockIdx.x * (int64_t)(kAssignThreads / 32) + (threadIdx.x >> 5);
    for (int64_t c0 = warp; c0 < n_chunks; c0 += kU * warps) {
        uint32_t bin[kU];
        int cnt[kU], ev[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t c = c0 + u * warps;
            const bool in = c < n_chunks;
            bin[u] = in ? __ldcs(A.vote_bin + c * kWarp + lane) : 0u;
            cnt[u] = in ? __ldg(A.chunk_count + c) : 0;
            ev[u] = in ? __ldg(A.chunk_event + c) : 0;
        }
        uint32_t maybe = 0;           // bit u: this lane's vote of chunk u passes the filter
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const uint32_t fb = cand_filter_bit(ev[u], bin[u]);
            const uint32_t fw = kOneEvent ? s_filter[fb >> 5]
                                          : __ldg(A.filter + (size_t)ev[u] * kFilterWords + (fb >> 5));
            const uint32_t f = (fw >> (fb & 31)) & 1u;
            maybe |= (lane < cnt[u] ? f : 0u) << u;
        }
        uint32_t mine = 0;            // bit u: this lane's vote of chunk u is a candidate vote
        if (__any_sync(kFull, maybe != 0)) {
            uint32_t word[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u)
                word[u] = ((maybe >> u) & 1u)
                              ? __ldg(A.cbits + (size_t)ev[u] * A.W + (bin[u] >> 5))
                              : 0u;
#pragma unroll
            for (int u = 0; u < kU; ++u)
                mine |= ((word[u] >> (bin[u] & 31)) & 1u) << u;
        }
        const int nm = __popc(mine);
        int incl = nm;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o)
                incl += v;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        if (total == 0)
            continue;
        unsigned long long base = 0;
        if (lane == 31)
            base = atomicAdd(&A.ctr->n_cvotes, (unsigned long long)total);
        base = __shfl_sync(kFull, base, 31);
        unsigned long long pos = base + (unsigned long long)(incl - nm);
        while (mine) {
            const int u = __ffs(mine) - 1;
            mine &= mine - 1;
            if ((int64_t)pos < A.cqueue_cap)
                A.cqueue[pos] = (unsigned long long)((c0 + u * warps) * kWarp + lane);
            ++pos;
        }
    }
}

// Assignment, part 2: thread per queued candidate vote -- its candidate index from the
// bitmap word prefix, a slot in the candidate's region by an atomic, and the three input
// hit ids (event-local) decoded from the vote code and its chunk's tile position.
__global__ void k_assign_cvotes(AssignArgs A)
{
    int64_t n = (int64_t)A.ctr->n_cvotes;
    if (n > A.cqueue_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0)
            atomicOr(&A.ctr->overflow, 2ull);
        n = A.cqueue_cap;
    }
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slot = (int64_t)A.cqueue[q];
        const int e = __ldg(A.chunk_event + (slot >> 5));
        const uint32_t bin = __ldg(A.vote_bin + slot);
        const size_t wpos = (size_t)e * A.W + (bin >> 5);
        const uint32_t word = __ldg(A.cbits + wpos);
        const int64_t c = (int64_t)A.wprefix[wpos] + __popc(word & ((1u << (bin & 31)) - 1u));
        if (c >= A.cand_cap)
            continue;
        const int4 loc = __ldg(A.chunk_loc + (slot >> 5));
        const uint32_t code = __ldg(A.vote_code + slot);
        const int fslot = atomicAdd(&A.fill[c], 1);
        const int64_t pos = A.vote_off[c] + 3 * (int64_t)fslot;
        if (pos + 3 > A.assign_cap) {
            atomicOr(&A.ctr->overflow, 2ull);
            continue;
        }
        const int ip = loc.x + (int)code_i(code);
        const int jp = loc.y + (int)code_j(code);
        const int kp = loc.z + (int)code_k(code);
        const int eb = (int)A.ev_begin[e];
        A.assign[pos] = __float_as_int(A.packed[ip].w) - eb;
        A.assign[pos + 1] = __float_as_int(A.packed[jp].w) - eb;
        A.assign[pos + 2] = __float_as_int(A.packed[kp].w) - eb;
    }
}

// Warp per candidate: bitmap over the event's hits -> sorted unique event-local ids,
// written back over the candidate's own assignment region.
__global__ void k_cand_hits(const trk_candidate *cand, const unsigned long long *n_cand_dev,
                            int64_t cand_cap, const int64_t *vote_off, int32_t *assign,
                            int64_t assign_cap, const CallArgs *args, int32_t *nhits,
                            int max_words)
{
    extern __shared__ uint32_t bm_all[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t *bm = bm_all + (size_t)w * max_words;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t n = (int64_t)*n_cand_dev;
    n = n < cand_cap ? n : cand_cap;
    for (int64_t c = warp0; c < n; c += nwarps) {
        const trk_candidate r = cand[c];
        const int64_t ne = args->offsets[r.event + 1] - args->offsets[r.event];
        const int words = (int)((ne + 31) / 32);
        const int64_t off = vote_off[c];
        int64_t m = 3 * (int64_t)r.votes;
        if (off + m > assign_cap)
            m = 0;
        for (int q = lane; q < words; q += 32)
            bm[q] = 0;
        __syncwarp();
        for (int64_t q = lane; q < m; q += 32) {
            const int id = assign[off + q];
            if ((unsigned)id < (unsigned)ne)
                atomicOr(&bm[id >> 5], 1u << (id & 31));
        }
        __syncwarp();
        int64_t run = 0;
        for (int q0 = 0; q0 < words; q0 += 32) {
            const int q = q0 + lane;
            uint32_t word = q < words ? bm[q] : 0u;
            const int pc = __popc(word);
            int inc = pc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(kFull, inc, o);
                if (lane >= o)
                    inc += u;
            }
            int64_t pos = off + run + inc - pc;
            while (word) {
                const int bit = __ffs(word) - 1;
                word &= word - 1;
                assign[pos++] = q * 32 + bit;
            }
            run += __shfl_sync(kFull, inc, 31);
        }
        if (lane == 0)
            nhits[c] = (int32_t)run;
        __syncwarp();
    }
}

__global__ void k_compact(trk_candidate *cand, const unsigned long long *n_cand_dev, int64_t cand_cap,
                          const int64_t *vote_off, const int32_t *assign, const int32_t *nhits,
                          const int64_t *hit_off, const int64_t *ev_begin, int32_t *hit_ids)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t n = (int64_t)*n_cand_dev;
    n = n < cand_cap ? n : cand_cap;
    for (int64_t c = warp0; c < n; c += nwarps) {
        const int e = cand[c].event;
        const int64_t src = vote_off[c], dst = hit_off[c];
        const int k = nhits[c];
        const int eb = (int)ev_begin[e];
        for (int q = lane; q < k; q += 32)
            hit_ids[dst + q] = assign[src + q] + eb;
        if (lane == 0) {
            cand[c].hit_off = dst;
            cand[c].n_hits = k;
        }
    }
}

// Per-event candidate offsets and the call's verdict.
__global__ void k_finalize(const uint32_t *wprefix, int64_t W, const CallArgs *args, Counters *ctr,
                           int64_t cand_cap, int64_t *cand_off, int32_t *status)
{
    const int n_events = args->n_events;
    const unsigned long long ncand = ctr->n_cand;
    const bool over = ctr->overflow != 0 || ncand > (unsigned long long)cand_cap;
    for (int e = threadIdx.x; e <= n_events; e += blockDim.x) {
        int64_t v = e < n_events ? (int64_t)wprefix[(size_t)e * W] : (int64_t)ncand;
        cand_off[e] = over ? 0 : v;
        if (over && e < n_events)
            status[e] |= TRK_EV_CAND_OVERFLOW;
    }
}

// Decode the vote list into (event, i, j, k) input indices and bins (debug helper).
__global__ void k_decode_votes(AssignArgs A, const int64_t *chunk_pos, int64_t n_chunks,
                               int32_t *dst, uint32_t *bins, int64_t cap)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int T = A.geo->n_triples;
    const int F = A.args->n_events * T;
    for (int64_t cid = warp0; cid < n_chunks; cid += nwarps) {
        const int item = A.chunk_item[cid];
        const int count = A.chunk_count[cid];
        if (item < 0 || count <= 0)
            continue;
        const ItemLoc loc = locate_item(item, A.item_off, F, T, A.geo, A.lay_off, A.ti, A.tj);
        if (lane >= count)
            continue;
        const int64_t out = chunk_pos[cid] + lane;
        if (out >= cap)
            continue;
        const uint32_t code = A.vote_code[cid * kWarp + lane];
        dst[4 * out] = loc.e;
        dst[4 * out + 1] = __float_as_int(A.packed[loc.a_first + (int)code_i(code)].w);
        dst[4 * out + 2] = __float_as_int(A.packed[loc.b_first + (int)code_j(code)].w);
        dst[4 * out + 3] = __float_as_int(A.packed[loc.c_first + (int)code_k(code)].w);
        bins[out] = A.vote_bin[cid * kWarp + lane];
    }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------

// Raise the dynamic shared-memory limits once (outside any stream capture).
cudaError_t prepare_pipeline_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(k_peak_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         100 * 1024);
    if (e != cudaSuccess)
        return e;
    e = cudaFuncSetAttribute(k_cand_hits, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
    if (e != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_assign_scan<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(uint32_t) * kFilterWords));
}

cudaError_t launch_pack(const CallArgs *args, int n_events, int L, int max_per_event,
                        float4 *packed, int32_t *lay_off, int64_t *ev_begin, int32_t *status,
                        cudaStream_t s)
{
    k_pack<<<n_events, kPackThreads, 0, s>>>(args, L, max_per_event, packed, lay_off, ev_begin,
                                             status);
    return cudaGetLastError();
}

cudaError_t launch_schedule(const CallArgs *args, const DevGeo *geo, const int32_t *lay_off,
                            const int32_t *status, int ti, int tj, int64_t *item_off,
                            Counters *ctr, cudaStream_t s)
{
    k_schedule<<<1, kSchedThreads, 0, s>>>(args, geo, lay_off, status, ti, tj, item_off, ctr);
    return cudaGetLastError();
}

size_t peak_pass1_smem(const FitConst &C, int td)
{
    return sizeof(int32_t) * (size_t)(td + 2) * C.n[3] * (C.n[4] + 1);
}

// Peak passes 1 and 2 for events [g0, g0 + G): sets the candidate bits of the strict
// maxima and lists the plateau maxima for the tie pass (cbits must be zeroed).
// vec_ok: hist is 16-byte aligned, so that pass 2 may read it with 16-byte loads.
cudaError_t launch_peaks(const int32_t *hist, int32_t *m3, const FitConst &C, int g0, int G,
                         int td, int threshold, const int32_t *status, uint32_t *cbits, int64_t W,
                         uint32_t *filter, unsigned long long *ties, unsigned long long *n_ties,
                         int64_t tie_cap, int n_sm, cudaStream_t s, bool vec_ok)
{
    const bool reg1 = vec_ok && C.n[3] <= 32 && C.n[4] % 4 == 0 && C.n[4] <= 16;
    if (reg1) {
        const int64_t warps = (int64_t)G * C.n[0] * C.n[1] * ((C.n[2] + kRun1 - 1) / kRun1);
        const unsigned grid1 =
            (unsigned)((warps + kPass1WarpsPerBlock - 1) / kPass1WarpsPerBlock);
        const unsigned bt = 32 * kPass1WarpsPerBlock;
        switch (C.n[4]) {
        case 4:
            k_peak_pass1r<4><<<grid1, bt, 0, s>>>(hist, m3, C, g0, G, status);
            break;
        case 8:
            k_peak_pass1r<8><<<grid1, bt, 0, s>>>(hist, m3, C, g0, G, status);
            break;
        case 12:
            k_peak_pass1r<12><<<grid1, bt, 0, s>>>(hist, m3, C, g0, G, status);
            break;
        default:
            k_peak_pass1r<16><<<grid1, bt, 0, s>>>(hist, m3, C, g0, G, status);
            break;
        }
    } else {
        const size_t sm = peak_pass1_smem(C, td);
        const int nslab = (C.n[2] + td - 1) / td;
        const int64_t grid1 = (int64_t)G * C.n[0] * C.n[1] * nslab;
        k_peak_pass1<<<(unsigned)grid1, kPeakThreads, sm, s>>>(hist, m3, C, g0, td, status);
    }
    const bool vec = vec_ok && (C.stride[1] % 4) == 0;
    const int64_t threads = (int64_t)G * C.n[1] * C.stride[1] / (vec ? 4 : 1) *
                            ((C.n[0] + kSeg - 1) / kSeg);
    int64_t grid2 = (threads + kPeakThreads - 1) / kPeakThreads;
    const int64_t cap2 = (int64_t)n_sm * 32;
    grid2 = grid2 < cap2 ? grid2 : cap2;
    const unsigned g2 = (unsigned)(grid2 > 0 ? grid2 : 1);
    if (vec)
        k_peak_pass2<4><<<g2, kPeakThreads, 0, s>>>(hist, m3, C, g0, G, threshold, status, cbits,
                                                     W, filter, ties, n_ties, tie_cap);
    else
        k_peak_pass2<1><<<g2, kPeakThreads, 0, s>>>(hist, m3, C, g0, G, threshold, status, cbits,
                                                     W, filter, ties, n_ties, tie_cap);
    return cudaGetLastError();
}

// The tie pass over the listed bins; sets the candidate bits (cbits must be zeroed).
cudaError_t launch_peak_ties(const int32_t *hist, const FitConst &C,
                             const unsigned long long *ties, const unsigned long long *n_ties,
                             int64_t tie_cap, uint32_t *cbits, int64_t W, uint32_t *filter,
                             unsigned long long *overflow, int n_sm, cudaStream_t s)
{
    k_peak_ties<<<n_sm * 8, 256, 0, s>>>(hist, C, ties, n_ties, tie_cap, cbits, W, filter,
                                         overflow);
    return cudaGetLastError();
}

cudaError_t launch_word_scan(const uint32_t *cbits, int64_t n_words, uint32_t *wprefix,
                             int64_t *bsum, unsigned long long *total, cudaStream_t s)
{
    return scan_exclusive(PopcVal{cbits}, nullptr, n_words, n_words, wprefix, bsum, total, s);
}

cudaError_t launch_cand_emit(const uint32_t *cbits, const uint32_t *wprefix, int64_t n_words,
                             int64_t W, const int32_t *hist, const FitConst &C,
                             trk_candidate *cand, int32_t *fill, int64_t cand_cap, Counters *ctr,
                             int n_sm, cudaStream_t s)
{
    int64_t grid = (n_words + 255) / 256;
    const int64_t cap = (int64_t)n_sm * 16;
    grid = grid < cap ? grid : cap;
    k_cand_emit<<<(unsigned)(grid > 0 ? grid : 1), 256, 0, s>>>(cbits, wprefix, n_words, W, hist,
                                                                 C, cand, fill, cand_cap, ctr);
    return cudaGetLastError();
}

cudaError_t launch_vote_offsets(const trk_candidate *cand, const unsigned long long *n_cand,
                                int64_t cand_cap, int64_t *vote_off, int64_t *bsum,
                                unsigned long long *total, cudaStream_t s)
{
    return scan_exclusive(CandVotes3{cand}, n_cand, 0, cand_cap, vote_off, bsum, total, s);
}

cudaError_t launch_assign(const AssignArgs &A, int n_events, int n_sm, cudaStream_t s)
{
    // the stream: persistent, one block per SM (a one-event call's filter takes most of
    // the shared memory)
    if (n_events == 1)
        k_assign_scan<true><<<n_sm, kAssignThreads, sizeof(uint32_t) * kFilterWords, s>>>(A);
    else
        k_assign_scan<false><<<n_sm, kAssignThreads, 0, s>>>(A);
    k_assign_cvotes<<<n_sm * 8, 256, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_cand_hits(const trk_candidate *cand, const unsigned long long *n_cand,
                             int64_t cand_cap, const int64_t *vote_off, int32_t *assign,
                             int64_t assign_cap, const CallArgs *args, int32_t *nhits,
                             int max_words, int n_sm, cudaStream_t s)
{
    int warps = (int)((96 * 1024) / ((size_t)max_words * 4));
    warps = warps < 1 ? 1 : (warps > 8 ? 8 : warps);
    const size_t sm = (size_t)warps * max_words * 4;
    k_cand_hits<<<n_sm * 8, warps * 32, sm, s>>>(cand, n_cand, cand_cap, vote_off, assign,
                                                  assign_cap, args, nhits, max_words);
    return cudaGetLastError();
}

cudaError_t launch_hit_offsets(const int32_t *nhits, const unsigned long long *n_cand,
                               int64_t cand_cap, int64_t *hit_off, int64_t *bsum,
                               unsigned long long *total, cudaStream_t s)
{
    return scan_exclusive(CandHits{nhits}, n_cand, 0, cand_cap, hit_off, bsum, total, s);
}

cudaError_t launch_compact(trk_candidate *cand, const unsigned long long *n_cand, int64_t cand_cap,
                           const int64_t *vote_off, const int32_t *assign, const int32_t *nhits,
                           const int64_t *hit_off, const int64_t *ev_begin, int32_t *hit_ids,
                           int n_sm, cudaStream_t s)
{
    k_compact<<<n_sm * 8, 256, 0, s>>>(cand, n_cand, cand_cap, vote_off, assign, nhits, hit_off,
                                        ev_begin, hit_ids);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const uint32_t *wprefix, int64_t W, const CallArgs *args,
                            Counters *ctr, int64_t cand_cap, int64_t *cand_off, int32_t *status,
                            cudaStream_t s)
{
    k_finalize<<<1, 256, 0, s>>>(wprefix, W, args, ctr, cand_cap, cand_off, status);
    return cudaGetLastError();
}

cudaError_t launch_chunk_positions(const int32_t *chunk_count, int64_t n_chunks, int64_t *pos,
                                   int64_t *bsum, unsigned long long *total, cudaStream_t s)
{
    return scan_exclusive(ChunkCount{chunk_count}, nullptr, n_chunks, n_chunks, pos, bsum, total,
                          s);
}

cudaError_t launch_decode_votes(const AssignArgs &A, const int64_t *chunk_pos, int64_t n_chunks,
                                int32_t *dst, uint32_t *bins, int64_t cap, int n_sm,
                                cudaStream_t s)
{
    k_decode_votes<<<n_sm * 8, 256, 0, s>>>(A, chunk_pos, n_chunks, dst, bins, cap);
    return cudaGetLastError();
}

}  // namespace trk
