// Internal device-side definitions shared by the kernels of libtrk (not part of the ABI).
//
// The helix-from-triplet arithmetic below follows the readings stated in include/trk.h
// (paper Sec. 8: a circle is fixed by centre and radius; a curved displaced track needs a
// parameter space beyond the interaction-point-constrained one).  It is written for FP32
// on the CUDA cores in forms that avoid cancellation, with an FP64 recomputation for the
// near-collinear fits (|D| / |p3 - p1| at or below a threshold, D == 0 included) and for
// any degenerate intermediate.  The library is compiled with -fmad=false: every fused
// multiply-add below is explicit, so the staged evaluation inside the vote kernel and the
// one-shot evaluation of trk_fit_triplets round identically.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "trk.h"

namespace trk {

constexpr double kGeVPerTeslaCm = 0.299792458e-2;
constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

// Constants of the fit and of the binning, passed by value to the kernels.
struct FitConst {
    float kB;            // K * B [GeV / cm]
    float inv_kB;        // 1 / (K * B)
    float pre_k2;        // curvature prefilter: 4 D^2 <= pre_k2 * |u|^2 |v|^2 |w|^2
    float sag2;          // FP64 recomputation when D^2 <= sag2 * |v|^2
    int periodic;        // bit 0 only (phi0)
    float lo[5], hi[5], inv_w[5];
    float period0;       // hi[0] - lo[0] when periodic
    int n[5];
    uint32_t stride[5];  // row-major strides, stride[4] = 1
    uint32_t nbins;
    double kB_d;
    double lo_d[5], hi_d[5], w_d[5];
};

// Geometry needed on the device.
struct DevGeo {
    int n_layers;
    int n_triples;
    int triples[TRK_MAX_TRIPLES][3];
};

// Per-call arguments, copied to the device before the launches so that a captured
// graph can be replayed for new inputs.
struct CallArgs {
    const trk_hit *hits;
    const int64_t *offsets;
    int64_t n_hits;
    int32_t n_events;
    int32_t pad;
};

// Device counters of one call (zeroed at its start).
struct Counters {
    unsigned long long work_next;    // persistent vote kernel work counter
    unsigned long long n_votes;      // votes appended (may exceed capacity)
    unsigned long long n_chunks;     // vote chunks appended
    unsigned long long n_fit;        // triplets through the full FP32 fit
    unsigned long long n_fp64;       // triplets recomputed in FP64
    unsigned long long n_items;      // work items of the call
    unsigned long long n_triplets;   // sum |La||Lb||Lc|
    unsigned long long n_cand;       // candidates (may exceed capacity)
    unsigned long long n_assign;     // 3 x votes over candidates
    unsigned long long n_hit_ids;    // assigned hit ids
    unsigned long long overflow;     // bit 0 candidate capacity, bit 1 assignment capacity
    unsigned long long n_exact;      // triplets through the exact longitudinal fit
    unsigned long long n_ties;       // bins whose count reaches their box maximum
    unsigned long long pad[1];
    unsigned long long n_cvotes;     // votes in candidate bins (assignment queue length)
    unsigned long long pad2[1];
};

// A run of consecutive votes of one work item in the vote list.
struct VoteChunk {
    int32_t item;
    int32_t count;
    int64_t offset;
};

// A vote is a bin and a code (i << 28) | (j << 24) | k, with i and j the inner and middle
// hit within the work item's tile (tiles are at most 16 x 16) and k the outer hit within
// its layer (< 2^24).  The vote list keeps bins and codes in two arrays of the same slots:
// the assignment streams the bins and reads the codes of candidate votes only.
__host__ __device__ inline uint32_t vote_code(uint32_t i, uint32_t j, uint32_t k)
{
    return (i << 28) | (j << 24) | (k & 0xffffffu);
}
__host__ __device__ inline uint32_t code_i(uint32_t code) { return code >> 28; }
__host__ __device__ inline uint32_t code_j(uint32_t code) { return (code >> 24) & 15u; }
__host__ __device__ inline uint32_t code_k(uint32_t code) { return code & 0xffffffu; }

// Arguments of the vote kernel.
struct VoteArgs {
    const float4 *packed;        // layer-sorted hits: x, y, z, input index (int bits)
    const int32_t *lay_off;      // [event][n_layers + 1] positions in `packed`
    const int64_t *item_off;     // [n_events * n_triples + 1] work-item prefix
    const DevGeo *geo;
    const CallArgs *args;
    int32_t *status;             // per-event status (vote overflow is or-ed in)
    int32_t *hist;               // [event][nbins]
    uint32_t *vote_bin;          // [chunk_cap * 32]
    uint32_t *vote_code;         // [chunk_cap * 32]
    int32_t *chunk_item;         // [chunk_cap] item of each 32-slot chunk (-1: empty)
    int32_t *chunk_count;        // [chunk_cap]
    int32_t *chunk_event;        // [chunk_cap] event of the chunk's item
    int4 *chunk_loc;             // [chunk_cap] packed index of the tile's first inner, middle
                                 // and outer-layer hit, and the item
    int64_t chunk_cap;
    Counters *ctr;
    FitConst C;
};

// Arguments of the assignment kernels.
// Candidate filter: per event, a one-hash Bloom filter of the event's candidate bins, sized
// to sit in one block's shared memory, that lets the assignment skip the random lookup in
// the candidate bitmap for most votes.  A set bit may be a false positive; a candidate's
// bit is always set, so the filter never drops a candidate vote.  A one-event call keeps
// its filter in shared memory; a batch reads the per-event filters (192 KB each, in L2)
// from global memory, so that the false-positive rate does not grow with the batch.
constexpr uint32_t kFilterBits = 192u * 1024u * 8u;
constexpr uint32_t kFilterWords = kFilterBits / 32u;

constexpr uint32_t kFilterEventMul = 0x9E3779B9u;

// The filter bit of (event, bin), with eh = event * kFilterEventMul.
__device__ __forceinline__ uint32_t cand_filter_bit_h(uint32_t eh, uint32_t bin)
{
    // multiplicative (Fibonacci) hashing of the key; the high product bits pick the bit
    return __umulhi((bin ^ eh) * 2654435761u, kFilterBits);
}

__device__ __forceinline__ uint32_t cand_filter_bit(int event, uint32_t bin)
{
    return cand_filter_bit_h((uint32_t)event * kFilterEventMul, bin);
}

struct AssignArgs {
    const uint32_t *vote_bin;
    const uint32_t *vote_code;
    const int32_t *chunk_item;
    const int32_t *chunk_count;
    const int32_t *chunk_event;
    const int4 *chunk_loc;
    int64_t chunk_cap;
    const int64_t *item_off;
    const DevGeo *geo;
    const int32_t *lay_off;
    const CallArgs *args;
    const float4 *packed;
    const int64_t *ev_begin;
    const uint32_t *cbits;
    const uint32_t *filter;      // kFilterWords words
    const uint32_t *wprefix;
    int64_t W;
    const int64_t *vote_off;
    int32_t *fill;
    int32_t *assign;
    int64_t assign_cap;
    unsigned long long *cqueue;  // vote slots of the candidate votes (assignment queue)
    int64_t cqueue_cap;
    int64_t cand_cap;
    Counters *ctr;
    int ti, tj;
};

// ---------------------------------------------------------------------------------------
// FP32 helix fit
// ---------------------------------------------------------------------------------------

// a*d - b*c with one rounding error of the products compensated (Kahan's FMA
// determinant; Jeannerod, Louvet, Muller, Math. Comp. 82 (2013): error <= 2 ulp).
__device__ __forceinline__ float det2(float a, float b, float c, float d)
{
    const float w = b * c;
    const float e = fmaf(-b, c, w);
    const float f = fmaf(a, d, -w);
    return f + e;
}

// Elementwise arithmetic on one value (float) or on two (float2).  The per-hit parts of
// the fit are written once over V and run on float2 for two hits of the same triplet.  The
// packed FP32 instructions of sm_100 and later (add/mul/fma .rn .f32x2; a subtraction is
// the addition of the negated operand, which is exact) round each half exactly as the
// scalar instruction does, and issue once for both.  Square roots, reciprocals,
// transcendentals, comparisons and selections stay per half.
struct M2 {
    bool x, y;
};
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b)
{
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ float2 vabs(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float2 vmin(float2 a, float2 b)
{
    return make_float2(fminf(a.x, b.x), fminf(a.y, b.y));
}
__device__ __forceinline__ bool vle(float a, float b) { return a <= b; }
__device__ __forceinline__ M2 vle(float2 a, float2 b) { return {a.x <= b.x, a.y <= b.y}; }
__device__ __forceinline__ bool vge(float a, float b) { return a >= b; }
__device__ __forceinline__ M2 vge(float2 a, float2 b) { return {a.x >= b.x, a.y >= b.y}; }
__device__ __forceinline__ bool vlt(float a, float b) { return a < b; }
__device__ __forceinline__ M2 vlt(float2 a, float2 b) { return {a.x < b.x, a.y < b.y}; }
__device__ __forceinline__ bool vnot(bool m) { return !m; }
__device__ __forceinline__ M2 vnot(M2 m) { return {!m.x, !m.y}; }
__device__ __forceinline__ float vsel(bool m, float a, float b) { return m ? a : b; }
__device__ __forceinline__ float2 vsel(M2 m, float2 a, float2 b)
{
    return make_float2(m.x ? a.x : b.x, m.y ? a.y : b.y);
}
template <class V> __device__ __forceinline__ V bc(float a);
template <> __device__ __forceinline__ float bc<float>(float a) { return a; }
template <> __device__ __forceinline__ float2 bc<float2>(float a) { return make_float2(a, a); }

// det2 (below) over V: a*d - b*c by Kahan's FMA determinant, per half for float2.
template <class V>
__device__ __forceinline__ V det2v(V a, V b, V c, V d)
{
    const V w = vmul(b, c);
    const V e = vfma(vneg(b), c, w);
    const V f = vfma(a, d, vneg(w));
    return vadd(f, e);
}

// Result of the transverse + longitudinal part of the fit, everything but phi0.
struct FitB {
    float cx, cy;        // circle centre
    float sgn;           // sign(D): +1 counter-clockwise
    float qopt, d0, cot, z0;
};

enum FitStatus { kReject = 0, kPass = 1, kNeedFp64 = 2 };

// Wraps the periodic dimension 0 into [lo, hi); returns false when p is out of range.
__device__ __forceinline__ bool bin_f32(const FitConst &C, int k, float p, uint32_t &idx)
{
    if (k == 0 && (C.periodic & 1)) {
        if (p >= C.hi[0])
            p -= C.period0;
        else if (p < C.lo[0])
            p += C.period0;
    }
    if (!(p >= C.lo[k] && p < C.hi[k]))
        return false;
    int i = (int)floorf((p - C.lo[k]) * C.inv_w[k]);
    i = i < 0 ? 0 : (i >= C.n[k] ? C.n[k] - 1 : i);
    idx = (uint32_t)i;
    return true;
}

__device__ __forceinline__ bool in_range_f32(const FitConst &C, int k, float p)
{
    return p >= C.lo[k] && p < C.hi[k];
}

// Square root and reciprocal through the special-function unit: the PTX instructions
// rsqrt.approx.ftz.f32 and rcp.approx.ftz.f32, one MUFU operation each, with subnormal
// inputs and results flushed to zero (no fix-up instructions around them).  Their errors
// are within 2 ulp, so each result is within about 3e-7 relative, 30 times inside the
// 1e-5 parameter tolerance.  Both the fit and the conservative bounds use them (the
// bounds' margins are 1e-4); correctly rounded square roots and divisions would cost
// several times the instructions in a kernel bound by instruction issue.  Subnormal
// magnitudes (below 1.2e-38) do not occur here: lengths are in mm, and every quantity
// that can vanish (D, |c|) is tested before it is inverted.
__device__ __forceinline__ float mufu_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mufu_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float approx_sqrt(float x)
{
    return x * mufu_rsqrt(fmaxf(x, 1e-30f));
}
__device__ __forceinline__ float approx_rcp(float x) { return mufu_rcp(x); }
__device__ __forceinline__ float approx_div(float a, float b) { return a * mufu_rcp(b); }
__device__ __forceinline__ float2 approx_sqrt(float2 x)
{
    return vmul(x, make_float2(mufu_rsqrt(fmaxf(x.x, 1e-30f)), mufu_rsqrt(fmaxf(x.y, 1e-30f))));
}

// asin(x) for 0 <= x <= 0.75 and atan(x) for 0 <= x <= 1, as x + x t (c1 + c2 t + ...),
// t = x^2: near-minimax polynomials of the relative error in t, degree 8, fitted by
// Lawson's algorithm (iteratively reweighted least squares); gen_minimax.py beside this
// file computes the coefficients and their worst FP32 error (0.89 ulp for the arcsine,
// 1.47 ulp for the arctangent, Horner with fused multiply-adds).  Nine FMAs and two
// multiplies, against the general library functions' range reduction and special cases.
template <class V>
__device__ __forceinline__ V asin_poly(V x)
{
    const V t = vmul(x, x);
    V r = bc<V>(1.939284503e-01f);
    r = vfma(r, t, bc<V>(-2.769452333e-01f));
    r = vfma(r, t, bc<V>(2.225385010e-01f));
    r = vfma(r, t, bc<V>(-5.583249032e-02f));
    r = vfma(r, t, bc<V>(4.723963886e-02f));
    r = vfma(r, t, bc<V>(4.264524207e-02f));
    r = vfma(r, t, bc<V>(7.511704415e-02f));
    r = vfma(r, t, bc<V>(1.666640490e-01f));
    return vfma(vmul(x, t), r, x);
}

__device__ __forceinline__ float atan_poly(float x)
{
    const float t = x * x;
    float r = 2.849888289e-03f;
    r = fmaf(r, t, -1.606862433e-02f);
    r = fmaf(r, t, 4.269151017e-02f);
    r = fmaf(r, t, -7.504294068e-02f);
    r = fmaf(r, t, 1.064093336e-01f);
    r = fmaf(r, t, -1.420364380e-01f);
    r = fmaf(r, t, 1.999261975e-01f);
    r = fmaf(r, t, -3.333307207e-01f);
    return fmaf(x * t, r, x);
}

// atan2(y, x) in [-pi, pi] from atan_poly of min(|x|, |y|) / max(|x|, |y|) (in [0, 1]) and
// the octant: pi/2 - a when |y| > |x|, pi - a when x < 0, the sign of y.  (x, y) = (0, 0)
// gives 0.  pi/2 and pi are added as a float pair (high part + the rounding remainder), so
// the reflections cost no more than the rounding of their sum.
__device__ __forceinline__ float atan2_poly(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float a = atan_poly(mn * mufu_rcp(fmaxf(mx, 1e-30f)));
    float r = ay > ax ? (1.57079637f - a) + -4.37113883e-08f : a;
    r = x < 0.0f ? (3.14159274f - r) + -8.74227766e-08f : r;
    return copysignf(r, y);
}

// Transverse part of the fit: circle, q/pT, d0 and the perigee.
struct Trans {
    float ux, uy, vx, vy, uu, vv;
    float sgn, qopt, d0;
    float cpx, cpy;      // centre - p1
    float cx, cy;        // centre
    float cn;            // |c|
    float R, inv2r;
    float px, py;        // perigee
};

__device__ __forceinline__ int fit_transverse(const float4 &p1, const float4 &p2,
                                              const float4 &p3, const FitConst &C, Trans &t)
{
    // Every quantity is computed for every triplet and the status decided at the end, in
    // the order of the tests (FP64 trigger, q/pT range, d0 range, unusable circle): no
    // early exit, so a warp runs the fit without divergent branches.  Values computed for a
    // triplet whose status is not kPass are meaningless.
    t.ux = p2.x - p1.x;
    t.uy = p2.y - p1.y;
    t.vx = p3.x - p1.x;
    t.vy = p3.y - p1.y;
    const float wx = p3.x - p2.x, wy = p3.y - p2.y;
    const float D = det2(t.ux, t.uy, t.vx, t.vy);
    t.uu = fmaf(t.ux, t.ux, t.uy * t.uy);
    t.vv = fmaf(t.vx, t.vx, t.vy * t.vy);
    const float ww = fmaf(wx, wx, wy * wy);
    const bool need64 = D * D <= C.sag2 * t.vv;
    // q/pT = -sign(D) / (K B R), R = |u||v||w| / (2|D|)
    const float sq = approx_sqrt(t.uu * t.vv * ww);
    const float rq = approx_rcp(sq);
    t.qopt = (-2.0f * D) * rq * C.inv_kB;
    const bool q_ok = in_range_f32(C, 1, t.qopt);
    // centre c = p1 + (v_y|u|^2 - u_y|v|^2, u_x|v|^2 - v_x|u|^2) / (2D)
    const float inv2d = 0.5f * approx_rcp(D);
    t.cpx = det2(t.vy, t.uy, t.vv, t.uu) * inv2d;
    t.cpy = det2(t.ux, t.vx, t.uu, t.vv) * inv2d;
    t.cx = p1.x + t.cpx;
    t.cy = p1.y + t.cpy;
    t.R = sq * fabsf(inv2d);
    t.inv2r = fabsf(D) * rq;
    t.cn = approx_sqrt(fmaf(t.cx, t.cx, t.cy * t.cy));
    // |c| - R = (|c|^2 - R^2) / (|c| + R), |c|^2 - R^2 = |p1|^2 + 2 p1.(c - p1)
    const float power = fmaf(p1.x, p1.x, p1.y * p1.y) + 2.0f * fmaf(p1.x, t.cpx, p1.y * t.cpy);
    const float dist = power * approx_rcp(t.cn + t.R);
    t.sgn = D > 0.0f ? 1.0f : -1.0f;
    t.d0 = t.sgn * dist;
    const bool d_ok = in_range_f32(C, 2, t.d0);
    const bool circle_ok = (t.cn > 0.0f) && (t.R < 3.0e37f);
    // perigee P = c (|c| - R) / |c|
    const float f = dist * approx_rcp(t.cn);
    t.px = t.cx * f;
    t.py = t.cy * f;
    return need64 ? kNeedFp64 : !(q_ok && d_ok) ? kReject : circle_ok ? kPass : kNeedFp64;
}

// Central angle (0 .. pi) of the arc from P to a hit `chord` away, with `sumlen` the
// length of (P - c) + (p - c): 2 asin(chord / 2R) up to x = 0.7, and pi - 2 asin(sumlen /
// 2R) beyond, where the first form is ill-conditioned in FP32.  Both points lie on the
// circle, so chord^2 + sumlen^2 = 4R^2: past x = 0.7 the second argument is below 0.715
// (up to rounding), and both stay inside the [0, 0.75] of asin_poly (the clamp at 0.75
// never binds for points on the circle).
template <class V>
__device__ __forceinline__ V central_angle(V chord, V sumlen, float inv2r)
{
    const V x = vmul(chord, bc<V>(inv2r));
    const auto far = vnot(vle(x, bc<V>(0.7f)));
    const V arg = vsel(far, vmin(vmul(sumlen, bc<V>(inv2r)), bc<V>(0.75f)), x);
    const V h = vmul(bc<V>(2.0f), asin_poly(arg));
    return vsel(far, vsub(bc<V>(3.14159265f), h), h);
}

// Accurate longitudinal part: signed path lengths from P and the least-squares line.
// The path length of the first hit, s_1 = +-R * angle(P - c, p1 - c), is computed
// directly (its error shifts all s alike, which the slope does not see); the others as
// s_1 + R psi_k, psi_k the signed angle from p1 to p_k about the centre taken from the
// exact hit difference e = p_k - p1: 2 asin(|e| / 2R) for short chords, and
// pi - 2 asin(|2b + e| / 2R), b = p1 - c, for long ones (the same central_angle as for
// s_1, one arcsine and no branch); its sign is that of b x e.  s_1 and R psi_k each lie in
// [-pi R, pi R], and so does s_k (a path length from the perigee goes at most half-way
// round), so a turn 2 pi R is removed or added when s_1 + R psi_k falls outside it; where
// rounding decides that, the hit is within 1e-6 pi of the point opposite the perigee, a
// case the definition leaves ambiguous.  The slope stays accurate when a hit with a large
// z residual has little lever.
__device__ __forceinline__ int fit_longitudinal(const float4 &p1, const float4 &p2,
                                                const float4 &p3, const Trans &t,
                                                const FitConst &C, float &cot, float &z0)
{
    const float rcn = approx_rcp(t.cn);
    const float ax = -t.R * t.cx * rcn, ay = -t.R * t.cy * rcn;          // P - c
    const float b0x = -t.cpx, b0y = -t.cpy;                              // p1 - c
    const float dx0 = p1.x - t.px, dy0 = p1.y - t.py;
    const float ch0 = approx_sqrt(fmaf(dx0, dx0, dy0 * dy0));
    const float sx = ax + b0x, sy = ay + b0y;
    const float th0 = central_angle(ch0, approx_sqrt(fmaf(sx, sx, sy * sy)), t.inv2r);
    const float s0 = (t.sgn * det2(dx0, dy0, t.cx, t.cy) >= 0.0f) ? t.R * th0 : -t.R * th0;
    const float turn = 6.2831853f * t.R;
    // hits 2 and 3 as a pair (.x, .y)
    const float2 ex = make_float2(t.ux, t.vx), ey = make_float2(t.uy, t.vy);
    const float2 ee = make_float2(t.uu, t.vv);
    const float2 cr = det2v(bc<float2>(b0x), bc<float2>(b0y), ex, ey);
    // (p1 - c) + (p_k - c) = 2 b + e for the complementary (long-chord) form
    const float2 qx = vfma(bc<float2>(2.0f), bc<float2>(b0x), ex);
    const float2 qy = vfma(bc<float2>(2.0f), bc<float2>(b0y), ey);
    const float2 psi =
        central_angle(approx_sqrt(ee), approx_sqrt(vfma(qx, qx, vmul(qy, qy))), t.inv2r);
    const float2 d = vsel(vge(vmul(bc<float2>(t.sgn), cr), bc<float2>(0.0f)),
                          vmul(bc<float2>(t.R), psi), vmul(bc<float2>(-t.R), psi));
    // s_k - s_1 = R psi_k, less or plus a turn when s_1 + R psi_k leaves [-pi R, pi R]
    const float half_turn = 0.5f * turn;
    const float2 sk = vadd(bc<float2>(s0), d);
    const float2 dl12 =
        vsel(vlt(bc<float2>(half_turn), sk), vsub(d, bc<float2>(turn)),
             vsel(vlt(sk, bc<float2>(-half_turn)), vadd(d, bc<float2>(turn)), d));
    const float dl[3] = {0.0f, dl12.x, dl12.y};
    const float dbar = (dl[1] + dl[2]) * (1.0f / 3.0f);
    const float sbar = s0 + dbar;
    const float zbar = (p1.z + p2.z + p3.z) * (1.0f / 3.0f);
    const float a0 = -dbar, a1 = dl[1] - dbar, a2 = dl[2] - dbar;
    const float sss = fmaf(a0, a0, fmaf(a1, a1, a2 * a2));
    const float ssz = fmaf(a0, p1.z - zbar, fmaf(a1, p2.z - zbar, a2 * (p3.z - zbar)));
    cot = approx_div(ssz, sss);
    z0 = fmaf(-cot, sbar, zbar);
    // status at the end, in the order of the tests (no early exit)
    return !(sss > 0.0f) ? kNeedFp64
                         : (in_range_f32(C, 3, cot) && in_range_f32(C, 4, z0)) ? kPass : kReject;
}

// Everything but phi0 for points p1, p2, p3 (x, y, z in .x .y .z).
__device__ __forceinline__ int fit_stage_b(const float4 &p1, const float4 &p2, const float4 &p3,
                                           const FitConst &C, FitB &r)
{
    Trans t;
    const int st = fit_transverse(p1, p2, p3, C, t);
    if (st != kPass)
        return st;
    float cot, z0;
    const int sl = fit_longitudinal(p1, p2, p3, t, C, cot, z0);
    if (sl != kPass)
        return sl;
    r.cx = t.cx;
    r.cy = t.cy;
    r.sgn = t.sgn;
    r.qopt = t.qopt;
    r.d0 = t.d0;
    r.cot = cot;
    r.z0 = z0;
    return kPass;
}

// phi0 (direction of motion at the perigee: sgn (c_y, -c_x) / |c|) and the bin.
// Returns false if some parameter falls out of range (only possible for phi0 when the
// phi0 range is not periodic).
__device__ __forceinline__ bool fit_stage_c(const FitB &r, const FitConst &C, float &phi0,
                                            uint32_t &bin)
{
    phi0 = atan2_poly(-r.sgn * r.cx, r.sgn * r.cy);
    uint32_t i0, i1, i2, i3, i4;
    if (!bin_f32(C, 0, phi0, i0) || !bin_f32(C, 1, r.qopt, i1) || !bin_f32(C, 2, r.d0, i2) ||
        !bin_f32(C, 3, r.cot, i3) || !bin_f32(C, 4, r.z0, i4))
        return false;
    bin = i0 * C.stride[0] + i1 * C.stride[1] + i2 * C.stride[2] + i3 * C.stride[3] + i4;
    return true;
}

// ---------------------------------------------------------------------------------------
// FP64 recomputation (near-collinear and degenerate FP32 fits)
// ---------------------------------------------------------------------------------------

enum { kFit64Accepted = 1, kFit64Degenerate = 2 };

__device__ __forceinline__ bool bin_f64(const FitConst &C, int k, double p, uint32_t &idx)
{
    if (k == 0 && (C.periodic & 1)) {
        const double period = C.hi_d[0] - C.lo_d[0];
        if (p >= C.hi_d[0])
            p -= period;
        else if (p < C.lo_d[0])
            p += period;
    }
    if (!(p >= C.lo_d[k] && p < C.hi_d[k]))
        return false;
    long long i = (long long)floor((p - C.lo_d[k]) / C.w_d[k]);
    i = i < 0 ? 0 : (i >= C.n[k] ? C.n[k] - 1 : i);
    idx = (uint32_t)i;
    return true;
}

// Full fit in FP64.  Returns kFit64Accepted with par and bin, 0 when out of range,
// kFit64Degenerate when the helix is undefined.
static __device__ __noinline__ int fit_f64(const float4 &q1, const float4 &q2, const float4 &q3,
                                    const FitConst &C, double par[5], uint32_t &bin)
{
    const double x1 = q1.x, y1 = q1.y, z1 = q1.z;
    const double x2 = q2.x, y2 = q2.y, z2 = q2.z;
    const double x3 = q3.x, y3 = q3.y, z3 = q3.z;
    const double ux = x2 - x1, uy = y2 - y1, vx = x3 - x1, vy = y3 - y1;
    const double D = __dsub_rn(__dmul_rn(ux, vy), __dmul_rn(uy, vx));
    double phi0, qopt, d0, px, py, R;
    const bool straight = (D == 0.0);
    if (!straight) {
        const double uu = __dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy));
        const double vv = __dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy));
        const double cpx = __dsub_rn(__dmul_rn(vy, uu), __dmul_rn(uy, vv)) / (2.0 * D);
        const double cpy = __dsub_rn(__dmul_rn(ux, vv), __dmul_rn(vx, uu)) / (2.0 * D);
        const double cx = x1 + cpx, cy = y1 + cpy;
        const double sgn = D > 0.0 ? 1.0 : -1.0;
        R = sqrt(__dadd_rn(__dmul_rn(cpx, cpx), __dmul_rn(cpy, cpy)));
        qopt = -sgn / (C.kB_d * R);
        const double cn = sqrt(__dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy)));
        if (cn == 0.0)
            return kFit64Degenerate;
        const double power = __dadd_rn(__dadd_rn(__dmul_rn(x1, x1), __dmul_rn(y1, y1)),
                                       2.0 * __dadd_rn(__dmul_rn(x1, cpx), __dmul_rn(y1, cpy)));
        const double cmr = power / (cn + R);
        px = cx * (cmr / cn);
        py = cy * (cmr / cn);
        phi0 = atan2(-sgn * cx, sgn * cy);
        d0 = __dadd_rn(__dmul_rn(-px, sin(phi0)), __dmul_rn(py, cos(phi0)));
    } else {
        const double vn = sqrt(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)));
        if (vn == 0.0)
            return kFit64Degenerate;
        const double tx = vx / vn, ty = vy / vn;
        const double along = __dadd_rn(__dmul_rn(x1, tx), __dmul_rn(y1, ty));
        px = x1 - along * tx;
        py = y1 - along * ty;
        phi0 = atan2(vy, vx);
        d0 = __dadd_rn(__dmul_rn(-px, sin(phi0)), __dmul_rn(py, cos(phi0)));
        qopt = 0.0;
        R = 0.0;
    }
    const double xs[3] = {x1, x2, x3}, ys[3] = {y1, y2, y3}, zs[3] = {z1, z2, z3};
    const double tx = cos(phi0), ty = sin(phi0);
    double s[3];
    for (int k = 0; k < 3; ++k) {
        const double dx = xs[k] - px, dy = ys[k] - py;
        const double chord = sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
        // signed path length: negative before the perigee in the direction of motion
        const double sign = __dadd_rn(__dmul_rn(dx, tx), __dmul_rn(dy, ty)) >= 0.0 ? 1.0 : -1.0;
        if (straight) {
            s[k] = sign * chord;
        } else {
            double a = chord / (2.0 * R);
            a = a > 1.0 ? 1.0 : a;
            s[k] = sign * (2.0 * R * asin(a));
        }
    }
    const double sbar = (s[0] + s[1] + s[2]) / 3.0;
    const double zbar = (zs[0] + zs[1] + zs[2]) / 3.0;
    double sss = 0.0, ssz = 0.0;
    for (int k = 0; k < 3; ++k) {
        sss = __dadd_rn(sss, __dmul_rn(s[k] - sbar, s[k] - sbar));
        ssz = __dadd_rn(ssz, __dmul_rn(s[k] - sbar, zs[k] - zbar));
    }
    if (sss == 0.0)
        return kFit64Degenerate;
    const double cot = ssz / sss;
    const double z0 = __dsub_rn(zbar, __dmul_rn(cot, sbar));
    par[0] = phi0;
    par[1] = qopt;
    par[2] = d0;
    par[3] = cot;
    par[4] = z0;
    uint32_t idx[5];
    for (int k = 0; k < 5; ++k)
        if (!bin_f64(C, k, par[k], idx[k]))
            return 0;
    bin = idx[0] * C.stride[0] + idx[1] * C.stride[1] + idx[2] * C.stride[2] +
          idx[3] * C.stride[3] + idx[4];
    return kFit64Accepted;
}

// ---------------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------------

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Largest f with off[f] <= x for a non-decreasing off[0..n] (off[0] <= x < off[n]).
__device__ __forceinline__ int upper_index(const int64_t *off, int n, int64_t x)
{
    int lo = 0, hi = n;   // invariant off[lo] <= x < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= x)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

}  // namespace trk
