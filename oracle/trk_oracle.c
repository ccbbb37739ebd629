/*
 * FP64 CPU oracle of the displaced-track Hough transform.  TEST INFRASTRUCTURE ONLY:
 * it is linked by the tests, by the entry point's smoke check and by the benchmark's CPU
 * baseline leg, and by nothing on the product path.  It shares no code, header or
 * constant with the CUDA library.
 *
 * What it computes (plain definition, no blocking, no pruning, no reordering):
 *   for every event, every listed layer triple (a, b, c), every hit i of layer a, j of
 *   layer b, k of layer c (input order), in double precision from the float32 hits:
 *     1. the circle through the three transverse points, its signed curvature and the
 *        helix perigee parameters (phi0, q/pT, d0) about the coordinate origin
 *        (no beam-spot constraint), the arc lengths s_k from the perigee and the
 *        unweighted least-squares line z = z0 + s cot(theta) over the three (s_k, z_k);
 *     2. the five bin indices; the triplet is accepted iff all five parameters lie in
 *        range, and then votes once into bin (phi0, q/pT, d0, cot, z0), row-major;
 *     3. ambiguity flags: some parameter lies within eps of a bin edge or range limit,
 *        eps = eps_rel * max(|p|, half-range) (bit 0), the triplet is rejected only by
 *        parameters within eps outside their ranges (bit 1), or a hit lies within
 *        eps_rel * pi of the point of the circle opposite the perigee (bit 2).
 *
 * Paper: Sec. 7 and Fig. 3 (each hit set maps to many parameter points, votes are
 * accumulated, peaks are tracks); Sec. 8 (curved features need more parameters,
 * circles by centre and radius; curved displaced tracks need a space beyond the
 * two-parameter interaction-point-constrained one).  The helix parameterisation,
 * the sign conventions, the arc length and the longitudinal fit are not given in the
 * paper; they are the stated readings:
 *   - pT = K B R, K = 0.299792458e-2 GeV/(T cm); positive charges turn clockwise
 *     seen from +z, so q = -sign(D) with D = (p2-p1) x (p3-p1), q/pT = -sign(D)/(K B R);
 *   - centre c = p1 + (v_y|u|^2 - u_y|v|^2, u_x|v|^2 - v_x|u|^2) / (2D), R = |c - p1|;
 *   - perigee P = c (1 - R/|c|); phi0 = direction of motion at P, in [-pi, pi);
 *     d0 = -P_x sin(phi0) + P_y cos(phi0); |c| - R is evaluated as
 *     (|c|^2 - R^2)/(|c| + R) with |c|^2 - R^2 = |p1|^2 + 2 p1.(c - p1) (an identity,
 *     used because the direct difference of two large numbers loses all digits);
 *   - D == 0: straight line through p1 and p3, q/pT = 0, P the foot of the normal;
 *   - s_k = +-2R asin(|p_k - P| / (2R)) (+-|p_k - P| on a straight line): the path length
 *     from the perigee, positive for a hit after P in the direction of motion and negative
 *     for one before it (the sign of (p_k - P) . (cos phi0, sin phi0), + when it is 0),
 *     so that z = z0 + s cot(theta) holds on both branches of the helix through P;
 *     a hit within eps of the point opposite P (where that sign is undefined) makes the
 *     triplet ambiguous;
 *   - bins: idx = floor((p - lo) / ((hi - lo)/n)), accepted iff lo <= p < hi; a periodic
 *     dimension is wrapped into [lo, hi) first.
 * Degenerate triplets (circle centred on the origin, or three equal arc lengths) have
 * no perigee or no slope and are rejected and counted.
 *
 * The candidate fit (orc_fit_track, orc_fit_tracks) is defined further down, with its own
 * readings.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_K 0.299792458e-2
#define ORC_PI 3.14159265358979323846

typedef struct {
    float x, y, z;
    int32_t layer;
} orc_hit;

typedef struct {
    double b_tesla;
    int32_t n_layers;
    int32_t n_triples;
    const int32_t *triples; /* n_triples x 3 layer ids */
    double lo[5], hi[5];
    int32_t n[5];
    int32_t periodic;       /* bit k set: dimension k is periodic */
    double eps_rel;
} orc_setup;

typedef struct {
    int64_t n_acc;          /* accepted triplets */
    int32_t *acc_event;     /* [n_acc] */
    int32_t *acc_ijk;       /* [n_acc * 3] input hit indices (global) */
    uint64_t *acc_bin;      /* [n_acc] row-major bin inside the event's histogram */
    uint8_t *acc_amb;       /* [n_acc] ambiguity bits (1 edge, 4 antipode) */
    double *acc_par;        /* [n_acc * 5] */
    int64_t n_near;         /* rejected, but every out-of-range parameter within eps, or
                               antipode-ambiguous */
    int32_t *near_event;
    int32_t *near_ijk;
    int64_t n_triplets;     /* sum over events and triples of |La||Lb||Lc| */
    int64_t n_degenerate;
} orc_result;

enum { ORC_OK = 0, ORC_DEGENERATE = 1 };

/* Helix of the triplet.  Returns ORC_OK and par = (phi0, q/pT, d0, cot, z0), or
 * ORC_DEGENERATE. */
int orc_fit_flags(const double *p1, const double *p2, const double *p3, double b_tesla,
                  double eps_rel, double *par, int *antipode)
{
    *antipode = 0;
    const double ux = p2[0] - p1[0], uy = p2[1] - p1[1];
    const double vx = p3[0] - p1[0], vy = p3[1] - p1[1];
    const double D = ux * vy - uy * vx;
    double phi0, qopt, d0, px, py, R;
    int straight = (D == 0.0);
    if (!straight) {
        const double uu = ux * ux + uy * uy, vv = vx * vx + vy * vy;
        const double cpx = (vy * uu - uy * vv) / (2.0 * D);
        const double cpy = (ux * vv - vx * uu) / (2.0 * D);
        const double cx = p1[0] + cpx, cy = p1[1] + cpy;
        const double sgn = D > 0.0 ? 1.0 : -1.0;
        R = sqrt(cpx * cpx + cpy * cpy);
        qopt = -sgn / (ORC_K * b_tesla * R);
        const double cn = sqrt(cx * cx + cy * cy);
        if (cn == 0.0)
            return ORC_DEGENERATE;
        const double power = (p1[0] * p1[0] + p1[1] * p1[1]) + 2.0 * (p1[0] * cpx + p1[1] * cpy);
        const double cn_minus_r = power / (cn + R);
        px = cx * (cn_minus_r / cn);
        py = cy * (cn_minus_r / cn);
        /* direction of motion at P: counter-clockwise (D > 0) is z x (P - c), and
         * P - c points from c towards the origin, so the tangent is sgn (c_y, -c_x)/|c| */
        phi0 = atan2(-sgn * cx, sgn * cy);
        d0 = -px * sin(phi0) + py * cos(phi0);
    } else {
        const double vn = sqrt(vx * vx + vy * vy);
        if (vn == 0.0)
            return ORC_DEGENERATE;
        const double tx = vx / vn, ty = vy / vn;
        const double along = p1[0] * tx + p1[1] * ty;
        px = p1[0] - along * tx;
        py = p1[1] - along * ty;
        phi0 = atan2(vy, vx);
        d0 = -px * sin(phi0) + py * cos(phi0);
        qopt = 0.0;
        R = INFINITY;
    }
    const double *pk[3] = {p1, p2, p3};
    const double tx = cos(phi0), ty = sin(phi0);
    double s[3];
    for (int k = 0; k < 3; ++k) {
        const double dx = pk[k][0] - px, dy = pk[k][1] - py;
        const double chord = sqrt(dx * dx + dy * dy);
        const double sign = (dx * tx + dy * ty) >= 0.0 ? 1.0 : -1.0;
        if (straight) {
            s[k] = sign * chord;
        } else {
            double a = chord / (2.0 * R);
            if (a > 1.0)
                a = 1.0;
            const double half_angle = asin(a);
            if (2.0 * half_angle >= ORC_PI * (1.0 - eps_rel))
                *antipode = 1;
            s[k] = sign * 2.0 * R * half_angle;
        }
    }
    const double sbar = (s[0] + s[1] + s[2]) / 3.0;
    const double zbar = (p1[2] + p2[2] + p3[2]) / 3.0;
    double sss = 0.0, ssz = 0.0;
    for (int k = 0; k < 3; ++k) {
        sss += (s[k] - sbar) * (s[k] - sbar);
        ssz += (s[k] - sbar) * (pk[k][2] - zbar);
    }
    if (sss == 0.0)
        return ORC_DEGENERATE;
    const double cot = ssz / sss;
    const double z0 = zbar - cot * sbar;
    par[0] = phi0;
    par[1] = qopt;
    par[2] = d0;
    par[3] = cot;
    par[4] = z0;
    return ORC_OK;
}

/* Helix of the triplet (see orc_fit_flags), without the antipode flag. */
int orc_fit(const double *p1, const double *p2, const double *p3, double b_tesla, double *par)
{
    int anti;
    return orc_fit_flags(p1, p2, p3, b_tesla, 1e-5, par, &anti);
}

/* Bin the parameters.  Returns 1 if accepted (all in range) with *bin set; sets *amb if
 * some parameter is within eps of an edge or range limit; *near = rejected but every
 * out-of-range parameter is within eps of its range limit. */
int orc_bin(const orc_setup *s, const double *par_in, uint64_t *bin, int *amb, int *near)
{
    int inside = 1, all_close = 1;
    uint64_t lin = 0;
    *amb = 0;
    for (int k = 0; k < 5; ++k) {
        double p = par_in[k];
        const double lo = s->lo[k], hi = s->hi[k];
        const double w = (hi - lo) / (double)s->n[k];
        if ((s->periodic >> k) & 1) {
            const double period = hi - lo;
            while (p >= hi)
                p -= period;
            while (p < lo)
                p += period;
        }
        const double half = 0.5 * (hi - lo);
        const double eps = s->eps_rel * (fabs(p) > half ? fabs(p) : half);
        int64_t idx;
        if (p < lo || p >= hi) {
            inside = 0;
            const double d = p < lo ? lo - p : p - hi;
            if (d > eps)
                all_close = 0;
            else
                *amb = 1;
            idx = 0;
        } else {
            const double t = (p - lo) / w;
            idx = (int64_t)floor(t);
            if (idx >= s->n[k])
                idx = s->n[k] - 1;
            const double below = t - floor(t), above = ceil(t) - t;
            const double dedge = (below < above ? below : above) * w;
            if (dedge <= eps)
                *amb = 1;
        }
        lin = lin * (uint64_t)s->n[k] + (uint64_t)idx;
    }
    *bin = lin;
    *near = (!inside) && all_close;
    return inside;
}

typedef struct {
    int64_t n, cap;
    int32_t *ijk;
    uint64_t *bin;
    uint8_t *amb;
    double *par;
    int64_t nn, ncap;
    int32_t *near_ijk;
    int64_t n_degenerate;
} unit_buf;

static void ub_push_acc(unit_buf *b, int32_t i, int32_t j, int32_t k, uint64_t bin, int amb,
                        const double *par)
{
    if (b->n == b->cap) {
        b->cap = b->cap ? 2 * b->cap : 64;
        b->ijk = realloc(b->ijk, (size_t)b->cap * 3 * sizeof(int32_t));
        b->bin = realloc(b->bin, (size_t)b->cap * sizeof(uint64_t));
        b->amb = realloc(b->amb, (size_t)b->cap);
        b->par = realloc(b->par, (size_t)b->cap * 5 * sizeof(double));
    }
    b->ijk[3 * b->n] = i;
    b->ijk[3 * b->n + 1] = j;
    b->ijk[3 * b->n + 2] = k;
    b->bin[b->n] = bin;
    b->amb[b->n] = (uint8_t)amb;
    memcpy(b->par + 5 * b->n, par, 5 * sizeof(double));
    b->n++;
}

static void ub_push_near(unit_buf *b, int32_t i, int32_t j, int32_t k)
{
    if (b->nn == b->ncap) {
        b->ncap = b->ncap ? 2 * b->ncap : 16;
        b->near_ijk = realloc(b->near_ijk, (size_t)b->ncap * 3 * sizeof(int32_t));
    }
    b->near_ijk[3 * b->nn] = i;
    b->near_ijk[3 * b->nn + 1] = j;
    b->near_ijk[3 * b->nn + 2] = k;
    b->nn++;
}

/* Run the whole definition over a batch of events.  Output order: event, layer triple
 * (list order), i, j, k (input order within each layer) -- independent of the thread
 * count.  Returns 0, or -1 on invalid input (layer id out of range, bad offsets). */
int orc_run(const orc_hit *hits, int64_t n_hits, const int64_t *offsets, int32_t n_events,
            const orc_setup *s, int32_t n_threads, orc_result *res)
{
    memset(res, 0, sizeof(*res));
    if (offsets[0] != 0 || offsets[n_events] != n_hits)
        return -1;
    for (int32_t e = 0; e < n_events; ++e)
        if (offsets[e + 1] < offsets[e])
            return -1;
    for (int64_t h = 0; h < n_hits; ++h)
        if (hits[h].layer < 0 || hits[h].layer >= s->n_layers)
            return -1;

    /* per event, per layer: the input indices of the layer's hits, in input order */
    const int L = s->n_layers;
    int64_t *lay_off = calloc((size_t)n_events * (L + 1), sizeof(int64_t));
    int32_t *lay_idx = malloc((size_t)(n_hits > 0 ? n_hits : 1) * sizeof(int32_t));
    for (int32_t e = 0; e < n_events; ++e) {
        int64_t *lo = lay_off + (size_t)e * (L + 1);
        for (int64_t h = offsets[e]; h < offsets[e + 1]; ++h)
            lo[hits[h].layer + 1]++;
        lo[0] = offsets[e];
        for (int l = 0; l < L; ++l)
            lo[l + 1] += lo[l];
        int64_t *fill = malloc((size_t)L * sizeof(int64_t));
        for (int l = 0; l < L; ++l)
            fill[l] = lo[l];
        for (int64_t h = offsets[e]; h < offsets[e + 1]; ++h)
            lay_idx[fill[hits[h].layer]++] = (int32_t)h;
        free(fill);
    }

    /* work units: (event, triple, inner hit) in output order */
    int64_t n_units = 0;
    for (int32_t e = 0; e < n_events; ++e)
        for (int t = 0; t < s->n_triples; ++t) {
            const int a = s->triples[3 * t], b = s->triples[3 * t + 1], c = s->triples[3 * t + 2];
            const int64_t *lo = lay_off + (size_t)e * (L + 1);
            const int64_t na = lo[a + 1] - lo[a], nb = lo[b + 1] - lo[b], nc = lo[c + 1] - lo[c];
            n_units += na;
            res->n_triplets += na * nb * nc;
        }
    int32_t *u_event = malloc((size_t)(n_units ? n_units : 1) * sizeof(int32_t));
    int32_t *u_triple = malloc((size_t)(n_units ? n_units : 1) * sizeof(int32_t));
    int64_t *u_i = malloc((size_t)(n_units ? n_units : 1) * sizeof(int64_t));
    {
        int64_t u = 0;
        for (int32_t e = 0; e < n_events; ++e)
            for (int t = 0; t < s->n_triples; ++t) {
                const int a = s->triples[3 * t];
                const int64_t *lo = lay_off + (size_t)e * (L + 1);
                for (int64_t i = lo[a]; i < lo[a + 1]; ++i) {
                    u_event[u] = e;
                    u_triple[u] = t;
                    u_i[u] = i;
                    ++u;
                }
            }
    }
    unit_buf *ub = calloc((size_t)(n_units ? n_units : 1), sizeof(unit_buf));

#ifdef _OPENMP
    if (n_threads > 0)
        omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t u = 0; u < n_units; ++u) {
        const int32_t e = u_event[u];
        const int t = u_triple[u];
        const int b = s->triples[3 * t + 1], c = s->triples[3 * t + 2];
        const int64_t *lo = lay_off + (size_t)e * (L + 1);
        const int32_t hi_ = lay_idx[u_i[u]];
        const double p1[3] = {hits[hi_].x, hits[hi_].y, hits[hi_].z};
        unit_buf *buf = ub + u;
        for (int64_t jj = lo[b]; jj < lo[b + 1]; ++jj) {
            const int32_t hj = lay_idx[jj];
            const double p2[3] = {hits[hj].x, hits[hj].y, hits[hj].z};
            for (int64_t kk = lo[c]; kk < lo[c + 1]; ++kk) {
                const int32_t hk = lay_idx[kk];
                const double p3[3] = {hits[hk].x, hits[hk].y, hits[hk].z};
                double par[5];
                int anti;
                if (orc_fit_flags(p1, p2, p3, s->b_tesla, s->eps_rel, par, &anti) != ORC_OK) {
                    buf->n_degenerate++;
                    continue;
                }
                uint64_t bin;
                int amb, near;
                if (orc_bin(s, par, &bin, &amb, &near))
                    ub_push_acc(buf, hi_, hj, hk, bin, amb | (anti ? 4 : 0), par);
                else if (near || anti)
                    ub_push_near(buf, hi_, hj, hk);
            }
        }
    }

    int64_t n_acc = 0, n_near = 0;
    for (int64_t u = 0; u < n_units; ++u) {
        n_acc += ub[u].n;
        n_near += ub[u].nn;
        res->n_degenerate += ub[u].n_degenerate;
    }
    res->n_acc = n_acc;
    res->n_near = n_near;
    res->acc_event = malloc((size_t)(n_acc ? n_acc : 1) * sizeof(int32_t));
    res->acc_ijk = malloc((size_t)(n_acc ? n_acc : 1) * 3 * sizeof(int32_t));
    res->acc_bin = malloc((size_t)(n_acc ? n_acc : 1) * sizeof(uint64_t));
    res->acc_amb = malloc((size_t)(n_acc ? n_acc : 1));
    res->acc_par = malloc((size_t)(n_acc ? n_acc : 1) * 5 * sizeof(double));
    res->near_event = malloc((size_t)(n_near ? n_near : 1) * sizeof(int32_t));
    res->near_ijk = malloc((size_t)(n_near ? n_near : 1) * 3 * sizeof(int32_t));
    int64_t pa = 0, pn = 0;
    for (int64_t u = 0; u < n_units; ++u) {
        unit_buf *b = ub + u;
        for (int64_t q = 0; q < b->n; ++q)
            res->acc_event[pa + q] = u_event[u];
        if (b->n) {
            memcpy(res->acc_ijk + 3 * pa, b->ijk, (size_t)b->n * 3 * sizeof(int32_t));
            memcpy(res->acc_bin + pa, b->bin, (size_t)b->n * sizeof(uint64_t));
            memcpy(res->acc_amb + pa, b->amb, (size_t)b->n);
            memcpy(res->acc_par + 5 * pa, b->par, (size_t)b->n * 5 * sizeof(double));
        }
        for (int64_t q = 0; q < b->nn; ++q)
            res->near_event[pn + q] = u_event[u];
        if (b->nn)
            memcpy(res->near_ijk + 3 * pn, b->near_ijk, (size_t)b->nn * 3 * sizeof(int32_t));
        pa += b->n;
        pn += b->nn;
        free(b->ijk);
        free(b->bin);
        free(b->amb);
        free(b->par);
        free(b->near_ijk);
    }
    free(ub);
    free(u_event);
    free(u_triple);
    free(u_i);
    free(lay_off);
    free(lay_idx);
    return 0;
}

void orc_result_free(orc_result *res)
{
    free(res->acc_event);
    free(res->acc_ijk);
    free(res->acc_bin);
    free(res->acc_amb);
    free(res->acc_par);
    free(res->near_event);
    free(res->near_ijk);
    memset(res, 0, sizeof(*res));
}

/* Fit and bin an explicit list of triplets (input hit indices), for sampled checks at
 * sizes the full enumeration cannot reach.  status[t]: 0 accepted, 1 rejected,
 * 2 degenerate; amb[t] ambiguity bits (1 edge, 2 near a range limit, 4 antipode);
 * par/bin filled when not degenerate. */
void orc_fit_list(const orc_hit *hits, const int32_t *ijk, int64_t n, const orc_setup *s,
                  int32_t n_threads, double *par, uint64_t *bin, int32_t *status,
                  uint8_t *amb)
{
#ifdef _OPENMP
    if (n_threads > 0)
        omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t t = 0; t < n; ++t) {
        const orc_hit *a = hits + ijk[3 * t], *b = hits + ijk[3 * t + 1], *c = hits + ijk[3 * t + 2];
        const double p1[3] = {a->x, a->y, a->z}, p2[3] = {b->x, b->y, b->z},
                     p3[3] = {c->x, c->y, c->z};
        int anti;
        if (orc_fit_flags(p1, p2, p3, s->b_tesla, s->eps_rel, par + 5 * t, &anti) != ORC_OK) {
            status[t] = 2;
            amb[t] = 0;
            bin[t] = 0;
            continue;
        }
        int am, near;
        const int acc = orc_bin(s, par + 5 * t, bin + t, &am, &near);
        status[t] = acc ? 0 : 1;
        amb[t] = (uint8_t)((am ? 1 : 0) | (near ? 2 : 0) | (anti ? 4 : 0));
    }
}

/* ---------------------------------------------------------------------------------------
 * The same definition restricted in its OUTPUT to blocks of the parameter space, for events
 * whose accepted-triplet list does not fit in memory.  Every triplet of the event is fitted
 * and binned exactly as in orc_run (same functions, same order within a work unit); only
 * what is kept afterwards differs.  A block is one (phi0 row, q/pT row) pair of bin indices
 * (i0, i1), holding the n2 * n3 * n4 bins that share them.  Per block:
 *   count_slot[i0 * n1 + i1] >= 0: the block's votes are counted in
 *       counts[slot * (n2 n3 n4) + (bin mod n2 n3 n4)];
 *   keep_sel: accepted triplets voting in the block are listed (hit indices and bin);
 *   flip_sel: accepted triplets voting in the block with a parameter within eps of a bin
 *       edge are listed (for explaining FP32 bin flips).
 * Rejected triplets whose out-of-range parameters all lie within eps of their range limits
 * (near-accepted), and triplets with a hit at the point opposite the perigee, are listed
 * wherever they fall.  One event per call.
 * --------------------------------------------------------------------------------------- */
typedef struct {
    int64_t n_keep;
    int32_t *keep_ijk;      /* [3 n_keep] input hit indices */
    uint64_t *keep_bin;
    int64_t n_flip;
    int32_t *flip_ijk;      /* [3 n_flip] */
    uint64_t *flip_bin;     /* the oracle's bin (accepted) or 0 (rejected) */
    uint8_t *flip_acc;      /* 1 accepted by the oracle, 0 rejected */
    int64_t n_triplets;
    int64_t n_degenerate;
} orc_block_result;

typedef struct {
    int64_t n, cap;
    int32_t *ijk;
    uint64_t *bin;
    uint8_t *acc;
} blk_buf;

static void blk_push(blk_buf *b, int32_t i, int32_t j, int32_t k, uint64_t bin, int acc)
{
    if (b->n == b->cap) {
        b->cap = b->cap ? 2 * b->cap : 64;
        b->ijk = realloc(b->ijk, (size_t)b->cap * 3 * sizeof(int32_t));
        b->bin = realloc(b->bin, (size_t)b->cap * sizeof(uint64_t));
        b->acc = realloc(b->acc, (size_t)b->cap);
    }
    b->ijk[3 * b->n] = i;
    b->ijk[3 * b->n + 1] = j;
    b->ijk[3 * b->n + 2] = k;
    b->bin[b->n] = bin;
    b->acc[b->n] = (uint8_t)acc;
    b->n++;
}

static void blk_flatten(blk_buf *bufs, int64_t n_units, int64_t *n_out, int32_t **ijk,
                        uint64_t **bin, uint8_t **acc)
{
    int64_t n = 0;
    for (int64_t u = 0; u < n_units; ++u)
        n += bufs[u].n;
    *n_out = n;
    *ijk = malloc((size_t)(n ? n : 1) * 3 * sizeof(int32_t));
    *bin = malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
    if (acc)
        *acc = malloc((size_t)(n ? n : 1));
    int64_t p = 0;
    for (int64_t u = 0; u < n_units; ++u) {
        blk_buf *b = bufs + u;
        if (b->n) {
            memcpy(*ijk + 3 * p, b->ijk, (size_t)b->n * 3 * sizeof(int32_t));
            memcpy(*bin + p, b->bin, (size_t)b->n * sizeof(uint64_t));
            if (acc)
                memcpy(*acc + p, b->acc, (size_t)b->n);
        }
        p += b->n;
        free(b->ijk);
        free(b->bin);
        free(b->acc);
    }
}

int orc_run_blocks(const orc_hit *hits, int64_t n_hits, const int64_t *offsets, int32_t n_events,
                   const orc_setup *s, int32_t n_threads, const int32_t *count_slot,
                   const uint8_t *keep_sel, const uint8_t *flip_sel, int32_t *counts,
                   orc_block_result *res)
{
    memset(res, 0, sizeof(*res));
    if (n_events != 1 || offsets[0] != 0 || offsets[1] != n_hits)
        return -1;
    for (int64_t h = 0; h < n_hits; ++h)
        if (hits[h].layer < 0 || hits[h].layer >= s->n_layers)
            return -1;
    const int L = s->n_layers;
    const uint64_t inner = (uint64_t)s->n[2] * s->n[3] * s->n[4];
    /* the layer lists, in input order */
    int64_t *lo = calloc((size_t)L + 1, sizeof(int64_t));
    int32_t *lay_idx = malloc((size_t)(n_hits > 0 ? n_hits : 1) * sizeof(int32_t));
    for (int64_t h = 0; h < n_hits; ++h)
        lo[hits[h].layer + 1]++;
    for (int l = 0; l < L; ++l)
        lo[l + 1] += lo[l];
    {
        int64_t *fill = malloc((size_t)L * sizeof(int64_t));
        for (int l = 0; l < L; ++l)
            fill[l] = lo[l];
        for (int64_t h = 0; h < n_hits; ++h)
            lay_idx[fill[hits[h].layer]++] = (int32_t)h;
        free(fill);
    }
    /* work units: (triple, inner hit) */
    int64_t n_units = 0;
    for (int t = 0; t < s->n_triples; ++t) {
        const int a = s->triples[3 * t], b = s->triples[3 * t + 1], c = s->triples[3 * t + 2];
        n_units += lo[a + 1] - lo[a];
        res->n_triplets += (lo[a + 1] - lo[a]) * (lo[b + 1] - lo[b]) * (lo[c + 1] - lo[c]);
    }
    int32_t *u_triple = malloc((size_t)(n_units ? n_units : 1) * sizeof(int32_t));
    int64_t *u_i = malloc((size_t)(n_units ? n_units : 1) * sizeof(int64_t));
    {
        int64_t u = 0;
        for (int t = 0; t < s->n_triples; ++t) {
            const int a = s->triples[3 * t];
            for (int64_t i = lo[a]; i < lo[a + 1]; ++i) {
                u_triple[u] = t;
                u_i[u] = i;
                ++u;
            }
        }
    }
    blk_buf *kb = calloc((size_t)(n_units ? n_units : 1), sizeof(blk_buf));
    blk_buf *fb = calloc((size_t)(n_units ? n_units : 1), sizeof(blk_buf));
    int64_t n_deg = 0;
#ifdef _OPENMP
    if (n_threads > 0)
        omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : n_deg)
#endif
    for (int64_t u = 0; u < n_units; ++u) {
        const int t = u_triple[u];
        const int b = s->triples[3 * t + 1], c = s->triples[3 * t + 2];
        const int32_t hi_ = lay_idx[u_i[u]];
        const double p1[3] = {hits[hi_].x, hits[hi_].y, hits[hi_].z};
        for (int64_t jj = lo[b]; jj < lo[b + 1]; ++jj) {
            const int32_t hj = lay_idx[jj];
            const double p2[3] = {hits[hj].x, hits[hj].y, hits[hj].z};
            for (int64_t kk = lo[c]; kk < lo[c + 1]; ++kk) {
                const int32_t hk = lay_idx[kk];
                const double p3[3] = {hits[hk].x, hits[hk].y, hits[hk].z};
                double par[5];
                int anti;
                if (orc_fit_flags(p1, p2, p3, s->b_tesla, s->eps_rel, par, &anti) != ORC_OK) {
                    n_deg++;
                    continue;
                }
                uint64_t bin;
                int amb, near;
                const int acc = orc_bin(s, par, &bin, &amb, &near);
                if (acc) {
                    const uint64_t blk = bin / inner;
                    const int32_t slot = count_slot[blk];
                    if (slot >= 0) {
#ifdef _OPENMP
#pragma omp atomic
#endif
                        counts[(uint64_t)slot * inner + bin % inner]++;
                    }
                    if (keep_sel[blk])
                        blk_push(kb + u, hi_, hj, hk, bin, 1);
                    if ((amb || anti) && (flip_sel[blk] || anti))
                        blk_push(fb + u, hi_, hj, hk, bin, 1);
                } else if (near || anti) {
                    blk_push(fb + u, hi_, hj, hk, 0, 0);
                }
            }
        }
    }
    res->n_degenerate = n_deg;
    blk_flatten(kb, n_units, &res->n_keep, &res->keep_ijk, &res->keep_bin, NULL);
    blk_flatten(fb, n_units, &res->n_flip, &res->flip_ijk, &res->flip_bin, &res->flip_acc);
    free(kb);
    free(fb);
    free(u_triple);
    free(u_i);
    free(lo);
    free(lay_idx);
    return 0;
}

void orc_block_result_free(orc_block_result *res)
{
    free(res->keep_ijk);
    free(res->keep_bin);
    free(res->flip_ijk);
    free(res->flip_bin);
    free(res->flip_acc);
    memset(res, 0, sizeof(*res));
}

/* The peak rule (Sec. 7 and Fig. 3: candidates are local maxima of the parameter space,
 * with the stated threshold and tie-break) for every bin of the keep blocks, from block
 * counts laid out as orc_run_blocks writes them.  Every neighbour block of a keep block must
 * be counted.  Writes candidates in increasing bin order; returns their number, or -1 if a
 * needed neighbour block is not counted, or -2 if cap is too small. */
int64_t orc_block_peaks(const orc_setup *s, const int32_t *count_slot, const int32_t *counts,
                        const uint8_t *keep_sel, int32_t threshold, uint64_t *out_bin,
                        int32_t *out_votes, int64_t cap)
{
    const int n0 = s->n[0], n1 = s->n[1], n2 = s->n[2], n3 = s->n[3], n4 = s->n[4];
    const uint64_t inner = (uint64_t)n2 * n3 * n4;
    int64_t nc = 0;
    for (int i0 = 0; i0 < n0; ++i0)
        for (int i1 = 0; i1 < n1; ++i1) {
            if (!keep_sel[i0 * n1 + i1])
                continue;
            const int32_t slot = count_slot[i0 * n1 + i1];
            if (slot < 0)
                return -1;
            for (uint64_t r = 0; r < inner; ++r) {
                const int32_t h = counts[(uint64_t)slot * inner + r];
                if (h < threshold)
                    continue;
                const int i2 = (int)(r / ((uint64_t)n3 * n4));
                const int i3 = (int)((r / (uint64_t)n4) % (uint64_t)n3);
                const int i4 = (int)(r % (uint64_t)n4);
                const uint64_t bin = ((uint64_t)i0 * n1 + (uint64_t)i1) * inner + r;
                int is_peak = 1;
                for (int d0 = -1; d0 <= 1 && is_peak; ++d0)
                    for (int d1 = -1; d1 <= 1 && is_peak; ++d1)
                        for (int d2 = -1; d2 <= 1 && is_peak; ++d2)
                            for (int d3 = -1; d3 <= 1 && is_peak; ++d3)
                                for (int d4 = -1; d4 <= 1 && is_peak; ++d4) {
                                    if (!d0 && !d1 && !d2 && !d3 && !d4)
                                        continue;
                                    int j0 = i0 + d0;
                                    const int j1 = i1 + d1, j2 = i2 + d2, j3 = i3 + d3,
                                              j4 = i4 + d4;
                                    if (s->periodic & 1)
                                        j0 = (j0 + n0) % n0;
                                    else if (j0 < 0 || j0 >= n0)
                                        continue;
                                    if (j1 < 0 || j1 >= n1 || j2 < 0 || j2 >= n2 || j3 < 0 ||
                                        j3 >= n3 || j4 < 0 || j4 >= n4)
                                        continue;
                                    const int32_t ns = count_slot[j0 * n1 + j1];
                                    if (ns < 0)
                                        return -1;
                                    const uint64_t nr = ((uint64_t)j2 * n3 + (uint64_t)j3) * n4 + (uint64_t)j4;
                                    const int32_t hn = counts[(uint64_t)ns * inner + nr];
                                    const uint64_t nbin = ((uint64_t)j0 * n1 + (uint64_t)j1) * inner + nr;
                                    if (hn > h || (hn == h && nbin < bin))
                                        is_peak = 0;
                                }
                if (is_peak) {
                    if (nc >= cap)
                        return -2;
                    out_bin[nc] = bin;
                    out_votes[nc] = h;
                    ++nc;
                }
            }
        }
    return nc;
}

int32_t orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------------------
 * Candidate fit (Sec. 8: the candidates found in the parameter space are then fitted to
 * their hits; Fig. 6 times such a fit on CPU cores).  The paper defines no fit; the stated
 * reading, computed here in double precision from the float32 hits, one candidate at a
 * time, hits in the order given (the candidate's sorted hit ids):
 *   1. circle: (a, b, c) minimise sum_k (w_k + a u_k + b v_k + c)^2 over the hits, with
 *      (u, v) = (x, y) - centroid and w = u^2 + v^2 (the algebraic, Kasa, circle fit; the
 *      centroid shift changes the minimiser only by the translation), solved through its
 *      3 x 3 normal equations by Cramer's rule.  Centre = centroid - (a, b)/2,
 *      R = sqrt(a^2/4 + b^2/4 - c).
 *   2. hit selection: with the circle of all hits, each layer keeps only its hit with the
 *      smallest | |p - centre| - R | (ties: the earlier hit); the circle is fitted again
 *      on the kept hits.
 *   3. sense: sgn = sign of twice the signed area of the polygon of the kept hits taken in
 *      layer order, sum_k p_k x p_k+1 closing back to the first (+ when 0); for three hits
 *      it is D of the triplet.  q/pT = -sgn / (K B R); perigee, phi0 and d0 as for a
 *      triplet, with |c|^2 - R^2 evaluated directly.
 *   4. s_k as for a triplet; (cot, z0) = least-squares line z = z0 + s cot over the kept
 *      hits.
 *   chi2_rphi = sum (|p - centre| - R)^2 and chi2_rz = sum (z - z0 - s cot)^2 over the kept
 *   hits.  status: 0 ok, 1 fewer than 3 layers, 2 degenerate (singular normal equations,
 *   centre on the origin, or all s equal).  amb: bit 0 a layer's two smallest residuals
 *   lie within eps_rel * R of each other (the selection is ambiguous), bit 2 a hit lies
 *   within eps_rel * pi of the point opposite the perigee.
 * --------------------------------------------------------------------------------------- */

static int circle_fit(const double *xyz, const uint8_t *use, int n, double *cx, double *cy,
                      double *R)
{
    double mx = 0.0, my = 0.0;
    int m = 0;
    for (int k = 0; k < n; ++k)
        if (use[k]) {
            mx += xyz[3 * k];
            my += xyz[3 * k + 1];
            ++m;
        }
    if (m < 3)
        return 1;
    mx /= m;
    my /= m;
    double suu = 0, suv = 0, svv = 0, su = 0, sv = 0, sw = 0, suw = 0, svw = 0;
    for (int k = 0; k < n; ++k) {
        if (!use[k])
            continue;
        const double u = xyz[3 * k] - mx, v = xyz[3 * k + 1] - my, w = u * u + v * v;
        suu += u * u;
        suv += u * v;
        svv += v * v;
        su += u;
        sv += v;
        sw += w;
        suw += u * w;
        svw += v * w;
    }
    /* normal equations M (a, b, c) = r */
    const double M[3][3] = {{suu, suv, su}, {suv, svv, sv}, {su, sv, (double)m}};
    const double r[3] = {-suw, -svw, -sw};
    const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                       M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                       M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    if (det == 0.0)
        return 2;
    double sol[3];
    for (int col = 0; col < 3; ++col) {
        double A[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                A[i][j] = (j == col) ? r[i] : M[i][j];
        sol[col] = (A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                    A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                    A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0])) / det;
    }
    const double r2 = sol[0] * sol[0] / 4.0 + sol[1] * sol[1] / 4.0 - sol[2];
    if (!(r2 > 0.0))
        return 2;
    *cx = mx - sol[0] / 2.0;
    *cy = my - sol[1] / 2.0;
    *R = sqrt(r2);
    return 0;
}

int orc_fit_track(const double *xyz, const int32_t *layer, int n, double b_tesla,
                  double eps_rel, uint8_t *use, double *par, double *chi2, int32_t *amb)
{
    *amb = 0;
    for (int k = 0; k < n; ++k)
        use[k] = 1;
    double cx, cy, R;
    int st = circle_fit(xyz, use, n, &cx, &cy, &R);
    if (st) {
        for (int k = 0; k < n; ++k)
            use[k] = 0;      /* no circle: nothing is kept */
        return st;
    }
    /* per layer, keep the hit closest to the circle */
    for (int k = 0; k < n; ++k)
        use[k] = 0;
    int n_layers_used = 0;
    for (int k = 0; k < n; ++k) {
        int seen = 0;
        for (int j = 0; j < k; ++j)
            if (layer[j] == layer[k])
                seen = 1;
        if (seen)
            continue;
        int best = -1;
        double rb = 0.0, second = INFINITY;
        for (int j = k; j < n; ++j) {
            if (layer[j] != layer[k])
                continue;
            const double dx = xyz[3 * j] - cx, dy = xyz[3 * j + 1] - cy;
            const double res = fabs(sqrt(dx * dx + dy * dy) - R);
            if (best < 0 || res < rb) {
                if (best >= 0)
                    second = rb;
                best = j;
                rb = res;
            } else if (res < second) {
                second = res;
            }
        }
        if (second - rb <= eps_rel * R)
            *amb |= 1;
        use[best] = 1;
        ++n_layers_used;
    }
    if (n_layers_used < 3)
        return 1;
    st = circle_fit(xyz, use, n, &cx, &cy, &R);
    if (st)
        return st;
    /* sense of rotation: twice the signed area of the polygon of the kept hits taken in
     * layer order (for three hits this is D of the triplet) */
    double area2 = 0.0;
    int first = -1, prev = -1;
    for (int L = 0; L < 64; ++L)
        for (int k = 0; k < n; ++k) {
            if (!use[k] || layer[k] != L)
                continue;
            if (first < 0)
                first = k;
            else
                area2 += xyz[3 * prev] * xyz[3 * k + 1] - xyz[3 * prev + 1] * xyz[3 * k];
            prev = k;
        }
    area2 += xyz[3 * prev] * xyz[3 * first + 1] - xyz[3 * prev + 1] * xyz[3 * first];
    const double sgn = area2 >= 0.0 ? 1.0 : -1.0;
    const double cn = sqrt(cx * cx + cy * cy);
    if (cn == 0.0)
        return 2;
    const double power = cx * cx + cy * cy - R * R;
    const double cn_minus_r = power / (cn + R);
    const double px = cx * (cn_minus_r / cn), py = cy * (cn_minus_r / cn);
    const double phi0 = atan2(-sgn * cx, sgn * cy);
    const double d0 = -px * sin(phi0) + py * cos(phi0);
    const double qopt = -sgn / (ORC_K * b_tesla * R);
    /* signed arcs from the perigee and the least-squares line */
    const double tx = cos(phi0), ty = sin(phi0);
    double sbar = 0.0, zbar = 0.0;
    int m = 0;
    double *s = (double *)malloc(sizeof(double) * (size_t)n);
    for (int k = 0; k < n; ++k) {
        if (!use[k])
            continue;
        const double dx = xyz[3 * k] - px, dy = xyz[3 * k + 1] - py;
        double a = sqrt(dx * dx + dy * dy) / (2.0 * R);
        if (a > 1.0)
            a = 1.0;
        const double half = asin(a);
        if (2.0 * half >= ORC_PI * (1.0 - eps_rel))
            *amb |= 4;
        s[k] = ((dx * tx + dy * ty) >= 0.0 ? 1.0 : -1.0) * 2.0 * R * half;
        sbar += s[k];
        zbar += xyz[3 * k + 2];
        ++m;
    }
    sbar /= m;
    zbar /= m;
    double sss = 0.0, ssz = 0.0;
    for (int k = 0; k < n; ++k)
        if (use[k]) {
            sss += (s[k] - sbar) * (s[k] - sbar);
            ssz += (s[k] - sbar) * (xyz[3 * k + 2] - zbar);
        }
    if (sss == 0.0) {
        free(s);
        return 2;
    }
    const double cot = ssz / sss, z0 = zbar - cot * sbar;
    double c2r = 0.0, c2z = 0.0;
    for (int k = 0; k < n; ++k)
        if (use[k]) {
            const double dx = xyz[3 * k] - cx, dy = xyz[3 * k + 1] - cy;
            const double rr = sqrt(dx * dx + dy * dy) - R;
            const double rz = xyz[3 * k + 2] - z0 - cot * s[k];
            c2r += rr * rr;
            c2z += rz * rz;
        }
    free(s);
    par[0] = phi0;
    par[1] = qopt;
    par[2] = d0;
    par[3] = cot;
    par[4] = z0;
    chi2[0] = c2r;
    chi2[1] = c2z;
    return 0;
}

/* Fit many candidates: hit lists concatenated in ids (indices into hits), candidate t
 * owns ids[off[t] .. off[t+1]).  use is parallel to ids. */
void orc_fit_tracks(const orc_hit *hits, const int64_t *ids, const int64_t *off, int64_t n_cand,
                    double b_tesla, double eps_rel, int32_t n_threads, uint8_t *use,
                    double *par, double *chi2, int32_t *status, int32_t *amb)
{
#ifdef _OPENMP
    if (n_threads > 0)
        omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t t = 0; t < n_cand; ++t) {
        const int n = (int)(off[t + 1] - off[t]);
        double *xyz = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
        int32_t *lay = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        for (int k = 0; k < n; ++k) {
            const orc_hit *h = hits + ids[off[t] + k];
            xyz[3 * k] = h->x;
            xyz[3 * k + 1] = h->y;
            xyz[3 * k + 2] = h->z;
            lay[k] = h->layer;
        }
        status[t] = orc_fit_track(xyz, lay, n, b_tesla, eps_rel, use + off[t], par + 5 * t,
                                  chi2 + 2 * t, amb + t);
        free(xyz);
        free(lay);
    }
}
