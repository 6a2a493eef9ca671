/*
 * Binary32 replica of the visibility-bitmask gather.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.
 *
 * Algorithm 1 of the paper (Section 3.1) with the ambient cones of Section 3.2,
 * in the binary32 operation sequence that decides the bitmasks: round to
 * nearest even, explicit fused multiply-adds where written (fmaf), no other
 * contraction (build with -ffp-contract=off), no flush to zero.  The sector
 * masks are built in O(1) as one run of ones (Section 3.1, "all occluded
 * sectors are set at once").  The GPU must reproduce these masks bit for bit;
 * its continuous outputs are compared against the FP64 oracle.
 *
 * Every reading of the paper is the same as in oracle_fp64.c.  The choices
 * specific to binary32 are:
 *   - the arccosine is Abramowitz and Stegun 4.4.46, sqrt(1-x) times a degree-7
 *     polynomial (|error| <= 2e-8 in exact arithmetic), with acos(-x) = pi - acos(x);
 *   - normalisation uses an own reciprocal square root: the integer seed
 *     0x5f3759df - (bits >> 1) (Lomont, "Fast inverse square root", 2003)
 *     refined by three Newton steps y <- y (1.5 - 0.5 x y^2);
 *   - the back endpoint uses l_b.v = l.v - t and |l_b|^2 = |l|^2 - 2t (l.v) + t^2,
 *     which follow from l_b = l - t v (v = -p/|p|);
 *   - the ambient cones weigh the SH environment written once per call as a quadratic form
 *     of the view-space direction, b.a + a^T Q a (coefficients in FP64, rounded once), so a
 *     slice's cones reduce to five weighted sums of their direction cosines and sines.
 * Op counts (the algorithmic work used by the roofline) are accumulated per
 * block, one per IEEE add/sub/mul/fma/div/sqrt, compare, select, min/max,
 * conversion, shift, logic op and popcount.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* Algorithmic op counts per block: one per IEEE add/sub/mul/fma/div/sqrt, compare, select,
 * min/max, conversion, shift, logic op and popcount the code below performs (memory loads and
 * stores are not ops).  W = 64-bit words of the mask (2 for 128 sectors, else 1). */
/* pi/2 rounded to binary32 */
static const float kHalfPi32 = 1.57079637050628662109375f;

#define RSQRT_OPS 13          /* max, shift, subtract, half, 3 x (square, fma, multiply) */
#define ACOS_OPS 13           /* 1 - a, max, sqrt, 7 fma, multiply, compare, select */
#define OPS_STEP_HEAD 12      /* loop compare + increment, j+1 and its conversion, offset fma,
                                 two roundings (fma, subtract), centre test (2 compares, and) */
#define OPS_STEP_QUAD 2       /* quadratic steps: square and scale */
#define OPS_STEP_PIXEL 11     /* two conversions, two adds, bounds test (4 compares, 3 ors) */
#define OPS_STEP_DEPTH 5      /* index multiply-add, geometry test (2 compares, and) */
#define OPS_FRONT_COS 14      /* sample ray 2, l 3, l.v 3, |l|^2 3, edge-band test 3 */
#define OPS_FRONT_ANGLE (RSQRT_OPS + 1 + ACOS_OPS + 3 + 1) /* rsqrt, cosine, acos, map + clamp, band test */
#define OPS_BACK (3 + RSQRT_OPS + 1 + ACOS_OPS + 3)        /* l_b.v, |l_b|^2, rsqrt, cosine, acos, map */
#define OPS_RUN(W) (2 + 17 + 4 * ((W) - 1) + ((W) == 1 ? 3 : 7) + (W) + 2)
                              /* endpoint selects 2; run: width test 2, ceil/floor path 6,
                                 empty test 1, two low-bit masks 6, and-not 2 (per extra word +4);
                                 newly: not, and, popcount (two words: 7); or; GI test 2 */
#define OPS_GI 17             /* two clamped cosines 10, weight 4, three fma */
#define OPS_CONE(W) (11 + 4 * ((W) - 1) + 4 + 2 + 2 + 5 + 2)
                              /* group mask and count 11, direction 4, weight 2, weighted
                                 cosine and sine 2, five sums 5, loop 2 */
#define OPS_AMB_SLICE 80      /* doubled sum 1, u 6, b.u 9, doublings 4, monomials 21,
                                 t_m 18, q_m t_m 18, accumulate 3 */

/* Abramowitz and Stegun 4.4.46 coefficients a0..a7. */
static const float AS0 = 1.5707963050f, AS1 = -0.2145988016f, AS2 = 0.0889789874f, AS3 = -0.0501743046f;
static const float AS4 = 0.0308918810f, AS5 = -0.0170881256f, AS6 = 0.0066700901f, AS7 = -0.0012624911f;

static float f_from_u(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t u_from_f(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

float orc32_rsqrt(float x) {
    x = fmaxf(x, 1.17549435e-38f); /* smallest normal: keeps 0 finite */
    float y = f_from_u(0x5f3759dfu - (u_from_f(x) >> 1));
    const float hx = 0.5f * x;
    for (int k = 0; k < 3; ++k) {
        const float t = y * y;
        const float u = fmaf(-hx, t, 1.5f);
        y = y * u;
    }
    return y;
}

float orc32_acos(float c) {
    const float a = fabsf(c);
    const float s = sqrtf(fmaxf(1.0f - a, 0.0f)); /* |c| > 1 (rounding) gives acos(+-1) */
    float P = fmaf(AS7, a, AS6);
    P = fmaf(P, a, AS5);
    P = fmaf(P, a, AS4);
    P = fmaf(P, a, AS3);
    P = fmaf(P, a, AS2);
    P = fmaf(P, a, AS1);
    P = fmaf(P, a, AS0);
    const float r = s * P;
    return c < 0.0f ? 3.14159265358979323846f - r : r;
}

/* Sector masks of up to 128 bits. */
typedef unsigned __int128 mask_t;

static mask_t low_bits(int k) { return k >= 128 ? ~(mask_t)0 : (((mask_t)1 << k) - 1); }

static int popc128(mask_t v) {
    return __builtin_popcountll((uint64_t)v) + __builtin_popcountll((uint64_t)(v >> 64));
}

/* The run [lo, hi) of one sample (lo >= hi: no sector), and its mask. */
static mask_t sector_run(float A, float B, int nb, int hit_rule, int *lo_out, int *hi_out) {
    int lo, hi;
    *lo_out = *hi_out = 0;
    if (hit_rule == 0) {
        /* sectors whose centre k + 1/2 lies in [A, B], provided B - A >= 1/2:
         * exactly the sectors covered at least half (Section 3.1 round criterion) */
        if (!(B - A >= 0.5f)) return 0;
        lo = (int)ceilf(A - 0.5f);
        hi = (int)floorf(B + 0.5f);
    } else {
        lo = (int)floorf(A);
        hi = lo + (int)ceilf(B - A);
        if (hi > nb) hi = nb;
    }
    if (hi <= lo) return 0;
    *lo_out = lo;
    *hi_out = hi;
    return low_bits(hi) & ~low_bits(lo);
}

uint64_t orc32_sector_mask(float A, float B, int nb, int hit_rule) {
    int lo, hi;
    return (uint64_t)sector_run(A, B, nb, hit_rule, &lo, &hi);
}

void orc32_sector_mask_words(float A, float B, int nb, int hit_rule, uint64_t *out2) {
    int lo, hi;
    const mask_t m = sector_run(A, B, nb, hit_rule, &lo, &hi);
    out2[0] = (uint64_t)m;
    out2[1] = (uint64_t)(m >> 64);
}

static int is_geometry(float z) { return z > 0.0f && z < INFINITY; }

static int validate(const orc_problem *pb) {
    if (!pb || pb->width <= 0 || pb->height <= 0 || !pb->depth || !pb->normal || !pb->radiance) return 1;
    if (pb->num_slices < 1 || pb->num_slices > 16) return 2;
    if (pb->steps_per_side < 1 || pb->steps_per_side > 64) return 3;
    if (pb->sector_count != 32 && pb->sector_count != 64 && pb->sector_count != 128) return 4;
    if (pb->hit_rule != 0 && pb->hit_rule != 1) return 5;
    if (!(pb->radius > 0.0f) || !(pb->radius < INFINITY)) return 6;
    if (!(pb->thickness > 0.0f) || !(pb->thickness_slope >= 0.0f) || !(pb->thickness_slope < INFINITY)) return 7;
    if (pb->ambient_cones < 0 || pb->ambient_cones > 8) return 8;
    if (pb->ambient_cones > 0 && (pb->sector_count % pb->ambient_cones != 0 || !pb->sh)) return 8;
    if (pb->step_mode != 0 && pb->step_mode != 1) return 9;
    return 0;
}

/* Per-call constants of the replica (binary32 unless noted), shared read-only by every pixel. */
typedef struct {
    int W, H, nd, ns, nb, na, words, inf_t, ops_run, ops_cone;
    float inv_fx, inv_fy, kx0, ninv_fy, ky0, Rfx, dn, K, half_nb, f_nb, inv_nb, inv_nd, t0, kt;
    float edge_hi, edge_lo, sdel, cdel;
    float dcos[16][16], dsin[16][16];
    float ccos[8], csin[8];
    float amb_b[3][3], amb_q[3][6]; /* the SH environment as L(a) = b.a + a^T Q a, view space */
} ctx32;

/* The 3-band SH environment (sh[3 m + channel], m the real SH basis y00, y1-1, y10, y11, y2-2,
 * y2-1, y20, y21, y22) as a quadratic form of the view-space direction a.  For a unit world direction
 * w = R a the sum of sh_m Y_m(w) is c + b_w.w + w^T M w, with c = Y00 sh0 - (Y20's constant term)
 * sh6, b_w = Y1 (sh3, sh1, sh2) and M the band-2 terms; c goes on the diagonal (c |a|^2 = c), so
 * b = R^T b_w and Q = R^T M R + c I.  FP64, each coefficient rounded once to binary32; Q is kept as
 * (xx, yy, zz, xy, xz, yz). */
static void ambient_form32(const float *R, const float *sh, float b_out[3][3], float q_out[3][6]) {
    const double y0 = 0.5 * sqrt(1.0 / M_PI), y1 = sqrt(3.0 / (4.0 * M_PI));
    const double y2 = 0.5 * sqrt(15.0 / M_PI), y3 = 0.25 * sqrt(5.0 / M_PI);
    const double y4 = 0.25 * sqrt(15.0 / M_PI);
    double Rd[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Rd[i][j] = (double)R[3 * i + j];
    for (int ch = 0; ch < 3; ++ch) {
        double h[9];
        for (int m = 0; m < 9; ++m) h[m] = (double)sh[3 * m + ch];
        const double cc = y0 * h[0] - y3 * h[6];
        const double bw[3] = {y1 * h[3], y1 * h[1], y1 * h[2]};
        const double Mw[3][3] = {{y4 * h[8], 0.5 * y2 * h[4], 0.5 * y2 * h[7]},
                                 {0.5 * y2 * h[4], -(y4 * h[8]), 0.5 * y2 * h[5]},
                                 {0.5 * y2 * h[7], 0.5 * y2 * h[5], 3.0 * y3 * h[6]}};
        double T[3][3], Q[3][3];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) T[i][k] = (Mw[i][0] * Rd[0][k] + Mw[i][1] * Rd[1][k]) + Mw[i][2] * Rd[2][k];
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) Q[j][k] = (Rd[0][j] * T[0][k] + Rd[1][j] * T[1][k]) + Rd[2][j] * T[2][k];
        for (int j = 0; j < 3; ++j) {
            b_out[ch][j] = (float)((Rd[0][j] * bw[0] + Rd[1][j] * bw[1]) + Rd[2][j] * bw[2]);
            Q[j][j] = Q[j][j] + cc;
        }
        q_out[ch][0] = (float)Q[0][0];
        q_out[ch][1] = (float)Q[1][1];
        q_out[ch][2] = (float)Q[2][2];
        q_out[ch][3] = (float)Q[0][1];
        q_out[ch][4] = (float)Q[0][2];
        q_out[ch][5] = (float)Q[1][2];
    }
}

static void setup32(const orc_problem *pb, ctx32 *c) {
    c->W = pb->width;
    c->H = pb->height;
    c->nd = pb->num_slices;
    c->ns = pb->steps_per_side;
    c->nb = pb->sector_count;
    c->na = pb->ambient_cones;
    c->words = c->nb == 128 ? 2 : 1;
    c->inf_t = isinf(pb->thickness);
    c->ops_run = OPS_RUN(c->words);
    c->ops_cone = OPS_CONE(c->words);
    c->inv_fx = 1.0f / pb->fx;
    c->inv_fy = 1.0f / pb->fy;
    c->kx0 = -(pb->cx * c->inv_fx);
    c->ninv_fy = -c->inv_fy;
    c->ky0 = pb->cy * c->inv_fy;
    c->Rfx = pb->radius * pb->fx;
    c->dn = 1.0f / (float)(c->ns + 1);
    c->K = (float)((double)c->nb / M_PI); /* sectors per radian, FP64 rounded once */
    c->half_nb = 0.5f * (float)c->nb;
    c->f_nb = (float)c->nb;
    c->inv_nb = 1.0f / (float)c->nb;
    c->inv_nd = 1.0f / (float)c->nd;
    c->t0 = pb->thickness;
    c->kt = pb->thickness_slope;
    c->edge_hi = pb->hit_rule == 0 ? c->f_nb - 0.5f : nextafterf(c->f_nb, 0.0f);
    c->edge_lo = pb->hit_rule == 0 ? 0.5f : nextafterf(0.0f, 1.0f);
    /* half a sector in radians (0 for the floor/ceil rule), its sine and cosine, FP64 rounded once */
    const double del = pb->hit_rule == 0 ? M_PI / (2.0 * c->nb) : 0.0;
    c->sdel = (float)sin(del);
    c->cdel = (float)cos(del);
    /* Direction table: cos, sin of (i + xi_phi) pi / N_d per noise class, FP64 rounded once. */
    for (int k = 0; k < 16; ++k) {
        const float xi = pb->noise ? pb->noise[2 * k] : 0.0f;
        for (int i = 0; i < c->nd; ++i) {
            const double phi = ((double)i + (double)xi) * M_PI / (double)c->nd;
            c->dcos[k][i] = (float)cos(phi);
            c->dsin[k][i] = (float)sin(phi);
        }
    }
    /* Cone table: group-centre angles -pi/2 + (k + 1/2) pi / N_a relative to the normal. */
    for (int k = 0; k < c->na; ++k) {
        const double th = -0.5 * M_PI + (k + 0.5) * M_PI / c->na;
        c->ccos[k] = (float)cos(th);
        c->csin[k] = (float)sin(th);
    }
    if (c->na > 0) ambient_form32(pb->view_to_world, pb->sh, c->amb_b, c->amb_q);
}

/* The per-launch ambient coefficients above, for a pin test: b_out[3 channel + j] = b_j,
 * q_out[6 channel + m] = Q's entry m (xx, yy, zz, xy, xz, yz). */
void orc32_ambient_form(const float *R, const float *sh, float *b_out, float *q_out) {
    float b[3][3], q[3][6];
    ambient_form32(R, sh, b, q);
    for (int ch = 0; ch < 3; ++ch) {
        for (int j = 0; j < 3; ++j) b_out[3 * ch + j] = b[ch][j];
        for (int m = 0; m < 6; ++m) q_out[6 * ch + m] = q[ch][m];
    }
}

/* One pixel of the replica.  cnt[7] accumulates the counters of orc32_pixels.  runs (may be NULL):
 * this pixel's [N_d][2][N_s] block of (lo, hi) sector runs, written for every step (0, 0 where the
 * step sets no sector).  ep (may be NULL): this pixel's [N_d][2][N_s] block of (X_f, X_b) pairs,
 * written only for the samples that reach the front angle (and the back one). */
static void pixel32(const orc_problem *pb, const ctx32 *c, int x, int y, float *o0, float *o1, uint64_t *mk,
                    int64_t *cnt, int16_t *runs, float *ep) {
    const int W = c->W, H = c->H, nd = c->nd, ns = c->ns, nb = c->nb, na = c->na, words = c->words;
    const size_t pix = (size_t)y * W + x;
    const float z = pb->depth[pix];
    int64_t ops = 3;
    ++cnt[0];
    if (runs) memset(runs, 0, sizeof(int16_t) * 2 * 2 * (size_t)nd * ns);
    if (!is_geometry(z)) {
        ++cnt[1];
        cnt[6] += ops + 8;
        if (o0) { o0[0] = o0[1] = o0[2] = 0.0f; o0[3] = 1.0f; }
        if (o1) { o1[0] = o1[1] = o1[2] = o1[3] = 0.0f; }
        if (mk)
            for (int i = 0; i < nd * words; ++i) mk[i] = 0;
        return;
    }

    /* Pixel setup: p, v, n_p, projected radius, step unit, thickness. */
    const float u = (float)x + 0.5f, v = (float)y + 0.5f;
    const float ax = fmaf(u, c->inv_fx, c->kx0), by = fmaf(v, c->ninv_fy, c->ky0);
    const float px = ax * z, py = by * z;
    const float rd = orc32_rsqrt(fmaf(ax, ax, fmaf(by, by, 1.0f)));
    const float vx = -(ax * rd), vy = -(by * rd), vz = rd;
    const float *nrm = pb->normal + 4 * pix;
    const float nx = nrm[0], ny = nrm[1], nz = nrm[2];
    const float rpx = fminf(c->Rfx / z, 1048576.0f);
    const int cls = (y & 3) * 4 + (x & 3);
    const float xi_s = pb->noise ? pb->noise[2 * cls + 1] : 0.0f;
    const float xidn = xi_s * c->dn;
    const float del = rpx * c->dn, xdel = xidn * rpx; /* step unit r/(N_s+1) and its jitter */
    float tp = 0.0f, t2 = 0.0f, m2t = 0.0f;
    if (!c->inf_t) {
        tp = fmaf(c->kt, z, c->t0);
        t2 = tp * tp;
        m2t = -2.0f * tp;
    }
    ops += 4 + 2 + 2 + RSQRT_OPS + 2 + 2 + 1 + 3 + 4;

    float AO = 0.0f, GIr = 0.0f, GIg = 0.0f, GIb = 0.0f, AMr = 0.0f, AMg = 0.0f, AMb = 0.0f;
    for (int i = 0; i < nd; ++i) {
        ++cnt[2];
        const float cphi = c->dcos[cls][i], sphi = c->dsin[cls][i];
        /* Slice plane: s = normalize(w3 - (w3.v) v), w3 = view-space image of omega. */
        const float w3x = cphi * c->inv_fx, w3y = -(sphi * c->inv_fy);
        const float wv = fmaf(w3x, vx, w3y * vy);
        const float sx0 = fmaf(-wv, vx, w3x), sy0 = fmaf(-wv, vy, w3y), sz0 = -(wv * vz);
        const float rs = orc32_rsqrt(fmaf(sx0, sx0, fmaf(sy0, sy0, sz0 * sz0)));
        const float sx = sx0 * rs, sy = sy0 * rs, sz = sz0 * rs;
        /* Projected normal: gamma, the signed angle from v to n projected into the slice plane. */
        const float nv = fmaf(nx, vx, fmaf(ny, vy, nz * vz));
        const float nsd = fmaf(nx, sx, fmaf(ny, sy, nz * sz));
        const float pn2 = fmaf(nv, nv, nsd * nsd);
        float cg = 1.0f, sg = 0.0f, gam = 0.0f;
        if (pn2 > 0.0f) {
            const float rpn = orc32_rsqrt(pn2);
            cg = nv * rpn;
            sg = nsd * rpn;
            /* |gamma| from whichever of its cosine and sine is the smaller in magnitude, where
             * the arccosine is well conditioned: within pi/4 of 0 or pi, |gamma| = asin|sg|
             * = pi/2 - acos|sg| (cg >= 0) or pi/2 + acos|sg| (cg < 0); else acos(cg). */
            if (fabsf(sg) <= fabsf(cg)) {
                const float a = orc32_acos(fabsf(sg));
                gam = cg >= 0.0f ? kHalfPi32 - a : kHalfPi32 + a;
            } else {
                gam = orc32_acos(cg);
            }
            if (nsd < 0.0f) gam = -gam;
            ops += RSQRT_OPS + 2 + ACOS_OPS + 2 + 4;
        }
        const float off = fmaf(-gam, c->K, c->half_nb);
        /* Cosine thresholds of the edge bands: a front direction whose cosine to v is below
         * thr_p (side +omega) or thr_m (side -omega) lies within the band next to that side's
         * hemisphere edge, i.e. at an angle from v above gamma + pi/2 - delta (side +) or
         * pi/2 - gamma - delta (side -), delta = half a sector (0 for the floor/ceil rule).
         * Angles outside [0, pi] give 2 (every direction) or -2 (none). */
        const float cu_p = fmaf(cg, c->cdel, sg * c->sdel), su_p = fmaf(sg, c->cdel, -(cg * c->sdel));
        const float cu_m = fmaf(cg, c->cdel, -(sg * c->sdel)), su_m = fmaf(sg, c->cdel, cg * c->sdel);
        const float thr_p = cu_p >= 0.0f ? -su_p : (su_p < 0.0f ? 2.0f : -2.0f);
        const float thr_m = cu_m >= 0.0f ? su_m : (su_m > 0.0f ? 2.0f : -2.0f);
        /* signed squares: the test "cosine below thr" is dv |dv| < thr |thr| |l|^2 */
        const float thr2_p = thr_p * fabsf(thr_p), thr2_m = thr_m * fabsf(thr_m);
        ops += 2 + 2 + 3 + 3 + RSQRT_OPS + 3 + 6 + 2 + 1 + 1 + 2 + 8 + 8 + 2;

        mask_t b = 0;
        for (int side = 0; side < 2; ++side) {
            const int pos = side == 1; /* side -omega first, then +omega */
            const float wsx = pos ? cphi : -cphi, wsy = pos ? sphi : -sphi;
            const float sK = pos ? c->K : -c->K;
            const float edge = pos ? c->f_nb : 0.0f;
            const float thr2 = pos ? thr2_p : thr2_m;
            for (int j = 0; j < ns; ++j) {
                ++cnt[3];
                const size_t entry = ((size_t)i * 2 + side) * ns + j;
                /* Step offset along the direction and the nearest pixel (ties to even). */
                float o;
                if (pb->step_mode == 0) {
                    o = fmaf((float)(j + 1), del, xdel);
                } else {
                    const float uj = fmaf((float)(j + 1), c->dn, xidn);
                    o = (uj * uj) * rpx;
                }
                /* nearest integer (ties to even) of the exact product, via a fused add of 1.5*2^23 */
                const float dxf = fmaf(o, wsx, 12582912.0f) - 12582912.0f;
                const float dyf = fmaf(o, wsy, 12582912.0f) - 12582912.0f;
                ops += OPS_STEP_HEAD + OPS_STEP_QUAD * (pb->step_mode != 0);
                if (dxf == 0.0f && dyf == 0.0f) { ++cnt[4]; continue; }
                const int qx = x + (int)dxf, qy = y + (int)dyf;
                ops += OPS_STEP_PIXEL;
                if (qx < 0 || qy < 0 || qx >= W || qy >= H) { ++cnt[4]; continue; }
                const size_t q = (size_t)qy * W + qx;
                const float zq = pb->depth[q];
                ops += OPS_STEP_DEPTH;
                if (!is_geometry(zq)) { ++cnt[4]; continue; }

                /* Front sample: l = s_f - p, its cosine to v, its sector coordinate.  The sample's
                 * view ray is the centre pixel's ray plus the pixel offset over the focal length. */
                const float aq = fmaf(dxf, c->inv_fx, ax), bq = fmaf(dyf, c->ninv_fy, by);
                const float lx = fmaf(aq, zq, -px), ly = fmaf(bq, zq, -py), lz = z - zq;
                const float dv = fmaf(lx, vx, fmaf(ly, vy, lz * vz));
                const float ll = fmaf(lx, lx, fmaf(ly, ly, lz * lz));
                ops += OPS_FRONT_COS;
                /* Inside the edge band (cosine dv / sqrt(ll) below thr, compared through the
                 * monotone map x -> x |x| without the square root): by the half-covered rule
                 * (Section 3.1) the sample occludes nothing, because its back endpoint lies
                 * still closer to that edge. */
                if (dv * fabsf(dv) < thr2 * ll) continue;
                float *e = ep ? ep + 2 * entry : NULL;
                const float rl = orc32_rsqrt(ll);
                const float cf = dv * rl;
                const float Xf_raw = fmaf(orc32_acos(cf), sK, off);
                const float Xf = fminf(fmaxf(Xf_raw, 0.0f), c->f_nb);
                if (e) e[0] = Xf_raw;
                ops += OPS_FRONT_ANGLE;
                /* The same band in sector units (exact for the computed endpoint). */
                if (pos ? Xf > c->edge_hi : Xf < c->edge_lo) continue;

                /* Back sample (constant thickness behind the front one). */
                float Xb;
                if (c->inf_t) {
                    Xb = edge;
                } else {
                    const float dvb = dv - tp;
                    const float llb = fmaf(m2t, dv, ll + t2);
                    const float cb = dvb * orc32_rsqrt(llb);
                    const float Xb_raw = fmaf(orc32_acos(cb), sK, off);
                    Xb = fminf(fmaxf(Xb_raw, 0.0f), c->f_nb);
                    if (e) e[1] = Xb_raw;
                    ops += OPS_BACK;
                }
                /* The back endpoint lies toward this side's edge: [A, B] = [X_f, X_b] on side +,
                 * [X_b, X_f] on side - (a rounding-level reversal leaves B < A: no sector). */
                const float A = pos ? Xf : Xb, B = pos ? Xb : Xf;
                int lo, hi;
                const mask_t bj = sector_run(A, B, nb, pb->hit_rule, &lo, &hi);
                if (runs && hi > lo) {
                    runs[2 * entry] = (int16_t)lo;
                    runs[2 * entry + 1] = (int16_t)hi;
                }
                const int newly = popc128(bj & ~b);
                b |= bj;
                ops += c->ops_run;

                /* Indirect light from the newly occluded sectors (Section 3.3). */
                if (newly > 0 && pb->gi) {
                    ++cnt[5];
                    const float *cj = pb->radiance + 4 * q, *nj = pb->normal + 4 * q;
                    const float cp = fmaxf(fmaf(nx, lx, fmaf(ny, ly, nz * lz)) * rl, 0.0f);
                    const float cq = fmaxf(-(fmaf(nj[0], lx, fmaf(nj[1], ly, nj[2] * lz)) * rl), 0.0f);
                    const float wgt = (((float)newly * c->inv_nb) * cp) * cq;
                    GIr = fmaf(wgt, cj[0], GIr);
                    GIg = fmaf(wgt, cj[1], GIg);
                    GIb = fmaf(wgt, cj[2], GIb);
                    ops += OPS_GI;
                }
            }
        }

        /* Slice end: unoccluded fraction, then the ambient cones (Section 3.2). */
        const int occ = popc128(b);
        AO += (float)(nb - occ) * c->inv_nb;
        ops += 5;
        if (na > 0) {
            /* Cone k's direction is a_k = c_k v + s_k s and the environment is L(a) = b.a + a^T Q a,
             * so sum_k w_k L(a_k) = b.u + sum_m q_m t_m: u = v sum w c + s sum w s, and t_m = (v's
             * monomial m) sum w c^2 + (s's) sum w s^2 + (the symmetric product's) 2 sum w c s. */
            const int g = nb / na;
            float Wc = 0.0f, Ws = 0.0f, Wcc = 0.0f, Wss = 0.0f, Wcs = 0.0f;
            for (int k = 0; k < na; ++k) {
                const mask_t Mk = low_bits((k + 1) * g) & ~low_bits(k * g);
                const int freek = popc128(~b & Mk);
                const float ck = fmaf(cg, c->ccos[k], -(sg * c->csin[k]));
                const float sk = fmaf(sg, c->ccos[k], cg * c->csin[k]);
                const float wt = (float)freek * c->inv_nb;
                const float tc = wt * ck, ts = wt * sk;
                Wc = Wc + tc;
                Ws = Ws + ts;
                Wcc = fmaf(tc, ck, Wcc);
                Wss = fmaf(ts, sk, Wss);
                Wcs = fmaf(tc, sk, Wcs);
                ops += c->ops_cone;
            }
            const float W2cs = Wcs + Wcs;
            const float ux = fmaf(vx, Wc, sx * Ws), uy = fmaf(vy, Wc, sy * Ws), uz = fmaf(vz, Wc, sz * Ws);
            float acc[3];
            for (int ch = 0; ch < 3; ++ch)
                acc[ch] = fmaf(c->amb_b[ch][2], uz, fmaf(c->amb_b[ch][1], uy, c->amb_b[ch][0] * ux));
            const float vx2 = vx + vx, vy2 = vy + vy, sx2 = sx + sx, sy2 = sy + sy;
            /* monomials of Q's entries xx, yy, zz, xy, xz, yz: of v, of s, and of the pair (v, s) */
            const float pv[6] = {vx * vx, vy * vy, vz * vz, vx2 * vy, vx2 * vz, vy2 * vz};
            const float ps[6] = {sx * sx, sy * sy, sz * sz, sx2 * sy, sx2 * sz, sy2 * sz};
            const float pc[6] = {vx * sx, vy * sy, vz * sz, fmaf(vx, sy, vy * sx), fmaf(vx, sz, vz * sx),
                                 fmaf(vy, sz, vz * sy)};
            for (int m = 0; m < 6; ++m) {
                const float t = fmaf(pv[m], Wcc, fmaf(ps[m], Wss, pc[m] * W2cs));
                for (int ch = 0; ch < 3; ++ch) acc[ch] = fmaf(c->amb_q[ch][m], t, acc[ch]);
            }
            AMr = AMr + acc[0];
            AMg = AMg + acc[1];
            AMb = AMb + acc[2];
            ops += OPS_AMB_SLICE;
        }
        if (mk) {
            mk[(size_t)i * words] = (uint64_t)b;
            if (words == 2) mk[(size_t)i * words + 1] = (uint64_t)(b >> 64);
        }
    }
    if (o0) { o0[0] = GIr * c->inv_nd; o0[1] = GIg * c->inv_nd; o0[2] = GIb * c->inv_nd; o0[3] = AO * c->inv_nd; }
    if (o1) { o1[0] = AMr * c->inv_nd; o1[1] = AMg * c->inv_nd; o1[2] = AMb * c->inv_nd; o1[3] = 0.0f; }
    cnt[6] += ops + 8;
}

int orc32_pixels_ex(const orc_problem *pb, int n, const int32_t *xy, float *out0, float *out1, uint64_t *masks,
                    int64_t *counts, int16_t *runs, float *endpoints) {
    int bad = validate(pb);
    if (bad) return bad;
    if (n < 0 || (n > 0 && !xy)) return 10;
    for (int pi = 0; pi < n; ++pi)
        if (xy[2 * pi] < 0 || xy[2 * pi + 1] < 0 || xy[2 * pi] >= pb->width || xy[2 * pi + 1] >= pb->height) return 10;
    ctx32 c;
    setup32(pb, &c);
    const size_t per_pixel = (size_t)c.nd * 2 * c.ns; /* entries of the run and endpoint blocks */
    int64_t c0 = 0, c1 = 0, c2 = 0, c3 = 0, c4 = 0, c5 = 0, c6 = 0;
    /* Pixels are independent and each writes only its own outputs, so the result does not depend
     * on how the loop is split over threads; the counters are integer sums. */
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : c0, c1, c2, c3, c4, c5, c6)
    for (int pi = 0; pi < n; ++pi) {
        int64_t cnt[7] = {0, 0, 0, 0, 0, 0, 0};
        pixel32(pb, &c, xy[2 * pi], xy[2 * pi + 1], out0 ? out0 + 4 * (size_t)pi : NULL,
                out1 ? out1 + 4 * (size_t)pi : NULL, masks ? masks + (size_t)pi * c.nd * c.words : NULL, cnt,
                runs ? runs + 2 * per_pixel * pi : NULL, endpoints ? endpoints + 2 * per_pixel * pi : NULL);
        c0 += cnt[0]; c1 += cnt[1]; c2 += cnt[2]; c3 += cnt[3]; c4 += cnt[4]; c5 += cnt[5]; c6 += cnt[6];
    }
    if (counts) {
        counts[0] = c0; counts[1] = c1; counts[2] = c2; counts[3] = c3;
        counts[4] = c4; counts[5] = c5; counts[6] = c6;
    }
    return 0;
}

int orc32_pixels(const orc_problem *pb, int n, const int32_t *xy, float *out0, float *out1, uint64_t *masks,
                 int64_t *counts) {
    return orc32_pixels_ex(pb, n, xy, out0, out1, masks, counts, NULL, NULL);
}

/* Test helper: sweep every binary32 value in [0, 1] (bit patterns 0 .. 0x3f800000).
 * Counts places where orc32_acos increases with its argument and returns the largest
 * absolute error against the C library's double-precision acos on every stride-th value. */
void orc32_acos_sweep(int stride, double *max_err, int64_t *increases) {
    float prev = orc32_acos(0.0f);
    double me = 0.0;
    int64_t inc = 0;
    for (uint32_t u = 1; u <= 0x3f800000u; ++u) {
        const float x = f_from_u(u);
        const float a = orc32_acos(x);
        if (a > prev) ++inc;
        prev = a;
        if (stride > 0 && (u % (uint32_t)stride) == 0) {
            const double e = fabs((double)a - acos((double)x));
            if (e > me) me = e;
        }
    }
    *max_err = me;
    *increases = inc;
}

/* Test helper: largest relative error of orc32_rsqrt over n values spread over [lo, hi]
 * geometrically, against the double-precision 1/sqrt. */
double orc32_rsqrt_sweep(double lo, double hi, int n) {
    double me = 0.0;
    for (int i = 0; i < n; ++i) {
        const double t = (n > 1) ? (double)i / (n - 1) : 0.0;
        const float x = (float)(lo * pow(hi / lo, t));
        const double ref = 1.0 / sqrt((double)x);
        const double e = fabs((double)orc32_rsqrt(x) - ref) / ref;
        if (e > me) me = e;
    }
    return me;
}
