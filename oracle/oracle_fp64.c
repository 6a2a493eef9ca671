/*
 * FP64 oracle of the visibility-bitmask gather.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.
 *
 * It follows Algorithm 1 (Section 3.1) in the paper's order, with the
 * directionally occluded ambient term of Section 3.2 and the sample ordering
 * of Section 3.3.  Geometry and angles are in double precision; the inputs are
 * the binary32 G-buffer values promoted exactly.  The sector hit rule is
 * evaluated per sector by brute force (overlap of [A, B] with [k, k+1]), and
 * indirect light is credited per sector to the first sample that sets it,
 * which equals Algorithm 1's countbits(b_j & ~b_i) form without bit tricks.
 *
 * Readings of the paper where it is silent or garbled (each is listed in the
 * design notes):
 *   - N_d slices i = 0..N_d-1 at azimuth (i + xi_phi) pi / N_d; N_s steps per
 *     side, j = 0..N_s-1, at offset (j + 1 + xi_s) r / (N_s + 1) (Algorithm 1,
 *     "stepsize r/(N_s+1)", "directions with random offset").
 *   - Both sides of the slice, side -omega first, then +omega, near to far
 *     (Section 3.1 "samples are still taken on each side"; Section 3.3 needs
 *     near samples to occlude far ones).
 *   - The back sample lies *behind* the front one, away from the camera along
 *     the centre pixel's view ray: s_b = s_f + t p/|p| (Figure 4 caption and
 *     the word "back"; the printed minus sign would put it in front).
 *   - Elevation h = sigma acos(l.v/|l|) measured from the view vector v in the
 *     slice; the sector frame is centred on the projected normal (Eq. 4),
 *     X = (h - gamma) N_b / pi + N_b / 2, clamped to [0, N_b].
 *   - Hit rule 0: a sector is set iff at least half of it is covered
 *     (Section 3.1 "round criterion", Figure 4 caption).  Hit rule 1: the
 *     floor/ceil form of Algorithm 1 without its stray +pi/2 in the width.
 *   - Indirect light weight: (newly set sectors / N_b) c_j max(0, n_p.l)
 *     max(0, -n_j.l), n_l read as the sample's normal n_j (Section 3.3).
 *   - Sample pixel: nearest pixel (round half to even) of sigma o omega; the
 *     sample is skipped when off-screen, equal to the centre pixel or sky.
 *     Which pixel a step reads is an integer decision taken from floating
 *     point, so it is taken here in binary32 exactly as the GPU takes it.
 *   - Thickness t(z) = t + k_t z (Section 3.1, linear increase with
 *     distance); t = +INF puts the back endpoint at the hemisphere edge of
 *     the sample's side (GTAO without falloff, Section 3.1).
 *   - Ambient (Section 3.2): N_a equal sector groups; the source is sampled in
 *     the direction at the centre of each group and weighted by the group's
 *     unoccluded sector count over N_b.
 *   - AO output is Algorithm 1's sum of (1 - countbits(b_i)/N_b) / N_d, i.e.
 *     the unoccluded fraction (1 = fully visible).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

typedef struct { double x, y, z; } d3;
static d3 mk3(double x, double y, double z) { d3 r = {x, y, z}; return r; }
static d3 sub3(d3 a, d3 b) { return mk3(a.x - b.x, a.y - b.y, a.z - b.z); }
static d3 add3(d3 a, d3 b) { return mk3(a.x + b.x, a.y + b.y, a.z + b.z); }
static d3 mul3(d3 a, double s) { return mk3(a.x * s, a.y * s, a.z * s); }
static double dot3(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static double len3(d3 a) { return sqrt(dot3(a, a)); }
static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

static int is_geometry(float z) { return z > 0.0f && z < INFINITY; }

/* View-space position of the pixel centre (u, v) at linear depth z (camera looks along -z). */
static d3 unproject(const orc_problem *pb, double u, double v, double z) {
    return mk3((u - pb->cx) / pb->fx * z, -(v - pb->cy) / pb->fy * z, -z);
}

/* Per-sector hit rule, brute force over the N_b sectors [k, k+1): set[k] = 1 when covered. */
static void sector_set(double A, double B, int nb, int hit_rule, unsigned char *set) {
    if (hit_rule == 0) {
        for (int k = 0; k < nb; ++k) {
            double lo = A > k ? A : (double)k;
            double hi = B < k + 1 ? B : (double)(k + 1);
            set[k] = hi - lo >= 0.5;
        }
    } else {
        /* Algorithm 1: a = floor(A), width = ceil(B - A), kept inside the N_b sectors */
        double a = floor(A);
        double w = ceil(B - A);
        for (int k = 0; k < nb; ++k) set[k] = k >= a && k < a + w;
    }
}

void orc64_sector_mask_words(double A, double B, int nb, int hit_rule, uint64_t *out2) {
    unsigned char set[128];
    sector_set(A, B, nb, hit_rule, set);
    out2[0] = out2[1] = 0;
    for (int k = 0; k < nb; ++k)
        if (set[k]) out2[k / 64] |= (uint64_t)1 << (k % 64);
}

uint64_t orc64_sector_mask(double A, double B, int nb, int hit_rule) {
    uint64_t w[2];
    orc64_sector_mask_words(A, B, nb, hit_rule, w);
    return w[0];
}

static double frac_dist(double v) { return fabs(v - nearbyint(v)); }

/* Distance of this sample's hit-rule decisions from their rounding boundaries, in sector
 * units.  rawA, rawB: the endpoints before clamping to [0, N_b].  An endpoint pinned by the
 * clamp cannot move until its unclamped value comes back inside, so for it the distance is
 * how far the unclamped value lies beyond the edge, not its distance to an integer. */
static double pinned(double raw, double nb) {
    if (raw > nb) return raw - nb;
    if (raw < 0.0) return -raw;
    return -1.0; /* not pinned */
}

static double decision_margin(double A, double B, double rawA, double rawB, int nb, int hit_rule) {
    if (hit_rule == 0) {
        double m = fabs((B - A) - 0.5);
        double ma = frac_dist(A - 0.5), mb = frac_dist(B + 0.5);
        if (ma < m) m = ma;
        if (mb < m) m = mb;
        return m;
    }
    const double pa = pinned(rawA, nb), pb = pinned(rawB, nb);
    double m = pa >= 0.0 ? pa : frac_dist(A);
    double mw = (pa >= 0.0 && pb >= 0.0 && A == B) ? (pa < pb ? pa : pb) : frac_dist(B - A);
    return mw < m ? mw : m;
}

/* Error bound of the binary32 evaluation, used only to tell rounding-level disagreements from real
 * ones.  eps = 2^-24 is the unit roundoff of binary32.  An angle taken as acos(c) from a cosine c
 * known to within dc has error at most dc / sqrt(1 - c^2), and never more than 2.23 sqrt(dc): acos
 * is Hoelder continuous with exponent 1/2 and constant pi/sqrt(2) (attained at the ends, where
 * acos(1 - d) ~ sqrt(2 d)).  1e-7 rad covers the own arccosine's polynomial error (2e-8) and the
 * rounding of its evaluation. */
static const double kEps32 = 5.9604644775390625e-8;

static double acos_error(double c, double dc) {
    const double s2 = 1.0 - c * c;
    double e = 2.23 * sqrt(dc);
    if (s2 > 0.0 && dc / sqrt(s2) < e) e = dc / sqrt(s2);
    return e + 1e-7;
}

/* Same decisions as decision_margin, each distance divided by the error bound of the endpoints it
 * depends on (eA, eB in sector units). */
static double decision_ratio(double A, double B, double rawA, double rawB, int nb, int hit_rule, double eA,
                             double eB) {
    if (hit_rule == 0) {
        double r = fabs((B - A) - 0.5) / (eA + eB);
        const double ra = frac_dist(A - 0.5) / eA, rb = frac_dist(B + 0.5) / eB;
        if (ra < r) r = ra;
        if (rb < r) r = rb;
        return r;
    }
    const double pa = pinned(rawA, nb), pb = pinned(rawB, nb);
    double r = (pa >= 0.0 ? pa : frac_dist(A)) / eA;
    const double rw = (pa >= 0.0 && pb >= 0.0 && A == B) ? (pa < pb ? pa / eA : pb / eB) : frac_dist(B - A) / (eA + eB);
    return rw < r ? rw : r;
}

/* Real spherical harmonics, 3 bands, in the order
 * Y00, Y1-1 (y), Y10 (z), Y11 (x), Y2-2 (xy), Y2-1 (yz), Y20 (3z^2-1), Y21 (xz), Y22 (x^2-y^2). */
static void sh9(d3 w, double Y[9]) {
    const double c0 = 0.5 * sqrt(1.0 / M_PI);
    const double c1 = sqrt(3.0 / (4.0 * M_PI));
    const double c2 = 0.5 * sqrt(15.0 / M_PI);
    const double c3 = 0.25 * sqrt(5.0 / M_PI);
    const double c4 = 0.25 * sqrt(15.0 / M_PI);
    Y[0] = c0;
    Y[1] = c1 * w.y;
    Y[2] = c1 * w.z;
    Y[3] = c1 * w.x;
    Y[4] = c2 * w.x * w.y;
    Y[5] = c2 * w.y * w.z;
    Y[6] = c3 * (3.0 * w.z * w.z - 1.0);
    Y[7] = c2 * w.x * w.z;
    Y[8] = c4 * (w.x * w.x - w.y * w.y);
}

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

/* One pixel of the FP64 oracle.  o0, o1, mk, mrg, rto: this pixel's outputs (each may be NULL).
 * forced (may be NULL): this pixel's [N_d][2][N_s] block of (lo, hi) sector runs; when given, each
 * sample sets exactly the sectors [lo, hi) instead of those of the FP64 hit rule, and everything
 * else (geometry, cosines, crediting, ambient) stays as below.  ep (may be NULL): this pixel's
 * [N_d][2][N_s] block of (X_f, X_b, e_f, e_b) entries, written for the samples visited.  steps (may be
 * NULL): this pixel's [N_d][2][N_s] block of the (dx, dy) pixel offsets every step reads. */
static void pixel64(const orc_problem *pb, int x, int y, double *o0, double *o1, uint64_t *mk, double *mrg_out,
                    double *rto_out, const int16_t *forced, double *ep, int32_t *steps) {
    const int W = pb->width, H = pb->height, nd = pb->num_slices, ns = pb->steps_per_side;
    const int nb = pb->sector_count, na = pb->ambient_cones;
    const int words = nb == 128 ? 2 : 1;
    const int inf_t = isinf(pb->thickness);
    const int want_ratio = rto_out != NULL || ep != NULL;
    const size_t pix = (size_t)y * W + x;
    const float zf = pb->depth[pix];

    /* Sky: nothing to occlude or bounce; fully visible. */
    if (!is_geometry(zf)) {
        if (o0) { o0[0] = o0[1] = o0[2] = 0.0; o0[3] = 1.0; }
        if (o1) { o1[0] = o1[1] = o1[2] = o1[3] = 0.0; }
        for (int i = 0; i < nd; ++i) {
            if (mk)
                for (int w = 0; w < words; ++w) mk[(size_t)i * words + w] = 0;
            if (mrg_out) mrg_out[i] = INFINITY;
            if (rto_out) rto_out[i] = INFINITY;
        }
        return;
    }

    /* Algorithm 1: t, N_b, p, n_p, r. */
    const double z = zf;
    const d3 p = unproject(pb, x + 0.5, y + 0.5, z);
    const double plen = len3(p);
    const d3 vhat = mul3(p, -1.0 / plen);
    const float *nrm = pb->normal + 4 * pix;
    const d3 np_ = mk3(nrm[0], nrm[1], nrm[2]);
    const double tp = inf_t ? INFINITY : (double)pb->thickness + (double)pb->thickness_slope * z;
    const int cls = (y & 3) * 4 + (x & 3);
    const float xi_phi = pb->noise ? pb->noise[2 * cls] : 0.0f;
    const float xi_s = pb->noise ? pb->noise[2 * cls + 1] : 0.0f;

    /* Step sizes: the sample pixel is an integer decision, taken in binary32 as on the GPU. */
    const float Rfx = pb->radius * pb->fx;
    const float rpx = fminf(Rfx / zf, 1048576.0f);
    const float dn = 1.0f / (float)(ns + 1);
    const float xidn = xi_s * dn;

    double AO = 0.0, GI[3] = {0, 0, 0}, AMB[3] = {0, 0, 0};
    for (int i = 0; i < nd; ++i) {
        /* Slice direction with random offset, rounded to binary32 (the direction table). */
        const double phi = ((double)i + (double)xi_phi) * M_PI / (double)nd;
        const float cphi = (float)cos(phi), sphi = (float)sin(phi);

        /* Slice plane: v and the in-plane direction s toward screen direction +omega. */
        const d3 w3 = mk3((double)cphi / pb->fx, -(double)sphi / pb->fy, 0.0);
        d3 s = sub3(w3, mul3(vhat, dot3(w3, vhat)));
        s = mul3(s, 1.0 / len3(s));

        /* Projected normal angle gamma: the signed angle from v to the normal's projection
         * into the slice plane, atan2(n.s, n.v); 0 if the projection is 0. */
        const double nv = dot3(np_, vhat), nsd = dot3(np_, s);
        const double pn = sqrt(nv * nv + nsd * nsd);
        const double gamma = pn > 0.0 ? atan2(nsd, nv) : 0.0;
        /* Binary32 error of gamma: n.v and n.s carry a few roundings of unit vectors (16 eps,
         * generously), scaled up by 1/|projN| when the projected normal is short.  The
         * binary32 spec takes |gamma| as an arccosine of whichever of cos and sin is below
         * 1/sqrt(2) in magnitude, where acos has slope at most sqrt(2); 3e-7 rad covers the own
         * arccosine, pi/2 in binary32 and the final rounding. */
        const double e_gamma = pn > 0.0 ? 1.5 * 16.0 * kEps32 / pn + 3e-7 : M_PI;

        unsigned char occ[128];
        memset(occ, 0, sizeof(occ));
        double mrg = INFINITY, rto = INFINITY;

        for (int side = 0; side < 2; ++side) {
            const int sigma = side == 0 ? -1 : 1;
            const float wsx = sigma > 0 ? cphi : -cphi;
            const float wsy = sigma > 0 ? sphi : -sphi;
            for (int j = 0; j < ns; ++j) {
                const size_t entry = ((size_t)i * 2 + side) * ns + j;
                /* Which pixel this step reads (binary32, nearest pixel, ties to even). */
                const float jp1 = (float)(j + 1);
                float off;
                if (pb->step_mode == 0) {
                    off = fmaf(jp1, rpx * dn, (xi_s * dn) * rpx);
                } else {
                    const float uj = fmaf(jp1, dn, xidn);
                    off = (uj * uj) * rpx;
                }
                const float dxf = fmaf(off, wsx, 12582912.0f) - 12582912.0f;
                const float dyf = fmaf(off, wsy, 12582912.0f) - 12582912.0f;
                if (steps) {
                    steps[2 * entry] = (int32_t)dxf;
                    steps[2 * entry + 1] = (int32_t)dyf;
                }
                if (dxf == 0.0f && dyf == 0.0f) continue;
                const int qx = x + (int)dxf, qy = y + (int)dyf;
                if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                const size_t q = (size_t)qy * W + qx;
                const float zq = pb->depth[q];
                if (!is_geometry(zq)) continue;

                /* Front sample s_f and its elevation in the slice. */
                const d3 sf = unproject(pb, qx + 0.5, qy + 0.5, (double)zq);
                const d3 l = sub3(sf, p);
                const double llen = len3(l);
                const double hf = sigma * acos(clampd(dot3(l, vhat) / llen, -1.0, 1.0));
                const double K = nb / M_PI;
                const double Xf_raw = (hf - gamma) * K + 0.5 * nb;
                double Xb_raw;
                if (inf_t) {
                    Xb_raw = sigma > 0 ? INFINITY : -INFINITY;
                } else {
                    /* Back sample s_b = s_f + t p/|p| (behind the front one). */
                    const d3 sb = add3(sf, mul3(p, tp / plen));
                    const d3 lb = sub3(sb, p);
                    const double hb = sigma * acos(clampd(dot3(lb, vhat) / len3(lb), -1.0, 1.0));
                    Xb_raw = (hb - gamma) * K + 0.5 * nb;
                }
                const double Xf = clampd(Xf_raw, 0.0, (double)nb), Xb = clampd(Xb_raw, 0.0, (double)nb);
                const double A = Xf < Xb ? Xf : Xb, B = Xf < Xb ? Xb : Xf;
                const double rawA = Xf < Xb ? Xf_raw : Xb_raw, rawB = Xf < Xb ? Xb_raw : Xf_raw;
                unsigned char bj[128];
                if (forced) {
                    /* the sectors of a run decided elsewhere */
                    const int lo = forced[2 * entry], hi = forced[2 * entry + 1];
                    for (int k = 0; k < nb; ++k) bj[k] = k >= lo && k < hi;
                } else {
                    sector_set(A, B, nb, pb->hit_rule, bj);
                }
                const double m = decision_margin(A, B, rawA, rawB, nb, pb->hit_rule);
                if (m < mrg) mrg = m;
                if (want_ratio) {
                    /* Binary32 error bounds of the two endpoints, in sector units.  The
                     * components of l = s_f - p carry a few roundings of values as large as
                     * |p| and |s_f| (8 eps of each, generously), which the cosine l.v/|l| sees
                     * divided by |l|: close samples cancel.  The back cosine adds the
                     * thickness and the cancellation in |l_b|^2 = |l|^2 + t^2 - 2 t l.v. */
                    const double El = 8.0 * kEps32 * (plen + len3(sf));
                    const double cf = clampd(dot3(l, vhat) / llen, -1.0, 1.0);
                    const double ef = acos_error(cf, 3.5 * El / llen + 12.0 * kEps32);
                    double eb = 0.0;
                    if (!inf_t) {
                        const d3 lb = sub3(add3(sf, mul3(p, tp / plen)), p);
                        const double lbl = len3(lb), dv = dot3(l, vhat);
                        const double cb = clampd(dot3(lb, vhat) / lbl, -1.0, 1.0);
                        const double dcb = 3.5 * (El + 8.0 * kEps32 * tp) / lbl + 12.0 * kEps32 +
                                           4.0 * kEps32 * (llen * llen + tp * tp + 2.0 * tp * fabs(dv)) / (lbl * lbl);
                        eb = acos_error(cb, dcb);
                    }
                    const double eround = 8.0 * kEps32 * nb;
                    const double eXf = K * (ef + e_gamma) + eround;
                    const double eXb = inf_t ? eround : K * (eb + e_gamma) + eround;
                    const double eA = Xf < Xb ? eXf : eXb, eB = Xf < Xb ? eXb : eXf;
                    const double r = decision_ratio(A, B, rawA, rawB, nb, pb->hit_rule, eA, eB);
                    if (r < rto) rto = r;
                    if (ep) {
                        double *e = ep + 4 * entry;
                        e[0] = Xf_raw;
                        e[1] = Xb_raw;
                        e[2] = eXf;
                        e[3] = eXb;
                    }
                }

                /* Indirect light: each newly occluded sector carries c_j cos cos / N_b. */
                int newly = 0;
                for (int k = 0; k < nb; ++k)
                    if (bj[k] && !occ[k]) { occ[k] = 1; ++newly; }
                if (newly > 0 && pb->gi) {
                    const float *cj = pb->radiance + 4 * q;
                    const float *nj = pb->normal + 4 * q;
                    const d3 lh = mul3(l, 1.0 / llen);
                    const double cp = fmax(0.0, dot3(np_, lh));
                    const double cq = fmax(0.0, -dot3(mk3(nj[0], nj[1], nj[2]), lh));
                    for (int k = 0; k < newly; ++k)
                        for (int c = 0; c < 3; ++c) GI[c] += (double)cj[c] * cp * cq / nb;
                }
            }
        }

        int set = 0;
        for (int k = 0; k < nb; ++k) set += occ[k];
        AO += 1.0 - (double)set / nb;

        if (na > 0) {
            /* Directionally occluded ambient: sample the source at each group's centre. */
            const int g = nb / na;
            for (int k = 0; k < na; ++k) {
                int unocc = 0;
                for (int s2 = k * g; s2 < (k + 1) * g; ++s2) unocc += !occ[s2];
                const double theta = gamma - 0.5 * M_PI + (k + 0.5) * M_PI / na;
                const d3 a = add3(mul3(vhat, cos(theta)), mul3(s, sin(theta)));
                const float *R = pb->view_to_world;
                const d3 wv = mk3(R[0] * a.x + R[1] * a.y + R[2] * a.z, R[3] * a.x + R[4] * a.y + R[5] * a.z,
                                  R[6] * a.x + R[7] * a.y + R[8] * a.z);
                double Y[9];
                sh9(wv, Y);
                for (int c = 0; c < 3; ++c) {
                    double L = 0.0;
                    for (int mm = 0; mm < 9; ++mm) L += (double)pb->sh[3 * mm + c] * Y[mm];
                    AMB[c] += L * unocc / nb;
                }
            }
        }

        if (mk) {
            uint64_t bm[2] = {0, 0};
            for (int k = 0; k < nb; ++k)
                if (occ[k]) bm[k / 64] |= (uint64_t)1 << (k % 64);
            for (int w = 0; w < words; ++w) mk[(size_t)i * words + w] = bm[w];
        }
        if (mrg_out) mrg_out[i] = mrg;
        if (rto_out) rto_out[i] = rto;
    }
    if (o0) { o0[0] = GI[0] / nd; o0[1] = GI[1] / nd; o0[2] = GI[2] / nd; o0[3] = AO / nd; }
    if (o1) { o1[0] = AMB[0] / nd; o1[1] = AMB[1] / nd; o1[2] = AMB[2] / nd; o1[3] = 0.0; }
}

int orc64_pixels_ex(const orc_problem *pb, int n, const int32_t *xy, double *out0, double *out1, uint64_t *masks,
                    double *margin, double *ratio, const int16_t *forced, double *endpoints, int32_t *steps) {
    int bad = validate(pb);
    if (bad) return bad;
    if (n < 0 || (n > 0 && !xy)) return 10;
    for (int pi = 0; pi < n; ++pi)
        if (xy[2 * pi] < 0 || xy[2 * pi + 1] < 0 || xy[2 * pi] >= pb->width || xy[2 * pi + 1] >= pb->height) return 10;
    if (forced) {
        for (size_t e = 0; e < (size_t)n * pb->num_slices * 2 * pb->steps_per_side; ++e) {
            const int lo = forced[2 * e], hi = forced[2 * e + 1];
            if (lo < 0 || hi > pb->sector_count || (hi > lo && lo >= pb->sector_count)) return 11;
        }
    }
    const int nd = pb->num_slices, words = pb->sector_count == 128 ? 2 : 1;
    const size_t per_pixel = (size_t)nd * 2 * pb->steps_per_side;
    /* Pixels are independent and each writes only its own outputs: the result does not depend on
     * how the loop is split over threads. */
#pragma omp parallel for schedule(dynamic, 16)
    for (int pi = 0; pi < n; ++pi)
        pixel64(pb, xy[2 * pi], xy[2 * pi + 1], out0 ? out0 + 4 * (size_t)pi : NULL,
                out1 ? out1 + 4 * (size_t)pi : NULL, masks ? masks + (size_t)pi * nd * words : NULL,
                margin ? margin + (size_t)pi * nd : NULL, ratio ? ratio + (size_t)pi * nd : NULL,
                forced ? forced + 2 * per_pixel * pi : NULL, endpoints ? endpoints + 4 * per_pixel * pi : NULL,
                steps ? steps + 2 * per_pixel * pi : NULL);
    return 0;
}

int orc64_pixels(const orc_problem *pb, int n, const int32_t *xy, double *out0, double *out1, uint64_t *masks,
                 double *margin, double *ratio) {
    return orc64_pixels_ex(pb, n, xy, out0, out1, masks, margin, ratio, NULL, NULL, NULL);
}

/* Threads the oracle's pixel loops use: n > 0 sets it; returns the current count (1 without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int orc_threads(int n) {
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
}
#else
int orc_threads(int n) {
    (void)n;
    return 1;
}
#endif
