/*
 * Seeded procedural G-buffer generator (input generation only).
 *
 * This module produces the synthetic inputs that both the CUDA gather and the
 * CPU oracle consume: linear view-space depth, view-space normals and direct
 * Lambert radiance of a procedural scene, ray-cast in double precision and
 * rounded to binary32.  It contains none of the screen-space method's
 * arithmetic (no slices, no sectors, no bitmasks).
 *
 * The paper measures on the Lumberyard Bistro scene (Section 4), which is not
 * available; this scene stands in for it: a ground plane, spheres resting on
 * it and 1 cm thin panels that model the thin geometry the paper targets
 * (Section 1, Section 3.1).
 *
 * Scene recipe (all draws from one SplitMix64 stream, Steele et al. 2014):
 *   light: elevation U[25,65] deg, azimuth U[0,360) deg, unit RGB intensity
 *   ground plane y = 0, albedo U[0.2,0.9]^3
 *   spheres: radius U[0.2,1.5] m resting on the ground, centre x U[-6,6],
 *            z U[-14,-3], albedo U[0.2,0.9]^3
 *   panels: boxes 1 cm thick, width U[0.5,2] m, height U[1,2.5] m, yaw U[0,pi),
 *           standing on the ground, x U[-6,6], z U[-14,-3], albedo U[0.2,0.9]^3
 *   camera: at (0,1.6,0), pitch -15 deg, 90 deg horizontal field of view,
 *           square pixels, principal point at the image centre.
 * View space is right-handed, camera at the origin looking along -z, +y up;
 * image y points down; the stored depth is z_lin = -z_view (> 0), +INF = sky.
 * Direct radiance = albedo * max(0, n.L) * shadow, so every channel is <= 1.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC (the result is the same with or
 * without OpenMP: every pixel is an independent pure function of the seed).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SG_FAR 200.0

typedef struct { double x, y, z; } v3;
static v3 v3m(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return v3m(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return v3m(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return v3m(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

/* SplitMix64 (Steele, Lea, Flood 2014). */
static uint64_t sm64_next(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double sm64_unif(uint64_t *s) { return (double)(sm64_next(s) >> 11) * 0x1.0p-53; }
static double unif(uint64_t *s, double a, double b) { return a + (b - a) * sm64_unif(s); }

typedef struct { v3 c; double r; v3 alb; } sphere_t;
typedef struct { double x, z, cy, sy, hw, ht, h; v3 alb; } panel_t; /* cy, sy: cos/sin of yaw */

typedef struct {
    v3 light;          /* unit vector toward the light (world) */
    v3 ground_alb;
    int ns, np;
    sphere_t *sph;
    panel_t *pan;
    double R[9];       /* view -> world rotation, row-major */
    v3 eye;
} scene_t;

void sg_camera(int W, int H, float *cam13) {
    /* fx fy cx cy, then the row-major view->world rotation (pitch -15 deg about x). */
    double fx = 0.5 * (double)W / tan(0.25 * M_PI);
    double th = -15.0 * M_PI / 180.0;
    double R[9] = {1, 0, 0, 0, cos(th), -sin(th), 0, sin(th), cos(th)};
    cam13[0] = (float)fx;
    cam13[1] = (float)fx;
    cam13[2] = (float)(0.5 * W);
    cam13[3] = (float)(0.5 * H);
    for (int i = 0; i < 9; ++i) cam13[4 + i] = (float)R[i];
}

static void build_scene(scene_t *sc, uint64_t seed, int n_spheres, int n_panels) {
    uint64_t s = seed;
    double el = unif(&s, 25.0, 65.0) * M_PI / 180.0;
    double az = unif(&s, 0.0, 360.0) * M_PI / 180.0;
    sc->light = v3m(cos(el) * cos(az), sin(el), cos(el) * sin(az));
    sc->ground_alb.x = unif(&s, 0.2, 0.9);
    sc->ground_alb.y = unif(&s, 0.2, 0.9);
    sc->ground_alb.z = unif(&s, 0.2, 0.9);
    sc->ns = n_spheres;
    sc->np = n_panels;
    sc->sph = (sphere_t *)calloc((size_t)(n_spheres > 0 ? n_spheres : 1), sizeof(sphere_t));
    sc->pan = (panel_t *)calloc((size_t)(n_panels > 0 ? n_panels : 1), sizeof(panel_t));
    for (int i = 0; i < n_spheres; ++i) {
        double r = unif(&s, 0.2, 1.5);
        double x = unif(&s, -6.0, 6.0);
        double z = unif(&s, -14.0, -3.0);
        sc->sph[i].c = v3m(x, r, z);
        sc->sph[i].r = r;
        sc->sph[i].alb.x = unif(&s, 0.2, 0.9);
        sc->sph[i].alb.y = unif(&s, 0.2, 0.9);
        sc->sph[i].alb.z = unif(&s, 0.2, 0.9);
    }
    for (int i = 0; i < n_panels; ++i) {
        double w = unif(&s, 0.5, 2.0);
        double h = unif(&s, 1.0, 2.5);
        double yaw = unif(&s, 0.0, M_PI);
        panel_t *p = &sc->pan[i];
        p->x = unif(&s, -6.0, 6.0);
        p->z = unif(&s, -14.0, -3.0);
        p->cy = cos(yaw);
        p->sy = sin(yaw);
        p->hw = 0.5 * w;
        p->ht = 0.005;
        p->h = h;
        p->alb.x = unif(&s, 0.2, 0.9);
        p->alb.y = unif(&s, 0.2, 0.9);
        p->alb.z = unif(&s, 0.2, 0.9);
    }
    double th = -15.0 * M_PI / 180.0;
    double R[9] = {1, 0, 0, 0, cos(th), -sin(th), 0, sin(th), cos(th)};
    memcpy(sc->R, R, sizeof(R));
    sc->eye = v3m(0.0, 1.6, 0.0);
}

/* Nearest hit along o + t d, t in (tmin, tmax).  Returns the object id
 * (-1 ground, 0..ns-1 spheres, ns.. panels) or -2 for no hit. */
static int trace(const scene_t *sc, v3 o, v3 d, double tmin, double tmax, int with_ground,
                 double *t_out, v3 *n_out) {
    int hit = -2;
    double tb = tmax;
    v3 nb = v3m(0, 0, 0);
    if (with_ground && d.y < 0.0) {
        double t = -o.y / d.y;
        if (t > tmin && t < tb) { tb = t; hit = -1; nb = v3m(0, 1, 0); }
    }
    for (int i = 0; i < sc->ns; ++i) {
        const sphere_t *s = &sc->sph[i];
        v3 oc = sub(o, s->c);
        double a = dot(d, d), b = dot(oc, d), c = dot(oc, oc) - s->r * s->r;
        double disc = b * b - a * c;
        if (disc < 0.0) continue;
        double sq = sqrt(disc);
        double t = (-b - sq) / a;
        if (!(t > tmin)) t = (-b + sq) / a;
        if (t > tmin && t < tb) {
            tb = t;
            hit = i;
            nb = scl(sub(add(o, scl(d, t)), s->c), 1.0 / s->r);
        }
    }
    for (int i = 0; i < sc->np; ++i) {
        const panel_t *p = &sc->pan[i];
        /* local frame: rotate by -yaw about y around (x, 0, z) */
        v3 q = v3m(o.x - p->x, o.y, o.z - p->z);
        v3 ol = v3m(p->cy * q.x - p->sy * q.z, q.y, p->sy * q.x + p->cy * q.z);
        v3 dl = v3m(p->cy * d.x - p->sy * d.z, d.y, p->sy * d.x + p->cy * d.z);
        double lo[3] = {-p->hw, 0.0, -p->ht}, hi[3] = {p->hw, p->h, p->ht};
        double oo[3] = {ol.x, ol.y, ol.z}, dd[3] = {dl.x, dl.y, dl.z};
        double t0 = tmin, t1 = tb;
        int ax = -1, sgn = 0, ok = 1;
        for (int k = 0; k < 3 && ok; ++k) {
            if (dd[k] == 0.0) {
                if (oo[k] < lo[k] || oo[k] > hi[k]) ok = 0;
                continue;
            }
            double ta = (lo[k] - oo[k]) / dd[k], tc = (hi[k] - oo[k]) / dd[k];
            int s_in = -1; /* entering face normal sign along axis k */
            if (ta > tc) { double tt = ta; ta = tc; tc = tt; s_in = 1; }
            if (ta > t0) { t0 = ta; ax = k; sgn = s_in; }
            if (tc < t1) t1 = tc;
            if (t0 > t1) ok = 0;
        }
        if (!ok || ax < 0 || !(t0 > tmin) || !(t0 < tb)) continue;
        double nl[3] = {0, 0, 0};
        nl[ax] = (double)sgn;
        /* back to world: rotate by +yaw */
        v3 nw = v3m(p->cy * nl[0] + p->sy * nl[2], nl[1], -p->sy * nl[0] + p->cy * nl[2]);
        tb = t0;
        hit = sc->ns + i;
        nb = nw;
    }
    *t_out = tb;
    *n_out = nb;
    return hit;
}

static v3 albedo_of(const scene_t *sc, int id) {
    if (id == -1) return sc->ground_alb;
    if (id < sc->ns) return sc->sph[id].alb;
    return sc->pan[id - sc->ns].alb;
}

/* Render a W x H G-buffer.  depth: [H*W]; normal, radiance: [H*W*4] (xyz, w=0).
 * cam13 receives fx fy cx cy and the row-major view->world rotation. */
int sg_render(uint64_t seed, int W, int H, int n_spheres, int n_panels,
              float *depth, float *normal, float *radiance, float *cam13) {
    if (W <= 0 || H <= 0 || n_spheres < 0 || n_panels < 0) return 1;
    scene_t sc;
    build_scene(&sc, seed, n_spheres, n_panels);
    sg_camera(W, H, cam13);
    const double fx = cam13[0], fy = cam13[1], cx = cam13[2], cy = cam13[3];
    const double *R = sc.R;
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            size_t i = (size_t)y * W + x;
            double u = x + 0.5, v = y + 0.5;
            v3 dv = v3m((u - cx) / fx, -(v - cy) / fy, -1.0);
            v3 dw = v3m(R[0] * dv.x + R[1] * dv.y + R[2] * dv.z,
                        R[3] * dv.x + R[4] * dv.y + R[5] * dv.z,
                        R[6] * dv.x + R[7] * dv.y + R[8] * dv.z);
            double t;
            v3 nw;
            int id = trace(&sc, sc.eye, dw, 1e-6, SG_FAR, 1, &t, &nw);
            float *nn = normal + 4 * i, *rr = radiance + 4 * i;
            if (id == -2) {
                depth[i] = INFINITY;
                nn[0] = nn[1] = nn[2] = nn[3] = 0.0f;
                rr[0] = rr[1] = rr[2] = rr[3] = 0.0f;
                continue;
            }
            /* face the normal toward the viewer (thin panels are seen from both sides) */
            if (dot(nw, dw) > 0.0) nw = scl(nw, -1.0);
            v3 P = add(sc.eye, scl(dw, t));
            double ndl = dot(nw, sc.light);
            double shade = 0.0;
            if (ndl > 0.0) {
                double ts;
                v3 ns_;
                int sh = trace(&sc, add(P, scl(nw, 1e-4)), sc.light, 1e-6, 1e30, 0, &ts, &ns_);
                shade = (sh == -2) ? ndl : 0.0;
            }
            v3 alb = albedo_of(&sc, id);
            /* view-space normal = R^T n_world */
            v3 nv = v3m(R[0] * nw.x + R[3] * nw.y + R[6] * nw.z,
                        R[1] * nw.x + R[4] * nw.y + R[7] * nw.z,
                        R[2] * nw.x + R[5] * nw.y + R[8] * nw.z);
            depth[i] = (float)t; /* the view ray has d_view.z = -1, so t is the linear depth */
            nn[0] = (float)nv.x;
            nn[1] = (float)nv.y;
            nn[2] = (float)nv.z;
            nn[3] = 0.0f;
            rr[0] = (float)(alb.x * shade);
            rr[1] = (float)(alb.y * shade);
            rr[2] = (float)(alb.z * shade);
            rr[3] = 0.0f;
        }
    }
    free(sc.sph);
    free(sc.pan);
    return 0;
}

/* 3-band real SH environment, 9 coefficients x RGB, [m][channel]:
 * band 0 U[0.5,1], higher bands U[-0.2,0.2]. */
void sg_sh(uint64_t seed, float *sh27) {
    uint64_t s = seed;
    for (int m = 0; m < 9; ++m)
        for (int c = 0; c < 3; ++c)
            sh27[3 * m + c] = (float)(m == 0 ? unif(&s, 0.5, 1.0) : unif(&s, -0.2, 0.2));
}

/* Uniform draws in [0,1) for host-side workload recipes. */
void sg_uniform(uint64_t seed, int n, double *out) {
    uint64_t s = seed;
    for (int i = 0; i < n; ++i) out[i] = sm64_unif(&s);
}
