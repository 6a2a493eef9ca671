/*
 * CPU oracle for the visibility-bitmask gather (Therrien, Levesque, Gilet,
 * "Screen Space Indirect Lighting with Visibility Bitmask", arXiv 2301.11376).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  The product path (the
 * CUDA library and its Python binding) never calls it and shares no code,
 * header, table or constant with it.
 *
 * Two independent programs live here:
 *   orc64_*  (oracle_fp64.c)  Algorithm 1 step by step in double precision,
 *            with the sector hit rule evaluated per sector by brute force.
 *   orc32_*  (replica_fp32.c) the binary32 operation sequence that decides
 *            the bitmasks, with the O(1) run-of-ones mask, written from the
 *            arithmetic specification; masks from the GPU must equal its
 *            masks bit for bit.
 * Both read the same problem description below.
 */
#ifndef SSILVB_ORACLE_H
#define SSILVB_ORACLE_H
#include <stdint.h>

typedef struct {
    int width, height;
    const float *depth;     /* [H*W], linear view depth z > 0; anything not in (0, +INF) is sky */
    const float *normal;    /* [H*W*4], view-space unit normal in xyz */
    const float *radiance;  /* [H*W*4], direct radiance in rgb */
    float fx, fy, cx, cy;   /* pinhole intrinsics in pixels; pixel centre at (x+0.5, y+0.5) */
    float view_to_world[9]; /* row-major rotation, used only for the ambient SH lookup */
    int num_slices;         /* N_d */
    int steps_per_side;     /* N_s */
    int sector_count;       /* N_b in {32, 64, 128} */
    int hit_rule;           /* 0 = at least half covered, 1 = floor/ceil of Algorithm 1 */
    int step_mode;          /* 0 = constant steps, 1 = quadratic ("exponential") steps */
    float radius;           /* R, metres */
    float thickness;        /* t, metres; +INF = horizon mode */
    float thickness_slope;  /* k_t: t(z) = t + k_t * z */
    const float *noise;     /* [16*2] (xi_phi, xi_s) per (y&3)*4 + (x&3); NULL = zero */
    int ambient_cones;      /* N_a, 0 = off */
    const float *sh;        /* [9*3] real SH radiance coefficients, [m][rgb] */
    int gi;                 /* 0 = skip the indirect-diffuse fetches (AO and ambient only) */
} orc_problem;

/* Per pixel listed in xy ([n*2] = x, y): out0[4] = (GI.rgb, AO), out1[4] = (ambient.rgb, 0),
 * masks[N_d][words] (words = 2 for N_b = 128, else 1; sector k is bit k % 64 of word k / 64),
 * margin[N_d] = smallest distance, in sector units, of any
 * hit-rule decision of that slice from its rounding boundary, and ratio[N_d] = smallest ratio of
 * such a distance to a bound on how far the binary32 evaluation of that decision's endpoints can
 * lie from these FP64 values (a ratio above 1: binary32 takes the same decision).  Any output
 * pointer may be NULL.  Returns 0, or a nonzero code for an invalid problem.  The pixel loop runs
 * on orc_threads() threads; every result is independent of the thread count. */
int orc64_pixels(const orc_problem *pb, int n, const int32_t *xy, double *out0, double *out1,
                 uint64_t *masks, double *margin, double *ratio);

/* orc64_pixels with two optional per-sample arrays, laid out per listed pixel as [N_d][2 sides][N_s]
 * entries (side -omega first):
 *   forced (input, int16 pairs (lo, hi)): the decision-forced evaluation.  Each visited sample sets
 *     exactly the sectors [lo, hi) (none when hi <= lo) instead of those of the FP64 hit rule; the
 *     geometry, the cosines, the per-sector crediting of indirect light, AO and the ambient cones
 *     stay in FP64.  Given the replica's runs (orc32_pixels_ex), it evaluates the outputs in FP64
 *     on the binary32 decisions.  margin and ratio still describe the FP64 decisions.  Returns 11
 *     for a run outside [0, N_b].
 *   endpoints (output, 4 doubles): (X_f, X_b, e_f, e_b), the unclamped FP64 sector coordinates and
 *     their binary32 error bounds, written for every visited sample, left as they were elsewhere.
 *   steps (output, 2 int32): (dx, dy), the pixel offset each step reads (the binary32 nearest-pixel
 *     decision), written for every step of a pixel with geometry, on screen or not. */
int orc64_pixels_ex(const orc_problem *pb, int n, const int32_t *xy, double *out0, double *out1,
                    uint64_t *masks, double *margin, double *ratio, const int16_t *forced, double *endpoints,
                    int32_t *steps);

/* Same, in the binary32 arithmetic of the gather.  counts (may be NULL) receives
 * [0] pixels, [1] sky pixels, [2] slices, [3] samples visited, [4] samples skipped,
 * [5] samples that set at least one new sector (GI fetches), [6] algorithmic ops. */
int orc32_pixels(const orc_problem *pb, int n, const int32_t *xy, float *out0, float *out1,
                 uint64_t *masks, int64_t *counts);

/* orc32_pixels with two optional per-sample arrays in the layout of orc64_pixels_ex:
 *   runs (output, int16 pairs): the sector run [lo, hi) each sample sets, (0, 0) where it sets none
 *     (skipped, in the edge band, or an empty run); written for every entry.
 *   endpoints (output, 2 floats): the unclamped binary32 sector coordinates (X_f, X_b) of every
 *     sample that reaches the front angle (X_b only past the edge-band test), left as they were
 *     elsewhere. */
int orc32_pixels_ex(const orc_problem *pb, int n, const int32_t *xy, float *out0, float *out1,
                    uint64_t *masks, int64_t *counts, int16_t *runs, float *endpoints);

/* Threads of the pixel loops: n > 0 sets the count; returns the count in use (1 when built without
 * OpenMP). */
int orc_threads(int n);

/* The replica's own arccosine (Abramowitz and Stegun 4.4.46 in binary32), exposed for tests. */
float orc32_acos(float x);
/* The replica's own reciprocal square root (integer seed + 3 Newton steps), for tests. */
float orc32_rsqrt(float x);
/* The replica's O(1) sector mask for endpoints A <= B (sector units), for tests. */
uint64_t orc32_sector_mask(float A, float B, int nb, int hit_rule);
/* Test helpers (replica_fp32.c): exhaustive arccosine sweep over [0, 1] and rsqrt error sweep. */
void orc32_acos_sweep(int stride, double *max_err, int64_t *increases);
double orc32_rsqrt_sweep(double lo, double hi, int n);
/* The FP64 oracle's per-sector brute-force mask, for tests (first word; all words). */
uint64_t orc64_sector_mask(double A, double B, int nb, int hit_rule);
void orc64_sector_mask_words(double A, double B, int nb, int hit_rule, uint64_t *out2);
/* The replica's O(1) mask as two 64-bit words, for tests. */
void orc32_sector_mask_words(float A, float B, int nb, int hit_rule, uint64_t *out2);
/* The replica's per-launch ambient coefficients: the SH environment sh[27] seen through the
 * view-to-world rotation R[9] as L(a) = b.a + a^T Q a per channel; b_out[9], q_out[18]
 * (Q as xx, yy, zz, xy, xz, yz). */
void orc32_ambient_form(const float *R, const float *sh, float *b_out, float *q_out);

#endif
