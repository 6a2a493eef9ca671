// Visibility-bitmask gather kernel for sm_103a (GB300).
//
// Per pixel: Algorithm 1 of Therrien, Levesque, Gilet, "Screen Space Indirect
// Lighting with Visibility Bitmask" (Section 3.1), the directionally occluded
// ambient cones of Section 3.2 and the indirect diffuse term of Section 3.3.
//
// The binary32 operation sequence on the bitmask path is fixed: round to
// nearest even, fused multiply-adds only where fmaf() is written (the file is
// built with -fmad=false; pfma/pmul/psub do two of the listed operations at
// once, each half exactly the scalar one), IEEE sqrt, no flush to zero.  Integer decisions
// taken from floating point (which pixel a step reads, which sectors a sample
// covers) are therefore reproducible bit for bit on any IEEE machine.
//
// Readings of the paper used here:
//   - slices i = 0..N_d-1 at azimuth (i + xi_phi) pi / N_d; steps j = 0..N_s-1
//     on each side at offset r (j+1+xi_s)/(N_s+1) (or its square for the
//     quadratic step mode), side -omega first, near to far;
//   - the back sample lies behind the front one along the centre pixel's view
//     ray, s_b = s_f + t p/|p| (Figure 4);
//   - elevation h = sigma acos(l.v/|l|), sector coordinate
//     X = (h - gamma) N_b/pi + N_b/2 clamped to [0, N_b], gamma the signed angle
//     of the projected normal (Eq. 4: the bit field is centred on it);
//   - a sector is occluded when at least half covered (round criterion), i.e.
//     the sectors whose centres lie in [A, B] when B - A >= 1/2, set at once;
//   - GI weight (newly occluded sectors / N_b) max(0, n_p.l) max(0, -n_j.l).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace ssilvb {

constexpr int kMaxSlices = 16;
constexpr int kMaxCones = 8;
constexpr int kSlots = 9;  // shared-memory words per thread for slice-end state (gather_pixel)

// Everything a launch needs, passed by value as a __grid_constant__ parameter.
struct GatherParams {
    const float *depth;
    const char *normal;
    const char *radiance;
    float *out0;
    float *out1;
    void *masks;
    char *light_out;       // multi-bounce light buffer for the next frame (or null)
    size_t light_pitch;    // bytes
    const char *direct;    // this frame's direct light for the bounce epilogue
    size_t direct_pitch;   // bytes
    float gain;            // bounce gain
    size_t depth_pitch;    // elements (floats)
    size_t normal_pitch;   // bytes
    size_t radiance_pitch; // bytes
    size_t out0_pitch;     // elements (floats)
    size_t out1_pitch;     // elements (floats)
    int W, H;
    int y0, y1;            // centre-pixel rows [y0, y1) this launch covers (samples read the whole frame)
    int band_rows;         // class mapping: patches run in bands of about this many patch rows, column by
                           // column within a band (1: raster order); the launch grid carries it
    int nd, ns, na;
    int hit_rule, step_mode, gi;
    // per-launch binary32 constants
    float inv_fx, inv_fy, kx0, ninv_fy, ky0;
    float Rfx, dn, K, half_nb, f_nb, inv_nb, inv_nd;
    float edge_hi, edge_lo;  // front endpoints beyond these occlude nothing (side +omega / -omega)
    float sdel, cdel;        // sine and cosine of half a sector (0 and 1 for the floor/ceil rule)
    float t0, kt;
    float xi_s[16];
    float dcos[16][kMaxSlices];
    float dsin[16][kMaxSlices];
    float ccos[kMaxCones], csin[kMaxCones];
    // The SH environment as a quadratic form of the view-space direction a: L(a) = b.a + a^T Q a
    // per channel, Q as (xx, yy, zz, xy, xz, yz) (Section 3.2's ambient light, 3 SH bands).
    float amb_b[3][3];
    float amb_q[3][6];
};

// Packed binary32 pairs (add/sub/mul/fma.rn.f32x2).  Each half is one IEEE binary32 operation
// rounded to nearest even with subnormals kept, i.e. exactly the scalar operation, so computing two
// independent values as a pair changes no result bit and takes one issue slot instead of two.
#define SSILVB_PAIR_OP3(name, op)                                                                    \
    __device__ __forceinline__ float2 name(float2 a, float2 b, float2 c) {                         \
        float2 d;                                                                                  \
        asm("{.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"      \
            "mov.b64 rc, {%6, %7};\n\t" op " rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"            \
            : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y)); \
        return d;                                                                                  \
    }
#define SSILVB_PAIR_OP2(name, op)                                                                    \
    __device__ __forceinline__ float2 name(float2 a, float2 b) {                                   \
        float2 d;                                                                                  \
        asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"          \
            op " rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"                                            \
            : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                     \
        return d;                                                                                  \
    }
SSILVB_PAIR_OP3(pfma, "fma.rn.f32x2")
SSILVB_PAIR_OP2(pmul, "mul.rn.f32x2")
SSILVB_PAIR_OP2(psub, "sub.rn.f32x2")
#undef SSILVB_PAIR_OP3
#undef SSILVB_PAIR_OP2
__device__ __forceinline__ float2 bcast(float a) { return make_float2(a, a); }

// Abramowitz and Stegun 4.4.46: acos(x) = sqrt(1 - x) (a0 + a1 x + ... + a7 x^7), 0 <= x <= 1.
__device__ __forceinline__ float own_acos(float c) {
    const float a = fabsf(c);
    const float s = sqrtf(fmaxf(1.0f - a, 0.0f));  // |c| > 1 (rounding) gives acos(+-1)
    float P = fmaf(-0.0012624911f, a, 0.0066700901f);
    P = fmaf(P, a, -0.0170881256f);
    P = fmaf(P, a, 0.0308918810f);
    P = fmaf(P, a, -0.0501743046f);
    P = fmaf(P, a, 0.0889789874f);
    P = fmaf(P, a, -0.2145988016f);
    P = fmaf(P, a, 1.5707963050f);
    const float r = s * P;
    return c < 0.0f ? 3.14159265358979323846f - r : r;
}

// Reciprocal square root: integer seed 0x5f3759df - (bits >> 1) (Lomont 2003), then
// three Newton steps y <- y (1.5 - 0.5 x y^2).  Branch-free; reproducible on any IEEE FPU.
__device__ __forceinline__ float own_rsqrt(float x) {
    x = fmaxf(x, 1.17549435e-38f);
    float y = __uint_as_float(0x5f3759dfu - (__float_as_uint(x) >> 1));
    const float hx = 0.5f * x;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float t = y * y;
        const float u = fmaf(-hx, t, 1.5f);
        y = y * u;
    }
    return y;
}

// own_rsqrt and own_acos of two arguments at once, operation for operation the same.
__device__ __forceinline__ float2 own_rsqrt_pair(float2 x) {
    x.x = fmaxf(x.x, 1.17549435e-38f);
    x.y = fmaxf(x.y, 1.17549435e-38f);
    float2 y = make_float2(__uint_as_float(0x5f3759dfu - (__float_as_uint(x.x) >> 1)),
                           __uint_as_float(0x5f3759dfu - (__float_as_uint(x.y) >> 1)));
    const float2 nhx = pmul(bcast(-0.5f), x);  // -(0.5 x), exactly
#pragma unroll
    for (int k = 0; k < 3; ++k) y = pmul(y, pfma(nhx, pmul(y, y), bcast(1.5f)));
    return y;
}

__device__ __forceinline__ float2 own_acos_pair(float2 c) {
    const float2 a = make_float2(fabsf(c.x), fabsf(c.y));
    const float2 om = psub(bcast(1.0f), a);
    const float2 s = make_float2(sqrtf(fmaxf(om.x, 0.0f)), sqrtf(fmaxf(om.y, 0.0f)));
    float2 Q = pfma(bcast(-0.0012624911f), a, bcast(0.0066700901f));
    Q = pfma(Q, a, bcast(-0.0170881256f));
    Q = pfma(Q, a, bcast(0.0308918810f));
    Q = pfma(Q, a, bcast(-0.0501743046f));
    Q = pfma(Q, a, bcast(0.0889789874f));
    Q = pfma(Q, a, bcast(-0.2145988016f));
    Q = pfma(Q, a, bcast(1.5707963050f));
    const float2 r = pmul(s, Q);
    return make_float2(c.x < 0.0f ? 3.14159265358979323846f - r.x : r.x,
                       c.y < 0.0f ? 3.14159265358979323846f - r.y : r.y);
}

// 1.5 * 2^23: adding it to |v| < 2^22 leaves round(v) in the low mantissa bits.
constexpr float kMagic = 12582912.0f;
constexpr float kHalfPi = 1.57079637050628662109375f;  // pi/2 rounded to binary32
constexpr int kMagicBits = 0x4B400000;

// Bits [lo, min(lo + cnt, 32)) of a 32-bit word, lo, cnt >= 0 (0 when lo >= 32 or cnt == 0).
__device__ __forceinline__ uint32_t run32(int lo, int cnt) {
    uint32_t r;
    asm("bmsk.clamp.b32 %0, %1, %2;" : "=r"(r) : "r"(lo), "r"(cnt));
    return r;
}

// 128 sectors: four 32-bit words, sector k in bit k % 32 of word k / 32.
struct Mask128 {
    uint32_t w[4];
    __device__ __forceinline__ Mask128() {}
    __device__ __forceinline__ Mask128(int zero) { w[0] = w[1] = w[2] = w[3] = (uint32_t)zero; }
    __device__ __forceinline__ Mask128 operator&(const Mask128 &o) const {
        Mask128 r;
        for (int i = 0; i < 4; ++i) r.w[i] = w[i] & o.w[i];
        return r;
    }
    __device__ __forceinline__ Mask128 operator~() const {
        Mask128 r;
        for (int i = 0; i < 4; ++i) r.w[i] = ~w[i];
        return r;
    }
    __device__ __forceinline__ Mask128 &operator|=(const Mask128 &o) {
        for (int i = 0; i < 4; ++i) w[i] |= o.w[i];
        return *this;
    }
};

template <int NB> struct MaskT;
template <> struct MaskT<32> { using T = uint32_t; };
template <> struct MaskT<64> { using T = unsigned long long; };
template <> struct MaskT<128> { using T = Mask128; };

template <int NB> __device__ __forceinline__ typename MaskT<NB>::T run_mask(int lo, int hi);
template <> __device__ __forceinline__ uint32_t run_mask<32>(int lo, int hi) { return run32(lo, hi - lo); }
// Runs for 64 and 128 sectors (0 <= lo <= hi): word i holds sectors [32 i, 32 i + 32); bmsk.clamp
// clips a run at the top of its word by itself, so only the start needs moving into the word.
template <> __device__ __forceinline__ unsigned long long run_mask<64>(int lo, int hi) {
    const uint32_t w0 = run32(lo, hi - lo);
    const int a1 = max(lo - 32, 0);
    const uint32_t w1 = run32(a1, max(hi - 32 - a1, 0));
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(w0), "r"(w1));
    return r;
}

template <> __device__ __forceinline__ Mask128 run_mask<128>(int lo, int hi) {
    Mask128 r;
    r.w[0] = run32(lo, hi - lo);
#pragma unroll
    for (int i = 1; i < 4; ++i) {
        const int a = max(lo - 32 * i, 0);
        r.w[i] = run32(a, max(hi - 32 * i - a, 0));
    }
    return r;
}

__device__ __forceinline__ int popc_(uint32_t v) { return __popc(v); }
__device__ __forceinline__ int popc_(unsigned long long v) { return __popcll(v); }
__device__ __forceinline__ int popc_(const Mask128 &v) {
    return __popc(v.w[0]) + __popc(v.w[1]) + __popc(v.w[2]) + __popc(v.w[3]);
}

// Sector run of a sample with endpoints A <= B (sector units, already in [0, N_b]).
template <int NB>
__device__ __forceinline__ typename MaskT<NB>::T sector_run(float A, float B, int hit_rule) {
    int lo, hi;
    if (hit_rule == 0) {
        // ceil(A - 1/2) and floor(B + 1/2), exact through a directed-rounding add of 1.5*2^23
        lo = __float_as_int(__fadd_ru(A - 0.5f, kMagic)) - kMagicBits;
        hi = __float_as_int(__fadd_rd(B + 0.5f, kMagic)) - kMagicBits;
        if (!(B - A >= 0.5f)) hi = lo;
    } else {
        lo = __float_as_int(__fadd_rd(A, kMagic)) - kMagicBits;
        hi = min(lo + (__float_as_int(__fadd_ru(B - A, kMagic)) - kMagicBits), NB);
    }
    hi = max(hi, lo);
    return run_mask<NB>(lo, hi);
}

template <bool F16>
__device__ __forceinline__ float3 load_xyz(const char *base, size_t pitch, int x, int y) {
    const char *row = base + (size_t)y * pitch;
    if (F16) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(row) + x);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
        return make_float3(a.x, a.y, b.x);
    } else {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(row) + x);
        return make_float3(v.x, v.y, v.z);
    }
}

// Storage of normals and radiance, the kernels' FMT parameter (the ABI's format codes): 0 two
// binary32 planes, 1 two binary16 planes, 2 one interleaved binary16 plane.
constexpr int kFmtF32 = 0, kFmtF16 = 1, kFmtF16x8 = 2;

// A sample's normal and radiance: from the two planes, or (FMT 2) from its one 16-byte interleaved
// record (n.x, n.y, n.z, c.r, c.g, c.b, -, -) in a single load.  The values are the same binary16
// numbers either way.
template <int FMT>
__device__ __forceinline__ void load_normal_radiance(const GatherParams &P, int x, int y, float3 &n, float3 &c) {
    constexpr bool F16 = FMT != kFmtF32;
    if (FMT == kFmtF16x8) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(P.normal + (size_t)y * P.normal_pitch) + x);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
        const float2 d = __half22float2(*reinterpret_cast<const __half2 *>(&v.z));
        n = make_float3(a.x, a.y, b.x);
        c = make_float3(b.y, d.x, d.y);
    } else {
        c = load_xyz<F16>(P.radiance, P.radiance_pitch, x, y);
        n = load_xyz<F16>(P.normal, P.normal_pitch, x, y);
    }
}

// The centre pixel's normal: its plane, or the first half of its interleaved record.
template <int FMT>
__device__ __forceinline__ float3 load_normal(const GatherParams &P, int x, int y) {
    constexpr bool F16 = FMT != kFmtF32;
    if (FMT == kFmtF16x8) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(P.normal + (size_t)y * P.normal_pitch) + 2 * x);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
        return make_float3(a.x, a.y, b.x);
    }
    return load_xyz<F16>(P.normal, P.normal_pitch, x, y);
}

// 0 < z < +INF (NaN and negative values fail): positive finite binary32 bit patterns are 1 .. 0x7f7fffff.
__device__ __forceinline__ bool is_geometry(float z) { return __float_as_uint(z) - 1u < 0x7f7fffffu; }

// Multi-bounce epilogue (Section 4.3): the next frame's light = direct + gain * GI.
template <int FMT>
__device__ __forceinline__ void write_light(const GatherParams &P, int x, int y, float gr, float gg, float gb) {
    constexpr bool F16 = FMT != kFmtF32;
    const float3 c = load_xyz<F16>(P.direct, P.direct_pitch, x, y);
    const float r = fmaf(P.gain, gr, c.x), g = fmaf(P.gain, gg, c.y), b = fmaf(P.gain, gb, c.z);
    char *row = P.light_out + (size_t)y * P.light_pitch;
    if (F16) {
        const __half2 h0 = __floats2half2_rn(r, g), h1 = __floats2half2_rn(b, 0.0f);
        uint2 v;
        v.x = *reinterpret_cast<const uint32_t *>(&h0);
        v.y = *reinterpret_cast<const uint32_t *>(&h1);
        reinterpret_cast<uint2 *>(row)[x] = v;
    } else {
        reinterpret_cast<float4 *>(row)[x] = make_float4(r, g, b, 0.0f);
    }
}

// Per-pixel state the sample loop reads.
struct Pixel {
    float z, ax, by, px, py, vx, vy, vz, tp, t2, m2t;
    float del, xdel;  // step unit r/(N_s+1) and the jitter xi_s times it (constant steps)
    float dn_, xidn, rpx;  // quadratic steps: 1/(N_s+1), xi_s/(N_s+1), r
    int qx0, qy0;     // x, y minus the bit pattern of 1.5*2^23
    float3 n;
};

// The rest of one sample of side POS (+omega when true) once its front cosine lies outside the
// side's edge band: front and back endpoints, sector run, mask update and indirect light.
// (lx, ly, lz) = l = s_f - p, dv = l.v, ll = |l|^2; (qx, qy) the sample pixel.
// Sector coordinates of a sample's front and back endpoints, and 1/|l|, for a sample outside the
// cosine band; false when its front endpoint still lies in the band in sector units (half a sector
// for the half-covered rule, the edge for floor/ceil), so that it occludes nothing.  The back sample
// lies thickness t behind the front one along the centre pixel's view ray; t = infinity puts the
// back endpoint on the side's hemisphere edge.  Both angles are one packed pair: a sample outside
// the cosine band almost always needs both.
template <bool INF_T, bool POS>
__device__ __forceinline__ bool endpoints(const GatherParams &P, const Pixel &X, float dv, float ll, float off,
                                          float &rl, float &Xf, float &Xb) {
    const float sK = POS ? P.K : -P.K;
    if (!INF_T) {
        const float dvb = dv - X.tp;
        const float llb = fmaf(X.m2t, dv, ll + X.t2);
        const float2 r2 = own_rsqrt_pair(make_float2(ll, llb));
        rl = r2.x;
        const float2 e2 = pfma(own_acos_pair(pmul(make_float2(dv, dvb), r2)), bcast(sK), bcast(off));
        Xf = fminf(fmaxf(e2.x, 0.0f), P.f_nb);
        Xb = fminf(fmaxf(e2.y, 0.0f), P.f_nb);
    } else {
        rl = own_rsqrt(ll);
        Xf = fminf(fmaxf(fmaf(own_acos(dv * rl), sK, off), 0.0f), P.f_nb);
        Xb = POS ? P.f_nb : 0.0f;
    }
    return !(POS ? Xf > P.edge_hi : Xf < P.edge_lo);
}

// Sector run [A, B] (the back endpoint lies toward this side's edge; a rounding-level reversal gives
// B < A and no sector), mask update, and the indirect light of the newly occluded sectors
// (Section 3.3).
template <int NB, int FMT, bool POS>
__device__ __forceinline__ void occlude(const GatherParams &P, const Pixel &X, float lx, float ly, float lz, float rl,
                                        float Xf, float Xb, int qx, int qy, typename MaskT<NB>::T &b, float &GIr,
                                        float &GIg, float &GIb) {
    using M = typename MaskT<NB>::T;
    const float A = POS ? Xf : Xb, B = POS ? Xb : Xf;
    const M bj = sector_run<NB>(A, B, P.hit_rule);
    const int newly = popc_(bj & ~b);
    b |= bj;
    if (newly > 0 && P.gi) {
        float3 cj, nj;
        load_normal_radiance<FMT>(P, qx, qy, nj, cj);
        const float cp = fmaxf(fmaf(X.n.x, lx, fmaf(X.n.y, ly, X.n.z * lz)) * rl, 0.0f);
        const float cq = fmaxf(-(fmaf(nj.x, lx, fmaf(nj.y, ly, nj.z * lz)) * rl), 0.0f);
        const float wgt = (((float)newly * P.inv_nb) * cp) * cq;
        GIr = fmaf(wgt, cj.x, GIr);
        GIg = fmaf(wgt, cj.y, GIg);
        GIb = fmaf(wgt, cj.z, GIb);
    }
}

// The rest of a step pair's samples that left the cosine band (fa / fb): endpoints, then the mask
// and indirect light, sample j before sample j + 1.
template <int NB, int FMT, bool INF_T, bool POS>
__device__ __forceinline__ void pair_full(const GatherParams &P, const Pixel &X, bool fa, bool fb, float2 lx,
                                          float2 ly, float2 lz, float2 dv, float2 ll, int qxa, int qya, int qxb,
                                          int qyb, float off, typename MaskT<NB>::T &b, float &GIr, float &GIg,
                                          float &GIb) {
    if (!(fa | fb)) return;  // the common case: one branch for the pair
    if (fa) {
        float rl, Xf, Xb;
        if (endpoints<INF_T, POS>(P, X, dv.x, ll.x, off, rl, Xf, Xb))
            occlude<NB, FMT, POS>(P, X, lx.x, ly.x, lz.x, rl, Xf, Xb, qxa, qya, b, GIr, GIg, GIb);
    }
    if (fb) {
        float rl, Xf, Xb;
        if (endpoints<INF_T, POS>(P, X, dv.y, ll.y, off, rl, Xf, Xb))
            occlude<NB, FMT, POS>(P, X, lx.y, ly.y, lz.y, rl, Xf, Xb, qxb, qyb, b, GIr, GIg, GIb);
    }
}

// Steps of one side, near to far, two per iteration.  What every step needs (offset, nearest
// pixel, depth, l = s_f - p, its cosine to v and |l|^2) is computed for steps j and j + 1 as
// packed pairs; the rest of each sample then runs for step j before step j + 1, so the bitmask and
// the indirect light see the samples in the same order as one step at a time.  Once a step leaves
// the screen every later step of that side does too (the rounded offset is monotone in j, x and
// y offsets alike, since the noise xi_s is in [0, 1)), so the side ends there.
template <int NB, int FMT, bool INF_T, int STEP_MODE, bool POS>
__device__ __forceinline__ void march_side(const GatherParams &P, const Pixel &X, int x, int y, float cphi,
                                           float sphi, float off, float thr2,
                                           typename MaskT<NB>::T &b, float &GIr, float &GIg, float &GIb) {
    const float wsx = POS ? cphi : -cphi, wsy = POS ? sphi : -sphi;
    int j0 = 0;
    {
        // Steps 0 .. J-1 provably stay on screen when the offset of step J-1 does (offsets grow with
        // j), which holds when ceil(o |w| + 1) is within the pixels left to the screen edge in this
        // side's direction along each axis (|round(o w)| <= o |w| + 1/2); and if the first step is
        // off the centre pixel so are the rest.  Each lane takes J = N_s when the last step fits,
        // else estimates J from the inverse of the offset formula and confirms it with that exact
        // bound, stepping back at most twice.  The warp runs the smallest J (in whole step pairs)
        // without the per-step screen and centre tests, then the remaining steps with them.  (A
        // copy of the checked loop rather than a template parameter of one loop: the shared form
        // compiled to 3 % slower code.)
        float o_first;
        if (STEP_MODE == 0) {
            o_first = fmaf(1.0f, X.del, X.xdel);
        } else {
            const float uf = fmaf(1.0f, X.dn_, X.xidn);
            o_first = (uf * uf) * X.rpx;
        }
        const bool off_centre = (fmaf(o_first, wsx, kMagic) != kMagic) | (fmaf(o_first, wsy, kMagic) != kMagic);
        int J = 0;
        if (off_centre) {
            const float ax = fabsf(wsx), ay = fabsf(wsy);
            const int dxi = wsx >= 0.0f ? P.W - 1 - x : x, dyi = wsy >= 0.0f ? P.H - 1 - y : y;
            auto fits = [&](int n) {  // step n - 1 (and so every earlier step) on screen
                float o;
                if (STEP_MODE == 0) {
                    o = fmaf((float)n, X.del, X.xdel);
                } else {
                    const float u = fmaf((float)n, X.dn_, X.xidn);
                    o = (u * u) * X.rpx;
                }
                return __float2int_ru(fmaf(o, ax, 1.0f)) <= dxi && __float2int_ru(fmaf(o, ay, 1.0f)) <= dyi;
            };
            if (fits(P.ns)) {
                J = P.ns;
            } else {
                // only an estimate (fast approximate division and square root; NaN converts to
                // 0): fits() decides
                const float t = fminf(__fdividef((float)dxi - 1.0f, ax), __fdividef((float)dyi - 1.0f, ay));
                float jm;
                if (STEP_MODE == 0) {
                    jm = __fdividef(t - X.xdel, X.del);
                } else {
                    const float q = __fdividef(fmaxf(t, 0.0f), X.rpx);
                    jm = __fdividef(q * rsqrtf(q) - X.xidn, X.dn_);
                }
                J = min(max(__float2int_rd(jm), 0), P.ns);
                if (J > 0 && !fits(J)) {
                    --J;
                    if (J > 0 && !fits(J)) J = 0;
                }
            }
        }
        const int Jw = __reduce_min_sync(__activemask(), J);
        j0 = Jw >= P.ns ? P.ns : (Jw & ~1);
        for (int j = 0; j < j0; j += 2) {
            const float2 jf = make_float2((float)(j + 1), (float)(j + 2));
            float2 o;
            if (STEP_MODE == 0) {
                o = pfma(jf, bcast(X.del), bcast(X.xdel));
            } else {
                const float2 uj = pfma(jf, bcast(X.dn_), bcast(X.xidn));
                o = pmul(pmul(uj, uj), bcast(X.rpx));
            }
            const float2 rx = pfma(o, bcast(wsx), bcast(kMagic)), ry = pfma(o, bcast(wsy), bcast(kMagic));
            const int qxa = __float_as_int(rx.x) + X.qx0, qya = __float_as_int(ry.x) + X.qy0;
            const int qxb = __float_as_int(rx.y) + X.qx0, qyb = __float_as_int(ry.y) + X.qy0;
            const bool onb = j + 1 < P.ns;  // false only for the last step of an odd N_s
            const float za = __ldg(P.depth + (unsigned)qya * (unsigned)P.depth_pitch + (unsigned)qxa);
            float zb = 0.0f;
            if (onb) zb = __ldg(P.depth + (unsigned)qyb * (unsigned)P.depth_pitch + (unsigned)qxb);
            const float2 dxf = psub(rx, bcast(kMagic)), dyf = psub(ry, bcast(kMagic));
            const float2 aq = pfma(dxf, bcast(P.inv_fx), bcast(X.ax)), bq = pfma(dyf, bcast(P.ninv_fy), bcast(X.by));
            const float2 zq = make_float2(za, zb);
            const float2 lx = pfma(aq, zq, bcast(-X.px)), ly = pfma(bq, zq, bcast(-X.py));
            const float2 lz = psub(bcast(X.z), zq);
            const float2 dv = pfma(lx, bcast(X.vx), pfma(ly, bcast(X.vy), pmul(lz, bcast(X.vz))));
            const float2 ll = pfma(lx, lx, pfma(ly, ly, pmul(lz, lz)));
            const float2 lim = pmul(bcast(thr2), ll);
            pair_full<NB, FMT, INF_T, POS>(P, X, is_geometry(za) && !(dv.x * fabsf(dv.x) < lim.x),
                                           is_geometry(zb) && !(dv.y * fabsf(dv.y) < lim.y), lx, ly, lz, dv, ll,
                                           qxa, qya, qxb, qyb, off, b, GIr, GIg, GIb);
        }
        if (j0 >= P.ns) return;
    }

    for (int j = j0; j < P.ns; j += 2) {
        // offsets r (j + 1 + xi_s)/(N_s + 1), or the quadratic form, of steps j and j + 1
        const float2 jf = make_float2((float)(j + 1), (float)(j + 2));
        float2 o;
        if (STEP_MODE == 0) {
            o = pfma(jf, bcast(X.del), bcast(X.xdel));
        } else {
            const float2 uj = pfma(jf, bcast(X.dn_), bcast(X.xidn));
            o = pmul(pmul(uj, uj), bcast(X.rpx));
        }
        // nearest pixels: fma(o, w, 1.5*2^23) rounds o*w to an integer (ties to even) in the low
        // mantissa bits, so q = bits - (0x4B400000 - x)
        const float2 rx = pfma(o, bcast(wsx), bcast(kMagic)), ry = pfma(o, bcast(wsy), bcast(kMagic));
        const int qxa = __float_as_int(rx.x) + X.qx0, qya = __float_as_int(ry.x) + X.qy0;
        if (!((unsigned)qxa < (unsigned)P.W && (unsigned)qya < (unsigned)P.H)) break;
        const int qxb = __float_as_int(rx.y) + X.qx0, qyb = __float_as_int(ry.y) + X.qy0;
        const bool onb = j + 1 < P.ns && (unsigned)qxb < (unsigned)P.W && (unsigned)qyb < (unsigned)P.H;
        // depths; 0 (not geometry) for the centre pixel and for a step past the screen or past N_s
        float za = 0.0f, zb = 0.0f;
        if ((qxa != x) | (qya != y)) za = __ldg(P.depth + (unsigned)qya * (unsigned)P.depth_pitch + (unsigned)qxa);
        if (onb && ((qxb != x) | (qyb != y)))
            zb = __ldg(P.depth + (unsigned)qyb * (unsigned)P.depth_pitch + (unsigned)qxb);
        // front samples: the view ray of the sample pixel is the centre ray plus the pixel offset
        // over the focal length; l = s_f - p, its cosine to v and |l|^2
        const float2 dxf = psub(rx, bcast(kMagic)), dyf = psub(ry, bcast(kMagic));
        const float2 aq = pfma(dxf, bcast(P.inv_fx), bcast(X.ax)), bq = pfma(dyf, bcast(P.ninv_fy), bcast(X.by));
        const float2 zq = make_float2(za, zb);
        const float2 lx = pfma(aq, zq, bcast(-X.px)), ly = pfma(bq, zq, bcast(-X.py));
        const float2 lz = psub(bcast(X.z), zq);
        const float2 dv = pfma(lx, bcast(X.vx), pfma(ly, bcast(X.vy), pmul(lz, bcast(X.vz))));
        const float2 ll = pfma(lx, lx, pfma(ly, ly, pmul(lz, lz)));
        // Inside this side's edge band (cosine dv/|l| below thr, compared as dv |dv| < thr |thr| |l|^2
        // through the monotone map x -> x |x|) the back endpoint lies still closer to the edge, so
        // no sector is half covered.
        const float2 lim = pmul(bcast(thr2), ll);
        pair_full<NB, FMT, INF_T, POS>(P, X, is_geometry(za) && !(dv.x * fabsf(dv.x) < lim.x),
                                       onb && is_geometry(zb) && !(dv.y * fabsf(dv.y) < lim.y), lx, ly, lz, dv, ll,
                                       qxa, qya, qxb, qyb, off, b, GIr, GIg, GIb);
        if (!onb) break;
    }
}

// The whole per-pixel gather (Algorithm 1 with Sections 3.2 and 3.3) for pixel (x, y) of
// noise class cls = (y & 3) * 4 + (x & 3).
//
// The state a slice touches only at its end (AO and ambient sums, and the slice frame cg, sg, s the
// ambient cones need) lives in shared memory: kSlots words per thread, word k at sl[k * STRIDE],
// STRIDE the block's thread count.  Kept in registers it is live across both step loops, and at 9
// blocks of 128 threads per SM the register budget then spills; in shared memory it costs a few
// accesses per slice.  `volatile` keeps each access a real one.
template <int NB, int FMT, bool INF_T, int STEP_MODE, int STRIDE>
__device__ __forceinline__ void gather_pixel(const GatherParams &P, int x, int y, volatile float *sl) {
    using M = typename MaskT<NB>::T;
    const float z = __ldg(P.depth + (unsigned)y * (unsigned)P.depth_pitch + (unsigned)x);
    float4 *o0 = reinterpret_cast<float4 *>(P.out0 + (size_t)y * P.out0_pitch) + x;
    if (!is_geometry(z)) {
        *o0 = make_float4(0.0f, 0.0f, 0.0f, 1.0f);
        if (P.na > 0) *(reinterpret_cast<float4 *>(P.out1 + (size_t)y * P.out1_pitch) + x) = make_float4(0, 0, 0, 0);
        if (P.masks)
            for (int i = 0; i < P.nd; ++i) reinterpret_cast<M *>(P.masks)[((size_t)i * P.H + y) * P.W + x] = 0;
        if (P.light_out) write_light<FMT>(P, x, y, 0.0f, 0.0f, 0.0f);
        return;
    }

    // Pixel setup (Algorithm 1: p, n_p, projected radius, step size).
    Pixel X;
    X.z = z;
    const float u = (float)x + 0.5f, v = (float)y + 0.5f;
    X.ax = fmaf(u, P.inv_fx, P.kx0);
    X.by = fmaf(v, P.ninv_fy, P.ky0);
    X.px = X.ax * z;
    X.py = X.by * z;
    const float rd = own_rsqrt(fmaf(X.ax, X.ax, fmaf(X.by, X.by, 1.0f)));
    X.vx = -(X.ax * rd);
    X.vy = -(X.by * rd);
    X.vz = rd;
    X.n = load_normal<FMT>(P, x, y);
    const float rpx = fminf(P.Rfx / z, 1048576.0f);
    const int cls = (y & 3) * 4 + (x & 3);
    const float xidn = P.xi_s[cls] * P.dn;
    X.del = rpx * P.dn;
    X.xdel = xidn * rpx;
    X.dn_ = P.dn;
    X.xidn = xidn;
    X.rpx = rpx;
    X.qx0 = x - kMagicBits;
    X.qy0 = y - kMagicBits;
    X.tp = X.t2 = X.m2t = 0.0f;
    if (!INF_T) {
        X.tp = fmaf(P.kt, z, P.t0);
        X.t2 = X.tp * X.tp;
        X.m2t = -2.0f * X.tp;
    }

    // slots: 0 AO, 1-3 ambient rgb, 4 cg, 5 sg, 6-8 s
    sl[0] = 0.0f;
    sl[STRIDE] = 0.0f;
    sl[2 * STRIDE] = 0.0f;
    sl[3 * STRIDE] = 0.0f;
    float GIr = 0.0f, GIg = 0.0f, GIb = 0.0f;
    for (int i = 0; i < P.nd; ++i) {
        const float cphi = P.dcos[cls][i], sphi = P.dsin[cls][i];
        // Slice plane: s = normalize(w3 - (w3.v) v), w3 the view-space image of omega.
        const float w3x = cphi * P.inv_fx, w3y = -(sphi * P.inv_fy);
        const float wv = fmaf(w3x, X.vx, w3y * X.vy);
        const float sx0 = fmaf(-wv, X.vx, w3x), sy0 = fmaf(-wv, X.vy, w3y), sz0 = -(wv * X.vz);
        const float rs = own_rsqrt(fmaf(sx0, sx0, fmaf(sy0, sy0, sz0 * sz0)));
        const float sx = sx0 * rs, sy = sy0 * rs, sz = sz0 * rs;
        // Projected normal angle gamma (the sector frame is centred on it, Eq. 4).
        const float nv = fmaf(X.n.x, X.vx, fmaf(X.n.y, X.vy, X.n.z * X.vz));
        const float nsd = fmaf(X.n.x, sx, fmaf(X.n.y, sy, X.n.z * sz));
        const float pn2 = fmaf(nv, nv, nsd * nsd);
        float cg = 1.0f, sg = 0.0f, gam = 0.0f;
        if (pn2 > 0.0f) {
            const float rpn = own_rsqrt(pn2);
            cg = nv * rpn;
            sg = nsd * rpn;
            // |gamma| from whichever of its cosine and sine is the smaller in magnitude, where the
            // arccosine is well conditioned: within pi/4 of 0 or pi, |gamma| = asin|sg| =
            // pi/2 - acos|sg| (cg >= 0) or pi/2 + acos|sg| (cg < 0); else acos(cg).
            if (fabsf(sg) <= fabsf(cg)) {
                const float a = own_acos(fabsf(sg));
                gam = cg >= 0.0f ? kHalfPi - a : kHalfPi + a;
            } else {
                gam = own_acos(cg);
            }
            if (nsd < 0.0f) gam = -gam;
        }
        const float off = fmaf(-gam, P.K, P.half_nb);
        // Edge-band cosine thresholds: a front direction at an angle from v above
        // gamma + pi/2 - delta (side +) or pi/2 - gamma - delta (side -), delta = half a sector
        // (0 for the floor/ceil rule), lies in the band; angles outside [0, pi] give 2 (all) or -2 (none).
        const float cu_p = fmaf(cg, P.cdel, sg * P.sdel), su_p = fmaf(sg, P.cdel, -(cg * P.sdel));
        const float cu_m = fmaf(cg, P.cdel, -(sg * P.sdel)), su_m = fmaf(sg, P.cdel, cg * P.sdel);
        const float thr_p = cu_p >= 0.0f ? -su_p : (su_p < 0.0f ? 2.0f : -2.0f);
        const float thr_m = cu_m >= 0.0f ? su_m : (su_m > 0.0f ? 2.0f : -2.0f);

        M b = 0;
        sl[4 * STRIDE] = cg;
        sl[5 * STRIDE] = sg;
        sl[6 * STRIDE] = sx;
        sl[7 * STRIDE] = sy;
        sl[8 * STRIDE] = sz;
        // Side -omega, then side +omega (Section 3.3: nearer samples occlude later ones first).
        march_side<NB, FMT, INF_T, STEP_MODE, false>(P, X, x, y, cphi, sphi, off, thr_m * fabsf(thr_m), b,
                                                     GIr, GIg, GIb);
        march_side<NB, FMT, INF_T, STEP_MODE, true>(P, X, x, y, cphi, sphi, off, thr_p * fabsf(thr_p), b,
                                                    GIr, GIg, GIb);

        // Slice end: unoccluded fraction, then the ambient cones (Section 3.2).
        sl[0] = sl[0] + (float)(NB - popc_(b)) * P.inv_nb;
        if (P.na > 0) {
            // Cone k's direction is a_k = c_k v + s_k s (c_k, s_k the cosine and sine of its angle from
            // v in the slice plane) and the environment is a quadratic form of a unit direction,
            // L(a) = b.a + a^T Q a.  The weighted sum over the cones, sum_k w_k L(a_k), is therefore
            // b.u + sum over Q's six entries of q_m t_m, with u = v sum w c + s sum w s and t_m the
            // entry's monomial of v times sum w c^2, plus that of s times sum w s^2, plus the symmetric
            // product of v and s times 2 sum w c s: five channel-independent sums over the cones.
            const float cg = sl[4 * STRIDE], sg = sl[5 * STRIDE];
            const int g = NB / P.na;
            float Wc = 0.0f, Ws = 0.0f, Wcc = 0.0f, Wss = 0.0f, Wcs = 0.0f;
#pragma unroll 1
            for (int k = 0; k < P.na; ++k) {
                const M Mk = run_mask<NB>(k * g, (k + 1) * g);
                const int freek = popc_(~b & Mk);
                const float ck = fmaf(cg, P.ccos[k], -(sg * P.csin[k]));
                const float sk = fmaf(sg, P.ccos[k], cg * P.csin[k]);
                const float wt = (float)freek * P.inv_nb;
                const float tc = wt * ck, ts = wt * sk;
                Wc = Wc + tc;
                Ws = Ws + ts;
                Wcc = fmaf(tc, ck, Wcc);
                Wss = fmaf(ts, sk, Wss);
                Wcs = fmaf(tc, sk, Wcs);
            }
            const float W2cs = Wcs + Wcs;
            const float sx = sl[6 * STRIDE], sy = sl[7 * STRIDE], sz = sl[8 * STRIDE];
            const float ux = fmaf(X.vx, Wc, sx * Ws), uy = fmaf(X.vy, Wc, sy * Ws), uz = fmaf(X.vz, Wc, sz * Ws);
            float acc[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) acc[ch] = fmaf(P.amb_b[ch][2], uz, fmaf(P.amb_b[ch][1], uy, P.amb_b[ch][0] * ux));
            const float vx2 = X.vx + X.vx, vy2 = X.vy + X.vy, sx2 = sx + sx, sy2 = sy + sy;
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                // Q's entries xx, yy, zz, xy, xz, yz: squares, doubled products, symmetric sums
                float pv, ps, pc;
                switch (m) {
                case 0: pv = X.vx * X.vx; ps = sx * sx; pc = X.vx * sx; break;
                case 1: pv = X.vy * X.vy; ps = sy * sy; pc = X.vy * sy; break;
                case 2: pv = X.vz * X.vz; ps = sz * sz; pc = X.vz * sz; break;
                case 3: pv = vx2 * X.vy; ps = sx2 * sy; pc = fmaf(X.vx, sy, X.vy * sx); break;
                case 4: pv = vx2 * X.vz; ps = sx2 * sz; pc = fmaf(X.vx, sz, X.vz * sx); break;
                default: pv = vy2 * X.vz; ps = sy2 * sz; pc = fmaf(X.vy, sz, X.vz * sy); break;
                }
                const float t = fmaf(pv, Wcc, fmaf(ps, Wss, pc * W2cs));
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) acc[ch] = fmaf(P.amb_q[ch][m], t, acc[ch]);
            }
            sl[STRIDE] = sl[STRIDE] + acc[0];
            sl[2 * STRIDE] = sl[2 * STRIDE] + acc[1];
            sl[3 * STRIDE] = sl[3 * STRIDE] + acc[2];
        }
        if (P.masks) reinterpret_cast<M *>(P.masks)[((size_t)i * P.H + y) * P.W + x] = b;
    }
    const float gr = GIr * P.inv_nd, gg = GIg * P.inv_nd, gb = GIb * P.inv_nd;
    *o0 = make_float4(gr, gg, gb, sl[0] * P.inv_nd);
    if (P.light_out) write_light<FMT>(P, x, y, gr, gg, gb);
    if (P.na > 0)
        *(reinterpret_cast<float4 *>(P.out1 + (size_t)y * P.out1_pitch) + x) =
            make_float4(sl[STRIDE] * P.inv_nd, sl[2 * STRIDE] * P.inv_nd, sl[3 * STRIDE] * P.inv_nd, 0.0f);
}

// Natural mapping: one thread per pixel, 32 x 8 pixel tiles.
template <int NB, int FMT, bool INF_T, int STEP_MODE>
__global__ void __launch_bounds__(256) gather_tile_kernel(const __grid_constant__ GatherParams P) {
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = P.y0 + blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= P.W || y >= P.y1) return;
    __shared__ float slots[kSlots * 256];
    gather_pixel<NB, FMT, INF_T, STEP_MODE, 256>(P, x, y, slots + threadIdx.x);
}

// Class-strided mapping.  A warp takes 8 x 4 pixels at stride 4 of a 32 x 16 pixel patch, all of
// one 4x4 noise class, so its 32 lanes share the slice directions and step offsets: their samples
// land on neighbouring pixels and their skip decisions mostly agree (a compact patch agrees more
// often than a 128-pixel row).  The 4 warps of a block take the 4 column classes of one row
// class; the row class is the fastest block index, so a patch's blocks run next to each other
// (the launch grid orders the patches: see the kernel).  MINB: blocks of 128 threads per SM the
// register budget is sized for.
__device__ __forceinline__ void patch_pixel(int patch_x, int patch_y, int row_class, int &x, int &y) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    x = patch_x * 32 + 4 * (lane & 7) + w;
    y = patch_y * 16 + 4 * (lane >> 3) + row_class;
}

template <int NB, int FMT, bool INF_T, int STEP_MODE, int MINB>
__global__ void __launch_bounds__(128, MINB) gather_class_kernel(const __grid_constant__ GatherParams P) {
    // The grid is (4 x band height, patch columns, bands) and blocks are numbered x fastest, so the
    // patches run band by band, column by column within a band (a band of one patch row is the
    // raster order).  On a large frame the blocks resident at once then cover a compact region
    // rather than a strip across the frame, and their indirect-light fetches share the L2.  Rows
    // past the launch's last one (a short last band) exit below.
    const int pcol = blockIdx.y, prow = blockIdx.z * (int)(gridDim.x >> 2) + (int)(blockIdx.x >> 2);
    int x, y;
    patch_pixel(pcol, prow, blockIdx.x & 3, x, y);
    y += P.y0;
    if (x >= P.W || y >= P.y1) return;
    __shared__ float slots[kSlots * 128];
    gather_pixel<NB, FMT, INF_T, STEP_MODE, 128>(P, x, y, slots + threadIdx.x);
}

// ---------------------------------------------------------------------------------------------
// Batched form: many frames of different sizes and parameters in one persistent launch.
// The work list is the concatenation of every frame's tiles: a tile is `rows` patch rows of one
// (patch column, row class) pair of the class-strided mapping, tiles_x = 4 ceil(W/32) of them per
// band of `rows` patch rows, bands top to bottom.  Each block takes the next tile from a queue
// counter in global memory; tiles are handed out in order, so a block's frame index only moves
// forward and the frame's parameters are copied to shared memory once per frame change.
struct FrameDesc {
    GatherParams P;
    int tile_begin;  // global index of the frame's first tile
    int tiles_x;     // tiles per band: 4 row classes per 32-pixel patch column
    int rows;        // patch rows (16 pixel rows each) per tile
    int pad;
};

struct BatchHeader {
    int n_frames;
    int total_tiles;
    int pad[2];
};

template <int NB, int FMT, bool INF_T, int STEP_MODE, int MINB>
__global__ void __launch_bounds__(128, MINB)
    gather_batch_kernel(const BatchHeader *__restrict__ hdr, const FrameDesc *__restrict__ frames,
                        unsigned *__restrict__ queue) {
    __shared__ GatherParams sP;
    __shared__ int s_tile, s_frame;
    __shared__ float slots[kSlots * 128];
    const int n_frames = hdr->n_frames, total = hdr->total_tiles;
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = (int)atomicAdd(queue, 1u);
            int f = cur < 0 ? 0 : cur;
            if (t < total)
                while (f + 1 < n_frames && __ldg(&frames[f + 1].tile_begin) <= t) ++f;
            s_tile = t;
            s_frame = f;
        }
        __syncthreads();
        const int t = s_tile, f = s_frame;
        if (t >= total) break;
        if (f != cur) {
            const int *src = reinterpret_cast<const int *>(&frames[f].P);
            int *dst = reinterpret_cast<int *>(&sP);
            for (int k = threadIdx.x; k < (int)(sizeof(GatherParams) / 4); k += blockDim.x) dst[k] = __ldg(src + k);
            cur = f;
            __syncthreads();
        }
        const int local = t - __ldg(&frames[f].tile_begin);
        const int tx = __ldg(&frames[f].tiles_x), rows = __ldg(&frames[f].rows);
        const int band = local / tx, xb = local - band * tx;
        for (int r = 0; r < rows; ++r) {
            int x, y;
            patch_pixel(xb >> 2, band * rows + r, xb & 3, x, y);
            if (y >= sP.H) break;
            if (x < sP.W) gather_pixel<NB, FMT, INF_T, STEP_MODE, 128>(sP, x, y, slots + threadIdx.x);
        }
        __syncthreads();  // everyone is done with s_tile, s_frame and sP before they change
    }
}

}  // namespace ssilvb
