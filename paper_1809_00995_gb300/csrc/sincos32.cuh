// sincos32.cuh -- single-precision sine and cosine of a link phase.
//
// Method (Cody & Waite's additive range reduction, written with fused
// multiply-adds): k = nearest integer to t * 2/pi, r = t - k pi/2 with pi/2
// split into three FP32 parts P1 + P2 + P3 (P1 = fl(pi/2), P2 = fl(pi/2 - P1),
// P3 = fl(pi/2 - P1 - P2); |pi/2 - P1 - P2 - P3| < 1.1e-23), so r is exact to
// an ulp for the arguments of this code.  On |r| <= pi/4 the Taylor
// polynomials of sin (through r^9) and cos (through r^10) leave truncation
// errors below |r|^11/11! < 2e-9 and |r|^12/12! < 2e-10; the quadrant k mod 4
// then selects and signs the two.  Arguments with |t| >= 2^17 (never reached by
// a link phase of this code in practice) go to the library sincosf.
#pragma once

namespace ah {

// sin r, cos r on |r| <= pi/4 (the polynomials above)
__device__ __forceinline__ void sincos_poly(float r, float *s, float *c)
{
    const float r2 = r * r;
    // sin r = r + r^3 (-1/3! + r^2 (1/5! + r^2 (-1/7! + r^2 / 9!)))
    float ps = fmaf(r2, 2.755731884e-06f, -1.984127011e-04f);
    ps = fmaf(r2, ps, 8.333333768e-03f);
    ps = fmaf(r2, ps, -1.666666716e-01f);
    *s = fmaf(r * r2, ps, r);
    // cos r = 1 + r^2 (-1/2! + r^2 (1/4! + r^2 (-1/6! + r^2 (1/8! - r^2 / 10!))))
    float pc = fmaf(r2, -2.755731998e-07f, 2.480158764e-05f);
    pc = fmaf(r2, pc, -1.388888923e-03f);
    pc = fmaf(r2, pc, 4.166666791e-02f);
    pc = fmaf(r2, pc, -0.5f);
    *c = fmaf(r2, pc, 1.0f);
}

__device__ __forceinline__ void sincos_link(float t, float *s, float *c)
{
    if (!(fabsf(t) < 131072.0f)) {
        sincosf(t, s, c);
        return;
    }
    const float kf = rintf(t * 0x1.45f306p-1f);          // 2/pi
    float r = fmaf(-kf, 0x1.921fb6p+0f, t);               // P1
    r = fmaf(-kf, -0x1.777a5cp-25f, r);                   // P2
    r = fmaf(-kf, -0x1.ee59dap-50f, r);                   // P3
    float sr, cr;
    sincos_poly(r, &sr, &cr);
    const int q = (int)kf;
    const float a = (q & 1) ? cr : sr;        // |sin t|
    const float b = (q & 1) ? sr : cr;        // |cos t|
    *s = (q & 2) ? -a : a;
    *c = ((q + 1) & 2) ? -b : b;
}

// The three links of a site.  When every active lane of the warp has all three
// phases in [-0.78, 0.78] the reduction is the identity (k = 0, r = t exactly)
// and the quadrant step selects (sin r, cos r), so the polynomials alone give
// the same bits as sincos_link; the test is one warp vote.
__device__ __forceinline__ void sincos_link3(const float t[3], float s[3], float c[3])
{
    const float m = fmaxf(fabsf(t[0]), fmaxf(fabsf(t[1]), fabsf(t[2])));
    if (__all_sync(__activemask(), m <= 0.78f)) {        // 0.78 * 2/pi < 1/2: k = 0
#pragma unroll
        for (int d = 0; d < 3; ++d) sincos_poly(t[d], &s[d], &c[d]);
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) sincos_link(t[d], &s[d], &c[d]);
    }
}

// sin r, cos r on |r| <= 2^-6 by the first two Taylor terms of each, r - r^3/3!
// and 1 - r^2/2!: the next terms are below |r| r^4/5! <= 2^-24 |r| / 120 and
// r^4/4! <= 2^-24 / 24, a few hundredths of an ulp of the results, so both
// stay within an ulp of the longer polynomials (and of sin, cos).
__device__ __forceinline__ void sincos_small(float r, float *s, float *c)
{
    const float r2 = r * r;
    *s = fmaf(r * r2, -1.666666716e-01f, r);
    *c = fmaf(r2, -0.5f, 1.0f);
}

// sincos_link3 for kernels specialised to weak gauge fields: one warp
// reduction of the largest |phase| picks the two-term forms when every phase
// of the active lanes is in [-2^-6, 2^-6], else the choice of sincos_link3.
// (In kernels for general states the extra tier costs more than it saves.)
__device__ __forceinline__ void sincos_link3_weak(const float t[3], float s[3], float c[3])
{
    const float m = fmaxf(fabsf(t[0]), fmaxf(fabsf(t[1]), fabsf(t[2])));
    const unsigned mb = __reduce_max_sync(__activemask(), __float_as_uint(m));   // m >= 0: bits order as values
    if (mb <= __float_as_uint(0x1p-6f)) {
#pragma unroll
        for (int d = 0; d < 3; ++d) sincos_small(t[d], &s[d], &c[d]);
    } else if (mb <= __float_as_uint(0.78f)) {
#pragma unroll
        for (int d = 0; d < 3; ++d) sincos_poly(t[d], &s[d], &c[d]);
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) sincos_link(t[d], &s[d], &c[d]);
    }
}

__device__ __forceinline__ void sincos_link(double t, double *s, double *c) { sincos(t, s, c); }
__device__ __forceinline__ void sincos_link3(const double t[3], double s[3], double c[3])
{
#pragma unroll
    for (int d = 0; d < 3; ++d) sincos(t[d], &s[d], &c[d]);
}

}  // namespace ah
