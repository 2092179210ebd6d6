// diag_common.cuh -- device helpers shared by the diagnostics kernels
// (k_diag.cu) and the fused step's diagnostics mode (k_fused.cu).
#pragma once

#include <climits>

#include "ah_internal.cuh"

namespace ah {

template <typename T>
struct C2 { T r, i; };
template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) { return { a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r }; }
template <typename T>
__device__ __forceinline__ C2<T> conj(C2<T> a) { return { a.r, -a.i }; }
// Relative margin to the negative real axis below which a winding is decided
// by the FP64 path instead of the FP32 carries.  An FP32 edge product
// conj(phi^a) U phi^b (U from sincos_link, error < 1e-7) has a relative error below
// 1e-6, the product of four of them below 3e-6; 2^-15 (3.1e-5) keeps a factor
// of ten between the two.  For FP64 data only values exactly on the axis (or
// zero) are sent there.
template <typename T> struct Margin;
template <> struct Margin<float> { static constexpr float v = 1.0f / 32768.0f; static constexpr float tiny = 1e-36f; };
template <> struct Margin<double> { static constexpr double v = 0.0; static constexpr double tiny = 1e-300; };

template <typename T>
__device__ __forceinline__ bool near_cut(C2<T> z)
{
    return z.r < T(0) && fabs(z.i) <= Margin<T>::v * fabs(z.r);
}
// z times the power of two 2^-floor(log2 max(|Re z|, |Im z|)): same Arg, exact,
// max(|Re|, |Im|) in [1, 2), so the chained products can neither underflow
// where |phi| is small nor overflow.  Returns false (z unscaled) when
// max(|Re z|, |Im z|) is not above Margin::tiny or is within a factor 16 of
// the largest finite value; such plaquettes go to the FP64 path.
__device__ __forceinline__ bool unit_scale(C2<float> &z)
{
    const float m = fmaxf(fabsf(z.r), fabsf(z.i));
    const int e = __float_as_int(m) >> 23;                  // biased exponent (m >= 0)
    if (!(m > Margin<float>::tiny) || e > 250) return false;
    const float s = __int_as_float((254 - e) << 23);        // 2^(127 - e)
    z.r *= s;
    z.i *= s;
    return true;
}
__device__ __forceinline__ bool unit_scale(C2<double> &z)
{
    const double m = fmax(fabs(z.r), fabs(z.i));
    const long long e = __double_as_longlong(m) >> 52;
    if (!(m > Margin<double>::tiny) || e > 2042) return false;
    const double s = __longlong_as_double((2046LL - e) << 52); // 2^(1023 - e)
    z.r *= s;
    z.i *= s;
    return true;
}
// unit_scale, or both parts NaN when z cannot be scaled (a plaquette with such
// an edge is then left to the FP64 path by winding_scaled)
template <typename T>
__device__ __forceinline__ void unit_scale_or_nan(C2<T> &z)
{
    if (!unit_scale(z)) z.r = z.i = T(NAN);
}
// carry c of Arg u + Arg v = Arg(uv) + 2 pi c, Arg in (-pi, pi]
template <typename T>
__device__ __forceinline__ int carry(C2<T> u, C2<T> v, C2<T> uv)
{
    const bool su = u.i >= T(0), sv = v.i >= T(0);
    if (su && sv) return uv.i < T(0) ? 1 : 0;
    if (!su && !sv) return uv.i >= T(0) ? -1 : 0;
    return 0;
}
// Winding of a plaquette from its four edge products, each already passed
// through unit_scale (orientation as Eq. 9), or INT_MIN when it must be
// decided by the FP64 path.
template <typename T>
__device__ __forceinline__ int winding_scaled(C2<T> z1, C2<T> z2, C2<T> z3, C2<T> z4)
{
    const C2<T> w3 = conj(z3), w4 = conj(z4);
    const C2<T> q2 = cmul(z1, z2), q3 = cmul(q2, w3), q4 = cmul(q3, w4);
    if (!(q4.r == q4.r)) return INT_MIN;            // an unscalable (NaN) edge
    if (near_cut(z1) | near_cut(z2) | near_cut(w3) | near_cut(w4) | near_cut(q4)) return INT_MIN;
    return carry(z1, z2, q2) + carry(q2, w3, q3) + carry(q3, w4, q4);
}
// The same from unscaled edge products.
template <typename T>
__device__ __forceinline__ int winding_carry(C2<T> z1, C2<T> z2, C2<T> z3, C2<T> z4)
{
    const bool ok = unit_scale(z1) & unit_scale(z2) & unit_scale(z3) & unit_scale(z4);
    return ok ? winding_scaled(z1, z2, z3, z4) : INT_MIN;
}

// 1 - cos Xi from e^{i Xi} = (c, s) without cancellation (in FP32 the
// quotient by the fast approximate division, a few ulp)
template <typename T>
__device__ __forceinline__ T one_minus_cos(T c, T s)
{
    if constexpr (sizeof(T) == 4)
        return c > 0.f ? __fdividef(s * s, 1.f + c) : 1.f - c;
    else
        return c > 0.0 ? s * s / (1.0 + c) : 1.0 - c;
}

// Double-float arithmetic (a value as the unevaluated sum hi + lo of two
// floats) from error-free transformations: Knuth's TwoSum, Dekker's
// Fast2Sum and the FMA-based TwoProduct.  The roundings are explicit
// (__fadd_rn, __fmul_rn are never contracted into a multiply-add), so every
// kernel that uses them gets the same bits from the same inputs.
struct DF { float h, l; };
__device__ __forceinline__ DF two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return { s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)) };
}
__device__ __forceinline__ DF fast_two_sum(float a, float b)      // |a| >= |b| or a == 0
{
    const float s = __fadd_rn(a, b);
    return { s, __fsub_rn(b, __fsub_rn(s, a)) };
}
__device__ __forceinline__ DF two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return { p, fmaf(a, b, -p) };
}
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const DF s = two_sum(a.h, b.h);
    return two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    const DF p = two_prod(a.h, b.h);
    return fast_two_sum(p.h, __fadd_rn(p.l, fmaf(a.h, b.l, __fmul_rn(a.l, b.h))));
}
__host__ __device__ __forceinline__ DF df_from(double x)
{
    const float h = (float)x;
    return { h, (float)(x - (double)h) };
}

// Compensated (Kahan) accumulator in the state precision (plain sum for FP64
// data); explicit roundings, as for the double-float arithmetic.
template <typename T>
struct Acc {
    T s = 0, c = 0;
    __device__ __forceinline__ void add(T v)
    {
        const T y = __fsub_rn(v, c);
        const T t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <>
struct Acc<double> {
    double s = 0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};

// Block-wide reduction into *out (thread 0 writes).
template <int NT>
__device__ __forceinline__ void block_reduce(double acc[kNumSums], double mx[kNumMax], long long ic[kNumInt],
                                             DiagPartial *out)
{
    __shared__ DiagPartial red[NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < kNumSums; ++k) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
#pragma unroll
        for (int k = 0; k < kNumMax; ++k) mx[k] = fmax(mx[k], __shfl_down_sync(0xffffffffu, mx[k], o));
#pragma unroll
        for (int k = 0; k < kNumInt; ++k) ic[k] += __shfl_down_sync(0xffffffffu, ic[k], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kNumSums; ++k) red[warp].sums[k] = acc[k];
#pragma unroll
        for (int k = 0; k < kNumMax; ++k) red[warp].maxv[k] = mx[k];
#pragma unroll
        for (int k = 0; k < kNumInt; ++k) red[warp].ints[k] = ic[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        DiagPartial r = red[0];
        for (int w = 1; w < NT / 32; ++w) {
            for (int k = 0; k < kNumSums; ++k) r.sums[k] += red[w].sums[k];
            for (int k = 0; k < kNumMax; ++k) r.maxv[k] = fmax(r.maxv[k], red[w].maxv[k]);
            for (int k = 0; k < kNumInt; ++k) r.ints[k] += red[w].ints[k];
        }
        *out = r;
    }
}

}  // namespace ah
