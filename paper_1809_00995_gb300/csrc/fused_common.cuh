// fused_common.cuh -- pieces shared by the z-marching step kernels
// (k_fused.cu: one step per pass; k_fused2.cu: two steps per pass): complex
// arithmetic on link exponentials U = e^{i theta}, plaquette products, the
// tile geometry with its one-site halo ring, row loads/stores, and the
// wave-quantisation model that picks the number of z chunks.
#pragma once
#include "ah_internal.cuh"

namespace ah {

// Number of z chunks for `tiles` XY tiles of an N-plane lattice when `slots`
// CTAs are resident at once: the grid runs in waves of `slots` CTAs, each CTA
// marching its chunk plus `extra` planes of prologue and look-ahead, so
// minimise ceil(tiles n / slots) (ceil(N / n) + extra) over n with chunks of
// at least min_chunk planes.
int choose_chunks(int N, long long tiles, int slots, int min_chunk, int extra = 2);
// Streaming multiprocessors of the current device (cached per device).
int device_sm_count();

namespace {

template <typename real>
struct cpx { real r, i; };

template <typename real>
__device__ __forceinline__ cpx<real> mul(cpx<real> a, cpx<real> b)
{
    return { a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r };
}
// Im(a b conj(c) conj(d)) = Im((a b) conj(c d))
template <typename real>
__device__ __forceinline__ real plaq(cpx<real> a, cpx<real> b, cpx<real> c, cpx<real> d)
{
    const cpx<real> ab = mul(a, b), cd = mul(c, d);
    return ab.i * cd.r - ab.r * cd.i;
}
// (a b) conj(c d) = e^{i Xi}: sine in .i, cosine in .r
template <typename real>
__device__ __forceinline__ cpx<real> plaq2(cpx<real> a, cpx<real> b, cpx<real> c, cpx<real> d)
{
    const cpx<real> ab = mul(a, b), cd = mul(c, d);
    return { ab.r * cd.r + ab.i * cd.i, ab.i * cd.r - ab.r * cd.i };
}
__device__ __forceinline__ int wrapm(int a, int N)
{
    a %= N;
    return a < 0 ? a + N : a;
}

template <typename real, int TY, int RX>
struct Geo {
    static constexpr int TX = 32 * RX, NT = 256, RY = TY / 8, NS = RX * RY;
    static constexpr int EX = TX + 2, EY = TY + 2, NE = EX * EY;
    static constexpr int NHALO = 2 * EX + 2 * TY;
    static constexpr int PX = TX + 1, PY = TY + 1, NP = PX * PY;
    static constexpr int NPHALO = PX + TY;
    static constexpr size_t smem = sizeof(cpx<real>) * (2 * 3 * NE + 2 * NE) + sizeof(real) * 3 * NP;
    // MODE_DIAG: the three scaled edge products of each site of plane z
    // (tile, right column, top row) after the step's arrays
    static constexpr size_t diag_off = (smem + 15) / 16 * 16;
    static constexpr size_t smem_diag = diag_off + sizeof(cpx<real>) * 3 * NE;
    static_assert(TY % 8 == 0 && NHALO <= NT && NPHALO <= NT && TX + TY <= NT, "tile shape");
};

// RX consecutive reals of one row (vector access when RX = 2; the pair never
// straddles the end of a row because N is even for these shapes).
template <typename real, int RX> struct Row;
template <typename real> struct Row<real, 1> {
    static __device__ __forceinline__ void ld(const real *p, real *o) { o[0] = *p; }
    static __device__ __forceinline__ void st(real *p, const real *i) { *p = i[0]; }
};
template <> struct Row<float, 2> {
    static __device__ __forceinline__ void ld(const float *p, float *o)
    { const float2 t = *reinterpret_cast<const float2 *>(p); o[0] = t.x; o[1] = t.y; }
    static __device__ __forceinline__ void st(float *p, const float *i)
    { *reinterpret_cast<float2 *>(p) = make_float2(i[0], i[1]); }
};
template <> struct Row<double, 2> {
    static __device__ __forceinline__ void ld(const double *p, double *o)
    { const double2 t = *reinterpret_cast<const double2 *>(p); o[0] = t.x; o[1] = t.y; }
    static __device__ __forceinline__ void st(double *p, const double *i)
    { *reinterpret_cast<double2 *>(p) = make_double2(i[0], i[1]); }
};

template <int V> struct IC { static constexpr int value = V; };

}  // namespace
}  // namespace ah
