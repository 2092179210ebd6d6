// k_init.cu -- random-phase initial state and host<->device field transfers.
//
// Initial state (Sec. 2 of arXiv:1809.00995): |phi| = sigma with a random
// phase at every site, Pi = theta = E = 0 (this satisfies the discrete Gauss
// law).  The phase is alpha = 2 pi u with u drawn by Philox-4x32-10 (Salmon
// et al., SC'11) keyed by the seed, counter = (0, 0, site index lo, hi): the
// first two output words give a 53-bit integer, word 0 above the top 21 bits of
// word 1.  For an FP64 state phi = sigma e^{i alpha} is evaluated in FP64; for
// an FP32 state in double-float arithmetic (FP32 pairs, within 1e-14 of the
// exact value) and rounded once to FP32, which gives the FP32 rounding of the
// FP64 formula except at a few sites in 10^6 (one ulp), from FP32 instructions
// only (GB300's FP64 rate is a small fraction of its FP32 rate).
#include "ah_internal.cuh"
#include "diag_common.cuh"

namespace ah {
namespace {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Float pairs (hi, lo) of pi/2 and 1/n!: hi the nearest float to the value,
// lo the nearest float to the remainder (from the decimal expansion of pi and
// the exact rationals).
__device__ __forceinline__ DF dfc(float h, float l) { return { h, l }; }
__device__ __forceinline__ DF half_pi() { return dfc(0x1.921fb6p+0f, -0x1.777a5cp-25f); }

// sin and cos of 2 pi u for u = m 2^-53 (m < 2^53) as float pairs, within
// 1e-14: the quadrant j is the nearest integer to 4u and the reduced angle
// beta = (pi/2)(4u - j), |beta| <= pi/4, comes from the exact integer
// remainder m - j 2^51; sin beta = beta S(beta^2) and cos beta = C(beta^2) are
// their Taylor series through beta^15 and beta^16 (Horner in x = beta^2, the
// terms of the highest orders, below 2^-24 of the sum, in plain FP32), then
// the quadrant's swap and signs.
__device__ __forceinline__ void sincos_2pi_pair(unsigned long long m, DF &sn, DF &cs)
{
    const long long j = (long long)((m + (1ULL << 50)) >> 51);
    const long long rem = (long long)m - (j << 51);              // |rem| <= 2^50
    const float th = (float)rem;
    const float tl = (float)(rem - (long long)th);                // drops at most 2 low bits
    const DF t = { th * 0x1p-51f, tl * 0x1p-51f };
    const DF b = df_mul(half_pi(), t);
    const DF x = df_mul(b, b);
    // S(x) = 1 - x/3! + x^2/5! - ... + x^6/13! - x^7/15!
    float p = fmaf(-0x1.ae7f3ep-41f, x.h, 0x1.612462p-33f);
    p = fmaf(p, x.h, -0x1.ae6456p-26f);
    DF P = { p, 0.f };
    P = df_add(df_mul(P, x), dfc(0x1.71de3ap-19f, 0x1.55b1ccp-45f));
    P = df_add(df_mul(P, x), dfc(-0x1.a01a02p-13f, 0x1.7f97fap-39f));
    P = df_add(df_mul(P, x), dfc(0x1.111112p-7f, -0x1.dddddep-32f));
    P = df_add(df_mul(P, x), dfc(-0x1.555556p-3f, 0x1.555556p-28f));
    P = df_add(df_mul(P, x), dfc(1.f, 0.f));
    const DF s = df_mul(b, P);
    // C(x) = 1 - x/2! + x^2/4! - ... - x^7/14! + x^8/16!
    float q = fmaf(0x1.ae7f3ep-45f, x.h, -0x1.93974ap-37f);
    q = fmaf(q, x.h, 0x1.1eed8ep-29f);
    q = fmaf(q, x.h, -0x1.27e4fcp-22f);
    DF Q = { q, 0.f };
    Q = df_add(df_mul(Q, x), dfc(0x1.a01a02p-16f, -0x1.7f97fap-42f));
    Q = df_add(df_mul(Q, x), dfc(-0x1.6c16c2p-10f, 0x1.27d27ep-35f));
    Q = df_add(df_mul(Q, x), dfc(0x1.555556p-5f, -0x1.555556p-30f));
    Q = df_add(df_mul(Q, x), dfc(-0.5f, 0.f));
    const DF c = df_add(df_mul(Q, x), dfc(1.f, 0.f));
    const DF ms = { -s.h, -s.l }, mc = { -c.h, -c.l };
    switch (j & 3) {
    case 0: sn = s; cs = c; break;
    case 1: sn = c; cs = ms; break;
    case 2: sn = ms; cs = mc; break;
    default: sn = mc; cs = s; break;
    }
}

template <typename real>
__global__ void k_init_phase(real *__restrict__ phr, real *__restrict__ phi, long long nsites,
                             uint64_t seed, double sigma)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const DF sig = df_from(sigma);
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < nsites; s += stride) {
        uint32_t c[4] = { 0u, 0u, (uint32_t)s, (uint32_t)((unsigned long long)s >> 32) };
        philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        const unsigned long long m = ((unsigned long long)c[0] << 21) ^ (unsigned long long)(c[1] >> 11);
        if constexpr (sizeof(real) == 4) {
            DF sn, cs;
            sincos_2pi_pair(m, sn, cs);
            const DF re = df_mul(sig, cs), im = df_mul(sig, sn);
            phr[s] = re.h + re.l;
            phi[s] = im.h + im.l;
        } else {
            const double u = (double)m * (1.0 / 9007199254740992.0);
            const double alpha = 2.0 * 3.141592653589793 * u;
            double sn, cs;
            sincos(alpha, &sn, &cs);
            phr[s] = (real)(sigma * cs);
            phi[s] = (real)(sigma * sn);
        }
    }
}

// Gather the window [x0, x0+nx) x [y0, ..) x [z0, ..) (mod N) into out as FP64,
// 10 components each nz*ny*nx, x fastest.
template <typename real>
__global__ void k_gather(Fields<real> F, int cur, int N, Box b, double *__restrict__ out)
{
    const long long nw = (long long)b.nx * b.ny * b.nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += stride) {
        const int i = (int)(w % b.nx);
        const int j = (int)((w / b.nx) % b.ny);
        const int k = (int)(w / ((long long)b.nx * b.ny));
        const int x = (b.x0 + i) % N, y = (b.y0 + j) % N, z = (b.z0 + k) % N;
        const long long s = x + (long long)N * (y + (long long)N * z);
        const real *src[10] = { F.phr[cur], F.phi[cur], F.pir, F.pii,
                                F.th[cur][0], F.th[cur][1], F.th[cur][2],
                                F.el[0], F.el[1], F.el[2] };
#pragma unroll
        for (int c = 0; c < 10; ++c) out[c * nw + w] = (double)src[c][s];
    }
}

template <typename real>
__global__ void k_scatter(Fields<real> F, int cur, long long nsites, const double *__restrict__ in)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < nsites; s += stride) {
        real *dst[10] = { F.phr[cur], F.phi[cur], F.pir, F.pii,
                          F.th[cur][0], F.th[cur][1], F.th[cur][2],
                          F.el[0], F.el[1], F.el[2] };
#pragma unroll
        for (int c = 0; c < 10; ++c) dst[c][s] = (real)in[c * nsites + s];
    }
}

int grid_for(long long n, int threads)
{
    long long g = (n + threads - 1) / threads;
    if (g > 152LL * 64) g = 152LL * 64;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

template <typename real>
cudaError_t launch_init_phase(real *phr, real *phi, int N, uint64_t seed, double sigma,
                              cudaStream_t st)
{
    const long long n = (long long)N * N * N;
    k_init_phase<real><<<grid_for(n, 256), 256, 0, st>>>(phr, phi, n, seed, sigma);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_gather_window(const Fields<real> &F, int cur, int N, Box b, double *out,
                                 cudaStream_t st)
{
    const long long n = (long long)b.nx * b.ny * b.nz;
    k_gather<real><<<grid_for(n, 256), 256, 0, st>>>(F, cur, N, b, out);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_scatter_all(const Fields<real> &F, int cur, int N, const double *in,
                               cudaStream_t st)
{
    const long long n = (long long)N * N * N;
    k_scatter<real><<<grid_for(n, 256), 256, 0, st>>>(F, cur, n, in);
    return cudaGetLastError();
}

template cudaError_t launch_init_phase<float>(float *, float *, int, uint64_t, double, cudaStream_t);
template cudaError_t launch_init_phase<double>(double *, double *, int, uint64_t, double, cudaStream_t);
template cudaError_t launch_gather_window<float>(const Fields<float> &, int, int, Box, double *, cudaStream_t);
template cudaError_t launch_gather_window<double>(const Fields<double> &, int, int, Box, double *, cudaStream_t);
template cudaError_t launch_scatter_all<float>(const Fields<float> &, int, int, const double *, cudaStream_t);
template cudaError_t launch_scatter_all<double>(const Fields<double> &, int, int, const double *, cudaStream_t);

}  // namespace ah
