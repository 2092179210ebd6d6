// k_init.cu -- random-phase initial state and host<->device field transfers.
//
// Initial state (Sec. 2 of arXiv:1809.00995): |phi| = sigma with a random
// phase at every site, Pi = theta = E = 0 (this satisfies the discrete Gauss
// law).  The phase is alpha = 2 pi u with u drawn by Philox-4x32-10 (Salmon
// et al., SC'11) keyed by the seed, counter = (0, 0, site index lo, hi): the
// first two output words give a 53-bit integer, word 0 above the top 21 bits of
// word 1.  phi is formed in FP64 and rounded once to the state precision, so
// the FP32 and FP64 states start from the same snapshot.
#include "ah_internal.cuh"

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

template <typename real>
__global__ void k_init_phase(real *__restrict__ phr, real *__restrict__ phi, long long nsites,
                             uint64_t seed, double sigma)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < nsites; s += stride) {
        uint32_t c[4] = { 0u, 0u, (uint32_t)s, (uint32_t)((unsigned long long)s >> 32) };
        philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        const unsigned long long m = ((unsigned long long)c[0] << 21) ^ (unsigned long long)(c[1] >> 11);
        const double u = (double)m * (1.0 / 9007199254740992.0);
        const double alpha = 2.0 * 3.141592653589793 * u;
        double sn, cs;
        sincos(alpha, &sn, &cs);
        phr[s] = (real)(sigma * cs);
        phi[s] = (real)(sigma * sn);
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
