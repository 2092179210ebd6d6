// k_plain.cu -- the "plain" leapfrog step: the paper's three-kernel structure
// (Sec. 3: stepA = Pi kick, Eq. up_pi; stepB = E kick, Eq. up_E; stepC =
// drifts, Eqs. up_phi and up_A), one thread per site, every neighbour read from
// global memory, every link exponential and plaquette sine evaluated where it
// is used.  It updates phi and theta in place (the kicks finish before the
// drift starts) and moves 9 + 11 + 15 = 35 reals per site.  It is the
// reference point for the fused kernel and, in FP64, the baseline path.
#include "ah_internal.cuh"

namespace ah {
namespace {

constexpr int BX = 32, BY = 8;

__device__ __forceinline__ void sc(float t, float *s, float *c) { sincosf(t, s, c); }
__device__ __forceinline__ void sc(double t, double *s, double *c) { sincos(t, s, c); }
__device__ __forceinline__ float sn(float t) { return sinf(t); }
__device__ __forceinline__ double sn(double t) { return sin(t); }

struct Nb {                    // periodic neighbour coordinates of one site
    int x, y, z, xp, xm, yp, ym, zp, zm;
};

__device__ __forceinline__ Nb neighbours(int x, int y, int z, int N)
{
    Nb n;
    n.x = x; n.y = y; n.z = z;
    n.xp = x + 1 == N ? 0 : x + 1; n.xm = x == 0 ? N - 1 : x - 1;
    n.yp = y + 1 == N ? 0 : y + 1; n.ym = y == 0 ? N - 1 : y - 1;
    n.zp = z + 1 == N ? 0 : z + 1; n.zm = z == 0 ? N - 1 : z - 1;
    return n;
}

__device__ __forceinline__ long long sid(int x, int y, int z, int N)
{
    return x + (long long)N * (y + (long long)N * z);
}

// stepA: Pi^{n+1/2} from phi^n, theta^n, Pi^{n-1/2} (Eq. up_pi).
template <typename real>
__global__ void __launch_bounds__(BX * BY) k_kick_pi(View<real> v, int N, KickCoef<real> c)
{
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
    if (x >= N || y >= N) return;
    const Nb n = neighbours(x, y, z, N);
    const long long s0 = sid(x, y, z, N);
    const long long sp[3] = { sid(n.xp, y, z, N), sid(x, n.yp, z, N), sid(x, y, n.zp, N) };
    const long long sm[3] = { sid(n.xm, y, z, N), sid(x, n.ym, z, N), sid(x, y, n.zm, N) };
    const real *th[3] = { v.th1, v.th2, v.th3 };
    const real ar = v.phr[s0], ai = v.phi[s0];
    real lr = 0, li = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        real s, cth;
        sc(th[d][s0], &s, &cth);                 // U_d^x
        const real br = v.phr[sp[d]], bi = v.phi[sp[d]];
        lr += cth * br - s * bi;
        li += cth * bi + s * br;
        sc(th[d][sm[d]], &s, &cth);              // conj(U_d^{x-d})
        const real mr = v.phr[sm[d]], mi = v.phi[sm[d]];
        lr += cth * mr + s * mi;
        li += cth * mi - s * mr;
    }
    lr -= real(6) * ar;
    li -= real(6) * ai;
    const real pot = c.c_pot * (ar * ar + ai * ai - c.sigma2);
    v.pir[s0] = c.c_damp * v.pir[s0] - pot * ar + c.c_lap * lr;
    v.pii[s0] = c.c_damp * v.pii[s0] - pot * ai + c.c_lap * li;
}

// stepB: E^{n+1/2} from phi^n, theta^n, E^{n-1/2} (Eq. up_E).
template <typename real>
__global__ void __launch_bounds__(BX * BY) k_kick_e(View<real> v, int N, KickCoef<real> c)
{
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
    if (x >= N || y >= N) return;
    const Nb n = neighbours(x, y, z, N);
    const int cx[3] = { n.x, n.y, n.z };
    const int cp[3] = { n.xp, n.yp, n.zp };
    const int cm[3] = { n.xm, n.ym, n.zm };
    const real *th[3] = { v.th1, v.th2, v.th3 };
    real *el[3] = { v.e1, v.e2, v.e3 };
    const long long s0 = sid(x, y, z, N);
    const real ar = v.phr[s0], ai = v.phi[s0];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        int q[3] = { cx[0], cx[1], cx[2] };
        q[i] = cp[i];
        const long long si = sid(q[0], q[1], q[2], N);
        real s, cth;
        sc(th[i][s0], &s, &cth);
        // conj(U_i) phi^x, then Im[conj(phi^{x+i}) (...)]
        const real wr = cth * ar + s * ai, wi = cth * ai - s * ar;
        const real br = v.phr[si], bi = v.phi[si];
        const real cur = br * wi - bi * wr;
        real curl = 0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (j == i) continue;
            int qj[3] = { cx[0], cx[1], cx[2] };  qj[j] = cp[j];       // x + j
            int qm[3] = { cx[0], cx[1], cx[2] };  qm[j] = cm[j];       // x - j
            int qim[3] = { qm[0], qm[1], qm[2] }; qim[i] = cp[i];      // x + i - j
            const long long sj = sid(qj[0], qj[1], qj[2], N);
            const long long smj = sid(qm[0], qm[1], qm[2], N);
            const long long simj = sid(qim[0], qim[1], qim[2], N);
            // Xi_ij^x = th_i^x + th_j^{x+i} - th_i^{x+j} - th_j^x
            const real xi0 = th[i][s0] + th[j][si] - th[i][sj] - th[j][s0];
            // Xi_ij^{x-j} = th_i^{x-j} + th_j^{x+i-j} - th_i^x - th_j^{x-j}
            const real xim = th[i][smj] + th[j][simj] - th[i][s0] - th[j][smj];
            curl += sn(xi0) - sn(xim);
        }
        el[i][s0] = c.c_edamp * el[i][s0] + c.c_cur * cur - c.c_curl * curl;
    }
}

// stepC: phi += dt Pi^{n+1/2}, theta += dt E^{n+1/2} (Eqs. up_phi, up_A),
// theta reduced to [-pi, pi] when wrap is set.
template <typename real>
__global__ void __launch_bounds__(256) k_drift(View<real> v, long long nsites, real dt, int wrap)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < nsites; s += stride) {
        v.ophr[s] = v.phr[s] + dt * v.pir[s];
        v.ophi[s] = v.phi[s] + dt * v.pii[s];
        real t1 = v.th1[s] + dt * v.e1[s], t2 = v.th2[s] + dt * v.e2[s], t3 = v.th3[s] + dt * v.e3[s];
        if (wrap) { t1 = wrap_phase(t1); t2 = wrap_phase(t2); t3 = wrap_phase(t3); }
        v.oth1[s] = t1;
        v.oth2[s] = t2;
        v.oth3[s] = t3;
    }
}

}  // namespace

template <typename real>
cudaError_t launch_plain_step(const View<real> &v, int N, const KickCoef<real> &c, cudaStream_t st)
{
    const dim3 blk(BX, BY), grd((N + BX - 1) / BX, (N + BY - 1) / BY, N);
    k_kick_pi<real><<<grd, blk, 0, st>>>(v, N, c);
    k_kick_e<real><<<grd, blk, 0, st>>>(v, N, c);
    const long long ns = (long long)N * N * N;
    long long g = (ns + 255) / 256;
    if (g > 152LL * 32) g = 152LL * 32;
    k_drift<real><<<(int)g, 256, 0, st>>>(v, ns, c.dt, c.wrap);
    return cudaGetLastError();
}

template cudaError_t launch_plain_step<float>(const View<float> &, int, const KickCoef<float> &, cudaStream_t);
template cudaError_t launch_plain_step<double>(const View<double> &, int, const KickCoef<double> &, cudaStream_t);

}  // namespace ah
