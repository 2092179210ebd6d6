// k_diag.cu -- network diagnostics of one state (Sec. 2 of arXiv:1809.00995).
//
// Per site, in FP64 whatever the state precision (values are converted on
// load), at tau_n with the state (phi^n, theta^n, Pi^{n-1/2}, E^{n-1/2}):
//   K = |Pi|^2, G2 = dx^-2 sum_i |U_i phi^{x+i} - phi^x|^2 (U = e^{i theta}),
//   V = a^2 lambda/4 (|phi|^2 - sigma^2)^2, E_el = sum E_i^2 / (2 e^2 a^2 dx^2),
//   B = sum_{i<j} (1 - cos Xi_ij) / (e^2 a^2 dx^4)          (Eqs. 2, 3),
//   L = K - G2 - V + E_el - B, rho = K + G2 + V + E_el + B,
//   p = K - G2/3 - V + (E_el + B)/3                          (Eqs. defR, defEoS),
//   Gauss residual G = e_-^-2 div E + 2 dx^2 a_-^2 Im(conj(phi) Pi),
//   winding W_ij through the plaquettes (12), (13), (23) based at the site
//   (Eq. 9): with edge products z_e = conj(phi^a) U_e phi^b,
//   2 pi W = Arg z1 + Arg z2 - Arg z3 - Arg z4 - Arg(z1 z2 conj(z3) conj(z4)),
//   Arg in (-pi, pi] (the -pi branch value is mapped to +pi).
// Each block accumulates its sites in a fixed order, reduces across the
// block with warp shuffles, and writes one partial; a single block then adds
// the partials in index order, so the result depends only on the launch
// shape, never on scheduling.
#include "ah_internal.cuh"

namespace ah {
namespace {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr double kPi = 3.141592653589793;

struct C2 { double r, i; };
__device__ __forceinline__ C2 cmul(C2 a, C2 b) { return { a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r }; }
__device__ __forceinline__ C2 conj(C2 a) { return { a.r, -a.i }; }
__device__ __forceinline__ C2 expi(double t) { double s, c; sincos(t, &s, &c); return { c, s }; }
__device__ __forceinline__ double arg_pi(C2 z)
{
    const double a = atan2(z.i, z.r);
    return a == -kPi ? kPi : a;
}

template <typename real>
struct Site {
    const View<real> &v;
    int N;
    __device__ long long id(int x, int y, int z) const
    {
        x = x >= N ? x - N : (x < 0 ? x + N : x);
        y = y >= N ? y - N : (y < 0 ? y + N : y);
        z = z >= N ? z - N : (z < 0 ? z + N : z);
        return x + (long long)N * (y + (long long)N * z);
    }
    __device__ C2 phi(long long s) const { return { (double)v.phr[s], (double)v.phi[s] }; }
    __device__ double th(int d, long long s) const
    {
        return (double)(d == 0 ? v.th1[s] : (d == 1 ? v.th2[s] : v.th3[s]));
    }
    __device__ double el(int d, long long s) const
    {
        return (double)(d == 0 ? v.e1[s] : (d == 1 ? v.e2[s] : v.e3[s]));
    }
};

template <typename real>
__device__ void diag_site(const Site<real> &S, int x, int y, int z, const DiagCoef &c,
                          double acc[kNumSums], double mx[kNumMax], long long ic[kNumInt])
{
    const int U[3][3] = { { 1, 0, 0 }, { 0, 1, 0 }, { 0, 0, 1 } };
    const long long s0 = S.id(x, y, z);
    const C2 p0 = S.phi(s0);
    const C2 pi = { (double)S.v.pir[s0], (double)S.v.pii[s0] };
    long long sp[3];
    C2 pp[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        sp[d] = S.id(x + U[d][0], y + U[d][1], z + U[d][2]);
        pp[d] = S.phi(sp[d]);
    }
    const double K = pi.r * pi.r + pi.i * pi.i;
    double G2 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const C2 up = cmul(expi(S.th(d, s0)), pp[d]);
        const double dr = up.r - p0.r, di = up.i - p0.i;
        G2 += dr * dr + di * di;
    }
    G2 *= c.inv_dx2;
    const double m2 = p0.r * p0.r + p0.i * p0.i - c.sigma2;
    const double V = c.v_coef * m2 * m2;
    double esq = 0.0, div = 0.0, tmax = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double e = S.el(d, s0);
        esq += e * e;
        div += e - S.el(d, S.id(x - U[d][0], y - U[d][1], z - U[d][2]));
        tmax = fmax(tmax, fabs(S.th(d, s0)));
    }
    const double Eel = c.eel_coef * esq;
    double bsum = 0.0;
    int q = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = i + 1; j < 3; ++j, ++q) {
            const long long si = sp[i], sj = sp[j];
            const long long sij = S.id(x + U[i][0] + U[j][0], y + U[i][1] + U[j][1], z + U[i][2] + U[j][2]);
            const double ti0 = S.th(i, s0), tj0 = S.th(j, s0), tji = S.th(j, si), tij = S.th(i, sj);
            bsum += 1.0 - cos(ti0 + tji - tij - tj0);
            const C2 pij = S.phi(sij);
            const C2 z1 = cmul(cmul(conj(p0), expi(ti0)), pp[i]);
            const C2 z2 = cmul(cmul(conj(pp[i]), expi(tji)), pij);
            const C2 z3 = cmul(cmul(conj(pp[j]), expi(tij)), pij);
            const C2 z4 = cmul(cmul(conj(p0), expi(tj0)), pp[j]);
            const C2 pr = cmul(cmul(cmul(z1, z2), conj(z3)), conj(z4));
            const double tot = arg_pi(z1) + arg_pi(z2) - arg_pi(z3) - arg_pi(z4) - arg_pi(pr);
            const long long w = llrint(tot / (2.0 * kPi));
            ic[q] += w < 0 ? -w : w;
            ic[3 + q] += w;
            ic[6] += w != 0;
        }
    }
    const double B = c.b_coef * bsum;
    const double L = K - G2 - V + Eel - B;
    const double rho = K + G2 + V + Eel + B;
    const double p = K - G2 / 3.0 - V + (Eel + B) / 3.0;
    const double g1 = c.g_div * div;
    const double g2 = c.g_phi * (p0.r * pi.i - p0.i * pi.r);
    const double G = g1 + g2, gs = fabs(g1) + fabs(g2);
    const double vals[kNumSums] = { L, rho, p, K, G2, V, Eel, B, K * V, G2 * V, K * L, G2 * L,
                                    p * L, rho * L, G * G, gs * gs };
#pragma unroll
    for (int k = 0; k < kNumSums; ++k) acc[k] += vals[k];
    mx[0] = fmax(mx[0], fabs(G));
    mx[1] = fmax(mx[1], tmax);
    ic[7] += !(isfinite(L) && isfinite(rho) && isfinite(p) && isfinite(G));
}

// Block-wide reduction of the thread's values into *out (thread 0 writes).
__device__ void block_reduce(double acc[kNumSums], double mx[kNumMax], long long ic[kNumInt],
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

template <typename real>
__global__ void __launch_bounds__(NT) k_diag(View<real> v, int N, Box b, DiagCoef c,
                                             DiagPartial *partials)
{
    double acc[kNumSums];
    double mx[kNumMax];
    long long ic[kNumInt];
#pragma unroll
    for (int k = 0; k < kNumSums; ++k) acc[k] = 0.0;
#pragma unroll
    for (int k = 0; k < kNumMax; ++k) mx[k] = 0.0;
#pragma unroll
    for (int k = 0; k < kNumInt; ++k) ic[k] = 0;
    const Site<real> S{ v, N };
    const int tx = (b.nx + TX - 1) / TX, ty = (b.ny + TY - 1) / TY;
    const long long ntiles = (long long)tx * ty * b.nz;
    const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int tz = (int)(t / ((long long)tx * ty));
        const int r = (int)(t % ((long long)tx * ty));
        const int i = (r % tx) * TX + lx, j = (r / tx) * TY + ly;
        if (i < b.nx && j < b.ny) {
            int x = b.x0 + i, y = b.y0 + j, z = b.z0 + tz;
            x -= x >= N ? N : 0; y -= y >= N ? N : 0; z -= z >= N ? N : 0;
            diag_site<real>(S, x, y, z, c, acc, mx, ic);
        }
    }
    block_reduce(acc, mx, ic, &partials[blockIdx.x]);
}

// Sum the partials in index order (one block; thread k owns sum k).
__global__ void k_diag_finish(const DiagPartial *partials, int n, DiagPartial *result)
{
    const int k = threadIdx.x;
    if (k < kNumSums) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s += partials[b].sums[k];
        result->sums[k] = s;
    } else if (k < kNumSums + kNumMax) {
        double m = 0.0;
        for (int b = 0; b < n; ++b) m = fmax(m, partials[b].maxv[k - kNumSums]);
        result->maxv[k - kNumSums] = m;
    } else if (k < kNumSums + kNumMax + kNumInt) {
        long long s = 0;
        for (int b = 0; b < n; ++b) s += partials[b].ints[k - kNumSums - kNumMax];
        result->ints[k - kNumSums - kNumMax] = s;
    }
}

}  // namespace

int diag_grid_blocks(int num_sms) { return num_sms * 4; }

template <typename real>
cudaError_t launch_diag(const View<real> &v, int N, Box b, const DiagCoef &c,
                        DiagPartial *partials, int nblocks, DiagPartial *result, cudaStream_t st)
{
    k_diag<real><<<nblocks, NT, 0, st>>>(v, N, b, c, partials);
    k_diag_finish<<<1, 32, 0, st>>>(partials, nblocks, result);
    return cudaGetLastError();
}

template cudaError_t launch_diag<float>(const View<float> &, int, Box, const DiagCoef &, DiagPartial *, int,
                                        DiagPartial *, cudaStream_t);
template cudaError_t launch_diag<double>(const View<double> &, int, Box, const DiagCoef &, DiagPartial *, int,
                                         DiagPartial *, cudaStream_t);

}  // namespace ah
