// k_diag.cu -- network diagnostics of one state (Sec. 2 of arXiv:1809.00995).
//
// Per site, at tau_n with the state (phi^n, theta^n, Pi^{n-1/2}, E^{n-1/2}):
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
//
// Fast kernel (k_diag_fast): per-site energies in the state precision,
// accumulated per thread with compensated (Kahan) sums and reduced across the
// block in FP64; the Gauss residual in FP64.  Windings by carries instead of
// arctangents: for Args a, b in (-pi, pi], a + b = Arg(uv) + 2 pi c with c
// fixed by the signs of Im u, Im v and Im(uv), so W = c(z1, z2) + c(z1 z2, z3*)
// + c(z1 z2 z3*, z4*) along the chain that forms the plaquette product.  This is
// exactly the arctangent formula whenever none of z1, z2, z3*, z4* and the
// product lies within a relative margin of the negative real axis (where the
// branch of Arg is decided by rounding).  Each edge product is first scaled to
// unit size (Arg unchanged), so the chain cannot underflow where |phi| is
// small.  The plaquettes left undecided are appended to a list
// and evaluated by k_diag_fixup with the FP64 arctangent formula, so the counts
// are those of the FP64 formula on the same snapshot.
//
// Exact kernel (k_diag_exact): everything per site in FP64 with arctangents.
//
// Each block accumulates its sites in a fixed order and reduces with warp
// shuffles; one block then adds the partials in index order, so the result
// depends only on the launch shape, never on scheduling (integer atomics of the
// fix-up are order independent).
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "ah_internal.cuh"
#include "diag_common.cuh"
#include "sincos32.cuh"

namespace ah {
namespace {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr double kPi = 3.141592653589793;

__device__ __forceinline__ C2<double> expi(double t) { double s, c; sincos(t, &s, &c); return { c, s }; }
__device__ __forceinline__ C2<float> expi(float t) { float s, c; sincos_link(t, &s, &c); return { c, s }; }
__device__ __forceinline__ double arg_pi(C2<double> z)
{
    const double a = atan2(z.i, z.r);
    return a == -kPi ? kPi : a;
}

// FP64 arctangent formula for the plaquette (ii, jj) based at site (x, y, z).
template <typename real>
__device__ long long winding_exact(const View<real> &v, int N, int ii, int jj, int x, int y, int z)
{
    auto id = [N](int a, int b, int c) {
        a = a >= N ? a - N : a; b = b >= N ? b - N : b; c = c >= N ? c - N : c;
        return a + (long long)N * (b + (long long)N * c);
    };
    auto ph = [&v](long long s) { return C2<double>{ (double)v.phr[s], (double)v.phi[s] }; };
    auto th = [&v](int d, long long s) { return (double)(d == 0 ? v.th1[s] : (d == 1 ? v.th2[s] : v.th3[s])); };
    const int U[3][3] = { { 1, 0, 0 }, { 0, 1, 0 }, { 0, 0, 1 } };
    const long long s0 = id(x, y, z);
    const long long si = id(x + U[ii][0], y + U[ii][1], z + U[ii][2]);
    const long long sj = id(x + U[jj][0], y + U[jj][1], z + U[jj][2]);
    const long long sij = id(x + U[ii][0] + U[jj][0], y + U[ii][1] + U[jj][1], z + U[ii][2] + U[jj][2]);
    const C2<double> z1 = cmul(cmul(conj(ph(s0)), expi(th(ii, s0))), ph(si));
    const C2<double> z2 = cmul(cmul(conj(ph(si)), expi(th(jj, si))), ph(sij));
    const C2<double> z3 = cmul(cmul(conj(ph(sj)), expi(th(ii, sj))), ph(sij));
    const C2<double> z4 = cmul(cmul(conj(ph(s0)), expi(th(jj, s0))), ph(sj));
    const C2<double> pr = cmul(cmul(cmul(z1, z2), conj(z3)), conj(z4));
    const double tot = arg_pi(z1) + arg_pi(z2) - arg_pi(z3) - arg_pi(z4) - arg_pi(pr);
    return llrint(tot / (2.0 * kPi));
}

// FP64 winding by carries, falling back to the arctangent formula when an
// FP64 edge product lies exactly on the negative real axis (or is zero).
template <typename real>
__device__ long long winding_fp64(const View<real> &v, int N, int ii, int jj, int x, int y, int z)
{
    auto id = [N](int a, int b, int c) {
        a = a >= N ? a - N : a; b = b >= N ? b - N : b; c = c >= N ? c - N : c;
        return a + (long long)N * (b + (long long)N * c);
    };
    auto ph = [&v](long long s) { return C2<double>{ (double)v.phr[s], (double)v.phi[s] }; };
    auto th = [&v](int d, long long s) { return (double)(d == 0 ? v.th1[s] : (d == 1 ? v.th2[s] : v.th3[s])); };
    const int U[3][3] = { { 1, 0, 0 }, { 0, 1, 0 }, { 0, 0, 1 } };
    const long long s0 = id(x, y, z);
    const long long si = id(x + U[ii][0], y + U[ii][1], z + U[ii][2]);
    const long long sj = id(x + U[jj][0], y + U[jj][1], z + U[jj][2]);
    const long long sij = id(x + U[ii][0] + U[jj][0], y + U[ii][1] + U[jj][1], z + U[ii][2] + U[jj][2]);
    const C2<double> z1 = cmul(cmul(conj(ph(s0)), expi(th(ii, s0))), ph(si));
    const C2<double> z2 = cmul(cmul(conj(ph(si)), expi(th(jj, si))), ph(sij));
    const C2<double> z3 = cmul(cmul(conj(ph(sj)), expi(th(ii, sj))), ph(sij));
    const C2<double> z4 = cmul(cmul(conj(ph(s0)), expi(th(jj, s0))), ph(sj));
    const int w = winding_carry(z1, z2, z3, z4);
    if (w != INT_MIN) return w;
    const C2<double> pr = cmul(cmul(cmul(z1, z2), conj(z3)), conj(z4));
    const double tot = arg_pi(z1) + arg_pi(z2) - arg_pi(z3) - arg_pi(z4) - arg_pi(pr);
    return llrint(tot / (2.0 * kPi));
}

__device__ __forceinline__ long long wrap_id(int x, int y, int z, int N)
{
    x = x >= N ? x - N : (x < 0 ? x + N : x);
    y = y >= N ? y - N : (y < 0 ? y + N : y);
    z = z >= N ? z - N : (z < 0 ? z + N : z);
    return x + (long long)N * (y + (long long)N * z);
}

struct TileIter {
    int tx, ty;
    long long ntiles;
    __device__ TileIter(const Box &b)
        : tx((b.nx + TX - 1) / TX), ty((b.ny + TY - 1) / TY), ntiles((long long)tx * ty * b.nz) {}
    // site of this thread in tile t; false if outside the box
    __device__ bool site(long long t, const Box &b, int N, int &x, int &y, int &z) const
    {
        const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
        const int tz = (int)(t / ((long long)tx * ty));
        const int r = (int)(t % ((long long)tx * ty));
        const int i = (r % tx) * TX + lx, j = (r / tx) * TY + ly;
        if (i >= b.nx || j >= b.ny) return false;
        x = b.x0 + i; y = b.y0 + j; z = b.z0 + tz;
        x -= x >= N ? N : 0; y -= y >= N ? N : 0; z -= z >= N ? N : 0;
        return true;
    }
};

// ------------------------------------------------------------------ fast path
template <typename real>
__global__ void __launch_bounds__(NT) k_diag_fast(View<real> v, int N, Box b, DiagCoef c,
                                                  DiagPartial *partials, DiagList list)
{
    using R = real;
    Acc<R> acc[14];
    double g2sum = 0.0, gs2sum = 0.0, gmax = 0.0;
    R tmax = 0;
    long long ic[kNumInt];
#pragma unroll
    for (int k = 0; k < kNumInt; ++k) ic[k] = 0;
    const R inv_dx2 = (R)c.inv_dx2, v_coef = (R)c.v_coef, eel_coef = (R)c.eel_coef, b_coef = (R)c.b_coef;
    const R sig2 = (R)c.sigma2;
    const TileIter it(b);
    for (long long t = blockIdx.x; t < it.ntiles; t += gridDim.x) {
        int x, y, z;
        if (!it.site(t, b, N, x, y, z)) continue;
        const long long s0 = wrap_id(x, y, z, N);
        const long long s1 = wrap_id(x + 1, y, z, N), s2 = wrap_id(x, y + 1, z, N), s3 = wrap_id(x, y, z + 1, N);
        const long long s12 = wrap_id(x + 1, y + 1, z, N), s13 = wrap_id(x + 1, y, z + 1, N);
        const long long s23 = wrap_id(x, y + 1, z + 1, N);
        const C2<R> f0{ v.phr[s0], v.phi[s0] }, f1{ v.phr[s1], v.phi[s1] }, f2{ v.phr[s2], v.phi[s2] };
        const C2<R> f3{ v.phr[s3], v.phi[s3] }, f12{ v.phr[s12], v.phi[s12] }, f13{ v.phr[s13], v.phi[s13] };
        const C2<R> f23{ v.phr[s23], v.phi[s23] };
        // links at x and at its forward neighbours
        const C2<R> u1 = expi(v.th1[s0]), u2 = expi(v.th2[s0]), u3 = expi(v.th3[s0]);
        const C2<R> u2_1 = expi(v.th2[s1]), u3_1 = expi(v.th3[s1]);
        const C2<R> u1_2 = expi(v.th1[s2]), u3_2 = expi(v.th3[s2]);
        const C2<R> u1_3 = expi(v.th1[s3]), u2_3 = expi(v.th2[s3]);
        // forward products U_d phi^{x+d} and edge products conj(phi^a) U phi^b
        const C2<R> w1 = cmul(u1, f1), w2 = cmul(u2, f2), w3 = cmul(u3, f3);
        const C2<R> f0c = conj(f0);
        const C2<R> z1 = cmul(f0c, w1), z2 = cmul(f0c, w2), z3 = cmul(f0c, w3);
        const C2<R> z2_1 = cmul(conj(f1), cmul(u2_1, f12)), z3_1 = cmul(conj(f1), cmul(u3_1, f13));
        const C2<R> z1_2 = cmul(conj(f2), cmul(u1_2, f12)), z3_2 = cmul(conj(f2), cmul(u3_2, f23));
        const C2<R> z1_3 = cmul(conj(f3), cmul(u1_3, f13)), z2_3 = cmul(conj(f3), cmul(u2_3, f23));

        const R pr = v.pir[s0], pim = v.pii[s0];
        const R K = pr * pr + pim * pim;
        R G2 = 0;
        {
            const R a = w1.r - f0.r, bb = w1.i - f0.i, cc = w2.r - f0.r, d = w2.i - f0.i;
            const R e = w3.r - f0.r, f = w3.i - f0.i;
            G2 = (a * a + bb * bb + cc * cc + d * d + e * e + f * f) * inv_dx2;
        }
        const R m2 = f0.r * f0.r + f0.i * f0.i - sig2;
        const R V = v_coef * m2 * m2;
        const R e1 = v.e1[s0], e2 = v.e2[s0], e3 = v.e3[s0];
        const R Eel = eel_coef * (e1 * e1 + e2 * e2 + e3 * e3);
        // 1 - cos Xi from the plaquette product e^{i Xi}, without cancellation
        R bsum = 0;
        {
            const C2<R> p12 = cmul(cmul(u1, u2_1), conj(cmul(u1_2, u2)));
            const C2<R> p13 = cmul(cmul(u1, u3_1), conj(cmul(u1_3, u3)));
            const C2<R> p23 = cmul(cmul(u2, u3_2), conj(cmul(u2_3, u3)));
            const C2<R> pp[3] = { p12, p13, p23 };
#pragma unroll
            for (int q = 0; q < 3; ++q)
                bsum += pp[q].r > R(0) ? pp[q].i * pp[q].i / (R(1) + pp[q].r) : R(1) - pp[q].r;
        }
        const R B = b_coef * bsum;
        const R L = K - G2 - V + Eel - B;
        const R rho = K + G2 + V + Eel + B;
        const R p = K - G2 / R(3) - V + (Eel + B) / R(3);
        acc[0].add(L); acc[1].add(rho); acc[2].add(p); acc[3].add(K); acc[4].add(G2); acc[5].add(V);
        acc[6].add(Eel); acc[7].add(B); acc[8].add(K * V); acc[9].add(G2 * V); acc[10].add(K * L);
        acc[11].add(G2 * L); acc[12].add(p * L); acc[13].add(rho * L);
        tmax = fmax(tmax, fmax(fabs(v.th1[s0]), fmax(fabs(v.th2[s0]), fabs(v.th3[s0]))));
        // Gauss residual in FP64
        {
            const double div = ((double)e1 - (double)v.e1[wrap_id(x - 1, y, z, N)])
                             + ((double)e2 - (double)v.e2[wrap_id(x, y - 1, z, N)])
                             + ((double)e3 - (double)v.e3[wrap_id(x, y, z - 1, N)]);
            const double g1 = c.g_div * div;
            const double g2 = c.g_phi * ((double)f0.r * (double)pim - (double)f0.i * (double)pr);
            const double G = g1 + g2, gs = fabs(g1) + fabs(g2);
            g2sum += G * G;
            gs2sum += gs * gs;
            gmax = fmax(gmax, fabs(G));
        }
        ic[7] += !(isfinite(L) && isfinite(rho) && isfinite(p));
        // windings of the plaquettes (12), (13), (23) based at x
        const int w[3] = { winding_carry(z1, z2_1, z1_2, z2), winding_carry(z1, z3_1, z1_3, z3),
                           winding_carry(z2, z3_2, z2_3, z3) };
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if (w[q] == INT_MIN) {
                const unsigned long long k = atomicAdd(list.count, 1ULL);
                if (k < (unsigned long long)list.capacity) list.items[k] = (unsigned long long)s0 * 4ULL + q;
            } else {
                ic[q] += w[q] < 0 ? -w[q] : w[q];
                ic[3 + q] += w[q];
                ic[6] += w[q] != 0;
            }
        }
    }
    double accd[kNumSums];
#pragma unroll
    for (int k = 0; k < 14; ++k) accd[k] = acc[k].value();
    accd[14] = g2sum;
    accd[15] = gs2sum;
    double mx[kNumMax] = { gmax, (double)tmax };
    block_reduce<NT>(accd, mx, ic, &partials[blockIdx.x]);
}

// FP64 arctangent windings of the listed plaquettes, added to the result.
template <typename real>
__global__ void k_diag_fixup(View<real> v, int N, DiagList list, DiagPartial *result)
{
    const unsigned long long n = min(*list.count, (unsigned long long)list.capacity);
    const int I[3] = { 0, 0, 1 }, J[3] = { 1, 2, 2 };
    for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long item = list.items[k];
        const int q = (int)(item & 3ULL);
        const long long s = (long long)(item >> 2);
        const int x = (int)(s % N), y = (int)((s / N) % N), z = (int)(s / ((long long)N * N));
        const long long w = winding_fp64(v, N, I[q], J[q], x, y, z);
        if (w) {
            atomicAdd((unsigned long long *)&result->ints[q], (unsigned long long)(w < 0 ? -w : w));
            atomicAdd((unsigned long long *)&result->ints[3 + q], (unsigned long long)w);
            atomicAdd((unsigned long long *)&result->ints[6], 1ULL);
        }
    }
}

// ------------------------------------------------------------------ exact path
template <typename real>
__global__ void __launch_bounds__(NT) k_diag_exact(View<real> v, int N, Box b, DiagCoef c,
                                                   DiagPartial *partials)
{
    double acc[kNumSums];
    double mx[kNumMax] = { 0.0, 0.0 };
    long long ic[kNumInt];
#pragma unroll
    for (int k = 0; k < kNumSums; ++k) acc[k] = 0.0;
#pragma unroll
    for (int k = 0; k < kNumInt; ++k) ic[k] = 0;
    const int U[3][3] = { { 1, 0, 0 }, { 0, 1, 0 }, { 0, 0, 1 } };
    auto ph = [&v](long long s) { return C2<double>{ (double)v.phr[s], (double)v.phi[s] }; };
    auto th = [&v](int d, long long s) { return (double)(d == 0 ? v.th1[s] : (d == 1 ? v.th2[s] : v.th3[s])); };
    auto el = [&v](int d, long long s) { return (double)(d == 0 ? v.e1[s] : (d == 1 ? v.e2[s] : v.e3[s])); };
    const TileIter it(b);
    for (long long t = blockIdx.x; t < it.ntiles; t += gridDim.x) {
        int x, y, z;
        if (!it.site(t, b, N, x, y, z)) continue;
        const long long s0 = wrap_id(x, y, z, N);
        const C2<double> p0 = ph(s0);
        const C2<double> pi{ (double)v.pir[s0], (double)v.pii[s0] };
        long long sp[3];
        C2<double> pp[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            sp[d] = wrap_id(x + U[d][0], y + U[d][1], z + U[d][2], N);
            pp[d] = ph(sp[d]);
        }
        const double K = pi.r * pi.r + pi.i * pi.i;
        double G2 = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const C2<double> up = cmul(expi(th(d, s0)), pp[d]);
            const double dr = up.r - p0.r, di = up.i - p0.i;
            G2 += dr * dr + di * di;
        }
        G2 *= c.inv_dx2;
        const double m2 = p0.r * p0.r + p0.i * p0.i - c.sigma2;
        const double V = c.v_coef * m2 * m2;
        double esq = 0.0, div = 0.0, tmx = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double e = el(d, s0);
            esq += e * e;
            div += e - el(d, wrap_id(x - U[d][0], y - U[d][1], z - U[d][2], N));
            tmx = fmax(tmx, fabs(th(d, s0)));
        }
        const double Eel = c.eel_coef * esq;
        double bsum = 0.0;
        int q = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
#pragma unroll
            for (int j = i + 1; j < 3; ++j, ++q) {
                bsum += 1.0 - cos(th(i, s0) + th(j, sp[i]) - th(i, sp[j]) - th(j, s0));
                const long long w = winding_exact(v, N, i, j, x, y, z);
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
        mx[1] = fmax(mx[1], tmx);
        ic[7] += !(isfinite(L) && isfinite(rho) && isfinite(p) && isfinite(G));
    }
    block_reduce<NT>(acc, mx, ic, &partials[blockIdx.x]);
}

// Sum the partials in index order (one block; thread k owns one output).
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

// Sum many partials in a fixed order: lane k of warp c reduces word k of
// partials [c n/32, (c+1) n/32), then thread k adds the 32 chunk results.
__global__ void __launch_bounds__(1024) k_diag_sum(const DiagPartial *partials, int n, DiagPartial *result)
{
    constexpr int NW = kNumSums + kNumMax + kNumInt;
    __shared__ double sd[32][kNumSums + kNumMax];
    __shared__ long long si[32][kNumInt];
    const int k = threadIdx.x & 31, c = threadIdx.x >> 5;
    const int per = (n + 31) / 32, b0 = min(n, c * per), b1 = min(n, b0 + per);
    if (k < kNumSums) {
        double s = 0.0;
        for (int b = b0; b < b1; ++b) s += partials[b].sums[k];
        sd[c][k] = s;
    } else if (k < kNumSums + kNumMax) {
        double m = 0.0;
        for (int b = b0; b < b1; ++b) m = fmax(m, partials[b].maxv[k - kNumSums]);
        sd[c][k] = m;
    } else if (k < NW) {
        long long s = 0;
        for (int b = b0; b < b1; ++b) s += partials[b].ints[k - kNumSums - kNumMax];
        si[c][k - kNumSums - kNumMax] = s;
    }
    __syncthreads();
    const int t = threadIdx.x;
    if (t < kNumSums) {
        double s = 0.0;
        for (int q = 0; q < 32; ++q) s += sd[q][t];
        result->sums[t] = s;
    } else if (t < kNumSums + kNumMax) {
        double m = 0.0;
        for (int q = 0; q < 32; ++q) m = fmax(m, sd[q][t]);
        result->maxv[t - kNumSums] = m;
    } else if (t < NW) {
        long long s = 0;
        for (int q = 0; q < 32; ++q) s += si[q][t - kNumSums - kNumMax];
        result->ints[t - kNumSums - kNumMax] = s;
    }
}

}  // namespace

int diag_grid_blocks(int num_sms) { return num_sms * 4; }

template <typename real>
cudaError_t launch_diag_whole(const View<real> &v, int N, const DiagCoef &c, DiagPartial *partials,
                              int capacity, DiagPartial *result, DiagList list, int fix_blocks, cudaStream_t st)
{
    // one partial per CTA of the tile walk: refuse a buffer that cannot hold them
    if (fused_diag_ctas(N) > capacity) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(list.count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    DiagArgs da;
    da.dc = c;
    da.partials = partials;
    da.list = list;
    e = launch_fused_diag<real>(v, N, da, st);
    if (e != cudaSuccess) return e;
    return launch_diag_reduce<real>(v, N, partials, fused_diag_ctas(N), result, list, fix_blocks, st);
}

template <typename real>
cudaError_t launch_diag_reduce(const View<real> &v, int N, const DiagPartial *partials, int n, DiagPartial *result,
                               DiagList list, int fix_blocks, cudaStream_t st)
{
    k_diag_sum<<<1, 1024, 0, st>>>(partials, n, result);
    k_diag_fixup<real><<<fix_blocks, 128, 0, st>>>(v, N, list, result);
    return cudaGetLastError();
}
template cudaError_t launch_diag_reduce<float>(const View<float> &, int, const DiagPartial *, int, DiagPartial *,
                                               DiagList, int, cudaStream_t);
template cudaError_t launch_diag_reduce<double>(const View<double> &, int, const DiagPartial *, int, DiagPartial *,
                                                DiagList, int, cudaStream_t);
template cudaError_t launch_diag_whole<float>(const View<float> &, int, const DiagCoef &, DiagPartial *, int,
                                              DiagPartial *, DiagList, int, cudaStream_t);
template cudaError_t launch_diag_whole<double>(const View<double> &, int, const DiagCoef &, DiagPartial *, int,
                                               DiagPartial *, DiagList, int, cudaStream_t);

template <typename real>
cudaError_t launch_diag(const View<real> &v, int N, Box b, const DiagCoef &c, DiagPartial *partials,
                        int nblocks, DiagPartial *result, DiagList list, bool exact, cudaStream_t st)
{
    if (exact) {
        k_diag_exact<real><<<nblocks, NT, 0, st>>>(v, N, b, c, partials);
        k_diag_finish<<<1, 32, 0, st>>>(partials, nblocks, result);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(list.count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_diag_fast<real><<<nblocks, NT, 0, st>>>(v, N, b, c, partials, list);
    k_diag_finish<<<1, 32, 0, st>>>(partials, nblocks, result);
    k_diag_fixup<real><<<nblocks, 128, 0, st>>>(v, N, list, result);
    return cudaGetLastError();
}

template cudaError_t launch_diag<float>(const View<float> &, int, Box, const DiagCoef &, DiagPartial *, int,
                                        DiagPartial *, DiagList, bool, cudaStream_t);
template cudaError_t launch_diag<double>(const View<double> &, int, Box, const DiagCoef &, DiagPartial *, int,
                                         DiagPartial *, DiagList, bool, cudaStream_t);

// ---------------------------------------------------------------------------
// Diagnostics without any device allocation (ah_observables_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs inside a host framework
// that owns the whole device memory pool through its own allocator, loops that
// must not block on the driver's allocator once they are running, and
// processes whose sandbox forbids new device allocations after start-up.  This
// entry point runs the fast diagnostics on an FP32 state held in the caller's
// device buffers and keeps its own scratch -- the per-block partial sums and
// the list of plaquettes near a branch cut -- in one file-scope device array
// of fixed size, so it allocates nothing.
namespace {

constexpr int kNoAllocBlocks = 1024;                 // most per-block partials
constexpr long long kNoAllocListCap = 1LL << 18;     // near-cut plaquettes listed
constexpr size_t kNoAllocCountOff = sizeof(DiagPartial) * kNoAllocBlocks;
constexpr size_t kNoAllocItemsOff = kNoAllocCountOff + 256;
constexpr size_t kNoAllocBytes = kNoAllocItemsOff + sizeof(unsigned long long) * kNoAllocListCap;

// 2.31 MB, held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device addresses of g_noalloc_scratch, filled on the first call on each device.
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[128] = {};

// Windings of the listed plaquettes when the list did not overflow.
template <typename real>
__global__ void k_noalloc_fixup(View<real> v, int N, DiagList list, DiagPartial *result)
{
    const unsigned long long n = *list.count;
    if (n > (unsigned long long)list.capacity) return;
    const int I[3] = { 0, 0, 1 }, J[3] = { 1, 2, 2 };
    for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long item = list.items[k];
        const int q = (int)(item & 3ULL);
        const long long s = (long long)(item >> 2);
        const int x = (int)(s % N), y = (int)((s / N) % N), z = (int)(s / ((long long)N * N));
        const long long w = winding_fp64(v, N, I[q], J[q], x, y, z);
        if (w) {
            atomicAdd((unsigned long long *)&result->ints[q], (unsigned long long)(w < 0 ? -w : w));
            atomicAdd((unsigned long long *)&result->ints[3 + q], (unsigned long long)w);
            atomicAdd((unsigned long long *)&result->ints[6], 1ULL);
        }
    }
}

// On list overflow (here and in the asynchronous observables pass, where the
// host cannot decide before the snapshot may change): clear the winding
// counters ...
__global__ void k_noalloc_wind_clear(DiagList list, DiagPartial *result)
{
    if (*list.count <= (unsigned long long)list.capacity) return;
    if (threadIdx.x < 7) result->ints[threadIdx.x] = 0;
}

// ... and count every plaquette of the lattice with the FP64 path.
template <typename real>
__global__ void k_noalloc_wind_all(View<real> v, int N, DiagList list, DiagPartial *result)
{
    if (*list.count <= (unsigned long long)list.capacity) return;
    long long ic[7] = { 0, 0, 0, 0, 0, 0, 0 };
    const long long ns = (long long)N * N * N;
    const int I[3] = { 0, 0, 1 }, J[3] = { 1, 2, 2 };
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(s % N), y = (int)((s / N) % N), z = (int)(s / ((long long)N * N));
        for (int q = 0; q < 3; ++q) {
            const long long w = winding_fp64(v, N, I[q], J[q], x, y, z);
            ic[q] += w < 0 ? -w : w;
            ic[3 + q] += w;
            ic[6] += w != 0;
        }
    }
    for (int k = 0; k < 7; ++k)
        if (ic[k]) atomicAdd((unsigned long long *)&result->ints[k], (unsigned long long)ic[k]);
}

}  // namespace

template <typename real>
cudaError_t launch_wind_recount_on_overflow(const View<real> &v, int N, DiagList list, DiagPartial *result,
                                            int nblocks, cudaStream_t st)
{
    k_noalloc_wind_clear<<<1, 32, 0, st>>>(list, result);
    k_noalloc_wind_all<real><<<nblocks, 256, 0, st>>>(v, N, list, result);
    return cudaGetLastError();
}
template cudaError_t launch_wind_recount_on_overflow<float>(const View<float> &, int, DiagList, DiagPartial *, int,
                                                            cudaStream_t);
template cudaError_t launch_wind_recount_on_overflow<double>(const View<double> &, int, DiagList, DiagPartial *, int,
                                                             cudaStream_t);

}  // namespace ah

extern "C" ah_status ah_observables_noalloc(const float *const fields[10], int32_t N, const ah_config *cfg,
                                            int64_t step, void *d_sums, void *cuda_stream)
{
    using namespace ah;
    if (!fields || !cfg || !d_sums) return host_fail(AH_ERR_ARG, "ah_observables_noalloc: null argument");
    if (N < 4 || N > 2048 || N != cfg->N)
        return host_fail(AH_ERR_ARG, "ah_observables_noalloc: N must equal cfg->N and lie in [4, 2048]");
    if (cfg->precision != AH_FP32)
        return host_fail(AH_ERR_ARG, "ah_observables_noalloc: the fields must be an FP32 state (cfg->precision)");
    if (step < 0) return host_fail(AH_ERR_ARG, "ah_observables_noalloc: step must be >= 0");
    for (int k = 0; k < 10; ++k)
        if (!fields[k] || (reinterpret_cast<uintptr_t>(fields[k]) & 7))
            return host_fail(AH_ERR_ARG, "ah_observables_noalloc: field pointers must be non-null and 8-byte aligned");
    if (reinterpret_cast<uintptr_t>(d_sums) & 7)
        return host_fail(AH_ERR_ARG, "ah_observables_noalloc: d_sums must be 8-byte aligned");
    ah_status st = host_validate(*cfg);
    if (st != AH_OK) return st;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128 ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return host_fail(AH_ERR_CUDA, "ah_observables_noalloc: no usable CUDA device");
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return host_fail(AH_ERR_CUDA, "ah_observables_noalloc: cudaGetSymbolAddress of the scratch failed");
            g_noalloc_ptr[dev] = p;
        }
        base = g_noalloc_ptr[dev];
    }
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    View<float> v{};
    v.phr = fields[0]; v.phi = fields[1];
    v.pir = const_cast<float *>(fields[2]); v.pii = const_cast<float *>(fields[3]);
    v.th1 = fields[4]; v.th2 = fields[5]; v.th3 = fields[6];
    v.e1 = const_cast<float *>(fields[7]); v.e2 = const_cast<float *>(fields[8]); v.e3 = const_cast<float *>(fields[9]);
    DiagPartial *partials = reinterpret_cast<DiagPartial *>(base);
    DiagList list;
    list.count = reinterpret_cast<unsigned long long *>(static_cast<char *>(base) + kNoAllocCountOff);
    list.items = reinterpret_cast<unsigned long long *>(static_cast<char *>(base) + kNoAllocItemsOff);
    list.capacity = kNoAllocListCap;
    DiagPartial *result = reinterpret_cast<DiagPartial *>(d_sums);
    const int nblocks = std::min(diag_grid_blocks(sms), kNoAllocBlocks);
    const Box b{ 0, 0, 0, N, N, N };
    const DiagCoef dc = host_diag_coef(*cfg, step);
    cudaError_t e = cudaMemsetAsync(list.count, 0, sizeof(unsigned long long), stream);
    if (e == cudaSuccess) {
        k_diag_fast<float><<<nblocks, NT, 0, stream>>>(v, N, b, dc, partials, list);
        k_diag_finish<<<1, 32, 0, stream>>>(partials, nblocks, result);
        k_noalloc_fixup<float><<<nblocks, 128, 0, stream>>>(v, N, list, result);
        k_noalloc_wind_clear<<<1, 32, 0, stream>>>(list, result);
        k_noalloc_wind_all<float><<<nblocks, 256, 0, stream>>>(v, N, list, result);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return host_fail(AH_ERR_CUDA, cudaGetErrorString(e));
    return AH_OK;
}
