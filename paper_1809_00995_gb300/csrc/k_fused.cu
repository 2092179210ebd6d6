// k_fused.cu -- fused leapfrog step: both kicks and both drifts of one time
// step (Eqs. up_pi, up_E, up_phi, up_A of arXiv:1809.00995) in one z-marching
// kernel.
//
// A CTA owns a TX x TY column of sites in the XY plane and a chunk of z planes.
// For each plane z it keeps, in shared memory, the link exponentials
// U_d = e^{i theta_d} and phi of planes z and z+1 on the tile plus a one-site
// halo ring, and the plaquette sines sin Xi_ij = Im(U_i U_j^{x+i} conj(U_i^{x+j})
// conj(U_j)) of plane z on the tile plus its low halos.  Each link exponential is
// computed once per site and shared by the covariant Laplacian, the scalar
// current and the three plaquettes; each plaquette sine is computed once and
// shared by the four E kicks that use it.  Values of plane z-1 that a site
// needs (phi, U_3, sin Xi_13, sin Xi_23) stay in the owning thread's registers
// as the CTA marches up in z, and the next plane's fields are prefetched into
// registers one plane ahead.
//
// phi and theta are read from one buffer and written to the other (ping-pong),
// Pi and E are updated in place, so every step reads and writes the 10-real
// state exactly once from DRAM; halo re-reads are served by L2.  Periodic
// boundaries are applied in the index arithmetic.
//
// The same tile walk serves three kernels: k_fused (one lattice, one step),
// k_fused_batch (persistent CTAs over the tiles of many lattices) and, in
// MODE_DIAG, k_fused_diag (the whole-lattice diagnostics of Sec. 2: energy
// sums, Gauss residual and plaquette windings of the current state, nothing
// written back).  The shapes (tile height, sites per thread in x, resident
// CTAs per SM) and the number of z chunks per column are chosen by the
// autotuner; a chunk count that fills the last wave of CTAs matters because
// each CTA marches a whole chunk.
#include "ah_internal.cuh"
#include "diag_common.cuh"
#include "sincos32.cuh"
#include "fused_common.cuh"

namespace ah {
namespace {

// Kernel modes: the step, or the diagnostics of the current state (the same
// tile walk with nothing written back).
enum { MODE_STEP = 0, MODE_DIAG = 1 };

// Each thread owns RX consecutive sites in x times RY rows (y stride 8).
// One work item of the fused step: tile (bx, by) of plane chunk bz, marched in z.

// IT: site-index type (int when N^3 < 2^31, so every field address is one
// 32 x 32 -> 64-bit multiply-add; long long otherwise).
template <typename real, int TY, int RX, typename IT, int MODE = MODE_STEP>
__device__ __forceinline__ void fused_tile(const View<real> &v, int N, int zc, const KickCoef<real> &c,
                                           int bx, int by, int bz, unsigned char *smem_raw,
                                           const DiagArgs *da = nullptr)
{
    using G = Geo<real, TY, RX>;
    using IO = Row<real, RX>;
    constexpr int TX = G::TX, RY = G::RY, NS = G::NS, EX = G::EX, EY = G::EY, NE = G::NE, PX = G::PX;
    cpx<real> *sU = reinterpret_cast<cpx<real> *>(smem_raw);   // [2 planes][3 dirs][NE]
    cpx<real> *sF = sU + 2 * 3 * NE;                            // [2 planes][NE] phi
    real *sP = reinterpret_cast<real *>(sF + 2 * NE);           // [3][NP] sin Xi_12, _13, _23
    C2<real> *sE = reinterpret_cast<C2<real> *>(smem_raw + G::diag_off);   // MODE_DIAG: [3][NE] edges

    const int tid = threadIdx.x, lx = tid & 31, wy = tid >> 5;
    const int x0 = bx * TX, y0 = by * TY;
    const int z0 = bz * zc;
    constexpr bool STEP = MODE == MODE_STEP, DIAG = MODE == MODE_DIAG;
    // per-thread diagnostic accumulators (MODE_DIAG): the energy sums of
    // ah_obs 3..13 (compensated, state precision; 0..2 follow from 3..7), the
    // Gauss residual sums and max (FP64), max |theta|, winding counters,
    // non-finite sites
    Acc<real> dacc[14];
    real dtmax = real(0);
    int dic[kNumInt] = { 0, 0, 0, 0, 0, 0, 0, 0 };   // per thread at most 3 x 2048 planes x |W| <= 2
    // Gauss residual G = g_div div E + g_phi Im(conj(phi) Pi): FP64 for FP64
    // data; for FP32 data in double-float arithmetic (each G to about 2^-44 of
    // |g_div div E| + |g_phi Im(conj(phi) Pi)|), G^2 and that scale^2 summed
    // with compensation after scaling by 2^60, max |G| kept as a double-float
    double dg2 = 0.0, dgs2 = 0.0, dgmax = 0.0;
    Acc<float> fg2, fgs2;
    DF fgmax{ 0.f, 0.f };
    DF cg_div{ 0.f, 0.f }, cg_phi{ 0.f, 0.f };
    real k_inv_dx2 = 0, k_v = 0, k_eel = 0, k_b = 0, k_sig2 = 0;
    if constexpr (DIAG) {
        const DiagCoef &dc = da->dc;
        cg_div = df_from(dc.g_div);
        cg_phi = df_from(dc.g_phi);
        k_inv_dx2 = (real)dc.inv_dx2; k_v = (real)dc.v_coef; k_eel = (real)dc.eel_coef;
        k_b = (real)dc.b_coef; k_sig2 = (real)dc.sigma2;
    }
    auto diag_flush = [&]() {
        if constexpr (DIAG) {
            double accd[kNumSums];
#pragma unroll
            for (int k = 3; k < 14; ++k) accd[k] = dacc[k].value();
            // the sums of L, rho and p are linear in those of K, G2, V, E_el, B
            accd[0] = accd[3] - accd[4] - accd[5] + accd[6] - accd[7];
            accd[1] = accd[3] + accd[4] + accd[5] + accd[6] + accd[7];
            accd[2] = accd[3] - accd[4] * (1.0 / 3.0) - accd[5] + (accd[6] + accd[7]) * (1.0 / 3.0);
            if constexpr (sizeof(real) == 4) {
                dg2 = fg2.value() * 0x1p-60;
                dgs2 = fgs2.value() * 0x1p-60;
                dgmax = (double)fgmax.h + (double)fgmax.l;
            }
            accd[14] = dg2;
            accd[15] = dgs2;
            double mx[kNumMax] = { dgmax, (double)dtmax };
            const int cta = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
            long long dil[kNumInt];
#pragma unroll
            for (int k = 0; k < kNumInt; ++k) dil[k] = dic[k];
            block_reduce<256>(accd, mx, dil, &da->partials[cta]);
        }
    };
    if (z0 >= N) { diag_flush(); return; }
    const int z1 = min(z0 + zc, N);
    const IT NN = (IT)N * (IT)N;

    // own rows: in-plane offset of the first of the RX sites, validity
    int roff[RY];
    bool wr[RY];
#pragma unroll
    for (int my = 0; my < RY; ++my) {
        const int gx = x0 + RX * lx, gy = y0 + wy + 8 * my;
        wr[my] = gx < N && gy < N;
        roff[my] = wrapm(gx, N) + N * wrapm(gy, N);
    }
    auto eix = [&](int m) { return (wy + 8 * (m / RX) + 1) * EX + RX * lx + (m % RX) + 1; };
    auto pix = [&](int m) { return (wy + 8 * (m / RX) + 1) * PX + RX * lx + (m % RX) + 1; };
    // halo task (tid < NHALO): one site of the halo ring
    const bool has_halo = tid < G::NHALO;
    int hoff, heix;
    {
        int ex = 0, ey = 0;
        const int h = tid;
        if (h < EX) { ex = h; ey = 0; }
        else if (h < 2 * EX) { ex = h - EX; ey = EY - 1; }
        else if (h < 2 * EX + TY) { ex = 0; ey = 1 + h - 2 * EX; }
        else { ex = EX - 1; ey = 1 + h - 2 * EX - TY; }
        hoff = wrapm(x0 + ex - 1, N) + N * wrapm(y0 + ey - 1, N);
        heix = ey * EX + ex;
    }

    // register prefetch of one plane's phi, theta: own sites [0, NS), halo [NS]
    real fth[NS + 1][3], fph[NS + 1][2];
    auto load_plane = [&](int z) {           // z in [-1, N + 1]
        const int zz = z < 0 ? z + N : (z >= N ? z - N : z);
        const IT base = (IT)zz * NN;
#pragma unroll
        for (int my = 0; my < RY; ++my) {
            const IT s = base + (IT)roff[my];
            real t[RX];
            IO::ld(v.th1 + s, t);
#pragma unroll
            for (int mx = 0; mx < RX; ++mx) fth[my * RX + mx][0] = t[mx];
            IO::ld(v.th2 + s, t);
#pragma unroll
            for (int mx = 0; mx < RX; ++mx) fth[my * RX + mx][1] = t[mx];
            IO::ld(v.th3 + s, t);
#pragma unroll
            for (int mx = 0; mx < RX; ++mx) fth[my * RX + mx][2] = t[mx];
            IO::ld(v.phr + s, t);
#pragma unroll
            for (int mx = 0; mx < RX; ++mx) fph[my * RX + mx][0] = t[mx];
            IO::ld(v.phi + s, t);
#pragma unroll
            for (int mx = 0; mx < RX; ++mx) fph[my * RX + mx][1] = t[mx];
        }
        if (has_halo) {
            const IT s = base + (IT)hoff;
            fth[NS][0] = v.th1[s]; fth[NS][1] = v.th2[s]; fth[NS][2] = v.th3[s];
            fph[NS][0] = v.phr[s]; fph[NS][1] = v.phi[s];
        }
    };
    // U and phi of the prefetched plane into shared buffer b
    auto store_plane = [&](int b) {
#pragma unroll
        for (int t = 0; t <= NS; ++t) {
            if (t < NS || has_halo) {
                const int e = t < NS ? eix(t) : heix;
                real sn[3], co[3];
                sincos_link3(fth[t], sn, co);
#pragma unroll
                for (int d = 0; d < 3; ++d) sU[(b * 3 + d) * NE + e] = { co[d], sn[d] };
                sF[b * NE + e] = { fph[t][0], fph[t][1] };
            }
        }
    };

    // own-site registers carried along z
    cpx<real> ph_m[NS], ph_0[NS], u3_m[NS];
    real th_0[NS][3], p13_m[NS], p23_m[NS];
    real e3_m[NS];                           // MODE_DIAG: E_3 of plane z-1
    // MODE_DIAG: scaled edge products conj(phi^x) U_d^x phi^{x+d} of the own
    // sites for d = 1, 2 in plane z (computed one plane ahead) and d = 3
    using Z = C2<real>;
    Z ed1[NS], ed2[NS], ed3[NS];
    auto zc_ = [](cpx<real> a) { return Z{ a.r, a.i }; };
    auto edge = [&](cpx<real> fa, cpx<real> u, cpx<real> fb) {
        Z z = cmul(conj(zc_(fa)), cmul(zc_(u), zc_(fb)));
        unit_scale_or_nan(z);
        return z;
    };
    if constexpr (DIAG) {
        const IT base = (IT)(z0 == 0 ? N - 1 : z0 - 1) * NN;
#pragma unroll
        for (int m = 0; m < NS; ++m) e3_m[m] = v.e3[base + (IT)roff[m / RX] + (IT)(m % RX)];
    }

    // prologue: planes z0-1 and z0
    // ring slot of plane z: (z - z0 + 1) & 1
    load_plane(z0 - 1);
    constexpr int bm = 0, b0 = 1;
    store_plane(bm);
#pragma unroll
    for (int m = 0; m < NS; ++m) ph_m[m] = { fph[m][0], fph[m][1] };
    load_plane(z0);
    store_plane(b0);
#pragma unroll
    for (int m = 0; m < NS; ++m) {
        ph_0[m] = { fph[m][0], fph[m][1] };
        th_0[m][0] = fth[m][0]; th_0[m][1] = fth[m][1]; th_0[m][2] = fth[m][2];
    }
    load_plane(z0 + 1);
    __syncthreads();
#pragma unroll
    for (int m = 0; m < NS; ++m) {
        const int e = eix(m);
        const cpx<real> *Um = sU + bm * 3 * NE, *U0 = sU + b0 * 3 * NE;
        u3_m[m] = Um[2 * NE + e];
        p13_m[m] = plaq(Um[e], Um[2 * NE + e + 1], U0[e], Um[2 * NE + e]);
        p23_m[m] = plaq(Um[NE + e], Um[2 * NE + e + EX], U0[NE + e], Um[2 * NE + e]);
        if constexpr (DIAG) {
            const cpx<real> *F0p = sF + b0 * NE;
            ed1[m] = edge(F0p[e], U0[e], F0p[e + 1]);
            ed2[m] = edge(F0p[e], U0[NE + e], F0p[e + EX]);
        }
    }
    __syncthreads();

    // one plane z; BC (compile time) is the ring slot of plane z
    auto plane_step = [&](int z, auto bc_tag) {
        constexpr int bc = decltype(bc_tag)::value, bn = 1 - bc;
        const IT base = (IT)z * NN;
        // Pi, E of plane z (consumed after two barriers)
        real pr[NS], pim[NS], e1[NS], e2[NS], e3[NS];
#pragma unroll
        for (int my = 0; my < RY; ++my) {
            const IT s = base + (IT)roff[my];
            IO::ld(v.pir + s, pr + my * RX);
            IO::ld(v.pii + s, pim + my * RX);
            IO::ld(v.e1 + s, e1 + my * RX);
            IO::ld(v.e2 + s, e2 + my * RX);
            IO::ld(v.e3 + s, e3 + my * RX);
        }
        // A: links and phi of plane z+1 from the prefetch, then prefetch z+2
        store_plane(bn);
        cpx<real> ph_p[NS];
        real th_p[NS][3];
#pragma unroll
        for (int m = 0; m < NS; ++m) {
            ph_p[m] = { fph[m][0], fph[m][1] };
            th_p[m][0] = fth[m][0]; th_p[m][1] = fth[m][1]; th_p[m][2] = fth[m][2];
        }
        load_plane(z + 2);
        __syncthreads();

        // B: plaquette sines of plane z on the tile (own sites) and its low halos
        const cpx<real> *U0 = sU + bc * 3 * NE, *U1p = sU + bn * 3 * NE;
        real p12[NS], p13[NS], p23[NS];
        [[maybe_unused]] Z ez1[NS], ez2[NS];      // MODE_DIAG: own d = 1, 2 edges of plane z+1
        // MODE_DIAG: a plaquette whose four edges all have |Arg| < pi/4 has
        // W = 0; when every edge that the CTA's plaquettes of plane z use passes
        // that test (smooth regions), the carry chains are skipped
        [[maybe_unused]] bool own_smooth = true;
        [[maybe_unused]] auto smooth1 = [](const Z &z) { return z.r > real(1.001) * fabs(z.i); };
        [[maybe_unused]] real bcos[NS];          // MODE_DIAG: 1 - cos Xi summed over the three orientations
#pragma unroll
        for (int m = 0; m < NS; ++m) {
            const int e = eix(m), p = pix(m);
            if constexpr (DIAG) {
                const cpx<real> x12 = plaq2(U0[e], U0[NE + e + 1], U0[e + EX], U0[NE + e]);
                const cpx<real> x13 = plaq2(U0[e], U0[2 * NE + e + 1], U1p[e], U0[2 * NE + e]);
                const cpx<real> x23 = plaq2(U0[NE + e], U0[2 * NE + e + EX], U1p[NE + e], U0[2 * NE + e]);
                p12[m] = x12.i; p13[m] = x13.i; p23[m] = x23.i;
                bcos[m] = one_minus_cos(x12.r, x12.i) + one_minus_cos(x13.r, x13.i) +
                          one_minus_cos(x23.r, x23.i);
            } else {
                p12[m] = plaq(U0[e], U0[NE + e + 1], U0[e + EX], U0[NE + e]);
                p13[m] = plaq(U0[e], U0[2 * NE + e + 1], U1p[e], U0[2 * NE + e]);
                p23[m] = plaq(U0[NE + e], U0[2 * NE + e + EX], U1p[NE + e], U0[2 * NE + e]);
            }
            if constexpr (STEP) {              // the sines feed only the E kick
                sP[p] = p12[m];
                sP[G::NP + p] = p13[m];
                sP[2 * G::NP + p] = p23[m];
            }
        }
        if constexpr (DIAG) {
            // own edges of plane z, then the right column's d = 2, 3 and the
            // top row's d = 1, 3 edges that the tile's last column / row need
            const cpx<real> *F0 = sF + bc * NE, *F1 = sF + bn * NE;
#pragma unroll
            for (int m = 0; m < NS; ++m) {
                const int e = eix(m);
                ed3[m] = edge(F0[e], U0[2 * NE + e], ph_p[m]);
                ez1[m] = edge(F1[e], U1p[e], F1[e + 1]);
                ez2[m] = edge(F1[e], U1p[NE + e], F1[e + EX]);
                sE[e] = ed1[m];
                sE[NE + e] = ed2[m];
                sE[2 * NE + e] = ed3[m];
                own_smooth = own_smooth && smooth1(ed1[m]) && smooth1(ed2[m]) && smooth1(ed3[m]) &&
                             smooth1(ez1[m]) && smooth1(ez2[m]);
            }
            if (tid < TY) {
                const int e = (tid + 1) * EX + EX - 1;
                const Z a = edge(F0[e], U0[NE + e], F0[e + EX]), b = edge(F0[e], U0[2 * NE + e], F1[e]);
                sE[NE + e] = a;
                sE[2 * NE + e] = b;
                own_smooth = own_smooth && smooth1(a) && smooth1(b);
            } else if (tid < TY + TX) {
                const int e = (EY - 1) * EX + tid - TY + 1;
                const Z a = edge(F0[e], U0[e], F0[e + 1]), b = edge(F0[e], U0[2 * NE + e], F1[e]);
                sE[e] = a;
                sE[2 * NE + e] = b;
                own_smooth = own_smooth && smooth1(a) && smooth1(b);
            }
        }
        if (STEP && tid < G::NPHALO) {
            const int px = tid < PX ? tid : 0, py = tid < PX ? 0 : tid - PX + 1;
            const int e = py * EX + px, p = py * PX + px;
            sP[p] = plaq(U0[e], U0[NE + e + 1], U0[e + EX], U0[NE + e]);
            sP[G::NP + p] = plaq(U0[e], U0[2 * NE + e + 1], U1p[e], U0[2 * NE + e]);
            sP[2 * G::NP + p] = plaq(U0[NE + e], U0[2 * NE + e + EX], U1p[NE + e], U0[2 * NE + e]);
        }
        [[maybe_unused]] bool smooth_cta = false;
        if constexpr (DIAG) smooth_cta = __syncthreads_and(own_smooth) != 0;
        else __syncthreads();

        // C: kicks and drifts of the own sites of plane z
        const cpx<real> *F0 = sF + bc * NE;
        real o_pr[NS], o_pi[NS], o_e1[NS], o_e2[NS], o_e3[NS], o_fr[NS], o_fi[NS], o_t1[NS], o_t2[NS], o_t3[NS];
#pragma unroll
        for (int m = 0; m < NS; ++m) {
            const int e = eix(m), p = pix(m);
            const cpx<real> f0 = ph_0[m];
            const cpx<real> u1 = U0[e], u2 = U0[NE + e], u3 = U0[2 * NE + e];
            const cpx<real> u1m = U0[e - 1], u2m = U0[NE + e - EX], u3m = u3_m[m];
            // forward products U_d phi^{x+d}; backward conj(U_d^{x-d}) phi^{x-d}
            const cpx<real> w1 = mul(u1, F0[e + 1]), w2 = mul(u2, F0[e + EX]), w3 = mul(u3, ph_p[m]);
            const cpx<real> b1 = mul({ u1m.r, -u1m.i }, F0[e - 1]);
            const cpx<real> b2 = mul({ u2m.r, -u2m.i }, F0[e - EX]);
            const cpx<real> b3 = mul({ u3m.r, -u3m.i }, ph_m[m]);
            const real lr = (w1.r + b1.r) + (w2.r + b2.r) + (w3.r + b3.r) - real(6) * f0.r;
            const real li = (w1.i + b1.i) + (w2.i + b2.i) + (w3.i + b3.i) - real(6) * f0.i;
            const real pot = c.c_pot * (f0.r * f0.r + f0.i * f0.i - c.sigma2);
            const real npr = c.c_damp * pr[m] - pot * f0.r + c.c_lap * lr;
            const real npi = c.c_damp * pim[m] - pot * f0.i + c.c_lap * li;
            // current Im[conj(U_i phi^{x+i}) phi^x]
            const real cu1 = w1.r * f0.i - w1.i * f0.r;
            const real cu2 = w2.r * f0.i - w2.i * f0.r;
            const real cu3 = w3.r * f0.i - w3.i * f0.r;
            // curls sum_{j != i} [sin Xi_ij^x - sin Xi_ij^{x-j}], Xi_ji = -Xi_ij
            const real q12 = p12[m], q13 = p13[m], q23 = p23[m];
            const real cl1 = (q12 - sP[p - PX]) + (q13 - p13_m[m]);
            const real cl2 = (sP[p - 1] - q12) + (q23 - p23_m[m]);
            const real cl3 = (sP[G::NP + p - 1] - q13) + (sP[2 * G::NP + p - PX] - q23);
            const real ne1 = c.c_edamp * e1[m] + c.c_cur * cu1 - c.c_curl * cl1;
            const real ne2 = c.c_edamp * e2[m] + c.c_cur * cu2 - c.c_curl * cl2;
            const real ne3 = c.c_edamp * e3[m] + c.c_cur * cu3 - c.c_curl * cl3;
            if constexpr (DIAG) if (wr[m / RX]) {
                const real K = pr[m] * pr[m] + pim[m] * pim[m];
                const real d1r = w1.r - f0.r, d1i = w1.i - f0.i, d2r = w2.r - f0.r, d2i = w2.i - f0.i;
                const real d3r = w3.r - f0.r, d3i = w3.i - f0.i;
                const real G2 = (d1r * d1r + d1i * d1i + d2r * d2r + d2i * d2i + d3r * d3r + d3i * d3i) *
                                k_inv_dx2;
                const real m2 = f0.r * f0.r + f0.i * f0.i - k_sig2;
                const real V = k_v * m2 * m2;
                const real Eel = k_eel * (e1[m] * e1[m] + e2[m] * e2[m] + e3[m] * e3[m]);
                const real B = k_b * bcos[m];
                const real L = K - G2 - V + Eel - B;
                const real rho = K + G2 + V + Eel + B;
                const real pp = K - G2 * real(1.0 / 3.0) - V + (Eel + B) * real(1.0 / 3.0);
                dacc[3].add(K); dacc[4].add(G2);
                dacc[5].add(V); dacc[6].add(Eel); dacc[7].add(B); dacc[8].add(K * V); dacc[9].add(G2 * V);
                dacc[10].add(K * L); dacc[11].add(G2 * L); dacc[12].add(pp * L); dacc[13].add(rho * L);
                dtmax = fmax(dtmax, fmax(fabs(th_0[m][0]), fmax(fabs(th_0[m][1]), fabs(th_0[m][2]))));
                dic[7] += !(isfinite(L) && isfinite(rho) && isfinite(pp));
                const int my = m / RX, mx = m % RX;
                const int gx = x0 + RX * lx + mx, gy = y0 + wy + 8 * my;
                // Gauss residual (nothing is written in this mode, so the
                // backward neighbours' E are the current ones)
                {
                    const IT s = base + (IT)roff[my] + (IT)mx;
                    const real e1b = v.e1[gx == 0 ? s + (IT)(N - 1) : s - 1];
                    const real e2b = v.e2[gy == 0 ? s + (NN - (IT)N) : s - (IT)N];
                    if constexpr (sizeof(real) == 8) {
                        const DiagCoef &dc = da->dc;
                        const double div = (e1[m] - e1b) + (e2[m] - e2b) + (e3[m] - e3_m[m]);
                        const double g1 = dc.g_div * div;
                        const double g2 = dc.g_phi * (f0.r * pim[m] - f0.i * pr[m]);
                        const double Gs = g1 + g2, gs = fabs(g1) + fabs(g2);
                        dg2 += Gs * Gs;
                        dgs2 += gs * gs;
                        dgmax = fmax(dgmax, fabs(Gs));
                    } else {
                        // differences and products of FP32 values are exact as pairs
                        const DF div = df_add(df_add(two_sum(e1[m], -e1b), two_sum(e2[m], -e2b)),
                                              two_sum(e3[m], -e3_m[m]));
                        const DF a = two_prod(f0.r, pim[m]), b = two_prod(f0.i, pr[m]);
                        const DF g1 = df_mul(cg_div, div), g2 = df_mul(cg_phi, df_add(a, { -b.h, -b.l }));
                        DF Gs = df_add(g1, g2);
                        if (Gs.h < 0.f) Gs = { -Gs.h, -Gs.l };
                        const float gs = fabsf(g1.h) + fabsf(g2.h);
                        const float sg = Gs.h * 0x1p30f, ss = gs * 0x1p30f;
                        fg2.add(sg * sg);
                        fgs2.add(ss * ss);
                        if (Gs.h > fgmax.h || (Gs.h == fgmax.h && Gs.l > fgmax.l)) fgmax = Gs;
                    }
                }
                // windings of the plaquettes (12), (13), (23) based at x (Eq. 9)
                // from their twelve edge products conj(phi^a) U phi^b: the own
                // ones (this plane and, for d = 1, 2, the next) and the x and y
                // neighbours' from shared memory
                const Z z2_1 = sE[NE + e + 1], z3_1 = sE[2 * NE + e + 1];
                const Z z1_2 = sE[e + EX], z3_2 = sE[2 * NE + e + EX];
                int wq[3] = { 0, 0, 0 };
                if (!smooth_cta) {
                    wq[0] = winding_scaled(ed1[m], z2_1, z1_2, ed2[m]);
                    wq[1] = winding_scaled(ed1[m], z3_1, ez1[m], ed3[m]);
                    wq[2] = winding_scaled(ed2[m], z3_2, ez2[m], ed3[m]);
                }
                const unsigned long long site =
                    (unsigned long long)((long long)z * N * (long long)N + (long long)roff[my] + mx);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (wq[q] == INT_MIN) {
                        const unsigned long long k = atomicAdd(da->list.count, 1ULL);
                        if (k < (unsigned long long)da->list.capacity) da->list.items[k] = site * 4ULL + q;
                    } else {
                        dic[q] += wq[q] < 0 ? -wq[q] : wq[q];
                        dic[3 + q] += wq[q];
                        dic[6] += wq[q] != 0;
                    }
                }
            }
            o_pr[m] = npr; o_pi[m] = npi;
            o_e1[m] = ne1; o_e2[m] = ne2; o_e3[m] = ne3;
            o_fr[m] = f0.r + c.dt * npr;
            o_fi[m] = f0.i + c.dt * npi;
            o_t1[m] = th_0[m][0] + c.dt * ne1;
            o_t2[m] = th_0[m][1] + c.dt * ne2;
            o_t3[m] = th_0[m][2] + c.dt * ne3;
            if (c.wrap) {
                o_t1[m] = wrap_phase(o_t1[m]);
                o_t2[m] = wrap_phase(o_t2[m]);
                o_t3[m] = wrap_phase(o_t3[m]);
            }
            // march: plane z becomes z-1
            if constexpr (DIAG) {
                e3_m[m] = e3[m];
                ed1[m] = ez1[m];
                ed2[m] = ez2[m];
            }
            ph_m[m] = f0;
            u3_m[m] = u3;
            p13_m[m] = q13;
            p23_m[m] = q23;
            ph_0[m] = ph_p[m];
            th_0[m][0] = th_p[m][0]; th_0[m][1] = th_p[m][1]; th_0[m][2] = th_p[m][2];
        }
#pragma unroll
        for (int my = 0; my < RY; ++my) {
            if (STEP && wr[my]) {
                const IT s = base + (IT)roff[my];
                const int k = my * RX;
                IO::st(v.pir + s, o_pr + k); IO::st(v.pii + s, o_pi + k);
                IO::st(v.e1 + s, o_e1 + k); IO::st(v.e2 + s, o_e2 + k); IO::st(v.e3 + s, o_e3 + k);
                IO::st(v.ophr + s, o_fr + k); IO::st(v.ophi + s, o_fi + k);
                IO::st(v.oth1 + s, o_t1 + k); IO::st(v.oth2 + s, o_t2 + k); IO::st(v.oth3 + s, o_t3 + k);
            }
        }
        __syncthreads();
    };
    for (int k = 0; z0 + k < z1; k += 2) {
        plane_step(z0 + k, IC<1>{});
        if (z0 + k + 1 < z1) plane_step(z0 + k + 1, IC<0>{});
    }
    diag_flush();
}

template <typename real, int TY, int RX, int MINB, typename IT>
__global__ void __launch_bounds__(256, MINB) k_fused(View<real> v, int N, int zc, KickCoef<real> c)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fused_tile<real, TY, RX, IT>(v, N, zc, c, blockIdx.x, blockIdx.y, blockIdx.z, smem_raw);
}

// Diagnostics of the current state through the step's tile walk (tile 32 x 8,
// nothing written back); one DiagPartial per CTA.
template <typename real, typename IT>
__global__ void __launch_bounds__(256) k_fused_diag(View<real> v, int N, int zc, DiagArgs da)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const KickCoef<real> c{};
    fused_tile<real, 8, 1, IT, MODE_DIAG>(v, N, zc, c, blockIdx.x, blockIdx.y, blockIdx.z, smem_raw, &da);
}

// Batched fused step: persistent CTAs take (lattice, tile) work items from a
// shared counter and advance every lattice of the batch by one step.  Lattices
// that have run all their steps are skipped; each lattice's step number, read
// buffer and coefficient table live in device memory (advanced by
// k_batch_advance), so the same launch sequence can be replayed from a graph.
template <int TY, int RX, int MINB>
__global__ void __launch_bounds__(256, MINB)
k_fused_batch(const BatchLattice *lat, BatchState *state, const int2 *items, const int *nitems,
              unsigned int *counter, int mode)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    const int n = *nitems;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n) break;
        const int L = items[it].x, local = items[it].y;
        const BatchLattice &B = lat[L];
        const int step = state[L].step;
        if (!batch_takes_single(B, step, mode)) continue;
        const int cur = state[L].cur, o = 1 - cur;
        float *const *q = B.q[state[L].pe];
        View<float> v;
        v.phr = B.F.phr[cur]; v.phi = B.F.phi[cur];
        v.th1 = B.F.th[cur][0]; v.th2 = B.F.th[cur][1]; v.th3 = B.F.th[cur][2];
        v.pir = q[0]; v.pii = q[1];
        v.e1 = q[2]; v.e2 = q[3]; v.e3 = q[4];
        v.ophr = B.F.phr[o]; v.ophi = B.F.phi[o];
        v.oth1 = B.F.th[o][0]; v.oth2 = B.F.th[o][1]; v.oth3 = B.F.th[o][2];
        const int bx = local % B.tiles_x, by = (local / B.tiles_x) % B.tiles_y, bz = local / (B.tiles_x * B.tiles_y);
        fused_tile<float, TY, RX, int>(v, B.N, B.zc, B.coefs[step], bx, by, bz, smem_raw);
        __syncthreads();
    }
}

// After a batched step: every lattice that took part (batch_takes_single)
// moves to its next step and swaps its phi/theta buffers; the work counter is
// reset.
__global__ void k_batch_advance(const BatchLattice *lat, BatchState *state, int nlat, unsigned int *counter,
                                int mode)
{
    for (int L = threadIdx.x; L < nlat; L += blockDim.x) {
        if (batch_takes_single(lat[L], state[L].step, mode)) {
            state[L].step += 1;
            state[L].cur ^= 1;
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// Compile-time shapes of the fused step: tile height TY (TY/8 rows per thread),
// RX sites per thread in x (tile width 32 RX; RX = 2 uses 8-byte vector
// accesses and needs an even N), and the minimum resident CTAs per SM the
// register allocation must allow; min_chunk is the shortest z chunk.  The z
// chunk count is either "about 16 waves of CTAs" or (_w) the wave-quantisation
// model of choose_chunks.
struct VariantInfo { int ty, rx, minb, min_chunk; bool wave_model; const char *name; };
constexpr VariantInfo kVariants32[] = {
    { 16, 1, 2, 16, false, "ty16_b2" }, { 16, 1, 3, 16, false, "ty16_b3" }, { 8, 1, 4, 16, false, "ty8_b4" },
    { 8, 1, 3, 16, false, "ty8_b3" },  { 32, 1, 1, 16, false, "ty32_b1" }, { 16, 1, 2, 64, false, "ty16_b2_z64" },
    { 8, 2, 3, 16, false, "x2_ty8_b3" }, { 8, 2, 2, 16, false, "x2_ty8_b2" }, { 16, 2, 2, 16, false, "x2_ty16_b2" },
    { 16, 2, 1, 16, false, "x2_ty16_b1" }, { 8, 1, 4, 16, true, "ty8_b4_w" }, { 8, 1, 3, 16, true, "ty8_b3_w" },
    { 8, 2, 2, 16, true, "x2_ty8_b2_w" }, { 16, 1, 2, 16, true, "ty16_b2_w" },
};
constexpr VariantInfo kVariants64[] = { { 16, 1, 1, 16, false, "ty16_b1" }, { 8, 1, 2, 16, false, "ty8_b2" },
                                        { 8, 2, 1, 16, false, "x2_ty8_b1" }, { 8, 1, 2, 16, true, "ty8_b2_w" } };

}  // namespace

int choose_chunks(int N, long long tiles, int slots, int min_chunk, int extra)
{
    const int nmax = std::max(1, std::min(N / std::max(1, min_chunk), 64));
    int best = 1;
    long long best_cost = -1;
    for (int n = 1; n <= nmax; ++n) {
        const long long waves = (tiles * n + slots - 1) / slots;
        const long long cost = waves * ((N + n - 1) / n + extra);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = n;
        }
    }
    return best;
}

int device_sm_count()
{
    static int sms[64] = {};
    int &n = sms[device_slot()];
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 152;
    }
    return n;
}

namespace {

template <typename real, int TY, int RX, int MINB>
cudaError_t launch_shape(const View<real> &v, int N, const KickCoef<real> &c, int min_chunk, bool wave_model,
                         cudaStream_t st)
{
    using G = Geo<real, TY, RX>;
    if (RX > 1 && (N & 1)) return cudaErrorInvalidValue;
    const bool idx32 = (long long)N * N * N < (1LL << 31);
    static unsigned long long configured = 0;   // per device, once per instantiation
    const unsigned long long dev_bit = 1ULL << device_slot();
    if (!(configured & dev_bit)) {
        cudaError_t e = cudaFuncSetAttribute(k_fused<real, TY, RX, MINB, int>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fused<real, TY, RX, MINB, long long>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem);
        if (e != cudaSuccess) return e;
        configured |= dev_bit;
    }
    const int tx = (N + G::TX - 1) / G::TX, ty = (N + TY - 1) / TY;
    int nch;
    if (wave_model) {
        nch = choose_chunks(N, (long long)tx * ty, device_sm_count() * MINB, min_chunk);
    } else {
        // enough z chunks for several waves of CTAs, chunks of at least min_chunk planes
        nch = (int)((16LL * device_sm_count() + (long long)tx * ty - 1) / ((long long)tx * ty));
        nch = max(1, min(nch, N / min_chunk));
    }
    const int zc = (N + nch - 1) / nch;
    nch = (N + zc - 1) / zc;
    if (idx32) k_fused<real, TY, RX, MINB, int><<<dim3(tx, ty, nch), G::NT, G::smem, st>>>(v, N, zc, c);
    else k_fused<real, TY, RX, MINB, long long><<<dim3(tx, ty, nch), G::NT, G::smem, st>>>(v, N, zc, c);
    return cudaGetLastError();
}

}  // namespace

// Shape used when a simulation is not autotuned: the fastest on GB300 at
// 512^3 and 1024^3 (any N; RX = 1).
template <>
int fused_default_variant<float>() { return 10; }      // ty8_b4_w
template <>
int fused_default_variant<double>() { return 1; }      // ty8_b2

template <>
int fused_variant_count<float>() { return (int)(sizeof(kVariants32) / sizeof(kVariants32[0])); }
template <>
int fused_variant_count<double>() { return (int)(sizeof(kVariants64) / sizeof(kVariants64[0])); }
template <>
const char *fused_variant_name<float>(int k) { return kVariants32[k].name; }
template <>
const char *fused_variant_name<double>(int k) { return kVariants64[k].name; }

template <>
bool fused_variant_ok<float>(int k, int N) { return kVariants32[k].rx == 1 || (N % 2 == 0); }
template <>
bool fused_variant_ok<double>(int k, int N) { return kVariants64[k].rx == 1 || (N % 2 == 0); }

template <>
cudaError_t launch_fused_step<float>(const View<float> &v, int N, const KickCoef<float> &c, int variant,
                                     cudaStream_t st)
{
    if (variant < 0 || variant >= fused_variant_count<float>()) return cudaErrorInvalidValue;
    const int mc = kVariants32[variant].min_chunk;
    const bool wm = kVariants32[variant].wave_model;
    switch (variant) {
    case 0: return launch_shape<float, 16, 1, 2>(v, N, c, mc, wm, st);
    case 1: return launch_shape<float, 16, 1, 3>(v, N, c, mc, wm, st);
    case 2: return launch_shape<float, 8, 1, 4>(v, N, c, mc, wm, st);
    case 3: return launch_shape<float, 8, 1, 3>(v, N, c, mc, wm, st);
    case 4: return launch_shape<float, 32, 1, 1>(v, N, c, mc, wm, st);
    case 5: return launch_shape<float, 16, 1, 2>(v, N, c, mc, wm, st);
    case 6: return launch_shape<float, 8, 2, 3>(v, N, c, mc, wm, st);
    case 7: return launch_shape<float, 8, 2, 2>(v, N, c, mc, wm, st);
    case 8: return launch_shape<float, 16, 2, 2>(v, N, c, mc, wm, st);
    case 9: return launch_shape<float, 16, 2, 1>(v, N, c, mc, wm, st);
    case 10: return launch_shape<float, 8, 1, 4>(v, N, c, mc, wm, st);
    case 11: return launch_shape<float, 8, 1, 3>(v, N, c, mc, wm, st);
    case 12: return launch_shape<float, 8, 2, 2>(v, N, c, mc, wm, st);
    case 13: return launch_shape<float, 16, 1, 2>(v, N, c, mc, wm, st);
    default: return cudaErrorInvalidValue;
    }
}
template <>
cudaError_t launch_fused_step<double>(const View<double> &v, int N, const KickCoef<double> &c, int variant,
                                      cudaStream_t st)
{
    if (variant < 0 || variant >= fused_variant_count<double>()) return cudaErrorInvalidValue;
    const int mc = kVariants64[variant].min_chunk;
    const bool wm = kVariants64[variant].wave_model;
    switch (variant) {
    case 0: return launch_shape<double, 16, 1, 1>(v, N, c, mc, wm, st);
    case 1: return launch_shape<double, 8, 1, 2>(v, N, c, mc, wm, st);
    case 2: return launch_shape<double, 8, 2, 1>(v, N, c, mc, wm, st);
    case 3: return launch_shape<double, 8, 1, 2>(v, N, c, mc, wm, st);
    default: return cudaErrorInvalidValue;
    }
}


// ---- diagnostics through the fused tile ----
namespace {
template <typename real, typename IT>
cudaError_t launch_diag_it(const View<real> &v, int N, const DiagArgs &da, cudaStream_t st)
{
    using G = Geo<real, 8, 1>;
    static unsigned long long configured = 0;   // per device; dynamic plus static smem may pass 48 KB
    const unsigned long long dev_bit = 1ULL << device_slot();
    if (!(configured & dev_bit)) {
        const cudaError_t e = cudaFuncSetAttribute(k_fused_diag<real, IT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)G::smem_diag);
        if (e != cudaSuccess) return e;
        configured |= dev_bit;
    }
    int tx, ty, nch, zc;
    fused_diag_grid(N, &tx, &ty, &nch, &zc);
    k_fused_diag<real, IT><<<dim3(tx, ty, nch), 256, G::smem_diag, st>>>(v, N, zc, da);
    return cudaGetLastError();
}
}  // namespace

void fused_diag_grid(int N, int *tx, int *ty, int *nch, int *zc)
{
    *tx = (N + 31) / 32;
    *ty = (N + 7) / 8;
    const int n = choose_chunks(N, (long long)*tx * *ty, 2 * device_sm_count(), 16);   // 2 CTAs / SM
    *zc = (N + n - 1) / n;
    *nch = (N + *zc - 1) / *zc;
}

int fused_diag_ctas(int N)
{
    int tx, ty, nch, zc;
    fused_diag_grid(N, &tx, &ty, &nch, &zc);
    return tx * ty * nch;
}

template <typename real>
cudaError_t launch_fused_diag(const View<real> &v, int N, const DiagArgs &da, cudaStream_t st)
{
    return (long long)N * N * N < (1LL << 31) ? launch_diag_it<real, int>(v, N, da, st)
                                              : launch_diag_it<real, long long>(v, N, da, st);
}
template cudaError_t launch_fused_diag<float>(const View<float> &, int, const DiagArgs &, cudaStream_t);
template cudaError_t launch_fused_diag<double>(const View<double> &, int, const DiagArgs &, cudaStream_t);

// ---- batched step ----
namespace {
struct BatchShape { int ty, rx, minb; };
constexpr BatchShape kBatchShapes[] = { { 8, 1, 4 }, { 16, 1, 2 }, { 8, 2, 2 } };

template <int TY, int RX, int MINB>
cudaError_t launch_batch_shape(const BatchLattice *lat, BatchState *state, int nlat, const int2 *items,
                               const int *nitems, unsigned int *counter, int num_sms, cudaStream_t st, int mode)
{
    using G = Geo<float, TY, RX>;
    static int blocks_per_sm_dev[64] = {};      // per device
    int &blocks_per_sm = blocks_per_sm_dev[device_slot()];
    if (!blocks_per_sm) {
        cudaError_t e = cudaFuncSetAttribute(k_fused_batch<TY, RX, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)G::smem);
        if (e != cudaSuccess) return e;
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_fused_batch<TY, RX, MINB>, 256, G::smem);
        if (e != cudaSuccess) return e;
        blocks_per_sm = b < 1 ? 1 : b;
    }
    k_fused_batch<TY, RX, MINB><<<num_sms * blocks_per_sm, 256, G::smem, st>>>(lat, state, items, nitems, counter,
                                                                              mode);
    k_batch_advance<<<1, 256, 0, st>>>(lat, state, nlat, counter, mode);
    return cudaGetLastError();
}
}  // namespace

int batch_shape_count() { return (int)(sizeof(kBatchShapes) / sizeof(kBatchShapes[0])); }

// Per-shape one-time set-up (shared-memory attribute, occupancy) done outside
// any stream capture: a launch of an empty work list.
cudaError_t batch_shape_prepare(int shape, int num_sms, cudaStream_t st, bool two)
{
    // a few bytes of device scratch per device, kept for the life of the process
    static BatchState *d_dummy_dev[64] = {};
    static int *d_zero_dev[64] = {};
    static unsigned int *d_cnt_dev[64] = {};
    const int ds = device_slot();
    BatchState *&d_dummy = d_dummy_dev[ds];
    int *&d_zero = d_zero_dev[ds];
    unsigned int *&d_cnt = d_cnt_dev[ds];
    if (!d_dummy) {
        BatchState *a = nullptr;
        int *z = nullptr;
        unsigned int *c = nullptr;
        cudaError_t e = cudaMalloc(&a, sizeof(BatchState));
        if (e == cudaSuccess) e = cudaMalloc(&z, sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&c, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemsetAsync(z, 0, sizeof(int), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c, 0, sizeof(unsigned int), st);
        if (e != cudaSuccess) {
            cudaFree(a); cudaFree(z); cudaFree(c);
            return e;
        }
        d_dummy = a; d_zero = z; d_cnt = c;
    }
    // nlat = 0: the advance kernel touches no lattice; nitems = 0: no work
    if (two) return launch_fused2_batch(shape, nullptr, d_dummy, 0, nullptr, d_zero, d_cnt, num_sms, st);
    return launch_fused_batch(shape, nullptr, d_dummy, 0, nullptr, d_zero, d_cnt, num_sms, st);
}

void batch_tiles(int shape, int N, int *tx, int *ty)
{
    const BatchShape &b = kBatchShapes[shape];
    *tx = (N + 32 * b.rx - 1) / (32 * b.rx);
    *ty = (N + b.ty - 1) / b.ty;
}

bool batch_shape_ok(int shape, int N) { return kBatchShapes[shape].rx == 1 || N % 2 == 0; }

cudaError_t launch_fused_batch(int shape, const BatchLattice *lat, BatchState *state, int nlat, const int2 *items,
                               const int *nitems, unsigned int *counter, int num_sms, cudaStream_t st,
                               int mode)
{
    switch (shape) {
    case 0: return launch_batch_shape<8, 1, 4>(lat, state, nlat, items, nitems, counter, num_sms, st, mode);
    case 1: return launch_batch_shape<16, 1, 2>(lat, state, nlat, items, nitems, counter, num_sms, st, mode);
    case 2: return launch_batch_shape<8, 2, 2>(lat, state, nlat, items, nitems, counter, num_sms, st, mode);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ah
