// k_fused2.cu -- two leapfrog steps per pass over the lattice (temporal
// blocking of Eqs. up_pi, up_E, up_phi, up_A of arXiv:1809.00995), FP32.
//
// One step reads and writes the 10-real state once (80 B per site-update);
// this kernel advances the state by two steps per read and write, so 40 B per
// site-update cross DRAM.  A CTA of 32 x TY threads owns the region R1 of
// 32 x TY sites of the XY plane and marches a chunk of z planes:
//
//   first step  (coefficients of step n) on all of R1, from the state n that
//               the CTA reads with a one-site halo ring (the tile walk of the
//               single-step kernel: link exponentials and phi of two planes
//               and the plaquette sines of one in shared memory, the plane
//               below in registers);
//   second step (coefficients of step n + 1) on the inner (32 - 2) x (TY - 2)
//               sites, one plane behind, from the first step's phi^{n+1} and
//               U^{n+1} = e^{i theta^{n+1}} of R1 kept in a two-plane ring of
//               shared memory; Pi, E and theta of step n + 1 of the own site
//               stay in registers.
//
// The second step needs the first one on the ring around its sites, so each
// CTA recomputes the first step on the sites that the neighbouring CTAs write.
// Those CTAs may already have stored their state n + 2 there, so nothing is
// updated in place: Pi and E are read from one buffer set and written to
// another, like phi and theta.  Three barriers per plane serve both steps.
// Each step evaluates the single-step kernel's formulas in the same order; the
// results agree with single steps to FP32 rounding (the compiler is free to
// fuse multiply-adds differently in the two kernels).
//
// k_fused2_diag is the same pass with the whole-lattice diagnostics of Sec. 2
// (energy sums, Gauss residual, plaquette windings) of the state n folded into
// the first step, which reads exactly that state: phi^n, theta^n and Pi, E at
// n - 1/2, none of which the pass overwrites.  Each CTA accumulates them on the
// sites it writes, so every site is counted once, and the diagnostics cost no
// read of the state of their own.
#include "ah_internal.cuh"
#include "diag_common.cuh"
#include "sincos32.cuh"
#include "fused_common.cuh"

namespace ah {
namespace {

template <int TY>
struct Geo2 {
    static constexpr int TX = 32, NT = 32 * TY;
    static constexpr int OX = TX - 2, OY = TY - 2;               // sites the second step writes
    static constexpr int EX = TX + 2, EY = TY + 2, NE = EX * EY;  // R1 plus the halo ring
    static constexpr int NHALO = 2 * EX + 2 * TY;
    static constexpr int PX = TX + 1, NP = PX * (TY + 1);         // R1 plus its low halos
    static constexpr int NPHALO = PX + TY;
    // [2 planes][3 dirs][NE] U, [2][NE] phi, [3][NP] sin Xi (first step);
    // [2 planes][4][NT] U'_1, U'_2, U'_3, phi' and [3][NT] sin Xi' (second step)
    static constexpr size_t off_P = sizeof(cpx<float>) * 8 * NE;
    static constexpr size_t off_V = (off_P + sizeof(float) * 3 * NP + 15) / 16 * 16;
    static constexpr size_t off_Q = off_V + sizeof(cpx<float>) * 8 * NT;
    static constexpr size_t smem = off_Q + sizeof(float) * 3 * NT;
    // k_fused2_diag: [2][NT] scaled edge products (d = 1, 3) and [NT] E_2 of
    // plane q, read by the neighbouring row
    static constexpr size_t off_D = (smem + 15) / 16 * 16;
    static constexpr size_t smem_diag = off_D + sizeof(C2<float>) * 2 * NT + sizeof(float) * NT;
    static_assert(NHALO <= NT && NPHALO <= NT, "tile shape");
};

__device__ __forceinline__ cpx<float> cj(cpx<float> a) { return { a.r, -a.i }; }

// Per-site diagnostic coefficients of step n in FP32 (the Gauss coefficients
// as double-float pairs), converted on the host from DiagCoef.
struct Diag2Coef {
    float inv_dx2, v_coef, eel_coef, b_coef, sigma2;
    DF g_div, g_phi;
};
struct Diag2Args {
    Diag2Coef c;
    DiagPartial *partials;     // one per CTA
    DiagList list;             // plaquettes left to the FP64 path
};

// Scaled edge product conj(phi^a) U phi^b of a winding (Eq. 9).
__device__ __forceinline__ C2<float> edge2(cpx<float> fa, cpx<float> u, cpx<float> fb)
{
    C2<float> z = cmul(conj(C2<float>{ fa.r, fa.i }), cmul(C2<float>{ u.r, u.i }, C2<float>{ fb.r, fb.i }));
    unit_scale_or_nan(z);
    return z;
}

// One thread's share of the whole-lattice diagnostics: the same per-site
// terms, in the same order and precision, as the diagnostics pass of the
// single-step tile walk (k_fused.cu, MODE_DIAG), so the two agree to FP32
// rounding and the windings exactly.
struct Diag2Acc {
    // ah_obs.sums 3..13: K, |D phi|^2, V, E_el, B, K V, |D phi|^2 V, K L,
    // |D phi|^2 L, p L, rho L (compensated; the sums of L, rho, p follow)
    Acc<float> s[11];
    Acc<float> g2, gs2;          // G^2 and scale^2 of the Gauss residual, times 2^60
    DF gmax{ 0.f, 0.f };         // max |G|
    float tmax = 0.f;            // max |theta|
    int ic[kNumInt] = { 0, 0, 0, 0, 0, 0, 0, 0 };

    // f0 = phi^x, w_d = U_d^x phi^{x+d}, E^{x - d}_d in e1b, e2b, e3b,
    // bcos = sum over the three plaquettes at x of 1 - cos Xi
    __device__ __forceinline__ void site(const Diag2Coef &c, float pr, float pim, cpx<float> f0, cpx<float> w1,
                                         cpx<float> w2, cpx<float> w3, float e1, float e2, float e3, float e1b,
                                         float e2b, float e3b, float bcos, float t1, float t2, float t3)
    {
        const float K = pr * pr + pim * pim;
        const float d1r = w1.r - f0.r, d1i = w1.i - f0.i, d2r = w2.r - f0.r, d2i = w2.i - f0.i;
        const float d3r = w3.r - f0.r, d3i = w3.i - f0.i;
        const float G2 = (d1r * d1r + d1i * d1i + d2r * d2r + d2i * d2i + d3r * d3r + d3i * d3i) * c.inv_dx2;
        const float m2 = f0.r * f0.r + f0.i * f0.i - c.sigma2;
        const float V = c.v_coef * m2 * m2;
        const float Eel = c.eel_coef * (e1 * e1 + e2 * e2 + e3 * e3);
        const float B = c.b_coef * bcos;
        const float L = K - G2 - V + Eel - B;
        const float rho = K + G2 + V + Eel + B;
        const float pp = K - G2 * (1.0f / 3.0f) - V + (Eel + B) * (1.0f / 3.0f);
        s[0].add(K); s[1].add(G2);
        s[2].add(V); s[3].add(Eel); s[4].add(B); s[5].add(K * V); s[6].add(G2 * V);
        s[7].add(K * L); s[8].add(G2 * L); s[9].add(pp * L); s[10].add(rho * L);
        tmax = fmaxf(tmax, fmaxf(fabsf(t1), fmaxf(fabsf(t2), fabsf(t3))));
        ic[7] += !(isfinite(L) && isfinite(rho) && isfinite(pp));
        // Gauss residual in double-float arithmetic
        const DF div = df_add(df_add(two_sum(e1, -e1b), two_sum(e2, -e2b)), two_sum(e3, -e3b));
        const DF a = two_prod(f0.r, pim), b = two_prod(f0.i, pr);
        const DF g1 = df_mul(c.g_div, div), gq = df_mul(c.g_phi, df_add(a, { -b.h, -b.l }));
        DF Gs = df_add(g1, gq);
        if (Gs.h < 0.f) Gs = { -Gs.h, -Gs.l };
        const float gs = fabsf(g1.h) + fabsf(gq.h);
        const float sg = Gs.h * 0x1p30f, ss = gs * 0x1p30f;
        g2.add(sg * sg);
        gs2.add(ss * ss);
        if (Gs.h > gmax.h || (Gs.h == gmax.h && Gs.l > gmax.l)) gmax = Gs;
    }
    // winding w of plaquette orientation q at site index `site`, or INT_MIN:
    // the plaquette goes to the list for the FP64 path
    __device__ __forceinline__ void wind(int q, int w, unsigned long long site, const DiagList &list)
    {
        if (w == INT_MIN) {
            const unsigned long long k = atomicAdd(list.count, 1ULL);
            if (k < (unsigned long long)list.capacity) list.items[k] = site * 4ULL + q;
        } else {
            ic[q] += w < 0 ? -w : w;
            ic[3 + q] += w;
            ic[6] += w != 0;
        }
    }
    template <int NT>
    __device__ __forceinline__ void flush(DiagPartial *out)
    {
        double accd[kNumSums];
#pragma unroll
        for (int k = 3; k < 14; ++k) accd[k] = s[k - 3].value();
        accd[0] = accd[3] - accd[4] - accd[5] + accd[6] - accd[7];
        accd[1] = accd[3] + accd[4] + accd[5] + accd[6] + accd[7];
        accd[2] = accd[3] - accd[4] * (1.0 / 3.0) - accd[5] + (accd[6] + accd[7]) * (1.0 / 3.0);
        accd[14] = g2.value() * 0x1p-60;
        accd[15] = gs2.value() * 0x1p-60;
        double mx[kNumMax] = { (double)gmax.h + (double)gmax.l, (double)tmax };
        long long il[kNumInt];
#pragma unroll
        for (int k = 0; k < kNumInt; ++k) il[k] = ic[k];
        block_reduce<NT>(accd, mx, il, out);
    }
};

// WEAK: the link exponentials by sincos_link3_weak (a kernel for states whose
// link phases are mostly within [-2^-6, 2^-6]; correct for any state).
template <int TY, int MINB, typename IT, bool WEAK = false>
__global__ void __launch_bounds__(32 * TY, MINB)
    k_fused2(View2<float> v, int N, int zc, KickCoef<float> c1, KickCoef<float> c2)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool AH2_DIAG = false;
    constexpr bool AH2_WEAK = WEAK;
    [[maybe_unused]] const Diag2Args da{};
#define AH2_BX (int)blockIdx.x
#define AH2_BY (int)blockIdx.y
#define AH2_BZ (int)blockIdx.z
#define AH2_SKIP_TILE return
#include "k_fused2_tile.cuh"
#undef AH2_BX
#undef AH2_BY
#undef AH2_BZ
#undef AH2_SKIP_TILE
}

// The two-step pass with the diagnostics of the state n (tile 32 x 8, two
// CTAs per SM: the accumulators take the register budget of a third); one
// DiagPartial per CTA.
template <typename IT>
__global__ void __launch_bounds__(256, 2)
    k_fused2_diag(View2<float> v, int N, int zc, KickCoef<float> c1, KickCoef<float> c2, Diag2Args da)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TY = 8;
    constexpr bool AH2_DIAG = true;
    constexpr bool AH2_WEAK = false;
#define AH2_BX (int)blockIdx.x
#define AH2_BY (int)blockIdx.y
#define AH2_BZ (int)blockIdx.z
#define AH2_SKIP_TILE return
#include "k_fused2_tile.cuh"
#undef AH2_BX
#undef AH2_BY
#undef AH2_BZ
#undef AH2_SKIP_TILE
}

// Batched two-step pass: persistent CTAs take (lattice, tile) work items of the
// two-step geometry from a shared counter and advance by two steps every
// lattice stepped in pairs with at least two steps to go to its next stop (its
// next diagnostic point or its end).  A lattice's phi/theta ping-pong index (cur) and Pi/E set
// (pe) select the buffers read; the other ones are written.
template <int TY, int MINB>
__global__ void __launch_bounds__(32 * TY, MINB)
    k_fused2_batch(const BatchLattice *lat, BatchState *state, const int2 *items, const int *nitems,
                   unsigned int *counter)
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
        if (!batch_takes_pair(B, step)) continue;
        // the item's pointers and coefficients in shared memory (in registers
        // they would spill at the 80-register budget of 3 CTAs per SM)
        __shared__ View2<float> sv;
        __shared__ KickCoef<float> sc[2];
        if (threadIdx.x == 0) {
            const int cur = state[L].cur, o = 1 - cur, pe = state[L].pe;
            float *const *q = B.q[pe];
            float *const *oq = B.q[1 - pe];
            View2<float> &w = sv;
            w.phr = B.F.phr[cur]; w.phi = B.F.phi[cur];
            w.th1 = B.F.th[cur][0]; w.th2 = B.F.th[cur][1]; w.th3 = B.F.th[cur][2];
            w.pir = q[0]; w.pii = q[1]; w.e1 = q[2]; w.e2 = q[3]; w.e3 = q[4];
            w.ophr = B.F.phr[o]; w.ophi = B.F.phi[o];
            w.oth1 = B.F.th[o][0]; w.oth2 = B.F.th[o][1]; w.oth3 = B.F.th[o][2];
            w.opir = oq[0]; w.opii = oq[1]; w.oe1 = oq[2]; w.oe2 = oq[3]; w.oe3 = oq[4];
            sc[0] = B.coefs[step];
            sc[1] = B.coefs[step + 1];
        }
        __syncthreads();
        const View2<float> &v = sv;
        const KickCoef<float> &c1 = sc[0], &c2 = sc[1];
        const int bx = local % B.tiles2_x, by = (local / B.tiles2_x) % B.tiles2_y;
        const int bz = local / (B.tiles2_x * B.tiles2_y);
        const int N = B.N, zc = B.zc2;
        using IT = int;
        constexpr bool AH2_DIAG = false;
        constexpr bool AH2_WEAK = false;
        [[maybe_unused]] const Diag2Args da{};
#define AH2_BX bx
#define AH2_BY by
#define AH2_BZ bz
#define AH2_SKIP_TILE continue
#include "k_fused2_tile.cuh"
#undef AH2_BX
#undef AH2_BY
#undef AH2_BZ
#undef AH2_SKIP_TILE
        __syncthreads();
    }
}

// After a batched two-step pass: every lattice that took part moves on by two
// steps, swaps its phi/theta buffers and its Pi/E set; the work counter is reset.
__global__ void k_batch_advance2(const BatchLattice *lat, BatchState *state, int nlat, unsigned int *counter)
{
    for (int L = threadIdx.x; L < nlat; L += blockDim.x) {
        if (batch_takes_pair(lat[L], state[L].step)) {
            state[L].step += 2;
            state[L].cur ^= 1;
            state[L].pe ^= 1;
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// Shapes: tile height TY (CTA of 32 TY threads; the second step writes
// 30 x (TY - 2) sites, so the first step computes 32 TY / (30 (TY - 2)) sites
// per written site) and the resident CTAs per SM the register allocation
// must allow.
struct Shape2 { int ty, minb; const char *name; };
constexpr Shape2 kShapes2[] = { { 8, 2, "two_ty8_b2" }, { 8, 3, "two_ty8_b3" }, { 16, 1, "two_ty16_b1" },
                                { 12, 2, "two_ty12_b2" } };

// WEAK (32-bit site indices only; the caller checks fused2_weak_ok)
template <int TY, int MINB, bool WEAK = false>
cudaError_t launch_shape2(const View2<float> &v, int N, const KickCoef<float> &c1, const KickCoef<float> &c2,
                          cudaStream_t st)
{
    using G = Geo2<TY>;
    const bool idx32 = (long long)N * N * N < (1LL << 31);
    static unsigned long long configured = 0;   // per device, once per instantiation
    const unsigned long long dev_bit = 1ULL << device_slot();
    if (!(configured & dev_bit)) {
        cudaError_t err = cudaFuncSetAttribute(k_fused2<TY, MINB, int, WEAK>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem);
        if (err == cudaSuccess && !WEAK)
            err = cudaFuncSetAttribute(k_fused2<TY, MINB, long long>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)G::smem);
        if (err != cudaSuccess) return err;
        configured |= dev_bit;
    }
    const int tx = (N + G::OX - 1) / G::OX, ty = (N + G::OY - 1) / G::OY;
    // each chunk also runs the first step on the planes below and above it
    int nch = choose_chunks(N, (long long)tx * ty, device_sm_count() * MINB, 16, 4);
    const int zc = (N + nch - 1) / nch;
    nch = (N + zc - 1) / zc;
    if constexpr (WEAK) {
        if (!idx32) return cudaErrorInvalidValue;
        k_fused2<TY, MINB, int, true><<<dim3(tx, ty, nch), G::NT, G::smem, st>>>(v, N, zc, c1, c2);
    } else if (idx32) {
        k_fused2<TY, MINB, int><<<dim3(tx, ty, nch), G::NT, G::smem, st>>>(v, N, zc, c1, c2);
    } else {
        k_fused2<TY, MINB, long long><<<dim3(tx, ty, nch), G::NT, G::smem, st>>>(v, N, zc, c1, c2);
    }
    return cudaGetLastError();
}

}  // namespace

bool fused2_weak_ok(int variant, int N) { return variant == 1 && (long long)N * N * N < (1LL << 31); }

cudaError_t launch_fused2_step(const View2<float> &v, int N, const KickCoef<float> &c1, const KickCoef<float> &c2,
                               int variant, cudaStream_t st, bool weak)
{
    if (N < 4) return cudaErrorInvalidValue;
    if (weak) return fused2_weak_ok(variant, N) ? launch_shape2<8, 3, true>(v, N, c1, c2, st) : cudaErrorInvalidValue;
    switch (variant) {
    case 0: return launch_shape2<8, 2>(v, N, c1, c2, st);
    case 1: return launch_shape2<8, 3>(v, N, c1, c2, st);
    case 2: return launch_shape2<16, 1>(v, N, c1, c2, st);
    case 3: return launch_shape2<12, 2>(v, N, c1, c2, st);
    default: return cudaErrorInvalidValue;
    }
}

// ---- batched two-step pass ----
namespace {
struct Batch2Shape { int ty, minb; };
constexpr Batch2Shape kBatch2Shapes[] = { { 8, 3 }, { 12, 2 } };

template <int TY, int MINB>
cudaError_t launch_batch2_shape(const BatchLattice *lat, BatchState *state, int nlat, const int2 *items,
                                const int *nitems, unsigned int *counter, int num_sms, cudaStream_t st)
{
    using G = Geo2<TY>;
    static int blocks_per_sm_dev[64] = {};      // per device
    int &blocks_per_sm = blocks_per_sm_dev[device_slot()];
    if (!blocks_per_sm) {
        cudaError_t e = cudaFuncSetAttribute(k_fused2_batch<TY, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)G::smem);
        if (e != cudaSuccess) return e;
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_fused2_batch<TY, MINB>, G::NT, G::smem);
        if (e != cudaSuccess) return e;
        blocks_per_sm = b < 1 ? 1 : b;
    }
    k_fused2_batch<TY, MINB><<<num_sms * blocks_per_sm, G::NT, G::smem, st>>>(lat, state, items, nitems, counter);
    k_batch_advance2<<<1, 256, 0, st>>>(lat, state, nlat, counter);
    return cudaGetLastError();
}
}  // namespace

int batch2_shape_count() { return (int)(sizeof(kBatch2Shapes) / sizeof(kBatch2Shapes[0])); }

void batch2_tiles(int shape, int N, int *tx, int *ty)
{
    const int oy = kBatch2Shapes[shape].ty - 2;
    *tx = (N + 29) / 30;
    *ty = (N + oy - 1) / oy;
}

cudaError_t launch_fused2_batch(int shape, const BatchLattice *lat, BatchState *state, int nlat, const int2 *items,
                                const int *nitems, unsigned int *counter, int num_sms, cudaStream_t st)
{
    switch (shape) {
    case 0: return launch_batch2_shape<8, 3>(lat, state, nlat, items, nitems, counter, num_sms, st);
    case 1: return launch_batch2_shape<12, 2>(lat, state, nlat, items, nitems, counter, num_sms, st);
    default: return cudaErrorInvalidValue;
    }
}

// ---- two-step pass with the diagnostics of the state n ----
void fused2_diag_grid(int N, int *tx, int *ty, int *nch, int *zc)
{
    using G = Geo2<8>;
    *tx = (N + G::OX - 1) / G::OX;
    *ty = (N + G::OY - 1) / G::OY;
    const int n = choose_chunks(N, (long long)*tx * *ty, 2 * device_sm_count(), 16, 4);   // 2 CTAs / SM
    *zc = (N + n - 1) / n;
    *nch = (N + *zc - 1) / *zc;
}

int fused2_diag_ctas(int N)
{
    int tx, ty, nch, zc;
    fused2_diag_grid(N, &tx, &ty, &nch, &zc);
    return tx * ty * nch;
}

cudaError_t launch_fused2_diag(const View2<float> &v, int N, const KickCoef<float> &c1, const KickCoef<float> &c2,
                               const DiagArgs &da, int capacity, cudaStream_t st)
{
    using G = Geo2<8>;
    if (N < 4) return cudaErrorInvalidValue;
    int tx, ty, nch, zc;
    fused2_diag_grid(N, &tx, &ty, &nch, &zc);
    if ((long long)tx * ty * nch > capacity) return cudaErrorInvalidValue;
    static unsigned long long configured = 0;   // per device
    const unsigned long long dev_bit = 1ULL << device_slot();
    if (!(configured & dev_bit)) {
        cudaError_t err = cudaFuncSetAttribute(k_fused2_diag<int>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)G::smem_diag);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(k_fused2_diag<long long>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)G::smem_diag);
        if (err != cudaSuccess) return err;
        configured |= dev_bit;
    }
    Diag2Args a;
    a.c.inv_dx2 = (float)da.dc.inv_dx2;
    a.c.v_coef = (float)da.dc.v_coef;
    a.c.eel_coef = (float)da.dc.eel_coef;
    a.c.b_coef = (float)da.dc.b_coef;
    a.c.sigma2 = (float)da.dc.sigma2;
    a.c.g_div = df_from(da.dc.g_div);
    a.c.g_phi = df_from(da.dc.g_phi);
    a.partials = da.partials;
    a.list = da.list;
    const dim3 grid(tx, ty, nch);
    if ((long long)N * N * N < (1LL << 31)) k_fused2_diag<int><<<grid, G::NT, G::smem_diag, st>>>(v, N, zc, c1, c2, a);
    else k_fused2_diag<long long><<<grid, G::NT, G::smem_diag, st>>>(v, N, zc, c1, c2, a);
    return cudaGetLastError();
}

int fused2_variant_count() { return (int)(sizeof(kShapes2) / sizeof(kShapes2[0])); }
const char *fused2_variant_name(int k) { return kShapes2[k].name; }
// two_ty8_b3: the fastest at 512^3 and 1024^3 on GB300 (80 registers, 24 warps
// per SM; the 64-register 8 x 4 shape spills and is a third slower)
int fused2_default_variant() { return 1; }

}  // namespace ah
