// k_tma.cu -- fused leapfrog step fed by the Tensor Memory Accelerator (FP32).
//
// Same update as k_fused.cu (Eqs. up_pi, up_E, up_phi, up_A of
// arXiv:1809.00995: both kicks and both drifts of one step in one z-marching
// kernel, link exponentials computed once per site, plaquette sines once per
// plaquette, phi/theta ping-pong), with the memory pipeline rebuilt for sm_103a:
//
//  * Tile 32 x 8 sites, one site per thread (256 threads).  The interior of
//    every plane -- phi, theta (5 fields) and Pi, E (5 fields) -- arrives by TMA
//    3D tensor-map box copies (cp.async.bulk.tensor.3d, box 32 x 8 x 1) issued
//    by one thread into shared-memory rings (4 stages for phi/theta, 3 for
//    Pi/E) several planes ahead of use; each stage completes on an mbarrier
//    (expected transaction bytes).  No register holds prefetched data.
//  * The one-site halo ring (periodic wrap in the index arithmetic) is read
//    with plain loads one plane ahead, and its link exponentials are split into
//    202 single-component tasks spread over the threads, so no warp carries
//    more than one extra sincos per plane.
//  * U = e^{i theta} and phi live in three-plane rings (planes z, z+1, z+2),
//    so each plane needs two block barriers: plaquettes of plane z, then the
//    update of plane z together with the links of plane z+2.
//
// Requires N % 32 == 0 (whole tiles; TMA boxes never cross the lattice edge).
// Every mbarrier wait is bounded (wait_limit clock cycles, 2^32 = about 2 s by
// default); on timeout the CTA records an error in *err, stops issuing copies,
// waits (each wait again bounded, 2^24 cycles) for the last copy it issued
// into each ring stage and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "ah_internal.cuh"
#include "sincos32.cuh"

namespace ah {
namespace {

constexpr int TX = 32, TY = 8, NT = 256;
constexpr int EX = TX + 2, EY = TY + 2, NE = EX * EY;     // extended tile (one-site halo)
constexpr int PX = TX + 1, PY = TY + 1, NP = PX * PY;     // plaquette region: tile + low halos
constexpr int FS = 4, QS = 3;                             // ring depths (phi/theta, Pi/E)
constexpr int BOX = TX * TY;                              // floats per box
constexpr int N_UHALO = 202, N_PHALO_PHI = 80, N_PHALO_P = 80;

struct cpx { float r, i; };
__device__ __forceinline__ cpx mul(cpx a, cpx b) { return { a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r }; }
__device__ __forceinline__ float plaq(cpx a, cpx b, cpx c, cpx d)
{
    const cpx ab = mul(a, b), cd = mul(c, d);
    return ab.i * cd.r - ab.r * cd.i;
}
__device__ __forceinline__ int wrapm(int a, int N) { a %= N; return a < 0 ? a + N : a; }

// ---- PTX wrappers (mbarrier, TMA) ----
__device__ __forceinline__ uint32_t sptr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sptr(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sptr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(sptr(b)), "r"(parity) : "memory");
    return ok != 0;
}
// Wait for phase `parity` of barrier b; false after about 2^32 cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, long long limit = 1LL << 32)
{
    if (mbar_try(b, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(b, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
__device__ __forceinline__ void tma3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];"
                 ::"r"(sptr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(sptr(bar))
                 : "memory");
}

struct Smem {
    float F[FS][5][BOX];      // phi.re, phi.im, th1, th2, th3 of one plane (interior)
    float Q[QS][5][BOX];      // Pi.re, Pi.im, E1, E2, E3 of one plane (interior)
    cpx U[3][3][NE];          // links of planes z, z+1, z+2 (ring), extended tile
    cpx Ph[3][NE];            // phi of the same planes, extended tile
    float P[3][NP];           // sin Xi_12, _13, _23 of plane z, tile + low halos
    uint64_t fbar[FS], qbar[QS];
    int err;
};

template <int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_fused_tma(const __grid_constant__ TmaMaps maps, View<float> v, int N, int zc, KickCoef<float> c, int *err,
            long long wait_limit, int drop_q)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int tid = threadIdx.x, lx = tid & 31, wy = tid >> 5;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * zc;
    if (z0 >= N) return;
    const int nz = min(zc, N - z0);          // planes updated by this CTA
    const int nF = nz + 2;                   // link planes z0-1 .. z0+nz
    const long long NN = (long long)N * N;
    const int e_own = (wy + 1) * EX + lx + 1, p_own = (wy + 1) * PX + lx + 1;
    const int off_own = (x0 + lx) + N * (y0 + wy);

    // halo link task of this thread: extended-tile slot, component, in-plane offset
    int hu_e = -1, hu_d = 0, hu_off = 0;
    if (tid < N_UHALO) {
        int ex, ey, d, t = tid;
        if (t < 24) { ex = 0; ey = 1 + t / 3; d = t % 3; }
        else if (t == 24) { ex = 0; ey = TY + 1; d = 0; }
        else if (t < 41) { t -= 25; ex = EX - 1; ey = 1 + t / 2; d = 1 + t % 2; }
        else if (t < 137) { t -= 41; ex = 1 + t / 3; ey = 0; d = t % 3; }
        else if (t == 137) { ex = EX - 1; ey = 0; d = 1; }
        else { t -= 138; ex = 1 + t / 2; ey = TY + 1; d = 2 * (t % 2); }
        hu_e = ey * EX + ex;
        hu_d = d;
        hu_off = wrapm(x0 + ex - 1, N) + N * wrapm(y0 + ey - 1, N);
    }
    // halo phi task (Laplacian neighbours): threads 255 down to 176
    int hp_e = -1, hp_off = 0;
    if (tid >= NT - N_PHALO_PHI) {
        const int p = NT - 1 - tid;
        int ex, ey;
        if (p < 8) { ex = 0; ey = 1 + p; }
        else if (p < 16) { ex = EX - 1; ey = 1 + p - 8; }
        else if (p < 48) { ex = 1 + p - 16; ey = 0; }
        else { ex = 1 + p - 48; ey = TY + 1; }
        hp_e = ey * EX + ex;
        hp_off = wrapm(x0 + ex - 1, N) + N * wrapm(y0 + ey - 1, N);
    }
    const float *hu_src = hu_d == 0 ? v.th1 : (hu_d == 1 ? v.th2 : v.th3);

    if (tid == 0) {
        for (int s = 0; s < FS; ++s) mbar_init(&S.fbar[s], 1);
        for (int s = 0; s < QS; ++s) mbar_init(&S.qbar[s], 1);
        S.err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // producer (thread 0): plane index f of the link planes is z0 - 1 + f.
    // f_last / q_last: the last plane whose copy went to each ring stage (-1:
    // none), so that an early exit waits exactly for the copies in flight.
    int f_last[FS], q_last[QS];
    for (int s = 0; s < FS; ++s) f_last[s] = -1;
    for (int s = 0; s < QS; ++s) q_last[s] = -1;
    auto issue_F = [&](int f) {
        if (f >= nF) return;
        const int s = f % FS, z = wrapm(z0 - 1 + f, N);
        mbar_arrive_tx(&S.fbar[s], 5 * BOX * 4);
        for (int k = 0; k < 5; ++k) tma3d(S.F[s][k], &maps.f[k], &S.fbar[s], x0, y0, z);
        f_last[s] = f;
    };
    // drop_q (fault injection for tests, -1 otherwise): the copy of Pi/E plane
    // drop_q is never issued, so the wait for it can only give up
    auto issue_Q = [&](int q) {
        if (q >= nz || q == drop_q) return;
        const int s = q % QS, z = z0 + q;
        mbar_arrive_tx(&S.qbar[s], 5 * BOX * 4);
        for (int k = 0; k < 5; ++k) tma3d(S.Q[s][k], &maps.q[k], &S.qbar[s], x0, y0, z);
        q_last[s] = q;
    };
    if (tid == 0) {
        for (int f = 0; f < FS; ++f) issue_F(f);
        for (int q = 0; q < QS; ++q) issue_Q(q);
    }

    // halo values of one link plane, one plane ahead, in registers
    float h_th = 0.f, h_pr = 0.f, h_pi = 0.f;
    auto load_halo = [&](int f) {
        if (f >= nF) return;
        const long long base = (long long)wrapm(z0 - 1 + f, N) * NN;
        if (hu_e >= 0) h_th = hu_src[base + hu_off];
        if (hp_e >= 0) { h_pr = v.phr[base + hp_off]; h_pi = v.phi[base + hp_off]; }
    };

    bool ok = true;     // block-uniform: refreshed from S.err after each barrier
    // A(f): links and phi of link plane f into ring slot f % 3; returns own theta
    auto phase_A = [&](int f, float th_own[3], cpx &ph_own) {
        const int s = f % FS, u = f % 3;
        if (!mbar_wait(&S.fbar[s], (f / FS) & 1, wait_limit)) atomicExch(&S.err, 1);
        const int i = wy * TX + lx;
        ph_own = { S.F[s][0][i], S.F[s][1][i] };
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            th_own[d] = S.F[s][2 + d][i];
            float sn, cs;
            sincos_link(th_own[d], &sn, &cs);
            S.U[u][d][e_own] = { cs, sn };
        }
        S.Ph[u][e_own] = ph_own;
        if (hu_e >= 0) {
            float sn, cs;
            sincos_link(h_th, &sn, &cs);
            S.U[u][hu_d][hu_e] = { cs, sn };
        }
        if (hp_e >= 0) S.Ph[u][hp_e] = { h_pr, h_pi };
    };

    // ---- prologue: link planes z0-1, z0, z0+1 ----
    float th_a[3], th_b[3], th_c[3];     // own theta of planes z, z+1 (and z+2 transient)
    cpx ph_m, ph_x, u3_m;
    float p13_m, p23_m;
    load_halo(0);
    phase_A(0, th_c, ph_m);              // plane z0-1: keep phi own
    load_halo(1);
    __syncthreads();
    ok = S.err == 0;
    if (tid == 0 && ok) { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); issue_F(FS); }
    phase_A(1, th_a, ph_x);              // plane z0
    load_halo(2);
    __syncthreads();
    ok = S.err == 0;
    if (tid == 0 && ok) { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); issue_F(FS + 1); }
    phase_A(2, th_b, ph_x);              // plane z0+1
    load_halo(3);
    __syncthreads();
    ok = S.err == 0;
    if (tid == 0 && ok) { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); issue_F(FS + 2); }
    {
        const cpx *Um = &S.U[0][0][0], *U0 = &S.U[1][0][0];
        u3_m = Um[2 * NE + e_own];
        p13_m = plaq(Um[e_own], Um[2 * NE + e_own + 1], U0[e_own], Um[2 * NE + e_own]);
        p23_m = plaq(Um[NE + e_own], Um[2 * NE + e_own + EX], U0[NE + e_own], Um[2 * NE + e_own]);
    }

    for (int k = 0; k < nz && ok; ++k) {
        const int z = z0 + k;
        const int uc = (k + 1) % 3, un = (k + 2) % 3;     // ring slots of planes z and z+1
        const cpx *U0 = &S.U[uc][0][0], *U1 = &S.U[un][0][0];

        // B: plaquette sines of plane z, own site and low halos
        const float p12 = plaq(U0[e_own], U0[NE + e_own + 1], U0[e_own + EX], U0[NE + e_own]);
        const float p13 = plaq(U0[e_own], U0[2 * NE + e_own + 1], U1[e_own], U0[2 * NE + e_own]);
        const float p23 = plaq(U0[NE + e_own], U0[2 * NE + e_own + EX], U1[NE + e_own], U0[2 * NE + e_own]);
        S.P[0][p_own] = p12;
        S.P[1][p_own] = p13;
        S.P[2][p_own] = p23;
        if (tid < N_PHALO_P) {
            int px, py, which;
            if (tid < 16) { px = 0; py = 1 + tid / 2; which = tid % 2; }             // P12, P13
            else { px = 1 + (tid - 16) / 2; py = 0; which = 2 * ((tid - 16) % 2); }  // P12, P23
            const int e = py * EX + px, p = py * PX + px;
            float val;
            if (which == 0) val = plaq(U0[e], U0[NE + e + 1], U0[e + EX], U0[NE + e]);
            else if (which == 1) val = plaq(U0[e], U0[2 * NE + e + 1], U1[e], U0[2 * NE + e]);
            else val = plaq(U0[NE + e], U0[2 * NE + e + EX], U1[NE + e], U0[2 * NE + e]);
            S.P[which][p] = val;
        }
        __syncthreads();

        // C: kicks and drifts of the own site of plane z
        {
            const int qs = k % QS;
            const bool landed = mbar_wait(&S.qbar[qs], (k / QS) & 1, wait_limit);
            if (!landed) atomicExch(&S.err, 1);
            const int i = wy * TX + lx;
            const float pr = S.Q[qs][0][i], pim = S.Q[qs][1][i];
            const float e1 = S.Q[qs][2][i], e2 = S.Q[qs][3][i], e3 = S.Q[qs][4][i];
            const cpx *F0 = S.Ph[uc];
            const cpx f0 = F0[e_own];
            const cpx u1 = U0[e_own], u2 = U0[NE + e_own], u3 = U0[2 * NE + e_own];
            const cpx u1m = U0[e_own - 1], u2m = U0[NE + e_own - EX];
            const cpx w1 = mul(u1, F0[e_own + 1]), w2 = mul(u2, F0[e_own + EX]), w3 = mul(u3, S.Ph[un][e_own]);
            const cpx b1 = mul({ u1m.r, -u1m.i }, F0[e_own - 1]);
            const cpx b2 = mul({ u2m.r, -u2m.i }, F0[e_own - EX]);
            const cpx b3 = mul({ u3_m.r, -u3_m.i }, ph_m);
            const float lr = (w1.r + b1.r) + (w2.r + b2.r) + (w3.r + b3.r) - 6.0f * f0.r;
            const float li = (w1.i + b1.i) + (w2.i + b2.i) + (w3.i + b3.i) - 6.0f * f0.i;
            const float pot = c.c_pot * (f0.r * f0.r + f0.i * f0.i - c.sigma2);
            const float npr = c.c_damp * pr - pot * f0.r + c.c_lap * lr;
            const float npi = c.c_damp * pim - pot * f0.i + c.c_lap * li;
            const float cu1 = w1.r * f0.i - w1.i * f0.r;
            const float cu2 = w2.r * f0.i - w2.i * f0.r;
            const float cu3 = w3.r * f0.i - w3.i * f0.r;
            const float cl1 = (p12 - S.P[0][p_own - PX]) + (p13 - p13_m);
            const float cl2 = (S.P[0][p_own - 1] - p12) + (p23 - p23_m);
            const float cl3 = (S.P[1][p_own - 1] - p13) + (S.P[2][p_own - PX] - p23);
            const float ne1 = c.c_edamp * e1 + c.c_cur * cu1 - c.c_curl * cl1;
            const float ne2 = c.c_edamp * e2 + c.c_cur * cu2 - c.c_curl * cl2;
            const float ne3 = c.c_edamp * e3 + c.c_cur * cu3 - c.c_curl * cl3;
            if (landed) {
                const long long s = (long long)z * NN + off_own;
                v.pir[s] = npr; v.pii[s] = npi;
                v.e1[s] = ne1; v.e2[s] = ne2; v.e3[s] = ne3;
                v.ophr[s] = f0.r + c.dt * npr;
                v.ophi[s] = f0.i + c.dt * npi;
                float t1 = th_a[0] + c.dt * ne1, t2 = th_a[1] + c.dt * ne2, t3 = th_a[2] + c.dt * ne3;
                if (c.wrap) { t1 = wrap_phase(t1); t2 = wrap_phase(t2); t3 = wrap_phase(t3); }
                v.oth1[s] = t1;
                v.oth2[s] = t2;
                v.oth3[s] = t3;
            }
            ph_m = f0;
            u3_m = u3;
            p13_m = p13;
            p23_m = p23;
        }
        // A: links of plane z+2 (link-plane index k+3) into the slot of plane z-1
        if (k + 3 < nF) {
            phase_A(k + 3, th_c, ph_x);
            load_halo(k + 4);
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) { th_a[d] = th_b[d]; th_b[d] = th_c[d]; }
        __syncthreads();
        ok = S.err == 0;
        if (tid == 0 && ok) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_F(k + 3 + FS);
            issue_Q(k + QS);
        }
    }
    if (!ok) {
        if (tid == 0) {
            atomicExch(err, 1);
            // drain: wait (bounded) for the last copy issued into each stage, so
            // that no copy into this CTA's shared memory is in flight at exit (the
            // wait returns at once for a copy that has landed)
            for (int s = 0; s < FS; ++s)
                if (f_last[s] >= 0) mbar_wait(&S.fbar[s], (f_last[s] / FS) & 1, 1LL << 24);
            for (int s = 0; s < QS; ++s)
                if (q_last[s] >= 0) mbar_wait(&S.qbar[s], (q_last[s] / QS) & 1, 1LL << 24);
        }
        __syncthreads();
    }
}

template <int MINB>
cudaError_t launch_minb(const TmaMaps &maps, const View<float> &v, int N, const KickCoef<float> &c, int *err,
                        int min_chunk, long long wait_limit, int drop_q, cudaStream_t st)
{
    static unsigned long long configured = 0;   // per device
    const unsigned long long dev_bit = 1ULL << device_slot();
    if (!(configured & dev_bit)) {
        cudaError_t e = cudaFuncSetAttribute(k_fused_tma<MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(Smem) + 128));
        if (e != cudaSuccess) return e;
        configured |= dev_bit;
    }
    const int tx = N / TX, ty = N / TY;
    int nch = (int)((152LL * 3 * 4 + (long long)tx * ty - 1) / ((long long)tx * ty));
    nch = max(1, min(nch, N / min_chunk));
    const int zc = (N + nch - 1) / nch;
    nch = (N + zc - 1) / zc;
    k_fused_tma<MINB><<<dim3(tx, ty, nch), NT, sizeof(Smem) + 128, st>>>(maps, v, N, zc, c, err, wait_limit,
                                                                         drop_q);
    return cudaGetLastError();
}

}  // namespace

bool tma_shape_ok(int N) { return N % TX == 0 && N % TY == 0 && N >= TX; }

size_t tma_smem_bytes() { return sizeof(Smem) + 128; }

cudaError_t launch_fused_tma(const TmaMaps &maps, const View<float> &v, int N, const KickCoef<float> &c, int *err,
                             int minb, int min_chunk, long long wait_limit, int drop_q, cudaStream_t st)
{
    if (!tma_shape_ok(N) || wait_limit < 0) return cudaErrorInvalidValue;
    if (minb == 3) return launch_minb<3>(maps, v, N, c, err, min_chunk, wait_limit, drop_q, st);
    return launch_minb<2>(maps, v, N, c, err, min_chunk, wait_limit, drop_q, st);
}

// Tensor maps of one FP32 field array (N^3, x fastest) with box 32 x 8 x 1.
cudaError_t make_tma_map(CUtensorMap *m, const float *base, int N)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[3] = { (cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)N };
    const cuuint64_t strides[2] = { (cuuint64_t)N * 4, (cuuint64_t)N * N * 4 };
    const cuuint32_t box[3] = { TX, TY, 1 };
    const cuuint32_t estr[3] = { 1, 1, 1 };
    CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace ah
