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
#include "ah_internal.cuh"
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
    static_assert(NHALO <= NT && NPHALO <= NT, "tile shape");
};

__device__ __forceinline__ cpx<float> cj(cpx<float> a) { return { a.r, -a.i }; }

template <int TY, int MINB, typename IT>
__global__ void __launch_bounds__(32 * TY, MINB)
    k_fused2(View2<float> v, int N, int zc, KickCoef<float> c1, KickCoef<float> c2)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
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

template <int TY, int MINB>
cudaError_t launch_shape2(const View2<float> &v, int N, const KickCoef<float> &c1, const KickCoef<float> &c2,
                          cudaStream_t st)
{
    using G = Geo2<TY>;
    const bool idx32 = (long long)N * N * N < (1LL << 31);
    static unsigned long long configured = 0;   // per device, once per instantiation
    const unsigned long long dev_bit = 1ULL << device_slot();
    if (!(configured & dev_bit)) {
        cudaError_t err = cudaFuncSetAttribute(k_fused2<TY, MINB, int>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)G::smem);
        if (err == cudaSuccess)
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
    if (idx32) k_fused2<TY, MINB, int><<<dim3(tx, ty, nch), G::NT, G::smem, st>>>(v, N, zc, c1, c2);
    else k_fused2<TY, MINB, long long><<<dim3(tx, ty, nch), G::NT, G::smem, st>>>(v, N, zc, c1, c2);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fused2_step(const View2<float> &v, int N, const KickCoef<float> &c1, const KickCoef<float> &c2,
                               int variant, cudaStream_t st)
{
    if (N < 4) return cudaErrorInvalidValue;
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

int fused2_variant_count() { return (int)(sizeof(kShapes2) / sizeof(kShapes2[0])); }
const char *fused2_variant_name(int k) { return kShapes2[k].name; }
// two_ty8_b3: the fastest at 512^3 and 1024^3 on GB300 (80 registers, 24 warps
// per SM; the 64-register 8 x 4 shape spills and is a third slower)
int fused2_default_variant() { return 1; }

}  // namespace ah
