// ah_internal.cuh -- types and kernel launchers shared by the CUDA sources of
// the library (not part of the public ABI; see include/ah.h).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/ah.h"

namespace ah {

// Device pointers of one state: 10 SoA arrays of N^3 reals (x fastest).
// phi and theta have two buffers each (ping-pong for the fused step);
// `cur` selects the buffer holding phi^n, theta^n.
template <typename real>
struct Fields {
    real *phr[2], *phi[2];
    real *th[2][3];
    real *pir, *pii;
    real *el[3];
    // second Pi, E set (Pi_r, Pi_i, E_1, E_2, E_3) for the two-step kernel,
    // which reads one set and writes the other; null unless allocated
    real *spare[5];
};

// View of one state for a kernel: the buffers it reads (and, for the fused
// step, the phi/theta buffers it writes).
template <typename real>
struct View {
    const real *phr, *phi, *th1, *th2, *th3;   // phi^n, theta^n
    real *pir, *pii, *e1, *e2, *e3;              // Pi, E (updated in place)
    real *ophr, *ophi, *oth1, *oth2, *oth3;      // phi^{n+1}, theta^{n+1}
};

// View of the two-step kernel: state n (phi^n, theta^n, Pi and E at n - 1/2)
// is read from one set of buffers and state n + 2 written to another, with
// nothing updated in place (a CTA recomputes the first step on a halo ring
// that neighbouring CTAs overwrite with their second step).
template <typename real>
struct View2 {
    const real *phr, *phi, *th1, *th2, *th3, *pir, *pii, *e1, *e2, *e3;
    real *ophr, *ophi, *oth1, *oth2, *oth3, *opir, *opii, *oe1, *oe2, *oe3;
};

// Coefficients of one leapfrog step n (Eqs. up_pi and up_E), computed in FP64
// on the host from tau_n, tau_n +- dt/2:
//   Pi+ = c_damp Pi- - c_pot (|phi|^2 - sigma^2) phi + c_lap * Laplacian
//   E+  = c_edamp E-  + c_cur * current - c_curl * curl
template <typename real>
struct KickCoef {
    real c_damp, c_pot, c_lap, c_edamp, c_cur, c_curl, dt, sigma2;
    int wrap;    // AH_FLAG_WRAP_THETA: reduce theta to [-pi, pi] after the drift
};

// theta - 2 pi k with k the nearest integer to theta / 2 pi, when |theta| > pi;
// 2 pi is split into its nearest value in the type plus the remainder, so
// the subtraction is accurate to the last bit of the result.
__device__ __forceinline__ float wrap_phase(float t)
{
    if (fabsf(t) > 3.14159265f) {
        const float k = rintf(t * 0.159154943f);
        t = fmaf(-k, 6.28318548f, t);                 // fl(2 pi)
        t = fmaf(-k, -1.74845553e-7f, t);             // 2 pi - fl(2 pi)
    }
    return t;
}
__device__ __forceinline__ double wrap_phase(double t)
{
    if (fabs(t) > 3.141592653589793) {
        const double k = rint(t * 0.15915494309189535);
        t = fma(-k, 6.283185307179586, t);            // fl(2 pi)
        t = fma(-k, 2.4492935982947064e-16, t);       // 2 pi - fl(2 pi)
    }
    return t;
}

// Per-site diagnostic coefficients at step n (FP64 always).
struct DiagCoef {
    double inv_dx2;    // 1 / dx^2
    double v_coef;     // a^2 lambda / 4
    double eel_coef;   // 1 / (2 e^2 a^2 dx^2)
    double b_coef;     // 1 / (e^2 a^2 dx^4)
    double g_div;      // 1 / e_-^2
    double g_phi;      // 2 dx^2 a_-^2
    double sigma2;
};

// Number of FP64 sums and integer counters produced by the diagnostics.
constexpr int kNumSums = 16;     // see ah_obs.sums
constexpr int kNumMax = 2;       // max |G|, max |theta|
constexpr int kNumInt = 8;       // |W| by plane (3), W by plane (3), pierced, nonfinite

// One block's partial results of the diagnostics reduction.
struct DiagPartial {
    double sums[kNumSums];
    double maxv[kNumMax];
    long long ints[kNumInt];
};

struct Box { int x0, y0, z0, nx, ny, nz; };

// Index (0..63) of the current device for per-device one-time set-up (kernel
// attributes are set, and scratch is allocated, once on each device used).
inline int device_slot()
{
    int d = 0;
    cudaGetDevice(&d);
    return d & 63;
}
struct DiagList;

// Plaquettes whose winding the fast diagnostics leave to the FP64 path:
// items[k] = site index * 4 + orientation (0: 12, 1: 13, 2: 23).
struct DiagList {
    unsigned long long *count;
    unsigned long long *items;
    long long capacity;
};

// ---- launchers (each returns the launch's cudaError_t) ----
template <typename real>
cudaError_t launch_init_phase(real *phr, real *phi, int N, uint64_t seed, double sigma,
                              cudaStream_t st);

template <typename real>
cudaError_t launch_gather_window(const Fields<real> &F, int cur, int N, Box b, double *out,
                                 cudaStream_t st);

template <typename real>
cudaError_t launch_scatter_all(const Fields<real> &F, int cur, int N, const double *in,
                               cudaStream_t st);

template <typename real>
cudaError_t launch_plain_step(const View<real> &v, int N, const KickCoef<real> &c,
                              cudaStream_t st);

// Fused step, compile-time shape `variant` in [0, fused_variant_count<real>()).
template <typename real>
cudaError_t launch_fused_step(const View<real> &v, int N, const KickCoef<real> &c, int variant,
                              cudaStream_t st);
template <typename real>
int fused_variant_count();
template <typename real>
const char *fused_variant_name(int variant);
template <typename real>
bool fused_variant_ok(int variant, int N);
template <typename real>
int fused_default_variant();

// Two leapfrog steps (coefficients c1 for step n, c2 for step n + 1) in one
// pass, FP32; shape `variant` in [0, fused2_variant_count()).
// weak: the kernel specialised to weak gauge fields (link phases mostly in
// [-2^-6, 2^-6]; same update, within an ulp per link exponential), available
// where fused2_weak_ok(variant, N).
cudaError_t launch_fused2_step(const View2<float> &v, int N, const KickCoef<float> &c1, const KickCoef<float> &c2,
                               int variant, cudaStream_t st, bool weak = false);
bool fused2_weak_ok(int variant, int N);
// Largest max |theta| at the last whole-lattice observables for which the
// two-step launches take the kernel specialised to weak gauge fields (half the
// bound of its short sine/cosine forms, 2^-6, so the phases may double before
// the next observables; beyond it the kernel stays correct, only slower).
constexpr double kWeakTheta = 0x1p-7;
int fused2_variant_count();
const char *fused2_variant_name(int variant);
int fused2_default_variant();

template <typename real>
cudaError_t launch_diag(const View<real> &v, int N, Box b, const DiagCoef &c,
                        DiagPartial *partials, int nblocks, DiagPartial *result,
                        DiagList list, bool exact, cudaStream_t st);

int diag_grid_blocks(int num_sms);

// If the near-cut list of a pass overflowed (checked on the device), clear the
// winding counters of *result and count every plaquette again in FP64.
template <typename real>
cudaError_t launch_wind_recount_on_overflow(const View<real> &v, int N, DiagList list, DiagPartial *result,
                                            int nblocks, cudaStream_t st);

// Whole-lattice diagnostics through the fused step's tile walk (tile 32 x 8,
// nothing written back): one DiagPartial per CTA of the grid that
// fused_diag_grid gives (fused_diag_ctas of them), near-cut plaquettes
// appended to the list.
struct DiagArgs {
    DiagCoef dc;
    DiagPartial *partials;
    DiagList list;
};
void fused_diag_grid(int N, int *tx, int *ty, int *nch, int *zc);
int fused_diag_ctas(int N);
template <typename real>
cudaError_t launch_fused_diag(const View<real> &v, int N, const DiagArgs &da, cudaStream_t st);
// The whole fast diagnostic: clear the list, launch_fused_diag, sum the
// partials in a fixed order into *result, FP64 windings of the listed
// plaquettes (fix_blocks x 128 threads).  partials holds `capacity` entries;
// cudaErrorInvalidValue (nothing launched) if the N^3 pass needs more
// (fused_diag_ctas(N), which is not monotonic in N).
template <typename real>
cudaError_t launch_diag_whole(const View<real> &v, int N, const DiagCoef &c, DiagPartial *partials,
                              int capacity, DiagPartial *result, DiagList list, int fix_blocks, cudaStream_t st);

// Two leapfrog steps (as launch_fused2_step, tile 32 x 8) that also take the
// whole-lattice diagnostics of the state n they read: one DiagPartial per CTA
// (fused2_diag_ctas(N) of them; cudaErrorInvalidValue, nothing launched, if
// that exceeds `capacity`), near-cut plaquettes appended to da.list, whose
// count the caller clears first.  The state n stays in the buffers v reads.
cudaError_t launch_fused2_diag(const View2<float> &v, int N, const KickCoef<float> &c1, const KickCoef<float> &c2,
                               const DiagArgs &da, int capacity, cudaStream_t st);
int fused2_diag_ctas(int N);
// Sum n partials in a fixed order into *result, then add the FP64 windings of
// the plaquettes listed in `list` (evaluated on the state v; fix_blocks x 128
// threads).
template <typename real>
cudaError_t launch_diag_reduce(const View<real> &v, int N, const DiagPartial *partials, int n, DiagPartial *result,
                               DiagList list, int fix_blocks, cudaStream_t st);

// Host helpers of ah_api.cu shared with other translation units.
KickCoef<float> host_kick_coef32(const ah_config &c, int64_t step);
void host_carve32(Fields<float> &F, void *base, size_t nsites, bool spare = false);
size_t host_state_bytes32(size_t nsites, bool spare = false);
void host_fill_obs(const ah_config &c, int64_t step, int64_t n_sites, const DiagPartial &r, ah_obs *out);
int64_t host_run_steps(const ah_config &c);    // round((tau_end - tau0) / dt)
DiagCoef host_diag_coef(const ah_config &c, int64_t step);
ah_status host_validate(const ah_config &c);
ah_status host_fail(ah_status st, const char *msg);

// Batched fused step (FP32): one descriptor per lattice, work items (lattice,
// tile index), device-side step counters.  q[0] = { F.pir, F.pii, F.el[0..2] };
// q[1] = F.spare, the second Pi/E set of the two-step pass (null unless the
// batch runs two steps per launch).
struct BatchLattice {
    Fields<float> F;
    float *q[2][5];
    int N, zc, tiles_x, tiles_y, nchunk;       // single-step work items
    int zc2, tiles2_x, tiles2_y, nchunk2;      // two-step work items
    int nsteps;                      // steps this lattice runs in total
    int diag_every;                  // diagnostic cadence (0: at the end only)
    int pairs;                       // advanced two steps per launch (two-step batches)
    const KickCoef<float> *coefs;    // [nsteps] coefficients of each step
};
// step: steps done; cur: phi/theta buffer holding phi^n, theta^n; pe: Pi/E set
// (index into BatchLattice::q) holding Pi^{n-1/2}, E^{n-1/2}
struct BatchState { int step; int cur; int pe; };
// Next stop of a lattice at step n: its next diagnostic point or its end.  In
// two-step batches a lattice advances in pairs of steps and takes a single
// step only when one step is left to its next stop, so the grouping of its
// steps does not depend on the other lattices of the batch.
__host__ __device__ inline int batch_stop(const BatchLattice &B, int n)
{
    if (B.diag_every <= 0) return B.nsteps;
    const long long d = ((long long)n / B.diag_every + 1) * B.diag_every;
    return d < B.nsteps ? (int)d : B.nsteps;
}
// Which lattices a batched launch advances, at step n.  A two-step pass: the
// lattices stepped in pairs with two or more steps to their next stop.  A
// single-step launch: BATCH_ALL every unfinished lattice (one step per launch
// throughout); BATCH_UNPAIRED the unfinished lattices not stepped in pairs;
// BATCH_ROUND_END those and the paired lattices one step before their stop.
enum { BATCH_ALL = 0, BATCH_UNPAIRED = 1, BATCH_ROUND_END = 2 };
__host__ __device__ inline bool batch_takes_pair(const BatchLattice &B, int n)
{
    return B.pairs && n + 2 <= batch_stop(B, n);
}
__host__ __device__ inline bool batch_takes_single(const BatchLattice &B, int n, int mode)
{
    if (mode == BATCH_ALL || !B.pairs) return n < B.nsteps;
    return mode == BATCH_ROUND_END && n + 1 == batch_stop(B, n);
}
int batch_shape_count();
bool batch_shape_ok(int shape, int N);
void batch_tiles(int shape, int N, int *tx, int *ty);
// Per-shape one-time set-up (kernel attributes, occupancy) of the batched
// single-step kernel, or of the batched two-step pass if `two`, outside any
// stream capture.
cudaError_t batch_shape_prepare(int shape, int num_sms, cudaStream_t st, bool two = false);
// mode: which lattices take part (BATCH_ALL, BATCH_UNPAIRED, BATCH_ROUND_END).
cudaError_t launch_fused_batch(int shape, const BatchLattice *lat, BatchState *state, int nlat, const int2 *items,
                               const int *nitems, unsigned int *counter, int num_sms, cudaStream_t st,
                               int mode = BATCH_ALL);
// Batched two-step pass (two leapfrog steps of every lattice per launch),
// shapes 0 (32 x 8 CTA tile, 3 CTAs per SM) and 1 (32 x 12, 2 per SM).
int batch2_shape_count();
void batch2_tiles(int shape, int N, int *tx, int *ty);
cudaError_t launch_fused2_batch(int shape, const BatchLattice *lat, BatchState *state, int nlat, const int2 *items,
                                const int *nitems, unsigned int *counter, int num_sms, cudaStream_t st);

// Fused step with paired FP32 arithmetic (N even), shapes 0..4.
bool pair_shape_ok(int N);
cudaError_t launch_pair_step(const View<float> &v, int N, const KickCoef<float> &c, int shape, cudaStream_t st);
constexpr int kPairShapes = 5;

// TMA-fed fused step (FP32, N % 32 == 0): tensor maps of the interior boxes of
// the read buffer (phi.re, phi.im, theta_1..3) and of Pi.re, Pi.im, E_1..3.
struct TmaMaps {
    CUtensorMap f[5];
    CUtensorMap q[5];
};
bool tma_shape_ok(int N);
size_t tma_smem_bytes();
cudaError_t make_tma_map(CUtensorMap *m, const float *base, int N);
// minb: resident CTAs per SM the registers must allow (2 or 3); *err is set to 1
// if a bounded wait (wait_limit clock cycles per wait) gave up.  drop_q >= 0
// (fault injection for tests) leaves the copy of that Pi/E plane of every CTA
// unissued, so its wait gives up.
constexpr long long kTmaWaitLimit = 1LL << 32;    // about 2 s at 2 GHz
cudaError_t launch_fused_tma(const TmaMaps &maps, const View<float> &v, int N, const KickCoef<float> &c,
                             int *err, int minb, int min_chunk, long long wait_limit, int drop_q, cudaStream_t st);

}  // namespace ah
