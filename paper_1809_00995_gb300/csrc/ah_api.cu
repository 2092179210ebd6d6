// ah_api.cu -- host side of the C ABI declared in include/ah.h.
//
// Owns the device state of each simulation, computes the per-step FP64
// coefficients of the leapfrog (Eqs. up_pi, up_E with the Eq. 7 couplings)
// and of the diagnostics, and enqueues the kernels.  No arithmetic of the
// method runs on the host besides those scalar coefficients and the final
// combination of the FP64 sums into the observables.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>

#include "../../include/ah.h"
#include "ah_internal.cuh"
#include "trace.h"

using namespace ah;

namespace {

thread_local std::string g_err;

ah_status fail(ah_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define AH_CUDA(call)                                                                  \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(e_ == cudaErrorMemoryAllocation ? AH_ERR_OOM : AH_ERR_CUDA,    \
                        "%s failed: %s", #call, cudaGetErrorString(e_));               \
    } while (0)

// Background of Sec. 2: a(tau) = (tau/tau_ref)^alpha, alpha = 0, 1, 2.
double scale_factor(const ah_config &c, double tau)
{
    const double r = tau / c.tau_ref;
    if (c.era == AH_RADIATION) return r;
    if (c.era == AH_MATTER) return r * r;
    return 1.0;
}
// exponent of Eq. 7 at time tau (AH_FLAG_CORE_GROWTH: s before tau_ref, 1 after)
double s_at(const ah_config &c, double tau)
{
    return (c.flags & AH_FLAG_CORE_GROWTH) && tau >= c.tau_ref ? 1.0 : c.s;
}
double coupling_e(const ah_config &c, double a, double tau) { return c.e0 * std::pow(a, s_at(c, tau) - 1.0); }
double coupling_lambda(const ah_config &c, double a, double tau)
{
    return c.lambda0 * std::pow(a, 2.0 * (s_at(c, tau) - 1.0));
}
double tau_of(const ah_config &c, int64_t n) { return c.tau0 + (double)n * c.dt; }

// Kick coefficients of step n (Eqs. up_pi, up_E), FP64, half-step scale
// factors evaluated at tau_n -+ dt/2.
template <typename real>
KickCoef<real> kick_coef(const ah_config &c, int64_t n)
{
    const double tn = tau_of(c, n), tm = tn - 0.5 * c.dt, tp = tn + 0.5 * c.dt;
    const double an = scale_factor(c, tn), am = scale_factor(c, tm), ap = scale_factor(c, tp);
    const double en = coupling_e(c, an, tn), em = coupling_e(c, am, tm), ep = coupling_e(c, ap, tp);
    const double lam = coupling_lambda(c, an, tn);
    const double idx2 = 1.0 / (c.dx * c.dx);
    KickCoef<real> k;
    k.c_damp = (real)((am / ap) * (am / ap));
    k.c_pot = (real)(c.dt * (an * an / ap) * (an * an / ap) * lam * 0.5);
    k.c_lap = (real)(c.dt * idx2 * (an / ap) * (an / ap));
    k.c_edamp = (real)((ep / em) * (ep / em));
    k.c_cur = (real)(2.0 * c.dt * an * an * ep * ep);
    k.c_curl = (real)(c.dt * idx2 * (ep / en) * (ep / en));
    k.dt = (real)c.dt;
    k.sigma2 = (real)(c.sigma * c.sigma);
    k.wrap = (c.flags & AH_FLAG_WRAP_THETA) != 0;
    return k;
}

DiagCoef diag_coef(const ah_config &c, int64_t n)
{
    const double tn = tau_of(c, n), tm = tn - 0.5 * c.dt;
    const double an = scale_factor(c, tn), am = scale_factor(c, tm);
    const double en = coupling_e(c, an, tn), em = coupling_e(c, am, tm);
    const double lam = coupling_lambda(c, an, tn);
    const double dx2 = c.dx * c.dx, e2a2 = en * en * an * an;
    DiagCoef d;
    d.inv_dx2 = 1.0 / dx2;
    d.v_coef = an * an * lam / 4.0;
    d.eel_coef = 1.0 / (2.0 * e2a2 * dx2);
    d.b_coef = 1.0 / (e2a2 * dx2 * dx2);
    d.g_div = 1.0 / (em * em);
    d.g_phi = 2.0 * dx2 * am * am;
    d.sigma2 = c.sigma * c.sigma;
    return d;
}

size_t padded(size_t n) { return (n + 63) & ~(size_t)63; }   // 256 B for floats

}  // namespace

struct ah_sim {
    ah_config cfg;
    int N;
    long long nsites;
    int64_t step;
    int cur;
    int device;
    int num_sms;
    void *dmem;
    size_t dbytes;
    Fields<float> f32;
    Fields<double> f64;
    DiagPartial *partials;
    int nparts;        // entries of partials before result
    DiagPartial *result;
    DiagPartial *host_result;
    unsigned long long *host_count;
    DiagList list;
    int diag_blocks;
    int variant;
    int variant2;      // two-step shape (AH_FLAG_TWO_STEP)
    bool two_step;
    bool pristine;     // state is the freshly initialised random-phase state
    bool tma_ready;    // tensor maps built (FP32, N % 32 == 0)
    TmaMaps tmaps[2];  // per read buffer (phi/theta ping-pong index)
    int *d_err;        // device error word of the bounded waits
    int *host_err;
    long long tma_wait_limit;   // clock cycles per bounded wait of the TMA-fed step
    int tma_drop_q;             // fault injection: Pi/E plane whose copy is never issued (-1: none)
    cudaStream_t stream;
    bool own_stream;
    // asynchronous observables (ah_observables_start / _finish): the pass runs
    // on aux after ev_snap; ev_done marks its end.  Until the main stream has
    // waited for ev_done (diag_fenced), a launch that would overwrite the
    // snapshot must wait first; in two-step mode the first two-step launch
    // after the start writes the other buffer set and may run alongside.
    // FP32 two-step simulations defer the pass instead (diag_deferred): the
    // next two-step launch takes it (k_fused2_diag on the main stream, ev_done
    // recorded there), or, if other work comes first, it runs on its own then.
    cudaStream_t aux;
    cudaEvent_t ev_snap, ev_done;
    bool diag_pending, diag_fenced, diag_deferred;
    int64_t fused_diag_passes;
    // fraction of the plaquettes pierced at the last whole-lattice observables
    // (1 before any): picks the fused or the separate pass for a deferral
    double pierced_frac;
    // the last whole-lattice observables found max |theta| <= kWeakTheta: the
    // two-step launches use the kernel specialised to weak gauge fields
    bool weak_links;
    int64_t weak_launches;
    int diag_free_pairs;
    int64_t diag_step;
};

namespace {

// Largest fraction of pierced plaquettes at which a deferred observables pass
// rides on the next two-step launch (k_fused2_diag) without AH_FLAG_FUSED_DIAG.
constexpr double kFusedDiagPierced = 1e-3;

template <typename real>
void carve(Fields<real> &F, char *base, size_t n, bool spare = false)
{
    real *p = (real *)base;
    const size_t pn = padded(n);
    for (int b = 0; b < 2; ++b) {
        F.phr[b] = p; p += pn;
        F.phi[b] = p; p += pn;
        for (int d = 0; d < 3; ++d) { F.th[b][d] = p; p += pn; }
    }
    F.pir = p; p += pn;
    F.pii = p; p += pn;
    for (int d = 0; d < 3; ++d) { F.el[d] = p; p += pn; }
    for (int k = 0; k < 5; ++k) {
        F.spare[k] = spare ? p : nullptr;
        if (spare) p += pn;
    }
}

template <typename real>
View<real> make_view(const Fields<real> &F, int cur, bool pingpong)
{
    const int o = pingpong ? 1 - cur : cur;
    View<real> v;
    v.phr = F.phr[cur]; v.phi = F.phi[cur];
    v.th1 = F.th[cur][0]; v.th2 = F.th[cur][1]; v.th3 = F.th[cur][2];
    v.pir = F.pir; v.pii = F.pii;
    v.e1 = F.el[0]; v.e2 = F.el[1]; v.e3 = F.el[2];
    v.ophr = F.phr[o]; v.ophi = F.phi[o];
    v.oth1 = F.th[o][0]; v.oth2 = F.th[o][1]; v.oth3 = F.th[o][2];
    return v;
}

ah_status validate(const ah_config &c)
{
    if (c.N < 4 || c.N > 2048) return fail(AH_ERR_ARG, "N=%d outside [4, 2048]", c.N);
    if (!(c.dx > 0) || !(c.dt > 0)) return fail(AH_ERR_ARG, "dx and dt must be > 0");
    if (!(c.e0 > 0) || !(c.lambda0 >= 0) || !(c.sigma > 0))
        return fail(AH_ERR_ARG, "need e0 > 0, lambda0 >= 0, sigma > 0");
    if (c.era < AH_MINKOWSKI || c.era > AH_MATTER) return fail(AH_ERR_ARG, "unknown era %d", c.era);
    if (c.precision != AH_FP32 && c.precision != AH_FP64)
        return fail(AH_ERR_ARG, "unknown precision %d", c.precision);
    if (c.kernel < AH_KERNEL_AUTO || c.kernel > AH_KERNEL_FUSED)
        return fail(AH_ERR_ARG, "unknown kernel %d", c.kernel);
    if (c.flags & ~(AH_FLAG_EXACT_DIAG | AH_FLAG_AUTOTUNE | AH_FLAG_WRAP_THETA | AH_FLAG_CORE_GROWTH |
                    AH_FLAG_TWO_STEP | AH_FLAG_FUSED_DIAG))
        return fail(AH_ERR_ARG, "unknown flags 0x%x", c.flags);
    if ((c.flags & AH_FLAG_FUSED_DIAG) && !(c.flags & AH_FLAG_TWO_STEP))
        return fail(AH_ERR_ARG, "AH_FLAG_FUSED_DIAG needs AH_FLAG_TWO_STEP");
    if ((c.flags & AH_FLAG_TWO_STEP) && (c.precision != AH_FP32 || c.kernel == AH_KERNEL_PLAIN))
        return fail(AH_ERR_ARG, "AH_FLAG_TWO_STEP needs FP32 and the fused kernel");
    if (!std::isfinite(c.s)) return fail(AH_ERR_ARG, "s must be finite");
    if (c.era != AH_MINKOWSKI && !(c.tau0 > 0)) return fail(AH_ERR_ARG, "tau0 must be > 0");
    if (!(c.tau_ref > 0)) return fail(AH_ERR_ARG, "tau_ref must be > 0");
    if (!(c.tau_end >= c.tau0)) return fail(AH_ERR_ARG, "tau_end must be >= tau0");
    if (c.dt * std::sqrt(3.0) > c.dx) return fail(AH_ERR_ARG, "Courant: need dt <= dx/sqrt(3)");
    // Leapfrog stability of the stiffest mode: lattice gradient (12/dx^2) plus the
    // scalar / vector mass terms lambda0 sigma^2 a^2s and 2 e0^2 sigma^2 a^2s, with
    // a^s largest at one end of [tau0, tau_end] (of each of the two stretches
    // with their own s under core growth).  Require dt^2 w^2 < 0.9 * 4.
    auto as2_over = [&c](double t0, double t1, double s) {
        return std::fmax(std::pow(scale_factor(c, t0), 2.0 * s), std::pow(scale_factor(c, t1), 2.0 * s));
    };
    double as2 = 0.0;
    if (!(c.flags & AH_FLAG_CORE_GROWTH) || c.tau_end < c.tau_ref)
        as2 = as2_over(c.tau0, c.tau_end, c.s);
    else if (c.tau0 >= c.tau_ref)
        as2 = as2_over(c.tau0, c.tau_end, 1.0);
    else
        as2 = std::fmax(as2_over(c.tau0, c.tau_ref, c.s), as2_over(c.tau_ref, c.tau_end, 1.0));
    const double m2 = std::fmax(c.lambda0, 2.0 * c.e0 * c.e0) * c.sigma * c.sigma * as2;
    const double w2dt2 = c.dt * c.dt * (12.0 / (c.dx * c.dx) + m2);
    if (!(w2dt2 < 3.6))
        return fail(AH_ERR_UNSTABLE, "leapfrog unstable: dt^2 w_max^2 = %.3g >= 3.6 (a^s up to %.3g)",
                    w2dt2, std::sqrt(as2));
    return AH_OK;
}

// FP32 shapes beyond the k_fused ones: the paired-arithmetic kernel (k_pair.cu)
// and the TMA-fed kernel (resident CTAs per SM, minimum z-chunk length).
struct TmaShape { int minb, min_chunk; const char *name; };
constexpr TmaShape kTmaShapes[] = { { 3, 16, "tma_b3" }, { 2, 16, "tma_b2" }, { 3, 64, "tma_b3_z64" } };
constexpr int kNumTma = (int)(sizeof(kTmaShapes) / sizeof(kTmaShapes[0]));
constexpr const char *kPairNames[kPairShapes] = { "pair_ty6_b3", "pair_ty6_b4", "pair_ty14_b1", "pair_ty14_b2",
                                                  "pair_ty30_b1" };

int n_variants(int precision)
{
    return precision == AH_FP32 ? fused_variant_count<float>() + kPairShapes + kNumTma : fused_variant_count<double>();
}
// FP32 variant families: 0 k_fused, 1 k_pair, 2 k_fused_tma; *idx = index within the family
int family(const ah_sim *h, int v, int *idx)
{
    if (h->cfg.precision != AH_FP32 || v < fused_variant_count<float>()) { *idx = v; return 0; }
    v -= fused_variant_count<float>();
    if (v < kPairShapes) { *idx = v; return 1; }
    *idx = v - kPairShapes;
    return 2;
}
bool variant_ok(const ah_sim *h, int v)
{
    if (h->two_step) return v >= 0 && v < fused2_variant_count();
    if (v < 0 || v >= n_variants(h->cfg.precision)) return false;
    int i;
    switch (family(h, v, &i)) {
    case 1: return pair_shape_ok(h->N);
    case 2: return h->tma_ready;
    default:
        return h->cfg.precision == AH_FP32 ? fused_variant_ok<float>(v, h->N) : fused_variant_ok<double>(v, h->N);
    }
}
const char *variant_name(const ah_sim *h, int v)
{
    if (h->two_step) return fused2_variant_name(v);
    if (h->cfg.precision == AH_FP64) return fused_variant_name<double>(v);
    int i;
    switch (family(h, v, &i)) {
    case 1: return kPairNames[i];
    case 2: return kTmaShapes[i].name;
    default: return fused_variant_name<float>(v);
    }
}

template <typename real>
ah_status diag_start(ah_sim *h);

// A deferred observables pass that no two-step launch took: run it on its own
// now (on aux, from the current state, which is still its snapshot).
ah_status diag_undefer(ah_sim *h)
{
    if (!h->diag_deferred) return AH_OK;
    h->diag_deferred = false;
    const ah_status st = diag_start<float>(h);
    if (st != AH_OK) return st;
    h->diag_fenced = false;
    h->diag_free_pairs = 0;
    return AH_OK;
}

// Make the simulation's stream wait for a pending asynchronous observables
// pass before work that would change its snapshot.
ah_status diag_fence(ah_sim *h)
{
    if (ah_status st = diag_undefer(h); st != AH_OK) return st;
    if (h->diag_pending && !h->diag_fenced) {
        AH_CUDA(cudaStreamWaitEvent(h->stream, h->ev_done, 0));
        h->diag_fenced = true;
    }
    return AH_OK;
}

template <typename real>
ah_status do_step(ah_sim *h, int64_t n)
{
    Fields<real> &F = *(Fields<real> *)(h->cfg.precision == AH_FP32 ? (void *)&h->f32 : (void *)&h->f64);
    const KickCoef<real> k = kick_coef<real>(h->cfg, n);
    if (h->cfg.kernel == AH_KERNEL_PLAIN) {
        AH_CUDA(launch_plain_step<real>(make_view(F, h->cur, false), h->N, k, h->stream));
    } else if (int idx; family(h, h->variant, &idx) != 0) {
        if constexpr (std::is_same<real, float>::value) {
            if (family(h, h->variant, &idx) == 1) {
                AH_CUDA(launch_pair_step(make_view(F, h->cur, true), h->N, k, idx, h->stream));
            } else {
                const TmaShape &t = kTmaShapes[idx];
                AH_CUDA(launch_fused_tma(h->tmaps[h->cur], make_view(F, h->cur, true), h->N, k, h->d_err, t.minb,
                                         t.min_chunk, h->tma_wait_limit, h->tma_drop_q, h->stream));
            }
            h->cur ^= 1;
        }
    } else {
        AH_CUDA(launch_fused_step<real>(make_view(F, h->cur, true), h->N, k, h->variant, h->stream));
        h->cur ^= 1;
    }
    return AH_OK;
}

// Steps n and n + 1 in one pass (AH_FLAG_TWO_STEP): phi, theta go to the
// other ping-pong buffer, Pi and E to the spare set, which then becomes the
// current one.
View2<float> step2_view(ah_sim *h)
{
    Fields<float> &F = h->f32;
    View2<float> v;
    const int o = 1 - h->cur;
    v.phr = F.phr[h->cur]; v.phi = F.phi[h->cur];
    v.th1 = F.th[h->cur][0]; v.th2 = F.th[h->cur][1]; v.th3 = F.th[h->cur][2];
    v.pir = F.pir; v.pii = F.pii; v.e1 = F.el[0]; v.e2 = F.el[1]; v.e3 = F.el[2];
    v.ophr = F.phr[o]; v.ophi = F.phi[o];
    v.oth1 = F.th[o][0]; v.oth2 = F.th[o][1]; v.oth3 = F.th[o][2];
    v.opir = F.spare[0]; v.opii = F.spare[1]; v.oe1 = F.spare[2]; v.oe2 = F.spare[3]; v.oe3 = F.spare[4];
    return v;
}
void step2_swap(ah_sim *h)
{
    Fields<float> &F = h->f32;
    h->cur = 1 - h->cur;
    std::swap(F.pir, F.spare[0]);
    std::swap(F.pii, F.spare[1]);
    for (int d = 0; d < 3; ++d) std::swap(F.el[d], F.spare[2 + d]);
}
ah_status do_step2(ah_sim *h, int64_t n)
{
    const bool weak = h->weak_links && fused2_weak_ok(h->variant2, h->N);
    AH_CUDA(launch_fused2_step(step2_view(h), h->N, kick_coef<float>(h->cfg, n), kick_coef<float>(h->cfg, n + 1),
                               h->variant2, h->stream, weak));
    h->weak_launches += weak;
    step2_swap(h);
    return AH_OK;
}
// What the last whole-lattice observables say about the state.
void note_obs(ah_sim *h, const ah_obs &o)
{
    h->pierced_frac = (double)o.n_pierced / (3.0 * (double)h->nsites);
    h->weak_links = h->two_step && o.max_abs_theta <= kWeakTheta;
}
// The same pass taking the deferred observables of the state n on the way:
// partial sums, then (on the state n, which the pass leaves in place) the
// FP64 windings of the listed plaquettes, a recount if the list overflowed,
// and the copy to the host, all on the main stream, ending at ev_done.
ah_status do_step2_diag(ah_sim *h, int64_t n)
{
    const View<float> vn = make_view(h->f32, h->cur, false);
    DiagArgs da;
    da.dc = diag_coef(h->cfg, n);
    da.partials = h->partials;
    da.list = h->list;
    if (fused2_diag_ctas(h->N) > h->nparts)
        return fail(AH_ERR_CUDA, "diagnostics scratch too small: the N=%d two-step pass needs %d partials, %d allocated",
                    h->N, fused2_diag_ctas(h->N), h->nparts);
    AH_CUDA(cudaMemsetAsync(h->list.count, 0, sizeof(unsigned long long), h->stream));
    AH_CUDA(launch_fused2_diag(step2_view(h), h->N, kick_coef<float>(h->cfg, n), kick_coef<float>(h->cfg, n + 1), da,
                               h->nparts, h->stream));
    AH_CUDA(launch_diag_reduce<float>(vn, h->N, h->partials, fused2_diag_ctas(h->N), h->result, h->list,
                                      h->diag_blocks, h->stream));
    AH_CUDA(launch_wind_recount_on_overflow<float>(vn, h->N, h->list, h->result, h->diag_blocks, h->stream));
    AH_CUDA(cudaMemcpyAsync(h->host_result, h->result, sizeof(DiagPartial), cudaMemcpyDeviceToHost, h->stream));
    AH_CUDA(cudaEventRecord(h->ev_done, h->stream));
    step2_swap(h);
    return AH_OK;
}

// Read and clear the device error word of the bounded waits (synchronous).
ah_status check_device_error(ah_sim *h)
{
    if (!h->d_err) return AH_OK;
    AH_CUDA(cudaMemcpyAsync(h->host_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    AH_CUDA(cudaStreamSynchronize(h->stream));
    if (*h->host_err) {
        *h->host_err = 0;
        cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
        return fail(AH_ERR_TIMEOUT, "a bounded wait in the fused step gave up; the state is not valid");
    }
    return AH_OK;
}

void fill_obs(const ah_config &c, int64_t step, int64_t n_sites, const DiagPartial &r, ah_obs *out);

template <typename real>
ah_status do_diag(ah_sim *h, Box b, ah_obs *out)
{
    Fields<real> &F = *(Fields<real> *)(h->cfg.precision == AH_FP32 ? (void *)&h->f32 : (void *)&h->f64);
    const DiagCoef dc = diag_coef(h->cfg, h->step);
    const View<real> v = make_view(F, h->cur, false);
    const bool exact = (h->cfg.flags & AH_FLAG_EXACT_DIAG) != 0;
    const bool whole = b.x0 == 0 && b.y0 == 0 && b.z0 == 0 && b.nx == h->N && b.ny == h->N && b.nz == h->N;
    if (whole && !exact && fused_diag_ctas(h->N) > h->nparts)
        return fail(AH_ERR_CUDA, "diagnostics scratch too small: the N=%d pass needs %d partials, %d allocated",
                    h->N, fused_diag_ctas(h->N), h->nparts);
    if (whole && !exact)
        AH_CUDA(launch_diag_whole<real>(v, h->N, dc, h->partials, h->nparts, h->result, h->list, h->diag_blocks,
                                        h->stream));
    else
        AH_CUDA(launch_diag<real>(v, h->N, b, dc, h->partials, h->diag_blocks, h->result, h->list, exact,
                                  h->stream));
    AH_CUDA(cudaMemcpyAsync(h->host_result, h->result, sizeof(DiagPartial), cudaMemcpyDeviceToHost,
                            h->stream));
    AH_CUDA(cudaMemcpyAsync(h->host_count, h->list.count, sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, h->stream));
    AH_CUDA(cudaMemcpyAsync(h->host_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    AH_CUDA(cudaStreamSynchronize(h->stream));
    if (*h->host_err) return check_device_error(h);
    if (!exact && *h->host_count > (unsigned long long)h->list.capacity) {
        // too many plaquettes near a branch cut for the list: redo all in FP64
        AH_CUDA(launch_diag<real>(v, h->N, b, dc, h->partials, h->diag_blocks, h->result, h->list, true,
                                  h->stream));
        AH_CUDA(cudaMemcpyAsync(h->host_result, h->result, sizeof(DiagPartial), cudaMemcpyDeviceToHost,
                                h->stream));
        AH_CUDA(cudaStreamSynchronize(h->stream));
    }
    fill_obs(h->cfg, h->step, (int64_t)b.nx * b.ny * b.nz, *h->host_result, out);
    if (whole) note_obs(h, *out);
    if (out->nonfinite)
        return fail(AH_ERR_NONFINITE, "%lld sites have non-finite diagnostics", (long long)out->nonfinite);
    return AH_OK;
}

// Observables (Eqs. defXiV2, defR, 9, defEoS, Gauss residual) from the raw sums.
void fill_obs(const ah_config &c, int64_t step, int64_t n_sites, const DiagPartial &r, ah_obs *out)
{
    ah_obs o;
    memset(&o, 0, sizeof o);
    o.step = step;
    o.tau = tau_of(c, step);
    o.a = scale_factor(c, o.tau);
    o.n_sites = n_sites;
    for (int k = 0; k < kNumSums; ++k) o.sums[k] = r.sums[k];
    for (int q = 0; q < 3; ++q) {
        o.wind_abs_plane[q] = r.ints[q];
        o.wind_plane[q] = r.ints[3 + q];
    }
    o.n_pierced = r.ints[6];
    o.nonfinite = r.ints[7];
    o.sum_abs_W = o.wind_abs_plane[0] + o.wind_abs_plane[1] + o.wind_abs_plane[2];
    const double ns = (double)o.n_sites;
    o.L_mean = o.sums[0] / ns;
    o.xi_L = std::sqrt(-2.0 * M_PI * c.sigma * c.sigma / o.L_mean);
    o.xi_W = std::sqrt(ns * c.dx * c.dx * c.dx / (M_PI / 6.0 * c.dx * (double)o.sum_abs_W));
    o.R_V = o.sums[8] / o.sums[9];
    o.R_L = o.sums[10] / o.sums[11];
    o.v2_V = 2.0 * o.R_V / (1.0 + o.R_V);
    o.v2_L = 2.0 * o.R_L / (1.0 + o.R_L);
    o.p_over_rho_L = o.sums[12] / o.sums[13];
    o.v2_omega = 0.5 * (1.0 + 3.0 * o.p_over_rho_L);
    o.gauss_rms = std::sqrt(o.sums[14] / ns);
    o.gauss_max = r.maxv[0];
    o.gauss_rel = std::sqrt(o.sums[14] / o.sums[15]);
    o.energy = c.dx * c.dx * c.dx * o.sums[1];
    o.max_abs_theta = r.maxv[1];
    *out = o;
}

// Random-phase initial state (Sec. 2): zero everything, then phi of buffer 0.
cudaError_t write_initial_state(ah_sim *h)
{
    h->cur = 0;
    h->step = 0;
    h->pristine = true;
    cudaError_t e = cudaMemsetAsync(h->dmem, 0, h->dbytes, h->stream);
    if (e != cudaSuccess) return e;
    if (h->cfg.precision == AH_FP32)
        return launch_init_phase<float>(h->f32.phr[0], h->f32.phi[0], h->N, h->cfg.seed, h->cfg.sigma, h->stream);
    return launch_init_phase<double>(h->f64.phr[0], h->f64.phi[0], h->N, h->cfg.seed, h->cfg.sigma, h->stream);
}

// process-wide autotune results per (device, N, precision, two-step mode)
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, bool>, int> g_tune;

int tune_cache_get(const ah_sim *h)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(h->device, h->N, h->cfg.precision, h->two_step));
    return it == g_tune.end() ? -1 : it->second;
}
void tune_cache_put(const ah_sim *h, int v)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[std::make_tuple(h->device, h->N, h->cfg.precision, h->two_step)] = v;
}

ah_status enter(const ah_sim *h)
{
    if (!h) return fail(AH_ERR_ARG, "null simulation handle");
    AH_CUDA(cudaSetDevice(h->device));
    return AH_OK;
}

}  // namespace

namespace ah {
KickCoef<float> host_kick_coef32(const ah_config &c, int64_t step) { return kick_coef<float>(c, step); }
void host_carve32(Fields<float> &F, void *base, size_t nsites, bool spare) { carve(F, (char *)base, nsites, spare); }
size_t host_state_bytes32(size_t nsites, bool spare) { return (spare ? 20 : 15) * padded(nsites) * sizeof(float); }
void host_fill_obs(const ah_config &c, int64_t step, int64_t n_sites, const DiagPartial &r, ah_obs *out)
{
    fill_obs(c, step, n_sites, r, out);
}
int64_t host_run_steps(const ah_config &c) { return (int64_t)std::llround((c.tau_end - c.tau0) / c.dt); }
DiagCoef host_diag_coef(const ah_config &c, int64_t step) { return diag_coef(c, step); }
ah_status host_validate(const ah_config &c) { return validate(c); }
ah_status host_fail(ah_status st, const char *msg) { return fail(st, "%s", msg); }
}  // namespace ah

namespace {
template <typename real>
ah_status diag_start(ah_sim *h)
{
    Fields<real> &F = *(Fields<real> *)(h->cfg.precision == AH_FP32 ? (void *)&h->f32 : (void *)&h->f64);
    const DiagCoef dc = diag_coef(h->cfg, h->step);
    const View<real> v = make_view(F, h->cur, false);
    const int N = h->N;
    AH_CUDA(cudaEventRecord(h->ev_snap, h->stream));
    AH_CUDA(cudaStreamWaitEvent(h->aux, h->ev_snap, 0));
    if (h->cfg.flags & AH_FLAG_EXACT_DIAG) {
        AH_CUDA(launch_diag<real>(v, N, Box{ 0, 0, 0, N, N, N }, dc, h->partials, h->diag_blocks, h->result, h->list,
                                  true, h->aux));
    } else {
        if (fused_diag_ctas(N) > h->nparts)
            return fail(AH_ERR_CUDA, "diagnostics scratch too small: the N=%d pass needs %d partials, %d allocated", N,
                        fused_diag_ctas(N), h->nparts);
        AH_CUDA(launch_diag_whole<real>(v, N, dc, h->partials, h->nparts, h->result, h->list, h->diag_blocks, h->aux));
        // a list overflow is settled on the device: the snapshot may change
        // before the host could look at the count
        AH_CUDA(launch_wind_recount_on_overflow<real>(v, N, h->list, h->result, h->diag_blocks, h->aux));
    }
    AH_CUDA(cudaMemcpyAsync(h->host_result, h->result, sizeof(DiagPartial), cudaMemcpyDeviceToHost, h->aux));
    AH_CUDA(cudaEventRecord(h->ev_done, h->aux));
    return AH_OK;
}
}  // namespace

extern "C" {

int ah_abi_version(void) { return 6; }

const char *ah_last_error(void) { return g_err.c_str(); }

void ah_config_default(ah_config *c, int32_t N)
{
    if (!c) return;
    memset(c, 0, sizeof *c);
    c->N = N;
    c->era = AH_RADIATION;
    c->precision = AH_FP32;
    c->kernel = AH_KERNEL_AUTO;
    c->dx = 0.5;
    c->dt = 0.1;
    c->s = 0.0;
    c->lambda0 = 2.0;
    c->e0 = 1.0;
    c->sigma = 1.0;
    c->tau0 = 1.0;
    c->tau_end = N * c->dx / 2.0;
    c->tau_ref = c->tau_end;
    c->seed = 1;
}

ah_status ah_create_ex(const ah_config *cfg, ah_sim **out)
{
    TraceRange tr("ah_create");
    if (!cfg || !out) return fail(AH_ERR_ARG, "null argument");
    *out = nullptr;
    ah_status st = validate(*cfg);
    if (st != AH_OK) return st;
    ah_sim *h = new (std::nothrow) ah_sim();
    if (!h) return fail(AH_ERR_OOM, "host allocation failed");
    h->cfg = *cfg;
    if (h->cfg.kernel == AH_KERNEL_AUTO) h->cfg.kernel = AH_KERNEL_FUSED;
    h->N = cfg->N;
    h->variant = cfg->precision == AH_FP32 ? fused_default_variant<float>() : fused_default_variant<double>();
    h->two_step = (cfg->flags & AH_FLAG_TWO_STEP) != 0;
    h->variant2 = fused2_default_variant();
    // fault injection for tests, read at creation: AH_TMA_DROP_COPY=q makes the
    // TMA-fed step leave the copy of Pi/E plane q of every CTA unissued, so that
    // the bounded wait for it gives up (AH_ERR_TIMEOUT from ah_sync);
    // AH_TMA_WAIT_LIMIT_CYCLES shortens that bound
    h->tma_wait_limit = kTmaWaitLimit;
    h->tma_drop_q = -1;
    if (const char *w = std::getenv("AH_TMA_WAIT_LIMIT_CYCLES")) h->tma_wait_limit = std::max(0LL, std::atoll(w));
    if (const char *q = std::getenv("AH_TMA_DROP_COPY")) h->tma_drop_q = std::max(-1, std::atoi(q));
    h->nsites = (long long)cfg->N * cfg->N * cfg->N;
    h->step = 0;
    h->cur = 0;
    h->pierced_frac = 1.0;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete h;
        return fail(AH_ERR_CUDA, "CUDA device setup failed: %s", cudaGetErrorString(e));
    }
    h->own_stream = true;
    const size_t esz = cfg->precision == AH_FP32 ? sizeof(float) : sizeof(double);
    h->dbytes = (h->two_step ? 20 : 15) * padded((size_t)h->nsites) * esz;
    h->diag_blocks = diag_grid_blocks(h->num_sms);
    const int nparts = std::max({ h->diag_blocks, fused_diag_ctas(h->N), h->two_step ? fused2_diag_ctas(h->N) : 0 });
    h->nparts = nparts;
    // expected near-cut plaquettes: about 5e-5 of the 3 N^3 plaquettes in FP32
    h->list.capacity = std::max<long long>(1LL << 20, h->nsites * 3 / 2000);
    e = cudaMalloc(&h->dmem, h->dbytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->partials, sizeof(DiagPartial) * (nparts + 1));
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&h->list.count, sizeof(unsigned long long) * (1 + h->list.capacity));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->host_result, sizeof(DiagPartial) + 32);
    if (e != cudaSuccess) {
        const double gb = h->dbytes / 1e9;
        cudaGetLastError();                  // a refused allocation is not a sticky error: clear it
        ah_destroy(h);
        return fail(AH_ERR_OOM, "allocation of %.3g GB failed: %s", gb, cudaGetErrorString(e));
    }
    h->result = h->partials + nparts;
    h->list.items = h->list.count + 1;
    h->host_count = (unsigned long long *)(h->host_result + 1);
    h->host_err = (int *)(h->host_count + 1);
    e = cudaMalloc((void **)&h->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
    if (e != cudaSuccess) {
        ah_destroy(h);
        return fail(AH_ERR_OOM, "allocation failed: %s", cudaGetErrorString(e));
    }
    if (cfg->precision == AH_FP32) carve(h->f32, (char *)h->dmem, (size_t)h->nsites, h->two_step);
    else carve(h->f64, (char *)h->dmem, (size_t)h->nsites);
    // the TMA maps hold the Pi and E buffers, which the two-step mode swaps
    if (cfg->precision == AH_FP32 && tma_shape_ok(h->N) && !h->two_step) {
        cudaError_t me = cudaSuccess;
        for (int b = 0; b < 2 && me == cudaSuccess; ++b) {
            const float *fs[5] = { h->f32.phr[b], h->f32.phi[b], h->f32.th[b][0], h->f32.th[b][1], h->f32.th[b][2] };
            const float *qs[5] = { h->f32.pir, h->f32.pii, h->f32.el[0], h->f32.el[1], h->f32.el[2] };
            for (int k = 0; k < 5 && me == cudaSuccess; ++k) me = make_tma_map(&h->tmaps[b].f[k], fs[k], h->N);
            for (int k = 0; k < 5 && me == cudaSuccess; ++k) me = make_tma_map(&h->tmaps[b].q[k], qs[k], h->N);
        }
        h->tma_ready = me == cudaSuccess;
    }
    e = write_initial_state(h);
    if (e != cudaSuccess) {
        ah_destroy(h);
        return fail(AH_ERR_CUDA, "initialisation failed: %s", cudaGetErrorString(e));
    }
    *out = h;
    if (cfg->flags & AH_FLAG_AUTOTUNE) {
        const int cached = tune_cache_get(h);
        if (cached >= 0) {
            (h->two_step ? h->variant2 : h->variant) = cached;
        } else if ((st = ah_autotune(h, 3, nullptr)) != AH_OK) {
            ah_destroy(h);
            *out = nullptr;
            return st;
        }
    }
    return AH_OK;
}

ah_sim *ah_create(int32_t N, double dx, double dt, int32_t era, double s, double lambda0, double e0,
                  uint64_t seed)
{
    ah_config c;
    ah_config_default(&c, N);
    c.dx = dx;
    c.dt = dt;
    c.era = era;
    c.s = s;
    c.lambda0 = lambda0;
    c.e0 = e0;
    c.seed = seed;
    c.tau_end = N * dx / 2.0;
    c.tau_ref = c.tau_end;
    ah_sim *h = nullptr;
    return ah_create_ex(&c, &h) == AH_OK ? h : nullptr;
}

ah_status ah_step(ah_sim *h, int64_t nsteps)
{
    TraceRange tr("ah_step");
    ah_status st = enter(h);
    if (st != AH_OK) return st;
    if (nsteps < 0) return fail(AH_ERR_ARG, "nsteps must be >= 0");
    if (nsteps > 0) h->pristine = false;
    int64_t q = 0;
    if (h->two_step) {
        for (; q + 2 <= nsteps; q += 2) {
            if (h->diag_deferred) {
                // the first pass after a deferred observables start takes it
                h->diag_deferred = false;
                if ((st = do_step2_diag(h, h->step)) != AH_OK) return st;
                ++h->fused_diag_passes;
            } else {
                // the first pass after an asynchronous observables start reads
                // the snapshot and writes the other set: it may overlap the pass
                if (h->diag_pending && !h->diag_fenced && h->diag_free_pairs > 0) --h->diag_free_pairs;
                else if ((st = diag_fence(h)) != AH_OK) return st;
                if ((st = do_step2(h, h->step)) != AH_OK) return st;
            }
            h->step += 2;
        }
    }
    if (q < nsteps && (st = diag_fence(h)) != AH_OK) return st;
    for (; q < nsteps; ++q) {
        st = h->cfg.precision == AH_FP32 ? do_step<float>(h, h->step) : do_step<double>(h, h->step);
        if (st != AH_OK) return st;
        ++h->step;
    }
    return AH_OK;
}

ah_status ah_observables_box(ah_sim *h, int32_t x0, int32_t y0, int32_t z0, int32_t nx, int32_t ny,
                             int32_t nz, ah_obs *out)
{
    TraceRange tr("ah_observables");
    ah_status st = enter(h);
    if (st != AH_OK) return st;
    if (!out) return fail(AH_ERR_ARG, "null output");
    if (h->diag_pending)
        return fail(AH_ERR_BUSY, "an asynchronous observables pass is pending: call ah_observables_finish first");
    const int N = h->N;
    if (nx < 1 || ny < 1 || nz < 1 || nx > N || ny > N || nz > N)
        return fail(AH_ERR_ARG, "box extent must be in [1, N]");
    auto md = [N](int v) { v %= N; return v < 0 ? v + N : v; };
    const Box b{ md(x0), md(y0), md(z0), nx, ny, nz };
    return h->cfg.precision == AH_FP32 ? do_diag<float>(h, b, out) : do_diag<double>(h, b, out);
}

ah_status ah_observables(ah_sim *h, ah_obs *out)
{
    if (!h) return fail(AH_ERR_ARG, "null simulation handle");
    return ah_observables_box(h, 0, 0, 0, h->N, h->N, h->N, out);
}

ah_status ah_observables_start(ah_sim *h)
{
    TraceRange tr("ah_observables_start");
    ah_status st = enter(h);
    if (st != AH_OK) return st;
    if (h->diag_pending) return fail(AH_ERR_BUSY, "an asynchronous observables pass is already pending");
    if (!h->aux) {
        AH_CUDA(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
        AH_CUDA(cudaEventCreateWithFlags(&h->ev_snap, cudaEventDisableTiming));
        AH_CUDA(cudaEventCreateWithFlags(&h->ev_done, cudaEventDisableTiming));
    }
    h->diag_step = h->step;
    // Fold the pass into the next two-step launch where that pays (measured at
    // 256^3 - 1024^3: 2-4 % faster than a launch plus a separate pass on string
    // networks in smooth fields, where most tiles skip the winding carries,
    // 4-8 % slower on rough fields, where the fused launch's accumulators cost
    // it a third of its resident CTAs)
    const bool fuse = (h->cfg.flags & AH_FLAG_FUSED_DIAG) || h->pierced_frac < kFusedDiagPierced;
    if (h->two_step && fuse && !(h->cfg.flags & AH_FLAG_EXACT_DIAG)) {
        // taken by the next two-step launch (or run on its own before other work)
        h->diag_pending = true;
        h->diag_deferred = true;
        h->diag_fenced = true;
        h->diag_free_pairs = 0;
        return AH_OK;
    }
    st = h->cfg.precision == AH_FP32 ? diag_start<float>(h) : diag_start<double>(h);
    if (st != AH_OK) return st;
    h->diag_pending = true;
    h->diag_fenced = false;
    h->diag_free_pairs = h->two_step ? 1 : 0;
    return AH_OK;
}

ah_status ah_observables_finish(ah_sim *h, ah_obs *out)
{
    TraceRange tr("ah_observables_finish");
    ah_status st = enter(h);
    if (st != AH_OK) return st;
    if (!out) return fail(AH_ERR_ARG, "null output");
    if (!h->diag_pending) return fail(AH_ERR_ARG, "no asynchronous observables pass was started");
    if ((st = diag_undefer(h)) != AH_OK) return st;
    const cudaError_t e = cudaEventSynchronize(h->ev_done);
    h->diag_pending = false;
    if (e != cudaSuccess) return fail(AH_ERR_CUDA, "asynchronous observables: %s", cudaGetErrorString(e));
    fill_obs(h->cfg, h->diag_step, h->nsites, *h->host_result, out);
    note_obs(h, *out);
    if (out->nonfinite)
        return fail(AH_ERR_NONFINITE, "%lld sites have non-finite diagnostics", (long long)out->nonfinite);
    return AH_OK;
}

ah_status ah_get_fields(ah_sim *h, int32_t x0, int32_t y0, int32_t z0, int32_t nx, int32_t ny, int32_t nz,
                        double *out)
{
    ah_status st = enter(h);
    if (st != AH_OK) return st;
    if (!out) return fail(AH_ERR_ARG, "null output");
    const int N = h->N;
    if (nx < 1 || ny < 1 || nz < 1 || nx > N || ny > N || nz > N)
        return fail(AH_ERR_ARG, "window extent must be in [1, N]");
    auto md = [N](int v) { v %= N; return v < 0 ? v + N : v; };
    const Box b{ md(x0), md(y0), md(z0), nx, ny, nz };
    const size_t bytes = sizeof(double) * 10 * (size_t)nx * ny * nz;
    double *tmp = nullptr;
    AH_CUDA(cudaMalloc(&tmp, bytes));
    cudaError_t e = h->cfg.precision == AH_FP32
                        ? launch_gather_window<float>(h->f32, h->cur, N, b, tmp, h->stream)
                        : launch_gather_window<double>(h->f64, h->cur, N, b, tmp, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return fail(AH_ERR_CUDA, "get_fields failed: %s", cudaGetErrorString(e));
    return AH_OK;
}

ah_status ah_set_fields(ah_sim *h, const double *in, int64_t step)
{
    ah_status st = enter(h);
    if (st != AH_OK) return st;
    if (!in || step < 0) return fail(AH_ERR_ARG, "null input or negative step");
    if ((st = diag_fence(h)) != AH_OK) return st;
    const size_t bytes = sizeof(double) * 10 * (size_t)h->nsites;
    double *tmp = nullptr;
    AH_CUDA(cudaMalloc(&tmp, bytes));
    cudaError_t e = cudaMemcpyAsync(tmp, in, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = h->cfg.precision == AH_FP32 ? launch_scatter_all<float>(h->f32, h->cur, h->N, tmp, h->stream)
                                        : launch_scatter_all<double>(h->f64, h->cur, h->N, tmp, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return fail(AH_ERR_CUDA, "set_fields failed: %s", cudaGetErrorString(e));
    h->step = step;
    h->pristine = false;
    h->pierced_frac = 1.0;              // nothing known about the new state
    h->weak_links = false;
    return AH_OK;
}

ah_status ah_set_stream(ah_sim *h, void *stream)
{
    ah_status st = enter(h);
    if (st != AH_OK) return st;
    if (h->diag_pending) AH_CUDA(cudaEventSynchronize(h->ev_done));
    h->diag_fenced = h->diag_pending;         // the pass has ended: no later work need wait
    AH_CUDA(cudaStreamSynchronize(h->stream));
    if (stream) {
        if (h->own_stream) cudaStreamDestroy(h->stream);
        h->stream = (cudaStream_t)stream;
        h->own_stream = false;
    } else if (!h->own_stream) {
        AH_CUDA(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    return AH_OK;
}

ah_status ah_sync(ah_sim *h)
{
    ah_status st = enter(h);
    if (st != AH_OK) return st;
    AH_CUDA(cudaStreamSynchronize(h->stream));
    return check_device_error(h);
}

int64_t ah_get_step(const ah_sim *h) { return h ? h->step : -1; }

double ah_get_tau(const ah_sim *h) { return h ? tau_of(h->cfg, h->step) : NAN; }

ah_status ah_get_info(const ah_sim *h, ah_info *out)
{
    if (!h || !out) return fail(AH_ERR_ARG, "null argument");
    const int64_t esz = h->cfg.precision == AH_FP32 ? 4 : 8;
    out->N = h->N;
    out->n_sites = h->nsites;
    out->precision = h->cfg.precision;
    out->kernel = h->cfg.kernel;
    out->state_bytes = (int64_t)h->dbytes;
    out->step_bytes = 20 * esz * h->nsites;
    out->step_launches = h->cfg.kernel == AH_KERNEL_PLAIN ? 3 : 1;
    out->variant = h->two_step ? h->variant2 : h->variant;
    out->n_variants = h->two_step ? fused2_variant_count() : n_variants(h->cfg.precision);
    const char *nm = variant_name(h, out->variant);
    snprintf(out->variant_name, sizeof out->variant_name, "%s", h->cfg.kernel == AH_KERNEL_PLAIN ? "plain" : nm);
    out->fused_diag_passes = h->fused_diag_passes;
    out->weak_field_launches = h->weak_launches;
    return AH_OK;
}

int32_t ah_variant_count(int32_t precision)
{
    return precision == AH_FP32 || precision == AH_FP64 ? n_variants(precision) : 0;
}

ah_status ah_set_variant(ah_sim *h, int32_t variant)
{
    if (!h) return fail(AH_ERR_ARG, "null simulation handle");
    if (!variant_ok(h, variant))
        return fail(AH_ERR_ARG, "variant %d not available (count %d, N=%d)", variant,
                    h->two_step ? fused2_variant_count() : n_variants(h->cfg.precision), h->N);
    (h->two_step ? h->variant2 : h->variant) = variant;
    return AH_OK;
}

ah_status ah_autotune(ah_sim *h, int32_t trial_steps, int32_t *chosen)
{
    TraceRange tr("ah_autotune");
    ah_status st = enter(h);
    if (st != AH_OK) return st;
    if (!h->pristine) return fail(AH_ERR_BUSY, "autotune needs the freshly created state");
    if (h->diag_pending) return fail(AH_ERR_BUSY, "an asynchronous observables pass is pending");
    if (trial_steps < 1) return fail(AH_ERR_ARG, "trial_steps must be >= 1");
    if (h->cfg.kernel == AH_KERNEL_PLAIN) {
        if (chosen) *chosen = h->variant;
        return AH_OK;
    }
    cudaEvent_t e0, e1;
    AH_CUDA(cudaEventCreate(&e0));
    AH_CUDA(cudaEventCreate(&e1));
    const int nv = h->two_step ? fused2_variant_count() : n_variants(h->cfg.precision);
    int &var = h->two_step ? h->variant2 : h->variant;
    // one step (a step pair in two-step mode) of the shape being timed
    auto trial = [h]() {
        if (h->two_step) return do_step2(h, 0);
        return h->cfg.precision == AH_FP32 ? do_step<float>(h, 0) : do_step<double>(h, 0);
    };
    int best = -1;
    float best_ms = 0.0f;
    for (int v = 0; v < nv && st == AH_OK; ++v) {
        if (!variant_ok(h, v)) continue;
        var = v;
        // one untimed step (first launch configures the kernel), then trial_steps timed
        st = trial();
        if (st != AH_OK) break;
        cudaEventRecord(e0, h->stream);
        for (int q = 0; q < trial_steps && st == AH_OK; ++q) st = trial();
        cudaEventRecord(e1, h->stream);
        cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) { st = fail(AH_ERR_CUDA, "autotune: %s", cudaGetErrorString(ce)); break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best < 0 || ms < best_ms) { best = v; best_ms = ms; }
        if ((st = check_device_error(h)) != AH_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != AH_OK) return st;
    if (best < 0) return fail(AH_ERR_ARG, "no step shape available for N=%d", h->N);
    var = best;
    tune_cache_put(h, best);
    AH_CUDA(write_initial_state(h));
    AH_CUDA(cudaStreamSynchronize(h->stream));
    if (chosen) *chosen = best;
    return AH_OK;
}

void ah_destroy(ah_sim *h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->aux) {
        cudaStreamSynchronize(h->aux);
        cudaStreamDestroy(h->aux);
    }
    if (h->ev_snap) cudaEventDestroy(h->ev_snap);
    if (h->ev_done) cudaEventDestroy(h->ev_done);
    if (h->dmem) cudaFree(h->dmem);
    if (h->partials) cudaFree(h->partials);
    if (h->list.count) cudaFree(h->list.count);
    if (h->d_err) cudaFree(h->d_err);
    if (h->host_result) cudaFreeHost(h->host_result);
    if (h->stream && h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"
