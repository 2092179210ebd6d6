/*
 * ah_oracle.c -- plain FP64 CPU oracle for the lattice Abelian-Higgs leapfrog
 * and its network diagnostics (Correia & Martins, arXiv:1809.00995, Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file.  The product path
 * (the CUDA library and its binding) never links, loads or calls it, and the
 * two share no code, header, table or helper.
 *
 * Everything is FP64 and goes one site at a time with no tiling, fusion or
 * reordering: each function follows the equation it cites.  Where the paper
 * is silent or inconsistent the reading taken is stated beside the code.
 *
 * Storage: one contiguous double array holding 10 components, each an M^3
 * periodic box with x fastest,
 *     f[c*M^3 + i + M*(j + M*k)],
 *     c = 0 phi.re, 1 phi.im, 2 Pi.re, 3 Pi.im, 4..6 theta_1..3, 7..9 E_1..3,
 * where theta_i = e*dx*A_i is the link phase on the link x -> x+k_i (Eq. 3)
 * and E_i its conjugate.  At integer step n the array holds phi^n, theta^n,
 * Pi^{n-1/2}, E^{n-1/2}.
 *
 * Parity status: every function here is pinned by a CPU test (Philox
 * known-answer vectors, closed-form lattice waves, exact scalar recurrences,
 * Gauss-law conservation, gauge invariance, O(dt^2) energy conservation,
 * analytic string windings, light-cone locality, the compact-theta and
 * core-growth identities, the tension of a Bogomolny string for xi_L); see
 * tests/test_oracle_pins.py; the Philox key/counter layout also equals
 * cuRAND's (tests/test_gpu_curand_layout.py).  The mapping of two Philox
 * words to a uniform double in aho_site_uniform is a convention of this code
 * (the paper draws its phases with cuRAND and states no mapping); it is pinned
 * to its written definition by golden values computed in exact integer
 * arithmetic (tests/golden/make_site_uniform.py) and checked for uniformity.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NCOMP 10
enum { PHR = 0, PHI = 1, PIR = 2, PII = 3, TH = 4, EL = 7 };

typedef struct {
    int64_t N;        /* side of the global periodic lattice (Philox counters) */
    double dx, dt;    /* lattice spacing Delta x, time step Delta eta */
    int32_t era;      /* 0 Minkowski (a=1), 1 radiation (a ~ tau), 2 matter (a ~ tau^2) */
    int32_t flags;    /* bit 0: theta reduced to [-pi, pi] after each drift;
                         bit 1: core growth (exponent s before tau_ref, 1 after) */
    double s;         /* coupling exponent of Eq. 7 */
    double lambda0, e0, sigma;
    double tau0;      /* conformal time at step 0 */
    double tau_ref;   /* a(tau_ref) = 1 */
    uint64_t seed;
} aho_params;

typedef struct {
    double sum_L, sum_rho, sum_p, sum_K, sum_G2, sum_V, sum_Eel, sum_B;
    double sum_KV, sum_G2V, sum_KL, sum_G2L, sum_pL, sum_rhoL;
    double sum_gauss2, max_gauss, sum_gscale2, max_abs_theta;
    int64_t sum_abs_W, n_pierced;
    int64_t sum_abs_W_plane[3];   /* plaquette orientation 12, 13, 23 */
    int64_t sum_W_plane[3];       /* signed sums, same orientations */
    int64_t nonfinite;
    int64_t n_sites;
} aho_diag_out;

/* ------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random
 * numbers: as easy as 1, 2, 3").  One round: two 32x32->64 multiplies by
 * the published constants, the high words XORed with the other two counter
 * words and the key; the key is bumped by the two Weyl constants between
 * rounds. */
void aho_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform u in [0,1) of the global site with linear index idx: Philox with
 * key = (seed lo, seed hi) and counter = (0, 0, idx lo, idx hi); the first
 * two output words give a 53-bit integer, w0 above w1's top 21 bits. */
double aho_site_uniform(uint64_t seed, uint64_t idx)
{
    uint32_t ctr[4] = { 0u, 0u, (uint32_t)idx, (uint32_t)(idx >> 32) };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t w[4];
    aho_philox4x32_10(ctr, key, w);
    uint64_t m = ((uint64_t)w[0] << 21) ^ (uint64_t)(w[1] >> 11);
    return (double)m * (1.0 / 9007199254740992.0);   /* 2^-53 */
}

/* ------------------------------------------------------------------ */
/* Background (Sec. 2, Eq. 7).  a(tau) = (tau/tau_ref)^alpha with alpha 0, 1, 2
 * for Minkowski, radiation, matter; e = e0 a^(s-1), lambda = lambda0 a^(2(s-1)). */
double aho_scale_factor(const aho_params *p, double tau)
{
    double r = tau / p->tau_ref;
    if (p->era == 1) return r;
    if (p->era == 2) return r * r;
    return 1.0;
}
/* Eq. 7.  Under core growth (Sec. 2: the comoving width is grown first, then
 * the true equations are evolved) the exponent is s before tau_ref and 1 from
 * tau_ref on; a(tau_ref) = 1 makes both branches give e0 and lambda0 there. */
static double exponent_s(const aho_params *p, double tau)
{
    return ((p->flags & 2) && tau >= p->tau_ref) ? 1.0 : p->s;
}
static double coupling_e(const aho_params *p, double a, double tau)
{
    return p->e0 * pow(a, exponent_s(p, tau) - 1.0);
}
static double coupling_lambda(const aho_params *p, double a, double tau)
{
    return p->lambda0 * pow(a, 2.0 * (exponent_s(p, tau) - 1.0));
}
/* tau_n = tau0 + n dt, taken from the integer n (never accumulated) */
double aho_tau(const aho_params *p, int64_t n) { return p->tau0 + (double)n * p->dt; }

/* ------------------------------------------------------------------ */
static inline int64_t wrap(int64_t a, int64_t M) { a %= M; return a < 0 ? a + M : a; }
static inline int64_t sidx(int64_t i, int64_t j, int64_t k, int64_t M)
{
    return wrap(i, M) + M * (wrap(j, M) + M * wrap(k, M));
}
/* unit vector k_d, d = 0,1,2 */
static const int UX[3][3] = { {1, 0, 0}, {0, 1, 0}, {0, 0, 1} };

typedef struct { double re, im; } cplx;
static inline cplx cmul(cplx a, cplx b) { cplx r = { a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re }; return r; }
static inline cplx cconj(cplx a) { cplx r = { a.re, -a.im }; return r; }
static inline cplx cexpi(double t) { cplx r = { cos(t), sin(t) }; return r; }

static inline cplx get_phi(const double *f, int64_t M3, int64_t s)
{ cplx r = { f[PHR * M3 + s], f[PHI * M3 + s] }; return r; }
static inline cplx get_pi(const double *f, int64_t M3, int64_t s)
{ cplx r = { f[PIR * M3 + s], f[PII * M3 + s] }; return r; }
static inline double get_th(const double *f, int64_t M3, int d, int64_t s)
{ return f[(TH + d) * M3 + s]; }
static inline double get_E(const double *f, int64_t M3, int d, int64_t s)
{ return f[(EL + d) * M3 + s]; }

/* Plaquette angle Xi_ij at site (x,y,z) (Eq. 3):
 * Xi_ij^x = theta_i^x + theta_j^{x+i} - theta_i^{x+j} - theta_j^x. */
static double plaquette(const double *f, int64_t M, int ii, int jj,
                        int64_t x, int64_t y, int64_t z)
{
    int64_t M3 = M * M * M;
    int64_t s0 = sidx(x, y, z, M);
    int64_t si = sidx(x + UX[ii][0], y + UX[ii][1], z + UX[ii][2], M);
    int64_t sj = sidx(x + UX[jj][0], y + UX[jj][1], z + UX[jj][2], M);
    return get_th(f, M3, ii, s0) + get_th(f, M3, jj, si)
         - get_th(f, M3, ii, sj) - get_th(f, M3, jj, s0);
}

/* ------------------------------------------------------------------ */
/* Initial conditions (Sec. 2): |phi| = sigma with a random phase
 * alpha = 2 pi u, u from Philox by global site index; Pi = theta = E = 0,
 * which satisfies the discrete Gauss law.  The M^3 box holds the global
 * sites ((x0+i) mod N, (y0+j) mod N, (z0+k) mod N): M = N, origin 0 gives
 * the whole lattice; a smaller M gives a window of it. */
void aho_init_box(const aho_params *p, double *f, int64_t M,
                  int64_t x0, int64_t y0, int64_t z0)
{
    int64_t M3 = M * M * M, N = p->N;
    memset(f, 0, sizeof(double) * NCOMP * (size_t)M3);
    for (int64_t k = 0; k < M; ++k)
        for (int64_t j = 0; j < M; ++j)
            for (int64_t i = 0; i < M; ++i) {
                int64_t gi = wrap(x0 + i, N), gj = wrap(y0 + j, N), gk = wrap(z0 + k, N);
                uint64_t gidx = (uint64_t)(gi + N * (gj + N * gk));
                double alpha = 2.0 * M_PI * aho_site_uniform(p->seed, gidx);
                int64_t s = i + M * (j + M * k);
                f[PHR * M3 + s] = p->sigma * cos(alpha);
                f[PHI * M3 + s] = p->sigma * sin(alpha);
            }
}

/* ------------------------------------------------------------------ */
/* Kicks (Eqs. up_pi and up_E) from step n: reads phi^n, theta^n, Pi^{n-1/2},
 * E^{n-1/2} in f; writes Pi^{n+1/2} into pi_new (2*M3) and E^{n+1/2} into
 * e_new (3*M3).  Half-step scale factors are a(tau_n -+ dt/2) evaluated
 * directly, not averaged. */
static void kicks(const aho_params *p, const double *f, int64_t M, int64_t n,
                  double *pi_new, double *e_new)
{
    const int64_t M3 = M * M * M;
    const double dt = p->dt, dx = p->dx, sig2 = p->sigma * p->sigma;
    const double tn = aho_tau(p, n), tm = tn - 0.5 * dt, tp = tn + 0.5 * dt;
    const double an = aho_scale_factor(p, tn), am = aho_scale_factor(p, tm), ap = aho_scale_factor(p, tp);
    const double en = coupling_e(p, an, tn), em = coupling_e(p, am, tm), ep = coupling_e(p, ap, tp);
    const double lam_n = coupling_lambda(p, an, tn);

#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < M; ++z)
        for (int64_t y = 0; y < M; ++y)
            for (int64_t x = 0; x < M; ++x) {
                const int64_t s0 = sidx(x, y, z, M);
                const cplx ph = get_phi(f, M3, s0);
                const cplx pi = get_pi(f, M3, s0);
                const double mod2 = ph.re * ph.re + ph.im * ph.im;

                /* Eq. up_pi: covariant Laplacian sum_j (U_j^x phi^{x+j} - 2 phi^x
                 * + conj(U_j^{x-j}) phi^{x-j}), U = exp(+i theta). */
                cplx lap = { 0.0, 0.0 };
                for (int d = 0; d < 3; ++d) {
                    int64_t sp = sidx(x + UX[d][0], y + UX[d][1], z + UX[d][2], M);
                    int64_t sm = sidx(x - UX[d][0], y - UX[d][1], z - UX[d][2], M);
                    cplx fwd = cmul(cexpi(get_th(f, M3, d, s0)), get_phi(f, M3, sp));
                    cplx bwd = cmul(cconj(cexpi(get_th(f, M3, d, sm))), get_phi(f, M3, sm));
                    lap.re += fwd.re - 2.0 * ph.re + bwd.re;
                    lap.im += fwd.im - 2.0 * ph.im + bwd.im;
                }
                const double c_damp = (am / ap) * (am / ap);
                const double c_pot = dt * (an * an / ap) * (an * an / ap) * lam_n / 2.0;
                const double c_lap = dt / (dx * dx) * (an / ap) * (an / ap);
                pi_new[s0]      = c_damp * pi.re - c_pot * (mod2 - sig2) * ph.re + c_lap * lap.re;
                pi_new[M3 + s0] = c_damp * pi.im - c_pot * (mod2 - sig2) * ph.im + c_lap * lap.im;

                /* Eq. up_E for each direction i */
                for (int i = 0; i < 3; ++i) {
                    int64_t si = sidx(x + UX[i][0], y + UX[i][1], z + UX[i][2], M);
                    /* current Im[ conj(phi^{x+i}) exp(-i theta_i^x) phi^x ] */
                    cplx t = cmul(cmul(cconj(get_phi(f, M3, si)), cconj(cexpi(get_th(f, M3, i, s0)))), ph);
                    /* curl: sum_{j != i} [ sin Xi_ij^x - sin Xi_ij^{x-j} ] */
                    double curl = 0.0;
                    for (int j = 0; j < 3; ++j) {
                        if (j == i) continue;
                        double xi0 = plaquette(f, M, i, j, x, y, z);
                        double xim = plaquette(f, M, i, j, x - UX[j][0], y - UX[j][1], z - UX[j][2]);
                        curl += sin(xi0) - sin(xim);
                    }
                    const double c_edamp = (ep / em) * (ep / em);
                    const double c_cur = 2.0 * dt * an * an * ep * ep;
                    const double c_curl = dt / (dx * dx) * (ep / en) * (ep / en);
                    e_new[i * M3 + s0] = c_edamp * get_E(f, M3, i, s0) + c_cur * t.im - c_curl * curl;
                }
            }
}

/* A link phase only enters through U = e^{i theta}, so theta and theta - 2 pi k
 * describe the same configuration: the compact reading keeps theta in
 * [-pi, pi] by subtracting 2 pi times the nearest integer to theta / 2 pi
 * whenever |theta| > pi. */
static double wrap_phase(double t)
{
    const double two_pi = 6.283185307179586476925287;
    if (fabs(t) > 0.5 * two_pi) t -= two_pi * nearbyint(t / two_pi);
    return t;
}

/* One leapfrog step n -> n+1 (Eqs. up_pi, up_E, up_phi, up_A): both kicks
 * read only step-n data, then phi += dt Pi^{n+1/2}, theta += dt E^{n+1/2}.
 * theta is non-compact (never wrapped) unless flag bit 0 is set. */
int aho_step(const aho_params *p, double *f, int64_t M, int64_t n)
{
    const int64_t M3 = M * M * M;
    double *pi_new = (double *)malloc(sizeof(double) * 2 * (size_t)M3);
    double *e_new = (double *)malloc(sizeof(double) * 3 * (size_t)M3);
    if (!pi_new || !e_new) { free(pi_new); free(e_new); return -1; }
    kicks(p, f, M, n, pi_new, e_new);
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < M3; ++s) {
        f[PIR * M3 + s] = pi_new[s];
        f[PII * M3 + s] = pi_new[M3 + s];
        for (int d = 0; d < 3; ++d) f[(EL + d) * M3 + s] = e_new[d * M3 + s];
        f[PHR * M3 + s] += p->dt * pi_new[s];
        f[PHI * M3 + s] += p->dt * pi_new[M3 + s];
        for (int d = 0; d < 3; ++d) {
            f[(TH + d) * M3 + s] += p->dt * e_new[d * M3 + s];
            if (p->flags & 1) f[(TH + d) * M3 + s] = wrap_phase(f[(TH + d) * M3 + s]);
        }
    }
    free(pi_new);
    free(e_new);
    return 0;
}

int aho_evolve(const aho_params *p, double *f, int64_t M, int64_t n0, int64_t nsteps)
{
    for (int64_t n = n0; n < n0 + nsteps; ++n)
        if (aho_step(p, f, M, n) != 0) return -1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Compensated (Neumaier) summation: the diagnostics are sums over up to
 * 10^9 sites, kept accurate to a few ulps of the result. */
typedef struct { double s, c; } ksum;
static inline void kadd(ksum *k, double v)
{
    double t = k->s + v;
    if (fabs(k->s) >= fabs(v)) k->c += (k->s - t) + v;
    else k->c += (v - t) + k->s;
    k->s = t;
}
static inline double kval(const ksum *k) { return k->s + k->c; }

/* Arg z in (-pi, pi]: the branch value -pi (from a negative zero imaginary
 * part) is mapped to +pi. */
static double arg_pi(cplx z)
{
    double a = atan2(z.im, z.re);
    return a == -M_PI ? M_PI : a;
}

/* Gauge-covariant edge product z = conj(phi^a) exp(i theta) phi^b on the
 * link a -> b = a + k_d. */
static cplx edge(const double *f, int64_t M, int d, int64_t x, int64_t y, int64_t z)
{
    int64_t M3 = M * M * M;
    int64_t sa = sidx(x, y, z, M);
    int64_t sb = sidx(x + UX[d][0], y + UX[d][1], z + UX[d][2], M);
    return cmul(cmul(cconj(get_phi(f, M3, sa)), cexpi(get_th(f, M3, d, sa))), get_phi(f, M3, sb));
}

/* Winding through plaquette (i,j) at site (x,y,z) (Eq. 9).  With
 * Y_e = [arg phi^b - arg phi^a + theta_e]_pi - theta_e, the bracket is Arg of
 * the edge product z_e, so 2 pi W = A_1 + A_2 - A_3 - A_4 - Xi.  theta is
 * non-compact, so Xi is replaced by its reduced value Arg(z_1 z_2 z_3* z_4*)
 * = [Xi]_pi: this equals the paper's W whenever |Xi| < pi and is invariant
 * under theta -> theta + 2 pi.  The result is an exact integer up to
 * rounding and is rounded to the nearest one. */
static int64_t winding(const double *f, int64_t M, int ii, int jj,
                       int64_t x, int64_t y, int64_t z)
{
    cplx z1 = edge(f, M, ii, x, y, z);                                   /* x -> x+i       */
    cplx z2 = edge(f, M, jj, x + UX[ii][0], y + UX[ii][1], z + UX[ii][2]); /* x+i -> x+i+j */
    cplx z3 = edge(f, M, ii, x + UX[jj][0], y + UX[jj][1], z + UX[jj][2]); /* x+j -> x+i+j */
    cplx z4 = edge(f, M, jj, x, y, z);                                   /* x -> x+j       */
    cplx prod = cmul(cmul(cmul(z1, z2), cconj(z3)), cconj(z4));
    double tot = arg_pi(z1) + arg_pi(z2) - arg_pi(z3) - arg_pi(z4) - arg_pi(prod);
    return (int64_t)llround(tot / (2.0 * M_PI));
}

/* Network diagnostics at integer step n over the sub-box
 * [bx0, bx0+bnx) x [by0, by0+bny) x [bz0, bz0+bnz) of the periodic M^3 box
 * (Sec. 2, Eqs. 2, defXiV2, defR, 9, defEoS).  Per site, with a, e, lambda at
 * tau_n:
 *   K = |Pi|^2,  G2 = |D phi|^2 = dx^-2 sum_i |U_i^x phi^{x+i} - phi^x|^2,
 *   V = (a^2 lambda / 4)(|phi|^2 - sigma^2)^2,
 *   Eel = sum_i E_i^2 / (2 e^2 a^2 dx^2),
 *   B = sum_{i<j} (1 - cos Xi_ij) / (e^2 a^2 dx^4),
 *   L = K - G2 - V + Eel - B   (Eq. 2 divided by a^2; the magnetic
 *       coefficient is the one the E-kick curl implies, twice the printed one),
 *   rho = K + G2 + V + Eel + B,  p = K - G2/3 - V + (Eel + B)/3.
 * Gauss residual (conserved by the scheme; a and e at tau_{n-1/2}):
 *   G = e_-^-2 sum_i (E_i^x - E_i^{x-i}) + 2 dx^2 a_-^2 Im(conj(phi^x) Pi^x),
 *   scale = |first term| + |second term|.
 * Windings are summed over the three plaquettes (12, 13, 23) based at each
 * site of the sub-box. */
void aho_diag(const aho_params *p, const double *f, int64_t M, int64_t n,
              int64_t bx0, int64_t by0, int64_t bz0,
              int64_t bnx, int64_t bny, int64_t bnz, aho_diag_out *out)
{
    const int64_t M3 = M * M * M;
    const double dx = p->dx, sig2 = p->sigma * p->sigma;
    const double tn = aho_tau(p, n), tm = tn - 0.5 * p->dt;
    const double an = aho_scale_factor(p, tn), am = aho_scale_factor(p, tm);
    const double en = coupling_e(p, an, tn), em = coupling_e(p, am, tm);
    const double lam_n = coupling_lambda(p, an, tn);
    const double e2a2 = en * en * an * an;

    /* per-plane partial sums, combined in plane order: the result does not
     * depend on the thread count */
    enum { NS = 17 };
    ksum *part = (ksum *)calloc((size_t)bnz * NS, sizeof(ksum));
    double *pmax = (double *)calloc((size_t)bnz * 2, sizeof(double));
    int64_t *pint = (int64_t *)calloc((size_t)bnz * 9, sizeof(int64_t));

#pragma omp parallel for schedule(static)
    for (int64_t kz = 0; kz < bnz; ++kz) {
        ksum *ps = part + kz * NS;
        double *pm = pmax + kz * 2;
        int64_t *pi_ = pint + kz * 9;
        for (int64_t ky = 0; ky < bny; ++ky)
            for (int64_t kx = 0; kx < bnx; ++kx) {
                const int64_t x = bx0 + kx, y = by0 + ky, z = bz0 + kz;
                const int64_t s0 = sidx(x, y, z, M);
                const cplx ph = get_phi(f, M3, s0);
                const cplx pi = get_pi(f, M3, s0);
                const double mod2 = ph.re * ph.re + ph.im * ph.im;

                double K = pi.re * pi.re + pi.im * pi.im;
                double G2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    int64_t sp = sidx(x + UX[d][0], y + UX[d][1], z + UX[d][2], M);
                    cplx up = cmul(cexpi(get_th(f, M3, d, s0)), get_phi(f, M3, sp));
                    double dre = up.re - ph.re, dim = up.im - ph.im;
                    G2 += dre * dre + dim * dim;
                }
                G2 /= dx * dx;
                double V = an * an * lam_n / 4.0 * (mod2 - sig2) * (mod2 - sig2);
                double Esq = 0.0;
                for (int d = 0; d < 3; ++d) Esq += get_E(f, M3, d, s0) * get_E(f, M3, d, s0);
                double Eel = Esq / (2.0 * e2a2 * dx * dx);
                double Bsum = 0.0;
                for (int i = 0; i < 3; ++i)
                    for (int j = i + 1; j < 3; ++j)
                        Bsum += 1.0 - cos(plaquette(f, M, i, j, x, y, z));
                double B = Bsum / (e2a2 * dx * dx * dx * dx);
                double L = K - G2 - V + Eel - B;
                double rho = K + G2 + V + Eel + B;
                double pr = K - G2 / 3.0 - V + (Eel + B) / 3.0;

                double div = 0.0;
                for (int d = 0; d < 3; ++d) {
                    int64_t sm = sidx(x - UX[d][0], y - UX[d][1], z - UX[d][2], M);
                    div += get_E(f, M3, d, s0) - get_E(f, M3, d, sm);
                }
                double g1 = div / (em * em);
                double g2 = 2.0 * dx * dx * am * am * (ph.re * pi.im - ph.im * pi.re);
                double G = g1 + g2, gs = fabs(g1) + fabs(g2);

                double vals[NS] = { L, rho, pr, K, G2, V, Eel, B,
                                    K * V, G2 * V, K * L, G2 * L, pr * L, rho * L,
                                    G * G, gs * gs, 0.0 };
                for (int q = 0; q < NS - 1; ++q) kadd(&ps[q], vals[q]);
                if (fabs(G) > pm[0]) pm[0] = fabs(G);
                double mt = 0.0;
                for (int d = 0; d < 3; ++d) if (fabs(get_th(f, M3, d, s0)) > mt) mt = fabs(get_th(f, M3, d, s0));
                if (mt > pm[1]) pm[1] = mt;
                int bad = !isfinite(rho) || !isfinite(pr) || !isfinite(L) || !isfinite(G);
                pi_[8] += bad;

                int q = 0;
                for (int i = 0; i < 3; ++i)
                    for (int j = i + 1; j < 3; ++j, ++q) {
                        int64_t w = winding(f, M, i, j, x, y, z);
                        pi_[q] += w < 0 ? -w : w;
                        pi_[3 + q] += w;
                        pi_[6] += w != 0;
                    }
            }
    }

    memset(out, 0, sizeof(*out));
    ksum tot[NS];
    memset(tot, 0, sizeof(tot));
    for (int64_t kz = 0; kz < bnz; ++kz) {
        for (int q = 0; q < NS - 1; ++q) {
            kadd(&tot[q], part[kz * NS + q].s);
            kadd(&tot[q], part[kz * NS + q].c);
        }
        if (pmax[kz * 2] > out->max_gauss) out->max_gauss = pmax[kz * 2];
        if (pmax[kz * 2 + 1] > out->max_abs_theta) out->max_abs_theta = pmax[kz * 2 + 1];
        for (int q = 0; q < 3; ++q) {
            out->sum_abs_W_plane[q] += pint[kz * 9 + q];
            out->sum_W_plane[q] += pint[kz * 9 + 3 + q];
        }
        out->n_pierced += pint[kz * 9 + 6];
        out->nonfinite += pint[kz * 9 + 8];
    }
    out->sum_L = kval(&tot[0]);   out->sum_rho = kval(&tot[1]); out->sum_p = kval(&tot[2]);
    out->sum_K = kval(&tot[3]);   out->sum_G2 = kval(&tot[4]);  out->sum_V = kval(&tot[5]);
    out->sum_Eel = kval(&tot[6]); out->sum_B = kval(&tot[7]);
    out->sum_KV = kval(&tot[8]);  out->sum_G2V = kval(&tot[9]); out->sum_KL = kval(&tot[10]);
    out->sum_G2L = kval(&tot[11]); out->sum_pL = kval(&tot[12]); out->sum_rhoL = kval(&tot[13]);
    out->sum_gauss2 = kval(&tot[14]); out->sum_gscale2 = kval(&tot[15]);
    out->sum_abs_W = out->sum_abs_W_plane[0] + out->sum_abs_W_plane[1] + out->sum_abs_W_plane[2];
    out->n_sites = bnx * bny * bnz;
    free(part);
    free(pmax);
    free(pint);
}

/* Time-centred total energy at step n (used in Minkowski, a = 1):
 * dx^3 sum_x [ (|Pi^-|^2 + |Pi^+|^2)/2 + G2 + V + (E^-^2 + E^+^2)/(4 e^2 a^2 dx^2)
 * + sum_{i<j}(1 - cos Xi)/(e^2 a^2 dx^4) ], with Pi^+, E^+ from the kicks of
 * step n.  This is the Hamiltonian whose Hamilton equations are Eqs. up_pi and
 * up_E at a = 1; the leapfrog keeps it to O(dt^2). */
double aho_energy(const aho_params *p, const double *f, int64_t M, int64_t n)
{
    const int64_t M3 = M * M * M;
    double *pi_new = (double *)malloc(sizeof(double) * 2 * (size_t)M3);
    double *e_new = (double *)malloc(sizeof(double) * 3 * (size_t)M3);
    if (!pi_new || !e_new) { free(pi_new); free(e_new); return NAN; }
    kicks(p, f, M, n, pi_new, e_new);
    aho_diag_out d;
    aho_diag(p, f, M, n, 0, 0, 0, M, M, M, &d);
    const double tn = aho_tau(p, n), an = aho_scale_factor(p, tn);
    const double en = coupling_e(p, an, tn), dx = p->dx;
    ksum kin = { 0.0, 0.0 }, el = { 0.0, 0.0 };
    for (int64_t s = 0; s < M3; ++s) {
        double k1 = f[PIR * M3 + s] * f[PIR * M3 + s] + f[PII * M3 + s] * f[PII * M3 + s];
        double k2 = pi_new[s] * pi_new[s] + pi_new[M3 + s] * pi_new[M3 + s];
        kadd(&kin, 0.5 * (k1 + k2));
        for (int d = 0; d < 3; ++d) {
            double e1 = f[(EL + d) * M3 + s], e2 = e_new[d * M3 + s];
            kadd(&el, 0.5 * (e1 * e1 + e2 * e2) / (2.0 * en * en * an * an * dx * dx));
        }
    }
    free(pi_new);
    free(e_new);
    return dx * dx * dx * (kval(&kin) + d.sum_G2 + d.sum_V + kval(&el) + d.sum_B);
}

/* Lattice gauge transform by angles alpha (M^3) (Eq. 3 invariance):
 * phi -> e^{i alpha_x} phi, Pi -> e^{i alpha_x} Pi,
 * theta_i^x -> theta_i^x + alpha_x - alpha_{x+i}, E unchanged. */
void aho_gauge_transform(double *f, int64_t M, const double *alpha)
{
    const int64_t M3 = M * M * M;
    double *th_new = (double *)malloc(sizeof(double) * 3 * (size_t)M3);
    for (int64_t z = 0; z < M; ++z)
        for (int64_t y = 0; y < M; ++y)
            for (int64_t x = 0; x < M; ++x) {
                int64_t s0 = sidx(x, y, z, M);
                for (int d = 0; d < 3; ++d) {
                    int64_t sp = sidx(x + UX[d][0], y + UX[d][1], z + UX[d][2], M);
                    th_new[d * M3 + s0] = get_th(f, M3, d, s0) + alpha[s0] - alpha[sp];
                }
            }
    for (int64_t s = 0; s < M3; ++s) {
        cplx g = cexpi(alpha[s]);
        cplx ph = cmul(g, get_phi(f, M3, s)), pi = cmul(g, get_pi(f, M3, s));
        f[PHR * M3 + s] = ph.re; f[PHI * M3 + s] = ph.im;
        f[PIR * M3 + s] = pi.re; f[PII * M3 + s] = pi.im;
        for (int d = 0; d < 3; ++d) f[(TH + d) * M3 + s] = th_new[d * M3 + s];
    }
    free(th_new);
}

/* Per-site winding numbers of the three plaquette orientations (12, 13, 23),
 * written to w (3*M^3, int8), for tests that compare them site by site. */
void aho_windings(const double *f, int64_t M, int8_t *w)
{
    const int64_t M3 = M * M * M;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < M; ++z)
        for (int64_t y = 0; y < M; ++y)
            for (int64_t x = 0; x < M; ++x) {
                int64_t s0 = sidx(x, y, z, M);
                int q = 0;
                for (int i = 0; i < 3; ++i)
                    for (int j = i + 1; j < 3; ++j, ++q)
                        w[q * M3 + s0] = (int8_t)winding(f, M, i, j, x, y, z);
            }
}

int aho_abi_version(void) { return 1; }
