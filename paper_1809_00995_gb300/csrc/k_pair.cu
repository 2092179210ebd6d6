// k_pair.cu -- fused leapfrog step with paired FP32 arithmetic (sm_100+ FFMA2).
//
// Same update as k_fused.cu (Eqs. up_pi, up_E, up_phi, up_A of
// arXiv:1809.00995 in one z-marching kernel, link exponentials once per site,
// plaquette sines once per plaquette, phi/theta ping-pong), arranged so that
// every lane works on two x-adjacent sites at once and every floating-point
// operation is a packed two-wide one (__ffma2_rn, __fmul2_rn, __fadd2_rn),
// halving the instructions issued per site -- the kernel is issue-bound, not
// bandwidth-bound, in its scalar form.
//
// Geometry: an extended row holds 64 sites (32 lane pairs): 62 own columns
// plus the two halo columns, so the tile is 62 x TY own sites and its extended
// tile is 64 x (TY + 2).  Warp w works on extended row w for the link
// exponentials (all warps) and the plaquettes (rows 0..TY), and warps 1..TY
// update their own row.  Tiles start at x = 62 bx + 1 so that every pair
// starts at an even x: global accesses are 8-byte vector loads and stores,
// and pairs never straddle the periodic seam (N even).  Sites past the end
// of a ragged tile are computed but never stored.
//
// Per plane z: B(z) plaquettes of plane z -> barrier -> C(z) update of plane z
// and A(z+2) link exponentials of plane z+2 -> barrier, with three-plane rings
// of U and phi in shared memory; the next plane's fields are prefetched into
// registers one plane ahead.
#include "ah_internal.cuh"

namespace ah {
namespace {

constexpr int EXW = 64;            // sites per extended row
constexpr int OWNW = 62;           // own sites per row

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// two complex numbers (one per site of the pair)
struct Z2 { float2 r, i; };
__device__ __forceinline__ Z2 zmul(Z2 a, Z2 b)
{
    return { fma2(a.r, b.r, mul2(neg2(a.i), b.i)), fma2(a.r, b.i, mul2(a.i, b.r)) };
}
__device__ __forceinline__ Z2 zconj(Z2 a) { return { a.r, neg2(a.i) }; }
// Im(a b conj(c) conj(d)) = Im((a b) conj(c d))
__device__ __forceinline__ float2 zplaq(Z2 a, Z2 b, Z2 c, Z2 d)
{
    const Z2 ab = zmul(a, b), cd = zmul(c, d);
    return fma2(ab.i, cd.r, mul2(neg2(ab.r), cd.i));
}

// Sine and cosine of a pair of link phases: the method of sincos32.cuh (Cody-Waite
// reduction with pi/2 = P1 + P2 + P3, Taylor polynomials through r^9 and r^10 on
// |r| <= pi/4) in packed form.  k = nearest integer to t 2/pi comes from adding
// 1.5 * 2^23, whose low mantissa bits then hold k mod 2^22.  Valid for |t| < 2^17;
// larger phases take the library sincosf.
__device__ __forceinline__ void sincos_pair(float2 t, float2 *s, float2 *c)
{
    if (!(fabsf(t.x) < 131072.0f && fabsf(t.y) < 131072.0f)) {
        sincosf(t.x, &s->x, &c->x);
        sincosf(t.y, &s->y, &c->y);
        return;
    }
    const float2 magic = f2(12582912.0f);                  // 1.5 * 2^23
    const float2 kb = fma2(t, f2(0x1.45f306p-1f), magic);  // t 2/pi + magic
    const int qx = __float_as_int(kb.x), qy = __float_as_int(kb.y);
    const float2 kf = sub2(kb, magic);
    float2 r = fma2(neg2(kf), f2(0x1.921fb6p+0f), t);
    r = fma2(neg2(kf), f2(-0x1.777a5cp-25f), r);
    r = fma2(neg2(kf), f2(-0x1.ee59dap-50f), r);
    const float2 r2 = mul2(r, r);
    float2 ps = fma2(r2, f2(2.755731884e-06f), f2(-1.984127011e-04f));
    ps = fma2(r2, ps, f2(8.333333768e-03f));
    ps = fma2(r2, ps, f2(-1.666666716e-01f));
    const float2 sr = fma2(mul2(r, r2), ps, r);
    float2 pc = fma2(r2, f2(-2.755731998e-07f), f2(2.480158764e-05f));
    pc = fma2(r2, pc, f2(-1.388888923e-03f));
    pc = fma2(r2, pc, f2(4.166666791e-02f));
    pc = fma2(r2, pc, f2(-0.5f));
    const float2 cr = fma2(r2, pc, f2(1.0f));
    const float ax = (qx & 1) ? cr.x : sr.x, bx = (qx & 1) ? sr.x : cr.x;
    const float ay = (qy & 1) ? cr.y : sr.y, by = (qy & 1) ? sr.y : cr.y;
    s->x = (qx & 2) ? -ax : ax;
    s->y = (qy & 2) ? -ay : ay;
    c->x = ((qx + 1) & 2) ? -bx : bx;
    c->y = ((qy + 1) & 2) ? -by : by;
}

__device__ __forceinline__ int wrapm(int a, int N) { a %= N; return a < 0 ? a + N : a; }
__device__ __forceinline__ float2 ldg2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void stg2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }

template <int TY>
struct PGeo {
    static constexpr int EY = TY + 2, NT = 32 * EY;
    static constexpr int ROWS = EY * EXW;              // floats of one planar field plane
    static constexpr int PLANE = 8 * ROWS;             // Ur[3], Ui[3], Fr, Fi
    static constexpr int PROWS = (TY + 1) * EXW;       // plaquette plane (rows 0..TY)
    static constexpr size_t smem = sizeof(float) * (3 * PLANE + 3 * PROWS);
};

template <int TY, int MINB>
__global__ void __launch_bounds__(32 * (TY + 2), MINB)
k_pair(View<float> v, int N, int zc, KickCoef<float> c)
{
    using G = PGeo<TY>;
    constexpr int ROWS = G::ROWS, PLANE = G::PLANE, PROWS = G::PROWS;
    extern __shared__ __align__(16) float sm[];
    float *const ring = sm;                     // [3][PLANE]
    float *const sP = sm + 3 * PLANE;           // [3][PROWS]: sin Xi_12, _13, _23

    const int lane = threadIdx.x & 31, ey = threadIdx.x >> 5;
    const int xs = OWNW * blockIdx.x + 2 * lane;        // unwrapped x of the pair's first site
    const int y0 = TY * blockIdx.y;
    const int z0 = blockIdx.z * zc;
    if (z0 >= N) return;
    const int z1 = min(z0 + zc, N);
    const long long NN = (long long)N * N;
    const int rowoff = wrapm(xs, N) + N * wrapm(y0 + ey - 1, N);   // in-plane offset of the pair
    const bool own_row = ey >= 1 && ey <= TY && y0 + ey - 1 < N;
    // own sites of the pair: ex = 2 lane (+1) in [1, 62] and unwrapped x <= N
    const bool okx = lane > 0 && xs <= N;
    const bool oky = lane < 31 && xs + 1 <= N;
    const int ep = ey * EXW + 2 * lane;          // pair slot in an extended plane
    const int pp = ey * EXW + 2 * lane;          // pair slot in a plaquette plane

    auto Ur = [&](int slot, int d) { return ring + slot * PLANE + d * ROWS; };
    auto Ui = [&](int slot, int d) { return ring + slot * PLANE + (3 + d) * ROWS; };
    auto Fr = [&](int slot) { return ring + slot * PLANE + 6 * ROWS; };
    auto Fi = [&](int slot) { return ring + slot * PLANE + 7 * ROWS; };
    auto ld2 = [](const float *p, int i) { return *reinterpret_cast<const float2 *>(p + i); };
    auto st2 = [](float *p, int i, float2 x) { *reinterpret_cast<float2 *>(p + i) = x; };

    // prefetched phi, theta of one plane for this lane's pair
    float2 q_t1, q_t2, q_t3, q_fr, q_fi;
    auto load_plane = [&](int z) {
        const long long s = (long long)wrapm(z, N) * NN + rowoff;
        q_t1 = ldg2(v.th1 + s); q_t2 = ldg2(v.th2 + s); q_t3 = ldg2(v.th3 + s);
        q_fr = ldg2(v.phr + s); q_fi = ldg2(v.phi + s);
    };
    // A: links and phi of the prefetched plane into ring slot `slot`
    auto phase_A = [&](int slot) {
        float2 sn, cs;
        sincos_pair(q_t1, &sn, &cs); st2(Ur(slot, 0), ep, cs); st2(Ui(slot, 0), ep, sn);
        sincos_pair(q_t2, &sn, &cs); st2(Ur(slot, 1), ep, cs); st2(Ui(slot, 1), ep, sn);
        sincos_pair(q_t3, &sn, &cs); st2(Ur(slot, 2), ep, cs); st2(Ui(slot, 2), ep, sn);
        st2(Fr(slot), ep, q_fr);
        st2(Fi(slot), ep, q_fi);
    };
    auto U = [&](int slot, int d, int i) { return Z2{ ld2(Ur(slot, d), i), ld2(Ui(slot, d), i) }; };
    // pair (i+1, i+2) from the pair (i, i+1) already in hand and the scalar at i+2
    auto Zright = [&](int slot, int d, Z2 own, int i) {
        return Z2{ make_float2(own.r.y, Ur(slot, d)[i + 2]), make_float2(own.i.y, Ui(slot, d)[i + 2]) };
    };
    auto Zleft = [&](int slot, int d, Z2 own, int i) {
        return Z2{ make_float2(Ur(slot, d)[i - 1], own.r.x), make_float2(Ui(slot, d)[i - 1], own.i.x) };
    };

    // own-pair registers carried along z
    Z2 ph_m, u3_m;
    float2 p13_m, p23_m;
    float2 th_a1, th_a2, th_a3, th_b1, th_b2, th_b3;   // theta of planes z and z+1

    // prologue: link planes z0-1 (slot 0), z0 (slot 1), z0+1 (slot 2)
    load_plane(z0 - 1);
    phase_A(0);
    ph_m = Z2{ q_fr, q_fi };
    load_plane(z0);
    phase_A(1);
    th_a1 = q_t1; th_a2 = q_t2; th_a3 = q_t3;
    load_plane(z0 + 1);
    phase_A(2);
    th_b1 = q_t1; th_b2 = q_t2; th_b3 = q_t3;
    load_plane(z0 + 2);
    __syncthreads();
    if (own_row) {
        const Z2 u1 = U(0, 0, ep), u3 = U(0, 2, ep), u2 = U(0, 1, ep);
        u3_m = u3;
        p13_m = zplaq(u1, Zright(0, 2, u3, ep), U(1, 0, ep), u3);
        p23_m = zplaq(u2, U(0, 2, ep + EXW), U(1, 1, ep), u3);
    }

    for (int k = 0; z0 + k < z1; ++k) {
        const int z = z0 + k;
        const int sc = (k + 1) % 3, sn = (k + 2) % 3, sa = k % 3;   // slots of planes z, z+1, z+2
        const long long base = (long long)z * NN;
        // Pi, E of plane z for the own pair (consumed after one barrier)
        float2 pr = make_float2(0.f, 0.f), pim = pr, e1 = pr, e2 = pr, e3 = pr;
        if (own_row) {
            const long long s = base + rowoff;
            pr = ldg2(v.pir + s); pim = ldg2(v.pii + s);
            e1 = ldg2(v.e1 + s); e2 = ldg2(v.e2 + s); e3 = ldg2(v.e3 + s);
        }
        // B: plaquette sines of plane z on rows 0..TY
        float2 p12 = make_float2(0.f, 0.f), p13 = p12, p23 = p12;
        if (ey <= TY) {
            const Z2 u1 = U(sc, 0, ep), u2 = U(sc, 1, ep), u3 = U(sc, 2, ep);
            p12 = zplaq(u1, Zright(sc, 1, u2, ep), U(sc, 0, ep + EXW), u2);
            p13 = zplaq(u1, Zright(sc, 2, u3, ep), U(sn, 0, ep), u3);
            p23 = zplaq(u2, U(sc, 2, ep + EXW), U(sn, 1, ep), u3);
            st2(sP, pp, p12);
            st2(sP + PROWS, pp, p13);
            st2(sP + 2 * PROWS, pp, p23);
        }
        __syncthreads();

        // C: kicks and drifts of the own pair of plane z
        if (own_row) {
            const Z2 f0{ ld2(Fr(sc), ep), ld2(Fi(sc), ep) };
            const Z2 fxp{ make_float2(f0.r.y, Fr(sc)[ep + 2]), make_float2(f0.i.y, Fi(sc)[ep + 2]) };
            const Z2 fxm{ make_float2(Fr(sc)[ep - 1], f0.r.x), make_float2(Fi(sc)[ep - 1], f0.i.x) };
            const Z2 fyp{ ld2(Fr(sc), ep + EXW), ld2(Fi(sc), ep + EXW) };
            const Z2 fym{ ld2(Fr(sc), ep - EXW), ld2(Fi(sc), ep - EXW) };
            const Z2 fzp{ ld2(Fr(sn), ep), ld2(Fi(sn), ep) };
            const Z2 u1 = U(sc, 0, ep), u2 = U(sc, 1, ep), u3 = U(sc, 2, ep);
            const Z2 u1m = Zleft(sc, 0, u1, ep), u2m = U(sc, 1, ep - EXW);
            // forward U_d phi^{x+d}, backward conj(U_d^{x-d}) phi^{x-d}
            const Z2 w1 = zmul(u1, fxp), w2 = zmul(u2, fyp), w3 = zmul(u3, fzp);
            const Z2 b1 = zmul(zconj(u1m), fxm), b2 = zmul(zconj(u2m), fym), b3 = zmul(zconj(u3_m), ph_m);
            const float2 six = f2(6.0f);
            const float2 lr = fma2(neg2(six), f0.r, add2(add2(add2(w1.r, b1.r), add2(w2.r, b2.r)), add2(w3.r, b3.r)));
            const float2 li = fma2(neg2(six), f0.i, add2(add2(add2(w1.i, b1.i), add2(w2.i, b2.i)), add2(w3.i, b3.i)));
            const float2 mod2 = fma2(f0.r, f0.r, mul2(f0.i, f0.i));
            const float2 pot = mul2(f2(c.c_pot), sub2(mod2, f2(c.sigma2)));
            const float2 npr = fma2(f2(c.c_lap), lr, fma2(f2(c.c_damp), pr, mul2(neg2(pot), f0.r)));
            const float2 npi = fma2(f2(c.c_lap), li, fma2(f2(c.c_damp), pim, mul2(neg2(pot), f0.i)));
            // currents Im[conj(U_i phi^{x+i}) phi^x]
            const float2 cu1 = fma2(w1.r, f0.i, mul2(neg2(w1.i), f0.r));
            const float2 cu2 = fma2(w2.r, f0.i, mul2(neg2(w2.i), f0.r));
            const float2 cu3 = fma2(w3.r, f0.i, mul2(neg2(w3.i), f0.r));
            // curls with sin Xi_ji = -sin Xi_ij
            const float2 p12xm = make_float2(sP[pp - 1], p12.x);
            const float2 p13xm = make_float2(sP[PROWS + pp - 1], p13.x);
            const float2 p12ym = ld2(sP, pp - EXW);
            const float2 p23ym = ld2(sP + 2 * PROWS, pp - EXW);
            const float2 cl1 = add2(sub2(p12, p12ym), sub2(p13, p13_m));
            const float2 cl2 = add2(sub2(p12xm, p12), sub2(p23, p23_m));
            const float2 cl3 = add2(sub2(p13xm, p13), sub2(p23ym, p23));
            const float2 ne1 = fma2(f2(-c.c_curl), cl1, fma2(f2(c.c_edamp), e1, mul2(f2(c.c_cur), cu1)));
            const float2 ne2 = fma2(f2(-c.c_curl), cl2, fma2(f2(c.c_edamp), e2, mul2(f2(c.c_cur), cu2)));
            const float2 ne3 = fma2(f2(-c.c_curl), cl3, fma2(f2(c.c_edamp), e3, mul2(f2(c.c_cur), cu3)));
            const float2 dt = f2(c.dt);
            const float2 ofr = fma2(dt, npr, f0.r), ofi = fma2(dt, npi, f0.i);
            float2 ot1 = fma2(dt, ne1, th_a1), ot2 = fma2(dt, ne2, th_a2), ot3 = fma2(dt, ne3, th_a3);
            if (c.wrap) {
                ot1 = make_float2(wrap_phase(ot1.x), wrap_phase(ot1.y));
                ot2 = make_float2(wrap_phase(ot2.x), wrap_phase(ot2.y));
                ot3 = make_float2(wrap_phase(ot3.x), wrap_phase(ot3.y));
            }
            const long long s = base + rowoff;
            if (okx && oky) {
                stg2(v.pir + s, npr); stg2(v.pii + s, npi);
                stg2(v.e1 + s, ne1); stg2(v.e2 + s, ne2); stg2(v.e3 + s, ne3);
                stg2(v.ophr + s, ofr); stg2(v.ophi + s, ofi);
                stg2(v.oth1 + s, ot1); stg2(v.oth2 + s, ot2); stg2(v.oth3 + s, ot3);
            } else {
                if (okx) {
                    v.pir[s] = npr.x; v.pii[s] = npi.x; v.e1[s] = ne1.x; v.e2[s] = ne2.x; v.e3[s] = ne3.x;
                    v.ophr[s] = ofr.x; v.ophi[s] = ofi.x; v.oth1[s] = ot1.x; v.oth2[s] = ot2.x; v.oth3[s] = ot3.x;
                }
                if (oky) {
                    const long long s1 = s + 1;
                    v.pir[s1] = npr.y; v.pii[s1] = npi.y; v.e1[s1] = ne1.y; v.e2[s1] = ne2.y; v.e3[s1] = ne3.y;
                    v.ophr[s1] = ofr.y; v.ophi[s1] = ofi.y; v.oth1[s1] = ot1.y; v.oth2[s1] = ot2.y; v.oth3[s1] = ot3.y;
                }
            }
            ph_m = f0;
            u3_m = u3;
            p13_m = p13;
            p23_m = p23;
        }
        // A: links of plane z+2 into the slot of plane z-1, then prefetch z+3
        if (z + 2 <= z1) {
            phase_A(sa);
            th_a1 = th_b1; th_a2 = th_b2; th_a3 = th_b3;
            th_b1 = q_t1; th_b2 = q_t2; th_b3 = q_t3;
            load_plane(z + 3);
        }
        __syncthreads();
    }
}

template <int TY, int MINB>
cudaError_t launch_pair_shape(const View<float> &v, int N, const KickCoef<float> &c, int min_chunk, cudaStream_t st)
{
    using G = PGeo<TY>;
    static unsigned long long configured = 0;   // per device
    const unsigned long long dev_bit = 1ULL << device_slot();
    if (!(configured & dev_bit)) {
        cudaError_t e = cudaFuncSetAttribute(k_pair<TY, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)G::smem);
        if (e != cudaSuccess) return e;
        configured |= dev_bit;
    }
    const int tx = (N + OWNW - 1) / OWNW, ty = (N + TY - 1) / TY;
    int nch = (int)((152LL * 16 + (long long)tx * ty - 1) / ((long long)tx * ty));
    nch = max(1, min(nch, N / min_chunk));
    const int zc = (N + nch - 1) / nch;
    nch = (N + zc - 1) / zc;
    k_pair<TY, MINB><<<dim3(tx, ty, nch), G::NT, G::smem, st>>>(v, N, zc, c);
    return cudaGetLastError();
}

}  // namespace

bool pair_shape_ok(int N) { return N % 2 == 0 && N >= 8; }

cudaError_t launch_pair_step(const View<float> &v, int N, const KickCoef<float> &c, int shape, cudaStream_t st)
{
    if (!pair_shape_ok(N)) return cudaErrorInvalidValue;
    switch (shape) {
    case 0: return launch_pair_shape<6, 3>(v, N, c, 16, st);
    case 1: return launch_pair_shape<6, 4>(v, N, c, 16, st);
    case 2: return launch_pair_shape<14, 1>(v, N, c, 16, st);
    case 3: return launch_pair_shape<14, 2>(v, N, c, 16, st);
    case 4: return launch_pair_shape<30, 1>(v, N, c, 16, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ah
