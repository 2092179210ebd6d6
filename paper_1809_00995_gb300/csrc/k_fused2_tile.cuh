// k_fused2_tile.cuh -- body of one work item of the two-step pass (k_fused2.cu):
// region R1 of tile (AH2_BX, AH2_BY), z chunk AH2_BZ (planes [AH2_BZ zc,
// AH2_BZ zc + zc)), two leapfrog steps with coefficients c1 (step n) and c2
// (step n + 1).  It is included as the body of the single-lattice kernel and
// inside the work-item loop of the batched kernel; in scope there: TY, IT, v
// (View2<float>), N, zc, c1, c2, smem_raw (dynamic shared memory), and
// AH2_SKIP_TILE, the statement that leaves an empty item, AH2_DIAG (with da,
// a Diag2Args), true in the kernel that also takes the diagnostics of the
// state n on the written sites, and AH2_WEAK, true in the kernel specialised
// to weak gauge fields (sincos_link3_weak).  (A function shared
// by the two kernels costs the single-lattice kernel a tenth of its speed:
// its pointers and coefficients then no longer stay kernel parameters.)
{
    using G = Geo2<TY>;
    using C = cpx<float>;
    constexpr int TX = G::TX, NT = G::NT, EX = G::EX, EY = G::EY, NE = G::NE, PX = G::PX, NP = G::NP;
    C *sU = reinterpret_cast<C *>(smem_raw);                 // [2][3][NE]
    C *sF = sU + 2 * 3 * NE;                                 // [2][NE]
    float *sP = reinterpret_cast<float *>(smem_raw + G::off_P);
    C *sV = reinterpret_cast<C *>(smem_raw + G::off_V);      // [2][4][NT]
    float *sQ = reinterpret_cast<float *>(smem_raw + G::off_Q);
    // AH2_DIAG: this thread's diagnostic sums; scaled edge products of R1
    // (d = 1, 3) and E_2 of plane q for the row above / below
    [[maybe_unused]] Diag2Acc dq;
    [[maybe_unused]] C2<float> *sE = reinterpret_cast<C2<float> *>(smem_raw + G::off_D);    // [2][NT]
    [[maybe_unused]] float *sG = reinterpret_cast<float *>(smem_raw + G::off_D + sizeof(C2<float>) * 2 * NT);

    const int tid = threadIdx.x, lx = tid & 31, wy = tid >> 5;
    // R1 origin; the written sites start one further in
    const int x0 = AH2_BX * G::OX - 1, y0 = AH2_BY * G::OY - 1;
    const int z0 = AH2_BZ * zc;
    if (z0 >= N) {
        if constexpr (AH2_DIAG)
            dq.flush<NT>(da.partials + (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)));
        AH2_SKIP_TILE;
    }
    const int z1 = min(z0 + zc, N);
    const IT NN = (IT)N * (IT)N;

    const int gx = x0 + lx, gy = y0 + wy;
    const int roff = wrapm(gx, N) + N * wrapm(gy, N);
    const bool inner = lx >= 1 && lx <= TX - 2 && wy >= 1 && wy <= TY - 2;
    const bool wr = inner && gx < N && gy < N;   // gx, gy >= 0 for inner sites
    const int e = (wy + 1) * EX + lx + 1;        // own site in the haloed tile
    const int p = (wy + 1) * PX + lx + 1;        // own site in the plaquette tile
    const int r = wy * TX + lx;                  // own site in R1
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

    // register prefetch of one plane of the state n: own site [0], halo [1]
    float fth[2][3], fph[2][2];
    auto load_plane = [&](int z) {               // z in [-2, N + 2]
        const int zz = z < 0 ? z + N : (z >= N ? z - N : z);
        const IT base = (IT)zz * NN;
        {
            const IT s = base + (IT)roff;
            fth[0][0] = v.th1[s]; fth[0][1] = v.th2[s]; fth[0][2] = v.th3[s];
            fph[0][0] = v.phr[s]; fph[0][1] = v.phi[s];
        }
        if (has_halo) {
            const IT s = base + (IT)hoff;
            fth[1][0] = v.th1[s]; fth[1][1] = v.th2[s]; fth[1][2] = v.th3[s];
            fph[1][0] = v.phr[s]; fph[1][1] = v.phi[s];
        }
    };
    auto store_plane = [&](int b) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            if (t == 0 || has_halo) {
                const int ei = t == 0 ? e : heix;
                float sn[3], co[3];
                if constexpr (AH2_WEAK) sincos_link3_weak(fth[t], sn, co);
                else sincos_link3(fth[t], sn, co);
#pragma unroll
                for (int d = 0; d < 3; ++d) sU[(b * 3 + d) * NE + ei] = { co[d], sn[d] };
                sF[b * NE + ei] = { fph[t][0], fph[t][1] };
            }
        }
    };

    // first step: own-site values of the plane below and of the current plane
    C ph_m, ph_0, u3_m;
    float th_0[3], p13_m, p23_m;
    // second step: own-site values of the plane below
    C ph2_m = { 0.f, 0.f }, u3_2m = { 0.f, 0.f };
    float q13_m = 0.f, q23_m = 0.f;
    // first-step results of the plane the second step works on
    float hpr = 0.f, hpi = 0.f, he1 = 0.f, he2 = 0.f, he3 = 0.f, ht1 = 0.f, ht2 = 0.f, ht3 = 0.f;
    // AH2_DIAG: own scaled edges d = 1, 2 of plane q (computed one plane
    // ahead) and E_3 of plane q - 1
    [[maybe_unused]] C2<float> ed1{ 1.f, 0.f }, ed2{ 1.f, 0.f };
    [[maybe_unused]] float e3_m = 0.f;

    // prologue: the first step starts at plane q0 = z0 - 1 (the second step
    // needs it below its first plane); ring slot of plane q: (q - q0 + 1) & 1
    const int q0 = z0 - 1;
    load_plane(q0 - 1);
    store_plane(0);
    ph_m = { fph[0][0], fph[0][1] };
    load_plane(q0);
    store_plane(1);
    ph_0 = { fph[0][0], fph[0][1] };
    th_0[0] = fth[0][0]; th_0[1] = fth[0][1]; th_0[2] = fth[0][2];
    load_plane(q0 + 1);
    __syncthreads();
    {
        const C *Um = sU, *U0 = sU + 3 * NE;
        u3_m = Um[2 * NE + e];
        p13_m = plaq(Um[e], Um[2 * NE + e + 1], U0[e], Um[2 * NE + e]);
        p23_m = plaq(Um[NE + e], Um[2 * NE + e + EX], U0[NE + e], Um[2 * NE + e]);
    }
    __syncthreads();

    // iterations k = 0 .. K - 1; the diagnostics cover planes q0 + 1 .. q0 + K - 2
    const int K = z1 - z0 + 2;

    // iteration k: first step at plane q = q0 + k, second step at plane q - 1
    // (plaquettes from k = 1, kicks and stores from k = 2).  BC (compile
    // time) is the ring slot of plane q in the first step's input ring; the
    // first step's output of plane q goes to slot 1 - BC of its ring, where
    // plane q - 1 is in slot BC.
    auto iter = [&](int k, auto bc_tag) {
        constexpr int bc = decltype(bc_tag)::value, bn = 1 - bc;
        const int q = q0 + k;
        const int zq = q < 0 ? q + N : (q >= N ? q - N : q);
        float pr, pim, e1, e2, e3;
        {
            const IT s = (IT)zq * NN + (IT)roff;
            pr = v.pir[s]; pim = v.pii[s]; e1 = v.e1[s]; e2 = v.e2[s]; e3 = v.e3[s];
        }
        // A: links and phi of plane q + 1 from the prefetch, then prefetch q + 2
        store_plane(bn);
        const C ph_p = { fph[0][0], fph[0][1] };
        const float tp0 = fth[0][0], tp1 = fth[0][1], tp2 = fth[0][2];
        load_plane(q + 2);
        __syncthreads();

        // B: first-step plaquette sines of plane q on R1 and its low halos
        const C *U0 = sU + bc * 3 * NE, *U1p = sU + bn * 3 * NE;
        float p12, p13, p23;
        [[maybe_unused]] float bcos = 0.f;       // AH2_DIAG: sum of 1 - cos Xi at the own site
        if constexpr (AH2_DIAG) {
            const C x12 = plaq2(U0[e], U0[NE + e + 1], U0[e + EX], U0[NE + e]);
            const C x13 = plaq2(U0[e], U0[2 * NE + e + 1], U1p[e], U0[2 * NE + e]);
            const C x23 = plaq2(U0[NE + e], U0[2 * NE + e + EX], U1p[NE + e], U0[2 * NE + e]);
            p12 = x12.i; p13 = x13.i; p23 = x23.i;
            bcos = one_minus_cos(x12.r, x12.i) + one_minus_cos(x13.r, x13.i) + one_minus_cos(x23.r, x23.i);
        } else {
            p12 = plaq(U0[e], U0[NE + e + 1], U0[e + EX], U0[NE + e]);
            p13 = plaq(U0[e], U0[2 * NE + e + 1], U1p[e], U0[2 * NE + e]);
            p23 = plaq(U0[NE + e], U0[2 * NE + e + EX], U1p[NE + e], U0[2 * NE + e]);
        }
        sP[p] = p12;
        sP[NP + p] = p13;
        sP[2 * NP + p] = p23;
        if (tid < G::NPHALO) {
            const int px = tid < PX ? tid : 0, py = tid < PX ? 0 : tid - PX + 1;
            const int eh = py * EX + px, ph = py * PX + px;
            sP[ph] = plaq(U0[eh], U0[NE + eh + 1], U0[eh + EX], U0[NE + eh]);
            sP[NP + ph] = plaq(U0[eh], U0[2 * NE + eh + 1], U1p[eh], U0[2 * NE + eh]);
            sP[2 * NP + ph] = plaq(U0[NE + eh], U0[2 * NE + eh + EX], U1p[NE + eh], U0[2 * NE + eh]);
        }
        // AH2_DIAG: the own edge d = 3 of plane q and d = 1, 2 of plane q + 1;
        // a plaquette whose four edges all have |Arg| < pi/4 has W = 0, and
        // when all edges of the CTA pass that test the carry chains are skipped
        [[maybe_unused]] C2<float> ed3, ez1, ez2;
        [[maybe_unused]] bool smooth_cta = false;
        if constexpr (AH2_DIAG) {
            const C *F1 = sF + bn * NE;
            ed3 = edge2(ph_0, U0[2 * NE + e], ph_p);
            ez1 = edge2(ph_p, U1p[e], F1[e + 1]);
            ez2 = edge2(ph_p, U1p[NE + e], F1[e + EX]);
            sE[r] = ed1;
            sE[NT + r] = ed3;
            sG[r] = e2;
            auto smooth1 = [](const C2<float> &z) { return z.r > 1.001f * fabsf(z.i); };
            const bool own_smooth = smooth1(ed1) && smooth1(ed2) && smooth1(ed3) && smooth1(ez1) && smooth1(ez2);
            smooth_cta = __syncthreads_and(own_smooth) != 0;
        } else {
            __syncthreads();
        }

        // C: first step (kicks and drifts) at the own site of plane q
        float npr, npi, ne1, ne2, ne3, nfr, nfi, nt[3];
        {
            const C *F0 = sF + bc * NE;
            const C f0 = ph_0;
            const C u1 = U0[e], u2 = U0[NE + e], u3 = U0[2 * NE + e];
            const C u1m = U0[e - 1], u2m = U0[NE + e - EX], u3m = u3_m;
            const C w1 = mul(u1, F0[e + 1]), w2 = mul(u2, F0[e + EX]), w3 = mul(u3, ph_p);
            const C b1 = mul(cj(u1m), F0[e - 1]);
            const C b2 = mul(cj(u2m), F0[e - EX]);
            const C b3 = mul(cj(u3m), ph_m);
            const float lr = (w1.r + b1.r) + (w2.r + b2.r) + (w3.r + b3.r) - 6.f * f0.r;
            const float li = (w1.i + b1.i) + (w2.i + b2.i) + (w3.i + b3.i) - 6.f * f0.i;
            const float pot = c1.c_pot * (f0.r * f0.r + f0.i * f0.i - c1.sigma2);
            npr = c1.c_damp * pr - pot * f0.r + c1.c_lap * lr;
            npi = c1.c_damp * pim - pot * f0.i + c1.c_lap * li;
            const float cu1 = w1.r * f0.i - w1.i * f0.r;
            const float cu2 = w2.r * f0.i - w2.i * f0.r;
            const float cu3 = w3.r * f0.i - w3.i * f0.r;
            const float cl1 = (p12 - sP[p - PX]) + (p13 - p13_m);
            const float cl2 = (sP[p - 1] - p12) + (p23 - p23_m);
            const float cl3 = (sP[NP + p - 1] - p13) + (sP[2 * NP + p - PX] - p23);
            ne1 = c1.c_edamp * e1 + c1.c_cur * cu1 - c1.c_curl * cl1;
            ne2 = c1.c_edamp * e2 + c1.c_cur * cu2 - c1.c_curl * cl2;
            ne3 = c1.c_edamp * e3 + c1.c_cur * cu3 - c1.c_curl * cl3;
            if constexpr (AH2_DIAG) {
                // E_1 of x - 1 and the edges of x + 1 from the neighbouring
                // lanes, E_2 of x - y and the edges of x + y from the rows
                // below and above (every written site is inner to R1)
                const float e1b = __shfl_up_sync(0xffffffffu, e1, 1);
                const C2<float> z2_1 = { __shfl_down_sync(0xffffffffu, ed2.r, 1),
                                         __shfl_down_sync(0xffffffffu, ed2.i, 1) };
                const C2<float> z3_1 = { __shfl_down_sync(0xffffffffu, ed3.r, 1),
                                         __shfl_down_sync(0xffffffffu, ed3.i, 1) };
                if (wr && k >= 1 && k <= K - 2) {
                    dq.site(da.c, pr, pim, f0, w1, w2, w3, e1, e2, e3, e1b, sG[r - TX], e3_m, bcos, th_0[0], th_0[1],
                            th_0[2]);
                    // windings of the plaquettes (12), (13), (23) based at x (Eq. 9)
                    const C2<float> z1_2 = sE[r + TX], z3_2 = sE[NT + r + TX];
                    int w12 = 0, w13 = 0, w23 = 0;
                    if (!smooth_cta) {
                        w12 = winding_scaled(ed1, z2_1, z1_2, ed2);
                        w13 = winding_scaled(ed1, z3_1, ez1, ed3);
                        w23 = winding_scaled(ed2, z3_2, ez2, ed3);
                    }
                    const unsigned long long site = (unsigned long long)q * (unsigned long long)NN + (unsigned)roff;
                    dq.wind(0, w12, site, da.list);
                    dq.wind(1, w13, site, da.list);
                    dq.wind(2, w23, site, da.list);
                }
                e3_m = e3;
                ed1 = ez1;
                ed2 = ez2;
            }
            nfr = f0.r + c1.dt * npr;
            nfi = f0.i + c1.dt * npi;
            nt[0] = th_0[0] + c1.dt * ne1;
            nt[1] = th_0[1] + c1.dt * ne2;
            nt[2] = th_0[2] + c1.dt * ne3;
            if (c1.wrap) {
                nt[0] = wrap_phase(nt[0]);
                nt[1] = wrap_phase(nt[1]);
                nt[2] = wrap_phase(nt[2]);
            }
            ph_m = f0;
            u3_m = u3;
            p13_m = p13;
            p23_m = p23;
        }
        ph_0 = ph_p;
        th_0[0] = tp0; th_0[1] = tp1; th_0[2] = tp2;
        // U' = e^{i theta'} and phi' of plane q into the second step's ring
        float sn[3], co[3];
        if constexpr (AH2_WEAK) sincos_link3_weak(nt, sn, co);
        else sincos_link3(nt, sn, co);
        C *Vq = sV + (1 - bc) * 4 * NT;
        Vq[r] = { co[0], sn[0] };
        Vq[NT + r] = { co[1], sn[1] };
        Vq[2 * NT + r] = { co[2], sn[2] };
        Vq[3 * NT + r] = { nfr, nfi };

        // D: second-step plaquette sines of plane q - 1 on R1 less its top row
        // and right column (the written sites and their low halos); the own
        // U'_1, U'_2 of plane q come from registers
        const C *W = sV + bc * 4 * NT;
        float r12 = 0.f, r13 = 0.f, r23 = 0.f;
        if (k >= 1 && lx < TX - 1 && wy < TY - 1) {
            const C w1 = W[r], w2 = W[NT + r], w3 = W[2 * NT + r];
            r12 = plaq(w1, W[NT + r + 1], W[r + TX], w2);
            r13 = plaq(w1, W[2 * NT + r + 1], C{ co[0], sn[0] }, w3);
            r23 = plaq(w2, W[2 * NT + r + TX], C{ co[1], sn[1] }, w3);
            sQ[r] = r12;
            sQ[NT + r] = r13;
            sQ[2 * NT + r] = r23;
        }
        __syncthreads();

        // E: second step at the inner sites of plane q - 1
        if (k >= 1) {
            const C f0 = W[3 * NT + r], u3 = W[2 * NT + r];
            if (k >= 2 && inner) {
                const C u1 = W[r], u2 = W[NT + r];
                const C u1m = W[r - 1], u2m = W[NT + r - TX], u3m = u3_2m;
                const C w1 = mul(u1, W[3 * NT + r + 1]), w2 = mul(u2, W[3 * NT + r + TX]);
                const C w3 = mul(u3, C{ nfr, nfi });
                const C b1 = mul(cj(u1m), W[3 * NT + r - 1]);
                const C b2 = mul(cj(u2m), W[3 * NT + r - TX]);
                const C b3 = mul(cj(u3m), ph2_m);
                const float lr = (w1.r + b1.r) + (w2.r + b2.r) + (w3.r + b3.r) - 6.f * f0.r;
                const float li = (w1.i + b1.i) + (w2.i + b2.i) + (w3.i + b3.i) - 6.f * f0.i;
                const float pot = c2.c_pot * (f0.r * f0.r + f0.i * f0.i - c2.sigma2);
                const float opr = c2.c_damp * hpr - pot * f0.r + c2.c_lap * lr;
                const float opi = c2.c_damp * hpi - pot * f0.i + c2.c_lap * li;
                const float cu1 = w1.r * f0.i - w1.i * f0.r;
                const float cu2 = w2.r * f0.i - w2.i * f0.r;
                const float cu3 = w3.r * f0.i - w3.i * f0.r;
                const float cl1 = (r12 - sQ[r - TX]) + (r13 - q13_m);
                const float cl2 = (sQ[r - 1] - r12) + (r23 - q23_m);
                const float cl3 = (sQ[NT + r - 1] - r13) + (sQ[2 * NT + r - TX] - r23);
                const float oe1 = c2.c_edamp * he1 + c2.c_cur * cu1 - c2.c_curl * cl1;
                const float oe2 = c2.c_edamp * he2 + c2.c_cur * cu2 - c2.c_curl * cl2;
                const float oe3 = c2.c_edamp * he3 + c2.c_cur * cu3 - c2.c_curl * cl3;
                float ot1 = ht1 + c2.dt * oe1, ot2 = ht2 + c2.dt * oe2, ot3 = ht3 + c2.dt * oe3;
                if (c2.wrap) {
                    ot1 = wrap_phase(ot1);
                    ot2 = wrap_phase(ot2);
                    ot3 = wrap_phase(ot3);
                }
                if (wr) {
                    const IT s = (IT)(q - 1) * NN + (IT)roff;    // q - 1 in [z0, z1)
                    v.opir[s] = opr; v.opii[s] = opi;
                    v.oe1[s] = oe1; v.oe2[s] = oe2; v.oe3[s] = oe3;
                    v.ophr[s] = f0.r + c2.dt * opr;
                    v.ophi[s] = f0.i + c2.dt * opi;
                    v.oth1[s] = ot1; v.oth2[s] = ot2; v.oth3[s] = ot3;
                }
            }
            ph2_m = f0;
            u3_2m = u3;
            q13_m = r13;
            q23_m = r23;
        }
        hpr = npr; hpi = npi; he1 = ne1; he2 = ne2; he3 = ne3;
        ht1 = nt[0]; ht2 = nt[1]; ht3 = nt[2];
    };
    for (int k = 0; k < K; k += 2) {
        iter(k, IC<1>{});
        if (k + 1 < K) iter(k + 1, IC<0>{});
    }
    if constexpr (AH2_DIAG)
        dq.flush<NT>(da.partials + (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)));
}
