// Discrete adjoint of the stabilized DG right-hand side (included by dgw_stage_impl.cuh).
//
// vjp_kernel computes, per cell e, the transpose-Jacobian-vector product of its own
// residual L_e = M^{-1} R_stab(U)_e (Eq. weak2 with the stabilization of Sec. 3 and the
// sensor of Sec. 4) applied to lam_e:
//     wself_e   = (dL_e / dU_e)^T lam_e,
//     wnb_e^f   = (dL_e / dU_nbr(e,f))^T lam_e      for the face neighbours f,
// differentiating the volume term, the LLF face flux, the viscosity nu_e (through the
// maximising Gauss point), gamma_e (through the Hermite candidates, nonlinear weights,
// seminorms and the ratio) and the stiffness term.  Non-smooth points use
// subgradients: d min(1, r)/dr = [r < 1]; d|x| = sign(x) with sign(0) = 0; a maximum
// picks its first maximising argument; the eps_s guard and the b threshold are
// constant pieces.  gather_kernel sums, per cell, wself and the partials its neighbours
// produced for it, and forms out = sum_i coef_i x_i + cvjp * (J_L^T lam).
// Periodic meshes, advection and Burgers fluxes.

template <int P>
__device__ __forceinline__ Real gram(const Tab<P>& T, int a, int b)
{
    return a == b ? T.Gu[a][a] : (a < b ? Real(0.5) * T.Gu[a][b] : Real(0.5) * T.Gu[b][a]);
}

// y = G x over modes >= 1 (parity-sparse symmetric Gram matrix)
template <int P>
__device__ __forceinline__ void gram_mv(const Tab<P>& T, const Real* x, Real* y)
{
    constexpr int N1 = P + 1, K = Tab<P>::K;
    y[0] = Real(0);
#pragma unroll
    for (int a = 1; a < K; ++a) {
        Real s = Real(0);
#pragma unroll
        for (int b = 1; b < K; ++b) {
            const int ia = a % N1, ja = a / N1, ib = b % N1, jb = b / N1;
            if (((ia + ib) & 1) == 0 && ((ja + jb) & 1) == 0) s = fma(gram<P>(T, a, b), x[b], s);
        }
        y[a] = s;
    }
}

// dH/du_own, dH/du_nbr of the LLF flux seen from a cell whose outward normal is
// sgn * e_axis, own trace uo, neighbour trace un.
template <int FLUX>
__device__ __forceinline__ void llf_grad(const KParams& A, int axis, Real sgn, Real uo, Real un, Real& ho, Real& hn)
{
    const Real an = sgn * (axis == 0 ? A.a0 : A.a1);
    if (FLUX == FLUX_ADVECT) {
        const Real s = fabs(an);
        ho = Real(0.5) * an + Real(0.5) * s;
        hn = Real(0.5) * an - Real(0.5) * s;
    } else {   // Burgers: H = an (uo^2 + un^2) / 4 - s (un - uo) / 2, s = |an| max(|uo|, |un|)
        const bool own_max = fabs(uo) >= fabs(un);
        const Real s = fabs(an) * (own_max ? fabs(uo) : fabs(un));
        const Real dso = own_max ? fabs(an) * (uo > Real(0) ? Real(1) : (uo < Real(0) ? Real(-1) : Real(0))) : Real(0);
        const Real dsn = own_max ? Real(0) : fabs(an) * (un > Real(0) ? Real(1) : (un < Real(0) ? Real(-1) : Real(0)));
        const Real jump = un - uo;
        ho = Real(0.5) * an * uo + Real(0.5) * s - Real(0.5) * jump * dso;
        hn = Real(0.5) * an * un - Real(0.5) * s - Real(0.5) * jump * dsn;
    }
}

// d|F'(u)|_2 / du (advection: 0; Burgers: |a| sign(u), 1D: |a0| sign(u))
template <int FLUX>
__device__ __forceinline__ Real dspeed(const KParams& A, Real u)
{
    if (FLUX == FLUX_ADVECT) return Real(0);
    const Real an = DIM == 1 ? fabs(A.a0) : sqrt_r(A.a0 * A.a0 + A.a1 * A.a1);
    return an * (u > Real(0) ? Real(1) : (u < Real(0) ? Real(-1) : Real(0)));
}

template <int P, int FLUX>
__global__ void __launch_bounds__(128, P <= 2 ? 4 : 1) vjp_kernel(const KParams A, const Real* __restrict__ lam,
                                                  Real* __restrict__ wself, Real* __restrict__ wnb)
{
    constexpr int N1 = P + 1, NQ = P + 2, K = Tab<P>::K, NF = 2 * DIM;
    constexpr int TN = DIM == 1 ? 1 : N1, NFQ = DIM == 1 ? 1 : NQ;
    const Tab<P>& T = tab<P>();
    const int64_t E = A.E;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int ix = (int)(e % A.nx), iy = DIM == 2 ? (int)(e / A.nx) : 0;
    const Real* __restrict__ U = A.Uk;

    Real c[K], v[K], ws[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int i = k % N1, j = k / N1;
        c[k] = U[k * E + e];
        Real mi = T.minv[i];
        if (DIM == 2) mi *= T.minv[j];
        v[k] = A.two_h * mi * lam[k * E + e];   // lam scaled by M^{-1}: the reference-sum units
        ws[k] = Real(0);
    }
    int64_t nb[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        int jx = ix + (f == 0 ? -1 : (f == 1 ? 1 : 0));
        int jy = iy + (f == 2 ? -1 : (f == 3 ? 1 : 0));
        jx = jx < 0 ? A.nx - 1 : (jx >= A.nx ? 0 : jx);
        if (DIM == 2) jy = jy < 0 ? A.ny - 1 : (jy >= A.ny ? 0 : jy);
        nb[f] = (int64_t)jy * A.nx + jx;
    }
    const bool need_lam = A.stab != STAB_DG && !A.lam_fixed;
    // maximising Gauss point of |F'(U_h)| (for nu_e): kind 0 volume (qa, qb), 1 face (f, q)
    // lambda_e = |F'(U_h)| over the volume and face points is |a| (advection) or |a| |u|
    // (Burgers): the points are compared by the key |u| (0 for advection) and the
    // maximiser kept as one code, kind * 256 + a * 16 + b (a, b < 16)
    Real kmax = Real(-1), u_at = Real(0);
    int at_code = 0;
    const Real speed_scale = DIM == 1 ? fabs(A.a0) : sqrt_r(A.a0 * A.a0 + A.a1 * A.a1);

    // ---------------- volume term ----------------
    if (DIM == 1) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            Real u = Real(0), g = Real(0);
#pragma unroll
            for (int i = 0; i < N1; ++i) { u = fma(c[i], T.B[q][i], u); g = fma(v[i], T.D[q][i], g); }
            const Real fp = FLUX == FLUX_ADVECT ? A.a0 : A.a0 * u;
            const Real s = T.w[q] * fp * g;
#pragma unroll
            for (int i = 0; i < N1; ++i) ws[i] = fma(T.B[q][i], s, ws[i]);
            if (need_lam) {
                const Real key = FLUX == FLUX_ADVECT ? Real(0) : fabs(u);
                if (key > kmax) { kmax = key; u_at = u; at_code = q * 16; }
            }
        }
    } else {
        Real tc[N1][NQ], tvd[N1][NQ], tvb[N1][NQ];
#pragma unroll
        for (int j = 0; j < N1; ++j)
#pragma unroll
            for (int qa = 0; qa < NQ; ++qa) {
                Real s0 = Real(0), s1 = Real(0), s2 = Real(0);
#pragma unroll
                for (int i = 0; i < N1; ++i) {
                    s0 = fma(c[i + N1 * j], T.B[qa][i], s0);
                    s1 = fma(v[i + N1 * j], T.D[qa][i], s1);
                    s2 = fma(v[i + N1 * j], T.B[qa][i], s2);
                }
                tc[j][qa] = s0;
                tvd[j][qa] = s1;
                tvb[j][qa] = s2;
            }
#pragma unroll
        for (int qb = 0; qb < NQ; ++qb) {
            Real row[N1];
#pragma unroll
            for (int i = 0; i < N1; ++i) row[i] = Real(0);
#pragma unroll
            for (int qa = 0; qa < NQ; ++qa) {
                Real u = Real(0), gx = Real(0), gy = Real(0);
#pragma unroll
                for (int j = 0; j < N1; ++j) {
                    u = fma(tc[j][qa], T.B[qb][j], u);
                    gx = fma(tvd[j][qa], T.B[qb][j], gx);
                    gy = fma(tvb[j][qa], T.D[qb][j], gy);
                }
                const Real fx = FLUX == FLUX_ADVECT ? A.a0 : A.a0 * u;
                const Real fy = FLUX == FLUX_ADVECT ? A.a1 : A.a1 * u;
                const Real s = T.w[qa] * T.w[qb] * (fx * gx + fy * gy);
#pragma unroll
                for (int i = 0; i < N1; ++i) row[i] = fma(T.B[qa][i], s, row[i]);
                if (need_lam) {
                    const Real key = FLUX == FLUX_ADVECT ? Real(0) : fabs(u);
                    if (key > kmax) { kmax = key; u_at = u; at_code = qa * 16 + qb; }
                }
            }
#pragma unroll
            for (int j = 0; j < N1; ++j)
#pragma unroll
                for (int i = 0; i < N1; ++i) ws[i + N1 * j] = fma(T.B[qb][j], row[i], ws[i + N1 * j]);
        }
    }

    // ---------------- faces: -sum_q w_q phi_k H(own, nbr) ----------------
    Real cn[NF][K];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int k = 0; k < K; ++k) cn[f][k] = U[k * E + nb[f]];
    Real wn[NF][K];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const int axis = f >> 1, side = f & 1;
        const Real sgn = side ? Real(1) : Real(-1);
#pragma unroll
        for (int k = 0; k < K; ++k) wn[f][k] = Real(0);
        Real to[TN], tn[TN], tv[TN];
#pragma unroll
        for (int t = 0; t < TN; ++t) {
            Real so = Real(0), sn = Real(0), sv = Real(0);
#pragma unroll
            for (int n = 0; n < N1; ++n) {
                const int k = DIM == 1 ? n : (axis == 0 ? n + N1 * t : t + N1 * n);
                const Real po = (side || (n % 2 == 0)) ? Real(1) : Real(-1);   // P_n(sgn)
                const Real pn = ((!side) || (n % 2 == 0)) ? Real(1) : Real(-1); // P_n(-sgn)
                so = fma(po, c[k], so);
                sn = fma(pn, cn[f][k], sn);
                sv = fma(po, v[k], sv);
            }
            to[t] = so;
            tn[t] = sn;
            tv[t] = sv;
        }
        Real eo[TN], en[TN];
#pragma unroll
        for (int t = 0; t < TN; ++t) { eo[t] = Real(0); en[t] = Real(0); }
#pragma unroll
        for (int q = 0; q < NFQ; ++q) {
            Real uo = Real(0), un = Real(0), a = Real(0);
            if (DIM == 1) { uo = to[0]; un = tn[0]; a = tv[0]; }
            else {
#pragma unroll
                for (int t = 0; t < TN; ++t) {
                    uo = fma(to[t], T.B[q][t], uo);
                    un = fma(tn[t], T.B[q][t], un);
                    a = fma(tv[t], T.B[q][t], a);
                }
                a *= T.w[q];
            }
            Real ho, hn;
            llf_grad<FLUX>(A, axis, sgn, uo, un, ho, hn);
            const Real go = -a * ho, gn = -a * hn;
#pragma unroll
            for (int t = 0; t < TN; ++t) {
                const Real bt = DIM == 1 ? Real(1) : T.B[q][t];
                eo[t] = fma(go, bt, eo[t]);
                en[t] = fma(gn, bt, en[t]);
            }
            if (need_lam) {
                const Real key = FLUX == FLUX_ADVECT ? Real(0) : fabs(uo);
                if (key > kmax) { kmax = key; u_at = uo; at_code = 256 + f * 16 + q; }
            }
        }
#pragma unroll
        for (int t = 0; t < TN; ++t)
#pragma unroll
            for (int n = 0; n < N1; ++n) {
                const int k = DIM == 1 ? n : (axis == 0 ? n + N1 * t : t + N1 * n);
                const Real po = (side || (n % 2 == 0)) ? Real(1) : Real(-1);
                const Real pn = ((!side) || (n % 2 == 0)) ? Real(1) : Real(-1);
                ws[k] = fma(po, eo[t], ws[k]);
                wn[f][k] = fma(pn, en[t], wn[f][k]);
            }
    }

    // ---------------- stabilization: -gamma (lambda/p) K_ref c ----------------
    if (A.stab != STAB_DG) {
        Real kc[K], kv[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = k % N1, j = k / N1;
            Real s1 = Real(0), s2 = Real(0), r1 = Real(0), r2 = Real(0);
#pragma unroll
            for (int m = 1; m < N1; ++m) {
                if (DIM == 1) {
                    if (((i + m) & 1) == 0 && i > 0) { s1 = fma(T.A1[i][m], c[m], s1); r1 = fma(T.A1[i][m], v[m], r1); }
                } else {
                    if (((i + m) & 1) == 0 && i > 0) { s1 = fma(T.A1[i][m], c[m + N1 * j], s1); r1 = fma(T.A1[i][m], v[m + N1 * j], r1); }
                    if (((j + m) & 1) == 0 && j > 0) { s2 = fma(T.A1[j][m], c[i + N1 * m], s2); r2 = fma(T.A1[j][m], v[i + N1 * m], r2); }
                }
            }
            kc[k] = DIM == 1 ? s1 : s1 * T.A0[j] + T.A0[i] * s2;
            kv[k] = DIM == 1 ? r1 : r1 * T.A0[j] + T.A0[i] * r2;
        }
        Real z = Real(0);
#pragma unroll
        for (int k = 0; k < K; ++k) z = fma(v[k], kc[k], z);
        const Real lam_max = FLUX == FLUX_ADVECT ? speed_scale : speed_scale * kmax;
        const Real lamv = A.lam_fixed ? A.lambda_nu : lam_max;

        // sensor forward (Sec. 4), keeping what the reverse sweep needs
        Real gamma = A.stab == STAB_LO ? Real(1) : Real(0);
        Real cbar[K];
#pragma unroll
        for (int k = 0; k < K; ++k) cbar[k] = Real(0);
        if (A.stab == STAB_WENO) {
            // (each divisor is inverted once and its quotients taken as products)
            Real cl[NF][K], beta[NF + 1], what[NF + 1], ib[NF + 1];   // ib: 1 / (eps_w + beta)
            const Real beta0 = qform<P>(T, c);
            beta[0] = beta0;
            const Real lin0 = Real(1) - Real(NF) * A.w_nbr;
            ib[0] = Real(1) / (A.eps_w + beta0);
            what[0] = lin0 * ib[0] * ib[0];
            Real W = what[0];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const int axis = f >> 1, side = f & 1;
#pragma unroll
                for (int k = 1; k < K; ++k) {
                    const int i = k % N1, j = k / N1;
                    const int a = axis == 0 ? i : j;
                    Real s = Real(0);
#pragma unroll
                    for (int m = 0; m < N1; ++m) {
                        if (m < a) continue;
                        const int km = axis == 0 ? m + N1 * j : i + N1 * m;
                        s = fma(T.T[side][a][m], cn[f][km], s);
                    }
                    cl[f][k] = s;
                }
                cl[f][0] = Real(0);
                beta[f + 1] = qform<P>(T, cl[f]);
                ib[f + 1] = Real(1) / (A.eps_w + beta[f + 1]);
                what[f + 1] = A.w_nbr * ib[f + 1] * ib[f + 1];
                W += what[f + 1];
            }
            const Real iW = Real(1) / W;
            Real d[K];
            d[0] = Real(0);
#pragma unroll
            for (int k = 1; k < K; ++k) {
                Real s = Real(0);
#pragma unroll
                for (int f = 0; f < NF; ++f) s = fma(what[f + 1], c[k] - cl[f][k], s);
                d[k] = s * iW;
            }
            const Real num = sqrt_r(fmax(qform<P>(T, d), Real(0)));
            bool smooth_part = false;
            Real r = Real(0), sb0 = Real(1);
            if (num <= A.eps_s) gamma = Real(0);
            else if (beta0 <= Real(0)) gamma = Real(1);
            else {
                sb0 = sqrt_r(beta0);
                r = num / sb0;
                gamma = r < Real(1) ? r : Real(1);
                if (!A.q_one) gamma = pow(gamma, A.q);
                smooth_part = r < Real(1) && !(r < A.b);
                if (r < A.b) gamma = Real(0);
            }
            // reverse sweep of gamma with gbar = d out / d gamma
            const Real gbar = -z * lamv * Real(1.0 / P);
            if (smooth_part && gbar != Real(0)) {
                const Real iden = Real(1) / sb0;
                const Real rbar = A.q_one ? gbar : gbar * A.q * pow(r, A.q - Real(1));
                const Real numbar = rbar * iden;
                const Real denbar = -rbar * r * iden;
                const Real n2bar = numbar / (Real(2) * num);
                Real b0bar = denbar * (Real(0.5) * iden);
                Real gd[K];
                gram_mv<P>(T, d, gd);
                Real dbar[K];
#pragma unroll
                for (int k = 0; k < K; ++k) dbar[k] = Real(2) * n2bar * gd[k];
                Real omb[NF], S = Real(0);
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    Real s = Real(0);
#pragma unroll
                    for (int k = 1; k < K; ++k) s = fma(dbar[k], c[k] - cl[f][k], s);
                    omb[f] = s;
                    S = fma(s, what[f + 1] * iW, S);
                }
                const Real w1 = (W - what[0]) * iW;   // sum of the neighbour weights
#pragma unroll
                for (int k = 1; k < K; ++k) cbar[k] = fma(w1, dbar[k], cbar[k]);
                // own weight: what_0 only enters through the normalisation
                const Real what0bar = -S * iW;
                b0bar += Real(-2) * what0bar * what[0] * ib[0];
                Real gc[K];
                gram_mv<P>(T, c, gc);
#pragma unroll
                for (int k = 1; k < K; ++k) cbar[k] = fma(Real(2) * b0bar, gc[k], cbar[k]);
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const int axis = f >> 1, side = f & 1;
                    const Real omega = what[f + 1] * iW;
                    const Real whatbar = (omb[f] - S) * iW;
                    const Real bbar = Real(-2) * whatbar * what[f + 1] * ib[f + 1];
                    Real gl[K];
                    gram_mv<P>(T, cl[f], gl);
                    Real clbar[K];
#pragma unroll
                    for (int k = 1; k < K; ++k) clbar[k] = -omega * dbar[k] + Real(2) * bbar * gl[k];
                    clbar[0] = Real(0);
                    // c_l(a, .) = sum_{m >= a} T[side][a][m] c_nbr(m, .) along the axis:
                    // transpose back, c_nbr_bar(m, .) = sum_{a <= m} T[side][a][m] c_l_bar(a, .)
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const int i = k % N1, j = k / N1;
                        const int m = axis == 0 ? i : j;
                        Real s = Real(0);
#pragma unroll
                        for (int a = 0; a < N1; ++a) {
                            if (a > m) continue;
                            const int ka = DIM == 1 ? a : (axis == 0 ? a + N1 * j : i + N1 * a);
                            s = fma(T.T[side][a][m], clbar[ka], s);
                        }
                        wn[f][k] += s;
                    }
                }
            }
        }
        const Real gs = gamma * lamv * Real(1.0 / P);
#pragma unroll
        for (int k = 0; k < K; ++k) ws[k] = ws[k] - gs * kv[k] + cbar[k];
        // nu_e through lambda_e = |F'(U_h)| at the maximising point
        if (need_lam && gamma != Real(0)) {
            const Real lbar = -z * gamma * Real(1.0 / P);
            const Real ds = lbar * dspeed<FLUX>(A, u_at);
            const int at_kind = at_code >> 8, at_a = (at_code >> 4) & 15, at_b = at_code & 15;
            if (ds != Real(0)) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int i = k % N1, j = k / N1;
                    Real phi;
                    if (at_kind == 0) {
                        phi = T.B[at_a][i];
                        if (DIM == 2) phi *= T.B[at_b][j];
                    } else {
                        const int axis = at_a >> 1, side = at_a & 1;
                        const int nax = axis == 0 ? i : j, tr = axis == 0 ? j : i;
                        const Real pe = (side || (nax % 2 == 0)) ? Real(1) : Real(-1);
                        phi = DIM == 1 ? pe : pe * T.B[at_b][tr];
                    }
                    ws[k] = fma(ds, phi, ws[k]);
                }
            }
        }
    }

#pragma unroll
    for (int k = 0; k < K; ++k) wself[k * E + e] = ws[k];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int k = 0; k < K; ++k) wnb[((int64_t)f * K + k) * E + e] = wn[f][k];
}

// out = sum_i coef_i x_i + cvjp * (wself_e + sum_f wnb^{opp(f)}_{nbr(e,f)})
template <int P>
__global__ void __launch_bounds__(128) gather_kernel(const int64_t E, const int nx, const int ny,
                                                     const Real* __restrict__ wself, const Real* __restrict__ wnb,
                                                     const Real* x0, const Real* x1, const Real* x2,
                                                     const Real c0, const Real c1, const Real c2, const Real cv,
                                                     Real* out)
{
    constexpr int K = Tab<P>::K, NF = 2 * DIM;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int ix = (int)(e % nx), iy = DIM == 2 ? (int)(e / nx) : 0;
    int64_t nb[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        int jx = ix + (f == 0 ? -1 : (f == 1 ? 1 : 0));
        int jy = iy + (f == 2 ? -1 : (f == 3 ? 1 : 0));
        jx = jx < 0 ? nx - 1 : (jx >= nx ? 0 : jx);
        if (DIM == 2) jy = jy < 0 ? ny - 1 : (jy >= ny ? 0 : jy);
        nb[f] = (int64_t)jy * nx + jx;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        Real g = wself[k * E + e];
#pragma unroll
        for (int f = 0; f < NF; ++f) g += wnb[((int64_t)(f ^ 1) * K + k) * E + nb[f]];
        Real o = cv * g;
        if (x0) o = fma(c0, x0[k * E + e], o);
        if (x1) o = fma(c1, x1[k * E + e], o);
        if (x2) o = fma(c2, x2[k * E + e], o);
        out[k * E + e] = o;
    }
}
