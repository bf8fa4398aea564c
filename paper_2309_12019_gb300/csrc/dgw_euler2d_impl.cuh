// Stage kernel of the 2D Euler system (Sec. 5.6, its 2D problems), included by the 2D
// stage translation units after the scalar kernel (it shares the tables, the launch
// scalars and the math helpers of dgw_stage_impl.cuh).
//
// State U = (rho, rho vx, rho vy, rho E), p = (gamma - 1)(rho E - rho |v|^2 / 2); mode
// k = i + (p+1) j of component comp of cell e at row comp K + k, K = (p+1)^2.
// One CTA of EX x EY = 32 x 4 threads owns a tile of as many cells, one per thread:
//   0. the tile's coefficients and a one-cell face halo (all four components) are
//      staged in shared memory by coalesced row loads; halo cells beyond a periodic side
//      are its images, beyond a wall or an outflow side they are absent; in float the
//      Un coefficients of the tile start to arrive by cp.async
//   1. per cell: the sensor of Sec. 4 on the density, the volume term at the (p+2)^2
//      Gauss points by sum factorisation, lambda_e over those points
//   2. every face of the tile once: both traces at the p+2 Gauss points, the ghost
//      state at a boundary (a wall mirrors the normal momentum), the LLF flux with s+
//      the larger |v.n| + c, lifted onto the face's Legendre modes; the largest own-side
//      |v| + c of each face for lambda_e
//   3. per cell: face terms, the stabilization of every component with the density's
//      gamma, M^{-1} and the Runge-Kutta combination Uout = cn Un + ck Uk + cl L(Uk)
// Constants are folded as in the scalar kernel:
//   L_k = (2/h) minv(i) minv(j) [acc_k - gamma lambda / p (K_ref c)_k].

constexpr int EX = kTileX2, EY = kTileY2, ENT = EX * EY;
using R2 = std::conditional_t<kF32, float2, double2>;   // a pair of state components
constexpr int EHX = EX + 2, EHY = EY + 2;          // staged columns / rows (one halo cell)

template <int P>
struct Euler2Smem {
    static constexpr int N1 = P + 1, K = N1 * N1;
    // the four components as two pairs (rho, rho vx), (rho vy, rho E), each pair one
    // 8-byte (float) or 16-byte (double) word, so that a pair is one shared load or store
    R2 u[2][K][EHY][EHX];           // coefficients; tile cell (lx, ly) at [ly + 1][lx + 1]
    R2 hx[2][N1][EY][EX + 1];       // lifted LLF flux of x-face f of row r (cells f - 1, f)
    R2 hy[2][N1][EY + 1][EX];       // lifted LLF flux of y-face r of column c (cells r - 1, r)
    Real sx[2][EY][EX + 1];         // max |v| + c of the minus (0) / plus (1) cell's own values on x-face f
    Real sy[2][EY + 1][EX];         // the same on y-face r
    int has[EHY][EHX];              // the staged cell exists
    // float: Un of the tile's cells, brought in by cp.async (in double this would halve
    // the CTAs per SM; double reads Un at the end)
    R2 un[kF32 ? 2 : 1][kF32 ? K : 1][EY][EX];
};

struct Euler2State {
    Real vx, vy, pr, inv_rho;
};

__device__ __forceinline__ Euler2State euler2_prim(const KParams& A, const Real* q)
{
    Euler2State s;
    s.inv_rho = rcp_e(q[0]);
    s.vx = q[1] * s.inv_rho;
    s.vy = q[2] * s.inv_rho;
    s.pr = A.gm1 * (q[3] - Real(0.5) * (q[1] * s.vx + q[2] * s.vy));
    return s;
}

// |v.n| + c for an axis normal (axis 0: x, 1: y), or |v| + c for axis < 0
__device__ __forceinline__ Real euler2_speed(const KParams& A, const Euler2State& s, int axis)
{
    const Real c = sqrt_e(A.gam * s.pr * s.inv_rho);
    const Real v = axis == 0 ? fabs(s.vx) : (axis == 1 ? fabs(s.vy) : sqrt_e(s.vx * s.vx + s.vy * s.vy));
    return v + c;
}

// F(U) e_axis
__device__ __forceinline__ void euler2_flux(const Euler2State& s, const Real* q, int axis, Real* F)
{
    const Real vn = axis == 0 ? s.vx : s.vy;
    F[0] = q[0] * vn;
    F[1] = q[1] * vn + (axis == 0 ? s.pr : Real(0));
    F[2] = q[2] * vn + (axis == 1 ? s.pr : Real(0));
    F[3] = (q[3] + s.pr) * vn;
}

// Sensor of Sec. 4 (or Zhao et al.'s, stab = ZHAO) of a 2D cell from the density
// coefficients of the cell (c) and of its face neighbours at staged position (r, col).
template <int P>
__device__ __forceinline__ Real sensor_2d(const KParams& A, const Tab<P>& T, const Real* c,
                                          const Euler2Smem<P>& S, int r, int col)
{
    constexpr int N1 = P + 1, K = N1 * N1;
    bool has[4];
    int me = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const int rr = r + (f == 2 ? -1 : (f == 3 ? 1 : 0)), cc = col + (f == 0 ? -1 : (f == 1 ? 1 : 0));
        has[f] = S.has[rr][cc] != 0;
        me += has[f] ? 1 : 0;
    }
    const Real beta0 = qform<P>(T, c);
    const Real d0 = A.eps_w + beta0;
    const Real w0 = div_w(Real(1) - Real(me) * A.w_nbr, d0 * d0);
    Real wsum = w0;
    Real wnb[4];
    Real dacc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) dacc[k] = Real(0);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        wnb[f] = Real(0);
        if (!has[f]) continue;
        const int axis = f >> 1, side = f & 1;
        const int rr = r + (f == 2 ? -1 : (f == 3 ? 1 : 0)), cc = col + (f == 0 ? -1 : (f == 1 ? 1 : 0));
        // Hermite candidate: the neighbour's polynomial continued into this cell (its
        // mean does not enter the seminorms)
        Real cl[K];
        cl[0] = Real(0);
#pragma unroll
        for (int k = 1; k < K; ++k) {
            const int i = k % N1, j = k / N1;
            const int a = axis == 0 ? i : j;
            Real s = Real(0);
#pragma unroll
            for (int m = 0; m < N1; ++m) {
                if (m < a) continue;
                const int km = axis == 0 ? m + N1 * j : i + N1 * m;
                s = fma(T.T[side][a][m], S.u[0][km][rr][cc].x, s);
            }
            cl[k] = s;
        }
        const Real dl = A.eps_w + qform<P>(T, cl);
        const Real wl = div_w(A.w_nbr, dl * dl);
        wsum += wl;
        wnb[f] = wl;
#pragma unroll
        for (int k = 1; k < K; ++k) dacc[k] = fma(wl, c[k] - cl[k], dacc[k]);
    }
    const Real inv = div_w(Real(1), wsum);
    if (A.stab == STAB_ZHAO) {
        if (me == 0) return Real(0);
        const Real lin0 = Real(1) - Real(me) * A.w_nbr;
        Real dev = zpow(A, fabs(w0 * inv / lin0 - Real(1)));
#pragma unroll
        for (int f = 0; f < 4; ++f)
            if (has[f]) dev += zpow(A, fabs(wnb[f] * inv / A.w_nbr - Real(1)));
        const Real minlin = lin0 < A.w_nbr ? lin0 : A.w_nbr;
        return dev * rcp_e(zpow(A, fabs(rcp_e(minlin) - Real(1))) + Real(me));
    }
#pragma unroll
    for (int k = 1; k < K; ++k) dacc[k] *= inv;
    dacc[0] = Real(0);
    const Real qd = fmax(qform<P>(T, dacc), Real(0));
    if (qd <= A.eps_s * A.eps_s) return Real(0);
    if (beta0 <= Real(0)) return Real(1);
    const Real r2 = qd * rcp_e(beta0);
    Real g = r2 < Real(1) ? sqrt_e(r2) : Real(1);
    if (!A.q_one) g = pow(g, A.q);
    if (r2 < A.b * A.b) g = Real(0);
    return g;
}

// MODE 0: stage / residual; MODE 1: sensor only (writes gamma_out).
template <int P, int MODE>
__global__ void __launch_bounds__(ENT, (P == 3 || !kF32) ? 2 : 3) euler2d_kernel(const __grid_constant__ KParams A)
{
    constexpr int N1 = P + 1, NQ = P + 2, K = N1 * N1;
    extern __shared__ __align__(16) unsigned char smem_e2[];
    Euler2Smem<P>& S = *reinterpret_cast<Euler2Smem<P>*>(smem_e2);
    const Tab<P>& T = tab<P>();
    const int tid = threadIdx.x;
    const int64_t E = A.E;
    const int tx0 = blockIdx.x * EX, ty0 = blockIdx.y * EY;
    // ---- 0. stage the tile and its face halo ----
    for (int idx = tid; idx < EHY * EHX; idx += ENT) {
        const int r = idx / EHX, cc = idx - r * EHX;
        const bool corner = (r == 0 || r == EHY - 1) && (cc == 0 || cc == EHX - 1);
        const int gx = wrap_x(A, tx0 - 1 + cc), gy = wrap_y(A, ty0 - 1 + r);
        const bool ok = !corner && gx >= 0 && gy >= 0;
        S.has[r][cc] = ok;
        const Real* src = A.Uk + (ok ? (int64_t)gy * A.nx + gx : 0);
#pragma unroll
        for (int comp = 0; comp < 4; ++comp)
#pragma unroll
            for (int k = 0; k < K; ++k) lane(S.u[comp >> 1][k][r][cc], comp & 1) = ok ? src[(int64_t)(comp * K + k) * E] : Real(0);
    }
    const int lx = tid % EX, ly = tid / EX;
    const int gx = tx0 + lx, gy = ty0 + ly;
    const bool in = gx < A.nx && gy < A.ny;
    const int64_t e = (int64_t)gy * A.nx + gx;
    // Un is read only by the final combination: each thread starts asynchronous copies
    // of its cell's Un coefficients into shared memory now (cp.async holds no
    // registers) and waits for them just before that combination
    const bool copy_un = kF32 && MODE == 0 && A.has_un && in;
    if (copy_un) {
#pragma unroll
        for (int comp = 0; comp < 4; ++comp)
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&lane(S.un[kF32 ? comp >> 1 : 0][kF32 ? k : 0][ly][lx], comp & 1));
                const Real* src = A.Un + e + (int64_t)(comp * K + k) * E;
                asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" :: "r"(dst), "l"(src), "n"((int)sizeof(Real))
                             : "memory");
            }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    __syncthreads();

    // ---- 1. sensor of the density; volume term; lambda_e over the volume points ----
    const int r0 = ly + 1, c0 = lx + 1;
    Real gamma = (MODE == 0 && A.stab == STAB_LO) ? Real(1) : Real(0);
    if (in && (MODE == 1 || A.stab >= STAB_WENO)) {
        Real c[K];
#pragma unroll
        for (int k = 0; k < K; ++k) c[k] = S.u[0][k][r0][c0].x;
        gamma = sensor_2d<P>(A, T, c, S, r0, c0);
        if (MODE == 1) A.gamma_out[e] = (double)gamma;
    }
    if (MODE == 1) return;

    const bool need_lam = A.stab != STAB_DG && !A.lam_fixed;
    // The four components in two pairs, (rho, rho vx) and (rho vy, rho E): every
    // contraction below runs on both components of a pair at once (packed FP32 in float).
    // cu(pr, k, r, c) = mode k of pair pr of the staged cell at (r, c).
    auto cu = [&](int pr, int k, int r, int cc) -> R2 { return S.u[pr][k][r][cc]; };
    R2 acc[2][K];
#pragma unroll
    for (int pr = 0; pr < 2; ++pr)
#pragma unroll
        for (int k = 0; k < K; ++k) acc[pr][k] = vbc<R2>(0);
    Real lam = Real(0);
    if (in) {
        // one Gauss row qy at a time (a rolled loop: one copy of its code): the polynomials
        // reduced to the row, their values at the row's points (symmetric nodes), the
        // fluxes there, projected as in the scalar kernel
#pragma unroll 1
        for (int qy = 0; qy < NQ; ++qy) {
            R2 rr[2][N1];
#pragma unroll
            for (int pr = 0; pr < 2; ++pr)
#pragma unroll
                for (int i = 0; i < N1; ++i) {
                    R2 e = cu(pr, i, r0, c0);
#pragma unroll
                    for (int j = 1; j < N1; ++j) e = vfma(T.B[qy][j], cu(pr, i + N1 * j, r0, c0), e);
                    rr[pr][i] = e;
                }
            R2 u[2][NQ], fx[2][NQ], fy[2][NQ];
            interp_sym<N1, NQ>(T.B, rr[0], u[0]);
            interp_sym<N1, NQ>(T.B, rr[1], u[1]);
#pragma unroll
            for (int qx = 0; qx < NQ; ++qx) {
                const Real q[4] = {u[0][qx].x, u[0][qx].y, u[1][qx].x, u[1][qx].y};
                const Euler2State st = euler2_prim(A, q);
                Real Fx[4], Fy[4];
                euler2_flux(st, q, 0, Fx);
                euler2_flux(st, q, 1, Fy);
                if (need_lam) lam = max_nan(lam, euler2_speed(A, st, -1));
                fx[0][qx].x = Fx[0]; fx[0][qx].y = Fx[1]; fx[1][qx].x = Fx[2]; fx[1][qx].y = Fx[3];
                fy[0][qx].x = Fy[0]; fy[0][qx].y = Fy[1]; fy[1][qx].x = Fy[2]; fy[1][qx].y = Fy[3];
            }
#pragma unroll
            for (int pr = 0; pr < 2; ++pr) {
                R2 px[N1], py[N1];
                project_sym<true, N1, NQ>(T.WD, fx[pr], px);     // px[0] = 0 (P_0' = 0)
                project_sym<false, N1, NQ>(T.WB, fy[pr], py);
#pragma unroll
                for (int j = 0; j < N1; ++j)
#pragma unroll
                    for (int i = 0; i < N1; ++i) {
                        R2 t = acc[pr][i + N1 * j];
                        if (i > 0) t = vfma(T.WB[qy][j], px[i], t);
                        if (j > 0) t = vfma(T.WD[qy][j], py[i], t);   // P_0' = 0
                        acc[pr][i + N1 * j] = t;
                    }
            }
        }
    }

    // ---- 2. faces: x-faces f = 0..EX of each row, y-faces r = 0..EY of each column ----
    constexpr int NFX = (EX + 1) * EY, NFY = EX * (EY + 1);
    // prescribed-state sides read the stage's time
    const bool state_sides = A.bc[0] == BC_STATE || A.bc[1] == BC_STATE || A.bc[2] == BC_STATE || A.bc[3] == BC_STATE;
    const Real tnow = state_sides ? (Real)(*A.t_dev + A.t_off) : Real(0);
    for (int item = tid; item < NFX + NFY; item += ENT) {
        const bool xf = item < NFX;
        int rm, cm, rp, cp, fr, fc;       // staged positions of the minus / plus cell; face index
        if (xf) {
            fr = item / (EX + 1);
            fc = item - fr * (EX + 1);
            rm = rp = fr + 1;
            cm = fc;
            cp = fc + 1;
        } else {
            const int it = item - NFX;
            fr = it / EX;
            fc = it - fr * EX;
            cm = cp = fc + 1;
            rm = fr;
            rp = fr + 1;
        }
        // the face exists if the cell on either side is a cell of this tile in the mesh
        const int gxm = tx0 + cm - 1, gym = ty0 + rm - 1, gxp = tx0 + cp - 1, gyp = ty0 + rp - 1;
        const bool tile_m = (xf ? cm >= 1 : rm >= 1) && gxm < A.nx && gym < A.ny && gxm >= 0 && gym >= 0;
        const bool tile_p = (xf ? cp <= EX : rp <= EY) && gxp < A.nx && gyp < A.ny;
        if (!(tile_m && (xf ? cm <= EX : rm <= EY)) && !tile_p) continue;
        const bool has_m = S.has[rm][cm] != 0, has_p = S.has[rp][cp] != 0;
        const int axis = xf ? 0 : 1;
        // trace coefficients along the face (Legendre index t), both sides, both pairs
        R2 tm[2][N1], tp[2][N1];
#pragma unroll
        for (int pr = 0; pr < 2; ++pr)
#pragma unroll
            for (int t = 0; t < N1; ++t) {
                R2 sm = cu(pr, xf ? N1 * t : t, rm, cm), sp = cu(pr, xf ? N1 * t : t, rp, cp);
#pragma unroll
                for (int n = 1; n < N1; ++n) {
                    const int k = xf ? n + N1 * t : t + N1 * n;
                    sm = vadd(sm, cu(pr, k, rm, cm));                                  // xi = +1 of the minus cell
                    sp = (n & 1) ? vsub(sp, cu(pr, k, rp, cp)) : vadd(sp, cu(pr, k, rp, cp));   // xi = -1 of the plus cell
                }
                tm[pr][t] = sm;
                tp[pr][t] = sp;
            }
        R2 um2[2][NQ], up2[2][NQ], H[2][NQ];
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {
            interp_sym<N1, NQ>(T.B, tm[pr], um2[pr]);
            interp_sym<N1, NQ>(T.B, tp[pr], up2[pr]);
        }
        Real spm = Real(0), spp = Real(0);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            Real um[4] = {um2[0][q].x, um2[0][q].y, um2[1][q].x, um2[1][q].y};
            Real up[4] = {up2[0][q].x, up2[0][q].y, up2[1][q].x, up2[1][q].y};
            if (!has_m || !has_p) {
                // ghost: the inner state, mirrored at a wall; on a prescribed-state side one
                // of two states or a wall, by the point's coordinate along the side against
                // the split bsplit + bspeed t
                const int side = (xf ? 0 : 2) + (has_m ? 1 : 0);
                bool refl = A.bc[side] == BC_REFLECT;
                int ch = -1;
                if (A.bc[side] == BC_STATE) {
                    const Real along = xf ? A.y0 + (Real(ty0 + fr) + Real(0.5)) * A.h + A.hh * T.g[q]
                                          : A.x0 + (Real(tx0 + fc) + Real(0.5)) * A.h + A.hh * T.g[q];
                    ch = along < A.bsplit[side] + A.bspeed[side] * tnow ? A.bbelow[side] : A.babove[side];
                    refl = ch == 2;
                }
                Real* gh = has_m ? up : um;                 // the ghost side
                const Real* in_ = has_m ? um : up;          // the inner side
#pragma unroll
                for (int comp = 0; comp < 4; ++comp)
                    gh[comp] = (ch == 0 || ch == 1) ? A.bstate[ch][comp] : in_[comp];
                if (refl && axis == 0) gh[1] = -in_[1];
                if (refl && axis == 1) gh[2] = -in_[2];
            }
            const Euler2State sl = euler2_prim(A, um), sr = euler2_prim(A, up);
            Real Fl[4], Fr[4];
            euler2_flux(sl, um, axis, Fl);
            euler2_flux(sr, up, axis, Fr);
            const Real snl = euler2_speed(A, sl, axis), snr = euler2_speed(A, sr, axis);
            const Real s = max_nan(snl, snr);
            if (need_lam) {
                spm = max_nan(spm, euler2_speed(A, sl, -1));
                spp = max_nan(spp, euler2_speed(A, sr, -1));
            }
            // H = ((F(U-) + F(U+)) - s+ (U+ - U-)) / 2, a pair at a time
#pragma unroll
            for (int pr = 0; pr < 2; ++pr) {
                R2 fs, du;
                fs.x = Fl[2 * pr] + Fr[2 * pr];
                fs.y = Fl[2 * pr + 1] + Fr[2 * pr + 1];
                du.x = up[2 * pr] - um[2 * pr];
                du.y = up[2 * pr + 1] - um[2 * pr + 1];
                H[pr][q] = vmul(Real(0.5), vfma(-s, du, fs));
            }
        }
        R2 hq[2][N1];
        project_sym<false, N1, NQ>(T.WB, H[0], hq[0]);
        project_sym<false, N1, NQ>(T.WB, H[1], hq[1]);
        if (xf) {
#pragma unroll
            for (int pr = 0; pr < 2; ++pr)
#pragma unroll
                for (int t = 0; t < N1; ++t) {
                    S.hx[pr][t][fr][fc] = hq[pr][t];
                }
            S.sx[0][fr][fc] = spm;
            S.sx[1][fr][fc] = spp;
        } else {
#pragma unroll
            for (int pr = 0; pr < 2; ++pr)
#pragma unroll
                for (int t = 0; t < N1; ++t) {
                    S.hy[pr][t][fr][fc] = hq[pr][t];
                }
            S.sy[0][fr][fc] = spm;
            S.sy[1][fr][fc] = spp;
        }
    }
    __syncthreads();
    if (!in) return;

    // ---- 3. face terms, stabilization, M^{-1}, Runge-Kutta combination ----
    if (need_lam)
        lam = max_nan(lam, max_nan(max_nan(S.sx[1][ly][lx], S.sx[0][ly][lx + 1]),
                                   max_nan(S.sy[1][ly][lx], S.sy[0][ly + 1][lx])));
    const Real ngs = A.stab == STAB_DG ? Real(0) : -(gamma * (A.lam_fixed ? A.lambda_nu : lam) * Real(1.0 / P));
    Real chk = Real(0);
    if (copy_un) asm volatile("cp.async.wait_all;" ::: "memory");   // this thread's own copies
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
#pragma unroll
        for (int t = 0; t < N1; ++t) {
            // even n: += (m - p); odd n: -= (m + p)
            const R2 xm = S.hx[pr][t][ly][lx], xp = S.hx[pr][t][ly][lx + 1];
            const R2 ym = S.hy[pr][t][ly][lx], yp = S.hy[pr][t][ly + 1][lx];
            const R2 dxe = vsub(xm, xp), dxo = vadd(xm, xp), dye = vsub(ym, yp), dyo = vadd(ym, yp);
#pragma unroll
            for (int n = 0; n < N1; ++n) {
                acc[pr][n + N1 * t] = (n & 1) ? vsub(acc[pr][n + N1 * t], dxo) : vadd(acc[pr][n + N1 * t], dxe);
                acc[pr][t + N1 * n] = (n & 1) ? vsub(acc[pr][t + N1 * n], dyo) : vadd(acc[pr][t + N1 * n], dye);
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = k % N1, j = k / N1;
            R2 s1 = vbc<R2>(0), s2 = vbc<R2>(0);
#pragma unroll
            for (int m = 1; m < N1; ++m) {
                if (((i + m) & 1) == 0 && i > 0) s1 = vfma(T.A1[i][m], cu(pr, m + N1 * j, r0, c0), s1);
                if (((j + m) & 1) == 0 && j > 0) s2 = vfma(T.A1[j][m], cu(pr, i + N1 * m, r0, c0), s2);
            }
            const R2 r = vfma(ngs, vfma(T.A0[i], s2, vmul(T.A0[j], s1)), acc[pr][k]);
            const R2 Lk = vmul(A.two_h * (T.minv[i] * T.minv[j]), r);
            R2 out = vfma(A.cl, Lk, vmul(A.ck, cu(pr, k, r0, c0)));
            if (A.has_un) {
                R2 unk;
                if constexpr (kF32) {
                    unk = S.un[pr][k][ly][lx];
                } else {
                    const Real* a0 = A.Un + e + (int64_t)(2 * pr * K + k) * E;
                    const Real* a1 = a0 + (int64_t)K * E;
                    unk.x = A.cg_loads ? __ldcg(a0) : *a0;
                    unk.y = A.cg_loads ? __ldcg(a1) : *a1;
                }
                out = vfma(A.cn, unk, out);
            }
            chk = fma(out.x, Real(0), fma(out.y, Real(0), chk));
            A.Uout[e + (int64_t)(2 * pr * K + k) * E] = out.x;
            A.Uout[e + (int64_t)((2 * pr + 1) * K + k) * E] = out.y;
        }
    }
    if (chk != chk) atomicOr(A.flag, 1u);
}

template <int P>
static cudaError_t launch_euler2d_p(const StageArgs& s, int mode, cudaStream_t st)
{
    const KParams a = make_params(s);
    dim3 grid((s.nx + EX - 1) / EX, (s.ny + EY - 1) / EY);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    const size_t smem = sizeof(Euler2Smem<P>);
    static bool opted[64][2] = {{false, false}};
    const int dev = cur_device();
    if (!opted[dev][mode]) {
        const void* fn = mode == 0 ? (const void*)euler2d_kernel<P, 0> : (const void*)euler2d_kernel<P, 1>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        opted[dev][mode] = true;
    }
    if (mode == 0) euler2d_kernel<P, 0><<<grid, ENT, smem, st>>>(a);
    else euler2d_kernel<P, 1><<<grid, ENT, smem, st>>>(a);
    return cudaGetLastError();
}

static cudaError_t launch_euler2d(const StageArgs& s, int p, int mode, cudaStream_t st)
{
    switch (p) {
    case 1: return launch_euler2d_p<1>(s, mode, st);
    case 2: return launch_euler2d_p<2>(s, mode, st);
    case 3: return launch_euler2d_p<3>(s, mode, st);
    default: return cudaErrorInvalidValue;
    }
}
