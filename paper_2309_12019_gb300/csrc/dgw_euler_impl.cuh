// Stage kernel of the 1D Euler system (Sec. 5.6), included by the 1D stage translation
// units after the scalar kernel (it shares the tables, the launch scalars and the math
// helpers of dgw_stage_impl.cuh).
//
// State U = (rho, rho v, rho E) with p = (gamma - 1)(rho E - rho v^2 / 2); coefficient k
// of component comp of cell e at row comp (p+1) + k, i.e. U[(comp (p+1) + k) E + e].
// One CTA of TX threads owns TX consecutive cells, one per thread:
//   0. each thread loads its cell (one coalesced row per coefficient) and puts its
//      density coefficients and its six end-point values in shared memory; two threads
//      fetch the cells on either side of the tile's cells (the periodic image, or none
//      beyond a wall or an outflow side)
//   1. the sensor of Sec. 4 applied to the density (Sec. 5.6), the volume term at the
//      p+2 Gauss points, and lambda_e = max (|v| + c) over those points and the ends
//   2. every face of the tile once: the LLF flux with s+ the larger |v| + c of the two
//      states; beyond a wall the ghost state mirrors the momentum, beyond an outflow
//      side it copies the inner state
//   3. face terms, the stabilization of every component with the density's gamma,
//      M^{-1} and the Runge-Kutta combination Uout = cn Un + ck Uk + cl L(Uk)
// The operator constants are folded as in the scalar kernel:
//   L_k = (2/h) minv(k) [acc_k - gamma lambda / p (K_ref c)_k].

template <int P>
struct EulerSmem {
    static constexpr int N1 = P + 1;
    Real rho[N1][TX + 2];     // density coefficients, column lx + 1; halo cells 0 and nt + 1
    Real tr[2][3][TX + 2];    // values at xi = -1 (0) and xi = +1 (1), same columns
    Real hf[3][TX + 1];       // LLF flux of face f, between columns f and f + 1
    Real sp[2][TX + 1];       // |v| + c of the left (0) and right (1) state of face f
    int has[2];               // the halo cell on the left / right exists
};

struct EulerState {
    Real v, pr, inv_rho;
};

__device__ __forceinline__ EulerState euler_prim(const KParams& A, Real rho, Real m, Real en)
{
    EulerState s;
    s.inv_rho = rcp_e(rho);
    s.v = m * s.inv_rho;
    s.pr = A.gm1 * (en - Real(0.5) * m * s.v);
    return s;
}

__device__ __forceinline__ Real euler_speed(const KParams& A, const EulerState& s)
{
    return fabs(s.v) + sqrt_e(A.gam * s.pr * s.inv_rho);
}

// F(U) = (rho v, rho v^2 + p, (rho E + p) v)
__device__ __forceinline__ void euler_flux(const EulerState& s, Real m, Real en, Real F[3])
{
    F[0] = m;
    F[1] = fma(m, s.v, s.pr);
    F[2] = (en + s.pr) * s.v;
}

// Sensor of Sec. 4 (or the comparison sensor of Zhao et al., stab = ZHAO) of a 1D cell
// with coefficients c from its face neighbours cn[0] (left) and cn[1] (right), where
// they exist.
template <int P>
__device__ __forceinline__ Real sensor_1d(const KParams& A, const Tab<P>& T, const Real* c, const Real (*cn)[P + 1],
                                          const bool* has)
{
    constexpr int N1 = P + 1;
    const int me = (has[0] ? 1 : 0) + (has[1] ? 1 : 0);
    const Real beta0 = qform<P>(T, c);
    const Real d0 = A.eps_w + beta0;
    const Real w0 = div_w(Real(1) - Real(me) * A.w_nbr, d0 * d0);
    Real wsum = w0;
    Real wnb[2] = {Real(0), Real(0)};
    Real dacc[N1];
#pragma unroll
    for (int k = 0; k < N1; ++k) dacc[k] = Real(0);
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        if (!has[f]) continue;
        // Hermite candidate: the neighbour's polynomial continued into this cell, mean
        // dropped (it does not enter the seminorms)
        Real cl[N1];
        cl[0] = Real(0);
#pragma unroll
        for (int k = 1; k < N1; ++k) {
            Real s = Real(0);
#pragma unroll
            for (int m = k; m < N1; ++m) s = fma(T.T[f][k][m], cn[f][m], s);
            cl[k] = s;
        }
        const Real dl = A.eps_w + qform<P>(T, cl);
        const Real wl = div_w(A.w_nbr, dl * dl);
        wsum += wl;
        wnb[f] = wl;
#pragma unroll
        for (int k = 1; k < N1; ++k) dacc[k] = fma(wl, c[k] - cl[k], dacc[k]);
    }
    const Real inv = div_w(Real(1), wsum);
    if (A.stab == STAB_ZHAO) {
        if (me == 0) return Real(0);
        const Real lin0 = Real(1) - Real(me) * A.w_nbr;
        Real dev = zpow(A, fabs(w0 * inv / lin0 - Real(1)));
#pragma unroll
        for (int f = 0; f < 2; ++f)
            if (has[f]) dev += zpow(A, fabs(wnb[f] * inv / A.w_nbr - Real(1)));
        const Real minlin = lin0 < A.w_nbr ? lin0 : A.w_nbr;
        return dev * rcp_e(zpow(A, fabs(rcp_e(minlin) - Real(1))) + Real(me));
    }
    // U - U* = sum_l w_l (c - c_l); the ratio r = ||U - U*|| / ||U|| is taken through
    // its square: r <= 1 iff qd <= beta0, r < b iff r^2 < b^2, ||U - U*|| <= eps_s iff
    // qd <= eps_s^2
#pragma unroll
    for (int k = 1; k < N1; ++k) dacc[k] *= inv;
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
__global__ void __launch_bounds__(TX, kF32 ? 8 : 4) euler_kernel(const __grid_constant__ KParams A)
{
    constexpr int N1 = P + 1, NQ = P + 2;
    __shared__ EulerSmem<P> S;
    const Tab<P>& T = tab<P>();
    const int tid = threadIdx.x;
    const int64_t E = A.E;
    const int tx0 = blockIdx.x * TX;
    const int nt = A.nx - tx0 < TX ? A.nx - tx0 : TX;     // cells of this tile
    const int gx = tx0 + tid;
    const bool in = tid < nt;

    // ---- 0. own cell, halo cells ----
    Real c[3][N1];
#pragma unroll
    for (int comp = 0; comp < 3; ++comp)
#pragma unroll
        for (int k = 0; k < N1; ++k) c[comp][k] = Real(0);
    auto put = [&](const Real (&q)[3][N1], int col) {
#pragma unroll
        for (int k = 0; k < N1; ++k) S.rho[k][col] = q[0][k];
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
            Real xm = Real(0), xp = Real(0);
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                xp += q[comp][k];
                xm = (k & 1) ? xm - q[comp][k] : xm + q[comp][k];
            }
            S.tr[0][comp][col] = xm;
            S.tr[1][comp][col] = xp;
        }
    };
    // Un is read only by the final combination: its loads are issued here, so that their
    // latency hides behind the sensor, volume and face work
    Real un[3][N1];
    if (in) {
        const Real* src = A.Uk + gx;
#pragma unroll
        for (int comp = 0; comp < 3; ++comp)
#pragma unroll
            for (int k = 0; k < N1; ++k) c[comp][k] = src[(int64_t)(comp * N1 + k) * E];
        if (MODE == 0 && A.has_un) {
            const Real* usrc = A.Un + gx;
#pragma unroll
            for (int comp = 0; comp < 3; ++comp)
#pragma unroll
                for (int k = 0; k < N1; ++k) {
                    const Real* a = usrc + (int64_t)(comp * N1 + k) * E;
                    un[comp][k] = A.cg_loads ? __ldcg(a) : *a;
                }
        }
        put(c, tid + 1);
    }
    if (tid < 2) {
        const int hx = wrap_x(A, tid == 0 ? tx0 - 1 : tx0 + nt);
        S.has[tid] = hx >= 0;
        if (hx >= 0) {
            Real q[3][N1];
            const Real* src = A.Uk + hx;
#pragma unroll
            for (int comp = 0; comp < 3; ++comp)
#pragma unroll
                for (int k = 0; k < N1; ++k) q[comp][k] = src[(int64_t)(comp * N1 + k) * E];
            put(q, tid == 0 ? 0 : nt + 1);
        }
    }
    __syncthreads();

    // ---- 1. sensor of the density ----
    Real gamma = (MODE == 0 && A.stab == STAB_LO) ? Real(1) : Real(0);
    if (in && (MODE == 1 || A.stab >= STAB_WENO)) {
        const bool has[2] = {tid > 0 || S.has[0] != 0, tid < nt - 1 || S.has[1] != 0};
        Real cn[2][N1];
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            cn[0][k] = has[0] ? S.rho[k][tid] : Real(0);
            cn[1][k] = has[1] ? S.rho[k][tid + 2] : Real(0);
        }
        gamma = sensor_1d<P>(A, T, c[0], cn, has);
        if (MODE == 1) A.gamma_out[gx] = (double)gamma;
    }
    if (MODE == 1) return;

    // ---- 1b. volume term: acc_i = sum_q W_q P_i'(g_q) F(U_h(g_q)); lambda_e ----
    Real acc[3][N1];
#pragma unroll
    for (int comp = 0; comp < 3; ++comp)
#pragma unroll
        for (int k = 0; k < N1; ++k) acc[comp][k] = Real(0);
    Real lam = Real(0);
    const bool need_lam = A.stab != STAB_DG && !A.lam_fixed;
    if (in) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            Real u[3];
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) {
                Real s = Real(0);
#pragma unroll
                for (int k = 0; k < N1; ++k) s = fma(T.B[q][k], c[comp][k], s);
                u[comp] = s;
            }
            const EulerState st = euler_prim(A, u[0], u[1], u[2]);
            Real F[3];
            euler_flux(st, u[1], u[2], F);
            if (need_lam) lam = max_nan(lam, euler_speed(A, st));
#pragma unroll
            for (int comp = 0; comp < 3; ++comp)
#pragma unroll
                for (int k = 0; k < N1; ++k) acc[comp][k] = fma(T.WD[q][k], F[comp], acc[comp][k]);
        }
    }

    // ---- 2. faces f = 0 .. nt of the tile ----
    for (int f = tid; f <= nt; f += TX) {
        Real uL[3], uR[3];
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
            uL[comp] = S.tr[1][comp][f];
            uR[comp] = S.tr[0][comp][f + 1];
        }
        const bool wall_l = f == 0 && !S.has[0];
        const bool wall_r = f == nt && !S.has[1];
        if (wall_l) {
            const bool refl = A.bc[0] == BC_REFLECT;
            uL[0] = uR[0]; uL[1] = refl ? -uR[1] : uR[1]; uL[2] = uR[2];
        } else if (wall_r) {
            const bool refl = A.bc[1] == BC_REFLECT;
            uR[0] = uL[0]; uR[1] = refl ? -uL[1] : uL[1]; uR[2] = uL[2];
        }
        const EulerState sl = euler_prim(A, uL[0], uL[1], uL[2]);
        const EulerState sr = euler_prim(A, uR[0], uR[1], uR[2]);
        Real FL[3], FR[3];
        euler_flux(sl, uL[1], uL[2], FL);
        euler_flux(sr, uR[1], uR[2], FR);
        const Real spl = euler_speed(A, sl), spr = euler_speed(A, sr);
        S.sp[0][f] = spl;
        S.sp[1][f] = spr;
        const Real s = max_nan(spl, spr);
#pragma unroll
        for (int comp = 0; comp < 3; ++comp)
            S.hf[comp][f] = Real(0.5) * ((FL[comp] + FR[comp]) - s * (uR[comp] - uL[comp]));
    }
    __syncthreads();
    if (!in) return;

    // ---- 3. face terms, stabilization, M^{-1}, Runge-Kutta combination ----
    // lambda_e: also |v| + c at the cell's two ends, its own states at faces tid, tid + 1
    if (need_lam) lam = max_nan(lam, max_nan(S.sp[1][tid], S.sp[0][tid + 1]));
    const Real ngs = A.stab == STAB_DG ? Real(0) : -(gamma * (A.lam_fixed ? A.lambda_nu : lam) * Real(1.0 / P));
    Real chk = Real(0);
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        const Real hm = S.hf[comp][tid], hp = S.hf[comp][tid + 1];
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            // -P_k(+1) H_right + P_k(-1) H_left
            Real r = acc[comp][k] + ((k & 1) ? -(hm + hp) : (hm - hp));
            if (k > 0) {
                Real kc = Real(0);
#pragma unroll
                for (int m = 1; m < N1; ++m)
                    if (((k + m) & 1) == 0) kc = fma(T.A1[k][m], c[comp][m], kc);
                r = fma(ngs, kc, r);
            }
            const Real Lk = (A.two_h * T.minv[k]) * r;
            const int64_t idx = (int64_t)(comp * N1 + k) * E + gx;
            Real out = fma(A.cl, Lk, A.ck * c[comp][k]);
            if (A.has_un) out = fma(A.cn, un[comp][k], out);
            chk = fma(out, Real(0), chk);
            A.Uout[idx] = out;
        }
    }
    if (chk != chk) atomicOr(A.flag, 1u);
}

template <int P>
static cudaError_t launch_euler_p(const StageArgs& s, int mode, cudaStream_t st)
{
    const KParams a = make_params(s);
    const unsigned grid = (unsigned)((s.nx + TX - 1) / TX);
    if (grid == 0) return cudaSuccess;
    if (mode == 0) euler_kernel<P, 0><<<grid, TX, 0, st>>>(a);
    else euler_kernel<P, 1><<<grid, TX, 0, st>>>(a);
    return cudaGetLastError();
}

static cudaError_t launch_euler(const StageArgs& s, int p, int mode, cudaStream_t st)
{
    switch (p) {
    case 1: return launch_euler_p<1>(s, mode, st);
    case 2: return launch_euler_p<2>(s, mode, st);
    case 3: return launch_euler_p<3>(s, mode, st);
    default: return cudaErrorInvalidValue;
    }
}
