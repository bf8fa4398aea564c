// Stage kernel of the WENO-stabilized RKDG scheme: one thread per element.
//
// Included by one translation unit per (precision, dimension) with DGW_REAL, DGW_DIM
// and DGW_NS defined.  Each unit owns its copy of the constant-memory operator tables.
//
// Per element e the kernel computes, from the state Uk,
//   volume  : sum_q W_q grad_ref(phi_k) . F(U_h(x_q))                 (Eq. weak2)
//   faces   : - sum_faces sum_q w_q phi_k(x_q) H_LLF(U-, U+, n)         (Sec. 2)
//   sensor  : Hermite candidates from the face neighbours, nonlinear weights,
//             gamma_e = min(1, ||U - U*||_e / ||U||_e)^q               (Sec. 4)
//   stab    : gamma_e nu_e K c with nu_e = lambda_e h / (2p)            (Sec. 3)
//   L       = M^{-1}(...), then  Uout = cn Un + ck Uk + cl L           (Eq. ssp)
// in the reference element, with all constant factors folded:
//   L_k = (2/h) minv(k) [acc_k - gamma lambda/p (K_ref c)_k].
#include <cmath>

#include "dgw_internal.h"

namespace dgw {
namespace DGW_NS {

using Real = DGW_REAL;
constexpr int DIM = DGW_DIM;

template <int P>
struct Tab {
    static constexpr int N1 = P + 1, NQ = P + 2, K = (DIM == 1) ? N1 : N1 * N1;
    Real g[NQ], w[NQ];
    Real B[NQ][N1];      // P_i(g_q)
    Real D[NQ][N1];      // P_i'(g_q)
    Real T[2][N1][N1];   // Hermite shift: coefficient of P_i in P_m(xi + 2) / P_m(xi - 2)
    Real Gu[K][K];       // seminorm Gram, upper triangle with doubled off-diagonal
    Real A1[N1][N1];     // int P_i' P_m'
    Real A0[N1];         // 2 / (2i + 1)
    Real minv[N1];       // (2i + 1) / 2
};

__constant__ Tab<1> c_tab1;
__constant__ Tab<2> c_tab2;
__constant__ Tab<3> c_tab3;

template <int P> __device__ __forceinline__ const Tab<P>& tab();
template <> __device__ __forceinline__ const Tab<1>& tab<1>() { return c_tab1; }
template <> __device__ __forceinline__ const Tab<2>& tab<2>() { return c_tab2; }
template <> __device__ __forceinline__ const Tab<3>& tab<3>() { return c_tab3; }

template <int P>
static cudaError_t upload(const HostTables& h)
{
    Tab<P> t;
    constexpr int N1 = Tab<P>::N1, NQ = Tab<P>::NQ, K = Tab<P>::K;
    for (int q = 0; q < NQ; ++q) {
        t.g[q] = (Real)h.g[q];
        t.w[q] = (Real)h.w[q];
        for (int i = 0; i < N1; ++i) { t.B[q][i] = (Real)h.B[q][i]; t.D[q][i] = (Real)h.D[q][i]; }
    }
    for (int s = 0; s < 2; ++s)
        for (int i = 0; i < N1; ++i)
            for (int m = 0; m < N1; ++m) t.T[s][i][m] = (Real)h.T[s][i][m];
    for (int a = 0; a < K; ++a)
        for (int b = 0; b < K; ++b) {
            double v = (DIM == 1) ? h.G1[a][b] : h.G2[a][b];
            t.Gu[a][b] = (Real)(b < a ? 0.0 : (b == a ? v : 2.0 * v));
        }
    for (int i = 0; i < N1; ++i) {
        for (int m = 0; m < N1; ++m) t.A1[i][m] = (Real)h.A1[i][m];
        t.A0[i] = (Real)h.A0[i];
        t.minv[i] = (Real)h.minv[i];
    }
    if (P == 1) return cudaMemcpyToSymbol(c_tab1, &t, sizeof(Tab<1>));
    if (P == 2) return cudaMemcpyToSymbol(c_tab2, &t, sizeof(Tab<2>));
    return cudaMemcpyToSymbol(c_tab3, &t, sizeof(Tab<3>));
}

// ------------------------------------------------------------------------------------
// math helpers
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void sincos_r(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_r(double x, double* s, double* c) { sincos(x, s, c); }

constexpr double kPi = 3.14159265358979323846;

struct FluxP {
    Real a0, a1, cx, cy, omega;
};

// Volume flux F(u) at (x, y) and |F'(u)|_2 (1D: only the x component).
template <int FLUX>
__device__ __forceinline__ void vol_flux(const FluxP& fp, Real u, Real x, Real y,
                                         Real& fx, Real& fy, Real& spd)
{
    if (FLUX == FLUX_ADVECT) {
        fx = fp.a0 * u; fy = fp.a1 * u;
        spd = DIM == 1 ? fabs(fp.a0) : sqrt(fp.a0 * fp.a0 + fp.a1 * fp.a1);
    } else if (FLUX == FLUX_ROTATION) {
        Real vx = fp.omega * (fp.cy - y), vy = fp.omega * (x - fp.cx);
        fx = vx * u; fy = vy * u;
        spd = DIM == 1 ? fabs(vx) : sqrt(vx * vx + vy * vy);
    } else if (FLUX == FLUX_BURGERS) {
        Real hu2 = Real(0.5) * u * u;
        fx = fp.a0 * hu2; fy = fp.a1 * hu2;
        spd = DIM == 1 ? fabs(fp.a0 * u) : sqrt(fp.a0 * fp.a0 + fp.a1 * fp.a1) * fabs(u);
    } else {  // KPP
        Real s, c;
        sincos_r(u, &s, &c);
        fx = s; fy = c;
        spd = DIM == 1 ? fabs(c) : Real(1);
    }
}

// |F'(u)|_2 only (for lambda_e at face points).
template <int FLUX>
__device__ __forceinline__ Real speed_norm(const FluxP& fp, Real u, Real x, Real y)
{
    Real fx, fy, spd;
    if (FLUX == FLUX_KPP && DIM == 2) return Real(1);
    vol_flux<FLUX>(fp, u, x, y, fx, fy, spd);
    return spd;
}

// F'(u) along the axis (for the inflow test of the ghost state).
template <int FLUX>
__device__ __forceinline__ Real dflux_axis(const FluxP& fp, int axis, Real u, Real x, Real y)
{
    if (FLUX == FLUX_ADVECT) return axis == 0 ? fp.a0 : fp.a1;
    if (FLUX == FLUX_ROTATION) return axis == 0 ? fp.omega * (fp.cy - y) : fp.omega * (x - fp.cx);
    if (FLUX == FLUX_BURGERS) return (axis == 0 ? fp.a0 : fp.a1) * u;
    Real s, c;
    sincos_r(u, &s, &c);
    return axis == 0 ? c : -s;
}

// Local Lax-Friedrichs flux for the normal sgn * e_axis (Sec. 2), with the exact
// maximal wave speed over the segment between um and up.
template <int FLUX>
__device__ __forceinline__ Real llf(const FluxP& fp, int axis, Real sgn, Real um, Real up,
                                    Real x, Real y)
{
    if (FLUX == FLUX_ADVECT || FLUX == FLUX_ROTATION) {
        Real v = FLUX == FLUX_ADVECT ? (axis == 0 ? fp.a0 : fp.a1)
                                     : (axis == 0 ? fp.omega * (fp.cy - y) : fp.omega * (x - fp.cx));
        Real vn = sgn * v;
        return Real(0.5) * vn * (um + up) - Real(0.5) * fabs(vn) * (up - um);
    } else if (FLUX == FLUX_BURGERS) {
        Real an = sgn * (axis == 0 ? fp.a0 : fp.a1);
        Real s = fabs(an) * fmax(fabs(um), fabs(up));
        return Real(0.25) * an * (um * um + up * up) - Real(0.5) * s * (up - um);
    } else {
        // x-normal: n.F = sgn sin u, |F'.n| = |cos u| (maximal at multiples of pi);
        // y-normal: n.F = sgn cos u, |F'.n| = |sin u| (maximal at pi/2 + multiples of pi).
        Real sm, cm, sp, cp;
        sincos_r(um, &sm, &cm);
        sincos_r(up, &sp, &cp);
        Real lo = fmin(um, up), hi = fmax(um, up);
        Real shift = axis == 0 ? Real(0) : Real(0.5 * kPi);
        Real k = ceil((lo - shift) / Real(kPi));
        Real s;
        if (k * Real(kPi) + shift <= hi) {
            s = Real(1);
        } else {
            s = axis == 0 ? fmax(fabs(cm), fabs(cp)) : fmax(fabs(sm), fabs(sp));
        }
        Real fm = axis == 0 ? sm : cm, fpl = axis == 0 ? sp : cp;
        return Real(0.5) * sgn * (fm + fpl) - Real(0.5) * s * (up - um);
    }
}

// Quadratic form v^T G v over modes >= 1 (row and column 0 of G vanish).  G is nonzero
// only where both Legendre degree pairs have even sums.
template <int P>
__device__ __forceinline__ Real qform(const Tab<P>& T, const Real* v)
{
    constexpr int N1 = P + 1, K = Tab<P>::K;
    Real s = Real(0);
#pragma unroll
    for (int a = 1; a < K; ++a) {
        Real t = Real(0);
#pragma unroll
        for (int b = a; b < K; ++b) {
            const int ia = a % N1, ja = a / N1, ib = b % N1, jb = b / N1;
            if (((ia + ib) & 1) == 0 && ((ja + jb) & 1) == 0) t += T.Gu[a][b] * v[b];
        }
        s += v[a] * t;
    }
    return s;
}

// Neighbour across face f (0:-x 1:+x 2:-y 3:+y); false at a non-periodic boundary.
__device__ __forceinline__ bool neighbour(const StageArgs& A, int ix, int iy, int f, int64_t& idx)
{
    int jx = ix + (f == 0 ? -1 : (f == 1 ? 1 : 0));
    int jy = iy + (f == 2 ? -1 : (f == 3 ? 1 : 0));
    if (jx < 0 || jx >= A.nx) {
        if (A.bc[f] != BC_PERIODIC) return false;
        jx = jx < 0 ? A.nx - 1 : 0;
    }
    if (DIM == 2 && (jy < 0 || jy >= A.ny)) {
        if (A.bc[f] != BC_PERIODIC) return false;
        jy = jy < 0 ? A.ny - 1 : 0;
    }
    idx = (int64_t)jy * A.nx + jx;
    return true;
}

// MODE 0: stage / residual; MODE 1: sensor only.
template <int P, int FLUX, int MODE>
__global__ void __launch_bounds__(128) stage_kernel(const StageArgs A)
{
    constexpr int N1 = P + 1, NQ = P + 2;
    constexpr int K = Tab<P>::K;
    const Tab<P>& T = tab<P>();
    const int64_t E = A.E;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const Real* __restrict__ Uk = static_cast<const Real*>(A.Uk);
    const int ix = (int)(e % A.nx);
    const int iy = DIM == 2 ? (int)(e / A.nx) : 0;

    Real c[K];
#pragma unroll
    for (int k = 0; k < K; ++k) c[k] = Uk[k * E + e];

    const Real h = (Real)A.h;
    const Real hh = (Real)(0.5 * A.h);
    const Real xc = (Real)(A.x0 + (ix + 0.5) * A.h);
    const Real yc = DIM == 2 ? (Real)(A.y0 + (iy + 0.5) * A.h) : Real(0);
    const FluxP fp{(Real)A.a0, (Real)A.a1, (Real)A.cx, (Real)A.cy, (Real)A.omega};
    const bool weno = (MODE == 1) || (A.stab == STAB_WENO);
    const bool need_lam = (MODE == 0) && (A.stab != STAB_DG) && !(A.lambda_nu > 0.0);

    Real acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = Real(0);
    Real lam = Real(0);

    // ---------------- volume term ----------------
    if (MODE == 0) {
        if (DIM == 1) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                Real u = Real(0);
#pragma unroll
                for (int i = 0; i < N1; ++i) u += c[i] * T.B[q][i];
                Real fx, fy, spd;
                vol_flux<FLUX>(fp, u, xc + hh * T.g[q], Real(0), fx, fy, spd);
                lam = fmax(lam, spd);
                const Real wf = T.w[q] * fx;
#pragma unroll
                for (int i = 0; i < N1; ++i) acc[i] += T.D[q][i] * wf;
            }
        } else {
            // tmp[j][qx] = sum_i c_ij P_i(g_qx)
            Real tmp[N1][NQ];
#pragma unroll
            for (int j = 0; j < N1; ++j)
#pragma unroll
                for (int qx = 0; qx < NQ; ++qx) {
                    Real s = Real(0);
#pragma unroll
                    for (int i = 0; i < N1; ++i) s += c[i + N1 * j] * T.B[qx][i];
                    tmp[j][qx] = s;
                }
#pragma unroll
            for (int qy = 0; qy < NQ; ++qy) {
                const Real y = yc + hh * T.g[qy];
                Real px[N1], py[N1];
#pragma unroll
                for (int i = 0; i < N1; ++i) { px[i] = Real(0); py[i] = Real(0); }
#pragma unroll
                for (int qx = 0; qx < NQ; ++qx) {
                    Real u = Real(0);
#pragma unroll
                    for (int j = 0; j < N1; ++j) u += tmp[j][qx] * T.B[qy][j];
                    Real fx, fy, spd;
                    vol_flux<FLUX>(fp, u, xc + hh * T.g[qx], y, fx, fy, spd);
                    lam = fmax(lam, spd);
                    const Real wfx = T.w[qx] * fx, wfy = T.w[qx] * fy;
#pragma unroll
                    for (int i = 0; i < N1; ++i) {
                        px[i] += T.D[qx][i] * wfx;
                        py[i] += T.B[qx][i] * wfy;
                    }
                }
#pragma unroll
                for (int j = 0; j < N1; ++j) {
                    const Real bj = T.w[qy] * T.B[qy][j], dj = T.w[qy] * T.D[qy][j];
#pragma unroll
                    for (int i = 0; i < N1; ++i) acc[i + N1 * j] += bj * px[i] + dj * py[i];
                }
            }
        }
    }

    // ------------- faces and sensor, one neighbour at a time -------------
    int me = 0;
    int64_t nidx[2 * DIM];
    bool has[2 * DIM];
#pragma unroll
    for (int f = 0; f < 2 * DIM; ++f) {
        has[f] = neighbour(A, ix, iy, f, nidx[f]);
        me += has[f] ? 1 : 0;
    }
    const Real w_nbr = (Real)A.w_nbr, eps_w = (Real)A.eps_w;
    const Real beta0 = weno ? qform<P>(T, c) : Real(0);
    Real wsum = Real(0);
    Real dacc[K];   // sum_l wt_l (c - c_l), modes >= 1
#pragma unroll
    for (int k = 0; k < K; ++k) dacc[k] = Real(0);
    if (weno) {
        const Real lin0 = Real(1) - Real(me) * w_nbr;
        const Real d0 = eps_w + beta0;
        wsum = lin0 / (d0 * d0);
    }

#pragma unroll
    for (int f = 0; f < 2 * DIM; ++f) {
        const int axis = f >> 1;
        const int side = f & 1;                   // 0: minus side, 1: plus side
        const Real sgn = side ? Real(1) : Real(-1);
        Real cn[K];
        if (has[f]) {
#pragma unroll
            for (int k = 0; k < K; ++k) cn[k] = Uk[k * E + nidx[f]];
        }
        if (MODE == 0) {
            // traces: own at xi_axis = sgn, neighbour at xi_axis = -sgn
            if (DIM == 1) {
                Real um = Real(0), up = Real(0);
#pragma unroll
                for (int i = 0; i < N1; ++i) {
                    const Real ps = (side || (i % 2 == 0)) ? Real(1) : Real(-1);   // P_i(sgn)
                    um += ps * c[i];
                    if (has[f]) up += ((!side) || (i % 2 == 0) ? Real(1) : Real(-1)) * cn[i];
                }
                const Real xf = xc + sgn * hh;
                if (!has[f]) up = (A.bc[f] == BC_INFLOW_ZERO && sgn * dflux_axis<FLUX>(fp, 0, um, xf, Real(0)) < Real(0)) ? Real(0) : um;
                if (need_lam) lam = fmax(lam, speed_norm<FLUX>(fp, um, xf, Real(0)));
                const Real H = llf<FLUX>(fp, 0, sgn, um, up, xf, Real(0));
#pragma unroll
                for (int i = 0; i < N1; ++i) {
                    const Real ps = (side || (i % 2 == 0)) ? Real(1) : Real(-1);
                    acc[i] -= ps * H;
                }
            } else {
                // trace coefficients along the face (index t runs along the face)
                Real to[N1], tn[N1];
#pragma unroll
                for (int t = 0; t < N1; ++t) {
                    Real so = Real(0), sn = Real(0);
#pragma unroll
                    for (int n = 0; n < N1; ++n) {
                        const int ko = axis == 0 ? n + N1 * t : t + N1 * n;
                        const Real po = (side || (n % 2 == 0)) ? Real(1) : Real(-1);
                        const Real pn = ((!side) || (n % 2 == 0)) ? Real(1) : Real(-1);
                        so += po * c[ko];
                        if (has[f]) sn += pn * cn[ko];
                    }
                    to[t] = so;
                    tn[t] = sn;
                }
                Real hq[N1];
#pragma unroll
                for (int t = 0; t < N1; ++t) hq[t] = Real(0);
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    Real um = Real(0), up = Real(0);
#pragma unroll
                    for (int t = 0; t < N1; ++t) { um += to[t] * T.B[q][t]; up += tn[t] * T.B[q][t]; }
                    const Real xq = axis == 0 ? xc + sgn * hh : xc + hh * T.g[q];
                    const Real yq = axis == 0 ? yc + hh * T.g[q] : yc + sgn * hh;
                    if (!has[f]) up = (A.bc[f] == BC_INFLOW_ZERO && sgn * dflux_axis<FLUX>(fp, axis, um, xq, yq) < Real(0)) ? Real(0) : um;
                    if (need_lam) lam = fmax(lam, speed_norm<FLUX>(fp, um, xq, yq));
                    const Real H = llf<FLUX>(fp, axis, sgn, um, up, xq, yq) * T.w[q];
#pragma unroll
                    for (int t = 0; t < N1; ++t) hq[t] += T.B[q][t] * H;
                }
#pragma unroll
                for (int t = 0; t < N1; ++t)
#pragma unroll
                    for (int n = 0; n < N1; ++n) {
                        const int k = axis == 0 ? n + N1 * t : t + N1 * n;
                        const Real ps = (side || (n % 2 == 0)) ? Real(1) : Real(-1);
                        acc[k] -= ps * hq[t];
                    }
            }
        }
        if (weno && has[f]) {
            // Hermite candidate: neighbour polynomial continued into K_e.  The neighbour
            // on the minus side sits at xi + 2 in its own coordinate (shift table 0).
            Real cl[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = k % N1, j = k / N1;
                const int a = axis == 0 ? i : j;   // index along the shift axis
                Real s = Real(0);
#pragma unroll
                for (int m = 0; m < N1; ++m) {
                    if (m < a) continue;           // P_m(xi +- 2) has degree m
                    const int km = axis == 0 ? m + N1 * j : i + N1 * m;
                    s += T.T[side][a][m] * cn[km];
                }
                cl[k] = s;
            }
            const Real bl = qform<P>(T, cl);
            const Real dl = eps_w + bl;
            const Real wl = w_nbr / (dl * dl);
            wsum += wl;
#pragma unroll
            for (int k = 1; k < K; ++k) dacc[k] += wl * (c[k] - cl[k]);
        }
    }

    // ---------------- sensor value ----------------
    Real gamma = Real(0);
    if (MODE == 1 || A.stab == STAB_LO) gamma = Real(1);
    if (weno) {
        Real diff[K];
        diff[0] = Real(0);
        const Real inv = Real(1) / wsum;
#pragma unroll
        for (int k = 1; k < K; ++k) diff[k] = dacc[k] * inv;
        const double num2 = (double)qform<P>(T, diff);
        const double den2 = (double)beta0;
        const double num = sqrt(fmax(num2, 0.0));
        double g;
        if (num <= A.eps_s) {
            g = 0.0;
        } else if (den2 <= 0.0) {
            g = 1.0;
        } else {
            const double r = num / sqrt(den2);
            g = r < 1.0 ? r : 1.0;
            if (A.q != 1.0) g = pow(g, A.q);
            if (r < A.b) g = 0.0;
        }
        gamma = (Real)g;
        if (MODE == 1) {
            A.gamma_out[e] = g;
            return;
        }
    }
    if (MODE == 1) return;

    // ---------------- stabilization, M^{-1}, RK combination ----------------
    const Real lamv = A.lambda_nu > 0.0 ? (Real)A.lambda_nu : lam;
    const Real gs = gamma * lamv / Real(P);   // gamma nu (2/h)
    const Real two_h = Real(2) / h;
    const Real* __restrict__ Un = static_cast<const Real*>(A.Un);
    Real* __restrict__ Uo = static_cast<Real*>(A.Uout);
    const Real cnc = (Real)A.cn, ckc = (Real)A.ck, clc = (Real)A.cl;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int i = k % N1, j = k / N1;
        Real r = acc[k];
        if (A.stab != STAB_DG && gamma != Real(0)) {
            Real kc = Real(0);
            if (DIM == 1) {
#pragma unroll
                for (int m = 1; m < N1; ++m)
                    if (((i + m) & 1) == 0 && i > 0) kc += T.A1[i][m] * c[m];
            } else {
                Real s1 = Real(0), s2 = Real(0);
#pragma unroll
                for (int m = 1; m < N1; ++m) {
                    if (((i + m) & 1) == 0 && i > 0) s1 += T.A1[i][m] * c[m + N1 * j];
                    if (((j + m) & 1) == 0 && j > 0) s2 += T.A1[j][m] * c[i + N1 * m];
                }
                kc = s1 * T.A0[j] + T.A0[i] * s2;
            }
            r -= gs * kc;
        }
        Real mi = T.minv[i];
        if (DIM == 2) mi *= T.minv[j];
        const Real L = two_h * mi * r;
        Real out = clc * L + ckc * c[k];
        if (A.cn != 0.0) out += cnc * Un[k * E + e];
        bad |= !isfinite(out);
        Uo[k * E + e] = out;
    }
    if (bad) atomicOr(A.flag, 1u);
}

template <int P, int FLUX>
static cudaError_t launch_pf(const StageArgs& a, int mode, cudaStream_t s)
{
    const int threads = 128;
    const int64_t blocks = (a.E + threads - 1) / threads;
    if (blocks <= 0) return cudaSuccess;
    if (mode == 0) stage_kernel<P, FLUX, 0><<<(unsigned)blocks, threads, 0, s>>>(a);
    else stage_kernel<P, FLUX, 1><<<(unsigned)blocks, threads, 0, s>>>(a);
    return cudaGetLastError();
}

template <int P>
static cudaError_t launch_p(const StageArgs& a, int flux, int mode, cudaStream_t s)
{
    switch (flux) {
    case FLUX_ADVECT: return launch_pf<P, FLUX_ADVECT>(a, mode, s);
    case FLUX_ROTATION: return launch_pf<P, FLUX_ROTATION>(a, mode, s);
    case FLUX_BURGERS: return launch_pf<P, FLUX_BURGERS>(a, mode, s);
    case FLUX_KPP: return launch_pf<P, FLUX_KPP>(a, mode, s);
    default: return cudaErrorInvalidValue;
    }
}

static cudaError_t launch(const StageArgs& a, int p, int flux, int mode, cudaStream_t s)
{
    switch (p) {
    case 1: return launch_p<1>(a, flux, mode, s);
    case 2: return launch_p<2>(a, flux, mode, s);
    case 3: return launch_p<3>(a, flux, mode, s);
    default: return cudaErrorInvalidValue;
    }
}

static cudaError_t upload_tables(const HostTables& t)
{
    switch (t.p) {
    case 1: return upload<1>(t);
    case 2: return upload<2>(t);
    case 3: return upload<3>(t);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace DGW_NS
}  // namespace dgw
