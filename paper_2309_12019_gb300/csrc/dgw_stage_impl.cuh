// Stage kernel of the WENO-stabilized RKDG scheme, tiled.
//
// Included by one translation unit per (precision, dimension) with DGW_REAL, DGW_DIM
// and DGW_NS defined.  Each unit owns its copy of the constant-memory operator tables.
//
// One CTA owns a TX x TY tile of cells (one thread per cell).  It stages the tile's
// modal coefficients plus a one-cell face halo in shared memory, then
//   A. evaluates every face of the tile once: traces from both sides, the local
//      Lax-Friedrichs flux (Sec. 2) at the p+2 Gauss points, lifted onto the face
//      Legendre modes, into shared memory;
//   B. per cell: the WENO sensor from the four face neighbours in shared memory
//      (Sec. 4), the volume term (Eq. weak2) by sum factorisation, the face
//      contributions, the stabilization gamma nu K c (Sec. 3), M^{-1} and the
//      SSP-RK3 combination Uout = cn Un + ck Uk + cl L(Uk) (Eq. ssp).
// Constant factors are folded so that, in the reference element,
//   L_k = (2/h) minv(k) [acc_k - gamma lambda / p (K_ref c)_k].
#include <cmath>
#include <cstdint>

#include "dgw_internal.h"
#include "dgw_math.cuh"

namespace dgw {
namespace DGW_NS {

using Real = DGW_REAL;
constexpr int DIM = DGW_DIM;
constexpr bool kF32 = sizeof(Real) == 4;

// tile: 128 threads, one cell each
constexpr int TX = DIM == 1 ? 128 : 32;
constexpr int TY = DIM == 1 ? 1 : 4;
constexpr int NT = TX * TY;
constexpr int HX = TX + 2;                 // staged columns (one halo cell each side)
constexpr int HY = DIM == 1 ? 1 : TY + 2;  // staged rows
constexpr int OY = DIM == 1 ? 0 : 1;       // row offset of the tile inside the stage

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

// Scalars of one launch, converted once on the host to the kernel precision.
struct KParams {
    const Real* Uk;
    const Real* Un;
    Real* Uout;
    double* gamma_out;
    unsigned* flag;
    int64_t E;
    int nx, ny;
    int bc[4];
    int stab;
    int lam_fixed;       // lambda_e given (1) or max |F'| over the cell's Gauss points (0)
    int q_one;           // q == 1
    int has_un;
    Real x0, y0, h, hh, two_h;
    Real a0, a1, cx, cy, omega, lambda_nu;
    Real q, b, w_nbr, eps_w, eps_s;
    Real cn, ck, cl;
};

// ------------------------------------------------------------------------------------
// math helpers
// ------------------------------------------------------------------------------------
// sin and cos: float uses the reduced-argument hardware path (dgw_math.cuh), double
// the library routine.
__device__ __forceinline__ void sincos_r(float x, float* s, float* c) { fast_sincos(x, s, c); }
__device__ __forceinline__ void sincos_r(double x, double* s, double* c) { sincos(x, s, c); }

__device__ __forceinline__ float sqrt_r(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }

constexpr double kPi = 3.14159265358979323846;

// Flux F(u) at (x, y) and |F'(u)|_2 (1D: only the x component).
template <int FLUX>
__device__ __forceinline__ void vol_flux(const KParams& A, Real u, Real x, Real y, Real& fx, Real& fy,
                                         Real& spd)
{
    if (FLUX == FLUX_ADVECT) {
        fx = A.a0 * u; fy = A.a1 * u;
        spd = DIM == 1 ? fabs(A.a0) : sqrt_r(A.a0 * A.a0 + A.a1 * A.a1);
    } else if (FLUX == FLUX_ROTATION) {
        const Real vx = A.omega * (A.cy - y), vy = A.omega * (x - A.cx);
        fx = vx * u; fy = vy * u;
        spd = DIM == 1 ? fabs(vx) : sqrt_r(vx * vx + vy * vy);
    } else if (FLUX == FLUX_BURGERS) {
        const Real hu2 = Real(0.5) * u * u;
        fx = A.a0 * hu2; fy = A.a1 * hu2;
        spd = DIM == 1 ? fabs(A.a0 * u) : sqrt_r(A.a0 * A.a0 + A.a1 * A.a1) * fabs(u);
    } else {  // KPP: F = (sin u, cos u), |F'| = 1 in 2D
        Real s, c;
        sincos_r(u, &s, &c);
        fx = s; fy = c;
        spd = DIM == 1 ? fabs(c) : Real(1);
    }
}

template <int FLUX>
__device__ __forceinline__ Real speed_norm(const KParams& A, Real u, Real x, Real y)
{
    if (FLUX == FLUX_KPP && DIM == 2) return Real(1);
    Real fx, fy, spd;
    vol_flux<FLUX>(A, u, x, y, fx, fy, spd);
    return spd;
}

// F'(u) along the axis (inflow test of the ghost state).
template <int FLUX>
__device__ __forceinline__ Real dflux_axis(const KParams& A, int axis, Real u, Real x, Real y)
{
    if (FLUX == FLUX_ADVECT) return axis == 0 ? A.a0 : A.a1;
    if (FLUX == FLUX_ROTATION) return axis == 0 ? A.omega * (A.cy - y) : A.omega * (x - A.cx);
    if (FLUX == FLUX_BURGERS) return (axis == 0 ? A.a0 : A.a1) * u;
    Real s, c;
    sincos_r(u, &s, &c);
    return axis == 0 ? c : -s;
}

// Local Lax-Friedrichs flux for the normal +e_axis from uL (minus side) to uR, with the
// exact maximal wave speed over the segment between the two states (Sec. 2).
template <int FLUX>
__device__ __forceinline__ Real llf(const KParams& A, int axis, Real uL, Real uR, Real x, Real y)
{
    if (FLUX == FLUX_ADVECT || FLUX == FLUX_ROTATION) {
        const Real v = FLUX == FLUX_ADVECT ? (axis == 0 ? A.a0 : A.a1)
                                           : (axis == 0 ? A.omega * (A.cy - y) : A.omega * (x - A.cx));
        return Real(0.5) * v * (uL + uR) - Real(0.5) * fabs(v) * (uR - uL);
    } else if (FLUX == FLUX_BURGERS) {
        const Real an = axis == 0 ? A.a0 : A.a1;
        const Real s = fabs(an) * fmax(fabs(uL), fabs(uR));
        return Real(0.25) * an * (uL * uL + uR * uR) - Real(0.5) * s * (uR - uL);
    } else {
        // x-normal: n.F = sin u, |F'.n| = |cos u| (maximal at multiples of pi);
        // y-normal: n.F = cos u, |F'.n| = |sin u| (maximal at pi/2 + multiples of pi).
        Real sL, cL, sR, cR;
        sincos_r(uL, &sL, &cL);
        sincos_r(uR, &sR, &cR);
        const Real lo = fmin(uL, uR), hi = fmax(uL, uR);
        const Real shift = axis == 0 ? Real(0) : Real(0.5 * kPi);
        const Real k = ceil((lo - shift) * Real(1.0 / kPi));
        Real s;
        if (fma(k, Real(kPi), shift) <= hi) s = Real(1);
        else s = axis == 0 ? fmax(fabs(cL), fabs(cR)) : fmax(fabs(sL), fabs(sR));
        const Real fL = axis == 0 ? sL : cL, fR = axis == 0 ? sR : cR;
        return Real(0.5) * (fL + fR) - Real(0.5) * s * (uR - uL);
    }
}

// v^T G v over modes >= 1; G vanishes unless both Legendre degree pairs have even sums.
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
            if (((ia + ib) & 1) == 0 && ((ja + jb) & 1) == 0) t = fma(T.Gu[a][b], v[b], t);
        }
        s = fma(v[a], t, s);
    }
    return s;
}

__device__ __forceinline__ void atomic_max_nonneg(float* a, float v)
{
    atomicMax(reinterpret_cast<int*>(a), __float_as_int(v));
}
__device__ __forceinline__ void atomic_max_nonneg(double* a, double v)
{
    atomicMax(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}

// Column gx (row gy) of a cell or of a face neighbour, gx in [-1, nx]: itself inside
// the domain, the periodic image for gx = -1 or nx, and -1 otherwise (no neighbour
// there, or a column of a ragged tile beyond the neighbour of the last cell).
__device__ __forceinline__ int wrap_x(const KParams& A, int gx)
{
    if (gx >= 0 && gx < A.nx) return gx;
    if (A.bc[0] != BC_PERIODIC) return -1;
    if (gx == -1) return A.nx - 1;
    if (gx == A.nx) return 0;
    return -1;
}
__device__ __forceinline__ int wrap_y(const KParams& A, int gy)
{
    if (gy >= 0 && gy < A.ny) return gy;
    if (A.bc[2] != BC_PERIODIC) return -1;
    if (gy == -1) return A.ny - 1;
    if (gy == A.ny) return 0;
    return -1;
}

// MODE 0: stage / residual; MODE 1: sensor only.
template <int P, int FLUX, int MODE>
__global__ void __launch_bounds__(NT) stage_kernel(const KParams A)
{
    constexpr int N1 = P + 1, NQ = P + 2;
    constexpr int K = Tab<P>::K;
    constexpr int NFX = (TX + 1) * TY;                 // x-faces of the tile
    constexpr int NFY = DIM == 2 ? TX * (TY + 1) : 0;  // y-faces
    const Tab<P>& T = tab<P>();

    __shared__ Real su[K][HY][HX];
    __shared__ Real hfx[TY][TX + 1][DIM == 1 ? 1 : N1];
    __shared__ Real hfy[DIM == 2 ? TY + 1 : 1][TX][DIM == 2 ? N1 : 1];
    __shared__ Real lam_s[TY][TX];

    const int tid = threadIdx.x;
    const int tx0 = blockIdx.x * TX;
    const int ty0 = DIM == 2 ? blockIdx.y * TY : 0;
    const int64_t E = A.E;
    const bool need_lam = (MODE == 0) && (A.stab != STAB_DG) && !A.lam_fixed;

    // ---- stage the tile and its face halo (corners are not needed) ----
    for (int idx = tid; idx < K * HY * HX; idx += NT) {
        const int k = idx / (HY * HX);
        const int rem = idx - k * (HY * HX);
        const int r = rem / HX, cc = rem - r * HX;
        const bool corner = DIM == 2 && (r == 0 || r == HY - 1) && (cc == 0 || cc == HX - 1);
        if (corner) continue;
        const int gx = wrap_x(A, tx0 - 1 + cc);
        const int gy = DIM == 2 ? wrap_y(A, ty0 - OY + r) : 0;
        if (gx < 0 || gy < 0) continue;
        su[k][r][cc] = A.Uk[k * E + (int64_t)gy * A.nx + gx];
    }
    if (need_lam) lam_s[tid / TX][tid % TX] = Real(0);
    __syncthreads();

    // ---- A. faces: each face of the tile once ----
    if (MODE == 0) {
        for (int f = tid; f < NFX + NFY; f += NT) {
            const bool xf = f < NFX;
            int lx, ly;              // tile position of the cell on the plus side of the face
            if (xf) { ly = f / (TX + 1); lx = f - ly * (TX + 1); }
            else { const int g = f - NFX; ly = g / TX; lx = g - ly * TX; }
            const int gx = tx0 + lx, gy = ty0 + ly;   // plus-side cell (global, unwrapped)
            // the face lies at x = x0 + gx h (x-face) or y = y0 + gy h (y-face)
            if (xf) { if (gx > A.nx || gy >= A.ny) continue; }
            else { if (gy > A.ny || gx >= A.nx) continue; }
            const int axis = xf ? 0 : 1;
            const bool minus_in = xf ? (gx - 1 >= 0 || A.bc[0] == BC_PERIODIC)
                                     : (gy - 1 >= 0 || A.bc[2] == BC_PERIODIC);
            const bool plus_in = xf ? (gx < A.nx || A.bc[1] == BC_PERIODIC)
                                    : (gy < A.ny || A.bc[3] == BC_PERIODIC);
            // stage coordinates of the two cells
            const int pr = ly + OY, pc = lx + 1;
            const int mr = xf ? pr : pr - 1, mc = xf ? pc - 1 : pc;
            // trace coefficients along the face: minus cell at xi = +1, plus cell at xi = -1
            Real tm[N1], tp[N1];
#pragma unroll
            for (int t = 0; t < N1; ++t) {
                Real sm = Real(0), sp = Real(0);
#pragma unroll
                for (int n = 0; n < N1; ++n) {
                    const int k = DIM == 1 ? n : (xf ? n + N1 * t : t + N1 * n);
                    if (DIM == 1 && t > 0) break;
                    if (minus_in) sm += su[k][mr][mc];
                    if (plus_in) sp += ((n & 1) ? Real(-1) : Real(1)) * su[k][pr][pc];
                }
                tm[t] = sm;
                tp[t] = sp;
            }
            Real hq[N1];
#pragma unroll
            for (int t = 0; t < N1; ++t) hq[t] = Real(0);
            Real lm = Real(0), lp = Real(0);
            constexpr int NFQ = DIM == 1 ? 1 : NQ;
#pragma unroll
            for (int q = 0; q < NFQ; ++q) {
                Real uL = Real(0), uR = Real(0);
                if (DIM == 1) { uL = tm[0]; uR = tp[0]; }
                else {
#pragma unroll
                    for (int t = 0; t < N1; ++t) { uL = fma(tm[t], T.B[q][t], uL); uR = fma(tp[t], T.B[q][t], uR); }
                }
                Real x, y;
                if (xf) { x = A.x0 + Real(gx) * A.h; y = DIM == 2 ? A.y0 + (Real(gy) + Real(0.5)) * A.h + A.hh * T.g[q] : Real(0); }
                else { x = A.x0 + (Real(gx) + Real(0.5)) * A.h + A.hh * T.g[q]; y = A.y0 + Real(gy) * A.h; }
                if (!minus_in) {
                    // ghost for the plus cell, whose outward normal is -e_axis
                    const int side = xf ? 0 : 2;
                    uL = (A.bc[side] == BC_INFLOW_ZERO && -dflux_axis<FLUX>(A, axis, uR, x, y) < Real(0)) ? Real(0) : uR;
                } else if (!plus_in) {
                    const int side = xf ? 1 : 3;
                    uR = (A.bc[side] == BC_INFLOW_ZERO && dflux_axis<FLUX>(A, axis, uL, x, y) < Real(0)) ? Real(0) : uL;
                }
                if (need_lam) {
                    lm = fmax(lm, speed_norm<FLUX>(A, uL, x, y));
                    lp = fmax(lp, speed_norm<FLUX>(A, uR, x, y));
                }
                const Real H = llf<FLUX>(A, axis, uL, uR, x, y) * (DIM == 1 ? Real(1) : T.w[q]);
#pragma unroll
                for (int t = 0; t < N1; ++t) hq[t] = fma(DIM == 1 ? Real(1) : T.B[q][t], H, hq[t]);
            }
            if (xf) {
#pragma unroll
                for (int t = 0; t < (DIM == 1 ? 1 : N1); ++t) hfx[ly][lx][t] = hq[t];
            } else {
#pragma unroll
                for (int t = 0; t < N1; ++t) hfy[DIM == 2 ? ly : 0][lx][t] = hq[t];
            }
            if (need_lam) {
                // only the traces of cells of this tile that lie in the domain count
                const int mlx = xf ? lx - 1 : lx, mly = xf ? ly : ly - 1;
                if (minus_in && mlx >= 0 && mly >= 0 && (xf ? gx - 1 < A.nx : gy - 1 < A.ny))
                    atomic_max_nonneg(&lam_s[mly][mlx], lm);
                if (plus_in && lx < TX && ly < TY && gx < A.nx && gy < A.ny)
                    atomic_max_nonneg(&lam_s[ly][lx], lp);
            }
        }
        __syncthreads();
    }

    // ---- B. per cell ----
    const int lx = tid % TX, ly = tid / TX;
    const int gx = tx0 + lx, gy = ty0 + ly;
    if (gx >= A.nx || (DIM == 2 && gy >= A.ny)) return;
    const int64_t e = (int64_t)gy * A.nx + gx;
    const int sr = ly + OY, sc = lx + 1;

    Real c[K];
#pragma unroll
    for (int k = 0; k < K; ++k) c[k] = su[k][sr][sc];

    // sensor (Sec. 4): Hermite candidates of the face neighbours, nonlinear weights
    Real gamma = (MODE == 0 && A.stab == STAB_LO) ? Real(1) : Real(0);
    if (MODE == 1 || A.stab == STAB_WENO) {
        bool has[2 * DIM];
        int me = 0;
#pragma unroll
        for (int f = 0; f < 2 * DIM; ++f) {
            const int nx_ = gx + (f == 0 ? -1 : (f == 1 ? 1 : 0));
            const int ny_ = gy + (f == 2 ? -1 : (f == 3 ? 1 : 0));
            has[f] = (f < 2) ? (wrap_x(A, nx_) >= 0) : (wrap_y(A, ny_) >= 0);
            me += has[f] ? 1 : 0;
        }
        const Real beta0 = qform<P>(T, c);
        const Real d0 = A.eps_w + beta0;
        Real wsum = (Real(1) - Real(me) * A.w_nbr) / (d0 * d0);
        Real dacc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) dacc[k] = Real(0);
#pragma unroll
        for (int f = 0; f < 2 * DIM; ++f) {
            if (!has[f]) continue;
            const int axis = f >> 1, side = f & 1;
            const int nr = sr + (f == 2 ? -1 : (f == 3 ? 1 : 0));
            const int nc = sc + (f == 0 ? -1 : (f == 1 ? 1 : 0));
            Real cl[K];
#pragma unroll
            for (int k = 1; k < K; ++k) {
                const int i = k % N1, j = k / N1;
                const int a = axis == 0 ? i : j;
                Real s = Real(0);
#pragma unroll
                for (int m = 0; m < N1; ++m) {
                    if (m < a) continue;   // P_m(xi +- 2) has degree m
                    const int km = axis == 0 ? m + N1 * j : i + N1 * m;
                    s = fma(T.T[side][a][m], su[km][nr][nc], s);
                }
                cl[k] = s;
            }
            cl[0] = Real(0);
            const Real dl = A.eps_w + qform<P>(T, cl);
            const Real wl = A.w_nbr / (dl * dl);
            wsum += wl;
#pragma unroll
            for (int k = 1; k < K; ++k) dacc[k] = fma(wl, c[k] - cl[k], dacc[k]);
        }
        // U - U* = sum_l w_l (c - c_l)
        const Real inv = Real(1) / wsum;
#pragma unroll
        for (int k = 1; k < K; ++k) dacc[k] *= inv;
        dacc[0] = Real(0);
        const Real num = sqrt_r(fmax(qform<P>(T, dacc), Real(0)));
        if (num <= A.eps_s) {
            gamma = Real(0);
        } else if (beta0 <= Real(0)) {
            gamma = Real(1);
        } else {
            const Real r = num / sqrt_r(beta0);
            gamma = r < Real(1) ? r : Real(1);
            if (!A.q_one) gamma = pow(gamma, A.q);
            if (r < A.b) gamma = Real(0);
        }
        if (MODE == 1) {
            A.gamma_out[e] = (double)gamma;
            return;
        }
    }
    if (MODE == 1) return;

    // volume term (Eq. weak2), sum-factorised: acc_ij = sum_q W_q [D_i B_j Fx + B_i D_j Fy]
    Real acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = Real(0);
    Real lam = need_lam ? lam_s[ly][lx] : Real(0);
    const Real xc = A.x0 + (Real(gx) + Real(0.5)) * A.h;
    const Real yc = DIM == 2 ? A.y0 + (Real(gy) + Real(0.5)) * A.h : Real(0);
    if (DIM == 1) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            Real u = Real(0);
#pragma unroll
            for (int i = 0; i < N1; ++i) u = fma(c[i], T.B[q][i], u);
            Real fx, fy, spd;
            vol_flux<FLUX>(A, u, xc + A.hh * T.g[q], Real(0), fx, fy, spd);
            lam = fmax(lam, spd);
            const Real wf = T.w[q] * fx;
#pragma unroll
            for (int i = 0; i < N1; ++i) acc[i] = fma(T.D[q][i], wf, acc[i]);
        }
    } else {
        Real tmp[N1][NQ];
#pragma unroll
        for (int j = 0; j < N1; ++j)
#pragma unroll
            for (int qx = 0; qx < NQ; ++qx) {
                Real s = Real(0);
#pragma unroll
                for (int i = 0; i < N1; ++i) s = fma(c[i + N1 * j], T.B[qx][i], s);
                tmp[j][qx] = s;
            }
#pragma unroll
        for (int qy = 0; qy < NQ; ++qy) {
            const Real y = yc + A.hh * T.g[qy];
            Real px[N1], py[N1];
#pragma unroll
            for (int i = 0; i < N1; ++i) { px[i] = Real(0); py[i] = Real(0); }
#pragma unroll
            for (int qx = 0; qx < NQ; ++qx) {
                Real u = Real(0);
#pragma unroll
                for (int j = 0; j < N1; ++j) u = fma(tmp[j][qx], T.B[qy][j], u);
                Real fx, fy, spd;
                vol_flux<FLUX>(A, u, xc + A.hh * T.g[qx], y, fx, fy, spd);
                lam = fmax(lam, spd);
                const Real wfx = T.w[qx] * fx, wfy = T.w[qx] * fy;
#pragma unroll
                for (int i = 0; i < N1; ++i) {
                    px[i] = fma(T.D[qx][i], wfx, px[i]);
                    py[i] = fma(T.B[qx][i], wfy, py[i]);
                }
            }
#pragma unroll
            for (int j = 0; j < N1; ++j) {
                const Real bj = T.w[qy] * T.B[qy][j], dj = T.w[qy] * T.D[qy][j];
#pragma unroll
                for (int i = 0; i < N1; ++i) acc[i + N1 * j] = fma(bj, px[i], fma(dj, py[i], acc[i + N1 * j]));
            }
        }
    }

    // faces: -phi_k(+1) H on the plus faces, +phi_k(-1) H on the minus faces
    if (DIM == 1) {
        const Real hm = hfx[0][lx][0], hp = hfx[0][lx + 1][0];
#pragma unroll
        for (int n = 0; n < N1; ++n) acc[n] += ((n & 1) ? -hm : hm) - hp;
    } else {
#pragma unroll
        for (int t = 0; t < N1; ++t) {
            const Real xm = hfx[ly][lx][t], xp = hfx[ly][lx + 1][t];
            const Real ym = hfy[ly][lx][t], yp = hfy[ly + 1][lx][t];
#pragma unroll
            for (int n = 0; n < N1; ++n) {
                acc[n + N1 * t] += ((n & 1) ? -xm : xm) - xp;
                acc[t + N1 * n] += ((n & 1) ? -ym : ym) - yp;
            }
        }
    }

    // stabilization (Sec. 3), M^{-1}, RK combination (Eq. ssp)
    const Real lamv = A.lam_fixed ? A.lambda_nu : lam;
    const Real gs = gamma * lamv / Real(P);   // gamma nu (2/h)
    bool bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int i = k % N1, j = k / N1;
        Real r = acc[k];
        if (gamma != Real(0)) {
            Real kc = Real(0);
            if (DIM == 1) {
#pragma unroll
                for (int m = 1; m < N1; ++m)
                    if (((i + m) & 1) == 0 && i > 0) kc = fma(T.A1[i][m], c[m], kc);
            } else {
                Real s1 = Real(0), s2 = Real(0);
#pragma unroll
                for (int m = 1; m < N1; ++m) {
                    if (((i + m) & 1) == 0 && i > 0) s1 = fma(T.A1[i][m], c[m + N1 * j], s1);
                    if (((j + m) & 1) == 0 && j > 0) s2 = fma(T.A1[j][m], c[i + N1 * m], s2);
                }
                kc = s1 * T.A0[j] + T.A0[i] * s2;
            }
            r -= gs * kc;
        }
        Real mi = T.minv[i];
        if (DIM == 2) mi *= T.minv[j];
        const Real L = A.two_h * mi * r;
        Real out = A.cl * L + A.ck * c[k];
        if (A.has_un) out += A.cn * A.Un[k * E + e];
        bad |= !isfinite(out);
        A.Uout[k * E + e] = out;
    }
    if (bad) atomicOr(A.flag, 1u);
}

static KParams make_params(const StageArgs& s)
{
    KParams a;
    a.Uk = static_cast<const Real*>(s.Uk);
    a.Un = static_cast<const Real*>(s.Un);
    a.Uout = static_cast<Real*>(s.Uout);
    a.gamma_out = s.gamma_out;
    a.flag = s.flag;
    a.E = s.E;
    a.nx = s.nx;
    a.ny = s.ny;
    for (int f = 0; f < 4; ++f) a.bc[f] = s.bc[f];
    a.stab = s.stab;
    a.lam_fixed = s.lambda_nu > 0.0;
    a.q_one = s.q == 1.0;
    a.has_un = s.cn != 0.0 && s.Un != nullptr;
    a.x0 = (Real)s.x0; a.y0 = (Real)s.y0; a.h = (Real)s.h; a.hh = (Real)(0.5 * s.h);
    a.two_h = (Real)(2.0 / s.h);
    a.a0 = (Real)s.a0; a.a1 = (Real)s.a1; a.cx = (Real)s.cx; a.cy = (Real)s.cy;
    a.omega = (Real)s.omega; a.lambda_nu = (Real)s.lambda_nu;
    a.q = (Real)s.q; a.b = (Real)s.b; a.w_nbr = (Real)s.w_nbr; a.eps_w = (Real)s.eps_w;
    a.eps_s = (Real)s.eps_s;
    a.cn = (Real)s.cn; a.ck = (Real)s.ck; a.cl = (Real)s.cl;
    return a;
}

template <int P, int FLUX>
static cudaError_t launch_pf(const StageArgs& s, int mode, cudaStream_t st)
{
    const KParams a = make_params(s);
    dim3 grid((s.nx + TX - 1) / TX, DIM == 2 ? (s.ny + TY - 1) / TY : 1);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    if (mode == 0) stage_kernel<P, FLUX, 0><<<grid, NT, 0, st>>>(a);
    else stage_kernel<P, FLUX, 1><<<grid, NT, 0, st>>>(a);
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
