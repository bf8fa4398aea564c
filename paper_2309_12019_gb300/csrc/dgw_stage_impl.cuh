// Stage kernel of the WENO-stabilized RKDG scheme, tiled.
//
// Included by one translation unit per (precision, dimension) with DGW_REAL, DGW_DIM
// and DGW_NS defined.  Each unit owns its copy of the constant-memory operator tables.
//
// One CTA of TX x TYT threads owns a tile of TX x (TYT L) cells: a thread advances L
// cells stacked in y, L = 2 in the float 2D stage kernel (the two cells' arithmetic
// issued as packed FP32 pairs), else 1.
//   0. It stages the modal coefficients of the tile plus a one-cell face halo in shared
//      memory: one TMA box load (2D, 16-byte aligned strides) waited on through an
//      mbarrier with a bounded spin, else cooperative coalesced loads; periodic halo
//      cells of boundary tiles are then filled from the wrapped side.
//   1. Per cell: the traces of its polynomial on its faces (shared memory), the WENO
//      sensor from the four face neighbours (Sec. 4), the volume term (Eq. weak2) by
//      sum factorisation, kept in registers.
//   2. Every face of the tile once: both traces at the p+2 Gauss points, the local
//      Lax-Friedrichs flux (Sec. 2), lifted onto the face Legendre modes, written over
//      the face's minus-side trace.
//   3. Per cell: face contributions, the stabilization gamma nu K c (Sec. 3), M^{-1}
//      and the SSP-RK3 combination Uout = cn Un + ck Uk + cl L(Uk) (Eq. ssp).
// Constant factors are folded so that, in the reference element,
//   L_k = (2/h) minv(k) [acc_k - gamma lambda / p (K_ref c)_k].
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "dgw_internal.h"
#include "dgw_math.cuh"

// The sensor-only instantiations of process_tile (MODE == 1) return before the volume
// phase, and the front end reports the rest of their body as unreachable.
#pragma nv_diag_suppress 128

namespace dgw {
namespace DGW_NS {

using Real = DGW_REAL;
constexpr int DIM = DGW_DIM;
constexpr bool kF32 = sizeof(Real) == 4;

// tiles: TX threads wide; the batch kernel runs TY thread rows of one cell each (NT
// threads), the stage kernel TYS rows of LS cells each (NTS threads)
constexpr int TX = DIM == 1 ? 128 : kTileX2;
constexpr int TY = DIM == 1 ? 1 : kTileY2;
constexpr int NT = TX * TY;
constexpr int TYS = DIM == 1 ? 1 : stage_thread_rows(!kF32);
constexpr int NTS = TX * TYS;
constexpr int HX = TX + 8;                 // staged columns: tile at [OX, OX+TX), halo OX-1, OX+TX
constexpr int OX = 4;
constexpr int OY = DIM == 1 ? 0 : 1;       // row offset of the tile inside the stage
constexpr int LS = DIM == 2 ? stage_lanes(!kF32) : 1;
static_assert(DIM == 1 || (HX == kBoxX2 && TYS * LS == stage_rows(!kF32)), "TMA box and stage layout disagree");

template <int P>
struct Tab {
    static constexpr int N1 = P + 1, NQ = P + 2, K = (DIM == 1) ? N1 : N1 * N1;
    Real g[NQ], w[NQ];
    Real B[NQ][N1];      // P_i(g_q)
    Real D[NQ][N1];      // P_i'(g_q)
    Real WB[NQ][N1];     // w_q P_i(g_q)
    Real WD[NQ][N1];     // w_q P_i'(g_q)
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
        for (int i = 0; i < N1; ++i) {
            t.B[q][i] = (Real)h.B[q][i];
            t.D[q][i] = (Real)h.D[q][i];
            t.WB[q][i] = (Real)(h.w[q] * h.B[q][i]);
            t.WD[q][i] = (Real)(h.w[q] * h.D[q][i]);
        }
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
    CUtensorMap tmap;    // TMA descriptor of Uk (valid when use_tma)
    CUtensorMap tmap_un; // TMA descriptor of Un, tile box (valid when use_tma_un)
    CUtensorMap tmap_p;  // persistent kernel: Uk box of kPRows + 2 rows, Un box of kPRows rows
    CUtensorMap tmap_un_p;
    int use_tma;
    int use_tma_un;
    int use_p_un;        // the persistent kernel stages Un (tmap_un_p valid)
    int cg_loads;        // load Uk / Un through L2 only (data written earlier in the same launch)
    int wait_limit;      // polls of a TMA mbarrier wait before it gives up (kWaitLimit)
    int tile_row0;       // first tile row of a stage launch over a band of rows
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
    Real theta;          // exponent of the Zhao et al. sensor (stab == STAB_ZHAO)
    int theta_one;       // theta == 1
    Real gam, gm1;       // Euler system: gamma and gamma - 1
    Real cn, ck, cl;
    // prescribed-state sides (2D Euler): the stage's time is *t_dev + t_off
    const double* t_dev;
    double t_off;
    Real bstate[2][4];
    Real bsplit[4], bspeed[4];
    int bbelow[4], babove[4];
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

// a / b for the sensor weights: the hardware reciprocal in float (at most 2 ulp; the
// divisors here lie in [1e-12, 1e30]), the correctly rounded quotient in double.
__device__ __forceinline__ float div_w(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double div_w(double a, double b) { return a / b; }

constexpr double kPi = 3.14159265358979323846;

// Products and sums rounded one way in every kernel that inlines them (intrinsics are not
// contracted into FMAs by the compiler): the positions and velocities of the
// position-dependent flux, so that the tile and persistent kernels round them alike.
__device__ __forceinline__ float mul_x(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_x(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_x(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_x(double a, double b, double c) { return __fma_rn(a, b, c); }

// Flux F(u) at (x, y) and |F'(u)|_2 (1D: only the x component).
template <int FLUX>
__device__ __forceinline__ void vol_flux(const KParams& A, Real u, Real x, Real y, Real& fx, Real& fy,
                                         Real& spd)
{
    if (FLUX == FLUX_ADVECT) {
        fx = mul_x(A.a0, u); fy = mul_x(A.a1, u);
        spd = DIM == 1 ? fabs(A.a0) : sqrt_r(fma_x(A.a0, A.a0, mul_x(A.a1, A.a1)));
    } else if (FLUX == FLUX_ROTATION) {
        const Real vx = mul_x(A.omega, A.cy - y), vy = mul_x(A.omega, x - A.cx);
        fx = mul_x(vx, u); fy = mul_x(vy, u);
        spd = DIM == 1 ? fabs(vx) : sqrt_r(fma_x(vx, vx, mul_x(vy, vy)));
    } else if (FLUX == FLUX_BURGERS) {
        const Real hu2 = mul_x(mul_x(Real(0.5), u), u);
        fx = mul_x(A.a0, hu2); fy = mul_x(A.a1, hu2);
        spd = DIM == 1 ? fabs(mul_x(A.a0, u)) : mul_x(sqrt_r(fma_x(A.a0, A.a0, mul_x(A.a1, A.a1))), fabs(u));
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

// ------------------------------------------------------------------------------------
// Cells per thread.  With L = 2 (float, 2D) a thread advances two cells stacked in y and
// each arithmetic step of the pair is one packed FP32 instruction (FFMA2 / FMUL2 / FADD2,
// sm_100 and later): V = float2, lane l holding cell l.  L = 1 is plain scalar code.
// ------------------------------------------------------------------------------------
template <int L> struct VecOf { using type = Real; };
template <> struct VecOf<2> { using type = float2; };

__device__ __forceinline__ Real& lane(Real& v, int) { return v; }
__device__ __forceinline__ Real lane(const Real& v, int) { return v; }
__device__ __forceinline__ float& lane(float2& v, int l) { return l ? v.y : v.x; }
__device__ __forceinline__ float lane(const float2& v, int l) { return l ? v.y : v.x; }

template <class V> __device__ __forceinline__ V vbc(Real s) { return s; }
template <> __device__ __forceinline__ float2 vbc<float2>(Real s) { return make_float2((float)s, (float)s); }

__device__ __forceinline__ Real vfma(Real a, Real b, Real c) { return fma(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vfma(float a, float2 b, float2 c) { return __ffma2_rn(make_float2(a, a), b, c); }
__device__ __forceinline__ Real vmul(Real a, Real b) { return a * b; }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vmul(float a, float2 b) { return __fmul2_rn(make_float2(a, a), b); }
__device__ __forceinline__ Real vadd(Real a, Real b) { return a + b; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ Real vsub(Real a, Real b) { return a - b; }
// a - b as one fused step: b * (-1) + a rounds once, exactly like the subtraction
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ Real vmax(Real a, Real b) { return fmax(a, b); }
__device__ __forceinline__ float2 vmax(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }

template <class V> struct Lanes { static constexpr int n = 1; };
template <> struct Lanes<float2> { static constexpr int n = 2; };

// Pairs of doubles (the Euler kernels keep two state components per pair, a float2 in
// the float kernels): the same helpers, one lane at a time.
__device__ __forceinline__ double& lane(double2& v, int l) { return l ? v.y : v.x; }
__device__ __forceinline__ double lane(const double2& v, int l) { return l ? v.y : v.x; }
template <> __device__ __forceinline__ double2 vbc<double2>(Real s) { return make_double2((double)s, (double)s); }
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) { return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y)); }
__device__ __forceinline__ double2 vfma(double a, double2 b, double2 c) { return make_double2(fma(a, b.x, c.x), fma(a, b.y, c.y)); }
__device__ __forceinline__ double2 vmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 vmul(double a, double2 b) { return make_double2(a * b.x, a * b.y); }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 vsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
template <> struct Lanes<double2> { static constexpr int n = 2; };

// sin and cos of every lane: float pairs reduce their arguments on the packed pipe
__device__ __forceinline__ void sincos_v(Real x, Real& s, Real& c) { sincos_r(x, &s, &c); }
__device__ __forceinline__ void sincos_v(float2 x, float2& s, float2& c) { fast_sincos2(x, &s, &c); }

template <int FLUX, class V>
__device__ __forceinline__ void vol_flux_v(const KParams& A, V u, Real x, V y, V& fx, V& fy, V& spd)
{
    if constexpr (FLUX == FLUX_KPP) {
        sincos_v(u, fx, fy);
#pragma unroll
        for (int l = 0; l < Lanes<V>::n; ++l) lane(spd, l) = DIM == 1 ? fabs(lane(fy, l)) : Real(1);
    } else {
#pragma unroll
        for (int l = 0; l < Lanes<V>::n; ++l) vol_flux<FLUX>(A, lane(u, l), x, lane(y, l), lane(fx, l), lane(fy, l), lane(spd, l));
    }
}

// ------------------------------------------------------------------------------------
// Quadrature on the symmetric Gauss nodes (g_{NQ-1-q} = -g_q, g = 0 at the centre of an
// odd rule).  P_i has the parity of i and P_i' the opposite one, so only the table rows
// of the positive nodes are used: u(+-g) = E(g) +- O(g) from the even and odd parts of
// the expansion, and a weighted sum over the nodes takes f(+g) + f(-g) or f(+g) - f(-g)
// per pair.  Terms that vanish by parity (P_odd(0), P_even'(0), P_0' = 0) and the
// factor P_0 = 1 are left out.
// ------------------------------------------------------------------------------------
// u[q] = sum_i r[i] P_i(g_q), q = 0 .. NQ-1 (nodes ascending)
template <int N1, int NQ, class V>
__device__ __forceinline__ void interp_sym(const Real (&B)[NQ][N1], const V (&r)[N1], V (&u)[NQ])
{
#pragma unroll
    for (int m = 0; m < NQ / 2; ++m) {
        const int qp = NQ - 1 - m;
        V e = r[0], o = vmul(B[qp][1], r[1]);
#pragma unroll
        for (int i = 2; i < N1; ++i) {
            if (i & 1) o = vfma(B[qp][i], r[i], o);
            else e = vfma(B[qp][i], r[i], e);
        }
        u[qp] = vadd(e, o);
        u[m] = vsub(e, o);
    }
    if constexpr ((NQ & 1) != 0) {
        constexpr int qc = NQ / 2;
        V e = r[0];
#pragma unroll
        for (int i = 2; i < N1; i += 2) e = vfma(B[qc][i], r[i], e);
        u[qc] = e;
    }
}

// out[i] = sum_q W[q][i] f[q] for a table W[q][i] = w_q P_i(g_q) (DERIV false) or
// w_q P_i'(g_q) (DERIV true; out[0] = 0 is then not written: callers skip it)
template <bool DERIV, int N1, int NQ, class V>
__device__ __forceinline__ void project_sym(const Real (&W)[NQ][N1], const V (&f)[NQ], V (&out)[N1])
{
    constexpr int NP = NQ / 2;
    V S[NP > 0 ? NP : 1], D[NP > 0 ? NP : 1];
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        S[m] = vadd(f[NQ - 1 - m], f[m]);
        D[m] = vsub(f[NQ - 1 - m], f[m]);
    }
#pragma unroll
    for (int i = DERIV ? 1 : 0; i < N1; ++i) {
        const bool even_fn = DERIV ? (i & 1) != 0 : (i & 1) == 0;   // parity of the table row
        V a;
        if ((NQ & 1) != 0 && even_fn) a = vmul(W[NQ / 2][i], f[NQ / 2]);
        else a = vmul(W[NQ - 1][i], even_fn ? S[0] : D[0]);
#pragma unroll
        for (int m = ((NQ & 1) != 0 && even_fn) ? 0 : 1; m < NP; ++m)
            a = vfma(W[NQ - 1 - m][i], even_fn ? S[m] : D[m], a);
        out[i] = a;
    }
}

// Local Lax-Friedrichs flux of the KPP problem (Sec. 5, F = (sin u, cos u)) across a face
// of normal +e_x, the states given as u' = u + sh: an x-face takes sh = 0
// (n.F = sin u, |F'.n| = |cos u|), a y-face sh = pi/2 (n.F = cos u = sin(u + pi/2),
// |F'.n| = |sin u| = |cos(u + pi/2)|), so that one body serves both orientations.  The
// wave speed is exact: 1 if [min, max] of the two states holds a multiple of pi (a
// maximiser of |cos|), else the larger end value.  The segment holds a multiple of pi
// exactly when it is at least pi long or sin changes sign over it (sin vanishes only
// there, and a shorter segment holds at most one zero); near a zero, where the computed
// sign of sin may err, both answers are 1 to within the square of the distance.
template <class V>
__device__ __forceinline__ V llf_kpp(V uL, V uR)
{
    V sL, cL, sR, cR;
    sincos_v(uL, sL, cL);
    sincos_v(uR, sR, cR);
    const V d = vsub(uR, uL), ss = vmul(sL, sR);
    V spd;
#pragma unroll
    for (int l = 0; l < Lanes<V>::n; ++l)
        lane(spd, l) = (lane(ss, l) <= Real(0) || fabs(lane(d, l)) >= Real(kPi))
                           ? Real(1) : fmax(fabs(lane(cL, l)), fabs(lane(cR, l)));
    // H = (sin uL' + sin uR') / 2 - s+ (uR' - uL') / 2
    return vfma(vmul(Real(-0.5), spd), d, vmul(Real(0.5), vadd(sL, sR)));
}

// F'(u) along the axis (inflow test of the ghost state).
template <int FLUX>
__device__ __forceinline__ Real dflux_axis(const KParams& A, int axis, Real u, Real x, Real y)
{
    if (FLUX == FLUX_ADVECT) return axis == 0 ? A.a0 : A.a1;
    if (FLUX == FLUX_ROTATION) return axis == 0 ? mul_x(A.omega, A.cy - y) : mul_x(A.omega, x - A.cx);
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
    // (products and sums in a fixed order: the tile and persistent kernels round alike)
    if (FLUX == FLUX_ADVECT || FLUX == FLUX_ROTATION) {
        const Real v = FLUX == FLUX_ADVECT ? (axis == 0 ? A.a0 : A.a1)
                                           : (axis == 0 ? mul_x(A.omega, A.cy - y) : mul_x(A.omega, x - A.cx));
        return fma_x(mul_x(Real(-0.5), fabs(v)), uR - uL, mul_x(mul_x(Real(0.5), v), uL + uR));
    } else if (FLUX == FLUX_BURGERS) {
        const Real an = axis == 0 ? A.a0 : A.a1;
        const Real s = mul_x(fabs(an), fmax(fabs(uL), fabs(uR)));
        return fma_x(mul_x(Real(-0.5), s), uR - uL, mul_x(mul_x(Real(0.25), an), fma_x(uL, uL, mul_x(uR, uR))));
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

// x^theta of the Zhao et al. sensor (theta = 1 in the paper)
template <class KP>
__device__ __forceinline__ Real zpow(const KP& A, Real x) { return A.theta_one ? x : pow(x, A.theta); }

// v^T G v over modes >= 1; G vanishes unless both Legendre degree pairs have even sums,
// so it splits into the four parity classes of (i, j), summed in independent chains.
template <int P, class V>
__device__ __forceinline__ V qform(const Tab<P>& T, const V* v)
{
    constexpr int N1 = P + 1, K = Tab<P>::K;
    V s[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) s[c] = vbc<V>(0);
#pragma unroll
    for (int a = 1; a < K; ++a) {
        V t = vbc<V>(0);
#pragma unroll
        for (int b = a; b < K; ++b) {
            const int ia = a % N1, ja = a / N1, ib = b % N1, jb = b / N1;
            if (((ia + ib) & 1) == 0 && ((ja + jb) & 1) == 0) t = vfma(T.Gu[a][b], v[b], t);
        }
        const int cls = ((a % N1) & 1) + 2 * ((a / N1) & 1);
        s[cls] = vfma(v[a], t, s[cls]);
    }
    return vadd(vadd(s[0], s[1]), vadd(s[2], s[3]));
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

// Bounded wait for the completion of the given phase parity of an mbarrier; false if
// it gave up after `limit` polls.
constexpr int kWaitLimit = 1 << 22;
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit = kWaitLimit)
{
    for (int it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

// Asynchronous copy of one word from global to shared memory (cp.async, cached at all
// levels; 4-byte words may start anywhere a float does, which the bulk copies do not
// allow).  The batch kernel's copies follow the acquire of its dependency counter.
__device__ __forceinline__ void cp_async_word(Real* dst, const Real* src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(Real) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Shared memory of one tile of TX x (TYT * L) cells (carved from dynamic shared memory).
template <int P, int L, int TYT>
struct TileSmem {
    static constexpr int N1 = P + 1, K = Tab<P>::K, TN = DIM == 1 ? 1 : N1;
    static constexpr int TYC = TYT * L;                   // cell rows
    static constexpr int HYC = DIM == 1 ? 1 : TYC + 2;    // staged rows
    using Stage = Real[K][HYC][HX];
    alignas(128) Stage su;
    // cell index innermost: a warp touches consecutive words (no bank conflicts).
    // The face phase overwrites the minus-side trace of every face with the face's
    // lifted flux: trx[r][1][t][c] becomes the flux of x-face c of row r (between cells
    // c - 1 and c), trys[r][1][t][c] that of y-face r of column c.  Each such slot is
    // read by its own face only, before the write.
    Real trx[TYC][2][TN][TX + 2];                         // x-traces, col = lx + 1
    Real trys[DIM == 2 ? TYC + 2 : 1][2][TN][TX];         // y-traces, row = cell row + 1
    Real lam_s[TYC][TX];
    alignas(8) uint64_t mbar;
    alignas(8) uint64_t mbar_un;   // persistent kernel: the Un box
    int fail_s;
};

// Pipelined staging of the batch kernel (cp.async, one commit group per call; the
// caller waits with cp_async_wait_all and a CTA barrier).  stage_tile_async: the tile's
// cells and their face halo of Uk into su, as the plain staging of process_tile lays
// them out (zeros where there is no cell).  stage_un_async: the tile's own cells of Un
// into su, laid out [K][TYC][TX] (zeros outside the mesh).
template <int P, int L, int TYT>
__device__ __forceinline__ void stage_tile_async(const KParams& A, const int tx0, const int ty0,
                                                 typename TileSmem<P, L, TYT>::Stage& su)
{
    constexpr int K = Tab<P>::K, NT = TX * TYT, HYC = TileSmem<P, L, TYT>::HYC;
    const int64_t E = A.E;
    for (int idx = threadIdx.x; idx < HYC * HX; idx += NT) {
        const int r = idx / HX, cc = idx - r * HX;
        if (cc < OX - 1 || cc > OX + TX) continue;
        const bool corner = DIM == 2 && (r == 0 || r == HYC - 1) && (cc == OX - 1 || cc == OX + TX);
        if (corner) continue;
        const int gx = wrap_x(A, tx0 - OX + cc);
        const int gy = DIM == 2 ? wrap_y(A, ty0 - OY + r) : 0;
        if (gx < 0 || gy < 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) su[k][r][cc] = Real(0);
            continue;
        }
        const Real* src = A.Uk + (int64_t)gy * A.nx + gx;
#pragma unroll
        for (int k = 0; k < K; ++k) cp_async_word(&su[k][r][cc], src + k * E);
    }
    cp_async_commit();
}

template <int P, int L, int TYT>
__device__ __forceinline__ void stage_un_async(const KParams& A, const int tx0, const int ty0,
                                               typename TileSmem<P, L, TYT>::Stage& su)
{
    constexpr int K = Tab<P>::K, NT = TX * TYT, TYC = TileSmem<P, L, TYT>::TYC;
    static_assert(TYC * TX <= TileSmem<P, L, TYT>::HYC * HX, "Un tile exceeds the stage buffer");
    const int64_t E = A.E;
    Real* sun = &su[0][0][0];
    for (int idx = threadIdx.x; idx < TYC * TX; idx += NT) {
        const int r = idx / TX, c = idx - r * TX;
        const int gx = tx0 + c, gy = ty0 + r;
        if (gx >= A.nx || (DIM == 2 && gy >= A.ny)) {
#pragma unroll
            for (int k = 0; k < K; ++k) sun[(k * TYC + r) * TX + c] = Real(0);
            continue;
        }
        const Real* src = A.Un + (int64_t)(DIM == 2 ? gy : 0) * A.nx + gx;
#pragma unroll
        for (int k = 0; k < K; ++k) cp_async_word(&sun[(k * TYC + r) * TX + c], src + k * E);
    }
    cp_async_commit();
}

// One tile of one stage.  Called by all TX x TYT threads of a CTA together (it contains
// CTA barriers); tx0, ty0: first cell of the tile.  MODE 0: stage / residual;
// MODE 1: sensor only.  Thread (lx, ly) owns the cells (lx, L ly + l), l < L; with
// L = 2 their arithmetic runs as packed pairs (lane l = cell l).  Lanes of cells outside
// the mesh (ragged tiles) compute on zero-filled data and store nothing.
// TMA: the TMA staging paths are compiled in (the batch kernel builds its launch scalars
// per work item in registers and never stages by TMA; taking the tensor map's address
// would put those scalars in local memory).
// PIPE 0: the tile stages itself (TMA box, or plain loads).
// PIPE 1 (batch kernel): the caller has staged the tile into *su_async with
// stage_tile_async and made it visible (wait and barrier); the Un tile is copied into
// the same buffer once the volume phase is done, and every copy still in flight (the
// caller's prefetch of its next tile too) is waited for before the face-lifting phase.
// PIPE 2 (persistent kernel): the caller has waited for the tile's box in S.su; once the
// volume phase is done the box of the next tile (origin nxt_x, nxt_y; nxt_x < 0: none) is
// requested into S.su on S.mbar, and Un, requested by the caller into un_p on S.mbar_un,
// is waited for (phase parity un_parity) before the Runge-Kutta combination.
template <int P, int FLUX, int MODE, int L, int TYT, bool TMA = true, int PIPE = 0>
__device__ __forceinline__ void process_tile(const KParams& A, const int tx0, const int ty0, TileSmem<P, L, TYT>& S,
                                             typename TileSmem<P, L, TYT>::Stage* su_async = nullptr,
                                             const int nxt_x = -1, const int nxt_y = 0, const Real* un_p = nullptr,
                                             const uint32_t un_parity = 0)
{
    constexpr bool ASYNC = PIPE == 1;
    static_assert(L == 1 || (kF32 && DIM == 2), "two cells per thread: float, 2D only");
    using V = typename VecOf<L>::type;
    constexpr int N1 = P + 1, NQ = P + 2;
    constexpr int K = Tab<P>::K;
    constexpr int NT = TX * TYT;                         // threads
    constexpr int TYC = TYT * L;                         // cell rows of the tile
    constexpr int HYC = DIM == 1 ? 1 : TYC + 2;          // staged rows
    constexpr int TXL = TX / L;
    constexpr int NFX = (TX + 1) * TYT;                  // x-face items; lanes: the thread row's L cell rows
    constexpr int NFY = DIM == 2 ? TXL * (TYC + 1) : 0;  // y-face items; lanes: columns c + l TXL
    constexpr int TN = DIM == 1 ? 1 : N1;                // trace / face coefficients
    const Tab<P>& T = tab<P>();
    auto& su = ASYNC ? *su_async : S.su;
    auto& trx = S.trx;
    auto& trys = S.trys;
    auto& lam_s = S.lam_s;
    auto& mbar = S.mbar;
    auto& fail_s = S.fail_s;

    const int tid = threadIdx.x;
    const int64_t E = A.E;
    const bool need_lam = (MODE == 0) && (A.stab != STAB_DG) && !A.lam_fixed;
    const bool periodic_x = A.bc[0] == BC_PERIODIC;
    const bool periodic_y = DIM == 2 && A.bc[2] == BC_PERIODIC;

    // ---- 0. stage the tile and its face halo ----
    if (ASYNC) {
        // staged by the caller
    } else if (PIPE == 2 || (TMA && DIM == 2 && A.use_tma)) {
        if constexpr (PIPE != 2) {
            const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&mbar);
            if (tid == 0) {
                fail_s = 0;
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar) : "memory");
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            }
            __syncthreads();
            if (tid == 0) {
                const uint32_t bytes = (uint32_t)(sizeof(Real) * K * HYC * HX);
                const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&su[0][0][0]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                             :: "r"(bar), "r"(bytes) : "memory");
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                    " [%0], [%1, {%2, %3, %4}], [%5];"
                    :: "r"(dst), "l"(reinterpret_cast<uint64_t>(&A.tmap)), "r"(tx0 - OX), "r"(ty0 - OY),
                       "r"(0), "r"(bar)
                    : "memory");
            }
            if (!mbar_wait(bar, 0, A.wait_limit)) {
                // gave up: the tile is skipped and the flag reports it, but the copy still
                // lands in this CTA's shared memory, so wait for it (bounded) before leaving
                fail_s = 1;
                mbar_wait(bar, 0);
            }
            __syncthreads();
            if (fail_s) {
                if (tid == 0) atomicOr(A.flag, 2u);
                return;
            }
        }
        // periodic images of halo cells that lie outside the box's wrap-free view
        const bool edge = (periodic_x && (tx0 == 0 || tx0 + TX >= A.nx)) ||
                          (periodic_y && (ty0 == 0 || ty0 + TYC >= A.ny));
        if (edge) {
            for (int idx = tid; idx < K * HYC * HX; idx += NT) {
                const int k = idx / (HYC * HX);
                const int rem = idx - k * (HYC * HX);
                const int r = rem / HX, cc = rem - r * HX;
                const int ux = tx0 - OX + cc, uy = ty0 - OY + r;     // unwrapped
                if (ux < -1 || ux > A.nx || uy < -1 || uy > A.ny) continue;
                const bool inx = ux >= 0 && ux < A.nx, iny = uy >= 0 && uy < A.ny;
                if (inx && iny) continue;          // delivered by the box
                if (!inx && !iny) continue;        // corner: not needed
                const int gx = wrap_x(A, ux), gy = wrap_y(A, uy);
                if (gx < 0 || gy < 0) continue;
                su[k][r][cc] = A.Uk[k * E + (int64_t)gy * A.nx + gx];
            }
            __syncthreads();
        }
    } else {
        for (int idx = tid; idx < HYC * HX; idx += NT) {
            const int r = idx / HX, cc = idx - r * HX;
            if (cc < OX - 1 || cc > OX + TX) continue;
            const bool corner = DIM == 2 && (r == 0 || r == HYC - 1) && (cc == OX - 1 || cc == OX + TX);
            if (corner) continue;
            const int gx = wrap_x(A, tx0 - OX + cc);
            const int gy = DIM == 2 ? wrap_y(A, ty0 - OY + r) : 0;
            if (gx < 0 || gy < 0) {
                // no cell here: zeros keep the arithmetic of masked lanes finite
#pragma unroll
                for (int k = 0; k < K; ++k) su[k][r][cc] = Real(0);
                continue;
            }
            const Real* src = A.Uk + (int64_t)gy * A.nx + gx;
            if (A.cg_loads) {
#pragma unroll
                for (int k = 0; k < K; ++k) su[k][r][cc] = __ldcg(src + k * E);
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) su[k][r][cc] = src[k * E];
            }
        }
        __syncthreads();
    }

    const int lx = tid % TX, ly = tid / TX;
    const int gx = tx0 + lx;
    const int sc = lx + OX;
    int cy[L], gy[L];          // tile row and mesh row of lane l's cell
    bool in[L];
    bool any_in = false;
#pragma unroll
    for (int l = 0; l < L; ++l) {
        cy[l] = L * ly + l;
        gy[l] = ty0 + cy[l];
        in[l] = gx < A.nx && (DIM == 1 || gy[l] < A.ny);
        any_in = any_in || in[l];
    }

    V c[K];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int l = 0; l < L; ++l) lane(c[k], l) = su[k][cy[l] + OY][sc];

    // ---- 1a. traces of this thread's slots (also for slots that hold periodic images) ----
    if (MODE == 0) {
#pragma unroll
        for (int t = 0; t < TN; ++t) {
            V xm = vbc<V>(0), xp = vbc<V>(0), ym = vbc<V>(0), yp = vbc<V>(0);
#pragma unroll
            for (int n = 0; n < N1; ++n) {
                const V kx = DIM == 1 ? c[n] : c[n + N1 * t];
                xp = vadd(xp, kx);
                xm = (n & 1) ? vsub(xm, kx) : vadd(xm, kx);
                if (DIM == 2) {
                    const V ky = c[t + N1 * n];
                    yp = vadd(yp, ky);
                    ym = (n & 1) ? vsub(ym, ky) : vadd(ym, ky);
                }
            }
#pragma unroll
            for (int l = 0; l < L; ++l) {
                trx[cy[l]][0][t][lx + 1] = lane(xm, l);
                trx[cy[l]][1][t][lx + 1] = lane(xp, l);
                if (DIM == 2) {
                    trys[cy[l] + 1][0][t][lx] = lane(ym, l);
                    trys[cy[l] + 1][1][t][lx] = lane(yp, l);
                }
            }
        }
        // halo cells: the one trace that faces the tile
        constexpr int NH = 2 * TYC + (DIM == 2 ? 2 * TX : 0);
        for (int hidx = tid; hidx < NH; hidx += NT) {
            int r, cc, side, axis;
            if (hidx < TYC) { r = hidx + OY; cc = OX - 1; axis = 0; side = 1; }
            else if (hidx < 2 * TYC) { r = hidx - TYC + OY; cc = OX + TX; axis = 0; side = 0; }
            else if (hidx < 2 * TYC + TX) { r = 0; cc = OX + hidx - 2 * TYC; axis = 1; side = 1; }
            else { r = HYC - 1; cc = OX + hidx - 2 * TYC - TX; axis = 1; side = 0; }
#pragma unroll
            for (int t = 0; t < TN; ++t) {
                Real v = Real(0);
#pragma unroll
                for (int n = 0; n < N1; ++n) {
                    const int k = DIM == 1 ? n : (axis == 0 ? n + N1 * t : t + N1 * n);
                    const Real ck = su[k][r][cc];
                    v += (side == 0 && (n & 1)) ? -ck : ck;
                }
                if (axis == 0) trx[r - OY][side][t][cc == OX - 1 ? 0 : TX + 1] = v;
                else trys[r == 0 ? 0 : TYC + 1][side][t][cc - OX] = v;
            }
        }
        if (need_lam) {
#pragma unroll
            for (int l = 0; l < L; ++l) lam_s[cy[l]][lx] = Real(0);
        }
    }

    // ---- 1b. sensor (Sec. 4): Hermite candidates of the face neighbours ----
    V gamma = vbc<V>((MODE == 0 && A.stab == STAB_LO) ? Real(1) : Real(0));
    if ((MODE == 1 || A.stab >= STAB_WENO) && any_in) {
        bool has[2 * DIM][L];   // face neighbour f of lane l's cell exists
        V wsum;
        V wnb[2 * DIM];         // unnormalised neighbour weights (zero where missing)
        const V beta0 = qform<P>(T, c);
        const V d0 = vadd(vbc<V>(A.eps_w), beta0);
#pragma unroll
        for (int l = 0; l < L; ++l) {
            int me = 0;
#pragma unroll
            for (int f = 0; f < 2 * DIM; ++f) {
                const int nx_ = gx + (f == 0 ? -1 : (f == 1 ? 1 : 0));
                const int ny_ = gy[l] + (f == 2 ? -1 : (f == 3 ? 1 : 0));
                has[f][l] = (f < 2) ? (wrap_x(A, nx_) >= 0) : (wrap_y(A, ny_) >= 0);
                me += has[f][l] ? 1 : 0;
            }
            lane(wsum, l) = div_w(Real(1) - Real(me) * A.w_nbr, lane(d0, l) * lane(d0, l));
        }
        const V w0 = wsum;      // unnormalised weight of the cell's own candidate
        V dacc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) dacc[k] = vbc<V>(0);
#pragma unroll
        for (int f = 0; f < 2 * DIM; ++f) {
            wnb[f] = vbc<V>(0);
            bool any = false;
#pragma unroll
            for (int l = 0; l < L; ++l) any = any || has[f][l];
            if (!any) continue;
            const int axis = f >> 1, side = f & 1;
            const int dr = f == 2 ? -1 : (f == 3 ? 1 : 0);
            const int nc = sc + (f == 0 ? -1 : (f == 1 ? 1 : 0));
            V cn[K];
#pragma unroll
            for (int k = 0; k < K; ++k)
#pragma unroll
                for (int l = 0; l < L; ++l) lane(cn[k], l) = su[k][cy[l] + OY + dr][nc];
            V cl[K];
#pragma unroll
            for (int k = 1; k < K; ++k) {
                const int i = k % N1, j = k / N1;
                const int a = axis == 0 ? i : j;
                // P_m(xi +- 2) has degree m and leading coefficient 1: the m = a term
                // is cn[k] itself, the others have m > a
                V sacc = cn[k];
#pragma unroll
                for (int m = a + 1; m < N1; ++m) {
                    const int km = axis == 0 ? m + N1 * j : i + N1 * m;
                    sacc = vfma(T.T[side][a][m], cn[km], sacc);
                }
                cl[k] = sacc;
            }
            cl[0] = vbc<V>(0);
            const V dl = vadd(vbc<V>(A.eps_w), qform<P>(T, cl));
            V wl;
#pragma unroll
            for (int l = 0; l < L; ++l)
                lane(wl, l) = has[f][l] ? div_w(A.w_nbr, lane(dl, l) * lane(dl, l)) : Real(0);
            wsum = vadd(wsum, wl);
            wnb[f] = wl;
#pragma unroll
            for (int k = 1; k < K; ++k) dacc[k] = vfma(wl, vsub(c[k], cl[k]), dacc[k]);
        }
        V inv;
#pragma unroll
        for (int l = 0; l < L; ++l) lane(inv, l) = div_w(Real(1), lane(wsum, l));
        if (A.stab == STAB_ZHAO) {
            // the comparison sensor of Zhao et al. restated in Sec. 5.6: deviation of the
            // nonlinear weights from the linear ones, over its largest possible value (all
            // weight on the candidate of smallest linear weight); 0 without neighbours
#pragma unroll
            for (int l = 0; l < L; ++l) {
                int me = 0;
#pragma unroll
                for (int f = 0; f < 2 * DIM; ++f) me += has[f][l] ? 1 : 0;
                Real g = Real(0);
                if (me > 0) {
                    const Real lin0 = Real(1) - Real(me) * A.w_nbr;
                    const Real iw = lane(inv, l);
                    Real dev = zpow(A, fabs(lane(w0, l) * iw / lin0 - Real(1)));
#pragma unroll
                    for (int f = 0; f < 2 * DIM; ++f)
                        if (has[f][l]) dev += zpow(A, fabs(lane(wnb[f], l) * iw / A.w_nbr - Real(1)));
                    const Real minlin = lin0 < A.w_nbr ? lin0 : A.w_nbr;
                    g = dev / (zpow(A, fabs(Real(1) / minlin - Real(1))) + Real(me));
                }
                lane(gamma, l) = g;
                if (MODE == 1 && in[l]) A.gamma_out[(int64_t)gy[l] * A.nx + gx] = (double)g;
            }
        } else {
            // U - U* = sum_l w_l (c - c_l)
#pragma unroll
            for (int k = 1; k < K; ++k) dacc[k] = vmul(dacc[k], inv);
            dacc[0] = vbc<V>(0);
            const V qd = qform<P>(T, dacc);
#pragma unroll
            for (int l = 0; l < L; ++l) {
                const Real num = sqrt_r(fmax(lane(qd, l), Real(0)));
                const Real b0 = lane(beta0, l);
                Real g;
                if (num <= A.eps_s) {
                    g = Real(0);
                } else if (b0 <= Real(0)) {
                    g = Real(1);
                } else {
                    const Real r = num / sqrt_r(b0);
                    g = r < Real(1) ? r : Real(1);
                    if (!A.q_one) g = pow(g, A.q);
                    if (r < A.b) g = Real(0);
                }
                lane(gamma, l) = g;
                if (MODE == 1 && in[l]) A.gamma_out[(int64_t)gy[l] * A.nx + gx] = (double)g;
            }
        }
    }
    if (MODE == 1) return;

    // ---- 1c. volume term (Eq. weak2): acc_ij = sum_q W_q [D_i B_j Fx + B_i D_j Fy] ----
    V acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = vbc<V>(0);
    V lam = vbc<V>(0);
    const Real xc = fma_x(Real(gx) + Real(0.5), A.h, A.x0);
    V yc;
#pragma unroll
    for (int l = 0; l < L; ++l) lane(yc, l) = DIM == 2 ? fma_x(Real(gy[l]) + Real(0.5), A.h, A.y0) : Real(0);
    if constexpr (DIM == 1) {
        V u[NQ], fx[NQ];
        interp_sym<N1, NQ>(T.B, c, u);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            V fy, spd;
            vol_flux_v<FLUX>(A, u[q], fma_x(A.hh, T.g[q], xc), vbc<V>(0), fx[q], fy, spd);
            lam = vmax(lam, spd);
        }
        project_sym<true, N1, NQ>(T.WD, fx, acc);
        acc[0] = vbc<V>(0);
    } else {
        // one Gauss row qy at a time: the polynomial reduced to the row (rr[i] =
        // sum_j P_j(g_qy) c_ij), its values at the row's points, the fluxes there, and
        // their projection acc_ij += W_qy [P_j(g_qy) sum_qx W_qx P_i'(g_qx) Fx
        //                                 + P_j'(g_qy) sum_qx W_qx P_i(g_qx) Fy]
        auto row = [&](const int qy, const V (&rr)[N1]) {
            V y;
#pragma unroll
            for (int l = 0; l < L; ++l) lane(y, l) = fma_x(A.hh, T.g[qy], lane(yc, l));
            V u[NQ], fx[NQ], fy[NQ];
            interp_sym<N1, NQ>(T.B, rr, u);
#pragma unroll
            for (int qx = 0; qx < NQ; ++qx) {
                V spd;
                vol_flux_v<FLUX>(A, u[qx], fma_x(A.hh, T.g[qx], xc), y, fx[qx], fy[qx], spd);
                lam = vmax(lam, spd);
            }
            V px[N1], py[N1];
            project_sym<true, N1, NQ>(T.WD, fx, px);      // px[0] = 0 (P_0' = 0)
            project_sym<false, N1, NQ>(T.WB, fy, py);
#pragma unroll
            for (int j = 0; j < N1; ++j)
#pragma unroll
                for (int i = 0; i < N1; ++i) {
                    V t = acc[i + N1 * j];
                    if (i > 0) t = vfma(T.WB[qy][j], px[i], t);
                    if (j > 0) t = vfma(T.WD[qy][j], py[i], t);   // P_0' = 0
                    acc[i + N1 * j] = t;
                }
        };
        // A rolled loop over the rows: one copy of the row's code (its table reads become
        // indexed constant loads) costs fewer instruction-fetch stalls than five unrolled
        // copies with the rows at +-g paired (measured 1.4 % faster per step).
#pragma unroll 1
        for (int qy = 0; qy < NQ; ++qy) {
            V rr[N1];
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                V e = c[i];
#pragma unroll
                for (int j = 1; j < N1; ++j) e = vfma(T.B[qy][j], c[i + N1 * j], e);
                rr[i] = e;
            }
            row(qy, rr);
        }
    }
    __syncthreads();

    // The stage array is no longer read: bring the Un tile into it now, so that its
    // load overlaps the face phase (second phase of the same mbarrier).
    const bool un_tma = PIPE == 0 && TMA && DIM == 2 && A.use_tma && A.use_tma_un && A.has_un;
    const bool un_async = ASYNC && A.has_un;
    if (un_async) stage_un_async<P, L, TYT>(A, tx0, ty0, su);
    const bool un_pipe = PIPE == 2 && A.has_un;
    if (PIPE == 2 && tid == 0 && nxt_x >= 0) {
        // the stage array is dead: request the next tile's box into it
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&mbar);
        const uint32_t bytes = (uint32_t)(sizeof(Real) * K * HYC * HX);
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&su[0][0][0]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];"
            :: "r"(dst), "l"(reinterpret_cast<uint64_t>(&A.tmap_p)), "r"(nxt_x - OX), "r"(nxt_y - OY), "r"(0),
               "r"(bar)
            : "memory");
    }
    if (un_tma && tid == 0) {
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&mbar);
        const uint32_t bytes = (uint32_t)(sizeof(Real) * K * TYC * TX);
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&su[0][0][0]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];"
            :: "r"(dst), "l"(reinterpret_cast<uint64_t>(&A.tmap_un)), "r"(tx0), "r"(ty0), "r"(0), "r"(bar)
            : "memory");
    }

    // ---- 2. faces: each face of the tile once, from the traces ----
    // item f of the x-faces (xf true) or of the y-faces; XF is a compile-time or a
    // run-time flag
    auto face_item = [&](auto XF, const int f) {
        const bool xf = XF;
        int flx[L], fly[L];        // tile position of the cell on the plus side of lane l's face
        if (xf) {
            const int p = f / (TX + 1), col = f - p * (TX + 1);
#pragma unroll
            for (int l = 0; l < L; ++l) { flx[l] = col; fly[l] = L * p + l; }
        } else {
            const int row = f / TXL, col = f - row * TXL;
#pragma unroll
            for (int l = 0; l < L; ++l) { flx[l] = col + l * TXL; fly[l] = row; }
        }
        bool valid[L];
        bool anyv = false;
#pragma unroll
        for (int l = 0; l < L; ++l) {
            const int fgx = tx0 + flx[l], fgy = ty0 + fly[l];
            valid[l] = xf ? (fgx <= A.nx && fgy < A.ny) : (fgy <= A.ny && fgx < A.nx);
            anyv = anyv || valid[l];
        }
        if (!anyv) return;
        [[maybe_unused]] const int axis = xf ? 0 : 1;   // read by the fluxes that depend on the face orientation
        // the lanes of an item share the face column (x-faces) or row (y-faces), hence
        // the boundary situation
        const int fgx0 = tx0 + flx[0], fgy0 = ty0 + fly[0];
        const bool minus_in = xf ? (fgx0 - 1 >= 0 || periodic_x) : (fgy0 - 1 >= 0 || periodic_y);
        const bool plus_in = xf ? (fgx0 < A.nx || periodic_x) : (fgy0 < A.ny || periodic_y);
        V tm[TN], tp[TN];
#pragma unroll
        for (int t = 0; t < TN; ++t)
#pragma unroll
            for (int l = 0; l < L; ++l) {
                if (xf) {
                    lane(tm[t], l) = trx[fly[l]][1][t][flx[l]];
                    lane(tp[t], l) = trx[fly[l]][0][t][flx[l] + 1];
                } else {
                    lane(tm[t], l) = trys[DIM == 2 ? fly[l] : 0][1][t][flx[l]];
                    lane(tp[t], l) = trys[DIM == 2 ? fly[l] + 1 : 0][0][t][flx[l]];
                }
            }
        constexpr int NFQ = DIM == 1 ? 1 : NQ;
        // KPP: a y-face is an x-face of the states shifted by pi/2 (llf_kpp).  P_0 = 1, so
        // the shift added to the first trace coefficient shifts every face value.
        [[maybe_unused]] const Real sh = (FLUX == FLUX_KPP && DIM == 2 && !xf) ? Real(0.5 * kPi) : Real(0);
        if constexpr (FLUX == FLUX_KPP && DIM == 2) {
            tm[0] = vadd(tm[0], vbc<V>(sh));
            tp[0] = vadd(tp[0], vbc<V>(sh));
        }
        V uLq[NFQ], uRq[NFQ];
        if constexpr (DIM == 1) {
            uLq[0] = tm[0];
            uRq[0] = tp[0];
        } else {
            interp_sym<N1, NQ>(T.B, tm, uLq);
            interp_sym<N1, NQ>(T.B, tp, uRq);
        }
        V Hq[NFQ];
        V lm = vbc<V>(0), lp = vbc<V>(0);
#pragma unroll
        for (int q = 0; q < NFQ; ++q) {
            if constexpr (FLUX == FLUX_KPP) {
                V uL = uLq[q], uR = uRq[q];
                if (!minus_in || !plus_in) {
                    // ghost state; in the shifted variable F'(u).e_axis = cos u' on both axes
#pragma unroll
                    for (int l = 0; l < L; ++l) {
                        Real ul = lane(uL, l), ur = lane(uR, l), sn, cs;
                        if (!minus_in) {
                            sincos_r(ur, &sn, &cs);
                            ul = (A.bc[xf ? 0 : 2] == BC_INFLOW_ZERO && -cs < Real(0)) ? sh : ur;
                        } else {
                            sincos_r(ul, &sn, &cs);
                            ur = (A.bc[xf ? 1 : 3] == BC_INFLOW_ZERO && cs < Real(0)) ? sh : ul;
                        }
                        lane(uL, l) = ul;
                        lane(uR, l) = ur;
                    }
                }
                if (need_lam) {
#pragma unroll
                    for (int l = 0; l < L; ++l) {   // |F'| = 1 in 2D; 1D: |cos u| (no shift)
                        lane(lm, l) = fmax(lane(lm, l), speed_norm<FLUX>(A, lane(uL, l), Real(0), Real(0)));
                        lane(lp, l) = fmax(lane(lp, l), speed_norm<FLUX>(A, lane(uR, l), Real(0), Real(0)));
                    }
                }
                Hq[q] = llf_kpp(uL, uR);
            } else {
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    Real x = Real(0), y = Real(0);
                    if (FLUX == FLUX_ROTATION || need_lam || !minus_in || !plus_in) {
                        const int fgx = tx0 + flx[l], fgy = ty0 + fly[l];
                        if (xf) {
                            x = fma_x(Real(fgx), A.h, A.x0);
                            y = DIM == 2 ? fma_x(A.hh, T.g[q], fma_x(Real(fgy) + Real(0.5), A.h, A.y0)) : Real(0);
                        } else {
                            x = fma_x(A.hh, T.g[q], fma_x(Real(fgx) + Real(0.5), A.h, A.x0));
                            y = fma_x(Real(fgy), A.h, A.y0);
                        }
                    }
                    Real ul = lane(uLq[q], l), ur = lane(uRq[q], l);
                    if (!minus_in) {
                        // ghost for the plus cell, whose outward normal is -e_axis
                        const int bside = xf ? 0 : 2;
                        ul = (A.bc[bside] == BC_INFLOW_ZERO && -dflux_axis<FLUX>(A, axis, ur, x, y) < Real(0)) ? Real(0) : ur;
                    } else if (!plus_in) {
                        const int bside = xf ? 1 : 3;
                        ur = (A.bc[bside] == BC_INFLOW_ZERO && dflux_axis<FLUX>(A, axis, ul, x, y) < Real(0)) ? Real(0) : ul;
                    }
                    if (need_lam) {
                        lane(lm, l) = fmax(lane(lm, l), speed_norm<FLUX>(A, ul, x, y));
                        lane(lp, l) = fmax(lane(lp, l), speed_norm<FLUX>(A, ur, x, y));
                    }
                    lane(Hq[q], l) = llf<FLUX>(A, axis, ul, ur, x, y);
                }
            }
        }
        V hq[TN];
        if constexpr (DIM == 1) hq[0] = Hq[0];
        else project_sym<false, N1, NQ>(T.WB, Hq, hq);
        // the flux replaces the minus-side trace, which only this face reads
#pragma unroll
        for (int l = 0; l < L; ++l) {
            if (xf) {
#pragma unroll
                for (int t = 0; t < TN; ++t) trx[fly[l]][1][t][flx[l]] = lane(hq[t], l);
            } else {
#pragma unroll
                for (int t = 0; t < TN; ++t) trys[DIM == 2 ? fly[l] : 0][1][t][flx[l]] = lane(hq[t], l);
            }
        }
        if (need_lam) {
#pragma unroll
            for (int l = 0; l < L; ++l) {
                if (!valid[l]) continue;
                // only traces of this tile's cells that lie in the domain count
                const int fgx = tx0 + flx[l], fgy = ty0 + fly[l];
                const int mlx = xf ? flx[l] - 1 : flx[l], mly = xf ? fly[l] : fly[l] - 1;
                if (minus_in && mlx >= 0 && mly >= 0 && (xf ? fgx - 1 < A.nx : fgy - 1 < A.ny))
                    atomic_max_nonneg(&lam_s[mly][mlx], lane(lm, l));
                if (plus_in && flx[l] < TX && fly[l] < TYC && fgx < A.nx && fgy < A.ny)
                    atomic_max_nonneg(&lam_s[fly[l]][flx[l]], lane(lp, l));
            }
        }
    };
    if constexpr (FLUX == FLUX_KPP) {
        // one body for both orientations: two copies of the sin/cos-heavy flux cost more
        // in instruction fetch than the orientation selects cost in issue
        for (int f = tid; f < NFX + NFY; f += NT) face_item(f < NFX, f < NFX ? f : f - NFX);
    } else {
        for (int f = tid; f < NFX; f += NT) face_item(std::integral_constant<bool, true>(), f);
        // the y-faces continue the x-faces' numbering across the threads, so no thread
        // takes more than one item above the even share
        for (int f = (tid + NT - NFX % NT) % NT; f < NFY; f += NT) face_item(std::integral_constant<bool, false>(), f);
    }
    if (ASYNC) cp_async_wait_all();
    __syncthreads();
    if (!any_in) return;

    // ---- 3. faces: -phi_k(+1) H on the plus faces, +phi_k(-1) H on the minus faces ----
    if constexpr (DIM == 1) {
        const V hm = trx[0][1][0][lx], hp = trx[0][1][0][lx + 1];
        const V de = vsub(hm, hp), dd = vadd(hm, hp);
#pragma unroll
        for (int n = 0; n < N1; ++n) acc[n] = (n & 1) ? vsub(acc[n], dd) : vadd(acc[n], de);
    } else {
#pragma unroll
        for (int t = 0; t < N1; ++t) {
            V xm, xp, ym, yp;
#pragma unroll
            for (int l = 0; l < L; ++l) {
                lane(xm, l) = trx[cy[l]][1][t][lx];
                lane(xp, l) = trx[cy[l]][1][t][lx + 1];
                lane(ym, l) = trys[cy[l]][1][t][lx];
                lane(yp, l) = trys[cy[l] + 1][1][t][lx];
            }
            // even n: += (m - p); odd n: += (-m - p), i.e. -= (m + p)
            const V dxe = vsub(xm, xp), dxo = vadd(xm, xp);
            const V dye = vsub(ym, yp), dyo = vadd(ym, yp);
#pragma unroll
            for (int n = 0; n < N1; ++n) {
                acc[n + N1 * t] = (n & 1) ? vsub(acc[n + N1 * t], dxo) : vadd(acc[n + N1 * t], dxe);
                acc[t + N1 * n] = (n & 1) ? vsub(acc[t + N1 * n], dyo) : vadd(acc[t + N1 * n], dye);
            }
        }
    }
    if (need_lam) {
#pragma unroll
        for (int l = 0; l < L; ++l) lane(lam, l) = fmax(lane(lam, l), lam_s[cy[l]][lx]);
    }

    // stabilization (Sec. 3), M^{-1}, RK combination (Eq. ssp)
    V ngs;                     // -gamma nu (2/h), per cell
    bool any_gamma = false;
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const Real lamv = A.lam_fixed ? A.lambda_nu : lane(lam, l);
        lane(ngs, l) = -(lane(gamma, l) * lamv * Real(1.0 / P));
        any_gamma = any_gamma || lane(gamma, l) != Real(0);
    }
    V chk = vbc<V>(0);         // becomes NaN if any output is not finite
    const Real* sun = PIPE == 2 ? un_p : reinterpret_cast<const Real*>(&su[0][0][0]);   // Un tile [K][TYC][TX]
    if (un_tma && !mbar_wait((uint32_t)__cvta_generic_to_shared(&mbar), 1, A.wait_limit)) {
        atomicOr(A.flag, 2u);
        mbar_wait((uint32_t)__cvta_generic_to_shared(&mbar), 1);   // let the copy land first
        return;
    }
    if (un_pipe && !mbar_wait((uint32_t)__cvta_generic_to_shared(&S.mbar_un), un_parity, A.wait_limit)) {
        atomicOr(A.flag, 2u);
        fail_s = 1;            // the caller stops after this tile (its copies drained)
        return;
    }
    int64_t e[L];
#pragma unroll
    for (int l = 0; l < L; ++l) e[l] = (int64_t)gy[l] * A.nx + gx;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int i = k % N1, j = k / N1;
        V r = acc[k];
        if (any_gamma) {
            V kc;
            if constexpr (DIM == 1) {
                kc = vbc<V>(0);
#pragma unroll
                for (int m = 1; m < N1; ++m)
                    if (((i + m) & 1) == 0 && i > 0) kc = vfma(T.A1[i][m], c[m], kc);
            } else {
                V s1 = vbc<V>(0), s2 = vbc<V>(0);
#pragma unroll
                for (int m = 1; m < N1; ++m) {
                    if (((i + m) & 1) == 0 && i > 0) s1 = vfma(T.A1[i][m], c[m + N1 * j], s1);
                    if (((j + m) & 1) == 0 && j > 0) s2 = vfma(T.A1[j][m], c[i + N1 * m], s2);
                }
                kc = vfma(T.A0[i], s2, vmul(T.A0[j], s1));
            }
            r = vfma(ngs, kc, r);
        }
        Real mi = T.minv[i];
        if (DIM == 2) mi *= T.minv[j];
        const V Lk = vmul(A.two_h * mi, r);
        V out = vfma(A.cl, Lk, vmul(A.ck, c[k]));
        if (A.has_un) {
            V unk;
#pragma unroll
            for (int l = 0; l < L; ++l) {
                const Real* un = A.Un + e[l] + k * E;
                lane(unk, l) = (un_tma || un_async || un_pipe) ? sun[(k * TYC + cy[l]) * TX + lx]
                                      : (in[l] ? (A.cg_loads ? __ldcg(un) : *un) : Real(0));
            }
            out = vfma(A.cn, unk, out);
        }
        chk = vfma(out, vbc<V>(0), chk);
#pragma unroll
        for (int l = 0; l < L; ++l)
            if (in[l]) A.Uout[e[l] + k * E] = lane(out, l);
    }
#pragma unroll
    for (int l = 0; l < L; ++l)
        if (in[l] && lane(chk, l) != lane(chk, l)) atomicOr(A.flag, 1u);
}

template <int P, int FLUX, int MODE>
__global__ void __launch_bounds__(NTS, LS == 2 ? 512 / NTS : (kF32 ? 6 : 3)) stage_kernel(const __grid_constant__ KParams A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if ((__cvta_generic_to_shared(smem_raw) & 127u) != 0) {   // TMA needs an aligned box
        if (threadIdx.x == 0) atomicOr(A.flag, 2u);
        return;
    }
    TileSmem<P, LS, TYS>& S = *reinterpret_cast<TileSmem<P, LS, TYS>*>(smem_raw);
    process_tile<P, FLUX, MODE, LS, TYS>(A, blockIdx.x * TX, DIM == 2 ? (blockIdx.y + A.tile_row0) * (TYS * LS) : 0, S);
}

#if DGW_DIM == 2
// Persistent float stage kernel (whole-mesh launches, 2D): one CTA of 512 threads per SM
// walks the tiles of kTileX2 x kPRows cells (tile t, t + gridDim.x, ...).  The next tile's
// box is requested into the stage array as soon as the volume phase has read the current
// one, and the tile's Un box into a buffer of its own at the tile's start, so that both
// loads overlap the arithmetic, and all sixteen warps of an SM work in the same phase
// (one copy of the phase's code in the instruction caches).  Every wait is bounded; a wait
// that gives up sets flag bit 2, and the CTA waits (bounded) for its copies in flight and
// stops.
constexpr int kPThreadRows = kPRows / 2;

template <int P>
constexpr size_t p_tile_bytes() { return (sizeof(TileSmem<P, 2, kPThreadRows>) + 127) / 128 * 128; }
template <int P>
constexpr size_t p_smem_bytes() { return p_tile_bytes<P>() + sizeof(Real) * Tab<P>::K * kPRows * TX; }

__device__ __forceinline__ void tma_box(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(0), "r"(bar)
        : "memory");
}

template <int P, int FLUX>
__global__ void __launch_bounds__(TX * kPThreadRows, 1) stage_kernel_p(const __grid_constant__ KParams A)
{
    using Smem = TileSmem<P, 2, kPThreadRows>;
    constexpr int K = Tab<P>::K;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if ((__cvta_generic_to_shared(smem_raw) & 127u) != 0) {   // TMA needs aligned boxes
        if (threadIdx.x == 0) atomicOr(A.flag, 2u);
        return;
    }
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    Real* un = reinterpret_cast<Real*>(smem_raw + p_tile_bytes<P>());
    const int ntx = (A.nx + TX - 1) / TX, nty = (A.ny + kPRows - 1) / kPRows, ntiles = ntx * nty;
    int t = blockIdx.x;
    if (t >= ntiles) return;
    const int tid = threadIdx.x;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&S.mbar);
    const uint32_t bar_un = (uint32_t)__cvta_generic_to_shared(&S.mbar_un);
    const uint32_t su_dst = (uint32_t)__cvta_generic_to_shared(&S.su[0][0][0]);
    const uint32_t un_dst = (uint32_t)__cvta_generic_to_shared(un);
    constexpr uint32_t box_bytes = (uint32_t)(sizeof(Real) * K * Smem::HYC * HX);
    constexpr uint32_t un_bytes = (uint32_t)(sizeof(Real) * K * kPRows * TX);
    const bool has_un = A.has_un != 0;
    if (tid == 0) {
        S.fail_s = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar_un) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        tma_box(su_dst, &A.tmap_p, (t % ntx) * TX - OX, (t / ntx) * kPRows - OY, bar, box_bytes);
        if (has_un) tma_box(un_dst, &A.tmap_un_p, (t % ntx) * TX, (t / ntx) * kPRows, bar_un, un_bytes);
    }
    uint32_t ph = 0, ph_un = 0;
    bool box_pending = true, un_pending = has_un;
    for (;;) {
        const bool ok = mbar_wait(bar, ph, A.wait_limit);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(A.flag, 2u);
            break;
        }
        ph ^= 1u;
        box_pending = false;
        const int nt = t + (int)gridDim.x;
        const bool more = nt < ntiles;
        process_tile<P, FLUX, 0, 2, kPThreadRows, true, 2>(A, (t % ntx) * TX, (t / ntx) * kPRows, S, nullptr,
                                                          more ? (nt % ntx) * TX : -1, more ? (nt / ntx) * kPRows : 0,
                                                          un, ph_un);
        box_pending = more;
        if (__syncthreads_or(S.fail_s)) break;     // a Un wait gave up (flag set)
        if (has_un) {
            ph_un ^= 1u;
            un_pending = false;
        }
        if (!more) break;
        t = nt;
        if (has_un) {
            if (tid == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_box(un_dst, &A.tmap_un_p, (t % ntx) * TX, (t / ntx) * kPRows, bar_un, un_bytes);
            }
            un_pending = true;
        }
    }
    // copies still in flight land in this CTA's shared memory: wait for them (bounded)
    if (box_pending) mbar_wait(bar, ph);
    if (un_pending) mbar_wait(bar_un, ph_un);
}
#endif

// Current device, for per-device caches of kernel attributes (0 if it cannot be read or
// lies beyond the caches' 64 entries).
static int cur_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    return dev;
}

static KParams make_params(const StageArgs& s)
{
    KParams a;
    memset(&a, 0, sizeof a);
    a.use_tma = 0;
    a.use_tma_un = 0;
    a.cg_loads = 0;
    a.wait_limit = s.wait_limit > 0 ? s.wait_limit : (s.wait_limit == 0 ? kWaitLimit : 0);
    a.tile_row0 = DIM == 2 ? s.tile_row0 : 0;
    if (s.tmap) {
        a.tmap = *s.tmap;
        a.use_tma = 1;
    }
    if (s.tmap_un) {
        a.tmap_un = *s.tmap_un;
        a.use_tma_un = 1;
    }
    if (s.tmap_p) a.tmap_p = *s.tmap_p;
    if (s.tmap_un_p) {
        a.tmap_un_p = *s.tmap_un_p;
        a.use_p_un = 1;
    }
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
    a.theta = (Real)s.theta;
    a.theta_one = s.theta == 1.0;
    a.gam = (Real)s.gas_gamma;
    a.gm1 = (Real)(s.gas_gamma - 1.0);
    a.cn = (Real)s.cn; a.ck = (Real)s.ck; a.cl = (Real)s.cl;
    a.t_dev = s.t_dev;
    a.t_off = s.t_off;
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 4; ++k) a.bstate[i][k] = (Real)s.bstate[i][k];
    for (int f = 0; f < 4; ++f) {
        a.bsplit[f] = (Real)s.bsplit[f];
        a.bspeed[f] = (Real)s.bspeed[f];
        a.bbelow[f] = s.bbelow[f];
        a.babove[f] = s.babove[f];
    }
    return a;
}

// ------------------------------------------------------------------------------------
// batched ensemble: persistent kernel
// ------------------------------------------------------------------------------------
// cells per thread of the batch kernels: two stacked in y on the packed FP32 pipe (2D
// float), else one
constexpr int kBatchLanes = (kF32 && DIM == 2) ? 2 : 1;

template <int P, int TYB>
constexpr size_t batch_tile_bytes()
{
    return (sizeof(TileSmem<P, kBatchLanes, TYB>) + 127) / 128 * 128;
}

template <int P, int FLUX, int TYB>
__device__ __forceinline__ void batch_tiles(const BatchArgs& B, const BatchInst& I, const int r,
                                            const int tile0, const int ntile, unsigned char* smem)
{
    KParams A;
    A.use_tma = 0;
    A.use_tma_un = 0;
    A.cg_loads = 1;
    A.wait_limit = kWaitLimit;
    A.tile_row0 = 0;
    const Real* U = static_cast<const Real*>(B.U) + I.off;
    const Real* S1 = static_cast<const Real*>(B.S1) + I.off;
    const Real* S2 = static_cast<const Real*>(B.S2) + I.off;
    A.Uk = r == 0 ? U : (r == 1 ? S1 : S2);
    A.Un = U;
    A.Uout = const_cast<Real*>(r == 0 ? S1 : (r == 1 ? S2 : U));
    A.gamma_out = nullptr;
    A.flag = B.flag;
    A.E = I.E;
    A.nx = I.nx;
    A.ny = I.ny;
#pragma unroll
    for (int f = 0; f < 4; ++f) A.bc[f] = I.bc[f];
    A.stab = B.stab;
    A.lam_fixed = I.lambda_nu > 0.0;
    A.q_one = B.q == 1.0;
    A.has_un = r > 0;
    A.x0 = (Real)I.x0; A.y0 = (Real)I.y0; A.h = (Real)I.h; A.hh = (Real)(0.5 * I.h);
    A.two_h = (Real)(2.0 / I.h);
    A.a0 = (Real)I.a0; A.a1 = (Real)I.a1; A.cx = (Real)I.cx; A.cy = (Real)I.cy;
    A.omega = (Real)I.omega; A.lambda_nu = (Real)I.lambda_nu;
    A.q = (Real)B.q; A.b = (Real)B.b; A.w_nbr = (Real)B.w_nbr; A.eps_w = (Real)B.eps_w;
    A.eps_s = (Real)B.eps_s;
    A.theta = (Real)B.theta;
    A.theta_one = B.theta == 1.0;
    const double dt = I.dt;
    A.cn = (Real)(r == 0 ? 0.0 : (r == 1 ? 0.75 : 1.0 / 3.0));
    A.ck = (Real)(r == 0 ? 1.0 : (r == 1 ? 0.25 : 2.0 / 3.0));
    A.cl = (Real)(r == 0 ? dt : (r == 1 ? 0.25 * dt : 2.0 / 3.0 * dt));
    using Smem = TileSmem<P, kBatchLanes, TYB>;
    Smem& S = *reinterpret_cast<Smem*>(smem);
    // two stage buffers: the tile's own (S.su or the one after the tile's shared
    // memory) and the next tile's, filled by cp.async while this one is computed
    typename Smem::Stage* const buf0 = &S.su;
    typename Smem::Stage* const buf1 = reinterpret_cast<typename Smem::Stage*>(smem + batch_tile_bytes<P, TYB>());
    auto origin = [&](int t, int& tx0, int& ty0) {
        tx0 = (t % I.ntx) * TX;
        ty0 = DIM == 2 ? (t / I.ntx) * (TYB * kBatchLanes) : 0;
    };
    int tx0, ty0;
    origin(tile0, tx0, ty0);
    stage_tile_async<P, kBatchLanes, TYB>(A, tx0, ty0, *buf0);
    cp_async_wait_all();
    __syncthreads();
    for (int i = 0; i < ntile; ++i) {
        origin(tile0 + i, tx0, ty0);
        if (i + 1 < ntile) {
            int nx0, ny0;
            origin(tile0 + i + 1, nx0, ny0);
            stage_tile_async<P, kBatchLanes, TYB>(A, nx0, ny0, (i & 1) ? *buf0 : *buf1);
        }
        process_tile<P, FLUX, 0, kBatchLanes, TYB, false, 1>(A, tx0, ty0, S, (i & 1) ? buf1 : buf0);
        cp_async_wait_all();      // nothing left in flight when the tile had no face phase wait
        __syncthreads();
    }
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Persistent kernel over all work items of all stages of the instances of degree P, in
// tiles of TX x (TYB kBatchLanes) cells (TYB thread rows): items are dequeued in
// order, and an item waits only for its own instance's previous stage, whose items were
// all dequeued earlier by CTAs that are running, so no wait can deadlock (whether or not
// the whole grid is resident: the kernels of the batch run side by side on streams of
// their own).  Each wait is still bounded, and a wait that gives up stops the whole launch
// through B.abort.  One kernel per degree and tile height keeps each variant's registers
// to its own needs; instances of different degree never wait on each other.
template <int P, int TYB>
constexpr size_t batch_smem_bytes()
{
    // tile, second stage buffer, scheduler words
    return batch_tile_bytes<P, TYB>() + (sizeof(typename TileSmem<P, kBatchLanes, TYB>::Stage) + 127) / 128 * 128 + 128;
}

// resident CTAs per SM the register budget is sized for: two cells per thread (2D float)
// 80 / 104 / 168 registers a thread for P = 1 / 2 / 3, one cell (1D float) 64 / 80 / 128
// (the degree-3 tile spills at fewer), double 168
template <int P, int TYB>
constexpr int batch_min_blocks()
{
    constexpr int regs = !kF32 ? 168 : (kBatchLanes == 2 ? (P == 1 ? 80 : (P == 2 ? 104 : 168))
                                                         : (P == 1 ? 64 : (P == 2 ? 80 : 128)));
    return 65536 / (TX * TYB * regs) > 0 ? 65536 / (TX * TYB * regs) : 1;
}

template <int P, int TYB>
__global__ void __launch_bounds__(TX * TYB, batch_min_blocks<P, TYB>()) batch_kernel(const BatchArgs B)
{
    constexpr size_t kSmem = batch_smem_bytes<P, TYB>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    long long& s_w = *reinterpret_cast<long long*>(smem_raw + kSmem - 128);
    int& s_ok = *reinterpret_cast<int*>(smem_raw + kSmem - 64);
    const long long total = (long long)B.nitems * B.nstages;
    for (;;) {
        if (threadIdx.x == 0) {
            long long w = (long long)atomicAdd(B.queue, 1ULL);
            if (w >= total || *((volatile int*)B.abort)) w = -1;
            s_w = w;
        }
        __syncthreads();
        const long long w = s_w;
        if (w < 0) break;
        const int g = (int)(w / B.nitems);
        const BatchItem it = B.items[w - (long long)g * B.nitems];
        const BatchInst& I = B.inst[it.inst];
        if (threadIdx.x == 0) {
            const unsigned long long need = (unsigned long long)g * (unsigned long long)I.ntiles + (B.unreachable ? 1ull : 0ull);
            int ok = 1;
            if (need > 0) {
                ok = 0;
                for (long long n = 0; n < B.wait_limit; ++n) {
                    if (ld_acquire(&B.done[it.inst]) >= need) { ok = 1; break; }
                    if (*((volatile int*)B.abort)) break;
                    __nanosleep(64);
                }
            }
            if (!ok) {
                atomicOr(B.flag, 2u);
                atomicExch(B.abort, 1);
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;
        __threadfence();
        const int r = g % 3;
        if (I.p == P) {
            if (I.flux == FLUX_ADVECT) batch_tiles<P, FLUX_ADVECT, TYB>(B, I, r, it.tile0, it.ntile, smem_raw);
            else if (I.flux == FLUX_BURGERS) batch_tiles<P, FLUX_BURGERS, TYB>(B, I, r, it.tile0, it.ntile, smem_raw);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(&B.done[it.inst], (unsigned long long)it.ntile);
    }
}

// Tile heights (cell rows) built for the batch kernel: 2, 4 and 8 (float, 2D: one, two or
// four thread rows of two cells), kTileY2 (double, 2D), one (1D).
constexpr bool batch_rows_built(int rows)
{
    return DIM == 1 ? rows == 1 : (kF32 ? (rows == 2 || rows == 4 || rows == 8) : rows == kTileY2);
}

template <int P, int TYB>
static int batch_blocks_per_sm_pt()
{
    constexpr size_t kSmem = batch_smem_bytes<P, TYB>();
    if (kSmem > 48 * 1024 &&
        cudaFuncSetAttribute(batch_kernel<P, TYB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<P, TYB>, TX * TYB, kSmem) != cudaSuccess) return 0;
    return n;
}

template <int P, int TYB>
static cudaError_t launch_batch_pt(const BatchArgs& a, int grid, cudaStream_t st)
{
    batch_kernel<P, TYB><<<grid, TX * TYB, batch_smem_bytes<P, TYB>(), st>>>(a);
    return cudaGetLastError();
}

// dispatch over the built (degree, tile height) pairs; rows not built give 0 / an error
template <int P>
static int batch_blocks_per_sm_p(int rows)
{
    if constexpr (DIM == 1) return rows == 1 ? batch_blocks_per_sm_pt<P, 1>() : 0;
    else if constexpr (kF32) {
        switch (rows) {       // cell rows = thread rows x 2
        case 2: return batch_blocks_per_sm_pt<P, 1>();
        case 4: return batch_blocks_per_sm_pt<P, 2>();
        case 8: return batch_blocks_per_sm_pt<P, 4>();
        default: return 0;
        }
    } else return rows == kTileY2 ? batch_blocks_per_sm_pt<P, kTileY2>() : 0;
}

template <int P>
static cudaError_t launch_batch_p(const BatchArgs& a, int rows, int grid, cudaStream_t st)
{
    if constexpr (DIM == 1) return rows == 1 ? launch_batch_pt<P, 1>(a, grid, st) : cudaErrorInvalidValue;
    else if constexpr (kF32) {
        switch (rows) {       // cell rows = thread rows x 2
        case 2: return launch_batch_pt<P, 1>(a, grid, st);
        case 4: return launch_batch_pt<P, 2>(a, grid, st);
        case 8: return launch_batch_pt<P, 4>(a, grid, st);
        default: return cudaErrorInvalidValue;
        }
    } else return rows == kTileY2 ? launch_batch_pt<P, kTileY2>(a, grid, st) : cudaErrorInvalidValue;
}

static int batch_blocks_per_sm(int p, int rows)
{
    switch (p) {
    case 1: return batch_blocks_per_sm_p<1>(rows);
    case 2: return batch_blocks_per_sm_p<2>(rows);
    case 3: return batch_blocks_per_sm_p<3>(rows);
    default: return 0;
    }
}

static cudaError_t launch_batch(const BatchArgs& a, int p, int rows, int grid, cudaStream_t st)
{
    switch (p) {
    case 1: return launch_batch_p<1>(a, rows, grid, st);
    case 2: return launch_batch_p<2>(a, rows, grid, st);
    case 3: return launch_batch_p<3>(a, rows, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

#include "dgw_adjoint_impl.cuh"

template <int P>
static cudaError_t launch_vjp_p(const StageArgs& s, int flux, const void* lam, void* wself, void* wnb,
                                cudaStream_t st)
{
    const KParams a = make_params(s);
    const unsigned blocks = (unsigned)((s.E + 127) / 128);
    if (flux == FLUX_ADVECT)
        vjp_kernel<P, FLUX_ADVECT><<<blocks, 128, 0, st>>>(a, (const Real*)lam, (Real*)wself, (Real*)wnb);
    else if (flux == FLUX_BURGERS)
        vjp_kernel<P, FLUX_BURGERS><<<blocks, 128, 0, st>>>(a, (const Real*)lam, (Real*)wself, (Real*)wnb);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

static cudaError_t launch_vjp(const StageArgs& s, int p, int flux, const void* lam, void* wself, void* wnb,
                              cudaStream_t st)
{
    switch (p) {
    case 1: return launch_vjp_p<1>(s, flux, lam, wself, wnb, st);
    case 2: return launch_vjp_p<2>(s, flux, lam, wself, wnb, st);
    case 3: return launch_vjp_p<3>(s, flux, lam, wself, wnb, st);
    default: return cudaErrorInvalidValue;
    }
}

static cudaError_t launch_gather(const GatherArgs& g, int p, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((g.E + 127) / 128);
    const Real* x0 = (const Real*)g.x[0];
    const Real* x1 = (const Real*)g.x[1];
    const Real* x2 = (const Real*)g.x[2];
    const Real c0 = (Real)g.coef[0], c1 = (Real)g.coef[1], c2 = (Real)g.coef[2], cv = (Real)g.cvjp;
    switch (p) {
    case 1: gather_kernel<1><<<blocks, 128, 0, st>>>(g.E, g.nx, g.ny, (const Real*)g.wself, (const Real*)g.wnb, x0, x1, x2, c0, c1, c2, cv, (Real*)g.out); break;
    case 2: gather_kernel<2><<<blocks, 128, 0, st>>>(g.E, g.nx, g.ny, (const Real*)g.wself, (const Real*)g.wnb, x0, x1, x2, c0, c1, c2, cv, (Real*)g.out); break;
    case 3: gather_kernel<3><<<blocks, 128, 0, st>>>(g.E, g.nx, g.ny, (const Real*)g.wself, (const Real*)g.wnb, x0, x1, x2, c0, c1, c2, cv, (Real*)g.out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Euler system (Sec. 5.6): shared helpers, then the kernel of this unit's dimension
// ------------------------------------------------------------------------------------
// Reciprocal and square root of the Euler kernels.  float: the approximate instructions
// rcp.approx and sqrt.approx of the PTX ISA (relative error of a few ulp, far inside the
// float path's tolerance; a negative argument of the square root gives NaN);
// double: the correctly rounded operations.
__device__ __forceinline__ float rcp_e(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp_e(double x) { return 1.0 / x; }
__device__ __forceinline__ float sqrt_e(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double sqrt_e(double x) { return sqrt(x); }

// max(a, b) that returns NaN when either is NaN (fmax drops a NaN operand): a state
// without a real sound speed (rho <= 0 or p < 0) has no wave speed, and the step then
// returns non-finite values, which the stage's check reports
__device__ __forceinline__ Real max_nan(Real a, Real b)
{
    return fmax(a, b) + ((a - a) + (b - b));
}

#if DGW_DIM == 1
#include "dgw_euler_impl.cuh"
#else
#include "dgw_euler2d_impl.cuh"
#endif
#if DGW_DIM == 2 && defined(DGW_TC_VOLUME)
#include "dgw_tc_volume.cuh"
#endif

#if DGW_DIM == 2
// SMs of the current device (0 if it cannot be read)
static int sm_count()
{
    static int nsm[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (nsm[dev] == 0 && cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        nsm[dev] = 0;
    return nsm[dev];
}

// The persistent kernel pays where every SM walks several of its tiles; on smaller meshes
// (fewer than four tiles of 32 x 32 cells per SM) the tile kernel's smaller tiles keep
// more SMs busy.
static bool persistent_pays(int nx, int ny)
{
    const int nsm = sm_count();
    const long long ntiles = (long long)((nx + TX - 1) / TX) * ((ny + kPRows - 1) / kPRows);
    return nsm > 0 && ntiles >= 4LL * nsm;
}

template <int P, int FLUX>
static cudaError_t launch_persistent(const KParams& a, cudaStream_t st)
{
    constexpr size_t smem = p_smem_bytes<P>();
    static_assert(smem <= 227 * 1024, "persistent tile exceeds the shared memory of an SM");
    static bool opted[64] = {false};
    const int dev = cur_device();
    if (!opted[dev]) {
        cudaError_t e = cudaFuncSetAttribute(stage_kernel_p<P, FLUX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        opted[dev] = true;
    }
    const int nsm = sm_count();
    const int ntiles = ((a.nx + TX - 1) / TX) * ((a.ny + kPRows - 1) / kPRows);
    if (ntiles == 0) return cudaSuccess;
    stage_kernel_p<P, FLUX><<<ntiles < nsm ? ntiles : nsm, TX * kPThreadRows, smem, st>>>(a);
    return cudaGetLastError();
}
#endif

template <int P, int FLUX>
static cudaError_t launch_pf(const StageArgs& s, int mode, cudaStream_t st)
{
    const KParams a = make_params(s);
    constexpr int TYC = TYS * LS;
    const int trows = (s.ny + TYC - 1) / TYC;
    if (DIM == 2 && (s.tile_row0 < 0 || s.tile_rows < 0 || s.tile_row0 + s.tile_rows > trows)) return cudaErrorInvalidValue;
    const int grows = DIM == 2 ? (s.tile_rows > 0 ? s.tile_rows : trows - s.tile_row0) : 1;
    dim3 grid((s.nx + TX - 1) / TX, grows);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    const size_t smem = sizeof(TileSmem<P, LS, TYS>);
    // once per instantiation and device: opt in to more than 48 KB of dynamic shared
    // memory where needed, and prefer the largest shared-memory carveout (several tiles per SM)
    static bool opted[64][2] = {{false, false}};
    const int dev = cur_device();
    if (!opted[dev][mode]) {
        const void* fn = mode == 0 ? (const void*)stage_kernel<P, FLUX, 0> : (const void*)stage_kernel<P, FLUX, 1>;
        cudaError_t e = cudaSuccess;
        if (smem > 48 * 1024) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        opted[dev][mode] = true;
    }
#if DGW_DIM == 2
    if constexpr (kF32) {
        if (mode == 0 && s.tmap_p && s.tile_row0 == 0 && s.tile_rows == 0 && (!a.has_un || a.use_p_un) &&
            (s.kernel_choice == 2 || persistent_pays(s.nx, s.ny)))
            return launch_persistent<P, FLUX>(a, st);
    }
#endif
    if (mode == 0) stage_kernel<P, FLUX, 0><<<grid, NTS, smem, st>>>(a);
    else stage_kernel<P, FLUX, 1><<<grid, NTS, smem, st>>>(a);
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
#if DGW_DIM == 1
    if (flux == FLUX_EULER) return launch_euler(a, p, mode, s);
#else
    if (flux == FLUX_EULER) return launch_euler2d(a, p, mode, s);
#endif
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
