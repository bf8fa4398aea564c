// Stage kernel of the WENO-stabilized RKDG scheme, tiled.
//
// Included by one translation unit per (precision, dimension) with DGW_REAL, DGW_DIM
// and DGW_NS defined.  Each unit owns its copy of the constant-memory operator tables.
//
// One CTA owns a TX x TY tile of cells (one thread per cell).
//   0. It stages the modal coefficients of the tile plus a one-cell face halo in shared
//      memory: one TMA box load (2D, 16-byte aligned strides) waited on through an
//      mbarrier with a bounded spin, else cooperative coalesced loads; periodic halo
//      cells of boundary tiles are then filled from the wrapped side.
//   1. Per cell: the traces of its polynomial on its faces (shared memory), the WENO
//      sensor from the four face neighbours (Sec. 4), the volume term (Eq. weak2) by
//      sum factorisation, kept in registers.
//   2. Every face of the tile once: both traces at the p+2 Gauss points, the local
//      Lax-Friedrichs flux (Sec. 2), lifted onto the face Legendre modes.
//   3. Per cell: face contributions, the stabilization gamma nu K c (Sec. 3), M^{-1}
//      and the SSP-RK3 combination Uout = cn Un + ck Uk + cl L(Uk) (Eq. ssp).
// Constant factors are folded so that, in the reference element,
//   L_k = (2/h) minv(k) [acc_k - gamma lambda / p (K_ref c)_k].
#include <cmath>
#include <cstdint>
#include <cstring>

#include "dgw_internal.h"
#include "dgw_math.cuh"

namespace dgw {
namespace DGW_NS {

using Real = DGW_REAL;
constexpr int DIM = DGW_DIM;
constexpr bool kF32 = sizeof(Real) == 4;

// tile: 128 threads, one cell each
constexpr int TX = DIM == 1 ? 128 : kTileX2;
constexpr int TY = DIM == 1 ? 1 : kTileY2;
constexpr int NT = TX * TY;
constexpr int HX = TX + 8;                 // staged columns: tile at [OX, OX+TX), halo OX-1, OX+TX
constexpr int OX = 4;
constexpr int HY = DIM == 1 ? 1 : TY + 2;  // staged rows
constexpr int OY = DIM == 1 ? 0 : 1;       // row offset of the tile inside the stage
static_assert(DIM == 1 || (HX == kBoxX2 && HY == kBoxY2), "TMA box and stage layout disagree");

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
struct alignas(64) KParams {
    CUtensorMap tmap;    // TMA descriptor of Uk (valid when use_tma)
    CUtensorMap tmap_un; // TMA descriptor of Un, tile box (valid when use_tma_un)
    int use_tma;
    int use_tma_un;
    int cg_loads;        // load Uk / Un through L2 only (data written earlier in the same launch)
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

// Bounded wait for the completion of the given phase parity of an mbarrier; false if
// it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 22); ++it) {
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

// Shared memory of one tile (carved from dynamic shared memory).
template <int P>
struct TileSmem {
    static constexpr int N1 = P + 1, K = Tab<P>::K, TN = DIM == 1 ? 1 : N1;
    alignas(128) Real su[K][HY][HX];
    // cell index innermost: a warp touches consecutive words (no bank conflicts)
    Real trx[TY][2][TN][TX + 2];                          // x-traces, col = lx + 1
    Real trys[DIM == 2 ? TY + 2 : 1][2][TN][TX];          // y-traces, row = ly + 1
    Real hfx[TY][TN][TX + 1];
    Real hfy[DIM == 2 ? TY + 1 : 1][TN][TX];
    Real lam_s[TY][TX];
    alignas(8) uint64_t mbar;
    int fail_s;
};

// One tile of one stage.  Called by all NT threads of a CTA together (it contains
// CTA barriers); tx0, ty0: first cell of the tile.  MODE 0: stage / residual;
// MODE 1: sensor only.
template <int P, int FLUX, int MODE>
__device__ __forceinline__ void process_tile(const KParams& A, const int tx0, const int ty0, TileSmem<P>& S)
{
    constexpr int N1 = P + 1, NQ = P + 2;
    constexpr int K = Tab<P>::K;
    constexpr int NFX = (TX + 1) * TY;                 // x-faces of the tile
    constexpr int NFY = DIM == 2 ? TX * (TY + 1) : 0;  // y-faces
    constexpr int TN = DIM == 1 ? 1 : N1;              // trace / face coefficients
    const Tab<P>& T = tab<P>();
    auto& su = S.su;
    auto& trx = S.trx;
    auto& trys = S.trys;
    auto& hfx = S.hfx;
    auto& hfy = S.hfy;
    auto& lam_s = S.lam_s;
    auto& mbar = S.mbar;
    auto& fail_s = S.fail_s;

    const int tid = threadIdx.x;
    const int64_t E = A.E;
    const bool need_lam = (MODE == 0) && (A.stab != STAB_DG) && !A.lam_fixed;
    const bool periodic_x = A.bc[0] == BC_PERIODIC;
    const bool periodic_y = DIM == 2 && A.bc[2] == BC_PERIODIC;

    // ---- 0. stage the tile and its face halo ----
    if (DIM == 2 && A.use_tma) {
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&mbar);
        if (tid == 0) {
            fail_s = 0;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (tid == 0) {
            const uint32_t bytes = (uint32_t)(sizeof(Real) * K * HY * HX);
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
        if (!mbar_wait(bar, 0)) fail_s = 1;
        __syncthreads();
        if (fail_s) {
            if (tid == 0) atomicOr(A.flag, 2u);
            return;
        }
        // periodic images of halo cells that lie outside the box's wrap-free view
        const bool edge = (periodic_x && (tx0 == 0 || tx0 + TX >= A.nx)) ||
                          (periodic_y && (ty0 == 0 || ty0 + TY >= A.ny));
        if (edge) {
            for (int idx = tid; idx < K * HY * HX; idx += NT) {
                const int k = idx / (HY * HX);
                const int rem = idx - k * (HY * HX);
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
        for (int idx = tid; idx < HY * HX; idx += NT) {
            const int r = idx / HX, cc = idx - r * HX;
            if (cc < OX - 1 || cc > OX + TX) continue;
            const bool corner = DIM == 2 && (r == 0 || r == HY - 1) && (cc == OX - 1 || cc == OX + TX);
            if (corner) continue;
            const int gx = wrap_x(A, tx0 - OX + cc);
            const int gy = DIM == 2 ? wrap_y(A, ty0 - OY + r) : 0;
            if (gx < 0 || gy < 0) continue;
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
    const int gx = tx0 + lx, gy = ty0 + ly;
    const bool in_domain = gx < A.nx && (DIM == 1 || gy < A.ny);
    const int sr = ly + OY, sc = lx + OX;

    Real c[K];
#pragma unroll
    for (int k = 0; k < K; ++k) c[k] = su[k][sr][sc];

    // ---- 1a. traces of this cell's slot (also for slots that hold periodic images) ----
    if (MODE == 0) {
#pragma unroll
        for (int t = 0; t < TN; ++t) {
            Real xm = Real(0), xp = Real(0), ym = Real(0), yp = Real(0);
#pragma unroll
            for (int n = 0; n < N1; ++n) {
                const Real kx = DIM == 1 ? c[n] : c[n + N1 * t];
                xp += kx;
                xm += (n & 1) ? -kx : kx;
                if (DIM == 2) {
                    const Real ky = c[t + N1 * n];
                    yp += ky;
                    ym += (n & 1) ? -ky : ky;
                }
            }
            trx[ly][0][t][lx + 1] = xm;
            trx[ly][1][t][lx + 1] = xp;
            if (DIM == 2) {
                trys[ly + 1][0][t][lx] = ym;
                trys[ly + 1][1][t][lx] = yp;
            }
        }
        // halo cells: the one trace that faces the tile
        constexpr int NH = 2 * TY + (DIM == 2 ? 2 * TX : 0);
        for (int hidx = tid; hidx < NH; hidx += NT) {
            int r, cc, side, axis;
            if (hidx < TY) { r = hidx + OY; cc = OX - 1; axis = 0; side = 1; }
            else if (hidx < 2 * TY) { r = hidx - TY + OY; cc = OX + TX; axis = 0; side = 0; }
            else if (hidx < 2 * TY + TX) { r = 0; cc = OX + hidx - 2 * TY; axis = 1; side = 1; }
            else { r = HY - 1; cc = OX + hidx - 2 * TY - TX; axis = 1; side = 0; }
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
                else trys[r == 0 ? 0 : TY + 1][side][t][cc - OX] = v;
            }
        }
        if (need_lam) lam_s[ly][lx] = Real(0);
    }

    // ---- 1b. sensor (Sec. 4): Hermite candidates of the face neighbours ----
    Real gamma = (MODE == 0 && A.stab == STAB_LO) ? Real(1) : Real(0);
    if ((MODE == 1 || A.stab == STAB_WENO) && in_domain) {
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
            Real cn[K];
#pragma unroll
            for (int k = 0; k < K; ++k) cn[k] = su[k][nr][nc];
            Real cl[K];
#pragma unroll
            for (int k = 1; k < K; ++k) {
                const int i = k % N1, j = k / N1;
                const int a = axis == 0 ? i : j;
                Real sacc = Real(0);
#pragma unroll
                for (int m = 0; m < N1; ++m) {
                    if (m < a) continue;   // P_m(xi +- 2) has degree m
                    const int km = axis == 0 ? m + N1 * j : i + N1 * m;
                    sacc = fma(T.T[side][a][m], cn[km], sacc);
                }
                cl[k] = sacc;
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
        if (MODE == 1) A.gamma_out[(int64_t)gy * A.nx + gx] = (double)gamma;
    }
    if (MODE == 1) return;

    // ---- 1c. volume term (Eq. weak2): acc_ij = sum_q W_q [D_i B_j Fx + B_i D_j Fy] ----
    Real acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = Real(0);
    Real lam = Real(0);
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
                Real sacc = Real(0);
#pragma unroll
                for (int i = 0; i < N1; ++i) sacc = fma(c[i + N1 * j], T.B[qx][i], sacc);
                tmp[j][qx] = sacc;
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
    __syncthreads();

    // The stage array is no longer read: bring the Un tile into it now, so that its
    // load overlaps the face phase (second phase of the same mbarrier).
    const bool un_tma = DIM == 2 && A.use_tma && A.use_tma_un && A.has_un;
    if (un_tma && tid == 0) {
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&mbar);
        const uint32_t bytes = (uint32_t)(sizeof(Real) * K * TY * TX);
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
    for (int f = tid; f < NFX + NFY; f += NT) {
        const bool xf = f < NFX;
        int flx, fly;              // tile position of the cell on the plus side of the face
        if (xf) { fly = f / (TX + 1); flx = f - fly * (TX + 1); }
        else { const int g = f - NFX; fly = g / TX; flx = g - fly * TX; }
        const int fgx = tx0 + flx, fgy = ty0 + fly;   // plus-side cell (global, unwrapped)
        if (xf) { if (fgx > A.nx || fgy >= A.ny) continue; }
        else { if (fgy > A.ny || fgx >= A.nx) continue; }
        const int axis = xf ? 0 : 1;
        const bool minus_in = xf ? (fgx - 1 >= 0 || periodic_x) : (fgy - 1 >= 0 || periodic_y);
        const bool plus_in = xf ? (fgx < A.nx || periodic_x) : (fgy < A.ny || periodic_y);
        Real tm[TN], tp[TN];
#pragma unroll
        for (int t = 0; t < TN; ++t) {
            if (xf) { tm[t] = trx[fly][1][t][flx]; tp[t] = trx[fly][0][t][flx + 1]; }
            else { tm[t] = trys[DIM == 2 ? fly : 0][1][t][flx]; tp[t] = trys[DIM == 2 ? fly + 1 : 0][0][t][flx]; }
        }
        Real hq[TN];
#pragma unroll
        for (int t = 0; t < TN; ++t) hq[t] = Real(0);
        Real lm = Real(0), lp = Real(0);
        constexpr int NFQ = DIM == 1 ? 1 : NQ;
#pragma unroll
        for (int q = 0; q < NFQ; ++q) {
            Real uL = Real(0), uR = Real(0);
            if (DIM == 1) { uL = tm[0]; uR = tp[0]; }
            else {
#pragma unroll
                for (int t = 0; t < TN; ++t) { uL = fma(tm[t], T.B[q][t], uL); uR = fma(tp[t], T.B[q][t], uR); }
            }
            Real x = Real(0), y = Real(0);
            if (FLUX == FLUX_ROTATION || need_lam || !minus_in || !plus_in) {
                if (xf) { x = A.x0 + Real(fgx) * A.h; y = DIM == 2 ? A.y0 + (Real(fgy) + Real(0.5)) * A.h + A.hh * T.g[q] : Real(0); }
                else { x = A.x0 + (Real(fgx) + Real(0.5)) * A.h + A.hh * T.g[q]; y = A.y0 + Real(fgy) * A.h; }
            }
            if (!minus_in) {
                // ghost for the plus cell, whose outward normal is -e_axis
                const int bside = xf ? 0 : 2;
                uL = (A.bc[bside] == BC_INFLOW_ZERO && -dflux_axis<FLUX>(A, axis, uR, x, y) < Real(0)) ? Real(0) : uR;
            } else if (!plus_in) {
                const int bside = xf ? 1 : 3;
                uR = (A.bc[bside] == BC_INFLOW_ZERO && dflux_axis<FLUX>(A, axis, uL, x, y) < Real(0)) ? Real(0) : uL;
            }
            if (need_lam) {
                lm = fmax(lm, speed_norm<FLUX>(A, uL, x, y));
                lp = fmax(lp, speed_norm<FLUX>(A, uR, x, y));
            }
            const Real H = llf<FLUX>(A, axis, uL, uR, x, y) * (DIM == 1 ? Real(1) : T.w[q]);
#pragma unroll
            for (int t = 0; t < TN; ++t) hq[t] = fma(DIM == 1 ? Real(1) : T.B[q][t], H, hq[t]);
        }
        if (xf) {
#pragma unroll
            for (int t = 0; t < TN; ++t) hfx[fly][t][flx] = hq[t];
        } else {
#pragma unroll
            for (int t = 0; t < TN; ++t) hfy[DIM == 2 ? fly : 0][t][flx] = hq[t];
        }
        if (need_lam) {
            // only traces of this tile's cells that lie in the domain count
            const int mlx = xf ? flx - 1 : flx, mly = xf ? fly : fly - 1;
            if (minus_in && mlx >= 0 && mly >= 0 && (xf ? fgx - 1 < A.nx : fgy - 1 < A.ny))
                atomic_max_nonneg(&lam_s[mly][mlx], lm);
            if (plus_in && flx < TX && fly < TY && fgx < A.nx && fgy < A.ny)
                atomic_max_nonneg(&lam_s[fly][flx], lp);
        }
    }
    __syncthreads();
    if (!in_domain) return;
    const int64_t e = (int64_t)gy * A.nx + gx;

    // ---- 3. faces: -phi_k(+1) H on the plus faces, +phi_k(-1) H on the minus faces ----
    if (DIM == 1) {
        const Real hm = hfx[0][0][lx], hp = hfx[0][0][lx + 1];
#pragma unroll
        for (int n = 0; n < N1; ++n) acc[n] += ((n & 1) ? -hm : hm) - hp;
    } else {
#pragma unroll
        for (int t = 0; t < N1; ++t) {
            const Real xm = hfx[ly][t][lx], xp = hfx[ly][t][lx + 1];
            const Real ym = hfy[DIM == 2 ? ly : 0][t][lx], yp = hfy[DIM == 2 ? ly + 1 : 0][t][lx];
#pragma unroll
            for (int n = 0; n < N1; ++n) {
                acc[n + N1 * t] += ((n & 1) ? -xm : xm) - xp;
                acc[t + N1 * n] += ((n & 1) ? -ym : ym) - yp;
            }
        }
    }
    if (need_lam) lam = fmax(lam, lam_s[ly][lx]);

    // stabilization (Sec. 3), M^{-1}, RK combination (Eq. ssp)
    const Real lamv = A.lam_fixed ? A.lambda_nu : lam;
    const Real gs = gamma * lamv / Real(P);   // gamma nu (2/h)
    Real chk = Real(0);                        // becomes NaN if any output is not finite
    const Real* __restrict__ un = A.Un + e;
    const Real* sun = reinterpret_cast<const Real*>(&su[0][0][0]);   // Un tile [K][TY][TX]
    if (un_tma && !mbar_wait((uint32_t)__cvta_generic_to_shared(&mbar), 1)) {
        atomicOr(A.flag, 2u);
        return;
    }
    Real* __restrict__ uo = A.Uout + e;
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
        if (A.has_un) {
            const Real unk = un_tma ? sun[(k * TY + ly) * TX + lx] : (A.cg_loads ? __ldcg(un + k * E) : un[k * E]);
            out += A.cn * unk;
        }
        chk = fma(out, Real(0), chk);
        uo[k * E] = out;
    }
    if (chk != chk) atomicOr(A.flag, 1u);
}

template <int P, int FLUX, int MODE>
__global__ void __launch_bounds__(NT, kF32 ? 6 : 3) stage_kernel(const __grid_constant__ KParams A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if ((__cvta_generic_to_shared(smem_raw) & 127u) != 0) {   // TMA needs an aligned box
        if (threadIdx.x == 0) atomicOr(A.flag, 2u);
        return;
    }
    TileSmem<P>& S = *reinterpret_cast<TileSmem<P>*>(smem_raw);
    process_tile<P, FLUX, MODE>(A, blockIdx.x * TX, DIM == 2 ? blockIdx.y * TY : 0, S);
}

static KParams make_params(const StageArgs& s)
{
    KParams a;
    memset(&a, 0, sizeof a);
    a.use_tma = 0;
    a.use_tma_un = 0;
    a.cg_loads = 0;
    if (s.tmap) {
        a.tmap = *s.tmap;
        a.use_tma = 1;
    }
    if (s.tmap_un) {
        a.tmap_un = *s.tmap_un;
        a.use_tma_un = 1;
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
    a.cn = (Real)s.cn; a.ck = (Real)s.ck; a.cl = (Real)s.cl;
    return a;
}

// ------------------------------------------------------------------------------------
// batched ensemble: persistent kernel
// ------------------------------------------------------------------------------------
template <int P, int FLUX>
__device__ __forceinline__ void batch_tiles(const BatchArgs& B, const BatchInst& I, const int r,
                                            const int tile0, const int ntile, unsigned char* smem)
{
    KParams A;
    A.use_tma = 0;
    A.use_tma_un = 0;
    A.cg_loads = 1;
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
    const double dt = I.dt;
    A.cn = (Real)(r == 0 ? 0.0 : (r == 1 ? 0.75 : 1.0 / 3.0));
    A.ck = (Real)(r == 0 ? 1.0 : (r == 1 ? 0.25 : 2.0 / 3.0));
    A.cl = (Real)(r == 0 ? dt : (r == 1 ? 0.25 * dt : 2.0 / 3.0 * dt));
    TileSmem<P>& S = *reinterpret_cast<TileSmem<P>*>(smem);
    for (int t = tile0; t < tile0 + ntile; ++t) {
        const int tx0 = (t % I.ntx) * TX;
        const int ty0 = DIM == 2 ? (t / I.ntx) * TY : 0;
        process_tile<P, FLUX, 0>(A, tx0, ty0, S);
        __syncthreads();
    }
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Persistent kernel over all work items of all stages: items are dequeued in order,
// so every item an item waits for was dequeued earlier by a resident CTA (the launch is
// cooperative, hence all CTAs are resident) and no wait can deadlock; each wait is
// still bounded, and a wait that gives up stops the whole launch through B.abort.
constexpr size_t kTileSmemMax = sizeof(TileSmem<3>) > sizeof(TileSmem<2>) ? sizeof(TileSmem<3>) : sizeof(TileSmem<2>);
constexpr size_t kBatchSmem = (kTileSmemMax + 127) / 128 * 128 + 128;   // tile + scheduler words

__global__ void __launch_bounds__(NT, kF32 ? 6 : 3) batch_kernel(const BatchArgs B)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    long long& s_w = *reinterpret_cast<long long*>(smem_raw + kBatchSmem - 128);
    int& s_ok = *reinterpret_cast<int*>(smem_raw + kBatchSmem - 64);
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
        switch (I.p * 8 + I.flux) {
        case 1 * 8 + FLUX_ADVECT: batch_tiles<1, FLUX_ADVECT>(B, I, r, it.tile0, it.ntile, smem_raw); break;
        case 2 * 8 + FLUX_ADVECT: batch_tiles<2, FLUX_ADVECT>(B, I, r, it.tile0, it.ntile, smem_raw); break;
        case 3 * 8 + FLUX_ADVECT: batch_tiles<3, FLUX_ADVECT>(B, I, r, it.tile0, it.ntile, smem_raw); break;
        case 1 * 8 + FLUX_BURGERS: batch_tiles<1, FLUX_BURGERS>(B, I, r, it.tile0, it.ntile, smem_raw); break;
        case 2 * 8 + FLUX_BURGERS: batch_tiles<2, FLUX_BURGERS>(B, I, r, it.tile0, it.ntile, smem_raw); break;
        case 3 * 8 + FLUX_BURGERS: batch_tiles<3, FLUX_BURGERS>(B, I, r, it.tile0, it.ntile, smem_raw); break;
        default: break;
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(&B.done[it.inst], (unsigned long long)it.ntile);
    }
}

static int batch_blocks_per_sm()
{
    if (kBatchSmem > 48 * 1024 &&
        cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel, NT, kBatchSmem) != cudaSuccess) return 0;
    return n;
}

static cudaError_t launch_batch(const BatchArgs& a, int grid, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = kBatchSmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_kernel, a);
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

template <int P, int FLUX>
static cudaError_t launch_pf(const StageArgs& s, int mode, cudaStream_t st)
{
    const KParams a = make_params(s);
    dim3 grid((s.nx + TX - 1) / TX, DIM == 2 ? (s.ny + TY - 1) / TY : 1);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    const size_t smem = sizeof(TileSmem<P>);
    if (smem > 48 * 1024) {
        // opt in once per instantiation to more than 48 KB of dynamic shared memory
        static bool opted[2] = {false, false};
        if (!opted[mode]) {
            cudaError_t e = mode == 0
                ? cudaFuncSetAttribute(stage_kernel<P, FLUX, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                : cudaFuncSetAttribute(stage_kernel<P, FLUX, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            opted[mode] = true;
        }
    }
    if (mode == 0) stage_kernel<P, FLUX, 0><<<grid, NT, smem, st>>>(a);
    else stage_kernel<P, FLUX, 1><<<grid, NT, smem, st>>>(a);
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
