/*
 * dgw_oracle.c -- plain, slow, FP64 CPU oracle for the WENO-stabilized RKDG method
 * of Vedral, "Dissipative WENO stabilization of high-order discontinuous Galerkin
 * methods for hyperbolic problems" (arXiv 2309.12019).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this
 * file: only the tests, the smoke check and the CPU-baseline leg of the benchmark use
 * it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Everything is written from the definitions, element by element, in physical
 * coordinates, with Gauss-Legendre quadrature and Legendre polynomials built from
 * their three-term recurrence.  No sum factorisation, no precomputed operator
 * matrices, no fusion.  Section / equation references are to the paper:
 *
 *   Sec. 2, Eq. (fesol)   modal expansion U_h^e = sum_j U_j phi_j (Legendre basis here;
 *                          the paper notes the method does not depend on the basis)
 *   Sec. 2, Eq. (weak2)   M dU/dt = R(U): volume term  int grad(phi_i).F(U_h)
 *                          minus face term int phi_i H(U-,U+,n)
 *   Sec. 2                local Lax-Friedrichs flux H_LLF with the exact maximal
 *                          wave speed s+ = max_{w in [0,1]} |F'(w U- + (1-w) U+).n|
 *   Sec. 2, Eq. (ssp)     optimal three-stage third-order SSP Runge-Kutta
 *   Sec. 3, Eq. (lostab)  low-order stabilization  nu_e int grad(phi_i).grad(U_h)
 *   Sec. 3, Eq. (visc)    nu_e = lambda_e h_e / (2p), lambda_e = ||F'(U_h)||_inf on K_e
 *   Sec. 3, Eq. (astab)   adaptive stabilization  gamma_e nu_e int grad(phi_i).grad(U_h)
 *   Sec. 4, Eq. (sensor)  gamma_e = min(1, ||U - U*||_e / ||U||_e)^q
 *   Sec. 4                scaled Sobolev seminorm sum_{1<=|k|<=p} h^{2|k|-d} int |D^k v|^2
 *   Sec. 4, Eq. (gensensor) thresholded sensor (gamma = 0 when the ratio is below b)
 *   Sec. 4                HWENO reconstruction U* = sum_l w_l U_{h,l}
 *   Sec. 5 (setup)        q = 1, linear weights 1 - m_e*0.01 (own cell), 0.01 (neighbours)
 *
 * Readings where the paper is silent (it defers the HWENO construction to another
 * paper that is not reproduced in it):
 *   R1 candidates: for every face neighbour K_l that exists, U_{h,l}^e is the
 *      neighbour's polynomial continued analytically into K_e, with its mean over K_e
 *      replaced by the mean of U_h^e (Hermite data: cell average of K_e, all derivatives
 *      of K_l).  U_{h,0}^e = U_h^e.  Missing neighbours (non-periodic boundary) are
 *      left out, so m_e shrinks.
 *   R2 U* lives in V_p(K_e) (Q_p on quadrilaterals).
 *   R3 nonlinear weights w_l = wt_l / sum_m wt_m, wt_l = lin_l / (eps_w + beta_l)^2 with
 *      beta_l = ||U_{h,l}^e||_e^2 (the same seminorm).
 *   R4 the seminorm sums over all multi-indices 1 <= |k| <= p, mixed ones included.
 *   R5 guard: numerator <= eps_s gives gamma = 0; otherwise a zero denominator gives
 *      gamma = 1; otherwise gamma = min(1, r)^q, and gamma = 0 if r < b.  The remark of
 *      Sec. 4 switches the sensor off below a prescribed tolerance; its value is the b of
 *      Eq. (gensensor).  The scalar problems use b = 0.1, one of the two values Sec. 5.6
 *      names: it reproduces the WENO columns of Tables 1-2 (equal to DG at p = 2, 3, and
 *      at p = 1 from 256 cells), which b = 0 does not (the sensor then falls only like
 *      h^p on smooth data and the error stays several times DG's).  The Euler runs of
 *      Sec. 5.6 use gamma_e itself (b = 0) and compare b = 0.1, 0.2 as a variant.  The
 *      caller passes b; this file has no default.
 *   R6 gamma is recomputed from the state each residual evaluation (every RK stage).
 *   R7 lambda_e = max |F'(U_h)|_2 over the element's volume and face Gauss points
 *      (unless a fixed value is given, as the paper does for the KPP problem).
 *   R8 boundary ghosts: periodic wrap; inflow-zero sets U+ = 0 where F'(U-).n < 0 and
 *      U+ = U- elsewhere; outflow sets U+ = U-.
 *   R15 Euler system (1D, Sec. 5.6): U = (rho, rho v, rho E), p = (gamma - 1)(rho E -
 *      rho v^2 / 2), F = (rho v, rho v^2 + p, (rho E + p) v); state layout
 *      U[(comp (p+1) + k) E + e].  s+ of the LLF flux is read as the larger of |v| + c at
 *      the two states (the maximum along the path in conservative variables has no
 *      closed form); lambda_e = max (|v| + c) over the element's volume and face points.
 *      A state without a real sound speed (rho <= 0 or p < 0) has no wave speed: s+ and
 *      lambda_e are then NaN, so that the step returns non-finite values rather than
 *      finite ones built on an undefined speed.
 *      Reflecting walls mirror the state: (rho, -rho v, rho E).  The sensor uses the
 *      density alone, applied to all components; beyond a wall, as beyond any
 *      non-periodic boundary, there is no neighbour candidate.
 *   R17 Euler system in 2D (Sec. 5.6, its 2D problems): U = (rho, rho vx, rho vy, rho E),
 *      F(U) n = (rho v.n, rho v (v.n) + p n, (rho E + p) v.n); layout
 *      U[(comp (p+1)^2 + k) E + e].  LLF at each face Gauss point with s+ the larger
 *      |v.n| + c of the two states; lambda_e = max (|v| + c) over the volume Gauss points
 *      and the element's own values at the face Gauss points.  A reflecting wall mirrors
 *      the normal momentum: m+ = m- - 2 (m-.n) n.  Stabilization and sensor as in R15.
 *   R19 prescribed boundary states (Euler system, the double Mach reflection of Sec. 5.6):
 *      a side of kind ORC_BC_STATE takes, at each face point, the ghost bstate[0] or
 *      bstate[1] or a reflecting wall, by whether the point's coordinate along the side
 *      lies below bsplit + bspeed t or not (t the time of the evaluation).  The SSP-RK
 *      steps evaluate stage residuals at their stage times: t, t + dt, t + dt / 2 (order 3),
 *      t, t + dt (order 2); order 4 holds every stage at the step's start time.
 *   R13 the comparison sensor of Zhao et al. (restated in Sec. 5.6), stab = ZHAO:
 *      gamma^Z = sum_l |w_l / lin_l - 1|^theta / (|1 / min_l lin_l - 1|^theta + m_e) with
 *      the weights of R3; with no neighbour candidate (m_e = 0) the weights are the linear
 *      ones and gamma^Z = 0.  It replaces gamma_e in Eq. (astab); q and b do not apply.
 *
 * Mode ordering: k = i + (p+1)*j, i the Legendre degree along x, j along y (1D: k = i).
 * State layout: U[k*E + e], element e = iy*nx + ix.
 *
 * Build: gcc -O2 -std=c11 -fPIC -shared -ffp-contract=off [-fopenmp].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXP 3
#define ORC_MAXK ((ORC_MAXP + 1) * (ORC_MAXP + 1))
#define ORC_MAXNQ 32

enum { ORC_BC_PERIODIC = 0, ORC_BC_INFLOW_ZERO = 1, ORC_BC_OUTFLOW = 2, ORC_BC_REFLECT = 3, ORC_BC_STATE = 4 };
enum { ORC_FLUX_ADVECT = 0, ORC_FLUX_ROTATION = 1, ORC_FLUX_BURGERS = 2, ORC_FLUX_KPP = 3, ORC_FLUX_EULER = 4 };
enum { ORC_STAB_DG = 0, ORC_STAB_LO = 1, ORC_STAB_WENO = 2, ORC_STAB_ZHAO = 3 };

typedef struct {
    int dim, nx, ny, p;
    double x0, x1, y0, y1;
    int bc[4];               /* faces -x, +x, -y, +y */
    int flux;
    double a[2];             /* advection velocity / Burgers direction */
    double center[2];        /* rotation centre */
    double omega;            /* rotation rate: v = omega*(cy - y, x - cx) */
    double lambda_nu;        /* > 0: fixed lambda_e for nu_e */
    int stab;
    double q, b, w_nbr, eps_w, eps_s;
    double theta;            /* exponent of the Zhao et al. sensor (stab = ZHAO) */
    double gas_gamma;        /* ratio of heat capacities (Euler) */
    double t;                /* time of the evaluation (prescribed boundary states, R19) */
    double bstate[2][4];     /* the two prescribed conservative states of ORC_BC_STATE sides */
    double bsplit[4];        /* per side: position along the side where its ghost changes, t = 0 */
    double bspeed[4];        /* per side: speed of that position */
    int bbelow[4], babove[4];/* per side, below / from the split: 0, 1 = bstate[0], [1]; 2 = wall */
} orc_problem;

/* ------------------------------------------------------------------------- */
/* Legendre polynomials                                                       */
/* ------------------------------------------------------------------------- */

/* P_n(x) by the three-term recurrence (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1}. */
static double leg(int n, double x)
{
    if (n == 0) return 1.0;
    double pm = 1.0, pc = x;
    for (int k = 1; k < n; ++k) {
        double pn = ((2.0 * k + 1.0) * x * pc - k * pm) / (k + 1.0);
        pm = pc;
        pc = pn;
    }
    return pc;
}

#define ORC_MAXDEG 8

/* Monomial coefficients of P_n (n <= ORC_MAXDEG), from the same recurrence applied to
 * coefficient arrays: mono[n][m] is the coefficient of x^m. */
static double g_mono[ORC_MAXDEG + 1][ORC_MAXDEG + 1];

static void build_monomials(void)
{
    memset(g_mono, 0, sizeof g_mono);
    g_mono[0][0] = 1.0;
    g_mono[1][1] = 1.0;
    for (int k = 1; k < ORC_MAXDEG; ++k) {
        for (int m = 0; m <= k; ++m) g_mono[k + 1][m + 1] += (2.0 * k + 1.0) * g_mono[k][m] / (k + 1.0);
        for (int m = 0; m <= k - 1; ++m) g_mono[k + 1][m] -= k * g_mono[k - 1][m] / (k + 1.0);
    }
}

/* a-th derivative of P_n at x: differentiate the monomial form a times, then Horner. */
static double leg_d(int n, int a, double x)
{
    if (a == 0) return leg(n, x);
    if (a > n) return 0.0;
    double c[ORC_MAXDEG + 1];
    for (int m = 0; m <= n; ++m) c[m] = g_mono[n][m];
    for (int t = 0; t < a; ++t)
        for (int m = 0; m <= n; ++m) c[m] = (m + 1 <= n) ? (m + 1) * c[m + 1] : 0.0;
    double s = 0.0;
    for (int m = n - a; m >= 0; --m) s = s * x + c[m];
    return s;
}

/* Gauss-Legendre rule on [-1,1]: Newton iteration on P_n from the Chebyshev guess. */
static void gauss_legendre_newton(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = leg(n, z), p1 = leg(n - 1, z);
            double dp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = leg(n, z), p1 = leg(n - 1, z);
        double dp = n * (z * p0 - p1) / (z * z - 1.0);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static int g_threads = 1;   /* OpenMP threads of the element loops */

/* Rules for n = 1..ORC_MAXNQ, computed once. */
static double g_gx[ORC_MAXNQ + 1][ORC_MAXNQ], g_gw[ORC_MAXNQ + 1][ORC_MAXNQ];
static int g_ready = 0;

static void orc_init(void)
{
    if (g_ready) return;
    build_monomials();
    for (int n = 1; n <= ORC_MAXNQ; ++n) gauss_legendre_newton(n, g_gx[n], g_gw[n]);
    g_ready = 1;
}

void orc_gauss_legendre(int n, double* x, double* w)
{
    orc_init();
    for (int i = 0; i < n; ++i) { x[i] = g_gx[n][i]; w[i] = g_gw[n][i]; }
}

/* ------------------------------------------------------------------------- */
/* Geometry and basis                                                         */
/* ------------------------------------------------------------------------- */

static int nmodes1(const orc_problem* P) { return P->p + 1; }
static int nmodes(const orc_problem* P) { return P->dim == 1 ? P->p + 1 : (P->p + 1) * (P->p + 1); }
static long nelem(const orc_problem* P) { return P->dim == 1 ? (long)P->nx : (long)P->nx * P->ny; }
static int ncomp(const orc_problem* P) { return P->flux == ORC_FLUX_EULER ? P->dim + 2 : 1; }
static long nstate(const orc_problem* P) { return nelem(P) * nmodes(P) * ncomp(P); }
static double hx_of(const orc_problem* P) { return (P->x1 - P->x0) / P->nx; }
static double hy_of(const orc_problem* P) { return P->dim == 1 ? 1.0 : (P->y1 - P->y0) / P->ny; }

static void elem_center(const orc_problem* P, long e, double* xc, double* yc)
{
    int ix = (int)(e % P->nx), iy = (int)(e / P->nx);
    *xc = P->x0 + (ix + 0.5) * hx_of(P);
    *yc = P->dim == 1 ? 0.0 : P->y0 + (iy + 0.5) * hy_of(P);
}

/* Physical derivative D^(kx,ky) of the basis function phi_k of an element, at the point
 * whose coordinates in that element's reference frame are (xi, eta), i.e.
 * x = x_e + h/2 xi (Eq. fesol: U_h^e is a polynomial on K_e).  Points outside [-1,1]^d
 * give the analytic continuation (used for the Hermite candidates).  Working in the
 * element's own frame keeps the Gauss nodes exact instead of recovering xi from x. */
static double phi_d(const orc_problem* P, int k, int kx, int ky, double xi, double eta)
{
    int n1 = nmodes1(P);
    int i = k % n1, j = k / n1;
    double v = leg_d(i, kx, xi) * pow(2.0 / hx_of(P), kx);
    if (P->dim == 2) v *= leg_d(j, ky, eta) * pow(2.0 / hy_of(P), ky);
    return v;
}

/* Physical derivative D^(kx,ky) of sum_k c_k phi_k at reference point (xi, eta). */
static double poly_d(const orc_problem* P, const double* c, int kx, int ky, double xi, double eta)
{
    double s = 0.0;
    for (int k = 0; k < nmodes(P); ++k) s += c[k] * phi_d(P, k, kx, ky, xi, eta);
    return s;
}

static void load_elem(const orc_problem* P, const double* U, long e, double* c)
{
    long E = nelem(P);
    for (int k = 0; k < nmodes(P); ++k) c[k] = U[k * E + e];
}

/* Quadrature over element e with nq points per direction: physical points (qx, qy),
 * the same points in the element's reference frame (qr, qs), and weights including
 * the Jacobian.  Returns the point count. */
static int elem_quad(const orc_problem* P, long e, int nq, double* qx, double* qy,
                     double* qr, double* qs, double* qw)
{
    double gx[ORC_MAXNQ], gw[ORC_MAXNQ], xc, yc;
    orc_gauss_legendre(nq, gx, gw);
    elem_center(P, e, &xc, &yc);
    double hx = hx_of(P), hy = hy_of(P);
    int n = 0;
    if (P->dim == 1) {
        for (int a = 0; a < nq; ++a) {
            qx[n] = xc + 0.5 * hx * gx[a]; qy[n] = 0.0;
            qr[n] = gx[a]; qs[n] = 0.0;
            qw[n] = gw[a] * 0.5 * hx; ++n;
        }
    } else {
        for (int b = 0; b < nq; ++b)
            for (int a = 0; a < nq; ++a) {
                qx[n] = xc + 0.5 * hx * gx[a];
                qy[n] = yc + 0.5 * hy * gx[b];
                qr[n] = gx[a]; qs[n] = gx[b];
                qw[n] = gw[a] * gw[b] * 0.25 * hx * hy;
                ++n;
            }
    }
    return n;
}

/* ------------------------------------------------------------------------- */
/* Flux functions (scalar conservation laws of the paper's scalar examples)   */
/* ------------------------------------------------------------------------- */

static void rot_velocity(const orc_problem* P, double x, double y, double v[2])
{
    v[0] = P->omega * (P->center[1] - y);
    v[1] = P->omega * (x - P->center[0]);
}

static void flux_F(const orc_problem* P, double u, double x, double y, double F[2])
{
    switch (P->flux) {
    case ORC_FLUX_ADVECT: F[0] = P->a[0] * u; F[1] = P->a[1] * u; break;
    case ORC_FLUX_ROTATION: { double v[2]; rot_velocity(P, x, y, v); F[0] = v[0] * u; F[1] = v[1] * u; } break;
    case ORC_FLUX_BURGERS: F[0] = P->a[0] * 0.5 * u * u; F[1] = P->a[1] * 0.5 * u * u; break;
    case ORC_FLUX_KPP: F[0] = sin(u); F[1] = cos(u); break;
    default: F[0] = F[1] = NAN;
    }
    if (P->dim == 1) F[1] = 0.0;
}

static void flux_dF(const orc_problem* P, double u, double x, double y, double v[2])
{
    switch (P->flux) {
    case ORC_FLUX_ADVECT: v[0] = P->a[0]; v[1] = P->a[1]; break;
    case ORC_FLUX_ROTATION: rot_velocity(P, x, y, v); break;
    case ORC_FLUX_BURGERS: v[0] = P->a[0] * u; v[1] = P->a[1] * u; break;
    case ORC_FLUX_KPP: v[0] = cos(u); v[1] = -sin(u); break;
    default: v[0] = v[1] = NAN;
    }
    if (P->dim == 1) v[1] = 0.0;
}

/* Exact s+ = max over the segment between um and up of |F'(u).n| (Sec. 2).
 * Normals are axis-aligned on the Cartesian meshes used here. */
static double wave_speed(const orc_problem* P, double um, double up, double x, double y,
                         const double n[2])
{
    double lo = um < up ? um : up, hi = um < up ? up : um;
    switch (P->flux) {
    case ORC_FLUX_ADVECT: return fabs(P->a[0] * n[0] + P->a[1] * n[1]);
    case ORC_FLUX_ROTATION: { double v[2]; rot_velocity(P, x, y, v); return fabs(v[0] * n[0] + v[1] * n[1]); }
    case ORC_FLUX_BURGERS: {
        /* F'(u).n = (a.n) u is linear in u: its modulus peaks at an endpoint. */
        double an = fabs(P->a[0] * n[0] + P->a[1] * n[1]);
        return an * (fabs(lo) > fabs(hi) ? fabs(lo) : fabs(hi));
    }
    case ORC_FLUX_KPP: {
        /* x-normal: |F'.n| = |cos u|, maximal (=1) at multiples of pi;
         * y-normal: |F'.n| = |sin u|, maximal (=1) at pi/2 + multiples of pi.
         * Between two maxima the modulus is unimodal with its minimum inside, so
         * without an interior maximum the segment maximum sits at an endpoint. */
        int xnormal = fabs(n[0]) > 0.5;
        double shift = xnormal ? 0.0 : 0.5 * M_PI;
        double kmin = ceil((lo - shift) / M_PI);
        if (kmin * M_PI + shift <= hi) return 1.0;
        double glo = xnormal ? fabs(cos(lo)) : fabs(sin(lo));
        double ghi = xnormal ? fabs(cos(hi)) : fabs(sin(hi));
        return glo > ghi ? glo : ghi;
    }
    default: return NAN;
    }
}

/* Local Lax-Friedrichs flux H(U-,U+,n) = n.(F(U-)+F(U+))/2 - s+/2 (U+ - U-) (Sec. 2). */
double orc_llf(const orc_problem* P, double um, double up, double x, double y, double nx, double ny)
{
    orc_init();
    double n[2] = {nx, ny}, Fm[2], Fp[2];
    flux_F(P, um, x, y, Fm);
    flux_F(P, up, x, y, Fp);
    double s = wave_speed(P, um, up, x, y, n);
    return 0.5 * (n[0] * (Fm[0] + Fp[0]) + n[1] * (Fm[1] + Fp[1])) - 0.5 * s * (up - um);
}

double orc_wave_speed(const orc_problem* P, double um, double up, double x, double y, double nx, double ny)
{
    orc_init();
    double n[2] = {nx, ny};
    return wave_speed(P, um, up, x, y, n);
}

/* ------------------------------------------------------------------------- */
/* Mesh connectivity                                                          */
/* ------------------------------------------------------------------------- */

/* Neighbour of e across face f (0:-x 1:+x 2:-y 3:+y), or -1 at a non-periodic
 * boundary.  *sx,*sy receive the offset of the neighbour's reference frame: a point
 * with coordinates (xi, eta) in K_e has coordinates (xi + sx, eta + sy) in the
 * neighbour, which sits next to e (periodic neighbours are placed adjacent, not at
 * their wrapped position): sx = +2 for the neighbour on the -x side. */
static long neighbour(const orc_problem* P, long e, int f, double* sx, double* sy)
{
    int ix = (int)(e % P->nx), iy = (int)(e / P->nx);
    int jx = ix, jy = iy;
    double ox = 0.0, oy = 0.0;
    if (f == 0) { jx = ix - 1; ox = 2.0; }
    if (f == 1) { jx = ix + 1; ox = -2.0; }
    if (f == 2) { jy = iy - 1; oy = 2.0; }
    if (f == 3) { jy = iy + 1; oy = -2.0; }
    if (jx < 0 || jx >= P->nx) {
        if (P->bc[f] != ORC_BC_PERIODIC) return -1;
        jx = (jx + P->nx) % P->nx;
    }
    if (P->dim == 2 && (jy < 0 || jy >= P->ny)) {
        if (P->bc[f] != ORC_BC_PERIODIC) return -1;
        jy = (jy + P->ny) % P->ny;
    }
    if (sx) *sx = ox;
    if (sy) *sy = oy;
    return (long)jy * P->nx + jx;
}

static int nfaces(const orc_problem* P) { return 2 * P->dim; }

/* Face f of element e: Gauss points (physical and in e's reference frame), weights
 * (with the face Jacobian), outward normal. */
static int face_quad(const orc_problem* P, long e, int f, int nq,
                     double* qx, double* qy, double* qr, double* qs, double* qw, double n[2])
{
    double xc, yc, gx[ORC_MAXNQ], gw[ORC_MAXNQ];
    elem_center(P, e, &xc, &yc);
    double hx = hx_of(P), hy = hy_of(P);
    n[0] = n[1] = 0.0;
    if (f == 0) n[0] = -1.0;
    if (f == 1) n[0] = 1.0;
    if (f == 2) n[1] = -1.0;
    if (f == 3) n[1] = 1.0;
    if (P->dim == 1) {
        qx[0] = xc + 0.5 * hx * n[0]; qy[0] = 0.0; qr[0] = n[0]; qs[0] = 0.0; qw[0] = 1.0;
        return 1;
    }
    orc_gauss_legendre(nq, gx, gw);
    for (int a = 0; a < nq; ++a) {
        if (f < 2) {
            qx[a] = xc + 0.5 * hx * n[0]; qy[a] = yc + 0.5 * hy * gx[a];
            qr[a] = n[0]; qs[a] = gx[a]; qw[a] = gw[a] * 0.5 * hy;
        } else {
            qx[a] = xc + 0.5 * hx * gx[a]; qy[a] = yc + 0.5 * hy * n[1];
            qr[a] = gx[a]; qs[a] = n[1]; qw[a] = gw[a] * 0.5 * hx;
        }
    }
    return nq;
}

/* ------------------------------------------------------------------------- */
/* Scaled Sobolev seminorm and WENO sensor (Sec. 4)                           */
/* ------------------------------------------------------------------------- */

/* ||v||_e^2 = sum_{1<=|k|<=p} h^{2|k|-d} int_{K_e} |D^k v|^2 dx, v = sum c_k phi_k of e. */
static double seminorm2(const orc_problem* P, long e, const double* c)
{
    double qx[ORC_MAXNQ * ORC_MAXNQ], qy[ORC_MAXNQ * ORC_MAXNQ], qw[ORC_MAXNQ * ORC_MAXNQ];
    double qr[ORC_MAXNQ * ORC_MAXNQ], qs[ORC_MAXNQ * ORC_MAXNQ];
    int nq = elem_quad(P, e, P->p + 2, qx, qy, qr, qs, qw);
    double h = hx_of(P);
    double s = 0.0;
    int kymax = P->dim == 2 ? P->p : 0;
    for (int ky = 0; ky <= kymax; ++ky)
        for (int kx = 0; kx <= P->p; ++kx) {
            int K = kx + ky;
            if (K < 1 || K > P->p) continue;
            double integral = 0.0;
            for (int t = 0; t < nq; ++t) {
                double d = poly_d(P, c, kx, ky, qr[t], qs[t]);
                integral += qw[t] * d * d;
            }
            s += pow(h, 2.0 * K - P->dim) * integral;
        }
    return s;
}

/* Hermite candidate from neighbour polynomial cn (frame offset sx,sy): its continuation
 * into K_e projected onto V_p(K_e) (exact: the integrand is a polynomial), then the
 * mode-0 coefficient (the mean over K_e) replaced by that of U_h^e. */
static void candidate(const orc_problem* P, long e, const double* ce, const double* cn,
                      double sx, double sy, double* cl)
{
    double qx[ORC_MAXNQ * ORC_MAXNQ], qy[ORC_MAXNQ * ORC_MAXNQ], qw[ORC_MAXNQ * ORC_MAXNQ];
    double qr[ORC_MAXNQ * ORC_MAXNQ], qs[ORC_MAXNQ * ORC_MAXNQ];
    int nq = elem_quad(P, e, P->p + 2, qx, qy, qr, qs, qw);
    double val[ORC_MAXNQ * ORC_MAXNQ];
    for (int t = 0; t < nq; ++t) val[t] = poly_d(P, cn, 0, 0, qr[t] + sx, qs[t] + sy);
    for (int k = 0; k < nmodes(P); ++k) {
        double num = 0.0, den = 0.0;
        for (int t = 0; t < nq; ++t) {
            double ph = phi_d(P, k, 0, 0, qr[t], qs[t]);
            num += qw[t] * ph * val[t];
            den += qw[t] * ph * ph;
        }
        cl[k] = num / den;
    }
    cl[0] = ce[0];
}

/* Sensor of element e.  Returns gamma_e; optional outputs: ratio, m_e, weights. */
static double sensor_elem(const orc_problem* P, const double* U, long e,
                          double* ratio_out, double* weights_out)
{
    int K = nmodes(P);
    double ce[ORC_MAXK], cand[5][ORC_MAXK], cn[ORC_MAXK];
    load_elem(P, U, e, ce);
    memcpy(cand[0], ce, sizeof(double) * K);
    int m = 0;
    for (int f = 0; f < nfaces(P); ++f) {
        double sx, sy;
        long nb = neighbour(P, e, f, &sx, &sy);
        if (nb < 0) continue;
        load_elem(P, U, nb, cn);
        ++m;
        candidate(P, e, ce, cn, sx, sy, cand[m]);
    }
    double lin[5], wt[5], beta[5], wsum = 0.0;
    lin[0] = 1.0 - m * P->w_nbr;
    for (int l = 1; l <= m; ++l) lin[l] = P->w_nbr;
    for (int l = 0; l <= m; ++l) {
        beta[l] = seminorm2(P, e, cand[l]);
        wt[l] = lin[l] / ((P->eps_w + beta[l]) * (P->eps_w + beta[l]));
        wsum += wt[l];
    }
    double ustar[ORC_MAXK] = {0}, diff[ORC_MAXK];
    for (int l = 0; l <= m; ++l) {
        double w = wt[l] / wsum;
        if (weights_out) weights_out[l] = w;
        for (int k = 0; k < K; ++k) ustar[k] += w * cand[l][k];
    }
    if (weights_out) for (int l = m + 1; l < 5; ++l) weights_out[l] = 0.0;
    for (int k = 0; k < K; ++k) diff[k] = ce[k] - ustar[k];
    double num = sqrt(seminorm2(P, e, diff));
    double den = sqrt(seminorm2(P, e, ce));
    double gamma, r;
    if (num <= P->eps_s) { gamma = 0.0; r = 0.0; }
    else if (den == 0.0) { gamma = 1.0; r = INFINITY; }
    else {
        r = num / den;
        gamma = pow(r < 1.0 ? r : 1.0, P->q);
        if (r < P->b) gamma = 0.0;
    }
    if (P->stab == ORC_STAB_ZHAO) {
        /* R13: deviation of the nonlinear weights from the linear ones, scaled by its
         * largest possible value (all weight on the candidate of smallest linear weight) */
        double minlin = lin[0];
        for (int l = 1; l <= m; ++l) minlin = lin[l] < minlin ? lin[l] : minlin;
        double dev = 0.0;
        for (int l = 0; l <= m; ++l) dev += pow(fabs(wt[l] / wsum / lin[l] - 1.0), P->theta);
        gamma = m == 0 ? 0.0 : dev / (pow(fabs(1.0 / minlin - 1.0), P->theta) + m);
    }
    if (ratio_out) *ratio_out = r;
    return gamma;
}

/* ------------------------------------------------------------------------- */
/* Residual  L = M^{-1} R_stab(U)  (Eq. weak2 with the stabilization of Sec. 3) */
/* ------------------------------------------------------------------------- */

/* lambda_e: fixed value, or max |F'(U_h)|_2 over the volume and face Gauss points. */
static double lambda_elem(const orc_problem* P, long e, const double* ce)
{
    if (P->lambda_nu > 0.0) return P->lambda_nu;
    double qx[ORC_MAXNQ * ORC_MAXNQ], qy[ORC_MAXNQ * ORC_MAXNQ], qw[ORC_MAXNQ * ORC_MAXNQ];
    double qr[ORC_MAXNQ * ORC_MAXNQ], qs[ORC_MAXNQ * ORC_MAXNQ];
    double v[2], n[2];
    int nq = P->p + 2;
    double lam = 0.0;
    int nv = elem_quad(P, e, nq, qx, qy, qr, qs, qw);
    for (int t = 0; t < nv; ++t) {
        flux_dF(P, poly_d(P, ce, 0, 0, qr[t], qs[t]), qx[t], qy[t], v);
        double s = sqrt(v[0] * v[0] + v[1] * v[1]);
        if (s > lam) lam = s;
    }
    for (int f = 0; f < nfaces(P); ++f) {
        int nf = face_quad(P, e, f, nq, qx, qy, qr, qs, qw, n);
        for (int t = 0; t < nf; ++t) {
            flux_dF(P, poly_d(P, ce, 0, 0, qr[t], qs[t]), qx[t], qy[t], v);
            double s = sqrt(v[0] * v[0] + v[1] * v[1]);
            if (s > lam) lam = s;
        }
    }
    return lam;
}

static void residual_elem(const orc_problem* P, const double* U, long e, double* Le,
                          double* gamma_out)
{
    int K = nmodes(P);
    int nq = P->p + 2;
    double ce[ORC_MAXK], cn[ORC_MAXK], R[ORC_MAXK] = {0};
    double qx[ORC_MAXNQ * ORC_MAXNQ], qy[ORC_MAXNQ * ORC_MAXNQ], qw[ORC_MAXNQ * ORC_MAXNQ];
    double qr[ORC_MAXNQ * ORC_MAXNQ], qs[ORC_MAXNQ * ORC_MAXNQ];
    double fx[ORC_MAXNQ], fy[ORC_MAXNQ], fr[ORC_MAXNQ], fs[ORC_MAXNQ], fw[ORC_MAXNQ];
    double F[2], n[2];
    load_elem(P, U, e, ce);

    /* volume: + int grad(phi_k) . F(U_h) dx */
    int nv = elem_quad(P, e, nq, qx, qy, qr, qs, qw);
    for (int t = 0; t < nv; ++t) {
        double u = poly_d(P, ce, 0, 0, qr[t], qs[t]);
        flux_F(P, u, qx[t], qy[t], F);
        for (int k = 0; k < K; ++k) {
            double g = phi_d(P, k, 1, 0, qr[t], qs[t]) * F[0];
            if (P->dim == 2) g += phi_d(P, k, 0, 1, qr[t], qs[t]) * F[1];
            R[k] += qw[t] * g;
        }
    }

    /* faces: - int_{dK} phi_k H(U-, U+, n) ds */
    for (int f = 0; f < nfaces(P); ++f) {
        double sx = 0.0, sy = 0.0;
        long nb = neighbour(P, e, f, &sx, &sy);
        if (nb >= 0) load_elem(P, U, nb, cn);
        int nf = face_quad(P, e, f, nq, fx, fy, fr, fs, fw, n);
        for (int t = 0; t < nf; ++t) {
            double um = poly_d(P, ce, 0, 0, fr[t], fs[t]);
            double up;
            if (nb >= 0) {
                up = poly_d(P, cn, 0, 0, fr[t] + sx, fs[t] + sy);
            } else if (P->bc[f] == ORC_BC_INFLOW_ZERO) {
                double v[2];
                flux_dF(P, um, fx[t], fy[t], v);
                up = (v[0] * n[0] + v[1] * n[1] < 0.0) ? 0.0 : um;
            } else {
                up = um;
            }
            double H = orc_llf(P, um, up, fx[t], fy[t], n[0], n[1]);
            for (int k = 0; k < K; ++k)
                R[k] -= fw[t] * phi_d(P, k, 0, 0, fr[t], fs[t]) * H;
        }
    }

    /* stabilization: - gamma_e nu_e int grad(phi_k) . grad(U_h) dx */
    double gamma = 0.0;
    if (P->stab != ORC_STAB_DG && P->p >= 1) {
        gamma = (P->stab == ORC_STAB_LO) ? 1.0 : sensor_elem(P, U, e, NULL, NULL);
        double nu = lambda_elem(P, e, ce) * hx_of(P) / (2.0 * P->p);
        for (int t = 0; t < nv; ++t) {
            double ux = poly_d(P, ce, 1, 0, qr[t], qs[t]);
            double uy = P->dim == 2 ? poly_d(P, ce, 0, 1, qr[t], qs[t]) : 0.0;
            for (int k = 0; k < K; ++k) {
                double g = phi_d(P, k, 1, 0, qr[t], qs[t]) * ux;
                if (P->dim == 2) g += phi_d(P, k, 0, 1, qr[t], qs[t]) * uy;
                R[k] -= gamma * nu * qw[t] * g;
            }
        }
    }
    if (gamma_out) *gamma_out = gamma;

    /* L = M^{-1} R with M_kk = int phi_k^2 dx (the Legendre basis is orthogonal) */
    for (int k = 0; k < K; ++k) {
        double m = 0.0;
        for (int t = 0; t < nv; ++t) {
            double ph = phi_d(P, k, 0, 0, qr[t], qs[t]);
            m += qw[t] * ph * ph;
        }
        Le[k] = R[k] / m;
    }
}

/* ------------------------------------------------------------------------- */
/* Euler system in 1D and 2D (Sec. 5.6; readings R15, R17)                    */
/* ------------------------------------------------------------------------- */

#define ORC_MAXC 4     /* conserved variables: rho, rho v (dim components), rho E */

/* velocity, pressure and sound speed squared of a conservative state */
static void euler_prim(const orc_problem* P, const double* q, double v[2], double* pr, double* c2)
{
    int d = P->dim;
    v[0] = q[1] / q[0];
    v[1] = d == 2 ? q[2] / q[0] : 0.0;
    double mv = q[1] * v[0] + (d == 2 ? q[2] * v[1] : 0.0);
    *pr = (P->gas_gamma - 1.0) * (q[d + 1] - 0.5 * mv);
    *c2 = P->gas_gamma * *pr / q[0];
}

/* F(U) n = (rho v.n, rho v (v.n) + p n, (rho E + p) v.n) */
static void euler_flux_n(const orc_problem* P, const double* q, double nx, double ny, double* F)
{
    int d = P->dim;
    double v[2], pr, c2;
    euler_prim(P, q, v, &pr, &c2);
    double vn = v[0] * nx + v[1] * ny;
    F[0] = q[0] * vn;
    F[1] = q[1] * vn + pr * nx;
    if (d == 2) F[2] = q[2] * vn + pr * ny;
    F[d + 1] = (q[d + 1] + pr) * vn;
}

/* |v.n| + c (the spectral radius of F'(U) n); |v| + c when n is NULL */
static double euler_speed(const orc_problem* P, const double* q, const double* n)
{
    double v[2], pr, c2;
    euler_prim(P, q, v, &pr, &c2);
    double vn = n ? fabs(v[0] * n[0] + v[1] * n[1]) : sqrt(v[0] * v[0] + v[1] * v[1]);
    return vn + sqrt(c2);
}

/* LLF flux across a face of outward unit normal n (R15: s+ = the larger |v.n| + c) */
static void euler_llf(const orc_problem* P, const double* um, const double* up, const double n[2], double* H)
{
    int m = P->dim + 2;
    double Fm[ORC_MAXC], Fp[ORC_MAXC];
    euler_flux_n(P, um, n[0], n[1], Fm);
    euler_flux_n(P, up, n[0], n[1], Fp);
    double sm = euler_speed(P, um, n), sp = euler_speed(P, up, n);
    double s = (isnan(sm) || isnan(sp)) ? NAN : (sm > sp ? sm : sp);
    for (int c = 0; c < m; ++c) H[c] = 0.5 * (Fm[c] + Fp[c]) - 0.5 * s * (up[c] - um[c]);
}

/* For tests: the LLF flux in 1D (normal n = +-1) and in 2D (normal (nx, ny)). */
void orc_euler_llf(const orc_problem* P, const double* um, const double* up, double n, double* H)
{
    double nn[2] = {n, 0.0};
    euler_llf(P, um, up, nn, H);
}
void orc_euler_llf2(const orc_problem* P, const double* um, const double* up, double nx, double ny, double* H)
{
    double nn[2] = {nx, ny};
    euler_llf(P, um, up, nn, H);
}

static void load_comp(const orc_problem* P, const double* U, long e, int comp, double* c)
{
    long E = nelem(P);
    int K = nmodes(P);
    for (int k = 0; k < K; ++k) c[k] = U[((long)comp * K + k) * E + e];
}

/* state at reference point (r, s) of an element with coefficients ce */
static void euler_state(const orc_problem* P, double ce[ORC_MAXC][ORC_MAXK], double r, double s, double* q)
{
    for (int c = 0; c < P->dim + 2; ++c) q[c] = poly_d(P, ce[c], 0, 0, r, s);
}

/* lambda_e of R15/R17: max (|v| + c) over the (p+2)^d volume Gauss points and the
 * element's own values at the face Gauss points (1D: the two end points); NaN if any
 * of them has no real sound speed */
static double euler_lambda_elem(const orc_problem* P, long e, double ce[ORC_MAXC][ORC_MAXK])
{
    int nq = P->p + 2;
    double qx[ORC_MAXNQ * ORC_MAXNQ], qy[ORC_MAXNQ * ORC_MAXNQ], qr[ORC_MAXNQ * ORC_MAXNQ];
    double qs[ORC_MAXNQ * ORC_MAXNQ], qw[ORC_MAXNQ * ORC_MAXNQ], n[2];
    double lam = 0.0, q[ORC_MAXC];
    int bad = 0;
    int nv = elem_quad(P, e, nq, qx, qy, qr, qs, qw);
    for (int t = 0; t < nv; ++t) {
        euler_state(P, ce, qr[t], qs[t], q);
        double sp = euler_speed(P, q, NULL);
        if (isnan(sp)) bad = 1;
        else if (sp > lam) lam = sp;
    }
    for (int f = 0; f < nfaces(P); ++f) {
        int nf = face_quad(P, e, f, nq, qx, qy, qr, qs, qw, n);
        for (int t = 0; t < nf; ++t) {
            euler_state(P, ce, qr[t], qs[t], q);
            double sp = euler_speed(P, q, NULL);
            if (isnan(sp)) bad = 1;
            else if (sp > lam) lam = sp;
        }
    }
    return bad ? NAN : lam;
}

static void euler_residual_elem(const orc_problem* P, const double* U, long e, double* Le, double* gamma_out)
{
    int K = nmodes(P), m = P->dim + 2;
    int nq = P->p + 2;
    double ce[ORC_MAXC][ORC_MAXK], cn[ORC_MAXC][ORC_MAXK], R[ORC_MAXC][ORC_MAXK];
    double qx[ORC_MAXNQ * ORC_MAXNQ], qy[ORC_MAXNQ * ORC_MAXNQ], qr[ORC_MAXNQ * ORC_MAXNQ];
    double qs[ORC_MAXNQ * ORC_MAXNQ], qw[ORC_MAXNQ * ORC_MAXNQ];
    double fx[ORC_MAXNQ], fy[ORC_MAXNQ], fr[ORC_MAXNQ], fs[ORC_MAXNQ], fw[ORC_MAXNQ], n[2];
    memset(R, 0, sizeof R);
    for (int c = 0; c < m; ++c) load_comp(P, U, e, c, ce[c]);

    /* volume: + int grad(phi_k) . F(U_h) dx, component by component */
    int nv = elem_quad(P, e, nq, qx, qy, qr, qs, qw);
    for (int t = 0; t < nv; ++t) {
        double q[ORC_MAXC], Fx[ORC_MAXC], Fy[ORC_MAXC];
        euler_state(P, ce, qr[t], qs[t], q);
        euler_flux_n(P, q, 1.0, 0.0, Fx);
        if (P->dim == 2) euler_flux_n(P, q, 0.0, 1.0, Fy);
        for (int k = 0; k < K; ++k) {
            double dx = phi_d(P, k, 1, 0, qr[t], qs[t]);
            double dy = P->dim == 2 ? phi_d(P, k, 0, 1, qr[t], qs[t]) : 0.0;
            for (int c = 0; c < m; ++c) R[c][k] += qw[t] * (dx * Fx[c] + (P->dim == 2 ? dy * Fy[c] : 0.0));
        }
    }

    /* faces: - int_{dK} phi_k H(U-, U+, n) ds */
    for (int f = 0; f < nfaces(P); ++f) {
        double sx = 0.0, sy = 0.0;
        long nb = neighbour(P, e, f, &sx, &sy);
        if (nb >= 0)
            for (int c = 0; c < m; ++c) load_comp(P, U, nb, c, cn[c]);
        int nf = face_quad(P, e, f, nq, fx, fy, fr, fs, fw, n);
        for (int t = 0; t < nf; ++t) {
            double um[ORC_MAXC], up[ORC_MAXC], H[ORC_MAXC];
            euler_state(P, ce, fr[t], fs[t], um);
            if (nb >= 0) {
                euler_state(P, cn, fr[t] + sx, fs[t] + sy, up);
            } else {
                for (int c = 0; c < m; ++c) up[c] = um[c];
                int wall = P->bc[f] == ORC_BC_REFLECT;
                if (P->bc[f] == ORC_BC_STATE) {
                    /* R19: the coordinate along the side against the moving split */
                    double s = f < 2 ? fy[t] : fx[t];
                    int ch = s < P->bsplit[f] + P->bspeed[f] * P->t ? P->bbelow[f] : P->babove[f];
                    if (ch == 2) wall = 1;
                    else for (int c = 0; c < m; ++c) up[c] = P->bstate[ch][c];
                }
                if (wall) {
                    /* mirror the normal momentum: m+ = m- - 2 (m-.n) n */
                    double mn = um[1] * n[0] + (P->dim == 2 ? um[2] * n[1] : 0.0);
                    up[1] = um[1] - 2.0 * mn * n[0];
                    if (P->dim == 2) up[2] = um[2] - 2.0 * mn * n[1];
                }
            }
            euler_llf(P, um, up, n, H);
            for (int k = 0; k < K; ++k) {
                double ph = phi_d(P, k, 0, 0, fr[t], fs[t]);
                for (int c = 0; c < m; ++c) R[c][k] -= fw[t] * ph * H[c];
            }
        }
    }

    /* stabilization of every component with the density's gamma */
    double gamma = 0.0;
    if (P->stab != ORC_STAB_DG && P->p >= 1) {
        gamma = (P->stab == ORC_STAB_LO) ? 1.0 : sensor_elem(P, U, e, NULL, NULL);
        double lam = P->lambda_nu > 0.0 ? P->lambda_nu : euler_lambda_elem(P, e, ce);
        double nu = lam * hx_of(P) / (2.0 * P->p);
        for (int t = 0; t < nv; ++t)
            for (int c = 0; c < m; ++c) {
                double ux = poly_d(P, ce[c], 1, 0, qr[t], qs[t]);
                double uy = P->dim == 2 ? poly_d(P, ce[c], 0, 1, qr[t], qs[t]) : 0.0;
                for (int k = 0; k < K; ++k) {
                    double g = phi_d(P, k, 1, 0, qr[t], qs[t]) * ux;
                    if (P->dim == 2) g += phi_d(P, k, 0, 1, qr[t], qs[t]) * uy;
                    R[c][k] -= gamma * nu * qw[t] * g;
                }
            }
    }
    if (gamma_out) *gamma_out = gamma;

    for (int k = 0; k < K; ++k) {
        double mk = 0.0;
        for (int t = 0; t < nv; ++t) {
            double ph = phi_d(P, k, 0, 0, qr[t], qs[t]);
            mk += qw[t] * ph * ph;
        }
        for (int c = 0; c < m; ++c) Le[c * K + k] = R[c][k] / mk;
    }
}

/* ------------------------------------------------------------------------- */
/* Public entry points (ctypes)                                               */
/* ------------------------------------------------------------------------- */

void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }

int orc_get_threads(void) { return g_threads; }

int orc_check(const orc_problem* P)
{
    orc_init();
    if (P->dim != 1 && P->dim != 2) return -1;
    if (P->p < 0 || P->p > ORC_MAXP) return -1;
    if (P->nx < 1 || (P->dim == 2 && P->ny < 1)) return -1;
    if (P->dim == 2) {
        double hx = hx_of(P), hy = hy_of(P);
        if (fabs(hx - hy) > 1e-12 * hx) return -1;
    }
    if (P->stab == ORC_STAB_ZHAO && !(P->w_nbr > 0.0 && P->theta > 0.0)) return -1;   /* lin_l > 0 */
    for (int f = 0; f < 2 * P->dim; ++f) {         /* walls and prescribed states: Euler system */
        if ((P->bc[f] == ORC_BC_REFLECT || P->bc[f] == ORC_BC_STATE) && P->flux != ORC_FLUX_EULER) return -1;
        if (P->bc[f] == ORC_BC_STATE && (P->bbelow[f] < 0 || P->bbelow[f] > 2 || P->babove[f] < 0 || P->babove[f] > 2))
            return -1;
    }
    if (P->flux == ORC_FLUX_EULER && !(P->gas_gamma > 1.0)) return -1;
    return 0;
}

void orc_residual(const orc_problem* P, const double* U, double* L)
{
    orc_init();
    long E = nelem(P);
    int K = nmodes(P);
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
    for (long e = 0; e < E; ++e) {
        double Le[ORC_MAXC * ORC_MAXK];
        if (P->flux == ORC_FLUX_EULER) {
            euler_residual_elem(P, U, e, Le, NULL);
            for (int k = 0; k < ncomp(P) * K; ++k) L[k * E + e] = Le[k];
        } else {
            residual_elem(P, U, e, Le, NULL);
            for (int k = 0; k < K; ++k) L[k * E + e] = Le[k];
        }
    }
}

void orc_sensor(const orc_problem* P, const double* U, double* gamma, double* ratio,
                double* weights /* E x 5 or NULL */)
{
    orc_init();
    long E = nelem(P);
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
    for (long e = 0; e < E; ++e) {
        double r, w[5];
        gamma[e] = sensor_elem(P, U, e, &r, w);
        if (ratio) ratio[e] = r;
        if (weights) for (int l = 0; l < 5; ++l) weights[e * 5 + l] = w[l];
    }
}

void orc_lambda(const orc_problem* P, const double* U, double* lam)
{
    orc_init();
    long E = nelem(P);
    for (long e = 0; e < E; ++e) {
        if (P->flux == ORC_FLUX_EULER) {
            double cq[ORC_MAXC][ORC_MAXK];
            for (int c = 0; c < ncomp(P); ++c) load_comp(P, U, e, c, cq[c]);
            lam[e] = euler_lambda_elem(P, e, cq);
            continue;
        }
        double ce[ORC_MAXK];
        load_elem(P, U, e, ce);
        lam[e] = lambda_elem(P, e, ce);
    }
}

/* Optimal third-order SSP Runge-Kutta (Eq. ssp), nsteps steps of size dt, in place. */
void orc_rk3(const orc_problem* P, double* U, double dt, int nsteps)
{
    long N = nstate(P);
    double* L = malloc(sizeof(double) * N);
    double* U1 = malloc(sizeof(double) * N);
    double* U2 = malloc(sizeof(double) * N);
    orc_problem Q = *P;                 /* the stage times (R19): t, t + dt, t + dt / 2 */
    for (int s = 0; s < nsteps; ++s) {
        const double t0 = P->t + s * dt;
        Q.t = t0;
        orc_residual(&Q, U, L);
        for (long i = 0; i < N; ++i) U1[i] = U[i] + dt * L[i];
        Q.t = t0 + dt;
        orc_residual(&Q, U1, L);
        for (long i = 0; i < N; ++i) U2[i] = 0.75 * U[i] + 0.25 * U1[i] + 0.25 * dt * L[i];
        Q.t = t0 + 0.5 * dt;
        orc_residual(&Q, U2, L);
        for (long i = 0; i < N; ++i) U[i] = U[i] / 3.0 + 2.0 / 3.0 * U2[i] + 2.0 / 3.0 * dt * L[i];
    }
    free(L); free(U1); free(U2);
}

/* SSP Runge-Kutta of order p + 1 for the convergence studies of Sec. 5 (reading R14: the
 * paper names no scheme).  Order 2: the two-stage SSP method (Heun),
 *   U1 = U + dt L(U),  U <- 1/2 U + 1/2 (U1 + dt L(U1)). */
void orc_rk2(const orc_problem* P, double* U, double dt, int nsteps)
{
    long N = nstate(P);
    double* L = malloc(sizeof(double) * N);
    double* U1 = malloc(sizeof(double) * N);
    orc_problem Q = *P;                 /* the stage times (R19): t, t + dt */
    for (int s = 0; s < nsteps; ++s) {
        Q.t = P->t + s * dt;
        orc_residual(&Q, U, L);
        for (long i = 0; i < N; ++i) U1[i] = U[i] + dt * L[i];
        Q.t = P->t + s * dt + dt;
        orc_residual(&Q, U1, L);
        for (long i = 0; i < N; ++i) U[i] = 0.5 * U[i] + 0.5 * U1[i] + 0.5 * dt * L[i];
    }
    free(L); free(U1);
}

/* Order 4: the ten-stage low-storage SSP method of Ketcheson (2008), two registers:
 *   q1 = q2 = U;  five times q1 <- q1 + dt/6 L(q1);
 *   q2 <- q2/25 + 9/25 q1;  q1 <- 15 q2 - 5 q1;
 *   four times q1 <- q1 + dt/6 L(q1);
 *   U <- q2 + 3/5 q1 + dt/10 L(q1). */
void orc_rk4(const orc_problem* P, double* U, double dt, int nsteps)
{
    long N = nstate(P);
    double* L = malloc(sizeof(double) * N);
    double* q1 = malloc(sizeof(double) * N);
    double* q2 = malloc(sizeof(double) * N);
    for (int s = 0; s < nsteps; ++s) {
        for (long i = 0; i < N; ++i) q1[i] = q2[i] = U[i];
        for (int k = 0; k < 5; ++k) {
            orc_residual(P, q1, L);
            for (long i = 0; i < N; ++i) q1[i] += dt / 6.0 * L[i];
        }
        for (long i = 0; i < N; ++i) {
            q2[i] = q2[i] / 25.0 + 9.0 / 25.0 * q1[i];
            q1[i] = 15.0 * q2[i] - 5.0 * q1[i];
        }
        for (int k = 0; k < 4; ++k) {
            orc_residual(P, q1, L);
            for (long i = 0; i < N; ++i) q1[i] += dt / 6.0 * L[i];
        }
        orc_residual(P, q1, L);
        for (long i = 0; i < N; ++i) U[i] = q2[i] + 3.0 / 5.0 * q1[i] + dt / 10.0 * L[i];
    }
    free(L); free(q1); free(q2);
}

/* Sample layout for projection / error: f[e*nq^d + a + nq*b] at the physical points
 * x = xc + hx/2 * g_a, y = yc + hy/2 * g_b of the nq-point Gauss-Legendre rule. */

/* L2 projection onto V_p: c_k = int f phi_k / int phi_k^2 with nq-point Gauss. */
void orc_project(const orc_problem* P, int nq, const double* f, double* U)
{
    orc_init();
    long E = nelem(P);
    int K = nmodes(P);
    int npt = P->dim == 1 ? nq : nq * nq;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
    for (long e = 0; e < E; ++e) {
        double qx[ORC_MAXNQ * ORC_MAXNQ], qy[ORC_MAXNQ * ORC_MAXNQ], qw[ORC_MAXNQ * ORC_MAXNQ];
        double qr[ORC_MAXNQ * ORC_MAXNQ], qs[ORC_MAXNQ * ORC_MAXNQ];
        elem_quad(P, e, nq, qx, qy, qr, qs, qw);
        for (int k = 0; k < K; ++k) {
            double num = 0.0, den = 0.0;
            for (int t = 0; t < npt; ++t) {
                double ph = phi_d(P, k, 0, 0, qr[t], qs[t]);
                num += qw[t] * ph * f[e * npt + t];
                den += qw[t] * ph * ph;
            }
            U[k * E + e] = num / den;
        }
    }
}

/* sum_e int_{K_e} |U_h - f| dx with nq-point Gauss and samples f as above. */
double orc_l1_error(const orc_problem* P, const double* U, int nq, const double* f)
{
    orc_init();
    long E = nelem(P);
    int npt = P->dim == 1 ? nq : nq * nq;
    double s = 0.0;
    for (long e = 0; e < E; ++e) {
        double qx[ORC_MAXNQ * ORC_MAXNQ], qy[ORC_MAXNQ * ORC_MAXNQ], qw[ORC_MAXNQ * ORC_MAXNQ];
        double qr[ORC_MAXNQ * ORC_MAXNQ], qs[ORC_MAXNQ * ORC_MAXNQ];
        double ce[ORC_MAXK];
        load_elem(P, U, e, ce);
        elem_quad(P, e, nq, qx, qy, qr, qs, qw);
        for (int t = 0; t < npt; ++t)
            s += qw[t] * fabs(poly_d(P, ce, 0, 0, qr[t], qs[t]) - f[e * npt + t]);
    }
    return s;
}

/* Values of U_h at the nq-point Gauss points (same layout as the samples). */
void orc_eval(const orc_problem* P, const double* U, int nq, double* out)
{
    orc_init();
    long E = nelem(P);
    int npt = P->dim == 1 ? nq : nq * nq;
    for (long e = 0; e < E; ++e) {
        double qx[ORC_MAXNQ * ORC_MAXNQ], qy[ORC_MAXNQ * ORC_MAXNQ], qw[ORC_MAXNQ * ORC_MAXNQ];
        double qr[ORC_MAXNQ * ORC_MAXNQ], qs[ORC_MAXNQ * ORC_MAXNQ];
        double ce[ORC_MAXK];
        load_elem(P, U, e, ce);
        elem_quad(P, e, nq, qx, qy, qr, qs, qw);
        for (int t = 0; t < npt; ++t) out[e * npt + t] = poly_d(P, ce, 0, 0, qr[t], qs[t]);
    }
}

/* Total mass sum_e int_{K_e} U_h dx (quadrature of the polynomial). */
double orc_mass(const orc_problem* P, const double* U)
{
    orc_init();
    long E = nelem(P);
    double s = 0.0;
    for (long e = 0; e < E; ++e) {
        double qx[ORC_MAXNQ * ORC_MAXNQ], qy[ORC_MAXNQ * ORC_MAXNQ], qw[ORC_MAXNQ * ORC_MAXNQ];
        double qr[ORC_MAXNQ * ORC_MAXNQ], qs[ORC_MAXNQ * ORC_MAXNQ];
        double ce[ORC_MAXK];
        load_elem(P, U, e, ce);
        int n = elem_quad(P, e, P->p + 2, qx, qy, qr, qs, qw);
        for (int t = 0; t < n; ++t) s += qw[t] * poly_d(P, ce, 0, 0, qr[t], qs[t]);
    }
    return s;
}

/* Seminorm^2 of an arbitrary coefficient vector on element 0 (for tests). */
double orc_seminorm2(const orc_problem* P, const double* c) {
    orc_init(); return seminorm2(P, 0, c); }

/* Hermite candidate of element e from its face-f neighbour (for tests); returns
 * 0, or -1 when that neighbour does not exist. */
int orc_candidate(const orc_problem* P, const double* U, long e, int f, double* cl)
{
    orc_init();
    double sx, sy, ce[ORC_MAXK], cn[ORC_MAXK];
    long nb = neighbour(P, e, f, &sx, &sy);
    if (nb < 0) return -1;
    load_elem(P, U, e, ce);
    load_elem(P, U, nb, cn);
    candidate(P, e, ce, cn, sx, sy, cl);
    return 0;
}

/* Legendre values for tests. */
double orc_legendre(int n, int a, double x) {
    orc_init(); return leg_d(n, a, x); }

/* Residual and sensor of selected elements only (for sampled checks on large meshes).
 * out[k*n + t] = L_k of element idx[t]; gamma[t] = gamma of element idx[t]. */
void orc_residual_at(const orc_problem* P, const double* U, const long* idx, long n, double* out)
{
    orc_init();
    int K = nmodes(P);
    const int KK = K * ncomp(P);
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
    for (long t = 0; t < n; ++t) {
        double Le[ORC_MAXC * ORC_MAXK];
        if (P->flux == ORC_FLUX_EULER) euler_residual_elem(P, U, idx[t], Le, NULL);
        else residual_elem(P, U, idx[t], Le, NULL);
        for (int k = 0; k < KK; ++k) out[k * n + t] = Le[k];
    }
}

void orc_sensor_at(const orc_problem* P, const double* U, const long* idx, long n, double* gamma)
{
    orc_init();
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
    for (long t = 0; t < n; ++t) gamma[t] = sensor_elem(P, U, idx[t], NULL, NULL);
}
