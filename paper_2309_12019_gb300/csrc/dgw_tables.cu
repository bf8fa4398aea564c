// Host-side construction of the operator tables of degree p, in double.
//
// All tables live on the reference interval [-1, 1] in the Legendre basis P_0..P_p
// (Sec. 2, Eq. fesol; the paper's method does not depend on the basis):
//   * Gauss-Legendre rule with p + 2 points (volume and face quadrature);
//   * P_i and P_i' at those points;
//   * Hermite shift matrices: P_m(xi +- 2) expanded in P_i.  A neighbour polynomial
//     continued into the cell (the candidate of Sec. 4) is this re-expansion applied
//     along the face-normal axis.  Computed exactly from the Taylor series
//     P_m(xi + s) = sum_a s^a / a! P_m^(a)(xi), a finite sum for polynomials;
//   * A^(a)_mn = int P_m^(a) P_n^(a), from the Legendre differentiation matrix,
//     giving the scaled seminorm of Sec. 4 on square cells,
//     G = sum_{1<=|k|<=p} 2^{2|k|-d} (x)_i A^(k_i)  (h cancels), and the stiffness
//     A^(1) used by the stabilization of Sec. 3.
#include <cmath>
#include <cstring>

#include "dgw_internal.h"

namespace dgw {

namespace {

// P_0..P_n and derivatives at x by the three-term recurrence and
// P'_{k+1} = P'_{k-1} + (2k+1) P_k.
void legendre_all(int n, double x, double* P, double* dP)
{
    P[0] = 1.0;
    dP[0] = 0.0;
    if (n == 0) return;
    P[1] = x;
    dP[1] = 1.0;
    for (int k = 1; k < n; ++k) {
        P[k + 1] = ((2 * k + 1) * x * P[k] - k * P[k - 1]) / (k + 1);
        dP[k + 1] = dP[k - 1] + (2 * k + 1) * P[k];
    }
}

void gauss_rule(int n, double* x, double* w)
{
    double P[16], dP[16];
    for (int i = 0; i < n; ++i) {
        // Chebyshev-like first guess of the (n-i)-th root, then Newton.
        double z = std::cos(M_PI * (4.0 * i + 3.0) / (4.0 * n + 2.0));
        for (int it = 0; it < 64; ++it) {
            legendre_all(n, z, P, dP);
            double dz = P[n] / dP[n];
            z -= dz;
            if (std::fabs(dz) <= 1e-17) break;
        }
        legendre_all(n, z, P, dP);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dP[n] * dP[n]);
    }
    // exactly symmetric nodes and weights (the kernels use the rows of the positive nodes
    // for both of a pair): mirror the positive half, centre at 0 for odd n
    for (int i = 0; i < n / 2; ++i) {
        x[i] = -x[n - 1 - i];
        w[i] = w[n - 1 - i];
    }
    if (n & 1) x[n / 2] = 0.0;
}

// Legendre differentiation matrix on coefficients: (D c)_r = sum_n D[r][n] c_n,
// P_n' = sum_{r < n, n - r odd} (2r + 1) P_r.
void diff_matrix(int p, double D[kMaxN1][kMaxN1])
{
    for (int r = 0; r <= p; ++r)
        for (int n = 0; n <= p; ++n) D[r][n] = (r < n && ((n - r) & 1)) ? 2.0 * r + 1.0 : 0.0;
}

void matmul(int p, const double A[kMaxN1][kMaxN1], const double B[kMaxN1][kMaxN1],
            double C[kMaxN1][kMaxN1])
{
    double T[kMaxN1][kMaxN1];
    for (int i = 0; i <= p; ++i)
        for (int j = 0; j <= p; ++j) {
            double s = 0.0;
            for (int k = 0; k <= p; ++k) s += A[i][k] * B[k][j];
            T[i][j] = s;
        }
    std::memcpy(C, T, sizeof T);
}

}  // namespace

void gauss_rule_public(int n, double* x, double* w) { gauss_rule(n, x, w); }

void build_tables(int p, HostTables* t)
{
    std::memset(t, 0, sizeof *t);
    t->p = p;
    const int nq = p + 2;
    gauss_rule(nq, t->g, t->w);
    for (int q = 0; q < nq; ++q) {
        double P[16], dP[16];
        legendre_all(p, t->g[q], P, dP);
        for (int i = 0; i <= p; ++i) { t->B[q][i] = P[i]; t->D[q][i] = dP[i]; }
    }

    // powers of the differentiation matrix: Dp[a] = D^a
    double D[kMaxN1][kMaxN1], Dp[kMaxN1 + 1][kMaxN1][kMaxN1];
    diff_matrix(p, D);
    std::memset(Dp, 0, sizeof Dp);
    for (int i = 0; i <= p; ++i) Dp[0][i][i] = 1.0;
    for (int a = 1; a <= p; ++a) matmul(p, D, Dp[a - 1], Dp[a]);

    // shift matrices: column m = sum_a s^a / a! D^a e_m
    for (int side = 0; side < 2; ++side) {
        const double s = side == 0 ? 2.0 : -2.0;
        for (int m = 0; m <= p; ++m)
            for (int i = 0; i <= p; ++i) {
                double v = 0.0, fac = 1.0, pw = 1.0;
                for (int a = 0; a <= p; ++a) {
                    if (a > 0) { fac *= a; pw *= s; }
                    v += pw / fac * Dp[a][i][m];
                }
                t->T[side][i][m] = v;
            }
    }

    // A^(a)_mn = sum_r (D^a)_rm (D^a)_rn 2/(2r+1)
    double A[kMaxN1 + 1][kMaxN1][kMaxN1];
    for (int a = 0; a <= p; ++a)
        for (int m = 0; m <= p; ++m)
            for (int n = 0; n <= p; ++n) {
                double s = 0.0;
                for (int r = 0; r <= p; ++r) s += Dp[a][r][m] * Dp[a][r][n] * 2.0 / (2 * r + 1);
                A[a][m][n] = s;
            }
    for (int i = 0; i <= p; ++i) {
        t->A0[i] = 2.0 / (2 * i + 1);
        t->minv[i] = (2 * i + 1) / 2.0;
        for (int m = 0; m <= p; ++m) t->A1[i][m] = A[1][i][m];
    }
    // seminorm Gram matrices
    for (int m = 0; m <= p; ++m)
        for (int n = 0; n <= p; ++n) {
            double s = 0.0;
            for (int a = 1; a <= p; ++a) s += std::ldexp(1.0, 2 * a - 1) * A[a][m][n];
            t->G1[m][n] = s;
        }
    const int n1 = p + 1;
    for (int k1 = 0; k1 < n1 * n1; ++k1)
        for (int k2 = 0; k2 < n1 * n1; ++k2) {
            const int i1 = k1 % n1, j1 = k1 / n1, i2 = k2 % n1, j2 = k2 / n1;
            double s = 0.0;
            for (int ky = 0; ky <= p; ++ky)
                for (int kx = 0; kx <= p; ++kx) {
                    const int kk = kx + ky;
                    if (kk < 1 || kk > p) continue;
                    s += std::ldexp(1.0, 2 * kk - 2) * A[kx][i1][i2] * A[ky][j1][j2];
                }
            t->G2[k1][k2] = s;
        }
}

}  // namespace dgw
