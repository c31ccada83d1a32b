// rules.cuh -- quadrature rules of the library (host and device).
//
// Volume rule for the operator: exact to degree max(2k, 3k-1); face rule:
// Gauss-Legendre exact to degree 3k; reconstruction points of Sec. 3.2 Step 5
// (the SCP rule the paper cites but does not print): a fully symmetric
// Np-point rule with positive weights exact to degree 2k.
//   k = 1: 3-point degree-2 rule, points (2/3,1/6,1/6) and permutations, weights 1/3
//   k = 2: 7-point degree-5 rule of Radon (closed form) for the volume; the
//          6-point degree-4 rule (two (a,a,1-2a) orbits) for the reconstruction,
//          found by Newton's method on its four symmetric moment conditions.
//   Gauss-Legendre, 2 points: +-1/sqrt(3); 4 points: closed form
//   +-sqrt(3/7 -+ (2/7) sqrt(6/5)), weights (18 +- sqrt(30))/36.
#pragma once
#include <math.h>

namespace csw {

struct TriRule {
    int n;
    double b[16][3];  // barycentric
    double w[16];     // weights, sum 1
};

__host__ __device__ inline void rule_orbit21(TriRule &R, double a, double w)
{
    const double c = 1.0 - 2.0 * a;
    const double P[3][3] = {{c, a, a}, {a, c, a}, {a, a, c}};
    for (int t = 0; t < 3; ++t) {
        R.b[R.n][0] = P[t][0];
        R.b[R.n][1] = P[t][1];
        R.b[R.n][2] = P[t][2];
        R.w[R.n] = w;
        R.n++;
    }
}

__host__ __device__ inline void rule_deg2(TriRule &R)
{
    R.n = 0;
    rule_orbit21(R, 1.0 / 6.0, 1.0 / 3.0);
}

__host__ __device__ inline void rule_deg5(TriRule &R)
{
    const double s15 = sqrt(15.0);
    R.n = 1;
    R.b[0][0] = R.b[0][1] = R.b[0][2] = 1.0 / 3.0;
    R.w[0] = 9.0 / 40.0;
    rule_orbit21(R, (6.0 - s15) / 21.0, (155.0 - s15) / 1200.0);
    rule_orbit21(R, (6.0 + s15) / 21.0, (155.0 + s15) / 1200.0);
}

// 6-point degree-4 rule: unknowns (a1, w1, a2, w2); conditions: the
// moments of lambda^p, p = 0, 2, 3, 4, which for an S3-symmetric rule give
// exactness on every polynomial of degree <= 4: sum = 2 p! / (p+2)!.
__host__ __device__ inline void rule_deg4(TriRule &R)
{
    double th[4] = {0.09, 0.11, 0.44, 0.22};
    const int pw[4] = {0, 2, 3, 4};
    for (int it = 0; it < 50; ++it) {
        double F[4], J[4][4];
        for (int e = 0; e < 4; ++e) {
            const int p = pw[e];
            double fac = 1.0;
            for (int i = 2; i <= p; ++i) fac *= i;
            double fac2 = 1.0;
            for (int i = 2; i <= p + 2; ++i) fac2 *= i;
            F[e] = -2.0 * fac / fac2;
            for (int o = 0; o < 2; ++o) {
                const double a = th[2 * o], w = th[2 * o + 1], c = 1.0 - 2.0 * a;
                const double ap = pow(a, p), cp = pow(c, p);
                F[e] += w * (2.0 * ap + cp);
                const double dap = (p > 0) ? p * pow(a, p - 1) : 0.0, dcp = (p > 0) ? p * pow(c, p - 1) : 0.0;
                J[e][2 * o] = w * (2.0 * dap - 2.0 * dcp);
                J[e][2 * o + 1] = 2.0 * ap + cp;
            }
        }
        // Gaussian elimination with partial pivoting on J d = -F
        double A[4][5];
        for (int r = 0; r < 4; ++r) {
            for (int c = 0; c < 4; ++c) A[r][c] = J[r][c];
            A[r][4] = -F[r];
        }
        for (int c = 0; c < 4; ++c) {
            int piv = c;
            for (int r = c + 1; r < 4; ++r)
                if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
            for (int q = 0; q < 5; ++q) { double tmp = A[c][q]; A[c][q] = A[piv][q]; A[piv][q] = tmp; }
            for (int r = c + 1; r < 4; ++r) {
                const double f = A[r][c] / A[c][c];
                for (int q = c; q < 5; ++q) A[r][q] -= f * A[c][q];
            }
        }
        double d[4];
        for (int r = 3; r >= 0; --r) {
            double s = A[r][4];
            for (int q = r + 1; q < 4; ++q) s -= A[r][q] * d[q];
            d[r] = s / A[r][r];
        }
        double dn = 0.0;
        for (int u = 0; u < 4; ++u) { th[u] += d[u]; dn += fabs(d[u]); }
        if (dn < 1e-16) break;
    }
    R.n = 0;
    rule_orbit21(R, th[0], th[1]);
    rule_orbit21(R, th[2], th[3]);
}

__host__ __device__ inline void gauss_legendre_01(int n, double *t, double *w)
{
    if (n == 2) {
        const double x = 1.0 / sqrt(3.0);
        t[0] = 0.5 * (1.0 - x); t[1] = 0.5 * (1.0 + x);
        w[0] = 0.5; w[1] = 0.5;
    } else {  // n == 4
        const double s = sqrt(6.0 / 5.0);
        const double x1 = sqrt(3.0 / 7.0 - 2.0 / 7.0 * s), x2 = sqrt(3.0 / 7.0 + 2.0 / 7.0 * s);
        const double w1 = (18.0 + sqrt(30.0)) / 36.0, w2 = (18.0 - sqrt(30.0)) / 36.0;
        t[0] = 0.5 * (1.0 - x2); t[1] = 0.5 * (1.0 - x1); t[2] = 0.5 * (1.0 + x1); t[3] = 0.5 * (1.0 + x2);
        w[0] = 0.5 * w2; w[1] = 0.5 * w1; w[2] = 0.5 * w1; w[3] = 0.5 * w2;
    }
}

}  // namespace csw
