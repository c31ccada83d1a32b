// tables.cuh -- host construction of the constant-memory tables (basis values
// and gradients at the volume points, basis values at the face Gauss points).
#pragma once
#include <algorithm>
#include <cmath>
#include "common.cuh"
#include "rules.cuh"

namespace csw {

// reference coordinates of a barycentric point: v0=(-1,-1), v1=(1,-1), v2=(-1,1)
__host__ __device__ inline void bary_to_rs(const double *b, double &r, double &s)
{
    r = -b[0] + b[1] - b[2];
    s = -b[0] - b[1] + b[2];
}

template <int K> __host__ __device__ inline void volume_rule(TriRule &R)
{
    if (K == 1) rule_deg2(R);
    else rule_deg5(R);
}

template <int K> __host__ __device__ inline void recon_rule(TriRule &R)
{
    if (K == 1) rule_deg2(R);
    else rule_deg4(R);
}

template <typename R, int K> inline void make_tab(Tab<R, K> &T)
{
    constexpr int NP = Deg<K>::NP, QV = Deg<K>::QV, QF = Deg<K>::QF;
    TriRule vr;
    volume_rule<K>(vr);
    for (int q = 0; q < QV; ++q) {
        double r, s;
        bary_to_rs(vr.b[q], r, s);
        T.vw[q] = (R)vr.w[q];
        for (int m = 0; m < NP; ++m) {
            double v, dr, ds;
            dubiner(K, m, r, s, v, dr, ds);
            T.vphi[q][m] = (R)v;
            T.vdr[q][m] = (R)dr;
            T.vds[q][m] = (R)ds;
            T.vdrw[q][m] = (R)(vr.w[q] * dr);
            T.vdsw[q][m] = (R)(vr.w[q] * ds);
        }
    }
    double t[4], w[4];
    gauss_legendre_01(QF, t, w);
    for (int g = 0; g < QF; ++g) { T.fw[g] = (R)w[g]; T.ft[g] = (R)t[g]; }
    for (int f = 0; f < 3; ++f)
        for (int g = 0; g < QF; ++g) {
            double b[3] = {0.0, 0.0, 0.0};
            b[f] = 1.0 - t[g];
            b[(f + 1) % 3] = t[g];
            // symmetric Gauss points: use the mirrored node for the upper half so
            // that point QF-1-g of the reversed edge is bit-identical
            if (g >= QF / 2) { b[f] = t[QF - 1 - g]; b[(f + 1) % 3] = 1.0 - t[QF - 1 - g]; }
            double r, s;
            bary_to_rs(b, r, s);
            for (int m = 0; m < NP; ++m) {
                double v, dr, ds;
                dubiner(K, m, r, s, v, dr, ds);
                T.fphi[f][g][m] = (R)v;
            }
        }
    for (int m = 0; m < NP; ++m) {
        double mx = 0.0;
        for (int q = 0; q < QV; ++q) mx = std::max(mx, std::fabs((double)T.vphi[q][m]));
        for (int f = 0; f < 3; ++f)
            for (int g = 0; g < QF; ++g) mx = std::max(mx, std::fabs((double)T.fphi[f][g][m]));
        T.pmax[m] = (R)(mx * (1.0 + 1e-5));
    }
    for (int f = 0; f < 3; ++f)
        for (int m = 0; m < NP; ++m) {
            double acc = 0.0;
            for (int g = 0; g < QF; ++g) acc += w[g] * (double)T.fphi[f][g][m];
            T.fint[f][m] = (R)acc;
        }
}

}  // namespace csw
