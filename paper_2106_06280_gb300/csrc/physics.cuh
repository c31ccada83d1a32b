// physics.cuh -- fluxes, local Lax-Friedrichs flux and boundary ghost states
// (device).  Burgers: Eq. 2dBurgers; Euler: Eq. 2dEulerEquations.
#pragma once
#include "common.cuh"

namespace csw {

template <typename R> __host__ __device__ __forceinline__ R rabs(R x) { return x < R(0) ? -x : x; }
template <typename R> __host__ __device__ __forceinline__ R rmax(R a, R b) { return a > b ? a : b; }
__host__ __device__ __forceinline__ float rsqroot(float x) { return sqrtf(x); }
// uncontracted products and sums (keep sign decisions identical to a plain evaluation)
__device__ __forceinline__ float rmul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd_rn(double a, double b) { return __dadd_rn(a, b); }
__host__ __device__ __forceinline__ double rsqroot(double x) { return sqrt(x); }

// reciprocal and square root: IEEE in FP64; in FP32-bulk the hardware
// approximations (MUFU, about 2 ulp)
__host__ __device__ __forceinline__ double rrcp(double x) { return 1.0 / x; }
__host__ __device__ __forceinline__ float rrcp(float x)
{
#ifdef __CUDA_ARCH__
    return __fdividef(1.0f, x);
#else
    return 1.0f / x;
#endif
}
__host__ __device__ __forceinline__ double rsqrt_fast(double x) { return sqrt(x); }
__host__ __device__ __forceinline__ float rsqrt_fast(float x)
{
#ifdef __CUDA_ARCH__
    return x > 0.0f ? x * rsqrtf(x) : sqrtf(x);
#else
    return sqrtf(x);
#endif
}

// reciprocal and square root of the stage kernel's fluxes: IEEE in FP64; in
// float the single-instruction approximations rcp.approx and sqrt.approx of
// the PTX ISA (sqrt.approx gives 0 at 0 and a NaN below it)
__host__ __device__ __forceinline__ double frcp(double x) { return 1.0 / x; }
__host__ __device__ __forceinline__ float frcp(float x)
{
#ifdef __CUDA_ARCH__
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
#else
    return 1.0f / x;
#endif
}
__host__ __device__ __forceinline__ double fsqrt(double x) { return sqrt(x); }
__host__ __device__ __forceinline__ float fsqrt(float x)
{
#ifdef __CUDA_ARCH__
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
#else
    return sqrtf(x);
#endif
}
// explicitly rounded fused multiply-add (never re-associated or re-contracted)
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// physical flux (f, g) at U
template <int EQ, typename R> __host__ __device__ __forceinline__ void flux_fg(const R *U, R gam, R *f, R *g)
{
    if (EQ == BURGERS) {
        const R h = R(0.5) * U[0] * U[0];
        f[0] = h;
        g[0] = h;
    } else {
        const R ir = frcp(U[0]);
        const R u = U[1] * ir, v = U[2] * ir;
        const R p = (gam - R(1)) * (U[3] - R(0.5) * (U[1] * u + U[2] * v));
        f[0] = U[1]; f[1] = U[1] * u + p; f[2] = U[2] * u; f[3] = (U[3] + p) * u;
        g[0] = U[2]; g[1] = U[1] * v;     g[2] = U[2] * v + p; g[3] = (U[3] + p) * v;
    }
}

// Twice the local Lax-Friedrichs flux (Sec. 2, the monotone flux f*, g*
// taken pointwise with the local maximum wave speed) through the unit normal n:
// 2F = (F(UL) + F(UR)).n - a (UR - UL), a = max |eigenvalue| along n.
// Every per-side quantity is computed by the same explicitly rounded sequence
// and the two sides meet only in commutative sums and in the maximum, so
//   llf2(UR, UL, -n) = -llf2(UL, UR, n)   bit for bit:
// the two cells of a face, each passing its own trace first and its own
// outward normal (the exact negative of the neighbour's), obtain exact
// negatives, and the cell means are conserved to the rounding of the update.
template <int EQ, typename R> __device__ __forceinline__ void llf2_side(const R *U, R nx, R ny, R gm1, R gh, R gam, R *fn, R &s)
{
    const R ir = frcp(U[0]);
    const R un = rmul_rn(rfma(U[1], nx, rmul_rn(U[2], ny)), ir);
    const R ke = rmul_rn(rfma(U[1], U[1], rmul_rn(U[2], U[2])), ir);
    const R p = rfma(-gh, ke, rmul_rn(gm1, U[3]));
    s = radd_rn(fabs(un), fsqrt(rmul_rn(rmul_rn(gam, p), ir)));
    fn[0] = rmul_rn(U[0], un);
    fn[1] = rfma(U[1], un, rmul_rn(p, nx));
    fn[2] = rfma(U[2], un, rmul_rn(p, ny));
    fn[3] = rmul_rn(radd_rn(U[3], p), un);
}

template <int EQ, typename R> __device__ __forceinline__ void llf2(const R *UL, const R *UR, R nx, R ny, R gam, R *F)
{
    if (EQ == BURGERS) {
        const R sn = radd_rn(nx, ny);
        const R a = rmul_rn(fmax(fabs(UL[0]), fabs(UR[0])), fabs(sn));
        const R q = rmul_rn(R(0.5) * radd_rn(rmul_rn(UL[0], UL[0]), rmul_rn(UR[0], UR[0])), sn);
        F[0] = rfma(-a, radd_rn(UR[0], -UL[0]), q);
    } else {
        const R gm1 = gam - R(1), gh = R(0.5) * gm1;
        R fl[4], fr[4], sl, sr;
        llf2_side<EQ, R>(UL, nx, ny, gm1, gh, gam, fl, sl);
        llf2_side<EQ, R>(UR, nx, ny, gm1, gh, gam, fr, sr);
        const R a = fmax(sl, sr);
#pragma unroll
        for (int v = 0; v < 4; ++v) F[v] = rfma(-a, radd_rn(UR[v], -UL[v]), radd_rn(fl[v], fr[v]));
    }
}

// ghost state of boundary face bf at edge parameter tp in [0,1], time t
template <int EQ, typename R>
__host__ __device__ __forceinline__ void ghost(const BFace &bf, const BcTab *bc, double tp, double t, const R *Uin, R *Ug)
{
    constexpr int NV = Eqn<EQ>::NV;
    const int kind = bc->kind[bf.tag];
    const double *P = bc->par[bf.tag];
    if (kind == BC_DIRICHLET) {
        for (int v = 0; v < NV; ++v) Ug[v] = (R)P[v];
    } else if (kind == BC_WALL && EQ == EULER) {
        const R nx = (R)bf.nx, ny = (R)bf.ny;
        const R mn = Uin[1] * nx + Uin[2] * ny;
        Ug[0] = Uin[0];
        Ug[1] = Uin[1] - R(2) * mn * nx;
        Ug[2] = Uin[2] - R(2) * mn * ny;
        Ug[NV - 1] = Uin[NV - 1];
    } else if (kind == BC_SHOCKLINE) {
        const double x = bf.ax + tp * (bf.bx - bf.ax), y = bf.ay + tp * (bf.by - bf.ay);
        const double xs = P[0] + y * P[1] + P[2] * t;
        const double *S = (x < xs) ? P + 3 : P + 3 + NV;
        for (int v = 0; v < NV; ++v) Ug[v] = (R)S[v];
    } else {
        for (int v = 0; v < NV; ++v) Ug[v] = Uin[v];
    }
}

// Reading R-pos as a detection trigger: 1 if the Euler polynomial with modes
// U[v][m] (internal scaling, table T) has a non-positive density or pressure at
// one of the volume points or face Gauss points.  A bound screens first: every
// point value of variable v lies within sum_{m>=1} |U_vm| max|psi_m| of the
// mean's share, and rho_lo > 0, E_lo > 0, 2 E_lo rho_lo > |m|_hi^2 imply
// 2 E rho > |m|^2 (p > 0) at every point; only cells that fail it are checked
// point by point (state precision with a relative margin, close calls in
// double), so the outcome is that of the point-by-point check.
template <int K, typename R>
__device__ __forceinline__ bool physical_by_bound(const R (&U)[4][Deg<K>::NP], const Tab<R, K> &T)
{
    constexpr int NP = Deg<K>::NP;
    R lo[4], hi[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        R d = R(0);
#pragma unroll
        for (int m = 1; m < NP; ++m) d += rabs(U[v][m]) * T.pmax[m];
        const R c = U[v][0] * T.vphi[0][0];
        lo[v] = c - d;
        hi[v] = c + d;
    }
    if (lo[0] > R(0) && lo[3] > R(0)) {
        const R mx = rmax(rabs(lo[1]), rabs(hi[1])), my = rmax(rabs(lo[2]), rabs(hi[2]));
        if (R(2) * lo[3] * lo[0] > R(1.001) * (mx * mx + my * my)) return true;
    }
    return false;
}

// the point-by-point check alone (1: non-physical at some point)
template <int K, typename R>
__device__ __forceinline__ bool nonphys_points_exact(const R (&U)[4][Deg<K>::NP], const Tab<R, K> &T, double gam)
{
    constexpr int NP = Deg<K>::NP, QV = Deg<K>::QV, QF = Deg<K>::QF;
#pragma unroll 1
    for (int q = 0; q < QV + 3 * QF; ++q) {
        const R *phi = (q < QV) ? T.vphi[q] : T.fphi[(q - QV) / QF][(q - QV) % QF];
        R P[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            R s = R(0);
#pragma unroll
            for (int m = 0; m < NP; ++m) s += U[v][m] * phi[m];
            P[v] = s;
        }
        const R two_e_rho = R(2) * P[3] * P[0], m2 = P[1] * P[1] + P[2] * P[2];
        const R qp = two_e_rho - m2;
        bool ok = (P[0] > R(0)) && (qp > R(1e-3) * (rabs(two_e_rho) + m2));
        if (!ok && P[0] > R(0) && !(qp < -R(1e-3) * (rabs(two_e_rho) + m2))) {
            const double r = (double)P[0], mxd = (double)P[1], myd = (double)P[2], E = (double)P[3];
            ok = (gam - 1.0) * (E - 0.5 * (mxd * mxd + myd * myd) / r) > 0.0;
        }
        if (!ok) return true;
    }
    return false;
}

template <int K, typename R>
__device__ __forceinline__ bool nonphys_points(const R (&U)[4][Deg<K>::NP], const Tab<R, K> &T, double gam)
{
    return !physical_by_bound<K, R>(U, T) && nonphys_points_exact<K, R>(U, T, gam);
}

}  // namespace csw
