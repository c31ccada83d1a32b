// physics.cuh -- fluxes, local Lax-Friedrichs flux and boundary ghost states
// (device).  Burgers: Eq. 2dBurgers; Euler: Eq. 2dEulerEquations.
#pragma once
#include "common.cuh"

namespace csw {

template <typename R> __host__ __device__ __forceinline__ R rabs(R x) { return x < R(0) ? -x : x; }
template <typename R> __host__ __device__ __forceinline__ R rmax(R a, R b) { return a > b ? a : b; }
__host__ __device__ __forceinline__ float rsqrt_(float x) { return sqrtf(x); }
// uncontracted products and sums (keep sign decisions identical to a plain evaluation)
__device__ __forceinline__ float rmul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd_rn(double a, double b) { return __dadd_rn(a, b); }
__host__ __device__ __forceinline__ double rsqrt_(double x) { return sqrt(x); }

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

// physical flux (f, g) at U
template <int EQ, typename R> __host__ __device__ __forceinline__ void flux_fg(const R *U, R gam, R *f, R *g)
{
    if (EQ == BURGERS) {
        const R h = R(0.5) * U[0] * U[0];
        f[0] = h;
        g[0] = h;
    } else {
        const R ir = rrcp(U[0]);
        const R u = U[1] * ir, v = U[2] * ir;
        const R p = (gam - R(1)) * (U[3] - R(0.5) * (U[1] * u + U[2] * v));
        f[0] = U[1]; f[1] = U[1] * u + p; f[2] = U[2] * u; f[3] = (U[3] + p) * u;
        g[0] = U[2]; g[1] = U[1] * v;     g[2] = U[2] * v + p; g[3] = (U[3] + p) * v;
    }
}

// local Lax-Friedrichs flux through a normal n of length nl (the stage kernel passes a unit normal):
// F = 1/2 (F(UL) + F(UR)).n - 1/2 a (UR - UL), a = max |eigenvalue| along n
template <int EQ, typename R> __host__ __device__ __forceinline__ void llf(const R *UL, const R *UR, R nx, R ny, R nl, R gam, R *F)
{
    if (EQ == BURGERS) {
        const R s = nx + ny;
        const R a = rmax(rabs(UL[0]), rabs(UR[0])) * rabs(s);
        F[0] = R(0.25) * (UL[0] * UL[0] + UR[0] * UR[0]) * s - R(0.5) * a * (UR[0] - UL[0]);
    } else {
        const R irl = rrcp(UL[0]), irr = rrcp(UR[0]);
        const R unl = (UL[1] * nx + UL[2] * ny) * irl, unr = (UR[1] * nx + UR[2] * ny) * irr;
        const R pl = (gam - R(1)) * (UL[3] - R(0.5) * (UL[1] * UL[1] + UL[2] * UL[2]) * irl);
        const R pr = (gam - R(1)) * (UR[3] - R(0.5) * (UR[1] * UR[1] + UR[2] * UR[2]) * irr);
        const R cl = rsqrt_fast(gam * pl * irl), cr = rsqrt_fast(gam * pr * irr);
        const R a = rmax(rabs(unl) + cl * nl, rabs(unr) + cr * nl);
        F[0] = R(0.5) * (UL[0] * unl + UR[0] * unr) - R(0.5) * a * (UR[0] - UL[0]);
        F[1] = R(0.5) * (UL[1] * unl + pl * nx + UR[1] * unr + pr * nx) - R(0.5) * a * (UR[1] - UL[1]);
        F[2] = R(0.5) * (UL[2] * unl + pl * ny + UR[2] * unr + pr * ny) - R(0.5) * a * (UR[2] - UL[2]);
        F[3] = R(0.5) * ((UL[3] + pl) * unl + (UR[3] + pr) * unr) - R(0.5) * a * (UR[3] - UL[3]);
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

}  // namespace csw
