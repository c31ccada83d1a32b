// adjoint.cu -- the hand-written adjoint of the RKDG operator: for a state u
// and an adjoint vector lambda (both in the internal layout and scaling),
// g = (d L_h / d u)^T lambda, where L_h is the operator of the stage kernel
// (volume quadrature, local Lax-Friedrichs face fluxes, boundary ghosts; the
// weak form of Sec. 2 with the quadrature rules the stage kernel uses).
//
// Owner-computes, one thread per cell, no atomics: cell c collects every term
// of sum_d lambda_d . L_d that depends on its own coefficients -- its volume
// integral, and at each of its faces the flux in its own residual and in the
// neighbour's residual (one flux value: the two cells of a face evaluate exact
// negatives of each other, see llf2).  Here each face is differentiated in the
// orientation of its lower-index cell.  Where the flux takes a maximum (the
// local Lax-Friedrichs speed) the derivative follows the larger side, as the
// forward evaluation does (at an exact tie either side is a valid choice).
#include "kernels.h"
#include "physics.cuh"
#include "tables.cuh"

namespace csw {

__constant__ Tab<float, 1> aT_f1;
__constant__ Tab<float, 2> aT_f2;
__constant__ Tab<double, 1> aT_d1;
__constant__ Tab<double, 2> aT_d2;

template <typename R, int K> __device__ __forceinline__ const Tab<R, K> &atab();
template <> __device__ __forceinline__ const Tab<float, 1> &atab<float, 1>() { return aT_f1; }
template <> __device__ __forceinline__ const Tab<float, 2> &atab<float, 2>() { return aT_f2; }
template <> __device__ __forceinline__ const Tab<double, 1> &atab<double, 1>() { return aT_d1; }
template <> __device__ __forceinline__ const Tab<double, 2> &atab<double, 2>() { return aT_d2; }

cudaError_t adjoint_upload_tables()
{
    static Tab<float, 1> f1;
    static Tab<float, 2> f2;
    static Tab<double, 1> d1;
    static Tab<double, 2> d2;
    make_tab(f1); make_tab(f2); make_tab(d1); make_tab(d2);
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(aT_f1, &f1, sizeof(f1))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(aT_f2, &f2, sizeof(f2))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(aT_d1, &d1, sizeof(d1))) != cudaSuccess) return e;
    return cudaMemcpyToSymbol(aT_d2, &d2, sizeof(d2));
}

// out = A(U)^T a + B(U)^T b: the gradient of a . f(U) + b . g(U) for the
// physical fluxes (f, g) of flux_fg.  Euler: the flux Jacobians in conserved
// variables, u = m_x/rho, v = m_y/rho, H = (E + p)/rho, gt = gamma - 1:
//   A = [0 1 0 0; gt q2/2 - u^2, (3-gamma)u, -gt v, gt; -uv, v, u, 0;
//        u(gt q2/2 - H), H - gt u^2, -gt uv, gamma u]
//   B = [0 0 1 0; -uv, v, u, 0; gt q2/2 - v^2, -gt u, (3-gamma)v, gt;
//        v(gt q2/2 - H), -gt uv, H - gt v^2, gamma v]
template <int EQ, typename R> __device__ __forceinline__ void flux_jac_T(const R *U, R gam, const R *a, const R *b, R *out)
{
    if (EQ == BURGERS) {
        out[0] = U[0] * (a[0] + b[0]);
        return;
    }
    const R ir = frcp(U[0]);
    const R u = U[1] * ir, v = U[2] * ir, gt = gam - R(1);
    const R q2 = u * u + v * v;
    const R p = gt * (U[3] - R(0.5) * U[0] * q2);
    const R H = (U[3] + p) * ir, k = R(0.5) * gt * q2;
    out[0] = a[1] * (k - u * u) - a[2] * u * v + a[3] * u * (k - H) - b[1] * u * v + b[2] * (k - v * v) + b[3] * v * (k - H);
    out[1] = a[0] + a[1] * (R(3) - gam) * u + a[2] * v + a[3] * (H - gt * u * u) + b[1] * v - b[2] * gt * u - b[3] * gt * u * v;
    out[2] = -a[1] * gt * v + a[2] * u - a[3] * gt * u * v + b[0] + b[1] * u + b[2] * (R(3) - gam) * v + b[3] * (H - gt * v * v);
    out[3] = a[1] * gt + a[3] * gam * u + b[2] * gt + b[3] * gam * v;
}

// gradient of the wave speed s = |u.n| + c of the local Lax-Friedrichs flux
template <typename R> __device__ __forceinline__ void speed_grad(const R *U, R gam, R nx, R ny, R *ds)
{
    const R ir = frcp(U[0]);
    const R u = U[1] * ir, v = U[2] * ir, gt = gam - R(1);
    const R q2 = u * u + v * v;
    const R p = gt * (U[3] - R(0.5) * U[0] * q2);
    const R c = fsqrt(gam * p * ir);
    const R un = u * nx + v * ny, sg = (un > R(0)) ? R(1) : ((un < R(0)) ? R(-1) : R(0));
    const R k = gam / (R(2) * c * U[0]);
    ds[0] = sg * (-un * ir) + k * (R(0.5) * gt * q2 - p * ir);
    ds[1] = sg * nx * ir - k * gt * u;
    ds[2] = sg * ny * ir - k * gt * v;
    ds[3] = k * gt;
}

// transposed derivatives of the local Lax-Friedrichs flux F(UL, UR; n) of
// physics.cuh (unit normal): gL = (dF/dUL)^T mu, gR = (dF/dUR)^T mu
template <int EQ, typename R>
__device__ __forceinline__ void llf_adj(const R *UL, const R *UR, R nx, R ny, R gam, const R *mu, R *gL, R *gR)
{
    constexpr int NV = Eqn<EQ>::NV;
    if (EQ == BURGERS) {
        const R s = nx + ny, as = rabs(s);
        const bool left = rabs(UL[0]) > rabs(UR[0]);
        const R a = (left ? rabs(UL[0]) : rabs(UR[0])) * as;
        const R jump = UR[0] - UL[0];
        const R dL = R(0.5) * UL[0] * s + R(0.5) * a - (left ? R(0.5) * jump * ((UL[0] > R(0)) ? as : -as) : R(0));
        const R dR = R(0.5) * UR[0] * s - R(0.5) * a - (left ? R(0) : R(0.5) * jump * ((UR[0] > R(0)) ? as : (UR[0] < R(0) ? -as : R(0))));
        gL[0] = dL * mu[0];
        gR[0] = dR * mu[0];
        return;
    }
    // speeds as the forward flux evaluates them
    const R irl = frcp(UL[0]), irr = frcp(UR[0]);
    const R unl = (UL[1] * nx + UL[2] * ny) * irl, unr = (UR[1] * nx + UR[2] * ny) * irr;
    const R pl = (gam - R(1)) * (UL[3] - R(0.5) * (UL[1] * UL[1] + UL[2] * UL[2]) * irl);
    const R pr = (gam - R(1)) * (UR[3] - R(0.5) * (UR[1] * UR[1] + UR[2] * UR[2]) * irr);
    const R cl = fsqrt(gam * pl * irl), cr = fsqrt(gam * pr * irr);
    const R sl = rabs(unl) + cl, sr = rabs(unr) + cr;
    const bool left = sl > sr;
    const R a = left ? sl : sr;
    R jm = R(0);
    for (int v = 0; v < NV; ++v) jm += (UR[v] - UL[v]) * mu[v];
    R an[NV], bn[NV];
    for (int v = 0; v < NV; ++v) { an[v] = nx * mu[v]; bn[v] = ny * mu[v]; }
    R tL[NV], tR[NV], ds[NV];
    flux_jac_T<EQ, R>(UL, gam, an, bn, tL);
    flux_jac_T<EQ, R>(UR, gam, an, bn, tR);
    speed_grad<R>(left ? UL : UR, gam, nx, ny, ds);
    for (int v = 0; v < NV; ++v) {
        gL[v] = R(0.5) * tL[v] + R(0.5) * a * mu[v] - (left ? R(0.5) * jm * ds[v] : R(0));
        gR[v] = R(0.5) * tR[v] - R(0.5) * a * mu[v] - (left ? R(0) : R(0.5) * jm * ds[v]);
    }
}

template <int EQ, int K, typename R>
__global__ void __launch_bounds__(128) k_rhs_adj(MeshDev<R> M, const R *__restrict__ u, const R *__restrict__ lam, R *grad,
                                                 double tfac, const Ctl *__restrict__ ctl, const R *x, R ax, const R *y, R ay,
                                                 R beta)
{
    constexpr int NP = Deg<K>::NP, QV = Deg<K>::QV, QF = Deg<K>::QF, NV = Eqn<EQ>::NV;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= M.nc) return;
    const Tab<R, K> &T = atab<R, K>();
    const int ld = M.ldc;
    const R gam = M.gammar;
    R uc[NV][NP], lc[NV][NP], g[NV][NP];
    load_cell<NV, NP>(u, c, uc);
    load_cell<NV, NP>(lam, c, lc);
    for (int v = 0; v < NV; ++v)
        for (int m = 0; m < NP; ++m) g[v][m] = R(0);
    const R g0 = M.geo[G_RX * ld + c], g1 = M.geo[G_RY * ld + c], g2 = M.geo[G_SX * ld + c], g3 = M.geo[G_SY * ld + c];

    // volume: d/du of sum_q w_q [ (dr psi)(g0 f + g1 g) + (ds psi)(g2 f + g3 g) ] . lambda
    for (int q = 0; q < QV; ++q) {
        R U[NV], a[NV], b[NV], t[NV], dx[NP], dy[NP];
        // physical derivatives of the basis at the point, weight folded in
        for (int m = 0; m < NP; ++m) {
            dx[m] = T.vdrw[q][m] * g0 + T.vdsw[q][m] * g2;
            dy[m] = T.vdrw[q][m] * g1 + T.vdsw[q][m] * g3;
        }
        for (int v = 0; v < NV; ++v) {
            R su = R(0), sa = R(0), sb = R(0);
            for (int m = 0; m < NP; ++m) {
                su += uc[v][m] * T.vphi[q][m];
                sa += lc[v][m] * dx[m];
                sb += lc[v][m] * dy[m];
            }
            U[v] = su;
            a[v] = sa;
            b[v] = sb;
        }
        flux_jac_T<EQ, R>(U, gam, a, b, t);
        for (int v = 0; v < NV; ++v)
            for (int m = 0; m < NP; ++m) g[v][m] += T.vphi[q][m] * t[v];
    }

    // faces: the canonical flux enters this cell's residual with -|n~| w_g psi and
    // the neighbour's with the neighbour's factors at the reversed point
    const unsigned nbf = M.nbf[c];
#pragma unroll 1
    for (int f = 0; f < 3; ++f) {
        const R nx = M.geo[(G_N0X + 3 * f) * ld + c], ny = M.geo[(G_N0Y + 3 * f) * ld + c], nl = M.geo[(G_N0L + 3 * f) * ld + c];
        const int code = M.nbr[f * ld + c];
        const int nf = (nbf >> (2 * f)) & 3;
        const bool swap = code >= 0 && code < c;
        const R snl = swap ? -nl : nl;
        R un_[NV][NP], ln[NV][NP];
        R snl_nb = R(0);
        BFace bf;
        int kind = BC_PERIODIC;
        if (code >= 0) {
            load_cell<NV, NP>(u, code, un_);
            load_cell<NV, NP>(lam, code, ln);
            const R nlb = M.geo[(G_N0L + 3 * nf) * ld + code];
            snl_nb = (c < code) ? -nlb : nlb;  // the neighbour swaps exactly when this cell is the lower index
        } else {
            bf = M.bf[-code - 1];
            kind = M.bc->kind[bf.tag];
        }
#pragma unroll 1
        for (int g_ = 0; g_ < QF; ++g_) {
            const int gr = QF - 1 - g_;
            R Ui[NV], Uo[NV], mu[NV];
            for (int v = 0; v < NV; ++v) {
                R s = R(0), sl = R(0);
                for (int m = 0; m < NP; ++m) {
                    s += uc[v][m] * T.fphi[f][g_][m];
                    sl += lc[v][m] * T.fphi[f][g_][m];
                }
                Ui[v] = s;
                mu[v] = -T.fw[g_] * snl * sl;
            }
            if (code >= 0) {
                for (int v = 0; v < NV; ++v) {
                    R s = R(0), sl = R(0);
                    for (int m = 0; m < NP; ++m) {
                        s += un_[v][m] * T.fphi[nf][gr][m];
                        sl += ln[v][m] * T.fphi[nf][gr][m];
                    }
                    Uo[v] = s;
                    mu[v] -= T.fw[gr] * snl_nb * sl;
                }
            } else if (kind == BC_TRANSMISSIVE) {
                for (int v = 0; v < NV; ++v) Uo[v] = uc[v][0] * T.vphi[0][0];  // the cell mean (reading R-bc)
            } else {
                ghost<EQ, R>(bf, M.bc, (double)T.ft[g_], stage_time(ctl, tfac), Ui, Uo);
            }
            R gL[NV], gR[NV], dUi[NV], dUo[NV];
            if (!swap) {
                llf_adj<EQ, R>(Ui, Uo, nx, ny, gam, mu, gL, gR);
                for (int v = 0; v < NV; ++v) { dUi[v] = gL[v]; dUo[v] = gR[v]; }
            } else {
                llf_adj<EQ, R>(Uo, Ui, -nx, -ny, gam, mu, gL, gR);
                for (int v = 0; v < NV; ++v) { dUi[v] = gR[v]; dUo[v] = gL[v]; }
            }
            if (code < 0) {
                // the ghost as a function of the interior: the cell mean (transmissive,
                // mode 0 only) or the trace (wall)
                if (kind == BC_TRANSMISSIVE) {
                    for (int v = 0; v < NV; ++v) g[v][0] += T.vphi[0][0] * dUo[v];
                } else if (kind == BC_PERIODIC) {
                    for (int v = 0; v < NV; ++v) dUi[v] += dUo[v];
                } else if (kind == BC_WALL) {
                    if (EQ == EULER) {
                        const R bx = (R)bf.nx, by = (R)bf.ny;
                        const R mn = dUo[1] * bx + dUo[2] * by;
                        dUi[0] += dUo[0];
                        dUi[1] += dUo[1] - R(2) * mn * bx;
                        dUi[2] += dUo[2] - R(2) * mn * by;
                        dUi[NV - 1] += dUo[NV - 1];
                    } else {
                        for (int v = 0; v < NV; ++v) dUi[v] += dUo[v];
                    }
                }  // Dirichlet and shock-line ghosts do not depend on the interior
            }
            for (int v = 0; v < NV; ++v)
                for (int m = 0; m < NP; ++m) g[v][m] += T.fphi[f][g_][m] * dUi[v];
        }
    }
    // epilogue: grad = ax x + ay y + beta g (x, y nullable; grad may alias x or
    // y, never u or lam: a cell reads and writes only its own entries of them)
    if (x || y) {
        R xv[NV][NP];
        if (x) {
            load_cell<NV, NP>(x, c, xv);
            for (int v = 0; v < NV; ++v)
                for (int m = 0; m < NP; ++m) g[v][m] = ax * xv[v][m] + beta * g[v][m];
        } else {
            for (int v = 0; v < NV; ++v)
                for (int m = 0; m < NP; ++m) g[v][m] = beta * g[v][m];
        }
        if (y) {
            load_cell<NV, NP>(y, c, xv);
            for (int v = 0; v < NV; ++v)
                for (int m = 0; m < NP; ++m) g[v][m] += ay * xv[v][m];
        }
    } else if (beta != R(1)) {
        for (int v = 0; v < NV; ++v)
            for (int m = 0; m < NP; ++m) g[v][m] = beta * g[v][m];
    }
    store_cell<NV, NP>(grad, c, g);
}

template <typename R>
void launch_rhs_adjoint(int eq, int k, const MeshDev<R> &M, const R *u, const R *lam, R *grad, double tfac, const Ctl *ctl,
                        cudaStream_t st, const R *x, R ax, const R *y, R ay, R beta)
{
    const int blk = 128, grd = (M.nc + blk - 1) / blk;
#define CSW_RA(E, KK) k_rhs_adj<E, KK, R><<<grd, blk, 0, st>>>(M, u, lam, grad, tfac, ctl, x, ax, y, ay, beta)
    if (eq == BURGERS && k == 1) CSW_RA(BURGERS, 1);
    else if (eq == BURGERS && k == 2) CSW_RA(BURGERS, 2);
    else if (eq == EULER && k == 1) CSW_RA(EULER, 1);
    else CSW_RA(EULER, 2);
#undef CSW_RA
}
template void launch_rhs_adjoint<float>(int, int, const MeshDev<float> &, const float *, const float *, float *, double, const Ctl *,
                                        cudaStream_t, const float *, float, const float *, float, float);
template void launch_rhs_adjoint<double>(int, int, const MeshDev<double> &, const double *, const double *, double *, double,
                                         const Ctl *, cudaStream_t, const double *, double, const double *, double, double);

// out = a x + b y (y nullable), elementwise over n entries (state arrays in
// the internal layout); out may alias x or y
template <typename R> __global__ void k_axpby(size_t n, R a, const R *x, R b, const R *y, R *out)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = y ? a * x[i] + b * y[i] : a * x[i];
}
template <typename R> void launch_axpby(size_t n, R a, const R *x, R b, const R *y, R *out, int grid, cudaStream_t st)
{
    k_axpby<R><<<grid, 256, 0, st>>>(n, a, x, b, y, out);
}
template void launch_axpby<float>(size_t, float, const float *, float, const float *, float *, int, cudaStream_t);
template void launch_axpby<double>(size_t, double, const double *, double, const double *, double *, int, cudaStream_t);

}  // namespace csw
