// common.cuh -- shared definitions of the CUDA RKDG + CSWENO library:
// problem constants, the orthonormal triangle basis (Sec. 2, Eq. triangleBasis),
// constant-memory quadrature/basis tables and the kernel argument blocks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define CSW_MAXTAG 16
#define CSW_MAXPAR 16

namespace csw {

enum { BURGERS = 0, EULER = 1 };
enum { BC_PERIODIC = 0, BC_DIRICHLET = 1, BC_TRANSMISSIVE = 2, BC_WALL = 3, BC_SHOCKLINE = 4 };
enum { ERR_NONPHYS = 1, ERR_LSQ = 2, ERR_TIMEOUT = 4 };

template <int K> struct Deg {
    static constexpr int NP = (K + 1) * (K + 2) / 2;  // modes
    static constexpr int QV = (K == 1) ? 3 : 7;       // volume rule points (degree 2 / 5)
    static constexpr int QF = (K == 1) ? 2 : 4;       // Gauss-Legendre points per face (degree 3 / 7)
    static constexpr int QS = NP;                     // reconstruction (SCP-role) points
    static constexpr int NM = (K == 1) ? 5 : 9;       // non-constant monomials of the top stencil polynomial
    static constexpr int NSLOT = (K == 1) ? 3 : 4;    // WENO polynomials p_1..p_NSLOT
    static constexpr int NSUB = 7;                    // subcells per neighbour: 3 thirds + 4 halves
    static constexpr int NROW = (K == 1) ? 9 : 15;    // rows of the top least-squares problem
};
template <int EQ> struct Eqn { static constexpr int NV = (EQ == BURGERS) ? 1 : 4; };

// ---------------------------------------------------------------------------
// Orthonormal Dubiner basis psi_m(r, s), Sec. 2 Eq. triangleBasis, with
// L2-normalised Jacobi polynomials; modes ordered i outer, j inner.
// ---------------------------------------------------------------------------
__host__ __device__ inline double jac_unnorm(int n, double a, double b, double x)
{
    double p0 = 1.0;
    if (n == 0) return p0;
    double p1 = 0.5 * ((a + b + 2.0) * x + (a - b));
    for (int m = 2; m <= n; ++m) {
        const double c = 2.0 * m + a + b;
        const double p2 = ((c - 1.0) * (c * (c - 2.0) * x + a * a - b * b) * p1 -
                           2.0 * (m + a - 1.0) * (m + b - 1.0) * c * p0) /
                          (2.0 * m * (m + a + b) * (c - 2.0));
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// 1 / sqrt(2^{alpha+1} / (2n + alpha + 1)), the L2 normalisation of P_n^{(alpha,0)}
__host__ __device__ inline double jac_inv_norm(int n, int alpha)
{
    return sqrt((2.0 * n + alpha + 1.0) / (double)(2 << alpha));
}

__host__ __device__ inline void mode_pair(int k, int m, int &i, int &j)
{
    int idx = 0;
    i = 0;
    j = 0;
    for (int a = 0; a <= k; ++a)
        for (int b = 0; b <= k - a; ++b) {
            if (idx == m) { i = a; j = b; }
            ++idx;
        }
}

// value and (r,s) gradient of psi_m
__host__ __device__ inline void dubiner(int k, int m, double r, double s, double &v, double &dr, double &ds)
{
    int i, j;
    mode_pair(k, m, i, j);
    const double omb = 1.0 - s;
    const double a = (omb > 0.0) ? 2.0 * (1.0 + r) / omb - 1.0 : -1.0;
    const double ni = jac_inv_norm(i, 0), nj = jac_inv_norm(j, 2 * i + 1);
    const double Pa = jac_unnorm(i, 0.0, 0.0, a) * ni;
    const double dPa = (i > 0) ? 0.5 * (i + 1.0) * jac_unnorm(i - 1, 1.0, 1.0, a) * ni : 0.0;
    const double Qb = jac_unnorm(j, 2.0 * i + 1.0, 0.0, s) * nj;
    const double dQb = (j > 0) ? 0.5 * (j + 2.0 * i + 2.0) * jac_unnorm(j - 1, 2.0 * i + 2.0, 1.0, s) * nj : 0.0;
    double wi = 1.0, wim1 = 0.0;
    for (int t = 0; t < i; ++t) { wim1 = wi; wi *= omb; }
    const double sq2 = 1.4142135623730951;
    v = sq2 * Pa * Qb * wi;
    dr = sq2 * dPa * Qb * 2.0 * wim1;
    ds = sq2 * (dPa * (1.0 + a) * Qb * wim1 + Pa * dQb * wi - i * Pa * Qb * wim1);
}

// ---------------------------------------------------------------------------
// Constant-memory tables (filled once per process from the host rules).
// ---------------------------------------------------------------------------
template <typename R, int K> struct Tab {
    R vphi[Deg<K>::QV][Deg<K>::NP];   // psi_m at the volume points
    R vdr[Deg<K>::QV][Deg<K>::NP];    // d psi_m / dr
    R vds[Deg<K>::QV][Deg<K>::NP];    // d psi_m / ds
    R vw[Deg<K>::QV];                 // volume weights (sum 1)
    R fphi[3][Deg<K>::QF][Deg<K>::NP];// psi_m at the Gauss points of local face f
    R fw[Deg<K>::QF];                 // face weights (sum 1)
    R ft[Deg<K>::QF];                 // Gauss points as edge parameters in [0,1]
    R fint[3][Deg<K>::NP];            // sum_g fw[g] psi_m(point g of face f): the face mean of psi_m
    R vdrw[Deg<K>::QV][Deg<K>::NP];   // vw[q] d psi_m / dr (weight folded in, rounded once)
    R vdsw[Deg<K>::QV][Deg<K>::NP];   // vw[q] d psi_m / ds
    R pmax[Deg<K>::NP];               // max of |psi_m| over the volume and face points (rounded up)
};

// Traces seen from the neighbour: psi_m at the Gauss points of local face nf
// in the reversed order (the adjacent cell's point g is the neighbour's point
// QF-1-g), in shared memory with rows padded to 16 bytes.  A __constant__
// table indexed by the per-thread face nf serialises a warp over its distinct
// faces; a shared-memory row is one or two vector loads.  Every thread of the
// block calls fill() before the first use (it ends with __syncthreads).
template <typename R, int K> struct NbrTraceTab {
    static constexpr int NP = Deg<K>::NP, QF = Deg<K>::QF;
    static constexpr int W = (sizeof(R) == 4) ? ((NP + 3) & ~3) : ((NP + 1) & ~1);
    __align__(16) R v[3 * QF * W];
    __device__ __forceinline__ void fill(const Tab<R, K> &T)
    {
        for (int i = threadIdx.x; i < 3 * QF * W; i += blockDim.x) {
            const int nf = i / (QF * W), g = (i / W) % QF, m = i % W;
            v[i] = (m < NP) ? T.fphi[nf][QF - 1 - g][m] : R(0);
        }
        __syncthreads();
    }
    // row of face nf, point g (adjacent cell's order) into registers
    __device__ __forceinline__ void row(int nf, int g, R (&p)[NP]) const
    {
        const R *q = v + (nf * QF + g) * W;
        if (sizeof(R) == 4) {
#pragma unroll
            for (int i = 0; i < W / 4; ++i) {
                const float4 x = reinterpret_cast<const float4 *>(q)[i];
                if (4 * i + 0 < NP) p[(4 * i + 0) % NP] = x.x;
                if (4 * i + 1 < NP) p[(4 * i + 1) % NP] = x.y;
                if (4 * i + 2 < NP) p[(4 * i + 2) % NP] = x.z;
                if (4 * i + 3 < NP) p[(4 * i + 3) % NP] = x.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < W / 2; ++i) {
                const double2 x = reinterpret_cast<const double2 *>(q)[i];
                if (2 * i + 0 < NP) p[(2 * i + 0) % NP] = (R)x.x;
                if (2 * i + 1 < NP) p[(2 * i + 1) % NP] = (R)x.y;
            }
        }
    }
};

// per-boundary-face data (double: used in boundary decisions)
struct BFace {
    double ax, ay, bx, by;  // endpoints, interior on the left of a->b
    double nx, ny;          // outward unit normal
    int32_t tag, pad;
};

struct BcTab {
    int32_t kind[CSW_MAXTAG];
    double par[CSW_MAXTAG][CSW_MAXPAR];
};

// step control words in device memory
struct Ctl {
    double t;        // time at the start of the current step
    double dt;       // step of the current step (0: inactive)
    unsigned long long lam_bits;  // max wave speed (bits of a non-negative double)
    double t_next;   // t + dt
    double cfl, t_end, dt_fixed, rmin;
    int32_t err;     // sticky error bits
    int32_t nflag;   // flagged-cell count of the last pass
    int32_t active;  // 1: kernels run; 0: step beyond t_end, kernels return
    float dtf;       // dt rounded to float (FP32-bulk stage update)
    long long nflag_sum;  // flagged cells summed over the limiter passes since the host last cleared it
};

// time t + tfac dt of the current stage, for boundary data.  The loads are
// volatile so that the FP64 arithmetic stays on the (rare) boundary-face path
// instead of being hoisted into every thread of an FP32 kernel.
__device__ __forceinline__ double stage_time(const Ctl *ctl, double tfac)
{
    const volatile Ctl *v = ctl;
    return v->t + tfac * v->dt;
}

// KXRCF precursors of a cell, written by the stage kernel for its new state
// (7 words per cell): the face means of the indicator variable on the three
// faces; per face the inflow weight (0 on an outflow face, where the mean
// velocity has v.n >= 0; |n~| on an inflow face to a neighbour, -|n~| on an
// inflow boundary face); the squared L2 coefficient norm of the indicator
// variable.  The stage kernel also checks the new means (ERR_NONPHYS).
enum { KX_I0 = 0, KX_I1, KX_I2, KX_W0, KX_W1, KX_W2, KX_NRM2, KX_COUNT };
// a cell's record is KX_STRIDE words: its own KX_COUNT words, then at KX_O0 + f
// the face mean that the neighbour across face f wrote for the shared face
// (so that the detection reads one record per cell and no neighbour's)
enum { KX_O0 = KX_COUNT, KX_STRIDE = 10 };

// geometry array indices (REAL, SoA with leading dimension ldc): 2 x inverse
// Jacobian; per face the outward unit normal and |n~| = 2 |e| / |K|; KXRCF scale
enum { G_RX = 0, G_RY, G_SX, G_SY, G_N0X, G_N0Y, G_N0L, G_N1X, G_N1Y, G_N1L, G_N2X, G_N2Y, G_N2L, G_KAPPA, G_COUNT };

// ---------------------------------------------------------------------------
// State layout in HBM: cell-major -- the NV*NP coefficients of cell c are
// contiguous, element (v, m) at [(c * NV + v) * NP + m] -- so that a cell (own
// or neighbour) is fetched with 16-byte (or 8-byte) vector loads.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ size_t sidx(int nv, int np, int v, int m, int c)
{
    return ((size_t)c * nv + v) * np + m;
}

template <typename R, int N> struct VecOf;  // widest aligned vector for a cell of N values
template <int N> struct VecOf<float, N> {
    static constexpr int W = (N % 4 == 0) ? 4 : (N % 2 == 0) ? 2 : 1;
};
template <int N> struct VecOf<double, N> {
    static constexpr int W = (N % 2 == 0) ? 2 : 1;
};

template <int NV, int NP, typename R>
__device__ __forceinline__ void load_cell(const R *__restrict__ p, int c, R (&u)[NV][NP])
{
    constexpr int N = NV * NP, W = VecOf<R, N>::W;
    R t[N];
    const R *q = p + (size_t)c * N;
    if (W == 4) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            const float4 x = __ldg(reinterpret_cast<const float4 *>(q) + i);
            t[4 * i] = x.x; t[4 * i + 1] = x.y; t[4 * i + 2] = x.z; t[4 * i + 3] = x.w;
        }
    } else if (W == 2 && sizeof(R) == 4) {
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            const float2 x = __ldg(reinterpret_cast<const float2 *>(q) + i);
            t[2 * i] = x.x; t[2 * i + 1] = x.y;
        }
    } else if (W == 2) {
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            const double2 x = __ldg(reinterpret_cast<const double2 *>(q) + i);
            t[2 * i] = (R)x.x; t[2 * i + 1] = (R)x.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) t[i] = __ldg(q + i);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int m = 0; m < NP; ++m) u[v][m] = t[v * NP + m];
}

// the NP coefficients of variable 0 of cell c (8-byte vector loads when aligned)
template <int NV, int NP, typename R>
__device__ __forceinline__ void load_var0(const R *__restrict__ p, int c, R (&a)[NP])
{
    const R *q = p + (size_t)c * NV * NP;
    if (sizeof(R) == 4 && (NV * NP) % 2 == 0 && NP % 2 == 0) {
#pragma unroll
        for (int i = 0; i < NP / 2; ++i) {
            const float2 x = __ldg(reinterpret_cast<const float2 *>(q) + i);
            a[2 * i] = (R)x.x;
            a[2 * i + 1] = (R)x.y;
        }
    } else {
#pragma unroll
        for (int m = 0; m < NP; ++m) a[m] = __ldg(q + m);
    }
}

template <int NV, int NP, typename R>
__device__ __forceinline__ void store_cell(R *p, int c, const R (&u)[NV][NP])
{
    constexpr int N = NV * NP, W = VecOf<R, N>::W;
    R *q = p + (size_t)c * N;
    if (W == 4) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i)
            reinterpret_cast<float4 *>(q)[i] = make_float4((float)u[(4 * i) / NP][(4 * i) % NP], (float)u[(4 * i + 1) / NP][(4 * i + 1) % NP],
                                                           (float)u[(4 * i + 2) / NP][(4 * i + 2) % NP],
                                                           (float)u[(4 * i + 3) / NP][(4 * i + 3) % NP]);
    } else if (W == 2 && sizeof(R) == 4) {
#pragma unroll
        for (int i = 0; i < N / 2; ++i)
            reinterpret_cast<float2 *>(q)[i] = make_float2((float)u[(2 * i) / NP][(2 * i) % NP], (float)u[(2 * i + 1) / NP][(2 * i + 1) % NP]);
    } else if (W == 2) {
#pragma unroll
        for (int i = 0; i < N / 2; ++i)
            reinterpret_cast<double2 *>(q)[i] = make_double2((double)u[(2 * i) / NP][(2 * i) % NP], (double)u[(2 * i + 1) / NP][(2 * i + 1) % NP]);
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) q[i] = u[i / NP][i % NP];
    }
}

// 8 KXRCF precursor words of cell c (32 or 64 bytes, vector stores / loads)
// records start at multiples of 40 (float) or 80 (double) bytes: 8-byte
// aligned in float, 16-byte aligned in double
template <typename R> __device__ __forceinline__ void store_kx(R *kx, int c, const R (&k)[KX_COUNT])
{
    R *q = kx + (size_t)c * KX_STRIDE;
    if (sizeof(R) == 4) {
#pragma unroll
        for (int i = 0; i < KX_COUNT / 2; ++i) reinterpret_cast<float2 *>(q)[i] = make_float2((float)k[2 * i], (float)k[2 * i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < KX_COUNT / 2; ++i) reinterpret_cast<double2 *>(q)[i] = make_double2((double)k[2 * i], (double)k[2 * i + 1]);
    }
    q[KX_COUNT - 1] = k[KX_COUNT - 1];
}
template <typename R> __device__ __forceinline__ void load_kx(const R *__restrict__ kx, int c, R (&k)[KX_STRIDE])
{
    const R *q = kx + (size_t)c * KX_STRIDE;
    if (sizeof(R) == 4) {
#pragma unroll
        for (int i = 0; i < KX_STRIDE / 2; ++i) {
            const float2 a = __ldg(reinterpret_cast<const float2 *>(q) + i);
            k[2 * i] = a.x; k[2 * i + 1] = a.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < KX_STRIDE / 2; ++i) {
            const double2 x = __ldg(reinterpret_cast<const double2 *>(q) + i);
            k[2 * i] = (R)x.x; k[2 * i + 1] = (R)x.y;
        }
    }
}

template <typename R> struct MeshDev {
    int nc;
    int ldc;
    const R *geo;           // [G_COUNT][ldc]
    const int32_t *nbr;     // [3][ldc]: >= 0 neighbour, < 0: -(bface+1)
    const uint8_t *nbf;     // [ldc]: neighbour local faces, 2 bits per face
    const BFace *bf;        // boundary faces
    const BcTab *bc;
    double gamma;
    R gammar;               // gamma in the state precision
};

}  // namespace csw
