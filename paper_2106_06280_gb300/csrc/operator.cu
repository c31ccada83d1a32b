// operator.cu -- the RKDG spatial operator fused with the SSP-RK stage update
// (Sec. 2, Eq. weakFormScheme2D with quadrature; Sec. 3.2, Eq. timeIntegrate),
// the CFL reduction, the initial-condition projection, conservation sums and
// the user-layout <-> internal-layout conversions.
//
// One thread per cell (owner-computes): a cell evaluates its volume integral
// and all three face integrals, reading its neighbours' modes (Morton order
// keeps them in L1/L2); the two cells of a face obtain exact negatives of one
// flux (llf2), so no face buffer in HBM, colouring or atomics are needed.
//
// State in HBM: cell-major [cell][var][mode], coefficients of the reference-orthonormal
// basis (u_tilde = sqrt(2/|K|) u_hat), so that
//   d u_tilde_i/dt = sum_q W_q grad_r psi_i . (G F(u_q))
//                   - sum_faces |n~| sum_g w_g psi_i(r_g) F*(u-, u+; n),
// with G = 2 (dr/dx, dr/dy, ds/dx, ds/dy), n the outward unit normal and
// |n~| = 2 |e| / |K|.
#include <mutex>

#include "../../include/cswdg.h"
#include "noalloc_limits.h"
#include "kernels.h"
#include "physics.cuh"
#include "tables.cuh"

namespace csw {

__constant__ Tab<float, 1> cT_f1;
__constant__ Tab<float, 2> cT_f2;
__constant__ Tab<double, 1> cT_d1;
__constant__ Tab<double, 2> cT_d2;

template <typename R, int K> __device__ __forceinline__ const Tab<R, K> &tab();
template <> __device__ __forceinline__ const Tab<float, 1> &tab<float, 1>() { return cT_f1; }
template <> __device__ __forceinline__ const Tab<float, 2> &tab<float, 2>() { return cT_f2; }
template <> __device__ __forceinline__ const Tab<double, 1> &tab<double, 1>() { return cT_d1; }
template <> __device__ __forceinline__ const Tab<double, 2> &tab<double, 2>() { return cT_d2; }

cudaError_t operator_upload_tables()
{
    static Tab<float, 1> f1;
    static Tab<float, 2> f2;
    static Tab<double, 1> d1;
    static Tab<double, 2> d2;
    make_tab(f1); make_tab(f2); make_tab(d1); make_tab(d2);
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(cT_f1, &f1, sizeof(f1))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(cT_f2, &f2, sizeof(f2))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(cT_d1, &d1, sizeof(d1))) != cudaSuccess) return e;
    return cudaMemcpyToSymbol(cT_d2, &d2, sizeof(d2));
}

// ---------------------------------------------------------------------------
// Largest wave speed of a cell mean (given as the four mean coefficients of
// psi_0 = sqrt(2)), in the state precision: sqrt(2)|u| (Burgers), |v| + c
// (Euler).  A NaN state gives 1e30, which forces a tiny step; the positivity
// check flags it.
template <int EQ, typename R> __device__ __forceinline__ R mean_wave_speed(const R *m0, R gam)
{
    const R is2 = R(0.70710678118654752440);
    if (EQ == BURGERS) return R(1.4142135623730951) * rabs(m0[0] * is2);
    const R r = m0[0] * is2, mx = m0[1] * is2, my = m0[2] * is2, E = m0[3] * is2;
    const R uu = mx / r, vv = my / r;
    const R p = (gam - R(1)) * (E - R(0.5) * (mx * uu + my * vv));
    const R lam = rsqroot(uu * uu + vv * vv) + rsqroot(gam * p / r);
    return (lam >= R(0)) ? lam : R(1e30);
}

// block-wide maximum of a non-negative value folded into ctl->lam_bits (the
// bits of a non-negative double order like the values); every thread of the
// block must call it
template <typename R> __device__ __forceinline__ void block_max_to_ctl(R lam, Ctl *ctl)
{
    for (int o = 16; o > 0; o >>= 1) lam = rmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
    __shared__ R sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = lam;
    __syncthreads();
    if (threadIdx.x == 0) {
        R m = sm[0];
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = rmax(m, sm[i]);
        atomicMax(&ctl->lam_bits, (unsigned long long)__double_as_longlong((double)m));
    }
}

// trace of the modes a at one point: the mean's share a0 (= a[v][0] psi_0) plus
// the higher modes in a fixed fused order, so that a cell's own trace and the
// same trace formed by its neighbour are equal bit for bit
template <int NV, int NP, typename R>
__device__ __forceinline__ void trace(const R (&a0)[NV], const R (&a)[NV][NP], const R *__restrict__ phi, R (&U)[NV])
{
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        R sv = a0[v];
#pragma unroll
        for (int m = 1; m < NP; ++m) sv = rfma(a[v][m], phi[m], sv);
        U[v] = sv;
    }
}

// one face point: twice the LLF flux between this cell's trace Ui (first) and
// the other side's Uo, through this cell's outward normal, weighted by
// wgt = w_g |n~| / 2 and taken off the residual against psi_i at the point
template <int NV, int NP, typename R>
__device__ __forceinline__ void face_scatter(const R (&F)[NV], R wgt, const R *__restrict__ phi, R (&acc)[NV][NP])
{
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const R wf = wgt * F[v];
#pragma unroll
        for (int m = 0; m < NP; ++m) acc[v][m] -= phi[m] * wf;
    }
}

template <int EQ, int NV, int NP, typename R>
__device__ __forceinline__ void face_point(const R (&Ui)[NV], const R (&Uo)[NV], R nx, R ny, R gam, R wgt,
                                           const R *__restrict__ phi, R (&acc)[NV][NP])
{
    R F[NV];
    llf2<EQ, R>(Ui, Uo, nx, ny, gam, F);
    face_scatter<NV, NP, R>(F, wgt, phi, acc);
}

// Stage kernel: out = ca*un + cb*up + (cl*dt)*L_h(up), L_h at t + tfac*dt.
// One thread per cell; each cell evaluates its volume integral and all three
// face integrals (the neighbour's trace is read from its modes), so no face
// buffer, colouring or atomics are needed.
// ---------------------------------------------------------------------------
// end of a cell's stage: the RK combination res = ca*un + cb*u + (cl*dt)*acc,
// its store, the KXRCF precursors of the new state (kx set) and, when lam_next
// is set, the largest wave speed of the new mean (else 0).  fg: (nx, ny, |n~|)
// of faces 0-2; fc0-fc2: neighbour codes; nbf: the neighbours' local faces.
template <int EQ, int K, typename R>
__device__ __forceinline__ R stage_finish(const MeshDev<R> &M, const R *un, R *out, R ca, R cb, R cl, int lam_next,
                                          R *__restrict__ kx, Ctl *__restrict__ ctl, int c,
                                          const R (&u)[Eqn<EQ>::NV][Deg<K>::NP], const R (&acc)[Eqn<EQ>::NV][Deg<K>::NP],
                                          const R (&fg)[9], int fc0, int fc1, int fc2, unsigned nbf)
{
    constexpr int NP = Deg<K>::NP, NV = Eqn<EQ>::NV;
    const Tab<R, K> &T = tab<R, K>();
    const R gam = M.gammar;
    const R cdt = cl * ((sizeof(R) == 4) ? (R)ctl->dtf : (R)ctl->dt);
    R res[NV][NP];
    if (un) {
        R w[NV][NP];
        load_cell<NV, NP>(un, c, w);
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int m = 0; m < NP; ++m) res[v][m] = cb * u[v][m] + cdt * acc[v][m] + ca * w[v][m];
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int m = 0; m < NP; ++m) res[v][m] = cb * u[v][m] + cdt * acc[v][m];
    }
    {
        store_cell<NV, NP>(out, c, res);
        // KXRCF precursors of the new state for the detection that follows
        if (kx) {
            R k7[KX_COUNT];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                R s = R(0);
#pragma unroll
                for (int m = 0; m < NP; ++m) s += res[0][m] * T.fint[f][m];
                k7[KX_I0 + f] = s;
            }
            R n2 = R(0);
#pragma unroll
            for (int m = 0; m < NP; ++m) n2 += res[0][m] * res[0][m];
            // reading R-pos: a polynomial that is non-physical at a quadrature point
            // makes the cell troubled.  Only the cheap bound runs here (one thread per
            // cell: the point-by-point check would stall whole warps); a cell that fails
            // it is handed to the detection as a candidate by a negated norm (n2 > 0
            // for any cell with a positive mean density)
            if constexpr (EQ == EULER)
                if (!physical_by_bound<K, R>(res, T)) n2 = -n2;
            k7[KX_NRM2] = n2;
            // the new means: physically admissible (Euler: rho > 0, p > 0; screened
            // in the state precision, close calls in double), and the mean velocity
            // direction (the momentum) that decides the inflow faces
            R vx, vy;
            if (EQ == EULER) {
                const R r = res[0][0], mx = res[1][0], my = res[2][0], E = res[NV - 1][0];
                const R q = R(2) * E * r - (mx * mx + my * my);
                bool ok = (r > R(0)) && (q > R(1e-3) * (R(2) * E * r));
                if (!ok && !(q != q)) {
                    const double rd = (double)r, mxd = (double)mx, myd = (double)my, Ed = (double)E;
                    ok = (rd > 0.0) && (2.0 * Ed * rd - (mxd * mxd + myd * myd) > 0.0);
                }
                if (!ok) atomicOr(&ctl->err, ERR_NONPHYS);
                vx = mx;
                vy = my;
            } else {
                vx = vy = res[0][0];
                if (!(vx == vx)) atomicOr(&ctl->err, ERR_NONPHYS);
            }
            // inflow weights: v.n < 0 (uncontracted, as a plain evaluation decides it)
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const R nx = fg[3 * f], ny = fg[3 * f + 1], nl = fg[3 * f + 2];
                const int code = (f == 0) ? fc0 : (f == 1) ? fc1 : fc2;
                const R vn = (EQ == BURGERS) ? vx * radd_rn(nx, ny) : radd_rn(rmul_rn(vx, nx), rmul_rn(vy, ny));
                k7[KX_W0 + f] = (vn < R(0)) ? ((code >= 0) ? nl : -nl) : R(0);
            }
            store_kx<R>(kx, c, k7);
            // this cell's face means also go to the neighbours' records, at the
            // slot of the shared face, so that the detection reads no neighbour
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const int code = (f == 0) ? fc0 : (f == 1) ? fc1 : fc2;
                if (code >= 0) kx[(size_t)code * KX_STRIDE + KX_O0 + ((nbf >> (2 * f)) & 3)] = k7[KX_I0 + f];
            }
        }
    }
    // last stage of a step: the largest wave speed of the new means, for the next
    // step's CFL rule (the reconstruction that follows keeps every cell mean)
    if (!lam_next) return R(0);
    R mn[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) mn[v] = res[v][0];
    return mean_wave_speed<EQ, R>(mn, gam);
}

// one cell of the stage; returns the largest wave speed of its new mean when
// lam_next is set (else 0)
template <int EQ, int K, typename R>
__device__ __forceinline__ R stage_cell(const MeshDev<R> &M, const R *un, const R *__restrict__ up, R *out, R ca, R cb, R cl,
                                        double tfac, int lam_next, R *__restrict__ kx, Ctl *__restrict__ ctl, int c)
{
    constexpr int NP = Deg<K>::NP, QV = Deg<K>::QV, QF = Deg<K>::QF, NV = Eqn<EQ>::NV;
    const Tab<R, K> &T = tab<R, K>();
    const int ld = M.ldc;
    const R gam = M.gammar;

    R u[NV][NP], acc[NV][NP];
    load_cell<NV, NP>(up, c, u);
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int m = 0; m < NP; ++m) acc[v][m] = R(0);
    const R g0 = M.geo[G_RX * ld + c], g1 = M.geo[G_RY * ld + c], g2 = M.geo[G_SX * ld + c], g3 = M.geo[G_SY * ld + c];
    // psi_0 is the same constant at every point: the mean's share of a trace is
    // formed once per cell (and once per neighbour), and every trace sum starts from it
    const R psi0 = T.vphi[0][0];
    R m0[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) m0[v] = u[v][0] * psi0;

    // the neighbour ids and the face normals are loaded with the cell's own data,
    // so that a face waits only for its neighbour's modes (one round trip)
    const int fc0 = M.nbr[c], fc1 = M.nbr[ld + c], fc2 = M.nbr[2 * ld + c];
    R fg[9];  // (nx, ny, |n~|) of faces 0, 1, 2
#pragma unroll
    for (int i = 0; i < 9; ++i) fg[i] = M.geo[(G_N0X + i) * ld + c];

    // volume integral
#pragma unroll
    for (int q = 0; q < QV; ++q) {
        R U[NV], f[NV], g[NV];
        trace<NV, NP, R>(m0, u, T.vphi[q], U);
        flux_fg<EQ, R>(U, gam, f, g);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const R Fr = g0 * f[v] + g1 * g[v];
            const R Fs = g2 * f[v] + g3 * g[v];
            // psi_0 is constant and psi_1..psi_K (Jacobi index i = 0) do not depend on r:
            // their derivative terms are exact zeros and are skipped; the volume
            // weight is folded into the derivative tables
#pragma unroll
            for (int m = 1; m < NP; ++m) acc[v][m] += (m > K) ? T.vdrw[q][m] * Fr + T.vdsw[q][m] * Fs : T.vdsw[q][m] * Fs;
        }
    }

    // face integrals: -|n~| sum_g w_g psi_i F*(u-, u+; n), n this cell's outward unit
    // normal; llf2 returns 2 F*, so the face factor carries 1/2 |n~|
    const unsigned nbf = M.nbf[c];
    // the face loop is not unrolled (the fully unrolled body ran slower:
    // instruction-cache misses and register pressure); its Gauss points are
#pragma unroll 1
    for (int f = 0; f < 3; ++f) {
        // selected, not indexed: an indexed register array would go to local memory
        const R nx = (f == 0) ? fg[0] : (f == 1) ? fg[3] : fg[6], ny = (f == 0) ? fg[1] : (f == 1) ? fg[4] : fg[7];
        const R hnl = R(0.5) * ((f == 0) ? fg[2] : (f == 1) ? fg[5] : fg[8]);
        const int code = (f == 0) ? fc0 : (f == 1) ? fc1 : fc2;
        if (code >= 0) {
            // interior face: the neighbour's trace from its modes, at the reversed
            // point of its local face nf
            const int nf = (nbf >> (2 * f)) & 3;
            R w[NV][NP], w0[NV];
            load_cell<NV, NP>(up, code, w);
#pragma unroll
            for (int v = 0; v < NV; ++v) w0[v] = w[v][0] * psi0;
#pragma unroll
            for (int g = 0; g < QF; ++g) {
                R Ui[NV], Uo[NV];
                trace<NV, NP, R>(m0, u, T.fphi[f][g], Ui);
                trace<NV, NP, R>(w0, w, T.fphi[nf][QF - 1 - g], Uo);
                face_point<EQ, NV, NP, R>(Ui, Uo, nx, ny, gam, T.fw[g] * hnl, T.fphi[f][g], acc);
            }
        } else {
            const BFace bf = M.bf[-code - 1];
            // a transmissive face takes the cell mean as the outside state (reading R-bc)
            const bool transmissive = M.bc->kind[bf.tag] == BC_TRANSMISSIVE;
#pragma unroll
            for (int g = 0; g < QF; ++g) {
                R Ui[NV], Uo[NV];
                trace<NV, NP, R>(m0, u, T.fphi[f][g], Ui);
                if (transmissive) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) Uo[v] = m0[v];
                } else {
                    ghost<EQ, R>(bf, M.bc, (double)T.ft[g], stage_time(ctl, tfac), Ui, Uo);
                }
                face_point<EQ, NV, NP, R>(Ui, Uo, nx, ny, gam, T.fw[g] * hnl, T.fphi[f][g], acc);
            }
        }
    }

    return stage_finish<EQ, K, R>(M, un, out, ca, cb, cl, lam_next, kx, ctl, c, u, acc, fg, fc0, fc1, fc2, nbf);
}

// Stage kernel: tiles of BLK consecutive cells (Morton order), one thread per
// cell; a block takes tiles blockIdx.x, blockIdx.x + gridDim.x, ... (the grid
// is either one block per tile or a persistent grid sized to the SMs, chosen by
// cswdg_autotune).
template <int EQ, int K, typename R, int BLK>
__global__ void __launch_bounds__(BLK, (sizeof(R) == 4) ? 512 / BLK : 1)
    k_stage(MeshDev<R> M, const R *un, const R *__restrict__ up, R *out, R ca, R cb, R cl, double tfac, int lam_next,
            R *__restrict__ kx, Ctl *__restrict__ ctl)
{
    if (!ctl->active) return;
    // the detection that follows this stage counts its flagged cells from zero
    // (a step beyond t_end keeps the count of the last active pass)
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->nflag = 0;
    const int ntiles = (M.nc + BLK - 1) / BLK;
    R lam = R(0);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int c = tile * BLK + threadIdx.x;
        if (c < M.nc) lam = rmax(lam, stage_cell<EQ, K, R>(M, un, up, out, ca, cb, cl, tfac, lam_next, kx, ctl, c));
    }
    if (lam_next) block_max_to_ctl<R>(lam, ctl);  // every thread of the block gets here
}

// ---------------------------------------------------------------------------
// Tile-shared stage kernel: the same stage as k_stage, with each face's work
// done once per tile.  A block takes a tile of BLK consecutive cells (Morton
// order) in three phases separated by block barriers:
//   1. every cell writes its traces at its 3 x QF face points to the shared
//      array S (slot (f, g) of cell a at S[((f * QF + g) * BLK + a) * NV]);
//   2. a face-parallel pass over the tile's face list.  A face between two
//      cells of the tile (listed once, by its lower-index cell a) reads both
//      traces and computes 2F = llf2(U_a, U_b, n_a) once: F goes into a's slot
//      and -F into b's slot at the matching point, which is what b's own call
//      llf2(U_b, U_a, -n_a) returns bit for bit (each slot belongs to one face,
//      so fluxes overwrite traces in place).  Where b's stored normal is not
//      the exact negative of a's (a periodic face), b's flux is computed from
//      its own normal.  A face to a cell of another tile forms that cell's
//      trace from its modes, a boundary face its ghost, as k_stage does;
//   3. every cell evaluates its volume integral, takes the fluxes off its
//      residual from its own slots in k_stage's order and finishes the stage.
// The list holds the tile's interior faces, then those to other tiles, then
// the boundary faces, so the warps of the face pass mostly run one kind.  The
// result equals k_stage's bit for bit.
template <int NV, typename R> __device__ __forceinline__ void sput(R *s, const R (&U)[NV])
{
    if constexpr (NV == 4 && sizeof(R) == 4) {
        *reinterpret_cast<float4 *>(s) = make_float4(U[0], U[1], U[2], U[3]);
    } else if constexpr (NV == 4) {
        reinterpret_cast<double2 *>(s)[0] = make_double2(U[0], U[1]);
        reinterpret_cast<double2 *>(s)[1] = make_double2(U[2], U[3]);
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) s[v] = U[v];
    }
}
template <int NV, typename R> __device__ __forceinline__ void sget(const R *s, R (&U)[NV])
{
    if constexpr (NV == 4 && sizeof(R) == 4) {
        const float4 x = *reinterpret_cast<const float4 *>(s);
        U[0] = x.x; U[1] = x.y; U[2] = x.z; U[3] = x.w;
    } else if constexpr (NV == 4) {
        const double2 x = reinterpret_cast<const double2 *>(s)[0], y = reinterpret_cast<const double2 *>(s)[1];
        U[0] = x.x; U[1] = x.y; U[2] = y.x; U[3] = y.y;
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) U[v] = s[v];
    }
}

// shared memory of one block of the tile-shared kernel (bytes): the slots, the
// cells' face normals (3 BLK pairs), neighbour codes (3 BLK), the face list
// (3 BLK entries) and the per-warp counts
template <int EQ, int K, typename R> constexpr size_t tile_smem_bytes(int blk)
{
    return (size_t)3 * Deg<K>::QF * blk * Eqn<EQ>::NV * sizeof(R) + (size_t)6 * blk * sizeof(R) + (size_t)6 * blk * sizeof(int) +
           32 * sizeof(int);
}

template <int EQ, int K, typename R, int BLK>
__global__ void __launch_bounds__(BLK, (sizeof(R) == 4) ? 512 / BLK : 1)
    k_stage_tiles(MeshDev<R> M, const R *un, const R *__restrict__ up, R *out, R ca, R cb, R cl, double tfac, int lam_next,
                  R *__restrict__ kx, Ctl *__restrict__ ctl)
{
    constexpr int NP = Deg<K>::NP, QV = Deg<K>::QV, QF = Deg<K>::QF, NV = Eqn<EQ>::NV;
    static_assert(BLK <= 256, "face-list counts are packed in 10-bit fields");
    extern __shared__ __align__(16) unsigned char tile_smem[];
    R *S = reinterpret_cast<R *>(tile_smem);
    R *nrm = S + (size_t)3 * QF * BLK * NV;  // (nx, ny) of face f of cell a at nrm[2 (f BLK + a)]
    int *codes = reinterpret_cast<int *>(nrm + 6 * BLK);  // neighbour code of face f of cell a at codes[f BLK + a]
    int *jobs = codes + 3 * BLK;
    int *wtot = jobs + 3 * BLK;
    auto slot = [&](int f, int g, int a) { return S + ((size_t)(f * QF + g) * BLK + a) * NV; };

    if (!ctl->active) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->nflag = 0;
    const Tab<R, K> &T = tab<R, K>();
    const int ld = M.ldc;
    const R gam = M.gammar;
    const R psi0 = T.vphi[0][0];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int ntiles = (M.nc + BLK - 1) / BLK;
    R lam = R(0);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int c0 = tile * BLK, c = c0 + t;
        const bool valid = c < M.nc;
        R u[NV][NP];
        R fg[9], g0 = R(0), g1 = R(0), g2 = R(0), g3 = R(0);
        int fc0 = -1, fc1 = -1, fc2 = -1;
        unsigned nbf = 0;
        if (valid) {
            load_cell<NV, NP>(up, c, u);
            fc0 = M.nbr[c]; fc1 = M.nbr[ld + c]; fc2 = M.nbr[2 * ld + c];
            nbf = M.nbf[c];
#pragma unroll
            for (int i = 0; i < 9; ++i) fg[i] = M.geo[(G_N0X + i) * ld + c];
            g0 = M.geo[G_RX * ld + c]; g1 = M.geo[G_RY * ld + c]; g2 = M.geo[G_SX * ld + c]; g3 = M.geo[G_SY * ld + c];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                nrm[2 * (f * BLK + t)] = fg[3 * f];
                nrm[2 * (f * BLK + t) + 1] = fg[3 * f + 1];
                codes[f * BLK + t] = (f == 0) ? fc0 : (f == 1) ? fc1 : fc2;
            }
        }
        // face list: counts of interior (taken by the lower-index cell), outer and
        // boundary faces packed in 10-bit fields, one block-wide exclusive scan
        unsigned cnt = 0;
        if (valid) {
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const int code = (f == 0) ? fc0 : (f == 1) ? fc1 : fc2;
                const int b = code - c0;
                // a face to itself (b == t) goes to the outer list, computed per side
                cnt += (code < 0) ? (1u << 20) : (b >= 0 && b < BLK && b != t) ? ((b > t) ? 1u : 0u) : (1u << 10);
            }
        }
        unsigned inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wtot[warp] = (int)inc;
        // phase 1: own traces at the face points
        if (valid) {
            R m0[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) m0[v] = u[v][0] * psi0;
#pragma unroll
            for (int f = 0; f < 3; ++f)
#pragma unroll
                for (int g = 0; g < QF; ++g) {
                    R Ui[NV];
                    trace<NV, NP, R>(m0, u, T.fphi[f][g], Ui);
                    sput<NV, R>(slot(f, g, t), Ui);
                }
        }
        __syncthreads();
        unsigned pre = 0, tot = 0;
        for (int w = 0; w < BLK / 32; ++w) {
            const unsigned x = (unsigned)wtot[w];
            if (w < warp) pre += x;
            tot += x;
        }
        const unsigned exc = pre + inc - cnt;
        const int nint = (int)(tot & 1023u), nout = (int)((tot >> 10) & 1023u), nall = nint + nout + (int)(tot >> 20);
        if (valid) {
            int pi = (int)(exc & 1023u), po = nint + (int)((exc >> 10) & 1023u), pb = nint + nout + (int)(exc >> 20);
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const int code = (f == 0) ? fc0 : (f == 1) ? fc1 : fc2;
                // entry: cell a (8 bits), face f (2), the neighbour's local face nf (2),
                // the neighbour's index in the tile b (8; interior faces)
                const int b = code - c0, nf = (int)((nbf >> (2 * f)) & 3u);
                const int job = t | (f << 8) | (nf << 10) | ((b & 255) << 12);
                if (code < 0) jobs[pb++] = job;
                else if (b >= 0 && b < BLK && b != t) { if (b > t) jobs[pi++] = job; }
                else jobs[po++] = job;
            }
        }
        __syncthreads();
        // phase 2: the face pass
        for (int j = t; j < nall; j += BLK) {
            const int job = jobs[j];
            const int a = job & 255, f = (job >> 8) & 3, nf = (job >> 10) & 3, ca_ = c0 + a;
            const R nx = nrm[2 * (f * BLK + a)], ny = nrm[2 * (f * BLK + a) + 1];
            if (j < nint) {
                const int b = (job >> 12) & 255;
                const R bx = nrm[2 * (nf * BLK + b)], by = nrm[2 * (nf * BLK + b) + 1];
                const bool mirrored = (bx == -nx) && (by == -ny);
#pragma unroll
                for (int g = 0; g < QF; ++g) {
                    R Ua[NV], Ub[NV], F[NV];
                    sget<NV, R>(slot(f, g, a), Ua);
                    sget<NV, R>(slot(nf, QF - 1 - g, b), Ub);
                    llf2<EQ, R>(Ua, Ub, nx, ny, gam, F);
                    R Fb[NV];
                    if (mirrored) {
#pragma unroll
                        for (int v = 0; v < NV; ++v) Fb[v] = -F[v];
                    } else {
                        llf2<EQ, R>(Ub, Ua, bx, by, gam, Fb);
                    }
                    sput<NV, R>(slot(f, g, a), F);
                    sput<NV, R>(slot(nf, QF - 1 - g, b), Fb);
                }
            } else if (j < nint + nout) {
                const int code = codes[f * BLK + a];
                R w[NV][NP], w0[NV];
                load_cell<NV, NP>(up, code, w);
#pragma unroll
                for (int v = 0; v < NV; ++v) w0[v] = w[v][0] * psi0;
#pragma unroll
                for (int g = 0; g < QF; ++g) {
                    R Ua[NV], Ub[NV], F[NV];
                    sget<NV, R>(slot(f, g, a), Ua);
                    trace<NV, NP, R>(w0, w, T.fphi[nf][QF - 1 - g], Ub);
                    llf2<EQ, R>(Ua, Ub, nx, ny, gam, F);
                    sput<NV, R>(slot(f, g, a), F);
                }
            } else {
                const BFace bf = M.bf[-codes[f * BLK + a] - 1];
                const bool transmissive = M.bc->kind[bf.tag] == BC_TRANSMISSIVE;
                R m0[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) m0[v] = up[((size_t)ca_ * NV + v) * NP] * psi0;
#pragma unroll
                for (int g = 0; g < QF; ++g) {
                    R Ua[NV], Uo[NV], F[NV];
                    sget<NV, R>(slot(f, g, a), Ua);
                    if (transmissive) {
#pragma unroll
                        for (int v = 0; v < NV; ++v) Uo[v] = m0[v];
                    } else {
                        ghost<EQ, R>(bf, M.bc, (double)T.ft[g], stage_time(ctl, tfac), Ua, Uo);
                    }
                    llf2<EQ, R>(Ua, Uo, nx, ny, gam, F);
                    sput<NV, R>(slot(f, g, a), F);
                }
            }
        }
        __syncthreads();
        // phase 3: volume integral, the fluxes from this cell's slots, the update
        if (valid) {
            R acc[NV][NP];
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int m = 0; m < NP; ++m) acc[v][m] = R(0);
            R m0[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) m0[v] = u[v][0] * psi0;
#pragma unroll
            for (int q = 0; q < QV; ++q) {
                R U[NV], f_[NV], g_[NV];
                trace<NV, NP, R>(m0, u, T.vphi[q], U);
                flux_fg<EQ, R>(U, gam, f_, g_);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const R Fr = g0 * f_[v] + g1 * g_[v];
                    const R Fs = g2 * f_[v] + g3 * g_[v];
#pragma unroll
                    for (int m = 1; m < NP; ++m) acc[v][m] += (m > K) ? T.vdrw[q][m] * Fr + T.vdsw[q][m] * Fs : T.vdsw[q][m] * Fs;
                }
            }
#pragma unroll 1
            for (int f = 0; f < 3; ++f) {
                const R hnl = R(0.5) * ((f == 0) ? fg[2] : (f == 1) ? fg[5] : fg[8]);
#pragma unroll
                for (int g = 0; g < QF; ++g) {
                    R F[NV];
                    sget<NV, R>(slot(f, g, t), F);
                    face_scatter<NV, NP, R>(F, T.fw[g] * hnl, T.fphi[f][g], acc);
                }
            }
            lam = rmax(lam, stage_finish<EQ, K, R>(M, un, out, ca, cb, cl, lam_next, kx, ctl, c, u, acc, fg, fc0, fc1, fc2, nbf));
        }
    }
    if (lam_next) block_max_to_ctl<R>(lam, ctl);  // every thread of the block gets here
}

// dynamic shared memory limits of the tile-shared kernels (above the 48 KB
// default for 256-cell tiles of the Euler state) on the current device
template <int EQ, int K, typename R> cudaError_t tile_smem_attr()
{
    cudaError_t e = cudaFuncSetAttribute(k_stage_tiles<EQ, K, R, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tile_smem_bytes<EQ, K, R>(128));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_stage_tiles<EQ, K, R, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tile_smem_bytes<EQ, K, R>(256));
}
cudaError_t stage_kernels_prepare()
{
    cudaError_t e;
    if ((e = tile_smem_attr<BURGERS, 1, float>()) != cudaSuccess) return e;
    if ((e = tile_smem_attr<BURGERS, 2, float>()) != cudaSuccess) return e;
    if ((e = tile_smem_attr<EULER, 1, float>()) != cudaSuccess) return e;
    if ((e = tile_smem_attr<EULER, 2, float>()) != cudaSuccess) return e;
    if ((e = tile_smem_attr<BURGERS, 1, double>()) != cudaSuccess) return e;
    if ((e = tile_smem_attr<BURGERS, 2, double>()) != cudaSuccess) return e;
    if ((e = tile_smem_attr<EULER, 1, double>()) != cudaSuccess) return e;
    return tile_smem_attr<EULER, 2, double>();
}

template <int EQ, int K, typename R>
void launch_stage_t(const MeshDev<R> &M, const R *un, const R *up, R *out, R ca, R cb, R cl, double tfac, int lam_next, R *kx,
                    Ctl *ctl, StageShape sh, cudaStream_t st)
{
    const int blk = (sh.blk == 64 || sh.blk == 256) ? sh.blk : 128;
    const int ntiles = (M.nc + blk - 1) / blk;
    const int grd = (sh.grid > 0 && sh.grid < ntiles) ? sh.grid : ntiles;
    if (sh.tile_faces && blk != 64) {
        const size_t sm = tile_smem_bytes<EQ, K, R>(blk);
        if (blk == 256) k_stage_tiles<EQ, K, R, 256><<<grd, 256, sm, st>>>(M, un, up, out, ca, cb, cl, tfac, lam_next, kx, ctl);
        else k_stage_tiles<EQ, K, R, 128><<<grd, 128, sm, st>>>(M, un, up, out, ca, cb, cl, tfac, lam_next, kx, ctl);
        return;
    }
    if (blk == 64) k_stage<EQ, K, R, 64><<<grd, 64, 0, st>>>(M, un, up, out, ca, cb, cl, tfac, lam_next, kx, ctl);
    else if (blk == 256) k_stage<EQ, K, R, 256><<<grd, 256, 0, st>>>(M, un, up, out, ca, cb, cl, tfac, lam_next, kx, ctl);
    else k_stage<EQ, K, R, 128><<<grd, 128, 0, st>>>(M, un, up, out, ca, cb, cl, tfac, lam_next, kx, ctl);
}

template <typename R>
void launch_stage(int eq, int k, const MeshDev<R> &M, const R *un, const R *up, R *out, R ca, R cb, R cl, double tfac,
                  int lam_next, R *kx, Ctl *ctl, StageShape sh, cudaStream_t st)
{
    if (eq == BURGERS && k == 1) launch_stage_t<BURGERS, 1, R>(M, un, up, out, ca, cb, cl, tfac, lam_next, kx, ctl, sh, st);
    else if (eq == BURGERS && k == 2) launch_stage_t<BURGERS, 2, R>(M, un, up, out, ca, cb, cl, tfac, lam_next, kx, ctl, sh, st);
    else if (eq == EULER && k == 1) launch_stage_t<EULER, 1, R>(M, un, up, out, ca, cb, cl, tfac, lam_next, kx, ctl, sh, st);
    else launch_stage_t<EULER, 2, R>(M, un, up, out, ca, cb, cl, tfac, lam_next, kx, ctl, sh, st);
}
template void launch_stage<float>(int, int, const MeshDev<float> &, const float *, const float *, float *, float, float, float,
                                  double, int, float *, Ctl *, StageShape, cudaStream_t);
template void launch_stage<double>(int, int, const MeshDev<double> &, const double *, const double *, double *, double, double,
                                   double, double, int, double *, Ctl *, StageShape, cudaStream_t);

// ---------------------------------------------------------------------------
// Time step control.  Max wave speed of the cell means (exact max, order free),
// then dt = cfl * rmin / lambda_max clipped to t_end (one thread).
// ---------------------------------------------------------------------------
template <int EQ, typename R>
__global__ void __launch_bounds__(256) k_cfl_max(MeshDev<R> M, int np, const R *__restrict__ u, Ctl *ctl)
{
    // largest wave speed of the cell means in the state precision (an exact
    // maximum, independent of the reduction order)
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    R lam = R(0);
    if (c < M.nc) {
        R m0[4];
        const int nv = (EQ == BURGERS) ? 1 : 4;
        for (int v = 0; v < nv; ++v) m0[v] = u[sidx(nv, np, v, 0, c)];
        lam = mean_wave_speed<EQ, R>(m0, M.gammar);
    }
    block_max_to_ctl<R>(lam, ctl);
}

// begin a step: t <- t_next, choose dt (fixed or CFL), clip to t_end
__global__ void k_begin_step(Ctl *ctl, int use_cfl)
{
    ctl->t = ctl->t_next;
    double dt = ctl->dt_fixed;
    if (use_cfl) {
        const double lam = __longlong_as_double((long long)ctl->lam_bits);
        dt = (lam > 0.0) ? ctl->cfl * ctl->rmin / lam : 0.0;
    }
    const double rem = ctl->t_end - ctl->t;
    if (dt > rem) dt = rem;
    if (!(dt > 0.0)) dt = 0.0;
    ctl->dt = dt;
    ctl->dtf = (float)dt;
    ctl->active = dt > 0.0;
    ctl->t_next = ctl->t + dt;
    // the last stage of an active step folds the next maximum into lam_bits; an
    // inactive step leaves the state, and so its maximum, unchanged
    if (dt > 0.0) ctl->lam_bits = 0ull;
}

template <typename R> void launch_cfl(int eq, const MeshDev<R> &M, int np, const R *u, Ctl *ctl, cudaStream_t st)
{
    const int blk = 256, grd = (M.nc + blk - 1) / blk;
    if (eq == BURGERS) k_cfl_max<BURGERS, R><<<grd, blk, 0, st>>>(M, np, u, ctl);
    else k_cfl_max<EULER, R><<<grd, blk, 0, st>>>(M, np, u, ctl);
}
template void launch_cfl<float>(int, const MeshDev<float> &, int, const float *, Ctl *, cudaStream_t);
template void launch_cfl<double>(int, const MeshDev<double> &, int, const double *, Ctl *, cudaStream_t);

// the step parameters of a cswdg_step call, set on the stream (no host round trip)
__global__ void k_set_step_params(Ctl *ctl, double dt_fixed, double cfl, double t_end)
{
    ctl->dt_fixed = dt_fixed;
    ctl->cfl = cfl;
    ctl->t_end = t_end;
}
void launch_set_step_params(Ctl *ctl, double dt_fixed, double cfl, double t_end, cudaStream_t st)
{
    k_set_step_params<<<1, 1, 0, st>>>(ctl, dt_fixed, cfl, t_end);
}

void launch_begin_step(Ctl *ctl, int use_cfl, cudaStream_t st) { k_begin_step<<<1, 1, 0, st>>>(ctl, use_cfl); }

// ---------------------------------------------------------------------------
// Initial condition: u_tilde_i = 2 sum_q W_q u(x_q) psi_i(r_q) (volume rule).
// vals: internal order, [cell][q][var] doubles.
// ---------------------------------------------------------------------------
template <int K, typename R>
__global__ void k_project(int nc, int ld, int nv, const double *__restrict__ vals, R *__restrict__ u)
{
    constexpr int NP = Deg<K>::NP, QV = Deg<K>::QV;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const Tab<double, K> &T = tab<double, K>();
    for (int v = 0; v < nv; ++v)
        for (int m = 0; m < NP; ++m) {
            double s = 0.0;
            for (int q = 0; q < QV; ++q) s += T.vw[q] * vals[((size_t)c * QV + q) * nv + v] * T.vphi[q][m];
            u[sidx(nv, NP, v, m, c)] = (R)(2.0 * s);
        }
}

template <typename R> void launch_project(int k, int nc, int ld, int nv, const double *vals, R *u, cudaStream_t st)
{
    const int blk = 128, grd = (nc + blk - 1) / blk;
    if (k == 1) k_project<1, R><<<grd, blk, 0, st>>>(nc, ld, nv, vals, u);
    else k_project<2, R><<<grd, blk, 0, st>>>(nc, ld, nv, vals, u);
}
template void launch_project<float>(int, int, int, int, const double *, float *, cudaStream_t);
template void launch_project<double>(int, int, int, int, const double *, double *, cudaStream_t);

// ---------------------------------------------------------------------------
// Layout conversions.  user[(uc*nv + v)*np + m] (double, physical basis) <->
// internal [(c*nv + v)*np + m], scaled by sc[c] = sqrt(2/|K|); perm[c] = user index.
// ---------------------------------------------------------------------------
template <typename R, typename U>
__global__ void __launch_bounds__(256) k_from_user(int nc, int ld, int nv, int np, const int32_t *__restrict__ perm,
                                                   const double *__restrict__ sc, const U *__restrict__ user, R *__restrict__ u)
{
    // one thread per coefficient: a warp covers consecutive coefficients of one
    // or two cells, so the reads of the cell's user row and the writes of its
    // internal row are both contiguous
    const int npv = nv * np;
    const size_t n = (size_t)nc * npv;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / npv), j = (int)(e - (size_t)c * npv);
        u[e] = (R)(sc[c] * (double)user[(size_t)perm[c] * npv + j]);
    }
}

template <typename R, typename U>
__global__ void __launch_bounds__(256) k_to_user(int nc, int ld, int nv, int np, const int32_t *__restrict__ perm,
                                                 const double *__restrict__ sc, const R *__restrict__ u, U *__restrict__ user)
{
    const int npv = nv * np;
    const size_t n = (size_t)nc * npv;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / npv), j = (int)(e - (size_t)c * npv);
        user[(size_t)perm[c] * npv + j] = (U)((1.0 / sc[c]) * (double)u[e]);
    }
}

__global__ void k_flags_to_user(int nc, const int32_t *__restrict__ perm, const uint8_t *__restrict__ fl, uint8_t *__restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nc) out[perm[c]] = fl[c];
}

template <typename R, typename U>
void launch_from_user(int nc, int ld, int nv, int np, const int32_t *perm, const double *sc, const U *user, R *u, cudaStream_t st)
{
    const size_t n = (size_t)nc * nv * np;
    const int grd = (int)std::min<size_t>((n + 255) / 256, 16384);
    k_from_user<R, U><<<grd, 256, 0, st>>>(nc, ld, nv, np, perm, sc, user, u);
}
template <typename R, typename U>
void launch_to_user(int nc, int ld, int nv, int np, const int32_t *perm, const double *sc, const R *u, U *user, cudaStream_t st)
{
    const size_t n = (size_t)nc * nv * np;
    const int grd = (int)std::min<size_t>((n + 255) / 256, 16384);
    k_to_user<R, U><<<grd, 256, 0, st>>>(nc, ld, nv, np, perm, sc, u, user);
}
#define CSW_UL(R, U)                                                                                                         \
    template void launch_from_user<R, U>(int, int, int, int, const int32_t *, const double *, const U *, R *, cudaStream_t); \
    template void launch_to_user<R, U>(int, int, int, int, const int32_t *, const double *, const R *, U *, cudaStream_t);
CSW_UL(float, double)
CSW_UL(double, double)
CSW_UL(float, float)
CSW_UL(double, float)
#undef CSW_UL

void launch_flags_to_user(int nc, const int32_t *perm, const uint8_t *fl, uint8_t *out, cudaStream_t st)
{
    k_flags_to_user<<<(nc + 255) / 256, 256, 0, st>>>(nc, perm, fl, out);
}

// ---------------------------------------------------------------------------
// Conservation sums sum_K |K| mean_K = sum_K |K| u_tilde_0 / sqrt(2):
// per-block partial sums, then one block adds them in a fixed order.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_cons_partial(int nc, int ld, int nv, int np, const double *__restrict__ area, const R *__restrict__ u,
                               double *__restrict__ part)
{
    __shared__ double sm[256];
    for (int v = 0; v < nv; ++v) {
        const int c = blockIdx.x * blockDim.x + threadIdx.x;
        sm[threadIdx.x] = (c < nc) ? area[c] * (double)u[sidx(nv, np, v, 0, c)] * 0.70710678118654752440 : 0.0;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(size_t)v * gridDim.x + blockIdx.x] = sm[0];
        __syncthreads();
    }
}

__global__ void k_cons_final(int nblk, int nv, const double *__restrict__ part, double *__restrict__ out)
{
    if (threadIdx.x != 0) return;
    for (int v = 0; v < nv; ++v) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[(size_t)v * nblk + b];
        out[v] = s;
    }
}

template <typename R>
void launch_conservation(int nc, int ld, int nv, int np, const double *area, const R *u, double *part, double *out, cudaStream_t st)
{
    const int nblk = (nc + 255) / 256;
    k_cons_partial<R><<<nblk, 256, 0, st>>>(nc, ld, nv, np, area, u, part);
    k_cons_final<<<1, 32, 0, st>>>(nblk, nv, part, out);
}
template void launch_conservation<float>(int, int, int, int, const double *, const float *, double *, double *, cudaStream_t);
template void launch_conservation<double>(int, int, int, int, const double *, const double *, double *, double *, cudaStream_t);

}  // namespace csw

// ---------------------------------------------------------------------------
// Allocation-free conservation sums.  The per-block partial sums live in this
// file-scope device array instead of a buffer allocated per solver; every GPU
// that loads the library holds it (2 MiB) until the process exits.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_partial[CSW_NOALLOC_MAX_BLOCKS * CSW_NOALLOC_MAX_VARS];

namespace {
constexpr int kMaxDevices = 64;
// device address of g_noalloc_partial on each device, looked up once per device
std::once_flag g_noalloc_once[kMaxDevices];
double *g_noalloc_ptr[kMaxDevices] = {nullptr};
cudaError_t g_noalloc_err[kMaxDevices] = {cudaSuccess};

// makes `dev` current for the lifetime of the guard and restores the caller's device
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev)
    {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
        else if (err == cudaSuccess) prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};
}  // namespace

extern "C" cswdg_status cswdg_conservation_noalloc(cswdg_solver *s, const void *modes_dev, double *sums_dev)
{
    int nc = 0, ld = 0, nv = 0, np = 0, fp32 = 0, dev = -1;
    const double *area = nullptr;
    cudaStream_t st = nullptr;
    if (!csw::solver_view(s, &nc, &ld, &nv, &np, &fp32, &area, (void **)&st, &dev) || !modes_dev || !sums_dev)
        return csw::solver_fail(s, CSWDG_EINVAL, "conservation_noalloc: no mesh or null pointer");
    if (!csw_noalloc_fits(nc, nv))
        return csw::solver_fail(s, CSWDG_EINVAL, "conservation_noalloc: %d cells exceed the fixed scratch (at most %d cells)", nc,
                                CSW_NOALLOC_MAX_BLOCKS * CSW_NOALLOC_CELLS_PER_BLOCK);
    if (dev < 0 || dev >= kMaxDevices) return csw::solver_fail(s, CSWDG_ECUDA, "conservation_noalloc: solver device %d", dev);
    // the solver's device is current for the look-up and the launches (its stream belongs to it)
    DeviceGuard guard(dev);
    if (guard.err != cudaSuccess)
        return csw::solver_fail(s, CSWDG_ECUDA, "conservation_noalloc: cudaSetDevice(%d): %s", dev, cudaGetErrorString(guard.err));
    std::call_once(g_noalloc_once[dev], [dev] {
        double *ptr = nullptr;
        g_noalloc_err[dev] = cudaGetSymbolAddress((void **)&ptr, g_noalloc_partial);
        g_noalloc_ptr[dev] = ptr;
    });
    if (g_noalloc_err[dev] != cudaSuccess || !g_noalloc_ptr[dev])
        return csw::solver_fail(s, CSWDG_ECUDA, "conservation_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(g_noalloc_err[dev]));
    if (fp32)
        csw::launch_conservation<float>(nc, ld, nv, np, area, (const float *)modes_dev, g_noalloc_ptr[dev], sums_dev, st);
    else
        csw::launch_conservation<double>(nc, ld, nv, np, area, (const double *)modes_dev, g_noalloc_ptr[dev], sums_dev, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return csw::solver_fail(s, CSWDG_ECUDA, "conservation_noalloc: %s", cudaGetErrorString(e));
    return CSWDG_OK;
}

// ---------------------------------------------------------------------------
// FP64 FMA throughput probe: the ceiling of the FP64-pipe-bound work (the
// FP64 mode and the double smoothness-indicator and weight arithmetic of the
// reconstruction).  Every thread runs 8 independent FMA chains; the grid fills
// every SM several times over.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_probe_dfma(int iters, double b, double c, double *sink)
{
    double a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = 1e-3 * (threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == 12345.678) sink[0] = s;  // keeps the chains live; never true for these inputs
}

extern "C" cswdg_status cswdg_probe_fp64_fma(void *stream, double *gflops_out)
{
    if (!gflops_out) return CSWDG_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CSWDG_ECUDA;
    double *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&sink, sizeof(double)) != cudaSuccess) return CSWDG_ENOMEM;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = nsm * 8, threads = 256, iters = 4096;
    // 1 - 1e-9 and 1e-9 keep every chain finite and away from zero
    k_probe_dfma<<<blocks, threads, 0, st>>>(iters, 1.0 - 1e-9, 1e-9, sink);  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < 5; ++r) k_probe_dfma<<<blocks, threads, 0, st>>>(iters, 1.0 - 1e-9, 1e-9, sink);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess || !(ms > 0.f)) return CSWDG_ECUDA;
    const double flops = 5.0 * blocks * (double)threads * iters * 8 * 2;
    *gflops_out = flops / (ms * 1e-3) / 1e9;
    return CSWDG_OK;
}
