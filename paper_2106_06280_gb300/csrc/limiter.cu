// limiter.cu -- KXRCF troubled-cell detection (Sec. 3.1, Eq.
// troubledCellIndicator) and the compact subcell WENO reconstruction of the
// flagged cells (Sec. 3.2), plus the set-up kernel that builds each cell's
// stencil operators once per mesh.
//
// Per flagged cell the reconstruction needs only immediate neighbours: their
// modes are turned into subcell means by fixed weights, the means into the
// least-squares stencil polynomials by fixed pseudo-inverses, the
// polynomials into smoothness indicators by a fixed quadratic form, and the
// weighted combination into modes by a fixed projection.  All of these depend
// on geometry only, so the set-up kernel computes them in FP64 (Householder
// QR, Cholesky) and stores one operator block per cell (Ops<K>); the
// per-stage kernel applies them.  The smoothness-indicator sums and nonlinear
// weights are evaluated in FP64 in the FP64 and FP32-bulk modes (in float, in
// quotient forms, in the FP32 mode); the KXRCF and positivity tests are
// screened in the state precision and close calls recomputed in FP64.
#include "kernels.h"
#include "physics.cuh"
#include "rules.cuh"
#include "tables.cuh"

namespace csw {

__constant__ Tab<float, 1> lT_f1;
__constant__ Tab<float, 2> lT_f2;
__constant__ Tab<double, 1> lT_d1;
__constant__ Tab<double, 2> lT_d2;

template <typename R, int K> __device__ __forceinline__ const Tab<R, K> &ltab();
template <> __device__ __forceinline__ const Tab<float, 1> &ltab<float, 1>() { return lT_f1; }
template <> __device__ __forceinline__ const Tab<float, 2> &ltab<float, 2>() { return lT_f2; }
template <> __device__ __forceinline__ const Tab<double, 1> &ltab<double, 1>() { return lT_d1; }
template <> __device__ __forceinline__ const Tab<double, 2> &ltab<double, 2>() { return lT_d2; }

cudaError_t limiter_upload_tables()
{
    static Tab<float, 1> f1;
    static Tab<float, 2> f2;
    static Tab<double, 1> d1;
    static Tab<double, 2> d2;
    make_tab(f1); make_tab(f2); make_tab(d1); make_tab(d2);
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(lT_f1, &f1, sizeof(f1))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(lT_f2, &f2, sizeof(f2))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(lT_d1, &d1, sizeof(d1))) != cudaSuccess) return e;
    return cudaMemcpyToSymbol(lT_d2, &d2, sizeof(d2));
}

// ===========================================================================
// Set-up: per-cell operators (FP64, one thread per cell)
// ===========================================================================

struct P2d { double x, y; };

__host__ __device__ inline P2d tri_pt(const P2d *T, const double *b)
{
    return P2d{b[0] * T[0].x + b[1] * T[1].x + b[2] * T[2].x, b[0] * T[0].y + b[1] * T[1].y + b[2] * T[2].y};
}

// physical point -> reference (r, s) of triangle V (vertex order as stored)
__host__ __device__ inline void to_ref(const P2d *V, P2d p, double &r, double &s)
{
    const double a11 = V[1].x - V[0].x, a12 = V[2].x - V[0].x, a21 = V[1].y - V[0].y, a22 = V[2].y - V[0].y;
    const double det = a11 * a22 - a12 * a21, dx = p.x - V[0].x, dy = p.y - V[0].y;
    r = 2.0 * (a22 * dx - a12 * dy) / det - 1.0;
    s = 2.0 * (-a21 * dx + a11 * dy) / det - 1.0;
}

__host__ __device__ inline P2d mirror(P2d a, P2d b, P2d p)
{
    const double ex = b.x - a.x, ey = b.y - a.y;
    const double t = ((p.x - a.x) * ex + (p.y - a.y) * ey) / (ex * ex + ey * ey);
    return P2d{2.0 * (a.x + t * ex) - p.x, 2.0 * (a.y + t * ey) - p.y};
}

// foot of the perpendicular from c on edge a->b; midpoint unless strictly inside [0.05, 0.95]
__host__ __device__ inline P2d perp_foot(P2d c, P2d a, P2d b)
{
    const double ex = b.x - a.x, ey = b.y - a.y;
    double t = ((c.x - a.x) * ex + (c.y - a.y) * ey) / (ex * ex + ey * ey);
    if (!(t >= 0.05 && t <= 0.95)) t = 0.5;
    return P2d{a.x + t * ex, a.y + t * ey};
}

// degree-graded monomials xi^a eta^b without the constant: index j -> (a, b)
__host__ __device__ inline void mono_ab(int j, int &a, int &b)
{
    int idx = 0;
    a = b = 0;
    for (int d = 1; d <= 4; ++d)
        for (int e = 0; e <= d; ++e) {
            if (idx == j) { a = d - e; b = e; }
            ++idx;
        }
}

__host__ __device__ inline double powi(double x, int n)
{
    double r = 1.0;
    for (int i = 0; i < n; ++i) r *= x;
    return r;
}

// d^{p+q}/dxi^p deta^q of xi^a eta^b at (xi, eta)
__host__ __device__ inline double dmono(int a, int b, int p, int q, double xi, double eta)
{
    if (p > a || q > b) return 0.0;
    double c = 1.0;
    for (int i = 0; i < p; ++i) c *= (a - i);
    for (int i = 0; i < q; ++i) c *= (b - i);
    return c * powi(xi, a - p) * powi(eta, b - q);
}

// Moore-Penrose pseudo-inverse of a full-column-rank m x n matrix (row-major)
// through Householder QR: P = R^{-1} Q^T, written P[j*m + i].  Returns 0 or -1.
// Kept out of line: inlined into the set-up kernel, the optimised sm_103a build
// (nvcc 13.0, -O3) returns wrong pseudo-inverses for both degrees (the limited
// modes then differ from the oracle's by 3-12 % relative), while the out-of-line
// call and the -G build agree with the oracle to 1e-11.  Every array here and in
// setup_cell covers its largest use (m <= 15 rows, n <= 9 columns, 16-entry
// scratch, 16-point rules) and every entry is written before it is read; the
// cause of the difference is not known.
__host__ __device__ __noinline__ int pinv_qr(int m, int n, double *A, double *P)
{
    double diag[16], beta[16];
    double rmax = 0.0;
    for (int j = 0; j < n; ++j) {
        double nrm = 0.0;
        for (int i = j; i < m; ++i) nrm += A[i * n + j] * A[i * n + j];
        nrm = sqrt(nrm);
        if (nrm == 0.0) return -1;
        const double alpha = (A[j * n + j] > 0.0) ? -nrm : nrm;
        A[j * n + j] -= alpha;  // v stored in column j below/at the diagonal
        double vv = 0.0;
        for (int i = j; i < m; ++i) vv += A[i * n + j] * A[i * n + j];
        beta[j] = (vv > 0.0) ? 2.0 / vv : 0.0;
        for (int col = j + 1; col < n; ++col) {
            double s = 0.0;
            for (int i = j; i < m; ++i) s += A[i * n + j] * A[i * n + col];
            s *= beta[j];
            for (int i = j; i < m; ++i) A[i * n + col] -= s * A[i * n + j];
        }
        diag[j] = alpha;
        if (fabs(alpha) > rmax) rmax = fabs(alpha);
    }
    for (int j = 0; j < n; ++j)
        if (fabs(diag[j]) < 1e-13 * rmax) return -1;
    for (int e = 0; e < m; ++e) {
        double y[16];
        for (int i = 0; i < m; ++i) y[i] = (i == e) ? 1.0 : 0.0;
        for (int j = 0; j < n; ++j) {  // y <- Q^T y
            double s = 0.0;
            for (int i = j; i < m; ++i) s += A[i * n + j] * y[i];
            s *= beta[j];
            for (int i = j; i < m; ++i) y[i] -= s * A[i * n + j];
        }
        for (int j = n - 1; j >= 0; --j) {  // R x = y
            double s = y[j];
            for (int col = j + 1; col < n; ++col) s -= A[j * n + col] * P[col * m + e];
            P[j * m + e] = s / diag[j];
        }
    }
    return 0;
}

// operator block of cell c; returns non-zero on a rank-deficient fit
template <int K>
__host__ __device__ int setup_cell(int c, int ld, const double *vtx, const double *nvtx, const int32_t *nbr, const uint8_t *nbf,
                                   double *op)
{
    using O = Ops<K>;
    constexpr int NP = Deg<K>::NP, NM = Deg<K>::NM, NSUBK = O::NSUBK;
    TriRule r2, r4, rs;
    rule_deg2(r2);
    rule_deg4(r4);
    recon_rule<K>(rs);

    P2d P[3];
    for (int i = 0; i < 3; ++i) P[i] = P2d{vtx[(size_t)c * 6 + 2 * i], vtx[(size_t)c * 6 + 2 * i + 1]};
    const double area = 0.5 * ((P[1].x - P[0].x) * (P[2].y - P[0].y) - (P[2].x - P[0].x) * (P[1].y - P[0].y));
    const double h0 = sqrt(area);
    const P2d x0{(P[0].x + P[1].x + P[2].x) / 3.0, (P[0].y + P[1].y + P[2].y) / 3.0};
    const double hbar = (hypot(P[1].x - P[0].x, P[1].y - P[0].y) + hypot(P[2].x - P[1].x, P[2].y - P[1].y) +
                         hypot(P[0].x - P[2].x, P[0].y - P[2].y)) / 3.0;

    // monomial means over Delta_0 (degree-4 rule, exact up to degree 4)
    double m0[NM];
    for (int j = 0; j < NM; ++j) {
        int a, b;
        mono_ab(j, a, b);
        double s = 0.0;
        for (int q = 0; q < r4.n; ++q) {
            const P2d p = tri_pt(P, r4.b[q]);
            s += r4.w[q] * powi((p.x - x0.x) / h0, a) * powi((p.y - x0.y) / h0, b);
        }
        m0[j] = s;
    }

    // least-squares rows: stencil cells in the order [i1 of slots 0..2, then per slot its other cells]
    double rowT[3][NSUBK][NM];  // mean_S(m_j) - m0_j for every subcell S
    for (int f = 0; f < 3; ++f) {
        const int code = nbr[f * ld + c];
        P2d X[3], NVt[3];
        int nfl = 0;
        if (code >= 0) {
            for (int i = 0; i < 3; ++i) NVt[i] = P2d{nvtx[((size_t)c * 3 + f) * 6 + 2 * i], nvtx[((size_t)c * 3 + f) * 6 + 2 * i + 1]};
            nfl = (nbf[c] >> (2 * f)) & 3;
            for (int i = 0; i < 3; ++i) X[i] = NVt[(nfl + i) % 3];
        } else {
            X[0] = P[(f + 1) % 3];
            X[1] = P[f];
            X[2] = mirror(P[f], P[(f + 1) % 3], P[(f + 2) % 3]);
        }
        const P2d cx{(X[0].x + X[1].x + X[2].x) / 3.0, (X[0].y + X[1].y + X[2].y) / 3.0};
        P2d S[7][3];
        S[0][0] = cx; S[0][1] = X[0]; S[0][2] = X[1];
        S[1][0] = cx; S[1][1] = X[1]; S[1][2] = X[2];
        S[2][0] = cx; S[2][1] = X[2]; S[2][2] = X[0];
        if (K == 2) {
            const P2d f2 = perp_foot(cx, X[1], X[2]), f3 = perp_foot(cx, X[2], X[0]);
            S[3][0] = cx; S[3][1] = X[1]; S[3][2] = f2;
            S[4][0] = cx; S[4][1] = f2;   S[4][2] = X[2];
            S[5][0] = cx; S[5][1] = f3;   S[5][2] = X[0];
            S[6][0] = cx; S[6][1] = X[2]; S[6][2] = f3;
        }
        for (int i = 0; i < NSUBK; ++i) {
            // subcell-mean weights: mean over S of psi_m of the neighbour (or, for a
            // ghost, of this cell at the mirrored point)
            for (int m = 0; m < NP; ++m) {
                double s = 0.0;
                for (int q = 0; q < r2.n; ++q) {
                    P2d p = tri_pt(S[i], r2.b[q]);
                    double rr, ss, v, dr, ds;
                    if (code >= 0) to_ref(NVt, p, rr, ss);
                    else {
                        p = mirror(P[f], P[(f + 1) % 3], p);
                        to_ref(P, p, rr, ss);
                    }
                    dubiner(K, m, rr, ss, v, dr, ds);
                    s += r2.w[q] * v;
                }
                op[O::W + (f * NSUBK + i) * NP + m] = s;
            }
            for (int j = 0; j < NM; ++j) {
                int a, b;
                mono_ab(j, a, b);
                double s = 0.0;
                for (int q = 0; q < r4.n; ++q) {
                    const P2d p = tri_pt(S[i], r4.b[q]);
                    s += r4.w[q] * powi((p.x - x0.x) / h0, a) * powi((p.y - x0.y) / h0, b);
                }
                rowT[f][i][j] = s - m0[j];
            }
        }
        // beta_1 map: centroids of the thirds in the (xi, eta) frame
        double cxs[3], cys[3];
        for (int i = 0; i < 3; ++i) {
            cxs[i] = ((S[i][0].x + S[i][1].x + S[i][2].x) / 3.0 - x0.x) / h0;
            cys[i] = ((S[i][0].y + S[i][1].y + S[i][2].y) / 3.0 - x0.y) / h0;
        }
        const double a11 = cxs[1] - cxs[0], a12 = cys[1] - cys[0], a21 = cxs[2] - cxs[0], a22 = cys[2] - cys[0];
        const double det = a11 * a22 - a12 * a21;
        op[O::MI + 4 * f + 0] = a22 / det;
        op[O::MI + 4 * f + 1] = -a12 / det;
        op[O::MI + 4 * f + 2] = -a21 / det;
        op[O::MI + 4 * f + 3] = a11 / det;
    }

    // pseudo-inverses
    double A[15 * 9], Pm[9 * 15];
    int bad = 0;
    for (int s = 0; s < 3; ++s)
        for (int j = 0; j < 2; ++j) A[s * 2 + j] = rowT[s][0][j];
    if (pinv_qr(3, 2, A, Pm)) bad = 1;
    for (int i = 0; i < 6; ++i) op[O::A2 + i] = Pm[i];
    {
        int r = 0;
        for (int s = 0; s < 3; ++s, ++r)
            for (int j = 0; j < 5; ++j) A[r * 5 + j] = rowT[s][0][j];
        for (int s = 0; s < 3; ++s)
            for (int i = 1; i < 3; ++i, ++r)
                for (int j = 0; j < 5; ++j) A[r * 5 + j] = rowT[s][i][j];
        if (pinv_qr(9, 5, A, Pm)) bad = 1;
        for (int i = 0; i < 45; ++i) op[O::A3 + i] = Pm[i];
    }
    if (K == 2) {
        int r = 0;
        for (int s = 0; s < 3; ++s, ++r)
            for (int j = 0; j < 9; ++j) A[r * 9 + j] = rowT[s][0][j];
        for (int s = 0; s < 3; ++s)
            for (int i = 3; i < NSUBK; ++i, ++r)
                for (int j = 0; j < 9; ++j) A[r * 9 + j] = rowT[s][i][j];
        if (pinv_qr(15, 9, A, Pm)) bad = 1;
        for (int i = 0; i < 135; ++i) op[O::A4 + i] = Pm[i];
    }

    // smoothness-indicator form H_jk = sum_{1<=|alpha|<=deg} int_{Delta_0 in xi} D^a m_j D^a m_k,
    // Delta_0 has unit area in the xi frame; integrand degree <= 4
    constexpr int DEG = (K == 1) ? 2 : 3;
    double H[NM][NM];
    for (int j = 0; j < NM; ++j)
        for (int k = 0; k < NM; ++k) H[j][k] = 0.0;
    for (int q = 0; q < r4.n; ++q) {
        const P2d p = tri_pt(P, r4.b[q]);
        const double xi = (p.x - x0.x) / h0, eta = (p.y - x0.y) / h0;
        for (int s = 1; s <= DEG; ++s)
            for (int qq = 0; qq <= s; ++qq) {
                const int pp = s - qq;
                double d[NM];
                for (int j = 0; j < NM; ++j) {
                    int a, b;
                    mono_ab(j, a, b);
                    d[j] = dmono(a, b, pp, qq, xi, eta);
                }
                for (int j = 0; j < NM; ++j)
                    for (int k = 0; k < NM; ++k) H[j][k] += r4.w[q] * d[j] * d[k];
            }
    }
    // Cholesky H = L L^T, packed rows of L
    double L[NM][NM];
    for (int i = 0; i < NM; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = H[i][j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > 0.0)) { bad = 1; s = 1e-300; }
                L[i][i] = sqrt(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    for (int i = 0, p = 0; i < NM; ++i)
        for (int j = 0; j <= i; ++j, ++p) op[O::LH + p] = L[i][j];

    // projection of sum_j c_j (m_j - m0_j) onto modes 1..NP-1 through the
    // reconstruction points: Phi_ij = 2 sum_q w_q (m_j(xi_q) - m0_j) psi_i(r_q)
    for (int i = 1; i < NP; ++i)
        for (int j = 0; j < NM; ++j) {
            int a, b;
            mono_ab(j, a, b);
            double s = 0.0;
            for (int q = 0; q < rs.n; ++q) {
                const P2d p = tri_pt(P, rs.b[q]);
                double rr, ss, v, dr, ds;
                bary_to_rs(rs.b[q], rr, ss);
                dubiner(K, i, rr, ss, v, dr, ds);
                s += rs.w[q] * (powi((p.x - x0.x) / h0, a) * powi((p.y - x0.y) / h0, b) - m0[j]) * v;
            }
            op[O::PHI + (i - 1) * NM + j] = 2.0 * s;
        }
    {
        // Step 2: gamma_bar_{l,m} = (1/h)^{l-1} normalised over the defined terms
        const double ih = 1.0 / hbar;
        const double s2 = 1.0 + ih, s3 = 1.0 + ih + ih * ih, s5 = 1.0 + ih + ih * ih + ih * ih * ih;
        double *g = op + O::GAM;
        g[0] = 1.0 / s3; g[1] = ih / s3; g[2] = ih * ih / s3;
        g[3] = 1.0 / s5; g[4] = ih / s5; g[5] = ih * ih / s5; g[6] = ih * ih * ih / s5;
        g[7] = s2 / ih;          // 1 / gamma_{2,2}
        g[8] = s3 / (ih * ih);   // 1 / gamma_{3,3}
        g[9] = s5 / (ih * ih * ih);  // 1 / gamma_{4,5}
        g[10] = ih / s3;         // gamma_{2,3}
        g[11] = hbar;
    }
    return bad;
}

template <int K>
__global__ void k_setup_ops(int nc, int ld, const double *__restrict__ vtx, const double *__restrict__ nvtx,
                            const int32_t *__restrict__ nbr, const uint8_t *__restrict__ nbf, double *__restrict__ ops,
                            int32_t *err)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    if (setup_cell<K>(c, ld, vtx, nvtx, nbr, nbf, ops + (size_t)c * Ops<K>::SIZE)) atomicOr(err, ERR_LSQ);
}

void launch_setup_ops(int k, int nc, int ld, const double *vtx, const double *nvtx, const int32_t *nbr, const uint8_t *nbf,
                      double *ops, int32_t *err, cudaStream_t st)
{
    const int blk = 64, grd = (nc + blk - 1) / blk;
    if (k == 1) k_setup_ops<1><<<grd, blk, 0, st>>>(nc, ld, vtx, nvtx, nbr, nbf, ops, err);
    else k_setup_ops<2><<<grd, blk, 0, st>>>(nc, ld, vtx, nvtx, nbr, nbf, ops, err);
}

__global__ void k_to_float(size_t n, const double *__restrict__ s, float *__restrict__ d)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) d[i] = (float)s[i];
}
void launch_ops_to_float(size_t n, const double *src, float *dst, cudaStream_t st) { k_to_float<<<1024, 256, 0, st>>>(n, src, dst); }

// ===========================================================================
// KXRCF detection + compaction of the flagged cells
// ===========================================================================

// ghost value of the indicator variable (variable 0) across a boundary face
template <int EQ, typename R>
__device__ __forceinline__ R ghost0(const BFace &bf, const BcTab *bc, double tp, double t, R Uin0)
{
    const int kind = bc->kind[bf.tag];
    const double *P = bc->par[bf.tag];
    if (kind == BC_DIRICHLET) return (R)P[0];
    if (kind == BC_SHOCKLINE) {
        constexpr int NV = Eqn<EQ>::NV;
        const double x = bf.ax + tp * (bf.bx - bf.ax), y = bf.ay + tp * (bf.by - bf.ay);
        return (R)((x < P[0] + y * P[1] + P[2] * t) ? P[3] : P[3 + NV]);
    }
    return Uin0;  // transmissive, and the wall keeps the density
}

// KXRCF indicator of cell c (Sec. 2.3): 1 when the jump of the indicator
// variable over the inflow faces, scaled by h^((k+1)/2) |K|^(1/2) and the L2
// norm of the cell's polynomial, exceeds C_K.  The modes of the three
// neighbours are fetched before the inflow test so that all gathers of a
// thread are in flight together.
template <int EQ, int K, typename R>
__device__ __forceinline__ int detect_cell(const MeshDev<R> &M, const R *__restrict__ u, Ctl *ctl, double tfac, double ck, R ck2,
                                           int all, int c, const NbrTraceTab<R, K> &ntab)
{
    constexpr int NP = Deg<K>::NP, QF = Deg<K>::QF, NVd = Eqn<EQ>::NV;
    const int ld = M.ldc;
    const Tab<R, K> &T = ltab<R, K>();
    int code[3];
    R w[3][NP];
    R a[NP];
    load_var0<NVd, NP>(u, c, a);
    if (!all) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            code[f] = M.nbr[f * ld + c];
            if (code[f] >= 0) load_var0<NVd, NP>(u, code[f], w[f]);
        }
    }
    // cell-mean velocity direction: v = (m_x, m_y) / rho with rho > 0 (Euler),
    // v = (u, u) (Burgers); only its sign against each normal is used
    R vx, vy;
    if (EQ == EULER) {
        const R r = a[0], mx = u[sidx(NVd, NP, 1, 0, c)], my = u[sidx(NVd, NP, 2, 0, c)], E = u[sidx(NVd, NP, 3, 0, c)];
        // positivity of the mean without division: rho > 0 and 2 E rho - |m|^2 > 0, decided in
        // FP64 (FP32 values are first screened with a relative margin; only close calls are
        // recomputed in FP64)
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
        vx = vy = a[0];
        if (!(vx == vx)) atomicOr(&ctl->err, ERR_NONPHYS);
    }
    if (all) return 1;
    // reading R-pos: non-physical at a volume or face quadrature point -> troubled
    if constexpr (EQ == EULER) {
        R uf[4][NP];
        load_cell<4, NP>(u, c, uf);
        if (nonphys_points<K, R>(uf, T, M.gamma)) return 1;
    }
    R num = R(0), lsum = R(0);
    const unsigned nbfc = M.nbf[c];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const R nx = M.geo[(G_N0X + 3 * f) * ld + c], ny = M.geo[(G_N0Y + 3 * f) * ld + c];
        // inflow test v.n < 0, evaluated without contraction (exact zero for v = (u, u) on n = (a, -a))
        const R vn = (EQ == BURGERS) ? vx * radd_rn(nx, ny) : radd_rn(rmul_rn(vx, nx), rmul_rn(vy, ny));
        if (!(vn < R(0))) continue;
        const R nl = M.geo[(G_N0L + 3 * f) * ld + c];
        const int nf = (nbfc >> (2 * f)) & 3;
        BFace bf;
        if (code[f] < 0) bf = M.bf[-code[f] - 1];
        R J = R(0);
#pragma unroll
        for (int g = 0; g < QF; ++g) {
            R ui = R(0), uo = R(0);
#pragma unroll
            for (int m = 0; m < NP; ++m) ui += a[m] * T.fphi[f][g][m];
            if (code[f] >= 0) {
                R ph[NP];
                ntab.row(nf, g, ph);
#pragma unroll
                for (int m = 0; m < NP; ++m) uo += w[f][m] * ph[m];
            } else {
                uo = ghost0<EQ, R>(bf, M.bc, (double)T.ft[g], stage_time(ctl, tfac), ui);
            }
            J += T.fw[g] * (ui - uo);
        }
        num += nl * J;
        lsum += nl;
    }
    R nrm2 = R(0);
#pragma unroll
    for (int m = 0; m < NP; ++m) nrm2 += a[m] * a[m];
    const R kap = M.geo[G_KAPPA * ld + c];
    // R_j = |num| / (lsum kap sqrt(nrm2)) > C_K, compared without division or root (all
    // factors non-negative; no inflow face or a zero jump never flags).  The comparison is
    // screened in the state precision with a relative margin; close calls are decided in FP64.
    int flag = 0;
    if (lsum > R(0)) {
        const R denr = lsum * kap;
        const R lhs = num * num, rhs = ck2 * denr * denr * nrm2;
        if (rabs(lhs - rhs) > R(1e-3) * (lhs + rhs)) {
            flag = lhs > rhs;
        } else {
            const double den = (double)lsum * (double)kap;
            flag = (double)num * (double)num > ck * ck * den * den * (double)nrm2;
        }
    }
    return flag;
}

// |L^T c|^2 for the leading N x N block of a packed lower-triangular L; the
// components in R, the sum of squares accumulated in W
template <int N, typename R, typename W>
__host__ __device__ __forceinline__ W quad_form(const R *__restrict__ L, const R *c)
{
    W acc = W(0);
#pragma unroll
    for (int j = 0; j < N; ++j) {
        R y = R(0);
#pragma unroll
        for (int i = j; i < N; ++i) y += L[i * (i + 1) / 2 + j] * c[i];
        acc += (W)y * (W)y;
    }
    return acc;
}

// ===========================================================================
// CSWENO reconstruction of one scalar field (Sec. 3.2 Steps 1-5 / Steps 1-4)
// t[f][i]: subcell means of slot f (thirds 0..2, halves 3..6), w0: cell mean.
// Reciprocal of a positive weight sum in W precision.  In double: the hardware
// seed rcp.approx.ftz.f64 (PTX ISA) refined by two Newton-Raphson steps for
// 1/x, r <- r + r (1 - x r), each of which about doubles the number of correct
// bits, so the result is within an ulp or two of 1/x (the IEEE division is a
// long FP64 sequence on this GPU).  The weights it normalises need no more.
__host__ __device__ __forceinline__ double wrcp(double x)
{
#ifdef __CUDA_ARCH__
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    r = fma(r, fma(-x, r, 1.0), r);
    return fma(r, fma(-x, r, 1.0), r);
#else
    return 1.0 / x;
#endif
}
__host__ __device__ __forceinline__ float wrcp(float x) { return rrcp(x); }

// ===========================================================================
// W: precision of the smoothness indicators, tau and the nonlinear weights
// (double: FP64 and FP32-bulk modes; float: FP32 mode)
template <int K, typename R, typename W = R>
__host__ __device__ __forceinline__ void weno_field(const R *__restrict__ op, const R (&t)[3][Ops<K>::NSUBK], R w0, R (&md)[Deg<K>::NP - 1])
{
    using O = Ops<K>;
    constexpr int NP = Deg<K>::NP, NM = Deg<K>::NM;
    const double eps = 1e-10;
    // Step 1: least-squares stencil polynomials (mean on Delta_0 built in)
    R q2[2], q3[5], q4[9];
    {
        R b[3];
        for (int s = 0; s < 3; ++s) b[s] = t[s][0] - w0;
        for (int j = 0; j < 2; ++j) {
            R acc = R(0);
            for (int s = 0; s < 3; ++s) acc += op[O::A2 + j * 3 + s] * b[s];
            q2[j] = acc;
        }
    }
    {
        R b[9];
        b[0] = t[0][0] - w0; b[1] = t[1][0] - w0; b[2] = t[2][0] - w0;
        for (int s = 0; s < 3; ++s) { b[3 + 2 * s] = t[s][1] - w0; b[4 + 2 * s] = t[s][2] - w0; }
        for (int j = 0; j < 5; ++j) {
            R acc = R(0);
            for (int s = 0; s < 9; ++s) acc += op[O::A3 + j * 9 + s] * b[s];
            q3[j] = acc;
        }
    }
    if (K == 2) {
        R b[15];
        b[0] = t[0][0] - w0; b[1] = t[1][0] - w0; b[2] = t[2][0] - w0;
        for (int s = 0; s < 3; ++s)
            for (int i = 0; i < 4; ++i) b[3 + 4 * s + i] = t[s][(3 + i) % Ops<K>::NSUBK] - w0;
        for (int j = 0; j < 9; ++j) {
            R acc = R(0);
            for (int s = 0; s < 15; ++s) acc += op[O::A4 + j * 15 + s] * b[s];
            q4[j] = acc;
        }
    }
    // Step 2: hierarchical polynomials with the linear weights precomputed per cell
    const R *gm = op + O::GAM;
    R p2[NM], p3[NM], p4[NM];
    for (int j = 0; j < NM; ++j) { p2[j] = R(0); p3[j] = R(0); p4[j] = R(0); }
    for (int j = 0; j < 2; ++j) p2[j] = q2[j] * gm[7];
    for (int j = 0; j < 5; ++j) p3[j] = (q3[j] - gm[10] * p2[j]) * gm[8];
    if (K == 2)
        for (int j = 0; j < 9; ++j) p4[j] = (q4[j] - gm[4] * p2[j] - gm[5] * p3[j]) * gm[9];
    // Step 3: smoothness indicators beta_l = |L^T c(p_l)|^2, summed in W
    W beta[4];
    beta[1] = quad_form<2, R, W>(op + O::LH, p2);
    beta[2] = quad_form<5, R, W>(op + O::LH, p3);
    if (K == 2) beta[3] = quad_form<9, R, W>(op + O::LH, p4);
    W om[4];
    if constexpr (sizeof(W) == 8) {
        // FP64: beta_1 magnified from the three linear fits through the thirds'
        // centroids (Eqs. sigmaEqn, smoothnessIndicatorT1), the sigma-weighted
        // average formed over a common denominator (one division)
        {
            // the gradients of p_{1,l} are stencil polynomials like p_l (state
            // precision); beta_{1,l} and everything after it in W
            W al[3], bl[3], b1[3], e[3];
            for (int f = 0; f < 3; ++f) {
                const R r1 = t[f][1] - t[f][0], r2 = t[f][2] - t[f][0];
                al[f] = (W)(op[O::MI + 4 * f + 0] * r1 + op[O::MI + 4 * f + 1] * r2);
                bl[f] = (W)(op[O::MI + 4 * f + 2] * r1 + op[O::MI + 4 * f + 3] * r2);
                b1[f] = al[f] * al[f] + bl[f] * bl[f];  // beta_{1,l}
                e[f] = b1[f] + W(eps);
            }
            // D: mean absolute difference of the beta_{1,l} (reading R-sigma)
            const W D = (fabs(b1[0] - b1[1]) + fabs(b1[1] - b1[2]) + fabs(b1[2] - b1[0])) * W(1.0 / 3.0);  // a product: a double division is slow on this FP64 pipe
            const W D2 = D * D;
            // sigma_l is proportional to (e_l + D^2) / e_l; multiply through by e_0 e_1 e_2
            const W w0 = (e[0] + D2) * e[1] * e[2], w1 = (e[1] + D2) * e[0] * e[2], w2 = (e[2] + D2) * e[0] * e[1];
            const W inv = wrcp(w0 + w1 + w2);
            const W ab = (w0 * al[0] + w1 * al[1] + w2 * al[2]) * inv, bb = (w0 * bl[0] + w1 * bl[1] + w2 * bl[2]) * inv;
            beta[0] = ab * ab + bb * bb;
        }
        // Step 4 (reading R-weno): tau the mean absolute difference to the top slot's beta,
        // omega_l proportional to gamma_l (1 + (tau / a_l)^(K+1)), a_l = eps + beta_l, formed
        // over the common denominator prod_m a_m^(K+1) (one reciprocal; in double every
        // factor stays in range: a^12 >= 1e-120)
        if (K == 1) {
            const W tau = (fabs(beta[2] - beta[0]) + fabs(beta[2] - beta[1])) * W(0.5);
            const W a0 = eps + beta[0], a1 = eps + beta[1], a2 = eps + beta[2];
            const W s0 = a0 * a0, s1 = a1 * a1, s2 = a2 * a2, t2 = tau * tau;
            const W w0 = (W)gm[0] * (s0 + t2) * s1 * s2, w1 = (W)gm[1] * (s1 + t2) * s0 * s2, w2 = (W)gm[2] * (s2 + t2) * s0 * s1;
            const W inv = wrcp(w0 + w1 + w2);
            om[0] = w0 * inv; om[1] = w1 * inv; om[2] = w2 * inv; om[3] = W(0);
        } else {
            const W tau = (fabs(beta[3] - beta[0]) + fabs(beta[3] - beta[1]) + fabs(beta[3] - beta[2])) * W(1.0 / 3.0);
            const W t3 = tau * tau * tau;
            W c[4];
            for (int l = 0; l < 4; ++l) { const W al_ = eps + beta[l]; c[l] = al_ * al_ * al_; }
            const W p01 = c[0] * c[1], p23 = c[2] * c[3];
            const W w[4] = {(W)gm[3] * (c[0] + t3) * c[1] * p23, (W)gm[4] * (c[1] + t3) * c[0] * p23,
                            (W)gm[5] * (c[2] + t3) * p01 * c[3], (W)gm[6] * (c[3] + t3) * p01 * c[2]};
            const W inv = wrcp(w[0] + w[1] + w[2] + w[3]);
            for (int l = 0; l < 4; ++l) om[l] = w[l] * inv;
        }
    } else {
        // FP32: the same weights in quotient form.  Products of three or four
        // (eps + beta) factors would leave the FP32 range (eps^4 = 1e-40), so each
        // weight is 1 + X / e_l with X = D^2 or tau; when X >= 1 every weight is
        // divided by X first (1/X + 1/e_l), which keeps all terms below about 1e10.
        {
            R al[3], bl[3], b1[3], ie[3];
            for (int f = 0; f < 3; ++f) {
                const R r1 = t[f][1] - t[f][0], r2 = t[f][2] - t[f][0];
                al[f] = op[O::MI + 4 * f + 0] * r1 + op[O::MI + 4 * f + 1] * r2;
                bl[f] = op[O::MI + 4 * f + 2] * r1 + op[O::MI + 4 * f + 3] * r2;
                b1[f] = al[f] * al[f] + bl[f] * bl[f];
                ie[f] = rrcp(b1[f] + R(eps));
            }
            const R D = (rabs(b1[0] - b1[1]) + rabs(b1[1] - b1[2]) + rabs(b1[2] - b1[0])) * R(1.0 / 3.0);
            R s[3];
            if (D >= R(1)) {
                const R iD = rrcp(D), iD2 = iD * iD;
                for (int f = 0; f < 3; ++f) s[f] = iD2 + ie[f];
            } else {
                const R D2 = D * D;
                for (int f = 0; f < 3; ++f) s[f] = R(1) + D2 * ie[f];
            }
            const R inv = rrcp(s[0] + s[1] + s[2]);
            const R ab = (s[0] * al[0] + s[1] * al[1] + s[2] * al[2]) * inv, bb = (s[0] * bl[0] + s[1] * bl[1] + s[2] * bl[2]) * inv;
            beta[0] = ab * ab + bb * bb;
        }
        constexpr int NL = (K == 1) ? 3 : 4;
        R tau = R(0);
        for (int l = 0; l < NL - 1; ++l) tau += rabs(beta[NL - 1] - beta[l]);
        tau *= (K == 1) ? R(0.5) : R(1.0 / 3.0);
        const R *gl = gm + ((K == 1) ? 0 : 3);
        // (tau / a)^(K+1) with a >= eps: when tau >= 1 every weight is divided by
        // tau^(K+1) first, so no term exceeds eps^-(K+1) = 1e30 (float range 3e38)
        R w[NL], wsum = R(0);
        if (tau >= R(1)) {
            const R it = rrcp(tau);
            R itp = it;
            for (int e = 0; e < K; ++e) itp *= it;
            for (int l = 0; l < NL; ++l) {
                const R ia = rrcp(beta[l] + R(eps));
                R iap = ia;
                for (int e = 0; e < K; ++e) iap *= ia;
                w[l] = gl[l] * (itp + iap);
            }
        } else {
            for (int l = 0; l < NL; ++l) {
                const R r = tau * rrcp(beta[l] + R(eps));
                R rp = r;
                for (int e = 0; e < K; ++e) rp *= r;
                w[l] = gl[l] * (R(1) + rp);
            }
        }
        for (int l = 0; l < NL; ++l) wsum += w[l];
        const R inv = rrcp(wsum);
        for (int l = 0; l < NL; ++l) om[l] = w[l] * inv;
        if (K == 1) om[3] = R(0);
    }
    // Step 5: combined polynomial (p_1 is the constant cell mean) projected onto modes 1..NP-1
    R cm[NM];
    for (int j = 0; j < NM; ++j) cm[j] = (R)om[1] * p2[j] + (R)om[2] * p3[j] + (R)om[3] * p4[j];
    for (int i = 0; i < NP - 1; ++i) {
        R acc = R(0);
        for (int j = 0; j < NM; ++j) acc += op[O::PHI + i * NM + j] * cm[j];
        md[i] = acc;
    }
}

// left/right eigenvectors of the Euler flux Jacobian along the unit direction (nx, ny)
template <typename R>
__host__ __device__ __forceinline__ void euler_eig(const R *U, R gam, R nx, R ny, R (&Rm)[4][4], R (&Lm)[4][4])
{
    const R rho = U[0], u = U[1] / rho, v = U[2] / rho;
    const R q2 = u * u + v * v;
    const R p = (gam - R(1)) * (U[3] - R(0.5) * rho * q2);
    const R c2 = gam * p / rho, c = rsqroot(c2), H = (U[3] + p) / rho;
    const R un = u * nx + v * ny, ut = -u * ny + v * nx, b = gam - R(1);
    // columns: acoustic (-), entropy, shear, acoustic (+)
    Rm[0][0] = R(1);          Rm[0][1] = R(1);          Rm[0][2] = R(0); Rm[0][3] = R(1);
    Rm[1][0] = u - c * nx;    Rm[1][1] = u;             Rm[1][2] = -ny;  Rm[1][3] = u + c * nx;
    Rm[2][0] = v - c * ny;    Rm[2][1] = v;             Rm[2][2] = nx;   Rm[2][3] = v + c * ny;
    Rm[3][0] = H - c * un;    Rm[3][1] = R(0.5) * q2;   Rm[3][2] = ut;   Rm[3][3] = H + c * un;
    const R i2c2 = R(1) / (R(2) * c2);
    Lm[0][0] = (R(0.5) * b * q2 + c * un) * i2c2; Lm[0][1] = -(b * u + c * nx) * i2c2; Lm[0][2] = -(b * v + c * ny) * i2c2; Lm[0][3] = b * i2c2;
    Lm[1][0] = R(1) - b * q2 * i2c2;              Lm[1][1] = R(2) * b * u * i2c2;     Lm[1][2] = R(2) * b * v * i2c2;     Lm[1][3] = -R(2) * b * i2c2;
    Lm[2][0] = -ut;                               Lm[2][1] = -ny;                     Lm[2][2] = nx;                      Lm[2][3] = R(0);
    Lm[3][0] = (R(0.5) * b * q2 - c * un) * i2c2; Lm[3][1] = -(b * u - c * nx) * i2c2; Lm[3][2] = -(b * v - c * ny) * i2c2; Lm[3][3] = b * i2c2;
}

// one characteristic field fl of euler_eig: the left eigenvector (row fl of
// Lm) and the right eigenvector (column fl of Rm), selected without indexing
// so that the eight-lane limiter keeps them in registers
template <typename R>
__host__ __device__ __forceinline__ void euler_eig_field(const R *U, R gam, R nx, R ny, int fl, R (&l)[4], R (&r)[4])
{
    const R rho = U[0], u = U[1] / rho, v = U[2] / rho;
    const R q2 = u * u + v * v;
    const R p = (gam - R(1)) * (U[3] - R(0.5) * rho * q2);
    const R c2 = gam * p / rho, c = rsqroot(c2), H = (U[3] + p) / rho;
    const R un = u * nx + v * ny, ut = -u * ny + v * nx, b = gam - R(1);
    const R i2c2 = R(1) / (R(2) * c2);
    if (fl == 1) {  // entropy
        r[0] = R(1); r[1] = u; r[2] = v; r[3] = R(0.5) * q2;
        l[0] = R(1) - b * q2 * i2c2; l[1] = R(2) * b * u * i2c2; l[2] = R(2) * b * v * i2c2; l[3] = -R(2) * b * i2c2;
    } else if (fl == 2) {  // shear
        r[0] = R(0); r[1] = -ny; r[2] = nx; r[3] = ut;
        l[0] = -ut; l[1] = -ny; l[2] = nx; l[3] = R(0);
    } else {  // acoustic, sg = -1 (fl = 0) or +1 (fl = 3)
        const R cs = (fl == 0) ? -c : c;
        r[0] = R(1); r[1] = u + cs * nx; r[2] = v + cs * ny; r[3] = H + cs * un;
        l[0] = (R(0.5) * b * q2 - cs * un) * i2c2; l[1] = -(b * u - cs * nx) * i2c2; l[2] = -(b * v - cs * ny) * i2c2;
        l[3] = b * i2c2;
    }
}

// reconstructed modes 1..NP-1 of every variable of flagged cell c (Sec. 3.2),
// from the unlimited state u, at limiter time tl
template <int EQ, int K, typename R, typename W = R>
__host__ __device__ __forceinline__ void limit_cell(const MeshDev<R> &M, const R *u, const R *op, int c, double tl,
                                                    R (&res)[Eqn<EQ>::NV][Deg<K>::NP - 1])
{
    using O = Ops<K>;
    constexpr int NP = Deg<K>::NP, NV = Eqn<EQ>::NV, NSUBK = O::NSUBK;
    const int ld = M.ldc;
    const R gam = (R)M.gamma;
    R u0[NV][NP];
    for (int v = 0; v < NV; ++v)
        for (int m = 0; m < NP; ++m) u0[v][m] = u[sidx(NV, NP, v, m, c)];
    R mean[NV][3][NSUBK];
    for (int f = 0; f < 3; ++f) {
        const int code = M.nbr[f * ld + c];
        R w[NV][NP];
        bool constant = false;
        if (code >= 0) {
            for (int v = 0; v < NV; ++v)
                for (int m = 0; m < NP; ++m) w[v][m] = u[sidx(NV, NP, v, m, code)];
        } else {
            const BFace bf = M.bf[-code - 1];
            const int kind = M.bc->kind[bf.tag];
            if (kind == BC_DIRICHLET || kind == BC_SHOCKLINE) {
                // constant ghost (shock line: decided at the face midpoint)
                R S[NV], dummy[NV];
                for (int v = 0; v < NV; ++v) dummy[v] = R(0);
                ghost<EQ, R>(bf, M.bc, 0.5, tl, dummy, S);
                for (int v = 0; v < NV; ++v)
                    for (int i = 0; i < NSUBK; ++i) mean[v][f][i] = S[v];
                constant = true;
            } else {
                for (int v = 0; v < NV; ++v)
                    for (int m = 0; m < NP; ++m) w[v][m] = u0[v][m];
                if (kind == BC_WALL && EQ == EULER) {
                    const R nx = (R)bf.nx, ny = (R)bf.ny;
                    for (int m = 0; m < NP; ++m) {
                        const R mn = w[1][m] * nx + w[2][m] * ny;
                        w[1][m] -= R(2) * mn * nx;
                        w[2][m] -= R(2) * mn * ny;
                    }
                }
            }
        }
        if (!constant)
            for (int i = 0; i < NSUBK; ++i)
                for (int v = 0; v < NV; ++v) {
                    R s = R(0);
                    for (int m = 0; m < NP; ++m) s += op[O::W + (f * NSUBK + i) * NP + m] * w[v][m];
                    mean[v][f][i] = s;
                }
    }
    R ub[NV];
    for (int v = 0; v < NV; ++v) ub[v] = u0[v][0] * R(0.70710678118654752440);
    if (EQ == BURGERS) {
        R md[NP - 1];
        weno_field<K, R, W>(op, mean[0], ub[0], md);
        for (int i = 0; i < NP - 1; ++i) res[0][i] = md[i];
    } else {
        for (int v = 0; v < NV; ++v)
            for (int i = 0; i < NP - 1; ++i) res[v][i] = R(0);
        for (int d = 0; d < 2; ++d) {
            R Rm[4][4], Lm[4][4];
            euler_eig<R>(ub, gam, d == 0 ? R(1) : R(0), d == 0 ? R(0) : R(1), Rm, Lm);
            for (int fl = 0; fl < 4; ++fl) {
                R tc[3][NSUBK];
                for (int f = 0; f < 3; ++f)
                    for (int i = 0; i < NSUBK; ++i) {
                        R s = R(0);
                        for (int v = 0; v < 4; ++v) s += Lm[fl][v] * mean[v][f][i];
                        tc[f][i] = s;
                    }
                R w0 = R(0);
                for (int v = 0; v < 4; ++v) w0 += Lm[fl][v] * ub[v];
                R md[NP - 1];
                weno_field<K, R, W>(op, tc, w0, md);
                for (int v = 0; v < 4; ++v)
                    for (int i = 0; i < NP - 1; ++i) res[v][i] += R(0.5) * Rm[v][fl] * md[i];
            }
        }
    }
}

// Euler: a reconstruction with non-positive density or pressure at a volume
// point or a face Gauss point of the cell keeps only the cell mean.  The
// QV + 3 QF points are shared by the eight lanes of the cell (point q on lane
// q mod 8).  With rho > 0 and gamma > 1, p > 0 is 2 E rho - |m|^2 > 0; that
// product form is decided in the state precision when it clears a relative
// margin, and close calls are recomputed in FP64 as (gamma - 1)(E - |m|^2 / 2 rho).
template <int K, typename R>
__device__ __forceinline__ bool positivity_bad_lane(const R *mean_modes, const R (&res)[4][Deg<K>::NP - 1], int lane8, double gam)
{
    constexpr int NP = Deg<K>::NP, QV = Deg<K>::QV, QF = Deg<K>::QF;
    const Tab<R, K> &T = ltab<R, K>();
    bool bad = false;
    for (int q = lane8; q < QV + 3 * QF; q += 8) {
        const R *phi = (q < QV) ? T.vphi[q] : T.fphi[(q - QV) / QF][(q - QV) % QF];
        R U[4];
        for (int v = 0; v < 4; ++v) {
            R s = mean_modes[v] * phi[0];
            for (int m = 1; m < NP; ++m) s += res[v][m - 1] * phi[m];
            U[v] = s;
        }
        const R two_e_rho = R(2) * U[3] * U[0], m2 = U[1] * U[1] + U[2] * U[2];
        const R qp = two_e_rho - m2;
        bool ok = (U[0] > R(0)) && (qp > R(1e-3) * (rabs(two_e_rho) + m2));
        if (!ok && U[0] > R(0) && !(qp < -R(1e-3) * (rabs(two_e_rho) + m2))) {
            const double r = (double)U[0], mx = (double)U[1], my = (double)U[2], E = (double)U[3];
            ok = (gam - 1.0) * (E - 0.5 * (mx * mx + my * my) / r) > 0.0;
        }
        bad = bad || !ok;
    }
    return bad;
}

// Euler: eight lanes per flagged cell, one per (direction d in {x, y},
// characteristic field); each lane transforms the neighbours' modes into its
// field, forms the subcell means, reconstructs (weno_field) and maps back by
// the right eigenvectors; the eight contributions are summed with shuffles.
template <int K, typename R, typename W = R>
__device__ __forceinline__ void limit_cell_euler_lane(const MeshDev<R> &M, const R *__restrict__ u, const R *__restrict__ op, int c,
                                                      double tl, int lane8, R (&res)[4][Deg<K>::NP - 1])
{
    using O = Ops<K>;
    constexpr int NP = Deg<K>::NP, NSUBK = O::NSUBK;
    const int ld = M.ldc;
    const int d = lane8 >> 2, fl = lane8 & 3;
    R u0[4][NP];
    load_cell<4, NP>(u, c, u0);
    R ub[4];
    for (int v = 0; v < 4; ++v) ub[v] = u0[v][0] * R(0.70710678118654752440);
    R Ll[4], Rr[4];
    euler_eig_field<R>(ub, M.gammar, d == 0 ? R(1) : R(0), d == 0 ? R(0) : R(1), fl, Ll, Rr);
    R tc[3][NSUBK];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const int code = M.nbr[f * ld + c];
        R wc[NP];  // neighbour modes projected on this lane's characteristic field
        bool constant = false;
        if (code >= 0) {
            R wn[4][NP];
            load_cell<4, NP>(u, code, wn);
            for (int m = 0; m < NP; ++m) {
                R s = R(0);
                for (int v = 0; v < 4; ++v) s += Ll[v] * wn[v][m];
                wc[m] = s;
            }
        } else {
            const BFace bf = M.bf[-code - 1];
            const int kind = M.bc->kind[bf.tag];
            if (kind == BC_DIRICHLET || kind == BC_SHOCKLINE) {
                R S[4], dummy[4] = {R(0), R(0), R(0), R(0)};
                ghost<EULER, R>(bf, M.bc, 0.5, tl, dummy, S);
                R sc = R(0);
                for (int v = 0; v < 4; ++v) sc += Ll[v] * S[v];
                for (int i = 0; i < NSUBK; ++i) tc[f][i] = sc;
                constant = true;
            } else {
                const R nx = (R)bf.nx, ny = (R)bf.ny;
                for (int m = 0; m < NP; ++m) {
                    R w1 = u0[1][m], w2 = u0[2][m];
                    if (kind == BC_WALL) {
                        const R mn = w1 * nx + w2 * ny;
                        w1 -= R(2) * mn * nx;
                        w2 -= R(2) * mn * ny;
                    }
                    wc[m] = Ll[0] * u0[0][m] + Ll[1] * w1 + Ll[2] * w2 + Ll[3] * u0[3][m];
                }
            }
        }
        if (!constant)
            for (int i = 0; i < NSUBK; ++i) {
                R s = R(0);
                for (int m = 0; m < NP; ++m) s += op[O::W + (f * NSUBK + i) * NP + m] * wc[m];
                tc[f][i] = s;
            }
    }
    R w0 = R(0);
    for (int v = 0; v < 4; ++v) w0 += Ll[v] * ub[v];
    R md[NP - 1];
    weno_field<K, R, W>(op, tc, w0, md);
    for (int v = 0; v < 4; ++v)
        for (int i = 0; i < NP - 1; ++i) res[v][i] = R(0.5) * Rr[v] * md[i];
}

// KXRCF detection, one thread per cell, and warp-aggregated compaction of the
// flagged cells into flist (ctl->nflag counts them)
template <int EQ, int K, typename R>
__global__ void __launch_bounds__(128) k_detect(MeshDev<R> M, const R *__restrict__ u, Ctl *ctl, double tfac, double ck, R ck2, int all,
                                                uint8_t *__restrict__ flags, int32_t *__restrict__ flist)
{
    if (!ctl->active) return;
    __shared__ NbrTraceTab<R, K> ntab;
    ntab.fill(ltab<R, K>());
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    int flag = 0;
    if (c < M.nc) {
        flag = detect_cell<EQ, K, R>(M, u, ctl, tfac, ck, ck2, all, c, ntab);
        flags[c] = (uint8_t)flag;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, flag);
    if (mask) {
        const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&ctl->nflag, __popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (flag) flist[base + __popc(mask & ((1u << lane) - 1u))] = c;
    }
}

template <typename R>
void launch_detect(int eq, int k, const MeshDev<R> &M, const R *u, Ctl *ctl, double tfac, double ck, int all, uint8_t *flags,
                   int32_t *flist, cudaStream_t st)
{
    const int blk = 128, grd = (M.nc + blk - 1) / blk;
    const R ck2 = (R)(ck * ck);  // screening threshold in the state precision
#define CSW_D(E, KK) k_detect<E, KK, R><<<grd, blk, 0, st>>>(M, u, ctl, tfac, ck, ck2, all, flags, flist)
    if (eq == BURGERS && k == 1) CSW_D(BURGERS, 1);
    else if (eq == BURGERS && k == 2) CSW_D(BURGERS, 2);
    else if (eq == EULER && k == 1) CSW_D(EULER, 1);
    else CSW_D(EULER, 2);
#undef CSW_D
}
template void launch_detect<float>(int, int, const MeshDev<float> &, const float *, Ctl *, double, double, int, uint8_t *, int32_t *,
                                   cudaStream_t);
template void launch_detect<double>(int, int, const MeshDev<double> &, const double *, Ctl *, double, double, int, uint8_t *,
                                    int32_t *, cudaStream_t);

// KXRCF detection inside a time step, from the precursors the stage kernel
// wrote for its output (kx: face means, coefficient norm and means of each
// cell).  The Gauss-rule jump integral over face f, divided by the face
// length, is the cell's face mean minus the neighbour's face mean on the same
// face (a face mean does not depend on the orientation of the points); on boundary
// faces the ghost is integrated at the Gauss points as in detect_cell.  The
// decision is the same product form, screened in the state precision, with
// FP64 close calls.
// KXRCF decision of cell c from its precursor record: the jump integral over
// the inflow faces in face order (Sec. 3.1), compared in product form
template <int EQ, int K, typename R>
__device__ __forceinline__ int kx_flag(const MeshDev<R> &M, const R *__restrict__ u, const R (&k8)[KX_STRIDE], R kap, const Ctl *ctl,
                                       double tfac, double ck, R ck2, int c)
{
    constexpr int QF = Deg<K>::QF;
    const Tab<R, K> &T = ltab<R, K>();
    R num = R(0), lsum = R(0);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const R w = k8[KX_W0 + f];
        if (w == R(0)) continue;  // outflow face
        R J, nl;
        if (w > R(0)) {
            nl = w;
            J = k8[KX_I0 + f] - k8[KX_O0 + f];
        } else {
            nl = -w;
            const int code = M.nbr[f * M.ldc + c];
            const BFace bf = M.bf[-code - 1];
            const int kind = M.bc->kind[bf.tag];
            if (kind == BC_DIRICHLET || kind == BC_SHOCKLINE) {
                R go = R(0);
                for (int g = 0; g < QF; ++g) go += T.fw[g] * ghost0<EQ, R>(bf, M.bc, (double)T.ft[g], stage_time(ctl, tfac), R(0));
                J = k8[KX_I0 + f] - go;
            } else {
                J = R(0);  // transmissive and wall: the ghost indicator is the interior trace
            }
        }
        num += nl * J;
        lsum += nl;
    }
    R nrm2 = k8[KX_NRM2];
    // a negated norm marks a candidate of reading R-pos: the stage kernel's bound did not
    // show the new polynomial physical at every quadrature point; check the points
    if (nrm2 < R(0)) {
        if constexpr (EQ == EULER) {
            R uf[4][Deg<K>::NP];
            load_cell<4, Deg<K>::NP>(u, c, uf);
            if (nonphys_points_exact<K, R>(uf, T, M.gamma)) return 1;
        }
        nrm2 = -nrm2;
    }
    if (!(lsum > R(0))) return 0;
    const R denr = lsum * kap;
    const R lhs = num * num, rhs = ck2 * denr * denr * nrm2;
    if (rabs(lhs - rhs) > R(1e-3) * (lhs + rhs)) return lhs > rhs;
    const double den = (double)lsum * (double)kap;
    return (double)num * (double)num > ck * ck * den * den * (double)nrm2;
}

// Detection after a stage kernel: CPT cells per thread (cells c0, c0 + 128, ...
// of the block's range, so every load instruction of a warp covers consecutive
// records), all records and kappas loaded before the read of the step's active
// flag; no load depends on another.  Flagged cells are compacted per warp.
template <int EQ, int K, typename R, int CPT>
__global__ void __launch_bounds__(128) k_detect_kx(MeshDev<R> M, const R *__restrict__ u, const R *__restrict__ kx, Ctl *ctl, double tfac,
                                                   double ck, R ck2, int all, uint8_t *__restrict__ flags, int32_t *__restrict__ flist)
{
    const int c0 = blockIdx.x * blockDim.x * CPT + threadIdx.x;
    R k8[CPT][KX_STRIDE] = {}, kap[CPT] = {};
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        const int c = c0 + i * (int)blockDim.x;
        if (c < M.nc) {
            load_kx<R>(kx, c, k8[i]);
            if (!all) kap[i] = M.geo[G_KAPPA * M.ldc + c];
        }
    }
    if (!ctl->active) return;
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        const int c = c0 + i * (int)blockDim.x;
        int flag = 0;
        if (c < M.nc) {
            flag = all ? 1 : kx_flag<EQ, K, R>(M, u, k8[i], kap[i], ctl, tfac, ck, ck2, c);
            flags[c] = (uint8_t)flag;
        }
        const unsigned mask = __ballot_sync(0xffffffffu, flag);
        if (mask) {
            const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(&ctl->nflag, __popc(mask));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (flag) flist[base + __popc(mask & ((1u << lane) - 1u))] = c;
        }
    }
}

template <typename R>
void launch_detect_kx(int eq, int k, const MeshDev<R> &M, const R *u, const R *kx, Ctl *ctl, double tfac, double ck, int all,
                      uint8_t *flags, int32_t *flist, cudaStream_t st)
{
    constexpr int CPT = 1;  // 2 and 4 cells per thread measured slower (fewer warps in flight)
    const int blk = 128, grd = (M.nc + blk * CPT - 1) / (blk * CPT);
    const R ck2 = (R)(ck * ck);
#define CSW_DK(E, KK) k_detect_kx<E, KK, R, CPT><<<grd, blk, 0, st>>>(M, u, kx, ctl, tfac, ck, ck2, all, flags, flist)
    if (eq == BURGERS && k == 1) CSW_DK(BURGERS, 1);
    else if (eq == BURGERS && k == 2) CSW_DK(BURGERS, 2);
    else if (eq == EULER && k == 1) CSW_DK(EULER, 1);
    else CSW_DK(EULER, 2);
#undef CSW_DK
}
template void launch_detect_kx<float>(int, int, const MeshDev<float> &, const float *, const float *, Ctl *, double, double, int,
                                      uint8_t *, int32_t *, cudaStream_t);
template void launch_detect_kx<double>(int, int, const MeshDev<double> &, const double *, const double *, Ctl *, double, double, int,
                                       uint8_t *, int32_t *, cudaStream_t);

// ---------------------------------------------------------------------------
// Asynchronous bulk copies global -> shared memory completed on an mbarrier
// (cp.async.bulk, mbarrier.*: PTX ISA 8.0+, sm_90+).  Waits are bounded.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy writes
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    uint64_t g;
    asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(src));
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
                 "l"(g), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// poll limit of every bounded mbarrier wait (well under a second on this GPU)
constexpr int MBAR_POLLS = 1 << 22;
// wait for the phase with the given parity, at most `limit` polls (each poll
// may itself suspend for a hardware-defined time); true when it completed
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, int limit)
{
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Self-test of the bounded-wait error path (no counterpart in the paper): one
// warp waits, with the reconstruction kernel's wait primitive and a short poll
// limit, on an mbarrier phase that needs two arrivals and receives one (no
// copy is pending on it).  The wait runs out, ERR_TIMEOUT is set for the host
// and the warp returns.
__global__ void k_selftest_timeout(Ctl *ctl, int polls)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 2);
        mbar_arrive(&bar);
    }
    __syncwarp();
    const bool done = mbar_wait_bounded(&bar, 0, polls);
    if (!__all_sync(0xffffffffu, done) && threadIdx.x == 0) atomicOr(&ctl->err, ERR_TIMEOUT);
}
void launch_selftest_timeout(Ctl *ctl, int polls, cudaStream_t st) { k_selftest_timeout<<<1, 32, 0, st>>>(ctl, polls); }

// CSWENO reconstruction of the flagged cells flist[0 .. nflag) into
// lim_out[idx], from the unlimited state u.  Euler: eight lanes per cell (four
// cells per warp), contributions summed with shuffles; Burgers: one lane per
// cell.  The flagged cells are spread over the whole grid (a grid-stride loop
// over the compacted list), so cells clustered along a shock do not queue up
// in a few warps.
template <int EQ, int K, typename R, typename W>
__global__ void __launch_bounds__(128) k_limit(MeshDev<R> M, const R *__restrict__ u, const R *__restrict__ ops,
                                               const int32_t *__restrict__ flist, const Ctl *__restrict__ ctl, double tfac,
                                               R *__restrict__ lim_out)
{
    constexpr int NP = Deg<K>::NP, NV = Eqn<EQ>::NV;
    constexpr int G = (EQ == EULER) ? 8 : 1;  // lanes per flagged cell
    if (!ctl->active) return;
    const int n = ctl->nflag;
    const double tl = stage_time(ctl, tfac);
    const int warp0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    // the trip count is uniform across a warp, so the shuffles below see every lane
    for (int base = warp0; base / G < n; base += stride) {
        const int idx = (base + lane) / G;
        const bool active = idx < n;
        R res[NV][NP - 1];
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int i = 0; i < NP - 1; ++i) res[v][i] = R(0);
        const int c = active ? flist[idx] : 0;
        if (active) {
            if (EQ == EULER)
                limit_cell_euler_lane<K, R, W>(M, u, ops + (size_t)c * Ops<K>::SIZE, c, tl, lane & 7,
                                            *reinterpret_cast<R(*)[4][NP - 1]>(&res));
            else
                limit_cell<EQ, K, R, W>(M, u, ops + (size_t)c * Ops<K>::SIZE, c, tl, res);
        }
        if (EQ == EULER) {
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int i = 0; i < NP - 1; ++i) {
                    R x = res[v][i];
                    x += __shfl_xor_sync(0xffffffffu, x, 1);
                    x += __shfl_xor_sync(0xffffffffu, x, 2);
                    x += __shfl_xor_sync(0xffffffffu, x, 4);
                    res[v][i] = x;
                }
            bool bad = false;
            if (active) {
                R m0[4];
                for (int v = 0; v < NV; ++v) m0[v] = u[sidx(NV, NP, v, 0, c)];
                bad = positivity_bad_lane<K, R>(m0, *reinterpret_cast<R(*)[4][NP - 1]>(&res), lane & 7, M.gamma);
            }
            const unsigned grp = (__ballot_sync(0xffffffffu, bad) >> (lane & ~7)) & 0xffu;
            if (grp)
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int i = 0; i < NP - 1; ++i) res[v][i] = R(0);
        }
        if (active && (lane % G) == 0)
            for (int v = 0; v < NV; ++v)
                for (int i = 0; i < NP - 1; ++i) lim_out[((size_t)idx * NV + v) * (NP - 1) + i] = res[v][i];
    }
}

// Euler reconstruction with the operator blocks staged in shared memory: each
// warp handles four flagged cells per pass (eight lanes per cell, as in
// k_limit); lane 0 copies the four blocks (SIZE words each, contiguous in HBM)
// with one cp.async.bulk per cell on the warp's mbarrier, so the ~430 operator
// words a lane reads come from shared memory instead of as many dependent
// global loads.  A copy that does not complete within the poll limit sets
// ERR_TIMEOUT and the warp returns after a second bounded wait.
template <int K, typename R, typename W>
__global__ void __launch_bounds__(128) k_limit_euler_staged(MeshDev<R> M, const R *__restrict__ u, const R *__restrict__ ops,
                                                            const int32_t *__restrict__ flist, Ctl *ctl, double tfac,
                                                            R *__restrict__ lim_out)
{
    constexpr int NP = Deg<K>::NP, NV = 4, SZ = Ops<K>::SIZE, G = 8, CPW = 32 / G;
    constexpr int POLLS = MBAR_POLLS;
    extern __shared__ __align__(16) unsigned char dsm[];
    if (!ctl->active) return;
    const int n = ctl->nflag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    R *sop = reinterpret_cast<R *>(dsm) + (size_t)warp * CPW * SZ;
    uint64_t *bar = reinterpret_cast<uint64_t *>(dsm + (size_t)(blockDim.x >> 5) * CPW * SZ * sizeof(R)) + warp;
    const int warp0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    const int stride = gridDim.x * blockDim.x;
    if (warp0 / G >= n) return;  // no cell for this warp (uniform)
    const double tl = stage_time(ctl, tfac);
    if (lane == 0) mbar_init(bar, 1);
    __syncwarp();
    unsigned parity = 0;
    for (int base = warp0; base / G < n; base += stride) {  // trip count uniform across the warp
        const int idx = (base + lane) / G;
        const bool active = idx < n;
        const int c = active ? flist[idx] : 0;
        const int ncell = min(CPW, n - base / G);
        int cj[CPW];
#pragma unroll
        for (int j = 0; j < CPW; ++j) cj[j] = __shfl_sync(0xffffffffu, c, j * G);
        if (lane == 0) {
            fence_proxy_async_smem();  // the previous pass's reads of sop came before these writes
            mbar_arrive_expect_tx(bar, (unsigned)(ncell * SZ * sizeof(R)));
            for (int j = 0; j < ncell; ++j)
                bulk_copy_g2s(sop + j * SZ, ops + (size_t)cj[j] * SZ, (unsigned)(SZ * sizeof(R)), bar);
        }
        const bool done = mbar_wait_bounded(bar, parity, POLLS);
        if (!__all_sync(0xffffffffu, done)) {
            if (lane == 0) atomicOr(&ctl->err, ERR_TIMEOUT);
            mbar_wait_bounded(bar, parity, POLLS);  // let the copies in flight land before the block exits
            return;
        }
        parity ^= 1u;
        R res[NV][NP - 1];
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int i = 0; i < NP - 1; ++i) res[v][i] = R(0);
        if (active) limit_cell_euler_lane<K, R, W>(M, u, sop + (lane / G) * SZ, c, tl, lane & 7, res);
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int i = 0; i < NP - 1; ++i) {
                R x = res[v][i];
                x += __shfl_xor_sync(0xffffffffu, x, 1);
                x += __shfl_xor_sync(0xffffffffu, x, 2);
                x += __shfl_xor_sync(0xffffffffu, x, 4);
                res[v][i] = x;
            }
        bool bad = false;
        if (active) {
            R m0[4];
            for (int v = 0; v < NV; ++v) m0[v] = u[sidx(NV, NP, v, 0, c)];
            bad = positivity_bad_lane<K, R>(m0, res, lane & 7, M.gamma);
        }
        const unsigned grp = (__ballot_sync(0xffffffffu, bad) >> (lane & ~7)) & 0xffu;
        if (active && (lane & 7) == 0)
            for (int v = 0; v < NV; ++v)
                for (int i = 0; i < NP - 1; ++i) lim_out[((size_t)idx * NV + v) * (NP - 1) + i] = grp ? R(0) : res[v][i];
        __syncwarp();  // every lane is done with sop before lane 0 refills it
    }
}

template <int K, typename R> size_t staged_smem_bytes(int blk) { return (size_t)(blk / 32) * 4 * Ops<K>::SIZE * sizeof(R) + (blk / 32) * 8; }

template <typename R, typename W>
void launch_limit_w(int eq, int k, const MeshDev<R> &M, const R *u, const R *ops, const int32_t *flist, const Ctl *ctl, double tfac,
                    R *lim_out, int grid, cudaStream_t st)
{
    const int blk = 128;
    if (eq == BURGERS && k == 1) k_limit<BURGERS, 1, R, W><<<grid, blk, 0, st>>>(M, u, ops, flist, ctl, tfac, lim_out);
    else if (eq == BURGERS && k == 2) k_limit<BURGERS, 2, R, W><<<grid, blk, 0, st>>>(M, u, ops, flist, ctl, tfac, lim_out);
    else if (eq == EULER && k == 1) {
        const size_t sm = staged_smem_bytes<1, R>(blk);
        k_limit_euler_staged<1, R, W><<<grid, blk, sm, st>>>(M, u, ops, flist, const_cast<Ctl *>(ctl), tfac, lim_out);
    } else {
        const size_t sm = staged_smem_bytes<2, R>(blk);
        static bool attr_set = false;  // FP64 P2 needs more than the default 48 KB
        if (!attr_set && sm > 48 * 1024) {
            cudaFuncSetAttribute(k_limit_euler_staged<2, R, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            attr_set = true;
        }
        k_limit_euler_staged<2, R, W><<<grid, blk, sm, st>>>(M, u, ops, flist, const_cast<Ctl *>(ctl), tfac, lim_out);
    }
}

template <typename R>
void launch_limit(int eq, int k, const MeshDev<R> &M, const R *u, const R *ops, const int32_t *flist, const Ctl *ctl, double tfac,
                  R *lim_out, int grid, int w32, cudaStream_t st)
{
    // smoothness indicators and weights in double unless the FP32 mode asks for float
    if (sizeof(R) == 4 && w32) launch_limit_w<R, float>(eq, k, M, u, ops, flist, ctl, tfac, lim_out, grid, st);
    else launch_limit_w<R, double>(eq, k, M, u, ops, flist, ctl, tfac, lim_out, grid, st);
}
template void launch_limit<float>(int, int, const MeshDev<float> &, const float *, const float *, const int32_t *, const Ctl *, double,
                                  float *, int, int, cudaStream_t);
template void launch_limit<double>(int, int, const MeshDev<double> &, const double *, const double *, const int32_t *, const Ctl *,
                                   double, double *, int, int, cudaStream_t);

// write the reconstructed modes 1..np-1 of the flagged cells back into u: one
// thread per (cell, coefficient), so the reads of lim_out are coalesced
template <typename R>
__global__ void k_scatter(int nv, int np, const int32_t *__restrict__ flist, const R *__restrict__ lim_out, R *__restrict__ u,
                          Ctl *__restrict__ ctl)
{
    if (!ctl->active) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->nflag_sum += ctl->nflag;
    const int per = nv * (np - 1);
    const long long total = (long long)ctl->nflag * per;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int idx = (int)(t / per), r = (int)(t % per);
        u[sidx(nv, np, r / (np - 1), r % (np - 1) + 1, flist[idx])] = lim_out[t];
    }
}

template <typename R>
void launch_scatter(int nv, int np, int ld, const int32_t *flist, const R *lim_out, R *u, Ctl *ctl, int grid, cudaStream_t st)
{
    (void)ld;
    k_scatter<R><<<grid, 256, 0, st>>>(nv, np, flist, lim_out, u, ctl);
}
template void launch_scatter<float>(int, int, int, const int32_t *, const float *, float *, Ctl *, int, cudaStream_t);
template void launch_scatter<double>(int, int, int, const int32_t *, const double *, double *, Ctl *, int, cudaStream_t);


// ===========================================================================
// Reverse mode of the reconstruction with the troubled-cell flags frozen
// (the adjoint of a limiter pass).  All derivatives in W.
// ===========================================================================

// forward-mode number for the derivatives of the eigenvector entries
template <typename T> struct Dual {
    T v, d;
    __host__ __device__ Dual(T a = T(0), T b = T(0)) : v(a), d(b) {}
};
template <typename T> __host__ __device__ inline Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <typename T> __host__ __device__ inline Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <typename T> __host__ __device__ inline Dual<T> operator-(Dual<T> a) { return {-a.v, -a.d}; }
template <typename T> __host__ __device__ inline Dual<T> operator*(Dual<T> a, Dual<T> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <typename T> __host__ __device__ inline Dual<T> operator/(Dual<T> a, Dual<T> b)
{
    const T q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
template <typename T> __host__ __device__ inline Dual<T> rsqroot(Dual<T> a)
{
    const T s = sqrt(a.v);
    return {s, a.d / (T(2) * s)};
}

// dJ/d(ub) through the eigenvector row Ll and column Rr of one characteristic
// field: sum_v Llb[v] dLl[v]/dub_k + Rrb[v] dRr[v]/dub_k, by one forward-mode
// pass per component of ub
template <typename W>
__device__ __forceinline__ void eig_field_grad(const W *ub, W gam, W nx, W ny, int fl, const W (&Llb)[4], const W (&Rrb)[4], W (&out)[4])
{
    for (int k = 0; k < 4; ++k) {
        Dual<W> U[4], L[4], Rv[4];
        for (int v = 0; v < 4; ++v) U[v] = Dual<W>(ub[v], v == k ? W(1) : W(0));
        euler_eig_field<Dual<W>>(U, Dual<W>(gam), Dual<W>(nx), Dual<W>(ny), fl, L, Rv);
        W s = W(0);
        for (int v = 0; v < 4; ++v) s += Llb[v] * L[v].d + Rrb[v] * Rv[v].d;
        out[k] = s;
    }
}

// reverse of weno_field: from mdb = dJ/dmd (modes 1..NP-1) to tb[f][i] +=
// dJ/dt[f][i] and w0b += dJ/dw0; the forward quantities are recomputed here in W
template <int K, typename R, typename W>
__device__ __forceinline__ void weno_field_vjp(const R *__restrict__ op, const R (&t)[3][Ops<K>::NSUBK], R w0r,
                                               const W (&mdb)[Deg<K>::NP - 1], W (&tb)[3][Ops<K>::NSUBK], W &w0b)
{
    using O = Ops<K>;
    constexpr int NP = Deg<K>::NP, NM = Deg<K>::NM, NSUBK = O::NSUBK, NL = (K == 1) ? 3 : 4;
    const W eps = W(1e-10);
    const W w0 = (W)w0r;
    // ---- forward: Step 1 least-squares fits ----
    W b2[3], b3[9], b4[15];
    for (int s = 0; s < 3; ++s) b2[s] = (W)t[s][0] - w0;
    b3[0] = b2[0]; b3[1] = b2[1]; b3[2] = b2[2];
    for (int s = 0; s < 3; ++s) { b3[3 + 2 * s] = (W)t[s][1] - w0; b3[4 + 2 * s] = (W)t[s][2] - w0; }
    if (K == 2) {
        b4[0] = b2[0]; b4[1] = b2[1]; b4[2] = b2[2];
        for (int s = 0; s < 3; ++s)
            for (int i = 0; i < 4; ++i) b4[3 + 4 * s + i] = (W)t[s][(3 + i) % NSUBK] - w0;
    }
    W q2[2], q3[5], q4[9];
    for (int j = 0; j < 2; ++j) { W a = W(0); for (int s = 0; s < 3; ++s) a += (W)op[O::A2 + j * 3 + s] * b2[s]; q2[j] = a; }
    for (int j = 0; j < 5; ++j) { W a = W(0); for (int s = 0; s < 9; ++s) a += (W)op[O::A3 + j * 9 + s] * b3[s]; q3[j] = a; }
    if (K == 2)
        for (int j = 0; j < 9; ++j) { W a = W(0); for (int s = 0; s < 15; ++s) a += (W)op[O::A4 + j * 15 + s] * b4[s]; q4[j] = a; }
    // ---- Step 2 hierarchy ----
    const R *gm = op + O::GAM;
    const W g7 = (W)gm[7], g8 = (W)gm[8], g9 = (W)gm[9], g10 = (W)gm[10], g4 = (W)gm[4], g5 = (W)gm[5];
    W p[3][NM];
    for (int l = 0; l < 3; ++l) for (int j = 0; j < NM; ++j) p[l][j] = W(0);
    for (int j = 0; j < 2; ++j) p[0][j] = q2[j] * g7;
    for (int j = 0; j < 5; ++j) p[1][j] = (q3[j] - g10 * p[0][j]) * g8;
    if (K == 2) for (int j = 0; j < 9; ++j) p[2][j] = (q4[j] - g4 * p[0][j] - g5 * p[1][j]) * g9;
    // ---- Step 3 smoothness indicators: y = L^T p_l, beta = |y|^2 ----
    const R *L = op + O::LH;
    const int nn[3] = {2, 5, 9};
    W y[3][NM], beta[4];
    for (int l = 0; l < NL - 1; ++l) {
        W acc = W(0);
        for (int j = 0; j < nn[l]; ++j) {
            W a = W(0);
            for (int i = j; i < nn[l]; ++i) a += (W)L[i * (i + 1) / 2 + j] * p[l][i];
            y[l][j] = a;
            acc += a * a;
        }
        beta[l + 1] = acc;
    }
    // beta_1 magnified (sigma weights in quotient form: the same normalised weights)
    W al[3], bl[3], b1[3], e[3];
    for (int f = 0; f < 3; ++f) {
        const W r1 = (W)t[f][1] - (W)t[f][0], r2 = (W)t[f][2] - (W)t[f][0];
        al[f] = (W)op[O::MI + 4 * f + 0] * r1 + (W)op[O::MI + 4 * f + 1] * r2;
        bl[f] = (W)op[O::MI + 4 * f + 2] * r1 + (W)op[O::MI + 4 * f + 3] * r2;
        b1[f] = al[f] * al[f] + bl[f] * bl[f];
        e[f] = b1[f] + eps;
    }
    // D: mean absolute difference of the beta_{1,l} (reading R-sigma); sgn: its derivative
    const W d01 = b1[0] - b1[1], d12 = b1[1] - b1[2], d20 = b1[2] - b1[0];
    const W s01 = (d01 > W(0)) ? W(1) : ((d01 < W(0)) ? W(-1) : W(0));
    const W s12 = (d12 > W(0)) ? W(1) : ((d12 < W(0)) ? W(-1) : W(0));
    const W s20 = (d20 > W(0)) ? W(1) : ((d20 < W(0)) ? W(-1) : W(0));
    const W D = (fabs(d01) + fabs(d12) + fabs(d20)) / W(3), D2 = D * D;
    W sg[3], Ss = W(0);
    for (int f = 0; f < 3; ++f) { sg[f] = W(1) + D2 / e[f]; Ss += sg[f]; }
    W ab = W(0), bb = W(0);
    for (int f = 0; f < 3; ++f) { ab += sg[f] * al[f]; bb += sg[f] * bl[f]; }
    ab /= Ss;
    bb /= Ss;
    beta[0] = ab * ab + bb * bb;
    // ---- Step 4 tau and weights (reading R-weno), in double whatever W: the ratio's
    // power K+1 and its derivative (tau / a)^(K+1) / a reach 1e40 when a beta vanishes ----
    constexpr int PW = K + 1;
    const double ctau = (K == 1) ? 0.5 : 1.0 / 3.0;
    double tau = 0.0, sgn[3];
    for (int l = 0; l < NL - 1; ++l) {
        const double d = (double)beta[NL - 1] - (double)beta[l];
        sgn[l] = (d > 0.0) ? 1.0 : ((d < 0.0) ? -1.0 : 0.0);
        tau += fabs(d);
    }
    tau *= ctau;
    const R *gl = gm + ((K == 1) ? 0 : 3);
    double a[4], rp[4], z[4], Sz = 0.0;
    W om[4];
    for (int l = 0; l < NL; ++l) {
        a[l] = 1e-10 + (double)beta[l];
        const double r = tau / a[l];
        rp[l] = r;
        for (int e = 1; e < PW; ++e) rp[l] *= r;  // (tau / a_l)^(K+1)
        z[l] = (double)gl[l] * (1.0 + rp[l]);
        Sz += z[l];
    }
    for (int l = 0; l < NL; ++l) om[l] = (W)(z[l] / Sz);
    // ---- reverse: Step 5 projection ----
    W cmb[NM];
    for (int j = 0; j < NM; ++j) {
        W s = W(0);
        for (int i = 0; i < NP - 1; ++i) s += (W)op[O::PHI + i * NM + j] * mdb[i];
        cmb[j] = s;
    }
    W omb[4] = {W(0), W(0), W(0), W(0)}, pb[3][NM];
    for (int l = 0; l < 3; ++l)
        for (int j = 0; j < NM; ++j) pb[l][j] = W(0);
    for (int l = 1; l < NL; ++l) {
        W s = W(0);
        for (int j = 0; j < NM; ++j) { s += cmb[j] * p[l - 1][j]; pb[l - 1][j] = om[l] * cmb[j]; }
        omb[l] = s;
    }
    // ---- Step 4 reverse: z_l = gamma_l (1 + (tau/a_l)^P), d z_l/d tau = gamma_l P (tau/a_l)^P / tau,
    // d z_l/d a_l = -gamma_l P (tau/a_l)^P / a_l ----
    double dot = 0.0;
    for (int l = 0; l < NL; ++l) dot += (double)omb[l] * (double)om[l];
    double betabd[4] = {0.0, 0.0, 0.0, 0.0}, taub = 0.0;
    for (int l = 0; l < NL; ++l) {
        const double zb = ((double)omb[l] - dot) / Sz;
        const double g = zb * (double)gl[l] * PW * rp[l];
        if (tau > 0.0) taub += g / tau;
        betabd[l] -= g / a[l];
    }
    for (int l = 0; l < NL - 1; ++l) {
        betabd[l] -= ctau * sgn[l] * taub;
        betabd[NL - 1] += ctau * sgn[l] * taub;
    }
    W betab[4];
    for (int l = 0; l < 4; ++l) betab[l] = (W)betabd[l];
    // ---- Step 3 reverse: beta_l = |L^T p|^2 -> p_b += 2 beta_b L y ----
    for (int l = 0; l < NL - 1; ++l)
        for (int i = 0; i < nn[l]; ++i) {
            W s = W(0);
            for (int j = 0; j <= i; ++j) s += (W)L[i * (i + 1) / 2 + j] * y[l][j];
            pb[l][i] += W(2) * betab[l + 1] * s;
        }
    // beta_1 magnification reverse
    {
        const W abb = W(2) * ab * betab[0], bbb = W(2) * bb * betab[0];
        W alb[3], blb[3], b1b[3], sgb[3];
        for (int f = 0; f < 3; ++f) {
            alb[f] = abb * sg[f] / Ss;
            blb[f] = bbb * sg[f] / Ss;
            sgb[f] = (abb * (al[f] - ab) + bbb * (bl[f] - bb)) / Ss;
        }
        W D2b = W(0);
        for (int f = 0; f < 3; ++f) { b1b[f] = -sgb[f] * D2 / (e[f] * e[f]); D2b += sgb[f] / e[f]; }
        const W Db = W(2) * D * D2b;
        b1b[0] += Db * (s01 - s20) / W(3);
        b1b[1] += Db * (s12 - s01) / W(3);
        b1b[2] += Db * (s20 - s12) / W(3);
        for (int f = 0; f < 3; ++f) {
            alb[f] += W(2) * al[f] * b1b[f];
            blb[f] += W(2) * bl[f] * b1b[f];
            const W r1b = (W)op[O::MI + 4 * f + 0] * alb[f] + (W)op[O::MI + 4 * f + 2] * blb[f];
            const W r2b = (W)op[O::MI + 4 * f + 1] * alb[f] + (W)op[O::MI + 4 * f + 3] * blb[f];
            tb[f][1] += r1b;
            tb[f][2] += r2b;
            tb[f][0] -= r1b + r2b;
        }
    }
    // ---- Step 2 reverse ----
    W q2b[2], q3b[5], q4b[9];
    if (K == 2)
        for (int j = 0; j < 9; ++j) {
            q4b[j] = g9 * pb[2][j];
            pb[0][j] -= g4 * g9 * pb[2][j];
            pb[1][j] -= g5 * g9 * pb[2][j];
        }
    for (int j = 0; j < 5; ++j) {
        q3b[j] = g8 * pb[1][j];
        pb[0][j] -= g10 * g8 * pb[1][j];
    }
    for (int j = 0; j < 2; ++j) q2b[j] = g7 * pb[0][j];
    // ---- Step 1 reverse ----
    W sumb = W(0);
    for (int s = 0; s < 3; ++s) {
        W bs = W(0);
        for (int j = 0; j < 2; ++j) bs += (W)op[O::A2 + j * 3 + s] * q2b[j];
        tb[s][0] += bs;
        sumb += bs;
    }
    for (int s = 0; s < 9; ++s) {
        W bs = W(0);
        for (int j = 0; j < 5; ++j) bs += (W)op[O::A3 + j * 9 + s] * q3b[j];
        if (s < 3) tb[s][0] += bs;
        else tb[(s - 3) / 2][1 + ((s - 3) & 1)] += bs;
        sumb += bs;
    }
    if (K == 2)
        for (int s = 0; s < 15; ++s) {
            W bs = W(0);
            for (int j = 0; j < 9; ++j) bs += (W)op[O::A4 + j * 15 + s] * q4b[j];
            if (s < 3) tb[s][0] += bs;
            else tb[(s - 3) / 4][(3 + (s - 3) % 4) % NSUBK] += bs;
            sumb += bs;
        }
    w0b -= sumb;
}

// One lane (direction d, characteristic field fl) of the reverse of
// limit_cell_euler_lane: rb = dJ/d(reconstructed modes 1..NP-1) of the cell.
// Adds to own[v][m] (the cell's own modes: the mean through the eigenvectors
// and w0, all modes through mirrored ghosts) and nb[f][v][m] (face f's
// neighbour).
template <int K, typename R, typename W>
__device__ __forceinline__ void limit_lane_euler_vjp(const MeshDev<R> &M, const R *__restrict__ u, const R *__restrict__ op, int c,
                                                     double tl, int lane8, const W (&rb)[4][Deg<K>::NP - 1], W (&own)[4][Deg<K>::NP],
                                                     W (&nb)[3][4][Deg<K>::NP])
{
    using O = Ops<K>;
    constexpr int NP = Deg<K>::NP, NSUBK = O::NSUBK;
    const int ld = M.ldc;
    const int d = lane8 >> 2, fl = lane8 & 3;
    const R is2 = R(0.70710678118654752440);
    R u0[4][NP];
    load_cell<4, NP>(u, c, u0);
    R ub[4];
    for (int v = 0; v < 4; ++v) ub[v] = u0[v][0] * is2;
    R Ll[4], Rr[4];
    const R nxd = d == 0 ? R(1) : R(0), nyd = d == 0 ? R(0) : R(1);
    euler_eig_field<R>(ub, M.gammar, nxd, nyd, fl, Ll, Rr);
    // forward: characteristic subcell means
    R tc[3][NSUBK], wcs[3][NP], S[3][4];
    int kinds[3], codes[3];
    for (int f = 0; f < 3; ++f) {
        const int code = M.nbr[f * ld + c];
        codes[f] = code;
        kinds[f] = -1;  // internal
        if (code >= 0) {
            R wn[4][NP];
            load_cell<4, NP>(u, code, wn);
            for (int m = 0; m < NP; ++m) {
                R s = R(0);
                for (int v = 0; v < 4; ++v) s += Ll[v] * wn[v][m];
                wcs[f][m] = s;
            }
        } else {
            const BFace bf = M.bf[-code - 1];
            kinds[f] = M.bc->kind[bf.tag];
            if (kinds[f] == BC_DIRICHLET || kinds[f] == BC_SHOCKLINE) {
                R dummy[4] = {R(0), R(0), R(0), R(0)};
                ghost<EULER, R>(bf, M.bc, 0.5, tl, dummy, S[f]);
                R sc = R(0);
                for (int v = 0; v < 4; ++v) sc += Ll[v] * S[f][v];
                for (int i = 0; i < NSUBK; ++i) tc[f][i] = sc;
                continue;
            }
            const R nx = (R)bf.nx, ny = (R)bf.ny;
            for (int m = 0; m < NP; ++m) {
                R w1 = u0[1][m], w2 = u0[2][m];
                if (kinds[f] == BC_WALL) {
                    const R mn = w1 * nx + w2 * ny;
                    w1 -= R(2) * mn * nx;
                    w2 -= R(2) * mn * ny;
                }
                wcs[f][m] = Ll[0] * u0[0][m] + Ll[1] * w1 + Ll[2] * w2 + Ll[3] * u0[3][m];
            }
        }
        for (int i = 0; i < NSUBK; ++i) {
            R s = R(0);
            for (int m = 0; m < NP; ++m) s += op[O::W + (f * NSUBK + i) * NP + m] * wcs[f][m];
            tc[f][i] = s;
        }
    }
    R w0 = R(0);
    for (int v = 0; v < 4; ++v) w0 += Ll[v] * ub[v];
    R md[NP - 1];
    weno_field<K, R, W>(op, tc, w0, md);
    // reverse: res[v][i] = 1/2 Rr[v] md[i]
    W mdb[NP - 1], Rrb[4], Llb[4], ubb[4];
    for (int i = 0; i < NP - 1; ++i) {
        W s = W(0);
        for (int v = 0; v < 4; ++v) s += W(0.5) * (W)Rr[v] * rb[v][i];
        mdb[i] = s;
    }
    for (int v = 0; v < 4; ++v) {
        W s = W(0);
        for (int i = 0; i < NP - 1; ++i) s += W(0.5) * (W)md[i] * rb[v][i];
        Rrb[v] = s;
    }
    W tcb[3][NSUBK], w0b = W(0);
    for (int f = 0; f < 3; ++f)
        for (int i = 0; i < NSUBK; ++i) tcb[f][i] = W(0);
    weno_field_vjp<K, R, W>(op, tc, w0, mdb, tcb, w0b);
    for (int v = 0; v < 4; ++v) { Llb[v] = w0b * (W)ub[v]; ubb[v] = w0b * (W)Ll[v]; }
    for (int f = 0; f < 3; ++f) {
        if (kinds[f] == BC_DIRICHLET || kinds[f] == BC_SHOCKLINE) {
            W s = W(0);
            for (int i = 0; i < NSUBK; ++i) s += tcb[f][i];
            for (int v = 0; v < 4; ++v) Llb[v] += s * (W)S[f][v];
            continue;
        }
        W wcb[NP];
        for (int m = 0; m < NP; ++m) {
            W s = W(0);
            for (int i = 0; i < NSUBK; ++i) s += (W)op[O::W + (f * NSUBK + i) * NP + m] * tcb[f][i];
            wcb[m] = s;
        }
        if (codes[f] >= 0) {
            R wn[4][NP];
            load_cell<4, NP>(u, codes[f], wn);
            for (int v = 0; v < 4; ++v)
                for (int m = 0; m < NP; ++m) {
                    nb[f][v][m] += (W)Ll[v] * wcb[m];
                    Llb[v] += wcb[m] * (W)wn[v][m];
                }
        } else {
            const BFace bf = M.bf[-codes[f] - 1];
            const W nx = (W)(R)bf.nx, ny = (W)(R)bf.ny;
            for (int m = 0; m < NP; ++m) {
                W w1 = (W)u0[1][m], w2 = (W)u0[2][m];
                W g1 = (W)Ll[1] * wcb[m], g2 = (W)Ll[2] * wcb[m];
                if (kinds[f] == BC_WALL) {
                    const W mn = w1 * nx + w2 * ny, gn = g1 * nx + g2 * ny;
                    w1 -= W(2) * mn * nx;
                    w2 -= W(2) * mn * ny;
                    g1 -= W(2) * gn * nx;  // the reflection is symmetric
                    g2 -= W(2) * gn * ny;
                }
                own[0][m] += (W)Ll[0] * wcb[m];
                own[1][m] += g1;
                own[2][m] += g2;
                own[3][m] += (W)Ll[3] * wcb[m];
                Llb[0] += wcb[m] * (W)u0[0][m];
                Llb[1] += wcb[m] * w1;
                Llb[2] += wcb[m] * w2;
                Llb[3] += wcb[m] * (W)u0[3][m];
            }
        }
    }
    W ubw[4], eg[4];
    for (int v = 0; v < 4; ++v) ubw[v] = (W)ub[v];
    eig_field_grad<W>(ubw, (W)M.gammar, (W)nxd, (W)nyd, fl, Llb, Rrb, eg);
    for (int v = 0; v < 4; ++v) own[v][0] += (ubb[v] + eg[v]) * (W)is2;
}

// Burgers: one lane per flagged cell, the reverse of limit_cell
template <int K, typename R, typename W>
__device__ __forceinline__ void limit_cell_burgers_vjp(const MeshDev<R> &M, const R *__restrict__ u, const R *__restrict__ op, int c,
                                                       double tl, const W (&rb)[Deg<K>::NP - 1], W (&own)[Deg<K>::NP],
                                                       W (&nb)[3][Deg<K>::NP])
{
    using O = Ops<K>;
    constexpr int NP = Deg<K>::NP, NSUBK = O::NSUBK;
    const int ld = M.ldc;
    R u0[NP];
    for (int m = 0; m < NP; ++m) u0[m] = u[sidx(1, NP, 0, m, c)];
    R t[3][NSUBK];
    int codes[3], kinds[3];
    for (int f = 0; f < 3; ++f) {
        const int code = M.nbr[f * ld + c];
        codes[f] = code;
        kinds[f] = -1;
        R w[NP];
        if (code >= 0) {
            for (int m = 0; m < NP; ++m) w[m] = u[sidx(1, NP, 0, m, code)];
        } else {
            const BFace bf = M.bf[-code - 1];
            kinds[f] = M.bc->kind[bf.tag];
            if (kinds[f] == BC_DIRICHLET || kinds[f] == BC_SHOCKLINE) {
                R Sv[1], dummy[1] = {R(0)};
                ghost<BURGERS, R>(bf, M.bc, 0.5, tl, dummy, Sv);
                for (int i = 0; i < NSUBK; ++i) t[f][i] = Sv[0];
                continue;
            }
            for (int m = 0; m < NP; ++m) w[m] = u0[m];
        }
        for (int i = 0; i < NSUBK; ++i) {
            R s = R(0);
            for (int m = 0; m < NP; ++m) s += op[O::W + (f * NSUBK + i) * NP + m] * w[m];
            t[f][i] = s;
        }
    }
    const R w0 = u0[0] * R(0.70710678118654752440);
    W tb[3][NSUBK], w0b = W(0);
    for (int f = 0; f < 3; ++f)
        for (int i = 0; i < NSUBK; ++i) tb[f][i] = W(0);
    weno_field_vjp<K, R, W>(op, t, w0, rb, tb, w0b);
    own[0] += w0b * W(0.70710678118654752440);
    for (int f = 0; f < 3; ++f) {
        if (kinds[f] == BC_DIRICHLET || kinds[f] == BC_SHOCKLINE) continue;
        for (int m = 0; m < NP; ++m) {
            W s = W(0);
            for (int i = 0; i < NSUBK; ++i) s += (W)op[O::W + (f * NSUBK + i) * NP + m] * tb[f][i];
            if (codes[f] >= 0) nb[f][m] += s;
            else own[m] += s;
        }
    }
}

// Adjoint of one limiter pass with the flags of the forward pass frozen:
// gout (prepared by the caller as gin with the flagged cells' modes 1..NP-1
// zeroed) += the reconstruction's transposed derivative applied to gin's
// modes 1..NP-1 of every flagged cell.  u: the state the forward pass
// reconstructed from (before it was limited).  A reconstruction that the
// forward pass replaced by the cell mean (positivity fallback) contributes
// nothing.  Contributions to shared neighbours are added atomically.
template <int EQ, int K, typename R, typename W>
__global__ void __launch_bounds__(128) k_limit_adj(MeshDev<R> M, const R *__restrict__ u, const R *__restrict__ ops,
                                                   const int32_t *__restrict__ flist, const int32_t *__restrict__ nflag_dev,
                                                   const Ctl *__restrict__ ctl, double tfac, const R *__restrict__ gin, R *gout)
{
    constexpr int NP = Deg<K>::NP, NV = Eqn<EQ>::NV;
    constexpr int G = (EQ == EULER) ? 8 : 1;
    const int n = *nflag_dev;
    const double tl = stage_time(ctl, tfac);
    const int warp0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    for (int base = warp0; base / G < n; base += stride) {  // trip count uniform across the warp
        const int idx = (base + lane) / G;
        const bool active = idx < n;
        const int c = active ? flist[idx] : 0;
        const R *op = ops + (size_t)c * Ops<K>::SIZE;
        if (EQ == EULER) {
            // forward result of the cell, to see whether the positivity fallback applied
            R res[4][NP - 1];
            for (int v = 0; v < 4; ++v)
                for (int i = 0; i < NP - 1; ++i) res[v][i] = R(0);
            if (active) limit_cell_euler_lane<K, R, W>(M, u, op, c, tl, lane & 7, res);
            for (int v = 0; v < 4; ++v)
                for (int i = 0; i < NP - 1; ++i) {
                    R x = res[v][i];
                    x += __shfl_xor_sync(0xffffffffu, x, 1);
                    x += __shfl_xor_sync(0xffffffffu, x, 2);
                    x += __shfl_xor_sync(0xffffffffu, x, 4);
                    res[v][i] = x;
                }
            bool bad = false;
            if (active) {
                R m0[4];
                for (int v = 0; v < 4; ++v) m0[v] = u[sidx(4, NP, v, 0, c)];
                bad = positivity_bad_lane<K, R>(m0, res, lane & 7, M.gamma);
            }
            const unsigned grp = (__ballot_sync(0xffffffffu, bad) >> (lane & ~7)) & 0xffu;
            W own[4][NP], nbg[3][4][NP], rb[4][NP - 1];
            for (int v = 0; v < 4; ++v)
                for (int m = 0; m < NP; ++m) {
                    own[v][m] = W(0);
                    for (int f = 0; f < 3; ++f) nbg[f][v][m] = W(0);
                }
            if (active && !grp) {
                for (int v = 0; v < 4; ++v)
                    for (int i = 0; i < NP - 1; ++i) rb[v][i] = (W)gin[sidx(4, NP, v, i + 1, c)];
                limit_lane_euler_vjp<K, R, W>(M, u, op, c, tl, lane & 7, rb, own, nbg);
            }
            // sum the eight lanes' contributions; lane 0 of the group adds them
            for (int v = 0; v < 4; ++v)
                for (int m = 0; m < NP; ++m) {
                    W x = own[v][m];
                    x += __shfl_xor_sync(0xffffffffu, x, 1);
                    x += __shfl_xor_sync(0xffffffffu, x, 2);
                    x += __shfl_xor_sync(0xffffffffu, x, 4);
                    own[v][m] = x;
                    for (int f = 0; f < 3; ++f) {
                        W y = nbg[f][v][m];
                        y += __shfl_xor_sync(0xffffffffu, y, 1);
                        y += __shfl_xor_sync(0xffffffffu, y, 2);
                        y += __shfl_xor_sync(0xffffffffu, y, 4);
                        nbg[f][v][m] = y;
                    }
                }
            if (active && !grp && (lane & 7) == 0) {
                for (int v = 0; v < 4; ++v)
                    for (int m = 0; m < NP; ++m) atomicAdd(&gout[sidx(4, NP, v, m, c)], (R)own[v][m]);
                for (int f = 0; f < 3; ++f) {
                    const int code = M.nbr[f * M.ldc + c];
                    if (code < 0) continue;
                    for (int v = 0; v < 4; ++v)
                        for (int m = 0; m < NP; ++m) atomicAdd(&gout[sidx(4, NP, v, m, code)], (R)nbg[f][v][m]);
                }
            }
        } else if (active) {
            W rb[NP - 1], own[NP], nbg[3][NP];
            for (int i = 0; i < NP - 1; ++i) rb[i] = (W)gin[sidx(1, NP, 0, i + 1, c)];
            for (int m = 0; m < NP; ++m) {
                own[m] = W(0);
                for (int f = 0; f < 3; ++f) nbg[f][m] = W(0);
            }
            limit_cell_burgers_vjp<K, R, W>(M, u, op, c, tl, rb, own, nbg);
            for (int m = 0; m < NP; ++m) atomicAdd(&gout[sidx(1, NP, 0, m, c)], (R)own[m]);
            for (int f = 0; f < 3; ++f) {
                const int code = M.nbr[f * M.ldc + c];
                if (code < 0) continue;
                for (int m = 0; m < NP; ++m) atomicAdd(&gout[sidx(1, NP, 0, m, code)], (R)nbg[f][m]);
            }
        }
    }
}

// zero modes 1..np-1 of the listed cells (the limited modes do not pass through)
template <typename R>
__global__ void k_zero_flagged(int nv, int np, const int32_t *__restrict__ flist, const int32_t *__restrict__ nflag_dev, R *g)
{
    const int n = *nflag_dev;
    const int per = nv * (np - 1);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * per; t += (long long)gridDim.x * blockDim.x) {
        const int idx = (int)(t / per), r = (int)(t % per);
        g[sidx(nv, np, r / (np - 1), r % (np - 1) + 1, flist[idx])] = R(0);
    }
}

template <typename R>
void launch_limit_adjoint(int eq, int k, const MeshDev<R> &M, const R *u, const R *ops, const int32_t *flist, const int32_t *nflag_dev,
                          const Ctl *ctl, double tfac, int w32, const R *gin, R *gout, int grid, cudaStream_t st)
{
    const int nv = (eq == EULER) ? 4 : 1, np = (k == 1) ? 3 : 6;
    k_zero_flagged<R><<<grid, 256, 0, st>>>(nv, np, flist, nflag_dev, gout);
#define CSW_LA(E, KK, WW) k_limit_adj<E, KK, R, WW><<<grid, 128, 0, st>>>(M, u, ops, flist, nflag_dev, ctl, tfac, gin, gout)
    if (sizeof(R) == 4 && w32) {
        if (eq == BURGERS && k == 1) CSW_LA(BURGERS, 1, float);
        else if (eq == BURGERS) CSW_LA(BURGERS, 2, float);
        else if (k == 1) CSW_LA(EULER, 1, float);
        else CSW_LA(EULER, 2, float);
    } else {
        if (eq == BURGERS && k == 1) CSW_LA(BURGERS, 1, double);
        else if (eq == BURGERS) CSW_LA(BURGERS, 2, double);
        else if (k == 1) CSW_LA(EULER, 1, double);
        else CSW_LA(EULER, 2, double);
    }
#undef CSW_LA
}
template void launch_limit_adjoint<float>(int, int, const MeshDev<float> &, const float *, const float *, const int32_t *,
                                          const int32_t *, const Ctl *, double, int, const float *, float *, int, cudaStream_t);
template void launch_limit_adjoint<double>(int, int, const MeshDev<double> &, const double *, const double *, const int32_t *,
                                           const int32_t *, const Ctl *, double, int, const double *, double *, int, cudaStream_t);

}  // namespace csw
