// kernels.h -- host-side launchers of the CUDA kernels (one translation unit
// per group of kernels; this header is the only coupling between them).
#pragma once
#include "../../include/cswdg.h"
#include "common.cuh"

namespace csw {

// per-cell CSWENO operator block (REAL values, one block per cell)
template <int K> struct Ops {
    static constexpr int NP = Deg<K>::NP, NM = Deg<K>::NM;
    static constexpr int NSUBK = (K == 1) ? 3 : 7;      // thirds (+ halves for P2)
    static constexpr int W = 0;                          // [3][NSUBK][NP] subcell-mean weights
    static constexpr int A2 = W + 3 * NSUBK * NP;        // [2][3]  pseudo-inverse, linear fit on T2
    static constexpr int A3 = A2 + 6;                    // [5][9]  quadratic fit on T3
    static constexpr int A4 = A3 + 45;                   // [9][15] cubic fit on T4 (P2)
    static constexpr int LH = A4 + ((K == 2) ? 135 : 0); // packed lower Cholesky factor of the beta form
    static constexpr int MI = LH + NM * (NM + 1) / 2;    // [3][2][2] beta_1 gradient maps
    static constexpr int PHI = MI + 12;                  // [NP-1][NM] projection to modes 1..NP-1
    // linear weights of Step 2 and their use: gamma_{l,3} (3), gamma_{l,5} (4),
    // 1/gamma_{2,2}, 1/gamma_{3,3}, 1/gamma_{4,5}, gamma_{2,3}, mean side length
    static constexpr int GAM = PHI + (NP - 1) * NM;
    // padded to four words: 16-byte rows for the bulk copies into shared memory
    static constexpr int SIZE = (GAM + 12 + 3) & ~3;
};

cudaError_t operator_upload_tables();
cudaError_t limiter_upload_tables();
cudaError_t adjoint_upload_tables();

// launch shape of the stage kernel: cells per block (64, 128, 256), the
// number of blocks (0: one block per tile of cells; > 0: a persistent grid) and
// the variant (tile_faces 0: k_stage, every cell computes its three faces;
// 1: k_stage_tiles, each face once per tile, 128 or 256 cells per block)
struct StageShape {
    int blk = 128, grid = 0, tile_faces = 0;
};
// sets the dynamic shared memory limits of the tile-shared stage kernels on
// the current device
cudaError_t stage_kernels_prepare();
template <typename R>
void launch_stage(int eq, int k, const MeshDev<R> &M, const R *un, const R *up, R *out, R ca, R cb, R cl, double tfac,
                  int lam_next, R *kx, Ctl *ctl, StageShape sh, cudaStream_t st);
template <typename R> void launch_cfl(int eq, const MeshDev<R> &M, int np, const R *u, Ctl *ctl, cudaStream_t st);
void launch_begin_step(Ctl *ctl, int use_cfl, cudaStream_t st);
void launch_set_step_params(Ctl *ctl, double dt_fixed, double cfl, double t_end, cudaStream_t st);
// one warp waits (at most polls polls) on an mbarrier phase that never
// completes; sets ERR_TIMEOUT
void launch_selftest_timeout(Ctl *ctl, int polls, cudaStream_t st);
template <typename R> void launch_project(int k, int nc, int ld, int nv, const double *vals, R *u, cudaStream_t st);
template <typename R, typename U>
void launch_from_user(int nc, int ld, int nv, int np, const int32_t *perm, const double *sc, const U *user, R *u, cudaStream_t st);
template <typename R, typename U>
void launch_to_user(int nc, int ld, int nv, int np, const int32_t *perm, const double *sc, const R *u, U *user, cudaStream_t st);
void launch_flags_to_user(int nc, const int32_t *perm, const uint8_t *fl, uint8_t *out, cudaStream_t st);
template <typename R>
void launch_conservation(int nc, int ld, int nv, int np, const double *area, const R *u, double *part, double *out, cudaStream_t st);

// adjoint of the operator at the stage time t + tfac dt, combined on output:
// grad = ax x + ay y + beta (d L_h / d u)^T lam (x, y nullable; grad may alias
// x or y but not u or lam)
template <typename R>
void launch_rhs_adjoint(int eq, int k, const MeshDev<R> &M, const R *u, const R *lam, R *grad, double tfac, const Ctl *ctl,
                        cudaStream_t st, const R *x = nullptr, R ax = R(0), const R *y = nullptr, R ay = R(0), R beta = R(1));

// adjoint of a limiter pass with frozen flags (flist, *nflag_dev): gout = gin
// with the flagged cells' modes 1..np-1 replaced by the reconstruction's
// transposed derivative contributions; u is the unlimited state of the pass
template <typename R>
void launch_limit_adjoint(int eq, int k, const MeshDev<R> &M, const R *u, const R *ops, const int32_t *flist, const int32_t *nflag_dev,
                          const Ctl *ctl, double tfac, int w32, const R *gin, R *gout, int grid, cudaStream_t st);

// out = a x + b y (y nullable) over n entries
template <typename R> void launch_axpby(size_t n, R a, const R *x, R b, const R *y, R *out, int grid, cudaStream_t st);

// read-only view of a solver for entry points outside api.cu (false: no mesh)
bool solver_view(const struct ::cswdg_solver *s, int *nc, int *ldc, int *nvar, int *np, int *fp32, const double **area,
                 void **stream, int *device);
// record an error on the solver and return the status
cswdg_status solver_fail(struct ::cswdg_solver *s, cswdg_status st, const char *fmt, ...);

// limiter
void launch_setup_ops(int k, int nc, int ld, const double *vtx, const double *nvtx, const int32_t *nbr, const uint8_t *nbf,
                      double *ops, int32_t *err, cudaStream_t st);
void launch_ops_to_float(size_t n, const double *src, float *dst, cudaStream_t st);
template <typename R>
void launch_detect(int eq, int k, const MeshDev<R> &M, const R *u, Ctl *ctl, double tfac, double ck, int all, uint8_t *flags,
                   int32_t *flist, cudaStream_t st);
// KXRCF detection from the precursors the stage kernel wrote (kx)
template <typename R>
void launch_detect_kx(int eq, int k, const MeshDev<R> &M, const R *u, const R *kx, Ctl *ctl, double tfac, double ck, int all,
                      uint8_t *flags, int32_t *flist, cudaStream_t st);
// w32: smoothness indicators and nonlinear weights in float (FP32 mode), else double
template <typename R>
void launch_limit(int eq, int k, const MeshDev<R> &M, const R *u, const R *ops, const int32_t *flist, const Ctl *ctl,
                  double tfac, R *lim_out, int grid, int w32, cudaStream_t st);
template <typename R>
void launch_scatter(int nv, int np, int ld, const int32_t *flist, const R *lim_out, R *u, Ctl *ctl, int grid, cudaStream_t st);

}  // namespace csw
