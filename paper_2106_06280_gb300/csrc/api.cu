// api.cu -- the C interface (include/cswdg.h): solver object, mesh upload
// (connectivity, periodic pairing, Morton locality order, geometry), device
// memory, the SSP-RK3 step as a captured CUDA graph, and read-back.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/cswdg.h"
#include "kernels.h"
#include "mesh_host.cuh"
#include "rules.cuh"
#include "tables.cuh"

using namespace csw;

struct cswdg_solver {
    cswdg_config cfg{};
    int nv = 1, np = 3, k = 1, eq = 0, fp32 = 0, w32 = 0;
    cudaStream_t stream = nullptr;
    int device = -1;  // the device that holds the solver's memory (current at mesh upload)
    std::string err;
    BcTab bc{};
    bool mesh_ready = false;
    // the state changed outside a step: ctl->lam_bits does not hold its maximum wave speed
    bool lam_stale = true;
    int nc = 0, ldc = 0, nbfaces = 0;
    double rmin = 0.0;
    std::vector<int32_t> perm;     // internal -> user
    std::vector<int32_t> iperm;    // user -> internal
    std::vector<double> vtx_user;  // 6 per user cell (for IC points)
    // device
    void *U = nullptr, *A = nullptr, *B = nullptr;  // state arrays
    void *geo = nullptr;
    int32_t *nbr = nullptr;
    uint8_t *nbf = nullptr;
    BFace *bf = nullptr;
    BcTab *bcd = nullptr;
    int32_t *dperm = nullptr;
    double *sc = nullptr, *area = nullptr;
    double *isc = nullptr;  // 1 / sc: the scaling of adjoint (dual) vectors
    void *ops = nullptr;
    uint8_t *flags = nullptr, *flags_user = nullptr;
    int32_t *flist = nullptr;
    void *lim_out = nullptr;
    void *kx = nullptr;  // KXRCF precursors written by the stage kernels of a step
    Ctl *ctl = nullptr;
    double *dev_user = nullptr, *cons_part = nullptr, *cons_out = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int lim_grid = 1;   // reconstruction kernel: blocks of 128 threads
    int scat_grid = 1;  // write-back kernel: blocks of 256 threads
    StageShape shape;   // stage kernel launch shape (cswdg_autotune)
};

namespace {

cswdg_status fail(cswdg_solver *s, cswdg_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    return st;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(s, CSWDG_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <typename T> cudaError_t dalloc(T **p, size_t n)
{
    return cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
}

bool tables_ready = false;

template <typename R> MeshDev<R> mesh_dev(const cswdg_solver *s)
{
    MeshDev<R> M;
    M.nc = s->nc;
    M.ldc = s->ldc;
    M.geo = (const R *)s->geo;
    M.nbr = s->nbr;
    M.nbf = s->nbf;
    M.bf = s->bf;
    M.bc = s->bcd;
    M.gamma = s->cfg.gamma;
    M.gammar = (R)s->cfg.gamma;
    return M;
}

void free_device(cswdg_solver *s)
{
    for (int i = 0; i < 2; ++i)
        if (s->graph[i]) { cudaGraphExecDestroy(s->graph[i]); s->graph[i] = nullptr; }
    void *ptrs[] = {s->U, s->A, s->B, s->geo, s->nbr, s->nbf, s->bf, s->bcd, s->dperm, s->sc, s->isc, s->area, s->ops, s->flags,
                    s->flags_user, s->flist, s->lim_out, s->kx, s->ctl, s->dev_user, s->cons_part, s->cons_out};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    s->U = s->A = s->B = s->geo = s->ops = s->lim_out = s->kx = nullptr;
    s->nbr = s->flist = s->dperm = nullptr;
    s->nbf = s->flags = s->flags_user = nullptr;
    s->bf = nullptr;
    s->bcd = nullptr;
    s->sc = s->isc = s->area = s->dev_user = s->cons_part = s->cons_out = nullptr;
    s->ctl = nullptr;
    s->mesh_ready = false;
}

// ---------------------------------------------------------------------------
// launch sequences.  `prof` (nullable) collects one event after every kernel
// launch, tagged with its kernel class, for cswdg_profile_step.
// ---------------------------------------------------------------------------
enum { KC_CFL = 0, KC_STAGE = 1, KC_DETECT = 2, KC_LIMIT = 3, KC_SCATTER = 4, KC_COUNT = 5 };
struct Prof {
    std::vector<std::pair<int, cudaEvent_t>> ev;
};

void mark(Prof *prof, int cls, cudaStream_t st)
{
    if (!prof) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, st);
    prof->ev.push_back({cls, e});
}

// after_stage: the stage kernel just before has reset the flagged count
cswdg_status limiter_pass(cswdg_solver *s, void *u, double tfac, cudaStream_t st, Prof *prof = nullptr, bool force_all = false,
                          bool after_stage = false)
{
    if (s->cfg.limiter == CSWDG_LIMITER_OFF) return CSWDG_OK;
    const int all = (s->cfg.limiter == CSWDG_LIMITER_ALL) || force_all;
    if (!after_stage) CK(cudaMemsetAsync(&s->ctl->nflag, 0, sizeof(int32_t), st));
    if (s->fp32) {
        MeshDev<float> M = mesh_dev<float>(s);
        if (after_stage)
            launch_detect_kx<float>(s->eq, s->k, M, (const float *)u, (const float *)s->kx, s->ctl, tfac, s->cfg.c_k, all, s->flags,
                                    s->flist, st);
        else
            launch_detect<float>(s->eq, s->k, M, (const float *)u, s->ctl, tfac, s->cfg.c_k, all, s->flags, s->flist, st);
        mark(prof, KC_DETECT, st);
        launch_limit<float>(s->eq, s->k, M, (const float *)u, (const float *)s->ops, s->flist, s->ctl, tfac, (float *)s->lim_out,
                            s->lim_grid, s->w32, st);
        mark(prof, KC_LIMIT, st);
        launch_scatter<float>(s->nv, s->np, s->ldc, s->flist, (const float *)s->lim_out, (float *)u, s->ctl, s->scat_grid, st);
        mark(prof, KC_SCATTER, st);
    } else {
        MeshDev<double> M = mesh_dev<double>(s);
        if (after_stage)
            launch_detect_kx<double>(s->eq, s->k, M, (const double *)u, (const double *)s->kx, s->ctl, tfac, s->cfg.c_k, all,
                                     s->flags, s->flist, st);
        else
            launch_detect<double>(s->eq, s->k, M, (const double *)u, s->ctl, tfac, s->cfg.c_k, all, s->flags, s->flist, st);
        mark(prof, KC_DETECT, st);
        launch_limit<double>(s->eq, s->k, M, (const double *)u, (const double *)s->ops, s->flist, s->ctl, tfac,
                             (double *)s->lim_out, s->lim_grid, 0, st);
        mark(prof, KC_LIMIT, st);
        launch_scatter<double>(s->nv, s->np, s->ldc, s->flist, (const double *)s->lim_out, (double *)u, s->ctl, s->scat_grid, st);
        mark(prof, KC_SCATTER, st);
    }
    CK(cudaGetLastError());
    return CSWDG_OK;
}

cswdg_status stage(cswdg_solver *s, const void *un, const void *up, void *out, double a, double b, double cl, double tfac,
                   cudaStream_t st, Prof *prof = nullptr, int lam_next = 0, bool write_kx = false)
{
    if (s->fp32) {
        // a convex combination keeps coefficients that sum to one after rounding
        // (1/3 and 2/3 rounded separately to float sum to 1 + 3e-8: a drift of the means)
        const float bf = (float)b, af = (std::fabs(a + b - 1.0) < 1e-12) ? 1.0f - bf : (float)a;
        launch_stage<float>(s->eq, s->k, mesh_dev<float>(s), (const float *)un, (const float *)up, (float *)out, af, bf,
                            (float)cl, tfac, lam_next, write_kx ? (float *)s->kx : nullptr, s->ctl, s->shape, st);
    } else {
        launch_stage<double>(s->eq, s->k, mesh_dev<double>(s), (const double *)un, (const double *)up, (double *)out, a, b, cl, tfac,
                             lam_next, write_kx ? (double *)s->kx : nullptr, s->ctl, s->shape, st);
    }
    mark(prof, KC_STAGE, st);
    CK(cudaGetLastError());
    return CSWDG_OK;
}

// One SSP-RK3 step (Table tvd): stage i evaluates L_h at t + (0, dt, dt/2)
// and the limiter after it sees t + (dt, dt/2, dt).
// The CFL rule of a step uses the maximum wave speed that the last stage of
// the previous step folded into ctl->lam_bits (refresh_lam computes it when the
// state was set from outside).
cswdg_status record_step(cswdg_solver *s, int use_cfl, cudaStream_t st, Prof *prof = nullptr)
{
    cswdg_status r;
    launch_begin_step(s->ctl, use_cfl, st);
    mark(prof, KC_CFL, st);
    CK(cudaGetLastError());
    const bool kx = s->cfg.limiter != CSWDG_LIMITER_OFF;
    if ((r = stage(s, nullptr, s->U, s->A, 0.0, 1.0, 1.0, 0.0, st, prof, 0, kx))) return r;
    if ((r = limiter_pass(s, s->A, 1.0, st, prof, false, true))) return r;
    if ((r = stage(s, s->U, s->A, s->B, 0.75, 0.25, 0.25, 1.0, st, prof, 0, kx))) return r;
    if ((r = limiter_pass(s, s->B, 0.5, st, prof, false, true))) return r;
    if ((r = stage(s, s->U, s->B, s->U, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, 0.5, st, prof, 1, kx))) return r;
    if ((r = limiter_pass(s, s->U, 1.0, st, prof, false, true))) return r;
    return CSWDG_OK;
}

cswdg_status read_ctl(cswdg_solver *s, Ctl *h);
cswdg_status write_ctl(cswdg_solver *s, const Ctl *hin);

// maximum wave speed of the current state into ctl->lam_bits (host copy h is
// updated and written); one launch, counted in *nl
cswdg_status refresh_lam(cswdg_solver *s, Ctl *h, int64_t *nl)
{
    h->lam_bits = 0ull;
    if (cswdg_status r = write_ctl(s, h)) return r;
    if (s->fp32) launch_cfl<float>(s->eq, mesh_dev<float>(s), s->np, (const float *)s->U, s->ctl, s->stream);
    else launch_cfl<double>(s->eq, mesh_dev<double>(s), s->np, (const double *)s->U, s->ctl, s->stream);
    CK(cudaGetLastError());
    if (nl) ++*nl;
    s->lam_stale = false;
    return read_ctl(s, h);
}

cswdg_status get_graph(cswdg_solver *s, int use_cfl)
{
    if (s->graph[use_cfl]) return CSWDG_OK;
    cudaStream_t cap;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cap);
        return fail(s, CSWDG_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    cswdg_status r = record_step(s, use_cfl, cap);
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (r) { if (g) cudaGraphDestroy(g); return r; }
    if (e != cudaSuccess) return fail(s, CSWDG_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&s->graph[use_cfl], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(s, CSWDG_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return CSWDG_OK;
}

cswdg_status read_ctl(cswdg_solver *s, Ctl *h)
{
    CK(cudaMemcpyAsync(h, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return CSWDG_OK;
}

cswdg_status write_ctl(cswdg_solver *s, const Ctl *hin)
{
    static thread_local Ctl h;
    h = *hin;
    h.dtf = (float)h.dt;
    CK(cudaMemcpyAsync(s->ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return CSWDG_OK;
}

cswdg_status check_err(cswdg_solver *s, Ctl *h)
{
    if (h->err & ERR_NONPHYS) {
        Ctl c = *h;
        c.err = 0;
        write_ctl(s, &c);
        return fail(s, CSWDG_ENONPHYS, "non-physical cell mean (rho <= 0, p <= 0 or NaN)");
    }
    if (h->err & ERR_TIMEOUT) {
        Ctl c = *h;
        c.err = 0;
        write_ctl(s, &c);
        return fail(s, CSWDG_ETIMEOUT, "bounded device wait expired");
    }
    return CSWDG_OK;
}

// user modes (physically orthonormal basis, user cell order) -> internal array;
// dual vectors (adjoint variables, gradients) pass dual = true: they scale
// with the inverse factor so that dot products are preserved
cswdg_status upload_modes(cswdg_solver *s, const double *modes, void *dst, bool dual = false)
{
    const size_t n = (size_t)s->nc * s->nv * s->np;
    const double *sc = dual ? s->isc : s->sc;
    CK(cudaMemcpyAsync(s->dev_user, modes, n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    if (s->fp32) launch_from_user<float>(s->nc, s->ldc, s->nv, s->np, s->dperm, sc, s->dev_user, (float *)dst, s->stream);
    else launch_from_user<double>(s->nc, s->ldc, s->nv, s->np, s->dperm, sc, s->dev_user, (double *)dst, s->stream);
    CK(cudaGetLastError());
    return CSWDG_OK;
}

cswdg_status download_modes(cswdg_solver *s, const void *src, double *modes, bool dual = false)
{
    const size_t n = (size_t)s->nc * s->nv * s->np;
    const double *sc = dual ? s->isc : s->sc;
    if (s->fp32) launch_to_user<float>(s->nc, s->ldc, s->nv, s->np, s->dperm, sc, (const float *)src, s->dev_user, s->stream);
    else launch_to_user<double>(s->nc, s->ldc, s->nv, s->np, s->dperm, sc, (const double *)src, s->dev_user, s->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(modes, s->dev_user, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return CSWDG_OK;
}

}  // namespace

namespace csw {
bool solver_view(const cswdg_solver *s, int *nc, int *ldc, int *nvar, int *np, int *fp32, const double **area, void **stream,
                 int *device)
{
    if (!s || !s->mesh_ready) return false;
    *device = s->device;
    *nc = s->nc;
    *ldc = s->ldc;
    *nvar = s->nv;
    *np = s->np;
    *fp32 = s->fp32;
    *area = s->area;
    *stream = (void *)s->stream;
    return true;
}

cswdg_status solver_fail(cswdg_solver *s, cswdg_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    return st;
}
}  // namespace csw

// ===========================================================================
// C interface
// ===========================================================================
extern "C" {

cswdg_status cswdg_create(const cswdg_config *cfg, cswdg_solver **out)
{
    if (!cfg || !out) return CSWDG_EINVAL;
    *out = nullptr;
    if ((cfg->equation != CSWDG_BURGERS && cfg->equation != CSWDG_EULER) || (cfg->degree != 1 && cfg->degree != 2) ||
        (cfg->precision != CSWDG_FP64 && cfg->precision != CSWDG_FP32_BULK && cfg->precision != CSWDG_FP32) || cfg->limiter < 0 || cfg->limiter > 2 ||
        !(cfg->gamma > 1.0))
        return CSWDG_EINVAL;
    cswdg_solver *s = new (std::nothrow) cswdg_solver();
    if (!s) return CSWDG_ENOMEM;
    s->cfg = *cfg;
    s->eq = cfg->equation;
    s->k = cfg->degree;
    s->nv = (s->eq == CSWDG_EULER) ? 4 : 1;
    s->np = (s->k + 1) * (s->k + 2) / 2;
    s->fp32 = (cfg->precision != CSWDG_FP64);
    s->w32 = (cfg->precision == CSWDG_FP32);
    s->stream = (cudaStream_t)cfg->stream;
    for (int t = 0; t < CSW_MAXTAG; ++t) s->bc.kind[t] = -1;
    if (!tables_ready) {
        cudaError_t e = operator_upload_tables();
        if (e == cudaSuccess) e = limiter_upload_tables();
        if (e == cudaSuccess) e = adjoint_upload_tables();
        if (e != cudaSuccess) {
            delete s;
            return CSWDG_ECUDA;
        }
        tables_ready = true;
    }
    *out = s;
    return CSWDG_OK;
}

void cswdg_destroy(cswdg_solver *s)
{
    if (!s) return;
    free_device(s);
    delete s;
}

const char *cswdg_last_error(const cswdg_solver *s)
{
    if (!s) return "null solver";
    return s->err.c_str();
}

cswdg_status cswdg_set_boundary(cswdg_solver *s, int32_t tag, int32_t kind, const double *params, int32_t nparams)
{
    if (!s) return CSWDG_EINVAL;
    if (tag < 0 || tag >= CSW_MAXTAG || kind < 0 || kind > CSWDG_BC_SHOCKLINE || nparams < 0 || nparams > CSW_MAXPAR ||
        (nparams > 0 && !params))
        return fail(s, CSWDG_EINVAL, "bad boundary tag/kind/params");
    const int need = (kind == CSWDG_BC_DIRICHLET) ? s->nv : (kind == CSWDG_BC_SHOCKLINE) ? 3 + 2 * s->nv : 0;
    if (nparams < need) return fail(s, CSWDG_EINVAL, "boundary kind %d needs %d parameters", kind, need);
    s->bc.kind[tag] = kind;
    for (int i = 0; i < CSW_MAXPAR; ++i) s->bc.par[tag][i] = (i < nparams) ? params[i] : 0.0;
    return CSWDG_OK;
}

cswdg_status cswdg_mesh_upload(cswdg_solver *s, int64_t nv, const double *xy, int64_t nc64, const int32_t *tri, int64_t nbf,
                               const int32_t *bface, const double *period)
{
    if (!s || !xy || !tri || nv < 3 || nc64 < 1 || nc64 > (1 << 30) || nbf < 0 || (nbf > 0 && !bface))
        return fail(s, CSWDG_EINVAL, "bad mesh arguments");
    free_device(s);
    HostMesh H;
    if (int st = build_host_mesh(s->k, s->bc.kind, nv, xy, nc64, tri, nbf, bface, period, H))
        return fail(s, (cswdg_status)st, "%s", H.msg.c_str());
    const int nc = H.nc;
    s->nc = nc;
    s->ldc = H.ldc;
    s->perm = H.perm;
    s->iperm = H.iperm;
    s->vtx_user = H.vtx_user;
    s->rmin = H.rmin;
    s->nbfaces = (int)H.bfs.size();
    const int ld = s->ldc;
    const double rmin = H.rmin;
    std::vector<double> &geo = H.geo, &scv = H.scv, &arv = H.arv, &vtx = H.vtx, &nvtx = H.nvtx;
    std::vector<int32_t> &nbr = H.nbr;
    std::vector<uint8_t> &nbfv = H.nbfv;
    std::vector<BFace> &bfs = H.bfs;
    // ---- device buffers ----
    const size_t rs = s->fp32 ? 4 : 8;
    const size_t nstate = (size_t)s->nv * s->np * ld;
    cudaError_t e = cudaSuccess;
    auto A_ = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A_(cudaGetDevice(&s->device));
    A_(stage_kernels_prepare());
    A_(cudaMalloc(&s->U, nstate * rs));
    A_(cudaMalloc(&s->A, nstate * rs));
    A_(cudaMalloc(&s->B, nstate * rs));
    A_(cudaMalloc(&s->geo, (size_t)G_COUNT * ld * rs));
    A_(dalloc(&s->nbr, (size_t)3 * ld));
    A_(dalloc(&s->nbf, (size_t)ld));
    A_(dalloc(&s->bf, bfs.size()));
    A_(dalloc(&s->bcd, 1));
    A_(dalloc(&s->dperm, (size_t)ld));
    A_(dalloc(&s->sc, (size_t)ld));
    A_(dalloc(&s->isc, (size_t)ld));
    A_(dalloc(&s->area, (size_t)ld));
    A_(dalloc(&s->flags, (size_t)ld));
    A_(dalloc(&s->flags_user, (size_t)ld));
    A_(dalloc(&s->flist, (size_t)ld));
    A_(cudaMalloc(&s->lim_out, (size_t)nc * s->nv * (s->np - 1) * rs));
    A_(cudaMalloc(&s->kx, (size_t)ld * KX_STRIDE * rs));
    A_(dalloc(&s->ctl, 1));
    A_(dalloc(&s->dev_user, std::max((size_t)nc * s->nv * s->np, (size_t)nc * 7 * s->nv)));
    A_(dalloc(&s->cons_part, (size_t)s->nv * ((nc + 255) / 256)));
    A_(dalloc(&s->cons_out, 4));
    if (e != cudaSuccess) { free_device(s); return fail(s, CSWDG_ENOMEM, "device allocation: %s", cudaGetErrorString(e)); }
    cudaStream_t st = s->stream;
    if (s->fp32) {
        std::vector<float> g32(geo.begin(), geo.end());
        CK(cudaMemcpyAsync(s->geo, g32.data(), g32.size() * 4, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    } else {
        CK(cudaMemcpyAsync(s->geo, geo.data(), geo.size() * 8, cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemcpyAsync(s->nbr, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s->nbf, nbfv.data(), nbfv.size(), cudaMemcpyHostToDevice, st));
    if (!bfs.empty()) CK(cudaMemcpyAsync(s->bf, bfs.data(), bfs.size() * sizeof(BFace), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s->bcd, &s->bc, sizeof(BcTab), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s->dperm, s->perm.data(), (size_t)nc * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s->sc, scv.data(), (size_t)ld * 8, cudaMemcpyHostToDevice, st));
    std::vector<double> iscv(ld);
    for (int i = 0; i < ld; ++i) iscv[i] = (scv[i] != 0.0) ? 1.0 / scv[i] : 0.0;
    CK(cudaMemcpyAsync(s->isc, iscv.data(), (size_t)ld * 8, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemcpyAsync(s->area, arv.data(), (size_t)ld * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(s->U, 0, nstate * rs, st));
    s->lam_stale = true;
    CK(cudaMemsetAsync(s->A, 0, nstate * rs, st));
    CK(cudaMemsetAsync(s->B, 0, nstate * rs, st));
    CK(cudaMemsetAsync(s->flags, 0, ld, st));
    Ctl h{};
    h.rmin = rmin;
    h.cfl = s->cfg.cfl;
    h.active = 1;
    CK(cudaMemcpyAsync(s->ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    // ---- per-cell CSWENO operators (set-up kernel, FP64) ----
    if (s->cfg.limiter != CSWDG_LIMITER_OFF) {
        const int osz = (s->k == 1) ? Ops<1>::SIZE : Ops<2>::SIZE;
        double *dops = nullptr, *dvtx = nullptr, *dnvtx = nullptr;
        e = cudaSuccess;
        A_(cudaMalloc((void **)&dops, (size_t)nc * osz * 8));
        A_(cudaMalloc((void **)&dvtx, vtx.size() * 8));
        A_(cudaMalloc((void **)&dnvtx, nvtx.size() * 8));
        if (e != cudaSuccess) {
            cudaFree(dops); cudaFree(dvtx); cudaFree(dnvtx);
            free_device(s);
            return fail(s, CSWDG_ENOMEM, "device allocation (stencil operators): %s", cudaGetErrorString(e));
        }
        CK(cudaMemsetAsync(dops, 0, (size_t)nc * osz * 8, st));  // padding words included
        CK(cudaMemcpyAsync(dvtx, vtx.data(), vtx.size() * 8, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(dnvtx, nvtx.data(), nvtx.size() * 8, cudaMemcpyHostToDevice, st));
        // the set-up kernel keeps its QR and Cholesky work arrays on the thread stack
        size_t stack = 0;
        CK(cudaDeviceGetLimit(&stack, cudaLimitStackSize));
        if (stack < 16384) CK(cudaDeviceSetLimit(cudaLimitStackSize, 16384));
        launch_setup_ops(s->k, nc, ld, dvtx, dnvtx, s->nbr, s->nbf, dops, &s->ctl->err, st);
        CK(cudaGetLastError());
        if (s->fp32) {
            CK(cudaMalloc(&s->ops, (size_t)nc * osz * 4));
            launch_ops_to_float((size_t)nc * osz, dops, (float *)s->ops, st);
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(st));
            cudaFree(dops);
        } else {
            s->ops = dops;
        }
        CK(cudaStreamSynchronize(st));
        cudaFree(dvtx);
        cudaFree(dnvtx);
        Ctl hc;
        if (cswdg_status r = read_ctl(s, &hc)) return r;
        if (hc.err & ERR_LSQ) { free_device(s); return fail(s, CSWDG_ELSQ, "rank-deficient stencil least squares"); }
    }
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    s->lim_grid = std::max(1, std::min((nc * (s->eq == CSWDG_EULER ? 8 : 1) + 127) / 128, nsm * 16));
    s->scat_grid = std::max(1, std::min((int)(((long long)nc * s->nv * (s->np - 1) + 255) / 256), nsm * 4));
    s->mesh_ready = true;
    return CSWDG_OK;
}

int32_t cswdg_num_ic_points(const cswdg_solver *s)
{
    if (!s) return 0;
    return (s->k == 1) ? Deg<1>::QV : Deg<2>::QV;
}

cswdg_status cswdg_ic_points(cswdg_solver *s, double *xy_host)
{
    if (!s || !s->mesh_ready || !xy_host) return fail(s, CSWDG_EINVAL, "ic_points: no mesh or null output");
    TriRule R;
    if (s->k == 1) volume_rule<1>(R);
    else volume_rule<2>(R);
    for (int c = 0; c < s->nc; ++c) {
        const double *v = &s->vtx_user[6 * (size_t)c];
        for (int q = 0; q < R.n; ++q) {
            xy_host[2 * ((size_t)c * R.n + q)] = R.b[q][0] * v[0] + R.b[q][1] * v[2] + R.b[q][2] * v[4];
            xy_host[2 * ((size_t)c * R.n + q) + 1] = R.b[q][0] * v[1] + R.b[q][1] * v[3] + R.b[q][2] * v[5];
        }
    }
    return CSWDG_OK;
}

cswdg_status cswdg_project_ic(cswdg_solver *s, const double *values, int32_t apply_limiter)
{
    if (!s || !s->mesh_ready || !values) return fail(s, CSWDG_EINVAL, "project_ic: no mesh or null input");
    const int Q = cswdg_num_ic_points(s);
    // values are in user cell order: gather into internal order on the host side of the copy
    std::vector<double> vals((size_t)s->nc * Q * s->nv);
    for (int i = 0; i < s->nc; ++i)
        memcpy(&vals[(size_t)i * Q * s->nv], &values[(size_t)s->perm[i] * Q * s->nv], sizeof(double) * Q * s->nv);
    CK(cudaMemcpyAsync(s->dev_user, vals.data(), vals.size() * 8, cudaMemcpyHostToDevice, s->stream));
    if (s->fp32) launch_project<float>(s->k, s->nc, s->ldc, s->nv, s->dev_user, (float *)s->U, s->stream);
    else launch_project<double>(s->k, s->nc, s->ldc, s->nv, s->dev_user, (double *)s->U, s->stream);
    s->lam_stale = true;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->stream));
    if (apply_limiter && s->cfg.limiter != CSWDG_LIMITER_OFF) {
        Ctl h;
        if (cswdg_status r = read_ctl(s, &h)) return r;
        Ctl w = h;
        w.dt = 0.0;
        w.active = 1;
        if (cswdg_status r = write_ctl(s, &w)) return r;
        if (cswdg_status r = limiter_pass(s, s->U, 0.0, s->stream, nullptr, apply_limiter == 2)) return r;
        Ctl after;
        if (cswdg_status r = read_ctl(s, &after)) return r;
        h.nflag = after.nflag;
        h.err = after.err;
        if (cswdg_status r = write_ctl(s, &h)) return r;
        if (cswdg_status r = check_err(s, &h)) return r;
    }
    return CSWDG_OK;
}

cswdg_status cswdg_step(cswdg_solver *s, double dt, int64_t nsteps, double t_end, double *t_out)
{
    if (!s || !s->mesh_ready || nsteps < 0) return fail(s, CSWDG_EINVAL, "step: no mesh or negative nsteps");
    const int use_cfl = !(dt > 0.0);
    // everything up to the final read of the control block is queued on the
    // stream: the step parameters, the CFL maximum of a state set from outside
    // (lam_bits cleared first), the step graphs; one host round trip per call
    launch_set_step_params(s->ctl, dt, s->cfg.cfl, t_end, s->stream);
    CK(cudaGetLastError());
    if (use_cfl && s->lam_stale) {
        CK(cudaMemsetAsync(&s->ctl->lam_bits, 0, sizeof(unsigned long long), s->stream));
        if (s->fp32) launch_cfl<float>(s->eq, mesh_dev<float>(s), s->np, (const float *)s->U, s->ctl, s->stream);
        else launch_cfl<double>(s->eq, mesh_dev<double>(s), s->np, (const double *)s->U, s->ctl, s->stream);
        CK(cudaGetLastError());
        s->lam_stale = false;
    }
    if (cswdg_status r = get_graph(s, use_cfl)) return r;
    // long runs towards a finite t_end: launch in chunks and stop once the device time
    // has reached t_end (steps past t_end do nothing, but each still launches)
    constexpr int64_t kChunk = 256;
    Ctl h;
    int64_t done = 0;
    while (done < nsteps) {
        const int64_t n = (t_end < 1e299 && nsteps - done > kChunk) ? kChunk : nsteps - done;
        for (int64_t i = 0; i < n; ++i) CK(cudaGraphLaunch(s->graph[use_cfl], s->stream));
        done += n;
        if (done < nsteps) {
            if (cswdg_status r = read_ctl(s, &h)) return r;
            if (h.err || !(h.t_next < t_end)) break;
        }
    }
    if (cswdg_status r = read_ctl(s, &h)) return r;
    h.t = h.t_next;
    if (t_out) *t_out = h.t_next;
    return check_err(s, &h);
}

cswdg_status cswdg_selftest_timeout(cswdg_solver *s, int32_t polls)
{
    if (!s || !s->mesh_ready || polls < 1 || polls > (1 << 22)) return fail(s, CSWDG_EINVAL, "selftest_timeout: no mesh or bad poll count");
    launch_selftest_timeout(s->ctl, polls, s->stream);
    CK(cudaGetLastError());
    Ctl h;
    if (cswdg_status r = read_ctl(s, &h)) return r;
    return check_err(s, &h);  // reports ETIMEOUT and clears the bit
}

cswdg_status cswdg_profile_step(cswdg_solver *s, double dt, int64_t nsteps, double t_end, double *ms_host, int64_t *launches_host)
{
    if (!s || !s->mesh_ready || nsteps < 0 || !ms_host) return fail(s, CSWDG_EINVAL, "profile_step");
    const int use_cfl = !(dt > 0.0);
    Ctl h;
    if (cswdg_status r = read_ctl(s, &h)) return r;
    h.dt_fixed = dt;
    h.cfl = s->cfg.cfl;
    h.t_end = t_end;
    int64_t nl = 0;
    if (use_cfl && s->lam_stale)
        if (cswdg_status r = refresh_lam(s, &h, &nl)) return r;
    if (cswdg_status r = write_ctl(s, &h)) return r;
    for (int i = 0; i < KC_COUNT; ++i) ms_host[i] = 0.0;
    for (int64_t it = 0; it < nsteps; ++it) {
        Prof prof;
        mark(&prof, -1, s->stream);
        if (cswdg_status r = record_step(s, use_cfl, s->stream, &prof)) return r;
        CK(cudaStreamSynchronize(s->stream));
        for (size_t i = 1; i < prof.ev.size(); ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, prof.ev[i - 1].second, prof.ev[i].second);
            ms_host[prof.ev[i].first] += ms;
        }
        nl += (int64_t)prof.ev.size() - 1;
        for (auto &e : prof.ev) cudaEventDestroy(e.second);
    }
    if (launches_host) *launches_host = nl;
    if (cswdg_status r = read_ctl(s, &h)) return r;
    return check_err(s, &h);
}

int32_t cswdg_launches_per_step(const cswdg_solver *s, int32_t use_cfl)
{
    if (!s) return 0;
    const int lim = (s->cfg.limiter != CSWDG_LIMITER_OFF) ? 3 : 0;
    (void)use_cfl;  // the CFL maximum is folded into the last stage
    return 1 + 3 * (1 + lim);
}

cswdg_status cswdg_get_time(cswdg_solver *s, double *t)
{
    if (!s || !s->mesh_ready || !t) return fail(s, CSWDG_EINVAL, "get_time");
    Ctl h;
    if (cswdg_status r = read_ctl(s, &h)) return r;
    *t = h.t_next;
    return CSWDG_OK;
}

cswdg_status cswdg_set_time(cswdg_solver *s, double t)
{
    if (!s || !s->mesh_ready) return fail(s, CSWDG_EINVAL, "set_time");
    Ctl h;
    if (cswdg_status r = read_ctl(s, &h)) return r;
    h.t = h.t_next = t;
    return write_ctl(s, &h);
}

cswdg_status cswdg_read_modes(cswdg_solver *s, double *modes)
{
    if (!s || !s->mesh_ready || !modes) return fail(s, CSWDG_EINVAL, "read_modes");
    return download_modes(s, s->U, modes);
}

cswdg_status cswdg_write_modes(cswdg_solver *s, const double *modes)
{
    if (!s || !s->mesh_ready || !modes) return fail(s, CSWDG_EINVAL, "write_modes");
    if (cswdg_status r = upload_modes(s, modes, s->U)) return r;
    s->lam_stale = true;
    CK(cudaStreamSynchronize(s->stream));
    return CSWDG_OK;
}

cswdg_status cswdg_read_modes_f32(cswdg_solver *s, float *modes)
{
    if (!s || !s->mesh_ready || !modes) return fail(s, CSWDG_EINVAL, "read_modes_f32");
    const size_t n = (size_t)s->nc * s->nv * s->np;
    float *stage = reinterpret_cast<float *>(s->dev_user);  // n floats fit the n-double staging buffer
    if (s->fp32) launch_to_user<float, float>(s->nc, s->ldc, s->nv, s->np, s->dperm, s->sc, (const float *)s->U, stage, s->stream);
    else launch_to_user<double, float>(s->nc, s->ldc, s->nv, s->np, s->dperm, s->sc, (const double *)s->U, stage, s->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(modes, stage, n * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return CSWDG_OK;
}

cswdg_status cswdg_write_modes_f32(cswdg_solver *s, const float *modes)
{
    if (!s || !s->mesh_ready || !modes) return fail(s, CSWDG_EINVAL, "write_modes_f32");
    const size_t n = (size_t)s->nc * s->nv * s->np;
    float *stage = reinterpret_cast<float *>(s->dev_user);
    CK(cudaMemcpyAsync(stage, modes, n * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    if (s->fp32) launch_from_user<float, float>(s->nc, s->ldc, s->nv, s->np, s->dperm, s->sc, stage, (float *)s->U, s->stream);
    else launch_from_user<double, float>(s->nc, s->ldc, s->nv, s->np, s->dperm, s->sc, stage, (double *)s->U, s->stream);
    CK(cudaGetLastError());
    s->lam_stale = true;
    CK(cudaStreamSynchronize(s->stream));
    return CSWDG_OK;
}

cswdg_status cswdg_read_flags(cswdg_solver *s, uint8_t *flags)
{
    if (!s || !s->mesh_ready || !flags) return fail(s, CSWDG_EINVAL, "read_flags");
    launch_flags_to_user(s->nc, s->dperm, s->flags, s->flags_user, s->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(flags, s->flags_user, s->nc, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return CSWDG_OK;
}

cswdg_status cswdg_num_flagged(cswdg_solver *s, int64_t *n)
{
    if (!s || !s->mesh_ready || !n) return fail(s, CSWDG_EINVAL, "num_flagged");
    Ctl h;
    if (cswdg_status r = read_ctl(s, &h)) return r;
    *n = h.nflag;
    return CSWDG_OK;
}

cswdg_status cswdg_conservation(cswdg_solver *s, double *sums)
{
    if (!s || !s->mesh_ready || !sums) return fail(s, CSWDG_EINVAL, "conservation");
    if (s->fp32) launch_conservation<float>(s->nc, s->ldc, s->nv, s->np, s->area, (const float *)s->U, s->cons_part, s->cons_out, s->stream);
    else launch_conservation<double>(s->nc, s->ldc, s->nv, s->np, s->area, (const double *)s->U, s->cons_part, s->cons_out, s->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(sums, s->cons_out, s->nv * 8, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return CSWDG_OK;
}

cswdg_status cswdg_eval_rhs(cswdg_solver *s, double t, const double *modes_in, double *rhs)
{
    if (!s || !s->mesh_ready || !modes_in || !rhs) return fail(s, CSWDG_EINVAL, "eval_rhs");
    Ctl h;
    if (cswdg_status r = read_ctl(s, &h)) return r;
    Ctl w = h;
    w.t = t;
    w.dt = 1.0;
    w.active = 1;
    if (cswdg_status r = write_ctl(s, &w)) return r;
    if (cswdg_status r = upload_modes(s, modes_in, s->U)) return r;
    s->lam_stale = true;
    if (cswdg_status r = stage(s, nullptr, s->U, s->A, 0.0, 0.0, 1.0, 0.0, s->stream)) return r;
    if (cswdg_status r = download_modes(s, s->A, rhs)) return r;
    return write_ctl(s, &h);
}

cswdg_status cswdg_limit(cswdg_solver *s, double t, const double *modes_in, double *modes_out, uint8_t *flags)
{
    if (!s || !s->mesh_ready || !modes_in) return fail(s, CSWDG_EINVAL, "limit");
    Ctl h;
    if (cswdg_status r = read_ctl(s, &h)) return r;
    Ctl w = h;
    w.t = t;
    w.dt = 0.0;
    w.active = 1;
    w.err = 0;
    if (cswdg_status r = write_ctl(s, &w)) return r;
    if (cswdg_status r = upload_modes(s, modes_in, s->U)) return r;
    s->lam_stale = true;
    if (s->cfg.limiter == CSWDG_LIMITER_OFF) CK(cudaMemsetAsync(s->flags, 0, s->ldc, s->stream));
    if (cswdg_status r = limiter_pass(s, s->U, 0.0, s->stream)) return r;
    if (modes_out)
        if (cswdg_status r = download_modes(s, s->U, modes_out)) return r;
    if (flags)
        if (cswdg_status r = cswdg_read_flags(s, flags)) return r;
    Ctl after;
    if (cswdg_status r = read_ctl(s, &after)) return r;
    h.nflag = after.nflag;
    h.err = after.err;
    if (cswdg_status r = write_ctl(s, &h)) return r;
    return check_err(s, &h);
}

cswdg_status cswdg_cfl_dt(cswdg_solver *s, double *dt)
{
    if (!s || !s->mesh_ready || !dt) return fail(s, CSWDG_EINVAL, "cfl_dt");
    Ctl h;
    if (cswdg_status r = read_ctl(s, &h)) return r;
    Ctl w = h;
    w.lam_bits = 0ull;
    if (cswdg_status r = write_ctl(s, &w)) return r;
    if (s->fp32) launch_cfl<float>(s->eq, mesh_dev<float>(s), s->np, (const float *)s->U, s->ctl, s->stream);
    else launch_cfl<double>(s->eq, mesh_dev<double>(s), s->np, (const double *)s->U, s->ctl, s->stream);
    CK(cudaGetLastError());
    Ctl after;
    if (cswdg_status r = read_ctl(s, &after)) return r;
    double lam;
    memcpy(&lam, &after.lam_bits, 8);
    *dt = (lam > 0.0) ? s->cfg.cfl * s->rmin / lam : 0.0;
    return write_ctl(s, &h);
}

cswdg_status cswdg_stage_dev(cswdg_solver *s, const void *un, const void *uprev, void *out, double a, double b, double dt, double t_rhs)
{
    if (!s || !s->mesh_ready || !uprev || !out || (a != 0.0 && !un)) return fail(s, CSWDG_EINVAL, "stage_dev");
    auto misaligned = [](const void *p) { return ((uintptr_t)p & 15u) != 0; };
    if (misaligned(uprev) || misaligned(out) || (a != 0.0 && misaligned(un)))
        return fail(s, CSWDG_EINVAL, "stage_dev: device pointers must be 16-byte aligned");
    Ctl h;
    if (cswdg_status r = read_ctl(s, &h)) return r;
    Ctl w = h;
    w.t = t_rhs;
    w.dt = dt;
    w.active = 1;
    if (cswdg_status r = write_ctl(s, &w)) return r;
    if (cswdg_status r = stage(s, a != 0.0 ? un : nullptr, uprev, out, a, b, b, 0.0, s->stream)) return r;
    CK(cudaStreamSynchronize(s->stream));
    return write_ctl(s, &h);
}

cswdg_status cswdg_stencil_operator(cswdg_solver *s, int64_t cell, double *out, int32_t *n)
{
    if (!s || !s->mesh_ready || cell < 0 || cell >= s->nc || !n) return fail(s, CSWDG_EINVAL, "stencil_operator");
    const int osz = (s->k == 1) ? Ops<1>::SIZE : Ops<2>::SIZE;
    *n = (s->cfg.limiter == CSWDG_LIMITER_OFF) ? 0 : osz;
    if (!out || *n == 0) return CSWDG_OK;
    const size_t off = (size_t)s->iperm[cell] * osz;
    if (s->fp32) {
        std::vector<float> tmp(osz);
        CK(cudaMemcpy(tmp.data(), (const float *)s->ops + off, osz * 4, cudaMemcpyDeviceToHost));
        for (int i = 0; i < osz; ++i) out[i] = tmp[i];
    } else {
        CK(cudaMemcpy(out, (const double *)s->ops + off, osz * 8, cudaMemcpyDeviceToHost));
    }
    return CSWDG_OK;
}

cswdg_status cswdg_internal_layout(cswdg_solver *s, int64_t *ldc, int32_t *perm)
{
    if (!s || !s->mesh_ready) return fail(s, CSWDG_EINVAL, "internal_layout");
    if (ldc) *ldc = s->ldc;
    if (perm)
        for (int c = 0; c < s->nc; ++c) perm[c] = s->iperm[c];
    return CSWDG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Launch-shape autotuner for the stage kernel: times each candidate on the
// current state (stage into the scratch array B, state untouched) and keeps
// the fastest.  The step graphs are re-captured with the chosen shape.
// ---------------------------------------------------------------------------
cswdg_status cswdg_autotune(cswdg_solver *s, double *ms_host, int32_t *chosen_host)
{
    if (!s || !s->mesh_ready) return fail(s, CSWDG_EINVAL, "autotune: no mesh");
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const StageShape cand[CSWDG_TUNE_CANDIDATES] = {{64, 0, 0},       {128, 0, 0},       {256, 0, 0},       {64, nsm * 8, 0},
                                                    {128, nsm * 4, 0}, {256, nsm * 2, 0}, {128, nsm * 8, 0}, {128, 0, 1},
                                                    {256, 0, 1},       {128, nsm * 4, 1}, {256, nsm * 2, 1}};
    Ctl h;
    if (cswdg_status r = read_ctl(s, &h)) return r;
    Ctl w = h;
    w.dt = 0.0;
    w.active = 1;
    if (cswdg_status r = write_ctl(s, &w)) return r;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = 1e300;
    int ib = 1;
    for (int i = 0; i < CSWDG_TUNE_CANDIDATES; ++i) {
        s->shape = cand[i];
        for (int it = 0; it < 2; ++it)
            if (cswdg_status r = stage(s, nullptr, s->U, s->B, 0.0, 1.0, 1.0, 0.0, s->stream)) return r;
        CK(cudaEventRecord(e0, s->stream));
        for (int it = 0; it < 5; ++it)
            if (cswdg_status r = stage(s, nullptr, s->U, s->B, 0.0, 1.0, 1.0, 0.0, s->stream)) return r;
        CK(cudaEventRecord(e1, s->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms_host) ms_host[i] = ms / 5.0;
        if (ms < best) { best = ms; ib = i; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->shape = cand[ib];
    for (int i = 0; i < 2; ++i)
        if (s->graph[i]) { cudaGraphExecDestroy(s->graph[i]); s->graph[i] = nullptr; }
    if (chosen_host) { chosen_host[0] = cand[ib].blk; chosen_host[1] = cand[ib].grid; chosen_host[2] = cand[ib].tile_faces; }
    return write_ctl(s, &h);
}

cswdg_status cswdg_set_stage_shape(cswdg_solver *s, int32_t cells_per_block, int32_t grid, int32_t tile_faces)
{
    if (!s || (cells_per_block != 64 && cells_per_block != 128 && cells_per_block != 256) || grid < 0 ||
        (tile_faces != 0 && tile_faces != 1) || (tile_faces == 1 && cells_per_block == 64))
        return fail(s, CSWDG_EINVAL,
                    "set_stage_shape: cells per block 64, 128 or 256 (128 or 256 with tile_faces); grid >= 0; tile_faces 0 or 1");
    s->shape.blk = cells_per_block;
    s->shape.grid = grid;
    s->shape.tile_faces = tile_faces;
    for (int i = 0; i < 2; ++i)
        if (s->graph[i]) { cudaGraphExecDestroy(s->graph[i]); s->graph[i] = nullptr; }
    return CSWDG_OK;
}

// ---------------------------------------------------------------------------
// Adjoint of the operator (host buffers in the user basis and cell order)
// ---------------------------------------------------------------------------
cswdg_status cswdg_rhs_adjoint(cswdg_solver *s, double t, const double *modes_in, const double *lambda_in, double *grad_out)
{
    if (!s || !s->mesh_ready || !modes_in || !lambda_in || !grad_out) return fail(s, CSWDG_EINVAL, "rhs_adjoint");
    Ctl h;
    if (cswdg_status r = read_ctl(s, &h)) return r;
    Ctl w = h;
    w.t = t;
    w.dt = 1.0;
    w.active = 1;
    if (cswdg_status r = write_ctl(s, &w)) return r;
    if (cswdg_status r = upload_modes(s, modes_in, s->U)) return r;
    s->lam_stale = true;
    if (cswdg_status r = upload_modes(s, lambda_in, s->A, true)) return r;
    if (s->fp32)
        launch_rhs_adjoint<float>(s->eq, s->k, mesh_dev<float>(s), (const float *)s->U, (const float *)s->A, (float *)s->B, 0.0, s->ctl,
                                  s->stream);
    else
        launch_rhs_adjoint<double>(s->eq, s->k, mesh_dev<double>(s), (const double *)s->U, (const double *)s->A, (double *)s->B, 0.0,
                                   s->ctl, s->stream);
    CK(cudaGetLastError());
    if (cswdg_status r = download_modes(s, s->B, grad_out, true)) return r;
    return write_ctl(s, &h);
}

// ---------------------------------------------------------------------------
// Adjoint of one limiter pass with the flags of the forward pass frozen
// ---------------------------------------------------------------------------
template <typename R>
static void limit_adjoint_dev(cswdg_solver *s, const void *u_pre, const int32_t *flist, const int32_t *nflag_dev, double tfac,
                              const void *gin, void *gout, size_t nstate, cudaStream_t st)
{
    cudaMemcpyAsync(gout, gin, nstate * sizeof(R), cudaMemcpyDeviceToDevice, st);
    launch_limit_adjoint<R>(s->eq, s->k, mesh_dev<R>(s), (const R *)u_pre, (const R *)s->ops, flist, nflag_dev, s->ctl, tfac, s->w32,
                            (const R *)gin, (R *)gout, s->lim_grid, st);
}

cswdg_status cswdg_limit_adjoint(cswdg_solver *s, double t, const double *modes_in, const double *lambda_in, double *grad_out,
                                 uint8_t *flags_out)
{
    if (!s || !s->mesh_ready || !modes_in || !lambda_in || !grad_out) return fail(s, CSWDG_EINVAL, "limit_adjoint");
    if (s->cfg.limiter == CSWDG_LIMITER_OFF) return fail(s, CSWDG_EINVAL, "limit_adjoint: the limiter is off");
    Ctl h;
    if (cswdg_status r = read_ctl(s, &h)) return r;
    Ctl w = h;
    w.t = t;
    w.dt = 0.0;
    w.active = 1;
    w.err = 0;
    if (cswdg_status r = write_ctl(s, &w)) return r;
    if (cswdg_status r = upload_modes(s, modes_in, s->U)) return r;
    s->lam_stale = true;
    // the forward pass (its flags and reconstructions), then the reverse
    CK(cudaMemcpyAsync(s->B, s->U, (size_t)s->nv * s->np * s->ldc * (s->fp32 ? 4 : 8), cudaMemcpyDeviceToDevice, s->stream));
    if (cswdg_status r = limiter_pass(s, s->B, 0.0, s->stream)) return r;
    if (cswdg_status r = upload_modes(s, lambda_in, s->A, true)) return r;
    const size_t nstate = (size_t)s->nv * s->np * s->ldc;
    if (s->fp32) limit_adjoint_dev<float>(s, s->U, s->flist, &s->ctl->nflag, 0.0, s->A, s->B, nstate, s->stream);
    else limit_adjoint_dev<double>(s, s->U, s->flist, &s->ctl->nflag, 0.0, s->A, s->B, nstate, s->stream);
    CK(cudaGetLastError());
    if (cswdg_status r = download_modes(s, s->B, grad_out, true)) return r;
    if (flags_out)
        if (cswdg_status r = cswdg_read_flags(s, flags_out)) return r;
    Ctl after;
    if (cswdg_status r = read_ctl(s, &after)) return r;
    h.nflag = after.nflag;
    h.err = after.err;
    if (cswdg_status r = write_ctl(s, &h)) return r;
    return check_err(s, &h);
}

// ---------------------------------------------------------------------------
// Reverse sweep of fixed-dt SSP-RK3 steps with checkpoints (hand-written
// adjoint; see the header).  Per step, with Lam_i the limiter pass after
// stage i (flags frozen), v1 = u0 + dt L(u0), u1 = Lam_1(v1),
// v2 = 3/4 u0 + 1/4 (u1 + dt L(u1)), u2 = Lam_2(v2),
// v3 = 1/3 u0 + 2/3 (u2 + dt L(u2)), u3 = Lam_3(v3):
//   b3 = Lam_3'^T g;  w = 2/3 b3;  h2 = w + dt L'(u2)^T w;  b2 = Lam_2'^T h2
//   g0 = 1/3 b3 + 3/4 b2;  w = 1/4 b2;  h1 = w + dt L'(u1)^T w;  b1 = Lam_1'^T h1
//   g0 += b1 + dt L'(u0)^T b1
// ---------------------------------------------------------------------------
// the time and step of one recomputed or reversed step of the adjoint sweep,
// set on the stream (no host round trip)
static __global__ void k_set_clock(Ctl *ctl, double t, double dt)
{
    ctl->t = t;
    ctl->dt = dt;
    ctl->dtf = (float)dt;
    ctl->active = 1;
}
static void launch_set_clock(Ctl *ctl, double t, double dt, cudaStream_t st) { k_set_clock<<<1, 1, 0, st>>>(ctl, t, dt); }

cswdg_status cswdg_adjoint_steps(cswdg_solver *s, double dt, int64_t nsteps, int32_t checkpoint_every, const double *u0_user,
                                 const double *gT_user, double *uT_user, double *g0_user, double *dt_host)
{
    if (!s || !s->mesh_ready || nsteps < 1 || checkpoint_every < 1 || !u0_user || !gT_user || !g0_user)
        return fail(s, CSWDG_EINVAL, "adjoint_steps: bad arguments");
    // dt <= 0: every step of the forward sweep takes the CFL rule; the sizes it
    // chose are then held fixed in the recomputation and the reverse sweep
    const int use_cfl = !(dt > 0.0);
    const bool lim = s->cfg.limiter != CSWDG_LIMITER_OFF;
    const size_t rs = s->fp32 ? 4 : 8, nstate = (size_t)s->nv * s->np * s->ldc, bytes = nstate * rs;
    const size_t flbytes = (size_t)s->ldc * 4;
    const int64_t ce = checkpoint_every, nck = (nsteps + ce - 1) / ce;
    // per step of a segment: u^n, the three unlimited stage outputs v1..v3 and the
    // limited u1, u2; the three flag lists and their counts
    const int NS = 6;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = nsm * 4;
    char *ck = nullptr, *seg = nullptr, *ga = nullptr, *gw = nullptr, *gt = nullptr, *gx = nullptr, *uN = nullptr;
    int32_t *fls = nullptr, *nfs = nullptr;
    double *dts = nullptr;
    cudaError_t e = cudaSuccess;
    auto A_ = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A_(cudaMalloc((void **)&dts, (size_t)nsteps * sizeof(double)));
    A_(cudaMalloc((void **)&ck, (size_t)nck * bytes));
    A_(cudaMalloc((void **)&seg, (size_t)NS * ce * bytes));
    A_(cudaMalloc((void **)&ga, bytes));
    A_(cudaMalloc((void **)&gw, bytes));
    A_(cudaMalloc((void **)&gt, bytes));
    A_(cudaMalloc((void **)&gx, bytes));
    A_(cudaMalloc((void **)&uN, bytes));
    if (lim) {
        A_(cudaMalloc((void **)&fls, (size_t)3 * ce * flbytes));
        A_(cudaMalloc((void **)&nfs, (size_t)3 * ce * 4));
    }
    auto release = [&]() {
        cudaFree(ck); cudaFree(seg); cudaFree(ga); cudaFree(gw); cudaFree(gt); cudaFree(gx); cudaFree(uN);
        cudaFree(fls); cudaFree(nfs); cudaFree(dts);
    };
    if (e != cudaSuccess) {
        release();
        return fail(s, CSWDG_ENOMEM, "adjoint_steps: device allocation: %s", cudaGetErrorString(e));
    }
#define CKR(x)                                                                                           \
    do {                                                                                                 \
        cudaError_t e_ = (x);                                                                            \
        if (e_ != cudaSuccess) { release(); return fail(s, CSWDG_ECUDA, "%s", cudaGetErrorString(e_)); } \
    } while (0)
#define STR(x)                                        \
    do {                                              \
        cswdg_status r_ = (x);                        \
        if (r_ != CSWDG_OK) { release(); return r_; } \
    } while (0)
    Ctl h;
    STR(read_ctl(s, &h));
    const double t0 = h.t_next;
    h.dt_fixed = dt;
    h.cfl = s->cfg.cfl;
    h.t_end = 1e300;
    STR(upload_modes(s, u0_user, s->U));
    s->lam_stale = true;
    if (use_cfl) STR(refresh_lam(s, &h, nullptr));
    STR(write_ctl(s, &h));
    STR(get_graph(s, use_cfl));
    // forward sweep, checkpoints of u^n every ce steps and the step sizes taken
    for (int64_t n = 0; n < nsteps; ++n) {
        if (n % ce == 0) CKR(cudaMemcpyAsync(ck + (size_t)(n / ce) * bytes, s->U, bytes, cudaMemcpyDeviceToDevice, s->stream));
        CKR(cudaGraphLaunch(s->graph[use_cfl], s->stream));
        CKR(cudaMemcpyAsync(dts + n, &s->ctl->dt, sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    }
    CKR(cudaMemcpyAsync(uN, s->U, bytes, cudaMemcpyDeviceToDevice, s->stream));
    std::vector<double> dtv((size_t)nsteps);
    CKR(cudaMemcpyAsync(dtv.data(), dts, (size_t)nsteps * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    Ctl hf;
    STR(read_ctl(s, &hf));
    if (cswdg_status r = check_err(s, &hf)) { release(); return r; }
    // the step times exactly as k_begin_step accumulated them
    std::vector<double> times((size_t)nsteps + 1);
    times[0] = t0;
    for (int64_t n = 0; n < nsteps; ++n) {
        if (!(dtv[n] > 0.0)) { release(); return fail(s, CSWDG_ENONPHYS, "adjoint_steps: step %lld has no positive size", (long long)n); }
        times[n + 1] = times[n] + dtv[n];
    }
    if (dt_host) std::copy(dtv.begin(), dtv.end(), dt_host);
    if (uT_user) STR(download_modes(s, s->U, uT_user));
    // reverse sweep; the four adjoint buffers change roles by pointer swaps
    char *pa = ga, *pt = gt, *pw = gw, *px = gx;
    STR(upload_modes(s, gT_user, pa, true));
    for (int64_t sg = nck - 1; sg >= 0; --sg) {
        const int64_t n0 = sg * ce, n1 = std::min(nsteps, n0 + ce);
        CKR(cudaMemcpyAsync(s->U, ck + (size_t)sg * bytes, bytes, cudaMemcpyDeviceToDevice, s->stream));
        // recompute the segment stage by stage, keeping what the reverse sweep reads
        for (int64_t n = n0; n < n1; ++n) {
            char *base = seg + (size_t)NS * (n - n0) * bytes;
            int32_t *fl = lim ? fls + (size_t)3 * (n - n0) * s->ldc : nullptr;
            int32_t *nf = lim ? nfs + 3 * (n - n0) : nullptr;
            launch_set_clock(s->ctl, times[n], dtv[n], s->stream);
            CKR(cudaMemcpyAsync(base, s->U, bytes, cudaMemcpyDeviceToDevice, s->stream));
            void *outs[3] = {s->A, s->B, s->U};
            const void *ins[3] = {s->U, s->A, s->B};
            const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0}, tf[3] = {0.0, 1.0, 0.5},
                         tl[3] = {1.0, 0.5, 1.0};
            for (int k = 0; k < 3; ++k) {
                STR(stage(s, k ? s->U : nullptr, ins[k], outs[k], ca[k], cb[k], cb[k], tf[k], s->stream, nullptr, 0, lim));
                CKR(cudaMemcpyAsync(base + (size_t)(1 + k) * bytes, outs[k], bytes, cudaMemcpyDeviceToDevice, s->stream));
                if (lim) {
                    STR(limiter_pass(s, outs[k], tl[k], s->stream, nullptr, false, true));
                    CKR(cudaMemcpyAsync(fl + (size_t)k * s->ldc, s->flist, flbytes, cudaMemcpyDeviceToDevice, s->stream));
                    CKR(cudaMemcpyAsync(nf + k, &s->ctl->nflag, 4, cudaMemcpyDeviceToDevice, s->stream));
                }
                if (k < 2) CKR(cudaMemcpyAsync(base + (size_t)(4 + k) * bytes, outs[k], bytes, cudaMemcpyDeviceToDevice, s->stream));
            }
        }
        for (int64_t n = n1 - 1; n >= n0; --n) {
            const char *base = seg + (size_t)NS * (n - n0) * bytes;
            const int32_t *fl = lim ? fls + (size_t)3 * (n - n0) * s->ldc : nullptr;
            const int32_t *nf = lim ? nfs + 3 * (n - n0) : nullptr;
            launch_set_clock(s->ctl, times[n], dtv[n], s->stream);
            const void *u0s = base, *v1 = base + bytes, *v2 = base + 2 * bytes, *v3 = base + 3 * bytes, *u1s = base + 4 * bytes,
                       *u2s = base + 5 * bytes;
            // the transposed stage updates with the linear combinations fused into
            // the operator adjoint's epilogue (it is linear in its adjoint input):
            //   h2 = 2/3 (b3 + dt L'(u2)^T b3);  a = 1/3 b3 + 3/4 b2;
            //   h1 = 1/4 (b2 + dt L'(u1)^T b2);  g0 = a + b1 + dt L'(u0)^T b1
            // limiter adjoints write a spare buffer, whose pointer then swaps in
            auto run = [&](auto tag) {
                using R = decltype(tag);
                const MeshDev<R> M = mesh_dev<R>(s);
                const R d = (R)dtv[n];
                R *a = (R *)pa, *t = (R *)pt, *w = (R *)pw, *x = (R *)px;
                if (lim) {  // b3 = Lam_3'^T g
                    limit_adjoint_dev<R>(s, v3, fl + 2 * (size_t)s->ldc, nf + 2, 1.0, a, x, nstate, s->stream);
                    std::swap(a, x);
                }
                launch_rhs_adjoint<R>(s->eq, s->k, M, (const R *)u2s, a, t, 0.5, s->ctl, s->stream, a, R(2) / R(3), nullptr, R(0),
                                      R(2) / R(3) * d);
                if (lim) {  // b2 = Lam_2'^T h2
                    limit_adjoint_dev<R>(s, v2, fl + (size_t)s->ldc, nf + 1, 0.5, t, x, nstate, s->stream);
                    std::swap(t, x);
                }
                launch_axpby<R>(nstate, R(1) / R(3), a, R(0.75), t, a, grid, s->stream);
                launch_rhs_adjoint<R>(s->eq, s->k, M, (const R *)u1s, t, w, 1.0, s->ctl, s->stream, t, R(0.25), nullptr, R(0),
                                      R(0.25) * d);
                if (lim) {  // b1 = Lam_1'^T h1
                    limit_adjoint_dev<R>(s, v1, fl, nf, 1.0, w, x, nstate, s->stream);
                    std::swap(w, x);
                }
                launch_rhs_adjoint<R>(s->eq, s->k, M, (const R *)u0s, w, a, 0.0, s->ctl, s->stream, a, R(1), w, R(1), d);
                pa = (char *)a; pt = (char *)t; pw = (char *)w; px = (char *)x;
            };
            if (s->fp32) run(float(0));
            else run(double(0));
            CKR(cudaGetLastError());
        }
    }
    STR(download_modes(s, pa, g0_user, true));
    // leave the solver at u^N and t^N
    CKR(cudaMemcpyAsync(s->U, uN, bytes, cudaMemcpyDeviceToDevice, s->stream));
    Ctl fin = hf;
    fin.t = fin.t_next = times[nsteps];
    STR(write_ctl(s, &fin));
    release();
#undef CKR
#undef STR
    return CSWDG_OK;
}

// host-side mesh processing alone, no device (see the header)
cswdg_status cswdg_host_mesh(int32_t degree, const int32_t *bc_kind_host, int64_t nv, const double *xy_host, int64_t nc64,
                             const int32_t *tri_host, int64_t nbf, const int32_t *bface_host, const double *period_host,
                             double *geo_host, int32_t *nbr_host, uint8_t *nbf_host, int32_t *perm_host)
{
    if ((degree != 1 && degree != 2) || !bc_kind_host || !xy_host || !tri_host || nv < 3 || nc64 < 1 || nc64 > (1 << 30) ||
        nbf < 0 || (nbf > 0 && !bface_host))
        return CSWDG_EINVAL;
    int32_t kinds[CSW_MAXTAG];
    for (int t = 0; t < CSW_MAXTAG; ++t) kinds[t] = bc_kind_host[t];
    HostMesh H;
    if (int st = build_host_mesh(degree, kinds, nv, xy_host, nc64, tri_host, nbf, bface_host, period_host, H))
        return (cswdg_status)st;
    const int nc = H.nc, ld = H.ldc;
    if (geo_host)
        for (int g = 0; g < G_COUNT; ++g)
            for (int c = 0; c < nc; ++c) geo_host[(size_t)g * nc + c] = H.geo[(size_t)g * ld + c];
    if (nbr_host)
        for (int f = 0; f < 3; ++f)
            for (int c = 0; c < nc; ++c) nbr_host[(size_t)f * nc + c] = H.nbr[(size_t)f * ld + c];
    if (nbf_host)
        for (int c = 0; c < nc; ++c) nbf_host[c] = H.nbfv[c];
    if (perm_host)
        for (int c = 0; c < nc; ++c) perm_host[c] = H.perm[c];
    return CSWDG_OK;
}
