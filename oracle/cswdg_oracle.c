/*
 * cswdg_oracle.c -- plain, slow FP64 CPU oracle for the RKDG method with the
 * compact subcell WENO (CSWENO) limiter of Kochi & Ramakrishna,
 * "A compact subcell WENO limiting strategy using immediate neighbors for
 * Runge-Kutta discontinuous Galerkin methods for unstructured meshes"
 * (arXiv 2106.06280).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path; both sides only consume the
 * same seeded meshes and initial data.
 *
 * Everything here follows the paper's steps in the paper's order, one cell or
 * one face at a time, with no blocking, fusion or precomputation:
 *   Sec. 2, Eq. (modalForm2D), Eq. (triangleBasis)   modal DG on triangles
 *   Sec. 2, Eq. (weakFormScheme2D), (massMatrix2D)    semi-discrete operator
 *   Sec. 3.1, Eq. (troubledCellIndicator)             KXRCF detector
 *   Sec. 3.2, Steps 1-5 (P1) and Steps 1-4 (P2)       CSWENO reconstruction
 *   Sec. 3.2, Eq. (timeIntegrate), Table (tvd)        SSP-RK3 with limiter
 * Where the paper is silent or garbled the reading taken is stated at the
 * function that implements it (readings R-*).
 *
 * Mode layout used at the interface: u[(c*nvar + v)*np + m] for cell c,
 * variable v, mode m; modes are coefficients of the physically orthonormal
 * basis psi^K_m(x) = sqrt(2/|K|) psi_m(r(x)) (reading R-basis), so the local
 * mass matrix is the identity and the cell mean is u_0 / sqrt(|K|).
 *
 * Built with -ffp-contract=off so the same source gives the same bits on
 * every host.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXNP 6
#define OR_MAXV 4
#define OR_MAXQ 64

enum { EQ_BURGERS = 0, EQ_EULER = 1 };
enum { LIM_OFF = 0, LIM_KXRCF = 1, LIM_ALL = 2 };
enum { BC_PERIODIC = 0, BC_DIRICHLET = 1, BC_TRANSMISSIVE = 2, BC_WALL = 3, BC_SHOCKLINE = 4 };
#define OR_MAXTAG 16
#define OR_MAXPAR 16

/* ======================================================================
 * 1. Jacobi polynomials and the orthonormal triangle basis
 *    (Sec. 2, Eq. triangleBasis; normalised Jacobi polynomials, reading
 *    R-basis: the text calls the basis orthonormal, so the Jacobi factors
 *    carry their L2 normalisation).
 * ====================================================================== */

/* Unnormalised P_n^{(a,b)}(x) by the classical three-term recurrence. */
static double jacobi_p(int n, double a, double b, double x)
{
    if (n == 0) return 1.0;
    double p0 = 1.0;
    double p1 = 0.5 * ((a + b + 2.0) * x + (a - b));
    for (int m = 2; m <= n; ++m) {
        double c = 2.0 * m + a + b;
        double d1 = 2.0 * m * (m + a + b) * (c - 2.0);
        double d2 = (c - 1.0) * (c * (c - 2.0) * x + a * a - b * b);
        double d3 = 2.0 * (m + a - 1.0) * (m + b - 1.0) * c;
        double p2 = (d2 * p1 - d3 * p0) / d1;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

/* sqrt of int_{-1}^{1} (1-x)^alpha P_n^{(alpha,0)}(x)^2 dx = 2^{alpha+1}/(2n+alpha+1). */
static double jacobi_norm(int n, int alpha)
{
    return sqrt(ldexp(1.0, alpha + 1) / (2.0 * n + alpha + 1.0));
}

static double jacobi_n(int n, int alpha, double x)
{
    return jacobi_p(n, alpha, 0.0, x) / jacobi_norm(n, alpha);
}

/* d/dx P_n^{(a,0)} = (n+a+1)/2 P_{n-1}^{(a+1,1)}. */
static double jacobi_n_dx(int n, int alpha, double x)
{
    if (n == 0) return 0.0;
    return 0.5 * (n + alpha + 1.0) * jacobi_p(n - 1, alpha + 1.0, 1.0, x) / jacobi_norm(n, alpha);
}

/* Mode m (0-based) <-> (i,j): i outer, j inner, i+j <= k; this is the
 * paper's m = j + (N+1)i + 1 - i(i-1)/2 shifted to start at 0. */
static void mode_ij(int k, int m, int *pi, int *pj)
{
    int idx = 0;
    for (int i = 0; i <= k; ++i)
        for (int j = 0; j <= k - i; ++j) {
            if (idx == m) { *pi = i; *pj = j; return; }
            ++idx;
        }
    *pi = *pj = 0;
}

/* psi_m(r,s) on I = {r,s >= -1, r+s <= 0} and its (r,s) gradient. */
static void psi_ref(int k, int m, double r, double s, double *val, double *dr, double *ds)
{
    int i, j;
    mode_ij(k, m, &i, &j);
    double b = s, omb = 1.0 - s;
    double a = (omb > 0.0) ? 2.0 * (1.0 + r) / omb - 1.0 : -1.0;
    double fa = jacobi_n(i, 0, a), dfa = jacobi_n_dx(i, 0, a);
    double gb = jacobi_n(j, 2 * i + 1, b), dgb = jacobi_n_dx(j, 2 * i + 1, b);
    double wi = pow(omb, i);
    double wim1 = (i >= 1) ? pow(omb, i - 1) : 0.0;
    if (val) *val = M_SQRT2 * fa * gb * wi;
    if (dr) *dr = M_SQRT2 * dfa * gb * 2.0 * wim1;
    if (ds) *ds = M_SQRT2 * (dfa * (1.0 + a) * gb * wim1 + fa * dgb * wi - i * fa * gb * wim1);
}

/* ======================================================================
 * 2. Quadrature rules (derived here; none is typed in from a table)
 * ====================================================================== */

/* Gauss-Legendre on [-1,1]: Newton iteration on the Legendre polynomial. */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int m = 2; m <= n; ++m) {
                double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 1) ? z : p1, pnm1 = (n == 1) ? 1.0 : p0;
            double dp = n * (z * pn - pnm1) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int m = 2; m <= n; ++m) {
            double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
            p0 = p1;
            p1 = p2;
        }
        double pn = (n == 1) ? z : p1, pnm1 = (n == 1) ? 1.0 : p0;
        double dp = n * (z * pn - pnm1) / (z * z - 1.0);
        x[n - 1 - i] = z; /* ascending */
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

typedef struct {
    int n;
    double b[OR_MAXQ][3]; /* barycentric coordinates */
    double w[OR_MAXQ];    /* weights summing to 1 */
} trirule;

/* Collapsed (Duffy) Gauss rule with m x m points: P = (1-u) v0 + u(1-w) v1 + u w v2,
 * Jacobian 2|T| u.  Exact for total degree 2m-2. */
static void duffy_rule(int m, trirule *R)
{
    double x[16], w[16];
    gauss_legendre(m, x, w);
    R->n = 0;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            double u = 0.5 * (x[i] + 1.0), v = 0.5 * (x[j] + 1.0);
            double wt = 0.25 * w[i] * w[j] * 2.0 * u;
            R->b[R->n][0] = 1.0 - u;
            R->b[R->n][1] = u * (1.0 - v);
            R->b[R->n][2] = u * v;
            R->w[R->n] = wt;
            R->n++;
        }
}

static double fact(int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= i; return f; }

/* Dense least squares min ||A c - b|| by Householder QR (A m x n row-major,
 * m >= n).  Returns 0, or -1 if a pivot falls below 1e-13 * the largest. */
static int lsq_qr(int m, int n, const double *A_in, const double *b_in, double *c)
{
    double A[32 * 32], b[32];
    if (m > 32 || n > 32 || m < n) return -2;
    memcpy(A, A_in, sizeof(double) * m * n);
    memcpy(b, b_in, sizeof(double) * m);
    double rmax = 0.0;
    for (int j = 0; j < n; ++j) {
        double nrm = 0.0;
        for (int i = j; i < m; ++i) nrm += A[i * n + j] * A[i * n + j];
        nrm = sqrt(nrm);
        if (nrm == 0.0) return -1;
        double alpha = (A[j * n + j] > 0.0) ? -nrm : nrm;
        double v[32];
        for (int i = 0; i < m; ++i) v[i] = 0.0;
        for (int i = j; i < m; ++i) v[i] = A[i * n + j];
        v[j] -= alpha;
        double vv = 0.0;
        for (int i = j; i < m; ++i) vv += v[i] * v[i];
        if (vv > 0.0) {
            for (int col = j; col < n; ++col) {
                double s = 0.0;
                for (int i = j; i < m; ++i) s += v[i] * A[i * n + col];
                s = 2.0 * s / vv;
                for (int i = j; i < m; ++i) A[i * n + col] -= s * v[i];
            }
            double s = 0.0;
            for (int i = j; i < m; ++i) s += v[i] * b[i];
            s = 2.0 * s / vv;
            for (int i = j; i < m; ++i) b[i] -= s * v[i];
        }
        if (fabs(A[j * n + j]) > rmax) rmax = fabs(A[j * n + j]);
    }
    for (int j = 0; j < n; ++j)
        if (fabs(A[j * n + j]) < 1e-13 * rmax) return -1;
    for (int j = n - 1; j >= 0; --j) {
        double s = b[j];
        for (int col = j + 1; col < n; ++col) s -= A[j * n + col] * c[col];
        c[j] = s / A[j * n + j];
    }
    return 0;
}

/* Fully symmetric triangle rules found by Gauss-Newton on the moment
 * equations sum_q w_q x_q^p y_q^q = 2 p! q!/(p+q+2)!, p+q <= degree, on the
 * unit triangle (x = lambda_2, y = lambda_3).  Orbit S3 is the centroid,
 * orbit S21(a) is the three points (a, a, 1-2a) and its permutations.  The
 * starting guesses only select which root is found; the result is exact to
 * rounding and checked by the residual.
 *   degree 2: S21           (3 points)  volume rule P1 and reconstruction points P1
 *   degree 4: S21 + S21     (6 points)  reconstruction points P2
 *   degree 5: S3 + S21 + S21 (7 points) volume rule P2
 */
static int sym_rule(int degree, trirule *R)
{
    int has_c = 0, norb = 0;
    double th[8];
    if (degree == 2) { norb = 1; th[0] = 0.2; th[1] = 1.0 / 3.0; }
    else if (degree == 4) { norb = 2; th[0] = 0.09; th[1] = 0.11; th[2] = 0.44; th[3] = 0.22; }
    else if (degree == 5) { has_c = 1; norb = 2; th[0] = 0.1; th[1] = 0.126; th[2] = 0.47; th[3] = 0.132; th[4] = 0.225; }
    else return -1;
    int nu = 2 * norb + has_c;
    int neq = (degree + 1) * (degree + 2) / 2;
    for (int it = 0; it < 60; ++it) {
        double res[64], J[64 * 8];
        int e = 0;
        for (int tot = 0; tot <= degree; ++tot)
            for (int q = 0; q <= tot; ++q) {
                int p = tot - q;
                double target = 2.0 * fact(p) * fact(q) / fact(p + q + 2);
                double s = 0.0;
                for (int u = 0; u < nu; ++u) J[e * nu + u] = 0.0;
                for (int o = 0; o < norb; ++o) {
                    double a = th[2 * o], w = th[2 * o + 1];
                    /* the three points in (x,y) = (lambda2, lambda3) and d/da */
                    double px[3] = {a, a, 1.0 - 2.0 * a}, py[3] = {a, 1.0 - 2.0 * a, a};
                    double dx[3] = {1.0, 1.0, -2.0}, dy[3] = {1.0, -2.0, 1.0};
                    for (int t = 0; t < 3; ++t) {
                        double f = pow(px[t], p) * pow(py[t], q);
                        double df = 0.0;
                        if (p > 0) df += p * pow(px[t], p - 1) * pow(py[t], q) * dx[t];
                        if (q > 0) df += q * pow(px[t], p) * pow(py[t], q - 1) * dy[t];
                        s += w * f;
                        J[e * nu + 2 * o] += w * df;
                        J[e * nu + 2 * o + 1] += f;
                    }
                }
                if (has_c) {
                    double f = pow(1.0 / 3.0, p + q);
                    s += th[2 * norb] * f;
                    J[e * nu + 2 * norb] = f;
                }
                res[e] = target - s;
                ++e;
            }
        double d[8];
        if (lsq_qr(neq, nu, J, res, d) != 0) return -1;
        double dn = 0.0;
        for (int u = 0; u < nu; ++u) { th[u] += d[u]; dn += fabs(d[u]); }
        if (dn < 1e-17) break;
    }
    R->n = 0;
    if (has_c) {
        R->b[0][0] = R->b[0][1] = R->b[0][2] = 1.0 / 3.0;
        R->w[0] = th[2 * norb];
        R->n = 1;
    }
    for (int o = 0; o < norb; ++o) {
        double a = th[2 * o], w = th[2 * o + 1];
        double pts[3][3] = {{1.0 - 2.0 * a, a, a}, {a, 1.0 - 2.0 * a, a}, {a, a, 1.0 - 2.0 * a}};
        for (int t = 0; t < 3; ++t) {
            R->b[R->n][0] = pts[t][0];
            R->b[R->n][1] = pts[t][1];
            R->b[R->n][2] = pts[t][2];
            R->w[R->n] = w;
            R->n++;
        }
    }
    /* residual check */
    for (int tot = 0; tot <= degree; ++tot)
        for (int q = 0; q <= tot; ++q) {
            int p = tot - q;
            double s = 0.0;
            for (int t = 0; t < R->n; ++t) s += R->w[t] * pow(R->b[t][1], p) * pow(R->b[t][2], q);
            if (fabs(s - 2.0 * fact(p) * fact(q) / fact(p + q + 2)) > 1e-14) return -1;
        }
    return 0;
}

/* ======================================================================
 * 3. The oracle object: mesh, connectivity, geometry, problem
 * ====================================================================== */

typedef struct {
    int eq, k, np, nvar, limiter;
    double ck, gam;
    int nv, nc;
    double *vx, *vy;
    int *tri;    /* 3*nc, counter-clockwise */
    int *nb;     /* 3*nc: neighbour across local face f (v_f -> v_{f+1}), -1 on a boundary */
    int *nbf;    /* 3*nc: the neighbour's local index of the shared face */
    double *sh;  /* 6*nc: add to the neighbour's coordinates to place it next to this cell */
    int *btag;   /* 3*nc: boundary tag of a boundary face */
    int bkind[OR_MAXTAG];
    double bpar[OR_MAXTAG][OR_MAXPAR];
    trirule vol, scp, duf2, duf3, duf4, duf6;
    int nfq;
    double fx[8], fw[8]; /* face Gauss points in [0,1] and weights summing to 1 */
    int err;
} Oracle;

typedef struct {
    double x[3], y[3];
} Tri;

static Tri cell_tri(const Oracle *o, int c, double shx, double shy)
{
    Tri t;
    for (int i = 0; i < 3; ++i) {
        t.x[i] = o->vx[o->tri[3 * c + i]] + shx;
        t.y[i] = o->vy[o->tri[3 * c + i]] + shy;
    }
    return t;
}

static double tri_area(const Tri *t)
{
    return 0.5 * ((t->x[1] - t->x[0]) * (t->y[2] - t->y[0]) - (t->x[2] - t->x[0]) * (t->y[1] - t->y[0]));
}

static void tri_point(const Tri *t, const double *bary, double *x, double *y)
{
    *x = bary[0] * t->x[0] + bary[1] * t->x[1] + bary[2] * t->x[2];
    *y = bary[0] * t->y[0] + bary[1] * t->y[1] + bary[2] * t->y[2];
}

/* Physical point -> reference (r,s) of the affine map of triangle t. */
static void tri_to_ref(const Tri *t, double x, double y, double *r, double *s)
{
    double a11 = t->x[1] - t->x[0], a12 = t->x[2] - t->x[0];
    double a21 = t->y[1] - t->y[0], a22 = t->y[2] - t->y[0];
    double det = a11 * a22 - a12 * a21;
    double dx = x - t->x[0], dy = y - t->y[0];
    double rho = (a22 * dx - a12 * dy) / det;
    double sig = (-a21 * dx + a11 * dy) / det;
    *r = 2.0 * rho - 1.0;
    *s = 2.0 * sig - 1.0;
}

/* Physical basis psi^K_m(x,y) = sqrt(2/|K|) psi_m(r(x,y)) and its x,y gradient
 * (reading R-basis: the physically orthonormal scaling that makes the
 * projection of Eq. finalMoments exact with weights summing to one). */
static void psi_phys(const Oracle *o, const Tri *t, int m, double x, double y, double *val, double *gx, double *gy)
{
    double r, s, v, dr, ds;
    tri_to_ref(t, x, y, &r, &s);
    psi_ref(o->k, m, r, s, &v, &dr, &ds);
    double area = tri_area(t);
    double sc = sqrt(2.0 / area);
    double a11 = t->x[1] - t->x[0], a12 = t->x[2] - t->x[0];
    double a21 = t->y[1] - t->y[0], a22 = t->y[2] - t->y[0];
    double det = a11 * a22 - a12 * a21;
    /* r = 2 rho - 1: dr/dx = 2 a22/det, dr/dy = -2 a12/det, ds/dx = -2 a21/det, ds/dy = 2 a11/det */
    double rx = 2.0 * a22 / det, ry = -2.0 * a12 / det, sx = -2.0 * a21 / det, sy = 2.0 * a11 / det;
    if (val) *val = sc * v;
    if (gx) *gx = sc * (dr * rx + ds * sx);
    if (gy) *gy = sc * (dr * ry + ds * sy);
}

/* u_h of cell c (all variables) at a physical point of the frame of c. */
static void eval_cell(const Oracle *o, const double *u, int c, const Tri *t, double x, double y, double *U)
{
    for (int v = 0; v < o->nvar; ++v) U[v] = 0.0;
    for (int m = 0; m < o->np; ++m) {
        double p;
        psi_phys(o, t, m, x, y, &p, NULL, NULL);
        for (int v = 0; v < o->nvar; ++v) U[v] += u[(c * o->nvar + v) * o->np + m] * p;
    }
}

typedef struct { long long key; int cell, face; } HalfEdge;

static int he_cmp(const void *a, const void *b)
{
    const HalfEdge *x = (const HalfEdge *)a, *y = (const HalfEdge *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return 0;
}

Oracle *or_create(int eq, int k, int limiter, double ck, double gam)
{
    Oracle *o = (Oracle *)calloc(1, sizeof(Oracle));
    o->eq = eq;
    o->k = k;
    o->np = (k + 1) * (k + 2) / 2;
    o->nvar = (eq == EQ_EULER) ? 4 : 1;
    o->limiter = limiter;
    o->ck = ck;
    o->gam = gam;
    /* Volume rule exact to degree max(2k, 3k-1) and face rule exact to degree
     * 3k (reading R-quad; the paper names no rule for the operator). */
    if (sym_rule(k == 1 ? 2 : 5, &o->vol) != 0) o->err = 1;
    /* Np-point symmetric rule exact to degree 2k standing in for the SCP rule
     * (reading R-scp; the paper cites the rule but prints no points). */
    if (sym_rule(k == 1 ? 2 : 4, &o->scp) != 0) o->err = 1;
    duffy_rule(2, &o->duf2);
    duffy_rule(3, &o->duf3);
    duffy_rule(4, &o->duf4);
    duffy_rule(6, &o->duf6);
    o->nfq = (k == 1) ? 2 : 4;
    double gx[8], gw[8];
    gauss_legendre(o->nfq, gx, gw);
    for (int g = 0; g < o->nfq; ++g) { o->fx[g] = 0.5 * (gx[g] + 1.0); o->fw[g] = 0.5 * gw[g]; }
    for (int t = 0; t < OR_MAXTAG; ++t) o->bkind[t] = -1;
    return o;
}

void or_destroy(Oracle *o)
{
    if (!o) return;
    free(o->vx); free(o->vy); free(o->tri); free(o->nb); free(o->nbf); free(o->sh); free(o->btag);
    free(o);
}

int or_error(const Oracle *o) { return o->err; }
int or_nvol(const Oracle *o) { return o->vol.n; }
int or_nscp(const Oracle *o) { return o->scp.n; }

void or_set_boundary(Oracle *o, int tag, int kind, const double *par, int npar)
{
    if (tag < 0 || tag >= OR_MAXTAG) return;
    o->bkind[tag] = kind;
    for (int i = 0; i < npar && i < OR_MAXPAR; ++i) o->bpar[tag][i] = par[i];
}

/* Mesh: vertices xy[2*nv], triangles tri[3*nc] (CCW), boundary faces
 * bface[3*nbf] = (v0, v1, tag).  Faces with a tag of kind BC_PERIODIC are
 * paired by a translation of (+-period[0], 0) or (0, +-period[1]). */
int or_mesh(Oracle *o, int nv, const double *xy, int nc, const int *tri, int nbf, const int *bface, const double *period)
{
    o->nv = nv;
    o->nc = nc;
    o->vx = (double *)malloc(sizeof(double) * nv);
    o->vy = (double *)malloc(sizeof(double) * nv);
    for (int i = 0; i < nv; ++i) { o->vx[i] = xy[2 * i]; o->vy[i] = xy[2 * i + 1]; }
    o->tri = (int *)malloc(sizeof(int) * 3 * nc);
    memcpy(o->tri, tri, sizeof(int) * 3 * nc);
    o->nb = (int *)malloc(sizeof(int) * 3 * nc);
    o->nbf = (int *)malloc(sizeof(int) * 3 * nc);
    o->sh = (double *)calloc(6 * (size_t)nc, sizeof(double));
    o->btag = (int *)malloc(sizeof(int) * 3 * nc);
    for (int i = 0; i < 3 * nc; ++i) { o->nb[i] = -1; o->nbf[i] = -1; o->btag[i] = -1; }
    for (int c = 0; c < nc; ++c) {
        Tri t = cell_tri(o, c, 0, 0);
        if (tri_area(&t) <= 0.0) return -1;
    }
    HalfEdge *he = (HalfEdge *)malloc(sizeof(HalfEdge) * 3 * nc);
    for (int c = 0; c < nc; ++c)
        for (int f = 0; f < 3; ++f) {
            long long a = tri[3 * c + f], b = tri[3 * c + (f + 1) % 3];
            long long lo = a < b ? a : b, hi = a < b ? b : a;
            he[3 * c + f].key = lo * (long long)nv + hi;
            he[3 * c + f].cell = c;
            he[3 * c + f].face = f;
        }
    qsort(he, 3 * (size_t)nc, sizeof(HalfEdge), he_cmp);
    for (int i = 0; i < 3 * nc;) {
        int j = i + 1;
        while (j < 3 * nc && he[j].key == he[i].key) ++j;
        if (j - i == 2) {
            int c0 = he[i].cell, f0 = he[i].face, c1 = he[i + 1].cell, f1 = he[i + 1].face;
            o->nb[3 * c0 + f0] = c1; o->nbf[3 * c0 + f0] = f1;
            o->nb[3 * c1 + f1] = c0; o->nbf[3 * c1 + f1] = f0;
        } else if (j - i > 2) {
            free(he);
            return -2; /* non-manifold */
        }
        i = j;
    }
    free(he);
    /* boundary tags (set_boundary must have been called for every tag) */
    {
        /* map boundary half-edges to their tags through a sorted key list */
        HalfEdge *bk = (HalfEdge *)malloc(sizeof(HalfEdge) * (nbf > 0 ? nbf : 1));
        for (int e = 0; e < nbf; ++e) {
            long long a = bface[3 * e], b = bface[3 * e + 1];
            long long lo = a < b ? a : b, hi = a < b ? b : a;
            bk[e].key = lo * (long long)nv + hi;
            bk[e].cell = bface[3 * e + 2];
            bk[e].face = e;
        }
        qsort(bk, nbf, sizeof(HalfEdge), he_cmp);
        for (int c = 0; c < nc; ++c)
            for (int f = 0; f < 3; ++f) {
                if (o->nb[3 * c + f] >= 0) continue;
                long long a = tri[3 * c + f], b = tri[3 * c + (f + 1) % 3];
                long long lo = a < b ? a : b, hi = a < b ? b : a;
                HalfEdge q;
                q.key = lo * (long long)nv + hi;
                HalfEdge *hit = (HalfEdge *)bsearch(&q, bk, nbf, sizeof(HalfEdge), he_cmp);
                if (!hit) { free(bk); return -3; }
                o->btag[3 * c + f] = hit->cell;
                if (hit->cell < 0 || hit->cell >= OR_MAXTAG) { free(bk); return -3; }
            }
        free(bk);
    }
    /* periodic pairing by translation */
    if (period) {
        double L[2] = {period[0], period[1]};
        double tol = 1e-9 * (fabs(L[0]) + fabs(L[1]));
        int nper = 0;
        for (int i = 0; i < 3 * nc; ++i)
            if (o->nb[i] < 0 && o->bkind[o->btag[i]] == BC_PERIODIC) ++nper;
        int *lst = (int *)malloc(sizeof(int) * (nper > 0 ? nper : 1));
        nper = 0;
        for (int i = 0; i < 3 * nc; ++i)
            if (o->nb[i] < 0 && o->bkind[o->btag[i]] == BC_PERIODIC) lst[nper++] = i;
        for (int p = 0; p < nper; ++p) {
            int i = lst[p];
            if (o->nb[i] >= 0) continue;
            int c = i / 3, f = i % 3;
            double ax = o->vx[o->tri[3 * c + f]], ay = o->vy[o->tri[3 * c + f]];
            double bx = o->vx[o->tri[3 * c + (f + 1) % 3]], by = o->vy[o->tri[3 * c + (f + 1) % 3]];
            for (int q = 0; q < nper; ++q) {
                int jj = lst[q];
                if (jj == i || o->nb[jj] >= 0) continue;
                int d = jj / 3, g = jj % 3;
                double cx = o->vx[o->tri[3 * d + g]], cy = o->vy[o->tri[3 * d + g]];
                double dx = o->vx[o->tri[3 * d + (g + 1) % 3]], dy = o->vy[o->tri[3 * d + (g + 1) % 3]];
                /* the partner runs the other way: a <-> d and b <-> c */
                double sx = ax - dx, sy = ay - dy;
                int okshift = (fabs(fabs(sx) - L[0]) < tol && fabs(sy) < tol) || (fabs(fabs(sy) - L[1]) < tol && fabs(sx) < tol);
                if (!okshift) continue;
                if (fabs(bx - cx - sx) > tol || fabs(by - cy - sy) > tol) continue;
                /* neighbour d seen from c: add (sx,sy) */
                o->nb[i] = d; o->nbf[i] = g;
                o->sh[2 * i] = sx; o->sh[2 * i + 1] = sy;
                o->nb[jj] = c; o->nbf[jj] = f;
                o->sh[2 * jj] = -sx; o->sh[2 * jj + 1] = -sy;
                break;
            }
            if (o->nb[i] < 0) { free(lst); return -4; }
        }
        free(lst);
    }
    for (int i = 0; i < 3 * nc; ++i)
        if (o->nb[i] < 0 && (o->btag[i] < 0 || o->bkind[o->btag[i]] < 0 || o->bkind[o->btag[i]] == BC_PERIODIC)) return -5;
    return 0;
}

/* ======================================================================
 * 4. Physics: Burgers (Eq. 2dBurgers) and Euler (Eq. 2dEulerEquations)
 * ====================================================================== */

static double euler_p(double gam, const double *U)
{
    return (gam - 1.0) * (U[3] - 0.5 * (U[1] * U[1] + U[2] * U[2]) / U[0]);
}

static void phys_flux(const Oracle *o, const double *U, double *f, double *g)
{
    if (o->eq == EQ_BURGERS) {
        f[0] = 0.5 * U[0] * U[0];
        g[0] = 0.5 * U[0] * U[0];
        return;
    }
    double rho = U[0], u = U[1] / rho, v = U[2] / rho, p = euler_p(o->gam, U);
    f[0] = U[1]; f[1] = U[1] * u + p; f[2] = U[2] * u; f[3] = (U[3] + p) * u;
    g[0] = U[2]; g[1] = U[1] * v; g[2] = U[2] * v + p; g[3] = (U[3] + p) * v;
}

/* largest |eigenvalue| of the flux Jacobian in direction n (unit) */
static double wave_speed(const Oracle *o, const double *U, double nx, double ny)
{
    if (o->eq == EQ_BURGERS) return fabs(U[0] * (nx + ny));
    double rho = U[0], un = (U[1] * nx + U[2] * ny) / rho;
    double c = sqrt(o->gam * euler_p(o->gam, U) / rho);
    return fabs(un) + c;
}

/* Local Lax-Friedrichs flux at one point (reading R-flux: the paper's
 * "Lax-Friedrichs" taken pointwise with the local maximum wave speed). */
static void llf_flux(const Oracle *o, const double *UL, const double *UR, double nx, double ny, double *F)
{
    double fL[4], gL[4], fR[4], gR[4];
    phys_flux(o, UL, fL, gL);
    phys_flux(o, UR, fR, gR);
    double aL = wave_speed(o, UL, nx, ny), aR = wave_speed(o, UR, nx, ny);
    double a = aL > aR ? aL : aR;
    for (int v = 0; v < o->nvar; ++v)
        F[v] = 0.5 * ((fL[v] + fR[v]) * nx + (gL[v] + gR[v]) * ny) - 0.5 * a * (UR[v] - UL[v]);
}

/* Ghost state across a boundary face (reading R-bc). */
static void ghost_state(const Oracle *o, int tag, const double *Uin, double x, double y, double nx, double ny, double t, double *Ug)
{
    int kind = o->bkind[tag];
    const double *P = o->bpar[tag];
    int nv = o->nvar;
    if (kind == BC_DIRICHLET) {
        for (int v = 0; v < nv; ++v) Ug[v] = P[v];
    } else if (kind == BC_WALL && o->eq == EQ_EULER) {
        double mn = Uin[1] * nx + Uin[2] * ny;
        Ug[0] = Uin[0];
        Ug[1] = Uin[1] - 2.0 * mn * nx;
        Ug[2] = Uin[2] - 2.0 * mn * ny;
        Ug[3] = Uin[3];
    } else if (kind == BC_SHOCKLINE) {
        /* params: x0, cot, speed, stateA[nv] (x < x0 + y cot + speed t), stateB[nv] */
        double xs = P[0] + y * P[1] + P[2] * t;
        const double *S = (x < xs) ? P + 3 : P + 3 + nv;
        for (int v = 0; v < nv; ++v) Ug[v] = S[v];
    } else {
        for (int v = 0; v < nv; ++v) Ug[v] = Uin[v];
    }
}

/* ======================================================================
 * 5. The semi-discrete operator L_h (Sec. 2, Eq. weakFormScheme2D)
 *
 * Reading R-weak: the printed form is the 1D/structured template with a
 * collocated flux f^_n = f(u^_n); the oracle takes the standard DG weak form
 * on triangles with quadrature,
 *   d u^_i/dt = int_K grad psi_i . F(u_h) dA - sum_faces int_e psi_i F*.n ds,
 * M = I for the physically orthonormal basis (Eq. massMatrix2D).
 * ====================================================================== */

static void face_geom(const Oracle *o, int c, int f, double *ax, double *ay, double *bx, double *by, double *nx, double *ny, double *len)
{
    *ax = o->vx[o->tri[3 * c + f]]; *ay = o->vy[o->tri[3 * c + f]];
    *bx = o->vx[o->tri[3 * c + (f + 1) % 3]]; *by = o->vy[o->tri[3 * c + (f + 1) % 3]];
    double dx = *bx - *ax, dy = *by - *ay;
    *len = sqrt(dx * dx + dy * dy);
    *nx = dy / *len;
    *ny = -dx / *len;
}

/* traces at face point P of cell c, local face f: inside and outside values */
static void face_traces(const Oracle *o, const double *u, int c, int f, double px, double py, double nx, double ny, double t, double *Uin, double *Uout)
{
    Tri tc = cell_tri(o, c, 0, 0);
    eval_cell(o, u, c, &tc, px, py, Uin);
    int n = o->nb[3 * c + f];
    if (n >= 0) {
        Tri tn = cell_tri(o, n, o->sh[2 * (3 * c + f)], o->sh[2 * (3 * c + f) + 1]);
        eval_cell(o, u, n, &tn, px, py, Uout);
    } else {
        ghost_state(o, o->btag[3 * c + f], Uin, px, py, nx, ny, t, Uout);
    }
}

/* L_h for one cell, written straight into L (cell c's block). */
static void rhs_cell(const Oracle *o, const double *u, double t, int c, double *L)
{
    int nv = o->nvar, np = o->np;
    Tri tc = cell_tri(o, c, 0, 0);
    double area = tri_area(&tc);
    for (int i = 0; i < nv * np; ++i) L[i] = 0.0;
    /* volume integral: int_K (dpsi_i/dx f + dpsi_i/dy g) dA */
    for (int q = 0; q < o->vol.n; ++q) {
        double x, y, U[4], f[4], g[4];
        tri_point(&tc, o->vol.b[q], &x, &y);
        eval_cell(o, u, c, &tc, x, y, U);
        phys_flux(o, U, f, g);
        for (int i = 0; i < np; ++i) {
            double gx, gy;
            psi_phys(o, &tc, i, x, y, NULL, &gx, &gy);
            for (int v = 0; v < nv; ++v) L[v * np + i] += area * o->vol.w[q] * (gx * f[v] + gy * g[v]);
        }
    }
    /* surface integrals with the local Lax-Friedrichs flux */
    for (int f = 0; f < 3; ++f) {
        double ax, ay, bx, by, nx, ny, len;
        face_geom(o, c, f, &ax, &ay, &bx, &by, &nx, &ny, &len);
        for (int g = 0; g < o->nfq; ++g) {
            double px = ax + o->fx[g] * (bx - ax), py = ay + o->fx[g] * (by - ay);
            double Uin[4], Uout[4], F[4];
            face_traces(o, u, c, f, px, py, nx, ny, t, Uin, Uout);
            /* reading R-bc: across a transmissive face the outside state of the flux is
             * the cell mean (zero-gradient extrapolation of the cell average); the
             * interior trace itself would leave the flux F(u-) without dissipation */
            if (o->nb[3 * c + f] < 0 && o->bkind[o->btag[3 * c + f]] == BC_TRANSMISSIVE)
                for (int v = 0; v < nv; ++v) Uout[v] = u[(size_t)(c * nv + v) * np] / sqrt(area);
            llf_flux(o, Uin, Uout, nx, ny, F);
            for (int i = 0; i < np; ++i) {
                double p;
                psi_phys(o, &tc, i, px, py, &p, NULL, NULL);
                for (int v = 0; v < nv; ++v) L[v * np + i] -= o->fw[g] * len * p * F[v];
            }
        }
    }
}

void or_rhs(const Oracle *o, const double *u, double t, double *L)
{
    #pragma omp parallel for schedule(dynamic, 64)
    for (int c = 0; c < o->nc; ++c) rhs_cell(o, u, t, c, L + (size_t)c * o->nvar * o->np);
}

void or_rhs_cells(const Oracle *o, const double *u, double t, int n, const int *cells, double *L)
{
    for (int i = 0; i < n; ++i) rhs_cell(o, u, t, cells[i], L + (size_t)i * o->nvar * o->np);
}

/* ======================================================================
 * 6. KXRCF troubled-cell indicator (Sec. 3.1, Eq. troubledCellIndicator)
 *
 * Readings R-kxrcf: inflow faces are those with vbar.n < 0, vbar from the
 * cell mean ((f'(u), g'(u)) = (u,u) for Burgers, the velocity for Euler);
 * the indicator variable is u (Burgers) or the density (Euler); ||U_j|| is
 * the L2 norm over the cell taken with respect to the cell's normalised
 * measure, (|K|^{-1} int_K U^2)^{1/2} = sqrt(sum_m u_m^2 / |K|) in the
 * orthonormal basis.  The un-normalised norm carries a factor |K|^{1/2} ~ h,
 * so R would not vanish on smooth P1 data (numerator O(h^{k+2}), denominator
 * O(h^{(k+1)/2} h h)) and the fixed threshold C_K = 1 of the cited KXRCF
 * indicator would flag smooth cells at every resolution; with the normalised
 * norm R = O(h^{(k+1)/2}) on smooth data and O(h^{-(k+1)/2}) at a jump, as
 * the indicator is designed.  h is the circumradius; no inflow face gives
 * R = 0; ||U_j|| = 0 flags the cell only if the jump integral is non-zero;
 * troubled iff R > C_K.
 * ====================================================================== */

static double circumradius(const Tri *t)
{
    double a = hypot(t->x[1] - t->x[0], t->y[1] - t->y[0]);
    double b = hypot(t->x[2] - t->x[1], t->y[2] - t->y[1]);
    double c = hypot(t->x[0] - t->x[2], t->y[0] - t->y[2]);
    return a * b * c / (4.0 * tri_area(t));
}

/* Reading R-pos (the paper states no positivity treatment): 1 if the Euler
 * polynomial with modes m[v*np + i] on cell c has a non-positive density or
 * pressure at one of the volume-rule points or the face Gauss points. */
static int nonphysical_points(const Oracle *o, int c, const double *m)
{
    int np = o->np;
    Tri tc = cell_tri(o, c, 0, 0);
    for (int q = 0; q < o->vol.n + 3 * o->nfq; ++q) {
        double x, y, U[4] = {0.0, 0.0, 0.0, 0.0};
        if (q < o->vol.n) {
            tri_point(&tc, o->vol.b[q], &x, &y);
        } else {
            int f = (q - o->vol.n) / o->nfq, g = (q - o->vol.n) % o->nfq;
            double ax, ay, bx, by, nx, ny, len;
            face_geom(o, c, f, &ax, &ay, &bx, &by, &nx, &ny, &len);
            x = ax + o->fx[g] * (bx - ax);
            y = ay + o->fx[g] * (by - ay);
        }
        for (int i = 0; i < np; ++i) {
            double pm;
            psi_phys(o, &tc, i, x, y, &pm, NULL, NULL);
            for (int v = 0; v < 4; ++v) U[v] += m[v * np + i] * pm;
        }
        if (!(U[0] > 0.0 && euler_p(o->gam, U) > 0.0)) return 1;
    }
    return 0;
}

static int detect_cell(const Oracle *o, const double *u, double t, int c, double *Rout)
{
    int nv = o->nvar, np = o->np;
    Tri tc = cell_tri(o, c, 0, 0);
    double area = tri_area(&tc);
    double sq = sqrt(area);
    double vx, vy;
    if (o->eq == EQ_BURGERS) {
        double ub = u[(size_t)c * nv * np] / sq;
        vx = ub; vy = ub;
    } else {
        double r = u[(size_t)(c * nv + 0) * np] / sq, mx = u[(size_t)(c * nv + 1) * np] / sq, my = u[(size_t)(c * nv + 2) * np] / sq;
        vx = mx / r; vy = my / r;
    }
    double jump = 0.0, inlen = 0.0;
    for (int f = 0; f < 3; ++f) {
        double ax, ay, bx, by, nx, ny, len;
        face_geom(o, c, f, &ax, &ay, &bx, &by, &nx, &ny, &len);
        if (!(vx * nx + vy * ny < 0.0)) continue;
        inlen += len;
        for (int g = 0; g < o->nfq; ++g) {
            double px = ax + o->fx[g] * (bx - ax), py = ay + o->fx[g] * (by - ay);
            double Uin[4], Uout[4];
            face_traces(o, u, c, f, px, py, nx, ny, t, Uin, Uout);
            jump += o->fw[g] * len * (Uin[0] - Uout[0]);
        }
    }
    double nrm = 0.0;
    for (int m = 0; m < np; ++m) {
        double a = u[(size_t)(c * nv + 0) * np + m];
        nrm += a * a;
    }
    nrm = sqrt(nrm / area);
    double h = circumradius(&tc);
    double hp = (o->k == 1) ? h : h * sqrt(h); /* h^{(k+1)/2} */
    double R;
    if (inlen == 0.0) R = 0.0;
    else if (nrm == 0.0) R = (fabs(jump) > 0.0) ? INFINITY : 0.0;
    else R = fabs(jump) / (hp * inlen * nrm);
    if (Rout) *Rout = R;
    /* Reading R-pos: a cell whose polynomial is non-physical at a quadrature
     * point is troubled whatever its indicator (the operator would take the
     * sound speed of a non-positive pressure there) */
    if (o->eq == EQ_EULER && nonphysical_points(o, c, u + (size_t)c * nv * np)) return 1;
    return R > o->ck;
}

void or_detect(const Oracle *o, const double *u, double t, unsigned char *flags, double *R)
{
    #pragma omp parallel for schedule(dynamic, 64)
    for (int c = 0; c < o->nc; ++c) flags[c] = (unsigned char)detect_cell(o, u, t, c, R ? R + c : NULL);
}

/* ======================================================================
 * 7. CSWENO reconstruction of one troubled cell (Sec. 3.2)
 * ====================================================================== */

/* Stencil geometry of cell c.  For each local face f the neighbour (or, on a
 * non-periodic boundary, the mirror image of the cell across the face -- reading
 * R-ghost) is split into subcells (Sec. 3.2, Fig. NeighborP1/NeighborP2, whose
 * drawings are missing; reading R-split):
 *   third 1 = (centroid, shared edge)          -> Delta_{i1}
 *   third 2 = (centroid, next edge CCW)        -> Delta_{i2}
 *   third 3 = (centroid, last edge)            -> Delta_{i3}
 *   P2: thirds 2 and 3 are halved by the segment from the centroid to the foot of
 *   the perpendicular on their outer edge (edge midpoint if the foot is not
 *   inside [0.05,0.95] of the edge); the half touching third 1 keeps the name
 *   Delta_{i2} (Delta_{i3}), the other is Delta_{i21} (Delta_{i31}).
 */
typedef struct {
    Tri nbr[3];        /* neighbour or ghost triangle, placed next to the cell */
    int ghost[3];      /* 1 if mirror image across a boundary face */
    Tri third[3][3];   /* [face][1..3] */
    Tri half[3][4];    /* [face]: i2 (half near i1), i21, i3 (half near i1), i31 */
} Stencil;

static Tri make_tri(double x0, double y0, double x1, double y1, double x2, double y2)
{
    Tri t;
    t.x[0] = x0; t.y[0] = y0; t.x[1] = x1; t.y[1] = y1; t.x[2] = x2; t.y[2] = y2;
    return t;
}

static void foot(double cx, double cy, double ax, double ay, double bx, double by, double *fx, double *fy)
{
    double ex = bx - ax, ey = by - ay;
    double tt = ((cx - ax) * ex + (cy - ay) * ey) / (ex * ex + ey * ey);
    if (!(tt >= 0.05 && tt <= 0.95)) tt = 0.5;
    *fx = ax + tt * ex;
    *fy = ay + tt * ey;
}

static void build_stencil(const Oracle *o, int c, Stencil *S)
{
    Tri tc = cell_tri(o, c, 0, 0);
    for (int f = 0; f < 3; ++f) {
        int n = o->nb[3 * c + f];
        double X[3], Y[3]; /* neighbour vertices ordered so that edge 0 is the shared edge */
        if (n >= 0) {
            Tri tn = cell_tri(o, n, o->sh[2 * (3 * c + f)], o->sh[2 * (3 * c + f) + 1]);
            int g = o->nbf[3 * c + f];
            for (int i = 0; i < 3; ++i) { X[i] = tn.x[(g + i) % 3]; Y[i] = tn.y[(g + i) % 3]; }
            S->nbr[f] = tn;
            S->ghost[f] = 0;
        } else {
            /* mirror of the cell across face f, counter-clockwise */
            double ax = tc.x[f], ay = tc.y[f], bx = tc.x[(f + 1) % 3], by = tc.y[(f + 1) % 3];
            double px = tc.x[(f + 2) % 3], py = tc.y[(f + 2) % 3];
            double ex = bx - ax, ey = by - ay;
            double tt = ((px - ax) * ex + (py - ay) * ey) / (ex * ex + ey * ey);
            double qx = ax + tt * ex, qy = ay + tt * ey;
            double mx = 2.0 * qx - px, my = 2.0 * qy - py;
            X[0] = bx; Y[0] = by; X[1] = ax; Y[1] = ay; X[2] = mx; Y[2] = my;
            S->nbr[f] = make_tri(X[0], Y[0], X[1], Y[1], X[2], Y[2]);
            S->ghost[f] = 1;
        }
        double cx = (X[0] + X[1] + X[2]) / 3.0, cy = (Y[0] + Y[1] + Y[2]) / 3.0;
        S->third[f][0] = make_tri(cx, cy, X[0], Y[0], X[1], Y[1]);
        S->third[f][1] = make_tri(cx, cy, X[1], Y[1], X[2], Y[2]);
        S->third[f][2] = make_tri(cx, cy, X[2], Y[2], X[0], Y[0]);
        double f2x, f2y, f3x, f3y;
        foot(cx, cy, X[1], Y[1], X[2], Y[2], &f2x, &f2y);
        foot(cx, cy, X[2], Y[2], X[0], Y[0], &f3x, &f3y);
        S->half[f][0] = make_tri(cx, cy, X[1], Y[1], f2x, f2y); /* Delta_{i2}  */
        S->half[f][1] = make_tri(cx, cy, f2x, f2y, X[2], Y[2]); /* Delta_{i21} */
        S->half[f][2] = make_tri(cx, cy, f3x, f3y, X[0], Y[0]); /* Delta_{i3}  */
        S->half[f][3] = make_tri(cx, cy, X[2], Y[2], f3x, f3y); /* Delta_{i31} */
    }
}

/* Mirror a point across the line of face f of cell c. */
static void mirror_point(const Tri *tc, int f, double x, double y, double *mx, double *my)
{
    double ax = tc->x[f], ay = tc->y[f], bx = tc->x[(f + 1) % 3], by = tc->y[(f + 1) % 3];
    double ex = bx - ax, ey = by - ay;
    double tt = ((x - ax) * ex + (y - ay) * ey) / (ex * ex + ey * ey);
    double qx = ax + tt * ex, qy = ay + tt * ey;
    *mx = 2.0 * qx - x;
    *my = 2.0 * qy - y;
}

/* Value of the neighbour function across face f at a point of the stencil:
 * the neighbour's DG polynomial, or on a boundary the ghost function
 * g(x) = B(u_c(mirror(x))) (reading R-ghost). */
static void stencil_value(const Oracle *o, const double *u, int c, int f, double t, double x, double y, double *U)
{
    int n = o->nb[3 * c + f];
    if (n >= 0) {
        Tri tn = cell_tri(o, n, o->sh[2 * (3 * c + f)], o->sh[2 * (3 * c + f) + 1]);
        eval_cell(o, u, n, &tn, x, y, U);
        return;
    }
    Tri tc = cell_tri(o, c, 0, 0);
    double mx, my, Uin[4], ax, ay, bx, by, nx, ny, len;
    mirror_point(&tc, f, x, y, &mx, &my);
    eval_cell(o, u, c, &tc, mx, my, Uin);
    face_geom(o, c, f, &ax, &ay, &bx, &by, &nx, &ny, &len);
    int tag = o->btag[3 * c + f];
    if (o->bkind[tag] == BC_SHOCKLINE) {
        /* constant ghost chosen at the face midpoint */
        ghost_state(o, tag, Uin, 0.5 * (ax + bx), 0.5 * (ay + by), nx, ny, t, U);
    } else {
        ghost_state(o, tag, Uin, x, y, nx, ny, t, U);
    }
}

/* mean over triangle T of the stencil function (exact: degree <= k) */
static void stencil_mean(const Oracle *o, const double *u, int c, int f, double t, const Tri *T, double *mean)
{
    int nv = o->nvar;
    for (int v = 0; v < nv; ++v) mean[v] = 0.0;
    for (int q = 0; q < o->duf3.n; ++q) {
        double x, y, U[4];
        tri_point(T, o->duf3.b[q], &x, &y);
        stencil_value(o, u, c, f, t, x, y, U);
        for (int v = 0; v < nv; ++v) mean[v] += o->duf3.w[q] * U[v];
    }
}

/* Monomials m_j(xi, eta), degree-graded without the constant:
 * xi, eta, xi^2, xi eta, eta^2, xi^3, ..., eta^4 (14 for degree 4). */
static int n_mono(int deg) { return (deg + 1) * (deg + 2) / 2 - 1; }

static void mono_exp(int j, int *a, int *b)
{
    int idx = 0;
    *a = *b = 0;
    for (int d = 1; d <= 8; ++d)
        for (int e = 0; e <= d; ++e) {
            if (idx == j) { *a = d - e; *b = e; return; }
            ++idx;
        }
}

static double ipow(double x, int n) { double r = 1.0; for (int i = 0; i < n; ++i) r *= x; return r; }

/* d^{p+q} / dxi^p deta^q of xi^a eta^b */
static double mono_deriv(int a, int b, int p, int q, double xi, double eta)
{
    if (p > a || q > b) return 0.0;
    double ca = 1.0, cb = 1.0;
    for (int i = 0; i < p; ++i) ca *= (a - i);
    for (int i = 0; i < q; ++i) cb *= (b - i);
    return ca * cb * ipow(xi, a - p) * ipow(eta, b - q);
}

typedef struct {
    double x0, y0, h0;    /* centroid and sqrt(area) of Delta_0 */
    double area, hbar;    /* area and mean side length of Delta_0 */
    Tri t0;
    double m0[14];        /* means of the monomials over Delta_0 */
} Frame;

static double mono_mean(const Frame *F, const Tri *T, int j, const trirule *R)
{
    int a, b;
    mono_exp(j, &a, &b);
    double s = 0.0;
    for (int q = 0; q < R->n; ++q) {
        double x, y;
        tri_point(T, R->b[q], &x, &y);
        s += R->w[q] * ipow((x - F->x0) / F->h0, a) * ipow((y - F->y0) / F->h0, b);
    }
    return s;
}

/* Constrained least squares of Sec. 3.2 Step 1 (reading R-lsq): q(x,y) =
 * ubar0 + sum_j c_j (m_j - mean_{Delta0} m_j) keeps the mean on Delta_0 and
 * fits the means on the other stencil cells in the unweighted least-squares
 * sense.  rows: list of stencil triangles, data: their means. */
static int lsq_poly(const Frame *F, const trirule *R, int deg, int nrows, const Tri *rows, const double *data, double ubar0, double *coef)
{
    int nm = n_mono(deg);
    double A[32 * 16], b[32];
    for (int r = 0; r < nrows; ++r) {
        for (int j = 0; j < nm; ++j) A[r * nm + j] = mono_mean(F, &rows[r], j, R) - F->m0[j];
        b[r] = data[r] - ubar0;
    }
    return lsq_qr(nrows, nm, A, b, coef);
}

/* value of ubar0 + sum_j c_j (m_j - m0_j) at a physical point */
static double poly_val(const Frame *F, int nm, const double *coef, double ubar0, double x, double y)
{
    double xi = (x - F->x0) / F->h0, eta = (y - F->y0) / F->h0, s = ubar0;
    for (int j = 0; j < nm; ++j) {
        int a, b;
        mono_exp(j, &a, &b);
        s += coef[j] * (ipow(xi, a) * ipow(eta, b) - F->m0[j]);
    }
    return s;
}

/* Smoothness indicator, Sec. 3.2 Step 3, Eq. smoothnessIndicator (reading
 * R-beta: the sum runs over multi-indices 1 <= |alpha| <= degree of p, each
 * d^{|alpha|}/dx^{a1} dy^{a2} once), evaluated literally in physical
 * coordinates with an exact rule on Delta_0. */
static double beta_poly(const Frame *F, const trirule *R, int nm, const double *coef, int deg)
{
    double beta = 0.0;
    for (int s = 1; s <= deg; ++s) {
        for (int q = 0; q <= s; ++q) {
            int p = s - q;
            double integral = 0.0;
            for (int k = 0; k < R->n; ++k) {
                double x, y;
                tri_point(&F->t0, R->b[k], &x, &y);
                double xi = (x - F->x0) / F->h0, eta = (y - F->y0) / F->h0;
                double d = 0.0;
                for (int j = 0; j < nm; ++j) {
                    int a, b;
                    mono_exp(j, &a, &b);
                    d += coef[j] * mono_deriv(a, b, p, q, xi, eta);
                }
                d /= ipow(F->h0, s); /* chain rule: d/dx = (1/h0) d/dxi */
                integral += F->area * R->w[k] * d * d;
            }
            beta += pow(F->area, s - 1) * integral;
        }
    }
    return beta;
}

typedef struct {
    double q2[2], q3[5], q4[9];   /* least-squares coefficients */
    double gam[5];                /* linear weights of the final combination */
    double beta[4], omega[4];
    double beta1l[3], sigma[3], tau; /* beta_{1,l}, sigma_l (Eq. sigmaEqn) and tau */
    int nslot;
    double modes[OR_MAXNP];       /* reconstructed modes 1..np-1 (mode 0 untouched) */
    int status;
} WenoOut;

#define OR_EPS 1e-10

/* One scalar field on one troubled cell: Sec. 3.2 Steps 1-5 (P1) and
 * Steps 1-4 + Eq. finalMoments (P2).  Inputs: ubar0 (mean on Delta_0), the
 * thirds' means th[f][0..2] and (P2) the halves' means hf[f][0..3].
 * force_linear != 0 replaces the nonlinear weights by the linear ones. */
static void weno_scalar(const Oracle *o, const Frame *F, const Stencil *S, double ubar0,
                        double th[3][3], double hf[3][4], int force_linear, WenoOut *W)
{
    int k = o->k;
    memset(W, 0, sizeof(*W));
    /* Step 1: q1 = ubar0, q2 on T2, q3 on T3 (and P2: the cubic q4 on T4,
     * reading R-p2: the quartic of the printed Step 1 made the every-cell
     * limited P2 scheme unstable, so the top polynomial is the cubic
     * least-squares fit on the same 16-cell stencil T4) */
    Tri rows[16];
    double data[16];
    for (int f = 0; f < 3; ++f) { rows[f] = S->third[f][0]; data[f] = th[f][0]; }
    if (lsq_poly(F, &o->duf3, 1, 3, rows, data, ubar0, W->q2)) W->status = -1;
    for (int f = 0; f < 3; ++f) {
        rows[3 + 2 * f] = S->third[f][1]; data[3 + 2 * f] = th[f][1];
        rows[4 + 2 * f] = S->third[f][2]; data[4 + 2 * f] = th[f][2];
    }
    if (lsq_poly(F, &o->duf3, 2, 9, rows, data, ubar0, W->q3)) W->status = -1;
    if (k == 2) {
        for (int f = 0; f < 3; ++f) {
            rows[3 + 4 * f + 0] = S->half[f][0]; data[3 + 4 * f + 0] = hf[f][0];
            rows[3 + 4 * f + 1] = S->half[f][1]; data[3 + 4 * f + 1] = hf[f][1];
            rows[3 + 4 * f + 2] = S->half[f][2]; data[3 + 4 * f + 2] = hf[f][2];
            rows[3 + 4 * f + 3] = S->half[f][3]; data[3 + 4 * f + 3] = hf[f][3];
        }
        if (lsq_poly(F, &o->duf3, 3, 15, rows, data, ubar0, W->q4)) W->status = -1;
    }
    /* Step 2: linear weights gamma_{l,m} = (1/h)^{l-1} normalised (h = mean
     * side length of Delta_0), and the hierarchical p_l (Eqs. equivalentOrder0-2;
     * for P2 Eq. equivalentOrder4's four weights gamma_{l,5}, l = 1..4, applied
     * to the top polynomial, reading R-p2). p_l = ubar0 + sum c(p_l)_j phi_j. */
    double h = F->hbar;
    double g2[2], g3[3], g5[4], s;
    s = 1.0 + 1.0 / h; g2[0] = 1.0 / s; g2[1] = (1.0 / h) / s;
    s = 1.0 + 1.0 / h + 1.0 / (h * h); g3[0] = 1.0 / s; g3[1] = (1.0 / h) / s; g3[2] = (1.0 / (h * h)) / s;
    s = 1.0 + 1.0 / h + 1.0 / (h * h) + 1.0 / (h * h * h);
    g5[0] = 1.0 / s; g5[1] = (1.0 / h) / s; g5[2] = (1.0 / (h * h)) / s; g5[3] = (1.0 / (h * h * h)) / s;
    double p2[14] = {0}, p3[14] = {0}, p4[14] = {0};
    for (int j = 0; j < 2; ++j) p2[j] = W->q2[j] / g2[1];
    for (int j = 0; j < 5; ++j) p3[j] = (W->q3[j] - g3[1] * p2[j]) / g3[2];
    if (k == 2)
        for (int j = 0; j < 9; ++j) p4[j] = (W->q4[j] - g5[1] * p2[j] - g5[2] * p3[j]) / g5[3];
    int nslot = (k == 1) ? 3 : 4;
    W->nslot = nslot;
    const double *gl = (k == 1) ? g3 : g5;
    for (int l = 0; l < nslot; ++l) W->gam[l] = gl[l];
    /* Step 3: smoothness indicators; beta_1 magnified (Eqs. sigmaEqn, smoothnessIndicatorT1) */
    double b11[3], al[3], bl[3];
    for (int f = 0; f < 3; ++f) {
        /* p_{1,l} = a (x - x_{l1}) + b (y - y_{l1}) through the centroids of the thirds */
        double cx[3], cy[3];
        for (int i = 0; i < 3; ++i) {
            cx[i] = (S->third[f][i].x[0] + S->third[f][i].x[1] + S->third[f][i].x[2]) / 3.0;
            cy[i] = (S->third[f][i].y[0] + S->third[f][i].y[1] + S->third[f][i].y[2]) / 3.0;
        }
        double m11 = cx[1] - cx[0], m12 = cy[1] - cy[0], m21 = cx[2] - cx[0], m22 = cy[2] - cy[0];
        double r1 = th[f][1] - th[f][0], r2 = th[f][2] - th[f][0];
        double det = m11 * m22 - m12 * m21;
        al[f] = (r1 * m22 - m12 * r2) / det;
        bl[f] = (m11 * r2 - m21 * r1) / det;
        b11[f] = F->area * (al[f] * al[f] + bl[f] * bl[f]);
    }
    /* Eq. sigmaEqn (reading R-sigma): the printed numerator squares each
     * difference inside an already squared mean; taken as the [zs4] form the
     * paper cites for this magnification, the square of the mean absolute
     * difference, sigma_l = (1/3) (1 + D^2 / (beta_{1,l} + eps)),
     * D = (|b11 - b12| + |b12 - b13| + |b13 - b11|) / 3. */
    double D = (fabs(b11[0] - b11[1]) + fabs(b11[1] - b11[2]) + fabs(b11[2] - b11[0])) / 3.0;
    double sig[3], sigsum = 0.0;
    for (int f = 0; f < 3; ++f) { sig[f] = (1.0 / 3.0) * (1.0 + D * D / (b11[f] + OR_EPS)); sigsum += sig[f]; }
    for (int f = 0; f < 3; ++f) { W->beta1l[f] = b11[f]; W->sigma[f] = sig[f]; }
    double abar = 0.0, bbar = 0.0;
    for (int f = 0; f < 3; ++f) { abar += sig[f] / sigsum * al[f]; bbar += sig[f] / sigsum * bl[f]; }
    W->beta[0] = F->area * (abar * abar + bbar * bbar);
    W->beta[1] = beta_poly(F, &o->duf4, 2, p2, 1);
    W->beta[2] = beta_poly(F, &o->duf4, 5, p3, 2);
    if (k == 2) W->beta[3] = beta_poly(F, &o->duf4, 9, p4, 3);
    /* Step 4: tau and nonlinear weights (Eqs. tauNonlinearWeightsP1/P2,
     * nonLinearWeightsP1/P2), reading R-weno: the paper takes these weights
     * from the WENO-Z recipe of [ccd], whose tau is built from absolute
     * differences of the smoothness indicators (linear in beta, so tau/beta
     * does not change when the data are scaled) and whose ratio tau/(eps+beta)
     * carries a power p.  tau is the mean absolute difference between the top
     * slot's beta and the others', and p = k + 1: with the paper's linear
     * weights gamma_{l,m} = O(h^{m-l}) this is the smallest power for which a
     * non-smooth top stencil drops out to O(h^{k+1}) against a smooth T1
     * (omega_top ~ h^{2p-(k+1)}), the order reduction Step 4 states. */
    double tau;
    if (k == 1) tau = (fabs(W->beta[2] - W->beta[0]) + fabs(W->beta[2] - W->beta[1])) / 2.0;
    else tau = (fabs(W->beta[3] - W->beta[0]) + fabs(W->beta[3] - W->beta[1]) + fabs(W->beta[3] - W->beta[2])) / 3.0;
    W->tau = tau;
    double wsum = 0.0, wb[4];
    for (int l = 0; l < nslot; ++l) {
        double r = tau / (OR_EPS + W->beta[l]), rp = r;
        for (int e = 1; e < k + 1; ++e) rp *= r; /* (tau / (eps + beta_l))^{k+1} */
        wb[l] = W->gam[l] * (1.0 + rp);
        wsum += wb[l];
    }
    for (int l = 0; l < nslot; ++l) W->omega[l] = force_linear ? W->gam[l] : wb[l] / wsum;
    /* Eq. WENOApprox...: u_q = sum_l omega_l p_l(x_q) at the reconstruction points */
    double zero[14] = {0};
    double uq[OR_MAXQ];
    for (int q = 0; q < o->scp.n; ++q) {
        double x, y;
        tri_point(&F->t0, o->scp.b[q], &x, &y);
        uq[q] = W->omega[0] * poly_val(F, 14, zero, ubar0, x, y);
        uq[q] += W->omega[1] * poly_val(F, 2, p2, ubar0, x, y);
        uq[q] += W->omega[2] * poly_val(F, 5, p3, ubar0, x, y);
        if (k == 2) uq[q] += W->omega[3] * poly_val(F, 9, p4, ubar0, x, y);
    }
    /* Step 5, Eq. finalMoments: u_i = |Delta_0| sum_q w_q u_q psi_i(x_q), i >= 1 */
    for (int i = 1; i < o->np; ++i) {
        double acc = 0.0;
        for (int q = 0; q < o->scp.n; ++q) {
            double x, y, p;
            tri_point(&F->t0, o->scp.b[q], &x, &y);
            psi_phys(o, &F->t0, i, x, y, &p, NULL, NULL);
            acc += o->scp.w[q] * uq[q] * p;
        }
        W->modes[i] = F->area * acc;
    }
}

static void make_frame(const Oracle *o, int c, Frame *F)
{
    F->t0 = cell_tri(o, c, 0, 0);
    F->area = tri_area(&F->t0);
    F->h0 = sqrt(F->area);
    F->x0 = (F->t0.x[0] + F->t0.x[1] + F->t0.x[2]) / 3.0;
    F->y0 = (F->t0.y[0] + F->t0.y[1] + F->t0.y[2]) / 3.0;
    F->hbar = (hypot(F->t0.x[1] - F->t0.x[0], F->t0.y[1] - F->t0.y[0]) + hypot(F->t0.x[2] - F->t0.x[1], F->t0.y[2] - F->t0.y[1]) +
               hypot(F->t0.x[0] - F->t0.x[2], F->t0.y[0] - F->t0.y[2])) / 3.0;
    for (int j = 0; j < 14; ++j) F->m0[j] = mono_mean(F, &F->t0, j, &o->duf3);
}

/* Right/left eigenvectors of the Euler flux Jacobian in direction (nx, ny)
 * at state U (closed forms for the ideal gas; reading R-char: characteristic
 * decomposition in x and in y separately, results averaged). R is column-major
 * by eigenvector: R[row*4+col]; L rows are the left eigenvectors. */
void or_euler_eigen(double gam, const double *U, double nx, double ny, double *R, double *L)
{
    double rho = U[0], u = U[1] / rho, v = U[2] / rho;
    double p = (gam - 1.0) * (U[3] - 0.5 * rho * (u * u + v * v));
    double c2 = gam * p / rho, c = sqrt(c2);
    double H = (U[3] + p) / rho, q2 = u * u + v * v, un = u * nx + v * ny, ut = -u * ny + v * nx;
    double b = gam - 1.0;
    double Rc[4][4] = {{1.0, u - c * nx, v - c * ny, H - c * un},
                       {1.0, u, v, 0.5 * q2},
                       {0.0, -ny, nx, ut},
                       {1.0, u + c * nx, v + c * ny, H + c * un}};
    for (int col = 0; col < 4; ++col)
        for (int row = 0; row < 4; ++row) R[row * 4 + col] = Rc[col][row];
    double Lr[4][4] = {{(0.5 * b * q2 + c * un) / (2.0 * c2), -(b * u + c * nx) / (2.0 * c2), -(b * v + c * ny) / (2.0 * c2), b / (2.0 * c2)},
                       {1.0 - b * q2 / (2.0 * c2), b * u / c2, b * v / c2, -b / c2},
                       {-ut, -ny, nx, 0.0},
                       {(0.5 * b * q2 - c * un) / (2.0 * c2), -(b * u - c * nx) / (2.0 * c2), -(b * v - c * ny) / (2.0 * c2), b / (2.0 * c2)}};
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) L[i * 4 + j] = Lr[i][j];
}

/* Limit cell c: reads the unlimited state u, writes the new modes of c into out
 * (nvar*np values; mode 0 of every variable is kept, Sec. 3.2). */
static int limit_cell_w(const Oracle *o, const double *u, double t, int c, double *out, int force_linear)
{
    int nv = o->nvar, np = o->np, k = o->k;
    Stencil S;
    Frame F;
    build_stencil(o, c, &S);
    make_frame(o, c, &F);
    /* subcell means of the neighbours' polynomials in conserved variables */
    double th[3][3][4], hf[3][4][4];
    for (int f = 0; f < 3; ++f) {
        for (int i = 0; i < 3; ++i) stencil_mean(o, u, c, f, t, &S.third[f][i], th[f][i]);
        if (k == 2)
            for (int i = 0; i < 4; ++i) stencil_mean(o, u, c, f, t, &S.half[f][i], hf[f][i]);
    }
    double ub[4];
    for (int v = 0; v < nv; ++v) ub[v] = u[(size_t)(c * nv + v) * np] / sqrt(F.area);
    for (int i = 0; i < nv * np; ++i) out[i] = u[(size_t)c * nv * np + i];
    int status = 0;
    if (o->eq == EQ_BURGERS) {
        double t1[3][3], h1[3][4];
        for (int f = 0; f < 3; ++f) {
            for (int i = 0; i < 3; ++i) t1[f][i] = th[f][i][0];
            for (int i = 0; i < 4; ++i) h1[f][i] = (k == 2) ? hf[f][i][0] : 0.0;
        }
        WenoOut W;
        weno_scalar(o, &F, &S, ub[0], t1, h1, force_linear, &W);
        for (int i = 1; i < np; ++i) out[i] = W.modes[i];
        return W.status;
    }
    /* Euler: local characteristic fields in x and in y (Sec. 3.2, last paragraph) */
    double acc[4][OR_MAXNP];
    for (int v = 0; v < 4; ++v)
        for (int i = 0; i < np; ++i) acc[v][i] = 0.0;
    for (int d = 0; d < 2; ++d) {
        double R[16], L[16];
        or_euler_eigen(o->gam, ub, d == 0 ? 1.0 : 0.0, d == 0 ? 0.0 : 1.0, R, L);
        double wmodes[4][OR_MAXNP];
        for (int fld = 0; fld < 4; ++fld) {
            double t1[3][3], h1[3][4], w0 = 0.0;
            for (int j = 0; j < 4; ++j) w0 += L[fld * 4 + j] * ub[j];
            for (int f = 0; f < 3; ++f) {
                for (int i = 0; i < 3; ++i) { t1[f][i] = 0.0; for (int j = 0; j < 4; ++j) t1[f][i] += L[fld * 4 + j] * th[f][i][j]; }
                for (int i = 0; i < 4; ++i) { h1[f][i] = 0.0; if (k == 2) for (int j = 0; j < 4; ++j) h1[f][i] += L[fld * 4 + j] * hf[f][i][j]; }
            }
            WenoOut W;
            weno_scalar(o, &F, &S, w0, t1, h1, force_linear, &W);
            if (W.status) status = W.status;
            for (int i = 1; i < np; ++i) wmodes[fld][i] = W.modes[i];
        }
        for (int v = 0; v < 4; ++v)
            for (int i = 1; i < np; ++i) {
                double s = 0.0;
                for (int fld = 0; fld < 4; ++fld) s += R[v * 4 + fld] * wmodes[fld][i];
                acc[v][i] += 0.5 * s;
            }
    }
    for (int v = 0; v < 4; ++v)
        for (int i = 1; i < np; ++i) out[v * np + i] = acc[v][i];
    /* Reading R-pos (the paper states no positivity treatment): if the
     * reconstructed polynomial has a non-positive density or pressure at a
     * volume-rule point or a face Gauss point of the cell, the cell keeps
     * only its mean. */
    if (nonphysical_points(o, c, out))
        for (int v = 0; v < 4; ++v)
            for (int i = 1; i < np; ++i) out[v * np + i] = 0.0;
    return status;
}

static int limit_cell(const Oracle *o, const double *u, double t, int c, double *out)
{
    return limit_cell_w(o, u, t, c, out, 0);
}

/* Limiter pass: flags (LIM_KXRCF: detected here; LIM_ALL: every cell), then
 * every flagged cell is rebuilt from the unlimited state u_in. */
int or_limit(const Oracle *o, const double *u_in, double t, double *u_out, unsigned char *flags)
{
    size_t n = (size_t)o->nc * o->nvar * o->np;
    memcpy(u_out, u_in, sizeof(double) * n);
    int status = 0;
    #pragma omp parallel for schedule(dynamic, 16) reduction(min : status)
    for (int c = 0; c < o->nc; ++c) {
        int fl = 0;
        if (o->limiter == LIM_ALL) fl = 1;
        else if (o->limiter == LIM_KXRCF) fl = detect_cell(o, u_in, t, c, NULL);
        if (flags) flags[c] = (unsigned char)fl;
        if (fl) {
            int s = limit_cell(o, u_in, t, c, u_out + (size_t)c * o->nvar * o->np);
            if (s) status = s;
        }
    }
    return status;
}

/* Limited modes of a list of cells (for sampled comparisons at full size). */
int or_limit_cells(const Oracle *o, const double *u_in, double t, int n, const int *cells, double *out)
{
    int status = 0;
    for (int i = 0; i < n; ++i) {
        int s = limit_cell(o, u_in, t, cells[i], out + (size_t)i * o->nvar * o->np);
        if (s) status = s;
    }
    return status;
}

void or_detect_cells(const Oracle *o, const double *u, double t, int n, const int *cells, unsigned char *flags, double *R)
{
    for (int i = 0; i < n; ++i) flags[i] = (unsigned char)detect_cell(o, u, t, cells[i], R ? R + i : NULL);
}

/* ======================================================================
 * 8. Time stepping: SSP-RK3 (Eq. timeIntegrate, Table tvd) with the
 *    limiter after every stage; time step from the CFL rule (reading R-cfl:
 *    the paper gives none; dt = CFL * min_K r_K / max_K lambda_K with r_K the
 *    inradius and lambda_K the largest wave speed of the cell mean).
 * ====================================================================== */

double or_cfl_dt(const Oracle *o, const double *u, double cfl)
{
    double rmin = INFINITY, lmax = 0.0;
    for (int c = 0; c < o->nc; ++c) {
        Tri t = cell_tri(o, c, 0, 0);
        double area = tri_area(&t);
        double per = hypot(t.x[1] - t.x[0], t.y[1] - t.y[0]) + hypot(t.x[2] - t.x[1], t.y[2] - t.y[1]) + hypot(t.x[0] - t.x[2], t.y[0] - t.y[2]);
        double r = 2.0 * area / per;
        if (r < rmin) rmin = r;
        double U[4];
        for (int v = 0; v < o->nvar; ++v) U[v] = u[(size_t)(c * o->nvar + v) * o->np] / sqrt(area);
        double lam;
        if (o->eq == EQ_BURGERS) lam = M_SQRT2 * fabs(U[0]);
        else {
            double uu = U[1] / U[0], vv = U[2] / U[0];
            lam = sqrt(uu * uu + vv * vv) + sqrt(o->gam * euler_p(o->gam, U) / U[0]);
        }
        if (lam > lmax) lmax = lam;
    }
    return cfl * rmin / lmax;
}

/* One SSP-RK3 step of size dt from time t, in place. Stage s evaluates L_h at
 * t + (0, dt, dt/2)[s] and the limiter after stage s sees t + (dt, dt/2, dt)[s]
 * (reading R-time). Returns a limiter status (0 ok). */
int or_step(const Oracle *o, double *u, double t, double dt, unsigned char *flags_last)
{
    size_t n = (size_t)o->nc * o->nvar * o->np;
    double *u1 = (double *)malloc(sizeof(double) * n), *u2 = (double *)malloc(sizeof(double) * n);
    double *L = (double *)malloc(sizeof(double) * n), *tmp = (double *)malloc(sizeof(double) * n);
    int status = 0, s;
    const double a[3] = {0.0, 0.75, 1.0 / 3.0}, b[3] = {1.0, 0.25, 2.0 / 3.0};
    const double tr[3] = {0.0, 1.0, 0.5}, tl[3] = {1.0, 0.5, 1.0};
    const double *src[3] = {u, u1, u2};
    double *dst[3] = {u1, u2, u};
    for (int st = 0; st < 3; ++st) {
        or_rhs(o, src[st], t + tr[st] * dt, L);
        /* u^(i) = alpha_i0 u^n + beta-part (u^(i-1) + dt L(u^(i-1))), Table tvd */
        for (size_t i = 0; i < n; ++i) tmp[i] = a[st] * u[i] + b[st] * (src[st][i] + dt * L[i]);
        if (o->limiter != LIM_OFF) {
            s = or_limit(o, tmp, t + tl[st] * dt, dst[st], st == 2 ? flags_last : NULL);
            if (s) status = s;
        } else {
            memcpy(dst[st], tmp, sizeof(double) * n);
        }
    }
    free(u1); free(u2); free(L); free(tmp);
    return status;
}

/* Advance from t0 to t_end with the CFL rule (last step clipped); returns the
 * number of steps, or -1 on a limiter failure. */
int or_run(const Oracle *o, double *u, double t0, double t_end, double cfl, int max_steps, double *t_out)
{
    double t = t0;
    int nsteps = 0;
    while (t < t_end && nsteps < max_steps) {
        double dt = or_cfl_dt(o, u, cfl);
        if (t + dt > t_end) dt = t_end - t;
        if (or_step(o, u, t, dt, NULL)) return -1;
        t += dt;
        ++nsteps;
    }
    if (t_out) *t_out = t;
    return nsteps;
}

/* ======================================================================
 * 9. Initial data, diagnostics and hooks used by the pins
 * ====================================================================== */

/* volume-rule points of every cell, xy[(c*Q + q)*2 + {0,1}] */
void or_volume_points(const Oracle *o, double *xy)
{
    for (int c = 0; c < o->nc; ++c) {
        Tri t = cell_tri(o, c, 0, 0);
        for (int q = 0; q < o->vol.n; ++q) tri_point(&t, o->vol.b[q], &xy[2 * ((size_t)c * o->vol.n + q)], &xy[2 * ((size_t)c * o->vol.n + q) + 1]);
    }
}

/* L2 projection of point values vals[(c*Q + q)*nvar + v] onto the modes with
 * the volume rule: u_i = |K| sum_q W_q u(x_q) psi^K_i(x_q). */
void or_project(const Oracle *o, const double *vals, double *u)
{
    int nv = o->nvar, np = o->np, Q = o->vol.n;
    for (int c = 0; c < o->nc; ++c) {
        Tri t = cell_tri(o, c, 0, 0);
        double area = tri_area(&t);
        for (int v = 0; v < nv; ++v)
            for (int i = 0; i < np; ++i) {
                double s = 0.0;
                for (int q = 0; q < Q; ++q) {
                    double x, y, p;
                    tri_point(&t, o->vol.b[q], &x, &y);
                    psi_phys(o, &t, i, x, y, &p, NULL, NULL);
                    s += o->vol.w[q] * vals[((size_t)c * Q + q) * nv + v] * p;
                }
                u[(size_t)(c * nv + v) * np + i] = area * s;
            }
    }
}

/* the same projection for a list of cells only (other cells untouched) */
void or_project_cells(const Oracle *o, int n, const int *cells, const double *vals, double *u)
{
    int nv = o->nvar, np = o->np, Q = o->vol.n;
    for (int ii = 0; ii < n; ++ii) {
        int c = cells[ii];
        Tri t = cell_tri(o, c, 0, 0);
        double area = tri_area(&t);
        for (int v = 0; v < nv; ++v)
            for (int i = 0; i < np; ++i) {
                double s = 0.0;
                for (int q = 0; q < Q; ++q) {
                    double x, y, p;
                    tri_point(&t, o->vol.b[q], &x, &y);
                    psi_phys(o, &t, i, x, y, &p, NULL, NULL);
                    s += o->vol.w[q] * vals[((size_t)ii * Q + q) * nv + v] * p;
                }
                u[(size_t)(c * nv + v) * np + i] = area * s;
            }
    }
}

/* sum_K |K| ubar_K per variable */
void or_conservation(const Oracle *o, const double *u, double *sums)
{
    for (int v = 0; v < o->nvar; ++v) sums[v] = 0.0;
    for (int c = 0; c < o->nc; ++c) {
        Tri t = cell_tri(o, c, 0, 0);
        double area = tri_area(&t);
        for (int v = 0; v < o->nvar; ++v) sums[v] += area * u[(size_t)(c * o->nvar + v) * o->np] / sqrt(area);
    }
}

/* u_h at n given points, one cell each: out[i*nvar + v] */
void or_eval_points(const Oracle *o, const double *u, int n, const int *cells, const double *xy, double *out)
{
    for (int i = 0; i < n; ++i) {
        Tri t = cell_tri(o, cells[i], 0, 0);
        eval_cell(o, u, cells[i], &t, xy[2 * i], xy[2 * i + 1], out + (size_t)i * o->nvar);
    }
}

/* exact-integration rule (degree 10) points of every cell for error norms */
int or_error_rule(const Oracle *o, double *xy, double *w)
{
    for (int c = 0; c < o->nc; ++c) {
        Tri t = cell_tri(o, c, 0, 0);
        double area = tri_area(&t);
        for (int q = 0; q < o->duf6.n; ++q) {
            tri_point(&t, o->duf6.b[q], &xy[2 * ((size_t)c * o->duf6.n + q)], &xy[2 * ((size_t)c * o->duf6.n + q) + 1]);
            w[(size_t)c * o->duf6.n + q] = area * o->duf6.w[q];
        }
    }
    return o->duf6.n;
}

void or_connectivity(const Oracle *o, int *nb, int *nbf, double *sh)
{
    memcpy(nb, o->nb, sizeof(int) * 3 * o->nc);
    memcpy(nbf, o->nbf, sizeof(int) * 3 * o->nc);
    memcpy(sh, o->sh, sizeof(double) * 6 * o->nc);
}

/* hooks for the pins */
void or_hook_gauss_legendre(int n, double *x, double *w) { gauss_legendre(n, x, w); }

int or_hook_rule(int which, int param, double *bary, double *w)
{
    trirule R;
    if (which == 0) { if (sym_rule(param, &R)) return -1; }
    else duffy_rule(param, &R);
    for (int q = 0; q < R.n; ++q) { bary[3 * q] = R.b[q][0]; bary[3 * q + 1] = R.b[q][1]; bary[3 * q + 2] = R.b[q][2]; w[q] = R.w[q]; }
    return R.n;
}

void or_hook_psi(int k, int m, double r, double s, double *out3) { psi_ref(k, m, r, s, &out3[0], &out3[1], &out3[2]); }

int or_hook_lsq(int m, int n, const double *A, const double *b, double *c) { return lsq_qr(m, n, A, b, c); }

/* stencil triangles of cell c: tri_out[(f*7 + i)*6] for i = thirds 0..2, halves 0..3 */
void or_hook_stencil(const Oracle *o, int c, double *tri_out, int *ghost)
{
    Stencil S;
    build_stencil(o, c, &S);
    for (int f = 0; f < 3; ++f) {
        ghost[f] = S.ghost[f];
        for (int i = 0; i < 7; ++i) {
            const Tri *T = (i < 3) ? &S.third[f][i] : &S.half[f][i - 3];
            for (int v = 0; v < 3; ++v) { tri_out[(f * 7 + i) * 6 + 2 * v] = T->x[v]; tri_out[(f * 7 + i) * 6 + 2 * v + 1] = T->y[v]; }
        }
    }
}

/* subcell means of the stencil function of variable 0..nvar-1: out[(f*7+i)*nvar + v] */
void or_hook_subcell_means(const Oracle *o, const double *u, int c, double t, double *out)
{
    Stencil S;
    build_stencil(o, c, &S);
    for (int f = 0; f < 3; ++f)
        for (int i = 0; i < 7; ++i) {
            const Tri *T = (i < 3) ? &S.third[f][i] : &S.half[f][i - 3];
            stencil_mean(o, u, c, f, t, T, out + (size_t)(f * 7 + i) * o->nvar);
        }
}

/* WENO on cell c from given means (scalar): th[9] (thirds), hf[12] (halves).
 * info: q2(2) q3(5) q4(9, padded to 14) gamma(4) beta(4) omega(4) -> 33 values; modes[np] */
int or_hook_weno(const Oracle *o, int c, double ubar0, const double *th_in, const double *hf_in, int force_linear, double *info, double *modes)
{
    Stencil S;
    Frame F;
    build_stencil(o, c, &S);
    make_frame(o, c, &F);
    double th[3][3], hf[3][4];
    for (int f = 0; f < 3; ++f) {
        for (int i = 0; i < 3; ++i) th[f][i] = th_in[3 * f + i];
        for (int i = 0; i < 4; ++i) hf[f][i] = hf_in ? hf_in[4 * f + i] : 0.0;
    }
    WenoOut W;
    weno_scalar(o, &F, &S, ubar0, th, hf, force_linear, &W);
    int p = 0;
    for (int j = 0; j < 2; ++j) info[p++] = W.q2[j];
    for (int j = 0; j < 5; ++j) info[p++] = W.q3[j];
    for (int j = 0; j < 9; ++j) info[p++] = W.q4[j];
    for (int j = 9; j < 14; ++j) info[p++] = 0.0;
    for (int j = 0; j < 4; ++j) info[p++] = W.gam[j];
    for (int j = 0; j < 4; ++j) info[p++] = W.beta[j];
    for (int j = 0; j < 4; ++j) info[p++] = W.omega[j];
    for (int j = 0; j < 3; ++j) info[p++] = W.beta1l[j];
    for (int j = 0; j < 3; ++j) info[p++] = W.sigma[j];
    info[p++] = W.tau;
    modes[0] = ubar0 * sqrt(F.area);
    for (int i = 1; i < o->np; ++i) modes[i] = W.modes[i];
    return W.status;
}

/* beta of a polynomial given by monomial coefficients on cell c's frame */
double or_hook_beta(const Oracle *o, int c, int nm, const double *coef, int deg)
{
    Frame F;
    make_frame(o, c, &F);
    return beta_poly(&F, &o->duf4, nm, coef, deg);
}

/* frame of cell c: x0, y0, h0, area, hbar, m0[14] -> 19 values */
void or_hook_frame(const Oracle *o, int c, double *out)
{
    Frame F;
    make_frame(o, c, &F);
    out[0] = F.x0; out[1] = F.y0; out[2] = F.h0; out[3] = F.area; out[4] = F.hbar;
    for (int j = 0; j < 14; ++j) out[5 + j] = F.m0[j];
}

void or_hook_flux(const Oracle *o, const double *UL, const double *UR, double nx, double ny, double *F) { llf_flux(o, UL, UR, nx, ny, F); }

int or_hook_limit_cell(const Oracle *o, const double *u, double t, int c, double *out) { return limit_cell(o, u, t, c, out); }
/* the same with the linear weights in every field (omega = gamma) */
int or_hook_limit_cell_linear(const Oracle *o, const double *u, double t, int c, double *out) { return limit_cell_w(o, u, t, c, out, 1); }
