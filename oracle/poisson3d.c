/* poisson3d.c -- TEST INFRASTRUCTURE ONLY: the plain FP64 CPU oracle of the 3D
 * pressure Poisson solve, used by tests/ and by the benchmark's CPU baseline to
 * check the GPU library.  It shares no code with the GPU path.
 *
 * Pressure equation of the projection in three dimensions (section "Continuous
 * equations of motion", d = 3; the discrete continuity equation of section
 * "Spatial discretization" with face coefficients beta_f): on an
 * nx x ny x nz cell grid (z vertical),
 *
 *   (A p)_c = sum over the six faces f of c of beta_f (p_c - p_nb(f)),
 *
 * the walls x = 0, x = lx, y = 0, y = ly and the bed z = 0 Neumann (their faces
 * drop out whatever coefficient they hold), the top z = lz Dirichlet p = 0 at
 * the face (ghost value -p_c, so the top face counts twice in the diagonal).
 *
 * Solver (the paper leaves it to PETSc; this is the library's own choice, the
 * same as in two dimensions): FGMRES(m) right-preconditioned by one geometric
 * multigrid V(nu1, nu2) cycle, classical Gram-Schmidt applied twice, Givens
 * rotations, converged when ||b - A x||_2 <= rtol ||b||_2 with the true
 * residual recomputed at the end of every cycle.  Multigrid: red-black
 * Gauss-Seidel (colour (i + j + k) mod 2, red first), coarsening by two in every
 * direction while all three sizes are even and at least 4, restriction = sum of
 * the eight children's residuals, piecewise-constant prolongation, coarse face
 * coefficient = half the sum of the four fine faces it covers (the face
 * coefficient of a rediscretised operator carries area / distance = h, so it
 * doubles from level to level; in two dimensions the same rule is the mean of
 * two faces), dense LU without pivoting on the coarsest level.
 *
 * Layouts, x fastest: cells [nz][ny][nx]; beta_x [nz][ny][nx+1]; beta_y
 * [nz][ny+1][nx]; beta_z [nz+1][ny][nx] (face (i, j, k) of beta_z is the bottom
 * face of cell (i, j, k)).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Loops whose iterations are independent (each writes only its own output
 * element; no reduction) may run on several host threads; every reduction and
 * every order-dependent loop stays serial, so results do not depend on the
 * thread count. */
#ifdef _OPENMP
#define ORACLE_PAR_FOR _Pragma("omp parallel for schedule(static)")
#else
#define ORACLE_PAR_FOR
#endif

typedef struct {
    int nx, ny, nz;
    double *bx, *by, *bz, *x, *b, *r;
} lev3;

#define BX(L, i, j, k) ((L)->bx[((size_t)(k) * (L)->ny + (j)) * ((L)->nx + 1) + (i)])
#define BY(L, i, j, k) ((L)->by[((size_t)(k) * ((L)->ny + 1) + (j)) * (L)->nx + (i)])
#define BZ(L, i, j, k) ((L)->bz[((size_t)(k) * (L)->ny + (j)) * (L)->nx + (i)])
#define CELL(L, i, j, k) (((size_t)(k) * (L)->ny + (j)) * (L)->nx + (i))

static double *zalloc(size_t n)
{
    double *p = (double *)calloc(n ? n : 1, sizeof(double));
    if (!p) abort();
    return p;
}

static size_t ncell(const lev3 *L) { return (size_t)L->nx * L->ny * L->nz; }

static double diag3(const lev3 *L, int i, int j, int k)
{
    double d = 0.0;
    if (i > 0) d += BX(L, i, j, k);
    if (i < L->nx - 1) d += BX(L, i + 1, j, k);
    if (j > 0) d += BY(L, i, j, k);
    if (j < L->ny - 1) d += BY(L, i, j + 1, k);
    if (k > 0) d += BZ(L, i, j, k);
    d += (k < L->nz - 1 ? 1.0 : 2.0) * BZ(L, i, j, k + 1);
    return d;
}

static double offsum3(const lev3 *L, const double *x, int i, int j, int k)
{
    double s = 0.0;
    if (i > 0) s += BX(L, i, j, k) * x[CELL(L, i - 1, j, k)];
    if (i < L->nx - 1) s += BX(L, i + 1, j, k) * x[CELL(L, i + 1, j, k)];
    if (j > 0) s += BY(L, i, j, k) * x[CELL(L, i, j - 1, k)];
    if (j < L->ny - 1) s += BY(L, i, j + 1, k) * x[CELL(L, i, j + 1, k)];
    if (k > 0) s += BZ(L, i, j, k) * x[CELL(L, i, j, k - 1)];
    if (k < L->nz - 1) s += BZ(L, i, j, k + 1) * x[CELL(L, i, j, k + 1)];
    return s;
}

static void apply3(const lev3 *L, const double *x, double *y)
{
    ORACLE_PAR_FOR
    for (int k = 0; k < L->nz; ++k)
        for (int j = 0; j < L->ny; ++j)
            for (int i = 0; i < L->nx; ++i)
                y[CELL(L, i, j, k)] = diag3(L, i, j, k) * x[CELL(L, i, j, k)] - offsum3(L, x, i, j, k);
}

static void rbgs3(lev3 *L)
{
    for (int color = 0; color < 2; ++color) {
        ORACLE_PAR_FOR
        for (int k = 0; k < L->nz; ++k)
            for (int j = 0; j < L->ny; ++j)
                for (int i = 0; i < L->nx; ++i)
                    if (((i + j + k) & 1) == color) {
                        size_t c = CELL(L, i, j, k);
                        L->x[c] = (L->b[c] + offsum3(L, L->x, i, j, k)) / diag3(L, i, j, k);
                    }
    }
}

/* Dense LU without pivoting (A is a symmetric M-matrix), columns A e_q. */
static void coarse3(lev3 *L)
{
    int n = (int)ncell(L);
    double *A = zalloc((size_t)n * n), *e = zalloc(n), *col = zalloc(n), *y = zalloc(n);
    for (int q = 0; q < n; ++q) {
        memset(e, 0, sizeof(double) * n);
        e[q] = 1.0;
        apply3(L, e, col);
        for (int r = 0; r < n; ++r) A[(size_t)r * n + q] = col[r];
    }
    for (int q = 0; q < n; ++q)
        for (int r = q + 1; r < n; ++r) {
            double f = A[(size_t)r * n + q] / A[(size_t)q * n + q];
            A[(size_t)r * n + q] = f;
            for (int c = q + 1; c < n; ++c) A[(size_t)r * n + c] -= f * A[(size_t)q * n + c];
        }
    for (int r = 0; r < n; ++r) {
        double s = L->b[r];
        for (int c = 0; c < r; ++c) s -= A[(size_t)r * n + c] * y[c];
        y[r] = s;
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = y[r];
        for (int c = r + 1; c < n; ++c) s -= A[(size_t)r * n + c] * L->x[c];
        L->x[r] = s / A[(size_t)r * n + r];
    }
    free(A);
    free(e);
    free(col);
    free(y);
}

typedef struct {
    int nlev, nu1, nu2;
    lev3 lev[32];
} hier3;

static void hier3_build(hier3 *H, int nx, int ny, int nz, const double *bx, const double *by, const double *bz,
                        int nu1, int nu2)
{
    H->nu1 = nu1;
    H->nu2 = nu2;
    H->nlev = 0;
    for (;;) {
        lev3 *L = &H->lev[H->nlev];
        L->nx = nx;
        L->ny = ny;
        L->nz = nz;
        size_t nfx = (size_t)(nx + 1) * ny * nz, nfy = (size_t)nx * (ny + 1) * nz, nfz = (size_t)nx * ny * (nz + 1);
        L->bx = zalloc(nfx);
        L->by = zalloc(nfy);
        L->bz = zalloc(nfz);
        L->x = zalloc(ncell(L));
        L->b = zalloc(ncell(L));
        L->r = zalloc(ncell(L));
        if (H->nlev == 0) {
            memcpy(L->bx, bx, sizeof(double) * nfx);
            memcpy(L->by, by, sizeof(double) * nfy);
            memcpy(L->bz, bz, sizeof(double) * nfz);
        } else {
            lev3 *F = &H->lev[H->nlev - 1];
            ORACLE_PAR_FOR
            for (int K = 0; K < nz; ++K)
                for (int J = 0; J < ny; ++J)
                    for (int I = 0; I <= nx; ++I) {
                        double s = 0.0;
                        for (int b = 0; b < 2; ++b)
                            for (int a = 0; a < 2; ++a) s += BX(F, 2 * I, 2 * J + a, 2 * K + b);
                        BX(L, I, J, K) = 0.5 * s;
                    }
            ORACLE_PAR_FOR
            for (int K = 0; K < nz; ++K)
                for (int J = 0; J <= ny; ++J)
                    for (int I = 0; I < nx; ++I) {
                        double s = 0.0;
                        for (int b = 0; b < 2; ++b)
                            for (int a = 0; a < 2; ++a) s += BY(F, 2 * I + a, 2 * J, 2 * K + b);
                        BY(L, I, J, K) = 0.5 * s;
                    }
            ORACLE_PAR_FOR
            for (int K = 0; K <= nz; ++K)
                for (int J = 0; J < ny; ++J)
                    for (int I = 0; I < nx; ++I) {
                        double s = 0.0;
                        for (int b = 0; b < 2; ++b)
                            for (int a = 0; a < 2; ++a) s += BZ(F, 2 * I + a, 2 * J + b, 2 * K);
                        BZ(L, I, J, K) = 0.5 * s;
                    }
        }
        H->nlev++;
        if (nx % 2 || ny % 2 || nz % 2 || nx < 4 || ny < 4 || nz < 4 || H->nlev == 32) break;
        nx /= 2;
        ny /= 2;
        nz /= 2;
    }
}

static void hier3_free(hier3 *H)
{
    for (int l = 0; l < H->nlev; ++l) {
        free(H->lev[l].bx);
        free(H->lev[l].by);
        free(H->lev[l].bz);
        free(H->lev[l].x);
        free(H->lev[l].b);
        free(H->lev[l].r);
    }
}

/* One V(nu1, nu2) cycle on level l from a zero guess: lev[l].x = M^{-1} lev[l].b. */
static void vcycle3(hier3 *H, int l)
{
    lev3 *L = &H->lev[l];
    size_t n = ncell(L);
    if (l == H->nlev - 1) {
        coarse3(L);
        return;
    }
    memset(L->x, 0, sizeof(double) * n);
    for (int s = 0; s < H->nu1; ++s) rbgs3(L);
    apply3(L, L->x, L->r);
    ORACLE_PAR_FOR
    for (size_t c = 0; c < n; ++c) L->r[c] = L->b[c] - L->r[c];
    lev3 *C = &H->lev[l + 1];
    ORACLE_PAR_FOR
    for (int K = 0; K < C->nz; ++K)
        for (int J = 0; J < C->ny; ++J)
            for (int I = 0; I < C->nx; ++I) {
                double s = 0.0;
                for (int c = 0; c < 2; ++c)
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a) s += L->r[CELL(L, 2 * I + a, 2 * J + b, 2 * K + c)];
                C->b[CELL(C, I, J, K)] = s;
            }
    vcycle3(H, l + 1);
    ORACLE_PAR_FOR
    for (int k = 0; k < L->nz; ++k)
        for (int j = 0; j < L->ny; ++j)
            for (int i = 0; i < L->nx; ++i) L->x[CELL(L, i, j, k)] += C->x[CELL(C, i / 2, j / 2, k / 2)];
    for (int s = 0; s < H->nu2; ++s) rbgs3(L);
}

static double dot3(const double *a, const double *b, size_t n)
{
    double s = 0.0;
    for (size_t c = 0; c < n; ++c) s += a[c] * b[c];
    return s;
}

/* FGMRES(m) of the module header; returns 0 (converged) or 3 (iteration cap). */
static int fgmres3(hier3 *H, const double *b, double *x, double rtol, int maxit, int m, int *iters, double *relres)
{
    lev3 *L0 = &H->lev[0];
    size_t n = ncell(L0);
    double bn = sqrt(dot3(b, b, n));
    *iters = 0;
    if (bn == 0.0) {
        memset(x, 0, sizeof(double) * n);
        *relres = 0.0;
        return 0;
    }
    double tol = rtol * bn;
    double *V = zalloc((size_t)(m + 1) * n), *Z = zalloc((size_t)m * n), *w = zalloc(n);
    double *Hm = zalloc((size_t)(m + 1) * m), *cs = zalloc(m), *sn = zalloc(m), *g = zalloc(m + 1);
    double *h = zalloc(m + 1), *y = zalloc(m);
    int its = 0, conv = 0;
    apply3(L0, x, w);
    ORACLE_PAR_FOR
    for (size_t c = 0; c < n; ++c) w[c] = b[c] - w[c];
    double beta = sqrt(dot3(w, w, n));
    if (beta <= tol) conv = 1;
    while (!conv && its < maxit) {
        ORACLE_PAR_FOR
        for (size_t c = 0; c < n; ++c) V[c] = w[c] / beta;
        for (int q = 0; q <= m; ++q) g[q] = 0.0;
        g[0] = beta;
        int used = 0;
        for (int j = 0; j < m; ++j) {
            /* z_j = M^{-1} v_j (one V-cycle), w = A z_j */
            memcpy(L0->b, V + (size_t)j * n, sizeof(double) * n);
            vcycle3(H, 0);
            memcpy(Z + (size_t)j * n, L0->x, sizeof(double) * n);
            apply3(L0, Z + (size_t)j * n, w);
            its++;
            for (int q = 0; q <= j; ++q) Hm[q * m + j] = 0.0;
            /* classical Gram-Schmidt, twice */
            for (int pass = 0; pass < 2; ++pass) {
                for (int q = 0; q <= j; ++q) h[q] = dot3(V + (size_t)q * n, w, n);
                for (int q = 0; q <= j; ++q) {
                    const double *vq = V + (size_t)q * n;
                    ORACLE_PAR_FOR
                    for (size_t c = 0; c < n; ++c) w[c] -= h[q] * vq[c];
                    Hm[q * m + j] += h[q];
                }
            }
            double hn = sqrt(dot3(w, w, n));
            Hm[(j + 1) * m + j] = hn;
            /* earlier rotations on column j, then the new one */
            for (int q = 0; q < j; ++q) {
                double a = Hm[q * m + j], c2 = Hm[(q + 1) * m + j];
                Hm[q * m + j] = cs[q] * a + sn[q] * c2;
                Hm[(q + 1) * m + j] = -sn[q] * a + cs[q] * c2;
            }
            double a = Hm[j * m + j], c2 = Hm[(j + 1) * m + j];
            double r = sqrt(a * a + c2 * c2);
            cs[j] = a / r;
            sn[j] = c2 / r;
            Hm[j * m + j] = r;
            Hm[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            used = j + 1;
            if (fabs(g[j + 1]) <= tol || its >= maxit || hn == 0.0) break;
            ORACLE_PAR_FOR
            for (size_t c = 0; c < n; ++c) V[(size_t)(j + 1) * n + c] = w[c] / hn;
        }
        /* x += Z y with R y = g */
        for (int q = used - 1; q >= 0; --q) {
            double s = g[q];
            for (int l = q + 1; l < used; ++l) s -= Hm[q * m + l] * y[l];
            y[q] = s / Hm[q * m + q];
        }
        for (int q = 0; q < used; ++q) {
            const double *zq = Z + (size_t)q * n;
            ORACLE_PAR_FOR
            for (size_t c = 0; c < n; ++c) x[c] += y[q] * zq[c];
        }
        apply3(L0, x, w);
        ORACLE_PAR_FOR
        for (size_t c = 0; c < n; ++c) w[c] = b[c] - w[c];
        beta = sqrt(dot3(w, w, n));
        if (beta <= tol) conv = 1;
    }
    *iters = its;
    *relres = beta / bn;
    free(V);
    free(Z);
    free(w);
    free(Hm);
    free(cs);
    free(sn);
    free(g);
    free(h);
    free(y);
    return conv ? 0 : 3;
}

/* ------------------------------------------------------------ entry points -- */
void oracle3_poisson_apply(int nx, int ny, int nz, const double *bx, const double *by, const double *bz,
                           const double *x, double *y)
{
    lev3 L = {nx, ny, nz, (double *)bx, (double *)by, (double *)bz, 0, 0, 0};
    apply3(&L, x, y);
}

/* Levels of the hierarchy and the coarsest level's sizes (out3). */
int oracle3_levels(int nx, int ny, int nz, int *out3)
{
    int nl = 1;
    while (!(nx % 2 || ny % 2 || nz % 2 || nx < 4 || ny < 4 || nz < 4) && nl < 32) {
        nx /= 2;
        ny /= 2;
        nz /= 2;
        nl++;
    }
    out3[0] = nx;
    out3[1] = ny;
    out3[2] = nz;
    return nl;
}

/* x = M^{-1} b, one V-cycle from a zero guess.  Returns the number of levels. */
int oracle3_vcycle(int nx, int ny, int nz, const double *bx, const double *by, const double *bz, int nu1, int nu2,
                   const double *b, double *x)
{
    hier3 H;
    hier3_build(&H, nx, ny, nz, bx, by, bz, nu1, nu2);
    size_t n = (size_t)nx * ny * nz;
    memcpy(H.lev[0].b, b, sizeof(double) * n);
    vcycle3(&H, 0);
    memcpy(x, H.lev[0].x, sizeof(double) * n);
    int nl = H.nlev;
    hier3_free(&H);
    return nl;
}

/* FGMRES solve from the guess in x.  Returns 0 or 3 (not converged). */
int oracle3_poisson_solve(int nx, int ny, int nz, const double *bx, const double *by, const double *bz,
                          const double *b, double *x, double rtol, int maxit, int restart, int nu1, int nu2,
                          int *iters, double *relres)
{
    hier3 H;
    hier3_build(&H, nx, ny, nz, bx, by, bz, nu1, nu2);
    int st = fgmres3(&H, b, x, rtol, maxit, restart, iters, relres);
    hier3_free(&H);
    return st;
}
