/* levelset3d.c -- TEST INFRASTRUCTURE ONLY: the plain FP64 CPU oracle of the
 * level-set part of the three-dimensional tank step (sections "Interface
 * tracking", "Level set advection" and "Density and viscosity specification",
 * d = 3), used by tests/ to check the GPU library.  It shares no code with the
 * GPU path.
 *
 * Grid: nx x ny x nz cells of size h, z vertical, still water at z = depth;
 * waves travel along x (uniform along y).  Layouts, x fastest: cells
 * [nz][ny][nx]; u [nz][ny][nx+1]; v [nz][ny+1][nx]; w [nz+1][ny][nx].
 *
 * The readings are the two-dimensional ones carried to three directions:
 *  - materials (two-stage, Eqs. ls_flow then ls_solid; smoothed Heaviside with
 *    half-width h): water/air from sigma, then the body from its SDF psi; the
 *    body is a vertical cylinder, psi = max(r - R, |z - z_c| - L / 2) with r the
 *    distance to its axis, solid density m / (pi R^2 L), solid viscosity mu_w;
 *  - advection (PPM, Colella-Woodward with van Leer-limited edge slopes, the
 *    CW84 parabola limiter and characteristic tracing, single stage):
 *    sigma* = sigma - dt Q, Q = sum over the three directions of the mean of the
 *    two face velocities times the difference of the upwind PPM face states / h;
 *    then the damping-zone blend toward z - depth with the Jacobsen weight;
 *  - ghosts of sigma: x < 0 the incident wave's z - depth - eta(x, t); x beyond
 *    the outlet and y outside the tank zero gradient; below the bed and above
 *    the top linear extrapolation;
 *  - reinitialisation (Sussman): sigma_tau + S(sigma0)(|grad sigma| - 1) = 0,
 *    S = sigma0 / sqrt(sigma0^2 + h^2), Godunov Hamiltonian on ENO-2 one-sided
 *    differences with minmod corrections, TVD-RK2, d tau = 0.3 h.
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

#define PI3 3.14159265358979323846

typedef struct {
    int nx, ny, nz;
    double h, depth;
    double rho_w, rho_a, mu_w, mu_a;
    int ncomp;
    const double *amp, *omega, *kwave, *phase;
    double damp_x0, damp_len;
    int has_body;
    double body_xc, body_yc, body_r, body_len, body_mass;
} oracle3_tank;

static int clamp3(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }
static double sq3(double a) { return a * a; }

static double eta3(const oracle3_tank *P, double x, double t)
{
    double e = 0.0;
    for (int c = 0; c < P->ncomp; ++c) e += P->amp[c] * cos(P->kwave[c] * x - P->omega[c] * t + P->phase[c]);
    return e;
}

static double heav3(double phi, double eps)
{
    if (phi < -eps) return 0.0;
    if (phi > eps) return 1.0;
    return 0.5 * (1.0 + phi / eps + sin(PI3 * phi / eps) / PI3);
}

static double psi3(const oracle3_tank *P, double x, double y, double z, double zc)
{
    if (!P->has_body) return 1.0e3;
    double r = sqrt((x - P->body_xc) * (x - P->body_xc) + (y - P->body_yc) * (y - P->body_yc));
    return fmax(r - P->body_r, fabs(z - zc) - 0.5 * P->body_len);
}

/* Cell materials, Eqs. ls_flow then ls_solid. */
void oracle3_materials(const oracle3_tank *P, const double *sg, double zc, double *rho, double *mu, double *rhof,
                       double *chi)
{
    double h = P->h;
    double rho_s = P->has_body ? P->body_mass / (PI3 * P->body_r * P->body_r * P->body_len) : P->rho_w;
    ORACLE_PAR_FOR
    for (int k = 0; k < P->nz; ++k)
        for (int j = 0; j < P->ny; ++j)
            for (int i = 0; i < P->nx; ++i) {
                size_t c = ((size_t)k * P->ny + j) * P->nx + i;
                double hf = heav3(sg[c], h);
                double hb = heav3(psi3(P, (i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h, zc), h);
                double rf = P->rho_w + (P->rho_a - P->rho_w) * hf;
                double mf = P->mu_w + (P->mu_a - P->mu_w) * hf;
                rho[c] = rho_s + (rf - rho_s) * hb;
                mu[c] = P->mu_w + (mf - P->mu_w) * hb;
                rhof[c] = rf;
                chi[c] = 1.0 - hb;
            }
}

/* sigma at (i, j, k) with its ghosts; the inflow ghost is the incident wave's
 * z - depth - eta at time ta, or, for a field that is the mean of two time
 * levels (ta != tb), with the mean of eta at ta and tb. */
static double sig3(const oracle3_tank *P, const double *s, int i, int j, int k, double ta, double tb)
{
    int nx = P->nx, ny = P->ny, nz = P->nz;
    if (i < 0) {
        double x = (i + 0.5) * P->h, e = eta3(P, x, ta);
        if (tb != ta) e = 0.5 * (e + eta3(P, x, tb));
        return (k + 0.5) * P->h - P->depth - e;
    }
    i = i > nx - 1 ? nx - 1 : i;
    j = clamp3(j, 0, ny - 1);
    size_t col = (size_t)j * nx + i, pl = (size_t)nx * ny;
    if (k < 0) return s[col] + k * (s[pl + col] - s[col]);
    if (k > nz - 1) {
        double a = s[(nz - 1) * pl + col], b = s[(nz - 2) * pl + col];
        return a + (k - (nz - 1)) * (a - b);
    }
    return s[k * pl + col];
}

static double vlslope3(double am, double a0, double ap)
{
    double dl = a0 - am, dr = ap - a0;
    if (dl * dr <= 0.0) return 0.0;
    double dc = 0.5 * (ap - am);
    double m = fmin(fabs(dc), fmin(2.0 * fabs(dl), 2.0 * fabs(dr)));
    return dc > 0.0 ? m : -m;
}

/* limited PPM edge values of the middle cell of a[0..4] */
static void ppmcell3(const double *a, double *aL, double *aR)
{
    double dm = vlslope3(a[0], a[1], a[2]), d0 = vlslope3(a[1], a[2], a[3]), dp = vlslope3(a[2], a[3], a[4]);
    double L = a[1] + 0.5 * (a[2] - a[1]) - (d0 - dm) / 6.0;
    double R = a[2] + 0.5 * (a[3] - a[2]) - (dp - d0) / 6.0;
    double c = a[2];
    if ((R - c) * (c - L) <= 0.0) {
        L = c;
        R = c;
    } else {
        double dA = R - L, m6 = dA * (c - 0.5 * (L + R)), q = dA * dA / 6.0;
        if (m6 > q)
            L = 3.0 * c - 2.0 * R;
        else if (-q > m6)
            R = 3.0 * c - 2.0 * L;
    }
    *aL = L;
    *aR = R;
}

/* time-centred upwind state at the face between a[2] and a[3] (a = cells f-3 .. f+2) */
static double ppmface3(const double *a, double vel, double dt, double h)
{
    double L, R;
    if (vel >= 0.0) {
        ppmcell3(a, &L, &R);
        double C = vel * dt / h, dA = R - L, a6 = 6.0 * (a[2] - 0.5 * (L + R));
        return R - 0.5 * C * (dA - (1.0 - 2.0 * C / 3.0) * a6);
    }
    ppmcell3(a + 1, &L, &R);
    double C = -vel * dt / h, dA = R - L, a6 = 6.0 * (a[3] - 0.5 * (L + R));
    return L + 0.5 * C * (dA + (1.0 - 2.0 * C / 3.0) * a6);
}

static double damp3(const oracle3_tank *P, double x)
{
    if (P->damp_len <= 0.0 || x <= P->damp_x0) return 0.0;
    double xi = (x - P->damp_x0) / P->damp_len;
    if (xi > 1.0) xi = 1.0;
    return (exp(pow(xi, 3.5)) - 1.0) / (exp(1.0) - 1.0);
}

/* sigma* at cell (i, j, k): base - dt Q(u, s), then the damping-zone blend
 * (base = s for the plain update; the ghosts of s at ta, tb as in sig3) */
static double advect_cell3(const oracle3_tank *P, const double *base, const double *s, const double *u,
                           const double *v, const double *w, double dt, double ta, double tb, int i, int j, int k)
{
    int nx = P->nx, ny = P->ny;
    double h = P->h, a[6];
    size_t r = (size_t)k * ny + j, c = r * nx + i;
    size_t fu = r * (nx + 1) + i, fv = ((size_t)k * (ny + 1) + j) * nx + i;
    double fx[2], fy[2], fz[2];
    for (int f = 0; f < 2; ++f) {
        for (int q = 0; q < 6; ++q) a[q] = sig3(P, s, i + f - 3 + q, j, k, ta, tb);
        fx[f] = ppmface3(a, u[fu + f], dt, h);
        for (int q = 0; q < 6; ++q) a[q] = sig3(P, s, i, j + f - 3 + q, k, ta, tb);
        fy[f] = ppmface3(a, v[fv + (size_t)f * nx], dt, h);
        for (int q = 0; q < 6; ++q) a[q] = sig3(P, s, i, j, k + f - 3 + q, ta, tb);
        fz[f] = ppmface3(a, w[c + (size_t)f * nx * ny], dt, h);
    }
    double ub = 0.5 * (u[fu] + u[fu + 1]);
    double vb = 0.5 * (v[fv] + v[fv + nx]);
    double wb = 0.5 * (w[c] + w[c + (size_t)nx * ny]);
    double Q = ub * (fx[1] - fx[0]) / h + vb * (fy[1] - fy[0]) / h + wb * (fz[1] - fz[0]) / h;
    double sa = base[c] - dt * Q;
    double al = damp3(P, (i + 0.5) * h);
    return (1.0 - al) * sa + al * ((k + 0.5) * h - P->depth);
}

void oracle3_advect(const oracle3_tank *P, const double *s, const double *u, const double *v, const double *w,
                    double dt, double t, double *out)
{
    ORACLE_PAR_FOR
    for (int k = 0; k < P->nz; ++k)
        for (int j = 0; j < P->ny; ++j)
            for (int i = 0; i < P->nx; ++i)
                out[((size_t)k * P->ny + j) * P->nx + i] = advect_cell3(P, s, s, u, v, w, dt, t, t, i, j, k);
}

/* The update of a fixed-point cycle k >= 1 (section "Time stepping scheme"):
 * out = base - dt Q(u, s) then the damping-zone blend, with base = sigma^n and
 * s, u the means of time levels n and n+1,k (inflow ghosts: the mean of the
 * incident wave at ta = t^n and tb = t^{n+1}). */
void oracle3_advect_half(const oracle3_tank *P, const double *base, const double *s, const double *u, const double *v,
                         const double *w, double dt, double ta, double tb, double *out)
{
    ORACLE_PAR_FOR
    for (int k = 0; k < P->nz; ++k)
        for (int j = 0; j < P->ny; ++j)
            for (int i = 0; i < P->nx; ++i)
                out[((size_t)k * P->ny + j) * P->nx + i] = advect_cell3(P, base, s, u, v, w, dt, ta, tb, i, j, k);
}

/* The same at ncell listed cells (cell index c = (k ny + j) nx + i). */
void oracle3_advect_cells(const oracle3_tank *P, const double *s, const double *u, const double *v, const double *w,
                          double dt, double t, const long long *cells, int ncell, double *out)
{
    for (int q = 0; q < ncell; ++q) {
        long long c = cells[q];
        int i = (int)(c % P->nx), j = (int)((c / P->nx) % P->ny), k = (int)(c / ((long long)P->nx * P->ny));
        out[q] = advect_cell3(P, s, s, u, v, w, dt, t, t, i, j, k);
    }
}

static double mm3(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

/* S(sigma0) (|grad sigma| - 1) at cell (i, j, k), Godunov on ENO-2 differences */
static double rrhs3(const oracle3_tank *P, const double *f, const double *s0, int i, int j, int k, double t)
{
    double h = P->h, c = sig3(P, f, i, j, k, t, t);
    double g[3];
    int sgn_pos = s0[((size_t)k * P->ny + j) * P->nx + i] > 0.0;
    for (int d = 0; d < 3; ++d) {
        int di = d == 0, dj = d == 1, dk = d == 2;
        double m2 = sig3(P, f, i - 2 * di, j - 2 * dj, k - 2 * dk, t, t), m1 = sig3(P, f, i - di, j - dj, k - dk, t, t);
        double p1 = sig3(P, f, i + di, j + dj, k + dk, t, t), p2 = sig3(P, f, i + 2 * di, j + 2 * dj, k + 2 * dk, t, t);
        double dm = m2 - 2.0 * m1 + c, d0 = m1 - 2.0 * c + p1, dp = c - 2.0 * p1 + p2;
        double a = (c - m1) / h + mm3(dm, d0) / (2.0 * h);
        double b = (p1 - c) / h - mm3(d0, dp) / (2.0 * h);
        if (sgn_pos)
            g[d] = fmax(sq3(fmax(a, 0.0)), sq3(fmin(b, 0.0)));
        else
            g[d] = fmax(sq3(fmin(a, 0.0)), sq3(fmax(b, 0.0)));
    }
    double sg0 = s0[((size_t)k * P->ny + j) * P->nx + i];
    double S = sg0 / sqrt(sg0 * sg0 + h * h);
    return S * (sqrt(g[0] + g[1] + g[2]) - 1.0);
}

void oracle3_reinit(const oracle3_tank *P, double *s, int nit, double t)
{
    size_t n = (size_t)P->nx * P->ny * P->nz;
    double dtau = 0.3 * P->h;
    double *s0 = (double *)malloc(n * sizeof(double)), *s1 = (double *)malloc(n * sizeof(double));
    double *s2 = (double *)malloc(n * sizeof(double));
    if (!s0 || !s1 || !s2) abort();
    memcpy(s0, s, n * sizeof(double));
    for (int it = 0; it < nit; ++it) {
        ORACLE_PAR_FOR
        for (int k = 0; k < P->nz; ++k)
            for (int j = 0; j < P->ny; ++j)
                for (int i = 0; i < P->nx; ++i) {
                    size_t c = ((size_t)k * P->ny + j) * P->nx + i;
                    s1[c] = s[c] - dtau * rrhs3(P, s, s0, i, j, k, t);
                }
        ORACLE_PAR_FOR
        for (int k = 0; k < P->nz; ++k)
            for (int j = 0; j < P->ny; ++j)
                for (int i = 0; i < P->nx; ++i) {
                    size_t c = ((size_t)k * P->ny + j) * P->nx + i;
                    s2[c] = s1[c] - dtau * rrhs3(P, s1, s0, i, j, k, t);
                }
        for (size_t c = 0; c < n; ++c) s[c] = 0.5 * (s[c] + s2[c]);
    }
    free(s0);
    free(s1);
    free(s2);
}
