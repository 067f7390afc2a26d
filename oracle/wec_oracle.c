/* Plain FP64 CPU oracle of one time step of the two-phase wave tank (2D).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py.  Slow, single-threaded, written to be checked
 * against the paper by eye.  It shares no code with the CUDA library.
 *
 * Paper sections followed (arxiv 2206.07732):
 *   Eq. momentum / continuity ........ multiphase INS with f_c (Section "Continuous equations of motion")
 *   Eq. brinkman_force, bp_discrete .. implicit Brinkman penalisation, chi = 1 - H_body
 *   Eqs. ls_flow, ls_solid, Hflow, Hbody .. two-stage material properties, n_cells = 1
 *   Section "Level set advection" .... explicit PPM advection of sigma
 *   Section "Interface tracking" ..... Sussman relaxation reinitialisation of sigma; psi analytic (CSG max)
 *   Eq. c_discrete_momentum .......... conservative momentum, consistent mass/momentum transport,
 *                                      Crank-Nicolson viscosity, flow-density gravity
 *   Eq. c_discrete_continuity ........ projection onto div u = 0
 *   Eq. ub_velocity, newton_u ........ heave-only rigid velocity and the heave equation
 *   Eq. int_fh ....................... hydrodynamic force as a face sum over the stair-step body
 *   Eq. spongelayer .................. vorticity damping zone at the top
 *   Section "Numerical wave tank" .... Dirichlet wave inflow, wave damping zone
 *   Section "Time stepping scheme" ... n_cycles = 1: cycle-0 values are the previous step's
 *   Eqs. first_order_wave_elev, irregular_elevation .. Airy components of the inflow
 * The pressure solver (FGMRES right-preconditioned by a geometric multigrid
 * V-cycle) is not described by the paper; it is the solver this library
 * specifies for the pressure equation.  Readings of unstated details are
 * listed next to the code that takes them.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "wec_oracle.h"

#define PI 3.14159265358979323846
#define REINIT_DTAU 0.3   /* pseudo-time step as a fraction of h */

typedef struct {
    oracle_params P;
    double h, rho_s, mu_s;
    double *amp, *omega, *kw, *phase;
    double t, yc, zdot, yc0, zdot_prev;
    double *sig, *u, *v, *p;
    /* last-step intermediates, kept for inspection */
    double *sig_adv, *us, *vs, *bu, *bv, *rhs, *rbu, *rbv;
} otank;

static double *dalloc(size_t n) { return (double *)calloc(n ? n : 1, sizeof(double)); }
static int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }
static double sq(double a) { return a * a; }

/* ------------------------------------------------------------------ waves -- */
/* Eq. irregular_elevation: eta = sum a_i cos(k_i x - w_i t + theta_i) */
static double eta_at(const otank *T, double x, double t)
{
    double e = 0.0;
    for (int c = 0; c < T->P.ncomp; ++c)
        e += T->amp[c] * cos(T->kw[c] * x - T->omega[c] * t + T->phase[c]);
    return e;
}

/* Smoothed Heaviside, Eqs. Hflow / Hbody with half-width eps = n_cells h. */
static double heav(double phi, double eps)
{
    if (phi < -eps) return 0.0;
    if (phi > eps) return 1.0;
    return 0.5 * (1.0 + phi / eps + sin(PI * phi / eps) / PI);
}

/* Linear (Airy) velocity of the wave field at (x, y, t).  Reading: the paper only
 * says Dirichlet velocities generate the waves; we use the linear-potential
 * velocities with Wheeler stretching y' = d y / (d + eta) up to the surface,
 * blended to zero in the air by 1 - H(y - d - eta). */
static void airy_velocity(const otank *T, double x, double y, double t, double *uo, double *vo)
{
    double d = T->P.depth;
    double e = eta_at(T, x, t);
    double ys = y < d + e ? y : d + e;
    double yp = d * ys / (d + e);
    double blend = 1.0 - heav(y - d - e, T->h);
    double su = 0.0, sv = 0.0;
    for (int c = 0; c < T->P.ncomp; ++c) {
        double k = T->kw[c], w = T->omega[c];
        double ph = k * x - w * t + T->phase[c];
        double sk = sinh(k * d);
        su += T->amp[c] * w * cosh(k * yp) / sk * cos(ph);
        sv += T->amp[c] * w * sinh(k * yp) / sk * sin(ph);
    }
    *uo = blend * su;
    *vo = blend * sv;
}

/* ------------------------------------------------------------ geometry -- */
/* Body SDF by CSG: a box is the intersection (max) of four half-planes. */
static double psi_at(const otank *T, double x, double y, double yc)
{
    if (!T->P.has_body) return 1.0e3;
    return fmax(fabs(x - T->P.body_xc) - 0.5 * T->P.body_w, fabs(y - yc) - 0.5 * T->P.body_h);
}

/* Two-stage material properties, Eqs. ls_flow then ls_solid. */
static void cell_mat(const otank *T, double sg, double ps, double *rho, double *mu,
                     double *rhof, double *chi)
{
    double hf = heav(sg, T->h), hb = heav(ps, T->h);
    double rf = T->P.rho_w + (T->P.rho_a - T->P.rho_w) * hf;
    double mf = T->P.mu_w + (T->P.mu_a - T->P.mu_w) * hf;
    if (rho) *rho = T->rho_s + (rf - T->rho_s) * hb;
    if (mu) *mu = T->mu_s + (mf - T->mu_s) * hb;
    if (rhof) *rhof = rf;
    if (chi) *chi = 1.0 - hb;
}

static void materials(const otank *T, const double *sg, double yc, double *rho, double *mu,
                      double *rhof, double *chi)
{
    int nx = T->P.nx, ny = T->P.ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double x = (i + 0.5) * T->h, y = (j + 0.5) * T->h;
            int c = j * nx + i;
            cell_mat(T, sg[c], psi_at(T, x, y, yc), rho ? rho + c : 0, mu ? mu + c : 0,
                     rhof ? rhof + c : 0, chi ? chi + c : 0);
        }
}

/* ------------------------------------------------------- ghost values -- */
/* sigma outside the domain.  Left: the incident wave's still-water-relative
 * distance y - d - eta(x, t); right: zero gradient; bottom/top: linear
 * extrapolation (keeps a signed distance's unit slope). */
static double sig_get(const otank *T, const double *s, int i, int j, double t)
{
    int nx = T->P.nx, ny = T->P.ny;
    if (i < 0) {
        double x = (i + 0.5) * T->h, y = (j + 0.5) * T->h;
        return y - T->P.depth - eta_at(T, x, t);
    }
    if (i > nx - 1) i = nx - 1;
    if (j < 0) return s[i] + j * (s[nx + i] - s[i]);
    if (j > ny - 1) {
        int m = j - (ny - 1);
        double a = s[(ny - 1) * nx + i], b = s[(ny - 2) * nx + i];
        return a + m * (a - b);
    }
    return s[j * nx + i];
}

/* u outside its array: nearest face (zero normal gradient / free slip). */
static double u_get(const otank *T, const double *u, int i, int j)
{
    int nx = T->P.nx, ny = T->P.ny;
    return u[clampi(j, 0, ny - 1) * (nx + 1) + clampi(i, 0, nx)];
}

/* v outside its array: bottom/top nearest face; right wall free slip;
 * left: odd reflection about the inflow tangential velocity v_in(y_j, t). */
static double v_get(const otank *T, const double *v, int i, int j, double t)
{
    int nx = T->P.nx, ny = T->P.ny;
    j = clampi(j, 0, ny);
    if (i > nx - 1) i = nx - 1;
    if (i < 0) {
        double ui, vi;
        airy_velocity(T, 0.0, j * T->h, t, &ui, &vi);
        return 2.0 * vi - v[j * nx + (-1 - i)];
    }
    return v[j * nx + i];
}

static double cell_get(const otank *T, const double *a, int i, int j)
{
    return a[clampi(j, 0, T->P.ny - 1) * T->P.nx + clampi(i, 0, T->P.nx - 1)];
}

/* -------------------------------------------------- sigma advection (PPM) -- */
static double vl_slope(double am, double a0, double ap)
{
    double dl = a0 - am, dr = ap - a0;
    if (dl * dr <= 0.0) return 0.0;
    double dc = 0.5 * (ap - am);
    double m = fmin(fabs(dc), fmin(2.0 * fabs(dl), 2.0 * fabs(dr)));
    return dc > 0.0 ? m : -m;
}

/* Colella-Woodward PPM edge values of the middle cell of a[0..4], limited. */
static void ppm_cell(const double *a, double *aL, double *aR)
{
    double dm = vl_slope(a[0], a[1], a[2]);
    double d0 = vl_slope(a[1], a[2], a[3]);
    double dp = vl_slope(a[2], a[3], a[4]);
    double L = a[1] + 0.5 * (a[2] - a[1]) - (d0 - dm) / 6.0;
    double R = a[2] + 0.5 * (a[3] - a[2]) - (dp - d0) / 6.0;
    double c = a[2];
    if ((R - c) * (c - L) <= 0.0) {
        L = c;
        R = c;
    } else {
        double dA = R - L;
        double m6 = dA * (c - 0.5 * (L + R));
        double q = dA * dA / 6.0;
        if (m6 > q)
            L = 3.0 * c - 2.0 * R;
        else if (-q > m6)
            R = 3.0 * c - 2.0 * L;
    }
    *aL = L;
    *aR = R;
}

/* Time-centred upwind state at a face; a[0..5] are the cells f-3 .. f+2, the
 * face lies between a[2] and a[3]. */
static double ppm_face(const double *a, double vel, double dt, double h)
{
    double L, R;
    if (vel >= 0.0) {
        ppm_cell(a, &L, &R);
        double C = vel * dt / h, dA = R - L, a6 = 6.0 * (a[2] - 0.5 * (L + R));
        return R - 0.5 * C * (dA - (1.0 - 2.0 * C / 3.0) * a6);
    } else {
        ppm_cell(a + 1, &L, &R);
        double C = -vel * dt / h, dA = R - L, a6 = 6.0 * (a[3] - 0.5 * (L + R));
        return L + 0.5 * C * (dA + (1.0 - 2.0 * C / 3.0) * a6);
    }
}

static double damp_alpha(const otank *T, double x)
{
    if (T->P.damp_len <= 0.0 || x <= T->P.damp_x0) return 0.0;
    double xi = (x - T->P.damp_x0) / T->P.damp_len;
    if (xi > 1.0) xi = 1.0;
    return (exp(pow(xi, 3.5)) - 1.0) / (exp(1.0) - 1.0);
}

/* sigma^{n+1,*} = sigma^n - dt Q(u^n, sigma^n), then the damping-zone relaxation
 * toward still water (Jacobsen weight).  Ghosts at time t (= t^n). */
static void advect(const otank *T, const double *s, const double *u, const double *v,
                   double dt, double t, double *out)
{
    int nx = T->P.nx, ny = T->P.ny;
    double h = T->h, a[6];
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double fx[2], fy[2];
            for (int f = 0; f < 2; ++f) {
                int fi = i + f;
                for (int q = 0; q < 6; ++q) a[q] = sig_get(T, s, fi - 3 + q, j, t);
                fx[f] = ppm_face(a, u[j * (nx + 1) + fi], dt, h);
                int fj = j + f;
                for (int q = 0; q < 6; ++q) a[q] = sig_get(T, s, i, fj - 3 + q, t);
                fy[f] = ppm_face(a, v[fj * nx + i], dt, h);
            }
            double ub = 0.5 * (u[j * (nx + 1) + i] + u[j * (nx + 1) + i + 1]);
            double vb = 0.5 * (v[j * nx + i] + v[(j + 1) * nx + i]);
            double Q = ub * (fx[1] - fx[0]) / h + vb * (fy[1] - fy[0]) / h;
            double sa = s[j * nx + i] - dt * Q;
            double al = damp_alpha(T, (i + 0.5) * h);
            double y = (j + 0.5) * h;
            out[j * nx + i] = (1.0 - al) * sa + al * (y - T->P.depth);
        }
}

/* ------------------------------------------------- reinitialisation -- */
static double minmod(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

/* Sussman relaxation: sigma_tau + S(sigma0)(|grad sigma| - 1) = 0, Godunov
 * Hamiltonian on ENO-2 one-sided differences. Returns S (|grad| - 1). */
static double reinit_rhs(const otank *T, const double *f, const double *s0, int i, int j,
                         double t)
{
    double h = T->h;
    double c = f[j * T->P.nx + i];
    double xm2 = sig_get(T, f, i - 2, j, t), xm1 = sig_get(T, f, i - 1, j, t);
    double xp1 = sig_get(T, f, i + 1, j, t), xp2 = sig_get(T, f, i + 2, j, t);
    double ym2 = sig_get(T, f, i, j - 2, t), ym1 = sig_get(T, f, i, j - 1, t);
    double yp1 = sig_get(T, f, i, j + 1, t), yp2 = sig_get(T, f, i, j + 2, t);
    double dxm = xm2 - 2.0 * xm1 + c, dx0 = xm1 - 2.0 * c + xp1, dxp = c - 2.0 * xp1 + xp2;
    double dym = ym2 - 2.0 * ym1 + c, dy0 = ym1 - 2.0 * c + yp1, dyp = c - 2.0 * yp1 + yp2;
    double a = (c - xm1) / h + minmod(dxm, dx0) / (2.0 * h);
    double b = (xp1 - c) / h - minmod(dx0, dxp) / (2.0 * h);
    double cc = (c - ym1) / h + minmod(dym, dy0) / (2.0 * h);
    double d = (yp1 - c) / h - minmod(dy0, dyp) / (2.0 * h);
    double sg0 = s0[j * T->P.nx + i];
    double S = sg0 / sqrt(sg0 * sg0 + h * h);
    double gx, gy;
    if (S > 0.0) {
        gx = fmax(sq(fmax(a, 0.0)), sq(fmin(b, 0.0)));
        gy = fmax(sq(fmax(cc, 0.0)), sq(fmin(d, 0.0)));
    } else {
        gx = fmax(sq(fmin(a, 0.0)), sq(fmax(b, 0.0)));
        gy = fmax(sq(fmin(cc, 0.0)), sq(fmax(d, 0.0)));
    }
    return S * (sqrt(gx + gy) - 1.0);
}

/* n_reinit TVD-RK2 pseudo-steps of size 0.3 h; sigma0 is the input. */
static void reinit(const otank *T, double *s, int nit, double t)
{
    int n = T->P.nx * T->P.ny, nx = T->P.nx;
    double dtau = REINIT_DTAU * T->h;
    double *s0 = dalloc(n), *s1 = dalloc(n), *s2 = dalloc(n);
    memcpy(s0, s, n * sizeof(double));
    for (int it = 0; it < nit; ++it) {
        for (int j = 0; j < T->P.ny; ++j)
            for (int i = 0; i < nx; ++i)
                s1[j * nx + i] = s[j * nx + i] - dtau * reinit_rhs(T, s, s0, i, j, t);
        for (int j = 0; j < T->P.ny; ++j)
            for (int i = 0; i < nx; ++i)
                s2[j * nx + i] = s1[j * nx + i] - dtau * reinit_rhs(T, s1, s0, i, j, t);
        for (int c = 0; c < n; ++c) s[c] = 0.5 * (s[c] + s2[c]);
    }
    free(s0);
    free(s1);
    free(s2);
}

/* ------------------------------------ consistent mass/momentum transport -- */
/* Koren-limited upwind face value from (far-upwind, upwind, downwind). */
static double koren(double quu, double qu, double qd)
{
    double d1 = qu - quu, d2 = qd - qu;
    if (d1 * d2 <= 0.0) return qu;
    double m = fmin(2.0 * fabs(d2), fmin((fabs(d1) + 2.0 * fabs(d2)) / 3.0, 2.0 * fabs(d1)));
    return d1 > 0.0 ? qu + 0.5 * m : qu - 0.5 * m;
}

/* Face between q1 (low side) and q2 (high side); q0, q3 are the next values out. */
static double upwind(double q0, double q1, double q2, double q3, double vel)
{
    return vel >= 0.0 ? koren(q0, q1, q2) : koren(q3, q2, q1);
}

typedef struct {
    const otank *T;
    const double *rc; /* cell density for the face averages */
    const double *u, *v;
    double t;
} tctx;

static double ru_get(const tctx *X, int i, int j)
{
    int nx = X->T->P.nx;
    i = clampi(i, 0, nx);
    j = clampi(j, 0, X->T->P.ny - 1);
    return 0.5 * (cell_get(X->T, X->rc, i - 1, j) + cell_get(X->T, X->rc, i, j));
}

static double rv_get(const tctx *X, int i, int j)
{
    int ny = X->T->P.ny;
    i = clampi(i, 0, X->T->P.nx - 1);
    j = clampi(j, 0, ny);
    return 0.5 * (cell_get(X->T, X->rc, i, j - 1) + cell_get(X->T, X->rc, i, j));
}

/* rho-breve and the convective term C for the u-face (i, j). */
static void transport_u(const tctx *X, int i, int j, double dt, double *rb, double *C)
{
    const otank *T = X->T;
    double h = T->h, m[4], f[4];
#define UU(a, b) u_get(T, X->u, a, b)
#define VV(a, b) v_get(T, X->v, a, b, X->t)
    /* east / west control-volume faces (at cell centres i and i-1) */
    for (int s = 0; s < 2; ++s) {
        int a = i - 1 + s; /* faces a and a+1 bound this CV face */
        double U = 0.5 * (UU(a, j) + UU(a + 1, j));
        double r = upwind(ru_get(X, a - 1, j), ru_get(X, a, j), ru_get(X, a + 1, j), ru_get(X, a + 2, j), U);
        double q = upwind(UU(a - 1, j), UU(a, j), UU(a + 1, j), UU(a + 2, j), U);
        m[s] = U * r;
        f[s] = m[s] * q;
    }
    /* south / north control-volume faces (at nodes (i, j) and (i, j+1)) */
    for (int s = 0; s < 2; ++s) {
        int b = j - 1 + s;
        double V = 0.5 * (VV(i - 1, b + 1) + VV(i, b + 1));
        double r = upwind(ru_get(X, i, b - 1), ru_get(X, i, b), ru_get(X, i, b + 1), ru_get(X, i, b + 2), V);
        double q = upwind(UU(i, b - 1), UU(i, b), UU(i, b + 1), UU(i, b + 2), V);
        m[2 + s] = V * r;
        f[2 + s] = m[2 + s] * q;
    }
    *rb = ru_get(X, i, j) - dt / h * ((m[1] - m[0]) + (m[3] - m[2]));
    *C = ((f[1] - f[0]) + (f[3] - f[2])) / h;
}

static void transport_v(const tctx *X, int i, int j, double dt, double *rb, double *C)
{
    const otank *T = X->T;
    double h = T->h, m[4], f[4];
    /* west / east control-volume faces (at nodes (i, j) and (i+1, j)) */
    for (int s = 0; s < 2; ++s) {
        int a = i - 1 + s;
        double U = 0.5 * (UU(a + 1, j - 1) + UU(a + 1, j));
        double r = upwind(rv_get(X, a - 1, j), rv_get(X, a, j), rv_get(X, a + 1, j), rv_get(X, a + 2, j), U);
        double q = upwind(VV(a - 1, j), VV(a, j), VV(a + 1, j), VV(a + 2, j), U);
        m[s] = U * r;
        f[s] = m[s] * q;
    }
    /* south / north control-volume faces (at cell centres j-1 and j) */
    for (int s = 0; s < 2; ++s) {
        int b = j - 1 + s;
        double V = 0.5 * (VV(i, b) + VV(i, b + 1));
        double r = upwind(rv_get(X, i, b - 1), rv_get(X, i, b), rv_get(X, i, b + 1), rv_get(X, i, b + 2), V);
        double q = upwind(VV(i, b - 1), VV(i, b), VV(i, b + 1), VV(i, b + 2), V);
        m[2 + s] = V * r;
        f[2 + s] = m[2 + s] * q;
    }
    *rb = rv_get(X, i, j) - dt / h * ((m[1] - m[0]) + (m[3] - m[2]));
    *C = ((f[1] - f[0]) + (f[3] - f[2])) / h;
#undef UU
#undef VV
}

/* ------------------------------------------------------- viscous term -- */
/* L_mu u = div[mu (grad u + grad u^T)] on the MAC grid: tau_xx, tau_yy at cell
 * centres, tau_xy at nodes with the four-cell mean viscosity. */
typedef struct {
    const otank *T;
    const double *mu, *u, *v;
    double t;
} vctx;

static double mnode(const vctx *X, int i, int j)
{
    return 0.25 * (cell_get(X->T, X->mu, i - 1, j - 1) + cell_get(X->T, X->mu, i, j - 1) +
                   cell_get(X->T, X->mu, i - 1, j) + cell_get(X->T, X->mu, i, j));
}

static double txx(const vctx *X, int i, int j)
{
    return 2.0 * cell_get(X->T, X->mu, i, j) *
           (u_get(X->T, X->u, i + 1, j) - u_get(X->T, X->u, i, j)) / X->T->h;
}

static double tyy(const vctx *X, int i, int j)
{
    return 2.0 * cell_get(X->T, X->mu, i, j) *
           (v_get(X->T, X->v, i, j + 1, X->t) - v_get(X->T, X->v, i, j, X->t)) / X->T->h;
}

static double txy(const vctx *X, int i, int j)
{
    double h = X->T->h;
    return mnode(X, i, j) * ((u_get(X->T, X->u, i, j) - u_get(X->T, X->u, i, j - 1)) / h +
                             (v_get(X->T, X->v, i, j, X->t) - v_get(X->T, X->v, i - 1, j, X->t)) / h);
}

static double visc_x(const vctx *X, int i, int j)
{
    double h = X->T->h;
    return (txx(X, i, j) - txx(X, i - 1, j)) / h + (txy(X, i, j + 1) - txy(X, i, j)) / h;
}

static double visc_y(const vctx *X, int i, int j)
{
    double h = X->T->h;
    return (tyy(X, i, j) - tyy(X, i, j - 1)) / h + (txy(X, i + 1, j) - txy(X, i, j)) / h;
}

/* Interior-formula diagonal of L_mu (used only as the Jacobi splitting). */
static double visc_diag_x(const vctx *X, int i, int j)
{
    double h = X->T->h;
    return -(2.0 * cell_get(X->T, X->mu, i, j) + 2.0 * cell_get(X->T, X->mu, i - 1, j) +
             mnode(X, i, j + 1) + mnode(X, i, j)) / (h * h);
}

static double visc_diag_y(const vctx *X, int i, int j)
{
    double h = X->T->h;
    return -(2.0 * cell_get(X->T, X->mu, i, j) + 2.0 * cell_get(X->T, X->mu, i, j - 1) +
             mnode(X, i + 1, j) + mnode(X, i, j)) / (h * h);
}

/* Vorticity damping coefficient g(z~) = rho_a (cos(pi z~) + 1) / (4 dt) over the
 * top four cells (Eq. spongelayer with z_max at the top of the domain). */
static double vort_damp(const otank *T, double y, double dt)
{
    double w = 4.0 * T->h;
    if (y < T->P.ly - w) return 0.0;
    double zt = (y - T->P.ly) / w;
    return T->P.rho_a * (cos(PI * zt) + 1.0) / (4.0 * dt);
}

/* ----------------------------------------------- pressure operator / MG -- */
/* A p = b with (A p)_c = sum_f beta_f (p_c - p_nb); walls (left, right, bottom)
 * are Neumann whatever their coefficient; the top face is Dirichlet p = 0 at
 * the face, i.e. a ghost -p_c, giving 2 beta_top p_c. */
typedef struct {
    int nx, ny;
    double *bu, *bv, *x, *b, *r;
} olev;

#define BU(L, i, j) ((L)->bu[(j) * ((L)->nx + 1) + (i)])
#define BV(L, i, j) ((L)->bv[(j) * (L)->nx + (i)])

static double op_diag(const olev *L, int i, int j)
{
    double d = 0.0;
    if (i > 0) d += BU(L, i, j);
    if (i < L->nx - 1) d += BU(L, i + 1, j);
    if (j > 0) d += BV(L, i, j);
    d += (j < L->ny - 1 ? 1.0 : 2.0) * BV(L, i, j + 1);
    return d;
}

static double op_offsum(const olev *L, const double *x, int i, int j)
{
    int nx = L->nx, c = j * nx + i;
    double s = 0.0;
    if (i > 0) s += BU(L, i, j) * x[c - 1];
    if (i < nx - 1) s += BU(L, i + 1, j) * x[c + 1];
    if (j > 0) s += BV(L, i, j) * x[c - nx];
    if (j < L->ny - 1) s += BV(L, i, j + 1) * x[c + nx];
    return s;
}

static void op_apply(const olev *L, const double *x, double *y)
{
    for (int j = 0; j < L->ny; ++j)
        for (int i = 0; i < L->nx; ++i)
            y[j * L->nx + i] = op_diag(L, i, j) * x[j * L->nx + i] - op_offsum(L, x, i, j);
}

static void rbgs(olev *L)
{
    for (int color = 0; color < 2; ++color)
        for (int j = 0; j < L->ny; ++j)
            for (int i = 0; i < L->nx; ++i)
                if (((i + j) & 1) == color) {
                    int c = j * L->nx + i;
                    L->x[c] = (L->b[c] + op_offsum(L, L->x, i, j)) / op_diag(L, i, j);
                }
}

/* Dense LU (no pivoting; A is a symmetric M-matrix) on the coarsest level. */
static void coarse_solve(olev *L)
{
    int n = L->nx * L->ny;
    double *A = dalloc((size_t)n * n), *y = dalloc(n), *e = dalloc(n), *col = dalloc(n);
    for (int k = 0; k < n; ++k) {
        memset(e, 0, n * sizeof(double));
        e[k] = 1.0;
        op_apply(L, e, col);
        for (int r = 0; r < n; ++r) A[r * n + k] = col[r];
    }
    for (int k = 0; k < n; ++k)
        for (int r = k + 1; r < n; ++r) {
            double f = A[r * n + k] / A[k * n + k];
            A[r * n + k] = f;
            for (int c = k + 1; c < n; ++c) A[r * n + c] -= f * A[k * n + c];
        }
    for (int r = 0; r < n; ++r) {
        double s = L->b[r];
        for (int c = 0; c < r; ++c) s -= A[r * n + c] * y[c];
        y[r] = s;
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = y[r];
        for (int c = r + 1; c < n; ++c) s -= A[r * n + c] * L->x[c];
        L->x[r] = s / A[r * n + r];
    }
    free(A);
    free(y);
    free(e);
    free(col);
}

typedef struct {
    int nlev, nu1, nu2;
    olev lev[32];
} ohier;

/* Coarsen by 2 in each direction while both sizes are even and at least 4.
 * Coarse face coefficient = mean of the two fine faces it covers. */
static void hier_build(ohier *H, int nx, int ny, const double *bu, const double *bv, int nu1, int nu2)
{
    H->nu1 = nu1;
    H->nu2 = nu2;
    H->nlev = 0;
    for (;;) {
        olev *L = &H->lev[H->nlev];
        L->nx = nx;
        L->ny = ny;
        L->bu = dalloc((size_t)(nx + 1) * ny);
        L->bv = dalloc((size_t)nx * (ny + 1));
        L->x = dalloc((size_t)nx * ny);
        L->b = dalloc((size_t)nx * ny);
        L->r = dalloc((size_t)nx * ny);
        if (H->nlev == 0) {
            memcpy(L->bu, bu, sizeof(double) * (nx + 1) * ny);
            memcpy(L->bv, bv, sizeof(double) * nx * (ny + 1));
        } else {
            olev *F = &H->lev[H->nlev - 1];
            for (int J = 0; J < ny; ++J)
                for (int I = 0; I <= nx; ++I)
                    BU(L, I, J) = 0.5 * (BU(F, 2 * I, 2 * J) + BU(F, 2 * I, 2 * J + 1));
            for (int J = 0; J <= ny; ++J)
                for (int I = 0; I < nx; ++I)
                    BV(L, I, J) = 0.5 * (BV(F, 2 * I, 2 * J) + BV(F, 2 * I + 1, 2 * J));
        }
        H->nlev++;
        if (nx % 2 || ny % 2 || nx < 4 || ny < 4 || H->nlev == 32) break;
        nx /= 2;
        ny /= 2;
    }
}

static void hier_free(ohier *H)
{
    for (int l = 0; l < H->nlev; ++l) {
        free(H->lev[l].bu);
        free(H->lev[l].bv);
        free(H->lev[l].x);
        free(H->lev[l].b);
        free(H->lev[l].r);
    }
}

/* One V(nu1, nu2) cycle on level l with zero initial guess. */
static void vcycle(ohier *H, int l)
{
    olev *L = &H->lev[l];
    int n = L->nx * L->ny;
    if (l == H->nlev - 1) {
        coarse_solve(L);
        return;
    }
    memset(L->x, 0, n * sizeof(double));
    for (int s = 0; s < H->nu1; ++s) rbgs(L);
    op_apply(L, L->x, L->r);
    for (int c = 0; c < n; ++c) L->r[c] = L->b[c] - L->r[c];
    olev *C = &H->lev[l + 1];
    for (int J = 0; J < C->ny; ++J)
        for (int I = 0; I < C->nx; ++I) {
            int nx = L->nx;
            C->b[J * C->nx + I] = L->r[(2 * J) * nx + 2 * I] + L->r[(2 * J) * nx + 2 * I + 1] +
                                  L->r[(2 * J + 1) * nx + 2 * I] + L->r[(2 * J + 1) * nx + 2 * I + 1];
        }
    vcycle(H, l + 1);
    for (int j = 0; j < L->ny; ++j)
        for (int i = 0; i < L->nx; ++i) L->x[j * L->nx + i] += C->x[(j / 2) * C->nx + i / 2];
    for (int s = 0; s < H->nu2; ++s) rbgs(L);
}

static double dot(const double *a, const double *b, int n)
{
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += a[c] * b[c];
    return s;
}

/* FGMRES(m), right-preconditioned by one V-cycle, classical Gram-Schmidt applied
 * twice, Givens rotations; converged when ||b - A x||_2 <= rtol ||b||_2 (the
 * true residual is recomputed at the end of every cycle). */
static int fgmres(ohier *H, const double *b, double *x, double rtol, int maxit, int m,
                  int *iters, double *relres)
{
    olev *L0 = &H->lev[0];
    int n = L0->nx * L0->ny;
    double bn = sqrt(dot(b, b, n));
    *iters = 0;
    if (bn == 0.0) {
        memset(x, 0, n * sizeof(double));
        *relres = 0.0;
        return 0;
    }
    double tol = rtol * bn;
    double *V = dalloc((size_t)(m + 1) * n), *Z = dalloc((size_t)m * n), *w = dalloc(n);
    double *Hm = dalloc((size_t)(m + 1) * m), *cs = dalloc(m), *sn = dalloc(m), *g = dalloc(m + 1);
    double *h1 = dalloc(m + 1), *y = dalloc(m);
    int its = 0, conv = 0;
    double beta;
    op_apply(L0, x, w);
    for (int c = 0; c < n; ++c) w[c] = b[c] - w[c];
    beta = sqrt(dot(w, w, n));
    if (beta <= tol) conv = 1;
    while (!conv && its < maxit) {
        for (int c = 0; c < n; ++c) V[c] = w[c] / beta;
        memset(g, 0, sizeof(double) * (m + 1));
        g[0] = beta;
        int jd = 0;
        for (int j = 0; j < m; ++j) {
            memcpy(L0->b, V + (size_t)j * n, n * sizeof(double));
            vcycle(H, 0);
            memcpy(Z + (size_t)j * n, L0->x, n * sizeof(double));
            op_apply(L0, Z + (size_t)j * n, w);
            its++;
            for (int k = 0; k <= j; ++k) Hm[k * m + j] = 0.0;
            for (int pass = 0; pass < 2; ++pass) {
                for (int k = 0; k <= j; ++k) h1[k] = dot(V + (size_t)k * n, w, n);
                for (int k = 0; k <= j; ++k) {
                    const double *vk = V + (size_t)k * n;
                    for (int c = 0; c < n; ++c) w[c] -= h1[k] * vk[c];
                    Hm[k * m + j] += h1[k];
                }
            }
            double hn = sqrt(dot(w, w, n));
            Hm[(j + 1) * m + j] = hn;
            for (int k = 0; k < j; ++k) {
                double a = Hm[k * m + j], bb = Hm[(k + 1) * m + j];
                Hm[k * m + j] = cs[k] * a + sn[k] * bb;
                Hm[(k + 1) * m + j] = -sn[k] * a + cs[k] * bb;
            }
            double a = Hm[j * m + j], bb = Hm[(j + 1) * m + j];
            double den = sqrt(a * a + bb * bb);
            cs[j] = a / den;
            sn[j] = bb / den;
            Hm[j * m + j] = den;
            Hm[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            jd = j + 1;
            if (fabs(g[j + 1]) <= tol || its >= maxit || hn == 0.0) break;
            for (int c = 0; c < n; ++c) V[(size_t)(j + 1) * n + c] = w[c] / hn;
        }
        for (int k = jd - 1; k >= 0; --k) {
            double s = g[k];
            for (int l = k + 1; l < jd; ++l) s -= Hm[k * m + l] * y[l];
            y[k] = s / Hm[k * m + k];
        }
        for (int k = 0; k < jd; ++k) {
            const double *zk = Z + (size_t)k * n;
            for (int c = 0; c < n; ++c) x[c] += y[k] * zk[c];
        }
        op_apply(L0, x, w);
        for (int c = 0; c < n; ++c) w[c] = b[c] - w[c];
        beta = sqrt(dot(w, w, n));
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
    free(h1);
    free(y);
    return conv ? 0 : 3;
}

/* --------------------------------------------------- hydrodynamic force -- */
/* Eq. int_fh, heave component, over faces whose two cells have opposite body-SDF
 * sign (the paper's face identification uses the body SDF psi).  Pressure at the
 * face is interpolated to the psi = 0 crossing with |psi| weights; the viscous
 * traction uses central differences at the face.  n_f points out of the body. */
static double hydro_force(const otank *T, const double *mu)
{
    int nx = T->P.nx, ny = T->P.ny;
    double h = T->h, F = 0.0;
    if (!T->P.has_body) return 0.0;
    for (int j = 1; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double x = (i + 0.5) * h;
            double pl = psi_at(T, x, (j - 0.5) * h, T->yc), pr = psi_at(T, x, (j + 0.5) * h, T->yc);
            if (!(pl * pr < 0.0)) continue;
            double ny_ = pl < 0.0 ? 1.0 : -1.0;
            double wl = fabs(pl), wr = fabs(pr);
            double pf = (T->p[(j - 1) * nx + i] * wr + T->p[j * nx + i] * wl) / (wl + wr);
            double muf = 0.5 * (mu[(j - 1) * nx + i] + mu[j * nx + i]);
            double dvdy = (v_get(T, T->v, i, j + 1, T->t) - v_get(T, T->v, i, j - 1, T->t)) / (2.0 * h);
            F += (-pf * ny_ + muf * 2.0 * dvdy * ny_) * h;
        }
    for (int j = 0; j < ny; ++j)
        for (int i = 1; i < nx; ++i) {
            double y = (j + 0.5) * h;
            double pl = psi_at(T, (i - 0.5) * h, y, T->yc), pr = psi_at(T, (i + 0.5) * h, y, T->yc);
            if (!(pl * pr < 0.0)) continue;
            double nx_ = pl < 0.0 ? 1.0 : -1.0;
            double muf = 0.5 * (mu[j * nx + i - 1] + mu[j * nx + i]);
            double dvdx = 0.5 * ((v_get(T, T->v, i, j, T->t) - v_get(T, T->v, i - 1, j, T->t)) +
                                 (v_get(T, T->v, i, j + 1, T->t) - v_get(T, T->v, i - 1, j + 1, T->t))) / h;
            double dudy = (u_get(T, T->u, i, j + 1) - u_get(T, T->u, i, j - 1)) / (2.0 * h);
            F += muf * (dvdx + dudy) * nx_ * h;
        }
    return F;
}

/* ------------------------------------------------------------ the step -- */
int oracle_step(void *handle, double dt, double f_pto_in, oracle_result *out)
{
    otank *T = (otank *)handle;
    int nx = T->P.nx, ny = T->P.ny, n = nx * ny;
    int nu = (nx + 1) * ny, nv = nx * (ny + 1);
    double h = T->h, t0 = T->t, t1 = T->t + dt;
    double *rho_n = dalloc(n), *mu_n = dalloc(n), *mu_1 = dalloc(n), *rf_1 = dalloc(n), *chi_1 = dalloc(n);
    double *Ru = dalloc(nu), *Rv = dalloc(nv), *Du = dalloc(nu), *Dv = dalloc(nv);
    double *ua = dalloc(nu), *va = dalloc(nv), *ub = dalloc(nu), *vb = dalloc(nv);

    /* (1) force on the body from p^{n-1/2}, u^n (cycle 0 = previous step), Eq. int_fh */
    materials(T, T->sig, T->yc, rho_n, mu_n, 0, 0);
    double F = hydro_force(T, mu_n);

    /* (2) heave, Eq. newton_u; the linear PTO damper acts on zdot^n.  Reading: with
     * the force taken from the previous step (n_cycles = 1) the update is unstable
     * once the added mass exceeds m, so an artificial added mass m_a is carried on
     * both sides: (m + m_a)(zdot^{n+1} - zdot^n) = dt (F - m g + F_PTO)
     *                                              + m_a (zdot^n - zdot^{n-1}).
     * m_a = 0 is Eq. newton_u exactly; the extra terms cancel for smooth motion. */
    double fpto = f_pto_in - T->P.pto_damping * T->zdot;
    double zd1 = T->zdot, yc1 = T->yc;
    if (T->P.has_body) {
        double m = T->P.body_mass, ma = T->P.added_mass;
        zd1 = T->zdot + (dt * (F - m * T->P.g + fpto) + ma * (T->zdot - T->zdot_prev)) / (m + ma);
        yc1 = T->yc + 0.5 * dt * (T->zdot + zd1);
    }

    /* (3) sigma: advection + damping-zone relaxation, then reinitialisation */
    advect(T, T->sig, T->u, T->v, dt, t0, T->sig_adv);
    double *sig1 = dalloc(n);
    memcpy(sig1, T->sig_adv, n * sizeof(double));
    reinit(T, sig1, T->P.n_reinit, t1);

    /* (4) materials at n+1 (psi analytic at the new body position) */
    materials(T, sig1, yc1, 0, mu_1, rf_1, chi_1);

    /* (5) consistent transport and momentum right-hand side */
    tctx X = {T, rho_n, T->u, T->v, t0};
    vctx Vn = {T, mu_n, T->u, T->v, t0};
    for (int j = 0; j < ny; ++j)
        for (int i = 1; i < nx; ++i) {
            int f = j * (nx + 1) + i;
            double rb, C;
            transport_u(&X, i, j, dt, &rb, &C);
            double x = i * h, y = (j + 0.5) * h;
            double chi = 0.5 * (cell_get(T, chi_1, i - 1, j) + cell_get(T, chi_1, i, j));
            T->rbu[f] = rb;
            Du[f] = rb / dt + chi / T->P.kappa_p + damp_alpha(T, x) * rb / dt + vort_damp(T, y, dt);
            Ru[f] = ru_get(&X, i, j) * T->u[f] / dt - C + 0.5 * visc_x(&Vn, i, j) -
                    (T->p[j * nx + i] - T->p[j * nx + i - 1]) / h;
        }
    for (int j = 1; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int f = j * nx + i;
            double rb, C;
            transport_v(&X, i, j, dt, &rb, &C);
            double x = (i + 0.5) * h, y = j * h;
            double chi = 0.5 * (cell_get(T, chi_1, i, j - 1) + cell_get(T, chi_1, i, j));
            double rf = 0.5 * (cell_get(T, rf_1, i, j - 1) + cell_get(T, rf_1, i, j));
            T->rbv[f] = rb;
            Dv[f] = rb / dt + chi / T->P.kappa_p + damp_alpha(T, x) * rb / dt + vort_damp(T, y, dt);
            /* pressure gradient of p^{n+1/2,0} = p^{n-1/2}; top face: p = 0 beyond it */
            double gp = j < ny ? (T->p[j * nx + i] - T->p[(j - 1) * nx + i]) / h
                               : -2.0 * T->p[(ny - 1) * nx + i] / h;
            Rv[f] = rv_get(&X, i, j) * T->v[f] / dt - C + 0.5 * visc_y(&Vn, i, j) - rf * T->P.g +
                    chi * zd1 / T->P.kappa_p - gp;
        }

    /* (6) Crank-Nicolson implicit half by Jacobi sweeps; Dirichlet faces at n+1 */
    memcpy(ua, T->u, nu * sizeof(double));
    memcpy(va, T->v, nv * sizeof(double));
    for (int j = 0; j < ny; ++j) {
        double uin, vin;
        airy_velocity(T, 0.0, (j + 0.5) * h, t1, &uin, &vin);
        ua[j * (nx + 1)] = uin;
        ua[j * (nx + 1) + nx] = 0.0;
    }
    for (int i = 0; i < nx; ++i) va[i] = 0.0;
    memcpy(ub, ua, nu * sizeof(double));
    memcpy(vb, va, nv * sizeof(double));
    for (int it = 0; it < T->P.n_jacobi; ++it) {
        vctx Vk = {T, mu_1, ua, va, t1};
        for (int j = 0; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                int f = j * (nx + 1) + i;
                double ld = visc_diag_x(&Vk, i, j);
                ub[f] = (Ru[f] + 0.5 * (visc_x(&Vk, i, j) - ld * ua[f])) / (Du[f] - 0.5 * ld);
            }
        for (int j = 1; j <= ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int f = j * nx + i;
                double ld = visc_diag_y(&Vk, i, j);
                vb[f] = (Rv[f] + 0.5 * (visc_y(&Vk, i, j) - ld * va[f])) / (Dv[f] - 0.5 * ld);
            }
        memcpy(ua, ub, nu * sizeof(double));
        memcpy(va, vb, nv * sizeof(double));
    }
    memcpy(T->us, ua, nu * sizeof(double));
    memcpy(T->vs, va, nv * sizeof(double));

    /* (7) pressure increment: A phi = b with beta_f = 1 / D_f, b = -h div u*,
     * phi from zero; p^{n+1/2} = p^{n-1/2} + phi */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            int f = j * (nx + 1) + i;
            T->bu[f] = (i == 0 || i == nx) ? 0.0 : 1.0 / Du[f];
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int f = j * nx + i;
            T->bv[f] = j == 0 ? 0.0 : 1.0 / Dv[f];
        }
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            T->rhs[j * nx + i] = -h * (T->us[j * (nx + 1) + i + 1] - T->us[j * (nx + 1) + i] +
                                       T->vs[(j + 1) * nx + i] - T->vs[j * nx + i]);
    ohier Hh;
    hier_build(&Hh, nx, ny, T->bu, T->bv, T->P.mg_pre, T->P.mg_post);
    int iters = 0;
    double relres = 0.0;
    double *phi = dalloc(n);
    int st = fgmres(&Hh, T->rhs, phi, T->P.rtol, T->P.max_iters, T->P.restart, &iters, &relres);
    hier_free(&Hh);

    /* (8) projection, Eq. c_discrete_continuity: u^{n+1} = u* - beta grad phi */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            int f = j * (nx + 1) + i;
            double uu = T->us[f];
            if (i > 0 && i < nx) uu -= T->bu[f] * (phi[j * nx + i] - phi[j * nx + i - 1]) / h;
            T->u[f] = uu;
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int f = j * nx + i;
            double vv = T->vs[f];
            if (j > 0 && j < ny) vv -= T->bv[f] * (phi[j * nx + i] - phi[(j - 1) * nx + i]) / h;
            if (j == ny) vv += 2.0 * T->bv[f] * phi[(ny - 1) * nx + i] / h;
            T->v[f] = vv;
        }
    for (int c = 0; c < n; ++c) T->p[c] += phi[c];
    free(phi);

    memcpy(T->sig, sig1, n * sizeof(double));
    T->t = t1;
    T->yc = yc1;
    T->zdot_prev = T->zdot;
    T->zdot = zd1;

    /* diagnostics: ||h div u||_2 and the surface elevation at the probe column */
    double dn = 0.0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            dn += sq(h * (T->u[j * (nx + 1) + i + 1] - T->u[j * (nx + 1) + i] + T->v[(j + 1) * nx + i] -
                          T->v[j * nx + i]));
    int ip = clampi((int)floor(T->P.probe_x / h), 0, nx - 1);
    double eta = NAN;
    for (int j = 0; j + 1 < ny; ++j) {
        double a = T->sig[j * nx + ip], b = T->sig[(j + 1) * nx + ip];
        if (a < 0.0 && b >= 0.0) {
            eta = (j + 0.5) * h + h * a / (a - b) - T->P.depth;
            break;
        }
    }
    if (out) {
        out->t = T->t;
        out->z = T->yc - T->yc0;
        out->zdot = T->zdot;
        out->f_hydro = F;
        out->f_pto = fpto;
        out->eta_probe = eta;
        out->residual = relres;
        out->div_norm = sqrt(dn);
        out->iters = iters;
    }
    free(rho_n); free(mu_n); free(mu_1); free(rf_1); free(chi_1);
    free(Ru); free(Rv); free(Du); free(Dv); free(ua); free(va); free(ub); free(vb); free(sig1);
    return st;
}

/* ------------------------------------------------------------ lifecycle -- */
void *oracle_create(const oracle_params *P)
{
    if (P->nx < 4 || P->ny < 4) return 0;
    otank *T = (otank *)calloc(1, sizeof(otank));
    T->P = *P;
    T->h = P->lx / P->nx;
    int nc = P->ncomp;
    T->amp = dalloc(nc);
    T->omega = dalloc(nc);
    T->kw = dalloc(nc);
    T->phase = dalloc(nc);
    for (int c = 0; c < nc; ++c) {
        T->amp[c] = P->amp[c];
        T->omega[c] = P->omega[c];
        T->kw[c] = P->kwave[c];
        T->phase[c] = P->phase[c];
    }
    T->P.amp = T->P.omega = T->P.kwave = T->P.phase = 0;
    /* Reading: solid density = mass / body area (uniform body), solid viscosity = water's. */
    T->rho_s = P->has_body ? P->body_mass / (P->body_w * P->body_h) : P->rho_w;
    T->mu_s = P->mu_w;
    T->yc = T->yc0 = P->body_yc;
    int nx = P->nx, ny = P->ny, n = nx * ny, nu = (nx + 1) * ny, nv = nx * (ny + 1);
    T->sig = dalloc(n); T->p = dalloc(n); T->u = dalloc(nu); T->v = dalloc(nv);
    T->sig_adv = dalloc(n); T->us = dalloc(nu); T->vs = dalloc(nv);
    T->bu = dalloc(nu); T->bv = dalloc(nv); T->rhs = dalloc(n); T->rbu = dalloc(nu); T->rbv = dalloc(nv);
    double h = T->h;
    /* initial state: sigma = y - (d + eta(x, 0)); Airy velocities; p = 0 */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            T->sig[j * nx + i] = (j + 0.5) * h - P->depth - eta_at(T, (i + 0.5) * h, 0.0);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            double uu, vv;
            airy_velocity(T, i * h, (j + 0.5) * h, 0.0, &uu, &vv);
            T->u[j * (nx + 1) + i] = (i == nx) ? 0.0 : uu;
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double uu, vv;
            airy_velocity(T, (i + 0.5) * h, j * h, 0.0, &uu, &vv);
            T->v[j * nx + i] = (j == 0) ? 0.0 : vv;
        }
    /* p^{-1/2}: the discrete hydrostatic pressure of the flow density, i.e. the
     * p that balances gravity at every y-face (p = 0 at the top face):
     * p_{ny-1} = rho_f(top) g h / 2, p_{j-1} = p_j + rho_f(face j) g h. */
    double *rf = dalloc(n);
    materials(T, T->sig, T->yc, 0, 0, rf, 0);
    for (int i = 0; i < nx; ++i) {
        double pj = 0.5 * rf[(ny - 1) * nx + i] * P->g * h;
        T->p[(ny - 1) * nx + i] = pj;
        for (int j = ny - 1; j >= 1; --j) {
            pj += 0.5 * (rf[(j - 1) * nx + i] + rf[j * nx + i]) * P->g * h;
            T->p[(j - 1) * nx + i] = pj;
        }
    }
    free(rf);
    return T;
}

void oracle_destroy(void *handle)
{
    otank *T = (otank *)handle;
    if (!T) return;
    free(T->amp); free(T->omega); free(T->kw); free(T->phase);
    free(T->sig); free(T->p); free(T->u); free(T->v); free(T->sig_adv); free(T->us); free(T->vs);
    free(T->bu); free(T->bv); free(T->rhs); free(T->rbu); free(T->rbv);
    free(T);
}

static double *field_ptr(otank *T, int f, size_t *n)
{
    size_t nc = (size_t)T->P.nx * T->P.ny, nu = (size_t)(T->P.nx + 1) * T->P.ny,
           nv = (size_t)T->P.nx * (T->P.ny + 1);
    switch (f) {
    case OF_SIGMA: *n = nc; return T->sig;
    case OF_U: *n = nu; return T->u;
    case OF_V: *n = nv; return T->v;
    case OF_P: *n = nc; return T->p;
    case OF_USTAR: *n = nu; return T->us;
    case OF_VSTAR: *n = nv; return T->vs;
    case OF_BETA_U: *n = nu; return T->bu;
    case OF_BETA_V: *n = nv; return T->bv;
    case OF_RHS: *n = nc; return T->rhs;
    case OF_SIGMA_ADV: *n = nc; return T->sig_adv;
    case OF_RHOB_U: *n = nu; return T->rbu;
    case OF_RHOB_V: *n = nv; return T->rbv;
    }
    *n = 0;
    return 0;
}

int oracle_get(void *handle, int f, double *dst)
{
    size_t n;
    double *p = field_ptr((otank *)handle, f, &n);
    if (!p) return 1;
    memcpy(dst, p, n * sizeof(double));
    return 0;
}

int oracle_set(void *handle, int f, const double *src)
{
    size_t n;
    double *p = field_ptr((otank *)handle, f, &n);
    if (!p) return 1;
    memcpy(p, src, n * sizeof(double));
    return 0;
}

void oracle_get_body(void *handle, double *out5)
{
    otank *T = (otank *)handle;
    out5[0] = T->t;
    out5[1] = T->yc;
    out5[2] = T->zdot;
    out5[3] = T->yc0;
    out5[4] = T->zdot_prev;
}

void oracle_set_body(void *handle, double t, double yc, double zdot, double zdot_prev)
{
    otank *T = (otank *)handle;
    T->t = t;
    T->yc = yc;
    T->zdot = zdot;
    T->zdot_prev = zdot_prev;
}

/* ---------------------------------------------- pieces, for the pin tests -- */
void oracle_advect(void *handle, double dt)
{
    otank *T = (otank *)handle;
    int n = T->P.nx * T->P.ny;
    advect(T, T->sig, T->u, T->v, dt, T->t, T->sig_adv);
    memcpy(T->sig, T->sig_adv, n * sizeof(double));
}

void oracle_reinit(void *handle, int nit)
{
    otank *T = (otank *)handle;
    reinit(T, T->sig, nit, T->t);
}

void oracle_materials(void *handle, double *rho, double *mu, double *rhof, double *chi)
{
    otank *T = (otank *)handle;
    materials(T, T->sig, T->yc, rho, mu, rhof, chi);
}

double oracle_heaviside(double phi, double eps) { return heav(phi, eps); }

void oracle_inflow(void *handle, double x, double y, double t, double *uv)
{
    airy_velocity((otank *)handle, x, y, t, uv, uv + 1);
}

void oracle_transport(void *handle, const double *rho_cell, double dt, double *rb_u, double *rb_v,
                      double *C_u, double *C_v)
{
    otank *T = (otank *)handle;
    int nx = T->P.nx, ny = T->P.ny;
    tctx X = {T, rho_cell, T->u, T->v, T->t};
    for (int j = 0; j < ny; ++j)
        for (int i = 1; i < nx; ++i)
            transport_u(&X, i, j, dt, rb_u + j * (nx + 1) + i, C_u + j * (nx + 1) + i);
    for (int j = 1; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) transport_v(&X, i, j, dt, rb_v + j * nx + i, C_v + j * nx + i);
}

void oracle_viscous(void *handle, const double *mu_cell, double *Lx, double *Ly)
{
    otank *T = (otank *)handle;
    int nx = T->P.nx, ny = T->P.ny;
    vctx X = {T, mu_cell, T->u, T->v, T->t};
    for (int j = 0; j < ny; ++j)
        for (int i = 1; i < nx; ++i) Lx[j * (nx + 1) + i] = visc_x(&X, i, j);
    for (int j = 1; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) Ly[j * nx + i] = visc_y(&X, i, j);
}

double oracle_force(void *handle)
{
    otank *T = (otank *)handle;
    double *mu = dalloc((size_t)T->P.nx * T->P.ny);
    materials(T, T->sig, T->yc, 0, mu, 0, 0);
    double F = hydro_force(T, mu);
    free(mu);
    return F;
}

/* Standalone pressure operator / solver on caller coefficients. */
void oracle_poisson_apply(int nx, int ny, const double *bu, const double *bv, const double *x, double *y)
{
    olev L = {nx, ny, (double *)bu, (double *)bv, 0, 0, 0};
    op_apply(&L, x, y);
}

int oracle_poisson_solve(int nx, int ny, const double *bu, const double *bv, const double *b, double *x,
                         double rtol, int maxit, int restart, int nu1, int nu2, int *iters, double *relres)
{
    ohier H;
    hier_build(&H, nx, ny, bu, bv, nu1, nu2);
    int st = fgmres(&H, b, x, rtol, maxit, restart, iters, relres);
    hier_free(&H);
    return st;
}

/* One V-cycle from a zero guess: x = M^{-1} b.  Returns the number of levels. */
int oracle_vcycle(int nx, int ny, const double *bu, const double *bv, int nu1, int nu2, const double *b,
                  double *x)
{
    ohier H;
    hier_build(&H, nx, ny, bu, bv, nu1, nu2);
    memcpy(H.lev[0].b, b, sizeof(double) * nx * ny);
    vcycle(&H, 0);
    memcpy(x, H.lev[0].x, sizeof(double) * nx * ny);
    int nl = H.nlev;
    hier_free(&H);
    return nl;
}


/* ---------------------------------------------------------------- NLFK ----
 * Non-linear Froude-Krylov force on a static grid (section "Non-linear
 * Froude-Krylov (NLFK) forces: A novel static grid approach based on implicit
 * surfaces"): on a box region R of cells around the body, sigma = y - (d + eta(x,
 * t)) marks water (sigma <= 0) and the body SDF psi marks the body; the incident
 * pressure of Eq. p_dynamic (mode 0, summed over the wave components) or the
 * hydrostatic p_H = -rho_w g z, z = y - d (mode 1, the nonlinear-buoyancy
 * variant) is zero where sigma > 0.  Eq. NLFK_p: F = sum over the faces whose two
 * cells have opposite psi sign of -p_f n_f h, p_f interpolated to psi = 0 with
 * |psi| weights (the same reading of the garbled sigma/psi wording as the heave
 * force), n_f out of the body.  y-faces give the heave force, x-faces the surge.
 * cosh(k (d + sigma)) / cosh(k d) is evaluated in an overflow-free form. */
static double nlfk_p(const oracle_nlfk_params *P, double x, double y, double t, int mode)
{
    double eta = 0.0;
    for (int c = 0; c < P->ncomp; ++c) eta += P->amp[c] * cos(P->kwave[c] * x - P->omega[c] * t + P->phase[c]);
    double sigma = y - (P->depth + eta);
    if (sigma > 0.0) return 0.0;
    if (mode == 1) return -P->rho_w * P->g * (y - P->depth);
    double p = 0.0;
    for (int c = 0; c < P->ncomp; ++c) {
        double k = P->kwave[c], d = P->depth;
        /* cosh(k (d + sigma)) / cosh(k d) = (e^{k sigma} + e^{-k (2 d + sigma)}) / (1 + e^{-2 k d}) */
        double ratio = (exp(k * sigma) + exp(-k * (2.0 * d + sigma))) / (1.0 + exp(-2.0 * k * d));
        p += P->rho_w * P->g * P->amp[c] * ratio * cos(k * x - P->omega[c] * t + P->phase[c]);
    }
    return p;
}

static double nlfk_psi(const oracle_nlfk_params *P, double x, double y, double yc)
{
    double a = fabs(x - P->body_xc) - 0.5 * P->body_w, b = fabs(y - yc) - 0.5 * P->body_h;
    return a > b ? a : b;
}

int oracle_nlfk(const oracle_nlfk_params *P, double t, double yc, int mode, double *fx, double *fy)
{
    const double h = P->h;
    double sx = 0.0, sy = 0.0;
    for (int j = 1; j < P->ny; ++j) /* y-faces between cells (i, j-1) and (i, j) */
        for (int i = 0; i < P->nx; ++i) {
            double x = P->x0 + (i + 0.5) * h, yl = P->y0 + (j - 0.5) * h, yr = P->y0 + (j + 0.5) * h;
            double pl = nlfk_psi(P, x, yl, yc), pr = nlfk_psi(P, x, yr, yc);
            if (!(pl * pr < 0.0)) continue;
            double wl = fabs(pl), wr = fabs(pr);
            double pf = (nlfk_p(P, x, yl, t, mode) * wr + nlfk_p(P, x, yr, t, mode) * wl) / (wl + wr);
            double ny = pl < 0.0 ? 1.0 : -1.0; /* out of the body */
            sy += -pf * ny * h;
        }
    for (int j = 0; j < P->ny; ++j) /* x-faces between cells (i-1, j) and (i, j) */
        for (int i = 1; i < P->nx; ++i) {
            double y = P->y0 + (j + 0.5) * h, xl = P->x0 + (i - 0.5) * h, xr = P->x0 + (i + 0.5) * h;
            double pl = nlfk_psi(P, xl, y, yc), pr = nlfk_psi(P, xr, y, yc);
            if (!(pl * pr < 0.0)) continue;
            double wl = fabs(pl), wr = fabs(pr);
            double pf = (nlfk_p(P, xl, y, t, mode) * wr + nlfk_p(P, xr, y, t, mode) * wl) / (wl + wr);
            double nx = pl < 0.0 ? 1.0 : -1.0;
            sx += -pf * nx * h;
        }
    *fx = sx;
    *fy = sy;
    return 0;
}
