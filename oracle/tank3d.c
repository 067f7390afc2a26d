/* tank3d.c -- TEST INFRASTRUCTURE ONLY: the plain FP64 CPU oracle of one time
 * step of the three-dimensional tank (sections "Continuous equations of motion"
 * through "Fluid-structure coupling" with d = 3), used by tests/ to check the
 * GPU library.  It shares no code with the GPU path; it calls the oracle's own
 * 3D level-set functions (levelset3d.c) and pressure solver (poisson3d.c).
 *
 * Grid nx x ny x nz, z vertical, still water at z = depth, waves along x.
 * Layouts, x fastest: cells [nz][ny][nx]; u [nz][ny][nx+1]; v [nz][ny+1][nx];
 * w [nz+1][ny][nx].  The step is the two-dimensional one (same order, same
 * readings) with three velocity components:
 *   (1) heave force from p^{n-1/2}, u^n (Eq. int_fh over the faces whose cells
 *       have opposite psi sign: pressure interpolated to psi = 0 and the normal
 *       viscous stress on z-faces, the shear stresses on x- and y-faces; face
 *       area h^2), (2) heave update with the artificial added mass of the 2D
 *       reading (here rho_w pi R^2 L), (3) sigma advection + damping zone, then
 *       reinitialisation, (4) materials at n+1, (5) consistent transport (Koren-
 *       limited upwind mass flux carrying the Koren-limited upwind velocity; the
 *       three pairs of control-volume faces summed x, then y, then z) and the
 *       momentum system: D = rho_breve / dt + chi / kappa_p + alpha rho_breve / dt
 *       + vorticity damping; R = rho u / dt - C + L_mu u / 2 - grad p^{n-1/2}
 *       (+ for w: - rho^flow g + chi zdot^{n+1} / kappa_p), (6) Crank-Nicolson
 *       Jacobi sweeps (Dirichlet: inflow u at x = 0, u = 0 at the outlet, v = 0 on
 *       the side walls, w = 0 on the bed; the top w face is solved), (7) the
 *       pressure increment A phi = -h div u* with beta_f = 1 / D_f (Neumann walls
 *       and bed, Dirichlet top) from zero, (8) projection and p += phi.
 *   Velocity ghosts: nearest face (free slip) except at the inflow, where v and
 *   w are reflected oddly about the incident wave's tangential velocity (0 for
 *   v).  Viscosity on edges: the mean of the four cells around the edge.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Loops whose iterations are independent (each writes only its own output
 * element; no reduction) may run on several host threads; every reduction and
 * every order-dependent loop stays serial, so results do not depend on the
 * thread count. */
#ifdef _OPENMP
#include <omp.h>
#define ORACLE_PAR_FOR _Pragma("omp parallel for schedule(static)")
#else
#define ORACLE_PAR_FOR
#endif

/* Host threads of the marked loops of every oracle file: n > 0 sets the count;
 * returns the count in use (1 when built without OpenMP). */
int oracle_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

#define PIT 3.14159265358979323846

/* the level-set oracle's parameter block (levelset3d.c) */
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

void oracle3_materials(const oracle3_tank *P, const double *sg, double zc, double *rho, double *mu, double *rhof,
                       double *chi);
void oracle3_advect(const oracle3_tank *P, const double *s, const double *u, const double *v, const double *w,
                    double dt, double t, double *out);
void oracle3_advect_half(const oracle3_tank *P, const double *base, const double *s, const double *u, const double *v,
                         const double *w, double dt, double ta, double tb, double *out);
void oracle3_reinit(const oracle3_tank *P, double *s, int nit, double t);
int oracle3_poisson_solve(int nx, int ny, int nz, const double *bx, const double *by, const double *bz,
                          const double *b, double *x, double rtol, int maxit, int restart, int nu1, int nu2,
                          int *iters, double *relres);

typedef struct {
    oracle3_tank L;
    double g, kappa_p, added_mass, pto_damping, probe_x, lz;
    double rtol;
    int max_iters, restart, n_reinit, n_jacobi, mg_pre, mg_post;
    int n_cycles; /* fixed-point cycles per step (section "Time stepping scheme"); 0 or 1: one */
} oracle3_params;

typedef struct {
    double t, z, zdot, f_hydro, f_pto, eta_probe, residual, div_norm, rhs_norm;
    int iters;
} oracle3_result;

typedef struct {
    oracle3_params P;
    double h, t, zc, zc0, zdot, zdot_prev;
    double *sig, *u, *v, *w, *p;
} o3tank;

/* ------------------------------------------------------------- helpers -- */
static int cl3(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }
static double sqt(double a) { return a * a; }

static double heavt(double phi, double eps)
{
    if (phi < -eps) return 0.0;
    if (phi > eps) return 1.0;
    return 0.5 * (1.0 + phi / eps + sin(PIT * phi / eps) / PIT);
}

static double etat(const o3tank *T, double x, double t)
{
    double e = 0.0;
    for (int c = 0; c < T->P.L.ncomp; ++c)
        e += T->P.L.amp[c] * cos(T->P.L.kwave[c] * x - T->P.L.omega[c] * t + T->P.L.phase[c]);
    return e;
}

/* Airy velocity (u, w) at (x, z, t): linear potential with Wheeler stretching up
 * to the surface, blended to zero in the air (the 2D reading). */
static void airyt(const o3tank *T, double x, double z, double t, double *uo, double *wo)
{
    double d = T->P.L.depth, e = etat(T, x, t);
    double zs = z < d + e ? z : d + e;
    double zp = d * zs / (d + e);
    double blend = 1.0 - heavt(z - d - e, T->h);
    double su = 0.0, sw = 0.0;
    for (int c = 0; c < T->P.L.ncomp; ++c) {
        double k = T->P.L.kwave[c], om = T->P.L.omega[c];
        double ph = k * x - om * t + T->P.L.phase[c], sk = sinh(k * d);
        su += T->P.L.amp[c] * om * cosh(k * zp) / sk * cos(ph);
        sw += T->P.L.amp[c] * om * sinh(k * zp) / sk * sin(ph);
    }
    *uo = blend * su;
    *wo = blend * sw;
}

static double psit(const o3tank *T, double x, double y, double z, double zc)
{
    if (!T->P.L.has_body) return 1.0e3;
    double r = sqrt(sqt(x - T->P.L.body_xc) + sqt(y - T->P.L.body_yc));
    return fmax(r - T->P.L.body_r, fabs(z - zc) - 0.5 * T->P.L.body_len);
}

#define NX (T->P.L.nx)
#define NY (T->P.L.ny)
#define NZ (T->P.L.nz)
#define CI(i, j, k) (((size_t)(k) * NY + (j)) * NX + (i))
#define UI(i, j, k) (((size_t)(k) * NY + (j)) * (NX + 1) + (i))
#define VI(i, j, k) (((size_t)(k) * (NY + 1) + (j)) * NX + (i))
#define WI(i, j, k) (((size_t)(k) * NY + (j)) * NX + (i))

static double cellt(const o3tank *T, const double *a, int i, int j, int k)
{
    return a[CI(cl3(i, 0, NX - 1), cl3(j, 0, NY - 1), cl3(k, 0, NZ - 1))];
}

/* velocity ghosts: nearest face; v and w at the inflow oddly reflected */
static double ut(const o3tank *T, const double *u, int i, int j, int k)
{
    return u[UI(cl3(i, 0, NX), cl3(j, 0, NY - 1), cl3(k, 0, NZ - 1))];
}

static double vt(const o3tank *T, const double *v, int i, int j, int k)
{
    j = cl3(j, 0, NY);
    k = cl3(k, 0, NZ - 1);
    if (i > NX - 1) i = NX - 1;
    if (i < 0) return -v[VI(-1 - i, j, k)];
    return v[VI(i, j, k)];
}

/* w with its ghosts; at the inflow the odd reflection about the incident wave's
 * w_in at time ta, or, for the mean of two time levels (ta != tb), about the
 * mean of w_in at ta and tb */
static double wt(const o3tank *T, const double *w, int i, int j, int k, double ta, double tb)
{
    k = cl3(k, 0, NZ);
    j = cl3(j, 0, NY - 1);
    if (i > NX - 1) i = NX - 1;
    if (i < 0) {
        double ui, wi;
        airyt(T, 0.0, k * T->h, ta, &ui, &wi);
        if (tb != ta) {
            double u2, w2;
            airyt(T, 0.0, k * T->h, tb, &u2, &w2);
            wi = 0.5 * (wi + w2);
        }
        return 2.0 * wi - w[WI(-1 - i, j, k)];
    }
    return w[WI(i, j, k)];
}

static double kor(double quu, double qu, double qd)
{
    double d1 = qu - quu, d2 = qd - qu;
    if (d1 * d2 <= 0.0) return qu;
    double m = fmin(2.0 * fabs(d2), fmin((fabs(d1) + 2.0 * fabs(d2)) / 3.0, 2.0 * fabs(d1)));
    return d1 > 0.0 ? qu + 0.5 * m : qu - 0.5 * m;
}

static double upw(double q0, double q1, double q2, double q3, double vel)
{
    return vel >= 0.0 ? kor(q0, q1, q2) : kor(q3, q2, q1);
}

/* face densities: the mean of the two cells of the face (indices clamped) */
static double rut(const o3tank *T, const double *rc, int i, int j, int k)
{
    i = cl3(i, 0, NX);
    j = cl3(j, 0, NY - 1);
    k = cl3(k, 0, NZ - 1);
    return 0.5 * (cellt(T, rc, i - 1, j, k) + cellt(T, rc, i, j, k));
}

static double rvt(const o3tank *T, const double *rc, int i, int j, int k)
{
    i = cl3(i, 0, NX - 1);
    j = cl3(j, 0, NY);
    k = cl3(k, 0, NZ - 1);
    return 0.5 * (cellt(T, rc, i, j - 1, k) + cellt(T, rc, i, j, k));
}

static double rwt(const o3tank *T, const double *rc, int i, int j, int k)
{
    i = cl3(i, 0, NX - 1);
    j = cl3(j, 0, NY - 1);
    k = cl3(k, 0, NZ);
    return 0.5 * (cellt(T, rc, i, j, k - 1) + cellt(T, rc, i, j, k));
}

typedef struct {
    const o3tank *T;
    const double *rc, *u, *v, *w;
    double t, t2; /* the velocity's time level(s): ghosts as in wt */
} tctx3;

/* rho-breve and C of the u-face (i, j, k) */
static void trans_u(const tctx3 *X, int i, int j, int k, double dt, double *rb, double *C)
{
    const o3tank *T = X->T;
    double h = T->h, m[6], f[6];
    for (int s = 0; s < 2; ++s) { /* x: CV faces at cell centres i-1+s */
        int a = i - 1 + s;
        double U = 0.5 * (ut(T, X->u, a, j, k) + ut(T, X->u, a + 1, j, k));
        double r = upw(rut(T, X->rc, a - 1, j, k), rut(T, X->rc, a, j, k), rut(T, X->rc, a + 1, j, k),
                       rut(T, X->rc, a + 2, j, k), U);
        double q = upw(ut(T, X->u, a - 1, j, k), ut(T, X->u, a, j, k), ut(T, X->u, a + 1, j, k),
                       ut(T, X->u, a + 2, j, k), U);
        m[s] = U * r;
        f[s] = m[s] * q;
    }
    for (int s = 0; s < 2; ++s) { /* y: CV faces on the xy-edges (i, j+s) */
        int b = j - 1 + s;
        double V = 0.5 * (vt(T, X->v, i - 1, b + 1, k) + vt(T, X->v, i, b + 1, k));
        double r = upw(rut(T, X->rc, i, b - 1, k), rut(T, X->rc, i, b, k), rut(T, X->rc, i, b + 1, k),
                       rut(T, X->rc, i, b + 2, k), V);
        double q = upw(ut(T, X->u, i, b - 1, k), ut(T, X->u, i, b, k), ut(T, X->u, i, b + 1, k),
                       ut(T, X->u, i, b + 2, k), V);
        m[2 + s] = V * r;
        f[2 + s] = m[2 + s] * q;
    }
    for (int s = 0; s < 2; ++s) { /* z: CV faces on the xz-edges (i, k+s) */
        int c = k - 1 + s;
        double W = 0.5 * (wt(T, X->w, i - 1, j, c + 1, X->t, X->t2) + wt(T, X->w, i, j, c + 1, X->t, X->t2));
        double r = upw(rut(T, X->rc, i, j, c - 1), rut(T, X->rc, i, j, c), rut(T, X->rc, i, j, c + 1),
                       rut(T, X->rc, i, j, c + 2), W);
        double q = upw(ut(T, X->u, i, j, c - 1), ut(T, X->u, i, j, c), ut(T, X->u, i, j, c + 1),
                       ut(T, X->u, i, j, c + 2), W);
        m[4 + s] = W * r;
        f[4 + s] = m[4 + s] * q;
    }
    *rb = rut(T, X->rc, i, j, k) - dt / h * (((m[1] - m[0]) + (m[3] - m[2])) + (m[5] - m[4]));
    *C = (((f[1] - f[0]) + (f[3] - f[2])) + (f[5] - f[4])) / h;
}

static void trans_v(const tctx3 *X, int i, int j, int k, double dt, double *rb, double *C)
{
    const o3tank *T = X->T;
    double h = T->h, m[6], f[6];
    for (int s = 0; s < 2; ++s) { /* x: CV faces on the xy-edges (i+s, j) */
        int a = i - 1 + s;
        double U = 0.5 * (ut(T, X->u, a + 1, j - 1, k) + ut(T, X->u, a + 1, j, k));
        double r = upw(rvt(T, X->rc, a - 1, j, k), rvt(T, X->rc, a, j, k), rvt(T, X->rc, a + 1, j, k),
                       rvt(T, X->rc, a + 2, j, k), U);
        double q = upw(vt(T, X->v, a - 1, j, k), vt(T, X->v, a, j, k), vt(T, X->v, a + 1, j, k),
                       vt(T, X->v, a + 2, j, k), U);
        m[s] = U * r;
        f[s] = m[s] * q;
    }
    for (int s = 0; s < 2; ++s) { /* y: CV faces at cell centres j-1+s */
        int b = j - 1 + s;
        double V = 0.5 * (vt(T, X->v, i, b, k) + vt(T, X->v, i, b + 1, k));
        double r = upw(rvt(T, X->rc, i, b - 1, k), rvt(T, X->rc, i, b, k), rvt(T, X->rc, i, b + 1, k),
                       rvt(T, X->rc, i, b + 2, k), V);
        double q = upw(vt(T, X->v, i, b - 1, k), vt(T, X->v, i, b, k), vt(T, X->v, i, b + 1, k),
                       vt(T, X->v, i, b + 2, k), V);
        m[2 + s] = V * r;
        f[2 + s] = m[2 + s] * q;
    }
    for (int s = 0; s < 2; ++s) { /* z: CV faces on the yz-edges (j, k+s) */
        int c = k - 1 + s;
        double W = 0.5 * (wt(T, X->w, i, j - 1, c + 1, X->t, X->t2) + wt(T, X->w, i, j, c + 1, X->t, X->t2));
        double r = upw(rvt(T, X->rc, i, j, c - 1), rvt(T, X->rc, i, j, c), rvt(T, X->rc, i, j, c + 1),
                       rvt(T, X->rc, i, j, c + 2), W);
        double q = upw(vt(T, X->v, i, j, c - 1), vt(T, X->v, i, j, c), vt(T, X->v, i, j, c + 1),
                       vt(T, X->v, i, j, c + 2), W);
        m[4 + s] = W * r;
        f[4 + s] = m[4 + s] * q;
    }
    *rb = rvt(T, X->rc, i, j, k) - dt / h * (((m[1] - m[0]) + (m[3] - m[2])) + (m[5] - m[4]));
    *C = (((f[1] - f[0]) + (f[3] - f[2])) + (f[5] - f[4])) / h;
}

static void trans_w(const tctx3 *X, int i, int j, int k, double dt, double *rb, double *C)
{
    const o3tank *T = X->T;
    double h = T->h, m[6], f[6];
    double t = X->t, t2 = X->t2;
    for (int s = 0; s < 2; ++s) { /* x: CV faces on the xz-edges (i+s, k) */
        int a = i - 1 + s;
        double U = 0.5 * (ut(T, X->u, a + 1, j, k - 1) + ut(T, X->u, a + 1, j, k));
        double r = upw(rwt(T, X->rc, a - 1, j, k), rwt(T, X->rc, a, j, k), rwt(T, X->rc, a + 1, j, k),
                       rwt(T, X->rc, a + 2, j, k), U);
        double q = upw(wt(T, X->w, a - 1, j, k, t, t2), wt(T, X->w, a, j, k, t, t2), wt(T, X->w, a + 1, j, k, t, t2),
                       wt(T, X->w, a + 2, j, k, t, t2), U);
        m[s] = U * r;
        f[s] = m[s] * q;
    }
    for (int s = 0; s < 2; ++s) { /* y: CV faces on the yz-edges (j+s, k) */
        int b = j - 1 + s;
        double V = 0.5 * (vt(T, X->v, i, b + 1, k - 1) + vt(T, X->v, i, b + 1, k));
        double r = upw(rwt(T, X->rc, i, b - 1, k), rwt(T, X->rc, i, b, k), rwt(T, X->rc, i, b + 1, k),
                       rwt(T, X->rc, i, b + 2, k), V);
        double q = upw(wt(T, X->w, i, b - 1, k, t, t2), wt(T, X->w, i, b, k, t, t2), wt(T, X->w, i, b + 1, k, t, t2),
                       wt(T, X->w, i, b + 2, k, t, t2), V);
        m[2 + s] = V * r;
        f[2 + s] = m[2 + s] * q;
    }
    for (int s = 0; s < 2; ++s) { /* z: CV faces at cell centres k-1+s */
        int c = k - 1 + s;
        double W = 0.5 * (wt(T, X->w, i, j, c, t, t2) + wt(T, X->w, i, j, c + 1, t, t2));
        double r = upw(rwt(T, X->rc, i, j, c - 1), rwt(T, X->rc, i, j, c), rwt(T, X->rc, i, j, c + 1),
                       rwt(T, X->rc, i, j, c + 2), W);
        double q = upw(wt(T, X->w, i, j, c - 1, t, t2), wt(T, X->w, i, j, c, t, t2), wt(T, X->w, i, j, c + 1, t, t2),
                       wt(T, X->w, i, j, c + 2, t, t2), W);
        m[4 + s] = W * r;
        f[4 + s] = m[4 + s] * q;
    }
    *rb = rwt(T, X->rc, i, j, k) - dt / h * (((m[1] - m[0]) + (m[3] - m[2])) + (m[5] - m[4]));
    *C = (((f[1] - f[0]) + (f[3] - f[2])) + (f[5] - f[4])) / h;
}

/* ------------------------------------------------------- viscous term -- */
typedef struct {
    const o3tank *T;
    const double *mu, *u, *v, *w;
    double t, t2; /* the velocity's time level(s): ghosts as in wt */
} vctx3;

#define MU(i, j, k) cellt(X->T, X->mu, i, j, k)
#define UT(i, j, k) ut(X->T, X->u, i, j, k)
#define VT(i, j, k) vt(X->T, X->v, i, j, k)
#define WT(i, j, k) wt(X->T, X->w, i, j, k, X->t, X->t2)

/* edge viscosities: the mean of the four cells around the edge */
static double mxy(const vctx3 *X, int i, int j, int k)
{
    return 0.25 * (MU(i - 1, j - 1, k) + MU(i, j - 1, k) + MU(i - 1, j, k) + MU(i, j, k));
}
static double mxz(const vctx3 *X, int i, int j, int k)
{
    return 0.25 * (MU(i - 1, j, k - 1) + MU(i, j, k - 1) + MU(i - 1, j, k) + MU(i, j, k));
}
static double myz(const vctx3 *X, int i, int j, int k)
{
    return 0.25 * (MU(i, j - 1, k - 1) + MU(i, j, k - 1) + MU(i, j - 1, k) + MU(i, j, k));
}

static double txx3(const vctx3 *X, int i, int j, int k) { return 2.0 * MU(i, j, k) * (UT(i + 1, j, k) - UT(i, j, k)) / X->T->h; }
static double tyy3(const vctx3 *X, int i, int j, int k) { return 2.0 * MU(i, j, k) * (VT(i, j + 1, k) - VT(i, j, k)) / X->T->h; }
static double tzz3(const vctx3 *X, int i, int j, int k) { return 2.0 * MU(i, j, k) * (WT(i, j, k + 1) - WT(i, j, k)) / X->T->h; }
static double txy3(const vctx3 *X, int i, int j, int k)
{
    double h = X->T->h;
    return mxy(X, i, j, k) * ((UT(i, j, k) - UT(i, j - 1, k)) / h + (VT(i, j, k) - VT(i - 1, j, k)) / h);
}
static double txz3(const vctx3 *X, int i, int j, int k)
{
    double h = X->T->h;
    return mxz(X, i, j, k) * ((UT(i, j, k) - UT(i, j, k - 1)) / h + (WT(i, j, k) - WT(i - 1, j, k)) / h);
}
static double tyz3(const vctx3 *X, int i, int j, int k)
{
    double h = X->T->h;
    return myz(X, i, j, k) * ((VT(i, j, k) - VT(i, j, k - 1)) / h + (WT(i, j, k) - WT(i, j - 1, k)) / h);
}

/* components of div[mu (grad u + grad u^T)] at the u-, v- and w-faces */
static double viscx3(const vctx3 *X, int i, int j, int k)
{
    double h = X->T->h;
    return ((txx3(X, i, j, k) - txx3(X, i - 1, j, k)) / h + (txy3(X, i, j + 1, k) - txy3(X, i, j, k)) / h) +
           (txz3(X, i, j, k + 1) - txz3(X, i, j, k)) / h;
}
static double viscy3(const vctx3 *X, int i, int j, int k)
{
    double h = X->T->h;
    return ((tyy3(X, i, j, k) - tyy3(X, i, j - 1, k)) / h + (txy3(X, i + 1, j, k) - txy3(X, i, j, k)) / h) +
           (tyz3(X, i, j, k + 1) - tyz3(X, i, j, k)) / h;
}
static double viscz3(const vctx3 *X, int i, int j, int k)
{
    double h = X->T->h;
    return ((tzz3(X, i, j, k) - tzz3(X, i, j, k - 1)) / h + (txz3(X, i + 1, j, k) - txz3(X, i, j, k)) / h) +
           (tyz3(X, i, j + 1, k) - tyz3(X, i, j, k)) / h;
}

/* interior-formula diagonals (the Jacobi splitting only) */
static double vdiagx3(const vctx3 *X, int i, int j, int k)
{
    double h = X->T->h;
    return -(2.0 * MU(i, j, k) + 2.0 * MU(i - 1, j, k) + mxy(X, i, j + 1, k) + mxy(X, i, j, k) +
             mxz(X, i, j, k + 1) + mxz(X, i, j, k)) / (h * h);
}
static double vdiagy3(const vctx3 *X, int i, int j, int k)
{
    double h = X->T->h;
    return -(2.0 * MU(i, j, k) + 2.0 * MU(i, j - 1, k) + mxy(X, i + 1, j, k) + mxy(X, i, j, k) +
             myz(X, i, j, k + 1) + myz(X, i, j, k)) / (h * h);
}
static double vdiagz3(const vctx3 *X, int i, int j, int k)
{
    double h = X->T->h;
    return -(2.0 * MU(i, j, k) + 2.0 * MU(i, j, k - 1) + mxz(X, i + 1, j, k) + mxz(X, i, j, k) +
             myz(X, i, j + 1, k) + myz(X, i, j, k)) / (h * h);
}

static double dampt(const o3tank *T, double x)
{
    if (T->P.L.damp_len <= 0.0 || x <= T->P.L.damp_x0) return 0.0;
    double xi = (x - T->P.L.damp_x0) / T->P.L.damp_len;
    if (xi > 1.0) xi = 1.0;
    return (exp(pow(xi, 3.5)) - 1.0) / (exp(1.0) - 1.0);
}

/* vorticity damping over the top four cells (Eq. spongelayer, z_max = the top) */
static double vortt(const o3tank *T, double z, double dt)
{
    double wd = 4.0 * T->h;
    if (z < T->P.lz - wd) return 0.0;
    double zt = (z - T->P.lz) / wd;
    return T->P.L.rho_a * (cos(PIT * zt) + 1.0) / (4.0 * dt);
}

/* heave force, Eq. int_fh */
static double force3(const o3tank *T, const double *mu, double tv)
{
    double h = T->h, F = 0.0, A = h * h;
    if (!T->P.L.has_body) return 0.0;
    for (int k = 1; k < NZ; ++k) /* z-faces: pressure and 2 mu dw/dz */
        for (int j = 0; j < NY; ++j)
            for (int i = 0; i < NX; ++i) {
                double x = (i + 0.5) * h, y = (j + 0.5) * h;
                double pl = psit(T, x, y, (k - 0.5) * h, T->zc), pr = psit(T, x, y, (k + 0.5) * h, T->zc);
                if (!(pl * pr < 0.0)) continue;
                double nz_ = pl < 0.0 ? 1.0 : -1.0, wl = fabs(pl), wr = fabs(pr);
                double pf = (T->p[CI(i, j, k - 1)] * wr + T->p[CI(i, j, k)] * wl) / (wl + wr);
                double muf = 0.5 * (mu[CI(i, j, k - 1)] + mu[CI(i, j, k)]);
                double dwdz = (wt(T, T->w, i, j, k + 1, tv, tv) - wt(T, T->w, i, j, k - 1, tv, tv)) / (2.0 * h);
                F += (-pf * nz_ + muf * 2.0 * dwdz * nz_) * A;
            }
    for (int k = 0; k < NZ; ++k) /* x-faces: mu (dw/dx + du/dz) */
        for (int j = 0; j < NY; ++j)
            for (int i = 1; i < NX; ++i) {
                double y = (j + 0.5) * h, z = (k + 0.5) * h;
                double pl = psit(T, (i - 0.5) * h, y, z, T->zc), pr = psit(T, (i + 0.5) * h, y, z, T->zc);
                if (!(pl * pr < 0.0)) continue;
                double nx_ = pl < 0.0 ? 1.0 : -1.0;
                double muf = 0.5 * (mu[CI(i - 1, j, k)] + mu[CI(i, j, k)]);
                double dwdx = 0.5 * ((wt(T, T->w, i, j, k, tv, tv) - wt(T, T->w, i - 1, j, k, tv, tv)) +
                                     (wt(T, T->w, i, j, k + 1, tv, tv) - wt(T, T->w, i - 1, j, k + 1, tv, tv))) / h;
                double dudz = (ut(T, T->u, i, j, k + 1) - ut(T, T->u, i, j, k - 1)) / (2.0 * h);
                F += muf * (dwdx + dudz) * nx_ * A;
            }
    for (int k = 0; k < NZ; ++k) /* y-faces: mu (dw/dy + dv/dz) */
        for (int j = 1; j < NY; ++j)
            for (int i = 0; i < NX; ++i) {
                double x = (i + 0.5) * h, z = (k + 0.5) * h;
                double pl = psit(T, x, (j - 0.5) * h, z, T->zc), pr = psit(T, x, (j + 0.5) * h, z, T->zc);
                if (!(pl * pr < 0.0)) continue;
                double ny_ = pl < 0.0 ? 1.0 : -1.0;
                double muf = 0.5 * (mu[CI(i, j - 1, k)] + mu[CI(i, j, k)]);
                double dwdy = 0.5 * ((wt(T, T->w, i, j, k, tv, tv) - wt(T, T->w, i, j - 1, k, tv, tv)) +
                                     (wt(T, T->w, i, j, k + 1, tv, tv) - wt(T, T->w, i, j - 1, k + 1, tv, tv))) / h;
                double dvdz = (vt(T, T->v, i, j, k + 1) - vt(T, T->v, i, j, k - 1)) / (2.0 * h);
                F += muf * (dwdy + dvdz) * ny_ * A;
            }
    return F;
}

static double *zal(size_t n)
{
    double *p = (double *)calloc(n ? n : 1, sizeof(double));
    if (!p) abort();
    return p;
}

/* ------------------------------------------------------------ the step -- */
int oracle3_step(void *handle, double dt, double f_pto_in, oracle3_result *out)
{
    o3tank *T = (o3tank *)handle;
    const int nx = NX, ny = NY, nz = NZ;
    size_t n = (size_t)nx * ny * nz, nu = (size_t)(nx + 1) * ny * nz, nv = (size_t)nx * (ny + 1) * nz,
           nw = (size_t)nx * ny * (nz + 1);
    double h = T->h, t0 = T->t, t1 = T->t + dt, g = T->P.g, kp = T->P.kappa_p;
    double *rho_n = zal(n), *mu_n = zal(n), *rf_n = zal(n), *chi_n = zal(n);
    double *mu_1 = zal(n), *rf_1 = zal(n), *chi_1 = zal(n), *rho_1 = zal(n);
    double *Ru = zal(nu), *Rv = zal(nv), *Rw = zal(nw), *Du = zal(nu), *Dv = zal(nv), *Dw = zal(nw);
    double *ua = zal(nu), *va = zal(nv), *wa = zal(nw), *ub = zal(nu), *vb = zal(nv), *wb = zal(nw);
    double *bx = zal(nu), *by = zal(nv), *bz = zal(nw), *rhs = zal(n), *phi = zal(n), *sig1 = zal(n);

    /* Fixed-point cycles k = 0 .. n_cycles - 1 (section "Time stepping scheme"):
     * the iterate (sigma, u, p, z)^{n+1,k} lives in the tank's fields and starts
     * from time level n (k = 0: u^n, p^{n-1/2}, sigma^n, the body at z^n); cycle
     * k takes the force from it, advects sigma^n with the means of levels n and
     * n+1,k, and solves the momentum system of level n with the pressure and
     * the body velocity of the iterate.  One cycle is the plain step. */
    const int ncyc = T->P.n_cycles > 1 ? T->P.n_cycles : 1;
    const double *sig_n = T->sig, *u_n = T->u, *v_n = T->v, *w_n = T->w;
    double *keep[4] = {0, 0, 0, 0}, *sh = 0, *uh = 0, *vh = 0, *wh = 0, *mk[4] = {0, 0, 0, 0};
    if (ncyc > 1) { /* level n, kept while the tank's fields hold the iterate */
        keep[0] = zal(n);
        keep[1] = zal(nu);
        keep[2] = zal(nv);
        keep[3] = zal(nw);
        memcpy(keep[0], T->sig, n * sizeof(double));
        memcpy(keep[1], T->u, nu * sizeof(double));
        memcpy(keep[2], T->v, nv * sizeof(double));
        memcpy(keep[3], T->w, nw * sizeof(double));
        sig_n = keep[0];
        u_n = keep[1];
        v_n = keep[2];
        w_n = keep[3];
        sh = zal(n);
        uh = zal(nu);
        vh = zal(nv);
        wh = zal(nw);
        for (int q = 0; q < 4; ++q) mk[q] = zal(n);
    }
    const double zc_n = T->zc, zd_n = T->zdot, zd_prev = T->zdot_prev;
    /* materials at level n: the explicit half of the momentum system, and the
     * force of the first cycle */
    oracle3_materials(&T->P.L, sig_n, zc_n, rho_n, mu_n, rf_n, chi_n);
    const double fpto = f_pto_in - T->P.pto_damping * zd_n;
    double F = 0.0, zd1 = zd_n, zc1 = zc_n, relres = 0.0, bn = 0.0;
    int iters = 0, st = 0;
    for (int cyc = 0; cyc < ncyc; ++cyc) {

    /* (1) force from p^{n+1/2,k}, u^{n+1,k} and the body at z^{n+1,k} (k = 0:
     * p^{n-1/2}, u^n, z^n) */
    if (cyc == 0) {
        F = force3(T, mu_n, t0);
    } else {
        oracle3_materials(&T->P.L, T->sig, T->zc, mk[0], mk[1], mk[2], mk[3]);
        F = force3(T, mk[1], t1);
    }

    /* (2) heave */
    zd1 = zd_n;
    zc1 = zc_n;
    if (T->P.L.has_body) {
        double m = T->P.L.body_mass, ma = T->P.added_mass;
        zd1 = zd_n + (dt * (F - m * g + fpto) + ma * (zd_n - zd_prev)) / (m + ma);
        zc1 = zc_n + 0.5 * dt * (zd_n + zd1);
    }

    /* (3) sigma: sigma^n advected with u^{n+1/2,k}, sigma^{n+1/2,k} */
    if (cyc == 0) {
        oracle3_advect(&T->P.L, sig_n, u_n, v_n, w_n, dt, t0, sig1);
    } else {
        ORACLE_PAR_FOR
        for (size_t c = 0; c < n; ++c) sh[c] = 0.5 * (sig_n[c] + T->sig[c]);
        for (size_t f = 0; f < nu; ++f) uh[f] = 0.5 * (u_n[f] + T->u[f]);
        for (size_t f = 0; f < nv; ++f) vh[f] = 0.5 * (v_n[f] + T->v[f]);
        for (size_t f = 0; f < nw; ++f) wh[f] = 0.5 * (w_n[f] + T->w[f]);
        oracle3_advect_half(&T->P.L, sig_n, sh, uh, vh, wh, dt, t0, t1, sig1);
    }
    oracle3_reinit(&T->P.L, sig1, T->P.n_reinit, t1);

    /* (4) materials at n+1 */
    oracle3_materials(&T->P.L, sig1, zc1, rho_1, mu_1, rf_1, chi_1);

    /* (5) transport (advecting velocity u^{n+1/2,k}) and the momentum system */
    tctx3 X = {T, rho_n, u_n, v_n, w_n, t0, t0};
    if (cyc > 0) {
        X.u = uh;
        X.v = vh;
        X.w = wh;
        X.t2 = t1;
    }
    vctx3 Vn = {T, mu_n, u_n, v_n, w_n, t0, t0};
    ORACLE_PAR_FOR
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                size_t f = UI(i, j, k);
                double rb, C;
                trans_u(&X, i, j, k, dt, &rb, &C);
                double chi = 0.5 * (cellt(T, chi_1, i - 1, j, k) + cellt(T, chi_1, i, j, k));
                Du[f] = rb / dt + chi / kp + dampt(T, i * h) * rb / dt + vortt(T, (k + 0.5) * h, dt);
                Ru[f] = rut(T, rho_n, i, j, k) * u_n[f] / dt - C + 0.5 * viscx3(&Vn, i, j, k) -
                        (T->p[CI(i, j, k)] - T->p[CI(i - 1, j, k)]) / h;
            }
    ORACLE_PAR_FOR
    for (int k = 0; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t f = VI(i, j, k);
                double rb, C;
                trans_v(&X, i, j, k, dt, &rb, &C);
                double chi = 0.5 * (cellt(T, chi_1, i, j - 1, k) + cellt(T, chi_1, i, j, k));
                Dv[f] = rb / dt + chi / kp + dampt(T, (i + 0.5) * h) * rb / dt + vortt(T, (k + 0.5) * h, dt);
                Rv[f] = rvt(T, rho_n, i, j, k) * v_n[f] / dt - C + 0.5 * viscy3(&Vn, i, j, k) -
                        (T->p[CI(i, j, k)] - T->p[CI(i, j - 1, k)]) / h;
            }
    ORACLE_PAR_FOR
    for (int k = 1; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t f = WI(i, j, k);
                double rb, C;
                trans_w(&X, i, j, k, dt, &rb, &C);
                double chi = 0.5 * (cellt(T, chi_1, i, j, k - 1) + cellt(T, chi_1, i, j, k));
                double rf = 0.5 * (cellt(T, rf_1, i, j, k - 1) + cellt(T, rf_1, i, j, k));
                Dw[f] = rb / dt + chi / kp + dampt(T, (i + 0.5) * h) * rb / dt + vortt(T, k * h, dt);
                double gp = k < nz ? (T->p[CI(i, j, k)] - T->p[CI(i, j, k - 1)]) / h
                                   : -2.0 * T->p[CI(i, j, nz - 1)] / h;
                Rw[f] = rwt(T, rho_n, i, j, k) * w_n[f] / dt - C + 0.5 * viscz3(&Vn, i, j, k) - rf * g +
                        chi * zd1 / kp - gp;
            }

    /* (6) Crank-Nicolson Jacobi sweeps; Dirichlet faces at n+1 */
    memcpy(ua, u_n, nu * sizeof(double));
    memcpy(va, v_n, nv * sizeof(double));
    memcpy(wa, w_n, nw * sizeof(double));
    for (int k = 0; k < nz; ++k) {
        double uin, win;
        airyt(T, 0.0, (k + 0.5) * h, t1, &uin, &win);
        for (int j = 0; j < ny; ++j) {
            ua[UI(0, j, k)] = uin;
            ua[UI(nx, j, k)] = 0.0;
        }
    }
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < nx; ++i) {
            va[VI(i, 0, k)] = 0.0;
            va[VI(i, ny, k)] = 0.0;
        }
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) wa[WI(i, j, 0)] = 0.0;
    memcpy(ub, ua, nu * sizeof(double));
    memcpy(vb, va, nv * sizeof(double));
    memcpy(wb, wa, nw * sizeof(double));
    for (int it = 0; it < T->P.n_jacobi; ++it) {
        vctx3 Vk = {T, mu_1, ua, va, wa, t1, t1};
        ORACLE_PAR_FOR
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 1; i < nx; ++i) {
                    size_t f = UI(i, j, k);
                    double ld = vdiagx3(&Vk, i, j, k);
                    ub[f] = (Ru[f] + 0.5 * (viscx3(&Vk, i, j, k) - ld * ua[f])) / (Du[f] - 0.5 * ld);
                }
        ORACLE_PAR_FOR
        for (int k = 0; k < nz; ++k)
            for (int j = 1; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t f = VI(i, j, k);
                    double ld = vdiagy3(&Vk, i, j, k);
                    vb[f] = (Rv[f] + 0.5 * (viscy3(&Vk, i, j, k) - ld * va[f])) / (Dv[f] - 0.5 * ld);
                }
        ORACLE_PAR_FOR
        for (int k = 1; k <= nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t f = WI(i, j, k);
                    double ld = vdiagz3(&Vk, i, j, k);
                    wb[f] = (Rw[f] + 0.5 * (viscz3(&Vk, i, j, k) - ld * wa[f])) / (Dw[f] - 0.5 * ld);
                }
        memcpy(ua, ub, nu * sizeof(double));
        memcpy(va, vb, nv * sizeof(double));
        memcpy(wa, wb, nw * sizeof(double));
    }

    /* (7) pressure increment */
    ORACLE_PAR_FOR
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 1; i < nx; ++i) bx[UI(i, j, k)] = 1.0 / Du[UI(i, j, k)];
    ORACLE_PAR_FOR
    for (int k = 0; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 0; i < nx; ++i) by[VI(i, j, k)] = 1.0 / Dv[VI(i, j, k)];
    ORACLE_PAR_FOR
    for (int k = 1; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) bz[WI(i, j, k)] = 1.0 / Dw[WI(i, j, k)];
    ORACLE_PAR_FOR
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                rhs[CI(i, j, k)] = -h * (((ua[UI(i + 1, j, k)] - ua[UI(i, j, k)]) + (va[VI(i, j + 1, k)] - va[VI(i, j, k)])) +
                                         (wa[WI(i, j, k + 1)] - wa[WI(i, j, k)]));
    memset(phi, 0, n * sizeof(double));
    st = oracle3_poisson_solve(nx, ny, nz, bx, by, bz, rhs, phi, T->P.rtol, T->P.max_iters, T->P.restart,
                               T->P.mg_pre, T->P.mg_post, &iters, &relres);
    bn = 0.0;
    for (size_t c = 0; c < n; ++c) bn += rhs[c] * rhs[c];

    /* (8) projection */
    ORACLE_PAR_FOR
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                size_t f = UI(i, j, k);
                double uu = ua[f];
                if (i > 0 && i < nx) uu -= bx[f] * (phi[CI(i, j, k)] - phi[CI(i - 1, j, k)]) / h;
                T->u[f] = uu;
            }
    ORACLE_PAR_FOR
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t f = VI(i, j, k);
                double vv = va[f];
                if (j > 0 && j < ny) vv -= by[f] * (phi[CI(i, j, k)] - phi[CI(i, j - 1, k)]) / h;
                T->v[f] = vv;
            }
    ORACLE_PAR_FOR
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t f = WI(i, j, k);
                double ww = wa[f];
                if (k > 0 && k < nz) ww -= bz[f] * (phi[CI(i, j, k)] - phi[CI(i, j, k - 1)]) / h;
                if (k == nz) ww += 2.0 * bz[f] * phi[CI(i, j, nz - 1)] / h;
                T->w[f] = ww;
            }
    ORACLE_PAR_FOR
    for (size_t c = 0; c < n; ++c) T->p[c] += phi[c];
    memcpy(T->sig, sig1, n * sizeof(double));
    T->zc = zc1;
    } /* cycles */
    T->t = t1;
    T->zdot_prev = zd_n;
    T->zdot = zd1;

    /* diagnostics: ||h div u||_2; eta at the probe column (x = probe_x, middle y) */
    double dn = 0.0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                dn += sqt(h * (((T->u[UI(i + 1, j, k)] - T->u[UI(i, j, k)]) + (T->v[VI(i, j + 1, k)] - T->v[VI(i, j, k)])) +
                               (T->w[WI(i, j, k + 1)] - T->w[WI(i, j, k)])));
    int ip = cl3((int)floor(T->P.probe_x / h), 0, nx - 1), jp = ny / 2;
    double eta = NAN;
    for (int k = 0; k + 1 < nz; ++k) {
        double a = T->sig[CI(ip, jp, k)], b = T->sig[CI(ip, jp, k + 1)];
        if (a < 0.0 && b >= 0.0) {
            eta = (k + 0.5) * h + h * a / (a - b) - T->P.L.depth;
            break;
        }
    }
    if (out) {
        out->t = T->t;
        out->z = T->zc - T->zc0;
        out->zdot = T->zdot;
        out->f_hydro = F;
        out->f_pto = fpto;
        out->eta_probe = eta;
        out->residual = relres;
        out->div_norm = sqrt(dn);
        out->rhs_norm = sqrt(bn);
        out->iters = iters;
    }
    double *fr[] = {rho_n, mu_n, rf_n, chi_n, mu_1, rf_1, chi_1, rho_1, Ru, Rv, Rw, Du, Dv, Dw,
                    ua, va, wa, ub, vb, wb, bx, by, bz, rhs, phi, sig1,
                    keep[0], keep[1], keep[2], keep[3], sh, uh, vh, wh, mk[0], mk[1], mk[2], mk[3]};
    for (size_t q = 0; q < sizeof(fr) / sizeof(fr[0]); ++q) free(fr[q]);
    return st;
}

/* ------------------------------------------------------------ lifecycle -- */
/* State at creation: sigma = z - depth - eta(x, 0), the Airy velocities of the
 * incident wave (u, w; v = 0), p = the discrete hydrostatic pressure of
 * rho^flow integrated down from the top face (p = 0 there), the body at zc. */
void *oracle3_create(const oracle3_params *P, double zc)
{
    o3tank *T = (o3tank *)calloc(1, sizeof(o3tank));
    if (!T) return 0;
    T->P = *P;
    T->h = P->L.h;
    int nx = P->L.nx, ny = P->L.ny, nz = P->L.nz;
    size_t n = (size_t)nx * ny * nz;
    T->sig = zal(n);
    T->u = zal((size_t)(nx + 1) * ny * nz);
    T->v = zal((size_t)nx * (ny + 1) * nz);
    T->w = zal((size_t)nx * ny * (nz + 1));
    T->p = zal(n);
    T->zc = T->zc0 = zc;
    double h = T->h;
    /* the incident wave does not depend on y: each value is evaluated once per
     * (x, z) and copied along y */
    ORACLE_PAR_FOR
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < nx; ++i) {
            double s = (k + 0.5) * h - P->L.depth - etat(T, (i + 0.5) * h, 0.0);
            for (int j = 0; j < ny; ++j) T->sig[CI(i, j, k)] = s;
        }
    ORACLE_PAR_FOR
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i <= nx; ++i) {
            double uu, ww;
            airyt(T, i * h, (k + 0.5) * h, 0.0, &uu, &ww);
            for (int j = 0; j < ny; ++j) T->u[UI(i, j, k)] = i == nx ? 0.0 : uu;
        }
    ORACLE_PAR_FOR
    for (int k = 1; k <= nz; ++k)
        for (int i = 0; i < nx; ++i) {
            double uu, ww;
            airyt(T, (i + 0.5) * h, k * h, 0.0, &uu, &ww);
            for (int j = 0; j < ny; ++j) T->w[WI(i, j, k)] = ww;
        }
    double *rho = zal(n), *mu = zal(n), *rf = zal(n), *chi = zal(n);
    oracle3_materials(&T->P.L, T->sig, zc, rho, mu, rf, chi);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double pp = 0.5 * rf[CI(i, j, nz - 1)] * P->g * h; /* half a cell below the top face */
            T->p[CI(i, j, nz - 1)] = pp;
            for (int k = nz - 2; k >= 0; --k) {
                pp += 0.5 * (rf[CI(i, j, k)] + rf[CI(i, j, k + 1)]) * P->g * h;
                T->p[CI(i, j, k)] = pp;
            }
        }
    free(rho);
    free(mu);
    free(rf);
    free(chi);
    return T;
}

void oracle3_destroy(void *handle)
{
    o3tank *T = (o3tank *)handle;
    if (!T) return;
    free(T->sig);
    free(T->u);
    free(T->v);
    free(T->w);
    free(T->p);
    free(T);
}

/* fields: 0 sigma, 1 u, 2 v, 3 w, 4 p */
static double *o3field(o3tank *T, int f, size_t *n)
{
    int nx = NX, ny = NY, nz = NZ;
    switch (f) {
    case 0: *n = (size_t)nx * ny * nz; return T->sig;
    case 1: *n = (size_t)(nx + 1) * ny * nz; return T->u;
    case 2: *n = (size_t)nx * (ny + 1) * nz; return T->v;
    case 3: *n = (size_t)nx * ny * (nz + 1); return T->w;
    case 4: *n = (size_t)nx * ny * nz; return T->p;
    default: *n = 0; return 0;
    }
}

int oracle3_get(void *handle, int f, double *dst)
{
    size_t n;
    double *p = o3field((o3tank *)handle, f, &n);
    if (!p) return 1;
    memcpy(dst, p, n * sizeof(double));
    return 0;
}

int oracle3_set(void *handle, int f, const double *src)
{
    size_t n;
    double *p = o3field((o3tank *)handle, f, &n);
    if (!p) return 1;
    memcpy(p, src, n * sizeof(double));
    return 0;
}

/* body state: t, zc, zdot, zc0, zdot_prev */
void oracle3_get_body(void *handle, double *out5)
{
    o3tank *T = (o3tank *)handle;
    out5[0] = T->t;
    out5[1] = T->zc;
    out5[2] = T->zdot;
    out5[3] = T->zc0;
    out5[4] = T->zdot_prev;
}

double oracle3_force(void *handle)
{
    o3tank *T = (o3tank *)handle;
    size_t n = (size_t)NX * NY * NZ;
    double *rho = zal(n), *mu = zal(n), *rf = zal(n), *chi = zal(n);
    oracle3_materials(&T->P.L, T->sig, T->zc, rho, mu, rf, chi);
    double F = force3(T, mu, T->t);
    free(rho);
    free(mu);
    free(rf);
    free(chi);
    return F;
}
