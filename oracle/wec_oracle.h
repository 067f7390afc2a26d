/* Plain FP64 CPU oracle of one wave-tank time step (2D) -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this library.  It shares no code, header or constant with the CUDA library.
 *
 * Field layouts (row-major, x fastest):
 *   cell  (sigma, p, rhs)  : [ny][nx]
 *   u on x-faces            : [ny][nx+1]   (face i at x = i h)
 *   v on y-faces            : [ny+1][nx]   (face j at y = j h)
 */
#ifndef WEC_ORACLE_H
#define WEC_ORACLE_H

typedef struct {
    int nx, ny;
    double lx, ly, depth;
    double rho_w, rho_a, mu_w, mu_a, g;
    int ncomp;
    const double *amp, *omega, *kwave, *phase;
    double damp_x0, damp_len, probe_x;
    int has_body;
    double body_xc, body_yc, body_w, body_h, body_mass, added_mass, kappa_p, pto_damping;
    double rtol;
    int max_iters, restart, n_reinit, n_jacobi, mg_pre, mg_post;
} oracle_params;

typedef struct {
    double t, z, zdot, f_hydro, f_pto, eta_probe, residual, div_norm;
    int iters;
} oracle_result;

enum {
    OF_SIGMA = 0, OF_U = 1, OF_V = 2, OF_P = 3, OF_USTAR = 4, OF_VSTAR = 5,
    OF_BETA_U = 6, OF_BETA_V = 7, OF_RHS = 8, OF_SIGMA_ADV = 9,
    OF_RHOB_U = 10, OF_RHOB_V = 11
};

/* Static-grid NLFK force: region R of nx x ny cells of size h with lower-left
 * corner (x0, y0); waves (ncomp components, wave numbers given); box body of
 * width body_w, height body_h centred at x = body_xc (y centre per call).
 * oracle_nlfk: mode 0 incident-wave pressure, 1 hydrostatic; heave force *fy,
 * surge force *fx (per unit span). */
typedef struct {
    double x0, y0, h;
    int nx, ny;
    double depth, rho_w, g;
    int ncomp;
    const double *amp, *omega, *kwave, *phase;
    double body_xc, body_w, body_h;
} oracle_nlfk_params;

int oracle_nlfk(const oracle_nlfk_params *P, double t, double yc, int mode, double *fx, double *fy);

#endif
