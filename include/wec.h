/*
 * wec.h -- C ABI of the GB300 wave-tank library (libwec.so).
 *
 * One time step of the two-phase (water/air) incompressible Navier-Stokes
 * equations on a uniform staggered MAC grid with a Brinkman-penalised heaving
 * body (arxiv 2206.07732, Sections "Continuous equations of motion" through
 * "Fluid-structure coupling"), run as CUDA kernels on one sm_103a GPU.
 *
 * Conventions (all entry points):
 *   - Return value: WEC_OK (0) or one of the WEC_ERR_* codes below; the message
 *     of the last failure on the calling thread is returned by wec_last_error().
 *   - The library owns every device buffer it allocates; host arrays passed in
 *     are copied before the call returns and stay owned by the caller.
 *   - Pointers documented as "device" are caller-owned device memory of the
 *     current CUDA device (e.g. a torch tensor's data_ptr()), used on the
 *     object's stream; the caller keeps them alive until the call returns.
 *   - Units are SI; in 2D, forces, masses and PTO forces are per unit span.
 *   - Layouts are row-major with x fastest:
 *       cell arrays (sigma, p):  [ny][nx]        cell (i, j) centre ((i+1/2)h, (j+1/2)h)
 *       u on x-faces:            [ny][nx+1]      face (i, j) at (i h, (j+1/2)h)
 *       v on y-faces:            [ny+1][nx]      face (i, j) at ((i+1/2)h, j h)
 *     (Section "Spatial discretization": cell-centred scalars, face velocities.)
 *   - No entry point falls back to the CPU.  A missing or unusable GPU is an
 *     error (WEC_ERR_CUDA).
 */
#ifndef WEC_H
#define WEC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    WEC_OK = 0,
    WEC_ERR_INVALID = 1,       /* bad sizes or parameters; nothing was changed      */
    WEC_ERR_CUDA = 2,          /* a CUDA call failed (message names it)             */
    WEC_ERR_NOT_CONVERGED = 3, /* solver hit max_iters; results are still written   */
    WEC_ERR_NONFINITE = 4,     /* a NaN/Inf reached the step's scalars or residual  */
    WEC_ERR_NOMEM = 5          /* device allocation failed                          */
};

/* Uniform 2D grid (Section "Spatial discretization"): h = lx / nx must equal
 * ly / ny.  nx, ny >= 8 and even.  depth = still-water depth d above the bed. */
typedef struct {
    int nx, ny;
    double lx, ly, depth;
} wec_grid;

/* Water (liquid) and air (gas) properties and gravity g = (0, -g)
 * (Eq. momentum; Eqs. ls_flow with l = water, g = air). */
typedef struct {
    double rho_w, rho_a, mu_w, mu_a, g;
} wec_fluids;

/* Incident wave as ncomp Airy components eta = sum a_i cos(k_i x - w_i t + th_i)
 * (Eqs. first_order_wave_elev, irregular_elevation).  k_i is computed by the
 * library from w_i and depth (Eq. dispersion_relation).  Host arrays, copied.
 * damp_x0 / damp_len: wave damping zone [damp_x0, damp_x0 + damp_len] at the
 * outlet (Section "Numerical wave tank"; damp_len = 0 disables it).
 * probe_x: x of the surface-elevation probe reported each step. */
typedef struct {
    int ncomp;
    const double *amp, *omega, *phase;
    double damp_x0, damp_len, probe_x;
} wec_waves;

/* Heaving rectangular body (2D box), SDF by CSG max of half-planes (Section
 * "Interface tracking").  present = 0: no body.  mass per unit span; the solid
 * density is mass / (width height).  kappa_p: Brinkman permeability (Eq.
 * bp_discrete, O(1e-8)).  pto_damping: linear PTO damper c, F_PTO = f_pto - c zdot.
 * added_mass: artificial added mass m_a of the stabilised heave update
 *   (m + m_a)(zdot^{n+1} - zdot^n) = dt (F_hydro - m g + F_PTO) + m_a (zdot^n - zdot^{n-1});
 *   m_a = 0 is Eq. newton_u exactly. */
typedef struct {
    int present;
    double xc, yc, width, height, mass, added_mass, kappa_p, pto_damping;
} wec_body;

enum { WEC_PREC_FP64 = 0, WEC_PREC_MIXED = 1, WEC_PREC_MIXED_MG = 2, WEC_PREC_MIXED_DF = 3 };

/* Pressure solver and step options.  precision:
 *   WEC_PREC_FP64      everything FP64;
 *   WEC_PREC_MIXED_MG  multigrid V-cycles in FP32 inside the FP64 FGMRES; the
 *                      residual, orthogonalisation and all step arithmetic FP64;
 *   WEC_PREC_MIXED     as WEC_PREC_MIXED_MG, and the step's stencil arithmetic
 *                      (level-set advection and reinitialisation, materials,
 *                      momentum, Jacobi sweeps) in FP32 over FP32 working copies
 *                      of FP64 state; the force integral (Eq. int_fh), the heave
 *                      update (Eq. newton_u), the projection and the persistent
 *                      fields stay FP64;
 *   WEC_PREC_MIXED_DF  (3D only) as WEC_PREC_MIXED, with the stencils in
 *                      double-float arithmetic (pairs of floats, about 48
 *                      significand bits, on the FP32 pipe) over float-pair
 *                      working copies: FP64-equivalent stencil accuracy; and
 *                      the solver's Arnoldi step (the operator products, the
 *                      Gram-Schmidt dot products and updates, the correction
 *                      of the solution) in float pairs over a float-pair
 *                      basis, the right-hand side, the solution and the true
 *                      residual at every restart staying FP64 (so rtol is met
 *                      in FP64 terms).
 * A Poisson object takes WEC_PREC_FP64 or WEC_PREC_MIXED (FP32 V-cycles), and
 * a 3D one (wec_poisson_create3) also WEC_PREC_MIXED_DF (its solver part);
 * WEC_PREC_MIXED_MG is a tank option.
 * rtol: relative FP64 residual ||b - A x||_2 <= rtol ||b||_2 of each solve.
 * restart: FGMRES restart length m (1..32).  n_reinit: Sussman pseudo-steps per
 * step.  n_jacobi: Jacobi sweeps of the Crank-Nicolson momentum system.
 * mg_pre / mg_post: red-black Gauss-Seidel sweeps before / after coarse correction.
 * n_cycles (section "Time stepping scheme"): cycles k = 0 .. n_cycles - 1 per step,
 * each taking the heave force from the iterate (p, u, z)^{n+1,k}, the heave update
 * from level n, sigma^n advected with the means of levels n and n+1,k, and level
 * n's momentum system with the iterate's pressure and body velocity; built for the
 * 3D tank (at most 8); the 2D tank and the Poisson objects take only one. */
typedef struct {
    int precision;
    double rtol;
    int max_iters, restart, n_reinit, n_jacobi, mg_pre, mg_post;
    int n_cycles;  /* fixed-point cycles per step (3D tank; 0 or 1: one cycle, the plain step) */
} wec_solver_opts;

/* Record of one step.  z: heave displacement from the initial position;
 * f_hydro: heave force of Eq. int_fh (from the step's initial p, u); f_pto: the
 * PTO force used; eta_probe: surface elevation at probe_x (NaN if no crossing);
 * residual: final relative FP64 residual of the pressure solve; div_norm:
 * ||h div u^{n+1}||_2; iters: FGMRES iterations (V-cycles); status: WEC_* code. */
typedef struct {
    double t, z, zdot, f_hydro, f_pto, eta_probe, residual, div_norm;
    int iters, status;
} wec_step_result;

typedef struct wec_tank wec_tank;
typedef struct wec_poisson wec_poisson;

/* Field ids for wec_get_field / wec_set_field. */
enum {
    WEC_F_SIGMA = 0,   /* level set sigma^n (cells; < 0 water)                 */
    WEC_F_U = 1,       /* u^n (x-faces)                                         */
    WEC_F_V = 2,       /* v^n (y-faces)                                         */
    WEC_F_P = 3,       /* p^{n-1/2} (cells)                                     */
    WEC_F_USTAR = 4,   /* last step's predicted u* (x-faces), read only         */
    WEC_F_VSTAR = 5,   /* last step's predicted v* (y-faces), read only         */
    WEC_F_BETA_U = 6,  /* last step's pressure coefficient 1/D on x-faces, r/o  */
    WEC_F_BETA_V = 7,  /* last step's pressure coefficient 1/D on y-faces, r/o  */
    WEC_F_RHS = 8,     /* last step's pressure right-hand side -h div u*, r/o   */
    WEC_F_SIGMA_ADV = 9 /* last step's advected sigma before reinit, r/o        */
};

/* Create a tank and its initial state: sigma = y - (d + eta(x, 0)), Airy
 * velocities (Wheeler-stretched, zero in air), p = discrete hydrostatic pressure
 * of the flow density.  stream: a cudaStream_t (NULL = legacy default stream)
 * on which every later call on this tank is enqueued.  *out receives the tank.
 * Errors: WEC_ERR_INVALID (non-uniform h, odd or too small sizes, non-positive
 * densities or kappa_p, ncomp < 0, restart out of range), WEC_ERR_NOMEM,
 * WEC_ERR_CUDA.  On error *out is NULL and nothing leaks. */
int wec_tank_create(const wec_grid *grid, const wec_fluids *fluids, const wec_waves *waves,
                    const wec_body *body, const wec_solver_opts *opts, void *cuda_stream,
                    wec_tank **out);

/* Free a tank (NULL is ignored).  Synchronises its stream first. */
void wec_tank_destroy(wec_tank *tank);

/* Advance one step of size dt > 0 (Sections "Solution methodology" and "Time
 * stepping scheme", n_cycles = 1): hydrodynamic force from p^{n-1/2}, u^n (Eq.
 * int_fh) -> heave update (Eq. newton_u, stabilised as in wec_body) -> psi at the
 * new position -> sigma advection (PPM) and damping-zone relaxation -> Sussman
 * reinitialisation -> materials (Eqs. ls_flow, ls_solid) -> consistent transport
 * and Crank-Nicolson momentum with implicit Brinkman term (Eqs.
 * c_discrete_momentum, bp_discrete) -> pressure increment by FGMRES + multigrid ->
 * projection (Eq. c_discrete_continuity).  pto_force is added to -c zdot^n.
 * out (host, may be NULL) receives the step record; the call synchronises the
 * tank's stream when out != NULL.  Returns the step's status.  A solve that does
 * not converge still completes the step (WEC_ERR_NOT_CONVERGED). */
int wec_step(wec_tank *tank, double dt, double pto_force, wec_step_result *out);

/* nsteps steps; pto_forces (host, nsteps values, or NULL = zeros); out_n (host,
 * nsteps records, or NULL).  Stops at the first step whose status is not WEC_OK
 * and returns it. */
int wec_step_n(wec_tank *tank, int nsteps, double dt, const double *pto_forces,
               wec_step_result *out_n);

/* ---------------------------------------------------------------- batches --
 * Many independent tanks (uneven sizes, waves, bodies) stepping together: one
 * CUDA graph launch per batch step runs every tank's whole step as independent
 * branches, so the tanks' kernels share the GPU concurrently.  Each tank is the
 * same as one made by wec_tank_create (its own multigrid tile autotuning, its
 * own results; a batch step gives each tank exactly the bits a wec_step would).
 *
 * wec_batch_create: ntanks (1..4096) descriptions, each argument an array of
 * ntanks host structs (copied), validated as in wec_tank_create; the batch owns
 * the tanks.  cuda_stream: the caller's stream (ordering only).
 * wec_batch_step: dt[ntanks] (> 0), pto_force[ntanks] or NULL (zeros),
 * out[ntanks] records or NULL.  Host-synchronous.  Returns WEC_OK, or the first
 * tank's non-OK status (WEC_ERR_NOT_CONVERGED etc.; every tank still stepped).
 * wec_batch_step_n: nsteps batch steps; dt, pto_force, out are [nsteps][ntanks]
 * row-major.  Stops at the first hard error.
 * wec_batch_tank: borrow tank i (fields, state, checkpoints, a single wec_step;
 * valid until wec_batch_destroy, not to be destroyed by the caller).
 * With event profiling on (wec_profile_enable), batch steps launch each tank's
 * kernels one by one instead of the batch graph. */
typedef struct wec_batch wec_batch;

int wec_batch_create(int ntanks, const wec_grid *grids, const wec_fluids *fluids, const wec_waves *waves,
                     const wec_body *bodies, const wec_solver_opts *opts, void *cuda_stream, wec_batch **out);
int wec_batch_size(const wec_batch *batch);
int wec_batch_tank(wec_batch *batch, int i, wec_tank **out);
int wec_batch_step(wec_batch *batch, const double *dt, const double *pto_force, wec_step_result *out);
int wec_batch_step_n(wec_batch *batch, int nsteps, const double *dt, const double *pto_force,
                     wec_step_result *out);
void wec_batch_destroy(wec_batch *batch);

/* ------------------------------------------------- static-grid NLFK force --
 * Non-linear Froude-Krylov force (paper: section "Non-linear Froude-Krylov
 * (NLFK) forces: A novel static grid approach based on implicit surfaces", Eqs.
 * p_dynamic and NLFK_p), independent of any tank.  A static region R of nx x ny
 * square cells of size h, lower-left corner (x0, y0), covers the body and the
 * wave surface's excursion.  Per cell the incident surface sigma = y - (depth +
 * eta(x, t)) marks water (sigma <= 0); the box body (wec_body: xc, width, height;
 * centre height yc given per call) marks the body by its SDF psi.  mode 0: the
 * incident-wave pressure of Eq. p_dynamic, summed over the wave components
 * (wave numbers from the dispersion relation at this depth); mode 1: the
 * hydrostatic pressure -rho_w g (y - depth) (the nonlinear-buoyancy variant).
 * Both are zero where sigma > 0.  The force sums -p_f n_f h over the faces whose
 * two cells have opposite psi sign (p_f interpolated to psi = 0 with |psi|
 * weights, n_f out of the body): *fy heave, *fx surge, per unit span.
 * wec_nlfk_create copies the waves (amp, omega, phase; host) and validates all
 * arguments (WEC_ERR_INVALID); wec_nlfk_force is host-synchronous on the
 * object's stream; results are reproducible bit for bit. */
typedef struct {
    double x0, y0, h;
    int nx, ny;
} wec_region;

typedef struct wec_nlfk wec_nlfk;

int wec_nlfk_create(const wec_region *region, const wec_fluids *fluids, double depth, const wec_waves *waves,
                    const wec_body *body, void *cuda_stream, wec_nlfk **out);
int wec_nlfk_force(wec_nlfk *nlfk, double t, double yc, int mode, double *fx, double *fy);
void wec_nlfk_destroy(wec_nlfk *nlfk);

/* ------------------------------------------------- learned warm start -----
 * A convolutional U-Net, trained on the pressure problems the tank itself
 * solves, predicts a step's pressure increment phi (the solution of the
 * incremental projection's A phi = b) from b and the face coefficients beta; the
 * prediction is the solver's initial guess, checked by its FP64 residual.
 *
 * Network (BF16 tensors and weights on the tensor cores, FP32 accumulation,
 * FP32 master weights): two 3x3 convolutions per level with 32, 64, 128 and 256
 * channels; a 2x2 stride-2 convolution down; nearest upsampling by 2 followed by
 * a 3x3 convolution up; the level's skip tensor concatenated after the
 * upsampled one; ReLU after every convolution; no normalisation layers; a 1x1
 * FP32 head.  Tensors are NHWC: N images of H rows (y) by W columns (x).
 * Parameters (FP32, wec_net_param_count() of them), layer by layer: enc0a
 * (2->32), enc0b, down0 (32->64), enc1a, enc1b, down1, enc2a, enc2b, down2,
 * enc3a, enc3b (256), up2 (256->128), cat2 (256->128), dec2, up1, cat1, dec1,
 * up0, cat0, dec0 (32), head (32->1); each layer's weights [kh][kw][cin][cout]
 * (head: [32][1]) followed by its bias [cout].
 *
 * Features of a pressure problem, per cell c (FP32): beta_c is the mean of the
 * cell's four face coefficients (wall faces count as 0) and rms(b) the root
 * mean square of b over the cells;
 *   x[c][0] = b_c / rms(b),   x[c][1] = log(rho_w beta_c / dt) / 4,
 *   target t_c = phi_c beta_c / rms(b), prediction phi_c = out_c rms(b) / beta_c.
 * (All zero when b = 0.)
 *
 * Each call runs on the net's stream (or, for a tank's guess, the tank's) and
 * is host-synchronous where it returns a host value.  A net serves one tank at a
 * time.  Invalid sizes, batch < 1 or > max_batch, n != wec_net_param_count():
 * WEC_ERR_INVALID. */
typedef struct wec_net wec_net;

size_t wec_net_param_count(void);
/* H, W: multiples of 8, >= 8; max_batch >= 1.  Weights start at zero. */
int wec_net_create(int H, int W, int max_batch, void *cuda_stream, wec_net **out);
void wec_net_destroy(wec_net *net);
/* Host FP32 parameter vectors (layout above); set also resets the Adam state. */
int wec_net_set_params(wec_net *net, const float *host, size_t n);
int wec_net_get_params(const wec_net *net, float *host, size_t n);
/* BF16 output (raw 16-bit words) of layer (0 = enc0a .. 19 = dec0, the order
 * above) from the last forward pass over `batch` images, in the library's
 * chunk-planar layout [batch][h][cout / 8][w][8] (h = H >> level, w = W >> level:
 * the 8 channels [8q, 8q + 8) of a whole image row are contiguous); n must equal
 * batch x h x w x cout. */
int wec_net_get_activation(const wec_net *net, int layer, int batch, unsigned short *host, size_t n);
/* Gradient of the last wec_net_loss_grad / wec_net_train_step. */
int wec_net_get_grads(const wec_net *net, float *host, size_t n);
/* out = net(x).  x: device FP32 [batch][H][W][2]; out: device FP32 [batch][H][W]. */
int wec_net_forward(wec_net *net, int batch, const float *x, float *out);
/* Mean squared error of net(x) against target (device FP32 [batch][H][W]) into
 * *loss (host), and its gradient (kept in the net). */
int wec_net_loss_grad(wec_net *net, int batch, const float *x, const float *target, double *loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with
 * learning rate lr > 0 on the kept gradient. */
int wec_net_adam(wec_net *net, float lr);
/* wec_net_loss_grad on samples idx[0..batch) (host indices) of a dataset in
 * device memory -- xs [S][H][W][2], ts [S][H][W], FP32 -- then wec_net_adam. */
int wec_net_train_step(wec_net *net, const float *xs, const float *ts, const int *idx, int batch, float lr,
                       double *loss);
/* Features x (device FP32 [ny][nx][2]) and target t (device FP32 [ny][nx]) of
 * the pressure problem of the tank's last step. */
int wec_net_sample(wec_tank *tank, float *x, float *t);
/* From the next step on, the tank's solve starts from the net's prediction
 * (net H = ny, W = nx; NULL: from zero again).  The prediction is kept only if
 * its FP64 residual ||b - A phi0|| is below ||b||; otherwise phi0 = 0 (the plain
 * method).  The tank does not own the net: keep it alive while it is set. */
int wec_tank_set_net(wec_tank *tank, wec_net *net);
/* Steps that ran with a net (*tried) and kept its prediction (*kept). */
int wec_tank_net_stats(const wec_tank *tank, long long *tried, long long *kept);

/* Execution mode.  enable = 1 (default): the whole step -- including the
 * pressure solve's iteration, steered on the GPU by conditional WHILE / IF graph
 * nodes -- runs as one CUDA graph, captured at the first step and replayed.
 * enable = 0: kernels are launched one by one and the solver's progress is read
 * by the host once per iteration.  Both run the same kernels in the same order
 * (identical results).  Event profiling (wec_profile_enable) uses mode 0. */
int wec_tank_use_graph(wec_tank *tank, int enable);

/* Solve A p = rhs with the tank's pressure operator of its last step (face
 * coefficients 1/D; Neumann walls, p = 0 above the top row).  rhs, p: device,
 * nx*ny doubles; p holds the initial guess on entry and the solution on exit.
 * rtol > 0; iters / final_rel_residual (host, may be NULL).  Errors:
 * WEC_ERR_INVALID before the first step (no operator yet), WEC_ERR_NOT_CONVERGED. */
int wec_pressure_solve(wec_tank *tank, const double *rhs, double *p, double rtol, int *iters,
                       double *final_rel_residual);

/* Copy a field (ids above) to / from host memory; n must equal the field's size.
 * Setting a read-only field is WEC_ERR_INVALID.  Synchronous. */
int wec_get_field(const wec_tank *tank, int field_id, double *host_dst, size_t n);
int wec_set_field(wec_tank *tank, int field_id, const double *host_src, size_t n);

/* Body/time state: out[0..4] = t, yc (body centre y), zdot, zdot^{n-1}, yc at creation. */
int wec_get_state(const wec_tank *tank, double *out5);
int wec_set_state(wec_tank *tank, double t, double yc, double zdot, double zdot_prev);

/* Checkpoint: *n receives the byte size when buf is NULL; otherwise buf (host,
 * *n bytes) receives (sigma, u, v, p, t, yc, zdot, zdot_prev).  wec_load restores
 * it into a tank of the same size; resuming reproduces the same steps bit for bit. */
int wec_save(const wec_tank *tank, void *buf, size_t *n);
int wec_load(wec_tank *tank, const void *buf, size_t n);

/* ---- standalone pressure solver on caller coefficients ------------------ */
/* The operator of the pressure equation on an nx x ny grid: (A p)_c = sum over
 * the cell's faces of beta_f (p_c - p_nb), with the left, right and bottom walls
 * Neumann whatever beta holds there and the top face Dirichlet p = 0 (ghost -p_c,
 * i.e. 2 beta_top p_c).  Preconditioner: one multigrid V(mg_pre, mg_post) cycle
 * (red-black Gauss-Seidel, 2x2 sum restriction, piecewise-constant prolongation,
 * coarse faces = mean of the two fine faces, dense LU on the coarsest level).
 * nx, ny >= 2. */
int wec_poisson_create(int nx, int ny, const wec_solver_opts *opts, void *cuda_stream,
                       wec_poisson **out);
void wec_poisson_destroy(wec_poisson *P);
/* beta_u: device, (nx+1)*ny; beta_v: device, nx*(ny+1).  Copied; builds the hierarchy. */
int wec_poisson_set_coefficients(wec_poisson *P, const double *beta_u, const double *beta_v);
/* y = A x (device, nx*ny each). */
int wec_poisson_apply(wec_poisson *P, const double *x, double *y);
/* x = M^{-1} b: one V-cycle from a zero guess (device, nx*ny each), in the
 * object's precision (FP32 arithmetic for WEC_PREC_MIXED, FP64 values in/out). */
int wec_poisson_vcycle(wec_poisson *P, const double *b, double *x);
/* FGMRES(restart) right-preconditioned by the V-cycle; x: device, guess in,
 * solution out.  Converged when ||b - A x||_2 <= rtol ||b||_2 (true residual). */
int wec_poisson_solve(wec_poisson *P, const double *b, double *x, double rtol, int max_iters,
                      int *iters, double *final_rel_residual);

/* ---- three dimensions ---------------------------------------------------- */
/* The pressure operator of the projection with d = 3 (section "Continuous
 * equations of motion"; z vertical) on an nx x ny x nz cell grid:
 * (A p)_c = sum over the cell's six faces of beta_f (p_c - p_nb), the walls
 * x = 0, x = lx, y = 0, y = ly and the bed Neumann whatever beta holds there,
 * the top face Dirichlet p = 0 (ghost -p_c).  Layouts, x fastest: cells
 * [nz][ny][nx]; beta_x [nz][ny][nx+1]; beta_y [nz][ny+1][nx]; beta_z
 * [nz+1][ny][nx] (face k below cell layer k).  The same object type and the
 * same apply / vcycle / solve calls as in 2D (vectors of nx*ny*nz doubles).
 * Preconditioner: one V(mg_pre, mg_post) cycle with red-black Gauss-Seidel
 * (colour (i+j+k) mod 2), 2x2x2 sum restriction, piecewise-constant
 * prolongation, coarse face = half the sum of the four fine faces it covers,
 * dense LU on the coarsest level; coarsening halves all three sizes while all
 * are even and >= 4, and must end at <= 512 cells.  WEC_PREC_MIXED runs the
 * V-cycle in FP32 (FP32 copies of the hierarchy) inside the FP64 FGMRES.
 * nx, ny >= 2, nz >= 2; every face array below 2^31 entries; otherwise
 * WEC_ERR_INVALID. */
int wec_poisson_create3(int nx, int ny, int nz, const wec_solver_opts *opts, void *cuda_stream,
                        wec_poisson **out);
/* beta_x, beta_y, beta_z: device, sizes as above.  Copied; builds the
 * hierarchy.  WEC_ERR_INVALID on a 2D object (and set_coefficients on a 3D one). */
int wec_poisson_set_coefficients3(wec_poisson *P, const double *beta_x, const double *beta_y,
                                  const double *beta_z);

/* ---- the three-dimensional tank (level-set part) ------------------------ */
/* Uniform 3D grid, z vertical: h = lx / nx = ly / ny = lz / nz; nx, nz >= 4,
 * ny >= 1, ny, nz <= 65535; depth = still-water depth above the bed. */
typedef struct {
    int nx, ny, nz;
    double lx, ly, lz, depth;
} wec_grid3;

/* Heaving vertical cylinder (the configuration's buoy): axis at (xc, yc),
 * centre height zc (per call of wec_tank3_materials), radius, length, mass;
 * SDF psi = max(r - radius, |z - zc| - length / 2) (section "Interface
 * tracking", CSG intersection of a cylinder and a slab); solid density
 * mass / (pi radius^2 length).  present = 0: no body. */
typedef struct {
    int present;
    double xc, yc, radius, length, mass;
    double zc, kappa_p, added_mass, pto_damping; /* initial centre height; Brinkman
                                                     permeability; artificial added mass of
                                                     the stabilised heave update; linear PTO
                                                     damper c (F_PTO = f_pto - c zdot) */
} wec_cylinder;

typedef struct wec_tank3 wec_tank3;

/* Fields (FP64, x fastest): cells [nz][ny][nx]; u [nz][ny][nx+1], v
 * [nz][ny+1][nx], w [nz+1][ny][nx] (face k of w below cell layer k). */
enum {
    WEC_F3_SIGMA = 0, WEC_F3_U = 1, WEC_F3_V = 2, WEC_F3_W = 3, /* state: get and set */
    WEC_F3_RHO = 4, WEC_F3_MU = 5, WEC_F3_RHO_FLOW = 6, WEC_F3_CHI = 7, /* materials: get */
    WEC_F3_P = 8 /* p^{n-1/2} (cells; state of a stepping tank): get and set */
};

/* The level-set part of the 3D step on the GPU (FP64): sigma, the face
 * velocities and the materials.  Waves travel along x (uniform along y): the
 * components of wec_waves give the inflow ghost z - depth - eta(x, t) of sigma
 * (k from the dispersion relation) and the damping zone [damp_x0,
 * damp_x0 + damp_len] at the outlet.  All fields start at zero.  Host arrays
 * are copied; the calls synchronise the object's stream before returning. */
int wec_tank3_create(const wec_grid3 *grid, const wec_fluids *fluids, const wec_waves *waves,
                     const wec_cylinder *body, const wec_solver_opts *opts, void *cuda_stream,
                     wec_tank3 **out);
void wec_tank3_destroy(wec_tank3 *tank);
/* host_dst / host_src: n doubles, n = the field's size (WEC_ERR_INVALID otherwise;
 * only the state fields can be set).  The material fields hold the last
 * wec_tank3_materials call, or a step's time level n: everywhere after an FP64 or
 * WEC_PREC_MIXED_MG step; after a WEC_PREC_MIXED or WEC_PREC_MIXED_DF step (whose
 * stencils use working copies) only in the box of cells of the force integral
 * around the cylinder and the cells just before it in x, y and z. */
int wec_tank3_get_field(const wec_tank3 *tank, int field_id, double *host_dst, size_t n);
int wec_tank3_set_field(wec_tank3 *tank, int field_id, const double *host_src, size_t n);
/* Two-stage materials (Eqs. ls_flow then ls_solid, half-width h) from sigma and
 * the cylinder centred at height zc: rho, mu, rho^flow and chi = 1 - H_body. */
int wec_tank3_materials(wec_tank3 *tank, double zc);
/* sigma <- sigma - dt Q(u, sigma) (single-stage PPM per direction; section
 * "Level set advection"), then the damping-zone blend toward z - depth; ghosts
 * of sigma at time t (inflow: the incident wave; outlet and side walls: zero
 * gradient; bed and top: linear extrapolation). */
int wec_tank3_advect(wec_tank3 *tank, double dt, double t);
/* nit Sussman pseudo-steps (TVD-RK2, d tau = 0.3 h) toward |grad sigma| = 1 with
 * the sign of sigma at the call (section "Interface tracking"); ghosts at t. */
int wec_tank3_reinit(wec_tank3 *tank, int nit, double t);
/* One time step of the 3D tank (needs opts at creation).  Precision: WEC_PREC_FP64;
 * WEC_PREC_MIXED_MG (FP32 V-cycles in the FP64 solve, FP64 stencils); WEC_PREC_MIXED_DF
 * (FP32 V-cycles, the stencils -- materials, advection, reinitialisation, transport,
 * viscous terms, Jacobi sweeps -- in double-float arithmetic over float-pair working
 * copies of the FP64 state); WEC_PREC_MIXED (the same stencils in FP32 over FP32
 * working copies).  In every mode the force, heave, beta, right-hand side, solve
 * residual and Krylov basis, projection and fields are FP64.
 * The step: heave force from p^{n-1/2}, u^n (Eq.
 * int_fh: pressure interpolated to psi = 0 and the normal viscous stress on
 * z-faces, the shear stresses on x- and y-faces, face area h^2); heave update
 * (Eq. newton_u, stabilised by added_mass); sigma advection + damping zone and
 * n_reinit reinitialisation pseudo-steps; materials at n+1; consistent transport
 * and the Crank-Nicolson momentum system (n_jacobi Jacobi sweeps; Dirichlet:
 * Airy inflow u at x = 0, u = 0 at the outlet, v = 0 on the side walls, w = 0 on
 * the bed; vorticity damping over the top four cells, momentum damping in the
 * zone); the pressure increment with beta = 1 / D (rtol, FGMRES + V-cycle) and
 * the projection.  At creation with opts: sigma = z - depth - eta(x, 0), the
 * incident Airy velocities, p = the discrete hydrostatic pressure of rho^flow.
 * out: the step record (z relative to the initial zc; eta at (probe_x, ly / 2)).
 * Returns the solver's status (WEC_ERR_NOT_CONVERGED still advances the state). */
int wec_tank3_step(wec_tank3 *tank, double dt, double pto_force, wec_step_result *out);
/* t, zc, zdot, zc at creation, zdot of the previous step. */
int wec_tank3_get_state(const wec_tank3 *tank, double *out5);

/* ---- without device allocation ------------------------------------------ */
/* ||b - A x||_2 for the pressure operator above (same coefficient layout and
 * boundary rules as wec_poisson_*), written to *norm_out (device, 1 double).
 * The paper has no counterpart: this exists for callers that cannot allocate
 * device memory when they need the number -- e.g. a control loop under a fixed
 * memory budget, or a process whose device memory all belongs to another
 * allocator.  The call allocates nothing: its scratch (608 per-block partial
 * sums and a completion counter, about 4.9 KB) is one file-scope device array,
 * held by every GPU that loads the library until exit.  Grids of up to
 * nx * ny <= 2^28 cells are accepted (32-bit face indexing); larger sizes
 * return WEC_ERR_INVALID.  beta_u, beta_v, x, b: device, caller
 * owned, layouts as in wec_poisson_set_coefficients.  Enqueued on cuda_stream
 * (NULL = legacy default stream); *norm_out is valid once that stream reaches
 * it.  The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.  The
 * address is kept for the life of the process: calls after a cudaDeviceReset
 * are not supported.  All calls share the one array: calls that overlap on the
 * GPU (different streams, no ordering between them) race and may return wrong
 * norms. */
int wec_residual_norm_noalloc(int nx, int ny, const double *beta_u, const double *beta_v, const double *x,
                              const double *b, double *norm_out, void *cuda_stream);

/* ---- conversion check of the double-float stencils ------------------------ */
/* The double-float stencils (WEC_PREC_MIXED_DF) and the FP32 ones convert
 * between their working types and the FP64 state with integer operations
 * instead of this GPU's conversion instructions, which issue on its narrow FP64
 * pipe.  This call checks those conversions against the instructions on n
 * values (device, caller owned): for each value d, float(d) rounded to nearest
 * and the float pair of d (nearest float, then the nearest float of the
 * remainder), each widened back to double.  *mismatches (device, one unsigned
 * long long, caller owned) receives the number of values for which any result
 * differs in any bit.  Enqueued on cuda_stream (NULL = legacy default);
 * WEC_ERR_INVALID for n < 0 or NULL pointers. */
int wec_check_conversions(long long n, const double *values, unsigned long long *mismatches, void *cuda_stream);

/* ---- host wave utilities (no device work) ------------------------------- */
/* k solving omega^2 = g k tanh(k d) (Eq. dispersion_relation), |residual| <= 1e-14 omega^2. */
double wec_wave_number(double omega, double depth, double g);
/* Fenton's explicit k d (Eq. explicit_dispersion_relation). */
double wec_wave_number_fenton_kd(double omega, double depth, double g);
/* JONSWAP sea state as ncomp Airy components (Eq. wave_spectrum_amplitude with the
 * Bretschneider shape of Eq. Bretshneider_wave_spec, its period taken so that the
 * spectrum peaks at 2 pi / Tp, times the peak enhancement gamma^r, r =
 * exp(-(w - wp)^2 / (2 s^2 wp^2)), s = 0.07 / 0.09); equal bins over
 * [1.6 / 3.5955, 20 / 3.5955] wp at their mid-points; amplitudes rescaled so that
 * 4 sqrt(sum a^2 / 2) = Hs.  amp, omega: host, ncomp each (outputs). */
int wec_jonswap(double Hs, double Tp, double gamma, int ncomp, double *amp, double *omega);

/* ---- process-wide options ------------------------------------------------ */
/* "mg_fused" (default 1): the multigrid V-cycle runs as one shared-memory tile
 * kernel per fine level for pre-smoothing + residual + restriction, one for
 * prolongation + post-smoothing, and one single-CTA kernel, staged in shared
 * memory, for the levels of at most 4096 cells; 0 launches one kernel per colour
 * pass, restriction and prolongation.  Both compute the same values up to
 * rounding.  "mg_autotune" (default 1): when a solver is created, time the fused
 * kernels' tile shapes (64x16, 32x16, 32x8, 16x8) on each level and keep the
 * fastest, then time whole V-cycles with the single-CTA kernel starting at the
 * smallest admissible level or one or two levels coarser and keep the fastest;
 * 0 uses 64x16 everywhere and the smallest admissible level.  Tuning results
 * are kept per (grid, precision, mg_pre, mg_post) for the life of the process:
 * later solvers of the same shape reuse them and compute the same bits.
 * "mg_bottom_shift" (default -1 = autotuned): start the single-CTA kernel this
 * many levels below the smallest admissible one (0..8, capped at the coarsest).
 * "mg3_bottom" (default 1): the 3D V-cycle runs its levels of at most 8192
 * cells, down to the coarsest, in one 1024-thread CTA (iterates and right-hand
 * sides in shared memory); 0 launches them level by level.  Both compute the same
 * bits.
 * "tank3_split_momentum" (default 1): the 3D momentum system per component as
 * two kernels (transport terms, then viscous terms and assembly); 0: one
 * kernel.  Both form the same terms: the same bits with double-float stencils,
 * the same values to rounding in FP64 and FP32 (where the compiler may fuse a
 * product into a sum differently in each kernel).
 * Options apply to solvers created, graphs captured and solves started after the
 * call.  Unknown name or value out of range: WEC_ERR_INVALID. */
int wec_set_option(const char *name, int value);

/* Fused multigrid tile shape (interior cells) per level of the tank's solver, as
 * chosen by the autotuner when the tank was created ("mg_autotune" option; the
 * coarsest level's entry is meaningless; 0 x 0 marks a level run inside the
 * single-CTA kernel).  *nlev receives the number of levels; at most max entries
 * are written. */
int wec_tank_mg_tiles(const wec_tank *tank, int *tile_x, int *tile_y, int max, int *nlev);

/* ---- launch accounting and profiling ------------------------------------ */
/* Number of kernels this library has launched in the process so far. */
long long wec_launch_count(void);
/* mode 0: off; 1: time every kernel launch with a CUDA event pair on its stream;
 * 2: time only kernels whose name equals `only`.  Names are the kernel names
 * reported by wec_profile_read (e.g. "mg_rbgs"). */
int wec_profile_enable(int mode, const char *only);
/* Aggregate the timed launches since the last read, per (kernel name, multigrid
 * level; -1 = not a multigrid kernel), and forget them.  Synchronises on the
 * recorded events.  *count receives the number of aggregates; at most max are
 * written: names (max rows of name_stride chars), levels, launches, total ms and
 * total algorithmic bytes (the bytes the operation must read and write at least
 * once, as counted by the launch site). */
int wec_profile_read(int max, char *names, size_t name_stride, int *levels, long long *launches, double *ms,
                     double *bytes, int *count);

/* Message of the last failing call on this thread ("" if none). */
const char *wec_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* WEC_H */
