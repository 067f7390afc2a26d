// Tank state and device helpers shared by the step kernels and the C ABI.
#pragma once

#include "internal.cuh"

namespace wec {

// Per-tank constants, passed to kernels by value.
// Tank constants the stencil kernels read, in their compute type (an FP32
// kernel reading FP64 constants would convert them on the FP64 pipe).
template <typename R>
struct TankC {
    R h, ih, depth, g, rho_w, rho_a, rho_s, mu_w, mu_a, mu_s, ikp, bxc, bw, bh;
};

struct TankP {
    int nx, ny;
    double h, ih, lx, ly, depth;  // ih = 1 / h
    double rho_w, rho_a, rho_s, mu_w, mu_a, mu_s, g;
    double damp_x0, damp_len, probe_x;
    int has_body;
    double bxc, bw, bh, mass, added_mass, kappa_p, ikp, pto_c;  // ikp = 1 / kappa_p
    int ncomp;
    const double *amp, *omega, *kw, *phase;  // device
    TankC<float> cf;                          // the constants above, FP32
    TankC<double> cd;                         // and FP64
};

// Device-resident scalars of the step (keeps the step free of host round trips).
struct StepScalars {
    double t, yc, zdot, zdot_prev, yc0;  // state at step n
    double yc1, zdot1;                   // body after the heave update
    double F, fpto;                      // force and PTO force of this step
    double div2, eta;                    // diagnostics of the finished step
    long long launches;                  // kernels executed by the last graph replay
};

// Boundary data of one step: inflow at x = 0 and eta at the three ghost columns.
struct Bc {
    double *uin1;  // [ny]   u_in(y_j+1/2, t^{n+1})
    double *vin0;  // [ny+1] v_in(y_j, t^n)
    double *vin1;  // [ny+1] v_in(y_j, t^{n+1})
    double *eta0;  // [3]    eta(-(g+1/2) h, t^n)
    double *eta1;  // [3]    eta(-(g+1/2) h, t^{n+1})
    double *eta_in;  // [2]  eta(0, t^n), eta(0, t^{n+1})
};

}  // namespace wec

struct wec_tank {
    wec::TankP P{};
    wec_solver_opts opts{};
    cudaStream_t st = nullptr;        // caller's stream (ordering only)
    cudaStream_t gst = nullptr;       // the tank's own stream: every kernel runs here
    cudaStream_t h1 = nullptr, h2 = nullptr;  // capture helpers for the solver's conditional bodies
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // the net's guess runs on its own stream beside the multigrid hierarchy build
    cudaStream_t nst = nullptr;
    cudaEvent_t ev_nf = nullptr, ev_nj = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool use_graph = true;
    int n_fixed = 0, n_body = 0, n_close = 0;  // kernels per replay: fixed, per iteration, per cycle
    double *inp = nullptr;            // device: dt, f_pto of the current step
    double *tabs = nullptr;           // device: damping weights / vorticity shape per column / row
    float *tabs32 = nullptr;          // device: the same tables in FP32 (mixed precision)
    double *sgn = nullptr;            // device: Sussman smoothed sign of the step's sigma0
    size_t nc = 0, nu = 0, nv = 0;
    double *sig = nullptr, *sa = nullptr, *r0 = nullptr, *r1 = nullptr, *rt = nullptr;
    double *u = nullptr, *v = nullptr, *us = nullptr, *vs = nullptr;
    double *ua = nullptr, *va = nullptr, *ub = nullptr, *vb = nullptr, *uc = nullptr, *vc = nullptr;
    double *Ru = nullptr, *Rv = nullptr, *Du = nullptr, *Dv = nullptr;
    double *p = nullptr, *phi = nullptr, *rhs = nullptr;
    double *rho_n = nullptr, *mu_n = nullptr, *mu_1 = nullptr, *rf_1 = nullptr, *chi_1 = nullptr;
    double *bcbuf = nullptr, *part = nullptr, *waves = nullptr;
    // Mixed precision: FP32 working copies that the step's stencils read (state
    // mirrors, materials, reinitialisation stages, momentum right-hand sides,
    // Jacobi iterates), one allocation.  nullptr for an FP64 tank.
    float *w32 = nullptr;
    wec::Bc bc{};
    wec::StepScalars *S = nullptr;   // device
    wec::StepScalars *Sh = nullptr;  // pinned host mirror
    wec_poisson solver;
    bool stepped = false;
    bool inp_owned = true;            // false when inp points into a batch's input array
    int last_iters = 0;
    double last_relres = 0.0;
    wec_net *net = nullptr;           // learned initial guess of the solve (not owned)
    long long *net_stats = nullptr;   // device: steps with a net, steps that kept its guess
};

namespace wec {
// Host-side checks of a tank description (no device call); WEC_ERR_INVALID + message.
int validate_tank(const wec_grid *grid, const wec_fluids *fl, const wec_waves *wv, const wec_body *body,
                  const wec_solver_opts *opts);
int tank_alloc_and_init(wec_tank *T);
int tank_init_pressure(wec_tank *T);  // after the host filled T->Sh (initial body state)
int tank_step(wec_tank *T, double dt, double fpto, wec_step_result *out);
// Count the kernels of one step (launch accounting); call before capturing.
int tank_prepare_capture(wec_tank *T);
// Enqueue one whole step (front, conditional-node solve, back, D2H of the step
// record and solver state) on st, which must be capturing; used by the tank's
// own graph and by a batch graph (one branch per tank).
int tank_capture_step(wec_tank *T, cudaStream_t st);
// After a replay that ran the captured step: launch accounting + the record.
int tank_finish_step(wec_tank *T, wec_step_result *out);
void tank_free(wec_tank *T);
// unet.cu: the learned initial guess of the tank's increment (enqueued in the
// step front in place of phi = 0), and the BF16 weight refresh it relies on.
int net_enqueue_guess(wec_tank *T, cudaStream_t st);
int net_sync_weights(wec_net *N);
}  // namespace wec
