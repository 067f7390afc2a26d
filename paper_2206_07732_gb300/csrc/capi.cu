// C ABI of libwec: argument checking, object lifetime, host<->device copies.
// Every compute step runs in the CUDA kernels of step.cu / solver.cu.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tank.cuh"

namespace wec {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    g_err = std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ") in " + what;
    return e == cudaErrorMemoryAllocation ? WEC_ERR_NOMEM : WEC_ERR_CUDA;
}

static int check_device()
{
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) return fail(WEC_ERR_CUDA, "no CUDA device available (libwec has no CPU path)");
    return WEC_OK;
}

static int check_opts(const wec_solver_opts *o)
{
    if (!o) return fail(WEC_ERR_INVALID, "solver options are NULL");
    if (o->precision != WEC_PREC_FP64 && o->precision != WEC_PREC_MIXED && o->precision != WEC_PREC_MIXED_MG &&
        o->precision != WEC_PREC_MIXED_DF)
        return fail(WEC_ERR_INVALID,
                    "precision must be WEC_PREC_FP64, WEC_PREC_MIXED, WEC_PREC_MIXED_MG or WEC_PREC_MIXED_DF");
    if (!(o->rtol > 0.0) || o->max_iters < 1) return fail(WEC_ERR_INVALID, "rtol must be > 0 and max_iters >= 1");
    if (o->restart < 1 || o->restart > kMaxRestart) return fail(WEC_ERR_INVALID, "restart must be in 1..32");
    if (o->n_reinit < 0 || o->n_jacobi < 1 || o->mg_pre < 1 || o->mg_post < 0 || o->mg_pre > 4 || o->mg_post > 4)
        return fail(WEC_ERR_INVALID, "need n_reinit >= 0, n_jacobi >= 1, 1 <= mg_pre <= 4, 0 <= mg_post <= 4");
    if (o->n_cycles > 1) return fail(WEC_ERR_INVALID, "n_cycles > 1 is built for the 3D tank (wec_tank3) only");
    return WEC_OK;
}

// Wait for the caller's stream and the tank's own stream.
static cudaError_t sync_tank(const wec_tank *T)
{
    cudaError_t e = cudaStreamSynchronize(T->st);
    if (e == cudaSuccess && T->gst) e = cudaStreamSynchronize(T->gst);
    return e;
}

static double *field_ptr(const wec_tank *T, int id, size_t *n, bool *writable)
{
    *writable = false;
    switch (id) {
    case WEC_F_SIGMA: *n = T->nc; *writable = true; return T->sig;
    case WEC_F_U: *n = T->nu; *writable = true; return T->u;
    case WEC_F_V: *n = T->nv; *writable = true; return T->v;
    case WEC_F_P: *n = T->nc; *writable = true; return T->p;
    case WEC_F_USTAR: *n = T->nu; return T->us;
    case WEC_F_VSTAR: *n = T->nv; return T->vs;
    case WEC_F_BETA_U: *n = T->nu; return T->solver.L64[0].bu;
    case WEC_F_BETA_V: *n = T->nv; return T->solver.L64[0].bv;
    case WEC_F_RHS: *n = T->nc; return T->rhs;
    case WEC_F_SIGMA_ADV: *n = T->nc; return T->sa;
    }
    *n = 0;
    return nullptr;
}

}  // namespace wec

using namespace wec;

namespace wec {

int validate_tank(const wec_grid *grid, const wec_fluids *fl, const wec_waves *wv, const wec_body *body,
                  const wec_solver_opts *opts)
{
    if (!grid || !fl || !wv || !body) return fail(WEC_ERR_INVALID, "NULL argument");
    if (int e = check_opts(opts)) return e;
    if (opts->precision == WEC_PREC_MIXED_DF)
        return fail(WEC_ERR_INVALID, "WEC_PREC_MIXED_DF is built for the 3D tank and 3D solver only");
    if (grid->nx < 8 || grid->ny < 8 || (grid->nx & 1) || (grid->ny & 1))
        return fail(WEC_ERR_INVALID, "nx, ny must be even and >= 8");
    double h = grid->lx / grid->nx;
    if (!(h > 0.0) || std::fabs(grid->ly / grid->ny - h) > 1e-12 * h)
        return fail(WEC_ERR_INVALID, "grid spacing must be uniform: lx / nx == ly / ny");
    if (!(grid->depth > 0.0 && grid->depth < grid->ly)) return fail(WEC_ERR_INVALID, "depth must be in (0, ly)");
    if (!(fl->rho_w > 0 && fl->rho_a > 0 && fl->mu_w >= 0 && fl->mu_a >= 0 && fl->g >= 0))
        return fail(WEC_ERR_INVALID, "densities must be > 0, viscosities and g >= 0");
    if (wv->ncomp < 0 || (wv->ncomp > 0 && (!wv->amp || !wv->omega || !wv->phase)))
        return fail(WEC_ERR_INVALID, "waves: ncomp < 0 or NULL component arrays");
    for (int c = 0; c < wv->ncomp; ++c)
        if (!(wv->omega[c] > 0.0) || !std::isfinite(wv->amp[c]) || !std::isfinite(wv->phase[c]))
            return fail(WEC_ERR_INVALID, "waves: omega must be > 0 and amp, phase finite");
    if (body->present) {
        if (!(body->width > 0 && body->height > 0 && body->mass > 0 && body->kappa_p > 0 && body->added_mass >= 0))
            return fail(WEC_ERR_INVALID, "body: width, height, mass, kappa_p must be > 0, added_mass >= 0");
    }
    return WEC_OK;
}

}  // namespace wec

extern "C" {

const char *wec_last_error(void) { return g_err.c_str(); }

int wec_tank_create(const wec_grid *grid, const wec_fluids *fl, const wec_waves *wv, const wec_body *body,
                    const wec_solver_opts *opts, void *cuda_stream, wec_tank **out)
{
    if (!out) return fail(WEC_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (int e = validate_tank(grid, fl, wv, body, opts)) return e;
    const double h = grid->lx / grid->nx;
    if (int e = check_device()) return e;

    wec_tank *T = new (std::nothrow) wec_tank();
    if (!T) return fail(WEC_ERR_NOMEM, "host allocation failed");
    T->opts = *opts;
    T->st = (cudaStream_t)cuda_stream;
    TankP &P = T->P;
    P.nx = grid->nx; P.ny = grid->ny; P.h = h; P.lx = grid->lx; P.ly = grid->ly; P.depth = grid->depth;
    P.rho_w = fl->rho_w; P.rho_a = fl->rho_a; P.mu_w = fl->mu_w; P.mu_a = fl->mu_a; P.g = fl->g;
    P.damp_x0 = wv->damp_x0; P.damp_len = wv->damp_len; P.probe_x = wv->probe_x;
    P.has_body = body->present ? 1 : 0;
    if (body->present) {
        P.bxc = body->xc; P.bw = body->width; P.bh = body->height; P.mass = body->mass;
        P.added_mass = body->added_mass; P.kappa_p = body->kappa_p; P.pto_c = body->pto_damping;
        P.rho_s = body->mass / (body->width * body->height);  // uniform solid
    } else {
        P.bw = P.bh = P.mass = 1.0;
        P.kappa_p = 1e-8;
        P.rho_s = fl->rho_w;
    }
    P.mu_s = fl->mu_w;
    P.ih = 1.0 / h;
    P.ikp = 1.0 / P.kappa_p;
    P.cd = TankC<double>{P.h, P.ih, P.depth, P.g, P.rho_w, P.rho_a, P.rho_s, P.mu_w, P.mu_a, P.mu_s, P.ikp,
                         P.bxc, P.bw, P.bh};
    P.cf = TankC<float>{(float)P.h, (float)P.ih, (float)P.depth, (float)P.g, (float)P.rho_w, (float)P.rho_a,
                        (float)P.rho_s, (float)P.mu_w, (float)P.mu_a, (float)P.mu_s, (float)P.ikp, (float)P.bxc,
                        (float)P.bw, (float)P.bh};
    P.ncomp = wv->ncomp;
    int rc = WEC_OK;
    {
        std::vector<double> hw(4 * (size_t)(wv->ncomp > 0 ? wv->ncomp : 1), 0.0);
        for (int c = 0; c < wv->ncomp; ++c) {
            hw[c] = wv->amp[c];
            hw[wv->ncomp + c] = wv->omega[c];
            hw[2 * wv->ncomp + c] = wave_number(wv->omega[c], grid->depth, fl->g);
            hw[3 * wv->ncomp + c] = wv->phase[c];
        }
        cudaError_t e = cudaMalloc(&T->waves, hw.size() * 8);
        if (e == cudaSuccess) e = cudaMemcpy(T->waves, hw.data(), hw.size() * 8, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = cuda_fail(e, "wave components");
        P.amp = T->waves;
        P.omega = T->waves + wv->ncomp;
        P.kw = T->waves + 2 * wv->ncomp;
        P.phase = T->waves + 3 * wv->ncomp;
    }
    if (rc == WEC_OK) rc = tank_alloc_and_init(T);
    if (rc == WEC_OK) {
        StepScalars &s = *T->Sh;
        s = StepScalars{};
        s.yc = s.yc0 = s.yc1 = body->present ? body->yc : 0.0;
        rc = tank_init_pressure(T);
    }
    if (rc != WEC_OK) {
        std::string msg = g_err;
        tank_free(T);
        delete T;
        g_err = msg;
        return rc;
    }
    *out = T;
    return WEC_OK;
}

void wec_tank_destroy(wec_tank *T)
{
    if (!T) return;
    cudaStreamSynchronize(T->st);
    if (T->gst) cudaStreamSynchronize(T->gst);
    tank_free(T);
    delete T;
}

int wec_step(wec_tank *T, double dt, double pto_force, wec_step_result *out)
{
    if (!T) return fail(WEC_ERR_INVALID, "tank is NULL");
    if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(pto_force))
        return fail(WEC_ERR_INVALID, "dt must be > 0 and finite, pto_force finite");
    return tank_step(T, dt, pto_force, out);
}

int wec_step_n(wec_tank *T, int nsteps, double dt, const double *pto, wec_step_result *out_n)
{
    if (!T || nsteps < 0) return fail(WEC_ERR_INVALID, "tank is NULL or nsteps < 0");
    for (int k = 0; k < nsteps; ++k) {
        int e = wec_step(T, dt, pto ? pto[k] : 0.0, out_n ? out_n + k : nullptr);
        if (e != WEC_OK) return e;
    }
    return WEC_OK;
}

int wec_set_option(const char *name, int value)
{
    if (!name) return fail(WEC_ERR_INVALID, "option name is NULL");
    if (std::string(name) == "mg_fused") {
        set_mg_fused(value != 0);
        return WEC_OK;
    }
    if (std::string(name) == "mg_autotune") {
        set_mg_autotune(value != 0);
        return WEC_OK;
    }
    if (std::string(name) == "mg3_bottom") {
        set_mg3_bottom(value != 0);
        return WEC_OK;
    }
    if (std::string(name) == "tank3_split_momentum") {
        set_tank3_split_momentum(value != 0);
        return WEC_OK;
    }
    if (std::string(name) == "mg_bottom_shift") {
        if (value < -1 || value > 8) return fail(WEC_ERR_INVALID, "mg_bottom_shift must be in -1..8");
        set_mg_bottom_shift(value);
        return WEC_OK;
    }
    return fail(WEC_ERR_INVALID, std::string("unknown option: ") + name);
}

int wec_tank_mg_tiles(const wec_tank *T, int *tile_x, int *tile_y, int max, int *nlev)
{
    if (!T || !nlev || (max > 0 && (!tile_x || !tile_y))) return fail(WEC_ERR_INVALID, "NULL argument");
    *nlev = T->solver.nlev;
    poisson_tiles(&T->solver, tile_x, tile_y, max);
    return WEC_OK;
}

int wec_tank_use_graph(wec_tank *T, int enable)
{
    if (!T) return fail(WEC_ERR_INVALID, "tank is NULL");
    T->use_graph = enable != 0;
    return WEC_OK;
}

int wec_pressure_solve(wec_tank *T, const double *rhs, double *p, double rtol, int *iters, double *relres)
{
    if (!T || !rhs || !p) return fail(WEC_ERR_INVALID, "NULL argument");
    if (!T->stepped) return fail(WEC_ERR_INVALID, "no pressure operator yet: take a step first");
    if (!(rtol > 0.0)) return fail(WEC_ERR_INVALID, "rtol must be > 0");
    // the caller's device buffers are ordered on the caller's stream
    WEC_CK(cudaEventRecord(T->ev_in, T->st));
    WEC_CK(cudaStreamWaitEvent(T->gst, T->ev_in, 0));
    T->solver.st = T->gst;
    int rc = poisson_solve(&T->solver, rhs, p, rtol, T->opts.max_iters, iters, relres);
    WEC_CK(cudaEventRecord(T->ev_out, T->gst));
    WEC_CK(cudaStreamWaitEvent(T->st, T->ev_out, 0));
    return rc;
}

int wec_get_field(const wec_tank *T, int id, double *dst, size_t n)
{
    if (!T || !dst) return fail(WEC_ERR_INVALID, "NULL argument");
    size_t m;
    bool w;
    double *src = field_ptr(T, id, &m, &w);
    if (!src) return fail(WEC_ERR_INVALID, "unknown field id");
    if (n != m) return fail(WEC_ERR_INVALID, "field size mismatch: expected " + std::to_string(m));
    WEC_CK(sync_tank(T));
    WEC_CK(cudaMemcpy(dst, src, n * 8, cudaMemcpyDeviceToHost));
    return WEC_OK;
}

int wec_set_field(wec_tank *T, int id, const double *src, size_t n)
{
    if (!T || !src) return fail(WEC_ERR_INVALID, "NULL argument");
    size_t m;
    bool w;
    double *dst = field_ptr(T, id, &m, &w);
    if (!dst) return fail(WEC_ERR_INVALID, "unknown field id");
    if (!w) return fail(WEC_ERR_INVALID, "field is read-only");
    if (n != m) return fail(WEC_ERR_INVALID, "field size mismatch: expected " + std::to_string(m));
    WEC_CK(sync_tank(T));
    WEC_CK(cudaMemcpy(dst, src, n * 8, cudaMemcpyHostToDevice));
    return WEC_OK;
}

int wec_get_state(const wec_tank *T, double *out5)
{
    if (!T || !out5) return fail(WEC_ERR_INVALID, "NULL argument");
    WEC_CK(sync_tank(T));
    StepScalars s;
    WEC_CK(cudaMemcpy(&s, T->S, sizeof(s), cudaMemcpyDeviceToHost));
    out5[0] = s.t; out5[1] = s.yc; out5[2] = s.zdot; out5[3] = s.zdot_prev; out5[4] = s.yc0;
    return WEC_OK;
}

int wec_set_state(wec_tank *T, double t, double yc, double zdot, double zdot_prev)
{
    if (!T) return fail(WEC_ERR_INVALID, "tank is NULL");
    WEC_CK(sync_tank(T));
    StepScalars s;
    WEC_CK(cudaMemcpy(&s, T->S, sizeof(s), cudaMemcpyDeviceToHost));
    s.t = t; s.yc = yc; s.zdot = zdot; s.zdot_prev = zdot_prev;
    WEC_CK(cudaMemcpy(T->S, &s, sizeof(s), cudaMemcpyHostToDevice));
    return WEC_OK;
}

static const uint64_t kMagic = 0x3143454b4e415457ull;  // "WTANKEC1"

int wec_save(const wec_tank *T, void *buf, size_t *n)
{
    if (!T || !n) return fail(WEC_ERR_INVALID, "NULL argument");
    size_t need = 16 + 8 * (2 * T->nc + T->nu + T->nv + 4);
    if (!buf) {
        *n = need;
        return WEC_OK;
    }
    if (*n < need) return fail(WEC_ERR_INVALID, "checkpoint buffer too small");
    WEC_CK(sync_tank(T));
    char *q = (char *)buf;
    uint64_t hdr[2] = {kMagic, ((uint64_t)T->P.nx << 32) | (uint32_t)T->P.ny};
    memcpy(q, hdr, 16);
    q += 16;
    WEC_CK(cudaMemcpy(q, T->sig, T->nc * 8, cudaMemcpyDeviceToHost)); q += T->nc * 8;
    WEC_CK(cudaMemcpy(q, T->u, T->nu * 8, cudaMemcpyDeviceToHost)); q += T->nu * 8;
    WEC_CK(cudaMemcpy(q, T->v, T->nv * 8, cudaMemcpyDeviceToHost)); q += T->nv * 8;
    WEC_CK(cudaMemcpy(q, T->p, T->nc * 8, cudaMemcpyDeviceToHost)); q += T->nc * 8;
    StepScalars s;
    WEC_CK(cudaMemcpy(&s, T->S, sizeof(s), cudaMemcpyDeviceToHost));
    double sc[4] = {s.t, s.yc, s.zdot, s.zdot_prev};
    memcpy(q, sc, 32);
    *n = need;
    return WEC_OK;
}

int wec_load(wec_tank *T, const void *buf, size_t n)
{
    if (!T || !buf) return fail(WEC_ERR_INVALID, "NULL argument");
    size_t need = 16 + 8 * (2 * T->nc + T->nu + T->nv + 4);
    if (n != need) return fail(WEC_ERR_INVALID, "checkpoint size does not match this tank");
    const char *q = (const char *)buf;
    uint64_t hdr[2];
    memcpy(hdr, q, 16);
    if (hdr[0] != kMagic || hdr[1] != (((uint64_t)T->P.nx << 32) | (uint32_t)T->P.ny))
        return fail(WEC_ERR_INVALID, "checkpoint header does not match this tank");
    q += 16;
    WEC_CK(sync_tank(T));
    WEC_CK(cudaMemcpy(T->sig, q, T->nc * 8, cudaMemcpyHostToDevice)); q += T->nc * 8;
    WEC_CK(cudaMemcpy(T->u, q, T->nu * 8, cudaMemcpyHostToDevice)); q += T->nu * 8;
    WEC_CK(cudaMemcpy(T->v, q, T->nv * 8, cudaMemcpyHostToDevice)); q += T->nv * 8;
    WEC_CK(cudaMemcpy(T->p, q, T->nc * 8, cudaMemcpyHostToDevice)); q += T->nc * 8;
    double sc[4];
    memcpy(sc, q, 32);
    return wec_set_state(T, sc[0], sc[1], sc[2], sc[3]);
}

static int poisson_create_any(int nx, int ny, int nz, const wec_solver_opts *opts, void *cuda_stream,
                              wec_poisson **out)
{
    if (!out) return fail(WEC_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (int e = check_opts(opts)) return e;
    if (int e = check_device()) return e;
    wec_poisson *P = new (std::nothrow) wec_poisson();
    if (!P) return fail(WEC_ERR_NOMEM, "host allocation failed");
    int rc = poisson_init(P, nx, ny, opts->precision, opts->restart, opts->mg_pre, opts->mg_post,
                          (cudaStream_t)cuda_stream, nz);
    if (rc != WEC_OK) {
        std::string msg = g_err;
        poisson_free(P);
        delete P;
        g_err = msg;
        return rc;
    }
    *out = P;
    return WEC_OK;
}

int wec_poisson_create(int nx, int ny, const wec_solver_opts *opts, void *cuda_stream, wec_poisson **out)
{
    return poisson_create_any(nx, ny, 1, opts, cuda_stream, out);
}

int wec_poisson_create3(int nx, int ny, int nz, const wec_solver_opts *opts, void *cuda_stream, wec_poisson **out)
{
    if (out) *out = nullptr;
    if (nz < 2) return fail(WEC_ERR_INVALID, "poisson3: nz must be >= 2");
    return poisson_create_any(nx, ny, nz, opts, cuda_stream, out);
}

void wec_poisson_destroy(wec_poisson *P)
{
    if (!P) return;
    cudaStreamSynchronize(P->st);
    poisson_free(P);
    delete P;
}

int wec_poisson_set_coefficients(wec_poisson *P, const double *bu, const double *bv)
{
    if (!P || !bu || !bv) return fail(WEC_ERR_INVALID, "NULL argument");
    if (P->nz > 1) return fail(WEC_ERR_INVALID, "a 3D operator takes wec_poisson_set_coefficients3");
    size_t nu = (size_t)(P->nx + 1) * P->ny, nv = (size_t)P->nx * (P->ny + 1);
    WEC_CK(cudaMemcpyAsync(P->L64[0].bu, bu, nu * 8, cudaMemcpyDeviceToDevice, P->st));
    WEC_CK(cudaMemcpyAsync(P->L64[0].bv, bv, nv * 8, cudaMemcpyDeviceToDevice, P->st));
    int e = poisson_build(P, P->st);
    if (e) return e;
    WEC_CK(cudaStreamSynchronize(P->st));
    return WEC_OK;
}

int wec_poisson_set_coefficients3(wec_poisson *P, const double *bx, const double *by, const double *bz)
{
    if (!P || !bx || !by || !bz) return fail(WEC_ERR_INVALID, "NULL argument");
    if (P->nz == 1) return fail(WEC_ERR_INVALID, "a 2D operator takes wec_poisson_set_coefficients");
    const size_t nx = P->nx, ny = P->ny, nz = P->nz;
    WEC_CK(cudaMemcpyAsync(P->L64[0].bu, bx, (nx + 1) * ny * nz * 8, cudaMemcpyDeviceToDevice, P->st));
    WEC_CK(cudaMemcpyAsync(P->L64[0].bv, by, nx * (ny + 1) * nz * 8, cudaMemcpyDeviceToDevice, P->st));
    WEC_CK(cudaMemcpyAsync(P->L64[0].bw, bz, nx * ny * (nz + 1) * 8, cudaMemcpyDeviceToDevice, P->st));
    int e = poisson_build(P, P->st);
    if (e) return e;
    WEC_CK(cudaStreamSynchronize(P->st));
    return WEC_OK;
}

int wec_poisson_apply(wec_poisson *P, const double *x, double *y)
{
    if (!P || !x || !y) return fail(WEC_ERR_INVALID, "NULL argument");
    if (!P->have_coef) return fail(WEC_ERR_INVALID, "set the coefficients first");
    int e = poisson_apply(P, x, y);
    if (e) return e;
    WEC_CK(cudaStreamSynchronize(P->st));
    return WEC_OK;
}

int wec_poisson_vcycle(wec_poisson *P, const double *b, double *x)
{
    if (!P || !b || !x) return fail(WEC_ERR_INVALID, "NULL argument");
    if (!P->have_coef) return fail(WEC_ERR_INVALID, "set the coefficients first");
    int e = poisson_vcycle(P, b, x);
    if (e) return e;
    WEC_CK(cudaStreamSynchronize(P->st));
    return WEC_OK;
}

int wec_poisson_solve(wec_poisson *P, const double *b, double *x, double rtol, int max_iters, int *iters,
                      double *relres)
{
    if (!P || !b || !x) return fail(WEC_ERR_INVALID, "NULL argument");
    if (!P->have_coef) return fail(WEC_ERR_INVALID, "set the coefficients first");
    if (!(rtol > 0.0) || max_iters < 1) return fail(WEC_ERR_INVALID, "rtol must be > 0, max_iters >= 1");
    return poisson_solve(P, b, x, rtol, max_iters, iters, relres);
}

double wec_wave_number(double omega, double depth, double g) { return wave_number(omega, depth, g); }

double wec_wave_number_fenton_kd(double omega, double depth, double g)
{
    return wave_number_fenton_kd(omega, depth, g);
}

int wec_jonswap(double Hs, double Tp, double gamma, int ncomp, double *amp, double *omega)
{
    if (ncomp < 1 || !amp || !omega || !(Hs >= 0) || !(Tp > 0) || !(gamma >= 1))
        return fail(WEC_ERR_INVALID, "jonswap: need ncomp >= 1, Hs >= 0, Tp > 0, gamma >= 1");
    return jonswap(Hs, Tp, gamma, ncomp, amp, omega);
}

}  // extern "C"
