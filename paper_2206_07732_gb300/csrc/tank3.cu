// The three-dimensional tank (wec_tank3): its level-set part -- materials,
// advection and reinitialisation of sigma on an nx x ny x nz grid with z
// vertical and a heaving vertical cylinder (sections "Interface tracking",
// "Level set advection", "Density and viscosity specification", d = 3) -- as
// FP64 kernels, one thread per cell, x fastest.  The 3D pressure equation is
// the wec_poisson object made by wec_poisson_create3.
//
// Readings (the two-dimensional ones carried to three directions):
//   materials: H_flow(sigma) then H_body(psi) with half-width h; psi of the
//     cylinder = max(r - R, |z - z_c| - L / 2), r the distance to its axis; solid
//     density m / (pi R^2 L), solid viscosity mu_w; chi = 1 - H_body;
//   advection: single-stage PPM (van Leer-limited edge slopes, CW84 limiter,
//     characteristic tracing) along each direction, sigma* = sigma - dt Q with
//     Q the sum over directions of the mean face velocity times the difference
//     of the upwind face states / h, then the Jacobsen damping-zone blend toward
//     z - depth;
//   ghosts of sigma: x < 0 the incident wave's z - depth - eta(x, t); beyond the
//     outlet and outside the side walls zero gradient; below the bed and above
//     the top linear extrapolation;
//   reinitialisation: Sussman relaxation, Godunov Hamiltonian on ENO-2
//     differences with minmod corrections, TVD-RK2, d tau = 0.3 h, sign of the
//     input field S = sigma0 / sqrt(sigma0^2 + h^2).
#include <cmath>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "internal.cuh"

struct Tank3P {
    int nx, ny, nz;
    double h, ih, depth, rho_w, rho_a, mu_w, mu_a, rho_s;
    int has_body;
    double bxc, byc, br, blen;
    int ncomp;
    const double *amp, *omega, *kw, *phase;  // device
    const double *damp;                       // device, [nx]: damping-zone weight of each column
};

struct wec_tank3 {
    Tank3P P{};
    cudaStream_t st = nullptr;
    size_t nc = 0, nu = 0, nv = 0, nw = 0;
    double *sig = nullptr, *tmp = nullptr, *s0 = nullptr, *s1 = nullptr;
    double *u = nullptr, *v = nullptr, *w = nullptr;
    double *rho = nullptr, *mu = nullptr, *rhof = nullptr, *chi = nullptr;
    double *consts = nullptr;  // wave components and damping table
};

namespace wec {
namespace {

constexpr double kPi3 = 3.14159265358979323846;

__device__ __forceinline__ double heav3(double phi, double eps)
{
    if (phi < -eps) return 0.0;
    if (phi > eps) return 1.0;
    return 0.5 * (1.0 + phi / eps + sin(kPi3 * phi / eps) / kPi3);
}

__device__ double eta3(const Tank3P &P, double x, double t)
{
    double e = 0.0;
    for (int c = 0; c < P.ncomp; ++c) e += P.amp[c] * cos(P.kw[c] * x - P.omega[c] * t + P.phase[c]);
    return e;
}

// sigma at (i, j, k), with the ghosts of the header
__device__ __forceinline__ double sig3(const Tank3P &P, const double *__restrict__ s, int i, int j, int k, double t)
{
    if (i < 0) return (k + 0.5) * P.h - P.depth - eta3(P, (i + 0.5) * P.h, t);
    i = min(i, P.nx - 1);
    j = min(max(j, 0), P.ny - 1);
    const long long col = (long long)j * P.nx + i, pl = (long long)P.nx * P.ny;
    if (k < 0) return s[col] + k * (s[pl + col] - s[col]);
    if (k > P.nz - 1) {
        const double a = s[(P.nz - 1) * pl + col], b = s[(P.nz - 2) * pl + col];
        return a + (k - (P.nz - 1)) * (a - b);
    }
    return s[k * pl + col];
}

__device__ __forceinline__ double vl3(double am, double a0, double ap)
{
    const double dl = a0 - am, dr = ap - a0;
    if (dl * dr <= 0.0) return 0.0;
    const double dc = 0.5 * (ap - am);
    const double m = fmin(fabs(dc), fmin(2.0 * fabs(dl), 2.0 * fabs(dr)));
    return dc > 0.0 ? m : -m;
}

// limited PPM edge values (eL, eR) of the middle cell of a[0..4]
__device__ __forceinline__ void ppm_edges3(const double *a, double &eL, double &eR)
{
    const double dm = vl3(a[0], a[1], a[2]), d0 = vl3(a[1], a[2], a[3]), dp = vl3(a[2], a[3], a[4]);
    double L = a[1] + 0.5 * (a[2] - a[1]) - (d0 - dm) / 6.0;
    double R = a[2] + 0.5 * (a[3] - a[2]) - (dp - d0) / 6.0;
    const double c = a[2];
    if ((R - c) * (c - L) <= 0.0) {
        L = c;
        R = c;
    } else {
        const double dA = R - L, m6 = dA * (c - 0.5 * (L + R)), q = dA * dA / 6.0;
        if (m6 > q)
            L = 3.0 * c - 2.0 * R;
        else if (-q > m6)
            R = 3.0 * c - 2.0 * L;
    }
    eL = L;
    eR = R;
}

// time-centred upwind state at the face between a[2] and a[3] (a: cells f-3 .. f+2)
__device__ __forceinline__ double ppm_face3(const double *a, double vel, double dt, double h)
{
    double L, R;
    if (vel >= 0.0) {
        ppm_edges3(a, L, R);
        const double C = vel * dt / h, dA = R - L, a6 = 6.0 * (a[2] - 0.5 * (L + R));
        return R - 0.5 * C * (dA - (1.0 - 2.0 * C / 3.0) * a6);
    }
    ppm_edges3(a + 1, L, R);
    const double C = -vel * dt / h, dA = R - L, a6 = 6.0 * (a[3] - 0.5 * (L + R));
    return L + 0.5 * C * (dA + (1.0 - 2.0 * C / 3.0) * a6);
}

struct Cell3 {
    int i, j, k;
    long long c;
};

__device__ __forceinline__ bool cell_of(const Tank3P &P, Cell3 &q)
{
    q.i = blockIdx.x * blockDim.x + threadIdx.x;
    q.j = blockIdx.y;
    q.k = blockIdx.z;
    if (q.i >= P.nx) return false;
    q.c = ((long long)q.k * P.ny + q.j) * P.nx + q.i;
    return true;
}

__global__ void __launch_bounds__(128) k3t_materials(Tank3P P, const double *__restrict__ sig, double zc,
                                                     double *__restrict__ rho, double *__restrict__ mu,
                                                     double *__restrict__ rhof, double *__restrict__ chi)
{
    pdl_entry();
    Cell3 q;
    if (!cell_of(P, q)) return;
    const double h = P.h;
    double psi = 1.0e3;
    if (P.has_body) {
        const double x = (q.i + 0.5) * h - P.bxc, y = (q.j + 0.5) * h - P.byc, z = (q.k + 0.5) * h - zc;
        psi = fmax(sqrt(x * x + y * y) - P.br, fabs(z) - 0.5 * P.blen);
    }
    const double hf = heav3(sig[q.c], h), hb = heav3(psi, h);
    const double rf = P.rho_w + (P.rho_a - P.rho_w) * hf;
    const double mf = P.mu_w + (P.mu_a - P.mu_w) * hf;
    rho[q.c] = P.rho_s + (rf - P.rho_s) * hb;
    mu[q.c] = P.mu_w + (mf - P.mu_w) * hb;
    rhof[q.c] = rf;
    chi[q.c] = 1.0 - hb;
}

__global__ void __launch_bounds__(128) k3t_advect(Tank3P P, const double *__restrict__ s, const double *__restrict__ u,
                                                  const double *__restrict__ v, const double *__restrict__ w, double dt,
                                                  double t, double *__restrict__ out)
{
    pdl_entry();
    Cell3 q;
    if (!cell_of(P, q)) return;
    const int nx = P.nx, ny = P.ny, i = q.i, j = q.j, k = q.k;
    const long long r = (long long)k * ny + j, fu = r * (nx + 1) + i, fv = ((long long)k * (ny + 1) + j) * nx + i;
    const long long pl = (long long)nx * ny;
    const double h = P.h;
    double a[6], fx[2], fy[2], fz[2];
    for (int f = 0; f < 2; ++f) {
#pragma unroll
        for (int m = 0; m < 6; ++m) a[m] = sig3(P, s, i + f - 3 + m, j, k, t);
        fx[f] = ppm_face3(a, u[fu + f], dt, h);
#pragma unroll
        for (int m = 0; m < 6; ++m) a[m] = sig3(P, s, i, j + f - 3 + m, k, t);
        fy[f] = ppm_face3(a, v[fv + f * nx], dt, h);
#pragma unroll
        for (int m = 0; m < 6; ++m) a[m] = sig3(P, s, i, j, k + f - 3 + m, t);
        fz[f] = ppm_face3(a, w[q.c + f * pl], dt, h);
    }
    const double ub = 0.5 * (u[fu] + u[fu + 1]);
    const double vb = 0.5 * (v[fv] + v[fv + nx]);
    const double wb = 0.5 * (w[q.c] + w[q.c + pl]);
    const double Q = ub * (fx[1] - fx[0]) / h + vb * (fy[1] - fy[0]) / h + wb * (fz[1] - fz[0]) / h;
    const double sa = s[q.c] - dt * Q;
    const double al = P.damp[i];
    out[q.c] = (1.0 - al) * sa + al * ((k + 0.5) * h - P.depth);
}

__device__ __forceinline__ double mm3(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

// S(sigma0) (|grad f| - 1) at a cell
__device__ double reinit_rhs3(const Tank3P &P, const double *__restrict__ f, const double *__restrict__ s0,
                              const Cell3 &q, double t)
{
    const double h = P.h, c = f[q.c];
    const double sg0 = s0[q.c];
    const bool pos = sg0 > 0.0;
    double g2 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int di = d == 0, dj = d == 1, dk = d == 2;
        const double m2 = sig3(P, f, q.i - 2 * di, q.j - 2 * dj, q.k - 2 * dk, t);
        const double m1 = sig3(P, f, q.i - di, q.j - dj, q.k - dk, t);
        const double p1 = sig3(P, f, q.i + di, q.j + dj, q.k + dk, t);
        const double p2 = sig3(P, f, q.i + 2 * di, q.j + 2 * dj, q.k + 2 * dk, t);
        const double dm = m2 - 2.0 * m1 + c, d0 = m1 - 2.0 * c + p1, dp = c - 2.0 * p1 + p2;
        const double a = (c - m1) / h + mm3(dm, d0) / (2.0 * h);
        const double b = (p1 - c) / h - mm3(d0, dp) / (2.0 * h);
        double g;
        if (pos) {
            const double x = fmax(a, 0.0), y = fmin(b, 0.0);
            g = fmax(x * x, y * y);
        } else {
            const double x = fmin(a, 0.0), y = fmax(b, 0.0);
            g = fmax(x * x, y * y);
        }
        g2 = d == 0 ? g : g2 + g;
    }
    const double S = sg0 / sqrt(sg0 * sg0 + h * h);
    return S * (sqrt(g2) - 1.0);
}

// stage 1: out = f - dtau L(f); stage 2: out = (out + (f - dtau L(f))) / 2 with
// out holding sigma at the start of the pseudo-step
__global__ void __launch_bounds__(128) k3t_reinit_stage(Tank3P P, const double *__restrict__ f,
                                                        const double *__restrict__ s0, double *out, double t,
                                                        double dtau, int stage)
{
    pdl_entry();
    Cell3 q;
    if (!cell_of(P, q)) return;
    const double y = f[q.c] - dtau * reinit_rhs3(P, f, s0, q, t);
    out[q.c] = stage == 1 ? y : 0.5 * (out[q.c] + y);
}

dim3 grid3(const Tank3P &P) { return dim3((P.nx + 127) / 128, P.ny, P.nz); }

int tank3_check(const wec_tank3 *T)
{
    if (!T) return fail(WEC_ERR_INVALID, "tank3 is NULL");
    return WEC_OK;
}

}  // namespace
}  // namespace wec

using namespace wec;

extern "C" {

int wec_tank3_create(const wec_grid3 *grid, const wec_fluids *fl, const wec_waves *wv, const wec_cylinder *body,
                     void *cuda_stream, wec_tank3 **out)
{
    if (!out) return fail(WEC_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!grid || !fl || !wv || !body) return fail(WEC_ERR_INVALID, "NULL argument");
    const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
    if (nx < 4 || ny < 1 || nz < 4) return fail(WEC_ERR_INVALID, "tank3: need nx >= 4, ny >= 1, nz >= 4");
    if (ny > 65535 || nz > 65535) return fail(WEC_ERR_INVALID, "tank3: ny, nz must be <= 65535");
    const double h = grid->lx / nx;
    if (!(h > 0.0) || std::fabs(grid->ly / ny - h) > 1e-9 * h || std::fabs(grid->lz / nz - h) > 1e-9 * h)
        return fail(WEC_ERR_INVALID, "tank3: the grid must be uniform (lx/nx = ly/ny = lz/nz)");
    if (!(fl->rho_w > 0.0) || !(fl->rho_a > 0.0) || !(fl->mu_w >= 0.0) || !(fl->mu_a >= 0.0))
        return fail(WEC_ERR_INVALID, "tank3: densities must be positive, viscosities non-negative");
    if (wv->ncomp < 0 || (wv->ncomp > 0 && (!wv->amp || !wv->omega || !wv->phase)))
        return fail(WEC_ERR_INVALID, "tank3: wave arrays are NULL");
    if (body->present && (!(body->radius > 0.0) || !(body->length > 0.0) || !(body->mass > 0.0)))
        return fail(WEC_ERR_INVALID, "tank3: the cylinder needs radius, length and mass > 0");
    if (int e = [] {
            int n = 0;
            return (cudaGetDeviceCount(&n) != cudaSuccess || n == 0)
                       ? fail(WEC_ERR_CUDA, "no CUDA device available (libwec has no CPU path)")
                       : WEC_OK;
        }())
        return e;
    wec_tank3 *T = new (std::nothrow) wec_tank3();
    if (!T) return fail(WEC_ERR_NOMEM, "host allocation failed");
    T->st = (cudaStream_t)cuda_stream;
    Tank3P &P = T->P;
    P.nx = nx; P.ny = ny; P.nz = nz; P.h = h; P.ih = 1.0 / h; P.depth = grid->depth;
    P.rho_w = fl->rho_w; P.rho_a = fl->rho_a; P.mu_w = fl->mu_w; P.mu_a = fl->mu_a;
    P.has_body = body->present ? 1 : 0;
    P.rho_s = fl->rho_w;
    if (P.has_body) {
        P.bxc = body->xc; P.byc = body->yc; P.br = body->radius; P.blen = body->length;
        P.rho_s = body->mass / (kPi3 * body->radius * body->radius * body->length);
    }
    P.ncomp = wv->ncomp;
    // host tables: wave components (k from the dispersion relation) and the
    // damping-zone weight of each column (Jacobsen's (e^{xi^3.5} - 1) / (e - 1))
    std::vector<double> hc(4 * (size_t)P.ncomp + nx);
    for (int c = 0; c < P.ncomp; ++c) {
        hc[c] = wv->amp[c];
        hc[P.ncomp + c] = wv->omega[c];
        hc[2 * P.ncomp + c] = wave_number(wv->omega[c], grid->depth, fl->g);
        hc[3 * P.ncomp + c] = wv->phase[c];
    }
    for (int i = 0; i < nx; ++i) {
        const double x = (i + 0.5) * h;
        double a = 0.0;
        if (wv->damp_len > 0.0 && x > wv->damp_x0) {
            double xi = (x - wv->damp_x0) / wv->damp_len;
            if (xi > 1.0) xi = 1.0;
            a = (std::exp(std::pow(xi, 3.5)) - 1.0) / (std::exp(1.0) - 1.0);
        }
        hc[4 * (size_t)P.ncomp + i] = a;
    }
    T->nc = (size_t)nx * ny * nz;
    T->nu = (size_t)(nx + 1) * ny * nz;
    T->nv = (size_t)nx * (ny + 1) * nz;
    T->nw = (size_t)nx * ny * (nz + 1);
    cudaError_t e = cudaSuccess;
    double **cells[] = {&T->sig, &T->tmp, &T->s0, &T->s1, &T->rho, &T->mu, &T->rhof, &T->chi};
    for (double **p : cells)
        if (e == cudaSuccess) e = cudaMalloc(p, T->nc * 8);
    if (e == cudaSuccess) e = cudaMalloc(&T->u, T->nu * 8);
    if (e == cudaSuccess) e = cudaMalloc(&T->v, T->nv * 8);
    if (e == cudaSuccess) e = cudaMalloc(&T->w, T->nw * 8);
    if (e == cudaSuccess) e = cudaMalloc(&T->consts, hc.size() * 8);
    if (e == cudaSuccess) e = cudaMemcpy(T->consts, hc.data(), hc.size() * 8, cudaMemcpyHostToDevice);
    for (double *p : {T->sig, T->tmp, T->s0, T->s1, T->rho, T->mu, T->rhof, T->chi})
        if (e == cudaSuccess && p) e = cudaMemset(p, 0, T->nc * 8);
    if (e == cudaSuccess) e = cudaMemset(T->u, 0, T->nu * 8);
    if (e == cudaSuccess) e = cudaMemset(T->v, 0, T->nv * 8);
    if (e == cudaSuccess) e = cudaMemset(T->w, 0, T->nw * 8);
    if (e != cudaSuccess) {
        wec_tank3_destroy(T);
        return cuda_fail(e, "tank3 allocation");
    }
    P.amp = T->consts;
    P.omega = T->consts + P.ncomp;
    P.kw = T->consts + 2 * P.ncomp;
    P.phase = T->consts + 3 * P.ncomp;
    P.damp = T->consts + 4 * P.ncomp;
    *out = T;
    return WEC_OK;
}

void wec_tank3_destroy(wec_tank3 *T)
{
    if (!T) return;
    cudaStreamSynchronize(T->st);
    for (double *p : {T->sig, T->tmp, T->s0, T->s1, T->rho, T->mu, T->rhof, T->chi, T->u, T->v, T->w, T->consts})
        cudaFree(p);
    delete T;
}

static double *field3(const wec_tank3 *T, int f, size_t *n)
{
    switch (f) {
    case WEC_F3_SIGMA: *n = T->nc; return T->sig;
    case WEC_F3_U: *n = T->nu; return T->u;
    case WEC_F3_V: *n = T->nv; return T->v;
    case WEC_F3_W: *n = T->nw; return T->w;
    case WEC_F3_RHO: *n = T->nc; return T->rho;
    case WEC_F3_MU: *n = T->nc; return T->mu;
    case WEC_F3_RHO_FLOW: *n = T->nc; return T->rhof;
    case WEC_F3_CHI: *n = T->nc; return T->chi;
    default: *n = 0; return nullptr;
    }
}

int wec_tank3_get_field(const wec_tank3 *T, int f, double *host, size_t n)
{
    if (int e = tank3_check(T)) return e;
    size_t m = 0;
    double *p = field3(T, f, &m);
    if (!p || !host || n != m) return fail(WEC_ERR_INVALID, "tank3_get_field: unknown field or wrong size");
    WEC_CK(cudaStreamSynchronize(T->st));
    WEC_CK(cudaMemcpy(host, p, m * 8, cudaMemcpyDeviceToHost));
    return WEC_OK;
}

int wec_tank3_set_field(wec_tank3 *T, int f, const double *host, size_t n)
{
    if (int e = tank3_check(T)) return e;
    size_t m = 0;
    double *p = field3(T, f, &m);
    if (!p || !host || n != m || f > WEC_F3_W) return fail(WEC_ERR_INVALID, "tank3_set_field: not a state field or wrong size");
    WEC_CK(cudaStreamSynchronize(T->st));
    WEC_CK(cudaMemcpy(p, host, m * 8, cudaMemcpyHostToDevice));
    return WEC_OK;
}

int wec_tank3_materials(wec_tank3 *T, double zc)
{
    if (int e = tank3_check(T)) return e;
    {
        WEC_PROF("tank3_materials", 0, 40.0 * T->nc, T->st);
        launch_k(k3t_materials, grid3(T->P), 128, 0, T->st, T->P, (const double *)T->sig, zc, T->rho, T->mu, T->rhof,
                 T->chi);
    }
    WEC_CK(cudaGetLastError());
    WEC_CK(cudaStreamSynchronize(T->st));
    return WEC_OK;
}

int wec_tank3_advect(wec_tank3 *T, double dt, double t)
{
    if (int e = tank3_check(T)) return e;
    if (!(dt >= 0.0)) return fail(WEC_ERR_INVALID, "tank3_advect: dt must be >= 0");
    {
        WEC_PROF("tank3_advect", 0, 8.0 * (2.0 * T->nc + T->nu + T->nv + T->nw), T->st);
        launch_k(k3t_advect, grid3(T->P), 128, 0, T->st, T->P, (const double *)T->sig, (const double *)T->u,
                 (const double *)T->v, (const double *)T->w, dt, t, T->tmp);
    }
    WEC_CK(cudaGetLastError());
    std::swap(T->sig, T->tmp);
    WEC_CK(cudaStreamSynchronize(T->st));
    return WEC_OK;
}

int wec_tank3_reinit(wec_tank3 *T, int nit, double t)
{
    if (int e = tank3_check(T)) return e;
    if (nit < 0) return fail(WEC_ERR_INVALID, "tank3_reinit: nit must be >= 0");
    const double dtau = 0.3 * T->P.h;
    WEC_CK(cudaMemcpyAsync(T->s0, T->sig, T->nc * 8, cudaMemcpyDeviceToDevice, T->st));
    for (int it = 0; it < nit; ++it) {
        {
            WEC_PROF("tank3_reinit", 0, 24.0 * T->nc, T->st);
            launch_k(k3t_reinit_stage, grid3(T->P), 128, 0, T->st, T->P, (const double *)T->sig,
                     (const double *)T->s0, T->s1, t, dtau, 1);
        }
        WEC_PROF("tank3_reinit", 0, 32.0 * T->nc, T->st);
        launch_k(k3t_reinit_stage, grid3(T->P), 128, 0, T->st, T->P, (const double *)T->s1, (const double *)T->s0,
                 T->sig, t, dtau, 2);
    }
    WEC_CK(cudaGetLastError());
    WEC_CK(cudaStreamSynchronize(T->st));
    return WEC_OK;
}

}  // extern "C"
