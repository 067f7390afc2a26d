// Static-grid non-linear Froude-Krylov force (paper: section "Non-linear
// Froude-Krylov (NLFK) forces: A novel static grid approach based on implicit
// surfaces", Eqs. p_dynamic and NLFK_p).
//
// A box region R of cells around the body is fixed in space.  Per cell, the
// incident-wave surface sigma = y - (d + eta(x, t)) marks water (sigma <= 0) and
// the body SDF psi (box, centre yc at the call's time) marks the body.  The
// incident pressure p_I of Eq. p_dynamic (mode 0, linear superposition over the
// wave components) or the hydrostatic p_H = -rho_w g (y - d) (mode 1, the
// nonlinear-buoyancy variant) is zero in air.  Eq. NLFK_p sums -p_f n_f h over
// the faces whose two cells have opposite psi sign, with p_f interpolated to
// psi = 0 by |psi| weights and n_f out of the body: y-faces give the heave
// force, x-faces the surge force.  One thread per face, fixed-order block and
// final sums (reproducible bit for bit).
#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

struct wec_nlfk {
    wec_region R{};
    double depth = 0.0, rho_w = 0.0, g = 0.0;
    double bxc = 0.0, bw = 0.0, bh = 0.0;
    int ncomp = 0;
    double *waves = nullptr;  // device: amp, omega, kwave, phase (ncomp each)
    double *part = nullptr;   // device: 2 x kNlfkBlocks block sums
    double *out = nullptr;    // device: fx, fy
    cudaStream_t st = nullptr;
};

namespace wec {
namespace {

constexpr int kNlfkThreads = 256;
constexpr int kNlfkBlocks = 304;

struct NlfkP {
    double x0, y0, h;
    int nx, ny;
    double depth, rho_w, g, bxc, bw, bh;
    int ncomp;
    const double *amp, *omega, *kw, *phase;
};

__device__ double nlfk_pressure(const NlfkP &P, double x, double y, double t, int mode)
{
    double eta = 0.0;
    for (int c = 0; c < P.ncomp; ++c) eta += P.amp[c] * cos(P.kw[c] * x - P.omega[c] * t + P.phase[c]);
    const double sigma = y - (P.depth + eta);
    if (sigma > 0.0) return 0.0;
    if (mode == 1) return -P.rho_w * P.g * (y - P.depth);
    double p = 0.0;
    for (int c = 0; c < P.ncomp; ++c) {
        const double k = P.kw[c], d = P.depth;
        // cosh(k (d + sigma)) / cosh(k d) without overflow
        const double ratio = (exp(k * sigma) + exp(-k * (2.0 * d + sigma))) / (1.0 + exp(-2.0 * k * d));
        p += P.rho_w * P.g * P.amp[c] * ratio * cos(k * x - P.omega[c] * t + P.phase[c]);
    }
    return p;
}

__device__ __forceinline__ double nlfk_psi(const NlfkP &P, double x, double y, double yc)
{
    return fmax(fabs(x - P.bxc) - 0.5 * P.bw, fabs(y - yc) - 0.5 * P.bh);
}

__device__ double nlfk_block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kNlfkThreads / 32; ++w) r += sh[w];
    __syncthreads();
    return r;
}

// Block sums of the face contributions: part[b] (fx), part[kNlfkBlocks + b] (fy).
__global__ void __launch_bounds__(kNlfkThreads) k_nlfk_partial(NlfkP P, double t, double yc, int mode, double *part)
{
    pdl_entry();
    __shared__ double sh[kNlfkThreads / 32];
    const long long nyf = (long long)(P.ny - 1) * P.nx, nxf = (long long)P.ny * (P.nx - 1);
    const double h = P.h;
    double fx = 0.0, fy = 0.0;
    for (long long k = blockIdx.x * (long long)kNlfkThreads + threadIdx.x; k < nyf + nxf;
         k += (long long)gridDim.x * kNlfkThreads) {
        double xl, yl, xr, yr;
        bool yface = k < nyf;
        if (yface) {  // between cells (i, j-1) and (i, j)
            const int i = (int)(k % P.nx), j = (int)(k / P.nx) + 1;
            xl = xr = P.x0 + (i + 0.5) * h;
            yl = P.y0 + (j - 0.5) * h;
            yr = P.y0 + (j + 0.5) * h;
        } else {  // between cells (i-1, j) and (i, j)
            const long long q = k - nyf;
            const int i = (int)(q % (P.nx - 1)) + 1, j = (int)(q / (P.nx - 1));
            yl = yr = P.y0 + (j + 0.5) * h;
            xl = P.x0 + (i - 0.5) * h;
            xr = P.x0 + (i + 0.5) * h;
        }
        const double pl = nlfk_psi(P, xl, yl, yc), pr = nlfk_psi(P, xr, yr, yc);
        if (!(pl * pr < 0.0)) continue;
        const double wl = fabs(pl), wr = fabs(pr);
        const double pf = (nlfk_pressure(P, xl, yl, t, mode) * wr + nlfk_pressure(P, xr, yr, t, mode) * wl) / (wl + wr);
        const double n = pl < 0.0 ? 1.0 : -1.0;  // out of the body
        if (yface)
            fy += -pf * n * h;
        else
            fx += -pf * n * h;
    }
    fx = nlfk_block_sum(fx, sh);
    fy = nlfk_block_sum(fy, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = fx;
        part[kNlfkBlocks + blockIdx.x] = fy;
    }
}

__global__ void __launch_bounds__(kNlfkThreads) k_nlfk_final(const double *part, double *out)
{
    pdl_entry();
    __shared__ double sh[kNlfkThreads / 32];
    for (int q = 0; q < 2; ++q) {
        double s = 0.0;
        for (int b = threadIdx.x; b < kNlfkBlocks; b += kNlfkThreads) s += part[q * kNlfkBlocks + b];
        s = nlfk_block_sum(s, sh);
        if (threadIdx.x == 0) out[q] = s;
    }
}

}  // namespace
}  // namespace wec

using namespace wec;

extern "C" {

int wec_nlfk_create(const wec_region *R, const wec_fluids *fl, double depth, const wec_waves *wv,
                    const wec_body *body, void *cuda_stream, wec_nlfk **out)
{
    if (!out) return fail(WEC_ERR_INVALID, "nlfk: out is NULL");
    *out = nullptr;
    if (!R || !fl || !wv || !body) return fail(WEC_ERR_INVALID, "nlfk: NULL argument");
    if (R->nx < 2 || R->ny < 2 || !(R->h > 0.0)) return fail(WEC_ERR_INVALID, "nlfk: region needs nx, ny >= 2 and h > 0");
    if ((long long)R->nx * R->ny > (1LL << 26)) return fail(WEC_ERR_INVALID, "nlfk: region larger than 2^26 cells");
    if (!(depth > 0.0) || !(fl->rho_w > 0.0) || !(fl->g >= 0.0)) return fail(WEC_ERR_INVALID, "nlfk: depth, rho_w > 0, g >= 0");
    if (!body->present || !(body->width > 0.0) || !(body->height > 0.0))
        return fail(WEC_ERR_INVALID, "nlfk: needs a body with width, height > 0");
    if (wv->ncomp < 0 || (wv->ncomp > 0 && (!wv->amp || !wv->omega || !wv->phase)))
        return fail(WEC_ERR_INVALID, "nlfk: ncomp < 0 or NULL component arrays");
    for (int c = 0; c < wv->ncomp; ++c)
        if (!(wv->omega[c] > 0.0) || !std::isfinite(wv->amp[c]) || !std::isfinite(wv->phase[c]))
            return fail(WEC_ERR_INVALID, "nlfk: omega must be > 0 and amp, phase finite");
    wec_nlfk *N = new (std::nothrow) wec_nlfk();
    if (!N) return fail(WEC_ERR_NOMEM, "nlfk: host allocation failed");
    N->R = *R;
    N->depth = depth;
    N->rho_w = fl->rho_w;
    N->g = fl->g;
    N->bxc = body->xc;
    N->bw = body->width;
    N->bh = body->height;
    N->ncomp = wv->ncomp;
    N->st = (cudaStream_t)cuda_stream;
    const int nc = std::max(wv->ncomp, 1);
    std::vector<double> hw(4 * (size_t)nc, 0.0);
    for (int c = 0; c < wv->ncomp; ++c) {
        hw[c] = wv->amp[c];
        hw[nc + c] = wv->omega[c];
        hw[2 * nc + c] = wave_number(wv->omega[c], depth, fl->g);
        hw[3 * nc + c] = wv->phase[c];
    }
    cudaError_t ce = cudaMalloc(&N->waves, hw.size() * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMemcpy(N->waves, hw.data(), hw.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMalloc(&N->part, 2 * kNlfkBlocks * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMalloc(&N->out, 2 * sizeof(double));
    if (ce != cudaSuccess) {
        cudaFree(N->waves);
        cudaFree(N->part);
        cudaFree(N->out);
        delete N;
        return cuda_fail(ce, "nlfk: allocation");
    }
    *out = N;
    return WEC_OK;
}

int wec_nlfk_force(wec_nlfk *N, double t, double yc, int mode, double *fx, double *fy)
{
    if (!N || !fx || !fy) return fail(WEC_ERR_INVALID, "nlfk_force: NULL argument");
    if (mode != 0 && mode != 1) return fail(WEC_ERR_INVALID, "nlfk_force: mode must be 0 (incident) or 1 (hydrostatic)");
    if (!std::isfinite(t) || !std::isfinite(yc)) return fail(WEC_ERR_INVALID, "nlfk_force: t and yc must be finite");
    const int nc = std::max(N->ncomp, 1);
    NlfkP P{N->R.x0, N->R.y0, N->R.h, N->R.nx, N->R.ny, N->depth, N->rho_w, N->g, N->bxc, N->bw, N->bh,
            N->ncomp, N->waves, N->waves + nc, N->waves + 2 * nc, N->waves + 3 * nc};
    {
        WEC_PROF("nlfk", -1, 8.0 * 2 * kNlfkBlocks, N->st);  // computed fields: only the block sums are stored
        WEC_CK(launch_k(k_nlfk_partial, kNlfkBlocks, kNlfkThreads, 0, N->st, P, t, yc, mode, N->part));
    }
    {
        WEC_PROF("nlfk", -1, 8.0 * 2 * kNlfkBlocks, N->st);
        WEC_CK(launch_k(k_nlfk_final, 1, kNlfkThreads, 0, N->st, (const double *)N->part, N->out));
    }
    double h[2];
    WEC_CK(cudaMemcpyAsync(h, N->out, sizeof(h), cudaMemcpyDeviceToHost, N->st));
    WEC_CK(cudaStreamSynchronize(N->st));
    *fx = h[0];
    *fy = h[1];
    return WEC_OK;
}

void wec_nlfk_destroy(wec_nlfk *N)
{
    if (!N) return;
    if (N->st) cudaStreamSynchronize(N->st);
    cudaFree(N->waves);
    cudaFree(N->part);
    cudaFree(N->out);
    delete N;
}

}  // extern "C"
