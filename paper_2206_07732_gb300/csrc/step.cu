// One time step of the two-phase wave tank on the GPU (2D, FP64).
//
// Paper (arxiv 2206.07732) passages implemented here:
//   Eq. int_fh ............ heave force as a sum over the faces where the body SDF
//                           changes sign (k_force_partial, k_heave)
//   Eq. newton_u .......... heave update, with an artificial added mass that keeps
//                           the n_cycles = 1 coupling stable (k_heave)
//   Section "Interface tracking" and "Level set advection" .. PPM advection of
//                           sigma (k_advect), Sussman reinitialisation (k_reinit),
//                           analytic body SDF psi by CSG max (psi_box)
//   Eqs. ls_flow, ls_solid, Hflow, Hbody .. materials (k_materials)
//   Eq. c_discrete_momentum .. consistent mass/momentum transport, Crank-Nicolson
//                           viscosity, flow-density gravity, implicit Brinkman term
//                           (Eq. bp_discrete) (k_mom_u, k_mom_v, k_jacobi)
//   Eq. spongelayer ....... vorticity damping over the top four cells
//   Section "Numerical wave tank" .. Airy inflow at x = 0, wave damping zone
//   Eq. c_discrete_continuity .. incremental projection (k_proj_rhs, solver, k_project)
// Layouts: cells [ny][nx], u [ny][nx+1], v [ny+1][nx]; one thread per cell/face,
// consecutive threads along x (coalesced rows).
#include <algorithm>
#include <cmath>
#include <utility>

#include "tank.cuh"

namespace wec {
namespace {

constexpr int TB = 256;

template <typename R>
__device__ __forceinline__ const TankC<R> &cst(const TankP &P)
{
    if constexpr (sizeof(R) == 4)
        return P.cf;
    else
        return P.cd;
}

__device__ __forceinline__ int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }
template <typename R>
__device__ __forceinline__ R sq(R a) { return a * a; }

// Smoothed Heaviside of Eqs. Hflow / Hbody, half-width eps = n_cells h (n_cells = 1).
template <typename R>
__device__ __forceinline__ R heav(R phi, R eps)
{
    if (phi < -eps) return R(0.0);
    if (phi > eps) return R(1.0);
    return R(0.5) * (R(1.0) + phi / eps + sin(R(kPi) * phi / eps) / R(kPi));
}

// Box SDF as the CSG intersection (max) of four half-planes.
template <typename R>
__device__ __forceinline__ R psi_box(const TankP &P, R x, R y, R yc)
{
    if (!P.has_body) return R(1.0e3);
    return fmax(fabs(x - cst<R>(P).bxc) - R(0.5) * cst<R>(P).bw, fabs(y - yc) - R(0.5) * cst<R>(P).bh);
}

__device__ double eta_at(const TankP &P, double x, double t)
{
    double e = 0.0;
    for (int c = 0; c < P.ncomp; ++c) e += P.amp[c] * cos(P.kw[c] * x - P.omega[c] * t + P.phase[c]);
    return e;
}

// Linear Airy velocity with Wheeler stretching y' = d y / (d + eta) up to the
// surface, blended to zero in the air by 1 - H(y - d - eta).
__device__ void airy_uv(const TankP &P, double x, double y, double t, double *uo, double *vo)
{
    double d = P.depth;
    double e = eta_at(P, x, t);
    double ys = y < d + e ? y : d + e;
    double yp = d * ys / (d + e);
    double blend = 1.0 - heav(y - d - e, P.h);
    double su = 0.0, sv = 0.0;
    for (int c = 0; c < P.ncomp; ++c) {
        double k = P.kw[c], w = P.omega[c];
        double ph = k * x - w * t + P.phase[c];
        double sk = sinh(k * d);
        su += P.amp[c] * w * cosh(k * yp) / sk * cos(ph);
        sv += P.amp[c] * w * sinh(k * yp) / sk * sin(ph);
    }
    *uo = blend * su;
    *vo = blend * sv;
}

// -------------------------------------------------------- ghost values ----
// sigma: left = incident wave y - d - eta(x, t) (eta precomputed per ghost column),
// right = zero gradient, bottom/top = linear extrapolation.
template <typename R, typename S>
__device__ __forceinline__ R sig_at(const TankP &P, const S *__restrict__ s,
                                         const double *__restrict__ etag, int i, int j)
{
    if (i < 0) return (j + R(0.5)) * cst<R>(P).h - cst<R>(P).depth - R(etag[-1 - i]);
    if (i > P.nx - 1) i = P.nx - 1;
    if (j < 0) return R(s[i]) + j * (R(s[P.nx + i]) - R(s[i]));
    if (j > P.ny - 1) {
        int m = j - (P.ny - 1);
        R a = R(s[(P.ny - 1) * P.nx + i]), b = R(s[(P.ny - 2) * P.nx + i]);
        return a + m * (a - b);
    }
    return R(s[j * P.nx + i]);
}

template <typename R, typename S>
__device__ __forceinline__ R u_at(const TankP &P, const S *__restrict__ u, int i, int j)
{
    return R(u[clampi(j, 0, P.ny - 1) * (P.nx + 1) + clampi(i, 0, P.nx)]);
}

// v: clamp rows; right wall free slip; left: odd reflection about v_in(y_j, t).
template <typename R, typename S>
__device__ __forceinline__ R v_at(const TankP &P, const S *__restrict__ v,
                                       const double *__restrict__ vin, int i, int j)
{
    j = clampi(j, 0, P.ny);
    if (i > P.nx - 1) i = P.nx - 1;
    if (i < 0) return R(2.0) * R(vin[j]) - R(v[j * P.nx + (-1 - i)]);
    return R(v[j * P.nx + i]);
}

template <typename R, typename S>
__device__ __forceinline__ R cell_at(const TankP &P, const S *__restrict__ a, int i, int j)
{
    return R(a[clampi(j, 0, P.ny - 1) * P.nx + clampi(i, 0, P.nx - 1)]);
}

// ----------------------------------------------------------------- PPM ----
template <typename R>
__device__ __forceinline__ R vl_slope(R am, R a0, R ap)
{
    R dl = a0 - am, dr = ap - a0;
    if (dl * dr <= R(0.0)) return R(0.0);
    R dc = R(0.5) * (ap - am);
    R m = fmin(fabs(dc), fmin(R(2.0) * fabs(dl), R(2.0) * fabs(dr)));
    return dc > R(0.0) ? m : -m;
}

// Limited Colella-Woodward edge values (left eL, right eR) of the middle cell of a[0..4].
template <typename R>
__device__ __forceinline__ void ppm_edges(const R *a, R &eL, R &eR)
{
    R dm = vl_slope<R>(a[0], a[1], a[2]);
    R d0 = vl_slope<R>(a[1], a[2], a[3]);
    R dp = vl_slope<R>(a[2], a[3], a[4]);
    eL = a[1] + R(0.5) * (a[2] - a[1]) - (d0 - dm) * (R(1.0) / R(6.0));
    eR = a[2] + R(0.5) * (a[3] - a[2]) - (dp - d0) * (R(1.0) / R(6.0));
    R c = a[2];
    if ((eR - c) * (c - eL) <= R(0.0)) {
        eL = c;
        eR = c;
    } else {
        R dA = eR - eL;
        R m6 = dA * (c - R(0.5) * (eL + eR));
        R q = dA * dA * (R(1.0) / R(6.0));
        if (m6 > q)
            eL = R(3.0) * c - R(2.0) * eR;
        else if (-q > m6)
            eR = R(3.0) * c - R(2.0) * eL;
    }
}

// Time-centred upwind face state; a[0..5] = cells f-3..f+2 around face f.
template <typename R>
__device__ __forceinline__ R ppm_face(const R *a, R vel, R dt, R ih)
{
    R eL, eR;
    if (vel >= R(0.0)) {
        ppm_edges<R>(a, eL, eR);
        R C = vel * dt * ih, dA = eR - eL, a6 = R(6.0) * (a[2] - R(0.5) * (eL + eR));
        return eR - R(0.5) * C * (dA - (R(1.0) - C * (R(2.0) / R(3.0))) * a6);
    }
    ppm_edges<R>(a + 1, eL, eR);
    R C = -vel * dt * ih, dA = eR - eL, a6 = R(6.0) * (a[3] - R(0.5) * (eL + eR));
    return eL + R(0.5) * C * (dA + (R(1.0) - C * (R(2.0) / R(3.0))) * a6);
}

// Damping-zone weight (Jacobsen) and the vorticity-damping shape (cos(pi z~) + 1),
// evaluated once per tank into tables (columns / rows) by k_tables.
__device__ __forceinline__ double damp_alpha_eval(const TankP &P, double x)
{
    if (P.damp_len <= 0.0 || x <= P.damp_x0) return 0.0;
    double xi = (x - P.damp_x0) / P.damp_len;
    if (xi > 1.0) xi = 1.0;
    return (exp(pow(xi, 3.5)) - 1.0) / (exp(1.0) - 1.0);
}

__device__ __forceinline__ double vort_shape_eval(const TankP &P, double y)
{
    double w = 4.0 * P.h;
    if (y < P.ly - w) return 0.0;
    double zt = (y - P.ly) / w;
    return cos(kPi * zt) + 1.0;
}

// g(z~) = rho_a (cos(pi z~) + 1) / (4 dt) (Eq. spongelayer) from the tabulated shape.
template <typename R>
__device__ __forceinline__ R vort_damp(const TankP &P, R shape, R idt)
{
    return cst<R>(P).rho_a * shape * (R(0.25) * idt);
}

template <typename R>
__device__ __forceinline__ R minmod(R a, R b)
{
    if (a * b <= R(0.0)) return R(0.0);
    return fabs(a) < fabs(b) ? a : b;
}

template <typename R>
__device__ __forceinline__ R koren(R quu, R qu, R qd)
{
    R d1 = qu - quu, d2 = qd - qu;
    if (d1 * d2 <= R(0.0)) return qu;
    R m = fmin(R(2.0) * fabs(d2), fmin((fabs(d1) + R(2.0) * fabs(d2)) * (R(1.0) / R(3.0)), R(2.0) * fabs(d1)));
    return d1 > R(0.0) ? qu + R(0.5) * m : qu - R(0.5) * m;
}

template <typename R>
__device__ __forceinline__ R upwind(R q0, R q1, R q2, R q3, R vel)
{
    return vel >= R(0.0) ? koren<R>(q0, q1, q2) : koren<R>(q3, q2, q1);
}

// ------------------------------------------------------------- kernels ----
template <typename R>
__device__ __forceinline__ R warp_sum_d(R v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// eta at x = 0 (for the inflow profile) and at the three ghost columns, at t^n
// and t^{n+1}: one warp per value, lanes over the wave components.
__global__ void k_bc_eta(TankP P, const StepScalars *S, const double *__restrict__ inp, Bc bc)
{
    pdl_entry();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;  // 8 warps: (time, position)
    const double t = (w & 1) ? S->t + inp[0] : S->t;
    const int pos = w >> 1;                                    // 0: x = 0; 1..3: ghost columns
    const double x = pos == 0 ? 0.0 : (-pos + 0.5) * P.h;
    double e = 0.0;
    for (int c = lane; c < P.ncomp; c += 32) e += P.amp[c] * cos(P.kw[c] * x - P.omega[c] * t + P.phase[c]);
    e = warp_sum_d(e);
    if (lane) return;
    if (pos == 0)
        bc.eta_in[w & 1] = e;
    else
        ((w & 1) ? bc.eta1 : bc.eta0)[pos - 1] = e;
}

// Inflow at x = 0: u_in(y_{j+1/2}, t^{n+1}) and v_in(y_j, t^n), v_in(y_j, t^{n+1}),
// Airy velocities with Wheeler stretching, blended to zero in the air.  One warp
// per row j, lanes over the components.
template <typename R>
__global__ void k_bc_rows(TankP P, const StepScalars *S, const double *__restrict__ inp, Bc bc)
{
    pdl_entry();
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j > P.ny) return;
    const R t0 = R(S->t), t1 = R(S->t) + R(inp[0]), d = cst<R>(P).depth;
    R out[3];
    for (int q = 0; q < 3; ++q) {
        const R t = q == 1 ? t0 : t1;
        const R y = q == 0 ? (j + R(0.5)) * cst<R>(P).h : j * cst<R>(P).h;
        const R e = R(bc.eta_in[q == 1 ? 0 : 1]);
        const R ys = y < d + e ? y : d + e;
        const R yp = d * ys / (d + e);
        R acc = R(0.0);
        for (int c = lane; c < P.ncomp; c += 32) {
            R k = R(P.kw[c]), w = R(P.omega[c]);
            R ph = -w * t + R(P.phase[c]);
            R ch, sh;  // cosh(k y') / sinh(k d) and sinh(k y') / sinh(k d)
            if constexpr (sizeof(R) == 4) {
                // overflow-free in FP32 (k d reaches ~120 for short components)
                R e1 = exp(k * (yp - d)), e2 = exp(-k * (yp + d)), den = R(1.0) - exp(R(-2.0) * k * d);
                ch = (e1 + e2) / den;
                sh = (e1 - e2) / den;
            } else {
                R sk = sinh(k * d);
                ch = cosh(k * yp) / sk;
                sh = sinh(k * yp) / sk;
            }
            if (q == 0)
                acc += R(P.amp[c]) * w * ch * cos(ph);
            else
                acc += R(P.amp[c]) * w * sh * sin(ph);
        }
        acc = warp_sum_d<R>(acc);
        out[q] = (R(1.0) - heav<R>(y - d - e, cst<R>(P).h)) * acc;
    }
    if (lane) return;
    if (j < P.ny) bc.uin1[j] = out[0];
    bc.vin0[j] = out[1];
    bc.vin1[j] = out[2];
}

// Cell materials from sigma and the body at yc (which = 0: y_c^n, 1: y_c^{n+1}).
template <typename R>
__global__ void k_materials(TankP P, const StepScalars *S, int which, const double *__restrict__ sig,
                            R *rho, R *mu, R *rhof, R *chi)
{
    pdl_entry();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.nx * P.ny) return;
    int i = c % P.nx, j = c / P.nx;
    R yc = which ? R(S->yc1) : R(S->yc);
    R ps = psi_box<R>(P, (i + R(0.5)) * cst<R>(P).h, (j + R(0.5)) * cst<R>(P).h, yc);
    R hf = heav<R>(R(sig[c]), cst<R>(P).h), hb = heav<R>(ps, cst<R>(P).h);
    R rf = cst<R>(P).rho_w + (cst<R>(P).rho_a - cst<R>(P).rho_w) * hf;
    R mf = cst<R>(P).mu_w + (cst<R>(P).mu_a - cst<R>(P).mu_w) * hf;
    if (rho) rho[c] = cst<R>(P).rho_s + (rf - cst<R>(P).rho_s) * hb;
    if (mu) mu[c] = cst<R>(P).mu_s + (mf - cst<R>(P).mu_s) * hb;
    if (rhof) rhof[c] = rf;
    if (chi) chi[c] = R(1.0) - hb;
}

__device__ double block_sum(double v, double *sh)
{
    int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
        if (t < s) sh[t] += sh[t + s];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// Eq. int_fh, heave component: faces whose two cells have opposite psi sign;
// pressure linearly interpolated to the psi = 0 crossing with |psi| weights;
// n_f out of the body; viscous traction by central differences at the face.
template <typename M>
__global__ void k_force_partial(TankP P, const StepScalars *S, const double *__restrict__ p,
                                const double *__restrict__ u, const double *__restrict__ v,
                                const M *__restrict__ mu, const double *__restrict__ vin0,
                                double *__restrict__ part)
{
    pdl_entry();
    __shared__ double sh[TB];
    const int nx = P.nx, ny = P.ny;
    const double h = P.h, yc = S->yc;
    // Only faces whose two cells straddle the box boundary contribute, and those
    // cells lie within one cell of it: walk cells i0..i1 x j0..j1, two cells
    // around the box (the same nonzero terms as a walk over every face).
    const int i0 = max(0, (int)floor((P.bxc - 0.5 * P.bw) / h) - 2);
    const int i1 = min(nx - 1, (int)ceil((P.bxc + 0.5 * P.bw) / h) + 2);
    const int j0 = max(0, (int)floor((yc - 0.5 * P.bh) / h) - 2);
    const int j1 = min(ny - 1, (int)ceil((yc + 0.5 * P.bh) / h) + 2);
    const int bi = i1 - i0 + 1, bj = j1 - j0 + 1;
    // y-faces: j in j0+1..j1, i in i0..i1; x-faces: i in i0+1..i1, j in j0..j1
    const long long ny_faces = bi > 0 && bj > 1 ? (long long)bi * (bj - 1) : 0;
    const long long nx_faces = bi > 1 && bj > 0 ? (long long)(bi - 1) * bj : 0;
    double acc = 0.0;
    if (P.has_body) {
        for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < ny_faces + nx_faces;
             k += (long long)gridDim.x * blockDim.x) {
            if (k < ny_faces) {
                int i = i0 + (int)(k % bi), j = j0 + 1 + (int)(k / bi);
                double x = (i + 0.5) * h;
                double pl = psi_box(P, x, (j - 0.5) * h, yc), pr = psi_box(P, x, (j + 0.5) * h, yc);
                if (!(pl * pr < 0.0)) continue;
                double nrm = pl < 0.0 ? 1.0 : -1.0;
                double wl = fabs(pl), wr = fabs(pr);
                double pf = (p[(j - 1) * nx + i] * wr + p[j * nx + i] * wl) / (wl + wr);
                double muf = 0.5 * (double(mu[(j - 1) * nx + i]) + double(mu[j * nx + i]));
                double dvdy = (v_at<double>(P, v, vin0, i, j + 1) - v_at<double>(P, v, vin0, i, j - 1)) / (2.0 * h);
                acc += (-pf * nrm + muf * 2.0 * dvdy * nrm) * h;
            } else {
                long long q = k - ny_faces;
                int i = i0 + 1 + (int)(q % (bi - 1)), j = j0 + (int)(q / (bi - 1));
                double y = (j + 0.5) * h;
                double pl = psi_box(P, (i - 0.5) * h, y, yc), pr = psi_box(P, (i + 0.5) * h, y, yc);
                if (!(pl * pr < 0.0)) continue;
                double nrm = pl < 0.0 ? 1.0 : -1.0;
                double muf = 0.5 * (double(mu[j * nx + i - 1]) + double(mu[j * nx + i]));
                double dvdx = 0.5 * ((v_at<double>(P, v, vin0, i, j) - v_at<double>(P, v, vin0, i - 1, j)) +
                                     (v_at<double>(P, v, vin0, i, j + 1) - v_at<double>(P, v, vin0, i - 1, j + 1))) / h;
                double dudy = (u_at<double>(P, u, i, j + 1) - u_at<double>(P, u, i, j - 1)) / (2.0 * h);
                acc += muf * (dvdx + dudy) * nrm * h;
            }
        }
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// Sum of the force partials (fixed order), then the stabilised heave update:
// (m + m_a)(zdot^{n+1} - zdot^n) = dt (F - m g + F_PTO) + m_a (zdot^n - zdot^{n-1}).
__global__ void k_heave(TankP P, StepScalars *S, const double *__restrict__ part, const double *__restrict__ inp)
{
    pdl_entry();
    const double dt = inp[0], fpto_in = inp[1];
    __shared__ double sh[TB];
    double s = 0.0;
    for (int b = threadIdx.x; b < kRedBlocks; b += blockDim.x) s += part[b];
    double F = block_sum(s, sh);
    if (threadIdx.x != 0) return;
    double fpto = fpto_in - P.pto_c * S->zdot;
    double zd1 = S->zdot, yc1 = S->yc;
    if (P.has_body) {
        double m = P.mass, ma = P.added_mass;
        zd1 = S->zdot + (dt * (F - m * P.g + fpto) + ma * (S->zdot - S->zdot_prev)) / (m + ma);
        yc1 = S->yc + 0.5 * dt * (S->zdot + zd1);
    }
    S->F = F;
    S->fpto = fpto;
    S->zdot1 = zd1;
    S->yc1 = yc1;
}

// sigma* = sigma^n - dt Q(u^n, sigma^n), then damping-zone relaxation.
template <typename R>
__global__ void k_advect(TankP P, const R *__restrict__ s, const R *__restrict__ u,
                         const R *__restrict__ v, const double *__restrict__ eta0,
                         const double *__restrict__ inp, const R *__restrict__ alpha_c,
                         double *__restrict__ out, R *__restrict__ out_w)
{
    pdl_entry();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.nx * P.ny) return;
    const R dt = R(inp[0]);
    const int nx = P.nx, i = c % nx, j = c / nx;
    const R h = cst<R>(P).h;
    R a[6], fx[2], fy[2];
    for (int f = 0; f < 2; ++f) {
        int fi = i + f;
        for (int q = 0; q < 6; ++q) a[q] = sig_at<R>(P, s, eta0, fi - 3 + q, j);
        fx[f] = ppm_face<R>(a, R(u[j * (nx + 1) + fi]), dt, cst<R>(P).ih);
        int fj = j + f;
        for (int q = 0; q < 6; ++q) a[q] = sig_at<R>(P, s, eta0, i, fj - 3 + q);
        fy[f] = ppm_face<R>(a, R(v[fj * nx + i]), dt, cst<R>(P).ih);
    }
    R ub = R(0.5) * (R(u[j * (nx + 1) + i]) + R(u[j * (nx + 1) + i + 1]));
    R vb = R(0.5) * (R(v[j * nx + i]) + R(v[(j + 1) * nx + i]));
    R Q = ub * (fx[1] - fx[0]) * cst<R>(P).ih + vb * (fy[1] - fy[0]) * cst<R>(P).ih;
    R sa = R(s[c]) - dt * Q;
    R al = alpha_c[i];
    const R r = (R(1.0) - al) * sa + al * ((j + R(0.5)) * h - cst<R>(P).depth);
    out[c] = r;
    if (out_w) out_w[c] = r;
}

// Sussman relaxation right-hand side S(sigma0)(|grad f| - 1), Godunov
// Hamiltonian on ENO-2 (minmod) one-sided differences.
template <typename R>
__device__ R reinit_rhs(const TankP &P, const R *__restrict__ f, const R *__restrict__ sgn,
                             const double *__restrict__ eta1, int i, int j)
{
    const R ih = cst<R>(P).ih, ih2 = R(0.5) * cst<R>(P).ih;
    R c = R(f[j * P.nx + i]);
    R xm2 = sig_at<R>(P, f, eta1, i - 2, j), xm1 = sig_at<R>(P, f, eta1, i - 1, j);
    R xp1 = sig_at<R>(P, f, eta1, i + 1, j), xp2 = sig_at<R>(P, f, eta1, i + 2, j);
    R ym2 = sig_at<R>(P, f, eta1, i, j - 2), ym1 = sig_at<R>(P, f, eta1, i, j - 1);
    R yp1 = sig_at<R>(P, f, eta1, i, j + 1), yp2 = sig_at<R>(P, f, eta1, i, j + 2);
    R dxm = xm2 - R(2.0) * xm1 + c, dx0 = xm1 - R(2.0) * c + xp1, dxp = c - R(2.0) * xp1 + xp2;
    R dym = ym2 - R(2.0) * ym1 + c, dy0 = ym1 - R(2.0) * c + yp1, dyp = c - R(2.0) * yp1 + yp2;
    R a = (c - xm1) * ih + minmod<R>(dxm, dx0) * ih2;
    R b = (xp1 - c) * ih - minmod<R>(dx0, dxp) * ih2;
    R cc = (c - ym1) * ih + minmod<R>(dym, dy0) * ih2;
    R d = (yp1 - c) * ih - minmod<R>(dy0, dyp) * ih2;
    R S = R(sgn[j * P.nx + i]);
    R gx, gy;
    if (S > R(0.0)) {
        gx = fmax(sq<R>(fmax(a, R(0.0))), sq<R>(fmin(b, R(0.0))));
        gy = fmax(sq<R>(fmax(cc, R(0.0))), sq<R>(fmin(d, R(0.0))));
    } else {
        gx = fmax(sq<R>(fmin(a, R(0.0))), sq<R>(fmax(b, R(0.0))));
        gy = fmax(sq<R>(fmin(cc, R(0.0))), sq<R>(fmax(d, R(0.0))));
    }
    return S * (sqrt(gx + gy) - R(1.0));
}

// Smoothed sign S(sigma0) = sigma0 / sqrt(sigma0^2 + h^2), fixed over the pseudo-steps.
template <typename R>
__global__ void k_reinit_sign(TankP P, const R *__restrict__ s0, R *__restrict__ sgn)
{
    pdl_entry();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.nx * P.ny) return;
    R g0 = s0[c];
    sgn[c] = g0 / sqrt(g0 * g0 + cst<R>(P).h * cst<R>(P).h);
}

// TVD-RK2 stage: stage 1 out = f - dtau L(f); stage 2 out = (fprev + (f - dtau L(f))) / 2.
template <typename R, typename TO>
__global__ void k_reinit(TankP P, const R *__restrict__ f, const R *__restrict__ sgn,
                         const R *__restrict__ fprev, const double *__restrict__ eta1, R dtau,
                         TO *__restrict__ out)
{
    pdl_entry();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.nx * P.ny) return;
    int i = c % P.nx, j = c / P.nx;
    R s1 = R(f[c]) - dtau * reinit_rhs<R>(P, f, sgn, eta1, i, j);
    out[c] = fprev ? R(0.5) * (R(fprev[c]) + s1) : s1;
}

// ---------------------------------------------------- momentum helpers ----
// Per-tank tables: alpha at cell centres [nx] and at u-faces [nx+1]; vorticity
// shape at cell-centre rows [ny] and at v-face rows [ny+1].
template <typename R>
struct Tabs {
    const R *alpha_c, *alpha_u, *vort_c, *vort_v;
};

// Layout of one table set: alpha_c [nx], alpha_u [nx+1], vort_c [ny], vort_v [ny+1].
// t32 (optional) receives the same tables in FP32.
__global__ void k_tables(TankP P, double *t, float *t32)
{
    pdl_entry();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = P.nx, ny = P.ny, o1 = nx, o2 = 2 * nx + 1, o3 = 2 * nx + 1 + ny;
    auto put = [&](int o, double val) {
        t[o] = val;
        if (t32) t32[o] = (float)val;
    };
    if (k < nx) put(k, damp_alpha_eval(P, (k + 0.5) * P.h));
    if (k <= nx) put(o1 + k, damp_alpha_eval(P, k * P.h));
    if (k < ny) put(o2 + k, vort_shape_eval(P, (k + 0.5) * P.h));
    if (k <= ny) put(o3 + k, vort_shape_eval(P, k * P.h));
}

template <typename R>
struct Fields {
    const R *rc;              // cell density rho^n (transport)
    const R *u, *v;           // velocities
    const double *vin;        // left tangential inflow for v ghosts
};

template <typename R>
__device__ __forceinline__ R ru_at(const TankP &P, const R *rc, int i, int j)
{
    i = clampi(i, 0, P.nx);
    j = clampi(j, 0, P.ny - 1);
    return R(0.5) * (cell_at<R>(P, rc, i - 1, j) + cell_at<R>(P, rc, i, j));
}

template <typename R>
__device__ __forceinline__ R rv_at(const TankP &P, const R *rc, int i, int j)
{
    i = clampi(i, 0, P.nx - 1);
    j = clampi(j, 0, P.ny);
    return R(0.5) * (cell_at<R>(P, rc, i, j - 1) + cell_at<R>(P, rc, i, j));
}

// Consistent transport on the u-face (i, j): rho-breve and C share the mass flux.
template <typename R>
__device__ void transport_u(const TankP &P, const Fields<R> &X, int i, int j, R dt, R &rb, R &C)
{
    R m[4], f[4];
    for (int s = 0; s < 2; ++s) {
        int a = i - 1 + s;
        R U = R(0.5) * (u_at<R>(P, X.u, a, j) + u_at<R>(P, X.u, a + 1, j));
        R r = upwind<R>(ru_at<R>(P, X.rc, a - 1, j), ru_at<R>(P, X.rc, a, j), ru_at<R>(P, X.rc, a + 1, j),
                          ru_at<R>(P, X.rc, a + 2, j), U);
        R q = upwind<R>(u_at<R>(P, X.u, a - 1, j), u_at<R>(P, X.u, a, j), u_at<R>(P, X.u, a + 1, j),
                          u_at<R>(P, X.u, a + 2, j), U);
        m[s] = U * r;
        f[s] = m[s] * q;
    }
    for (int s = 0; s < 2; ++s) {
        int b = j - 1 + s;
        R V = R(0.5) * (v_at<R>(P, X.v, X.vin, i - 1, b + 1) + v_at<R>(P, X.v, X.vin, i, b + 1));
        R r = upwind<R>(ru_at<R>(P, X.rc, i, b - 1), ru_at<R>(P, X.rc, i, b), ru_at<R>(P, X.rc, i, b + 1),
                          ru_at<R>(P, X.rc, i, b + 2), V);
        R q = upwind<R>(u_at<R>(P, X.u, i, b - 1), u_at<R>(P, X.u, i, b), u_at<R>(P, X.u, i, b + 1),
                          u_at<R>(P, X.u, i, b + 2), V);
        m[2 + s] = V * r;
        f[2 + s] = m[2 + s] * q;
    }
    rb = ru_at<R>(P, X.rc, i, j) - dt * cst<R>(P).ih * ((m[1] - m[0]) + (m[3] - m[2]));
    C = ((R(f[1]) - R(f[0])) + (R(f[3]) - R(f[2]))) * cst<R>(P).ih;
}

template <typename R>
__device__ void transport_v(const TankP &P, const Fields<R> &X, int i, int j, R dt, R &rb, R &C)
{
    R m[4], f[4];
    for (int s = 0; s < 2; ++s) {
        int a = i - 1 + s;
        R U = R(0.5) * (u_at<R>(P, X.u, a + 1, j - 1) + u_at<R>(P, X.u, a + 1, j));
        R r = upwind<R>(rv_at<R>(P, X.rc, a - 1, j), rv_at<R>(P, X.rc, a, j), rv_at<R>(P, X.rc, a + 1, j),
                          rv_at<R>(P, X.rc, a + 2, j), U);
        R q = upwind<R>(v_at<R>(P, X.v, X.vin, a - 1, j), v_at<R>(P, X.v, X.vin, a, j),
                          v_at<R>(P, X.v, X.vin, a + 1, j), v_at<R>(P, X.v, X.vin, a + 2, j), U);
        m[s] = U * r;
        f[s] = m[s] * q;
    }
    for (int s = 0; s < 2; ++s) {
        int b = j - 1 + s;
        R V = R(0.5) * (v_at<R>(P, X.v, X.vin, i, b) + v_at<R>(P, X.v, X.vin, i, b + 1));
        R r = upwind<R>(rv_at<R>(P, X.rc, i, b - 1), rv_at<R>(P, X.rc, i, b), rv_at<R>(P, X.rc, i, b + 1),
                          rv_at<R>(P, X.rc, i, b + 2), V);
        R q = upwind<R>(v_at<R>(P, X.v, X.vin, i, b - 1), v_at<R>(P, X.v, X.vin, i, b),
                          v_at<R>(P, X.v, X.vin, i, b + 1), v_at<R>(P, X.v, X.vin, i, b + 2), V);
        m[2 + s] = V * r;
        f[2 + s] = m[2 + s] * q;
    }
    rb = rv_at<R>(P, X.rc, i, j) - dt * cst<R>(P).ih * ((m[1] - m[0]) + (m[3] - m[2]));
    C = ((R(f[1]) - R(f[0])) + (R(f[3]) - R(f[2]))) * cst<R>(P).ih;
}

// L_mu u = div[mu (grad u + grad u^T)]: tau_xx / tau_yy at cells, tau_xy at
// nodes with the four-cell mean viscosity.
template <typename R>
struct Visc {
    const R *mu, *u, *v;
    const double *vin;
};

template <typename R>
__device__ __forceinline__ R mnode(const TankP &P, const Visc<R> &X, int i, int j)
{
    return R(0.25) * (cell_at<R>(P, X.mu, i - 1, j - 1) + cell_at<R>(P, X.mu, i, j - 1) + cell_at<R>(P, X.mu, i - 1, j) +
                   cell_at<R>(P, X.mu, i, j));
}

template <typename R>
__device__ __forceinline__ R txx(const TankP &P, const Visc<R> &X, int i, int j)
{
    return R(2.0) * cell_at<R>(P, X.mu, i, j) * (u_at<R>(P, X.u, i + 1, j) - u_at<R>(P, X.u, i, j)) * cst<R>(P).ih;
}

template <typename R>
__device__ __forceinline__ R tyy(const TankP &P, const Visc<R> &X, int i, int j)
{
    return R(2.0) * cell_at<R>(P, X.mu, i, j) * (v_at<R>(P, X.v, X.vin, i, j + 1) - v_at<R>(P, X.v, X.vin, i, j)) * cst<R>(P).ih;
}

template <typename R>
__device__ __forceinline__ R txy(const TankP &P, const Visc<R> &X, int i, int j)
{
    return mnode<R>(P, X, i, j) * ((u_at<R>(P, X.u, i, j) - u_at<R>(P, X.u, i, j - 1)) * cst<R>(P).ih +
                                (v_at<R>(P, X.v, X.vin, i, j) - v_at<R>(P, X.v, X.vin, i - 1, j)) * cst<R>(P).ih);
}

template <typename R>
__device__ __forceinline__ R visc_x(const TankP &P, const Visc<R> &X, int i, int j)
{
    return (txx<R>(P, X, i, j) - txx<R>(P, X, i - 1, j)) * cst<R>(P).ih + (txy<R>(P, X, i, j + 1) - txy<R>(P, X, i, j)) * cst<R>(P).ih;
}

template <typename R>
__device__ __forceinline__ R visc_y(const TankP &P, const Visc<R> &X, int i, int j)
{
    return (tyy<R>(P, X, i, j) - tyy<R>(P, X, i, j - 1)) * cst<R>(P).ih + (txy<R>(P, X, i + 1, j) - txy<R>(P, X, i, j)) * cst<R>(P).ih;
}

template <typename R>
__device__ __forceinline__ R visc_diag_x(const TankP &P, const Visc<R> &X, int i, int j)
{
    return -(R(2.0) * cell_at<R>(P, X.mu, i, j) + R(2.0) * cell_at<R>(P, X.mu, i - 1, j) + mnode<R>(P, X, i, j + 1) +
             mnode<R>(P, X, i, j)) * (cst<R>(P).ih * cst<R>(P).ih);
}

template <typename R>
__device__ __forceinline__ R visc_diag_y(const TankP &P, const Visc<R> &X, int i, int j)
{
    return -(R(2.0) * cell_at<R>(P, X.mu, i, j) + R(2.0) * cell_at<R>(P, X.mu, i, j - 1) + mnode<R>(P, X, i + 1, j) +
             mnode<R>(P, X, i, j)) * (cst<R>(P).ih * cst<R>(P).ih);
}

// Right-hand side R and diagonal D of the u-momentum system; also the first
// Jacobi iterate (u^n with the Dirichlet faces at t^{n+1}).
template <typename R>
__global__ void k_mom_u(TankP P, const StepScalars *S, const double *__restrict__ inp, Tabs<R> tb,
                        const R *__restrict__ rho_n, const R *__restrict__ mu_n, const R *__restrict__ chi_1,
                        const R *__restrict__ u, const R *__restrict__ v, const double *__restrict__ p,
                        Bc bc, R *Ru, R *Du, R *ua)
{
    pdl_entry();
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = P.nx;
    if (f >= (nx + 1) * P.ny) return;
    const R dt = R(inp[0]);
    int i = f % (nx + 1), j = f / (nx + 1);
    if (i == 0) {
        ua[f] = bc.uin1[j];
        return;
    }
    if (i == nx) {
        ua[f] = R(0.0);
        return;
    }
    ua[f] = R(u[f]);
    Fields<R> X{rho_n, u, v, bc.vin0};
    Visc<R> Vn{mu_n, u, v, bc.vin0};
    R rb, C;
    transport_u<R>(P, X, i, j, dt, rb, C);
    R chi = R(0.5) * (cell_at<R>(P, chi_1, i - 1, j) + cell_at<R>(P, chi_1, i, j));
    const R idt = R(1.0) / dt;
    Du[f] = rb * idt + chi * cst<R>(P).ikp + tb.alpha_u[i] * rb * idt + vort_damp<R>(P, tb.vort_c[j], idt);
    Ru[f] = ru_at<R>(P, rho_n, i, j) * R(u[f]) * idt - C + R(0.5) * visc_x<R>(P, Vn, i, j) -
            R(p[j * nx + i] - p[j * nx + i - 1]) * cst<R>(P).ih;
}

template <typename R>
__global__ void k_mom_v(TankP P, const StepScalars *S, const double *__restrict__ inp, Tabs<R> tb,
                        const R *__restrict__ rho_n, const R *__restrict__ mu_n, const R *__restrict__ chi_1,
                        const R *__restrict__ rf_1, const R *__restrict__ u, const R *__restrict__ v,
                        const double *__restrict__ p, Bc bc, R *Rv, R *Dv, R *va)
{
    pdl_entry();
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = P.nx, ny = P.ny;
    if (f >= nx * (ny + 1)) return;
    const R dt = R(inp[0]);
    int i = f % nx, j = f / nx;
    if (j == 0) {
        va[f] = R(0.0);
        return;
    }
    va[f] = R(v[f]);
    Fields<R> X{rho_n, u, v, bc.vin0};
    Visc<R> Vn{mu_n, u, v, bc.vin0};
    R rb, C;
    transport_v<R>(P, X, i, j, dt, rb, C);
    R chi = R(0.5) * (cell_at<R>(P, chi_1, i, j - 1) + cell_at<R>(P, chi_1, i, j));
    R rf = R(0.5) * (cell_at<R>(P, rf_1, i, j - 1) + cell_at<R>(P, rf_1, i, j));
    const R idt = R(1.0) / dt;
    Dv[f] = rb * idt + chi * cst<R>(P).ikp + tb.alpha_c[i] * rb * idt + vort_damp<R>(P, tb.vort_v[j], idt);
    R gp = j < ny ? R(p[j * nx + i] - p[(j - 1) * nx + i]) * cst<R>(P).ih : -R(2.0) * R(p[(ny - 1) * nx + i]) * cst<R>(P).ih;
    Rv[f] = rv_at<R>(P, rho_n, i, j) * R(v[f]) * idt - C + R(0.5) * visc_y<R>(P, Vn, i, j) - rf * cst<R>(P).g +
            chi * R(S->zdot1) * cst<R>(P).ikp - gp;
}

// Working buffers the stencil kernels read, in the compute type R.  An FP64 tank
// points them at its FP64 buffers (sig, u, v are the state itself); a mixed tank
// points them into its FP32 slab, where sig, u, v are mirrors refreshed at the
// start of each step.  Loading FP32 directly keeps the FP32 kernels off the FP64
// pipe, which a per-load FP64 -> FP32 conversion would otherwise saturate.
template <typename R>
struct Work {
    R *sig, *u, *v;                           // state (or its FP32 mirror)
    R *sa, *sgn, *r0, *r1, *rt;               // advected sigma, reinitialisation
    R *rho_n, *mu_n, *mu_1, *rf_1, *chi_1;    // materials
    R *Ru, *Du, *ua, *ub, *uc, *Rv, *Dv, *va, *vb, *vc;  // momentum systems, Jacobi iterates
};

// sig, u, v -> FP32 mirrors (one thread per cell / face of the largest set).
__global__ void k_mirror(long long nc, long long nu, long long nv, const double *__restrict__ sig,
                         const double *__restrict__ u, const double *__restrict__ v, float *__restrict__ sig32,
                         float *__restrict__ u32, float *__restrict__ v32)
{
    pdl_entry();
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < nc) sig32[k] = float(sig[k]);
    if (k < nu) u32[k] = float(u[k]);
    if (k < nv) v32[k] = float(v[k]);
}

// One Jacobi sweep of (D - L_mu / 2) u* = R (Crank-Nicolson implicit half),
// splitting on the interior diagonal of L_mu; Dirichlet faces are copied.
template <typename R, typename TO>
__global__ void k_jacobi(TankP P, const R *__restrict__ mu_1, const double *__restrict__ vin1,
                         const R *__restrict__ Ru, const R *__restrict__ Du,
                         const R *__restrict__ Rv, const R *__restrict__ Dv,
                         const R *__restrict__ ua, const R *__restrict__ va, TO *__restrict__ ub,
                         TO *__restrict__ vb)
{
    pdl_entry();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = P.nx, ny = P.ny;
    const int nu = (nx + 1) * ny, nv = nx * (ny + 1);
    Visc<R> Vk{mu_1, ua, va, vin1};
    if (k < nu) {
        int i = k % (nx + 1), j = k / (nx + 1);
        if (i == 0 || i == nx) {
            ub[k] = R(ua[k]);
            return;
        }
        R ld = visc_diag_x<R>(P, Vk, i, j);
        ub[k] = (R(Ru[k]) + R(0.5) * (visc_x<R>(P, Vk, i, j) - ld * R(ua[k]))) / (R(Du[k]) - R(0.5) * ld);
    } else if (k < nu + nv) {
        int f = k - nu;
        int i = f % nx, j = f / nx;
        if (j == 0) {
            vb[f] = R(va[f]);
            return;
        }
        R ld = visc_diag_y<R>(P, Vk, i, j);
        vb[f] = (R(Rv[f]) + R(0.5) * (visc_y<R>(P, Vk, i, j) - ld * R(va[f]))) / (R(Dv[f]) - R(0.5) * ld);
    }
}

// b = -h div u*, face coefficients beta = 1 / D (zero on Neumann walls).
template <typename TD>
__global__ void k_proj_rhs(TankP P, const double *__restrict__ us, const double *__restrict__ vs,
                           const TD *__restrict__ Du, const TD *__restrict__ Dv, double *rhs,
                           double *bu, double *bv)
{
    pdl_entry();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = P.nx, ny = P.ny;
    const int nc = nx * ny, nu = (nx + 1) * ny, nv = nx * (ny + 1);
    if (k < nc) {
        int i = k % nx, j = k / nx;
        rhs[k] = -P.h * (us[j * (nx + 1) + i + 1] - us[j * (nx + 1) + i] + vs[(j + 1) * nx + i] - vs[j * nx + i]);
    } else if (k < nc + nu) {
        int f = k - nc, i = f % (nx + 1);
        bu[f] = (i == 0 || i == nx) ? 0.0 : 1.0 / double(Du[f]);
    } else if (k < nc + nu + nv) {
        int f = k - nc - nu, j = f / nx;
        bv[f] = j == 0 ? 0.0 : 1.0 / double(Dv[f]);
    }
}

// u^{n+1} = u* - beta grad phi; p^{n+1/2} = p^{n-1/2} + phi.
__global__ void k_project(TankP P, const double *__restrict__ us, const double *__restrict__ vs,
                          const double *__restrict__ bu, const double *__restrict__ bv,
                          const double *__restrict__ phi, double *u, double *v, double *p)
{
    pdl_entry();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = P.nx, ny = P.ny;
    const int nc = nx * ny, nu = (nx + 1) * ny, nv = nx * (ny + 1);
    if (k < nu) {
        int i = k % (nx + 1), j = k / (nx + 1);
        double uu = us[k];
        if (i > 0 && i < nx) uu -= bu[k] * (phi[j * nx + i] - phi[j * nx + i - 1]) * P.ih;
        u[k] = uu;
    } else if (k < nu + nv) {
        int f = k - nu, i = f % nx, j = f / nx;
        double vv = vs[f];
        if (j > 0 && j < ny) vv -= bv[f] * (phi[j * nx + i] - phi[(j - 1) * nx + i]) * P.ih;
        if (j == ny) vv += 2.0 * bv[f] * phi[(ny - 1) * nx + i] * P.ih;
        v[f] = vv;
    } else if (k < nu + nv + nc) {
        int c = k - nu - nv;
        p[c] += phi[c];
    }
}

__global__ void k_div_partial(TankP P, const double *__restrict__ u, const double *__restrict__ v,
                              double *__restrict__ part)
{
    pdl_entry();
    __shared__ double sh[TB];
    const int nx = P.nx;
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nx * P.ny; c += gridDim.x * blockDim.x) {
        int i = c % nx, j = c / nx;
        acc += sq(P.h * (u[j * (nx + 1) + i + 1] - u[j * (nx + 1) + i] + v[(j + 1) * nx + i] - v[j * nx + i]));
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// Close the step: divergence norm, probe elevation, advance time and body state,
// and account the kernels a graph replay executed (fixed part + per-iteration
// and per-cycle parts of the solve).
__global__ void k_finalize(TankP P, StepScalars *S, const double *__restrict__ part,
                           const double *__restrict__ sig, const double *__restrict__ inp, const KState *ks,
                           int n_fixed, int n_body, int n_close)
{
    pdl_entry();
    __shared__ double sh[TB];
    double s = 0.0;
    for (int b = threadIdx.x; b < kRedBlocks; b += blockDim.x) s += part[b];
    double d2 = block_sum(s, sh);
    // probe: the lowest row j of the probe column with sigma_j < 0 <= sigma_{j+1}
    __shared__ int jmin;
    if (threadIdx.x == 0) jmin = P.ny;
    __syncthreads();
    const int ip = clampi((int)floor(P.probe_x / P.h), 0, P.nx - 1);
    for (int j = threadIdx.x; j + 1 < P.ny; j += blockDim.x) {
        double a = sig[j * P.nx + ip], b = sig[(j + 1) * P.nx + ip];
        if (a < 0.0 && b >= 0.0) atomicMin(&jmin, j);
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double eta = nan("");
    if (jmin < P.ny) {
        const int j = jmin;
        double a = sig[j * P.nx + ip], b = sig[(j + 1) * P.nx + ip];
        eta = (j + 0.5) * P.h + P.h * a / (a - b) - P.depth;
    }
    S->div2 = d2;
    S->eta = eta;
    S->t = S->t + inp[0];
    S->yc = S->yc1;
    S->zdot_prev = S->zdot;
    S->zdot = S->zdot1;
    S->launches = (long long)n_fixed + (long long)ks->its * n_body + (long long)ks->ncycles * n_close;
}

// Initial state: sigma = y - (d + eta(x, 0)); Airy velocities (u = 0 on the
// right wall, v = 0 on the bed).
__global__ void k_init_fields(TankP P, double *sig, double *u, double *v)
{
    pdl_entry();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = P.nx, ny = P.ny;
    const int nc = nx * ny, nu = (nx + 1) * ny, nv = nx * (ny + 1);
    const double h = P.h;
    double uu, vv;
    if (k < nc) {
        int i = k % nx, j = k / nx;
        sig[k] = (j + 0.5) * h - P.depth - eta_at(P, (i + 0.5) * h, 0.0);
    } else if (k < nc + nu) {
        int f = k - nc, i = f % (nx + 1), j = f / (nx + 1);
        airy_uv(P, i * h, (j + 0.5) * h, 0.0, &uu, &vv);
        u[f] = i == nx ? 0.0 : uu;
    } else if (k < nc + nu + nv) {
        int f = k - nc - nu, i = f % nx, j = f / nx;
        airy_uv(P, (i + 0.5) * h, j * h, 0.0, &uu, &vv);
        v[f] = j == 0 ? 0.0 : vv;
    }
}

// p^{-1/2}: discrete hydrostatic pressure of the flow density (p = 0 at the top
// face): p_{ny-1} = rho_f g h / 2, p_{j-1} = p_j + (face mean rho_f) g h.
__global__ void k_init_pressure(TankP P, const double *__restrict__ rf, double *p)
{
    pdl_entry();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = P.nx, ny = P.ny;
    if (i >= nx) return;
    double pj = 0.5 * rf[(ny - 1) * nx + i] * P.g * P.h;
    p[(ny - 1) * nx + i] = pj;
    for (int j = ny - 1; j >= 1; --j) {
        pj += 0.5 * (rf[(j - 1) * nx + i] + rf[j * nx + i]) * P.g * P.h;
        p[(j - 1) * nx + i] = pj;
    }
}

inline size_t pad64(size_t n) { return (n + 63) & ~size_t(63); }

// FP32 slab of a mixed tank: 11 cell arrays, 6 u-face and 6 v-face arrays, each
// starting on a 256-byte boundary.
size_t work_floats(size_t nc, size_t nu, size_t nv) { return 11 * pad64(nc) + 6 * pad64(nu) + 6 * pad64(nv); }

Work<double> work64(wec_tank *T)
{
    return Work<double>{T->sig, T->u, T->v, T->sa, T->sgn, T->r0, T->r1, T->rt, T->rho_n, T->mu_n, T->mu_1,
                        T->rf_1, T->chi_1, T->Ru, T->Du, T->ua, T->ub, T->uc, T->Rv, T->Dv, T->va, T->vb,
                        T->vc};
}

Work<float> work32(wec_tank *T)
{
    float *q = T->w32;
    auto take = [&q](size_t n) { float *r = q; q += pad64(n); return r; };
    Work<float> W;
    float **cells[] = {&W.sig, &W.sa, &W.sgn, &W.r0, &W.r1, &W.rt, &W.rho_n, &W.mu_n, &W.mu_1, &W.rf_1, &W.chi_1};
    for (float **c : cells) *c = take(T->nc);
    float **uf[] = {&W.u, &W.Ru, &W.Du, &W.ua, &W.ub, &W.uc};
    for (float **c : uf) *c = take(T->nu);
    float **vf[] = {&W.v, &W.Rv, &W.Dv, &W.va, &W.vb, &W.vc};
    for (float **c : vf) *c = take(T->nv);
    return W;
}

}  // namespace

int tank_alloc_and_init(wec_tank *T)
{
    const TankP &P = T->P;
    T->nc = (size_t)P.nx * P.ny;
    T->nu = (size_t)(P.nx + 1) * P.ny;
    T->nv = (size_t)P.nx * (P.ny + 1);
    size_t nc = T->nc, nu = T->nu, nv = T->nv;
    WEC_CK(cudaStreamCreateWithFlags(&T->gst, cudaStreamNonBlocking));
    WEC_CK(cudaStreamCreateWithFlags(&T->h1, cudaStreamNonBlocking));
    WEC_CK(cudaStreamCreateWithFlags(&T->h2, cudaStreamNonBlocking));
    WEC_CK(cudaEventCreateWithFlags(&T->ev_in, cudaEventDisableTiming));
    WEC_CK(cudaEventCreateWithFlags(&T->ev_out, cudaEventDisableTiming));
    WEC_CK(cudaStreamCreateWithFlags(&T->nst, cudaStreamNonBlocking));
    WEC_CK(cudaEventCreateWithFlags(&T->ev_nf, cudaEventDisableTiming));
    WEC_CK(cudaEventCreateWithFlags(&T->ev_nj, cudaEventDisableTiming));
    double **cells[] = {&T->sig, &T->sa, &T->r0, &T->r1, &T->rt, &T->p, &T->phi, &T->rhs,
                        &T->rho_n, &T->mu_n, &T->mu_1, &T->rf_1, &T->chi_1};
    for (double **q : cells) {
        WEC_CK(cudaMalloc(q, nc * 8));
        WEC_CK(cudaMemset(*q, 0, nc * 8));
    }
    double **ufaces[] = {&T->u, &T->us, &T->ua, &T->ub, &T->uc, &T->Ru, &T->Du};
    for (double **q : ufaces) {
        WEC_CK(cudaMalloc(q, nu * 8));
        WEC_CK(cudaMemset(*q, 0, nu * 8));
    }
    double **vfaces[] = {&T->v, &T->vs, &T->va, &T->vb, &T->vc, &T->Rv, &T->Dv};
    if (T->opts.precision == WEC_PREC_MIXED) {
        const size_t e = work_floats(nc, nu, nv);
        WEC_CK(cudaMalloc(&T->w32, e * 4));
        WEC_CK(cudaMemset(T->w32, 0, e * 4));
    }
    for (double **q : vfaces) {
        WEC_CK(cudaMalloc(q, nv * 8));
        WEC_CK(cudaMemset(*q, 0, nv * 8));
    }
    size_t nbc = (size_t)P.ny + 2 * (P.ny + 1) + 8;
    WEC_CK(cudaMalloc(&T->bcbuf, nbc * 8));
    T->bc.uin1 = T->bcbuf;
    T->bc.vin0 = T->bc.uin1 + P.ny;
    T->bc.vin1 = T->bc.vin0 + P.ny + 1;
    T->bc.eta0 = T->bc.vin1 + P.ny + 1;
    T->bc.eta1 = T->bc.eta0 + 3;
    T->bc.eta_in = T->bc.eta1 + 3;
    WEC_CK(cudaMalloc(&T->part, kRedBlocks * 8));
    WEC_CK(cudaMalloc(&T->tabs, (size_t)(2 * P.nx + 1 + 2 * P.ny + 1) * 8));
    if (T->opts.precision == WEC_PREC_MIXED) WEC_CK(cudaMalloc(&T->tabs32, (size_t)(2 * P.nx + 1 + 2 * P.ny + 1) * 4));
    WEC_CK(cudaMalloc(&T->sgn, nc * 8));
    {
        WEC_PROF("init", -1, 8.0 * (2 * P.nx + 2 * P.ny + 2), T->gst);
        launch_k(k_tables, nblk(std::max(P.nx, P.ny) + 1, 128), 128, 0, T->gst, P, T->tabs, T->tabs32);
    }
    WEC_CK(cudaMalloc(&T->inp, 2 * 8));
    WEC_CK(cudaMemset(T->inp, 0, 2 * 8));
    WEC_CK(cudaMalloc(&T->S, sizeof(StepScalars)));
    WEC_CK(cudaMallocHost(&T->Sh, sizeof(StepScalars)));
    *T->Sh = StepScalars{};
    // the solver runs FP32 V-cycles for both mixed modes
    const int sprec = T->opts.precision == WEC_PREC_FP64 ? WEC_PREC_FP64 : WEC_PREC_MIXED;
    if (int e = poisson_init(&T->solver, P.nx, P.ny, sprec, T->opts.restart, T->opts.mg_pre,
                             T->opts.mg_post, T->gst))
        return e;
    long long ninit = (long long)nc + nu + nv;
    WEC_PROF("init", -1, 8.0 * ninit, T->gst);
    launch_k(k_init_fields, nblk(ninit, TB), TB, 0, T->gst, P, T->sig, T->u, T->v);
    WEC_CK(cudaGetLastError());
    return WEC_OK;
}

// Called after the host filled Sh (initial body state): hydrostatic p from the initial sigma.
int tank_init_pressure(wec_tank *T)
{
    WEC_CK(cudaMemcpyAsync(T->S, T->Sh, sizeof(StepScalars), cudaMemcpyHostToDevice, T->gst));
    const TankP &P = T->P;
    {
        WEC_PROF("materials", -1, 16.0 * T->nc, T->gst);
        launch_k(k_materials<double>, nblk(T->nc, TB), TB, 0, T->gst, P, T->S, 0, T->sig, (double *)nullptr,
                 (double *)nullptr, T->rf_1, (double *)nullptr);
    }
    {
        WEC_PROF("init", -1, 16.0 * T->nc, T->gst);
        launch_k(k_init_pressure, nblk(P.nx, 128), 128, 0, T->gst, P, T->rf_1, T->p);
    }
    WEC_CK(cudaGetLastError());
    WEC_CK(cudaStreamSynchronize(T->gst));
    return WEC_OK;
}

namespace {

template <typename R>
Tabs<R> tabs(const wec_tank *T)
{
    const int nx = T->P.nx, ny = T->P.ny;
    const R *t;
    if constexpr (sizeof(R) == 4)
        t = T->tabs32;
    else
        t = T->tabs;
    return Tabs<R>{t, t + nx, t + 2 * nx + 1, t + 2 * nx + 1 + ny};
}

// Everything before the pressure solve: steps (1)-(7) of the step, stencils in
// the compute type R over the working set W.
template <typename R>
void enqueue_front_t(wec_tank *T, const Work<R> &W, cudaStream_t st)
{
    const TankP &P = T->P;
    const long long nc = T->nc, nu = T->nu, nv = T->nv;
    const double fb = 8.0, rb = sizeof(R);  // bytes of FP64 storage / of the working type
    constexpr bool f32 = sizeof(R) == 4;
    if constexpr (f32) {
        WEC_PROF("mirror", -1, (fb + rb) * (nc + nu + nv), st);
        launch_k(k_mirror, nblk(std::max(nc, std::max(nu, nv)), TB), TB, 0, st, nc, nu, nv, T->sig, T->u, T->v, W.sig,
                                                                            W.u, W.v);
    }
    // (1) inflow / ghost data at t^n and t^{n+1}
    {
        WEC_PROF("bc", -1, fb * 8.0, st);
        launch_k(k_bc_eta, 1, 256, 0, st, P, T->S, T->inp, T->bc);
    }
    {
        WEC_PROF("bc", -1, fb * (3.0 * P.ny + 2), st);
        launch_k(k_bc_rows<R>, nblk(P.ny + 1, 2), 64, 0, st, P, T->S, T->inp, T->bc);
    }
    // (2) materials at n, force from p^{n-1/2}, u^n (Eq. int_fh), heave (Eq. newton_u)
    {
        WEC_PROF("materials", -1, (fb + 2.0 * rb) * nc, st);
        launch_k(k_materials<R>, nblk(nc, TB), TB, 0, st, P, T->S, 0, T->sig, W.rho_n, W.mu_n, nullptr, nullptr);
    }
    {
        WEC_PROF("force", -1, fb * kRedBlocks, st);
        launch_k(k_force_partial<R>, kRedBlocks, TB, 0, st, P, T->S, T->p, T->u, T->v, W.mu_n, T->bc.vin0, T->part);
    }
    {
        WEC_PROF("scalar", -1, fb * kRedBlocks, st);
        launch_k(k_heave, 1, TB, 0, st, P, T->S, T->part, T->inp);
    }
    // (3) sigma advection + damping-zone relaxation, then reinitialisation; the
    // last pseudo-step writes sigma^{n+1} over sigma^n (no longer needed).
    {
        WEC_PROF("advect", -1, rb * (nc + nu + nv) + (fb + (f32 ? rb : 0.0)) * nc, st);
        launch_k(k_advect<R>, nblk(nc, TB), TB, 0, st, P, W.sig, W.u, W.v, T->bc.eta0, T->inp, tabs<R>(T).alpha_c, T->sa,
                                                 f32 ? W.sa : nullptr);
    }
    const R dtau = R(0.3 * P.h);
    const R *f = W.sa;
    R *bufs[2] = {W.r0, W.r1};
    const int nr = T->opts.n_reinit;
    if (nr > 0) {
        WEC_PROF("reinit", -1, rb * 2.0 * nc, st);
        launch_k(k_reinit_sign<R>, nblk(nc, TB), TB, 0, st, P, W.sa, W.sgn);
    }
    for (int it = 0; it < nr; ++it) {
        {
            WEC_PROF("reinit", -1, rb * 3.0 * nc, st);
            launch_k(k_reinit<R, R>, nblk(nc, TB), TB, 0, st, P, f, W.sgn, nullptr, T->bc.eta1, dtau, W.rt);
        }
        WEC_PROF("reinit", -1, rb * 3.0 * nc + (it == nr - 1 ? fb : rb) * nc, st);
        if (it == nr - 1) {
            launch_k(k_reinit<R, double>, nblk(nc, TB), TB, 0, st, P, W.rt, W.sgn, f, T->bc.eta1, dtau, T->sig);
        } else {
            R *dst = bufs[it & 1];
            launch_k(k_reinit<R, R>, nblk(nc, TB), TB, 0, st, P, W.rt, W.sgn, f, T->bc.eta1, dtau, dst);
            f = dst;
        }
    }
    if (nr == 0) cudaMemcpyAsync(T->sig, T->sa, nc * 8, cudaMemcpyDeviceToDevice, st);
    // (4) materials at n+1 (psi at the new body position)
    {
        WEC_PROF("materials", -1, (fb + 3.0 * rb) * nc, st);
        launch_k(k_materials<R>, nblk(nc, TB), TB, 0, st, P, T->S, 1, T->sig, nullptr, W.mu_1, W.rf_1, W.chi_1);
    }
    // (5) momentum right-hand side and diagonal, (6) Crank-Nicolson Jacobi sweeps
    {
        WEC_PROF("mom_u", -1, rb * (3.0 * nc + nu + nv + 2.0 * nu) + fb * (nc + nu), st);
        launch_k(k_mom_u<R>, nblk(nu, TB), TB, 0, st, P, T->S, T->inp, tabs<R>(T), W.rho_n, W.mu_n, W.chi_1, W.u, W.v, T->p,
                                                T->bc, W.Ru, W.Du, W.ua);
    }
    {
        WEC_PROF("mom_v", -1, rb * (4.0 * nc + nu + nv + 2.0 * nv) + fb * (nc + nv), st);
        launch_k(k_mom_v<R>, nblk(nv, TB), TB, 0, st, P, T->S, T->inp, tabs<R>(T), W.rho_n, W.mu_n, W.chi_1, W.rf_1, W.u,
                                                W.v, T->p, T->bc, W.Rv, W.Dv, W.va);
    }
    const R *ju = W.ua, *jv = W.va;
    R *tu[2] = {W.ub, W.uc}, *tv[2] = {W.vb, W.vc};
    const int nj = T->opts.n_jacobi;
    for (int it = 0; it < nj; ++it) {
        const bool last = it == nj - 1;
        WEC_PROF("jacobi", -1, rb * (nc + 4.0 * (nu + nv)) + fb * (nu + nv) + (last ? fb - rb : 0.0) * (nu + nv),
                 st);
        if (last) {
            launch_k(k_jacobi<R, double>, nblk(nu + nv, TB), TB, 0, st, P, W.mu_1, T->bc.vin1, W.Ru, W.Du, W.Rv, W.Dv,
                                                                  ju, jv, T->us, T->vs);
        } else {
            launch_k(k_jacobi<R, R>, nblk(nu + nv, TB), TB, 0, st, P, W.mu_1, T->bc.vin1, W.Ru, W.Du, W.Rv, W.Dv, ju,
                                                             jv, tu[it & 1], tv[it & 1]);
            ju = tu[it & 1];
            jv = tv[it & 1];
        }
    }
    // (7) pressure increment: A phi = -h div u*, beta = 1/D; phi from zero
    wec_poisson *S = &T->solver;
    {
        WEC_PROF("proj_rhs", -1, fb * (nc + 3.0 * (nu + nv)), st);
        launch_k(k_proj_rhs<R>, nblk(nc + nu + nv, TB), TB, 0, st, P, T->us, T->vs, W.Du, W.Dv, T->rhs, S->L64[0].bu,
                                                          S->L64[0].bv);
    }
    if (T->net) {
        // the guess reads the right-hand side and the level-0 coefficients only:
        // it runs on the net's stream while this one builds the hierarchy
        // (launch errors surface at the capture / the step's error check)
        cudaEventRecord(T->ev_nf, st);
        cudaStreamWaitEvent(T->nst, T->ev_nf, 0);
        net_enqueue_guess(T, T->nst);
        cudaEventRecord(T->ev_nj, T->nst);
        poisson_build(S, st);
        cudaStreamWaitEvent(st, T->ev_nj, 0);
    } else {
        poisson_build(S, st);
        cudaMemsetAsync(T->phi, 0, nc * 8, st);
    }
}

void enqueue_front(wec_tank *T, cudaStream_t st)
{
    if (T->opts.precision == WEC_PREC_MIXED)
        enqueue_front_t<float>(T, work32(T), st);
    else
        enqueue_front_t<double>(T, work64(T), st);
}

// (8) projection and the close of the step.
void enqueue_back(wec_tank *T, cudaStream_t st)
{
    const TankP &P = T->P;
    const long long nc = T->nc, nu = T->nu, nv = T->nv;
    const double fb = 8.0;
    wec_poisson *S = &T->solver;
    {
        WEC_PROF("project", -1, fb * (3.0 * nc + 3.0 * (nu + nv)), st);
        launch_k(k_project, nblk(nu + nv + nc, TB), TB, 0, st, P, T->us, T->vs, S->L64[0].bu, S->L64[0].bv, T->phi,
                                                         T->u, T->v, T->p);
    }
    {
        WEC_PROF("divergence", -1, fb * (nu + nv), st);
        launch_k(k_div_partial, kRedBlocks, TB, 0, st, P, T->u, T->v, T->part);
    }
    WEC_PROF("scalar", -1, fb * (kRedBlocks + P.ny), st);
    launch_k(k_finalize, 1, TB, 0, st, P, T->S, T->part, T->sig, T->inp, S->ks, T->n_fixed, T->n_body, T->n_close);
}

// Kernels per replay (front + the solve's opening + back once, then the
// Arnoldi-step kernels per iteration and the cycle-closing kernels per cycle),
// counted on a throwaway capture; k_finalize uses them to report launches.
int count_kernels(wec_tank *T)
{
    wec_poisson *S = &T->solver;
    cudaGraph_t tmp = nullptr;
    WEC_CK(cudaStreamBeginCapture(T->h1, cudaStreamCaptureModeThreadLocal));
    prof::begin_capture();
    enqueue_front(T, T->h1);
    enqueue_back(T, T->h1);
    long long nfb = prof::captured();
    prof::end_capture();
    WEC_CK(cudaStreamEndCapture(T->h1, &tmp));
    if (tmp) cudaGraphDestroy(tmp);
    int nbeg = 0, nb = 0, ncl = 0;
    if (int e = poisson_count_kernels(S, T->h1, &nbeg, &nb, &ncl)) return e;
    T->n_fixed = (int)nfb + nbeg;
    T->n_body = nb;
    T->n_close = ncl;
    return WEC_OK;
}

int build_graph(wec_tank *T)
{
    if (int e = count_kernels(T)) return e;
    WEC_CK(cudaStreamBeginCapture(T->gst, cudaStreamCaptureModeThreadLocal));
    int e = tank_capture_step(T, T->gst);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(T->gst, &g);
    if (e) {
        if (g) cudaGraphDestroy(g);
        return e;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture (step graph)");
    T->graph = g;
    WEC_CK(cudaGraphInstantiate(&T->exec, g, 0));
    return WEC_OK;
}

int finish_step(wec_tank *T, int status, wec_step_result *out)
{
    const StepScalars &s = *T->Sh;
    int iters = 0;
    double relres = 0.0;
    int st = solve_result(&T->solver, &iters, &relres);
    if (status == WEC_OK) status = st;
    T->stepped = true;
    T->last_iters = iters;
    T->last_relres = relres;
    if (status == WEC_OK && !(std::isfinite(s.zdot) && std::isfinite(s.F) && std::isfinite(relres)))
        status = fail(WEC_ERR_NONFINITE, "step: non-finite body state or residual");
    if (out) {
        out->t = s.t;
        out->z = s.yc - s.yc0;
        out->zdot = s.zdot;
        out->f_hydro = s.F;
        out->f_pto = s.fpto;
        out->eta_probe = s.eta;
        out->residual = relres;
        out->div_norm = sqrt(s.div2);
        out->iters = iters;
        out->status = status;
    }
    return status;
}

}  // namespace

int tank_prepare_capture(wec_tank *T) { return count_kernels(T); }

int tank_capture_step(wec_tank *T, cudaStream_t st)
{
    wec_poisson *S = &T->solver;
    S->st = st;
    prof::begin_capture();
    enqueue_front(T, st);
    int e = poisson_capture_solve(S, T->rhs, T->phi, T->opts.rtol, T->opts.max_iters, st, T->h1, T->h2);
    enqueue_back(T, st);
    cudaMemcpyAsync(T->Sh, T->S, sizeof(StepScalars), cudaMemcpyDeviceToHost, st);
    poisson_state_to_host(S, st);
    prof::end_capture();
    return e;
}

int tank_finish_step(wec_tank *T, wec_step_result *out)
{
    prof::add_launches(T->Sh->launches);
    return finish_step(T, WEC_OK, out);
}

int tank_step(wec_tank *T, double dt, double fpto, wec_step_result *out)
{
    cudaStream_t st = T->gst;
    // order after the caller's stream, and the caller's stream after this step
    WEC_CK(cudaEventRecord(T->ev_in, T->st));
    WEC_CK(cudaStreamWaitEvent(st, T->ev_in, 0));
    double in[2] = {dt, fpto};
    WEC_CK(cudaMemcpyAsync(T->inp, in, sizeof(in), cudaMemcpyHostToDevice, st));  // pageable: staged before return
    const bool graph = T->use_graph && !prof::enabled();
    int status = WEC_OK;
    if (T->net)
        if (int e = net_sync_weights(T->net)) return e;
    if (graph) {
        if (!T->exec)
            if (int e = build_graph(T)) return e;
        WEC_CK(cudaGraphLaunch(T->exec, st));
        WEC_CK(cudaStreamSynchronize(st));
        prof::add_launches(T->Sh->launches);
    } else {
        wec_poisson *S = &T->solver;
        S->st = st;
        enqueue_front(T, st);
        WEC_CK(cudaGetLastError());
        int iters = 0;
        double relres = 0.0;
        status = poisson_solve(S, T->rhs, T->phi, T->opts.rtol, T->opts.max_iters, &iters, &relres);
        if (status != WEC_OK && status != WEC_ERR_NOT_CONVERGED) return status;
        enqueue_back(T, st);
        WEC_CK(cudaGetLastError());
        WEC_CK(cudaMemcpyAsync(T->Sh, T->S, sizeof(StepScalars), cudaMemcpyDeviceToHost, st));
        WEC_CK(cudaStreamSynchronize(st));
        status = WEC_OK;
    }
    WEC_CK(cudaEventRecord(T->ev_out, st));
    WEC_CK(cudaStreamWaitEvent(T->st, T->ev_out, 0));
    return finish_step(T, status, out);
}

void tank_free(wec_tank *T)
{
    if (T->exec) cudaGraphExecDestroy(T->exec);
    if (T->graph) cudaGraphDestroy(T->graph);
    double *all[] = {T->sig, T->sa, T->r0, T->r1, T->rt, T->p, T->phi, T->rhs, T->rho_n, T->mu_n, T->mu_1,
                     T->rf_1, T->chi_1, T->u, T->us, T->ua, T->ub, T->uc, T->Ru, T->Du, T->v, T->vs,
                     T->va, T->vb, T->vc, T->Rv, T->Dv, T->bcbuf, T->part, T->waves,
                     T->tabs, T->sgn};
    for (double *q : all) cudaFree(q);
    if (T->inp_owned) cudaFree(T->inp);
    cudaFree(T->w32);
    cudaFree(T->tabs32);
    cudaFree(T->net_stats);
    cudaFree(T->S);
    if (T->Sh) cudaFreeHost(T->Sh);
    poisson_free(&T->solver);
    if (T->ev_in) cudaEventDestroy(T->ev_in);
    if (T->ev_out) cudaEventDestroy(T->ev_out);
    if (T->ev_nf) cudaEventDestroy(T->ev_nf);
    if (T->ev_nj) cudaEventDestroy(T->ev_nj);
    if (T->nst) cudaStreamDestroy(T->nst);
    if (T->h1) cudaStreamDestroy(T->h1);
    if (T->h2) cudaStreamDestroy(T->h2);
    if (T->gst) cudaStreamDestroy(T->gst);
}

}  // namespace wec
