// The three-dimensional tank (wec_tank3): one time step of the two-phase flow
// with a heaving vertical cylinder on an nx x ny x nz grid with z vertical
// (sections "Continuous equations of motion" through "Fluid-structure
// coupling", d = 3), one thread per cell or face, x fastest; the pressure
// increment is solved by a 3D wec_poisson object the tank owns (FP64, or FP32
// V-cycles for WEC_PREC_MIXED_MG and WEC_PREC_MIXED).  The stencils are FP64,
// or, for WEC_PREC_MIXED, FP32 over FP32 working copies of the FP64 state (the
// force integral, the heave update, the projection and the persistent fields
// stay FP64).  The step is the
// two-dimensional one with three velocity components: heave force (Eq. int_fh)
// and update, sigma advection + damping zone and reinitialisation, materials,
// consistent transport and the Crank-Nicolson momentum system by Jacobi
// sweeps, the pressure increment, the projection.
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
#include <algorithm>
#include <initializer_list>
#include <new>
#include <optional>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "df64.cuh"
#include "internal.cuh"

// the tank's constants in the working type of a kernel
template <typename R>
struct Tank3C {
    R h, ih, depth, rho_w, rho_a, mu_w, mu_a, rho_s, bxc, byc, br, blen;
};

struct Tank3P {
    int nx, ny, nz;
    double h, ih, depth, rho_w, rho_a, mu_w, mu_a, rho_s;
    int has_body;
    double bxc, byc, br, blen;
    int ncomp;
    int idx32;  // every face array's index fits in 32 bits (the interior stencils' indexing)
    const double *amp, *omega, *kw, *phase;  // device
    const double *damp;                       // device, [nx]: damping-zone weight of each column
    const float *dampf;                       // the same in FP32
    const wec::df64 *dampd;                   // the same as float pairs
    Tank3C<float> cf;
    Tank3C<double> cd;
    Tank3C<wec::df64> cdf;
};

// the working arrays of one precision of the step's stencils
template <typename R>
struct Work3 {
    R *sig = nullptr, *tmp = nullptr, *s0 = nullptr, *s1 = nullptr, *u = nullptr, *v = nullptr, *w = nullptr;
    R *rho = nullptr, *mu = nullptr, *rf = nullptr, *chi = nullptr, *mu1 = nullptr, *rf1 = nullptr, *chi1 = nullptr;
    R *D[3] = {}, *R3[3] = {}, *A[3] = {}, *B[3] = {};
    R *E[3] = {};        // edge viscosities (xy, xz, yz) of the viscosity the current kernels read
    R *RF[3] = {};       // face densities of rho^n at the u-, v-, w-faces
    R *Q[3] = {};        // Jacobi factor (1/2 h^-2) / (D + L / (2 h^2)) per solved face
    R *sh = nullptr, *uh[3] = {};  // n_cycles > 1: the means of levels n and n+1,k (sigma; u, v, w)
    R *bc = nullptr;     // u_in(t1) [nz], w_in(t0) [nz+1], w_in(t1) [nz+1], vorticity damping [nz], [nz+1],
                         // mean of w_in(t0) and w_in(t1) [nz+1]
    R *dampu = nullptr;  // damping weight of the u-faces [nx+1]
};

struct wec_tank3 {
    Tank3P P{};
    cudaStream_t st = nullptr;
    size_t nc = 0, nu = 0, nv = 0, nw = 0;
    double *sig = nullptr, *tmp = nullptr, *s0 = nullptr, *s1 = nullptr;
    double *u = nullptr, *v = nullptr, *w = nullptr;
    double *rho = nullptr, *mu = nullptr, *rhof = nullptr, *chi = nullptr;
    double *consts = nullptr;  // wave components and damping table
    // the step
    wec_solver_opts opts{};
    double g = 9.81, lz = 0, kappa_p = 1e-8, mass = 0, added_mass = 0, pto_c = 0, probe_x = 0;
    double t = 0, zc = 0, zc0 = 0, zdot = 0, zdot_prev = 0;
    double *p = nullptr, *phi = nullptr, *rhs = nullptr;
    double *mu1 = nullptr, *rf1 = nullptr, *chi1 = nullptr;
    double *D[3] = {}, *R[3] = {}, *A[3] = {}, *B[3] = {};  // per component u, v, w
    double *E[3] = {}, *RF[3] = {}, *Q[3] = {};             // as Work3: edge viscosities, face densities, Jacobi factors
    double *sh = nullptr, *uh[3] = {};                      // as Work3 (FP64 stencils, n_cycles > 1)
    double *uk[3] = {}, *muk = nullptr;                     // n_cycles > 1: the iterate u^{n+1,k}; its force's mu
    double *bc = nullptr;    // [nz] u_in(t1) at the cell layers; [nz+1] w_in(t0), w_in(t1) at the faces
    double *tabs = nullptr;  // damping weight of the u-faces [nx+1]; vorticity damping at cell / face heights
    double *part = nullptr;  // reduction partials
    wec_poisson *solver = nullptr;
    bool stepping = false;   // created with solver options
    Work3<float> wf;         // FP32 working copies (WEC_PREC_MIXED)
    Work3<wec::df64> wd;     // float-pair working copies (WEC_PREC_MIXED_DF)
    float *fconsts = nullptr;
    wec::df64 *dconsts = nullptr;
    std::vector<double> hwave;  // host copy of the wave components: amp, omega, k, phase
};

namespace wec {
namespace {

constexpr double kPi3 = 3.14159265358979323846;
bool g_split_momentum = true;  // wec_set_option "tank3_split_momentum"

// The stencils are templates on their working type R: double (WEC_PREC_FP64,
// WEC_PREC_MIXED_MG), float pairs (df64, about 48 significand bits, on the
// FP32 pipe: WEC_PREC_MIXED_DF) or float (WEC_PREC_MIXED), the last two over
// working copies of the FP64 state.  The FP64 pipe of this GPU runs at 1/64 of
// the FP32 rate, so a kernel reads its constants in its own type (cst3) and
// converts nothing in its inner loops; the force integral, the heave, the
// solve and the projection stay FP64.  FP64 division and square root expand into long FMA sequences:
// the kernels multiply by reciprocals formed once (1/h, 1/6, ...), which differs
// from dividing by at most an ulp.
template <typename R>
constexpr bool is_f64 = std::is_same<R, double>::value;
template <typename R>
constexpr bool is_df = std::is_same<R, df64>::value;
// v of lane + 1 of the warp (every lane taking part)
template <typename R>
__device__ __forceinline__ R shfl_down1(R v)
{
    if constexpr (is_df<R>)
        return R(__shfl_down_sync(0xffffffffu, v.hi, 1), __shfl_down_sync(0xffffffffu, v.lo, 1));
    else
        return __shfl_down_sync(0xffffffffu, v, 1);
}
// FP64 state <-> working type, the conversions on the integer pipe (df64.cuh)
template <typename R>
__device__ __forceinline__ R narrow_r(double d)
{
    if constexpr (is_f64<R>) return d; else if constexpr (is_df<R>) return from_double(d); else return d2f_rn(d);
}
template <typename R>
__device__ __forceinline__ double widen_r(R a)
{
    if constexpr (is_f64<R>) return a; else if constexpr (is_df<R>) return to_double(a); else return f2d_exact(a);
}
// k x for k a power of two (2 or 1/2 here): exact; for a float pair, both
// floats scaled (the value of the full pair product, in two multiplications)
template <typename R>
__device__ __forceinline__ R scl2(float k, R x)
{
    if constexpr (is_df<R>) return R(k * x.hi, k * x.lo); else return R(k) * x;
}

template <typename R>
__device__ __forceinline__ const Tank3C<R> &cst3(const Tank3P &P)
{
    if constexpr (is_f64<R>) return P.cd; else if constexpr (is_df<R>) return P.cdf; else return P.cf;
}

template <typename R>
__device__ __forceinline__ R dampc(const Tank3P &P, int i)
{
    if constexpr (is_f64<R>) return P.damp[i]; else if constexpr (is_df<R>) return P.dampd[i]; else return P.dampf[i];
}

template <typename R>
__device__ __forceinline__ R heav3(R phi, R eps, R ieps)
{
    if (phi < -eps) return R(0);
    if (phi > eps) return R(1);
    const R r = phi * ieps;
    return scl2<R>(0.5f, R(1) + r + sin(R(kPi3) * r) * R(1.0 / kPi3));
}

// The incident surface at the three ghost columns x = -(m + 1/2) h, m = 0, 1, 2,
// at the time of a call (eta of the wave components, summed on the host): the
// inflow ghost of sigma.  Summing the components per ghost read on the GPU ran
// 128 FP64 cosines in the first warp of every row, which serialised those
// warps on the FP64 pipe and dominated the level-set kernels.
struct Ghost3 {
    double e[3];
};

// sigma at (i, j, k), with the ghosts of the header (the inflow ghost in FP64)
template <typename R>
__device__ __forceinline__ R sig3(const Tank3P &P, const R *__restrict__ s, int i, int j, int k, const Ghost3 &G)
{
    if (i < 0) return narrow_r<R>((k + 0.5) * P.h - P.depth - G.e[-1 - i]);
    i = min(i, P.nx - 1);
    j = min(max(j, 0), P.ny - 1);
    const long long col = (long long)j * P.nx + i, pl = (long long)P.nx * P.ny;
    if (k < 0) return s[col] + R(k) * (s[pl + col] - s[col]);
    if (k > P.nz - 1) {
        const R a = s[(P.nz - 1) * pl + col], b = s[(P.nz - 2) * pl + col];
        return a + R(k - (P.nz - 1)) * (a - b);
    }
    return s[k * pl + col];
}

// Sign and magnitude decisions of the FP64 stencils on the integer pipe: for
// finite doubles the bit pattern orders magnitudes (sign bit shifted out) and
// carries the sign, and this GPU issues FP64 compares, min / max and products
// at 1/64 of its FP32 rate.  The FP32 stencils keep plain float compares.
__device__ __forceinline__ unsigned long long mag_bits(double a)
{
    return (unsigned long long)__double_as_longlong(a) << 1;
}
// a * b <= 0 (opposite signs, or a zero factor)
template <typename R>
__device__ __forceinline__ bool nonpos_prod(R a, R b)
{
    if constexpr (is_f64<R>) {
        const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
        return (ia ^ ib) < 0 || (ia << 1) == 0 || (ib << 1) == 0;
    } else if constexpr (is_df<R>) {  // the signs of the leading floats
        return (a.hi < 0.f) != (b.hi < 0.f) || a.hi == 0.f || b.hi == 0.f;
    } else {
        return a * b <= R(0);
    }
}
// |a| < |b|
template <typename R>
__device__ __forceinline__ bool abs_lt(R a, R b)
{
    if constexpr (is_f64<R>) return mag_bits(a) < mag_bits(b); else return fabs(a) < fabs(b);
}
// a > 0
template <typename R>
__device__ __forceinline__ bool positive(R a)
{
    if constexpr (is_f64<R>) return __double_as_longlong(a) > 0; else return a > R(0);
}

// van Leer slope of the middle cell: 0 at an extremum, else the smallest of
// |dc|, 2|dl|, 2|dr| with the sign of dc (the magnitude choice and the sign on
// the integer pipe in FP64)
template <typename R>
__device__ __forceinline__ R vl3(R am, R a0, R ap)
{
    const R dl = a0 - am, dr = ap - a0;
    if (nonpos_prod(dl, dr)) return R(0);
    const R dc = scl2<R>(0.5f, ap - am), tl = scl2<R>(2.f, dl), tr = scl2<R>(2.f, dr);
    if constexpr (is_f64<R>) {
        unsigned long long m = mag_bits(dc);
        const unsigned long long ml = mag_bits(tl), mr = mag_bits(tr);
        m = ml < m ? ml : m;
        m = mr < m ? mr : m;
        // |result| = the smallest magnitude, sign of dc
        const unsigned long long sgn = (unsigned long long)__double_as_longlong(dc) & 0x8000000000000000ull;
        return __longlong_as_double((long long)((m >> 1) | sgn));
    } else {
        const R m = fmin(fabs(dc), fmin(fabs(tl), fabs(tr)));
        return dc > R(0) ? m : -m;
    }
}

// a > b for b >= 0 (FP64 on the integer pipe: the signed bit patterns order
// a against a non-negative b)
template <typename R>
__device__ __forceinline__ bool gt_nonneg(R a, R b)
{
    if constexpr (is_f64<R>) return __double_as_longlong(a) > __double_as_longlong(b); else return a > b;
}

// limited PPM edge values (eL, eR) of the middle cell of a[0..4]
template <typename R>
__device__ __forceinline__ void ppm_edges3(const R *a, R &eL, R &eR)
{
    const R i6 = R(1.0 / 6.0);
    const R dm = vl3(a[0], a[1], a[2]), d0 = vl3(a[1], a[2], a[3]), dp = vl3(a[2], a[3], a[4]);
    R L = a[1] + scl2<R>(0.5f, a[2] - a[1]) - (d0 - dm) * i6;
    R Rr = a[2] + scl2<R>(0.5f, a[3] - a[2]) - (dp - d0) * i6;
    const R c = a[2];
    if (nonpos_prod(Rr - c, c - L)) {
        L = c;
        Rr = c;
    } else {
        const R dA = Rr - L, m6 = dA * (c - scl2<R>(0.5f, L + Rr)), q = dA * dA * i6;
        if (gt_nonneg(m6, q))
            L = R(3) * c - scl2<R>(2.f, Rr);
        else if (gt_nonneg(-m6, q))
            Rr = R(3) * c - scl2<R>(2.f, L);
    }
    eL = L;
    eR = Rr;
}

// time-centred upwind state at the face between a[2] and a[3] (a: cells f-3 .. f+2);
// dtih = dt / h.  The upwind cell's five-cell window is selected first and its
// parabola built once: vel >= 0 takes the right edge of a[2]'s parabola,
// Rr - C/2 (dA - (1 - 2C/3) a6), vel < 0 the left edge of a[3]'s, L + C/2 (dA +
// (1 - 2C/3) a6), with C = |vel| dt / h -- one copy of the edge code and no
// divergence between the two cases.
template <typename R>
__device__ __forceinline__ R ppm_face3(const R *a, R vel, R dtih)
{
    const R t3 = R(2.0 / 3.0);
    bool up;
    if constexpr (is_f64<R>)  // vel >= 0, -0 included
        up = __double_as_longlong(vel) >= 0 || (__double_as_longlong(vel) << 1) == 0;
    else
        up = vel >= R(0);
    R b[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) b[m] = up ? a[m] : a[m + 1];
    R L, Rr;
    ppm_edges3(b, L, Rr);
    const R C = (up ? vel : -vel) * dtih, dA = Rr - L, a6 = R(6) * (b[2] - scl2<R>(0.5f, L + Rr));
    const R e = (R(1) - C * t3) * a6, hc = scl2<R>(0.5f, C);
    return (up ? Rr : L) + (up ? -hc : hc) * (dA + (up ? -e : e));
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

// (cell layers k0 + blockIdx.z)
template <typename R>
__global__ void __launch_bounds__(128) k3t_materials(Tank3P P, const R *__restrict__ sig, R zc,
                                                     R *__restrict__ rho, R *__restrict__ mu, R *__restrict__ rhof,
                                                     R *__restrict__ chi, int k0, int i0, int j0)
{
    pdl_entry();
    // (the grid covers cells from (i0, j0, k0) on: a box, or the whole grid)
    Cell3 q;
    q.i = i0 + blockIdx.x * blockDim.x + threadIdx.x;
    q.j = j0 + blockIdx.y;
    q.k = k0 + blockIdx.z;
    if (q.i >= P.nx || q.j >= P.ny) return;
    q.c = ((long long)q.k * P.ny + q.j) * P.nx + q.i;
    const Tank3C<R> &K = cst3<R>(P);
    const R h = K.h;
    R psi = R(1.0e3);
    if (P.has_body) {
        const R x = (R(q.i) + R(0.5)) * h - K.bxc, y = (R(q.j) + R(0.5)) * h - K.byc,
                z = (R(q.k) + R(0.5)) * h - zc;
        psi = fmax(sqrt(x * x + y * y) - K.br, fabs(z) - scl2<R>(0.5f, K.blen));
    }
    const R hf = heav3<R>(sig[q.c], h, K.ih), hb = heav3<R>(psi, h, K.ih);
    const R rf = K.rho_w + (K.rho_a - K.rho_w) * hf;
    const R mf = K.mu_w + (K.mu_a - K.mu_w) * hf;
    rho[q.c] = K.rho_s + (rf - K.rho_s) * hb;
    mu[q.c] = K.mu_w + (mf - K.mu_w) * hb;
    rhof[q.c] = rf;
    chi[q.c] = R(1) - hb;
}

// The PPM value of s on every face of direction D (x, y, z = 0, 1, 2), upwind by
// the face velocity: a face value depends on the face alone -- the six cells
// along D around it and its velocity -- so it is formed once and read by the two
// cells beside it (k3t_advect) instead of once by each.  One 128-thread row per
// face row (gridf); F and vel in the face layout of component D.
// (x: the grid covers nx faces per row, the thread of face 0 forming the last
// one, nx, as well -- an extra block per row would hold one face)
template <int D, typename R>
__global__ void __launch_bounds__(128) k3t_ppm_faces(Tank3P P, const R *__restrict__ s, const R *__restrict__ vel,
                                                     R dt, Ghost3 G, R *__restrict__ F)
{
    pdl_entry();
    const int nx = P.nx, ny = P.ny, nz = P.nz, nxf = nx + (D == 0), nyf = ny + (D == 1);
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i0 >= nx) return;
    const Tank3C<R> &K = cst3<R>(P);
    const R dtih = dt * K.ih;
    // the face lies below cell (i, j, k) along D; its stencil is the cells -3 .. 2
    // from that cell along D, at fixed offsets (32-bit indices) when all six are
    // inside, else through sig3 (ghost cells)
    constexpr int di = D == 0, dj = D == 1, dk = D == 2;
    const int sd = D == 0 ? 1 : D == 1 ? nx : nx * ny;
    auto face = [&](int i) {
        const long long f = ((long long)k * nyf + j) * nxf + i;
        const int cd = D == 0 ? i : D == 1 ? j : k, nd = D == 0 ? nx : D == 1 ? ny : nz;
        R a[6];
        if (cd >= 3 && cd + 2 < nd) {
            const int c32 = (k * ny + j) * nx + i;
#pragma unroll
            for (int m = 0; m < 6; ++m) a[m] = s[c32 + (m - 3) * sd];
        } else {
#pragma unroll
            for (int m = 0; m < 6; ++m) a[m] = sig3<R>(P, s, i + (m - 3) * di, j + (m - 3) * dj, k + (m - 3) * dk, G);
        }
        F[f] = ppm_face3<R>(a, vel[f], dtih);
    };
    face(i0);
    if (D == 0 && i0 == 0) face(nx);
}

// out = base - dt Q(u, s), then the damping-zone blend (base = s for the plain
// update; a fixed-point cycle k >= 1 passes sigma^n as base and the means of
// levels n and n+1,k as s and u).  Q = sum over the directions of the cell
// velocity (the mean of its two faces') times the difference of the upper and
// lower face values of s (k3t_ppm_faces: Fx, Fy, Fz) over h.
template <typename R>
__global__ void __launch_bounds__(128) k3t_advect(Tank3P P, const R *__restrict__ base, const R *__restrict__ Fx,
                                                  const R *__restrict__ Fy, const R *__restrict__ Fz,
                                                  const R *__restrict__ u, const R *__restrict__ v,
                                                  const R *__restrict__ w, R dt, R *__restrict__ out)
{
    pdl_entry();
    Cell3 q;
    if (!cell_of(P, q)) return;
    const Tank3C<R> &K = cst3<R>(P);
    const int nx = P.nx, ny = P.ny, i = q.i, j = q.j, k = q.k;
    const long long r = (long long)k * ny + j, fu = r * (nx + 1) + i, fv = ((long long)k * (ny + 1) + j) * nx + i;
    const long long pl = (long long)nx * ny;
    const R ih = K.ih;
    R Q = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const long long o = d == 0 ? fu : d == 1 ? fv : q.c;  // the cell's lower face along d
        const R *vel = (d == 0 ? u : d == 1 ? v : w) + o;
        const R *Fd = (d == 0 ? Fx : d == 1 ? Fy : Fz) + o;
        const long long vs = d == 0 ? 1 : d == 1 ? nx : pl;  // face stride along d
        const R vb = scl2<R>(0.5f, vel[0] + vel[vs]);
        Q = Q + vb * (Fd[vs] - Fd[0]) * ih;
    }
    const R sa = base[q.c] - dt * Q;
    const R al = dampc<R>(P, i);
    out[q.c] = (R(1) - al) * sa + al * ((R(k) + R(0.5)) * K.h - K.depth);
}

template <typename R>
__device__ __forceinline__ R mm3(R a, R b)
{
    if (nonpos_prod(a, b)) return R(0);
    return abs_lt(a, b) ? a : b;
}

// S(sigma0) (|grad f| - 1) at a cell; S = sigma0 / sqrt(sigma0^2 + h^2), formed
// once per reinitialisation (k3t_reinit_sign).  The one-sided ENO-2 slopes are
// taken in units of 1/h (a_h = h a) and the Godunov Hamiltonian's squares
// summed before the single scaling by 1/h^2; max(max(a, 0)^2, min(b, 0)^2) for
// S > 0 (mirrored for S <= 0) is the square of the largest of a, -b and 0.
template <typename R>
__device__ __forceinline__ R reinit_rhs3(const Tank3P &P, const R *__restrict__ f, const R *__restrict__ sg,
                                         const Cell3 &q, const Ghost3 &G)
{
    const Tank3C<R> &K = cst3<R>(P);
    const R c = f[q.c];
    const R S = sg[q.c];
    const bool pos = positive(S);
    // cells two or more from every boundary read their neighbours at fixed
    // offsets (no ghosts, 32-bit indices); the others through sig3
    const bool inner = q.i >= 2 && q.i < P.nx - 2 && q.j >= 2 && q.j < P.ny - 2 && q.k >= 2 && q.k < P.nz - 2;
    const int c32 = (int)q.c, st3[3] = {1, P.nx, P.nx * P.ny};
    R g2 = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int di = d == 0, dj = d == 1, dk = d == 2;
        R m2, m1, p1, p2;
        if (inner) {
            const int o = st3[d];
            m2 = f[c32 - 2 * o];
            m1 = f[c32 - o];
            p1 = f[c32 + o];
            p2 = f[c32 + 2 * o];
        } else {
            m2 = sig3<R>(P, f, q.i - 2 * di, q.j - 2 * dj, q.k - 2 * dk, G);
            m1 = sig3<R>(P, f, q.i - di, q.j - dj, q.k - dk, G);
            p1 = sig3<R>(P, f, q.i + di, q.j + dj, q.k + dk, G);
            p2 = sig3<R>(P, f, q.i + 2 * di, q.j + 2 * dj, q.k + 2 * dk, G);
        }
        R a, nb;  // nb = -b
        if constexpr (is_df<R>) {
            // float pairs: the second differences from the four first differences
            // (seven pair subtractions instead of nine operations and two
            // scalings; the same values to the pairs' rounding)
            const R em = m1 - m2, e0 = c - m1, e1 = p1 - c, ep = p2 - p1;
            const R dm = e0 - em, d0 = e1 - e0, dp = ep - e1;
            a = e0 + scl2<R>(0.5f, mm3(dm, d0));
            nb = scl2<R>(0.5f, mm3(d0, dp)) - e1;
        } else {
            const R dm = m2 - scl2<R>(2.f, m1) + c, d0 = m1 - scl2<R>(2.f, c) + p1, dp = c - scl2<R>(2.f, p1) + p2;
            a = (c - m1) + scl2<R>(0.5f, mm3(dm, d0));
            nb = (c - p1) + scl2<R>(0.5f, mm3(d0, dp));
        }
        // pos: the largest of a, -b and 0; else of -a, b and 0
        const R x = pos ? a : -a, y = pos ? nb : -nb;
        R m = positive(x) ? x : R(0);
        bool ybig;
        if constexpr (is_f64<R>)
            ybig = positive(y) && mag_bits(y) > mag_bits(m);
        else
            ybig = y > m;
        if (ybig) m = y;
        g2 += m * m;
    }
    return S * (sqrt(g2 * K.ih * K.ih) - R(1));
}

// S(sigma0) = sigma0 / sqrt(sigma0^2 + h^2) of the field s into s0
template <typename R>
__global__ void __launch_bounds__(128) k3t_reinit_sign(Tank3P P, const R *__restrict__ s, R *__restrict__ s0)
{
    pdl_entry();
    Cell3 q;
    if (!cell_of(P, q)) return;
    const R h = cst3<R>(P).h, g = s[q.c];
    s0[q.c] = g * rsqrt(g * g + h * h);
}

// stage 1: out = f - dtau L(f); stage 2: out = (out + (f - dtau L(f))) / 2 with
// out holding sigma at the start of the pseudo-step
template <typename R>
__global__ void __launch_bounds__(128) k3t_reinit_stage(Tank3P P, const R *__restrict__ f, const R *__restrict__ sg,
                                                        R *out, Ghost3 G, R dtau, int stage)
{
    pdl_entry();
    Cell3 q;
    if (!cell_of(P, q)) return;
    const R y = f[q.c] - dtau * reinit_rhs3<R>(P, f, sg, q, G);
    out[q.c] = stage == 1 ? y : scl2<R>(0.5f, out[q.c] + y);
}

// ------------------------------------------------------------ the step ----
// Velocity ghosts: nearest face (free slip); at the inflow v is reflected oddly
// about 0 and w about the incident wave's w_in (win: [nz+1] at the time used).
template <bool IN, typename R>
__device__ __forceinline__ R cellq(const Tank3P &P, const R *__restrict__ a, int i, int j, int k)
{
    if constexpr (IN) return a[(k * P.ny + j) * P.nx + i];
    i = min(max(i, 0), P.nx - 1);
    j = min(max(j, 0), P.ny - 1);
    k = min(max(k, 0), P.nz - 1);
    return a[((long long)k * P.ny + j) * P.nx + i];
}
template <bool IN, typename R>
__device__ __forceinline__ R uq(const Tank3P &P, const R *__restrict__ u, int i, int j, int k)
{
    if constexpr (IN) return u[(k * P.ny + j) * (P.nx + 1) + i];
    i = min(max(i, 0), P.nx);
    j = min(max(j, 0), P.ny - 1);
    k = min(max(k, 0), P.nz - 1);
    return u[((long long)k * P.ny + j) * (P.nx + 1) + i];
}
template <bool IN, typename R>
__device__ __forceinline__ R vq(const Tank3P &P, const R *__restrict__ v, int i, int j, int k)
{
    if constexpr (IN) return v[(k * (P.ny + 1) + j) * P.nx + i];
    j = min(max(j, 0), P.ny);
    k = min(max(k, 0), P.nz - 1);
    if (i > P.nx - 1) i = P.nx - 1;
    if (i < 0) return -v[((long long)k * (P.ny + 1) + j) * P.nx + (-1 - i)];
    return v[((long long)k * (P.ny + 1) + j) * P.nx + i];
}
template <bool IN, typename R>
__device__ __forceinline__ R wq(const Tank3P &P, const R *__restrict__ w, const R *__restrict__ win, int i, int j,
                                int k)
{
    if constexpr (IN) return w[(k * P.ny + j) * P.nx + i];
    k = min(max(k, 0), P.nz);
    j = min(max(j, 0), P.ny - 1);
    if (i > P.nx - 1) i = P.nx - 1;
    if (i < 0) return scl2<R>(2.f, win[k]) - w[((long long)k * P.ny + j) * P.nx + (-1 - i)];
    return w[((long long)k * P.ny + j) * P.nx + i];
}

// Koren-limited upwind face value: qu at an extremum, else qu + m/2 with m the
// smallest of 2|d2|, (|d1| + 2|d2|)/3, 2|d1| carrying the sign of d1 (FP64: the
// choice and the sign on the integer pipe)
template <typename R>
__device__ __forceinline__ R koren3(R quu, R qu, R qd)
{
    const R d1 = qu - quu, d2 = qd - qu;
    if (nonpos_prod(d1, d2)) return qu;
    if constexpr (is_f64<R>) {
        const R t2 = scl2<R>(2.f, d2), t1 = scl2<R>(2.f, d1), tm = (fabs(d1) + fabs(t2)) * R(1.0 / 3.0);
        unsigned long long m = mag_bits(t2);
        const unsigned long long mm = mag_bits(tm), m1 = mag_bits(t1);
        m = mm < m ? mm : m;
        m = m1 < m ? m1 : m;
        const unsigned long long sgn = (unsigned long long)__double_as_longlong(d1) & 0x8000000000000000ull;
        return qu + scl2<R>(0.5f, __longlong_as_double((long long)((m >> 1) | sgn)));
    } else {
        const R m = fmin(scl2<R>(2.f, fabs(d2)), fmin((fabs(d1) + scl2<R>(2.f, fabs(d2))) * R(1.0 / 3.0), scl2<R>(2.f, fabs(d1))));
        return d1 > R(0) ? qu + scl2<R>(0.5f, m) : qu - scl2<R>(0.5f, m);
    }
}
template <typename R>
__device__ __forceinline__ R upw3(R q0, R q1, R q2, R q3, R vel)
{
    bool up;
    if constexpr (is_f64<R>)  // vel >= 0, -0 included
        up = __double_as_longlong(vel) >= 0 || (__double_as_longlong(vel) << 1) == 0;
    else
        up = vel >= R(0);
    // the upwind triple selected first: one copy of the limiter, no divergence
    return koren3(up ? q0 : q3, up ? q1 : q2, up ? q2 : q1);
}
// face densities: the mean of the face's two cells (face index clamped first)
template <bool IN, typename R>
__device__ __forceinline__ R ruq(const Tank3P &P, const R *rc, int i, int j, int k)
{
    if constexpr (!IN) {
        i = min(max(i, 0), P.nx);
        j = min(max(j, 0), P.ny - 1);
        k = min(max(k, 0), P.nz - 1);
    }
    return scl2<R>(0.5f, cellq<IN>(P, rc, i - 1, j, k) + cellq<IN>(P, rc, i, j, k));
}
template <bool IN, typename R>
__device__ __forceinline__ R rvq(const Tank3P &P, const R *rc, int i, int j, int k)
{
    if constexpr (!IN) {
        i = min(max(i, 0), P.nx - 1);
        j = min(max(j, 0), P.ny);
        k = min(max(k, 0), P.nz - 1);
    }
    return scl2<R>(0.5f, cellq<IN>(P, rc, i, j - 1, k) + cellq<IN>(P, rc, i, j, k));
}
template <bool IN, typename R>
__device__ __forceinline__ R rwq(const Tank3P &P, const R *rc, int i, int j, int k)
{
    if constexpr (!IN) {
        i = min(max(i, 0), P.nx - 1);
        j = min(max(j, 0), P.ny - 1);
        k = min(max(k, 0), P.nz);
    }
    return scl2<R>(0.5f, cellq<IN>(P, rc, i, j, k - 1) + cellq<IN>(P, rc, i, j, k));
}

template <typename R>
struct Vel3 {
    const R *u, *v, *w, *win;
};

// Face density arrays of rho^n (the mean of the face's two cells, ruq / rvq /
// rwq), read at the face index clamped as those accessors clamp it: the same
// values, formed once per step instead of at every read.
template <bool IN, typename R>
__device__ __forceinline__ R frq(const Tank3P &P, const R *__restrict__ a, int comp, int i, int j, int k)
{
    const int nx = P.nx, ny = P.ny;
    if constexpr (IN) {
        if (comp == 0) return a[(k * ny + j) * (nx + 1) + i];
        if (comp == 1) return a[(k * (ny + 1) + j) * nx + i];
        return a[(k * ny + j) * nx + i];
    }
    if (comp == 0) {
        i = min(max(i, 0), nx);
        j = min(max(j, 0), ny - 1);
        k = min(max(k, 0), P.nz - 1);
        return a[((long long)k * ny + j) * (nx + 1) + i];
    }
    if (comp == 1) {
        i = min(max(i, 0), nx - 1);
        j = min(max(j, 0), ny);
        k = min(max(k, 0), P.nz - 1);
        return a[((long long)k * (ny + 1) + j) * nx + i];
    }
    i = min(max(i, 0), nx - 1);
    j = min(max(j, 0), ny - 1);
    k = min(max(k, 0), P.nz);
    return a[((long long)k * ny + j) * nx + i];
}

// One face of a momentum control volume -- direction d, side s (0 lower, 1
// upper) -- of comp's CV at face (i, j, k): its mass flux m = U r and momentum
// flux f = m q, with U the d-velocity at the CV face and r, q the upwind values of
// the face density and the velocity.  A CV face is shared by the two CVs beside
// it along d and depends on it alone: side 1 of (i, j, k) is side 0 of the next
// CV along d, the same values.
template <bool IN, typename R>
__device__ __forceinline__ void tface(const Tank3P &P, const R *__restrict__ rfc, const Vel3<R> &V, int comp, int i,
                                      int j, int k, int d, int s, R &m, R &f)
{
#define QV(a, b, c) (comp == 0 ? uq<IN>(P, V.u, a, b, c) : comp == 1 ? vq<IN>(P, V.v, a, b, c) : wq<IN>(P, V.w, V.win, a, b, c))
    R U;
    if (d == comp) {  // CV faces at the cell centres on either side
        const int o = s - 1;
        U = comp == 0   ? scl2<R>(0.5f, uq<IN>(P, V.u, i + o, j, k) + uq<IN>(P, V.u, i + o + 1, j, k))
            : comp == 1 ? scl2<R>(0.5f, vq<IN>(P, V.v, i, j + o, k) + vq<IN>(P, V.v, i, j + o + 1, k))
                        : scl2<R>(0.5f, wq<IN>(P, V.w, V.win, i, j, k + o) + wq<IN>(P, V.w, V.win, i, j, k + o + 1));
    } else {  // CV faces on the edges: the d-velocity averaged over the comp direction
        const int e = s;
        if (d == 0)
            U = comp == 1 ? scl2<R>(0.5f, uq<IN>(P, V.u, i + e, j - 1, k) + uq<IN>(P, V.u, i + e, j, k))
                          : scl2<R>(0.5f, uq<IN>(P, V.u, i + e, j, k - 1) + uq<IN>(P, V.u, i + e, j, k));
        else if (d == 1)
            U = comp == 0 ? scl2<R>(0.5f, vq<IN>(P, V.v, i - 1, j + e, k) + vq<IN>(P, V.v, i, j + e, k))
                          : scl2<R>(0.5f, vq<IN>(P, V.v, i, j + e, k - 1) + vq<IN>(P, V.v, i, j + e, k));
        else
            U = comp == 0 ? scl2<R>(0.5f, wq<IN>(P, V.w, V.win, i - 1, j, k + e) + wq<IN>(P, V.w, V.win, i, j, k + e))
                          : scl2<R>(0.5f, wq<IN>(P, V.w, V.win, i, j - 1, k + e) + wq<IN>(P, V.w, V.win, i, j, k + e));
    }
    const int a0 = s - 1;  // the stencil runs over (base + a0 - 1 .. base + a0 + 2) along d
    const int di = d == 0, dj = d == 1, dk = d == 2;
    R rr[4], qq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int o = a0 - 1 + q;
        rr[q] = frq<IN>(P, rfc, comp, i + o * di, j + o * dj, k + o * dk);
        qq[q] = QV(i + o * di, j + o * dj, k + o * dk);
    }
    const R r = upw3(rr[0], rr[1], rr[2], rr[3], U);
    const R qv = upw3(qq[0], qq[1], qq[2], qq[3], U);
    m = U * r;
    f = m * qv;
#undef QV
}

// rho-breve and C of a momentum control volume: comp 0 u-face, 1 v-face, 2 w-face;
// the three pairs of CV faces summed x, then y, then z.  rfc: the face
// densities of component comp; dtih = dt / h.
template <bool IN, typename R>
__device__ __forceinline__ void transport3(const Tank3P &P, const R *__restrict__ rfc, const Vel3<R> &V, int comp,
                                           int i, int j, int k, R dtih, R &rb, R &C)
{
    const R ih = cst3<R>(P).ih;
    R m[6], f[6];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int s = 0; s < 2; ++s) tface<IN, R>(P, rfc, V, comp, i, j, k, d, s, m[2 * d + s], f[2 * d + s]);
    rb = frq<IN>(P, rfc, comp, i, j, k) - dtih * (((m[1] - m[0]) + (m[3] - m[2])) + (m[5] - m[4]));
    C = (((f[1] - f[0]) + (f[3] - f[2])) + (f[5] - f[4])) * ih;
}

// The viscous operator div[mu (grad u + grad u^T)] of component comp at a face,
// with cell viscosities and the edge viscosities ex[0] (xy), ex[1] (xz), ex[2]
// (yz) -- each the mean of the four cells around its edge, formed once per
// viscosity field.  Returned as h^2 L_mu(u) = S - Lc u_f: S the sum over the
// face's neighbours (its own component and the cross terms), Lc the sum of the
// six coefficients (the diagonal, which the Jacobi splitting moves to the left).
// Edge arrays: xy [nz][ny+1][nx+1], xz [nz+1][ny][nx+1], yz [nz+1][ny+1][nx].
template <typename R>
struct Edges3 {
    const R *xy, *xz, *yz;
};
template <bool IN, typename R>
__device__ __forceinline__ R exy_at(const Tank3P &P, const R *__restrict__ a, int i, int j, int k)
{
    if constexpr (IN) return a[(k * (P.ny + 1) + j) * (P.nx + 1) + i];
    return a[((long long)k * (P.ny + 1) + j) * (P.nx + 1) + i];
}
template <bool IN, typename R>
__device__ __forceinline__ R exz_at(const Tank3P &P, const R *__restrict__ a, int i, int j, int k)
{
    if constexpr (IN) return a[(k * P.ny + j) * (P.nx + 1) + i];
    return a[((long long)k * P.ny + j) * (P.nx + 1) + i];
}
template <bool IN, typename R>
__device__ __forceinline__ R eyz_at(const Tank3P &P, const R *__restrict__ a, int i, int j, int k)
{
    if constexpr (IN) return a[(k * (P.ny + 1) + j) * P.nx + i];
    return a[((long long)k * (P.ny + 1) + j) * P.nx + i];
}
template <bool IN, typename R>
__device__ __forceinline__ void offdiag3(const Tank3P &P, const R *__restrict__ mu, const Edges3<R> &E,
                                         const Vel3<R> &V, int comp, int i, int j, int k, R &S, R &Lc)
{
#define U3(a, b, c) uq<IN>(P, V.u, a, b, c)
#define V3(a, b, c) vq<IN>(P, V.v, a, b, c)
#define W3(a, b, c) wq<IN>(P, V.w, V.win, a, b, c)
    if (comp == 0) {
        const R m1 = cellq<IN>(P, mu, i, j, k), m0 = cellq<IN>(P, mu, i - 1, j, k);
        const R e1 = exy_at<IN>(P, E.xy, i, j + 1, k), e0 = exy_at<IN>(P, E.xy, i, j, k);
        const R f1 = exz_at<IN>(P, E.xz, i, j, k + 1), f0 = exz_at<IN>(P, E.xz, i, j, k);
        S = scl2<R>(2.f, m1 * U3(i + 1, j, k) + m0 * U3(i - 1, j, k)) +
            ((e1 * ((U3(i, j + 1, k) + V3(i, j + 1, k)) - V3(i - 1, j + 1, k)) +
              e0 * ((U3(i, j - 1, k) - V3(i, j, k)) + V3(i - 1, j, k))) +
             (f1 * ((U3(i, j, k + 1) + W3(i, j, k + 1)) - W3(i - 1, j, k + 1)) +
              f0 * ((U3(i, j, k - 1) - W3(i, j, k)) + W3(i - 1, j, k))));
        Lc = scl2<R>(2.f, m1 + m0) + ((e1 + e0) + (f1 + f0));
    } else if (comp == 1) {
        const R m1 = cellq<IN>(P, mu, i, j, k), m0 = cellq<IN>(P, mu, i, j - 1, k);
        const R e1 = exy_at<IN>(P, E.xy, i + 1, j, k), e0 = exy_at<IN>(P, E.xy, i, j, k);
        const R f1 = eyz_at<IN>(P, E.yz, i, j, k + 1), f0 = eyz_at<IN>(P, E.yz, i, j, k);
        S = scl2<R>(2.f, m1 * V3(i, j + 1, k) + m0 * V3(i, j - 1, k)) +
            ((e1 * ((V3(i + 1, j, k) + U3(i + 1, j, k)) - U3(i + 1, j - 1, k)) +
              e0 * ((V3(i - 1, j, k) - U3(i, j, k)) + U3(i, j - 1, k))) +
             (f1 * ((V3(i, j, k + 1) + W3(i, j, k + 1)) - W3(i, j - 1, k + 1)) +
              f0 * ((V3(i, j, k - 1) - W3(i, j, k)) + W3(i, j - 1, k))));
        Lc = scl2<R>(2.f, m1 + m0) + ((e1 + e0) + (f1 + f0));
    } else {
        const R m1 = cellq<IN>(P, mu, i, j, k), m0 = cellq<IN>(P, mu, i, j, k - 1);
        const R e1 = exz_at<IN>(P, E.xz, i + 1, j, k), e0 = exz_at<IN>(P, E.xz, i, j, k);
        const R f1 = eyz_at<IN>(P, E.yz, i, j + 1, k), f0 = eyz_at<IN>(P, E.yz, i, j, k);
        S = scl2<R>(2.f, m1 * W3(i, j, k + 1) + m0 * W3(i, j, k - 1)) +
            ((e1 * ((W3(i + 1, j, k) + U3(i + 1, j, k)) - U3(i + 1, j, k - 1)) +
              e0 * ((W3(i - 1, j, k) - U3(i, j, k)) + U3(i, j, k - 1))) +
             (f1 * ((W3(i, j + 1, k) + V3(i, j + 1, k)) - V3(i, j + 1, k - 1)) +
              f0 * ((W3(i, j - 1, k) - V3(i, j, k)) + V3(i, j, k - 1))));
        Lc = scl2<R>(2.f, m1 + m0) + ((e1 + e0) + (f1 + f0));
    }
#undef U3
#undef V3
#undef W3
}

// solved faces of component comp: u i = 1..nx-1; v j = 1..ny-1; w k = 1..nz
__device__ __forceinline__ bool face_of(const Tank3P &P, int comp, int &i, int &j, int &k, long long &f)
{
    i = blockIdx.x * blockDim.x + threadIdx.x;
    j = blockIdx.y;
    k = blockIdx.z;
    if (comp == 0) {
        i += 1;
        if (i > P.nx - 1) return false;
        f = ((long long)k * P.ny + j) * (P.nx + 1) + i;
    } else if (comp == 1) {
        j += 1;
        if (i > P.nx - 1 || j > P.ny - 1) return false;
        f = ((long long)k * (P.ny + 1) + j) * P.nx + i;
    } else {
        k += 1;
        if (i > P.nx - 1) return false;
        f = ((long long)k * P.ny + j) * P.nx + i;
    }
    return true;
}

// edge viscosities of the cell field mu (cells clamped into the grid, as the
// stencils' accessors clamp them): one thread per (i, j, k) of the corner lattice
template <typename R>
__global__ void __launch_bounds__(128) k3t_edges(Tank3P P, const R *__restrict__ mu, R *__restrict__ xy,
                                                 R *__restrict__ xz, R *__restrict__ yz)
{
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    if (i > nx) return;
    if (k < nz)
        xy[((long long)k * (ny + 1) + j) * (nx + 1) + i] =
            R(0.25) * (cellq<false>(P, mu, i - 1, j - 1, k) + cellq<false>(P, mu, i, j - 1, k) +
                       cellq<false>(P, mu, i - 1, j, k) + cellq<false>(P, mu, i, j, k));
    if (j < ny)
        xz[((long long)k * ny + j) * (nx + 1) + i] =
            R(0.25) * (cellq<false>(P, mu, i - 1, j, k - 1) + cellq<false>(P, mu, i, j, k - 1) +
                       cellq<false>(P, mu, i - 1, j, k) + cellq<false>(P, mu, i, j, k));
    if (i < nx)
        yz[((long long)k * (ny + 1) + j) * nx + i] =
            R(0.25) * (cellq<false>(P, mu, i, j - 1, k - 1) + cellq<false>(P, mu, i, j, k - 1) +
                       cellq<false>(P, mu, i, j - 1, k) + cellq<false>(P, mu, i, j, k));
}

// face densities of the cell field rho: the u-, v- and w-face arrays
template <typename R>
__global__ void __launch_bounds__(128) k3t_face_rho(Tank3P P, const R *__restrict__ rho, R *__restrict__ ru,
                                                    R *__restrict__ rv, R *__restrict__ rw)
{
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    if (i > nx) return;
    if (j < ny && k < nz) ru[((long long)k * ny + j) * (nx + 1) + i] = ruq<false>(P, rho, i, j, k);
    if (i < nx && k < nz) rv[((long long)k * (ny + 1) + j) * nx + i] = rvq<false>(P, rho, i, j, k);
    if (i < nx && j < ny) rw[((long long)k * ny + j) * nx + i] = rwq<false>(P, rho, i, j, k);
}

template <typename R>
struct MomIn {
    const R *rfc[3];                       // face densities of rho^n (u-, v-, w-faces)
    const R *mu_n, *chi1, *rf1;
    Edges3<R> E;                           // edge viscosities of mu^n
    const double *p;                       // p^{n+1/2,k} (FP64: its differences are taken before rounding)
    Vel3<R> V;                             // the advecting velocity: u^n (cycle 0) or the mean of n and n+1,k
    Vel3<R> Vn;                            // u^n, v^n, w^n with w_in(t^n): the explicit half of the system
    const R *dampu, *vortc, *vortf;        // damping weight at u-faces; vorticity damping at cell / face heights
    R dt, idt, dtih, ih2, zd1, g, ikp;
};

// faces whose whole stencil (three cells each way) lies inside the grid: there
// every ghost rule of the accessors is inactive, so the unclamped form computes
// the same values
__device__ __forceinline__ bool interior3(const Tank3P &P, int i, int j, int k)
{
    return P.idx32 && i >= 3 && i <= P.nx - 4 && j >= 3 && j <= P.ny - 4 && k >= 3 && k <= P.nz - 4;
}

// the momentum system at a face from its transport terms rb (rho-breve) and C
template <bool IN, typename R>
__device__ __forceinline__ void momentum_finish(const Tank3P &P, const MomIn<R> &M, int comp, int i, int j, int k,
                                                long long f, R rb, R C, R *__restrict__ Dout, R *__restrict__ Rout)
{
    R S, Lc;
    offdiag3<IN, R>(P, M.mu_n, M.E, M.Vn, comp, i, j, k, S, Lc);
    const R uc = comp == 0 ? M.Vn.u[f] : comp == 1 ? M.Vn.v[f] : M.Vn.w[f];
    const R visc = (S - Lc * uc) * M.ih2;
    const double ih = P.ih;
    const int ci = comp == 0 ? i - 1 : i, cj = comp == 1 ? j - 1 : j, ck = comp == 2 ? k - 1 : k;
    const R chi = scl2<R>(0.5f, cellq<IN>(P, M.chi1, ci, cj, ck) + cellq<IN>(P, M.chi1, i, j, k));
    const R al = comp == 0 ? M.dampu[i] : dampc<R>(P, i);
    const R vd = comp == 2 ? M.vortf[k] : M.vortc[k];
    const R rbdt = rb * M.idt;
    Dout[f] = rbdt + chi * M.ikp + al * rbdt + vd;
    const double pc = k < P.nz ? M.p[((long long)k * P.ny + j) * P.nx + i] : 0.0;
    const R adv = frq<IN>(P, M.rfc[comp], comp, i, j, k) * uc * M.idt - C + scl2<R>(0.5f, visc);
    if (comp == 0) {
        Rout[f] = adv - narrow_r<R>((pc - M.p[((long long)k * P.ny + j) * P.nx + i - 1]) * ih);
    } else if (comp == 1) {
        Rout[f] = adv - narrow_r<R>((pc - M.p[((long long)k * P.ny + j - 1) * P.nx + i]) * ih);
    } else {
        const R rf = scl2<R>(0.5f, cellq<IN>(P, M.rf1, i, j, k - 1) + cellq<IN>(P, M.rf1, i, j, k));
        const double pb = M.p[((long long)(k - 1) * P.ny + j) * P.nx + i];
        const double gp = k < P.nz ? (pc - pb) * ih : -2.0 * pb * ih;
        Rout[f] = adv - rf * M.g + chi * M.zd1 * M.ikp - narrow_r<R>(gp);
    }
}

template <bool IN, typename R>
__device__ __forceinline__ void momentum_at(const Tank3P &P, const MomIn<R> &M, int comp, int i, int j, int k,
                                            long long f, R *__restrict__ Dout, R *__restrict__ Rout)
{
    R rb, C;
    transport3<IN, R>(P, M.rfc[comp], M.V, comp, i, j, k, M.dtih, rb, C);
    momentum_finish<IN, R>(P, M, comp, i, j, k, f, rb, C, Dout, Rout);
}

template <int COMP, typename R>
__global__ void __launch_bounds__(128) k3t_momentum(Tank3P P, MomIn<R> M, R *__restrict__ Dout, R *__restrict__ Rout)
{
    pdl_entry();
    int i, j, k;
    long long f;
    if (!face_of(P, COMP, i, j, k, f)) return;
    if (interior3(P, i, j, k))
        momentum_at<true, R>(P, M, COMP, i, j, k, f, Dout, Rout);
    else
        momentum_at<false, R>(P, M, COMP, i, j, k, f, Dout, Rout);
}

// The same in two kernels (option "tank3_split_momentum", the default): the
// transport terms (rb into Dout, C into Rout), then the viscous terms and the
// assembly, which read them back at the same face.  Two smaller kernels: the
// float-pair momentum went from 19.9 to 13.0 ms per step at 512x256x256 (fewer
// registers, fewer instruction-fetch stalls), FP64 unchanged (its FP64 pipe
// bounds both forms)
template <int COMP, typename R>
__global__ void __launch_bounds__(128, 8) k3t_transport(Tank3P P, MomIn<R> M, R *__restrict__ Dout, R *__restrict__ Rout)
{
    pdl_entry();
    // a warp covers 31 CVs along x: lane l forms the lower x face of CV cv0 + l
    // and takes the upper one from lane l + 1 (the same face); lane 31 supplies
    // its lower face only.  (Transport3's terms in its order: the same values.)
    const int lane = threadIdx.x & 31;
    const int ncv = P.nx - (COMP == 0 ? 1 : 0);  // solved faces along x in the row
    const int cv = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 31 + lane;
    const int i = cv + (COMP == 0 ? 1 : 0), j = blockIdx.y + (COMP == 1 ? 1 : 0), k = blockIdx.z + (COMP == 2 ? 1 : 0);
    const bool in = interior3(P, i, j, k);
    const R *rfc = M.rfc[COMP];
    R m0 = R(0), f0 = R(0);
    if (cv <= ncv) {
        if (in)
            tface<true, R>(P, rfc, M.V, COMP, i, j, k, 0, 0, m0, f0);
        else
            tface<false, R>(P, rfc, M.V, COMP, i, j, k, 0, 0, m0, f0);
    }
    const R m1 = shfl_down1<R>(m0), f1 = shfl_down1<R>(f0);
    if (lane == 31 || cv >= ncv) return;
    R m[4], f[4], r0;
    if (in) {
#pragma unroll
        for (int q = 0; q < 4; ++q) tface<true, R>(P, rfc, M.V, COMP, i, j, k, 1 + q / 2, q & 1, m[q], f[q]);
        r0 = frq<true>(P, rfc, COMP, i, j, k);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) tface<false, R>(P, rfc, M.V, COMP, i, j, k, 1 + q / 2, q & 1, m[q], f[q]);
        r0 = frq<false>(P, rfc, COMP, i, j, k);
    }
    const long long fi = COMP == 0   ? ((long long)k * P.ny + j) * (P.nx + 1) + i
                         : COMP == 1 ? ((long long)k * (P.ny + 1) + j) * P.nx + i
                                     : ((long long)k * P.ny + j) * P.nx + i;
    Dout[fi] = r0 - M.dtih * (((m1 - m0) + (m[1] - m[0])) + (m[3] - m[2]));
    Rout[fi] = (((f1 - f0) + (f[1] - f[0])) + (f[3] - f[2])) * cst3<R>(P).ih;
}
template <int COMP, typename R>
__global__ void __launch_bounds__(128) k3t_momentum_finish(Tank3P P, MomIn<R> M, R *__restrict__ Dout,
                                                           R *__restrict__ Rout)
{
    pdl_entry();
    int i, j, k;
    long long f;
    if (!face_of(P, COMP, i, j, k, f)) return;
    const R rb = Dout[f], C = Rout[f];
    if (interior3(P, i, j, k))
        momentum_finish<true, R>(P, M, COMP, i, j, k, f, rb, C, Dout, Rout);
    else
        momentum_finish<false, R>(P, M, COMP, i, j, k, f, rb, C, Dout, Rout);
}

// The Crank-Nicolson system of component comp, split on its diagonal:
// B = (R + (L(A) - ld A) / 2) / (D - ld / 2) with h^2 (L(A) - ld A) = S(A) and
// -h^2 ld = Lc.  Formed once per step (mu^{n+1} is fixed during the sweeps):
// Rr <- R / (D + Lc / (2 h^2)) and Q = (1 / (2 h^2)) / (D + Lc / (2 h^2)), so that a
// sweep is B = Rr + Q S(A).
template <int COMP, typename R>
__global__ void __launch_bounds__(128) k3t_jprep(Tank3P P, const R *__restrict__ mu1, Edges3<R> E,
                                                 const R *__restrict__ D, R *__restrict__ Rr, R *__restrict__ Qo,
                                                 R ih2)
{
    pdl_entry();
    int i, j, k;
    long long f;
    if (!face_of(P, COMP, i, j, k, f)) return;
    R Lc;
    if (COMP == 0)
        Lc = scl2<R>(2.f, cellq<false>(P, mu1, i, j, k) + cellq<false>(P, mu1, i - 1, j, k)) +
             ((exy_at<false>(P, E.xy, i, j + 1, k) + exy_at<false>(P, E.xy, i, j, k)) +
              (exz_at<false>(P, E.xz, i, j, k + 1) + exz_at<false>(P, E.xz, i, j, k)));
    else if (COMP == 1)
        Lc = scl2<R>(2.f, cellq<false>(P, mu1, i, j, k) + cellq<false>(P, mu1, i, j - 1, k)) +
             ((exy_at<false>(P, E.xy, i + 1, j, k) + exy_at<false>(P, E.xy, i, j, k)) +
              (eyz_at<false>(P, E.yz, i, j, k + 1) + eyz_at<false>(P, E.yz, i, j, k)));
    else
        Lc = scl2<R>(2.f, cellq<false>(P, mu1, i, j, k) + cellq<false>(P, mu1, i, j, k - 1)) +
             ((exz_at<false>(P, E.xz, i + 1, j, k) + exz_at<false>(P, E.xz, i, j, k)) +
              (eyz_at<false>(P, E.yz, i, j + 1, k) + eyz_at<false>(P, E.yz, i, j, k)));
    const R hi2 = scl2<R>(0.5f, ih2);
    const R inv = R(1) / (D[f] + hi2 * Lc);
    Rr[f] = Rr[f] * inv;
    Qo[f] = hi2 * inv;
}

// one Crank-Nicolson Jacobi sweep of component comp: B = Rr + Q S(A)
template <int COMP, typename R>
__global__ void __launch_bounds__(128) k3t_jacobi(Tank3P P, const R *__restrict__ mu1, Edges3<R> E, Vel3<R> A,
                                                  const R *__restrict__ Rr, const R *__restrict__ Qf,
                                                  R *__restrict__ B)
{
    pdl_entry();
    int i, j, k;
    long long f;
    if (!face_of(P, COMP, i, j, k, f)) return;
    R S, Lc;
    if (interior3(P, i, j, k))
        offdiag3<true, R>(P, mu1, E, A, COMP, i, j, k, S, Lc);
    else
        offdiag3<false, R>(P, mu1, E, A, COMP, i, j, k, S, Lc);
    B[f] = Rr[f] + Qf[f] * S;
}

// Dirichlet faces of the predictor: u_in(t1) at x = 0, u = 0 at the outlet, v = 0
// on the side walls, w = 0 on the bed
template <typename R>
__global__ void k3t_dirichlet(Tank3P P, const R *__restrict__ uin1, R *u, R *v, R *w)
{
    pdl_entry();
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    if (a < ny * nz) {
        const int k = a / ny, j = a - k * ny;
        const long long r = ((long long)k * ny + j) * (nx + 1);
        u[r] = uin1[k];
        u[r + nx] = R(0);
    }
    if (a < nx * nz) {
        const int k = a / nx, i = a - k * nx;
        v[((long long)k * (ny + 1)) * nx + i] = R(0);
        v[((long long)k * (ny + 1) + ny) * nx + i] = R(0);
    }
    if (a < nx * ny) w[a] = R(0);
}

// a = src (n values)
template <typename R>
__global__ void __launch_bounds__(256) k3t_copy(long long n, const R *__restrict__ src, R *__restrict__ a)
{
    pdl_entry();
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= n) return;
    a[q] = src[q];
}

// beta = 1 / D on the solved faces, 0 on the walls and the bed (FP64 coefficients);
// one block row per face row (gridf)
template <typename R>
__global__ void __launch_bounds__(128) k3t_beta(Tank3P P, int comp, const R *__restrict__ D,
                                                double *__restrict__ beta)
{
    pdl_entry();
    const int nxf = P.nx + (comp == 0), nyf = P.ny + (comp == 1);
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nxf) return;
    const long long f = ((long long)k * nyf + j) * nxf + i;
    const bool wall = comp == 0 ? (i == 0 || i == P.nx) : comp == 1 ? (j == 0 || j == P.ny) : k == 0;
    beta[f] = wall ? 0.0 : widen_r<R>(R(1) / D[f]);
}

// rhs = -h div u* (FP64 from the predictor's values)
template <typename R>
__global__ void __launch_bounds__(128) k3t_rhs(Tank3P P, Vel3<R> S, double *__restrict__ rhs)
{
    pdl_entry();
    Cell3 q;
    if (!cell_of(P, q)) return;
    const int nx = P.nx, ny = P.ny;
    const long long fu = ((long long)q.k * ny + q.j) * (nx + 1) + q.i, fv = ((long long)q.k * (ny + 1) + q.j) * nx + q.i;
    const long long pl = (long long)nx * ny;
    if constexpr (is_df<R>) {  // the sum in pairs, widened once (two FP64 operations, not twelve)
        rhs[q.c] = -P.h * widen_r<R>(((S.u[fu + 1] - S.u[fu]) + (S.v[fv + nx] - S.v[fv])) + (S.w[q.c + pl] - S.w[q.c]));
    } else {
        rhs[q.c] = -P.h * (((widen_r<R>(S.u[fu + 1]) - widen_r<R>(S.u[fu])) +
                            (widen_r<R>(S.v[fv + nx]) - widen_r<R>(S.v[fv]))) +
                           (widen_r<R>(S.w[q.c + pl]) - widen_r<R>(S.w[q.c])));
    }
}

// u^{n+1} = u* - beta grad phi in FP64 (top w face: the ghost -phi); p += phi
template <typename R>
__global__ void __launch_bounds__(128) k3t_project(Tank3P P, int comp, const R *__restrict__ S,
                                                   const double *__restrict__ beta, const double *__restrict__ phi,
                                                   double *__restrict__ out)
{
    pdl_entry();
    const int nx = P.nx, ny = P.ny, nz = P.nz, nxf = nx + (comp == 0), nyf = ny + (comp == 1);
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nxf) return;
    const long long f = ((long long)k * nyf + j) * nxf + i;
    const double ih = P.ih;
    double a = widen_r<R>(S[f]);
    if (comp == 0) {
        const long long c = ((long long)k * ny + j) * nx + i;
        if (i > 0 && i < nx) a -= beta[f] * (phi[c] - phi[c - 1]) * ih;
    } else if (comp == 1) {
        if (j > 0 && j < ny) {
            const long long c = ((long long)k * ny + j) * nx + i;
            a -= beta[f] * (phi[c] - phi[c - nx]) * ih;
        }
    } else {
        const long long pl = (long long)nx * ny;
        if (k > 0 && k < nz) a -= beta[f] * (phi[f] - phi[f - pl]) * ih;
        if (k == nz) a += 2.0 * beta[f] * phi[f - pl] * ih;
    }
    out[f] = a;
}

__global__ void k3t_add(long long n, const double *__restrict__ a, double *__restrict__ b)
{
    pdl_entry();
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c < n) b[c] += a[c];
}

// working copies: out = R(in) (float, or the nearest float and its remainder)
// and back, out = double(in)
template <typename R>
__global__ void k3t_narrow(long long n, const double *__restrict__ in, R *__restrict__ out)
{
    pdl_entry();
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c < n) out[c] = narrow_r<R>(in[c]);
}
template <typename R>
__global__ void k3t_widen(long long n, const R *__restrict__ in, double *__restrict__ out)
{
    pdl_entry();
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c < n) out[c] = widen_r<R>(in[c]);
}
// the mean of two time levels: out = (a + b) / 2 (b in the working type or FP64)
template <typename R, typename RB>
__global__ void k3t_mean(long long n, const R *__restrict__ a, const RB *__restrict__ b, R *__restrict__ out)
{
    pdl_entry();
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= n) return;
    if constexpr (std::is_same<RB, double>::value)
        out[c] = scl2<R>(0.5f, a[c] + narrow_r<R>(b[c]));
    else
        out[c] = scl2<R>(0.5f, a[c] + b[c]);
}

constexpr int kRT = 256;  // threads of the reduction kernels

__device__ double block_sum3(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kRT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    return sh[0];
}

// heave force, Eq. int_fh (FP64), over the faces of a box around the cylinder
// [i0, i1) x [j0, j1) x [k0, k1) of cells (a block per (layer k, face kind))
__global__ void __launch_bounds__(kRT) k3t_force(Tank3P P, const double *__restrict__ p, const double *__restrict__ mu,
                                                 Vel3<double> V, double zc, int i0, int i1, int j0, int j1, int k0,
                                                 int k1, double *__restrict__ part)
{
    pdl_entry();
    __shared__ double sh[kRT];
    const int kind = blockIdx.y, k = k0 + blockIdx.x;  // kind 0: z-faces below cell k; 1: x-faces; 2: y-faces
    const double h = P.h, A = h * h;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    auto psi = [&](double x, double y, double z) {
        const double r = sqrt((x - P.bxc) * (x - P.bxc) + (y - P.byc) * (y - P.byc));
        return fmax(r - P.br, fabs(z - zc) - 0.5 * P.blen);
    };
    double acc = 0.0;
    const int ni = i1 - i0, nj = j1 - j0;
    for (int q = threadIdx.x; q < ni * nj; q += kRT) {
        const int i = i0 + q % ni, j = j0 + q / ni;
        if (kind == 0) {
            if (k < 1 || k > nz - 1) continue;
            const double x = (i + 0.5) * h, y = (j + 0.5) * h;
            const double pl = psi(x, y, (k - 0.5) * h), pr = psi(x, y, (k + 0.5) * h);
            if (!(pl * pr < 0.0)) continue;
            const double nz_ = pl < 0.0 ? 1.0 : -1.0, wl = fabs(pl), wr = fabs(pr);
            const long long c = ((long long)k * ny + j) * nx + i, cb = c - (long long)nx * ny;
            const double pf = (p[cb] * wr + p[c] * wl) / (wl + wr);
            const double muf = 0.5 * (mu[cb] + mu[c]);
            const double dwdz = (wq<false>(P, V.w, V.win, i, j, k + 1) - wq<false>(P, V.w, V.win, i, j, k - 1)) / (2.0 * h);
            acc += (-pf * nz_ + muf * 2.0 * dwdz * nz_) * A;
        } else if (kind == 1) {
            if (i < 1 || k > nz - 1) continue;
            const double y = (j + 0.5) * h, z = (k + 0.5) * h;
            const double pl = psi((i - 0.5) * h, y, z), pr = psi((i + 0.5) * h, y, z);
            if (!(pl * pr < 0.0)) continue;
            const double nx_ = pl < 0.0 ? 1.0 : -1.0;
            const long long c = ((long long)k * ny + j) * nx + i;
            const double muf = 0.5 * (mu[c - 1] + mu[c]);
            const double dwdx = 0.5 * ((wq<false>(P, V.w, V.win, i, j, k) - wq<false>(P, V.w, V.win, i - 1, j, k)) +
                                       (wq<false>(P, V.w, V.win, i, j, k + 1) - wq<false>(P, V.w, V.win, i - 1, j, k + 1))) / h;
            const double dudz = (uq<false>(P, V.u, i, j, k + 1) - uq<false>(P, V.u, i, j, k - 1)) / (2.0 * h);
            acc += muf * (dwdx + dudz) * nx_ * A;
        } else {
            if (j < 1 || k > nz - 1) continue;
            const double x = (i + 0.5) * h, z = (k + 0.5) * h;
            const double pl = psi(x, (j - 0.5) * h, z), pr = psi(x, (j + 0.5) * h, z);
            if (!(pl * pr < 0.0)) continue;
            const double ny_ = pl < 0.0 ? 1.0 : -1.0;
            const long long c = ((long long)k * ny + j) * nx + i;
            const double muf = 0.5 * (mu[c - nx] + mu[c]);
            const double dwdy = 0.5 * ((wq<false>(P, V.w, V.win, i, j, k) - wq<false>(P, V.w, V.win, i, j - 1, k)) +
                                       (wq<false>(P, V.w, V.win, i, j, k + 1) - wq<false>(P, V.w, V.win, i, j - 1, k + 1))) / h;
            const double dvdz = (vq<false>(P, V.v, i, j, k + 1) - vq<false>(P, V.v, i, j, k - 1)) / (2.0 * h);
            acc += muf * (dwdy + dvdz) * ny_ * A;
        }
    }
    const double s = block_sum3(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// sum of n partials in order (one block)
__global__ void __launch_bounds__(kRT) k3t_sum(const double *__restrict__ part, int n, double *__restrict__ out)
{
    pdl_entry();
    __shared__ double sh[kRT];
    double a = 0.0;
    for (int q = threadIdx.x; q < n; q += kRT) a += part[q];
    const double s = block_sum3(a, sh);
    if (threadIdx.x == 0) *out = s;
}

// ||h div u||^2 partials, one per block of cells
__global__ void __launch_bounds__(kRT) k3t_div2(Tank3P P, Vel3<double> S, double *__restrict__ part)
{
    pdl_entry();
    __shared__ double sh[kRT];
    double a = 0.0;
    // row by row (one 32-bit division per row, none per cell)
    const int nx = P.nx, ny = P.ny;
    const long long rows = (long long)ny * P.nz, pl = (long long)nx * ny;
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const int k = (int)(r / ny), j = (int)(r - (long long)k * ny);
        const long long c0 = r * nx, fu0 = r * (nx + 1), fv0 = ((long long)k * (ny + 1) + j) * nx;
        for (int i = threadIdx.x; i < nx; i += kRT) {
            const double d = P.h * (((S.u[fu0 + i + 1] - S.u[fu0 + i]) + (S.v[fv0 + i + nx] - S.v[fv0 + i])) +
                                    (S.w[c0 + i + pl] - S.w[c0 + i]));
            a += d * d;
        }
    }
    const double s = block_sum3(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// initial state: sigma = z - depth - eta(x) (eta per column given), u and w from
// (x, z) tables broadcast along y, v = 0
__global__ void __launch_bounds__(128) k3t_init(Tank3P P, const double *__restrict__ eta, const double *__restrict__ uxz,
                                                const double *__restrict__ wxz, double *sig, double *u, double *w)
{
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    const int nx = P.nx, ny = P.ny;
    if (i <= nx) u[((long long)k * ny + j) * (nx + 1) + i] = uxz[(long long)k * (nx + 1) + i];
    if (i < nx) {
        sig[((long long)k * ny + j) * nx + i] = (k + 0.5) * P.h - P.depth - eta[i];
        w[((long long)(k + 1) * ny + j) * nx + i] = wxz[(long long)(k + 1) * nx + i];
        if (k == 0) w[(long long)j * nx + i] = 0.0;
    }
}

// p^{-1/2}: the discrete hydrostatic pressure of rho^flow from the top face down
__global__ void k3t_hydrostatic(Tank3P P, const double *__restrict__ rf, double g, double *__restrict__ p)
{
    pdl_entry();
    const long long col = blockIdx.x * (long long)blockDim.x + threadIdx.x, pl = (long long)P.nx * P.ny;
    if (col >= pl) return;
    double pp = 0.5 * rf[(P.nz - 1) * pl + col] * g * P.h;
    p[(P.nz - 1) * pl + col] = pp;
    for (int k = P.nz - 2; k >= 0; --k) {
        pp += 0.5 * (rf[k * pl + col] + rf[(k + 1) * pl + col]) * g * P.h;
        p[k * pl + col] = pp;
    }
}

// Inflow data of a step at x = 0: the Airy velocity of the incident components,
// Wheeler-stretched up to the surface and blended to zero in the air over a
// half-width h (the arithmetic of airy_host) -- u_in(t1) at the cell layers,
// w_in(t0), w_in(t1) and their mean at the face heights -- into bc (FP64; the
// host has written the vorticity-damping entries), and all entries narrowed
// into bcr (nullable).  One warp per layer: rows 0..nz-1 the cells, nz..2nz the
// faces (both times); the components are split over the lanes.  Evaluated on
// the host, these ~6 x 10^5 transcendentals per step kept the GPU idle for
// several milliseconds at the start of every step.
__device__ __forceinline__ double warp_sum_d(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename R>
__global__ void __launch_bounds__(128) k3t_inflow(Tank3P P, double t0, double t1, double *__restrict__ bc, R *bcr)
{
    pdl_entry();
    const int nz = P.nz, lane = threadIdx.x & 31, row = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (row > 2 * nz) return;
    double *uin1 = bc, *win0 = uin1 + nz, *win1 = win0 + nz + 1, *vc = win1 + nz + 1, *vf = vc + nz,
           *wmean = vf + nz + 1;
    const bool cell = row < nz;
    const int k = cell ? row : row - nz;
    const double z = cell ? (k + 0.5) * P.h : k * P.h, d = P.depth;
    double out[2] = {0.0, 0.0};
    for (int tt = 0; tt < (cell ? 1 : 2); ++tt) {
        const double t = cell || tt == 1 ? t1 : t0;
        double e = 0.0;  // eta at x = 0
        for (int c = lane; c < P.ncomp; c += 32) e += P.amp[c] * cos(P.kw[c] * 0.0 - P.omega[c] * t + P.phase[c]);
        e = warp_sum_d(e);
        const double zs = z < d + e ? z : d + e, zp = d * zs / (d + e), phi = z - d - e;
        const double blend = 1.0 - (phi < -P.h ? 0.0 : phi > P.h ? 1.0
                                    : 0.5 * (1.0 + phi / P.h + sin(kPi3 * phi / P.h) / kPi3));
        double s = 0.0;
        for (int c = lane; c < P.ncomp; c += 32) {
            const double kk = P.kw[c], om = P.omega[c], ph = kk * 0.0 - om * t + P.phase[c], sk = sinh(kk * d);
            s += cell ? P.amp[c] * om * cosh(kk * zp) / sk * cos(ph) : P.amp[c] * om * sinh(kk * zp) / sk * sin(ph);
        }
        out[tt] = blend * warp_sum_d(s);
    }
    if (lane != 0) return;
    if (cell) {
        uin1[k] = out[0];
        if (bcr) bcr[k] = R(out[0]);
    } else {
        const double m = 0.5 * (out[0] + out[1]);
        win0[k] = out[0];
        win1[k] = out[1];
        wmean[k] = m;
        if (bcr) {
            bcr[nz + k] = R(out[0]);
            bcr[2 * nz + 1 + k] = R(out[1]);
            bcr[5 * nz + 3 + k] = R(m);
        }
    }
    if (bcr && row < nz) bcr[3 * nz + 2 + row] = R(vc[row]);
    if (bcr && row < nz + 1) bcr[4 * nz + 2 + row] = R(vf[row]);
}

dim3 grid3(const Tank3P &P) { return dim3((P.nx + 127) / 128, P.ny, P.nz); }
// the faces of component comp, one 128-thread row per face row
dim3 gridf(const Tank3P &P, int comp)
{
    return dim3((P.nx + (comp == 0) + 127) / 128, P.ny + (comp == 1), P.nz + (comp == 2));
}

// sigma advected: the face values of s in the three directions into F (face
// layouts of u, v, w), then the cells' update from them into out
template <typename R>
void advect3(const Tank3P &P, const size_t nf[3], const R *base, const R *s, const Vel3<R> &V, R dt,
             const Ghost3 &G, R *const F[3], R *out, cudaStream_t st)
{
    const double nc = (double)P.nx * P.ny * P.nz;
    {
        WEC_PROF("tank3_advect_faces", 0, sizeof(R) * (nc + 2.0 * nf[0]), st);
        launch_k(k3t_ppm_faces<0, R>, grid3(P), 128, 0, st, P, s, V.u, dt, G, F[0]);
    }
    {
        WEC_PROF("tank3_advect_faces", 1, sizeof(R) * (nc + 2.0 * nf[1]), st);
        launch_k(k3t_ppm_faces<1, R>, gridf(P, 1), 128, 0, st, P, s, V.v, dt, G, F[1]);
    }
    {
        WEC_PROF("tank3_advect_faces", 2, sizeof(R) * (nc + 2.0 * nf[2]), st);
        launch_k(k3t_ppm_faces<2, R>, gridf(P, 2), 128, 0, st, P, s, V.w, dt, G, F[2]);
    }
    WEC_PROF("tank3_advect", 0, sizeof(R) * (2.0 * nc + 2.0 * (nf[0] + nf[1] + nf[2])), st);
    launch_k(k3t_advect<R>, grid3(P), 128, 0, st, P, base, (const R *)F[0], (const R *)F[1], (const R *)F[2], V.u,
             V.v, V.w, dt, out);
}

int tank3_check(const wec_tank3 *T)
{
    if (!T) return fail(WEC_ERR_INVALID, "tank3 is NULL");
    return WEC_OK;
}

// host copies of the wave components: amp, omega, k, phase (4 x ncomp)
struct Waves3 {
    int n;
    const double *amp, *om, *k, *ph;
};

double eta_host(const Waves3 &W, double x, double t)
{
    double e = 0.0;
    for (int c = 0; c < W.n; ++c) e += W.amp[c] * std::cos(W.k[c] * x - W.om[c] * t + W.ph[c]);
    return e;
}

double heav_host(double phi, double eps)
{
    if (phi < -eps) return 0.0;
    if (phi > eps) return 1.0;
    return 0.5 * (1.0 + phi / eps + std::sin(kPi3 * phi / eps) / kPi3);
}

// Airy (u, w) at (x, z, t): linear potential with Wheeler stretching up to the
// surface, blended to zero in the air over a half-width h
void airy_host(const Waves3 &W, double depth, double h, double x, double z, double t, double *uo, double *wo)
{
    const double e = eta_host(W, x, t);
    const double zs = z < depth + e ? z : depth + e;
    const double zp = depth * zs / (depth + e);
    const double blend = 1.0 - heav_host(z - depth - e, h);
    double su = 0.0, sw = 0.0;
    for (int c = 0; c < W.n; ++c) {
        const double k = W.k[c], om = W.om[c], ph = k * x - om * t + W.ph[c], sk = std::sinh(k * depth);
        su += W.amp[c] * om * std::cosh(k * zp) / sk * std::cos(ph);
        sw += W.amp[c] * om * std::sinh(k * zp) / sk * std::sin(ph);
    }
    *uo = blend * su;
    *wo = blend * sw;
}

// eta at the three ghost columns at time t (host, FP64)
Ghost3 ghost_at(const wec_tank3 *T, double t)
{
    const int n = T->P.ncomp;
    const Waves3 W{n, T->hwave.data(), T->hwave.data() + n, T->hwave.data() + 2 * n, T->hwave.data() + 3 * n};
    Ghost3 G;
    for (int m = 0; m < 3; ++m) G.e[m] = eta_host(W, -(m + 0.5) * T->P.h, t);
    return G;
}

// nit Sussman pseudo-steps on the field s (scratch s0, s1 of the same type)
template <typename R>
int reinit_buf(wec_tank3 *T, R *s, R *s0, R *s1, int nit, double t)
{
    const double dtau = 0.3 * T->P.h, b = sizeof(R);
    {
        WEC_PROF("tank3_reinit", 1, 2.0 * b * T->nc, T->st);
        launch_k(k3t_reinit_sign<R>, grid3(T->P), 128, 0, T->st, T->P, (const R *)s, s0);
    }
    for (int it = 0; it < nit; ++it) {
        {
            WEC_PROF("tank3_reinit", 0, 3.0 * b * T->nc, T->st);
            launch_k(k3t_reinit_stage<R>, grid3(T->P), 128, 0, T->st, T->P, (const R *)s, (const R *)s0, s1,
                     ghost_at(T, t), dtau, 1);
        }
        WEC_PROF("tank3_reinit", 0, 4.0 * b * T->nc, T->st);
        launch_k(k3t_reinit_stage<R>, grid3(T->P), 128, 0, T->st, T->P, (const R *)s1, (const R *)s0, s,
                 ghost_at(T, t), dtau, 2);
    }
    WEC_CK(cudaGetLastError());
    return WEC_OK;
}

}  // namespace
}  // namespace wec

using namespace wec;

// One step in working type R (double: the FP64 stencils; float pairs or float:
// working copies of sigma and the velocities, refreshed from the FP64 state at
// the start of the step, with materials, advection, reinitialisation,
// transport, viscous terms and Jacobi sweeps in that type).  The force (from
// the FP64 materials at n), the heave, beta and the right-hand side, the solve,
// the projection and the persistent fields are FP64 in all of them.
template <typename R>
static int tank3_step_impl(wec_tank3 *T, Work3<R> &W, double dt, double pto_force, wec_step_result *out)
{
    constexpr bool f32 = !is_f64<R>;  // working copies
    const Tank3P &P = T->P;
    cudaStream_t st = T->st;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const double h = P.h, t0 = T->t, t1 = T->t + dt;
    // the step's phases on the GPU timeline: profile name "tank3_section",
    // level = phase (0 set-up, 1 force and heave, 2 advection, 3 reinitialisation,
    // 4 materials and face data, 5 transport and momentum, 6 Jacobi sweeps, 7 beta,
    // hierarchy and right-hand side, 8 pressure solve, 9 projection, 10 close)
    std::optional<prof::Scope> sec;
    auto section = [&](int id) {
        sec.reset();
        sec.emplace("tank3_section", id, 0.0, st);
    };
    section(0);
    // boundary data of this step: u_in(t1) at the cell layers, w_in(t0) and
    // w_in(t1) at the face heights and their mean (k3t_inflow, on the device),
    // vorticity damping at cell / face heights (here)
    std::vector<double> hb((size_t)6 * nz + 4, 0.0);
    double *vc = hb.data() + 3 * nz + 2, *vf = vc + nz;
    auto vort = [&](double z) {
        const double wd = 4.0 * h;
        if (z < T->lz - wd) return 0.0;
        const double zt = (z - T->lz) / wd;
        return P.rho_a * (std::cos(kPi3 * zt) + 1.0) / (4.0 * dt);
    };
    for (int k = 0; k < nz; ++k) vc[k] = vort((k + 0.5) * h);
    for (int k = 0; k <= nz; ++k) vf[k] = vort(k * h);
    WEC_CK(cudaMemcpyAsync(T->bc, hb.data(), hb.size() * 8, cudaMemcpyHostToDevice, st));
    launch_k(k3t_inflow<R>, nblk(2 * nz + 1, 4), 128, 0, st, P, t0, t1, T->bc, f32 ? W.bc : (R *)nullptr);
    const double *d_win0 = T->bc + nz, *d_win1 = d_win0 + nz + 1;
    const R *r_uin1 = W.bc, *r_win0 = r_uin1 + nz, *r_win1 = r_win0 + nz + 1, *r_vc = r_win1 + nz + 1,
            *r_vf = r_vc + nz;
    if constexpr (f32) {  // working copies of the state
        WEC_PROF("convert", 0, (8.0 + sizeof(R)) * (T->nc + T->nu + T->nv + T->nw), st);
        launch_k(k3t_narrow<R>, nblk((long long)T->nc, 256), 256, 0, st, (long long)T->nc, (const double *)T->sig,
                 W.sig);
        launch_k(k3t_narrow<R>, nblk((long long)T->nu, 256), 256, 0, st, (long long)T->nu, (const double *)T->u, W.u);
        launch_k(k3t_narrow<R>, nblk((long long)T->nv, 256), 256, 0, st, (long long)T->nv, (const double *)T->v, W.v);
        launch_k(k3t_narrow<R>, nblk((long long)T->nw, 256), 256, 0, st, (long long)T->nw, (const double *)T->w, W.w);
    }

    // Fixed-point cycles k = 0 .. n_cycles - 1 (section "Time stepping scheme"):
    // the iterate (sigma, u, p, z)^{n+1,k} starts from time level n (k = 0:
    // sigma^n, u^n, p^{n-1/2}, the body at z^n); cycle k takes the force from
    // it, the heave from level n, advects sigma^n with the means of levels n
    // and n+1,k, and solves level n's momentum system with the iterate's
    // pressure and body velocity.  One cycle is the plain step.  Between
    // cycles the iterate's sigma is in W.tmp, its velocity in T->uk (FP64), its
    // pressure in T->p; the last cycle's projection writes T->u.
    const int ncyc = T->opts.n_cycles > 1 ? T->opts.n_cycles : 1;
    const double fpto = pto_force - T->pto_c * T->zdot;
    const double zc_n = T->zc, zd_n = T->zdot, zd_prev = T->zdot_prev;
    double F = 0.0, zd1 = zd_n, zc1 = zc_n, relres = 0.0;
    int iters = 0, rc = WEC_OK;
    const dim3 gcorner((nx + 1 + 127) / 128, ny + 1, nz + 1);
    const double b = sizeof(R);
    const dim3 gu((nx - 1 + 127) / 128, ny, nz), gv((nx + 127) / 128, ny - 1 > 0 ? ny - 1 : 1, nz),
        gw((nx + 127) / 128, ny, nz);
    const dim3 gc[3] = {gu, gv, gw};
    const size_t nf[3] = {T->nu, T->nv, T->nw};
    const R *r_whalf = r_vf + nz + 1;
    const Ghost3 G0 = ghost_at(T, t0), G1 = ghost_at(T, t1);
    Ghost3 Gh;  // the ghost of the mean of sigma^n and sigma^{n+1,k}
    for (int m = 0; m < 3; ++m) Gh.e[m] = 0.5 * (G0.e[m] + G1.e[m]);
    wec_poisson *S = T->solver;
    double *beta[3] = {S->L64[0].bu, S->L64[0].bv, S->L64[0].bw};

    // materials at level n: the stencils' (W.rho, W.mu) and, FP64, the force's
    if constexpr (f32) {
        WEC_PROF("tank3_materials", 0, 20.0 * T->nc, st);
        launch_k(k3t_materials<R>, grid3(P), 128, 0, st, P, (const R *)W.sig, T->zc, W.rho, W.mu, W.rf, W.chi, 0, 0, 0);
    } else {
        WEC_PROF("tank3_materials", 0, 40.0 * T->nc, st);
        launch_k(k3t_materials<double>, grid3(P), 128, 0, st, P, (const double *)T->sig, T->zc, T->rho, T->mu,
                 T->rhof, T->chi, 0, 0, 0);
    }
    for (int cyc = 0; cyc < ncyc; ++cyc) {
        section(1);
        // (1) the heave force (Eq. int_fh) from p^{n+1/2,k}, u^{n+1,k} over a box
        // of cells around the cylinder at z^{n+1,k}
        const double zck = T->zc;
        const int kcb = (int)(zck / h), mkb = (int)std::ceil(0.5 * P.blen / h) + 3;
        const bool force_box = P.has_body && std::min(nz, kcb + mkb + 1) > std::max(0, kcb - mkb);
        const int fk0 = std::max(0, kcb - mkb), fk1 = std::min(nz, kcb + mkb + 1), sk0 = std::max(0, fk0 - 1);
        // the box's columns; its FP64 materials on them and the column before each side
        const int mi = (int)std::ceil((P.br) / h) + 3;
        const int ic = (int)(P.bxc / h), jc = (int)(P.byc / h);
        const int i0 = std::max(0, ic - mi), i1 = std::min(nx, ic + mi + 1), j0 = std::max(0, jc - mi),
                  j1 = std::min(ny, jc + mi + 1);
        const int si0 = std::max(0, i0 - 1), sj0 = std::max(0, j0 - 1);
        const dim3 gbox((i1 - si0 + 127) / 128, std::max(1, j1 - sj0), std::max(1, fk1 - sk0));
        const double fbox = (double)(i1 - si0) * (j1 - sj0) * (fk1 - sk0);  // cells
        const double *fmu = T->mu;  // FP64 viscosity of the force integral
        if (force_box && cyc == 0 && f32) {
            // the stencils read materials in their own type; the FP64 ones are
            // needed by the force only: the box and the cells before it in x, y, z
            WEC_PROF("tank3_materials", 0, 40.0 * fbox, st);
            launch_k(k3t_materials<double>, gbox, 128, 0, st, P, (const double *)T->sig, zck, T->rho, T->mu, T->rhof,
                     T->chi, sk0, si0, sj0);
        }
        if (force_box && cyc > 0) {
            // materials of the iterate (sigma^{n+1,k} in FP64 in T->tmp) on the force layers
            if constexpr (f32)
                launch_k(k3t_widen<R>, nblk((long long)T->nc, 256), 256, 0, st, (long long)T->nc, (const R *)W.tmp,
                         T->tmp);
            WEC_PROF("tank3_materials", 0, 40.0 * fbox, st);
            launch_k(k3t_materials<double>, gbox, 128, 0, st, P, (const double *)T->tmp, zck, T->s0, T->muk, T->s1,
                     T->phi, sk0, si0, sj0);
            fmu = T->muk;
        }
        if (force_box) {
            const int k0 = fk0, k1 = fk1;
            const Vel3<double> Vk = cyc == 0 ? Vel3<double>{T->u, T->v, T->w, d_win0}
                                             : Vel3<double>{T->uk[0], T->uk[1], T->uk[2], d_win1};
            {
                WEC_PROF("tank3_force", 0, 0.0, st);
                launch_k(k3t_force, dim3(k1 - k0, 3), kRT, 0, st, P, (const double *)T->p, fmu, Vk, zck, i0, i1, j0,
                         j1, k0, k1, T->part);
            }
            launch_k(k3t_sum, 1, kRT, 0, st, (const double *)T->part, 3 * (k1 - k0), T->part + 3 * nz + 1024);
            WEC_CK(cudaMemcpyAsync(&F, T->part + 3 * nz + 1024, 8, cudaMemcpyDeviceToHost, st));
            WEC_CK(cudaStreamSynchronize(st));
        }
        // (2) heave from level n (the stabilised update of the 2D reading)
        zd1 = zd_n;
        zc1 = zc_n;
        if (P.has_body) {
            const double m = T->mass, ma = T->added_mass;
            zd1 = zd_n + (dt * (F - m * T->g + fpto) + ma * (zd_n - zd_prev)) / (m + ma);
            zc1 = zc_n + 0.5 * dt * (zd_n + zd1);
        }
        section(2);
        // (3) sigma: sigma^n advected with u^{n+1/2,k}, sigma^{n+1/2,k} (cycle 0:
        // u^n, sigma^n; ghosts at t0), damping zone, reinitialisation (ghosts at t1)
        Vel3<R> Vt{W.u, W.v, W.w, r_win0};
        const R *sadv = W.sig;
        Ghost3 Ga = G0;
        if (cyc > 0) {
            launch_k(k3t_mean<R, R>, nblk((long long)T->nc, 256), 256, 0, st, (long long)T->nc, (const R *)W.sig,
                     (const R *)W.tmp, W.sh);
            const R *un[3] = {W.u, W.v, W.w};
            for (int c = 0; c < 3; ++c)
                launch_k(k3t_mean<R, double>, nblk((long long)nf[c], 256), 256, 0, st, (long long)nf[c], un[c],
                         (const double *)T->uk[c], W.uh[c]);
            Vt = Vel3<R>{W.uh[0], W.uh[1], W.uh[2], r_whalf};
            sadv = W.sh;
            Ga = Gh;
        }
        {
            // (the face values in the Jacobi buffers B: free until the momentum system)
            const size_t nfa[3] = {T->nu, T->nv, T->nw};
            R *const Fs[3] = {W.B[0], W.B[1], W.B[2]};
            advect3<R>(P, nfa, (const R *)W.sig, sadv, Vt, dt, Ga, Fs, W.tmp, st);
        }
        section(3);
        if (int e = reinit_buf<R>(T, W.tmp, W.s0, W.s1, T->opts.n_reinit, t1)) return e;
        section(4);
        // (4) materials at n+1,k+1 (rho itself is not used: s1 is scratch)
        {
            WEC_PROF("tank3_materials", 0, 5.0 * sizeof(R) * T->nc, st);
            launch_k(k3t_materials<R>, grid3(P), 128, 0, st, P, (const R *)W.tmp, zc1, W.s1, W.mu1, W.rf1, W.chi1,
                     0, 0, 0);
        }
        // (5) transport and the momentum system: face densities of rho^n and
        // edge viscosities of mu^n, then one kernel per component
        {
            WEC_PROF("tank3_faces_edges", 0, b * (T->nc + T->nu + T->nv + T->nw), st);
            launch_k(k3t_face_rho<R>, gcorner, 128, 0, st, P, (const R *)W.rho, W.RF[0], W.RF[1], W.RF[2]);
        }
        {
            WEC_PROF("tank3_faces_edges", 0, b * 4.0 * T->nc, st);
            launch_k(k3t_edges<R>, gcorner, 128, 0, st, P, (const R *)W.mu, W.E[0], W.E[1], W.E[2]);
        }
        const Edges3<R> E{W.E[0], W.E[1], W.E[2]};
        MomIn<R> M{{W.RF[0], W.RF[1], W.RF[2]}, W.mu, W.chi1, W.rf1, E, T->p, Vt, Vel3<R>{W.u, W.v, W.w, r_win0},
                   W.dampu, r_vc, r_vf, R(dt), R(1.0 / dt), R(dt / h), R(1.0 / (h * h)), R(zd1), R(T->g),
                   R(1.0 / T->kappa_p)};
        section(5);
        for (int c = 0; c < 3; ++c) {
            if (c == 1 && ny < 2) continue;
            // face density, mu, two edge arrays, chi (+ rho^flow for w), p, u, v, w in; D, R out
            WEC_PROF("tank3_momentum", c,
                     b * (nf[c] + (c == 2 ? 5.0 : 4.0) * T->nc + T->nu + T->nv + T->nw + 2.0 * nf[c]) + 8.0 * T->nc,
                     st);
            if (g_split_momentum) {
                auto k1 = c == 0 ? k3t_transport<0, R> : c == 1 ? k3t_transport<1, R> : k3t_transport<2, R>;
                auto k2 = c == 0 ? k3t_momentum_finish<0, R>
                          : c == 1 ? k3t_momentum_finish<1, R>
                                   : k3t_momentum_finish<2, R>;
                const dim3 gt((nx - (c == 0 ? 1 : 0) + 123) / 124, gc[c].y, gc[c].z);  // 4 warps x 31 CVs
                launch_k(k1, gt, 128, 0, st, P, M, W.D[c], W.R3[c]);
                launch_k(k2, gc[c], 128, 0, st, P, M, W.D[c], W.R3[c]);
            } else {
                auto kern = c == 0 ? k3t_momentum<0, R> : c == 1 ? k3t_momentum<1, R> : k3t_momentum<2, R>;
                launch_k(kern, gc[c], 128, 0, st, P, M, W.D[c], W.R3[c]);
            }
        }
        section(6);
        // (6) Crank-Nicolson Jacobi sweeps from u^n with the Dirichlet faces at
        // n+1: edge viscosities of mu^{n+1}, the per-face factors, then the sweeps
        {
            WEC_PROF("tank3_faces_edges", 0, b * 4.0 * T->nc, st);
            launch_k(k3t_edges<R>, gcorner, 128, 0, st, P, (const R *)W.mu1, W.E[0], W.E[1], W.E[2]);
        }
        for (int c = 0; c < 3; ++c) {
            if (c == 1 && ny < 2) continue;
            WEC_PROF("tank3_jprep", c, b * (3.0 * T->nc + 4.0 * nf[c]), st);
            auto kern = c == 0 ? k3t_jprep<0, R> : c == 1 ? k3t_jprep<1, R> : k3t_jprep<2, R>;
            launch_k(kern, gc[c], 128, 0, st, P, (const R *)W.mu1, E, (const R *)W.D[c], W.R3[c], W.Q[c],
                     R(1.0 / (h * h)));
        }
        // the first sweep buffer starts as u^n, both with the Dirichlet faces at
        // n+1 (the sweeps write every solved face, so the second needs no more)
        const R *src[3] = {W.u, W.v, W.w};
        for (int c = 0; c < 3; ++c) {
            WEC_PROF("tank3_jacobi", c, 2.0 * b * nf[c], st);
            launch_k(k3t_copy<R>, nblk((long long)nf[c], 256), 256, 0, st, (long long)nf[c], src[c], W.A[c]);
        }
        {
            const long long nd = std::max({(long long)ny * nz, (long long)nx * nz, (long long)nx * ny});
            launch_k(k3t_dirichlet<R>, nblk(nd, 256), 256, 0, st, P, r_uin1, W.A[0], W.A[1], W.A[2]);
            launch_k(k3t_dirichlet<R>, nblk(nd, 256), 256, 0, st, P, r_uin1, W.B[0], W.B[1], W.B[2]);
        }
        for (int it = 0; it < T->opts.n_jacobi; ++it) {
            const Vel3<R> Va{W.A[0], W.A[1], W.A[2], r_win1};
            for (int c = 0; c < 3; ++c) {
                if (c == 1 && ny < 2) continue;
                // mu, two edge arrays, u, v, w, Rr, Q in; B out
                WEC_PROF("tank3_jacobi", c, b * (3.0 * T->nc + T->nu + T->nv + T->nw + 3.0 * nf[c]), st);
                auto kern = c == 0 ? k3t_jacobi<0, R> : c == 1 ? k3t_jacobi<1, R> : k3t_jacobi<2, R>;
                launch_k(kern, gc[c], 128, 0, st, P, (const R *)W.mu1, E, Va, (const R *)W.R3[c], (const R *)W.Q[c],
                         W.B[c]);
            }
            for (int c = 0; c < 3; ++c) std::swap(W.A[c], W.B[c]);
        }
        section(7);
        // (7) pressure increment: beta = 1 / D, b = -h div u* (FP64), phi from zero
        for (int c = 0; c < 3; ++c)
            launch_k(k3t_beta<R>, gridf(P, c), 128, 0, st, P, c, (const R *)W.D[c], beta[c]);
        if (int e = poisson_build(S, st)) return e;
        launch_k(k3t_rhs<R>, grid3(P), 128, 0, st, P, Vel3<R>{W.A[0], W.A[1], W.A[2], r_win1}, T->rhs);
        WEC_CK(cudaMemsetAsync(T->phi, 0, T->nc * 8, st));
        WEC_CK(cudaGetLastError());
        section(8);
        rc = poisson_solve(S, T->rhs, T->phi, T->opts.rtol, T->opts.max_iters, &iters, &relres);
        if (rc != WEC_OK && rc != WEC_ERR_NOT_CONVERGED) return rc;
        section(9);
        // (8) projection (FP64) and p^{n+1/2,k+1} = p^{n+1/2,k} + phi: into the
        // iterate's velocity, the last cycle into the tank's
        double *dst[3] = {T->u, T->v, T->w};
        if (cyc + 1 < ncyc)
            for (int c = 0; c < 3; ++c) dst[c] = T->uk[c];
        for (int c = 0; c < 3; ++c)
            launch_k(k3t_project<R>, gridf(P, c), 128, 0, st, P, c, (const R *)W.A[c], (const double *)beta[c],
                     (const double *)T->phi, dst[c]);
        launch_k(k3t_add, nblk((long long)T->nc, 256), 256, 0, st, (long long)T->nc, (const double *)T->phi, T->p);
        T->zc = zc1;
    }
    section(10);
    // sigma^{n+1}
    if constexpr (f32)
        launch_k(k3t_widen<R>, nblk((long long)T->nc, 256), 256, 0, st, (long long)T->nc, (const R *)W.tmp, T->sig);
    else
        std::swap(T->sig, T->tmp);
    // diagnostics: ||h div u||, eta at the probe column (x = probe_x, middle y)
    const int G = 1024;
    launch_k(k3t_div2, G, kRT, 0, st, P, Vel3<double>{T->u, T->v, T->w, d_win1}, T->part);
    launch_k(k3t_sum, 1, kRT, 0, st, (const double *)T->part, G, T->part + 3 * nz + 1024 + 1);
    double d2 = 0.0;
    WEC_CK(cudaMemcpyAsync(&d2, T->part + 3 * nz + 1024 + 1, 8, cudaMemcpyDeviceToHost, st));
    const int ip = std::min(std::max((int)std::floor(T->probe_x / h), 0), nx - 1), jp = ny / 2;
    std::vector<double> col(nz);
    WEC_CK(cudaMemcpy2DAsync(col.data(), 8, T->sig + (size_t)jp * nx + ip, (size_t)nx * ny * 8, 8, nz,
                             cudaMemcpyDeviceToHost, st));
    WEC_CK(cudaGetLastError());
    sec.reset();
    WEC_CK(cudaStreamSynchronize(st));
    double eta = std::nan("");
    for (int k = 0; k + 1 < nz; ++k)
        if (col[k] < 0.0 && col[k + 1] >= 0.0) {
            eta = (k + 0.5) * h + h * col[k] / (col[k] - col[k + 1]) - P.depth;
            break;
        }
    T->t = t1;
    T->zc = zc1;
    T->zdot_prev = zd_n;
    T->zdot = zd1;
    if (out) {
        out->t = T->t;
        out->z = T->zc - T->zc0;
        out->zdot = T->zdot;
        out->f_hydro = F;
        out->f_pto = fpto;
        out->eta_probe = eta;
        out->residual = relres;
        out->div_norm = std::sqrt(d2);
        out->iters = iters;
        out->status = rc;
    }
    return rc;
}

namespace wec {
void set_tank3_split_momentum(bool on) { g_split_momentum = on; }
}  // namespace wec

extern "C" {

int wec_tank3_create(const wec_grid3 *grid, const wec_fluids *fl, const wec_waves *wv, const wec_cylinder *body,
                     const wec_solver_opts *opts, void *cuda_stream, wec_tank3 **out)
{
    if (!out) return fail(WEC_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!grid || !fl || !wv || !body) return fail(WEC_ERR_INVALID, "NULL argument");
    const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
    if (nx < 4 || ny < 1 || nz < 4) return fail(WEC_ERR_INVALID, "tank3: need nx >= 4, ny >= 1, nz >= 4");
    if (ny > 65534 || nz > 65534) return fail(WEC_ERR_INVALID, "tank3: ny, nz must be <= 65534");
    const double h = grid->lx / nx;
    if (!(h > 0.0) || std::fabs(grid->ly / ny - h) > 1e-9 * h || std::fabs(grid->lz / nz - h) > 1e-9 * h)
        return fail(WEC_ERR_INVALID, "tank3: the grid must be uniform (lx/nx = ly/ny = lz/nz)");
    if (!(fl->rho_w > 0.0) || !(fl->rho_a > 0.0) || !(fl->mu_w >= 0.0) || !(fl->mu_a >= 0.0))
        return fail(WEC_ERR_INVALID, "tank3: densities must be positive, viscosities non-negative");
    if (wv->ncomp < 0 || (wv->ncomp > 0 && (!wv->amp || !wv->omega || !wv->phase)))
        return fail(WEC_ERR_INVALID, "tank3: wave arrays are NULL");
    if (body->present && (!(body->radius > 0.0) || !(body->length > 0.0) || !(body->mass > 0.0) ||
                          !(body->kappa_p > 0.0) || !(body->added_mass >= 0.0)))
        return fail(WEC_ERR_INVALID, "tank3: the cylinder needs radius, length, mass, kappa_p > 0, added_mass >= 0");
    if (opts) {
        if (opts->precision != WEC_PREC_FP64 && opts->precision != WEC_PREC_MIXED_MG &&
            opts->precision != WEC_PREC_MIXED && opts->precision != WEC_PREC_MIXED_DF)
            return fail(WEC_ERR_INVALID, "tank3: unknown precision");
        if (!(opts->rtol > 0.0) || opts->max_iters < 1 || opts->restart < 1 || opts->restart > kMaxRestart ||
            opts->n_reinit < 0 || opts->n_jacobi < 1 || opts->mg_pre < 1 || opts->mg_pre > 4 || opts->mg_post < 0 ||
            opts->mg_post > 4)
            return fail(WEC_ERR_INVALID, "tank3: invalid solver options");
        if (opts->n_cycles < 0 || opts->n_cycles > 8)
            return fail(WEC_ERR_INVALID, "tank3: n_cycles must be 0..8 (0 and 1: one cycle)");
    }
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
    P.idx32 = (double)(nx + 1) * (ny + 1) * (nz + 1) < 2147483647.0 ? 1 : 0;
    P.rho_s = fl->rho_w;
    if (P.has_body) {
        P.bxc = body->xc; P.byc = body->yc; P.br = body->radius; P.blen = body->length;
        P.rho_s = body->mass / (kPi3 * body->radius * body->radius * body->length);
    }
    T->g = fl->g;
    T->lz = grid->lz;
    T->probe_x = wv->probe_x;
    if (P.has_body) {
        T->kappa_p = body->kappa_p;
        T->mass = body->mass;
        T->added_mass = body->added_mass;
        T->pto_c = body->pto_damping;
        T->zc = T->zc0 = body->zc;
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
    T->hwave.assign(hc.begin(), hc.begin() + 4 * (size_t)P.ncomp);
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
    {  // the constants in both working types, and the damping table in FP32
        P.cd = Tank3C<double>{P.h, P.ih, P.depth, P.rho_w, P.rho_a, P.mu_w, P.mu_a, P.rho_s, P.bxc, P.byc, P.br, P.blen};
        P.cf = Tank3C<float>{(float)P.h, (float)P.ih, (float)P.depth, (float)P.rho_w, (float)P.rho_a, (float)P.mu_w,
                             (float)P.mu_a, (float)P.rho_s, (float)P.bxc, (float)P.byc, (float)P.br, (float)P.blen};
        P.cdf = Tank3C<df64>{df64(P.h), df64(P.ih), df64(P.depth), df64(P.rho_w), df64(P.rho_a), df64(P.mu_w),
                             df64(P.mu_a), df64(P.rho_s), df64(P.bxc), df64(P.byc), df64(P.br), df64(P.blen)};
        std::vector<float> df(nx);
        std::vector<df64> dd(nx);
        for (int i = 0; i < nx; ++i) {
            df[i] = (float)hc[4 * (size_t)P.ncomp + i];
            dd[i] = df64(hc[4 * (size_t)P.ncomp + i]);
        }
        e = cudaMalloc(&T->fconsts, (size_t)nx * 4);
        if (e == cudaSuccess) e = cudaMemcpy(T->fconsts, df.data(), (size_t)nx * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&T->dconsts, (size_t)nx * sizeof(df64));
        if (e == cudaSuccess) e = cudaMemcpy(T->dconsts, dd.data(), (size_t)nx * sizeof(df64), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            wec_tank3_destroy(T);
            return cuda_fail(e, "tank3 allocation");
        }
        P.dampf = T->fconsts;
        P.dampd = T->dconsts;
    }
    if (opts) {  // the step: its buffers, its solver, the initial state
        T->opts = *opts;
        T->stepping = true;
        size_t nf[3] = {T->nu, T->nv, T->nw};
        for (double **q : {&T->p, &T->phi, &T->rhs, &T->mu1, &T->rf1, &T->chi1})
            if (e == cudaSuccess) e = cudaMalloc(q, T->nc * 8);
        for (int c = 0; c < 3; ++c)
            for (double **q : {&T->D[c], &T->R[c], &T->A[c], &T->B[c], &T->RF[c], &T->Q[c]})
                if (e == cudaSuccess) e = cudaMalloc(q, nf[c] * 8);
        const size_t ne[3] = {(size_t)nz * (ny + 1) * (nx + 1), (size_t)(nz + 1) * ny * (nx + 1),
                              (size_t)(nz + 1) * (ny + 1) * nx};
        const bool f64_stencils = opts->precision == WEC_PREC_FP64 || opts->precision == WEC_PREC_MIXED_MG;
        if (f64_stencils)
            for (int c = 0; c < 3; ++c)
                if (e == cudaSuccess) e = cudaMalloc(&T->E[c], ne[c] * 8);
        if (opts->n_cycles > 1) {  // the iterate's velocity and its force's viscosity (+ FP64 means)
            for (int c = 0; c < 3; ++c)
                if (e == cudaSuccess) e = cudaMalloc(&T->uk[c], nf[c] * 8);
            if (e == cudaSuccess) e = cudaMalloc(&T->muk, T->nc * 8);
            if (f64_stencils) {
                if (e == cudaSuccess) e = cudaMalloc(&T->sh, T->nc * 8);
                for (int c = 0; c < 3; ++c)
                    if (e == cudaSuccess) e = cudaMalloc(&T->uh[c], nf[c] * 8);
            }
        }
        if (e == cudaSuccess) e = cudaMalloc(&T->bc, (size_t)(6 * nz + 4) * 8);
        if (e == cudaSuccess) e = cudaMalloc(&T->tabs, (size_t)(nx + 1) * 8);
        if (e == cudaSuccess) e = cudaMalloc(&T->part, (size_t)(3 * nz + 1024 + 8) * 8);
        if (e != cudaSuccess) {
            wec_tank3_destroy(T);
            return cuda_fail(e, "tank3 step allocation");
        }
        T->solver = new (std::nothrow) wec_poisson();
        if (!T->solver) {
            wec_tank3_destroy(T);
            return fail(WEC_ERR_NOMEM, "host allocation failed");
        }
        // FP32 V-cycles; the double-float path also runs the Arnoldi step in float pairs
        const int sprec = opts->precision == WEC_PREC_FP64      ? WEC_PREC_FP64
                          : opts->precision == WEC_PREC_MIXED_DF ? WEC_PREC_MIXED_DF
                                                                 : WEC_PREC_MIXED;
        if (int rc = poisson_init(T->solver, nx, ny, sprec, opts->restart, opts->mg_pre, opts->mg_post, T->st, nz)) {
            std::string msg = wec_last_error();
            wec_tank3_destroy(T);
            return fail(rc, msg);
        }
        // damping weight at the u-faces (x = i h)
        std::vector<double> du(nx + 1);
        for (int i = 0; i <= nx; ++i) {
            const double x = i * h;
            double a = 0.0;
            if (wv->damp_len > 0.0 && x > wv->damp_x0) {
                double xi = (x - wv->damp_x0) / wv->damp_len;
                if (xi > 1.0) xi = 1.0;
                a = (std::exp(std::pow(xi, 3.5)) - 1.0) / (std::exp(1.0) - 1.0);
            }
            du[i] = a;
        }
        // initial state: sigma = z - depth - eta(x, 0), Airy u and w (v = 0), p the
        // discrete hydrostatic pressure of rho^flow from the top face (p = 0 there)
        const Waves3 W{P.ncomp, hc.data(), hc.data() + P.ncomp, hc.data() + 2 * P.ncomp, hc.data() + 3 * P.ncomp};
        std::vector<double> eta(nx), uxz((size_t)nz * (nx + 1)), wxz((size_t)(nz + 1) * nx, 0.0);
        for (int i = 0; i < nx; ++i) eta[i] = eta_host(W, (i + 0.5) * h, 0.0);
        for (int k = 0; k < nz; ++k)
            for (int i = 0; i <= nx; ++i) {
                double uu, ww;
                airy_host(W, grid->depth, h, i * h, (k + 0.5) * h, 0.0, &uu, &ww);
                uxz[(size_t)k * (nx + 1) + i] = i == nx ? 0.0 : uu;
            }
        for (int k = 1; k <= nz; ++k)
            for (int i = 0; i < nx; ++i) {
                double uu, ww;
                airy_host(W, grid->depth, h, (i + 0.5) * h, k * h, 0.0, &uu, &ww);
                wxz[(size_t)k * nx + i] = ww;
            }
        double *dtab = nullptr;
        e = cudaMalloc(&dtab, (eta.size() + uxz.size() + wxz.size()) * 8);
        if (e == cudaSuccess) e = cudaMemcpy(dtab, eta.data(), eta.size() * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dtab + eta.size(), uxz.data(), uxz.size() * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(dtab + eta.size() + uxz.size(), wxz.data(), wxz.size() * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(T->tabs, du.data(), du.size() * 8, cudaMemcpyHostToDevice);
        // working copies of the stencils: FP32 (WEC_PREC_MIXED) or float pairs (WEC_PREC_MIXED_DF)
        auto alloc_work = [&](auto &F) {
            using RW = std::remove_pointer_t<decltype(F.sig)>;
            const size_t b = sizeof(RW);
            for (RW **q : std::initializer_list<RW **>{&F.sig, &F.tmp, &F.s0, &F.s1, &F.rho, &F.mu, &F.rf, &F.chi,
                                                       &F.mu1, &F.rf1, &F.chi1})
                if (e == cudaSuccess) e = cudaMalloc(q, T->nc * b);
            const size_t nf3[3] = {T->nu, T->nv, T->nw};
            if (e == cudaSuccess) e = cudaMalloc(&F.u, T->nu * b);
            if (e == cudaSuccess) e = cudaMalloc(&F.v, T->nv * b);
            if (e == cudaSuccess) e = cudaMalloc(&F.w, T->nw * b);
            for (int c = 0; c < 3; ++c)
                for (RW **q : std::initializer_list<RW **>{&F.D[c], &F.R3[c], &F.A[c], &F.B[c], &F.RF[c], &F.Q[c]})
                    if (e == cudaSuccess) e = cudaMalloc(q, nf3[c] * b);
            for (int c = 0; c < 3; ++c)
                if (e == cudaSuccess) e = cudaMalloc(&F.E[c], ne[c] * b);
            if (opts->n_cycles > 1) {  // the means of levels n and n+1,k
                if (e == cudaSuccess) e = cudaMalloc(&F.sh, T->nc * b);
                for (int c = 0; c < 3; ++c)
                    if (e == cudaSuccess) e = cudaMalloc(&F.uh[c], nf3[c] * b);
            }
            if (e == cudaSuccess) e = cudaMalloc(&F.bc, (size_t)(6 * nz + 4) * b);
            if (e == cudaSuccess) e = cudaMalloc(&F.dampu, (size_t)(nx + 1) * b);
            std::vector<RW> duw;
            for (double x : du) duw.push_back(RW(x));
            if (e == cudaSuccess) e = cudaMemcpy(F.dampu, duw.data(), duw.size() * b, cudaMemcpyHostToDevice);
        };
        if (e == cudaSuccess && opts->precision == WEC_PREC_MIXED) alloc_work(T->wf);
        if (e == cudaSuccess && opts->precision == WEC_PREC_MIXED_DF) alloc_work(T->wd);
        if (e != cudaSuccess) {
            cudaFree(dtab);
            wec_tank3_destroy(T);
            return cuda_fail(e, "tank3 initial state");
        }
        launch_k(k3t_init, dim3((nx + 128) / 128, ny, nz), 128, 0, T->st, T->P, (const double *)dtab,
                 (const double *)(dtab + eta.size()), (const double *)(dtab + eta.size() + uxz.size()), T->sig, T->u,
                 T->w);
        launch_k(k3t_materials<double>, grid3(T->P), 128, 0, T->st, T->P, (const double *)T->sig, T->zc, T->rho,
                 T->mu, T->rhof, T->chi, 0, 0, 0);
        launch_k(k3t_hydrostatic, nblk((long long)nx * ny, 128), 128, 0, T->st, T->P, (const double *)T->rhof, T->g,
                 T->p);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(T->st);
        cudaFree(dtab);
        if (e != cudaSuccess) {
            wec_tank3_destroy(T);
            return cuda_fail(e, "tank3 initial state");
        }
    }
    *out = T;
    return WEC_OK;
}

void wec_tank3_destroy(wec_tank3 *T)
{
    if (!T) return;
    cudaStreamSynchronize(T->st);
    for (double *p : {T->sig, T->tmp, T->s0, T->s1, T->rho, T->mu, T->rhof, T->chi, T->u, T->v, T->w, T->consts,
                      T->p, T->phi, T->rhs, T->mu1, T->rf1, T->chi1, T->bc, T->tabs, T->part})
        cudaFree(p);
    for (int c = 0; c < 3; ++c)
        for (double *p : {T->D[c], T->R[c], T->A[c], T->B[c], T->E[c], T->RF[c], T->Q[c], T->uk[c], T->uh[c]})
            cudaFree(p);
    cudaFree(T->muk);
    cudaFree(T->sh);
    auto free_work = [](auto &F) {
        using RW = std::remove_pointer_t<decltype(F.sig)>;
        for (RW *p : std::initializer_list<RW *>{F.sig, F.tmp, F.s0, F.s1, F.u, F.v, F.w, F.rho, F.mu, F.rf, F.chi,
                                                 F.mu1, F.rf1, F.chi1, F.bc, F.dampu, F.sh, F.uh[0], F.uh[1], F.uh[2]})
            cudaFree(p);
        for (int c = 0; c < 3; ++c)
            for (RW *p : std::initializer_list<RW *>{F.D[c], F.R3[c], F.A[c], F.B[c], F.E[c], F.RF[c], F.Q[c]})
                cudaFree(p);
    };
    free_work(T->wf);
    free_work(T->wd);
    cudaFree(T->fconsts);
    cudaFree(T->dconsts);
    if (T->solver) {
        poisson_free(T->solver);
        delete T->solver;
    }
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
    case WEC_F3_P: *n = T->p ? T->nc : 0; return T->p;
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
    if (!p || !host || n != m || (f > WEC_F3_W && f != WEC_F3_P))
        return fail(WEC_ERR_INVALID, "tank3_set_field: not a state field or wrong size");
    WEC_CK(cudaStreamSynchronize(T->st));
    WEC_CK(cudaMemcpy(p, host, m * 8, cudaMemcpyHostToDevice));
    return WEC_OK;
}

int wec_tank3_materials(wec_tank3 *T, double zc)
{
    if (int e = tank3_check(T)) return e;
    {
        WEC_PROF("tank3_materials", 0, 40.0 * T->nc, T->st);
        launch_k(k3t_materials<double>, grid3(T->P), 128, 0, T->st, T->P, (const double *)T->sig, zc, T->rho, T->mu, T->rhof,
                 T->chi, 0, 0, 0);
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
        // the face values in stream-ordered scratch (a level-set tank has no step buffers)
        const size_t nfa[3] = {T->nu, T->nv, T->nw};
        double *F = nullptr;
        WEC_CK(cudaMallocAsync(&F, (nfa[0] + nfa[1] + nfa[2]) * 8, T->st));
        double *const Fs[3] = {F, F + nfa[0], F + nfa[0] + nfa[1]};
        advect3<double>(T->P, nfa, (const double *)T->sig, (const double *)T->sig,
                        Vel3<double>{T->u, T->v, T->w, nullptr}, dt, ghost_at(T, t), Fs, T->tmp, T->st);
        WEC_CK(cudaFreeAsync(F, T->st));
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
    if (int e = reinit_buf<double>(T, T->sig, T->s0, T->s1, nit, t)) return e;
    WEC_CK(cudaStreamSynchronize(T->st));
    return WEC_OK;
}

int wec_tank3_get_state(const wec_tank3 *T, double *out5)
{
    if (int e = tank3_check(T)) return e;
    if (!out5) return fail(WEC_ERR_INVALID, "NULL argument");
    out5[0] = T->t;
    out5[1] = T->zc;
    out5[2] = T->zdot;
    out5[3] = T->zc0;
    out5[4] = T->zdot_prev;
    return WEC_OK;
}

int wec_tank3_step(wec_tank3 *T, double dt, double pto_force, wec_step_result *out)
{
    if (int e = tank3_check(T)) return e;
    if (!T->stepping) return fail(WEC_ERR_INVALID, "tank3_step: the tank was created without solver options");
    if (!(dt > 0.0)) return fail(WEC_ERR_INVALID, "tank3_step: dt must be > 0");
    if (T->opts.precision == WEC_PREC_MIXED) return tank3_step_impl<float>(T, T->wf, dt, pto_force, out);
    if (T->opts.precision == WEC_PREC_MIXED_DF) return tank3_step_impl<df64>(T, T->wd, dt, pto_force, out);
    Work3<double> W;
    W.sig = T->sig; W.tmp = T->tmp; W.s0 = T->s0; W.s1 = T->s1; W.u = T->u; W.v = T->v; W.w = T->w;
    W.rho = T->rho; W.mu = T->mu; W.rf = T->rhof; W.chi = T->chi; W.mu1 = T->mu1; W.rf1 = T->rf1; W.chi1 = T->chi1;
    for (int c = 0; c < 3; ++c) {
        W.D[c] = T->D[c]; W.R3[c] = T->R[c]; W.A[c] = T->A[c]; W.B[c] = T->B[c];
        W.E[c] = T->E[c]; W.RF[c] = T->RF[c]; W.Q[c] = T->Q[c]; W.uh[c] = T->uh[c];
    }
    W.sh = T->sh;
    W.bc = T->bc;
    W.dampu = T->tabs;
    const int rc = tank3_step_impl<double>(T, W, dt, pto_force, out);
    for (int c = 0; c < 3; ++c) {  // the Jacobi ping-pong swapped the buffers
        T->A[c] = W.A[c]; T->B[c] = W.B[c];
    }
    return rc;
}

}  // extern "C"
