// Pressure solver: FGMRES(m) right-preconditioned by one geometric multigrid
// V-cycle, for the variable-coefficient pressure equation of the projection
// (Eq. c_discrete_continuity; the paper leaves the solver to PETSc and does
// not name it -- this is the solver the library specifies).
//
// Operator on an nx x ny cell grid: (A p)_c = sum_f beta_f (p_c - p_nb), the
// left/right/bottom walls Neumann, the top face Dirichlet p = 0 (ghost -p_c).
// Multigrid: red-black Gauss-Seidel, sum-of-four restriction of the residual,
// piecewise-constant prolongation, coarse face coefficient = mean of the two
// fine faces it covers, dense LU on the coarsest level (<= 512 cells).
// Mixed precision: the V-cycle runs in FP32 on FP32 copies of the hierarchy;
// the Krylov basis, Hessenberg, residuals and the solution stay FP64.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "internal.cuh"

namespace wec {
namespace {

// ------------------------------------------------------------ stencil ----
template <typename T>
__device__ __forceinline__ T diag_at(const T *bu, const T *bv, int nx, int ny, int i, int j)
{
    T d = T(0);
    if (i > 0) d += bu[j * (nx + 1) + i];
    if (i < nx - 1) d += bu[j * (nx + 1) + i + 1];
    if (j > 0) d += bv[j * nx + i];
    d += (j < ny - 1 ? T(1) : T(2)) * bv[(j + 1) * nx + i];
    return d;
}

template <typename T, typename TX>
__device__ __forceinline__ T offsum_at(const T *bu, const T *bv, const TX *x, int nx, int ny, int i,
                                       int j)
{
    int c = j * nx + i;
    T s = T(0);
    if (i > 0) s += bu[j * (nx + 1) + i] * T(x[c - 1]);
    if (i < nx - 1) s += bu[j * (nx + 1) + i + 1] * T(x[c + 1]);
    if (j > 0) s += bv[j * nx + i] * T(x[c - nx]);
    if (j < ny - 1) s += bv[(j + 1) * nx + i] * T(x[c + nx]);
    return s;
}

// y = A x (FP64 operator; x may be FP32 storage of a preconditioned vector)
template <typename TX>
__global__ void k_apply(int nx, int ny, const double *__restrict__ bu, const double *__restrict__ bv,
                        const TX *__restrict__ x, double *__restrict__ y)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx * ny) return;
    int i = c % nx, j = c / nx;
    double d = diag_at(bu, bv, nx, ny, i, j);
    y[c] = d * double(x[c]) - offsum_at(bu, bv, x, nx, ny, i, j);
}

// w = b - A x
__global__ void k_residual(int nx, int ny, const double *__restrict__ bu, const double *__restrict__ bv,
                           const double *__restrict__ x, const double *__restrict__ b, double *__restrict__ w)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx * ny) return;
    int i = c % nx, j = c / nx;
    double d = diag_at(bu, bv, nx, ny, i, j);
    double ax = d * x[c] - offsum_at(bu, bv, x, nx, ny, i, j);
    w[c] = b[c] - ax;
}

// One colour of a red-black Gauss-Seidel sweep; thread k -> k-th cell of the
// colour (nx even on every smoothed level).  first != 0: the sweep starts from
// x = 0, so the red pass writes b / d and zeroes the black cells.
template <typename T>
__global__ void k_rbgs(int nx, int ny, const T *__restrict__ bu, const T *__restrict__ bv, T *x,
                       const T *__restrict__ b, int color, int first)
{
    int half = nx >> 1;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= half * ny) return;
    int j = k / half;
    int i = 2 * (k - j * half) + ((j & 1) ^ color);
    int c = j * nx + i;
    T d = diag_at(bu, bv, nx, ny, i, j);
    if (first) {
        x[c] = (b[c] + T(0)) / d;
        x[c + (i & 1 ? -1 : 1)] = T(0);  // the black neighbour in the same row
        return;
    }
    x[c] = (b[c] + offsum_at(bu, bv, x, nx, ny, i, j)) / d;
}

// Coarse right-hand side = sum of the residuals of the four children.
template <typename T>
__global__ void k_resid_restrict(int nx, int ny, const T *__restrict__ bu, const T *__restrict__ bv,
                                 const T *__restrict__ x, const T *__restrict__ b, T *__restrict__ bc)
{
    int ncx = nx >> 1, ncy = ny >> 1;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncx * ncy) return;
    int I = k % ncx, J = k / ncx;
    T r[4];
    int q = 0;
    for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
            int i = 2 * I + di, j = 2 * J + dj, c = j * nx + i;
            T d = diag_at(bu, bv, nx, ny, i, j);
            T ax = d * x[c] - offsum_at(bu, bv, x, nx, ny, i, j);
            r[q++] = b[c] - ax;
        }
    bc[k] = ((r[0] + r[1]) + r[2]) + r[3];
}

template <typename T>
__global__ void k_prolong(int nx, int ny, T *__restrict__ x, const T *__restrict__ xc)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx * ny) return;
    int i = c % nx, j = c / nx;
    x[c] += xc[(j >> 1) * (nx >> 1) + (i >> 1)];
}

template <typename T>
__global__ void k_coarsen(int nx, int ny, const T *__restrict__ fu, const T *__restrict__ fv,
                          T *__restrict__ cu, T *__restrict__ cv)
{
    int ncx = nx >> 1, ncy = ny >> 1;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int nu = (ncx + 1) * ncy, nv = ncx * (ncy + 1);
    if (k < nu) {
        int I = k % (ncx + 1), J = k / (ncx + 1);
        cu[k] = T(0.5) * (fu[(2 * J) * (nx + 1) + 2 * I] + fu[(2 * J + 1) * (nx + 1) + 2 * I]);
    } else if (k < nu + nv) {
        int q = k - nu;
        int I = q % ncx, J = q / ncx;
        cv[q] = T(0.5) * (fv[(2 * J) * nx + 2 * I] + fv[(2 * J) * nx + 2 * I + 1]);
    }
}

template <typename TO, typename TI>
__global__ void k_convert(long long n, const TI *__restrict__ in, TO *__restrict__ out)
{
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c < n) out[c] = TO(in[c]);
}

// Dense LU of the coarsest operator (no pivoting: A is a symmetric M-matrix).
// One block; the matrix lives in global memory (n <= 512).
template <typename T>
__global__ void k_lu_factor(int nx, int ny, const T *__restrict__ bu, const T *__restrict__ bv, T *A)
{
    int n = nx * ny;
    for (long long q = threadIdx.x; q < (long long)n * n; q += blockDim.x) A[q] = T(0);
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        int i = r % nx, j = r / nx;
        A[(long long)r * n + r] = diag_at(bu, bv, nx, ny, i, j);
        if (i > 0) A[(long long)r * n + r - 1] = -bu[j * (nx + 1) + i];
        if (i < nx - 1) A[(long long)r * n + r + 1] = -bu[j * (nx + 1) + i + 1];
        if (j > 0) A[(long long)r * n + r - nx] = -bv[j * nx + i];
        if (j < ny - 1) A[(long long)r * n + r + nx] = -bv[(j + 1) * nx + i];
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        T piv = A[(long long)k * n + k];
        for (int r = k + 1 + threadIdx.x; r < n; r += blockDim.x) {
            T f = A[(long long)r * n + k] / piv;
            A[(long long)r * n + k] = f;
            for (int c = k + 1; c < n; ++c) A[(long long)r * n + c] -= f * A[(long long)k * n + c];
        }
        __syncthreads();
    }
}

// x = U^{-1} L^{-1} b, one warp.
template <typename T>
__global__ void k_lu_solve(int n, const T *__restrict__ A, const T *__restrict__ b, T *__restrict__ x)
{
    int lane = threadIdx.x;
    for (int r = 0; r < n; ++r) {
        T s = T(0);
        for (int c = lane; c < r; c += 32) s += A[(long long)r * n + c] * x[c];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x[r] = b[r] - s;
        __syncwarp();
    }
    for (int r = n - 1; r >= 0; --r) {
        T s = T(0);
        for (int c = r + 1 + lane; c < n; c += 32) s += A[(long long)r * n + c] * x[c];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x[r] = (x[r] - s) / A[(long long)r * n + r];
        __syncwarp();
    }
}

// ---------------------------------------------------------- reductions ----
__device__ __forceinline__ double block_sum(double v, double *sh)
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

// part[k * kRedBlocks + b] = partial sum of V_k . w over block b's elements
__global__ void k_dots_partial(int n, const double *__restrict__ V, const double *__restrict__ w,
                               double *__restrict__ part)
{
    __shared__ double sh[kRedThreads];
    int k = blockIdx.y;
    const double *vk = V + (long long)k * n;
    double s = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) s += vk[c] * w[c];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[k * kRedBlocks + blockIdx.x] = s;
}

__global__ void k_dots_final(const double *__restrict__ part, double *__restrict__ out)
{
    __shared__ double sh[kRedThreads];
    int k = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < kRedBlocks; b += blockDim.x) s += part[k * kRedBlocks + b];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[k] = s;
}

// w -= sum_k h[k] V_k
__global__ void k_axpy_multi(int n, int nvec, const double *__restrict__ V, const double *__restrict__ hcoef,
                             double *__restrict__ w)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double a = w[c];
    for (int k = 0; k < nvec; ++k) a -= hcoef[k] * V[(long long)k * n + c];
    w[c] = a;
}

__global__ void k_scale_div(int n, const double *__restrict__ w, const double *__restrict__ s,
                            double *__restrict__ out)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) out[c] = w[c] / s[0];
}

__global__ void k_sqrt(double *a) { a[0] = sqrt(a[0]); }

// Column j of the Hessenberg matrix from the two Gram-Schmidt passes, Givens
// rotations, residual estimate.  scal[2] = |g_{j+1}|, scal[3] = h_{j+1,j}.
__global__ void k_givens(int j, int m, const double *__restrict__ h1, const double *__restrict__ h2,
                         const double *__restrict__ hn2, double *H, double *cs, double *sn, double *g,
                         double *scal)
{
    for (int k = 0; k <= j; ++k) H[k * m + j] = (0.0 + h1[k]) + h2[k];
    double hn = sqrt(hn2[0]);
    H[(j + 1) * m + j] = hn;
    for (int k = 0; k < j; ++k) {
        double a = H[k * m + j], b = H[(k + 1) * m + j];
        H[k * m + j] = cs[k] * a + sn[k] * b;
        H[(k + 1) * m + j] = -sn[k] * a + cs[k] * b;
    }
    double a = H[j * m + j], b = H[(j + 1) * m + j];
    double den = sqrt(a * a + b * b);
    cs[j] = a / den;
    sn[j] = b / den;
    H[j * m + j] = den;
    H[(j + 1) * m + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    scal[2] = fabs(g[j + 1]);
    scal[3] = hn;
}

__global__ void k_cycle_init(int m, const double *beta, double *g)
{
    for (int k = 0; k <= m; ++k) g[k] = 0.0;
    g[0] = beta[0];
}

__global__ void k_backsolve(int jd, int m, const double *__restrict__ H, const double *__restrict__ g,
                            double *__restrict__ y)
{
    for (int k = jd - 1; k >= 0; --k) {
        double s = g[k];
        for (int l = k + 1; l < jd; ++l) s -= H[k * m + l] * y[l];
        y[k] = s / H[k * m + k];
    }
}

template <typename TZ>
__global__ void k_update_x(int n, int jd, const double *__restrict__ y, const TZ *__restrict__ Z,
                           double *__restrict__ x)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double a = x[c];
    for (int k = 0; k < jd; ++k) a += y[k] * double(Z[(long long)k * n + c]);
    x[c] = a;
}

// ------------------------------------------------------------ V-cycle ----
template <typename T>
void vcycle_t(wec_poisson *P, Level<T> *L, const T *b0, T *x0)
{
    cudaStream_t st = P->st;
    const int TB = 256;
    const double ts = sizeof(T);
    for (int l = 0; l < P->nlev; ++l) {
        Level<T> &A = L[l];
        const T *b = l == 0 ? b0 : A.b;
        T *x = l == 0 ? x0 : A.x;
        const double n = (double)A.nx * A.ny, nf = (double)(A.nx + 1) * A.ny + (double)A.nx * (A.ny + 1);
        if (l == P->nlev - 1) {
            T *lu = nullptr;
            if constexpr (sizeof(T) == 8) lu = (T *)P->lu64; else lu = (T *)P->lu32;
            WEC_PROF("mg_lu_solve", l, (n * n + 2 * n) * ts, st);
            k_lu_solve<T><<<1, 32, 0, st>>>(A.nx * A.ny, lu, b, x);
            break;
        }
        int nh = (A.nx >> 1) * A.ny;
        for (int s = 0; s < P->nu1; ++s) {
            {
                WEC_PROF("mg_rbgs", l, (1.5 * n + nf) * ts, st);
                k_rbgs<T><<<nblk(nh, TB), TB, 0, st>>>(A.nx, A.ny, A.bu, A.bv, x, b, 0, s == 0);
            }
            {
                WEC_PROF("mg_rbgs", l, (1.5 * n + nf) * ts, st);
                k_rbgs<T><<<nblk(nh, TB), TB, 0, st>>>(A.nx, A.ny, A.bu, A.bv, x, b, 1, 0);
            }
        }
        if (P->nu1 == 0) cudaMemsetAsync(x, 0, sizeof(T) * A.nx * A.ny, st);
        Level<T> &C = L[l + 1];
        WEC_PROF("mg_resid_restrict", l, (2.25 * n + nf) * ts, st);
        k_resid_restrict<T><<<nblk(C.nx * C.ny, TB), TB, 0, st>>>(A.nx, A.ny, A.bu, A.bv, x, b, C.b);
    }
    for (int l = P->nlev - 2; l >= 0; --l) {
        Level<T> &A = L[l];
        const T *b = l == 0 ? b0 : A.b;
        T *x = l == 0 ? x0 : A.x;
        const double n = (double)A.nx * A.ny, nf = (double)(A.nx + 1) * A.ny + (double)A.nx * (A.ny + 1);
        int nh = (A.nx >> 1) * A.ny;
        {
            WEC_PROF("mg_prolong", l, 2.25 * n * ts, st);
            k_prolong<T><<<nblk(A.nx * A.ny, TB), TB, 0, st>>>(A.nx, A.ny, x, L[l + 1].x);
        }
        for (int s = 0; s < P->nu2; ++s) {
            {
                WEC_PROF("mg_rbgs", l, (1.5 * n + nf) * ts, st);
                k_rbgs<T><<<nblk(nh, TB), TB, 0, st>>>(A.nx, A.ny, A.bu, A.bv, x, b, 0, 0);
            }
            {
                WEC_PROF("mg_rbgs", l, (1.5 * n + nf) * ts, st);
                k_rbgs<T><<<nblk(nh, TB), TB, 0, st>>>(A.nx, A.ny, A.bu, A.bv, x, b, 1, 0);
            }
        }
    }
}

// z = M^{-1} v for the FGMRES basis vector v (FP64); z in the object's precision.
void precond(wec_poisson *P, const double *v, void *z)
{
    int n = P->nx * P->ny;
    if (P->prec == WEC_PREC_FP64) {
        vcycle_t<double>(P, P->L64, v, (double *)z);
    } else {
        {
            WEC_PROF("convert", -1, 12.0 * n, P->st);
            k_convert<float, double><<<nblk(n, 256), 256, 0, P->st>>>(n, v, P->L32[0].b);
        }
        vcycle_t<float>(P, P->L32, P->L32[0].b, (float *)z);
    }
}

int read_scal(wec_poisson *P, int count)
{
    WEC_CK(cudaMemcpyAsync(P->host, P->scal, sizeof(double) * count, cudaMemcpyDeviceToHost, P->st));
    WEC_CK(cudaStreamSynchronize(P->st));
    return WEC_OK;
}

void dots(wec_poisson *P, const double *V, int nvec, const double *w, double *out)
{
    int n = P->nx * P->ny;
    dim3 grid(kRedBlocks, nvec);
    {
        WEC_PROF("krylov_dots", -1, 8.0 * n * (nvec + 1), P->st);
        k_dots_partial<<<grid, kRedThreads, 0, P->st>>>(n, V, w, P->part);
    }
    WEC_PROF("reduce_final", -1, 8.0 * nvec * (kRedBlocks + 1), P->st);
    k_dots_final<<<nvec, kRedThreads, 0, P->st>>>(P->part, out);
}

}  // namespace

void launch_norm2(const double *a, int n, double *part, double *out, cudaStream_t st)
{
    dim3 grid(kRedBlocks, 1);
    {
        WEC_PROF("krylov_dots", -1, 8.0 * n, st);
        k_dots_partial<<<grid, kRedThreads, 0, st>>>(n, a, a, part);
    }
    {
        WEC_PROF("reduce_final", -1, 8.0 * (kRedBlocks + 1), st);
        k_dots_final<<<1, kRedThreads, 0, st>>>(part, out);
    }
    WEC_PROF("scalar", -1, 16.0, st);
    k_sqrt<<<1, 1, 0, st>>>(out);
}

int poisson_init(wec_poisson *P, int nx, int ny, int prec, int restart, int nu1, int nu2, cudaStream_t st)
{
    if (nx < 2 || ny < 2) return fail(WEC_ERR_INVALID, "poisson: nx, ny must be >= 2");
    if (restart < 1 || restart > kMaxRestart) return fail(WEC_ERR_INVALID, "poisson: restart must be in 1..32");
    if (nu1 < 0 || nu2 < 0 || nu1 + nu2 == 0) return fail(WEC_ERR_INVALID, "poisson: need at least one smoothing sweep");
    if (prec != WEC_PREC_FP64 && prec != WEC_PREC_MIXED) return fail(WEC_ERR_INVALID, "poisson: unknown precision");
    P->nx = nx; P->ny = ny; P->prec = prec; P->restart = restart; P->nu1 = nu1; P->nu2 = nu2; P->st = st;
    // levels: coarsen while both sizes are even and >= 4
    int lx = nx, ly = ny, nl = 0;
    for (;;) {
        P->L64[nl].nx = lx; P->L64[nl].ny = ly;
        P->L32[nl].nx = lx; P->L32[nl].ny = ly;
        nl++;
        if ((lx & 1) || (ly & 1) || lx < 4 || ly < 4 || nl == kMaxLevels) break;
        lx >>= 1; ly >>= 1;
    }
    P->nlev = nl;
    P->ncoarse = lx * ly;
    if (P->ncoarse > kMaxCoarse)
        return fail(WEC_ERR_INVALID, "poisson: the grid must coarsen (by halving even sizes) to at most 512 cells; got " +
                                         std::to_string(lx) + "x" + std::to_string(ly));
    for (int l = 0; l < nl; ++l) {
        size_t nc = (size_t)P->L64[l].nx * P->L64[l].ny;
        size_t nu = (size_t)(P->L64[l].nx + 1) * P->L64[l].ny, nv = (size_t)P->L64[l].nx * (P->L64[l].ny + 1);
        WEC_CK(cudaMalloc(&P->L64[l].bu, nu * 8));
        WEC_CK(cudaMalloc(&P->L64[l].bv, nv * 8));
        WEC_CK(cudaMemset(P->L64[l].bu, 0, nu * 8));
        WEC_CK(cudaMemset(P->L64[l].bv, 0, nv * 8));
        if (l > 0) {
            WEC_CK(cudaMalloc(&P->L64[l].x, nc * 8));
            WEC_CK(cudaMalloc(&P->L64[l].b, nc * 8));
        }
        P->bytes += (nu + nv) * 8 + (l > 0 ? 2 * nc * 8 : 0);
        if (prec == WEC_PREC_MIXED) {
            WEC_CK(cudaMalloc(&P->L32[l].bu, nu * 4));
            WEC_CK(cudaMalloc(&P->L32[l].bv, nv * 4));
            WEC_CK(cudaMalloc(&P->L32[l].x, nc * 4));
            WEC_CK(cudaMalloc(&P->L32[l].b, nc * 4));
            P->bytes += (nu + nv + 2 * nc) * 4;
        }
    }
    WEC_CK(cudaMalloc(&P->lu64, (size_t)P->ncoarse * P->ncoarse * 8));
    if (prec == WEC_PREC_MIXED) WEC_CK(cudaMalloc(&P->lu32, (size_t)P->ncoarse * P->ncoarse * 4));
    size_t n = (size_t)nx * ny;
    int m = restart;
    WEC_CK(cudaMalloc(&P->V, (m + 1) * n * 8));
    WEC_CK(cudaMalloc(&P->Z, m * n * (prec == WEC_PREC_FP64 ? 8 : 4)));
    WEC_CK(cudaMalloc(&P->w, n * 8));
    WEC_CK(cudaMalloc(&P->part, (size_t)(kMaxRestart + 1) * kRedBlocks * 8));
    WEC_CK(cudaMalloc(&P->dots, 3 * (kMaxRestart + 2) * 8));
    size_t nh = (size_t)(m + 1) * m + 3 * (m + 1) + m + 8;
    WEC_CK(cudaMalloc(&P->hess, nh * 8));
    WEC_CK(cudaMemset(P->hess, 0, nh * 8));
    P->cs = P->hess + (m + 1) * m;
    P->sn = P->cs + (m + 1);
    P->g = P->sn + (m + 1);
    P->y = P->g + (m + 1);
    P->scal = P->y + m;
    WEC_CK(cudaMallocHost(&P->host, 8 * 8));
    P->bytes += ((m + 1) * n + n) * 8 + m * n * (prec == WEC_PREC_FP64 ? 8 : 4);
    return WEC_OK;
}

void poisson_free(wec_poisson *P)
{
    for (int l = 0; l < P->nlev; ++l) {
        cudaFree(P->L64[l].bu); cudaFree(P->L64[l].bv); cudaFree(P->L64[l].x); cudaFree(P->L64[l].b);
        cudaFree(P->L32[l].bu); cudaFree(P->L32[l].bv); cudaFree(P->L32[l].x); cudaFree(P->L32[l].b);
    }
    cudaFree(P->lu64); cudaFree(P->lu32);
    cudaFree(P->V); cudaFree(P->Z); cudaFree(P->w); cudaFree(P->part); cudaFree(P->dots); cudaFree(P->hess);
    if (P->host) cudaFreeHost(P->host);
    *P = wec_poisson();
}

int poisson_build(wec_poisson *P)
{
    cudaStream_t st = P->st;
    for (int l = 0; l + 1 < P->nlev; ++l) {
        Level<double> &F = P->L64[l], &C = P->L64[l + 1];
        int cnt = (C.nx + 1) * C.ny + C.nx * (C.ny + 1);
        WEC_PROF("mg_coarsen", l, 24.0 * cnt, st);
        k_coarsen<double><<<nblk(cnt, 256), 256, 0, st>>>(F.nx, F.ny, F.bu, F.bv, C.bu, C.bv);
    }
    Level<double> &Lc = P->L64[P->nlev - 1];
    {
        const double nn = (double)Lc.nx * Lc.ny;
        WEC_PROF("mg_lu_factor", P->nlev - 1, 8.0 * nn * nn, st);
        k_lu_factor<double><<<1, 256, 0, st>>>(Lc.nx, Lc.ny, Lc.bu, Lc.bv, P->lu64);
    }
    if (P->prec == WEC_PREC_MIXED) {
        for (int l = 0; l < P->nlev; ++l) {
            long long nu = (long long)(P->L64[l].nx + 1) * P->L64[l].ny, nv = (long long)P->L64[l].nx * (P->L64[l].ny + 1);
            {
                WEC_PROF("convert", l, 12.0 * nu, st);
                k_convert<float, double><<<nblk(nu, 256), 256, 0, st>>>(nu, P->L64[l].bu, P->L32[l].bu);
            }
            WEC_PROF("convert", l, 12.0 * nv, st);
            k_convert<float, double><<<nblk(nv, 256), 256, 0, st>>>(nv, P->L64[l].bv, P->L32[l].bv);
        }
        Level<float> &Lf = P->L32[P->nlev - 1];
        const double nn = (double)Lf.nx * Lf.ny;
        WEC_PROF("mg_lu_factor", P->nlev - 1, 4.0 * nn * nn, st);
        k_lu_factor<float><<<1, 256, 0, st>>>(Lf.nx, Lf.ny, Lf.bu, Lf.bv, P->lu32);
    }
    WEC_CK(cudaGetLastError());
    P->have_coef = true;
    return WEC_OK;
}

int poisson_apply(wec_poisson *P, const double *x, double *y)
{
    int n = P->nx * P->ny;
    WEC_PROF("krylov_matvec", -1, 8.0 * (2.0 * n + (P->nx + 1.0) * P->ny + P->nx * (P->ny + 1.0)), P->st);
    k_apply<double><<<nblk(n, 256), 256, 0, P->st>>>(P->nx, P->ny, P->L64[0].bu, P->L64[0].bv, x, y);
    WEC_CK(cudaGetLastError());
    return WEC_OK;
}

int poisson_vcycle(wec_poisson *P, const double *b, double *x)
{
    int n = P->nx * P->ny;
    if (P->prec == WEC_PREC_FP64) {
        vcycle_t<double>(P, P->L64, b, x);
    } else {
        {
            WEC_PROF("convert", -1, 12.0 * n, P->st);
            k_convert<float, double><<<nblk(n, 256), 256, 0, P->st>>>(n, b, P->L32[0].b);
        }
        vcycle_t<float>(P, P->L32, P->L32[0].b, P->L32[0].x);
        WEC_PROF("convert", -1, 12.0 * n, P->st);
        k_convert<double, float><<<nblk(n, 256), 256, 0, P->st>>>(n, P->L32[0].x, x);
    }
    WEC_CK(cudaGetLastError());
    return WEC_OK;
}

int poisson_solve(wec_poisson *P, const double *b, double *x, double rtol, int maxit, int *iters, double *relres)
{
    cudaStream_t st = P->st;
    const int n = P->nx * P->ny, m = P->restart, TB = 256;
    const size_t zsz = P->prec == WEC_PREC_FP64 ? 8 : 4;
    double *bn_d = P->scal + 0, *beta_d = P->scal + 1;
    const double *bu = P->L64[0].bu, *bv = P->L64[0].bv;
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    launch_norm2(b, n, P->part, bn_d, st);
    if (int e = read_scal(P, 1)) return e;
    double bn = P->host[0];
    if (!std::isfinite(bn)) return fail(WEC_ERR_NONFINITE, "pressure solve: right-hand side is not finite");
    if (bn == 0.0) {
        WEC_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
        return WEC_OK;
    }
    double tol = rtol * bn;
    const double nf = (P->nx + 1.0) * P->ny + P->nx * (P->ny + 1.0);
    {
        WEC_PROF("krylov_residual", -1, 8.0 * (3.0 * n + nf), st);
        k_residual<<<nblk(n, TB), TB, 0, st>>>(P->nx, P->ny, bu, bv, x, b, P->w);
    }
    launch_norm2(P->w, n, P->part, beta_d, st);
    if (int e = read_scal(P, 2)) return e;
    double beta = P->host[1];
    int its = 0;
    bool conv = beta <= tol;
    double *h1 = P->dots, *h2 = P->dots + (kMaxRestart + 2), *hn2 = P->dots + 2 * (kMaxRestart + 2);
    while (!conv && its < maxit) {
        {
            WEC_PROF("krylov_scale", -1, 16.0 * n, st);
            k_scale_div<<<nblk(n, TB), TB, 0, st>>>(n, P->w, beta_d, P->V);
        }
        {
            WEC_PROF("scalar", -1, 8.0 * (m + 2), st);
            k_cycle_init<<<1, 1, 0, st>>>(m, beta_d, P->g);
        }
        int jd = 0;
        for (int j = 0; j < m; ++j) {
            double *vj = P->V + (size_t)j * n;
            void *zj = (char *)P->Z + (size_t)j * n * zsz;
            precond(P, vj, zj);
            {
                WEC_PROF("krylov_matvec", -1, 8.0 * (n + nf) + (double)zsz * n, st);
                if (P->prec == WEC_PREC_FP64)
                    k_apply<double><<<nblk(n, TB), TB, 0, st>>>(P->nx, P->ny, bu, bv, (const double *)zj, P->w);
                else
                    k_apply<float><<<nblk(n, TB), TB, 0, st>>>(P->nx, P->ny, bu, bv, (const float *)zj, P->w);
            }
            its++;
            dots(P, P->V, j + 1, P->w, h1);
            {
                WEC_PROF("krylov_axpy", -1, 8.0 * n * (j + 3), st);
                k_axpy_multi<<<nblk(n, TB), TB, 0, st>>>(n, j + 1, P->V, h1, P->w);
            }
            dots(P, P->V, j + 1, P->w, h2);
            {
                WEC_PROF("krylov_axpy", -1, 8.0 * n * (j + 3), st);
                k_axpy_multi<<<nblk(n, TB), TB, 0, st>>>(n, j + 1, P->V, h2, P->w);
            }
            dots(P, P->w, 1, P->w, hn2);
            {
                WEC_PROF("scalar", -1, 8.0 * (3 * (j + 2) + 4), st);
                k_givens<<<1, 1, 0, st>>>(j, m, h1, h2, hn2, P->hess, P->cs, P->sn, P->g, P->scal);
            }
            if (int e = read_scal(P, 4)) return e;
            double est = P->host[2], hn = P->host[3];
            jd = j + 1;
            if (!std::isfinite(est)) return fail(WEC_ERR_NONFINITE, "pressure solve: residual estimate is not finite");
            if (est <= tol || its >= maxit || hn == 0.0) break;
            WEC_PROF("krylov_scale", -1, 16.0 * n, st);
            k_scale_div<<<nblk(n, TB), TB, 0, st>>>(n, P->w, P->scal + 3, P->V + (size_t)(j + 1) * n);
        }
        {
            WEC_PROF("scalar", -1, 8.0 * (jd * jd + 2 * jd), st);
            k_backsolve<<<1, 1, 0, st>>>(jd, m, P->hess, P->g, P->y);
        }
        {
            WEC_PROF("krylov_update_x", -1, 16.0 * n + (double)zsz * n * jd, st);
            if (P->prec == WEC_PREC_FP64)
                k_update_x<double><<<nblk(n, TB), TB, 0, st>>>(n, jd, P->y, (const double *)P->Z, x);
            else
                k_update_x<float><<<nblk(n, TB), TB, 0, st>>>(n, jd, P->y, (const float *)P->Z, x);
        }
        {
            WEC_PROF("krylov_residual", -1, 8.0 * (3.0 * n + nf), st);
            k_residual<<<nblk(n, TB), TB, 0, st>>>(P->nx, P->ny, bu, bv, x, b, P->w);
        }
        launch_norm2(P->w, n, P->part, beta_d, st);
        if (int e = read_scal(P, 2)) return e;
        beta = P->host[1];
        if (!std::isfinite(beta)) return fail(WEC_ERR_NONFINITE, "pressure solve: residual is not finite");
        conv = beta <= tol;
    }
    WEC_CK(cudaGetLastError());
    if (iters) *iters = its;
    if (relres) *relres = beta / bn;
    if (!conv) return fail(WEC_ERR_NOT_CONVERGED, "pressure solve: not converged within max_iters");
    return WEC_OK;
}

}  // namespace wec
