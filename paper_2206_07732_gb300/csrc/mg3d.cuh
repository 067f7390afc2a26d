// Multigrid level kernels of the three-dimensional pressure operator (included
// by solver.cu inside its anonymous namespace; uses at_sel, k_widen, k_lu_solve).
//
// Operator and layouts as in poisson_op.cuh (diag3_at / offsum3_at).  Red-black
// Gauss-Seidel with colour (i + j + k) mod 2, restriction = sum of the eight
// children's residuals, piecewise-constant prolongation, coarse face = half the
// sum of the four fine faces it covers, dense LU on the coarsest level.  Every
// smoothed level has nx, ny, nz even.  One thread per cell (per cell of one
// colour for the smoother): x fastest, so a warp reads 32 consecutive cells of
// one row and its neighbours in the rows above and below come from L1 / L2.

// One colour of a red-black sweep; thread q -> the q-th cell of the colour.
// first != 0: the sweep starts from x = 0, so the red pass writes b / d and
// zeroes the black cell beside it in the row.
template <typename T>
__global__ void __launch_bounds__(256) k3_rbgs(int nx, int ny, int nz, const T *__restrict__ bx,
                                               const T *__restrict__ by, const T *__restrict__ bz,
                                               const T *__restrict__ id, T *x, const T *__restrict__ b, int color,
                                               int first, const int *bsel, const int *xsel)
{
    pdl_entry();
    const int half = nx >> 1;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= half * ny * nz) return;
    const long long n = (long long)nx * ny * nz;
    x = at_sel(x, xsel, n);
    b = at_sel(b, bsel, n);
    const int r = q / half, ih = q - r * half;
    const int k = r / ny, j = r - k * ny;
    const int i = 2 * ih + ((j + k + color) & 1);
    const int c = r * nx + i;
    if (first) {
        x[c] = (b[c] + T(0)) * id[c];
        x[c ^ 1] = T(0);  // nx even: c and i have the same parity
        return;
    }
    x[c] = (b[c] + offsum3_at(bx, by, bz, x, nx, ny, nz, i, j, k)) * id[c];
}

// Coarse right-hand side = sum of the residuals of the eight children.  dg
// (nullable): the level's diagonal, already formed (the FP64 level 0 has one),
// read instead of summing the six faces again.
template <typename T>
__global__ void __launch_bounds__(256) k3_resid_restrict(int nx, int ny, int nz, const T *__restrict__ bx,
                                                         const T *__restrict__ by, const T *__restrict__ bz,
                                                         const T *__restrict__ dg, const T *__restrict__ x,
                                                         const T *__restrict__ b, T *__restrict__ bc,
                                                         const int *bsel, const int *xsel)
{
    pdl_entry();
    const int cx = nx >> 1, cy = ny >> 1, cz = nz >> 1;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cx * cy * cz) return;
    const long long n = (long long)nx * ny * nz;
    x = at_sel(x, xsel, n);
    b = at_sel(b, bsel, n);
    const int R = q / cx, I = q - R * cx, K = R / cy, J = R - K * cy;
    T s = T(0);
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk, c = (k * ny + j) * nx + i;
                const T d = dg ? dg[c] : diag3_at(bx, by, bz, nx, ny, nz, i, j, k);
                const T ax = d * x[c] - offsum3_at(bx, by, bz, x, nx, ny, nz, i, j, k);
                s += b[c] - ax;
            }
    bc[q] = s;
}

template <typename T>
__global__ void __launch_bounds__(256) k3_prolong(int nx, int ny, int nz, T *__restrict__ x,
                                                  const T *__restrict__ xc, const int *sel)
{
    pdl_entry();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx * ny * nz) return;
    x = at_sel(x, sel, (long long)nx * ny * nz);
    const int r = c / nx, i = c - r * nx, k = r / ny, j = r - k * ny;
    x[c] += xc[((k >> 1) * (ny >> 1) + (j >> 1)) * (nx >> 1) + (i >> 1)];
}

// Coarse faces of the level below (nx, ny, nz: the fine sizes), one thread per
// coarse face over beta_x, beta_y, beta_z in turn.
template <typename T>
__global__ void k3_coarsen(int nx, int ny, int nz, const T *__restrict__ fx, const T *__restrict__ fy,
                           const T *__restrict__ fz, T *__restrict__ cx, T *__restrict__ cy, T *__restrict__ cz)
{
    pdl_entry();
    const int X = nx >> 1, Y = ny >> 1, Z = nz >> 1;
    const int nfx = (X + 1) * Y * Z, nfy = X * (Y + 1) * Z, nfz = X * Y * (Z + 1);
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nfx) {
        const int R = q / (X + 1), I = q - R * (X + 1), K = R / Y, J = R - K * Y;
        T s = T(0);
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) s += fx[((2 * K + b) * ny + 2 * J + a) * (nx + 1) + 2 * I];
        cx[q] = T(0.5) * s;
        return;
    }
    q -= nfx;
    if (q < nfy) {
        const int R = q / X, I = q - R * X, K = R / (Y + 1), J = R - K * (Y + 1);
        T s = T(0);
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) s += fy[((2 * K + b) * (ny + 1) + 2 * J) * nx + 2 * I + a];
        cy[q] = T(0.5) * s;
        return;
    }
    q -= nfy;
    if (q < nfz) {
        const int R = q / X, I = q - R * X, K = R / Y, J = R - K * Y;
        T s = T(0);
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) s += fz[((2 * K) * ny + 2 * J + b) * nx + 2 * I + a];
        cz[q] = T(0.5) * s;
    }
}

// y = A x (FP64 operator; x may be FP32 storage)
template <typename TX>
__global__ void __launch_bounds__(256) k3_apply(int nx, int ny, int nz, const double *__restrict__ bx,
                                                const double *__restrict__ by, const double *__restrict__ bz,
                                                const TX *__restrict__ x, double *__restrict__ y)
{
    pdl_entry();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx * ny * nz) return;
    const int r = c / nx, i = c - r * nx, k = r / ny, j = r - k * ny;
    y[c] = diag3_at(bx, by, bz, nx, ny, nz, i, j, k) * double(x[c]) - offsum3_at(bx, by, bz, x, nx, ny, nz, i, j, k);
}

// d = diag(A) of level 0 (FP64), once per set of coefficients.
__global__ void k3_diag0(int nx, int ny, int nz, const double *__restrict__ bx, const double *__restrict__ by,
                         const double *__restrict__ bz, double *__restrict__ d)
{
    pdl_entry();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx * ny * nz) return;
    const int r = c / nx, i = c - r * nx, k = r / ny, j = r - k * ny;
    d[c] = diag3_at(bx, by, bz, nx, ny, nz, i, j, k);
}

template <typename T>
struct Level3Diag {
    int nlev;
    int nx[kMaxLevels], ny[kMaxLevels], nz[kMaxLevels];
    long long off[kMaxLevels + 1];
    const T *bx[kMaxLevels], *by[kMaxLevels], *bz[kMaxLevels];
    T *id[kMaxLevels];
};

// 1 / d of every cell of levels 0..nlev-1 in one launch.
template <typename T>
__global__ void k3_invdiag(Level3Diag<T> D)
{
    pdl_entry();
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= D.off[D.nlev]) return;
    int l = 0;
    while (q >= D.off[l + 1]) ++l;
    const int c = (int)(q - D.off[l]), nx = D.nx[l], ny = D.ny[l];
    const int r = c / nx, i = c - r * nx, k = r / ny, j = r - k * ny;
    D.id[l][c] = T(1) / diag3_at(D.bx[l], D.by[l], D.bz[l], nx, ny, D.nz[l], i, j, k);
}

// Dense operator of the coarsest level (n <= kMaxCoarse cells) into A (n x n,
// zeroed here), then its LU without pivoting (a symmetric M-matrix), one block.
template <typename T>
__global__ void k3_lu_factor(int nx, int ny, int nz, const T *__restrict__ bx, const T *__restrict__ by,
                             const T *__restrict__ bz, T *A)
{
    pdl_entry();
    const int n = nx * ny * nz, pl = nx * ny;
    for (long long q = threadIdx.x; q < (long long)n * n; q += blockDim.x) A[q] = T(0);
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const int r = c / nx, i = c - r * nx, k = r / ny, j = r - k * ny;
        const int fx = r * (nx + 1) + i, fy = (r + k) * nx + i;
        T *row = A + (long long)c * n;
        row[c] = diag3_at(bx, by, bz, nx, ny, nz, i, j, k);
        if (i > 0) row[c - 1] = -bx[fx];
        if (i < nx - 1) row[c + 1] = -bx[fx + 1];
        if (j > 0) row[c - nx] = -by[fy];
        if (j < ny - 1) row[c + nx] = -by[fy + nx];
        if (k > 0) row[c - pl] = -bz[c];
        if (k < nz - 1) row[c + pl] = -bz[c + pl];
    }
    __syncthreads();
    for (int p = 0; p < n; ++p) {
        const T piv = A[(long long)p * n + p];
        for (int r = p + 1 + threadIdx.x; r < n; r += blockDim.x) {
            const T f = A[(long long)r * n + p] / piv;
            A[(long long)r * n + p] = f;
            for (int c = p + 1; c < n; ++c) A[(long long)r * n + c] -= f * A[(long long)p * n + c];
        }
        __syncthreads();
    }
}

// x0 = M^{-1} b0, one V-cycle over the 3D levels L (precision T).
template <typename T>
void vcycle3_unfused(wec_poisson *P, Level<T> *L, const T *b0, T *x0, const int *bsel, const int *xsel,
                     cudaStream_t st)
{
    const int TB = 256;
    const double ts = sizeof(T);
    for (int l = 0; l < P->nlev; ++l) {
        Level<T> &A = L[l];
        const T *b = l == 0 ? b0 : A.b;
        T *x = l == 0 ? x0 : A.x;
        const int *bs = l == 0 ? bsel : nullptr, *xs = l == 0 ? xsel : nullptr;
        const double n = (double)A.nx * A.ny * A.nz;
        const double nf = (A.nx + 1.0) * A.ny * A.nz + A.nx * (A.ny + 1.0) * A.nz + A.nx * A.ny * (A.nz + 1.0);
        if (l == P->nlev - 1) {
            T *lu = nullptr;
            if constexpr (sizeof(T) == 8) lu = (T *)P->lu64; else lu = (T *)P->lu32;
            WEC_PROF("mg_lu_solve", l, (n * n + 2 * n) * ts, st);
            launch_k(k_lu_solve<T>, 1, 32, 0, st, (int)n, lu, b, x, bs, xs);
            break;
        }
        const int nh = (A.nx >> 1) * A.ny * A.nz;
        for (int q = 0; q < P->nu1; ++q)
            for (int color = 0; color < 2; ++color) {
                WEC_PROF("mg3_rbgs", l, (2.0 * n + nf) * ts, st);
                launch_k(k3_rbgs<T>, nblk(nh, TB), TB, 0, st, A.nx, A.ny, A.nz, A.bu, A.bv, A.bw, A.id, x, b, color,
                         q == 0 && color == 0, bs, xs);
            }
        Level<T> &C = L[l + 1];
        const T *dg = nullptr;
        if constexpr (sizeof(T) == 8) dg = l == 0 ? (const T *)P->d0 : nullptr;
        {
            WEC_PROF("mg3_resid_restrict", l, (2.125 * n + nf + (dg ? n : 0.0)) * ts, st);
            launch_k(k3_resid_restrict<T>, nblk(C.nx * C.ny * C.nz, TB), TB, 0, st, A.nx, A.ny, A.nz, A.bu, A.bv,
                     A.bw, dg, x, b, C.b, bs, xs);
        }
    }
    for (int l = P->nlev - 2; l >= 0; --l) {
        Level<T> &A = L[l];
        const T *b = l == 0 ? b0 : A.b;
        T *x = l == 0 ? x0 : A.x;
        const int *bs = l == 0 ? bsel : nullptr, *xs = l == 0 ? xsel : nullptr;
        const double n = (double)A.nx * A.ny * A.nz;
        const double nf = (A.nx + 1.0) * A.ny * A.nz + A.nx * (A.ny + 1.0) * A.nz + A.nx * A.ny * (A.nz + 1.0);
        {
            WEC_PROF("mg3_prolong", l, 2.125 * n * ts, st);
            launch_k(k3_prolong<T>, nblk((long long)n, TB), TB, 0, st, A.nx, A.ny, A.nz, x, L[l + 1].x, xs);
        }
        const int nh = (A.nx >> 1) * A.ny * A.nz;
        for (int q = 0; q < P->nu2; ++q)
            for (int color = 0; color < 2; ++color) {
                WEC_PROF("mg3_rbgs", l, (2.0 * n + nf) * ts, st);
                launch_k(k3_rbgs<T>, nblk(nh, TB), TB, 0, st, A.nx, A.ny, A.nz, A.bu, A.bv, A.bw, A.id, x, b, color,
                         0, bs, xs);
            }
    }
}

// result stored in TO (an FP32 V-cycle may deliver FP64): the one-colour
// kernels smooth in place, so a mixed V-cycle runs on the FP32 level-0 scratch
// and is widened into the FP64 column.
template <typename T, typename TO>
void vcycle3_t(wec_poisson *P, Level<T> *L, const T *b0, TO *x0, const int *bsel, const int *xsel, cudaStream_t st)
{
    if constexpr (std::is_same<T, TO>::value) {
        vcycle3_unfused<T>(P, L, b0, x0, bsel, xsel, st);
    } else {
        const long long n = (long long)L[0].nx * L[0].ny * L[0].nz;
        vcycle3_unfused<T>(P, L, b0, L[0].x, bsel, nullptr, st);
        WEC_PROF("convert", 0, 12.0 * n, st);
        launch_k(k_widen, nblk(n, 256), 256, 0, st, n, L[0].x, x0, xsel);
    }
}
