// Multigrid level kernels of the three-dimensional pressure operator (included
// by solver.cu inside its anonymous namespace; uses at_sel, k_lu_solve).
//
// Operator and layouts as in poisson_op.cuh (diag3_at / offsum3_at).  Red-black
// Gauss-Seidel with colour (i + j + k) mod 2, restriction = sum of the eight
// children's residuals, piecewise-constant prolongation, coarse face = half the
// sum of the four fine faces it covers, dense LU on the coarsest level.  Every
// smoothed level has nx, ny, nz even.
//
// Cell layouts.  FP64 levels keep x, b and 1/d in the natural order (x fastest).
// FP32 levels above the coarsest keep x and 1/d -- and b below level 0, whose
// b is written by the Krylov kernels -- colour-packed: the cells of colour 0,
// then those of colour 1, each block row by row with i / 2 fastest (pk3).  A
// one-colour pass then reads and writes only its own colour's x, 1/d and b, in
// full sectors, and its other-colour neighbours contiguously; in the natural
// order it fetched whole sectors of which it used half.  Faces stay natural.

// index of cell (i, j, k) in a colour-packed array (nx even)
__device__ __forceinline__ int pk3(int nx, int ny, int nz, int i, int j, int k)
{
    return ((((i + j + k) & 1) * nz + k) * ny + j) * (nx >> 1) + (i >> 1);
}
__device__ __forceinline__ int ix3(bool pk, int nx, int ny, int nz, int i, int j, int k)
{
    return pk ? pk3(nx, ny, nz, i, j, k) : (k * ny + j) * nx + i;
}

// offsum3_at with x colour-packed: the six neighbours have the other colour,
// the y and z ones at the cell's own i / 2 in the rows beside it; the same
// terms in the same order (the same value).
template <typename T>
__device__ __forceinline__ T offsum3_pk(const T *bx, const T *by, const T *bz, const T *x, int nx, int ny, int nz,
                                        int i, int j, int k)
{
    const int r = k * ny + j, fx = r * (nx + 1) + i, fy = (r + k) * nx + i, c = r * nx + i, pl = nx * ny;
    const int half = nx >> 1, ih = i >> 1;
    const T *xo = x + (1 - ((i + j + k) & 1)) * nz * ny * half + r * half;  // the other colour's row of the cell
    T s = T(0);
    if (i > 0) s = fma3(bx[fx], xo[(i - 1) >> 1], s);
    if (i < nx - 1) s = fma3(bx[fx + 1], xo[(i + 1) >> 1], s);
    if (j > 0) s = fma3(by[fy], xo[ih - half], s);
    if (j < ny - 1) s = fma3(by[fy + nx], xo[ih + half], s);
    if (k > 0) s = fma3(bz[c], xo[ih - ny * half], s);
    if (k < nz - 1) s = fma3(bz[c + pl], xo[ih + ny * half], s);
    return s;
}

// offsum3_pk for the black pass of a sweep from zero: its red neighbours are
// the values the red pass from zero gives them, (b + 0) (1/d), formed here
// instead of read -- the same terms in the same order (the same value)
template <typename T>
__device__ __forceinline__ T offsum3_pk_z(const T *bx, const T *by, const T *bz, const T *b, int bpk, const T *id,
                                          int nx, int ny, int nz, int i, int j, int k)
{
    const int r = k * ny + j, fx = r * (nx + 1) + i, fy = (r + k) * nx + i, c = r * nx + i, pl = nx * ny;
    const int half = nx >> 1, ih = i >> 1;
    const int q0 = (1 - ((i + j + k) & 1)) * nz * ny * half + r * half;  // the other colour's row of the cell
    auto red = [&](int q, int cn) { return (b[bpk ? q : cn] + T(0)) * id[q]; };
    T s = T(0);
    if (i > 0) s = fma3(bx[fx], red(q0 + ((i - 1) >> 1), c - 1), s);
    if (i < nx - 1) s = fma3(bx[fx + 1], red(q0 + ((i + 1) >> 1), c + 1), s);
    if (j > 0) s = fma3(by[fy], red(q0 + ih - half, c - nx), s);
    if (j < ny - 1) s = fma3(by[fy + nx], red(q0 + ih + half, c + nx), s);
    if (k > 0) s = fma3(bz[c], red(q0 + ih - ny * half, c - pl), s);
    if (k < nz - 1) s = fma3(bz[c + pl], red(q0 + ih + ny * half, c + pl), s);
    return s;
}

// One colour of a red-black sweep on a natural-order level (FP64); thread q ->
// the q-th cell of the colour.  first != 0: the sweep starts from x = 0, so the
// red pass writes b / d (the black cells' starting values are never read: a
// cell's new value depends on the other colour only).
template <typename T>
__global__ void __launch_bounds__(256) k3_rbgs(int nx, int ny, int nz, const T *__restrict__ bx,
                                               const T *__restrict__ by, const T *__restrict__ bz,
                                               const T *__restrict__ id, T *x, const T *__restrict__ b, int color,
                                               int first, const int *bsel, const int *xsel)
{
    pdl_entry();
    const int half = nx >> 1, nh = half * ny * nz;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nh) return;
    const long long n = (long long)nx * ny * nz;
    x = at_sel(x, xsel, n);
    b = at_sel(b, bsel, n);
    const int r = q / half, ih = q - r * half;
    const int k = r / ny, j = r - k * ny;
    const int i = 2 * ih + ((j + k + color) & 1);
    const int c = r * nx + i;
    if (first) {
        x[c] = (b[c] + T(0)) * id[c];
        return;
    }
    x[c] = (b[c] + offsum3_at(bx, by, bz, x, nx, ny, nz, i, j, k)) * id[c];
}

// The same pass on a colour-packed level.  One block row per (j, k) = (blockIdx.y,
// blockIdx.z), CPT cells of the row per thread, blockDim.x apart: no index
// division, and every load of the CPT cells is issued before the first store.
// bpk: b colour-packed too (levels below 0).  first: as in k3_rbgs.
// out (nullable): the last pass of the V-cycle writes the finished iterate in
// the natural order and in OT -- its own cell and the other-colour cell beside
// it in the row (i ^ 1), whose pass came before -- instead of its packed x
// (nothing reads that after it), so no separate pass reads it again.
// (OT: the result's type, FP64, FP32 or float pairs)
template <typename OT>
__device__ __forceinline__ OT widen_out(float v)
{
    if constexpr (std::is_same<OT, double>::value)
        return f2d_exact(v);
    else if constexpr (std::is_same<OT, float>::value)
        return v;
    else
        return OT(v, 0.f);
}
// Z1: the black pass of the first pre-smoothing sweep with its red pass folded
// in (offsum3_pk_z; the red values are not stored: with two or more sweeps the
// next red pass replaces them before anything reads them).
template <typename T, int CPT, typename OT = double, bool Z1 = false>
__global__ void __launch_bounds__(128) k3_rbgs_pk(int nx, int ny, int nz, const T *__restrict__ bx,
                                                  const T *__restrict__ by, const T *__restrict__ bz,
                                                  const T *__restrict__ id, T *x, const T *__restrict__ b, int color,
                                                  int first, int bpk, OT *out, const int *osel)
{
    pdl_entry();
    const int half = nx >> 1, nh = half * ny * nz, j = blockIdx.y, k = blockIdx.z, r = k * ny + j;
    const int p = (j + k + color) & 1;  // i = 2 ih + p
    T v[CPT], w[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
        const int ih = (blockIdx.x * CPT + u) * blockDim.x + threadIdx.x;
        if (ih >= half) continue;
        const int i = 2 * ih + p, q = r * half + ih, xo = color * nh + q;
        const T bv = b[bpk ? xo : r * nx + i];
        if (first) {
            v[u] = (bv + T(0)) * id[xo];
        } else if constexpr (Z1) {
            v[u] = (bv + offsum3_pk_z(bx, by, bz, b, bpk, id, nx, ny, nz, i, j, k)) * id[xo];
        } else {
            v[u] = (bv + offsum3_pk(bx, by, bz, x, nx, ny, nz, i, j, k)) * id[xo];
            if (out) w[u] = x[(1 - color) * nh + q];
        }
    }
    if (out) out = at_sel(out, osel, (long long)nx * ny * nz);
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
        const int ih = (blockIdx.x * CPT + u) * blockDim.x + threadIdx.x;
        if (ih >= half) continue;
        const int c = r * nx + 2 * ih + p, q = r * half + ih;
        if (!out) x[color * nh + q] = v[u];
        if (!first && out) {
            out[c] = widen_out<OT>(v[u]);
            out[c ^ 1] = widen_out<OT>(w[u]);
        }
    }
}

// Coarse right-hand side = sum of the residuals of the eight children.  dg
// (nullable): the level's diagonal, already formed (the FP64 level 0 has one),
// read instead of summing the six faces again.  Natural-order levels.
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
                const T ax = fma3(d, x[c], -offsum3_at(bx, by, bz, x, nx, ny, nz, i, j, k));
                s += b[c] - ax;
            }
    bc[q] = s;
}

// The same from a colour-packed level (b too when bpk) into a coarse b that is
// colour-packed when cpk; one block row per coarse (J, K) = (blockIdx.y, blockIdx.z).
template <typename T>
__global__ void __launch_bounds__(128) k3_resid_restrict_pk(int nx, int ny, int nz, const T *__restrict__ bx,
                                                            const T *__restrict__ by, const T *__restrict__ bz,
                                                            const T *__restrict__ x, const T *__restrict__ b,
                                                            T *__restrict__ bc, int bpk, int cpk)
{
    pdl_entry();
    const int cx = nx >> 1, cy = ny >> 1, cz = nz >> 1, J = blockIdx.y, K = blockIdx.z;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= cx) return;
    T s = T(0);
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk, c = (k * ny + j) * nx + i;
                const int pq = pk3(nx, ny, nz, i, j, k);
                const T d = diag3_at(bx, by, bz, nx, ny, nz, i, j, k);
                const T ax = fma3(d, x[pq], -offsum3_pk(bx, by, bz, x, nx, ny, nz, i, j, k));
                s += b[bpk ? pq : c] - ax;
            }
    bc[cpk ? pk3(cx, cy, cz, I, J, K) : (K * cy + J) * cx + I] = s;
}

// x += the coarse correction, piecewise constant.  Natural-order levels.
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

// The same into a colour-packed level from a coarse x that is colour-packed
// when cpk: threads along the packed rows, (j, k) = (blockIdx.y, blockIdx.z),
// nbx blocks per row and colour, colours c0.. in turn along blockIdx.x.  c0 = 1
// (post-smoothing follows): the black cells only -- the red pass that comes next
// reads the black values and never the red cells' own.
template <typename T>
__global__ void __launch_bounds__(128) k3_prolong_pk(int nx, int ny, int nz, T *__restrict__ x,
                                                     const T *__restrict__ xc, int cpk, int nbx, int c0)
{
    pdl_entry();
    const int col = c0 + (blockIdx.x >= nbx ? 1 : 0), half = nx >> 1, j = blockIdx.y, k = blockIdx.z;
    const int ih = (blockIdx.x - (col - c0) * nbx) * blockDim.x + threadIdx.x;
    if (ih >= half) return;
    const int i = 2 * ih + ((j + k + col) & 1);
    x[(col * nz * ny + k * ny + j) * half + ih] += xc[ix3(cpk, nx >> 1, ny >> 1, nz >> 1, i >> 1, j >> 1, k >> 1)];
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
    unsigned pk;  // bit l: level l colour-packed
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
    D.id[l][ix3((D.pk >> l) & 1u, nx, ny, D.nz[l], i, j, k)] = T(1) / diag3_at(D.bx[l], D.by[l], D.bz[l], nx, ny, D.nz[l], i, j, k);
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

// The coarse levels lb .. nlev-1 of a 3D V-cycle in one CTA: the same passes
// in the same order and per-cell arithmetic as the per-level kernels (so the
// same bits), each level's iterate and right-hand side in shared memory, the
// faces and 1/d read through L1 from the hierarchy.  Below a few thousand cells
// a per-level launch costs ~6 us whatever its size; here a level costs its
// passes' barriers.  b of level lb is read from bg, its x written to xg.  In
// shared memory every level is in the natural order; with pk set, the levels
// above the coarsest are colour-packed in global memory (1/d, bg, xg).
constexpr int kBottom3Max = 8192;   // cells of the first level run in the CTA
constexpr int kBottom3Levels = 8;
constexpr int kBottom3Smem = 227 * 1024;  // dynamic shared memory opted in for k3_bottom
template <typename T>
struct Bot3 {
    int lb, nlev, nu1, nu2, ncoarse, pk;
    int nx[kBottom3Levels], ny[kBottom3Levels], nz[kBottom3Levels];
    const T *bx[kBottom3Levels], *by[kBottom3Levels], *bz[kBottom3Levels], *id[kBottom3Levels];
    const T *lu;
};

template <typename T>
__global__ void __launch_bounds__(1024) k3_bottom(Bot3<T> B, const T *__restrict__ bg, T *__restrict__ xg)
{
    pdl_entry();
    extern __shared__ __align__(16) unsigned char k3b_smem[];
    T *const sm = reinterpret_cast<T *>(k3b_smem);
    const int nt = blockDim.x, tid = threadIdx.x;
    const int L = B.nlev - B.lb;  // levels in the CTA (local index 0 = level lb)
    int off[kBottom3Levels];
    {
        int o = 0;
        for (int q = 0; q < L; ++q) {
            off[q] = o;
            o += 2 * B.nx[q] * B.ny[q] * B.nz[q];
        }
    }
    auto X = [&](int q) { return sm + off[q]; };
    auto Bv = [&](int q) { return sm + off[q] + B.nx[q] * B.ny[q] * B.nz[q]; };
    const bool pk0 = B.pk && L > 1;  // level lb colour-packed in global memory
    // natural index of the t-th cell of level lb's global arrays
    auto nat0 = [&](int t) {
        if (!pk0) return t;
        const int nx = B.nx[0], ny = B.ny[0], half = nx >> 1, nh = half * ny * B.nz[0];
        const int col = t >= nh ? 1 : 0, u = t - col * nh, r = u / half, ih = u - r * half;
        const int k = r / ny, j = r - k * ny;
        return r * nx + 2 * ih + ((j + k + col) & 1);
    };
    {
        const int n0 = B.nx[0] * B.ny[0] * B.nz[0];
        for (int t = tid; t < n0; t += nt) Bv(0)[nat0(t)] = bg[t];
    }
    __syncthreads();
    // one colour of a red-black sweep on local level q (first: from x = 0)
    auto pass = [&](int q, int color, bool first) {
        const int nx = B.nx[q], ny = B.ny[q], nz = B.nz[q], half = nx >> 1, nh = half * ny * nz;
        const bool pq = B.pk && q < L - 1;  // 1/d of this level colour-packed
        T *x = X(q);
        const T *b = Bv(q);
        for (int t = tid; t < nh; t += nt) {
            const int r = t / half, ih = t - r * half;
            const int k = r / ny, j = r - k * ny;
            const int i = 2 * ih + ((j + k + color) & 1);
            const int c = r * nx + i;
            const T id = B.id[q][pq ? color * nh + t : c];
            if (first) {
                x[c] = (b[c] + T(0)) * id;
                x[c ^ 1] = T(0);
            } else {
                x[c] = (b[c] + offsum3_at(B.bx[q], B.by[q], B.bz[q], x, nx, ny, nz, i, j, k)) * id;
            }
        }
        __syncthreads();
    };
    for (int q = 0; q + 1 < L; ++q) {
        for (int s = 0; s < B.nu1; ++s) {
            pass(q, 0, s == 0);
            pass(q, 1, false);
        }
        // residual of the eight children into the coarse right-hand side
        const int nx = B.nx[q], ny = B.ny[q], nz = B.nz[q];
        const int cx = nx >> 1, cy = ny >> 1, cz = nz >> 1;
        const T *x = X(q), *b = Bv(q);
        T *bc = Bv(q + 1);
        for (int t = tid; t < cx * cy * cz; t += nt) {
            const int R = t / cx, I = t - R * cx, K = R / cy, J = R - K * cy;
            T s = T(0);
            for (int dk = 0; dk < 2; ++dk)
                for (int dj = 0; dj < 2; ++dj)
                    for (int di = 0; di < 2; ++di) {
                        const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk, c = (k * ny + j) * nx + i;
                        const T d = diag3_at(B.bx[q], B.by[q], B.bz[q], nx, ny, nz, i, j, k);
                        const T ax = fma3(d, x[c], -offsum3_at(B.bx[q], B.by[q], B.bz[q], x, nx, ny, nz, i, j, k));
                        s += b[c] - ax;
                    }
            bc[t] = s;
        }
        __syncthreads();
    }
    // coarsest level: the dense LU factors, one warp (the arithmetic of k_lu_solve)
    if (tid < 32) {
        const int n = B.ncoarse, lane = tid;
        const T *A = B.lu, *b = Bv(L - 1);
        T *x = X(L - 1);
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
    __syncthreads();
    for (int q = L - 2; q >= 0; --q) {
        const int nx = B.nx[q], ny = B.ny[q], nz = B.nz[q];
        T *x = X(q);
        const T *xc = X(q + 1);
        for (int c = tid; c < nx * ny * nz; c += nt) {
            const int r = c / nx, i = c - r * nx, k = r / ny, j = r - k * ny;
            x[c] += xc[((k >> 1) * (ny >> 1) + (j >> 1)) * (nx >> 1) + (i >> 1)];
        }
        __syncthreads();
        for (int s = 0; s < B.nu2; ++s) {
            pass(q, 0, false);
            pass(q, 1, false);
        }
    }
    const int n0 = B.nx[0] * B.ny[0] * B.nz[0];
    for (int t = tid; t < n0; t += nt) xg[t] = X(0)[nat0(t)];
}

// out (natural order: FP64, FP32 or float pairs) = x of an FP32 level (colour-packed if pk)
template <typename TO>
__global__ void __launch_bounds__(256) k3_unpack(int nx, int ny, int nz, const float *__restrict__ x, int pk, TO *out,
                                                 const int *outsel)
{
    pdl_entry();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx * ny * nz) return;
    out = at_sel(out, outsel, (long long)nx * ny * nz);
    const int r = c / nx, i = c - r * nx, k = r / ny, j = r - k * ny;
    const float v = x[ix3(pk, nx, ny, nz, i, j, k)];
    if constexpr (std::is_same<TO, float>::value) out[c] = v; else out[c] = widen_out<TO>(v);
}

// x0 = M^{-1} b0, one V-cycle over the 3D levels L (precision T).  FP32: x0
// is the level-0 iterate (colour-packed unless level 0 is the coarsest), b0 in
// the natural order; xout (nullable): where the last level-0 pass also writes
// the result in FP64 (osel: its column).  Returns whether it did.
template <typename T, typename OT = double>
bool vcycle3_unfused(wec_poisson *P, Level<T> *L, const T *b0, T *x0, const int *bsel, const int *xsel,
                     cudaStream_t st, OT *xout = nullptr, const int *osel = nullptr)
{
    bool wrote = false;
    const int TB = 256;
    const double ts = sizeof(T);
    constexpr bool PK = std::is_same<T, float>::value;  // levels above the coarsest colour-packed
    auto packed = [&](int l) { return PK && l < P->nlev - 1 ? 1 : 0; };
    // (the colour-packed kernels take the level-0 vectors unselected: bsel, and
    // xsel when x0 is the FP32 iterate, are null for an FP32 V-cycle)
    // a row of w cells over nb blocks of tx threads (a multiple of 32, at most
    // 128), cpt cells per thread, the blocks as even as the warps allow
    struct Split {
        int tx, nb;
    };
    auto rows = [](int w, int cpt) {
        const int nb = (w + 128 * cpt - 1) / (128 * cpt);
        return Split{((w + nb * cpt - 1) / (nb * cpt) + 31) / 32 * 32, nb};
    };
    auto rbgs = [&](int l, Level<T> &A, T *x, const T *b, const int *bs, const int *xs, int color, int first,
                    OT *o, const int *os, bool z1) {
        if constexpr (PK) {
            const int half = A.nx >> 1, cpt = half >= 64 ? 2 : 1;
            const Split sp = rows(half, cpt);
            const int tx = sp.tx;
            const dim3 g(sp.nb, A.ny, A.nz);
            auto kern = cpt == 2 ? (z1 ? k3_rbgs_pk<T, 2, OT, true> : k3_rbgs_pk<T, 2, OT, false>)
                                 : (z1 ? k3_rbgs_pk<T, 1, OT, true> : k3_rbgs_pk<T, 1, OT, false>);
            launch_k(kern, g, tx, 0, st, A.nx, A.ny, A.nz, A.bu, A.bv, A.bw, A.id, x, b, color, first, l > 0 ? 1 : 0, o,
                     os);
        } else {
            const int nh = (A.nx >> 1) * A.ny * A.nz;
            launch_k(k3_rbgs<T>, nblk(nh, TB), TB, 0, st, A.nx, A.ny, A.nz, A.bu, A.bv, A.bw, A.id, x, b, color,
                     first, bs, xs);
        }
    };
    // the coarse levels from lb down run in one CTA (option "mg3_bottom")
    int lb = P->nlev;
    if (g_mg3_bottom) {
        lb = 1;
        while (lb < P->nlev - 1 && (long long)L[lb].nx * L[lb].ny * L[lb].nz > kBottom3Max) ++lb;
        size_t sm = 0;
        for (int l = lb; l < P->nlev; ++l) sm += 2 * sizeof(T) * (size_t)L[l].nx * L[l].ny * L[l].nz;
        if (P->nlev - lb > kBottom3Levels || lb >= P->nlev || sm > (size_t)kBottom3Smem) lb = P->nlev;
    }
    for (int l = 0; l < P->nlev; ++l) {
        Level<T> &A = L[l];
        const T *b = l == 0 ? b0 : A.b;
        T *x = l == 0 ? x0 : A.x;
        const int *bs = l == 0 ? bsel : nullptr, *xs = l == 0 ? xsel : nullptr;
        const double n = (double)A.nx * A.ny * A.nz;
        const double nf = (A.nx + 1.0) * A.ny * A.nz + A.nx * (A.ny + 1.0) * A.nz + A.nx * A.ny * (A.nz + 1.0);
        if (l == lb) {
            Bot3<T> Bt{};
            Bt.lb = lb;
            Bt.nlev = P->nlev;
            Bt.nu1 = P->nu1;
            Bt.nu2 = P->nu2;
            Bt.ncoarse = P->ncoarse;
            Bt.pk = PK ? 1 : 0;
            if constexpr (sizeof(T) == 8) Bt.lu = (const T *)P->lu64; else Bt.lu = (const T *)P->lu32;
            size_t smem = 0;
            double bytes = 0.0;
            for (int q = 0; q < P->nlev - lb; ++q) {
                const Level<T> &C = L[lb + q];
                Bt.nx[q] = C.nx;
                Bt.ny[q] = C.ny;
                Bt.nz[q] = C.nz;
                Bt.bx[q] = C.bu;
                Bt.by[q] = C.bv;
                Bt.bz[q] = C.bw;
                Bt.id[q] = C.id;
                const double nq = (double)C.nx * C.ny * C.nz;
                smem += (size_t)(2 * nq) * sizeof(T);
                bytes += (nq + (C.nx + 1.0) * C.ny * C.nz + C.nx * (C.ny + 1.0) * C.nz + C.nx * C.ny * (C.nz + 1.0)) * ts;
            }
            WEC_PROF("mg3_bottom", lb, bytes + 2.0 * n * ts, st);
            launch_k(k3_bottom<T>, 1, 1024, smem, st, Bt, (const T *)A.b, A.x);
            break;
        }
        if (l == P->nlev - 1) {
            T *lu = nullptr;
            if constexpr (sizeof(T) == 8) lu = (T *)P->lu64; else lu = (T *)P->lu32;
            WEC_PROF("mg_lu_solve", l, (n * n + 2 * n) * ts, st);
            launch_k(k_lu_solve<T>, 1, 32, 0, st, (int)n, lu, b, x, bs, xs);
            break;
        }
        for (int q = 0; q < P->nu1; ++q)
            for (int color = 0; color < 2; ++color) {
                // packed levels with two or more sweeps: the first sweep's red pass
                // folded into its black pass (which reads b and 1/d of the red
                // cells instead of their x); else the red pass from zero reads
                // no neighbours (b, 1/d in, x out)
                const bool z1 = PK && P->nu1 >= 2 && q == 0;
                if (z1 && color == 0) continue;
                const bool from0 = q == 0;
                WEC_PROF(from0 ? "mg3_rbgs_from0" : "mg3_rbgs", l,
                         (z1 ? 2.5 * n + nf : from0 && color == 0 ? 1.5 * n : 2.0 * n + nf) * ts, st);
                rbgs(l, A, x, b, bs, xs, color, q == 0 && color == 0, (OT *)nullptr, nullptr, z1);
            }
        Level<T> &C = L[l + 1];
        const T *dg = nullptr;
        if constexpr (sizeof(T) == 8) dg = l == 0 ? (const T *)P->d0 : nullptr;
        {
            WEC_PROF("mg3_resid_restrict", l, (2.125 * n + nf + (dg ? n : 0.0)) * ts, st);
            if constexpr (PK) {
                const Split sp = rows(C.nx, 1);
                const int tx = sp.tx;
                launch_k(k3_resid_restrict_pk<T>, dim3(sp.nb, C.ny, C.nz), tx, 0, st, A.nx, A.ny,
                         A.nz, A.bu, A.bv, A.bw, (const T *)x, b, C.b, l > 0 ? 1 : 0, packed(l + 1));
            } else {
                launch_k(k3_resid_restrict<T>, nblk(C.nx * C.ny * C.nz, TB), TB, 0, st, A.nx, A.ny, A.nz, A.bu,
                         A.bv, A.bw, dg, x, b, C.b, bs, xs);
            }
        }
    }
    // ascent: from the level above the coarsest, or above the levels the CTA finished
    for (int l = (lb < P->nlev ? lb : P->nlev - 1) - 1; l >= 0; --l) {
        Level<T> &A = L[l];
        const T *b = l == 0 ? b0 : A.b;
        T *x = l == 0 ? x0 : A.x;
        const int *bs = l == 0 ? bsel : nullptr, *xs = l == 0 ? xsel : nullptr;
        const double n = (double)A.nx * A.ny * A.nz;
        const double nf = (A.nx + 1.0) * A.ny * A.nz + A.nx * (A.ny + 1.0) * A.nz + A.nx * A.ny * (A.nz + 1.0);
        {
            // colour-packed, post-smoothing next: the black cells only (their
            // values are all the next red pass reads; the red cells' are replaced)
            const int c0 = PK && P->nu2 > 0 ? 1 : 0;
            WEC_PROF("mg3_prolong", l, (c0 ? 1.125 : 2.125) * n * ts, st);
            if constexpr (PK) {
                const Split sp = rows(A.nx >> 1, 1);
                const int tx = sp.tx, nbx = sp.nb;
                launch_k(k3_prolong_pk<T>, dim3((2 - c0) * nbx, A.ny, A.nz), tx, 0, st, A.nx, A.ny, A.nz, x,
                         (const T *)L[l + 1].x, packed(l + 1), nbx, c0);
            } else {
                launch_k(k3_prolong<T>, nblk((long long)n, TB), TB, 0, st, A.nx, A.ny, A.nz, x, L[l + 1].x, xs);
            }
        }
        for (int q = 0; q < P->nu2; ++q)
            for (int color = 0; color < 2; ++color) {
                const bool last = PK && l == 0 && xout && q == P->nu2 - 1 && color == 1;
                // (+ the FP64 result and the other colour's values it reads)
                WEC_PROF("mg3_rbgs", l, (2.0 * n + nf) * ts + (last ? (2.0 + sizeof(OT)) * n : 0.0), st);
                rbgs(l, A, x, b, bs, xs, color, 0, last ? xout : (OT *)nullptr, last ? osel : nullptr, false);
                wrote = wrote || last;
            }
    }
    return wrote;
}

// result stored in TO: an FP32 V-cycle runs on its level-0 iterate, and its
// last level-0 pass writes the FP64 result into x0 (without post-smoothing, or
// for FP32 storage other than that iterate, a separate pass unpacks it); the
// FP64 V-cycle smooths x0 in place.
template <typename T, typename TO>
void vcycle3_t(wec_poisson *P, Level<T> *L, const T *b0, TO *x0, const int *bsel, const int *xsel, cudaStream_t st)
{
    if constexpr (std::is_same<T, double>::value) {
        static_assert(std::is_same<TO, double>::value, "an FP64 V-cycle delivers FP64");
        vcycle3_unfused<T>(P, L, b0, x0, bsel, xsel, st);
    } else {
        // the natural-order result (FP64, FP32 or float pairs) is written by the
        // last level-0 pass where there is one
        if constexpr (std::is_same<TO, float>::value) {
            if (x0 == L[0].x) {
                vcycle3_unfused<T>(P, L, b0, L[0].x, bsel, nullptr, st);
                return;
            }
        }
        if (vcycle3_unfused<T, TO>(P, L, b0, L[0].x, bsel, nullptr, st, x0, xsel)) return;
        const long long n = (long long)L[0].nx * L[0].ny * L[0].nz;
        WEC_PROF("convert", 0, (4.0 + sizeof(TO)) * n, st);
        launch_k(k3_unpack<TO>, nblk(n, 256), 256, 0, st, L[0].nx, L[0].ny, L[0].nz, (const float *)L[0].x,
                 P->nlev > 1 ? 1 : 0, x0, xsel);
    }
}
