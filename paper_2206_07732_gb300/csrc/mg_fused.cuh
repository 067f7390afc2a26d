// Fused multigrid V-cycle kernels (included by solver.cu).
//
// The V-cycle of solver.cu -- red-black Gauss-Seidel, residual restriction by
// the sum of four children, piecewise-constant prolongation -- launched as:
//   k_mg_pre    per fine level: nu1 smoothing sweeps from x = 0, the residual and
//               its restriction, in one kernel.  Each CTA owns a TX x TY tile and
//               loads it with a halo of H = 2 max(nu1, nu2) cells into shared
//               memory; every colour pass shrinks the valid region by one cell
//               (the first red pass from x = 0 reads no neighbour), so after
//               2 nu1 passes the tile and one ring around it are exact, which is
//               what the residual needs.  Halo cells are recomputed redundantly.
//   k_mg_bottom one CTA for all levels of at most kBottomCells cells, staged in
//               shared memory, down to the dense LU of the coarsest level and
//               back up, with __syncthreads() between colour passes.
//   k_mg_post   per fine level: prolongation + correction and nu2 sweeps, same
//               tiling.
// Every cell update is the same arithmetic, in the same order, as the one-pass
// kernels (diag_at / offsum_at), so the fused and unfused V-cycles agree bit for bit.
#pragma once

namespace wec {
namespace {

// Tile shapes (interior cells) of the fused level kernels; the autotuner picks
// one per level and precision.
constexpr int kNumTiles = 4;
constexpr int kTileX[kNumTiles] = {64, 32, 32, 16};
constexpr int kTileY[kNumTiles] = {16, 16, 8, 8};
constexpr int kBottomCells = 4096;      // levels up to this size run inside one CTA (shared memory)
constexpr int kBottomSmemMax = 200 * 1024;
constexpr int kBottomThreads = 1024;

template <typename T>
struct TileView {
    int ex, ey, gx0, gy0, nx, ny;
    T *x, *b, *bu, *bv;  // shared: x[ey][ex], b[ey][ex], bu[ey][ex+1], bv[ey+1][ex]

    __device__ __forceinline__ T diag(int li, int lj) const
    {
        const int gi = gx0 + li, gj = gy0 + lj;
        T d = T(0);
        if (gi > 0) d += bu[lj * (ex + 1) + li];
        if (gi < nx - 1) d += bu[lj * (ex + 1) + li + 1];
        if (gj > 0) d += bv[lj * ex + li];
        d += (gj < ny - 1 ? T(1) : T(2)) * bv[(lj + 1) * ex + li];
        return d;
    }

    __device__ __forceinline__ T offsum(int li, int lj) const
    {
        const int gi = gx0 + li, gj = gy0 + lj, c = lj * ex + li;
        T s = T(0);
        if (gi > 0) s += bu[lj * (ex + 1) + li] * x[c - 1];
        if (gi < nx - 1) s += bu[lj * (ex + 1) + li + 1] * x[c + 1];
        if (gj > 0) s += bv[lj * ex + li] * x[c - ex];
        if (gj < ny - 1) s += bv[(lj + 1) * ex + li] * x[c + ex];
        return s;
    }
};

template <typename T>
__device__ void tile_load(TileView<T> &t, const T *__restrict__ bu, const T *__restrict__ bv,
                          const T *__restrict__ b, const T *xg, const T *__restrict__ xc)
{
    const int nx = t.nx, ny = t.ny, ex = t.ex, ey = t.ey;
    for (int k = threadIdx.x; k < ex * ey; k += blockDim.x) {
        int li = k % ex, lj = k / ex, gi = t.gx0 + li, gj = t.gy0 + lj;
        bool in = gi >= 0 && gi < nx && gj >= 0 && gj < ny;
        t.b[k] = in ? b[gj * nx + gi] : T(0);
        T xv = T(0);
        if (in && xg) xv = xg[gj * nx + gi] + xc[(gj >> 1) * (nx >> 1) + (gi >> 1)];
        t.x[k] = xv;
    }
    for (int k = threadIdx.x; k < (ex + 1) * ey; k += blockDim.x) {
        int li = k % (ex + 1), lj = k / (ex + 1), gi = t.gx0 + li, gj = t.gy0 + lj;
        bool in = gi >= 0 && gi <= nx && gj >= 0 && gj < ny;
        t.bu[k] = in ? bu[gj * (nx + 1) + gi] : T(0);
    }
    for (int k = threadIdx.x; k < ex * (ey + 1); k += blockDim.x) {
        int li = k % ex, lj = k / ex, gi = t.gx0 + li, gj = t.gy0 + lj;
        bool in = gi >= 0 && gi < nx && gj >= 0 && gj <= ny;
        t.bv[k] = in ? bv[gj * nx + gi] : T(0);
    }
    __syncthreads();
}

// One colour pass over the tile cells at margin >= m (inside the domain): the
// threads walk the cells of that colour only, row by row.
template <typename T>
__device__ void tile_pass(TileView<T> &t, int color, int m, int first)
{
    const int ex = t.ex, ey = t.ey;
    const int w = ex - 2 * m, hgt = ey - 2 * m, wh = (w + 1) >> 1;
    for (int k = threadIdx.x; k < wh * hgt; k += blockDim.x) {
        const int r = k / wh, q = k - r * wh;
        const int lj = m + r;
        const int li = m + ((color - (t.gx0 + m) - (t.gy0 + lj)) & 1) + 2 * q;
        const int gi = t.gx0 + li, gj = t.gy0 + lj;
        if (li >= ex - m || gi < 0 || gi >= t.nx || gj < 0 || gj >= t.ny) continue;
        int c = lj * ex + li;
        T d = t.diag(li, lj);
        if (first)
            t.x[c] = (t.b[c] + T(0)) / d;
        else
            t.x[c] = (t.b[c] + t.offsum(li, lj)) / d;
    }
    __syncthreads();
}

// nu1 sweeps from zero, then the smoothed iterate (tile interior) into xp and
// the restricted residual into bc.
template <typename T, int kTX, int kTY>
__global__ void __launch_bounds__(256) k_mg_pre(int nx, int ny, const T *__restrict__ bu, const T *__restrict__ bv,
                                                const T *__restrict__ b, T *__restrict__ xp, T *__restrict__ bc,
                                                int nu1, int H, const int *bsel)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const long long n = (long long)nx * ny;
    b = at_sel(b, bsel, n);
    T *x = xp;
    TileView<T> t;
    t.nx = nx;
    t.ny = ny;
    t.ex = kTX + 2 * H;
    t.ey = kTY + 2 * H;
    t.gx0 = blockIdx.x * kTX - H;
    t.gy0 = blockIdx.y * kTY - H;
    T *p = reinterpret_cast<T *>(smem_raw);
    t.x = p;
    t.b = t.x + t.ex * t.ey;
    t.bu = t.b + t.ex * t.ey;
    t.bv = t.bu + (t.ex + 1) * t.ey;
    tile_load(t, bu, bv, b, (const T *)nullptr, (const T *)nullptr);
    int pass = 0;
    for (int q = 0; q < nu1; ++q) {
        // pass 0 (red, from zero) is exact on the whole tile; pass p is exact at margin >= p
        tile_pass(t, 0, pass, q == 0);
        ++pass;
        tile_pass(t, 1, pass, 0);
        ++pass;
    }
    const int ncx = nx >> 1, ncy = ny >> 1;
    for (int k = threadIdx.x; k < (kTX / 2) * (kTY / 2); k += blockDim.x) {
        int I = k % (kTX / 2), J = k / (kTX / 2);
        int gI = blockIdx.x * (kTX / 2) + I, gJ = blockIdx.y * (kTY / 2) + J;
        if (gI >= ncx || gJ >= ncy) continue;
        T r[4];
        int qq = 0;
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                int li = H + 2 * I + di, lj = H + 2 * J + dj, c = lj * t.ex + li;
                T d = t.diag(li, lj);
                T ax = d * t.x[c] - t.offsum(li, lj);
                r[qq++] = t.b[c] - ax;
            }
        bc[gJ * ncx + gI] = ((r[0] + r[1]) + r[2]) + r[3];
    }
    for (int k = threadIdx.x; k < kTX * kTY; k += blockDim.x) {
        int li = H + k % kTX, lj = H + k / kTX, gi = t.gx0 + li, gj = t.gy0 + lj;
        if (gi < nx && gj < ny) x[gj * nx + gi] = t.x[lj * t.ex + li];
    }
}

// x = xp + P x_c, then nu2 sweeps; writes the tile interior of x.  Reads xp and
// writes x (different arrays): tiles read their halos while others write.
template <typename T, int kTX, int kTY>
__global__ void __launch_bounds__(256) k_mg_post(int nx, int ny, const T *__restrict__ bu, const T *__restrict__ bv,
                                                 const T *__restrict__ b, const T *__restrict__ xp, T *x,
                                                 const T *__restrict__ xc, int nu2, int H, const int *bsel,
                                                 const int *xsel)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const long long n = (long long)nx * ny;
    b = at_sel(b, bsel, n);
    x = at_sel(x, xsel, n);
    TileView<T> t;
    t.nx = nx;
    t.ny = ny;
    t.ex = kTX + 2 * H;
    t.ey = kTY + 2 * H;
    t.gx0 = blockIdx.x * kTX - H;
    t.gy0 = blockIdx.y * kTY - H;
    T *p = reinterpret_cast<T *>(smem_raw);
    t.x = p;
    t.b = t.x + t.ex * t.ey;
    t.bu = t.b + t.ex * t.ey;
    t.bv = t.bu + (t.ex + 1) * t.ey;
    tile_load(t, bu, bv, b, xp, xc);
    int pass = 1;  // loaded x is exact everywhere; pass p is exact at margin >= p
    for (int q = 0; q < nu2; ++q) {
        tile_pass(t, 0, pass, 0);
        ++pass;
        tile_pass(t, 1, pass, 0);
        ++pass;
    }
    for (int k = threadIdx.x; k < kTX * kTY; k += blockDim.x) {
        int li = H + k % kTX, lj = H + k / kTX, gi = t.gx0 + li, gj = t.gy0 + lj;
        if (gi < nx && gj < ny) x[gj * nx + gi] = t.x[lj * t.ex + li];
    }
}

template <typename T>
struct BottomLevels {
    int lb, nlev, nu1, nu2;
    int nx[kMaxLevels], ny[kMaxLevels];
    const T *bu[kMaxLevels], *bv[kMaxLevels];
    T *x[kMaxLevels], *b[kMaxLevels];
    const T *lu;
};

// Shared-memory elements the bottom kernel stages for levels lb.. (x, b, bu, bv each).
template <typename T>
__host__ __device__ inline long long bottom_elems(const BottomLevels<T> &L, int lb)
{
    long long e = 0;
    for (int l = lb; l < L.nlev; ++l)
        e += 2LL * L.nx[l] * L.ny[l] + (long long)(L.nx[l] + 1) * L.ny[l] + (long long)L.nx[l] * (L.ny[l] + 1);
    return e;
}

// One colour pass of a level held in shared memory by the whole CTA.
template <typename T>
__device__ void sm_pass(int nx, int ny, const T *bu, const T *bv, T *x, const T *b, int color, int first)
{
    const int half = nx >> 1;
    for (int k = threadIdx.x; k < half * ny; k += blockDim.x) {
        int j = k / half;
        int i = 2 * (k - j * half) + ((j & 1) ^ color);
        int c = j * nx + i;
        T d = diag_at(bu, bv, nx, ny, i, j);
        if (first) {
            x[c] = (b[c] + T(0)) / d;
            x[c + (i & 1 ? -1 : 1)] = T(0);
        } else {
            x[c] = (b[c] + offsum_at(bu, bv, x, nx, ny, i, j)) / d;
        }
    }
    __syncthreads();
}

// Levels lb .. nlev-1 of the V-cycle in one CTA, all staged in shared memory:
// load b of level lb and every level's coefficients, smooth / restrict down to
// the dense LU of the coarsest level, prolong / smooth back up, store x of level lb.
template <typename T>
__global__ void __launch_bounds__(kBottomThreads) k_mg_bottom(BottomLevels<T> L, const int *bsel,
                                                               const int *xsel)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long off[kMaxLevels];
    const int lb = L.lb, last = L.nlev - 1;
    if (threadIdx.x == 0) {
        long long o = 0;
        for (int l = lb; l < L.nlev; ++l) {
            off[l] = o;
            o += 2LL * L.nx[l] * L.ny[l] + (long long)(L.nx[l] + 1) * L.ny[l] + (long long)L.nx[l] * (L.ny[l] + 1);
        }
    }
    __syncthreads();
    T *sm = reinterpret_cast<T *>(smem_raw);
    auto X = [&](int l) { return sm + off[l]; };
    auto B = [&](int l) { return sm + off[l] + (long long)L.nx[l] * L.ny[l]; };
    auto BU = [&](int l) { return sm + off[l] + 2LL * L.nx[l] * L.ny[l]; };
    auto BV = [&](int l) { return sm + off[l] + 2LL * L.nx[l] * L.ny[l] + (long long)(L.nx[l] + 1) * L.ny[l]; };
    for (int l = lb; l < L.nlev; ++l) {
        const int nx = L.nx[l], ny = L.ny[l];
        T *su = BU(l), *sv = BV(l);
        for (int k = threadIdx.x; k < (nx + 1) * ny; k += blockDim.x) su[k] = L.bu[l][k];
        for (int k = threadIdx.x; k < nx * (ny + 1); k += blockDim.x) sv[k] = L.bv[l][k];
    }
    {
        const long long n = (long long)L.nx[lb] * L.ny[lb];
        const T *bg = lb == 0 ? at_sel((const T *)L.b[lb], bsel, n) : L.b[lb];
        T *sb = B(lb);
        for (int k = threadIdx.x; k < n; k += blockDim.x) sb[k] = bg[k];
    }
    __syncthreads();
    for (int l = lb; l < last; ++l) {
        const int nx = L.nx[l], ny = L.ny[l];
        T *x = X(l), *b = B(l), *su = BU(l), *sv = BV(l);
        for (int q = 0; q < L.nu1; ++q) {
            sm_pass(nx, ny, su, sv, x, b, 0, q == 0);
            sm_pass(nx, ny, su, sv, x, b, 1, 0);
        }
        const int ncx = nx >> 1, ncy = ny >> 1;
        T *bc = B(l + 1);
        for (int k = threadIdx.x; k < ncx * ncy; k += blockDim.x) {
            int I = k % ncx, J = k / ncx;
            T r[4];
            int qq = 0;
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    int i = 2 * I + di, j = 2 * J + dj, c = j * nx + i;
                    T d = diag_at(su, sv, nx, ny, i, j);
                    T ax = d * x[c] - offsum_at(su, sv, x, nx, ny, i, j);
                    r[qq++] = b[c] - ax;
                }
            bc[k] = ((r[0] + r[1]) + r[2]) + r[3];
        }
        __syncthreads();
    }
    {
        const int n = L.nx[last] * L.ny[last];
        T *x = X(last);
        const T *b = B(last);
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            for (int r = 0; r < n; ++r) {
                T s = T(0);
                for (int c = lane; c < r; c += 32) s += L.lu[(long long)r * n + c] * x[c];
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) x[r] = b[r] - s;
                __syncwarp();
            }
            for (int r = n - 1; r >= 0; --r) {
                T s = T(0);
                for (int c = r + 1 + lane; c < n; c += 32) s += L.lu[(long long)r * n + c] * x[c];
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) x[r] = (x[r] - s) / L.lu[(long long)r * n + r];
                __syncwarp();
            }
        }
        __syncthreads();
    }
    for (int l = last - 1; l >= lb; --l) {
        const int nx = L.nx[l], ny = L.ny[l];
        T *x = X(l), *b = B(l), *su = BU(l), *sv = BV(l);
        const T *xc = X(l + 1);
        for (int k = threadIdx.x; k < nx * ny; k += blockDim.x) {
            int i = k % nx, j = k / nx;
            x[k] += xc[(j >> 1) * (nx >> 1) + (i >> 1)];
        }
        __syncthreads();
        for (int q = 0; q < L.nu2; ++q) {
            sm_pass(nx, ny, su, sv, x, b, 0, 0);
            sm_pass(nx, ny, su, sv, x, b, 1, 0);
        }
    }
    {
        const long long n = (long long)L.nx[lb] * L.ny[lb];
        T *xg = lb == 0 ? at_sel(L.x[lb], xsel, n) : L.x[lb];
        const T *x = X(lb);
        for (int k = threadIdx.x; k < n; k += blockDim.x) xg[k] = x[k];
    }
}

template <typename T>
size_t tile_smem(int H, int kTX, int kTY)
{
    const size_t ex = kTX + 2 * H, ey = kTY + 2 * H;
    return sizeof(T) * (2 * ex * ey + (ex + 1) * ey + ex * (ey + 1));
}

}  // namespace
}  // namespace wec
