// Fused multigrid V-cycle kernels (included by solver.cu).
//
// The V-cycle of solver.cu -- red-black Gauss-Seidel, residual restriction by
// the sum of four children, piecewise-constant prolongation -- launched as:
//   k_mg_pre    per fine level: nu1 smoothing sweeps from x = 0, the residual and
//               its restriction, in one kernel.  Each CTA owns a TX x TY tile and
//               loads it with a halo of H = 2 max(nu1, nu2) cells into shared
//               memory; a colour pass leaves exact values one cell further in
//               than the previous one (the first red pass from x = 0 reads no
//               neighbour), so after 2 nu1 passes the tile and one ring around
//               it are exact, which is what the residual needs.  Halo cells are
//               recomputed redundantly.
//   k_mg_bottom one CTA for all levels of at most kBottomCells cells, staged in
//               shared memory, down to the dense LU of the coarsest level and
//               back up, with __syncthreads() between colour passes.
//   k_mg_post   per fine level: prolongation + correction and nu2 sweeps, same
//               tiling.
// A cell update is x = (b + sum_f beta_f x_nb) * (1 / d) with the reciprocal of
// the diagonal formed once per coefficient set (poisson_build) and staged with
// the tile (the one-pass kernels of solver.cu divide by d instead: the two
// V-cycles agree to rounding).  Face
// coefficients are zero on the Neumann walls and x is zero outside the domain,
// so a tile update needs no boundary branches (the staging zeroes the wall
// faces); 1/d is zero outside the domain, which keeps those cells at zero.
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

// q = k / d for 0 <= k < 2^16, 2 <= d < 2^16 by one multiply-high with m = magic_u16(d):
// with m = floor(2^32 / d) + 1 the error term k (m - 2^32 / d) / 2^32 < 2^-16 < 1 / d.
__host__ __device__ inline unsigned magic_u16(unsigned d) { return 0xffffffffu / d + 1u; }
__device__ __forceinline__ int div_u16(int k, unsigned m) { return (int)__umulhi((unsigned)k, m); }

// One element global -> shared without a register round trip (cp.async); with
// in == false the element is zero-filled and nothing is read (src must still be
// a valid address).  Completed by cp_async_wait_all() + __syncthreads().
template <typename T>
__device__ __forceinline__ void cp_async_el(T *dst, const T *src, bool in = true)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = in ? (int)sizeof(T) : 0;
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T>
struct TileView {
    int ex, ey, gx0, gy0, nx, ny;
    T *x, *b, *id, *bu, *bv;  // shared: x, b, 1/d [ey][ex]; bu[ey][ex+1]; bv[ey+1][ex]

    // d of cell (li, lj), as diag_at: the top row's Dirichlet face counts twice
    __device__ __forceinline__ T diag(int li, int lj) const
    {
        const T f = gy0 + lj == ny - 1 ? T(2) : T(1);
        return ((bu[lj * (ex + 1) + li] + bu[lj * (ex + 1) + li + 1]) + bv[lj * ex + li]) + f * bv[(lj + 1) * ex + li];
    }

    // sum_f beta_f x_nb, as offsum_at (walls have beta = 0, outside x = 0)
    __device__ __forceinline__ T offsum(int li, int lj) const
    {
        const int c = lj * ex + li;
        return ((bu[lj * (ex + 1) + li] * x[c - 1] + bu[lj * (ex + 1) + li + 1] * x[c + 1]) + bv[lj * ex + li] * x[c - ex]) +
               bv[(lj + 1) * ex + li] * x[c + ex];
    }
};

// Stage b, 1/d, x (xg + prolonged xc when xg is given, else 0), bu, bv of the
// tile (zero outside the domain; bu, bv also zero on the Neumann walls).
template <typename T>
__device__ void tile_load(TileView<T> &t, const T *__restrict__ bu, const T *__restrict__ bv,
                          const T *__restrict__ b, const T *__restrict__ idg, const T *xg, const T *__restrict__ xc)
{
    const int nx = t.nx, ny = t.ny, ex = t.ex, ey = t.ey;
    const unsigned mex = magic_u16(ex), mex1 = magic_u16(ex + 1);
    for (int k = threadIdx.x; k < ex * ey; k += blockDim.x) {
        const int lj = div_u16(k, mex), li = k - lj * ex, gi = t.gx0 + li, gj = t.gy0 + lj;
        const bool in = gi >= 0 && gi < nx && gj >= 0 && gj < ny;
        cp_async_el(t.b + k, in ? b + gj * nx + gi : b, in);
        cp_async_el(t.id + k, in ? idg + gj * nx + gi : idg, in);
    }
    for (int k = threadIdx.x; k < (ex + 1) * ey; k += blockDim.x) {
        const int lj = div_u16(k, mex1), li = k - lj * (ex + 1), gi = t.gx0 + li, gj = t.gy0 + lj;
        const bool in = gi > 0 && gi < nx && gj >= 0 && gj < ny;  // Neumann wall faces count as zero
        cp_async_el(t.bu + k, in ? bu + gj * (nx + 1) + gi : bu, in);
    }
    for (int k = threadIdx.x; k < ex * (ey + 1); k += blockDim.x) {
        const int lj = div_u16(k, mex), li = k - lj * ex, gi = t.gx0 + li, gj = t.gy0 + lj;
        const bool in = gi >= 0 && gi < nx && gj > 0 && gj <= ny;  // bottom wall zero, top (Dirichlet) kept
        cp_async_el(t.bv + k, in ? bv + gj * nx + gi : bv, in);
    }
#pragma unroll 4
    for (int k = threadIdx.x; k < ex * ey; k += blockDim.x) {
        const int lj = div_u16(k, mex), li = k - lj * ex, gi = t.gx0 + li, gj = t.gy0 + lj;
        T xv = T(0);
        if (xg && gi >= 0 && gi < nx && gj >= 0 && gj < ny)
            xv = xg[gj * nx + gi] + xc[(gj >> 1) * (nx >> 1) + (gi >> 1)];
        t.x[k] = xv;
    }
    cp_async_wait_all();
    __syncthreads();
}

// One colour pass over the tile.  The first pass (from x = 0) sets every cell
// of its colour to b / d; later passes update the cells off the outermost ring
// (their neighbours exist in the tile).  Threads walk the cells of the colour.
template <typename T>
__device__ void tile_pass(TileView<T> &t, int color, bool first, unsigned mwh)
{
    const int ex = t.ex, ey = t.ey, wh = ex >> 1;
    const int par = (color - t.gx0 - t.gy0) & 1;  // column parity of the colour in row 0
    for (int k = threadIdx.x; k < wh * ey; k += blockDim.x) {
        const int lj = div_u16(k, mwh), q = k - lj * wh;
        const int li = 2 * q + ((par - lj) & 1);
        const int c = lj * ex + li;
        if (first) {
            t.x[c] = t.b[c] * t.id[c];
        } else if (li > 0 && li < ex - 1 && lj > 0 && lj < ey - 1) {
            t.x[c] = (t.b[c] + t.offsum(li, lj)) * t.id[c];
        }
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void tile_setup(TileView<T> &t, unsigned char *smem_raw, int nx, int ny, int kTX, int kTY,
                                           int H)
{
    t.nx = nx;
    t.ny = ny;
    t.ex = kTX + 2 * H;
    t.ey = kTY + 2 * H;
    t.gx0 = blockIdx.x * kTX - H;
    t.gy0 = blockIdx.y * kTY - H;
    T *p = reinterpret_cast<T *>(smem_raw);
    t.x = p;
    t.b = t.x + t.ex * t.ey;
    t.id = t.b + t.ex * t.ey;
    t.bu = t.id + t.ex * t.ey;
    t.bv = t.bu + (t.ex + 1) * t.ey;
}

// nu1 sweeps from zero, then the smoothed iterate (tile interior) into xp and
// the restricted residual into bc.
template <typename T, int kTX, int kTY>
__global__ void __launch_bounds__(256) k_mg_pre(int nx, int ny, const T *__restrict__ bu, const T *__restrict__ bv,
                                                const T *__restrict__ b, const T *__restrict__ idg,
                                                T *__restrict__ xp, T *__restrict__ bc, int nu1, int H,
                                                const int *bsel)
{
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const long long n = (long long)nx * ny;
    b = at_sel(b, bsel, n);
    TileView<T> t;
    tile_setup(t, smem_raw, nx, ny, kTX, kTY, H);
    const unsigned mwh = magic_u16(t.ex >> 1);
    tile_load(t, bu, bv, b, idg, (const T *)nullptr, (const T *)nullptr);
    for (int q = 0; q < nu1; ++q) {
        tile_pass(t, 0, q == 0, mwh);
        tile_pass(t, 1, false, mwh);
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
                T ax = t.diag(li, lj) * t.x[c] - t.offsum(li, lj);
                r[qq++] = t.b[c] - ax;
            }
        bc[gJ * ncx + gI] = ((r[0] + r[1]) + r[2]) + r[3];
    }
    for (int k = threadIdx.x; k < kTX * kTY; k += blockDim.x) {
        int li = H + k % kTX, lj = H + k / kTX, gi = t.gx0 + li, gj = t.gy0 + lj;
        if (gi < nx && gj < ny) xp[gj * nx + gi] = t.x[lj * t.ex + li];
    }
}

// x = xp + P x_c, then nu2 sweeps; writes the tile interior of x (in TO: the
// level-0 result of an FP32 V-cycle is stored widened to FP64).  Reads xp and
// writes x (different arrays): tiles read their halos while others write.
template <typename T, int kTX, int kTY, typename TO>
__global__ void __launch_bounds__(256) k_mg_post(int nx, int ny, const T *__restrict__ bu, const T *__restrict__ bv,
                                                 const T *__restrict__ b, const T *__restrict__ idg,
                                                 const T *__restrict__ xp, TO *x, const T *__restrict__ xc,
                                                 int nu2, int H, const int *bsel, const int *xsel)
{
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const long long n = (long long)nx * ny;
    b = at_sel(b, bsel, n);
    x = at_sel(x, xsel, n);
    TileView<T> t;
    tile_setup(t, smem_raw, nx, ny, kTX, kTY, H);
    const unsigned mwh = magic_u16(t.ex >> 1);
    tile_load(t, bu, bv, b, idg, xp, xc);
    for (int q = 0; q < nu2; ++q) {
        tile_pass(t, 0, false, mwh);
        tile_pass(t, 1, false, mwh);
    }
    for (int k = threadIdx.x; k < kTX * kTY; k += blockDim.x) {
        int li = H + k % kTX, lj = H + k / kTX, gi = t.gx0 + li, gj = t.gy0 + lj;
        if (gi < nx && gj < ny) x[gj * nx + gi] = TO(t.x[lj * t.ex + li]);
    }
}

template <typename T>
struct BottomLevels {
    int lb, nlev, nu1, nu2;
    int nx[kMaxLevels], ny[kMaxLevels];
    const T *bu[kMaxLevels], *bv[kMaxLevels];
    T *x[kMaxLevels], *b[kMaxLevels];
    const T *id[kMaxLevels];
    const T *lu;
    const T *inv;  // explicit inverse of the coarsest operator, or nullptr (use lu)
    double *x0d;  // when set (lb = 0, FP32 levels): level-0 result stored widened here instead of x[0]
};

// The coarsest level's explicit inverse (n <= kInvMax), or else its LU, is
// staged in shared memory when it takes at most 16 KB (n <= 64 cells in FP32, 45
// in FP64); a larger LU is read from global.
template <typename T>
__host__ __device__ inline bool lu_staged(const BottomLevels<T> &L)
{
    const long long n = (long long)L.nx[L.nlev - 1] * L.ny[L.nlev - 1];
    return L.inv || n * n * (long long)sizeof(T) <= 16 * 1024;
}

template <typename T>
__host__ __device__ inline long long level_elems(const BottomLevels<T> &L, int l)
{
    return 3LL * L.nx[l] * L.ny[l] + (long long)(L.nx[l] + 1) * L.ny[l] + (long long)L.nx[l] * (L.ny[l] + 1);
}

// Shared-memory elements the bottom kernel stages for levels lb.. (x, b, 1/d,
// bu, bv each) and, when staged, the coarsest LU.
template <typename T>
__host__ __device__ inline long long bottom_elems(const BottomLevels<T> &L, int lb)
{
    long long e = 0;
    for (int l = lb; l < L.nlev; ++l) e += level_elems(L, l);
    if (lu_staged(L)) {
        const long long n = (long long)L.nx[L.nlev - 1] * L.ny[L.nlev - 1];
        e += n * n;
    }
    return e;
}

// One colour pass of a level held in shared memory by the whole CTA (nx even).
// first: from x = 0 (the other colour is set to zero alongside).
template <typename T>
__device__ void sm_pass(int nx, int ny, const T *bu, const T *bv, const T *id, T *x, const T *b, int color,
                        bool first)
{
    const int half = nx >> 1;
    const unsigned mh = magic_u16(half);
    for (int k = threadIdx.x; k < half * ny; k += blockDim.x) {
        const int j = div_u16(k, mh);
        const int i = 2 * (k - j * half) + ((j & 1) ^ color);
        const int c = j * nx + i;
        if (first) {
            x[c] = b[c] * id[c];
            x[c + (i & 1 ? -1 : 1)] = T(0);
        } else {
            x[c] = (b[c] + offsum_at(bu, bv, x, nx, ny, i, j)) * id[c];
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
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long off[kMaxLevels + 1];
    const int lb = L.lb, last = L.nlev - 1;
    if (threadIdx.x == 0) {
        long long o = 0;
        for (int l = lb; l < L.nlev; ++l) {
            off[l] = o;
            o += level_elems(L, l);
        }
        off[kMaxLevels] = o;  // the staged LU
    }
    __syncthreads();
    T *sm = reinterpret_cast<T *>(smem_raw);
    auto X = [&](int l) { return sm + off[l]; };
    auto B = [&](int l) { return sm + off[l] + (long long)L.nx[l] * L.ny[l]; };
    auto ID = [&](int l) { return sm + off[l] + 2LL * L.nx[l] * L.ny[l]; };
    auto BU = [&](int l) { return sm + off[l] + 3LL * L.nx[l] * L.ny[l]; };
    auto BV = [&](int l) { return sm + off[l] + 3LL * L.nx[l] * L.ny[l] + (long long)(L.nx[l] + 1) * L.ny[l]; };
    // stage b of level lb, every level's coefficients and the LU, all copies in flight at once
    {
        const long long n = (long long)L.nx[lb] * L.ny[lb];
        const T *bg = lb == 0 ? at_sel((const T *)L.b[lb], bsel, n) : L.b[lb];
        T *sb = B(lb);
        for (int k = threadIdx.x; k < n; k += blockDim.x) cp_async_el(sb + k, bg + k);
    }
    for (int l = lb; l < L.nlev; ++l) {
        const int nx = L.nx[l], ny = L.ny[l];
        T *su = BU(l), *sv = BV(l);
        const T *gu = L.bu[l], *gv = L.bv[l];
        for (int k = threadIdx.x; k < (nx + 1) * ny; k += blockDim.x) cp_async_el(su + k, gu + k);
        for (int k = threadIdx.x; k < nx * (ny + 1); k += blockDim.x) cp_async_el(sv + k, gv + k);
        T *sid = ID(l);
        const T *gid = L.id[l];
        for (int k = threadIdx.x; k < nx * ny; k += blockDim.x) cp_async_el(sid + k, gid + k);
    }
    // the coarsest level's explicit inverse, or its LU when that is staged
    const int nlu = L.nx[last] * L.ny[last];
    const T *csrc = L.inv ? L.inv : L.lu;
    const bool c_sm = lu_staged(L);
    const T *lu = c_sm ? sm + off[kMaxLevels] : L.lu;
    if (c_sm)
        for (int k = threadIdx.x; k < nlu * nlu; k += blockDim.x) cp_async_el(sm + off[kMaxLevels] + k, csrc + k);
    cp_async_wait_all();
    __syncthreads();
    for (int l = lb; l < last; ++l) {
        const int nx = L.nx[l], ny = L.ny[l];
        T *x = X(l), *b = B(l), *su = BU(l), *sv = BV(l), *id = ID(l);
        for (int q = 0; q < L.nu1; ++q) {
            sm_pass(nx, ny, su, sv, id, x, b, 0, q == 0);
            sm_pass(nx, ny, su, sv, id, x, b, 1, false);
        }
        const int ncx = nx >> 1, ncy = ny >> 1;
        const unsigned mc = magic_u16(ncx);
        T *bc = B(l + 1);
        for (int k = threadIdx.x; k < ncx * ncy; k += blockDim.x) {
            const int J = div_u16(k, mc), I = k - J * ncx;
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
    if (L.inv) {
        // x = A^{-1} b: one warp per row, lanes over columns, fixed shuffle tree
        const int n = nlu;
        T *x = X(last);
        const T *b = B(last);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int r = w; r < n; r += kBottomThreads / 32) {
            T s = lane < n ? lu[r * n + lane] * b[lane] : T(0);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) x[r] = s;
        }
        __syncthreads();
    } else {
        const int n = nlu;
        T *x = X(last);
        const T *b = B(last);
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            for (int r = 0; r < n; ++r) {
                T s = T(0);
                for (int c = lane; c < r; c += 32) s += lu[(long long)r * n + c] * x[c];
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) x[r] = b[r] - s;
                __syncwarp();
            }
            for (int r = n - 1; r >= 0; --r) {
                T s = T(0);
                for (int c = r + 1 + lane; c < n; c += 32) s += lu[(long long)r * n + c] * x[c];
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) x[r] = (x[r] - s) / lu[(long long)r * n + r];
                __syncwarp();
            }
        }
        __syncthreads();
    }
    for (int l = last - 1; l >= lb; --l) {
        const int nx = L.nx[l], ny = L.ny[l];
        T *x = X(l), *b = B(l), *su = BU(l), *sv = BV(l), *id = ID(l);
        const T *xc = X(l + 1);
        const unsigned mx = magic_u16(nx);
        for (int k = threadIdx.x; k < nx * ny; k += blockDim.x) {
            const int j = div_u16(k, mx), i = k - j * nx;
            x[k] += xc[(j >> 1) * (nx >> 1) + (i >> 1)];
        }
        __syncthreads();
        for (int q = 0; q < L.nu2; ++q) {
            sm_pass(nx, ny, su, sv, id, x, b, 0, false);
            sm_pass(nx, ny, su, sv, id, x, b, 1, false);
        }
    }
    {
        const long long n = (long long)L.nx[lb] * L.ny[lb];
        const T *x = X(lb);
        if (lb == 0 && L.x0d) {
            double *xg = at_sel(L.x0d, xsel, n);
            for (int k = threadIdx.x; k < n; k += blockDim.x) xg[k] = double(x[k]);
        } else {
            T *xg = lb == 0 ? at_sel(L.x[lb], xsel, n) : L.x[lb];
            for (int k = threadIdx.x; k < n; k += blockDim.x) xg[k] = x[k];
        }
    }
}

template <typename T>
size_t tile_smem(int H, int kTX, int kTY)
{
    const size_t ex = kTX + 2 * H, ey = kTY + 2 * H;
    return sizeof(T) * (3 * ex * ey + (ex + 1) * ey + ex * (ey + 1));
}

}  // namespace
}  // namespace wec
