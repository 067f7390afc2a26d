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
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include <cooperative_groups.h>

#include "df64.cuh"
#include "internal.cuh"
#include "poisson_op.cuh"

namespace cg = cooperative_groups;

namespace wec {
namespace {

// Level-0 vectors of the V-cycle are FGMRES basis columns: base + j * n with j
// read on the device (so a captured graph serves every Arnoldi index).
template <typename T>
__device__ __forceinline__ T *at_sel(T *p, const int *sel, long long stride)
{
    return sel ? p + (long long)(*sel) * stride : p;
}

// ------------------------------------------------------------ stencil ----
// y = A x (FP64 operator; x may be FP32 storage of a preconditioned vector)
template <typename TX>
__global__ void k_apply(int nx, int ny, const double *__restrict__ bu, const double *__restrict__ bv,
                        const TX *__restrict__ x, double *__restrict__ y)
{
    pdl_entry();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx * ny) return;
    int i = c % nx, j = c / nx;
    double d = diag_at(bu, bv, nx, ny, i, j);
    y[c] = d * double(x[c]) - offsum_at(bu, bv, x, nx, ny, i, j);
}

// One colour of a red-black Gauss-Seidel sweep; thread k -> k-th cell of the
// colour (nx even on every smoothed level).  first != 0: the sweep starts from
// x = 0, so the red pass writes b / d and zeroes the black cells.
template <typename T>
__global__ void k_rbgs(int nx, int ny, const T *__restrict__ bu, const T *__restrict__ bv, T *x,
                       const T *__restrict__ b, int color, int first, const int *bsel, const int *xsel)
{
    pdl_entry();
    int half = nx >> 1;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= half * ny) return;
    const long long n = (long long)nx * ny;
    x = at_sel(x, xsel, n);
    b = at_sel(b, bsel, n);
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
                                 const T *__restrict__ x, const T *__restrict__ b, T *__restrict__ bc,
                                 const int *bsel, const int *xsel)
{
    pdl_entry();
    int ncx = nx >> 1, ncy = ny >> 1;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncx * ncy) return;
    const long long n = (long long)nx * ny;
    x = at_sel(x, xsel, n);
    b = at_sel(b, bsel, n);
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
__global__ void k_prolong(int nx, int ny, T *__restrict__ x, const T *__restrict__ xc, const int *sel)
{
    pdl_entry();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx * ny) return;
    x = at_sel(x, sel, (long long)nx * ny);
    int i = c % nx, j = c / nx;
    x[c] += xc[(j >> 1) * (nx >> 1) + (i >> 1)];
}

template <typename T>
__global__ void k_coarsen(int nx, int ny, const T *__restrict__ fu, const T *__restrict__ fv,
                          T *__restrict__ cu, T *__restrict__ cv)
{
    pdl_entry();
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

// out (column outsel, if given) = in widened to FP64
__global__ void k_widen(long long n, const float *__restrict__ in, double *out, const int *outsel)
{
    pdl_entry();
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= n) return;
    out = at_sel(out, outsel, n);
    out[c] = f2d_exact(in[c]);
}

// out = the float pairs of in (n values)
__global__ void k_to_pairs(long long n, const double *__restrict__ in, df64 *__restrict__ out)
{
    pdl_entry();
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c < n) out[c] = from_double(in[c]);
}

// both lower-precision copies of an FP64 array in one pass: float pairs and FP32
// (the pair's leading float is the nearest float, the FP32 copy's value)
__global__ void k_to_pairs_f32(long long n, const double *__restrict__ in, df64 *__restrict__ out,
                               float *__restrict__ out32)
{
    pdl_entry();
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= n) return;
    const df64 p = from_double(in[c]);
    out[c] = p;
    out32[c] = p.hi;
}

template <typename TO, typename TI>
__global__ void k_convert(long long n, const TI *__restrict__ in, TO *__restrict__ out, const int *insel)
{
    pdl_entry();
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= n) return;
    in = at_sel(in, insel, n);
    if constexpr (std::is_same<TO, float>::value && std::is_same<TI, double>::value)
        out[c] = d2f_rn(in[c]);
    else if constexpr (std::is_same<TO, double>::value && std::is_same<TI, float>::value)
        out[c] = f2d_exact(in[c]);
    else
        out[c] = TO(in[c]);
}

// Dense LU of the coarsest operator (no pivoting: A is a symmetric M-matrix).
// One block; the matrix lives in global memory (n <= 512).  inv (n <= kInvMax,
// else nullptr): also A^{-1}, column t by thread t from the two triangular solves.
template <typename T>
__global__ void k_lu_factor(int nx, int ny, const T *__restrict__ bu, const T *__restrict__ bv, T *A, T *inv)
{
    pdl_entry();
    // small systems (n <= 64) are built, factored and inverted in shared memory
    constexpr int kSmallN = 64;
    __shared__ T Ms[kSmallN * kSmallN];
    __shared__ T Is[kInvMax * kInvMax];
    const int n = nx * ny;
    const bool small = n <= kSmallN;
    T *M = small ? Ms : A;
    for (long long q = threadIdx.x; q < (long long)n * n; q += blockDim.x) M[q] = T(0);
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        int i = r % nx, j = r / nx;
        M[(long long)r * n + r] = diag_at(bu, bv, nx, ny, i, j);
        if (i > 0) M[(long long)r * n + r - 1] = -bu[j * (nx + 1) + i];
        if (i < nx - 1) M[(long long)r * n + r + 1] = -bu[j * (nx + 1) + i + 1];
        if (j > 0) M[(long long)r * n + r - nx] = -bv[j * nx + i];
        if (j < ny - 1) M[(long long)r * n + r + nx] = -bv[(j + 1) * nx + i];
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        T piv = M[(long long)k * n + k];
        for (int r = k + 1 + threadIdx.x; r < n; r += blockDim.x) {
            T f = M[(long long)r * n + k] / piv;
            M[(long long)r * n + k] = f;
            for (int c = k + 1; c < n; ++c) M[(long long)r * n + c] -= f * M[(long long)k * n + c];
        }
        __syncthreads();
    }
    if (small)
        for (int q = threadIdx.x; q < n * n; q += blockDim.x) A[q] = M[q];
    if (!inv) return;  // inv is given only for n <= kInvMax
    const int t = threadIdx.x;
    if (t < n) {
        for (int r = 0; r < n; ++r) {  // L y = e_t (unit lower), y in column t of Is
            T s = r == t ? T(1) : T(0);
            for (int c = 0; c < r; ++c) s -= M[(long long)r * n + c] * Is[c * n + t];
            Is[r * n + t] = s;
        }
        for (int r = n - 1; r >= 0; --r) {  // U x = y
            T s = Is[r * n + t];
            for (int c = r + 1; c < n; ++c) s -= M[(long long)r * n + c] * Is[c * n + t];
            Is[r * n + t] = s / M[(long long)r * n + r];
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) inv[q] = Is[q];
}

// 1/d of every cell of levels 0..nlev-1 (one launch; thread per cell of the
// concatenated levels, level found from the prefix offsets).
template <typename T>
struct LevelDiag {
    int nlev;
    int nx[kMaxLevels], ny[kMaxLevels];
    long long off[kMaxLevels + 1];
    const T *bu[kMaxLevels], *bv[kMaxLevels];
    T *id[kMaxLevels];
};

template <typename T>
__global__ void k_invdiag(LevelDiag<T> D)
{
    pdl_entry();
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= D.off[D.nlev]) return;
    int l = 0;
    while (k >= D.off[l + 1]) ++l;
    const int c = (int)(k - D.off[l]), nx = D.nx[l], j = c / nx, i = c - j * nx;
    D.id[l][c] = T(1) / diag_at(D.bu[l], D.bv[l], nx, D.ny[l], i, j);
}

// x = U^{-1} L^{-1} b, one warp.
template <typename T>
__global__ void k_lu_solve(int n, const T *__restrict__ A, const T *__restrict__ b, T *__restrict__ x,
                           const int *bsel, const int *xsel)
{
    pdl_entry();
    int lane = threadIdx.x;
    b = at_sel(b, bsel, n);
    x = at_sel(x, xsel, n);
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

}  // namespace
}  // namespace wec

#include "mg_fused.cuh"

namespace wec {
namespace {

bool g_mg_fused = true;  // fused V-cycle kernels (wec_set_option "mg_fused")
bool g_mg3_bottom = true;  // the 3D coarse levels in one CTA (wec_set_option "mg3_bottom")

#include "mg3d.cuh"

// --------------------------------------------------- Krylov (FP64 outer) ----
// Device-resident FGMRES state: the iteration is steered by the GPU, so the
// same kernels run host-polled (one status read per iteration) or inside one
// CUDA graph whose WHILE / IF conditional nodes read the state.
//
// Reductions run in three fixed-order stages, so every result is reproducible
// bit for bit: a shuffle tree per warp and the warps in order within a CTA; the
// 8 CTAs of a thread-block cluster in rank order through distributed shared
// memory; then the cluster partials, in the rank-0 CTA of the cluster that
// finishes last.  Grids are multiples of the cluster size and fit one wave: 2
// CTAs per SM, about 3.4 elements per thread on the 1024 x 256 grid, so the
// warp reductions (FP64 adds) are spread over several elements.
constexpr int KT = 256;   // threads of every fused Krylov kernel (8 warps)
constexpr int kCl = 8;    // CTAs per cluster of the reduction kernels
constexpr int KMAXV = kMaxRestart + 1;

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block's 256 threads in a fixed tree; valid in thread 0.
__device__ double block_sum(double v, double *sh8)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh8[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < KT / 32; ++w) r += sh8[w];
    __syncthreads();
    return r;
}

// bsm[k] (k < nk, one per CTA, in shared memory) -> the cluster's sum over its 8
// CTAs in rank order, written by the rank-0 CTA to part[k * NC + cluster].
// Every CTA of the cluster calls it (two cluster barriers: the second keeps each
// CTA's shared memory alive until rank 0 has read it).
__device__ void cluster_partials(double *bsm, int nk, double *part)
{
    cg::cluster_group cl = cg::this_cluster();
    const int NC = gridDim.x / kCl;
    cl.sync();
    if (cl.block_rank() == 0 && threadIdx.x < nk) {
        double s = 0.0;
        for (int r = 0; r < kCl; ++r) s += cl.map_shared_rank(bsm, r)[threadIdx.x];
        part[threadIdx.x * NC + blockIdx.x / kCl] = s;
    }
    cl.sync();
}

// Called by every CTA after cluster_partials: true in the rank-0 CTA of the
// cluster that finishes last (all cluster partials are then visible).
__device__ bool last_cluster(unsigned int *cnt)
{
    __shared__ int s_last;
    if (cg::this_cluster().block_rank() != 0) return false;
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(cnt, 1u) == gridDim.x / kCl - 1;
    }
    __syncthreads();
    return s_last != 0;
}

// Deterministic total of the G partials of one quantity (one CTA).
__device__ double final_sum(const double *part, int G, double *sh8)
{
    double s0 = 0.0, s1 = 0.0;
    int b = threadIdx.x;
    for (; b + KT < G; b += 2 * KT) {
        s0 += __ldcg(part + b);
        s1 += __ldcg(part + b + KT);
    }
    for (; b < G; b += KT) s0 += __ldcg(part + b);
    return block_sum(s0 + s1, sh8);
}

// out[k] = sum over the G partials part[k * G + c] (k < nk), one warp per k,
// lanes over c in a fixed assignment, fixed shuffle tree.
__device__ __forceinline__ void final_partials(const double *part, int nk, int G, double *out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = warp; k < nk; k += KT / 32) {
        double s0 = 0.0, s1 = 0.0;
        const double *pk = part + k * G;
        int b = lane;
        for (; b + 32 < G; b += 64) {
            s0 += __ldcg(pk + b);
            s1 += __ldcg(pk + b + 32);
        }
        for (; b < G; b += 32) s0 += __ldcg(pk + b);
        double s = warp_sum(s0 + s1);
        if (lane == 0) out[k] = s;
    }
}

// Warp reduce-scatter of K values per lane (K a power of two, at most 32): each
// exchange halves the values a lane holds, so the warp spends K - 1 + 5 - log2 K
// adds per lane instead of 5 K (FP64 adds are as scarce as FP64 FMAs on this
// GPU).  Afterwards a[0] of lane l is the warp total of value l >> (5 - log2 K).
// The exchange pattern is fixed: results are reproducible bit for bit.
template <int M, int O, int K>
__device__ __forceinline__ void wrs_stage(double (&a)[K], int lane)
{
    if constexpr (O > 0) {
        if constexpr (M > 1) {
            constexpr int H = M / 2;
            const bool up = (lane & O) != 0;
#pragma unroll
            for (int q = 0; q < H; ++q) {
                const double send = up ? a[q] : a[H + q];
                const double keep = up ? a[H + q] : a[q];
                a[q] = keep + __shfl_xor_sync(0xffffffffu, send, O);
            }
            wrs_stage<H, O / 2, K>(a, lane);
        } else {
            a[0] += __shfl_xor_sync(0xffffffffu, a[0], O);
            wrs_stage<1, O / 2, K>(a, lane);
        }
    }
}

template <int K>
__device__ __forceinline__ void warp_reduce_scatter(double (&a)[K], int lane)
{
    wrs_stage<K, 16, K>(a, lane);
}

// Krylov values: FP64, or float pairs over the same 8 bytes
__device__ __forceinline__ double vt_double(double a) { return a; }
__device__ __forceinline__ double vt_double(df64 a) { return to_double(a); }
template <typename VT>
__device__ __forceinline__ VT vt_from(double a)
{
    if constexpr (std::is_same<VT, double>::value) return a; else return from_double(a);
}
__device__ __forceinline__ float vt_float(double a) { return d2f_rn(a); }
__device__ __forceinline__ float vt_float(df64 a) { return a.hi; }  // the nearest float but in exact ties

// The CTA's partials of V_k . w (k < nk <= 32) into bsm[k], in fixed order, over
// one pass that also produces w: wof(c, v, i, r) returns w[c] (storing it if it
// makes it) given v[q] = V_q[c] for q < nk when HOLD (the columns read once per
// element, kept in registers for the update and the dots); without HOLD (K = 32,
// where 2 K held values would not fit the register budget) v is unset and the
// dots read V_q[c] again, from L1 right after the update read it.  The pass is
// grid-stride over the elements, or (ROWS, nx > 0) over rows of nx elements --
// row r = blockIdx.x + t gridDim.x, element i along it, c = r nx + i -- so a
// stencil needs no index division per element.
template <int K, bool ROWS, typename VT, typename F>
__device__ __forceinline__ void block_dots_k(const VT *V, long long n, int nx, int nk, F &&wof,
                                             double (*sh)[KMAXV], double *bsm)
{
    constexpr bool HOLD = K <= 16;
    constexpr int P2 = K >= 32 ? 5 : K >= 16 ? 4 : K >= 8 ? 3 : K >= 4 ? 2 : K >= 2 ? 1 : 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    VT av[K];
#pragma unroll
    for (int q = 0; q < K; ++q) av[q] = VT(0.0);
    auto elem = [&](long long c, int i, int r) {
        VT v[HOLD ? K : 1];
        if constexpr (HOLD) {
#pragma unroll
            for (int q = 0; q < K; ++q) v[q] = q < nk ? V[(long long)q * n + c] : VT(0.0);
        }
        const VT wc = wof(c, v, i, r);
#pragma unroll
        for (int q = 0; q < K; ++q)
            if (q < nk) av[q] += (HOLD ? v[HOLD ? q : 0] : V[(long long)q * n + c]) * wc;
    };
    if constexpr (ROWS) {
        const int nrows = (int)(n / nx);
        for (int r = blockIdx.x; r < nrows; r += gridDim.x)
            for (int i = threadIdx.x; i < nx; i += KT) elem((long long)r * nx + i, i, r);
    } else {
        for (long long c = blockIdx.x * (long long)KT + threadIdx.x; c < n; c += (long long)gridDim.x * KT)
            elem(c, 0, 0);
    }
    // the thread's sums, FP64 from here on
    double a[K];
#pragma unroll
    for (int q = 0; q < K; ++q) a[q] = vt_double(av[q]);
    warp_reduce_scatter<K>(a, lane);
    if ((lane & ((32 >> P2) - 1)) == 0) {
        const int k = lane >> (5 - P2);
        if (k < nk) sh[warp][k] = a[0];
    }
    __syncthreads();
    if (threadIdx.x < nk) {
        double r = 0.0;
        for (int q = 0; q < KT / 32; ++q) r += sh[q][threadIdx.x];
        bsm[threadIdx.x] = r;
    }
}

// nk <= KB (KB = 8: restarts up to 8, whose kernels hold few values per thread
// and run more CTAs per SM; KB = 32: any restart)
template <int KB, bool ROWS = false, typename VT, typename F>
__device__ __forceinline__ void block_dots(const VT *V, long long n, int nx, int nk, F &&wof, double (*sh)[KMAXV],
                                          double *bsm)
{
    if (nk <= 1) {
        block_dots_k<1, ROWS>(V, n, nx, nk, wof, sh, bsm);
    } else if (nk <= 2) {
        block_dots_k<2, ROWS>(V, n, nx, nk, wof, sh, bsm);
    } else if (nk <= 4 || KB <= 4) {  // (KB <= 4: nk <= 4)
        block_dots_k<4, ROWS>(V, n, nx, nk, wof, sh, bsm);
    } else if constexpr (KB <= 8) {
        block_dots_k<8, ROWS>(V, n, nx, nk, wof, sh, bsm);
    } else {
        if (nk <= 8)
            block_dots_k<8, ROWS>(V, n, nx, nk, wof, sh, bsm);
        else if (nk <= 16)
            block_dots_k<16, ROWS>(V, n, nx, nk, wof, sh, bsm);
        else
            block_dots_k<32, ROWS>(V, n, nx, nk, wof, sh, bsm);
    }
}

// CTAs per SM the matrix-vector kernel is compiled for: 4 (64 registers) where
// the dot products hold at most 8 sums per thread, else 2 (the Gram-Schmidt
// kernel, holding the basis values as well: 3 and 2)
constexpr int kb_blocks(int KB) { return KB <= 4 ? 6 : KB <= 8 ? 4 : 2; }

__device__ __forceinline__ void set_cond(unsigned long long h, int use, unsigned int v)
{
    if (use) cudaGraphSetConditional((cudaGraphConditionalHandle)h, v);
}

__global__ void k_ks_init(KState *ks, double rtol, int maxit, int m)
{
    pdl_entry();
    ks->rtol = rtol;
    ks->maxit = maxit;
    ks->m = m;
    ks->its = 0;
    ks->status = 0;
    ks->done = 0;
    ks->j = 0;
    ks->jd = 0;
    ks->cycle_end = 0;
    ks->ncycles = 0;
}

// The level-0 operator seen by the Krylov kernels: D = 2 (bx, by = beta_u,
// beta_v; nz = 1) or D = 3 (beta_x, beta_y, beta_z); FP64, or float pairs (VT =
// df64) for the pair-arithmetic Arnoldi step.
template <typename VT>
struct OpT {
    int nx, ny, nz;
    const VT *bx, *by, *bz;
};
using Op0 = OpT<double>;

template <int D, typename VT>
__device__ __forceinline__ VT op_offsum(const OpT<VT> &o, const VT *__restrict__ x, long long c)
{
    if constexpr (D == 2) {
        const int j = (int)(c / o.nx), i = (int)(c - (long long)j * o.nx);
        return offsum_at(o.bx, o.by, x, o.nx, o.ny, i, j);
    } else {
        const int cc = (int)c, r = cc / o.nx, i = cc - r * o.nx, k = r / o.ny, j = r - k * o.ny;
        return offsum3_at(o.bx, o.by, o.bz, x, o.nx, o.ny, o.nz, i, j, k);
    }
}

// d = diag(A) of level 0 (FP64), once per set of coefficients.
__global__ void k_diag0(int nx, int ny, const double *__restrict__ bu, const double *__restrict__ bv,
                        double *__restrict__ d)
{
    pdl_entry();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx * ny) return;
    const int j = c / nx, i = c - j * nx;
    d[c] = diag_at(bu, bv, nx, ny, i, j);
}

// bn = ||b||_2, tol = rtol bn.
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(KT, 4)
    k_bnorm(long long n, const double *__restrict__ b, double *part, KState *ks)
{
    pdl_entry();
    __shared__ double sh[KT / 32];
    __shared__ double bsm[1];
    double a = 0.0;
    for (long long c = blockIdx.x * (long long)KT + threadIdx.x; c < n; c += (long long)gridDim.x * KT)
        a += b[c] * b[c];
    a = block_sum(a, sh);
    if (threadIdx.x == 0) bsm[0] = a;
    cluster_partials(bsm, 1, part);
    if (!last_cluster(&ks->cnt[0])) return;
    double t = final_sum(part, gridDim.x / kCl, sh);
    if (threadIdx.x == 0) {
        double bn = sqrt(t);
        ks->bn = bn;
        ks->tol = ks->rtol * bn;
        ks->cnt[0] = 0;
    }
}

// u_0 = b - A x into V's column 0 (and its FP32 copy b32 for a mixed V-cycle),
// beta = ||u_0||, scale s_0 = 1 / beta.  mode 0 (start): converged if beta <= tol.
// mode 1 (end of a cycle): converged, out of iterations, or restart.
// A zero right-hand side gives x = 0.  Opens a new Arnoldi cycle unless done and
// sets the WHILE condition to !done.
template <int D, typename VT = double>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(KT, 4)
    k_residual_norm(Op0 op, const double *__restrict__ d0, const double *__restrict__ b, double *x,
                    VT *__restrict__ w, float *__restrict__ b32, double *sc, double *part, KState *ks, double *g,
                    int mode, unsigned long long hwhile, int use)
{
    pdl_entry();
    __shared__ double sh[KT / 32];
    __shared__ double bsm[1];
    const long long n = (long long)op.nx * op.ny * op.nz;
    const bool zero = ks->bn == 0.0;
    double a = 0.0;
    // s: the cell's off-diagonal sum
    auto cell = [&](long long c, double s) {
        if (zero) {
            x[c] = 0.0;
            w[c] = VT(0.0);
            return;
        }
        const double r = b[c] - (d0[c] * x[c] - s);
        w[c] = vt_from<VT>(r);
        if (b32) b32[c] = d2f_rn(r);  // (float)r on the integer pipe
        a += r * r;
    };
    if constexpr (D == 3) {  // along the grid's rows: one index division per row
        const int nrows = op.ny * op.nz;
        for (int row = blockIdx.x; row < nrows; row += gridDim.x) {
            const int k = row / op.ny, j = row - k * op.ny;
            for (int i = threadIdx.x; i < op.nx; i += KT) {
                const long long c = (long long)row * op.nx + i;
                cell(c, zero ? 0.0 : offsum3_at(op.bx, op.by, op.bz, (const double *)x, op.nx, op.ny, op.nz, i, j, k));
            }
        }
    } else {
        for (long long c = blockIdx.x * (long long)KT + threadIdx.x; c < n; c += (long long)gridDim.x * KT)
            cell(c, zero ? 0.0 : op_offsum<D, double>(op, x, c));
    }
    a = block_sum(a, sh);
    if (threadIdx.x == 0) bsm[0] = a;
    cluster_partials(bsm, 1, part);
    if (!last_cluster(&ks->cnt[1])) return;
    double t = final_sum(part, gridDim.x / kCl, sh);
    if (threadIdx.x == 0) {
        double beta = sqrt(t);
        ks->beta = beta;
        ks->ibeta = beta != 0.0 ? 1.0 / beta : 0.0;
        sc[0] = ks->ibeta;
        if (mode == 1) ks->ncycles += 1;
        int done;
        if (zero) {
            done = 1;
        } else if (!isfinite(beta)) {
            done = 1;
            ks->status = WEC_ERR_NONFINITE;
        } else if (beta <= ks->tol) {
            done = 1;
        } else if (mode == 1 && ks->its >= ks->maxit) {
            done = 1;
            ks->status = WEC_ERR_NOT_CONVERGED;
        } else {
            done = 0;
        }
        ks->done = done;
        if (!done) {
            g[0] = beta;
            for (int k = 1; k <= ks->m; ++k) g[k] = 0.0;
            ks->j = 0;
            ks->cycle_end = 0;
        }
        ks->cnt[1] = 0;
        set_cond(hwhile, use, done ? 0u : 1u);
    }
}

// Arnoldi step j on the unnormalised basis u_k = ||u_k|| v_k (V's columns, scales
// s_k = 1 / ||u_k|| in sc): the new vector w is built in place in column j+1.
// w = A z_j = s_j A z'_j (z'_j = M u_j, the V-cycle being linear), and the
// first Gram-Schmidt dot products h1_k = v_k . w = s_k (u_k . w), k <= j.
template <int D, int KB, typename VT = double, typename ZT = VT>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(KT, kb_blocks(KB))
    k_matvec_dots(OpT<VT> op, const VT *__restrict__ d0, const ZT *__restrict__ Z, VT *V,
                  const double *__restrict__ sc, double *part, double *h1, KState *ks)
{
    pdl_entry();
    __shared__ double sh[KT / 32][KMAXV];
    __shared__ double bsm[KMAXV];
    const long long n = (long long)op.nx * op.ny * op.nz;
    const int j = ks->j, nk = j + 1;
    const ZT *z = Z + (long long)j * n;  // (float pairs: the FP32 V-cycle's columns as floats)
    VT *w = V + (long long)(j + 1) * n;
    const VT sj = VT(sc[j]);  // (once per thread of the grid-stride loop)
    // w and its dots in one pass (w is not read back); 3D: along the grid's rows
    block_dots<KB, D == 3>(
        V, n, op.nx, nk,
        [&](long long c, const auto &, int i, int row) {
            VT s;
            if constexpr (D == 3) {
                const int k = row / op.ny, j = row - k * op.ny;
                s = offsum3_at(op.bx, op.by, op.bz, z, op.nx, op.ny, op.nz, i, j, k);
            } else {
                s = op_offsum<D, VT>(op, z, c);
            }
            const VT r = sj * (d0[c] * VT(z[c]) - s);
            w[c] = r;
            return r;
        },
        sh, bsm);
    cluster_partials(bsm, nk, part);
    if (!last_cluster(&ks->cnt[2])) return;
    final_partials(part, nk, gridDim.x / kCl, h1);
    __syncthreads();
    if (threadIdx.x < nk) h1[threadIdx.x] *= sc[threadIdx.x];
    if (threadIdx.x == 0) ks->cnt[2] = 0;
}

// First Gram-Schmidt update w -= sum_k h1_k v_k = w - sum_k (h1_k s_k) u_k, then
// h2_k = v_k . w.
template <int KB, typename VT = double>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(KT, KB <= 4 ? 4 : KB <= 8 ? 3 : 2)
    k_orth_dots(long long n, VT *V, const double *__restrict__ sc, const double *__restrict__ h1, double *part,
                double *h2, KState *ks)
{
    pdl_entry();
    __shared__ double sh[KT / 32][KMAXV];
    __shared__ double bsm[KMAXV];
    __shared__ VT hs[KMAXV];
    const int j = ks->j, nk = j + 1;
    VT *w = V + (long long)(j + 1) * n;
    if (threadIdx.x < nk) hs[threadIdx.x] = VT(h1[threadIdx.x] * sc[threadIdx.x]);
    __syncthreads();
    // the update and the second dots in one pass over the basis (V_k[c] read once)
    block_dots<KB>(
        V, n, 0, nk,
        [&](long long c, const auto &v, int, int) {
            constexpr int KH = std::extent<std::remove_reference_t<decltype(v)>>::value;
            VT a = w[c];
            if (nk <= KH) {
#pragma unroll
                for (int k = 0; k < KH; ++k)
                    if (k < nk) a -= hs[k] * v[k];
            } else {
                for (int k = 0; k < nk; ++k) a -= hs[k] * V[(long long)k * n + c];
            }
            w[c] = a;
            return a;
        },
        sh, bsm);
    cluster_partials(bsm, nk, part);
    if (!last_cluster(&ks->cnt[2])) return;
    final_partials(part, nk, gridDim.x / kCl, h2);
    __syncthreads();
    if (threadIdx.x < nk) h2[threadIdx.x] *= sc[threadIdx.x];
    if (threadIdx.x == 0) ks->cnt[2] = 0;
}

// Second update w -= sum_k (h2_k s_k) u_k, which leaves u_{j+1} = w in column j+1
// (and its FP32 copy b32 for the next mixed V-cycle), h_{j+1,j} = ||w||, s_{j+1} =
// 1 / h_{j+1,j}; the last cluster applies the Givens rotations to column j,
// counts the iteration, decides whether the cycle ends (converged estimate,
// iteration cap, breakdown, or full basis), advances j otherwise, and sets the
// IF condition.
template <typename VT = double>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(KT, std::is_same<VT, double>::value ? 4 : 6)
    k_orth_norm(long long n, VT *V, double *sc, float *__restrict__ b32, const double *__restrict__ h1,
                const double *__restrict__ h2, double *part, KState *ks, double *H, double *cs, double *sn,
                double *g, unsigned long long hif, int use)
{
    pdl_entry();
    __shared__ double sh[KT / 32];
    __shared__ double bsm[1];
    __shared__ VT hs[KMAXV];
    const int j = ks->j;
    VT *w = V + (long long)(j + 1) * n;
    if (threadIdx.x <= j) hs[threadIdx.x] = VT(h2[threadIdx.x] * sc[threadIdx.x]);
    __syncthreads();
    VT av2 = VT(0.0);
    for (long long c = blockIdx.x * (long long)KT + threadIdx.x; c < n; c += (long long)gridDim.x * KT) {
        VT a = w[c];
#pragma unroll 4
        for (int k = 0; k <= j; ++k) a -= hs[k] * V[(long long)k * n + c];
        w[c] = a;
        if (b32) b32[c] = vt_float(a);
        av2 += a * a;
    }
    double a2 = block_sum(vt_double(av2), sh);
    if (threadIdx.x == 0) bsm[0] = a2;
    cluster_partials(bsm, 1, part);
    if (!last_cluster(&ks->cnt[2])) return;
    double t = final_sum(part, gridDim.x / kCl, sh);
    if (threadIdx.x != 0) return;
    const int m = ks->m;
    for (int k = 0; k <= j; ++k) H[k * m + j] = (0.0 + h1[k]) + h2[k];
    double hn = sqrt(t);
    H[(j + 1) * m + j] = hn;
    for (int k = 0; k < j; ++k) {
        double p = H[k * m + j], q = H[(k + 1) * m + j];
        H[k * m + j] = cs[k] * p + sn[k] * q;
        H[(k + 1) * m + j] = -sn[k] * p + cs[k] * q;
    }
    double p = H[j * m + j], q = H[(j + 1) * m + j];
    double den = sqrt(p * p + q * q);
    cs[j] = p / den;
    sn[j] = q / den;
    H[j * m + j] = den;
    H[(j + 1) * m + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    ks->its += 1;
    ks->jd = j + 1;
    ks->hn = hn;
    ks->ihn = hn != 0.0 ? 1.0 / hn : 0.0;
    sc[j + 1] = ks->ihn;
    double est = fabs(g[j + 1]);
    int ce = est <= ks->tol || ks->its >= ks->maxit || hn == 0.0 || j + 1 == m || !isfinite(est);
    if (!isfinite(est)) ks->status = WEC_ERR_NONFINITE;
    ks->cycle_end = ce;
    if (!ce) ks->j = j + 1;  // every CTA read j at its start
    ks->cnt[2] = 0;
    set_cond(hif, use, (unsigned)ce);
}

// y from the triangular system, then y_k s_k: the preconditioned vectors are
// stored for the unnormalised basis (z'_k = z_k / s_k), so x += sum_k (y_k s_k) z'_k.
__global__ void k_backsolve(int m, const double *__restrict__ H, const double *__restrict__ g, double *__restrict__ y,
                            const double *__restrict__ sc, const KState *ks)
{
    pdl_entry();
    const int jd = ks->jd;
    for (int k = jd - 1; k >= 0; --k) {
        double s = g[k];
        for (int l = k + 1; l < jd; ++l) s -= H[k * m + l] * y[l];
        y[k] = s / H[k * m + k];
    }
    for (int k = 0; k < jd; ++k) y[k] *= sc[k];
}

template <typename VT = double>
__global__ void k_update_x(long long n, const double *__restrict__ y, const VT *__restrict__ Z, double *__restrict__ x,
                           const KState *ks)
{
    pdl_entry();
    const int jd = ks->jd;
    if constexpr (std::is_same<VT, double>::value) {
        long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
        if (c >= n) return;
        double a = x[c];
#pragma unroll 4
        for (int k = 0; k < jd; ++k) a += y[k] * Z[(long long)k * n + c];
        x[c] = a;
    } else {  // FP32 columns (the FP32 V-cycle's values, widened exactly): the same FP64 update
        long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
        if (c >= n) return;
        double a = x[c];
#pragma unroll 4
        for (int k = 0; k < jd; ++k) a += y[k] * f2d_exact(Z[(long long)k * n + c]);
        x[c] = a;
    }
}

// ------------------------------------------------------------ V-cycle ----
// bsel / xsel: device index of the level-0 right-hand side / solution column
// (nullptr: the pointer is used as is).
template <typename T>
void vcycle_unfused(wec_poisson *P, Level<T> *L, const T *b0, T *x0, const int *bsel, const int *xsel,
                    cudaStream_t st)
{
    const int TB = 256;
    const double ts = sizeof(T);
    for (int l = 0; l < P->nlev; ++l) {
        Level<T> &A = L[l];
        const T *b = l == 0 ? b0 : A.b;
        T *x = l == 0 ? x0 : A.x;
        const int *bs = l == 0 ? bsel : nullptr, *xs = l == 0 ? xsel : nullptr;
        const double n = (double)A.nx * A.ny, nf = (double)(A.nx + 1) * A.ny + (double)A.nx * (A.ny + 1);
        if (l == P->nlev - 1) {
            T *lu = nullptr;
            if constexpr (sizeof(T) == 8) lu = (T *)P->lu64; else lu = (T *)P->lu32;
            WEC_PROF("mg_lu_solve", l, (n * n + 2 * n) * ts, st);
            launch_k(k_lu_solve<T>, 1, 32, 0, st, A.nx * A.ny, lu, b, x, bs, xs);
            break;
        }
        int nh = (A.nx >> 1) * A.ny;
        for (int q = 0; q < P->nu1; ++q) {
            {
                WEC_PROF("mg_rbgs", l, (1.5 * n + nf) * ts, st);
                launch_k(k_rbgs<T>, nblk(nh, TB), TB, 0, st, A.nx, A.ny, A.bu, A.bv, x, b, 0, q == 0, bs, xs);
            }
            {
                WEC_PROF("mg_rbgs", l, (1.5 * n + nf) * ts, st);
                launch_k(k_rbgs<T>, nblk(nh, TB), TB, 0, st, A.nx, A.ny, A.bu, A.bv, x, b, 1, 0, bs, xs);
            }
        }
        Level<T> &C = L[l + 1];
        WEC_PROF("mg_resid_restrict", l, (2.25 * n + nf) * ts, st);
        launch_k(k_resid_restrict<T>, nblk(C.nx * C.ny, TB), TB, 0, st, A.nx, A.ny, A.bu, A.bv, x, b, C.b, bs, xs);
    }
    for (int l = P->nlev - 2; l >= 0; --l) {
        Level<T> &A = L[l];
        const T *b = l == 0 ? b0 : A.b;
        T *x = l == 0 ? x0 : A.x;
        const int *bs = l == 0 ? bsel : nullptr, *xs = l == 0 ? xsel : nullptr;
        const double n = (double)A.nx * A.ny, nf = (double)(A.nx + 1) * A.ny + (double)A.nx * (A.ny + 1);
        int nh = (A.nx >> 1) * A.ny;
        {
            WEC_PROF("mg_prolong", l, 2.25 * n * ts, st);
            launch_k(k_prolong<T>, nblk(A.nx * A.ny, TB), TB, 0, st, A.nx, A.ny, x, L[l + 1].x, xs);
        }
        for (int q = 0; q < P->nu2; ++q) {
            {
                WEC_PROF("mg_rbgs", l, (1.5 * n + nf) * ts, st);
                launch_k(k_rbgs<T>, nblk(nh, TB), TB, 0, st, A.nx, A.ny, A.bu, A.bv, x, b, 0, 0, bs, xs);
            }
            {
                WEC_PROF("mg_rbgs", l, (1.5 * n + nf) * ts, st);
                launch_k(k_rbgs<T>, nblk(nh, TB), TB, 0, st, A.nx, A.ny, A.bu, A.bv, x, b, 1, 0, bs, xs);
            }
        }
    }
}

template <typename T, int TX, int TY>
int set_attrs_one()
{
    const int mx = (int)tile_smem<T>(8, TX, TY);
    WEC_CK(cudaFuncSetAttribute(k_mg_pre<T, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    WEC_CK(cudaFuncSetAttribute(k_mg_post<T, TX, TY, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    if constexpr (sizeof(T) == 4)
        WEC_CK(cudaFuncSetAttribute(k_mg_post<T, TX, TY, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    return WEC_OK;
}

int set_tile_attrs()
{
    int e = set_attrs_one<double, 64, 16>();
    if (!e) e = set_attrs_one<double, 32, 16>();
    if (!e) e = set_attrs_one<double, 32, 8>();
    if (!e) e = set_attrs_one<double, 16, 8>();
    if (!e) e = set_attrs_one<float, 64, 16>();
    if (!e) e = set_attrs_one<float, 32, 16>();
    if (!e) e = set_attrs_one<float, 32, 8>();
    if (!e) e = set_attrs_one<float, 16, 8>();
    return e;
}

template <typename T, int TX, int TY>
void launch_pre_t(const Level<T> &A, const T *b, T *bc, int nu1, int H, const int *bsel, cudaStream_t st)
{
    dim3 grid((A.nx + TX - 1) / TX, (A.ny + TY - 1) / TY);
    launch_k(k_mg_pre<T, TX, TY>, grid, 256, tile_smem<T>(H, TX, TY), st, A.nx, A.ny, A.bu, A.bv, b, A.id, A.xp, bc, nu1,
                                                                     H, bsel);
}

template <typename T, int TX, int TY, typename TO>
void launch_post_t(const Level<T> &A, const T *b, TO *x, const T *xc, int nu2, int H, const int *bsel,
                   const int *xsel, cudaStream_t st)
{
    dim3 grid((A.nx + TX - 1) / TX, (A.ny + TY - 1) / TY);
    launch_k(k_mg_post<T, TX, TY, TO>, grid, 256, tile_smem<T>(H, TX, TY), st, A.nx, A.ny, A.bu, A.bv, b, A.id, A.xp, x,
                                                                         xc, nu2, H, bsel, xsel);
}

template <typename T>
void launch_pre(int tile, const Level<T> &A, const T *b, T *bc, int nu1, int H, const int *bsel, cudaStream_t st)
{
    switch (tile) {
    case 1: launch_pre_t<T, 32, 16>(A, b, bc, nu1, H, bsel, st); break;
    case 2: launch_pre_t<T, 32, 8>(A, b, bc, nu1, H, bsel, st); break;
    case 3: launch_pre_t<T, 16, 8>(A, b, bc, nu1, H, bsel, st); break;
    default: launch_pre_t<T, 64, 16>(A, b, bc, nu1, H, bsel, st); break;
    }
}

template <typename T, typename TO>
void launch_post(int tile, const Level<T> &A, const T *b, TO *x, const T *xc, int nu2, int H, const int *bsel,
                 const int *xsel, cudaStream_t st)
{
    switch (tile) {
    case 1: launch_post_t<T, 32, 16, TO>(A, b, x, xc, nu2, H, bsel, xsel, st); break;
    case 2: launch_post_t<T, 32, 8, TO>(A, b, x, xc, nu2, H, bsel, xsel, st); break;
    case 3: launch_post_t<T, 16, 8, TO>(A, b, x, xc, nu2, H, bsel, xsel, st); break;
    default: launch_post_t<T, 64, 16, TO>(A, b, x, xc, nu2, H, bsel, xsel, st); break;
    }
}

// Fused V-cycle: per fine level one pre and one post kernel, one CTA for the
// levels of at most kBottomCells cells.  The level-0 result x0 is stored in TO.
template <typename T, typename TO>
void vcycle_fused(wec_poisson *P, Level<T> *L, const T *b0, TO *x0, const int *bsel, const int *xsel,
                  cudaStream_t st)
{
    const double ts = sizeof(T);
    const int H = 2 * std::max(P->nu1, P->nu2);
    const int *tiles = sizeof(T) == 8 ? P->tile64 : P->tile32;
    BottomLevels<T> B;
    B.nlev = P->nlev;
    B.nu1 = P->nu1;
    B.nu2 = P->nu2;
    if constexpr (sizeof(T) == 8) {
        B.lu = (const T *)P->lu64;
        B.inv = (const T *)P->inv64;
    } else {
        B.lu = (const T *)P->lu32;
        B.inv = (const T *)P->inv32;
    }
    for (int l = 0; l < P->nlev; ++l) {
        B.nx[l] = L[l].nx;
        B.ny[l] = L[l].ny;
        B.bu[l] = L[l].bu;
        B.bv[l] = L[l].bv;
        B.id[l] = L[l].id;
        B.x[l] = l == 0 ? nullptr : L[l].x;
        B.b[l] = l == 0 ? (T *)b0 : L[l].b;
    }
    if constexpr (std::is_same<T, TO>::value) {
        B.x[0] = x0;
        B.x0d = nullptr;
    } else {
        B.x0d = x0;  // FP32 levels, FP64 level-0 result
    }
    // first level small enough, whose staging (with all coarser levels) fits in shared memory
    int lb = 0;
    while (lb < P->nlev - 1 &&
           ((long long)L[lb].nx * L[lb].ny > kBottomCells || bottom_elems(B, lb) * (long long)sizeof(T) > kBottomSmemMax))
        ++lb;
    lb = std::min(lb + P->bottom_shift, P->nlev - 1);  // autotuned: coarser levels may run faster in one CTA
    B.lb = lb;
    P->bottom_level = lb;
    for (int l = 0; l < lb; ++l) {
        Level<T> &A = L[l];
        const double n = (double)A.nx * A.ny, nf = (double)(A.nx + 1) * A.ny + (double)A.nx * (A.ny + 1);
        WEC_PROF("mg_pre", l, (2.25 * n + nf) * ts, st);
        launch_pre<T>(tiles[l], A, l == 0 ? b0 : A.b, L[l + 1].b, P->nu1, H, l == 0 ? bsel : nullptr, st);
    }
    {
        // algorithmic bytes: b and x of level lb, every level's coefficients, the LU
        const double nb = (double)L[lb].nx * L[lb].ny, nc = (double)L[P->nlev - 1].nx * L[P->nlev - 1].ny;
        double bytes = (2.0 * nb + nc * nc) * ts;
        for (int l = lb; l < P->nlev; ++l) bytes += ((L[l].nx + 1.0) * L[l].ny + L[l].nx * (L[l].ny + 1.0)) * ts;
        const size_t smem_b = (size_t)bottom_elems(B, lb) * sizeof(T);
        WEC_PROF("mg_bottom", lb, bytes, st);
        launch_k(k_mg_bottom<T>, 1, kBottomThreads, smem_b, st, B, bsel, xsel);
    }
    for (int l = lb - 1; l >= 0; --l) {
        Level<T> &A = L[l];
        const double n = (double)A.nx * A.ny, nf = (double)(A.nx + 1) * A.ny + (double)A.nx * (A.ny + 1);
        WEC_PROF("mg_post", l, (3.25 * n + nf) * ts, st);
        if (l == 0)
            launch_post<T, TO>(tiles[0], A, b0, x0, L[1].x, P->nu2, H, bsel, xsel, st);
        else
            launch_post<T, T>(tiles[l], A, A.b, A.x, L[l + 1].x, P->nu2, H, nullptr, nullptr, st);
    }
}

bool g_mg_autotune = true;     // wec_set_option "mg_autotune"
int g_mg_bottom_shift = -1;    // wec_set_option "mg_bottom_shift" (-1: autotune)

// Autotuner of the fused level kernels: on each non-coarsest level, time the
// pre + post pair of every tile shape (3 runs each, CUDA events on the solver's
// stream) and keep the fastest.  Runs once per solver, on placeholder
// coefficients (all 1), before anything is captured.
template <typename T>
int autotune_levels(wec_poisson *P, Level<T> *L, int *tiles, cudaStream_t st)
{
    const int H = 2 * std::max(P->nu1, P->nu2);
    cudaEvent_t e0, e1;
    WEC_CK(cudaEventCreate(&e0));
    WEC_CK(cudaEventCreate(&e1));
    int rc = WEC_OK;
    for (int l = 0; l + 1 < P->nlev && rc == WEC_OK; ++l) {
        Level<T> &A = L[l];
        const long long n = (long long)A.nx * A.ny;
        T *b = l == 0 ? (T *)P->w : A.b;  // scratch stand-ins for the level-0 vectors
        T *x = l == 0 ? (T *)P->w : A.x;
        if (l == 0 && !A.b) cudaMemsetAsync(P->w, 0, n * sizeof(double), st);
        float best = 1e30f;
        tiles[l] = 0;
        for (int t = 0; t < kNumTiles; ++t) {
            float tmin = 1e30f;
            for (int r = 0; r < 3; ++r) {
                cudaEventRecord(e0, st);
                launch_pre<T>(t, A, b, L[l + 1].b, P->nu1, H, nullptr, st);
                launch_post<T, T>(t, A, b, x, L[l + 1].x, P->nu2, H, nullptr, nullptr, st);
                cudaEventRecord(e1, st);
                cudaError_t e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "autotune timing");
                    break;
                }
                if (r > 0) tmin = std::min(tmin, ms);  // first run warms up
            }
            if (rc != WEC_OK) break;
            if (tmin < best) {
                best = tmin;
                tiles[l] = t;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

// Where the single-CTA bottom starts: time whole fused V-cycles with the bottom
// at the smallest admissible level and up to two levels coarser (tiled kernels
// above it), keep the fastest.  Runs after the tile shapes are tuned.
template <typename T>
int autotune_bottom(wec_poisson *P, Level<T> *L, cudaStream_t st)
{
    cudaEvent_t e0, e1;
    WEC_CK(cudaEventCreate(&e0));
    WEC_CK(cudaEventCreate(&e1));
    // level-0 stand-ins in V (at least 2 n doubles; overwritten at the start of every solve)
    const long long n0 = (long long)L[0].nx * L[0].ny;
    T *b = (T *)P->V, *x = (T *)P->V + n0;
    float best = 1e30f;
    int best_shift = 0;
    for (int shift = 0; shift <= 2; ++shift) {
        P->bottom_shift = shift;
        vcycle_fused<T, T>(P, L, b, x, nullptr, nullptr, st);  // sets bottom_level
        if (shift > 0 && P->bottom_level >= P->nlev - 1) break;
        float tmin = 1e30f;
        for (int r = 0; r < 4; ++r) {
            cudaEventRecord(e0, st);
            vcycle_fused<T, T>(P, L, b, x, nullptr, nullptr, st);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            tmin = std::min(tmin, ms);
        }
        if (tmin < best) {
            best = tmin;
            best_shift = shift;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    P->bottom_shift = best_shift;
    vcycle_fused<T, T>(P, L, b, x, nullptr, nullptr, st);  // records the chosen bottom level
    const cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? WEC_OK : cuda_fail(ce, "autotune_bottom");
}

template <typename T>
__global__ void k_fill(long long n, T *a, T v)
{
    pdl_entry();
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c < n) a[c] = v;
}

// Tuning results per (nx, ny, precision, nu1, nu2), shared by every solver of
// the process: the first solver of a shape times the candidates, later ones
// reuse its choices, so equal tanks run the same kernels and give the same bits
// (the bottom split changes rounding; timings alone would not repeat).
struct TuneResult {
    int tile[kMaxLevels];
    int bottom_shift, bottom_level;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, TuneResult> g_tune_cache;

int poisson_autotune(wec_poisson *P, cudaStream_t st)
{
    for (int l = 0; l < kMaxLevels; ++l) P->tile64[l] = P->tile32[l] = 0;
    P->bottom_shift = g_mg_bottom_shift > 0 ? g_mg_bottom_shift : 0;
    if (!g_mg_autotune || P->nlev < 2) return WEC_OK;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const auto key = std::make_tuple(P->nx, P->ny, P->prec, P->nu1, P->nu2);
    int *tiles = P->prec == WEC_PREC_FP64 ? P->tile64 : P->tile32;
    auto hit = g_tune_cache.find(key);
    if (hit != g_tune_cache.end()) {
        for (int l = 0; l < kMaxLevels; ++l) tiles[l] = hit->second.tile[l];
        P->bottom_shift = g_mg_bottom_shift >= 0 ? g_mg_bottom_shift : hit->second.bottom_shift;
        P->bottom_level = g_mg_bottom_shift >= 0 ? -1 : hit->second.bottom_level;
        P->tuned = true;
        return WEC_OK;
    }
    // placeholder coefficients (the real ones are set before every solve)
    for (int l = 0; l < P->nlev; ++l) {
        long long nu = (long long)(P->L64[l].nx + 1) * P->L64[l].ny, nv = (long long)P->L64[l].nx * (P->L64[l].ny + 1);
        launch_k(k_fill<double>, nblk(nu, 256), 256, 0, st, nu, P->L64[l].bu, 1.0);
        launch_k(k_fill<double>, nblk(nv, 256), 256, 0, st, nv, P->L64[l].bv, 1.0);
        if (P->prec == WEC_PREC_MIXED) {
            launch_k(k_fill<float>, nblk(nu, 256), 256, 0, st, nu, P->L32[l].bu, 1.0f);
            launch_k(k_fill<float>, nblk(nv, 256), 256, 0, st, nv, P->L32[l].bv, 1.0f);
        }
    }
    // the placeholder operator's hierarchy, diagonals and coarsest factors, so the
    // trial V-cycles run on finite values
    if (int e = poisson_build(P, st)) return e;
    int e = P->prec == WEC_PREC_FP64 ? autotune_levels<double>(P, P->L64, P->tile64, st)
                                     : autotune_levels<float>(P, P->L32, P->tile32, st);
    if (!e && g_mg_bottom_shift < 0)
        e = P->prec == WEC_PREC_FP64 ? autotune_bottom<double>(P, P->L64, st) : autotune_bottom<float>(P, P->L32, st);
    if (e) return e;
    if (g_mg_bottom_shift < 0) {  // a forced split is not a tuning result
        TuneResult r;
        for (int l = 0; l < kMaxLevels; ++l) r.tile[l] = tiles[l];
        r.bottom_shift = P->bottom_shift;
        r.bottom_level = P->bottom_level;
        g_tune_cache[key] = r;
    } else {
        P->bottom_shift = g_mg_bottom_shift;
    }
    P->have_coef = false;  // the real operator must still be set
    P->tuned = true;
    WEC_CK(cudaStreamSynchronize(st));
    return WEC_OK;
}

// x0 = M^{-1} b0 by one V-cycle over the levels L (precision T); the level-0
// result is stored in TO (an FP32 V-cycle may deliver FP64).
template <typename T, typename TO>
void vcycle_t(wec_poisson *P, Level<T> *L, const T *b0, TO *x0, const int *bsel, const int *xsel, cudaStream_t st)
{
    if (P->nz > 1) {
        vcycle3_t<T, TO>(P, L, b0, x0, bsel, xsel, st);
    } else if (g_mg_fused) {
        vcycle_fused<T, TO>(P, L, b0, x0, bsel, xsel, st);
    } else if constexpr (std::is_same<T, TO>::value) {
        vcycle_unfused<T>(P, L, b0, x0, bsel, xsel, st);
    } else {
        // one-pass kernels smooth in place: run on the FP32 level-0 scratch, then widen
        const long long n = (long long)L[0].nx * L[0].ny;
        vcycle_unfused<T>(P, L, b0, L[0].x, bsel, nullptr, st);
        WEC_PROF("convert", 0, 12.0 * n, st);
        launch_k(k_widen, nblk(n, 256), 256, 0, st, n, L[0].x, x0, xsel);
    }
}

// CTAs of the cluster reduction kernels that run as one wave on this GPU: the
// scheduler places whole clusters inside a GPC, so the count comes from the
// occupancy query, not from SMs x CTAs per SM.  Set once by poisson_init.
// the largest grid (CTAs) of each Krylov reduction kernel: its resident
// clusters, at most kKrylovBlocks; res[d3], mv[d3][restart <= 8], od[restart <= 8]
struct KGrids {
    int bnorm = kCl, on = kCl, res[2] = {kCl, kCl}, mv[2][2] = {{kCl, kCl}, {kCl, kCl}}, od[2] = {kCl, kCl};
    // the float-pair Arnoldi kernels (3D): residual, matvec[restart <= 8], orth dots[restart <= 8], orth norm
    int res_df = kCl, mv_df[2] = {kCl, kCl}, od_df[2] = {kCl, kCl}, on_df = kCl;
    int mv_df4 = kCl, od_df4 = kCl;  // their variants for at most 4 basis vectors (more CTAs per SM)
};
KGrids g_kg;

template <typename K>
int clusters_resident(K kern, int *out)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kCl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(kKrylovBlocks);
    cfg.blockDim = dim3(KT);
    cfg.attrs = at;
    cfg.numAttrs = 1;
    WEC_CK(cudaOccupancyMaxActiveClusters(out, (void *)kern, &cfg));
    return WEC_OK;
}

int set_kgrid_max()
{
    // at most 4 CTAs per SM (608), the four-vector pair kernels 6 (912)
    auto r = [](auto kern, int &g, int cap = 4 * 152) {
        int c = 0;
        if (int e = clusters_resident(kern, &c)) return e;
        g = std::max(1, std::min(c, cap / kCl)) * kCl;
        return (int)WEC_OK;
    };
    KGrids &k = g_kg;
    int e = r(k_bnorm, k.bnorm);
    if (!e) e = r(k_orth_norm<double>, k.on);
    if (!e) e = r(k_residual_norm<2>, k.res[0]);
    if (!e) e = r(k_residual_norm<3>, k.res[1]);
    if (!e) e = r(k_matvec_dots<2, 32>, k.mv[0][0]);
    if (!e) e = r(k_matvec_dots<2, 8>, k.mv[0][1]);
    if (!e) e = r(k_matvec_dots<3, 32>, k.mv[1][0]);
    if (!e) e = r(k_matvec_dots<3, 8>, k.mv[1][1]);
    if (!e) e = r(k_orth_dots<32>, k.od[0]);
    if (!e) e = r(k_orth_dots<8>, k.od[1]);
    if (!e) e = r(k_residual_norm<3, df64>, k.res_df);
    if (!e) e = r(k_matvec_dots<3, 32, df64, float>, k.mv_df[0]);
    if (!e) e = r(k_matvec_dots<3, 8, df64, float>, k.mv_df[1]);
    if (!e) e = r(k_matvec_dots<3, 4, df64, float>, k.mv_df4, kKrylovBlocks);
    if (!e) e = r(k_orth_dots<4, df64>, k.od_df4, kKrylovBlocks);
    if (!e) e = r(k_orth_dots<32, df64>, k.od_df[0]);
    if (!e) e = r(k_orth_dots<8, df64>, k.od_df[1]);
    if (!e) e = r(k_orth_norm<df64>, k.on_df, kKrylovBlocks);
    return e;
}

// Reduction kernels: a multiple of the cluster size, at most one wave of the
// kernel's resident clusters (gmax).  Vectors that stay in L2 (up to 2^22
// cells) take at most 2 CTAs per SM: those passes are latency-bound and half
// the partials shorten the final reduction.
int kgrid(long long n, int gmax)
{
    if (n <= (1ll << 22)) gmax = std::min(gmax, 2 * 152);
    const long long g = std::min<long long>(nblk(n, KT), gmax);
    return (int)((g + kCl - 1) / kCl * kCl);
}

// ---------------------------------------------------------- FGMRES parts ----
Op0 op0(const wec_poisson *P)
{
    return Op0{P->nx, P->ny, P->nz, P->L64[0].bu, P->L64[0].bv, P->L64[0].bw};
}
// the pair copies of the level-0 operator (P->kdf)
OpT<df64> op0df(const wec_poisson *P)
{
    return OpT<df64>{P->nx, P->ny, P->nz, (const df64 *)P->kdf_face[0], (const df64 *)P->kdf_face[1],
                     (const df64 *)P->kdf_face[2]};
}

long long ncells(const wec_poisson *P) { return (long long)P->nx * P->ny * P->nz; }

// faces of the level-0 operator (bytes accounting)
double nfaces(const wec_poisson *P)
{
    const double nx = P->nx, ny = P->ny, nz = P->nz;
    if (P->nz == 1) return (nx + 1.0) * ny + nx * (ny + 1.0);
    return (nx + 1.0) * ny * nz + nx * (ny + 1.0) * nz + nx * ny * (nz + 1.0);
}

void launch_residual_norm(wec_poisson *P, const double *b, double *x, float *b32, int mode, unsigned long long hw,
                          int use, cudaStream_t st)
{
    if (P->kdf) {  // (3D) the FP64 residual into the pair basis
        launch_k(k_residual_norm<3, df64>, kgrid(ncells(P), g_kg.res_df), KT, 0, st, op0(P), P->d0, b, x,
                 (df64 *)P->V, b32, P->sc, P->part, P->ks, P->g, mode, hw, use);
        return;
    }
    const int G = kgrid(ncells(P), g_kg.res[P->nz > 1 ? 1 : 0]);
    if (P->nz > 1)
        launch_k(k_residual_norm<3>, G, KT, 0, st, op0(P), P->d0, b, x, P->V, b32, P->sc, P->part, P->ks, P->g, mode,
                 hw, use);
    else
        launch_k(k_residual_norm<2>, G, KT, 0, st, op0(P), P->d0, b, x, P->V, b32, P->sc, P->part, P->ks, P->g, mode,
                 hw, use);
}

void enqueue_begin(wec_poisson *P, const double *b, double *x, double rtol, int maxit, unsigned long long hw,
                   int use, cudaStream_t st)
{
    const long long n = ncells(P);
    const double nf = nfaces(P);
    float *b32 = P->prec == WEC_PREC_MIXED ? P->L32[0].b : nullptr;
    {
        WEC_PROF("scalar", -1, 64.0, st);
        launch_k(k_ks_init, 1, 1, 0, st, P->ks, rtol, maxit, P->restart);
    }
    {
        WEC_PROF("krylov_norm", -1, 8.0 * n, st);
        launch_k(k_bnorm, kgrid(n, g_kg.bnorm), KT, 0, st, n, b, P->part, P->ks);
    }
    WEC_PROF("krylov_residual", -1, 8.0 * (4.0 * n + nf) + (b32 ? 4.0 * n : 0.0), st);
    launch_residual_norm(P, b, x, b32, 0, hw, use, st);
}

// One Arnoldi step j (preconditioner, matvec, CGS2 in place in V's column j+1,
// Givens).  Algorithmic bytes of the Krylov kernels are counted at the largest
// j (m - 1).  jh: j when the host knows it (a host-polled solve reads the state
// after every step), else -1; with j + 1 <= 4 the pair Arnoldi step takes the
// kernels compiled for at most four basis vectors (fewer registers, more CTAs
// per SM; the kernels still read j on the device).
void enqueue_body(wec_poisson *P, unsigned long long hif, int use, cudaStream_t st, int jh = -1)
{
    const long long n = ncells(P);
    const double nf = nfaces(P);
    const int m = P->restart, d3 = P->nz > 1 ? 1 : 0, kb8 = m <= 8 ? 1 : 0;
    const bool mixed = P->prec == WEC_PREC_MIXED;
    double *h1 = P->dots, *h2 = P->dots + (kMaxRestart + 2);
    // the mixed V-cycle reads u_j in FP32, written beside it by k_residual_norm / k_orth_norm
    if (P->kdf) {  // (3D, FP32 V-cycles) the float-pair Arnoldi step
        vcycle3_t<float, float>(P, P->L32, P->L32[0].b, (float *)P->Z, nullptr, &P->ks->j, st);
        const bool k4 = jh >= 0 && jh + 1 <= 4;
        {
            WEC_PROF("krylov_matvec_dots", -1, 8.0 * (2.0 * n + nf) + 4.0 * n + 8.0 * n * m, st);
            auto kern = k4    ? k_matvec_dots<3, 4, df64, float>
                        : kb8 ? k_matvec_dots<3, 8, df64, float>
                              : k_matvec_dots<3, 32, df64, float>;
            launch_k(kern, kgrid(n, k4 ? g_kg.mv_df4 : g_kg.mv_df[kb8]), KT, 0, st, op0df(P),
                     (const df64 *)P->kdf_d0, (const float *)P->Z, (df64 *)P->V, P->sc, P->part, h1, P->ks);
        }
        {
            WEC_PROF("krylov_orth_dots", -1, 8.0 * n * (m + 2), st);
            auto kern = k4 ? k_orth_dots<4, df64> : kb8 ? k_orth_dots<8, df64> : k_orth_dots<32, df64>;
            launch_k(kern, kgrid(n, k4 ? g_kg.od_df4 : g_kg.od_df[kb8]), KT, 0, st, n, (df64 *)P->V, P->sc, h1,
                     P->part, h2, P->ks);
        }
        WEC_PROF("krylov_orth_norm", -1, 8.0 * n * (m + 2) + 4.0 * n, st);
        launch_k(k_orth_norm<df64>, kgrid(n, g_kg.on_df), KT, 0, st, n, (df64 *)P->V, P->sc, P->L32[0].b, h1, h2,
                 P->part, P->ks, P->hess, P->cs, P->sn, P->g, hif, use);
        return;
    }
    if (!mixed)
        vcycle_t<double, double>(P, P->L64, P->V, P->Z, &P->ks->j, &P->ks->j, st);
    else
        vcycle_t<float, double>(P, P->L32, P->L32[0].b, P->Z, nullptr, &P->ks->j, st);
    {
        WEC_PROF("krylov_matvec_dots", -1, 8.0 * (3.0 * n + nf) + 8.0 * n * m, st);
        auto kern = d3 ? (kb8 ? k_matvec_dots<3, 8> : k_matvec_dots<3, 32>)
                       : (kb8 ? k_matvec_dots<2, 8> : k_matvec_dots<2, 32>);
        launch_k(kern, kgrid(n, g_kg.mv[d3][kb8]), KT, 0, st, op0(P), P->d0, P->Z, P->V, P->sc, P->part, h1, P->ks);
    }
    {
        WEC_PROF("krylov_orth_dots", -1, 8.0 * n * (m + 2), st);
        launch_k(kb8 ? k_orth_dots<8> : k_orth_dots<32>, kgrid(n, g_kg.od[kb8]), KT, 0, st, n, P->V, P->sc, h1,
                 P->part, h2, P->ks);
    }
    WEC_PROF("krylov_orth_norm", -1, 8.0 * n * (m + 2) + (mixed ? 4.0 * n : 0.0), st);
    launch_k(k_orth_norm<double>, kgrid(n, g_kg.on), KT, 0, st, n, P->V, P->sc, mixed ? P->L32[0].b : nullptr, h1, h2, P->part, P->ks,
             P->hess, P->cs, P->sn, P->g, hif, use);
}

// End of a cycle: y from the triangular system, x += Z y, true residual, then
// converge / stop / restart.
void enqueue_close(wec_poisson *P, const double *b, double *x, unsigned long long hw, int use, cudaStream_t st)
{
    const long long n = ncells(P);
    const double nf = nfaces(P);
    const int m = P->restart;
    const bool mixed = P->prec == WEC_PREC_MIXED;
    {
        WEC_PROF("scalar", -1, 8.0 * m * m, st);
        launch_k(k_backsolve, 1, 1, 0, st, m, P->hess, P->g, P->y, P->sc, P->ks);
    }
    {
        WEC_PROF("krylov_update_x", -1, 16.0 * n + (P->kdf ? 4.0 : 8.0) * n * m, st);
        if (P->kdf)
            launch_k(k_update_x<float>, nblk(n, 256), 256, 0, st, n, P->y, (const float *)P->Z, x, P->ks);
        else
            launch_k(k_update_x<double>, nblk(n, 256), 256, 0, st, n, P->y, P->Z, x, P->ks);
    }
    WEC_PROF("krylov_residual", -1, 8.0 * (4.0 * n + nf) + (mixed ? 4.0 * n : 0.0), st);
    launch_residual_norm(P, b, x, mixed ? P->L32[0].b : nullptr, 1, hw, use, st);
}

int read_state(wec_poisson *P, cudaStream_t st)
{
    WEC_CK(cudaMemcpyAsync(P->ksh, P->ks, sizeof(KState), cudaMemcpyDeviceToHost, st));
    WEC_CK(cudaStreamSynchronize(st));
    return WEC_OK;
}

}  // namespace

void set_mg_fused(bool on) { g_mg_fused = on; }
void set_mg_autotune(bool on) { g_mg_autotune = on; }
void set_mg3_bottom(bool on) { g_mg3_bottom = on; }
void set_mg_bottom_shift(int shift) { g_mg_bottom_shift = shift; }

void poisson_tiles(const wec_poisson *P, int *tx, int *ty, int max)
{
    const int *t = P->prec == WEC_PREC_FP64 ? P->tile64 : P->tile32;
    for (int l = 0; l < max && l < P->nlev; ++l) {
        const bool tiled = P->nz == 1 && (P->bottom_level < 0 || l < P->bottom_level);  // 0 x 0: not a fused tile
        tx[l] = tiled ? kTileX[t[l]] : 0;
        ty[l] = tiled ? kTileY[t[l]] : 0;
    }
}

int poisson_init(wec_poisson *P, int nx, int ny, int prec, int restart, int nu1, int nu2, cudaStream_t st, int nz)
{
    static bool attrs_done = false;
    if (!attrs_done) {
        // shared-memory tiles of the fused level kernels exceed the 48 KB default (H <= 8)
        if (int e = set_tile_attrs()) return e;
        WEC_CK(cudaFuncSetAttribute(k_mg_bottom<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBottomSmemMax));
        WEC_CK(cudaFuncSetAttribute(k_mg_bottom<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBottomSmemMax));
        WEC_CK(cudaFuncSetAttribute(k3_bottom<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBottom3Smem));
        WEC_CK(cudaFuncSetAttribute(k3_bottom<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBottom3Smem));
        if (int e = set_kgrid_max()) return e;
        attrs_done = true;
    }
    if (nx < 2 || ny < 2 || nz < 1) return fail(WEC_ERR_INVALID, "poisson: nx, ny must be >= 2");
    if (nz > 1) {  // 3D: every face array below 2^31 entries (32-bit index arithmetic in the kernels)
        const long long big = std::max({(long long)(nx + 1) * ny * nz, (long long)nx * (ny + 1) * nz,
                                        (long long)nx * ny * (nz + 1)});
        if (big >= (1ll << 31)) return fail(WEC_ERR_INVALID, "poisson: 3D grid too large (a face array >= 2^31)");
    }
    if (restart < 1 || restart > kMaxRestart) return fail(WEC_ERR_INVALID, "poisson: restart must be in 1..32");
    if (nu1 < 1 || nu2 < 0 || nu1 > 4 || nu2 > 4)
        return fail(WEC_ERR_INVALID, "poisson: need 1 <= mg_pre <= 4 and 0 <= mg_post <= 4");
    // WEC_PREC_MIXED_DF (3D): FP32 V-cycles and the Arnoldi step in float pairs
    bool kdf = false;
    if (prec == WEC_PREC_MIXED_DF) {
        if (nz <= 1) return fail(WEC_ERR_INVALID, "poisson: WEC_PREC_MIXED_DF is for the 3D operator");
        prec = WEC_PREC_MIXED;
        kdf = true;
    }
    if (prec != WEC_PREC_FP64 && prec != WEC_PREC_MIXED) return fail(WEC_ERR_INVALID, "poisson: unknown precision");
    P->nx = nx; P->ny = ny; P->nz = nz; P->prec = prec; P->restart = restart; P->nu1 = nu1; P->nu2 = nu2; P->st = st;
    P->kdf = kdf;
    const bool d3 = nz > 1;
    int lx = nx, ly = ny, lz = nz, nl = 0;
    for (;;) {
        P->L64[nl].nx = lx; P->L64[nl].ny = ly; P->L64[nl].nz = lz;
        P->L32[nl].nx = lx; P->L32[nl].ny = ly; P->L32[nl].nz = lz;
        nl++;
        if ((lx & 1) || (ly & 1) || lx < 4 || ly < 4 || nl == kMaxLevels) break;
        if (d3 && ((lz & 1) || lz < 4)) break;
        lx >>= 1; ly >>= 1;
        if (d3) lz >>= 1;
    }
    P->nlev = nl;
    P->ncoarse = lx * ly * lz;
    if (P->ncoarse > kMaxCoarse)
        return fail(WEC_ERR_INVALID, "poisson: the grid must coarsen (by halving even sizes) to at most 512 cells; got " +
                                         std::to_string(lx) + "x" + std::to_string(ly) +
                                         (d3 ? "x" + std::to_string(lz) : std::string()));
    for (int l = 0; l < nl; ++l) {
        const size_t Nx = P->L64[l].nx, Ny = P->L64[l].ny, Nz = P->L64[l].nz;
        size_t nc = Nx * Ny * Nz;
        size_t nu = (Nx + 1) * Ny * Nz, nv = Nx * (Ny + 1) * Nz, nw = d3 ? Nx * Ny * (Nz + 1) : 0;
        WEC_CK(cudaMalloc(&P->L64[l].bu, nu * 8));
        WEC_CK(cudaMalloc(&P->L64[l].bv, nv * 8));
        WEC_CK(cudaMemset(P->L64[l].bu, 0, nu * 8));
        WEC_CK(cudaMemset(P->L64[l].bv, 0, nv * 8));
        if (d3) {
            WEC_CK(cudaMalloc(&P->L64[l].bw, nw * 8));
            WEC_CK(cudaMemset(P->L64[l].bw, 0, nw * 8));
        }
        if (l > 0) {
            WEC_CK(cudaMalloc(&P->L64[l].x, nc * 8));
            WEC_CK(cudaMalloc(&P->L64[l].b, nc * 8));
        }
        P->bytes += (nu + nv + nw) * 8 + (l > 0 ? 2 * nc * 8 : 0);
        if (l < nl - 1 && !d3) {  // may be a tiled level of the fused V-cycle
            WEC_CK(cudaMalloc(&P->L64[l].xp, nc * 8));
            if (prec == WEC_PREC_MIXED) WEC_CK(cudaMalloc(&P->L32[l].xp, nc * 4));
        }
        if (prec == WEC_PREC_FP64) {
            WEC_CK(cudaMalloc(&P->L64[l].id, nc * 8));
            WEC_CK(cudaMemset(P->L64[l].id, 0, nc * 8));
        }
        if (prec == WEC_PREC_MIXED) {
            WEC_CK(cudaMalloc(&P->L32[l].id, nc * 4));
            WEC_CK(cudaMemset(P->L32[l].id, 0, nc * 4));
            WEC_CK(cudaMalloc(&P->L32[l].bu, nu * 4));
            WEC_CK(cudaMalloc(&P->L32[l].bv, nv * 4));
            if (d3) WEC_CK(cudaMalloc(&P->L32[l].bw, nw * 4));
            WEC_CK(cudaMalloc(&P->L32[l].x, nc * 4));
            WEC_CK(cudaMalloc(&P->L32[l].b, nc * 4));
            P->bytes += (nu + nv + nw + 2 * nc) * 4;
        }
    }
    WEC_CK(cudaMalloc(&P->lu64, (size_t)P->ncoarse * P->ncoarse * 8));
    if (prec == WEC_PREC_MIXED) WEC_CK(cudaMalloc(&P->lu32, (size_t)P->ncoarse * P->ncoarse * 4));
    if (P->ncoarse <= kInvMax) {
        if (prec == WEC_PREC_FP64)
            WEC_CK(cudaMalloc(&P->inv64, (size_t)P->ncoarse * P->ncoarse * 8));
        else
            WEC_CK(cudaMalloc(&P->inv32, (size_t)P->ncoarse * P->ncoarse * 4));
    }
    size_t n = (size_t)nx * ny * nz;
    int m = restart;
    WEC_CK(cudaMalloc(&P->V, (m + 1) * n * 8));
    WEC_CK(cudaMalloc(&P->Z, m * n * 8));
    WEC_CK(cudaMalloc(&P->w, n * 8));
    WEC_CK(cudaMalloc(&P->d0, n * 8));
    if (P->kdf) {  // pair copies of the level-0 operator: faces and diagonal
        const size_t nf3[3] = {(size_t)(nx + 1) * ny * nz, (size_t)nx * (ny + 1) * nz, (size_t)nx * ny * (nz + 1)};
        for (int q = 0; q < 3; ++q) WEC_CK(cudaMalloc(&P->kdf_face[q], nf3[q] * 8));
        WEC_CK(cudaMalloc(&P->kdf_d0, n * 8));
        P->bytes += (nf3[0] + nf3[1] + nf3[2] + n) * 8;
    }
    // reduction partials: one per cluster and quantity
    WEC_CK(cudaMalloc(&P->part, (size_t)(kMaxRestart + 2) * (kKrylovBlocks / kCl) * 8));
    WEC_CK(cudaMalloc(&P->dots, 2 * (kMaxRestart + 2) * 8));
    size_t nh = (size_t)(m + 1) * m + 3 * (m + 1) + m + 8 + (m + 1);
    WEC_CK(cudaMalloc(&P->hess, nh * 8));
    WEC_CK(cudaMemset(P->hess, 0, nh * 8));
    P->cs = P->hess + (m + 1) * m;
    P->sn = P->cs + (m + 1);
    P->g = P->sn + (m + 1);
    P->y = P->g + (m + 1);
    P->sc = P->y + m + 8;
    WEC_CK(cudaMalloc(&P->ks, sizeof(KState)));
    WEC_CK(cudaMemset(P->ks, 0, sizeof(KState)));
    WEC_CK(cudaMallocHost(&P->ksh, sizeof(KState)));
    P->bytes += ((m + 1) * n + n) * 8 + m * n * 8;
    if (d3) return WEC_OK;  // the 3D V-cycle has no tile shapes to tune
    return poisson_autotune(P, st);
}

void poisson_free(wec_poisson *P)
{
    for (int l = 0; l < P->nlev; ++l) {
        cudaFree(P->L64[l].bu); cudaFree(P->L64[l].bv); cudaFree(P->L64[l].x); cudaFree(P->L64[l].b);
        cudaFree(P->L32[l].bu); cudaFree(P->L32[l].bv); cudaFree(P->L32[l].x); cudaFree(P->L32[l].b);
        cudaFree(P->L64[l].bw); cudaFree(P->L32[l].bw);
        cudaFree(P->L64[l].xp); cudaFree(P->L32[l].xp);
        cudaFree(P->L64[l].id); cudaFree(P->L32[l].id);
    }
    cudaFree(P->lu64); cudaFree(P->lu32);
    cudaFree(P->inv64); cudaFree(P->inv32);
    cudaFree(P->V); cudaFree(P->Z); cudaFree(P->w); cudaFree(P->d0); cudaFree(P->part); cudaFree(P->dots); cudaFree(P->hess);
    for (double *&q : P->kdf_face) {
        cudaFree(q);
        q = nullptr;
    }
    cudaFree(P->kdf_d0);
    P->kdf_d0 = nullptr;
    cudaFree(P->ks);
    if (P->ksh) cudaFreeHost(P->ksh);
    *P = wec_poisson();
}

template <typename T>
int build_invdiag(wec_poisson *P, Level<T> *L, cudaStream_t st)
{
    LevelDiag<T> D;
    D.nlev = P->nlev;
    D.off[0] = 0;
    for (int l = 0; l < P->nlev; ++l) {
        D.nx[l] = L[l].nx;
        D.ny[l] = L[l].ny;
        D.bu[l] = L[l].bu;
        D.bv[l] = L[l].bv;
        D.id[l] = L[l].id;
        D.off[l + 1] = D.off[l] + (long long)L[l].nx * L[l].ny;
    }
    const long long tot = D.off[P->nlev];
    WEC_PROF("mg_invdiag", -1, (double)sizeof(T) * 4.0 * tot, st);
    launch_k(k_invdiag<T>, nblk(tot, 256), 256, 0, st, D);
    WEC_CK(cudaGetLastError());
    return WEC_OK;
}

template <typename T>
int build_invdiag3(wec_poisson *P, Level<T> *L, cudaStream_t st)
{
    Level3Diag<T> D;
    D.nlev = P->nlev;
    D.off[0] = 0;
    // FP32 levels above the coarsest are colour-packed (mg3d.cuh)
    D.pk = std::is_same<T, float>::value ? (1u << (P->nlev - 1)) - 1u : 0u;
    for (int l = 0; l < P->nlev; ++l) {
        D.nx[l] = L[l].nx;
        D.ny[l] = L[l].ny;
        D.nz[l] = L[l].nz;
        D.bx[l] = L[l].bu;
        D.by[l] = L[l].bv;
        D.bz[l] = L[l].bw;
        D.id[l] = L[l].id;
        D.off[l + 1] = D.off[l] + (long long)L[l].nx * L[l].ny * L[l].nz;
    }
    const long long tot = D.off[P->nlev];
    WEC_PROF("mg_invdiag", -1, (double)sizeof(T) * 5.0 * tot, st);
    launch_k(k3_invdiag<T>, nblk(tot, 256), 256, 0, st, D);
    WEC_CK(cudaGetLastError());
    return WEC_OK;
}

template <typename T>
int build_hierarchy3(wec_poisson *P, Level<T> *L, T *lu, cudaStream_t st)
{
    for (int l = 0; l + 1 < P->nlev; ++l) {
        Level<T> &F = L[l], &C = L[l + 1];
        const long long cnt = (C.nx + 1ll) * C.ny * C.nz + C.nx * (C.ny + 1ll) * C.nz + (long long)C.nx * C.ny * (C.nz + 1);
        WEC_PROF("mg_coarsen", l, 5.0 * sizeof(T) * cnt, st);
        launch_k(k3_coarsen<T>, nblk(cnt, 256), 256, 0, st, F.nx, F.ny, F.nz, F.bu, F.bv, F.bw, C.bu, C.bv, C.bw);
    }
    Level<T> &Lc = L[P->nlev - 1];
    const double nn = (double)Lc.nx * Lc.ny * Lc.nz;
    WEC_PROF("mg_lu_factor", P->nlev - 1, sizeof(T) * nn * nn, st);
    launch_k(k3_lu_factor<T>, 1, 256, 0, st, Lc.nx, Lc.ny, Lc.nz, Lc.bu, Lc.bv, Lc.bw, lu);
    return build_invdiag3<T>(P, L, st);
}

int poisson_build3(wec_poisson *P, cudaStream_t st)
{
    const long long n = ncells(P);
    {
        WEC_PROF("diag", 0, 8.0 * (n + nfaces(P)), st);
        launch_k(k3_diag0, nblk(n, 256), 256, 0, st, P->nx, P->ny, P->nz, P->L64[0].bu, P->L64[0].bv, P->L64[0].bw,
                 P->d0);
    }
    if (P->kdf) {  // the pair copy of the level-0 diagonal (the faces' with their FP32 copies below)
        WEC_PROF("convert", 0, 16.0 * n, st);
        launch_k(k_to_pairs, nblk(n, 256), 256, 0, st, n, (const double *)P->d0, (df64 *)P->kdf_d0);
    }
    int e;
    if (P->prec == WEC_PREC_MIXED) {
        // the V-cycle is FP32 throughout: level-0 faces converted once (float
        // pairs in the same pass for the pair Arnoldi step)
        Level<double> &A = P->L64[0];
        Level<float> &F = P->L32[0];
        const long long nf[3] = {(A.nx + 1ll) * A.ny * A.nz, A.nx * (A.ny + 1ll) * A.nz,
                                 (long long)A.nx * A.ny * (A.nz + 1)};
        const double *src[3] = {A.bu, A.bv, A.bw};
        float *dst[3] = {F.bu, F.bv, F.bw};
        for (int q = 0; q < 3; ++q) {
            if (P->kdf) {
                WEC_PROF("convert", 0, 20.0 * nf[q], st);
                launch_k(k_to_pairs_f32, nblk(nf[q], 256), 256, 0, st, nf[q], src[q], (df64 *)P->kdf_face[q],
                         dst[q]);
            } else {
                WEC_PROF("convert", 0, 12.0 * nf[q], st);
                launch_k(k_convert<float, double>, nblk(nf[q], 256), 256, 0, st, nf[q], src[q], dst[q], nullptr);
            }
        }
        e = build_hierarchy3<float>(P, P->L32, P->lu32, st);
    } else {
        e = build_hierarchy3<double>(P, P->L64, P->lu64, st);
    }
    if (e) return e;
    WEC_CK(cudaGetLastError());
    P->have_coef = true;
    return WEC_OK;
}

int poisson_build(wec_poisson *P, cudaStream_t st)
{
    if (P->nz > 1) return poisson_build3(P, st);
    {
        const int n = P->nx * P->ny;
        WEC_PROF("diag", 0, 8.0 * (n + (P->nx + 1.0) * P->ny + P->nx * (P->ny + 1.0)), st);
        launch_k(k_diag0, nblk(n, 256), 256, 0, st, P->nx, P->ny, P->L64[0].bu, P->L64[0].bv, P->d0);
    }
    if (P->prec == WEC_PREC_MIXED) {
        // the V-cycle is FP32 throughout: level 0 converted once, coarse levels
        // and the coarsest LU formed in FP32 (the FP64 operator is level 0 only)
        Level<double> &A = P->L64[0];
        Level<float> &F = P->L32[0];
        const long long nu = (long long)(A.nx + 1) * A.ny, nv = (long long)A.nx * (A.ny + 1);
        {
            WEC_PROF("convert", 0, 12.0 * nu, st);
            launch_k(k_convert<float, double>, nblk(nu, 256), 256, 0, st, nu, A.bu, F.bu, nullptr);
        }
        {
            WEC_PROF("convert", 0, 12.0 * nv, st);
            launch_k(k_convert<float, double>, nblk(nv, 256), 256, 0, st, nv, A.bv, F.bv, nullptr);
        }
        for (int l = 0; l + 1 < P->nlev; ++l) {
            Level<float> &Fl = P->L32[l], &C = P->L32[l + 1];
            int cnt = (C.nx + 1) * C.ny + C.nx * (C.ny + 1);
            WEC_PROF("mg_coarsen", l, 12.0 * cnt, st);
            launch_k(k_coarsen<float>, nblk(cnt, 256), 256, 0, st, Fl.nx, Fl.ny, Fl.bu, Fl.bv, C.bu, C.bv);
        }
        Level<float> &Lf = P->L32[P->nlev - 1];
        const double nn = (double)Lf.nx * Lf.ny;
        WEC_PROF("mg_lu_factor", P->nlev - 1, 4.0 * nn * nn, st);
        launch_k(k_lu_factor<float>, 1, 256, 0, st, Lf.nx, Lf.ny, Lf.bu, Lf.bv, P->lu32, P->inv32);
        if (int e = build_invdiag<float>(P, P->L32, st)) return e;
    } else {
        for (int l = 0; l + 1 < P->nlev; ++l) {
            Level<double> &F = P->L64[l], &C = P->L64[l + 1];
            int cnt = (C.nx + 1) * C.ny + C.nx * (C.ny + 1);
            WEC_PROF("mg_coarsen", l, 24.0 * cnt, st);
            launch_k(k_coarsen<double>, nblk(cnt, 256), 256, 0, st, F.nx, F.ny, F.bu, F.bv, C.bu, C.bv);
        }
        Level<double> &Lc = P->L64[P->nlev - 1];
        const double nn = (double)Lc.nx * Lc.ny;
        WEC_PROF("mg_lu_factor", P->nlev - 1, 8.0 * nn * nn, st);
        launch_k(k_lu_factor<double>, 1, 256, 0, st, Lc.nx, Lc.ny, Lc.bu, Lc.bv, P->lu64, P->inv64);
        if (int e = build_invdiag<double>(P, P->L64, st)) return e;
    }
    WEC_CK(cudaGetLastError());
    P->have_coef = true;
    return WEC_OK;
}

int poisson_apply(wec_poisson *P, const double *x, double *y)
{
    if (P->nz > 1) {
        const long long n = ncells(P);
        WEC_PROF("krylov_matvec", -1, 8.0 * (2.0 * n + nfaces(P)), P->st);
        launch_k(k3_apply<double>, nblk(n, 256), 256, 0, P->st, P->nx, P->ny, P->nz, P->L64[0].bu, P->L64[0].bv,
                 P->L64[0].bw, x, y);
        WEC_CK(cudaGetLastError());
        return WEC_OK;
    }
    int n = P->nx * P->ny;
    WEC_PROF("krylov_matvec", -1, 8.0 * (2.0 * n + (P->nx + 1.0) * P->ny + P->nx * (P->ny + 1.0)), P->st);
    launch_k(k_apply<double>, nblk(n, 256), 256, 0, P->st, P->nx, P->ny, P->L64[0].bu, P->L64[0].bv, x, y);
    WEC_CK(cudaGetLastError());
    return WEC_OK;
}

int poisson_vcycle(wec_poisson *P, const double *b, double *x)
{
    const long long n = ncells(P);
    cudaStream_t st = P->st;
    if (P->prec == WEC_PREC_FP64) {
        vcycle_t<double, double>(P, P->L64, b, x, nullptr, nullptr, st);
    } else {
        {
            WEC_PROF("convert", -1, 12.0 * n, st);
            launch_k(k_convert<float, double>, nblk(n, 256), 256, 0, st, n, b, P->L32[0].b, nullptr);
        }
        if (P->nz > 1) {  // unpacked from the colour-packed level-0 iterate into x
            vcycle_t<float, double>(P, P->L32, P->L32[0].b, x, nullptr, nullptr, st);
        } else {
            vcycle_t<float, float>(P, P->L32, P->L32[0].b, P->L32[0].x, nullptr, nullptr, st);
            WEC_PROF("convert", -1, 12.0 * n, st);
            launch_k(k_convert<double, float>, nblk(n, 256), 256, 0, st, n, P->L32[0].x, x, nullptr);
        }
    }
    WEC_CK(cudaGetLastError());
    return WEC_OK;
}

// Host-polled solve: one state read per Arnoldi step.
int poisson_solve(wec_poisson *P, const double *b, double *x, double rtol, int maxit, int *iters, double *relres)
{
    cudaStream_t st = P->st;
    enqueue_begin(P, b, x, rtol, maxit, 0ull, 0, st);
    WEC_CK(cudaGetLastError());
    if (int e = read_state(P, st)) return e;
    while (!P->ksh->done) {
        enqueue_body(P, 0ull, 0, st, P->ksh->j);
        WEC_CK(cudaGetLastError());
        if (int e = read_state(P, st)) return e;
        if (P->ksh->cycle_end) {
            enqueue_close(P, b, x, 0ull, 0, st);
            WEC_CK(cudaGetLastError());
            if (int e = read_state(P, st)) return e;
        }
    }
    return solve_result(P, iters, relres);
}

int solve_result(wec_poisson *P, int *iters, double *relres)
{
    const KState &k = *P->ksh;
    if (iters) *iters = k.its;
    if (relres) *relres = k.bn > 0.0 ? k.beta / k.bn : 0.0;
    if (k.status == WEC_ERR_NONFINITE) return fail(WEC_ERR_NONFINITE, "pressure solve: residual is not finite");
    if (k.status == WEC_ERR_NOT_CONVERGED) return fail(WEC_ERR_NOT_CONVERGED, "pressure solve: not converged within max_iters");
    return WEC_OK;
}

// Record the whole solve into the graph being captured on st: WHILE(not done)
// { Arnoldi step; IF(cycle ends) { close cycle } }.  h1, h2: idle streams used to
// capture the two conditional bodies.
int poisson_capture_solve(wec_poisson *P, const double *b, double *x, double rtol, int maxit, cudaStream_t st,
                          cudaStream_t h1, cudaStream_t h2)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    WEC_CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
    if (cs != cudaStreamCaptureStatusActive) return fail(WEC_ERR_CUDA, "capture_solve: stream is not capturing");
    cudaGraphConditionalHandle hw, hi;
    WEC_CK(cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault));
    WEC_CK(cudaGraphConditionalHandleCreate(&hi, g, 0, cudaGraphCondAssignDefault));
    enqueue_begin(P, b, x, rtol, maxit, (unsigned long long)hw, 1, st);
    WEC_CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    WEC_CK(cudaGraphAddNode(&wnode, g, deps, nullptr, nd, &wp));
    cudaGraph_t wbody = wp.conditional.phGraph_out[0];
    WEC_CK(cudaStreamUpdateCaptureDependencies(st, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));

    WEC_CK(cudaStreamBeginCaptureToGraph(h1, wbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    enqueue_body(P, (unsigned long long)hi, 1, h1);
    cudaGraph_t g1 = nullptr;
    const cudaGraphNode_t *d1 = nullptr;
    size_t n1 = 0;
    WEC_CK(cudaStreamGetCaptureInfo(h1, &cs, nullptr, &g1, &d1, nullptr, &n1));
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hi;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t inode;
    WEC_CK(cudaGraphAddNode(&inode, g1, d1, nullptr, n1, &ip));
    cudaGraph_t ibody = ip.conditional.phGraph_out[0];
    WEC_CK(cudaStreamUpdateCaptureDependencies(h1, &inode, nullptr, 1, cudaStreamSetCaptureDependencies));
    WEC_CK(cudaStreamBeginCaptureToGraph(h2, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    enqueue_close(P, b, x, (unsigned long long)hw, 1, h2);
    cudaGraph_t tmp;
    WEC_CK(cudaStreamEndCapture(h2, &tmp));
    WEC_CK(cudaStreamEndCapture(h1, &tmp));
    WEC_CK(cudaGetLastError());
    return WEC_OK;
}

// Kernels enqueued by the solve's opening, by one Arnoldi step and by one cycle
// close (counted on a throwaway capture of the same enqueue code).
int poisson_count_kernels(wec_poisson *P, cudaStream_t s, int *n_begin, int *n_body, int *n_close)
{
    cudaGraph_t tmp = nullptr;
    WEC_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    prof::begin_capture();
    enqueue_begin(P, P->w, P->w, 1.0, 1, 0ull, 0, s);
    long long a = prof::captured();
    enqueue_body(P, 0ull, 0, s);
    long long b = prof::captured();
    enqueue_close(P, P->w, P->w, 0ull, 0, s);
    long long c = prof::captured();
    prof::end_capture();
    WEC_CK(cudaStreamEndCapture(s, &tmp));
    if (tmp) cudaGraphDestroy(tmp);
    *n_begin = (int)a;
    *n_body = (int)(b - a);
    *n_close = (int)(c - b);
    return WEC_OK;
}

// After a captured solve ran: state -> host (enqueued on st; caller synchronises).
int poisson_state_to_host(wec_poisson *P, cudaStream_t st)
{
    WEC_CK(cudaMemcpyAsync(P->ksh, P->ks, sizeof(KState), cudaMemcpyDeviceToHost, st));
    return WEC_OK;
}

}  // namespace wec
