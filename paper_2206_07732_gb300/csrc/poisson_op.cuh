// The pressure operator (A x)_c = d_c x_c - sum_nb beta_f x_nb on the cell grid
// [ny][nx] with face coefficients beta_u [ny][nx+1], beta_v [ny+1][nx] (zero on
// the Neumann walls); the top face's ghost value -x_c (Dirichlet p = 0 on the
// top boundary) doubles its weight in the diagonal.
#pragma once

#include <type_traits>

namespace wec {

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

// a * b + c rounded once, written out: the 3D multigrid forms the same terms in
// its per-level kernels and in its one-CTA coarse levels, and left to the
// compiler the contraction of a product into a sum differs between them
template <typename T>
__device__ __forceinline__ T fma3(T a, T b, T c)
{
    if constexpr (std::is_same<T, float>::value)
        return __fmaf_rn(a, b, c);
    else if constexpr (std::is_same<T, double>::value)
        return __fma_rn(a, b, c);
    else
        return a * b + c;  // float pairs: the pair product and sum
}

// Three dimensions (z vertical): cells [nz][ny][nx], beta_x [nz][ny][nx+1],
// beta_y [nz][ny+1][nx], beta_z [nz+1][ny][nx] (face k of beta_z is the bottom
// face of cell layer k); the walls and the bed are Neumann, the top face
// Dirichlet (counted twice in the diagonal).  c = (k ny + j) nx + i; index
// arithmetic in 32 bits (the library caps every array below 2^31 entries).
template <typename T>
__device__ __forceinline__ T diag3_at(const T *bx, const T *by, const T *bz, int nx, int ny, int nz, int i, int j,
                                      int k)
{
    const int r = k * ny + j, fx = r * (nx + 1) + i, fy = (r + k) * nx + i, c = r * nx + i;
    T d = T(0);
    if (i > 0) d += bx[fx];
    if (i < nx - 1) d += bx[fx + 1];
    if (j > 0) d += by[fy];
    if (j < ny - 1) d += by[fy + nx];
    if (k > 0) d += bz[c];
    d += (k < nz - 1 ? T(1) : T(2)) * bz[c + nx * ny];
    return d;
}

template <typename T, typename TX>
__device__ __forceinline__ T offsum3_at(const T *bx, const T *by, const T *bz, const TX *x, int nx, int ny, int nz,
                                        int i, int j, int k)
{
    const int r = k * ny + j, fx = r * (nx + 1) + i, fy = (r + k) * nx + i, c = r * nx + i, pl = nx * ny;
    T s = T(0);
    if (i > 0) s = fma3(bx[fx], T(x[c - 1]), s);
    if (i < nx - 1) s = fma3(bx[fx + 1], T(x[c + 1]), s);
    if (j > 0) s = fma3(by[fy], T(x[c - nx]), s);
    if (j < ny - 1) s = fma3(by[fy + nx], T(x[c + nx]), s);
    if (k > 0) s = fma3(bz[c], T(x[c - pl]), s);
    if (k < nz - 1) s = fma3(bz[c + pl], T(x[c + pl]), s);
    return s;
}

}  // namespace wec
