// The pressure operator (A x)_c = d_c x_c - sum_nb beta_f x_nb on the cell grid
// [ny][nx] with face coefficients beta_u [ny][nx+1], beta_v [ny+1][nx] (zero on
// the Neumann walls); the top face's ghost value -x_c (Dirichlet p = 0 on the
// top boundary) doubles its weight in the diagonal.
#pragma once

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

}  // namespace wec
