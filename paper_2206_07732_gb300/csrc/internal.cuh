// Internal declarations of libwec (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "wec.h"

namespace wec {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxLevels = 24;
constexpr int kMaxRestart = 32;
constexpr int kMaxCoarse = 512;      // cells on the coarsest multigrid level
constexpr int kRedBlocks = 304;      // partial-sum blocks of every reduction (2 x 152 SMs)
constexpr int kRedThreads = 256;

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define WEC_CK(call)                                                  \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return ::wec::cuda_fail(e_, #call);    \
    } while (0)

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

// Launch accounting (profile.cu): open one Scope around every kernel launch.
namespace prof {
class Scope {
  public:
    Scope(const char *name, int level, double bytes, cudaStream_t st);
    ~Scope();

  private:
    int slot_;
    cudaStream_t st_;
};
}  // namespace prof

#define WEC_PROF(NAME, LEVEL, BYTES, ST) ::wec::prof::Scope wec_prof_scope_((NAME), (LEVEL), (double)(BYTES), (ST))

// ------------------------------------------------------------------ solver --
template <typename T>
struct Level {
    int nx = 0, ny = 0;
    T *bu = nullptr, *bv = nullptr, *x = nullptr, *b = nullptr;
};

}  // namespace wec

struct wec_poisson {
    int nx = 0, ny = 0, nlev = 0, prec = 0, restart = 20, nu1 = 2, nu2 = 2;
    cudaStream_t st = nullptr;
    bool have_coef = false;
    wec::Level<double> L64[wec::kMaxLevels];
    wec::Level<float> L32[wec::kMaxLevels];
    int ncoarse = 0;
    double *lu64 = nullptr;
    float *lu32 = nullptr;
    // FGMRES workspace (FP64 outer iteration)
    double *V = nullptr;        // (m+1) x n
    void *Z = nullptr;          // m x n, double (FP64) or float (mixed)
    double *w = nullptr;        // n
    double *part = nullptr;     // kMaxRestart+1 x kRedBlocks partial sums
    double *dots = nullptr;     // kMaxRestart+1 results
    double *hess = nullptr;     // (m+1) x m Hessenberg, then cs, sn, g, y, scalars
    double *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr, *scal = nullptr;
    double *host = nullptr;     // pinned mirror of a few scalars
    size_t bytes = 0;
};

namespace wec {

// solver.cu
int poisson_init(wec_poisson *P, int nx, int ny, int prec, int restart, int nu1, int nu2,
                 cudaStream_t st);
void poisson_free(wec_poisson *P);
// Level-0 coefficients already in P->L64[0].bu / bv (device): build coarse levels,
// FP32 copies and the coarse LU.
int poisson_build(wec_poisson *P);
int poisson_solve(wec_poisson *P, const double *b, double *x, double rtol, int maxit, int *iters,
                  double *relres);
int poisson_apply(wec_poisson *P, const double *x, double *y);
int poisson_vcycle(wec_poisson *P, const double *b, double *x);

// Deterministic reductions: partial sums per block, then one block per result.
void launch_norm2(const double *a, int n, double *part, double *out, cudaStream_t st);

// waves.cpp
double wave_number(double omega, double depth, double g);
double wave_number_fenton_kd(double omega, double depth, double g);
int jonswap(double Hs, double Tp, double gamma, int ncomp, double *amp, double *omega);

}  // namespace wec
