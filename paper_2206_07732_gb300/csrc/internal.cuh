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
constexpr int kInvMax = 32;         // coarsest levels up to this size also get an explicit inverse
constexpr int kMaxCoarse = 512;      // cells on the coarsest multigrid level
constexpr int kRedBlocks = 304;      // partial-sum blocks of the step's reductions (2 x 152 SMs)
constexpr int kRedThreads = 256;
constexpr int kKrylovBlocks = 912;   // max CTAs of the Krylov reduction kernels (6 x 152 SMs)

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define WEC_CK(call)                                                  \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return ::wec::cuda_fail(e_, #call);    \
    } while (0)

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

// Programmatic dependent launch.  Every kernel of the library starts with
// pdl_entry(), which waits until the previous kernel on the stream has
// completed and its writes are visible -- the same ordering as plain stream
// order -- while the launch itself (launch_k) may be processed before that
// kernel ends.  No kernel triggers its dependents early: measured, an early
// trigger let waiting grids take SM slots and slowed the step by 6 %.
__device__ __forceinline__ void pdl_entry()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

namespace prof {
void count_launch();  // one kernel launch (or one kernel node recorded into a graph being captured)
}

// kern<<<grid, block, smem, st>>>(args...) with programmatic dependent launch
// allowed (captured into graphs as programmatic edges); every launch is counted.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args &&...args)
{
    prof::count_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<Args &&>(args)...);
}

// Per-kernel event profiling (profile.cu): a Scope around a launch names the
// kernel, its level and its algorithmic bytes.
namespace prof {
class Scope {
  public:
    Scope(const char *name, int level, double bytes, cudaStream_t st);
    ~Scope();

  private:
    int slot_;
    cudaStream_t st_;
};
void begin_capture();          // launch scopes on this thread are being recorded into a graph
long long captured();          // scopes opened since begin_capture()
void end_capture();
void add_launches(long long n);  // kernels a graph replay executed
bool enabled();                // event profiling on (graphs are then not used)
}  // namespace prof

#define WEC_PROF(NAME, LEVEL, BYTES, ST) ::wec::prof::Scope wec_prof_scope_((NAME), (LEVEL), (double)(BYTES), (ST))

// ------------------------------------------------------------------ solver --
template <typename T>
struct Level {
    int nx = 0, ny = 0, nz = 1;  // nz > 1: a level of the 3D operator (bu, bv, bw = beta_x, beta_y, beta_z)
    T *bu = nullptr, *bv = nullptr, *x = nullptr, *b = nullptr;
    T *bw = nullptr;
    T *xp = nullptr;  // pre-smoothed iterate of a tiled (fused) level, read by its post kernel
    T *id = nullptr;  // 1 / diagonal per cell, formed by poisson_build (fused V-cycle)
};

// FGMRES state on the device (read by the kernels that steer the iteration).
struct KState {
    int j, its, jd, cycle_end, done, status, maxit, m, ncycles, pad_;
    unsigned int cnt[4];  // last-block counters of the fused reductions
    double bn, tol, beta, hn, rtol;
    double ibeta, ihn;    // 1 / beta, 1 / hn (set with them)
};

}  // namespace wec

struct wec_poisson {
    int nx = 0, ny = 0, nlev = 0, prec = 0, restart = 20, nu1 = 2, nu2 = 2;
    int nz = 1;                 // > 1: the 3D operator (wec_poisson_create3)
    cudaStream_t st = nullptr;
    bool have_coef = false;
    wec::Level<double> L64[wec::kMaxLevels];
    wec::Level<float> L32[wec::kMaxLevels];
    int ncoarse = 0;
    double *lu64 = nullptr;
    float *lu32 = nullptr;
    double *inv64 = nullptr;  // explicit inverse of the coarsest operator (at most kInvMax cells)
    float *inv32 = nullptr;
    // FGMRES workspace (FP64 outer iteration)
    double *V = nullptr;        // (m+1) x n
    double *Z = nullptr;        // m x n preconditioned vectors (FP64 in both precisions)
    double *w = nullptr;        // n
    double *d0 = nullptr;       // n: diagonal of the FP64 level-0 operator
    double *part = nullptr;     // (kMaxRestart+2) x (kKrylovBlocks / 8) cluster partial sums
    double *dots = nullptr;     // h1, h2 of the two Gram-Schmidt passes
    double *hess = nullptr;     // (m+1) x m Hessenberg, then cs, sn, g, y
    double *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
    double *sc = nullptr;       // m+1: 1 / ||u_k|| of the unnormalised basis vectors u_k (V's columns)
    // Arnoldi arithmetic in float pairs (3D, WEC_PREC_MIXED_DF): V then holds pairs
    // (8 bytes, as FP64), Z the FP32 V-cycle's columns as floats (n floats apart),
    // and the level-0 faces and diagonal have pair copies
    bool kdf = false;
    double *kdf_face[3] = {};   // beta_x, beta_y, beta_z as float pairs
    double *kdf_d0 = nullptr;   // the diagonal as float pairs
    int tile64[wec::kMaxLevels] = {}, tile32[wec::kMaxLevels] = {};  // fused tile shape per level (autotuned)
    bool tuned = false;
    int bottom_shift = 0;       // bottom kernel starts this many levels below the smallest admissible one (autotuned)
    int bottom_level = -1;      // the level the bottom kernel starts at (set by the last fused V-cycle)
    wec::KState *ks = nullptr;  // device
    wec::KState *ksh = nullptr; // pinned host mirror
    size_t bytes = 0;
};

namespace wec {

// solver.cu
int poisson_init(wec_poisson *P, int nx, int ny, int prec, int restart, int nu1, int nu2,
                 cudaStream_t st, int nz = 1);
void poisson_free(wec_poisson *P);
// Level-0 coefficients already in P->L64[0].bu / bv (/ bw in 3D) (device): build coarse levels,
// FP32 copies and the coarse LU (enqueued on st).
int poisson_build(wec_poisson *P, cudaStream_t st);
// Host-polled FGMRES solve on P->st.
int poisson_solve(wec_poisson *P, const double *b, double *x, double rtol, int maxit, int *iters,
                  double *relres);
// Record the same solve into the graph being captured on st (conditional nodes).
int poisson_capture_solve(wec_poisson *P, const double *b, double *x, double rtol, int maxit, cudaStream_t st,
                          cudaStream_t h1, cudaStream_t h2);
int poisson_state_to_host(wec_poisson *P, cudaStream_t st);
int poisson_count_kernels(wec_poisson *P, cudaStream_t s, int *n_begin, int *n_body, int *n_close);
// Status / iterations / relative residual from the host mirror of the state.
int solve_result(wec_poisson *P, int *iters, double *relres);
int poisson_apply(wec_poisson *P, const double *x, double *y);
void set_mg_fused(bool on);
void set_mg_autotune(bool on);
void set_mg_bottom_shift(int shift);  // -1: autotune
void set_tank3_split_momentum(bool on);
void set_mg3_bottom(bool on);
void poisson_tiles(const wec_poisson *P, int *tx, int *ty, int max);
int poisson_vcycle(wec_poisson *P, const double *b, double *x);

// waves.cpp
double wave_number(double omega, double depth, double g);
double wave_number_fenton_kd(double omega, double depth, double g);
int jonswap(double Hs, double Tp, double gamma, int ncomp, double *amp, double *omega);

}  // namespace wec
