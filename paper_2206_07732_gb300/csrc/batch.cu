// Many independent tanks stepping together: one CUDA graph launch per batch step.
//
// Each tank keeps its own kernels, stream, multigrid hierarchy and autotuned
// tile shapes (tanks differ in size, waves and body).  The batch graph is one
// stream capture: the batch stream forks to every tank's stream, each tank
// enqueues its whole step there (front kernels, the conditional WHILE / IF
// FGMRES solve, back kernels, the D2H copies of its step record), and the
// branches join back.  The tanks have no dependencies on one another, so the
// GPU runs their kernels concurrently and small tanks fill the SMs that one
// tank alone would leave idle.  The (dt, F_PTO) inputs of all tanks live in one
// device array, filled by one host-to-device copy per step.
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "tank.cuh"

struct wec_batch {
    std::vector<wec_tank *> tanks;
    cudaStream_t st = nullptr;   // caller's stream (ordering only)
    cudaStream_t bst = nullptr;  // the batch's launch stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
    double *inp = nullptr;  // device [2 n]: dt, f_pto per tank
    double *inh = nullptr;  // pinned host staging of inp
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace wec {
namespace {

void batch_free(wec_batch *B)
{
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    for (wec_tank *T : B->tanks) wec_tank_destroy(T);
    for (cudaEvent_t e : B->ev_join)
        if (e) cudaEventDestroy(e);
    if (B->ev_in) cudaEventDestroy(B->ev_in);
    if (B->ev_out) cudaEventDestroy(B->ev_out);
    if (B->ev_fork) cudaEventDestroy(B->ev_fork);
    if (B->bst) cudaStreamDestroy(B->bst);
    cudaFree(B->inp);
    if (B->inh) cudaFreeHost(B->inh);
}

// Capture every tank's step as one branch of a single graph.
int batch_build_graph(wec_batch *B)
{
    for (wec_tank *T : B->tanks)
        if (int e = tank_prepare_capture(T)) return e;
    WEC_CK(cudaStreamBeginCapture(B->bst, cudaStreamCaptureModeThreadLocal));
    int e = WEC_OK;
    cudaError_t ce = cudaEventRecord(B->ev_fork, B->bst);
    for (size_t i = 0; i < B->tanks.size() && e == WEC_OK && ce == cudaSuccess; ++i) {
        wec_tank *T = B->tanks[i];
        ce = cudaStreamWaitEvent(T->gst, B->ev_fork, 0);
        if (ce != cudaSuccess) break;
        e = tank_capture_step(T, T->gst);
        if (e) break;
        ce = cudaEventRecord(B->ev_join[i], T->gst);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(B->bst, B->ev_join[i], 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t ce2 = cudaStreamEndCapture(B->bst, &g);
    if (e || ce != cudaSuccess || ce2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (e) return e;
        return cuda_fail(ce != cudaSuccess ? ce : ce2, "batch graph capture");
    }
    B->graph = g;
    WEC_CK(cudaGraphInstantiate(&B->exec, g, 0));
    return WEC_OK;
}

}  // namespace
}  // namespace wec

using namespace wec;

extern "C" {

int wec_batch_create(int ntanks, const wec_grid *grids, const wec_fluids *fluids, const wec_waves *waves,
                     const wec_body *bodies, const wec_solver_opts *opts, void *cuda_stream, wec_batch **out)
{
    if (!out) return fail(WEC_ERR_INVALID, "batch: out is NULL");
    *out = nullptr;
    if (ntanks < 1 || ntanks > 4096) return fail(WEC_ERR_INVALID, "batch: ntanks must be in 1..4096");
    if (!grids || !fluids || !waves || !bodies || !opts) return fail(WEC_ERR_INVALID, "batch: NULL argument");
    for (int i = 0; i < ntanks; ++i)  // every description checked before any device work
        if (validate_tank(grids + i, fluids + i, waves + i, bodies + i, opts + i))
            return fail(WEC_ERR_INVALID, "batch: tank " + std::to_string(i) + ": " + wec_last_error());
    wec_batch *B = new (std::nothrow) wec_batch();
    if (!B) return fail(WEC_ERR_NOMEM, "batch: host allocation failed");
    B->st = (cudaStream_t)cuda_stream;
    auto bail = [B](int e) {
        std::string msg = wec_last_error();
        batch_free(B);
        delete B;
        return fail(e, msg);
    };
    for (int i = 0; i < ntanks; ++i) {
        wec_tank *T = nullptr;
        if (int e = wec_tank_create(grids + i, fluids + i, waves + i, bodies + i, opts + i, cuda_stream, &T)) {
            std::string msg = "batch: tank " + std::to_string(i) + ": " + wec_last_error();
            batch_free(B);
            delete B;
            return fail(e, msg);
        }
        B->tanks.push_back(T);
    }
    cudaError_t ce = cudaStreamCreateWithFlags(&B->bst, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming);
    B->ev_join.assign(ntanks, nullptr);
    for (int i = 0; i < ntanks && ce == cudaSuccess; ++i) ce = cudaEventCreateWithFlags(&B->ev_join[i], cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaMalloc(&B->inp, 2 * sizeof(double) * ntanks);
    if (ce == cudaSuccess) ce = cudaMallocHost(&B->inh, 2 * sizeof(double) * ntanks);
    if (ce == cudaSuccess) ce = cudaMemset(B->inp, 0, 2 * sizeof(double) * ntanks);
    if (ce != cudaSuccess) {
        cuda_fail(ce, "batch: allocation");
        return bail(WEC_ERR_CUDA);
    }
    // every tank reads its (dt, f_pto) from the batch's array from now on
    for (int i = 0; i < ntanks; ++i) {
        wec_tank *T = B->tanks[i];
        cudaStreamSynchronize(T->gst);
        if (T->inp_owned) cudaFree(T->inp);
        T->inp = B->inp + 2 * i;
        T->inp_owned = false;
        if (T->exec) {  // a tank graph captured before would hold the old pointer
            cudaGraphExecDestroy(T->exec);
            cudaGraphDestroy(T->graph);
            T->exec = nullptr;
            T->graph = nullptr;
        }
    }
    *out = B;
    return WEC_OK;
}

int wec_batch_size(const wec_batch *B) { return B ? (int)B->tanks.size() : 0; }

int wec_batch_tank(wec_batch *B, int i, wec_tank **out)
{
    if (!B || !out) return fail(WEC_ERR_INVALID, "batch_tank: NULL argument");
    if (i < 0 || i >= (int)B->tanks.size()) return fail(WEC_ERR_INVALID, "batch_tank: index out of range");
    *out = B->tanks[i];
    return WEC_OK;
}

int wec_batch_step(wec_batch *B, const double *dt, const double *pto_force, wec_step_result *out)
{
    if (!B || !dt) return fail(WEC_ERR_INVALID, "batch_step: NULL argument");
    const int n = (int)B->tanks.size();
    for (int i = 0; i < n; ++i)
        if (!(dt[i] > 0.0) || !std::isfinite(dt[i])) return fail(WEC_ERR_INVALID, "batch_step: dt must be > 0");
    if (prof::enabled()) {
        // per-kernel profiling needs one-by-one launches: step the tanks in turn
        int status = WEC_OK;
        for (int i = 0; i < n; ++i) {
            int e = tank_step(B->tanks[i], dt[i], pto_force ? pto_force[i] : 0.0, out ? out + i : nullptr);
            if (e != WEC_OK && e != WEC_ERR_NOT_CONVERGED) return e;
            if (status == WEC_OK) status = e;
        }
        return status;
    }
    if (!B->exec)
        if (int e = batch_build_graph(B)) return e;
    WEC_CK(cudaEventRecord(B->ev_in, B->st));
    WEC_CK(cudaStreamWaitEvent(B->bst, B->ev_in, 0));
    for (int i = 0; i < n; ++i) {
        B->inh[2 * i] = dt[i];
        B->inh[2 * i + 1] = pto_force ? pto_force[i] : 0.0;
    }
    WEC_CK(cudaMemcpyAsync(B->inp, B->inh, 2 * sizeof(double) * n, cudaMemcpyHostToDevice, B->bst));
    WEC_CK(cudaGraphLaunch(B->exec, B->bst));
    WEC_CK(cudaStreamSynchronize(B->bst));
    WEC_CK(cudaEventRecord(B->ev_out, B->bst));
    WEC_CK(cudaStreamWaitEvent(B->st, B->ev_out, 0));
    int status = WEC_OK;
    for (int i = 0; i < n; ++i) {
        int e = tank_finish_step(B->tanks[i], out ? out + i : nullptr);
        if (status == WEC_OK) status = e;
    }
    return status;
}

int wec_batch_step_n(wec_batch *B, int nsteps, const double *dt, const double *pto_force, wec_step_result *out)
{
    if (!B || !dt) return fail(WEC_ERR_INVALID, "batch_step_n: NULL argument");
    if (nsteps < 0) return fail(WEC_ERR_INVALID, "batch_step_n: nsteps < 0");
    const int n = (int)B->tanks.size();
    int status = WEC_OK;
    for (int s = 0; s < nsteps; ++s) {
        int e = wec_batch_step(B, dt + (size_t)s * n, pto_force ? pto_force + (size_t)s * n : nullptr,
                               out ? out + (size_t)s * n : nullptr);
        if (e != WEC_OK && e != WEC_ERR_NOT_CONVERGED) return e;
        if (status == WEC_OK) status = e;
    }
    return status;
}

void wec_batch_destroy(wec_batch *B)
{
    if (!B) return;
    if (B->st) cudaStreamSynchronize(B->st);
    if (B->bst) cudaStreamSynchronize(B->bst);
    batch_free(B);
    delete B;
}

}  // extern "C"
