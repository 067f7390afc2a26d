// Launch counter and per-kernel CUDA-event profiler of libwec.
//
// Every kernel launch goes through launch_k, which counts it (a launch recorded
// into a graph is counted each time the graph runs).  Launch sites of the
// kernels worth timing open a prof::Scope naming the kernel, its multigrid
// level (or -1) and its algorithmic bytes (the bytes the operation must move
// at least once: inputs read, outputs written); when profiling is on, the
// scope records a CUDA event pair on the launching stream.
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

namespace wec {
namespace prof {
namespace {

struct Rec {
    const char *name;
    int level;
    double bytes;
    cudaEvent_t a, b;
};

std::mutex g_mu;
long long g_launches = 0;
thread_local int t_capturing = 0;
thread_local long long t_captured = 0;
int g_mode = 0;
std::string g_only;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

void count_launch()
{
    if (t_capturing) {  // recorded into a graph: counted when the graph runs
        ++t_captured;
        return;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    ++g_launches;
}

Scope::Scope(const char *name, int level, double bytes, cudaStream_t st) : slot_(-1), st_(st)
{
    if (t_capturing) return;  // graph bodies hold no events
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_mode == 0 || (g_mode == 2 && g_only != name)) return;
    Rec r{name, level, bytes, take_event(), take_event()};
    cudaEventRecord(r.a, st);
    slot_ = (int)g_recs.size();
    g_recs.push_back(r);
}

Scope::~Scope()
{
    if (slot_ < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(g_recs[slot_].b, st_);
}

void begin_capture()
{
    t_capturing = 1;
    t_captured = 0;
}

long long captured()
{
    return t_captured;
}

void end_capture()
{
    t_capturing = 0;
}

void add_launches(long long n)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_launches += n;
}

bool enabled()
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_mode != 0;
}

}  // namespace prof
}  // namespace wec

using namespace wec;

extern "C" {

long long wec_launch_count(void)
{
    std::lock_guard<std::mutex> lk(prof::g_mu);
    return prof::g_launches;
}

int wec_profile_enable(int mode, const char *only)
{
    if (mode < 0 || mode > 2 || (mode == 2 && !only)) return fail(WEC_ERR_INVALID, "profile: bad mode");
    std::lock_guard<std::mutex> lk(prof::g_mu);
    prof::g_mode = mode;
    prof::g_only = only ? only : "";
    return WEC_OK;
}

int wec_profile_read(int max, char *names, size_t name_stride, int *levels, long long *launches, double *ms,
                     double *bytes, int *count)
{
    if (!count || (max > 0 && (!names || name_stride < 2 || !levels || !launches || !ms || !bytes)))
        return fail(WEC_ERR_INVALID, "profile: NULL output");
    std::lock_guard<std::mutex> lk(prof::g_mu);
    struct Agg {
        std::string name;
        int level;
        long long n;
        double ms, bytes;
    };
    std::vector<Agg> agg;
    int rc = WEC_OK;
    for (auto &r : prof::g_recs) {
        cudaError_t e = cudaEventSynchronize(r.b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) rc = cuda_fail(e, "profile: event timing");
        size_t k = 0;
        while (k < agg.size() && !(agg[k].name == r.name && agg[k].level == r.level)) ++k;
        if (k == agg.size()) agg.push_back({r.name, r.level, 0, 0.0, 0.0});
        agg[k].n += 1;
        agg[k].ms += t;
        agg[k].bytes += r.bytes;
        prof::g_pool.push_back(r.a);
        prof::g_pool.push_back(r.b);
    }
    prof::g_recs.clear();
    *count = (int)agg.size();
    for (int k = 0; k < (int)agg.size() && k < max; ++k) {
        snprintf(names + (size_t)k * name_stride, name_stride, "%s", agg[k].name.c_str());
        levels[k] = agg[k].level;
        launches[k] = agg[k].n;
        ms[k] = agg[k].ms;
        bytes[k] = agg[k].bytes;
    }
    return rc;
}

}  // extern "C"
