// Check of the integer-pipe float <-> double conversions (df64.cuh) against the
// conversion instructions, value by value (wec_check_conversions).
#include "df64.cuh"
#include "internal.cuh"

namespace wec {
namespace {

__device__ __forceinline__ bool same_bits(double a, double b)
{
    return __double_as_longlong(a) == __double_as_longlong(b);
}
__device__ __forceinline__ bool same_bits(float a, float b) { return __float_as_uint(a) == __float_as_uint(b); }

__global__ void __launch_bounds__(256) k_check_conversions(long long n, const double *__restrict__ v,
                                                           unsigned long long *bad)
{
    pdl_entry();
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double d = v[q];
    const float f = d2f_rn(d), fr = __double2float_rn(d);
    bool ok = same_bits(f, fr) && same_bits(f2d_exact(fr), (double)fr);
    const df64 p = from_double(d), pr(d);  // the constructor's value, by the conversion instructions
    ok = ok && same_bits(p.hi, pr.hi) && same_bits(p.lo, pr.lo);
    ok = ok && same_bits(to_double(pr), (double)pr.hi + (double)pr.lo);
    if (!ok) atomicAdd(bad, 1ull);
}

}  // namespace
}  // namespace wec

using namespace wec;

extern "C" int wec_check_conversions(long long n, const double *values, unsigned long long *mismatches,
                                     void *cuda_stream)
{
    if (n < 0 || !mismatches || (n > 0 && !values)) return fail(WEC_ERR_INVALID, "check_conversions: bad arguments");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    WEC_CK(cudaMemsetAsync(mismatches, 0, sizeof(unsigned long long), st));
    if (n > 0) WEC_CK(launch_k(k_check_conversions, nblk(n, 256), 256, 0, st, n, values, mismatches));
    WEC_CK(cudaGetLastError());
    return WEC_OK;
}
