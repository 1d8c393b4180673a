// edac_conversion_check: the library's integer-pipe fp32 <-> fp64 conversions (f2d, d2f of
// the internal header) against the hardware conversions, on the device.
//
// Widening is checked on every one of the 2^32 float bit patterns; narrowing on sampled
// double bit patterns drawn with the splitmix64 generator of the index (a third uniform over
// all bit patterns, a third with the exponent in the float range and the 29 dropped mantissa
// bits at or next to the half-way point of the rounding, a third near the overflow and
// underflow edges of the float range).  NaN results count as equal whatever their payload.
#include "edac.h"
#include "edac_internal.cuh"

using namespace edac;

namespace {

static __device__ unsigned long long g_bad_f2d;
static __device__ unsigned long long g_bad_d2f;

__global__ void k_check_widen(unsigned long long n)
{
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const float f = __uint_as_float((unsigned)i);
        const double h = (double)f, s = f2d(f);
        const bool nan = h != h && s != s;
        if (__double_as_longlong(h) != __double_as_longlong(s) && !nan) atomicAdd(&g_bad_f2d, 1ull);
    }
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_check_narrow(unsigned long long n)
{
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const int mode = (int)(i % 3);
        unsigned long long r = splitmix64(i);
        if (mode == 1) {  // float range, dropped bits at or next to the tie
            const unsigned long long e = 880 + splitmix64(r) % 290;
            unsigned long long m = r & 0xfffffffffffffull;
            const unsigned long long k = splitmix64(r + 1) & 7;
            if (k < 3) m = (m & ~0x1fffffffull) | 0x10000000ull;
            else if (k < 5) m = (m & ~0x1fffffffull) | (0x10000000ull + k - 4);
            r = (r & 0x8000000000000000ull) | (e << 52) | m;
        } else if (mode == 2) {  // overflow and underflow edges
            const unsigned long long e = (splitmix64(r) & 1) ? 1140 + splitmix64(r + 3) % 20
                                                             : 860 + splitmix64(r + 5) % 45;
            r = (r & 0x800fffffffffffffull) | (e << 52);
        }
        const double x = __longlong_as_double((long long)r);
        const float h = __double2float_rn(x), s = d2f(x);
        const bool nan = h != h && s != s;
        if (__float_as_uint(h) != __float_as_uint(s) && !nan) atomicAdd(&g_bad_d2f, 1ull);
    }
}

}  // namespace

extern "C" edac_status edac_conversion_check(void *cuda_stream, int all_floats,
                                             uint64_t n_doubles, uint64_t *float_mismatches,
                                             uint64_t *double_mismatches)
{
    if (!float_mismatches || !double_mismatches) return EDAC_E_INVALID;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const unsigned long long zero = 0ull;
    if (cudaMemcpyToSymbolAsync(g_bad_f2d, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyToSymbolAsync(g_bad_d2f, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
        return EDAC_E_CUDA;
    if (all_floats) k_check_widen<<<152 * 16, 256, 0, st>>>(1ull << 32);
    if (n_doubles) k_check_narrow<<<152 * 16, 256, 0, st>>>((unsigned long long)n_doubles);
    if (cudaGetLastError() != cudaSuccess) return EDAC_E_CUDA;
    unsigned long long a = 0, b = 0;
    if (cudaMemcpyFromSymbolAsync(&a, g_bad_f2d, sizeof(a), 0, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyFromSymbolAsync(&b, g_bad_d2f, sizeof(b), 0, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return EDAC_E_CUDA;
    *float_mismatches = a;
    *double_mismatches = b;
    return EDAC_OK;
}
