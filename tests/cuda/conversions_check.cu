// Checks the integer-pipe binary64 <-> binary32 conversions of the mixed
// precision push against the conversion instructions: every float bit
// pattern through f32_to_f64, and random, tie and boundary doubles through
// f64_to_f32_rn and is_nan_f64.  Prints the number of mismatches.
#include <cstdio>
#include <cstdint>

#include "dust_device.cuh"

using namespace dust;

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ bool same_float(float a, float b)
{
    if (a != a && b != b) return true;
    return __float_as_uint(a) == __float_as_uint(b);
}

__device__ bool same_double(double a, double b)
{
    if (a != a && b != b) return true;
    return __double_as_longlong(a) == __double_as_longlong(b);
}

__global__ void all_floats(unsigned long long *bad)
{
    unsigned long long nb = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (1ull << 32);
         i += (uint64_t)gridDim.x * blockDim.x) {
        const float f = __uint_as_float((unsigned)i);
        if (!same_double(f32_to_f64(f), (double)f)) ++nb;
    }
    if (nb) atomicAdd(bad, nb);
}

__global__ void doubles(uint64_t n, unsigned long long *bad)
{
    unsigned long long nb = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = mix64(i);
        double x;
        switch (i & 3) {
        case 0:  // any bit pattern
            x = __longlong_as_double((long long)r);
            break;
        case 1: {  // exponents around the float range
            const uint64_t ex = 880 + (r >> 56) % 290;
            x = __longlong_as_double((long long)((r & 0x800fffffffffffffull) | (ex << 52)));
            break;
        }
        case 2: {  // exact ties and their neighbours between two floats
            const uint64_t ex = 897 + (r >> 56) % 254;
            uint64_t b = (r & 0x800fffffe0000000ull) | (ex << 52) | 0x10000000ull;
            b += (uint64_t)((int64_t)((r >> 40) % 3) - 1);
            x = __longlong_as_double((long long)b);
            break;
        }
        default: {  // offsets from zone centres of a unit grid
            const double c = ((double)(r >> 40) + 0.5) / 128.0;
            const double q = c + ((double)(r & 0xfffff) / 1048576.0 - 0.5) / 128.0;
            x = q - c;
            break;
        }
        }
        if (!same_float(f64_to_f32_rn(x), __double2float_rn(x))) ++nb;
        if (is_nan_f64(x) != (x != x)) ++nb;
    }
    if (nb) atomicAdd(bad, nb);
}

int main()
{
    unsigned long long *bad = nullptr, h[2] = {0, 0};
    if (cudaMalloc(&bad, 2 * sizeof(unsigned long long)) != cudaSuccess) return 2;
    cudaMemset(bad, 0, 2 * sizeof(unsigned long long));
    all_floats<<<4096, 256>>>(bad);
    doubles<<<4096, 256>>>(1ull << 30, bad + 1);
    if (cudaMemcpy(h, bad, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
    cudaFree(bad);
    printf("f32_to_f64 mismatches %llu\nf64_to_f32 mismatches %llu\n", h[0], h[1]);
    return (h[0] || h[1]) ? 1 : 0;
}
