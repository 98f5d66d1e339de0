// Accuracy of the library's reciprocals against the IEEE division, on the GPU
// (compiled and run by test_gpu_recip.py):
//   sgn::recip<double>  the hardware approximation refined by one third-order
//                       step; the bar is one ulp of the correctly rounded 1/h;
//   sgn::recip<float>   the float reciprocal of the FP32 kernels; the bar is
//                       one ulp of the correctly rounded 1/h;
//   sgn::recip_df64     the float approximation refined by one Newton step in
//                       double-word arithmetic; relative error against 1/h.
// Prints "samples N", "f64_max_ulp U", "f64_not_rounded C", "f32_max_ulp U",
// "f32_not_rounded C", "df64_max_rel R".
#include <cstdio>
#include <cstring>
#include <cuda_runtime.h>

#include "sgn_kernels.cuh"

__device__ unsigned long long g_max_ulp, g_not_rounded, g_max_ulp32, g_not_rounded32, g_max_rel_bits;

__global__ void check(long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long z = (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9ull; z ^= z >> 27; z *= 0x94D049BB133111EBull; z ^= z >> 31;
    // h = 2^s (1 + m), s in [-20, 20], m uniform in [0, 1) with 52 random bits
    const double m = (double)(z >> 12) * (1.0 / 4503599627370496.0);
    const int s = (int)(i % 41) - 20;
    const double h = ldexp(1.0 + m, s);
    const double ref = 1.0 / h;                                   // IEEE division
    const double r = sgn::recip<double>(h);
    const long long d = __double_as_longlong(r) - __double_as_longlong(ref);
    const unsigned long long ulp = (unsigned long long)(d < 0 ? -d : d);
    atomicMax(&g_max_ulp, ulp);
    if (ulp) atomicAdd(&g_not_rounded, 1ull);
    // float: h rounded to float (the same exponent range), against the IEEE quotient
    const float hf = __double2float_rn(h);
    const float ref32 = __fdiv_rn(1.0f, hf);
    const int d32 = __float_as_int(sgn::recip<float>(hf)) - __float_as_int(ref32);
    const unsigned long long ulp32 = (unsigned long long)(d32 < 0 ? -d32 : d32);
    atomicMax(&g_max_ulp32, ulp32);
    if (ulp32) atomicAdd(&g_not_rounded32, 1ull);
    const sgn::df64 w = sgn::recip_df64(sgn::df64_from_double(h));
    const double rel = fabs((sgn::double_of_df64(w) - ref) / ref);
    atomicMax(&g_max_rel_bits, (unsigned long long)__double_as_longlong(rel));
}

int main() {
    const long long n = 1LL << 24;
    check<<<(unsigned)((n + 255) / 256), 256>>>(n);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        printf("error %s\n", cudaGetErrorString(e));
        return 1;
    }
    unsigned long long ulp = 0, cnt = 0, ulp32 = 0, cnt32 = 0, rb = 0;
    cudaMemcpyFromSymbol(&ulp, g_max_ulp, sizeof(ulp));
    cudaMemcpyFromSymbol(&cnt, g_not_rounded, sizeof(cnt));
    cudaMemcpyFromSymbol(&ulp32, g_max_ulp32, sizeof(ulp32));
    cudaMemcpyFromSymbol(&cnt32, g_not_rounded32, sizeof(cnt32));
    cudaMemcpyFromSymbol(&rb, g_max_rel_bits, sizeof(rb));
    double rel;
    memcpy(&rel, &rb, sizeof(rel));
    printf("samples %lld\nf64_max_ulp %llu\nf64_not_rounded %llu\nf32_max_ulp %llu\nf32_not_rounded %llu\n"
           "df64_max_rel %.6e\n", n, ulp, cnt, ulp32, cnt32, rel);
    return 0;
}
