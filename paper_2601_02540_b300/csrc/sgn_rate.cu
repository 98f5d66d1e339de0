// sgn_rate.cu - sgn_measure_fp64_fma: the FP64 fused multiply-add rate of the
// current device, measured with a kernel of independent FMA chains.  The FP64
// stage kernels are bound by the FP64 pipe on B300 (two thread-operations per
// SM and clock against 128 for FP32), so their roofline is stated against
// this measured rate rather than a nominal figure.
#include "sgn.h"

#include <cuda_runtime.h>

// defined in sgn_api.cu (not exported)
void sgn_record_error(const char* msg);
void sgn_count_launches(unsigned long long n);

namespace {

constexpr int kChains = 16;         // independent chains per thread (hides the FMA latency)
constexpr int kUnroll = 4;          // iterations per loop trip (loop overhead off the issue path)
constexpr int kBlock = 256;
constexpr int kBlocksPerSm = 8;

// Each thread advances kChains values x <- x a + c, `iters` times (a multiple
// of kUnroll); with 0 < a < 1 every chain converges to c / (1 - a) (no
// overflow, no subnormals).  The sum of the chains is stored so that no FMA is dead code.
__global__ void __launch_bounds__(kBlock) k_fma_chains(int iters, double a, double c, double* out) {
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = 1.0 + 0.125 * k + 1e-9 * threadIdx.x;
    for (int it = 0; it < iters; it += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++)
#pragma unroll
            for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    out[(long long)blockIdx.x * kBlock + threadIdx.x] = s;
}

sgn_status fail(sgn_status st, const char* msg) {
    sgn_record_error(msg);
    return st;
}

}  // namespace

extern "C" SGN_API sgn_status sgn_measure_fp64_fma(int iters, double* fma_count, double* seconds,
                                                  void* stream) {
    if (!fma_count || !seconds) return fail(SGN_E_INVAL, "fma_count and seconds must not be NULL");
    if (iters < 1 || iters > (1 << 20) || iters % kUnroll != 0)
        return fail(SGN_E_INVAL, "iters must be a multiple of 4 in [4, 2^20]");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return fail(SGN_E_CUDA, "cannot read the SM count of the current device");
    }
    const long long blocks = (long long)sms * kBlocksPerSm;
    const long long threads = blocks * kBlock;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&out, (size_t)threads * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SGN_E_NOMEM, "sgn_measure_fp64_fma: output buffer");
    }
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        k_fma_chains<<<(unsigned)blocks, kBlock, 0, s>>>(iters, 0.999999, 1e-6, out);
        sgn_count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return fail(SGN_E_CUDA, cudaGetErrorString(e));
    *fma_count = (double)threads * kChains * (double)iters;
    *seconds = ms * 1e-3;
    return SGN_OK;
}
