// sgn_noalloc.cu - sgn_mass_energy_noalloc: the diagnostics reduction for
// callers that may not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework whose allocator owns and accounts for every byte of device memory,
// latency-critical loops where cudaMalloc/cudaFree would implicitly
// synchronize the device, and plugins or callbacks that are not permitted to
// create allocations of their own.  sgn_mass_energy needs a context (created
// by sgn_create, which allocates the RK registers and the reduction partials).
// This entry point needs no context: the caller passes the grid parameters,
// the bathymetry and the state, and the per-band partial sums live in the
// file-scope array below, which every GPU that loads the library holds until
// the process exits.
#include "sgn.h"
#include "sgn_kernels.cuh"

#include <cmath>
#include <mutex>

// defined in sgn_api.cu (not exported): stores the message sgn_last_error() returns
void sgn_record_error(const char* msg);

namespace {

// Largest grid the static scratch serves, counted in blocks of 32x16 nodes:
// 32768 blocks = 16,777,216 nodes, e.g. 4096 x 4096.  The diagnostics kernel
// (the FP64 stage kernel's tiles, 32 x kTileY nodes) writes one partial per
// 32 x 8 band: at most kMaxBands = 2 kMaxBlocks of them.
constexpr long long kMaxBlocks = 32768;
constexpr long long kMaxBands = 2 * kMaxBlocks;
constexpr int kTileY = sgn::THREADS_Y * sgn::StageShape<double>::rows;
constexpr size_t kSmem = sgn::stage_smem_bytes<double, sgn::MODE_DIAG>(sgn::StageShape<double>::rows);
// Layout of the scratch, in doubles: [partials: kMaxBands * NDIAG | out: NDIAG |
// flag (one int in the next double slot)].
constexpr long long kOutOffset = kMaxBands * sgn::NDIAG;
constexpr long long kFlagOffset = kOutOffset + sgn::NDIAG;
constexpr long long kScratchDoubles = kFlagOffset + 1;

// Device-side scratch.  In host code this name is only a stand-in; the device
// address is obtained with cudaGetSymbolAddress (see scratch_on_device).
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

sgn_status fail(sgn_status s, const char* msg) {
    sgn_record_error(msg);  // reported by sgn_last_error()
    return s;
}

bool device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Once per device, with that device current: the device address of the
// scratch array, and the shared-memory attribute of the kernel.
cudaError_t scratch_on_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        double* p = nullptr;
        e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        const size_t smem = kSmem;
        e = cudaFuncSetAttribute(sgn::k_stage<double, double, double, sgn::BC_PERIODIC, sgn::MODE_DIAG>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(sgn::k_stage<double, double, double, sgn::BC_REFLECTING, sgn::MODE_DIAG>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" SGN_API sgn_status sgn_mass_energy_noalloc(const sgn_params* p, const void* b_dev,
                                                      const void* q_dev, double* out, void* stream) {
    if (!p || !out) return fail(SGN_E_INVAL, "params and out must not be NULL");
    if (p->prec != SGN_F64) return fail(SGN_E_UNSUPPORTED, "only SGN_F64 (double state and bathymetry)");
    if (p->nx < 3 || p->ny < 3) return fail(SGN_E_INVAL, "need nx, ny >= 3");
    if (p->bc != SGN_BC_PERIODIC && p->bc != SGN_BC_REFLECTING) return fail(SGN_E_INVAL, "bad bc");
    if (!(std::isfinite(p->xmin) && std::isfinite(p->xmax) && p->xmax > p->xmin &&
          std::isfinite(p->ymin) && std::isfinite(p->ymax) && p->ymax > p->ymin))
        return fail(SGN_E_INVAL, "domain must be finite with xmax > xmin and ymax > ymin");
    if (!(std::isfinite(p->g) && p->g > 0.0) || !(std::isfinite(p->lambda) && p->lambda >= 0.0))
        return fail(SGN_E_INVAL, "need g > 0 and lambda >= 0, finite");
    const long long gx = (p->nx + sgn::TILE_X - 1) / sgn::TILE_X;
    const long long gy = (p->ny + kTileY - 1) / kTileY;
    if (gx * ((p->ny + 15) / 16) > kMaxBlocks)
        return fail(SGN_E_INVAL, "grid too large for the static scratch: at most 32768 blocks of "
                                 "32x16 nodes (16,777,216 nodes, e.g. 4096x4096)");
    if (!device_ptr(b_dev) || !device_ptr(q_dev)) return fail(SGN_E_INVAL, "b_dev and q_dev must be device memory");
    if (reinterpret_cast<uintptr_t>(q_dev) % 16 != 0) return fail(SGN_E_INVAL, "q_dev must be 16-byte aligned");

    double* scratch = nullptr;
    cudaError_t e = scratch_on_device(&scratch);
    if (e != cudaSuccess) return fail(SGN_E_CUDA, cudaGetErrorString(e));
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    const bool per = p->bc == SGN_BC_PERIODIC;
    const double dx = per ? (p->xmax - p->xmin) / p->nx : (p->xmax - p->xmin) / (p->nx - 1);
    const double dy = per ? (p->ymax - p->ymin) / p->ny : (p->ymax - p->ymin) / (p->ny - 1);
    sgn::StageArgs<double, double, double> a{};
    a.X = static_cast<const double*>(q_dev);
    a.b = static_cast<const double*>(b_dev);
    a.b64 = a.b;
    a.partials = scratch;
    a.flag = reinterpret_cast<int*>(scratch + kFlagOffset);
    sgn::fill_geom(a.G, p->nx, p->ny, dx, dy, p->g, p->lambda);

    // the flag must start at zero; the partials and out are fully overwritten
    e = cudaMemsetAsync(a.flag, 0, sizeof(int), s);
    if (e != cudaSuccess) return fail(SGN_E_CUDA, cudaGetErrorString(e));
    const dim3 grid((unsigned)gx, (unsigned)gy);
    const size_t smem = kSmem;
    if (per)
        sgn::k_stage<double, double, double, sgn::BC_PERIODIC, sgn::MODE_DIAG>
            <<<grid, dim3(sgn::TILE_X, sgn::THREADS_Y), smem, s>>>(a);
    else
        sgn::k_stage<double, double, double, sgn::BC_REFLECTING, sgn::MODE_DIAG>
            <<<grid, dim3(sgn::TILE_X, sgn::THREADS_Y), smem, s>>>(a);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        const long long nband = gx * ((p->ny + sgn::THREADS_Y - 1) / sgn::THREADS_Y);
        sgn::k_reduce_partials<<<1, 256, 0, s>>>(scratch, nband, scratch + kOutOffset);
        e = cudaGetLastError();
    }
    int flag = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, scratch + kOutOffset, sgn::NDIAG * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, a.flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(SGN_E_CUDA, cudaGetErrorString(e));
    if (flag & sgn::FLAG_BOUNDS) return fail(SGN_E_INVAL, "checked build: a tile index left its plane");
    if (flag & sgn::FLAG_NONFINITE) return fail(SGN_E_NONFINITE, "a state value had a non-finite water height");
    if (flag) return fail(SGN_E_NONPOSITIVE_H, "a state value had a non-positive water height");
    return SGN_OK;
}
