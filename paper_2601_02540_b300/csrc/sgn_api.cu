// sgn_api.cu - host side of libsgn.so: argument validation, context scratch,
// kernel dispatch and the C ABI declared in include/sgn.h.
#include "sgn.h"
#include "sgn_kernels.cuh"
#include "sgn_adjoint.cuh"
#include "sgn_adaptive.cuh"
#include "sgn_p5.cuh"
#include "sgn_rrk.cuh"
#include "sgn_mms.cuh"
#include "sgn_fused.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

using sgn::Geom;
using sgn::StageArgs;

namespace {

thread_local char g_err[512] = "";
std::atomic<unsigned long long> g_launches{0};

sgn_status fail(sgn_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

sgn_status cuda_fail(cudaError_t e, const char* what) {
    return fail(SGN_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(call, what)                               \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// launches recorded into a CUDA graph are counted when the graph is replayed
thread_local bool g_capturing = false;

void count_launch() {
    if (!g_capturing) g_launches.fetch_add(1, std::memory_order_relaxed);
}

}  // namespace

// Message for sgn_last_error() and the launch counter, for the other translation
// units of the library.
void sgn_record_error(const char* msg) { fail(SGN_E_INVAL, "%s", msg); }
void sgn_count_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

constexpr int kHostOut = sgn::NDIAG > sgn::NRRK ? sgn::NDIAG : sgn::NRRK;

struct sgn_ctx {
    sgn_params p;
    Geom G;
    size_t tc_size, ta_size;     // compute/stage-state and state element sizes
    double* b64 = nullptr;       // bathymetry in double
    void* bT = nullptr;          // bathymetry in the compute type (aliases b64 for F64)
    void* acc = nullptr;         // RK accumulator, state type
    void* Qa = nullptr;          // stage states, compute type
    void* Qb = nullptr;
    double* partials = nullptr;  // NDIAG per 32 x 8 band (diagnostics) or per block (adaptive error)
    double* dout = nullptr;      // NDIAG device
    double* hout = nullptr;      // pinned host results (kHostOut doubles: diagnostics, relaxation sums)
    int* flag = nullptr;         // device error bits
    int* hflag = nullptr;        // pinned host copy
    long long nblk = 0;          // blocks of the stage launch
    long long nband = 0;         // 32 x 8 bands of the grid: partials of the diagnostics
    dim3 grid;                   // blocks of the compute type's stage tile (StageShape)
    int rows = 0;                // tile height of the RK4 / RHS / diagnostics launches of k_stage
    int fuse = 0;                // FP32: two RK4 stages per launch (sgn_set_stage_fusion)
    dim3 gridr;                  // FP64: blocks of the 32 x (8 rows) tiles of the chosen height
    double* adj = nullptr;       // adjoint scratch (FP64): accumulator + two cotangents
    double* bs = nullptr;        // adaptive integrator scratch (8-byte slots, 40 planes)
    double* rrk = nullptr;       // relaxation scratch (FP64): plain RK4 update (5 planes), partials, sums
    double* mon = nullptr;       // per-step monitor sums of sgn_step_diag (NDIAG per step)
    int mon_cap = 0;
    void* hq = nullptr;          // device state of sgn_step_host (5 planes, state type)
    long long rrk_nblk = 0;
    // sgn_step on small grids: kGraphSteps RK4 steps captured once per (q, dt)
    // on a private stream and replayed on the caller's stream
    cudaStream_t cap = nullptr;
    cudaGraphExec_t step_exec = nullptr;
    const void* exec_q = nullptr;
    double exec_dt = 0.0;
};

namespace {

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

sgn_status check_state_ptr(const void* p, const char* name) {
    if (!p) return fail(SGN_E_INVAL, "%s is NULL", name);
    if (reinterpret_cast<uintptr_t>(p) % 16 != 0) return fail(SGN_E_INVAL, "%s is not 16-byte aligned", name);
    if (!is_device_ptr(p)) return fail(SGN_E_INVAL, "%s is not device memory", name);
    return SGN_OK;
}

// The opt-in to more than 48 KB of dynamic shared memory.  The runtime keeps
// this attribute per device, so it is set once per (kernel, device), with the
// device current; the result of that first call is kept for later launches.
constexpr int kMaxDevices = 64;
template <auto Kern>
cudaError_t smem_optin(size_t smem) {
    static std::once_flag once[kMaxDevices];
    static cudaError_t err[kMaxDevices];
    int dev = 0;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [&] {
        err[dev] = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    return err[dev];
}

template <typename TC, typename TIN, typename TA, int BC, int MODE, int R = sgn::StageShape<TC>::rows,
          bool TAPE = false>
cudaError_t stage_attr() {
    return smem_optin<sgn::k_stage<TC, TIN, TA, BC, MODE, R, TAPE>>(sgn::stage_smem_bytes<TC, MODE>(R));
}

template <typename TC, typename TIN, typename TA, int BC, int MODE, int R, bool TAPE>
cudaError_t launch_rows(dim3 grid, const StageArgs<TC, TIN, TA>& a, cudaStream_t s) {
    const cudaError_t attr_err = stage_attr<TC, TIN, TA, BC, MODE, R, TAPE>();
    if (attr_err != cudaSuccess) return attr_err;
    sgn::k_stage<TC, TIN, TA, BC, MODE, R, TAPE>
        <<<grid, dim3(sgn::TILE_X, sgn::THREADS_Y), sgn::stage_smem_bytes<TC, MODE>(R), s>>>(a);
    count_launch();
    return cudaGetLastError();
}

// The stage kernel with the context's tile height: FP64 contexts take the
// height sgn_create chose (c->rows: 32 x 8, 32 x 16 or 32 x 24 tiles), all
// others the compute type's StageShape.  TAPE: the FP64 kernel that also
// writes the tape.
template <typename TC, typename TIN, typename TA, int BC, int MODE, bool TAPE = false>
cudaError_t launch_stage(const sgn_ctx* c, const StageArgs<TC, TIN, TA>& a, cudaStream_t s) {
    if constexpr (std::is_same<TC, double>::value) {
        static_assert(sgn::StageShape<double>::rows == 3, "FP64 tile heights 8, 16, 24");
        if (c->rows == 1) return launch_rows<TC, TIN, TA, BC, MODE, 1, TAPE>(c->gridr, a, s);
        if (c->rows == 2) return launch_rows<TC, TIN, TA, BC, MODE, 2, TAPE>(c->gridr, a, s);
    }
    constexpr int R = sgn::StageShape<TC>::rows;
    const cudaError_t attr_err = stage_attr<TC, TIN, TA, BC, MODE, R, TAPE>();
    if (attr_err != cudaSuccess) return attr_err;
    const size_t smem = sgn::stage_smem_bytes<TC, MODE>(R);
    sgn::k_stage<TC, TIN, TA, BC, MODE, R, TAPE><<<c->grid, dim3(sgn::TILE_X, sgn::THREADS_Y), smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <typename TC, typename TIN, typename TA>
StageArgs<TC, TIN, TA> base_args(const sgn_ctx* c) {
    StageArgs<TC, TIN, TA> a;
    std::memset(&a, 0, sizeof(a));
    a.b = static_cast<const TC*>(c->bT);
    a.b64 = c->b64;
    a.flag = c->flag;
    a.G = c->G;
    return a;
}

// nsteps RK4 steps; with `mon` the fourth stage also reduces the mass and
// energies of each new state into mon[NDIAG n ..] (mode S4D).
// FP32 steps with two stages per launch (sgn_fused.cuh): S12 and S34 per
// step; q_{n+1} goes to the other of q and the context's Qb (S34 reads q_n on
// its halo), and an odd step count ends with a copy back into q.
template <typename TC, typename TA, int BC>
cudaError_t run_steps_fused(sgn_ctx* c, TA* q, double dt, int nsteps, cudaStream_t s) {
    constexpr int R = sgn::StageShape<TC>::rows;
    constexpr bool kW = sgn::kFusedW32<BC, sgn::FUSED_S34>;
    // 32-bit element offsets (where the kernel takes them) for planes below 2^32 nodes
    const bool w32 = kW && (unsigned long long)c->G.plane <= 0xffffffffull;
    const size_t smem = sgn::FusedLayout<R>::template bytes<TC>();
    cudaError_t e = smem_optin<sgn::k_fused<TC, TA, BC, sgn::FUSED_S12, R>>(smem);
    if (e == cudaSuccess) e = smem_optin<sgn::k_fused<TC, TA, BC, sgn::FUSED_S34, R>>(smem);
    if (e == cudaSuccess && kW) e = smem_optin<sgn::k_fused<TC, TA, BC, sgn::FUSED_S34, R, kW>>(smem);
    if (e != cudaSuccess) return e;
    sgn::FusedArgs<TC, TA> f;
    std::memset(&f, 0, sizeof(f));
    f.b = static_cast<const TC*>(c->bT);
    f.flag = c->flag;
    f.G = c->G;
    f.acc = static_cast<TA*>(c->acc);
    // the coefficients of run_steps, rounded the same way
    f.c_a1 = (TA)(dt / 6.0); f.c_a2 = (TA)(dt / 3.0); f.c_a3 = (TA)(dt / 3.0); f.c_a4 = (TA)(dt / 6.0);
    f.c_q1 = (TA)(dt / 2.0); f.c_q2 = (TA)(dt / 2.0); f.c_q3 = (TA)dt;
    static_assert(std::is_same<TC, TA>::value, "Qb holds a state");
    TA* cur = q;
    TA* nxt = static_cast<TA*>(c->Qb);
    const dim3 block(sgn::TILE_X, sgn::THREADS_Y);
    for (int n = 0; n < nsteps; n++) {
        sgn::FusedArgs<TC, TA> f12 = f;
        f12.q = cur;
        f12.Qout = static_cast<TC*>(c->Qa);
        sgn::k_fused<TC, TA, BC, sgn::FUSED_S12, R><<<c->grid, block, smem, s>>>(f12);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        sgn::FusedArgs<TC, TA> f34 = f;
        f34.q = cur;
        f34.X = static_cast<const TC*>(c->Qa);
        f34.out = nxt;
        if (w32)
            sgn::k_fused<TC, TA, BC, sgn::FUSED_S34, R, kW><<<c->grid, block, smem, s>>>(f34);
        else
            sgn::k_fused<TC, TA, BC, sgn::FUSED_S34, R><<<c->grid, block, smem, s>>>(f34);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        std::swap(cur, nxt);
    }
    if (cur != q) e = cudaMemcpyAsync(q, cur, (size_t)5 * c->G.plane * sizeof(TA), cudaMemcpyDeviceToDevice, s);
    return e;
}

template <typename TC, typename TA, int BC>
cudaError_t run_steps(sgn_ctx* c, TA* q, double dt, int nsteps, cudaStream_t s, double* mon = nullptr) {
    if constexpr (sgn::kStoreK1<TC, TA>) {
        if (c->fuse && !mon) return run_steps_fused<TC, TA, BC>(c, q, dt, nsteps, s);
    }
    TA* acc = static_cast<TA*>(c->acc);
    TC* Qa = static_cast<TC*>(c->Qa);
    TC* Qb = static_cast<TC*>(c->Qb);
    const TA dt6 = (TA)(dt / 6.0), dt3 = (TA)(dt / 3.0), dt2 = (TA)(dt / 2.0), dt1 = (TA)dt;
    StageArgs<TC, TA, TA> a1 = base_args<TC, TA, TA>(c);
    a1.X = q; a1.qn = q; a1.acc = acc; a1.Qout = Qa; a1.c_acc = dt6; a1.c_q = dt2;
    StageArgs<TC, TC, TA> a2 = base_args<TC, TC, TA>(c);
    a2.X = Qa; a2.qn = q; a2.acc = acc; a2.Qout = Qb; a2.c_acc = dt3; a2.c_q = dt2;
    StageArgs<TC, TC, TA> a3 = a2;
    a3.X = Qb; a3.Qout = Qa; a3.c_acc = dt3; a3.c_q = dt1;
    StageArgs<TC, TC, TA> a4 = base_args<TC, TC, TA>(c);
    a4.X = Qa; a4.acc = acc; a4.out = q; a4.c_acc = dt6;
    // FP32: stage 1 stores only k1 (in Qa) and stage 2 forms q_n + dt/2 k1 and
    // the accumulator itself (modes S1K, S2K; kStoreK1)
    constexpr bool kK1 = sgn::kStoreK1<TC, TA>;
    a2.c_acc1 = dt6;
    a2.c_q1 = dt2;
    for (int n = 0; n < nsteps; n++) {
        cudaError_t e;
        if constexpr (kK1) {
            // k1 = f(q_n) -> Qa; k2 = f(q_n + dt/2 k1), acc = q_n + dt/6 k1 + dt/3 k2
            if ((e = launch_stage<TC, TA, TA, BC, sgn::MODE_S1K>(c, a1, s)) != cudaSuccess) return e;
            if ((e = launch_stage<TC, TC, TA, BC, sgn::MODE_S2K>(c, a2, s)) != cudaSuccess) return e;
        } else {
            // k1 = f(q_n)
            if ((e = launch_stage<TC, TA, TA, BC, sgn::MODE_S1>(c, a1, s)) != cudaSuccess) return e;
            // k2 = f(q_n + dt/2 k1)
            if ((e = launch_stage<TC, TC, TA, BC, sgn::MODE_S2>(c, a2, s)) != cudaSuccess) return e;
        }
        // k3 = f(q_n + dt/2 k2)
        if ((e = launch_stage<TC, TC, TA, BC, sgn::MODE_S3>(c, a3, s)) != cudaSuccess) return e;
        // k4 = f(q_n + dt k3); q_{n+1} = acc + dt/6 k4
        if (!mon) {
            if ((e = launch_stage<TC, TC, TA, BC, sgn::MODE_S4>(c, a4, s)) != cudaSuccess) return e;
        } else {
            StageArgs<TC, TC, TA> a4d = a4;
            a4d.partials = c->partials;
            if ((e = launch_stage<TC, TC, TA, BC, sgn::MODE_S4D>(c, a4d, s)) != cudaSuccess) return e;
            sgn::k_reduce_partials<<<1, 256, 0, s>>>(c->partials, c->nband, mon + (long long)n * sgn::NDIAG);
            count_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

template <typename TC, typename TA, int BC>
cudaError_t run_rhs(sgn_ctx* c, const TA* q, TA* dq, cudaStream_t s) {
    StageArgs<TC, TA, TA> a = base_args<TC, TA, TA>(c);
    a.X = q; a.out = dq;
    return launch_stage<TC, TA, TA, BC, sgn::MODE_RHS>(c, a, s);
}

template <typename TC, typename TA, int BC>
cudaError_t run_diag(sgn_ctx* c, const TA* q, cudaStream_t s) {
    StageArgs<TC, TA, TA> a = base_args<TC, TA, TA>(c);
    a.X = q; a.partials = c->partials;
    cudaError_t e = launch_stage<TC, TA, TA, BC, sgn::MODE_DIAG>(c, a, s);
    if (e != cudaSuccess) return e;
    sgn::k_reduce_partials<<<1, 256, 0, s>>>(c->partials, c->nband, c->dout);
    count_launch();
    return cudaGetLastError();
}

template <typename TA, int BC>
cudaError_t run_init(sgn_ctx* c, TA* q, cudaStream_t s) {
    dim3 blk(32, 8), grd((c->p.nx + 31) / 32, (c->p.ny + 7) / 8);
    sgn::k_init_aux<TA, BC><<<grd, blk, 0, s>>>(q, c->b64, c->G);
    count_launch();
    return cudaGetLastError();
}

// dispatch on (precision, boundary) to a functor templated on <TC, TA, BC>
template <typename F>
cudaError_t dispatch(const sgn_ctx* c, F& f) {
    const bool refl = c->p.bc == SGN_BC_REFLECTING;
    switch (c->p.prec) {
    case SGN_F64:
        return refl ? f.template operator()<double, double, sgn::BC_REFLECTING>()
                    : f.template operator()<double, double, sgn::BC_PERIODIC>();
    case SGN_F32:
        return refl ? f.template operator()<float, float, sgn::BC_REFLECTING>()
                    : f.template operator()<float, float, sgn::BC_PERIODIC>();
    case SGN_DF64:
        return refl ? f.template operator()<sgn::df64, double, sgn::BC_REFLECTING>()
                    : f.template operator()<sgn::df64, double, sgn::BC_PERIODIC>();
    default:
        return refl ? f.template operator()<float, double, sgn::BC_REFLECTING>()
                    : f.template operator()<float, double, sgn::BC_PERIODIC>();
    }
}

struct RhsOp {
    sgn_ctx* c; const void* q; void* dq; cudaStream_t s;
    template <typename TC, typename TA, int BC>
    cudaError_t operator()() { return run_rhs<TC, TA, BC>(c, static_cast<const TA*>(q), static_cast<TA*>(dq), s); }
};

struct StepOp {
    sgn_ctx* c; void* q; double dt; int n; cudaStream_t s;
    template <typename TC, typename TA, int BC>
    cudaError_t operator()() { return run_steps<TC, TA, BC>(c, static_cast<TA*>(q), dt, n, s); }
};

struct StepDiagOp {
    sgn_ctx* c; void* q; double dt; int n; double* mon; cudaStream_t s;
    template <typename TC, typename TA, int BC>
    cudaError_t operator()() { return run_steps<TC, TA, BC>(c, static_cast<TA*>(q), dt, n, s, mon); }
};

// the shared-memory opt-in of the four RK4 stage kernels of a context
struct AttrOp {
    sgn_ctx* c;
    template <typename TC, typename TA, int BC>
    cudaError_t operator()() {
        if constexpr (std::is_same<TC, double>::value) {
            if (c->rows == 1) return attrs<TC, TA, BC, 1>();
            if (c->rows == 2) return attrs<TC, TA, BC, 2>();
        }
        return attrs<TC, TA, BC, sgn::StageShape<TC>::rows>();
    }
    template <typename TC, typename TA, int BC, int R>
    cudaError_t attrs() {
        constexpr bool kK1 = sgn::kStoreK1<TC, TA>;     // the stage modes run_steps launches
        if constexpr (kK1) {
            // the fused kernels of run_steps_fused
            const size_t smem = sgn::FusedLayout<R>::template bytes<TC>();
            constexpr bool kW = sgn::kFusedW32<BC, sgn::FUSED_S34>;
            cudaError_t ef = smem_optin<sgn::k_fused<TC, TA, BC, sgn::FUSED_S12, R>>(smem);
            if (ef == cudaSuccess) ef = smem_optin<sgn::k_fused<TC, TA, BC, sgn::FUSED_S34, R>>(smem);
            if (ef == cudaSuccess && kW) ef = smem_optin<sgn::k_fused<TC, TA, BC, sgn::FUSED_S34, R, kW>>(smem);
            if (ef != cudaSuccess) return ef;
        }
        cudaError_t e = stage_attr<TC, TA, TA, BC, kK1 ? sgn::MODE_S1K : sgn::MODE_S1, R>();
        if (e == cudaSuccess) e = stage_attr<TC, TC, TA, BC, kK1 ? sgn::MODE_S2K : sgn::MODE_S2, R>();
        if (e == cudaSuccess) e = stage_attr<TC, TC, TA, BC, sgn::MODE_S3, R>();
        if (e == cudaSuccess) e = stage_attr<TC, TC, TA, BC, sgn::MODE_S4, R>();
        return e;
    }
};

struct DiagOp {
    sgn_ctx* c; const void* q; cudaStream_t s;
    template <typename TC, typename TA, int BC>
    cudaError_t operator()() { return run_diag<TC, TA, BC>(c, static_cast<const TA*>(q), s); }
};

// Small grids are launch-bound (four short launches per step): sgn_step
// replays a CUDA graph of kGraphSteps steps there.  The graph is captured once
// per (state pointer, dt) on the context's private stream (the same launches
// as the direct path, so the same results bit for bit) and launched on the
// caller's stream; a caller that is itself capturing gets the direct launches.
constexpr int kGraphSteps = 50;
constexpr long long kGraphMaxCells = 1LL << 21;

sgn_status step_graph(sgn_ctx* c, void* q, double dt) {
    if (c->step_exec && c->exec_q == q && c->exec_dt == dt) return SGN_OK;
    if (c->step_exec) {
        cudaGraphExecDestroy(c->step_exec);
        c->step_exec = nullptr;
    }
    if (!c->cap) CUDA_TRY(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking), "capture stream");
    AttrOp fa{c};                // kernel attributes are set outside the capture
    CUDA_TRY(dispatch(c, fa), "stage kernel attributes");
    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    StepOp f{c, q, dt, kGraphSteps, c->cap};
    g_capturing = true;
    const cudaError_t el = dispatch(c, f);
    g_capturing = false;
    const cudaError_t ec = cudaStreamEndCapture(c->cap, &graph);
    if (el != cudaSuccess || ec != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(el != cudaSuccess ? el : ec, "capture");
    }
    const cudaError_t ei = cudaGraphInstantiate(&c->step_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        c->step_exec = nullptr;
        return cuda_fail(ei, "instantiate graph");
    }
    c->exec_q = q;
    c->exec_dt = dt;
    return SGN_OK;
}

sgn_status read_flag(sgn_ctx* c, cudaStream_t s) {
    CUDA_TRY(cudaMemcpyAsync(c->hflag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, s), "read flag");
    CUDA_TRY(cudaStreamSynchronize(s), "synchronize");
    const int f = *c->hflag;
    if (f) {
        CUDA_TRY(cudaMemsetAsync(c->flag, 0, sizeof(int), s), "clear flag");
        CUDA_TRY(cudaStreamSynchronize(s), "synchronize");
        if (f & sgn::FLAG_BOUNDS) return fail(SGN_E_INVAL, "checked build: a tile index left its plane");
        if (f & sgn::FLAG_NONFINITE) return fail(SGN_E_NONFINITE, "a stage input had a non-finite water height");
        return fail(SGN_E_NONPOSITIVE_H, "a stage input had a non-positive water height");
    }
    return SGN_OK;
}

void free_ctx(sgn_ctx* c) {
    if (!c) return;
    if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->bT && c->bT != c->b64) cudaFree(c->bT);
    cudaFree(c->b64);
    cudaFree(c->acc);
    cudaFree(c->Qa);
    cudaFree(c->Qb);
    cudaFree(c->partials);
    cudaFree(c->dout);
    cudaFree(c->flag);
    cudaFree(c->adj);
    cudaFree(c->bs);
    cudaFree(c->rrk);
    cudaFree(c->mon);
    cudaFree(c->hq);
    cudaFreeHost(c->hout);
    cudaFreeHost(c->hflag);
    delete c;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// The compute-type copy of the bathymetry (float or df64) from the double one.
cudaError_t convert_bathymetry(sgn_ctx* c, cudaStream_t s) {
    const long long n = c->G.plane;
    if (c->p.prec == SGN_DF64)
        sgn::k_convert<sgn::df64><<<592, 256, 0, s>>>(c->b64, static_cast<sgn::df64*>(c->bT), n);
    else
        sgn::k_convert<float><<<592, 256, 0, s>>>(c->b64, static_cast<float*>(c->bT), n);
    count_launch();
    return cudaGetLastError();
}

// The tape of f(X) (TAPE mode of the FP64 stage kernel), for a VJP whose
// caller recorded none.
template <int BC>
cudaError_t launch_tape(const sgn_ctx* c, const double* X, double* tape, cudaStream_t s) {
    StageArgs<double, double, double> t = base_args<double, double, double>(c);
    t.X = X;
    t.tape = tape;
    return launch_stage<double, double, double, BC, sgn::MODE_TAPE, true>(c, t, s);
}

// J(X)^T (sigma A): the tape of f(X) from a.tape or, when that is NULL, from a
// TAPE launch into `scratch_tape`; then the two adjoint passes.
template <int BC, int MODE>
cudaError_t launch_adjoint(const sgn_ctx* c, sgn::AdjArgs a, double* scratch_tape, cudaStream_t s) {
    cudaError_t e;
    if (!a.tape) {
        if ((e = launch_tape<BC>(c, a.X, scratch_tape, s)) != cudaSuccess) return e;
        a.tape = scratch_tape;
    }
    const unsigned blocks = (unsigned)((c->G.plane + sgn::ADJ_BLOCK - 1) / sgn::ADJ_BLOCK);
    sgn::k_adj_point<BC><<<blocks, sgn::ADJ_BLOCK, 0, s>>>(a);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    sgn::k_adj_gather<BC, MODE><<<blocks, sgn::ADJ_BLOCK, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

// Adjoint scratch, allocated on first use: the RK accumulator of the
// cotangents (5 planes), two buffers of weights and node parts
// (ADJ_SCRATCH_PLANES each: a chained walk alternates them), two tapes
// (N_TAPE each).
constexpr long long kAdjScratchA = 5;
constexpr long long kAdjScratchB = kAdjScratchA + sgn::ADJ_SCRATCH_PLANES;
constexpr long long kAdjTapeOffset = kAdjScratchA + 2 * sgn::ADJ_SCRATCH_PLANES;
static_assert(SGN_TAPE_PLANES == sgn::N_TAPE, "the header's tape size");

template <int MODE>
cudaError_t adjoint(const sgn_ctx* c, const sgn::AdjArgs& a, cudaStream_t s) {
    double* scratch_tape = c->adj + kAdjTapeOffset * c->G.plane;
    return c->p.bc == SGN_BC_REFLECTING ? launch_adjoint<sgn::BC_REFLECTING, MODE>(c, a, scratch_tape, s)
                                        : launch_adjoint<sgn::BC_PERIODIC, MODE>(c, a, scratch_tape, s);
}

// The walk of one step: pass 1 of stage 4, then pass 2 of stages 4, 3, 2
// each chained with pass 1 of the stage before it (k_adj_gather_point,
// alternating the two weight buffers), then pass 2 of stage 1: five launches.
// `g[s]` are the stage-mode arguments of stage s+1 (weights in buffer A for
// stages 4 and 2, B for 3 and 1).  With `tapes`, the tape of each stage is
// first computed from its state (a TAPE launch) into g[s].tape, just before
// the launch that first reads it: nine launches.
template <int BC>
cudaError_t chained_walk(const sgn_ctx* c, const sgn::AdjArgs g[4], bool tapes, cudaStream_t s) {
    const unsigned blocks = (unsigned)((c->G.plane + sgn::ADJ_BLOCK - 1) / sgn::ADJ_BLOCK);
    cudaError_t e = cudaSuccess;
    if (tapes && (e = launch_tape<BC>(c, g[3].X, const_cast<double*>(g[3].tape), s)) != cudaSuccess) return e;
    sgn::k_adj_point<BC><<<blocks, sgn::ADJ_BLOCK, 0, s>>>(g[3]);
    count_launch();
    e = cudaGetLastError();
    for (int st = 3; st >= 1 && e == cudaSuccess; st--) {
        if (tapes && (e = launch_tape<BC>(c, g[st - 1].X, const_cast<double*>(g[st - 1].tape), s)) != cudaSuccess)
            return e;
        sgn::k_adj_gather_point<BC><<<blocks, sgn::ADJ_BLOCK, 0, s>>>(g[st], g[st - 1]);
        count_launch();
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    sgn::k_adj_gather<BC, sgn::ADJ_MODE_STAGE><<<blocks, sgn::ADJ_BLOCK, 0, s>>>(g[0]);
    count_launch();
    return cudaGetLastError();
}

sgn_status adjoint_scratch(sgn_ctx* c) {
    if (c->adj) return SGN_OK;
    const size_t bytes = (size_t)(kAdjTapeOffset + 2 * sgn::N_TAPE) * (size_t)c->G.plane * sizeof(double);
    if (cudaMalloc(&c->adj, bytes) != cudaSuccess) {
        cudaGetLastError();
        c->adj = nullptr;
        return fail(SGN_E_NOMEM, "adjoint scratch (%zu bytes)", bytes);
    }
    return SGN_OK;
}

// One RK4 step that also records its stage states: stash = [q_n | Q2 | Q3 | Q4],
// and, with TAPE, the tapes of its four right-hand sides: tape = [T1 | T2 | T3 | T4]
// (N_TAPE planes each), written by the stage kernels themselves.
template <int BC, bool TAPE>
cudaError_t record_step(sgn_ctx* c, double* q, double dt, double* stash, double* tape, cudaStream_t s) {
    const long long P5 = 5 * c->G.plane;
    const long long PT = (long long)sgn::N_TAPE * c->G.plane;
    double* acc = static_cast<double*>(c->acc);
    cudaError_t e = cudaMemcpyAsync(stash, q, P5 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    StageArgs<double, double, double> a1 = base_args<double, double, double>(c);
    a1.X = q; a1.qn = q; a1.acc = acc; a1.Qout = stash + P5; a1.c_acc = dt / 6.0; a1.c_q = dt / 2.0;
    a1.tape = tape;
    if ((e = launch_stage<double, double, double, BC, sgn::MODE_S1, TAPE>(c, a1, s)) != cudaSuccess) return e;
    StageArgs<double, double, double> a2 = a1;
    a2.X = stash + P5; a2.Qout = stash + 2 * P5; a2.c_acc = dt / 3.0; a2.c_q = dt / 2.0;
    a2.tape = TAPE ? tape + PT : nullptr;
    if ((e = launch_stage<double, double, double, BC, sgn::MODE_S2, TAPE>(c, a2, s)) != cudaSuccess) return e;
    StageArgs<double, double, double> a3 = a1;
    a3.X = stash + 2 * P5; a3.Qout = stash + 3 * P5; a3.c_acc = dt / 3.0; a3.c_q = dt;
    a3.tape = TAPE ? tape + 2 * PT : nullptr;
    if ((e = launch_stage<double, double, double, BC, sgn::MODE_S3, TAPE>(c, a3, s)) != cudaSuccess) return e;
    StageArgs<double, double, double> a4 = base_args<double, double, double>(c);
    a4.X = stash + 3 * P5; a4.acc = acc; a4.out = q; a4.c_acc = dt / 6.0;
    a4.tape = TAPE ? tape + 3 * PT : nullptr;
    return launch_stage<double, double, double, BC, sgn::MODE_S4, TAPE>(c, a4, s);
}

sgn_status need_f64(const sgn_ctx* c, const char* what) {
    if (c->p.prec != SGN_F64) return fail(SGN_E_UNSUPPORTED, "%s: the adjoint is implemented for SGN_F64 only", what);
    return SGN_OK;
}

// ---- adaptive integrator (Sec. 6), second pair: Bogacki-Shampine 3(2), host-side control
template <typename TC, int BC, int MODE, int R>
cudaError_t launch_bs3_rows(dim3 grid, const sgn::BsArgs& a, cudaStream_t s) {
    const size_t smem = sgn::stage_smem_bytes<TC, sgn::MODE_RHS>(R);
    const cudaError_t attr_err = smem_optin<sgn::k_bs3_stage<TC, BC, MODE, R>>(smem);
    if (attr_err != cudaSuccess) return attr_err;
    sgn::k_bs3_stage<TC, BC, MODE, R><<<grid, dim3(sgn::TILE_X, sgn::THREADS_Y), smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

// The pair's stage kernels take the context's FP64 tile height, as the RK4
// stage kernels do (the last stage writes one error partial per block).
template <typename TC, int BC, int MODE>
cudaError_t launch_bs3(const sgn_ctx* c, const sgn::BsArgs& a, cudaStream_t s) {
    if constexpr (std::is_same<TC, double>::value) {
        if (c->rows == 1) return launch_bs3_rows<TC, BC, MODE, 1>(c->gridr, a, s);
        if (c->rows == 2) return launch_bs3_rows<TC, BC, MODE, 2>(c->gridr, a, s);
    }
    return launch_bs3_rows<TC, BC, MODE, sgn::StageShape<TC>::rows>(c->grid, a, s);
}

// Blocks of the adaptive pairs' launches (error partials to reduce).
template <typename TC>
long long pair_blocks(const sgn_ctx* c) {
    if (std::is_same<TC, double>::value) return (long long)c->gridr.x * c->gridr.y;
    return c->nblk;
}

// Bogacki-Shampine 3(2): weights of the third-order solution and of the
// embedded second-order one (its stage 4 is f(q_{n+1}), the FSAL stage).
constexpr double BS_B1 = 2.0 / 9.0, BS_B2 = 1.0 / 3.0, BS_B3 = 4.0 / 9.0;
constexpr double BS_E1 = 2.0 / 9.0 - 7.0 / 24.0, BS_E2 = 1.0 / 3.0 - 1.0 / 4.0;
constexpr double BS_E3 = 4.0 / 9.0 - 1.0 / 3.0, BS_E4 = -1.0 / 8.0;
// step-size control: dt_next = dt min(QMAX, max(QMIN, SAFETY err^(-1/3)))
constexpr double BS_SAFETY = 0.9, BS_QMIN = 0.2, BS_QMAX = 10.0;

template <typename TC, int BC>
sgn_status run_adaptive(sgn_ctx* c, double* q_user, double t0, double t_end, double dt0, double rtol,
                        double atol, int max_attempts, double* hist, double* stats, cudaStream_t s) {
    const long long P5 = 5 * c->G.plane;
    const size_t bytes5 = (size_t)P5 * sizeof(double);
    static_assert(sizeof(TC) == sizeof(double), "the slots below hold 8-byte values");
    TC* k1 = reinterpret_cast<TC*>(c->bs);
    TC* k2 = reinterpret_cast<TC*>(c->bs + P5);
    TC* k3 = reinterpret_cast<TC*>(c->bs + 2 * P5);
    TC* k4 = reinterpret_cast<TC*>(c->bs + 3 * P5);
    TC* Y3 = reinterpret_cast<TC*>(c->bs + 4 * P5);
    double* q1 = c->bs + 5 * P5;
    double* qc = c->bs + 6 * P5;
    CUDA_TRY(cudaMemcpyAsync(qc, q_user, bytes5, cudaMemcpyDeviceToDevice, s), "copy q");
    {
        // k1 = f(q), stored in the compute type
        StageArgs<TC, double, TC> r = base_args<TC, double, TC>(c);
        r.X = qc;
        r.out = k1;
        CUDA_TRY((launch_stage<TC, double, TC, BC, sgn::MODE_RHS>(c, r, s)), "k1");
    }
    sgn_status st = read_flag(c, s);
    if (st != SGN_OK) return st;

    sgn::BsArgs a;
    std::memset(&a, 0, sizeof(a));
    a.b = c->bT;                 // bathymetry in the compute type (the double one for FP64)
    a.flag = c->flag;
    a.G = c->G;
    a.rtol = rtol;
    a.atol = atol;
    a.partials = c->partials;
    double t = t0, dt = dt0;
    int acc = 0, rej = 0, n = 0;
    while (t < t_end && n < max_attempts) {
        const bool last = dt >= t_end - t;
        const double h = last ? t_end - t : dt;
        a.q = qc;
        a.k1 = k1;
        a.k2 = k2;
        a.k3 = k3;
        // k2 = f(q + h/2 k1); Y3 = q + 3h/4 k2
        a.c_in = 0.5 * h;
        a.c_y = 0.75 * h;
        a.kout = k2;
        a.Y3 = Y3;
        a.q1 = q1;
        CUDA_TRY((launch_bs3<TC, BC, sgn::BS_K2>(c, a, s)), "adaptive stage 2");
        // k3 = f(Y3); q1 = q + h (b1 k1 + b2 k2 + b3 k3)
        a.kout = k3;
        a.cb1 = h * BS_B1;
        a.cb2 = h * BS_B2;
        a.cb3 = h * BS_B3;
        CUDA_TRY((launch_bs3<TC, BC, sgn::BS_K3>(c, a, s)), "adaptive stage 3");
        // k4 = f(q1); error partial sums
        a.kout = k4;
        a.ce1 = h * BS_E1;
        a.ce2 = h * BS_E2;
        a.ce3 = h * BS_E3;
        a.ce4 = h * BS_E4;
        CUDA_TRY((launch_bs3<TC, BC, sgn::BS_K4>(c, a, s)), "adaptive stage 4");
        sgn::k_reduce_partials<<<1, 256, 0, s>>>(c->partials, pair_blocks<TC>(c), c->dout);
        count_launch();
        CUDA_TRY(cudaGetLastError(), "error reduction");
        CUDA_TRY(cudaMemcpyAsync(c->hout, c->dout, sizeof(double), cudaMemcpyDeviceToHost, s), "copy error");
        CUDA_TRY(cudaMemcpyAsync(c->hflag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, s), "copy flag");
        CUDA_TRY(cudaStreamSynchronize(s), "synchronize");
        double err;
        if (*c->hflag) {
            // a trial stage left the admissible states: reject as an infinite error
            CUDA_TRY(cudaMemsetAsync(c->flag, 0, sizeof(int), s), "clear flag");
            err = INFINITY;
        } else {
            err = std::sqrt(c->hout[0] / (double)P5);
        }
        const bool ok = err <= 1.0;
        const double fac = err == 0.0 ? BS_QMAX
                                      : std::fmin(BS_QMAX, std::fmax(BS_QMIN, BS_SAFETY * std::pow(err, -1.0 / 3.0)));
        if (hist) {
            hist[3 * n] = h;
            hist[3 * n + 1] = err;
            hist[3 * n + 2] = ok ? 1.0 : 0.0;
        }
        if (ok) {
            std::swap(qc, q1);
            std::swap(k1, k4);
            t = last ? t_end : t + h;
            acc++;
        } else {
            rej++;
        }
        dt = h * fac;
        n++;
    }
    CUDA_TRY(cudaMemcpyAsync(q_user, qc, bytes5, cudaMemcpyDeviceToDevice, s), "copy q back");
    CUDA_TRY(cudaStreamSynchronize(s), "synchronize");
    stats[0] = acc;
    stats[1] = rej;
    stats[2] = t;
    stats[3] = dt;
    stats[4] = n;
    return SGN_OK;
}

// ---- the five-stage third-order FSAL pair (Sec. 6) -------------------------
// Butcher matrix of the two-register form (a_ij = b_j for j < i-1): the
// sub-diagonal a21, a32, a43, a54, the weights b and the embedded weights bhat
// over k1..k5 and k6 = f(q_{n+1}).  Constructed for this library: stability
// polynomial 1 + z + z^2/2 + z^3/6 + 0.0324 z^4 + 0.006 z^5 (imaginary-axis
// stability up to |z| = 3.8798), third order, embedded second order.
constexpr double P5_A21 = 0.3464, P5_A32 = 0.5544, P5_A43 = 0.3078, P5_A54 = 0.25084211224332113157;
constexpr double P5_B[5] = {-0.077114705798502101362, 0.51296293729322573879, -0.53636230691175187515,
                            0.69586264419699749322, 0.40465143122003074449};
constexpr double P5_BHAT[6] = {0.14576960111557976478, 0.13123039888442023522, 0.103, 0.1816, 0.1978, 0.2406};
// Step-size control with the limiter rho(x) = 1 + atan(x - 1) and
// eps = 0.9 / max(err, 1e-10): an accepted attempt sets dt_next = dt rho(x)
// with x = eps^(0.7/3) eps_prev^(-0.4/3) (Gustafsson's stabilized PI control;
// eps_prev of the previous accepted attempt, 1 before the first), a rejected
// one dt_next = dt rho(eps^(1/3)).
constexpr double P5_PI_B1 = 0.7, P5_PI_B2 = -0.4, P5_PI_K = 3.0, P5_ERR_FLOOR = 1e-10, P5_SAFETY = 0.9;

template <typename TC, int BC, int MODE, int R>
cudaError_t launch_p5_rows(dim3 grid, const sgn::P5Args& a, cudaStream_t s) {
    const size_t smem = sgn::stage_smem_bytes<TC, sgn::MODE_RHS>(R);
    const cudaError_t attr_err = smem_optin<sgn::k_p5_stage<TC, BC, MODE, R>>(smem);
    if (attr_err != cudaSuccess) return attr_err;
    sgn::k_p5_stage<TC, BC, MODE, R><<<grid, dim3(sgn::TILE_X, sgn::THREADS_Y), smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

// The pair's stage kernels take the context's FP64 tile height, as the RK4
// stage kernels do (the FSAL stage writes one error partial per block).
template <typename TC, int BC, int MODE>
cudaError_t launch_p5(const sgn_ctx* c, const sgn::P5Args& a, cudaStream_t s) {
    if constexpr (std::is_same<TC, double>::value) {
        if (c->rows == 1) return launch_p5_rows<TC, BC, MODE, 1>(c->gridr, a, s);
        if (c->rows == 2) return launch_p5_rows<TC, BC, MODE, 2>(c->gridr, a, s);
    }
    return launch_p5_rows<TC, BC, MODE, sgn::StageShape<TC>::rows>(c->grid, a, s);
}


template <typename TC, int BC>
sgn_status run_adaptive_p5(sgn_ctx* c, double* q_user, double t0, double t_end, double dt0, double rtol,
                           double atol, int max_attempts, double* hist, double* stats, cudaStream_t s) {
    const long long P5 = 5 * c->G.plane;
    const size_t bytes5 = (size_t)P5 * sizeof(double);
    static_assert(sizeof(TC) == sizeof(double), "the slots below hold 8-byte values");
    TC* k1 = reinterpret_cast<TC*>(c->bs);
    TC* k6 = reinterpret_cast<TC*>(c->bs + P5);
    TC* Ya = reinterpret_cast<TC*>(c->bs + 2 * P5);
    TC* Yb = reinterpret_cast<TC*>(c->bs + 3 * P5);
    TC* U = reinterpret_cast<TC*>(c->bs + 4 * P5);
    TC* E = reinterpret_cast<TC*>(c->bs + 5 * P5);
    double* q1 = c->bs + 6 * P5;
    double* qc = c->bs + 7 * P5;
    CUDA_TRY(cudaMemcpyAsync(qc, q_user, bytes5, cudaMemcpyDeviceToDevice, s), "copy q");
    {
        // k1 = f(q), stored in the compute type
        StageArgs<TC, double, TC> r = base_args<TC, double, TC>(c);
        r.X = qc;
        r.out = k1;
        CUDA_TRY((launch_stage<TC, double, TC, BC, sgn::MODE_RHS>(c, r, s)), "k1");
    }
    sgn_status st = read_flag(c, s);
    if (st != SGN_OK) return st;

    sgn::P5Args a;
    std::memset(&a, 0, sizeof(a));
    a.b = c->bT;
    a.flag = c->flag;
    a.G = c->G;
    a.rtol = rtol;
    a.atol = atol;
    a.partials = c->partials;
    a.U = U;
    a.E = E;
    a.q1 = q1;
    double t = t0, dt = dt0, eps_prev = 1.0;
    int acc = 0, rej = 0, n = 0;
    while (t < t_end && n < max_attempts) {
        const bool last = dt >= t_end - t;
        const double h = last ? t_end - t : dt;
        a.q = qc;
        a.k1 = k1;
        // stage 2: Y2 = q + h a21 k1; writes Y3, U3, E3
        a.c_in = h * P5_A21;
        a.c_u1 = h * P5_B[0];
        a.c_e1 = P5_B[0] - P5_BHAT[0];
        a.c_y = h * P5_A32;
        a.c_u = h * P5_B[1];
        a.c_e = P5_B[1] - P5_BHAT[1];
        a.Yout = Ya;
        CUDA_TRY((launch_p5<TC, BC, sgn::P5_S2>(c, a, s)), "pair stage 2");
        // stage 3: Y3 -> Y4, U4, E4
        a.Yin = Ya;
        a.Yout = Yb;
        a.c_y = h * P5_A43;
        a.c_u = h * P5_B[2];
        a.c_e = P5_B[2] - P5_BHAT[2];
        CUDA_TRY((launch_p5<TC, BC, sgn::P5_MID>(c, a, s)), "pair stage 3");
        // stage 4: Y4 -> Y5, U5, E5
        a.Yin = Yb;
        a.Yout = Ya;
        a.c_y = h * P5_A54;
        a.c_u = h * P5_B[3];
        a.c_e = P5_B[3] - P5_BHAT[3];
        CUDA_TRY((launch_p5<TC, BC, sgn::P5_MID>(c, a, s)), "pair stage 4");
        // stage 5: Y5 -> q1 = U5 + h b5 k5, E6
        a.Yin = Ya;
        a.c_u = h * P5_B[4];
        a.c_e = P5_B[4] - P5_BHAT[4];
        CUDA_TRY((launch_p5<TC, BC, sgn::P5_S5>(c, a, s)), "pair stage 5");
        // k6 = f(q1) and the error partial sums
        a.kout = k6;
        a.c_e6 = 0.0 - P5_BHAT[5];
        a.dt = h;
        CUDA_TRY((launch_p5<TC, BC, sgn::P5_FSAL>(c, a, s)), "pair FSAL stage");
        sgn::k_reduce_partials<<<1, 256, 0, s>>>(c->partials, pair_blocks<TC>(c), c->dout);
        count_launch();
        CUDA_TRY(cudaGetLastError(), "error reduction");
        CUDA_TRY(cudaMemcpyAsync(c->hout, c->dout, sizeof(double), cudaMemcpyDeviceToHost, s), "copy error");
        CUDA_TRY(cudaMemcpyAsync(c->hflag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, s), "copy flag");
        CUDA_TRY(cudaStreamSynchronize(s), "synchronize");
        double err;
        if (*c->hflag) {
            // a trial stage left the admissible states: reject as an infinite error
            CUDA_TRY(cudaMemsetAsync(c->flag, 0, sizeof(int), s), "clear flag");
            err = INFINITY;
        } else {
            err = std::sqrt(c->hout[0] / (double)P5);
        }
        const bool ok = err <= 1.0;
        const double eps = P5_SAFETY / std::fmax(err, P5_ERR_FLOOR);
        const double x = ok ? std::pow(eps, P5_PI_B1 / P5_PI_K) * std::pow(eps_prev, P5_PI_B2 / P5_PI_K)
                            : std::pow(eps, 1.0 / P5_PI_K);
        const double fac = 1.0 + std::atan(x - 1.0);
        if (hist) {
            hist[3 * n] = h;
            hist[3 * n + 1] = err;
            hist[3 * n + 2] = ok ? 1.0 : 0.0;
        }
        if (ok) {
            std::swap(qc, q1);
            std::swap(k1, k6);
            a.q1 = q1;
            t = last ? t_end : t + h;
            eps_prev = eps;
            acc++;
        } else {
            rej++;
        }
        dt = h * fac;
        n++;
    }
    CUDA_TRY(cudaMemcpyAsync(q_user, qc, bytes5, cudaMemcpyDeviceToDevice, s), "copy q back");
    CUDA_TRY(cudaStreamSynchronize(s), "synchronize");
    stats[0] = acc;
    stats[1] = rej;
    stats[2] = t;
    stats[3] = dt;
    stats[4] = n;
    return SGN_OK;
}

// ---- manufactured solution (Sec. 6.1.2): forced RK4 stages
sgn::MmsTime mms_time(double t) {
    const double pi = 3.14159265358979323846;
    return {std::sin(2.0 * pi * t), std::cos(2.0 * pi * t)};
}

template <int BC, int MODE, int FORCING>
cudaError_t launch_forced(const sgn_ctx* c, const sgn::MmsArgs& m, cudaStream_t s) {
    auto kern = sgn::k_forced_stage<BC, MODE, FORCING>;
    const size_t smem = sgn::stage_smem_bytes<double, sgn::MODE_RHS>(sgn::StageShape<double>::rows);
    const cudaError_t attr_err = smem_optin<sgn::k_forced_stage<BC, MODE, FORCING>>(smem);
    if (attr_err != cudaSuccess) return attr_err;
    kern<<<c->grid, dim3(sgn::TILE_X, sgn::THREADS_Y), smem, s>>>(m);
    count_launch();
    return cudaGetLastError();
}

template <int BC, int FORCING>
cudaError_t run_forced_steps(sgn_ctx* c, double* q, double t0, double dt, int nsteps, const sgn::MmsArgs& proto,
                             cudaStream_t s) {
    double* acc = static_cast<double*>(c->acc);
    double* Qa = static_cast<double*>(c->Qa);
    double* Qb = static_cast<double*>(c->Qb);
    sgn::MmsArgs m1 = proto, m2 = proto, m3 = proto, m4 = proto;
    m1.st = base_args<double, double, double>(c);
    m1.st.X = q; m1.st.qn = q; m1.st.acc = acc; m1.st.Qout = Qa; m1.st.c_acc = dt / 6.0; m1.st.c_q = dt / 2.0;
    m2.st = base_args<double, double, double>(c);
    m2.st.X = Qa; m2.st.qn = q; m2.st.acc = acc; m2.st.Qout = Qb; m2.st.c_acc = dt / 3.0; m2.st.c_q = dt / 2.0;
    m3.st = m2.st;
    m3.st.X = Qb; m3.st.Qout = Qa; m3.st.c_acc = dt / 3.0; m3.st.c_q = dt;
    m4.st = base_args<double, double, double>(c);
    m4.st.X = Qa; m4.st.acc = acc; m4.st.out = q; m4.st.c_acc = dt / 6.0;
    cudaError_t e;
    for (int n = 0; n < nsteps; n++) {
        const double t = t0 + n * dt;
        m1.T = mms_time(t);
        m2.T = m3.T = mms_time(t + 0.5 * dt);
        m4.T = mms_time(t + dt);
        if ((e = launch_forced<BC, sgn::MODE_S1, FORCING>(c, m1, s)) != cudaSuccess) return e;
        if ((e = launch_forced<BC, sgn::MODE_S2, FORCING>(c, m2, s)) != cudaSuccess) return e;
        if ((e = launch_forced<BC, sgn::MODE_S3, FORCING>(c, m3, s)) != cudaSuccess) return e;
        if ((e = launch_forced<BC, sgn::MODE_S4, FORCING>(c, m4, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

sgn::MmsArgs forced_proto(const sgn_ctx* c) {
    sgn::MmsArgs m;
    std::memset(&m, 0, sizeof(m));
    m.xmin = c->p.xmin;
    m.ymin = c->p.ymin;
    m.xmax = c->p.xmax;
    m.ymax = c->p.ymax;
    return m;
}

// ---- relaxation RK4: gamma from E(q + gamma d) = E(q), host-side Newton
// Newton on F(gamma) = (E(q + gamma d) - E(q)) / gamma from the six sums of
// k_rrk_sums about gamma_c; returns false if it does not converge.
bool rrk_newton(const double* S, double gamma_c, double* gamma) {
    double g = gamma_c;
    for (int it = 0; it < 50; it++) {
        const double tau = g - gamma_c;
        const double F = S[0] + g * (S[1] + g * S[2]) + S[3] + tau * (S[4] + tau * S[5]);
        const double dF = S[1] + 2.0 * g * S[2] + S[4] + 2.0 * tau * S[5];
        if (!(std::isfinite(F) && std::isfinite(dF)) || dF == 0.0) return false;
        const double step = F / dF;
        g -= step;
        if (std::fabs(step) <= 1e-16 * std::fabs(g)) {
            *gamma = g;
            return std::isfinite(g) && g > 0.0;
        }
    }
    *gamma = g;
    return std::isfinite(g) && g > 0.0;
}

template <int BC>
sgn_status run_relaxed(sgn_ctx* c, double* q, double dt, int nsteps, double* gammas, double* t_out,
                       cudaStream_t s) {
    const long long P5 = 5 * c->G.plane;
    double* q1 = c->rrk;
    double* part = c->rrk + P5;
    double* dsum = part + c->rrk_nblk * sgn::NRRK;
    double* acc = static_cast<double*>(c->acc);
    double* Qa = static_cast<double*>(c->Qa);
    double* Qb = static_cast<double*>(c->Qb);
    StageArgs<double, double, double> a1 = base_args<double, double, double>(c);
    a1.X = q; a1.qn = q; a1.acc = acc; a1.Qout = Qa; a1.c_acc = dt / 6.0; a1.c_q = dt / 2.0;
    StageArgs<double, double, double> a2 = base_args<double, double, double>(c);
    a2.X = Qa; a2.qn = q; a2.acc = acc; a2.Qout = Qb; a2.c_acc = dt / 3.0; a2.c_q = dt / 2.0;
    StageArgs<double, double, double> a3 = a2;
    a3.X = Qb; a3.Qout = Qa; a3.c_acc = dt / 3.0; a3.c_q = dt;
    StageArgs<double, double, double> a4 = base_args<double, double, double>(c);
    a4.X = Qa; a4.acc = acc; a4.out = q1; a4.c_acc = dt / 6.0;    // plain RK4 update, kept apart
    double t = 0.0;
    for (int n = 0; n < nsteps; n++) {
        CUDA_TRY((launch_stage<double, double, double, BC, sgn::MODE_S1>(c, a1, s)), "relaxed stage 1");
        CUDA_TRY((launch_stage<double, double, double, BC, sgn::MODE_S2>(c, a2, s)), "relaxed stage 2");
        CUDA_TRY((launch_stage<double, double, double, BC, sgn::MODE_S3>(c, a3, s)), "relaxed stage 3");
        CUDA_TRY((launch_stage<double, double, double, BC, sgn::MODE_S4>(c, a4, s)), "relaxed stage 4");
        double gamma_c = 1.0, gamma = 1.0;
        bool done = false;
        for (int pass = 0; pass < 8 && !done; pass++) {
            sgn::k_rrk_sums<BC><<<sgn::RRK_GRID, sgn::RRK_BLOCK, 0, s>>>(q, q1, c->b64, c->G, gamma_c, part);
            count_launch();
            sgn::k_rrk_reduce<<<1, 256, 0, s>>>(part, c->rrk_nblk, dsum);
            count_launch();
            CUDA_TRY(cudaGetLastError(), "relaxation sums");
            CUDA_TRY(cudaMemcpyAsync(c->hout, dsum, sgn::NRRK * sizeof(double), cudaMemcpyDeviceToHost, s),
                     "copy relaxation sums");
            sgn_status st = read_flag(c, s);     // synchronizes
            if (st != SGN_OK) return st;
            if (!rrk_newton(c->hout, gamma_c, &gamma))
                return fail(SGN_E_NONFINITE, "relaxation: no energy-conserving gamma near 1 (step %d)", n);
            done = std::fabs(gamma - gamma_c) <= 1e-3;
            gamma_c = gamma;
        }
        if (!done) return fail(SGN_E_NONFINITE, "relaxation: gamma did not settle (step %d)", n);
        sgn::k_rrk_update<<<592, 256, 0, s>>>(q, q1, gamma, P5);
        count_launch();
        CUDA_TRY(cudaGetLastError(), "relaxed update");
        if (gammas) gammas[n] = gamma;
        t += gamma * dt;
    }
    CUDA_TRY(cudaStreamSynchronize(s), "synchronize");
    if (t_out) *t_out = t;
    return SGN_OK;
}

// nsteps recorded RK4 steps (stash: 20 planes per step; tape: 4 N_TAPE planes
// per step, or NULL for none).
sgn_status record_steps(sgn_ctx* c, void* q_dev, double dt, int nsteps, void* stash_dev, void* tape_dev,
                        void* stream, const char* what) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    sgn_status st = need_f64(c, what);
    if (st == SGN_OK) st = check_state_ptr(q_dev, "q_dev");
    if (st == SGN_OK && nsteps > 0) st = check_state_ptr(stash_dev, "stash_dev");
    if (st == SGN_OK && nsteps > 0 && tape_dev) st = check_state_ptr(tape_dev, "tape_dev");
    if (st != SGN_OK) return st;
    if (!finite_pos(dt)) return fail(SGN_E_INVAL, "dt must be finite and > 0");
    if (nsteps < 0) return fail(SGN_E_INVAL, "nsteps must be >= 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* q = static_cast<double*>(q_dev);
    double* stash = static_cast<double*>(stash_dev);
    double* tape = static_cast<double*>(tape_dev);
    const long long P20 = 20 * c->G.plane;
    const long long PT = 4LL * sgn::N_TAPE * c->G.plane;
    const bool refl = c->p.bc == SGN_BC_REFLECTING;
    for (int n = 0; n < nsteps; n++) {
        double* sn = stash + n * P20;
        cudaError_t e;
        if (tape)
            e = refl ? record_step<sgn::BC_REFLECTING, true>(c, q, dt, sn, tape + n * PT, s)
                     : record_step<sgn::BC_PERIODIC, true>(c, q, dt, sn, tape + n * PT, s);
        else
            e = refl ? record_step<sgn::BC_REFLECTING, false>(c, q, dt, sn, nullptr, s)
                     : record_step<sgn::BC_PERIODIC, false>(c, q, dt, sn, nullptr, s);
        if (e != cudaSuccess) return cuda_fail(e, what);
    }
    return SGN_OK;
}

// The VJP of one recorded RK4 step (tape: the step's four tapes, or NULL to
// compute each stage's tape from its recorded state).
sgn_status step_vjp(sgn_ctx* c, const void* stash_dev, const void* tape_dev, void* qbar_dev, void* bbar_dev,
                    double dt, void* stream, const char* what) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    sgn_status st = need_f64(c, what);
    if (st == SGN_OK) st = check_state_ptr(stash_dev, "stash_dev");
    if (st == SGN_OK && tape_dev) st = check_state_ptr(tape_dev, "tape_dev");
    if (st == SGN_OK) st = check_state_ptr(qbar_dev, "qbar_dev");
    if (st == SGN_OK) st = check_state_ptr(bbar_dev, "bbar_dev");
    if (st != SGN_OK) return st;
    if (!finite_pos(dt)) return fail(SGN_E_INVAL, "dt must be finite and > 0");
    const long long P5 = 5 * c->G.plane;
    const long long PT = (long long)sgn::N_TAPE * c->G.plane;
    st = adjoint_scratch(c);
    if (st != SGN_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double* stash = static_cast<const double*>(stash_dev);
    const double* tape = static_cast<const double*>(tape_dev);
    double* qbar = static_cast<double*>(qbar_dev);
    double* qacc = c->adj;
    // The cotangent of stage s is sigma_s * A_s: sigma_4 = dt/6, A_4 = qbar', and
    // k_{s-1} = c' qbar' + cbar Qbar_s gives sigma_{s-1} = cbar sigma_s and
    // A_{s-1} = (c' / sigma_{s-1}) qbar' + J^T A_s (one FMA per value).
    const double sig4 = dt / 6.0, sig3 = dt * sig4, sig2 = 0.5 * dt * sig3, sig1 = 0.5 * dt * sig2;
    const double kap3 = (dt / 3.0) / sig3, kap2 = (dt / 3.0) / sig2, kap1 = (dt / 6.0) / sig1;
    if (!(std::isnormal(sig1) && std::isfinite(kap1)))
        return fail(SGN_E_INVAL, "dt = %g is outside the range of the scaled adjoint recurrence", dt);
    auto tape_of = [&](int stage) { return tape ? tape + (stage - 1) * PT : nullptr; };
    sgn::AdjArgs a;
    std::memset(&a, 0, sizeof(a));
    a.b = c->b64;
    a.scratch = c->adj + kAdjScratchA * c->G.plane;
    a.bbar = static_cast<double*>(bbar_dev);
    a.qprime = qbar;
    a.flag = c->flag;
    a.G = c->G;
    // The chained walk (see chained_walk).  Without recorded tapes each
    // stage's tape is computed from its recorded state just before the launch
    // that first reads it, into two scratch tapes used alternately (stages 4
    // and 2 in one, 3 and 1 in the other).
    double* tA = c->adj + kAdjTapeOffset * c->G.plane;
    double* tB = c->adj + (kAdjTapeOffset + sgn::N_TAPE) * c->G.plane;
    sgn::AdjArgs g[4];
    for (int k = 0; k < 4; k++) {
        g[k] = a;
        g[k].X = stash + k * P5;
        g[k].tape = tape ? tape_of(k + 1) : ((k % 2 == 1) ? tA : tB);
        g[k].scratch = c->adj + ((k % 2 == 1) ? kAdjScratchA : kAdjScratchB) * c->G.plane;
        g[k].Anext = nullptr;
    }
    // stage 4: k4bar = dt/6 qbar'; Q4bar = J(Q4)^T k4bar; k3bar = dt/3 qbar' + dt Q4bar
    g[3].A = qbar; g[3].sigma = sig4; g[3].first = 1; g[3].qacc_out = qacc; g[3].kappa = kap3;
    // stage 3: Q3bar = J(Q3)^T k3bar; k2bar = dt/3 qbar' + dt/2 Q3bar
    g[2].sigma = sig3; g[2].first = 0; g[2].qacc_in = qacc; g[2].qacc_out = qacc; g[2].kappa = kap2;
    // stage 2: Q2bar = J(Q2)^T k2bar; k1bar = dt/6 qbar' + dt/2 Q2bar
    g[1].sigma = sig2; g[1].first = 0; g[1].qacc_in = qacc; g[1].qacc_out = qacc; g[1].kappa = kap1;
    // stage 1: Q1bar = J(q_n)^T k1bar; qbar = qbar' + Q1bar + Q2bar + Q3bar + Q4bar
    g[0].sigma = sig1; g[0].first = 0; g[0].qacc_in = qacc; g[0].qacc_out = qbar;
    const cudaError_t e = c->p.bc == SGN_BC_REFLECTING ? chained_walk<sgn::BC_REFLECTING>(c, g, !tape, s)
                                                       : chained_walk<sgn::BC_PERIODIC>(c, g, !tape, s);
    if (e != cudaSuccess) return cuda_fail(e, what);
    return SGN_OK;
}

}  // namespace

extern "C" {

const char* sgn_status_str(sgn_status s) {
    switch (s) {
    case SGN_OK: return "SGN_OK";
    case SGN_E_INVAL: return "SGN_E_INVAL";
    case SGN_E_NOMEM: return "SGN_E_NOMEM";
    case SGN_E_CUDA: return "SGN_E_CUDA";
    case SGN_E_NONPOSITIVE_H: return "SGN_E_NONPOSITIVE_H";
    case SGN_E_NONFINITE: return "SGN_E_NONFINITE";
    case SGN_E_TIMEOUT: return "SGN_E_TIMEOUT";
    case SGN_E_UNSUPPORTED: return "SGN_E_UNSUPPORTED";
    }
    return "SGN_E_UNKNOWN";
}

const char* sgn_last_error(void) { return g_err; }

unsigned long long sgn_launch_count(void) { return g_launches.load(); }

sgn_status sgn_create(const sgn_params* p, const void* b_dev, sgn_ctx** out) {
    if (!out) return fail(SGN_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!p) return fail(SGN_E_INVAL, "params is NULL");
    if (p->nx < 3 || p->ny < 3) return fail(SGN_E_INVAL, "grid %dx%d: need nx, ny >= 3", p->nx, p->ny);
    // tile height of the stage kernels for this compute type (StageShape)
    const int tile_y = sgn::THREADS_Y * (p->prec == SGN_DF64  ? sgn::StageShape<sgn::df64>::rows
                                         : p->prec == SGN_F64 ? sgn::StageShape<double>::rows
                                                              : sgn::StageShape<float>::rows);
    // every launch over the grid fits the launch grid's y limit of 65535 blocks
    // (the 32 x 8 launches, init_aux among them, are the tallest grids)
    if ((p->ny + sgn::THREADS_Y - 1) / sgn::THREADS_Y > 65535 || (p->ny + tile_y - 1) / tile_y > 65535)
        return fail(SGN_E_INVAL, "ny = %d exceeds the launch-grid limit (ny <= %d)", p->ny, 65535 * sgn::THREADS_Y);
    // the float-based kernels address a plane with 32-bit offsets
    if (p->prec != SGN_F64 && (long long)p->nx * p->ny > 0xffffffffLL)
        return fail(SGN_E_INVAL, "grids of 2^32 or more nodes need SGN_F64 (%d x %d)", p->nx, p->ny);
    if (!(std::isfinite(p->xmin) && std::isfinite(p->xmax) && p->xmax > p->xmin &&
          std::isfinite(p->ymin) && std::isfinite(p->ymax) && p->ymax > p->ymin))
        return fail(SGN_E_INVAL, "domain must be finite with xmax > xmin and ymax > ymin");
    if (p->bc != SGN_BC_PERIODIC && p->bc != SGN_BC_REFLECTING) return fail(SGN_E_INVAL, "bc = %d", p->bc);
    if (p->prec != SGN_F64 && p->prec != SGN_F32 && p->prec != SGN_F32_F64ACC && p->prec != SGN_DF64)
        return fail(SGN_E_INVAL, "prec = %d", p->prec);
    if (!finite_pos(p->g)) return fail(SGN_E_INVAL, "g must be finite and > 0");
    if (!(std::isfinite(p->lambda) && p->lambda >= 0.0)) return fail(SGN_E_INVAL, "lambda must be finite and >= 0");
    if (!b_dev) return fail(SGN_E_INVAL, "b_dev is NULL");
    if (!is_device_ptr(b_dev)) return fail(SGN_E_INVAL, "b_dev is not device memory");

    sgn_ctx* c = new (std::nothrow) sgn_ctx();
    if (!c) return fail(SGN_E_NOMEM, "host allocation");
    c->p = *p;
    const bool per = p->bc == SGN_BC_PERIODIC;
    const double dx = per ? (p->xmax - p->xmin) / p->nx : (p->xmax - p->xmin) / (p->nx - 1);
    const double dy = per ? (p->ymax - p->ymin) / p->ny : (p->ymax - p->ymin) / (p->ny - 1);
    Geom& G = c->G;
    sgn::fill_geom(G, p->nx, p->ny, dx, dy, p->g, p->lambda);
    c->tc_size = (p->prec == SGN_F64 || p->prec == SGN_DF64) ? 8 : sizeof(float);
    c->ta_size = p->prec == SGN_F32 ? sizeof(float) : sizeof(double);
    c->grid = dim3((p->nx + sgn::TILE_X - 1) / sgn::TILE_X, (p->ny + tile_y - 1) / tile_y);
    c->nblk = (long long)c->grid.x * c->grid.y;
    c->nband = (long long)c->grid.x * ((p->ny + sgn::THREADS_Y - 1) / sgn::THREADS_Y);   // >= nblk
    c->rows = tile_y / sgn::THREADS_Y;
    c->gridr = c->grid;
    c->fuse = p->prec == SGN_F32;
    if (p->prec == SGN_F64) {
        // The FP64 stage kernels are bound by each SM's FP64 pipe, so a launch
        // takes as long as its most loaded SM: ceil(b/S) blocks of b over S
        // SMs.  A 32 x 8R tile costs 256 R nodes x 68.75 FP64 operations (RHS
        // and stage algebra) plus 34 (8R + 2) halo nodes x 15 (operands).  The
        // height with the least work on the most loaded SM is taken (a lower
        // one only where it saves more than 2%).
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0) {
            auto cost = [&](int R) {
                const double blocks = (double)c->grid.x * (double)((p->ny + 8 * R - 1) / (8 * R));
                return std::ceil(blocks / sms) * (256.0 * R * 68.75 + 34.0 * (8 * R + 2) * 15.0);
            };
            double best = cost(c->rows);
            for (int R = c->rows - 1; R >= 1; R--) {
                const long long gy = (p->ny + 8 * R - 1) / (8 * R);
                const double cr = cost(R);
                if (gy <= 65535 && cr < 0.98 * best) {
                    best = cr;
                    c->rows = R;
                }
            }
            c->gridr = dim3(c->grid.x, (unsigned)((p->ny + 8 * c->rows - 1) / (8 * c->rows)));
        } else {
            cudaGetLastError();
        }
    }

    const size_t plane = (size_t)G.plane;
    bool ok = cudaMalloc(&c->b64, plane * sizeof(double)) == cudaSuccess;
    if (ok && p->prec != SGN_F64) ok = cudaMalloc(&c->bT, plane * c->tc_size) == cudaSuccess;
    if (ok && p->prec == SGN_F64) c->bT = c->b64;
    ok = ok && cudaMalloc(&c->acc, 5 * plane * c->ta_size) == cudaSuccess;
    ok = ok && cudaMalloc(&c->Qa, 5 * plane * c->tc_size) == cudaSuccess;
    ok = ok && cudaMalloc(&c->Qb, 5 * plane * c->tc_size) == cudaSuccess;
    ok = ok && cudaMalloc(&c->partials, (size_t)c->nband * sgn::NDIAG * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc(&c->dout, sgn::NDIAG * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc(&c->flag, sizeof(int)) == cudaSuccess;
    ok = ok && cudaMallocHost(&c->hout, kHostOut * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMallocHost(&c->hflag, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        const size_t need = 5 * plane * (c->ta_size + 2 * c->tc_size);
        free_ctx(c);
        return fail(SGN_E_NOMEM, "allocating about %zu bytes of scratch", need);
    }
    cudaError_t e = cudaMemset(c->flag, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(c->b64, b_dev, plane * sizeof(double), cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess && p->prec != SGN_F64) e = convert_bathymetry(c, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        sgn_status st = cuda_fail(e, "sgn_create");
        free_ctx(c);
        return st;
    }
    *out = c;
    return SGN_OK;
}

sgn_status sgn_destroy(sgn_ctx* c) {
    if (!c) return SGN_OK;
    cudaError_t e = cudaDeviceSynchronize();
    free_ctx(c);
    if (e != cudaSuccess) return cuda_fail(e, "sgn_destroy");
    return SGN_OK;
}

sgn_status sgn_set_bathymetry(sgn_ctx* c, const void* b_dev, void* stream) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    if (!b_dev || !is_device_ptr(b_dev)) return fail(SGN_E_INVAL, "b_dev is not device memory");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t plane = (size_t)c->G.plane;
    CUDA_TRY(cudaMemcpyAsync(c->b64, b_dev, plane * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy b");
    if (c->p.prec != SGN_F64) CUDA_TRY(convert_bathymetry(c, s), "convert b");
    return SGN_OK;
}

sgn_status sgn_init_aux(sgn_ctx* c, void* q_dev, void* stream) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    sgn_status st = check_state_ptr(q_dev, "q_dev");
    if (st != SGN_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const bool refl = c->p.bc == SGN_BC_REFLECTING;
    if (c->p.prec == SGN_F32)
        e = refl ? run_init<float, sgn::BC_REFLECTING>(c, static_cast<float*>(q_dev), s)
                 : run_init<float, sgn::BC_PERIODIC>(c, static_cast<float*>(q_dev), s);
    else
        e = refl ? run_init<double, sgn::BC_REFLECTING>(c, static_cast<double*>(q_dev), s)
                 : run_init<double, sgn::BC_PERIODIC>(c, static_cast<double*>(q_dev), s);
    if (e != cudaSuccess) return cuda_fail(e, "sgn_init_aux");
    return SGN_OK;
}

sgn_status sgn_rhs(sgn_ctx* c, const void* q_dev, void* dq_dev, void* stream) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    sgn_status st = check_state_ptr(q_dev, "q_dev");
    if (st == SGN_OK) st = check_state_ptr(dq_dev, "dq_dev");
    if (st != SGN_OK) return st;
    if (q_dev == dq_dev) return fail(SGN_E_INVAL, "q_dev and dq_dev must not overlap");
    RhsOp f{c, q_dev, dq_dev, static_cast<cudaStream_t>(stream)};
    cudaError_t e = dispatch(c, f);
    if (e != cudaSuccess) return cuda_fail(e, "sgn_rhs");
    return SGN_OK;
}

sgn_status sgn_step(sgn_ctx* c, void* q_dev, double dt, int nsteps, void* stream) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    sgn_status st = check_state_ptr(q_dev, "q_dev");
    if (st != SGN_OK) return st;
    if (!finite_pos(dt)) return fail(SGN_E_INVAL, "dt must be finite and > 0");
    if (nsteps < 0) return fail(SGN_E_INVAL, "nsteps must be >= 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int left = nsteps;
    if (left >= kGraphSteps && c->G.plane <= kGraphMaxCells) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CUDA_TRY(cudaStreamIsCapturing(s, &cs), "capture status");
        if (cs == cudaStreamCaptureStatusNone) {
            st = step_graph(c, q_dev, dt);
            if (st != SGN_OK) return st;
            while (left >= kGraphSteps) {
                CUDA_TRY(cudaGraphLaunch(c->step_exec, s), "graph launch");
                g_launches.fetch_add((c->fuse ? 2ull : 4ull) * kGraphSteps, std::memory_order_relaxed);
                left -= kGraphSteps;
            }
        }
    }
    StepOp f{c, q_dev, dt, left, s};
    cudaError_t e = dispatch(c, f);
    if (e != cudaSuccess) return cuda_fail(e, "sgn_step");
    return SGN_OK;
}

sgn_status sgn_step_diag(sgn_ctx* c, void* q_dev, double dt, int nsteps, double* out, void* stream) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    if (!out && nsteps > 0) return fail(SGN_E_INVAL, "out is NULL");
    sgn_status st = check_state_ptr(q_dev, "q_dev");
    if (st != SGN_OK) return st;
    if (!finite_pos(dt)) return fail(SGN_E_INVAL, "dt must be finite and > 0");
    if (nsteps < 0) return fail(SGN_E_INVAL, "nsteps must be >= 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (nsteps > c->mon_cap) {
        CUDA_TRY(cudaStreamSynchronize(s), "synchronize");
        cudaFree(c->mon);
        c->mon = nullptr;
        c->mon_cap = 0;
        if (cudaMalloc(&c->mon, (size_t)nsteps * sgn::NDIAG * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            c->mon = nullptr;
            return fail(SGN_E_NOMEM, "monitor buffer for %d steps", nsteps);
        }
        c->mon_cap = nsteps;
    }
    StepDiagOp f{c, q_dev, dt, nsteps, c->mon, s};
    cudaError_t e = dispatch(c, f);
    if (e != cudaSuccess) return cuda_fail(e, "sgn_step_diag");
    if (nsteps == 0) return read_flag(c, s);
    std::vector<double> tmp((size_t)nsteps * sgn::NDIAG);
    CUDA_TRY(cudaMemcpyAsync(tmp.data(), c->mon, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost, s),
             "copy monitor");
    st = read_flag(c, s);
    for (int n = 0; n < nsteps; n++)
        for (int k = 0; k < 3; k++) out[3 * n + k] = tmp[(size_t)n * sgn::NDIAG + k];
    return st;
}

sgn_status sgn_step_host(sgn_ctx* c, void* q_host, double dt, int nsteps, double* out, void* stream) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    if (!q_host) return fail(SGN_E_INVAL, "q_host is NULL");
    if (is_device_ptr(q_host)) return fail(SGN_E_INVAL, "q_host is device memory (sgn_step takes device states)");
    if (!finite_pos(dt)) return fail(SGN_E_INVAL, "dt must be finite and > 0");
    if (nsteps < 0) return fail(SGN_E_INVAL, "nsteps must be >= 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)5 * (size_t)c->G.plane * c->ta_size;
    if (!c->hq) {
        if (cudaMalloc(&c->hq, bytes) != cudaSuccess) {
            cudaGetLastError();
            c->hq = nullptr;
            return fail(SGN_E_NOMEM, "device state of %zu bytes", bytes);
        }
    }
    CUDA_TRY(cudaMemcpyAsync(c->hq, q_host, bytes, cudaMemcpyHostToDevice, s), "copy the state in");
    sgn_status st = out ? sgn_step_diag(c, c->hq, dt, nsteps, out, stream) : sgn_step(c, c->hq, dt, nsteps, stream);
    if (st != SGN_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(q_host, c->hq, bytes, cudaMemcpyDeviceToHost, s), "copy the state out");
    return read_flag(c, s);
}

sgn_status sgn_mass_energy(sgn_ctx* c, const void* q_dev, double* out, void* stream) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    if (!out) return fail(SGN_E_INVAL, "out is NULL");
    sgn_status st = check_state_ptr(q_dev, "q_dev");
    if (st != SGN_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DiagOp f{c, q_dev, s};
    cudaError_t e = dispatch(c, f);
    if (e != cudaSuccess) return cuda_fail(e, "sgn_mass_energy");
    CUDA_TRY(cudaMemcpyAsync(c->hout, c->dout, sgn::NDIAG * sizeof(double), cudaMemcpyDeviceToHost, s),
             "copy diagnostics");
    st = read_flag(c, s);
    for (int k = 0; k < sgn::NDIAG; k++) out[k] = c->hout[k];
    return st;
}

sgn_status sgn_check(sgn_ctx* c, void* stream) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    return read_flag(c, static_cast<cudaStream_t>(stream));
}

sgn_status sgn_set_tile_rows(sgn_ctx* c, int rows) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    if (c->p.prec != SGN_F64) return fail(SGN_E_UNSUPPORTED, "the tile height is chosen for SGN_F64 contexts only");
    if (rows < 1 || rows > 3) return fail(SGN_E_INVAL, "rows = %d: need 1, 2 or 3", rows);
    const long long gy = (c->p.ny + 8LL * rows - 1) / (8LL * rows);
    if (gy > 65535) return fail(SGN_E_INVAL, "ny = %d exceeds the launch-grid limit at rows = %d", c->p.ny, rows);
    if (rows != c->rows && c->step_exec) {
        // the replayed graph holds the launches of the old tile height
        cudaGraphExecDestroy(c->step_exec);
        c->step_exec = nullptr;
    }
    c->rows = rows;
    c->gridr = dim3(c->grid.x, (unsigned)gy);
    return SGN_OK;
}

sgn_status sgn_set_stage_fusion(sgn_ctx* c, int on) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    if (on != 0 && on != 1) return fail(SGN_E_INVAL, "on must be 0 or 1");
    if (c->p.prec != SGN_F32) return fail(SGN_E_UNSUPPORTED, "stage fusion serves SGN_F32 contexts");
    if (on != c->fuse && c->step_exec) {
        // the replayed graph holds the other kernels
        cudaGraphExecDestroy(c->step_exec);
        c->step_exec = nullptr;
    }
    c->fuse = on;
    return SGN_OK;
}

sgn_status sgn_tile_rows(const sgn_ctx* c, int* rows) {
    if (!c || !rows) return fail(SGN_E_INVAL, "ctx and rows must not be NULL");
    *rows = c->rows;
    return SGN_OK;
}

sgn_status sgn_rhs_vjp(sgn_ctx* c, const void* q_dev, const void* abar_dev, void* qbar_dev,
                       void* bbar_dev, void* stream) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    sgn_status st = need_f64(c, "sgn_rhs_vjp");
    if (st == SGN_OK) st = check_state_ptr(q_dev, "q_dev");
    if (st == SGN_OK) st = check_state_ptr(abar_dev, "abar_dev");
    if (st == SGN_OK) st = check_state_ptr(qbar_dev, "qbar_dev");
    if (st == SGN_OK) st = check_state_ptr(bbar_dev, "bbar_dev");
    if (st != SGN_OK) return st;
    if (qbar_dev == q_dev || qbar_dev == abar_dev) return fail(SGN_E_INVAL, "qbar_dev must not overlap the inputs");
    st = adjoint_scratch(c);
    if (st != SGN_OK) return st;
    sgn::AdjArgs a;
    std::memset(&a, 0, sizeof(a));
    a.scratch = c->adj + kAdjScratchA * c->G.plane;
    a.X = static_cast<const double*>(q_dev);
    a.b = c->b64;
    a.A = static_cast<const double*>(abar_dev);
    a.sigma = 1.0;
    a.qbar = static_cast<double*>(qbar_dev);
    a.bbar = static_cast<double*>(bbar_dev);
    a.flag = c->flag;
    a.G = c->G;
    cudaError_t e = adjoint<sgn::ADJ_MODE_RHS>(c, a, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "sgn_rhs_vjp");
    return SGN_OK;
}

sgn_status sgn_step_record(sgn_ctx* c, void* q_dev, double dt, int nsteps, void* stash_dev, void* stream) {
    return record_steps(c, q_dev, dt, nsteps, stash_dev, nullptr, stream, "sgn_step_record");
}

sgn_status sgn_step_record_tape(sgn_ctx* c, void* q_dev, double dt, int nsteps, void* stash_dev,
                                void* tape_dev, void* stream) {
    if (nsteps > 0 && !tape_dev) return fail(SGN_E_INVAL, "tape_dev is NULL");
    return record_steps(c, q_dev, dt, nsteps, stash_dev, tape_dev, stream, "sgn_step_record_tape");
}

sgn_status sgn_step_vjp(sgn_ctx* c, const void* stash_dev, void* qbar_dev, void* bbar_dev, double dt,
                        void* stream) {
    return step_vjp(c, stash_dev, nullptr, qbar_dev, bbar_dev, dt, stream, "sgn_step_vjp");
}

sgn_status sgn_step_vjp_tape(sgn_ctx* c, const void* stash_dev, const void* tape_dev, void* qbar_dev,
                             void* bbar_dev, double dt, void* stream) {
    if (!tape_dev) return fail(SGN_E_INVAL, "tape_dev is NULL");
    return step_vjp(c, stash_dev, tape_dev, qbar_dev, bbar_dev, dt, stream, "sgn_step_vjp_tape");
}

sgn_status sgn_mms_exact(sgn_ctx* c, double t, void* q_dev, void* b_dev, void* stream) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    sgn_status st = check_state_ptr(q_dev, "q_dev");
    if (st == SGN_OK && b_dev) st = check_state_ptr(b_dev, "b_dev");
    if (st != SGN_OK) return st;
    if (!std::isfinite(t)) return fail(SGN_E_INVAL, "t must be finite");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    dim3 blk(32, 8), grd((c->p.nx + 31) / 32, (c->p.ny + 7) / 8);
    sgn::k_mms_exact<<<grd, blk, 0, s>>>(static_cast<double*>(q_dev), static_cast<double*>(b_dev), c->G, c->p.xmin,
                                         c->p.ymin, mms_time(t));
    count_launch();
    CUDA_TRY(cudaGetLastError(), "sgn_mms_exact");
    return SGN_OK;
}

sgn_status sgn_mms_source(sgn_ctx* c, double t, void* s_dev, void* stream) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    sgn_status st = check_state_ptr(s_dev, "s_dev");
    if (st != SGN_OK) return st;
    if (!std::isfinite(t)) return fail(SGN_E_INVAL, "t must be finite");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    dim3 blk(32, 8), grd((c->p.nx + 31) / 32, (c->p.ny + 7) / 8);
    sgn::k_mms_source<<<grd, blk, 0, s>>>(static_cast<double*>(s_dev), c->G, c->p.xmin, c->p.ymin, mms_time(t));
    count_launch();
    CUDA_TRY(cudaGetLastError(), "sgn_mms_source");
    return SGN_OK;
}

sgn_status sgn_step_mms(sgn_ctx* c, void* q_dev, double t0, double dt, int nsteps, void* stream) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    if (c->p.prec != SGN_F64) return fail(SGN_E_UNSUPPORTED, "sgn_step_mms needs an SGN_F64 context");
    sgn_status st = check_state_ptr(q_dev, "q_dev");
    if (st != SGN_OK) return st;
    if (!std::isfinite(t0)) return fail(SGN_E_INVAL, "t0 must be finite");
    if (!finite_pos(dt)) return fail(SGN_E_INVAL, "dt must be finite and > 0");
    if (nsteps < 0) return fail(SGN_E_INVAL, "nsteps must be >= 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* q = static_cast<double*>(q_dev);
    const sgn::MmsArgs proto = forced_proto(c);
    cudaError_t e =
        c->p.bc == SGN_BC_REFLECTING
            ? run_forced_steps<sgn::BC_REFLECTING, sgn::FORCING_MMS>(c, q, t0, dt, nsteps, proto, s)
            : run_forced_steps<sgn::BC_PERIODIC, sgn::FORCING_MMS>(c, q, t0, dt, nsteps, proto, s);
    if (e != cudaSuccess) return cuda_fail(e, "sgn_step_mms");
    return SGN_OK;
}

sgn_status sgn_step_sponge(sgn_ctx* c, void* q_dev, double dt, int nsteps, const void* q0_dev, double width_x,
                           double width_y, double sigma_max, void* stream) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    if (c->p.prec != SGN_F64) return fail(SGN_E_UNSUPPORTED, "sgn_step_sponge needs an SGN_F64 context");
    sgn_status st = check_state_ptr(q_dev, "q_dev");
    if (st == SGN_OK) st = check_state_ptr(q0_dev, "q0_dev");
    if (st != SGN_OK) return st;
    if (q0_dev == q_dev) return fail(SGN_E_INVAL, "q0_dev must not overlap q_dev");
    if (!finite_pos(dt)) return fail(SGN_E_INVAL, "dt must be finite and > 0");
    if (nsteps < 0) return fail(SGN_E_INVAL, "nsteps must be >= 0");
    if (!(std::isfinite(width_x) && width_x >= 0.0 && std::isfinite(width_y) && width_y >= 0.0))
        return fail(SGN_E_INVAL, "zone widths must be finite and >= 0");
    if (!(std::isfinite(sigma_max) && sigma_max >= 0.0)) return fail(SGN_E_INVAL, "sigma_max must be finite and >= 0");
    sgn::MmsArgs proto = forced_proto(c);
    proto.q0 = static_cast<const double*>(q0_dev);
    proto.wx = width_x;
    proto.wy = width_y;
    proto.smax = sigma_max;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* q = static_cast<double*>(q_dev);
    cudaError_t e =
        c->p.bc == SGN_BC_REFLECTING
            ? run_forced_steps<sgn::BC_REFLECTING, sgn::FORCING_SPONGE>(c, q, 0.0, dt, nsteps, proto, s)
            : run_forced_steps<sgn::BC_PERIODIC, sgn::FORCING_SPONGE>(c, q, 0.0, dt, nsteps, proto, s);
    if (e != cudaSuccess) return cuda_fail(e, "sgn_step_sponge");
    return SGN_OK;
}

sgn_status sgn_step_relaxed(sgn_ctx* c, void* q_dev, double dt, int nsteps, double* gammas, double* t_out,
                            void* stream) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    if (c->p.prec != SGN_F64) return fail(SGN_E_UNSUPPORTED, "sgn_step_relaxed needs an SGN_F64 context");
    sgn_status st = check_state_ptr(q_dev, "q_dev");
    if (st != SGN_OK) return st;
    if (!finite_pos(dt)) return fail(SGN_E_INVAL, "dt must be finite and > 0");
    if (nsteps < 0) return fail(SGN_E_INVAL, "nsteps must be >= 0");
    if (!c->rrk) {
        const long long nblk = sgn::RRK_GRID;
        const size_t bytes = ((size_t)5 * (size_t)c->G.plane + (size_t)(nblk + 1) * sgn::NRRK) * sizeof(double);
        if (cudaMalloc(&c->rrk, bytes) != cudaSuccess) {
            cudaGetLastError();
            c->rrk = nullptr;
            return fail(SGN_E_NOMEM, "relaxation scratch (%zu bytes)", bytes);
        }
        c->rrk_nblk = nblk;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* q = static_cast<double*>(q_dev);
    return c->p.bc == SGN_BC_REFLECTING ? run_relaxed<sgn::BC_REFLECTING>(c, q, dt, nsteps, gammas, t_out, s)
                                        : run_relaxed<sgn::BC_PERIODIC>(c, q, dt, nsteps, gammas, t_out, s);
}

sgn_status sgn_step_adaptive(sgn_ctx* c, void* q_dev, double t0, double t_end, double dt0, double rtol,
                             double atol, int max_attempts, int pair, double* hist, double* stats,
                             void* stream) {
    if (!c) return fail(SGN_E_INVAL, "ctx is NULL");
    if (c->p.prec != SGN_F64 && c->p.prec != SGN_DF64)
        return fail(SGN_E_UNSUPPORTED, "sgn_step_adaptive needs an SGN_F64 or SGN_DF64 context");
    sgn_status st = check_state_ptr(q_dev, "q_dev");
    if (st != SGN_OK) return st;
    if (!stats) return fail(SGN_E_INVAL, "stats is NULL");
    if (!(std::isfinite(t0) && std::isfinite(t_end) && t_end >= t0))
        return fail(SGN_E_INVAL, "need finite t0 <= t_end");
    if (!finite_pos(dt0)) return fail(SGN_E_INVAL, "dt0 must be finite and > 0");
    if (!(finite_pos(rtol) || rtol == 0.0) || !(finite_pos(atol) || atol == 0.0) || rtol + atol <= 0.0)
        return fail(SGN_E_INVAL, "rtol, atol must be finite, >= 0 and not both 0");
    if (max_attempts < 0) return fail(SGN_E_INVAL, "max_attempts must be >= 0");
    if (pair != SGN_PAIR_P5S3 && pair != SGN_PAIR_BS3) return fail(SGN_E_INVAL, "pair = %d", pair);
    if (!c->bs) {
        const size_t bytes = (size_t)40 * (size_t)c->G.plane * sizeof(double);
        if (cudaMalloc(&c->bs, bytes) != cudaSuccess) {
            cudaGetLastError();
            c->bs = nullptr;
            return fail(SGN_E_NOMEM, "adaptive integrator scratch (%zu bytes)", bytes);
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* q = static_cast<double*>(q_dev);
    const bool refl = c->p.bc == SGN_BC_REFLECTING;
    if (pair == SGN_PAIR_P5S3) {
        if (c->p.prec == SGN_DF64)
            return refl ? run_adaptive_p5<sgn::df64, sgn::BC_REFLECTING>(c, q, t0, t_end, dt0, rtol, atol,
                                                                        max_attempts, hist, stats, s)
                        : run_adaptive_p5<sgn::df64, sgn::BC_PERIODIC>(c, q, t0, t_end, dt0, rtol, atol,
                                                                      max_attempts, hist, stats, s);
        return refl ? run_adaptive_p5<double, sgn::BC_REFLECTING>(c, q, t0, t_end, dt0, rtol, atol, max_attempts,
                                                                  hist, stats, s)
                    : run_adaptive_p5<double, sgn::BC_PERIODIC>(c, q, t0, t_end, dt0, rtol, atol, max_attempts,
                                                                hist, stats, s);
    }
    if (c->p.prec == SGN_DF64)
        return refl ? run_adaptive<sgn::df64, sgn::BC_REFLECTING>(c, q, t0, t_end, dt0, rtol, atol, max_attempts,
                                                                 hist, stats, s)
                    : run_adaptive<sgn::df64, sgn::BC_PERIODIC>(c, q, t0, t_end, dt0, rtol, atol, max_attempts,
                                                               hist, stats, s);
    return refl ? run_adaptive<double, sgn::BC_REFLECTING>(c, q, t0, t_end, dt0, rtol, atol, max_attempts, hist,
                                                           stats, s)
                : run_adaptive<double, sgn::BC_PERIODIC>(c, q, t0, t_end, dt0, rtol, atol, max_attempts, hist,
                                                         stats, s);
}

}  // extern "C"
