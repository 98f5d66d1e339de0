// sgn_batch.cu - ragged ensembles: many independent grids advanced by one
// launch per RK4 stage (sgn_batch_* in include/sgn.h), replayed from CUDA
// graphs, with the tile height chosen by timing (sgn_batch_autotune).
#include "sgn.h"
#include "sgn_batch.cuh"
#include "sgn_persist.cuh"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

void sgn_record_error(const char* msg);
void sgn_count_launches(unsigned long long n);

namespace {

sgn_status bfail(sgn_status s, const char* msg) {
    sgn_record_error(msg);
    return s;
}

sgn_status bcuda(cudaError_t e, const char* what) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    sgn_record_error(buf);
    return SGN_E_CUDA;
}

constexpr int kGraphSteps = 26;   // RK4 steps captured per graph replay (even: the two-stage
                                  // FP32 launches end an odd step count with a copy of the state)

}  // namespace

struct sgn_batch {
    int ninst = 0;
    int prec = SGN_F64;
    int rows = 2;                      // rows per thread (tile height 8*rows)
    long long cells = 0;
    size_t tc = 8, ta = 8;
    std::vector<sgn::InstDesc> hdesc;
    sgn::InstDesc* desc = nullptr;     // device
    sgn::PTile* tiles[3] = {nullptr, nullptr, nullptr};   // tile records for rows = 1, 2, 4
    long long ntiles[3] = {0, 0, 0};
    long long nper2 = 0;               // periodic tiles, at the front of the rows-2 list
    bool w32 = false;                  // every instance's plane below 2^32 nodes (fused: 32-bit offsets)
    // the persistent kernel (float compute types, rows = 1, 2): its grid per
    // (rows, stage), resident blocks per SM x SMs
    int pgrid[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    int persist = 0;                   // 1: RK4 stages by the persistent kernel
    int fuse = 0;                      // 1 (FP32): two RK4 stages per launch (k_batch_fused)
    double* b64 = nullptr;
    void* bT = nullptr;
    void* acc = nullptr;
    void* Qa = nullptr;
    void* Qb = nullptr;
    double* partials = nullptr;        // NDIAG per tile (largest tile list)
    double* dout = nullptr;
    int* flag = nullptr;
    cudaStream_t cap = nullptr;        // private stream used only for graph capture
    cudaGraphExec_t exec = nullptr;
    const void* exec_q = nullptr;
    int exec_rows = 0;
    int exec_persist = 0;
    int exec_fuse = 0;
    bool capturing = false;            // launches recorded into a graph are counted on replay
};

namespace {

// Kernel launches per RK4 step of the batched path as configured.
unsigned long long fused_launches_per_step(const sgn_batch* B) {
    if (!(B->fuse && !B->persist && B->prec == SGN_F32)) return 4ull;
    return 2ull * ((B->nper2 > 0 ? 1ull : 0ull) + (B->ntiles[1] > B->nper2 ? 1ull : 0ull));
}

int rows_index(int rows) { return rows == 1 ? 0 : (rows == 2 ? 1 : 2); }

template <typename TC, typename TIN, typename TA, int MODE, int ROWS>
cudaError_t blaunch(const sgn_batch* B, const sgn::BatchArgs<TC, TIN, TA>& a, cudaStream_t s) {
    const int ri = rows_index(ROWS);
    const size_t smem = sgn::stage_smem_bytes<TC, MODE, sgn::kBatchFact<TC>>(ROWS);
    sgn::BatchArgs<TC, TIN, TA> b = a;
    b.tiles = B->tiles[ri];
    sgn::k_batch_stage<TC, TIN, TA, MODE, ROWS>
        <<<(unsigned)B->ntiles[ri], dim3(sgn::TILE_X, sgn::THREADS_Y), smem, s>>>(b);
    if (!B->capturing) sgn_count_launches(1);
    return cudaGetLastError();
}

// the persistent kernel: one grid of resident blocks walks the tile list
template <typename TC, typename TIN, typename TA, int MODE, int ROWS>
cudaError_t plaunch(const sgn_batch* B, const sgn::PersistArgs<TC, TIN, TA>& a, cudaStream_t s) {
    const int ri = ROWS == 1 ? 0 : 1;
    sgn::PersistArgs<TC, TIN, TA> b = a;
    b.tiles = B->tiles[ri];
    b.ntiles = B->ntiles[ri];
    const int stage = MODE - sgn::MODE_S1;
    sgn::k_batch_persist<TC, TIN, TA, MODE, ROWS>
        <<<(unsigned)B->pgrid[ri][stage], dim3(sgn::TILE_X, sgn::THREADS_Y), sgn::PersistLayout<TC, TIN, ROWS>::bytes,
           s>>>(b);
    if (!B->capturing) sgn_count_launches(1);
    return cudaGetLastError();
}

// shared-memory opt-in and grid (resident blocks per SM x SMs, at most one
// block per tile) of one persistent kernel
template <typename TC, typename TIN, typename TA, int MODE, int ROWS>
cudaError_t set_persist(sgn_batch* B, int sms) {
    auto kern = sgn::k_batch_persist<TC, TIN, TA, MODE, ROWS>;
    const size_t smem = sgn::PersistLayout<TC, TIN, ROWS>::bytes;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, sgn::BLOCK_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int ri = ROWS == 1 ? 0 : 1;
    const long long g = std::min<long long>((long long)per_sm * sms, B->ntiles[ri]);
    B->pgrid[ri][MODE - sgn::MODE_S1] = (int)std::max<long long>(g, 1);
    return cudaSuccess;
}

template <typename TC, typename TA, int ROWS>
cudaError_t set_persist_rows(sgn_batch* B, int sms) {
    cudaError_t e = set_persist<TC, TA, TA, sgn::MODE_S1, ROWS>(B, sms);
    if (e == cudaSuccess) e = set_persist<TC, TC, TA, sgn::MODE_S2, ROWS>(B, sms);
    if (e == cudaSuccess) e = set_persist<TC, TC, TA, sgn::MODE_S3, ROWS>(B, sms);
    if (e == cudaSuccess) e = set_persist<TC, TC, TA, sgn::MODE_S4, ROWS>(B, sms);
    return e;
}

template <typename TC, typename TIN, typename TA, int MODE, int ROWS>
cudaError_t set_attr() {
    const size_t smem = sgn::stage_smem_bytes<TC, MODE, sgn::kBatchFact<TC>>(ROWS);
    return cudaFuncSetAttribute(sgn::k_batch_stage<TC, TIN, TA, MODE, ROWS>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename TC, typename TA, int ROWS>
cudaError_t set_attrs_rows() {
    cudaError_t e = set_attr<TC, TA, TA, sgn::MODE_S1, ROWS>();
    if (e == cudaSuccess) e = set_attr<TC, TC, TA, sgn::MODE_S2, ROWS>();
    if constexpr (sgn::kStoreK1<TC, TA>) {
        if (e == cudaSuccess) e = set_attr<TC, TA, TA, sgn::MODE_S1K, ROWS>();
        if (e == cudaSuccess) e = set_attr<TC, TC, TA, sgn::MODE_S2K, ROWS>();
    }
    if (e == cudaSuccess) e = set_attr<TC, TC, TA, sgn::MODE_S3, ROWS>();
    if (e == cudaSuccess) e = set_attr<TC, TC, TA, sgn::MODE_S4, ROWS>();
    if (e == cudaSuccess) e = set_attr<TC, TA, TA, sgn::MODE_DIAG, ROWS>();
    return e;
}

template <typename TC, typename TA>
cudaError_t set_attrs() {
    if constexpr (sgn::kStoreK1<TC, TA>) {
        const size_t smem = sgn::FusedLayout<2>::template bytes<TC>();
        const void* fk[8] = {
            (const void*)sgn::k_batch_fused<TC, TA, sgn::FUSED_S12, sgn::CLS_PERIODIC, false>,
            (const void*)sgn::k_batch_fused<TC, TA, sgn::FUSED_S12, sgn::CLS_REFLECTING, false>,
            (const void*)sgn::k_batch_fused<TC, TA, sgn::FUSED_S34, sgn::CLS_PERIODIC, false>,
            (const void*)sgn::k_batch_fused<TC, TA, sgn::FUSED_S34, sgn::CLS_REFLECTING, false>,
            (const void*)sgn::k_batch_fused<TC, TA, sgn::FUSED_S12, sgn::CLS_PERIODIC, true>,
            (const void*)sgn::k_batch_fused<TC, TA, sgn::FUSED_S12, sgn::CLS_REFLECTING, true>,
            (const void*)sgn::k_batch_fused<TC, TA, sgn::FUSED_S34, sgn::CLS_PERIODIC, true>,
            (const void*)sgn::k_batch_fused<TC, TA, sgn::FUSED_S34, sgn::CLS_REFLECTING, true>};
        for (const void* k : fk) {
            const cudaError_t ef = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (ef != cudaSuccess) return ef;
        }
    }
    cudaError_t e = set_attrs_rows<TC, TA, 1>();
    if (e == cudaSuccess) e = set_attrs_rows<TC, TA, 2>();
    if (e == cudaSuccess) e = set_attrs_rows<TC, TA, 4>();
    return e;
}

// One fused launch over the tiles of one class: with 32-bit element offsets
// when every instance's plane is below 2^32 nodes (measured 0.6% faster on
// the ensemble; the same states bit for bit).
template <typename TC, typename TA, int PAIR, int CLS>
cudaError_t launch_fused_class(sgn_batch* B, dim3 grid, size_t smem, const sgn::BatchFusedArgs<TC, TA>& fa,
                               cudaStream_t s) {
    const dim3 block(sgn::TILE_X, sgn::THREADS_Y);
    if (B->w32)
        sgn::k_batch_fused<TC, TA, PAIR, CLS, true><<<grid, block, smem, s>>>(fa);
    else
        sgn::k_batch_fused<TC, TA, PAIR, CLS, false><<<grid, block, smem, s>>>(fa);
    if (!B->capturing) sgn_count_launches(1);
    return cudaGetLastError();
}

// nsteps FP32 steps, two stages per launch over the 32 x 16 tiles: q_{n+1}
// goes to the other of q and Qb (the second launch reads q_n on its halo),
// and an odd step count ends with a copy back into q.
template <typename TC, typename TA>
cudaError_t bsteps_fused(sgn_batch* B, TA* q, int nsteps, cudaStream_t s) {
    static_assert(std::is_same<TC, TA>::value, "Qb holds a state");
    const size_t smem = sgn::FusedLayout<2>::template bytes<TC>();
    sgn::BatchFusedArgs<TC, TA> f;
    std::memset(&f, 0, sizeof(f));
    f.desc = B->desc;
    f.tiles = B->tiles[1];
    f.b = static_cast<const TC*>(B->bT);
    f.acc = static_cast<TA*>(B->acc);
    f.flag = B->flag;
    TA* cur = q;
    TA* nxt = static_cast<TA*>(B->Qb);
    // one launch per tile class (periodic tiles first), each with the
    // registers of its own boundary treatment
    const long long np = B->nper2, nr = B->ntiles[1] - B->nper2;
    cudaError_t e = cudaSuccess;
    for (int n = 0; n < nsteps; n++) {
        sgn::BatchFusedArgs<TC, TA> f12 = f;
        f12.q = cur;
        f12.Qout = static_cast<TC*>(B->Qa);
        sgn::BatchFusedArgs<TC, TA> f34 = f;
        f34.q = cur;
        f34.X = static_cast<const TC*>(B->Qa);
        f34.out = nxt;
        for (int pair = 0; pair < 2; pair++) {
            sgn::BatchFusedArgs<TC, TA> fa = pair == 0 ? f12 : f34;
            for (int cls = 0; cls < 2; cls++) {
                const long long nt = cls == 0 ? np : nr;
                if (nt == 0) continue;
                fa.first = cls == 0 ? 0 : np;
                const dim3 grid((unsigned)nt);
                if (pair == 0)
                    e = cls == 0 ? launch_fused_class<TC, TA, sgn::FUSED_S12, sgn::CLS_PERIODIC>(B, grid, smem, fa, s)
                                 : launch_fused_class<TC, TA, sgn::FUSED_S12, sgn::CLS_REFLECTING>(B, grid, smem, fa, s);
                else
                    e = cls == 0 ? launch_fused_class<TC, TA, sgn::FUSED_S34, sgn::CLS_PERIODIC>(B, grid, smem, fa, s)
                                 : launch_fused_class<TC, TA, sgn::FUSED_S34, sgn::CLS_REFLECTING>(B, grid, smem, fa, s);
                if (e != cudaSuccess) return e;
            }
        }
        std::swap(cur, nxt);
    }
    if (cur != q) e = cudaMemcpyAsync(q, cur, (size_t)5 * B->cells * sizeof(TA), cudaMemcpyDeviceToDevice, s);
    return e;
}

// nsteps RK4 steps, four launches each (ping-pong stage states as sgn_step),
// or two stage pairs per step by bsteps_fused
template <typename TC, typename TA, int ROWS>
cudaError_t bsteps(sgn_batch* B, TA* q, int nsteps, cudaStream_t s) {
    if constexpr (sgn::kStoreK1<TC, TA>) {
        if (B->fuse && !B->persist) return bsteps_fused<TC, TA>(B, q, nsteps, s);
    }
    sgn::BatchArgs<TC, TA, TA> a1;
    std::memset(&a1, 0, sizeof(a1));
    a1.desc = B->desc;
    a1.b = static_cast<const TC*>(B->bT);
    a1.flag = B->flag;
    a1.X = q; a1.qn = q; a1.acc = static_cast<TA*>(B->acc); a1.Qout = static_cast<TC*>(B->Qa); a1.stage = 0;
    sgn::BatchArgs<TC, TC, TA> a2;
    std::memset(&a2, 0, sizeof(a2));
    a2.desc = B->desc;
    a2.b = a1.b;
    a2.flag = B->flag;
    a2.qn = q; a2.acc = a1.acc; a2.X = static_cast<TC*>(B->Qa); a2.Qout = static_cast<TC*>(B->Qb); a2.stage = 1;
    sgn::BatchArgs<TC, TC, TA> a3 = a2;
    a3.X = static_cast<TC*>(B->Qb); a3.Qout = static_cast<TC*>(B->Qa); a3.stage = 2;
    sgn::BatchArgs<TC, TC, TA> a4 = a2;
    a4.X = static_cast<TC*>(B->Qa); a4.Qout = nullptr; a4.qn = nullptr; a4.out = q; a4.stage = 3;
    if constexpr (sgn::TileLayout<TC>::factored && ROWS <= 2) {
        if (B->persist) {
            // the same four stages by the persistent kernel
            sgn::PersistArgs<TC, TA, TA> p1;
            std::memset(&p1, 0, sizeof(p1));
            p1.desc = B->desc; p1.b = a1.b; p1.flag = B->flag;
            p1.X = q; p1.qn = q; p1.acc = a1.acc; p1.Qout = a1.Qout; p1.stage = 0;
            sgn::PersistArgs<TC, TC, TA> p2;
            std::memset(&p2, 0, sizeof(p2));
            p2.desc = B->desc; p2.b = a1.b; p2.flag = B->flag;
            p2.X = a2.X; p2.qn = q; p2.acc = a1.acc; p2.Qout = a2.Qout; p2.stage = 1;
            sgn::PersistArgs<TC, TC, TA> p3 = p2;
            p3.X = a3.X; p3.Qout = a3.Qout; p3.stage = 2;
            sgn::PersistArgs<TC, TC, TA> p4 = p2;
            p4.X = a4.X; p4.Qout = nullptr; p4.qn = nullptr; p4.out = q; p4.stage = 3;
            for (int n = 0; n < nsteps; n++) {
                cudaError_t e;
                if ((e = plaunch<TC, TA, TA, sgn::MODE_S1, ROWS>(B, p1, s)) != cudaSuccess) return e;
                if ((e = plaunch<TC, TC, TA, sgn::MODE_S2, ROWS>(B, p2, s)) != cudaSuccess) return e;
                if ((e = plaunch<TC, TC, TA, sgn::MODE_S3, ROWS>(B, p3, s)) != cudaSuccess) return e;
                if ((e = plaunch<TC, TC, TA, sgn::MODE_S4, ROWS>(B, p4, s)) != cudaSuccess) return e;
            }
            return cudaSuccess;
        }
    }
    for (int n = 0; n < nsteps; n++) {
        cudaError_t e;
        if constexpr (sgn::kStoreK1<TC, TA>) {
            // FP32: stage 1 stores k1 only, stage 2 forms the rest
            if ((e = blaunch<TC, TA, TA, sgn::MODE_S1K, ROWS>(B, a1, s)) != cudaSuccess) return e;
            if ((e = blaunch<TC, TC, TA, sgn::MODE_S2K, ROWS>(B, a2, s)) != cudaSuccess) return e;
        } else {
            if ((e = blaunch<TC, TA, TA, sgn::MODE_S1, ROWS>(B, a1, s)) != cudaSuccess) return e;
            if ((e = blaunch<TC, TC, TA, sgn::MODE_S2, ROWS>(B, a2, s)) != cudaSuccess) return e;
        }
        if ((e = blaunch<TC, TC, TA, sgn::MODE_S3, ROWS>(B, a3, s)) != cudaSuccess) return e;
        if ((e = blaunch<TC, TC, TA, sgn::MODE_S4, ROWS>(B, a4, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename TC, typename TA>
cudaError_t bsteps_rows(sgn_batch* B, void* q, int nsteps, int rows, cudaStream_t s) {
    TA* qq = static_cast<TA*>(q);
    if (rows == 1) return bsteps<TC, TA, 1>(B, qq, nsteps, s);
    if (rows == 4) return bsteps<TC, TA, 4>(B, qq, nsteps, s);
    return bsteps<TC, TA, 2>(B, qq, nsteps, s);
}

cudaError_t bsteps_any(sgn_batch* B, void* q, int nsteps, int rows, cudaStream_t s) {
    switch (B->prec) {
    case SGN_F64: return bsteps_rows<double, double>(B, q, nsteps, rows, s);
    case SGN_F32: return bsteps_rows<float, float>(B, q, nsteps, rows, s);
    default: return bsteps_rows<float, double>(B, q, nsteps, rows, s);
    }
}

template <typename TC, typename TA, int ROWS>
cudaError_t bdiag(sgn_batch* B, const TA* q, cudaStream_t s) {
    sgn::BatchArgs<TC, TA, TA> a;
    std::memset(&a, 0, sizeof(a));
    a.desc = B->desc;
    a.b = static_cast<const TC*>(B->bT);
    a.b64 = B->b64;
    a.flag = B->flag;
    a.X = q;
    a.partials = B->partials;
    cudaError_t e = blaunch<TC, TA, TA, sgn::MODE_DIAG, ROWS>(B, a, s);
    if (e != cudaSuccess) return e;
    sgn::k_batch_reduce<<<B->ninst, 256, 0, s>>>(B->desc, B->partials, B->dout);
    sgn_count_launches(1);
    return cudaGetLastError();
}

template <typename TC, typename TA>
cudaError_t bdiag_rows(sgn_batch* B, const void* q, cudaStream_t s) {
    const TA* qq = static_cast<const TA*>(q);
    if (B->rows == 1) return bdiag<TC, TA, 1>(B, qq, s);
    if (B->rows == 4) return bdiag<TC, TA, 4>(B, qq, s);
    return bdiag<TC, TA, 2>(B, qq, s);
}

void free_batch(sgn_batch* B) {
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->cap) cudaStreamDestroy(B->cap);
    cudaFree(B->desc);
    for (auto* t : B->tiles) cudaFree(t);
    if (B->bT && B->bT != B->b64) cudaFree(B->bT);
    cudaFree(B->b64);
    cudaFree(B->acc);
    cudaFree(B->Qa);
    cudaFree(B->Qb);
    cudaFree(B->partials);
    cudaFree(B->dout);
    cudaFree(B->flag);
    delete B;
}

bool devptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// (re)build the graph of kGraphSteps RK4 steps for this state pointer and tiling
sgn_status ensure_graph(sgn_batch* B, void* q) {
    if (B->exec && B->exec_q == q && B->exec_rows == B->rows && B->exec_persist == B->persist &&
        B->exec_fuse == B->fuse)
        return SGN_OK;
    if (B->exec) {
        cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(e, "begin capture");
    B->capturing = true;
    cudaError_t el = bsteps_any(B, q, kGraphSteps, B->rows, B->cap);
    B->capturing = false;
    e = cudaStreamEndCapture(B->cap, &graph);
    if (el != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return bcuda(el != cudaSuccess ? el : e, "capture");
    }
    e = cudaGraphInstantiate(&B->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        B->exec = nullptr;
        return bcuda(e, "instantiate graph");
    }
    B->exec_q = q;
    B->exec_rows = B->rows;
    B->exec_persist = B->persist;
    B->exec_fuse = B->fuse;
    return SGN_OK;
}

}  // namespace

extern "C" {

sgn_status sgn_batch_create(const sgn_instance* inst, int ninst, int prec, const void* b_dev, sgn_batch** out) {
    if (!out) return bfail(SGN_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!inst || ninst <= 0) return bfail(SGN_E_INVAL, "need at least one instance");
    if (prec != SGN_F64 && prec != SGN_F32 && prec != SGN_F32_F64ACC) return bfail(SGN_E_INVAL, "bad prec");
    if (!devptr(b_dev)) return bfail(SGN_E_INVAL, "b_dev is not device memory");
    sgn_batch* B = new (std::nothrow) sgn_batch();
    if (!B) return bfail(SGN_E_NOMEM, "host allocation");
    B->ninst = ninst;
    B->prec = prec;
    B->fuse = prec == SGN_F32;
    B->tc = prec == SGN_F64 ? 8 : 4;
    B->ta = prec == SGN_F32 ? 4 : 8;
    B->hdesc.resize(ninst);
    std::vector<int4> tl[3];
    long long off = 0;
    for (int k = 0; k < ninst; k++) {
        const sgn_instance& p = inst[k];
        // ny bound: the per-instance 32 x 8 launches (init_aux) fit the launch grid's y limit
        // and below 2^32 nodes for the float-based kernels (32-bit offsets within a plane)
        if (p.nx < 3 || p.ny < 3 || p.ny > 65535 * sgn::THREADS_Y ||
            (prec != SGN_F64 && (long long)p.nx * p.ny > 0xffffffffLL) ||
            (p.bc != SGN_BC_PERIODIC && p.bc != SGN_BC_REFLECTING) ||
            !(std::isfinite(p.xmin) && std::isfinite(p.xmax) && p.xmax > p.xmin && std::isfinite(p.ymin) &&
              std::isfinite(p.ymax) && p.ymax > p.ymin) ||
            !(std::isfinite(p.g) && p.g > 0) || !(std::isfinite(p.lambda) && p.lambda >= 0) ||
            !(std::isfinite(p.dt) && p.dt > 0)) {
            free_batch(B);
            return bfail(SGN_E_INVAL, "invalid instance parameters");
        }
        sgn::InstDesc& d = B->hdesc[k];
        std::memset(&d, 0, sizeof(d));
        const bool per = p.bc == SGN_BC_PERIODIC;
        const double dx = per ? (p.xmax - p.xmin) / p.nx : (p.xmax - p.xmin) / (p.nx - 1);
        const double dy = per ? (p.ymax - p.ymin) / p.ny : (p.ymax - p.ymin) / (p.ny - 1);
        sgn::fill_geom(d.G, p.nx, p.ny, dx, dy, p.g, p.lambda);
        d.bc = p.bc;
        d.off = off;
        // same coefficients, computed the same way, as sgn_step
        d.c_acc[0] = p.dt / 6.0; d.c_q[0] = p.dt / 2.0;
        d.c_acc[1] = p.dt / 3.0; d.c_q[1] = p.dt / 2.0;
        d.c_acc[2] = p.dt / 3.0; d.c_q[2] = p.dt;
        d.c_acc[3] = p.dt / 6.0; d.c_q[3] = 0.0;
        off += d.G.plane;
    }
    B->cells = off;
    B->w32 = true;
    for (const sgn::InstDesc& d : B->hdesc)
        if ((unsigned long long)d.G.plane > 0xffffffffull) B->w32 = false;
    // tile lists for the three tile heights (rows = 1: the 32 x 8 bands)
    for (int ri = 0; ri < 3; ri++) {
        const int th = sgn::THREADS_Y * (ri == 0 ? 1 : (ri == 1 ? 2 : 4));
        // rows 2 (the fused launches): the periodic instances' tiles first
        for (int pass = 0; pass < (ri == 1 ? 2 : 1); pass++) {
            for (int k = 0; k < ninst; k++) {
                if (ri == 1 && (B->hdesc[k].bc == SGN_BC_PERIODIC) != (pass == 0)) continue;
                const sgn::Geom& G = B->hdesc[k].G;
                for (int j0 = 0; j0 < G.ny; j0 += th)
                    for (int i0 = 0; i0 < G.nx; i0 += sgn::TILE_X) tl[ri].push_back(make_int4(k, i0, j0, 0));
            }
            if (ri == 1 && pass == 0) B->nper2 = (long long)tl[ri].size();
        }
        B->ntiles[ri] = (long long)tl[ri].size();
    }
    if (B->ntiles[0] > 2147483647LL) {
        free_batch(B);
        return bfail(SGN_E_INVAL, "too many tiles");
    }
    const size_t n = (size_t)B->cells;
    bool ok = cudaMalloc(&B->desc, sizeof(sgn::InstDesc) * ninst) == cudaSuccess;
    for (int ri = 0; ri < 3 && ok; ri++)
        ok = cudaMalloc(&B->tiles[ri], sizeof(sgn::PTile) * tl[ri].size()) == cudaSuccess;
    ok = ok && cudaMalloc(&B->b64, n * sizeof(double)) == cudaSuccess;
    if (ok && prec != SGN_F64) ok = cudaMalloc(&B->bT, n * sizeof(float)) == cudaSuccess;
    if (ok && prec == SGN_F64) B->bT = B->b64;
    ok = ok && cudaMalloc(&B->acc, 5 * n * B->ta) == cudaSuccess;
    ok = ok && cudaMalloc(&B->Qa, 5 * n * B->tc) == cudaSuccess;
    ok = ok && cudaMalloc(&B->Qb, 5 * n * B->tc) == cudaSuccess;
    ok = ok && cudaMalloc(&B->partials, (size_t)B->ntiles[0] * sgn::NDIAG * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc(&B->dout, (size_t)ninst * sgn::NDIAG * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc(&B->flag, sizeof(int)) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_batch(B);
        return bfail(SGN_E_NOMEM, "batch scratch");
    }
    cudaError_t e = cudaSuccess;
    for (int ri = 0; ri < 3 && e == cudaSuccess; ri++) {
        std::vector<sgn::PTile> pt(tl[ri].size());
        for (size_t k = 0; k < pt.size(); k++) {
            const sgn::InstDesc& d = B->hdesc[tl[ri][k].x];
            pt[k].off = d.off;
            pt[k].inst = tl[ri][k].x;
            pt[k].i0 = tl[ri][k].y;
            pt[k].j0 = tl[ri][k].z;
            pt[k].nx = d.G.nx;
            pt[k].ny = d.G.ny;
            pt[k].bc = d.bc;
        }
        e = cudaMemcpy(B->tiles[ri], pt.data(), sizeof(sgn::PTile) * pt.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(B->flag, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(B->b64, b_dev, n * sizeof(double), cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess && prec != SGN_F64) {
        sgn::k_convert<float><<<592, 256>>>(B->b64, static_cast<float*>(B->bT), (long long)n);
        sgn_count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        switch (prec) {
        case SGN_F64: e = set_attrs<double, double>(); break;
        case SGN_F32: e = set_attrs<float, float>(); break;
        default: e = set_attrs<float, double>(); break;
        }
    }
    if (e == cudaSuccess && prec != SGN_F64) {
        int dev = 0, sms = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = prec == SGN_F32 ? set_persist_rows<float, float, 1>(B, sms) : set_persist_rows<float, double, 1>(B, sms);
        if (e == cudaSuccess)
            e = prec == SGN_F32 ? set_persist_rows<float, float, 2>(B, sms) : set_persist_rows<float, double, 2>(B, sms);
    }
    if (e == cudaSuccess) {
        // descriptors with the band ranges: the rows = 1 tiles are the 32 x 8
        // bands, enumerated instance by instance in band-major order
        std::vector<long long> first(ninst, -1), count(ninst, 0);
        for (size_t k = 0; k < tl[0].size(); k++) {
            const int i = tl[0][k].x;
            if (first[i] < 0) first[i] = (long long)k;
            count[i]++;
        }
        for (int i = 0; i < ninst; i++) {
            B->hdesc[i].band0 = first[i];
            B->hdesc[i].nbands = (int)count[i];
        }
        e = cudaMemcpy(B->desc, B->hdesc.data(), sizeof(sgn::InstDesc) * ninst, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        sgn_status st = bcuda(e, "sgn_batch_create");
        free_batch(B);
        return st;
    }
    *out = B;
    return SGN_OK;
}

sgn_status sgn_batch_destroy(sgn_batch* B) {
    if (!B) return SGN_OK;
    cudaError_t e = cudaDeviceSynchronize();
    free_batch(B);
    return e == cudaSuccess ? SGN_OK : bcuda(e, "sgn_batch_destroy");
}

long long sgn_batch_cells(const sgn_batch* B) { return B ? B->cells : -1; }

sgn_status sgn_batch_set_rows(sgn_batch* B, int rows) {
    if (!B) return bfail(SGN_E_INVAL, "batch is NULL");
    if (rows != 1 && rows != 2 && rows != 4) return bfail(SGN_E_INVAL, "rows must be 1, 2 or 4");
    if (rows == 4 && B->persist)
        return bfail(SGN_E_UNSUPPORTED, "the persistent kernel serves rows 1 and 2");
    B->rows = rows;
    return SGN_OK;
}

sgn_status sgn_batch_set_persistent(sgn_batch* B, int on) {
    if (!B) return bfail(SGN_E_INVAL, "batch is NULL");
    if (on != 0 && on != 1) return bfail(SGN_E_INVAL, "on must be 0 or 1");
    if (on && (B->prec == SGN_F64 || B->rows == 4))
        return bfail(SGN_E_UNSUPPORTED, "the persistent kernel serves float compute types with rows 1 or 2");
    B->persist = on;
    return SGN_OK;
}

sgn_status sgn_batch_set_stage_fusion(sgn_batch* B, int on) {
    if (!B) return bfail(SGN_E_INVAL, "batch is NULL");
    if (on != 0 && on != 1) return bfail(SGN_E_INVAL, "on must be 0 or 1");
    if (on && B->prec != SGN_F32) return bfail(SGN_E_UNSUPPORTED, "stage fusion serves SGN_F32 ensembles");
    B->fuse = on;
    return SGN_OK;
}

sgn_status sgn_batch_stage_fusion(const sgn_batch* B, int* on) {
    if (!B || !on) return bfail(SGN_E_INVAL, "batch and on must not be NULL");
    *on = B->fuse;
    return SGN_OK;
}

sgn_status sgn_batch_tiling(const sgn_batch* B, int* rows, int* persistent) {
    if (!B || !rows || !persistent) return bfail(SGN_E_INVAL, "batch, rows and persistent must not be NULL");
    *rows = B->rows;
    *persistent = B->persist;
    return SGN_OK;
}

sgn_status sgn_batch_step(sgn_batch* B, void* q_dev, int nsteps, void* stream) {
    if (!B) return bfail(SGN_E_INVAL, "batch is NULL");
    if (!devptr(q_dev) || reinterpret_cast<uintptr_t>(q_dev) % 16 != 0)
        return bfail(SGN_E_INVAL, "q_dev must be 16-byte aligned device memory");
    if (nsteps < 0) return bfail(SGN_E_INVAL, "nsteps must be >= 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int left = nsteps;
    if (left >= kGraphSteps) {
        sgn_status st = ensure_graph(B, q_dev);
        if (st != SGN_OK) return st;
        while (left >= kGraphSteps) {
            cudaError_t e = cudaGraphLaunch(B->exec, s);
            if (e != cudaSuccess) return bcuda(e, "graph launch");
            sgn_count_launches(fused_launches_per_step(B) * kGraphSteps);
            left -= kGraphSteps;
        }
    }
    if (left > 0) {
        cudaError_t e = bsteps_any(B, q_dev, left, B->rows, s);
        if (e != cudaSuccess) return bcuda(e, "sgn_batch_step");
    }
    return SGN_OK;
}

sgn_status sgn_batch_mass_energy(sgn_batch* B, const void* q_dev, double* out, void* stream) {
    if (!B || !out) return bfail(SGN_E_INVAL, "batch and out must not be NULL");
    if (!devptr(q_dev)) return bfail(SGN_E_INVAL, "q_dev is not device memory");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // band partials: the same sums whatever the tile height
    cudaError_t e;
    switch (B->prec) {
    case SGN_F64: e = bdiag_rows<double, double>(B, q_dev, s); break;
    case SGN_F32: e = bdiag_rows<float, float>(B, q_dev, s); break;
    default: e = bdiag_rows<float, double>(B, q_dev, s); break;
    }
    if (e != cudaSuccess) return bcuda(e, "sgn_batch_mass_energy");
    int flag = 0;
    e = cudaMemcpyAsync(out, B->dout, (size_t)B->ninst * sgn::NDIAG * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, B->flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bcuda(e, "sgn_batch_mass_energy");
    if (flag) {
        cudaMemset(B->flag, 0, sizeof(int));
        if (flag & sgn::FLAG_NONFINITE) return bfail(SGN_E_NONFINITE, "a stage input had a non-finite water height");
        return bfail(SGN_E_NONPOSITIVE_H, "a stage input had a non-positive water height");
    }
    return SGN_OK;
}

sgn_status sgn_batch_autotune(sgn_batch* B, const void* q_dev, int* rows_out, void* stream) {
    if (!B) return bfail(SGN_E_INVAL, "batch is NULL");
    if (!devptr(q_dev)) return bfail(SGN_E_INVAL, "q_dev is not device memory");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = 5 * (size_t)B->cells * B->ta;
    void* work = nullptr;
    if (cudaMalloc(&work, bytes) != cudaSuccess) {
        cudaGetLastError();
        return bfail(SGN_E_NOMEM, "autotune work copy");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        cudaFree(work);
        return bfail(SGN_E_NOMEM, "autotune events");
    }
    // three rounds over the candidate tilings, each timing 8 steps after 2
    // warm-up steps; a candidate's time is its fastest round (robust to a slow
    // round, e.g. while the clocks ramp up)
    // (FP32 also two stages per launch over 32 x 16 tiles)
    const int cand_rows[6] = {1, 2, 4, 1, 2, 2};
    const int cand_persist[6] = {0, 0, 0, 1, 1, 0};
    const int cand_fuse[6] = {0, 0, 0, 0, 0, 1};
    const int ncand = B->prec == SGN_F64 ? 3 : (B->prec == SGN_F32 ? 6 : 5);
    float tmin[6] = {1e30f, 1e30f, 1e30f, 1e30f, 1e30f, 1e30f};
    const int keep_persist = B->persist, keep_fuse = B->fuse;
    cudaError_t e = cudaSuccess;
    for (int round = 0; round < 3 && e == cudaSuccess; round++) {
        for (int k = 0; k < ncand && e == cudaSuccess; k++) {
            B->persist = cand_persist[k];
            B->fuse = cand_fuse[k];
            e = cudaMemcpyAsync(work, q_dev, bytes, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = bsteps_any(B, work, 2, cand_rows[k], s);   // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = bsteps_any(B, work, 8, cand_rows[k], s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && ms < tmin[k]) tmin[k] = ms;
        }
    }
    B->persist = keep_persist;
    B->fuse = keep_fuse;
    float best = 1e30f;
    int best_k = -1;
    for (int k = 0; k < ncand; k++)
        if (tmin[k] < best) {
            best = tmin[k];
            best_k = k;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(work);
    if (e != cudaSuccess) return bcuda(e, "sgn_batch_autotune");
    if (best_k >= 0) {
        B->rows = cand_rows[best_k];
        B->persist = cand_persist[best_k];
        B->fuse = cand_fuse[best_k];
    }
    if (rows_out) *rows_out = B->rows;
    return SGN_OK;
}

sgn_status sgn_batch_init_aux(sgn_batch* B, void* q_dev, void* stream) {
    if (!B) return bfail(SGN_E_INVAL, "batch is NULL");
    if (!devptr(q_dev)) return bfail(SGN_E_INVAL, "q_dev is not device memory");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int k = 0; k < B->ninst; k++) {
        const sgn::InstDesc& d = B->hdesc[k];
        const dim3 blk(32, 8), grd((d.G.nx + 31) / 32, (d.G.ny + 7) / 8);
        if (B->prec == SGN_F32) {
            float* q = static_cast<float*>(q_dev) + 5 * d.off;
            if (d.bc == SGN_BC_REFLECTING) sgn::k_init_aux<float, sgn::BC_REFLECTING><<<grd, blk, 0, s>>>(q, B->b64 + d.off, d.G);
            else sgn::k_init_aux<float, sgn::BC_PERIODIC><<<grd, blk, 0, s>>>(q, B->b64 + d.off, d.G);
        } else {
            double* q = static_cast<double*>(q_dev) + 5 * d.off;
            if (d.bc == SGN_BC_REFLECTING) sgn::k_init_aux<double, sgn::BC_REFLECTING><<<grd, blk, 0, s>>>(q, B->b64 + d.off, d.G);
            else sgn::k_init_aux<double, sgn::BC_PERIODIC><<<grd, blk, 0, s>>>(q, B->b64 + d.off, d.G);
        }
        sgn_count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return bcuda(e, "sgn_batch_init_aux");
    }
    return SGN_OK;
}

}  // extern "C"
