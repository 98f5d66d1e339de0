// sgn_batch.cuh - one launch per RK4 stage over a ragged ensemble of grids.
//
// The instances (each its own size, boundary treatment, parameters and time
// step) are packed back to back in one state buffer; a tile list enumerates
// every 32 x (8*ROWS) tile of every instance, instance by instance.  Block k
// takes tile k, reads its tile record and instance descriptor and runs the
// same halo-tile evaluation of the split-form RHS (eq. (sd_periodic_2D_SGN) /
// eq. (semi_2D))
// and RK4 stage algebra as the single-grid kernel, with the same arithmetic in
// the same order, so a batched run equals the per-instance runs bit for bit.
// ROWS (rows per thread: 1, 2 or 4) sets the tile height; the autotuner picks
// it by timing.
#pragma once

#include "sgn_kernels.cuh"
#include "sgn_fused.cuh"

namespace sgn {

struct InstDesc {
    Geom G;
    int bc;
    long long off;         // element offset of the instance's first plane (b); state: 5 * off
    double c_acc[4];       // per-stage coefficients of the accumulator update
    double c_q[4];         // per-stage coefficients of the next stage state
    long long band0;       // first diagnostics partial (32 x 8 band) of the instance
    int nbands;            // its bands: ceil(nx/32) ceil(ny/8), band-major
};

// One tile of a tile list: the instance and where its planes start, the
// instance's grid and boundary treatment (so that a block can address its
// tile from this one record), and the tile's first node.
struct PTile {
    long long off;         // element offset of the instance's bathymetry plane (state: 5 off)
    int inst;              // instance (descriptor index)
    int i0, j0;            // first node of the tile
    int nx, ny;            // the instance's grid
    int bc;
};
static_assert(sizeof(PTile) == 32, "one 32-byte record per tile");

template <typename TC, typename TIN, typename TA>
struct BatchArgs {
    const InstDesc* desc;
    const PTile* tiles;
    const TIN* X;          // packed stage input
    const TC* b;           // packed bathymetry (compute type)
    const double* b64;     // packed bathymetry (double; diagnostics)
    const TA* qn;
    TA* acc;
    TC* Qout;
    TA* out;
    double* partials;      // DIAG: NDIAG per 32 x 8 band of every instance
    int* flag;
    int stage;             // 0..3: index into c_acc / c_q
};

// Shared-memory layout of the batched kernel: the factored tile for the float
// compute type, as in the single-grid kernel (measured 6.5% faster than the
// full tile on the ensemble workload; SGN_BATCH_FACT=0 builds the full tile).
#ifndef SGN_BATCH_FACT
#define SGN_BATCH_FACT 1
#endif
template <typename TC>
constexpr bool kBatchFact = SGN_BATCH_FACT && TileLayout<TC>::factored;

// Resident blocks per SM the registers of the batched kernel must allow in
// the FP32 mode: six (40 registers) for S1K and five (48) for the last stage,
// which move few bytes per node and gain from more blocks in flight (the last
// stage's reflecting branch would spill at 40), four (64) for the middle ones
// (S2K among them), which would spill at 48; no bound in the mixed mode, whose
// double registers would spill under these.
template <typename TC, typename TA, int MODE>
constexpr int kBatchMinBlocks = !(TileLayout<TC>::factored && sizeof(TA) == 4)            ? 1
                                : (MODE == MODE_S2 || MODE == MODE_S3 || MODE == MODE_S2K) ? 4
                                : MODE == MODE_S1K                                         ? 6
                                                                                            : 5;

template <typename TC, typename TIN, typename TA, int MODE, int ROWS>
__global__ void __launch_bounds__(BLOCK_THREADS, (kBatchMinBlocks<TC, TA, MODE>))
k_batch_stage(BatchArgs<TC, TIN, TA> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TC* sm = reinterpret_cast<TC*>(smem_raw);
    const PTile T = a.tiles[blockIdx.x];
    const InstDesc& d = a.desc[T.inst];
    // The tile is addressed from its record alone (one dependent load before
    // the tile's loads can issue); the grid constants come from the
    // descriptor by loads that do not hold up the tile's.
    Geom G = d.G;
    G.nx = T.nx;
    G.ny = T.ny;
    G.plane = (long long)T.nx * T.ny;
    StageArgs<TC, TIN, TA> s;
    const long long so = 5 * T.off;
    s.X = a.X + so;
    s.b = a.b + T.off;
    s.qn = a.qn ? a.qn + so : nullptr;
    s.acc = a.acc ? a.acc + so : nullptr;
    s.Qout = a.Qout ? a.Qout + so : nullptr;
    s.out = a.out ? a.out + so : nullptr;
    s.partials = nullptr;
    s.b64 = a.b64 ? a.b64 + T.off : nullptr;
    s.flag = a.flag;
    s.G = G;
    s.c_acc = (TA)d.c_acc[a.stage];
    s.c_q = (TA)d.c_q[a.stage];
    s.c_acc1 = (TA)d.c_acc[0];       // S2K: the first stage's dt/6 and dt/2
    s.c_q1 = (TA)d.c_q[0];
    // the band partials of the instance, laid out as those of a single-grid launch
    const long long nbx = (T.nx + TILE_X - 1) / TILE_X;
    double* slot = a.partials ? a.partials + (d.band0 + (T.j0 / THREADS_Y) * nbx + T.i0 / TILE_X) * NDIAG
                              : nullptr;
    // the tile layout of kBatchFact: same products, same rounding either way
    if (T.bc == BC_REFLECTING)
        stage_tile<TC, TIN, TA, BC_REFLECTING, MODE, ROWS, kBatchFact<TC>>(s, G, T.i0, T.j0, sm, slot, nbx * NDIAG);
    else
        stage_tile<TC, TIN, TA, BC_PERIODIC, MODE, ROWS, kBatchFact<TC>>(s, G, T.i0, T.j0, sm, slot, nbx * NDIAG);
}

// Two RK4 stages per launch over the ensemble (FP32; see sgn_fused.cuh):
// block k takes the 32 x 16 tile of record first + k and runs fused_tile with the
// instance's planes, grid and coefficients, so every instance advances as
// its single-grid fused (and unfused) steps do, bit for bit.
template <typename TC, typename TA>
struct BatchFusedArgs {
    const InstDesc* desc;
    const PTile* tiles;    // the 32 x 16 tiles (rows 2)
    const TA* q;           // packed q_n
    const TC* X;           // S34: packed Q3
    const TC* b;           // packed bathymetry (compute type)
    TA* acc;
    TC* Qout;              // S12: packed Q3
    TA* out;               // S34: packed q_{n+1}
    int* flag;
    long long first;       // the launch's first tile record
};

// Tile classes of a fused launch: every tile periodic, every tile reflecting,
// or either (the boundary treatment read from the record).  W32: 32-bit
// element offsets (every instance's plane below 2^32 nodes); in the batched
// kernels they measured faster for both pairs and both classes.
enum { CLS_MIXED = 0, CLS_PERIODIC = 1, CLS_REFLECTING = 2 };
// (registers as the single-grid kernels of the class: the reflecting S34 for
// three blocks per SM)
template <typename TC, typename TA, int PAIR, int CLS, bool W32 = false>
__global__ void __launch_bounds__(BLOCK_THREADS, (kFusedMinBlocks<CLS == CLS_PERIODIC ? BC_PERIODIC : BC_REFLECTING, PAIR>))
k_batch_fused(BatchFusedArgs<TC, TA> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const PTile T = a.tiles[a.first + blockIdx.x];
    const InstDesc& d = a.desc[T.inst];
    Geom G = d.G;
    G.nx = T.nx;
    G.ny = T.ny;
    G.plane = (long long)T.nx * T.ny;
    FusedArgs<TC, TA> f;
    const long long so = 5 * T.off;
    f.q = a.q + so;
    f.X = a.X ? a.X + so : nullptr;
    f.b = a.b + T.off;
    f.acc = a.acc + so;
    f.Qout = a.Qout ? a.Qout + so : nullptr;
    f.out = a.out ? a.out + so : nullptr;
    f.flag = a.flag;
    // the coefficients as the single-grid path rounds them: (TA)(dt/6) etc.
    f.c_a1 = (TA)d.c_acc[0];
    f.c_a2 = (TA)d.c_acc[1];
    f.c_a3 = (TA)d.c_acc[2];
    f.c_a4 = (TA)d.c_acc[3];
    f.c_q1 = (TA)d.c_q[0];
    f.c_q2 = (TA)d.c_q[1];
    f.c_q3 = (TA)d.c_q[2];
    TC* sm = reinterpret_cast<TC*>(smem_raw);
    if (CLS == CLS_PERIODIC || (CLS == CLS_MIXED && T.bc == BC_PERIODIC))
        fused_tile<TC, TA, BC_PERIODIC, PAIR, 2, W32>(f, G, T.i0, T.j0, sm);
    else
        fused_tile<TC, TA, BC_REFLECTING, PAIR, 2, W32>(f, G, T.i0, T.j0, sm);
}

// Per-instance sums of the band partials, in band order (one block each; the
// same fixed-order sum as k_reduce_partials over a single grid's bands).
static __global__ void __launch_bounds__(256) k_batch_reduce(const InstDesc* __restrict__ desc,
                                                              const double* __restrict__ partials,
                                                              double* __restrict__ out) {
    __shared__ double red[256][NDIAG];
    const InstDesc& d = desc[blockIdx.x];
    double s[NDIAG] = {0.0, 0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < d.nbands; k += 256)
#pragma unroll
        for (int q = 0; q < NDIAG; q++) s[q] += partials[(d.band0 + k) * NDIAG + q];
#pragma unroll
    for (int q = 0; q < NDIAG; q++) red[threadIdx.x][q] = s[q];
    __syncthreads();
    for (int stride = 128; stride > 0; stride >>= 1) {
        if ((int)threadIdx.x < stride)
#pragma unroll
            for (int q = 0; q < NDIAG; q++) red[threadIdx.x][q] += red[threadIdx.x + stride][q];
        __syncthreads();
    }
    if (threadIdx.x < NDIAG) out[(long long)blockIdx.x * NDIAG + threadIdx.x] = red[0][threadIdx.x];
}

}  // namespace sgn
