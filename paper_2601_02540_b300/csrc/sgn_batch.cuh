// sgn_batch.cuh - one launch per RK4 stage over a ragged ensemble of grids.
//
// The instances (each its own size, boundary treatment, parameters and time
// step) are packed back to back in one state buffer; a tile list enumerates
// every 32 x (8*ROWS) tile of every instance, instance by instance.  Block k
// takes tile k, reads its instance descriptor and runs the same halo-tile
// evaluation of the split-form RHS (eq. (sd_periodic_2D_SGN) / eq. (semi_2D))
// and RK4 stage algebra as the single-grid kernel, with the same arithmetic in
// the same order, so a batched run equals the per-instance runs bit for bit.
// ROWS (rows per thread: 1, 2 or 4) sets the tile height; the autotuner picks
// it by timing.
#pragma once

#include "sgn_kernels.cuh"

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

template <typename TC, typename TIN, typename TA>
struct BatchArgs {
    const InstDesc* desc;
    const int4* tiles;     // {instance, i0, j0, 0}
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

template <typename TC, typename TIN, typename TA, int MODE, int ROWS>
__global__ void __launch_bounds__(BLOCK_THREADS)
k_batch_stage(BatchArgs<TC, TIN, TA> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TC* sm = reinterpret_cast<TC*>(smem_raw);
    const int4 tile = a.tiles[blockIdx.x];
    const InstDesc& d = a.desc[tile.x];
    // the instance's planes and stage coefficients, then the shared tile body
    StageArgs<TC, TIN, TA> s;
    const long long so = 5 * d.off;
    s.X = a.X + so;
    s.b = a.b + d.off;
    s.qn = a.qn ? a.qn + so : nullptr;
    s.acc = a.acc ? a.acc + so : nullptr;
    s.Qout = a.Qout ? a.Qout + so : nullptr;
    s.out = a.out ? a.out + so : nullptr;
    s.partials = nullptr;
    s.b64 = a.b64 ? a.b64 + d.off : nullptr;
    s.flag = a.flag;
    s.G = d.G;
    s.c_acc = (TA)d.c_acc[a.stage];
    s.c_q = (TA)d.c_q[a.stage];
    // the band partials of the instance, laid out as those of a single-grid launch
    const long long nbx = (d.G.nx + TILE_X - 1) / TILE_X;
    double* slot = a.partials ? a.partials + (d.band0 + (tile.z / THREADS_Y) * nbx + tile.y / TILE_X) * NDIAG
                              : nullptr;
    // the tile layout of kBatchFact: same products, same rounding either way
    if (d.bc == BC_REFLECTING)
        stage_tile<TC, TIN, TA, BC_REFLECTING, MODE, ROWS, kBatchFact<TC>>(s, d.G, tile.y, tile.z, sm, slot, nbx * NDIAG);
    else
        stage_tile<TC, TIN, TA, BC_PERIODIC, MODE, ROWS, kBatchFact<TC>>(s, d.G, tile.y, tile.z, sm, slot, nbx * NDIAG);
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
