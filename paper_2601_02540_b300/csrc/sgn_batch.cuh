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
    long long tile0;       // first tile of the instance in the tile list
    int ntiles;
};

template <typename TC, typename TIN, typename TA>
struct BatchArgs {
    const InstDesc* desc;
    const int4* tiles;     // {instance, i0, j0, 0}
    const TIN* X;          // packed stage input
    const TC* b;           // packed bathymetry (compute type)
    const TA* qn;
    TA* acc;
    TC* Qout;
    TA* out;
    double* partials;      // DIAG: NDIAG per tile
    int* flag;
    int stage;             // 0..3: index into c_acc / c_q
};

template <typename TC, typename TIN, typename TA, int BC, int MODE, int ROWS>
__device__ __forceinline__ void batch_tile(const BatchArgs<TC, TIN, TA>& a, const InstDesc& d, int i0,
                                           int j0, TC* sm) {
    constexpr int TY = THREADS_Y * ROWS;
    constexpr int HX = TILE_X + 2;
    constexpr int HN = HX * (TY + 2);
    const Geom& G = d.G;
    const long long P = G.plane;
    const TIN* X = a.X + 5 * d.off;
    const TC* bp = a.b + d.off;
    const int tid = threadIdx.y * TILE_X + threadIdx.x;
    int bad = 0;
    for (int t = tid; t < HN; t += BLOCK_THREADS) {
        const int li = t % HX, lj = t / HX;
        const int gi = halo_index<BC>(i0 - 1 + li, G.nx);
        const int gj = halo_index<BC>(j0 - 1 + lj, G.ny);
        const long long c = (long long)gj * G.nx + gi;
        const TC h = (TC)X[c];
        const TC u = (TC)X[P + c];
        const TC v = (TC)X[2 * P + c];
        const TC w = (TC)X[3 * P + c];
        const TC eta = (TC)X[4 * P + c];
        const TC bb = bp[c];
        if (!(h > TC(0))) bad |= (h <= TC(0)) ? FLAG_NONPOSITIVE : FLAG_NONFINITE;
        else if (!(h < pos_inf<TC>())) bad |= FLAG_NONFINITE;
        store_operands<TC, HN>(sm, t, h, u, v, w, eta, bb);
    }
    if (bad) atomicOr(a.flag, bad);
    __syncthreads();

    const TA c_acc = (TA)d.c_acc[a.stage], c_q = (TA)d.c_q[a.stage];
    const long long soff = 5 * d.off;
    double dsum[NDIAG] = {0.0, 0.0, 0.0, 0.0};
    const int gi = i0 + threadIdx.x;
#pragma unroll
    for (int ry = 0; ry < ROWS; ry++) {
        const int ly = threadIdx.y + ry * THREADS_Y;
        const int gj = j0 + ly;
        if (gi >= G.nx || gj >= G.ny) continue;
        const int t = (ly + 1) * HX + (threadIdx.x + 1);
        TC k[5];
        node_rhs<TC, BC, HX, HN>(sm, t, gi, gj, G, k);
        const long long c = soff + (long long)gj * G.nx + gi;
        if (MODE == MODE_S1 || MODE == MODE_S2 || MODE == MODE_S3) {
#pragma unroll
            for (int f = 0; f < 5; f++) {
                const TA qv = a.qn[f * P + c];
                const TA kv = (TA)k[f];
                const TA av = (MODE == MODE_S1) ? qv : a.acc[f * P + c];
                a.acc[f * P + c] = fma_(c_acc, kv, av);
                a.Qout[f * P + c] = (TC)fma_(c_q, kv, qv);
            }
        } else if (MODE == MODE_S4) {
#pragma unroll
            for (int f = 0; f < 5; f++) a.out[f * P + c] = fma_(c_acc, (TA)k[f], a.acc[f * P + c]);
        } else if (MODE == MODE_DIAG) {
            node_diag<TC, BC, HN>(sm, t, gi, gj, G, k, dsum);
        }
    }
    if (MODE == MODE_DIAG) {
        __shared__ double red[BLOCK_THREADS / 32][NDIAG];
        const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
        for (int q = 0; q < NDIAG; q++) {
            double x = dsum[q];
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) red[warp][q] = x;
        }
        __syncthreads();
        if (tid < NDIAG) {
            double x = 0.0;
            for (int wgi = 0; wgi < BLOCK_THREADS / 32; wgi++) x += red[wgi][tid];
            a.partials[(long long)blockIdx.x * NDIAG + tid] = x;
        }
    }
}

template <typename TC, typename TIN, typename TA, int MODE, int ROWS>
__global__ void __launch_bounds__(BLOCK_THREADS)
k_batch_stage(BatchArgs<TC, TIN, TA> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TC* sm = reinterpret_cast<TC*>(smem_raw);
    const int4 tile = a.tiles[blockIdx.x];
    const InstDesc& d = a.desc[tile.x];
    if (d.bc == BC_REFLECTING)
        batch_tile<TC, TIN, TA, BC_REFLECTING, MODE, ROWS>(a, d, tile.y, tile.z, sm);
    else
        batch_tile<TC, TIN, TA, BC_PERIODIC, MODE, ROWS>(a, d, tile.y, tile.z, sm);
}

// Per-instance sums of the per-tile partials, in tile order (one block each).
static __global__ void __launch_bounds__(256) k_batch_reduce(const InstDesc* __restrict__ desc,
                                                              const double* __restrict__ partials,
                                                              double* __restrict__ out) {
    __shared__ double red[256][NDIAG];
    const InstDesc& d = desc[blockIdx.x];
    double s[NDIAG] = {0.0, 0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < d.ntiles; k += 256)
#pragma unroll
        for (int q = 0; q < NDIAG; q++) s[q] += partials[(d.tile0 + k) * NDIAG + q];
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
