// sgn_fused.cuh - two classical RK4 stages per launch (temporal blocking) for
// the FP32 mode, which is bound by memory traffic.  The stages evaluate the
// split-form SBP right-hand side of eq. (sd_periodic_2D_SGN) / eq. (semi_2D)
// as the single-stage kernels do (node_rhs_src).
//
// The unfused FP32 step moves 74 planes per node (S1K 11, S2K 21, S3 26, S4
// 16, see the stage modes).  Here one kernel advances stages 1 and 2 and one
// stages 3 and 4:
//   S12: reads q_n, b; writes acc = (q_n + dt/6 k1) + dt/3 k2 and
//        Q3 = q_n + dt/2 k2                                      16 planes
//   S34: reads Q3, b, q_n, acc; writes q_{n+1} = (acc + dt/3 k3) + dt/6 k4
//                                                               21 planes
// so a step moves 37 planes.  The first stage of a pair is evaluated on the
// output tile grown by one node (the halo the second stage needs), from
// operands staged on the tile grown by two nodes; its result (the second
// stage's input Q2 or Q4) never leaves shared memory.  Every node performs the
// operations of the unfused kernels in the same order and precision (k1, k2,
// k3, k4 by node_rhs_src; the stage states and the accumulator as S1K, S2K,
// S3 and S4 form them), so the states equal the unfused path's bit for bit;
// the nodes of the one-node ring are computed by both neighbouring blocks.
// S34 reads q_n on its halo, so q_{n+1} goes to another buffer than q_n.
#pragma once

#include "sgn_kernels.cuh"

namespace sgn {

enum { FUSED_S12 = 0, FUSED_S34 = 1 };

template <typename TC, typename TA>
struct FusedArgs {
    const TA* q;            // q_n (5 planes)
    const TC* X;            // S34: the stage-3 input Q3 (5 planes)
    const TC* b;            // bathymetry (compute type)
    TA* acc;                // S12: written; S34: read
    TC* Qout;               // S12: Q3
    TA* out;                // S34: q_{n+1}, not aliasing q
    int* flag;              // latched error bits
    Geom G;
    TA c_a1, c_a2, c_a3, c_a4;   // accumulator weights dt/6, dt/3, dt/3, dt/6
    TA c_q1, c_q2, c_q3;         // stage-input weights dt/2, dt/2, dt
};

// Grid index of coordinate k, which may lie up to two tiles' widths outside
// [0, n): periodic wrap (any k), reflecting clamp (such nodes are never read:
// the one-sided end rows use the wall node itself).
template <int BC>
__device__ __forceinline__ int wrap_index(int k, int n) {
    if (k >= 0 && k < n) return k;
    if (BC == BC_PERIODIC) {
        const int m = k % n;
        return m < 0 ? m + n : m;
    }
    return k < 0 ? 0 : n - 1;
}

// Shared-memory layout of a fused tile with R rows per thread (output tile
// 32 x 8R): the tile grown by two nodes (X2) holds the eight factored operand
// planes of the pair's input, then its eta and b; the tile grown by one node
// (X1) holds the factored operands of the second stage's input.
template <int R>
struct FusedLayout {
    static constexpr int TY = THREADS_Y * R;
    static constexpr int HX2 = TILE_X + 4, HN2 = HX2 * (TY + 4);
    static constexpr int HX1 = TILE_X + 2, HN1 = HX1 * (TY + 2);
    static constexpr int P2_ETA = NF_OPS, P2_B = NF_OPS + 1, NP2 = NF_OPS + 2;
    static constexpr int NPER2 = (HN2 + BLOCK_THREADS - 1) / BLOCK_THREADS;
    static constexpr int RING = 2 * HX1 + 2 * TY;      // the one-node ring around the output tile
    static constexpr int NIT = R + 1;                  // first-stage items per thread
    template <typename TC>
    static constexpr size_t bytes() { return ((size_t)NP2 * HN2 + (size_t)NF_OPS * HN1) * sizeof(TC); }
};

// Global element offsets within a plane: 64-bit, or with W32 32-bit (one
// multiply-add forms each address from the plane's base; planes of fewer than
// 2^32 nodes).  The single-grid launches use 32-bit offsets where they
// measured faster: the periodic S34 (1.1% on the FP32 step at 8192^2; slower
// in S12 and in the reflecting S34); the batched kernels in every pair (see
// k_batch_fused).  The results are the same bit for bit.
template <int BC, int PAIR>
constexpr bool kFusedW32 = BC == BC_PERIODIC && PAIR == FUSED_S34;


// One fused output tile (32 x 8R nodes at (i0, j0)) of the pair PAIR.
template <typename TC, typename TA, int BC, int PAIR, int R, bool W32 = false>
__device__ __forceinline__ void fused_tile(const FusedArgs<TC, TA>& a, const Geom& G, int i0, int j0,
                                           TC* __restrict__ sm) {
    static_assert(TileLayout<TC>::factored && std::is_same<TC, TA>::value, "the FP32 mode");
    using L = FusedLayout<R>;
    constexpr int HX2 = L::HX2, HN2 = L::HN2, HX1 = L::HX1, HN1 = L::HN1, TY = L::TY, NIT = L::NIT;
    constexpr int NPER2 = L::NPER2;
    TC* s2 = sm;
    TC* s1 = sm + L::NP2 * HN2;
    const long long P = G.plane;
    using IX = typename std::conditional<W32, unsigned, long long>::type;
    const int tid = threadIdx.y * TILE_X + threadIdx.x;
    int bad = 0;

    // First-stage items: this thread's output nodes (one per row of the tile)
    // and, for the first RING threads, one node of the ring around the tile.
    // it1 < 0: no item (or, on a reflecting grid, a node outside the walls,
    // which no second-stage evaluation reads).
    int it1[NIT], it2[NIT], igx[NIT], igy[NIT];
#pragma unroll
    for (int k = 0; k < NIT; k++) {
        int lx = -1, ly = -1;                   // position in the tile grown by one node
        if (k < R) {
            lx = threadIdx.x + 1;
            ly = threadIdx.y + k * THREADS_Y + 1;
        } else if (tid < L::RING) {
            const int r = tid;
            if (r < HX1) { lx = r; ly = 0; }                                   // row above
            else if (r < 2 * HX1) { lx = r - HX1; ly = TY + 1; }               // row below
            else if (r < 2 * HX1 + TY) { lx = 0; ly = r - 2 * HX1 + 1; }       // left column
            else { lx = HX1 - 1; ly = r - 2 * HX1 - TY + 1; }                  // right column
        }
        it1[k] = -1;
        it2[k] = 0;
        igx[k] = igy[k] = 0;
        if (lx < 0) continue;
        const int rx = i0 - 1 + lx, ry = j0 - 1 + ly;
        if (BC == BC_REFLECTING && (rx < 0 || rx >= G.nx || ry < 0 || ry >= G.ny)) continue;
        it1[k] = ly * HX1 + lx;
        it2[k] = (ly + 1) * HX2 + lx + 1;
        igx[k] = wrap_index<BC>(rx, G.nx);
        igy[k] = wrap_index<BC>(ry, G.ny);
    }

    // S34: q_n at the items and the accumulator at the output nodes, loaded
    // first so that their latency overlaps the staging below
    TA qn[NIT][5], av[R][5];
#pragma unroll
    for (int k = 0; k < NIT; k++)
#pragma unroll
        for (int f = 0; f < 5; f++) qn[k][f] = TA(0);
#pragma unroll
    for (int k = 0; k < R; k++)
#pragma unroll
        for (int f = 0; f < 5; f++) av[k][f] = TA(0);
    if constexpr (PAIR == FUSED_S34) {
#pragma unroll
        for (int k = 0; k < NIT; k++) {
            if (it1[k] < 0) continue;
            const IX c = (IX)igy[k] * (IX)G.nx + (IX)igx[k];
#pragma unroll
            for (int f = 0; f < 5; f++) qn[k][f] = plane_at<W32>(a.q, f, P, c);
        }
#pragma unroll
        for (int k = 0; k < R; k++) {
            const int gi = i0 + threadIdx.x, gj = j0 + threadIdx.y + k * THREADS_Y;
            if (gi >= G.nx || gj >= G.ny) continue;
            const IX c = (IX)gj * (IX)G.nx + (IX)gi;
#pragma unroll
            for (int f = 0; f < 5; f++) av[k][f] = plane_at<W32>(a.acc, f, P, c);
        }
    }

    // ---- phase 1: the pair's input on the tile grown by two nodes (every
    // load of this thread's share issued before any is used)
    if constexpr (kChecked) {
        for (int k = tid; k < L::NP2 * HN2 + NF_OPS * HN1; k += BLOCK_THREADS) sm[k] = poison<TC>();
        __syncthreads();
    }
    TC rv[NPER2][5], rb[NPER2];
    bool ok[NPER2];
#pragma unroll
    for (int k = 0; k < NPER2; k++) {
        const int t = tid + k * BLOCK_THREADS;
        ok[k] = false;
        if (t >= HN2) continue;
        const int gx = wrap_index<BC>(i0 - 2 + t % HX2, G.nx);
        const int gy = wrap_index<BC>(j0 - 2 + t / HX2, G.ny);
        if (kChecked && (gx < 0 || gx >= G.nx || gy < 0 || gy >= G.ny)) {
            bad |= FLAG_BOUNDS;
            continue;
        }
        ok[k] = true;
        const IX c = (IX)gy * (IX)G.nx + (IX)gx;
#pragma unroll
        for (int f = 0; f < 5; f++) rv[k][f] = (PAIR == FUSED_S12) ? cvt<TC>(plane_at<W32>(a.q, f, P, c)) : plane_at<W32>(a.X, f, P, c);
        rb[k] = a.b[c];
    }
#pragma unroll
    for (int k = 0; k < NPER2; k++) {
        if (!ok[k]) continue;
        const int t = tid + k * BLOCK_THREADS;
        bad |= h_flags(rv[k][0]);
        store_operands_factored<TC, HN2>(s2, t, rv[k][0], rv[k][1], rv[k][2], rv[k][3], rv[k][4], rb[k], G);
        s2[L::P2_ETA * HN2 + t] = rv[k][4];
        s2[L::P2_B * HN2 + t] = rb[k];
    }
    __syncthreads();

    // ---- phase 2: the first stage at the items: its slope, the second
    // stage's input (S12: Q2 = q_n + dt/2 k1; S34: Q4 = q_n + dt k3) and that
    // input's operands on the tile grown by one node
    TC k1[R][5];        // S12: k1 at the output nodes
    TA qk[R][5];        // S12: q_n at the output nodes
    TA a3[R][5];        // S34: acc + dt/3 k3 at the output nodes
#pragma unroll
    for (int k = 0; k < NIT; k++) {
        if (it1[k] < 0) continue;
        const int t2 = it2[k];
        TC kk[5];
        node_rhs<TC, BC, HX2, HN2, true>(s2, t2, igx[k], igy[k], G, kk);
        TA qv[5];
        if constexpr (PAIR == FUSED_S12) {
            qv[0] = cvt<TA>(s2[FP_H * HN2 + t2]);
            qv[1] = cvt<TA>(s2[FP_U * HN2 + t2]);
            qv[2] = cvt<TA>(s2[FP_V * HN2 + t2]);
            qv[3] = cvt<TA>(s2[FP_W * HN2 + t2]);
            qv[4] = cvt<TA>(s2[L::P2_ETA * HN2 + t2]);
        } else {
#pragma unroll
            for (int f = 0; f < 5; f++) qv[f] = qn[k][f];
        }
        const TA cq = (PAIR == FUSED_S12) ? a.c_q1 : a.c_q3;
        TC y[5];
#pragma unroll
        for (int f = 0; f < 5; f++) y[f] = stage_state<TC, TA>(cq, kk[f], cvt<TA>(kk[f]), qv[f]);
        bad |= h_flags(y[0]);
        store_operands_factored<TC, HN1>(s1, it1[k], y[0], y[1], y[2], y[3], y[4], s2[L::P2_B * HN2 + t2], G);
        if (k < R) {
#pragma unroll
            for (int f = 0; f < 5; f++) {
                if constexpr (PAIR == FUSED_S12) {
                    k1[k][f] = kk[f];
                    qk[k][f] = qv[f];
                } else {
                    a3[k][f] = fma_(a.c_a3, cvt<TA>(kk[f]), av[k][f]);
                }
            }
        }
    }
    __syncthreads();

    // ---- phase 3: the second stage at the output nodes
#pragma unroll
    for (int k = 0; k < R; k++) {
        const int gi = i0 + threadIdx.x, gj = j0 + threadIdx.y + k * THREADS_Y;
        if (gi >= G.nx || gj >= G.ny) continue;
        const int t1 = (threadIdx.y + k * THREADS_Y + 1) * HX1 + threadIdx.x + 1;
        TC kk[5];
        node_rhs<TC, BC, HX1, HN1, true>(s1, t1, gi, gj, G, kk);
        const IX c = (IX)gj * (IX)G.nx + (IX)gi;
#pragma unroll
        for (int f = 0; f < 5; f++) {
            const TA kv = cvt<TA>(kk[f]);
            if constexpr (PAIR == FUSED_S12) {
                // as S2K: acc = (q_n + dt/6 k1) + dt/3 k2, Q3 = q_n + dt/2 k2
                plane_at<W32>(a.acc, f, P, c) = fma_(a.c_a2, kv, fma_(a.c_a1, cvt<TA>(k1[k][f]), qk[k][f]));
                plane_at<W32>(a.Qout, f, P, c) = stage_state<TC, TA>(a.c_q2, kk[f], kv, qk[k][f]);
            } else {
                // as S4: q_{n+1} = (acc + dt/3 k3) + dt/6 k4
                plane_at<W32>(a.out, f, P, c) = fma_(a.c_a4, kv, a3[k][f]);
            }
        }
    }
    if (bad) atomicOr(a.flag, bad);
}

// The fused kernels: registers for four resident blocks per SM (their shared
// memory, 48 KB at 32 x 16 tiles, allows four), except the reflecting S34,
// which would spill under that bound and runs 4% faster with three.
template <int BC, int PAIR>
constexpr int kFusedMinBlocks = (BC == BC_REFLECTING && PAIR == FUSED_S34) ? 3 : 4;
template <typename TC, typename TA, int BC, int PAIR, int R, bool W32 = false>
__global__ void __launch_bounds__(BLOCK_THREADS, (kFusedMinBlocks<BC, PAIR>)) k_fused(FusedArgs<TC, TA> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fused_tile<TC, TA, BC, PAIR, R, W32>(a, a.G, blockIdx.x * TILE_X, blockIdx.y * (THREADS_Y * R),
                                    reinterpret_cast<TC*>(smem_raw));
}

}  // namespace sgn
