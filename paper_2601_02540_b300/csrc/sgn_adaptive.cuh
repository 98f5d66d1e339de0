// sgn_adaptive.cuh - stage kernels of the adaptive integrator's second pair.
//
// The paper advances the semi-discretization (eq. (sd_periodic_2D_SGN) /
// eq. (semi_2D)) with an explicit third-order, five-stage Runge-Kutta pair
// that has the first-same-as-last (FSAL) property, an embedded error estimate
// and automatic step-size control (Sec. 6); it does not print the pair.  The
// five-stage pair of that kind is in sgn_p5.cuh; this file holds the second
// pair sgn_step_adaptive offers (SGN_PAIR_BS3), the Bogacki-Shampine 3(2) pair:
//   k1 = f(q_n)                      (the k4 of the previous accepted step)
//   k2 = f(Y2),  Y2 = q_n + dt/2 k1
//   k3 = f(Y3),  Y3 = q_n + 3dt/4 k2
//   q1 = q_n + dt (2/9 k1 + 1/3 k2 + 4/9 k3),  k4 = f(q1)
//   e  = dt (-5/72 k1 + 1/12 k2 + 1/9 k3 - 1/8 k4)   (third minus second order)
// Three launches per attempt, each the halo-tile RHS evaluation of k_stage
// (same operands, same node_rhs) with its own load and epilogue:
//   BS_K2  forms Y2 = q_n + c_in k1 while staging the halo tile, writes k2 and
//          Y3 = q_n + c_y k2 at its nodes;
//   BS_K3  stages Y3, writes k3 and q1 = q_n + cb1 k1 + cb2 k2 + cb3 k3;
//   BS_K4  stages q1, writes k4 and the per-block sum of
//          (e / (atol + rtol max(|q_n|, |q1|)))^2 over its nodes and fields
//          (fixed-order reduction; the host takes the root mean square).
// Compute type FP64 or df64 (float pairs); the state, the stage slopes and the
// error arithmetic are double in both.
#pragma once

#include "sgn_kernels.cuh"

namespace sgn {

enum { BS_K2 = 0, BS_K3 = 1, BS_K4 = 2 };

struct BsArgs {
    const double* q;       // q_n (5 planes, double)
    const void* k1;        // f(q_n)            (compute type)
    const void* k2;        // BS_K3, BS_K4      (compute type)
    const void* k3;        // BS_K4             (compute type)
    void* Y3;              // written by BS_K2, staged by BS_K3 (compute type)
    double* q1;            // written by BS_K3, staged by BS_K4 (double: the candidate state)
    const void* b;         // bathymetry in the compute type
    void* kout;            // this stage's k    (compute type)
    double* partials;      // BS_K4: NDIAG doubles per block, the sum in slot 0
    int* flag;
    Geom G;
    double c_in, c_y;              // dt/2, 3dt/4
    double cb1, cb2, cb3;          // dt b1, dt b2, dt b3
    double ce1, ce2, ce3, ce4;     // dt (b_i - bhat_i)
    double rtol, atol;
};

// TC: compute type of the RHS (double, or df64 with the float-pair stage
// arithmetic).  The slopes and Y3 are stored in the compute type (a float pair
// takes 8 bytes, like a double); the state q_n and the candidate q1 in double.
// R: rows per thread (tile height 8 R): the compute type's StageShape, or for
// FP64 the context's height.
template <typename TC, int BC, int MODE, int R = StageShape<TC>::rows>
__global__ void __launch_bounds__(BLOCK_THREADS, StageShape<TC>::min_blocks) k_bs3_stage(BsArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TC* sm = reinterpret_cast<TC*>(smem_raw);
    constexpr int HX = TILE_X + 2, HN = HX * (THREADS_Y * R + 2);
    const Geom& G = a.G;
    const long long P = G.plane;
    const int i0 = blockIdx.x * TILE_X, j0 = blockIdx.y * (THREADS_Y * R);
    const int tid = threadIdx.y * TILE_X + threadIdx.x;
    const TC* __restrict__ k1 = static_cast<const TC*>(a.k1);
    const TC* __restrict__ k2 = static_cast<const TC*>(a.k2);
    const TC* __restrict__ k3 = static_cast<const TC*>(a.k3);
    TC* __restrict__ kout = static_cast<TC*>(a.kout);
    TC* __restrict__ Y3 = static_cast<TC*>(a.Y3);

    // ---- phase 1: halo tile of the stage input and of its products
    int bad = 0;
    const TC c_in = cvt<TC>(a.c_in);
    if constexpr (kChecked) {                   // checked builds: poison the tile first
        for (int k = tid; k < N_OPS * HN; k += BLOCK_THREADS) sm[k] = poison<TC>();
        __syncthreads();
    }
    if constexpr (std::is_same<TC, df64>::value) {
        // df64 (bound by instruction issue): every load of the thread's share of
        // the tile is issued before the stage input is formed and staged
        constexpr int NPER = (HN + BLOCK_THREADS - 1) / BLOCK_THREADS;
        TC ka[NPER][5], bv[NPER];
        double qa[NPER][5];
#pragma unroll
        for (int k = 0; k < NPER; k++) {
            const int t = tid + k * BLOCK_THREADS;
            if (t >= HN) continue;
            const int gx = halo_index<BC>(i0 - 1 + t % HX, G.nx);
            const int gy = halo_index<BC>(j0 - 1 + t / HX, G.ny);
            if (kChecked && (gx < 0 || gx >= G.nx || gy < 0 || gy >= G.ny)) {
                bad |= FLAG_BOUNDS;
                continue;
            }
            const long long c = (long long)gy * G.nx + gx;
#pragma unroll
            for (int f = 0; f < 5; f++) {
                if (MODE == BS_K2) {
                    ka[k][f] = k1[f * P + c];
                    qa[k][f] = a.q[f * P + c];
                } else if (MODE == BS_K3) {
                    ka[k][f] = Y3[f * P + c];
                } else {
                    qa[k][f] = a.q1[f * P + c];
                }
            }
            bv[k] = static_cast<const TC*>(a.b)[c];
        }
#pragma unroll
        for (int k = 0; k < NPER; k++) {
            const int t = tid + k * BLOCK_THREADS;
            if (t >= HN) continue;
            if constexpr (kChecked) {
                const int gx = halo_index<BC>(i0 - 1 + t % HX, G.nx);
                const int gy = halo_index<BC>(j0 - 1 + t / HX, G.ny);
                if (gx < 0 || gx >= G.nx || gy < 0 || gy >= G.ny) continue;
            }
            TC y[5];
#pragma unroll
            for (int f = 0; f < 5; f++)
                y[f] = (MODE == BS_K2)   ? fma_(c_in, ka[k][f], cvt<TC>(qa[k][f]))
                       : (MODE == BS_K3) ? ka[k][f]
                                         : cvt<TC>(qa[k][f]);
            bad |= h_flags(y[0]);
            store_operands<TC, HN>(sm, t, y[0], y[1], y[2], y[3], y[4], bv[k], G);
        }
    } else {
        for (int t = tid; t < HN; t += BLOCK_THREADS) {
            const int li = t % HX, lj = t / HX;
            const int gx = halo_index<BC>(i0 - 1 + li, G.nx);
            const int gy = halo_index<BC>(j0 - 1 + lj, G.ny);
            if (kChecked && (gx < 0 || gx >= G.nx || gy < 0 || gy >= G.ny)) {
                bad |= FLAG_BOUNDS;
                continue;
            }
            const long long c = (long long)gy * G.nx + gx;
            TC y[5];
#pragma unroll
            for (int f = 0; f < 5; f++)
                y[f] = (MODE == BS_K2)   ? fma_(c_in, k1[f * P + c], cvt<TC>(a.q[f * P + c]))
                       : (MODE == BS_K3) ? Y3[f * P + c]
                                         : cvt<TC>(a.q1[f * P + c]);
            bad |= h_flags(y[0]);
            store_operands<TC, HN>(sm, t, y[0], y[1], y[2], y[3], y[4], static_cast<const TC*>(a.b)[c], G);
        }
    }
    if (bad) atomicOr(a.flag, bad);
    __syncthreads();

    // ---- phase 2: k at this thread's nodes and the stage epilogue
    double esum = 0.0;
    const int gi = i0 + threadIdx.x;
    const TC c_y = cvt<TC>(a.c_y), cb1 = cvt<TC>(a.cb1), cb2 = cvt<TC>(a.cb2), cb3 = cvt<TC>(a.cb3);
    const TC ce1 = cvt<TC>(a.ce1), ce2 = cvt<TC>(a.ce2), ce3 = cvt<TC>(a.ce3), ce4 = cvt<TC>(a.ce4);
#pragma unroll
    for (int ry = 0; ry < R; ry++) {
        const int ly = threadIdx.y + ry * THREADS_Y;
        const int gj = j0 + ly;
        if (gi >= G.nx || gj >= G.ny) continue;
        const int t = (ly + 1) * HX + (threadIdx.x + 1);
        TC k[5];
        node_rhs<TC, BC, HX, HN>(sm, t, gi, gj, G, k);
        const long long c = (long long)gj * G.nx + gi;
#pragma unroll
        for (int f = 0; f < 5; f++) {
            const long long o = f * P + c;
            kout[o] = k[f];
            if (MODE == BS_K2) {
                Y3[o] = fma_(c_y, k[f], cvt<TC>(a.q[o]));
            } else if (MODE == BS_K3) {
                a.q1[o] = cvt<double>(fma_(cb3, k[f], fma_(cb2, k2[o], fma_(cb1, k1[o], cvt<TC>(a.q[o])))));
            } else {
                const double e = cvt<double>(fma_(ce4, k[f], fma_(ce3, k3[o], fma_(ce2, k2[o], mul_(ce1, k1[o])))));
                const double q1 = a.q1[o];                // this node's stage input
                const double sc = fma_(a.rtol, fmax(fabs(a.q[o]), fabs(q1)), a.atol);
                const double r = mul_(e, recip<double>(sc));
                esum = fma_(r, r, esum);
            }
        }
    }

    if (MODE == BS_K4) {
        // fixed-order block sum: warp shuffle, then thread 0 over the warps
        __shared__ double red[BLOCK_THREADS / 32];
        const int lane = tid & 31, warp = tid >> 5;
        double x = esum;
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) red[warp] = x;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int wg = 0; wg < BLOCK_THREADS / 32; wg++) s += red[wg];
            double* slot = a.partials + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * NDIAG;
            slot[0] = s;
            slot[1] = 0.0;
            slot[2] = 0.0;
            slot[3] = 0.0;
        }
    }
}

}  // namespace sgn
