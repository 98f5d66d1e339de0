// sgn_p5.cuh - stage kernels of the five-stage third-order FSAL pair used by
// the adaptive integrator (Sec. 6 names an explicit third-order five-stage
// pair with the first-same-as-last property and an embedded error estimator,
// optimized for stability-limited hyperbolic problems, without printing it;
// the coefficients, constructed for this library, are in sgn_api.cu).
//
// The pair's Butcher matrix has the two-register form a_ij = b_j for j < i-1,
// so with U_i = q_n + dt sum_{j<i} b_j k_j (U_1 = q_n) the stages are
//   Y_{i+1} = U_i + dt a_{i+1,i} k_i,   U_{i+1} = U_i + dt b_i k_i,
//   q_{n+1} = U_5 + dt b_5 k_5,          k6 = f(q_{n+1})  (the next k1),
// and the error estimate e = dt sum_{i<=6} (b_i - bhat_i) k_i is carried as
// E_i = sum_{j<i} (b_j - bhat_j) k_j.  Only k1 (and k6) are stored; k2..k5
// live in registers for one epilogue each.  Five launches per attempt, each
// the halo-tile RHS evaluation of k_stage (same operands, same node_rhs) with
// its own load and epilogue:
//   P5_S2    stages Y2 = q_n + dt a21 k1 (formed while loading the tile);
//            writes Y3, U3 = U2 + dt b2 k2 with U2 = q_n + dt b1 k1, and E3;
//   P5_MID   (stages 3 and 4) stages Y_i; writes Y_{i+1}, U_{i+1}, E_{i+1};
//   P5_S5    stages Y5; writes q_{n+1} (double) and E6;
//   P5_FSAL  stages q_{n+1}; writes k6 and the per-block sum of
//            (dt (E6 + (0 - bhat6) k6) / (atol + rtol max(|q_n|, |q_{n+1}|)))^2
//            (fixed order; the host takes the root mean square).
// Compute type FP64 or df64 (float pairs): k1, k6, the stage inputs Y, the
// accumulator U and E are stored in the compute type (8 bytes either way);
// q_n, q_{n+1} and the error norm are double.
#pragma once

#include "sgn_kernels.cuh"

namespace sgn {

enum { P5_S2 = 0, P5_MID = 1, P5_S5 = 2, P5_FSAL = 3 };

struct P5Args {
    const double* q;       // q_n (5 planes)
    const void* k1;        // f(q_n)                      (compute type)
    const void* Yin;       // P5_MID, P5_S5: stage input  (compute type)
    void* Yout;            // P5_S2, P5_MID: next stage input
    void* U;               // accumulator U_i             (compute type)
    void* E;               // error combination E_i       (compute type)
    double* q1;            // q_{n+1}: written by P5_S5, staged by P5_FSAL
    const void* b;         // bathymetry in the compute type
    void* kout;            // P5_FSAL: k6
    double* partials;      // P5_FSAL: NDIAG doubles per block, the sum in slot 0
    int* flag;
    Geom G;
    double c_in;           // P5_S2: dt a21
    double c_u1, c_e1;     // P5_S2: dt b1, b1 - bhat1 (the k1 terms)
    double c_y, c_u, c_e;  // this stage: dt a_{i+1,i}, dt b_i, b_i - bhat_i
    double c_e6, dt;       // P5_FSAL: 0 - bhat6, dt
    double rtol, atol;
};

// The stage input of one node, in the compute type.
template <typename TC, int MODE>
__device__ __forceinline__ void p5_input(const P5Args& a, long long c, long long P, TC c_in, TC y[5]) {
    const TC* __restrict__ k1 = static_cast<const TC*>(a.k1);
    const TC* __restrict__ Yin = static_cast<const TC*>(a.Yin);
#pragma unroll
    for (int f = 0; f < 5; f++) {
        const long long o = f * P + c;
        if (MODE == P5_S2) y[f] = fma_(c_in, k1[o], cvt<TC>(a.q[o]));
        else if (MODE == P5_FSAL) y[f] = cvt<TC>(a.q1[o]);
        else y[f] = Yin[o];
    }
}

// R: rows per thread (tile height 8 R): the compute type's StageShape, or
// for FP64 the context's height (32 x 8, 32 x 16 or 32 x 24, see sgn_create).
template <typename TC, int BC, int MODE, int R = StageShape<TC>::rows>
__global__ void __launch_bounds__(BLOCK_THREADS, StageShape<TC>::min_blocks) k_p5_stage(P5Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TC* sm = reinterpret_cast<TC*>(smem_raw);
    constexpr int HX = TILE_X + 2, HN = HX * (THREADS_Y * R + 2);
    const Geom& G = a.G;
    const long long P = G.plane;
    const int i0 = blockIdx.x * TILE_X, j0 = blockIdx.y * (THREADS_Y * R);
    const int tid = threadIdx.y * TILE_X + threadIdx.x;
    const TC* __restrict__ bT = static_cast<const TC*>(a.b);

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
                const long long o = f * P + c;
                if (MODE == P5_S2) {
                    ka[k][f] = static_cast<const TC*>(a.k1)[o];
                    qa[k][f] = a.q[o];
                } else if (MODE == P5_FSAL) {
                    qa[k][f] = a.q1[o];
                } else {
                    ka[k][f] = static_cast<const TC*>(a.Yin)[o];
                }
            }
            bv[k] = bT[c];
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
                y[f] = (MODE == P5_S2)     ? fma_(c_in, ka[k][f], cvt<TC>(qa[k][f]))
                       : (MODE == P5_FSAL) ? cvt<TC>(qa[k][f])
                                           : ka[k][f];
            bad |= h_flags(y[0]);
            store_operands<TC, HN>(sm, t, y[0], y[1], y[2], y[3], y[4], bv[k], G);
        }
    } else {
        for (int t = tid; t < HN; t += BLOCK_THREADS) {
            const int gx = halo_index<BC>(i0 - 1 + t % HX, G.nx);
            const int gy = halo_index<BC>(j0 - 1 + t / HX, G.ny);
            if (kChecked && (gx < 0 || gx >= G.nx || gy < 0 || gy >= G.ny)) {
                bad |= FLAG_BOUNDS;
                continue;
            }
            const long long c = (long long)gy * G.nx + gx;
            TC y[5];
            p5_input<TC, MODE>(a, c, P, c_in, y);
            bad |= h_flags(y[0]);
            store_operands<TC, HN>(sm, t, y[0], y[1], y[2], y[3], y[4], bT[c], G);
        }
    }
    if (bad) atomicOr(a.flag, bad);
    __syncthreads();

    // ---- phase 2: k at this thread's nodes and the stage epilogue
    const TC* __restrict__ k1 = static_cast<const TC*>(a.k1);
    TC* __restrict__ Yout = static_cast<TC*>(a.Yout);
    TC* __restrict__ U = static_cast<TC*>(a.U);
    TC* __restrict__ E = static_cast<TC*>(a.E);
    TC* __restrict__ kout = static_cast<TC*>(a.kout);
    const TC c_u1 = cvt<TC>(a.c_u1), c_e1 = cvt<TC>(a.c_e1);
    const TC c_y = cvt<TC>(a.c_y), c_u = cvt<TC>(a.c_u), c_e = cvt<TC>(a.c_e), c_e6 = cvt<TC>(a.c_e6);
    double esum = 0.0;
    const int gi = i0 + threadIdx.x;
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
            if (MODE == P5_S2) {
                const TC k1v = k1[o];
                const TC u2 = fma_(c_u1, k1v, cvt<TC>(a.q[o]));       // U2 = q_n + dt b1 k1
                Yout[o] = fma_(c_y, k[f], u2);
                U[o] = fma_(c_u, k[f], u2);
                E[o] = fma_(c_e, k[f], mul_(c_e1, k1v));
            } else if (MODE == P5_MID) {
                const TC uv = U[o];
                Yout[o] = fma_(c_y, k[f], uv);
                U[o] = fma_(c_u, k[f], uv);
                E[o] = fma_(c_e, k[f], E[o]);
            } else if (MODE == P5_S5) {
                a.q1[o] = cvt<double>(fma_(c_u, k[f], U[o]));
                E[o] = fma_(c_e, k[f], E[o]);
            } else {
                kout[o] = k[f];
                const double e = mul_(a.dt, cvt<double>(fma_(c_e6, k[f], E[o])));
                const double sc = fma_(a.rtol, fmax(fabs(a.q[o]), fabs(a.q1[o])), a.atol);
                const double r = mul_(e, recip<double>(sc));
                esum = fma_(r, r, esum);
            }
        }
    }

    if (MODE == P5_FSAL) {
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
