// sgn_rrk.cuh - relaxation Runge-Kutta: the energy-conserving scaling of an
// RK4 update (the paper names relaxation RK as future work; its energy is the
// 1^T M E of Thm. 4.1 / 4.2).
//
// With q the state at t_n and q1 its plain RK4 update, d = q1 - q, the relaxed
// step is q + gamma d with gamma the root near 1 of E(q + gamma d) = E(q).  Per
// node the energy change is, exactly (x' = x + gamma dx for every field),
//   E(q + gamma d) - E(q) = gamma (a1 + gamma a2 + gamma^2 a3)
//                         + gamma lam/6 (n0 + gamma n1) / (h (h + gamma dh))
// with s0 = (u^2+v^2)/2 + w^2/6, s1 = u du + v dv + w dw/3,
// s2 = (du^2+dv^2)/2 + dw^2/6, a1 = h s1 + dh s0 + g dh (h+b),
// a2 = h s2 + dh s1 + g/2 dh^2, a3 = dh s2, A = eta - h, al = deta - dh,
// n0 = 2 A al h - A^2 dh, n1 = al^2 h: no term is a difference of two
// energies, so the root is found without cancellation.  k_rrk_sums reduces, per
// block and in a fixed order, M times
//   a1, a2, a3 and the value, first and second gamma-derivative terms of the
//   rational part expanded about gamma_c: with D = h + gamma_c dh,
//   rho = dh / D, F0 = n0 + gamma_c n1,
//   lam/6 F0/(h D),  lam/6 (n1 - F0 rho)/(h D),  lam/6 (F0 rho^2 - n1 rho)/(h D)
// (the expansion in tau = gamma - gamma_c drops O(tau^3 rho^2) terms; the host
// re-centres when |gamma - gamma_c| > 1e-3).  A fixed grid of RRK_GRID blocks:
// each thread accumulates its strided nodes, then the block sums its threads
// in a fixed order (one partial per block).  k_rrk_update writes q + gamma d.
#pragma once

#include "sgn_kernels.cuh"

namespace sgn {

constexpr int NRRK = 6;
constexpr int RRK_BLOCK = 256;
constexpr int RRK_GRID = 148 * 4;     // a fixed grid: every thread sums a strided set of nodes

template <int BC>
__global__ void __launch_bounds__(RRK_BLOCK) k_rrk_sums(const double* __restrict__ q, const double* __restrict__ q1,
                                                        const double* __restrict__ b, Geom G, double gamma_c,
                                                        double* __restrict__ partials) {
    const long long P = G.plane;
    double s[NRRK] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long c = (long long)blockIdx.x * RRK_BLOCK + threadIdx.x; c < P;
         c += (long long)RRK_GRID * RRK_BLOCK) {
        const int j = (int)(c / G.nx), i = (int)(c - (long long)j * G.nx);
        double wx = G.dx, wy = G.dy;
        if (BC == BC_REFLECTING) {
            if (i == 0 || i == G.nx - 1) wx = 0.5 * wx;
            if (j == 0 || j == G.ny - 1) wy = 0.5 * wy;
        }
        const double M = wx * wy;
        const double h = q[c], u = q[P + c], v = q[2 * P + c], w = q[3 * P + c], eta = q[4 * P + c];
        const double dh = q1[c] - h, du = q1[P + c] - u, dv = q1[2 * P + c] - v;
        const double dw = q1[3 * P + c] - w, de = q1[4 * P + c] - eta;
        const double bb = b[c];
        const double s0 = fma(0.5 * u, u, fma(0.5 * v, v, w * w * (1.0 / 6.0)));
        const double s1 = fma(u, du, fma(v, dv, w * dw * (1.0 / 3.0)));
        const double s2 = fma(0.5 * du, du, fma(0.5 * dv, dv, dw * dw * (1.0 / 6.0)));
        const double a1 = fma(h, s1, dh * fma(G.g, h + bb, s0));
        const double a2 = fma(h, s2, dh * fma(0.5 * G.g, dh, s1));
        const double a3 = dh * s2;
        const double A = eta - h, al = de - dh;
        const double n0 = A * fma(2.0 * al, h, -A * dh), n1 = al * al * h;
        const double D = fma(gamma_c, dh, h);
        const double rD = recip<double>(h * D);        // 1 / (h D)
        const double rho = dh * h * rD;                  // dh / D
        const double F0 = fma(gamma_c, n1, n0);
        s[0] = fma(M, a1, s[0]);
        s[1] = fma(M, a2, s[1]);
        s[2] = fma(M, a3, s[2]);
        const double ml = M * G.lam6 * rD;
        s[3] = fma(ml, F0, s[3]);
        s[4] = fma(ml, fma(-F0, rho, n1), s[4]);
        s[5] = fma(ml * rho, fma(F0, rho, -n1), s[5]);
    }
    // fixed-order block sum: warp shuffle, then thread q over the warps
    __shared__ double red[RRK_BLOCK / 32][NRRK];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NRRK; k++) {
        double x = s[k];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) red[warp][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < NRRK) {
        double x = 0.0;
        for (int wg = 0; wg < RRK_BLOCK / 32; wg++) x += red[wg][threadIdx.x];
        partials[(long long)blockIdx.x * NRRK + threadIdx.x] = x;
    }
}

// Sums of the per-block partials in a fixed order (one block).
static __global__ void __launch_bounds__(256) k_rrk_reduce(const double* __restrict__ partials, long long nblk,
                                                           double* __restrict__ out) {
    __shared__ double red[256][NRRK];
    double s[NRRK] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long k = threadIdx.x; k < nblk; k += 256)
#pragma unroll
        for (int q = 0; q < NRRK; q++) s[q] += partials[k * NRRK + q];
#pragma unroll
    for (int q = 0; q < NRRK; q++) red[threadIdx.x][q] = s[q];
    __syncthreads();
    for (int stride = 128; stride > 0; stride >>= 1) {
        if ((int)threadIdx.x < stride)
#pragma unroll
            for (int q = 0; q < NRRK; q++) red[threadIdx.x][q] += red[threadIdx.x + stride][q];
        __syncthreads();
    }
    if (threadIdx.x < NRRK) out[threadIdx.x] = red[0][threadIdx.x];
}

// q <- q + gamma (q1 - q), five planes.
static __global__ void __launch_bounds__(256) k_rrk_update(double* __restrict__ q, const double* __restrict__ q1,
                                                           double gamma, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const double x = q[k];
        q[k] = fma(gamma, q1[k] - x, x);
    }
}

}  // namespace sgn
