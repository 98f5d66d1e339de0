// sgn_adjoint.cuh - the exact discrete adjoint (vector-Jacobian product) of the
// split-form SBP right-hand side and of one classical RK4 step.  The paper has
// no adjoint; this is the transpose of the Jacobian of the RHS of
// eq. (sd_periodic_2D_SGN) / eq. (semi_2D) as the forward kernels evaluate it.
//
// Structure.  At node c the RHS is  k_f(c) = sum_t coef_{f,t}(q_c, b_c) (D P_t)(c)
// + pointwise_f(q_c), where P_t are the differentiated products of the forward
// kernel and every coefficient depends on node c only.  So for a cotangent a:
//   - "pointwise" part: d k_f / d q_c with every D P_t held fixed (needs the
//     differences at c);
//   - "product" part: P̄_t(n) = sum_c D_{c,n} V_t(c) with
//     V_t(c) = sum_f a_f(c) coef_{f,t}(c), a gather over the rows c of the SBP
//     operator that touch column n (periodic: V(n-1) - V(n+1); reflecting: the
//     one-sided end rows add their own node), followed by the chain rule
//     through P_t(q_n, b_n).
// The gather form writes each output node once: no atomics.
//
// One 32x8 tile per 256-thread block (one node per thread), halo 1.  Shared
// memory: products and 1/h (16 planes), the cotangent (5) and one set of 12
// direction weights V (x first, then reused for y): 33 planes of 34x10 doubles.
#pragma once

#include "sgn_kernels.cuh"

namespace sgn {

constexpr int ADJ_TX = 32;
constexpr int ADJ_TY = 8;
constexpr int ADJ_HX = ADJ_TX + 2;
constexpr int ADJ_HY = ADJ_TY + 2;
constexpr int ADJ_HN = ADJ_HX * ADJ_HY;
constexpr int ADJ_THREADS = ADJ_TX * ADJ_TY;
constexpr int ADJ_A = N_OPS;            // first cotangent plane
constexpr int ADJ_V = N_OPS + 5;        // first direction-weight plane
constexpr int ADJ_PLANES = N_OPS + 5 + 12;

// direction-weight slots: x uses {H,U,V,W,ETA,B,HS,UU,HU,HUV,HUW,E2H},
// y uses {H,U,V,W,ETA,B,HS,VV,HV,HUV,HVW,E2H}; slot 7..10 differ
enum { VW_H, VW_U, VW_V, VW_W, VW_ETA, VW_B, VW_HS, VW_SQ, VW_HM, VW_HUV, VW_HMW, VW_E2H };

enum { ADJ_MODE_RHS = 0, ADJ_MODE_STAGE = 1 };

struct AdjArgs {
    const double* X;       // state at which the Jacobian is taken (5 planes)
    const double* b;       // bathymetry
    const double* A;       // cotangent (5 planes), used as a_scale * A
    double a_scale;
    double* qbar;          // RHS mode: output J^T a (5 planes)
    double* bbar;          // accumulated (1 plane)
    // stage mode: Qbar = J^T a;  qacc_out = (first ? qprime : qacc_in) + Qbar;
    //             Anext = c_prime * qprime + c_bar * Qbar (when Anext != nullptr)
    const double* qprime;
    const double* qacc_in;
    double* qacc_out;
    double* Anext;
    double c_prime, c_bar;
    int first;
    Geom G;
};

// Direction weights V_t(c) (see the header comment) at the node in slot t of the
// halo tile, for the x (DIR = 0) or y (DIR = 1) differences, scaled by the row
// factor s (1/(2 dx) inside, 1/dx on a reflecting end row).
template <int DIR>
__device__ __forceinline__ void dir_weights(const double* __restrict__ sm, int t, double s,
                                            const Geom& G, double* __restrict__ out) {
    const double h = sm[OP_H * ADJ_HN + t], u = sm[OP_U * ADJ_HN + t], v = sm[OP_V * ADJ_HN + t];
    const double w = sm[OP_W * ADJ_HN + t], eta = sm[OP_ETA * ADJ_HN + t], bb = sm[OP_B * ADJ_HN + t];
    const double r = sm[OP_R * ADJ_HN + t];
    const double ah = sm[(ADJ_A + 0) * ADJ_HN + t], au = sm[(ADJ_A + 1) * ADJ_HN + t];
    const double av = sm[(ADJ_A + 2) * ADJ_HN + t], aw = sm[(ADJ_A + 3) * ADJ_HN + t];
    const double ae = sm[(ADJ_A + 4) * ADJ_HN + t];
    const double rho = eta * r, om = 1.0 - rho, sfs = h + bb;
    const double ru = -r * au, rv = -r * av, rw = -0.5 * r * aw;   // d k / d B for u, v, w
    const double hu = h * u, hv = h * v, hw = h * w;
    if (DIR == 0) {
        const double C1 = G.lam6 * rho * rho - G.g * sfs - 0.5 * u * u;
        out[VW_H] = s * (-u * ah + ru * C1 - 0.5 * rv * u * v - rw * u * w);
        out[VW_U] = s * (-h * ah - 0.5 * ru * hu - 0.5 * rv * hv - rw * hw);
        out[VW_V] = s * (0.5 * rv * hu);
        out[VW_W] = s * (rw * hu);
        out[VW_ETA] = s * (ru * G.lam3 * om - u * ae);
        out[VW_B] = s * (ru * G.lam2 * om - 1.5 * u * ae);
        out[VW_HS] = s * (ru * G.g);
        out[VW_SQ] = s * (0.5 * ru * h);    // u^2
        out[VW_HM] = s * (0.5 * ru * u);    // hu
        out[VW_HUV] = s * (0.5 * rv);
        out[VW_HMW] = s * rw;               // huw
        out[VW_E2H] = s * (-G.lam6 * ru);
    } else {
        const double C2 = G.lam6 * rho * rho - G.g * sfs - 0.5 * v * v;
        out[VW_H] = s * (-v * ah + rv * C2 - 0.5 * ru * u * v - rw * v * w);
        out[VW_V] = s * (-h * ah - 0.5 * rv * hv - 0.5 * ru * hu - rw * hw);
        out[VW_U] = s * (0.5 * ru * hv);
        out[VW_W] = s * (rw * hv);
        out[VW_ETA] = s * (rv * G.lam3 * om - v * ae);
        out[VW_B] = s * (rv * G.lam2 * om - 1.5 * v * ae);
        out[VW_HS] = s * (rv * G.g);
        out[VW_SQ] = s * (0.5 * rv * h);    // v^2
        out[VW_HM] = s * (0.5 * rv * v);    // hv
        out[VW_HUV] = s * (0.5 * ru);
        out[VW_HMW] = s * rw;               // hvw
        out[VW_E2H] = s * (-G.lam6 * rv);
    }
}

template <int BC>
__device__ __forceinline__ double row_scale(int k, int n, double c2, double c1) {
    if (BC == BC_REFLECTING && (k == 0 || k == n - 1)) return c1;
    return c2;
}

template <int BC, int MODE>
__global__ void __launch_bounds__(ADJ_THREADS)
k_adjoint(AdjArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sm = reinterpret_cast<double*>(smem_raw);
    const Geom& G = a.G;
    const int i0 = blockIdx.x * ADJ_TX, j0 = blockIdx.y * ADJ_TY;
    const long long P = G.plane;
    const int tid = threadIdx.y * ADJ_TX + threadIdx.x;

    // ---- phase 1: state, products, 1/h and the cotangent on the halo tile
    for (int t = tid; t < ADJ_HN; t += ADJ_THREADS) {
        const int li = t % ADJ_HX, lj = t / ADJ_HX;
        const int gi = halo_index<BC>(i0 - 1 + li, G.nx);
        const int gj = halo_index<BC>(j0 - 1 + lj, G.ny);
        const long long c = (long long)gj * G.nx + gi;
        const double h = a.X[c], u = a.X[P + c], v = a.X[2 * P + c], w = a.X[3 * P + c];
        const double eta = a.X[4 * P + c], bb = a.b[c];
        const double r = 1.0 / h, hu = h * u, hv = h * v;
        sm[OP_H * ADJ_HN + t] = h;
        sm[OP_U * ADJ_HN + t] = u;
        sm[OP_V * ADJ_HN + t] = v;
        sm[OP_W * ADJ_HN + t] = w;
        sm[OP_ETA * ADJ_HN + t] = eta;
        sm[OP_B * ADJ_HN + t] = bb;
        sm[OP_HS * ADJ_HN + t] = h * (h + bb);
        sm[OP_UU * ADJ_HN + t] = u * u;
        sm[OP_VV * ADJ_HN + t] = v * v;
        sm[OP_HU * ADJ_HN + t] = hu;
        sm[OP_HV * ADJ_HN + t] = hv;
        sm[OP_HUV * ADJ_HN + t] = hu * v;
        sm[OP_HUW * ADJ_HN + t] = hu * w;
        sm[OP_HVW * ADJ_HN + t] = hv * w;
        sm[OP_E2H * ADJ_HN + t] = eta * eta * r;
        sm[OP_R * ADJ_HN + t] = r;
#pragma unroll
        for (int f = 0; f < 5; f++) sm[(ADJ_A + f) * ADJ_HN + t] = a.a_scale * a.A[f * P + c];
    }
    __syncthreads();

    const int li = threadIdx.x + 1, lj = threadIdx.y + 1;
    const int gi = i0 + threadIdx.x, gj = j0 + threadIdx.y;
    const int t = lj * ADJ_HX + li;
    const bool active = gi < G.nx && gj < G.ny;
    // P̄ over the 15 product slots: h u v w eta b hs uu vv hu hv huv huw hvw e2h
    double pb[N_OPS - 1];
#pragma unroll
    for (int k = 0; k < N_OPS - 1; k++) pb[k] = 0.0;

    // ---- phases 2-3: x weights on the halo tile, then the x gather
    for (int tt = tid; tt < ADJ_HN; tt += ADJ_THREADS) {
        const int gx = halo_index<BC>(i0 - 1 + tt % ADJ_HX, G.nx);
        double vw[12];
        dir_weights<0>(sm, tt, row_scale<BC>(gx, G.nx, G.cx2, G.cx1), G, vw);
#pragma unroll
        for (int k = 0; k < 12; k++) sm[(ADJ_V + k) * ADJ_HN + tt] = vw[k];
    }
    __syncthreads();
    if (active) {
        // P̄(n) = V(n-1) - V(n+1) (periodic); reflecting: V(n-1) if n >= 1,
        // -V(n+1) if n <= N-2, +V(n) on the last row, -V(n) on the first row.
        const bool has_l = BC == BC_PERIODIC || gi >= 1;
        const bool has_r = BC == BC_PERIODIC || gi <= G.nx - 2;
        const double self = (BC == BC_REFLECTING) ? ((gi == G.nx - 1 ? 1.0 : 0.0) - (gi == 0 ? 1.0 : 0.0)) : 0.0;
        const int slot_of[12] = {OP_H, OP_U, OP_V, OP_W, OP_ETA, OP_B, OP_HS, OP_UU, OP_HU, OP_HUV, OP_HUW, OP_E2H};
#pragma unroll
        for (int k = 0; k < 12; k++) {
            const double* V = sm + (ADJ_V + k) * ADJ_HN;
            double g = self * V[t];
            if (has_l) g += V[t - 1];
            if (has_r) g -= V[t + 1];
            pb[slot_of[k]] += g;
        }
    }
    __syncthreads();

    // ---- phases 4-5: y weights, then the y gather
    for (int tt = tid; tt < ADJ_HN; tt += ADJ_THREADS) {
        const int gy = halo_index<BC>(j0 - 1 + tt / ADJ_HX, G.ny);
        double vw[12];
        dir_weights<1>(sm, tt, row_scale<BC>(gy, G.ny, G.cy2, G.cy1), G, vw);
#pragma unroll
        for (int k = 0; k < 12; k++) sm[(ADJ_V + k) * ADJ_HN + tt] = vw[k];
    }
    __syncthreads();
    if (!active) return;
    {
        const bool has_b = BC == BC_PERIODIC || gj >= 1;
        const bool has_t = BC == BC_PERIODIC || gj <= G.ny - 2;
        const double self = (BC == BC_REFLECTING) ? ((gj == G.ny - 1 ? 1.0 : 0.0) - (gj == 0 ? 1.0 : 0.0)) : 0.0;
        const int slot_of[12] = {OP_H, OP_U, OP_V, OP_W, OP_ETA, OP_B, OP_HS, OP_VV, OP_HV, OP_HUV, OP_HVW, OP_E2H};
#pragma unroll
        for (int k = 0; k < 12; k++) {
            const double* V = sm + (ADJ_V + k) * ADJ_HN;
            double g = self * V[t];
            if (has_b) g += V[t - ADJ_HX];
            if (has_t) g -= V[t + ADJ_HX];
            pb[slot_of[k]] += g;
        }
    }

    // ---- pointwise part: d k / d q at this node with every difference fixed
    int tl = t - 1, tr = t + 1, tb = t - ADJ_HX, tu = t + ADJ_HX;
    double sx = G.cx2, sy = G.cy2, sgx = 0.0, sgy = 0.0;
    if (BC == BC_REFLECTING) {
        if (gi == 0) { tl = t; sx = G.cx1; sgx = -G.satx; }
        if (gi == G.nx - 1) { tr = t; sx = G.cx1; sgx = G.satx; }
        if (gj == 0) { tb = t; sy = G.cy1; sgy = -G.saty; }
        if (gj == G.ny - 1) { tu = t; sy = G.cy1; sgy = G.saty; }
    }
#define DX_(op) (sx * (sm[(op) * ADJ_HN + tr] - sm[(op) * ADJ_HN + tl]))
#define DY_(op) (sy * (sm[(op) * ADJ_HN + tu] - sm[(op) * ADJ_HN + tb]))
    const double h = sm[OP_H * ADJ_HN + t], u = sm[OP_U * ADJ_HN + t], v = sm[OP_V * ADJ_HN + t];
    const double w = sm[OP_W * ADJ_HN + t], eta = sm[OP_ETA * ADJ_HN + t], bb = sm[OP_B * ADJ_HN + t];
    const double r = sm[OP_R * ADJ_HN + t];
    const double ah = sm[(ADJ_A + 0) * ADJ_HN + t], au = sm[(ADJ_A + 1) * ADJ_HN + t];
    const double av = sm[(ADJ_A + 2) * ADJ_HN + t], aw = sm[(ADJ_A + 3) * ADJ_HN + t];
    const double ae = sm[(ADJ_A + 4) * ADJ_HN + t];
    const double rho = eta * r, om = 1.0 - rho, sfs = h + bb;
    const double hu = h * u, hv = h * v, hw = h * w, uv = u * v, uw = u * w, vw_ = v * w;
    const double xh = DX_(OP_H), xu = DX_(OP_U), xv = DX_(OP_V), xw = DX_(OP_W), xe = DX_(OP_ETA), xb = DX_(OP_B);
    const double yh = DY_(OP_H), yu = DY_(OP_U), yv = DY_(OP_V), yw = DY_(OP_W), ye = DY_(OP_ETA), yb = DY_(OP_B);
    const double xhs = DX_(OP_HS), xuu = DX_(OP_UU), xhu = DX_(OP_HU), xhuv = DX_(OP_HUV), xhuw = DX_(OP_HUW);
    const double xe2h = DX_(OP_E2H);
    const double yhs = DY_(OP_HS), yvv = DY_(OP_VV), yhv = DY_(OP_HV), yhuv = DY_(OP_HUV), yhvw = DY_(OP_HVW);
    const double ye2h = DY_(OP_E2H);
#undef DX_
#undef DY_
    const double C1 = G.lam6 * rho * rho - G.g * sfs - 0.5 * u * u;
    const double C2 = G.lam6 * rho * rho - G.g * sfs - 0.5 * v * v;
    const double Bu = xh * C1 + xe * G.lam3 * om + xb * G.lam2 * om + G.g * xhs + 0.5 * h * xuu
                    + 0.5 * u * xhu - 0.5 * hu * xu - G.lam6 * xe2h
                    + 0.5 * (yhuv - uv * yh + hv * yu - hu * yv);
    const double Bv = yh * C2 + ye * G.lam3 * om + yb * G.lam2 * om + G.g * yhs + 0.5 * h * yvv
                    + 0.5 * v * yhv - 0.5 * hv * yv - G.lam6 * ye2h
                    + 0.5 * (xhuv - uv * xh + hu * xv - hv * xu);
    const double Bw = G.lam * om - 0.5 * (xhuw + hu * xw - uw * xh - hw * xu
                                          + yhvw + hv * yw - vw_ * yh - hw * yv);
    const double ku = -r * Bu, kv = -r * Bv, kw = r * Bw;
    const double lr = G.lam3 * rho * r;   // d/dh and d/deta helpers
    const double dBu_dh = xh * (-G.lam3 * rho * rho * r - G.g) + xe * lr + xb * G.lam2 * rho * r
                        + 0.5 * xuu - 0.5 * u * xu + 0.5 * (v * yu - u * yv);
    const double dBv_dh = yh * (-G.lam3 * rho * rho * r - G.g) + ye * lr + yb * G.lam2 * rho * r
                        + 0.5 * yvv - 0.5 * v * yv + 0.5 * (u * xv - v * xu);
    const double dBw_dh = G.lam * rho * r - 0.5 * (u * xw - w * xu + v * yw - w * yv);

    double hb = ah * (-(xu + yv) + sgx * u + sgy * v)
              + au * (-r * ku - r * dBu_dh) + av * (-r * kv - r * dBv_dh) + aw * (-r * kw + r * dBw_dh);
    double ub = ah * (-xh + sgx * h) - au * r * (-u * xh + 0.5 * xhu - 0.5 * h * xu - 0.5 * (v * yh + h * yv))
              - av * r * 0.5 * (-v * xh + h * xv) - aw * 0.5 * r * (h * xw - w * xh) - ae * (xe + 1.5 * xb);
    double vb = ah * (-yh + sgy * h) - au * r * 0.5 * (-u * yh + h * yu)
              - av * r * (-v * yh + 0.5 * yhv - 0.5 * h * yv - 0.5 * (u * xh + h * xu))
              - aw * 0.5 * r * (h * yw - w * yh) - ae * (ye + 1.5 * yb);
    double wb = aw * 0.5 * r * (u * xh + h * xu + v * yh + h * yv) + ae;
    double eb = -au * r * (xh * lr - xe * G.lam3 * r - xb * G.lam2 * r)
              - av * r * (yh * lr - ye * G.lam3 * r - yb * G.lam2 * r) - aw * G.lam * r * r;
    double bbar = r * G.g * (au * xh + av * yh);

    // ---- chain rule through the products
    hb += pb[OP_H] + (2.0 * h + bb) * pb[OP_HS] + u * pb[OP_HU] + v * pb[OP_HV] + uv * pb[OP_HUV]
        + uw * pb[OP_HUW] + vw_ * pb[OP_HVW] - rho * rho * pb[OP_E2H];
    ub += pb[OP_U] + 2.0 * u * pb[OP_UU] + h * pb[OP_HU] + hv * pb[OP_HUV] + hw * pb[OP_HUW];
    vb += pb[OP_V] + 2.0 * v * pb[OP_VV] + h * pb[OP_HV] + hu * pb[OP_HUV] + hw * pb[OP_HVW];
    wb += pb[OP_W] + hu * pb[OP_HUW] + hv * pb[OP_HVW];
    eb += pb[OP_ETA] + 2.0 * rho * pb[OP_E2H];
    bbar += pb[OP_B] + h * pb[OP_HS];

    const long long c = (long long)gj * G.nx + gi;
    const double qb[5] = {hb, ub, vb, wb, eb};
    a.bbar[c] += bbar;
    if (MODE == ADJ_MODE_RHS) {
#pragma unroll
        for (int f = 0; f < 5; f++) a.qbar[f * P + c] = qb[f];
    } else {
#pragma unroll
        for (int f = 0; f < 5; f++) {
            const double base = a.first ? a.qprime[f * P + c] : a.qacc_in[f * P + c];
            a.qacc_out[f * P + c] = base + qb[f];
            if (a.Anext) a.Anext[f * P + c] = a.c_prime * a.qprime[f * P + c] + a.c_bar * qb[f];
        }
    }
}

}  // namespace sgn
