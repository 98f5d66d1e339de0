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
//     V_t(c) = sum_f a_f(c) coef_{f,t}(c) (the row factor of D included), a
//     gather over the rows c of the SBP operator that touch column n
//     (periodic: V(n-1) - V(n+1); reflecting: V(n-1) for n >= 1, -V(n+1) for
//     n <= N-2, and the one-sided end rows add +V(N-1) at n = N-1 and -V(0) at
//     n = 0), then the chain rule through P_t(q_n, b_n).
// Two passes, both one node per thread and free of halos and atomics:
//   k_adj_weights  products P_t, 1/h and the 24 direction weights of each node
//                  into scratch planes;
//   k_adj_gather   differences, pointwise part, gathers of the weights of the
//                  neighbours, chain rule, and (stage mode) the reverse RK4
//                  stage algebra.
#pragma once

#include "sgn_kernels.cuh"

namespace sgn {

// scratch layout (planes): products and 1/h (N_OPS), x weights (12), y weights (12)
constexpr int ADJ_WX = N_OPS;
constexpr int ADJ_WY = N_OPS + 12;
constexpr int ADJ_SCRATCH_PLANES = N_OPS + 24;
constexpr int ADJ_BLOCK = 256;

// weight slots: x uses {H,U,V,W,ETA,B,HS,UU,HU,HUV,HUW,E2H},
// y uses {H,U,V,W,ETA,B,HS,VV,HV,HUV,HVW,E2H}
enum { VW_H, VW_U, VW_V, VW_W, VW_ETA, VW_B, VW_HS, VW_SQ, VW_HM, VW_HUV, VW_HMW, VW_E2H };

enum { ADJ_MODE_RHS = 0, ADJ_MODE_STAGE = 1 };

struct AdjArgs {
    const double* X;       // state at which the Jacobian is taken (5 planes)
    const double* b;       // bathymetry
    const double* A;       // cotangent (5 planes), used as a_scale * A
    double a_scale;
    double* scratch;       // ADJ_SCRATCH_PLANES planes
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

template <int BC>
__device__ __forceinline__ double row_scale(int k, int n, double c2, double c1) {
    if (BC == BC_REFLECTING && (k == 0 || k == n - 1)) return c1;
    return c2;
}

// Pass 1: products, 1/h and the direction weights V^x, V^y of one node.
template <int BC>
__global__ void __launch_bounds__(ADJ_BLOCK) k_adj_weights(AdjArgs a) {
    const Geom& G = a.G;
    const long long P = G.plane;
    const long long c = (long long)blockIdx.x * ADJ_BLOCK + threadIdx.x;
    if (c >= P) return;
    const int j = (int)(c / G.nx), i = (int)(c - (long long)j * G.nx);
    const double h = a.X[c], u = a.X[P + c], v = a.X[2 * P + c], w = a.X[3 * P + c];
    const double eta = a.X[4 * P + c], bb = a.b[c];
    const double r = recip<double>(h);
    const double hu = h * u, hv = h * v, hw = h * w;
    double* S = a.scratch;
    S[OP_H * P + c] = h;
    S[OP_U * P + c] = u;
    S[OP_V * P + c] = v;
    S[OP_W * P + c] = w;
    S[OP_ETA * P + c] = eta;
    S[OP_B * P + c] = bb;
    S[OP_HS * P + c] = h * (h + bb);
    S[OP_UU * P + c] = u * u;
    S[OP_VV * P + c] = v * v;
    S[OP_HU * P + c] = hu;
    S[OP_HV * P + c] = hv;
    S[OP_HUV * P + c] = hu * v;
    S[OP_HUW * P + c] = hu * w;
    S[OP_HVW * P + c] = hv * w;
    S[OP_E2H * P + c] = eta * eta * r;
    S[OP_R * P + c] = r;

    const double s = a.a_scale;
    const double ah = s * a.A[c], au = s * a.A[P + c], av = s * a.A[2 * P + c];
    const double aw = s * a.A[3 * P + c], ae = s * a.A[4 * P + c];
    const double rho = eta * r, om = 1.0 - rho;
    const double cc = G.lam6 * rho * rho - G.g * (h + bb);   // common part of C1, C2
    const double ra = -r * au, rb = -r * av, rc = -0.5 * r * aw;  // d k / d B for u, v, w
    // x weights (row factor of column i)
    {
        const double sx = row_scale<BC>(i, G.nx, G.cx2, G.cx1);
        const double ru = sx * ra, rv = sx * rb, rw = sx * rc, sah = sx * ah, sae = sx * ae;
        double* W = S + ADJ_WX * P + c;
        W[VW_H * P] = -u * sah + ru * (cc - 0.5 * u * u) - 0.5 * rv * (u * v) - rw * (u * w);
        W[VW_U * P] = -h * sah - 0.5 * ru * hu - 0.5 * rv * hv - rw * hw;
        W[VW_V * P] = 0.5 * rv * hu;
        W[VW_W * P] = rw * hu;
        W[VW_ETA * P] = ru * G.lam3 * om - u * sae;
        W[VW_B * P] = ru * G.lam2 * om - 1.5 * u * sae;
        W[VW_HS * P] = ru * G.g;
        W[VW_SQ * P] = 0.5 * ru * h;      // u^2
        W[VW_HM * P] = 0.5 * ru * u;      // hu
        W[VW_HUV * P] = 0.5 * rv;
        W[VW_HMW * P] = rw;               // huw
        W[VW_E2H * P] = -G.lam6 * ru;
    }
    // y weights (row factor of row j)
    {
        const double sy = row_scale<BC>(j, G.ny, G.cy2, G.cy1);
        const double ru = sy * ra, rv = sy * rb, rw = sy * rc, sah = sy * ah, sae = sy * ae;
        double* W = S + ADJ_WY * P + c;
        W[VW_H * P] = -v * sah + rv * (cc - 0.5 * v * v) - 0.5 * ru * (u * v) - rw * (v * w);
        W[VW_V * P] = -h * sah - 0.5 * rv * hv - 0.5 * ru * hu - rw * hw;
        W[VW_U * P] = 0.5 * ru * hv;
        W[VW_W * P] = rw * hv;
        W[VW_ETA * P] = rv * G.lam3 * om - v * sae;
        W[VW_B * P] = rv * G.lam2 * om - 1.5 * v * sae;
        W[VW_HS * P] = rv * G.g;
        W[VW_SQ * P] = 0.5 * rv * h;      // v^2
        W[VW_HM * P] = 0.5 * rv * v;      // hv
        W[VW_HUV * P] = 0.5 * ru;
        W[VW_HMW * P] = rw;               // hvw
        W[VW_E2H * P] = -G.lam6 * rv;
    }
}

// Pass 2: everything else at one node.
template <int BC, int MODE>
__global__ void __launch_bounds__(ADJ_BLOCK, 2) k_adj_gather(AdjArgs a) {
    const Geom& G = a.G;
    const long long P = G.plane;
    const long long c = (long long)blockIdx.x * ADJ_BLOCK + threadIdx.x;
    if (c >= P) return;
    const int j = (int)(c / G.nx), i = (int)(c - (long long)j * G.nx);
    const double* __restrict__ S = a.scratch;

    // neighbours: left/right/below/above (periodic wrap; clamped at walls)
    const long long row = (long long)j * G.nx;
    long long cl, cr, cb, ct;
    if (BC == BC_PERIODIC) {
        cl = row + (i == 0 ? G.nx - 1 : i - 1);
        cr = row + (i == G.nx - 1 ? 0 : i + 1);
        cb = (long long)(j == 0 ? G.ny - 1 : j - 1) * G.nx + i;
        ct = (long long)(j == G.ny - 1 ? 0 : j + 1) * G.nx + i;
    } else {
        cl = i > 0 ? c - 1 : c;
        cr = i < G.nx - 1 ? c + 1 : c;
        cb = j > 0 ? c - G.nx : c;
        ct = j < G.ny - 1 ? c + G.nx : c;
    }

    // ---- product part: gathers of the neighbours' weights
    double pb[N_OPS - 1];
#pragma unroll
    for (int k = 0; k < N_OPS - 1; k++) pb[k] = 0.0;
    {
        const bool has_l = BC == BC_PERIODIC || i >= 1;
        const bool has_r = BC == BC_PERIODIC || i <= G.nx - 2;
        const double self = (BC == BC_REFLECTING) ? ((i == G.nx - 1 ? 1.0 : 0.0) - (i == 0 ? 1.0 : 0.0)) : 0.0;
        const int slot_of[12] = {OP_H, OP_U, OP_V, OP_W, OP_ETA, OP_B, OP_HS, OP_UU, OP_HU, OP_HUV, OP_HUW, OP_E2H};
#pragma unroll
        for (int k = 0; k < 12; k++) {
            const double* V = S + (ADJ_WX + k) * P;
            double g = 0.0;
            if (BC == BC_REFLECTING && self != 0.0) g = self * V[c];
            if (has_l) g += V[cl];
            if (has_r) g -= V[cr];
            pb[slot_of[k]] += g;
        }
    }
    {
        const bool has_b = BC == BC_PERIODIC || j >= 1;
        const bool has_t = BC == BC_PERIODIC || j <= G.ny - 2;
        const double self = (BC == BC_REFLECTING) ? ((j == G.ny - 1 ? 1.0 : 0.0) - (j == 0 ? 1.0 : 0.0)) : 0.0;
        const int slot_of[12] = {OP_H, OP_U, OP_V, OP_W, OP_ETA, OP_B, OP_HS, OP_VV, OP_HV, OP_HUV, OP_HVW, OP_E2H};
#pragma unroll
        for (int k = 0; k < 12; k++) {
            const double* V = S + (ADJ_WY + k) * P;
            double g = 0.0;
            if (BC == BC_REFLECTING && self != 0.0) g = self * V[c];
            if (has_b) g += V[cb];
            if (has_t) g -= V[ct];
            pb[slot_of[k]] += g;
        }
    }

    // ---- pointwise part: d k / d q at this node with every difference fixed
    double sx = G.cx2, sy = G.cy2, sgx = 0.0, sgy = 0.0;
    if (BC == BC_REFLECTING) {
        if (i == 0) { sx = G.cx1; sgx = -G.satx; }
        if (i == G.nx - 1) { sx = G.cx1; sgx = G.satx; }
        if (j == 0) { sy = G.cy1; sgy = -G.saty; }
        if (j == G.ny - 1) { sy = G.cy1; sgy = G.saty; }
    }
#define DX_(op) (sx * (S[(op) * P + cr] - S[(op) * P + cl]))
#define DY_(op) (sy * (S[(op) * P + ct] - S[(op) * P + cb]))
    const double h = S[OP_H * P + c], u = S[OP_U * P + c], v = S[OP_V * P + c];
    const double w = S[OP_W * P + c], eta = S[OP_ETA * P + c], bb = S[OP_B * P + c];
    const double r = S[OP_R * P + c];
    const double sc = a.a_scale;
    const double ah = sc * a.A[c], au = sc * a.A[P + c], av = sc * a.A[2 * P + c];
    const double aw = sc * a.A[3 * P + c], ae = sc * a.A[4 * P + c];
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
    const double lr = G.lam3 * rho * r;
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
