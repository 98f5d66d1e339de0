// sgn_adjoint.cuh - the exact discrete adjoint (vector-Jacobian product) of the
// split-form SBP right-hand side and of one classical RK4 step.  The paper has
// no adjoint; this is the transpose of the Jacobian of the RHS of
// eq. (sd_periodic_2D_SGN) / eq. (semi_2D) in the regrouped form the forward
// kernels evaluate (node_rhs_src), differentiated step by step in reverse.
//
// Structure.  At node c the forward RHS is a function of
//   - the operands of node c itself: h, u, v, w, rho = eta/h, r = 1/h,
//     hu, hv and P2 = 2g h(h+b) - lam/3 eta^2/h, and
//   - twenty unscaled differences d(c) = f(R(c)) - f(L(c)) of operand planes
//     f (x: h, u, v, w, F = eta + 3/2 b, P2, u^2, hu, huv, huw; y: h, u, v, w,
//     F, P2, v^2, hv, huv, hvw), where R, L are the right and left neighbours
//     (the node itself on a reflecting wall: the one-sided end rows).
// For a cotangent a at c, reverse differentiation of node_rhs_src gives the
// cotangents of the twenty differences ("weights" W) and of the node's own
// operands; a difference weight W(c) reaches the operand f at node n through
// the transposed operator, sum_c W(c) (delta(R(c), n) - delta(L(c), n)).
// Two passes per RK stage, both one node per thread, without halos or atomics:
//   k_adj_point   the weights and the node's own part (pointwise, no neighbours);
//   k_adj_gather  gathers the neighbours' weights, adds the node's own part,
//                 applies the chain rule from the operands to (h, u, v, w, eta, b),
//                 and (stage mode) the reverse RK4 stage algebra.
// The forward intermediates the reverse sweep needs (differences, A_x, A_y,
// D(hu) - A_x, k_u, k_v, k_w, 1/h, -P2/h) are not recomputed: they come from
// the tape of the forward evaluation at the same state (TP_ planes), written
// by the FP64 stage kernel while it advances the state (sgn_step_record_tape)
// or by a TAPE-mode launch.  The kernels are FP64-pipe bound, so the formulas
// use the fewest FP64 operations: r h = 1 cancels factors exactly up to
// rounding (the derivatives of k_u, k_v, k_w with respect to r are k/r), and
// the cotangent of a stage is carried as sigma * A with the scale sigma
// applied only where a result is accumulated (see AdjArgs).
#pragma once

#include "sgn_kernels.cuh"

namespace sgn {

// Weight planes (cotangents of the unscaled differences at each node): x
// uses {H, U, V, W, F, P2, UU, HU, HUV, HUW}, y uses {H, U, V, W, F, P2, VV,
// HV, HUV, HVW}; slot k of x and slot k of y differentiate the same operand
// for k < VW_SQ and for VW_HUV.
enum { VW_H, VW_U, VW_V, VW_W, VW_F, VW_P2, VW_SQ, VW_HM, VW_HUV, VW_HMW, ADJ_NW };
// the node's own part of the cotangents of h, u, v, w, eta (the operands
// rho, r, hu, hv already reduced to them) and of its P2
enum { AC_H, AC_U, AC_V, AC_W, AC_E, AC_P2, ADJ_NC };
constexpr int ADJ_WX = 0;
constexpr int ADJ_WY = ADJ_NW;
constexpr int ADJ_C = 2 * ADJ_NW;
constexpr int ADJ_SCRATCH_PLANES = 2 * ADJ_NW + ADJ_NC;
constexpr int ADJ_BLOCK = 256;

enum { ADJ_MODE_RHS = 0, ADJ_MODE_STAGE = 1 };

struct AdjArgs {
    const double* X;       // state at which the Jacobian is taken (5 planes)
    const double* tape;    // the tape of f(X) (N_TAPE planes)
    const double* b;       // bathymetry
    const double* A;       // cotangent direction (5 planes); the cotangent is sigma * A
    double sigma;          // scale of the cotangent, applied to every result
    double* scratch;       // ADJ_SCRATCH_PLANES planes
    double* qbar;          // RHS mode: output J^T (sigma A) (5 planes)
    double* bbar;          // accumulated (1 plane)
    // stage mode, with Qbar = J^T (sigma A):
    //   qacc_out = (first ? qprime : qacc_in) + Qbar
    //   Anext    = kappa * qprime + J^T A   (when Anext != nullptr)
    // so that the next stage's cotangent c' qprime + cbar Qbar equals
    // sigma' * Anext with sigma' = cbar sigma and kappa = c' / sigma'.
    const double* qprime;
    const double* qacc_in;
    double* qacc_out;
    double* Anext;
    double kappa;
    int first;
    Geom G;
    int* flag;             // latched error bits (FLAG_BOUNDS of checked builds)
};

// x with its sign bit flipped where m has it set (an exact negation).
__device__ __forceinline__ double flip_sign(double x, unsigned long long m) {
    return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(x) ^ m));
}

// Pass 1: the difference weights and the node's own cotangents at one node,
// for the cotangent direction A (sigma is applied by the gather pass).  The
// names follow node_rhs_src: Xu, Yu, ... are its bracket sums, A_x, A_y its
// continuity fluxes, base2 = -P2/h, lom2 = 2 lam/3 (1 - rho), and a trailing
// "b" marks a cotangent.
template <int BC>
__device__ __forceinline__ void adj_point_node(const AdjArgs& a, long long c, int i, int j, double ah, double au,
                                               double av, double aw, double ae) {
    const Geom& G = a.G;
    const long long P = G.plane;
    const double* __restrict__ T = a.tape + c;
    const double r = T[TP_R * P], base2 = T[TP_BASE2 * P];
    const double dxh = T[TP_DXH * P], dyh = T[TP_DYH * P], dxu = T[TP_DXU * P], dyu = T[TP_DYU * P];
    const double dxv = T[TP_DXV * P], dyv = T[TP_DYV * P], dxw = T[TP_DXW * P], dyw = T[TP_DYW * P];
    const double dxf = T[TP_DXF * P], dyf = T[TP_DYF * P], dxuu = T[TP_DXUU * P], dyvv = T[TP_DYVV * P];
    const double xhu = T[TP_XHU * P], yhv = T[TP_YHV * P], Ax = T[TP_AX * P], Ay = T[TP_AY * P];
    const double ku = T[TP_KU * P], kv = T[TP_KV * P], kw = T[TP_KW * P];
    const double h = a.X[c], u = a.X[P + c], v = a.X[2 * P + c], w = a.X[3 * P + c], eta = a.X[4 * P + c];

    // the operator's row factors at this node (one-sided rows on a reflecting wall)
    const bool wx = BC == BC_REFLECTING && (i == 0 || i == G.nx - 1);
    const bool wy = BC == BC_REFLECTING && (j == 0 || j == G.ny - 1);
    const double sx = wx ? G.cx1 : G.cx2, hsx = wx ? G.hcx1 : G.hcx2;
    const double sy = wy ? G.cy1 : G.cy2, hsy = wy ? G.hcy1 : G.hcy2;

    const double rho = eta * r;
    const double lom2 = fma(-G.lam23, rho, G.lam23);
    const double hu = h * u, hv = h * v;
    const double al = r * hsx, be = r * hsy;           // hrsx, hrsy of the forward
    // k_u = -(al Xu + be Yu), k_v = -(be Yv + al Xv), k_w = r lam (1 - rho) - (al Xw + be Yw)
    const double Xub = -al * au, Yub = -be * au;
    const double Yvb = -be * av, Xvb = -al * av;
    const double Xwb = -al * aw, Ywb = -be * aw;
    // k_h = -(sx A_x + sy A_y) + SAT, k_eta = w - u sx D_x F - v sy D_y F
    const double ex = sx * ae, ey = sy * ae;

    // Xu = base2 dxh + dxP2 + u (dxhu - A_x) + h dxuu + lom2 dxf and Xv, Xw into A_x
    const double WxHU = Xub * u, WxUU = Xub * h;
    double Axb = fma(-sx, ah, -WxHU);
    Axb = fma(-Xvb, v, Axb);
    Axb = fma(-Xwb, w, Axb);
    const double WyHV = Yvb * v, WyVV = Yvb * h;
    double Ayb = fma(-sy, ah, -WyHV);
    Ayb = fma(-Yub, u, Ayb);
    Ayb = fma(-Ywb, w, Ayb);

    double* __restrict__ S = a.scratch + c;
    double* WX = S + ADJ_WX * P;
    double* WY = S + ADJ_WY * P;
    WX[VW_H * P] = fma(Xub, base2, Axb * u);
    WX[VW_U * P] = Axb * h;
    WX[VW_V * P] = Xvb * hu;
    WX[VW_W * P] = Xwb * hu;
    WX[VW_F * P] = fma(Xub, lom2, -u * ex);
    WX[VW_P2 * P] = Xub;
    WX[VW_SQ * P] = WxUU;
    WX[VW_HM * P] = WxHU;
    WX[VW_HUV * P] = Xvb;
    WX[VW_HMW * P] = Xwb;
    WY[VW_H * P] = fma(Yvb, base2, Ayb * v);
    WY[VW_U * P] = Yub * hv;
    WY[VW_V * P] = Ayb * h;
    WY[VW_W * P] = Ywb * hv;
    WY[VW_F * P] = fma(Yvb, lom2, -v * ey);
    WY[VW_P2 * P] = Yvb;
    WY[VW_SQ * P] = WyVV;
    WY[VW_HM * P] = WyHV;
    WY[VW_HUV * P] = Yub;
    WY[VW_HMW * P] = Ywb;

    // the node's own operands
    double ub = fma(Xub, xhu, -ex * dxf);
    ub = fma(-Yub, Ay, ub);
    ub = fma(Axb, dxh, ub);
    double vb = fma(Yvb, yhv, -ey * dyf);
    vb = fma(-Xvb, Ax, vb);
    vb = fma(Ayb, dyh, vb);
    double wb = fma(-Xwb, Ax, ae);
    wb = fma(-Ywb, Ay, wb);
    double hb = fma(Yvb, dyvv, Xub * dxuu);
    hb = fma(Axb, dxu, hb);
    hb = fma(Ayb, dyv, hb);
    double hub = fma(Xvb, dxv, Xwb * dxw);
    double hvb = fma(Yub, dyu, Ywb * dyw);
    if (BC == BC_REFLECTING) {
        // SAT of the h equation: -+ satx hu, -+ saty hv on the walls
        if (i == 0) hub = fma(-G.satx, ah, hub);
        if (i == G.nx - 1) hub = fma(G.satx, ah, hub);
        if (j == 0) hvb = fma(-G.saty, ah, hvb);
        if (j == G.ny - 1) hvb = fma(G.saty, ah, hvb);
    }
    const double Bb = fma(Xub, dxh, Yvb * dyh);        // base2
    const double Lb = fma(Xub, dxf, Yvb * dyf);        // lom2
    // r: d k_f / d r = k_f / r = h k_f (f = u, v, w), d base2 / d r = h base2
    const double rb = h * fma(Bb, base2, fma(aw, kw, fma(av, kv, au * ku)));
    // rho: lom2 and k_w
    const double rhob = -fma(G.lam23, Lb, G.lam * (r * aw));
    // rho = eta r, r = 1/h, hu, hv, base2 = -P2 r (P2 waits for the gathered part)
    const double eb = r * rhob;
    hb = fma(-(r * r), fma(eta, rhob, rb), hb);
    hb = fma(u, hub, hb);
    hb = fma(v, hvb, hb);
    ub = fma(h, hub, ub);
    vb = fma(h, hvb, vb);
    double* C = S + ADJ_C * P;
    C[AC_H * P] = hb;
    C[AC_U * P] = ub;
    C[AC_V * P] = vb;
    C[AC_W * P] = wb;
    C[AC_E * P] = eb;
    C[AC_P2 * P] = -r * Bb;
}

#ifndef SGN_ADJ_POINT_MINB
#define SGN_ADJ_POINT_MINB 3
#endif
template <int BC>
__global__ void __launch_bounds__(ADJ_BLOCK, SGN_ADJ_POINT_MINB) k_adj_point(AdjArgs a) {
    const long long P = a.G.plane;
    const long long c = (long long)blockIdx.x * ADJ_BLOCK + threadIdx.x;
    if (c >= P) return;
    const int j = (int)(c / a.G.nx), i = (int)(c - (long long)j * a.G.nx);
    adj_point_node<BC>(a, c, i, j, a.A[c], a.A[P + c], a.A[2 * P + c], a.A[3 * P + c], a.A[4 * P + c]);
}

// Pass 2: the transposed differences (gathers of the neighbours' weights),
// the chain rule from the operands to the state and bathymetry, and the
// stage algebra, at one node.  CHAIN (stage mode): the next stage's
// cotangent direction kappa qprime + J^T A is returned in an[] instead of
// being stored.
template <int BC, int MODE, bool CHAIN>
__device__ __forceinline__ void adj_gather_node(const AdjArgs& a, long long c, int i, int j, double an[5]) {
    const Geom& G = a.G;
    const long long P = G.plane;
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
    if constexpr (kChecked) {
        // every neighbour must lie in this node's row (x) or column (y); an
        // index that does not is flagged and replaced by the node itself
        const bool bad_x = cl < row || cl >= row + G.nx || cr < row || cr >= row + G.nx;
        const bool bad_y = cb < 0 || cb >= P || ct < 0 || ct >= P || cb % G.nx != i || ct % G.nx != i;
        if (bad_x || bad_y) {
            atomicOr(a.flag, FLAG_BOUNDS);
            if (bad_x) cl = cr = c;
            if (bad_y) cb = ct = c;
        }
    }

    // Transposed differences: the weight of node m reaches node n with +1 if
    // n = R(m) and -1 if n = L(m).  Inside, that is W(n-1) - W(n+1); at a
    // reflecting wall the clamped neighbour index is the node itself, whose
    // one-sided row has the node as its L (first node) or R (last node), so
    // its weight enters with a flipped sign.
    unsigned long long fl = 0ull, fr = 0ull, fb = 0ull, ft = 0ull;
    if (BC == BC_REFLECTING) {
        const unsigned long long sgn_bit = 0x8000000000000000ull;
        fl = i == 0 ? sgn_bit : 0ull;
        fr = i == G.nx - 1 ? sgn_bit : 0ull;
        fb = j == 0 ? sgn_bit : 0ull;
        ft = j == G.ny - 1 ? sgn_bit : 0ull;
    }
    const double* __restrict__ WX = S + ADJ_WX * P;
    const double* __restrict__ WY = S + ADJ_WY * P;
    const double* __restrict__ C = S + ADJ_C * P + c;
#define GX_(k) (flip_sign(WX[(k) * P + cl], fl) - flip_sign(WX[(k) * P + cr], fr))
#define GY_(k) (flip_sign(WY[(k) * P + cb], fb) - flip_sign(WY[(k) * P + ct], ft))
    double hb = GX_(VW_H) + GY_(VW_H) + C[AC_H * P];
    double ub = GX_(VW_U) + GY_(VW_U) + C[AC_U * P];
    double vb = GX_(VW_V) + GY_(VW_V) + C[AC_V * P];
    double wb = GX_(VW_W) + GY_(VW_W) + C[AC_W * P];
    const double Fb = GX_(VW_F) + GY_(VW_F);
    const double P2b = GX_(VW_P2) + GY_(VW_P2) + C[AC_P2 * P];
    const double HUVb = GX_(VW_HUV) + GY_(VW_HUV);
    const double UUb = GX_(VW_SQ), HUb = GX_(VW_HM), HUWb = GX_(VW_HMW);
    const double VVb = GY_(VW_SQ), HVb = GY_(VW_HM), HVWb = GY_(VW_HMW);
#undef GX_
#undef GY_

    // chain rule from the operands to (h, u, v, w, eta, b) at this node:
    // F = eta + 3/2 b; P2 = 2g h(h+b) - lam/3 eta^2/h with dP2/dh = 2g(2h+b) + lam/3 rho^2,
    // dP2/deta = -2 lam/3 rho, dP2/db = 2g h; u^2, v^2, hu, hv, huv, huw, hvw
    const double h = a.X[c], u = a.X[P + c], v = a.X[2 * P + c], w = a.X[3 * P + c];
    const double eta = a.X[4 * P + c], bb = a.b[c];
    const double r = a.tape[TP_R * P + c];
    const double rho = eta * r;
    const double hu = h * u, hv = h * v, hw = h * w, uv = u * v, uw = u * w, vw_ = v * w;
    double eb = C[AC_E * P] + Fb;
    double bbar = 1.5 * Fb;
    hb = fma(fma(G.g2, fma(2.0, h, bb), G.lam3 * (rho * rho)), P2b, hb);
    eb = fma(-G.lam23 * rho, P2b, eb);
    bbar = fma(G.g2 * h, P2b, bbar);
    ub = fma(u + u, UUb, ub);
    vb = fma(v + v, VVb, vb);
    hb = fma(vw_, HVWb, fma(uw, HUWb, fma(uv, HUVb, fma(v, HVb, fma(u, HUb, hb)))));
    ub = fma(hw, HUWb, fma(hv, HUVb, fma(h, HUb, ub)));
    vb = fma(hw, HVWb, fma(hu, HUVb, fma(h, HVb, vb)));
    wb = fma(hv, HVWb, fma(hu, HUWb, wb));

    const double qb[5] = {hb, ub, vb, wb, eb};
    const double sg = a.sigma;
    a.bbar[c] = fma(sg, bbar, a.bbar[c]);
    if (MODE == ADJ_MODE_RHS) {
#pragma unroll
        for (int f = 0; f < 5; f++) a.qbar[f * P + c] = sg * qb[f];
    } else {
#pragma unroll
        for (int f = 0; f < 5; f++) {
            const double qp = a.qprime[f * P + c];
            const double base = a.first ? qp : a.qacc_in[f * P + c];
            a.qacc_out[f * P + c] = fma(sg, qb[f], base);
            if constexpr (CHAIN) an[f] = fma(a.kappa, qp, qb[f]);
            else if (a.Anext) a.Anext[f * P + c] = fma(a.kappa, qp, qb[f]);
        }
    }
}

template <int BC, int MODE>
__global__ void __launch_bounds__(ADJ_BLOCK) k_adj_gather(AdjArgs a) {
    const long long c = (long long)blockIdx.x * ADJ_BLOCK + threadIdx.x;
    if (c >= a.G.plane) return;
    const int j = (int)(c / a.G.nx), i = (int)(c - (long long)j * a.G.nx);
    double an[5];
    adj_gather_node<BC, MODE, false>(a, c, i, j, an);
}

// Pass 2 of a stage followed, at the same node, by pass 1 of the stage before
// it (a step's walk, stages 4-2): the point pass takes the cotangent direction
// the gather pass forms, without storing it.  `n` addresses the earlier
// stage's state, tape and a second weight buffer (the gather pass still reads
// the neighbours' weights of this stage from `a`).
template <int BC>
__global__ void __launch_bounds__(ADJ_BLOCK, SGN_ADJ_POINT_MINB) k_adj_gather_point(AdjArgs a, AdjArgs n) {
    const long long c = (long long)blockIdx.x * ADJ_BLOCK + threadIdx.x;
    if (c >= a.G.plane) return;
    const int j = (int)(c / a.G.nx), i = (int)(c - (long long)j * a.G.nx);
    double an[5];
    adj_gather_node<BC, ADJ_MODE_STAGE, true>(a, c, i, j, an);
    adj_point_node<BC>(n, c, i, j, an[0], an[1], an[2], an[3], an[4]);
}

}  // namespace sgn
