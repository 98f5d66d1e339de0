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
//   k_adj_weights  products P_t, 1/h and the 20 direction weights of each node
//                  into scratch planes;
//   k_adj_gather   differences, pointwise part, gathers of the weights of the
//                  neighbours, chain rule, and (stage mode) the reverse RK4
//                  stage algebra.
// The kernels are FP64-pipe bound, so the formulas are arranged for the fewest
// FP64 instructions: h r = 1 (r = 1/h) is used to cancel factors exactly up to
// rounding, constant factors of the differences are folded on the host, and
// the cotangent of a stage is carried as sigma * A with the scale sigma applied
// only where a result is accumulated (see AdjArgs).
#pragma once

#include "sgn_kernels.cuh"

namespace sgn {

// scratch layout (planes): the differentiated products and 1/h (the state
// planes themselves are read from the state), then the x weights (10) and the
// y weights (10).  P = g h(h+b) - lam/6 eta^2/h: g D(h(h+b)) - lam/6 D(eta^2/h)
// = D P (D is linear), so the two products of the brackets share one plane
// and one weight slot.
enum { AP_P, AP_HU, AP_HV, AP_HUV, AP_HUW, AP_HVW, AP_E15, AP_R, ADJ_NP };
constexpr int ADJ_NW = 10;
constexpr int ADJ_WX = ADJ_NP;
constexpr int ADJ_WY = ADJ_NP + ADJ_NW;
constexpr int ADJ_SCRATCH_PLANES = ADJ_NP + 2 * ADJ_NW;
constexpr int ADJ_BLOCK = 256;

// weight slots: x uses {H,U,V,W,E15,P,UU,HU,HUV,HUW},
// y uses {H,U,V,W,E15,P,VV,HV,HUV,HVW}.  eta and b enter the forward RHS
// only through eta + 3/2 b and P, so one E15 slot carries both
// (d/d eta = 1, d/d b = 3/2).
enum { VW_H, VW_U, VW_V, VW_W, VW_E15, VW_P, VW_SQ, VW_HM, VW_HUV, VW_HMW };

enum { ADJ_MODE_RHS = 0, ADJ_MODE_STAGE = 1 };

// Per-direction constants of the pointwise part, for interior rows ([0]) and
// the one-sided boundary rows ([1]): s = row factor of D, hs = s/2.
struct AdjDir {
    double s, hs;
};

struct AdjArgs {
    const double* X;       // state at which the Jacobian is taken (5 planes)
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
    AdjDir kx[2], ky[2];
    int* flag;             // latched error bits (FLAG_BOUNDS of checked builds)
    double m2lam3;         // -2 lambda / 3
    double lam2x;          // 2 lambda
};

// Host: the derived constants of AdjArgs.
inline void fill_adj_constants(AdjArgs& a) {
    const Geom& G = a.G;
    const double sx[2] = {G.cx2, G.cx1}, sy[2] = {G.cy2, G.cy1};
    for (int k = 0; k < 2; k++) {
        a.kx[k] = {sx[k], 0.5 * sx[k]};
        a.ky[k] = {sy[k], 0.5 * sy[k]};
    }
    a.m2lam3 = -2.0 * G.lam3;
    a.lam2x = 2.0 * G.lam;
}

// x with its sign bit flipped where m has it set (an exact negation).
__device__ __forceinline__ double flip_sign(double x, unsigned long long m) {
    return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(x) ^ m));
}

// Pass 1: products, 1/h and the direction weights V^x, V^y of one node
// (for the cotangent direction A; sigma is applied by the gather pass).
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
    const double hu = h * u, hv = h * v;
    const double hsum = h + bb, rho = eta * r;
    double* S = a.scratch;
    S[AP_P * P + c] = fma(G.g * h, hsum, -(G.lam6 * rho) * eta);
    S[AP_HU * P + c] = hu;
    S[AP_HV * P + c] = hv;
    S[AP_HUV * P + c] = hu * v;
    S[AP_HUW * P + c] = hu * w;
    S[AP_HVW * P + c] = hv * w;
    S[AP_E15 * P + c] = fma(1.5, bb, eta);
    S[AP_R * P + c] = r;

    const double ah = a.A[c], au = a.A[P + c], av = a.A[2 * P + c];
    const double aw = a.A[3 * P + c], ae = a.A[4 * P + c];
    const double lom = G.lam3 * (1.0 - rho);                       // lam/3 (1 - rho)
    const double cc = fma(G.lam6 * rho, rho, -G.g * hsum);         // lam/6 rho^2 - g (h + b)
    const double ra = -r * au, rb = -r * av, rc = (-0.5 * r) * aw; // d k / d B for u, v, w
    // The D h and D u weights share T = s a_h + (r/2) s (u a_u + v a_v + w a_w)
    // (the coefficients of the continuity flux u D h + h D u in the h equation
    // and in the split brackets): V_h = -r s a_u (lam/6 rho^2 - g (h+b)) - u T,
    // V_u = -h T (and the same with v for y).
    // x weights (row factor s of column i)
    {
        const bool wall = BC == BC_REFLECTING && (i == 0 || i == G.nx - 1);
        const double sx = wall ? a.kx[1].s : a.kx[0].s, hsx = wall ? a.kx[1].hs : a.kx[0].hs;
        const double ru = sx * ra, rw = sx * rc, sah = sx * ah, sae = sx * ae;
        const double hru = 0.5 * ru, hrv = hsx * rb;
        const double T = fma(hru, u, fma(hrv, v, fma(rw, w, sah)));
        double* W = S + ADJ_WX * P + c;
        W[VW_H * P] = fma(ru, cc, -u * T);
        W[VW_U * P] = -h * T;
        W[VW_V * P] = hrv * hu;
        W[VW_W * P] = rw * hu;
        W[VW_E15 * P] = fma(ru, lom, -u * sae);
        W[VW_P * P] = ru;
        W[VW_SQ * P] = hru * h;          // u^2
        W[VW_HM * P] = hru * u;          // hu
        W[VW_HUV * P] = hrv;
        W[VW_HMW * P] = rw;              // huw
    }
    // y weights (row factor s of row j)
    {
        const bool wall = BC == BC_REFLECTING && (j == 0 || j == G.ny - 1);
        const double sy = wall ? a.ky[1].s : a.ky[0].s, hsy = wall ? a.ky[1].hs : a.ky[0].hs;
        const double rv = sy * rb, rw = sy * rc, sah = sy * ah, sae = sy * ae;
        const double hrv = 0.5 * rv, hru = hsy * ra;
        const double T = fma(hru, u, fma(hrv, v, fma(rw, w, sah)));
        double* W = S + ADJ_WY * P + c;
        W[VW_H * P] = fma(rv, cc, -v * T);
        W[VW_V * P] = -h * T;
        W[VW_U * P] = hru * hv;
        W[VW_W * P] = rw * hv;
        W[VW_E15 * P] = fma(rv, lom, -v * sae);
        W[VW_P * P] = rv;
        W[VW_SQ * P] = hrv * h;          // v^2
        W[VW_HM * P] = hrv * v;          // hv
        W[VW_HUV * P] = hru;
        W[VW_HMW * P] = rw;              // hvw
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

    // ---- product part: gathers of the neighbours' weights.  At a reflecting
    // wall the clamped neighbour index is the node itself and its weight enters
    // with a flipped sign (the one-sided end rows of the SBP operator).
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
#define GX_(k) (flip_sign(WX[(k) * P + cl], fl) - flip_sign(WX[(k) * P + cr], fr))
#define GY_(k) (flip_sign(WY[(k) * P + cb], fb) - flip_sign(WY[(k) * P + ct], ft))
    const double pH = GX_(VW_H) + GY_(VW_H), pU = GX_(VW_U) + GY_(VW_U);
    const double pV = GX_(VW_V) + GY_(VW_V), pW = GX_(VW_W) + GY_(VW_W);
    const double pF = GX_(VW_E15) + GY_(VW_E15), pP = GX_(VW_P) + GY_(VW_P);
    const double pHUV = GX_(VW_HUV) + GY_(VW_HUV);
    const double pUU = GX_(VW_SQ), pHU = GX_(VW_HM), pHUW = GX_(VW_HMW);
    const double pVV = GY_(VW_SQ), pHV = GY_(VW_HM), pHVW = GY_(VW_HMW);
#undef GX_
#undef GY_

    // ---- pointwise part: d k / d q at this node with every difference fixed.
    // With k_u = -r B_u, k_w = r B_w (B the brackets of the forward kernel) the
    // h-derivatives combine as d(k_u)/dh = r^2 G_u, d(k_v)/dh = r^2 G_v,
    // d(k_w)/dh = r^2 G_w, where (using r h = 1; the dropped terms are rounding)
    //   G_u = D_x h (lam/2 rho^2 - u^2/2 - g b) + lam/3 (1 - 2 rho) D_x(eta + 3/2 b)
    //         + D_x P + u/2 D_x(hu) + (D_y(huv) - uv D_y h)/2   (P = g h(h+b) - lam/6 eta^2/h),
    //   G_w = lam (2 rho - 1) + (D_x(huw) - uw D_x h + D_y(hvw) - vw D_y h)/2,
    // eta and b enter only through D(eta + 3/2 b), and r h = 1 also reduces the
    // u-, v- and w-derivatives to the forms below.
    const bool wx = BC == BC_REFLECTING && (i == 0 || i == G.nx - 1);
    const bool wy = BC == BC_REFLECTING && (j == 0 || j == G.ny - 1);
    const AdjDir kx = wx ? a.kx[1] : a.kx[0];
    const AdjDir ky = wy ? a.ky[1] : a.ky[0];
    double sgx = 0.0, sgy = 0.0;
    if (BC == BC_REFLECTING) {
        if (i == 0) sgx = -G.satx;
        if (i == G.nx - 1) sgx = G.satx;
        if (j == 0) sgy = -G.saty;
        if (j == G.ny - 1) sgy = G.saty;
    }
    const double* __restrict__ X = a.X;
#define RX_(base) ((base)[cr] - (base)[cl])
#define RY_(base) ((base)[ct] - (base)[cb])
    const double h = X[c], u = X[P + c], v = X[2 * P + c], w = X[3 * P + c], eta = X[4 * P + c];
    const double bb = a.b[c];
    const double r = S[AP_R * P + c];
    const double ah = a.A[c], au = a.A[P + c], av = a.A[2 * P + c];
    const double aw = a.A[3 * P + c], ae = a.A[4 * P + c];
    // differences used more than once, scaled
    const double xh = kx.s * RX_(X), xu = kx.s * RX_(X + P), xv = kx.s * RX_(X + 2 * P);
    const double xw = kx.s * RX_(X + 3 * P), xf = kx.s * RX_(S + AP_E15 * P);
    const double yh = ky.s * RY_(X), yu = ky.s * RY_(X + P), yv = ky.s * RY_(X + 2 * P);
    const double yw = ky.s * RY_(X + 3 * P), yf = ky.s * RY_(S + AP_E15 * P);
    const double hxhu = kx.hs * RX_(S + AP_HU * P), hyhv = ky.hs * RY_(S + AP_HV * P);  // D(hu)/2, D(hv)/2

    const double ar = r * au, br = r * av, cr_ = r * aw;
    const double rho = eta * r, rho2 = rho * rho;
    const double hu = h * u, hv = h * v, hw = h * w, uv = u * v, uw = u * w, vw_ = v * w;
    const double q2 = fma(G.lam2, rho2, -G.g * bb);       // lam/2 rho^2 - g b
    const double l12 = fma(a.m2lam3, rho, G.lam3);        // lam/3 (1 - 2 rho)
    const double huv = 0.5 * uv;
    double Gu = xh * fma(-0.5 * u, u, q2);
    Gu = fma(l12, xf, Gu);
    Gu = fma(kx.s, RX_(S + AP_P * P), Gu);
    Gu = fma(u, hxhu, Gu);
    Gu = fma(ky.hs, RY_(S + AP_HUV * P), Gu);
    Gu = fma(-huv, yh, Gu);
    double Gv = yh * fma(-0.5 * v, v, q2);
    Gv = fma(l12, yf, Gv);
    Gv = fma(ky.s, RY_(S + AP_P * P), Gv);
    Gv = fma(v, hyhv, Gv);
    Gv = fma(kx.hs, RX_(S + AP_HUV * P), Gv);
    Gv = fma(-huv, xh, Gv);
    double Gw = fma(a.lam2x, rho, -G.lam);
    Gw = fma(kx.hs, RX_(S + AP_HUW * P), Gw);
    Gw = fma(ky.hs, RY_(S + AP_HVW * P), Gw);
    Gw = fma(-0.5, fma(uw, xh, vw_ * yh), Gw);
#undef RX_
#undef RY_

    const double divu = xu + yv;
    double hb = fma(-ah, divu, r * fma(ar, Gu, fma(br, Gv, cr_ * Gw)));
    const double aru = ar * u, brv = br * v, crw = cr_ * w;
    const double hau = 0.5 * au, hav = 0.5 * av, haw = 0.5 * aw;
    double ub = xh * (fma(0.5, brv + crw, aru) - ah);
    ub = fma(ar, fma(0.5 * v, yh, -hxhu), ub);
    ub = fma(-ae, xf, fma(-haw, xw, fma(-hav, xv, fma(hau, divu, ub))));
    double vb = yh * (fma(0.5, aru + crw, brv) - ah);
    vb = fma(br, fma(0.5 * u, xh, -hyhv), vb);
    vb = fma(-ae, yf, fma(-haw, yw, fma(-hau, yu, fma(hav, divu, vb))));
    double wb = fma(0.5 * cr_, fma(u, xh, v * yh), fma(haw, divu, ae));
    // d/d eta: only rho and 1 - rho depend on eta (d rho / d eta = r)
    double eb = fma(ar, fma(rho, xh, -xf), br * fma(rho, yh, -yf));
    eb = -r * fma(G.lam3, eb, G.lam * cr_);
    double bbar = G.g * fma(ar, xh, br * yh);
    if (BC == BC_REFLECTING) {
        // SAT of the h equation: d/dh and d/du, d/dv of (sgx hu + sgy hv)
        hb = fma(ah, fma(sgx, u, sgy * v), hb);
        ub = fma(ah * sgx, h, ub);
        vb = fma(ah * sgy, h, vb);
    }

    // ---- chain rule through the products
    // dP/dh = g (2h + b) + lam/6 rho^2, dP/deta = -lam/3 rho, dP/db = g h
    hb = fma(vw_, pHVW, fma(uw, pHUW, fma(uv, pHUV, fma(v, pHV, fma(u, pHU,
         fma(fma(G.g, fma(2.0, h, bb), G.lam6 * rho2), pP, hb + pH))))));
    ub = fma(hw, pHUW, fma(hv, pHUV, fma(h, pHU, fma(2.0 * u, pUU, ub + pU))));
    vb = fma(hw, pHVW, fma(hu, pHUV, fma(h, pHV, fma(2.0 * v, pVV, vb + pV))));
    wb = fma(hv, pHVW, fma(hu, pHUW, wb + pW));
    eb = fma(-G.lam3 * rho, pP, eb + pF);
    bbar = fma(G.g * h, pP, fma(1.5, pF, bbar));

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
            if (a.Anext) a.Anext[f * P + c] = fma(a.kappa, qp, qb[f]);
        }
    }
}

}  // namespace sgn
