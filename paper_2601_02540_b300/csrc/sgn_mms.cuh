// sgn_mms.cuh - pointwise forcings inside fused RK4 stage kernels: the
// manufactured solution of Sec. 6.1.2 (its exact fields and the source terms
// S = q_t - F(q) that make it an exact solution of the continuum system eq.
// (2D_hyperbolic_SGN)) and the relaxation zones of the wave-tank experiments
// (Sec. 6).
//
// Manufactured solution (Sec. 6.1.2, any domain; the paper uses [-1,1]^2):
//   b   = 0.08 (cos 2pi x cos 2pi y + 1/2 cos 4pi x cos 4pi y)
//   h   = 2 + 1/2 sin 2pi x sin 2pi y cos 2pi t - b
//   u   = 0.3 sin 2pi x sin 2pi t,   v = 0.3 sin 2pi y sin 2pi t
//   eta = h,  w = -h (u_x + v_y) + 3/2 (u b_x + v b_y)
// F is the continuum right-hand side in primitive variables, from the
// conservative form with p = lambda/3 (eta/h) (1 - eta/h):
//   h_t = -(hu)_x - (hv)_y
//   (hu)_t = -(hu^2 + g h^2/2 + h p)_x - (huv)_y - (g h + 3/2 (h/eta) p) b_x
//   (hv)_t = -(hvu)_x - (hv^2 + g h^2/2 + h p)_y - (g h + 3/2 (h/eta) p) b_y
//   (h eta)_t = h w - (h eta u)_x - (h eta v)_y - 3/2 h (u b_x + v b_y)
//   (hw)_t = lambda (1 - eta/h) - (hwu)_x - (hwv)_y
// and f_t = ((h f)_t - f h_t) / h for f = u, v, eta, w.  Every derivative is
// taken by forward-mode differentiation: a Jet carries a value and its x, y
// and t derivatives through the arithmetic; the second derivatives that w's
// derivatives need (u_xx, v_yy, b_xx, b_xy, b_yy, u_xt, v_yt) are written out.
#pragma once

#include "sgn_kernels.cuh"

namespace sgn {

struct Jet {
    double v, x, y, t;
};
__device__ __forceinline__ Jet jconst(double c) { return {c, 0.0, 0.0, 0.0}; }
__device__ __forceinline__ Jet operator+(Jet a, Jet b) { return {a.v + b.v, a.x + b.x, a.y + b.y, a.t + b.t}; }
__device__ __forceinline__ Jet operator-(Jet a, Jet b) { return {a.v - b.v, a.x - b.x, a.y - b.y, a.t - b.t}; }
__device__ __forceinline__ Jet operator*(double c, Jet a) { return {c * a.v, c * a.x, c * a.y, c * a.t}; }
__device__ __forceinline__ Jet operator*(Jet a, Jet b) {
    return {a.v * b.v, a.x * b.v + a.v * b.x, a.y * b.v + a.v * b.y, a.t * b.v + a.v * b.t};
}
__device__ __forceinline__ Jet operator/(Jet a, Jet b) {
    const double q = a.v / b.v, r = 1.0 / b.v;
    return {q, (a.x - q * b.x) * r, (a.y - q * b.y) * r, (a.t - q * b.t) * r};
}

// Sines and cosines of the solution at (x, y) and the time factors sin 2pi t,
// cos 2pi t (computed once per launch on the host).
struct MmsTime {
    double st, ct;     // sin(2 pi t), cos(2 pi t)
};

struct MmsFields {
    Jet h, u, v, w, eta;
    double b, bx, by;
};

__device__ __forceinline__ MmsFields mms_fields(double x, double y, MmsTime T) {
    const double pi = 3.14159265358979323846;
    const double tp = 2.0 * pi, tp2 = tp * tp;
    double s1x, c1x, s1y, c1y;
    sincospi(2.0 * x, &s1x, &c1x);
    sincospi(2.0 * y, &s1y, &c1y);
    const double s2x = 2.0 * s1x * c1x, c2x = c1x * c1x - s1x * s1x;    // sin, cos of 4 pi x
    const double s2y = 2.0 * s1y * c1y, c2y = c1y * c1y - s1y * s1y;
    const double st = T.st, ct = T.ct;
    // bathymetry and its derivatives up to second order
    const double b = 0.08 * (c1x * c1y + 0.5 * c2x * c2y);
    const double bx = 0.08 * (-tp * s1x * c1y - tp * s2x * c2y);
    const double by = 0.08 * (-tp * c1x * s1y - tp * c2x * s2y);
    const double bxx = 0.08 * (-tp2 * c1x * c1y - 2.0 * tp2 * c2x * c2y);
    const double byy = bxx;
    const double bxy = 0.08 * (tp2 * s1x * s1y + 2.0 * tp2 * s2x * s2y);
    MmsFields F;
    F.b = b;
    F.bx = bx;
    F.by = by;
    // h = 2 + 1/2 sx sy ct - b
    F.h = {2.0 + 0.5 * s1x * s1y * ct - b, 0.5 * tp * c1x * s1y * ct - bx, 0.5 * tp * s1x * c1y * ct - by,
           -0.5 * tp * s1x * s1y * st};
    F.u = {0.3 * s1x * st, 0.3 * tp * c1x * st, 0.0, 0.3 * tp * s1x * ct};
    F.v = {0.3 * s1y * st, 0.0, 0.3 * tp * c1y * st, 0.3 * tp * s1y * ct};
    // jets of u_x, v_y, b_x, b_y (value and first derivatives)
    const Jet ux = {0.3 * tp * c1x * st, -0.3 * tp2 * s1x * st, 0.0, 0.3 * tp2 * c1x * ct};
    const Jet vy = {0.3 * tp * c1y * st, 0.0, -0.3 * tp2 * s1y * st, 0.3 * tp2 * c1y * ct};
    const Jet Bx = {bx, bxx, bxy, 0.0};
    const Jet By = {by, bxy, byy, 0.0};
    F.w = 1.5 * (F.u * Bx + F.v * By) - F.h * (ux + vy);
    F.eta = F.h;
    return F;
}

// S = q_t - F(q) at (x, y) and time factors T.
__device__ __forceinline__ void mms_source(double x, double y, MmsTime T, double g, double lam, double S[5]) {
    const MmsFields F = mms_fields(x, y, T);
    const Jet h = F.h, u = F.u, v = F.v, w = F.w, eta = F.eta;
    const Jet rho = eta / h;
    const Jet p = (lam / 3.0) * (rho * (jconst(1.0) - rho));
    const Jet hu = h * u, hv = h * v;
    const double ht = -(hu.x + hv.y);
    const Jet Fx = hu * u + (0.5 * g) * (h * h) + h * p;     // x flux of hu
    const Jet Fy = hv * v + (0.5 * g) * (h * h) + h * p;     // y flux of hv
    const double coef = g * h.v + 1.5 * (h.v / eta.v) * p.v;
    const double hut = -(Fx.x + (hu * v).y + coef * F.bx);
    const double hvt = -((hv * u).x + Fy.y + coef * F.by);
    const Jet he = h * eta;
    const double hetat = h.v * w.v - (he * u).x - (he * v).y - 1.5 * h.v * (u.v * F.bx + v.v * F.by);
    const Jet hw = h * w;
    const double hwt = lam * (1.0 - eta.v / h.v) - (hw * u).x - (hw * v).y;
    const double ut = (hut - u.v * ht) / h.v;
    const double vt = (hvt - v.v * ht) / h.v;
    const double wt = (hwt - w.v * ht) / h.v;
    const double etat = (hetat - eta.v * ht) / h.v;
    S[0] = h.t - ht;
    S[1] = u.t - ut;
    S[2] = v.t - vt;
    S[3] = w.t - wt;
    S[4] = eta.t - etat;
}

// Pointwise forcings added to the split-form RHS inside the RK4 stages:
//   FORCING_MMS     the manufactured-solution source S(x, y, t_stage);
//   FORCING_SPONGE  relaxation zones (Sec. 6, wave-tank experiments):
//                   -sigma(x, y) (q - q0), q0 the rest state, sigma rising
//                   quadratically from 0 at the inner edge of a zone of width
//                   wx (wy) to smax at the domain boundary; corners take the sum.
enum { FORCING_MMS = 0, FORCING_SPONGE = 1 };

struct MmsArgs {
    StageArgs<double, double, double> st;   // the RK4 stage operands (as k_stage)
    double xmin, ymin;                      // node (i, j) at (xmin + i dx, ymin + j dy)
    double xmax, ymax;                      // domain ends (relaxation-zone distances)
    MmsTime T;                              // time factors of this stage (MMS)
    const double* q0;                       // rest state (sponge), 5 planes
    double wx, wy, smax;                    // zone widths (0: none) and the boundary value of sigma
};

__device__ __forceinline__ double sponge_sigma(double x, double y, const MmsArgs& m) {
    double s = 0.0;
    if (m.wx > 0.0) {
        const double d = fmin(x - m.xmin, m.xmax - x);
        if (d < m.wx) {
            const double r = (m.wx - d) / m.wx;
            s += m.smax * r * r;
        }
    }
    if (m.wy > 0.0) {
        const double d = fmin(y - m.ymin, m.ymax - y);
        if (d < m.wy) {
            const double r = (m.wy - d) / m.wy;
            s += m.smax * r * r;
        }
    }
    return s;
}

// RK4 stage (modes S1..S4 of k_stage) with a pointwise forcing added to the
// split-form RHS at every node.
template <int BC, int MODE, int FORCING>
__global__ void __launch_bounds__(BLOCK_THREADS) k_forced_stage(MmsArgs m) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sm = reinterpret_cast<double*>(smem_raw);
    const StageArgs<double, double, double>& a = m.st;
    const Geom& G = a.G;
    const long long P = G.plane;
    constexpr int R = StageShape<double>::rows;
    constexpr int HY = THREADS_Y * R + 2, HN = HALO_X * HY;
    const int i0 = blockIdx.x * TILE_X, j0 = blockIdx.y * (THREADS_Y * R);
    const int tid = threadIdx.y * TILE_X + threadIdx.x;
    int bad = 0;
    if constexpr (kChecked) {                   // checked builds: poison the tile first
        for (int k = tid; k < N_OPS * HN; k += BLOCK_THREADS) sm[k] = poison<double>();
        __syncthreads();
    }
    for (int t = tid; t < HN; t += BLOCK_THREADS) {
        const int li = t % HALO_X, lj = t / HALO_X;
        const int gx = halo_index<BC>(i0 - 1 + li, G.nx);
        const int gy = halo_index<BC>(j0 - 1 + lj, G.ny);
        if (kChecked && (gx < 0 || gx >= G.nx || gy < 0 || gy >= G.ny)) {
            bad |= FLAG_BOUNDS;
            continue;
        }
        const long long c = (long long)gy * G.nx + gx;
        const double h = a.X[c];
        bad |= h_flags(h);
        store_operands<double, HN>(sm, t, h, a.X[P + c], a.X[2 * P + c], a.X[3 * P + c], a.X[4 * P + c],
                                       a.b[c], G);
    }
    if (bad) atomicOr(a.flag, bad);
    __syncthreads();
    const int gi = i0 + threadIdx.x;
#pragma unroll
    for (int ry = 0; ry < R; ry++) {
        const int ly = threadIdx.y + ry * THREADS_Y;
        const int gj = j0 + ly;
        if (gi >= G.nx || gj >= G.ny) continue;
        const int t = (ly + 1) * HALO_X + (threadIdx.x + 1);
        double k[5], S[5];
        node_rhs<double, BC, HALO_X, HN>(sm, t, gi, gj, G, k);
        const long long c = (long long)gj * G.nx + gi;
        const double x = m.xmin + gi * G.dx, y = m.ymin + gj * G.dy;
        if (FORCING == FORCING_MMS) {
            mms_source(x, y, m.T, G.g, G.lam, S);
        } else {
            const double sg = sponge_sigma(x, y, m);
#pragma unroll
            for (int f = 0; f < 5; f++) S[f] = -sg * (a.X[f * P + c] - m.q0[f * P + c]);
        }
#pragma unroll
        for (int f = 0; f < 5; f++) {
            const double kv = k[f] + S[f];
            const long long o = f * P + c;
            if (MODE == MODE_S4) {
                a.out[o] = fma(a.c_acc, kv, a.acc[o]);
            } else {
                const double qv = a.qn[o];
                a.acc[o] = fma(a.c_acc, kv, MODE == MODE_S1 ? qv : a.acc[o]);
                a.Qout[o] = fma(a.c_q, kv, qv);
            }
        }
    }
}

// The exact manufactured state (h, u, v, w, eta) at the time of T into q, and
// (if b is not null) the bathymetry.
static __global__ void __launch_bounds__(256) k_mms_exact(double* __restrict__ q, double* __restrict__ b, Geom G,
                                                          double xmin, double ymin, MmsTime T) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= G.nx || j >= G.ny) return;
    const long long P = G.plane, c = (long long)j * G.nx + i;
    const MmsFields F = mms_fields(xmin + i * G.dx, ymin + j * G.dy, T);
    q[c] = F.h.v;
    q[P + c] = F.u.v;
    q[2 * P + c] = F.v.v;
    q[3 * P + c] = F.w.v;
    q[4 * P + c] = F.eta.v;
    if (b) b[c] = F.b;
}

// The source S(x, y, t) at every node (for checking it against an independent
// evaluation).
static __global__ void __launch_bounds__(256) k_mms_source(double* __restrict__ s, Geom G, double xmin, double ymin,
                                                           MmsTime T) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= G.nx || j >= G.ny) return;
    const long long P = G.plane, c = (long long)j * G.nx + i;
    double S[5];
    mms_source(xmin + i * G.dx, ymin + j * G.dy, T, G.g, G.lam, S);
#pragma unroll
    for (int f = 0; f < 5; f++) s[f * P + c] = S[f];
}

}  // namespace sgn
