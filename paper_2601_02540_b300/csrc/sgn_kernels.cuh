// sgn_kernels.cuh - sm_103a kernels for the split-form SBP semi-discretization of
// the 2D hyperbolized Serre-Green-Naghdi equations (arXiv 2601.02540, Sec. 4),
// fused with the stages of classical RK4.
//
// One thread block owns a TILE_X x TILE_Y tile of output nodes.  It reads the
// six input planes (h, u, v, w, eta, b) of the tile plus a one-node halo,
// forms every operand that is differentiated (h, u, v, w, u^2, v^2, hu, hv,
// huv, huw, hvw, eta + 3/2 b and P2 = 2g h(h+b) - lam/3 eta^2/h) together with
// eta/h and 1/h once per node and stages them in shared memory, then
// each thread evaluates the right-hand side of eq. (sd_periodic_2D_SGN) /
// eq. (semi_2D) at its nodes and applies the RK4 stage algebra.  The halo is
// wrapped (periodic) or clamped (reflecting: the one-sided boundary rows of
// the SBP operator never read beyond the wall).
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "sgn_df64.cuh"

namespace sgn {

enum { BC_PERIODIC = 0, BC_REFLECTING = 1 };

// RK4 stage modes.  RHS writes dq; S1..S4 are the four stages of classical RK4
// on three registers (q_n, acc, Q):
//   S1: k = f(q_n); acc = q_n + dt/6 k; Q = q_n + dt/2 k
//   S2: k = f(Q);   acc += dt/3 k;      Q' = q_n + dt/2 k
//   S3: k = f(Q');  acc += dt/3 k;      Q  = q_n + dt k
//   S4: k = f(Q);   q_n = acc + dt/6 k
// DIAG computes k = f(q) and reduces mass, energy and the energy rate.
// S4D is S4 that also reduces the mass and energies of the new state q_{n+1}
// (the per-step monitor, fused into the stage that produces the state).
// S1K and S2K replace S1 and S2 in the FP32 mode, which is bound by memory
// traffic: S1K stores only k1 (in Qout, 5 planes instead of the
// 10 of acc and Q), and S2K forms Q = q_n + dt/2 k1 while staging its tile
// from q_n and k1 (X) and the accumulator q_n + dt/6 k1 + dt/3 k2 at its
// nodes, with the same roundings in the same order as S1 and S2:
//   S1K: k1 = f(q_n) -> Qout
//   S2K: k2 = f(q_n + dt/2 k1); acc = (q_n + dt/6 k1) + dt/3 k2; Q' = q_n + dt/2 k2
// so that the first two stages move 11 + 21 planes instead of 16 + 26.
// TAPE evaluates f(X) and writes only its tape (the TP_ planes below), the
// intermediate values of the right-hand side that the adjoint kernels read
// instead of recomputing them; FP64 stage kernels instantiated with their
// TAPE flag write the same tape beside the stage update.
enum { MODE_RHS = 0, MODE_S1 = 1, MODE_S2 = 2, MODE_S3 = 3, MODE_S4 = 4, MODE_DIAG = 5, MODE_S4D = 6,
       MODE_S1K = 7, MODE_S2K = 8, MODE_TAPE = 9 };
// Whether RK4 steps use S1K and S2K: the FP32 mode (float state and compute
// type; the mixed mode's S2K, holding double q_n and float k1 of its halo
// nodes, measured 3% slower than S1 and S2).
template <typename TC, typename TA>
constexpr bool kStoreK1 = sizeof(TC) == 4 && sizeof(TA) == 4;

constexpr int TILE_X = 32;
constexpr int THREADS_Y = 8;
constexpr int ROWS_PER_THREAD = 2;
constexpr int TILE_Y = THREADS_Y * ROWS_PER_THREAD;
constexpr int HALO_X = TILE_X + 2;
constexpr int HALO_Y = TILE_Y + 2;
constexpr int HALO_N = HALO_X * HALO_Y;
constexpr int BLOCK_THREADS = TILE_X * THREADS_Y;

// shared-memory planes: the fields h, u, v, w, then rho = eta/h and r = 1/h
// (read at the node only), eta + 3/2 b and P2 = 2g h(h+b) - lam/3 eta^2/h (eta
// and b are differentiated only through these two, see node_rhs_src), and the
// differentiated products
enum {
    OP_H, OP_U, OP_V, OP_W, OP_RHO, OP_R, OP_E15, OP_P2,
    OP_UU, OP_VV, OP_HU, OP_HV, OP_HUV, OP_HUW, OP_HVW, N_OPS
};

// The tape of one right-hand-side evaluation: per node, FP64 values of
// node_rhs_src in its own rounding (the differences are unscaled, f_+ - f_-):
//   R      1/h                       BASE2  -P2/h
//   DXH .. DYF   D_x, D_y of h, u, v, w and eta + 3/2 b
//   DXUU, DYVV   D_x(u^2), D_y(v^2)
//   XHU    D_x(hu) - A_x              YHV    D_y(hv) - A_y
//   AX, AY the continuity fluxes u D_x h + h D_x u, v D_y h + h D_y v
//   KU, KV, KW   the right-hand side of u, v, w
enum {
    TP_R, TP_BASE2, TP_DXH, TP_DYH, TP_DXU, TP_DYU, TP_DXV, TP_DYV, TP_DXW, TP_DYW, TP_DXF, TP_DYF,
    TP_DXUU, TP_DYVV, TP_XHU, TP_YHV, TP_AX, TP_AY, TP_KU, TP_KV, TP_KW, N_TAPE
};

constexpr int NDIAG = 4;
constexpr int FLAG_NONPOSITIVE = 1;
constexpr int FLAG_NONFINITE = 2;
constexpr int FLAG_BOUNDS = 4;

// Checked builds (-DSGN_CHECKED, libsgn_checked.so): the stage kernels fill
// their shared-memory tile with NaN before staging it, so that a tile entry
// read but never written turns the results into NaN, and check every global
// index of the tile loads against its plane; an index out of range sets
// FLAG_BOUNDS and the load is skipped.  A substitute for a memory checker.
#ifdef SGN_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

struct Geom {
    int nx, ny;
    long long plane;       // nx * ny
    double cx2, cy2;       // 1 / (2 dx), 1 / (2 dy): central rows
    double cx1, cy1;       // 1 / dx, 1 / dy: one-sided boundary rows
    double hcx2, hcy2;     // halves of the above (the 1/2 of the split forms folded in)
    double hcx1, hcy1;
    double satx, saty;     // 2 / dx, 2 / dy: SAT weights
    double dx, dy;         // mass-matrix spacing
    double g, lam;
    double lam2, lam3, lam6;  // lambda/2, lambda/3, lambda/6
    double g2, lam23;         // 2 g, 2 lambda/3
    // the same constants rounded to float, so that float kernels never convert
    // (a double-to-float conversion occupies the FP64 pipe), and as df64 pairs
    float f_cx2, f_cy2, f_cx1, f_cy1, f_hcx2, f_hcy2, f_hcx1, f_hcy1, f_satx, f_saty;
    float f_lam, f_lam3, f_g2, f_lam23;
    df64 w_cx2, w_cy2, w_cx1, w_cy1, w_hcx2, w_hcy2, w_hcx1, w_hcy1, w_satx, w_saty;
    df64 w_lam, w_lam3, w_g2, w_lam23;
};

// Host: a double as a df64 pair (hi the nearest float, lo the nearest float
// to the remainder).
inline df64 host_df64(double x) {
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

// Host: fill a Geom for an nx x ny grid with spacing (dx, dy).
inline void fill_geom(Geom& G, int nx, int ny, double dx, double dy, double g, double lam) {
    G.nx = nx;
    G.ny = ny;
    G.plane = (long long)nx * ny;
    G.cx2 = 1.0 / (2.0 * dx);
    G.cy2 = 1.0 / (2.0 * dy);
    G.cx1 = 1.0 / dx;
    G.cy1 = 1.0 / dy;
    G.hcx2 = 0.5 * G.cx2;
    G.hcy2 = 0.5 * G.cy2;
    G.hcx1 = 0.5 * G.cx1;
    G.hcy1 = 0.5 * G.cy1;
    G.satx = 2.0 / dx;
    G.saty = 2.0 / dy;
    G.dx = dx;
    G.dy = dy;
    G.g = g;
    G.lam = lam;
    G.lam2 = lam / 2.0;
    G.lam3 = lam / 3.0;
    G.lam6 = lam / 6.0;
    G.g2 = 2.0 * g;
    G.lam23 = 2.0 * lam / 3.0;
#define SGN_FILL_COPIES_(name) G.f_##name = (float)G.name; G.w_##name = host_df64(G.name)
    SGN_FILL_COPIES_(cx2);
    SGN_FILL_COPIES_(cy2);
    SGN_FILL_COPIES_(cx1);
    SGN_FILL_COPIES_(cy1);
    SGN_FILL_COPIES_(hcx2);
    SGN_FILL_COPIES_(hcy2);
    SGN_FILL_COPIES_(hcx1);
    SGN_FILL_COPIES_(hcy1);
    SGN_FILL_COPIES_(satx);
    SGN_FILL_COPIES_(saty);
    SGN_FILL_COPIES_(lam);
    SGN_FILL_COPIES_(lam3);
    SGN_FILL_COPIES_(g2);
    SGN_FILL_COPIES_(lam23);
#undef SGN_FILL_COPIES_
}

// A grid constant in the compute type TC (the double or the float copy).
template <typename TC>
__device__ __forceinline__ TC gsel(double d, float f, df64 w);
template <>
__device__ __forceinline__ double gsel<double>(double d, float, df64) { return d; }
template <>
__device__ __forceinline__ float gsel<float>(double, float f, df64) { return f; }
template <>
__device__ __forceinline__ df64 gsel<df64>(double, float, df64 w) { return w; }
#define GC(TC, name) gsel<TC>(G.name, G.f_##name, G.w_##name)

// A small literal (0.5, 1, 1.5: exact in float) in the compute type.
template <typename TC>
__device__ __forceinline__ TC tc_const(double d) { return (TC)d; }
template <>
__device__ __forceinline__ df64 tc_const<df64>(double d) { return df64_of_float((float)d); }

// A quiet NaN in the compute type (the poison of checked builds).
template <typename TC>
__device__ __forceinline__ TC poison();
template <>
__device__ __forceinline__ double poison<double>() { return __longlong_as_double(0x7ff8000000000000LL); }
template <>
__device__ __forceinline__ float poison<float>() { return __int_as_float(0x7fc00000); }
template <>
__device__ __forceinline__ df64 poison<df64>() { return {__int_as_float(0x7fc00000), 0.0f}; }

// Conversions between the storage and compute types (df64 by integer
// operations on the bit patterns, see sgn_df64.cuh).
template <typename TO, typename TI>
__device__ __forceinline__ TO cvt(TI x) { return (TO)x; }
template <>
__device__ __forceinline__ df64 cvt<df64, double>(double x) { return df64_from_double(x); }
template <>
__device__ __forceinline__ df64 cvt<df64, df64>(df64 x) { return x; }
template <>
__device__ __forceinline__ double cvt<double, df64>(df64 x) { return double_of_df64(x); }
// float <-> double (the mixed-precision mode) without the FP64-pipe conversion
// instructions: round to nearest even by integer operations, and the exact
// widening of a normal float (below 2^-126 flushes to zero)
template <>
__device__ __forceinline__ float cvt<float, double>(double x) { return float_of_double_rn(x); }
template <>
__device__ __forceinline__ double cvt<double, float>(float x) { return double_of_float_bits(x); }

template <typename TC, typename TIN, typename TA>
struct StageArgs {
    const TIN* X;        // stage input state (5 planes)
    const TC* b;         // bathymetry (1 plane)
    const TA* qn;        // q_n (stages 1-3)
    TA* acc;             // RK accumulator
    TC* Qout;            // next stage state
    TA* out;             // dq (RHS) or q_{n+1} (stage 4)
    double* partials;    // DIAG, S4D: NDIAG doubles per 32 x 8 band (band-major)
    const double* b64;   // DIAG, S4D: bathymetry in double
    int* flag;           // latched error bits
    Geom G;
    TA c_acc, c_q;       // stage coefficients (see the modes)
    TA c_acc1, c_q1;     // S2K: the first stage's dt/6 and dt/2
    double* tape;        // TAPE mode and TAPE-flagged kernels: N_TAPE planes (FP64)
};

template <typename T>
__device__ __forceinline__ T pos_inf();
template <>
__device__ __forceinline__ double pos_inf<double>() { return __longlong_as_double(0x7ff0000000000000LL); }
template <>
__device__ __forceinline__ float pos_inf<float>() { return __int_as_float(0x7f800000); }

// Error bits for a water height: 0 if h is positive and finite.  Tested on the
// bit pattern (integer pipe): positive finite values are exactly the patterns
// strictly between +0 and +inf; NaN (either sign) is non-finite, everything
// else at or below zero (including -inf) is non-positive.
__device__ __forceinline__ int h_flags(double h) {
    const long long bits = __double_as_longlong(h);
    if (bits > 0 && bits < 0x7ff0000000000000LL) return 0;
    const long long mag = bits & 0x7fffffffffffffffLL;
    return (mag > 0x7ff0000000000000LL || bits == 0x7ff0000000000000LL) ? FLAG_NONFINITE : FLAG_NONPOSITIVE;
}
__device__ __forceinline__ int h_flags(float h);
__device__ __forceinline__ int h_flags(df64 h) { return h_flags(h.hi); }
__device__ __forceinline__ int h_flags(float h) {
    const int bits = __float_as_int(h);
    if (bits > 0 && bits < 0x7f800000) return 0;
    const int mag = bits & 0x7fffffff;
    return (mag > 0x7f800000 || bits == 0x7f800000) ? FLAG_NONFINITE : FLAG_NONPOSITIVE;
}

// 1/h.  Double: from the hardware's approximate reciprocal x (PTX
// rcp.approx.ftz.f64, relative error below 2^-19 as measured on B300) one
// third-order step of the reciprocal iteration: with e = 1 - h x,
// 1/h = x / (1 - e) = x (1 + e + e^2 + ...), so x' = x + x (e + e^2) leaves
// the residual 1 - h x' = e^3 (below 2^-57).  This is the truncated series
// 1/(1 - e) = 1 + e + e^2 + ... used for division by functional iteration
// (M. J. Flynn, "On division by functional iteration", IEEE Trans. Computers
// C-19 (1970); J.-M. Muller et al., Handbook of Floating-Point Arithmetic,
// 2nd ed. (2018), the chapter on Newton-Raphson-based division), written out
// as above.  Three fused multiply-adds; the
// result is within one ulp of the correctly rounded quotient (0.03% of values
// one ulp off, none further; tests/test_gpu_recip.py checks this against the
// IEEE division), at a fraction of the FP64-pipe cost of a division.
// Float: the same construction one order lower, x' = x + x e (the Newton
// step for 1/h), from PTX rcp.approx.ftz.f32: the residual e^2 is far below
// half an ulp, and on the test's 1.7e7 values the result equals the correctly
// rounded quotient every time.  Three instructions with no branch, against
// the longer sequence of the IEEE division with its range check; h is a
// water height, positive and normal wherever the kernels use it.
template <typename T>
__device__ __forceinline__ T recip(T h);
template <>
__device__ __forceinline__ double recip<double>(double h) {
    double x;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(h));
    const double e = fma(-h, x, 1.0);
    return fma(x, fma(e, e, e), x);
}
template <>
__device__ __forceinline__ float recip<float>(float h) {
    float x;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(x) : "f"(h));
    return __fmaf_rn(x, __fmaf_rn(-h, x, 1.0f), x);
}
template <>
__device__ __forceinline__ df64 recip<df64>(df64 h) { return recip_df64(h); }

// Element offsets within a plane: 32-bit for the float-based compute types
// (each address one multiply-add from the plane's base; sgn_create and
// sgn_batch_create admit their grids only below 2^32 nodes, which every such
// grid that fits in the device's memory is), 64-bit for FP64.  Measured: the
// mixed-mode step 5% faster, the single-stage FP32 step 0.5%; the FP64 and
// df64 kernels unchanged.
template <typename TC>
constexpr bool kW32 = !std::is_same<TC, double>::value;
template <typename TC>
using SIdx = typename std::conditional<kW32<TC>, unsigned, long long>::type;
// Element c of plane f of a plane-major array (plane size P).
template <bool W32, typename T, typename IX>
__device__ __forceinline__ T& plane_at(T* base, int f, long long P, IX c) {
    if constexpr (W32)
        return (base + f * P)[c];
    else
        return base[f * P + c];
}

// Explicitly rounded arithmetic for the per-node RHS and stage algebra:
// products and sums that the compiler may not fuse, and fused multiply-adds
// where fusion is intended.  Every kernel that inlines the same code then
// rounds identically (the batched and single-grid paths agree bit for bit).
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// The stencil differences f_+ - f_- (df64: without renormalization, see sgn_df64.cuh).
#ifndef SGN_DF64_DIFF
#define SGN_DF64_DIFF 1
#endif
__device__ __forceinline__ double diff_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float diff_(float a, float b) { return __fsub_rn(a, b); }

// Index of the halo node at global coordinate k (k may be -1 or >= n).
template <int BC>
__device__ __forceinline__ int halo_index(int k, int n) {
    if (k < 0) return BC == BC_PERIODIC ? n - 1 : 0;
    if (k >= n) return (BC == BC_PERIODIC && k == n) ? 0 : n - 1;
    return k;
}

// The pointwise operands that do not need the products of the fields: 1/h,
// eta/h, eta + 3/2 b and P2 = 2g h(h+b) - lam/3 eta^2/h, the last formed as
// h (2g (h+b)) - (lam/3 rho) eta.
template <typename TC>
struct PointOps {
    TC r, rho, e15, p2;
};
template <typename TC>
__device__ __forceinline__ PointOps<TC> point_ops(TC h, TC eta, TC bb, const Geom& G) {
    PointOps<TC> o;
    o.r = recip<TC>(h);
    o.rho = mul_(eta, o.r);
    o.e15 = fma_(tc_const<TC>(1.5), bb, eta);
    o.p2 = fma_(h, mul_(GC(TC, g2), add_(h, bb)), -mul_(mul_(GC(TC, lam3), o.rho), eta));
    return o;
}

// The shared-memory operands of one node (see the OP_ planes).
template <typename TC>
__device__ __forceinline__ void make_ops(TC h, TC u, TC v, TC w, TC eta, TC bb, const Geom& G, TC o[N_OPS]) {
    const PointOps<TC> p = point_ops<TC>(h, eta, bb, G);
    const TC hu = mul_(h, u), hv = mul_(h, v);
    o[OP_H] = h;
    o[OP_U] = u;
    o[OP_V] = v;
    o[OP_W] = w;
    o[OP_RHO] = p.rho;
    o[OP_R] = p.r;
    o[OP_E15] = p.e15;
    o[OP_P2] = p.p2;
    o[OP_UU] = mul_(u, u);
    o[OP_VV] = mul_(v, v);
    o[OP_HU] = hu;
    o[OP_HV] = hv;
    o[OP_HUV] = mul_(hu, v);
    o[OP_HUW] = mul_(hu, w);
    o[OP_HVW] = mul_(hv, w);
}

template <typename TC, int HN>
__device__ __forceinline__ void store_operands(TC* __restrict__ sm, int t, TC h, TC u, TC v, TC w,
                                               TC eta, TC bb, const Geom& G) {
    TC o[N_OPS];
    make_ops<TC>(h, u, v, w, eta, bb, G, o);
#pragma unroll
    for (int op = 0; op < N_OPS; op++) sm[op * HN + t] = o[op];
}

// The factored tile (float compute type): only the fields and the pointwise
// operands (1/h, eta/h, eta + 3/2 b, P2) are staged; the products are formed
// from the fields wherever node_rhs asks for them, with the same rounded
// operations as make_ops (so the results are those of the full tile).  Float
// arithmetic is plentiful and the float kernels are bound by memory traffic
// and shared-memory instruction throughput, which this halves.
enum { FP_H, FP_U, FP_V, FP_W, FP_RHO, FP_R, FP_E15, FP_P2, NF_OPS };

template <typename TC>
struct TileLayout {
    static constexpr bool factored = false;
    static constexpr int planes = N_OPS;
};
template <>
struct TileLayout<float> {
    static constexpr bool factored = true;
    static constexpr int planes = NF_OPS;
};

template <typename TC, int HN>
__device__ __forceinline__ void store_operands_factored(TC* __restrict__ sm, int t, TC h, TC u, TC v, TC w,
                                                        TC eta, TC bb, const Geom& G) {
    const PointOps<TC> p = point_ops<TC>(h, eta, bb, G);
    sm[FP_H * HN + t] = h;
    sm[FP_U * HN + t] = u;
    sm[FP_V * HN + t] = v;
    sm[FP_W * HN + t] = w;
    sm[FP_RHO * HN + t] = p.rho;
    sm[FP_R * HN + t] = p.r;
    sm[FP_E15 * HN + t] = p.e15;
    sm[FP_P2 * HN + t] = p.p2;
}


// Where node_rhs reads its operands: position 0 is the node itself, 1-4 its
// left, right, lower and upper neighbours (already resolved to the node itself
// on a reflecting wall, where the one-sided row uses it).
enum { POS_C = 0, POS_L = 1, POS_R = 2, POS_B = 3, POS_T = 4 };

template <typename TC, int HN>
struct SmemOps {            // operands staged in a shared-memory halo tile
    const TC* sm;
    int idx[5];
    __device__ __forceinline__ TC get(int op, int pos) const { return sm[op * HN + idx[pos]]; }
};

template <typename TC, int HN>
struct FactoredOps {        // the factored tile: products formed on request
    const TC* sm;
    int idx[5];
    __device__ __forceinline__ TC at(int plane, int pos) const { return sm[plane * HN + idx[pos]]; }
    __device__ __forceinline__ TC get(int op, int pos) const {
        switch (op) {
        case OP_H: return at(FP_H, pos);
        case OP_U: return at(FP_U, pos);
        case OP_V: return at(FP_V, pos);
        case OP_W: return at(FP_W, pos);
        case OP_RHO: return at(FP_RHO, pos);
        case OP_R: return at(FP_R, pos);
        case OP_E15: return at(FP_E15, pos);
        case OP_P2: return at(FP_P2, pos);
        case OP_UU: {
            const TC u = at(FP_U, pos);
            return mul_(u, u);
        }
        case OP_VV: {
            const TC v = at(FP_V, pos);
            return mul_(v, v);
        }
        case OP_HU: return mul_(at(FP_H, pos), at(FP_U, pos));
        case OP_HV: return mul_(at(FP_H, pos), at(FP_V, pos));
        case OP_HUV: return mul_(mul_(at(FP_H, pos), at(FP_U, pos)), at(FP_V, pos));
        case OP_HUW: return mul_(mul_(at(FP_H, pos), at(FP_U, pos)), at(FP_W, pos));
        default: return mul_(mul_(at(FP_H, pos), at(FP_V, pos)), at(FP_W, pos));   // OP_HVW
        }
    }
};

// Right-hand side at node (gi, gj), its operands read from S (S.get(op, pos)).
// Every term of eq. (sd_periodic_2D_SGN) / (semi_2D) appears once, in a
// regrouping that is exact in real arithmetic and saves operations:
//  - eta and b are differentiated only through eta + 3/2 b and P2:
//    lam/3 (1 - rho) D eta + lam/2 (1 - rho) D b = lam/3 (1 - rho) D(eta + 3/2 b),
//    u D eta + 3/2 u D b = u D(eta + 3/2 b) (D is linear), and
//    g D(h(h+b)) - lam/6 D(eta^2/h) = 1/2 D P2, P2 = 2g h(h+b) - lam/3 eta^2/h;
//  - the coefficient of D h in the u and v brackets,
//    lam/6 rho^2 - g (h+b) = -P2/(2h), comes from P2 at the node (rho = eta/h);
//  - the continuity flux A = u D h + h D u recurs: -1/2 u^2 D h - 1/2 hu D u =
//    -1/2 u A_x, -1/2 uv D_y h - 1/2 hu D_y v = -1/2 u A_y (and the same with v),
//    -uw D_x h - hw D_x u = -w A_x;
//  - the factor 1/2 of the split forms and 1/h go into one scale r/2 per
//    direction, applied once per equation.
// The differences are unscaled (f_+ - f_-); sx, sy hold the operator's row
// factor (1/(2dx) central, 1/dx on a reflecting wall's one-sided row).
// With TAPE, tp (registers) receives the node's tape values (the TP_ enum).
template <typename TC, int BC, typename Src, bool TAPE = false>
__device__ __forceinline__ void node_rhs_src(const Src& S, int gi, int gj, const Geom& G, TC k[5],
                                             TC* tp = nullptr) {
#define TPUT(slot, val)                          \
    do {                                         \
        if constexpr (TAPE) tp[(slot)] = (val);  \
    } while (0)
    TC sx = GC(TC, cx2), sy = GC(TC, cy2), hsx = GC(TC, hcx2), hsy = GC(TC, hcy2);
    if (BC == BC_REFLECTING) {
        // one-sided first/last rows of the reflecting operator: (f1 - f0)/dx
        if (gi == 0 || gi == G.nx - 1) {
            sx = GC(TC, cx1);
            hsx = GC(TC, hcx1);
        }
        if (gj == 0 || gj == G.ny - 1) {
            sy = GC(TC, cy1);
            hsy = GC(TC, hcy1);
        }
    }
#define SM_(op, pos) S.get(op, pos)
#if SGN_DF64_DIFF
#define DXU(op) diff_(SM_(op, POS_R), SM_(op, POS_L))
#define DYU(op) diff_(SM_(op, POS_T), SM_(op, POS_B))
#else
#define DXU(op) sub_(SM_(op, POS_R), SM_(op, POS_L))
#define DYU(op) sub_(SM_(op, POS_T), SM_(op, POS_B))
#endif
    const TC h = SM_(OP_H, POS_C), u = SM_(OP_U, POS_C), v = SM_(OP_V, POS_C), w = SM_(OP_W, POS_C);
    const TC rho = SM_(OP_RHO, POS_C), r = SM_(OP_R, POS_C);
    const TC hu = SM_(OP_HU, POS_C), hv = SM_(OP_HV, POS_C);
    const TC lam = GC(TC, lam), lam23 = GC(TC, lam23);
    const TC hrsx = mul_(r, hsx), hrsy = mul_(r, hsy);          // r/(4dx) central
    const TC base2 = mul_(-SM_(OP_P2, POS_C), r);               // lam/3 rho^2 - 2g (h+b)
    const TC lom2 = fma_(-lam23, rho, lam23);                   // 2 lam/3 (1 - rho)
    TPUT(TP_R, r);
    TPUT(TP_BASE2, base2);

    const TC dxh = DXU(OP_H), dxu = DXU(OP_U), dxv = DXU(OP_V), dxw = DXU(OP_W), dxf = DXU(OP_E15);
    const TC dyh = DYU(OP_H), dyu = DYU(OP_U), dyv = DYU(OP_V), dyw = DYU(OP_W), dyf = DYU(OP_E15);
    const TC Ax = fma_(u, dxh, mul_(h, dxu));                   // u D_x h + h D_x u (unscaled)
    const TC Ay = fma_(v, dyh, mul_(h, dyv));
    TPUT(TP_DXH, dxh); TPUT(TP_DYH, dyh); TPUT(TP_DXU, dxu); TPUT(TP_DYU, dyu);
    TPUT(TP_DXV, dxv); TPUT(TP_DYV, dyv); TPUT(TP_DXW, dxw); TPUT(TP_DYW, dyw);
    TPUT(TP_DXF, dxf); TPUT(TP_DYF, dyf); TPUT(TP_AX, Ax); TPUT(TP_AY, Ay);
    if constexpr (TAPE) {
        // values the expressions below form (the same operations on the same
        // operands, so the same roundings)
        TPUT(TP_XHU, sub_(DXU(OP_HU), Ax));
        TPUT(TP_DXUU, DXU(OP_UU));
        TPUT(TP_YHV, sub_(DYU(OP_HV), Ay));
        TPUT(TP_DYVV, DYU(OP_VV));
    }

    // h_t = -(u D_x h + h D_x u + v D_y h + h D_y v) + SAT
    TC kh = -fma_(sx, Ax, mul_(sy, Ay));
    if (BC == BC_REFLECTING) {
        // M^{-1} R^T B N_x R (hu) + M^{-1} R^T B N_y R (hv); corners get both
        if (gi == 0) kh = fma_(-GC(TC, satx), hu, kh);
        if (gi == G.nx - 1) kh = fma_(GC(TC, satx), hu, kh);
        if (gj == 0) kh = fma_(-GC(TC, saty), hv, kh);
        if (gj == G.ny - 1) kh = fma_(GC(TC, saty), hv, kh);
    }

    // 2h u_t = -[ D_x P2 + (lam/3 rho^2 - 2g(h+b)) D_x h + u (D_x(hu) - A_x) + h D_x(u^2)
    //             + 2 lam/3 (1 - rho) D_x(eta + 3/2 b) ]_x - [ D_y(huv) + hv D_y u - u A_y ]_y
    TC Xu = fma_(base2, dxh, DXU(OP_P2));
    Xu = fma_(u, sub_(DXU(OP_HU), Ax), Xu);
    Xu = fma_(h, DXU(OP_UU), Xu);
    Xu = fma_(lom2, dxf, Xu);
    const TC Yu = fma_(-u, Ay, fma_(hv, dyu, DYU(OP_HUV)));
    const TC ku = -fma_(hrsx, Xu, mul_(hrsy, Yu));
    TPUT(TP_KU, ku);

    // 2h v_t: the same with x and y (and u and v) exchanged
    TC Yv = fma_(base2, dyh, DYU(OP_P2));
    Yv = fma_(v, sub_(DYU(OP_HV), Ay), Yv);
    Yv = fma_(h, DYU(OP_VV), Yv);
    Yv = fma_(lom2, dyf, Yv);
    const TC Xv = fma_(-v, Ax, fma_(hu, dxv, DXU(OP_HUV)));
    const TC kv = -fma_(hrsy, Yv, mul_(hrsx, Xv));
    TPUT(TP_KV, kv);

    // h w_t = lam (1 - rho) - 1/2 [ D_x(huw) + hu D_x w - w A_x + D_y(hvw) + hv D_y w - w A_y ]
    const TC Xw = fma_(-w, Ax, fma_(hu, dxw, DXU(OP_HUW)));
    const TC Yw = fma_(-w, Ay, fma_(hv, dyw, DYU(OP_HVW)));
    const TC kw = fma_(r, fma_(-lam, rho, lam), -fma_(hrsx, Xw, mul_(hrsy, Yw)));
    TPUT(TP_KW, kw);

    // eta_t = w - u D_x(eta + 3/2 b) - v D_y(eta + 3/2 b)
    const TC ke = fma_(-v, mul_(sy, dyf), fma_(-u, mul_(sx, dxf), w));
    k[0] = kh; k[1] = ku; k[2] = kv; k[3] = kw; k[4] = ke;
#undef TPUT
#undef DXU
#undef DYU
#undef SM_
}

// Right-hand side at the node held in shared-memory slot t of a halo tile with
// row stride HX and plane size HN, global (gi, gj).
template <typename TC, int BC, int HX = HALO_X, int HN = HALO_N, bool FACT = TileLayout<TC>::factored,
          bool TAPE = false>
__device__ __forceinline__ void node_rhs(const TC* __restrict__ sm, int t, int gi, int gj,
                                         const Geom& G, TC k[5], TC* tp = nullptr) {
    using Src = typename std::conditional<FACT, FactoredOps<TC, HN>, SmemOps<TC, HN>>::type;
    Src S;
    S.sm = sm;
    S.idx[POS_C] = t;
    S.idx[POS_L] = t - 1;
    S.idx[POS_R] = t + 1;
    S.idx[POS_B] = t - HX;
    S.idx[POS_T] = t + HX;
    if (BC == BC_REFLECTING) {
        if (gi == 0) S.idx[POS_L] = t;
        if (gi == G.nx - 1) S.idx[POS_R] = t;
        if (gj == 0) S.idx[POS_B] = t;
        if (gj == G.ny - 1) S.idx[POS_T] = t;
    }
    node_rhs_src<TC, BC, Src, TAPE>(S, gi, gj, G, k, tp);
}

// Mass weight of node (gi, gj): dx dy, halved on each reflecting wall.
template <int BC>
__device__ __forceinline__ double mass_weight(int gi, int gj, const Geom& G) {
    double wx = G.dx, wy = G.dy;
    if (BC == BC_REFLECTING) {
        if (gi == 0 || gi == G.nx - 1) wx = mul_(0.5, wx);
        if (gj == 0 || gj == G.ny - 1) wy = mul_(0.5, wy);
    }
    return mul_(wx, wy);
}

// Pointwise energy of Thm. 4.1 and its parts, explicitly rounded:
// E = h ((u^2+v^2)/2 + w^2/6 + g/2 (h + 2b) + lambda/6 (eta/h - 1)^2) and the
// shifted E' = E + g b^2/2 = h (kin + w^2/6 + relax) + g/2 (h + b)^2.
struct NodeEnergy {
    double rho, kin, w26, s, E, Es;
};
__device__ __forceinline__ NodeEnergy node_energy(double h, double u, double v, double w, double eta, double bb,
                                                  const Geom& G) {
    NodeEnergy e;
    e.rho = mul_(eta, recip<double>(h));
    const double rm1 = sub_(e.rho, 1.0);
    e.kin = mul_(0.5, fma_(u, u, mul_(v, v)));
    e.w26 = mul_(mul_(w, w), 1.0 / 6.0);
    const double relax = mul_(G.lam6, mul_(rm1, rm1));
    e.E = mul_(h, add_(add_(e.kin, e.w26), fma_(0.5 * G.g, fma_(2.0, bb, h), relax)));
    e.s = add_(h, bb);
    e.Es = fma_(h, add_(add_(e.kin, e.w26), relax), mul_(0.5 * G.g, mul_(e.s, e.s)));
    return e;
}

// Diagnostics of one node, accumulated into dsum: mass M h, energy M E,
// shifted energy M E' (E' = E + g b^2/2) and the rate M <d_q E, k> with the
// derivatives listed after eq. (splitcondition); explicitly rounded.
// The state and the bathymetry are taken as stored (in double), not as the
// compute-type copies of the tile, so that the diagnostics of a float-stage
// context are those of its double state.
template <typename TC, int BC>
__device__ __forceinline__ void node_diag(const double q[5], double bb, int gi, int gj, const Geom& G,
                                          const TC k[5], double dsum[4]) {
    const double h = q[0], u = q[1], v = q[2], w = q[3], eta = q[4];
    const double M = mass_weight<BC>(gi, gj, G);
    const NodeEnergy e = node_energy(h, u, v, w, eta, bb, G);
    const double dEh = add_(add_(e.kin, e.w26), fma_(G.g, e.s, mul_(G.lam6, fma_(-e.rho, e.rho, 1.0))));
    double rate = mul_(dEh, cvt<double>(k[0]));
    rate = fma_(mul_(h, u), cvt<double>(k[1]), rate);
    rate = fma_(mul_(h, v), cvt<double>(k[2]), rate);
    rate = fma_(mul_(mul_(h, w), 1.0 / 3.0), cvt<double>(k[3]), rate);
    rate = fma_(-mul_(G.lam3, sub_(1.0, e.rho)), cvt<double>(k[4]), rate);
    dsum[0] = fma_(M, h, dsum[0]);
    dsum[1] = fma_(M, e.E, dsum[1]);
    dsum[2] = fma_(M, e.Es, dsum[2]);
    dsum[3] = fma_(M, rate, dsum[3]);
}

// Mass and energies of a node's new state (mode S4D): the first three
// diagnostics of node_diag, the same arithmetic.
template <int BC>
__device__ __forceinline__ void node_mass_energy(const double q[5], double bb, int gi, int gj, const Geom& G,
                                                 double dsum[4]) {
    const double M = mass_weight<BC>(gi, gj, G);
    const NodeEnergy e = node_energy(q[0], q[1], q[2], q[3], q[4], bb, G);
    dsum[0] = fma_(M, q[0], dsum[0]);
    dsum[1] = fma_(M, e.E, dsum[1]);
    dsum[2] = fma_(M, e.Es, dsum[2]);
}

// Next stage state Q = q_n + c k in the compute type: in the state type and
// rounded (float, double), or, for df64, entirely in float-pair arithmetic
// (no FP64-pipe instruction).
template <typename TC, typename TA>
__device__ __forceinline__ TC stage_state(TA c, TC k, TA kv, TA qv) {
    return cvt<TC>(fma_(c, kv, qv));
}
template <>
__device__ __forceinline__ df64 stage_state<df64, double>(double c, df64 k, double, double qv) {
    return fma_(df64_from_double(c), k, df64_from_double(qv));
}

// Dynamic shared memory of a stage launch: the halo tile of the operands.
template <typename TC, int MODE, bool FACT = TileLayout<TC>::factored>
constexpr size_t stage_smem_bytes(int rows) {
    return (size_t)(FACT ? (int)NF_OPS : (int)N_OPS) * (TILE_X + 2) * (THREADS_Y * rows + 2) * sizeof(TC);
}

#ifndef SGN_DF64_EARLY
#define SGN_DF64_EARLY 1
#endif
#ifndef SGN_F64_EARLY
#define SGN_F64_EARLY 0
#endif
// The stage inputs of one halo tile held in registers: thread tid holds the
// tile nodes t = tid + k * BLOCK_THREADS, k < NPER.
template <typename TC, int NPER>
struct TileIn {
    TC h[NPER], u[NPER], v[NPER], w[NPER], e[NPER], b[NPER];
    int bad;                                    // FLAG_BOUNDS of checked builds
};

// Global -> registers: the six input planes of the halo tile at (i0, j0)
// (S2K: the stage input formed from q_n and k1 = X, see the modes).
template <typename TC, typename TIN, typename TA, int BC, int HALO_X, int HALO_N, int NPER, int MODE = MODE_RHS>
__device__ __forceinline__ void tile_load(const StageArgs<TC, TIN, TA>& a, const Geom& G, int i0, int j0,
                                          TileIn<TC, NPER>& in) {
    const long long P = G.plane;
    const int tid = threadIdx.y * TILE_X + threadIdx.x;
    in.bad = 0;
    TIN rh[NPER] = {}, ru[NPER] = {}, rv[NPER] = {}, rw[NPER] = {}, re[NPER] = {};
    TA qh[NPER] = {}, qu[NPER] = {}, qv[NPER] = {}, qw[NPER] = {}, qe[NPER] = {};
#pragma unroll
    for (int k = 0; k < NPER; k++) {
        const int t = tid + k * BLOCK_THREADS;
        if (t >= HALO_N) continue;
        const int li = t % HALO_X, lj = t / HALO_X;
        const int gx = halo_index<BC>(i0 - 1 + li, G.nx);
        const int gy = halo_index<BC>(j0 - 1 + lj, G.ny);
        if (kChecked && (gx < 0 || gx >= G.nx || gy < 0 || gy >= G.ny)) {
            in.bad |= FLAG_BOUNDS;
            continue;
        }
        const SIdx<TC> c = (SIdx<TC>)gy * (SIdx<TC>)G.nx + (SIdx<TC>)gx;
        rh[k] = plane_at<kW32<TC>>(a.X, 0, P, c);
        ru[k] = plane_at<kW32<TC>>(a.X, 1, P, c);
        rv[k] = plane_at<kW32<TC>>(a.X, 2, P, c);
        rw[k] = plane_at<kW32<TC>>(a.X, 3, P, c);
        re[k] = plane_at<kW32<TC>>(a.X, 4, P, c);
        if (MODE == MODE_S2K) {
            qh[k] = plane_at<kW32<TC>>(a.qn, 0, P, c);
            qu[k] = plane_at<kW32<TC>>(a.qn, 1, P, c);
            qv[k] = plane_at<kW32<TC>>(a.qn, 2, P, c);
            qw[k] = plane_at<kW32<TC>>(a.qn, 3, P, c);
            qe[k] = plane_at<kW32<TC>>(a.qn, 4, P, c);
        }
        in.b[k] = a.b[c];
    }
    // conversions to the compute type after every load is issued (a conversion
    // right behind its load would wait for it before the next load issues)
#pragma unroll
    for (int k = 0; k < NPER; k++) {
        if constexpr (MODE == MODE_S2K) {
            // Q = q_n + dt/2 k1, as stage 1 forms it (stage_state)
            static_assert(std::is_same<TIN, TC>::value, "S2K stages k1 stored in the compute type");
            in.h[k] = stage_state<TC, TA>(a.c_q1, rh[k], cvt<TA>(rh[k]), qh[k]);
            in.u[k] = stage_state<TC, TA>(a.c_q1, ru[k], cvt<TA>(ru[k]), qu[k]);
            in.v[k] = stage_state<TC, TA>(a.c_q1, rv[k], cvt<TA>(rv[k]), qv[k]);
            in.w[k] = stage_state<TC, TA>(a.c_q1, rw[k], cvt<TA>(rw[k]), qw[k]);
            in.e[k] = stage_state<TC, TA>(a.c_q1, re[k], cvt<TA>(re[k]), qe[k]);
        } else {
            in.h[k] = cvt<TC>(rh[k]);
            in.u[k] = cvt<TC>(ru[k]);
            in.v[k] = cvt<TC>(rv[k]);
            in.w[k] = cvt<TC>(rw[k]);
            in.e[k] = cvt<TC>(re[k]);
        }
    }
}

template <int ROWS>
__host__ __device__ constexpr int tile_nper() {
    return ((TILE_X + 2) * (THREADS_Y * ROWS + 2) + BLOCK_THREADS - 1) / BLOCK_THREADS;
}

// One output tile (TILE_X x 8*ROWS nodes at (i0, j0)) of a stage launch: the
// body shared by the single-grid and the batched kernels.  The pointers of `a`
// address this grid's planes; `G` is its geometry.  DIAG and S4D reduce their
// per-node sums over each 32 x 8 band of the tile (band ry = rows
// j0 + 8 ry .. j0 + 8 ry + 7) in a fixed order and write the band's NDIAG
// sums to partial_band0 + ry * band_stride.  The band sums do not depend on
// the tile height, so every launch shape (and the batched kernel) produces the
// same partials for the same state.
// With TAPE (FP64), every node also writes its tape to a.tape (N_TAPE planes).
template <typename TC, typename TIN, typename TA, int BC, int MODE, int ROWS,
          bool FACT = TileLayout<TC>::factored, bool TAPE = false>
__device__ __forceinline__ void stage_tile(const StageArgs<TC, TIN, TA>& a, const Geom& G, int i0, int j0,
                                           TC* __restrict__ sm, double* partial_band0, long long band_stride) {
    constexpr int ROWS_PER_THREAD = ROWS;
    constexpr int HALO_X = TILE_X + 2;
    constexpr int HALO_N = HALO_X * (THREADS_Y * ROWS + 2);
    const long long P = G.plane;
    const int tid = threadIdx.y * TILE_X + threadIdx.x;

    // Memory-bound (float compute type, FP32 and mixed) variants issue every
    // global load of the block early so that more bytes are in flight: the
    // stage operands of this thread's output nodes first, then all halo-tile
    // inputs of its share of the tile.
    constexpr bool kEarly = sizeof(TC) == 4 || (SGN_DF64_EARLY && std::is_same<TC, df64>::value) ||
                            (SGN_F64_EARLY && std::is_same<TC, double>::value);
    constexpr bool kEarlyStage = kEarly;
    static_assert(kEarly || (MODE != MODE_S1K && MODE != MODE_S2K), "S1K and S2K serve the early-load kernels");
    constexpr int NPER = tile_nper<ROWS>();
    const int gi = i0 + threadIdx.x;
    TA pq[ROWS_PER_THREAD][5], pa[ROWS_PER_THREAD][5];
    TC pk[ROWS_PER_THREAD][5];          // S2K: k1 at this thread's nodes
    if (kEarlyStage && (MODE == MODE_S1 || MODE == MODE_S2 || MODE == MODE_S3 || MODE == MODE_S4 ||
                        MODE == MODE_S4D)) {
#pragma unroll
        for (int ry = 0; ry < ROWS_PER_THREAD; ry++) {
            const int gj = j0 + threadIdx.y + ry * THREADS_Y;
            if (gi >= G.nx || gj >= G.ny) continue;
            const SIdx<TC> c = (SIdx<TC>)gj * (SIdx<TC>)G.nx + (SIdx<TC>)gi;
#pragma unroll
            for (int f = 0; f < 5; f++) {
                if (MODE != MODE_S4 && MODE != MODE_S4D) pq[ry][f] = plane_at<kW32<TC>>(a.qn, f, P, c);
                if (MODE != MODE_S1) pa[ry][f] = plane_at<kW32<TC>>(a.acc, f, P, c);
            }
        }
    }

    // ---- phase 1: halo tile of the inputs and of every differentiated product
    int bad = 0;
    if constexpr (kChecked) {
        constexpr int NP = FACT ? (int)NF_OPS : (int)N_OPS;
        for (int k = tid; k < NP * HALO_N; k += BLOCK_THREADS) sm[k] = poison<TC>();
        __syncthreads();
    }
    if constexpr (MODE == MODE_S2K) {
        // Halo items of this thread: first its own output nodes (one per row
        // of the tile), then, for the first RING threads, one node of the
        // ring around the tile.  Its nodes' q_n and k1 stay in registers for
        // the epilogue, so S2K loads every value once.
        static_assert(std::is_same<TIN, TC>::value, "S2K stages k1 stored in the compute type");
        constexpr int TY = THREADS_Y * ROWS_PER_THREAD;
        constexpr int RING = 2 * HALO_X + 2 * TY;
        constexpr int NIT = ROWS_PER_THREAD + 1;
        static_assert(RING <= BLOCK_THREADS && HALO_N == TILE_X * TY + RING, "one ring node per thread");
        TIN rk[NIT][5];
        TA rq[NIT][5];
        TC rb[NIT];
        int tt[NIT];
#pragma unroll
        for (int k = 0; k < NIT; k++) {
            int t = -1;
            if (k < ROWS_PER_THREAD) {
                t = (threadIdx.y + k * THREADS_Y + 1) * HALO_X + threadIdx.x + 1;
            } else if (tid < RING) {
                const int r = tid;
                if (r < HALO_X) t = r;                                          // row above
                else if (r < 2 * HALO_X) t = (TY + 1) * HALO_X + (r - HALO_X);  // row below
                else if (r < 2 * HALO_X + TY) t = (r - 2 * HALO_X + 1) * HALO_X;               // left column
                else t = (r - 2 * HALO_X - TY + 1) * HALO_X + HALO_X - 1;                     // right column
            }
            tt[k] = t;
            if (t < 0) continue;
            const int gx = halo_index<BC>(i0 - 1 + t % HALO_X, G.nx);
            const int gy = halo_index<BC>(j0 - 1 + t / HALO_X, G.ny);
            if (kChecked && (gx < 0 || gx >= G.nx || gy < 0 || gy >= G.ny)) {
                bad |= FLAG_BOUNDS;
                tt[k] = -1;
                continue;
            }
            const SIdx<TC> c = (SIdx<TC>)gy * (SIdx<TC>)G.nx + (SIdx<TC>)gx;
#pragma unroll
            for (int f = 0; f < 5; f++) {
                rk[k][f] = plane_at<kW32<TC>>(a.X, f, P, c);
                rq[k][f] = plane_at<kW32<TC>>(a.qn, f, P, c);
            }
            rb[k] = a.b[c];
        }
#pragma unroll
        for (int k = 0; k < NIT; k++) {
            if (tt[k] < 0) continue;
            TC y[5];
#pragma unroll
            for (int f = 0; f < 5; f++) y[f] = stage_state<TC, TA>(a.c_q1, rk[k][f], cvt<TA>(rk[k][f]), rq[k][f]);
            bad |= h_flags(y[0]);
            if constexpr (FACT)
                store_operands_factored<TC, HALO_N>(sm, tt[k], y[0], y[1], y[2], y[3], y[4], rb[k], G);
            else
                store_operands<TC, HALO_N>(sm, tt[k], y[0], y[1], y[2], y[3], y[4], rb[k], G);
        }
#pragma unroll
        for (int ry = 0; ry < ROWS_PER_THREAD; ry++)
#pragma unroll
            for (int f = 0; f < 5; f++) {
                pq[ry][f] = rq[ry][f];
                pk[ry][f] = rk[ry][f];
            }
    }
    TileIn<TC, NPER> in;
    if (kEarly && MODE != MODE_S2K) {
        tile_load<TC, TIN, TA, BC, HALO_X, HALO_N, NPER, MODE>(a, G, i0, j0, in);
        bad |= in.bad;
    }
#pragma unroll
    for (int k = 0; k < NPER; k++) {
        if (MODE == MODE_S2K) break;
        const int t = tid + k * BLOCK_THREADS;
        if (t >= HALO_N) continue;
        TC h, u, v, w, eta, bb;
        if (kEarly) {
            if constexpr (kChecked) {            // the early load skipped an out-of-range index
                const int gx = halo_index<BC>(i0 - 1 + t % HALO_X, G.nx);
                const int gy = halo_index<BC>(j0 - 1 + t / HALO_X, G.ny);
                if (gx < 0 || gx >= G.nx || gy < 0 || gy >= G.ny) continue;
            }
            h = in.h[k]; u = in.u[k]; v = in.v[k]; w = in.w[k]; eta = in.e[k]; bb = in.b[k];
        } else {
            const int li = t % HALO_X, lj = t / HALO_X;
            const int gx = halo_index<BC>(i0 - 1 + li, G.nx);
            const int gy = halo_index<BC>(j0 - 1 + lj, G.ny);
            if (kChecked && (gx < 0 || gx >= G.nx || gy < 0 || gy >= G.ny)) {
                bad |= FLAG_BOUNDS;
                continue;
            }
            const SIdx<TC> c = (SIdx<TC>)gy * (SIdx<TC>)G.nx + (SIdx<TC>)gx;
            h = cvt<TC>(plane_at<kW32<TC>>(a.X, 0, P, c));
            u = cvt<TC>(plane_at<kW32<TC>>(a.X, 1, P, c));
            v = cvt<TC>(plane_at<kW32<TC>>(a.X, 2, P, c));
            w = cvt<TC>(plane_at<kW32<TC>>(a.X, 3, P, c));
            eta = cvt<TC>(plane_at<kW32<TC>>(a.X, 4, P, c));
            bb = a.b[c];
        }
        bad |= h_flags(h);
        if constexpr (FACT)
            store_operands_factored<TC, HALO_N>(sm, t, h, u, v, w, eta, bb, G);
        else
            store_operands<TC, HALO_N>(sm, t, h, u, v, w, eta, bb, G);
    }
    if (bad) atomicOr(a.flag, bad);
    __syncthreads();

    // ---- phase 2: right-hand side and stage algebra at this thread's nodes
    double dsum[ROWS_PER_THREAD][NDIAG];
#pragma unroll
    for (int ry = 0; ry < ROWS_PER_THREAD; ry++)
#pragma unroll
        for (int q = 0; q < NDIAG; q++) dsum[ry][q] = 0.0;
#pragma unroll
    for (int ry = 0; ry < ROWS_PER_THREAD; ry++) {
        const int ly = threadIdx.y + ry * THREADS_Y;
        const int gj = j0 + ly;
        if (gi >= G.nx || gj >= G.ny) continue;
        const int t = (ly + 1) * HALO_X + (threadIdx.x + 1);
        TC k[5];
        const SIdx<TC> c = (SIdx<TC>)gj * (SIdx<TC>)G.nx + (SIdx<TC>)gi;
        if constexpr (TAPE) {
            static_assert(std::is_same<TC, double>::value, "the tape is written by the FP64 kernels");
            TC tp[N_TAPE];
            node_rhs<TC, BC, HALO_X, HALO_N, FACT, true>(sm, t, gi, gj, G, k, tp);
#pragma unroll
            for (int p = 0; p < N_TAPE; p++) a.tape[p * P + c] = tp[p];
        } else {
            static_assert(MODE != MODE_TAPE, "the TAPE mode needs the TAPE flag");
            node_rhs<TC, BC, HALO_X, HALO_N, FACT>(sm, t, gi, gj, G, k);
        }
        if (MODE == MODE_RHS) {
#pragma unroll
            for (int f = 0; f < 5; f++) plane_at<kW32<TC>>(a.out, f, P, c) = cvt<TA>(k[f]);
        } else if (MODE == MODE_S1 || MODE == MODE_S2 || MODE == MODE_S3) {
#pragma unroll
            for (int f = 0; f < 5; f++) {
                const TA qv = kEarlyStage ? pq[ry][f] : plane_at<kW32<TC>>(a.qn, f, P, c);
                const TA kv = cvt<TA>(k[f]);
                const TA av = (MODE == MODE_S1) ? qv : (kEarlyStage ? pa[ry][f] : plane_at<kW32<TC>>(a.acc, f, P, c));
                plane_at<kW32<TC>>(a.acc, f, P, c) = fma_(a.c_acc, kv, av);
                plane_at<kW32<TC>>(a.Qout, f, P, c) = stage_state<TC, TA>(a.c_q, k[f], kv, qv);
            }
        } else if (MODE == MODE_S1K) {
#pragma unroll
            for (int f = 0; f < 5; f++) plane_at<kW32<TC>>(a.Qout, f, P, c) = k[f];
        } else if (MODE == MODE_S2K) {
#pragma unroll
            for (int f = 0; f < 5; f++) {
                const TA qv = pq[ry][f];
                const TA kv = cvt<TA>(k[f]);
                plane_at<kW32<TC>>(a.acc, f, P, c) = fma_(a.c_acc, kv, fma_(a.c_acc1, cvt<TA>(pk[ry][f]), qv));
                plane_at<kW32<TC>>(a.Qout, f, P, c) = stage_state<TC, TA>(a.c_q, k[f], kv, qv);
            }
        } else if (MODE == MODE_S4 || MODE == MODE_S4D) {
            double qn1[5];
#pragma unroll
            for (int f = 0; f < 5; f++) {
                const TA o = fma_(a.c_acc, cvt<TA>(k[f]), kEarlyStage ? pa[ry][f] : plane_at<kW32<TC>>(a.acc, f, P, c));
                plane_at<kW32<TC>>(a.out, f, P, c) = o;
                qn1[f] = cvt<double>(o);
            }
            if (MODE == MODE_S4D) node_mass_energy<BC>(qn1, a.b64[c], gi, gj, G, dsum[ry]);
        } else if (MODE == MODE_DIAG) {
            double qd[5];
#pragma unroll
            for (int f = 0; f < 5; f++) qd[f] = cvt<double>(plane_at<kW32<TC>>(a.X, f, P, c));
            node_diag<TC, BC>(qd, a.b64[c], gi, gj, G, k, dsum[ry]);
        }
    }

    if (MODE == MODE_DIAG || MODE == MODE_S4D) {
        // Fixed-order band sums through shared memory (the operand tile is no
        // longer read): value (ry, q) of thread tid at red[(ry NDIAG + q) 256 + tid];
        // warp w sums the pairs (ry, q) = w, w + 8, ...: lane l adds the
        // column-l nodes of the band's eight rows in row order, then a shuffle
        // tree over the lanes.  Nodes outside the grid contribute +0.
        constexpr int NPAIR = ROWS_PER_THREAD * NDIAG;
        static_assert((size_t)(FACT ? (int)NF_OPS : (int)N_OPS) * HALO_N * sizeof(TC) >=
                          (size_t)NPAIR * BLOCK_THREADS * sizeof(double),
                      "the operand tile must hold the band sums");
        double* red = reinterpret_cast<double*>(sm);
        __syncthreads();
#pragma unroll
        for (int ry = 0; ry < ROWS_PER_THREAD; ry++)
#pragma unroll
            for (int q = 0; q < NDIAG; q++) red[(ry * NDIAG + q) * BLOCK_THREADS + tid] = dsum[ry][q];
        __syncthreads();
        const int lane = tid & 31, warp = tid >> 5;
        for (int pr = warp; pr < NPAIR; pr += BLOCK_THREADS / 32) {
            const double* v = red + pr * BLOCK_THREADS;
            double x = v[lane];
#pragma unroll
            for (int r8 = 1; r8 < THREADS_Y; r8++) x += v[r8 * TILE_X + lane];
            for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
            const int ry = pr / NDIAG, q = pr % NDIAG;
            if (lane == 0 && j0 + ry * THREADS_Y < G.ny) partial_band0[ry * band_stride + q] = x;
        }
    }
}

// Tile shape of the single-grid stage kernel per compute type: rows per
// thread (tile height 8 rows) and the blocks per SM the registers must allow
// (measured choices; the macros allow other builds).  FP64 is bound by the
// FP64 pipe: 32x24 tiles (106 KB of operands, two blocks per SM) recompute
// the fewest halo operands.  Float: 32x16, registers for five blocks per SM
// (the FP32 mode; the mixed mode's limit is StageMinBlocks).  df64 is bound by
// the latency of its dependent float operations, so it takes 32x8 tiles and
// four resident blocks.
#ifndef SGN_F64_ROWS
#define SGN_F64_ROWS 3
#endif
#ifndef SGN_DF64_ROWS
#define SGN_DF64_ROWS 1
#endif
#ifndef SGN_DF64_MINB
#define SGN_DF64_MINB 4
#endif
#ifndef SGN_F32_MINB
#define SGN_F32_MINB 5
#endif
template <typename TC>
struct StageShape {
    static constexpr int rows = ROWS_PER_THREAD;
    static constexpr int min_blocks = SGN_F32_MINB;
};
template <>
struct StageShape<double> {
    static constexpr int rows = SGN_F64_ROWS;
    static constexpr int min_blocks = 1;
};
template <>
struct StageShape<df64> {
    static constexpr int rows = SGN_DF64_ROWS;
    static constexpr int min_blocks = SGN_DF64_MINB;
};

// Resident blocks per SM the registers of the stage kernel must allow: the
// compute type's, except for the mixed mode (float RHS, double registers).
#ifndef SGN_MIX_MINB
#define SGN_MIX_MINB 4
#endif
template <typename TC, typename TA>
struct StageMinBlocks {
    static constexpr int value = StageShape<TC>::min_blocks;
};
template <>
struct StageMinBlocks<float, double> {
    static constexpr int value = SGN_MIX_MINB;
};

// S2K holds q_n and k1 of its halo nodes between their loads and the stage
// input they form: with reflecting walls (the one-sided rows and SATs) one
// block per SM fewer than the other stages, which it needs to avoid spills.
// The FP32 S1K and (periodic) S4 move few bytes per node and are bound by
// the latency of their loads: six blocks per SM (40 registers, no spills).
#ifndef SGN_F32_LIGHT_MINB
#define SGN_F32_LIGHT_MINB 6
#endif
template <typename TC, typename TA, int MODE, int BC>
constexpr int kStageMinBlocks =
    (MODE == MODE_S2K && BC == BC_REFLECTING) ? StageMinBlocks<TC, TA>::value - 1
    : (kStoreK1<TC, TA> && (MODE == MODE_S1K || (MODE == MODE_S4 && BC == BC_PERIODIC))) ? SGN_F32_LIGHT_MINB
                                                                                          : StageMinBlocks<TC, TA>::value;

// R: rows per thread (tile height 8 R); the compute type's StageShape, or,
// for FP64 grids whose 32 x 24 tiles would load the SMs unevenly, 1 or 2.
// TAPE: also write the tape of every right-hand-side evaluation (FP64).  The
// tape's values stay in registers until the node's stores; with 32 x 8 and
// 32 x 16 tiles (35 and 73 KB of shared memory) the registers are limited to
// what SGN_TAPE_MINB resident blocks per SM allow (32 x 24 tiles: two blocks
// by shared memory).
#ifndef SGN_TAPE_MINB
#define SGN_TAPE_MINB 3
#endif
template <typename TC, int MODE, int BC, int R, bool TAPE>
constexpr int kStageLaunchMinBlocks =
    TAPE ? (R <= 2 ? SGN_TAPE_MINB : 2) : kStageMinBlocks<TC, TC, MODE, BC>;
template <typename TC, typename TIN, typename TA, int BC, int MODE, int R = StageShape<TC>::rows,
          bool TAPE = false>
__global__ void __launch_bounds__(BLOCK_THREADS,
                                  (TAPE ? kStageLaunchMinBlocks<TC, MODE, BC, R, true>
                                        : kStageMinBlocks<TC, TA, MODE, BC>))
k_stage(StageArgs<TC, TIN, TA> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TC* sm = reinterpret_cast<TC*>(smem_raw);
    // band partials in band-major order: band (blockIdx.y R + ry), column block blockIdx.x
    stage_tile<TC, TIN, TA, BC, MODE, R, TileLayout<TC>::factored, TAPE>(a, a.G, blockIdx.x * TILE_X, blockIdx.y * (THREADS_Y * R), sm,
                                         a.partials ? a.partials + (blockIdx.y * R * (long long)gridDim.x +
                                                                    blockIdx.x) * NDIAG
                                                    : nullptr,
                                         (long long)gridDim.x * NDIAG);
}

// Second pass of the reductions: one block sums the partials (per band for the
// diagnostics, per block for the adaptive error) in a fixed order (each thread
// a strided slice, then a fixed tree).
static __global__ void __launch_bounds__(256) k_reduce_partials(const double* __restrict__ partials,
                                                          long long nblk, double* __restrict__ out) {
    __shared__ double red[256][NDIAG];
    double s[NDIAG] = {0.0, 0.0, 0.0, 0.0};
    for (long long k = threadIdx.x; k < nblk; k += 256)
#pragma unroll
        for (int q = 0; q < NDIAG; q++) s[q] += partials[k * NDIAG + q];
#pragma unroll
    for (int q = 0; q < NDIAG; q++) red[threadIdx.x][q] = s[q];
    __syncthreads();
    for (int stride = 128; stride > 0; stride >>= 1) {
        if ((int)threadIdx.x < stride)
#pragma unroll
            for (int q = 0; q < NDIAG; q++) red[threadIdx.x][q] += red[threadIdx.x + stride][q];
        __syncthreads();
    }
    if (threadIdx.x < NDIAG) out[threadIdx.x] = red[0][threadIdx.x];
}

// Initialization of the auxiliary variables, eq. (initialization):
// eta = h, w = -h (D_x u + D_y v) + 3/2 (u D_x b + v D_y b), evaluated in double.
template <typename TS, int BC>
__global__ void __launch_bounds__(256) k_init_aux(TS* __restrict__ q, const double* __restrict__ b, Geom G) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= G.nx || j >= G.ny) return;
    const long long P = G.plane;
    int il = i - 1, ir = i + 1, jb = j - 1, jt = j + 1;
    double sx = G.cx2, sy = G.cy2;
    if (BC == BC_PERIODIC) {
        if (il < 0) il = G.nx - 1;
        if (ir >= G.nx) ir = 0;
        if (jb < 0) jb = G.ny - 1;
        if (jt >= G.ny) jt = 0;
    } else {
        if (i == 0) { il = 0; sx = G.cx1; }
        if (i == G.nx - 1) { ir = G.nx - 1; sx = G.cx1; }
        if (j == 0) { jb = 0; sy = G.cy1; }
        if (j == G.ny - 1) { jt = G.ny - 1; sy = G.cy1; }
    }
    const long long c = (long long)j * G.nx + i;
    const long long cl = (long long)j * G.nx + il, cr = (long long)j * G.nx + ir;
    const long long cb = (long long)jb * G.nx + i, ct = (long long)jt * G.nx + i;
    const double h = (double)q[c], u = (double)q[P + c], v = (double)q[2 * P + c];
    const double dxu = sx * ((double)q[P + cr] - (double)q[P + cl]);
    const double dyv = sy * ((double)q[2 * P + ct] - (double)q[2 * P + cb]);
    const double dxb = sx * (b[cr] - b[cl]);
    const double dyb = sy * (b[ct] - b[cb]);
    q[3 * P + c] = (TS)(-h * (dxu + dyv) + 1.5 * (u * dxb + v * dyb));
    q[4 * P + c] = (TS)h;
}

template <typename TD>
__global__ void k_convert(const double* __restrict__ src, TD* __restrict__ dst, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        dst[k] = cvt<TD>(src[k]);
}

}  // namespace sgn
