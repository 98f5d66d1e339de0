// sgn_persist.cuh - the persistent RK4 stage kernel of ragged ensembles.
//
// The per-tile batched kernel (sgn_batch.cuh) starts one block per tile; each
// block loads its halo tile, waits for it, computes and stores.  On the float
// ensemble that leaves the stages that move few bytes per node (the first and
// the last: 64 B) latency-bound, with too few loads in flight.  Here a grid of
// resident blocks (blocks per SM x SMs) walks the tile list with a stride of
// the grid size, and while a block evaluates one tile it already fetches the
// next one: the raw stage inputs of the next halo tile (five state planes and
// the bathymetry) are copied into a second shared-memory buffer with cp.async,
// and the next tile's geometry into a second descriptor slot, so the memory
// system always has the next tile's bytes in flight.  The per-node arithmetic
// (store_operands_factored, node_rhs, the stage algebra of the modes S1-S4) is
// that of stage_tile, so the results equal the per-tile kernel's bit for bit.
#pragma once

#include "sgn_batch.cuh"

namespace sgn {

template <typename TC, typename TIN, typename TA>
struct PersistArgs {
    const InstDesc* desc;
    const PTile* tiles;
    long long ntiles;
    const TIN* X;          // packed stage input
    const TC* b;           // packed bathymetry (compute type)
    const TA* qn;
    TA* acc;
    TC* Qout;
    TA* out;
    int* flag;
    int stage;             // 0..3: index into the descriptors' c_acc / c_q
};

__device__ __forceinline__ void cp_async_elem(void* smem, const float* g) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_elem(void* smem, const double* g) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Halo index with the boundary treatment known at run time (halo_index<BC>).
__device__ __forceinline__ int halo_index_rt(int k, int n, bool periodic) {
    if (k < 0) return periodic ? n - 1 : 0;
    if (k >= n) return (periodic && k == n) ? 0 : n - 1;
    return k;
}

// Shared-memory layout of one block: two geometry slots, two raw-input
// buffers (five state planes of TIN, one bathymetry plane of TC, over the halo
// tile), the factored operand tile.
template <typename TC, typename TIN, int ROWS>
struct PersistLayout {
    static constexpr int HX = TILE_X + 2;
    static constexpr int HN = HX * (THREADS_Y * ROWS + 2);
    static constexpr size_t geom = (sizeof(InstDesc) + 15) / 16 * 16;     // one instance descriptor
    static constexpr size_t raw = ((size_t)5 * HN * sizeof(TIN) + (size_t)HN * sizeof(TC) + 15) / 16 * 16;
    static constexpr size_t ops = (size_t)NF_OPS * HN * sizeof(TC);
    static constexpr size_t bytes = 2 * geom + 2 * raw + ops;
};

// Resident blocks per SM the registers must allow: three with 16-node-high
// tiles, four with 8-node-high ones (the most without large spills).
template <int ROWS>
constexpr int kPersistMinBlocks = ROWS == 1 ? 4 : 3;

template <typename TC, typename TIN, typename TA, int MODE, int ROWS>
__global__ void __launch_bounds__(BLOCK_THREADS, kPersistMinBlocks<ROWS>)
k_batch_persist(PersistArgs<TC, TIN, TA> a) {
    static_assert(TileLayout<TC>::factored, "the persistent kernel serves the float compute type");
    static_assert(MODE == MODE_S1 || MODE == MODE_S2 || MODE == MODE_S3 || MODE == MODE_S4, "RK4 stages");
    using L = PersistLayout<TC, TIN, ROWS>;
    constexpr int HX = L::HX, HN = L::HN;
    constexpr int NPER = tile_nper<ROWS>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* rawbase = smem_raw + 2 * L::geom;
    TC* ops = reinterpret_cast<TC*>(smem_raw + 2 * L::geom + 2 * L::raw);
    const int tid = threadIdx.y * TILE_X + threadIdx.x;
    auto desc_slot = [&](int s) { return reinterpret_cast<InstDesc*>(smem_raw + s * L::geom); };
    auto raw_x = [&](int s) { return reinterpret_cast<TIN*>(rawbase + s * L::raw); };
    auto raw_b = [&](int s) { return reinterpret_cast<TC*>(rawbase + s * L::raw + (size_t)5 * HN * sizeof(TIN)); };

    int bad = 0;
    // fetch tile T into buffer s, all by cp.async (nothing waits here): its
    // instance descriptor (geometry and RK coefficients) and the raw inputs of
    // this thread's share of the halo tile
    auto fetch = [&](const PTile& T, int s) {
        static_assert(sizeof(InstDesc) % sizeof(float) == 0, "copied in 4-byte words");
        const float* src = reinterpret_cast<const float*>(&a.desc[T.inst]);
        float* dst = reinterpret_cast<float*>(desc_slot(s));
        for (int k = tid; k < (int)(sizeof(InstDesc) / sizeof(float)); k += BLOCK_THREADS)
            cp_async_elem(dst + k, src + k);
        const bool per = T.bc == BC_PERIODIC;
        const long long P = (long long)T.nx * T.ny;
        const TIN* X = a.X + 5 * T.off;
        const TC* bb = a.b + T.off;
        TIN* rx = raw_x(s);
        TC* rb = raw_b(s);
#pragma unroll
        for (int k = 0; k < NPER; k++) {
            const int t = tid + k * BLOCK_THREADS;
            if (t >= HN) continue;
            const int gx = halo_index_rt(T.i0 - 1 + t % HX, T.nx, per);
            const int gy = halo_index_rt(T.j0 - 1 + t / HX, T.ny, per);
            if (kChecked && (gx < 0 || gx >= T.nx || gy < 0 || gy >= T.ny)) {
                bad |= FLAG_BOUNDS;
                continue;
            }
            const long long c = (long long)gy * T.nx + gx;
#pragma unroll
            for (int f = 0; f < 5; f++) cp_async_elem(rx + f * HN + t, X + f * P + c);
            cp_async_elem(rb + t, bb + c);
        }
        cp_async_commit();
    };

    // one tile: operands of this thread's halo nodes from buffer s, then the
    // right-hand side and the stage algebra at its output nodes
    auto evaluate = [&](const PTile& T, int s, auto bc_tag) {
        constexpr int BC = decltype(bc_tag)::value;
        const InstDesc& d = *desc_slot(s);
        const Geom& G = d.G;
        const long long P = G.plane;
        const long long so = 5 * T.off;
        if constexpr (kChecked) {       // poison the operand tile of every tile
            for (int k = tid; k < (int)(NF_OPS * HN); k += BLOCK_THREADS) ops[k] = poison<TC>();
            __syncthreads();
        }
        const TA c_acc = (TA)d.c_acc[a.stage], c_q = (TA)d.c_q[a.stage];
        const int gi = T.i0 + threadIdx.x;
        // the stage operands at this thread's output nodes, loaded before the
        // operands are formed so that their latency overlaps that work
        TA pq[ROWS][5], pa[ROWS][5];
#pragma unroll
        for (int ry = 0; ry < ROWS; ry++) {
            const int gj = T.j0 + threadIdx.y + ry * THREADS_Y;
            if (gi >= G.nx || gj >= G.ny) continue;
            const long long c = so + (long long)gj * G.nx + gi;
#pragma unroll
            for (int f = 0; f < 5; f++) {
                if (MODE != MODE_S4) pq[ry][f] = a.qn[f * P + c];
                if (MODE != MODE_S1) pa[ry][f] = a.acc[f * P + c];
            }
        }
        const TIN* rx = raw_x(s);
        const TC* rb = raw_b(s);
#pragma unroll
        for (int k = 0; k < NPER; k++) {
            const int t = tid + k * BLOCK_THREADS;
            if (t >= HN) continue;
            if constexpr (kChecked) {
                const int gx = halo_index<BC>(T.i0 - 1 + t % HX, G.nx);
                const int gy = halo_index<BC>(T.j0 - 1 + t / HX, G.ny);
                if (gx < 0 || gx >= G.nx || gy < 0 || gy >= G.ny) continue;
            }
            const TC h = cvt<TC>(rx[t]);
            bad |= h_flags(h);
            store_operands_factored<TC, HN>(ops, t, h, cvt<TC>(rx[HN + t]), cvt<TC>(rx[2 * HN + t]),
                                            cvt<TC>(rx[3 * HN + t]), cvt<TC>(rx[4 * HN + t]), rb[t], G);
        }
        __syncthreads();
#pragma unroll
        for (int ry = 0; ry < ROWS; ry++) {
            const int ly = threadIdx.y + ry * THREADS_Y;
            const int gj = T.j0 + ly;
            if (gi >= G.nx || gj >= G.ny) continue;
            const int t = (ly + 1) * HX + (threadIdx.x + 1);
            TC k[5];
            node_rhs<TC, BC, HX, HN, true>(ops, t, gi, gj, G, k);
            const long long c = so + (long long)gj * G.nx + gi;
            if (MODE == MODE_S4) {
#pragma unroll
                for (int f = 0; f < 5; f++) a.out[f * P + c] = fma_(c_acc, cvt<TA>(k[f]), pa[ry][f]);
            } else {
#pragma unroll
                for (int f = 0; f < 5; f++) {
                    const TA qv = pq[ry][f];
                    const TA kv = cvt<TA>(k[f]);
                    const TA av = (MODE == MODE_S1) ? qv : pa[ry][f];
                    a.acc[f * P + c] = fma_(c_acc, kv, av);
                    a.Qout[f * P + c] = stage_state<TC, TA>(c_q, k[f], kv, qv);
                }
            }
        }
        __syncthreads();        // the operand tile and descriptor slot s are free again
    };

    long long tile = blockIdx.x;
    if (tile >= a.ntiles) return;
    const long long stride = gridDim.x;
    PTile cur = a.tiles[tile];
    // the record of the tile after next is loaded one iteration ahead, so that
    // no fetch waits for a record
    PTile nxt = tile + stride < a.ntiles ? a.tiles[tile + stride] : cur;
    fetch(cur, 0);
    int s = 0;
    for (; tile < a.ntiles; tile += stride) {
        const bool more = tile + stride < a.ntiles;
        const PTile after = tile + 2 * stride < a.ntiles ? a.tiles[tile + 2 * stride] : nxt;
        if (more) {
            fetch(nxt, s ^ 1);          // in flight while this tile is evaluated
            cp_async_wait<1>();         // this tile's copies (this thread's) have landed
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();                // everyone's copies of this tile are visible
        if (cur.bc == BC_REFLECTING)
            evaluate(cur, s, std::integral_constant<int, BC_REFLECTING>{});
        else
            evaluate(cur, s, std::integral_constant<int, BC_PERIODIC>{});
        cur = nxt;
        nxt = after;
        s ^= 1;
    }
    if (bad) atomicOr(a.flag, bad);
}

}  // namespace sgn
