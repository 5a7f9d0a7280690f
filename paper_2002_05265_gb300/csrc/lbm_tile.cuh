// Bulk-copy staged step kernel: the copy engine (cp.async.bulk, completing on mbarriers)
// streams the nine pulled row segments of each tile into a ring of shared-memory stages
// while eight consumer warps collide the previous tiles from shared memory and store their
// results straight to HBM.  Loads stay in flight independently of the collision arithmetic,
// which the register-staged kernels of lbm_device.cuh cannot do once the per-node
// arithmetic is long (16-bit storage, central-moment models).
//
// Two tile shapes, chosen per lattice:
//  * segment tiles (nx > W/2): one row segment of up to W consecutive nodes (the last
//    segment of a row may be shorter).  For population i the segment of row y - xi_iy
//    (periodic) is copied, starting at the tile's first node x0; planes with xi_ix = +1 also
//    take the 16-byte chunk that ends at node x0 - 1 (periodic), planes with xi_ix = -1 the
//    chunk that starts at node x0 + w (periodic);
//  * row-block tiles (nx <= W/2): R = floor(W / nx) whole rows, so that small lattices still
//    give every consumer thread work; the periodic wrap in x stays inside each copied row.
//    Source rows y - xi_iy that are consecutive in memory (pitch == nx) move as one copy.
// Every copy starts on a 16-byte boundary because the kernel is used only for lattices whose
// row length nx * sizeof(S) is a multiple of 16 bytes (rows are padded to a pitch of a
// multiple of 32 elements).  Pull: node x of the tile reads element x - xi_ix of its
// plane's slot, one element left or right of its own vector.
//
// Stage layout (per population i): [16-byte left chunk][W elements][16-byte right chunk].
// Barriers: full[s] (one producer arrival plus the copies' byte count) and empty[s] (one
// arrival per consumer warp).  Every wait is bounded: after about two seconds of waiting a
// thread sets the caller's flag, and the producer first lets its own copies land.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr int kTileConsumerWarps = 8;
constexpr int kTileThreads = (kTileConsumerWarps + 1) * 32;

// Nodes a consumer thread collides per pass (one vector access per population): 16 bytes
// for FP64/FP32; for the 16-bit types LBM_TILE_HALF_CV nodes (4 = 8-byte accesses in two
// passes over a tile, which halves the registers of 8 nodes per pass).
#ifndef LBM_TILE_HALF_CV
#define LBM_TILE_HALF_CV 4
#endif
template <typename S> struct Tile {
    static constexpr int VEC = (sizeof(S) == 2) ? LBM_TILE_HALF_CV : 16 / (int)sizeof(S);
    static constexpr int W = kTileConsumerWarps * 32 * 16 / (int)sizeof(S);   // nodes per tile (4 KB a plane)
    static constexpr int PASSES = W / (kTileConsumerWarps * 32 * VEC);         // consumer passes per tile
    static constexpr int H = 16 / (int)sizeof(S);              // elements of one halo chunk
    static constexpr int PLANE = (W + 2 * H) * (int)sizeof(S); // bytes of one population slot
    static constexpr int STAGE = 9 * PLANE;                    // bytes of one stage
};

struct TileEntry {
    const void* src;    // buffers of the storage type of the launch
    void* dst;
    StepArgs a;
    int model;          // lbm::Model
    int eq_order;       // 4, or 2 (BGK only)
    int ntx;            // segment tiles: tiles per row, ceil(nx / W); row-block tiles: 0
    int rows;           // row-block tiles: rows per tile, floor(W / nx) >= 2; segment tiles: 1
    unsigned begin;     // first tile index of this lattice
};
struct TileArgs {
    int n;              // lattices
    unsigned total;     // tiles of all lattices
    int* flag;          // device int set to 1 when a wait gives up
    TileEntry e[kGroupMax];
};

// ---- shared-memory barriers and the bulk copy (PTX) -------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for the phase of parity `parity` to complete; false after about two seconds of
// polling (and at least 2^20 polls, so a preempted kernel is not cut short).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint64_t it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 1023u) == 0 && it > (1u << 20) && global_ns() - t0 > 2000000000ull) return false;
    }
}
// global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned),
// completing on the transaction count of `bar`
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// ---- tile geometry ------------------------------------------------------------------------
struct TilePos {
    int e;      // lattice
    int y;      // (first) row
    int x0;     // first node of the row segment (0 for row-block tiles)
    int w;      // nodes per row in the tile
    int rows;   // rows in the tile (1 for segment tiles)
};
template <typename S>
__device__ __forceinline__ TilePos tile_pos(const TileArgs& g, unsigned t) {
    TilePos q;
    int e = 0;
    while (e + 1 < g.n && t >= g.e[e + 1].begin) ++e;
    const TileEntry& E = g.e[e];
    const unsigned lt = t - E.begin;
    q.e = e;
    if (E.ntx > 0) {
        q.y = (int)(lt / (unsigned)E.ntx);
        q.x0 = (int)(lt - (unsigned)q.y * (unsigned)E.ntx) * Tile<S>::W;
        q.w = min(Tile<S>::W, E.a.nx - q.x0);
        q.rows = 1;
    } else {
        q.y = (int)lt * E.rows;
        q.x0 = 0;
        q.w = E.a.nx;
        q.rows = min(E.rows, E.a.ny - q.y);
    }
    return q;
}

// ---- consumer: collide VEC nodes of a staged tile --------------------------------------------
template <int MODEL, int EQ, typename S, bool SHIFT>
__device__ __forceinline__ void tile_collide(const unsigned char* stage, const TileEntry& E, const TilePos& q, int p) {
    using T = typename Conv<S>::T;
    constexpr int VEC = Tile<S>::VEC;
    const Consts<T> c = make_consts<T>(E.a);
    // slot indices of the elements one node left of p and one node right of p + VEC - 1:
    // the halo chunks for segment tiles, the other end of the same row for row-block tiles
    int r = 0, x = p, li = p - 1, ri = p + VEC;
    if (q.rows > 1 || E.ntx == 0) {
        r = p / q.w;
        x = p - r * q.w;
        if (x == 0) li = p + q.w - 1;
        if (x + VEC == q.w) ri = p + VEC - q.w;
    }
    T f[9][VEC];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const S* b = reinterpret_cast<const S*>(stage + i * Tile<S>::PLANE + 16);
        T v[VEC];
        vload<S, VEC>(b + p, v);
        if (ex_of(i) == 0) {
#pragma unroll
            for (int j = 0; j < VEC; ++j) f[i][j] = v[j];
        } else if (ex_of(i) == 1) {
            f[i][0] = Conv<S>::to_T(b[li]);
#pragma unroll
            for (int j = 1; j < VEC; ++j) f[i][j] = v[j - 1];
        } else {
#pragma unroll
            for (int j = 0; j < VEC - 1; ++j) f[i][j] = v[j + 1];
            f[i][VEC - 1] = Conv<S>::to_T(b[ri]);
        }
    }
    T out[9][VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        T gin[9], gout[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) gin[i] = f[i][j];
        T rho, ux, uy;
        collide<MODEL, EQ, T, SHIFT>(gin, gout, c, rho, ux, uy);
#pragma unroll
        for (int i = 0; i < 9; ++i) out[i][j] = gout[i];
    }
    S* dst = static_cast<S*>(E.dst) + (long long)(q.y + r) * E.a.pitch + q.x0 + x;
#pragma unroll
    for (int i = 0; i < 9; ++i) vstore<S, VEC>(dst + (long long)i * E.a.plane, out[i]);
}

template <typename S, bool SHIFT>
__device__ __forceinline__ void tile_consume(const unsigned char* stage, const TileEntry& E, const TilePos& q, int p) {
    switch (E.model) {
        case BGK:
            if (E.eq_order == 2) tile_collide<BGK, 2, S, SHIFT>(stage, E, q, p);
            else tile_collide<BGK, 4, S, SHIFT>(stage, E, q, p);
            break;
        case RM: tile_collide<RM, 4, S, SHIFT>(stage, E, q, p); break;
        case HM: tile_collide<HM, 4, S, SHIFT>(stage, E, q, p); break;
        case CM: tile_collide<CM, 4, S, SHIFT>(stage, E, q, p); break;
        case CHM: tile_collide<CHM, 4, S, SHIFT>(stage, E, q, p); break;
        case CUM: tile_collide<CUM, 4, S, SHIFT>(stage, E, q, p); break;
        case PR: tile_collide<PR, 4, S, SHIFT>(stage, E, q, p); break;
        default: tile_collide<RR, 4, S, SHIFT>(stage, E, q, p); break;
    }
}

// ---- the kernel ------------------------------------------------------------------------------
// Persistent: CTA b processes tiles b, b + gridDim.x, ...; warp 8 is the producer (one
// lane issues the copies), warps 0-7 consume.  NS = stages in the ring.
template <typename S, bool SHIFT, int NS>
__global__ void __launch_bounds__(kTileThreads, 1) tile_step_kernel(const __grid_constant__ TileArgs g) {
    using TS = Tile<S>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * TS::STAGE);
    uint64_t* empty = full + NS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_addr(&full[s]), 1);
            mbar_init(smem_addr(&empty[s]), kTileConsumerWarps);
        }
        mbar_init_fence();
    }
    __syncthreads();

    if (warp == kTileConsumerWarps) {
        if (lane != 0) return;
        // ---------------- producer ----------------
        int k = 0;
        bool ok = true;
        for (unsigned t = blockIdx.x; t < g.total; t += gridDim.x, ++k) {
            const int st = k % NS;
            const uint32_t ph = (uint32_t)(k / NS) & 1u;
            if (k >= NS && !mbar_wait(smem_addr(&empty[st]), ph ^ 1u)) {
                ok = false;
                break;
            }
            const TilePos q = tile_pos<S>(g, t);
            const TileEntry& E = g.e[q.e];
            const int nx = E.a.nx, ny = E.a.ny;
            const uint32_t bar = smem_addr(&full[st]);
            const S* src = static_cast<const S*>(E.src);
            const uint32_t sb = smem_addr(smem + st * TS::STAGE);
            const uint32_t row_bytes = (uint32_t)(q.w * (int)sizeof(S));
            if (E.ntx > 0) {
                // segment tile: body + one halo chunk for each x-shifted population
                const int ym = (q.y == 0) ? ny - 1 : q.y - 1;
                const int yp = (q.y == ny - 1) ? 0 : q.y + 1;
                mbar_arrive_expect_tx(bar, 9 * row_bytes + 6 * 16);
                const int xl = (q.x0 == 0) ? nx - TS::H : q.x0 - TS::H;     // chunk ending at x0 - 1
                const int xr = (q.x0 + q.w >= nx) ? 0 : q.x0 + q.w;        // chunk starting at x0 + w
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const int row = (ey_of(i) == 1) ? ym : ((ey_of(i) == -1) ? yp : q.y);
                    const S* r = src + (long long)i * E.a.plane + (long long)row * E.a.pitch;
                    const uint32_t slot = sb + i * TS::PLANE;
                    bulk_g2s(slot + 16, r + q.x0, row_bytes, bar);
                    if (ex_of(i) == 1) bulk_g2s(slot, r + xl, 16, bar);
                    if (ex_of(i) == -1) bulk_g2s(slot + 16 + row_bytes, r + xr, 16, bar);
                }
            } else {
                // row-block tile: rows y - xi_iy of every population, consecutive rows merged
                mbar_arrive_expect_tx(bar, 9 * (uint32_t)q.rows * row_bytes);
                const bool dense = E.a.pitch == nx;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const S* pl = src + (long long)i * E.a.plane;
                    const uint32_t slot = sb + i * TS::PLANE + 16;
                    int r = 0;
                    while (r < q.rows) {
                        int row = q.y + r - ey_of(i);
                        row = row < 0 ? row + ny : (row >= ny ? row - ny : row);
                        int run = 1;
                        if (dense) {
                            const int lim = min(q.rows - r, ny - row);   // stay inside the plane
                            while (run < lim) {
                                int nr = q.y + r + run - ey_of(i);
                                nr = nr < 0 ? nr + ny : (nr >= ny ? nr - ny : nr);
                                if (nr != row + run) break;
                                ++run;
                            }
                        }
                        bulk_g2s(slot + r * row_bytes, pl + (long long)row * E.a.pitch, run * row_bytes, bar);
                        r += run;
                    }
                }
            }
        }
        if (!ok) {
            atomicExch(g.flag, 1);
            // let the copies already issued land before the CTA's shared memory goes away
            for (int j = (k > NS ? k - NS : 0); j < k; ++j)
                mbar_wait(smem_addr(&full[j % NS]), (uint32_t)(j / NS) & 1u);
        }
        return;
    }

    // ---------------- consumers ----------------
    int k = 0;
    for (unsigned t = blockIdx.x; t < g.total; t += gridDim.x, ++k) {
        const int st = k % NS;
        const uint32_t ph = (uint32_t)(k / NS) & 1u;
        const TilePos q = tile_pos<S>(g, t);
        // every lane waits (acquiring the copied bytes); the warp leaves together on a timeout
        const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&full[st]), ph));
        if (!ok) {
            if (lane == 0) atomicExch(g.flag, 1);
            return;
        }
#pragma unroll
        for (int pass = 0; pass < TS::PASSES; ++pass) {
            const int p = (pass * kTileConsumerWarps * 32 + (int)threadIdx.x) * TS::VEC;
            if (p < q.w * q.rows) tile_consume<S, SHIFT>(smem + st * TS::STAGE, g.e[q.e], q, p);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&empty[st]));
    }
}

// dynamic shared memory of tile_step_kernel<S, *, NS>
template <typename S> constexpr int tile_smem_bytes(int ns) { return ns * Tile<S>::STAGE + 2 * ns * 8; }

}  // namespace lbm
