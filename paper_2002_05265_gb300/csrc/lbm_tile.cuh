// Bulk-copy staged step kernel: the copy engine (cp.async.bulk, completing on mbarriers)
// streams the nine pulled row segments of each tile into a ring of shared-memory stages
// while the consumer warps (4, 8 or 16 per CTA, by kernel form) collide the previous tiles
// from shared memory and store their results straight to HBM.  Loads stay in flight
// independently of the collision arithmetic, which the register-staged kernels of
// lbm_device.cuh cannot do once the per-node arithmetic is long (16-bit storage,
// central-moment models).
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
// Several time steps per launch: tile t of step s is the global work item s * T + t (T tiles
// per step), and CTA b takes items b, b + grid, ... in order.  A tile of step s >= 1 may be
// copied only when the rows it pulls from (its own and the neighbouring rows or row blocks)
// are complete in step s - 1.  A signal warp (one lane) follows the consumers: each consumer
// warp, after its stores, adds one to its stage's completion count in shared memory (release
// at CTA scope); when the count shows all consumer warps done with a tile, the signal lane
// issues a GPU-scope fence (cumulative over those stores) and adds one to the tile's per-row
// (per row-block) counter in global memory.  It runs beside the copy pipeline, never gating
// it: the producer reuses a stage as soon as the consumers release it (mbarrier `empty`),
// and the stage counts are monotone, so the signal lane may lag.  The producer reads the
// counters it needs with overlapped relaxed loads, then one acquire fence and one
// async-proxy fence, before it waits for a free stage and issues the copies; the consumers
// never wait on memory fences.  That condition also covers the buffer reuse: the
// rows a tile overwrites were last read by exactly those step s - 1 tiles.  Dependencies
// point to smaller work items only, and the grid is launched cooperatively (all CTAs
// resident), so the waits always end.
//
// Wavefront order (lattices of one geometry): the steps of a launch are interleaved so that
// a unit (row or row block) is advanced again a few units behind the front of the previous
// step, while what that step wrote is still in the L2; the intermediate states then never
// reach HBM (rows are overwritten two steps later while still resident), and a launch of K
// steps moves about one read and two writes of the populations through HBM instead of K of
// each.  Step s visits the units in the order u = (j + s) mod U, j = 0, 1, ..., and unit
// index j of step s is ordered at key j + s * D: the units a tile pulls from in step s - 1
// have j' in {j, j + 1, j + 2} (mod U), so with D >= 3 every dependency has a smaller key,
// across the periodic wrap too.
//
// Stage layout (per population i): [16-byte left chunk][W elements][16-byte right chunk].
// Barriers: full[s] (one producer arrival plus the copies' byte count) and empty[s] (one
// arrival per consumer warp); done[s] counts the consumer warps' completed tiles of stage s.  Every wait is bounded: after about two seconds of waiting a
// thread sets the caller's flag, and the producer first lets its own copies land.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// Kernel forms.  Every form runs the same pipeline (one producer warp, CW consumer warps, one
// signal warp per CTA); they differ in the consumer warps per CTA, the resident CTAs per SM the
// registers are sized for, and the models compiled in:
//  * FORM 0, general: every model, 8 consumer warps, 2 CTAs per SM (FP64: 1).  Serves
//    multi-step launches (groups of small lattices, the adjoint's recomputation), where the
//    row-counter waits want several CTAs per SM.
//  * FORM 1, light: one-step launches whose lattices all run BGK, RM, HM or PR.  FP32: 4
//    consumer warps and 2 CTAs per SM with 110-115 registers (tiles of 512 nodes; measured
//    1.02 of the copy bandwidth at 16384^2 and 1.01 at 4096^2, against 0.98-0.99 for 8 warps
//    at 1 CTA per SM, 0.94 for 4 warps at 3 CTAs per SM with 96 registers, 0.95 for the
//    general form).
//    16-bit: 8 consumer warps at 1 CTA per SM and one pass of 8 nodes per thread with the values
//    kept packed (tile_collide_packed): 16-byte accesses and half the passes, which their short
//    collision affords.  It is a separate kernel because the packed path's register pressure
//    makes the compiler spill in the loop every model shares (measured: the central-moment
//    models then lose 2-4 %, and with 8 nodes at once themselves 3-6 %).
//  * FORM 2, wide: every model, 16 consumer warps at 1 CTA per SM (tiles of 8 KB a plane).
//    Serves one-step launches of the other groups (and of BF16 light-model groups, 0.99-1.00
//    against 0.965-0.98 in the light form): at 16384^2 the central-moment models run at
//    0.98-1.01 (FP32) and 0.99-1.02 (16-bit) of the copy bandwidth, against 0.95-0.96 and
//    0.96-0.99 in the general form; the benchmark's eight 1024^2 lattices one step per launch
//    at 0.97-0.98, against 0.95 in the general form's 100-step launches.  In multi-step launches
//    the single CTA stalls its SM at every row-counter wait (0.83), so those keep the general
//    form.
// Nodes a consumer thread collides per pass (one vector access per population): 16 bytes
// for FP64 / FP32; for the 16-bit types LBM_TILE_HALF_CV nodes (4: 8-byte accesses, two
// passes over a tile).
#ifndef LBM_TILE_HALF_CV
#define LBM_TILE_HALF_CV 4
#endif
#ifndef LBM_TILE_PDL
#define LBM_TILE_PDL 1   // programmatic dependent launch of one-step launches (see the kernel)
#endif
template <typename S, int FORM> struct TileForm {
    static constexpr int CW = FORM == 2 ? 16 : ((FORM == 1 && sizeof(S) == 4) ? 4 : 8);   // consumer warps
    static constexpr int MINB = sizeof(S) == 8 ? 1 : (FORM == 0 ? 2 : ((FORM == 1 && sizeof(S) == 4) ? 2 : 1));
    static constexpr int THREADS = (CW + 2) * 32;   // + producer warp + signal warp
};
template <typename S, int CW> struct Tile {
    static constexpr int VEC = (sizeof(S) == 2) ? LBM_TILE_HALF_CV : 16 / (int)sizeof(S);
    static constexpr int W = CW * 32 * 16 / (int)sizeof(S);   // nodes per tile (CW / 2 KB a plane)
    static constexpr int PASSES = W / (CW * 32 * VEC);         // consumer passes per tile
    static constexpr int H = 16 / (int)sizeof(S);              // elements of one halo chunk
    static constexpr int PLANE = (W + 2 * H) * (int)sizeof(S); // bytes of one population slot
    static constexpr int STAGE = 9 * PLANE;                    // bytes of one stage
};

struct TileEntry {
    const void* buf[2]; // the lattice's two buffers (storage type of the launch): time step s of
    int cur;            // the launch reads buf[(cur + s) & 1] and writes buf[(cur + s + 1) & 1];
    long long ring;     // or, when ring > 0, reads buf[0] + s * ring and writes buf[0] + (s + 1) * ring
                        // (elements; the recomputed states of the adjoint)
    unsigned cbase;     // first completion counter of this lattice (one per row or row block)
    StepArgs a;
    int model;          // lbm::Model
    int eq_order;       // 4, or 2 / 3 (BGK only)
    int ntx;            // segment tiles: tiles per row, ceil(nx / W); row-block tiles: 0
    int rows;           // row-block tiles: rows per tile, floor(W / nx) >= 2; segment tiles: 1
    unsigned begin;     // first tile index of this lattice
};
struct TileArgs {
    int n;              // lattices
    unsigned total;     // tiles of all lattices in one time step
    int nsteps;         // time steps of the launch
    int* flag;          // device int set to 1 when a wait gives up
    unsigned* cnt;      // completion counters, zero at launch (used when nsteps > 1)
    // Work-item order.  wave = 0: step-major (item s * total + t).  wave = 1 (lattices of one
    // geometry: wU units of wntx tiles each): wavefront, item ((k * nsteps + s) * n + e) * wntx
    // + x is segment x of unit u = (k - s * wD + s) mod wU of lattice e at step s, valid when
    // 0 <= k - s * wD < wU; witems items in all.
    // wave = 2: step order with contiguous tiles per CTA: item i = c + gridDim.x * k is the
    // k-th item of CTA c, tile c * wD + (k mod wD) of step k / wD (wD tiles per CTA and step),
    // so a CTA keeps to one lattice (one collision model) within a step.
    int wave, wU, wntx, wD;
    unsigned witems;
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
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void smem_add_release(unsigned* p, unsigned v) {
    asm volatile("red.release.cta.shared::cta.add.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned smem_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
    return v;
}
__device__ __forceinline__ void red_add_relaxed(unsigned* p, unsigned v) {
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// orders this thread's generic-proxy global accesses with its bulk (async-proxy) copies
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
// Waits until all three counters are >= need (relaxed loads, issued together); the caller
// then fences.  False after about two seconds (and at least 2^20 polls).
__device__ __forceinline__ bool counters_wait(const unsigned* a, const unsigned* b, const unsigned* c,
                                              unsigned need) {
    uint64_t t0 = 0;
    for (uint64_t it = 0;; ++it) {
        const unsigned va = ld_relaxed(a), vb = ld_relaxed(b), vc = ld_relaxed(c);
        if (va >= need && vb >= need && vc >= need) return true;
        if (it == 0) t0 = global_ns();
        if ((it & 1023u) == 1023u && it > (1u << 20) && global_ns() - t0 > 2000000000ull) return false;
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
    int unit;   // completion counter of the tile within its lattice: row, or row block
};
template <int W>   // W: nodes per tile of the kernel form
__device__ __forceinline__ TilePos tile_pos(const TileArgs& g, unsigned t) {
    TilePos q;
    int e = 0;
    while (e + 1 < g.n && t >= g.e[e + 1].begin) ++e;
    const TileEntry& E = g.e[e];
    const unsigned lt = t - E.begin;
    q.e = e;
    if (E.ntx > 0) {
        q.y = (int)(lt / (unsigned)E.ntx);
        q.x0 = (int)(lt - (unsigned)q.y * (unsigned)E.ntx) * W;
        q.w = min(W, E.a.nx - q.x0);
        q.rows = 1;
        q.unit = q.y;
    } else {
        q.y = (int)lt * E.rows;
        q.x0 = 0;
        q.w = E.a.nx;
        q.rows = min(E.rows, E.a.ny - q.y);
        q.unit = (int)lt;
    }
    return q;
}

// Work item i -> (step, tile of the step); false for the padding items of the wavefront order.
__device__ __forceinline__ bool item_at(const TileArgs& g, unsigned i, int& step, unsigned& t) {
    if (!g.wave) {
        step = (int)(i / g.total);
        t = i - (unsigned)step * g.total;
        return true;
    }
    if (g.wave == 2) {
        const unsigned c = i % gridDim.x, k = i / gridDim.x;
        step = (int)(k / (unsigned)g.wD);
        t = c * (unsigned)g.wD + (k - (unsigned)step * (unsigned)g.wD);
        return t < g.total;
    }
    const unsigned x = i % (unsigned)g.wntx;
    i /= (unsigned)g.wntx;
    const unsigned e = i % (unsigned)g.n;
    i /= (unsigned)g.n;
    const int s = (int)(i % (unsigned)g.nsteps);
    const int j = (int)(i / (unsigned)g.nsteps) - s * g.wD;
    if (j < 0 || j >= g.wU) return false;
    const unsigned u = (unsigned)(j + s % g.wU) % (unsigned)g.wU;
    const TileEntry& E = g.e[e];
    step = s;
    t = E.begin + (E.ntx > 0 ? u * (unsigned)E.ntx + x : u);
    return true;
}
__device__ __forceinline__ unsigned item_count(const TileArgs& g) {
    return g.wave ? g.witems : (unsigned)g.nsteps * g.total;
}

// ---- consumer: collide VEC nodes of a staged tile --------------------------------------------
template <int MODEL, int EQ, typename S, bool SHIFT, int CW>
__device__ __forceinline__ void tile_collide(const unsigned char* stage, S* dstbuf, const TileEntry& E, const TilePos& q,
                                             int p) {
    using T = typename Conv<S>::T;
    constexpr int VEC = Tile<S, CW>::VEC;
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
        const S* b = reinterpret_cast<const S*>(stage + i * Tile<S, CW>::PLANE + 16);
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
    S* dst = dstbuf + (long long)(q.y + r) * E.a.pitch + q.x0 + x;
#pragma unroll
    for (int i = 0; i < 9; ++i) vstore<S, VEC>(dst + (long long)i * E.a.plane, out[i]);
}

// 16-bit storage, 8 nodes per thread: one 16-byte shared-memory load and one 16-byte global
// store per population; the elements stay packed (two per register) until the node that uses
// them converts its own one (the pull shift only changes which half it reads).
template <typename S> struct Half16;
template <> struct Half16<__half> {
    __device__ static __forceinline__ float lo(uint32_t u) {
        __half2 h;
        memcpy(&h, &u, 4);
        return __low2float(h);
    }
    __device__ static __forceinline__ float hi(uint32_t u) {
        __half2 h;
        memcpy(&h, &u, 4);
        return __high2float(h);
    }
    __device__ static __forceinline__ float one(__half s) { return __half2float(s); }
};
template <> struct Half16<__nv_bfloat16> {
    // a bfloat16 is the upper half of the FP32 with the same value
    __device__ static __forceinline__ float lo(uint32_t u) { return __uint_as_float(u << 16); }
    __device__ static __forceinline__ float hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }
    __device__ static __forceinline__ float one(__nv_bfloat16 s) { return __bfloat162float(s); }
};

template <int MODEL, int EQ, typename S, bool SHIFT, int CW>
__device__ __forceinline__ void tile_collide_packed(const unsigned char* stage, S* dstbuf, const TileEntry& E,
                                                    const TilePos& q, int p) {
    constexpr int VEC = 8;
    const Consts<float> c = make_consts<float>(E.a);
    int r = 0, x = p, li = p - 1, ri = p + VEC;
    if (q.rows > 1 || E.ntx == 0) {
        r = p / q.w;
        x = p - r * q.w;
        if (x == 0) li = p + q.w - 1;
        if (x + VEC == q.w) ri = p + VEC - q.w;
    }
    uint32_t in[9][4];
    float edge[9];   // the element one node left (xi_x = +1) or right (xi_x = -1) of the 8
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const S* b = reinterpret_cast<const S*>(stage + i * Tile<S, CW>::PLANE + 16);
        const uint4 v = *reinterpret_cast<const uint4*>(b + p);
        in[i][0] = v.x; in[i][1] = v.y; in[i][2] = v.z; in[i][3] = v.w;
        edge[i] = ex_of(i) == 1 ? Half16<S>::one(b[li]) : (ex_of(i) == -1 ? Half16<S>::one(b[ri]) : 0.0f);
    }
    uint32_t out[9][4];
    float prev[9];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        float gin[9], gout[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int k = j - ex_of(i);   // element of the slot this node pulls, -1 .. 8
            gin[i] = (k < 0 || k >= VEC) ? edge[i]
                                         : ((k & 1) ? Half16<S>::hi(in[i][k >> 1]) : Half16<S>::lo(in[i][k >> 1]));
        }
        float rho, ux, uy;
        collide<MODEL, EQ, float, SHIFT>(gin, gout, c, rho, ux, uy);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (j & 1) out[i][j >> 1] = pack2(S(), prev[i], gout[i]);
            else prev[i] = gout[i];
        }
    }
    S* dst = dstbuf + (long long)(q.y + r) * E.a.pitch + q.x0 + x;
#pragma unroll
    for (int i = 0; i < 9; ++i)
        *reinterpret_cast<uint4*>(dst + (long long)i * E.a.plane) = make_uint4(out[i][0], out[i][1], out[i][2], out[i][3]);
}

// Collides every node of a staged tile that this consumer thread owns.
template <int MODEL, int EQ, typename S, bool SHIFT, bool PACKED, int CW>
__device__ __forceinline__ void tile_collide_all(const unsigned char* stage, S* dst, const TileEntry& E,
                                                 const TilePos& q) {
    using TS = Tile<S, CW>;
    if constexpr (PACKED && sizeof(S) == 2) {
        static_assert(TS::W == CW * 32 * 8, "one packed pass of 8 nodes per consumer thread covers the tile");
        const int p = (int)threadIdx.x * 8;
        if (p < q.w * q.rows) tile_collide_packed<MODEL, EQ, S, SHIFT, CW>(stage, dst, E, q, p);
    } else {
        // the passes are not unrolled: unrolled, the consumers' code of one model outgrows the
        // instruction cache (ncu, 16-bit K at 8192^2: 2.6x the fetch stalls of CHM, 0.926 of
        // HBM; rolled: the stalls of CHM, 0.956)
#pragma unroll 1
        for (int pass = 0; pass < TS::PASSES; ++pass) {
            const int p = (pass * CW * 32 + (int)threadIdx.x) * TS::VEC;
            if (p < q.w * q.rows) tile_collide<MODEL, EQ, S, SHIFT, CW>(stage, dst, E, q, p);
        }
    }
}

template <typename S, bool SHIFT, int FORM>
__device__ __forceinline__ void tile_consume(const unsigned char* stage, S* dst, const TileEntry& E, const TilePos& q) {
    constexpr int CW = TileForm<S, FORM>::CW;
    if constexpr (FORM == 1) {
        // light form: only the models it is launched for
        switch (E.model) {
            case BGK:
                if (E.eq_order == 2) tile_collide_all<BGK, 2, S, SHIFT, true, CW>(stage, dst, E, q);
                else if (E.eq_order == 3) tile_collide_all<BGK, 3, S, SHIFT, true, CW>(stage, dst, E, q);
                else tile_collide_all<BGK, 4, S, SHIFT, true, CW>(stage, dst, E, q);
                break;
            case RM: tile_collide_all<RM, 4, S, SHIFT, true, CW>(stage, dst, E, q); break;
            case HM: tile_collide_all<HM, 4, S, SHIFT, true, CW>(stage, dst, E, q); break;
            default: tile_collide_all<PR, 4, S, SHIFT, true, CW>(stage, dst, E, q); break;
        }
        return;
    }
    switch (E.model) {
        case BGK:
            if (E.eq_order == 2) tile_collide_all<BGK, 2, S, SHIFT, false, CW>(stage, dst, E, q);
            else if (E.eq_order == 3) tile_collide_all<BGK, 3, S, SHIFT, false, CW>(stage, dst, E, q);
            else tile_collide_all<BGK, 4, S, SHIFT, false, CW>(stage, dst, E, q);
            break;
        case RM: tile_collide_all<RM, 4, S, SHIFT, false, CW>(stage, dst, E, q); break;
        case HM: tile_collide_all<HM, 4, S, SHIFT, false, CW>(stage, dst, E, q); break;
        case CM: tile_collide_all<CM, 4, S, SHIFT, false, CW>(stage, dst, E, q); break;
        case CHM: tile_collide_all<CHM, 4, S, SHIFT, false, CW>(stage, dst, E, q); break;
        case CUM: tile_collide_all<CUM, 4, S, SHIFT, false, CW>(stage, dst, E, q); break;
        case PR: tile_collide_all<PR, 4, S, SHIFT, false, CW>(stage, dst, E, q); break;
        default: tile_collide_all<RR, 4, S, SHIFT, false, CW>(stage, dst, E, q); break;
    }
}

// ---- the kernel ------------------------------------------------------------------------------
// Persistent: CTA b processes tiles b, b + gridDim.x, ...; warps 0 .. CW - 1 consume, warp CW
// is the producer (one lane issues the copies), warp CW + 1 the signal warp.  NS = stages in
// the ring; FORM as in TileForm.  Registers (no spills): general FP32 / 16-bit 96, wide 96,
// light FP32 110-115, light 16-bit 168 (the packed pass; with 4 stages one CTA keeps as many
// bytes in flight as two did with 2).  In a multi-step launch one CTA per SM stalls its SM at
// every row-counter wait (0.49-0.83 against 0.71-0.97 for groups of eight 1024^2 lattices),
// hence the single-CTA forms serve one-step launches.
template <typename S, bool SHIFT, int NS, int FORM>
__global__ void __launch_bounds__(TileForm<S, FORM>::THREADS, TileForm<S, FORM>::MINB)
    tile_step_kernel(const __grid_constant__ TileArgs g) {
    constexpr int CW = TileForm<S, FORM>::CW;
    using TS = Tile<S, CW>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * TS::STAGE);
    uint64_t* empty = full + NS;
    unsigned* done = reinterpret_cast<unsigned*>(empty + NS);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_addr(&full[s]), 1);
            mbar_init(smem_addr(&empty[s]), CW);
            done[s] = 0u;
        }
        mbar_init_fence();
#if LBM_TILE_PDL
        // A one-step launch is made with programmatic stream serialization: the next step's
        // launch may be scheduled now; its CTAs take the SM slots this launch's CTAs free as
        // they exit (every form fills its SMs' registers or shared memory, so none start
        // earlier), overlapping its launch and set-up with this launch's last tiles.
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
    }
    __syncthreads();
    // CTA b takes work items b, b + gridDim.x, ... (all three roles in the same order)
    const unsigned items = item_count(g);

    if (warp == CW + 1) {
        if (lane != 0 || g.nsteps == 1) return;   // a single-step launch has no dependencies
        // ---------------- signal ----------------
        int k = 0;
        for (unsigned i = blockIdx.x; i < items; i += gridDim.x) {
            int step;
            unsigned t;
            if (!item_at(g, i, step, t)) continue;
            const int st = k % NS;
            const unsigned need = (unsigned)CW * (unsigned)(k / NS + 1);
            // all consumer warps done with this tile (monotone count: lagging is harmless)
            bool ok = smem_ld_acquire(&done[st]) >= need;
            if (!ok) {
                const uint64_t w0 = global_ns();
                for (uint64_t it = 0; !ok; ++it) {
                    __nanosleep(64);
                    ok = smem_ld_acquire(&done[st]) >= need;
                    if (!ok && (it & 255u) == 255u && it > (1u << 16) && global_ns() - w0 > 2000000000ull) break;
                }
            }
            if (!ok) {
                atomicExch(g.flag, 1);
                return;
            }
            if (step + 1 < g.nsteps) {
                const TilePos q = tile_pos<TS::W>(g, t);
                fence_acq_rel_gpu();   // the consumers' stores, ordered before by the count
                red_add_relaxed(g.cnt + g.e[q.e].cbase + q.unit, 1u);
            }
            ++k;
        }
        return;
    }

    if (warp == CW) {
        if (lane != 0) return;
        // ---------------- producer ----------------
#if LBM_TILE_PDL
        // Wait until the previous kernel on the stream has completed and its writes are
        // visible (immediate when this launch was not made with programmatic serialization).
        // Every global access of this CTA comes after it: the consumers and the signal warp
        // touch global memory only for tiles whose copies this thread issues afterwards.
        asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
        int k = 0;
        bool ok = true;
        for (unsigned i = blockIdx.x; i < items; i += gridDim.x) {
            int step;
            unsigned t;
            if (!item_at(g, i, step, t)) continue;
            const int st = k % NS;
            const uint32_t ph = (uint32_t)(k / NS) & 1u;
            const TilePos q = tile_pos<TS::W>(g, t);
            const TileEntry& E = g.e[q.e];
            const int nx = E.a.nx, ny = E.a.ny;
            if (step > 0) {
                // the rows this tile pulls from must be complete in the previous step (checked
                // before waiting for the stage, so the counter latency overlaps the consumers)
                const int units = E.ntx > 0 ? ny : (ny + E.rows - 1) / E.rows;
                const unsigned need = (unsigned)step * (unsigned)(E.ntx > 0 ? E.ntx : 1);
                const int um = q.unit == 0 ? units - 1 : q.unit - 1;
                const int up = q.unit == units - 1 ? 0 : q.unit + 1;
                const unsigned* c = g.cnt + E.cbase;
                if (!counters_wait(c + um, c + q.unit, c + up, need)) {
                    ok = false;
                    break;
                }
                fence_acq_rel_gpu();          // acquire: the rows' stores happen before the copies
                fence_proxy_async_global();   // ... including for the copy engine's reads
            }
            // a free stage: every consumer warp has released it
            if (k >= NS && !mbar_wait(smem_addr(&empty[st]), ph ^ 1u)) {
                ok = false;
                break;
            }
            const uint32_t bar = smem_addr(&full[st]);
            const S* src = E.ring > 0 ? static_cast<const S*>(E.buf[0]) + (long long)step * E.ring
                                      : static_cast<const S*>(E.buf[(E.cur + step) & 1]);
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
                for (int pi = 0; pi < 9; ++pi) {
                    const int row = (ey_of(pi) == 1) ? ym : ((ey_of(pi) == -1) ? yp : q.y);
                    const S* r = src + (long long)pi * E.a.plane + (long long)row * E.a.pitch;
                    const uint32_t slot = sb + pi * TS::PLANE;
                    bulk_g2s(slot + 16, r + q.x0, row_bytes, bar);
                    if (ex_of(pi) == 1) bulk_g2s(slot, r + xl, 16, bar);
                    if (ex_of(pi) == -1) bulk_g2s(slot + 16 + row_bytes, r + xr, 16, bar);
                }
            } else {
                // row-block tile: rows y - xi_iy of every population, consecutive rows merged
                mbar_arrive_expect_tx(bar, 9 * (uint32_t)q.rows * row_bytes);
                const bool dense = E.a.pitch == nx;
#pragma unroll
                for (int pi = 0; pi < 9; ++pi) {
                    const S* pl = src + (long long)pi * E.a.plane;
                    const uint32_t slot = sb + pi * TS::PLANE + 16;
                    int r = 0;
                    while (r < q.rows) {
                        int row = q.y + r - ey_of(pi);
                        row = row < 0 ? row + ny : (row >= ny ? row - ny : row);
                        int run = 1;
                        if (dense) {
                            const int lim = min(q.rows - r, ny - row);   // stay inside the plane
                            while (run < lim) {
                                int nr = q.y + r + run - ey_of(pi);
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
            ++k;
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
    for (unsigned i = blockIdx.x; i < items; i += gridDim.x) {
        int step;
        unsigned t;
        if (!item_at(g, i, step, t)) continue;
        const int st = k % NS;
        const uint32_t ph = (uint32_t)(k / NS) & 1u;
        const TilePos q = tile_pos<TS::W>(g, t);
        const TileEntry& E = g.e[q.e];
        S* dst = E.ring > 0 ? static_cast<S*>(const_cast<void*>(E.buf[0])) + (long long)(step + 1) * E.ring
                            : static_cast<S*>(const_cast<void*>(E.buf[(E.cur + step + 1) & 1]));
        // every lane waits (acquiring the copied bytes); the warp leaves together on a timeout
        const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&full[st]), ph));
        if (!ok) {
            if (lane == 0) atomicExch(g.flag, 1);
            return;
        }
        tile_consume<S, SHIFT, FORM>(smem + st * TS::STAGE, dst, E, q);
        __syncwarp();
        if (lane == 0) {
            if (g.nsteps > 1) smem_add_release(&done[st], 1u);   // for the signal warp
            mbar_arrive(smem_addr(&empty[st]));
        }
        ++k;
    }
}

// dynamic shared memory of tile_step_kernel<S, *, NS, FORM>
template <typename S, int FORM> constexpr int tile_smem_bytes(int ns) {
    return ns * Tile<S, TileForm<S, FORM>::CW>::STAGE + 2 * ns * 8 + ns * 4;
}

}  // namespace lbm
