// The C ABI of include/lbm.h: contexts, argument validation, host/device pointer staging,
// time stepping with CUDA-graph replay, blow-up checks and multi-lattice groups.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_tile.cuh"

using lbm::CheckArgs;
using lbm::FieldArgs;
using lbm::StepArgs;

struct lbm_ctx {
    int nx = 0, ny = 0, pitch = 0, nseg = 0, vec = 0;
    int model = 0, storage = 0, eq_order = 4;
    double rho0 = 1.0;
    double urx = 0.0, ury = 0.0;       // shift reference velocity: g = f - f^eq(rho0, u_ref)
    lbm_rates rates{};
    cudaStream_t stream = nullptr;     // caller's stream; all work goes here
    long long plane = 0;               // elements per population plane
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;                       // buffer holding the current state
    long long steps = 0;               // steps since the last init
    const void* kernel = nullptr;      // step kernel for (storage, model, eq_order)
    int grid = 0, block = 256;
    // staging for host pointers, reduction scratch, device-side status
    double* stage = nullptr;
    size_t stage_elems = 0;
    double* partials = nullptr;
    double* red_out = nullptr;         // 8 doubles
    int* status = nullptr;             // device int: 0 or LBM_ERR_BLOWUP
    long long* blowup_step = nullptr;  // device
    long long check_every = 0;
    double ke_ref = 0.0, ke_factor = 1.0, uref_x = 0.0, uref_y = 0.0;
    int path = LBM_PATH_AUTO;          // kernel family (lbm_set_kernel_path)
    int stages = 0;                    // bulk-copy ring stages, 0 = default
    int launch_steps = 0;              // bulk-copy time steps per launch, 0 = default (lbm_set_launch_shape)
    int launch_order = LBM_ORDER_AUTO; // bulk-copy work order
    int tile_form = LBM_FORM_AUTO;     // bulk-copy kernel form (lbm_set_tile_form)
    lbm_group* own_group = nullptr;    // used by lbm_step
    unsigned gen = 0;                  // bumped when kernel arguments change (graphs re-record)
    char err[512] = {0};
};

struct lbm_group {
    std::vector<lbm_ctx*> ctx;
    int fused = 0;                     // one multi-lattice launch per time step
    const void* gkernel[2] = {nullptr, nullptr};   // default shift / reference-velocity shift
    int ggrid[2] = {0, 0};
    std::vector<unsigned> begin;       // padded segment offsets of the contexts
    unsigned padded_total = 0;
    int tiled = 0;                     // bulk-copy staged launches
    int tform = 0;                     // their kernel form: 0 general, 1 light, 2 wide
    int tone = 0;                      // 1: a form that runs one time step per launch by default
    int tthreads = 0;                  // CTA size of the form
    int twidth = 0;                    // nodes per tile of the form
    const void* tkernel[2] = {nullptr, nullptr};   // default shift / reference-velocity shift
    int tgrid[2] = {0, 0};
    int tsmem = 0;                     // dynamic shared memory of the bulk-copy kernel
    std::vector<unsigned> tbegin;      // first tile of each context
    unsigned ttotal = 0;
    std::vector<unsigned> cbase;       // first completion counter of each context
    unsigned* cnt = nullptr;           // completion counters of multi-step launches (device)
    unsigned cunits = 0;
    int same_geometry = 0;             // every context has the same units and tiles per unit
    int wU = 0, wntx = 0;              // that geometry
    long long state_bytes = 0;         // both buffers of every context
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;
    std::vector<cudaStream_t> side;    // concurrent blow-up checks (launch_checks)
    std::vector<cudaEvent_t> side_done;
    cudaEvent_t fork = nullptr;
    int graph_steps = 0;
    cudaGraphExec_t exec = nullptr;
    std::vector<int> exec_parity;      // ctx->cur of each context when the graph was recorded
    std::vector<unsigned> exec_gen;    // ctx->gen of each context when the graph was recorded
    int timing = 0;
    std::vector<cudaEvent_t> ev;       // pairs (start, stop) of timed replays
    size_t ev_used = 0;
    double replay_ms = 0.0;
    long long replay_lattice_steps = 0;
    long long pending_lattice_steps = 0;
    long long replay_kernels = 0;
    long long pending_kernels = 0;
};

namespace {

int set_err(lbm_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define LBM_CK(ctx, call)                                                                       \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return set_err((ctx), e_ == cudaErrorMemoryAllocation ? LBM_ERR_NOMEM : LBM_ERR_CUDA, \
                           "%s failed: %s", #call, cudaGetErrorString(e_));                     \
    } while (0)

bool rate_ok(double w) { return std::isfinite(w) && w > 0.0 && w < 2.0; }

// The cumulant readings LBM_K_PRE / LBM_K_EQ run the kernels of LBM_K with other constants.
int kernel_model(int model) { return (model == LBM_K_PRE || model == LBM_K_EQ) ? LBM_K : model; }
int cumulant_read(int model) { return model == LBM_K_PRE ? 1 : (model == LBM_K_EQ ? 2 : 0); }

bool rates_ok(const lbm_rates& r) { return rate_ok(r.omega_nu) && rate_ok(r.omega3) && rate_ok(r.omega4); }

const void* pick_kernel(int storage, int model, int eq_order, bool shifted) {
    switch (storage) {
        case LBM_F64: return lbm::step_kernel_f64(model, eq_order, shifted);
        case LBM_F32: return lbm::step_kernel_f32(model, eq_order, shifted);
        case LBM_F16: return lbm::step_kernel_f16(model, eq_order, shifted);
        case LBM_BF16: return lbm::step_kernel_bf16(model, eq_order, shifted);
        default: return nullptr;
    }
}

bool is_shifted(const lbm_ctx* c) { return c->urx != 0.0 || c->ury != 0.0; }

// resident-CTA grid for a kernel, capped by the warps of work
int resident_grid(const void* kernel, int block, long long work_threads) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    long long g = (long long)sms * per_sm;
    const long long need = (work_threads + block - 1) / block;
    if (need < g) g = need;
    return (int)(g < 1 ? 1 : g);
}

int select_kernel(lbm_ctx* c) {
    const void* k = pick_kernel(c->storage, kernel_model(c->model), c->eq_order, is_shifted(c));
    if (!k) return set_err(c, LBM_ERR_UNSUPPORTED, "no kernel for this configuration");
    c->kernel = k;
    const long long work = ((long long)c->ny * c->nseg + 31) / 32 * 32;
    c->grid = resident_grid(k, c->block, work);
    return LBM_OK;
}

StepArgs step_args(const lbm_ctx* c) {
    StepArgs a;
    a.nx = c->nx; a.ny = c->ny; a.pitch = c->pitch; a.nseg = c->nseg; a.plane = c->plane;
    a.w_nu = c->rates.omega_nu;
    a.w3 = (c->model == LBM_PR) ? 1.0 : c->rates.omega3;
    a.w4 = (c->model == LBM_PR) ? 1.0 : c->rates.omega4;
    a.rho0 = c->rho0;
    a.urx = c->urx;
    a.ury = c->ury;
    a.kread = cumulant_read(c->model);
    lbm::fill_consts(a);
    return a;
}

FieldArgs field_args(const lbm_ctx* c) {
    FieldArgs a;
    a.nx = c->nx; a.ny = c->ny; a.pitch = c->pitch; a.plane = c->plane; a.rho0 = c->rho0;
    a.urx = c->urx; a.ury = c->ury;
    return a;
}

const void* pick_group_kernel(int storage, bool shifted) {
    switch (storage) {
        case LBM_F64: return lbm::group_kernel_f64(shifted);
        case LBM_F32: return lbm::group_kernel_f32(shifted);
        case LBM_F16: return lbm::group_kernel_f16(shifted);
        case LBM_BF16: return lbm::group_kernel_bf16(shifted);
        default: return nullptr;
    }
}

// rows of a whole number of 16-byte chunks: every bulk copy of the tile kernel is aligned
bool row_aligned(const lbm_ctx* c) { return ((long long)c->nx * lbm::storage_bytes(c->storage)) % 16 == 0; }

bool pick_tile_kernel(int storage, bool shifted, int stages, int form, lbm::TileKernelInfo* out) {
    switch (storage) {
        case LBM_F64: return lbm::tile_kernel_f64(shifted, stages, form, out);
        case LBM_F32: return lbm::tile_kernel_f32(shifted, stages, form, out);
        case LBM_F16: return lbm::tile_kernel_f16(shifted, stages, form, out);
        case LBM_BF16: return lbm::tile_kernel_bf16(shifted, stages, form, out);
        default: return false;
    }
}
// the light kernel form (float, half, bfloat16) serves groups whose lattices all run BGK, RM,
// HM or PR
bool light_model(int m) { return m == LBM_BGK || m == LBM_RM || m == LBM_HM || m == LBM_PR; }
bool light_models(lbm_ctx* const* ctxs, int n) {
    for (int k = 0; k < n; ++k)
        if (!light_model(ctxs[k]->model)) return false;
    return true;
}
// rows per row-block tile (>= 2), or 1 for row-segment tiles
int tile_rows(const lbm_ctx* c, int W) { return 2 * c->nx <= W ? W / c->nx : 1; }
unsigned tile_count(const lbm_ctx* c, int W) {
    const int R = tile_rows(c, W);
    if (R > 1) return (unsigned)((c->ny + R - 1) / R);
    return (unsigned)c->ny * (unsigned)((c->nx + W - 1) / W);
}
// shared-memory stages of the bulk-copy kernel when the caller chose none: 4 for the light
// 16-bit form (one CTA per SM, half-size stages), else 2 (measured at 16384^2: 3 stages lose
// 1-2 % in the general and wide forms, and 3 or 4 lose 2-9 % in the light FP32 forms)
int default_stages(int storage, int form) {
    return (form == 1 && (storage == LBM_F16 || storage == LBM_BF16)) ? 4 : 2;
}
// One-step forms (light, wide): chosen by default when a time step has at least this many
// tiles per resident CTA; below it the fill and drain of every launch's copy pipeline cost
// more than the general form's row-counter waits in multi-step launches (measured, FP32
// groups of 1024^2 lattices: 8 lattices, 27 wide tiles per CTA, 0.97 of the copy bandwidth in
// the wide form against 0.96 in the general form; 6 lattices, 20 per CTA, 0.95 against 0.96).
#ifndef LBM_ONE_STEP_TILES_PER_CTA
#define LBM_ONE_STEP_TILES_PER_CTA 24
#endif

// true when p is device-accessible memory the kernels may read/write directly
bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int ensure_stage(lbm_ctx* c, size_t elems) {
    if (c->stage_elems >= elems) return LBM_OK;
    if (c->stage) {
        LBM_CK(c, cudaStreamSynchronize(c->stream));
        cudaFree(c->stage);
        c->stage = nullptr;
        c->stage_elems = 0;
    }
    LBM_CK(c, cudaMalloc(&c->stage, elems * sizeof(double)));
    c->stage_elems = elems;
    return LBM_OK;
}

int launch_step_once(lbm_ctx* c, cudaStream_t s) {
    StepArgs a = step_args(c);
    const void* src = c->buf[c->cur];
    void* dst = c->buf[c->cur ^ 1];
    void* args[] = {(void*)&src, (void*)&dst, (void*)&a};
    LBM_CK(c, cudaLaunchKernel(c->kernel, dim3(c->grid), dim3(c->block), args, 0, s));
    c->cur ^= 1;
    c->steps += 1;
    return LBM_OK;
}

// one time step of every context of a fused group, as one multi-lattice launch (all contexts
// must agree on the default vs reference-velocity shift)
int launch_group_once(lbm_group* g, cudaStream_t s, int sh) {
    lbm::GroupArgs ga;
    ga.n = (int)g->ctx.size();
    ga.padded_total = g->padded_total;
    for (size_t k = 0; k < g->ctx.size(); ++k) {
        lbm_ctx* c = g->ctx[k];
        lbm::GroupEntry& e = ga.e[k];
        e.src = c->buf[c->cur];
        e.dst = c->buf[c->cur ^ 1];
        e.a = step_args(c);
        e.model = kernel_model(c->model);
        e.eq_order = c->eq_order;
        e.begin = g->begin[k];
        e.total = (unsigned)c->ny * (unsigned)c->nseg;
    }
    void* args[] = {(void*)&ga};
    LBM_CK(g->ctx[0], cudaLaunchKernel(g->gkernel[sh], dim3(g->ggrid[sh]), dim3(256), args, 0, s));
    for (lbm_ctx* c : g->ctx) {
        c->cur ^= 1;
        c->steps += 1;
    }
    return LBM_OK;
}

// Wavefront order: when asked, and by default for a single lattice of a few hundred MB or
// more that runs several steps per launch anyway (measured: 0.95-1.01 of HBM vs 0.92-0.95
// in step order at 4096^2; mixed-model groups and one-step launches lose with it).
bool use_wave(const lbm_group* g) {
    const int order = g->ctx[0]->launch_order;
    if (!g->same_geometry || order == LBM_ORDER_STEP || order == LBM_ORDER_BLOCK) return false;
    if (order == LBM_ORDER_WAVE) return true;
    const int grid = std::max(1, std::max(g->tgrid[0], g->tgrid[1]));
    return g->ctx.size() == 1 && g->state_bytes > (256ll << 20) && g->ttotal < 64u * (unsigned)grid;
}

// bulk-copy staged launch of a tiled group: `nsteps` time steps of every context k, reading
// buf0[k] at the first step (buffers buf0[k] and buf1[k] alternate; with nsteps = 1 they are
// simply source and destination, as for the recomputation ring of the adjoint)
cudaError_t launch_tile(lbm_group* g, const void* const* buf0, void* const* buf1, int nsteps, cudaStream_t s,
                        int sh, long long ring = 0) {
    lbm::TileArgs ta;
    ta.n = (int)g->ctx.size();
    ta.total = g->ttotal;
    ta.nsteps = nsteps;
    ta.flag = g->ctx[0]->status + 1;   // second int of the first context's status word
    ta.cnt = g->cnt;
    const int W = g->twidth;
    for (size_t k = 0; k < g->ctx.size(); ++k) {
        lbm_ctx* c = g->ctx[k];
        lbm::TileEntry& e = ta.e[k];
        e.buf[0] = buf0[k];
        e.buf[1] = buf1[k];
        e.cur = 0;
        e.ring = ring;
        e.cbase = g->cbase[k];
        e.a = step_args(c);
        e.model = kernel_model(c->model);
        e.eq_order = c->eq_order;
        e.rows = tile_rows(c, W);
        e.ntx = e.rows > 1 ? 0 : (c->nx + W - 1) / W;
        e.begin = g->tbegin[k];
    }
    // work order of a multi-step launch: step order (round-robin tiles, or contiguous tiles per
    // CTA), or the wavefront for lattices of one geometry
    ta.wave = 0;
    ta.wU = ta.wntx = ta.wD = 0;
    ta.witems = 0;
    const int order = g->ctx[0]->launch_order;
    unsigned long long items = (unsigned long long)nsteps * g->ttotal;
    if (nsteps > 1 && use_wave(g)) {
        // skew: a dependency lies about two grid-widths of work items back
        const long long per_key = (long long)nsteps * (long long)ta.n * g->wntx;
        const int D = (int)std::max<long long>(4, (2LL * g->tgrid[sh] + per_key - 1) / per_key + 1);
        const unsigned long long w = (unsigned long long)(g->wU + (long long)(nsteps - 1) * D) * per_key;
        if (w < (1ull << 32)) {
            ta.wave = 1;
            ta.wU = g->wU;
            ta.wntx = g->wntx;
            ta.wD = D;
            ta.witems = (unsigned)w;
            items = w;
        }
    }
    int grid = (int)std::min<unsigned long long>((unsigned long long)g->tgrid[sh], items);
    if (nsteps > 1 && !ta.wave && order == LBM_ORDER_BLOCK) {
        // contiguous tiles per CTA: every resident CTA, wD = ceil(total / grid) tiles per step
        grid = g->tgrid[sh];
        ta.wave = 2;
        ta.wD = (int)((g->ttotal + (unsigned)grid - 1) / (unsigned)grid);
        items = (unsigned long long)grid * (unsigned long long)ta.wD * (unsigned long long)nsteps;
        ta.witems = (unsigned)std::min<unsigned long long>(items, 0xffffffffull);
    }
    if (items >= (1ull << 32)) return cudaErrorInvalidValue;   // the caller splits longer runs
    cudaError_t e = cudaSuccess;
    if (nsteps > 1) e = cudaMemsetAsync(g->cnt, 0, sizeof(unsigned) * g->cunits, s);
    if (e != cudaSuccess) return e;
    // wavefront items cycle fastest through segments, lattices and steps (power-of-two
    // extents in practice); an odd grid keeps a CTA from being pinned to one lattice or step
    if (ta.wave == 1 && grid > 1 && (grid % 2) == 0) grid -= 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(g->tthreads);
    cfg.dynamicSmemBytes = (size_t)g->tsmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;   // CTAs of a multi-step launch wait on one another
    attr[0].val.cooperative = nsteps > 1 ? 1 : 0;
    // one-step launches: programmatic dependent launch (the kernel's producer waits for the
    // previous kernel on the stream before its first copy)
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = (LBM_TILE_PDL && nsteps == 1) ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    void* args[] = {(void*)&ta};
    return cudaLaunchKernelExC(&cfg, g->tkernel[sh], args);
}

// `n` time steps of every context of a tiled group in one bulk-copy staged launch
int launch_tile_steps(lbm_group* g, cudaStream_t s, int sh, int n) {
    std::vector<const void*> b0(g->ctx.size());
    std::vector<void*> b1(g->ctx.size());
    for (size_t k = 0; k < g->ctx.size(); ++k) {
        b0[k] = g->ctx[k]->buf[g->ctx[k]->cur];
        b1[k] = g->ctx[k]->buf[g->ctx[k]->cur ^ 1];
    }
    LBM_CK(g->ctx[0], launch_tile(g, b0.data(), b1.data(), n, s, sh));
    for (lbm_ctx* c : g->ctx) {
        c->cur ^= (n & 1);
        c->steps += n;
    }
    return LBM_OK;
}

// shift family of a tiled group's launch: 0 / 1 when every context uses the default /
// reference-velocity shift, -1 when they differ (then each context is stepped on its own)
int tile_shift(const lbm_group* g) {
    int nsh = 0;
    for (lbm_ctx* c : g->ctx) nsh += is_shifted(c) ? 1 : 0;
    return nsh == 0 ? 0 : (nsh == (int)g->ctx.size() ? 1 : -1);
}

int group_step_once(lbm_group* g, cudaStream_t s) {
    if (g->tiled && tile_shift(g) >= 0) return launch_tile_steps(g, s, tile_shift(g), 1);
    if (g->fused) {
        int nsh = 0;
        for (lbm_ctx* c : g->ctx) nsh += is_shifted(c) ? 1 : 0;
        if (nsh == 0) return launch_group_once(g, s, 0);
        if (nsh == (int)g->ctx.size()) return launch_group_once(g, s, 1);
    }
    for (lbm_ctx* c : g->ctx) {
        int rc = launch_step_once(c, s);
        if (rc != LBM_OK) return rc;
    }
    return LBM_OK;
}

// Most time steps in one launch of the bulk-copy kernel (longer runs are split).
#ifndef LBM_TILE_STEPS_PER_LAUNCH
#define LBM_TILE_STEPS_PER_LAUNCH (1 << 20)
#endif

// Steps per launch of a tiled group: a launch whose step has few tiles per CTA loses a
// noticeable share of its time to ramping up and draining the copy pipeline, so such groups
// run many steps per launch in the general form (with the row-completion counters); the
// one-step forms (light, wide) and large lattices run one step per launch, where the
// counters' fences would only add latency to the copy pipeline.
int tile_steps_per_launch(const lbm_group* g) {
    int per;
    if (g->ctx[0]->launch_steps > 0) {
        per = g->ctx[0]->launch_steps;
    } else if (g->tone) {
        per = 1;
    } else if (use_wave(g)) {
        per = 16;   // wavefront: the intermediate states stay in the L2
    } else {
        const int grid = std::max(1, std::max(g->tgrid[0], g->tgrid[1]));
        per = g->ttotal < 64u * (unsigned)grid ? LBM_TILE_STEPS_PER_LAUNCH : 1;
    }
    // keep the work items of one launch within 32 bits
    const long long cap = std::max<long long>(1, ((1ll << 31) / std::max(1u, g->ttotal)) / 2);
    return (int)std::min<long long>(std::min<long long>(per, cap), LBM_TILE_STEPS_PER_LAUNCH);
}

// n time steps of the group: bulk-copy launches for a tiled group, else n launches
int group_advance(lbm_group* g, cudaStream_t s, long long n) {
    if (n <= 0) return LBM_OK;
    if (g->tiled && tile_shift(g) >= 0) {
        const int per = tile_steps_per_launch(g);
        for (long long done = 0; done < n;) {
            const int chunk = (int)std::min<long long>(n - done, per);
            int rc = launch_tile_steps(g, s, tile_shift(g), chunk);
            if (rc != LBM_OK) return rc;
            done += chunk;
        }
        return LBM_OK;
    }
    for (long long t = 0; t < n; ++t) {
        int rc = group_step_once(g, s);
        if (rc != LBM_OK) return rc;
    }
    return LBM_OK;
}

int launch_check(lbm_ctx* c, double* out8_dev, int apply, cudaStream_t s = nullptr) {
    if (!s) s = c->stream;
    CheckArgs ck;
    ck.ke_ref = c->ke_ref; ck.ke_factor = c->ke_factor; ck.uref_x = c->uref_x; ck.uref_y = c->uref_y;
    ck.step = c->steps; ck.apply = apply;
    unsigned* counter = reinterpret_cast<unsigned*>(c->partials + 8 * lbm::reduce_blocks());
    LBM_CK(c, lbm::launch_reduce(c->storage, c->buf[c->cur], field_args(c), c->partials, counter, out8_dev,
                                 c->status, c->blowup_step, ck, s));
    return LBM_OK;
}

// The blow-up checks of several contexts of a group that fall due together: one check is a
// short, single-wave reduction (about 23 us for a 1024^2 FP32 lattice, SMs 59 % active), so
// run one after another they leave most of the GPU idle.  Contexts of one storage type share
// one launch (lbm::launch_reduce_group, each context's results bitwise those of its own
// check); otherwise each check runs on its own stream forked from and joined back to the
// group's stream.  Each context has its own scratch, result and status words.
int launch_checks(lbm_group* g, const std::vector<lbm_ctx*>& due) {
    lbm_ctx* c0 = g->ctx[0];
    bool one = due.size() >= 2 && due.size() <= (size_t)lbm::kReduceGroupMax;
    for (lbm_ctx* c : due) one = one && c->storage == due[0]->storage;
    if (one) {
        lbm::ReduceGroupArgs ra;
        ra.n = (int)due.size();
        for (size_t k = 0; k < due.size(); ++k) {
            lbm_ctx* c = due[k];
            lbm::ReduceJob& J = ra.j[k];
            J.buf = c->buf[c->cur];
            J.a = field_args(c);
            J.partials = c->partials;
            J.counter = reinterpret_cast<unsigned*>(c->partials + 8 * lbm::reduce_blocks());
            J.out = c->red_out;
            J.status = c->status;
            J.blowup_step = c->blowup_step;
            J.c.ke_ref = c->ke_ref; J.c.ke_factor = c->ke_factor; J.c.uref_x = c->uref_x; J.c.uref_y = c->uref_y;
            J.c.step = c->steps; J.c.apply = 1;
        }
        LBM_CK(c0, lbm::launch_reduce_group(due[0]->storage, ra, g->stream));
        return LBM_OK;
    }
    if (due.size() < 2) {
        for (lbm_ctx* c : due) {
            int rc = launch_check(c, c->red_out, 1);
            if (rc != LBM_OK) return rc;
        }
        return LBM_OK;
    }
    while (g->side.size() < due.size()) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        LBM_CK(c0, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        g->side.push_back(st);
        LBM_CK(c0, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        g->side_done.push_back(ev);
    }
    if (!g->fork) LBM_CK(c0, cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming));
    LBM_CK(c0, cudaEventRecord(g->fork, g->stream));
    for (size_t k = 0; k < due.size(); ++k) {
        LBM_CK(c0, cudaStreamWaitEvent(g->side[k], g->fork, 0));
        int rc = launch_check(due[k], due[k]->red_out, 1, g->side[k]);
        if (rc != LBM_OK) return rc;
        LBM_CK(c0, cudaEventRecord(g->side_done[k], g->side[k]));
        LBM_CK(c0, cudaStreamWaitEvent(g->stream, g->side_done[k], 0));
    }
    return LBM_OK;
}


int group_record(lbm_group* g) {
    lbm_ctx* c0 = g->ctx[0];
    if (g->exec) {
        cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
    }
    // record on the private stream; the buffers alternate, so after an even number of steps
    // every context is back on the buffer it started from and the graph can be replayed
    std::vector<int> cur0(g->ctx.size());
    std::vector<long long> steps0(g->ctx.size());
    for (size_t k = 0; k < g->ctx.size(); ++k) { cur0[k] = g->ctx[k]->cur; steps0[k] = g->ctx[k]->steps; }
    LBM_CK(c0, cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeThreadLocal));
    int rc = LBM_OK;
    rc = group_advance(g, g->capture, g->graph_steps);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(g->capture, &graph);
    for (size_t k = 0; k < g->ctx.size(); ++k) { g->ctx[k]->cur = cur0[k]; g->ctx[k]->steps = steps0[k]; }
    if (rc != LBM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return set_err(c0, LBM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g->exec = nullptr;
        return set_err(c0, LBM_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    g->exec_parity = cur0;
    g->exec_gen.resize(g->ctx.size());
    for (size_t k = 0; k < g->ctx.size(); ++k) g->exec_gen[k] = g->ctx[k]->gen;
    return LBM_OK;
}

int group_replay(lbm_group* g) {
    lbm_ctx* c0 = g->ctx[0];
    bool same = g->exec != nullptr;
    for (size_t k = 0; same && k < g->ctx.size(); ++k)
        same = (g->ctx[k]->cur == g->exec_parity[k]) && (g->ctx[k]->gen == g->exec_gen[k]);
    if (!same) {
        int rc = group_record(g);
        if (rc != LBM_OK) return rc;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (g->timing) {
        if (g->ev_used + 2 > g->ev.size()) {
            for (int k = 0; k < 2; ++k) {
                cudaEvent_t ev;
                LBM_CK(c0, cudaEventCreate(&ev));
                g->ev.push_back(ev);
            }
        }
        e0 = g->ev[g->ev_used];
        e1 = g->ev[g->ev_used + 1];
        g->ev_used += 2;
        LBM_CK(c0, cudaEventRecord(e0, g->stream));
    }
    LBM_CK(c0, cudaGraphLaunch(g->exec, g->stream));
    if (g->timing) {
        LBM_CK(c0, cudaEventRecord(e1, g->stream));
        g->pending_lattice_steps += (long long)g->graph_steps * (long long)g->ctx.size();
        g->pending_kernels += (g->tiled && tile_shift(g) >= 0)
                                  ? (long long)(g->graph_steps + tile_steps_per_launch(g) - 1) / tile_steps_per_launch(g)
                                  : (long long)g->graph_steps * (g->fused ? 1LL : (long long)g->ctx.size());
    }
    for (lbm_ctx* c : g->ctx) c->steps += g->graph_steps;   // even: buffers end where they began
    return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_version(void) { return "liblbm 1.0 (D2Q9, sm_103a)"; }

const char* lbm_error_string(int code) {
    switch (code) {
        case LBM_OK: return "ok";
        case LBM_ERR_INVALID_ARG: return "invalid argument";
        case LBM_ERR_UNSUPPORTED: return "unsupported";
        case LBM_ERR_CUDA: return "CUDA error";
        case LBM_ERR_BLOWUP: return "blow-up detected";
        case LBM_ERR_TIMEOUT: return "device wait timed out";
        case LBM_ERR_NOMEM: return "out of device memory";
        default: return "unknown error";
    }
}

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->err : "null context"; }

int lbm_rates_from_nu(double nu, int preset, lbm_rates* out) {
    if (!out || !std::isfinite(nu) || nu <= 0.0) return LBM_ERR_INVALID_ARG;
    const double w = 1.0 / (nu * 3.0 + 0.5);   // omega_nu = 1 / (nu / c_s^2 + 1/2)
    if (preset == LBM_PRESET_SRT) {
        *out = lbm_rates{w, w, w};
    } else if (preset == LBM_PRESET_REG) {
        *out = lbm_rates{w, 1.0, 1.0};
    } else {
        return LBM_ERR_INVALID_ARG;
    }
    return LBM_OK;
}

int lbm_create(lbm_ctx** out, int nx, int ny, int periodic, int model, lbm_rates rates, int eq_order,
               int storage, double rho0, void* cuda_stream) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (nx < 3 || ny < 3 || (long long)nx * (long long)ny > (1LL << 31)) return LBM_ERR_INVALID_ARG;
    if (model < LBM_BGK || model > LBM_K_EQ || storage < LBM_F64 || storage > LBM_BF16) return LBM_ERR_INVALID_ARG;
    if (!rates_ok(rates) || !(std::isfinite(rho0) && rho0 > 0.0)) return LBM_ERR_INVALID_ARG;
    if (eq_order < 2 || eq_order > 4) return LBM_ERR_INVALID_ARG;
    if (periodic != 1) return LBM_ERR_UNSUPPORTED;
    if (eq_order != 4 && model != LBM_BGK) return LBM_ERR_UNSUPPORTED;

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ERR_NOMEM;
    c->nx = nx; c->ny = ny; c->model = model; c->storage = storage; c->eq_order = eq_order;
    c->rho0 = rho0; c->rates = rates; c->stream = (cudaStream_t)cuda_stream;
    c->vec = lbm::storage_vec(storage);
    c->pitch = (nx + 31) / 32 * 32;
    c->nseg = (nx + c->vec - 1) / c->vec;
    c->plane = (long long)ny * c->pitch;
    int rc = LBM_OK;
    const size_t bytes = (size_t)9 * (size_t)c->plane * (size_t)lbm::storage_bytes(storage);
    do {
        rc = select_kernel(c);
        if (rc != LBM_OK) break;
        cudaError_t e;
        for (int b = 0; b < 2; ++b) {
            e = cudaMalloc(&c->buf[b], bytes);
            if (e != cudaSuccess) break;
            e = cudaMemsetAsync(c->buf[b], 0, bytes, c->stream);
            if (e != cudaSuccess) break;
        }
        if (e == cudaSuccess) e = cudaMalloc(&c->partials, lbm::reduce_scratch_bytes());
        if (e == cudaSuccess) e = cudaMemsetAsync(c->partials, 0, lbm::reduce_scratch_bytes(), c->stream);
        if (e == cudaSuccess) e = cudaMalloc(&c->red_out, sizeof(double) * 8);
        if (e == cudaSuccess) e = cudaMalloc(&c->status, sizeof(int) + sizeof(long long) * 2);
        if (e == cudaSuccess) {
            c->blowup_step = reinterpret_cast<long long*>(reinterpret_cast<char*>(c->status) + sizeof(long long));
            e = cudaMemsetAsync(c->status, 0, sizeof(long long), c->stream);
        }
        if (e == cudaSuccess) {
            const long long minus1 = -1;
            e = cudaMemcpyAsync(c->blowup_step, &minus1, sizeof(minus1), cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        }
        if (e != cudaSuccess) {
            rc = (e == cudaErrorMemoryAllocation) ? LBM_ERR_NOMEM : LBM_ERR_CUDA;
            set_err(c, rc, "create: %s", cudaGetErrorString(e));
            break;
        }
    } while (0);
    if (rc != LBM_OK) {
        lbm_destroy(c);
        return rc;
    }
    *out = c;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    if (c->stream || c->buf[0]) cudaStreamSynchronize(c->stream);
    if (c->own_group) lbm_group_destroy(c->own_group);
    for (int b = 0; b < 2; ++b) if (c->buf[b]) cudaFree(c->buf[b]);
    if (c->stage) cudaFree(c->stage);
    if (c->partials) cudaFree(c->partials);
    if (c->red_out) cudaFree(c->red_out);
    if (c->status) cudaFree(c->status);
    delete c;
}

int lbm_set_rates(lbm_ctx* c, lbm_rates r) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (!rates_ok(r)) return set_err(c, LBM_ERR_INVALID_ARG, "relaxation rates must lie in (0, 2)");
    c->rates = r;
    c->gen += 1;   // kernel arguments are baked into recorded graphs
    return LBM_OK;
}

int lbm_set_shift_velocity(lbm_ctx* c, double urx, double ury) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (!std::isfinite(urx) || !std::isfinite(ury) || std::fabs(urx) >= 1.0 || std::fabs(ury) >= 1.0)
        return set_err(c, LBM_ERR_INVALID_ARG, "shift velocity must be finite with |u| < 1");
    if (c->eq_order != 4 && (urx != 0.0 || ury != 0.0))
        return set_err(c, LBM_ERR_UNSUPPORTED, "a shift velocity needs the extended equilibrium");
    if (urx == c->urx && ury == c->ury) return LBM_OK;
    // re-encode the current state: gather f with the old shift, scatter with the new one
    const size_t n = (size_t)c->nx * c->ny;
    int rc = ensure_stage(c, 9 * n);
    if (rc) return rc;
    LBM_CK(c, lbm::launch_gather(c->storage, c->buf[c->cur], field_args(c), c->stage, nullptr, nullptr, nullptr,
                                 nullptr, nullptr, nullptr, c->stream));
    c->urx = urx;
    c->ury = ury;
    LBM_CK(c, lbm::launch_scatter(c->storage, c->buf[c->cur], field_args(c), c->stage, c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    c->gen += 1;
    return select_kernel(c);
}

int lbm_init_equilibrium(lbm_ctx* c, const double* rho, const double* ux, const double* uy) {
    if (!c || !rho || !ux || !uy) return c ? set_err(c, LBM_ERR_INVALID_ARG, "null field") : LBM_ERR_INVALID_ARG;
    const size_t n = (size_t)c->nx * c->ny;
    const double* in[3] = {rho, ux, uy};
    const double* dev[3];
    bool host = false;
    for (int k = 0; k < 3; ++k) host |= !is_device_ptr(in[k]);
    if (host) {
        int rc = ensure_stage(c, 3 * n);
        if (rc) return rc;
    }
    for (int k = 0; k < 3; ++k) {
        if (is_device_ptr(in[k])) {
            dev[k] = in[k];
        } else {
            LBM_CK(c, cudaMemcpyAsync(c->stage + k * n, in[k], n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            dev[k] = c->stage + k * n;
        }
    }
    LBM_CK(c, lbm::launch_init_eq(c->storage, c->buf[c->cur], field_args(c), c->eq_order, dev[0], dev[1], dev[2], c->stream));
    c->steps = 0;
    const long long reset[2] = {0, -1};
    LBM_CK(c, cudaMemcpyAsync(c->status, reset, sizeof(reset), cudaMemcpyHostToDevice, c->stream));
    // `reset` lives on this stack frame and the staging buffer may be reused by the next call
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_set_populations(lbm_ctx* c, const double* f) {
    if (!c || !f) return c ? set_err(c, LBM_ERR_INVALID_ARG, "null populations") : LBM_ERR_INVALID_ARG;
    const size_t n = (size_t)c->nx * c->ny;
    const double* d = f;
    if (!is_device_ptr(f)) {
        int rc = ensure_stage(c, 9 * n);
        if (rc) return rc;
        LBM_CK(c, cudaMemcpyAsync(c->stage, f, 9 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        d = c->stage;
    }
    LBM_CK(c, lbm::launch_scatter(c->storage, c->buf[c->cur], field_args(c), d, c->stream));
    if (d != f) LBM_CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_get_populations(lbm_ctx* c, double* f) {
    if (!c || !f) return c ? set_err(c, LBM_ERR_INVALID_ARG, "null populations") : LBM_ERR_INVALID_ARG;
    const size_t n = (size_t)c->nx * c->ny;
    if (is_device_ptr(f)) {
        LBM_CK(c, lbm::launch_gather(c->storage, c->buf[c->cur], field_args(c), f, nullptr, nullptr, nullptr,
                                     nullptr, nullptr, nullptr, c->stream));
        return LBM_OK;
    }
    int rc = ensure_stage(c, 9 * n);
    if (rc) return rc;
    LBM_CK(c, lbm::launch_gather(c->storage, c->buf[c->cur], field_args(c), c->stage, nullptr, nullptr, nullptr,
                                 nullptr, nullptr, nullptr, c->stream));
    LBM_CK(c, cudaMemcpyAsync(f, c->stage, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_moments(lbm_ctx* c, double* rho, double* ux, double* uy, double* pxx, double* pxy, double* pyy) {
    if (!c) return LBM_ERR_INVALID_ARG;
    const size_t n = (size_t)c->nx * c->ny;
    double* outs[6] = {rho, ux, uy, pxx, pxy, pyy};
    double* dev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int nhost = 0;
    for (int k = 0; k < 6; ++k)
        if (outs[k] && !is_device_ptr(outs[k])) ++nhost;
    if (nhost) {
        int rc = ensure_stage(c, 6 * n);
        if (rc) return rc;
    }
    for (int k = 0; k < 6; ++k) {
        if (!outs[k]) continue;
        dev[k] = is_device_ptr(outs[k]) ? outs[k] : c->stage + k * n;
    }
    LBM_CK(c, lbm::launch_gather(c->storage, c->buf[c->cur], field_args(c), nullptr, dev[0], dev[1], dev[2], dev[3],
                                 dev[4], dev[5], c->stream));
    if (nhost) {
        for (int k = 0; k < 6; ++k)
            if (outs[k] && dev[k] != outs[k])
                LBM_CK(c, cudaMemcpyAsync(outs[k], dev[k], n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        LBM_CK(c, cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

int lbm_halo_pack(lbm_ctx* c, void* send_up, void* send_down) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (!send_up || !send_down || !is_device_ptr(send_up) || !is_device_ptr(send_down))
        return set_err(c, LBM_ERR_INVALID_ARG, "halo messages must be device pointers");
    LBM_CK(c, lbm::launch_halo(c->storage, c->buf[c->cur], field_args(c), send_up, send_down, true, c->stream));
    return LBM_OK;
}

int lbm_halo_unpack(lbm_ctx* c, const void* from_below, const void* from_above) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (!from_below || !from_above || !is_device_ptr(from_below) || !is_device_ptr(from_above))
        return set_err(c, LBM_ERR_INVALID_ARG, "halo messages must be device pointers");
    LBM_CK(c, lbm::launch_halo(c->storage, c->buf[c->cur], field_args(c), const_cast<void*>(from_below),
                               const_cast<void*>(from_above), false, c->stream));
    return LBM_OK;
}

int lbm_reduce(lbm_ctx* c, double* out8) {
    if (!c || !out8) return c ? set_err(c, LBM_ERR_INVALID_ARG, "null output") : LBM_ERR_INVALID_ARG;
    const bool dev = is_device_ptr(out8);
    int rc = launch_check(c, dev ? out8 : c->red_out, 0);
    if (rc) return rc;
    if (!dev) {
        LBM_CK(c, cudaMemcpyAsync(out8, c->red_out, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        LBM_CK(c, cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

int lbm_set_check(lbm_ctx* c, long long every, double ke_ref, double ke_factor, double uref_x, double uref_y) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (every < 0 || !std::isfinite(ke_ref) || !std::isfinite(ke_factor) || !std::isfinite(uref_x) ||
        !std::isfinite(uref_y))
        return set_err(c, LBM_ERR_INVALID_ARG, "invalid check parameters");
    c->check_every = every; c->ke_ref = ke_ref; c->ke_factor = ke_factor; c->uref_x = uref_x; c->uref_y = uref_y;
    return LBM_OK;
}

int lbm_status(lbm_ctx* c, int* status, long long* blowup_step, long long* steps) {
    if (!c) return LBM_ERR_INVALID_ARG;
    long long h[2] = {0, -1};
    LBM_CK(c, cudaMemcpyAsync(h, c->status, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    const int timeout = (int)((unsigned long long)h[0] >> 32);   // set by a bulk-copy kernel's bounded wait
    if (status) *status = timeout ? LBM_ERR_TIMEOUT : (int)(h[0] & 0xffffffff);
    if (blowup_step) *blowup_step = h[1];
    if (steps) *steps = c->steps;
    return LBM_OK;
}

int lbm_synchronize(lbm_ctx* c) {
    if (!c) return LBM_ERR_INVALID_ARG;
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_get_layout(const lbm_ctx* c, int* pitch, int* grid, int* block) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (pitch) *pitch = c->pitch;
    if (grid) *grid = c->grid;
    if (block) *block = c->block;
    return LBM_OK;
}

int lbm_set_kernel_path(lbm_ctx* c, int path, int stages) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (path < LBM_PATH_AUTO || path > LBM_PATH_BULK || stages < 0 || stages == 1 || stages > 4)
        return set_err(c, LBM_ERR_INVALID_ARG, "unknown kernel path or stage count");
    if (path == LBM_PATH_BULK && !row_aligned(c))
        return set_err(c, LBM_ERR_UNSUPPORTED, "the bulk-copy kernel needs rows of a multiple of 16 bytes");
    c->path = path;
    c->stages = stages;
    if (c->own_group) {   // rebuilt with the new path at the next lbm_step
        lbm_group_destroy(c->own_group);
        c->own_group = nullptr;
    }
    c->gen += 1;
    return LBM_OK;
}

int lbm_set_launch_shape(lbm_ctx* c, int steps_per_launch, int order) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (steps_per_launch < 0 || order < LBM_ORDER_AUTO || order > LBM_ORDER_BLOCK)
        return set_err(c, LBM_ERR_INVALID_ARG, "invalid steps per launch or work order");
    c->launch_steps = steps_per_launch;
    c->launch_order = order;
    if (c->own_group) {   // rebuilt at the next lbm_step
        lbm_group_destroy(c->own_group);
        c->own_group = nullptr;
    }
    c->gen += 1;
    return LBM_OK;
}

int lbm_set_tile_form(lbm_ctx* c, int form) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (form < LBM_FORM_AUTO || form > LBM_FORM_WIDE) return set_err(c, LBM_ERR_INVALID_ARG, "unknown kernel form");
    if (form == LBM_FORM_LIGHT && (c->storage == LBM_F64 || !light_model(c->model)))
        return set_err(c, LBM_ERR_UNSUPPORTED, "the light form serves BGK, RM, HM and PR in FP32 / 16-bit storage");
    if (form == LBM_FORM_WIDE && c->storage == LBM_F64)
        return set_err(c, LBM_ERR_UNSUPPORTED, "FP64 storage has the general form only");
    c->tile_form = form;
    if (c->own_group) {   // rebuilt at the next lbm_step
        lbm_group_destroy(c->own_group);
        c->own_group = nullptr;
    }
    c->gen += 1;
    return LBM_OK;
}

int lbm_group_create(lbm_group** out, lbm_ctx* const* ctxs, int n, int graph_steps) {
    if (!out || !ctxs || n < 1 || graph_steps < 0 || (graph_steps % 2) != 0) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    for (int k = 0; k < n; ++k) {
        if (!ctxs[k]) return LBM_ERR_INVALID_ARG;
        if (ctxs[k]->stream != ctxs[0]->stream)
            return set_err(ctxs[0], LBM_ERR_INVALID_ARG, "group contexts must share one stream");
        for (int j = 0; j < k; ++j)
            if (ctxs[j] == ctxs[k]) return set_err(ctxs[0], LBM_ERR_INVALID_ARG, "context listed twice");
    }
    lbm_group* g = new (std::nothrow) lbm_group();
    if (!g) return LBM_ERR_NOMEM;
    g->ctx.assign(ctxs, ctxs + n);
    g->stream = ctxs[0]->stream;
    g->graph_steps = graph_steps;
    // lattices of one storage type whose rows are whole 16-byte chunks: one bulk-copy
    // staged launch per time step (unless a context asks for the register-staged kernels)
    bool tile = n <= lbm::kGroupMax;
    for (int k = 0; tile && k < n; ++k)
        tile = ctxs[k]->storage == ctxs[0]->storage && ctxs[k]->path != LBM_PATH_VECTOR && row_aligned(ctxs[k]);
    if (tile) {
        const int storage = ctxs[0]->storage;
        for (int k = 0; k < n; ++k) g->state_bytes += 2LL * 9 * ctxs[k]->plane * lbm::storage_bytes(storage);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // kernels (unshifted, shifted), shared memory, grids and tile geometry of one kernel
        // form; false if a kernel is missing or cannot be resident
        auto plan = [&](int form) {
            const int stages = ctxs[0]->stages > 0 ? ctxs[0]->stages : default_stages(storage, form);
            lbm::TileKernelInfo info[2];
            int grid[2];
            for (int sh = 0; sh < 2; ++sh) {
                int per_sm = 0;
                if (!pick_tile_kernel(storage, sh == 1, stages, form, &info[sh]) ||
                    cudaFuncSetAttribute(info[sh].kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, info[sh].smem) != cudaSuccess ||
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, info[sh].kernel, info[sh].threads, info[sh].smem) != cudaSuccess ||
                    per_sm < 1) {
                    cudaGetLastError();
                    return false;
                }
                grid[sh] = sms * per_sm;   // all resident CTAs (a multi-step launch needs them co-resident)
            }
            g->tform = form;
            g->tthreads = info[0].threads;
            g->twidth = info[0].width;
            g->tsmem = info[0].smem;
            for (int sh = 0; sh < 2; ++sh) {
                g->tkernel[sh] = info[sh].kernel;
                g->tgrid[sh] = grid[sh];
            }
            // tiles (rows or row blocks of the form's width) and completion counters per lattice
            const int W = g->twidth;
            unsigned off = 0, units = 0;
            g->tbegin.clear();
            g->cbase.clear();
            g->same_geometry = 1;
            for (int k = 0; k < n; ++k) {
                g->tbegin.push_back(off);
                off += tile_count(ctxs[k], W);
                g->cbase.push_back(units);
                const int R = tile_rows(ctxs[k], W);
                const int U = R > 1 ? (ctxs[k]->ny + R - 1) / R : ctxs[k]->ny;
                const int ntx = R > 1 ? 1 : (ctxs[k]->nx + W - 1) / W;
                units += (unsigned)U;
                if (k == 0) {
                    g->wU = U;
                    g->wntx = ntx;
                } else if (U != g->wU || ntx != g->wntx || R != tile_rows(ctxs[0], W)) {
                    g->same_geometry = 0;
                }
            }
            g->ttotal = off;
            g->cunits = units;
            return true;
        };
        // The form (the first context's choice, lbm_set_tile_form, where the group's lattices
        // allow it).  By default the one-step form of the group's models (light for BGK, RM, HM,
        // PR in FP32 / FP16, else wide; BF16 light models measured 0.99-1.00 of the copy
        // bandwidth at 16384^2 in the wide form, 0.965-0.98 in the light one) when one step per
        // launch is asked for, or when a step has at least LBM_ONE_STEP_TILES_PER_CTA of that
        // form's tiles per resident CTA and no multi-step work order is asked for -- except
        // that the wide form leaves a single lattice to the general form's wavefront launches
        // where those apply (measured, FP32: 4096^2 0.96 of the copy bandwidth in the wavefront
        // against 0.91 in the wide form; 8192^2 wide 0.96 against 0.94 for the general form's
        // one-step launches); otherwise the general form.
        const bool light = storage != LBM_F64 && light_models(ctxs, n);
        const int one_form = storage == LBM_F64 ? -1 : ((light && storage != LBM_BF16) ? 1 : 2);
        const lbm_ctx* c0 = ctxs[0];
        int form = -1;
        if (c0->tile_form == LBM_FORM_GENERAL || storage == LBM_F64) {
            form = 0;
        } else if (c0->tile_form == LBM_FORM_LIGHT && light) {
            form = 1;
        } else if (c0->tile_form == LBM_FORM_WIDE) {
            form = 2;
        } else if (c0->launch_steps <= 1 && c0->launch_order != LBM_ORDER_WAVE && c0->launch_order != LBM_ORDER_BLOCK) {
            const bool general_wave = c0->launch_steps == 0 && plan(0) && use_wave(g);
            if ((one_form == 1 || !general_wave) && plan(one_form)) {
                const int grid = std::max(g->tgrid[0], g->tgrid[1]);
                if (c0->launch_steps == 1 || g->ttotal >= (unsigned)LBM_ONE_STEP_TILES_PER_CTA * (unsigned)grid)
                    form = one_form;
            }
        }
        if (form < 0) form = 0;
        tile = plan(form);
        if (!tile && form != 0) tile = plan(form = 0);   // a form that cannot be resident
        g->tone = tile && form != 0 ? 1 : 0;
        // the library's choice: a step with fewer tiles than resident CTAs leaves the copy
        // pipeline mostly idle (latency-bound); the register-staged kernels do better there
        bool forced = false;
        for (int k = 0; k < n; ++k) forced = forced || ctxs[k]->path == LBM_PATH_BULK;
        if (tile && !forced && g->ttotal < (unsigned)std::max(g->tgrid[0], g->tgrid[1])) tile = false;
        if (tile && cudaMalloc(&g->cnt, sizeof(unsigned) * g->cunits) != cudaSuccess) {
            cudaGetLastError();
            g->cnt = nullptr;
            tile = false;
        }
        if (!tile) {
            g->tbegin.clear();
            g->cbase.clear();
            g->ttotal = 0;
            g->tone = 0;
        }
        g->tiled = tile ? 1 : 0;
    }
    // several lattices of one storage type: one fused launch per time step
    bool same = !g->tiled && n > 1 && n <= lbm::kGroupMax;
    for (int k = 1; same && k < n; ++k) same = ctxs[k]->storage == ctxs[0]->storage;
    if (same) {
        unsigned off = 0;
        for (int k = 0; k < n; ++k) {
            g->begin.push_back(off);
            const unsigned segs = (unsigned)ctxs[k]->ny * (unsigned)ctxs[k]->nseg;
            off += (segs + 31u) / 32u * 32u;
        }
        g->padded_total = off;
        for (int sh = 0; sh < 2; ++sh) {
            g->gkernel[sh] = pick_group_kernel(ctxs[0]->storage, sh == 1);
            g->ggrid[sh] = resident_grid(g->gkernel[sh], 256, off);
        }
        g->fused = 1;
    }
    if (graph_steps > 0) {
        cudaError_t e = cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete g;
            return set_err(ctxs[0], LBM_ERR_CUDA, "group stream: %s", cudaGetErrorString(e));
        }
    }
    *out = g;
    return LBM_OK;
}

void lbm_group_destroy(lbm_group* g) {
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
    if (g->capture) cudaStreamDestroy(g->capture);
    for (cudaStream_t st : g->side) cudaStreamDestroy(st);
    for (cudaEvent_t e : g->side_done) cudaEventDestroy(e);
    if (g->fork) cudaEventDestroy(g->fork);
    if (g->cnt) cudaFree(g->cnt);
    delete g;
}

int lbm_group_step(lbm_group* g, long long nsteps) {
    if (!g || nsteps < 0) return LBM_ERR_INVALID_ARG;
    long long done = 0;
    while (done < nsteps) {
        // steps until the next due check of any context
        long long chunk = nsteps - done;
        for (lbm_ctx* c : g->ctx)
            if (c->check_every > 0) {
                const long long to_check = c->check_every - (c->steps % c->check_every);
                if (to_check < chunk) chunk = to_check;
            }
        long long left = chunk;
        while (g->graph_steps > 0 && left >= g->graph_steps) {
            int rc = group_replay(g);
            if (rc) return rc;
            left -= g->graph_steps;
        }
        int rc = group_advance(g, g->stream, left);
        if (rc) return rc;
        done += chunk;
        std::vector<lbm_ctx*> due;
        for (lbm_ctx* c : g->ctx)
            if (c->check_every > 0 && c->steps % c->check_every == 0) due.push_back(c);
        rc = launch_checks(g, due);
        if (rc) return rc;
    }
    return LBM_OK;
}

int lbm_group_set_timing(lbm_group* g, int enable) {
    if (!g) return LBM_ERR_INVALID_ARG;
    g->timing = enable ? 1 : 0;
    g->ev_used = 0;
    g->replay_ms = 0.0;
    g->replay_lattice_steps = 0;
    g->pending_lattice_steps = 0;
    g->replay_kernels = 0;
    g->pending_kernels = 0;
    return LBM_OK;
}

int lbm_group_describe(const lbm_group* g, int* family, int* form, int* steps_per_launch, int* tiles, int* grid,
                       int* block) {
    if (!g) return LBM_ERR_INVALID_ARG;
    const bool bulk = g->tiled && tile_shift(g) >= 0;
    if (family) *family = bulk ? LBM_PATH_BULK : LBM_PATH_VECTOR;
    if (form) *form = bulk ? (g->tform == 0 ? LBM_FORM_GENERAL : (g->tform == 1 ? LBM_FORM_LIGHT : LBM_FORM_WIDE))
                           : LBM_FORM_AUTO;
    if (steps_per_launch) *steps_per_launch = bulk ? tile_steps_per_launch(g) : 0;
    if (tiles) *tiles = bulk ? (int)g->ttotal : 0;
    if (grid) *grid = bulk ? std::max(g->tgrid[0], g->tgrid[1]) : 0;
    if (block) *block = bulk ? g->tthreads : 0;
    return LBM_OK;
}

int lbm_group_timing(lbm_group* g, double* replay_ms, long long* lattice_steps, long long* kernel_launches) {
    if (!g) return LBM_ERR_INVALID_ARG;
    lbm_ctx* c0 = g->ctx[0];
    LBM_CK(c0, cudaStreamSynchronize(g->stream));
    for (size_t k = 0; k + 1 < g->ev_used; k += 2) {
        float ms = 0.f;
        LBM_CK(c0, cudaEventElapsedTime(&ms, g->ev[k], g->ev[k + 1]));
        g->replay_ms += ms;
    }
    g->ev_used = 0;
    g->replay_lattice_steps += g->pending_lattice_steps;
    g->pending_lattice_steps = 0;
    g->replay_kernels += g->pending_kernels;
    g->pending_kernels = 0;
    if (replay_ms) *replay_ms = g->replay_ms;
    if (lattice_steps) *lattice_steps = g->replay_lattice_steps;
    if (kernel_launches) *kernel_launches = g->replay_kernels;
    return LBM_OK;
}

int lbm_adjoint_run(lbm_ctx* c, long long nsteps, int loss, const double* ux_target, const double* uy_target,
                    int checkpoint_every, double* grad_ux0, double* grad_uy0, double* grad_rates3, double* loss_out,
                    double* times_ms2) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (nsteps < 1 || (loss != 0 && loss != 1) || checkpoint_every < 0 || !grad_ux0 || !grad_uy0 || !grad_rates3 ||
        !loss_out || (loss == 0 && (!ux_target || !uy_target)))
        return set_err(c, LBM_ERR_INVALID_ARG, "invalid adjoint arguments");
    if ((c->storage != LBM_F64 && c->storage != LBM_F32) || c->eq_order != 4)
        return set_err(c, LBM_ERR_UNSUPPORTED, "the adjoint supports FP64/FP32 storage and the extended equilibrium");
    const StepArgs sa = step_args(c);
    lbm::AdjointPlan plan;
    int rc = lbm::adjoint_plan(c->storage, kernel_model(c->model), cumulant_read(c->model), c->nx, c->ny, c->pitch, c->plane, sa.w_nu, sa.w3, sa.w4, c->rho0,
                               c->urx, c->ury, &plan);
    if (rc) return set_err(c, rc, "no adjoint kernel for this configuration");
    const long long N = nsteps;
    long long K = checkpoint_every > 0 ? checkpoint_every : (long long)std::ceil(std::sqrt((double)N));
    if (checkpoint_every <= 0 && K % 2) ++K;   // even segments keep the lambda parity fixed
    if (K > N) K = N;
    const long long nseg = (N + K - 1) / K;
    const size_t n = (size_t)c->nx * c->ny;
    const size_t bufb = (size_t)9 * c->plane * lbm::storage_bytes(c->storage);
    const size_t lamb = (size_t)9 * c->plane * (c->storage == LBM_F64 ? sizeof(double) : sizeof(float));
    char* ckpt = nullptr;
    char* ring = nullptr;
    char* lam = nullptr;
    double* rate_part = nullptr;
    double* loss_part = nullptr;
    double* dev_io = nullptr;   // targets (2n) and gradients (2n) staged on the device
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    std::vector<double> rp((size_t)plan.grid_adj * 3), lp((size_t)lbm::adjoint_seed_blocks());
    const bool tdev = loss == 1 || (is_device_ptr(ux_target) && is_device_ptr(uy_target));
    const bool gdev = is_device_ptr(grad_ux0) && is_device_ptr(grad_uy0);
    cudaError_t e = cudaSuccess;
    const double* uxt = ux_target;
    const double* uyt = uy_target;
    double* gux = grad_ux0;
    double* guy = grad_uy0;
    int cur_l = 0;
    float fwd_ms = 0.f, bwd_ms = 0.f;
#define LBM_ADJ(call) do { if (e == cudaSuccess) e = (call); } while (0)
    LBM_ADJ(cudaMalloc(&ckpt, (size_t)nseg * bufb));
    LBM_ADJ(cudaMalloc(&lam, 2 * lamb));
    LBM_ADJ(cudaMalloc(&rate_part, rp.size() * sizeof(double)));
    LBM_ADJ(cudaMalloc(&loss_part, lp.size() * sizeof(double)));
    LBM_ADJ(cudaMalloc(&dev_io, 4 * n * sizeof(double)));
    for (int k = 0; k < 3; ++k) LBM_ADJ(cudaEventCreate(&ev[k]));
    if (e == cudaSuccess && !tdev) {
        LBM_ADJ(cudaMemcpyAsync(dev_io, ux_target, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        LBM_ADJ(cudaMemcpyAsync(dev_io + n, uy_target, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        uxt = dev_io;
        uyt = dev_io + n;
    }
    if (!gdev) {
        gux = dev_io + 2 * n;
        guy = dev_io + 3 * n;
    }
    // forward: checkpoint every K steps
    LBM_ADJ(cudaEventRecord(ev[0], c->stream));
    for (long long s2 = 0; s2 < nseg && e == cudaSuccess; ++s2) {
        LBM_ADJ(cudaMemcpyAsync(ckpt + s2 * bufb, c->buf[c->cur], bufb, cudaMemcpyDeviceToDevice, c->stream));
        if (e == cudaSuccess) {
            const int r = lbm_step(c, std::min(K, N - s2 * K));
            if (r != LBM_OK) rc = r;
        }
        if (rc != LBM_OK) break;
    }
    LBM_ADJ(cudaEventRecord(ev[1], c->stream));
    // the recomputation takes the forward run's kernel family (the context's own group); with
    // the register-staged kernels each adjoint launch also recomputes a step of the next
    // segment into a second ring (fused launches)
    lbm_group* fg = (c->own_group && c->own_group->tiled) ? c->own_group : nullptr;
    const bool fused = !fg && plan.grid_fused > 0 && nseg > 1 && K > 1;
    LBM_ADJ(cudaMalloc(&ring, (size_t)(fused ? 2 : 1) * K * bufb));
    // seed lambda^N and the loss from f^N
    LBM_ADJ(lbm::adjoint_launch_seed(plan, c->buf[c->cur], loss, uxt, uyt, lam, loss_part, c->stream));
    LBM_ADJ(cudaMemsetAsync(rate_part, 0, rp.size() * sizeof(double), c->stream));
    // backward, segment by segment from the last one: restore the checkpoint, recompute the
    // segment's states into the ring, run its adjoint steps backwards.  A full segment is one
    // CUDA-graph replay (one graph per starting parity of the lambda ping-pong).
    cudaGraphExec_t seg_exec[2] = {nullptr, nullptr};
    cudaGraphExec_t pair_exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    cudaStream_t cap = nullptr;
    LBM_ADJ(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    auto enqueue_segment = [&](long long len, int parity, cudaStream_t st) {
        cudaError_t r = cudaSuccess;
        if (fg && len > 1) {   // the whole recomputation in one multi-step launch along the ring
            const void* a = ring;
            void* b = ring;
            r = launch_tile(fg, &a, &b, (int)(len - 1), st, is_shifted(c) ? 1 : 0,
                            (long long)(bufb / lbm::storage_bytes(c->storage)));
        }
        for (long long k = 0; !fg && k + 1 < len && r == cudaSuccess; ++k)
            r = lbm::adjoint_launch_fwd(plan, sa, ring + k * bufb, ring + (k + 1) * bufb, st);
        int pl = parity;
        for (long long k = len - 1; k >= 0 && r == cudaSuccess; --k) {
            r = lbm::adjoint_launch_step(plan, ring + k * bufb, lam + pl * lamb, lam + (pl ^ 1) * lamb, rate_part, st);
            pl ^= 1;
        }
        return r;
    };
    // fused: the adjoint steps of the segment in ring `slot` (len states) together with the
    // recomputation of the next segment (lenn states) into ring `slot ^ 1`
    char* rings[2] = {ring, fused ? ring + (size_t)K * bufb : ring};
    auto enqueue_pair = [&](long long len, long long lenn, int slot, int parity, cudaStream_t st) {
        cudaError_t r = cudaSuccess;
        int pl = parity;
        const long long nl = std::max(len, lenn - 1);
        for (long long j = 0; j < nl && r == cudaSuccess; ++j) {
            const bool adj = j < len, fw = j + 1 < lenn;
            const long long k = len - 1 - j;
            char* nx = rings[slot ^ 1];
            if (adj && fw)
                r = lbm::adjoint_launch_fused(plan, rings[slot] + k * bufb, lam + pl * lamb, lam + (pl ^ 1) * lamb,
                                              rate_part, sa, nx + j * bufb, nx + (j + 1) * bufb, st);
            else if (adj)
                r = lbm::adjoint_launch_step(plan, rings[slot] + k * bufb, lam + pl * lamb, lam + (pl ^ 1) * lamb,
                                             rate_part, st);
            else
                r = lbm::adjoint_launch_fwd(plan, sa, nx + j * bufb, nx + (j + 1) * bufb, st);
            if (adj) pl ^= 1;
        }
        return r;
    };
    if (fused) {
        // the first segment processed (the last in time) is recomputed on its own
        const long long s0 = nseg - 1, len0 = std::min(K, N - s0 * K);
        LBM_ADJ(cudaMemcpyAsync(rings[0], ckpt + s0 * bufb, bufb, cudaMemcpyDeviceToDevice, c->stream));
        for (long long k = 0; k + 1 < len0 && e == cudaSuccess; ++k)
            LBM_ADJ(lbm::adjoint_launch_fwd(plan, sa, rings[0] + k * bufb, rings[0] + (k + 1) * bufb, c->stream));
    }
    for (long long q = 0; fused && q < nseg && e == cudaSuccess && rc == LBM_OK; ++q) {
        const long long s2 = nseg - 1 - q;
        const long long len = std::min(K, N - s2 * K);
        const long long lenn = (q + 1 < nseg) ? K : 0;   // every segment before the last is full
        const int slot = (int)(q & 1);
        if (lenn > 0)
            LBM_ADJ(cudaMemcpyAsync(rings[slot ^ 1], ckpt + (s2 - 1) * bufb, bufb, cudaMemcpyDeviceToDevice,
                                    c->stream));
        if (len == K && lenn == K) {
            cudaGraphExec_t& ex = pair_exec[slot][cur_l];
            if (!ex && e == cudaSuccess) {
                cudaGraph_t graph = nullptr;
                LBM_ADJ(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
                const cudaError_t r = enqueue_pair(len, lenn, slot, cur_l, cap);
                const cudaError_t r2 = cudaStreamEndCapture(cap, &graph);
                LBM_ADJ(r);
                LBM_ADJ(r2);
                if (graph) {
                    LBM_ADJ(cudaGraphInstantiate(&ex, graph, 0));
                    cudaGraphDestroy(graph);
                }
            }
            LBM_ADJ(cudaGraphLaunch(ex, c->stream));
        } else {
            LBM_ADJ(enqueue_pair(len, lenn, slot, cur_l, c->stream));
        }
        if (len % 2) cur_l ^= 1;
    }
    for (long long s2 = nseg - 1; !fused && s2 >= 0 && e == cudaSuccess && rc == LBM_OK; --s2) {
        const long long len = std::min(K, N - s2 * K);
        LBM_ADJ(cudaMemcpyAsync(ring, ckpt + s2 * bufb, bufb, cudaMemcpyDeviceToDevice, c->stream));
        if (len == K && K > 1) {
            if (!seg_exec[cur_l] && e == cudaSuccess) {
                cudaGraph_t graph = nullptr;
                LBM_ADJ(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
                const cudaError_t r = enqueue_segment(len, cur_l, cap);
                const cudaError_t r2 = cudaStreamEndCapture(cap, &graph);
                LBM_ADJ(r);
                LBM_ADJ(r2);
                if (graph) {
                    LBM_ADJ(cudaGraphInstantiate(&seg_exec[cur_l], graph, 0));
                    cudaGraphDestroy(graph);
                }
            }
            LBM_ADJ(cudaGraphLaunch(seg_exec[cur_l], c->stream));
        } else {
            LBM_ADJ(enqueue_segment(len, cur_l, c->stream));
        }
        if (len % 2) cur_l ^= 1;
    }
    for (int k = 0; k < 2; ++k) {
        if (seg_exec[k]) cudaGraphExecDestroy(seg_exec[k]);
        for (int j = 0; j < 2; ++j)
            if (pair_exec[k][j]) cudaGraphExecDestroy(pair_exec[k][j]);
    }
    if (cap) cudaStreamDestroy(cap);
    // dL/du0 from lambda^0 and the initial state (checkpoint 0)
    LBM_ADJ(lbm::adjoint_launch_init(plan, ckpt, lam + cur_l * lamb, gux, guy, c->stream));
    LBM_ADJ(cudaEventRecord(ev[2], c->stream));
    if (!gdev) {
        LBM_ADJ(cudaMemcpyAsync(grad_ux0, gux, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        LBM_ADJ(cudaMemcpyAsync(grad_uy0, guy, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    LBM_ADJ(cudaMemcpyAsync(rp.data(), rate_part, rp.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LBM_ADJ(cudaMemcpyAsync(lp.data(), loss_part, lp.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LBM_ADJ(cudaStreamSynchronize(c->stream));
    if (e == cudaSuccess) {
        cudaEventElapsedTime(&fwd_ms, ev[0], ev[1]);
        cudaEventElapsedTime(&bwd_ms, ev[1], ev[2]);
    }
#undef LBM_ADJ
    cudaFree(ckpt);
    cudaFree(ring);
    cudaFree(lam);
    cudaFree(rate_part);
    cudaFree(loss_part);
    cudaFree(dev_io);
    for (int k = 0; k < 3; ++k)
        if (ev[k]) cudaEventDestroy(ev[k]);
    if (rc != LBM_OK) return rc;
    if (e != cudaSuccess)
        return set_err(c, e == cudaErrorMemoryAllocation ? LBM_ERR_NOMEM : LBM_ERR_CUDA, "adjoint: %s",
                       cudaGetErrorString(e));
    // fixed-order FP64 folds of the per-block partials
    double gr[3] = {0.0, 0.0, 0.0}, L = 0.0;
    for (size_t b = 0; b < rp.size() / 3; ++b)
        for (int k = 0; k < 3; ++k) gr[k] += rp[b * 3 + k];
    for (double v : lp) L += v;
    if (c->model == LBM_PR) gr[1] = gr[2] = 0.0;
    if (is_device_ptr(grad_rates3)) {
        LBM_CK(c, cudaMemcpy(grad_rates3, gr, sizeof(gr), cudaMemcpyHostToDevice));
    } else {
        for (int k = 0; k < 3; ++k) grad_rates3[k] = gr[k];
    }
    if (is_device_ptr(loss_out)) {
        LBM_CK(c, cudaMemcpy(loss_out, &L, sizeof(L), cudaMemcpyHostToDevice));
    } else {
        *loss_out = L;
    }
    if (times_ms2) {
        times_ms2[0] = fwd_ms;
        times_ms2[1] = bwd_ms;
    }
    return LBM_OK;
}

int lbm_step(lbm_ctx* c, long long n) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (n < 0) return set_err(c, LBM_ERR_INVALID_ARG, "negative step count");
    if (!c->own_group) {
        lbm_ctx* one[1] = {c};
        int rc = lbm_group_create(&c->own_group, one, 1, 32);
        if (rc) return rc;
    }
    return lbm_group_step(c->own_group, n);
}

}  // extern "C"
