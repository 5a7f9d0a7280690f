// The C ABI of include/lbm.h: contexts, argument validation, host/device pointer staging,
// time stepping with CUDA-graph replay, blow-up checks and multi-lattice groups.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"

using lbm::CheckArgs;
using lbm::FieldArgs;
using lbm::StepArgs;

struct lbm_ctx {
    int nx = 0, ny = 0, pitch = 0, nseg = 0, vec = 0;
    int model = 0, storage = 0, eq_order = 4;
    double rho0 = 1.0;
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
    lbm_group* own_group = nullptr;    // used by lbm_step
    unsigned gen = 0;                  // bumped when kernel arguments change (graphs re-record)
    char err[512] = {0};
};

struct lbm_group {
    std::vector<lbm_ctx*> ctx;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;
    int graph_steps = 0;
    cudaGraphExec_t exec = nullptr;
    std::vector<int> exec_parity;      // ctx->cur of each context when the graph was recorded
    std::vector<unsigned> exec_gen;    // ctx->gen of each context when the graph was recorded
    int timing = 0;
    std::vector<cudaEvent_t> ev;       // pairs (start, stop) of timed replays
    size_t ev_used = 0;
    double replay_ms = 0.0;
    long long replay_launches = 0;
    long long pending_launches = 0;
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

bool rates_ok(const lbm_rates& r) { return rate_ok(r.omega_nu) && rate_ok(r.omega3) && rate_ok(r.omega4); }

const void* pick_kernel(int storage, int model, int eq_order) {
    switch (storage) {
        case LBM_F64: return lbm::step_kernel_f64(model, eq_order);
        case LBM_F32: return lbm::step_kernel_f32(model, eq_order);
        case LBM_F16: return lbm::step_kernel_f16(model, eq_order);
        case LBM_BF16: return lbm::step_kernel_bf16(model, eq_order);
        default: return nullptr;
    }
}

StepArgs step_args(const lbm_ctx* c) {
    StepArgs a;
    a.nx = c->nx; a.ny = c->ny; a.pitch = c->pitch; a.nseg = c->nseg; a.plane = c->plane;
    a.w_nu = c->rates.omega_nu;
    a.w3 = (c->model == LBM_PR) ? 1.0 : c->rates.omega3;
    a.w4 = (c->model == LBM_PR) ? 1.0 : c->rates.omega4;
    a.rho0 = c->rho0;
    return a;
}

FieldArgs field_args(const lbm_ctx* c) {
    FieldArgs a;
    a.nx = c->nx; a.ny = c->ny; a.pitch = c->pitch; a.plane = c->plane; a.rho0 = c->rho0;
    return a;
}

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

int launch_check(lbm_ctx* c, double* out8_dev, int apply) {
    CheckArgs ck;
    ck.ke_ref = c->ke_ref; ck.ke_factor = c->ke_factor; ck.uref_x = c->uref_x; ck.uref_y = c->uref_y;
    ck.step = c->steps; ck.apply = apply;
    LBM_CK(c, lbm::launch_reduce(c->storage, c->buf[c->cur], field_args(c), c->partials, out8_dev,
                                 c->status, c->blowup_step, ck, c->stream));
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
    for (int t = 0; t < g->graph_steps && rc == LBM_OK; ++t)
        for (lbm_ctx* c : g->ctx) {
            rc = launch_step_once(c, g->capture);
            if (rc != LBM_OK) break;
        }
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
        g->pending_launches += (long long)g->graph_steps * (long long)g->ctx.size();
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
    if (model < LBM_BGK || model > LBM_RR || storage < LBM_F64 || storage > LBM_BF16) return LBM_ERR_INVALID_ARG;
    if (!rates_ok(rates) || !(std::isfinite(rho0) && rho0 > 0.0)) return LBM_ERR_INVALID_ARG;
    if (eq_order != 2 && eq_order != 4) return LBM_ERR_INVALID_ARG;
    if (periodic != 1) return LBM_ERR_UNSUPPORTED;
    if (eq_order == 2 && model != LBM_BGK) return LBM_ERR_UNSUPPORTED;

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ERR_NOMEM;
    c->nx = nx; c->ny = ny; c->model = model; c->storage = storage; c->eq_order = eq_order;
    c->rho0 = rho0; c->rates = rates; c->stream = (cudaStream_t)cuda_stream;
    c->vec = lbm::storage_vec(storage);
    c->pitch = (nx + 31) / 32 * 32;
    c->nseg = (nx + c->vec - 1) / c->vec;
    c->plane = (long long)ny * c->pitch;
    c->kernel = pick_kernel(storage, model, eq_order);
    int rc = LBM_OK;
    const size_t bytes = (size_t)9 * (size_t)c->plane * (size_t)lbm::storage_bytes(storage);
    do {
        if (!c->kernel) { rc = set_err(c, LBM_ERR_UNSUPPORTED, "no kernel for this configuration"); break; }
        cudaError_t e;
        for (int b = 0; b < 2; ++b) {
            e = cudaMalloc(&c->buf[b], bytes);
            if (e != cudaSuccess) break;
            e = cudaMemsetAsync(c->buf[b], 0, bytes, c->stream);
            if (e != cudaSuccess) break;
        }
        if (e == cudaSuccess) e = cudaMalloc(&c->partials, sizeof(double) * 8 * lbm::reduce_blocks());
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
        // grid: resident CTAs of the whole GPU (grid-stride loop inside the kernel)
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c->kernel, c->block, 0);
        if (e != cudaSuccess || per_sm < 1) per_sm = 1;
        const long long work_warps = ((long long)ny * c->nseg + 31) / 32;
        long long g = (long long)sms * per_sm;
        const long long need = (work_warps * 32 + c->block - 1) / c->block;
        if (need < g) g = need;
        c->grid = (int)(g < 1 ? 1 : g);
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
    if (status) *status = (int)(h[0] & 0xffffffff);
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
        for (long long t = 0; t < left; ++t)
            for (lbm_ctx* c : g->ctx) {
                int rc = launch_step_once(c, g->stream);
                if (rc) return rc;
            }
        done += chunk;
        for (lbm_ctx* c : g->ctx)
            if (c->check_every > 0 && c->steps % c->check_every == 0) {
                int rc = launch_check(c, c->red_out, 1);
                if (rc) return rc;
            }
    }
    return LBM_OK;
}

int lbm_group_set_timing(lbm_group* g, int enable) {
    if (!g) return LBM_ERR_INVALID_ARG;
    g->timing = enable ? 1 : 0;
    g->ev_used = 0;
    g->replay_ms = 0.0;
    g->replay_launches = 0;
    g->pending_launches = 0;
    return LBM_OK;
}

int lbm_group_timing(lbm_group* g, double* replay_ms, long long* step_launches) {
    if (!g) return LBM_ERR_INVALID_ARG;
    lbm_ctx* c0 = g->ctx[0];
    LBM_CK(c0, cudaStreamSynchronize(g->stream));
    for (size_t k = 0; k + 1 < g->ev_used; k += 2) {
        float ms = 0.f;
        LBM_CK(c0, cudaEventElapsedTime(&ms, g->ev[k], g->ev[k + 1]));
        g->replay_ms += ms;
    }
    g->ev_used = 0;
    g->replay_launches += g->pending_launches;
    g->pending_launches = 0;
    if (replay_ms) *replay_ms = g->replay_ms;
    if (step_launches) *step_launches = g->replay_launches;
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
