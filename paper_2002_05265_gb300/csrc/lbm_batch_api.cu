// C ABI of the batched stability sweep (lbm_batch_* in include/lbm.h): instance layout in one
// slab, batched equilibrium initialisation, the graph-captured persistent launch, results,
// and the autotuner that picks the kernel's (vector width, CTA size).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <numeric>
#include <vector>

#include "lbm.h"
#include "lbm_batch.cuh"
#include "lbm_internal.h"

using lbm::BatchInstance;
using lbm::BatchState;

struct lbm_batch {
    int n = 0;
    int storage = LBM_F32;
    double rho0 = 1.0;
    cudaStream_t stream = nullptr;
    std::vector<BatchInstance> inst;
    std::vector<long long> node_off;   // dense node offset of each instance (concatenated fields)
    long long nodes = 0;
    BatchInstance* d_inst = nullptr;
    BatchState* d_state = nullptr;
    int* d_order = nullptr;
    int* d_queue = nullptr;
    long long* d_node_off = nullptr;
    void* slab = nullptr;
    size_t slab_bytes = 0;
    double* stage = nullptr;           // host-pointer staging for init (lazy)
    size_t stage_elems = 0;
    int vec = 0, block = 0, grid = 0;
    const void* kernel = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long g_target = -1;
    int g_check = -1;
    double g_growth = -1.0;
    const void* g_kernel = nullptr;
    char err[512] = {0};
};

namespace {

int berr(lbm_batch* b, int code, const char* fmt, ...) {
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof(b->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define LBM_BCK(b, call)                                                                         \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return berr((b), e_ == cudaErrorMemoryAllocation ? LBM_ERR_NOMEM : LBM_ERR_CUDA,     \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                         \
    } while (0)

const void* pick_batch_kernel(int storage, int vec, int block) {
    switch (storage) {
        case LBM_F64: return lbm::batch_kernel_f64(vec, block);
        case LBM_F32: return lbm::batch_kernel_f32(vec, block);
        case LBM_F16: return lbm::batch_kernel_f16(vec, block);
        case LBM_BF16: return lbm::batch_kernel_bf16(vec, block);
        default: return nullptr;
    }
}

void default_shape(int storage, int* vec, int* block) {
    *vec = 16 / lbm::storage_bytes(storage);
    *block = 256;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int set_shape(lbm_batch* b, int vec, int block) {
    const void* k = pick_batch_kernel(b->storage, vec, block);
    if (!k) return berr(b, LBM_ERR_UNSUPPORTED, "no batch kernel with vec=%d block=%d for this storage", vec, block);
    int dev = 0, sms = 0, per_sm = 0;
    LBM_BCK(b, cudaGetDevice(&dev));
    LBM_BCK(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LBM_BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, 0));
    if (per_sm < 1) return berr(b, LBM_ERR_UNSUPPORTED, "batch kernel cannot be resident");
    b->kernel = k;
    b->vec = vec;
    b->block = block;
    // resident CTAs only (a persistent grid); never more CTAs than instances
    b->grid = std::min(sms * per_sm, b->n);
    return LBM_OK;
}

// Equilibrium initialisation of every instance from concatenated dense fields.
template <typename S>
__global__ void batch_init_kernel(S* slab, const BatchInstance* __restrict__ inst, const BatchState* __restrict__ st,
                                  const long long* __restrict__ node_off, int n, long long nodes,
                                  const double* __restrict__ rho, const double* __restrict__ ux,
                                  const double* __restrict__ uy) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nodes;
         k += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = n - 1;   // last instance whose node_off <= k
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (node_off[mid] <= k) lo = mid; else hi = mid - 1;
        }
        const BatchInstance& I = inst[lo];
        const lbm::StepArgs& a = I.a;
        const long long local = k - node_off[lo];
        const int y = (int)(local / a.nx), x = (int)(local - (long long)y * a.nx);
        S* buf = slab + I.off + (long long)st[lo].cur * 9 * a.plane;
        const double r = rho[k], vx = ux[k], vy = uy[k], dr = r - a.rho0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sx = lbm::ex_of(i), sy = lbm::ey_of(i);
            // Eq. extendedFeq, product form, minus the shift rho0 phi(u_ref,x) phi(u_ref,y)
            const double Px = lbm::phi1d(sx, a.urx), Py = lbm::phi1d(sy, a.ury);
            const double dux = vx - a.urx, sux = vx + a.urx, duy = vy - a.ury, suy = vy + a.ury;
            const double Dx = sx ? 0.5 * dux * (sux + sx) : -dux * sux;
            const double Dy = sy ? 0.5 * duy * (suy + sy) : -duy * suy;
            const double g = Px * Py * dr + r * (Px * Dy + Dx * (Py + Dy));
            int xs = x - sx, ys = y - sy;
            xs = xs < 0 ? xs + a.nx : (xs >= a.nx ? xs - a.nx : xs);
            ys = ys < 0 ? ys + a.ny : (ys >= a.ny ? ys - a.ny : ys);
            buf[(long long)i * a.plane + (long long)ys * a.pitch + xs] = lbm::Conv<S>::from_double(g);
        }
    }
}

cudaError_t launch_batch_init(lbm_batch* b, const double* r, const double* x, const double* y) {
    const int block = 256;
    long long g = (b->nodes + block - 1) / block;
    if (g > 152 * 32) g = 152 * 32;
    switch (b->storage) {
        case LBM_F64: batch_init_kernel<double><<<(int)g, block, 0, b->stream>>>((double*)b->slab, b->d_inst, b->d_state, b->d_node_off, b->n, b->nodes, r, x, y); break;
        case LBM_F32: batch_init_kernel<float><<<(int)g, block, 0, b->stream>>>((float*)b->slab, b->d_inst, b->d_state, b->d_node_off, b->n, b->nodes, r, x, y); break;
        case LBM_F16: batch_init_kernel<__half><<<(int)g, block, 0, b->stream>>>((__half*)b->slab, b->d_inst, b->d_state, b->d_node_off, b->n, b->nodes, r, x, y); break;
        default: batch_init_kernel<__nv_bfloat16><<<(int)g, block, 0, b->stream>>>((__nv_bfloat16*)b->slab, b->d_inst, b->d_state, b->d_node_off, b->n, b->nodes, r, x, y); break;
    }
    return cudaGetLastError();
}

int reset_states(lbm_batch* b) {
    std::vector<BatchState> s(b->n);
    for (auto& x : s) {
        x.steps = 0; x.blowup_step = -1; x.pert0 = -1.0;
        x.pert = x.ke = x.rho_min = x.nonfinite = 0.0;
        x.status = 0; x.cur = 0;
    }
    LBM_BCK(b, cudaMemcpyAsync(b->d_state, s.data(), sizeof(BatchState) * b->n, cudaMemcpyHostToDevice, b->stream));
    LBM_BCK(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

// records {queue = 0; persistent kernel} into a graph for the current parameters
int record_run(lbm_batch* b, long long target, int check_every, double growth) {
    if (b->exec && b->g_target == target && b->g_check == check_every && b->g_growth == growth &&
        b->g_kernel == b->kernel)
        return LBM_OK;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaStream_t cap = nullptr;
    LBM_BCK(b, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(b->d_queue, 0, sizeof(int), cap);
        void* slab = b->slab;
        const BatchInstance* di = b->d_inst;
        BatchState* ds = b->d_state;
        const int* dord = b->d_order;
        int n = b->n;
        int* dq = b->d_queue;
        long long tg = target;
        int ce = check_every;
        double gr = growth;
        void* args[] = {&slab, &di, &ds, &dord, &n, &dq, &tg, &ce, &gr};
        cudaLaunchKernel(b->kernel, dim3(b->grid), dim3(b->block), args, 0, cap);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&b->exec, graph, 0);
            cudaGraphDestroy(graph);
        }
    }
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return berr(b, LBM_ERR_CUDA, "batch graph: %s", cudaGetErrorString(e));
    }
    b->g_target = target;
    b->g_check = check_every;
    b->g_growth = growth;
    b->g_kernel = b->kernel;
    return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : "null batch"; }

int lbm_batch_create(lbm_batch** out, int n, const lbm_instance_desc* desc, int storage, double rho0,
                     void* cuda_stream) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || !desc || storage < LBM_F64 || storage > LBM_BF16 || !(rho0 > 0.0) || !std::isfinite(rho0))
        return LBM_ERR_INVALID_ARG;
    const int esz = lbm::storage_bytes(storage);
    const int align_elems = 32 / esz;   // 32-byte rows: every 16-byte vector stays aligned
    long long off = 0, nodes = 0;
    std::vector<BatchInstance> inst(n);
    std::vector<long long> node_off(n);
    for (int k = 0; k < n; ++k) {
        const lbm_instance_desc& d = desc[k];
        if (d.nx < 3 || d.ny < 3 || (long long)d.nx * d.ny > (1LL << 31)) return LBM_ERR_INVALID_ARG;
        if (d.model < LBM_BGK || d.model > LBM_K_EQ) return LBM_ERR_INVALID_ARG;
        const lbm_rates& r = d.rates;
        for (double w : {r.omega_nu, r.omega3, r.omega4})
            if (!(std::isfinite(w) && w > 0.0 && w < 2.0)) return LBM_ERR_INVALID_ARG;
        if (!std::isfinite(d.ux_ref) || !std::isfinite(d.uy_ref) || std::fabs(d.ux_ref) >= 1.0 ||
            std::fabs(d.uy_ref) >= 1.0 || !std::isfinite(d.ke_ref) || !std::isfinite(d.ke_factor))
            return LBM_ERR_INVALID_ARG;
        BatchInstance& I = inst[k];
        I.a.nx = d.nx;
        I.a.ny = d.ny;
        I.a.pitch = (d.nx + align_elems - 1) / align_elems * align_elems;
        I.a.nseg = 0;
        I.a.plane = (long long)d.ny * I.a.pitch;
        I.a.w_nu = r.omega_nu;
        I.a.w3 = d.model == LBM_PR ? 1.0 : r.omega3;
        I.a.w4 = d.model == LBM_PR ? 1.0 : r.omega4;
        I.a.rho0 = rho0;
        I.a.urx = d.ux_ref;
        I.a.ury = d.uy_ref;
        // the cumulant readings LBM_K_PRE / LBM_K_EQ: the kernels of LBM_K, other constants
        I.a.kread = d.model == LBM_K_PRE ? 1 : (d.model == LBM_K_EQ ? 2 : 0);
        lbm::fill_consts(I.a);
        I.model = (d.model == LBM_K_PRE || d.model == LBM_K_EQ) ? LBM_K : d.model;
        I.pad = 0;
        I.ke_ref = d.ke_ref;
        I.ke_factor = d.ke_factor;
        off = (off + 127) / 128 * 128;   // 256-byte aligned or better for every storage type
        I.off = off;
        off += 2 * 9 * I.a.plane;
        node_off[k] = nodes;
        nodes += (long long)d.nx * d.ny;
    }
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_NOMEM;
    b->n = n;
    b->storage = storage;
    b->rho0 = rho0;
    b->stream = (cudaStream_t)cuda_stream;
    b->inst = inst;
    b->node_off = node_off;
    b->nodes = nodes;
    b->slab_bytes = (size_t)off * esz;
    // largest instances first (longest-processing-time order for the dynamic queue)
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return (long long)inst[a].a.nx * inst[a].a.ny > (long long)inst[c].a.nx * inst[c].a.ny;
    });
    int rc = LBM_OK;
    cudaError_t e = cudaMalloc(&b->slab, b->slab_bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->slab, 0, b->slab_bytes, b->stream);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_inst, sizeof(BatchInstance) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_state, sizeof(BatchState) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_order, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_queue, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_node_off, sizeof(long long) * n);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_inst, inst.data(), sizeof(BatchInstance) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_node_off, node_off.data(), sizeof(long long) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        rc = e == cudaErrorMemoryAllocation ? LBM_ERR_NOMEM : LBM_ERR_CUDA;
    } else {
        rc = reset_states(b);
        if (rc == LBM_OK) {
            int vec, block;
            default_shape(storage, &vec, &block);
            rc = set_shape(b, vec, block);
        }
    }
    if (rc != LBM_OK) {
        lbm_batch_destroy(b);
        return rc;
    }
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    cudaFree(b->slab);
    cudaFree(b->d_inst);
    cudaFree(b->d_state);
    cudaFree(b->d_order);
    cudaFree(b->d_queue);
    cudaFree(b->d_node_off);
    cudaFree(b->stage);
    delete b;
}

long long lbm_batch_nodes(const lbm_batch* b) { return b ? b->nodes : -1; }

int lbm_batch_init_equilibrium(lbm_batch* b, const double* rho, const double* ux, const double* uy) {
    if (!b || !rho || !ux || !uy) return b ? berr(b, LBM_ERR_INVALID_ARG, "null field") : LBM_ERR_INVALID_ARG;
    int rc = reset_states(b);
    if (rc) return rc;
    const double* in[3] = {rho, ux, uy};
    const double* dev[3];
    const size_t n = (size_t)b->nodes;
    for (int k = 0; k < 3; ++k) {
        if (is_device_ptr(in[k])) {
            dev[k] = in[k];
            continue;
        }
        if (b->stage_elems < 3 * n) {
            cudaFree(b->stage);
            b->stage = nullptr;
            b->stage_elems = 0;
            LBM_BCK(b, cudaMalloc(&b->stage, 3 * n * sizeof(double)));
            b->stage_elems = 3 * n;
        }
        LBM_BCK(b, cudaMemcpyAsync(b->stage + k * n, in[k], n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
        dev[k] = b->stage + k * n;
    }
    LBM_BCK(b, launch_batch_init(b, dev[0], dev[1], dev[2]));
    LBM_BCK(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

int lbm_batch_run(lbm_batch* b, long long target_steps, int check_every, double growth) {
    if (!b) return LBM_ERR_INVALID_ARG;
    if (target_steps < 0 || check_every < 0 || !(growth > 1.0) || !std::isfinite(growth))
        return berr(b, LBM_ERR_INVALID_ARG, "invalid run parameters");
    int rc = record_run(b, target_steps, check_every, growth);
    if (rc) return rc;
    LBM_BCK(b, cudaGraphLaunch(b->exec, b->stream));
    return LBM_OK;
}

int lbm_batch_status(lbm_batch* b, int* status, long long* blowup_step, long long* steps, double* diag4) {
    if (!b) return LBM_ERR_INVALID_ARG;
    std::vector<BatchState> s(b->n);
    LBM_BCK(b, cudaMemcpyAsync(s.data(), b->d_state, sizeof(BatchState) * b->n, cudaMemcpyDeviceToHost, b->stream));
    LBM_BCK(b, cudaStreamSynchronize(b->stream));
    for (int k = 0; k < b->n; ++k) {
        if (status) status[k] = s[k].status;
        if (blowup_step) blowup_step[k] = s[k].blowup_step;
        if (steps) steps[k] = s[k].steps;
        if (diag4) {
            diag4[4 * k + 0] = s[k].pert;
            diag4[4 * k + 1] = s[k].ke;
            diag4[4 * k + 2] = s[k].rho_min;
            diag4[4 * k + 3] = s[k].pert0;
        }
    }
    return LBM_OK;
}

int lbm_batch_get_populations(lbm_batch* b, int index, double* f) {
    if (!b || !f || index < 0 || index >= b->n)
        return b ? berr(b, LBM_ERR_INVALID_ARG, "bad instance index or null output") : LBM_ERR_INVALID_ARG;
    BatchState s;
    LBM_BCK(b, cudaMemcpyAsync(&s, b->d_state + index, sizeof(s), cudaMemcpyDeviceToHost, b->stream));
    LBM_BCK(b, cudaStreamSynchronize(b->stream));
    const BatchInstance& I = b->inst[index];
    lbm::FieldArgs a;
    a.nx = I.a.nx; a.ny = I.a.ny; a.pitch = I.a.pitch; a.plane = I.a.plane; a.rho0 = I.a.rho0;
    a.urx = I.a.urx; a.ury = I.a.ury;
    const char* base = static_cast<const char*>(b->slab) +
                       (size_t)(I.off + (long long)s.cur * 9 * I.a.plane) * lbm::storage_bytes(b->storage);
    const size_t n = (size_t)I.a.nx * I.a.ny;
    double* dst = f;
    double* tmp = nullptr;
    if (!is_device_ptr(f)) {
        LBM_BCK(b, cudaMalloc(&tmp, 9 * n * sizeof(double)));
        dst = tmp;
    }
    cudaError_t e = lbm::launch_gather(b->storage, base, a, dst, nullptr, nullptr, nullptr, nullptr, nullptr,
                                       nullptr, b->stream);
    if (e == cudaSuccess && tmp) e = cudaMemcpyAsync(f, tmp, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return berr(b, LBM_ERR_CUDA, "get_populations: %s", cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_batch_set_shape(lbm_batch* b, int vec, int block) {
    if (!b) return LBM_ERR_INVALID_ARG;
    return set_shape(b, vec, block);
}

int lbm_batch_get_shape(const lbm_batch* b, int* vec, int* block, int* grid) {
    if (!b) return LBM_ERR_INVALID_ARG;
    if (vec) *vec = b->vec;
    if (block) *block = b->block;
    if (grid) *grid = b->grid;
    return LBM_OK;
}

int lbm_batch_autotune(lbm_batch* b, long long trial_steps, int check_every, int* vec, int* block, double* best_ms) {
    if (!b || trial_steps < 1 || check_every < 0) return b ? berr(b, LBM_ERR_INVALID_ARG, "bad trial") : LBM_ERR_INVALID_ARG;
    static const int cand[][2] = {{2, 128}, {2, 256}, {2, 512}, {4, 128}, {4, 256}, {4, 512}, {8, 128}, {8, 256}};
    // save the state, time each shape from it, restore it after every trial
    std::vector<BatchState> s0(b->n);
    LBM_BCK(b, cudaMemcpyAsync(s0.data(), b->d_state, sizeof(BatchState) * b->n, cudaMemcpyDeviceToHost, b->stream));
    LBM_BCK(b, cudaStreamSynchronize(b->stream));
    long long start = 0;
    for (const auto& x : s0) start = std::max(start, x.steps);
    void* saved = nullptr;
    LBM_BCK(b, cudaMalloc(&saved, b->slab_bytes));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t e = cudaMemcpyAsync(saved, b->slab, b->slab_bytes, cudaMemcpyDeviceToDevice, b->stream);
    const int v0 = b->vec, k0 = b->block;
    int best_v = v0, best_b = k0;
    double best = 1e300;
    int rc = LBM_OK;
    for (const auto& c : cand) {
        if (e != cudaSuccess) break;
        if (!pick_batch_kernel(b->storage, c[0], c[1])) continue;
        if (set_shape(b, c[0], c[1]) != LBM_OK) continue;
        rc = record_run(b, start + trial_steps, check_every, 1e4);
        if (rc != LBM_OK) break;
        cudaEventRecord(e0, b->stream);
        e = cudaGraphLaunch(b->exec, b->stream);
        cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) { best = ms; best_v = c[0]; best_b = c[1]; }
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->slab, saved, b->slab_bytes, cudaMemcpyDeviceToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_state, s0.data(), sizeof(BatchState) * b->n, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(saved);
    if (rc != LBM_OK) return rc;
    if (e != cudaSuccess) return berr(b, LBM_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
    rc = set_shape(b, best_v, best_b);
    if (rc) return rc;
    if (vec) *vec = best_v;
    if (block) *block = best_b;
    if (best_ms) *best_ms = best;
    return LBM_OK;
}

}  // extern "C"
