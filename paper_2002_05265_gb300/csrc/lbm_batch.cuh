// Batched stability sweep: thousands of independent periodic lattices of uneven size, each
// with its own collision model, relaxation rates and blow-up state, advanced by ONE
// persistent launch (the numerical-stability study of Sec. 5b run as a batch).
//
// Scheduling: the grid holds as many CTAs as the GPU keeps resident.  Each CTA repeatedly
// claims the next instance from a global counter (instances ordered largest first), and
// advances that instance alone from its current step to the target step: every time step is
// one sweep of the CTA over the instance's vector segments followed by __syncthreads(), which
// is the per-instance barrier (an instance never spans CTAs, so no inter-CTA waits exist and
// nothing can deadlock).  Every `check_every` steps the sweep also accumulates the blow-up
// diagnostics of the pre-collision state in FP64 (perturbation energy, kinetic energy,
// minimum density, non-finite count), folded across the CTA; an instance that blows up stops
// and its CTA claims the next one.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

struct BatchInstance {   // read-only during a run
    long long off;       // element offset of buffer 0 in the slab; buffer 1 at off + 9 * plane
    StepArgs a;          // geometry (nseg is recomputed for the kernel's VEC), rates, shift
    int model;           // lbm::Model
    int pad;
    double ke_ref, ke_factor;   // optional <|u|^2> > ke_factor * ke_ref criterion (ke_ref > 0)
};

struct BatchState {      // updated by the kernel, one per instance
    long long steps;     // time steps taken
    long long blowup_step;   // step of the check that fired, -1 if none
    double pert0;        // <|u - u_ref|^2> at the first check (-1 until taken)
    double pert, ke, rho_min, nonfinite;   // diagnostics of the last check
    int status;          // 0 = running or finished, LBM_ERR_BLOWUP (-4) = blown up
    int cur;             // buffer holding the current state
};

constexpr double kPertFloor = 1e-20;   // <|u - u_ref|^2> below this counts as "no perturbation"

template <int MODEL, typename S, int VEC, int BLOCK>
__device__ __forceinline__ void batch_instance_loop(S* __restrict__ buf0, S* __restrict__ buf1, const StepArgs& a,
                                                    const BatchInstance& I, BatchState& st, long long target,
                                                    int check_every, double growth, double (*s_red)[4],
                                                    int* s_stop) {
    using T = typename Conv<S>::T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned total = (unsigned)a.ny * (unsigned)a.nseg;
    const Consts<T> c = make_consts<T>(a);
    long long t = st.steps;
    int cur = st.cur;
    const double nodes = (double)a.nx * (double)a.ny;
    while (t < target) {
        const bool check = (check_every > 0) && (t % check_every == 0);
        const S* src = cur ? buf1 : buf0;
        S* dst = cur ? buf0 : buf1;
        Diag dg = {0.0, 0.0, 1e300, 0.0};
        if (check) {
            for (unsigned base = threadIdx.x & ~31u; base < total; base += BLOCK)
                step_segment<MODEL, 4, S, VEC, true, true>(src, dst, a, c, base + lane, total, lane, dg);
            // fold the diagnostics over the CTA
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                dg.pert += __shfl_down_sync(0xffffffffu, dg.pert, o);
                dg.ke += __shfl_down_sync(0xffffffffu, dg.ke, o);
                dg.rho_min = fmin(dg.rho_min, __shfl_down_sync(0xffffffffu, dg.rho_min, o));
                dg.nonfinite += __shfl_down_sync(0xffffffffu, dg.nonfinite, o);
            }
            if (lane == 0) {
                s_red[warp][0] = dg.pert; s_red[warp][1] = dg.ke;
                s_red[warp][2] = dg.rho_min; s_red[warp][3] = dg.nonfinite;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double p = 0.0, k = 0.0, r = 1e300, nf = 0.0;
                for (int w = 0; w < BLOCK / 32; ++w) {
                    p += s_red[w][0]; k += s_red[w][1]; r = fmin(r, s_red[w][2]); nf += s_red[w][3];
                }
                p /= nodes;
                k /= nodes;
                st.pert = p; st.ke = k; st.rho_min = r; st.nonfinite = nf;
                bool blown = (nf > 0.0) || !(r > 0.0);
                if (st.pert0 < 0.0) st.pert0 = p;
                else if (p > growth * fmax(st.pert0, kPertFloor)) blown = true;
                if (I.ke_ref > 0.0 && k > I.ke_factor * I.ke_ref) blown = true;
                if (blown) {
                    st.status = -4;   // LBM_ERR_BLOWUP
                    st.blowup_step = t;
                }
                *s_stop = blown ? 1 : 0;
            }
        } else {
            for (unsigned base = threadIdx.x & ~31u; base < total; base += BLOCK)
                step_segment<MODEL, 4, S, VEC, false, true>(src, dst, a, c, base + lane, total, lane, dg);
        }
        __syncthreads();   // step t complete (stores visible to the CTA) before step t + 1 reads
        cur ^= 1;
        ++t;
        if (check && *s_stop) break;
    }
    if (threadIdx.x == 0) {
        st.steps = t;
        st.cur = cur;
    }
}

template <typename S, int VEC, int BLOCK>
__global__ void __launch_bounds__(BLOCK) batch_kernel(S* slab, const BatchInstance* __restrict__ inst,
                                                      BatchState* state, const int* __restrict__ order, int n,
                                                      int* queue, long long target, int check_every, double growth) {
    __shared__ int s_id;
    __shared__ int s_stop;
    __shared__ double s_red[BLOCK / 32][4];
    for (;;) {
        if (threadIdx.x == 0) {
            const int q = atomicAdd(queue, 1);
            s_id = (q < n) ? order[q] : -1;
        }
        __syncthreads();
        const int id = s_id;
        if (id < 0) return;
        const BatchInstance I = inst[id];
        BatchState& st = state[id];
        // every thread reads the same state words; only thread 0 writes them, after barriers
        const bool live = (st.status == 0) && (st.steps < target);
        if (live) {
            StepArgs a = I.a;
            a.nseg = (a.nx + VEC - 1) / VEC;
            S* b0 = slab + I.off;
            S* b1 = b0 + 9 * a.plane;
            switch (I.model) {
                case BGK: batch_instance_loop<BGK, S, VEC, BLOCK>(b0, b1, a, I, st, target, check_every, growth, s_red, &s_stop); break;
                case RM: batch_instance_loop<RM, S, VEC, BLOCK>(b0, b1, a, I, st, target, check_every, growth, s_red, &s_stop); break;
                case HM: batch_instance_loop<HM, S, VEC, BLOCK>(b0, b1, a, I, st, target, check_every, growth, s_red, &s_stop); break;
                case CM: batch_instance_loop<CM, S, VEC, BLOCK>(b0, b1, a, I, st, target, check_every, growth, s_red, &s_stop); break;
                case CHM: batch_instance_loop<CHM, S, VEC, BLOCK>(b0, b1, a, I, st, target, check_every, growth, s_red, &s_stop); break;
                case CUM: batch_instance_loop<CUM, S, VEC, BLOCK>(b0, b1, a, I, st, target, check_every, growth, s_red, &s_stop); break;
                case PR: batch_instance_loop<PR, S, VEC, BLOCK>(b0, b1, a, I, st, target, check_every, growth, s_red, &s_stop); break;
                default: batch_instance_loop<RR, S, VEC, BLOCK>(b0, b1, a, I, st, target, check_every, growth, s_red, &s_stop); break;
            }
        }
        __syncthreads();   // state written and s_id consumed before the next claim
    }
}

}  // namespace lbm
