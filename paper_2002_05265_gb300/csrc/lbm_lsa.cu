// Linear stability analysis of the stream-and-collide scheme on the GPU (App. A): the
// perturbed iteration f'(x + xi_i, t + 1) = G f'(x, t), G = d f* / d f the Jacobian of the
// collision map at a uniform equilibrium state, and plane waves f' ~ exp(i(k.x - omega t))
// give the eigenproblem E^D(k) G A = exp(-i omega) A with E^D = diag(exp(-i xi_i . k))
// (Eq. EigenvaluePbDiscrete); the growth rate of a mode is Im(omega) = ln |exp(-i omega)|.
//
// G is exact: row i is the reverse-mode derivative of the kernels' own collision (collide_vjp)
// applied to the unit adjoint e_i.  The eigenvalues of the 9 x 9 complex matrix come from a
// per-thread Householder reduction to upper Hessenberg form and the shifted QR iteration
// (Francis / Wilkinson shift from the trailing 2 x 2 block, Givens rotations, deflation on
// negligible subdiagonal entries), in FP64.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "lbm.h"
#include "lbm_adjoint.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace {

struct Cx {
    double re, im;
};
__device__ __forceinline__ Cx cx(double r, double i = 0.0) { return Cx{r, i}; }
__device__ __forceinline__ Cx operator+(Cx a, Cx b) { return Cx{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ Cx operator-(Cx a, Cx b) { return Cx{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ Cx operator*(Cx a, Cx b) {
    return Cx{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ Cx operator*(double s, Cx a) { return Cx{s * a.re, s * a.im}; }
__device__ __forceinline__ Cx conj(Cx a) { return Cx{a.re, -a.im}; }
__device__ __forceinline__ double cabs(Cx a) { return hypot(a.re, a.im); }
__device__ __forceinline__ Cx cdiv(Cx a, Cx b) {
    const double d = b.re * b.re + b.im * b.im;
    return Cx{(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
// principal square root
__device__ __forceinline__ Cx csqrt(Cx a) {
    const double r = cabs(a);
    if (r == 0.0) return cx(0.0);
    const double t = sqrt(0.5 * (r + fabs(a.re)));
    if (a.re >= 0.0) return Cx{t, a.im / (2.0 * t)};
    return Cx{fabs(a.im) / (2.0 * t), a.im >= 0.0 ? t : -t};
}

constexpr int N = 9;

// Eigenvalues of the complex N x N matrix a (row-major, overwritten).  Returns the number of
// QR sweeps, or -1 if an eigenvalue did not converge within the sweep limit.
__device__ int eig9(Cx (&a)[N][N], Cx (&lam)[N]) {
    // Householder reduction to upper Hessenberg form: for column c, zero a[c+2..][c]
    for (int c = 0; c < N - 2; ++c) {
        double alpha2 = 0.0;
        for (int r = c + 1; r < N; ++r) alpha2 += a[r][c].re * a[r][c].re + a[r][c].im * a[r][c].im;
        const double alpha = sqrt(alpha2);
        if (alpha == 0.0) continue;
        const Cx x0 = a[c + 1][c];
        const double ax0 = cabs(x0);
        const Cx ph = ax0 > 0.0 ? Cx{x0.re / ax0, x0.im / ax0} : cx(1.0);
        // v = x + ph * alpha e_1, H = I - 2 v v^H / (v^H v)
        Cx v[N];
        for (int r = 0; r < N; ++r) v[r] = cx(0.0);
        for (int r = c + 1; r < N; ++r) v[r] = a[r][c];
        v[c + 1] = v[c + 1] + alpha * ph;
        double vn = 0.0;
        for (int r = c + 1; r < N; ++r) vn += v[r].re * v[r].re + v[r].im * v[r].im;
        if (vn == 0.0) continue;
        const double s = 2.0 / vn;
        // a <- H a
        for (int j = 0; j < N; ++j) {
            Cx d = cx(0.0);
            for (int r = c + 1; r < N; ++r) d = d + conj(v[r]) * a[r][j];
            for (int r = c + 1; r < N; ++r) a[r][j] = a[r][j] - s * (v[r] * d);
        }
        // a <- a H
        for (int i = 0; i < N; ++i) {
            Cx d = cx(0.0);
            for (int r = c + 1; r < N; ++r) d = d + a[i][r] * v[r];
            for (int r = c + 1; r < N; ++r) a[i][r] = a[i][r] - s * (d * conj(v[r]));
        }
        for (int r = c + 2; r < N; ++r) a[r][c] = cx(0.0);
    }
    // shifted QR on the active block [lo, hi]; a subdiagonal entry is negligible against its
    // two diagonal neighbours, or against the matrix norm when both are tiny (zero eigenvalues:
    // with omega_3 = omega_4 = 1 the collision removes whole moments)
    double anorm = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) anorm += a[i][j].re * a[i][j].re + a[i][j].im * a[i][j].im;
    anorm = sqrt(anorm);
    int hi = N - 1, sweeps = 0;
    while (hi >= 0) {
        if (hi == 0) {
            lam[0] = a[0][0];
            break;
        }
        // deflation: find the start of the unreduced block ending at hi
        int lo = hi;
        while (lo > 0) {
            const double sc = cabs(a[lo][lo]) + cabs(a[lo - 1][lo - 1]);
            if (cabs(a[lo][lo - 1]) <= 1e-15 * fmax(sc, 1e-3 * anorm)) {
                a[lo][lo - 1] = cx(0.0);
                break;
            }
            --lo;
        }
        if (lo == hi) {
            lam[hi] = a[hi][hi];
            --hi;
            continue;
        }
        if (++sweeps > 60 * N) return -1;
        // Wilkinson shift: eigenvalue of the trailing 2 x 2 block closest to a[hi][hi]
        const Cx p = a[hi - 1][hi - 1], q = a[hi - 1][hi], r = a[hi][hi - 1], t = a[hi][hi];
        const Cx half_tr = 0.5 * (p + t);
        const Cx disc = csqrt(0.25 * ((p - t) * (p - t)) + q * r);
        const Cx e1 = half_tr + disc, e2 = half_tr - disc;
        Cx mu = cabs(e1 - t) < cabs(e2 - t) ? e1 : e2;
        if (sweeps % 11 == 10) {   // exceptional shift, rotating in the complex plane
            const double e = 0.75 * (cabs(a[hi][hi - 1]) + cabs(a[hi - 1][hi - 2 >= 0 ? hi - 2 : 0]));
            double sn, cn;
            sincos(0.7 * sweeps, &sn, &cn);
            mu = a[hi][hi] + Cx{e * cn, e * sn};
        }
        // QR step on a[lo..hi] - mu I with Givens rotations, then RQ + mu I
        Cx cs[N];
        double cc[N];
        for (int k = lo; k <= hi; ++k) a[k][k] = a[k][k] - mu;
        for (int k = lo; k < hi; ++k) {
            const Cx x = a[k][k], y = a[k + 1][k];
            const double nrm = hypot(cabs(x), cabs(y));
            double c;
            Cx sgn;
            if (nrm == 0.0) {
                c = 1.0;
                sgn = cx(0.0);
            } else {
                c = cabs(x) / nrm;
                const Cx ph = cabs(x) > 0.0 ? Cx{x.re / cabs(x), x.im / cabs(x)} : cx(1.0);
                sgn = (1.0 / nrm) * (ph * conj(y));   // s such that [c s; -conj(s) c] [x; y] = [., 0]
            }
            cc[k] = c;
            cs[k] = sgn;
            for (int j = k; j < N; ++j) {
                const Cx u = a[k][j], w = a[k + 1][j];
                a[k][j] = c * u + sgn * w;
                a[k + 1][j] = c * w - conj(sgn) * u;
            }
        }
        for (int k = lo; k < hi; ++k) {
            const double c = cc[k];
            const Cx sgn = cs[k];
            const int top = (k + 2 <= hi) ? k + 2 : hi;
            for (int i = 0; i <= top; ++i) {
                const Cx u = a[i][k], w = a[i][k + 1];
                a[i][k] = c * u + conj(sgn) * w;
                a[i][k + 1] = c * w - sgn * u;
            }
        }
        for (int k = lo; k <= hi; ++k) a[k][k] = a[k][k] + mu;
    }
    return sweeps;
}

// G (row-major 9 x 9, FP64) of the collision map at f = f^eq(rho, u) for each base flow.
template <int MODEL>
__global__ void lsa_jacobian_kernel(const double* __restrict__ flows, int nflows, VjpConsts<double> c,
                                    double* __restrict__ G) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nflows) return;
    const double rho = flows[3 * f], ux = flows[3 * f + 1], uy = flows[3 * f + 2];
    double g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i)   // f^eq (Eq. extendedFeq, product form) minus the shift w_i rho0
        g[i] = rho * phi1d(ex_of(i), ux) * phi1d(ey_of(i), uy) - weight_of(i) * c.rho0;
    for (int i = 0; i < 9; ++i) {
        double v[9], gb[9], wb, w3b, w4b;
#pragma unroll
        for (int j = 0; j < 9; ++j) v[j] = (j == i) ? 1.0 : 0.0;
        collide_vjp<MODEL, double>(g, v, gb, c, wb, w3b, w4b);
#pragma unroll
        for (int j = 0; j < 9; ++j) G[(long long)f * 81 + i * 9 + j] = gb[j];
    }
}

// G of BGK with the second-order (eq_order 2) or partial third-order (3) equilibrium, in
// closed form: f*_i = f_i - omega (f_i - rho p_i(u)) with rho = sum f, u = sum xi f / rho, so
// d f*_i / d f_j = (1 - omega) delta_ij + omega (p_i + dp_i/du_x (xi_jx - u_x) + dp_i/du_y (xi_jy - u_y)).
//   order 2: p_i = w_i (1 + 3 xi.u + 9/2 (xi.u)^2 - 3/2 u^2) (Sec. 2, textbook polynomial);
//   order 3: p_i = phi_sx(u_x) phi_sy(u_y) - u_x^2 u_y^2 b(sx) b(sy) (Eq. extendedFeq minus its
//            A_22 term; b(0) = 1, b(+-1) = -1/2).
__global__ void lsa_jacobian_bgk_kernel(const double* __restrict__ flows, int nflows, double omega, int eq_order,
                                        double* __restrict__ G) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nflows) return;
    const double ux = flows[3 * f + 1], uy = flows[3 * f + 2];
    for (int i = 0; i < 9; ++i) {
        const int sx = ex_of(i), sy = ey_of(i);
        double p, px, py;
        if (eq_order == 2) {
            const double w = weight_of(i), eu = sx * ux + sy * uy;
            p = w * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * (ux * ux + uy * uy));
            px = w * (3.0 * sx + 9.0 * eu * sx - 3.0 * ux);
            py = w * (3.0 * sy + 9.0 * eu * sy - 3.0 * uy);
        } else {
            const double fx = phi1d(sx, ux), fy = phi1d(sy, uy);
            const double dfx = sx ? ux + 0.5 * sx : -2.0 * ux, dfy = sy ? uy + 0.5 * sy : -2.0 * uy;
            const double b = (sx ? -0.5 : 1.0) * (sy ? -0.5 : 1.0);
            p = fx * fy - ux * ux * uy * uy * b;
            px = dfx * fy - 2.0 * ux * uy * uy * b;
            py = fx * dfy - 2.0 * ux * ux * uy * b;
        }
        for (int j = 0; j < 9; ++j)
            G[(long long)f * 81 + i * 9 + j] =
                (i == j ? 1.0 - omega : 0.0) + omega * (p + px * (ex_of(j) - ux) + py * (ey_of(j) - uy));
    }
}

// growth[f * nk + k] = max_j ln |lambda_j(E^D(k) G_f)|; eig (optional) the eigenvalues.
__global__ void lsa_growth_kernel(const double* __restrict__ G, int nflows, const double* __restrict__ kvec, int nk,
                                  double* __restrict__ growth, double* __restrict__ eig, int* __restrict__ failed) {
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= (long long)nflows * nk) return;
    const int f = (int)(id / nk), k = (int)(id - (long long)f * nk);
    const double kx = kvec[2 * k], ky = kvec[2 * k + 1];
    Cx a[N][N], lam[N];
    for (int i = 0; i < N; ++i) {
        double sn, cn;
        sincos(-(ex_of(i) * kx + ey_of(i) * ky), &sn, &cn);
        for (int j = 0; j < N; ++j) {
            const double gij = G[(long long)f * 81 + i * 9 + j];
            a[i][j] = Cx{cn * gij, sn * gij};
        }
    }
    if (eig9(a, lam) < 0) {
        atomicExch(failed, 1);
        growth[id] = nan("");
        return;
    }
    double best = -1e300;
    for (int i = 0; i < N; ++i) {
        const double m = log(cabs(lam[i]));
        best = m > best ? m : best;
        if (eig) {
            eig[id * 18 + 2 * i] = lam[i].re;
            eig[id * 18 + 2 * i + 1] = lam[i].im;
        }
    }
    growth[id] = best;
}

template <int MODEL>
void launch_jacobian(const double* flows, int nflows, const VjpConsts<double>& c, double* G, cudaStream_t s) {
    lsa_jacobian_kernel<MODEL><<<(nflows + 127) / 128, 128, 0, s>>>(flows, nflows, c, G);
}

bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_lsa_growth(int model, lbm_rates rates, int eq_order, const double* flows, int nflows,
                              const double* k, int nk, double* growth, double* eig, double* jac, void* stream) {
    using namespace lbm;
    if (model < LBM_BGK || model > LBM_K_EQ || !flows || !k || !growth || nflows < 1 || nk < 1 ||
        (long long)nflows * nk > (1LL << 31) || eq_order < 2 || eq_order > 4)
        return LBM_ERR_INVALID_ARG;
    if (eq_order != 4 && model != LBM_BGK) return LBM_ERR_UNSUPPORTED;
    const double r[3] = {rates.omega_nu, rates.omega3, rates.omega4};
    for (double w : r)
        if (!(std::isfinite(w) && w > 0.0 && w < 2.0)) return LBM_ERR_INVALID_ARG;
    for (const double* p : {flows, k, (const double*)growth})
        if (!on_device(p)) return LBM_ERR_INVALID_ARG;
    if ((eig && !on_device(eig)) || (jac && !on_device(jac))) return LBM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    VjpConsts<double> c;
    c.w = rates.omega_nu;
    c.w3 = model == LBM_PR ? 1.0 : rates.omega3;
    c.w4 = model == LBM_PR ? 1.0 : rates.omega4;
    c.rho0 = 1.0;
    c.urx = c.ury = 0.0;
    c.Xr = c.Yr = 1.0 / 3.0;
    // cumulant readings: LBM_K_PRE / LBM_K_EQ take the K Jacobian with kappa = 1 / 0
    const int kread = model == LBM_K_PRE ? 1 : (model == LBM_K_EQ ? 2 : 0);
    c.kap = cumulant_kappa(kread, rates.omega_nu);
    c.kapw = kread == 0 ? -1.0 : 0.0;
    if (kread) model = LBM_K;
    double* G = jac;
    int* failed = nullptr;
    cudaError_t e = cudaSuccess;
    if (!G) e = cudaMalloc(&G, sizeof(double) * 81 * (size_t)nflows);
    if (e == cudaSuccess) e = cudaMalloc(&failed, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(failed, 0, sizeof(int), s);
    if (e == cudaSuccess && eq_order != 4) {
        lsa_jacobian_bgk_kernel<<<(nflows + 127) / 128, 128, 0, s>>>(flows, nflows, rates.omega_nu, eq_order, G);
        e = cudaGetLastError();
    } else if (e == cudaSuccess) {
        switch (model) {
            case LBM_BGK: launch_jacobian<BGK>(flows, nflows, c, G, s); break;
            case LBM_RM: launch_jacobian<RM>(flows, nflows, c, G, s); break;
            case LBM_HM: launch_jacobian<HM>(flows, nflows, c, G, s); break;
            case LBM_CM: launch_jacobian<CM>(flows, nflows, c, G, s); break;
            case LBM_CHM: launch_jacobian<CHM>(flows, nflows, c, G, s); break;
            case LBM_K: launch_jacobian<CUM>(flows, nflows, c, G, s); break;
            case LBM_PR: launch_jacobian<PR>(flows, nflows, c, G, s); break;
            default: launch_jacobian<RR>(flows, nflows, c, G, s); break;
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const long long n = (long long)nflows * nk;
        lsa_growth_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(G, nflows, k, nk, growth, eig, failed);
        e = cudaGetLastError();
    }
    int h_failed = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_failed, failed, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (failed) cudaFree(failed);
    if (G && G != jac) cudaFree(G);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LBM_ERR_NOMEM : LBM_ERR_CUDA;
    return h_failed ? LBM_ERR_TIMEOUT : LBM_OK;
}
