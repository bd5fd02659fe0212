// The frame approximation on the device (Sec. III-B, Eq. afr / afrm; 2-D: Eq. twodframe,
// twodframeB): the minimum-norm least-squares image x = E^+ v of the data frame
// E_jp = exp(-2 pi i lambda_j . p / N), computed by CGLS (conjugate gradients on the normal
// equations, Hestenes-Stiefel form) with the plan's gridded operators standing in for E
// (ftcg_forward) and E^H (ftcg_adjoint). Optional row weights w_j (for example the FTCG weights)
// turn the problem into min || W^(1/2) (E x - v) ||: started from zero, the first iterate is a
// multiple of E^H W v, the FTCG image, and the FTCG weights act as a preconditioner (Sec. V-C's
// condition numbers of Psi and C_2).
//
// Vectors are FP32 complex (the operators' precision); the scalars of the recursion (the squared
// norms gamma = ||E^H W r||^2 and ||W^(1/2) E p||^2) are FP64 device reductions, and the step
// lengths are formed on the device from them, so an iteration queues its kernels without any
// host synchronisation; the host reads the residual history once at the end. An iteration whose
// gamma has fallen to tol^2 gamma_0 (or whose search direction vanished) freezes the iterate.

#include <cmath>
#include <vector>

#include "ftcg_internal.cuh"

namespace ftcg {

namespace {

constexpr int kThreads = 256;

// device scalars of the recursion
enum { SC_GAMMA = 0, SC_QQ = 1, SC_GNEW = 2, SC_GAMMA0 = 3, SC_TOL2 = 4, SC_N = 8 };

int blocks_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > 152 * 8) b = 152 * 8;
    return (int)b;
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double part[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < kThreads / 32 ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;                                   // valid in thread 0
}

__device__ __forceinline__ bool frozen(const double* sc) {
    return !(sc[SC_GAMMA] > sc[SC_TOL2] * sc[SC_GAMMA0]) || !(sc[SC_QQ] > 0.0);
}

// sw_j = sqrt(w_j) (1 without weights); r = sw v
__global__ void k_init(const float2* __restrict__ v, const double* __restrict__ w, int64_t M,
                       float* __restrict__ sw, float2* __restrict__ r) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        const float s = w ? (float)sqrt(w[j]) : 1.0f;
        sw[j] = s;
        r[j] = make_float2(s * v[j].x, s * v[j].y);
    }
}

// out += sum |x|^2 (x optionally scaled in place by sw first)
__global__ void k_norm2(float2* __restrict__ x, const float* __restrict__ sw, int64_t n,
                        double* __restrict__ out) {
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float2 a = x[i];
        if (sw) {
            a.x *= sw[i];
            a.y *= sw[i];
            x[i] = a;
        }
        acc += (double)a.x * a.x + (double)a.y * a.y;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) atomicAdd(out, acc);
}

// gamma_0 = gamma, the history's first entry, and the tolerance
__global__ void k_start(double* __restrict__ sc, double tol2, double* __restrict__ hist) {
    sc[SC_GAMMA0] = sc[SC_GAMMA];
    sc[SC_TOL2] = tol2;
    sc[SC_QQ] = 1.0;                            // no direction has vanished yet
    hist[0] = sqrt(sc[SC_GAMMA]);
}

__global__ void k_copy(const float2* __restrict__ a, float2* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

__global__ void k_zero_scalar(double* __restrict__ x) { *x = 0.0; }

// x += a p over the image, r -= a q over the samples, a = gamma / qq (0 once frozen)
__global__ void k_step(float2* __restrict__ x, const float2* __restrict__ p, int64_t nimg,
                       float2* __restrict__ r, const float2* __restrict__ q, int64_t M,
                       const double* __restrict__ sc) {
    const float a = frozen(sc) ? 0.0f : (float)(sc[SC_GAMMA] / sc[SC_QQ]);
    const int64_t n = nimg > M ? nimg : M;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nimg) {
            const float2 pi = p[i];
            float2 xi = x[i];
            xi.x = fmaf(a, pi.x, xi.x);
            xi.y = fmaf(a, pi.y, xi.y);
            x[i] = xi;
        }
        if (i < M) {
            const float2 qi = q[i];
            float2 ri = r[i];
            ri.x = fmaf(-a, qi.x, ri.x);
            ri.y = fmaf(-a, qi.y, ri.y);
            r[i] = ri;
        }
    }
}

// p = s + (gamma_new / gamma) p (p unchanged once frozen)
__global__ void k_direction(const float2* __restrict__ s, float2* __restrict__ p, int64_t n,
                            const double* __restrict__ sc) {
    if (frozen(sc)) return;
    const float beta = (float)(sc[SC_GNEW] / sc[SC_GAMMA]);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 si = s[i];
        float2 pi = p[i];
        pi.x = fmaf(beta, pi.x, si.x);
        pi.y = fmaf(beta, pi.y, si.y);
        p[i] = pi;
    }
}

// gamma = gamma_new (unless frozen), history entry k, scalars of the next iteration zeroed
__global__ void k_next(double* __restrict__ sc, double* __restrict__ hist, int k) {
    const bool fz = frozen(sc);
    if (!fz) sc[SC_GAMMA] = sc[SC_GNEW];
    hist[k] = sqrt(sc[SC_GAMMA]);
    sc[SC_GNEW] = 0.0;
}

}  // namespace

}  // namespace ftcg

using namespace ftcg;

extern "C" ftcg_status_t ftcg_cgls(ftcg_plan_t plan, const void* d_values,
                                   const double* d_row_weights, int32_t iters, double tol,
                                   void* d_image, double* h_resnorms, int32_t* h_iters,
                                   ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!plan || !d_image) {
        set_error("ftcg_cgls: plan or image is NULL");
        return FTCG_ERR_INVALID_VALUE;
    }
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (p->M > 0 && !d_values) {
        set_error("ftcg_cgls: values pointer is NULL");
        return FTCG_ERR_INVALID_VALUE;
    }
    if (iters < 0 || iters > 100000 || !(tol >= 0.0) || !std::isfinite(tol)) {
        set_error("ftcg_cgls: iters must be in 0..100000 and tol >= 0");
        return FTCG_ERR_INVALID_VALUE;
    }
    if (p->opts.precision != FTCG_PREC_FP32) {
        set_error("ftcg_cgls: needs an FP32 plan (the row weights are applied in FP32)");
        return FTCG_ERR_NOT_SUPPORTED;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    p->last_stream = s;
    const int64_t M = p->M, nimg = (int64_t)p->N * p->N;
    float2* x = reinterpret_cast<float2*>(d_image);
    FTCG_CK(cudaMemsetAsync(x, 0, nimg * sizeof(float2), s));
    if (M == 0) {
        if (h_resnorms)
            for (int k = 0; k <= iters; ++k) h_resnorms[k] = 0.0;
        if (h_iters) *h_iters = 0;
        return FTCG_SUCCESS;
    }
    float *sw = nullptr;
    float2 *r = nullptr, *q = nullptr, *sv = nullptr, *pv = nullptr;
    double *sc = nullptr, *hist = nullptr;
    FTCG_CK(pool_malloc(&sw, M * sizeof(float), s));
    FTCG_CK(pool_malloc(&r, M * sizeof(float2), s));
    FTCG_CK(pool_malloc(&q, M * sizeof(float2), s));
    FTCG_CK(pool_malloc(&sv, nimg * sizeof(float2), s));
    FTCG_CK(pool_malloc(&pv, nimg * sizeof(float2), s));
    FTCG_CK(pool_malloc(&sc, SC_N * sizeof(double), s));
    FTCG_CK(pool_malloc(&hist, (size_t)(iters + 1) * sizeof(double), s));
    FTCG_CK(cudaMemsetAsync(sc, 0, SC_N * sizeof(double), s));
    ftcg_status_t st = FTCG_SUCCESS;
    auto run = [&]() -> ftcg_status_t {
        k_init<<<blocks_for(M), kThreads, 0, s>>>(reinterpret_cast<const float2*>(d_values),
                                                 d_row_weights, M, sw, r);
        FTCG_CK(cudaGetLastError());
        // the plan's adjoint spreads with its installed weights: sw for the iteration, so that
        // adjoint(r) = E^H (sw r)
        FTCG_TRY(install_alpha(*p, sw, FTCG_WEIGHTS_F32, s));
        FTCG_TRY(adjoint_device(p, r, FTCG_VALUES_C64, sv, s, false));   // s = E^H W v
        k_norm2<<<blocks_for(nimg), kThreads, 0, s>>>(sv, nullptr, nimg, sc + SC_GAMMA);
        k_start<<<1, 1, 0, s>>>(sc, tol * tol, hist);
        k_copy<<<blocks_for(nimg), kThreads, 0, s>>>(sv, pv, nimg);
        FTCG_CK(cudaGetLastError());
        for (int k = 1; k <= iters; ++k) {
            k_zero_scalar<<<1, 1, 0, s>>>(sc + SC_QQ);
            FTCG_TRY(forward_device(p, pv, q, s));                       // q = E p
            k_norm2<<<blocks_for(M), kThreads, 0, s>>>(q, sw, M, sc + SC_QQ);   // q = sw q
            k_step<<<blocks_for(nimg > M ? nimg : M), kThreads, 0, s>>>(x, pv, nimg, r, q, M, sc);
            FTCG_CK(cudaGetLastError());
            FTCG_TRY(adjoint_device(p, r, FTCG_VALUES_C64, sv, s, false));   // s = E^H (sw r)
            k_norm2<<<blocks_for(nimg), kThreads, 0, s>>>(sv, nullptr, nimg, sc + SC_GNEW);
            k_direction<<<blocks_for(nimg), kThreads, 0, s>>>(sv, pv, nimg, sc);
            k_next<<<1, 1, 0, s>>>(sc, hist, k);
            FTCG_CK(cudaGetLastError());
        }
        return FTCG_SUCCESS;
    };
    st = run();
    // restore the plan's own weights whatever happened above
    ftcg_status_t rs = install_alpha(*p, p->alpha_cur, FTCG_WEIGHTS_F32, s);
    if (st == FTCG_SUCCESS) st = rs;
    std::vector<double> h(iters + 1, 0.0);
    if (st == FTCG_SUCCESS) {
        cudaError_t ce = cudaMemcpyAsync(h.data(), hist, (iters + 1) * sizeof(double),
                                         cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) {
            set_error("ftcg_cgls: reading the residual history: %s", cudaGetErrorString(ce));
            st = FTCG_ERR_CUDA;
        }
    }
    pool_free(sw, s);
    pool_free(r, s);
    pool_free(q, s);
    pool_free(sv, s);
    pool_free(pv, s);
    pool_free(sc, s);
    pool_free(hist, s);
    if (st != FTCG_SUCCESS) return st;
    int done = iters;
    for (int k = 0; k <= iters; ++k)
        if (!(h[k] > tol * h[0])) {
            done = k;
            break;
        }
    if (h_resnorms)
        for (int k = 0; k <= iters; ++k) h_resnorms[k] = h[k];
    if (h_iters) *h_iters = done;
    return FTCG_SUCCESS;
    FTCG_API_END
}
