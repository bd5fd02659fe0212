// Exact FTCG diagonal weights at band r = 1, in FP64 on the device (Eq. difopt).
//
// With T the data-frame Gram matrix on the N x N pixel lattice,
//     T_jk = (1/N^2) sum_p exp(2 pi i (lambda_k - lambda_j) . p / N),
// min_D || T D - I ||_F separates by columns and gives alpha_k = conj(T_kk) / || T_{:,k} ||^2 =
// 1 / S_k, S_k = sum_j F_N(lambda_jx - lambda_kx) F_N(lambda_jy - lambda_ky), F_N the normalised
// Fejer kernel. Expanding F_N(d) = sum_{|m| < N} ((N - |m|) / N^2) exp(2 pi i d m / N):
//     S_k = sum_m c(m) exp(-2 pi i lambda_k . m / N) H(m),   H(m) = sum_j exp(+2 pi i lambda_j . m / N),
// c(m) = prod_i (N - |m_i|) / N^2 for m in {-N..N-1}^2 (c = 0 at m_i = -N). H is a gridded adjoint
// of unit strengths at 2 lambda on a 2N lattice (W1), the product with c (W2) happens on the
// fine grid together with both window divisions, and S is a gridded forward transform at 2 lambda
// (W3). alpha = 1 / Re S (W4); S >= 1 in exact arithmetic (the j = k term), so S <= 0 or a
// non-finite S flags FTCG_ERR_NUMERIC.

#include <cuda_runtime.h>

#include "ftcg_internal.cuh"

namespace ftcg {

namespace {

__device__ __forceinline__ double es64(double t, double inv_hw, double beta) {
    double z = t * inv_hw;
    double q = 1.0 - z * z;
    return q >= 0.0 ? exp(beta * (sqrt(q) - 1.0)) : 0.0;
}

struct Origin64 {
    long long c;
    double d;
    bool ok;
};

__device__ __forceinline__ Origin64 origin64(double lam, double scale, int W) {
    Origin64 o;
    double u = __dmul_rn(scale, lam);
    o.ok = isfinite(u) && fabs(u) < 1125899906842624.0;
    if (!o.ok) {
        o.c = 0;
        o.d = 0;
        return o;
    }
    double c = ceil(__dsub_rn(u, 0.5 * W));
    o.c = (long long)c;
    o.d = __dsub_rn(u, c);
    return o;
}

__device__ __forceinline__ int wrapi(long long c, int G) {
    long long r = c % G;
    return (int)(r < 0 ? r + G : r);
}

// W1: g_l += phi(u_x - l_x) phi(u_y - l_y) (real, unit strengths), one 16-lane group per sample:
// lane l evaluates tap l of both axes once, the row factors are broadcast by shuffles, and lane l
// adds its column with FP64 global atomics on the real part of a complex128 grid.
__global__ void __launch_bounds__(256)
    k_w1_spread(const double* __restrict__ lam, int64_t M, double scale, int G, int W,
                double beta, double inv_hw, double* __restrict__ grid) {
    const int l = threadIdx.x & 15;
    const unsigned gmask = 0xffffu << ((threadIdx.x & 31) & 16);
    const int64_t ngr = (int64_t)gridDim.x * (blockDim.x / 16);
    const int64_t j0 = blockIdx.x * (int64_t)(blockDim.x / 16) + threadIdx.x / 16;
    for (int64_t j = j0; j < M; j += ngr) {
        Origin64 ox = origin64(lam[2 * j], scale, W);
        Origin64 oy = origin64(lam[2 * j + 1], scale, W);
        if (!ox.ok || !oy.ok) continue;                       // uniform within the group
        const double fx = l < W ? es64(ox.d - l, inv_hw, beta) : 0.0;
        const double fyl = l < W ? es64(oy.d - l, inv_hw, beta) : 0.0;
        const int col = wrapi(ox.c + l, G);
        int row = wrapi(oy.c, G);
        for (int r = 0; r < W; ++r) {
            const double fy = __shfl_sync(gmask, fyl, r, 16);
            if (l < W) atomicAdd(grid + 2 * ((int64_t)row * G + col), fx * fy);
            if (++row == G) row = 0;
        }
    }
}

// W2: on the fine grid after the inverse FFT, keep q = m mod G for m in {-N..N-1}^2 and multiply
// by r(m_x) r(m_y) (adjoint window division) * c(m) * r(m_x) r(m_y) (forward window division);
// zero every other cell. r has 2N entries for m = -N..N-1.
__global__ void k_w2_lag(double2* __restrict__ grid, int G, int N, const double* __restrict__ r) {
    const int64_t total = (int64_t)G * G;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int qy = (int)(i / G), qx = (int)(i - (int64_t)qy * G);
        int my = qy < N ? qy : (qy >= G - N ? qy - G : INT32_MIN);
        int mx = qx < N ? qx : (qx >= G - N ? qx - G : INT32_MIN);
        double2 v = grid[i];
        if (my == INT32_MIN || mx == INT32_MIN) {
            v.x = 0.0;
            v.y = 0.0;
        } else {
            const double ry = r[my + N], rx = r[mx + N];
            const double cx = (double)(N - (mx < 0 ? -mx : mx)) / ((double)N * N);
            const double cy = (double)(N - (my < 0 ? -my : my)) / ((double)N * N);
            const double f = rx * rx * ry * ry * cx * cy;
            v.x *= f;
            v.y *= f;
        }
        grid[i] = v;
    }
}

// W3 + W4: S_k = sum_taps phi phi h_l at 2 lambda_k; alpha_k = 1 / Re S_k.
__global__ void __launch_bounds__(256)
    k_w3_interp(const double* __restrict__ lam, int64_t M, double scale, int G, int W,
                double beta, double inv_hw, const double2* __restrict__ grid,
                double* __restrict__ alpha, unsigned* __restrict__ status) {
    const int l = threadIdx.x & 15;
    const unsigned gmask = 0xffffu << ((threadIdx.x & 31) & 16);
    const int64_t ngr = (int64_t)gridDim.x * (blockDim.x / 16);
    for (int64_t j = blockIdx.x * (int64_t)(blockDim.x / 16) + threadIdx.x / 16; j < M; j += ngr) {
        Origin64 ox = origin64(lam[2 * j], scale, W);
        Origin64 oy = origin64(lam[2 * j + 1], scale, W);
        const bool ok = ox.ok && oy.ok;                       // uniform within the group
        double sr = 0.0;
        if (ok) {
            const double fx = l < W ? es64(ox.d - l, inv_hw, beta) : 0.0;
            const double fyl = l < W ? es64(oy.d - l, inv_hw, beta) : 0.0;
            const int col = wrapi(ox.c + l, G);
            int row = wrapi(oy.c, G);
            for (int r = 0; r < W; ++r) {
                const double fy = __shfl_sync(gmask, fyl, r, 16);
                if (l < W) sr += fy * grid[(int64_t)row * G + col].x;
                if (++row == G) row = 0;
            }
            sr *= fx;
        }
        for (int o = 8; o > 0; o >>= 1) sr += __shfl_xor_sync(gmask, sr, o, 16);
        if (l == 0) {
            if (!ok) {
                alpha[j] = 0.0;
            } else if (!(sr > 0.0) || !isfinite(sr)) {
                alpha[j] = 0.0;
                atomicOr(status, STATUS_BAD_WEIGHT_SUM);
            } else {
                alpha[j] = 1.0 / sr;
            }
        }
    }
}

int nblocks(int64_t n, int t) {
    int64_t b = (n + t - 1) / t;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

}  // namespace

ftcg_status_t compute_weights(Plan& p, double* d_alpha_out, cudaStream_t s) {
    if (p.M == 0) return FTCG_SUCCESS;
    const int Wa = p.opts.weight_width > 0 ? p.opts.weight_width : 12;
    const int N2 = 2 * p.N;
    const int G2 = 2 * p.G;                      // sigma * (2N)
    const double scale = 2.0 * p.sigma;          // u = sigma * (2 lambda)
    Window wa{Wa, es_beta(Wa, p.sigma)};
    const double inv_hw = 2.0 / Wa;

    double* r2 = nullptr;
    double2* g = nullptr;
    double* alpha = d_alpha_out;
    bool own_alpha = false;
    unsigned before = 0;
    const size_t gbytes = (size_t)G2 * G2 * sizeof(double2);
    FTCG_CK(cudaMalloc(&r2, N2 * sizeof(double)));
    cudaError_t e = cudaMalloc(&g, gbytes);
    if (e != cudaSuccess) {
        cudaFree(r2);
        set_error("ftcg_weights: cannot allocate the %zu-byte FP64 lag grid", gbytes);
        return FTCG_ERR_OUT_OF_MEMORY;
    }
    if (!alpha) {
        e = cudaMalloc(&alpha, p.M * sizeof(double));
        if (e != cudaSuccess) {
            cudaFree(r2);
            cudaFree(g);
            set_error("ftcg_weights: cannot allocate the weight array");
            return FTCG_ERR_OUT_OF_MEMORY;
        }
        own_alpha = true;
    }
    cufftHandle plan2 = 0;
    ftcg_status_t st = FTCG_SUCCESS;
    do {
        if ((st = window_factors(r2, N2, G2, wa, s)) != FTCG_SUCCESS) break;
        if (cudaMemsetAsync(g, 0, gbytes, s) != cudaSuccess) { st = FTCG_ERR_CUDA; break; }
        k_w1_spread<<<nblocks(p.M * 16, 256), 256, 0, s>>>(p.lambda, p.M, scale, G2, Wa, wa.beta,
                                                            inv_hw, reinterpret_cast<double*>(g));
        if (cufftPlan2d(&plan2, G2, G2, CUFFT_Z2Z) != CUFFT_SUCCESS) {
            set_error("ftcg_weights: cufftPlan2d(Z2Z %d) failed", G2);
            st = FTCG_ERR_CUDA;
            break;
        }
        cufftSetStream(plan2, s);
        if (cufftExecZ2Z(plan2, reinterpret_cast<cufftDoubleComplex*>(g),
                         reinterpret_cast<cufftDoubleComplex*>(g), CUFFT_INVERSE) != CUFFT_SUCCESS) {
            set_error("ftcg_weights: inverse Z2Z failed");
            st = FTCG_ERR_CUDA;
            break;
        }
        k_w2_lag<<<nblocks((int64_t)G2 * G2, 256), 256, 0, s>>>(g, G2, p.N, r2);
        if (cufftExecZ2Z(plan2, reinterpret_cast<cufftDoubleComplex*>(g),
                         reinterpret_cast<cufftDoubleComplex*>(g), CUFFT_FORWARD) != CUFFT_SUCCESS) {
            set_error("ftcg_weights: forward Z2Z failed");
            st = FTCG_ERR_CUDA;
            break;
        }
        if (cudaMemcpyAsync(&before, p.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess) { st = FTCG_ERR_CUDA; break; }
        k_w3_interp<<<nblocks(p.M * 16, 256), 256, 0, s>>>(p.lambda, p.M, scale, G2, Wa, wa.beta,
                                                            inv_hw, g, alpha, p.status);
        if (cudaGetLastError() != cudaSuccess) { st = FTCG_ERR_CUDA; break; }
        if ((st = launch_set_alpha(p, alpha, FTCG_WEIGHTS_F64, s)) != FTCG_SUCCESS) break;
        unsigned after = 0;
        if (cudaMemcpyAsync(&after, p.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            set_error("ftcg_weights: %s", cudaGetErrorString(cudaGetLastError()));
            st = FTCG_ERR_CUDA;
            break;
        }
        if ((after & STATUS_BAD_WEIGHT_SUM) && !(before & STATUS_BAD_WEIGHT_SUM)) {
            set_error("ftcg_weights: a weight sum S_k was <= 0 or not finite (weight set to 0)");
            st = FTCG_ERR_NUMERIC;
        }
    } while (0);
    if (st == FTCG_ERR_CUDA && ftcg_last_error()[0] == 0)
        set_error("ftcg_weights: %s", cudaGetErrorString(cudaGetLastError()));
    cudaStreamSynchronize(s);
    if (plan2) cufftDestroy(plan2);
    cudaFree(r2);
    cudaFree(g);
    if (own_alpha) cudaFree(alpha);
    return st;
}

}  // namespace ftcg
