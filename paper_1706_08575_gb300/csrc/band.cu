// The banded FTCG coefficient matrix C for band r > 1 (Sec. III-C, Eq. ftcg, Eq. cr; in 2-D C_2
// of Eq. twodftcg), reading (i): C minimises || T C - I ||_F over matrices that are zero outside
// the band |j - k| <= r - 1 of the acquisition order (the minimisation of Eq. difopt with its
// diagonal constraint widened to 2r - 1 diagonals). T = Psi Omega is taken as the data-frame Gram
// matrix on the N x N pixel lattice, T_jk = Dx(lambda_k - lambda_j) Dy(lambda_k - lambda_j) with
// the Dirichlet kernel D(d) = N^-1 sum_p exp(2 pi i d p / N) = exp(-i pi d / N) sin(pi d) /
// (N sin(pi d / N)), p in {-N/2 .. N/2 - 1}.
//
// The problem separates over the columns of C: column k solves the least-squares problem
// T[:, S_k] c = e_k over its band rows S_k, whose normal equations are
// (T^2)[S_k, S_k] c = T[S_k, k] (T is Hermitian). At r = 1 this is alpha_k = 1 / S_k (the
// diagonal weights); with the whole index range as band it is C = T^+ (Eq. dif3), whose image is
// the frame approximation (Eq. insert).
//
// Everything runs in FP64 on the device: T (M x M, one thread per entry), the band of T^2
// ((T^2)_{a,a+o}, o = 0..2r-2, one warp per entry reducing over all M samples), and one
// Cholesky solve of the (2r-1) x (2r-1) Hermitian system per column. The cost is O(M^2 r) and
// the memory 16 M^2 bytes, so the path accepts M <= 8192 (the size of the paper's rasters and of
// the tiny configuration). ftcg_adjoint then forms tau = C v (2r - 1 terms per sample) and
// spreads tau with unit weights (Eq. ftcg: tau = C f^).

#include <cmath>

#include "ftcg_internal.cuh"

namespace ftcg {

namespace {

constexpr int kBandMaxR = 12;                 // 2r - 1 <= 23 unknowns per column (the paper's
                                              // largest band, 23 for the asterisk raster)
constexpr int kBandMaxM = 8192;

struct cd {
    double x, y;
};
__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cd cmulc(cd a, cd b) {           // a * conj(b)
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}

// D(d) = exp(-i pi d / N) sin(pi d) / (N sin(pi d / N)). For even N, D is N-periodic, so d is
// first reduced exactly to d' = d - N round(d / N) in [-N/2, N/2] (Sterbenz: no rounding), which
// keeps sin(pi d' / N) away from its aliased zeros; D(0) = 1.
__device__ __forceinline__ cd dirichlet(double d, int N) {
    const double m = rint(d / N);
    const double dr = d - m * N;
    if (dr == 0.0) return {1.0, 0.0};
    double s, c;
    sincospi(dr / N, &s, &c);
    const double ratio = sinpi(dr) / (N * s);
    return {ratio * c, -ratio * s};           // exp(-i pi d' / N) * ratio
}

// T[a * M + j] = T_aj = Dx(lambda_j - lambda_a) Dy(lambda_j - lambda_a)
__global__ void k_gram(const double* __restrict__ lam, int M, int N, cd* __restrict__ T) {
    const int64_t n = (int64_t)M * M;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(i / M), j = (int)(i - (int64_t)a * M);
        const cd dx = dirichlet(lam[2 * j] - lam[2 * a], N);
        const cd dy = dirichlet(lam[2 * j + 1] - lam[2 * a + 1], N);
        T[i] = cmul(dx, dy);
    }
}

// G2[a * nb + o] = (T^2)_{a, a+o} = sum_j T_aj T_j,a+o = sum_j T_aj conj(T_{a+o, j}), one warp
// per (a, o), o = 0..nb-1
__global__ void k_gram2_band(const cd* __restrict__ T, int M, int nb, cd* __restrict__ G2) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int a = warp / nb, o = warp - a * nb;
    if (a >= M) return;
    const int b = a + o;
    double sx = 0.0, sy = 0.0;
    if (b < M) {
        const cd* ra = T + (int64_t)a * M;
        const cd* rb = T + (int64_t)b * M;
        for (int j = lane; j < M; j += 32) {
            const cd p = cmulc(ra[j], rb[j]);
            sx += p.x;
            sy += p.y;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, off);
        sy += __shfl_xor_sync(0xffffffffu, sy, off);
    }
    if (lane == 0) G2[(int64_t)a * nb + o] = {sx, sy};
}

// Column k: A c = rhs with A_il = (T^2)_{S_i, S_l}, rhs_i = T_{S_i, k}, S = k0..k1; Cholesky
// A = L L^H in FP64 (complex), forward and back substitution. Coefficients C[k * nc + (i - k +
// r - 1)] for the band rows i = S; rows outside [0, M) stay zero. A status bit records a
// non-positive pivot (a column whose band is rank deficient; its coefficients stay zero).
// kSolveCols columns per block, each thread with its packed lower triangle (row i from
// i (i + 1) / 2) and right-hand side in shared memory.
constexpr int kSolveCols = 8;

__host__ __device__ constexpr int packed_len(int nc) { return nc * (nc + 1) / 2 + nc; }

__global__ void k_band_solve(const cd* __restrict__ T, const cd* __restrict__ G2, int M, int r,
                             int nb, cd* __restrict__ C, unsigned* __restrict__ status) {
    extern __shared__ cd sm_band[];
    const int k = blockIdx.x * kSolveCols + threadIdx.x;
    if (k >= M) return;
    const int nc = 2 * r - 1;
    cd* L = sm_band + threadIdx.x * packed_len(nc);
    cd* y = L + nc * (nc + 1) / 2;
    auto at = [&](int i, int l) -> cd& { return L[i * (i + 1) / 2 + l]; };
    const int k0 = max(0, k - r + 1), k1 = min(M - 1, k + r - 1);
    const int n = k1 - k0 + 1;
    // lower triangle of A: A_il, i >= l: (T^2)_{S_i, S_l} = conj((T^2)_{S_l, S_i})
    for (int i = 0; i < n; ++i)
        for (int l = 0; l <= i; ++l) {
            const cd g = G2[(int64_t)(k0 + l) * nb + (i - l)];
            at(i, l) = {g.x, -g.y};
        }
    bool ok = true;
    for (int l = 0; l < n && ok; ++l) {
        double d = at(l, l).x;
        for (int m = 0; m < l; ++m) d -= at(l, m).x * at(l, m).x + at(l, m).y * at(l, m).y;
        if (!(d > 0.0)) {
            ok = false;
            break;
        }
        const double dl = sqrt(d);
        at(l, l) = {dl, 0.0};
        for (int i = l + 1; i < n; ++i) {
            cd v = at(i, l);
            for (int m = 0; m < l; ++m) {
                const cd t = cmulc(at(i, m), at(l, m));
                v.x -= t.x;
                v.y -= t.y;
            }
            at(i, l) = {v.x / dl, v.y / dl};
        }
    }
    cd* out = C + (int64_t)k * nc;
    for (int i = 0; i < nc; ++i) out[i] = {0.0, 0.0};
    if (!ok) {
        atomicOr(status, STATUS_BAD_WEIGHT_SUM);
        return;
    }
    for (int i = 0; i < n; ++i) {                          // L y = rhs
        cd v = T[(int64_t)(k0 + i) * M + k];               // T_{S_i, k}
        for (int m = 0; m < i; ++m) {
            const cd t = cmul(at(i, m), y[m]);
            v.x -= t.x;
            v.y -= t.y;
        }
        y[i] = {v.x / at(i, i).x, v.y / at(i, i).x};
    }
    for (int i = n - 1; i >= 0; --i) {                     // L^H c = y
        cd v = y[i];
        for (int m = i + 1; m < n; ++m) {
            const cd t = cmulc(y[m], at(m, i));            // conj(L_mi) c_m
            v.x -= t.x;
            v.y -= t.y;
        }
        y[i] = {v.x / at(i, i).x, v.y / at(i, i).x};
    }
    for (int i = 0; i < n; ++i) out[k0 + i - k + r - 1] = y[i];
}

}  // namespace

// tau_j = sum_k C_jk v_k over the band: column k's coefficient of row j = k + o sits at
// C[k * nc + o + r - 1]
__global__ void k_band_apply(const cd* __restrict__ C, const float2* __restrict__ v, int64_t M,
                             int r, float2* __restrict__ tau) {
    const int nc = 2 * r - 1;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        double sx = 0.0, sy = 0.0;
        for (int o = -(r - 1); o <= r - 1; ++o) {
            const int64_t k = j - o;
            if (k < 0 || k >= M) continue;
            const cd c = C[k * nc + o + r - 1];
            const float2 vk = v[k];
            sx += c.x * vk.x - c.y * vk.y;
            sy += c.x * vk.y + c.y * vk.x;
        }
        tau[j] = make_float2((float)sx, (float)sy);
    }
}

ftcg_status_t band_apply(const Plan& p, const void* vals, cudaStream_t s) {
    int64_t b = (p.M + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    if (b < 1) b = 1;
    k_band_apply<<<(unsigned)b, 256, 0, s>>>(reinterpret_cast<const cd*>(p.band_c),
                                             reinterpret_cast<const float2*>(vals), p.M,
                                             p.band_r, reinterpret_cast<float2*>(p.band_tau));
    FTCG_CK(cudaGetLastError());
    return FTCG_SUCCESS;
}

void release_band(Plan* p) {
    if (p->band_c) cudaFree(p->band_c);
    if (p->band_tau) cudaFree(p->band_tau);
    p->band_c = nullptr;
    p->band_tau = nullptr;
    p->band_r = 0;
}

}  // namespace ftcg

using namespace ftcg;

extern "C" ftcg_status_t ftcg_band(ftcg_plan_t plan, int32_t r, void* d_coef_out,
                                   ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!plan) {
        set_error("ftcg_band: plan is NULL");
        return FTCG_ERR_INVALID_VALUE;
    }
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (r < 1 || r > kBandMaxR) {
        set_error("ftcg_band: r must be in 1..%d", kBandMaxR);
        return FTCG_ERR_INVALID_VALUE;
    }
    if (p->M > kBandMaxM) {
        set_error("ftcg_band: M = %lld > %d: the exact band costs O(M^2 r) and 16 M^2 bytes",
                  (long long)p->M, kBandMaxM);
        return FTCG_ERR_NOT_SUPPORTED;
    }
    if (p->opts.precision != FTCG_PREC_FP32) {
        set_error("ftcg_band: needs an FP32 plan");
        return FTCG_ERR_NOT_SUPPORTED;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    p->last_stream = s;
    const int M = (int)p->M;
    release_band(p);
    if (M == 0) return FTCG_SUCCESS;
    const int nc = 2 * r - 1, nb = 2 * r - 1;      // unknowns per column, offsets of T^2
    cd *T = nullptr, *G2 = nullptr, *C = nullptr;
    FTCG_CK(pool_malloc(&T, (size_t)M * M * sizeof(cd), s));
    FTCG_CK(pool_malloc(&G2, (size_t)M * nb * sizeof(cd), s));
    FTCG_CK(cudaMalloc(&C, (size_t)M * nc * sizeof(cd)));
    p->band_c = C;
    FTCG_CK(cudaMalloc(&p->band_tau, (size_t)M * sizeof(float2)));
    p->band_r = r;
    int64_t nT = (int64_t)M * M;
    k_gram<<<(unsigned)std::min<int64_t>((nT + 255) / 256, 152 * 64), 256, 0, s>>>(p->lambda, M,
                                                                                   p->N, T);
    const int64_t warps = (int64_t)M * nb;
    k_gram2_band<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(T, M, nb, G2);
    const size_t sm = (size_t)kSolveCols * packed_len(nc) * sizeof(cd);
    k_band_solve<<<(M + kSolveCols - 1) / kSolveCols, kSolveCols, sm, s>>>(T, G2, M, r, nb, C,
                                                                           p->status);
    FTCG_CK(cudaGetLastError());
    if (d_coef_out)
        FTCG_CK(cudaMemcpyAsync(d_coef_out, C, (size_t)M * nc * sizeof(cd),
                                cudaMemcpyDeviceToDevice, s));
    FTCG_CK(pool_free(T, s));
    FTCG_CK(pool_free(G2, s));
    // C replaces the diagonal weights: spread tau = C v with unit weights
    FTCG_TRY(launch_set_alpha(*p, nullptr, FTCG_WEIGHTS_F64, s));
    p->band_r = r;
    unsigned st = 0;
    FTCG_CK(cudaMemcpyAsync(&st, p->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    FTCG_CK(cudaStreamSynchronize(s));
    if (st & STATUS_BAD_WEIGHT_SUM) {
        FTCG_CK(cudaMemsetAsync(p->status, 0, sizeof(unsigned), s));
        set_error("ftcg_band: a column's band normal matrix is not positive definite (its "
                  "coefficients are set to zero)");
        return FTCG_ERR_NUMERIC;
    }
    return FTCG_SUCCESS;
    FTCG_API_END
}
