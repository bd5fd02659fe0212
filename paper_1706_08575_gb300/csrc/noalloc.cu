// ftcg_adjoint_small_noalloc: the weighted adjoint of ftcg_adjoint for small images, for callers
// that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a stream is being captured into a
// CUDA graph (allocation is not a capturable operation), real-time sonar processing loops that
// fix their memory footprint at start-up and forbid allocation afterwards, and host frameworks
// that own the device memory pool and hand a library only its inputs and outputs. This entry point
// serves them. Its scratch memory is three file-scope device arrays of fixed size that every GPU
// loading the library holds until the process exits:
//   na_grid   : the sigma-oversampled fine grid, at most kNaMaxGrid^2 complex64 (2 MiB),
//   na_rows   : the grid after the transform along x, at most kNaMaxGrid x kNaMaxGrid complex64
//               (2 MiB),
//   na_deapod : the window factors, at most kNaMaxGrid float64.
// It makes no allocation of any kind (no cudaMalloc, cudaFree, cuFFT plan or host heap). The
// spreading uses global float atomics on na_grid, the inverse transform is a separable direct sum
// (rows, then columns), so only grids of side G = sigma N <= kNaMaxGrid are accepted.
//
// Because every call uses the same arrays, two calls whose work overlaps on the GPU (on different
// streams, or from different host threads without ordering) race and corrupt each other's
// results; calls queued on one stream are ordered and safe. Each call clears na_grid before it
// spreads, so the contents left by the previous call never leak into a result.
//
// Set-up: the first call on each device looks up the device addresses of the arrays with
// cudaGetSymbolAddress (with that device current) and caches them. That first call should
// therefore come before any stream capture on that device.

#include <cmath>
#include <cstring>
#include <mutex>

#include "ftcg_internal.cuh"

namespace {

constexpr int kNaMaxGrid = 512;
constexpr int kNaMaxDevices = 64;
constexpr int kNaQuad = 96;

static __device__ __align__(256) float2 na_grid[kNaMaxGrid * kNaMaxGrid];
static __device__ __align__(256) float2 na_rows[kNaMaxGrid * kNaMaxGrid];
static __device__ __align__(256) double na_deapod[kNaMaxGrid];

struct NaPtrs {
    float2* grid;
    float2* rows;
    double* deapod;
    int sms;          // multiprocessors of the device (sizes the grid-stride spreading launch)
    bool ready;
};
NaPtrs g_na[kNaMaxDevices];
std::mutex g_na_mu;

struct NaQuad {
    double th[kNaQuad];
    double wt[kNaQuad];
};

// Gauss-Legendre nodes on [0, pi/2] (Newton iteration on P_n), into fixed arrays.
void na_quadrature(NaQuad& q) {
    const double pi = 3.14159265358979323846;
    const int n = kNaQuad;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        const double w = 2.0 / ((1.0 - z * z) * dp * dp);
        q.th[i] = 0.25 * pi * (1.0 - z);
        q.th[n - 1 - i] = 0.25 * pi * (1.0 + z);
        q.wt[i] = q.wt[n - 1 - i] = 0.25 * pi * w;
    }
}

__device__ __forceinline__ float na_es32(float t, float inv_hw, float beta) {
    const float z = t * inv_hw;
    const float z2 = z * z;
    const float q = 1.0f - z2;
    return q >= 0.0f ? expf(-beta * z2 / (1.0f + sqrtf(q))) : 0.0f;
}

// 1 / phi^(p / G), p = -N/2 .. N/2-1, in FP64 (same quadrature as the plan's factors).
__global__ void k_na_deapod(double* __restrict__ out, int N, int G, int W, double beta, NaQuad q) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double pi = 3.14159265358979323846;
    const double xi = (double)(i - N / 2) / (double)G, half = 0.5 * W;
    double s = 0.0;
    for (int k = 0; k < kNaQuad; ++k) {
        double sn, cs;
        sincos(q.th[k], &sn, &cs);
        s += q.wt[k] * exp(beta * (cs - 1.0)) * cos(2.0 * pi * xi * half * sn) * half * cs;
    }
    out[i] = 1.0 / (2.0 * s);
}

__global__ void k_na_zero(float2* __restrict__ grid, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        grid[i] = make_float2(0.f, 0.f);
}

// Spreading with global atomics: one 16-lane group per sample, lane l = tap column l.
__global__ void __launch_bounds__(256)
    k_na_spread(const double* __restrict__ lam, const float2* __restrict__ v,
                const double* __restrict__ alpha, int64_t M, double sigma, int G, int W,
                float beta, float inv_hw, float2* __restrict__ grid) {
    const int l = threadIdx.x & 15;
    const unsigned gmask = 0xffffu << ((threadIdx.x & 31) & 16);
    const int64_t ngr = (int64_t)gridDim.x * (blockDim.x / 16);
    for (int64_t j = blockIdx.x * (int64_t)(blockDim.x / 16) + threadIdx.x / 16; j < M; j += ngr) {
        const double ux = __dmul_rn(sigma, lam[2 * j]), uy = __dmul_rn(sigma, lam[2 * j + 1]);
        const bool ok = isfinite(ux) && isfinite(uy) && fabs(ux) < 1125899906842624.0 &&
                        fabs(uy) < 1125899906842624.0;
        if (!ok) continue;                                     // uniform within the group
        const double cx = ceil(__dsub_rn(ux, 0.5 * W)), cy = ceil(__dsub_rn(uy, 0.5 * W));
        const float dx = (float)__dsub_rn(ux, cx), dy = (float)__dsub_rn(uy, cy);
        long long rx = (long long)cx % G, ry = (long long)cy % G;
        if (rx < 0) rx += G;
        if (ry < 0) ry += G;
        const float a = alpha ? (float)alpha[j] : 1.0f;
        const float2 c = v[j];
        const float fx = l < W ? na_es32(dx - (float)l, inv_hw, beta) : 0.0f;
        const float fyl = l < W ? na_es32(dy - (float)l, inv_hw, beta) : 0.0f;
        int col = (int)rx + l;
        if (col >= G) col -= G;
        int row = (int)ry;
        const float xr = a * c.x * fx, xi = a * c.y * fx;
        for (int r = 0; r < W; ++r) {
            const float fy = __shfl_sync(gmask, fyl, r, 16);
            if (l < W) {
                atomicAdd(&grid[row * G + col].x, xr * fy);
                atomicAdd(&grid[row * G + col].y, xi * fy);
            }
            if (++row == G) row = 0;
        }
    }
}

// Transform along x: rows[ly][ix] = sum_lx grid[ly][lx] exp(+2 pi i lx px / G), px = ix - N/2.
__global__ void k_na_rows(const float2* __restrict__ grid, float2* __restrict__ rows, int G,
                          int N) {
    __shared__ float2 s_row[kNaMaxGrid];
    const int ly = blockIdx.x;
    for (int x = threadIdx.x; x < G; x += blockDim.x) s_row[x] = grid[ly * G + x];
    __syncthreads();
    for (int ix = threadIdx.x; ix < N; ix += blockDim.x) {
        int pm = (ix - N / 2) % G;
        if (pm < 0) pm += G;
        float re = 0.f, im = 0.f;
        for (int lx = 0; lx < G; ++lx) {
            const int k = (int)(((long long)lx * pm) % G);
            float sn, cs;
            sincospif(2.0f * (float)k / (float)G, &sn, &cs);
            const float2 g = s_row[lx];
            re += g.x * cs - g.y * sn;
            im += g.x * sn + g.y * cs;
        }
        rows[ly * N + ix] = make_float2(re, im);
    }
}

// Transform along y, window division and crop into the N x N image.
__global__ void k_na_cols(const float2* __restrict__ rows, const double* __restrict__ r,
                          float2* __restrict__ img, int G, int N) {
    const int iy = blockIdx.x;
    int pm = (iy - N / 2) % G;
    if (pm < 0) pm += G;
    for (int ix = threadIdx.x; ix < N; ix += blockDim.x) {
        float re = 0.f, im = 0.f;
        for (int ly = 0; ly < G; ++ly) {
            const int k = (int)(((long long)ly * pm) % G);
            float sn, cs;
            sincospif(2.0f * (float)k / (float)G, &sn, &cs);
            const float2 g = rows[ly * N + ix];
            re += g.x * cs - g.y * sn;
            im += g.x * sn + g.y * cs;
        }
        const double f = r[iy] * r[ix];
        img[iy * N + ix] = make_float2((float)(re * f), (float)(im * f));
    }
}

ftcg_status_t na_fail(ftcg_status_t st, const char* msg) {
    ftcg::set_error("%s", msg);
    return st;
}

}  // namespace

extern "C" ftcg_status_t ftcg_adjoint_small_noalloc(const double* d_lambda, const void* d_values,
                                                    const double* d_alpha, int64_t M, int32_t N,
                                                    double sigma, int32_t w, void* d_image,
                                                    ftcg_stream_t stream) {
    FTCG_API_BEGIN
    ftcg::clear_error();
    if (M < 0) return na_fail(FTCG_ERR_INVALID_VALUE, "ftcg_adjoint_small_noalloc: M < 0");
    if (M > 0 && (!d_lambda || !d_values))
        return na_fail(FTCG_ERR_INVALID_VALUE, "ftcg_adjoint_small_noalloc: NULL input pointer");
    if (!d_image) return na_fail(FTCG_ERR_INVALID_VALUE, "ftcg_adjoint_small_noalloc: image is NULL");
    if (N < 2 || (N & 1))
        return na_fail(FTCG_ERR_INVALID_VALUE, "ftcg_adjoint_small_noalloc: N must be even >= 2");
    if (w < 2 || w > 16)
        return na_fail(FTCG_ERR_INVALID_VALUE, "ftcg_adjoint_small_noalloc: w must be in 2..16");
    if (!(sigma >= 1.0) || !std::isfinite(sigma))
        return na_fail(FTCG_ERR_INVALID_VALUE, "ftcg_adjoint_small_noalloc: sigma must be >= 1");
    const double Gd = sigma * N;
    const long long G = std::llround(Gd);
    if (std::fabs(Gd - (double)G) > 1e-9 * Gd || (G & 1))
        return na_fail(FTCG_ERR_INVALID_VALUE,
                       "ftcg_adjoint_small_noalloc: sigma * N must be an even integer");
    if (G < 2 * w)
        return na_fail(FTCG_ERR_INVALID_VALUE, "ftcg_adjoint_small_noalloc: needs G >= 2 w");
    if (G > kNaMaxGrid) {
        ftcg::set_error("ftcg_adjoint_small_noalloc: G = sigma N = %lld exceeds the fixed scratch "
                        "limit %d (use ftcg_plan / ftcg_adjoint)", G, kNaMaxGrid);
        return FTCG_ERR_NOT_SUPPORTED;
    }
    int dev = 0;
    FTCG_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices)
        return na_fail(FTCG_ERR_NOT_SUPPORTED, "ftcg_adjoint_small_noalloc: device index too large");
    NaPtrs ptrs;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na[dev].ready) {
            NaPtrs p{};
            FTCG_CK(cudaGetSymbolAddress(reinterpret_cast<void**>(&p.grid), na_grid));
            FTCG_CK(cudaGetSymbolAddress(reinterpret_cast<void**>(&p.rows), na_rows));
            FTCG_CK(cudaGetSymbolAddress(reinterpret_cast<void**>(&p.deapod), na_deapod));
            FTCG_CK(cudaDeviceGetAttribute(&p.sms, cudaDevAttrMultiProcessorCount, dev));
            // load every kernel of this entry point now (with lazy module loading a kernel is
            // otherwise loaded at its first launch, which a later captured call could be)
            cudaFuncAttributes fa;
            FTCG_CK(cudaFuncGetAttributes(&fa, k_na_deapod));
            FTCG_CK(cudaFuncGetAttributes(&fa, k_na_zero));
            FTCG_CK(cudaFuncGetAttributes(&fa, k_na_spread));
            FTCG_CK(cudaFuncGetAttributes(&fa, k_na_rows));
            FTCG_CK(cudaFuncGetAttributes(&fa, k_na_cols));
            p.ready = true;
            g_na[dev] = p;
        }
        ptrs = g_na[dev];
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int Gi = (int)G;
    const double beta = ftcg::es_beta(w, sigma);
    NaQuad q;
    na_quadrature(q);
    k_na_deapod<<<(N + 127) / 128, 128, 0, s>>>(ptrs.deapod, N, Gi, w, beta, q);
    k_na_zero<<<256, 256, 0, s>>>(ptrs.grid, Gi * Gi);
    if (M > 0) {
        int64_t blocks = (M * 16 + 255) / 256;
        if (blocks > (int64_t)ptrs.sms * 16) blocks = (int64_t)ptrs.sms * 16;
        k_na_spread<<<(unsigned)blocks, 256, 0, s>>>(
            d_lambda, reinterpret_cast<const float2*>(d_values), d_alpha, M, sigma, Gi, w,
            (float)beta, (float)(2.0 / w), ptrs.grid);
    }
    k_na_rows<<<Gi, 256, 0, s>>>(ptrs.grid, ptrs.rows, Gi, N);
    k_na_cols<<<N, 256, 0, s>>>(ptrs.rows, ptrs.deapod, reinterpret_cast<float2*>(d_image), Gi, N);
    FTCG_CK(cudaGetLastError());
    return FTCG_SUCCESS;
    FTCG_API_END
}
