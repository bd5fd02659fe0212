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
//
// The W1 grid is real (unit strengths, real window), so H is Hermitian, and so is H c (c and the
// window factors are real and even); the result of W3's transform is then real. The transforms
// are therefore a real-to-complex FFT (D2Z, exponent sign -, which gives conj(H) for a real grid)
// and a complex-to-real FFT (Z2D, sign +): conj(sum_m H(m) c(m) e^{-...}) = the real S grid. Both
// are in place on a real grid padded to G + 2 doubles per row. W1 stores each sample's 2 w window
// values so that W3 reads them instead of evaluating the window again.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <utility>

#include "ftcg_internal.cuh"

namespace ftcg {

namespace {

// The window on the weight path, in FP64, as one polynomial per tap: the first-tap offset d lies in
// (w/2 - 1, w/2], so tap l's argument d - l covers one unit interval, and with s = d - (w/2 - 1)
// in (0, 1] phi(d - l) = p_l(2 s - 1). p_l has degree kPolyDeg and interpolates phi at the
// Chebyshev points of its interval (coefficients from window_poly on the host). The end
// intervals hold the window's square-root branch point, where phi = exp(-beta); the interpolation
// error there is about exp(-beta) / 2 of phi(0) (6e-13 at w = 12, sigma = 2; 1e-10 at w = 12,
// sigma = 1.25) and far smaller inside, i.e. at the level of the window's own truncation.
constexpr int kPolyDeg = 14;
constexpr int kPolyMaxW = 16;

struct PolyCoef {
    double c[kPolyMaxW][kPolyDeg + 1];   // c[l][k]: coefficient of x^k in p_l
};

__device__ __forceinline__ double poly_eval(const double* c, double x) {
    double v = c[kPolyDeg];
#pragma unroll
    for (int k = kPolyDeg - 1; k >= 0; --k) v = fma(v, x, c[k]);
    return v;
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
// lane l evaluates tap l of both axes once with its polynomial (and stores both values in the
// sample's row of phi), the row factors are broadcast by shuffles, and lane l adds its column with
// FP64 global atomics to the real grid (row stride ld).
__global__ void __launch_bounds__(256)
    k_w1_spread(const double* __restrict__ lam, int64_t M, double scale, int G, int64_t ld, int W,
                const PolyCoef* __restrict__ pc, double* __restrict__ grid,
                double* __restrict__ phi) {
    const int l = threadIdx.x & 15;
    const unsigned gmask = 0xffffu << ((threadIdx.x & 31) & 16);
    double c[kPolyDeg + 1];                  // this lane's tap polynomial
#pragma unroll
    for (int k = 0; k <= kPolyDeg; ++k) c[k] = l < W ? pc->c[l][k] : 0.0;
    const double s0 = 0.5 * W - 1.0;
    const int64_t ngr = (int64_t)gridDim.x * (blockDim.x / 16);
    const int64_t j0 = blockIdx.x * (int64_t)(blockDim.x / 16) + threadIdx.x / 16;
    for (int64_t j = j0; j < M; j += ngr) {
        Origin64 ox = origin64(lam[2 * j], scale, W);
        Origin64 oy = origin64(lam[2 * j + 1], scale, W);
        if (!ox.ok || !oy.ok) continue;                       // uniform within the group
        const double fx = l < W ? poly_eval(c, 2.0 * (ox.d - s0) - 1.0) : 0.0;
        const double fyl = l < W ? poly_eval(c, 2.0 * (oy.d - s0) - 1.0) : 0.0;
        if (l < W) {
            phi[j * 2 * W + l] = fx;
            phi[j * 2 * W + W + l] = fyl;
        }
        const int col = wrapi(ox.c + l, G);
        int row = wrapi(oy.c, G);
        for (int r = 0; r < W; ++r) {
            const double fy = __shfl_sync(gmask, fyl, r, 16);
            if (l < W) atomicAdd(grid + (int64_t)row * ld + col, fx * fy);
            if (++row == G) row = 0;
        }
    }
}

// W2: on the half spectrum of the real-to-complex transform (G rows x (G/2 + 1) columns) keep
// q = m mod G for m in {-N..N-1}^2 and multiply by r(m_x) r(m_y) (adjoint window division) * c(m) *
// r(m_x) r(m_y) (forward window division); zero every other cell. The columns q_x < N hold
// m_x = q_x; m_x < 0 lies in the implicit conjugate half (q_x >= G - N > G / 2), and m_x = N
// (q_x = N) has c = 0. r has 2N entries for m = -N..N-1.
__global__ void k_w2_lag(double2* __restrict__ spec, int G, int N, const double* __restrict__ r) {
    const int H = G / 2 + 1;
    const int64_t total = (int64_t)G * H;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int qy = (int)(i / H), qx = (int)(i - (int64_t)qy * H);
        const int my = qy < N ? qy : (qy >= G - N ? qy - G : INT32_MIN);
        double2 v = spec[i];
        if (my == INT32_MIN || qx >= N) {
            v.x = 0.0;
            v.y = 0.0;
        } else {
            const int mx = qx;
            const double ry = r[my + N], rx = r[mx + N];
            const double cx = (double)(N - mx) / ((double)N * N);
            const double cy = (double)(N - (my < 0 ? -my : my)) / ((double)N * N);
            const double f = rx * rx * ry * ry * cx * cy;
            v.x *= f;
            v.y *= f;
        }
        spec[i] = v;
    }
}

// W3 + W4: S_k = sum_taps phi phi h_l at 2 lambda_k, with the window values W1 stored; alpha_k =
// 1 / S_k.
__global__ void __launch_bounds__(256)
    k_w3_interp(const double* __restrict__ lam, int64_t M, double scale, int G, int64_t ld, int W,
                const double* __restrict__ grid, const double* __restrict__ phi,
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
            const double fx = l < W ? phi[j * 2 * W + l] : 0.0;
            const double fyl = l < W ? phi[j * 2 * W + W + l] : 0.0;
            const int col = wrapi(ox.c + l, G);
            int row = wrapi(oy.c, G);
            for (int r = 0; r < W; ++r) {
                const double fy = __shfl_sync(gmask, fyl, r, 16);
                if (l < W) sr += fy * grid[(int64_t)row * ld + col];
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

namespace {

// cuFFT plans of the lag grid, one pair per (device, G), created once and shared; they own no
// workspace (each call passes its own), and their use is serialised by the mutex.
struct LagFft {
    cufftHandle d2z = 0, z2d = 0;
    size_t ws = 0;
};
std::mutex g_lag_mu;
std::map<std::pair<int, int>, LagFft> g_lag;

ftcg_status_t lag_fft_locked(int G, LagFft* out) {
    int dev = 0;
    FTCG_CK(cudaGetDevice(&dev));
    auto it = g_lag.find({dev, G});
    if (it == g_lag.end()) {
        LagFft f;
        size_t w1 = 0, w2 = 0;
        FTCG_CKFFT(cufftCreate(&f.d2z));
        FTCG_CKFFT(cufftSetAutoAllocation(f.d2z, 0));
        FTCG_CKFFT(cufftMakePlan2d(f.d2z, G, G, CUFFT_D2Z, &w1));
        FTCG_CKFFT(cufftCreate(&f.z2d));
        FTCG_CKFFT(cufftSetAutoAllocation(f.z2d, 0));
        FTCG_CKFFT(cufftMakePlan2d(f.z2d, G, G, CUFFT_Z2D, &w2));
        f.ws = std::max(w1, w2);
        it = g_lag.emplace(std::make_pair(dev, G), f).first;
    }
    *out = it->second;
    return FTCG_SUCCESS;
}

// Device buffers of one weight computation, released on every path.
struct WeightBuffers {
    double* r2 = nullptr;
    double* grid = nullptr;
    double* phi = nullptr;
    void* work = nullptr;
    PolyCoef* coef = nullptr;
    double* alpha = nullptr;
    bool own_alpha = false;
    cudaStream_t s = nullptr;            // allocated from the pool on s, freed on s
    ~WeightBuffers() {
        void* all[6] = {r2, grid, phi, work, coef, own_alpha ? alpha : nullptr};
        for (void* q : all)
            if (q) pool_free(q, s);
    }
};

// p_l interpolates phi(s + w/2 - 1 - l), s = (x + 1) / 2, at the kPolyDeg + 1 Chebyshev points
// x_i = cos(pi (i + 1/2) / n); the Chebyshev coefficients a_k = (2 - [k = 0]) / n sum_i f_i T_k(x_i)
// are converted to powers of x with T_{k+1} = 2 x T_k - T_{k-1}.
void window_poly(int W, double beta, PolyCoef* out) {
    const double pi = 3.14159265358979323846;
    const int n = kPolyDeg + 1;
    auto phi_host = [&](double t) {
        const double z = 2.0 * t / W;
        const double q = 1.0 - z * z;
        return q >= 0.0 ? std::exp(beta * (std::sqrt(q) - 1.0)) : 0.0;
    };
    for (int l = 0; l < kPolyMaxW; ++l)
        for (int k = 0; k <= kPolyDeg; ++k) out->c[l][k] = 0.0;
    for (int l = 0; l < W; ++l) {
        double f[kPolyDeg + 1], a[kPolyDeg + 1];
        for (int i = 0; i < n; ++i) {
            const double x = std::cos(pi * (i + 0.5) / n);
            f[i] = phi_host(0.5 * (x + 1.0) + 0.5 * W - 1.0 - l);
        }
        for (int k = 0; k < n; ++k) {
            double acc = 0.0;
            for (int i = 0; i < n; ++i) acc += f[i] * std::cos(pi * k * (i + 0.5) / n);
            a[k] = (k == 0 ? 1.0 : 2.0) * acc / n;
        }
        double tm[kPolyDeg + 1] = {0}, tc[kPolyDeg + 1] = {0}, tn[kPolyDeg + 1];
        tm[0] = 1.0;                                 // T_0
        tc[1] = 1.0;                                 // T_1
        out->c[l][0] += a[0];
        for (int k = 1; k < n; ++k) {
            for (int j = 0; j <= kPolyDeg; ++j) out->c[l][j] += a[k] * tc[j];
            if (k + 1 < n) {
                for (int j = 0; j <= kPolyDeg; ++j)
                    tn[j] = (j > 0 ? 2.0 * tc[j - 1] : 0.0) - tm[j];
                for (int j = 0; j <= kPolyDeg; ++j) {
                    tm[j] = tc[j];
                    tc[j] = tn[j];
                }
            }
        }
    }
}

}  // namespace

ftcg_status_t compute_weights(Plan& p, double* d_alpha_out, cudaStream_t s) {
    if (p.M == 0) return FTCG_SUCCESS;
    const int Wa = p.opts.weight_width > 0 ? p.opts.weight_width : 12;
    const int N2 = 2 * p.N;
    const int G2 = 2 * p.G;                      // sigma * (2N)
    const int64_t ld = G2 + 2;                   // real row stride of the in-place transforms
    const double scale = 2.0 * p.sigma;          // u = sigma * (2 lambda)
    Window wa{Wa, es_beta(Wa, p.sigma)};

    std::lock_guard<std::mutex> lk(g_lag_mu);
    LagFft fft;
    FTCG_TRY(lag_fft_locked(G2, &fft));
    WeightBuffers b;
    const size_t gbytes = (size_t)G2 * ld * sizeof(double);
    const size_t pbytes = (size_t)p.M * 2 * Wa * sizeof(double);
    b.s = s;
    if (pool_malloc(&b.r2, N2 * sizeof(double), s) != cudaSuccess ||
        pool_malloc(&b.grid, gbytes, s) != cudaSuccess || pool_malloc(&b.phi, pbytes, s) != cudaSuccess ||
        pool_malloc(&b.coef, sizeof(PolyCoef), s) != cudaSuccess ||
        (fft.ws > 0 && pool_malloc(&b.work, fft.ws, s) != cudaSuccess)) {
        cudaGetLastError();
        set_error("ftcg_weights: cannot allocate the FP64 lag grid (%zu bytes), the window table "
                  "(%zu bytes) or the FFT workspace (%zu bytes)", gbytes, pbytes, fft.ws);
        return FTCG_ERR_OUT_OF_MEMORY;
    }
    b.alpha = d_alpha_out;
    if (!b.alpha) {
        if (pool_malloc(&b.alpha, p.M * sizeof(double), s) != cudaSuccess) {
            cudaGetLastError();
            set_error("ftcg_weights: cannot allocate the weight array");
            return FTCG_ERR_OUT_OF_MEMORY;
        }
        b.own_alpha = true;
    }
    PolyCoef hc;
    window_poly(Wa, wa.beta, &hc);
    FTCG_CK(cudaMemcpyAsync(b.coef, &hc, sizeof(PolyCoef), cudaMemcpyHostToDevice, s));
    FTCG_TRY(window_factors(b.r2, N2, G2, wa, s));
    FTCG_CK(cudaMemsetAsync(b.grid, 0, gbytes, s));
    k_w1_spread<<<nblocks(p.M * 16, 256), 256, 0, s>>>(p.lambda, p.M, scale, G2, ld, Wa, b.coef,
                                                        b.grid, b.phi);
    FTCG_CK(cudaGetLastError());
    cufftDoubleComplex* spec = reinterpret_cast<cufftDoubleComplex*>(b.grid);
    FTCG_CKFFT(cufftSetStream(fft.d2z, s));
    FTCG_CKFFT(cufftSetWorkArea(fft.d2z, b.work));
    FTCG_CKFFT(cufftExecD2Z(fft.d2z, b.grid, spec));
    k_w2_lag<<<nblocks((int64_t)G2 * (G2 / 2 + 1), 256), 256, 0, s>>>(
        reinterpret_cast<double2*>(b.grid), G2, p.N, b.r2);
    FTCG_CK(cudaGetLastError());
    FTCG_CKFFT(cufftSetStream(fft.z2d, s));
    FTCG_CKFFT(cufftSetWorkArea(fft.z2d, b.work));
    FTCG_CKFFT(cufftExecZ2D(fft.z2d, spec, b.grid));
    unsigned before = 0;
    FTCG_CK(cudaMemcpyAsync(&before, p.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    k_w3_interp<<<nblocks(p.M * 16, 256), 256, 0, s>>>(p.lambda, p.M, scale, G2, ld, Wa, b.grid,
                                                        b.phi, b.alpha, p.status);
    FTCG_CK(cudaGetLastError());
    FTCG_TRY(launch_set_alpha(p, b.alpha, FTCG_WEIGHTS_F64, s));
    unsigned after = 0;
    FTCG_CK(cudaMemcpyAsync(&after, p.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    FTCG_CK(cudaStreamSynchronize(s));            // the buffers are freed on return
    if ((after & STATUS_BAD_WEIGHT_SUM) && !(before & STATUS_BAD_WEIGHT_SUM)) {
        set_error("ftcg_weights: a weight sum S_k was <= 0 or not finite (weight set to 0)");
        return FTCG_ERR_NUMERIC;
    }
    return FTCG_SUCCESS;
}

}  // namespace ftcg
