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
// window factors are real and even); the result of W3's transform is then real. The forward
// transform (exponent sign -, which gives conj(H) for a real grid) is taken column-first: real-to-
// complex along y, keeping the half spectrum m_y >= 0, then complex along x; the inverse (sign +)
// is complex along x, then complex-to-real along y: conj(sum_m H(m) c(m) e^{-...}) = the real S
// grid. Both are pruned to what the method uses: the y transforms run only over the column blocks
// that some footprint reaches (W3 reads nothing else; a polar wedge reaches about half of them),
// and the x transforms only over the N rows m_y = 0..N-1 where c is non-zero. W1 stores each
// sample's 2 w window values and its tap origins so that W3 reads them instead of evaluating
// them again.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <utility>

#include "ftcg_internal.cuh"

namespace ftcg {

namespace {

// The window on the weight path, in FP64, as two polynomials per tap: the first-tap offset d lies
// in (w/2 - 1, w/2], so tap l's argument d - l covers one unit interval; with s = d - (w/2 - 1) in
// (0, 1] and x = 2 s - 1, phi(d - l) = p_{l,h}(2 x + 1 - 2 h) on the half h = [x >= 0] of the
// interval. Each p_{l,h} has degree kPolyDeg and interpolates phi at the Chebyshev points of its
// half interval (coefficients from window_poly on the host); halving the interval brings degree
// 9 to the accuracy that degree 14 gives on the whole interval. The end intervals hold the
// window's square-root branch point, where phi = exp(-beta); the interpolation error there is
// about exp(-beta) / 2 of phi(0) (6e-13 at w = 12, sigma = 2; 1.2e-10 at w = 12, sigma = 1.25)
// and far smaller inside, i.e. at the level of the window's own truncation.
constexpr int kPolyDeg = 9;
constexpr int kPolyMaxW = 16;

struct PolyCoef {
    double c[kPolyMaxW][2][kPolyDeg + 1];   // c[l][h][k]: coefficient of y^k in p_{l,h}
};

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

// W1: g_l += phi(u_x - l_x) phi(u_y - l_y) (real, unit strengths). The FP64 pipe bounds this
// kernel, so every FP64 instruction is given 32 useful lanes. A warp takes 32 samples at a time:
// lane i first computes sample i's tap origins and polynomial arguments (the origins are stored
// for W3); then groups of 8 lanes take the samples four at a time. For one sample, the group's
// lanes evaluate its 2 w tap polynomials (polynomial p is x-tap p for p < w and y-tap p - w
// otherwise; lane l takes p = l, l + 8, ...), store the values in the sample's row of phi and in
// shared memory, and add the w^2 products of the row-major footprint (tap t = l, l + 8, ...)
// with FP64 global atomics to the real grid (row stride ld).
constexpr int kW1Threads = 256;

__global__ void __launch_bounds__(kW1Threads)
    k_w1_spread(const double* __restrict__ lam, int64_t M, double scale, int G, int64_t ld, int W,
                const PolyCoef* __restrict__ pc, double* __restrict__ grid,
                double* __restrict__ phi, int2* __restrict__ org) {
    __shared__ double s_c[kPolyMaxW][2][kPolyDeg + 1];
    __shared__ double s_v[kW1Threads / 8][2 * kPolyMaxW];   // per group: its sample's values
    for (int i = threadIdx.x; i < kPolyMaxW * 2 * (kPolyDeg + 1); i += kW1Threads)
        (&s_c[0][0][0])[i] = (&pc->c[0][0][0])[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, l = lane & 7, gi = lane >> 3;
    const unsigned gmask = 0xffu << (lane & 24);
    double* v = s_v[threadIdx.x >> 3];
    const double s0 = 0.5 * W - 1.0;
    const int np = 2 * W, nt = W * W;
    const int r0 = l / W, c0 = l - r0 * W;               // this lane's first footprint tap
    const int64_t step = (int64_t)gridDim.x * kW1Threads;
    for (int64_t base = ((int64_t)blockIdx.x * kW1Threads + (threadIdx.x & ~31)); base < M;
         base += step) {
        const int64_t ji = base + lane;
        double ax = 0.0, ay = 0.0;
        int cx = 0, cy = 0, ok = 0;
        if (ji < M) {
            const Origin64 ox = origin64(lam[2 * ji], scale, W);
            const Origin64 oy = origin64(lam[2 * ji + 1], scale, W);
            ok = ox.ok && oy.ok;
            if (ok) {
                cx = wrapi(ox.c, G);
                cy = wrapi(oy.c, G);
                ax = 2.0 * (ox.d - s0) - 1.0;
                ay = 2.0 * (oy.d - s0) - 1.0;
            }
            org[ji] = ok ? make_int2(cx, cy) : make_int2(-1, -1);
        }
        const int nb = (int)(M - base < 32 ? M - base : 32);
        for (int q = 0; q < 8; ++q) {                     // samples 4 q + gi of the block
            const int src = 4 * q + gi;
            const double sx = __shfl_sync(0xffffffffu, ax, src);
            const double sy = __shfl_sync(0xffffffffu, ay, src);
            const int scx = __shfl_sync(0xffffffffu, cx, src);
            const int scy = __shfl_sync(0xffffffffu, cy, src);
            const int sok = __shfl_sync(0xffffffffu, ok, src);
            if (src >= nb || !sok) continue;               // uniform within the group
            const int64_t j = base + src;
            for (int p = l; p < np; p += 8) {
                const int tap = p < W ? p : p - W;
                const double x = p < W ? sx : sy;
                const int h = x >= 0.0 ? 1 : 0;
                const double y = fma(2.0, x, h ? -1.0 : 1.0);
                const double* cf = s_c[tap][h];
                double acc = cf[kPolyDeg];
#pragma unroll
                for (int k = kPolyDeg - 1; k >= 0; --k) acc = fma(acc, y, cf[k]);
                v[p] = acc;
                phi[j * np + p] = acc;
            }
            __syncwarp(gmask);
            int r = r0, c = c0;
            for (int t = l; t < nt; t += 8) {
                int row = scy + r, col = scx + c;
                if (row >= G) row -= G;
                if (col >= G) col -= G;
                atomicAdd(grid + (int64_t)row * ld + col, v[c] * v[W + r]);
                c += 8;
                while (c >= W) {
                    c -= W;
                    ++r;
                }
            }
            __syncwarp(gmask);
        }
    }
}

// W2 on the column-first half spectrum B[q_y][q_x] (q_y in 0..G/2 along the rows of B, q_x in
// 0..G-1, row width G): the first N rows hold m_y = q_y in 0..N-1; in them q_x < N holds
// m_x = q_x and q_x >= G - N holds m_x = q_x - G. Those cells are multiplied by r(m_x) r(m_y)
// (adjoint window division) * c(m) * r(m_x) r(m_y) (forward window division); every other cell of
// the first N rows is zeroed (rows N..G/2, m_y >= N where c = 0, are zeroed by the caller). r has
// 2N entries for m = -N..N-1.
__global__ void k_w2_lag(double2* __restrict__ B, int G, int N, const double* __restrict__ r) {
    const int64_t total = (int64_t)N * G;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int my = (int)(i / G), qx = (int)(i - (int64_t)my * G);
        const int mx = qx < N ? qx : (qx >= G - N ? qx - G : INT32_MIN);
        double2 v = B[i];
        if (mx == INT32_MIN) {
            v.x = 0.0;
            v.y = 0.0;
        } else {
            const double ry = r[my + N], rx = r[mx + N];
            const double cx = (double)(N - (mx < 0 ? -mx : mx)) / ((double)N * N);
            const double cy = (double)(N - my) / ((double)N * N);
            const double f = rx * rx * ry * ry * cx * cy;
            v.x *= f;
            v.y *= f;
        }
        B[i] = v;
    }
}

// The grid columns that some sample's footprint reaches (W3 reads only those): occ[x] = 1.
__global__ void k_mark_cols(const int2* __restrict__ org, int64_t M, int G, int W,
                            unsigned char* __restrict__ occ) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M * W;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / W;
        const int t = (int)(i - j * W);
        const int x0 = org[j].x;
        if (x0 < 0) continue;
        int x = x0 + t;
        if (x >= G) x -= G;
        occ[x] = 1;
    }
}

// W3 + W4: S_k = sum_taps phi phi h_l at 2 lambda_k from the origins and window values W1
// stored; alpha_k = 1 / S_k. Four lanes per sample (eight samples per warp, so every FP64
// instruction has 32 useful lanes): lane q sums the columns q, q + 4, ... of the footprint over
// all w rows, weights them with the column factors, and the four partial sums are added.
__global__ void __launch_bounds__(256)
    k_w3_interp(const int2* __restrict__ org, int64_t M, int G, int64_t ld, int W,
                const double* __restrict__ grid, const double* __restrict__ phi,
                double* __restrict__ alpha, unsigned* __restrict__ status) {
    const int q = threadIdx.x & 3;
    const unsigned qmask = 0xfu << ((threadIdx.x & 31) & ~3);
    const int64_t ngr = (int64_t)gridDim.x * (blockDim.x / 4);
    for (int64_t j = blockIdx.x * (int64_t)(blockDim.x / 4) + threadIdx.x / 4; j < M; j += ngr) {
        const int2 o = org[j];
        const bool ok = o.x >= 0;                             // uniform within the group
        double sr = 0.0;
        if (ok) {
            const double* ph = phi + j * 2 * W;
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            int col[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                col[c] = o.x + q + 4 * c;
                if (col[c] >= G) col[c] -= G;
            }
            int row = o.y;
            for (int r = 0; r < W; ++r) {
                const double fy = ph[W + r];
                const double* g = grid + (int64_t)row * ld;
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (q + 4 * c < W) acc[c] = fma(fy, g[col[c]], acc[c]);
                if (++row == G) row = 0;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (q + 4 * c < W) sr = fma(ph[q + 4 * c], acc[c], sr);
        }
        sr += __shfl_xor_sync(qmask, sr, 1, 4);
        sr += __shfl_xor_sync(qmask, sr, 2, 4);
        if (q == 0) {
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

// cuFFT plans of the lag transforms, created on first use and shared; they own no workspace
// (each call passes its own) and their use is serialised by the mutex. Per device and grid side
// G: column transforms along y of a batch of adjacent columns (D2Z from the real grid, row stride
// G + 2, into B, row width G; Z2D back), batches being runs of kLagColBlock-column blocks, and
// row transforms along x of the first N rows of B (Z2Z).
constexpr int kLagColBlock = 128;
enum LagKind { LAG_D2Z_Y = 0, LAG_Z2D_Y = 1, LAG_Z2Z_X = 2 };
struct LagKey {
    int dev, G, kind, batch;
    bool operator<(const LagKey& o) const {
        if (dev != o.dev) return dev < o.dev;
        if (G != o.G) return G < o.G;
        if (kind != o.kind) return kind < o.kind;
        return batch < o.batch;
    }
};
struct LagPlan {
    cufftHandle h = 0;
    size_t ws = 0;
};
std::mutex g_lag_mu;
std::map<LagKey, LagPlan> g_lag;

ftcg_status_t lag_plan_locked(int dev, int G, int kind, int batch, LagPlan* out) {
    const LagKey key{dev, G, kind, batch};
    auto it = g_lag.find(key);
    if (it == g_lag.end()) {
        LagPlan pl;
        int n[1] = {G};
        const int ld = G + 2, H = G / 2 + 1;
        int inembed[1] = {G}, onembed[1] = {G};
        FTCG_CKFFT(cufftCreate(&pl.h));
        FTCG_CKFFT(cufftSetAutoAllocation(pl.h, 0));
        cufftResult r;
        if (kind == LAG_D2Z_Y) {
            onembed[0] = H;
            r = cufftMakePlanMany(pl.h, 1, n, inembed, ld, 1, onembed, G, 1, CUFFT_D2Z, batch,
                                  &pl.ws);
        } else if (kind == LAG_Z2D_Y) {
            inembed[0] = H;
            r = cufftMakePlanMany(pl.h, 1, n, inembed, G, 1, onembed, ld, 1, CUFFT_Z2D, batch,
                                  &pl.ws);
        } else {
            r = cufftMakePlanMany(pl.h, 1, n, inembed, 1, G, onembed, 1, G, CUFFT_Z2Z, batch,
                                  &pl.ws);
        }
        if (r != CUFFT_SUCCESS) {
            cufftDestroy(pl.h);
            set_error("cuFFT plan of the lag transforms failed (%d)", (int)r);
            return FTCG_ERR_CUDA;
        }
        it = g_lag.emplace(key, pl).first;
    }
    *out = it->second;
    return FTCG_SUCCESS;
}

// Runs [x0, x0 + n) of kLagColBlock-column blocks (the last block may be shorter) holding an
// occupied column.
std::vector<std::pair<int, int>> lag_runs(const std::vector<unsigned char>& occ, int G) {
    std::vector<std::pair<int, int>> runs;
    const int nblk = (G + kLagColBlock - 1) / kLagColBlock;
    int start = -1;
    for (int b = 0; b <= nblk; ++b) {
        bool any = false;
        if (b < nblk)
            for (int x = b * kLagColBlock; x < std::min(G, (b + 1) * kLagColBlock) && !any; ++x)
                any = occ[x] != 0;
        if (any && start < 0) start = b;
        if (!any && start >= 0) {
            const int x0 = start * kLagColBlock;
            runs.push_back({x0, std::min(G, b * kLagColBlock) - x0});
            start = -1;
        }
    }
    return runs;
}

// Device buffers of one weight computation, released on every path.
struct WeightBuffers {
    double* r2 = nullptr;
    double* grid = nullptr;
    double2* spec = nullptr;
    double* phi = nullptr;
    int2* org = nullptr;
    unsigned char* occ = nullptr;
    void* work = nullptr;
    PolyCoef* coef = nullptr;
    double* alpha = nullptr;
    bool own_alpha = false;
    cudaStream_t s = nullptr;            // allocated from the pool on s, freed on s
    ~WeightBuffers() {
        void* all[9] = {r2, grid, spec, phi, org, occ, work, coef, own_alpha ? alpha : nullptr};
        for (void* q : all)
            if (q) pool_free(q, s);
    }
};

// p_{l,h} interpolates phi(s + w/2 - 1 - l), s = (x + 1) / 2, x = (y - 1) / 2 + h, at the
// kPolyDeg + 1 Chebyshev points y_i = cos(pi (i + 1/2) / n); the Chebyshev coefficients
// a_k = (2 - [k = 0]) / n sum_i f_i T_k(y_i) are converted to powers of y with
// T_{k+1} = 2 y T_k - T_{k-1}.
void window_poly(int W, double beta, PolyCoef* out) {
    const double pi = 3.14159265358979323846;
    const int n = kPolyDeg + 1;
    auto phi_host = [&](double t) {
        const double z = 2.0 * t / W;
        const double q = 1.0 - z * z;
        return q >= 0.0 ? std::exp(beta * (std::sqrt(q) - 1.0)) : 0.0;
    };
    for (int l = 0; l < kPolyMaxW; ++l)
        for (int h = 0; h < 2; ++h)
            for (int k = 0; k <= kPolyDeg; ++k) out->c[l][h][k] = 0.0;
    for (int l = 0; l < W; ++l) {
        for (int h = 0; h < 2; ++h) {
            double f[kPolyDeg + 1], a[kPolyDeg + 1];
            for (int i = 0; i < n; ++i) {
                const double y = std::cos(pi * (i + 0.5) / n);
                const double x = 0.5 * (y - 1.0) + h;
                f[i] = phi_host(0.5 * (x + 1.0) + 0.5 * W - 1.0 - l);
            }
            for (int k = 0; k < n; ++k) {
                double acc = 0.0;
                for (int i = 0; i < n; ++i) acc += f[i] * std::cos(pi * k * (i + 0.5) / n);
                a[k] = (k == 0 ? 1.0 : 2.0) * acc / n;
            }
            double* c = out->c[l][h];
            double tm[kPolyDeg + 1] = {0}, tc[kPolyDeg + 1] = {0}, tn[kPolyDeg + 1];
            tm[0] = 1.0;                                 // T_0
            tc[1] = 1.0;                                 // T_1
            c[0] += a[0];
            for (int k = 1; k < n; ++k) {
                for (int j = 0; j <= kPolyDeg; ++j) c[j] += a[k] * tc[j];
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
}

}  // namespace

ftcg_status_t compute_weights(Plan& p, double* d_alpha_out, cudaStream_t s) {
    if (p.M == 0) return FTCG_SUCCESS;
    const int Wa = p.opts.weight_width > 0 ? p.opts.weight_width : 12;
    const int N2 = 2 * p.N;
    const int G2 = 2 * p.G;                      // sigma * (2N)
    const int64_t ld = G2 + 2;                   // row stride of the real lag grid
    const int H = G2 / 2 + 1;                    // rows of the column-first half spectrum
    const double scale = 2.0 * p.sigma;          // u = sigma * (2 lambda)
    Window wa{Wa, es_beta(Wa, p.sigma)};

    std::lock_guard<std::mutex> lk(g_lag_mu);
    int dev = 0;
    FTCG_CK(cudaGetDevice(&dev));
    WeightBuffers b;
    const size_t gbytes = (size_t)G2 * ld * sizeof(double);
    const size_t sbytes = (size_t)H * G2 * sizeof(double2);
    const size_t pbytes = (size_t)p.M * 2 * Wa * sizeof(double);
    b.s = s;
    if (pool_malloc(&b.r2, N2 * sizeof(double), s) != cudaSuccess ||
        pool_malloc(&b.grid, gbytes, s) != cudaSuccess ||
        pool_malloc(&b.spec, sbytes, s) != cudaSuccess ||
        pool_malloc(&b.phi, pbytes, s) != cudaSuccess ||
        pool_malloc(&b.org, (size_t)p.M * sizeof(int2), s) != cudaSuccess ||
        pool_malloc(&b.occ, (size_t)G2, s) != cudaSuccess ||
        pool_malloc(&b.coef, sizeof(PolyCoef), s) != cudaSuccess) {
        cudaGetLastError();
        set_error("ftcg_weights: cannot allocate the FP64 lag grid (%zu bytes), its spectrum "
                  "(%zu bytes), the window table (%zu bytes) or the tap origins", gbytes, sbytes,
                  pbytes);
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
    FTCG_CK(cudaMemsetAsync(b.occ, 0, (size_t)G2, s));
    k_w1_spread<<<nblocks(p.M, kW1Threads), kW1Threads, 0, s>>>(p.lambda, p.M, scale, G2, ld, Wa,
                                                                b.coef, b.grid, b.phi, b.org);
    k_mark_cols<<<nblocks(p.M * Wa, 256), 256, 0, s>>>(b.org, p.M, G2, Wa, b.occ);
    FTCG_CK(cudaGetLastError());
    // The lag transforms, column-first and pruned: along y only over the column blocks that
    // footprints reach (W3 reads nothing else), keeping the half spectrum m_y >= 0; along x only
    // over the N rows m_y = 0..N-1 that the lag weights keep.
    std::vector<unsigned char> occ((size_t)G2);
    FTCG_CK(cudaMemcpyAsync(occ.data(), b.occ, (size_t)G2, cudaMemcpyDeviceToHost, s));
    FTCG_CK(cudaStreamSynchronize(s));
    const std::vector<std::pair<int, int>> runs = lag_runs(occ, G2);
    std::vector<LagPlan> fwd(runs.size()), inv(runs.size());
    LagPlan rows;
    size_t ws = 0;
    for (size_t k = 0; k < runs.size(); ++k) {
        FTCG_TRY(lag_plan_locked(dev, G2, LAG_D2Z_Y, runs[k].second, &fwd[k]));
        FTCG_TRY(lag_plan_locked(dev, G2, LAG_Z2D_Y, runs[k].second, &inv[k]));
        ws = std::max(ws, std::max(fwd[k].ws, inv[k].ws));
    }
    FTCG_TRY(lag_plan_locked(dev, G2, LAG_Z2Z_X, p.N, &rows));
    ws = std::max(ws, rows.ws);
    if (ws > 0 && pool_malloc(&b.work, ws, s) != cudaSuccess) {
        cudaGetLastError();
        set_error("ftcg_weights: cannot allocate the FFT workspace (%zu bytes)", ws);
        return FTCG_ERR_OUT_OF_MEMORY;
    }
    cufftDoubleComplex* spec = reinterpret_cast<cufftDoubleComplex*>(b.spec);
    FTCG_CK(cudaMemsetAsync(b.spec, 0, (size_t)p.N * G2 * sizeof(double2), s));
    for (size_t k = 0; k < runs.size(); ++k) {
        FTCG_CKFFT(cufftSetStream(fwd[k].h, s));
        FTCG_CKFFT(cufftSetWorkArea(fwd[k].h, b.work));
        FTCG_CKFFT(cufftExecD2Z(fwd[k].h, b.grid + runs[k].first, spec + runs[k].first));
    }
    // rows N..G/2 (m_y >= N, lag weight 0) are zero for the inverse
    FTCG_CK(cudaMemsetAsync(b.spec + (size_t)p.N * G2, 0,
                            (size_t)(H - p.N) * G2 * sizeof(double2), s));
    FTCG_CKFFT(cufftSetStream(rows.h, s));
    FTCG_CKFFT(cufftSetWorkArea(rows.h, b.work));
    FTCG_CKFFT(cufftExecZ2Z(rows.h, spec, spec, CUFFT_FORWARD));
    k_w2_lag<<<nblocks((int64_t)p.N * G2, 256), 256, 0, s>>>(b.spec, G2, p.N, b.r2);
    FTCG_CK(cudaGetLastError());
    FTCG_CKFFT(cufftExecZ2Z(rows.h, spec, spec, CUFFT_INVERSE));
    for (size_t k = 0; k < runs.size(); ++k) {
        FTCG_CKFFT(cufftSetStream(inv[k].h, s));
        FTCG_CKFFT(cufftSetWorkArea(inv[k].h, b.work));
        FTCG_CKFFT(cufftExecZ2D(inv[k].h, spec + runs[k].first, b.grid + runs[k].first));
    }
    unsigned before = 0;
    FTCG_CK(cudaMemcpyAsync(&before, p.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    k_w3_interp<<<nblocks(p.M * 4, 256), 256, 0, s>>>(b.org, p.M, G2, ld, Wa, b.grid, b.phi,
                                                       b.alpha, p.status);
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
