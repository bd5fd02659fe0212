// The window and its Fourier transform, in FP64 on the device.
//
// Division by the window (zeta_n = psi_n / w(x), Eq. newadm) becomes, on the sigma-oversampled
// grid, division by phi^(p / G) (the m = 0 term of the Poisson sum of Eq. twodcg):
//     phi^(xi) = int phi(t) exp(-2 pi i xi t) dt = 2 int_0^{pi/2} phi(w/2 sin th) cos(pi w xi sin th)
//                (w/2) cos th dth,
// the substitution t = (w/2) sin th removing the square-root edge of the ES and Kaiser-Bessel
// windows (the truncated Gaussian is smooth inside its support). The integral
// is taken by Gauss-Legendre quadrature whose nodes are computed here by Newton iteration on the
// Legendre polynomial P_n (three-term recurrence), then the N reciprocals are evaluated in FP64.

#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "ftcg_internal.cuh"

namespace ftcg {

namespace {

constexpr int kQuadNodes = 96;

// Gauss-Legendre nodes and weights on [-1, 1].
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& wt) {
    x.resize(n);
    wt.resize(n);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            // p1 = P_n(z), p0 = P_{n-1}(z)
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        wt[i] = wt[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

struct Quad {
    double th[kQuadNodes];   // angles in [0, pi/2]
    double wt[kQuadNodes];   // weights including the dth Jacobian
};

__global__ void k_window_factors(double* __restrict__ out, int N, int G, int W, double beta,
                                 int kind, Quad q) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double pi = 3.14159265358979323846;
    double xi = (double)(i - N / 2) / (double)G;
    double half = 0.5 * W;
    double s = 0.0;
    for (int k = 0; k < kQuadNodes; ++k) {
        double sn, cs;
        sincos(q.th[k], &sn, &cs);
        // the window at t = (w/2) sin th, where sqrt(1 - (2t/w)^2) = cos th
        double ph;
        if (kind == FTCG_WINDOW_KB) ph = cyl_bessel_i0(beta * cs) / cyl_bessel_i0(beta);
        else if (kind == FTCG_WINDOW_GAUSS) ph = exp(-beta * sn * sn);
        else ph = exp(beta * (cs - 1.0));
        s += q.wt[k] * ph * cos(2.0 * pi * xi * half * sn) * half * cs;
    }
    out[i] = 1.0 / (2.0 * s);
}

}  // namespace

double es_beta(int w, double sigma) {
    const double pi = 3.14159265358979323846;
    return 0.97 * pi * (1.0 - 0.5 / sigma) * w;
}

// Shape parameter of each window family for width w and oversampling sigma: ES as es_beta
// (Barnett, Magland, af Klinteberg 2019); Kaiser-Bessel beta = pi sqrt((w/sigma)^2 (sigma - 1/2)^2
// - 0.8) (Beatty, Nishimura, Pauly 2005; NaN where the root is not real); truncated Gaussian
// exp(-beta z^2) with beta = (pi w / 2) (1 - 1/(2 sigma)).
double kernel_beta(int w, double sigma, int kind) {
    const double pi = 3.14159265358979323846;
    if (kind == FTCG_WINDOW_KB) {
        const double a = (w / sigma) * (w / sigma) * (sigma - 0.5) * (sigma - 0.5) - 0.8;
        return a > 0.0 ? pi * std::sqrt(a) : std::nan("");
    }
    if (kind == FTCG_WINDOW_GAUSS) return 0.5 * pi * w * (1.0 - 0.5 / sigma);
    return es_beta(w, sigma);
}

Win32 win32_of(const Window& win) {
    Win32 r;
    r.beta = (float)win.beta;
    r.inv_hw = (float)(2.0 / win.w);
    r.norm = win.kind == FTCG_WINDOW_KB ? (float)(1.0 / std::cyl_bessel_i(0.0, win.beta)) : 1.0f;
    r.kind = win.kind;
    return r;
}

double window64(double t, int w, double beta, int kind) {
    const double z = 2.0 * t / w;
    if (std::fabs(z) > 1.0) return 0.0;
    if (kind == FTCG_WINDOW_KB) return std::cyl_bessel_i(0.0, beta * std::sqrt(1.0 - z * z)) /
                                       std::cyl_bessel_i(0.0, beta);
    if (kind == FTCG_WINDOW_GAUSS) return std::exp(-beta * z * z);
    return std::exp(beta * (std::sqrt(1.0 - z * z) - 1.0));
}

namespace {

// Factors already computed, per (device, N, G, w, beta): plans of the same shape (ping after
// ping) copy them instead of repeating the FP64 quadrature. Held until the process exits.
struct FactorKey {
    int dev, N, G, w, kind;
    uint64_t beta_bits;
    bool operator<(const FactorKey& o) const {
        if (dev != o.dev) return dev < o.dev;
        if (N != o.N) return N < o.N;
        if (G != o.G) return G < o.G;
        if (w != o.w) return w < o.w;
        if (kind != o.kind) return kind < o.kind;
        return beta_bits < o.beta_bits;
    }
};
std::mutex g_factor_mu;
std::map<FactorKey, double*> g_factors;

}  // namespace

ftcg_status_t window_factors(double* d_out, int N, int G, const Window& win, cudaStream_t s) {
    if (N <= 0) return FTCG_SUCCESS;
    FactorKey key{0, N, G, win.w, win.kind, 0};
    FTCG_CK(cudaGetDevice(&key.dev));
    std::memcpy(&key.beta_bits, &win.beta, sizeof(double));
    std::lock_guard<std::mutex> lk(g_factor_mu);
    auto it = g_factors.find(key);
    if (it == g_factors.end()) {
        std::vector<double> x, wt;
        gauss_legendre(kQuadNodes, x, wt);
        Quad q;
        const double pi = 3.14159265358979323846;
        for (int k = 0; k < kQuadNodes; ++k) {
            q.th[k] = 0.25 * pi * (x[k] + 1.0);
            q.wt[k] = 0.25 * pi * wt[k];
        }
        double* d = nullptr;
        FTCG_CK(cudaMalloc(&d, (size_t)N * sizeof(double)));
        k_window_factors<<<(N + 127) / 128, 128, 0, s>>>(d, N, G, win.w, win.beta, win.kind, q);
        FTCG_CK(cudaGetLastError());
        FTCG_CK(cudaStreamSynchronize(s));       // complete before another stream reads it
        it = g_factors.emplace(key, d).first;
    }
    FTCG_CK(cudaMemcpyAsync(d_out, it->second, (size_t)N * sizeof(double),
                            cudaMemcpyDeviceToDevice, s));
    return FTCG_SUCCESS;
}

__global__ void k_split_factors(const double* __restrict__ r, float2* __restrict__ r2, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float hi = __double2float_rn(r[i]);
    r2[i] = make_float2(hi, __double2float_rn(r[i] - (double)hi));
}

ftcg_status_t split_factors(const double* r, float2* r2, int n, cudaStream_t s) {
    if (n == 0) return FTCG_SUCCESS;
    k_split_factors<<<(n + 127) / 128, 128, 0, s>>>(r, r2, n);
    FTCG_CK(cudaGetLastError());
    return FTCG_SUCCESS;
}

}  // namespace ftcg
