// Spreading (Omega_2 D_2 f^, Eq. twodcgmatrix), deapodisation + crop (division by the window,
// Eq. newadm, and the restriction to p in {-N/2..N/2-1}^2), the gridded forward transform and the
// installation of per-sample weights.
//
// Spreading: one CTA owns one T x T tile of the periodic G x G grid and accumulates it in shared
// memory. It reads the tile's sorted entries (every (tile, sample) pair whose w x w footprint
// touches the tile, built by plan.cu), splits them into equal contiguous chunks, one per group of
// GW lanes (GW = 4, 8 or 16 >= w), and for each entry the group's lane l handles tap column l: it
// evaluates phi(dx - l) and phi(dy - l) in FP32, broadcasts the w row factors with shuffles, and
// adds c phi(dx - l) phi(dy - r) to the cells it owns with shared-memory atomics (taps outside
// the tile are another tile's). The tile is then stored once, coalesced, so every grid cell is
// written exactly once and no zero-fill or global atomics are needed.

#include "ftcg_internal.cuh"

namespace ftcg {

namespace {

constexpr int kSpreadThreads = 256;

__device__ __forceinline__ float es32(float t, float inv_hw, float beta) {
    float z = t * inv_hw;
    float q = fmaf(-z, z, 1.0f);
    return q >= 0.0f ? __expf(beta * (sqrtf(q) - 1.0f)) : 0.0f;
}

__device__ __forceinline__ float bf16_bits_to_float(uint32_t bits) {
    return __uint_as_float((bits & 0xffffu) << 16);
}

template <bool VBF>
__device__ __forceinline__ float2 load_value(const void* __restrict__ vals, uint32_t j) {
    if (VBF) {
        __nv_bfloat162 b = reinterpret_cast<const __nv_bfloat162*>(vals)[j];
        return __bfloat1622float2(b);
    } else {
        return reinterpret_cast<const float2*>(vals)[j];
    }
}

// GW: lanes per entry (power of two >= w); WT: compile-time w (0 = runtime w <= GW).
template <int GW, int WT, int T, bool VBF, bool ABF>
__global__ void __launch_bounds__(kSpreadThreads)
    k_spread(const Entry* __restrict__ ent, const int* __restrict__ colptr,
             const void* __restrict__ vals, float2* __restrict__ grid, int G, int ntx, int Wrt,
             float beta, float inv_hw) {
    constexpr int LD = T + 1;
    constexpr int NG = kSpreadThreads / GW;
    const int W = WT > 0 ? WT : Wrt;
    const int ncb = T + W - 1;
    extern __shared__ float smem[];
    float* s_re = smem;
    float* s_im = smem + T * LD;
    int* s_col = reinterpret_cast<int*>(smem + 2 * T * LD);

    const int tile = blockIdx.x;
    const int tyi = tile / ntx, txi = tile - tyi * ntx;
    const int X0 = txi * T, Y0 = tyi * T;
    const int Tw = min(T, G - X0), Th = min(T, G - Y0);

    for (int i = threadIdx.x; i < 2 * T * LD; i += kSpreadThreads) smem[i] = 0.0f;
    for (int i = threadIdx.x; i <= ncb; i += kSpreadThreads) s_col[i] = colptr[(int64_t)tile * ncb + i];
    __syncthreads();

    const int e0 = s_col[0], e1 = s_col[ncb];
    const int n = e1 - e0;
    const int g = threadIdx.x / GW, l = threadIdx.x % GW;
    const unsigned gmask = (GW == 32 ? 0xffffffffu : ((1u << GW) - 1u)) << ((threadIdx.x & 31) & ~(GW - 1));
    const int per = (n + NG - 1) / NG;
    const int a = e0 + g * per;
    const int b = min(e1, a + per);

    for (int base = a; base < b; base += GW) {
        const int idx = base + l;
        float dx = 0.f, dy = 0.f, cre = 0.f, cim = 0.f;
        int cxl = 0, cyl = 0;
        if (idx < b) {
            Entry e = ent[idx];
            const uint32_t j = e.packed & kSampleMask;
            cyl = (int)(e.packed >> kSampleBits) - (W - 1);
            int lo = 0, hi = ncb - 1;             // column bin: last k with s_col[k] <= idx
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (s_col[mid] <= idx) lo = mid; else hi = mid - 1;
            }
            cxl = lo - (W - 1);
            const float al = ABF ? bf16_bits_to_float(e.alpha) : __uint_as_float(e.alpha);
            const float2 v = load_value<VBF>(vals, j);
            cre = al * v.x;
            cim = al * v.y;
            dx = e.dx;
            dy = e.dy;
        }
        const int cnt = min(GW, b - base);
        for (int k = 0; k < cnt; ++k) {
            const float kdx = __shfl_sync(gmask, dx, k, GW);
            const float kdy = __shfl_sync(gmask, dy, k, GW);
            const float kre = __shfl_sync(gmask, cre, k, GW);
            const float kim = __shfl_sync(gmask, cim, k, GW);
            const int kcx = __shfl_sync(gmask, cxl, k, GW);
            const int kcy = __shfl_sync(gmask, cyl, k, GW);
            const bool lane_tap = l < W;
            const float fx = lane_tap ? es32(kdx - (float)l, inv_hw, beta) : 0.0f;
            const float fy = lane_tap ? es32(kdy - (float)l, inv_hw, beta) : 0.0f;
            const int col = kcx + l;
            const bool okx = lane_tap && col >= 0 && col < Tw;
            const float ar = kre * fx, ai = kim * fx;
            float* pre = s_re + col;
            float* pim = s_im + col;
#pragma unroll
            for (int r = 0; r < (WT > 0 ? WT : GW); ++r) {
                if (WT == 0 && r >= W) break;
                const float py = __shfl_sync(gmask, fy, r, GW);
                const int row = kcy + r;
                if (okx && row >= 0 && row < Th) {
                    atomicAdd(pre + row * LD, ar * py);
                    atomicAdd(pim + row * LD, ai * py);
                }
            }
        }
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int y = warp; y < Th; y += kSpreadThreads / 32) {
        float2* dst = grid + (int64_t)(Y0 + y) * G + X0;
        for (int x = lane; x < Tw; x += 32) dst[x] = make_float2(s_re[y * LD + x], s_im[y * LD + x]);
    }
}

template <int GW, int WT, int T, bool VBF, bool ABF>
ftcg_status_t run_spread(const Plan& p, const void* vals, float2* grid, cudaStream_t s) {
    const Binning& b = p.bin;
    const size_t smem = (size_t)(2 * T * (T + 1)) * sizeof(float) + (size_t)(b.ncb + 1) * sizeof(int);
    auto kern = k_spread<GW, WT, T, VBF, ABF>;
    FTCG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const float beta = (float)p.win.beta;
    const float inv_hw = (float)(2.0 / p.win.w);
    kern<<<b.ntiles, kSpreadThreads, smem, s>>>(b.ent, b.colptr, vals, grid, b.G, b.ntx, b.W, beta,
                                                inv_hw);
    FTCG_CK(cudaGetLastError());
    return FTCG_SUCCESS;
}

template <int T, bool VBF, bool ABF>
ftcg_status_t dispatch_w(const Plan& p, const void* vals, float2* grid, cudaStream_t s) {
    switch (p.w) {
        case 6: return run_spread<8, 6, T, VBF, ABF>(p, vals, grid, s);
        case 8: return run_spread<8, 8, T, VBF, ABF>(p, vals, grid, s);
        default:
            if (p.w <= 4) return run_spread<4, 0, T, VBF, ABF>(p, vals, grid, s);
            if (p.w <= 8) return run_spread<8, 0, T, VBF, ABF>(p, vals, grid, s);
            return run_spread<16, 0, T, VBF, ABF>(p, vals, grid, s);
    }
}

template <bool VBF, bool ABF>
ftcg_status_t dispatch_t(const Plan& p, const void* vals, float2* grid, cudaStream_t s) {
    if (p.bin.T == 32) return dispatch_w<32, VBF, ABF>(p, vals, grid, s);
    return dispatch_w<64, VBF, ABF>(p, vals, grid, s);
}

// ---- deapodisation and crop: I_p = h_{p mod G} / (phi^(p_x/G) phi^(p_y/G)), FP64 factors ----
__global__ void k_deapod_crop(const float2* __restrict__ grid, float2* __restrict__ img,
                              const double* __restrict__ r, int N, int G) {
    const int64_t total = (int64_t)N * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int iy = (int)(i / N), ix = (int)(i - (int64_t)iy * N);
        int qy = iy - N / 2, qx = ix - N / 2;
        if (qy < 0) qy += G;
        if (qx < 0) qx += G;
        const float2 h = grid[(int64_t)qy * G + qx];
        const double f = r[iy] * r[ix];
        img[i] = make_float2((float)((double)h.x * f), (float)((double)h.y * f));
    }
}

// ---- forward: zero grid, place I_p / (phi^ phi^) at p mod G -----------------------------------
__global__ void k_pad_apod(const float2* __restrict__ img, float2* __restrict__ grid,
                           const double* __restrict__ r, int N, int G) {
    const int64_t total = (int64_t)N * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int iy = (int)(i / N), ix = (int)(i - (int64_t)iy * N);
        int qy = iy - N / 2, qx = ix - N / 2;
        if (qy < 0) qy += G;
        if (qx < 0) qx += G;
        const float2 v = img[i];
        const double f = r[iy] * r[ix];
        grid[(int64_t)qy * G + qx] = make_float2((float)((double)v.x * f), (float)((double)v.y * f));
    }
}

// ---- forward interpolation: f_j = sum_taps phi(dx - tx) phi(dy - ty) h[(c + t) mod G] ---------
template <int GW>
__global__ void __launch_bounds__(256)
    k_interp(const int4* __restrict__ samp, int64_t M, const float2* __restrict__ grid,
             float2* __restrict__ out, int G, int W, float beta, float inv_hw) {
    const int l = threadIdx.x % GW;
    const unsigned gmask = ((1u << GW) - 1u) << ((threadIdx.x & 31) & ~(GW - 1));
    const int64_t groups_total = (int64_t)gridDim.x * (blockDim.x / GW);
    for (int64_t j = blockIdx.x * (int64_t)(blockDim.x / GW) + threadIdx.x / GW; j < M;
         j += groups_total) {
        const int4 sm = samp[j];
        float re = 0.f, im = 0.f;
        if (sm.x >= 0) {
            const float dx = __int_as_float(sm.z), dy = __int_as_float(sm.w);
            const bool lane_tap = l < W;
            const float fx = lane_tap ? es32(dx - (float)l, inv_hw, beta) : 0.0f;
            const float fy = lane_tap ? es32(dy - (float)l, inv_hw, beta) : 0.0f;
            int col = sm.x + l;
            if (col >= G) col -= G;
            for (int r = 0; r < W; ++r) {
                const float py = __shfl_sync(gmask, fy, r, GW);
                int row = sm.y + r;
                if (row >= G) row -= G;
                if (lane_tap) {
                    const float2 h = grid[(int64_t)row * G + col];
                    re = fmaf(py, h.x, re);
                    im = fmaf(py, h.y, im);
                }
            }
            re *= fx;
            im *= fx;
        }
        for (int o = GW / 2; o > 0; o >>= 1) {
            re += __shfl_xor_sync(gmask, re, o, GW);
            im += __shfl_xor_sync(gmask, im, o, GW);
        }
        if (l == 0) out[j] = make_float2(re, im);
    }
}

// ---- per-entry weights ---------------------------------------------------------------------
__global__ void k_set_alpha(Entry* __restrict__ ent, int64_t n, const void* __restrict__ alpha,
                            int dtype, bool bf16) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = ent[i].packed & kSampleMask;
        float a = 1.0f;
        if (alpha) {
            a = dtype == FTCG_WEIGHTS_F64 ? (float)reinterpret_cast<const double*>(alpha)[j]
                                          : reinterpret_cast<const float*>(alpha)[j];
        }
        ent[i].alpha = bf16 ? (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a))
                            : __float_as_uint(a);
    }
}

int blocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

}  // namespace

ftcg_status_t launch_spread(const Plan& p, const void* vals, int vdtype, float2* grid,
                            cudaStream_t s) {
    if (p.bin.n_entries == 0) {
        FTCG_CK(cudaMemsetAsync(grid, 0, (size_t)p.G * p.G * sizeof(float2), s));
        return FTCG_SUCCESS;
    }
    const bool vbf = vdtype == FTCG_VALUES_BF16X2;
    const bool abf = p.opts.precision == FTCG_PREC_BF16;
    if (vbf && abf) return dispatch_t<true, true>(p, vals, grid, s);
    if (vbf) return dispatch_t<true, false>(p, vals, grid, s);
    if (abf) return dispatch_t<false, true>(p, vals, grid, s);
    return dispatch_t<false, false>(p, vals, grid, s);
}

ftcg_status_t launch_deapod_crop(const Plan& p, const float2* grid, float2* img, cudaStream_t s) {
    const int64_t n = (int64_t)p.N * p.N;
    k_deapod_crop<<<blocks_for(n, 256), 256, 0, s>>>(grid, img, p.deapod, p.N, p.G);
    FTCG_CK(cudaGetLastError());
    return FTCG_SUCCESS;
}

ftcg_status_t launch_pad_apod(const Plan& p, const float2* img, float2* grid, cudaStream_t s) {
    FTCG_CK(cudaMemsetAsync(grid, 0, (size_t)p.G * p.G * sizeof(float2), s));
    const int64_t n = (int64_t)p.N * p.N;
    k_pad_apod<<<blocks_for(n, 256), 256, 0, s>>>(img, grid, p.deapod, p.N, p.G);
    FTCG_CK(cudaGetLastError());
    return FTCG_SUCCESS;
}

ftcg_status_t launch_interp(const Plan& p, const float2* grid, float2* vals, cudaStream_t s) {
    if (p.M == 0) return FTCG_SUCCESS;
    const float beta = (float)p.win.beta;
    const float inv_hw = (float)(2.0 / p.win.w);
    if (p.w <= 8) {
        k_interp<8><<<blocks_for(p.M * 8, 256), 256, 0, s>>>(p.samp, p.M, grid, vals, p.G, p.w,
                                                             beta, inv_hw);
    } else {
        k_interp<16><<<blocks_for(p.M * 16, 256), 256, 0, s>>>(p.samp, p.M, grid, vals, p.G, p.w,
                                                               beta, inv_hw);
    }
    FTCG_CK(cudaGetLastError());
    return FTCG_SUCCESS;
}

ftcg_status_t launch_set_alpha(const Plan& p, const void* alpha, int dtype, cudaStream_t s) {
    if (p.bin.n_entries == 0) return FTCG_SUCCESS;
    k_set_alpha<<<blocks_for(p.bin.n_entries, 256), 256, 0, s>>>(
        p.bin.ent, p.bin.n_entries, alpha, dtype, p.opts.precision == FTCG_PREC_BF16);
    FTCG_CK(cudaGetLastError());
    return FTCG_SUCCESS;
}

}  // namespace ftcg
