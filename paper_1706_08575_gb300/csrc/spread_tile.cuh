// The spreading tile body shared by the single-ping kernel (spread.cu) and the persistent
// batched kernel (batch.cu). See spread.cu for the algorithm.
#pragma once

#include "ftcg_internal.cuh"

namespace ftcg {
namespace tile {

constexpr int kSpreadThreads = 256;

// ES window in FP32: exp(beta (sqrt(1 - z^2) - 1)) written as exp(-beta z^2 / (1 + sqrt(1 - z^2)))
// so that no cancellation occurs near the centre (sqrt(1 - z^2) - 1 loses all its digits there).
__device__ __forceinline__ float es32(float t, float inv_hw, float beta) {
    const float z = t * inv_hw;
    const float z2 = z * z;
    const float q = 1.0f - z2;
    return q >= 0.0f ? __expf(__fdividef(-beta * z2, 1.0f + sqrtf(q))) : 0.0f;
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

// One tile, by the whole CTA. GW: lanes per group (power of two >= w); WT: compile-time w
// (0 = runtime w <= GW). smem holds 2 T (T + 1) floats + (T + w) ints.
template <int GW, int WT, int T, bool VBF, bool ABF>
__device__ __forceinline__ void spread_tile(const Entry* __restrict__ ent,
                                            const int* __restrict__ colptr,
                                            const void* __restrict__ vals,
                                            float2* __restrict__ grid, int G, int ntx, int Wrt,
                                            float beta, float inv_hw, int tile, float* smem) {
    constexpr int LD = T + 1;
    constexpr int NG = kSpreadThreads / GW;
    constexpr int WMAX = WT > 0 ? WT : GW;
    const int W = WT > 0 ? WT : Wrt;
    const int ncb = T + W - 1;
    float* s_re = smem;
    float* s_im = smem + T * LD;
    int* s_col = reinterpret_cast<int*>(smem + 2 * T * LD);

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
    const bool lane_tap = l < W;

    float ar[WMAX], ai[WMAX];
#pragma unroll
    for (int r = 0; r < WMAX; ++r) ar[r] = ai[r] = 0.0f;
    int cur_cx = -(1 << 30);   // column bin of the window (local first-tap column), none yet
    int yb = 0;                // local row of window slot 0

    // add the whole window to the tile (rows outside the tile belong to other tiles)
    auto flush_all = [&]() {
        const int col = cur_cx + l;
        const bool okx = lane_tap && col >= 0 && col < Tw;
#pragma unroll
        for (int r = 0; r < WMAX; ++r) {
            const int row = yb + r;
            if (okx && r < W && row >= 0 && row < Th) {
                atomicAdd(s_re + row * LD + col, ar[r]);
                atomicAdd(s_im + row * LD + col, ai[r]);
            }
            ar[r] = ai[r] = 0.0f;
        }
    };

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
            if (kcx != cur_cx || kcy - yb >= W) {
                flush_all();
                cur_cx = kcx;
                yb = kcy;
            } else {
                while (yb < kcy) {               // rows below kcy are final for this column bin
                    const int col = cur_cx + l;
                    if (lane_tap && col >= 0 && col < Tw && yb >= 0 && yb < Th) {
                        atomicAdd(s_re + yb * LD + col, ar[0]);
                        atomicAdd(s_im + yb * LD + col, ai[0]);
                    }
#pragma unroll
                    for (int r = 0; r + 1 < WMAX; ++r) {
                        ar[r] = ar[r + 1];
                        ai[r] = ai[r + 1];
                    }
                    ar[WMAX - 1] = ai[WMAX - 1] = 0.0f;
                    ++yb;
                }
            }
            const float fx = lane_tap ? es32(kdx - (float)l, inv_hw, beta) : 0.0f;
            const float fy = lane_tap ? es32(kdy - (float)l, inv_hw, beta) : 0.0f;
            const float xr = kre * fx, xi = kim * fx;
#pragma unroll
            for (int r = 0; r < WMAX; ++r) {
                const float py = __shfl_sync(gmask, fy, r, GW);   // zero for r >= W
                ar[r] = fmaf(xr, py, ar[r]);
                ai[r] = fmaf(xi, py, ai[r]);
            }
        }
    }
    flush_all();
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int y = warp; y < Th; y += kSpreadThreads / 32) {
        float2* dst = grid + (int64_t)(Y0 + y) * G + X0;
        for (int x = lane; x < Tw; x += 32) dst[x] = make_float2(s_re[y * LD + x], s_im[y * LD + x]);
    }
}

}  // namespace tile
}  // namespace ftcg
