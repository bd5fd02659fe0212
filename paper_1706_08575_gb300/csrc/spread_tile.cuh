// The spreading tile body shared by the single-ping kernel (spread.cu) and the persistent
// batched kernel (batch.cu). See spread.cu for the algorithm.
#pragma once

#include "ftcg_internal.cuh"

namespace ftcg {
namespace tile {

// Build-time knobs of the spreading kernels (the defaults are the tuned values):
//   FTCG_SPREAD_THREADS  threads per CTA; FTCG_SPREAD_MINB  minimum resident CTAs per SM requested
//   from the register allocator; FTCG_SPREAD_WINDOW  1 = rolling row window, 0 = one shared
//   atomic per tap.
#ifndef FTCG_SPREAD_THREADS
#define FTCG_SPREAD_THREADS 256
#endif
#ifndef FTCG_SPREAD_MINB
#define FTCG_SPREAD_MINB 1
#endif
#ifndef FTCG_SPREAD_WINDOW
#define FTCG_SPREAD_WINDOW 1
#endif
constexpr int kSpreadThreads = FTCG_SPREAD_THREADS;

// ES window in FP32: exp(beta (sqrt(1 - z^2) - 1)) written as exp(-beta z^2 / (1 + sqrt(1 - z^2)))
// so that no cancellation occurs near the centre (sqrt(1 - z^2) - 1 loses all its digits there).
__device__ __forceinline__ float es32(float t, float inv_hw, float beta) {
    const float z = t * inv_hw;
    const float z2 = z * z;
    const float q = 1.0f - z2;
    return q >= 0.0f ? __expf(__fdividef(-beta * z2, 1.0f + sqrtf(q))) : 0.0f;
}

// A BF16-stored weight is a float32 whose low 16 bits are zero (the bfloat16 rounding of the
// weight); masking also reads an unrounded float32 (such as the plan's default 1.0) as bfloat16.
__device__ __forceinline__ float bf16_bits_to_float(uint32_t bits) {
    return __uint_as_float(bits & 0xffff0000u);
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

    if (a < b) {
        // the column bin of the first entry (last k with s_col[k] <= a), then walk the bins
        int lo = 0, hi = ncb - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_col[mid] <= a) lo = mid; else hi = mid - 1;
        }
        int bin = lo;
        int bin_end = s_col[bin + 1];
        cur_cx = bin - (W - 1);
        // every lane of the group reads the same entry (one broadcast load per group); entries
        // are prefetched two ahead and values one ahead
        Entry ec = ent[a];
        float2 vc = load_value<VBF>(vals, ec.packed & kSampleMask);
        Entry en = a + 1 < b ? ent[a + 1] : ec;
        yb = (int)(ec.packed >> kSampleBits) - (W - 1);
        for (int idx = a; idx < b; ++idx) {
            const Entry e2 = idx + 2 < b ? ent[idx + 2] : en;
            const float2 vn = idx + 1 < b ? load_value<VBF>(vals, en.packed & kSampleMask) : vc;
            const int cyl = (int)(ec.packed >> kSampleBits) - (W - 1);
            if (idx >= bin_end) {                // the next column bin (empty bins skipped)
                flush_all();
                do {
                    ++bin;
                } while (s_col[bin + 1] <= idx);
                bin_end = s_col[bin + 1];
                cur_cx = bin - (W - 1);
                yb = cyl;
            } else if (cyl - yb >= W) {
                flush_all();
                yb = cyl;
            } else {
                while (yb < cyl) {               // rows below cyl are final for this column bin
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
            const float al = ABF ? bf16_bits_to_float(ec.alpha) : __uint_as_float(ec.alpha);
            const float fx = lane_tap ? es32(ec.dx - (float)l, inv_hw, beta) : 0.0f;
            const float fy = lane_tap ? es32(ec.dy - (float)l, inv_hw, beta) : 0.0f;
            const float ax = al * fx;
            const float xr = vc.x * ax, xi = vc.y * ax;
#if FTCG_SPREAD_WINDOW
#pragma unroll
            for (int r = 0; r < WMAX; ++r) {
                const float py = __shfl_sync(gmask, fy, r, GW);   // zero for r >= W
                ar[r] = fmaf(xr, py, ar[r]);
                ai[r] = fmaf(xi, py, ai[r]);
            }
#else
            {
                const int col = cur_cx + l;
                const bool okx = lane_tap && col >= 0 && col < Tw;
#pragma unroll
                for (int r = 0; r < WMAX; ++r) {
                    const float py = __shfl_sync(gmask, fy, r, GW);
                    const int row = cyl + r;
                    if (okx && r < W && row >= 0 && row < Th) {
                        atomicAdd(s_re + row * LD + col, xr * py);
                        atomicAdd(s_im + row * LD + col, xi * py);
                    }
                }
            }
#endif
            ec = en;
            vc = vn;
            en = e2;
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
