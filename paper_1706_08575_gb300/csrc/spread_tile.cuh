// The spreading tile body shared by the single-ping kernel (spread.cu) and the persistent
// batched kernel (batch.cu). See spread.cu for the algorithm.
#pragma once

#include "ftcg_internal.cuh"

namespace ftcg {
namespace tile {

// Build-time knobs of the spreading kernels (the defaults are the tuned values):
//   FTCG_SPREAD_THREADS  threads per CTA;
//   FTCG_SPREAD_MINB     minimum resident CTAs per SM requested from the register allocator;
//   FTCG_SPREAD_UNROLL   unroll factor of the entry loop;
//   FTCG_SPREAD_CPL8 / FTCG_SPREAD_CPL16  tap columns per lane for 4 < w <= 8 / 8 < w <= 16
//                        (a group then has 8 / CPL8 resp. 16 / CPL16 lanes).
#ifndef FTCG_SPREAD_THREADS
#define FTCG_SPREAD_THREADS 256
#endif
#ifndef FTCG_SPREAD_MINB
#define FTCG_SPREAD_MINB 4
#endif
#ifndef FTCG_SPREAD_UNROLL
#define FTCG_SPREAD_UNROLL 2
#endif
#ifndef FTCG_SPREAD_CPL8
#define FTCG_SPREAD_CPL8 1
#endif
#ifndef FTCG_SPREAD_CPL16
#define FTCG_SPREAD_CPL16 1
#endif
constexpr int kSpreadThreads = FTCG_SPREAD_THREADS;
constexpr int kCpl8 = FTCG_SPREAD_CPL8, kCpl16 = FTCG_SPREAD_CPL16;
constexpr int kSpreadUnroll = FTCG_SPREAD_UNROLL;

// The gridding window in FP32 at offset t (cells), zero outside |t| <= w/2. ES:
// exp(beta (sqrt(1 - z^2) - 1)) written as exp(-beta z^2 / (1 + sqrt(1 - z^2))) so that no
// cancellation occurs near the centre (sqrt(1 - z^2) - 1 loses all its digits there); Kaiser-
// Bessel: I0(beta sqrt(1 - z^2)) / I0(beta); truncated Gaussian: exp(-beta z^2). The family is
// uniform across a launch, so the branch costs no divergence; es32 is the ES branch alone (the
// kernels instantiate it separately, which saves the family test in their inner loops).
__device__ __forceinline__ float es32(float t, const Win32& w) {
    const float z = t * w.inv_hw;
    const float z2 = z * z;
    const float q = 1.0f - z2;
    return q >= 0.0f ? __expf(__fdividef(-w.beta * z2, 1.0f + sqrtf(q))) : 0.0f;
}

__device__ __forceinline__ float win32(float t, const Win32& w) {
    const float z = t * w.inv_hw;
    const float z2 = z * z;
    const float q = 1.0f - z2;
    if (!(q >= 0.0f)) return 0.0f;
    if (w.kind == FTCG_WINDOW_KB) return cyl_bessel_i0f(w.beta * sqrtf(q)) * w.norm;
    if (w.kind == FTCG_WINDOW_GAUSS) return __expf(-w.beta * z2);
    return __expf(__fdividef(-w.beta * z2, 1.0f + sqrtf(q)));
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

// Side of the shared accumulator: the tile, plus the overflow strips in the halo layout.
template <int T, int WMAX, bool HALO>
__host__ __device__ constexpr int acc_side() { return HALO ? T + WMAX - 1 : T; }

// Dynamic shared memory of one tile body: two accumulator planes and T + w + 1 column offsets.
template <int T, int WMAX, bool HALO>
__host__ __device__ constexpr size_t tile_smem_bytes() {
    return (size_t)(2 * acc_side<T, WMAX, HALO>() * (acc_side<T, WMAX, HALO>() + 1)) * sizeof(float) +
           (size_t)(T + WMAX + 1) * sizeof(int);
}

// Store a finished tile from its shared accumulator planes (row stride LD): the tile's own
// Tw x Th cells to the grid, coalesced (every cell written once), and in the halo layout the
// overflow strips to the tile's slots of the halo buffer: right strip (rows 0..Th+w-2, columns
// Tw..Tw+w-2), then bottom strip (rows Th..Th+w-2, columns 0..Tw-1); the slot layout is fixed
// by T so that k_halo_add can decode it. Called by every thread of the CTA after a barrier.
template <bool HALO, int NT>
__device__ __forceinline__ void store_tile(const float* __restrict__ s_re,
                                           const float* __restrict__ s_im, int LD,
                                           float2* __restrict__ grid, int G, int X0, int Y0,
                                           int Tw, int Th, int T, int W, float2* __restrict__ hb,
                                           int halo_cells) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int y = warp; y < Th; y += NT / 32) {
        float2* dst = grid + (int64_t)(Y0 + y) * G + X0;
        for (int x = lane; x < Tw; x += 32) dst[x] = make_float2(s_re[y * LD + x], s_im[y * LD + x]);
    }
    if (HALO) {
        const int right = (T + W - 1) * (W - 1);
        for (int k = threadIdx.x; k < halo_cells; k += NT) {
            int y, x;
            if (k < right) {
                y = k / (W - 1);
                x = Tw + (k - y * (W - 1));
                if (y >= Th + W - 1) continue;
            } else {
                const int kk = k - right;
                y = Th + kk / T;
                x = kk - (kk / T) * T;
                if (x >= Tw) continue;
            }
            hb[k] = make_float2(s_re[y * LD + x], s_im[y * LD + x]);
        }
    }
}

// Store zeros over an empty tile's own cells (its halo strips are never read: k_halo_add skips
// empty tiles).
template <int NT>
__device__ __forceinline__ void store_zero_tile(float2* __restrict__ grid, int G, int X0, int Y0,
                                                int Tw, int Th) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int y = warp; y < Th; y += NT / 32) {
        float2* dst = grid + (int64_t)(Y0 + y) * G + X0;
        for (int x = lane; x < Tw; x += 32) dst[x] = make_float2(0.f, 0.f);
    }
}

// One tile, by the whole CTA. GW: lanes per group (power of two); CPL: tap columns per lane
// (lane l owns columns l, l + GW, ..., so GW * CPL >= w); WT: compile-time w (0 = runtime
// w <= GW * CPL). HALO: the tile's entries are the samples whose first tap lies in it; the
// accumulator covers the tile plus w - 1 cells to the right and below, the tile's own cells go to
// the grid and the overflow strips to halo_buf (added to the neighbours by k_halo_add).
// ES: the window is the exponential of semicircle (es32), otherwise any family (win32).
template <int GW, int WT, int T, bool VBF, bool ABF, bool HALO, int CPL, bool ES = true>
__device__ __forceinline__ void spread_tile(const Entry* __restrict__ ent,
                                            const int* __restrict__ colptr,
                                            const void* __restrict__ vals,
                                            float2* __restrict__ grid, int G, int ntx, int Wrt,
                                            Win32 win, int tile, float* smem,
                                            float2* __restrict__ halo_buf, int halo_cells) {
    constexpr int WMAX = WT > 0 ? WT : GW * CPL;
    static_assert(WMAX <= GW * CPL, "a group must cover the kernel width");
    constexpr int PT = acc_side<T, WMAX, HALO>();
    constexpr int LD = PT + 1;
    constexpr int NG = kSpreadThreads / GW;
    const int W = WT > 0 ? WT : Wrt;
    const int ncb = T + W - 1;
    float* s_re = smem;
    float* s_im = smem + PT * LD;
    int* s_col = reinterpret_cast<int*>(smem + 2 * PT * LD);

    const int tyi = tile / ntx, txi = tile - tyi * ntx;
    const int X0 = txi * T, Y0 = tyi * T;
    const int Tw = min(T, G - X0), Th = min(T, G - Y0);

    if (colptr[(int64_t)tile * ncb] == colptr[(int64_t)(tile + 1) * ncb]) {
        // an empty tile (common under a polar footprint): store zeros, no accumulator, no halo
        store_zero_tile<kSpreadThreads>(grid, G, X0, Y0, Tw, Th);
        return;
    }
    for (int i = threadIdx.x; i < 2 * PT * LD; i += kSpreadThreads) smem[i] = 0.0f;
    for (int i = threadIdx.x; i <= ncb; i += kSpreadThreads) s_col[i] = colptr[(int64_t)tile * ncb + i];
    __syncthreads();

    const int e0 = s_col[0], e1 = s_col[ncb];
    const int n = e1 - e0;
    const int g = threadIdx.x / GW, l = threadIdx.x % GW;
    const unsigned gmask = (GW == 32 ? 0xffffffffu : ((1u << GW) - 1u)) << ((threadIdx.x & 31) & ~(GW - 1));
    const int per = (n + NG - 1) / NG;
    const int a = e0 + g * per;
    const int b = min(e1, a + per);
    bool tap[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) tap[c] = l + c * GW < W;

    float ar[CPL][WMAX], ai[CPL][WMAX];
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
        for (int r = 0; r < WMAX; ++r) ar[c][r] = ai[c][r] = 0.0f;
    int cur_cx = -(1 << 30);   // column bin of the window (local first-tap column), none yet
    int yb = 0;                // local row of window slot 0

    // add the whole window to the tile (rows outside the tile belong to other tiles)
    auto flush_all = [&]() {
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int col = cur_cx + l + c * GW;
            const bool okx = tap[c] && (HALO || (col >= 0 && col < Tw));
#pragma unroll
            for (int r = 0; r < WMAX; ++r) {
                const int row = yb + r;
                if (okx && r < W && (HALO || (row >= 0 && row < Th))) {
                    atomicAdd(s_re + row * LD + col, ar[c][r]);
                    atomicAdd(s_im + row * LD + col, ai[c][r]);
                }
                ar[c][r] = ai[c][r] = 0.0f;
            }
        }
    };

    // flush window row 0 (tile row yb) and shift the window by one row
    auto advance_row = [&]() {
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int col = cur_cx + l + c * GW;
            if (tap[c] && (HALO || (col >= 0 && col < Tw && yb >= 0 && yb < Th))) {
                atomicAdd(s_re + yb * LD + col, ar[c][0]);
                atomicAdd(s_im + yb * LD + col, ai[c][0]);
            }
#pragma unroll
            for (int r = 0; r + 1 < WMAX; ++r) {
                ar[c][r] = ar[c][r + 1];
                ai[c][r] = ai[c][r + 1];
            }
            ar[c][WMAX - 1] = ai[c][WMAX - 1] = 0.0f;
        }
        ++yb;
    };

    // add entry e (value v) to window rows 0..w-1
    auto add_entry = [&](const Entry& e, float2 v) {
        const float al = ABF ? bf16_bits_to_float(e.alpha) : __uint_as_float(e.alpha);
        float xr[CPL], xi[CPL], fy[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const float tx = e.dx - (float)(l + c * GW), ty = e.dy - (float)(l + c * GW);
            const float fx = tap[c] ? (ES ? es32(tx, win) : win32(tx, win)) : 0.0f;
            fy[c] = tap[c] ? (ES ? es32(ty, win) : win32(ty, win)) : 0.0f;
            const float ax = al * fx;
            xr[c] = v.x * ax;
            xi[c] = v.y * ax;
        }
#pragma unroll
        for (int r = 0; r < WMAX; ++r) {
            // row factor r lives in lane r % GW, slot r / GW (zero for r >= W)
            const float py = __shfl_sync(gmask, fy[r / GW], r % GW, GW);
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                ar[c][r] = fmaf(xr[c], py, ar[c][r]);
                ai[c][r] = fmaf(xi[c], py, ai[c][r]);
            }
        }
    };

    // the column bin of entry i (last k with s_col[k] <= i)
    auto find_bin = [&](int i) {
        int lo = 0, hi = ncb - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_col[mid] <= i) lo = mid; else hi = mid - 1;
        }
        return lo;
    };

    if (a < b) {
        int bin = find_bin(a);
        int bin_end = s_col[bin + 1];
        cur_cx = bin - (W - 1);
        // every lane of the group reads the same entry (one broadcast load per group); entries
        // are prefetched two ahead and values one ahead (the entry array is padded, so the
        // prefetch needs no bounds test)
        Entry ec = ent[a];
        float2 vc = load_value<VBF>(vals, ec.packed & kSampleMask);
        Entry en = ent[a + 1];
        yb = (int)(ec.packed >> kSampleBits) - (W - 1);
#pragma unroll kSpreadUnroll
        for (int idx = a; idx < b; ++idx) {
            const Entry e2 = ent[idx + 2];
            const float2 vn = load_value<VBF>(vals, en.packed & kSampleMask);
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
                while (yb < cyl) advance_row();   // rows below cyl are final for this bin
            }
            add_entry(ec, vc);
            ec = en;
            vc = vn;
            en = e2;
        }
        flush_all();                              // only groups that held a window flush it
    }
    __syncthreads();
    store_tile<HALO, kSpreadThreads>(s_re, s_im, LD, grid, G, X0, Y0, Tw, Th, T, W,
                                     halo_buf + (int64_t)tile * halo_cells, halo_cells);
}

// Adds the overflow strips of a halo-layout tile to the grid cells they belong to (wrapping mod
// G). Cells receive at most three such additions (left, upper and upper-left tile), so float
// atomics are cheap; the tiles' own cells were stored by the spreading kernel before. colptr:
// the binning's, to skip an empty tile (it wrote no strips); nullptr when the caller launches
// non-empty tiles only.
__device__ __forceinline__ void halo_add_tile(const float2* __restrict__ halo_buf, int halo_cells,
                                              const int* __restrict__ colptr, int ncb,
                                              float2* __restrict__ grid, int G, int T, int W,
                                              int ntx, int tile) {
    if (colptr && colptr[(int64_t)(tile + 1) * ncb] == colptr[(int64_t)tile * ncb]) return;
    const int tyi = tile / ntx, txi = tile - tyi * ntx;
    const int X0 = txi * T, Y0 = tyi * T;
    const int Tw = min(T, G - X0), Th = min(T, G - Y0);
    const float2* hb = halo_buf + (int64_t)tile * halo_cells;
    const int right = (T + W - 1) * (W - 1);
    for (int k = threadIdx.x; k < halo_cells; k += blockDim.x) {
        int y, x;
        if (k < right) {
            y = k / (W - 1);
            x = Tw + (k - y * (W - 1));
            if (y >= Th + W - 1) continue;
        } else {
            const int kk = k - right;
            y = Th + kk / T;
            x = kk - (kk / T) * T;
            if (x >= Tw) continue;
        }
        int gy = Y0 + y, gx = X0 + x;
        if (gy >= G) gy -= G;
        if (gx >= G) gx -= G;
        atomicAdd(grid + (int64_t)gy * G + gx, hb[k]);     // one 8-byte vector atomic
    }
}

}  // namespace tile
}  // namespace ftcg
