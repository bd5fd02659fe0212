// The tensor-core spreading tile body (see spread_mma.cu for the method), shared by the
// single-ping kernel and the persistent batched kernel (batch.cu).
#pragma once

#include "spread_tile.cuh"

namespace ftcg {
namespace mma {

// Build-time knobs (defaults are the tuned values): FTCG_MMA_THREADS threads per CTA,
// FTCG_MMA_MINB minimum resident CTAs per SM requested from the register allocator.
#ifndef FTCG_MMA_THREADS
#define FTCG_MMA_THREADS 256
#endif
#ifndef FTCG_MMA_MINB
#define FTCG_MMA_MINB 3
#endif
constexpr int kThreads = FTCG_MMA_THREADS;
constexpr int kWarps = kThreads / 32;
constexpr int kMinBlocks = FTCG_MMA_MINB;
// chunks the loop reads ahead of the one it computes: slots two ahead, values one ahead
constexpr int kPrefetchChunks = 2;

// Dynamic shared memory of one tile: the two accumulator planes of the (T + 7)^2 block.
__host__ __device__ constexpr size_t tile_smem_bytes(int T) {
    return (size_t)2 * (T + kMmaMaxW - 1) * (T + kMmaMaxW) * sizeof(float);
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// x = hi + lo, both TF32 (lo rounded too, so the MMA reads it without further truncation)
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = tf32_rna(x);
    lo = tf32_rna(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float horner(const float (&c)[kMmaDeg + 1], float s) {
    float p = c[kMmaDeg];
#pragma unroll
    for (int k = kMmaDeg - 1; k >= 0; --k) p = fmaf(p, s, c[k]);
    return p;
}

template <bool VBF>
__device__ __forceinline__ float2 chunk_value(const void* __restrict__ vals, uint32_t packed) {
    return (packed & kMmaPad) ? make_float2(0.f, 0.f)
                              : tile::load_value<VBF>(vals, packed & kSampleMask);
}

// One halo-layout tile by the whole CTA (kThreads threads): its chunks [tile_chunk[tile],
// tile_chunk[tile + 1]) split into contiguous ranges, one per warp; then the tile and its
// overflow strips are stored. smem: tile_smem_bytes(T).
template <int T, bool VBF, bool ABF>
__device__ __forceinline__ void spread_tile(const MmaEntry* __restrict__ cent,
                                            const uint32_t* __restrict__ chdr,
                                            const int* __restrict__ tile_chunk,
                                            const void* __restrict__ vals,
                                            float2* __restrict__ grid, int G, int ntx, int W,
                                            const MmaPoly& poly, float2* __restrict__ halo_buf,
                                            int halo_cells, int tile, float* smem) {
    constexpr int PT = T + kMmaMaxW - 1;     // accumulator side (tile + overflow strips)
    constexpr int LD = PT + 1;
    float* s_re = smem;
    float* s_im = smem + PT * LD;
    const int c0 = tile_chunk[tile], c1 = tile_chunk[tile + 1];
    const int tyi = tile / ntx, txi = tile - tyi * ntx;
    const int X0 = txi * T, Y0 = tyi * T;
    const int Tw = min(T, G - X0), Th = min(T, G - Y0);
    if (c0 == c1) {
        tile::store_zero_tile<kThreads>(grid, G, X0, Y0, Tw, Th);
        return;
    }
    for (int i = threadIdx.x; i < 2 * PT * LD; i += kThreads) smem[i] = 0.0f;
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;     // MMA fragment row group and column pair
    float cf[kMmaDeg + 1];                     // window polynomial of tap g
#pragma unroll
    for (int k = 0; k <= kMmaDeg; ++k) cf[k] = poly.c[g][k];
    const int n = c1 - c0;
    const int ca = c0 + (int)((int64_t)n * warp / kWarps);
    const int cb = c0 + (int)((int64_t)n * (warp + 1) / kWarps);
    // D fragments: real and imaginary plane, rows g (d[0], d[1]) and g + 8 (d[2], d[3]) of the
    // window, columns 2t and 2t + 1
    float dr[4] = {0.f, 0.f, 0.f, 0.f}, di[4] = {0.f, 0.f, 0.f, 0.f};
    int cur_cx = -1, cur_yb = 0;
    auto flush_half = [&](int h) {             // window rows g + 8h into the tile accumulator
        const int row = cur_yb + g + 8 * h;
        if (row < PT) {
            const int o = row * LD + cur_cx + 2 * t;   // cur_cx + 2t + 1 <= T + 6 < PT
            atomicAdd(s_re + o, dr[2 * h]);
            atomicAdd(s_re + o + 1, dr[2 * h + 1]);
            atomicAdd(s_im + o, di[2 * h]);
            atomicAdd(s_im + o + 1, di[2 * h + 1]);
        }
    };

    if (ca < cb) {
        // software pipeline: the slots of chunk c + 2 and the values of chunk c + 1 are in
        // flight while chunk c is computed (the chunk array ends with kPrefetchChunks padding
        // chunks, so the reads ahead need no bounds test; padding slots load no value)
        MmaEntry e1 = cent[(int64_t)ca * kMmaChunk + t];
        MmaEntry e2 = cent[(int64_t)ca * kMmaChunk + t + 4];
        float2 v1 = chunk_value<VBF>(vals, e1.packed);
        float2 v2 = chunk_value<VBF>(vals, e2.packed);
        MmaEntry n1 = cent[(int64_t)(ca + 1) * kMmaChunk + t];
        MmaEntry n2 = cent[(int64_t)(ca + 1) * kMmaChunk + t + 4];
        for (int c = ca; c < cb; ++c) {
            const uint32_t h = chdr[c];
            const float2 nv1 = chunk_value<VBF>(vals, n1.packed);
            const float2 nv2 = chunk_value<VBF>(vals, n2.packed);
            const MmaEntry nn1 = cent[(int64_t)(c + 2) * kMmaChunk + t];
            const MmaEntry nn2 = cent[(int64_t)(c + 2) * kMmaChunk + t + 4];
            const int cx = (int)(h & 0xffu), yb = (int)((h >> 8) & 0xffu);
            if (cx != cur_cx || (yb != cur_yb && yb != cur_yb + 8)) {      // a new window
                if (cur_cx >= 0) {
                    flush_half(0);
                    flush_half(1);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) dr[i] = di[i] = 0.f;
                cur_cx = cx;
                cur_yb = yb;
            } else if (yb != cur_yb) {             // the window moves down by 8 rows
                flush_half(0);
                dr[0] = dr[2];
                dr[1] = dr[3];
                di[0] = di[2];
                di[1] = di[3];
                dr[2] = dr[3] = di[2] = di[3] = 0.f;
                cur_yb = yb;
            }
            const float al1 = ABF ? tile::bf16_bits_to_float(e1.alpha) : __uint_as_float(e1.alpha);
            const float al2 = ABF ? tile::bf16_bits_to_float(e2.alpha) : __uint_as_float(e2.alpha);
            // column factor (tap g) with the weight, row factor of tap g of each sample
            const float fx1 = horner(cf, e1.sx) * al1, fx2 = horner(cf, e2.sx) * al2;
            const float fy1 = horner(cf, e1.sy), fy2 = horner(cf, e2.sy);
            const int off1 = (int)((e1.packed >> kSampleBits) & 15u);
            const int off2 = (int)((e2.packed >> kSampleBits) & 15u);
            // A[r][k]: window row r = g or g + 8 takes tap (g - off) mod 8 of sample k, held by
            // lane ((g - off) & 7, t) (every lane with the same t evaluates the same samples)
            const float a1 = __shfl_sync(0xffffffffu, fy1, (((g - off1) & 7) << 2) | t);
            const float a2 = __shfl_sync(0xffffffffu, fy2, (((g - off2) & 7) << 2) | t);
            const bool low1 = g >= off1, low2 = g >= off2;
            uint32_t a1h, a1l, a2h, a2l;
            split_tf32(a1, a1h, a1l);
            split_tf32(a2, a2h, a2l);
            uint32_t b1rh, b1rl, b1ih, b1il, b2rh, b2rl, b2ih, b2il;
            split_tf32(v1.x * fx1, b1rh, b1rl);
            split_tf32(v1.y * fx1, b1ih, b1il);
            split_tf32(v2.x * fx2, b2rh, b2rl);
            split_tf32(v2.y * fx2, b2ih, b2il);
            const uint32_t ah0 = low1 ? a1h : 0u, ah1 = low1 ? 0u : a1h;
            const uint32_t ah2 = low2 ? a2h : 0u, ah3 = low2 ? 0u : a2h;
            const uint32_t al0 = low1 ? a1l : 0u, al1r = low1 ? 0u : a1l;
            const uint32_t al2r = low2 ? a2l : 0u, al3 = low2 ? 0u : a2l;
            mma_tf32(dr, ah0, ah1, ah2, ah3, b1rh, b2rh);
            mma_tf32(dr, ah0, ah1, ah2, ah3, b1rl, b2rl);
            mma_tf32(dr, al0, al1r, al2r, al3, b1rh, b2rh);
            mma_tf32(di, ah0, ah1, ah2, ah3, b1ih, b2ih);
            mma_tf32(di, ah0, ah1, ah2, ah3, b1il, b2il);
            mma_tf32(di, al0, al1r, al2r, al3, b1ih, b2ih);
            e1 = n1;
            e2 = n2;
            v1 = nv1;
            v2 = nv2;
            n1 = nn1;
            n2 = nn2;
        }
        flush_half(0);
        flush_half(1);
    }
    __syncthreads();
    tile::store_tile<true, kThreads>(s_re, s_im, LD, grid, G, X0, Y0, Tw, Th, T, W,
                                     halo_buf + (int64_t)tile * halo_cells, halo_cells);
}

}  // namespace mma
}  // namespace ftcg
