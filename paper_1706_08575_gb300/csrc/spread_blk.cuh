// The block tensor-core spreading tile body (see spread_mma.cu for the method), shared by the
// single-ping kernel and the persistent batched kernel (batch.cu).
//
// A chunk holds up to 8 samples whose first taps lie in one 8 x 8 block of cells of the tile; its
// window is the 16 x 16 cells from the block's origin, which every tap of those samples falls
// in. The window's sum over the chunk is two matrix products per plane,
//
//   g[by + r][bx + 8h + n] += sum_k phi(dy_k - (r - offy_k)) * (alpha_k v_k phi(dx_k - (8h + n - offx_k))),
//
// r in 0..15, n in 0..7, h in {0, 1} (the two 8-column halves), A and B zero outside the sample's
// taps, so 12 split-TF32 mma.sync.m16n8k8 per chunk (3 products x 2 planes x 2 halves). The
// chunks of a block follow one another and share the window, which stays in the D fragments until
// the block changes; then its 16 x 16 cells are added to the tile's shared accumulator. There is
// no window to shift: the bookkeeping per chunk is one comparison.
#pragma once

#include "spread_mma.cuh"

namespace ftcg {
namespace blk {

using mma::kThreads;
using mma::kWarps;
using mma::StagedSlot;
using mma::kStageChunks;
using mma::kStageSlots;

// Bits of a block chunk slot's packed word: sample index (kSampleBits), then the first tap's
// column and row within the block (3 bits each), then the padding flag (kMmaPad).
constexpr int kOffXShift = kSampleBits;
constexpr int kOffYShift = kSampleBits + 3;

// Load slot i of the chunk array (a padding slot, or an index past the warp's range, gives
// c = 0): its offsets, weighted value, and the 6-bit (offx | offy << 3) position in the block.
template <bool VBF, bool ABF>
__device__ __forceinline__ void load_block_slot(const MmaEntry* __restrict__ cent,
                                          const void* __restrict__ vals, int64_t i, int64_t end,
                                          StagedSlot& out, int& pos) {
    const bool live = i < end;
    const MmaEntry e = cent[live ? i : end - 1];
    const float2 v = tile::load_value<VBF>(vals, e.packed & kSampleMask);
    float al = ABF ? tile::bf16_bits_to_float(e.alpha) : __uint_as_float(e.alpha);
    al = (live && !(e.packed & kMmaPad)) ? al : 0.0f;
    out.sx = e.sx;
    out.sy = e.sy;
    out.cr = al * v.x;
    out.ci = al * v.y;
    pos = (int)((e.packed >> kOffXShift) & 63u);
}

// One halo-layout tile by the whole CTA (kThreads threads): its block chunks
// [tile_chunk[tile], tile_chunk[tile + 1]) split into contiguous ranges, one per warp; then the
// tile and its overflow strips are stored. smem: mma::tile_smem_bytes(T).
template <int T, bool VBF, bool ABF>
__device__ __forceinline__ void spread_tile(const MmaEntry* __restrict__ cent,
                                            const uint32_t* __restrict__ chdr,
                                            const int* __restrict__ tile_chunk,
                                            const void* __restrict__ vals,
                                            float2* __restrict__ grid, int G, int ntx, int W,
                                            const MmaPoly& poly, float2* __restrict__ halo_buf,
                                            int halo_cells, int tile, float* smem) {
    constexpr int PR = mma::acc_rows(T);     // accumulator rows (a window reaches row T + 7)
    constexpr int LD = T + kMmaMaxW;         // row pitch (a window reaches column T + 7)
    float* s_re = smem;
    float* s_im = smem + PR * LD;
    const int c0 = tile_chunk[tile], c1 = tile_chunk[tile + 1];
    const int tyi = tile / ntx, txi = tile - tyi * ntx;
    const int X0 = txi * T, Y0 = tyi * T;
    const int Tw = min(T, G - X0), Th = min(T, G - Y0);
    if (c0 == c1) {
        tile::store_zero_tile<kThreads>(grid, G, X0, Y0, Tw, Th);
        return;
    }
    for (int i = threadIdx.x; i < 2 * PR * LD; i += kThreads) smem[i] = 0.0f;
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;     // MMA fragment row group and column pair
    float cf[kMmaDeg + 1];                     // window polynomial of tap g
#pragma unroll
    for (int k = 0; k <= kMmaDeg; ++k) cf[k] = poly.c[g][k];
    const int n = c1 - c0;
    const int ca = c0 + (int)((int64_t)n * warp / kWarps);
    const int cb = c0 + (int)((int64_t)n * (warp + 1) / kWarps);
    // D fragments of the two column halves, real and imaginary plane: rows g (d[0], d[1]) and
    // g + 8 (d[2], d[3]), columns 8h + 2t and 8h + 2t + 1
    float r0[4] = {0.f, 0.f, 0.f, 0.f}, i0[4] = {0.f, 0.f, 0.f, 0.f};
    float r1[4] = {0.f, 0.f, 0.f, 0.f}, i1[4] = {0.f, 0.f, 0.f, 0.f};
    int cur_bx = -1, cur_by = 0;
    auto flush = [&]() {                       // the window into the accumulator, then clear
        const int o = (cur_by + g) * LD + cur_bx + 2 * t;
        atomicAdd(s_re + o, r0[0]);
        atomicAdd(s_re + o + 1, r0[1]);
        atomicAdd(s_re + o + 8 * LD, r0[2]);
        atomicAdd(s_re + o + 8 * LD + 1, r0[3]);
        atomicAdd(s_im + o, i0[0]);
        atomicAdd(s_im + o + 1, i0[1]);
        atomicAdd(s_im + o + 8 * LD, i0[2]);
        atomicAdd(s_im + o + 8 * LD + 1, i0[3]);
        atomicAdd(s_re + o + 8, r1[0]);
        atomicAdd(s_re + o + 9, r1[1]);
        atomicAdd(s_re + o + 8 * LD + 8, r1[2]);
        atomicAdd(s_re + o + 8 * LD + 9, r1[3]);
        atomicAdd(s_im + o + 8, i1[0]);
        atomicAdd(s_im + o + 9, i1[1]);
        atomicAdd(s_im + o + 8 * LD + 8, i1[2]);
        atomicAdd(s_im + o + 8 * LD + 9, i1[3]);
#pragma unroll
        for (int q = 0; q < 4; ++q) r0[q] = i0[q] = r1[q] = i1[q] = 0.f;
    };

    // per-warp staging buffers after the accumulator planes (the layout of the column kernel)
    StagedSlot* st_slot = reinterpret_cast<StagedSlot*>(smem + 2 * PR * LD) + warp * kStageSlots;
    int* st_pos = reinterpret_cast<int*>(reinterpret_cast<StagedSlot*>(smem + 2 * PR * LD) +
                                         kWarps * kStageSlots) + warp * kStageSlots;
    uint32_t* st_hdr = reinterpret_cast<uint32_t*>(reinterpret_cast<StagedSlot*>(smem + 2 * PR * LD) +
                                                   kWarps * kStageSlots) +
                       kWarps * kStageSlots + warp * kStageChunks;
    if (ca < cb) {
        // each lane loads one slot of the next kStageChunks chunks; the registers hold the next
        // batch while the current one is computed from shared memory
        const int64_t send = (int64_t)cb * kMmaChunk;
        StagedSlot nxt;
        int npos;
        uint32_t nhdr = 0;
        load_block_slot<VBF, ABF>(cent, vals, (int64_t)ca * kMmaChunk + lane, send, nxt, npos);
        if (lane < kStageChunks) nhdr = chdr[min(ca + lane, cb - 1)];
        for (int cbase = ca; cbase < cb; cbase += kStageChunks) {
            __syncwarp();
            st_slot[lane] = nxt;
            st_pos[lane] = npos;
            if (lane < kStageChunks) st_hdr[lane] = nhdr;
            __syncwarp();
            if (cbase + kStageChunks < cb) {
                load_block_slot<VBF, ABF>(cent, vals,
                                    (int64_t)(cbase + kStageChunks) * kMmaChunk + lane, send, nxt,
                                    npos);
                if (lane < kStageChunks) nhdr = chdr[min(cbase + kStageChunks + lane, cb - 1)];
            }
            const int nk = min(kStageChunks, cb - cbase);
#pragma unroll mma::kBatchUnroll
            for (int k = 0; k < kStageChunks; ++k) {
                if (k >= nk) break;
                const uint32_t h = st_hdr[k];
                const int bx = (int)(h & 0xffu), by = (int)((h >> 8) & 0xffu);
                if (bx != cur_bx || by != cur_by) {    // a new block: flush the last one
                    if (cur_bx >= 0) flush();
                    cur_bx = bx;
                    cur_by = by;
                }
                const StagedSlot e1 = st_slot[k * kMmaChunk + t];
                const StagedSlot e2 = st_slot[k * kMmaChunk + t + 4];
                const int p1 = st_pos[k * kMmaChunk + t], p2 = st_pos[k * kMmaChunk + t + 4];
                const int ox1 = p1 & 7, oy1 = p1 >> 3, ox2 = p2 & 7, oy2 = p2 >> 3;
                // tap g of samples t and t + 4 along x and y; window row (column) g takes tap
                // (g - off) mod 8, held by lane ((g - off) & 7, t), in the lower half when
                // g >= off and in the upper half (row or column g + 8) otherwise
                const float fx1 = mma::horner(cf, e1.sx), fx2 = mma::horner(cf, e2.sx);
                const float fy1 = mma::horner(cf, e1.sy), fy2 = mma::horner(cf, e2.sy);
                const float a1 = __shfl_sync(0xffffffffu, fy1, (((g - oy1) & 7) << 2) | t);
                const float a2 = __shfl_sync(0xffffffffu, fy2, (((g - oy2) & 7) << 2) | t);
                const float x1 = __shfl_sync(0xffffffffu, fx1, (((g - ox1) & 7) << 2) | t);
                const float x2 = __shfl_sync(0xffffffffu, fx2, (((g - ox2) & 7) << 2) | t);
                const bool ly1 = g >= oy1, ly2 = g >= oy2, lx1 = g >= ox1, lx2 = g >= ox2;
                uint32_t a1h, a1l, a2h, a2l;
                mma::split_tf32(a1, a1h, a1l);
                mma::split_tf32(a2, a2h, a2l);
                const uint32_t ah0 = ly1 ? a1h : 0u, ah1 = ly1 ? 0u : a1h;
                const uint32_t ah2 = ly2 ? a2h : 0u, ah3 = ly2 ? 0u : a2h;
                const uint32_t al0 = ly1 ? a1l : 0u, al1 = ly1 ? 0u : a1l;
                const uint32_t al2 = ly2 ? a2l : 0u, al3 = ly2 ? 0u : a2l;
                uint32_t r1h, r1l, j1h, j1l, r2h, r2l, j2h, j2l;
                mma::split_tf32(e1.cr * x1, r1h, r1l);
                mma::split_tf32(e1.ci * x1, j1h, j1l);
                mma::split_tf32(e2.cr * x2, r2h, r2l);
                mma::split_tf32(e2.ci * x2, j2h, j2l);
                const uint32_t m1 = lx1 ? 0xffffffffu : 0u, m2 = lx2 ? 0xffffffffu : 0u;
                // column half 0 (columns g) and half 1 (columns g + 8)
                mma::mma_tf32(r0, ah0, ah1, ah2, ah3, r1h & m1, r2h & m2);
                mma::mma_tf32(i0, ah0, ah1, ah2, ah3, j1h & m1, j2h & m2);
                mma::mma_tf32(r1, ah0, ah1, ah2, ah3, r1h & ~m1, r2h & ~m2);
                mma::mma_tf32(i1, ah0, ah1, ah2, ah3, j1h & ~m1, j2h & ~m2);
                mma::mma_tf32(r0, ah0, ah1, ah2, ah3, r1l & m1, r2l & m2);
                mma::mma_tf32(i0, ah0, ah1, ah2, ah3, j1l & m1, j2l & m2);
                mma::mma_tf32(r1, ah0, ah1, ah2, ah3, r1l & ~m1, r2l & ~m2);
                mma::mma_tf32(i1, ah0, ah1, ah2, ah3, j1l & ~m1, j2l & ~m2);
                mma::mma_tf32(r0, al0, al1, al2, al3, r1h & m1, r2h & m2);
                mma::mma_tf32(i0, al0, al1, al2, al3, j1h & m1, j2h & m2);
                mma::mma_tf32(r1, al0, al1, al2, al3, r1h & ~m1, r2h & ~m2);
                mma::mma_tf32(i1, al0, al1, al2, al3, j1h & ~m1, j2h & ~m2);
            }
        }
        flush();
    }
    __syncthreads();
    tile::store_tile<true, kThreads>(s_re, s_im, LD, grid, G, X0, Y0, Tw, Th, T, W,
                                     halo_buf + (int64_t)tile * halo_cells, halo_cells);
}

}  // namespace blk
}  // namespace ftcg
