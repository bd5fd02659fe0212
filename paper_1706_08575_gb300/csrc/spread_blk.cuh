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
// taps. Window row r and row r + 8 take the same tap index mod 8, so a lane holds one tap value
// per sample and dimension and it belongs to exactly one of the two rows (columns). Only the
// lower rows of A and the left half of B are masked: the upper rows carry the tap whichever row
// it belongs to, and so does the right half of B. The MMAs then accumulate the partial sums
//   S00 = q00,  S10 = q00 + q10,  S01 = q00 + q01,  S11 = q00 + q10 + q01 + q11
// of the window's four 8 x 8 quadrants q (rows, columns), which the flush turns back into the
// quadrants by differences; 12 split-TF32 mma.sync.m16n8k8 per chunk (3 products x 2 planes x 2
// halves) with half the operand masking. The chunks of a block follow one another and share the
// window, which stays in the D fragments until the block changes; then its 16 x 16 cells are
// added to the tile's shared accumulator. There is no window to shift: the bookkeeping per chunk
// is one comparison.
#pragma once

#include "spread_mma.cuh"

namespace ftcg {
namespace blk {

using mma::kThreads;
using mma::kWarps;
using mma::StagedSlot;
using mma::kStageChunks;
using mma::kStageSlots;

// Dynamic shared memory of one tile: the column kernel's (accumulator planes, staging buffers),
// then the tap polynomials (8 x 8 floats).
__host__ __device__ constexpr size_t tile_smem_bytes(int T) {
    return mma::tile_smem_bytes(T) + (size_t)kMmaMaxW * (kMmaDeg + 1) * sizeof(float);
}

// Bits of a block chunk slot's packed word: sample index (kSampleBits), then the first tap's
// column and row within the block (3 bits each), then the padding flag (kMmaPad).
constexpr int kOffXShift = kSampleBits;
constexpr int kOffYShift = kSampleBits + 3;

// Load slot i of the chunk array (a padding slot, or an index past the warp's range, gives
// c = 0): its offsets, weighted value, and its first tap's place in the block as
// q = 4 offx | (4 offy) << 16, so that (lane + 32) * 0x10001 - q holds lane - 4 offx + 32 in its
// low half and lane - 4 offy + 32 in its high half, both in 4..63 (no borrow between the halves).
template <bool VBF, bool ABF>
__device__ __forceinline__ void load_block_slot(const MmaEntry* __restrict__ cent,
                                                const void* __restrict__ vals, int64_t i,
                                                int64_t end, StagedSlot& out, uint32_t& q) {
    const bool live = i < end;
    const MmaEntry e = cent[live ? i : end - 1];
    const float2 v = tile::load_value<VBF>(vals, e.packed & kSampleMask);
    float al = ABF ? tile::bf16_bits_to_float(e.alpha) : __uint_as_float(e.alpha);
    al = (live && !(e.packed & kMmaPad)) ? al : 0.0f;
    out.sx = e.sx;
    out.sy = e.sy;
    out.cr = al * v.x;
    out.ci = al * v.y;
    q = (((e.packed >> kOffXShift) & 7u) << 2) | (((e.packed >> kOffYShift) & 7u) << 18);
}

// One halo-layout tile by the whole CTA (kThreads threads): its block chunks
// [tile_chunk[tile], tile_chunk[tile + 1]) split into contiguous ranges, one per warp; then the
// tile and its overflow strips are stored. smem: blk::tile_smem_bytes(T).
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
    // the tap polynomials after the staging buffers; read per chunk (asm volatile, so that they
    // are not hoisted into 8 more live registers, which would spill at 80 per thread)
    float* s_cf = smem + 2 * PR * LD + kWarps * (kStageSlots * 5 + kStageChunks);
    if (threadIdx.x < kMmaMaxW * (kMmaDeg + 1))
        s_cf[threadIdx.x] = poly.c[threadIdx.x >> 3][threadIdx.x & 7];
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;     // MMA fragment row group and column pair
    const uint32_t cf_addr = (uint32_t)__cvta_generic_to_shared(s_cf + 8 * g);   // tap g's
    const int n = c1 - c0;
    const int ca = c0 + (int)((int64_t)n * warp / kWarps);
    const int cb = c0 + (int)((int64_t)n * (warp + 1) / kWarps);
    // D fragments of the two column halves, real and imaginary plane: rows g (d[0], d[1]) and
    // g + 8 (d[2], d[3]), columns 8h + 2t and 8h + 2t + 1; they hold the partial sums S (rows
    // g + 8: S1x, half 1: Sx1)
    float r0[4] = {0.f, 0.f, 0.f, 0.f}, i0[4] = {0.f, 0.f, 0.f, 0.f};
    float r1[4] = {0.f, 0.f, 0.f, 0.f}, i1[4] = {0.f, 0.f, 0.f, 0.f};
    uint32_t cur = 0xffffffffu;                // the block in the fragments (its header)
    // one plane's window quadrants from its partial sums, added to the accumulator at o
    auto flush_plane = [&](float* acc, int o, float (&d0)[4], float (&d1)[4]) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float q10 = d0[2 + j] - d0[j];
            atomicAdd(acc + o + j, d0[j]);
            atomicAdd(acc + o + 8 * LD + j, q10);
            atomicAdd(acc + o + 8 + j, d1[j] - d0[j]);
            atomicAdd(acc + o + 8 * LD + 8 + j, (d1[2 + j] - d1[j]) - q10);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) d0[q] = d1[q] = 0.f;
    };
    auto flush = [&]() {
        const int o = ((int)(cur >> 8) + g) * LD + (int)(cur & 0xffu) + 2 * t;
        flush_plane(s_re, o, r0, r1);
        flush_plane(s_im, o, i0, i1);
    };
    // (lane + 32) in both halves: minus a slot's q, the shuffle source lanes (mod 32) of its
    // taps and, in bit 5 of each half, whether this lane's row (column) g is at or after the
    // first tap's
    const uint32_t lane2 = (uint32_t)(lane + 32) * 0x10001u;

    // per-warp staging buffers after the accumulator planes (the layout of the column kernel)
    StagedSlot* st_slot = reinterpret_cast<StagedSlot*>(smem + 2 * PR * LD) + warp * kStageSlots;
    uint32_t* st_pos = reinterpret_cast<uint32_t*>(reinterpret_cast<StagedSlot*>(smem + 2 * PR * LD) +
                                                   kWarps * kStageSlots) + warp * kStageSlots;
    uint32_t* st_hdr = reinterpret_cast<uint32_t*>(reinterpret_cast<StagedSlot*>(smem + 2 * PR * LD) +
                                                   kWarps * kStageSlots) +
                       kWarps * kStageSlots + warp * kStageChunks;
    if (ca < cb) {
        // each lane loads one slot of the next kStageChunks chunks; the registers hold the next
        // batch while the current one is computed from shared memory
        const int64_t send = (int64_t)cb * kMmaChunk;
        StagedSlot nxt;
        uint32_t npos;
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
                if (h != cur) {                        // a new block: flush the last one
                    if (cur != 0xffffffffu) flush();
                    cur = h;
                }
                const StagedSlot e1 = st_slot[k * kMmaChunk + t];
                const StagedSlot e2 = st_slot[k * kMmaChunk + t + 4];
                const uint32_t d1 = lane2 - st_pos[k * kMmaChunk + t];
                const uint32_t d2 = lane2 - st_pos[k * kMmaChunk + t + 4];
                // tap g of samples t and t + 4 along x and y; window row (column) g takes tap
                // (g - off) mod 8, held by lane ((g - off) & 7, t): the low 5 bits of d's halves
                float cf[kMmaDeg + 1];
                asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                             : "=f"(cf[0]), "=f"(cf[1]), "=f"(cf[2]), "=f"(cf[3]) : "r"(cf_addr));
                asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                             : "=f"(cf[4]), "=f"(cf[5]), "=f"(cf[6]), "=f"(cf[7]) : "r"(cf_addr + 16));
                const float fx1 = mma::horner(cf, e1.sx), fx2 = mma::horner(cf, e2.sx);
                const float fy1 = mma::horner(cf, e1.sy), fy2 = mma::horner(cf, e2.sy);
                const float a1 = __shfl_sync(0xffffffffu, fy1, (int)(d1 >> 16));
                const float a2 = __shfl_sync(0xffffffffu, fy2, (int)(d2 >> 16));
                const float x1 = __shfl_sync(0xffffffffu, fx1, (int)d1);
                const float x2 = __shfl_sync(0xffffffffu, fx2, (int)d2);
                // the tap is in row (column) g when g >= off, else in g + 8
                const bool ly1 = d1 & 0x200000u, ly2 = d2 & 0x200000u;
                const uint32_t m1 = (d1 & 0x20u) ? 0xffffffffu : 0u;
                const uint32_t m2 = (d2 & 0x20u) ? 0xffffffffu : 0u;
                uint32_t a1h, a1l, a2h, a2l;
                mma::split_tf32(a1, a1h, a1l);
                mma::split_tf32(a2, a2h, a2l);
                // rows g masked, rows g + 8 unmasked (partial sums S1x)
                const uint32_t ah0 = ly1 ? a1h : 0u, ah2 = ly2 ? a2h : 0u;
                const uint32_t al0 = ly1 ? a1l : 0u, al2 = ly2 ? a2l : 0u;
                uint32_t r1h, r1l, j1h, j1l, r2h, r2l, j2h, j2l;
                mma::split_tf32(e1.cr * x1, r1h, r1l);
                mma::split_tf32(e1.ci * x1, j1h, j1l);
                mma::split_tf32(e2.cr * x2, r2h, r2l);
                mma::split_tf32(e2.ci * x2, j2h, j2l);
                // column half 0 masked, half 1 unmasked (partial sums Sx1)
                mma::mma_tf32(r0, ah0, a1h, ah2, a2h, r1h & m1, r2h & m2);
                mma::mma_tf32(i0, ah0, a1h, ah2, a2h, j1h & m1, j2h & m2);
                mma::mma_tf32(r1, ah0, a1h, ah2, a2h, r1h, r2h);
                mma::mma_tf32(i1, ah0, a1h, ah2, a2h, j1h, j2h);
                mma::mma_tf32(r0, ah0, a1h, ah2, a2h, r1l & m1, r2l & m2);
                mma::mma_tf32(i0, ah0, a1h, ah2, a2h, j1l & m1, j2l & m2);
                mma::mma_tf32(r1, ah0, a1h, ah2, a2h, r1l, r2l);
                mma::mma_tf32(i1, ah0, a1h, ah2, a2h, j1l, j2l);
                mma::mma_tf32(r0, al0, a1l, al2, a2l, r1h & m1, r2h & m2);
                mma::mma_tf32(i0, al0, a1l, al2, a2l, j1h & m1, j2h & m2);
                mma::mma_tf32(r1, al0, a1l, al2, a2l, r1h, r2h);
                mma::mma_tf32(i1, al0, a1l, al2, a2l, j1h, j2h);
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
