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

// Raw chunk slots in flight per warp: two batches of kStageSlots entries (16 bytes) and of
// kStageChunks headers, filled by cp.async one batch ahead of their staging.
constexpr int kRawStages = 2;

// Dynamic shared memory of one tile: the column kernel's (accumulator planes, staging buffers),
// then the tap polynomials (8 x 8 floats), then each warp's raw entries and headers.
__host__ __device__ constexpr size_t tile_smem_bytes(int T) {
    return mma::tile_smem_bytes(T) + (size_t)kMmaMaxW * (kMmaDeg + 1) * sizeof(float) +
           (size_t)kWarps * kRawStages * (kStageSlots * sizeof(MmaEntry) +
                                          kStageChunks * sizeof(uint32_t));
}

// Asynchronous global -> shared copies (cp.async): 16 bytes, of which the first n come from src
// and the rest are zero (n = 0 reads nothing); 4 bytes; commit; wait for all of this thread's.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t n) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(__cvta_generic_to_global(src)), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Bits of a block chunk slot's packed word: sample index (kSampleBits), then the first tap's
// column and row within the block (3 bits each), then the padding flag (kMmaPad).
constexpr int kOffXShift = kSampleBits;
constexpr int kOffYShift = kSampleBits + 3;

// The staged form of raw slot e with its value v (in_range: the slot lies within the warp's
// chunks): its offsets, c = alpha v (zero for a padding slot or past the end), and
// its first tap's place in the block as q = 4 offx | (4 offy) << 16, so that
// (lane + 32) * 0x10001 - q holds lane - 4 offx + 32 in its low half and lane - 4 offy + 32 in
// its high half, both in 4..63 (no borrow between the halves).
template <bool ABF>
__device__ __forceinline__ void stage_block_slot(const MmaEntry& e, float2 v, bool in_range,
                                                 StagedSlot& out, uint32_t& q) {
    const float al = ABF ? tile::bf16_bits_to_float(e.alpha) : __uint_as_float(e.alpha);
    const bool live = in_range && !(e.packed & kMmaPad);
    out.sx = e.sx;
    out.sy = e.sy;
    out.cr = live ? al * v.x : 0.0f;
    out.ci = live ? al * v.y : 0.0f;
    q = (((e.packed >> kOffXShift) & 7u) << 2) | (((e.packed >> kOffYShift) & 7u) << 18);
}

// One halo-layout tile by the whole CTA (kThreads threads): its block chunks
// [tile_chunk[tile], tile_chunk[tile + 1]) split into contiguous ranges, one per warp (or all to
// warp 0 with one_warp); then the tile and its overflow strips are stored. smem: blk::tile_smem_bytes(T).
template <int T, bool VBF, bool ABF>
__device__ __forceinline__ void spread_tile(const MmaEntry* __restrict__ cent,
                                            const uint32_t* __restrict__ chdr,
                                            const int* __restrict__ tile_chunk,
                                            const void* __restrict__ vals,
                                            float2* __restrict__ grid, int G, int ntx, int W,
                                            const MmaPoly& poly, float2* __restrict__ halo_buf,
                                            int halo_cells, int tile, float* smem,
                                            bool one_warp = false) {
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
    // each warp a contiguous range of the tile's chunks; one_warp (deterministic plans): warp 0
    // takes them all, in plan order
    const int ca = one_warp ? (warp == 0 ? c0 : c1) : c0 + (int)((int64_t)n * warp / kWarps);
    const int cb = one_warp ? c1 : c0 + (int)((int64_t)n * (warp + 1) / kWarps);
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
    // then, after the tap polynomials, each warp's raw slots and headers (kRawStages batches)
    MmaEntry* raw_all = reinterpret_cast<MmaEntry*>(s_cf + kMmaMaxW * (kMmaDeg + 1));
    MmaEntry* raw = raw_all + warp * kRawStages * kStageSlots;
    uint32_t* raw_hdr = reinterpret_cast<uint32_t*>(raw_all + kWarps * kRawStages * kStageSlots) +
                        warp * kRawStages * kStageChunks;
    if (ca < cb) {
        // batch j: chunks ca + 4j .. ca + 4j + 3, one slot per lane. Its raw slots and headers
        // are copied by cp.async two batches ahead; the value gather of batch j + 1 is issued
        // before batch j is computed and staged after it, so that after the first batch neither
        // load is waited for.
        // this lane's slot of batch 0, and how many of the warp's slots remain from it (batch j's
        // slot is live while 32 j < left; past the end the copy reads nothing and fills zeros)
        const MmaEntry* src = cent + (int64_t)ca * kMmaChunk + lane;
        const int left = (cb - ca) * kMmaChunk - lane;
        const uint32_t* hsrc = chdr + ca;
        const int nb = (cb - ca + kStageChunks - 1) / kStageChunks;
        auto issue = [&](int j) {                // batch j's copies into ring stage j & 1
            const int o = kStageSlots * j;
            cp_async16(raw + (j & 1) * kStageSlots + lane, src + min(o, left - 1),
                       o < left ? 16u : 0u);
            if (lane < kStageChunks)
                cp_async4(raw_hdr + (j & 1) * kStageChunks + lane,
                          hsrc + min(kStageChunks * j + lane, cb - ca - 1));
            cp_async_commit();
        };
        auto stage = [&](int j, float2 v) {      // batch j from its ring stage, with values v
            const MmaEntry e = raw[(j & 1) * kStageSlots + lane];
            StagedSlot sl;
            uint32_t q;
            stage_block_slot<ABF>(e, v, kStageSlots * j < left, sl, q);
            st_slot[lane] = sl;
            st_pos[lane] = q;
            if (lane < kStageChunks) st_hdr[lane] = raw_hdr[(j & 1) * kStageChunks + lane];
        };
        issue(0);
        if (nb > 1) issue(1);
        cp_async_wait_all();
        __syncwarp();
        stage(0, tile::load_value<VBF>(vals, raw[lane].packed & kSampleMask));
        __syncwarp();
        for (int j = 0; j < nb; ++j) {
            const bool more = j + 1 < nb;
            float2 v = make_float2(0.0f, 0.0f);
            if (more) {
                cp_async_wait_all();               // batch j + 1's raw slots (this lane's)
                v = tile::load_value<VBF>(
                    vals, raw[((j + 1) & 1) * kStageSlots + lane].packed & kSampleMask);
                if (j + 2 < nb) issue(j + 2);      // into batch j's stage, staged already
            }
            const int nk = min(kStageChunks, cb - (ca + kStageChunks * j));
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
            if (more) {
                __syncwarp();                      // every lane is done with batch j's slots
                stage(j + 1, v);
                __syncwarp();
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
