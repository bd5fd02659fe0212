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
// FTCG_MMA_UNROLL: 1 unrolls the loop over a staged batch's chunks
#ifndef FTCG_MMA_UNROLL
#define FTCG_MMA_UNROLL 1
#endif
constexpr int kThreads = FTCG_MMA_THREADS;
constexpr int kWarps = kThreads / 32;
constexpr int kMinBlocks = FTCG_MMA_MINB;
constexpr int kBatchUnroll = FTCG_MMA_UNROLL ? 4 : 1;
// padding chunks after the last one (a read past the end stays inside the array)
constexpr int kPrefetchChunks = 1;

// Rows of the tile's accumulator planes: a window starts on a row of the tile (0..T-1) and its
// upper half reaches row T + 14; rows past T + 6 only ever receive zeros, so flushes need no
// bounds test.
__host__ __device__ constexpr int acc_rows(int T) { return T + 2 * kMmaMaxW - 1; }

// Dynamic shared memory of one tile: the two accumulator planes (acc_rows(T) rows of T + 8
// floats), then each warp's staging buffers (32 slots of 16 bytes, 32 row offsets, 4 chunk
// headers).
__host__ __device__ constexpr size_t tile_smem_bytes(int T) {
    return (size_t)2 * acc_rows(T) * (T + kMmaMaxW) * sizeof(float) +
           (size_t)kWarps * (32 * (16 + sizeof(int)) + 4 * sizeof(uint32_t));
}

// x = hi + lo with hi = x rounded to TF32 (10 stored significand bits; the magnitude rounded half
// away from zero by an integer add on the bit pattern) and lo = x - hi, which is exact in FP32
// and at most 2^-11 |x|. The MMA reads lo as TF32 (its low 13 bits ignored), so the pair carries
// x to within 2^-21 |x|.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
    lo = __float_as_uint(x - __uint_as_float(hi));
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

// One staged slot: the chunk slot's offsets within its taps' unit interval and its weighted
// value c = alpha v (zero for padding), 16 bytes; its row offset within the chunk window
// (0..8) is kept beside it.
struct __align__(16) StagedSlot {
    float sx, sy, cr, ci;
};

// Per-warp staging of kStageChunks chunks (kStageChunks * 8 slots, one per lane when 4).
constexpr int kStageChunks = 4;
constexpr int kStageSlots = kStageChunks * kMmaChunk;
static_assert(kStageSlots == 32, "one staged slot per lane");

// Load slot i (a padding slot, or an index past the warp's range, gives c = 0): the slot and its
// sample's value; no branch (padding slots name sample 0, whose value is read and discarded).
template <bool VBF, bool ABF>
__device__ __forceinline__ void load_slot(const MmaEntry* __restrict__ cent,
                                          const void* __restrict__ vals, int64_t i, int64_t end,
                                          StagedSlot& out, int& off) {
    const bool live = i < end;
    const MmaEntry e = cent[live ? i : end - 1];
    const float2 v = tile::load_value<VBF>(vals, e.packed & kSampleMask);
    float al = ABF ? tile::bf16_bits_to_float(e.alpha) : __uint_as_float(e.alpha);
    al = (live && !(e.packed & kMmaPad)) ? al : 0.0f;
    out.sx = e.sx;
    out.sy = e.sy;
    out.cr = al * v.x;
    out.ci = al * v.y;
    off = (int)((e.packed >> kSampleBits) & 15u);
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
    constexpr int PR = acc_rows(T);          // accumulator rows
    constexpr int LD = T + kMmaMaxW;         // row pitch: the tile + overflow columns, + 1
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
    // D fragments: real and imaginary plane, rows g (d[0], d[1]) and g + 8 (d[2], d[3]),
    // columns 2t and 2t + 1; the hi x hi products and the two cross products accumulate
    // separately, so that the MMAs of a chunk do not wait on one another. The window's lower
    // half (rows yb .. yb + 7) lives in D half ph (0: rows g, 1: rows g + 8): a window that moves
    // down by 8 rows flushes and clears that half and flips ph instead of moving registers.
    float dr[4] = {0.f, 0.f, 0.f, 0.f}, di[4] = {0.f, 0.f, 0.f, 0.f};
    float er[4] = {0.f, 0.f, 0.f, 0.f}, ei[4] = {0.f, 0.f, 0.f, 0.f};
    int cur_cx = -1, cur_yb = 0, ph = 0;
    auto flush_d0 = [&](int o) {               // D rows g into the accumulator at offset o
        atomicAdd(s_re + o, dr[0] + er[0]);
        atomicAdd(s_re + o + 1, dr[1] + er[1]);
        atomicAdd(s_im + o, di[0] + ei[0]);
        atomicAdd(s_im + o + 1, di[1] + ei[1]);
        dr[0] = dr[1] = di[0] = di[1] = er[0] = er[1] = ei[0] = ei[1] = 0.f;
    };
    auto flush_d1 = [&](int o) {               // D rows g + 8
        atomicAdd(s_re + o, dr[2] + er[2]);
        atomicAdd(s_re + o + 1, dr[3] + er[3]);
        atomicAdd(s_im + o, di[2] + ei[2]);
        atomicAdd(s_im + o + 1, di[3] + ei[3]);
        dr[2] = dr[3] = di[2] = di[3] = er[2] = er[3] = ei[2] = ei[3] = 0.f;
    };
    auto flush_window = [&]() {                // both halves (window rows cur_yb + g, + 8)
        const int o = (cur_yb + g) * LD + cur_cx + 2 * t;
        if (ph) {
            flush_d1(o);
            flush_d0(o + 8 * LD);
        } else {
            flush_d0(o);
            flush_d1(o + 8 * LD);
        }
    };

    // per-warp staging buffers after the accumulator planes
    StagedSlot* st_slot = reinterpret_cast<StagedSlot*>(smem + 2 * PR * LD) + warp * kStageSlots;
    int* st_off = reinterpret_cast<int*>(reinterpret_cast<StagedSlot*>(smem + 2 * PR * LD) +
                                         kWarps * kStageSlots) + warp * kStageSlots;
    uint32_t* st_hdr = reinterpret_cast<uint32_t*>(reinterpret_cast<StagedSlot*>(smem + 2 * PR * LD) +
                                                   kWarps * kStageSlots) +
                       kWarps * kStageSlots + warp * kStageChunks;
    if (ca < cb) {
        // each lane loads one slot of the next kStageChunks chunks (coalesced 16-byte loads, one
        // value gather per slot); the registers hold the next batch while the current one is
        // computed from shared memory
        const int64_t send = (int64_t)cb * kMmaChunk;
        StagedSlot nxt;
        int noff;
        uint32_t nhdr = 0;
        load_slot<VBF, ABF>(cent, vals, (int64_t)ca * kMmaChunk + lane, send, nxt, noff);
        if (lane < kStageChunks) nhdr = chdr[min(ca + lane, cb - 1)];
        for (int cbase = ca; cbase < cb; cbase += kStageChunks) {
            __syncwarp();
            st_slot[lane] = nxt;
            st_off[lane] = noff;
            if (lane < kStageChunks) st_hdr[lane] = nhdr;
            __syncwarp();
            if (cbase + kStageChunks < cb) {
                load_slot<VBF, ABF>(cent, vals,
                                    (int64_t)(cbase + kStageChunks) * kMmaChunk + lane, send, nxt,
                                    noff);
                if (lane < kStageChunks) nhdr = chdr[min(cbase + kStageChunks + lane, cb - 1)];
            }
            const int nk = min(kStageChunks, cb - cbase);
#pragma unroll kBatchUnroll
            for (int k = 0; k < kStageChunks; ++k) {
                if (k >= nk) break;
                const uint32_t h = st_hdr[k];
                const int cx = (int)(h & 0xffu), yb = (int)((h >> 8) & 0xffu);
                if (cx != cur_cx || (yb != cur_yb && yb != cur_yb + 8)) {   // a new window
                    if (cur_cx >= 0) flush_window();
                    cur_cx = cx;
                    cur_yb = yb;
                    ph = 0;
                } else if (yb != cur_yb) {         // the window moves down by 8 rows
                    const int o = (cur_yb + g) * LD + cur_cx + 2 * t;
                    if (ph) flush_d1(o);
                    else flush_d0(o);
                    ph ^= 1;
                    cur_yb = yb;
                }
                const StagedSlot e1 = st_slot[k * kMmaChunk + t];
                const StagedSlot e2 = st_slot[k * kMmaChunk + t + 4];
                const int off1 = st_off[k * kMmaChunk + t], off2 = st_off[k * kMmaChunk + t + 4];
                // column factor of tap g times the weighted value; row factor of tap g
                const float fx1 = horner(cf, e1.sx), fx2 = horner(cf, e2.sx);
                const float fy1 = horner(cf, e1.sy), fy2 = horner(cf, e2.sy);
                // A[r][k]: window row r = g or g + 8 takes tap (g - off) mod 8 of sample k, held
                // by lane ((g - off) & 7, t) (every lane with the same t evaluates the same
                // samples)
                const float a1 = __shfl_sync(0xffffffffu, fy1, (((g - off1) & 7) << 2) | t);
                const float a2 = __shfl_sync(0xffffffffu, fy2, (((g - off2) & 7) << 2) | t);
                // window row g (lower half) or g + 8, mapped to the D half that holds it
                const bool low1 = (g >= off1) != (ph != 0), low2 = (g >= off2) != (ph != 0);
                uint32_t a1h, a1l, a2h, a2l;
                split_tf32(a1, a1h, a1l);
                split_tf32(a2, a2h, a2l);
                uint32_t b1rh, b1rl, b1ih, b1il, b2rh, b2rl, b2ih, b2il;
                split_tf32(e1.cr * fx1, b1rh, b1rl);
                split_tf32(e1.ci * fx1, b1ih, b1il);
                split_tf32(e2.cr * fx2, b2rh, b2rl);
                split_tf32(e2.ci * fx2, b2ih, b2il);
                const uint32_t ah0 = low1 ? a1h : 0u, ah1 = low1 ? 0u : a1h;
                const uint32_t ah2 = low2 ? a2h : 0u, ah3 = low2 ? 0u : a2h;
                const uint32_t al0 = low1 ? a1l : 0u, al1 = low1 ? 0u : a1l;
                const uint32_t al2 = low2 ? a2l : 0u, al3 = low2 ? 0u : a2l;
                mma_tf32(dr, ah0, ah1, ah2, ah3, b1rh, b2rh);
                mma_tf32(di, ah0, ah1, ah2, ah3, b1ih, b2ih);
                mma_tf32(er, ah0, ah1, ah2, ah3, b1rl, b2rl);
                mma_tf32(ei, ah0, ah1, ah2, ah3, b1il, b2il);
                mma_tf32(er, al0, al1, al2, al3, b1rh, b2rh);
                mma_tf32(ei, al0, al1, al2, al3, b1ih, b2ih);
            }
        }
        flush_window();
    }
    __syncthreads();
    tile::store_tile<true, kThreads>(s_re, s_im, LD, grid, G, X0, Y0, Tw, Th, T, W,
                                     halo_buf + (int64_t)tile * halo_cells, halo_cells);
}

}  // namespace mma
}  // namespace ftcg
