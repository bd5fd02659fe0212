// Spreading on the tensor cores (Omega_2 D_2 f^, Eq. twodcgmatrix), halo layout, w <= 8.
//
// The spreading sum of one column bin (samples whose first tap lies in one column cx of a tile)
// over a window of 16 grid rows starting at row yb is a matrix product:
//
//   g[yb + r][cx + n] += sum_k  phi(dy_k - (r - off_k)) * (alpha_k v_k phi(dx_k - n)),
//                               `-------- A[r][k] ------'   `------- B[k][n] ---------'
//
// with r in 0..15 (A is zero outside the sample's w rows r = off_k .. off_k + w - 1, off_k =
// first-tap row - yb in 0..8), n in 0..7 the tap columns and k over 8 samples: one
// mma.sync.m16n8k8 per output plane (real and imaginary part of B). The products run in TF32
// with both operands split into a high and a low TF32 part (a = a_hi + a_lo with |a_lo| <=
// 2^-11 |a|, keeping three of the four cross products), which keeps the FP32 image accuracy.
//
// The plan regroups each tile's sorted entries into chunks of 8 samples of one column bin that
// fit one window position (first-tap rows within yb .. yb + 8), padding the last chunk of a
// window with flagged empty slots; consecutive windows of a bin move down by 8 rows, so that the
// window's accumulator, held in the MMA's D fragments, only ever loses its lower half (that half
// is flushed and cleared, and the two D halves swap roles: the A operands are routed to the
// half that holds each window row, so no register moves). Each
// warp of the tile's CTA takes a contiguous range of chunks; windows that are left or shifted
// are added to the tile's shared accumulator with shared-memory atomics, and the tile is stored
// once (coalesced) with its halo strips, exactly as the register-window kernel does.
//
// The block kernel (FTCG_SPREAD_BLOCK; tile body in spread_blk.cuh) groups the samples by the
// 8 x 8 block of cells their first taps lie in instead of by column bin: a chunk of up to 8 of
// them spreads into the 16 x 16 cells from the block's origin, two column halves of 16 x 8, and
// the window stays put for all of the block's chunks (no shifts, one flush per block and warp).
// Its chunks are built here as well (k_blk_count, k_blk_emit).
//
// The window values are evaluated as per-tap degree-7 polynomials in s (the sample's offset
// within the tap's unit interval), fitted on the host by Chebyshev interpolation of the FP64
// window; the fit error is checked when the plan is built (the path is used only when it is
// below 1e-6 of the window's peak).

#include <algorithm>
#include <cmath>
#include <cstring>

#include "spread_blk.cuh"
#include "spread_mma.cuh"

namespace ftcg {

namespace {

constexpr double kMmaPolyBound = 1e-6;

}  // namespace

// Chebyshev interpolation of phi(s + w/2 - 1/2 - l) on s in [-1/2, 1/2] at the 8 Chebyshev
// points (phi the plan's window, in FP64), converted to monomial coefficients in s. The error is
// measured on 257 points per tap.
bool mma_window_poly(int W, double beta, int kind, MmaPoly* out, double* max_err) {
    std::memset(out, 0, sizeof(*out));
    *max_err = 0.0;
    if (W > kMmaMaxW || W < 2) {
        *max_err = INFINITY;
        return false;
    }
    constexpr int n = kMmaDeg + 1;
    double worst = 0.0;
    for (int l = 0; l < W; ++l) {
        const double shift = 0.5 * W - 0.5 - l;
        double f[n], y[n];
        for (int k = 0; k < n; ++k) {
            y[k] = std::cos(M_PI * (k + 0.5) / n);     // in [-1, 1], s = y / 2
            f[k] = window64(0.5 * y[k] + shift, W, beta, kind);
        }
        // Chebyshev coefficients in y
        double cheb[n];
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += f[k] * std::cos(M_PI * j * (k + 0.5) / n);
            cheb[j] = acc * (j == 0 ? 1.0 : 2.0) / n;
        }
        // monomials in y: sum_j cheb[j] T_j(y), T_{j+1} = 2 y T_j - T_{j-1}
        double mono[n] = {0}, tm1[n] = {0}, t0[n] = {0}, t1[n] = {0};
        t0[0] = 1.0;                                   // T_0
        for (int j = 0; j < n; ++j) {
            const double* tj = j == 0 ? t0 : t1;
            if (j == 1) {
                std::memset(t1, 0, sizeof(t1));
                t1[1] = 1.0;                           // T_1
                tj = t1;
                std::memcpy(tm1, t0, sizeof(t0));
            } else if (j >= 2) {
                double nx[n] = {0};
                for (int k = 0; k + 1 < n; ++k) nx[k + 1] += 2.0 * t1[k];
                for (int k = 0; k < n; ++k) nx[k] -= tm1[k];
                std::memcpy(tm1, t1, sizeof(t1));
                std::memcpy(t1, nx, sizeof(nx));
                tj = t1;
            }
            for (int k = 0; k < n; ++k) mono[k] += cheb[j] * tj[k];
        }
        // y = 2 s
        double c[n];
        for (int k = 0; k < n; ++k) c[k] = mono[k] * std::ldexp(1.0, k);
        for (int k = 0; k < n; ++k) out->c[l][k] = (float)c[k];
        for (int i = 0; i <= 256; ++i) {
            const double s = -0.5 + i / 256.0;
            double p = c[n - 1];
            for (int k = n - 2; k >= 0; --k) p = p * s + c[k];
            worst = std::max(worst, std::fabs(p - window64(s + shift, W, beta, kind)));
        }
    }
    *max_err = worst;
    return worst <= kMmaPolyBound;
}

namespace {

// ---- chunk construction (plan time) ----------------------------------------------------------
// The greedy walk over one (tile, column bin) segment, entries sorted by first-tap row r:
// a window starts at the first row; a chunk takes up to 8 following entries with r <= yb + 8;
// an entry beyond yb + 8 but within yb + 16 moves the window down by 8, one beyond starts a new
// window at its own row.
struct ChunkWalk {
    int yb = -1;
    __device__ __forceinline__ int next(const Entry* __restrict__ e, int i, int n, int W, int* ybo) {
        const int r0 = (int)(e[i].packed >> kSampleBits) - (W - 1);
        if (yb < 0 || r0 > yb + 16) yb = r0;
        else if (r0 > yb + 8) yb += 8;
        int j = i;
        while (j < n && j - i < kMmaChunk &&
               (int)(e[j].packed >> kSampleBits) - (W - 1) <= yb + 8)
            ++j;
        *ybo = yb;
        return j;
    }
};

__global__ void k_chunk_count(const Entry* __restrict__ ent, const int* __restrict__ colptr,
                              int64_t nseg, int W, int* __restrict__ cnt) {
    for (int64_t sgi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sgi < nseg;
         sgi += (int64_t)gridDim.x * blockDim.x) {
        const int a = colptr[sgi], n = colptr[sgi + 1] - a;
        ChunkWalk wk;
        int c = 0, yb;
        for (int i = 0; i < n;) {
            i = wk.next(ent + a, i, n, W, &yb);
            ++c;
        }
        cnt[sgi] = c;
    }
}

__global__ void k_chunk_emit(const Entry* __restrict__ ent, const int* __restrict__ colptr,
                             const int* __restrict__ off, int64_t nseg, int ncb, int W,
                             MmaEntry* __restrict__ cent, uint32_t* __restrict__ chdr) {
    const float c0 = 0.5f * W - 0.5f;
    for (int64_t sgi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sgi < nseg;
         sgi += (int64_t)gridDim.x * blockDim.x) {
        const int a = colptr[sgi], n = colptr[sgi + 1] - a;
        if (n == 0) continue;
        const int cx = (int)(sgi % ncb) - (W - 1);     // local first-tap column (halo: >= 0)
        int64_t c = off[sgi];
        ChunkWalk wk;
        int yb;
        for (int i = 0; i < n; ++c) {
            const int j = wk.next(ent + a, i, n, W, &yb);
            chdr[c] = (uint32_t)cx | ((uint32_t)yb << 8);
            for (int k = 0; k < kMmaChunk; ++k) {
                MmaEntry m;
                if (i + k < j) {
                    const Entry e = ent[a + i + k];
                    const int r = (int)(e.packed >> kSampleBits) - (W - 1);
                    m.sx = e.dx - c0;                  // exact (Sterbenz: dx within c0 +- 1/2)
                    m.sy = e.dy - c0;
                    m.alpha = e.alpha;
                    m.packed = (e.packed & kSampleMask) | ((uint32_t)(r - yb) << kSampleBits);
                } else {
                    m.sx = m.sy = 0.0f;
                    m.alpha = 0u;
                    m.packed = kMmaPad;
                }
                cent[c * kMmaChunk + k] = m;
            }
            i = j;
        }
    }
}

__global__ void k_pad_chunks(MmaEntry* __restrict__ slots, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) slots[i] = MmaEntry{0.f, 0.f, 0u, kMmaPad};
}

// tile_chunk[t] = off[t * ncb], tile_chunk[ntiles] = total
__global__ void k_tile_chunk(const int* __restrict__ off, int ntiles, int ncb, int total,
                             int* __restrict__ tile_chunk) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= ntiles; t += gridDim.x * blockDim.x)
        tile_chunk[t] = t < ntiles ? off[(int64_t)t * ncb] : total;
}

// ---- the tensor-core spreading kernel: one CTA per tile (heaviest first) -----------------------
template <int T, bool VBF, bool ABF>
__global__ void __launch_bounds__(mma::kThreads, mma::kMinBlocks)
    k_spread_mma(const MmaEntry* __restrict__ cent, const uint32_t* __restrict__ chdr,
                 const int* __restrict__ tile_chunk, const int* __restrict__ tile_order,
                 const void* __restrict__ vals, float2* __restrict__ grid, int G, int ntx, int W,
                 const __grid_constant__ MmaPoly poly, float2* __restrict__ halo_buf,
                 int halo_cells) {
    extern __shared__ float smem[];
    pdl_allow_next();                          // the fix-up may be scheduled during the tail
    mma::spread_tile<T, VBF, ABF>(cent, chdr, tile_chunk, vals, grid, G, ntx, W, poly, halo_buf,
                                  halo_cells, tile_order[blockIdx.x], smem);
}

__global__ void k_set_alpha_mma(MmaEntry* __restrict__ cent, int64_t n,
                                const void* __restrict__ alpha, int dtype, bool bf16) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t pk = cent[i].packed;
        if (pk & kMmaPad) continue;                    // padding slots keep alpha = 0
        const uint32_t j = pk & kSampleMask;
        float a = 1.0f;
        if (alpha) {
            a = dtype == FTCG_WEIGHTS_F64 ? (float)reinterpret_cast<const double*>(alpha)[j]
                                          : reinterpret_cast<const float*>(alpha)[j];
        }
        cent[i].alpha = bf16 ? (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) << 16
                             : __float_as_uint(a);
    }
}

int blocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

template <int T, bool VBF, bool ABF>
ftcg_status_t run_mma(const Plan& p, const void* vals, float2* grid, cudaStream_t s, int nt) {
    const Binning& b = p.bin;
    const size_t smem = mma::tile_smem_bytes(T);
    auto kern = k_spread_mma<T, VBF, ABF>;
    FTCG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FTCG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared));
    kern<<<nt, mma::kThreads, smem, s>>>(b.cent, b.chdr, b.tile_chunk, b.tile_order, vals, grid,
                                       b.G, b.ntx, b.W, b.poly, b.halo_buf, b.halo_cells);
    FTCG_CK(cudaGetLastError());
    return launch_halo_add(p, grid, s);
}

template <bool VBF, bool ABF>
ftcg_status_t dispatch_mma_t(const Plan& p, const void* vals, float2* grid, cudaStream_t s,
                             int nt) {
    if (p.bin.T == 32) return run_mma<32, VBF, ABF>(p, vals, grid, s, nt);
    return run_mma<64, VBF, ABF>(p, vals, grid, s, nt);
}

// ---- block chunks (plan time): one thread per (tile, 8 x 8 block of first-tap cells) ----------
// The block's entries are those of its 8 column bins (halo layout: bin = first-tap column + w - 1)
// whose first-tap row lies in the block's 8 rows, taken bin by bin in row order (deterministic).
__device__ __forceinline__ int blk_row(const Entry& e, int W) {
    return (int)(e.packed >> kSampleBits) - (W - 1);
}

__global__ void k_blk_count(const Entry* __restrict__ ent, const int* __restrict__ colptr,
                            int ntiles, int ncb, int T, int W, int* __restrict__ cnt) {
    const int nbs = T / 8, nb = nbs * nbs;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)ntiles * nb;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t tile = i / nb;
        const int b = (int)(i - tile * nb), bxi = b % nbs, byi = b / nbs;
        int c = 0;
        for (int bin = 8 * bxi + W - 1; bin < 8 * bxi + 8 + W - 1 && bin < ncb; ++bin) {
            const int a0 = colptr[tile * ncb + bin], a1 = colptr[tile * ncb + bin + 1];
            for (int e = a0; e < a1; ++e) c += (blk_row(ent[e], W) >> 3) == byi;
        }
        cnt[i] = (c + kMmaChunk - 1) / kMmaChunk;
    }
}

__global__ void k_blk_emit(const Entry* __restrict__ ent, const int* __restrict__ colptr,
                           const int* __restrict__ off, int ntiles, int ncb, int T, int W,
                           MmaEntry* __restrict__ cent, uint32_t* __restrict__ chdr) {
    const int nbs = T / 8, nb = nbs * nbs;
    const float c0 = 0.5f * W - 0.5f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)ntiles * nb;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t tile = i / nb;
        const int b = (int)(i - tile * nb), bxi = b % nbs, byi = b / nbs;
        const int64_t first = off[i];
        int64_t k = 0;
        for (int bin = 8 * bxi + W - 1; bin < 8 * bxi + 8 + W - 1 && bin < ncb; ++bin) {
            const int a0 = colptr[tile * ncb + bin], a1 = colptr[tile * ncb + bin + 1];
            const int ox = bin - (W - 1) - 8 * bxi;              // first-tap column in the block
            for (int e = a0; e < a1; ++e) {
                const Entry en = ent[e];
                const int r = blk_row(en, W);
                if ((r >> 3) != byi) continue;
                MmaEntry m;
                m.sx = en.dx - c0;                              // as the column chunks
                m.sy = en.dy - c0;
                m.alpha = en.alpha;
                m.packed = (en.packed & kSampleMask) | ((uint32_t)ox << blk::kOffXShift) |
                           ((uint32_t)(r - 8 * byi) << blk::kOffYShift);
                cent[first * kMmaChunk + k] = m;
                ++k;
            }
        }
        const int64_t nch = (k + kMmaChunk - 1) / kMmaChunk;
        for (; k < nch * kMmaChunk; ++k) cent[first * kMmaChunk + k] = MmaEntry{0.f, 0.f, 0u, kMmaPad};
        for (int64_t c = 0; c < nch; ++c)
            chdr[first + c] = (uint32_t)(8 * bxi) | ((uint32_t)(8 * byi) << 8);
    }
}

template <int T, bool VBF, bool ABF>
__global__ void __launch_bounds__(mma::kThreads, mma::kMinBlocks)
    k_spread_blk(const MmaEntry* __restrict__ cent, const uint32_t* __restrict__ chdr,
                 const int* __restrict__ tile_chunk, const int* __restrict__ tile_order,
                 const void* __restrict__ vals, float2* __restrict__ grid, int G, int ntx, int W,
                 const __grid_constant__ MmaPoly poly, float2* __restrict__ halo_buf,
                 int halo_cells, bool one_warp) {
    extern __shared__ float smem[];
    pdl_allow_next();                          // the fix-up may be scheduled during the tail
    blk::spread_tile<T, VBF, ABF>(cent, chdr, tile_chunk, vals, grid, G, ntx, W, poly, halo_buf,
                                  halo_cells, tile_order[blockIdx.x], smem, one_warp);
}

template <int T, bool VBF, bool ABF>
ftcg_status_t run_blk(const Plan& p, const void* vals, float2* grid, cudaStream_t s, int nt) {
    const Binning& b = p.bin;
    const size_t smem = blk::tile_smem_bytes(T);
    auto kern = k_spread_blk<T, VBF, ABF>;
    FTCG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FTCG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared));
    kern<<<nt, mma::kThreads, smem, s>>>(b.cent, b.chdr, b.tile_chunk, b.tile_order, vals, grid,
                                       b.G, b.ntx, b.W, b.poly, b.halo_buf, b.halo_cells, b.det);
    FTCG_CK(cudaGetLastError());
    return b.det ? launch_halo_gather(p, grid, s, nt) : launch_halo_add(p, grid, s);
}

template <bool VBF, bool ABF>
ftcg_status_t dispatch_blk_t(const Plan& p, const void* vals, float2* grid, cudaStream_t s,
                             int nt) {
    if (p.bin.T == 32) return run_blk<32, VBF, ABF>(p, vals, grid, s, nt);
    return run_blk<64, VBF, ABF>(p, vals, grid, s, nt);
}

}  // namespace

void free_chunks(Binning& b) {
    if (b.cent) cudaFree(b.cent);
    if (b.chdr) cudaFree(b.chdr);
    if (b.tile_chunk) cudaFree(b.tile_chunk);
    b.cent = nullptr;
    b.chdr = nullptr;
    b.tile_chunk = nullptr;
    b.n_chunks = 0;
    b.mma = false;
    b.blk = false;
}

ftcg_status_t build_chunks(Binning& b, cudaStream_t s, int64_t* bytes, bool block) {
    if (!b.halo || b.W > kMmaMaxW || (b.T != 32 && b.T != 64)) {
        set_error("build_chunks: the tensor-core path needs the halo layout, w <= 8, T = 32 or 64");
        return FTCG_ERR_NOT_SUPPORTED;
    }
    b.blk = block;
    // segments: (tile, column bin) for column chunks, (tile, 8 x 8 block) for block chunks
    const int per_tile = block ? (b.T / 8) * (b.T / 8) : b.ncb;
    const int64_t nseg = (int64_t)b.ntiles * per_tile;
    FTCG_CK(pool_malloc(&b.tile_chunk, (b.ntiles + 1) * sizeof(int), s));
    *bytes += (b.ntiles + 1) * sizeof(int);
    if (b.n_entries == 0) {
        FTCG_CK(cudaMemsetAsync(b.tile_chunk, 0, (b.ntiles + 1) * sizeof(int), s));
        b.n_chunks = 0;
        b.mma = true;
        return FTCG_SUCCESS;
    }
    int* cnt = nullptr;
    int* off = nullptr;
    FTCG_CK(pool_malloc(&cnt, nseg * sizeof(int), s));
    FTCG_CK(pool_malloc(&off, nseg * sizeof(int), s));
    if (block)
        k_blk_count<<<blocks_for(nseg, 256), 256, 0, s>>>(b.ent, b.colptr, b.ntiles, b.ncb, b.T,
                                                          b.W, cnt);
    else
        k_chunk_count<<<blocks_for(nseg, 256), 256, 0, s>>>(b.ent, b.colptr, nseg, b.W, cnt);
    FTCG_CK(cudaGetLastError());
    FTCG_TRY(exclusive_scan_i32(cnt, off, nseg, s));
    int last_off = 0, last_cnt = 0;
    FTCG_CK(cudaMemcpyAsync(&last_off, off + nseg - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    FTCG_CK(cudaMemcpyAsync(&last_cnt, cnt + nseg - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    FTCG_CK(cudaStreamSynchronize(s));
    const int total = last_off + last_cnt;
    b.n_chunks = total;
    // padding chunks after the last (slots flagged as padding), for the kernel's reads ahead
    constexpr int kPad = mma::kPrefetchChunks;
    const size_t ent_bytes = (size_t)(total + kPad) * kMmaChunk * sizeof(MmaEntry);
    FTCG_CK(pool_malloc(&b.cent, ent_bytes, s));
    FTCG_CK(pool_malloc(&b.chdr, (size_t)(total + kPad) * sizeof(uint32_t), s));
    *bytes += (int64_t)ent_bytes + (int64_t)(total + kPad) * sizeof(uint32_t);
    k_pad_chunks<<<1, kPad * kMmaChunk, 0, s>>>(b.cent + (size_t)total * kMmaChunk,
                                                kPad * kMmaChunk);
    FTCG_CK(cudaGetLastError());
    FTCG_CK(cudaMemsetAsync(b.chdr + total, 0, kPad * sizeof(uint32_t), s));
    if (block)
        k_blk_emit<<<blocks_for(nseg, 256), 256, 0, s>>>(b.ent, b.colptr, off, b.ntiles, b.ncb,
                                                         b.T, b.W, b.cent, b.chdr);
    else
        k_chunk_emit<<<blocks_for(nseg, 256), 256, 0, s>>>(b.ent, b.colptr, off, nseg, b.ncb, b.W,
                                                           b.cent, b.chdr);
    FTCG_CK(cudaGetLastError());
    k_tile_chunk<<<blocks_for(b.ntiles + 1, 256), 256, 0, s>>>(off, b.ntiles, per_tile, total,
                                                               b.tile_chunk);
    FTCG_CK(cudaGetLastError());
    FTCG_CK(pool_free(cnt, s));
    FTCG_CK(pool_free(off, s));
    b.mma = true;
    return FTCG_SUCCESS;
}

ftcg_status_t launch_spread_mma(const Plan& p, const void* vals, bool vbf, float2* grid,
                                cudaStream_t s, int nt) {
    const bool abf = p.opts.precision == FTCG_PREC_BF16;
    if (p.bin.blk) {
        if (vbf && abf) return dispatch_blk_t<true, true>(p, vals, grid, s, nt);
        if (vbf) return dispatch_blk_t<true, false>(p, vals, grid, s, nt);
        if (abf) return dispatch_blk_t<false, true>(p, vals, grid, s, nt);
        return dispatch_blk_t<false, false>(p, vals, grid, s, nt);
    }
    if (vbf && abf) return dispatch_mma_t<true, true>(p, vals, grid, s, nt);
    if (vbf) return dispatch_mma_t<true, false>(p, vals, grid, s, nt);
    if (abf) return dispatch_mma_t<false, true>(p, vals, grid, s, nt);
    return dispatch_mma_t<false, false>(p, vals, grid, s, nt);
}

ftcg_status_t launch_set_alpha_mma(const Plan& p, const void* alpha, int dtype, cudaStream_t s) {
    if (!p.bin.mma || p.bin.n_chunks == 0) return FTCG_SUCCESS;
    const int64_t n = p.bin.n_chunks * kMmaChunk;
    k_set_alpha_mma<<<blocks_for(n, 256), 256, 0, s>>>(p.bin.cent, n, alpha, dtype,
                                                      p.opts.precision == FTCG_PREC_BF16);
    FTCG_CK(cudaGetLastError());
    return FTCG_SUCCESS;
}

}  // namespace ftcg
