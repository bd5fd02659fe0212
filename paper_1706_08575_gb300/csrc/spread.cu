// Spreading (Omega_2 D_2 f^, Eq. twodcgmatrix), deapodisation + crop (division by the window,
// Eq. newadm, and the restriction to p in {-N/2..N/2-1}^2), the gridded forward transform and the
// installation of per-sample weights.
//
// Spreading: one CTA owns one T x T tile of the periodic G x G grid and accumulates it in shared
// memory; tiles are launched heaviest first. The tile's sorted entries (every (tile, sample) pair
// whose w x w footprint touches the tile, ordered by first-tap column then first-tap row, built
// by plan.cu) are split into equal contiguous chunks, one per group of GW lanes (GW = 4, 8 or
// 16, GW x CPL >= w). Lane l of a group owns tap columns l, l + GW, ... (CPL of them) of the
// current column bin and keeps a rolling window of w rows of each in registers: an entry adds
// c phi(dx - l) phi(dy - r) to window row r (the w row factors are computed by the lanes and
// broadcast by shuffles); when the next entry starts on a later row, the rows it can no longer
// reach leave the window with one shared-memory atomic each. A row thus receives one atomic per
// (column bin, chunk) instead of one per entry. The tile is then stored once, coalesced: every
// grid cell is written exactly once, with no zero-fill. In the halo layout the accumulator also
// holds the w - 1 overflow rows and columns, which k_halo_add adds to the neighbouring tiles.

#include "spread_window.cuh"

namespace ftcg {

namespace {

using tile::kSpreadThreads;
using tile::win32;

// one CTA per non-empty tile (the first n_nonempty of the heaviest-first order)
__global__ void __launch_bounds__(256)
    k_halo_add(const float2* __restrict__ halo_buf, int halo_cells, const int* __restrict__ colptr,
               const int* __restrict__ tile_order, int ncb, float2* __restrict__ grid, int G,
               int T, int W, int ntx) {
    pdl_wait();                                // the spreading kernel's tiles and strips
    pdl_allow_next();
    tile::halo_add_tile(halo_buf, halo_cells, colptr, ncb, grid, G, T, W, ntx,
                        tile_order[blockIdx.x]);
}

// Deterministic plans (every tile full): the overflow strips added without atomics, by one
// thread per receiving cell in a fixed order. Cell (lx, ly) of tile (tx, ty) takes, when
// lx < w - 1, the right strip of tile (tx - 1, ty) at row ly and, when also ly < w - 1, that of
// tile (tx - 1, ty - 1) at row T + ly; then, when ly < w - 1, the bottom strip of tile
// (tx, ty - 1) (neighbours mod G; only tiles that wrote strips, full[] = 1). One CTA per tile
// of the spreading launch.
__global__ void __launch_bounds__(256)
    k_halo_gather(const float2* __restrict__ halo_buf, int halo_cells,
                  const unsigned char* __restrict__ full, const int* __restrict__ tile_order,
                  float2* __restrict__ grid, int G, int T, int W, int ntx) {
    pdl_wait();                                // the spreading kernel's tiles and strips
    pdl_allow_next();
    const int tile = tile_order[blockIdx.x];
    const int tyi = tile / ntx, txi = tile - tyi * ntx;
    const int X0 = txi * T, Y0 = tyi * T;
    const int W1 = W - 1, right = (T + W1) * W1;
    const int txl = (txi == 0 ? ntx : txi) - 1, tyu = (tyi == 0 ? ntx : tyi) - 1;
    const int tl = tyi * ntx + txl, tu = tyu * ntx + txi, tul = tyu * ntx + txl;
    const bool fl = full[tl] != 0, fu = full[tu] != 0, ful = full[tul] != 0;
    if (!fl && !fu && !ful) return;
    // the receiving cells: the first w - 1 columns of every row, then the rest of the first
    // w - 1 rows
    const int ncol = T * W1, nrow = W1 * (T - W1);
    for (int k = threadIdx.x; k < ncol + nrow; k += blockDim.x) {
        int lx, ly;
        if (k < ncol) {
            ly = k / W1;
            lx = k - ly * W1;
        } else {
            const int kk = k - ncol;
            ly = kk / (T - W1);
            lx = W1 + (kk - ly * (T - W1));
        }
        float2* c = grid + (int64_t)(Y0 + ly) * G + X0 + lx;
        float2 v = *c;
        auto add = [&](int t, int i) {
            const float2 a = halo_buf[(int64_t)t * halo_cells + i];
            v.x += a.x;
            v.y += a.y;
        };
        if (lx < W1) {
            if (fl) add(tl, ly * W1 + lx);
            if (ly < W1 && ful) add(tul, (T + ly) * W1 + lx);
        }
        if (ly < W1 && fu) add(tu, right + ly * T + lx);
        *c = v;
    }
}

// ---- deapodisation and crop (the body is deapod_crop_block) -------------------------------------
__global__ void __launch_bounds__(kDeapodThreads)
    k_deapod_crop(const float2* __restrict__ grid, float2* __restrict__ img,
                  const float2* __restrict__ r2, int N, int G, bool vec) {
    deapod_crop_block(grid, img, r2, N, G, vec);
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
             float2* __restrict__ out, int G, int W, Win32 win) {
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
            const float fx = lane_tap ? win32(dx - (float)l, win) : 0.0f;
            const float fy = lane_tap ? win32(dy - (float)l, win) : 0.0f;
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
        ent[i].alpha = bf16 ? (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) << 16
                            : __float_as_uint(a);
    }
}

__global__ void k_alpha_f32(const void* __restrict__ alpha, int dtype, int64_t M,
                            float* __restrict__ out) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x)
        out[j] = dtype == FTCG_WEIGHTS_F64 ? (float)reinterpret_cast<const double*>(alpha)[j]
                                           : reinterpret_cast<const float*>(alpha)[j];
}

int blocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

}  // namespace

ftcg_status_t launch_halo_add(const Plan& p, float2* grid, cudaStream_t s) {
    const Binning& b = p.bin;
    if (!b.halo || b.n_nonempty == 0) return FTCG_SUCCESS;
    // the first n_nonempty tiles of the launch order are the non-empty ones: no emptiness test
    FTCG_CK(launch_pdl(k_halo_add, dim3(b.n_nonempty), dim3(256), 0, s,
                       (const float2*)b.halo_buf, b.halo_cells, (const int*)nullptr,
                       (const int*)b.tile_order, b.ncb, grid, b.G, b.T, b.W, b.ntx));
    return FTCG_SUCCESS;
}

ftcg_status_t launch_halo_gather(const Plan& p, float2* grid, cudaStream_t s, int nt) {
    const Binning& b = p.bin;
    if (!b.halo || b.n_nonempty == 0) return FTCG_SUCCESS;
    FTCG_CK(launch_pdl(k_halo_gather, dim3(nt), dim3(256), 0, s, (const float2*)b.halo_buf,
                       b.halo_cells, (const unsigned char*)b.tile_full, (const int*)b.tile_order,
                       grid, b.G, b.T, b.W, b.ntx));
    return FTCG_SUCCESS;
}

ftcg_status_t launch_spread(const Plan& p, const void* vals, int vdtype, float2* grid,
                            cudaStream_t s, bool pruned) {
    if (p.bin.n_entries == 0) {
        FTCG_CK(cudaMemsetAsync(grid, 0, (size_t)p.G * p.G * sizeof(float2), s));
        return FTCG_SUCCESS;
    }
    // the pruned transform reads only the tiles in the first n_read of the launch order
    const int nt = pruned && p.bin.n_read > 0 ? p.bin.n_read : p.bin.ntiles;
    const bool vbf = vdtype == FTCG_VALUES_BF16X2;
    if (p.bin.mma) return launch_spread_mma(p, vals, vbf, grid, s, nt);
    if (p.win.kind == FTCG_WINDOW_ES) return swin::launch_window_spread<true>(p, vals, vbf, grid, s, nt);
    return swin::launch_window_spread_any(p, vals, vbf, grid, s, nt);
}

ftcg_status_t launch_deapod_crop(const Plan& p, const float2* grid, float2* img, cudaStream_t s) {
    const dim3 blocks((p.N + 2 * kDeapodThreads - 1) / (2 * kDeapodThreads),
                      (p.N + kDeapodRows - 1) / kDeapodRows);
    k_deapod_crop<<<blocks, kDeapodThreads, 0, s>>>(grid, img, p.deapod2, p.N, p.G,
                                                    deapod_vec_ok(grid, img, p.N));
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
    const Win32 win = win32_of(p.win);
    if (p.w <= 8) {
        k_interp<8><<<blocks_for(p.M * 8, 256), 256, 0, s>>>(p.samp, p.M, grid, vals, p.G, p.w,
                                                             win);
    } else {
        k_interp<16><<<blocks_for(p.M * 16, 256), 256, 0, s>>>(p.samp, p.M, grid, vals, p.G, p.w,
                                                               win);
    }
    FTCG_CK(cudaGetLastError());
    return FTCG_SUCCESS;
}

ftcg_status_t install_alpha(const Plan& p, const void* alpha, int dtype, cudaStream_t s) {
    if (p.bin.n_entries == 0) return FTCG_SUCCESS;
    k_set_alpha<<<blocks_for(p.bin.n_entries, 256), 256, 0, s>>>(
        p.bin.ent, p.bin.n_entries, alpha, dtype, p.opts.precision == FTCG_PREC_BF16);
    FTCG_CK(cudaGetLastError());
    return launch_set_alpha_mma(p, alpha, dtype, s);
}

ftcg_status_t launch_set_alpha(Plan& p, const void* alpha, int dtype, cudaStream_t s) {
    if (!alpha) {
        if (p.alpha_cur) FTCG_CK(pool_free(p.alpha_cur, s));
        p.alpha_cur = nullptr;
    } else if (p.M > 0) {
        if (!p.alpha_cur) FTCG_CK(pool_malloc(&p.alpha_cur, (size_t)p.M * sizeof(float), s));
        k_alpha_f32<<<blocks_for(p.M, 256), 256, 0, s>>>(alpha, dtype, p.M, p.alpha_cur);
        FTCG_CK(cudaGetLastError());
    }
    return install_alpha(p, alpha, dtype, s);
}

}  // namespace ftcg
