// The register-window spreading kernel and its launch (the tile body is spread_tile.cuh), split
// over two translation units: spread.cu instantiates it for the ES window, spread_any.cu for the
// other window families, so that the two compile in parallel.
#pragma once

#include "spread_tile.cuh"

namespace ftcg {
namespace swin {

using tile::kSpreadThreads;

template <int GW, int WT, int T, bool VBF, bool ABF, bool HALO, int CPL, bool ES>
__global__ void __launch_bounds__(tile::kSpreadThreads, FTCG_SPREAD_MINB)
    k_spread(const Entry* __restrict__ ent, const int* __restrict__ colptr,
             const int* __restrict__ tile_order, const void* __restrict__ vals,
             float2* __restrict__ grid, int G, int ntx, int Wrt, Win32 win,
             float2* __restrict__ halo_buf, int halo_cells) {
    extern __shared__ float smem[];
    pdl_allow_next();                          // the fix-up may be scheduled during the tail
    const int t = tile_order ? tile_order[blockIdx.x] : (int)blockIdx.x;
    tile::spread_tile<GW, WT, T, VBF, ABF, HALO, CPL, ES>(ent, colptr, vals, grid, G, ntx, Wrt,
                                                          win, t, smem, halo_buf, halo_cells);
}

template <int GW, int WT, int T, bool VBF, bool ABF, bool HALO, int CPL = 1, bool ES = true>
ftcg_status_t run_spread(const Plan& p, const void* vals, float2* grid, cudaStream_t s, int nt) {
    const Binning& b = p.bin;
    constexpr int WMAX = WT > 0 ? WT : GW * CPL;
    const size_t smem = tile::tile_smem_bytes<T, WMAX, HALO>();
    auto kern = k_spread<GW, WT, T, VBF, ABF, HALO, CPL, ES>;
    FTCG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FTCG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared));
    kern<<<nt, kSpreadThreads, smem, s>>>(b.ent, b.colptr, b.tile_order, vals, grid, b.G,
                                                b.ntx, b.W, win32_of(p.win), b.halo_buf,
                                                b.halo_cells);
    FTCG_CK(cudaGetLastError());
    if (HALO) return launch_halo_add(p, grid, s);
    return FTCG_SUCCESS;
}

template <int T, bool VBF, bool ABF, bool HALO, bool ES>
ftcg_status_t dispatch_w(const Plan& p, const void* vals, float2* grid, cudaStream_t s, int nt) {
    using tile::kCpl8;
    using tile::kCpl16;
    if constexpr (!ES) {                       // other window families: runtime width only
        if (p.w <= 4) return run_spread<4, 0, T, VBF, ABF, HALO, 1, false>(p, vals, grid, s, nt);
        if (p.w <= 8)
            return run_spread<8 / kCpl8, 0, T, VBF, ABF, HALO, kCpl8, false>(p, vals, grid, s, nt);
        return run_spread<16 / kCpl16, 0, T, VBF, ABF, HALO, kCpl16, false>(p, vals, grid, s, nt);
    } else {
        switch (p.w) {
            case 6: return run_spread<8 / kCpl8, 6, T, VBF, ABF, HALO, kCpl8>(p, vals, grid, s, nt);
            case 8: return run_spread<8 / kCpl8, 8, T, VBF, ABF, HALO, kCpl8>(p, vals, grid, s, nt);
            default:
                if (p.w <= 4) return run_spread<4, 0, T, VBF, ABF, HALO>(p, vals, grid, s, nt);
                if (p.w <= 8)
                    return run_spread<8 / kCpl8, 0, T, VBF, ABF, HALO, kCpl8>(p, vals, grid, s,
                                                                              nt);
                return run_spread<16 / kCpl16, 0, T, VBF, ABF, HALO, kCpl16>(p, vals, grid, s,
                                                                             nt);
        }
    }
}

template <bool VBF, bool ABF, bool ES>
ftcg_status_t dispatch_t(const Plan& p, const void* vals, float2* grid, cudaStream_t s, int nt) {
    if (p.bin.halo) {
        if (p.bin.T == 32) return dispatch_w<32, VBF, ABF, true, ES>(p, vals, grid, s, nt);
        return dispatch_w<64, VBF, ABF, true, ES>(p, vals, grid, s, nt);
    }
    if (p.bin.T == 32) return dispatch_w<32, VBF, ABF, false, ES>(p, vals, grid, s, nt);
    return dispatch_w<64, VBF, ABF, false, ES>(p, vals, grid, s, nt);
}

// The register-window spreading launch (with the halo fix-up) for ES (ES = true, instantiated
// in spread.cu) or the other window families (spread_any.cu).
template <bool ES>
ftcg_status_t launch_window_spread(const Plan& p, const void* vals, bool vbf, float2* grid,
                                   cudaStream_t s, int nt) {
    const bool abf = p.opts.precision == FTCG_PREC_BF16;
    if (vbf && abf) return dispatch_t<true, true, ES>(p, vals, grid, s, nt);
    if (vbf) return dispatch_t<true, false, ES>(p, vals, grid, s, nt);
    if (abf) return dispatch_t<false, true, ES>(p, vals, grid, s, nt);
    return dispatch_t<false, false, ES>(p, vals, grid, s, nt);
}

// defined in spread_any.cu
ftcg_status_t launch_window_spread_any(const Plan& p, const void* vals, bool vbf, float2* grid,
                                       cudaStream_t s, int nt);

}  // namespace swin
}  // namespace ftcg
