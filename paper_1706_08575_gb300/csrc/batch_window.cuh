// The persistent register-window spreading launch of a batch: CTAs take (ping, tile) items from
// an atomic counter, heaviest first, and run the same tile body as the single-ping
// register-window kernel, specialised for the ES window (no family test in the inner loop) or
// generic. Its instantiations are split over two translation units (batch_window.cu for ES,
// batch_window_any.cu for the other families) so that they compile in parallel with batch.cu.
#pragma once

#include <algorithm>

#include "batch_desc.cuh"

namespace ftcg {
namespace bwin {

template <int GW, int WT, bool VBF, bool ABF, int CPL, bool ES>
__global__ void __launch_bounds__(tile::kSpreadThreads, FTCG_SPREAD_MINB)
    k_spread_batch(const PingDesc* __restrict__ desc, const int2* __restrict__ items, int nitems,
                   int* __restrict__ counter, int Wrt, Win32 win) {
    extern __shared__ float smem[];
    __shared__ int s_item;
    for (;;) {
        __syncthreads();   // the previous item's tile is stored and s_item consumed
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) return;
        const int2 pt = items[it];
        const PingDesc d = desc[pt.x];
        if (d.halo) {
            if (d.T == 64)
                tile::spread_tile<GW, WT, 64, VBF, ABF, true, CPL, ES>(d.ent, d.colptr, d.vals, d.grid, d.G,
                                                              d.ntx, Wrt, win, pt.y, smem,
                                                              d.halo_buf, d.halo_cells);
            else
                tile::spread_tile<GW, WT, 32, VBF, ABF, true, CPL, ES>(d.ent, d.colptr, d.vals, d.grid, d.G,
                                                              d.ntx, Wrt, win, pt.y, smem,
                                                              d.halo_buf, d.halo_cells);
        } else {
            if (d.T == 64)
                tile::spread_tile<GW, WT, 64, VBF, ABF, false, CPL, ES>(d.ent, d.colptr, d.vals, d.grid,
                                                               d.G, d.ntx, Wrt, win, pt.y,
                                                               smem, nullptr, 0);
            else
                tile::spread_tile<GW, WT, 32, VBF, ABF, false, CPL, ES>(d.ent, d.colptr, d.vals, d.grid,
                                                               d.G, d.ntx, Wrt, win, pt.y,
                                                               smem, nullptr, 0);
        }
    }
}

struct WindowLaunch {
    const PingDesc* desc;
    const int2* items;
    int nitems;
    int* counter;
    int w;
    Win32 win;
    int* persistent_ctas;
};

template <int GW, int WT, bool VBF, bool ABF, int CPL = 1, bool ES = true>
ftcg_status_t launch_t(const WindowLaunch& a, cudaStream_t s) {
    auto kern = k_spread_batch<GW, WT, VBF, ABF, CPL, ES>;
    const size_t smem = spread_smem<(WT > 0 ? WT : GW * CPL)>();
    FTCG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FTCG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared));
    if (*a.persistent_ctas == 0) {
        int dev = 0, sms = 0, per = 0;
        FTCG_CK(cudaGetDevice(&dev));
        FTCG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        FTCG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, tile::kSpreadThreads,
                                                              smem));
        *a.persistent_ctas = std::max(1, sms * std::max(1, per));
    }
    kern<<<*a.persistent_ctas, tile::kSpreadThreads, smem, s>>>(a.desc, a.items, a.nitems,
                                                                a.counter, a.w, a.win);
    FTCG_CK(cudaGetLastError());
    return FTCG_SUCCESS;
}

// Launch for one value/weight precision and one kind of window (ES or any other family).
template <bool VBF, bool ABF, bool ES>
ftcg_status_t launch_w(const WindowLaunch& a, cudaStream_t s) {
    using tile::kCpl8;
    using tile::kCpl16;
    if constexpr (!ES) {                       // other window families: runtime width only
        if (a.w <= 4) return launch_t<4, 0, VBF, ABF, 1, false>(a, s);
        if (a.w <= 8) return launch_t<8 / kCpl8, 0, VBF, ABF, kCpl8, false>(a, s);
        return launch_t<16 / kCpl16, 0, VBF, ABF, kCpl16, false>(a, s);
    } else {
        switch (a.w) {
            case 6: return launch_t<8 / kCpl8, 6, VBF, ABF, kCpl8>(a, s);
            case 8: return launch_t<8 / kCpl8, 8, VBF, ABF, kCpl8>(a, s);
            default:
                if (a.w <= 4) return launch_t<4, 0, VBF, ABF>(a, s);
                if (a.w <= 8) return launch_t<8 / kCpl8, 0, VBF, ABF, kCpl8>(a, s);
                return launch_t<16 / kCpl16, 0, VBF, ABF, kCpl16>(a, s);
        }
    }
}

template <bool ES>
ftcg_status_t launch_family(const WindowLaunch& a, bool vbf, bool abf, cudaStream_t s) {
    if (vbf && abf) return launch_w<true, true, ES>(a, s);
    if (vbf) return launch_w<true, false, ES>(a, s);
    if (abf) return launch_w<false, true, ES>(a, s);
    return launch_w<false, false, ES>(a, s);
}

// defined in batch_window_any.cu
ftcg_status_t launch_any(const WindowLaunch& a, bool vbf, bool abf, cudaStream_t s);

}  // namespace bwin
}  // namespace ftcg
