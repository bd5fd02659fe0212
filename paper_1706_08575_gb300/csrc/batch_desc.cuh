// The per-ping descriptor of a batch on the device, shared by the batch's translation units
// (batch.cu: planning, the tensor-core and transform launches; batch_window.cu: the persistent
// register-window spreading launch).
#pragma once

#include "spread_tile.cuh"

namespace ftcg {

struct PingDesc {
    const Entry* ent;
    const int* colptr;
    const void* vals;
    float2* grid;
    float2* img;
    const float2* deapod2;
    float2* halo_buf;
    const unsigned* col_mask;    // shared-memory FFT: column blocks that taps reach
    int G, ntx, T, N;
    int halo, halo_cells, ncb, W;
    int fused;                   // 1: the row pass writes the image (no k_deapod_batch)
    // tensor-core spreading (halo layout, w <= 8): the ping's chunks
    const MmaEntry* cent;
    const uint32_t* chdr;
    const int* tile_chunk;
    int blk;                     // 1: the chunks are 8 x 8-cell blocks (spread_blk.cuh)
};

// Dynamic shared memory of the register-window tile body for any tile side and layout a batch
// may hold.
template <int WMAX>
size_t spread_smem() {
    return std::max(std::max(tile::tile_smem_bytes<64, WMAX, true>(),
                             tile::tile_smem_bytes<64, WMAX, false>()),
                    tile::tile_smem_bytes<32, WMAX, true>());
}

// The persistent register-window spreading launch over the items [0, nitems) of d_items
// (CTAs take items from *d_counter): the window family `kind` with width w and oversampling
// sigma, BF16 values / weights as flagged. *persistent_ctas (0 on the first call) receives the
// grid size, resident CTAs per SM x SMs.
ftcg_status_t launch_batch_window(const PingDesc* d_desc, const int2* d_items, int nitems,
                                  int* d_counter, int w, double sigma, int kind, bool vbf,
                                  bool abf, int* persistent_ctas, cudaStream_t s);

}  // namespace ftcg
