// The inverse FFT of the adjoint for power-of-two grid sides, as two passes of shared-memory
// transforms, the second fused with the window division and crop (Eq. twodcg's sum over l, then
// Eq. newadm):
//   pass A  one CTA per block of kColBlock adjacent grid columns that some tap reaches: the
//           columns are loaded into shared memory, transformed along y (length G) and stored back;
//           columns no tap reaches are zero and stay zero, so they are skipped;
//   pass B  one CTA per image row: grid row (p_y mod G) is loaded, transformed along x, and only
//           the N kept frequencies p_x are written, each divided by the window transforms
//           (I_p = h_p / (phi^(p_x / G) phi^(p_y / G))), straight into the image.
// Each 1-D transform is a self-sorting (Stockham) sequence of radix-16/8/4/2 stages: with
// Ns the size of the transforms already done, a stage takes the R values
// x[j + r L / R] (r = 0..R-1), multiplies value r by w^(r k L / (Ns R)), k = j mod Ns,
// w = exp(+2 pi i / L), takes their R-point DFT V_q (sign +) and writes V_q to
// y[(j - k) R + k + q Ns]; after the last stage (Ns = L) the output is in natural order.
// Twiddles come from per-stage tables of w^m computed in FP64 and rounded to FP32; shared-memory
// indices are padded by one element per 16 to spread strided accesses over the banks.

#include "fft_smem.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace ftcg {

namespace {

using namespace sfft;

template <int L>
__global__ void __launch_bounds__(kColThreads, kColMinBlocks)
    k_fft_cols(float2* __restrict__ grid, const int* __restrict__ blocks,
               const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    pdl_wait();                                // the grid is complete
    pdl_allow_next();
    cols_body<L>(grid, blocks[blockIdx.x] * kColBlock, tw, sm);
}

template <int L>
__global__ void __launch_bounds__(row_threads(L))
    k_fft_rows_crop(const float2* __restrict__ grid, const unsigned* __restrict__ mask,
                    const float2* __restrict__ tw, const float2* __restrict__ r2, int N,
                    float2* __restrict__ img) {
    extern __shared__ float2 sm[];
    pdl_wait();                                // the column pass is complete
    rows_body<L>(grid, mask, tw, r2, N, img, blockIdx.x, sm);
}

template <int L>
ftcg_status_t run_smem_fft(const Plan& p, float2* img, cudaStream_t s, cudaEvent_t mid) {
    const size_t smA = (size_t)kColBlock * col_stride(L) * sizeof(float2);
    const size_t smB = (size_t)padded_len(L) * sizeof(float2);
    FTCG_CK(cudaFuncSetAttribute(k_fft_cols<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smA));
    FTCG_CK(cudaFuncSetAttribute(k_fft_rows_crop<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smB));
    if (p.n_col_blocks > 0) {
        FTCG_CK(launch_pdl(k_fft_cols<L>, dim3(p.n_col_blocks), dim3(kColThreads), smA, s,
                           p.grid, (const int*)p.col_blocks, (const float2*)p.tw));
    }
    if (mid) FTCG_CK(cudaEventRecord(mid, s));
    FTCG_CK(launch_pdl(k_fft_rows_crop<L>, dim3(p.N), dim3(row_threads(L)), smB, s,
                       (const float2*)p.grid, (const unsigned*)p.col_mask, (const float2*)p.tw,
                       (const float2*)p.deapod2, p.N, img));
    return FTCG_SUCCESS;
}

}  // namespace

bool smem_fft_supported(int G) {
    return G >= 256 && G <= 4096 && (G & (G - 1)) == 0;
}

ftcg_status_t build_smem_fft(Plan* p, const std::vector<unsigned char>& occ, cudaStream_t s,
                             int64_t* bytes) {
    const int G = p->G;
    std::vector<int> blocks;
    for (int b = 0; b < G / kColBlock; ++b) {
        bool any = false;
        for (int c = 0; c < kColBlock; ++c) any = any || occ[b * kColBlock + c];
        if (any) blocks.push_back(b);
    }
    p->n_col_blocks = (int)blocks.size();
    std::vector<unsigned> mask((G / kColBlock + 31) / 32, 0u);
    for (int b : blocks) mask[b >> 5] |= 1u << (b & 31);
    FTCG_CK(pool_malloc(&p->col_mask, mask.size() * sizeof(unsigned), s));
    *bytes += mask.size() * sizeof(unsigned);
    FTCG_CK(cudaMemcpyAsync(p->col_mask, mask.data(), mask.size() * sizeof(unsigned),
                            cudaMemcpyHostToDevice, s));
    std::vector<float2> tw;
    switch (G) {
        case 256: tw = stage_twiddles<256>(); break;
        case 512: tw = stage_twiddles<512>(); break;
        case 1024: tw = stage_twiddles<1024>(); break;
        case 2048: tw = stage_twiddles<2048>(); break;
        default: tw = stage_twiddles<4096>(); break;
    }
    FTCG_CK(pool_malloc(&p->tw, tw.size() * sizeof(float2), s));
    *bytes += tw.size() * sizeof(float2);
    FTCG_CK(cudaMemcpyAsync(p->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
    if (!blocks.empty()) {
        FTCG_CK(pool_malloc(&p->col_blocks, blocks.size() * sizeof(int), s));
        *bytes += blocks.size() * sizeof(int);
        FTCG_CK(cudaMemcpyAsync(p->col_blocks, blocks.data(), blocks.size() * sizeof(int),
                                cudaMemcpyHostToDevice, s));
    }
    FTCG_CK(cudaStreamSynchronize(s));          // the host vectors go out of scope
    p->smem_fft = true;
    return FTCG_SUCCESS;
}

ftcg_status_t exec_smem_fft(Plan* p, float2* img, cudaStream_t s, cudaEvent_t mid) {
    switch (p->G) {
        case 256: return run_smem_fft<256>(*p, img, s, mid);
        case 512: return run_smem_fft<512>(*p, img, s, mid);
        case 1024: return run_smem_fft<1024>(*p, img, s, mid);
        case 2048: return run_smem_fft<2048>(*p, img, s, mid);
        case 4096: return run_smem_fft<4096>(*p, img, s, mid);
        default:
            set_error("internal: no shared-memory FFT for G = %d", p->G);
            return FTCG_ERR_NOT_SUPPORTED;
    }
}

void release_smem_fft(Plan* p) {
    if (p->tw) cudaFree(p->tw);
    if (p->col_blocks) cudaFree(p->col_blocks);
    if (p->col_mask) cudaFree(p->col_mask);
    p->col_mask = nullptr;
    p->tw = nullptr;
    p->col_blocks = nullptr;
    p->n_col_blocks = 0;
    p->smem_fft = false;
}

}  // namespace ftcg
