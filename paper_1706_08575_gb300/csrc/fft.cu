// The inverse FFT of the adjoint (the sum over l in Eq. twodcg), pruned to what the crop keeps.
//
// The image needs the G x G inverse DFT of the grid only at the N x N frequencies
// p in {-N/2..N/2-1}^2, i.e. rows and columns [0, N/2) and [G - N/2, G). The 2-D transform is done
// as 1-D column transforms (along y) followed by 1-D row transforms (along x):
//   * a column whose cells are all zero transforms to zero, so only the columns that some
//     sample's w taps reach are transformed (the occupied set, found at plan time, is covered by
//     at most two contiguous runs of the periodic column index);
//   * of the row transforms only the N rows of the crop are needed.
// The other cells of the grid are left as they are (never read). The arithmetic of every kept
// output is that of a full 2-D inverse FFT. For power-of-two G from 256 to 4096 the 1-D transforms
// are this library's shared-memory kernels (fft_smem.cu, with the window division and crop fused
// into the row pass); otherwise cuFFT is the 1-D engine.

#include "ftcg_internal.cuh"

#include <vector>

namespace ftcg {

namespace {

// occ[x] = 1 for every column x that one of a sample's w tap columns reaches (mod G)
__global__ void k_col_occupancy(const int4* __restrict__ samp, int64_t M, int G, int W,
                                unsigned char* __restrict__ occ) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int cx = samp[j].x;
        if (cx < 0) continue;                       // dropped (non-finite) sample
        for (int t = 0; t < W; ++t) {
            int x = cx + t;
            if (x >= G) x -= G;
            occ[x] = 1;
        }
    }
}

// Smallest cyclic interval [x0, x0 + n) covering every occupied column: the complement of the
// longest cyclic run of empty columns. n = 0 when nothing is occupied.
void covering_interval(const std::vector<unsigned char>& occ, int* x0, int* n) {
    const int G = (int)occ.size();
    int first = -1;
    for (int x = 0; x < G; ++x)
        if (occ[x]) { first = x; break; }
    if (first < 0) { *x0 = 0; *n = 0; return; }
    // walk one period starting at an occupied column; track the longest empty run
    int best_len = 0, best_end = first, run = 0;
    for (int k = 1; k <= G; ++k) {
        const int x = (first + k) % G;
        if (!occ[x]) {
            ++run;
        } else {
            if (run > best_len) { best_len = run; best_end = x; }
            run = 0;
        }
    }
    if (best_len == 0) {            // every column occupied: one run
        *x0 = 0;
        *n = G;
        return;
    }
    *x0 = best_end;                 // first occupied column after the longest empty run
    *n = G - best_len;
}

cufftResult plan_columns(cufftHandle* h, int G, int batch) {
    int n[1] = {G};
    int emb[1] = {G};
    return cufftPlanMany(h, 1, n, emb, G, 1, emb, G, 1, CUFFT_C2C, batch);
}

}  // namespace

ftcg_status_t column_occupancy(const Plan* p, cudaStream_t s, std::vector<unsigned char>* occ) {
    if ((int)p->bin.col_occ.size() == p->G) {     // derived from the binning on the host
        *occ = p->bin.col_occ;
        return FTCG_SUCCESS;
    }
    occ->assign(p->G, 0);
    if (p->M == 0) return FTCG_SUCCESS;
    unsigned char* d_occ = nullptr;
    FTCG_CK(cudaMallocAsync(&d_occ, p->G, s));
    FTCG_CK(cudaMemsetAsync(d_occ, 0, p->G, s));
    const int blocks = (int)std::min<int64_t>((p->M + 255) / 256, 4096);
    k_col_occupancy<<<blocks, 256, 0, s>>>(p->samp, p->M, p->G, p->w, d_occ);
    FTCG_CK(cudaGetLastError());
    FTCG_CK(cudaMemcpyAsync(occ->data(), d_occ, p->G, cudaMemcpyDeviceToHost, s));
    FTCG_CK(cudaFreeAsync(d_occ, s));
    FTCG_CK(cudaStreamSynchronize(s));
    return FTCG_SUCCESS;
}

ftcg_status_t build_pruned_fft(Plan* p, cudaStream_t s, int64_t* bytes) {
    const int G = p->G, N = p->N;
    int x0 = 0, n = 0;
    if (p->M > 0) {
        std::vector<unsigned char> occ;
        FTCG_TRY(column_occupancy(p, s, &occ));
        covering_interval(occ, &x0, &n);
        if (smem_fft_supported(G)) return build_smem_fft(p, occ, s, bytes);
    } else if (smem_fft_supported(G)) {
        return build_smem_fft(p, std::vector<unsigned char>(G, 0), s, bytes);
    }
    // at most two runs of columns: [x0, min(G, x0 + n)) and [0, x0 + n - G)
    p->col_x0[0] = x0;
    p->col_n[0] = std::min(n, G - x0);
    p->col_x0[1] = 0;
    p->col_n[1] = n - p->col_n[0];
    size_t ws = 0;
    for (int k = 0; k < 2; ++k) {
        if (p->col_n[k] == 0) continue;
        FTCG_CKFFT(plan_columns(&p->fft_col[k], G, p->col_n[k]));
        if (cufftGetSize(p->fft_col[k], &ws) == CUFFT_SUCCESS) *bytes += (int64_t)ws;
    }
    int nr[1] = {G};
    int emb[1] = {G};
    FTCG_CKFFT(cufftPlanMany(&p->fft_row, 1, nr, emb, 1, G, emb, 1, G, CUFFT_C2C, N / 2));
    if (cufftGetSize(p->fft_row, &ws) == CUFFT_SUCCESS) *bytes += (int64_t)ws;
    p->pruned_ok = true;
    return FTCG_SUCCESS;
}

ftcg_status_t exec_pruned_inverse(Plan* p, cudaStream_t s) {
    cufftComplex* g = reinterpret_cast<cufftComplex*>(p->grid);
    const int G = p->G, N = p->N;
    for (int k = 0; k < 2; ++k) {
        if (p->col_n[k] == 0) continue;
        FTCG_CKFFT(cufftSetStream(p->fft_col[k], s));
        FTCG_CKFFT(cufftExecC2C(p->fft_col[k], g + p->col_x0[k], g + p->col_x0[k], CUFFT_INVERSE));
    }
    FTCG_CKFFT(cufftSetStream(p->fft_row, s));
    FTCG_CKFFT(cufftExecC2C(p->fft_row, g, g, CUFFT_INVERSE));                    // rows [0, N/2)
    cufftComplex* hi = g + (int64_t)(G - N / 2) * G;
    FTCG_CKFFT(cufftExecC2C(p->fft_row, hi, hi, CUFFT_INVERSE));                  // rows [G-N/2, G)
    return FTCG_SUCCESS;
}

void release_pruned_fft(Plan* p) {
    release_smem_fft(p);
    for (int k = 0; k < 2; ++k)
        if (p->fft_col[k]) cufftDestroy(p->fft_col[k]);
    if (p->fft_row) cufftDestroy(p->fft_row);
    p->fft_col[0] = p->fft_col[1] = 0;
    p->fft_row = 0;
    p->pruned_ok = false;
}

}  // namespace ftcg
