// Internal declarations shared by the translation units of libftcg (not installed).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cufft.h>
#include <stdint.h>

#include <exception>
#include <new>
#include <string>
#include <vector>

#include "../../include/ftcg.h"

namespace ftcg {

// ---------------------------------------------------------------------------------------------
// Errors: a thread-local message plus a status code; never exceptions across the ABI.
// ---------------------------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

#define FTCG_CK(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            ::ftcg::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),      \
                              __FILE__, __LINE__);                                          \
            return e_ == cudaErrorMemoryAllocation ? FTCG_ERR_OUT_OF_MEMORY : FTCG_ERR_CUDA; \
        }                                                                                   \
    } while (0)

#define FTCG_CKFFT(call)                                                                    \
    do {                                                                                    \
        cufftResult r_ = (call);                                                            \
        if (r_ != CUFFT_SUCCESS) {                                                          \
            ::ftcg::set_error("%s failed: cufft error %d (%s:%d)", #call, (int)r_, __FILE__,  \
                              __LINE__);                                                    \
            return r_ == CUFFT_ALLOC_FAILED ? FTCG_ERR_OUT_OF_MEMORY : FTCG_ERR_CUDA;       \
        }                                                                                   \
    } while (0)

// Every C entry point's body runs inside FTCG_API_BEGIN / FTCG_API_END, so that what the C++
// library may throw (a failed host allocation in a std::vector, say) becomes a status and a
// message instead of crossing the C ABI.
#define FTCG_API_BEGIN try {
#define FTCG_API_END                                                                        \
    }                                                                                       \
    catch (const std::bad_alloc&) {                                                         \
        ::ftcg::set_error("host allocation failed");                                        \
        return FTCG_ERR_OUT_OF_MEMORY;                                                      \
    }                                                                                       \
    catch (const std::exception& ex_) {                                                     \
        ::ftcg::set_error("host exception: %s", ex_.what());                                \
        return FTCG_ERR_INVALID_VALUE;                                                      \
    }                                                                                       \
    catch (...) {                                                                           \
        ::ftcg::set_error("unknown host exception");                                        \
        return FTCG_ERR_INVALID_VALUE;                                                      \
    }

#define FTCG_TRY(expr)                                                                      \
    do {                                                                                    \
        ftcg_status_t s_ = (expr);                                                          \
        if (s_ != FTCG_SUCCESS) return s_;                                                  \
    } while (0)

// Device status word bits (ftcg_check).
enum : unsigned {
    STATUS_NONFINITE_COORD = 1u,
    STATUS_BAD_WEIGHT_SUM = 2u,
};

// Packed entry word: sample index in the low 25 bits, (cy + w - 1) in the high 7 bits.
constexpr int kSampleBits = 25;
constexpr uint32_t kSampleMask = (1u << kSampleBits) - 1u;
constexpr int64_t kMaxSamples = (int64_t(1) << kSampleBits) - 1;
// Zeroed entries after the last one (sample 0, which exists whenever there are entries), so that
// the spreading loop may prefetch up to two entries past its chunk without a bounds test.
constexpr int kEntryPad = 2;

// One sorted (tile, sample) entry of the spreading plan: 16 bytes, read with one vector load.
//   dx, dy : sigma lambda - first tap, in (w/2 - 1, w/2]   (float32)
//   alpha  : per-sample weight, float32 (FTCG_PREC_BF16: rounded to bfloat16, low 16 bits zero)
//   packed : sample index | (cy_local + w - 1) << 25
struct __align__(16) Entry {
    float dx, dy;
    uint32_t alpha;
    uint32_t packed;
};

// One slot of a tensor-core spreading chunk (spread_mma.cu): 16 bytes, one vector load.
//   sx, sy : first-tap offsets relative to the centre of the tap's unit interval,
//            s = d - (w/2 - 1/2) in (-1/2, 1/2]  (float32; the window's tap polynomials take s)
//   alpha  : per-sample weight (same storage as Entry::alpha)
//   packed : sample index | (first-tap row - chunk window row, 0..8) << 25 | padding flag << 31
struct __align__(16) MmaEntry {
    float sx, sy;
    uint32_t alpha;
    uint32_t packed;
};
constexpr uint32_t kMmaPad = 1u << 31;
constexpr int kMmaChunk = 8;          // samples per chunk (the k extent of one m16n8k8 product)
constexpr int kMmaMaxW = 8;           // widest window of the tensor-core path
constexpr int kMmaDeg = 7;            // degree of the per-tap window polynomials

// The window on tap l's unit interval as a polynomial in s (see MmaEntry), coefficients of
// s^0..s^7 for taps l = 0..7; taps l >= w are zero.
struct MmaPoly {
    float c[kMmaMaxW][kMmaDeg + 1];
};

// The window: ES kernel parameters for one (w, sigma).
struct Window {
    int w;
    double beta;
    int kind = FTCG_WINDOW_ES;             // FTCG_WINDOW_ES, _KB or _GAUSS
};

// The gridding window in FP32 on the device (one of three families, shape parameter beta, with
// inv_hw = 2 / w and norm = 1 / I0(beta) for Kaiser-Bessel).
struct Win32 {
    float beta, inv_hw, norm;
    int kind;
};

// Launch with programmatic dependent launch: the kernel may be scheduled while the previous
// kernel in the stream is finishing (its CTAs start once every CTA of that kernel has started or
// signalled), and it must call pdl_wait() before reading what the previous kernel wrote.
template <typename... K, typename... A>
cudaError_t launch_pdl(void (*kern)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<K>(args)...);
}

// Wait until the previous kernel in the stream has completed and its writes are visible (a no-op
// when the kernel was launched normally); let the next kernel's CTAs be scheduled.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_allow_next() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Stream-ordered allocation from the library's per-device pool (pool.cu); bytes == 0 gives
// nullptr. Free with pool_free on a stream, or with cudaFree.
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t s);
cudaError_t pool_free(void* p, cudaStream_t s);
template <typename T>
cudaError_t pool_malloc(T** p, size_t bytes, cudaStream_t s) {
    return pool_malloc(reinterpret_cast<void**>(p), bytes, s);
}

// A binning of samples into square tiles of a G x G periodic grid.
struct Binning {
    int G = 0, T = 0, W = 0;
    int ntx = 0, ntiles = 0, ncb = 0;   // ncb = T + W - 1 column bins per tile
    int64_t n_entries = 0;
    Entry* ent = nullptr;               // n_entries, sorted by (tile, column bin, row)
    int* colptr = nullptr;              // ntiles * ncb + 1 start offsets
    int* tile_order = nullptr;          // tiles by decreasing entry count (launch order)
    int n_nonempty = 0;                 // tiles with at least one entry (a prefix of tile_order)
    std::vector<unsigned char> col_occ; // host: 1 for every grid column some tap reaches
    std::vector<int> tile_cnt;          // host: entries per tile
    std::vector<int> h_order;           // host copy of tile_order
    int n_read = 0;                     // tiles the pruned inverse transform reads (a prefix of
                                        // tile_order holding the non-empty ones; 0 = all)
    bool halo = false;                  // FTCG_LAYOUT_HALO: one entry per sample + halo strips
    int halo_cells = 0;                 // halo cells per tile
    float2* halo_buf = nullptr;         // ntiles * halo_cells overflow values (halo layout)
    // opts.deterministic: entries of one first-tap cell in sample order, one warp per tile, the
    // strips gathered in a fixed order (k_halo_gather, which reads tile_full)
    bool det = false;
    unsigned char* tile_full = nullptr; // 1 per non-empty tile (deterministic halo plans)
    std::vector<unsigned char> h_full;  // host copy
    // Tensor-core spreading (halo layout, w <= 8): each tile's entries regrouped into chunks of 8
    // samples of one column bin whose first-tap rows fit one 16-row window (spread_mma.cu).
    bool mma = false;
    bool blk = false;                   // the chunks are 8 x 8-cell blocks (spread_blk.cuh)
    int64_t n_chunks = 0;
    MmaEntry* cent = nullptr;           // n_chunks * 8 slots, tile by tile (padding slots flagged)
    uint32_t* chdr = nullptr;           // per chunk: first-tap column | window row << 8
    int* tile_chunk = nullptr;          // ntiles + 1 chunk offsets
    MmaPoly poly{};
};

struct Plan {
    int64_t M = 0;
    int N = 0, G = 0, w = 0;
    double sigma = 0;
    ftcg_opts_t opts{};
    Window win{};
    Binning bin;
    double* lambda = nullptr;           // M x 2 copy (FP64), for the weight construction
    int4* samp = nullptr;               // per sample: (cx mod G, cy mod G, float dx bits, dy bits)
    double* deapod = nullptr;           // N factors 1 / phi^(p / G), p = -N/2 .. N/2-1
    float2* deapod2 = nullptr;          // the same factors split into FP32 (hi, lo) pairs
    float2* grid = nullptr;             // G x G complex64 work grid
    cufftHandle fft = 0;
    bool fft_ok = false;
    // Pruned inverse FFT of the adjoint (fft.cu): 1-D column transforms over the occupied columns
    // (at most two runs, [col_x0[k], col_x0[k] + col_n[k])), then row transforms of the N rows
    // the crop keeps.
    cufftHandle fft_col[2] = {0, 0};
    int col_x0[2] = {0, 0}, col_n[2] = {0, 0};
    cufftHandle fft_row = 0;
    bool pruned_ok = false;
    // Shared-memory transforms for power-of-two G (fft_smem.cu): the column blocks that taps
    // reach, and the FP32 twiddle tables of the transform stages.
    bool smem_fft = false;
    int* col_blocks = nullptr;
    int n_col_blocks = 0;
    unsigned* col_mask = nullptr;       // the same blocks as a bit mask
    float2* tw = nullptr;
    unsigned* status = nullptr;         // device status word
    // banded FTCG coefficients (band.cu): M x (2 band_r - 1) complex128 and the values buffer
    // tau = C v that the adjoint spreads; band_r = 0 when the diagonal weights are in use
    int band_r = 0;
    void* band_c = nullptr;
    void* band_tau = nullptr;
    float* alpha_cur = nullptr;         // the installed weights in acquisition order (FP32;
                                        // nullptr while alpha = 1)
    void* stage_vals = nullptr;         // ftcg_adjoint_host staging (device)
    void* stage_img = nullptr;
    // ftcg_adjoint_host_async: two value staging buffers, a copy stream, and per buffer an event
    // when its upload is done and one when the adjoint that read it is done
    void* pipe_vals[2] = {nullptr, nullptr};
    cudaStream_t pipe_copy = nullptr;
    cudaEvent_t pipe_up[2] = {nullptr, nullptr}, pipe_used[2] = {nullptr, nullptr};
    int pipe_next = 0;
    cudaStream_t last_stream = nullptr;
    int64_t device_bytes = 0;
    // stage profiling: 4 events per recorded adjoint call
    bool profiling = false;
    int prof_calls = 0;
    cudaEvent_t* prof_ev = nullptr;     // kMaxProfiled * 4, created on first use
};
constexpr int kMaxProfiled = 1024;

// api.cu: argument checks of ftcg_plan (fills the default tile) and plan construction.
ftcg_status_t validate_plan_args(int64_t M, int32_t N, double sigma, int32_t w, ftcg_opts_t* o);
ftcg_status_t make_plan(Plan* p, const double* d_lambda, cudaStream_t s, bool own_grid);
// batch.cu: the autotuner of tile side, layout and spreading kernel (cached per grid side, w,
// precision and density bucket).
ftcg_status_t tune_tile(const double* d_lambda, int64_t M, int N, double sigma, int w,
                        const ftcg_opts_t& opts, cudaStream_t s, int* T_out, int* layout_out,
                        int* skern_out);
void release_plan(Plan* p);

// ---------------------------------------------------------------------------------------------
// Launchers (defined in the .cu files)
// ---------------------------------------------------------------------------------------------
// plan.cu
ftcg_status_t build_binning(Binning& b, const double* d_lambda, int64_t M, double scale,
                            int G, int T, int W, bool halo, unsigned* d_status, int4* d_samp,
                            cudaStream_t s, int64_t* bytes);
void free_binning(Binning& b);
ftcg_status_t exclusive_scan_i32(const int* d_in, int* d_out, int64_t n, cudaStream_t s);
// spread.cu
// pruned: only the tiles the pruned inverse transform reads (adjoint with shared-memory FFT);
// otherwise every tile of the grid is stored
ftcg_status_t launch_spread(const Plan& p, const void* vals, int vdtype, float2* grid,
                            cudaStream_t s, bool pruned = false);
ftcg_status_t launch_deapod_crop(const Plan& p, const float2* grid, float2* img, cudaStream_t s);
// spread_mma.cu: the tensor-core spreading path (halo layout, w <= 8)
// fit the per-tap window polynomials; returns false if their error exceeds the path's bound
bool mma_window_poly(int W, double beta, int kind, MmaPoly* out, double* max_err);
ftcg_status_t build_chunks(Binning& b, cudaStream_t s, int64_t* bytes, bool block = false);
void free_chunks(Binning& b);
ftcg_status_t launch_spread_mma(const Plan& p, const void* vals, bool vbf, float2* grid,
                                cudaStream_t s, int nt);
ftcg_status_t launch_set_alpha_mma(const Plan& p, const void* alpha, int dtype, cudaStream_t s);
// launch a plan's k_halo_add fix-up after a halo-layout spreading kernel (spread.cu)
ftcg_status_t launch_halo_add(const Plan& p, float2* grid, cudaStream_t s);
// deterministic plans: the strips gathered per receiving cell in a fixed order (spread.cu) over
// the first nt tiles of the launch order
ftcg_status_t launch_halo_gather(const Plan& p, float2* grid, cudaStream_t s, int nt);
// occ[x] = 1 for every grid column x that some sample's taps reach
ftcg_status_t column_occupancy(const Plan* p, cudaStream_t s, std::vector<unsigned char>* occ);
ftcg_status_t build_pruned_fft(Plan* p, cudaStream_t s, int64_t* bytes);
bool smem_fft_supported(int G);
ftcg_status_t build_smem_fft(Plan* p, const std::vector<unsigned char>& occ, cudaStream_t s,
                             int64_t* bytes);
// the inverse transform and the window division + crop into img; mid (may be null) is recorded
// between the column and the row pass
ftcg_status_t exec_smem_fft(Plan* p, float2* img, cudaStream_t s, cudaEvent_t mid);
void release_smem_fft(Plan* p);
ftcg_status_t exec_pruned_inverse(Plan* p, cudaStream_t s);
void release_pruned_fft(Plan* p);

// An FP64 factor r held as an unevaluated FP32 pair r = hi + lo (hi = fl32(r), lo = fl32(r - hi)),
// so |r - hi - lo| <= 2^-48 |r|.
ftcg_status_t split_factors(const double* r, float2* r2, int n, cudaStream_t s);

// The product of two factors held as (hi, lo) pairs, rounded once to FP32: the dropped lo*lo term
// and the rounding of the inner FMA are both below 2^-46 of the product, so the result is the
// FP32 rounding of the FP64 product, or (within 2^-46 of a rounding boundary) its neighbour.
__device__ __forceinline__ float df_product(float2 a, float2 b) {
    return fmaf(a.x, b.x, fmaf(a.x, b.y, a.y * b.x));
}

// Window division + crop, I_p = h_{p mod G} / (phi^(p_x / G) phi^(p_y / G)) for
// p in {-N/2..N/2-1}^2 (Eq. newadm). The per-pixel product of the FP64 factors (passed as FP32
// pairs) is rounded once to FP32. One thread takes two adjacent columns (ix, ix + 1) of
// kDeapodRows rows, all loads first. vec: 16-byte accesses, valid when N % 4 == 0 (then N/2 is even, so a
// pair never straddles the wrap of the crop) and grid and img are 16-byte aligned.
constexpr int kDeapodThreads = 128, kDeapodRows = 4;
__device__ __forceinline__ void deapod_crop_block(const float2* __restrict__ grid,
                                                  float2* __restrict__ img,
                                                  const float2* __restrict__ r2, int N, int G,
                                                  bool vec) {
    const int ix = 2 * (blockIdx.x * kDeapodThreads + threadIdx.x);
    if (ix >= N) return;                        // N is even, so ix + 1 < N as well
    const int iy0 = blockIdx.y * kDeapodRows;
    const int h = N / 2;
    const int qx0 = ix - h < 0 ? ix - h + G : ix - h;
    const int qx1 = ix + 1 - h < 0 ? ix + 1 - h + G : ix + 1 - h;
    float2 a[kDeapodRows], b[kDeapodRows];
#pragma unroll
    for (int k = 0; k < kDeapodRows; ++k) {
        const int iy = iy0 + k;
        if (iy < N) {
            const float2* row = grid + (int64_t)(iy - h < 0 ? iy - h + G : iy - h) * G;
            if (vec) {
                const float4 v = *reinterpret_cast<const float4*>(row + qx0);
                a[k] = make_float2(v.x, v.y);
                b[k] = make_float2(v.z, v.w);
            } else {
                a[k] = row[qx0];
                b[k] = row[qx1];
            }
        }
    }
    const float2 rx0 = r2[ix], rx1 = r2[ix + 1];
#pragma unroll
    for (int k = 0; k < kDeapodRows; ++k) {
        const int iy = iy0 + k;
        if (iy < N) {
            const float2 ry = r2[iy];
            const float f0 = df_product(ry, rx0), f1 = df_product(ry, rx1);
            float2* out = img + (int64_t)iy * N + ix;
            if (vec) {
                *reinterpret_cast<float4*>(out) =
                    make_float4(a[k].x * f0, a[k].y * f0, b[k].x * f1, b[k].y * f1);
            } else {
                out[0] = make_float2(a[k].x * f0, a[k].y * f0);
                out[1] = make_float2(b[k].x * f1, b[k].y * f1);
            }
        }
    }
}

inline bool deapod_vec_ok(const void* grid, const void* img, int N) {
    return N % 4 == 0 && (reinterpret_cast<uintptr_t>(grid) & 15) == 0 &&
           (reinterpret_cast<uintptr_t>(img) & 15) == 0;
}
ftcg_status_t launch_pad_apod(const Plan& p, const float2* img, float2* grid, cudaStream_t s);
ftcg_status_t launch_interp(const Plan& p, const float2* grid, float2* vals, cudaStream_t s);
// install weights (NULL: alpha = 1) in the plan's entries and keep their FP32 copy in alpha_cur
ftcg_status_t launch_set_alpha(Plan& p, const void* alpha, int dtype, cudaStream_t s);
// install weights in the entries only (alpha_cur unchanged)
ftcg_status_t install_alpha(const Plan& p, const void* alpha, int dtype, cudaStream_t s);
// api.cu: the plan's operators on device buffers (stream-ordered, no host synchronisation);
// with use_band the adjoint applies the installed banded coefficients first (tau = C v)
ftcg_status_t adjoint_device(Plan* p, const void* vals, int32_t vdtype, void* img, cudaStream_t s,
                             bool use_band = true);
// band.cu: tau = C v into p.band_tau; release the band
ftcg_status_t band_apply(const Plan& p, const void* vals, cudaStream_t s);
void release_band(Plan* p);
ftcg_status_t forward_device(Plan* p, const void* img, void* vals, cudaStream_t s);
// window.cu
ftcg_status_t window_factors(double* d_out, int N, int G, const Window& win, cudaStream_t s);
double es_beta(int w, double sigma);
double kernel_beta(int w, double sigma, int kind);
double window64(double t, int w, double beta, int kind);   // the window in FP64 on the host
Win32 win32_of(const Window& win);
// weights.cu
ftcg_status_t compute_weights(Plan& p, double* d_alpha_out, cudaStream_t s);
// judge.cu: exact Fejer sums at K samples, the verdict, and its installation
ftcg_status_t judge_launch(const Plan& p, const double* d_alpha, int K, double* d_S, double* d_a,
                           cudaStream_t s);
bool judge_decide(const double* S, const double* a, int K, double max_rel_err, double* stats);
ftcg_status_t judge_install(Plan& p, const double* d_alpha, bool accept, double med,
                            cudaStream_t s);

}  // namespace ftcg
