// Batched pings: many independent geometries, sample counts and image sides gridded together.
//
// Each ping keeps its own binning (plan.cu) and window factors. Persistent spreading launches
// cover the (ping, tile) work items, one per spreading kernel and tile side present (normally
// one): CTAs (one per resident slot of the GPU) take items from an atomic counter, heaviest
// items first, and run the same tile body as the single-ping kernel.
// The fine grids of pings with the same side G are contiguous, so one batched cuFFT per distinct
// G follows, then one window-division + crop launch for all pings. The whole sequence is
// stream-ordered with no host synchronisation and can be captured once in a CUDA graph.
//
// The tile side, layout and spreading kernel of each ping are chosen by a small autotuner: for
// every (G, w, precision, half-octave bucket of samples per cell) it times the candidates and
// keeps the fastest for the life of the process. A single plan is timed on its own launch; the
// pings of a batch are timed as a batched launch over up to 16 pings of the same class, since a
// batch pays per tile and per column bin, not for how one small ping fills the GPU.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <set>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "fft_smem.cuh"
#include "spread_blk.cuh"
#include "spread_mma.cuh"
#include "batch_desc.cuh"
#include "spread_tile.cuh"

namespace ftcg {

namespace {

constexpr int kTcGroups = 4;   // tensor-core batch groups: {column, block} x {T = 32, T = 64}


// The persistent tensor-core spreading launches, one per (kernel, tile side) group of pings: CTAs
// take the group's (ping, tile) items from an atomic counter, heaviest first. BLK selects the
// block kernel (else the column-bin kernel).
template <bool BLK, int T, bool VBF, bool ABF>
__global__ void __launch_bounds__(mma::kThreads, mma::kMinBlocks)
    k_spread_batch_tc(const PingDesc* __restrict__ desc, const int2* __restrict__ items,
                      int nitems, int* __restrict__ counter, const __grid_constant__ MmaPoly poly) {
    extern __shared__ float smem[];
    __shared__ int s_item;
    for (;;) {
        __syncthreads();   // the previous item's tile is stored and s_item consumed
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) return;
        const int2 pt = items[it];
        const PingDesc& d = desc[pt.x];
        if constexpr (BLK)
            blk::spread_tile<T, VBF, ABF>(d.cent, d.chdr, d.tile_chunk, d.vals, d.grid, d.G, d.ntx,
                                          d.W, poly, d.halo_buf, d.halo_cells, pt.y, smem);
        else
            mma::spread_tile<T, VBF, ABF>(d.cent, d.chdr, d.tile_chunk, d.vals, d.grid, d.G, d.ntx,
                                          d.W, poly, d.halo_buf, d.halo_cells, pt.y, smem);
    }
}

// the overflow strips of every halo-layout (ping, tile) item, after the spreading launch
__global__ void __launch_bounds__(256)
    k_halo_add_batch(const PingDesc* __restrict__ desc, const int2* __restrict__ items) {
    const int2 pt = items[blockIdx.x];        // a non-empty tile of a halo-layout ping
    const PingDesc d = desc[pt.x];
    tile::halo_add_tile(d.halo_buf, d.halo_cells, nullptr, d.ncb, d.grid, d.G, d.T, d.W, d.ntx,
                        pt.y);
}

__global__ void __launch_bounds__(kDeapodThreads) k_deapod_batch(const PingDesc* __restrict__ desc) {
    const PingDesc d = desc[blockIdx.z];
    if (d.fused || blockIdx.y * kDeapodRows >= d.N) return;
    const bool vec = d.N % 4 == 0 && (reinterpret_cast<uintptr_t>(d.grid) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(d.img) & 15) == 0;
    deapod_crop_block(d.grid, d.img, d.deapod2, d.N, d.G, vec);
}

// Shared-memory FFT passes of a size class with power-of-two side L: the column pass over the
// class's (ping, column block) items, then one CTA per (image row, ping of the class).
template <int L>
__global__ void __launch_bounds__(sfft::kColThreads, sfft::kColMinBlocks)
    k_fft_cols_batch(const PingDesc* __restrict__ desc, const int2* __restrict__ items,
                     const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    const int2 it = items[blockIdx.x];
    sfft::cols_body<L>(desc[it.x].grid, it.y * sfft::kColBlock, tw, sm);
}

template <int L>
__global__ void __launch_bounds__(sfft::row_threads(L))
    k_fft_rows_batch(const PingDesc* __restrict__ desc, const int* __restrict__ pings,
                     const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    const PingDesc d = desc[pings[blockIdx.y]];
    sfft::rows_body<L>(d.grid, d.col_mask, tw, d.deapod2, d.N, d.img, blockIdx.x, sm);
}


// ---- autotuner ----------------------------------------------------------------------------
struct TuneKey {
    int G, w, prec, bucket, tile, layout;   // tile / layout: the caller's fixed choices (0 = free)
    int skern;                              // the caller's spreading-kernel choice
    int batch;                              // 1: chosen for pings of a batch (timed batched)
    int win;                                // the gridding window (FTCG_WINDOW_*)
    bool operator<(const TuneKey& o) const {
        if (G != o.G) return G < o.G;
        if (w != o.w) return w < o.w;
        if (prec != o.prec) return prec < o.prec;
        if (bucket != o.bucket) return bucket < o.bucket;
        if (tile != o.tile) return tile < o.tile;
        if (layout != o.layout) return layout < o.layout;
        if (skern != o.skern) return skern < o.skern;
        if (batch != o.batch) return batch < o.batch;
        return win < o.win;
    }
};
// the tuner's choice for a key: tile side, layout and spreading kernel
struct TuneVal {
    int T, layout, skern;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

int density_bucket(int64_t M, int G) {
    const double d = (double)M / ((double)G * G);
    return d <= 0 ? -100 : (int)std::lround(2.0 * std::log2(d));
}

// The integer after "key": on a line of the tuner file; false if the key is absent.
bool json_int(const std::string& line, const char* key, int* out) {
    const std::string k = std::string("\"") + key + "\":";
    const size_t at = line.find(k);
    if (at == std::string::npos) return false;
    const char* p = line.c_str() + at + k.size();
    char* end = nullptr;
    const long v = std::strtol(p, &end, 10);
    if (end == p || v < INT32_MIN || v > INT32_MAX) return false;
    *out = (int)v;
    return true;
}

// Device memory and events released on every return path.
struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// Time the spreading kernel of a plan (values are irrelevant to the cost: zeros), in the launch
// the adjoint makes: only the tiles the shared-memory transform reads when G takes that path.
ftcg_status_t time_spread(const Plan& p, const void* zeros, float2* grid, cudaStream_t s,
                          float* ms) {
    EventPair ev;
    FTCG_CK(cudaEventCreate(&ev.a));
    FTCG_CK(cudaEventCreate(&ev.b));
    const bool pruned = smem_fft_supported(p.G);
    FTCG_TRY(launch_spread(p, zeros, FTCG_VALUES_C64, grid, s, pruned));   // warm-up
    FTCG_CK(cudaEventRecord(ev.a, s));
    for (int r = 0; r < 3; ++r)
        FTCG_TRY(launch_spread(p, zeros, FTCG_VALUES_C64, grid, s, pruned));
    FTCG_CK(cudaEventRecord(ev.b, s));
    FTCG_CK(cudaEventSynchronize(ev.b));
    FTCG_CK(cudaEventElapsedTime(ms, ev.a, ev.b));
    return FTCG_SUCCESS;
}

}  // namespace

// The (tile side, layout, spreading kernel) candidates the tuner times for the caller's options:
// in the halo layout both kernels where the tensor-core kernel applies and the caller left the
// choice open, otherwise the caller's (or the only) kernel.
std::vector<TuneVal> tune_candidates(int w, double sigma, const ftcg_opts_t& opts) {
    std::vector<int> tiles, layouts;
    if (opts.tile) tiles.push_back(opts.tile); else tiles = {32, 64};
    if (opts.layout) layouts.push_back(opts.layout);
    else if (opts.spread_kernel == FTCG_SPREAD_TENSOR || opts.spread_kernel == FTCG_SPREAD_BLOCK)
        layouts.push_back(FTCG_LAYOUT_HALO);
    else layouts = {FTCG_LAYOUT_DUPLICATE, FTCG_LAYOUT_HALO};
    MmaPoly poly;
    double perr = 0;
    const bool tensor_ok = w <= kMmaMaxW && mma_window_poly(w, kernel_beta(w, sigma, opts.kernel),
                                                            opts.kernel, &poly, &perr);
    std::vector<TuneVal> out;
    for (int T : tiles)
        for (int layout : layouts) {
            if (layout == FTCG_LAYOUT_HALO && tensor_ok && opts.spread_kernel == FTCG_SPREAD_AUTO) {
                out.push_back({T, layout, FTCG_SPREAD_TENSOR});
                out.push_back({T, layout, FTCG_SPREAD_BLOCK});
                out.push_back({T, layout, FTCG_SPREAD_WINDOW});
            } else if (layout == FTCG_LAYOUT_HALO && (opts.spread_kernel == FTCG_SPREAD_TENSOR ||
                                                     opts.spread_kernel == FTCG_SPREAD_BLOCK)) {
                out.push_back({T, layout, opts.spread_kernel});
            } else {
                out.push_back({T, layout, FTCG_SPREAD_WINDOW});
            }
        }
    return out;
}

ftcg_status_t tune_tile(const double* d_lambda, int64_t M, int N, double sigma, int w,
                        const ftcg_opts_t& opts, cudaStream_t s, int* T_out, int* layout_out,
                        int* skern_out) {
    const int G = (int)std::llround(sigma * N);
    const TuneKey key{G, w, opts.precision, density_bucket(M, G), opts.tile, opts.layout,
                      opts.spread_kernel, 0, opts.kernel};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            *T_out = it->second.T;
            *layout_out = it->second.layout;
            *skern_out = it->second.skern;
            return FTCG_SUCCESS;
        }
    }
    const std::vector<TuneVal> cand = tune_candidates(w, sigma, opts);
    if (cand.size() == 1) {
        *T_out = cand[0].T;
        *layout_out = cand[0].layout;
        *skern_out = cand[0].skern;
        return FTCG_SUCCESS;
    }
    DevBuf zbuf, gbuf;
    FTCG_CK(cudaMalloc(&zbuf.p, (size_t)std::max<int64_t>(M, 1) * sizeof(float2)));
    FTCG_CK(cudaMemsetAsync(zbuf.p, 0, (size_t)std::max<int64_t>(M, 1) * sizeof(float2), s));
    FTCG_CK(cudaMalloc(&gbuf.p, (size_t)G * G * sizeof(float2)));
    const void* zeros = zbuf.p;
    float2* grid = reinterpret_cast<float2*>(gbuf.p);
    TuneVal best = cand[0];
    float best_ms = 1e30f;
    for (const TuneVal& c : cand) {
        Plan* p = new (std::nothrow) Plan();
        if (!p) {
            set_error("tuner: host allocation failed");
            return FTCG_ERR_OUT_OF_MEMORY;
        }
        p->M = M; p->N = N; p->G = G; p->w = w; p->sigma = sigma;
        p->opts = opts;
        p->opts.tile = c.T;
        p->opts.layout = c.layout;
        p->opts.spread_kernel = c.skern;
        p->win = Window{w, kernel_beta(w, sigma, opts.kernel), opts.kernel};
        ftcg_status_t st = make_plan(p, d_lambda, s, false);
        float ms = 1e30f;
        if (st == FTCG_SUCCESS || st == FTCG_ERR_NUMERIC) st = time_spread(*p, zeros, grid, s, &ms);
        release_plan(p);
        if (st != FTCG_SUCCESS) return st;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = best;
    }
    *T_out = best.T;
    *layout_out = best.layout;
    *skern_out = best.skern;
    return FTCG_SUCCESS;
}

namespace {

struct Batch {
    int n = 0, w = 0;
    double sigma = 0;
    ftcg_opts_t opts{};
    std::vector<Plan*> pings;
    struct Class {
        int G = 0, count = 0, N = 0;
        float2* grids = nullptr;
        cufftHandle fft = 0;
        bool fft_ok = false;
        // shared-memory FFT (power-of-two G in 256..4096): twiddle tables, (ping, column block)
        // items of the column pass, and the class's pings for the row pass
        bool smem = false;
        float2* tw = nullptr;
        int2* col_items = nullptr;
        int n_col_items = 0;
        int* pings = nullptr;
    };
    std::vector<Class> classes;
    std::vector<int> cls_of, slot_of;
    PingDesc* h_desc = nullptr;   // pinned
    PingDesc* d_desc = nullptr;
    // (ping, tile) work items: the n_mma items of tensor-core pings first, grouped by kernel and
    // tile side (group k = 2 blk + (T == 64): items [tc_off[k], tc_off[k + 1])), then the others
    int2* d_items = nullptr;
    int nitems = 0, n_mma = 0;
    int tc_off[kTcGroups + 1] = {};
    int* d_counter = nullptr;     // kTcGroups + 1 counters: the groups', the register-window one
    int2* d_halo_items = nullptr; // the non-empty (ping, tile) items of halo-layout pings
    int n_halo = 0;
    MmaPoly poly{};               // the window polynomials (every ping has the same w, sigma)
    int persistent_ctas_tc[kTcGroups] = {};
    unsigned* d_masks = nullptr;  // shared-memory FFT column-block masks of all pings
    int max_N = 0;
    int persistent_ctas = 0;
    int64_t entries = 0, device_bytes = 0;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t last = nullptr;
    // stage profiling of ftcg_adjoint_batch: 3 events per recorded call
    bool profiling = false;
    int prof_calls = 0;
    std::vector<cudaEvent_t> prof_ev;
};
constexpr int kBatchProfiled = 256;

void release_batch(Batch* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    for (Plan* p : b->pings) release_plan(p);
    for (auto& c : b->classes) {
        if (c.grids) cudaFree(c.grids);
        if (c.fft_ok) cufftDestroy(c.fft);
        if (c.tw) cudaFree(c.tw);
        if (c.col_items) cudaFree(c.col_items);
        if (c.pings) cudaFree(c.pings);
    }
    if (b->h_desc) cudaFreeHost(b->h_desc);
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_counter) cudaFree(b->d_counter);
    if (b->d_halo_items) cudaFree(b->d_halo_items);
    if (b->d_masks) cudaFree(b->d_masks);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (cudaEvent_t e : b->prof_ev) cudaEventDestroy(e);
    delete b;
}

template <bool BLK, int T, bool VBF, bool ABF>
ftcg_status_t launch_batch_tc_group(Batch& b, int k, cudaStream_t s) {
    auto kern = k_spread_batch_tc<BLK, T, VBF, ABF>;
    const size_t smem = BLK ? blk::tile_smem_bytes(T) : mma::tile_smem_bytes(T);
    FTCG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FTCG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared));
    if (b.persistent_ctas_tc[k] == 0) {
        int dev = 0, sms = 0, per = 0;
        FTCG_CK(cudaGetDevice(&dev));
        FTCG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        FTCG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, mma::kThreads, smem));
        b.persistent_ctas_tc[k] = std::max(1, sms * std::max(1, per));
    }
    const int n = b.tc_off[k + 1] - b.tc_off[k];
    kern<<<std::min(b.persistent_ctas_tc[k], n), mma::kThreads, smem, s>>>(
        b.d_desc, b.d_items + b.tc_off[k], n, b.d_counter + k, b.poly);
    FTCG_CK(cudaGetLastError());
    return FTCG_SUCCESS;
}

template <bool VBF, bool ABF>
ftcg_status_t launch_batch_spread_mma(Batch& b, cudaStream_t s) {
    for (int k = 0; k < kTcGroups; ++k) {
        if (b.tc_off[k + 1] == b.tc_off[k]) continue;
        switch (k) {
            case 0: FTCG_TRY((launch_batch_tc_group<false, 32, VBF, ABF>(b, k, s))); break;
            case 1: FTCG_TRY((launch_batch_tc_group<false, 64, VBF, ABF>(b, k, s))); break;
            case 2: FTCG_TRY((launch_batch_tc_group<true, 32, VBF, ABF>(b, k, s))); break;
            default: FTCG_TRY((launch_batch_tc_group<true, 64, VBF, ABF>(b, k, s))); break;
        }
    }
    return FTCG_SUCCESS;
}

template <int L>
ftcg_status_t launch_class_fft_t(Batch& b, const Batch::Class& c, cudaStream_t s) {
    const size_t smA = (size_t)sfft::kColBlock * sfft::col_stride(L) * sizeof(float2);
    const size_t smB = (size_t)sfft::padded_len(L) * sizeof(float2);
    FTCG_CK(cudaFuncSetAttribute(k_fft_cols_batch<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smA));
    FTCG_CK(cudaFuncSetAttribute(k_fft_rows_batch<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smB));
    if (c.n_col_items > 0) {
        k_fft_cols_batch<L><<<c.n_col_items, sfft::kColThreads, smA, s>>>(b.d_desc, c.col_items,
                                                                          c.tw);
        FTCG_CK(cudaGetLastError());
    }
    k_fft_rows_batch<L><<<dim3(c.N, c.count), sfft::row_threads(L), smB, s>>>(b.d_desc, c.pings,
                                                                             c.tw);
    FTCG_CK(cudaGetLastError());
    return FTCG_SUCCESS;
}

ftcg_status_t launch_class_fft(Batch& b, const Batch::Class& c, cudaStream_t s) {
    switch (c.G) {
        case 256: return launch_class_fft_t<256>(b, c, s);
        case 512: return launch_class_fft_t<512>(b, c, s);
        case 1024: return launch_class_fft_t<1024>(b, c, s);
        case 2048: return launch_class_fft_t<2048>(b, c, s);
        case 4096: return launch_class_fft_t<4096>(b, c, s);
        default:
            set_error("internal: no shared-memory FFT for G = %d", c.G);
            return FTCG_ERR_NOT_SUPPORTED;
    }
}

std::vector<float2> class_twiddles(int G) {
    switch (G) {
        case 256: return sfft::stage_twiddles<256>();
        case 512: return sfft::stage_twiddles<512>();
        case 1024: return sfft::stage_twiddles<1024>();
        case 2048: return sfft::stage_twiddles<2048>();
        default: return sfft::stage_twiddles<4096>();
    }
}

// The spreading stage of a batch whose descriptors (values included) are on the device: the
// persistent tensor-core and register-window launches, then the halo fix-up.
ftcg_status_t batch_spread(Batch& b, bool vbf, cudaStream_t s) {
    FTCG_CK(cudaMemsetAsync(b.d_counter, 0, (kTcGroups + 1) * sizeof(int), s));
    const bool abf = b.opts.precision == FTCG_PREC_BF16;
    if (b.n_mma > 0) {
        if (vbf && abf) FTCG_TRY((launch_batch_spread_mma<true, true>(b, s)));
        else if (vbf) FTCG_TRY((launch_batch_spread_mma<true, false>(b, s)));
        else if (abf) FTCG_TRY((launch_batch_spread_mma<false, true>(b, s)));
        else FTCG_TRY((launch_batch_spread_mma<false, false>(b, s)));
    }
    if (b.nitems > b.n_mma)
        FTCG_TRY(launch_batch_window(b.d_desc, b.d_items + b.n_mma, b.nitems - b.n_mma,
                                     b.d_counter + kTcGroups, b.w, b.sigma, b.opts.kernel, vbf, abf,
                                     &b.persistent_ctas, s));
    if (b.n_halo > 0) {
        k_halo_add_batch<<<b.n_halo, 256, 0, s>>>(b.d_desc, b.d_halo_items);
        FTCG_CK(cudaGetLastError());
    }
    return FTCG_SUCCESS;
}

// profile: record the stage events of a profiled batch (not while a graph is being captured)
ftcg_status_t batch_enqueue(Batch& b, const void* const* vals, int32_t vdtype, void* const* imgs,
                            cudaStream_t s, bool profile = false) {
    for (int i = 0; i < b.n; ++i) {
        b.h_desc[i].vals = vals[i];
        b.h_desc[i].img = reinterpret_cast<float2*>(imgs[i]);
    }
    FTCG_CK(cudaMemcpyAsync(b.d_desc, b.h_desc, b.n * sizeof(PingDesc), cudaMemcpyHostToDevice, s));
    cudaEvent_t* ev = nullptr;
    if (profile && b.profiling && b.prof_calls < kBatchProfiled)
        ev = b.prof_ev.data() + 3 * b.prof_calls++;
    if (ev) FTCG_CK(cudaEventRecord(ev[0], s));
    FTCG_TRY(batch_spread(b, vdtype == FTCG_VALUES_BF16X2, s));
    if (ev) FTCG_CK(cudaEventRecord(ev[1], s));
    bool any_cufft = false;
    for (auto& c : b.classes) {
        if (c.smem) {
            FTCG_TRY(launch_class_fft(b, c, s));
            continue;
        }
        any_cufft = true;
        FTCG_CKFFT(cufftSetStream(c.fft, s));
        FTCG_CKFFT(cufftExecC2C(c.fft, reinterpret_cast<cufftComplex*>(c.grids),
                                reinterpret_cast<cufftComplex*>(c.grids), CUFFT_INVERSE));
    }
    if (any_cufft) {
        const dim3 blocks((b.max_N + 2 * kDeapodThreads - 1) / (2 * kDeapodThreads),
                          (b.max_N + kDeapodRows - 1) / kDeapodRows, b.n);
        k_deapod_batch<<<blocks, kDeapodThreads, 0, s>>>(b.d_desc);
        FTCG_CK(cudaGetLastError());
    }
    if (ev) FTCG_CK(cudaEventRecord(ev[2], s));
    return FTCG_SUCCESS;
}

// Builds the pings' plans with up to kPlanThreads host threads, each on its own stream ordered
// after s: a plan's build waits several times for its own small transfers (entry totals, tile
// offsets, status word), and other pings' builds fill those waits. Every plan is complete when
// this returns (make_plan ends with a synchronisation of its stream). Per-ping status and error
// text go to sts and msgs; the return value reports failures of the thread or stream set-up.
constexpr int kPlanThreads = 4;

ftcg_status_t make_plans_parallel(const std::vector<Plan*>& pings, const double* const* d_lambda,
                                  cudaStream_t s, std::vector<ftcg_status_t>& sts,
                                  std::vector<std::string>& msgs) {
    const int n = (int)pings.size();
    const int nt = std::min(kPlanThreads, n);
    if (nt <= 1) {
        for (int i = 0; i < n; ++i) {
            sts[i] = make_plan(pings[i], d_lambda[i], s, false);
            if (sts[i] != FTCG_SUCCESS) msgs[i] = ftcg_last_error();
        }
        return FTCG_SUCCESS;
    }
    int dev = 0;
    FTCG_CK(cudaGetDevice(&dev));
    cudaEvent_t ready = nullptr;
    FTCG_CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    std::vector<cudaStream_t> ws(nt, nullptr);
    cudaError_t ce = cudaEventRecord(ready, s);
    for (int k = 0; k < nt && ce == cudaSuccess; ++k) {
        ce = cudaStreamCreateWithFlags(&ws[k], cudaStreamNonBlocking);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(ws[k], ready, 0);
    }
    if (ce == cudaSuccess) {
        std::atomic<int> next{0};
        auto work = [&](int k) {
            cudaSetDevice(dev);                  // the current device is per host thread
            for (int i; (i = next.fetch_add(1)) < n;) {
                clear_error();
                try {                            // nothing may leave a host thread
                    sts[i] = make_plan(pings[i], d_lambda[i], ws[k], false);
                    if (sts[i] != FTCG_SUCCESS) msgs[i] = ftcg_last_error();
                } catch (...) {
                    sts[i] = FTCG_ERR_OUT_OF_MEMORY;
                    msgs[i] = "host exception while building the plan";
                }
            }
        };
        std::vector<std::thread> th;
        th.reserve(nt - 1);
        for (int k = 1; k < nt; ++k) th.emplace_back(work, k);
        work(0);
        for (auto& t : th) t.join();
    }
    for (cudaStream_t w : ws)
        if (w) {
            cudaStreamSynchronize(w);
            cudaStreamDestroy(w);
        }
    cudaEventDestroy(ready);
    FTCG_CK(ce);
    return FTCG_SUCCESS;
}

// The tuner key of a ping of batch b (batch = 1: chosen by timing batched launches).
TuneKey batch_key(const Batch& b, int64_t M, int G) {
    return TuneKey{G, b.w, b.opts.precision, density_bucket(M, G), b.opts.tile, b.opts.layout,
                   b.opts.spread_kernel, 1, b.opts.kernel};
}

ftcg_status_t tune_batch(const Batch& b, const double* const* d_lambda, const int64_t* M,
                         const int32_t* N, cudaStream_t s);

ftcg_status_t plan_batch_impl(Batch& b, const double* const* d_lambda, const int64_t* M,
                              const int32_t* N, cudaStream_t s) {
    // per-ping plans: the tile side, layout and spreading kernel (unless given) come from the
    // batch tuner, which times batched launches per class of pings before any plan is built
    // (concurrent work would disturb its timings); then the plans are built
    const bool tuning = b.opts.tile == 0 || b.opts.layout == 0;
    if (tuning) FTCG_TRY(tune_batch(b, d_lambda, M, N, s));
    std::vector<int> Gs(b.n);
    for (int i = 0; i < b.n; ++i) {
        const int G = (int)std::llround(b.sigma * N[i]);
        Gs[i] = G;
        int T = b.opts.tile, layout = b.opts.layout, skern = b.opts.spread_kernel;
        if (tuning) {
            bool found = false;
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                auto it = g_tune.find(batch_key(b, M[i], G));
                if (it != g_tune.end()) {
                    T = it->second.T;
                    layout = it->second.layout;
                    skern = it->second.skern;
                    found = true;
                }
            }
            if (!found)
                FTCG_TRY(tune_tile(d_lambda[i], M[i], N[i], b.sigma, b.w, b.opts, s, &T, &layout,
                                   &skern));
        }
        Plan* p = new (std::nothrow) Plan();
        if (!p) {
            set_error("ftcg_plan_batch: host allocation failed");
            return FTCG_ERR_OUT_OF_MEMORY;
        }
        p->M = M[i]; p->N = N[i]; p->G = G; p->w = b.w; p->sigma = b.sigma;
        p->opts = b.opts;
        p->opts.tile = T;
        p->opts.layout = layout;
        p->opts.spread_kernel = skern;
        p->win = Window{b.w, kernel_beta(b.w, b.sigma, b.opts.kernel), b.opts.kernel};
        b.pings.push_back(p);
    }
    std::vector<ftcg_status_t> sts(b.n, FTCG_SUCCESS);
    std::vector<std::string> msgs(b.n);
    FTCG_TRY(make_plans_parallel(b.pings, d_lambda, s, sts, msgs));
    for (int i = 0; i < b.n; ++i) {
        // coordinates that are not finite drop those samples and leave the plan usable
        if (sts[i] != FTCG_SUCCESS && sts[i] != FTCG_ERR_NUMERIC) {
            set_error("ftcg_plan_batch: ping %d: %s", i, msgs[i].c_str());
            return sts[i];
        }
        Plan* p = b.pings[i];
        b.entries += p->bin.n_entries;
        b.device_bytes += p->device_bytes;
        b.max_N = std::max(b.max_N, N[i]);
    }
    // size classes: contiguous grids and one batched FFT per distinct G
    std::vector<int> uniq(Gs);
    std::sort(uniq.begin(), uniq.end());
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    b.classes.resize(uniq.size());
    b.cls_of.resize(b.n);
    b.slot_of.resize(b.n);
    for (size_t c = 0; c < uniq.size(); ++c) b.classes[c].G = uniq[c];
    for (int i = 0; i < b.n; ++i) {
        const int c = (int)(std::lower_bound(uniq.begin(), uniq.end(), Gs[i]) - uniq.begin());
        b.cls_of[i] = c;
        b.slot_of[i] = b.classes[c].count++;
    }
    for (auto& c : b.classes) {
        const size_t per = (size_t)c.G * c.G;
        FTCG_CK(cudaMalloc(&c.grids, per * c.count * sizeof(float2)));
        b.device_bytes += (int64_t)(per * c.count * sizeof(float2));
        c.N = (int)std::llround(c.G / b.sigma);
        if (smem_fft_supported(c.G)) {
            c.smem = true;
            continue;                       // set up with the descriptors below
        }
        int dims[2] = {c.G, c.G};
        FTCG_CKFFT(cufftPlanMany(&c.fft, 2, dims, nullptr, 1, (int)per, nullptr, 1, (int)per,
                                 CUFFT_C2C, c.count));
        c.fft_ok = true;
        size_t ws = 0;
        cufftGetSize(c.fft, &ws);
        b.device_bytes += (int64_t)ws;
    }
    // descriptors and the heaviest-first work list over (ping, tile)
    FTCG_CK(cudaMallocHost(&b.h_desc, b.n * sizeof(PingDesc)));
    FTCG_CK(cudaMalloc(&b.d_desc, b.n * sizeof(PingDesc)));
    struct Item {
        int cnt, ping, tile, grp;   // grp: the tensor-core group (2 blk + (T == 64))
    };
    std::vector<Item> items, items_mma;
    for (int i = 0; i < b.n; ++i) {
        Plan* p = b.pings[i];
        const Binning& bn = p->bin;
        auto& c = b.classes[b.cls_of[i]];
        PingDesc& d = b.h_desc[i];
        d.ent = bn.ent;
        d.colptr = bn.colptr;
        d.vals = nullptr;
        d.grid = c.grids + (size_t)b.slot_of[i] * c.G * c.G;
        d.img = nullptr;
        d.deapod2 = p->deapod2;
        d.G = p->G;
        d.ntx = bn.ntx;
        d.T = bn.T;
        d.N = p->N;
        d.halo = bn.halo ? 1 : 0;
        d.halo_buf = bn.halo_buf;
        d.halo_cells = bn.halo_cells;
        d.ncb = bn.ncb;
        d.W = bn.W;
        d.col_mask = nullptr;
        d.fused = c.smem ? 1 : 0;
        d.cent = bn.cent;
        d.chdr = bn.chdr;
        d.tile_chunk = bn.tile_chunk;
        d.blk = bn.blk ? 1 : 0;
        if (bn.mma) b.poly = bn.poly;
        std::vector<Item>& list = bn.mma ? items_mma : items;
        const int grp = bn.mma ? 2 * (bn.blk ? 1 : 0) + (bn.T == 64 ? 1 : 0) : 0;
        if (c.smem && bn.n_read > 0 && (int)bn.tile_cnt.size() == bn.ntiles &&
            (int)bn.h_order.size() == bn.ntiles) {
            // the shared-memory transforms read only the column blocks that taps reach: the
            // tiles of the pruned launch order (non-empty ones, then empty ones in those columns)
            for (int k = 0; k < bn.n_read; ++k) {
                const int t = bn.h_order[k];
                list.push_back({bn.tile_cnt[t], i, t, grp});
            }
        } else if ((int)bn.tile_cnt.size() == bn.ntiles) {
            for (int t = 0; t < bn.ntiles; ++t) list.push_back({bn.tile_cnt[t], i, t, grp});
        } else {
            std::vector<int> cp((size_t)bn.ntiles * bn.ncb + 1);
            FTCG_CK(cudaMemcpy(cp.data(), bn.colptr, cp.size() * sizeof(int),
                               cudaMemcpyDeviceToHost));
            for (int t = 0; t < bn.ntiles; ++t)
                list.push_back({cp[(size_t)(t + 1) * bn.ncb] - cp[(size_t)t * bn.ncb], i, t, grp});
        }
    }
    // shared-memory FFT classes: per ping the column blocks that taps reach (items of the column
    // pass and a bit mask for the row pass), per class the twiddles and the ping list
    std::vector<std::vector<int2>> col_items(b.classes.size());
    std::vector<std::vector<int>> cls_pings(b.classes.size());
    std::vector<unsigned> masks;                 // all pings' masks, one upload
    std::vector<size_t> mask_off(b.n, 0);
    for (int i = 0; i < b.n; ++i) {
        const int ci = b.cls_of[i];
        if (!b.classes[ci].smem) continue;
        Plan* p = b.pings[i];
        std::vector<unsigned char> occ;
        FTCG_TRY(column_occupancy(p, s, &occ));
        const int nblk = p->G / sfft::kColBlock;
        mask_off[i] = masks.size();
        masks.resize(masks.size() + (nblk + 31) / 32, 0u);
        unsigned* mask = masks.data() + mask_off[i];
        for (int k = 0; k < nblk; ++k) {
            bool any = false;
            for (int c = 0; c < sfft::kColBlock; ++c) any = any || occ[k * sfft::kColBlock + c];
            if (!any) continue;
            col_items[ci].push_back(make_int2(i, k));
            mask[k >> 5] |= 1u << (k & 31);
        }
        cls_pings[ci].push_back(i);
    }
    if (!masks.empty()) {
        FTCG_CK(cudaMalloc(&b.d_masks, masks.size() * sizeof(unsigned)));
        FTCG_CK(cudaMemcpy(b.d_masks, masks.data(), masks.size() * sizeof(unsigned),
                           cudaMemcpyHostToDevice));
        b.device_bytes += (int64_t)(masks.size() * sizeof(unsigned));
        for (int i = 0; i < b.n; ++i)
            if (b.classes[b.cls_of[i]].smem) b.h_desc[i].col_mask = b.d_masks + mask_off[i];
    }
    for (size_t ci = 0; ci < b.classes.size(); ++ci) {
        auto& c = b.classes[ci];
        if (!c.smem) continue;
        const std::vector<float2> tw = class_twiddles(c.G);
        FTCG_CK(cudaMalloc(&c.tw, tw.size() * sizeof(float2)));
        FTCG_CK(cudaMemcpy(c.tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
        c.n_col_items = (int)col_items[ci].size();
        if (c.n_col_items > 0) {
            FTCG_CK(cudaMalloc(&c.col_items, col_items[ci].size() * sizeof(int2)));
            FTCG_CK(cudaMemcpy(c.col_items, col_items[ci].data(), col_items[ci].size() * sizeof(int2),
                               cudaMemcpyHostToDevice));
        }
        FTCG_CK(cudaMalloc(&c.pings, cls_pings[ci].size() * sizeof(int)));
        FTCG_CK(cudaMemcpy(c.pings, cls_pings[ci].data(), cls_pings[ci].size() * sizeof(int),
                           cudaMemcpyHostToDevice));
        b.device_bytes += (int64_t)(tw.size() * sizeof(float2) +
                                    col_items[ci].size() * sizeof(int2) +
                                    cls_pings[ci].size() * sizeof(int));
    }
    auto heavy_first = [](const Item& x, const Item& y) { return x.cnt > y.cnt; };
    std::stable_sort(items.begin(), items.end(), heavy_first);
    std::stable_sort(items_mma.begin(), items_mma.end(), [](const Item& x, const Item& y) {
        return x.grp != y.grp ? x.grp < y.grp : x.cnt > y.cnt;
    });
    b.n_mma = (int)items_mma.size();
    for (int k = 0; k <= kTcGroups; ++k) b.tc_off[k] = 0;
    for (const Item& x : items_mma) ++b.tc_off[x.grp + 1];
    for (int k = 0; k < kTcGroups; ++k) b.tc_off[k + 1] += b.tc_off[k];
    b.nitems = (int)(items_mma.size() + items.size());
    std::vector<int2> it2;
    it2.reserve(b.nitems);
    for (const Item& x : items_mma) it2.push_back(make_int2(x.ping, x.tile));
    for (const Item& x : items) it2.push_back(make_int2(x.ping, x.tile));
    FTCG_CK(cudaMalloc(&b.d_items, std::max<size_t>(1, it2.size()) * sizeof(int2)));
    if (!it2.empty())
        FTCG_CK(cudaMemcpy(b.d_items, it2.data(), it2.size() * sizeof(int2), cudaMemcpyHostToDevice));
    FTCG_CK(cudaMalloc(&b.d_counter, (kTcGroups + 1) * sizeof(int)));
    std::vector<int2> halo_it;      // the fix-up's items: non-empty tiles of halo-layout pings
    for (const std::vector<Item>* list : {&items_mma, &items})
        for (const Item& x : *list)
            if (x.cnt > 0 && b.pings[x.ping]->bin.halo) halo_it.push_back(make_int2(x.ping, x.tile));
    b.n_halo = (int)halo_it.size();
    if (b.n_halo > 0) {
        FTCG_CK(cudaMalloc(&b.d_halo_items, halo_it.size() * sizeof(int2)));
        FTCG_CK(cudaMemcpy(b.d_halo_items, halo_it.data(), halo_it.size() * sizeof(int2),
                           cudaMemcpyHostToDevice));
        b.device_bytes += (int64_t)(halo_it.size() * sizeof(int2));
    }
    b.device_bytes += (int64_t)(it2.size() * sizeof(int2) + b.n * sizeof(PingDesc));
    return FTCG_SUCCESS;
}

ftcg_status_t check_ptr_array(const void* const* a, int n, const char* what) {
    if (!a) {
        set_error("%s: pointer array is NULL", what);
        return FTCG_ERR_INVALID_VALUE;
    }
    for (int i = 0; i < n; ++i)
        if (!a[i]) {
            set_error("%s: pointer %d is NULL", what, i);
            return FTCG_ERR_INVALID_VALUE;
        }
    return FTCG_SUCCESS;
}

// Spreading-stage time of one candidate over a sub-batch of pings (values: zeros).
ftcg_status_t time_batch_candidate(const Batch& parent, const TuneVal& c,
                                   const std::vector<const double*>& L,
                                   const std::vector<int64_t>& m, const std::vector<int32_t>& n,
                                   const void* zeros, cudaStream_t s, float* ms) {
    Batch* sub = new (std::nothrow) Batch();
    if (!sub) {
        set_error("tuner: host allocation failed");
        return FTCG_ERR_OUT_OF_MEMORY;
    }
    sub->n = (int)L.size();
    sub->w = parent.w;
    sub->sigma = parent.sigma;
    sub->opts = parent.opts;
    sub->opts.tile = c.T;
    sub->opts.layout = c.layout;
    sub->opts.spread_kernel = c.skern;
    sub->last = s;
    ftcg_status_t st = plan_batch_impl(*sub, L.data(), m.data(), n.data(), s);
    if (st == FTCG_SUCCESS) {
        for (int i = 0; i < sub->n; ++i) sub->h_desc[i].vals = zeros;
        EventPair ev;
        cudaError_t ce = cudaMemcpyAsync(sub->d_desc, sub->h_desc, sub->n * sizeof(PingDesc),
                                         cudaMemcpyHostToDevice, s);
        if (ce == cudaSuccess) ce = cudaEventCreate(&ev.a);
        if (ce == cudaSuccess) ce = cudaEventCreate(&ev.b);
        if (ce != cudaSuccess) {
            set_error("tuner: %s", cudaGetErrorString(ce));
            st = FTCG_ERR_CUDA;
        }
        if (st == FTCG_SUCCESS) st = batch_spread(*sub, false, s);               // warm-up
        if (st == FTCG_SUCCESS) {
            cudaError_t e = cudaEventRecord(ev.a, s);
            for (int r = 0; r < 3 && e == cudaSuccess && st == FTCG_SUCCESS; ++r)
                st = batch_spread(*sub, false, s);
            if (e == cudaSuccess && st == FTCG_SUCCESS) e = cudaEventRecord(ev.b, s);
            if (e == cudaSuccess && st == FTCG_SUCCESS) e = cudaEventSynchronize(ev.b);
            if (e == cudaSuccess && st == FTCG_SUCCESS) e = cudaEventElapsedTime(ms, ev.a, ev.b);
            if (e != cudaSuccess) {
                set_error("tuner: %s", cudaGetErrorString(e));
                st = FTCG_ERR_CUDA;
            }
        }
    }
    release_batch(sub);
    return st;
}

// The batch tuner: one (tile side, layout, kernel) for all pings whose tuner key (grid side, w,
// precision, half-octave density bucket, the caller's fixed choices) is not decided yet. Each
// candidate is timed as the persistent spreading launch over a sample of up to kTuneBatchPings of
// those pings (evenly spaced in the order of decreasing sample count, so that the sample has the
// batch's mix of sizes), planned for that candidate; the fastest is recorded for every undecided
// key. Timing the mix, not each key's pings alone, matters: most keys of a batch hold one or two
// pings, and a launch over so few measures how one small ping fills the GPU rather than what it
// costs inside the whole batch's launch. Batches without samples take the first candidate.
constexpr int kTuneBatchPings = 16;

ftcg_status_t tune_batch(const Batch& b, const double* const* d_lambda, const int64_t* M,
                         const int32_t* N, cudaStream_t s) {
    std::set<TuneKey> keys;
    std::vector<int> todo;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (int i = 0; i < b.n; ++i) {
            const TuneKey k = batch_key(b, M[i], (int)std::llround(b.sigma * N[i]));
            if (g_tune.count(k)) continue;
            keys.insert(k);
            if (M[i] > 0) todo.push_back(i);
        }
    }
    if (keys.empty()) return FTCG_SUCCESS;
    const std::vector<TuneVal> cand = tune_candidates(b.w, b.sigma, b.opts);
    TuneVal best = cand[0];
    if (cand.size() > 1 && !todo.empty()) {
        std::stable_sort(todo.begin(), todo.end(), [&](int x, int y) { return M[x] > M[y]; });
        const int size = (int)todo.size();
        const int k = std::min(size, kTuneBatchPings);
        std::vector<const double*> L(k);
        std::vector<int64_t> m(k);
        std::vector<int32_t> n(k);
        int64_t max_m = 1;
        for (int j = 0; j < k; ++j) {
            const int i = todo[(int64_t)j * size / k];
            L[j] = d_lambda[i];
            m[j] = M[i];
            n[j] = N[i];
            max_m = std::max(max_m, M[i]);
        }
        DevBuf zbuf;
        FTCG_CK(cudaMalloc(&zbuf.p, (size_t)max_m * sizeof(float2)));
        FTCG_CK(cudaMemsetAsync(zbuf.p, 0, (size_t)max_m * sizeof(float2), s));
        float best_ms = 1e30f;
        for (const TuneVal& c : cand) {
            float ms = 1e30f;
            FTCG_TRY(time_batch_candidate(b, c, L, m, n, zbuf.p, s, &ms));
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const TuneKey& k : keys) g_tune.emplace(k, best);
    return FTCG_SUCCESS;
}

}  // namespace
}  // namespace ftcg

using namespace ftcg;

extern "C" {

ftcg_status_t ftcg_plan_batch(ftcg_batch_t* out, int32_t n, const double* const* d_lambda,
                              const int64_t* M, const int32_t* N, double sigma, int32_t w,
                              const ftcg_opts_t* opts, ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!out) {
        set_error("ftcg_plan_batch: out is NULL");
        return FTCG_ERR_INVALID_VALUE;
    }
    *out = nullptr;
    if (n < 1 || !d_lambda || !M || !N) {
        set_error("ftcg_plan_batch: n >= 1 and non-NULL arrays are required");
        return FTCG_ERR_INVALID_VALUE;
    }
    ftcg_opts_t o{};
    if (opts) o = *opts;
    if (o.deterministic) {
        set_error("ftcg_plan_batch: opts.deterministic is for single plans (ftcg_plan)");
        return FTCG_ERR_NOT_SUPPORTED;
    }
    for (int i = 0; i < n; ++i) {
        if (M[i] < 0 || (M[i] > 0 && !d_lambda[i])) {
            set_error("ftcg_plan_batch: ping %d has a bad sample count or NULL coordinates", i);
            return FTCG_ERR_INVALID_VALUE;
        }
        ftcg_opts_t oi = o;                    // the checks of ftcg_plan, ping by ping
        ftcg_status_t st = validate_plan_args(M[i], N[i], sigma, w, &oi);
        if (st != FTCG_SUCCESS) return st;
    }
    Batch* b = new (std::nothrow) Batch();
    if (!b) {
        set_error("ftcg_plan_batch: host allocation failed");
        return FTCG_ERR_OUT_OF_MEMORY;
    }
    b->n = n;
    b->w = w;
    b->sigma = sigma;
    b->opts = o;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    b->last = s;
    ftcg_status_t st = plan_batch_impl(*b, d_lambda, M, N, s);
    if (st != FTCG_SUCCESS) {
        release_batch(b);
        return st;
    }
    *out = reinterpret_cast<ftcg_batch_t>(b);
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_batch_set_weights(ftcg_batch_t batch, const void* const* d_alpha,
                                     int32_t dtype, ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!batch) {
        set_error("ftcg_batch_set_weights: batch is NULL");
        return FTCG_ERR_INVALID_VALUE;
    }
    if (dtype != FTCG_WEIGHTS_F64 && dtype != FTCG_WEIGHTS_F32) {
        set_error("ftcg_batch_set_weights: bad dtype");
        return FTCG_ERR_INVALID_VALUE;
    }
    Batch* b = reinterpret_cast<Batch*>(batch);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    b->last = s;
    for (int i = 0; i < b->n; ++i)
        FTCG_TRY(launch_set_alpha(*b->pings[i], d_alpha ? d_alpha[i] : nullptr, dtype, s));
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_batch_weights(ftcg_batch_t batch, double* const* d_alpha_out,
                                 ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!batch) {
        set_error("ftcg_batch_weights: batch is NULL");
        return FTCG_ERR_INVALID_VALUE;
    }
    Batch* b = reinterpret_cast<Batch*>(batch);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    b->last = s;
    ftcg_status_t worst = FTCG_SUCCESS;
    for (int i = 0; i < b->n; ++i) {
        ftcg_status_t st = compute_weights(*b->pings[i], d_alpha_out ? d_alpha_out[i] : nullptr, s);
        if (st == FTCG_ERR_NUMERIC) worst = st;
        else if (st != FTCG_SUCCESS) return st;
    }
    return worst;
    FTCG_API_END
}

ftcg_status_t ftcg_adjoint_batch(ftcg_batch_t batch, const void* const* d_values, int32_t vdtype,
                                 void* const* d_images, ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!batch) {
        set_error("ftcg_adjoint_batch: batch is NULL");
        return FTCG_ERR_INVALID_VALUE;
    }
    Batch* b = reinterpret_cast<Batch*>(batch);
    if (vdtype != FTCG_VALUES_C64 && vdtype != FTCG_VALUES_BF16X2) {
        set_error("ftcg_adjoint_batch: unknown value dtype %d", vdtype);
        return FTCG_ERR_INVALID_VALUE;
    }
    FTCG_TRY(check_ptr_array(d_images, b->n, "ftcg_adjoint_batch images"));
    if (!d_values) {
        set_error("ftcg_adjoint_batch: values pointer array is NULL");
        return FTCG_ERR_INVALID_VALUE;
    }
    for (int i = 0; i < b->n; ++i)
        if (b->pings[i]->M > 0 && !d_values[i]) {
            set_error("ftcg_adjoint_batch: values pointer %d is NULL", i);
            return FTCG_ERR_INVALID_VALUE;
        }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    b->last = s;
    return batch_enqueue(*b, d_values, vdtype, d_images, s, true);
    FTCG_API_END
}

ftcg_status_t ftcg_batch_weights_judge(ftcg_batch_t batch, const double* const* d_alpha, int32_t K,
                                      double max_rel_err, int32_t* h_accepted, double* h_stats,
                                      ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!batch) {
        set_error("ftcg_batch_weights_judge: batch is NULL");
        return FTCG_ERR_INVALID_VALUE;
    }
    Batch* b = reinterpret_cast<Batch*>(batch);
    FTCG_TRY(check_ptr_array(reinterpret_cast<const void* const*>(d_alpha), b->n,
                             "ftcg_batch_weights_judge weights"));
    if (K < 1 || K > 65536 || !(max_rel_err >= 0.0)) {
        set_error("ftcg_batch_weights_judge: K must be in 1..65536 and max_rel_err >= 0");
        return FTCG_ERR_INVALID_VALUE;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    b->last = s;
    // every ping's sums in flight together, one read-back, then the verdicts
    std::vector<int> Ks(b->n);
    std::vector<size_t> off(b->n + 1, 0);
    for (int i = 0; i < b->n; ++i) {
        Ks[i] = (int)std::min<int64_t>(K, b->pings[i]->M);
        off[i + 1] = off[i] + 2 * (size_t)Ks[i];
    }
    double* d = nullptr;
    FTCG_CK(pool_malloc(&d, std::max<size_t>(1, off[b->n]) * sizeof(double), s));
    for (int i = 0; i < b->n; ++i)
        if (Ks[i] > 0)
            FTCG_TRY(judge_launch(*b->pings[i], d_alpha[i], Ks[i], d + off[i], d + off[i] + Ks[i],
                                  s));
    std::vector<double> h(std::max<size_t>(1, off[b->n]));
    FTCG_CK(cudaMemcpyAsync(h.data(), d, off[b->n] * sizeof(double), cudaMemcpyDeviceToHost, s));
    FTCG_CK(cudaStreamSynchronize(s));
    FTCG_CK(pool_free(d, s));
    for (int i = 0; i < b->n; ++i) {
        double st[3] = {1.0, 0.0, 0.0};
        bool ok = true;
        if (Ks[i] > 0) ok = judge_decide(h.data() + off[i], h.data() + off[i] + Ks[i], Ks[i],
                                         max_rel_err, st);
        if (h_accepted) h_accepted[i] = ok ? 1 : 0;
        if (h_stats)
            for (int k = 0; k < 3; ++k) h_stats[3 * i + k] = st[k];
        if (b->pings[i]->M > 0) FTCG_TRY(judge_install(*b->pings[i], d_alpha[i], ok, st[0], s));
    }
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_batch_profile(ftcg_batch_t batch, int32_t enable) {
    FTCG_API_BEGIN
    clear_error();
    if (!batch) {
        set_error("ftcg_batch_profile: batch is NULL");
        return FTCG_ERR_INVALID_VALUE;
    }
    Batch* b = reinterpret_cast<Batch*>(batch);
    if (enable && b->prof_ev.empty()) {
        b->prof_ev.reserve(3 * kBatchProfiled);
        for (int i = 0; i < 3 * kBatchProfiled; ++i) {
            cudaEvent_t e = nullptr;
            cudaError_t ce = cudaEventCreate(&e);
            if (ce != cudaSuccess) {
                for (cudaEvent_t x : b->prof_ev) cudaEventDestroy(x);
                b->prof_ev.clear();
                set_error("ftcg_batch_profile: cudaEventCreate: %s", cudaGetErrorString(ce));
                return FTCG_ERR_CUDA;
            }
            b->prof_ev.push_back(e);
        }
    }
    b->profiling = enable != 0;
    b->prof_calls = 0;
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_batch_stage_times(ftcg_batch_t batch, float* ms, int32_t* calls) {
    FTCG_API_BEGIN
    clear_error();
    if (!batch || !ms) {
        set_error("ftcg_batch_stage_times: NULL argument");
        return FTCG_ERR_INVALID_VALUE;
    }
    Batch* b = reinterpret_cast<Batch*>(batch);
    const int n = b->prof_calls;
    ms[0] = ms[1] = 0.f;
    if (calls) *calls = n;
    if (n == 0) return FTCG_SUCCESS;
    FTCG_CK(cudaEventSynchronize(b->prof_ev[3 * (n - 1) + 2]));
    double acc[2] = {0, 0};
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 2; ++k) {
            float t = 0.f;
            FTCG_CK(cudaEventElapsedTime(&t, b->prof_ev[3 * i + k], b->prof_ev[3 * i + k + 1]));
            acc[k] += t;
        }
    for (int k = 0; k < 2; ++k) ms[k] = (float)(acc[k] / n);
    b->prof_calls = 0;
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_batch_capture(ftcg_batch_t batch, const void* const* d_values, int32_t vdtype,
                                 void* const* d_images, ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!batch) {
        set_error("ftcg_batch_capture: batch is NULL");
        return FTCG_ERR_INVALID_VALUE;
    }
    Batch* b = reinterpret_cast<Batch*>(batch);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!s) {
        set_error("ftcg_batch_capture: capture needs a non-default stream");
        return FTCG_ERR_INVALID_VALUE;
    }
    // first a plain run: sets the kernel attributes and the persistent grid size outside capture
    FTCG_TRY(ftcg_adjoint_batch(batch, d_values, vdtype, d_images, stream));
    FTCG_CK(cudaStreamSynchronize(s));
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    FTCG_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    ftcg_status_t st = batch_enqueue(*b, d_values, vdtype, d_images, s);
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != FTCG_SUCCESS) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    FTCG_CK(e);
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    FTCG_CK(e);
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_batch_launch(ftcg_batch_t batch, ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!batch) {
        set_error("ftcg_batch_launch: batch is NULL");
        return FTCG_ERR_INVALID_VALUE;
    }
    Batch* b = reinterpret_cast<Batch*>(batch);
    if (!b->gexec) {
        set_error("ftcg_batch_launch: no captured graph (call ftcg_batch_capture first)");
        return FTCG_ERR_INVALID_VALUE;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    b->last = s;
    FTCG_CK(cudaGraphLaunch(b->gexec, s));
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_batch_info(ftcg_batch_t batch, int32_t* tiles, int64_t* entries,
                              int64_t* device_bytes) {
    FTCG_API_BEGIN
    clear_error();
    if (!batch) {
        set_error("ftcg_batch_info: batch is NULL");
        return FTCG_ERR_INVALID_VALUE;
    }
    Batch* b = reinterpret_cast<Batch*>(batch);
    if (tiles)
        for (int i = 0; i < b->n; ++i) tiles[i] = b->pings[i]->bin.T;
    if (entries) *entries = b->entries;
    if (device_bytes) *device_bytes = b->device_bytes;
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_batch_destroy(ftcg_batch_t batch) {
    FTCG_API_BEGIN
    clear_error();
    release_batch(reinterpret_cast<Batch*>(batch));
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_tuner_save(const char* path) {
    FTCG_API_BEGIN
    clear_error();
    if (!path) {
        set_error("ftcg_tuner_save: path is NULL");
        return FTCG_ERR_INVALID_VALUE;
    }
    std::map<TuneKey, TuneVal> snap;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        snap = g_tune;
    }
    FILE* f = std::fopen(path, "w");
    if (!f) {
        set_error("ftcg_tuner_save: cannot open %s for writing", path);
        return FTCG_ERR_INVALID_VALUE;
    }
    std::fprintf(f, "{\"ftcg_tuner\": 1, \"entries\": [\n");
    size_t k = 0;
    for (const auto& e : snap) {
        std::fprintf(f,
                     "{\"G\": %d, \"w\": %d, \"precision\": %d, \"bucket\": %d, "
                     "\"tile_req\": %d, \"layout_req\": %d, \"spread_req\": %d, "
                     "\"batch\": %d, \"window\": %d, \"tile\": %d, \"layout\": %d, "
                     "\"spread\": %d}%s\n",
                     e.first.G, e.first.w, e.first.prec, e.first.bucket, e.first.tile,
                     e.first.layout, e.first.skern, e.first.batch, e.first.win, e.second.T,
                     e.second.layout, e.second.skern, ++k < snap.size() ? "," : "");
    }
    std::fprintf(f, "]}\n");
    if (std::fclose(f) != 0) {
        set_error("ftcg_tuner_save: writing %s failed", path);
        return FTCG_ERR_INVALID_VALUE;
    }
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_tuner_load(const char* path) {
    FTCG_API_BEGIN
    clear_error();
    if (!path) {
        set_error("ftcg_tuner_load: path is NULL");
        return FTCG_ERR_INVALID_VALUE;
    }
    FILE* f = std::fopen(path, "r");
    if (!f) {
        set_error("ftcg_tuner_load: cannot open %s", path);
        return FTCG_ERR_INVALID_VALUE;
    }
    std::vector<std::pair<TuneKey, TuneVal>> got;
    std::string line;
    bool header = false, bad = false;
    int lineno = 0;
    for (int c; !bad;) {
        line.clear();
        while ((c = std::fgetc(f)) != EOF && c != '\n') line.push_back((char)c);
        if (c == EOF && line.empty()) break;
        ++lineno;
        if (line.find("\"ftcg_tuner\": 1") != std::string::npos) header = true;
        if (line.find("\"G\":") == std::string::npos) continue;
        TuneKey k{};
        int tile = 0, layout = 0, spread = FTCG_SPREAD_AUTO;
        if (!json_int(line, "spread_req", &k.skern)) k.skern = FTCG_SPREAD_AUTO;   // older files
        if (!json_int(line, "spread", &spread)) spread = FTCG_SPREAD_AUTO;
        if (!json_int(line, "batch", &k.batch)) k.batch = 0;
        if (!json_int(line, "window", &k.win)) k.win = FTCG_WINDOW_ES;
        const bool ok = json_int(line, "G", &k.G) && json_int(line, "w", &k.w) &&
                        json_int(line, "precision", &k.prec) &&
                        json_int(line, "bucket", &k.bucket) &&
                        json_int(line, "tile_req", &k.tile) &&
                        json_int(line, "layout_req", &k.layout) && json_int(line, "tile", &tile) &&
                        json_int(line, "layout", &layout);
        const bool valid = ok && k.G >= 2 && (k.G & 1) == 0 && k.w >= 2 && k.w <= 16 &&
                           (k.prec == FTCG_PREC_FP32 || k.prec == FTCG_PREC_BF16) &&
                           (k.tile == 0 || k.tile == 32 || k.tile == 64) &&
                           (k.layout >= FTCG_LAYOUT_AUTO && k.layout <= FTCG_LAYOUT_HALO) &&
                           (k.skern >= FTCG_SPREAD_AUTO && k.skern <= FTCG_SPREAD_BLOCK) &&
                           (k.skern < FTCG_SPREAD_TENSOR || layout == FTCG_LAYOUT_HALO) &&
                           (spread >= FTCG_SPREAD_AUTO && spread <= FTCG_SPREAD_BLOCK) &&
                           (spread < FTCG_SPREAD_TENSOR || layout == FTCG_LAYOUT_HALO) &&
                           (k.skern == FTCG_SPREAD_AUTO || spread == k.skern) &&
                           (k.batch == 0 || k.batch == 1) &&
                           (k.win >= FTCG_WINDOW_ES && k.win <= FTCG_WINDOW_GAUSS) &&
                           (tile == 32 || tile == 64) &&
                           (layout == FTCG_LAYOUT_DUPLICATE || layout == FTCG_LAYOUT_HALO) &&
                           (k.tile == 0 || k.tile == tile) && (k.layout == 0 || k.layout == layout);
        if (!valid) {
            set_error("ftcg_tuner_load: %s line %d is not a valid tuner entry", path, lineno);
            bad = true;
            break;
        }
        got.push_back({k, TuneVal{tile, layout, spread}});
    }
    std::fclose(f);
    if (bad) return FTCG_ERR_INVALID_VALUE;
    if (!header) {
        set_error("ftcg_tuner_load: %s is not a tuner file", path);
        return FTCG_ERR_INVALID_VALUE;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& e : got) g_tune[e.first] = e.second;
    return FTCG_SUCCESS;
    FTCG_API_END
}

}  // extern "C"
