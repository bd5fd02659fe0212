// The C ABI (include/ftcg.h): argument validation, plan lifecycle and the call sequences of the
// weighted adjoint (Eq. twodcg): spread -> inverse FFT (cuFFT C2C) -> window division + crop.

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "ftcg_internal.cuh"

namespace ftcg {

namespace {
thread_local char g_err[512];
}

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

}  // namespace ftcg

using namespace ftcg;

namespace {

ftcg_status_t invalid(const char* msg) {
    set_error("%s", msg);
    return FTCG_ERR_INVALID_VALUE;
}

}  // namespace

namespace ftcg {

void release_plan(Plan* p) {
    if (!p) return;
    cudaDeviceSynchronize();
    free_binning(p->bin);
    if (p->lambda) cudaFree(p->lambda);
    if (p->samp) cudaFree(p->samp);
    if (p->deapod) cudaFree(p->deapod);
    if (p->deapod2) cudaFree(p->deapod2);
    if (p->grid) cudaFree(p->grid);
    if (p->status) cudaFree(p->status);
    if (p->stage_vals) cudaFree(p->stage_vals);
    if (p->alpha_cur) cudaFree(p->alpha_cur);
    release_band(p);
    if (p->stage_img) cudaFree(p->stage_img);
    for (int k = 0; k < 2; ++k) {
        if (p->pipe_vals[k]) cudaFree(p->pipe_vals[k]);
        if (p->pipe_up[k]) cudaEventDestroy(p->pipe_up[k]);
        if (p->pipe_used[k]) cudaEventDestroy(p->pipe_used[k]);
    }
    if (p->pipe_copy) cudaStreamDestroy(p->pipe_copy);
    if (p->fft_ok) cufftDestroy(p->fft);
    release_pruned_fft(p);
    if (p->prof_ev) {
        for (int i = 0; i < kMaxProfiled * 4; ++i) cudaEventDestroy(p->prof_ev[i]);
        delete[] p->prof_ev;
    }
    delete p;
}

ftcg_status_t make_plan(Plan* p, const double* d_lambda, cudaStream_t s, bool own_grid) {
    int64_t bytes = 0;
    const int64_t M = p->M;
    FTCG_CK(pool_malloc(&p->status, sizeof(unsigned), s));
    FTCG_CK(cudaMemsetAsync(p->status, 0, sizeof(unsigned), s));
    if (M > 0) {
        FTCG_CK(pool_malloc(&p->lambda, (size_t)M * 2 * sizeof(double), s));
        FTCG_CK(cudaMemcpyAsync(p->lambda, d_lambda, (size_t)M * 2 * sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
        FTCG_CK(pool_malloc(&p->samp, (size_t)M * sizeof(int4), s));
        bytes += (int64_t)M * (2 * sizeof(double) + sizeof(int4));
    }
    FTCG_CK(pool_malloc(&p->deapod, (size_t)p->N * sizeof(double), s));
    bytes += (int64_t)p->N * sizeof(double);
    FTCG_TRY(window_factors(p->deapod, p->N, p->G, p->win, s));
    FTCG_CK(pool_malloc(&p->deapod2, (size_t)p->N * sizeof(float2), s));
    bytes += (int64_t)p->N * sizeof(float2);
    FTCG_TRY(split_factors(p->deapod, p->deapod2, p->N, s));
    p->bin.det = p->opts.deterministic != 0;
    FTCG_TRY(build_binning(p->bin, p->lambda, M, p->sigma, p->G, p->opts.tile, p->w,
                           p->opts.layout == FTCG_LAYOUT_HALO, p->status, p->samp, s, &bytes));
    if (p->bin.halo && p->opts.spread_kernel != FTCG_SPREAD_WINDOW && p->w <= kMmaMaxW) {
        double err = 0;
        if (mma_window_poly(p->w, p->win.beta, p->win.kind, &p->bin.poly, &err))
            // AUTO (tile side and layout given, so no tuner): the block kernel, the faster one
            FTCG_TRY(build_chunks(p->bin, s, &bytes,
                                  p->opts.spread_kernel != FTCG_SPREAD_TENSOR));
    }
    if (own_grid) {
        FTCG_CK(pool_malloc(&p->grid, (size_t)p->G * p->G * sizeof(float2), s));
        bytes += (int64_t)p->G * p->G * sizeof(float2);
        // the full 2-D plan serves only the forward operator: created on its first call
        FTCG_TRY(build_pruned_fft(p, s, &bytes));
    }
    p->device_bytes = bytes;
    unsigned st = 0;
    FTCG_CK(cudaMemcpyAsync(&st, p->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    FTCG_CK(cudaStreamSynchronize(s));
    if (st & STATUS_NONFINITE_COORD) {
        FTCG_CK(cudaMemsetAsync(p->status, 0, sizeof(unsigned), s));
        set_error("ftcg_plan: some coordinates are not finite (or |sigma lambda| >= 2^50); those "
                  "samples are dropped");
        return FTCG_ERR_NUMERIC;
    }
    return FTCG_SUCCESS;
}

ftcg_status_t validate_plan_args(int64_t M, int32_t N, double sigma, int32_t w, ftcg_opts_t* po) {
    if (M < 0) return invalid("ftcg_plan: M < 0");
    if (N < 2 || (N & 1)) return invalid("ftcg_plan: N must be even and >= 2");
    if (!(sigma >= 1.0) || !std::isfinite(sigma)) return invalid("ftcg_plan: sigma must be >= 1");
    if (w < 2 || w > 16) return invalid("ftcg_plan: w must be in 2..16");
    const double Gd = sigma * N;
    const long long G = std::llround(Gd);
    if (std::fabs(Gd - (double)G) > 1e-9 * Gd || (G & 1))
        return invalid("ftcg_plan: sigma * N must be an even integer");
    if (G < 2 * w) return invalid("ftcg_plan: the grid must hold at least two windows (G >= 2 w)");
    ftcg_opts_t& o = *po;
    if (o.reserved != 0) return invalid("ftcg_plan: opts.reserved must be zero");
    if (o.deterministic != 0 && o.deterministic != 1)
        return invalid("ftcg_plan: opts.deterministic must be 0 or 1");
    if (o.deterministic) {
        // one fixed configuration: the block kernel, halo layout, T = 32 (or the given 64)
        if (o.layout == FTCG_LAYOUT_DUPLICATE ||
            (o.spread_kernel != FTCG_SPREAD_AUTO && o.spread_kernel != FTCG_SPREAD_BLOCK)) {
            set_error("ftcg_plan: opts.deterministic runs the block kernel in the halo layout");
            return FTCG_ERR_NOT_SUPPORTED;
        }
        o.layout = FTCG_LAYOUT_HALO;
        o.spread_kernel = FTCG_SPREAD_BLOCK;
        if (o.tile == 0) o.tile = 32;
        if (o.tile != 0 && o.tile != 32 && o.tile != 64)
            return invalid("ftcg_plan: opts.tile must be 0, 32 or 64");
        if (G % o.tile != 0) {
            set_error("ftcg_plan: opts.deterministic needs G = sigma N (%lld) to be a multiple "
                      "of the tile side %d", G, o.tile);
            return FTCG_ERR_NOT_SUPPORTED;
        }
    }
    if (o.layout < FTCG_LAYOUT_AUTO || o.layout > FTCG_LAYOUT_HALO)
        return invalid("ftcg_plan: opts.layout must be 0, 1 or 2");
    if (o.spread_kernel < FTCG_SPREAD_AUTO || o.spread_kernel > FTCG_SPREAD_BLOCK)
        return invalid("ftcg_plan: opts.spread_kernel must be 0, 1, 2 or 3");
    if (o.kernel < FTCG_WINDOW_ES || o.kernel > FTCG_WINDOW_GAUSS)
        return invalid("ftcg_plan: opts.kernel must be 0 (ES), 1 (Kaiser-Bessel) or 2 (Gaussian)");
    const double beta = kernel_beta(w, sigma, o.kernel);
    if (!std::isfinite(beta)) {
        set_error("ftcg_plan: no Kaiser-Bessel shape parameter for w = %d, sigma = %g "
                  "((w / sigma)^2 (sigma - 1/2)^2 <= 0.8)", w, sigma);
        return FTCG_ERR_NOT_SUPPORTED;
    }
    if (o.spread_kernel == FTCG_SPREAD_TENSOR || o.spread_kernel == FTCG_SPREAD_BLOCK) {
        MmaPoly poly;
        double err = 0;
        if (o.layout == FTCG_LAYOUT_DUPLICATE || w > kMmaMaxW ||
            !mma_window_poly(w, beta, o.kernel, &poly, &err)) {
            set_error("ftcg_plan: the tensor-core spreading kernel needs the halo layout, w <= 8 "
                      "and a window within 1e-6 of its tap polynomials (w = %d, sigma = %g: %.1e)",
                      w, sigma, err);
            return FTCG_ERR_NOT_SUPPORTED;
        }
    }
    if (o.precision != FTCG_PREC_FP32 && o.precision != FTCG_PREC_BF16)
        return invalid("ftcg_plan: opts.precision must be 0 (FP32) or 1 (BF16)");
    if (o.tile != 0 && o.tile != 32 && o.tile != 64)
        return invalid("ftcg_plan: opts.tile must be 0, 32 or 64");
    if (o.weight_width != 0 && (o.weight_width < 4 || o.weight_width > 16))
        return invalid("ftcg_plan: opts.weight_width must be 0 or 4..16");
    if (M > kMaxSamples) {
        set_error("ftcg_plan: M > %lld is beyond this build's entry format", (long long)kMaxSamples);
        return FTCG_ERR_NOT_SUPPORTED;
    }
    if (G > 65536 || N > 32768) {
        set_error("ftcg_plan: G = sigma N > 65536 or N > 32768 is not supported");
        return FTCG_ERR_NOT_SUPPORTED;
    }
    const int tmin = o.tile ? o.tile : 32;      // the smallest tile the autotuner may pick
    const long long ntx = (G + tmin - 1) / tmin;
    const long long ncb = (o.tile ? o.tile : 64) + w - 1;
    if (ntx * ntx * ncb * ncb >= (1LL << 31)) {
        set_error("ftcg_plan: the binning key space is too large for G = %lld", G);
        return FTCG_ERR_NOT_SUPPORTED;
    }
    return FTCG_SUCCESS;
}

}  // namespace ftcg

namespace ftcg {

// the full G x G C2C plan (forward operator; adjoint fallback), created on first use
ftcg_status_t ensure_full_fft(Plan* p) {
    if (p->fft_ok) return FTCG_SUCCESS;
    FTCG_CKFFT(cufftPlan2d(&p->fft, p->G, p->G, CUFFT_C2C));
    p->fft_ok = true;
    size_t ws = 0;
    if (cufftGetSize(p->fft, &ws) == CUFFT_SUCCESS) p->device_bytes += (int64_t)ws;
    return FTCG_SUCCESS;
}

ftcg_status_t adjoint_device(Plan* p, const void* vals, int32_t vdtype, void* img, cudaStream_t s,
                             bool use_band) {
    p->last_stream = s;
    if (use_band && p->band_r > 0 && p->M > 0) {
        if (vdtype != FTCG_VALUES_C64) {
            set_error("adjoint with banded coefficients: values must be complex64");
            return FTCG_ERR_NOT_SUPPORTED;
        }
        FTCG_TRY(band_apply(*p, vals, s));     // tau = C v, spread with unit weights
        vals = p->band_tau;
    }
    cudaEvent_t* ev = nullptr;
    if (p->profiling && p->prof_calls < kMaxProfiled) ev = p->prof_ev + 4 * p->prof_calls++;
    if (ev) FTCG_CK(cudaEventRecord(ev[0], s));
    FTCG_TRY(launch_spread(*p, vals, vdtype, p->grid, s, p->smem_fft));
    if (ev) FTCG_CK(cudaEventRecord(ev[1], s));
    if (p->smem_fft) {                         // both passes, the second writes the image
        FTCG_TRY(exec_smem_fft(p, reinterpret_cast<float2*>(img), s, ev ? ev[2] : nullptr));
        if (ev) FTCG_CK(cudaEventRecord(ev[3], s));
        return FTCG_SUCCESS;
    }
    if (p->pruned_ok) {
        FTCG_TRY(exec_pruned_inverse(p, s));
    } else {
        FTCG_TRY(ensure_full_fft(p));
        FTCG_CKFFT(cufftSetStream(p->fft, s));
        FTCG_CKFFT(cufftExecC2C(p->fft, reinterpret_cast<cufftComplex*>(p->grid),
                                reinterpret_cast<cufftComplex*>(p->grid), CUFFT_INVERSE));
    }
    if (ev) FTCG_CK(cudaEventRecord(ev[2], s));
    FTCG_TRY(launch_deapod_crop(*p, p->grid, reinterpret_cast<float2*>(img), s));
    if (ev) FTCG_CK(cudaEventRecord(ev[3], s));
    return FTCG_SUCCESS;
}

ftcg_status_t forward_device(Plan* p, const void* img, void* vals, cudaStream_t s) {
    p->last_stream = s;
    FTCG_TRY(ensure_full_fft(p));
    FTCG_TRY(launch_pad_apod(*p, reinterpret_cast<const float2*>(img), p->grid, s));
    FTCG_CKFFT(cufftSetStream(p->fft, s));
    FTCG_CKFFT(cufftExecC2C(p->fft, reinterpret_cast<cufftComplex*>(p->grid),
                            reinterpret_cast<cufftComplex*>(p->grid), CUFFT_FORWARD));
    return launch_interp(*p, p->grid, reinterpret_cast<float2*>(vals), s);
}

}  // namespace ftcg

namespace {

ftcg_status_t check_values(const Plan* p, const void* v, int32_t vdtype, const char* what) {
    if (vdtype != FTCG_VALUES_C64 && vdtype != FTCG_VALUES_BF16X2) {
        set_error("%s: unknown value dtype %d", what, vdtype);
        return FTCG_ERR_INVALID_VALUE;
    }
    if (p->M > 0 && !v) {
        set_error("%s: values pointer is NULL", what);
        return FTCG_ERR_INVALID_VALUE;
    }
    return FTCG_SUCCESS;
}

}  // namespace

extern "C" {

ftcg_status_t ftcg_plan(ftcg_plan_t* out, const double* d_lambda, int64_t M, int32_t N,
                        double sigma, int32_t w, const ftcg_opts_t* opts, ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!out) return invalid("ftcg_plan: out is NULL");
    *out = nullptr;
    if (M > 0 && !d_lambda) return invalid("ftcg_plan: d_lambda is NULL");
    ftcg_opts_t o{};
    if (opts) o = *opts;
    FTCG_TRY(validate_plan_args(M, N, sigma, w, &o));
    const long long G = std::llround(sigma * N);
    Plan* p = new (std::nothrow) Plan();
    if (!p) {
        set_error("ftcg_plan: host allocation failed");
        return FTCG_ERR_OUT_OF_MEMORY;
    }
    p->M = M;
    p->N = N;
    p->G = (int)G;
    p->w = w;
    p->sigma = sigma;
    p->opts = o;
    p->win = Window{w, kernel_beta(w, sigma, o.kernel), o.kernel};
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    p->last_stream = s;
    if (o.tile == 0 || o.layout == FTCG_LAYOUT_AUTO) {
        ftcg_status_t tst =
            tune_tile(d_lambda, M, N, sigma, w, o, s, &p->opts.tile, &p->opts.layout,
                      &p->opts.spread_kernel);
        if (tst != FTCG_SUCCESS) {
            delete p;
            return tst;
        }
    }
    ftcg_status_t st = make_plan(p, d_lambda, s, true);
    if (st != FTCG_SUCCESS && st != FTCG_ERR_NUMERIC) {
        release_plan(p);
        return st;
    }
    *out = reinterpret_cast<ftcg_plan_t>(p);
    return st;
    FTCG_API_END
}

ftcg_status_t ftcg_plan_info(ftcg_plan_t plan, ftcg_plan_info_t* info) {
    FTCG_API_BEGIN
    clear_error();
    if (!plan || !info) return invalid("ftcg_plan_info: NULL argument");
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    info->M = p->M;
    info->N = p->N;
    info->G = p->G;
    info->w = p->w;
    info->tile = p->bin.T;
    info->tiles_x = p->bin.ntx;
    info->layout = p->bin.halo ? FTCG_LAYOUT_HALO : FTCG_LAYOUT_DUPLICATE;
    info->entries = p->bin.n_entries;
    info->beta = p->win.beta;
    info->device_bytes = p->device_bytes;
    info->spread_kernel = !p->bin.mma ? FTCG_SPREAD_WINDOW
                          : p->bin.blk ? FTCG_SPREAD_BLOCK
                                       : FTCG_SPREAD_TENSOR;
    info->pad0 = 0;
    info->chunks = p->bin.n_chunks;
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_weights(ftcg_plan_t plan, double* d_alpha_out, ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!plan) return invalid("ftcg_weights: plan is NULL");
    Plan* p = reinterpret_cast<Plan*>(plan);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    p->last_stream = s;
    release_band(p);                           // the diagonal weights replace a band
    return compute_weights(*p, d_alpha_out, s);
    FTCG_API_END
}

ftcg_status_t ftcg_set_weights(ftcg_plan_t plan, const void* d_alpha, int32_t dtype,
                               ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!plan) return invalid("ftcg_set_weights: plan is NULL");
    if (dtype != FTCG_WEIGHTS_F64 && dtype != FTCG_WEIGHTS_F32)
        return invalid("ftcg_set_weights: dtype must be FTCG_WEIGHTS_F64 or FTCG_WEIGHTS_F32");
    Plan* p = reinterpret_cast<Plan*>(plan);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    p->last_stream = s;
    release_band(p);                           // the diagonal weights replace a band
    return launch_set_alpha(*p, d_alpha, dtype, s);
    FTCG_API_END
}

ftcg_status_t ftcg_spread(ftcg_plan_t plan, const void* d_values, int32_t vdtype, void* d_grid,
                          ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!plan) return invalid("ftcg_spread: plan is NULL");
    Plan* p = reinterpret_cast<Plan*>(plan);
    FTCG_TRY(check_values(p, d_values, vdtype, "ftcg_spread"));
    if (!d_grid) return invalid("ftcg_spread: grid pointer is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    p->last_stream = s;
    return launch_spread(*p, d_values, vdtype, reinterpret_cast<float2*>(d_grid), s);
    FTCG_API_END
}

ftcg_status_t ftcg_adjoint(ftcg_plan_t plan, const void* d_values, int32_t vdtype, void* d_image,
                           ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!plan) return invalid("ftcg_adjoint: plan is NULL");
    Plan* p = reinterpret_cast<Plan*>(plan);
    FTCG_TRY(check_values(p, d_values, vdtype, "ftcg_adjoint"));
    if (!d_image) return invalid("ftcg_adjoint: image pointer is NULL");
    return adjoint_device(p, d_values, vdtype, d_image, reinterpret_cast<cudaStream_t>(stream));
    FTCG_API_END
}

ftcg_status_t ftcg_adjoint_host(ftcg_plan_t plan, const void* h_values, int32_t vdtype,
                                void* h_image, ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!plan) return invalid("ftcg_adjoint_host: plan is NULL");
    Plan* p = reinterpret_cast<Plan*>(plan);
    FTCG_TRY(check_values(p, h_values, vdtype, "ftcg_adjoint_host"));
    if (!h_image) return invalid("ftcg_adjoint_host: image pointer is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t vbytes = (size_t)p->M * (vdtype == FTCG_VALUES_C64 ? 8 : 4);
    const size_t ibytes = (size_t)p->N * p->N * sizeof(float2);
    if (!p->stage_vals && p->M > 0) FTCG_CK(pool_malloc(&p->stage_vals, (size_t)p->M * 8, s));
    // A page-locked (pinned or registered) image the device can address is written in place by
    // the last kernel (no staging copy, the transfer overlaps that kernel); any other host
    // memory goes through a device staging image and one copy.
    void* img_dev = nullptr;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, h_image) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer) {
        img_dev = at.devicePointer;
    } else {
        cudaGetLastError();
        if (!p->stage_img) FTCG_CK(pool_malloc(&p->stage_img, ibytes, s));
    }
    if (vbytes) FTCG_CK(cudaMemcpyAsync(p->stage_vals, h_values, vbytes, cudaMemcpyHostToDevice, s));
    if (img_dev) {
        FTCG_TRY(adjoint_device(p, p->stage_vals, vdtype, img_dev, s));
    } else {
        FTCG_TRY(adjoint_device(p, p->stage_vals, vdtype, p->stage_img, s));
        FTCG_CK(cudaMemcpyAsync(h_image, p->stage_img, ibytes, cudaMemcpyDeviceToHost, s));
    }
    FTCG_CK(cudaStreamSynchronize(s));
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_adjoint_host_async(ftcg_plan_t plan, const void* h_values, int32_t vdtype,
                                      void* h_image, ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!plan) return invalid("ftcg_adjoint_host_async: plan is NULL");
    Plan* p = reinterpret_cast<Plan*>(plan);
    FTCG_TRY(check_values(p, h_values, vdtype, "ftcg_adjoint_host_async"));
    if (!h_image) return invalid("ftcg_adjoint_host_async: image pointer is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    p->last_stream = s;
    const size_t vbytes = (size_t)p->M * (vdtype == FTCG_VALUES_C64 ? 8 : 4);
    const size_t ibytes = (size_t)p->N * p->N * sizeof(float2);
    if (!p->pipe_copy) {
        FTCG_CK(cudaStreamCreateWithFlags(&p->pipe_copy, cudaStreamNonBlocking));
        for (int k = 0; k < 2; ++k) {
            FTCG_CK(cudaEventCreateWithFlags(&p->pipe_up[k], cudaEventDisableTiming));
            FTCG_CK(cudaEventCreateWithFlags(&p->pipe_used[k], cudaEventDisableTiming));
            if (p->M > 0) FTCG_CK(cudaMalloc(&p->pipe_vals[k], (size_t)p->M * 8));
        }
    }
    void* img_dev = nullptr;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, h_image) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer) {
        img_dev = at.devicePointer;
    } else {
        cudaGetLastError();
        if (!p->stage_img) FTCG_CK(pool_malloc(&p->stage_img, ibytes, s));
    }
    const int k = p->pipe_next;
    p->pipe_next ^= 1;
    // upload into buffer k on the copy stream once the adjoint that last read it is done; the
    // adjoint on `stream` waits for the upload only, so the next call's upload overlaps it
    FTCG_CK(cudaStreamWaitEvent(p->pipe_copy, p->pipe_used[k], 0));
    if (vbytes)
        FTCG_CK(cudaMemcpyAsync(p->pipe_vals[k], h_values, vbytes, cudaMemcpyHostToDevice,
                                p->pipe_copy));
    FTCG_CK(cudaEventRecord(p->pipe_up[k], p->pipe_copy));
    FTCG_CK(cudaStreamWaitEvent(s, p->pipe_up[k], 0));
    if (img_dev) {
        FTCG_TRY(adjoint_device(p, p->pipe_vals[k], vdtype, img_dev, s));
    } else {
        FTCG_TRY(adjoint_device(p, p->pipe_vals[k], vdtype, p->stage_img, s));
        FTCG_CK(cudaMemcpyAsync(h_image, p->stage_img, ibytes, cudaMemcpyDeviceToHost, s));
    }
    FTCG_CK(cudaEventRecord(p->pipe_used[k], s));
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_forward(ftcg_plan_t plan, const void* d_image, void* d_values,
                           ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!plan) return invalid("ftcg_forward: plan is NULL");
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!d_image) return invalid("ftcg_forward: image pointer is NULL");
    if (p->M > 0 && !d_values) return invalid("ftcg_forward: values pointer is NULL");
    return forward_device(p, d_image, d_values, reinterpret_cast<cudaStream_t>(stream));
    FTCG_API_END
}

ftcg_status_t ftcg_check(ftcg_plan_t plan) {
    FTCG_API_BEGIN
    clear_error();
    if (!plan) return invalid("ftcg_check: plan is NULL");
    Plan* p = reinterpret_cast<Plan*>(plan);
    unsigned st = 0;
    FTCG_CK(cudaStreamSynchronize(p->last_stream));
    FTCG_CK(cudaGetLastError());
    FTCG_CK(cudaMemcpy(&st, p->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    FTCG_CK(cudaMemset(p->status, 0, sizeof(unsigned)));
    if (st) {
        set_error("device status 0x%x:%s%s", st,
                  (st & STATUS_NONFINITE_COORD) ? " non-finite coordinate" : "",
                  (st & STATUS_BAD_WEIGHT_SUM) ? " weight sum <= 0 or not finite" : "");
        return FTCG_ERR_NUMERIC;
    }
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_plan_entries(ftcg_plan_t plan, int32_t* h_tile, int32_t* h_cx, int32_t* h_cy,
                                int32_t* h_sample, float* h_dx, float* h_dy) {
    FTCG_API_BEGIN
    clear_error();
    if (!plan) return invalid("ftcg_plan_entries: plan is NULL");
    Plan* p = reinterpret_cast<Plan*>(plan);
    const Binning& b = p->bin;
    const int64_t n = b.n_entries;
    if (n == 0) return FTCG_SUCCESS;
    const int64_t nbins = (int64_t)b.ntiles * b.ncb;
    Entry* he = new (std::nothrow) Entry[n];
    int* hc = new (std::nothrow) int[nbins + 1];
    if (!he || !hc) {
        delete[] he;
        delete[] hc;
        set_error("ftcg_plan_entries: host allocation failed");
        return FTCG_ERR_OUT_OF_MEMORY;
    }
    cudaError_t e1 = cudaMemcpy(he, b.ent, n * sizeof(Entry), cudaMemcpyDeviceToHost);
    cudaError_t e2 = cudaMemcpy(hc, b.colptr, (nbins + 1) * sizeof(int), cudaMemcpyDeviceToHost);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        delete[] he;
        delete[] hc;
        set_error("ftcg_plan_entries: copy failed");
        return FTCG_ERR_CUDA;
    }
    int64_t bin = 0;
    for (int64_t i = 0; i < n; ++i) {
        while (bin + 1 <= nbins && hc[bin + 1] <= i) ++bin;
        const int tile = (int)(bin / b.ncb);
        const int cb = (int)(bin % b.ncb);
        if (h_tile) h_tile[i] = tile;
        if (h_cx) h_cx[i] = cb - (b.W - 1);
        if (h_cy) h_cy[i] = (int)(he[i].packed >> kSampleBits) - (b.W - 1);
        if (h_sample) h_sample[i] = (int)(he[i].packed & kSampleMask);
        if (h_dx) h_dx[i] = he[i].dx;
        if (h_dy) h_dy[i] = he[i].dy;
    }
    delete[] he;
    delete[] hc;
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_profile(ftcg_plan_t plan, int32_t enable) {
    FTCG_API_BEGIN
    clear_error();
    if (!plan) return invalid("ftcg_profile: plan is NULL");
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (enable && !p->prof_ev) {
        cudaEvent_t* ev = new (std::nothrow) cudaEvent_t[kMaxProfiled * 4];
        if (!ev) {
            set_error("ftcg_profile: host allocation failed");
            return FTCG_ERR_OUT_OF_MEMORY;
        }
        for (int i = 0; i < kMaxProfiled * 4; ++i) {
            cudaError_t e = cudaEventCreate(&ev[i]);
            if (e != cudaSuccess) {
                for (int k = 0; k < i; ++k) cudaEventDestroy(ev[k]);
                delete[] ev;
                set_error("ftcg_profile: cudaEventCreate: %s", cudaGetErrorString(e));
                return FTCG_ERR_CUDA;
            }
        }
        p->prof_ev = ev;
    }
    p->profiling = enable != 0;
    p->prof_calls = 0;
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_stage_times(ftcg_plan_t plan, float* ms, int32_t* calls) {
    FTCG_API_BEGIN
    clear_error();
    if (!plan || !ms) return invalid("ftcg_stage_times: NULL argument");
    Plan* p = reinterpret_cast<Plan*>(plan);
    const int n = p->prof_calls;
    ms[0] = ms[1] = ms[2] = 0.f;
    if (calls) *calls = n;
    if (n == 0) return FTCG_SUCCESS;
    FTCG_CK(cudaEventSynchronize(p->prof_ev[4 * (n - 1) + 3]));
    double acc[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) {
            float t = 0.f;
            FTCG_CK(cudaEventElapsedTime(&t, p->prof_ev[4 * i + k], p->prof_ev[4 * i + k + 1]));
            acc[k] += t;
        }
    }
    for (int k = 0; k < 3; ++k) ms[k] = (float)(acc[k] / n);
    p->prof_calls = 0;
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_destroy(ftcg_plan_t plan) {
    FTCG_API_BEGIN
    clear_error();
    release_plan(reinterpret_cast<Plan*>(plan));
    return FTCG_SUCCESS;
    FTCG_API_END
}

const char* ftcg_status_string(ftcg_status_t s) {
    switch (s) {
        case FTCG_SUCCESS: return "FTCG_SUCCESS";
        case FTCG_ERR_INVALID_VALUE: return "FTCG_ERR_INVALID_VALUE";
        case FTCG_ERR_OUT_OF_MEMORY: return "FTCG_ERR_OUT_OF_MEMORY";
        case FTCG_ERR_CUDA: return "FTCG_ERR_CUDA";
        case FTCG_ERR_NOT_SUPPORTED: return "FTCG_ERR_NOT_SUPPORTED";
        case FTCG_ERR_NUMERIC: return "FTCG_ERR_NUMERIC";
        case FTCG_ERR_TIMEOUT: return "FTCG_ERR_TIMEOUT";
    }
    return "FTCG_ERR_UNKNOWN";
}

const char* ftcg_last_error(void) { return g_err; }

// FTCG_SOURCE_HASH: a hash of the sources the library was built from (set by the build script;
// "unknown" when built otherwise), so that a library can be matched to its sources.
#ifndef FTCG_SOURCE_HASH
#define FTCG_SOURCE_HASH "unknown"
#endif
const char* ftcg_version(void) { return "ftcg 0.2 sm_103a ftcg-src-hash:" FTCG_SOURCE_HASH; }

}  // extern "C"
