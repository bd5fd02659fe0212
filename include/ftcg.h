/*
 * ftcg.h -- C ABI of the GB300 (sm_103a) frame theoretic convolutional gridding library.
 *
 * The library computes the weighted 2-D adjoint non-uniform Fourier transform at the heart of
 * frame theoretic convolutional gridding (FTCG, McKay, Gelb, Monga, Raj; Sec. IV, Eq. twodcg,
 * twodcgmatrix and twodftcg at band r = 1):
 *
 *     I_p = sum_j alpha_j v_j exp(+2 pi i lambda_j . p / N),   p in {-N/2 .. N/2-1}^2,
 *
 * approximated by convolutional gridding: the weighted samples alpha_j v_j (D_2 f^) are spread
 * with a width-w window onto a periodic sigma-oversampled G x G grid (Omega_2), G = sigma N,
 * transformed by an unnormalised inverse 2-D FFT (the sum over l in I_L of exp(2 pi i <l, x>)),
 * divided by the window's Fourier transform (zeta_n = psi_n / w(x), Eq. newadm) and cropped.
 *
 * Conventions shared by every call:
 *   - lambda: M x 2 float64, interleaved (x, y), cycles per field of view; any real value (the
 *     grid is periodic, lambda and lambda + N k give the same image).
 *   - values v: M complex samples in acquisition order, complex64 (interleaved float re, im) or
 *     bf16x2 (interleaved bfloat16 re, im).
 *   - image: N x N complex64, row-major, element (p_y + N/2) * N + (p_x + N/2).
 *   - fine grid: G x G complex64, row-major, element l_y * G + l_x, l in [0, G).
 *   - the window is the exponential of semicircle (ES) kernel
 *       phi(t) = exp(beta (sqrt(1 - (2t/w)^2) - 1)), |t| <= w/2, beta = 0.97 pi (1 - 1/(2 sigma)) w;
 *     taps are the w cells from ceil(sigma lambda - w/2) (mod G).
 *   - every call that takes a stream is asynchronous on it unless stated; device pointers must
 *     stay valid until the stream reaches the call. A plan is used by one stream at a time.
 *   - no call throws, aborts or traps: errors are returned as ftcg_status_t and a thread-local
 *     message (ftcg_last_error). Argument errors are detected before any device work is queued.
 *     Device-side conditions (non-finite coordinates, non-positive weight sums) set a status
 *     word that ftcg_check reads.
 */
#ifndef FTCG_H
#define FTCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* ftcg_stream_t;
typedef struct ftcg_plan_s* ftcg_plan_t;
typedef struct ftcg_batch_s* ftcg_batch_t;

typedef enum {
    FTCG_SUCCESS = 0,
    FTCG_ERR_INVALID_VALUE = 1,   /* a bad argument; nothing was queued                       */
    FTCG_ERR_OUT_OF_MEMORY = 2,   /* a device or pinned-host allocation failed                 */
    FTCG_ERR_CUDA = 3,            /* a CUDA runtime or cuFFT call failed (see ftcg_last_error) */
    FTCG_ERR_NOT_SUPPORTED = 4,   /* valid but outside this build's limits                     */
    FTCG_ERR_NUMERIC = 5,         /* non-finite coordinate or value, or a weight sum <= 0      */
    FTCG_ERR_TIMEOUT = 6          /* a bounded device wait gave up                             */
} ftcg_status_t;

/* Value storage for ftcg_adjoint / ftcg_spread. */
enum { FTCG_VALUES_C64 = 0, FTCG_VALUES_BF16X2 = 1 };
/* Weight storage for ftcg_set_weights. */
enum { FTCG_WEIGHTS_F64 = 0, FTCG_WEIGHTS_F32 = 1 };
/* Plan precision: how the per-sample weight is stored next to the sorted coordinates. */
enum { FTCG_PREC_FP32 = 0, FTCG_PREC_BF16 = 1 };
/* How footprints that cross a tile edge are handled by the spreading kernel:
 *   DUPLICATE: a sample is listed in every tile its footprint touches; each tile keeps its cells.
 *   HALO:      a sample is listed once, in the tile of its first tap; the tile accumulates a
 *              (tile + w - 1)^2 padded block, stores its own cells and hands the overflow strips to
 *              a second kernel that adds them to the neighbouring tiles' cells.
 * AUTO lets the autotuner choose, together with the tile side. */
enum { FTCG_LAYOUT_AUTO = 0, FTCG_LAYOUT_DUPLICATE = 1, FTCG_LAYOUT_HALO = 2 };
/* Which spreading kernel a plan uses (same result within the FP32 bound):
 *   AUTO:    where the autotuner runs (tile side or layout left to it), it times the kernels
 *            that apply and keeps the faster; with the tile side and layout given, the block
 *            tensor-core kernel where it applies, otherwise the register-window kernel.
 *   WINDOW:  the register-window kernel (FP32 multiply-adds into a rolling window of rows).
 *   TENSOR:  the tensor-core kernel (per column bin, 8 samples x a 16-row window per
 *            mma.sync.m16n8k8 in split TF32); it applies in the halo layout with w <= 8 and a
 *            window whose per-tap degree-7 polynomials are within 1e-6 of it (w >= 7 for any
 *            sigma >= 1.25, w = 6 at sigma = 2); NOT_SUPPORTED elsewhere.
 *   BLOCK:   the tensor-core kernel on 8 x 8-cell blocks (chunks of 8 samples whose first taps
 *            share a block, a 16 x 16-cell window per block, 12 split-TF32 MMAs per chunk);
 *            same conditions as TENSOR. */
enum { FTCG_SPREAD_AUTO = 0, FTCG_SPREAD_WINDOW = 1, FTCG_SPREAD_TENSOR = 2, FTCG_SPREAD_BLOCK = 3 };

/* Gridding window (Sec. III-A leaves the choice open; the exact weights' internal lag route
 * always uses ES): exponential of semicircle exp(beta (sqrt(1 - z^2) - 1)), Kaiser-Bessel
 * I0(beta sqrt(1 - z^2)) / I0(beta) and truncated Gaussian exp(-beta z^2), z = 2 t / w, zero for
 * |z| > 1; beta from w and sigma as ftcg_plan_info reports. */
enum { FTCG_WINDOW_ES = 0, FTCG_WINDOW_KB = 1, FTCG_WINDOW_GAUSS = 2 };

typedef struct {
    int32_t kernel;        /* FTCG_WINDOW_ES (default), _KB or _GAUSS                          */
    int32_t precision;     /* FTCG_PREC_FP32 (default) or FTCG_PREC_BF16 weight storage        */
    int32_t tile;          /* fine-grid tile side of the spreading kernel: 0 = auto, 32 or 64 */
    int32_t weight_width;  /* window width of the FP64 weight construction: 0 = 12, else 4..16 */
    int32_t layout;        /* FTCG_LAYOUT_AUTO (default), _DUPLICATE or _HALO                  */
    int32_t spread_kernel; /* FTCG_SPREAD_AUTO (default), _WINDOW, _TENSOR or _BLOCK            */
    int32_t deterministic; /* 1: adjoints bitwise reproducible (see below); 0 (default): fastest */
    int32_t reserved;      /* must be zero                                                      */
} ftcg_opts_t;
/* opts.deterministic = 1 fixes every summation order of the spreading, for debugging and
 * regression tests: the plan orders the samples of each first-tap cell by sample index, one
 * warp per tile accumulates its block chunks in plan order (the block tensor-core kernel, halo
 * layout, T = 32 unless opts.tile gives 64), and the overflow strips are added by one thread per
 * cell in a fixed order (left, upper-left, upper neighbour) instead of by atomics. Two plans
 * built from the same inputs then give bitwise equal adjoints (one warp per tile: the large ping's
 * spreading stage takes 203 us against 76 us). Needs what the block kernel needs (w <= 8, see FTCG_SPREAD_BLOCK) and G = sigma N a
 * multiple of the tile side; FTCG_ERR_NOT_SUPPORTED otherwise, and for batches. The FP64
 * weights of ftcg_weights are not covered (their first step sums with atomics). */

typedef struct {
    int64_t M;             /* samples                                                           */
    int32_t N, G, w, tile; /* image side, grid side, window width, tile side                    */
    int32_t tiles_x;       /* tiles per grid row (tiles are tile x tile, the last one ragged)    */
    int32_t layout;        /* FTCG_LAYOUT_DUPLICATE or FTCG_LAYOUT_HALO                         */
    int64_t entries;       /* sorted (tile, sample) entries                                     */
    double beta;           /* window shape parameter                                            */
    int64_t device_bytes;  /* device memory the plan holds                                      */
    int32_t spread_kernel; /* FTCG_SPREAD_WINDOW, _TENSOR or _BLOCK: the kernel the plan uses   */
    int32_t pad0;
    int64_t chunks;        /* tensor-core chunks of 8 sample slots (0 for the other kernel)     */
} ftcg_plan_info_t;

/*
 * ftcg_plan -- bin a geometry once (the sparsity of Omega_2, Eq. twodcgmatrix; taps
 * ceil(sigma lambda - w/2) + {0..w-1}^2 mod G).
 *   out      [out] receives the plan handle (owned by the caller, release with ftcg_destroy).
 *   d_lambda device, M x 2 float64 (x, y) interleaved; read during the call, may be freed after.
 *   M        0 .. 33,554,431 samples (M = 0 gives a plan whose images are zero).
 *   N        even, >= 2.
 *   sigma    >= 1; G = sigma N must be an even integer with G >= 2 w.
 *   w        2 .. 16.
 *   opts     nullable (NULL = defaults); reserved fields must be zero.
 *   stream   stream for the planning kernels. This call synchronises the stream once (to size
 *            the sorted entry array) and is not capturable; the calls that use the plan are.
 * Errors: INVALID_VALUE for bad arguments; NOT_SUPPORTED for sizes beyond the limits above;
 * NUMERIC if a coordinate is not finite (that sample is dropped and the plan is still returned);
 * OUT_OF_MEMORY; CUDA.
 */
ftcg_status_t ftcg_plan(ftcg_plan_t* out, const double* d_lambda, int64_t M, int32_t N,
                        double sigma, int32_t w, const ftcg_opts_t* opts, ftcg_stream_t stream);

/* Plan sizes; host call, no device work. */
ftcg_status_t ftcg_plan_info(ftcg_plan_t plan, ftcg_plan_info_t* info);

/*
 * ftcg_weights -- the exact FTCG diagonal weights at band r = 1 (Eq. difopt, C_2 of Eq.
 * twodftcg restricted to its diagonal): alpha_k = 1 / S_k with
 *     S_k = sum_j F_N(lambda_jx - lambda_kx) F_N(lambda_jy - lambda_ky),
 *     F_N(d) = sin^2(pi d) / (N^2 sin^2(pi d / N))   (normalised Fejer kernel),
 * i.e. the column-wise least-squares optimum of || T D - I ||_F with T the data-frame Gram matrix
 * on the N x N pixel lattice. Computed in FP64 on the device by the lag route: a gridded adjoint
 * of unit strengths at 2 lambda on a 2N lattice, a product with c(d) = prod (N - |d_i|) / N^2, and
 * a gridded forward transform at 2 lambda (window width opts.weight_width).
 * The weights are installed in the plan (used by every later ftcg_adjoint) and, if d_alpha_out is
 * not NULL, written there as M float64 in acquisition order. Temporary device memory (about
 * 16 (2 sigma N)^2 bytes) is allocated and freed inside the call; the call synchronises.
 * Errors: NUMERIC if some S_k <= 0 or is not finite (those weights are set to 0); CUDA; OOM.
 */
ftcg_status_t ftcg_weights(ftcg_plan_t plan, double* d_alpha_out, ftcg_stream_t stream);

/*
 * ftcg_set_weights -- install caller-supplied per-sample weights alpha (D_2 of Eq.
 * twodcgmatrix), M entries in acquisition order, FTCG_WEIGHTS_F64 or FTCG_WEIGHTS_F32.
 * Passing d_alpha = NULL restores alpha = 1 (plain gridding). Asynchronous.
 */
ftcg_status_t ftcg_set_weights(ftcg_plan_t plan, const void* d_alpha, int32_t dtype,
                               ftcg_stream_t stream);

/*
 * ftcg_spread -- the spreading step alone: g = Omega_2 D_2 v on the G x G fine grid
 * (Eq. twodcgmatrix), written to d_grid (G x G complex64, caller-owned, fully overwritten).
 * d_values: M values in acquisition order, layout given by vdtype. Asynchronous.
 */
ftcg_status_t ftcg_spread(ftcg_plan_t plan, const void* d_values, int32_t vdtype, void* d_grid,
                          ftcg_stream_t stream);

/*
 * ftcg_adjoint -- the full weighted adjoint (Eq. twodcg with D_2 = diag(alpha)): spread, inverse
 * 2-D FFT of the plan's fine grid, division by phi^(p_x/G) phi^(p_y/G) (FP64 factors) and crop.
 * d_image: N x N complex64, caller-owned, fully overwritten. Asynchronous and capturable.
 */
ftcg_status_t ftcg_adjoint(ftcg_plan_t plan, const void* d_values, int32_t vdtype, void* d_image,
                           ftcg_stream_t stream);

/*
 * ftcg_adjoint_host -- ftcg_adjoint on HOST buffers: copies h_values to the device, runs the
 * adjoint and returns the image in h_image, all on `stream`, then synchronises it. A page-locked
 * h_image (cudaHostAlloc / cudaHostRegister, e.g. torch pin_memory) is written in place by the
 * device; any other h_image receives one copy of a device staging image. Pinned h_values give
 * the fastest copy; pageable memory also works.
 */
ftcg_status_t ftcg_adjoint_host(ftcg_plan_t plan, const void* h_values, int32_t vdtype,
                                void* h_image, ftcg_stream_t stream);

/*
 * ftcg_adjoint_host_async -- ftcg_adjoint_host without the final synchronisation, for streams of
 * pings through one plan: the upload of h_values runs on a copy stream of the plan into one of
 * two device buffers (alternating), and the adjoint on `stream` waits for it, so the upload of
 * the next call overlaps the adjoint of this one (and its image write-back into a page-locked
 * h_image). Returns once the work is enqueued. h_values must stay unchanged, and h_image is not
 * complete, until `stream` has reached this call's work (synchronise it, or record an event
 * after the call). Calls in flight need distinct h_image buffers; a plan takes one such stream
 * of calls at a time.
 */
ftcg_status_t ftcg_adjoint_host_async(ftcg_plan_t plan, const void* h_values, int32_t vdtype,
                                      void* h_image, ftcg_stream_t stream);

/*
 * ftcg_forward -- the gridded transpose of ftcg_adjoint without weights (the data frame of
 * Eq. twoddataframe applied to an image): f_k ~= sum_p I_p exp(-2 pi i lambda_k . p / N).
 * d_image: N x N complex64; d_values: M complex64 out, acquisition order. Asynchronous.
 */
ftcg_status_t ftcg_forward(ftcg_plan_t plan, const void* d_image, void* d_values,
                           ftcg_stream_t stream);

/* Synchronise the plan's last stream and report the device status word (NUMERIC if a
 * non-finite coordinate or weight sum was seen), then clear it. */
ftcg_status_t ftcg_check(ftcg_plan_t plan);

/* Copy the plan's sorted (tile, sample) entries to host memory, for inspection and tests.
 * h_tile, h_cx, h_cy: int32 tile index and local first-tap cell of each entry (cx, cy in
 * [-(w-1), tile-1] with FTCG_LAYOUT_DUPLICATE, in [0, tile-1] with FTCG_LAYOUT_HALO); h_sample: int32 sample index; h_dx, h_dy: float32 offset of the sample from
 * its first tap, sigma lambda - ceil(sigma lambda - w/2). Each array holds info.entries elements.
 * Any pointer may be NULL. Synchronous. */
ftcg_status_t ftcg_plan_entries(ftcg_plan_t plan, int32_t* h_tile, int32_t* h_cx, int32_t* h_cy,
                                int32_t* h_sample, float* h_dx, float* h_dy);

/*
 * Stage profiling. With enable != 0, every later ftcg_adjoint records CUDA events on its stream
 * around its three stages (spread, inverse FFT, window division + crop); ftcg_stage_times
 * synchronises on the last recorded event and returns the mean duration in milliseconds of each
 * stage (ms[0] spread, ms[1] FFT, ms[2] deapodise + crop) over the calls recorded since the
 * previous read (count in *calls), then starts a new count. At most 1024 calls are recorded
 * between reads; later ones are not timed.
 */
ftcg_status_t ftcg_profile(ftcg_plan_t plan, int32_t enable);
ftcg_status_t ftcg_stage_times(ftcg_plan_t plan, float* ms, int32_t* calls);

/*
 * Batched pings. Many independent pings (each its own geometry, sample count and image side N)
 * are gridded together: one persistent spreading launch over every (ping, tile) work item, one
 * batched inverse FFT per distinct grid side, one window division + crop launch (Eq. twodcg per
 * ping). The sequence has no host synchronisation and can be captured once in a CUDA graph.
 *
 * ftcg_plan_batch -- plan n pings. d_lambda, M, N: host arrays of n entries (d_lambda[i] a device
 * M[i] x 2 float64 array, read during the call); sigma, w, opts shared, with the checks of
 * ftcg_plan per ping. opts->tile = 0 or opts->layout = 0 lets the built-in autotuner pick the
 * tile side, layout and spreading kernel of each ping: a ping's choice is keyed by (grid side, w,
 * precision, half-octave bucket of samples per grid cell); for the keys not decided yet, each
 * candidate is timed as the batched spreading launch over up to 16 of their pings (spread over
 * the batch's range of sizes), and the fastest is kept for all of those keys for the life of the
 * process. After the tuning (on `stream`), the pings'
 * plans are built by up to four host threads, each on its own stream that waits for `stream`
 * first. A ping whose coordinates are not all finite drops those samples (as ftcg_plan does) and
 * the batch is still built. Synchronises.
 */
ftcg_status_t ftcg_plan_batch(ftcg_batch_t* out, int32_t n, const double* const* d_lambda,
                              const int64_t* M, const int32_t* N, double sigma, int32_t w,
                              const ftcg_opts_t* opts, ftcg_stream_t stream);

/*
 * The autotuner's choices as a small JSON file (one entry per line: grid side, w, precision,
 * density bucket, the requested tile, layout and spreading kernel, whether the choice was timed
 * for single plans (batch 0) or batches (batch 1), and the chosen tile side, layout and kernel),
 * so that a later process can reuse them instead of timing trial launches again. ftcg_tuner_save writes the
 * choices made or loaded so far in this process; ftcg_tuner_load adds a file's entries (they
 * replace choices with the same key), after checking every entry (nothing is added when one is
 * invalid: FTCG_ERR_INVALID_VALUE naming the line). Host only: no device work, no stream.
 */
ftcg_status_t ftcg_tuner_save(const char* path);
ftcg_status_t ftcg_tuner_load(const char* path);

/* Per-ping weights: d_alpha is a host array of n device pointers (M[i] entries each, dtype as in
 * ftcg_set_weights) or NULL for alpha = 1 everywhere. Asynchronous. */
ftcg_status_t ftcg_batch_set_weights(ftcg_batch_t batch, const void* const* d_alpha, int32_t dtype,
                                     ftcg_stream_t stream);

/* Exact FTCG weights of every ping (ftcg_weights ping by ping); d_alpha_out: NULL or a host array
 * of n device pointers to M[i] float64 outputs. Synchronises. */
ftcg_status_t ftcg_batch_weights(ftcg_batch_t batch, double* const* d_alpha_out,
                                 ftcg_stream_t stream);

/* Weighted adjoints of all pings: d_values[i] (M[i] values, vdtype) -> d_images[i] (N[i] x N[i]
 * complex64); host arrays of n device pointers. Asynchronous, no host synchronisation. */
ftcg_status_t ftcg_adjoint_batch(ftcg_batch_t batch, const void* const* d_values, int32_t vdtype,
                                 void* const* d_images, ftcg_stream_t stream);

/* Run ftcg_adjoint_batch once, then capture it on `stream` (which must not be the legacy default
 * stream) into a CUDA graph bound to these buffers; ftcg_batch_launch replays it. */
ftcg_status_t ftcg_batch_capture(ftcg_batch_t batch, const void* const* d_values, int32_t vdtype,
                                 void* const* d_images, ftcg_stream_t stream);
ftcg_status_t ftcg_batch_launch(ftcg_batch_t batch, ftcg_stream_t stream);

/* tiles: NULL or n int32 (the tile side chosen for each ping); totals of entries and device
 * bytes held. Host call. */
ftcg_status_t ftcg_batch_info(ftcg_batch_t batch, int32_t* tiles, int64_t* entries,
                              int64_t* device_bytes);
ftcg_status_t ftcg_batch_destroy(ftcg_batch_t batch);
/*
 * Stage profiling of a batch, as ftcg_profile for a plan: with enable != 0 every later
 * ftcg_adjoint_batch (not the captured graph) records CUDA events on its stream around its two
 * stages; ftcg_batch_stage_times synchronises on the last one and returns the mean milliseconds
 * of ms[0] = spreading (the persistent launches and the halo fix-up) and ms[1] = the inverse
 * FFTs with window division and crop, over the calls recorded since the previous read (count in
 * *calls; at most 256 between reads).
 */
ftcg_status_t ftcg_batch_profile(ftcg_batch_t batch, int32_t enable);
ftcg_status_t ftcg_batch_stage_times(ftcg_batch_t batch, float* ms, int32_t* calls);

/*
 * Learned weights. A small MLP predicts each sample's FTCG weight (Eq. difopt at r = 1) from its
 * local k-space neighbourhood, so that pings with fresh jittered geometry need not run the exact
 * construction; ftcg_weights provides the labels and remains the reference.
 *
 * ftcg_features -- per sample k, 48 bfloat16: the offsets lambda_j - lambda_k (x, y) of the 16
 * nearest other samples in Euclidean distance (ties by smaller index), then d_aux[k] (a
 * caller-chosen scalar such as the normalised range wavenumber; NULL = 0), then 15 zeros.
 * d_lambda: device M x 2 float64; d_features: device M x 48 bfloat16 (out); d_neighbors: NULL or
 * device M x 16 int32 (out, -1 where fewer than 16 other samples exist). The neighbour sets are
 * exact (a spatial hash with a ring search that stops only when no unvisited sample can be
 * closer). Allocates temporaries and synchronises. FTCG_ERR_NUMERIC (nothing written) if a
 * coordinate is not finite.
 */
ftcg_status_t ftcg_features(const double* d_lambda, const double* d_aux, int64_t M,
                            void* d_features, int32_t* d_neighbors, ftcg_stream_t stream);
/*
 * ftcg_features_batch -- ftcg_features of n independent rasters in one request (neighbours are
 * searched within each raster only): raster i has d_lambda[i] (M[i] x 2 float64), d_aux[i]
 * (NULL, or d_aux itself NULL for all), d_features[i] (M[i] x 48 bfloat16, out) and
 * d_neighbors[i] (NULL, or d_neighbors itself NULL for all); M[i] = 0 is allowed. The pointer
 * arrays are host arrays of device pointers; outputs are bit-identical to n single calls. The
 * bounding boxes of all rasters are read back with one synchronisation, then the sorts and
 * searches run back to back over a few side streams ordered after and before `stream`; the call
 * synchronises before it returns. FTCG_ERR_NUMERIC (nothing written) if any raster has a
 * non-finite coordinate; FTCG_ERR_INVALID_VALUE names the first bad raster.
 */
ftcg_status_t ftcg_features_batch(int32_t n, const double* const* d_lambda,
                                  const double* const* d_aux, const int64_t* M,
                                  void* const* d_features, int32_t* const* d_neighbors,
                                  ftcg_stream_t stream);

typedef struct ftcg_mlp_s* ftcg_mlp_t;
enum { FTCG_MLP_PARAMS = 10561 };
/*
 * The network: 33 -> 64 -> 64 -> 64 -> 1, GELU (tanh form) on the hidden layers, output
 * y = log alpha; BF16 tensor-core matrix products with FP32 accumulation, FP32 master parameters.
 * Parameters are packed FP32 in this order: W1 [33][64], b1 [64], W2 [64][64], b2, W3 [64][64],
 * b3, w4 [64], b4 [1], each W as [input][output], row-major.
 */
ftcg_status_t ftcg_mlp_create(ftcg_mlp_t* out, const float* h_params);
/* Read (set = 0) or write (set = 1) the parameters, the Adam moments and the step count (any
 * pointer may be NULL); host buffers of FTCG_MLP_PARAMS floats. Synchronises. */
ftcg_status_t ftcg_mlp_state(ftcg_mlp_t mlp, float* h_params, float* h_m, float* h_v,
                             int64_t* step, int32_t set);
/* alpha_k = exp(y_k) for M feature rows, written as float64 (installable with
 * ftcg_set_weights). Asynchronous. */
ftcg_status_t ftcg_mlp_predict(ftcg_mlp_t mlp, const void* d_features, int64_t M,
                               double* d_alpha_out, ftcg_stream_t stream);
/* Gradients of the mean squared error of y against d_target (log alpha, float64) over a batch
 * of B rows: row r is feature/target row d_index[r] (or r when d_index is NULL). h_grads: NULL
 * or FTCG_MLP_PARAMS floats (packed like the parameters); h_loss: NULL or one float.
 * Synchronises. */
ftcg_status_t ftcg_mlp_grads(ftcg_mlp_t mlp, const void* d_features, const double* d_target,
                             const int32_t* d_index, int64_t B, float* h_grads, float* h_loss,
                             ftcg_stream_t stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on such a batch; h_loss
 * (NULL or one float) receives the batch loss before the step and then synchronises. */
ftcg_status_t ftcg_mlp_train_step(ftcg_mlp_t mlp, const void* d_features, const double* d_target,
                                  const int32_t* d_index, int64_t B, float lr, float* h_loss,
                                  ftcg_stream_t stream);
ftcg_status_t ftcg_mlp_destroy(ftcg_mlp_t mlp);

/*
 * ftcg_weights_judge -- the exact judge and fallback of predicted weights (the exact FTCG
 * construction of Eq. difopt at r = 1 keeps the last word). For K samples spread evenly over the
 * acquisition order it sums S_k = sum_j F_N(lambda_jx - lambda_kx) F_N(lambda_jy - lambda_ky)
 * directly over all M samples (FP32 Fejer terms of lags reduced exactly modulo N, compensated
 * FP32 sums per thread combined in FP64; about 1e-7 relative) and forms the ratios
 * alpha_pred_k S_k. Their median is a calibration factor; the rms of the calibrated ratios around
 * 1 estimates the relative weight error (the image error follows it). Samples with a non-finite
 * coordinate are left out of the sums and of the ratios.
 * If that rms is at most max_rel_err the calibrated weights alpha_pred / median are installed
 * (*h_accepted = 1); otherwise the exact weights are computed (ftcg_weights) and installed
 * (*h_accepted = 0). h_stats: NULL or 3 doubles {median ratio, rms, max |calibrated error|}.
 *   d_alpha  device, M float64 predicted weights (for example ftcg_mlp_predict's output).
 *   K        1 .. min(M, 65536) samples judged (cost K M Fejer terms).
 * Synchronises (one read-back of 2K doubles). Errors: those of ftcg_weights on a fallback.
 */
ftcg_status_t ftcg_weights_judge(ftcg_plan_t plan, const double* d_alpha, int32_t K,
                                 double max_rel_err, int32_t* h_accepted, double* h_stats,
                                 ftcg_stream_t stream);
/* The same for every ping of a batch (d_alpha: n device pointers; K capped at each ping's M;
 * h_accepted: NULL or n int32; h_stats: NULL or 3 n doubles); all pings' sums are computed
 * before one read-back, then each ping is accepted or falls back on its own. */
ftcg_status_t ftcg_batch_weights_judge(ftcg_batch_t batch, const double* const* d_alpha, int32_t K,
                                       double max_rel_err, int32_t* h_accepted, double* h_stats,
                                       ftcg_stream_t stream);

/*
 * ftcg_adjoint_small_noalloc -- the weighted adjoint of ftcg_adjoint, without a plan and without
 * any allocation, for small images. The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory, such as code running while a stream is captured
 * into a CUDA graph, real-time processing loops that fix their memory at start-up, or frameworks
 * that own the device memory pool.
 *   d_lambda  device, M x 2 float64 (x, y); d_values device, M complex64; d_alpha device, M
 *             float64 weights or NULL (alpha = 1); d_image device, N x N complex64 (output, fully
 *             overwritten); all owned by the caller.
 *   N, sigma, w as in ftcg_plan, with the grid side G = sigma N limited to 512: larger sizes
 *             return FTCG_ERR_NOT_SUPPORTED before any work is queued.
 * Scratch lives in fixed device arrays inside the library (about 4 MiB per GPU that loads it,
 * held until the process exits). The first call on a device looks up their addresses and loads
 * this entry point's kernels (it must come before any stream capture on that device). The
 * addresses are kept for the life of the process: after cudaDeviceReset on that device the
 * entry point must not be called again. Every call reuses the same arrays, so calls
 * that overlap on the GPU (different streams or unordered threads) race; calls on one stream are
 * safe. Samples with non-finite coordinates are skipped. Asynchronous on `stream`.
 */
ftcg_status_t ftcg_adjoint_small_noalloc(const double* d_lambda, const void* d_values,
                                         const double* d_alpha, int64_t M, int32_t N, double sigma,
                                         int32_t w, void* d_image, ftcg_stream_t stream);

/*
 * ftcg_band -- the banded FTCG coefficient matrix C for band r >= 1 (Sec. III-C, Eq. ftcg and
 * Eq. cr; C_2 of Eq. twodftcg), read as the banded least-squares problem
 *     C = argmin || T C - I ||_F over C with C_jk = 0 for |j - k| > r - 1 (acquisition order),
 * T_jk = Dx(lambda_k - lambda_j) Dy(lambda_k - lambda_j) the data-frame Gram matrix on the N x N
 * pixel lattice (D the Dirichlet kernel N^-1 sum_p exp(2 pi i d p / N)). Column k solves the
 * normal equations (T^2)[S_k, S_k] c = T[S_k, k] over its 2r - 1 band rows S_k (clipped at the
 * ends) in FP64 on the device. r = 1 gives the diagonal weights of ftcg_weights; a band covering
 * every index gives T^+ (Eq. dif3) and the frame approximation (Eq. insert).
 * The coefficients are installed in the plan: later ftcg_adjoint calls form tau = C v (complex64
 * values only) and spread tau with unit weights (ftcg_weights / ftcg_set_weights remove the
 * band again). d_coef_out: NULL or device M x (2r - 1) complex128, row k holding column k of C at
 * rows k - r + 1 .. k + r - 1 (zero outside 0..M-1).
 * Limits: 1 <= r <= 12; M <= 8192 (the construction costs O(M^2 r) FP64 work and 16 M^2 bytes
 * of temporary device memory), NOT_SUPPORTED above; FP32 plans only. Synchronises.
 * Errors: NUMERIC if some column's band system is not positive definite (rank-deficient band;
 * that column's coefficients are set to zero).
 */
ftcg_status_t ftcg_band(ftcg_plan_t plan, int32_t r, void* d_coef_out, ftcg_stream_t stream);

/*
 * ftcg_cgls -- the frame approximation (Sec. III-B, Eq. afr / afrm; in 2-D Eq. twodframe and
 * twodframeB): the minimum-norm least-squares image x = argmin || W^(1/2) (E x - v) ||_2 of the
 * data frame E_jp = exp(-2 pi i lambda_j . p / N), computed by CGLS from x = 0 with the plan's
 * gridded operators for E (ftcg_forward) and E^H (ftcg_adjoint with unit weights).
 *   d_values       device, M complex64, acquisition order.
 *   d_row_weights  device, M float64 row weights w_j > 0 (for example the FTCG weights of
 *                  ftcg_weights, which make the first iterate a multiple of the FTCG image and
 *                  precondition the iteration), or NULL for w = 1 (the plain frame approximation).
 *   iters          iterations (0..100000); tol >= 0: an iteration whose normal-equation residual
 *                  || E^H W (v - E x) || has fallen to tol times its initial value freezes x
 *                  (tol = 0: all iterations run).
 *   d_image        device, N x N complex64 (output, the last iterate).
 *   h_resnorms     host, NULL or iters + 1 doubles: the residual norm before each iteration.
 *   h_iters        host, NULL or the number of iterations that changed x.
 * FP32 vectors, FP64 reductions; no host synchronisation between iterations, one at the end.
 * Temporary device memory (2 M + 2 N^2 complex64 values) comes from the library pool; the plan's
 * installed weights are left as they were. FP32 plans only (NOT_SUPPORTED for BF16 plans).
 */
ftcg_status_t ftcg_cgls(ftcg_plan_t plan, const void* d_values, const double* d_row_weights,
                        int32_t iters, double tol, void* d_image, double* h_resnorms,
                        int32_t* h_iters, ftcg_stream_t stream);

/* Release a plan and all device memory it holds (synchronises). NULL is accepted. */
ftcg_status_t ftcg_destroy(ftcg_plan_t plan);

const char* ftcg_status_string(ftcg_status_t status);
/* Detail of the last error on the calling thread ("" if none). */
const char* ftcg_last_error(void);
/* Library version string, e.g. "ftcg 0.1 sm_103a". */
const char* ftcg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FTCG_H */
