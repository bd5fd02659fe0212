// Plan construction: sample binning into grid tiles (Omega_2's sparsity, Eq. twodcgmatrix).
//
// Each sample j has the first tap c_j = ceil(sigma lambda_j - w/2) and covers the w x w cells
// c_j + {0..w-1}^2 (mod G). The grid is cut into T x T tiles (the last row/column of tiles may
// be ragged). A sample becomes one entry per (tile, wrap copy) that its footprint touches, so a
// tile's spreading CTA sees every contribution to its cells and owns them exclusively (no
// global atomics, every grid cell written exactly once).
//
// Entries are ordered by (tile, local first-tap column, local first-tap row) with a counting sort
// (one wide radix digit: the whole key). Keys are few enough (tiles * (T + w - 1)^2) that one
// histogram + one exclusive scan + one scatter replace a multi-pass radix sort.

#include <algorithm>
#include <cstdio>
#include <numeric>
#include <vector>

#include "ftcg_internal.cuh"

namespace ftcg {

namespace {

constexpr int kThreads = 256;

// First tap and fractional offset in FP64, with explicitly rounded operations so that the
// decision ceil(sigma lambda - w/2) is the same IEEE result on every machine (no contraction).
struct TapOrigin {
    long long c;      // first tap (unwrapped)
    double d;         // u - c in (w/2 - 1, w/2]
    bool ok;
};

__device__ __forceinline__ TapOrigin tap_origin(double lam, double scale, int W) {
    TapOrigin t;
    double u = __dmul_rn(scale, lam);
    // |u| < 2^50 keeps ceil() and the int64 arithmetic exact.
    t.ok = isfinite(u) && fabs(u) < 1125899906842624.0;
    if (!t.ok) {
        t.c = 0;
        t.d = 0;
        return t;
    }
    double c = ceil(__dsub_rn(u, 0.5 * W));
    t.c = (long long)c;
    t.d = __dsub_rn(u, c);
    return t;
}

__device__ __forceinline__ int wrap(long long c, int G) {
    long long r = c % G;
    return (int)(r < 0 ? r + G : r);
}

// The (tile, local first column) runs of one axis: a new run starts at tap 0, at a tile boundary
// and where the footprint wraps. At most 3 runs because T >= w and only the last tile is ragged.
struct Runs {
    int n;
    int tile[3];
    int local[3];   // local column of tap 0 of this run's entry, in [-(w-1), T-1]
};

__device__ __forceinline__ Runs axis_runs(int cw, int G, int T, int W, bool halo) {
    Runs r;
    r.n = 0;
    if (halo) {                       // listed once, in the tile of the first tap
        r.n = 1;
        r.tile[0] = cw / T;
        r.local[0] = cw - r.tile[0] * T;
        return r;
    }
    for (int t = 0; t < W; ++t) {
        int col = cw + t;
        if (col >= G) col -= G;
        if (t == 0 || col == 0 || (col % T) == 0) {
            int tile = col / T;
            if (r.n < 3) {
                r.tile[r.n] = tile;
                r.local[r.n] = col - tile * T - t;
                ++r.n;
            }
        }
    }
    return r;
}

__global__ void k_bin_count(const double* __restrict__ lam, int64_t M, double scale, int G, int T,
                            int W, int ntx, int ncb, bool halo, int* __restrict__ hist,
                            unsigned* __restrict__ status, int4* __restrict__ samp) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        TapOrigin ox = tap_origin(lam[2 * j], scale, W);
        TapOrigin oy = tap_origin(lam[2 * j + 1], scale, W);
        if (!ox.ok || !oy.ok) {
            atomicOr(status, STATUS_NONFINITE_COORD);
            if (samp) samp[j] = make_int4(-1, -1, 0, 0);
            continue;
        }
        int cxw = wrap(ox.c, G), cyw = wrap(oy.c, G);
        if (samp)
            samp[j] = make_int4(cxw, cyw, __float_as_int(__double2float_rn(ox.d)),
                                __float_as_int(__double2float_rn(oy.d)));
        Runs rx = axis_runs(cxw, G, T, W, halo);
        Runs ry = axis_runs(cyw, G, T, W, halo);
        for (int a = 0; a < ry.n; ++a)
            for (int b = 0; b < rx.n; ++b) {
                int64_t tile = (int64_t)ry.tile[a] * ntx + rx.tile[b];
                int64_t key = (tile * ncb + (rx.local[b] + W - 1)) * ncb + (ry.local[a] + W - 1);
                atomicAdd(hist + key, 1);
            }
    }
}

// Deterministic plans: the entries of each (tile, column bin, row) key in sample order (the
// scatter's atomic cursors leave them in arrival order). One thread per key; a key holds the
// few samples whose first tap is one cell, so an insertion sort. end: the cursors after the
// scatter (one past each key's last entry), cnt: the key's count.
__global__ void k_key_sort(const int* __restrict__ cnt, const int* __restrict__ end,
                           int64_t nkeys, Entry* __restrict__ ent) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nkeys;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int n = cnt[k];
        if (n < 2) continue;
        Entry* e = ent + (end[k] - n);
        for (int i = 1; i < n; ++i) {
            const Entry x = e[i];
            const uint32_t xi = x.packed & kSampleMask;
            int j = i - 1;
            while (j >= 0 && (e[j].packed & kSampleMask) > xi) {
                e[j + 1] = e[j];
                --j;
            }
            e[j + 1] = x;
        }
    }
}

__global__ void k_bin_scatter(const double* __restrict__ lam, int64_t M, double scale, int G,
                              int T, int W, int ntx, int ncb, bool halo,
                              int* __restrict__ cursor, Entry* __restrict__ ent) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        TapOrigin ox = tap_origin(lam[2 * j], scale, W);
        TapOrigin oy = tap_origin(lam[2 * j + 1], scale, W);
        if (!ox.ok || !oy.ok) continue;
        int cxw = wrap(ox.c, G), cyw = wrap(oy.c, G);
        Entry e;
        e.dx = __double2float_rn(ox.d);
        e.dy = __double2float_rn(oy.d);
        e.alpha = __float_as_uint(1.0f);
        Runs rx = axis_runs(cxw, G, T, W, halo);
        Runs ry = axis_runs(cyw, G, T, W, halo);
        for (int a = 0; a < ry.n; ++a)
            for (int b = 0; b < rx.n; ++b) {
                int64_t tile = (int64_t)ry.tile[a] * ntx + rx.tile[b];
                int64_t key = (tile * ncb + (rx.local[b] + W - 1)) * ncb + (ry.local[a] + W - 1);
                int pos = atomicAdd(cursor + key, 1);
                e.packed = (uint32_t)j | ((uint32_t)(ry.local[a] + W - 1) << kSampleBits);
                ent[pos] = e;
            }
    }
}

// colptr[t * ncb + k] = start of column bin k of tile t (= scan at its first row key).
__global__ void k_colptr(const int* __restrict__ offs, int64_t nbins, int ncb, int total,
                         int* __restrict__ colptr) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= nbins;
         i += (int64_t)gridDim.x * blockDim.x)
        colptr[i] = i < nbins ? offs[i * ncb] : total;
}

// ---- exclusive scan of int32 (three phases: block sums, scan of sums, block rescan) ----------
constexpr int kScanItems = 16;
constexpr int kScanBlock = kThreads * kScanItems;   // 4096 items per block

__device__ __forceinline__ int block_exclusive_sum(int v, int* total) {
    __shared__ int warp_sums[kThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < kThreads / 32 ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    int before = (wid > 0 ? warp_sums[wid - 1] : 0) + x - v;
    *total = warp_sums[kThreads / 32 - 1];
    __syncthreads();
    return before;
}

__global__ void k_scan_sums(const int* __restrict__ in, int64_t n, int* __restrict__ bsum) {
    int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    int total;
    block_exclusive_sum(s, &total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// One block scans the (few) block sums in place, exclusive, looping with a carry.
__global__ void k_scan_single(int* __restrict__ a, int64_t n) {
    int carry = 0;
    for (int64_t base = 0; base < n; base += kScanBlock) {
        int64_t i0 = base + (int64_t)threadIdx.x * kScanItems;
        int vals[kScanItems];
        int s = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            vals[i] = (i0 + i < n) ? a[i0 + i] : 0;
            s += vals[i];
        }
        int total;
        int run = block_exclusive_sum(s, &total) + carry;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            if (i0 + i < n) a[i0 + i] = run;
            run += vals[i];
        }
        carry += total;
    }
}

__global__ void k_scan_apply(const int* __restrict__ in, int64_t n, const int* __restrict__ boff,
                             int* __restrict__ out) {
    int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
    int vals[kScanItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        vals[i] = (base + i < n) ? in[base + i] : 0;
        s += vals[i];
    }
    int total;
    int run = block_exclusive_sum(s, &total) + boff[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += vals[i];
    }
}

int grid_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (int)b;
}

}  // namespace

ftcg_status_t exclusive_scan_i32(const int* d_in, int* d_out, int64_t n, cudaStream_t s) {
    if (n <= 0) return FTCG_SUCCESS;
    int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    int* bsum = nullptr;
    FTCG_CK(pool_malloc(&bsum, nb * sizeof(int), s));
    k_scan_sums<<<(unsigned)nb, kThreads, 0, s>>>(d_in, n, bsum);
    k_scan_single<<<1, kThreads, 0, s>>>(bsum, nb);
    k_scan_apply<<<(unsigned)nb, kThreads, 0, s>>>(d_in, n, bsum, d_out);
    FTCG_CK(cudaGetLastError());
    FTCG_CK(pool_free(bsum, s));
    return FTCG_SUCCESS;
}

void free_binning(Binning& b) {
    free_chunks(b);
    if (b.ent) cudaFree(b.ent);
    if (b.colptr) cudaFree(b.colptr);
    if (b.tile_order) cudaFree(b.tile_order);
    if (b.halo_buf) cudaFree(b.halo_buf);
    if (b.tile_full) cudaFree(b.tile_full);
    b.halo_buf = nullptr;
    b.tile_full = nullptr;
    b.ent = nullptr;
    b.colptr = nullptr;
    b.tile_order = nullptr;
    b.n_entries = 0;
    b.col_occ.clear();
}

// Launch order of the tiles: decreasing entry count, so that the heaviest tiles start first and
// the light (often empty) ones fill the tail.
static ftcg_status_t order_tiles(Binning& b, cudaStream_t s, int64_t* bytes) {
    const int64_t nbins = (int64_t)b.ntiles * b.ncb;
    std::vector<int> cp(nbins + 1);
    FTCG_CK(cudaMemcpyAsync(cp.data(), b.colptr, (nbins + 1) * sizeof(int), cudaMemcpyDeviceToHost,
                            s));
    FTCG_CK(cudaStreamSynchronize(s));
    b.tile_cnt.resize(b.ntiles);
    for (int t = 0; t < b.ntiles; ++t)
        b.tile_cnt[t] = cp[(int64_t)(t + 1) * b.ncb] - cp[(int64_t)t * b.ncb];
    std::vector<int>& order = b.h_order;
    order.resize(b.ntiles);
    std::iota(order.begin(), order.end(), 0);
    auto cnt = [&](int t) { return b.tile_cnt[t]; };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cnt(x) > cnt(y); });
    b.n_nonempty = 0;
    while (b.n_nonempty < b.ntiles && cnt(order[b.n_nonempty]) > 0) ++b.n_nonempty;
    // grid columns that taps reach: an entry in column bin k of tile column tx has its first tap
    // (of the tile's run) at X0 + k - (w - 1), and the sample's taps of that run follow it
    std::vector<unsigned char> first(b.G, 0);   // columns where some run of taps starts
    for (int i = 0; i < b.n_nonempty; ++i) {
        const int t = order[i];
        const int X0 = (t % b.ntx) * b.T;
        const int64_t base = (int64_t)t * b.ncb;
        for (int k = 0; k < b.ncb; ++k) {
            if (cp[base + k + 1] == cp[base + k]) continue;
            int x = X0 + k - (b.W - 1);
            if (x < 0) x += b.G;
            if (x >= b.G) x -= b.G;
            first[x] = 1;
        }
    }
    b.col_occ.assign(b.G, 0);                    // the w columns from each start (mod G)
    for (int x = 0, run = 0; x < b.G + b.W - 1; ++x) {
        run = first[x % b.G] ? b.W : run - 1;
        if (run > 0) b.col_occ[x % b.G] = 1;
    }
    // launch order: non-empty tiles (heaviest first), then the empty tiles in columns that taps
    // reach (a pruned inverse transform reads them, so they must hold zeros), then the rest
    {
        std::vector<int> read, skip;
        for (int i = b.n_nonempty; i < b.ntiles; ++i) {
            const int x0 = (order[i] % b.ntx) * b.T;
            bool any = false;
            for (int x = x0; x < std::min(b.G, x0 + b.T) && !any; ++x) any = b.col_occ[x] != 0;
            (any ? read : skip).push_back(order[i]);
        }
        std::copy(read.begin(), read.end(), order.begin() + b.n_nonempty);
        std::copy(skip.begin(), skip.end(), order.begin() + b.n_nonempty + read.size());
        b.n_read = b.n_nonempty + (int)read.size();
    }
    if (b.det && b.halo) {
        b.h_full.resize(b.ntiles);
        for (int t = 0; t < b.ntiles; ++t) b.h_full[t] = b.tile_cnt[t] > 0 ? 1 : 0;
        FTCG_CK(pool_malloc(&b.tile_full, b.ntiles, s));
        *bytes += b.ntiles;
        FTCG_CK(cudaMemcpyAsync(b.tile_full, b.h_full.data(), b.ntiles, cudaMemcpyHostToDevice, s));
    }
    FTCG_CK(pool_malloc(&b.tile_order, b.ntiles * sizeof(int), s));
    *bytes += b.ntiles * sizeof(int);
    // the host order stays alive with the binning, so the copy needs no synchronisation here
    FTCG_CK(cudaMemcpyAsync(b.tile_order, order.data(), b.ntiles * sizeof(int),
                            cudaMemcpyHostToDevice, s));
    return FTCG_SUCCESS;
}

ftcg_status_t build_binning(Binning& b, const double* d_lambda, int64_t M, double scale, int G,
                            int T, int W, bool halo, unsigned* d_status, int4* d_samp,
                            cudaStream_t s, int64_t* bytes) {
    b.G = G;
    b.T = T;
    b.W = W;
    b.halo = halo;
    b.ntx = (G + T - 1) / T;
    b.ntiles = b.ntx * b.ntx;
    b.ncb = T + W - 1;
    const int64_t nbins = (int64_t)b.ntiles * b.ncb;      // (tile, column bin)
    const int64_t nkeys = nbins * b.ncb;                  // (tile, column bin, row)
    FTCG_CK(pool_malloc(&b.colptr, (nbins + 1) * sizeof(int), s));
    *bytes += (nbins + 1) * sizeof(int);
    if (M == 0) {
        FTCG_CK(cudaMemsetAsync(b.colptr, 0, (nbins + 1) * sizeof(int), s));
        b.n_entries = 0;
        return FTCG_SUCCESS;
    }
    int* hist = nullptr;
    int* offs = nullptr;
    FTCG_CK(pool_malloc(&hist, nkeys * sizeof(int), s));
    FTCG_CK(pool_malloc(&offs, nkeys * sizeof(int), s));
    FTCG_CK(cudaMemsetAsync(hist, 0, nkeys * sizeof(int), s));
    k_bin_count<<<grid_for(M), kThreads, 0, s>>>(d_lambda, M, scale, G, T, W, b.ntx, b.ncb, halo,
                                                 hist, d_status, d_samp);
    FTCG_CK(cudaGetLastError());
    FTCG_TRY(exclusive_scan_i32(hist, offs, nkeys, s));
    int last_off = 0, last_cnt = 0;
    FTCG_CK(cudaMemcpyAsync(&last_off, offs + nkeys - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    FTCG_CK(cudaMemcpyAsync(&last_cnt, hist + nkeys - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    FTCG_CK(cudaStreamSynchronize(s));
    const int total = last_off + last_cnt;
    b.n_entries = total;
    k_colptr<<<grid_for(nbins + 1), kThreads, 0, s>>>(offs, nbins, b.ncb, total, b.colptr);
    FTCG_CK(cudaGetLastError());
    if (total > 0) {
        FTCG_CK(pool_malloc(&b.ent, (size_t)(total + kEntryPad) * sizeof(Entry), s));
        *bytes += (int64_t)(total + kEntryPad) * sizeof(Entry);
        FTCG_CK(cudaMemsetAsync(b.ent + total, 0, kEntryPad * sizeof(Entry), s));
        k_bin_scatter<<<grid_for(M), kThreads, 0, s>>>(d_lambda, M, scale, G, T, W, b.ntx, b.ncb,
                                                       halo, offs, b.ent);
        FTCG_CK(cudaGetLastError());
        if (b.det) {
            k_key_sort<<<grid_for(nkeys), kThreads, 0, s>>>(hist, offs, nkeys, b.ent);
            FTCG_CK(cudaGetLastError());
        }
    }
    FTCG_CK(pool_free(hist, s));
    FTCG_CK(pool_free(offs, s));
    if (halo) {
        // per tile: the right strip (T + w - 1) x (w - 1) and the bottom strip (w - 1) x T
        b.halo_cells = (T + W - 1) * (W - 1) + (W - 1) * T;
        const size_t hb = (size_t)b.ntiles * b.halo_cells * sizeof(float2);
        FTCG_CK(pool_malloc(&b.halo_buf, hb, s));
        *bytes += (int64_t)hb;
    }
    return order_tiles(b, s, bytes);
}

}  // namespace ftcg
