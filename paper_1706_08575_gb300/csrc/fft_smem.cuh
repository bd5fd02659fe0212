// Shared-memory 1-D FFTs of power-of-two length (256..4096) along the columns and rows of a
// G x G grid: the Stockham stages, twiddle tables and the two pass bodies used by the single-ping
// kernels (fft_smem.cu) and the batched ones (batch.cu). See fft_smem.cu for the method.
#pragma once

#include "ftcg_internal.cuh"

#include <cmath>
#include <vector>

namespace ftcg {
namespace sfft {
namespace {

// grid columns per pass-A CTA (2, 4 or 8) and its threads
#ifndef FTCG_FFT_COL_BLOCK
#define FTCG_FFT_COL_BLOCK 4
#endif
#ifndef FTCG_FFT_COL_THREADS
#define FTCG_FFT_COL_THREADS 256
#endif
#ifndef FTCG_FFT_COL_MINB
#define FTCG_FFT_COL_MINB 1
#endif
constexpr int kColBlock = FTCG_FFT_COL_BLOCK;
constexpr int kColThreads = FTCG_FFT_COL_THREADS;
constexpr int kColMinBlocks = FTCG_FFT_COL_MINB;   // resident pass-A CTAs per SM to reserve

__host__ __device__ constexpr int padded(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int L) { return L + (L >> 4); }
// distance between the transforms of a block in shared memory: 4 extra elements shift each
// column by 8 banks, so that the four columns a half-warp touches (4 rows each) do not collide
__host__ __device__ constexpr int col_stride(int L) { return padded_len(L) + 4; }

// radix of stage s for a transform of length L: 16 while at least 16 remains, then the rest
__host__ __device__ constexpr int stage_radix(int L, int s) {
    int rem = L;
    for (int i = 0; i < s; ++i) rem /= (rem >= 16 ? 16 : rem);
    return rem >= 16 ? 16 : rem;
}
__host__ __device__ constexpr int num_stages(int L) {
    int n = 0;
    for (int rem = L; rem > 1; rem /= (rem >= 16 ? 16 : rem)) ++n;
    return n;
}
__host__ __device__ constexpr int log2i(int x) {
    int n = 0;
    while ((1 << n) < x) ++n;
    return n;
}
// transforms already done before stage S
__host__ __device__ constexpr int stage_ns(int L, int S) {
    int ns = 1;
    for (int i = 0; i < S; ++i) ns *= stage_radix(L, i);
    return ns;
}
// Twiddle table: for stage S (radix R, NS, step L / (NS R)) the entries w^(2^i k L / (NS R)),
// i < log2 R, k < NS, at tw_offset(L, S) + i NS + k, so that lanes with consecutive k read
// consecutive entries.
__host__ __device__ constexpr int tw_offset(int L, int S) {
    int off = 0;
    for (int i = 0; i < S; ++i) off += log2i(stage_radix(L, i)) * stage_ns(L, i);
    return off;
}
__host__ __device__ constexpr int tw_total(int L) { return tw_offset(L, num_stages(L)); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// cos(2 pi m / 16), m = 0..15
__constant__ float kCos16[16] = {1.0f, 0.92387953251128674f, 0.70710678118654752f,
                                 0.38268343236508977f, 0.0f, -0.38268343236508977f,
                                 -0.70710678118654752f, -0.92387953251128674f, -1.0f,
                                 -0.92387953251128674f, -0.70710678118654752f,
                                 -0.38268343236508977f, 0.0f, 0.38268343236508977f,
                                 0.70710678118654752f, 0.92387953251128674f};

// exp(+2 pi i m / 16) for a compile-time m; sin(t) = cos(t - pi/2)
template <int m>
__device__ __forceinline__ float2 unit16() {
    return make_float2(kCos16[m & 15], kCos16[(m + 12) & 15]);
}

__host__ __device__ constexpr int bitrev(int i, int R) {
    int r = 0;
    for (int b = 1; b < R; b <<= 1) r = (r << 1) | ((i & b) ? 1 : 0);
    return r;
}

// Butterflies of length LEN over v (radix-2 decimation in time), for every block i, offset k.
template <int R, int LEN, int K = 0>
__device__ __forceinline__ void butterflies(float2 (&v)[R]) {
    if constexpr (K < LEN / 2) {
#pragma unroll
        for (int i = 0; i < R; i += LEN) {
            const float2 a = v[i + K];
            const float2 b = K == 0 ? v[i + K + LEN / 2]
                                    : cmul(v[i + K + LEN / 2], unit16<K * (16 / LEN)>());
            v[i + K] = make_float2(a.x + b.x, a.y + b.y);
            v[i + K + LEN / 2] = make_float2(a.x - b.x, a.y - b.y);
        }
        butterflies<R, LEN, K + 1>(v);
    }
}

template <int R, int LEN = 2>
__device__ __forceinline__ void levels(float2 (&v)[R]) {
    if constexpr (LEN <= R) {
        butterflies<R, LEN>(v);
        levels<R, LEN * 2>(v);
    }
}

// V_q = sum_r v_r exp(+2 pi i r q / R) in place (R <= 16): bit-reversed reordering, then log2 R
// levels of butterflies
template <int R>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
    float2 t[R];
#pragma unroll
    for (int i = 0; i < R; ++i) t[i] = v[bitrev(i, R)];
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = t[i];
    levels<R>(v);
}

// One Stockham stage (radix R, NS transforms of size NS already done) over CB transforms of length
// L stored at s + c * col_stride(L), by NT threads. Every size is a compile-time constant; the
// first radix is 16 (or L), so NS is 1 or a multiple of 16 and the padded addresses of a
// butterfly's values are its first address plus constant offsets. Butterfly id maps to
// transform c = id % CB and index j = id / CB, so that the lanes of a warp cover CB adjacent
// columns of consecutive rows. The first stage may read its values from global memory through
// ld(c, index) instead of shared memory, and the last may hand its results to st(c, index, value).
template <int L, int R, int NS, int CB, int NT, int S, bool FIRST, bool LAST, typename LD,
          typename ST>
__device__ __forceinline__ void stage(float2* s, const float2* __restrict__ tw, const LD& ld,
                                      const ST& st) {
    constexpr int NJ = L / R;
    constexpr int NB = CB * NJ;
    constexpr int BPT = (NB + NT - 1) / NT;
    constexpr int IN_STEP = padded(NJ);               // NJ is a multiple of 16 (or the stride is 1)
    constexpr int OUT_STEP = NS == 1 ? 1 : padded(NS);
    static_assert(NJ % 16 == 0, "input stride must keep the padding linear");
    static_assert(NS == 1 || NS % 16 == 0, "output stride must keep the padding linear");
    float2 v[BPT][R];
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int id = threadIdx.x + b * NT;
        if (NB % NT == 0 || id < NB) {
            const int c = id % CB, j = id / CB;
            if constexpr (FIRST) {
#pragma unroll
                for (int r = 0; r < R; ++r) v[b][r] = ld(c, j + r * NJ);
            } else {
                const float2* src = s + c * col_stride(L) + padded(j);
#pragma unroll
                for (int r = 0; r < R; ++r) v[b][r] = src[r * IN_STEP];
            }
            if constexpr (NS > 1) {                   // the first stage has k = 0
                // w^(r k TSTEP) for the powers of two r from the table, the rest as products
                // of at most three table values
                const int k = j & (NS - 1);
                const float2* t = tw + tw_offset(L, S) + k;
                float2 w[R];
#pragma unroll
                for (int p2 = 1, i = 0; p2 < R; p2 *= 2, ++i) {
                    w[p2] = __ldg(t + i * NS);
#pragma unroll
                    for (int q = 1; q < p2; ++q) w[p2 + q] = cmul(w[p2], w[q]);
                }
#pragma unroll
                for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], w[r]);
            }
        }
    }
    if constexpr (!FIRST) __syncthreads();            // in place: every read before any write
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int id = threadIdx.x + b * NT;
        if (NB % NT == 0 || id < NB) {
            const int c = id % CB, j = id / CB;
            const int k = j & (NS - 1);
            dft<R>(v[b]);
            if constexpr (LAST) {
#pragma unroll
                for (int q = 0; q < R; ++q) st(c, (j - k) * R + k + q * NS, v[b][q]);
            } else {
                float2* dst = s + c * col_stride(L) + padded((j - k) * R + k);
#pragma unroll
                for (int q = 0; q < R; ++q) dst[q * OUT_STEP] = v[b][q];
            }
        }
    }
    if constexpr (!LAST) __syncthreads();
}

template <int L, int CB, int NT, typename LD, typename ST, int S = 0, int NS = 1>
__device__ __forceinline__ void transform(float2* s, const float2* __restrict__ tw, const LD& ld,
                                          const ST& st) {
    if constexpr (S < num_stages(L)) {
        constexpr int R = stage_radix(L, S);
        stage<L, R, NS, CB, NT, S, S == 0, S + 1 == num_stages(L)>(s, tw, ld, st);
        transform<L, CB, NT, LD, ST, S + 1, NS * R>(s, tw, ld, st);
    }
}

// The first or last stage of the column pass with each thread on two adjacent columns of the
// same butterfly index (columns c0 and c0 + 1, c0 even): the first reads both columns' values of
// a row with one 16-byte ld4(c0, index), the last writes them with one st4(c0, index, a, b), so
// the pass issues half the global memory instructions. Otherwise as stage().
template <int L, int R, int NS, int CB, int NT, int S, bool FIRST, bool LAST, typename LD4,
          typename ST4>
__device__ __forceinline__ void stage_paired(float2* s, const float2* __restrict__ tw,
                                             const LD4& ld4, const ST4& st4) {
    static_assert(CB % 2 == 0 && (FIRST != LAST), "pairs of columns, first or last stage");
    constexpr int NJ = L / R;
    constexpr int HB = CB / 2;
    constexpr int NP = HB * NJ;                       // (column pair, butterfly) items
    constexpr int PPT = (NP + NT - 1) / NT;
    constexpr int IN_STEP = padded(NJ);
    constexpr int OUT_STEP = NS == 1 ? 1 : padded(NS);
    static_assert(NJ % 16 == 0, "input stride must keep the padding linear");
    static_assert(NS == 1 || NS % 16 == 0, "output stride must keep the padding linear");
    float2 v[PPT][2][R];
#pragma unroll
    for (int b = 0; b < PPT; ++b) {
        const int p = threadIdx.x + b * NT;
        if (NP % NT == 0 || p < NP) {
            const int c0 = 2 * (p % HB), j = p / HB;
            if constexpr (FIRST) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float4 q = ld4(c0, j + r * NJ);
                    v[b][0][r] = make_float2(q.x, q.y);
                    v[b][1][r] = make_float2(q.z, q.w);
                }
            } else {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2* src = s + (c0 + h) * col_stride(L) + padded(j);
#pragma unroll
                    for (int r = 0; r < R; ++r) v[b][h][r] = src[r * IN_STEP];
                }
            }
            if constexpr (NS > 1) {
                const int k = j & (NS - 1);
                const float2* t = tw + tw_offset(L, S) + k;
                float2 w[R];
#pragma unroll
                for (int p2 = 1, i = 0; p2 < R; p2 *= 2, ++i) {
                    w[p2] = __ldg(t + i * NS);
#pragma unroll
                    for (int q = 1; q < p2; ++q) w[p2 + q] = cmul(w[p2], w[q]);
                }
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int r = 1; r < R; ++r) v[b][h][r] = cmul(v[b][h][r], w[r]);
            }
        }
    }
    if constexpr (!FIRST) __syncthreads();            // in place: every read before any write
#pragma unroll
    for (int b = 0; b < PPT; ++b) {
        const int p = threadIdx.x + b * NT;
        if (NP % NT == 0 || p < NP) {
            const int c0 = 2 * (p % HB), j = p / HB;
            const int k = j & (NS - 1);
            dft<R>(v[b][0]);
            dft<R>(v[b][1]);
            if constexpr (LAST) {
#pragma unroll
                for (int q = 0; q < R; ++q) st4(c0, (j - k) * R + k + q * NS, v[b][0][q], v[b][1][q]);
            } else {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float2* dst = s + (c0 + h) * col_stride(L) + padded((j - k) * R + k);
#pragma unroll
                    for (int q = 0; q < R; ++q) dst[q * OUT_STEP] = v[b][h][q];
                }
            }
        }
    }
    if constexpr (!LAST) __syncthreads();
}

// The column pass's sequence: paired first and last stages, stage() between them.
template <int L, int CB, int NT, typename LD4, typename ST4, int S = 0, int NS = 1>
__device__ __forceinline__ void transform_cols(float2* s, const float2* __restrict__ tw,
                                               const LD4& ld4, const ST4& st4) {
    if constexpr (S < num_stages(L)) {
        constexpr int R = stage_radix(L, S);
        constexpr bool first = S == 0, last = S + 1 == num_stages(L);
        if constexpr (first || last)
            stage_paired<L, R, NS, CB, NT, S, first, last>(s, tw, ld4, st4);
        else
            stage<L, R, NS, CB, NT, S, false, false>(s, tw, ld4, st4);
        transform_cols<L, CB, NT, LD4, ST4, S + 1, NS * R>(s, tw, ld4, st4);
    }
}

#ifndef FTCG_FFT_ROW_DIV
#define FTCG_FFT_ROW_DIV 16
#endif
// threads of a pass-B CTA: L / FTCG_FFT_ROW_DIV (at least one warp)
__host__ __device__ constexpr int row_threads(int L) {
    return L / FTCG_FFT_ROW_DIV >= 32 ? L / FTCG_FFT_ROW_DIV : 32;
}

// pass A body: transform along y the kColBlock columns x0 .. x0 + kColBlock - 1 of the L x L grid,
// in place: the first stage reads the columns from the grid, the last writes them back (a thread
// takes two adjacent columns of a row per 16-byte access, a warp kColBlock columns of
// 32 / (kColBlock / 2) consecutive rows); the stages between exchange through shared memory (sm: kColBlock *
// col_stride(L) elements).
template <int L>
__device__ __forceinline__ void cols_body(float2* __restrict__ grid, int x0,
                                          const float2* __restrict__ tw, float2* sm) {
    // two adjacent cells per access (x0 is a multiple of kColBlock, c0 even: 16-byte aligned)
    auto ld4 = [&](int c, int y) {
        return *reinterpret_cast<const float4*>(grid + (int64_t)y * L + x0 + c);
    };
    auto st4 = [&](int c, int y, float2 a, float2 b) {
        *reinterpret_cast<float4*>(grid + (int64_t)y * L + x0 + c) = make_float4(a.x, a.y, b.x, b.y);
    };
    transform_cols<L, kColBlock, kColThreads>(sm, tw, ld4, st4);
}

// pass B body: image row iy from grid row (iy - N/2) mod L, transformed along x; the first stage
// reads the row from the grid (only the column blocks marked in mask, the ones taps reach; the
// others are zero) and the last writes the N kept frequencies straight into the image, divided
// by the window transforms (FP32 pairs, see df_product). sm: padded_len(L) elements;
// row_threads(L) threads.
template <int L>
__device__ __forceinline__ void rows_body(const float2* __restrict__ grid,
                                          const unsigned* __restrict__ mask,
                                          const float2* __restrict__ tw,
                                          const float2* __restrict__ r2, int N,
                                          float2* __restrict__ img, int iy, float2* sm) {
    constexpr int NT = row_threads(L);
    const int qy = iy - N / 2 < 0 ? iy - N / 2 + L : iy - N / 2;
    const float2* row = grid + (int64_t)qy * L;
    auto ld = [&](int, int x) {
        const int blk = x / kColBlock;
        return ((__ldg(mask + (blk >> 5)) >> (blk & 31)) & 1u) ? row[x] : make_float2(0.f, 0.f);
    };
    const float2 ry = r2[iy];
    float2* out = img + (int64_t)iy * N;
    auto st = [&](int, int kx, float2 h) {
        int ix;
        if (kx < N / 2) {
            ix = kx + N / 2;
        } else if (kx >= L - N / 2) {
            ix = kx - (L - N / 2);
        } else {
            return;                                   // outside the crop
        }
        const float f = df_product(ry, r2[ix]);
        out[ix] = make_float2(h.x * f, h.y * f);
    };
    transform<L, 1, NT>(sm, tw, ld, st);
}

// the stage tables of a transform of length L (see tw_offset), in FP64 rounded to FP32
template <int L>
std::vector<float2> stage_twiddles() {
    std::vector<float2> t(tw_total(L));
    const double pi = 3.14159265358979323846;
    for (int S = 0; S < num_stages(L); ++S) {
        const int R = stage_radix(L, S), NS = stage_ns(L, S);
        for (int i = 0; (1 << i) < R; ++i)
            for (int k = 0; k < NS; ++k) {
                const long long m = ((long long)(1 << i) * k * (L / (NS * R))) % L;
                t[tw_offset(L, S) + i * NS + k] =
                    make_float2((float)std::cos(2.0 * pi * m / L), (float)std::sin(2.0 * pi * m / L));
            }
    }
    return t;
}

}  // namespace
}  // namespace sfft
}  // namespace ftcg
