// Learned FTCG weights: a small MLP predicts each sample's diagonal weight (Eq. difopt at r = 1)
// from its local k-space neighbourhood, so that the expensive exact construction is not needed
// per ping. The exact weights stay available (ftcg_weights) as the training labels and the judge.
//
// Features of sample k: the offsets lambda_j - lambda_k of its 16 nearest other samples (ordered
// by distance, ties by index; 32 values) and one caller-supplied scalar (the normalised range
// wavenumber), stored as 48 bfloat16 (zero padded to three k-steps of 16).
// Network: 33 -> 64 -> 64 -> 64 -> 1 with the tanh form of GELU; output y = log alpha.
//
// kNN: the samples are hashed into square cells of side h (about two samples per cell) by a
// counting sort; the query searches rings of cells around its own, keeping the best 16 (distance,
// index) pairs, and stops after ring r once the 16th distance is below r h (no unvisited sample can
// be closer), so the neighbour sets are exact.
// MLP: BF16 tensor-core mma.sync m16n8k16 with FP32 accumulation; one warp owns 16 rows, and the
// FP32 accumulator fragment of one layer is repacked in registers as the A fragment of the next.
// Training: forward (activations kept), a row-wise backward that produces dz3, dz2, dz1 with the
// same MMAs against the untransposed weights, a weight-gradient kernel that reduces act^T dz over
// the batch with MMAs (activations staged transposed in shared memory), and Adam on an FP32
// master copy.

#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "ftcg_internal.cuh"

namespace ftcg {
namespace {

constexpr int kNb = 16;                 // neighbours
constexpr int kIn = 2 * kNb + 1;        // 33 inputs
constexpr int kInPad = 48;              // three k-steps of 16
constexpr int kHid = 64;
constexpr int kLd1 = kInPad + 8;        // shared-memory row strides (bank-conflict padding)
constexpr int kLdH = kHid + 8;
// packed FP32 parameters: W1 [33][64], b1, W2 [64][64], b2, W3 [64][64], b3, w4 [64], b4
constexpr int oW1 = 0, ob1 = oW1 + kIn * kHid, oW2 = ob1 + kHid, ob2 = oW2 + kHid * kHid;
constexpr int oW3 = ob2 + kHid, ob3 = oW3 + kHid * kHid, ow4 = ob3 + kHid, ob4 = ow4 + kHid;
constexpr int kParams = ob4 + 1;        // 10561

// ---------------------------------------------------------------------------------------------
// kNN features
// ---------------------------------------------------------------------------------------------
__global__ void k_bbox(const double* __restrict__ lam, int64_t M, double* __restrict__ out) {
    __shared__ double s[4][256];
    double mnx = 1e300, mny = 1e300, mxx = -1e300, mxy = -1e300;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = lam[2 * i], y = lam[2 * i + 1];
        mnx = fmin(mnx, x); mny = fmin(mny, y); mxx = fmax(mxx, x); mxy = fmax(mxy, y);
        if (isnan(x) || isnan(y)) mxx = INFINITY;   // fmin / fmax skip NaN: make it visible
    }
    s[0][threadIdx.x] = mnx; s[1][threadIdx.x] = mny; s[2][threadIdx.x] = mxx; s[3][threadIdx.x] = mxy;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s[0][threadIdx.x] = fmin(s[0][threadIdx.x], s[0][threadIdx.x + o]);
            s[1][threadIdx.x] = fmin(s[1][threadIdx.x], s[1][threadIdx.x + o]);
            s[2][threadIdx.x] = fmax(s[2][threadIdx.x], s[2][threadIdx.x + o]);
            s[3][threadIdx.x] = fmax(s[3][threadIdx.x], s[3][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[4 * blockIdx.x + 0] = s[0][0];
        out[4 * blockIdx.x + 1] = s[1][0];
        out[4 * blockIdx.x + 2] = s[2][0];
        out[4 * blockIdx.x + 3] = s[3][0];
    }
}

struct Hash {
    double x0, y0, h, inv_h;
    int nx, ny;
};

__device__ __forceinline__ int cell_of(double v, double v0, double inv_h, int n) {
    int c = (int)floor((v - v0) * inv_h);
    return c < 0 ? 0 : (c >= n ? n - 1 : c);
}

__global__ void k_cell_count(const double* __restrict__ lam, int64_t M, Hash hs,
                             int* __restrict__ cnt, int* __restrict__ cell) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int cx = cell_of(lam[2 * i], hs.x0, hs.inv_h, hs.nx);
        const int cy = cell_of(lam[2 * i + 1], hs.y0, hs.inv_h, hs.ny);
        const int c = cy * hs.nx + cx;
        cell[i] = c;
        atomicAdd(cnt + c, 1);
    }
}

__global__ void k_cell_scatter(int64_t M, const int* __restrict__ cell, int* __restrict__ cursor,
                               int* __restrict__ sorted) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x)
        sorted[atomicAdd(cursor + cell[i], 1)] = (int)i;
}

// Sorted copies of the coordinates: pts[s] = lambda_{sorted[s]} (FP64) and pts32[s] = the same
// relative to the bounding-box corner, rounded to FP32 (for the candidate filter).
__global__ void k_gather_pts(const double* __restrict__ lam, int64_t M, const int* __restrict__ sorted,
                             double x0, double y0, double2* __restrict__ pts,
                             float2* __restrict__ pts32) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < M;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int j = sorted[s];
        const double x = lam[2 * j], y = lam[2 * j + 1];
        pts[s] = make_double2(x, y);
        pts32[s] = make_float2((float)(x - x0), (float)(y - y0));
    }
}

// Exact 16 nearest neighbours, one thread per query, queries in cell order (a warp's queries are
// neighbours). The ring search visits cells at Chebyshev distance r = 0, 1, ... and stops once the
// 16th best squared distance is below (r h)^2. A candidate is first tested in FP32 against the
// current 16th distance d16 with the slack T(d16) = 2^-16 d16 + 4 e sqrt(d16) + 4 e^2, where
// e bounds the FP32 offset error (2^-24 of twice the bounding-box extent): a candidate whose FP32
// distance exceeds d16 + T cannot beat d16 exactly. The others get the FP64 distance
// (dx dx + dy dy, rounded like the brute force) and enter the list, ordered by (distance, index);
// distances are compared as the integer images of their non-negative FP64 bit patterns.
__global__ void __launch_bounds__(128)
    k_knn(const double* __restrict__ lam, const double* __restrict__ aux, int64_t M, Hash hs,
          const int* __restrict__ start, const int* __restrict__ sorted,
          const double2* __restrict__ pts, const float2* __restrict__ pts32, float err,
          __nv_bfloat16* __restrict__ feat, int* __restrict__ nbr, bool vec) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < M;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = sorted[t];
        const double2 pi = pts[t];
        const float2 qi = pts32[t];
        const int cx = cell_of(pi.x, hs.x0, hs.inv_h, hs.nx);
        const int cy = cell_of(pi.y, hs.y0, hs.inv_h, hs.ny);
        unsigned long long bk[kNb];
        int bj[kNb];
#pragma unroll
        for (int k = 0; k < kNb; ++k) {
            bk[k] = ~0ull;
            bj[k] = 0x7fffffff;
        }
        float thr = INFINITY;
        const int rmax = max(hs.nx, hs.ny);
        for (int r = 0; r <= rmax; ++r) {
            for (int dy = -r; dy <= r; ++dy) {
                const int yy = cy + dy;
                if (yy < 0 || yy >= hs.ny) continue;
                const int step = (dy == -r || dy == r) ? 1 : 2 * r;
                for (int dx = -r; dx <= r; dx += (step > 0 ? step : 1)) {
                    const int xx = cx + dx;
                    if (xx < 0 || xx >= hs.nx) continue;
                    const int c = yy * hs.nx + xx;
                    const int s1 = start[c + 1];
                    for (int s = start[c]; s < s1; ++s) {
                        if (s == (int)t) continue;
                        const float2 q = pts32[s];
                        const float fx = q.x - qi.x, fy = q.y - qi.y;
                        if (fmaf(fx, fx, fy * fy) > thr) continue;
                        const double2 pj = pts[s];
                        const double ddx = __dsub_rn(pj.x, pi.x);
                        const double ddy = __dsub_rn(pj.y, pi.y);
                        const double d2 = __dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy));
                        const unsigned long long key = (unsigned long long)__double_as_longlong(d2);
                        const int j = sorted[s];
                        if (key > bk[kNb - 1] || (key == bk[kNb - 1] && j > bj[kNb - 1])) continue;
                        bk[kNb - 1] = key;
                        bj[kNb - 1] = j;
#pragma unroll
                        for (int k = kNb - 1; k > 0; --k) {
                            const bool sw = bk[k] < bk[k - 1] || (bk[k] == bk[k - 1] && bj[k] < bj[k - 1]);
                            if (sw) {
                                const unsigned long long tk = bk[k]; bk[k] = bk[k - 1]; bk[k - 1] = tk;
                                const int tj = bj[k]; bj[k] = bj[k - 1]; bj[k - 1] = tj;
                            }
                        }
                        if (bj[kNb - 1] != 0x7fffffff) {
                            const float d16 = (float)__longlong_as_double((long long)bk[kNb - 1]);
                            thr = d16 + (d16 * 1.52587890625e-5f + 4.0f * err * sqrtf(d16) +
                                         4.0f * err * err);
                        }
                    }
                }
            }
            // unvisited samples lie at least r h away (less a rounding margin of the cell index)
            const double reach = r * hs.h * (1.0 - 1e-9);
            if (bj[kNb - 1] != 0x7fffffff &&
                __longlong_as_double((long long)bk[kNb - 1]) < reach * reach)
                break;
        }
        // the feature row (offsets of the 16 neighbours, aux, zero padding) as 24 bf16 pairs,
        // stored as six 16-byte vectors (vec) or pair by pair
        uint32_t row[kInPad / 2];
#pragma unroll
        for (int k = 0; k < kNb; ++k) {
            const int j = bj[k] == 0x7fffffff ? i : bj[k];   // fewer than 16 samples in all
            const uint32_t lo = __bfloat16_as_ushort(__double2bfloat16(__dsub_rn(lam[2 * j], pi.x)));
            const uint32_t hi =
                __bfloat16_as_ushort(__double2bfloat16(__dsub_rn(lam[2 * j + 1], pi.y)));
            row[k] = lo | (hi << 16);
        }
        row[kNb] = __bfloat16_as_ushort(__double2bfloat16(aux ? aux[i] : 0.0));
#pragma unroll
        for (int k = kNb + 1; k < kInPad / 2; ++k) row[k] = 0u;
        if (vec) {
            uint4* f4 = reinterpret_cast<uint4*>(feat + (int64_t)i * kInPad);
#pragma unroll
            for (int q = 0; q < kInPad / 8; ++q)
                f4[q] = make_uint4(row[4 * q], row[4 * q + 1], row[4 * q + 2], row[4 * q + 3]);
            if (nbr) {
                int4* n4 = reinterpret_cast<int4*>(nbr + (int64_t)i * kNb);
#pragma unroll
                for (int q = 0; q < kNb / 4; ++q) {
                    int v[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        v[r] = bj[4 * q + r] == 0x7fffffff ? -1 : bj[4 * q + r];
                    n4[q] = make_int4(v[0], v[1], v[2], v[3]);
                }
            }
        } else {
            uint32_t* f2 = reinterpret_cast<uint32_t*>(feat + (int64_t)i * kInPad);
#pragma unroll
            for (int k = 0; k < kInPad / 2; ++k) f2[k] = row[k];
            if (nbr) {
#pragma unroll
                for (int k = 0; k < kNb; ++k)
                    nbr[(int64_t)i * kNb + k] = bj[k] == 0x7fffffff ? -1 : bj[k];
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// MLP on BF16 tensor cores
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const uint32_t l = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t h = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return l | (h << 16);
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float gelu(float z) {
    const float c = 0.7978845608028654f;
    return 0.5f * z * (1.0f + tanhf(c * (z + 0.044715f * z * z * z)));
}

__device__ __forceinline__ float gelu_grad(float z) {
    const float c = 0.7978845608028654f;
    const float t = tanhf(c * (z + 0.044715f * z * z * z));
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * c * (1.0f + 3.0f * 0.044715f * z * z);
}

// BF16 weights in shared memory: forward layout Wt[out][in] (B fragment pairs along in), backward
// layout Wn[in][out] (pairs along out), biases and w4 in FP32.
struct MlpSmem {
    __nv_bfloat16 w1t[kHid * kLd1];
    __nv_bfloat16 w2t[kHid * kLdH], w3t[kHid * kLdH];
    __nv_bfloat16 w2n[kHid * kLdH], w3n[kHid * kLdH];
    float b1[kHid], b2[kHid], b3[kHid], w4[kHid], b4;
};

__device__ void load_smem(MlpSmem& s, const float* __restrict__ P, bool backward) {
    for (int i = threadIdx.x; i < kHid * kLd1; i += blockDim.x) {
        const int o = i / kLd1, k = i % kLd1;
        s.w1t[i] = __float2bfloat16_rn(k < kIn ? P[oW1 + k * kHid + o] : 0.f);
    }
    for (int i = threadIdx.x; i < kHid * kLdH; i += blockDim.x) {
        const int r = i / kLdH, c = i % kLdH;
        const bool ok = c < kHid;
        s.w2t[i] = __float2bfloat16_rn(ok ? P[oW2 + c * kHid + r] : 0.f);
        s.w3t[i] = __float2bfloat16_rn(ok ? P[oW3 + c * kHid + r] : 0.f);
        if (backward) {
            s.w2n[i] = __float2bfloat16_rn(ok ? P[oW2 + r * kHid + c] : 0.f);
            s.w3n[i] = __float2bfloat16_rn(ok ? P[oW3 + r * kHid + c] : 0.f);
        }
    }
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
        s.b1[i] = P[ob1 + i];
        s.b2[i] = P[ob2 + i];
        s.b3[i] = P[ob3 + i];
        s.w4[i] = bf16r(P[ow4 + i]);
    }
    if (threadIdx.x == 0) s.b4 = P[ob4];
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) {
    return *reinterpret_cast<const uint32_t*>(p);
}

// acc[8][4] = A(16 x 16 ksteps) * W, B fragments from Wt (row = output, ld = stride)
template <int KSTEPS>
__device__ __forceinline__ void gemm_rows(float (*acc)[4], const uint32_t (*a)[4],
                                          const __nv_bfloat16* wt, int ld, int g, int t) {
#pragma unroll
    for (int kk = 0; kk < KSTEPS; ++kk)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const __nv_bfloat16* p = wt + (8 * nt + g) * ld + 16 * kk + 2 * t;
            mma16816(acc[nt], a[kk], ld32(p), ld32(p + 8));
        }
}

// bias (+) then GELU on the accumulators; z saved (training); A fragments of the next layer
__device__ __forceinline__ void act_layer(float (*acc)[4], uint32_t (*anext)[4], float* zsave,
                                          __nv_bfloat16* hsave, int64_t r0, int64_t M, int g,
                                          int t) {
    float h[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) h[nt][q] = bf16r(gelu(acc[nt][q]));
    if (zsave) {
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int64_t row = r0 + g + 8 * hh;
                if (row < M) {
                    const int col = 8 * nt + 2 * t;
                    zsave[row * kHid + col] = acc[nt][2 * hh];
                    zsave[row * kHid + col + 1] = acc[nt][2 * hh + 1];
                    hsave[row * kHid + col] = __float2bfloat16_rn(h[nt][2 * hh]);
                    hsave[row * kHid + col + 1] = __float2bfloat16_rn(h[nt][2 * hh + 1]);
                }
            }
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        anext[kk][0] = pack_bf16(h[2 * kk][0], h[2 * kk][1]);
        anext[kk][1] = pack_bf16(h[2 * kk][2], h[2 * kk][3]);
        anext[kk][2] = pack_bf16(h[2 * kk + 1][0], h[2 * kk + 1][1]);
        anext[kk][3] = pack_bf16(h[2 * kk + 1][2], h[2 * kk + 1][3]);
    }
    if (!zsave) return;
    (void)hsave;
}

__device__ __forceinline__ void init_bias(float (*acc)[4], const float* b, int t) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        acc[nt][0] = acc[nt][2] = b[8 * nt + 2 * t];
        acc[nt][1] = acc[nt][3] = b[8 * nt + 2 * t + 1];
    }
}

// Forward: rows idx[r] (or r) of X; y = log alpha. With TRAIN the pre-activations z1..z3 (FP32)
// and activations h1..h3 (BF16) of batch row r are stored at row r.
template <bool TRAIN>
__global__ void __launch_bounds__(128)
    k_mlp_forward(const __nv_bfloat16* __restrict__ X, const int* __restrict__ idx, int64_t M,
                  const float* __restrict__ P, float* __restrict__ y, double* __restrict__ alpha,
                  float* __restrict__ z1, float* __restrict__ z2, float* __restrict__ z3,
                  __nv_bfloat16* __restrict__ h1, __nv_bfloat16* __restrict__ h2,
                  __nv_bfloat16* __restrict__ h3) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem& s = *reinterpret_cast<MlpSmem*>(smem_raw);
    load_smem(s, P, false);
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t tile = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
         tile * 16 < M; tile += nwarps) {
        const int64_t r0 = tile * 16;
        uint32_t a1[3][4];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int64_t row = r0 + g + 8 * hh;
            const bool ok = row < M;
            const int64_t src = ok ? (idx ? (int64_t)idx[row] : row) : 0;
            const __nv_bfloat16* xr = X + src * kInPad;
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
                a1[kk][hh] = ok ? ld32(xr + 16 * kk + 2 * t) : 0u;
                a1[kk][2 + hh] = ok ? ld32(xr + 16 * kk + 8 + 2 * t) : 0u;
            }
        }
        float acc[8][4];
        uint32_t an[4][4];
        init_bias(acc, s.b1, t);
        gemm_rows<3>(acc, a1, s.w1t, kLd1, g, t);
        act_layer(acc, an, TRAIN ? z1 : nullptr, h1, r0, M, g, t);
        init_bias(acc, s.b2, t);
        gemm_rows<4>(acc, an, s.w2t, kLdH, g, t);
        act_layer(acc, an, TRAIN ? z2 : nullptr, h2, r0, M, g, t);
        init_bias(acc, s.b3, t);
        gemm_rows<4>(acc, an, s.w3t, kLdH, g, t);
        act_layer(acc, an, TRAIN ? z3 : nullptr, h3, r0, M, g, t);
        // output layer in FP32 on the BF16-rounded h3 (the A fragments hold exactly those values)
        float part[2] = {0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const uint32_t lo = an[kk][hh], hi = an[kk][2 + hh];
                const int c0 = 16 * kk + 2 * t;
                part[hh] += __uint_as_float(lo << 16) * s.w4[c0] +
                            __uint_as_float(lo & 0xffff0000u) * s.w4[c0 + 1] +
                            __uint_as_float(hi << 16) * s.w4[c0 + 8] +
                            __uint_as_float(hi & 0xffff0000u) * s.w4[c0 + 9];
            }
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            part[hh] += __shfl_xor_sync(0xffffffffu, part[hh], 1);
            part[hh] += __shfl_xor_sync(0xffffffffu, part[hh], 2);
        }
        if (t == 0)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int64_t row = r0 + g + 8 * hh;
                if (row < M) {
                    const float yy = part[hh] + s.b4;
                    if (y) y[row] = yy;
                    if (alpha) alpha[row] = exp((double)yy);
                }
            }
    }
}

// Row-wise backward of the mean squared error: dy -> dz3 -> dz2 -> dz1 (BF16, row-major), loss.
__global__ void __launch_bounds__(128)
    k_mlp_backward(const double* __restrict__ target, const int* __restrict__ idx, int64_t B,
                   const float* __restrict__ P, const float* __restrict__ y,
                   const float* __restrict__ z1, const float* __restrict__ z2,
                   const float* __restrict__ z3, float* __restrict__ dy,
                   __nv_bfloat16* __restrict__ dz1, __nv_bfloat16* __restrict__ dz2,
                   __nv_bfloat16* __restrict__ dz3, float* __restrict__ loss) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem& s = *reinterpret_cast<MlpSmem*>(smem_raw);
    load_smem(s, P, true);
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    float lsum = 0.f;
    for (int64_t tile = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
         tile * 16 < B; tile += nwarps) {
        const int64_t r0 = tile * 16;
        float d[2];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int64_t row = r0 + g + 8 * hh;
            d[hh] = 0.f;
            if (row < B) {
                const double tv = target[idx ? idx[row] : row];
                const float e = y[row] - (float)tv;
                d[hh] = 2.0f * e / (float)B;
                if (t == 0) {
                    dy[row] = d[hh];
                    lsum += e * e / (float)B;
                }
            }
        }
        // dz3 = dy w4 * gelu'(z3), in accumulator layout
        float dz[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int hh = q >> 1;
                const int64_t row = r0 + g + 8 * hh;
                const int col = 8 * nt + 2 * t + (q & 1);
                dz[nt][q] = row < B ? d[hh] * s.w4[col] * gelu_grad(z3[row * kHid + col]) : 0.f;
            }
        const float* zs[2] = {z2, z1};
        __nv_bfloat16* dzs[3] = {dz3, dz2, dz1};
        const __nv_bfloat16* wn[2] = {s.w3n, s.w2n};
#pragma unroll
        for (int layer = 0; layer < 3; ++layer) {
            uint32_t a[4][4];
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                a[kk][0] = pack_bf16(dz[2 * kk][0], dz[2 * kk][1]);
                a[kk][1] = pack_bf16(dz[2 * kk][2], dz[2 * kk][3]);
                a[kk][2] = pack_bf16(dz[2 * kk + 1][0], dz[2 * kk + 1][1]);
                a[kk][3] = pack_bf16(dz[2 * kk + 1][2], dz[2 * kk + 1][3]);
            }
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int64_t row = r0 + g + 8 * hh;
                    if (row < B) {
                        const int col = 8 * nt + 2 * t;
                        dzs[layer][row * kHid + col] = __float2bfloat16_rn(dz[nt][2 * hh]);
                        dzs[layer][row * kHid + col + 1] = __float2bfloat16_rn(dz[nt][2 * hh + 1]);
                    }
                }
            if (layer == 2) break;
            float dh[8][4];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) dh[nt][0] = dh[nt][1] = dh[nt][2] = dh[nt][3] = 0.f;
            gemm_rows<4>(dh, a, wn[layer], kLdH, g, t);     // dh = dz W^T
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int64_t row = r0 + g + 8 * (q >> 1);
                    const int col = 8 * nt + 2 * t + (q & 1);
                    dz[nt][q] = row < B ? dh[nt][q] * gelu_grad(zs[layer][row * kHid + col]) : 0.f;
                }
        }
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) atomicAdd(loss, lsum);
}

// part[cta][m][n] = sum over the CTA's rows of act[row][m] dz[row][n]: one warp per 16
// activation features, rows in chunks of 16 staged transposed in shared memory. The partials are
// summed over CTAs in a fixed order by k_reduce_parts, so gradients are bitwise reproducible.
// act: BF16 rows of width lda (gathered through idx when given), features 0..ma-1.
__global__ void __launch_bounds__(128)
    k_mlp_wgrad(const __nv_bfloat16* __restrict__ act, int lda, const int* __restrict__ idx,
                int ma, const __nv_bfloat16* __restrict__ dz, int64_t B, int64_t rows_per_cta,
                float* __restrict__ part) {
    __shared__ __align__(16) __nv_bfloat16 sa[kHid][16 + 8];
    __shared__ __align__(16) __nv_bfloat16 sd[kHid][16 + 8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t rb = blockIdx.x * rows_per_cta;
    const int64_t re = min(B, rb + rows_per_cta);
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    for (int64_t r0 = rb; r0 < re; r0 += 16) {
        __syncthreads();
        for (int i = threadIdx.x; i < 16 * kHid; i += blockDim.x) {
            const int rr = i / kHid, f = i % kHid;
            const int64_t row = r0 + rr;
            const bool ok = row < re;
            const int64_t src = ok ? (idx ? (int64_t)idx[row] : row) : 0;
            sa[f][rr] = (ok && f < ma) ? act[src * lda + f] : __float2bfloat16(0.f);
            sd[f][rr] = ok ? dz[row * kHid + f] : __float2bfloat16(0.f);
        }
        __syncthreads();
        if (16 * warp < ma) {
            uint32_t a[4];
            a[0] = ld32(&sa[16 * warp + g][2 * t]);
            a[1] = ld32(&sa[16 * warp + g + 8][2 * t]);
            a[2] = ld32(&sa[16 * warp + g][2 * t + 8]);
            a[3] = ld32(&sa[16 * warp + g + 8][2 * t + 8]);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
                mma16816(acc[nt], a, ld32(&sd[8 * nt + g][2 * t]), ld32(&sd[8 * nt + g][2 * t + 8]));
        }
    }
    if (16 * warp < ma) {
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = 16 * warp + g + 8 * (q >> 1);
                const int n = 8 * nt + 2 * t + (q & 1);
                if (m < ma) part[((int64_t)blockIdx.x * ma + m) * kHid + n] = acc[nt][q];
            }
    }
}

// bias gradients and the output layer, per block: part[blk][0..319] = (sum dz1, sum dz2,
// sum dz3, sum h3 dy) per column and sum dy at 256; summed over blocks by k_reduce_parts.
constexpr int kSmallParts = 4 * kHid + 1;
constexpr int64_t kRowsPerCta = 1024;          // rows reduced by one weight-gradient CTA
constexpr int64_t kSmallBlocks = 152 * 4;      // blocks of the small-gradient kernel
__global__ void k_mlp_small_grads(const __nv_bfloat16* __restrict__ dz1,
                                  const __nv_bfloat16* __restrict__ dz2,
                                  const __nv_bfloat16* __restrict__ dz3,
                                  const __nv_bfloat16* __restrict__ h3,
                                  const float* __restrict__ dy, int64_t B,
                                  float* __restrict__ part) {
    __shared__ float s[4][5][kHid];
    const int col = threadIdx.x & 63;     // 256 threads: 4 row phases x 64 columns
    const int ph = threadIdx.x >> 6;
    float s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f, s5 = 0.f;
    for (int64_t r = blockIdx.x * 4 + ph; r < B; r += (int64_t)gridDim.x * 4) {
        s1 += __bfloat162float(dz1[r * kHid + col]);
        s2 += __bfloat162float(dz2[r * kHid + col]);
        s3 += __bfloat162float(dz3[r * kHid + col]);
        s4 += __bfloat162float(h3[r * kHid + col]) * dy[r];
        if (col == 0) s5 += dy[r];
    }
    s[ph][0][col] = s1; s[ph][1][col] = s2; s[ph][2][col] = s3; s[ph][3][col] = s4;
    s[ph][4][col] = s5;
    __syncthreads();
    if (ph == 0) {
        float* p = part + (int64_t)blockIdx.x * kSmallParts;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            p[q * kHid + col] = ((s[0][q][col] + s[1][q][col]) + s[2][q][col]) + s[3][q][col];
        if (col == 0) p[4 * kHid] = ((s[0][4][0] + s[1][4][0]) + s[2][4][0]) + s[3][4][0];
    }
}

// out[i] = sum over blocks b = 0..nblk-1 of part[b * stride + i], in that order
__global__ void k_reduce_parts(const float* __restrict__ part, int nblk, int64_t stride, int count,
                               float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float acc = 0.f;
    for (int b = 0; b < nblk; ++b) acc += part[(int64_t)b * stride + i];
    out[i] = acc;
}

// ob1 = 1 - b1 and ob2 = 1 - b2 are formed in FP64 by the caller: 1.f - 0.999f in FP32 is
// 1.3e-5 away from 0.001.
__global__ void k_adam(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int n, float lr, float b1, float b2,
                       float ob1, float ob2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + ob1 * gi;
    const float vi = b2 * v[i] + ob2 * (gi * gi);
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

int nb(int64_t n, int t, int cap = 152 * 16) {
    int64_t b = (n + t - 1) / t;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

}  // namespace

struct Mlp {
    float* P = nullptr;      // FP32 master parameters (kParams)
    float* m = nullptr;      // Adam moments
    float* v = nullptr;
    float* grad = nullptr;
    float* loss = nullptr;
    int64_t step = 0;
    // training scratch (grown on demand)
    int64_t cap = 0;
    float *y = nullptr, *dy = nullptr, *z1 = nullptr, *z2 = nullptr, *z3 = nullptr;
    __nv_bfloat16 *h1 = nullptr, *h2 = nullptr, *h3 = nullptr;
    __nv_bfloat16 *d1 = nullptr, *d2 = nullptr, *d3 = nullptr;
    float* part = nullptr;       // per-CTA gradient partials
};

namespace {

void free_mlp_scratch(Mlp* q) {
    void* ps[] = {q->y, q->dy, q->z1, q->z2, q->z3, q->h1, q->h2, q->h3, q->d1, q->d2, q->d3,
                  q->part};
    for (void* p : ps)
        if (p) cudaFree(p);
    q->y = q->dy = q->z1 = q->z2 = q->z3 = nullptr;
    q->h1 = q->h2 = q->h3 = q->d1 = q->d2 = q->d3 = nullptr;
    q->part = nullptr;
    q->cap = 0;
}

ftcg_status_t ensure_scratch(Mlp* q, int64_t B) {
    if (B <= q->cap) return FTCG_SUCCESS;
    free_mlp_scratch(q);
    const size_t nf = (size_t)B * kHid;
    FTCG_CK(cudaMalloc(&q->y, B * sizeof(float)));
    FTCG_CK(cudaMalloc(&q->dy, B * sizeof(float)));
    FTCG_CK(cudaMalloc(&q->z1, nf * sizeof(float)));
    FTCG_CK(cudaMalloc(&q->z2, nf * sizeof(float)));
    FTCG_CK(cudaMalloc(&q->z3, nf * sizeof(float)));
    FTCG_CK(cudaMalloc(&q->h1, nf * 2));
    FTCG_CK(cudaMalloc(&q->h2, nf * 2));
    FTCG_CK(cudaMalloc(&q->h3, nf * 2));
    FTCG_CK(cudaMalloc(&q->d1, nf * 2));
    FTCG_CK(cudaMalloc(&q->d2, nf * 2));
    FTCG_CK(cudaMalloc(&q->d3, nf * 2));
    const int64_t nwb = (B + kRowsPerCta - 1) / kRowsPerCta;
    const int64_t nsb = std::min<int64_t>((B + 3) / 4, kSmallBlocks);
    FTCG_CK(cudaMalloc(&q->part, (size_t)std::max<int64_t>(nwb * kHid * kHid, nsb * kSmallParts) * sizeof(float)));
    q->cap = B;
    return FTCG_SUCCESS;
}

ftcg_status_t mlp_fail(const char* m) {
    set_error("%s", m);
    return FTCG_ERR_INVALID_VALUE;
}

size_t fwd_smem() { return sizeof(MlpSmem); }

ftcg_status_t launch_forward(Mlp* q, const __nv_bfloat16* X, const int* idx, int64_t M, bool train,
                             double* alpha, cudaStream_t s) {
    const size_t sm = fwd_smem();
    const int blocks = nb((M + 63) / 64, 1, 152 * 8);
    if (train) {
        FTCG_CK(cudaFuncSetAttribute(k_mlp_forward<true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_mlp_forward<true><<<blocks, 128, sm, s>>>(X, idx, M, q->P, q->y, nullptr, q->z1, q->z2,
                                                    q->z3, q->h1, q->h2, q->h3);
    } else {
        FTCG_CK(cudaFuncSetAttribute(k_mlp_forward<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_mlp_forward<false><<<blocks, 128, sm, s>>>(X, idx, M, q->P, nullptr, alpha, nullptr,
                                                     nullptr, nullptr, nullptr, nullptr, nullptr);
    }
    FTCG_CK(cudaGetLastError());
    return FTCG_SUCCESS;
}

// forward + backward + gradients of one batch into q->grad (zeroed first); loss into q->loss
ftcg_status_t batch_grads(Mlp* q, const __nv_bfloat16* X, const double* target, const int* idx,
                          int64_t B, cudaStream_t s) {
    FTCG_TRY(ensure_scratch(q, B));
    FTCG_CK(cudaMemsetAsync(q->grad, 0, kParams * sizeof(float), s));
    FTCG_CK(cudaMemsetAsync(q->loss, 0, sizeof(float), s));
    FTCG_TRY(launch_forward(q, X, idx, B, true, nullptr, s));
    const size_t sm = fwd_smem();
    FTCG_CK(cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_mlp_backward<<<nb((B + 63) / 64, 1, 152 * 8), 128, sm, s>>>(
        target, idx, B, q->P, q->y, q->z1, q->z2, q->z3, q->dy, q->d1, q->d2, q->d3, q->loss);
    const int wb = (int)((B + kRowsPerCta - 1) / kRowsPerCta);
    const __nv_bfloat16* acts[3] = {X, q->h1, q->h2};
    const __nv_bfloat16* dzs[3] = {q->d1, q->d2, q->d3};
    const int ldas[3] = {kInPad, kHid, kHid};
    const int mas[3] = {kIn, kHid, kHid};
    const int offs[3] = {oW1, oW2, oW3};
    for (int l = 0; l < 3; ++l) {
        k_mlp_wgrad<<<wb, 128, 0, s>>>(acts[l], ldas[l], l == 0 ? idx : nullptr, mas[l], dzs[l], B,
                                       kRowsPerCta, q->part);
        const int cnt = mas[l] * kHid;
        k_reduce_parts<<<(cnt + 255) / 256, 256, 0, s>>>(q->part, wb, cnt, cnt, q->grad + offs[l]);
    }
    const int sb = (int)std::min<int64_t>((B + 3) / 4, kSmallBlocks);
    k_mlp_small_grads<<<sb, 256, 0, s>>>(q->d1, q->d2, q->d3, q->h3, q->dy, B, q->part);
    // the groups b1, b2, b3, w4 and b4 go to their places in the packed gradient
    const int goff[5] = {ob1, ob2, ob3, ow4, ob4};
    for (int gi = 0; gi < 5; ++gi)
        k_reduce_parts<<<1, 64, 0, s>>>(q->part + gi * kHid, sb, kSmallParts, gi < 4 ? kHid : 1,
                                        q->grad + goff[gi]);
    FTCG_CK(cudaGetLastError());
    return FTCG_SUCCESS;
}

// ---------------------------------------------------------------------------------------------
// kNN feature requests (one or many rasters)
// ---------------------------------------------------------------------------------------------
struct FeatJob {
    const double* lam;
    const double* aux;
    int64_t M;
    __nv_bfloat16* out;
    int32_t* nbr;
};

// The spatial hash of a raster from the per-block partials of its bounding box: square cells of
// about one sample each (at most 4096 per axis, also when the samples lie on a line), and the
// bound on the FP32 offset error (2^-24 of twice the extent, with a 1% margin). False when a
// coordinate is not finite.
bool hash_from_box(const double* part, int nblk, int64_t M, Hash* hs, float* err) {
    double x0 = 1e300, y0 = 1e300, x1 = -1e300, y1 = -1e300;
    for (int i = 0; i < nblk; ++i) {
        x0 = std::min(x0, part[4 * i]);
        y0 = std::min(y0, part[4 * i + 1]);
        x1 = std::max(x1, part[4 * i + 2]);
        y1 = std::max(y1, part[4 * i + 3]);
    }
    if (!std::isfinite(x0) || !std::isfinite(y0) || !std::isfinite(x1) || !std::isfinite(y1))
        return false;
    const double area = std::max((x1 - x0) * (y1 - y0), 1e-300);
    double h = std::sqrt(area / (double)M);
    if (!(h > 0)) h = 1.0;
    h = std::max(h, std::max(x1 - x0, y1 - y0) / 4096.0);
    if (!(h > 0)) h = 1.0;
    hs->x0 = x0;
    hs->y0 = y0;
    hs->h = h;
    hs->inv_h = 1.0 / h;
    hs->nx = std::max(1, (int)std::ceil((x1 - x0) / h + 1e-9));
    hs->ny = std::max(1, (int)std::ceil((y1 - y0) / h + 1e-9));
    *err = (float)(2.0 * std::max(x1 - x0, y1 - y0) * 5.9604644775390625e-8 * 1.01);
    return true;
}

// The counting sort of one raster into its hash cells and the kNN search, enqueued on s
// (asynchronous; the temporaries come from the pool and are released on s).
ftcg_status_t launch_knn(const FeatJob& j, const Hash& hs, float err, cudaStream_t s) {
    const int64_t M = j.M;
    const int64_t ncell = (int64_t)hs.nx * hs.ny;
    int *cnt = nullptr, *start = nullptr, *cell = nullptr, *sorted = nullptr;
    double2* pts = nullptr;
    float2* pts32 = nullptr;
    FTCG_CK(pool_malloc(&cnt, (ncell + 1) * sizeof(int), s));
    FTCG_CK(pool_malloc(&start, (ncell + 1) * sizeof(int), s));
    FTCG_CK(pool_malloc(&cell, M * sizeof(int), s));
    FTCG_CK(pool_malloc(&sorted, M * sizeof(int), s));
    FTCG_CK(pool_malloc(&pts, M * sizeof(double2), s));
    FTCG_CK(pool_malloc(&pts32, M * sizeof(float2), s));
    FTCG_CK(cudaMemsetAsync(cnt, 0, (ncell + 1) * sizeof(int), s));
    k_cell_count<<<nb(M, 256), 256, 0, s>>>(j.lam, M, hs, cnt, cell);
    FTCG_TRY(exclusive_scan_i32(cnt, start, ncell + 1, s));
    FTCG_CK(cudaMemcpyAsync(cnt, start, (ncell + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
    k_cell_scatter<<<nb(M, 256), 256, 0, s>>>(M, cell, cnt, sorted);
    k_gather_pts<<<nb(M, 256), 256, 0, s>>>(j.lam, M, sorted, hs.x0, hs.y0, pts, pts32);
    // 16-byte row stores need 16-byte aligned outputs (rows are 96 and 64 bytes)
    const bool vec = (reinterpret_cast<uintptr_t>(j.out) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(j.nbr) & 15) == 0;
    k_knn<<<nb(M, 128, 152 * 32), 128, 0, s>>>(j.lam, j.aux, M, hs, start, sorted, pts, pts32, err,
                                                  j.out, j.nbr, vec);
    const cudaError_t e = cudaGetLastError();
    pool_free(cnt, s);
    pool_free(start, s);
    pool_free(cell, s);
    pool_free(sorted, s);
    pool_free(pts, s);
    pool_free(pts32, s);
    FTCG_CK(e);
    return FTCG_SUCCESS;
}

// Side streams over which the searches of a multi-raster request are spread (created once per
// device, non-blocking; ordered after and before the caller's stream by events).
constexpr int kFeatStreams = 4;

ftcg_status_t feat_streams(cudaStream_t* out) {
    static std::mutex mu;
    static std::map<int, std::vector<cudaStream_t>> by_dev;
    int dev = 0;
    FTCG_CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    auto& v = by_dev[dev];
    while ((int)v.size() < kFeatStreams) {
        cudaStream_t st = nullptr;
        FTCG_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        v.push_back(st);
    }
    for (int k = 0; k < kFeatStreams; ++k) out[k] = v[k];
    return FTCG_SUCCESS;
}

// Features of n rasters: the bounding boxes of all of them with one synchronisation, then the
// rasters' sorts and searches back to back (spread over the side streams when n > 1), then one
// synchronisation. A raster with a non-finite coordinate fails the request before any search.
ftcg_status_t features_impl(const FeatJob* jobs, int n, cudaStream_t s, const char* what) {
    std::vector<int> nblk(n, 0), boff(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        nblk[i] = jobs[i].M > 0 ? nb(jobs[i].M, 256, 1024) : 0;
        boff[i + 1] = boff[i] + nblk[i];
    }
    if (boff[n] == 0) return FTCG_SUCCESS;
    double* bb = nullptr;
    FTCG_CK(pool_malloc(&bb, (size_t)boff[n] * 4 * sizeof(double), s));
    for (int i = 0; i < n; ++i)
        if (nblk[i]) k_bbox<<<nblk[i], 256, 0, s>>>(jobs[i].lam, jobs[i].M, bb + 4 * boff[i]);
    std::vector<double> hb((size_t)boff[n] * 4);
    FTCG_CK(cudaGetLastError());
    FTCG_CK(cudaMemcpyAsync(hb.data(), bb, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    FTCG_CK(cudaStreamSynchronize(s));
    pool_free(bb, s);
    std::vector<Hash> hs(n);
    std::vector<float> err(n, 0.f);
    for (int i = 0; i < n; ++i) {
        if (!nblk[i]) continue;
        if (!hash_from_box(hb.data() + 4 * boff[i], nblk[i], jobs[i].M, &hs[i], &err[i])) {
            if (n == 1)
                set_error("%s: non-finite coordinates", what);
            else
                set_error("%s: raster %d has non-finite coordinates", what, i);
            return FTCG_ERR_NUMERIC;
        }
    }
    int active = 0;
    for (int i = 0; i < n; ++i) active += nblk[i] ? 1 : 0;
    if (active == 1) {
        for (int i = 0; i < n; ++i)
            if (nblk[i]) FTCG_TRY(launch_knn(jobs[i], hs[i], err[i], s));
        FTCG_CK(cudaStreamSynchronize(s));
        return FTCG_SUCCESS;
    }
    cudaStream_t side[kFeatStreams];
    FTCG_TRY(feat_streams(side));
    cudaEvent_t ev[kFeatStreams + 1];
    for (auto& e : ev) FTCG_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ftcg_status_t st = FTCG_SUCCESS;
    cudaError_t ce = cudaEventRecord(ev[kFeatStreams], s);
    for (int k = 0; k < kFeatStreams && ce == cudaSuccess; ++k)
        ce = cudaStreamWaitEvent(side[k], ev[kFeatStreams], 0);
    for (int i = 0, k = 0; i < n && ce == cudaSuccess && st == FTCG_SUCCESS; ++i) {
        if (!nblk[i]) continue;
        st = launch_knn(jobs[i], hs[i], err[i], side[k]);
        k = (k + 1) % kFeatStreams;
    }
    // the caller's stream waits for every side stream, also after a failed launch
    for (int k = 0; k < kFeatStreams; ++k) {
        cudaEventRecord(ev[k], side[k]);
        cudaStreamWaitEvent(s, ev[k], 0);
    }
    const cudaError_t se = cudaStreamSynchronize(s);
    for (auto& e : ev) cudaEventDestroy(e);
    if (st != FTCG_SUCCESS) return st;
    FTCG_CK(ce);
    FTCG_CK(se);
    return FTCG_SUCCESS;
}

}  // namespace
}  // namespace ftcg

using namespace ftcg;

extern "C" {

ftcg_status_t ftcg_features(const double* d_lambda, const double* d_aux, int64_t M,
                            void* d_features, int32_t* d_neighbors, ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (M < 0 || (M > 0 && (!d_lambda || !d_features)))
        return mlp_fail("ftcg_features: bad arguments");
    if (M > (int64_t)INT32_MAX / kNb) return mlp_fail("ftcg_features: M too large");
    const FeatJob job{d_lambda, d_aux, M, reinterpret_cast<__nv_bfloat16*>(d_features), d_neighbors};
    return features_impl(&job, 1, reinterpret_cast<cudaStream_t>(stream), "ftcg_features");
    FTCG_API_END
}

ftcg_status_t ftcg_features_batch(int32_t n, const double* const* d_lambda,
                                  const double* const* d_aux, const int64_t* M,
                                  void* const* d_features, int32_t* const* d_neighbors,
                                  ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (n < 0 || (n > 0 && (!d_lambda || !M || !d_features)))
        return mlp_fail("ftcg_features_batch: bad arguments");
    std::vector<FeatJob> jobs(n);
    for (int i = 0; i < n; ++i) {
        if (M[i] < 0 || (M[i] > 0 && (!d_lambda[i] || !d_features[i]))) {
            set_error("ftcg_features_batch: bad arguments for raster %d", i);
            return FTCG_ERR_INVALID_VALUE;
        }
        if (M[i] > (int64_t)INT32_MAX / kNb) {
            set_error("ftcg_features_batch: raster %d: M too large", i);
            return FTCG_ERR_INVALID_VALUE;
        }
        jobs[i] = FeatJob{d_lambda[i], d_aux ? d_aux[i] : nullptr, M[i],
                          reinterpret_cast<__nv_bfloat16*>(d_features[i]),
                          d_neighbors ? d_neighbors[i] : nullptr};
    }
    return features_impl(jobs.data(), n, reinterpret_cast<cudaStream_t>(stream),
                         "ftcg_features_batch");
    FTCG_API_END
}

ftcg_status_t ftcg_mlp_create(ftcg_mlp_t* out, const float* h_params) {
    FTCG_API_BEGIN
    clear_error();
    if (!out || !h_params) return mlp_fail("ftcg_mlp_create: NULL argument");
    *out = nullptr;
    Mlp* q = new (std::nothrow) Mlp();
    if (!q) return mlp_fail("ftcg_mlp_create: host allocation failed");
    const size_t bytes = kParams * sizeof(float);
    if (cudaMalloc(&q->P, bytes) != cudaSuccess || cudaMalloc(&q->m, bytes) != cudaSuccess ||
        cudaMalloc(&q->v, bytes) != cudaSuccess || cudaMalloc(&q->grad, bytes) != cudaSuccess ||
        cudaMalloc(&q->loss, sizeof(float)) != cudaSuccess) {
        cudaFree(q->P); cudaFree(q->m); cudaFree(q->v); cudaFree(q->grad); cudaFree(q->loss);
        delete q;
        set_error("ftcg_mlp_create: device allocation failed");
        return FTCG_ERR_OUT_OF_MEMORY;
    }
    cudaMemcpy(q->P, h_params, bytes, cudaMemcpyHostToDevice);
    cudaMemset(q->m, 0, bytes);
    cudaMemset(q->v, 0, bytes);
    *out = reinterpret_cast<ftcg_mlp_t>(q);
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_mlp_state(ftcg_mlp_t mlp, float* h_params, float* h_m, float* h_v,
                             int64_t* step, int32_t set) {
    FTCG_API_BEGIN
    clear_error();
    if (!mlp) return mlp_fail("ftcg_mlp_state: NULL model");
    Mlp* q = reinterpret_cast<Mlp*>(mlp);
    const size_t bytes = kParams * sizeof(float);
    const cudaMemcpyKind k = set ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    FTCG_CK(cudaDeviceSynchronize());
    if (h_params) FTCG_CK(set ? cudaMemcpy(q->P, h_params, bytes, k) : cudaMemcpy(h_params, q->P, bytes, k));
    if (h_m) FTCG_CK(set ? cudaMemcpy(q->m, h_m, bytes, k) : cudaMemcpy(h_m, q->m, bytes, k));
    if (h_v) FTCG_CK(set ? cudaMemcpy(q->v, h_v, bytes, k) : cudaMemcpy(h_v, q->v, bytes, k));
    if (step) {
        if (set) q->step = *step;
        else *step = q->step;
    }
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_mlp_predict(ftcg_mlp_t mlp, const void* d_features, int64_t M,
                               double* d_alpha_out, ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!mlp || M < 0 || (M > 0 && (!d_features || !d_alpha_out)))
        return mlp_fail("ftcg_mlp_predict: bad arguments");
    if (M == 0) return FTCG_SUCCESS;
    Mlp* q = reinterpret_cast<Mlp*>(mlp);
    return launch_forward(q, reinterpret_cast<const __nv_bfloat16*>(d_features), nullptr, M, false,
                          d_alpha_out, reinterpret_cast<cudaStream_t>(stream));
    FTCG_API_END
}

ftcg_status_t ftcg_mlp_grads(ftcg_mlp_t mlp, const void* d_features, const double* d_target,
                             const int32_t* d_index, int64_t B, float* h_grads, float* h_loss,
                             ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!mlp || B <= 0 || !d_features || !d_target) return mlp_fail("ftcg_mlp_grads: bad arguments");
    Mlp* q = reinterpret_cast<Mlp*>(mlp);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    FTCG_TRY(batch_grads(q, reinterpret_cast<const __nv_bfloat16*>(d_features), d_target, d_index,
                         B, s));
    if (h_grads)
        FTCG_CK(cudaMemcpyAsync(h_grads, q->grad, kParams * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (h_loss) FTCG_CK(cudaMemcpyAsync(h_loss, q->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    FTCG_CK(cudaStreamSynchronize(s));
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_mlp_train_step(ftcg_mlp_t mlp, const void* d_features, const double* d_target,
                                  const int32_t* d_index, int64_t B, float lr, float* h_loss,
                                  ftcg_stream_t stream) {
    FTCG_API_BEGIN
    clear_error();
    if (!mlp || B <= 0 || !d_features || !d_target || !(lr > 0))
        return mlp_fail("ftcg_mlp_train_step: bad arguments");
    Mlp* q = reinterpret_cast<Mlp*>(mlp);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    FTCG_TRY(batch_grads(q, reinterpret_cast<const __nv_bfloat16*>(d_features), d_target, d_index,
                         B, s));
    q->step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - std::pow(b1, (double)q->step));
    const float c2 = (float)(1.0 - std::pow(b2, (double)q->step));
    k_adam<<<(kParams + 255) / 256, 256, 0, s>>>(q->P, q->m, q->v, q->grad, kParams, lr,
                                                 (float)b1, (float)b2, (float)(1.0 - b1),
                                                 (float)(1.0 - b2), 1e-8f, c1, c2);
    FTCG_CK(cudaGetLastError());
    if (h_loss) {
        FTCG_CK(cudaMemcpyAsync(h_loss, q->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        FTCG_CK(cudaStreamSynchronize(s));
    }
    return FTCG_SUCCESS;
    FTCG_API_END
}

ftcg_status_t ftcg_mlp_destroy(ftcg_mlp_t mlp) {
    FTCG_API_BEGIN
    clear_error();
    if (!mlp) return FTCG_SUCCESS;
    Mlp* q = reinterpret_cast<Mlp*>(mlp);
    cudaDeviceSynchronize();
    free_mlp_scratch(q);
    cudaFree(q->P);
    cudaFree(q->m);
    cudaFree(q->v);
    cudaFree(q->grad);
    cudaFree(q->loss);
    delete q;
    return FTCG_SUCCESS;
    FTCG_API_END
}

}  // extern "C"
