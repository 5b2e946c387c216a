// GB300 (sm_103a) kernels of the learned warm start (include/mmpc_mlp.h):
// scene features, the MLP forward / backward / AdamW kernels, and the
// encoding between solutions of Algorithm 1 (Sec. III-E) and network outputs.
//
// The network is small (64 -> 256 -> 256 -> 256 -> 6n) and its cost is
// negligible next to the solves it warm-starts, so its products run as a
// tiled FP32 SIMT GEMM (64 x 64 tiles, 4 x 4 outputs per thread, operands
// staged through shared memory) with the bfloat16 weights widened on load
// and every epilogue fused: bias + GELU (keeping the pre-activation for the
// backward pass), the GELU derivative on the backward product, split-K
// partial sums for the weight gradients reduced in a fixed order (so training
// is deterministic).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mmpc_mlp.h"

namespace {

thread_local std::string g_mlp_error = "no error";

int fail(int code, const std::string& msg)
{
    g_mlp_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(MMPC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// Features, encoding, statistics
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool key_less(float ki, int i, float kj, int j)
{
    const bool ni = isnan(ki), nj = isnan(kj);
    if (ni || nj) return (!ni && nj) || (ni && nj && i < j);
    return ki < kj || (ki == kj && i < j);
}

__device__ __forceinline__ float lane_of(float y)
{
    const float q = floorf(__fdiv_rn(__fadd_rn(y, 7.f), 3.5f));
    return fminf(fmaxf(q, 0.f), 3.f);
}

// One CTA per scene: ranking keys of the obstacles, the scene part of the
// feature row in shared memory, then every goal's row.
__global__ void __launch_bounds__(128) features_kernel(const mmpc_warm_scene* __restrict__ sc, int S, float a,
                                                       float b)
{
    const int s = blockIdx.x;
    if (s >= S) return;
    const mmpc_warm_scene d = sc[s];
    __shared__ float key[MMPC_MAX_OBST];
    __shared__ int slot[MMPC_MLP_NEAREST];
    __shared__ float row[MMPC_MLP_FEATURES];
    const int tid = threadIdx.x;
    const float y0 = d.ego[0], v0 = d.ego[1];
    const int m = min(max(d.m, 0), MMPC_MAX_OBST);
    for (int j = tid; j < m; j += blockDim.x) {
        const float ux = __fdiv_rn(d.obst[4 * j], a);
        const float uy = __fdiv_rn(__fsub_rn(d.obst[4 * j + 1], y0), b);
        key[j] = __fadd_rn(__fmul_rn(ux, ux), __fmul_rn(uy, uy));
    }
    if (tid < MMPC_MLP_NEAREST) slot[tid] = -1;
    __syncthreads();
    for (int j = tid; j < m; j += blockDim.x) {
        const float kj = key[j];
        int rank = 0;
        for (int i = 0; i < m && rank < MMPC_MLP_NEAREST; ++i) rank += key_less(key[i], i, kj, j) ? 1 : 0;
        if (rank < MMPC_MLP_NEAREST) slot[rank] = j;
    }
    __syncthreads();
    if (tid < MMPC_MLP_FEATURES) {
        float v = 0.f;
        if (tid == 0) v = y0 / 3.5f;
        else if (tid == 1) v = v0 / 20.f;
        else if (tid == 2) v = d.ego[2];
        else if (tid == 3) v = d.ego[3] / 4.f;
        else if (tid < 4 + 5 * MMPC_MLP_NEAREST) {
            const int sl = (tid - 4) / 5, f = (tid - 4) % 5;
            const int j = slot[sl];
            if (j < 0) {
                v = f == 0 ? 10.f : 0.f;
            } else {
                const float* o = d.obst + 4 * j;
                v = f == 0 ? o[0] / 100.f
                  : f == 1 ? (o[1] - y0) / 3.5f
                  : f == 2 ? (o[2] - v0) / 20.f
                  : f == 3 ? o[3] / 20.f
                           : lane_of(o[1]) - lane_of(y0);
            }
        } else if (tid == 57) {
            v = 1.f;
        }
        row[tid] = v;
    }
    __syncthreads();
    const int B = max(d.B, 0);
    for (int e = tid; e < B * MMPC_MLP_FEATURES; e += blockDim.x) {
        const int r = e / MMPC_MLP_FEATURES, c = e % MMPC_MLP_FEATURES;
        float v = row[c];
        if (c == 54) v = (d.goals[3 * r] - y0) / 3.5f;
        else if (c == 55) v = d.goals[3 * r + 1] / 20.f;
        else if (c == 56) v = d.goals[3 * r + 2] / 4.f;
        d.X[(size_t)r * MMPC_MLP_FEATURES + c] = v;
    }
}

// shift of column k of the encoding: v0 lin_k for c_x, y0 for c_y, 0 else
__device__ __forceinline__ float enc_shift(int k, int n, float T, float y0, float v0)
{
    if (k < n) return v0 * (T * (float)k / (float)(n - 1));
    if (k < 2 * n) return y0;
    return 0.f;
}

// Thread per (row, axis): the axis' n coefficients from the outputs, then its
// multipliers -- predicted (6n outputs), Q c (3n outputs and Q given), or 0.
__global__ void decode_kernel(const mmpc_warm_scene* __restrict__ sc, int S, int n, float T, int outputs,
                              const float* __restrict__ mu, const float* __restrict__ sigma,
                              const float* __restrict__ Q)
{
    const int s = blockIdx.x;
    if (s >= S) return;
    __shared__ float q[MMPC_MAX_COEF * MMPC_MAX_COEF];
    if (Q)
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) q[e] = Q[e];
    __syncthreads();
    const mmpc_warm_scene d = sc[s];
    const float y0 = d.ego[0], v0 = d.ego[1];
    const int W = outputs, B = max(d.B, 0);
    for (int u = threadIdx.x; u < 3 * B; u += blockDim.x) {
        const int r = u / 3, ax = u % 3;
        const float* y = d.Y + (size_t)r * W;
        float c[MMPC_MAX_COEF];
        for (int k = 0; k < n; ++k) {
            const int col = ax * n + k;
            c[k] = fmaf(y[col], sigma[col], mu[col]) + enc_shift(col, n, T, y0, v0);
            d.coef[(size_t)r * 3 * n + col] = c[k];
        }
        if (!d.lam) continue;
        float* lo = d.lam + (size_t)r * 3 * n + ax * n;
        for (int k = 0; k < n; ++k) {
            float v = 0.f;
            if (W == 6 * n) {
                const int col = 3 * n + ax * n + k;
                v = fmaf(y[col], sigma[col], mu[col]);
            } else if (Q) {
                for (int j = 0; j < n; ++j) v = fmaf(q[k * n + j], c[j], v);
            }
            lo[k] = v;
        }
    }
}

__global__ void encode_kernel(const mmpc_warm_scene* __restrict__ sc, int S, int n, float T, int outputs,
                              const float* __restrict__ mu, const float* __restrict__ sigma)
{
    const int s = blockIdx.x;
    if (s >= S) return;
    const mmpc_warm_scene d = sc[s];
    const float y0 = d.ego[0], v0 = d.ego[1];
    const int W = outputs, B = max(d.B, 0);
    for (int e = threadIdx.x; e < B * W; e += blockDim.x) {
        const int r = e / W, k = e % W;
        const float t = k < 3 * n ? d.coef[(size_t)r * 3 * n + k] - enc_shift(k, n, T, y0, v0)
                                  : d.lam[(size_t)r * 3 * n + (k - 3 * n)];
        d.Z[e] = (t - mu[k]) / sigma[k];
    }
}

// One CTA per column, float64 sums, two passes (mean, then squared deviations).
__global__ void __launch_bounds__(256) column_stats_kernel(const float* __restrict__ X, int rows, int cols,
                                                           float* __restrict__ mean_out, float* __restrict__ std_out)
{
    const int c = blockIdx.x;
    __shared__ double part[256];
    __shared__ double s_mean;
    double acc = 0.0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) acc += X[(size_t)r * cols + c];
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) s_mean = part[0] / rows;
    __syncthreads();
    const double mean = s_mean;
    acc = 0.0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const double dv = X[(size_t)r * cols + c] - mean;
        acc += dv * dv;
    }
    __syncthreads();
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double sd = sqrt(part[0] / rows);
        mean_out[c] = (float)mean;
        std_out[c] = sd > 0.0 ? (float)sd : 1.f;
    }
}

__global__ void standardize_kernel(const float* __restrict__ X, int rows, int cols, const float* __restrict__ mean,
                                   const float* __restrict__ sd, float* __restrict__ out)
{
    const size_t total = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % cols);
        out[e] = (X[e] - mean[c]) / sd[c];
    }
}

__global__ void gather_kernel(const float* __restrict__ src, int src_rows, int cols, const int* __restrict__ idx,
                              int rows, float* __restrict__ out)
{
    const size_t total = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e % cols);
        const int i = idx[r];
        out[e] = (i >= 0 && i < src_rows) ? src[(size_t)i * cols + c] : __int_as_float(0x7fc00000);
    }
}

// ---------------------------------------------------------------------------
// GEMM with fused epilogues
//   C[i][j] = sum_{k in chunk z} A(i, k) B(k, j)
//   A(i, k) = TA ? A[k lda + i] : A[i lda + k]     (float)
//   B(k, j) = TBT ? B[j ldb + k] : B[k ldb + j]    (float or bfloat16)
// ---------------------------------------------------------------------------
constexpr int BM = 64, BN = 64, BK = 16;

enum Epi { EPI_BIAS = 0, EPI_BIAS_GELU = 1, EPI_GELU_GRAD = 2, EPI_PARTIAL = 3 };

__device__ __forceinline__ float ld(const float* p) { return *p; }
__device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

template <typename TBt, bool TA, bool TBT, int EPI>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, int kchunk, const float* __restrict__ A,
                                                   int lda, const TBt* __restrict__ B, int ldb, float* __restrict__ C,
                                                   int ldc, const float* __restrict__ bias, float* __restrict__ pre,
                                                   const float* __restrict__ aux)
{
    __shared__ __align__(16) float As[BK][BM + 4];
    __shared__ __align__(16) float Bs[BK][BN + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
    for (int k0 = kb; k0 < ke; k0 += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += 256) {
            int ii, kk;
            if (TA) { ii = e % BM; kk = e / BM; }
            else { kk = e % BK; ii = e / BK; }
            const int gi = i0 + ii, gk = k0 + kk;
            float v = 0.f;
            if (gi < M && gk < ke) v = TA ? A[(size_t)gk * lda + gi] : A[(size_t)gi * lda + gk];
            As[kk][ii] = v;
        }
        for (int e = threadIdx.x; e < BK * BN; e += 256) {
            int kk, jj;
            if (TBT) { kk = e % BK; jj = e / BK; }
            else { jj = e % BN; kk = e / BN; }
            const int gk = k0 + kk, gj = j0 + jj;
            float v = 0.f;
            if (gk < ke && gj < N) v = ld(TBT ? B + (size_t)gj * ldb + gk : B + (size_t)gk * ldb + gj);
            Bs[kk][jj] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
            const float4 bb = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float bv[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
        }
        __syncthreads();
    }
    float* Cz = C + (EPI == EPI_PARTIAL ? (size_t)blockIdx.z * M * ldc : 0);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int gi = i0 + ty * 4 + r;
        if (gi >= M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int gj = j0 + tx * 4 + c;
            if (gj >= N) continue;
            const size_t o = (size_t)gi * ldc + gj;
            float v = acc[r][c];
            if (EPI == EPI_BIAS) {
                Cz[o] = v + bias[gj];
            } else if (EPI == EPI_BIAS_GELU) {
                v += bias[gj];
                if (pre) pre[o] = v;
                Cz[o] = gelu(v);
            } else if (EPI == EPI_GELU_GRAD) {
                Cz[o] = v * gelu_grad(aux[o]);
            } else {
                Cz[o] = v;
            }
        }
    }
}

// out[e] = sum_{z < Z} part[z][e], z in increasing order (deterministic).
__global__ void reduce_partials_kernel(const float* __restrict__ part, int Z, size_t count, float* __restrict__ out)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < Z; ++z) s += part[(size_t)z * count + e];
        out[e] = s;
    }
}

// db[j] = sum_r D[r][j]: one warp per column, lanes over rows, fixed order.
__global__ void __launch_bounds__(256) colsum_kernel(const float* __restrict__ D, int rows, int cols,
                                                     float* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= cols) return;
    float s = 0.f;
    for (int r = lane; r < rows; r += 32) s += D[(size_t)r * cols + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[j] = s;
}

// D = 2 (y - z) / count; loss += sum (y - z)^2 / count.
__global__ void __launch_bounds__(256) mse_kernel(const float* __restrict__ Y, const float* __restrict__ Z,
                                                  size_t count, float* __restrict__ D, float* __restrict__ loss)
{
    const float inv = 1.f / (float)count;
    float acc = 0.f;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
        const float r = Y[e] - Z[e];
        D[e] = 2.f * r * inv;
        acc = fmaf(r * inv, r, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (loss && (threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// AdamW on one parameter array (wd = 0 for biases); refreshes the bfloat16 copy.
__global__ void adamw_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                             float* __restrict__ v, __nv_bfloat16* __restrict__ w16, size_t count, float lr,
                             float beta1, float beta2, float eps, float wd, float c1, float c2)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
        const float ge = g[e];
        const float me = fmaf(beta1, m[e], (1.f - beta1) * ge);
        const float ve = fmaf(beta2, v[e], (1.f - beta2) * ge * ge);
        m[e] = me;
        v[e] = ve;
        const float mh = me * c1, vh = ve * c2;
        const float we = w[e] - lr * (mh / (sqrtf(vh) + eps) + wd * w[e]);
        w[e] = we;
        if (w16) w16[e] = __float2bfloat16_rn(we);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ w16, size_t count)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
        w16[e] = __float2bfloat16_rn(w[e]);
}

// ---------------------------------------------------------------------------
// Tensor-core GEMM (tcgen05) for the network's inference pass
//   C[i][j] = epi(sum_k A[i][k] Bt[j][k] + bias[j])
// A [M][K]: float32 (the features; rounded to bfloat16 as they are staged) or
// bfloat16 (hidden activations written by the previous layer's epilogue);
// Bt bfloat16 [N][K] (the transposed weights).  One CTA per 128 rows and BN
// (<= 128, a multiple of 16) columns; the accumulator tile lives in tensor
// memory, lane = row.  Operands are staged K-major in the unswizzled
// canonical layout of 8 x 8 bfloat16 core matrices (128 B, row r at 16 r),
// with the cores of one K group adjacent along the rows (stride-dimension
// offset 128 B) and K groups R / 8 x 128 B apart (leading-dimension offset),
// so that each thread writes whole 16-byte core rows and a warp's stores are
// contiguous.  Two stage buffers: while the MMAs of one 64-wide K stage run,
// the threads stage the next one; one elected thread issues the four
// tcgen05.mma (K = 16 each) of a stage and commits them to that buffer's
// mbarrier, which is waited (bounded) before the buffer is refilled.  The
// epilogue reads the accumulators with tcgen05.ld, adds the bias, applies
// GELU, and stores float32 or bfloat16 (the next layer's input; the same
// rounding the staging would apply).
// ---------------------------------------------------------------------------
namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int THREADS = 128;
constexpr int MAXBN = 128;
constexpr unsigned ERR_MBAR_TIMEOUT = 1u;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K direction) and
// stride (row-group direction) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Bounded wait on an mbarrier phase; on timeout sets the error word.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned* err)
{
    uint32_t done = 0;
    for (int pass = 0; pass < 2 && !done; ++pass) {
        for (int it = 0; it < (1 << 22) && !done; ++it) {
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(bar), "r"(parity)
                : "memory");
        }
        if (!done && pass == 0) atomicOr(err, ERR_MBAR_TIMEOUT);
    }
    return done != 0;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// One 16-byte core row (8 consecutive K elements of row `row`), as bfloat16.
template <typename TA>
__device__ __forceinline__ uint4 load_core_row(const TA* __restrict__ A, int lda, int row, int rows, int k, int K);

template <>
__device__ __forceinline__ uint4 load_core_row<float>(const float* __restrict__ A, int lda, int row, int rows, int k,
                                                      int K)
{
    float v[8];
    if (row < rows && k + 8 <= K && (lda & 3) == 0) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(A + (size_t)row * lda + k));
        const float4 b = __ldg(reinterpret_cast<const float4*>(A + (size_t)row * lda + k + 4));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (row < rows && k + e < K) ? A[(size_t)row * lda + k + e] : 0.f;
    }
    return make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
}

template <>
__device__ __forceinline__ uint4 load_core_row<__nv_bfloat16>(const __nv_bfloat16* __restrict__ A, int lda, int row,
                                                              int rows, int k, int K)
{
    if (row < rows && k + 8 <= K && (lda & 7) == 0)
        return __ldg(reinterpret_cast<const uint4*>(A + (size_t)row * lda + k));
    uint16_t u[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const __nv_bfloat16 h = (row < rows && k + e < K) ? A[(size_t)row * lda + k + e] : __float2bfloat16_rn(0.f);
        u[e] = *reinterpret_cast<const uint16_t*>(&h);
    }
    return make_uint4(u[0] | (uint32_t)u[1] << 16, u[2] | (uint32_t)u[3] << 16, u[4] | (uint32_t)u[5] << 16,
                      u[6] | (uint32_t)u[7] << 16);
}

template <typename TA, typename TC, bool GELU>
__global__ void __launch_bounds__(THREADS, 1) umma_gemm_kernel(int M, int N, int K, const TA* __restrict__ A, int lda,
                                                          const __nv_bfloat16* __restrict__ Bt,
                                                          const float* __restrict__ bias, TC* __restrict__ C, int ldc,
                                                          int BN, uint32_t ncols, unsigned* err)
{
    extern __shared__ __align__(1024) unsigned char tsm[];
    // per buffer: A [8 K groups][128 rows] core rows (16 KB), then B [8][BN] core rows
    const int a_bytes = BM * BK * 2, b_bytes = BN * BK * 2;
    unsigned char* buf[2] = {tsm, tsm + a_bytes + b_bytes};
    __shared__ __align__(8) unsigned long long s_mbar[2];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
    const uint32_t bar[2] = {saddr(&s_mbar[0]), saddr(&s_mbar[1])};
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s_tmem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar[0]), "r"(1) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar[1]), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    // instruction descriptor: D float32, A and B bfloat16, both K-major, N = BN, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    const int stages = (K + BK - 1) / BK;
    bool ok = true;
    for (int st = 0; st < stages && ok; ++st) {
        const int b = st & 1;
        if (st >= 2) ok = __syncthreads_and(mbar_wait(bar[b], (uint32_t)(((st - 2) >> 1) & 1), err) ? 1 : 0) != 0;
        if (!ok) break;
        const int k0 = st * BK;
        unsigned char* As = buf[b];
        unsigned char* Bs = buf[b] + a_bytes;
        {   // A: thread = row, 8 core rows (all loads first)
            uint4 v[8];
#pragma unroll
            for (int kc = 0; kc < 8; ++kc) v[kc] = load_core_row<TA>(A, lda, i0 + tid, M, k0 + 8 * kc, K);
#pragma unroll
            for (int kc = 0; kc < 8; ++kc) *reinterpret_cast<uint4*>(As + kc * (BM * 16) + tid * 16) = v[kc];
        }
        for (int r = tid; r < BN; r += THREADS) {  // B: thread = output column
            uint4 v[8];
#pragma unroll
            for (int kc = 0; kc < 8; ++kc)
                v[kc] = load_core_row<__nv_bfloat16>(Bt, K, j0 + r, N, k0 + 8 * kc, K);
#pragma unroll
            for (int kc = 0; kc < 8; ++kc) *reinterpret_cast<uint4*>(Bs + kc * (BN * 16) + r * 16) = v[kc];
        }
        // generic-proxy stores -> visible to the tensor core's async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t a_base = saddr(As), b_base = saddr(Bs);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                // K groups 2 kk, 2 kk + 1: leading offset = one K group; stride offset = 8 rows
                const uint64_t ad = smem_desc(a_base + (uint32_t)(2 * kk * BM * 16), (uint32_t)(BM * 16), 128u);
                const uint64_t bd = smem_desc(b_base + (uint32_t)(2 * kk * BN * 16), (uint32_t)(BN * 16), 128u);
                const uint32_t acc = (st > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar[b])
                         : "memory");
        }
    }
    // the last commit tracks every MMA issued before it
    if (ok && stages > 0)
        ok = __syncthreads_and(mbar_wait(bar[(stages - 1) & 1], (uint32_t)(((stages - 1) >> 1) & 1), err) ? 1 : 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const int gi = i0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(trow + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (gi < M) {
                float v[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int gj = j0 + c0 + c;
                    v[c] = __uint_as_float(r[c]) + (gj < N ? bias[gj] : 0.f);
                    if (GELU) v[c] = gelu(v[c]);
                }
                TC* out = C + (size_t)gi * ldc + j0 + c0;
                const bool full = j0 + c0 + 16 <= N;
                if (sizeof(TC) == 4) {
                    if (full && (ldc & 3) == 0) {
#pragma unroll
                        for (int c = 0; c < 16; c += 4)
                            *reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + c) =
                                make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
                    } else {
                        for (int c = 0; c < 16; ++c)
                            if (j0 + c0 + c < N) reinterpret_cast<float*>(out)[c] = v[c];
                    }
                } else {
                    if (full && (ldc & 7) == 0) {
#pragma unroll
                        for (int c = 0; c < 16; c += 8)
                            *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(out) + c) =
                                make_uint4(pack_bf16(v[c], v[c + 1]), pack_bf16(v[c + 2], v[c + 3]),
                                           pack_bf16(v[c + 4], v[c + 5]), pack_bf16(v[c + 6], v[c + 7]));
                    } else {
                        for (int c = 0; c < 16; ++c)
                            if (j0 + c0 + c < N) reinterpret_cast<__nv_bfloat16*>(out)[c] = __float2bfloat16_rn(v[c]);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// ---------------------------------------------------------------------------
// The same GEMM fed by TMA and pipelined (the inference path when every width
// is a multiple of 8): bfloat16 A [M][K] and Bt [N][K] come from tensor maps
// into a ring of S stages; each K step of an operand is one TMA box of {64
// elements, rows} in the 128-byte swizzle (rows of 128 B, their 16-byte chunks
// permuted within 8-row atoms), which the MMA descriptors read as is.  Warp specialisation (one
// elected lane each): warp 16 issues the TMA copies up to S stages ahead,
// warp 17 the MMAs, committing each stage to its `empty` barrier and each
// finished tile to its TMEM buffer's `full` barrier, so the tensor pipe is
// never left waiting for a copy to be issued; warps 0-15 drain the
// accumulators (four warps per TMEM sub-partition, every fourth 16-column
// chunk each), add the bias, apply GELU, store, and release the buffer.  Two
// TMEM accumulators, so the epilogue of one tile overlaps the loads and MMAs
// of the next; persistent CTAs loop over the tiles.  Every wait is bounded and
// records its expiry in the error word.
// ---------------------------------------------------------------------------
constexpr int TMA_STAGES = 4;
constexpr int EPI_WARPS = 16;
constexpr int EPI_PARTS = EPI_WARPS / 4;  // epilogue warps per TMEM sub-partition
constexpr int TMA_WARP = EPI_WARPS, MMA_WARP = EPI_WARPS + 1;
constexpr int TMA_THREADS = 32 * (EPI_WARPS + 2);

// GELU of two lanes with fused multiply-adds only: x Phi(x) with
// Phi(x) = sat(1/2 + x k(x^2)), k a degree-12 polynomial in
// u = 2 min(x^2, 25) / 25 - 1 (coefficients from csrc/fit_gelu.py: least
// squares on Chebyshev nodes, weighted by x^2, refined towards the minimax)
// and sat the clamp to [0, 1], which also gives the limits x and 0 beyond
// |x| = 5 without a branch.  |error| < 1.5e-6 in float32 -- far below the
// bfloat16 rounding the activations then undergo.
__device__ __forceinline__ float2 gelu_poly2(float2 x)
{
    constexpr float P[13] = {4.817027657e-04f,  -1.503391657e-03f, 2.027839655e-03f,  -2.940212376e-03f,
                             6.143897772e-03f,  -1.095324289e-02f, 1.650539227e-02f,  -2.334370278e-02f,
                             3.142509237e-02f,  -4.043198377e-02f, 5.152147263e-02f,  -7.029668987e-02f,
                             1.413637847e-01f};
    const float2 t = __fmul2_rn(x, x);
    const float2 u = __ffma2_rn(make_float2(fminf(t.x, 25.f), fminf(t.y, 25.f)), make_float2(0.08f, 0.08f),
                                make_float2(-1.f, -1.f));
    float2 p = make_float2(P[0], P[0]);
#pragma unroll
    for (int i = 1; i < 13; ++i) p = __ffma2_rn(p, u, make_float2(P[i], P[i]));
    const float2 phi = make_float2(__saturatef(__fmaf_rn(x.x, p.x, 0.5f)), __saturatef(__fmaf_rn(x.y, p.y, 0.5f)));
    return __fmul2_rn(x, phi);
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout that TMA writes with CU_TENSOR_MAP_SWIZZLE_128B: rows of
// 64 bfloat16 (128 B), 8-row atoms of 1024 B (the stride-dimension offset),
// the 16-byte chunks of row r at chunk ^ (r mod 8); atoms 1024-byte aligned so
// that the K offset inside an atom can be added to the start address.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// 16 accumulator columns of this thread's TMEM lane (row)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// What the pipelined kernel's epilogue makes of a 128 x BN accumulator tile.
enum : int {
    TE_HID = 0,    // inference, hidden layer: GELU(acc + bias) -> bfloat16 rows
    TE_OUT = 1,    // last layer: acc + bias -> float32 rows
    TE_TRAIN = 2,  // training, hidden layer: pre = acc + bias -> float32 rows (kept for the
                   // backward pass); GELU(pre) -> bfloat16 rows (the next layer's input) and
                   // bfloat16 columns (its input transposed, for the weight gradient)
    TE_DX = 3,     // backward product: acc * gelu'(pre) -> float32 rows (bias gradient),
                   // bfloat16 rows and columns (the operands of the next two products)
    TE_WGRAD = 4,  // weight gradient: acc -> float32 rows of split z's partial sum
};

// Destinations of the epilogue (row i, column j of the tile's product).
struct Epi {
    const float* bias;   // [N]: TE_HID, TE_OUT, TE_TRAIN
    float* f32;          // float32 rows, f32[z * zstride + i * ld32 + j]
    int ld32;
    __nv_bfloat16* r16;  // bfloat16 rows, r16[i * ld16 + j]
    int ld16;
    __nv_bfloat16* t16;  // bfloat16 columns, t16[j * ldT + i]
    int ldT;
    const float* pre;    // TE_DX: pre-activations pre[i * ldp + j]
    int ldp;
    size_t zstride;      // TE_WGRAD: elements between consecutive splits' partials
};

__device__ __forceinline__ void store_f32_16(float* o, const float2 (&v)[8], int cnt, bool vec)
{
    if (cnt >= 16 && vec) {
        float4* o4 = reinterpret_cast<float4*>(o);
#pragma unroll
        for (int c = 0; c < 4; ++c) o4[c] = make_float4(v[2 * c].x, v[2 * c].y, v[2 * c + 1].x, v[2 * c + 1].y);
    } else {
#pragma unroll
        for (int c = 0; c < 16; ++c)
            if (c < cnt) o[c] = (c & 1) ? v[c >> 1].y : v[c >> 1].x;
    }
}

__device__ __forceinline__ void store_bf16_16(__nv_bfloat16* o, const float2 (&v)[8], int cnt, bool vec)
{
    if (cnt >= 16 && vec) {
        uint4* o4 = reinterpret_cast<uint4*>(o);
        o4[0] = make_uint4(pack_bf16(v[0].x, v[0].y), pack_bf16(v[1].x, v[1].y), pack_bf16(v[2].x, v[2].y),
                           pack_bf16(v[3].x, v[3].y));
        o4[1] = make_uint4(pack_bf16(v[4].x, v[4].y), pack_bf16(v[5].x, v[5].y), pack_bf16(v[6].x, v[6].y),
                           pack_bf16(v[7].x, v[7].y));
    } else {
#pragma unroll
        for (int c = 0; c < 16; ++c)
            if (c < cnt) o[c] = __float2bfloat16_rn((c & 1) ? v[c >> 1].y : v[c >> 1].x);
    }
}

// column j0 + c of row gi at t[(j0 + c) * ldT + gi]: the 32 lanes of a warp
// (consecutive rows) write 64 contiguous bytes per column
__device__ __forceinline__ void store_bf16_cols(__nv_bfloat16* t, int ldT, int gi, int j0, const float2 (&v)[8],
                                                int cnt)
{
#pragma unroll
    for (int c = 0; c < 16; ++c)
        if (c < cnt) t[(size_t)(j0 + c) * ldT + gi] = __float2bfloat16_rn((c & 1) ? v[c >> 1].y : v[c >> 1].x);
}

// the epilogue of columns j0 .. j0 + 16 of row gi (sb: the bias of those
// columns in shared memory, 16-byte aligned; read only by the modes with a bias)
template <int MODE>
__device__ __forceinline__ void epilogue16(const uint32_t (&r)[16], const float* sb, int gi, int M, int j0, int N,
                                           int z, const Epi& e)
{
    float2 v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = make_float2(__uint_as_float(r[2 * c]), __uint_as_float(r[2 * c + 1]));
    if (MODE == TE_HID || MODE == TE_OUT || MODE == TE_TRAIN) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float4 b4 = reinterpret_cast<const float4*>(sb)[c];
            v[2 * c] = __fadd2_rn(v[2 * c], make_float2(b4.x, b4.y));
            v[2 * c + 1] = __fadd2_rn(v[2 * c + 1], make_float2(b4.z, b4.w));
        }
    }
    if (MODE == TE_HID) {
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = gelu_poly2(v[c]);
    }
    if (gi >= M) return;
    const int cnt = min(16, N - j0);
    if (MODE == TE_HID) {
        store_bf16_16(e.r16 + (size_t)gi * e.ld16 + j0, v, cnt, (e.ld16 & 7) == 0);
    } else if (MODE == TE_OUT) {
        store_f32_16(e.f32 + (size_t)gi * e.ld32 + j0, v, cnt, (e.ld32 & 3) == 0);
    } else if (MODE == TE_TRAIN) {
        store_f32_16(e.f32 + (size_t)gi * e.ld32 + j0, v, cnt, (e.ld32 & 3) == 0);
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = gelu_poly2(v[c]);
        store_bf16_16(e.r16 + (size_t)gi * e.ld16 + j0, v, cnt, (e.ld16 & 7) == 0);
        store_bf16_cols(e.t16, e.ldT, gi, j0, v, cnt);
    } else if (MODE == TE_DX) {
        const float* p = e.pre + (size_t)gi * e.ldp + j0;
        float pv[16];
        if (cnt >= 16 && (e.ldp & 3) == 0) {
#pragma unroll
            for (int c = 0; c < 16; c += 4) {
                const float4 t4 = *reinterpret_cast<const float4*>(p + c);
                pv[c] = t4.x; pv[c + 1] = t4.y; pv[c + 2] = t4.z; pv[c + 3] = t4.w;
            }
        } else {
#pragma unroll
            for (int c = 0; c < 16; ++c) pv[c] = c < cnt ? p[c] : 0.f;
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = make_float2(v[c].x * gelu_grad(pv[2 * c]), v[c].y * gelu_grad(pv[2 * c + 1]));
        store_f32_16(e.f32 + (size_t)gi * e.ld32 + j0, v, cnt, (e.ld32 & 3) == 0);
        store_bf16_16(e.r16 + (size_t)gi * e.ld16 + j0, v, cnt, (e.ld16 & 7) == 0);
        store_bf16_cols(e.t16, e.ldT, gi, j0, v, cnt);
    } else {
        store_f32_16(e.f32 + (size_t)z * e.zstride + (size_t)gi * e.ld32 + j0, v, cnt, (e.ld32 & 3) == 0);
    }
}

// The pipelined product C = A Bt^T over work units: a unit is one output
// tile and one of Z splits of the reduction (Z > 1 only for the weight
// gradients, whose reduction runs over the batch rows); split z covers the
// KS steps of BK from z KS BK, and steps past the operands' extent read the
// tensor maps' zero fill.  Unit u is tile u mod tiles, split u / tiles; the
// CTAs take units blockIdx.x, + gridDim.x, ...
template <int MODE>
__global__ void __launch_bounds__(TMA_THREADS, 1)
    umma_tma_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M,
                         int N, int KS, int Z, const Epi epi, int BN, uint32_t ncols, unsigned* err)
{
    extern __shared__ __align__(1024) unsigned char tsm_raw[];
    // the ring starts on a 1024-byte boundary (the request carries 1 KB of slack)
    unsigned char* tsm = tsm_raw + ((1024u - (saddr(tsm_raw) & 1023u)) & 1023u);
    const int a_bytes = BM * BK * 2, b_bytes = BN * BK * 2, st_bytes = a_bytes + b_bytes;
    __shared__ __align__(8) unsigned long long s_full[TMA_STAGES], s_empty[TMA_STAGES], s_tfull[2], s_tempty[2];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(16) float s_bias[MMPC_MLP_MAX_WIDTH];  // the layer's bias (N <= MMPC_MLP_MAX_WIDTH)
    constexpr bool has_bias = MODE == TE_HID || MODE == TE_OUT || MODE == TE_TRAIN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = (M + BM - 1) / BM, nt = (N + BN - 1) / BN, tiles = mt * nt, units = tiles * Z;
    if (has_bias)
        for (int j = tid; j < MMPC_MLP_MAX_WIDTH; j += blockDim.x) s_bias[j] = j < N ? epi.bias[j] : 0.f;
    if (warp == TMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s_tmem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < TMA_STAGES; ++i) {
            mbar_init(saddr(&s_full[i]), 1);
            mbar_init(saddr(&s_empty[i]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(saddr(&s_tfull[i]), 1);
            mbar_init(saddr(&s_tempty[i]), 32 * EPI_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t half = ncols / 2;  // columns per accumulator buffer
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    bool ok = true;
    // local units of this CTA: blockIdx.x, + gridDim.x, ...
    const int my_units = blockIdx.x < units ? (units - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int total = my_units * KS;  // K steps of this CTA, over its units in order
    if (warp == TMA_WARP) {
        // producer: fill stage g % S with the A and B tiles of K step g once
        // the MMAs of step g - S have released it
        if (lane == 0) {
            for (int g = 0; g < total && ok; ++g) {
                const int s = g % TMA_STAGES;
                if (g >= TMA_STAGES) ok = mbar_wait(saddr(&s_empty[s]), (uint32_t)(((g / TMA_STAGES) - 1) & 1), err);
                if (!ok) break;
                const int ui = g / KS, ks = g % KS;
                const int unit = (int)blockIdx.x + ui * (int)gridDim.x;
                const int tile = unit % tiles, z = unit / tiles;
                const int m0 = (tile % mt) * BM, n0 = (tile / mt) * BN, k0 = (z * KS + ks) * BK;
                const uint32_t full = saddr(&s_full[s]);
                const uint32_t base = saddr(tsm + (size_t)s * st_bytes);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full), "r"(st_bytes)
                             : "memory");
                tma_load_2d(base, &mapA, k0, m0, full);
                tma_load_2d(base + (uint32_t)a_bytes, &mapB, k0, n0, full);
            }
        }
        __syncwarp();
    } else if (warp == MMA_WARP) {
        // MMA issuer: step g once its stage has landed (and, at a unit's
        // first step, once the epilogue has drained the TMEM buffer of two
        // units back); each step's commit frees its stage, a unit's last
        // commit hands the accumulator to the epilogue
        if (lane == 0) {
            int g = 0;
            for (; g < total && ok; ++g) {
                const int s = g % TMA_STAGES;
                const int ui = g / KS, ks = g % KS, b = ui & 1;
                if (ks == 0 && ui >= 2) {
                    ok = mbar_wait(saddr(&s_tempty[b]), (uint32_t)(((ui - 2) >> 1) & 1), err);
                    if (!ok) break;
                }
                ok = mbar_wait(saddr(&s_full[s]), (uint32_t)((g / TMA_STAGES) & 1), err);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a_base = saddr(tsm + (size_t)s * st_bytes), b_base = a_base + (uint32_t)a_bytes;
                const uint32_t dtm = tmem + (uint32_t)b * half;
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {  // 16 K elements = 32 B further along each row
                    const uint64_t ad = sw128_desc(a_base + (uint32_t)(kk * 32));
                    const uint64_t bd = sw128_desc(b_base + (uint32_t)(kk * 32));
                    const uint32_t acc = (ks > 0 || kk > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtm),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 saddr(&s_empty[s]))
                             : "memory");
                if (ks == KS - 1)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     saddr(&s_tfull[b]))
                                 : "memory");
            }
            // after an expired wait, let the copies the producer issued land
            // before the CTA exits (bounded as well)
            for (int gg = g; gg < total && gg < g + TMA_STAGES; ++gg)
                mbar_wait(saddr(&s_full[gg % TMA_STAGES]), (uint32_t)((gg / TMA_STAGES) & 1), err);
        }
        __syncwarp();
    } else {
        // warp: TMEM sub-partition q (its 32 rows of the tile), and every
        // EPI_PARTS-th 16-column chunk starting at `part`
        const int q = warp & 3, part = warp >> 2, chunks = BN / 16;
        for (int ui = 0; ui < my_units && ok; ++ui) {
            const int b = ui & 1;
            const int unit = (int)blockIdx.x + ui * (int)gridDim.x;
            const int tile = unit % tiles, z = unit / tiles;
            const int m0 = (tile % mt) * BM, n0 = (tile / mt) * BN;
            const int gi = m0 + q * 32 + lane;
            const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)b * half;
            ok = mbar_wait(saddr(&s_tfull[b]), (uint32_t)((ui >> 1) & 1), err);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // this warp's chunks part, part + EPI_PARTS, ...: the TMEM load of
            // the next chunk is issued before the current one is processed (a
            // wait::ld covers every load issued so far)
            const int nch = chunks > part ? (chunks - part + EPI_PARTS - 1) / EPI_PARTS : 0;
            uint32_t ra[16], rb[16];
            if (nch > 0) tmem_ld16(trow + (uint32_t)(part * 16), ra);
            for (int i = 0; i < nch; i += 2) {
                const int ca = part + EPI_PARTS * i, cb = ca + EPI_PARTS;
                tmem_wait_ld();
                if (i + 1 < nch) tmem_ld16(trow + (uint32_t)(cb * 16), rb);
                epilogue16<MODE>(ra, s_bias + n0 + ca * 16, gi, M, n0 + ca * 16, N, z, epi);
                if (i + 1 < nch) {
                    tmem_wait_ld();
                    if (i + 2 < nch) tmem_ld16(trow + (uint32_t)((cb + EPI_PARTS) * 16), ra);
                    epilogue16<MODE>(rb, s_bias + n0 + cb * 16, gi, M, n0 + cb * 16, N, z, epi);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(saddr(&s_tempty[b]));
        }
    }
    // the last MMAs are complete once the epilogue has drained the last unit;
    // a CTA that gave up waits (bounded) for its outstanding commits first
    if (!ok && warp == MMA_WARP && lane == 0 && my_units > 0) {
        const int last = my_units - 1;
        mbar_wait(saddr(&s_tfull[last & 1]), (uint32_t)((last >> 1) & 1), err);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == TMA_WARP)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// ---------------------------------------------------------------------------
// The whole network in one persistent kernel (inference).  A CTA takes pairs
// of 128-row tiles; each tile's layer input lives in shared memory (the
// 128-byte-swizzled K-major layout the MMA descriptors read, 16 KB per 64
// columns), so hidden activations never leave the SM: the epilogue of layer l
// writes layer l + 1's input in place of layer l's, which the MMAs of layer
// l have finished reading.  The weights stream from L2 by TMA through a ring
// of boxes {64 K, 128 N} (16 KB), each box feeding the MMAs of both tiles, in
// the order (pair, layer, K block, N half) that the producer can run ahead in
// without waiting for activations.  Accumulators: tile t in TMEM columns
// [256 t, 256 t + 256).  Warp roles: 16 epilogue warps (tile t = warp / 8;
// TMEM sub-partition warp % 4; column chunks alternate between the two warps
// of a sub-partition), warp 16 the weight TMA, warp 17 the MMAs.  The
// features are read (float32, coalesced) and rounded to bfloat16 by the
// epilogue warps; the last layer's float32 outputs are staged in the tile's
// buffer and copied out in contiguous rows.  Every wait is bounded.
// ---------------------------------------------------------------------------
constexpr int FUSED_MAX_RING = 6;

struct FusedArgs {
    CUtensorMap wmap[MMPC_MLP_MAX_LAYERS];  // transposed bfloat16 weights [N_l][K_l], boxes {64, 128}
    const float* bias[MMPC_MLP_MAX_LAYERS];
    int width[MMPC_MLP_MAX_LAYERS + 1];
    int L, M, stages, bias_total;
    uint32_t h_bytes;                       // one tile's buffer (a multiple of 1024)
    const float* X;                         // [M][width[0]]
    float* Y;                               // [M][width[L]]
    unsigned* err;
};

// 16 bytes into the tile buffer: row r, 16-byte chunk j (8 bfloat16 columns)
// of 64-column block kb, at (j ^ (r mod 8)) within the row (the 128-byte
// swizzle of 8-row, 1024-byte atoms)
__device__ __forceinline__ void st_sw128(uint32_t hbase, int r, int kb, int j, uint4 v)
{
    const uint32_t a = hbase + (uint32_t)kb * 16384u + (uint32_t)(r >> 3) * 1024u + (uint32_t)(r & 7) * 128u +
                       ((uint32_t)(j ^ (r & 7)) << 4);
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

// bounded wait on an mbarrier completed by `count` arrivals of a group of
// warps (tile-local synchronisation of the epilogue warps)
__device__ __forceinline__ bool group_sync(uint32_t bar, uint32_t parity, unsigned* err)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
    return mbar_wait(bar, parity, err);
}

// 32 accumulator columns of this thread's TMEM lane, loaded and waited for in
// one statement (the registers are defined only once the wait returns)
__device__ __forceinline__ void tmem_ld32_wait(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

// one 16-column chunk c of a hidden layer's epilogue for row r (accumulators
// rv[o .. o + 16)): GELU(acc + b) as bfloat16 into the tile buffer (zeros for
// a chunk past N)
__device__ __forceinline__ void hidden_chunk(const uint32_t (&rv)[32], int o, const float* bl, uint32_t hbase, int r,
                                             int c, int N)
{
    uint4 lo = make_uint4(0, 0, 0, 0), hi = lo;
    if (c * 16 < N) {
        float2 v[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 b4 = reinterpret_cast<const float4*>(bl + c * 16)[k];
            v[2 * k] = gelu_poly2(__fadd2_rn(
                make_float2(__uint_as_float(rv[o + 4 * k]), __uint_as_float(rv[o + 4 * k + 1])), make_float2(b4.x, b4.y)));
            v[2 * k + 1] = gelu_poly2(__fadd2_rn(
                make_float2(__uint_as_float(rv[o + 4 * k + 2]), __uint_as_float(rv[o + 4 * k + 3])),
                make_float2(b4.z, b4.w)));
        }
        lo = make_uint4(pack_bf16(v[0].x, v[0].y), pack_bf16(v[1].x, v[1].y), pack_bf16(v[2].x, v[2].y),
                        pack_bf16(v[3].x, v[3].y));
        hi = make_uint4(pack_bf16(v[4].x, v[4].y), pack_bf16(v[5].x, v[5].y), pack_bf16(v[6].x, v[6].y),
                        pack_bf16(v[7].x, v[7].y));
    }
    st_sw128(hbase, r, c >> 2, (c & 3) * 2, lo);
    st_sw128(hbase, r, c >> 2, (c & 3) * 2 + 1, hi);
}

__global__ void __launch_bounds__(TMA_THREADS, 1) umma_mlp_fused_kernel(const __grid_constant__ FusedArgs args)
{
    extern __shared__ __align__(1024) unsigned char fsm_raw[];
    unsigned char* fsm = fsm_raw + ((1024u - (saddr(fsm_raw) & 1023u)) & 1023u);
    // [tile 0 buffer | tile 1 buffer | ring of stages x 16 KB | biases]
    const uint32_t hb = args.h_bytes;
    const uint32_t h0 = saddr(fsm), ring = h0 + 2 * hb;
    float* s_bias = reinterpret_cast<float*>(fsm + 2 * hb + (size_t)args.stages * 16384);
    __shared__ __align__(8) unsigned long long s_full[FUSED_MAX_RING], s_empty[FUSED_MAX_RING];
    __shared__ __align__(8) unsigned long long s_acc[2], s_ready[2], s_tile[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_boff[MMPC_MLP_MAX_LAYERS];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int L = args.L, M = args.M, S = args.stages;
    unsigned* err = args.err;
    if (tid == 0) {
        int o = 0;
        for (int l = 0; l < L; ++l) {
            s_boff[l] = o;
            o += (args.width[l + 1] + 15) / 16 * 16;
        }
    }
    if (warp == TMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s_tmem)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(saddr(&s_full[i]), 1);
            mbar_init(saddr(&s_empty[i]), 1);
        }
        for (int t = 0; t < 2; ++t) {
            mbar_init(saddr(&s_acc[t]), 1);
            mbar_init(saddr(&s_ready[t]), EPI_WARPS / 2);
            mbar_init(saddr(&s_tile[t]), EPI_WARPS / 2);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    for (int l = 0; l < L; ++l) {
        const int nl = args.width[l + 1], off = s_boff[l];
        for (int j = tid; j < (nl + 15) / 16 * 16; j += blockDim.x) s_bias[off + j] = j < nl ? args.bias[l][j] : 0.f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const int pairs = (M + 255) / 256;
    const int my_pairs = blockIdx.x < pairs ? (pairs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    bool ok = true;
    if (warp == TMA_WARP) {
        if (lane == 0) {
            int g = 0;
            for (int pi = 0; pi < my_pairs && ok; ++pi)
                for (int lt = 0; lt < 2 * L && ok; ++lt) {
                    const int l = lt >> 1;
                    const int KB = (args.width[l] + 63) / 64, NH = (args.width[l + 1] + 127) / 128;
                    for (int kb = 0; kb < KB && ok; ++kb)
                        for (int h = 0; h < NH && ok; ++h, ++g) {
                            const int s = g % S;
                            if (g >= S) ok = mbar_wait(saddr(&s_empty[s]), (uint32_t)(((g / S) - 1) & 1), err);
                            if (!ok) break;
                            const uint32_t full = saddr(&s_full[s]);
                            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full),
                                         "r"(16384)
                                         : "memory");
                            tma_load_2d(ring + (uint32_t)s * 16384u, &args.wmap[l], kb * 64, h * 128, full);
                        }
                }
        }
        __syncwarp();
    } else if (warp == MMA_WARP) {
        if (lane == 0) {
            int g = 0, issued0 = 0, issued1 = 0;  // layers committed per tile
            for (int pi = 0; pi < my_pairs && ok; ++pi)
                for (int lt = 0; lt < 2 * L && ok; ++lt) {
                    const int l = lt >> 1, t = lt & 1, e = pi * L + l;
                    ok = mbar_wait(saddr(&s_ready[t]), (uint32_t)(e & 1), err);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int N = args.width[l + 1];
                    const int KB = (args.width[l] + 63) / 64, NH = (N + 127) / 128;
                    for (int kb = 0; kb < KB && ok; ++kb)
                        for (int h = 0; h < NH && ok; ++h, ++g) {
                            const int s = g % S;
                            ok = mbar_wait(saddr(&s_full[s]), (uint32_t)((g / S) & 1), err);
                            if (!ok) break;
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const int nh = (min(128, N - 128 * h) + 15) / 16 * 16;
                            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nh >> 3) << 17) |
                                                   ((uint32_t)(BM >> 4) << 24);
                            const uint32_t bst = ring + (uint32_t)s * 16384u;
                            const uint32_t dtm = tmem + (uint32_t)(256 * t + 128 * h);
                            const uint32_t ast = h0 + (uint32_t)t * hb + (uint32_t)kb * 16384u;
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk) {
                                const uint64_t ad = sw128_desc(ast + (uint32_t)(kk * 32));
                                const uint64_t bd = sw128_desc(bst + (uint32_t)(kk * 32));
                                const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                                asm volatile(
                                    "{\n\t.reg .pred p;\n\t"
                                    "setp.ne.b32 p, %4, 0;\n\t"
                                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtm),
                                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                                    : "memory");
                            }
                            asm volatile(
                                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                    saddr(&s_empty[s]))
                                : "memory");
                        }
                    if (!ok) break;
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     saddr(&s_acc[t]))
                                 : "memory");
                    (t ? issued1 : issued0) = e + 1;
                }
            // after an expired wait: the copies issued by the producer land,
            // and the last committed layer's MMAs complete, before the CTA
            // exits (bounded as well)
            if (!ok) {
                for (int gg = g; gg < g + S; ++gg) mbar_wait(saddr(&s_full[gg % S]), (uint32_t)((gg / S) & 1), err);
                if (issued0 > 0) mbar_wait(saddr(&s_acc[0]), (uint32_t)((issued0 - 1) & 1), err);
                if (issued1 > 0) mbar_wait(saddr(&s_acc[1]), (uint32_t)((issued1 - 1) & 1), err);
            }
        }
        __syncwarp();
    } else {
        // epilogue warps: tile t, TMEM sub-partition q (rows 32 q .. 32 q + 31),
        // chunks part, part + 2, ... of 16 columns
        const int t = warp >> 3, q = warp & 3, part = (warp >> 2) & 1;
        const int r = q * 32 + lane;           // this thread's row in the tile
        const int tt = tid & 255;              // index among the tile's 256 threads
        const uint32_t hbase = h0 + (uint32_t)t * hb;
        float* stage = reinterpret_cast<float*>(fsm + (size_t)t * hb);
        const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(256 * t);
        const int w0 = args.width[0];
        int tsync = 0;  // completed phases of this tile's group barrier
        for (int pi = 0; pi < my_pairs && ok; ++pi) {
            const int m0 = ((int)blockIdx.x + pi * (int)gridDim.x) * 256 + t * 128;
            // the features: 8 float32 per thread and group, coalesced rows,
            // rounded to bfloat16 into block 0.. of the buffer; zeros past
            // width[0] (up to the 64-column block) and past M.  Two groups'
            // loads are in flight before the first is stored.
            const int kb0 = (w0 + 63) / 64, groups = 128 * kb0 * 8;
            for (int e0 = tt; e0 < groups; e0 += 2 * 256) {
                float4 va[2], vb[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int e8 = e0 + u * 256;
                    const int rr = e8 / (kb0 * 8), c0 = (e8 % (kb0 * 8)) * 8, gr = m0 + rr;
                    va[u] = vb[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (e8 < groups && gr < M) {
                        const float* src = args.X + (size_t)gr * w0 + c0;
                        if (c0 + 8 <= w0) {
                            va[u] = __ldg(reinterpret_cast<const float4*>(src));
                            vb[u] = __ldg(reinterpret_cast<const float4*>(src + 4));
                        } else if (c0 < w0) {
                            float v[8];
#pragma unroll
                            for (int k = 0; k < 8; ++k) v[k] = c0 + k < w0 ? src[k] : 0.f;
                            va[u] = make_float4(v[0], v[1], v[2], v[3]);
                            vb[u] = make_float4(v[4], v[5], v[6], v[7]);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int e8 = e0 + u * 256;
                    if (e8 >= groups) break;
                    const int rr = e8 / (kb0 * 8), cj = e8 % (kb0 * 8);
                    st_sw128(hbase, rr, cj >> 3, cj & 7,
                             make_uint4(pack_bf16(va[u].x, va[u].y), pack_bf16(va[u].z, va[u].w),
                                        pack_bf16(vb[u].x, vb[u].y), pack_bf16(vb[u].z, vb[u].w)));
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(saddr(&s_ready[t]));
            for (int l = 0; l < L && ok; ++l) {
                const int e = pi * L + l;
                ok = mbar_wait(saddr(&s_acc[t]), (uint32_t)(e & 1), err);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int N = args.width[l + 1];
                const float* bl = s_bias + s_boff[l];
                if (l < L - 1) {
                    // hidden layer: GELU(acc + b) as bfloat16 into the buffer
                    // (the next layer's input), zeros up to the 64-column block
                    // column groups of 32 (chunks 2 g, 2 g + 1), alternating
                    // between the two warps of the sub-partition
                    const int ngr = (N + 63) / 64 * 2;
                    for (int gq = part; gq < ngr; gq += 2) {
                        uint32_t rv[32];
                        if (gq * 32 < N) tmem_ld32_wait(trow + (uint32_t)(gq * 32), rv);
                        hidden_chunk(rv, 0, bl, hbase, r, 2 * gq, N);
                        hidden_chunk(rv, 16, bl, hbase, r, 2 * gq + 1, N);
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(saddr(&s_ready[t]));
                } else {
                    // last layer: acc + b (float32) staged as rows of N in the
                    // tile's buffer, then copied out as one contiguous range
                    for (int gq = part; gq * 32 < N; gq += 2) {
                        uint32_t rv[32];
                        tmem_ld32_wait(trow + (uint32_t)(gq * 32), rv);
                        const int cnt = min(32, N - gq * 32);
#pragma unroll
                        for (int k = 0; k < 32; ++k)
                            if (k < cnt) stage[r * N + gq * 32 + k] = __uint_as_float(rv[k]) + bl[gq * 32 + k];
                    }
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    ok = group_sync(saddr(&s_tile[t]), (uint32_t)(tsync & 1), err);
                    ++tsync;
                    if (!ok) break;
                    const int rows = max(0, min(128, M - m0));
                    const size_t total = (size_t)rows * N;
                    float* dst = args.Y + (size_t)min(m0, M) * N;
                    if ((N & 3) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
                        for (size_t i4 = tt; i4 < total / 4; i4 += 256)
                            reinterpret_cast<float4*>(dst)[i4] = reinterpret_cast<const float4*>(stage)[i4];
                    } else {
                        for (size_t i = tt; i < total; i += 256) dst[i] = stage[i];
                    }
                    // the buffer is free for the next pair's features
                    ok = group_sync(saddr(&s_tile[t]), (uint32_t)(tsync & 1), err);
                    ++tsync;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == TMA_WARP)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// features (float32) -> bfloat16 rows, the first layer's TMA operand
__global__ void rows_to_bf16_kernel(const float* __restrict__ X, size_t count, __nv_bfloat16* __restrict__ Y)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
        Y[e] = __float2bfloat16_rn(X[e]);
}

// float32 rows X [M][cols] (row stride ldx) -> bfloat16 rows R [M][ldr] and
// bfloat16 columns T [cols][ldT] (T[j ldT + i] = X[i][j]): the operands of a
// layer's two training products.  32 x 32 tiles pass through shared memory,
// so that the reads and both writes are coalesced.
__global__ void __launch_bounds__(256) rows_cols_bf16_kernel(const float* __restrict__ X, int M, int cols, int ldx,
                                                             __nv_bfloat16* __restrict__ R, int ldr,
                                                             __nv_bfloat16* __restrict__ T, int ldT)
{
    __shared__ float tile[32][33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + r, j = j0 + tx;
        float v = 0.f;
        if (i < M && j < cols) {
            v = X[(size_t)i * ldx + j];
            R[(size_t)i * ldr + j] = __float2bfloat16_rn(v);
        }
        tile[r][tx] = v;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int j = j0 + r, i = i0 + tx;
        if (j < cols && i < M) T[(size_t)j * ldT + i] = __float2bfloat16_rn(tile[tx][r]);
    }
}

// bfloat16 copy of W [K][N] transposed: Wt [N][K]
__global__ void to_bf16_t_kernel(const float* __restrict__ W, int K, int N, __nv_bfloat16* __restrict__ Wt)
{
    const size_t total = (size_t)K * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int n = (int)(e / K), k = (int)(e % K);
        Wt[e] = __float2bfloat16_rn(W[(size_t)k * N + n]);
    }
}

// bfloat16 copy of W [K][N] with rows padded to ldp >= N elements (16-byte
// rows for the tensor maps; the padding is never read)
__global__ void to_bf16_padded_kernel(const float* __restrict__ W, int K, int N, int ldp, __nv_bfloat16* __restrict__ Wp)
{
    const size_t total = (size_t)K * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / N), j = (int)(e % N);
        Wp[(size_t)k * ldp + j] = __float2bfloat16_rn(W[e]);
    }
}

}  // namespace tc

int grid_for(size_t count, int threads = 256)
{
    return (int)std::max<size_t>(1, std::min<size_t>((count + threads - 1) / threads, 152 * 16));
}

}  // namespace

// ---------------------------------------------------------------------------
// The network object
// ---------------------------------------------------------------------------
struct mmpc_mlp {
    mmpc_mlp_config cfg{};
    int L = 0, maxw = 0, inf_rows = 0, ksplit_rows = 512;
    std::vector<float*> W, b, gW, gb, mW, vW, mb, vb;
    std::vector<__nv_bfloat16*> W16;
    std::vector<__nv_bfloat16*> W16T;  // transposed copies [width[i+1]][width[i]] for the tensor-core path
    int tensor = 0;                    // inference: 0 SIMT, 1 TMA-fed tcgen05 pipeline, 2 single-stage tcgen05
    bool tma_widths = false;           // every layer input width a multiple of 8 (16-byte TMA rows)
    int sms = 0;
    __nv_bfloat16* Xb = nullptr;       // the features as bfloat16 [inf_rows][width[0]], the pipeline's first operand
    unsigned* d_err = nullptr;         // bounded-wait error word of the tensor-core kernels
    std::vector<float*> H;    // H[i]: input of layer i (i >= 1), [max_batch][width[i]]
    std::vector<float*> P;    // P[i]: pre-activation of layer i (hidden), [max_batch][width[i+1]]
    float* Yb = nullptr;      // [max_batch][width[L]]
    float* D0 = nullptr;      // backward ping-pong [max_batch][maxw]
    float* D1 = nullptr;
    float* part = nullptr;    // split-K partials of a weight gradient
    size_t part_count = 0;
    float* I0 = nullptr;      // inference ping-pong [inf_rows][maxw]
    float* I1 = nullptr;
    long long step = 0;
    // training on the tensor cores (mmpc_mlp_set_train_tensor_cores): the
    // bfloat16 operands of the three products of every layer, allocated on
    // first use
    int train_tensor = 0;
    int ldT = 0;                         // row stride of the column (transposed) buffers: max_batch rounded up to 8
    __nv_bfloat16* X16 = nullptr;        // features as bfloat16 rows [max_batch][width[0]]
    std::vector<__nv_bfloat16*> H16;     // H16[i] (i >= 1): layer i's input as bfloat16 rows [max_batch][width[i]]
    std::vector<__nv_bfloat16*> HT;      // HT[i]: layer i's input as bfloat16 columns [width[i]][ldT] (HT[0]: features)
    __nv_bfloat16* G16[2] = {nullptr, nullptr};  // output gradients, bfloat16 rows [max_batch][ld8(maxw)]
    __nv_bfloat16* GT[2] = {nullptr, nullptr};   // and columns [maxw][ldT]
    std::vector<__nv_bfloat16*> W16P;    // W16P[i]: bfloat16 W[i] with rows padded to ld8(width[i+1]) (only where width[i+1] % 8 != 0)
    float* tpart = nullptr;              // split partial sums of a weight gradient
    size_t tpart_count = 0;
    // the whole network in one kernel (inference, mode 1): shapes that fit,
    // its tensor maps of the transposed weights (made once: the buffers are
    // refreshed in place), and its launch shape
    bool fused_ok = false;
    tc::FusedArgs fused{};
    size_t fused_smem = 0;
};

namespace {

size_t wcount(const mmpc_mlp* n, int i) { return (size_t)n->cfg.width[i] * n->cfg.width[i + 1]; }

void mlp_free(mmpc_mlp* n)
{
    if (!n) return;
    auto f = [](void* p) { if (p) cudaFree(p); };
    for (auto* v : {&n->W, &n->b, &n->gW, &n->gb, &n->mW, &n->vW, &n->mb, &n->vb, &n->H, &n->P})
        for (float* p : *v) f(p);
    for (auto* p : n->W16) f(p);
    for (auto* p : n->W16T) f(p);
    for (auto* p : n->H16) f(p);
    for (auto* p : n->HT) f(p);
    for (auto* p : n->W16P) f(p);
    f(n->X16); f(n->G16[0]); f(n->G16[1]); f(n->GT[0]); f(n->GT[1]); f(n->tpart);
    f(n->d_err);
    f(n->Yb); f(n->D0); f(n->D1); f(n->part); f(n->I0); f(n->I1); f(n->Xb);
    delete n;
}

template <typename TBt, bool TA, bool TBT, int EPI>
void gemm(int M, int N, int K, int splits, const float* A, int lda, const TBt* B, int ldb, float* C, int ldc,
          const float* bias, float* pre, const float* aux, cudaStream_t st)
{
    const int kchunk = splits > 1 ? ((K + splits - 1) / splits + BK - 1) / BK * BK : K;
    const int z = splits > 1 ? (K + kchunk - 1) / kchunk : 1;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, z);
    gemm_kernel<TBt, TA, TBT, EPI><<<grid, 256, 0, st>>>(M, N, K, kchunk, A, lda, B, ldb, C, ldc, bias, pre, aux);
}

int splits_for(const mmpc_mlp* n, int rows) { return std::max(1, (rows + n->ksplit_rows - 1) / n->ksplit_rows); }

int ld8(int c) { return (c + 7) / 8 * 8; }

constexpr int MAX_WGRAD_SPLITS = 64;  // split partial sums of a weight gradient

void refresh_bf16(mmpc_mlp* n, int i, cudaStream_t st)
{
    const size_t wc = wcount(n, i);
    tc::to_bf16_t_kernel<<<grid_for(wc), 256, 0, st>>>(n->W[i], n->cfg.width[i], n->cfg.width[i + 1], n->W16T[i]);
    if (i < (int)n->W16P.size() && n->W16P[i])
        tc::to_bf16_padded_kernel<<<grid_for(wc), 256, 0, st>>>(n->W[i], n->cfg.width[i], n->cfg.width[i + 1],
                                                                 ld8(n->cfg.width[i + 1]), n->W16P[i]);
}

// Launch shape of the tensor-core GEMM for N outputs: BN columns per CTA
// (grid.y covers the rest), a power-of-two TMEM allocation, and a
// shared-memory request that keeps the CTAs resident on an SM within its 512
// TMEM columns.
struct TcShape {
    int BN;
    uint32_t ncols;
    size_t smem;
};

TcShape tc_shape(int N)
{
    TcShape t{};
    t.BN = std::min(tc::MAXBN, (N + 15) / 16 * 16);
    t.ncols = 32;
    while ((int)t.ncols < t.BN) t.ncols <<= 1;
    const size_t need = 2 * ((size_t)tc::BM * tc::BK * 2 + (size_t)t.BN * tc::BK * 2);
    const int per_sm = 512 / (int)t.ncols;
    const size_t cap = (size_t)(227 * 1024) / per_sm - 2048;
    t.smem = std::max(need, std::min<size_t>(cap, 227 * 1024));
    return t;
}

template <typename TA, typename TC, bool GELU>
void tc_launch(int M, int N, int K, const TA* A, const __nv_bfloat16* Bt, const float* bias, TC* C, unsigned* err,
               cudaStream_t st)
{
    const TcShape t = tc_shape(N);
    dim3 grid((M + tc::BM - 1) / tc::BM, (N + t.BN - 1) / t.BN);
    tc::umma_gemm_kernel<TA, TC, GELU><<<grid, tc::THREADS, t.smem, st>>>(M, N, K, A, K, Bt, bias, C, N, t.BN, t.ncols, err);
}

// cuTensorMapEncodeTiled, resolved once through the runtime (no link
// against the driver library); nullptr when the driver does not offer it.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder()
{
    static const EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (EncodeTiledFn) nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// Row-major bfloat16 matrix [rows][cols] with a row stride of ld elements
// (a multiple of 8: 16-byte rows; base 16-byte aligned) as a 2-D tensor map
// with boxes of {64 columns, box_rows rows} in the 128-byte swizzle: one K
// step (64 elements = 128 B per row) of box_rows rows per copy, landing in the
// layout the MMA descriptors read; outside the matrix (columns >= cols, rows
// >= rows) the box reads zeros.
bool encode_rows(CUtensorMap* map, const void* base, int cols, int ld, int rows, int box_rows)
{
    const EncodeTiledFn fn = tensor_map_encoder();
    if (!fn || ld % 8 != 0 || cols < 1 || cols > ld || rows < 1 || box_rows < 1 || box_rows > 256 ||
        (reinterpret_cast<uintptr_t>(base) & 15) != 0)
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1u, 1u};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Pipelined kernel's tile width for N outputs (one tile spans N <= 256), its
// TMEM allocation (two accumulators, a power of two >= 32 columns) and its
// shared memory (the ring of stages).  With the ring's size the CTAs that fit
// on an SM never ask for more than its 512 TMEM columns.
int tma_bn(int N) { return std::min(256, (N + 15) / 16 * 16); }

size_t tma_smem(int BN)
{
    return (size_t)tc::TMA_STAGES * ((size_t)tc::BM * tc::BK * 2 + (size_t)BN * tc::BK * 2) + 1024;
}

// C = A Bt^T through the pipelined kernel: A [M][K] (row stride lda), Bt
// [N][K] (row stride ldb), both bfloat16; the epilogue `epi` of MODE.  Z > 1
// splits the reduction into Z ranges of whole K steps, each unit writing its
// partial sum (TE_WGRAD); *splits_out (if given) receives the number of
// splits launched (ranges past K are dropped).  False when a tensor map
// cannot be made (nothing launched).
template <int MODE>
bool tma_run(const mmpc_mlp* n, int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* Bt,
             int ldb, int Z, const tc::Epi& epi, cudaStream_t st, int* splits_out = nullptr)
{
    const int BN = tma_bn(N);
    CUtensorMap ma, mb;
    if (!encode_rows(&ma, A, K, lda, M, tc::BM) || !encode_rows(&mb, Bt, K, ldb, N, BN)) return false;
    uint32_t ncols = 32;
    while ((int)ncols < 2 * BN) ncols <<= 1;
    const size_t smem = tma_smem(BN);
    const int ks_total = (K + tc::BK - 1) / tc::BK;
    Z = std::max(1, std::min(Z, ks_total));
    const int KS = (ks_total + Z - 1) / Z;
    Z = (ks_total + KS - 1) / KS;
    const int units = ((M + tc::BM - 1) / tc::BM) * ((N + BN - 1) / BN) * Z;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc::umma_tma_gemm_kernel<MODE>, tc::TMA_THREADS,
                                                      smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return false;
    }
    const int grid = std::max(1, std::min(units, n->sms * per_sm));
    tc::umma_tma_gemm_kernel<MODE><<<grid, tc::TMA_THREADS, smem, st>>>(ma, mb, M, N, KS, Z, epi, BN, ncols, n->d_err);
    if (splits_out) *splits_out = Z;
    return true;
}

// one inference layer: GELU + bfloat16 rows (hidden) or float32 rows (last)
template <typename TC, bool GELU>
bool tma_launch(const mmpc_mlp* n, int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* Bt,
                const float* bias, TC* C, cudaStream_t st)
{
    tc::Epi e{};
    e.bias = bias;
    if (GELU) {
        e.r16 = reinterpret_cast<__nv_bfloat16*>(C);
        e.ld16 = N;
        return tma_run<tc::TE_HID>(n, M, N, K, A, K, Bt, K, 1, e, st);
    }
    e.f32 = reinterpret_cast<float*>(C);
    e.ld32 = N;
    return tma_run<tc::TE_OUT>(n, M, N, K, A, K, Bt, K, 1, e, st);
}

// Inference on the tensor cores: hidden activations travel as bfloat16, the
// last layer writes float32.  The pipelined kernel reads its operands through
// tensor maps, so the features are first rounded to bfloat16 rows; the
// single-stage kernel (and any layer whose maps cannot be made) reads the
// float32 features itself.
void forward_tensor(mmpc_mlp* n, const float* X, int M, float* Y, float* b0, float* b1, cudaStream_t st)
{
    const int L = n->L;
    __nv_bfloat16* h[2] = {reinterpret_cast<__nv_bfloat16*>(b0), reinterpret_cast<__nv_bfloat16*>(b1)};
    const bool tma = n->tensor == 1 && n->tma_widths;
    if (tma) {
        const size_t cnt = (size_t)M * n->cfg.width[0];
        tc::rows_to_bf16_kernel<<<grid_for(cnt), 256, 0, st>>>(X, cnt, n->Xb);
    }
    for (int i = 0; i < L; ++i) {
        const int K = n->cfg.width[i], N = n->cfg.width[i + 1];
        const bool last = i == L - 1;
        const __nv_bfloat16* in = i == 0 ? n->Xb : h[(i + 1) & 1];
        __nv_bfloat16* out = h[i & 1];
        if (tma && (last ? tma_launch<float, false>(n, M, N, K, in, n->W16T[i], n->b[i], Y, st)
                         : tma_launch<__nv_bfloat16, true>(n, M, N, K, in, n->W16T[i], n->b[i], out, st)))
            continue;
        if (tma && i == 0) {
            if (last)
                tc_launch<__nv_bfloat16, float, false>(M, N, K, in, n->W16T[i], n->b[i], Y, n->d_err, st);
            else
                tc_launch<__nv_bfloat16, __nv_bfloat16, true>(M, N, K, in, n->W16T[i], n->b[i], out, n->d_err, st);
        } else if (i == 0 && last)
            tc_launch<float, float, false>(M, N, K, X, n->W16T[i], n->b[i], Y, n->d_err, st);
        else if (i == 0)
            tc_launch<float, __nv_bfloat16, true>(M, N, K, X, n->W16T[i], n->b[i], out, n->d_err, st);
        else if (last)
            tc_launch<__nv_bfloat16, float, false>(M, N, K, in, n->W16T[i], n->b[i], Y, n->d_err, st);
        else
            tc_launch<__nv_bfloat16, __nv_bfloat16, true>(M, N, K, in, n->W16T[i], n->b[i], out, n->d_err, st);
    }
}

// Forward over M <= rows of the buffers; keep = store pre-activations and
// layer inputs for the backward pass.
void forward_rows(mmpc_mlp* n, const float* X, int M, float* Y, bool keep, float* b0, float* b1, cudaStream_t st)
{
    const int L = n->L;
    const float* in = X;
    for (int i = 0; i < L; ++i) {
        const int K = n->cfg.width[i], N = n->cfg.width[i + 1];
        const bool last = i == L - 1;
        float* out = last ? Y : (keep ? n->H[i + 1] : (i % 2 == 0 ? b0 : b1));
        if (last)
            gemm<__nv_bfloat16, false, false, EPI_BIAS>(M, N, K, 1, in, K, n->W16[i], N, out, N, n->b[i], nullptr,
                                                        nullptr, st);
        else
            gemm<__nv_bfloat16, false, false, EPI_BIAS_GELU>(M, N, K, 1, in, K, n->W16[i], N, out, N, n->b[i],
                                                             keep ? n->P[i] : nullptr, nullptr, st);
        in = out;
    }
}

// Buffers of tensor-core training (first use); false on an allocation error.
bool ensure_train_buffers(mmpc_mlp* n)
{
    if (n->X16) return true;
    const int L = n->L;
    const int* w = n->cfg.width;
    const size_t mb = (size_t)n->cfg.max_batch;
    n->ldT = ld8(n->cfg.max_batch);
    cudaError_t e = cudaSuccess;
    auto bf = [&](__nv_bfloat16** p, size_t cnt) {
        if (e == cudaSuccess) e = cudaMalloc(p, sizeof(__nv_bfloat16) * std::max<size_t>(cnt, 1));
    };
    n->H16.assign(L, nullptr);
    n->HT.assign(L, nullptr);
    n->W16P.assign(L, nullptr);
    bf(&n->X16, mb * w[0]);
    for (int i = 0; i < L; ++i) {
        if (i >= 1) bf(&n->H16[i], mb * w[i]);
        bf(&n->HT[i], (size_t)w[i] * n->ldT);
        if (w[i + 1] % 8 != 0) bf(&n->W16P[i], (size_t)w[i] * ld8(w[i + 1]));
    }
    for (int k = 0; k < 2; ++k) {
        bf(&n->G16[k], mb * ld8(n->maxw));
        bf(&n->GT[k], (size_t)n->maxw * n->ldT);
    }
    size_t maxw_count = 0;
    for (int i = 0; i < L; ++i) maxw_count = std::max(maxw_count, wcount(n, i));
    n->tpart_count = maxw_count * MAX_WGRAD_SPLITS;
    if (e == cudaSuccess) e = cudaMalloc(&n->tpart, sizeof(float) * n->tpart_count);
    for (int i = 0; i < L && e == cudaSuccess; ++i) {
        refresh_bf16(n, i, 0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        // leave no half-made set behind: the next call retries from scratch
        auto f = [](void* p) { if (p) cudaFree(p); };
        for (auto* p : n->H16) f(p);
        for (auto* p : n->HT) f(p);
        for (auto* p : n->W16P) f(p);
        f(n->X16); f(n->G16[0]); f(n->G16[1]); f(n->GT[0]); f(n->GT[1]); f(n->tpart);
        n->H16.clear(); n->HT.clear(); n->W16P.clear();
        n->X16 = nullptr; n->G16[0] = n->G16[1] = n->GT[0] = n->GT[1] = nullptr; n->tpart = nullptr;
        cuda_fail(e, "tensor-core training buffers");
        return false;
    }
    return true;
}

void rows_cols(const float* X, int M, int cols, __nv_bfloat16* R, int ldr, __nv_bfloat16* T, int ldT, cudaStream_t st)
{
    dim3 grid((cols + 31) / 32, (M + 31) / 32);
    tc::rows_cols_bf16_kernel<<<grid, 256, 0, st>>>(X, M, cols, cols, R, ldr, T, ldT);
}

// Splits of a weight gradient's reduction over M rows: enough units to cover
// the SMs, at least two K steps (128 rows) per split.
int wgrad_splits(const mmpc_mlp* n, int K_out, int N_out, int M)
{
    const int tiles = ((K_out + tc::BM - 1) / tc::BM) * ((N_out + tma_bn(N_out) - 1) / tma_bn(N_out));
    const int ks = (M + tc::BK - 1) / tc::BK;
    return std::max(1, std::min({(n->sms + tiles - 1) / tiles, ks / 2, MAX_WGRAD_SPLITS}));
}

// Loss and gradients with the three products of every layer on the tensor
// cores (bfloat16 operands, float32 accumulation):
//   forward    P_i = H_i W_i + b_i, H_{i+1} = GELU(P_i)     A = H_i rows, Bt = W_i^T
//   backward   D_{i-1} = (D_i W_i^T) * GELU'(P_{i-1})       A = D_i rows, Bt = W_i
//   gradient   dW_i = H_i^T D_i, split over the rows        A = H_i columns, Bt = D_i columns
// with db_i the column sums of the float32 D_i.  Every epilogue writes the
// bfloat16 operands the later products read (rows and columns), so no
// separate rounding or transposition pass runs except for the features and
// the loss gradient.  Returns false if a tensor map could not be made.
bool loss_grad_tensor(mmpc_mlp* n, const float* X, const float* Z, int M, float* loss_out, cudaStream_t st)
{
    const int L = n->L;
    const int* w = n->cfg.width;
    rows_cols(X, M, w[0], n->X16, w[0], n->HT[0], n->ldT, st);
    for (int i = 0; i < L; ++i) {
        const __nv_bfloat16* in = i == 0 ? n->X16 : n->H16[i];
        tc::Epi e{};
        e.bias = n->b[i];
        if (i < L - 1) {
            e.f32 = n->P[i]; e.ld32 = w[i + 1];
            e.r16 = n->H16[i + 1]; e.ld16 = w[i + 1];
            e.t16 = n->HT[i + 1]; e.ldT = n->ldT;
            if (!tma_run<tc::TE_TRAIN>(n, M, w[i + 1], w[i], in, w[i], n->W16T[i], w[i], 1, e, st)) return false;
        } else {
            e.f32 = n->Yb; e.ld32 = w[L];
            if (!tma_run<tc::TE_OUT>(n, M, w[L], w[i], in, w[i], n->W16T[i], w[i], 1, e, st)) return false;
        }
    }
    const size_t cnt = (size_t)M * w[L];
    if (loss_out) cudaMemsetAsync(loss_out, 0, sizeof(float), st);
    mse_kernel<<<grid_for(cnt), 256, 0, st>>>(n->Yb, Z, cnt, n->D0, loss_out);
    rows_cols(n->D0, M, w[L], n->G16[0], ld8(w[L]), n->GT[0], n->ldT, st);
    float* Df = n->D0;
    float* Dn = n->D1;
    int cur = 0;
    for (int i = L - 1; i >= 0; --i) {
        const int K = w[i], N = w[i + 1];
        tc::Epi g{};
        g.f32 = n->tpart; g.ld32 = N; g.zstride = (size_t)K * N;
        int z = 1;
        if (!tma_run<tc::TE_WGRAD>(n, K, N, M, n->HT[i], n->ldT, n->GT[cur], n->ldT, wgrad_splits(n, K, N, M), g, st,
                                   &z))
            return false;
        reduce_partials_kernel<<<grid_for((size_t)K * N), 256, 0, st>>>(n->tpart, z, (size_t)K * N, n->gW[i]);
        colsum_kernel<<<(N + 7) / 8, 256, 0, st>>>(Df, M, N, n->gb[i]);
        if (i > 0) {
            tc::Epi d{};
            d.f32 = Dn; d.ld32 = K;
            d.r16 = n->G16[cur ^ 1]; d.ld16 = ld8(K);
            d.t16 = n->GT[cur ^ 1]; d.ldT = n->ldT;
            d.pre = n->P[i - 1]; d.ldp = K;
            const __nv_bfloat16* Wb = n->W16P[i] ? n->W16P[i] : n->W16[i];
            if (!tma_run<tc::TE_DX>(n, M, K, N, n->G16[cur], ld8(N), Wb, ld8(N), 1, d, st)) return false;
            std::swap(Df, Dn);
            cur ^= 1;
        }
    }
    return true;
}

// Shapes the single-kernel network takes: TMA rows of the weights (every
// layer input width a multiple of 8), inputs and hidden widths of at most
// 256 (four 64-column blocks per tile buffer, one 256-column accumulator per
// tile), an output of at most 128 columns (staged in a tile buffer), and a
// ring of at least two weight boxes beside the two tile buffers.  Makes the
// weights' tensor maps; false (and the layer-by-layer path) otherwise.
bool fused_setup(mmpc_mlp* n)
{
    const int L = n->L;
    const int* w = n->cfg.width;
    if (!n->tma_widths || !tensor_map_encoder() || L > MMPC_MLP_MAX_LAYERS || w[L] > 128) return false;
    int kbmax = 1, bias = 0;
    for (int l = 0; l < L; ++l) {
        if (w[l] > 256) return false;
        kbmax = std::max(kbmax, (w[l] + 63) / 64);
        bias += (w[l + 1] + 15) / 16 * 16;
    }
    tc::FusedArgs& f = n->fused;
    f = tc::FusedArgs{};
    const size_t stage = (size_t)tc::BM * w[L] * 4;
    f.h_bytes = (uint32_t)std::max<size_t>((size_t)kbmax * 16384, (stage + 1023) / 1024 * 1024);
    const size_t fixed = 2 * (size_t)f.h_bytes + (size_t)bias * 4 + 1024;
    const size_t cap = 227 * 1024;
    if (fixed + 2 * 16384 > cap) return false;
    f.stages = (int)std::min<size_t>(tc::FUSED_MAX_RING, (cap - fixed) / 16384);
    f.L = L;
    f.bias_total = bias;
    for (int l = 0; l <= L; ++l) f.width[l] = w[l];
    for (int l = 0; l < L; ++l) {
        f.bias[l] = n->b[l];
        if (!encode_rows(&f.wmap[l], n->W16T[l], w[l], w[l], w[l + 1], 128)) return false;
    }
    f.err = n->d_err;
    n->fused_smem = fixed + (size_t)f.stages * 16384;
    return cudaFuncSetAttribute(tc::umma_mlp_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)n->fused_smem) == cudaSuccess;
}

// Y [M][width[L]] = network(X [M][width[0]]) in one launch: one CTA per SM
// (the kernel takes all 512 TMEM columns), pairs of 128-row tiles.
bool fused_launch(mmpc_mlp* n, const float* X, int M, float* Y, cudaStream_t st)
{
    tc::FusedArgs f = n->fused;
    f.M = M;
    f.X = X;
    f.Y = Y;
    const int pairs = (M + 255) / 256;
    const int grid = std::max(1, std::min(pairs, n->sms));
    tc::umma_mlp_fused_kernel<<<grid, tc::TMA_THREADS, n->fused_smem, st>>>(f);
    return true;
}

bool valid_cfg(const mmpc_mlp_config* c)
{
    if (!c || c->layers < 1 || c->layers > MMPC_MLP_MAX_LAYERS || c->max_batch < 1) return false;
    for (int i = 0; i <= c->layers; ++i)
        if (c->width[i] < 1 || c->width[i] > MMPC_MLP_MAX_WIDTH) return false;
    return std::isfinite(c->beta1) && std::isfinite(c->beta2) && std::isfinite(c->eps) && std::isfinite(c->weight_decay) &&
           c->beta1 >= 0.f && c->beta1 < 1.f && c->beta2 >= 0.f && c->beta2 < 1.f && c->eps > 0.f && c->weight_decay >= 0.f;
}

int check_scenes(const mmpc_warm_scene* sc, int S)
{
    if (S < 0 || (S > 0 && !sc)) return fail(MMPC_ERR_INVALID_ARG, "scene table is NULL or S < 0");
    return MMPC_OK;
}

}  // namespace

extern "C" {

const char* mmpc_mlp_last_error(void) { return g_mlp_error.c_str(); }

int mmpc_features(const mmpc_warm_scene* scenes, int S, float a, float b, void* stream)
{
    int rc = check_scenes(scenes, S);
    if (rc) return rc;
    if (!(a > 0.f) || !(b > 0.f)) return fail(MMPC_ERR_INVALID_ARG, "ellipse semi-axes must be positive");
    if (S == 0) return MMPC_OK;
    features_kernel<<<S, 128, 0, (cudaStream_t)stream>>>(scenes, S, a, b);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MMPC_OK : cuda_fail(e, "features_kernel");
}

int mmpc_warm_decode(const mmpc_warm_scene* scenes, int S, int n, float T, int outputs, const float* mu,
                     const float* sigma, const float* Q, void* stream)
{
    int rc = check_scenes(scenes, S);
    if (rc) return rc;
    if (n < MMPC_MIN_COEF || n > MMPC_MAX_COEF || !(T > 0.f) || !mu || !sigma || (outputs != 3 * n && outputs != 6 * n))
        return fail(MMPC_ERR_INVALID_ARG, "bad n, T, outputs or NULL mu / sigma");
    if (S == 0) return MMPC_OK;
    decode_kernel<<<S, 256, 0, (cudaStream_t)stream>>>(scenes, S, n, T, outputs, mu, sigma, Q);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MMPC_OK : cuda_fail(e, "decode_kernel");
}

int mmpc_warm_encode(const mmpc_warm_scene* scenes, int S, int n, float T, int outputs, const float* mu,
                     const float* sigma, void* stream)
{
    int rc = check_scenes(scenes, S);
    if (rc) return rc;
    if (n < MMPC_MIN_COEF || n > MMPC_MAX_COEF || !(T > 0.f) || !mu || !sigma || (outputs != 3 * n && outputs != 6 * n))
        return fail(MMPC_ERR_INVALID_ARG, "bad n, T, outputs or NULL mu / sigma");
    if (S == 0) return MMPC_OK;
    encode_kernel<<<S, 256, 0, (cudaStream_t)stream>>>(scenes, S, n, T, outputs, mu, sigma);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MMPC_OK : cuda_fail(e, "encode_kernel");
}

int mmpc_column_stats(const float* X, int rows, int cols, float* mean_out, float* std_out, void* stream)
{
    if (!X || !mean_out || !std_out || rows < 1 || cols < 1) return fail(MMPC_ERR_INVALID_ARG, "bad column_stats arguments");
    column_stats_kernel<<<cols, 256, 0, (cudaStream_t)stream>>>(X, rows, cols, mean_out, std_out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MMPC_OK : cuda_fail(e, "column_stats_kernel");
}

int mmpc_standardize(const float* X, int rows, int cols, const float* mean, const float* sd, float* out, void* stream)
{
    if (!X || !mean || !sd || !out || rows < 0 || cols < 1) return fail(MMPC_ERR_INVALID_ARG, "bad standardize arguments");
    if (rows == 0) return MMPC_OK;
    standardize_kernel<<<grid_for((size_t)rows * cols), 256, 0, (cudaStream_t)stream>>>(X, rows, cols, mean, sd, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MMPC_OK : cuda_fail(e, "standardize_kernel");
}

int mmpc_gather_rows(const float* src, int src_rows, int cols, const int* idx, int rows, float* out, void* stream)
{
    if (!src || !idx || !out || src_rows < 0 || cols < 1 || rows < 0) return fail(MMPC_ERR_INVALID_ARG, "bad gather arguments");
    if (rows == 0) return MMPC_OK;
    gather_kernel<<<grid_for((size_t)rows * cols), 256, 0, (cudaStream_t)stream>>>(src, src_rows, cols, idx, rows, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MMPC_OK : cuda_fail(e, "gather_kernel");
}

int mmpc_mlp_create(const mmpc_mlp_config* cfg, const float* const* W, const float* const* b, mmpc_mlp** out)
{
    if (out) *out = nullptr;
    if (!out || !W || !b) return fail(MMPC_ERR_INVALID_ARG, "NULL argument");
    if (!valid_cfg(cfg)) return fail(MMPC_ERR_INVALID_ARG, "invalid network configuration");
    for (int i = 0; i < cfg->layers; ++i)
        if (!W[i] || !b[i]) return fail(MMPC_ERR_INVALID_ARG, "NULL weight or bias array");
    mmpc_mlp* n = new mmpc_mlp();
    n->cfg = *cfg;
    n->L = cfg->layers;
    n->maxw = *std::max_element(cfg->width, cfg->width + cfg->layers + 1);
    // inference chunk: four 128-row tiles per SM (every persistent CTA of
    // the pipelined GEMM gets the same share), at least 65536 rows; the
    // bfloat16 activations of a chunk stay in L2 between layers
    int dev0 = 0, sms0 = 0;
    if (cudaGetDevice(&dev0) != cudaSuccess || cudaDeviceGetAttribute(&sms0, cudaDevAttrMultiProcessorCount, dev0) != cudaSuccess)
        sms0 = 128;
    cudaGetLastError();
    n->inf_rows = std::max(cfg->max_batch, std::max(65536, sms0 * 128 * 4));
    const size_t mb = (size_t)cfg->max_batch;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](float** p, size_t cnt) {
        if (e == cudaSuccess) e = cudaMalloc(p, sizeof(float) * std::max<size_t>(cnt, 1));
    };
    const int L = n->L;
    n->W.assign(L, nullptr); n->b.assign(L, nullptr); n->gW.assign(L, nullptr); n->gb.assign(L, nullptr);
    n->mW.assign(L, nullptr); n->vW.assign(L, nullptr); n->mb.assign(L, nullptr); n->vb.assign(L, nullptr);
    n->W16.assign(L, nullptr); n->W16T.assign(L, nullptr); n->H.assign(L, nullptr); n->P.assign(L, nullptr);
    if (e == cudaSuccess) e = cudaMalloc(&n->d_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(n->d_err, 0, sizeof(unsigned));
    size_t maxw_count = 0;
    for (int i = 0; i < L; ++i) {
        const size_t wc = wcount(n, i), bc = cfg->width[i + 1];
        maxw_count = std::max(maxw_count, wc);
        alloc(&n->W[i], wc); alloc(&n->gW[i], wc); alloc(&n->mW[i], wc); alloc(&n->vW[i], wc);
        alloc(&n->b[i], bc); alloc(&n->gb[i], bc); alloc(&n->mb[i], bc); alloc(&n->vb[i], bc);
        if (e == cudaSuccess) e = cudaMalloc(&n->W16[i], sizeof(__nv_bfloat16) * wc);
        if (e == cudaSuccess) e = cudaMalloc(&n->W16T[i], sizeof(__nv_bfloat16) * wc);
        if (i >= 1) alloc(&n->H[i], mb * cfg->width[i]);
        if (i < L - 1) alloc(&n->P[i], mb * cfg->width[i + 1]);
    }
    alloc(&n->Yb, mb * cfg->width[L]);
    alloc(&n->D0, mb * n->maxw);
    alloc(&n->D1, mb * n->maxw);
    const int zmax = splits_for(n, cfg->max_batch);
    n->part_count = maxw_count * zmax;
    alloc(&n->part, n->part_count);
    alloc(&n->I0, (size_t)n->inf_rows * n->maxw);
    alloc(&n->I1, (size_t)n->inf_rows * n->maxw);
    if (e == cudaSuccess) e = cudaMalloc(&n->Xb, sizeof(__nv_bfloat16) * (size_t)n->inf_rows * cfg->width[0]);
    n->tma_widths = true;
    for (int i = 0; i < L; ++i) n->tma_widths = n->tma_widths && cfg->width[i] % 8 == 0;
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, dev);
    for (int i = 0; i < L && e == cudaSuccess; ++i) {
        const size_t wc = wcount(n, i), bc = cfg->width[i + 1];
        e = cudaMemcpy(n->W[i], W[i], sizeof(float) * wc, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(n->b[i], b[i], sizeof(float) * bc, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(n->mW[i], 0, sizeof(float) * wc);
        if (e == cudaSuccess) e = cudaMemset(n->vW[i], 0, sizeof(float) * wc);
        if (e == cudaSuccess) e = cudaMemset(n->mb[i], 0, sizeof(float) * bc);
        if (e == cudaSuccess) e = cudaMemset(n->vb[i], 0, sizeof(float) * bc);
        if (e == cudaSuccess) e = cudaMemset(n->gW[i], 0, sizeof(float) * wc);
        if (e == cudaSuccess) e = cudaMemset(n->gb[i], 0, sizeof(float) * bc);
        if (e == cudaSuccess) {
            to_bf16_kernel<<<grid_for(wc), 256>>>(n->W[i], n->W16[i], wc);
            refresh_bf16(n, i, 0);
            e = cudaGetLastError();
        }
    }
    size_t tc_smem = 0;  // the attribute must cover every layer's request
    for (int i = 0; i < L; ++i) tc_smem = std::max(tc_smem, tc_shape(cfg->width[i + 1]).smem);
    const void* tc_kernels[] = {(const void*)tc::umma_gemm_kernel<float, float, false>,
                                (const void*)tc::umma_gemm_kernel<float, __nv_bfloat16, true>,
                                (const void*)tc::umma_gemm_kernel<__nv_bfloat16, float, false>,
                                (const void*)tc::umma_gemm_kernel<__nv_bfloat16, __nv_bfloat16, true>};
    for (const void* kf : tc_kernels)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem);
    size_t tma_max = 0;
    for (int i = 0; i <= L; ++i) tma_max = std::max(tma_max, tma_smem(tma_bn(cfg->width[i])));
    const void* tma_kernels[] = {(const void*)tc::umma_tma_gemm_kernel<tc::TE_HID>,
                                 (const void*)tc::umma_tma_gemm_kernel<tc::TE_OUT>,
                                 (const void*)tc::umma_tma_gemm_kernel<tc::TE_TRAIN>,
                                 (const void*)tc::umma_tma_gemm_kernel<tc::TE_DX>,
                                 (const void*)tc::umma_tma_gemm_kernel<tc::TE_WGRAD>};
    for (const void* kf : tma_kernels)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_max);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) {
        n->fused_ok = fused_setup(n);
        cudaGetLastError();  // a refused shape leaves the layer-by-layer path
    }
    if (e != cudaSuccess) {
        mlp_free(n);
        return cuda_fail(e, "mmpc_mlp_create");
    }
    *out = n;
    return MMPC_OK;
}

int mmpc_mlp_forward(mmpc_mlp* n, const float* X, int M, float* Y, void* stream)
{
    if (!n) return fail(MMPC_ERR_NOT_SETUP, "NULL network");
    if (M < 0 || (M > 0 && (!X || !Y))) return fail(MMPC_ERR_INVALID_ARG, "bad forward arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int in = n->cfg.width[0], outw = n->cfg.width[n->L];
    if (n->tensor == 1 && n->fused_ok && M > 0 && fused_launch(n, X, M, Y, st)) {
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? MMPC_OK : cuda_fail(e, "mmpc_mlp_forward");
    }
    for (int r0 = 0; r0 < M; r0 += n->inf_rows) {
        const int rows = std::min(n->inf_rows, M - r0);
        if (n->tensor)
            forward_tensor(n, X + (size_t)r0 * in, rows, Y + (size_t)r0 * outw, n->I0, n->I1, st);
        else
            forward_rows(n, X + (size_t)r0 * in, rows, Y + (size_t)r0 * outw, false, n->I0, n->I1, st);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MMPC_OK : cuda_fail(e, "mmpc_mlp_forward");
}

int mmpc_mlp_loss_grad(mmpc_mlp* n, const float* X, const float* Z, int M, float* loss_out, void* stream)
{
    if (!n) return fail(MMPC_ERR_NOT_SETUP, "NULL network");
    if (!X || !Z || M < 1 || M > n->cfg.max_batch) return fail(MMPC_ERR_INVALID_ARG, "bad loss_grad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    if (n->train_tensor) {
        if (!loss_grad_tensor(n, X, Z, M, loss_out, st))
            return fail(MMPC_ERR_CUDA, "mmpc_mlp_loss_grad: a tensor map could not be made");
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? MMPC_OK : cuda_fail(e, "mmpc_mlp_loss_grad");
    }
    const int L = n->L;
    forward_rows(n, X, M, n->Yb, true, nullptr, nullptr, st);
    const size_t cnt = (size_t)M * n->cfg.width[L];
    if (loss_out) cudaMemsetAsync(loss_out, 0, sizeof(float), st);
    mse_kernel<<<grid_for(cnt), 256, 0, st>>>(n->Yb, Z, cnt, n->D0, loss_out);
    float* D = n->D0;
    float* Dn = n->D1;
    const int splits = splits_for(n, M);
    for (int i = L - 1; i >= 0; --i) {
        const int K = n->cfg.width[i], N = n->cfg.width[i + 1];
        const float* Hin = i == 0 ? X : n->H[i];
        // dW[i] = H^T D: (K x M) (M x N), split over the M rows, reduced in order
        gemm<float, true, false, EPI_PARTIAL>(K, N, M, splits, Hin, K, D, N, n->part, N, nullptr, nullptr, nullptr, st);
        const int kchunk = ((M + splits - 1) / splits + BK - 1) / BK * BK;
        const int z = (M + kchunk - 1) / kchunk;
        reduce_partials_kernel<<<grid_for((size_t)K * N), 256, 0, st>>>(n->part, z, (size_t)K * N, n->gW[i]);
        colsum_kernel<<<(N + 7) / 8, 256, 0, st>>>(D, M, N, n->gb[i]);
        if (i > 0) {
            // D_prev = (D W^T) * gelu'(P[i-1])
            gemm<__nv_bfloat16, false, true, EPI_GELU_GRAD>(M, K, N, 1, D, N, n->W16[i], N, Dn, K, nullptr, nullptr,
                                                            n->P[i - 1], st);
            std::swap(D, Dn);
        }
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MMPC_OK : cuda_fail(e, "mmpc_mlp_loss_grad");
}

int mmpc_mlp_adamw(mmpc_mlp* n, float lr, void* stream)
{
    if (!n) return fail(MMPC_ERR_NOT_SETUP, "NULL network");
    if (!std::isfinite(lr) || lr < 0.f) return fail(MMPC_ERR_INVALID_ARG, "bad learning rate");
    cudaStream_t st = (cudaStream_t)stream;
    n->step += 1;
    const mmpc_mlp_config& c = n->cfg;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)c.beta1, (double)n->step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)c.beta2, (double)n->step)));
    for (int i = 0; i < n->L; ++i) {
        const size_t wc = wcount(n, i), bc = c.width[i + 1];
        adamw_kernel<<<grid_for(wc), 256, 0, st>>>(n->W[i], n->gW[i], n->mW[i], n->vW[i], n->W16[i], wc, lr, c.beta1,
                                                   c.beta2, c.eps, c.weight_decay, c1, c2);
        adamw_kernel<<<grid_for(bc), 256, 0, st>>>(n->b[i], n->gb[i], n->mb[i], n->vb[i], nullptr, bc, lr, c.beta1,
                                                   c.beta2, c.eps, 0.f, c1, c2);
        refresh_bf16(n, i, st);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MMPC_OK : cuda_fail(e, "mmpc_mlp_adamw");
}

int mmpc_mlp_read(mmpc_mlp* n, int what, int layer, float* host, size_t count)
{
    if (!n) return fail(MMPC_ERR_NOT_SETUP, "NULL network");
    if (layer < 0 || layer >= n->L || !host || what < 0 || what > 7) return fail(MMPC_ERR_INVALID_ARG, "bad read arguments");
    const bool isw = what == 0 || what == 2 || what == 4 || what == 5;
    const size_t want = isw ? wcount(n, layer) : (size_t)n->cfg.width[layer + 1];
    if (count != want) return fail(MMPC_ERR_SHAPE, "count does not match the array size");
    const float* src = what == 0 ? n->W[layer] : what == 1 ? n->b[layer] : what == 2 ? n->gW[layer]
                     : what == 3 ? n->gb[layer] : what == 4 ? n->mW[layer] : what == 5 ? n->vW[layer]
                     : what == 6 ? n->mb[layer] : n->vb[layer];
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host, src, sizeof(float) * count, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "mmpc_mlp_read");
    unsigned err = 0;
    e = cudaMemcpy(&err, n->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "mmpc_mlp_read");
    if (err) return fail(MMPC_ERR_TIMEOUT, "a tensor-core wait expired in an earlier forward pass");
    return MMPC_OK;
}

int mmpc_mlp_write(mmpc_mlp* n, int what, int layer, const float* host, size_t count)
{
    if (!n) return fail(MMPC_ERR_NOT_SETUP, "NULL network");
    if (layer < 0 || layer >= n->L || !host || (what != 0 && what != 1)) return fail(MMPC_ERR_INVALID_ARG, "bad write arguments");
    const size_t want = what == 0 ? wcount(n, layer) : (size_t)n->cfg.width[layer + 1];
    if (count != want) return fail(MMPC_ERR_SHAPE, "count does not match the array size");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(what == 0 ? n->W[layer] : n->b[layer], host, sizeof(float) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && what == 0) {
        to_bf16_kernel<<<grid_for(count), 256>>>(n->W[layer], n->W16[layer], count);
        refresh_bf16(n, layer, 0);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    return e == cudaSuccess ? MMPC_OK : cuda_fail(e, "mmpc_mlp_write");
}

int mmpc_mlp_forward_launches(mmpc_mlp* n, int M)
{
    if (!n || M < 0) return -1;
    if (M == 0) return 0;
    if (n->tensor == 1 && n->fused_ok) return 1;
    const int chunks = (M + n->inf_rows - 1) / n->inf_rows;
    const int per_chunk = n->L + ((n->tensor == 1 && n->tma_widths) ? 1 : 0);
    return chunks * per_chunk;
}

int mmpc_mlp_set_tensor_cores(mmpc_mlp* n, int on)
{
    if (!n) return fail(MMPC_ERR_NOT_SETUP, "NULL network");
    if (on < 0 || on > 2) return fail(MMPC_ERR_INVALID_ARG, "tensor-core mode must be 0, 1 or 2");
    n->tensor = on;
    return MMPC_OK;
}

int mmpc_mlp_set_train_tensor_cores(mmpc_mlp* n, int on)
{
    if (!n) return fail(MMPC_ERR_NOT_SETUP, "NULL network");
    if (on != 0 && on != 1) return fail(MMPC_ERR_INVALID_ARG, "training mode must be 0 or 1");
    if (on) {
        if (!n->tma_widths || !tensor_map_encoder())
            return fail(MMPC_ERR_INVALID_ARG, "tensor-core training needs every layer input width a multiple of 8");
        if (n->cfg.max_batch > 65535 * 32) return fail(MMPC_ERR_INVALID_ARG, "max_batch too large for tensor-core training");
        if (!ensure_train_buffers(n)) return MMPC_ERR_CUDA;
    }
    n->train_tensor = on;
    return MMPC_OK;
}

int mmpc_mlp_status(mmpc_mlp* n)
{
    if (!n) return fail(MMPC_ERR_NOT_SETUP, "NULL network");
    unsigned err = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&err, n->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "mmpc_mlp_status");
    return err ? fail(MMPC_ERR_TIMEOUT, "a tensor-core wait expired") : MMPC_OK;
}

void mmpc_mlp_destroy(mmpc_mlp* n)
{
    if (!n) return;
    cudaDeviceSynchronize();
    mlp_free(n);
}

}  // extern "C"
