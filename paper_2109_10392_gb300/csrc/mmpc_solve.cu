// GB300 (sm_103a) kernels and C ABI of the batch non-holonomic trajectory
// optimizer (Adajania et al., arXiv 2109.10392, Algorithm 1 of Sec. III-E).
//
// Solve kernel: one CTA per trajectory l of the batch, one thread per pair of
// time samples (2i, 2i+1), whose arithmetic runs as packed f32x2 operations
// (FFMA2 / FADD2 / FMUL2: one issue slot for two samples in the projections,
// for two coefficients in the basis products).  Every quantity that
// Algorithm 1 carries from one iteration to the next for trajectory l --
// c_x, c_y, c_psi and lambda_x, lambda_y, lambda_psi -- stays on chip for all
// iterations (in registers: with 1-2 warps per trajectory every warp runs the
// small QP steps on the same partial sums, with more warps warp 0 alone does
// and shares the coefficients through shared memory); the auxiliary
// variables v, alpha, d, alpha_a, d_a of Eqs.
// split_v, split_alpha_o and split_alpha_a are closed-form functions of the
// coefficients and are recomputed in registers where they are used.  The
// shared matrices (basis rows, KKT inverse blocks) are staged once per CTA
// into shared memory by a TMA bulk copy.
//
// Arithmetic forms used here (each exact in real arithmetic; chosen because
// FP32 carries them to 1e-4 m where the textbook forms lose 0.1 m):
//  * F^T g without F: F_o is P stacked m times (Sec. III-B), so the obstacle
//    block contributes P^T sum_j (...), a sum over obstacles per sample.
//  * Step (split_xy) as an increment.  With the KKT identity K11 M + K12 A = I
//    (M = Q + rho F^T F) and A c^k = b, Eq. lin_solve_xy_2 becomes
//        c^{k+1} = c^k + K11 (lambda^k - Q c^k - rho F^T (F c^k - g^k)),
//    whose right-hand side holds only residual-sized numbers.  The FP32 sum
//    c^k + delta is compensated (carry e), and K11 is applied as hi + lo FP32.
//  * Step (split_alpha_o) without trigonometry: with alpha from its closed
//    form, the unconstrained d equals the ellipse-normalised distance
//    r = |((x - xi_x)/a, (y - xi_y)/b)|, so the target xi + (a d cos alpha,
//    b d sin alpha) equals x + w max(0, 1/r - 1) with w = (x - xi_x, y - xi_y).
//  * x is carried relative to x_ref(t) = v0 t (coefficients v0 lin), and the
//    obstacles in that moving frame; velocity rows add v0 back.  This keeps
//    the carried coefficients small; outputs are in the road frame.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mmpc.h"
#include "mmpc_internal.h"

namespace mmpc {

namespace {
thread_local std::string g_error = "no error";
}
void set_global_error(const std::string& msg) { g_error = msg; }

// ---------------------------------------------------------------------------
// Device constant blob (FP32), section offsets in floats, every section on a
// 16-byte boundary.  Three regions:
//   [pair rows | common | sample rows]
// The pair-sample kernel stages [pair rows | common] into shared memory, the
// one-sample kernel [common | sample rows]; the scoring kernels read the
// sample rows from global memory.
//   pair rows:   PP, PdP, PddP [NPT][RS]  basis rows of samples (2i, 2i+1),
//                per coefficient pair (2j, 2j+1) the 16-byte block (2i: 2j,
//                2j+1; 2i+1: 2j, 2j+1) (RS = pair_stride(NC) floats with the
//                padding), NPT = ceil(N/2) + 1: the pairs and one zero row
//                that lanes without a pair read (values of samples >= N and
//                of every k >= n are zero, so they contribute exact zeros);
//                tP [NPT][2] times
//   common:      brow [6][NC] (P, Pd, Pdd at t = 0 and t = T); lin [NC]; Q,
//                K11 (x hi, x lo, y hi, y lo), K11_psi [NC][KS] (KS =
//                k_stride(NC) floats per row with the padding); then the
//                blocks used only by the first step (from `init`): K12_psi
//                [NC][4]; K12_x, K12_y, C0_x, C0_y [NC][8]; C0_psi [NC][4]
// The pair kernel stages [pair rows | common up to init] and reads the
// first-step blocks from global memory.
//   sample rows: P, Pd, Pdd [NST][NC]; t [NST], NST = N rounded up to whole
//                warps (zero rows beyond N)
// ---------------------------------------------------------------------------
struct BlobLayout {
    int PP, PdP, PddP, tP;                                                        // pair rows
    int PPl, PdPl, PddPl;  // lo parts of the pair rows (split precision modes; else = the hi rows)
    int brow, lin, Q, Kxh, Kxl, Kyh, Kyl, Kp11, Kp12, K12x, K12y, C0x, C0y, C0p;  // common
    int P, Pd, Pdd, t;                                                            // sample rows
    int common, init, rows1, total;  // region starts (common, first-step blocks, sample rows) and end
};

// Floats per row of the per-thread (or per-lane) matrices in shared memory.
// A warp's 128-bit loads are served 8 threads at a time and are conflict-free
// when the row stride is an odd multiple of 16 B.  Sample-pair rows: 2 NC + 4
// floats (112 B for NC = 12, 144 B for 16; unpadded, 96 B gave a 2-way and
// 128 B an 8-way conflict).  Rows of Q and K11 (one per lane): NC floats for
// NC = 12 (48 B), 20 for NC = 16 (80 B instead of 64 B).
__host__ __device__ constexpr int pair_stride(int NC) { return 2 * NC + 4; }
__host__ __device__ constexpr int k_stride(int NC) { return NC == 16 ? 20 : NC; }

static BlobLayout blob_layout(int N, int NC, bool split = false)
{
    auto up4 = [](int v) { return (v + 3) & ~3; };
    // pair rows: the ceil(N/2) pairs, then one zero row that every lane
    // beyond them reads; sample rows 32 ceil(N/32) samples, one per thread of
    // the launch, zero beyond N
    const int NP = (N + 1) / 2 + 1;
    const int NS = 32 * ((N + 31) / 32);
    BlobLayout B{};
    int o = 0;
    B.PP = o; o += NP * pair_stride(NC);
    B.PdP = o; o += NP * pair_stride(NC);
    B.PddP = o; o += NP * pair_stride(NC);
    if (split) {
        B.PPl = o; o += NP * pair_stride(NC);
        B.PdPl = o; o += NP * pair_stride(NC);
        B.PddPl = o; o += NP * pair_stride(NC);
    } else {
        B.PPl = B.PP; B.PdPl = B.PdP; B.PddPl = B.PddP;
    }
    B.tP = o; o += up4(NP * 2);
    B.common = o;
    B.brow = o; o += 6 * NC;
    B.lin = o; o += up4(NC);
    B.Q = o; o += NC * k_stride(NC);
    B.Kxh = o; o += NC * k_stride(NC);
    B.Kxl = o; o += NC * k_stride(NC);
    B.Kyh = o; o += NC * k_stride(NC);
    B.Kyl = o; o += NC * k_stride(NC);
    B.Kp11 = o; o += NC * k_stride(NC);
    B.init = o;
    B.Kp12 = o; o += NC * 4;
    B.K12x = o; o += NC * 8;
    B.K12y = o; o += NC * 8;
    B.C0x = o; o += NC * 8;
    B.C0y = o; o += NC * 8;
    B.C0p = o; o += NC * 4;
    o = up4(o);
    B.rows1 = o;
    B.P = o; o += NS * NC;
    B.Pd = o; o += NS * NC;
    B.Pdd = o; o += NS * NC;
    B.t = o; o += NS;
    B.total = o;
    return B;
}

struct SolveArgs {
    int N, n, m, B, iters, check_every, cull;
    float rho, a, b, inv_a, inv_b, v_min, v_max, a_max, tol, stall_tol, stall_ratio;
    BlobLayout L;
    const float* blob;
    const float* ego;
    const float* obst;
    const float* goals;
    const float* warm_c;
    const float* warm_l;
    float* coef_out;
    float* lam_out;
    float* resid_out;
    int* iters_out;
    unsigned* err_flag;
    unsigned long long* work;  // evaluated obstacle-sample pairs (summed over CTAs)
    int missing_tx;            // 0; 16 under the failure-path test hook (mmpc_debug_expire_wait)
};

struct ScoreArgs {
    int N, n, B, kind;
    float w1, w2, v_ref, y_ref, psi_max;
    BlobLayout L;
    const float* blob;
    const float* coef;
    float* cost_out;
    int* argmin_out;
    unsigned long long* best;  // packed (cost bits << 32 | index), reset to ~0 after each call
    unsigned* ticket;          // CTA completion counter, reset to 0 after each call
};

constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned ERR_TMA_TIMEOUT = 1u;

// ---------------------------------------------------------------------------
// Warp reduce-scatter.  C values per lane; after the call lane L holds in
// v[0 .. rs_count(C)) the warp sums of the value indices rs_base(C, L) + i.
// Halving steps exchange half of the values; odd counts fall back to a
// butterfly over the remaining ones.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int rs_count(int c)
{
    for (int off = 16; off > 0; off >>= 1)
        if (c % 2 == 0) c /= 2;
    return c;
}
__device__ __forceinline__ int rs_base(int c, int lane)
{
    int base = 0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        if (c % 2 == 0) {
            c /= 2;
            if (lane & off) base += c;
        }
    return base;
}
__device__ __forceinline__ bool rs_writer(int c, int lane)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        if (c % 2 == 0) c /= 2;
        else if (lane & off) return false;
    }
    return true;
}

template <int C, int OFF, int VM>
__device__ __forceinline__ void warp_rs(float (&v)[VM], int lane)
{
    if constexpr (OFF > 0) {
        if constexpr (C % 2 == 0) {
            constexpr int H = C / 2;
            const bool up = (lane & OFF) != 0;
#pragma unroll
            for (int i = 0; i < H; ++i) {
                float send = up ? v[i] : v[i + H];
                float keep = up ? v[i + H] : v[i];
                v[i] = keep + __shfl_xor_sync(FULL, send, OFF);
            }
            warp_rs<H, OFF / 2, VM>(v, lane);
        } else {
#pragma unroll
            for (int i = 0; i < C; ++i) v[i] += __shfl_xor_sync(FULL, v[i], OFF);
            warp_rs<C, OFF / 2, VM>(v, lane);
        }
    }
}

// Reduce-scatter the C values of every warp and store the per-warp sums at
// red[warp * stride + index].
// dst = this lane's store address for C values (see rs_dst), or nullptr for
// lanes that hold duplicates.
template <int C>
__device__ __forceinline__ void reduce_store(float (&v)[C], float* dst, int lane)
{
    warp_rs<C, 16, C>(v, lane);
    constexpr int K = rs_count(C);
    if (dst) {
#pragma unroll
        for (int i = 0; i < K; ++i) dst[i] = v[i];
    }
}

// Where this lane stores its share of a reduce-scatter of C values into
// red[warp * stride + index]; nullptr if it holds a duplicate.
__device__ __forceinline__ float* rs_dst(int c, float* red, int warp, int stride, int lane)
{
    return rs_writer(c, lane) ? red + warp * stride + rs_base(c, lane) : nullptr;
}

// ---------------------------------------------------------------------------
// TMA bulk copy of the constant blob with a bounded mbarrier wait.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long WAIT_LIMIT_NS = 200000000ull;  // 0.2 s per pass of a bounded wait
constexpr int WAIT_MAX_POLLS = 1 << 24;                     // backstop should the timer stall

// `missing`: bytes the barrier expects beyond the copy (0; a test of the
// failure path sets 16 so that the wait runs out).
__device__ __forceinline__ bool stage_blob(float* dst, const float* src, int bytes, unsigned long long* mbar,
                                           unsigned* err_flag, int missing)
{
    const uint32_t bar = smem_u32(mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes + missing)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(dst)),
            "l"(src), "r"(bytes), "r"(bar)
            : "memory");
    }
    // Bounded wait: a copy that has not landed after 0.2 s (device global
    // timer; a poll count as a backstop) flags an error, and the CTA waits
    // once more, again bounded, before it gives up, so that it never leaves
    // with the copy in flight unless the second bound also expires.
    uint32_t done = 0;
    for (int pass = 0; pass < 2 && !done; ++pass) {
        const unsigned long long t0 = global_ns();
        for (int it = 0; it < WAIT_MAX_POLLS && !done; ++it) {
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(bar), "r"(0)
                : "memory");
            if (!done && (it & 63) == 63 && global_ns() - t0 > WAIT_LIMIT_NS) break;
        }
        if (!done && pass == 0 && threadIdx.x == 0) atomicOr(err_flag, ERR_TMA_TIMEOUT);
    }
    const bool ok = __syncthreads_and(done) != 0;
    // every thread has seen the phase complete: retire the barrier so that a
    // CTA that stages again (one item after another) initialises a fresh one
    if (ok && threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
    return ok;
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float2 lo2(float4 v) { return f2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return f2(v.z, v.w); }
__device__ __forceinline__ float2 hsum2(float2 a, float2 b) { return f2(a.x + a.y, b.x + b.y); }

// Error-free sum of two floats (Knuth's TwoSum): a + b = s + e exactly.
// Intrinsics, so that no contraction or reassociation can change the steps.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// Compensated dot product of NC floats (algorithm Dot2 of Ogita, Rump and
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005): the
// rounding error of each product (by FMA) and of each sum (by TwoSum) is
// carried and added at the end, so the result is as accurate as a dot
// product in twice the working precision, rounded once; four interleaved
// partial sums for ILP, themselves added by TwoSum.  Used for K11 u, where
// the terms (K11 entries of ~1e3 with alternating signs times multipliers of
// up to ~1e3) cancel by five orders of magnitude: the plain FP32 sum of such
// terms loses ~1e-2 of the increment per iteration.
// The columns j < J0 are skipped: for K11 the first three (the coefficients
// fixed by the initial position, speed and acceleration) are zero.
template <int NC, int J0 = 0>
__device__ __forceinline__ float dot2(const float* __restrict__ row, const float* __restrict__ v)
{
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = J0 & ~3; j < NC; j += 4) {
        const float4 r4 = *reinterpret_cast<const float4*>(row + j), w4 = *reinterpret_cast<const float4*>(v + j);
        const float rr[4] = {r4.x, r4.y, r4.z, r4.w}, ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (j + q < J0) continue;
            const float pq = __fmul_rn(rr[q], ww[q]);
            const float pe = __fmaf_rn(rr[q], ww[q], -pq);
            float t;
            two_sum(s[q], pq, s[q], t);
            c[q] = __fadd_rn(c[q], __fadd_rn(pe, t));
        }
    }
    float S = s[0], E = __fadd_rn(__fadd_rn(c[0], c[1]), __fadd_rn(c[2], c[3]));
#pragma unroll
    for (int q = 1; q < 4; ++q) {
        float t;
        two_sum(S, s[q], S, t);
        E = __fadd_rn(E, t);
    }
    return __fadd_rn(S, E);
}

// Basis evaluations at a sample pair.  A pair row holds, for each coefficient
// pair (2j, 2j + 1), the 16-byte block (P[s0][2j], P[s0][2j+1], P[s1][2j],
// P[s1][2j+1]) of its two samples s0 = 2i, s1 = 2i + 1; coefficient vectors
// are plain [NC] arrays, so one 16-byte load covers two blocks.  Each
// sample's value runs through one FFMA2 chain over the coefficient pairs
// (even coefficients in the low half, odd in the high half) and the halves
// are added at the end.  The five evaluations of the projection phase share
// every load: x = P cx, y = P cy, xdd = Pdd cx, ydd = Pdd cy, psi = P cpsi.
template <int NC>
__device__ __forceinline__ void eval_pair5(const float* __restrict__ P, const float* __restrict__ Pdd,
                                           const float* __restrict__ cx, const float* __restrict__ cy,
                                           const float* __restrict__ cp, float2& x, float2& y, float2& xdd,
                                           float2& ydd, float2& ps)
{
    static_assert(NC % 4 == 0, "coefficient vectors are read 16 bytes at a time");
    const float2 z = f2(0.f);
    float2 x0 = z, x1 = z, y0 = z, y1 = z, p0 = z, p1 = z, xa0 = z, xa1 = z, ya0 = z, ya1 = z;
#pragma unroll
    for (int k = 0; k < NC; k += 4) {
        const float4 a = ld4(cx + k), b = ld4(cy + k), c = ld4(cp + k);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 r = ld4(P + 2 * k + 4 * h), d = ld4(Pdd + 2 * k + 4 * h);
            const float2 av = h ? hi2(a) : lo2(a), bv = h ? hi2(b) : lo2(b), cv = h ? hi2(c) : lo2(c);
            x0 = __ffma2_rn(lo2(r), av, x0);
            x1 = __ffma2_rn(hi2(r), av, x1);
            y0 = __ffma2_rn(lo2(r), bv, y0);
            y1 = __ffma2_rn(hi2(r), bv, y1);
            p0 = __ffma2_rn(lo2(r), cv, p0);
            p1 = __ffma2_rn(hi2(r), cv, p1);
            xa0 = __ffma2_rn(lo2(d), av, xa0);
            xa1 = __ffma2_rn(hi2(d), av, xa1);
            ya0 = __ffma2_rn(lo2(d), bv, ya0);
            ya1 = __ffma2_rn(hi2(d), bv, ya1);
        }
    }
    x = hsum2(x0, x1);
    y = hsum2(y0, y1);
    ps = hsum2(p0, p1);
    xdd = hsum2(xa0, xa1);
    ydd = hsum2(ya0, ya1);
}

// The heading phase's two evaluations, xd = Pd cx and yd = Pd cy, sharing the
// row loads.
template <int NC>
__device__ __forceinline__ void eval_pair2(const float* __restrict__ Pd, const float* __restrict__ cx,
                                           const float* __restrict__ cy, float2& xd, float2& yd)
{
    const float2 z = f2(0.f);
    float2 x0 = z, x1 = z, y0 = z, y1 = z;
#pragma unroll
    for (int k = 0; k < NC; k += 4) {
        const float4 a = ld4(cx + k), b = ld4(cy + k);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 r = ld4(Pd + 2 * k + 4 * h);
            const float2 av = h ? hi2(a) : lo2(a), bv = h ? hi2(b) : lo2(b);
            x0 = __ffma2_rn(lo2(r), av, x0);
            x1 = __ffma2_rn(hi2(r), av, x1);
            y0 = __ffma2_rn(lo2(r), bv, y0);
            y1 = __ffma2_rn(hi2(r), bv, y1);
        }
    }
    xd = hsum2(x0, x1);
    yd = hsum2(y0, y1);
}

// ---------------------------------------------------------------------------
// Precision modes (mmpc_params.precision): the operands of the basis products
// rounded as the tensor cores take them, FP32 products and accumulation.  The
// same integer rounding on the host (staged basis rows) and in the kernels
// (coefficients, per-sample targets, theta): TF32 keeps 10 significand bits,
// to nearest with ties away from zero; BF16 keeps 7, ties to even; non-finite
// values pass unchanged.  Split modes carry hi = rnd(a), lo = rnd(a - hi) and
// form a b as a_hi b_hi + a_hi b_lo + a_lo b_hi.
// ---------------------------------------------------------------------------
__host__ __device__ inline float round_operand(float x, int prec)
{
    if (prec == MMPC_PREC_FP32) return x;
    unsigned u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) {
        if (prec == MMPC_PREC_TF32 || prec == MMPC_PREC_TF32_SPLIT) u = (u + 0x1000u) & 0xffffe000u;
        else u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
    }
    memcpy(&x, &u, 4);
    return x;
}

__host__ __device__ constexpr bool prec_split(int prec)
{
    return prec == MMPC_PREC_TF32_SPLIT || prec == MMPC_PREC_BF16_SPLIT;
}

template <int PREC>
__device__ __forceinline__ float2 rnd2(float2 a)
{
    return f2(round_operand(a.x, PREC), round_operand(a.y, PREC));
}

// acc + a b with a = (ah, al) and b = (bh, bl) as the mode takes them
template <int PREC>
__device__ __forceinline__ float2 pfma(float2 ah, float2 al, float2 bh, float2 bl, float2 acc)
{
    acc = __ffma2_rn(ah, bh, acc);
    if constexpr (prec_split(PREC)) {
        acc = __ffma2_rn(ah, bl, acc);
        acc = __ffma2_rn(al, bh, acc);
    }
    return acc;
}

// hi and lo parts of a pair of values as the mode takes them
template <int PREC>
__device__ __forceinline__ void split2(float2 v, float2& h, float2& l)
{
    h = rnd2<PREC>(v);
    l = rnd2<PREC>(__fadd2_rn(v, f2(-h.x, -h.y)));
}

// eval_pair5 / eval_pair2 in a precision mode: rows (hi, and lo rows in the
// split modes) staged rounded by the host, coefficients rounded here.
template <int NC, int PREC>
__device__ __forceinline__ void eval_pair5_prec(const float* __restrict__ P, const float* __restrict__ Pdd,
                                                const float* __restrict__ Pl, const float* __restrict__ Pddl,
                                                const float* __restrict__ cx, const float* __restrict__ cy,
                                                const float* __restrict__ cp, float2& x, float2& y, float2& xdd,
                                                float2& ydd, float2& ps)
{
    const float2 z = f2(0.f);
    float2 x0 = z, x1 = z, y0 = z, y1 = z, p0 = z, p1 = z, xa0 = z, xa1 = z, ya0 = z, ya1 = z;
#pragma unroll
    for (int k = 0; k < NC; k += 4) {
        const float4 a = ld4(cx + k), b = ld4(cy + k), c = ld4(cp + k);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 r = ld4(P + 2 * k + 4 * h), d = ld4(Pdd + 2 * k + 4 * h);
            const float4 rl = ld4(Pl + 2 * k + 4 * h), dl = ld4(Pddl + 2 * k + 4 * h);
            float2 ah, al, bh, bl, ch, cl;
            split2<PREC>(h ? hi2(a) : lo2(a), ah, al);
            split2<PREC>(h ? hi2(b) : lo2(b), bh, bl);
            split2<PREC>(h ? hi2(c) : lo2(c), ch, cl);
            x0 = pfma<PREC>(lo2(r), lo2(rl), ah, al, x0);
            x1 = pfma<PREC>(hi2(r), hi2(rl), ah, al, x1);
            y0 = pfma<PREC>(lo2(r), lo2(rl), bh, bl, y0);
            y1 = pfma<PREC>(hi2(r), hi2(rl), bh, bl, y1);
            p0 = pfma<PREC>(lo2(r), lo2(rl), ch, cl, p0);
            p1 = pfma<PREC>(hi2(r), hi2(rl), ch, cl, p1);
            xa0 = pfma<PREC>(lo2(d), lo2(dl), ah, al, xa0);
            xa1 = pfma<PREC>(hi2(d), hi2(dl), ah, al, xa1);
            ya0 = pfma<PREC>(lo2(d), lo2(dl), bh, bl, ya0);
            ya1 = pfma<PREC>(hi2(d), hi2(dl), bh, bl, ya1);
        }
    }
    x = hsum2(x0, x1);
    y = hsum2(y0, y1);
    ps = hsum2(p0, p1);
    xdd = hsum2(xa0, xa1);
    ydd = hsum2(ya0, ya1);
}

template <int NC, int PREC>
__device__ __forceinline__ void eval_pair2_prec(const float* __restrict__ Pd, const float* __restrict__ Pdl,
                                                const float* __restrict__ cx, const float* __restrict__ cy,
                                                float2& xd, float2& yd)
{
    const float2 z = f2(0.f);
    float2 x0 = z, x1 = z, y0 = z, y1 = z;
#pragma unroll
    for (int k = 0; k < NC; k += 4) {
        const float4 a = ld4(cx + k), b = ld4(cy + k);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 r = ld4(Pd + 2 * k + 4 * h), rl = ld4(Pdl + 2 * k + 4 * h);
            float2 ah, al, bh, bl;
            split2<PREC>(h ? hi2(a) : lo2(a), ah, al);
            split2<PREC>(h ? hi2(b) : lo2(b), bh, bl);
            x0 = pfma<PREC>(lo2(r), lo2(rl), ah, al, x0);
            x1 = pfma<PREC>(hi2(r), hi2(rl), ah, al, x1);
            y0 = pfma<PREC>(lo2(r), lo2(rl), bh, bl, y0);
            y1 = pfma<PREC>(hi2(r), hi2(rl), bh, bl, y1);
        }
    }
    xd = hsum2(x0, x1);
    yd = hsum2(y0, y1);
}

// Sum over obstacles at the sample pair (Eq. split_alpha_o).  With n = w / (a,
// b) the ellipse-normalised offset of obstacle j and s = max(0, 1/|n| - 1),
// S += n s; the rows of F_o c - g_o at a sample sum to (-a Sx, -b Sy).  With
// RESID the squared row residuals sum_j |(a nx s, b ny s)|^2 are accumulated
// too.  obs holds per obstacle (-x0/a, -x0/a, -vx/a, -vx/a) and (-y0/b, -y0/b,
// -vy/b, -vy/b) in the frame moving with v0, so n = N + fma(-v, t, -x0) is
// two packed instructions per coordinate for both samples.
template <bool RESID, bool LIST>
__device__ __forceinline__ void obstacle_sum2(const float4* __restrict__ obs, const int* __restrict__ list, int m,
                                              float2 Xn, float2 Yn, float2 tt, float a2, float b2, float2& Sx,
                                              float2& Sy, float2& R2)
{
    // The per-obstacle terms are independent; they are accumulated in
    // obstacle order through one chain, so that skipping obstacles whose term
    // is exactly zero (culling) leaves every sum bit-identical.
    float2 sx = f2(0.f), sy = f2(0.f), r = f2(0.f);
    const float2 m1 = f2(-1.f);
    int j = 0;
#pragma unroll 2
    for (; j + 1 < m; j += 2) {
        const int j0 = LIST ? list[j] : j;
        const int j1 = LIST ? list[j + 1] : j + 1;
        const float4 ax0 = obs[2 * j0], ay0 = obs[2 * j0 + 1];
        const float4 ax1 = obs[2 * j1], ay1 = obs[2 * j1 + 1];
        const float2 nx0 = __fadd2_rn(Xn, __ffma2_rn(f2(ax0.z, ax0.w), tt, f2(ax0.x, ax0.y)));
        const float2 ny0 = __fadd2_rn(Yn, __ffma2_rn(f2(ay0.z, ay0.w), tt, f2(ay0.x, ay0.y)));
        const float2 nx1 = __fadd2_rn(Xn, __ffma2_rn(f2(ax1.z, ax1.w), tt, f2(ax1.x, ax1.y)));
        const float2 ny1 = __fadd2_rn(Yn, __ffma2_rn(f2(ay1.z, ay1.w), tt, f2(ay1.x, ay1.y)));
        const float2 q0 = __ffma2_rn(nx0, nx0, __fmul2_rn(ny0, ny0));
        const float2 q1 = __ffma2_rn(nx1, nx1, __fmul2_rn(ny1, ny1));
        float2 s0 = __fadd2_rn(f2(rsqrtf(q0.x), rsqrtf(q0.y)), m1);
        float2 s1 = __fadd2_rn(f2(rsqrtf(q1.x), rsqrtf(q1.y)), m1);
        s0 = f2(fmaxf(s0.x, 0.f), fmaxf(s0.y, 0.f));
        s1 = f2(fmaxf(s1.x, 0.f), fmaxf(s1.y, 0.f));
        sx = __ffma2_rn(nx1, s1, __ffma2_rn(nx0, s0, sx));
        sy = __ffma2_rn(ny1, s1, __ffma2_rn(ny0, s0, sy));
        if (RESID) {
            const float2 w0 = __ffma2_rn(__fmul2_rn(f2(a2), nx0), nx0, __fmul2_rn(__fmul2_rn(f2(b2), ny0), ny0));
            const float2 w1 = __ffma2_rn(__fmul2_rn(f2(a2), nx1), nx1, __fmul2_rn(__fmul2_rn(f2(b2), ny1), ny1));
            r = __ffma2_rn(__fmul2_rn(s1, s1), w1, __ffma2_rn(__fmul2_rn(s0, s0), w0, r));
        }
    }
    if (j < m) {
        const int j0 = LIST ? list[j] : j;
        const float4 ax0 = obs[2 * j0], ay0 = obs[2 * j0 + 1];
        const float2 nx0 = __fadd2_rn(Xn, __ffma2_rn(f2(ax0.z, ax0.w), tt, f2(ax0.x, ax0.y)));
        const float2 ny0 = __fadd2_rn(Yn, __ffma2_rn(f2(ay0.z, ay0.w), tt, f2(ay0.x, ay0.y)));
        const float2 q0 = __ffma2_rn(nx0, nx0, __fmul2_rn(ny0, ny0));
        float2 s0 = __fadd2_rn(f2(rsqrtf(q0.x), rsqrtf(q0.y)), m1);
        s0 = f2(fmaxf(s0.x, 0.f), fmaxf(s0.y, 0.f));
        sx = __ffma2_rn(nx0, s0, sx);
        sy = __ffma2_rn(ny0, s0, sy);
        if (RESID) {
            const float2 w0 = __ffma2_rn(__fmul2_rn(f2(a2), nx0), nx0, __fmul2_rn(__fmul2_rn(f2(b2), ny0), ny0));
            r = __ffma2_rn(__fmul2_rn(s0, s0), w0, r);
        }
    }
    Sx = sx;
    Sy = sy;
    R2 = r;
}

// The same sum for one sample (h = 0 or 1 of the pair), slowly, with the
// degenerate case of a sample exactly at an obstacle centre (w = 0): there
// alpha = atan2(0, 0) = 0 and d = 1, so the target is xi + (a, 0) and the row
// of F_o c - g_o is (-a, 0).
__device__ __noinline__ void obstacle_sum_exact(const float4* __restrict__ obs, int m, float Xn, float Yn, float tt,
                                                float a2, float b2, float& Sx, float& Sy, float& R2)
{
    Sx = 0.f;
    Sy = 0.f;
    R2 = 0.f;
    for (int j = 0; j < m; ++j) {
        const float4 ax = obs[2 * j], ay = obs[2 * j + 1];
        const float nx = Xn + fmaf(ax.z, tt, ax.x);
        const float ny = Yn + fmaf(ay.z, tt, ay.x);
        const float q = fmaf(nx, nx, ny * ny);
        if (q == 0.f) {
            Sx += 1.f;
            R2 += a2;
        } else {
            const float sj = fmaxf(rsqrtf(q) - 1.f, 0.f);
            Sx = fmaf(nx, sj, Sx);
            Sy = fmaf(ny, sj, Sy);
            R2 = fmaf(sj * sj, fmaf(a2 * nx, nx, b2 * ny * ny), R2);
        }
    }
}

// Exact culling for Eq. split_alpha_o.  The warp's samples span a box
// (ellipse-normalised, moving frame) over the time window [tw_lo, tw_hi]; an
// obstacle moves along a segment over that window.  When the two boxes are
// apart by more than 1 (plus a margin far above the FP32 rounding of the
// coordinates) along x or y, every sample of the warp has |n| > 1 for that
// obstacle, so s = max(1/|n| - 1, 0) = 0 and the obstacle adds exactly
// nothing.  The remaining obstacles' indices go to a warp-private list, in
// increasing order.  A non-finite coordinate keeps every obstacle, so NaN
// propagates as without culling.
__device__ __forceinline__ float warp_min(float v)
{
    float r;
    asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float warp_max(float v)
{
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

// Warp-private culling list with reuse.  The list is built for an
// enlarged box (the warp's sample box grown by LIST_MARGIN) and kept while
// the sample box stays inside it, so the obstacle tests run only when the
// trajectory has moved noticeably.  Every obstacle that is not provably apart
// from the list box is in the list, so a reused list is still exact.
struct CullState {
    float xlo, xhi, ylo, yhi;  // list box (empty at the start)
    int count;
};

constexpr float CULL_MARGIN = 1.001f;  // normalised distance beyond which a term is exactly zero
constexpr float LIST_MARGIN = 0.25f;   // growth of the list box

__device__ __forceinline__ void cull_init(CullState& cs)
{
    const float inf = __int_as_float(0x7f800000);
    cs.xlo = inf; cs.xhi = -inf; cs.ylo = inf; cs.yhi = -inf;
    cs.count = 0;
}

// PAIRED: obstacles stored as two duplicated float4 (pair kernel), else one
// float4 (p_x, p_y, pv_x, pv_y) (one-sample kernel); p and pv are negated.
template <bool PAIRED>
__device__ __forceinline__ int cull_update(CullState& cs, int m, float xlo, float xhi, float ylo, float yhi,
                                           bool any_bad, float tw_lo, float tw_hi, int* list, int lane,
                                           const float4* __restrict__ obs)
{
    const float inf = __int_as_float(0x7f800000);
    if (!any_bad && xlo >= cs.xlo && xhi <= cs.xhi && ylo >= cs.ylo && yhi <= cs.yhi) return cs.count;
    if (any_bad) {  // a non-finite coordinate: keep every obstacle from now on
        cs.xlo = -inf; cs.xhi = inf; cs.ylo = -inf; cs.yhi = inf;
    } else {
        cs.xlo = xlo - LIST_MARGIN; cs.xhi = xhi + LIST_MARGIN;
        cs.ylo = ylo - LIST_MARGIN; cs.yhi = yhi + LIST_MARGIN;
    }
    const unsigned below = (1u << lane) - 1u;
    int count = 0;
    for (int j0 = 0; j0 < m; j0 += 32) {
        const int j = j0 + lane;
        bool keep = false;
        if (j < m) {
            float2 ox, oy;  // (p, pv) along x and y
            if (PAIRED) {
                const float4 a = obs[2 * j], b = obs[2 * j + 1];
                ox = f2(a.x, a.z);
                oy = f2(b.x, b.z);
            } else {
                const float4 a = obs[j];
                ox = f2(a.x, a.z);
                oy = f2(a.y, a.w);
            }
            // the obstacle centre is -(p + pv t) in the stored (negated) form
            const float e1 = -fmaf(ox.y, tw_lo, ox.x), e2 = -fmaf(ox.y, tw_hi, ox.x);
            const float f1 = -fmaf(oy.y, tw_lo, oy.x), g1 = -fmaf(oy.y, tw_hi, oy.x);
            const bool apart = (cs.xlo - fmaxf(e1, e2) >= CULL_MARGIN) || (fminf(e1, e2) - cs.xhi >= CULL_MARGIN) ||
                               (cs.ylo - fmaxf(f1, g1) >= CULL_MARGIN) || (fminf(f1, g1) - cs.yhi >= CULL_MARGIN);
            keep = any_bad || !apart;
        }
        const unsigned bal = __ballot_sync(FULL, keep);
        if (keep) list[count + __popc(bal & below)] = j;
        count += __popc(bal);
    }
    __syncwarp();
    cs.count = count;
    return count;
}

// Whether a sample lies in the list box (always for a lane without that
// sample; never for a NaN coordinate).  When every sample of the warp does,
// the warp's box lies inside the list box and the list is reused exactly as
// cull_update would.
__device__ __forceinline__ bool in_list_box(float x, float y, float valid, const CullState& cs)
{
    return !(valid > 0.f) || (x >= cs.xlo && x <= cs.xhi && y >= cs.ylo && y <= cs.yhi);
}

// The warp's sample box for the pair kernel; returns whether a valid sample
// has a non-finite coordinate.
__device__ __forceinline__ bool box_pair(float2 Xn, float2 Yn, float2 valid, float& xlo, float& xhi, float& ylo,
                                         float& yhi)
{
    const float inf = __int_as_float(0x7f800000);
    float a = inf, b = -inf, c = inf, d = -inf;
    if (valid.x > 0.f) { a = Xn.x; b = Xn.x; c = Yn.x; d = Yn.x; }
    if (valid.y > 0.f) { a = fminf(a, Xn.y); b = fmaxf(b, Xn.y); c = fminf(c, Yn.y); d = fmaxf(d, Yn.y); }
    const bool bad = (valid.x > 0.f && !(isfinite(Xn.x) && isfinite(Yn.x))) ||
                     (valid.y > 0.f && !(isfinite(Xn.y) && isfinite(Yn.y)));
    xlo = warp_min(a);
    xhi = warp_max(b);
    ylo = warp_min(c);
    yhi = warp_max(d);
    return __any_sync(FULL, bad);
}

// atan2 for two samples at once: octant reduction to a = min(|x|, |y|) /
// max(|x|, |y|) in [0, 1], atan(a) = a p(a^2) with the degree-7 polynomial
// fitted by csrc/fit_atan.py (maximum error 1.6e-7 rad in FP32 evaluation),
// then the octant fix-ups atan2 = pi/2 - r (|y| > |x|), pi - r (x < 0, the
// sign bit deciding, so -0 counts as negative as in IEEE atan2) and the sign
// of y.  atan2(0, 0) = 0.
__device__ __forceinline__ float2 atan2_pair(float2 y, float2 x)
{
    const float ax0 = fabsf(x.x), ax1 = fabsf(x.y), ay0 = fabsf(y.x), ay1 = fabsf(y.y);
    const float hi0 = fmaxf(fmaxf(ax0, ay0), 1e-30f), hi1 = fmaxf(fmaxf(ax1, ay1), 1e-30f);
    const float2 a = f2(__fdividef(fminf(ax0, ay0), hi0), __fdividef(fminf(ax1, ay1), hi1));
    const float2 z = __fmul2_rn(a, a);
    float2 p = f2(-4.062573425e-03f);
    p = __ffma2_rn(p, z, f2(2.189946361e-02f));
    p = __ffma2_rn(p, z, f2(-5.597937107e-02f));
    p = __ffma2_rn(p, z, f2(9.648545831e-02f));
    p = __ffma2_rn(p, z, f2(-1.391191483e-01f));
    p = __ffma2_rn(p, z, f2(1.994746774e-01f));
    p = __ffma2_rn(p, z, f2(-3.332997561e-01f));
    p = __ffma2_rn(p, z, f2(9.999994040e-01f));
    float2 r = __fmul2_rn(a, p);
    const float2 c1 = __fadd2_rn(f2(1.5707963268f), f2(-r.x, -r.y));
    r = f2(ay0 > ax0 ? c1.x : r.x, ay1 > ax1 ? c1.y : r.y);
    const float2 c2 = __fadd2_rn(f2(3.1415926536f), f2(-r.x, -r.y));
    r = f2(__float_as_int(x.x) < 0 ? c2.x : r.x, __float_as_int(x.y) < 0 ? c2.y : r.y);
    return f2(copysignf(r.x, y.x), copysignf(r.y, y.y));
}

__device__ __forceinline__ float atan2_own(float y, float x)
{
    return atan2_pair(f2(y, 0.f), f2(x, 1.f)).x;
}

// sin and cos of two headings.  Cody-Waite reduction r = psi - q pi/2 with
// q = rint(psi 2/pi) and pi/2 split into a float32 head and tail (two FMAs),
// then sin r = r + r^3 S(r^2) and cos r = 1 - r^2/2 + r^4 C(r^2) on
// [-pi/4, pi/4] with the polynomials fitted by csrc/fit_sincos.py (maximum
// error 6.6e-8 in float32 evaluation for |psi| <= 20), and the quadrant
// q mod 4 swapping and negating them.  The accuracy matters: the multiplier
// update integrates any bias of the non-holonomic targets v (cos psi,
// sin psi) over the iterations, so an approximation with errors of a few
// 1e-7 drifts the iterate by millimetres within 100 iterations.  Headings of
// magnitude 1e5 or more (never a real heading) take the library sincosf.
__device__ __forceinline__ void sincos_pair(const float2 ps, float2& sn, float2& cs)
{
    const float2 qs = __fmul2_rn(ps, f2(6.366197723675814e-01f));
    const float2 q = f2(rintf(qs.x), rintf(qs.y));
    const float2 nq = f2(-q.x, -q.y);
    float2 r = __ffma2_rn(nq, f2(1.570796371e+00f), ps);
    r = __ffma2_rn(nq, f2(-4.371138829e-08f), r);
    const float2 z = __fmul2_rn(r, r);
    float2 ps_ = __ffma2_rn(f2(-1.949599100e-04f), z, f2(8.331981488e-03f));
    ps_ = __ffma2_rn(ps_, z, f2(-1.666665077e-01f));
    float2 pc = __ffma2_rn(f2(2.443822632e-05f), z, f2(-1.388736535e-03f));
    pc = __ffma2_rn(pc, z, f2(4.166664556e-02f));
    const float2 s = __ffma2_rn(__fmul2_rn(z, r), ps_, r);
    const float2 c = __ffma2_rn(z, __ffma2_rn(z, pc, f2(-0.5f)), f2(1.f));
    const int j0 = (int)q.x, j1 = (int)q.y;
    sn.x = (j0 & 1) ? c.x : s.x;
    sn.y = (j1 & 1) ? c.y : s.y;
    cs.x = (j0 & 1) ? s.x : c.x;
    cs.y = (j1 & 1) ? s.y : c.y;
    if (j0 & 2) sn.x = -sn.x;
    if (j1 & 2) sn.y = -sn.y;
    if ((j0 + 1) & 2) cs.x = -cs.x;
    if ((j1 + 1) & 2) cs.y = -cs.y;
    if (fabsf(ps.x) >= 1e5f) sincosf(ps.x, &sn.x, &cs.x);
    if (fabsf(ps.y) >= 1e5f) sincosf(ps.y, &sn.y, &cs.y);
}

__device__ __forceinline__ void heading_sincos(float ps, float* sn, float* cs)
{
    float2 s, c;
    sincos_pair(f2(ps, 0.f), s, c);
    *sn = s.x;
    *cs = c.x;
}

// ---------------------------------------------------------------------------
// The fused AM kernel.  Grid: one CTA per trajectory; block: 32 ceil(ceil(N/2)
// / 32) threads (at most 8 warps), thread i owns samples 2i and 2i+1.  A warp
// that runs the QP steps holds the whole coefficient state -- lane k (k < NC)
// coefficient k of the x axis and of psi, lane 16 + k coefficient k of the y
// axis.  With 1-2 warps every warp runs the two small QP steps itself from the
// CTA's partial sums: all warps compute bit-identical values, so an iteration
// needs only two CTA barriers (after the partial sums of P^T theta and after
// those of F^T (F c - g)).  With more warps warp 0 alone runs them and the
// others read its coefficient vectors after two more barriers.
// ---------------------------------------------------------------------------
template <int NC>
struct SolveSmem {
    static constexpr int VD = 3 * NC + 4;  // values reduced per thread in the projection phase
    static constexpr int RSD = (VD + 3) & ~3;
    static constexpr int RSB = NC;
};

constexpr int MAX_WARPS = 8;

template <int NC, int MAXT>
struct MinBlocks {
    // NC = 16 with 128 threads (N = 129..256): 3 CTAs per SM and the
    // register budget that allows (no spills); a fourth CTA at 128 registers
    // spills and was slower (11.0 against 10.4 ms at N = 200).  NC = 12 with
    // 64 threads: a bound of 7 (the kernel still takes 128 registers, so 8
    // CTAs fit) measured 1.4 % faster than 8 on the 1024-goal scene.
    static constexpr int value = MAXT <= 64 ? (NC == 12 ? 7 : 8) : (MAXT <= 128 ? (NC == 16 ? 3 : 4) : 2);
};

// dot product of two 16-byte aligned vectors of NC floats; four partial
// sums for ILP.
template <int NC>
__device__ __forceinline__ float dot_vec(const float* __restrict__ row, const float* __restrict__ v)
{
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < NC; j += 4) {
        const float4 r = ld4(row + j), w = ld4(v + j);
        acc[0] = fmaf(r.x, w.x, acc[0]);
        acc[1] = fmaf(r.y, w.y, acc[1]);
        acc[2] = fmaf(r.z, w.z, acc[2]);
        acc[3] = fmaf(r.w, w.w, acc[3]);
    }
    return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// The pair kernel's work for trajectory l of the problem A, by the whole CTA.
// Warps beyond ceil(ceil(N/2) / 32) (a CTA sized for a longer horizon, in a
// batch of scenes) hold no samples: they only follow the coefficient state
// through the barriers.
template <int NC, int MAXT, int PREC = MMPC_PREC_FP32>
__device__ __forceinline__ bool pair_body(const SolveArgs& A, const int l)
{
    constexpr int VD = SolveSmem<NC>::VD;
    constexpr int RSD = SolveSmem<NC>::RSD;
    constexpr int RSB = SolveSmem<NC>::RSB;
    constexpr int WARPS = MAXT / 32;
    extern __shared__ __align__(16) float smem[];
    // per-warp copies of the coefficient vectors
    __shared__ __align__(16) float s_cx[WARPS][NC];
    __shared__ __align__(16) float s_cy[WARPS][NC];
    __shared__ __align__(16) float s_cp[WARPS][NC];
    __shared__ __align__(16) float s_vec[WARPS][2][NC];  // per-warp scratch vectors (x, y)
    __shared__ __align__(8) unsigned long long s_mbar;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int N = A.N, m = A.m;
    const int NP = (N + 1) >> 1;
    const int nwarps = (NP + 31) >> 5;  // warps that hold samples
    const bool idle = warp >= nwarps;
    const BlobLayout& L = A.L;

    float* blob = smem;
    float4* obs = reinterpret_cast<float4*>(smem + L.init);
    float* red1 = reinterpret_cast<float*>(obs + 2 * m);   // [warp][RSB]: P^T theta
    float* red2 = red1 + WARPS * RSB;                       // [warp][RSD]: F^T (F c - g), ...
    int* olist = reinterpret_cast<int*>(red2 + WARPS * RSD) + warp * m;  // this warp's active obstacles
    // SOLO (CTAs of more than 2 warps): warp 0 alone runs the QP steps and
    // every warp reads its coefficient vectors after a CTA barrier (two more
    // barriers per iteration, the other warps' issue slots freed); with 1-2
    // warps every warp runs them on its own copy (two barriers per iteration)
    constexpr bool SOLO = MAXT > 64;
    float* cxv = s_cx[SOLO ? 0 : warp];
    float* cyv = s_cy[SOLO ? 0 : warp];
    float* cpv = s_cp[SOLO ? 0 : warp];

    // Scene: ego (Sec. III, x0 = 0) and obstacles, normalised by the ellipse
    // axes, negated, duplicated for the sample pair, in the frame moving with v0.
    const float y0 = __ldg(A.ego + 0), v0 = __ldg(A.ego + 1), psi0 = __ldg(A.ego + 2), acc0 = __ldg(A.ego + 3);
    for (int j = tid; j < m; j += blockDim.x) {
        const float* o = A.obst + 4 * j;
        const float px = -__ldg(o + 0) * A.inv_a, pvx = -(__ldg(o + 2) - v0) * A.inv_a;
        const float py = -__ldg(o + 1) * A.inv_b, pvy = -__ldg(o + 3) * A.inv_b;
        obs[2 * j] = make_float4(px, px, pvx, pvx);
        obs[2 * j + 1] = make_float4(py, py, pvy, pvy);
    }
    if (!stage_blob(blob, A.blob, L.init * 4, &s_mbar, A.err_flag, A.missing_tx)) return false;
    const float* __restrict__ gblob = A.blob;  // first-step blocks: read once, from global memory

    const float rho = A.rho;
    const float a2 = A.a * A.a, b2 = A.b * A.b;
    const int ip = (idle || tid >= NP) ? NP : tid;  // lanes beyond the pairs read the zero row NP
    constexpr int RS = pair_stride(NC);
    const float* PP = blob + L.PP + ip * RS;
    const float* PdP = blob + L.PdP + ip * RS;
    const float* PddP = blob + L.PddP + ip * RS;
    const float* PPl = blob + L.PPl + ip * RS;  // lo parts (split precision modes)
    const float* PdPl = blob + L.PdPl + ip * RS;
    const float* PddPl = blob + L.PddPl + ip * RS;
    const float2 tt = f2(blob[L.tP + 2 * ip], blob[L.tP + 2 * ip + 1]);
    const bool has_pair = !idle && tid < NP;
    const float2 valid = f2(has_pair ? 1.f : 0.f, (has_pair && 2 * ip + 1 < N) ? 1.f : 0.f);
    // the warp's samples [64 warp, 64 warp + 64) and their time window
    const int w_first = idle ? 0 : 64 * warp;
    const int w_last = idle ? 0 : min(N, 64 * warp + 64) - 1;
    const float tw_lo = blob[L.tP + w_first], tw_hi = blob[L.tP + w_last];
    unsigned long long work = 0;  // evaluated obstacle-sample pairs (lane 0)
    CullState cull;
    cull_init(cull);
    if (!A.cull && !idle) {  // one code path for the obstacle sum: the identity list
        for (int j = lane; j < m; j += 32) olist[j] = j;
        __syncwarp();
    }

    // ---- coefficient state, identical in every warp ---------------------------
    const bool isy = lane >= 16;
    const int k = lane & 15;
    const bool act = k < NC;
    const int kk = act ? k : 0;
    float c = 0.f, e = 0.f, lam = 0.f, lampsi = 0.f, cbp = 0.f, corr = 0.f;
    float* own = isy ? cyv : cxv;
    float* vec = s_vec[warp][isy ? 1 : 0];
    {
        const float* g = A.goals + 3 * l;
        const float yg = __ldg(g + 0), vg = __ldg(g + 1), ag = __ldg(g + 2);
        float cpsi, spsi;
        sincosf(psi0, &spsi, &cpsi);
        // boundary values (see mmpc.h), x relative to v0 t
        const float bx[6] = {0.f, v0 * cpsi - v0, acc0 * cpsi, vg - v0, ag, 0.f};
        const float by[6] = {y0, v0 * spsi, acc0 * spsi, yg, 0.f, 0.f};
        const float bp[4] = {psi0, 0.f, 0.f, 0.f};
        const int nb = isy ? 6 : 5;
        if (A.warm_c) {
            c = act && k < A.n ? __ldg(A.warm_c + (size_t)l * 3 * A.n + (isy ? A.n : 0) + k) : 0.f;
            if (!isy && act && k < A.n) c -= v0 * blob[L.lin + k];
        } else {
            const float* C0 = gblob + (isy ? L.C0y : L.C0x) + kk * 8;
            float sacc = 0.f;
#pragma unroll
            for (int r = 0; r < 6; ++r)
                if (r < nb) sacc = fmaf(C0[r], isy ? by[r] : bx[r], sacc);
            c = act ? sacc : 0.f;
        }
        // K12 (b - A c^0): zero for an exact cold start.  Eq. lin_solve_xy_2
        // from any c^0 equals c^0 + K12 (b - A c^0) + K11 u^0 with u^0 taken at
        // c^0 itself, so this term is added by the first step (the
        // auxiliaries of iterate 0 are those of the start as given).
        {
            // boundary rows: x uses (P0, Pd0, Pdd0, PdT, PddT), y (P0, Pd0, Pdd0, PT, PdT, PddT)
            const int rx[6] = {0, 1, 2, 4, 5, 5};
            const float* K12 = gblob + (isy ? L.K12y : L.K12x) + kk * 8;
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                const int row = isy ? r : rx[r];
                float ac = act ? blob[L.brow + row * NC + kk] * c : 0.f;  // A_r c over the 16 lanes of the axis group
                ac += __shfl_xor_sync(FULL, ac, 8);
                ac += __shfl_xor_sync(FULL, ac, 4);
                ac += __shfl_xor_sync(FULL, ac, 2);
                ac += __shfl_xor_sync(FULL, ac, 1);
                if (r < nb) corr = fmaf(K12[r], (isy ? by[r] : bx[r]) - ac, corr);
            }
            if (!act) corr = 0.f;
        }
        {
            const float* Kp12 = gblob + L.Kp12 + kk * 4;
            float sacc = 0.f;
#pragma unroll
            for (int r = 0; r < 4; ++r) sacc = fmaf(Kp12[r], bp[r], sacc);
            cbp = (act && !isy) ? sacc : 0.f;
        }
        float cp0 = 0.f;
        if (!isy && act) {
            if (A.warm_c) {
                cp0 = k < A.n ? __ldg(A.warm_c + (size_t)l * 3 * A.n + 2 * A.n + k) : 0.f;
            } else {
                const float* C0 = gblob + L.C0p + kk * 4;
#pragma unroll
                for (int r = 0; r < 4; ++r) cp0 = fmaf(C0[r], bp[r], cp0);
            }
        }
        if (A.warm_l && act && k < A.n) {
            lam = __ldg(A.warm_l + (size_t)l * 3 * A.n + (isy ? A.n : 0) + k);
            if (!isy) lampsi = __ldg(A.warm_l + (size_t)l * 3 * A.n + 2 * A.n + k);
        }
        if ((!SOLO || warp == 0) && act) {
            own[k] = c;
            if (!isy) cpv[k] = cp0;
        }
    }
    if constexpr (SOLO) __syncthreads();
    else __syncwarp();

    float2 xd = f2(0.f), yd = f2(0.f), theta = f2(0.f);
    float rsum[4] = {0.f, 0.f, 0.f, 0.f};
    float rh1 = INFINITY, rh2 = INFINITY;  // convergence residuals of the last two checks
    float* const dstB = rs_dst(RSB, red1, warp, RSB, lane);  // this lane's reduce-scatter outputs
    float* const dstD = rs_dst(VD, red2, warp, RSD, lane);
    int kit = 0;
    const int iters = A.iters;

    // Projection phase: Eqs. split_v, split_alpha_o, split_alpha_a at the
    // current coefficients, then the per-warp partial sums of F^T (F c - g),
    // P^T (P c_psi - theta) and the squared residuals.
    auto project = [&](bool resid) {
        float v[VD];
#pragma unroll
        for (int i = 0; i < VD; ++i) v[i] = 0.f;
        {  // lanes without a sample pair read zero rows: their terms vanish
            float2 x, y, xdd, ydd, ps;
            if constexpr (PREC != MMPC_PREC_FP32)
                eval_pair5_prec<NC, PREC>(PP, PddP, PPl, PddPl, cxv, cyv, cpv, x, y, xdd, ydd, ps);
            else
                eval_pair5<NC>(PP, PddP, cxv, cyv, cpv, x, y, xdd, ydd, ps);
            // Eq. v_update and the non-holonomic rows v (cos psi, sin psi)
            const float2 sp2 = __ffma2_rn(xd, xd, __fmul2_rn(yd, yd));
            const float2 nvel = f2(-fminf(fmaxf(sqrtf(sp2.x), A.v_min), A.v_max),
                                   -fminf(fmaxf(sqrtf(sp2.y), A.v_min), A.v_max));
            float2 sn, cs;
            sincos_pair(ps, sn, cs);
            const float2 evx = __ffma2_rn(nvel, cs, xd);
            const float2 evy = __ffma2_rn(nvel, sn, yd);
            // Eq. split_alpha_a: projection of (xddot, yddot) on the disk of radius a_max
            const float2 an2 = __ffma2_rn(xdd, xdd, __fmul2_rn(ydd, ydd));
            const float2 fr = f2(1.f - fminf(1.f, A.a_max * rsqrtf(an2.x)), 1.f - fminf(1.f, A.a_max * rsqrtf(an2.y)));
            const float2 eax = __fmul2_rn(xdd, fr);
            const float2 eay = __fmul2_rn(ydd, fr);
            // Eq. split_alpha_o, summed over the obstacles
            const float2 Xn = __fmul2_rn(x, f2(A.inv_a)), Yn = __fmul2_rn(y, f2(A.inv_b));
            float2 Sx, Sy, R2;
            int cnt = m;  // without culling the list holds every obstacle in order
            if (A.cull) {
                // the list stays valid while every sample is inside its box (a
                // vote); otherwise the warp's box is formed and the list rebuilt
                if (__all_sync(FULL, in_list_box(Xn.x, Yn.x, valid.x, cull) && in_list_box(Xn.y, Yn.y, valid.y, cull))) {
                    cnt = cull.count;
                } else {
                    float bxlo, bxhi, bylo, byhi;
                    const bool bad = box_pair(Xn, Yn, valid, bxlo, bxhi, bylo, byhi);
                    cnt = cull_update<true>(cull, m, bxlo, bxhi, bylo, byhi, bad, tw_lo, tw_hi, olist, lane, obs);
                }
            }
            if (lane == 0) work += (unsigned long long)cnt * (unsigned)(w_last - w_first + 1);
            if (resid) obstacle_sum2<true, true>(obs, olist, cnt, Xn, Yn, tt, a2, b2, Sx, Sy, R2);
            else obstacle_sum2<false, true>(obs, olist, cnt, Xn, Yn, tt, a2, b2, Sx, Sy, R2);
            if (isnan(Sx.x) || isnan(Sy.x)) obstacle_sum_exact(obs, m, Xn.x, Yn.x, tt.x, a2, b2, Sx.x, Sy.x, R2.x);
            if (isnan(Sx.y) || isnan(Sy.y)) obstacle_sum_exact(obs, m, Xn.y, Yn.y, tt.y, a2, b2, Sx.y, Sy.y, R2.y);
            const float2 eox = __fmul2_rn(Sx, f2(-A.a));
            const float2 eoy = __fmul2_rn(Sy, f2(-A.b));
            const float2 dpsi = __fadd2_rn(ps, f2(-theta.x, -theta.y));
            // The contractions P^T e over the pair: for each coefficient pair
            // one FFMA2 chain through both samples' rows, the per-sample
            // operands duplicated (e_s, e_s).
            if constexpr (PREC != MMPC_PREC_FP32) {
                // the per-sample operands of the contractions, hi and lo
                float2 eh[7], el[7];
                const float2 ev[7] = {eox, eax, evx, eoy, eay, evy, dpsi};
#pragma unroll
                for (int i = 0; i < 7; ++i) split2<PREC>(ev[i], eh[i], el[i]);
#pragma unroll
                for (int q = 0; q < NC; q += 2) {
                    const float4 p4 = ld4(PP + 2 * q), d4 = ld4(PdP + 2 * q), dd4 = ld4(PddP + 2 * q);
                    const float4 pl4 = ld4(PPl + 2 * q), dl4 = ld4(PdPl + 2 * q), ddl4 = ld4(PddPl + 2 * q);
                    float2 sx = f2(0.f), sy = f2(0.f), sp = f2(0.f);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float2 pr = h ? hi2(p4) : lo2(p4), prl = h ? hi2(pl4) : lo2(pl4);
                        const float2 dr = h ? hi2(d4) : lo2(d4), drl = h ? hi2(dl4) : lo2(dl4);
                        const float2 ddr = h ? hi2(dd4) : lo2(dd4), ddrl = h ? hi2(ddl4) : lo2(ddl4);
                        float2 H[7], Lo[7];
#pragma unroll
                        for (int i = 0; i < 7; ++i) {
                            H[i] = f2(h ? eh[i].y : eh[i].x);
                            Lo[i] = f2(h ? el[i].y : el[i].x);
                        }
                        sx = pfma<PREC>(dr, drl, H[2], Lo[2], sx);
                        sx = pfma<PREC>(ddr, ddrl, H[1], Lo[1], sx);
                        sx = pfma<PREC>(pr, prl, H[0], Lo[0], sx);
                        sy = pfma<PREC>(dr, drl, H[5], Lo[5], sy);
                        sy = pfma<PREC>(ddr, ddrl, H[4], Lo[4], sy);
                        sy = pfma<PREC>(pr, prl, H[3], Lo[3], sy);
                        sp = pfma<PREC>(pr, prl, H[6], Lo[6], sp);
                    }
                    v[q] = sx.x;
                    v[q + 1] = sx.y;
                    v[NC + q] = sy.x;
                    v[NC + q + 1] = sy.y;
                    v[2 * NC + q] = sp.x;
                    v[2 * NC + q + 1] = sp.y;
                }
            } else {
                const float2 ox0 = f2(eox.x), ox1 = f2(eox.y), ax0 = f2(eax.x), ax1 = f2(eax.y);
                const float2 vx0 = f2(evx.x), vx1 = f2(evx.y), oy0 = f2(eoy.x), oy1 = f2(eoy.y);
                const float2 ay0 = f2(eay.x), ay1 = f2(eay.y), vy0 = f2(evy.x), vy1 = f2(evy.y);
                const float2 dp0 = f2(dpsi.x), dp1 = f2(dpsi.y);
#pragma unroll
                for (int q = 0; q < NC; q += 2) {
                    const float4 p4 = ld4(PP + 2 * q), d4 = ld4(PdP + 2 * q), dd4 = ld4(PddP + 2 * q);
                    float2 sx = __fmul2_rn(lo2(d4), vx0);
                    sx = __ffma2_rn(lo2(dd4), ax0, sx);
                    sx = __ffma2_rn(lo2(p4), ox0, sx);
                    sx = __ffma2_rn(hi2(d4), vx1, sx);
                    sx = __ffma2_rn(hi2(dd4), ax1, sx);
                    sx = __ffma2_rn(hi2(p4), ox1, sx);
                    float2 sy = __fmul2_rn(lo2(d4), vy0);
                    sy = __ffma2_rn(lo2(dd4), ay0, sy);
                    sy = __ffma2_rn(lo2(p4), oy0, sy);
                    sy = __ffma2_rn(hi2(d4), vy1, sy);
                    sy = __ffma2_rn(hi2(dd4), ay1, sy);
                    sy = __ffma2_rn(hi2(p4), oy1, sy);
                    const float2 sp = __ffma2_rn(hi2(p4), dp1, __fmul2_rn(lo2(p4), dp0));
                    v[q] = sx.x;
                    v[q + 1] = sx.y;
                    v[NC + q] = sy.x;
                    v[NC + q + 1] = sy.y;
                    v[2 * NC + q] = sp.x;
                    v[2 * NC + q + 1] = sp.y;
                }
            }
            if (resid) {
                const float2 ra = __ffma2_rn(eax, eax, __fmul2_rn(eay, eay));
                const float2 rv = __ffma2_rn(evx, evx, __fmul2_rn(evy, evy));
                const float2 rp = __fmul2_rn(dpsi, dpsi);
                v[3 * NC + 0] = fmaf(R2.x, valid.x, R2.y * valid.y);
                v[3 * NC + 1] = fmaf(ra.x, valid.x, ra.y * valid.y);
                v[3 * NC + 2] = fmaf(rv.x, valid.x, rv.y * valid.y);
                v[3 * NC + 3] = fmaf(rp.x, valid.x, rp.y * valid.y);
            }
        }
        reduce_store<VD>(v, dstD, lane);
    };

    // Velocity directions and the heading target theta = atan2(ydot, xdot)
    // (Eq. split_psi), and the partial sums of P^T theta.
    auto heading = [&](bool reduce) {
        float2 xd0;
        if constexpr (PREC != MMPC_PREC_FP32) eval_pair2_prec<NC, PREC>(PdP, PdPl, cxv, cyv, xd0, yd);
        else eval_pair2<NC>(PdP, cxv, cyv, xd0, yd);
        xd = __fadd2_rn(xd0, f2(v0));
        theta = atan2_pair(yd, xd);
        if (reduce) {
            float v[NC];
            if constexpr (PREC != MMPC_PREC_FP32) {
                float2 th, tl;
                split2<PREC>(theta, th, tl);
                const float2 th0 = f2(th.x), th1 = f2(th.y), tl0 = f2(tl.x), tl1 = f2(tl.y);
#pragma unroll
                for (int q = 0; q < NC; q += 2) {
                    const float4 p4 = ld4(PP + 2 * q), l4 = ld4(PPl + 2 * q);
                    const float2 s = pfma<PREC>(hi2(p4), hi2(l4), th1, tl1, pfma<PREC>(lo2(p4), lo2(l4), th0, tl0, f2(0.f)));
                    v[q] = s.x;
                    v[q + 1] = s.y;
                }
            } else {
                const float2 th0 = f2(theta.x), th1 = f2(theta.y);
#pragma unroll
                for (int q = 0; q < NC; q += 2) {
                    const float4 p4 = ld4(PP + 2 * q);
                    const float2 s = __ffma2_rn(hi2(p4), th1, __fmul2_rn(lo2(p4), th0));
                    v[q] = s.x;
                    v[q + 1] = s.y;
                }
            }
            reduce_store<NC>(v, dstB, lane);
        }
    };

    // Eq. split_psi / lin_solve_psi_2: c_psi = K11_psi (rho P^T theta +
    // lambda_psi) + K12_psi b_psi, in every warp.
    auto psi_step = [&]() {
        float pth = 0.f;
        for (int w = 0; w < nwarps; ++w) pth += red1[w * RSB + kk];
        if (!isy && act) vec[k] = fmaf(rho, pth, lampsi);
        __syncwarp();
        if (!isy && act) cpv[k] = cbp + dot_vec<NC>(blob + L.Kp11 + kk * k_stride(NC), vec);
        __syncwarp();
    };

    // After a projection phase, in every warp: multiplier update (Sec. III-E,
    // "Multiplier Update") unless `first`, the increment u = lambda - Q c -
    // rho F^T (F c - g), the residual check, then step (split_xy) unless done.
    // Returns done.
    auto finish = [&](bool first, bool check) -> bool {
        float ftd = 0.f, pd = 0.f;
        for (int w = 0; w < nwarps; ++w) {
            ftd += red2[w * RSD + (isy ? NC : 0) + kk];
            pd += red2[w * RSD + 2 * NC + kk];
        }
        if (check) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float sacc = 0.f;
                for (int w = 0; w < nwarps; ++w) sacc += red2[w * RSD + 3 * NC + r];
                rsum[r] = sacc;
            }
        }
        if (!first && act) {
            lam = fmaf(-rho, ftd, lam);
            if (!isy) lampsi = fmaf(-rho, pd, lampsi);
        }
        const float qc = dot_vec<NC>(blob + L.Q + kk * k_stride(NC), own);
        const float u = act ? (lam - qc - rho * ftd) : 0.f;
        bool done = kit >= iters;
        if (check && kit % A.check_every == 0 && (A.tol > 0.f || A.stall_tol > 0.f)) {
            const float conv = fmaxf(sqrtf(rsum[0]), fmaxf(sqrtf(rsum[1]), sqrtf(rsum[2])));
            if (!first) {
                if (A.tol > 0.f) done = done || conv <= A.tol;
                // stall stop: far from the target and not closing in over two checks
                if (A.stall_tol > 0.f && kit >= 2 * A.check_every && conv > A.stall_tol &&
                    conv > A.stall_ratio * rh2)
                    done = true;
            }
            rh2 = rh1;
            rh1 = conv;
        }
        if (!done) {
            // Eq. lin_solve_xy_2 in increment form, K11 applied as hi + lo
            if (act) vec[k] = u;
            __syncwarp();
            if (act) {
                const float d0 = dot2<NC, 3>(blob + (isy ? L.Kyh : L.Kxh) + kk * k_stride(NC), vec);
                const float d1 = dot_vec<NC>(blob + (isy ? L.Kyl : L.Kxl) + kk * k_stride(NC), vec);
                const float dd = (d0 + d1) + (first ? e + corr : e);
                const float snew = c + dd;
                e = dd - (snew - c);
                c = snew;
            }
            __syncwarp();
            if (act) own[k] = c;
            __syncwarp();
        }
        return done;
    };

    // ---- initial iterate: auxiliaries of c^0, no multiplier update -------
    if (!idle) {
        heading(false);
        project(true);
    }
    __syncthreads();
    __shared__ int s_done;
    bool done;
    if constexpr (SOLO) {
        if (warp == 0) {
            const bool d = finish(true, true);
            if (lane == 0) s_done = d;
        }
        __syncthreads();
        done = s_done != 0;
    } else {
        done = finish(true, true);
    }

    // ---- Algorithm 1 ---------------------------------------------------------
    while (!done) {
        ++kit;
        const bool check = (kit % A.check_every == 0) || kit >= iters;
        if (!idle) heading(true);   // theta and the partial sums of P^T theta
        __syncthreads();
        if constexpr (SOLO) {
            if (warp == 0) psi_step();  // Eq. split_psi
            __syncthreads();
        } else {
            psi_step();
        }
        if (!idle) project(check);  // Eqs. split_v, split_alpha_o, split_alpha_a; partial sums
        __syncthreads();
        if constexpr (SOLO) {       // multipliers, residual check, step (split_xy)
            if (warp == 0) {
                const bool d = finish(false, check);
                if (lane == 0) s_done = d;
            }
            __syncthreads();
            done = s_done != 0;
        } else {
            done = finish(false, check);
        }
    }

    // ---- outputs -------------------------------------------------------------
    if (warp == 0) {
        const int n = A.n;
        const size_t o = (size_t)l * 3 * n;
        if (act && k < n) {
            if (!isy) {
                A.coef_out[o + k] = (c + e) + v0 * blob[L.lin + k];
                A.coef_out[o + 2 * n + k] = cpv[k];
            } else {
                A.coef_out[o + n + k] = c + e;
            }
            if (A.lam_out) {
                A.lam_out[o + (isy ? n : 0) + k] = lam;
                if (!isy) A.lam_out[o + 2 * n + k] = lampsi;
            }
        }
        if (A.resid_out && lane < 4) A.resid_out[(size_t)l * 4 + lane] = sqrtf(rsum[lane]);
        if (A.iters_out && lane == 0) A.iters_out[l] = kit;
    }
    if (lane == 0 && A.work && !idle) atomicAdd(A.work, work);
    return true;
}

template <int NC, int MAXT, int PREC = MMPC_PREC_FP32>
__global__ void __launch_bounds__(MAXT, MinBlocks<NC, MAXT>::value) am_solve_kernel(const __grid_constant__ SolveArgs A)
{
    pair_body<NC, MAXT, PREC>(A, blockIdx.x);
}

// ---------------------------------------------------------------------------
// One-sample variant of the fused AM kernel: thread t owns sample t (block:
// 32 ceil(N/32) threads, at most 8 warps), for batches too small to give the
// pair kernel enough warps.  Same algorithm, state layout and barriers; the
// obstacle terms are the same expressions on scalars, accumulated in the
// same obstacle order.
// ---------------------------------------------------------------------------

// obs1 holds per obstacle (-x0/a, -y0/b, -vx/a, -vy/b) in the moving frame.
template <bool RESID, bool LIST>
__device__ __forceinline__ void obstacle_sum1(const float4* __restrict__ obs, const int* __restrict__ list, int m,
                                              float Xn, float Yn, float tt, float a2, float b2, float& Sx, float& Sy,
                                              float& R2)
{
    float sx = 0.f, sy = 0.f, r = 0.f;
    int j = 0;
#pragma unroll 2
    for (; j + 1 < m; j += 2) {
        const float4 o0 = obs[LIST ? list[j] : j];
        const float4 o1 = obs[LIST ? list[j + 1] : j + 1];
        const float nx0 = Xn + fmaf(o0.z, tt, o0.x), ny0 = Yn + fmaf(o0.w, tt, o0.y);
        const float nx1 = Xn + fmaf(o1.z, tt, o1.x), ny1 = Yn + fmaf(o1.w, tt, o1.y);
        const float s0 = fmaxf(rsqrtf(fmaf(nx0, nx0, ny0 * ny0)) - 1.f, 0.f);
        const float s1 = fmaxf(rsqrtf(fmaf(nx1, nx1, ny1 * ny1)) - 1.f, 0.f);
        sx = fmaf(nx1, s1, fmaf(nx0, s0, sx));
        sy = fmaf(ny1, s1, fmaf(ny0, s0, sy));
        if (RESID)
            r = fmaf(s1 * s1, fmaf(a2 * nx1, nx1, b2 * ny1 * ny1), fmaf(s0 * s0, fmaf(a2 * nx0, nx0, b2 * ny0 * ny0), r));
    }
    if (j < m) {
        const float4 o0 = obs[LIST ? list[j] : j];
        const float nx0 = Xn + fmaf(o0.z, tt, o0.x), ny0 = Yn + fmaf(o0.w, tt, o0.y);
        const float s0 = fmaxf(rsqrtf(fmaf(nx0, nx0, ny0 * ny0)) - 1.f, 0.f);
        sx = fmaf(nx0, s0, sx);
        sy = fmaf(ny0, s0, sy);
        if (RESID) r = fmaf(s0 * s0, fmaf(a2 * nx0, nx0, b2 * ny0 * ny0), r);
    }
    Sx = sx;
    Sy = sy;
    R2 = r;
}

__device__ __noinline__ void obstacle_sum1_exact(const float4* __restrict__ obs, int m, float Xn, float Yn, float tt,
                                                 float a2, float b2, float& Sx, float& Sy, float& R2)
{
    Sx = 0.f;
    Sy = 0.f;
    R2 = 0.f;
    for (int j = 0; j < m; ++j) {
        const float4 o = obs[j];
        const float nx = Xn + fmaf(o.z, tt, o.x);
        const float ny = Yn + fmaf(o.w, tt, o.y);
        const float q = fmaf(nx, nx, ny * ny);
        if (q == 0.f) {  // alpha = atan2(0, 0) = 0, d = 1: the row is (-a, 0)
            Sx += 1.f;
            R2 += a2;
        } else {
            const float sj = fmaxf(rsqrtf(q) - 1.f, 0.f);
            Sx = fmaf(nx, sj, Sx);
            Sy = fmaf(ny, sj, Sy);
            R2 = fmaf(sj * sj, fmaf(a2 * nx, nx, b2 * ny * ny), R2);
        }
    }
}

// dot product of two 16-byte aligned vectors of NC floats; four partial sums.
template <int NC>
__device__ __forceinline__ float dot_plain(const float* __restrict__ a, const float* __restrict__ b)
{
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < NC; j += 4) {
        const float4 x = *reinterpret_cast<const float4*>(a + j);
        const float4 y = *reinterpret_cast<const float4*>(b + j);
        acc[0] = fmaf(x.x, y.x, acc[0]);
        acc[1] = fmaf(x.y, y.y, acc[1]);
        acc[2] = fmaf(x.z, y.z, acc[2]);
        acc[3] = fmaf(x.w, y.w, acc[3]);
    }
    return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// single dot product chain (the sample-row evaluations)
template <int NC>
__device__ __forceinline__ float dot_row(const float* __restrict__ row, const float* __restrict__ c)
{
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < NC; j += 4) {
        const float4 x = *reinterpret_cast<const float4*>(row + j);
        const float4 y = *reinterpret_cast<const float4*>(c + j);
        acc = fmaf(x.x, y.x, acc);
        acc = fmaf(x.y, y.y, acc);
        acc = fmaf(x.z, y.z, acc);
        acc = fmaf(x.w, y.w, acc);
    }
    return acc;
}

template <int MAXT>
struct MinBlocks1 {
    static constexpr int value = MAXT <= 128 ? 7 : (MAXT <= 256 ? 3 : 1);
};

template <int NC, int MAXT>
__global__ void __launch_bounds__(MAXT, MinBlocks1<MAXT>::value) am_solve_kernel1(const SolveArgs A)
{
    constexpr int VD = SolveSmem<NC>::VD;
    constexpr int RSD = SolveSmem<NC>::RSD;
    constexpr int RSB = SolveSmem<NC>::RSB;
    extern __shared__ __align__(16) float smem[];
    __shared__ __align__(16) float s_cx[MAX_WARPS][NC];  // per-warp copies of the coefficient vectors
    __shared__ __align__(16) float s_cy[MAX_WARPS][NC];
    __shared__ __align__(16) float s_cp[MAX_WARPS][NC];
    __shared__ __align__(16) float s_vec[MAX_WARPS][2][NC];
    __shared__ __align__(8) unsigned long long s_mbar;

    const int l = blockIdx.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int N = A.N, m = A.m;
    const BlobLayout& L = A.L;
    const int base = L.common;  // the staged region starts at the common section

    float* blob = smem;  // blob[x - base] holds global section offset x
    float4* obs = reinterpret_cast<float4*>(smem + (L.total - base));
    float* red1 = reinterpret_cast<float*>(obs + m);
    float* red2 = red1 + MAX_WARPS * RSB;
    int* olist = reinterpret_cast<int*>(red2 + MAX_WARPS * RSD) + warp * m;
    float* cx = s_cx[warp];
    float* cy = s_cy[warp];
    float* cpv = s_cp[warp];

    const float y0 = __ldg(A.ego + 0), v0 = __ldg(A.ego + 1), psi0 = __ldg(A.ego + 2), acc0 = __ldg(A.ego + 3);
    for (int j = tid; j < m; j += blockDim.x) {
        const float* o = A.obst + 4 * j;
        obs[j] = make_float4(-__ldg(o + 0) * A.inv_a, -__ldg(o + 1) * A.inv_b, -(__ldg(o + 2) - v0) * A.inv_a,
                             -__ldg(o + 3) * A.inv_b);
    }
    if (!stage_blob(blob, A.blob + base, (L.total - base) * 4, &s_mbar, A.err_flag, A.missing_tx)) return;

    const float rho = A.rho;
    const float a2 = A.a * A.a, b2 = A.b * A.b;
    const bool has_t = tid < N;
    const int ts = tid;  // rows are padded to the thread count (zero rows beyond N)
    const float valid = has_t ? 1.f : 0.f;
    const float* Prow = blob + (L.P - base) + ts * NC;
    const float* Pdrow = blob + (L.Pd - base) + ts * NC;
    const float* Pddrow = blob + (L.Pdd - base) + ts * NC;
    const float tt = blob[(L.t - base) + ts];
    const int w_first = 32 * warp;
    const int w_last = min(N, 32 * warp + 32) - 1;
    const float tw_lo = blob[(L.t - base) + w_first], tw_hi = blob[(L.t - base) + w_last];
    unsigned long long work = 0;
    CullState cull;
    cull_init(cull);

    const bool isy = lane >= 16;
    const int k = lane & 15;
    const bool act = k < NC;
    const int kk = act ? k : 0;
    float c = 0.f, e = 0.f, lam = 0.f, lampsi = 0.f, cbp = 0.f, corr = 0.f;
    float* own = isy ? cy : cx;
    float* vec = s_vec[warp][isy ? 1 : 0];
    {
        const float* g = A.goals + 3 * l;
        const float yg = __ldg(g + 0), vg = __ldg(g + 1), ag = __ldg(g + 2);
        float cpsi, spsi;
        sincosf(psi0, &spsi, &cpsi);
        const float bx[6] = {0.f, v0 * cpsi - v0, acc0 * cpsi, vg - v0, ag, 0.f};
        const float by[6] = {y0, v0 * spsi, acc0 * spsi, yg, 0.f, 0.f};
        const float bp[4] = {psi0, 0.f, 0.f, 0.f};
        const int nb = isy ? 6 : 5;
        if (A.warm_c) {
            c = act && k < A.n ? __ldg(A.warm_c + (size_t)l * 3 * A.n + (isy ? A.n : 0) + k) : 0.f;
            if (!isy && act && k < A.n) c -= v0 * blob[(L.lin - base) + k];
        } else {
            const float* C0 = blob + ((isy ? L.C0y : L.C0x) - base) + kk * 8;
            float sacc = 0.f;
#pragma unroll
            for (int r = 0; r < 6; ++r)
                if (r < nb) sacc = fmaf(C0[r], isy ? by[r] : bx[r], sacc);
            c = act ? sacc : 0.f;
        }
        {  // K12 (b - A c^0), added by the first step (see the pair kernel)
            const int rx[6] = {0, 1, 2, 4, 5, 5};
            const float* K12 = blob + ((isy ? L.K12y : L.K12x) - base) + kk * 8;
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                const int row = isy ? r : rx[r];
                float ac = act ? blob[(L.brow - base) + row * NC + kk] * c : 0.f;
                ac += __shfl_xor_sync(FULL, ac, 8);
                ac += __shfl_xor_sync(FULL, ac, 4);
                ac += __shfl_xor_sync(FULL, ac, 2);
                ac += __shfl_xor_sync(FULL, ac, 1);
                if (r < nb) corr = fmaf(K12[r], (isy ? by[r] : bx[r]) - ac, corr);
            }
            if (!act) corr = 0.f;
        }
        {
            const float* Kp12 = blob + (L.Kp12 - base) + kk * 4;
            float sacc = 0.f;
#pragma unroll
            for (int r = 0; r < 4; ++r) sacc = fmaf(Kp12[r], bp[r], sacc);
            cbp = (act && !isy) ? sacc : 0.f;
        }
        float cp0 = 0.f;
        if (!isy && act) {
            if (A.warm_c) {
                cp0 = k < A.n ? __ldg(A.warm_c + (size_t)l * 3 * A.n + 2 * A.n + k) : 0.f;
            } else {
                const float* C0 = blob + (L.C0p - base) + kk * 4;
#pragma unroll
                for (int r = 0; r < 4; ++r) cp0 = fmaf(C0[r], bp[r], cp0);
            }
        }
        if (A.warm_l && act && k < A.n) {
            lam = __ldg(A.warm_l + (size_t)l * 3 * A.n + (isy ? A.n : 0) + k);
            if (!isy) lampsi = __ldg(A.warm_l + (size_t)l * 3 * A.n + 2 * A.n + k);
        }
        if (act) {
            own[k] = c;
            if (!isy) cpv[k] = cp0;
        }
    }
    __syncwarp();

    float xd = 0.f, yd = 0.f, theta = 0.f;
    float rsum[4] = {0.f, 0.f, 0.f, 0.f};
    float rh1 = INFINITY, rh2 = INFINITY;  // convergence residuals of the last two checks
    float* const dstB = rs_dst(RSB, red1, warp, RSB, lane);
    float* const dstD = rs_dst(VD, red2, warp, RSD, lane);
    int kit = 0;
    const int iters = A.iters;

    auto project = [&](bool resid) {
        float v[VD];
#pragma unroll
        for (int i = 0; i < VD; ++i) v[i] = 0.f;
        {
            const float x = dot_row<NC>(Prow, cx);
            const float y = dot_row<NC>(Prow, cy);
            const float xdd = dot_row<NC>(Pddrow, cx);
            const float ydd = dot_row<NC>(Pddrow, cy);
            const float ps = dot_row<NC>(Prow, cpv);
            const float vel = fminf(fmaxf(sqrtf(fmaf(xd, xd, yd * yd)), A.v_min), A.v_max);
            float sn, cs;
            heading_sincos(ps, &sn, &cs);
            const float evx = fmaf(-vel, cs, xd);
            const float evy = fmaf(-vel, sn, yd);
            const float an2 = fmaf(xdd, xdd, ydd * ydd);
            const float fr = 1.f - fminf(1.f, A.a_max * rsqrtf(an2));
            const float eax = xdd * fr, eay = ydd * fr;
            const float Xn = x * A.inv_a, Yn = y * A.inv_b;
            float Sx, Sy, R2;
            if (A.cull) {
                const float inf = __int_as_float(0x7f800000);
                const float bxlo = warp_min(has_t ? Xn : inf), bxhi = warp_max(has_t ? Xn : -inf);
                const float bylo = warp_min(has_t ? Yn : inf), byhi = warp_max(has_t ? Yn : -inf);
                const bool bad = __any_sync(FULL, has_t && !(isfinite(Xn) && isfinite(Yn)));
                const int cnt =
                    cull_update<false>(cull, m, bxlo, bxhi, bylo, byhi, bad, tw_lo, tw_hi, olist, lane, obs);
                if (lane == 0) work += (unsigned long long)cnt * (unsigned)(w_last - w_first + 1);
                if (resid) obstacle_sum1<true, true>(obs, olist, cnt, Xn, Yn, tt, a2, b2, Sx, Sy, R2);
                else obstacle_sum1<false, true>(obs, olist, cnt, Xn, Yn, tt, a2, b2, Sx, Sy, R2);
            } else {
                if (lane == 0) work += (unsigned long long)m * (unsigned)(w_last - w_first + 1);
                if (resid) obstacle_sum1<true, false>(obs, nullptr, m, Xn, Yn, tt, a2, b2, Sx, Sy, R2);
                else obstacle_sum1<false, false>(obs, nullptr, m, Xn, Yn, tt, a2, b2, Sx, Sy, R2);
            }
            if (isnan(Sx) || isnan(Sy)) obstacle_sum1_exact(obs, m, Xn, Yn, tt, a2, b2, Sx, Sy, R2);
            const float eox = -A.a * Sx, eoy = -A.b * Sy;
            const float dpsi = ps - theta;
#pragma unroll
            for (int q = 0; q < NC; q += 4) {
                const float4 p4 = *reinterpret_cast<const float4*>(Prow + q);
                const float4 d4 = *reinterpret_cast<const float4*>(Pdrow + q);
                const float4 dd4 = *reinterpret_cast<const float4*>(Pddrow + q);
                const float pr[4] = {p4.x, p4.y, p4.z, p4.w};
                const float dr[4] = {d4.x, d4.y, d4.z, d4.w};
                const float ddr[4] = {dd4.x, dd4.y, dd4.z, dd4.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    v[q + i] = fmaf(pr[i], eox, fmaf(ddr[i], eax, dr[i] * evx));
                    v[NC + q + i] = fmaf(pr[i], eoy, fmaf(ddr[i], eay, dr[i] * evy));
                    v[2 * NC + q + i] = pr[i] * dpsi;
                }
            }
            if (resid) {
                v[3 * NC + 0] = R2 * valid;
                v[3 * NC + 1] = fmaf(eax, eax, eay * eay) * valid;
                v[3 * NC + 2] = fmaf(evx, evx, evy * evy) * valid;
                v[3 * NC + 3] = dpsi * dpsi * valid;
            }
        }
        reduce_store<VD>(v, dstD, lane);
    };

    auto heading = [&](bool reduce) {
        xd = dot_row<NC>(Pdrow, cx) + v0;
        yd = dot_row<NC>(Pdrow, cy);
        theta = atan2_own(yd, xd);
        if (reduce) {
            float v[NC];
#pragma unroll
            for (int q = 0; q < NC; q += 4) {
                const float4 p4 = *reinterpret_cast<const float4*>(Prow + q);
                v[q + 0] = p4.x * theta;
                v[q + 1] = p4.y * theta;
                v[q + 2] = p4.z * theta;
                v[q + 3] = p4.w * theta;
            }
            reduce_store<NC>(v, dstB, lane);
        }
    };

    auto psi_step = [&]() {
        float pth = 0.f;
        for (int w = 0; w < nwarps; ++w) pth += red1[w * RSB + kk];
        if (!isy && act) vec[k] = fmaf(rho, pth, lampsi);
        __syncwarp();
        if (!isy && act) cpv[k] = cbp + dot_plain<NC>(blob + (L.Kp11 - base) + kk * k_stride(NC), vec);
        __syncwarp();
    };

    auto finish = [&](bool first, bool check) -> bool {
        float ftd = 0.f, pd = 0.f;
        for (int w = 0; w < nwarps; ++w) {
            ftd += red2[w * RSD + (isy ? NC : 0) + kk];
            pd += red2[w * RSD + 2 * NC + kk];
        }
        if (check) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float sacc = 0.f;
                for (int w = 0; w < nwarps; ++w) sacc += red2[w * RSD + 3 * NC + r];
                rsum[r] = sacc;
            }
        }
        if (!first && act) {
            lam = fmaf(-rho, ftd, lam);
            if (!isy) lampsi = fmaf(-rho, pd, lampsi);
        }
        const float qc = dot_plain<NC>(blob + (L.Q - base) + kk * k_stride(NC), own);
        const float u = act ? (lam - qc - rho * ftd) : 0.f;
        bool done = kit >= iters;
        if (check && kit % A.check_every == 0 && (A.tol > 0.f || A.stall_tol > 0.f)) {
            const float conv = fmaxf(sqrtf(rsum[0]), fmaxf(sqrtf(rsum[1]), sqrtf(rsum[2])));
            if (!first) {
                if (A.tol > 0.f) done = done || conv <= A.tol;
                // stall stop: far from the target and not closing in over two checks
                if (A.stall_tol > 0.f && kit >= 2 * A.check_every && conv > A.stall_tol &&
                    conv > A.stall_ratio * rh2)
                    done = true;
            }
            rh2 = rh1;
            rh1 = conv;
        }
        if (!done) {
            if (act) vec[k] = u;
            __syncwarp();
            if (act) {
                const float d0 = dot2<NC, 3>(blob + ((isy ? L.Kyh : L.Kxh) - base) + kk * k_stride(NC), vec);
                const float d1 = dot_plain<NC>(blob + ((isy ? L.Kyl : L.Kxl) - base) + kk * k_stride(NC), vec);
                const float dd = (d0 + d1) + (first ? e + corr : e);
                const float snew = c + dd;
                e = dd - (snew - c);
                c = snew;
            }
            __syncwarp();
            if (act) own[k] = c;
            __syncwarp();
        }
        return done;
    };

    heading(false);
    project(true);
    __syncthreads();
    bool done = finish(true, true);
    while (!done) {
        ++kit;
        const bool check = (kit % A.check_every == 0) || kit >= iters;
        heading(true);
        __syncthreads();
        psi_step();
        project(check);
        __syncthreads();
        done = finish(false, check);
    }

    if (warp == 0) {
        const int n = A.n;
        const size_t o = (size_t)l * 3 * n;
        if (act && k < n) {
            if (!isy) {
                A.coef_out[o + k] = (c + e) + v0 * blob[(L.lin - base) + k];
                A.coef_out[o + 2 * n + k] = cpv[k];
            } else {
                A.coef_out[o + n + k] = c + e;
            }
            if (A.lam_out) {
                A.lam_out[o + (isy ? n : 0) + k] = lam;
                if (!isy) A.lam_out[o + 2 * n + k] = lampsi;
            }
        }
        if (A.resid_out && lane < 4) A.resid_out[(size_t)l * 4 + lane] = sqrtf(rsum[lane]);
        if (A.iters_out && lane == 0) A.iters_out[l] = kit;
    }
    if (lane == 0 && A.work) atomicAdd(A.work, work);
}

// Which misses go (mode, see mmpc_batch_set_fallback): 1 every miss; 2 not a
// miss that the stall rule stopped before the iteration budget (iters_out <
// iters), whose residual trace already showed it far from the target and no
// longer closing in; 3 as 2, and only near misses, whose residual is at most
// near x tol.  A NaN residual always goes.
__device__ __forceinline__ bool fallback_takes(int mode, float near, bool nan, float conv, float tol, int iters_run,
                                               int budget)
{
    if (nan) return true;
    if (conv <= tol) return false;
    if (mode >= 2 && iters_run < budget) return false;
    if (mode == 3 && !(conv <= near * tol)) return false;
    return true;
}

#include "mmpc_tc.cuh"

// ---------------------------------------------------------------------------
// Meta cost (Sec. III-F) and batch argmin.  One warp per trajectory, lanes
// over samples; the argmin is a packed 64-bit atomicMin of (cost bits << 32 |
// index) -- costs are non-negative, so their bit patterns order like the
// values -- finished by the last CTA, which also resets the scratch words.
// ---------------------------------------------------------------------------
// Meta cost of trajectory l (warp-collective; every lane returns it).
template <int NC>
__device__ __forceinline__ float traj_cost(const ScoreArgs& S, int l, int lane)
{
    const int n = S.n, N = S.N;
    const float* cf = S.coef + (size_t)l * 3 * n;
    float cx[NC], cy[NC], cp[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        cx[k] = k < n ? __ldg(cf + k) : 0.f;
        cy[k] = k < n ? __ldg(cf + n + k) : 0.f;
        cp[k] = k < n ? __ldg(cf + 2 * n + k) : 0.f;
    }
    float cost = 0.f;
    bool bad = false;
    for (int t = lane; t < N; t += 32) {
        const float* P = S.blob + S.L.P + t * NC;
        const float* Pd = S.blob + S.L.Pd + t * NC;
        float xd = 0.f, yd = 0.f, y = 0.f, ps = 0.f;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const float p = __ldg(P + k), d = __ldg(Pd + k);
            xd = fmaf(d, cx[k], xd);
            yd = fmaf(d, cy[k], yd);
            y = fmaf(p, cy[k], y);
            ps = fmaf(p, cp[k], ps);
        }
        const float vel = sqrtf(fmaf(xd, xd, yd * yd));
        const float dv = vel - S.v_ref, dy = y - S.y_ref;
        if (S.kind == MMPC_META_CRUISE) cost = fmaf(dv, dv, cost);
        else if (S.kind == MMPC_META_HSRL) cost += S.w1 * dv * dv + S.w2 * dy * dy;
        else cost += S.w1 * fabsf(dv) + S.w2 * fabsf(dy);
        if (S.psi_max > 0.f && fabsf(ps) > S.psi_max) bad = true;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) cost += __shfl_xor_sync(FULL, cost, off);
    bad = __any_sync(FULL, bad);
    if (bad || isnan(cost)) cost = __int_as_float(0x7f800000);
    return cost;
}

__device__ __forceinline__ unsigned long long cost_key(float cost, int l)
{
    return ((unsigned long long)__float_as_uint(cost) << 32) | (unsigned)l;
}

__device__ __forceinline__ int key_argmin(unsigned long long key)
{
    return ((unsigned)(key >> 32) >= 0x7f800000u) ? -1 : (int)(key & 0xffffffffu);
}

template <int NC>
__global__ void __launch_bounds__(256) score_kernel(const ScoreArgs S)
{
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw < S.B) {
        const float cost = traj_cost<NC>(S, gw, lane);
        if (lane == 0) {
            S.cost_out[gw] = cost;
            atomicMin(S.best, cost_key(cost, gw));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(S.ticket, 1u);
        if (ticket == gridDim.x - 1) {
            __threadfence();
            const unsigned long long key = atomicAdd(S.best, 0ull);
            *S.argmin_out = key_argmin(key);
            atomicExch(S.best, ~0ull);
            atomicExch(S.ticket, 0u);
        }
    }
}

// ---------------------------------------------------------------------------
// Batches of scenes.  One persistent launch of the pair kernel body: each CTA
// takes (scene, trajectory) items from a queue (an atomic counter over the
// item list, whose order the schedule sets) until the list is exhausted, and
// stamps each scene's completion time (%globaltimer) when it finishes one of
// its trajectories.  Scoring is one launch over all items with a packed
// 64-bit atomicMin key per scene, and a finalising launch.
// Scratch words: [0] queue counter, [1] earliest CTA start, [2, 2 + S) scene
// completion times, [2 + S, 2 + 2S) scene argmin keys, then one queue counter
// per horizon group (the grouped schedule launches one kernel per group).
// ---------------------------------------------------------------------------
// (global_ns: the device global timer, defined with the staging wait)

template <int NC, int MAXT>
__global__ void __launch_bounds__(MAXT, MinBlocks<NC, MAXT>::value)
    am_solve_batch_kernel(const SolveArgs* __restrict__ scenes, const int2* __restrict__ items,
                          const int* __restrict__ total_ptr, unsigned long long* scratch,
                          unsigned long long* queue)
{
    __shared__ int s_item;
    const int total = *total_ptr;  // written by an earlier launch on the stream
    for (;;) {
        __syncthreads();  // the previous item is finished by every thread
        if (threadIdx.x == 0) {
            s_item = (int)atomicAdd(reinterpret_cast<unsigned*>(queue), 1u);
            atomicMin(scratch + 1, global_ns());
        }
        __syncthreads();
        const int it = s_item;
        if (it >= total) break;
        const int2 sl = items[it];
        // a staging copy that never landed (flagged in the scene's error word)
        // stops this CTA: nothing may be staged over a copy still in flight
        if (!pair_body<NC, MAXT>(scenes[sl.x], sl.y)) break;
        __syncthreads();
        if (threadIdx.x == 0) atomicMax(scratch + 2 + sl.x, global_ns());
    }
}

template <int NC>
__global__ void __launch_bounds__(256) score_batch_kernel(const ScoreArgs* __restrict__ sc,
                                                          const int2* __restrict__ items, int total,
                                                          unsigned long long* keys)
{
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= total) return;
    const int2 sl = items[gw];
    const ScoreArgs& S = sc[sl.x];
    const float cost = traj_cost<NC>(S, sl.y, lane);
    if (lane == 0) {
        S.cost_out[sl.y] = cost;
        atomicMin(keys + sl.x, cost_key(cost, sl.y));
    }
}

__global__ void batch_reset_kernel(unsigned long long* scratch, int S, int G, int* fb_count)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 + 2 * S + G; i += gridDim.x * blockDim.x)
        scratch[i] = (i == 1 || (i >= 2 + S && i < 2 + 2 * S)) ? ~0ull : 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) *fb_count = 0;
}

// Fallback of warm-started trajectories: every item of a scene with a warm
// start whose convergence residual (the largest of the obstacle,
// acceleration and non-holonomic residuals) missed the scene's tol > 0, or is
// NaN, and that fallback_takes selects, goes to the fallback list, to be
// solved again from the cold start.  The list order depends on timing; each
// trajectory's solve does not.  Also rewinds the work queue for the next
// persistent launch.
__global__ void fallback_compact_kernel(const SolveArgs* __restrict__ warm, const int2* __restrict__ items, int total,
                                        int2* __restrict__ fb_items, int* __restrict__ fb_count,
                                        unsigned long long* scratch, int mode, float near)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) scratch[0] = 0ull;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int2 sl = items[i];
        const SolveArgs& A = warm[sl.x];
        if (!A.warm_c || !A.resid_out || !(A.tol > 0.f)) continue;
        const float* r = A.resid_out + (size_t)sl.y * 4;
        const float conv = fmaxf(fmaxf(r[0], r[1]), r[2]);
        const bool nan = isnan(r[0]) || isnan(r[1]) || isnan(r[2]);
        const int run = A.iters_out ? A.iters_out[sl.y] : A.iters;
        if (!fallback_takes(mode, near, nan, conv, A.tol, run, A.iters)) continue;
        fb_items[atomicAdd(fb_count, 1)] = sl;
    }
}

__global__ void batch_finish_kernel(const ScoreArgs* __restrict__ sc, int S, const unsigned long long* keys)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x)
        *sc[s].argmin_out = key_argmin(keys[s]);
}

}  // namespace mmpc

// ---------------------------------------------------------------------------
// Context and C ABI
// ---------------------------------------------------------------------------
struct mmpc_ctx {
    mmpc_params p;
    int m;
    int NC;
    mmpc::BlobLayout L;
    float* d_blob = nullptr;
    unsigned long long* d_scratch = nullptr;  // [0] packed argmin key, [1] low: ticket, high: error flags, [2] work count
    int sm_count = -1;                        // SMs of the device (queried on the first solve)
    int last_variant = 0;
    int debug_missing = 0;  // mmpc_debug_expire_wait: bytes the staging wait expects beyond the copy
    mmpc::TcLayout tc{};             // variant 3: layout of the tensor-core operand blob
    unsigned char* d_tc = nullptr;   // variant 3: the blob (device)
    int* d_order = nullptr;          // variant 3: bucket counts [TC_BUCKETS], then the slot order [order_cap]
    int order_cap = 0;
    std::string err = "no error";
    // device buffers of mmpc_step_host, grown on demand: inputs (ego, obstacles,
    // goals) and outputs (coef, resid, iters, cost, argmin) for up to host_cap goals
    float* h_in = nullptr;
    float* h_out = nullptr;
    int host_cap = 0;
};

namespace {

using namespace mmpc;

int fail(mmpc_ctx* ctx, int code, const std::string& msg)
{
    if (ctx) ctx->err = msg;
    else set_global_error(msg);
    return code;
}

int cuda_fail(mmpc_ctx* ctx, cudaError_t e, const char* what)
{
    return fail(ctx, MMPC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename K>
int launch_kernel(mmpc_ctx* ctx, K kern, const SolveArgs& a, int threads, size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
    kern<<<a.B, threads, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "solve launch");
    return MMPC_OK;
}

// Variant 3, the tensor-core kernel: persistent CTAs (384 threads, all 512
// tensor-memory columns, one per SM) taking items of 32 goals from a queue.
template <int NC>
void* tc_kernel(int prec)
{
    switch (prec) {
    case MMPC_PREC_TF32: return (void*)am_solve_tc_kernel<NC, MMPC_PREC_TF32>;
    case MMPC_PREC_TF32_SPLIT: return (void*)am_solve_tc_kernel<NC, MMPC_PREC_TF32_SPLIT>;
    case MMPC_PREC_BF16: return (void*)am_solve_tc_kernel<NC, MMPC_PREC_BF16>;
    default: return (void*)am_solve_tc_kernel<NC, MMPC_PREC_BF16_SPLIT>;
    }
}

void* tc_kernel_of(const mmpc_ctx* ctx)
{
    return ctx->NC == 12 ? tc_kernel<12>(ctx->p.precision) : tc_kernel<16>(ctx->p.precision);
}

size_t tc_smem(const mmpc_ctx* ctx, int m)
{
    const int nmat = ctx->L.init - ctx->L.Q;
    return (size_t)ctx->tc.bytes + sizeof(float) * (size_t)((nmat + 3) & ~3) + 128 * (size_t)m +
           sizeof(int) * (size_t)(TC_THREADS / 32) * m + sizeof(float) * 3 * 128 * 4 +
           sizeof(float) * (size_t)ctx->tc.NSP;
}

int launch_tc(mmpc_ctx* ctx, const SolveArgs& a, int B, cudaStream_t st)
{
    if (ctx->sm_count < 0) {
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "device query");
        ctx->sm_count = sms;
    }
    if (B > ctx->order_cap) {  // grown on demand (a first solve of a larger batch, outside graph capture)
        const int cap = std::max(B, 2 * ctx->order_cap);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
            cudaFree(ctx->d_order);
            ctx->d_order = nullptr;
            ctx->order_cap = 0;
            e = cudaMalloc(&ctx->d_order, sizeof(int) * ((size_t)4 + TC_BUCKETS + cap));
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "variant 3 order buffer");
        ctx->order_cap = cap;
    }
    int* queue = ctx->d_order;  // [queue | pad to 4 | bucket counts | order]
    int* count = ctx->d_order + 4;
    int* order = ctx->d_order + 4 + TC_BUCKETS;
    const int og = std::min(1024, (B + 255) / 256);
    cudaError_t e0 = cudaMemsetAsync(ctx->d_order, 0, sizeof(int) * (4 + TC_BUCKETS), st);
    if (e0 != cudaSuccess) return cuda_fail(ctx, e0, "cudaMemsetAsync");
    tc_order_count<<<og, 256, 0, st>>>(a.goals, B, count);
    tc_order_scan<<<1, 1024, 0, st>>>(count);
    tc_order_scatter<<<og, 256, 0, st>>>(a.goals, B, count, order);
    TcArgs T{};
    T.blob = ctx->d_tc;
    T.L = ctx->tc;
    T.scenes = nullptr;
    T.items = nullptr;
    T.n_items = (B + 31) / 32;
    T.order = order;
    T.queue = queue;
    // at least 116 KB, so that one CTA holds an SM (it allocates all of the
    // SM's tensor memory; a second CTA would only wait in tcgen05.alloc)
    const size_t smem = std::max<size_t>(tc_smem(ctx, a.m), 116 * 1024);
    if (smem > 227 * 1024) return fail(ctx, MMPC_ERR_SHAPE, "scene does not fit in shared memory");
    using K = void (*)(const SolveArgs, const TcArgs);
    K kern = reinterpret_cast<K>(ctx->NC == 12 ? tc_kernel<12>(ctx->p.precision) : tc_kernel<16>(ctx->p.precision));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
    // persistent: one CTA per SM (or fewer, four items each to start)
    const int grid = std::max(1, std::min(ctx->sm_count, (T.n_items + 3) / 4));
    kern<<<grid, TC_THREADS, smem, st>>>(a, T);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tensor-core solve launch");
    ctx->last_variant = 3;
    return MMPC_OK;
}

// The pair kernel: ceil(N/2) pair threads rounded up to warps.
template <int NC>
void* pair_kernel(int threads)
{
    if (threads <= 64) return (void*)am_solve_kernel<NC, 64>;
    if (threads <= 128) return (void*)am_solve_kernel<NC, 128>;
    return (void*)am_solve_kernel<NC, 256>;
}

// The one-sample kernel: N threads rounded up to warps.
template <int NC>
void* single_kernel(int threads)
{
    if (threads <= 128) return (void*)am_solve_kernel1<NC, 128>;
    return (void*)am_solve_kernel1<NC, 256>;
}

struct LaunchShape {
    void* kern;
    int threads;
    size_t smem;
};

// Launch bound (template MAXT) of the pair kernel for a block of `threads`.
int pair_maxt(int threads) { return threads <= 64 ? 64 : (threads <= 128 ? 128 : 256); }

// Dynamic shared memory of the pair kernel body: the staged rows and common
// block (`staged` floats), the obstacles, the partial-sum rows of every warp
// of the launch bound, and the culling lists of the block's warps.
size_t pair_smem(int staged, int m, int NC, int threads)
{
    const int RSD = NC == 12 ? SolveSmem<12>::RSD : SolveSmem<16>::RSD;
    const int warps = pair_maxt(threads) / 32;
    return sizeof(float) * (size_t)staged + 32 * (size_t)m + sizeof(float) * (size_t)warps * (NC + RSD) +
           sizeof(int) * (size_t)(threads / 32) * m;
}

LaunchShape shape_for(const mmpc_ctx* ctx, int variant, int m)
{
    const int N = ctx->p.N;
    const int RSD = ctx->NC == 12 ? SolveSmem<12>::RSD : SolveSmem<16>::RSD;
    const int RSB = ctx->NC;
    const size_t red = sizeof(float) * (size_t)MAX_WARPS * (RSB + RSD);
    LaunchShape s{};
    if (variant == 1) {
        s.threads = 32 * ((N + 31) / 32);
        s.smem = sizeof(float) * (size_t)(ctx->L.total - ctx->L.common) + 16 * (size_t)m + red +
                 sizeof(int) * (size_t)(s.threads / 32) * m;
        s.kern = ctx->NC == 12 ? single_kernel<12>(s.threads) : single_kernel<16>(s.threads);
    } else {
        const int NP = (N + 1) / 2;
        s.threads = 32 * ((NP + 31) / 32);
        s.smem = pair_smem(ctx->L.init, m, ctx->NC, s.threads);
        s.kern = ctx->NC == 12 ? pair_kernel<12>(s.threads) : pair_kernel<16>(s.threads);
    }
    return s;
}

bool finite4(float v) { return std::isfinite(v); }

}  // namespace

extern "C" int mmpc_setup(const mmpc_params* p, int m, const double* buf, size_t buf_len, mmpc_ctx** out)
{
    if (out) *out = nullptr;
    if (!out) return fail(nullptr, MMPC_ERR_INVALID_ARG, "out is NULL");
    std::string err = check_params(p);
    if (!err.empty()) return fail(nullptr, (p && !sizes_ok(p->N, p->n)) ? MMPC_ERR_SHAPE : MMPC_ERR_INVALID_ARG, err);
    if (m < 0 || m > MMPC_MAX_OBST) return fail(nullptr, MMPC_ERR_SHAPE, "m out of range");
    const int N = p->N, n = p->n;
    const ProblemLayout PL = layout(N, n);
    if (!buf || buf_len < PL.total) return fail(nullptr, MMPC_ERR_INVALID_ARG, "problem buffer missing or too small");
    for (size_t i = 0; i < PL.total; ++i)
        if (!std::isfinite(buf[i])) return fail(nullptr, MMPC_ERR_INVALID_ARG, "problem buffer holds a non-finite value");

    if (p->variant == 3 && m > TC_MAX_M) return fail(nullptr, MMPC_ERR_SHAPE, "variant 3 takes at most 128 obstacles");
    const int NC = n <= 12 ? 12 : 16;
    // the CUDA-core rows carry the emulated precision modes (variants 0 and
    // 2); with variant 3 the tensor cores take the precision and these rows
    // (used by the FP32 fallback and scoring) stay FP32
    const int prec = p->variant == 3 ? MMPC_PREC_FP32 : p->precision;
    const BlobLayout L = blob_layout(N, NC, prec_split(prec));
    std::vector<float> h(L.total, 0.f);
    auto h_set = [&](int i, float v) { h[i] = v; };
    auto mat = [&](size_t src, int dst, int rows, int cols, int dcols, bool lo) {
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c) {
                const double v = buf[src + (size_t)r * cols + c];
                const float hi = (float)v;
                h[dst + r * dcols + c] = lo ? (float)(v - (double)hi) : hi;
            }
    };
    // basis rows of the sample pairs (2i, 2i+1): per coefficient pair (2j,
    // 2j+1) the block (s0 2j, s0 2j+1, s1 2j, s1 2j+1)
    const int NP = (N + 1) / 2;
    // (precision modes: the rows rounded as the tensor cores would take them,
    // hi into the rows and lo into the lo rows in the split modes)
    auto pairs = [&](size_t src, int dst, int dst_lo) {
        for (int i = 0; i < NP; ++i)
            for (int h = 0; h < 2; ++h) {
                const int smp = 2 * i + h;
                if (smp >= N) continue;
                for (int c = 0; c < n; ++c) {
                    const float f = (float)buf[src + (size_t)smp * n + c];
                    const float hi = round_operand(f, prec);
                    const int at = i * pair_stride(NC) + 4 * (c >> 1) + 2 * h + (c & 1);
                    h_set(dst + at, hi);
                    if (prec_split(prec)) h_set(dst_lo + at, round_operand(f - hi, prec));
                }
            }
    };
    pairs(PL.P, L.PP, L.PPl);
    pairs(PL.Pd, L.PdP, L.PdPl);
    pairs(PL.Pdd, L.PddP, L.PddPl);
    for (int smp = 0; smp < N; ++smp) h_set(L.tP + smp, (float)buf[PL.t + smp]);
    const size_t brow_src[6] = {PL.P, PL.Pd, PL.Pdd, PL.P + (size_t)(N - 1) * n, PL.Pd + (size_t)(N - 1) * n,
                                PL.Pdd + (size_t)(N - 1) * n};
    for (int r = 0; r < 6; ++r) mat(brow_src[r], L.brow + r * NC, 1, n, n, false);
    mat(PL.P, L.P, N, n, NC, false);
    mat(PL.Pd, L.Pd, N, n, NC, false);
    mat(PL.Pdd, L.Pdd, N, n, NC, false);
    mat(PL.t, L.t, 1, N, N, false);
    mat(PL.lin, L.lin, 1, n, n, false);
    mat(PL.Q, L.Q, n, n, k_stride(NC), false);
    mat(PL.K11x, L.Kxh, n, n, k_stride(NC), false);
    mat(PL.K11x, L.Kxl, n, n, k_stride(NC), true);
    mat(PL.K11y, L.Kyh, n, n, k_stride(NC), false);
    mat(PL.K11y, L.Kyl, n, n, k_stride(NC), true);
    mat(PL.K11p, L.Kp11, n, n, k_stride(NC), false);
    mat(PL.K12p, L.Kp12, n, MMPC_NEQ_PSI, 4, false);
    mat(PL.K12x, L.K12x, n, MMPC_NEQ_X, 8, false);
    mat(PL.K12y, L.K12y, n, MMPC_NEQ_Y, 8, false);
    mat(PL.C0x, L.C0x, n, MMPC_NEQ_X, 8, false);
    mat(PL.C0y, L.C0y, n, MMPC_NEQ_Y, 8, false);
    mat(PL.C0p, L.C0p, n, MMPC_NEQ_PSI, 4, false);

    // variant 3: the basis blocks as the tensor cores' B operands (layouts at
    // TcLayout), rounded to the precision's type, hi and (split) lo
    std::vector<unsigned char> htc;
    TcLayout TL{};
    if (p->variant == 3) {
        const int tprec = p->precision;
        const bool bf = tprec == MMPC_PREC_BF16 || tprec == MMPC_PREC_BF16_SPLIT;
        const int esz = bf ? 2 : 4, per = 16 / esz;
        TL = tc_layout(N, esz, prec_split(tprec) ? 2 : 1);
        htc.assign(TL.bytes, 0);
        const size_t src[3] = {PL.P, PL.Pd, PL.Pdd};
        auto put = [&](int off, float v) {
            if (bf) {
                unsigned u;
                memcpy(&u, &v, 4);
                const uint16_t hbits = (uint16_t)(u >> 16);  // v is already rounded to BF16
                memcpy(&htc[off], &hbits, 2);
            } else {
                memcpy(&htc[off], &v, 4);
            }
        };
        for (int b = 0; b < 3; ++b)
            for (int smp = 0; smp < N; ++smp)
                for (int k = 0; k < n; ++k) {
                    const double v = buf[src[b] + (size_t)smp * n + k];
                    const float hi = round_operand((float)v, tprec);
                    const float lo = round_operand((float)(v - (double)hi), tprec);
                    for (int part = 0; part < TL.parts; ++part) {
                        const float x = part == 0 ? hi : lo;
                        put(TL.eb[b][part] + (k / per) * TL.NSP * 16 + 16 * smp + (k % per) * esz, x);
                        put(TL.cb[b][part] + (smp / per) * 256 + 16 * k + (smp % per) * esz, x);
                    }
                }
    }

    mmpc_ctx* ctx = new mmpc_ctx();
    ctx->p = *p;
    ctx->m = m;
    ctx->NC = NC;
    ctx->L = L;
    ctx->tc = TL;
    cudaError_t e = cudaMalloc(&ctx->d_blob, sizeof(float) * L.total);
    if (e == cudaSuccess && !htc.empty()) e = cudaMalloc(&ctx->d_tc, htc.size());
    if (e == cudaSuccess && !htc.empty()) e = cudaMemcpy(ctx->d_tc, htc.data(), htc.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_scratch, 3 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(ctx->d_blob, h.data(), sizeof(float) * L.total, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const unsigned long long init[3] = {~0ull, 0ull, 0ull};
        e = cudaMemcpy(ctx->d_scratch, init, sizeof(init), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        std::string msg = std::string("mmpc_setup: ") + cudaGetErrorString(e);
        cudaFree(ctx->d_blob);
        cudaFree(ctx->d_scratch);
        cudaFree(ctx->d_tc);
        delete ctx;
        return fail(nullptr, MMPC_ERR_CUDA, msg);
    }
    *out = ctx;
    return MMPC_OK;
}

extern "C" int mmpc_solve(mmpc_ctx* ctx, const float* ego, const float* obst, int m, const float* goals, int B,
                          const float* warm_coef, const float* warm_lam, float* coef_out, float* lam_out,
                          float* resid_out, int* iters_out, void* stream)
{
    if (!ctx || !ctx->d_blob) return fail(nullptr, MMPC_ERR_NOT_SETUP, "context not set up");
    if (B < 0) return fail(ctx, MMPC_ERR_SHAPE, "B < 0");
    if (m != ctx->m) return fail(ctx, MMPC_ERR_SHAPE, "m differs from the m of mmpc_setup");
    if (!ego || (m > 0 && !obst) || (B > 0 && (!goals || !coef_out)))
        return fail(ctx, MMPC_ERR_INVALID_ARG, "NULL pointer argument");
    if (B == 0) return MMPC_OK;
    const mmpc_params& p = ctx->p;
    SolveArgs a{};
    a.N = p.N; a.n = p.n; a.m = m; a.B = B; a.iters = p.iters; a.check_every = p.check_every;
    a.rho = (float)p.rho; a.a = (float)p.a; a.b = (float)p.b;
    a.inv_a = (float)(1.0 / p.a); a.inv_b = (float)(1.0 / p.b);
    a.v_min = (float)p.v_min; a.v_max = (float)p.v_max; a.a_max = (float)p.a_max; a.tol = p.tol;
    a.stall_tol = p.stall_tol; a.stall_ratio = p.stall_ratio;
    a.L = ctx->L;
    a.blob = ctx->d_blob;
    a.ego = ego; a.obst = obst; a.goals = goals; a.warm_c = warm_coef; a.warm_l = warm_lam;
    a.coef_out = coef_out; a.lam_out = lam_out; a.resid_out = resid_out; a.iters_out = iters_out;
    a.err_flag = reinterpret_cast<unsigned*>(ctx->d_scratch + 1) + 1;
    a.work = ctx->d_scratch + 2;
    a.missing_tx = ctx->debug_missing;
    a.cull = p.cull ? 1 : 0;
    int variant = p.variant;
    if (variant == 0) {
        // automatic: the pair kernel (half the instructions per sample),
        // except for batches of at most one trajectory per SM, where the
        // one-sample kernel's four warps per trajectory shorten the latency
        variant = 2;
        if (p.N <= 256) {
            if (ctx->sm_count < 0) {
                int dev = 0, sms = 0;
                cudaError_t e = cudaGetDevice(&dev);
                if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "device query");
                ctx->sm_count = sms;
            }
            if (B <= ctx->sm_count) variant = 1;
        }
    }
    if (variant == 3) return launch_tc(ctx, a, B, reinterpret_cast<cudaStream_t>(stream));
    if (p.precision != MMPC_PREC_FP32) variant = 2;  // the emulated precision modes exist in the pair kernel only
    LaunchShape sh = shape_for(ctx, variant, m);
    if (p.precision != MMPC_PREC_FP32) {  // NC = 16, 128 threads (checked at setup)
        using K = void (*)(const SolveArgs);
        const K kp[5] = {nullptr, am_solve_kernel<16, 128, MMPC_PREC_TF32>, am_solve_kernel<16, 128, MMPC_PREC_TF32_SPLIT>,
                         am_solve_kernel<16, 128, MMPC_PREC_BF16>, am_solve_kernel<16, 128, MMPC_PREC_BF16_SPLIT>};
        sh.kern = (void*)kp[p.precision];
    }
    if (sh.smem > 227 * 1024) return fail(ctx, MMPC_ERR_SHAPE, "scene does not fit in shared memory");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    using KernT = void (*)(const SolveArgs);
    ctx->last_variant = variant;
    return launch_kernel(ctx, reinterpret_cast<KernT>(sh.kern), a, sh.threads, sh.smem, st);
}

extern "C" int mmpc_score(mmpc_ctx* ctx, const mmpc_meta* meta, const float* coef, int B, float* cost_out,
                          int* argmin_out, void* stream)
{
    if (!ctx || !ctx->d_blob) return fail(nullptr, MMPC_ERR_NOT_SETUP, "context not set up");
    if (!meta || !argmin_out || (B > 0 && (!coef || !cost_out))) return fail(ctx, MMPC_ERR_INVALID_ARG, "NULL pointer argument");
    if (B < 0) return fail(ctx, MMPC_ERR_SHAPE, "B < 0");
    if (meta->kind < MMPC_META_CRUISE || meta->kind > MMPC_META_ABS) return fail(ctx, MMPC_ERR_INVALID_ARG, "unknown meta kind");
    if (!(meta->w1 >= 0.f) || !(meta->w2 >= 0.f) || !finite4(meta->w1) || !finite4(meta->w2) || !finite4(meta->v_ref) ||
        !finite4(meta->y_ref) || std::isnan(meta->psi_max))
        return fail(ctx, MMPC_ERR_INVALID_ARG, "meta weights must be finite and >= 0");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (B == 0) {
        cudaError_t e = cudaMemsetAsync(argmin_out, 0xff, sizeof(int), st);  // -1
        return e == cudaSuccess ? MMPC_OK : cuda_fail(ctx, e, "cudaMemsetAsync");
    }
    ScoreArgs s{};
    s.N = ctx->p.N; s.n = ctx->p.n; s.B = B; s.kind = meta->kind;
    s.w1 = meta->w1; s.w2 = meta->w2; s.v_ref = meta->v_ref; s.y_ref = meta->y_ref; s.psi_max = meta->psi_max;
    s.L = ctx->L; s.blob = ctx->d_blob; s.coef = coef; s.cost_out = cost_out; s.argmin_out = argmin_out;
    s.best = ctx->d_scratch;
    s.ticket = reinterpret_cast<unsigned*>(ctx->d_scratch + 1);
    const int wpb = 8;
    const int grid = (B + wpb - 1) / wpb;
    if (ctx->NC == 12) score_kernel<12><<<grid, 32 * wpb, 0, st>>>(s);
    else score_kernel<16><<<grid, 32 * wpb, 0, st>>>(s);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MMPC_OK : cuda_fail(ctx, e, "score launch");
}

extern "C" int mmpc_take_work_count(mmpc_ctx* ctx, unsigned long long* elements)
{
    if (!ctx || !ctx->d_blob) return fail(nullptr, MMPC_ERR_NOT_SETUP, "context not set up");
    if (!elements) return fail(ctx, MMPC_ERR_INVALID_ARG, "NULL pointer argument");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(elements, ctx->d_scratch + 2, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_scratch + 2, 0, sizeof(unsigned long long));
    return e == cudaSuccess ? MMPC_OK : cuda_fail(ctx, e, "mmpc_take_work_count");
}

namespace {

// Reads and clears the device error word of a context (device scratch [1],
// high half) after the stream has drained.
int take_error_word(mmpc_ctx* ctx, cudaStream_t st, unsigned* word)
{
    unsigned* d_word = reinterpret_cast<unsigned*>(ctx->d_scratch + 1) + 1;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(word, d_word, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && *word) e = cudaMemset(d_word, 0, sizeof(unsigned));
    return e == cudaSuccess ? MMPC_OK : cuda_fail(ctx, e, "mmpc_status");
}

}  // namespace

extern "C" int mmpc_status(mmpc_ctx* ctx, void* stream)
{
    if (!ctx || !ctx->d_blob) return fail(nullptr, MMPC_ERR_NOT_SETUP, "context not set up");
    unsigned word = 0;
    const int rc = take_error_word(ctx, reinterpret_cast<cudaStream_t>(stream), &word);
    if (rc != MMPC_OK) return rc;
    return word ? fail(ctx, MMPC_ERR_TIMEOUT, "a bounded device wait expired (staging of the constants)") : MMPC_OK;
}

extern "C" int mmpc_debug_expire_wait(mmpc_ctx* ctx, int on)
{
    if (!ctx || !ctx->d_blob) return fail(nullptr, MMPC_ERR_NOT_SETUP, "context not set up");
    ctx->debug_missing = on ? 16 : 0;
    return MMPC_OK;
}

extern "C" int mmpc_step_host(mmpc_ctx* ctx, const mmpc_meta* meta, const float* ego, const float* obst, int m,
                              const float* goals, int B, float* coef_out, float* resid_out, float* cost_out,
                              int* argmin_out, void* stream)
{
    if (!ctx || !ctx->d_blob) return fail(nullptr, MMPC_ERR_NOT_SETUP, "context not set up");
    if (!meta || !ego || (m > 0 && !obst) || !argmin_out || (B > 0 && (!goals || !coef_out || !cost_out)))
        return fail(ctx, MMPC_ERR_INVALID_ARG, "NULL pointer argument");
    if (B < 0) return fail(ctx, MMPC_ERR_SHAPE, "B < 0");
    if (m != ctx->m) return fail(ctx, MMPC_ERR_SHAPE, "m differs from the m of mmpc_setup");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int n = ctx->p.n;
    // device layout: in = [ego 4 | obst 4m | goals 3B], out = [coef 3nB | resid 4B | cost B | iters B | argmin 1]
    if (B > ctx->host_cap || !ctx->h_in) {
        const int cap = std::max(B, std::max(1, 2 * ctx->host_cap));
        cudaError_t e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) { cudaFree(ctx->h_in); cudaFree(ctx->h_out); ctx->h_in = nullptr; ctx->h_out = nullptr; }
        if (e == cudaSuccess) e = cudaMalloc(&ctx->h_in, sizeof(float) * (4 + 4 * (size_t)m + 3 * (size_t)cap));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->h_out, sizeof(float) * ((3 * (size_t)n + 6) * cap + 1));
        if (e != cudaSuccess) { ctx->host_cap = 0; return cuda_fail(ctx, e, "mmpc_step_host buffers"); }
        ctx->host_cap = cap;
    }
    float* d_ego = ctx->h_in;
    float* d_obst = d_ego + 4;
    float* d_goals = d_obst + 4 * (size_t)m;
    float* d_coef = ctx->h_out;
    float* d_resid = d_coef + 3 * (size_t)n * B;
    float* d_cost = d_resid + 4 * (size_t)B;
    int* d_iters = reinterpret_cast<int*>(d_cost + B);
    int* d_argmin = d_iters + B;
    // one host->device copy of the inputs when the host holds them contiguously in the
    // device order (ego, obstacles, goals), else one copy per array
    cudaError_t e = cudaSuccess;
    const bool in_contig = (m == 0 || obst == ego + 4) && (B == 0 || goals == ego + 4 + 4 * (size_t)m);
    if (in_contig) {
        e = cudaMemcpyAsync(d_ego, ego, sizeof(float) * (4 + 4 * (size_t)m + 3 * (size_t)B), cudaMemcpyHostToDevice, st);
    } else {
        e = cudaMemcpyAsync(d_ego, ego, sizeof(float) * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && m > 0)
            e = cudaMemcpyAsync(d_obst, obst, sizeof(float) * 4 * (size_t)m, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && B > 0)
            e = cudaMemcpyAsync(d_goals, goals, sizeof(float) * 3 * (size_t)B, cudaMemcpyHostToDevice, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mmpc_step_host input copy");
    int rc = mmpc_solve(ctx, d_ego, m ? d_obst : nullptr, m, d_goals, B, nullptr, nullptr, d_coef, nullptr, d_resid,
                        d_iters, stream);
    if (rc != MMPC_OK) return rc;
    rc = mmpc_score(ctx, meta, d_coef, B, d_cost, d_argmin, stream);
    if (rc != MMPC_OK) return rc;
    // the outputs are contiguous on the device (coef, resid, cost): one device->host
    // copy when the host asks for all three, contiguously in that order
    e = cudaSuccess;
    const bool out_contig = resid_out && resid_out == coef_out + 3 * (size_t)n * B && cost_out == resid_out + 4 * (size_t)B;
    if (B > 0 && out_contig) {
        e = cudaMemcpyAsync(coef_out, d_coef, sizeof(float) * (3 * (size_t)n + 5) * B, cudaMemcpyDeviceToHost, st);
    } else if (B > 0) {
        e = cudaMemcpyAsync(coef_out, d_coef, sizeof(float) * 3 * (size_t)n * B, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && resid_out)
            e = cudaMemcpyAsync(resid_out, d_resid, sizeof(float) * 4 * (size_t)B, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cost_out, d_cost, sizeof(float) * (size_t)B, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(argmin_out, d_argmin, sizeof(int), cudaMemcpyDeviceToHost, st);
    // the context's error word rides along: an expired device wait is reported here
    unsigned word = 0;
    unsigned* d_word = reinterpret_cast<unsigned*>(ctx->d_scratch + 1) + 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&word, d_word, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && word) {
        e = cudaMemset(d_word, 0, sizeof(unsigned));
        if (e == cudaSuccess) return fail(ctx, MMPC_ERR_TIMEOUT, "a bounded device wait expired (staging of the constants)");
    }
    return e == cudaSuccess ? MMPC_OK : cuda_fail(ctx, e, "mmpc_step_host");
}

extern "C" void mmpc_destroy(mmpc_ctx* ctx)
{
    if (!ctx) return;
    cudaDeviceSynchronize();
    cudaFree(ctx->d_blob);
    cudaFree(ctx->d_scratch);
    cudaFree(ctx->d_tc);
    cudaFree(ctx->d_order);
    cudaFree(ctx->h_in);
    cudaFree(ctx->h_out);
    delete ctx;
}

extern "C" const char* mmpc_last_error(const mmpc_ctx* ctx)
{
    if (ctx) return ctx->err.c_str();
    return mmpc::g_error.c_str();
}

extern "C" int mmpc_version(void) { return 2; }

// ---------------------------------------------------------------------------
// Allocation-free scoring (mmpc_score_static).
//
// For callers that must not allocate device memory once they are running --
// a hard real-time control loop whose memory is all reserved at start-up, or
// a host framework that hands out device memory only from its own pool and
// forbids raw cudaMalloc/cudaFree -- this entry point scores a batch without a
// context and without any allocation.  Its scratch (a ticket counter and one
// partial argmin key per CTA) lives in the file-scope array below, which every
// GPU that loads this library holds until the process exits.  Consequences:
//  * all calls share the array and it keeps the last call's contents; the
//    ticket is cleared by each call before its kernel runs, and each CTA
//    writes its own key before the last CTA reads it;
//  * calls whose kernels overlap on the GPU (different streams, or several
//    host threads) race on the array and must be serialised by the caller;
//  * the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it; make that
//    first call before any stream capture.
// ---------------------------------------------------------------------------
namespace mmpc {

constexpr int STATIC_WARPS_PER_CTA = 8;
constexpr int STATIC_MAX_CTAS = MMPC_STATIC_SCORE_MAX_B / STATIC_WARPS_PER_CTA;

// [0]: ticket counter (low 32 bits); [1 + i]: best packed key of CTA i.
static __device__ __align__(256) unsigned long long g_static_score_scratch[1 + STATIC_MAX_CTAS];

struct StaticScoreArgs {
    int N, n, B, kind;
    float w1, w2, v_ref, y_ref, psi_max;
    const float* P;   // [N][n]
    const float* Pd;  // [N][n]
    const float* coef;
    float* cost_out;
    int* argmin_out;
    unsigned long long* scratch;
};

template <int NC>
__global__ void __launch_bounds__(32 * STATIC_WARPS_PER_CTA) score_static_kernel(const StaticScoreArgs S)
{
    __shared__ unsigned long long s_key[STATIC_WARPS_PER_CTA];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * STATIC_WARPS_PER_CTA + warp;
    unsigned long long key = ~0ull;
    if (gw < S.B) {
        const int n = S.n, N = S.N;
        const float* cf = S.coef + (size_t)gw * 3 * n;
        float cx[NC], cy[NC], cp[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            cx[k] = k < n ? __ldg(cf + k) : 0.f;
            cy[k] = k < n ? __ldg(cf + n + k) : 0.f;
            cp[k] = k < n ? __ldg(cf + 2 * n + k) : 0.f;
        }
        float cost = 0.f;
        bool bad = false;
        for (int t = lane; t < N; t += 32) {
            float xd = 0.f, yd = 0.f, y = 0.f, ps = 0.f;
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                const float p = k < n ? __ldg(S.P + t * n + k) : 0.f;
                const float d = k < n ? __ldg(S.Pd + t * n + k) : 0.f;
                xd = fmaf(d, cx[k], xd);
                yd = fmaf(d, cy[k], yd);
                y = fmaf(p, cy[k], y);
                ps = fmaf(p, cp[k], ps);
            }
            const float vel = sqrtf(fmaf(xd, xd, yd * yd));
            const float dv = vel - S.v_ref, dy = y - S.y_ref;
            if (S.kind == MMPC_META_CRUISE) cost = fmaf(dv, dv, cost);
            else if (S.kind == MMPC_META_HSRL) cost += S.w1 * dv * dv + S.w2 * dy * dy;
            else cost += S.w1 * fabsf(dv) + S.w2 * fabsf(dy);
            if (S.psi_max > 0.f && fabsf(ps) > S.psi_max) bad = true;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) cost += __shfl_xor_sync(FULL, cost, off);
        bad = __any_sync(FULL, bad);
        if (bad || isnan(cost)) cost = __int_as_float(0x7f800000);
        if (lane == 0) S.cost_out[gw] = cost;
        key = ((unsigned long long)__float_as_uint(cost) << 32) | (unsigned)gw;
    }
    if (lane == 0) s_key[warp] = key;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long best = s_key[0];
        for (int w = 1; w < STATIC_WARPS_PER_CTA; ++w) best = s_key[w] < best ? s_key[w] : best;
        S.scratch[1 + blockIdx.x] = best;
        __threadfence();
        const unsigned ticket = atomicAdd(reinterpret_cast<unsigned*>(S.scratch), 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) {  // the last CTA reduces the per-CTA keys
        __threadfence();
        unsigned long long best = ~0ull;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
            const unsigned long long k = *reinterpret_cast<volatile unsigned long long*>(S.scratch + 1 + i);
            best = k < best ? k : best;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(FULL, best, off);
            best = o < best ? o : best;
        }
        if (lane == 0) s_key[warp] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            best = s_key[0];
            for (int w = 1; w < STATIC_WARPS_PER_CTA; ++w) best = s_key[w] < best ? s_key[w] : best;
            const unsigned bits = (unsigned)(best >> 32);
            *S.argmin_out = (bits >= 0x7f800000u) ? -1 : (int)(best & 0xffffffffu);
            atomicExch(reinterpret_cast<unsigned*>(S.scratch), 0u);
        }
    }
}

}  // namespace mmpc

namespace {

std::mutex g_static_mu;
unsigned long long* g_static_ptr[64] = {};  // per device ordinal

int static_fail(const std::string& msg, int code)
{
    mmpc::set_global_error(msg);
    return code;
}

}  // namespace

extern "C" int mmpc_score_static(const mmpc_meta* meta, int N, int n, const float* P, const float* Pd,
                                 const float* coef, int B, float* cost_out, int* argmin_out, void* stream)
{
    using namespace mmpc;
    if (!meta || !P || !Pd || !argmin_out || (B > 0 && (!coef || !cost_out)))
        return static_fail("mmpc_score_static: NULL pointer argument", MMPC_ERR_INVALID_ARG);
    if (!sizes_ok(N, n)) return static_fail("mmpc_score_static: N or n out of the supported range", MMPC_ERR_SHAPE);
    if (B < 0 || B > MMPC_STATIC_SCORE_MAX_B)
        return static_fail("mmpc_score_static: B must be in [0, MMPC_STATIC_SCORE_MAX_B = " +
                               std::to_string(MMPC_STATIC_SCORE_MAX_B) + "]",
                           MMPC_ERR_SHAPE);
    if (meta->kind < MMPC_META_CRUISE || meta->kind > MMPC_META_ABS)
        return static_fail("mmpc_score_static: unknown meta kind", MMPC_ERR_INVALID_ARG);
    if (!(meta->w1 >= 0.f) || !(meta->w2 >= 0.f) || !std::isfinite(meta->w1) || !std::isfinite(meta->w2) ||
        !std::isfinite(meta->v_ref) || !std::isfinite(meta->y_ref) || std::isnan(meta->psi_max))
        return static_fail("mmpc_score_static: meta weights must be finite and >= 0", MMPC_ERR_INVALID_ARG);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(std::string("cudaGetDevice: ") + cudaGetErrorString(e), MMPC_ERR_CUDA);
    if (dev < 0 || dev >= 64) return static_fail("mmpc_score_static: device ordinal >= 64", MMPC_ERR_CUDA);
    unsigned long long* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_ptr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_static_score_scratch);
            if (e != cudaSuccess)
                return static_fail(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e), MMPC_ERR_CUDA);
            g_static_ptr[dev] = static_cast<unsigned long long*>(ptr);
        }
        scratch = g_static_ptr[dev];
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (B == 0) {
        e = cudaMemsetAsync(argmin_out, 0xff, sizeof(int), st);  // -1
        return e == cudaSuccess ? MMPC_OK : static_fail(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e), MMPC_ERR_CUDA);
    }
    e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), st);  // the ticket starts at zero
    if (e != cudaSuccess) return static_fail(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e), MMPC_ERR_CUDA);
    StaticScoreArgs s{};
    s.N = N; s.n = n; s.B = B; s.kind = meta->kind;
    s.w1 = meta->w1; s.w2 = meta->w2; s.v_ref = meta->v_ref; s.y_ref = meta->y_ref; s.psi_max = meta->psi_max;
    s.P = P; s.Pd = Pd; s.coef = coef; s.cost_out = cost_out; s.argmin_out = argmin_out; s.scratch = scratch;
    const int grid = (B + STATIC_WARPS_PER_CTA - 1) / STATIC_WARPS_PER_CTA;
    if (n <= 12) score_static_kernel<12><<<grid, 32 * STATIC_WARPS_PER_CTA, 0, st>>>(s);
    else score_static_kernel<16><<<grid, 32 * STATIC_WARPS_PER_CTA, 0, st>>>(s);
    e = cudaGetLastError();
    return e == cudaSuccess ? MMPC_OK : static_fail(std::string("score_static launch: ") + cudaGetErrorString(e), MMPC_ERR_CUDA);
}

// ---------------------------------------------------------------------------
// Batches of scenes (host side)
// ---------------------------------------------------------------------------
struct mmpc_batch {
    int S = 0, NC = 12, total = 0, threads = 0, grid = 0, schedule = 0;
    size_t smem = 0;
    void* kern = nullptr;
    std::vector<mmpc_scene> scenes;
    std::vector<mmpc::SolveArgs> args;
    std::vector<mmpc::ScoreArgs> sargs;
    mmpc::SolveArgs* d_args = nullptr;
    mmpc::SolveArgs* d_args_cold = nullptr;  // the same with the warm starts removed (fallback)
    mmpc::ScoreArgs* d_sargs = nullptr;
    int2* d_items = nullptr;
    int2* d_fb_items = nullptr;               // fallback list
    int* d_counts = nullptr;                  // [0] items, [1] fallback items, [2 + g] items of group g
    int fallback = 0;  // 0 off, 1 every miss, 2 misses that ran the whole budget, 3 of those the near misses
    float near = 5.f;  // mode 3: a near miss has residual <= near x tol
    // one context of variant 3 for every scene: the solve runs on the
    // tensor-core kernel over items of 32 goals (the fallback stays FP32)
    bool tc = false;     // the batch can run on the tensor-core kernel
    bool use_tc = false;  // and does (schedule 5; 1-4 run the FP32 kernel)
    std::string signature;  // the autotuner's cache key
    int tc_items = 0;
    size_t tc_smem_bytes = 0;
    int4* d_tc_items = nullptr;  // (scene, first position, count, order offset)
    int* d_tc_off = nullptr;     // order offset of each scene
    int* d_tc_order = nullptr;   // [queue | pad to 4 | goal index of each position]
    int* d_tc_fb = nullptr;      // fallback: [queue | pad to 4 | the misses of each scene, in its segment]
    int4* d_tc_fb_items = nullptr;  // fallback: one item per scene
    bool any_warm = false;
    cudaEvent_t timing[4] = {};  // optional: around the solve launch(es) and the fallback launch
    // horizon groups (schedule 4): scenes with the same pair-thread count,
    // one right-sized persistent launch each, on forked streams
    struct Group {
        int threads = 0, grid = 0, total = 0, offset = 0;
        size_t smem = 0;
        void* kern = nullptr;
        cudaStream_t stream = nullptr;
        cudaEvent_t done = nullptr;
    };
    std::vector<Group> groups;
    std::vector<int> scene_threads;
    int2* d_gitems = nullptr;  // all groups' items, group after group
    cudaEvent_t fork = nullptr;
    unsigned long long* d_scratch = nullptr;  // [2 + 2S], laid out as the batch kernels describe
};

namespace {

int batch_fail(const std::string& msg, int code)
{
    mmpc::set_global_error(msg);
    return code;
}

void batch_free(mmpc_batch* b)
{
    if (!b) return;
    cudaFree(b->d_args);
    cudaFree(b->d_args_cold);
    cudaFree(b->d_tc_items);
    cudaFree(b->d_tc_off);
    cudaFree(b->d_tc_order);
    cudaFree(b->d_tc_fb);
    cudaFree(b->d_tc_fb_items);
    cudaFree(b->d_sargs);
    cudaFree(b->d_items);
    cudaFree(b->d_fb_items);
    cudaFree(b->d_counts);
    cudaFree(b->d_scratch);
    cudaFree(b->d_gitems);
    for (auto& g : b->groups) {
        if (g.stream) cudaStreamDestroy(g.stream);
        if (g.done) cudaEventDestroy(g.done);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

// Item order for a schedule: 1 scene by scene in the given order, 2 scenes by
// decreasing work per trajectory (N (m + 32): obstacle-sample pairs plus the
// per-sample work), 3 round-robin over the scenes in the order of 2, one
// trajectory of each at a time.
std::vector<int2> batch_items(const mmpc_batch* b, int schedule)
{
    std::vector<int> order(b->S);
    for (int s = 0; s < b->S; ++s) order[s] = s;
    auto cost = [&](int s) {
        const mmpc_ctx* c = b->scenes[s].ctx;
        return (double)c->p.N * (double)(c->m + 32);
    };
    if (schedule >= 2)
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
    std::vector<int2> items;
    items.reserve(b->total);
    if (schedule == 3) {
        // round-robin over the scenes in decreasing-work order: the longest
        // trajectories start first and every scene progresses from the start
        int maxB = 0;
        for (int s : order) maxB = std::max(maxB, b->scenes[s].B);
        for (int l = 0; l < maxB; ++l)
            for (int s : order)
                if (l < b->scenes[s].B) items.push_back(make_int2(s, l));
    } else {
        for (int s : order)
            for (int l = 0; l < b->scenes[s].B; ++l) items.push_back(make_int2(s, l));
    }
    return items;
}

}  // namespace

namespace {

void* batch_kernel_for(int NC, int threads)
{
    if (NC == 12)
        return threads <= 64 ? (void*)am_solve_batch_kernel<12, 64>
             : threads <= 128 ? (void*)am_solve_batch_kernel<12, 128> : (void*)am_solve_batch_kernel<12, 256>;
    return threads <= 64 ? (void*)am_solve_batch_kernel<16, 64>
         : threads <= 128 ? (void*)am_solve_batch_kernel<16, 128> : (void*)am_solve_batch_kernel<16, 256>;
}

// Work per trajectory of a scene, for ordering: N (m + 32), obstacle-sample
// pairs plus the per-sample work.
double scene_cost(const mmpc_ctx* c) { return (double)c->p.N * (double)(c->m + 32); }

}  // namespace

extern "C" int mmpc_batch_create(const mmpc_scene* scenes, int S, const mmpc_meta* meta, mmpc_batch** out)
{
    using namespace mmpc;
    if (out) *out = nullptr;
    if (!out || !scenes || !meta || S < 1) return batch_fail("mmpc_batch_create: bad arguments", MMPC_ERR_INVALID_ARG);
    if (meta->kind < MMPC_META_CRUISE || meta->kind > MMPC_META_ABS || !(meta->w1 >= 0.f) || !(meta->w2 >= 0.f) ||
        !std::isfinite(meta->w1) || !std::isfinite(meta->w2) || !std::isfinite(meta->v_ref) ||
        !std::isfinite(meta->y_ref) || std::isnan(meta->psi_max))
        return batch_fail("mmpc_batch_create: invalid meta cost", MMPC_ERR_INVALID_ARG);
    mmpc_batch* b = new mmpc_batch();
    b->S = S;
    b->scenes.assign(scenes, scenes + S);
    int max_m = 0, maxN = 0, maxRows = 0;
    for (int s = 0; s < S; ++s) {
        const mmpc_scene& sc = scenes[s];
        const mmpc_ctx* c = sc.ctx;
        if (!c || !c->d_blob) { batch_free(b); return batch_fail("mmpc_batch_create: scene without a set-up context", MMPC_ERR_NOT_SETUP); }
        if (s == 0) b->NC = c->NC;
        if (c->NC != b->NC) { batch_free(b); return batch_fail("mmpc_batch_create: scenes mix n <= 12 and n > 12", MMPC_ERR_SHAPE); }
        if (s == 0) b->tc = c->p.variant == 3;
        if (c->p.precision != MMPC_PREC_FP32 && !(b->tc && c == scenes[0].ctx)) {
            batch_free(b);
            return batch_fail("mmpc_batch_create: precision modes run in batches only as variant 3 with one context "
                              "for every scene", MMPC_ERR_INVALID_ARG);
        }
        if (b->tc && c != scenes[0].ctx) {
            batch_free(b);
            return batch_fail("mmpc_batch_create: a variant 3 batch takes one context for every scene", MMPC_ERR_INVALID_ARG);
        }
        if (b->tc && sc.B > TC_RANK_MAX) {
            batch_free(b);
            return batch_fail("mmpc_batch_create: variant 3 batches take at most 8192 goals per scene", MMPC_ERR_SHAPE);
        }
        if (sc.B < 0 || !sc.ego || (c->m > 0 && !sc.obst) || (sc.B > 0 && (!sc.goals || !sc.coef_out || !sc.cost_out)) || !sc.argmin_out) {
            batch_free(b);
            return batch_fail("mmpc_batch_create: NULL pointer in scene " + std::to_string(s), MMPC_ERR_INVALID_ARG);
        }
        b->total += sc.B;
        max_m = std::max(max_m, c->m);
        maxN = std::max(maxN, c->p.N);
        maxRows = std::max(maxRows, c->L.init);
    }
    const int NP = (maxN + 1) / 2;
    b->threads = 32 * ((NP + 31) / 32);
    b->smem = pair_smem(maxRows, max_m, b->NC, b->threads);
    if (b->smem > 227 * 1024) { batch_free(b); return batch_fail("mmpc_batch_create: scenes do not fit in shared memory", MMPC_ERR_SHAPE); }
    b->kern = batch_kernel_for(b->NC, b->threads);

    // horizon groups: scenes with the same pair-thread count, longest first;
    // inside a group, scenes by decreasing work per trajectory
    b->scene_threads.resize(S);
    std::vector<int> keys;
    for (int s = 0; s < S; ++s) {
        const int np = (scenes[s].ctx->p.N + 1) / 2;
        b->scene_threads[s] = 32 * ((np + 31) / 32);
        if (std::find(keys.begin(), keys.end(), b->scene_threads[s]) == keys.end()) keys.push_back(b->scene_threads[s]);
    }
    std::sort(keys.begin(), keys.end(), std::greater<int>());
    std::vector<int2> gitems;
    for (int th : keys) {
        mmpc_batch::Group g;
        g.threads = th;
        g.offset = (int)gitems.size();
        int gm = 0, grows = 0;
        std::vector<int> ss;
        for (int s = 0; s < S; ++s)
            if (b->scene_threads[s] == th) {
                ss.push_back(s);
                gm = std::max(gm, scenes[s].ctx->m);
                grows = std::max(grows, scenes[s].ctx->L.init);
            }
        std::stable_sort(ss.begin(), ss.end(), [&](int x, int y) { return scene_cost(scenes[x].ctx) > scene_cost(scenes[y].ctx); });
        for (int s : ss)
            for (int l = 0; l < scenes[s].B; ++l) gitems.push_back(make_int2(s, l));
        g.total = (int)gitems.size() - g.offset;
        g.smem = pair_smem(grows, gm, b->NC, th);
        g.kern = batch_kernel_for(b->NC, th);
        b->groups.push_back(g);
    }
    // each kernel's dynamic shared memory attribute covers its largest request
    cudaError_t e = cudaSuccess;
    std::vector<std::pair<void*, size_t>> attrs{{b->kern, b->smem}};
    for (const auto& g : b->groups) {
        bool found = false;
        for (auto& a : attrs)
            if (a.first == g.kern) { a.second = std::max(a.second, g.smem); found = true; }
        if (!found) attrs.push_back({g.kern, g.smem});
    }
    for (const auto& a : attrs)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(a.first, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.second);
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b->kern, b->threads, b->smem);
    for (auto& g : b->groups) {
        int per = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, g.kern, g.threads, g.smem);
        g.grid = std::max(1, std::min(g.total, sms * std::max(per, 1)));
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e != cudaSuccess || per_sm < 1) {
        batch_free(b);
        return batch_fail(std::string("mmpc_batch_create: occupancy query: ") + cudaGetErrorString(e), MMPC_ERR_CUDA);
    }
    b->grid = std::max(1, std::min(b->total, sms * per_sm));

    b->args.resize(S);
    b->sargs.resize(S);
    for (int s = 0; s < S; ++s) {
        const mmpc_scene& sc = scenes[s];
        const mmpc_ctx* c = sc.ctx;
        const mmpc_params& p = c->p;
        SolveArgs& a = b->args[s];
        a = SolveArgs{};
        a.N = p.N; a.n = p.n; a.m = c->m; a.B = sc.B; a.iters = p.iters; a.check_every = p.check_every;
        a.cull = p.cull ? 1 : 0;
        a.rho = (float)p.rho; a.a = (float)p.a; a.b = (float)p.b;
        a.inv_a = (float)(1.0 / p.a); a.inv_b = (float)(1.0 / p.b);
        a.v_min = (float)p.v_min; a.v_max = (float)p.v_max; a.a_max = (float)p.a_max; a.tol = p.tol;
        a.stall_tol = p.stall_tol; a.stall_ratio = p.stall_ratio;
        a.L = c->L;
        a.blob = c->d_blob;
        a.ego = sc.ego; a.obst = sc.obst; a.goals = sc.goals; a.warm_c = sc.warm_coef; a.warm_l = sc.warm_lam;
        if (sc.warm_coef) b->any_warm = true;
        a.coef_out = sc.coef_out; a.lam_out = sc.lam_out; a.resid_out = sc.resid_out; a.iters_out = sc.iters_out;
        a.err_flag = reinterpret_cast<unsigned*>(c->d_scratch + 1) + 1;
        a.work = c->d_scratch + 2;  // counted per scene, read with mmpc_take_work_count
        a.missing_tx = c->debug_missing;
        ScoreArgs& g = b->sargs[s];
        g = ScoreArgs{};
        g.N = p.N; g.n = p.n; g.B = sc.B; g.kind = meta->kind;
        g.w1 = meta->w1; g.w2 = meta->w2; g.v_ref = meta->v_ref; g.y_ref = meta->y_ref; g.psi_max = meta->psi_max;
        g.L = c->L; g.blob = c->d_blob; g.coef = sc.coef_out; g.cost_out = sc.cost_out; g.argmin_out = sc.argmin_out;
    }
    const int G = (int)b->groups.size();
    const size_t nscratch = 2 + 2 * (size_t)S + G;
    std::vector<SolveArgs> cold(b->args);
    for (auto& a : cold) { a.warm_c = nullptr; a.warm_l = nullptr; }
    e = cudaMalloc(&b->d_args, sizeof(SolveArgs) * S);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_args_cold, sizeof(SolveArgs) * S);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sargs, sizeof(ScoreArgs) * S);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(int2) * std::max(1, b->total));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_fb_items, sizeof(int2) * std::max(1, b->total));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counts, sizeof(int) * (2 + G));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_gitems, sizeof(int2) * std::max<size_t>(1, gitems.size()));
    if (e == cudaSuccess && !gitems.empty())
        e = cudaMemcpy(b->d_gitems, gitems.data(), sizeof(int2) * gitems.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_scratch, sizeof(unsigned long long) * nscratch);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_args, b->args.data(), sizeof(SolveArgs) * S, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_args_cold, cold.data(), sizeof(SolveArgs) * S, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        std::vector<int> counts{b->total, 0};
        for (const auto& g : b->groups) counts.push_back(g.total);
        e = cudaMemcpy(b->d_counts, counts.data(), sizeof(int) * counts.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(b->d_sargs, b->sargs.data(), sizeof(ScoreArgs) * S, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_scratch, 0, sizeof(unsigned long long) * nscratch);
    if (e == cudaSuccess && b->tc) {
        // items of 32 goals in each scene's slot order (the order itself is
        // computed on the device by every run, from the current goals)
        // item size: a whole scene when there are enough scenes to keep every
        // sub-partition busy (about 8 items per SM), else blocks of whole warps
        std::vector<int4> items;
        std::vector<int> off(S);
        int o = 0;
        const double target = 8.0 * std::max(1, sms);
        for (int s = 0; s < S; ++s) {
            off[s] = o;
            const int Bs = scenes[s].B;
            const int ks = std::max(1, (int)std::ceil((double)Bs * target / std::max(1, b->total)));
            const int block = 32 * std::max(1, (int)std::ceil((double)Bs / (32.0 * ks)));
            for (int p0 = 0; p0 < Bs; p0 += block) items.push_back(make_int4(s, p0, std::min(block, Bs - p0), o));
            o += Bs;
        }
        b->tc_items = (int)items.size();
        const mmpc_ctx* c = scenes[0].ctx;
        b->tc_smem_bytes = std::max<size_t>(tc_smem(c, c->m), 116 * 1024);
        if (b->tc_smem_bytes > 227 * 1024) {
            batch_free(b);
            return batch_fail("mmpc_batch_create: scenes do not fit in shared memory", MMPC_ERR_SHAPE);
        }
        e = cudaMalloc(&b->d_tc_items, sizeof(int4) * std::max<size_t>(1, items.size()));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_tc_off, sizeof(int) * S);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_tc_order, sizeof(int) * (4 + (size_t)std::max(1, o)));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_tc_fb, sizeof(int) * (4 + (size_t)std::max(1, o)));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_tc_fb_items, sizeof(int4) * S);
        if (e == cudaSuccess && !items.empty())
            e = cudaMemcpy(b->d_tc_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_tc_off, off.data(), sizeof(int) * S, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(tc_kernel_of(c), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->tc_smem_bytes);
    }
    if (e != cudaSuccess) {
        batch_free(b);
        return batch_fail(std::string("mmpc_batch_create: ") + cudaGetErrorString(e), MMPC_ERR_CUDA);
    }
    *out = b;
    {   // the autotuner's key: the shapes of the scenes, in order, and the kernel family
        std::string key = std::to_string(S) + (b->tc ? "/tc" + std::to_string(scenes[0].ctx->p.precision) : "");
        for (int s = 0; s < S; ++s) {
            const mmpc_ctx* c = scenes[s].ctx;
            key += ";" + std::to_string(scenes[s].B) + "," + std::to_string(c->p.N) + "," + std::to_string(c->p.n) +
                   "," + std::to_string(c->m) + "," + std::to_string(scenes[s].warm_coef ? 1 : 0);
        }
        b->signature = key;
    }
    return mmpc_batch_set_schedule(b, b->tc ? 5 : 1);
}

extern "C" int mmpc_batch_set_schedule(mmpc_batch* b, int schedule)
{
    if (!b) return batch_fail("mmpc_batch_set_schedule: NULL batch", MMPC_ERR_NOT_SETUP);
    if (schedule == 5) {
        if (!b->tc)
            return batch_fail("mmpc_batch_set_schedule: schedule 5 needs one context of variant 3 for every scene",
                              MMPC_ERR_INVALID_ARG);
        // the (scene, trajectory) items of scene order still serve the scoring
        std::vector<int2> items = batch_items(b, 1);
        if (b->total > 0) {
            cudaError_t e = cudaMemcpy(b->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return batch_fail(std::string("mmpc_batch_set_schedule: ") + cudaGetErrorString(e), MMPC_ERR_CUDA);
        }
        b->use_tc = true;
        b->schedule = 5;
        return MMPC_OK;
    }
    b->use_tc = false;
    if (schedule < 1 || schedule > 4) return batch_fail("mmpc_batch_set_schedule: schedule must be 1 to 5", MMPC_ERR_INVALID_ARG);
    std::vector<int2> items = batch_items(b, schedule == 4 ? 2 : schedule);
    if (b->total > 0) {
        cudaError_t e = cudaMemcpy(b->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return batch_fail(std::string("mmpc_batch_set_schedule: ") + cudaGetErrorString(e), MMPC_ERR_CUDA);
    }
    b->schedule = schedule;
    return MMPC_OK;
}

extern "C" int mmpc_batch_run(mmpc_batch* b, void* stream)
{
    using namespace mmpc;
    if (!b) return batch_fail("mmpc_batch_run: NULL batch", MMPC_ERR_NOT_SETUP);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int G = (int)b->groups.size();
    batch_reset_kernel<<<1, 256, 0, st>>>(b->d_scratch, b->S, G, b->d_counts + 1);
    if (b->total > 0) {
        if (b->timing[0]) cudaEventRecord(b->timing[0], st);
        using KernT = void (*)(const SolveArgs*, const int2*, const int*, unsigned long long*, unsigned long long*);
        if (b->use_tc) {
            // tensor-core kernel over every scene: each scene's goals ordered
            // (one CTA per scene), then persistent CTAs over the item queue
            const mmpc_ctx* c = b->scenes[0].ctx;
            cudaMemsetAsync(b->d_tc_order, 0, sizeof(int) * 4, st);
            tc_order_rank<<<b->S, 256, 0, st>>>(b->d_args, b->d_tc_off, b->d_tc_order + 4);
            TcArgs T{};
            T.blob = c->d_tc;
            T.L = c->tc;
            T.scenes = b->d_args;
            T.items = b->d_tc_items;
            T.n_items = b->tc_items;
            T.order = b->d_tc_order + 4;
            T.queue = b->d_tc_order;
            int sms = c->sm_count;
            if (sms < 0) {
                int dev = 0;
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            }
            const int grid = std::max(1, std::min(sms, (b->tc_items + 3) / 4));
            using K3 = void (*)(const SolveArgs, const TcArgs);
            reinterpret_cast<K3>(tc_kernel_of(c))<<<grid, TC_THREADS, b->tc_smem_bytes, st>>>(b->args[0], T);
        } else if (b->schedule == 4) {
            // one right-sized persistent launch per horizon group, on forked
            // streams joined back before scoring (capturable in a graph)
            cudaEventRecord(b->fork, st);
            for (int gi = 0; gi < G; ++gi) {
                const auto& g = b->groups[gi];
                cudaStreamWaitEvent(g.stream, b->fork, 0);
                reinterpret_cast<KernT>(g.kern)<<<g.grid, g.threads, g.smem, g.stream>>>(
                    b->d_args, b->d_gitems + g.offset, b->d_counts + 2 + gi, b->d_scratch,
                    b->d_scratch + 2 + 2 * b->S + gi);
                cudaEventRecord(g.done, g.stream);
                cudaStreamWaitEvent(st, g.done, 0);
            }
        } else {
            reinterpret_cast<KernT>(b->kern)<<<b->grid, b->threads, b->smem, st>>>(b->d_args, b->d_items, b->d_counts,
                                                                                b->d_scratch, b->d_scratch);
        }
        if (b->timing[1]) cudaEventRecord(b->timing[1], st);
        if (b->fallback && b->any_warm && b->use_tc && b->fallback != 3) {
            // the misses of each scene, in its slot order, solved again from
            // the cold start on the tensor-core kernel (one item per scene).
            // The near misses of mode 3 (a few per scene) go to the pair
            // kernel below instead: one CTA per trajectory, where a
            // tensor-core item of a few goals would leave most of its
            // sub-partition's 32 lanes idle.
            const mmpc_ctx* c = b->scenes[0].ctx;
            cudaMemsetAsync(b->d_tc_fb, 0, sizeof(int) * 4, st);
            tc_fallback_compact<<<b->S, 256, 0, st>>>(b->d_args, b->d_tc_off, b->d_tc_order + 4, b->fallback, b->near,
                                                     b->d_tc_fb + 4, b->d_tc_fb_items, b->d_counts + 1);
            if (b->timing[2]) cudaEventRecord(b->timing[2], st);
            TcArgs T{};
            T.blob = c->d_tc;
            T.L = c->tc;
            T.scenes = b->d_args_cold;
            T.items = b->d_tc_fb_items;
            T.n_items = b->S;
            T.order = b->d_tc_fb + 4;
            T.queue = b->d_tc_fb;
            int sms = c->sm_count;
            if (sms < 0) {
                int dev = 0;
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            }
            const int grid = std::max(1, std::min(sms, (b->S + 3) / 4));
            using K3 = void (*)(const SolveArgs, const TcArgs);
            SolveArgs a0 = b->args[0];
            a0.warm_c = nullptr;
            a0.warm_l = nullptr;
            reinterpret_cast<K3>(tc_kernel_of(c))<<<grid, TC_THREADS, b->tc_smem_bytes, st>>>(a0, T);
            if (b->timing[3]) cudaEventRecord(b->timing[3], st);
        } else if (b->fallback && b->any_warm) {
            fallback_compact_kernel<<<std::min(1024, (b->total + 255) / 256), 256, 0, st>>>(
                b->d_args, b->d_items, b->total, b->d_fb_items, b->d_counts + 1, b->d_scratch, b->fallback, b->near);
            if (b->timing[2]) cudaEventRecord(b->timing[2], st);
            reinterpret_cast<KernT>(b->kern)<<<b->grid, b->threads, b->smem, st>>>(b->d_args_cold, b->d_fb_items,
                                                                                b->d_counts + 1, b->d_scratch,
                                                                                b->d_scratch);
            if (b->timing[3]) cudaEventRecord(b->timing[3], st);
        }
        const int wpb = 8;
        const int sgrid = (b->total + wpb - 1) / wpb;
        if (b->NC == 12) score_batch_kernel<12><<<sgrid, 32 * wpb, 0, st>>>(b->d_sargs, b->d_items, b->total, b->d_scratch + 2 + b->S);
        else score_batch_kernel<16><<<sgrid, 32 * wpb, 0, st>>>(b->d_sargs, b->d_items, b->total, b->d_scratch + 2 + b->S);
    }
    batch_finish_kernel<<<(b->S + 255) / 256, 256, 0, st>>>(b->d_sargs, b->S, b->d_scratch + 2 + b->S);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MMPC_OK : batch_fail(std::string("mmpc_batch_run: ") + cudaGetErrorString(e), MMPC_ERR_CUDA);
}

extern "C" int mmpc_batch_times(mmpc_batch* b, float* scene_ms, float* makespan_ms)
{
    if (!b) return batch_fail("mmpc_batch_times: NULL batch", MMPC_ERR_NOT_SETUP);
    std::vector<unsigned long long> h(1 + (size_t)b->S);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), b->d_scratch + 1, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return batch_fail(std::string("mmpc_batch_times: ") + cudaGetErrorString(e), MMPC_ERR_CUDA);
    const unsigned long long t0 = h[0];
    float mk = 0.f;
    for (int s = 0; s < b->S; ++s) {
        const float ms = (h[1 + s] >= t0 && h[1 + s] != 0ull) ? (float)((h[1 + s] - t0) * 1e-6) : 0.f;
        if (scene_ms) scene_ms[s] = ms;
        mk = std::max(mk, ms);
    }
    if (makespan_ms) *makespan_ms = mk;
    return MMPC_OK;
}

namespace {
std::mutex g_tune_mu;
std::vector<std::pair<std::string, int>> g_tune_cache;  // batch signature -> chosen schedule
}  // namespace

extern "C" int mmpc_batch_autotune(mmpc_batch* b, void* stream, int* chosen)
{
    if (!b) return batch_fail("mmpc_batch_autotune: NULL batch", MMPC_ERR_NOT_SETUP);
    {   // a batch of the same signature was tuned before: take its choice
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (const auto& kv : g_tune_cache)
            if (kv.first == b->signature) {
                if (chosen) *chosen = kv.second;
                return mmpc_batch_set_schedule(b, kv.second);
            }
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return batch_fail("mmpc_batch_autotune: cudaEventCreate failed", MMPC_ERR_CUDA);
    int best = 1;
    float best_ms = 1e30f;
    int rc = MMPC_OK;
    const int last = b->tc ? 5 : 4;
    for (int sch = 1; sch <= last && rc == MMPC_OK; ++sch) {
        rc = mmpc_batch_set_schedule(b, sch);
        if (rc == MMPC_OK) rc = mmpc_batch_run(b, stream);  // warm-up
        float total = 0.f;
        for (int r = 0; r < 2 && rc == MMPC_OK; ++r) {
            cudaEventRecord(e0, st);
            rc = mmpc_batch_run(b, stream);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            total += ms;
        }
        if (rc == MMPC_OK && total < best_ms) { best_ms = total; best = sch; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MMPC_OK) return rc;
    rc = mmpc_batch_set_schedule(b, best);
    if (chosen) *chosen = best;
    if (rc == MMPC_OK) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache.emplace_back(b->signature, best);
    }
    return rc;
}

extern "C" int mmpc_batch_describe(mmpc_batch* b, int* schedule, int* launches, mmpc_launch_shape* out, int max)
{
    if (!b) return batch_fail("mmpc_batch_describe: NULL batch", MMPC_ERR_NOT_SETUP);
    if (max < 0 || (max > 0 && !out)) return batch_fail("mmpc_batch_describe: bad output array", MMPC_ERR_INVALID_ARG);
    std::vector<mmpc_launch_shape> v;
    if (b->use_tc) {
        int sms = b->scenes[0].ctx->sm_count;
        if (sms < 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaGetLastError();
        }
        v.push_back({1, mmpc::TC_THREADS, std::max(1, std::min(sms, (b->tc_items + 3) / 4)), (int)b->tc_smem_bytes,
                     b->total});
    } else if (b->schedule == 4) {
        for (const auto& g : b->groups) v.push_back({0, g.threads, g.grid, (int)g.smem, g.total});
    } else {
        v.push_back({0, b->threads, b->grid, (int)b->smem, b->total});
    }
    if (schedule) *schedule = b->schedule;
    if (launches) *launches = (int)v.size();
    for (int i = 0; i < std::min(max, (int)v.size()); ++i) out[i] = v[i];
    return MMPC_OK;
}

extern "C" int mmpc_batch_set_fallback(mmpc_batch* b, int on)
{
    if (!b) return batch_fail("mmpc_batch_set_fallback: NULL batch", MMPC_ERR_NOT_SETUP);
    if (on < 0 || on > 3) return batch_fail("mmpc_batch_set_fallback: mode must be 0, 1, 2 or 3", MMPC_ERR_INVALID_ARG);
    b->fallback = on;
    return MMPC_OK;
}

extern "C" int mmpc_batch_set_fallback_near(mmpc_batch* b, float near)
{
    if (!b) return batch_fail("mmpc_batch_set_fallback_near: NULL batch", MMPC_ERR_NOT_SETUP);
    if (!(near >= 1.f) || !std::isfinite(near))
        return batch_fail("mmpc_batch_set_fallback_near: the factor must be finite and >= 1", MMPC_ERR_INVALID_ARG);
    b->near = near;
    return MMPC_OK;
}

extern "C" int mmpc_batch_set_timing(mmpc_batch* b, void* const* events)
{
    if (!b) return batch_fail("mmpc_batch_set_timing: NULL batch", MMPC_ERR_NOT_SETUP);
    for (int i = 0; i < 4; ++i) b->timing[i] = events ? reinterpret_cast<cudaEvent_t>(events[i]) : nullptr;
    return MMPC_OK;
}

extern "C" int mmpc_batch_status(mmpc_batch* b, void* stream)
{
    if (!b) return fail(nullptr, MMPC_ERR_NOT_SETUP, "batch not created");
    bool expired = false;
    for (const mmpc_scene& sc : b->scenes) {
        unsigned word = 0;
        const int rc = take_error_word(sc.ctx, reinterpret_cast<cudaStream_t>(stream), &word);
        if (rc != MMPC_OK) return rc;
        expired = expired || word != 0;
    }
    return expired ? fail(nullptr, MMPC_ERR_TIMEOUT, "a bounded device wait expired (staging of the constants)")
                   : MMPC_OK;
}

extern "C" int mmpc_batch_fallbacks(mmpc_batch* b, int* count)
{
    if (!b || !count) return batch_fail("mmpc_batch_fallbacks: NULL argument", b ? MMPC_ERR_INVALID_ARG : MMPC_ERR_NOT_SETUP);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(count, b->d_counts + 1, sizeof(int), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MMPC_OK : batch_fail(std::string("mmpc_batch_fallbacks: ") + cudaGetErrorString(e), MMPC_ERR_CUDA);
}

extern "C" void mmpc_batch_destroy(mmpc_batch* b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    batch_free(b);
}
