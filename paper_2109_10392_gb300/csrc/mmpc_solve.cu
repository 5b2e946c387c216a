// GB300 (sm_103a) kernels and C ABI of the batch non-holonomic trajectory
// optimizer (Adajania et al., arXiv 2109.10392, Algorithm 1 of Sec. III-E).
//
// Solve kernel: one CTA per trajectory l of the batch, one thread per time
// sample t.  Every quantity that Algorithm 1 carries from one iteration to the
// next for trajectory l -- c_x, c_y, c_psi and lambda_x, lambda_y, lambda_psi
// -- stays on chip (registers of warp 0, broadcast through shared memory) for
// all iterations; the auxiliary variables v, alpha, d, alpha_a, d_a of Eqs.
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
// Device constant blob (FP32), section offsets in floats.  Every section
// starts on a 16-byte boundary; per-coefficient rows are padded to NC.
// ---------------------------------------------------------------------------
struct BlobLayout {
    int P, Pd, Pdd, t, lin, Q, Kxh, Kxl, Kyh, Kyl, Kp11, Kp12, K12x, K12y, C0x, C0y, C0p, total;
};

static BlobLayout blob_layout(int N, int NC)
{
    auto up4 = [](int v) { return (v + 3) & ~3; };
    BlobLayout B{};
    int o = 0;
    B.P = o; o += up4(N * NC);
    B.Pd = o; o += up4(N * NC);
    B.Pdd = o; o += up4(N * NC);
    B.t = o; o += up4(N);
    B.lin = o; o += up4(NC);
    B.Q = o; o += NC * NC;
    B.Kxh = o; o += NC * NC;
    B.Kxl = o; o += NC * NC;
    B.Kyh = o; o += NC * NC;
    B.Kyl = o; o += NC * NC;
    B.Kp11 = o; o += NC * NC;
    B.Kp12 = o; o += NC * 4;
    B.K12x = o; o += NC * 8;
    B.K12y = o; o += NC * 8;
    B.C0x = o; o += NC * 8;
    B.C0y = o; o += NC * 8;
    B.C0p = o; o += NC * 4;
    B.total = up4(o);
    return B;
}

struct SolveArgs {
    int N, n, m, B, iters, check_every;
    float rho, a, b, inv_a, inv_b, v_min, v_max, a_max, tol;
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
template <int C>
__device__ __forceinline__ void reduce_store(float (&v)[C], float* red, int warp, int stride, int lane)
{
    warp_rs<C, 16, C>(v, lane);
    constexpr int K = rs_count(C);
    if (rs_writer(C, lane)) {
        const int base = rs_base(C, lane);
#pragma unroll
        for (int i = 0; i < K; ++i) red[warp * stride + base + i] = v[i];
    }
}

// ---------------------------------------------------------------------------
// TMA bulk copy of the constant blob with a bounded mbarrier wait.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool stage_blob(float* dst, const float* src, int bytes, unsigned long long* mbar,
                                           unsigned* err_flag)
{
    const uint32_t bar = smem_u32(mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(dst)),
            "l"(src), "r"(bytes), "r"(bar)
            : "memory");
    }
    // Bounded wait: a copy that has not landed after ~2^22 polls (well over a
    // second) flags an error, and the CTA waits once more, again bounded,
    // before it gives up, so that it never leaves with the copy in flight
    // unless the second bound also expires.
    uint32_t done = 0;
    for (int pass = 0; pass < 2 && !done; ++pass) {
        for (int it = 0; it < (1 << 22) && !done; ++it) {
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(bar), "r"(0)
                : "memory");
        }
        if (!done && pass == 0 && threadIdx.x == 0) atomicOr(err_flag, ERR_TMA_TIMEOUT);
    }
    return __syncthreads_and(done) != 0;
}

// Dot product of a 16-byte aligned row with NC coefficients in shared memory.
template <int NC>
__device__ __forceinline__ float dot_row(const float* __restrict__ row, const float* __restrict__ c)
{
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NC; k += 4) {
        const float4 r = *reinterpret_cast<const float4*>(row + k);
        const float4 q = *reinterpret_cast<const float4*>(c + k);
        s = fmaf(r.x, q.x, s);
        s = fmaf(r.y, q.y, s);
        s = fmaf(r.z, q.z, s);
        s = fmaf(r.w, q.w, s);
    }
    return s;
}

// Sum over obstacles at one sample (Eq. split_alpha_o): with n = w / (a, b)
// the ellipse-normalised offset of obstacle j and s = max(0, 1/|n| - 1),
// S += n s; the constraint rows of F_o c - g_o at this sample sum to
// (-a Sx, -b Sy).  With RESID the squared residual sum_j |a nx s, b ny s|^2
// is accumulated too.  Two interleaved accumulator pairs for ILP.
template <bool RESID>
__device__ __forceinline__ void obstacle_sum(const float4* __restrict__ obs, int m, float Xn, float Yn, float tt,
                                             float a2, float b2, float& Sx, float& Sy, float& R2)
{
    float sx0 = 0.f, sy0 = 0.f, sx1 = 0.f, sy1 = 0.f, r0 = 0.f, r1 = 0.f;
    int j = 0;
#pragma unroll 2
    for (; j + 1 < m; j += 2) {
        const float4 o0 = obs[j];
        const float4 o1 = obs[j + 1];
        const float nx0 = Xn - fmaf(o0.z, tt, o0.x);
        const float ny0 = Yn - fmaf(o0.w, tt, o0.y);
        const float nx1 = Xn - fmaf(o1.z, tt, o1.x);
        const float ny1 = Yn - fmaf(o1.w, tt, o1.y);
        const float q0 = fmaf(nx0, nx0, ny0 * ny0);
        const float q1 = fmaf(nx1, nx1, ny1 * ny1);
        const float s0 = fmaxf(rsqrtf(q0) - 1.f, 0.f);
        const float s1 = fmaxf(rsqrtf(q1) - 1.f, 0.f);
        sx0 = fmaf(nx0, s0, sx0);
        sy0 = fmaf(ny0, s0, sy0);
        sx1 = fmaf(nx1, s1, sx1);
        sy1 = fmaf(ny1, s1, sy1);
        if (RESID) {
            r0 = fmaf(s0 * s0, fmaf(a2 * nx0, nx0, b2 * ny0 * ny0), r0);
            r1 = fmaf(s1 * s1, fmaf(a2 * nx1, nx1, b2 * ny1 * ny1), r1);
        }
    }
    if (j < m) {
        const float4 o0 = obs[j];
        const float nx0 = Xn - fmaf(o0.z, tt, o0.x);
        const float ny0 = Yn - fmaf(o0.w, tt, o0.y);
        const float q0 = fmaf(nx0, nx0, ny0 * ny0);
        const float s0 = fmaxf(rsqrtf(q0) - 1.f, 0.f);
        sx0 = fmaf(nx0, s0, sx0);
        sy0 = fmaf(ny0, s0, sy0);
        if (RESID) r0 = fmaf(s0 * s0, fmaf(a2 * nx0, nx0, b2 * ny0 * ny0), r0);
    }
    Sx = sx0 + sx1;
    Sy = sy0 + sy1;
    R2 = r0 + r1;
}

// The same sum, slowly, with the degenerate case of an ego sample exactly at
// an obstacle centre (w = 0): there alpha = atan2(0, 0) = 0 and d = 1, so the
// target is xi + (a, 0) and the row of F_o c - g_o is (-a, 0).
__device__ __noinline__ void obstacle_sum_exact(const float4* __restrict__ obs, int m, float Xn, float Yn, float tt,
                                                float a2, float b2, float& Sx, float& Sy, float& R2)
{
    Sx = 0.f;
    Sy = 0.f;
    R2 = 0.f;
    for (int j = 0; j < m; ++j) {
        const float4 o = obs[j];
        const float nx = Xn - fmaf(o.z, tt, o.x);
        const float ny = Yn - fmaf(o.w, tt, o.y);
        const float q = fmaf(nx, nx, ny * ny);
        if (q == 0.f) {
            Sx += 1.f;
            R2 += a2;
        } else {
            const float s = fmaxf(rsqrtf(q) - 1.f, 0.f);
            Sx = fmaf(nx, s, Sx);
            Sy = fmaf(ny, s, Sy);
            R2 = fmaf(s * s, fmaf(a2 * nx, nx, b2 * ny * ny), R2);
        }
    }
}

// ---------------------------------------------------------------------------
// The fused AM kernel.  Grid: one CTA per trajectory; block: 32 ceil(N/32)
// threads, thread t owns sample t.  Warp 0 owns the coefficient state: lane k
// (k < NC) coefficient k of the x axis (and of psi), lane 16 + k coefficient k
// of the y axis.
// ---------------------------------------------------------------------------
template <int NC>
struct SolveSmem {
    static constexpr int VD = 3 * NC + 4;  // values reduced per sample in the projection phase
    static constexpr int RSD = (VD + 3) & ~3;
    static constexpr int RSB = NC;
};

template <int NC, int MAXT>
__global__ void __launch_bounds__(MAXT, (MAXT <= 128) ? 7 : ((MAXT <= 256) ? 3 : 1)) am_solve_kernel(const SolveArgs A)
{
    constexpr int VD = SolveSmem<NC>::VD;
    constexpr int RSD = SolveSmem<NC>::RSD;
    constexpr int RSB = SolveSmem<NC>::RSB;
    extern __shared__ __align__(16) float smem[];
    __shared__ __align__(16) float s_cx[NC];
    __shared__ __align__(16) float s_cy[NC];
    __shared__ __align__(16) float s_cp[NC];
    __shared__ __align__(8) unsigned long long s_mbar;
    __shared__ int s_done;

    const int l = blockIdx.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int N = A.N, m = A.m;
    const BlobLayout& L = A.L;

    float* blob = smem;
    float4* obs = reinterpret_cast<float4*>(smem + L.total);
    float* red = reinterpret_cast<float*>(obs + m);

    // Scene: ego (Sec. III, x0 = 0) and obstacles, normalised by the ellipse
    // axes and expressed in the frame moving with v0 along x.
    const float y0 = __ldg(A.ego + 0), v0 = __ldg(A.ego + 1), psi0 = __ldg(A.ego + 2), acc0 = __ldg(A.ego + 3);
    for (int j = tid; j < m; j += blockDim.x) {
        const float* o = A.obst + 4 * j;
        obs[j] = make_float4(__ldg(o + 0) * A.inv_a, __ldg(o + 1) * A.inv_b, (__ldg(o + 2) - v0) * A.inv_a,
                             __ldg(o + 3) * A.inv_b);
    }
    if (!stage_blob(blob, A.blob, L.total * 4, &s_mbar, A.err_flag)) return;

    const float rho = A.rho;
    const float a2 = A.a * A.a, b2 = A.b * A.b;
    const bool has_t = tid < N;
    const int ts = has_t ? tid : 0;
    const float* Prow = blob + L.P + ts * NC;
    const float* Pdrow = blob + L.Pd + ts * NC;
    const float* Pddrow = blob + L.Pdd + ts * NC;
    const float tt = blob[L.t + ts];

    // ---- warp-0 coefficient state -----------------------------------------
    const bool isy = lane >= 16;
    const int k = lane & 15;
    const bool act = k < NC && warp == 0;
    const int kk = k < NC ? k : 0;
    const int gbase = lane & 16;
    float c = 0.f, e = 0.f, lam = 0.f, u = 0.f, lampsi = 0.f, cbp = 0.f, corr = 0.f;

    if (warp == 0) {
        const float* g = A.goals + 3 * l;
        const float yg = __ldg(g + 0), vg = __ldg(g + 1), ag = __ldg(g + 2);
        float cpsi, spsi;
        sincosf(psi0, &spsi, &cpsi);
        // boundary values (see mmpc.h), x relative to v0 t
        float bx[5] = {0.f, v0 * cpsi - v0, acc0 * cpsi, vg - v0, ag};
        float by[6] = {y0, v0 * spsi, acc0 * spsi, yg, 0.f, 0.f};
        float bp[4] = {psi0, 0.f, 0.f, 0.f};
        const int nb = isy ? 6 : 5;
        const float* bb = isy ? by : bx;
        if (A.warm_c) {
            c = act && k < A.n ? __ldg(A.warm_c + (size_t)l * 3 * A.n + (isy ? A.n : 0) + k) : 0.f;
            if (!isy && act && k < A.n) c -= v0 * blob[L.lin + k];
        } else {
            const float* C0 = blob + (isy ? L.C0y : L.C0x) + kk * 8;
            float s = 0.f;
            for (int r = 0; r < nb; ++r) s = fmaf(C0[r], bb[r], s);
            c = act ? s : 0.f;
        }
        // K12 (b - A c^0): zero for an exact cold start.  Eq. lin_solve_xy_2
        // from any c^0 equals c^0 + K12 (b - A c^0) + K11 u^0 with u^0 taken at
        // c^0 itself, so this term is added by the first step (the
        // auxiliaries of iterate 0 are those of the start as given).
        {
            const float* rows[6];
            if (!isy) {
                rows[0] = blob + L.P; rows[1] = blob + L.Pd; rows[2] = blob + L.Pdd;
                rows[3] = blob + L.Pd + (N - 1) * NC; rows[4] = blob + L.Pdd + (N - 1) * NC; rows[5] = rows[4];
            } else {
                rows[0] = blob + L.P; rows[1] = blob + L.Pd; rows[2] = blob + L.Pdd;
                rows[3] = blob + L.P + (N - 1) * NC; rows[4] = blob + L.Pd + (N - 1) * NC;
                rows[5] = blob + L.Pdd + (N - 1) * NC;
            }
            const float* K12 = blob + (isy ? L.K12y : L.K12x) + kk * 8;
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                float ac = act ? rows[r][kk] * c : 0.f;  // A_r c, summed over the 16 lanes of the axis group
                ac += __shfl_xor_sync(FULL, ac, 8);
                ac += __shfl_xor_sync(FULL, ac, 4);
                ac += __shfl_xor_sync(FULL, ac, 2);
                ac += __shfl_xor_sync(FULL, ac, 1);
                if (r < nb) corr = fmaf(K12[r], bb[r] - ac, corr);
            }
            if (!act) corr = 0.f;
        }
        if (!isy) {
            const float* Kp12 = blob + L.Kp12 + kk * 4;
            float s = 0.f;
            for (int r = 0; r < 4; ++r) s = fmaf(Kp12[r], bp[r], s);
            cbp = act ? s : 0.f;
        }
        float cp0 = 0.f;
        if (!isy && act) {
            if (A.warm_c) {
                cp0 = k < A.n ? __ldg(A.warm_c + (size_t)l * 3 * A.n + 2 * A.n + k) : 0.f;
            } else {
                const float* C0 = blob + L.C0p + kk * 4;
                for (int r = 0; r < 4; ++r) cp0 = fmaf(C0[r], bp[r], cp0);
            }
        }
        if (A.warm_l && act && k < A.n) {
            lam = __ldg(A.warm_l + (size_t)l * 3 * A.n + (isy ? A.n : 0) + k);
            if (!isy) lampsi = __ldg(A.warm_l + (size_t)l * 3 * A.n + 2 * A.n + k);
        }
        if (act) {
            (isy ? s_cy : s_cx)[k] = c;
            if (!isy) s_cp[k] = cp0;
        }
        if (lane == 0) s_done = 0;
    }
    __syncthreads();

    float xd = 0.f, yd = 0.f, theta = 0.f;
    float rsum[4] = {0.f, 0.f, 0.f, 0.f};
    int kit = 0;
    const int iters = A.iters;

    // Projection phase: Eqs. split_v, split_alpha_o, split_alpha_a at the
    // current coefficients, then the per-warp partial sums of F^T (F c - g),
    // P^T (P c_psi - theta) and the squared residuals.
    auto project = [&](bool resid) {
        float v[VD];
#pragma unroll
        for (int i = 0; i < VD; ++i) v[i] = 0.f;
        if (has_t) {
            const float x = dot_row<NC>(Prow, s_cx);
            const float y = dot_row<NC>(Prow, s_cy);
            const float xdd = dot_row<NC>(Pddrow, s_cx);
            const float ydd = dot_row<NC>(Pddrow, s_cy);
            const float ps = dot_row<NC>(Prow, s_cp);
            // Eq. v_update and the non-holonomic rows v (cos psi, sin psi)
            const float spd = sqrtf(fmaf(xd, xd, yd * yd));
            const float vel = fminf(fmaxf(spd, A.v_min), A.v_max);
            float sn, cs;
            sincosf(ps, &sn, &cs);
            const float evx = fmaf(-vel, cs, xd);
            const float evy = fmaf(-vel, sn, yd);
            // Eq. split_alpha_a: projection of (xddot, yddot) on the disk of radius a_max
            const float an2 = fmaf(xdd, xdd, ydd * ydd);
            const float sc = fminf(1.f, A.a_max * rsqrtf(an2));
            const float eax = xdd * (1.f - sc);
            const float eay = ydd * (1.f - sc);
            // Eq. split_alpha_o, summed over the obstacles
            float Sx, Sy, R2;
            const float Xn = x * A.inv_a, Yn = y * A.inv_b;
            if (resid) obstacle_sum<true>(obs, m, Xn, Yn, tt, a2, b2, Sx, Sy, R2);
            else obstacle_sum<false>(obs, m, Xn, Yn, tt, a2, b2, Sx, Sy, R2);
            if (isnan(Sx) || isnan(Sy)) obstacle_sum_exact(obs, m, Xn, Yn, tt, a2, b2, Sx, Sy, R2);
            const float eox = -A.a * Sx;
            const float eoy = -A.b * Sy;
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
                v[3 * NC + 0] = R2;
                v[3 * NC + 1] = fmaf(eax, eax, eay * eay);
                v[3 * NC + 2] = fmaf(evx, evx, evy * evy);
                v[3 * NC + 3] = dpsi * dpsi;
            }
        }
        reduce_store<VD>(v, red, warp, RSD, lane);
    };

    // Velocity directions and the heading target theta = atan2(ydot, xdot)
    // (Eq. split_psi), and the partial sums of P^T theta.
    auto heading = [&](bool reduce) {
        if (has_t) {
            xd = dot_row<NC>(Pdrow, s_cx) + v0;
            yd = dot_row<NC>(Pdrow, s_cy);
            theta = atan2f(yd, xd);
        }
        if (reduce) {
            float v[NC];
#pragma unroll
            for (int q = 0; q < NC; q += 4) {
                const float4 p4 = *reinterpret_cast<const float4*>(Prow + q);
                v[q + 0] = has_t ? p4.x * theta : 0.f;
                v[q + 1] = has_t ? p4.y * theta : 0.f;
                v[q + 2] = has_t ? p4.z * theta : 0.f;
                v[q + 3] = has_t ? p4.w * theta : 0.f;
            }
            reduce_store<NC>(v, red, warp, RSB, lane);
        }
    };

    // Warp 0 after a projection phase: multiplier update (Sec. III-E,
    // "Multiplier Update") unless `first`, the increment u = lambda - Q c -
    // rho F^T (F c - g), residual check; then step (split_xy) if not done.
    auto finish = [&](bool first, bool check) {
        float ftd = 0.f, pd = 0.f;
        for (int w = 0; w < nwarps; ++w) {
            ftd += red[w * RSD + (isy ? NC : 0) + kk];
            pd += red[w * RSD + 2 * NC + kk];
        }
        if (check) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float s = 0.f;
                for (int w = 0; w < nwarps; ++w) s += red[w * RSD + 3 * NC + r];
                rsum[r] = s;
            }
        }
        if (!first && act) {
            lam = fmaf(-rho, ftd, lam);
            if (!isy) lampsi = fmaf(-rho, pd, lampsi);
        }
        const float* Qrow = blob + L.Q + kk * NC;
        float qc = 0.f;
#pragma unroll
        for (int j = 0; j < NC; ++j) qc = fmaf(Qrow[j], __shfl_sync(FULL, c, gbase + j), qc);
        u = act ? (lam - qc - rho * ftd) : 0.f;
        bool done = kit >= iters;
        if (!first && check && A.tol > 0.f && kit % A.check_every == 0) {
            const float conv = fmaxf(sqrtf(rsum[0]), fmaxf(sqrtf(rsum[1]), sqrtf(rsum[2])));
            done = done || conv <= A.tol;
        }
        if (!done) {
            // Eq. lin_solve_xy_2 in increment form, K11 applied as hi + lo
            const float* Kh = blob + (isy ? L.Kyh : L.Kxh) + kk * NC;
            const float* Kl = blob + (isy ? L.Kyl : L.Kxl) + kk * NC;
            float d0 = 0.f, d1 = 0.f;
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                const float uj = __shfl_sync(FULL, u, gbase + j);
                d0 = fmaf(Kh[j], uj, d0);
                d1 = fmaf(Kl[j], uj, d1);
            }
            if (act) {
                const float dd = (d0 + d1) + (first ? e + corr : e);
                const float s = c + dd;
                e = dd - (s - c);
                c = s;
                (isy ? s_cy : s_cx)[k] = c;
            }
        }
        if (lane == 0) s_done = done ? 1 : 0;
    };

    // ---- initial iterate: auxiliaries of c^0, no multiplier update -------
    heading(false);
    project(true);
    __syncthreads();
    if (warp == 0) finish(true, true);
    __syncthreads();

    // ---- Algorithm 1 ---------------------------------------------------------
    while (!*reinterpret_cast<volatile int*>(&s_done)) {
        ++kit;
        const bool check = (kit % A.check_every == 0) || kit >= iters;
        // Eq. split_psi: theta and P^T theta
        heading(true);
        __syncthreads();
        if (warp == 0 && !isy) {
            float pth = 0.f;
            for (int w = 0; w < nwarps; ++w) pth += red[w * RSB + kk];
            const float r = fmaf(rho, pth, lampsi);
            const float* Kp = blob + L.Kp11 + kk * NC;
            float cp = cbp;
#pragma unroll
            for (int j = 0; j < NC; ++j) cp = fmaf(Kp[j], __shfl_sync(0x0000ffffu, r, j), cp);
            if (act) s_cp[k] = cp;
        }
        __syncthreads();
        // Eqs. split_v, split_alpha_o, split_alpha_a and the partial sums
        project(check);
        __syncthreads();
        // multipliers, residual check and the next step (split_xy)
        if (warp == 0) finish(false, check);
        __syncthreads();
    }

    // ---- outputs -------------------------------------------------------------
    if (warp == 0) {
        const int n = A.n;
        const size_t o = (size_t)l * 3 * n;
        if (act && k < n) {
            if (!isy) {
                A.coef_out[o + k] = (c + e) + v0 * blob[L.lin + k];
                A.coef_out[o + 2 * n + k] = s_cp[k];
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
}

// ---------------------------------------------------------------------------
// Meta cost (Sec. III-F) and batch argmin.  One warp per trajectory, lanes
// over samples; the argmin is a packed 64-bit atomicMin of (cost bits << 32 |
// index) -- costs are non-negative, so their bit patterns order like the
// values -- finished by the last CTA, which also resets the scratch words.
// ---------------------------------------------------------------------------
template <int NC>
__global__ void __launch_bounds__(256) score_kernel(const ScoreArgs S)
{
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
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
        if (lane == 0) {
            S.cost_out[gw] = cost;
            const unsigned long long key = ((unsigned long long)__float_as_uint(cost) << 32) | (unsigned)gw;
            atomicMin(S.best, key);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(S.ticket, 1u);
        if (ticket == gridDim.x - 1) {
            __threadfence();
            const unsigned long long key = atomicAdd(S.best, 0ull);
            const unsigned bits = (unsigned)(key >> 32);
            *S.argmin_out = (bits >= 0x7f800000u) ? -1 : (int)(key & 0xffffffffu);
            atomicExch(S.best, ~0ull);
            atomicExch(S.ticket, 0u);
        }
    }
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
    unsigned long long* d_scratch = nullptr;  // [0] packed argmin key, [1] low: ticket, high: error flags
    std::string err = "no error";
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

template <int NC, int MAXT>
int launch_solve_t(mmpc_ctx* ctx, const SolveArgs& a, int threads, size_t smem, cudaStream_t st)
{
    auto kern = am_solve_kernel<NC, MAXT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
    kern<<<a.B, threads, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "solve launch");
    return MMPC_OK;
}

template <int NC>
int launch_solve_nc(mmpc_ctx* ctx, const SolveArgs& a, int threads, size_t smem, cudaStream_t st)
{
    if (threads <= 128) return launch_solve_t<NC, 128>(ctx, a, threads, smem, st);
    if (threads <= 256) return launch_solve_t<NC, 256>(ctx, a, threads, smem, st);
    return launch_solve_t<NC, 512>(ctx, a, threads, smem, st);
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

    const int NC = n <= 12 ? 12 : 16;
    const BlobLayout L = blob_layout(N, NC);
    std::vector<float> h(L.total, 0.f);
    auto mat = [&](size_t src, int dst, int rows, int cols, int dcols, bool lo) {
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c) {
                const double v = buf[src + (size_t)r * cols + c];
                const float hi = (float)v;
                h[dst + r * dcols + c] = lo ? (float)(v - (double)hi) : hi;
            }
    };
    mat(PL.P, L.P, N, n, NC, false);
    mat(PL.Pd, L.Pd, N, n, NC, false);
    mat(PL.Pdd, L.Pdd, N, n, NC, false);
    mat(PL.t, L.t, 1, N, N, false);
    mat(PL.lin, L.lin, 1, n, n, false);
    mat(PL.Q, L.Q, n, n, NC, false);
    mat(PL.K11x, L.Kxh, n, n, NC, false);
    mat(PL.K11x, L.Kxl, n, n, NC, true);
    mat(PL.K11y, L.Kyh, n, n, NC, false);
    mat(PL.K11y, L.Kyl, n, n, NC, true);
    mat(PL.K11p, L.Kp11, n, n, NC, false);
    mat(PL.K12p, L.Kp12, n, MMPC_NEQ_PSI, 4, false);
    mat(PL.K12x, L.K12x, n, MMPC_NEQ_X, 8, false);
    mat(PL.K12y, L.K12y, n, MMPC_NEQ_Y, 8, false);
    mat(PL.C0x, L.C0x, n, MMPC_NEQ_X, 8, false);
    mat(PL.C0y, L.C0y, n, MMPC_NEQ_Y, 8, false);
    mat(PL.C0p, L.C0p, n, MMPC_NEQ_PSI, 4, false);

    mmpc_ctx* ctx = new mmpc_ctx();
    ctx->p = *p;
    ctx->m = m;
    ctx->NC = NC;
    ctx->L = L;
    cudaError_t e = cudaMalloc(&ctx->d_blob, sizeof(float) * L.total);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_scratch, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(ctx->d_blob, h.data(), sizeof(float) * L.total, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const unsigned long long init[2] = {~0ull, 0ull};
        e = cudaMemcpy(ctx->d_scratch, init, sizeof(init), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        std::string msg = std::string("mmpc_setup: ") + cudaGetErrorString(e);
        cudaFree(ctx->d_blob);
        cudaFree(ctx->d_scratch);
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
    a.L = ctx->L;
    a.blob = ctx->d_blob;
    a.ego = ego; a.obst = obst; a.goals = goals; a.warm_c = warm_coef; a.warm_l = warm_lam;
    a.coef_out = coef_out; a.lam_out = lam_out; a.resid_out = resid_out; a.iters_out = iters_out;
    a.err_flag = reinterpret_cast<unsigned*>(ctx->d_scratch + 1) + 1;
    const int threads = 32 * ((p.N + 31) / 32);
    const int nw = threads / 32;
    const int RSD = ctx->NC == 12 ? SolveSmem<12>::RSD : SolveSmem<16>::RSD;
    const size_t smem = sizeof(float) * (size_t)ctx->L.total + 16 * (size_t)m + sizeof(float) * (size_t)nw * RSD;
    if (smem > 227 * 1024) return fail(ctx, MMPC_ERR_SHAPE, "scene does not fit in shared memory");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    return ctx->NC == 12 ? launch_solve_nc<12>(ctx, a, threads, smem, st) : launch_solve_nc<16>(ctx, a, threads, smem, st);
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

extern "C" void mmpc_destroy(mmpc_ctx* ctx)
{
    if (!ctx) return;
    cudaDeviceSynchronize();
    cudaFree(ctx->d_blob);
    cudaFree(ctx->d_scratch);
    delete ctx;
}

extern "C" const char* mmpc_last_error(const mmpc_ctx* ctx)
{
    if (ctx) return ctx->err.c_str();
    return mmpc::g_error.c_str();
}

extern "C" int mmpc_version(void) { return 1; }

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
