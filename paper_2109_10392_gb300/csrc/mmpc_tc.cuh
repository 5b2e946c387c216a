// Trajectory-tiled tensor-core form of Algorithm 1 (Sec. III-E) for large
// batches: the shared-matrix products -- the evaluations P c of x, y, psi and
// their derivatives (Eq. param) and the contractions P^T e of Eqs.
// lin_solve_xy_2 / lin_solve_psi_2 -- run as tcgen05.mma on the tensor
// cores, in TF32 (kind::tf32) or BF16 (kind::f16) with FP32 accumulation in
// tensor memory, optionally as hi + lo splits; the projections of Eqs.
// split_v, split_alpha_o, split_alpha_a, the QP increments (K11 as FP32
// hi + lo) and the multipliers stay FP32 on the CUDA cores.
//
// One CTA holds a tile of up to 128 trajectories of one scene: tensor-memory
// lane t is trajectory slot t for every matrix.
//  * Evaluation, per chunk of 16 samples and channel (x, y, psi, xdot, ydot,
//    xddot, yddot): D[t][s] = sum_k C[t][k] B[k][s], M = 128 trajectories,
//    N = 16 samples, K = 16 coefficients; A = the coefficient rows C in
//    tensor memory (written by the thread that owns the trajectory's axis),
//    B = the basis block (P, Pdot or Pddot) from shared memory.
//  * Contraction: D[t][k] += sum_s E[t][s] B[s][k], N = 16 coefficients,
//    K = the chunk's samples; A = the residual rows E written in place over
//    the evaluated chunk in tensor memory, B = the transposed basis block.
//    The three blocks of F^T (F c - g) per axis (obstacles with P,
//    non-holonomic with Pdot, acceleration with Pddot) accumulate into one
//    16-column accumulator, so no reduction over samples runs on the CUDA
//    cores.
// Threads: three groups of four warps; group g owns axis g (x, y, psi) for the
// QP steps and processes the chunks c with c % 3 == g, one thread per
// trajectory (warp 4 g + q serves lanes 32 q .. 32 q + 31, the tensor-memory
// sub-partition it may access).  Per round of three chunks one thread issues
// the evaluation MMAs and commits them to an mbarrier; the groups read their
// chunk (tcgen05.ld), project every sample on the CUDA cores and write the
// residuals back (tcgen05.st); after a CTA barrier the same thread issues
// the contraction MMAs.  tcgen05.mma from one thread execute in issue order,
// so the next round's evaluations never overwrite residuals not yet read.
//
// Tensor memory (512 columns, 32-bit): [0, 64) the contraction accumulators
// (x, y, psi - theta, theta), [64, 160) the coefficient operands (axis x, y,
// psi; hi, lo), [160, 496) three chunk buffers of 7 channels x 16 samples.

// Precision of the tensor-core operands (MMPC_PREC_*): element size and the
// K extent of one MMA (32 bytes of K).
template <int PREC>
struct TcType {
    static constexpr bool BF16 = PREC == MMPC_PREC_BF16 || PREC == MMPC_PREC_BF16_SPLIT;
    static constexpr bool SPLIT = PREC == MMPC_PREC_TF32_SPLIT || PREC == MMPC_PREC_BF16_SPLIT;
    static constexpr int ESZ = BF16 ? 2 : 4;       // bytes per element
    static constexpr int PER = 16 / ESZ;            // elements per 16-byte core row
    static constexpr int KMMA = 2 * PER;            // K of one MMA (two core-row groups)
    static constexpr int KSTEPS = 16 / KMMA;        // MMAs over the 16 coefficients
    static constexpr int CSTEPS = 16 / KMMA;        // MMAs over a chunk of 16 samples
    static constexpr int PARTS = SPLIT ? 2 : 1;     // hi (+ lo)
    static constexpr int ACOLS = BF16 ? 8 : 16;     // tensor-memory columns of 16 coefficients
    static constexpr uint32_t FMT = BF16 ? 1u : 2u; // instruction-descriptor operand format
};

constexpr int TC_THREADS = 384;
constexpr int TC_GROUPS = 3;
constexpr int TC_CS = 16;         // samples per chunk
constexpr int TC_CH = 7;          // channels per chunk
constexpr uint32_t TC_COLS = 512; // tensor-memory allocation
constexpr uint32_t TC_DC = 0;     // contraction accumulators: x, y, psi - theta, theta (16 columns each)
constexpr uint32_t TC_AC = 64;    // coefficient operands
constexpr uint32_t TC_BUF = 160;  // round buffer: 7 channels x TC_RW columns
constexpr int TC_RW = 48;         // columns per channel: the three chunks of a round
constexpr int TC_MAX_M = 128;     // obstacles

// Layout of the tensor-core constant blob (bytes): per basis block (P, Pdot,
// Pddot) and part (hi, lo) the evaluation operand EB (16 coefficients x NSP
// samples, K-major over the coefficients: element (k, s) at
// (k / PER) NSP 16 + 16 s + (k % PER) ESZ) and the contraction operand CB
// (NSP samples x 16 coefficients, K-major over the samples: element (s, k) at
// (s / PER) 256 + 16 k + (s % PER) ESZ).  NSP = N rounded up to 16; rows of
// samples >= N and of coefficients >= n are zero.
struct TcLayout {
    int NSP, esz, parts;
    int eb[3][2], cb[3][2];
    int bytes;
};

static TcLayout tc_layout(int N, int esz, int parts)
{
    TcLayout T{};
    T.NSP = (N + TC_CS - 1) / TC_CS * TC_CS;
    T.esz = esz;
    T.parts = parts;
    const int blk = T.NSP * 16 * esz;
    int o = 0;
    for (int b = 0; b < 3; ++b)
        for (int p = 0; p < parts; ++p) {
            T.eb[b][p] = o; o += blk;
            T.cb[b][p] = o; o += blk;
        }
    for (int b = 0; b < 3; ++b)
        for (int p = parts; p < 2; ++p) { T.eb[b][p] = T.eb[b][0]; T.cb[b][p] = T.cb[b][0]; }
    T.bytes = o;
    return T;
}

// Work of the persistent kernel: items of up to 32 trajectories of one scene
// (one warp's lanes), taken from a queue.  An item is (scene, first position
// in the scene's slot order, count, offset of the scene's order entries).
struct TcArgs {
    const unsigned char* blob;  // device, tc_layout bytes
    TcLayout L;
    const SolveArgs* scenes;    // per-scene arguments (device), or NULL: one scene, the kernel's own
    const int4* items;          // device, or NULL: one scene, items of 32 consecutive positions
    int n_items;
    const int* order;           // goal index (within its scene) of each position
    int* queue;                 // item counter, zero at the launch
};

// Slot order: trajectories with similar goals share a warp, so that the
// warp's culling box (the union over its 32 trajectories) stays tight.  A
// counting sort over buckets of the goal's terminal lateral offset (0.5 m
// bins over [-8, 8) m) and speed (0.5 m/s bins over [0, 32) m/s); the order
// inside a bucket is arbitrary.  Each trajectory's arithmetic is independent
// of its slot (the MMA rows are independent, and culling only skips exact
// zero terms), so the order changes no result.
constexpr int TC_YBINS = 32, TC_VBINS = 64, TC_BUCKETS = TC_YBINS * TC_VBINS;

__device__ __forceinline__ int tc_bucket(const float* __restrict__ goal)
{
    const float y = __ldg(goal + 0), v = __ldg(goal + 1);
    const float fy = (y + 8.f) * 2.f, fv = v * 2.f;
    const int by = fy >= 0.f ? min(TC_YBINS - 1, (int)fy) : 0;  // NaN -> 0
    const int bv = fv >= 0.f ? min(TC_VBINS - 1, (int)fv) : 0;
    return by * TC_VBINS + bv;
}

__global__ void tc_order_count(const float* __restrict__ goals, int B, int* __restrict__ count)
{
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < B; l += gridDim.x * blockDim.x)
        atomicAdd(count + tc_bucket(goals + 3 * l), 1);
}

// exclusive scan of the bucket counts in place (one CTA of 1024 threads)
__global__ void __launch_bounds__(1024) tc_order_scan(int* __restrict__ count)
{
    __shared__ int part[1024];
    const int t = threadIdx.x;
    constexpr int PER = TC_BUCKETS / 1024;
    int v[PER], sum = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        v[i] = count[t * PER + i];
        sum += v[i];
    }
    part[t] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int add = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += add;
        __syncthreads();
    }
    int run = part[t] - sum;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        count[t * PER + i] = run;
        run += v[i];
    }
}

__global__ void tc_order_scatter(const float* __restrict__ goals, int B, int* __restrict__ next, int* __restrict__ order)
{
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < B; l += gridDim.x * blockDim.x)
        order[atomicAdd(next + tc_bucket(goals + 3 * l), 1)] = l;
}

// Misses of a warm-started scene for the cold fallback on the tensor cores
// (one CTA per scene): the trajectories whose convergence residual missed
// tol (or is NaN), as selected by the fallback mode (fallback_takes) --
// written in the scene's slot order to its segment of `list`, and the
// scene's item (scene, 0, count, segment offset); counts added to *total.
__global__ void __launch_bounds__(256) tc_fallback_compact(const SolveArgs* __restrict__ sc,
                                                           const int* __restrict__ scene_off,
                                                           const int* __restrict__ order, int mode, float near,
                                                           int* __restrict__ list, int4* __restrict__ items,
                                                           int* __restrict__ total)
{
    __shared__ int warp_cnt[8];
    __shared__ int base;
    const SolveArgs& A = sc[blockIdx.x];
    const int off = scene_off[blockIdx.x];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const bool warm = A.warm_c && A.resid_out && A.tol > 0.f;
    for (int p0 = 0; p0 < A.B; p0 += 256) {
        const int pp = p0 + threadIdx.x;
        const int i = pp < A.B ? order[off + pp] : 0;  // in the scene's slot order
        bool miss = false;
        if (warm && pp < A.B) {
            const float* r = A.resid_out + (size_t)i * 4;
            const bool nan = isnan(r[0]) || isnan(r[1]) || isnan(r[2]);
            const float conv = fmaxf(fmaxf(r[0], r[1]), r[2]);
            miss = fallback_takes(mode, near, nan, conv, A.tol, A.iters_out ? A.iters_out[i] : A.iters, A.iters);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, miss);
        if (lane == 0) warp_cnt[w] = __popc(bal);
        __syncthreads();
        int before = base;
        for (int v = 0; v < w; ++v) before += warp_cnt[v];
        if (miss) list[off + before + __popc(bal & ((1u << lane) - 1u))] = i;
        __syncthreads();
        if (threadIdx.x == 0) {
            int add = 0;
            for (int v = 0; v < 8; ++v) add += warp_cnt[v];
            base += add;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        items[blockIdx.x] = make_int4(blockIdx.x, 0, base, off);
        if (base) atomicAdd(total, base);
    }
}

// The same order for every scene of a batch (one CTA per scene, at most
// TC_RANK_MAX goals): goal i goes to position rank(i) = #{j : (bucket_j, j) <
// (bucket_i, i)}, a stable, deterministic sort.
constexpr int TC_RANK_MAX = 8192;

__global__ void __launch_bounds__(256) tc_order_rank(const SolveArgs* __restrict__ sc, const int* __restrict__ scene_off,
                                                     int* __restrict__ order)
{
    __shared__ short key[TC_RANK_MAX];
    const SolveArgs& A = sc[blockIdx.x];
    const int B = A.B;
    const int off = scene_off[blockIdx.x];
    for (int i = threadIdx.x; i < B; i += blockDim.x) key[i] = (short)tc_bucket(A.goals + 3 * i);
    __syncthreads();
    for (int i = threadIdx.x; i < B; i += blockDim.x) {
        const int ki = key[i];
        int r = 0;
        for (int j = 0; j < B; ++j) {
            const int kj = key[j];
            r += (kj < ki || (kj == ki && j < i)) ? 1 : 0;
        }
        order[off + r] = i;
    }
}

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    // shared-memory matrix descriptor: start, leading (K) and stride (8-row)
    // byte offsets in 16-byte units, descriptor version 1, no swizzle
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// tcgen05.mma with A in tensor memory: D (+)= A B
template <bool BF16>
__device__ __forceinline__ void tc_mma(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    if (BF16)
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
                     "r"(a), "l"(b), "r"(idesc), "r"(acc)
                     : "memory");
    else
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
                     "r"(a), "l"(b), "r"(idesc), "r"(acc)
                     : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 8 or 16 consecutive 32-bit columns (warp-collective).  The
// wait is inside the same asm statement, so no use of the loaded registers
// can be scheduled before the load has completed.
__device__ __forceinline__ void tc_ld8(uint32_t addr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_ld16(uint32_t addr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(addr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Two consecutive columns of each of the 7 channels of a round buffer slot
// (channel stride TC_RW columns), one wait for all seven loads.
__device__ __forceinline__ void tc_ld7x2(uint32_t addr, float (&v)[TC_CH][2])
{
    uint32_t r[14];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%14];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%2, %3}, [%15];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4, %5}, [%16];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%6, %7}, [%17];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%8, %9}, [%18];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%10, %11}, [%19];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%12, %13}, [%20];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13])
                 : "r"(addr), "r"(addr + TC_RW), "r"(addr + 2 * TC_RW), "r"(addr + 3 * TC_RW), "r"(addr + 4 * TC_RW),
                   "r"(addr + 5 * TC_RW), "r"(addr + 6 * TC_RW)
                 : "memory");
#pragma unroll
    for (int ch = 0; ch < TC_CH; ++ch) {
        v[ch][0] = __uint_as_float(r[2 * ch]);
        v[ch][1] = __uint_as_float(r[2 * ch + 1]);
    }
}

// The same loads without the wait, for prefetching: the registers may be
// used only after tc_ld_wait14 on them (whose "+r" operands keep every use
// after the wait).
__device__ __forceinline__ void tc_ld7x2_issue(uint32_t addr, uint32_t (&r)[14])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%14];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%2, %3}, [%15];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4, %5}, [%16];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%6, %7}, [%17];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%8, %9}, [%18];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%10, %11}, [%19];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%12, %13}, [%20];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13])
                 : "r"(addr), "r"(addr + TC_RW), "r"(addr + 2 * TC_RW), "r"(addr + 3 * TC_RW), "r"(addr + 4 * TC_RW),
                   "r"(addr + 5 * TC_RW), "r"(addr + 6 * TC_RW)
                 : "memory");
}

__device__ __forceinline__ void tc_ld_wait14(uint32_t (&r)[14])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13])
                 :
                 : "memory");
}

__device__ __forceinline__ void tc_ld2(uint32_t addr, float (&v)[2])
{
    uint32_t r0, r1;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r0), "=r"(r1)
                 : "r"(addr)
                 : "memory");
    v[0] = __uint_as_float(r0);
    v[1] = __uint_as_float(r1);
}

__device__ __forceinline__ void tc_st1(uint32_t addr, uint32_t r0)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(addr), "r"(r0) : "memory");
}

__device__ __forceinline__ void tc_st2(uint32_t addr, uint32_t r0, uint32_t r1)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(r0), "r"(r1) : "memory");
}

__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tc_st4(uint32_t addr, const uint32_t (&r)[4])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(r[0]), "r"(r[1]),
                 "r"(r[2]), "r"(r[3])
                 : "memory");
}

__device__ __forceinline__ void tc_st8(uint32_t addr, const uint32_t (&r)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(addr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

// Round to TF32 (10-bit significand, to nearest, ties away from zero) -- the
// operand the tensor core takes, so nothing is left to its own truncation.
__device__ __forceinline__ uint32_t tf32_bits(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint32_t bf16_pair(float lo_elem, float hi_elem)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo_elem, hi_elem);
    return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ float bf16_val(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Bounded wait on an mbarrier phase (device global timer, a poll count as a
// backstop); false when it expired.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done = 0;
    const unsigned long long t0 = global_ns();
    for (int it = 0; it < WAIT_MAX_POLLS && !done; ++it) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (!done && (it & 63) == 63 && global_ns() - t0 > WAIT_LIMIT_NS) break;
    }
    return done != 0;
}

// Instruction descriptor: D float32, A and B of the precision's format, both
// K-major, M = 128, N = n_cols.
template <int PREC>
__device__ __forceinline__ uint32_t tc_idesc(int n_cols)
{
    return (1u << 4) | (TcType<PREC>::FMT << 7) | (TcType<PREC>::FMT << 10) | ((uint32_t)(n_cols >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

// Channels of the round buffer: evaluated value (basis block, coefficient
// axis), and, written in place, the residual whose contraction uses the same
// block: 0 x (P, x) -> obstacle x; 1 y (P, y) -> obstacle y; 2 psi (P, psi)
// -> psi - theta; 3 xdot (Pdot, x) -> non-holonomic x (theta in the heading
// phase); 4 ydot (Pdot, y) -> non-holonomic y; 5 xddot (Pddot, x) ->
// acceleration x; 6 yddot (Pddot, y) -> acceleration y.  Each channel holds
// the round's three chunks side by side (TC_RW columns; chunk g of the round
// at column 16 g), so one MMA evaluates a channel for the whole round.
// (block of channel ch: ch < 3 ? P : ch < 5 ? Pdot : Pddot; coefficient axis
// and contraction target: ch < 3 ? ch : (ch - 3) & 1)

// Evaluation MMAs of one round (samples s0 .. s0 + 16 nc - 1) for channels
// [CH0, CH1): D = C B with C = hi (+ lo) coefficient rows, B = the block's
// hi (+ lo) rows; split products a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi.
// The shared-memory descriptors differ only in their start address, so each
// is a constant or'ed with (address >> 4) (addresses stay below 256 KB).
template <int PREC, int CH0, int CH1>
__device__ __forceinline__ void tc_issue_eval(uint32_t tmem, uint32_t sm_base, const TcLayout& L, int s0, int nc)
{
    using TY = TcType<PREC>;
    const uint32_t idesc = tc_idesc<PREC>(TC_CS * nc);
    const uint32_t lbo4 = (uint32_t)L.NSP;  // NSP 16 bytes in 16-byte units
    const uint64_t hi = ((uint64_t)(lbo4 & 0x3FFFu) << 16) | ((uint64_t)(128u >> 4) << 32) | (1ull << 46);
    const uint32_t row4 = (sm_base >> 4) + (uint32_t)s0;  // s0 rows of 16 bytes
#pragma unroll
    for (int ch = CH0; ch < CH1; ++ch) {
        const int blk = ch < 3 ? 0 : (ch < 5 ? 1 : 2), ax = ch < 3 ? ch : ((ch - 3) & 1);
        const uint32_t d = tmem + TC_BUF + (uint32_t)(ch * TC_RW);
        const uint32_t b_hi = row4 + ((uint32_t)L.eb[blk][0] >> 4);
        const uint32_t b_lo = row4 + ((uint32_t)L.eb[blk][1] >> 4);
#pragma unroll
        for (int ks = 0; ks < TY::KSTEPS; ++ks) {
#pragma unroll
            for (int pr = 0; pr < (TY::SPLIT ? 3 : 1); ++pr) {
                const int pa = pr == 2 ? 1 : 0;  // coefficient part: hi, hi, lo
                const uint32_t a = tmem + TC_AC + (uint32_t)((2 * ax + pa) * TY::ACOLS + ks * 8);
                const uint64_t b = hi | (uint64_t)((pr == 1 ? b_lo : b_hi) + (uint32_t)(2 * ks) * lbo4);
                tc_mma<TY::BF16>(d, a, b, idesc, (ks == 0 && pr == 0) ? 0u : 1u);
            }
        }
    }
}

// Contraction MMAs of one chunk (samples s0 .. s0 + 15, column `col` of each
// channel): for channels [CH0, CH1) the residual rows E (in place) times the
// transposed block, accumulated into the channel's target (THETA: theta in
// the xdot channel, with P, into target 3).  `first`: the round's first
// chunk of the phase, whose first product per target overwrites it.
template <int PREC, int CH0, int CH1, bool THETA>
__device__ __forceinline__ void tc_issue_contr(uint32_t tmem, uint32_t sm_base, const TcLayout& L, int s0,
                                               uint32_t col, bool first)
{
    using TY = TcType<PREC>;
    const uint32_t idesc = tc_idesc<PREC>(16);
    const uint64_t hi = ((uint64_t)(256u >> 4) << 16) | ((uint64_t)(128u >> 4) << 32) | (1ull << 46);
    const uint32_t grp4 = (sm_base >> 4) + (uint32_t)(s0 / TY::PER) * 16u;  // 256-byte K groups
#pragma unroll
    for (int ch = CH0; ch < CH1; ++ch) {
        const int blk = THETA ? 0 : (ch < 3 ? 0 : (ch < 5 ? 1 : 2));
        const int dst = THETA ? 3 : (ch < 3 ? ch : ((ch - 3) & 1));
        const bool lead = THETA || ch < 3;  // the target's first channel
        const uint32_t d = tmem + TC_DC + (uint32_t)(dst * 16);
#pragma unroll
        for (int ks = 0; ks < TY::CSTEPS; ++ks) {
            const uint32_t a = tmem + col + (uint32_t)(ch * TC_RW + ks * 8);
#pragma unroll
            for (int pb = 0; pb < TY::PARTS; ++pb) {
                const uint64_t b = hi | (uint64_t)(grp4 + ((uint32_t)L.cb[blk][pb] >> 4) + (uint32_t)(32 * ks));
                const uint32_t acc = (first && lead && ks == 0 && pb == 0) ? 0u : 1u;
                tc_mma<TY::BF16>(d, a, b, idesc, acc);
            }
        }
    }
}

// Culling list of one warp for one chunk, rebuilt every time (the exact test
// of cull_update, with no growth of the box: the list holds every obstacle
// not provably apart from the box of the warp's samples over the chunk's time
// window, in increasing index order).
__device__ __forceinline__ int tc_cull(int m, float xlo, float xhi, float ylo, float yhi, bool any_bad, float tw_lo,
                                       float tw_hi, int* list, int lane, const float4* __restrict__ obs)
{
    const unsigned below = (1u << lane) - 1u;
    int count = 0;
    for (int j0 = 0; j0 < m; j0 += 32) {
        const int j = j0 + lane;
        bool keep = false;
        if (j < m) {
            const float4 ox = obs[2 * j], oy = obs[2 * j + 1];  // (p, p, pv, pv) per axis
            const float e1 = -fmaf(ox.z, tw_lo, ox.x), e2 = -fmaf(ox.z, tw_hi, ox.x);
            const float f1 = -fmaf(oy.z, tw_lo, oy.x), g1 = -fmaf(oy.z, tw_hi, oy.x);
            const bool apart = (xlo - fmaxf(e1, e2) >= CULL_MARGIN) || (fminf(e1, e2) - xhi >= CULL_MARGIN) ||
                               (ylo - fmaxf(f1, g1) >= CULL_MARGIN) || (fminf(f1, g1) - yhi >= CULL_MARGIN);
            keep = any_bad || !apart;
        }
        const unsigned bal = __ballot_sync(FULL, keep);
        if (keep) list[count + __popc(bal & below)] = j;
        count += __popc(bal);
    }
    __syncwarp();
    return count;
}

// Residuals of a pair of samples, as packed f32x2 arithmetic (Eqs. split_v,
// split_alpha_o, split_alpha_a in the trigonometry-free forms of the pair
// kernel; x and the obstacles in the frame moving with v0): e = (obstacle x,
// obstacle y, psi - theta, non-holonomic x, y, acceleration x, y), and the
// squared residual norms of the valid samples.
template <bool LIST, bool RESID>
__device__ __forceinline__ void tc_pair(const SolveArgs& A, const float (&v)[TC_CH][2], float2 tt, float2 valid,
                                        float v0, const float4* __restrict__ obs, const int* __restrict__ list, int cnt,
                                        float2 (&e)[TC_CH], float (&r)[4])
{
    const float2 x = f2(v[0][0], v[0][1]), y = f2(v[1][0], v[1][1]), ps = f2(v[2][0], v[2][1]);
    const float2 xd = __fadd2_rn(f2(v[3][0], v[3][1]), f2(v0)), yd = f2(v[4][0], v[4][1]);
    const float2 xdd = f2(v[5][0], v[5][1]), ydd = f2(v[6][0], v[6][1]);
    const float2 theta = atan2_pair(yd, xd);
    const float2 sp2 = __ffma2_rn(xd, xd, __fmul2_rn(yd, yd));
    const float2 nvel = f2(-fminf(fmaxf(sqrtf(sp2.x), A.v_min), A.v_max), -fminf(fmaxf(sqrtf(sp2.y), A.v_min), A.v_max));
    float2 sn, cs;
    sincos_pair(ps, sn, cs);
    const float2 evx = __ffma2_rn(nvel, cs, xd);
    const float2 evy = __ffma2_rn(nvel, sn, yd);
    const float2 an2 = __ffma2_rn(xdd, xdd, __fmul2_rn(ydd, ydd));
    const float2 fr = f2(1.f - fminf(1.f, A.a_max * rsqrtf(an2.x)), 1.f - fminf(1.f, A.a_max * rsqrtf(an2.y)));
    const float2 eax = __fmul2_rn(xdd, fr);
    const float2 eay = __fmul2_rn(ydd, fr);
    const float2 Xn = __fmul2_rn(x, f2(A.inv_a)), Yn = __fmul2_rn(y, f2(A.inv_b));
    const float a2 = A.a * A.a, b2 = A.b * A.b;
    float2 Sx, Sy, R2;
    obstacle_sum2<RESID, LIST>(obs, list, cnt, Xn, Yn, tt, a2, b2, Sx, Sy, R2);
    // a sample exactly at an obstacle centre (rare): the exact sum, through
    // temporaries so that the common path keeps its values in registers
    if (isnan(Sx.x) || isnan(Sy.x)) {
        float sx, sy, r2;
        obstacle_sum_exact(obs, A.m, Xn.x, Yn.x, tt.x, a2, b2, sx, sy, r2);
        Sx.x = sx; Sy.x = sy; R2.x = r2;
    }
    if (isnan(Sx.y) || isnan(Sy.y)) {
        float sx, sy, r2;
        obstacle_sum_exact(obs, A.m, Xn.y, Yn.y, tt.y, a2, b2, sx, sy, r2);
        Sx.y = sx; Sy.y = sy; R2.y = r2;
    }
    e[0] = __fmul2_rn(Sx, f2(-A.a));
    e[1] = __fmul2_rn(Sy, f2(-A.b));
    e[2] = __fadd2_rn(ps, f2(-theta.x, -theta.y));
    e[3] = evx;
    e[4] = evy;
    e[5] = eax;
    e[6] = eay;
    if (RESID) {
        const float2 ra = __ffma2_rn(eax, eax, __fmul2_rn(eay, eay));
        const float2 rv = __ffma2_rn(evx, evx, __fmul2_rn(evy, evy));
        const float2 rp = __fmul2_rn(e[2], e[2]);
        r[0] = fmaf(R2.y, valid.y, fmaf(R2.x, valid.x, r[0]));
        r[1] = fmaf(ra.y, valid.y, fmaf(ra.x, valid.x, r[1]));
        r[2] = fmaf(rv.y, valid.y, fmaf(rv.x, valid.x, r[2]));
        r[3] = fmaf(rp.y, valid.y, fmaf(rp.x, valid.x, r[3]));
    }
}

// 8 values of one channel into tensor memory as the MMA's A operand: TF32
// bits (8 columns) or BF16 pairs (4 columns).
template <int PREC>
__device__ __forceinline__ void tc_store8(uint32_t addr_tf32, uint32_t addr_bf16, const float (&v)[8])
{
    if (TcType<PREC>::BF16) {
        uint32_t r[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) r[j] = bf16_pair(v[2 * j], v[2 * j + 1]);
        tc_st4(addr_bf16, r);
    } else {
        uint32_t r[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) r[j] = tf32_bits(v[j]);
        tc_st8(addr_tf32, r);
    }
}

// The values of samples 2j, 2j + 1 of one channel slot as the MMA's A
// operand: TF32 bits in columns 2j, 2j + 1, or one BF16 pair in column j.
template <int PREC>
__device__ __forceinline__ void tc_store_pair(uint32_t slot, int j, float a, float b)
{
    if (TcType<PREC>::BF16) tc_st1(slot + (uint32_t)j, bf16_pair(a, b));
    else tc_st2(slot + (uint32_t)(2 * j), tf32_bits(a), tf32_bits(b));
}

// The coefficient rows of one axis (hi and, split, lo) into tensor memory.
template <int PREC>
__device__ __forceinline__ void tc_write_coef(uint32_t lane_tmem, int axis, const float (&c)[16])
{
    using TY = TcType<PREC>;
    const uint32_t base = lane_tmem + TC_AC + (uint32_t)(2 * axis * TY::ACOLS);
    float hi[16], lo[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        hi[k] = TY::BF16 ? bf16_val(c[k]) : __uint_as_float(tf32_bits(c[k]));
        lo[k] = c[k] - hi[k];
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = hi[8 * h + j];
        tc_store8<PREC>(base + 8 * h, base + 4 * h, v);
    }
    if (TY::SPLIT) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = lo[8 * h + j];
            tc_store8<PREC>(base + TY::ACOLS + 8 * h, base + TY::ACOLS + 4 * h, v);
        }
    }
}

// 16-wide dot product of a shared-memory row with a register vector; four
// partial sums.
template <int NC>
__device__ __forceinline__ float tc_dot(const float* __restrict__ row, const float (&v)[16])
{
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < NC; j += 4) {
        const float4 x = *reinterpret_cast<const float4*>(row + j);
        acc[0] = fmaf(x.x, v[j], acc[0]);
        acc[1] = fmaf(x.y, v[j + 1], acc[1]);
        acc[2] = fmaf(x.z, v[j + 2], acc[2]);
        acc[3] = fmaf(x.w, v[j + 3], acc[3]);
    }
    return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// x - y for packed pairs, as one rounding (fma(y, -1, x) is exactly x - y
// rounded): the error-free transformations below need plain subtractions
__device__ __forceinline__ float2 sub2(float2 x, float2 y) { return __ffma2_rn(y, f2(-1.f), x); }

// Knuth's TwoSum on packed pairs: a + b = s + e exactly, per lane.
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e)
{
    s = __fadd2_rn(a, b);
    const float2 z = sub2(s, a);
    e = __fadd2_rn(sub2(a, sub2(s, z)), sub2(b, z));
}

// Compensated dot products (Dot2 of Ogita, Rump and Oishi, "Accurate sum and
// dot product", SIAM J. Sci. Comput. 26, 2005) of two rows r0, r1 with v over
// the columns [J0, J1), the two rows in the two lanes of packed f32x2
// arithmetic: each product's rounding error (by FMA) and each sum's (by
// TwoSum) is carried to the end, so each result is as accurate as a dot
// product in twice the working precision, rounded once.  K11 u needs it: u
// carries the multipliers, which grow in K11's near-null directions, and the
// products (entries of ~1e3 times ~1e3) cancel by five orders of magnitude.
template <int J0, int J1>
__device__ __forceinline__ float2 tc_dot2_rows(const float* __restrict__ r0, const float* __restrict__ r1,
                                               const float (&v)[16])
{
    float2 s[2] = {f2(0.f), f2(0.f)}, c[2] = {f2(0.f), f2(0.f)};
#pragma unroll
    for (int j = J0 & ~3; j < J1; j += 4) {
        const float4 x = *reinterpret_cast<const float4*>(r0 + j), y = *reinterpret_cast<const float4*>(r1 + j);
        const float k0[4] = {x.x, x.y, x.z, x.w}, k1[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (j + q < J0 || j + q >= J1) continue;
            const int h = (j + q) & 1;  // two interleaved partial sums per row
            const float2 kk = f2(k0[q], k1[q]), uu = f2(v[j + q]);
            const float2 pq = __fmul2_rn(kk, uu);
            const float2 pe = __ffma2_rn(kk, uu, f2(-pq.x, -pq.y));
            float2 t;
            two_sum2(s[h], pq, s[h], t);
            c[h] = __fadd2_rn(c[h], __fadd2_rn(pe, t));
        }
    }
    float2 S, t;
    two_sum2(s[0], s[1], S, t);
    return __fadd2_rn(S, __fadd2_rn(__fadd2_rn(c[0], c[1]), t));
}

// Plain dot products of two rows over the columns [J0, J1) (the K11 lo part:
// small terms), packed as above.
template <int J0, int J1>
__device__ __forceinline__ float2 tc_dot_rows(const float* __restrict__ r0, const float* __restrict__ r1,
                                              const float (&v)[16])
{
    float2 acc[2] = {f2(0.f), f2(0.f)};
#pragma unroll
    for (int j = J0 & ~3; j < J1; j += 4) {
        const float4 x = *reinterpret_cast<const float4*>(r0 + j), y = *reinterpret_cast<const float4*>(r1 + j);
        const float k0[4] = {x.x, x.y, x.z, x.w}, k1[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (j + q >= J0 && j + q < J1) acc[(j + q) & 1] = __ffma2_rn(f2(k0[q], k1[q]), f2(v[j + q]), acc[(j + q) & 1]);
    }
    return __fadd2_rn(acc[0], acc[1]);
}

// Step (split_xy) in increment form for one axis, c += K11 u with K11 as
// hi + lo, over the rows and columns [K0, K1): the coefficients fixed by the
// boundary rows (the first three of each axis; the last three of y, whose end
// position, speed and acceleration are all given) have zero rows and columns
// in K11 and take only their carry (which holds the first step's boundary
// correction of a warm start).  Rows go in pairs through the packed products.
template <int NC, int K0, int K1, int KS>
__device__ __forceinline__ void tc_xy_step(const float* __restrict__ Kh, const float* __restrict__ Kl,
                                           const float (&u)[16], float (&c)[16], float (&e)[16])
{
    float dd[16];
#pragma unroll
    for (int k = 0; k < NC; ++k) dd[k] = 0.f;
#pragma unroll
    for (int k = K0; k < K1; k += 2) {
        const int k1 = k + 1 < K1 ? k + 1 : k;
        const float2 hi = tc_dot2_rows<K0, K1>(Kh + k * KS, Kh + k1 * KS, u);
        const float2 lo = tc_dot_rows<K0, K1>(Kl + k * KS, Kl + k1 * KS, u);
        dd[k] = hi.x + lo.x;
        if (k + 1 < K1) dd[k + 1] = hi.y + lo.y;
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const float d = dd[k] + e[k];
        const float snew = c[k] + d;
        e[k] = d - (snew - c[k]);
        c[k] = snew;
    }
}

__device__ __forceinline__ void tc_sync()
{
    tc_wait_st();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

template <int NC, int PREC>
__global__ void __launch_bounds__(TC_THREADS, 1) am_solve_tc_kernel(const __grid_constant__ SolveArgs A,
                                                                    const __grid_constant__ TcArgs T)
{
    using TY = TcType<PREC>;
    constexpr int KS = k_stride(NC);
    extern __shared__ __align__(128) unsigned char tsm[];
    __shared__ __align__(8) unsigned long long s_stage;
    __shared__ __align__(8) unsigned long long s_mma;
    __shared__ uint32_t s_tmem;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = warp >> 2, q = warp & 3;  // axis group, tensor-memory sub-partition
    const int t = 32 * q + lane;            // trajectory slot
    const int N = A.N, m = A.m;
    const BlobLayout& L = A.L;
    const TcLayout& TL = T.L;

    // shared memory: [tensor-core blob | Q, K11 x hi, lo, y hi, lo, K11_psi |
    // obstacles of each sub-partition's scene [4][m][2] | culling lists |
    // residual partial sums | sample times]
    float* mats = reinterpret_cast<float*>(tsm + TL.bytes);
    const int nmat = L.init - L.Q;
    float4* obs_all = reinterpret_cast<float4*>(mats + ((nmat + 3) & ~3));
    int* lists = reinterpret_cast<int*>(obs_all + 8 * m);
    float* part = reinterpret_cast<float*>(lists + 12 * m);  // [3][128][4]
    float* tgrid = part + 3 * 128 * 4;                       // sample times [NSP]
    int* olist = lists + warp * m;
    const float4* obs = obs_all + q * 2 * m;                 // this warp's scene
    __shared__ int4 s_item[4];     // current item of each sub-partition
    __shared__ int s_new[4];       // whether it was taken at this refill
    __shared__ int s_next[4];      // next goal of the item
    __shared__ int s_pos[128];     // goal (position within the item) each slot takes at this refill
    __shared__ float4 s_ego[4];    // (y0, v0, psi0, acc0) of its scene

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(TC_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < nmat; i += TC_THREADS) mats[i] = __ldg(A.blob + L.Q + i);
    for (int i = tid; i < TL.NSP; i += TC_THREADS) tgrid[i] = i < N ? __ldg(A.blob + L.t + i) : 0.f;
    if (tid < 4) {
        s_item[tid] = make_int4(-1, 0, 0, 0);
        s_next[tid] = 0;
    }
    const bool staged = stage_blob(reinterpret_cast<float*>(tsm), reinterpret_cast<const float*>(T.blob), TL.bytes,
                                   &s_stage, A.err_flag, A.missing_tx);
    const uint32_t bar = smem_u32(&s_mma);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);  // this warp's lanes
    const uint32_t sm_base = smem_u32(tsm);
    uint32_t mma_phase = 0;
    bool ok = staged;
    const int n = A.n;

    // ---- state of this thread's axis (g: 0 x, 1 y, 2 psi) for slot t ----
    float c[16], e[16], lam[16];  // e: compensation (x, y); K12_psi b_psi (psi)
#pragma unroll
    for (int k = 0; k < 16; ++k) c[k] = e[k] = lam[k] = 0.f;
    int l = 0;            // the slot's goal within its scene
    float v0 = 0.f;       // speed of the sub-partition's ego (the moving frame)

    // initial iterate of goal l of scene As (cold start, or warm start
    // projected onto the boundary rows by the first step)
    auto init_slot = [&](const SolveArgs& As, float4 ego) {
        const float y0 = ego.x, psi0 = ego.z, acc0 = ego.w;
#pragma unroll
        for (int k = 0; k < 16; ++k) c[k] = e[k] = lam[k] = 0.f;
        const float* gl = As.goals + 3 * l;
        const float yg = __ldg(gl + 0), vg = __ldg(gl + 1), ag = __ldg(gl + 2);
        float cpsi, spsi;
        sincosf(psi0, &spsi, &cpsi);
        const size_t wo = (size_t)l * 3 * n;
        if (g < 2) {
            const bool isy = g == 1;
            const float bx[6] = {0.f, v0 * cpsi - v0, acc0 * cpsi, vg - v0, ag, 0.f};
            const float by[6] = {y0, v0 * spsi, acc0 * spsi, yg, 0.f, 0.f};
            const int nb = isy ? 6 : 5;
            const float* C0 = A.blob + (isy ? L.C0y : L.C0x);
            const float* K12 = A.blob + (isy ? L.K12y : L.K12x);
            if (As.warm_c) {
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k < n)
                        c[k] = __ldg(As.warm_c + wo + (isy ? n : 0) + k) - (isy ? 0.f : v0 * __ldg(A.blob + L.lin + k));
            } else {
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    float sacc = 0.f;
#pragma unroll
                    for (int r = 0; r < 6; ++r)
                        if (r < nb) sacc = fmaf(__ldg(C0 + k * 8 + r), isy ? by[r] : bx[r], sacc);
                    c[k] = sacc;
                }
            }
            // K12 (b - A c^0): added by the first step (the start's boundary rows)
            const int rx[6] = {0, 1, 2, 4, 5, 5};
            float res[6];
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                const int row = isy ? r : rx[r];
                float sacc = 0.f;
#pragma unroll
                for (int k = 0; k < NC; ++k) sacc = fmaf(__ldg(A.blob + L.brow + row * NC + k), c[k], sacc);
                res[r] = (isy ? by[r] : bx[r]) - sacc;
            }
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                float sacc = 0.f;
#pragma unroll
                for (int r = 0; r < 6; ++r)
                    if (r < nb) sacc = fmaf(__ldg(K12 + k * 8 + r), res[r], sacc);
                e[k] = sacc;
            }
            if (As.warm_l) {
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k < n) lam[k] = __ldg(As.warm_l + wo + (isy ? n : 0) + k);
            }
        } else {
            const float bp[4] = {psi0, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                float sacc = 0.f, s0 = 0.f;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    sacc = fmaf(__ldg(A.blob + L.Kp12 + k * 4 + r), bp[r], sacc);
                    s0 = fmaf(__ldg(A.blob + L.C0p + k * 4 + r), bp[r], s0);
                }
                e[k] = sacc;
                c[k] = s0;
            }
            if (As.warm_c) {
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k < n) c[k] = __ldg(As.warm_c + wo + 2 * n + k);
            }
            if (As.warm_l) {
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k < n) lam[k] = __ldg(As.warm_l + wo + 2 * n + k);
            }
        }
    };

    bool done = true;    // the slot holds no active trajectory
    bool fresh = false;  // its trajectory was placed at this iteration (its pass 0)
    int kit = 0, it = 0;
    float rsum[4] = {0.f, 0.f, 0.f, 0.f};
    float rh1 = INFINITY, rh2 = INFINITY;  // convergence residuals of the last two checks
    unsigned long long work = 0;
    auto scene = [&](int sidx) -> const SolveArgs& { return T.scenes ? T.scenes[sidx] : A; };

    // Refill, at the start of every iteration.  A sub-partition holds one
    // item (goals of one scene) at a time: each free slot takes the item's
    // next goal; when the item is exhausted and every slot of the
    // sub-partition is free, it takes the next item from the queue, and its
    // scene's obstacles (moving frame of its ego speed) go to the
    // sub-partition's shared-memory block.  Slots run their own iteration
    // counts; a pass forms the residual sums when any slot checks.
    auto refill = [&]() {
        if (g == 0) {
            const bool empty = __all_sync(FULL, done);
            if (lane == 0) {
                int take = 0;
                const int4 cur = s_item[q];
                if (empty && cur.x != -2 && s_next[q] >= cur.z) {
                    for (;;) {  // the next item with goals (a fallback item may hold none)
                        const int k = atomicAdd(T.queue, 1);
                        if (k >= T.n_items) {
                            s_item[q] = make_int4(-2, 0, 0, 0);  // drained
                            break;
                        }
                        const int4 it4 = T.items ? T.items[k] : make_int4(0, 32 * k, min(32, A.B - 32 * k), 0);
                        if (it4.z > 0) {
                            s_item[q] = it4;
                            s_next[q] = 0;
                            take = 1;
                            break;
                        }
                    }
                }
                s_new[q] = take;
            }
        }
        __syncthreads();
        if (g == 0 && s_new[q]) {
            const SolveArgs& As = scene(s_item[q].x);
            const float4 eg = make_float4(__ldg(As.ego + 0), __ldg(As.ego + 1), __ldg(As.ego + 2), __ldg(As.ego + 3));
            if (lane == 0) s_ego[q] = eg;
            float4* ob = obs_all + q * 2 * m;
            for (int j = lane; j < m; j += 32) {
                const float* o = As.obst + 4 * j;
                const float px = -__ldg(o + 0) * A.inv_a, py = -__ldg(o + 1) * A.inv_b;
                const float pvx = -(__ldg(o + 2) - eg.y) * A.inv_a, pvy = -__ldg(o + 3) * A.inv_b;
                ob[2 * j] = make_float4(px, px, pvx, pvx);
                ob[2 * j + 1] = make_float4(py, py, pvy, pvy);
            }
        }
        if (g == 0) {  // free slots take the item's next goals
            int pos = -1;
            const int4 cur = s_item[q];
            if (done && cur.x >= 0 && s_next[q] < cur.z) {
                pos = atomicAdd(&s_next[q], 1);
                if (pos >= cur.z) pos = -1;
            }
            s_pos[t] = pos;
        }
        __syncthreads();
        if (s_new[q]) v0 = s_ego[q].y;
        const int pos = s_pos[t];
        if (pos >= 0) {
            const int4 item = s_item[q];
            const int posn = item.y + pos;
            l = T.order ? T.order[item.w + posn] : posn;
            init_slot(scene(item.x), s_ego[q]);
            done = false;
            fresh = true;
            kit = 0;
            rh1 = rh2 = INFINITY;
#pragma unroll
            for (int r = 0; r < 4; ++r) rsum[r] = 0.f;
        }
    };

    // this slot's outputs (its axis; group 0 also residuals and iterations)
    auto write_out = [&]() {
        const SolveArgs& As = scene(s_item[q].x);
        const size_t o = (size_t)l * 3 * n;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (k < n) {
                const float v =
                    g == 0 ? (c[k] + e[k]) + v0 * __ldg(A.blob + L.lin + k) : (g == 1 ? c[k] + e[k] : c[k]);
                As.coef_out[o + g * n + k] = v;
                if (As.lam_out) As.lam_out[o + g * n + k] = lam[k];
            }
        }
        if (g == 0) {
            if (As.resid_out) {
#pragma unroll
                for (int r = 0; r < 4; ++r) As.resid_out[(size_t)l * 4 + r] = sqrtf(rsum[r]);
            }
            if (As.iters_out) As.iters_out[l] = kit;
        }
    };
    const int nch = TL.NSP / TC_CS;
    const uint32_t gslot = TC_BUF + (uint32_t)(g * TC_CS);  // this group's 16 columns of each channel

    // projections of one chunk (samples s0 .. s0 + 15) of this group's slot:
    // evaluated channels in, residual rows out (in place)
    auto chunk_project = [&](int cidx, bool check, float (&r4)[4]) {
        const int s0 = cidx * TC_CS;
        const bool act = !done;
        const unsigned amask = __ballot_sync(FULL, act);
        if (!amask) return;
        const uint32_t ba = tl + gslot;
        const int nval = min(TC_CS, N - s0);
        int cnt = m;
        if (A.cull && m > 0) {
            const float inf = __int_as_float(0x7f800000);
            float xlo = inf, xhi = -inf, ylo = inf, yhi = -inf;
            bool bad = false;
            {
                float X[16], Y[16];
                tc_ld16(ba + 0, X);
                tc_ld16(ba + TC_RW, Y);
                if (act) {
#pragma unroll
                    for (int i = 0; i < TC_CS; ++i)
                        if (i < nval) {
                            const float Xn = X[i] * A.inv_a, Yn = Y[i] * A.inv_b;
                            xlo = fminf(xlo, Xn); xhi = fmaxf(xhi, Xn);
                            ylo = fminf(ylo, Yn); yhi = fmaxf(yhi, Yn);
                            bad = bad || !(isfinite(Xn) && isfinite(Yn));
                        }
                }
            }
            xlo = warp_min(xlo); xhi = warp_max(xhi);
            ylo = warp_min(ylo); yhi = warp_max(yhi);
            const bool any_bad = __any_sync(FULL, bad);
            cnt = tc_cull(m, xlo, xhi, ylo, yhi, any_bad, tgrid[s0], tgrid[s0 + nval - 1], olist, lane, obs);
        }
        if (lane == 0) work += (unsigned long long)cnt * (unsigned)nval * (unsigned)__popc(amask);
        uint32_t rn[14];
        tc_ld7x2_issue(ba, rn);
#pragma unroll 2
        for (int j = 0; j < TC_CS / 2; ++j) {
            tc_ld_wait14(rn);
            float v[TC_CH][2];
#pragma unroll
            for (int ch = 0; ch < TC_CH; ++ch) {
                v[ch][0] = __uint_as_float(rn[2 * ch]);
                v[ch][1] = __uint_as_float(rn[2 * ch + 1]);
            }
            if (j + 1 < TC_CS / 2) tc_ld7x2_issue(ba + 2 * (j + 1), rn);  // the next pair, while this one runs
            const int sa = s0 + 2 * j;
            const float2 valid = f2(act && sa < N ? 1.f : 0.f, act && sa + 1 < N ? 1.f : 0.f);
            const float2 tt = f2(tgrid[sa], tgrid[sa + 1]);
            float2 e2[TC_CH];
            if (check) {
                if (A.cull) tc_pair<true, true>(A, v, tt, valid, v0, obs, olist, cnt, e2, r4);
                else tc_pair<false, true>(A, v, tt, valid, v0, obs, nullptr, m, e2, r4);
            } else {
                if (A.cull) tc_pair<true, false>(A, v, tt, valid, v0, obs, olist, cnt, e2, r4);
                else tc_pair<false, false>(A, v, tt, valid, v0, obs, nullptr, m, e2, r4);
            }
            float ev[2][7];
#pragma unroll
            for (int ch = 0; ch < TC_CH; ++ch) {
                ev[0][ch] = e2[ch].x;
                ev[1][ch] = e2[ch].y;
            }
#pragma unroll
            for (int ch = 0; ch < TC_CH; ++ch) tc_store_pair<PREC>(ba + ch * TC_RW, j, ev[0][ch], ev[1][ch]);
        }
    };

    // heading of one chunk: theta = atan2(ydot, xdot) written over the xdot channel
    auto chunk_heading = [&](int cidx) {
        const int s0 = cidx * TC_CS;
        const bool act = !done;
        if (!__any_sync(FULL, act)) return;
        const uint32_t ba = tl + gslot;
#pragma unroll 2
        for (int j = 0; j < TC_CS / 2; ++j) {
            float vx[2], vy[2];
            tc_ld2(ba + 3 * TC_RW + 2 * j, vx);
            tc_ld2(ba + 4 * TC_RW + 2 * j, vy);
            const float2 th = atan2_pair(f2(vy[0], vy[1]), __fadd2_rn(f2(vx[0], vx[1]), f2(v0)));
            tc_store_pair<PREC>(ba + 3 * TC_RW, j, th.x, th.y);
        }
    };

    // one pass over the samples: rounds of three chunks (evaluation MMAs,
    // projections on the CUDA cores, contraction MMAs); heading: the
    // channels xdot, ydot only and the contraction P^T theta
    auto phase = [&](bool heading, bool check, float (&r4)[4]) -> bool {
        const int rounds = (nch + TC_GROUPS - 1) / TC_GROUPS;
        for (int r = 0; r < rounds; ++r) {
            const int nc = min(TC_GROUPS, nch - TC_GROUPS * r);
            if (tid == 0) {
                if (heading) tc_issue_eval<PREC, 3, 5>(tmem, sm_base, TL, r * TC_RW, nc);
                else tc_issue_eval<PREC, 0, TC_CH>(tmem, sm_base, TL, r * TC_RW, nc);
                tc_commit(bar);
            }
            const bool w = __syncthreads_and(tc_wait(bar, mma_phase)) != 0;
            mma_phase ^= 1u;
            if (!w) return false;
            tc_fence_after();
            const int ci = TC_GROUPS * r + g;
            if (g < nc) {
                if (heading) chunk_heading(ci);
                else chunk_project(ci, check, r4);
            }
            tc_sync();
            if (tid == 0)
                for (int gg = 0; gg < nc; ++gg) {
                    const int sc = (TC_GROUPS * r + gg) * TC_CS;
                    const uint32_t col = TC_BUF + (uint32_t)(gg * TC_CS);
                    const bool first = r == 0 && gg == 0;
                    if (heading) tc_issue_contr<PREC, 3, 4, true>(tmem, sm_base, TL, sc, col, first);
                    else tc_issue_contr<PREC, 0, TC_CH, false>(tmem, sm_base, TL, sc, col, first);
                }
        }
        if (tid == 0) tc_commit(bar);
        const bool w = __syncthreads_and(tc_wait(bar, mma_phase)) != 0;
        mma_phase ^= 1u;
        tc_fence_after();
        return w;
    };

    // residual sums of the three groups, added in a fixed order
    auto exchange = [&](const float (&r4)[4]) {
#pragma unroll
        for (int r = 0; r < 4; ++r) part[(g * 128 + t) * 4 + r] = r4[r];
        __syncthreads();
        if (!done) {  // a finished trajectory keeps the residuals of its last check
#pragma unroll
            for (int r = 0; r < 4; ++r)
                rsum[r] = (part[(0 * 128 + t) * 4 + r] + part[(1 * 128 + t) * 4 + r]) + part[(2 * 128 + t) * 4 + r];
        }
        __syncthreads();
    };

    // multiplier update, convergence check and the xy QP increment (Sec.
    // III-E), from the contraction accumulators of the pass just run
    auto finish = [&](bool first, bool check) {
        float ftd[16];
        tc_ld16(tl + TC_DC + (uint32_t)(16 * g), ftd);  // x, y: F^T (F c - g); psi: P^T (P c_psi - theta)
        if (done) return;
        const float rho = A.rho;
        float u[16];
        if (!first) {
#pragma unroll
            for (int k = 0; k < 16; ++k) lam[k] = k < NC ? fmaf(-rho, ftd[k], lam[k]) : 0.f;
        }
        if (g < 2) {
#pragma unroll
            for (int k = 0; k < 16; ++k)
                u[k] = k < NC ? lam[k] - tc_dot<NC>(mats + k * KS, c) - rho * ftd[k] : 0.f;
        }
        bool dn = kit >= A.iters;
        if (check && kit % A.check_every == 0 && (A.tol > 0.f || A.stall_tol > 0.f)) {
            const float conv = fmaxf(sqrtf(rsum[0]), fmaxf(sqrtf(rsum[1]), sqrtf(rsum[2])));
            if (!first) {
                if (A.tol > 0.f) dn = dn || conv <= A.tol;
                // stall stop: far from the target and not closing in over two checks
                if (A.stall_tol > 0.f && kit >= 2 * A.check_every && conv > A.stall_tol && conv > A.stall_ratio * rh2)
                    dn = true;
            }
            rh2 = rh1;
            rh1 = conv;
        }
        if (dn) {
            write_out();
            done = true;
            return;
        }
        if (g < 2) {
            const float* Kh = mats + (L.Q - L.Q) + (1 + 2 * g) * NC * KS;  // K11 hi of this axis
            const float* Kl = Kh + NC * KS;
            if (g == 0 || A.n != NC) tc_xy_step<NC, 3, NC, KS>(Kh, Kl, u, c, e);
            else tc_xy_step<NC, 3, NC - 3, KS>(Kh, Kl, u, c, e);
        }
    };

    // heading QP (Eq. lin_solve_psi_2): c_psi = K12_psi b_psi + K11_psi (rho P^T theta + lambda_psi)
    auto psi_step = [&]() {
        float pth[16];
        tc_ld16(tl + TC_DC + 48u, pth);
        if (done || fresh || g != 2) return;
        float vec[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) vec[k] = k < NC ? fmaf(A.rho, pth[k], lam[k]) : 0.f;
        const float* Kp = mats + 5 * NC * KS;
#pragma unroll
        for (int k = 0; k < NC; ++k) c[k] = e[k] + tc_dot<NC>(Kp + k * KS, vec);
    };

    // One iteration of every slot per pass of the loop; a slot placed at
    // this iteration runs its initial pass (iterate 0: auxiliaries and
    // F^T (F c^0 - g^0), then the first step) while the others run Algorithm
    // 1's iteration (heading QP, projections, multipliers, xy QP).
    while (ok) {
        refill();
        if (!__syncthreads_or(!done)) break;  // every slot done and the queue drained
        if (!done) kit = fresh ? 0 : kit + 1;
        const bool need = !done && (fresh || kit % A.check_every == 0 || kit >= A.iters);
        const bool check = __syncthreads_or(need) != 0;
        if (__syncthreads_or(!done && !fresh)) {
            if (g < 2) tc_write_coef<PREC>(tl, g, c);
            tc_sync();
            float rz[4] = {0.f, 0.f, 0.f, 0.f};
            ok = phase(true, false, rz);
            if (!ok) break;
            psi_step();
        }
        tc_write_coef<PREC>(tl, g, c);
        tc_sync();
        float rr[4] = {0.f, 0.f, 0.f, 0.f};
        ok = phase(false, check, rr);
        if (!ok) break;
        if (check) exchange(rr);
        finish(fresh, need);
        fresh = false;
        ++it;
    }
    if (!ok) {
        // an expired wait: record it, then let the tensor core finish what was
        // issued (bounded) before the tensor memory is released
        if (tid == 0) atomicOr(A.err_flag, ERR_TMA_TIMEOUT);
        if (staged) {
            if (tid == 0) tc_commit(bar);
            tc_wait(bar, mma_phase);
        }
    }
    if (lane == 0 && A.work && work) atomicAdd(A.work, work);
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS) : "memory");
}
