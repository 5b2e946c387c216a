/* Learned warm start of the batch trajectory optimizer: scene features, a
 * small MLP with its own training kernels, and the encoding between
 * solutions (c, lambda) and network outputs.
 *
 * The paper has no learned component; it names supervision of learning
 * from its batch solutions as a use of the method (Sec. V).  Here an MLP maps
 * a (scene, goal) feature row to an initial iterate (c^0, lambda^0) of
 * Algorithm 1 (Sec. III-E), replacing the cold start; mmpc_solve takes it as
 * warm_coef / warm_lam.  Its first step projects c^0 onto the boundary rows
 * A c = b (the K12 (b - A c^0) term), so the network's output need not satisfy
 * them.
 *
 * Conventions: all arrays row-major float32; "device" pointers are CUDA
 * device memory owned by the caller; calls taking a stream are asynchronous
 * on it.  Return codes are those of mmpc.h (0 = MMPC_OK, negative = error);
 * mmpc_mlp_last_error() returns the calling thread's last message.
 */
#ifndef MMPC_MLP_H
#define MMPC_MLP_H

#include <stddef.h>

#include "mmpc.h"

#ifdef __cplusplus
extern "C" {
#endif

#define MMPC_MLP_FEATURES 64   /* width of a feature row (61 used, padded) */
#define MMPC_MLP_NEAREST 10    /* obstacles in a feature row */
#define MMPC_MLP_MAX_LAYERS 8
#define MMPC_MLP_MAX_WIDTH 1024

/* One scene of a feature / decode batch (all pointers device memory). */
typedef struct {
    const float* ego;    /* [4]: y0, v0, psi0, acc0 (x0 = 0) */
    const float* obst;   /* [m][4]: x0, y0, vx, vy at t = 0; may be NULL if m = 0 */
    int m;               /* obstacles, 0..MMPC_MAX_OBST */
    const float* goals;  /* [B][3]: y_g, v_g, a_g */
    int B;               /* goals, >= 0 */
    float* X;            /* [B][64] feature rows (written by mmpc_features) */
    const float* Y;      /* [B][6n] standardised network outputs (read by mmpc_warm_decode) */
    float* coef;         /* [B][3n] c_x, c_y, c_psi (mmpc_warm_decode out / mmpc_warm_encode in) */
    float* lam;          /* [B][3n] lambda_x, lambda_y, lambda_psi (same) */
    float* Z;            /* [B][6n] standardised targets (written by mmpc_warm_encode) */
} mmpc_warm_scene;

/* Feature rows of S scenes (`scenes`: device array of S descriptors; uses
 * ego, obst, m, goals, B, X).  Row layout, for goal l of a scene:
 *   0-3    y0 / 3.5, v0 / 20, psi0, acc0 / 4
 *   4-53   10 slots of 5, nearest obstacle first: x0 / 100, (y0_j - y0) / 3.5,
 *          (vx_j - v0) / 20, vy_j / 20, lane(y0_j) - lane(y0) with
 *          lane(y) = clip(floor((y + 7) / 3.5), 0, 3); an empty slot
 *          (m < 10) holds (10, 0, 0, 0, 0)
 *   54-56  (y_g - y0) / 3.5, v_g / 20, a_g / 4
 *   57     1;  58-63  0
 * "Nearest" orders the obstacles by (x0/a)^2 + ((y0_j - y0)/b)^2 evaluated in
 * float32 with one rounding per operation (ties: lower index; NaN last).
 * Errors: MMPC_ERR_INVALID_ARG (NULL, S < 0, a or b <= 0), MMPC_ERR_CUDA. */
int mmpc_features(const mmpc_warm_scene* scenes, int S, float a, float b, void* stream);

/* Network outputs -> warm start (uses ego, B, Y, coef, lam).  The outputs
 * are 3n (coefficients only) or 6n (coefficients and multipliers) per row;
 * with t = Y sigma + mu per column (mu, sigma: device float[outputs]),
 *   c_x = t[0:n] + v0 lin,  c_y = t[n:2n] + y0,  c_psi = t[2n:3n],
 *   lin_k = T k / (n - 1)  (the coefficients of f(t) = t),
 * and lambda = t[3n:6n] (6n outputs), else per axis lambda = Q c when Q
 * (device float[n][n], the Q = Pdd^T Pdd of mmpc_build) is given, else 0.
 * lambda = Q c are the multipliers of a fixed point of Algorithm 1: there
 * F c = g, and the step (split_xy) leaves c unchanged iff K11 (lambda - Q c)
 * = 0.  lam may be NULL.  n in [MMPC_MIN_COEF, MMPC_MAX_COEF].  Errors as
 * mmpc_features. */
int mmpc_warm_decode(const mmpc_warm_scene* scenes, int S, int n, float T, int outputs, const float* mu,
                     const float* sigma, const float* Q, void* stream);

/* The inverse (uses ego, B, coef, lam, Z): Z = (t - mu) / sigma with t the
 * encoding above (3n or 6n columns).  With mu = 0 and sigma = 1 it writes
 * the raw t. */
int mmpc_warm_encode(const mmpc_warm_scene* scenes, int S, int n, float T, int outputs, const float* mu,
                     const float* sigma, void* stream);

/* Column means and standard deviations (population) of a device matrix
 * X [rows][cols], in two passes in float64: mean_out, std_out device
 * float[cols]; a zero deviation is replaced by 1.  rows >= 1. */
int mmpc_column_stats(const float* X, int rows, int cols, float* mean_out, float* std_out, void* stream);

/* out[r][c] = (X[r][c] - mean[c]) / sd[c] (device arrays; out may be X). */
int mmpc_standardize(const float* X, int rows, int cols, const float* mean, const float* sd, float* out, void* stream);

/* out[r] = src[idx[r]] for rows of `cols` floats (device idx int[rows]).
 * Indices are checked against src_rows on the device; a bad index writes a
 * row of NaN. */
int mmpc_gather_rows(const float* src, int src_rows, int cols, const int* idx, int rows, float* out, void* stream);

/* ---- The MLP --------------------------------------------------------------
 * width[0] -> width[1] -> ... -> width[layers]; GELU (0.5 x (1 + erf(x /
 * sqrt 2))) after every layer but the last.  Weights are held as float32
 * master copies and used as bfloat16 (round to nearest even) in every
 * product; products and sums are float32.  Training minimises the mean of
 * (y - Z)^2 over all outputs with AdamW (bias-corrected moments, decoupled
 * weight decay on the weight matrices only). */
typedef struct mmpc_mlp mmpc_mlp;

typedef struct {
    int layers;                          /* 1..MMPC_MLP_MAX_LAYERS */
    int width[MMPC_MLP_MAX_LAYERS + 1];  /* each 1..MMPC_MLP_MAX_WIDTH */
    int max_batch;                       /* rows per training call (mmpc_mlp_loss_grad), >= 1 */
    float beta1, beta2, eps, weight_decay;
} mmpc_mlp_config;

/* W[i]: host float[width[i]][width[i+1]] (row i of W = input unit i), b[i]:
 * host float[width[i+1]]; copied.  Allocates all device buffers (synchronous). */
int mmpc_mlp_create(const mmpc_mlp_config* cfg, const float* const* W, const float* const* b, mmpc_mlp** out);

/* Y [M][width[L]] = network(X [M][width[0]]) for any M >= 0 (device
 * pointers; processed in chunks, no allocation). */
int mmpc_mlp_forward(mmpc_mlp* net, const float* X, int M, float* Y, void* stream);

/* Forward with the activations kept, loss = mean (y - Z)^2 written to the
 * device float loss_out (may be NULL), and the gradients of the loss with
 * respect to every W and b stored in the network.  1 <= M <= max_batch. */
int mmpc_mlp_loss_grad(mmpc_mlp* net, const float* X, const float* Z, int M, float* loss_out, void* stream);

/* One AdamW step with the stored gradients and learning rate lr; the step
 * counter (for the bias correction) advances by one. */
int mmpc_mlp_adamw(mmpc_mlp* net, float lr, void* stream);

/* Copies of the network's state, synchronous (host buffers of `count`
 * floats, count = the array's size).  what: 0 W (master), 1 b, 2 dW, 3 db,
 * 4 first moment of W, 5 second moment of W, 6 first moment of b, 7 second
 * moment of b.  mmpc_mlp_write accepts what 0 and 1 (restores weights and
 * refreshes the bfloat16 copy). */
int mmpc_mlp_read(mmpc_mlp* net, int what, int layer, float* host, size_t count);
int mmpc_mlp_write(mmpc_mlp* net, int what, int layer, const float* host, size_t count);

/* Inference (mmpc_mlp_forward) on the tensor cores or the FP32 SIMT path.
 * on = 0: SIMT (the default).  on = 1: the pipelined tcgen05 GEMM, operands
 * fed by TMA through a ring of shared-memory stages, warp-specialised, two
 * TMEM accumulators, persistent CTAs; it needs every layer input width to be
 * a multiple of 8 and takes the single-stage kernel for any layer where that
 * (or the tensor map) fails.  on = 2: the single-stage tcgen05 GEMM for every
 * layer.  Both tensor-core paths use bfloat16 operands and float32
 * accumulation in tensor memory: each layer's input (the features, then every
 * hidden activation) is rounded to bfloat16 (nearest even), where the SIMT
 * path keeps it in float32; the two give the same result up to the order of
 * the float32 sums.  Other values of on: MMPC_ERR_INVALID_ARG.  Training
 * is set separately (mmpc_mlp_set_train_tensor_cores). */
int mmpc_mlp_set_tensor_cores(mmpc_mlp* net, int on);

/* Training (mmpc_mlp_loss_grad) on the tensor cores (on = 1) or the FP32
 * SIMT kernels (on = 0, the default).  With on = 1 the three products of
 * every layer -- forward H W, backward D W^T and weight gradient H^T D --
 * run on the pipelined tcgen05 GEMM with bfloat16 operands and float32
 * accumulation: the layer inputs (features, hidden activations) and the
 * output gradients D are rounded to bfloat16 (nearest even) where the SIMT
 * path keeps them in float32; the pre-activations, the GELU derivative, the
 * loss and the bias gradients (column sums of the float32 D) stay float32.
 * The weight gradient's sum over the M rows is split into ranges whose
 * float32 partial sums are added in a fixed order, so results are
 * deterministic.  Enabling allocates the bfloat16 operand buffers
 * (synchronous, ~ max_batch x (sum of widths) x 4 bytes) and needs every
 * layer input width (width[0 .. layers-1]) to be a multiple of 8 and
 * max_batch <= 2,097,120: otherwise MMPC_ERR_INVALID_ARG and the mode is
 * unchanged.  Other values of on: MMPC_ERR_INVALID_ARG. */
int mmpc_mlp_set_train_tensor_cores(mmpc_mlp* net, int on);

/* Number of kernel launches mmpc_mlp_forward enqueues for M rows in the
 * current mode (one for the single-kernel network of mode 1; per inference
 * chunk one per layer, plus the rounding of the features in mode 1 where the
 * single kernel does not take the shape); -1 for a NULL network or M < 0. */
int mmpc_mlp_forward_launches(mmpc_mlp* net, int M);

/* Synchronises the device and reports MMPC_ERR_TIMEOUT if a bounded wait of
 * a tensor-core kernel expired since the network was created. */
int mmpc_mlp_status(mmpc_mlp* net);

void mmpc_mlp_destroy(mmpc_mlp* net);
const char* mmpc_mlp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MMPC_MLP_H */
