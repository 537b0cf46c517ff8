/*
 * nk.h -- C ABI of libnk: convolutional (Myrtle) and fully-connected NNGP
 * kernel blocks and the kernel-ridge PCG solve, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Adlam et al., "Kernel Regression with Infinite-Width Neural Networks
 * on Millions of Examples" (arXiv 2303.05420).  The paper gives its kernels as
 * Neural Tangents architecture listings (Appendix A) and computes the kernel
 * matrix as independent blocks of its upper triangle (Figure 1, top); it
 * solves (K + lambda I) A = Y by preconditioned conjugate gradients with one
 * CG per target column (Section 2 "Iterative solvers"; Appendix B.3).
 *
 * Conventions for every call
 *   - Pointers named X*, q*, K, Y, A, dK, dX* are DEVICE pointers owned by the
 *     caller; the library never frees them.  `iters` / `relres` outputs of
 *     nk_pcg_solve are HOST pointers.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     nk_self_diag, nk_block and nk_block_backward are stream-ordered and
 *     asynchronous; nk_pcg_solve synchronises the stream before returning.
 *   - Invalid arguments return NK_ERR_INVALID_ARG synchronously, before any
 *     work is enqueued.  CUDA errors return NK_ERR_CUDA.  Errors that the
 *     kernels detect on the device (q <= 0 or NaN feeding a ReLU map, a spin
 *     limit) are recorded in a device status word of the handle and reported by
 *     nk_sync_status, which synchronises the stream.
 *   - nk_last_error gives a one-line description of the last failure.
 *   - Images are NHWC float32: X[n][H][W][C], contiguous.
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef NK_H
#define NK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NK_OK = 0,
  NK_ERR_INVALID_ARG = 1,
  NK_ERR_CUDA = 2,
  NK_ERR_NUMERICAL = 3,     /* q <= 0 / NaN met by a ReLU map on the device */
  NK_ERR_NOT_CONVERGED = 4, /* PCG hit maxit; A holds the best iterate */
  NK_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
  NK_ERR_NO_MEMORY = 6,
  NK_ERR_UNSUPPORTED = 7    /* valid request that the library does not implement */
} nk_status;

/* Arithmetic of nk_block:
 *  NK_PREC_MIXED      fused single-launch path: FP64 self-variances, FP32
 *                     pixel-pair recursion held on chip, FP64 final combine;
 *                     K is float*.
 *  NK_PREC_PLAIN_FP32 layer-wise path, one launch per layer, pixel-pair
 *                     tensors in HBM, FP32; K is float*.
 *  NK_PREC_PLAIN_FP64 the same in FP64; K is double*. */
typedef enum { NK_PREC_PLAIN_FP64 = 0, NK_PREC_PLAIN_FP32 = 1, NK_PREC_MIXED = 2 } nk_prec;

/* Activations: the ReLU of the Myrtle listings (Appendix A), the identity
 * (a linear network, tests only) and Erf, one of the activations of the
 * paper's architecture search (Appendix on tuning the Myrtle architecture;
 * stax.Erf also serves its graph-network listing). */
enum { NK_ACT_RELU = 0, NK_ACT_IDENTITY = 1, NK_ACT_ERF = 2 };
/* Normalisation between each conv and its activation: none (the Myrtle
 * listings) or the tuned Myrtle listing's LayerNorm over pixels and channels
 * of each image (stax.LayerNorm(axis=(1, 2, 3))). */
enum { NK_NORM_NONE = 0, NK_NORM_LAYER = 1 };
/* Readout after the last conv layer: GlobalAvgPool then Dense (the Myrtle
 * listings) or Flatten then Dense (the CV8 listing, Appendix A).  A Flatten
 * readout's weights are independent per pixel, so only the pixel pairs p = p'
 * of the last layer enter: K = sigma_w2 mean_p Kt(p, p) + sigma_b2. */
enum { NK_READOUT_GAP = 0, NK_READOUT_FLATTEN = 1 };
enum { NK_PRECOND_NONE = 0, NK_PRECOND_JACOBI = 1, NK_PRECOND_PIVCHOL = 2 };

/* Myrtle-family architecture (Appendix A, Myrtle listing): n_stages stages;
 * stage s holds convs[s] layers of conv(filter x filter, SAME) [+ norm] +
 * activation; a 2x2 stride-2 average pool sits between consecutive stages;
 * the last stage ends in a global average pool and a Dense readout.
 * Myrtle-10 = {3, {3,3,3}}; the Myrtle-5 of the benchmark = {3, {2,1,0}}.
 * With norm = NK_NORM_LAYER each layer's covariance is divided by
 * sqrt(m m'), m = the pixel mean of that layer's self-variances of each
 * image (the infinite-width limit of a LayerNorm over pixels and channels),
 * and the activation sees the self-variances q / m. */
typedef struct {
  int n_stages;   /* 1..4 */
  int convs[4];   /* convs[0] >= 1 */
  int filter;     /* 3 (paper) or 1 */
  int activation; /* NK_ACT_RELU, NK_ACT_ERF or NK_ACT_IDENTITY */
  int norm;       /* NK_NORM_NONE or NK_NORM_LAYER (not with NK_ACT_IDENTITY) */
  int readout;    /* NK_READOUT_GAP or NK_READOUT_FLATTEN (no norm) */
} nk_arch;

/* sigma_w^2 = W_std^2 and sigma_b^2 = b_std^2 of every Conv / Dense layer
 * (Appendix A listings use W_std = sqrt(2), b_std = 0.1). */
typedef struct {
  double sigma_w2;
  double sigma_b2;
} nk_params;

typedef struct nk_handle nk_handle;

nk_status nk_create(nk_handle** h);
void nk_destroy(nk_handle* h);
const char* nk_status_string(nk_status s);
/* Copies the description of the last failure on this handle into buf. */
nk_status nk_last_error(nk_handle* h, char* buf, size_t len);
/* Synchronises `stream`, then reads and clears the handle's device status
 * word: NK_OK, NK_ERR_NUMERICAL or NK_ERR_TIMEOUT. */
nk_status nk_sync_status(nk_handle* h, void* stream);

/* Number of per-image self-variance entries: the sum over activation layers
 * l of H_l * W_l (H_l, W_l the resolution of layer l's stage), plus one
 * entry per layer (its LayerNorm divisor m_l) with NK_NORM_LAYER.  Returns -1
 * for an invalid architecture or size. */
int64_t nk_q_size(const nk_arch* arch, int H, int W);

/* Number of CUDA kernels launched through this handle since nk_create (a
 * host-side count, for measurement). */
int64_t nk_launch_count(nk_handle* h);

/* The ridge lambda used by the last nk_pcg_solve on this handle. */
double nk_last_lambda(nk_handle* h);

/* Per-pixel self-variances q_l(p) = K_l(p, p; x, x) for every image and every
 * activation layer (needed by the activation maps, stax.Relu / stax.Erf in
 * Appendix A), q_l being the conv's output before any LayerNorm.
 *   X   [n][H][W][C] float32 (device)
 *   qd  [n][nq] float64 (device, out): q, layer-major then row-major pixels;
 *       with NK_NORM_LAYER the last n_layers entries of a row are the
 *       divisors m_l = mean_p q_l(p)
 *   qs  [n][nq][2] float32 (device, out, may be NULL): the per-pixel factors
 *       (a, b) with which every kernel evaluates the activation of a pixel
 *       pair from its un-normalised covariance K:
 *         ReLU: a = 1/sqrt(q), b = sqrt(q / m): Kt = b b' J(K a a') / (2 pi),
 *               (0, 0) where q == 0;
 *         Erf:  a = sqrt(2 / (m + 2 q)), b = 1: Kt = b b' (2/pi) asin(K a a');
 *       m = 1 without a norm.
 * with nq = nk_q_size(arch, H, W).  Computed in FP64 from the banded self
 * covariance K_l(p, p + D; x, x), |D| <= r_s per stage (r = 0 at the last
 * stage with an activation, r_prev = 2 r + 1 across each pool).  m <= 0 (an
 * all-zero representation under a LayerNorm) is NK_ERR_NUMERICAL. */
nk_status nk_self_diag(nk_handle* h, const nk_arch* arch, const nk_params* prm,
                       const float* X, int64_t n, int H, int W, int C,
                       double* qd, float* qs, void* stream);

/* Kernel block K[i - a0][j - b0] = NNGP(Xa[i], Xb[j]) for i in [a0, a1),
 * j in [b0, b1) (Figure 1, top: blocks of the kernel matrix are computed
 * independently).
 *   Xa, Xb      image sets [na][H][W][C], [nb][H][W][C] float32 (device)
 *   qda, qdb    their nk_self_diag FP64 outputs (used by PLAIN_FP64)
 *   qsa, qsb    their nk_self_diag FP32 (1/sqrt q, sqrt q) outputs (used by
 *               MIXED and PLAIN_FP32)
 *   K, ldk      output, row-major, leading dimension ldk >= b1 - b0;
 *               float* for MIXED / PLAIN_FP32, double* for PLAIN_FP64
 *   symmetric   nonzero when Xa == Xb and [a0,a1) == [b0,b1): only i <= j is
 *               evaluated and mirrored.
 * The Myrtle readout is K = sigma_w2 * mean_{P,P'} Kt(P, P') + sigma_b2
 * (GlobalAvgPool then Dense).  MIXED requires filter 3, C <= 3 and
 * zero-conv stages only at the end; with ReLU H = W in {8, 16, 32} and stage
 * patterns (2,1,0) (2,1,1) (3,3,3) (1) (1,1,1), or H = W = 64 and (2,1,0) (1)
 * (1,1); with Erf the tiled form only: H = W in {32, 64} and (2,1,0) (1)
 * (1,1); either with or without a LayerNorm.  With NK_READOUT_FLATTEN
 * (the CV8 listing: one stage of convs, no pools) MIXED carries only the
 * p = p' diagonal of each pair, which the diagonal stencil keeps closed: H
 * in {8, 16, 32}, W <= 32, ReLU or Erf, C <= 4; one warp per pair, FP32
 * recursion, FP64 readout sum.  Other valid requests there return
 * NK_ERR_UNSUPPORTED; the layer-wise PLAIN forms take every architecture.  At 64x64
 * MIXED runs the tiled form: stage-0 tasks over row bands and groups of
 * super-plane shifts, the pooled stage-1 tensor of each pair (4 MB) in a
 * ring of slots in the handle's workspace, one stage-1 task per pair; the
 * workspace holds the ring (sized for four CTAs per SM: about 170 MB with
 * 64x64 pairs, 250 MB when 32x32 blocks share the queue, 80 MB with 32x32
 * pairs only) plus 16 bytes per pair of the block, and is allocated on first
 * use.  The same form is the default at
 * 32x32 for these stage patterns (see nk_autotune).  At 32x32 the tiled form
 * also takes the three-stage ReLU patterns (3,3,3) and (2,1,1): its stage-1
 * task pools into an 8x8 stage-2 tile in shared memory and runs stage 2 on
 * the same CTA (one CTA of 512 threads per SM; 1.5x the cluster kernel on
 * Myrtle-10 blocks).
 * Device-side waits are bounded and report NK_ERR_TIMEOUT through
 * nk_sync_status. */
nk_status nk_block(nk_handle* h, const nk_arch* arch, const nk_params* prm, nk_prec prec,
                   const float* Xa, const double* qda, const float* qsa, int64_t a0, int64_t a1,
                   const float* Xb, const double* qdb, const float* qsb, int64_t b0, int64_t b1,
                   int H, int W, int C, void* K, int64_t ldk, int symmetric, void* stream);

/* Fully-connected ReLU NNGP block (Appendix A, FC3 listing: Dense + Relu
 * `depth` times, Dense readout):
 *   K_0 = x . x' / d;  K = sigma_w2 K_0 + sigma_b2;
 *   depth times: K <- sigma_w2 * relu_map(K) + sigma_b2
 * for rows i in [a0, a1) of Xa and j in [b0, b1) of Xb (row-major [n][d]
 * float32, device), into K[i - a0][j - b0] (float32, leading dimension
 * ldk).  The Gram is a split-BF16 tcgen05 GEMM (x = hi + lo, three BF16
 * products per pair of elements, FP32 accumulation in TMEM, the small
 * cross products first and even / odd K blocks in two accumulators added by
 * the epilogue) with the recursion fused into its epilogue; the per-row
 * self-variances are FP64.
 * symmetric: Xa == Xb, equal ranges; tiles below the diagonal are skipped and
 * each entry is stored at (i, j) and (j, i).  depth 0..8.  Uses a handle
 * workspace of (na + nb) * 6 d bytes for the split operands.  A device wait
 * that runs out is reported by nk_sync_status as NK_ERR_TIMEOUT. */
nk_status nk_fc_block(nk_handle* h, int depth, const nk_params* prm, const float* Xa, int64_t a0, int64_t a1,
                      const float* Xb, int64_t b0, int64_t b1, int d, float* K, int64_t ldk, int symmetric,
                      void* stream);

/* Adjoint of nk_block (no counterpart printed in the paper; it differentiates
 * the Appendix A Myrtle kernel for a kernel-ridge loss).  Given the upstream
 * gradient dK of the block [a0,a1) x [b0,b1), ACCUMULATES (+=)
 *   dXa[i][H][W][C] for i in [a0, a1)   (absolute image index; may be NULL)
 *   dXb[j][H][W][C] for j in [b0, b1)   (may be NULL)
 *   *dsw2, *dsb2                        (device doubles)
 * through the whole recursion, including the dependence of the self-variances
 * q on the images and on sigma_w2, sigma_b2.
 *   prec   NK_PREC_PLAIN_FP32 or NK_PREC_MIXED: float dK, dXa, dXb; FP32
 *          pixel-pair tensors; NK_PREC_PLAIN_FP64: double dK, dXa, dXb.
 *          The self-variance adjoint is FP64 in all cases.  Every pair's
 *          contribution carries FP32 rounding of about 1e-7 in the FP32
 *          forms, so an upstream gradient whose contributions cancel
 *          strongly (a kernel-ridge loss at a near-singular ridge, where
 *          the sum is about 1e-3 of its terms) loses accuracy in
 *          proportion; PLAIN_FP64 is the form for such gradients.
 *   qda, qdb   nk_self_diag FP64 outputs (required); qsa, qsb its FP32 scale
 *              tables (required unless PLAIN_FP64).
 *   symmetric  the block is the upper triangle of Xa x Xa: dK[i][j] and
 *              dK[j][i] both count for that entry; dXa must equal dXb.
 * Needs sigma_w2 > 0, C <= 4, 3x3 filters, square images whose stage sides
 * are powers of two up to 64, ReLU or identity, no norm and the global-average readout (other
 * architectures: NK_ERR_UNSUPPORTED).  Per chunk of pairs the forward recursion is recomputed
 * and each layer's pre-activation kept in the handle's workspace; every pass
 * applies the previous map (forward) or this layer's map adjoint (reverse)
 * while it loads the stored tensor. */
nk_status nk_block_backward(nk_handle* h, const nk_arch* arch, const nk_params* prm, nk_prec prec,
                            const float* Xa, const double* qda, const float* qsa, int64_t a0, int64_t a1,
                            const float* Xb, const double* qdb, const float* qsb, int64_t b0, int64_t b1,
                            int H, int W, int C, const void* dK, int64_t lddk, int symmetric, void* dXa,
                            void* dXb, double* dsw2, double* dsb2, void* stream);

/* Autotuner for the fused (NK_PREC_MIXED) kernel, the block-tile queue's
 * launch shape (Figure 1, top: independent blocks are grouped so that each
 * fills the device).  Times each launch variant of the fused kernel for this
 * architecture, image size, channel count and sigma_b2 == 0 or not, on a
 * synthetic 12 x 12 block of hashed images (allocated and freed here), and
 * caches the fastest in the handle; later nk_block calls with the same key
 * use it.  Variants at 32x32: 0 = super-plane cluster kernel, 768 threads x
 * 8 row parts, 1 = 512 x 8, 2 = 512 x 4, 3 = the tiled form of the 64x64
 * blocks (stage patterns (2,1,0), (1), (1,1), and with ReLU (3,3,3), (2,1,1)
 * at 32x32; it needs the handle's workspace, which grows on first use);
 * other sizes have one.  Without a tuned entry nk_block uses variant 3
 * where it exists, else 0.  *variant
 * (may be NULL) receives the choice.  Synchronises `stream`. */
nk_status nk_autotune(nk_handle* h, const nk_arch* arch, const nk_params* prm, int H, int W, int C,
                      int* variant, void* stream);

/* Pins the fused-kernel launch variant for a key without timing (e.g. a
 * choice saved from an earlier nk_autotune).  NK_ERR_INVALID_ARG for a
 * variant this size does not have. */
nk_status nk_autotune_set(nk_handle* h, const nk_arch* arch, const nk_params* prm, int H, int W, int C,
                          int variant);

/* Fused (NK_PREC_MIXED) kernel block that allocates no device memory and
 * needs no handle.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc when they need a block -- a process
 * whose device memory is reserved up front by its own allocator and which
 * forbids new device allocations while it serves, or a plugin whose host
 * framework owns all device memory -- since nk_create allocates.  Arguments and results are those of
 * nk_block with prec = NK_PREC_MIXED (qsa / qsb from nk_self_diag, computed
 * beforehand); the launch variant is 0.  The kernel's scratch (two
 * accumulator slots of 12 bytes per 4-CTA or 1-CTA cluster) is a fixed
 * 16 KB device array inside the library, shared by all calls on a device:
 *   - the first call on a device (and the first after that device's
 *     context was reset) looks up the array's device address with the
 *     device current;
 *   - each call clears the slots it uses (stream-ordered) before its kernel;
 *   - calls whose kernels overlap on the GPU (unordered streams) race on the
 *     array; order them on one stream;
 *   - a GPU whose SM count needs more than 16 KB (over 682 SMs) is rejected
 *     with NK_ERR_INVALID_ARG.
 * err_buf (may be NULL) receives a one-line description of any failure. */
nk_status nk_block_fused_noalloc(const nk_arch* arch, const nk_params* prm,
                                 const float* Xa, const float* qsa, int64_t a0, int64_t a1,
                                 const float* Xb, const float* qsb, int64_t b0, int64_t b1,
                                 int H, int W, int C, float* K, int64_t ldk, int symmetric,
                                 void* stream, char* err_buf, size_t err_len);

/* Neural tangent kernel block (the first widening of the hot path: the
 * Myrtle NTK, Figure 1 computes NNGP and NTK kernels alike) together with
 * the NNGP block, in the NTK parameterisation of the Appendix A listings
 * (standard-normal parameters scaled in the forward pass):
 *   Theta_0 = 0; conv: K' = sw2 A(Kt) + sb2, Theta' = K' + sw2 A(Theta_t);
 *   ReLU: Kt = relu map of K, Theta_t = Theta (pi - arccos c) / (2 pi);
 *   pools on both; readout K = sw2 mean Kt + sb2, Theta = K + sw2 mean Theta_t.
 * Arguments as nk_block; K and Theta are [a1 - a0][ldk] outputs of the
 * precision's type.  ReLU or identity, no norm, global-average readout.
 * NK_PREC_PLAIN_FP32 / NK_PREC_PLAIN_FP64: the layer-wise forms (K and Theta
 * as pixel-pair tensors in HBM).  NK_PREC_MIXED: the fused tiled form of
 * nk_block with the tangent rows carried beside K on chip (FP32 recursion,
 * FP64 global averages; qsa / qsb needed, float outputs): ReLU, filter 3,
 * C <= 3, H == W in {32, 64} with the stage pattern (2,1,0), or H == W == 32
 * with (3,3,3) (Myrtle-10) or (2,1,1), otherwise NK_ERR_UNSUPPORTED.  Its K is nk_block's MIXED K (the same arithmetic; the
 * pooled sums are atomic adds, so the last bits may differ).  The tiled form's
 * slot ring holds both pooled tensors, so the workspace is twice nk_block's;
 * waits are bounded as there (NK_ERR_TIMEOUT through nk_sync_status). */
nk_status nk_block_ntk(nk_handle* h, const nk_arch* arch, const nk_params* prm, nk_prec prec,
                       const float* Xa, const double* qda, const float* qsa, int64_t a0, int64_t a1,
                       const float* Xb, const double* qdb, const float* qsb, int64_t b0, int64_t b1, int H,
                       int W, int C, void* K, void* Theta, int64_t ldk, int symmetric, void* stream);

/* One block of a kernel-block queue (nk_block_queue).  Images NHWC float32
 * of side H == W, self-variance pairs qs from nk_self_diag for that size,
 * output K[(i - a0) * ldk + (j - b0)] as in nk_block. */
typedef struct {
  const float* Xa;
  const float* qsa;
  int64_t a0, a1;
  const float* Xb;
  const float* qsb;
  int64_t b0, b1;
  int H, W;
  float* K;
  int64_t ldk;
  int symmetric;
} nk_block_task;

#define NK_QUEUE_MAX 8

/* Several kernel blocks (Figure 1: blocks of the kernel matrix are computed
 * independently and batched to fill the device), possibly of different image
 * sizes, in ONE persistent launch of the fused MIXED kernel.  Every block uses
 * the same architecture, parameters and channel count C; image sides 8, 16
 * or 32, or 64 and 32 (other mixes: NK_ERR_UNSUPPORTED).  Without 64x64
 * blocks a 32x32 pair is computed by a 4-CTA cluster, a 16x16 or 8x8 pair by
 * one CTA, and the launch allocates nothing (the handle's 64 KB scratch holds
 * the global-average slots).  With 64x64 blocks every pair runs in the tiled
 * form of nk_block (stage patterns (2,1,0) (1) (1,1)); its slot ring lives in
 * the handle's workspace, which grows on the first such call, so make one
 * call before capturing the queue in a CUDA graph.  Larger images are queued
 * first.  Stream-ordered and asynchronous; calls on one handle must be
 * stream-ordered.  n_tasks in 0..NK_QUEUE_MAX; tasks is a host array. */
nk_status nk_block_queue(nk_handle* h, const nk_arch* arch, const nk_params* prm, int C,
                         const nk_block_task* tasks, int n_tasks, void* stream);

/* Bound of every device-side wait of later calls on this handle (Section 2:
 * kernel blocks are computed by independent, preemption-safe routines, so a
 * block that cannot finish must end with an error, never hang).  The tiled
 * MIXED kernel waits for earlier items of its queue (each poll about
 * 0.25-1 us; default 2^22 polls, seconds); the FC kernel's pipeline waits on
 * its mbarriers (each poll a bounded try_wait; default 2^26 polls), and so
 * does the tensor-core first layer of nk_block_backward (FP32, same bound).  A wait
 * that runs out sets NK_ERR_TIMEOUT (read by nk_sync_status), the kernel
 * stops taking work, and the results of that call are undefined; the handle
 * stays usable.  The waits a kernel makes before it exits, for its own copies
 * and tensor-core operations in flight, keep a fixed bound.
 *   polls >= 0: the bound in polls (0: give up at the first unmet check);
 *   polls < 0: the defaults. */
nk_status nk_set_wait_limit(nk_handle* h, int64_t polls);

/* Warm start of later nk_pcg_solve calls on this handle (on != 0): A holds
 * the initial iterate on entry instead of being overwritten with zero, so a
 * solve can resume from a saved iterate (Section 2: the block-wise pipeline
 * is preemption-safe; CG's iterate is usable at any point).  MIXED refines
 * it (its first sweep forms the true residual of the given A); the plain
 * precisions solve one correction (K + lambda I) D = Y - (K + lambda I) A to
 * the relative tolerance that brings every column to tol, then A += D.  The
 * Krylov space of the interrupted solve is not kept, only its iterate.
 * Default off; NK_OK. */
nk_status nk_pcg_set_warm_start(nk_handle* h, int on);

/* Rank of the partial pivoted Cholesky preconditioner (NK_PRECOND_PIVCHOL)
 * used by later nk_pcg_solve calls on this handle (default 100; at most N is
 * used).  rank in 1..1024, else NK_ERR_INVALID_ARG. */
nk_status nk_pcg_set_rank(nk_handle* h, int rank);

/* Kernel-ridge solve (K + lambda I) A = Y by preconditioned CG, one CG per
 * column run in lock-step (Section 2 "Iterative solvers"; Appendix B.3).
 *   precond: NK_PRECOND_NONE, NK_PRECOND_JACOBI (M = diag(K) + lambda) or
 *   NK_PRECOND_PIVCHOL (Section 2's partial pivoted Cholesky: K ~ L^T L from
 *   the rank (nk_pcg_set_rank) largest-remaining-diagonal pivots, built on
 *   the device in FP64 for each call; M = L^T L + lambda I applied through
 *   the Woodbury identity).
 *   K [N][ldk] float32 (symmetric; device memory, or pinned host memory the
 *   device reads directly (cudaHostAlloc / cudaHostRegister; on a Grace
 *   system over the chip-to-chip link): the solve is then out of core, for
 *   kernels larger than HBM), Y [N][R] float64 (device, row
 *   major), A [N][R] float64 (device, out; in and out after
 *   nk_pcg_set_warm_start(h, 1)).
 *   prec = NK_PREC_MIXED: iterative refinement: the true residual
 *          Y - (K + lambda I) A is formed in double-FP32 arithmetic (exact
 *          FP32 products and two-float sums, about 2^-48 relative per step),
 *          the correction is solved by CG with FP32 K@P (FP32 chunks of 256
 *          products summed in FP64) and FP64 vectors and scalars, A += D
 *          (at most refine_max corrections);
 *   prec = NK_PREC_PLAIN_FP32: FP32 K@P, FP64 vectors and scalars, no
 *          refinement;
 *   prec = NK_PREC_PLAIN_FP64: every product in FP64.
 *   lambda  >= 0: the ridge; < 0: relative ridge, lambda_used =
 *           -lambda * tr(K) / N with tr(K) summed on the device in FP64
 *           (nk_last_lambda returns lambda_used);
 *   tol     stop when every column has ||r_j|| / ||y_j|| <= tol, r the true
 *           residual against the float32 K upcast to FP64;
 *   maxit   bound on the total number of CG iterations;
 *   iters   (host, out) CG iterations performed (max over columns);
 *   relres  (host, out, may be NULL) [R] final true relative residuals.
 * Returns NK_ERR_NOT_CONVERGED (A = best iterate) when maxit is reached.
 * Synchronises `stream`. */
nk_status nk_pcg_solve(nk_handle* h, const float* K, int64_t ldk, int64_t N,
                       const double* Y, int R, double lambda, int precond, nk_prec prec,
                       double tol, int maxit, int refine_max,
                       double* A, int* iters, double* relres, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NK_H */
