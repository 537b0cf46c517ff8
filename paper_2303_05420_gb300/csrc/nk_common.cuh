// Internal definitions shared by the libnk translation units (CUDA side only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nk.h"

#define NK_MAX_STAGES 4
#define NK_MAX_LAYERS 32

// Device status word bits (see nk_sync_status).
#define NK_DEV_NUMERICAL 1u
#define NK_DEV_TIMEOUT 2u

// Architecture + image size resolved into per-stage / per-layer geometry.
// Layers are the conv(+activation) layers in network order; their
// self-variances live at q[layer_qoff[l] + i * W_l + j].
struct NkGeom {
  int n_stages;
  int convs[NK_MAX_STAGES];
  int filter;
  int act;
  int norm;           // NK_NORM_NONE / NK_NORM_LAYER
  int readout;        // NK_READOUT_GAP / NK_READOUT_FLATTEN
  int C;
  int Hs[NK_MAX_STAGES];
  int Ws[NK_MAX_STAGES];
  int n_layers;
  int layer_stage[NK_MAX_LAYERS];
  int layer_qoff[NK_MAX_LAYERS];
  int nq;             // per-image stride of qd / qs: nq_base + (norm ? n_layers : 0)
  int nq_base;        // sum over layers of H_l W_l; the LayerNorm divisors m_l follow at nq_base + l
  int last_act_stage;  // last stage holding an activation layer (-1: none)
  int gap_stage;       // the stage whose activations feed the global average pool
  int radius[NK_MAX_STAGES];  // self-covariance band radius needed per stage
};

// Returns false (and fills why) when the request is invalid.
bool nk_make_geom(const nk_arch* arch, int H, int W, int C, NkGeom* g, const char** why);

// Handle internals.
struct nk_handle {
  char err[512];
  unsigned int* dstatus;   // device status word
  void* ws;                // workspace (device)
  size_t ws_bytes;
  int sm_count;
  int device;
  int64_t launches;        // kernels launched through this handle
  double last_lambda;      // ridge used by the last nk_pcg_solve
  void* small_ws;          // 64 KB for per-launch counters / accumulators
  // autotune cache: fused-kernel launch variant per (stage pattern, size, C, bias)
  int tune_n;
  int tune_key[16][8];
  int tune_variant[16];
  // PCG scratch
  void* pcg_ws;
  size_t pcg_bytes;
  int pcg_rank;            // pivoted Cholesky preconditioner rank
  int pcg_warm;            // nk_pcg_solve starts from the caller's A (nk_pcg_set_warm_start)
  long long wait_polls;    // bound of device waits (nk_set_wait_limit); < 0: defaults
};

// Default bounds of the device-side waits: polls of the tiled kernel's
// dependency waits (each about 0.25-1 us) and of the FC kernel's mbarrier
// waits (each a try_wait of up to a few us).
#define NK_TILED_WAIT_DEFAULT (1ll << 22)
#define NK_FC_WAIT_DEFAULT (1u << 26)

nk_status nk_fail(nk_handle* h, nk_status s, const char* fmt, ...);
nk_status nk_cuda_check(nk_handle* h, cudaError_t e, const char* what);
nk_status nk_workspace(nk_handle* h, size_t bytes, void** out);

// Launchers (each returns a CUDA error, arguments already validated).
cudaError_t nk_launch_self_diag(const NkGeom& g, double sw2, double sb2, const float* X,
                                int64_t n, double* qd, float* qs, double* ws, int grid,
                                unsigned int* dstatus, cudaStream_t st);
size_t nk_self_diag_ws_per_cta(const NkGeom& g);

// Layer-wise Myrtle NTK block (K and Theta); workspace 2 * nk_plain_ws_bytes.
cudaError_t nk_launch_myrtle_plain_ntk(const NkGeom& g, int fp64, double sw2, double sb2, const float* Xa,
                                       const double* qda, const float* qsa, int64_t a0, int64_t a1,
                                       const float* Xb, const double* qdb, const float* qsb, int64_t b0,
                                       int64_t b1, void* K, void* Th, int64_t ldk, int symmetric, void* ws,
                                       int64_t chunk, unsigned int* dstatus, cudaStream_t st, int64_t* launches);

// Fused (MIXED) Myrtle block.  Returns cudaErrorNotSupported when the
// architecture / size has no fused instantiation.
cudaError_t nk_launch_myrtle_fused(const NkGeom& g, double sw2, double sb2, const float* Xa,
                                   const float* qsa, int64_t a0, int64_t a1, const float* Xb,
                                   const float* qsb, int64_t b0, int64_t b1, float* K,
                                   int64_t ldk, int symmetric, int sm_count, void* scratch,
                                   size_t scratch_bytes, int variant, cudaStream_t st);
// Number of launch variants of the fused form at 32x32 (nk_autotune): three
// super-plane cluster launches and the tiled form.
#define NK_FUSED_VARIANTS 4
#define NK_TILED_VARIANT 3
bool nk_myrtle_fused_supported(const NkGeom& g);
bool nk_cluster_pattern(const int c[3]);

// Flatten-readout (CV8) block by the diagonal recursion (cv_diag.cu).
bool nk_cv_supported(const NkGeom& g);
cudaError_t nk_launch_cv_diag(const NkGeom& g, double sw2, double sb2, const float* Xa, const float* qsa,
                              int64_t a0, int64_t a1, const float* Xb, const float* qsb, int64_t b0, int64_t b1,
                              float* K, int64_t ldk, int symmetric, int sm_count, cudaStream_t st);

// FC NNGP block on the tensor cores (fc_gram.cu).
size_t nk_fc_ws_bytes(int64_t na, int64_t nb, int d, int depth);
cudaError_t nk_launch_fc_block(int depth, double sw2, double sb2, const float* Xa, int64_t a0, int64_t a1,
                               const float* Xb, int64_t b0, int64_t b1, int d, float* K, int64_t ldk, int sym,
                               void* ws, int sm, unsigned int* dstatus, uint32_t wait_limit, cudaStream_t st,
                               int64_t* launches);

// Adjoint of the Myrtle block (layer-wise, FP32 or FP64 pixel-pair tensors).
// The first layer as a patch Gram on the tensor cores (seed_gemm.cu): FP32
// pre-activation K_1[pair][p][p'] of an image-pair chunk, written row-major.
bool nk_seed_gemm_supported(int H, int W, int C, int filter);
size_t nk_seed_patch_bytes(int64_t n_images, int H, int W);
cudaError_t nk_seed_patches(const float* X, int64_t n, int H, int W, int C, void* patches, cudaStream_t st);
cudaError_t nk_launch_seed_gemm(const void* pa, int64_t na, const void* pb, int64_t nb, int sym, int64_t pair0,
                                int64_t np, int H, int W, int C, double sw2, double sb2, float* out, int sm,
                                unsigned int* dstatus, uint32_t wait_limit, cudaStream_t st);
size_t nk_backward_ws_bytes(const NkGeom& g, int fp64, int64_t npairs, int64_t na, int64_t nb, int sym,
                            int sm);
cudaError_t nk_launch_backward(const NkGeom& g, int fp64, double sw2, double sb2, const float* Xa,
                               const double* qda, const float* qsa, int64_t a0, int64_t a1, const float* Xb,
                               const double* qdb, const float* qsb, int64_t b0, int64_t b1, const void* dK,
                               int64_t lddk, int sym, void* dXa, void* dXb, double* dsw2, double* dsb2,
                               void* ws, int sm, uint32_t wait_limit, cudaStream_t st, int64_t* launches,
                               unsigned int* dstatus);

// Plain layer-wise Myrtle block (FP32 or FP64).
size_t nk_plain_ws_bytes(const NkGeom& g, int fp64, int64_t pairs_per_chunk);
cudaError_t nk_launch_myrtle_plain(const NkGeom& g, int fp64, double sw2, double sb2,
                                   const float* Xa, const double* qda, const float* qsa,
                                   int64_t a0, int64_t a1, const float* Xb, const double* qdb,
                                   const float* qsb, int64_t b0, int64_t b1, void* K, int64_t ldk,
                                   int symmetric, void* ws, int64_t pairs_per_chunk,
                                   unsigned int* dstatus, cudaStream_t st, int64_t* launches);
