// libnk C ABI: handle, argument validation and dispatch (declared in nk.h).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "myrtle_fused.cuh"
#include "nk_common.cuh"

nk_status nk_pcg_impl(nk_handle* h, const float* K, int64_t ldk, int64_t N, const double* Y, int R,
                      double lam, int precond, nk_prec prec, double tol, int maxit, int refine_max,
                      double* A, int* iters, double* relres, cudaStream_t st);

nk_status nk_fail(nk_handle* h, nk_status s, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof(h->err), fmt, ap);
    va_end(ap);
  }
  return s;
}

nk_status nk_cuda_check(nk_handle* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return NK_OK;
  if (e == cudaErrorMemoryAllocation) {
    (void)cudaGetLastError();
    return nk_fail(h, NK_ERR_NO_MEMORY, "%s: %s", what, cudaGetErrorString(e));
  }
  return nk_fail(h, NK_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

nk_status nk_workspace(nk_handle* h, size_t bytes, void** out) {
  if (bytes > h->ws_bytes) {
    if (h->ws) cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
    cudaError_t e = cudaMalloc(&h->ws, bytes);
    if (e != cudaSuccess) return nk_cuda_check(h, e, "workspace allocation");
    h->ws_bytes = bytes;
  }
  *out = h->ws;
  return NK_OK;
}

bool nk_make_geom(const nk_arch* arch, int H, int W, int C, NkGeom* g, const char** why) {
  memset(g, 0, sizeof(*g));
  if (!arch) { *why = "arch is NULL"; return false; }
  if (arch->n_stages < 1 || arch->n_stages > NK_MAX_STAGES) { *why = "n_stages outside 1..4"; return false; }
  if (arch->filter != 1 && arch->filter != 3) { *why = "filter must be 1 or 3"; return false; }
  if (arch->activation != NK_ACT_RELU && arch->activation != NK_ACT_IDENTITY && arch->activation != NK_ACT_ERF) {
    *why = "unknown activation";
    return false;
  }
  if (arch->norm != NK_NORM_NONE && arch->norm != NK_NORM_LAYER) { *why = "unknown norm"; return false; }
  if (arch->norm == NK_NORM_LAYER && arch->activation == NK_ACT_IDENTITY) {
    *why = "a LayerNorm needs the ReLU or Erf activation";
    return false;
  }
  if (arch->readout != NK_READOUT_GAP && arch->readout != NK_READOUT_FLATTEN) { *why = "unknown readout"; return false; }
  if (arch->readout == NK_READOUT_FLATTEN && arch->norm != NK_NORM_NONE) {
    *why = "a Flatten readout is supported without a norm only";
    return false;
  }
  if (arch->convs[0] < 1) { *why = "the first stage needs at least one conv"; return false; }
  if (H < 1 || W < 1 || C < 1) { *why = "H, W and C must be positive"; return false; }
  g->n_stages = arch->n_stages;
  g->filter = arch->filter;
  g->act = arch->activation;
  g->norm = arch->norm;
  g->readout = arch->readout;
  g->C = C;
  int h = H, w = W, nl = 0, off = 0;
  g->last_act_stage = -1;
  for (int s = 0; s < g->n_stages; ++s) {
    if (arch->convs[s] < 0) { *why = "negative conv count"; return false; }
    if (s > 0) {
      if ((h & 1) || (w & 1)) { *why = "2x2 pooling of an odd-sized image"; return false; }
      h /= 2;
      w /= 2;
    }
    g->convs[s] = arch->convs[s];
    g->Hs[s] = h;
    g->Ws[s] = w;
    for (int k = 0; k < arch->convs[s]; ++k) {
      if (nl >= NK_MAX_LAYERS) { *why = "too many layers"; return false; }
      g->layer_stage[nl] = s;
      g->layer_qoff[nl] = off;
      off += h * w;
      ++nl;
    }
    if (arch->convs[s] > 0) g->last_act_stage = s;
  }
  g->n_layers = nl;
  g->nq_base = off;
  g->nq = off + (g->norm == NK_NORM_LAYER ? nl : 0);
  g->gap_stage = g->n_stages - 1;
  int r = 0;
  for (int s = g->last_act_stage; s >= 0; --s) {
    g->radius[s] = r;
    r = 2 * r + 1;
  }
  return true;
}

namespace {

void tune_key(const NkGeom& g, bool bias, int* key) {
  key[0] = g.n_stages > 0 ? g.convs[0] : 0;
  key[1] = g.n_stages > 1 ? g.convs[1] : 0;
  key[2] = g.n_stages > 2 ? g.convs[2] : 0;
  key[3] = g.n_stages;
  key[4] = g.Hs[0];
  key[5] = g.Ws[0];
  key[6] = g.C;
  key[7] = bias ? 1 : 0;
}

int tune_lookup(const nk_handle* h, const int* key, int fallback) {
  for (int i = 0; i < h->tune_n; ++i)
    if (memcmp(h->tune_key[i], key, sizeof(int) * 8) == 0) return h->tune_variant[i];
  return fallback;
}

// Stage pattern (first three stages) of a geometry.
void stage_pattern(const NkGeom& g, int* c) {
  c[0] = g.convs[0];
  c[1] = g.n_stages > 1 ? g.convs[1] : 0;
  c[2] = g.n_stages > 2 ? g.convs[2] : 0;
}

// Launch variants of the fused form at this size: at 32x32 the three
// super-plane cluster launches, plus the tiled form (variant 3) where the
// stage pattern has one; one variant elsewhere.
bool fused_variant_valid(const NkGeom& g, int v) {
  if (g.Hs[0] != 32) return v == 0;
  if (v < 0 || v >= NK_FUSED_VARIANTS) return false;
  int c[3];
  stage_pattern(g, c);
  if (v == NK_TILED_VARIANT)
    return nkf::tiled_supported(c) || (g.act == NK_ACT_RELU && nkf::tiled3_supported(c));
  return g.act == NK_ACT_RELU && nk_cluster_pattern(c);  // the cluster launches
}

// Default variant without a tuned entry: the tiled form where it exists
// (measured faster than the cluster launches at 32x32: 1.15x for (2,1,0),
// 1.5x for Myrtle-10 (3,3,3)), else variant 0.
int fused_default_variant(const NkGeom& g) {
  return fused_variant_valid(g, NK_TILED_VARIANT) ? NK_TILED_VARIANT : 0;
}

// Bounds of the device waits (nk_set_wait_limit): the tiled queue's item waits,
// and the mbarrier waits of the FC Gram and of the adjoint's tensor-core first
// layer.
long long tiled_wait_limit(const nk_handle* h) {
  return h->wait_polls < 0 ? NK_TILED_WAIT_DEFAULT : h->wait_polls;
}
uint32_t fc_wait_limit(const nk_handle* h) {
  if (h->wait_polls < 0) return NK_FC_WAIT_DEFAULT;
  return h->wait_polls > 0xFFFFFFFFll ? 0xFFFFFFFFu : (uint32_t)h->wait_polls;
}

// One fused (MIXED) block: the tiled form at 64x64 and for variant 3, the
// super-plane cluster kernel otherwise.
nk_status fused_block(nk_handle* h, const NkGeom& g, const nk_params* prm, const float* Xa, const float* qsa,
                      int64_t a0, int64_t a1, const float* Xb, const float* qsb, int64_t b0, int64_t b1, float* K,
                      int64_t ldk, int symmetric, int variant, cudaStream_t st, const char* what) {
  if (g.Hs[0] == 64 || variant == NK_TILED_VARIANT) {
    int c[3];
    stage_pattern(g, c);
    nkf::FusedParams P = nk_fused_params(g, prm->sigma_w2, prm->sigma_b2, Xa, qsa, a0, a1, Xb, qsb, b0, b1, K,
                                         ldk, symmetric);
    const int R[1] = {g.Hs[0]};
    const int64_t np[1] = {P.npairs};
    void* ws = nullptr;
    nk_status s = nk_workspace(h, nkf::tiled_ws_bytes(c, R, np, 1, h->sm_count), &ws);
    if (s != NK_OK) return s;
    h->launches += 1;
    if (!nkf::tiled_supported(c))  // three-stage nets at 32x32
      return nk_cuda_check(h, nkf::launch_tiled3(c, prm->sigma_b2 != 0.0, false, R, &P, 1, h->sm_count, ws,
                                                 h->ws_bytes, h->dstatus, tiled_wait_limit(h), st), what);
    return nk_cuda_check(h, nkf::launch_tiled(c, prm->sigma_b2 != 0.0, g.act, R, &P, 1, h->sm_count, ws,
                                              h->ws_bytes, h->dstatus, tiled_wait_limit(h), st), what);
  }
  h->launches += 1;
  return nk_cuda_check(h, nk_launch_myrtle_fused(g, prm->sigma_w2, prm->sigma_b2, Xa, qsa, a0, a1, Xb, qsb, b0,
                                                 b1, K, ldk, symmetric, h->sm_count, h->small_ws, 65536,
                                                 variant, st), what);
}

void tune_store(nk_handle* h, const int* key, int v) {
  for (int i = 0; i < h->tune_n; ++i)
    if (memcmp(h->tune_key[i], key, sizeof(int) * 8) == 0) {
      h->tune_variant[i] = v;
      return;
    }
  const int i = (h->tune_n < 16) ? h->tune_n++ : 15;
  memcpy(h->tune_key[i], key, sizeof(int) * 8);
  h->tune_variant[i] = v;
}

// Synthetic images for timing: a counter hash mapped to [-1.7, 1.7].
__global__ void k_synth_images(float* x, int64_t n, uint32_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t v = (uint32_t)i * 0x9E3779B1u ^ seed;
    v ^= v >> 16;
    v *= 0x85EBCA6Bu;
    v ^= v >> 13;
    v *= 0xC2B2AE35u;
    v ^= v >> 16;
    x[i] = ((float)(v >> 8) * (1.0f / 16777216.0f) - 0.5f) * 3.4f;
  }
}

}  // namespace

extern "C" {

const char* nk_status_string(nk_status s) {
  switch (s) {
    case NK_OK: return "ok";
    case NK_ERR_INVALID_ARG: return "invalid argument";
    case NK_ERR_CUDA: return "CUDA error";
    case NK_ERR_NUMERICAL: return "numerical error (q <= 0 or NaN)";
    case NK_ERR_NOT_CONVERGED: return "not converged";
    case NK_ERR_TIMEOUT: return "device wait timed out";
    case NK_ERR_NO_MEMORY: return "out of device memory";
    case NK_ERR_UNSUPPORTED: return "unsupported by the library";
  }
  return "unknown status";
}

nk_status nk_create(nk_handle** out) {
  if (!out) return NK_ERR_INVALID_ARG;
  *out = nullptr;
  nk_handle* h = new nk_handle();
  memset(h, 0, sizeof(*h));
  h->pcg_rank = 100;
  h->wait_polls = -1;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) e = cudaMalloc(&h->dstatus, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(h->dstatus, 0, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&h->small_ws, 65536);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    if (h->dstatus) cudaFree(h->dstatus);
    if (h->small_ws) cudaFree(h->small_ws);
    delete h;
    return e == cudaErrorMemoryAllocation ? NK_ERR_NO_MEMORY : NK_ERR_CUDA;
  }
  *out = h;
  return NK_OK;
}

void nk_destroy(nk_handle* h) {
  if (!h) return;
  if (h->ws) cudaFree(h->ws);
  if (h->pcg_ws) cudaFree(h->pcg_ws);
  if (h->dstatus) cudaFree(h->dstatus);
  if (h->small_ws) cudaFree(h->small_ws);
  delete h;
}

nk_status nk_last_error(nk_handle* h, char* buf, size_t len) {
  if (!h || !buf || len == 0) return NK_ERR_INVALID_ARG;
  snprintf(buf, len, "%s", h->err);
  return NK_OK;
}

nk_status nk_sync_status(nk_handle* h, void* stream) {
  if (!h) return NK_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, h->dstatus, sizeof(v), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->dstatus, 0, sizeof(unsigned int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return nk_cuda_check(h, e, "nk_sync_status");
  if (v & NK_DEV_TIMEOUT) return nk_fail(h, NK_ERR_TIMEOUT, "a device wait gave up");
  if (v & NK_DEV_NUMERICAL) return nk_fail(h, NK_ERR_NUMERICAL, "q <= 0 or NaN met by a ReLU map");
  return NK_OK;
}

int64_t nk_launch_count(nk_handle* h) { return h ? h->launches : 0; }

double nk_last_lambda(nk_handle* h) { return h ? h->last_lambda : 0.0; }

int64_t nk_q_size(const nk_arch* arch, int H, int W) {
  NkGeom g;
  const char* why = nullptr;
  if (!nk_make_geom(arch, H, W, 1, &g, &why)) return -1;
  return g.nq;
}

nk_status nk_self_diag(nk_handle* h, const nk_arch* arch, const nk_params* prm, const float* X,
                       int64_t n, int H, int W, int C, double* qd, float* qs, void* stream) {
  if (!h) return NK_ERR_INVALID_ARG;
  NkGeom g;
  const char* why = nullptr;
  if (!nk_make_geom(arch, H, W, C, &g, &why)) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_self_diag: %s", why);
  if (!prm) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_self_diag: params is NULL");
  if (n < 0) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_self_diag: n < 0");
  if (n == 0) return NK_OK;
  if (!X || !qd) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_self_diag: X or qd is NULL");
  if (!(prm->sigma_w2 >= 0.0) || !(prm->sigma_b2 >= 0.0))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_self_diag: negative variance");
  const int grid = (int)std::min<int64_t>(n, 2 * (int64_t)h->sm_count);
  const size_t per = nk_self_diag_ws_per_cta(g);
  void* ws = nullptr;
  nk_status s = nk_workspace(h, per * grid, &ws);
  if (s != NK_OK) return s;
  h->launches += 1;
  cudaError_t e = nk_launch_self_diag(g, prm->sigma_w2, prm->sigma_b2, X, n, qd, qs, (double*)ws, grid,
                                      h->dstatus, (cudaStream_t)stream);
  return nk_cuda_check(h, e, "nk_self_diag launch");
}

nk_status nk_block(nk_handle* h, const nk_arch* arch, const nk_params* prm, nk_prec prec,
                   const float* Xa, const double* qda, const float* qsa, int64_t a0, int64_t a1,
                   const float* Xb, const double* qdb, const float* qsb, int64_t b0, int64_t b1,
                   int H, int W, int C, void* K, int64_t ldk, int symmetric, void* stream) {
  if (!h) return NK_ERR_INVALID_ARG;
  NkGeom g;
  const char* why = nullptr;
  if (!nk_make_geom(arch, H, W, C, &g, &why)) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block: %s", why);
  if (!prm) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block: params is NULL");
  if (!(prm->sigma_w2 >= 0.0) || !(prm->sigma_b2 >= 0.0))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block: negative variance");
  if (prec != NK_PREC_PLAIN_FP64 && prec != NK_PREC_PLAIN_FP32 && prec != NK_PREC_MIXED)
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block: unknown precision");
  if (a0 < 0 || b0 < 0 || a1 < a0 || b1 < b0)
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block: bad index range");
  if (a1 == a0 || b1 == b0) return NK_OK;
  if (!Xa || !Xb || !K) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block: NULL image or output pointer");
  if (ldk < b1 - b0) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block: ldk < b1 - b0");
  if (symmetric && (Xa != Xb || a0 != b0 || a1 != b1))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block: symmetric needs Xa == Xb and equal ranges");
  const bool needq = (g.act == NK_ACT_RELU);
  if (needq && prec == NK_PREC_PLAIN_FP64 && (!qda || !qdb))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block: PLAIN_FP64 needs qda and qdb");
  if (needq && prec != NK_PREC_PLAIN_FP64 && (!qsa || !qsb))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block: FP32 paths need qsa and qsb");
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == NK_PREC_MIXED && g.readout == NK_READOUT_FLATTEN) {
    if (!nk_cv_supported(g))
      return nk_fail(h, NK_ERR_UNSUPPORTED,
                     "nk_block MIXED with a Flatten readout: needs one stage of filter-3 convs, ReLU or Erf, "
                     "H in {8,16,32}, W <= 32, C <= 4");
    h->launches += 1;
    return nk_cuda_check(h, nk_launch_cv_diag(g, prm->sigma_w2, prm->sigma_b2, Xa, qsa, a0, a1, Xb, qsb, b0, b1,
                                              (float*)K, ldk, symmetric, h->sm_count, st),
                         "nk_block flatten-readout launch");
  }
  if (prec == NK_PREC_MIXED) {
    if (!nk_myrtle_fused_supported(g))
      return nk_fail(h, NK_ERR_UNSUPPORTED,
                     "nk_block MIXED: needs filter 3, C <= 3 and, with ReLU, H == W in {8,16,32} with one "
                     "of the stage patterns (2,1,0) (2,1,1) (3,3,3) (1) (1,1,1), or H == W in {32,64} with "
                     "(2,1,0) (1) (1,1); with Erf H == W in {32,64} and (2,1,0) (1) (1,1)");
    int key[8];
    tune_key(g, prm->sigma_b2 != 0.0, key);
    return fused_block(h, g, prm, Xa, qsa, a0, a1, Xb, qsb, b0, b1, (float*)K, ldk, symmetric,
                       tune_lookup(h, key, fused_default_variant(g)), st, "nk_block fused launch");
  }
  const int fp64 = (prec == NK_PREC_PLAIN_FP64);
  const int64_t na = a1 - a0, nb = b1 - b0;
  const int64_t npairs = symmetric ? na * (na + 1) / 2 : na * nb;
  const size_t per_pair = nk_plain_ws_bytes(g, fp64, 1);
  const size_t budget = (size_t)1 << 30;
  int64_t chunk = (int64_t)std::max<size_t>(1, budget / per_pair);
  chunk = std::min<int64_t>(chunk, npairs);
  void* ws = nullptr;
  nk_status s = nk_workspace(h, per_pair * chunk, &ws);
  if (s != NK_OK) return s;
  cudaError_t e = nk_launch_myrtle_plain(g, fp64, prm->sigma_w2, prm->sigma_b2, Xa, qda, qsa, a0, a1, Xb,
                                         qdb, qsb, b0, b1, K, ldk, symmetric, ws, chunk, h->dstatus, st,
                                         &h->launches);
  return nk_cuda_check(h, e, "nk_block plain launch");
}

nk_status nk_block_ntk(nk_handle* h, const nk_arch* arch, const nk_params* prm, nk_prec prec,
                       const float* Xa, const double* qda, const float* qsa, int64_t a0, int64_t a1,
                       const float* Xb, const double* qdb, const float* qsb, int64_t b0, int64_t b1, int H,
                       int W, int C, void* K, void* Theta, int64_t ldk, int symmetric, void* stream) {
  if (!h) return NK_ERR_INVALID_ARG;
  NkGeom g;
  const char* why = nullptr;
  if (!nk_make_geom(arch, H, W, C, &g, &why)) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_ntk: %s", why);
  if (!prm) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_ntk: params is NULL");
  if (!(prm->sigma_w2 >= 0.0) || !(prm->sigma_b2 >= 0.0))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_ntk: negative variance");
  if (g.act == NK_ACT_ERF || g.norm != NK_NORM_NONE || g.readout != NK_READOUT_GAP)
    return nk_fail(h, NK_ERR_UNSUPPORTED, "nk_block_ntk: ReLU or identity, no norm, global-average readout only");
  if (prec != NK_PREC_PLAIN_FP64 && prec != NK_PREC_PLAIN_FP32 && prec != NK_PREC_MIXED)
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_ntk: unknown precision");
  int pat[3];
  stage_pattern(g, pat);
  const bool ntk3 = nkf::tiled3_supported(pat) && g.Hs[0] == 32;
  if (prec == NK_PREC_MIXED &&
      (g.act != NK_ACT_RELU || g.filter != 3 || g.C > 3 || g.Hs[0] != g.Ws[0] ||
       !(((g.Hs[0] == 32 || g.Hs[0] == 64) && nkf::tiled_ntk_supported(pat)) || ntk3)))
    return nk_fail(h, NK_ERR_UNSUPPORTED,
                   "nk_block_ntk MIXED: needs ReLU, filter 3, C <= 3 and H == W in {32, 64} with the stage "
                   "pattern (2,1,0), or H == W == 32 with (3,3,3) or (2,1,1)");
  if (a0 < 0 || b0 < 0 || a1 < a0 || b1 < b0)
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_ntk: bad index range");
  if (a1 == a0 || b1 == b0) return NK_OK;
  if (!Xa || !Xb || !K || !Theta) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_ntk: NULL image or output");
  if (ldk < b1 - b0) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_ntk: ldk < b1 - b0");
  if (symmetric && (Xa != Xb || a0 != b0 || a1 != b1))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_ntk: symmetric needs Xa == Xb and equal ranges");
  const bool needq = (g.act == NK_ACT_RELU);
  if (needq && prec == NK_PREC_PLAIN_FP64 && (!qda || !qdb))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_ntk: PLAIN_FP64 needs qda and qdb");
  if (needq && prec != NK_PREC_PLAIN_FP64 && (!qsa || !qsb))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_ntk: FP32 paths need qsa and qsb");
  if (prec == NK_PREC_MIXED) {
    // the tiled row stream with the tangent rows beside K
    nkf::FusedParams P = nk_fused_params(g, prm->sigma_w2, prm->sigma_b2, Xa, qsa, a0, a1, Xb, qsb, b0, b1,
                                         (float*)K, ldk, symmetric);
    P.Th = (float*)Theta;
    const int R[1] = {g.Hs[0]};
    const int64_t np[1] = {P.npairs};
    void* ws = nullptr;
    nk_status s = nk_workspace(h, nkf::tiled_ws_bytes(pat, R, np, 1, h->sm_count, 2), &ws);
    if (s != NK_OK) return s;
    h->launches += 1;
    if (ntk3)
      return nk_cuda_check(h,
                           nkf::launch_tiled3(pat, prm->sigma_b2 != 0.0, true, R, &P, 1, h->sm_count, ws,
                                              h->ws_bytes, h->dstatus, tiled_wait_limit(h), (cudaStream_t)stream),
                           "nk_block_ntk tiled launch");
    return nk_cuda_check(h,
                         nkf::launch_tiled_ntk(pat, prm->sigma_b2 != 0.0, R, &P, 1, h->sm_count, ws, h->ws_bytes,
                                               h->dstatus, tiled_wait_limit(h), (cudaStream_t)stream),
                         "nk_block_ntk tiled launch");
  }
  const int fp64 = (prec == NK_PREC_PLAIN_FP64);
  const int64_t na = a1 - a0, nb = b1 - b0;
  const int64_t npairs = symmetric ? na * (na + 1) / 2 : na * nb;
  const size_t per_pair = 2 * nk_plain_ws_bytes(g, fp64, 1);
  const size_t budget = (size_t)1 << 30;
  int64_t chunk = (int64_t)std::max<size_t>(1, budget / per_pair);
  chunk = std::min<int64_t>(chunk, npairs);
  void* ws = nullptr;
  nk_status s = nk_workspace(h, per_pair * chunk, &ws);
  if (s != NK_OK) return s;
  cudaError_t e = nk_launch_myrtle_plain_ntk(g, fp64, prm->sigma_w2, prm->sigma_b2, Xa, qda, qsa, a0, a1, Xb, qdb,
                                             qsb, b0, b1, K, Theta, ldk, symmetric, ws, chunk, h->dstatus,
                                             (cudaStream_t)stream, &h->launches);
  return nk_cuda_check(h, e, "nk_block_ntk launch");
}

nk_status nk_block_queue(nk_handle* h, const nk_arch* arch, const nk_params* prm, int C,
                         const nk_block_task* tasks, int n_tasks, void* stream) {
  if (!h) return NK_ERR_INVALID_ARG;
  if (!prm) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_queue: params is NULL");
  if (!(prm->sigma_w2 >= 0.0) || !(prm->sigma_b2 >= 0.0))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_queue: negative variance");
  if (n_tasks < 0 || n_tasks > NK_QUEUE_MAX)
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_queue: n_tasks outside 0..%d", NK_QUEUE_MAX);
  if (n_tasks > 0 && !tasks) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_queue: tasks is NULL");
  // validate every block before anything is enqueued
  struct Item {
    int R;
    nkf::FusedParams P;
  } items[NK_QUEUE_MAX];
  int n = 0;
  int c[3] = {0, 0, 0};
  int act = NK_ACT_RELU;
  for (int t = 0; t < n_tasks; ++t) {
    const nk_block_task& T = tasks[t];
    NkGeom g;
    const char* why = nullptr;
    if (!nk_make_geom(arch, T.H, T.W, C, &g, &why))
      return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_queue task %d: %s", t, why);
    if (T.a0 < 0 || T.b0 < 0 || T.a1 < T.a0 || T.b1 < T.b0)
      return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_queue task %d: bad index range", t);
    if (T.a1 == T.a0 || T.b1 == T.b0) continue;
    if (!T.Xa || !T.Xb || !T.K || !T.qsa || !T.qsb)
      return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_queue task %d: NULL pointer", t);
    if (T.ldk < T.b1 - T.b0) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_queue task %d: ldk < b1 - b0", t);
    if (T.symmetric && (T.Xa != T.Xb || T.a0 != T.b0 || T.a1 != T.b1))
      return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_queue task %d: symmetric needs Xa == Xb and equal ranges",
                     t);
    if (!nk_myrtle_fused_supported(g))
      return nk_fail(h, NK_ERR_UNSUPPORTED,
                     "nk_block_queue task %d: needs filter 3, C <= 3 and, with ReLU, H == W in {8,16,32} with "
                     "one of the stage patterns (2,1,0) (2,1,1) (3,3,3) (1) (1,1,1), or 64 with (2,1,0) (1) "
                     "(1,1); with Erf 64x64 and 32x32 blocks of (2,1,0) (1) (1,1)",
                     t);
    c[0] = g.convs[0];
    c[1] = g.n_stages > 1 ? g.convs[1] : 0;
    c[2] = g.n_stages > 2 ? g.convs[2] : 0;
    act = g.act;
    items[n].R = T.H;
    items[n].P = nk_fused_params(g, prm->sigma_w2, prm->sigma_b2, T.Xa, T.qsa, T.a0, T.a1, T.Xb, T.qsb, T.b0,
                                 T.b1, T.K, T.ldk, T.symmetric);
    ++n;
  }
  if (n == 0) return NK_OK;
  // largest images first (their items are the longest)
  std::stable_sort(items, items + n, [](const Item& x, const Item& y) { return x.R > y.R; });
  if (items[0].R == 64) {
    // 64x64 blocks: the tiled form, which also takes the 32x32 blocks
    int R[NK_QUEUE_MAX];
    int64_t np[NK_QUEUE_MAX];
    nkf::FusedParams B[NK_QUEUE_MAX];
    for (int b = 0; b < n; ++b) {
      if (items[b].R != 64 && items[b].R != 32)
        return nk_fail(h, NK_ERR_UNSUPPORTED,
                       "nk_block_queue: a queue with 64x64 blocks takes 64x64 and 32x32 blocks only");
      R[b] = items[b].R;
      np[b] = items[b].P.npairs;
      B[b] = items[b].P;
    }
    if (!nkf::tiled_supported(c))
      return nk_fail(h, NK_ERR_UNSUPPORTED,
                     "nk_block_queue: a queue with 64x64 blocks needs the stage pattern (2,1,0) (1) or (1,1)");
    void* ws = nullptr;
    nk_status s = nk_workspace(h, nkf::tiled_ws_bytes(c, R, np, n, h->sm_count), &ws);
    if (s != NK_OK) return s;
    h->launches += 1;
    cudaError_t e = nkf::launch_tiled(c, prm->sigma_b2 != 0.0, act, R, B, n, h->sm_count, ws, h->ws_bytes,
                                      h->dstatus, tiled_wait_limit(h), (cudaStream_t)stream);
    return nk_cuda_check(h, e, "nk_block_queue tiled launch");
  }
  if (act != NK_ACT_RELU || !nk_cluster_pattern(c))
    return nk_fail(h, NK_ERR_UNSUPPORTED,
                   "nk_block_queue: without 64x64 blocks the queue takes ReLU networks of the patterns (2,1,0) "
                   "(2,1,1) (3,3,3) (1) (1,1,1)");
  nkf::QueueParams Q = {};
  Q.n = n;
  Q.item0[0] = 0;
  for (int b = 0; b < n; ++b) {
    Q.R[b] = items[b].R;
    Q.B[b] = items[b].P;
    const int64_t np = items[b].P.npairs;
    const int64_t nit = (items[b].R == 32) ? np : (np + nkf::QUEUE_CL - 1) / nkf::QUEUE_CL;
    Q.item0[b + 1] = Q.item0[b] + nit;
  }
  h->launches += 1;
  cudaError_t e = nkf::launch_queue(c, prm->sigma_b2 != 0.0, Q, h->sm_count, h->small_ws, 65536,
                                    (cudaStream_t)stream);
  return nk_cuda_check(h, e, "nk_block_queue launch");
}

nk_status nk_block_backward(nk_handle* h, const nk_arch* arch, const nk_params* prm, nk_prec prec,
                            const float* Xa, const double* qda, const float* qsa, int64_t a0, int64_t a1,
                            const float* Xb, const double* qdb, const float* qsb, int64_t b0, int64_t b1,
                            int H, int W, int C, const void* dK, int64_t lddk, int symmetric, void* dXa,
                            void* dXb, double* dsw2, double* dsb2, void* stream) {
  if (!h) return NK_ERR_INVALID_ARG;
  NkGeom g;
  const char* why = nullptr;
  if (!nk_make_geom(arch, H, W, C, &g, &why))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_backward: %s", why);
  if (!prm || !(prm->sigma_w2 > 0.0) || !(prm->sigma_b2 >= 0.0))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_backward: needs sigma_w2 > 0 and sigma_b2 >= 0");
  if (prec != NK_PREC_PLAIN_FP64 && prec != NK_PREC_PLAIN_FP32 && prec != NK_PREC_MIXED)
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_backward: unknown precision");
  if (C > 4) return nk_fail(h, NK_ERR_UNSUPPORTED, "nk_block_backward: C > 4");
  bool widths_ok = g.filter == 3;
  for (int s = 0; s <= g.last_act_stage && s < g.n_stages; ++s) {
    const int w = g.Ws[s];
    if (w != 1 && w != 2 && w != 4 && w != 8 && w != 16 && w != 32 && w != 64) widths_ok = false;
    if (g.Hs[s] != w) widths_ok = false;  // square stages
  }
  if (!widths_ok)
    return nk_fail(h, NK_ERR_UNSUPPORTED,
                   "nk_block_backward: needs 3x3 filters and square stages of side 1, 2, 4, ..., 64");
  if (g.act == NK_ACT_ERF || g.norm != NK_NORM_NONE || g.readout != NK_READOUT_GAP)
    return nk_fail(h, NK_ERR_UNSUPPORTED,
                   "nk_block_backward: ReLU or identity, no norm, global-average readout only");
  if (a0 < 0 || b0 < 0 || a1 < a0 || b1 < b0)
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_backward: bad index range");
  if (a1 == a0 || b1 == b0) return NK_OK;
  if (!Xa || !Xb || !dK || !dsw2 || !dsb2)
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_backward: NULL image, dK or dsigma pointer");
  if (lddk < b1 - b0) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_backward: lddk < b1 - b0");
  if (symmetric && (Xa != Xb || a0 != b0 || a1 != b1 || dXa != dXb))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_backward: symmetric needs Xa == Xb, equal ranges, dXa == dXb");
  const bool relu = (g.act == NK_ACT_RELU);
  const int fp64 = (prec == NK_PREC_PLAIN_FP64);
  if (relu && (!qda || !qdb || (!fp64 && (!qsa || !qsb))))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_block_backward: needs qda, qdb (and qsa, qsb for FP32)");
  const int64_t na = a1 - a0, nb = b1 - b0;
  const int64_t npairs = symmetric ? na * (na + 1) / 2 : na * nb;
  void* ws = nullptr;
  nk_status s = nk_workspace(h, nk_backward_ws_bytes(g, fp64, npairs, na, nb, symmetric, h->sm_count), &ws);
  if (s != NK_OK) return s;
  cudaError_t e = nk_launch_backward(g, fp64, prm->sigma_w2, prm->sigma_b2, Xa, qda, qsa, a0, a1, Xb, qdb, qsb,
                                     b0, b1, dK, lddk, symmetric, dXa, dXb, dsw2, dsb2, ws, h->sm_count,
                                     fc_wait_limit(h), (cudaStream_t)stream, &h->launches, h->dstatus);
  return nk_cuda_check(h, e, "nk_block_backward");
}

nk_status nk_fc_block(nk_handle* h, int depth, const nk_params* prm, const float* Xa, int64_t a0, int64_t a1,
                      const float* Xb, int64_t b0, int64_t b1, int d, float* K, int64_t ldk, int symmetric,
                      void* stream) {
  if (!h) return NK_ERR_INVALID_ARG;
  if (depth < 0 || depth > 8) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_fc_block: depth outside 0..8");
  if (!prm || !(prm->sigma_w2 >= 0.0) || !(prm->sigma_b2 >= 0.0))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_fc_block: bad params");
  if (d < 1) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_fc_block: d < 1");
  if (a0 < 0 || b0 < 0 || a1 < a0 || b1 < b0)
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_fc_block: bad index range");
  if (a1 == a0 || b1 == b0) return NK_OK;
  if (!Xa || !Xb || !K) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_fc_block: NULL pointer");
  if (ldk < b1 - b0) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_fc_block: ldk < b1 - b0");
  if (symmetric && (Xa != Xb || a0 != b0 || a1 != b1))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_fc_block: symmetric needs Xa == Xb and equal ranges");
  if (a1 - a0 > (1 << 30) || b1 - b0 > (1 << 30))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_fc_block: more than 2^30 rows");
  void* ws = nullptr;
  nk_status s = nk_workspace(h, nk_fc_ws_bytes(a1 - a0, b1 - b0, d, depth), &ws);
  if (s != NK_OK) return s;
  cudaError_t e = nk_launch_fc_block(depth, prm->sigma_w2, prm->sigma_b2, Xa, a0, a1, Xb, b0, b1, d, K, ldk,
                                     symmetric, ws, h->sm_count, h->dstatus, fc_wait_limit(h), (cudaStream_t)stream,
                                     &h->launches);
  if (e == cudaErrorInvalidValue) return nk_fail(h, NK_ERR_CUDA, "nk_fc_block: tensor map encoding failed");
  if (e == cudaErrorInvalidConfiguration)
    return nk_fail(h, NK_ERR_CUDA, "nk_fc_block: the Gram kernel was built with another register count than its "
                                   "warpgroup register split assumes");
  return nk_cuda_check(h, e, "nk_fc_block");
}

nk_status nk_autotune(nk_handle* h, const nk_arch* arch, const nk_params* prm, int H, int W, int C,
                      int* variant, void* stream) {
  if (!h) return NK_ERR_INVALID_ARG;
  NkGeom g;
  const char* why = nullptr;
  if (!nk_make_geom(arch, H, W, C, &g, &why)) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_autotune: %s", why);
  if (!prm || !(prm->sigma_w2 >= 0.0) || !(prm->sigma_b2 >= 0.0))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_autotune: bad params");
  if (!nk_myrtle_fused_supported(g))
    return nk_fail(h, NK_ERR_UNSUPPORTED, "nk_autotune: no fused kernel for this architecture / size");
  int key[8];
  tune_key(g, prm->sigma_b2 != 0.0, key);
  const int nvar = (g.Hs[0] == 32) ? NK_FUSED_VARIANTS : 1;
  if (nvar == 1) {
    const int v = fused_default_variant(g);
    tune_store(h, key, v);
    if (variant) *variant = v;
    return NK_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // synthetic block: na x nb pairs, about four pairs per 4-CTA cluster
  const int na = 12, nb = 12, n = na + nb;
  const size_t nimg = (size_t)n * H * W * C;
  float* X = nullptr;
  double* qd = nullptr;
  float* qs = nullptr;
  float* K = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  nk_status ret = NK_OK;
  cudaError_t e = cudaMalloc(&X, nimg * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&qd, (size_t)n * g.nq * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&qs, (size_t)n * g.nq * 2 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&K, (size_t)na * nb * sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int best = 0;
  if (e == cudaSuccess) {
    ++h->launches;
    k_synth_images<<<64, 256, 0, st>>>(X, (int64_t)nimg, 0x1234567u);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    nk_status s = nk_self_diag(h, arch, prm, X, n, H, W, C, qd, qs, stream);
    if (s != NK_OK) ret = s;
  }
  float best_ms = 1e30f;
  for (int v = 0; v < nvar && e == cudaSuccess && ret == NK_OK; ++v) {
    if (!fused_variant_valid(g, v)) continue;
    float ms_min = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess && ret == NK_OK; ++rep) {
      e = cudaEventRecord(e0, st);
      if (e == cudaSuccess)
        ret = fused_block(h, g, prm, X, qs, 0, na, X, qs, na, n, K, nb, 0, v, st, "nk_autotune");
      if (ret != NK_OK) break;
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < ms_min) ms_min = ms;  // first run warms up
    }
    if (e == cudaSuccess && ms_min < best_ms) {
      best_ms = ms_min;
      best = v;
    }
  }
  if (e != cudaSuccess && ret == NK_OK) ret = nk_cuda_check(h, e, "nk_autotune");
  if (ret == NK_OK) {
    tune_store(h, key, best);
    if (variant) *variant = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(X);
  cudaFree(qd);
  cudaFree(qs);
  cudaFree(K);
  return ret;
}

nk_status nk_autotune_set(nk_handle* h, const nk_arch* arch, const nk_params* prm, int H, int W, int C,
                          int variant) {
  if (!h) return NK_ERR_INVALID_ARG;
  NkGeom g;
  const char* why = nullptr;
  if (!nk_make_geom(arch, H, W, C, &g, &why)) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_autotune_set: %s", why);
  if (!prm) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_autotune_set: params is NULL");
  if (!fused_variant_valid(g, variant))
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_autotune_set: variant %d does not exist for this size and stage "
                   "pattern (0..%d at 32x32, 3 = tiled for (2,1,0) and (1); 0 elsewhere)", variant,
                   NK_FUSED_VARIANTS - 1);
  int key[8];
  tune_key(g, prm->sigma_b2 != 0.0, key);
  tune_store(h, key, variant);
  return NK_OK;
}

nk_status nk_set_wait_limit(nk_handle* h, int64_t polls) {
  if (!h) return NK_ERR_INVALID_ARG;
  h->wait_polls = polls < 0 ? -1 : (long long)polls;
  return NK_OK;
}

nk_status nk_pcg_set_warm_start(nk_handle* h, int on) {
  if (!h) return NK_ERR_INVALID_ARG;
  h->pcg_warm = on != 0;
  return NK_OK;
}

nk_status nk_pcg_set_rank(nk_handle* h, int rank) {
  if (!h) return NK_ERR_INVALID_ARG;
  if (rank < 1 || rank > 1024) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_pcg_set_rank: rank outside 1..1024");
  h->pcg_rank = rank;
  return NK_OK;
}

nk_status nk_pcg_solve(nk_handle* h, const float* K, int64_t ldk, int64_t N, const double* Y, int R,
                       double lambda, int precond, nk_prec prec, double tol, int maxit, int refine_max,
                       double* A, int* iters, double* relres, void* stream) {
  if (!h) return NK_ERR_INVALID_ARG;
  if (iters) *iters = 0;
  if (N < 0 || R < 0) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_pcg_solve: negative size");
  if (N == 0 || R == 0) return NK_OK;
  if (R > 256) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_pcg_solve: R > 256");
  if (!K || !Y || !A) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_pcg_solve: NULL pointer");
  if (ldk < N) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_pcg_solve: ldk < N");
  if (lambda != lambda) return nk_fail(h, NK_ERR_INVALID_ARG, "nk_pcg_solve: lambda is NaN");
  if (precond != NK_PRECOND_NONE && precond != NK_PRECOND_JACOBI && precond != NK_PRECOND_PIVCHOL)
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_pcg_solve: unknown preconditioner");
  if (prec != NK_PREC_PLAIN_FP64 && prec != NK_PREC_PLAIN_FP32 && prec != NK_PREC_MIXED)
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_pcg_solve: unknown precision");
  if (!(tol >= 0.0) || maxit < 0 || refine_max < 0)
    return nk_fail(h, NK_ERR_INVALID_ARG, "nk_pcg_solve: bad tol / maxit / refine_max");
  return nk_pcg_impl(h, K, ldk, N, Y, R, lambda, precond, prec, tol, maxit, refine_max, A, iters, relres,
                     (cudaStream_t)stream);
}

}  // extern "C"
