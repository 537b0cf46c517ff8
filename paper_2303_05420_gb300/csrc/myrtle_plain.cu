// Plain layer-wise Myrtle NNGP block (NK_PREC_PLAIN_FP32 / NK_PREC_PLAIN_FP64).
//
// The straightforward GPU form: the full pixel-pair tensor K[pair][p][p'] of
// every layer of the Appendix A Myrtle listing is materialised in HBM and each
// layer is one launch (input covariance, conv, ReLU map, 2x2 pool, global
// average pool + Dense readout).  Pairs are processed in chunks.  It handles
// every architecture nk_block accepts (any filter, identity activation,
// zero-conv stages) and serves as the baseline the fused path is measured
// against.  FP32 uses CUDA's acosf / asinf / sqrtf; FP64 uses acos / asin /
// sqrt.  Activations ReLU, Erf or identity, with or without a LayerNorm.
#include "myrtle_plain.cuh"

namespace {

using namespace nkp;

template <typename T>
cudaError_t run_plain(const NkGeom& g, double sw2, double sb2, const float* Xa, const double* qda,
                      const float* qsa, int64_t a0, int64_t a1, const float* Xb, const double* qdb,
                      const float* qsb, int64_t b0, int64_t b1, T* K, int64_t ldk, int symmetric,
                      void* ws, int64_t chunk, unsigned int* dstatus, cudaStream_t st,
                      int64_t* launches) {
  const int64_t na = a1 - a0, nb = b1 - b0;
  const int64_t npairs_total = symmetric ? na * (na + 1) / 2 : na * nb;
  const int64_t HW0 = (int64_t)g.Hs[0] * g.Ws[0];
  T* buf0 = reinterpret_cast<T*>(ws);
  T* buf1 = buf0 + chunk * HW0 * HW0;
  const T a_conv = (T)(sw2 / (double)(g.filter * g.filter));
  for (int64_t pair0 = 0; pair0 < npairs_total; pair0 += chunk) {
    const int64_t np = (npairs_total - pair0 < chunk) ? npairs_total - pair0 : chunk;
    T* cur = buf0;
    T* nxt = buf1;
    *launches += 2;  // input covariance + global average
    k_input_cov<T><<<pair_grid(np, HW0 * HW0), 256, 0, st>>>(Xa, Xb, a0, b0, na, nb, symmetric,
                                                             pair0, np, g.Hs[0], g.Ws[0], g.C, cur);
    int layer = 0;
    int H = g.Hs[0], W = g.Ws[0];
    for (int s = 0; s < g.n_stages; ++s) {
      if (s > 0) {
        ++*launches;
        k_pool<T><<<grid_for(np * (int64_t)(H / 2) * (W / 2) * (H / 2) * (W / 2)), 256, 0, st>>>(
            cur, nxt, np, H, W);
        T* t = cur; cur = nxt; nxt = t;
        H /= 2;
        W /= 2;
      }
      const int64_t HW = (int64_t)H * W;
      for (int k = 0; k < g.convs[s]; ++k, ++layer) {
        const bool act = (g.act == NK_ACT_RELU || g.act == NK_ACT_ERF);
        *launches += act ? 2 : 1;
        conv_layer<T>(cur, nxt, np, H, W, g.filter, a_conv, (T)sb2, st);
        T* t = cur; cur = nxt; nxt = t;
        if (act)
          k_act<T><<<pair_grid(np, HW * HW), 256, 0, st>>>(
              cur, np, (int)HW, na, nb, symmetric, pair0, a0, b0, qda, qdb, qsa, qsb, g.nq, g.layer_qoff[layer],
              g.act, g.norm == NK_NORM_LAYER ? g.nq_base + layer : -1, dstatus);
      }
    }
    const int64_t HW = (int64_t)H * W;
    if (g.readout == NK_READOUT_FLATTEN)
      k_flatten<T><<<(unsigned)np, 256, 0, st>>>(cur, (int)HW, na, nb, symmetric, pair0, (T)sw2, (T)sb2, K, ldk);
    else
      k_gap<T><<<(unsigned)np, 256, 0, st>>>(cur, HW * HW, na, nb, symmetric, pair0, (T)sw2, (T)sb2, K, ldk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Layer-wise NTK: the NNGP tensor K and the tangent tensor Theta side by side
// (Theta_0 = 0; conv: Theta' = K' + a S(Theta_t); ReLU: Theta_t = Theta
// E[relu' relu']; pools on both; readout Theta = K + sw2 mean Theta_t).
template <typename T>
cudaError_t run_plain_ntk(const NkGeom& g, double sw2, double sb2, const float* Xa, const double* qda,
                          const float* qsa, int64_t a0, int64_t a1, const float* Xb, const double* qdb,
                          const float* qsb, int64_t b0, int64_t b1, T* K, T* Th, int64_t ldk, int symmetric,
                          void* ws, int64_t chunk, unsigned int* dstatus, cudaStream_t st, int64_t* launches) {
  const int64_t na = a1 - a0, nb = b1 - b0;
  const int64_t npairs_total = symmetric ? na * (na + 1) / 2 : na * nb;
  const int64_t HW0 = (int64_t)g.Hs[0] * g.Ws[0];
  T* kb0 = reinterpret_cast<T*>(ws);
  T* kb1 = kb0 + chunk * HW0 * HW0;
  T* tb0 = kb1 + chunk * HW0 * HW0;
  T* tb1 = tb0 + chunk * HW0 * HW0;
  const T a_conv = (T)(sw2 / (double)(g.filter * g.filter));
  for (int64_t pair0 = 0; pair0 < npairs_total; pair0 += chunk) {
    const int64_t np = (npairs_total - pair0 < chunk) ? npairs_total - pair0 : chunk;
    T *kc = kb0, *kn = kb1, *tc = tb0, *tn = tb1;
    *launches += 2;
    k_input_cov<T><<<pair_grid(np, HW0 * HW0), 256, 0, st>>>(Xa, Xb, a0, b0, na, nb, symmetric, pair0, np,
                                                             g.Hs[0], g.Ws[0], g.C, kc);
    cudaError_t e = cudaMemsetAsync(tc, 0, (size_t)np * HW0 * HW0 * sizeof(T), st);
    if (e != cudaSuccess) return e;
    int layer = 0;
    int H = g.Hs[0], W = g.Ws[0];
    for (int s = 0; s < g.n_stages; ++s) {
      if (s > 0) {
        const unsigned grid = grid_for(np * (int64_t)(H / 2) * (W / 2) * (H / 2) * (W / 2));
        *launches += 2;
        k_pool<T><<<grid, 256, 0, st>>>(kc, kn, np, H, W);
        k_pool<T><<<grid, 256, 0, st>>>(tc, tn, np, H, W);
        T* t = kc; kc = kn; kn = t;
        t = tc; tc = tn; tn = t;
        H /= 2;
        W /= 2;
      }
      const int64_t HW = (int64_t)H * W;
      for (int k = 0; k < g.convs[s]; ++k, ++layer) {
        *launches += 2;
        conv_layer<T>(kc, kn, np, H, W, g.filter, a_conv, (T)sb2, st);
        conv_layer<T>(tc, tn, np, H, W, g.filter, a_conv, (T)0, st, kn);  // + K'
        T* t = kc; kc = kn; kn = t;
        t = tc; tc = tn; tn = t;
        if (g.act == NK_ACT_RELU) {
          ++*launches;
          k_relu_ntk<T><<<pair_grid(np, HW * HW), 256, 0, st>>>(kc, tc, np, (int)HW, na, nb, symmetric, pair0,
                                                                a0, b0, qda, qdb, qsa, qsb, g.nq,
                                                                g.layer_qoff[layer], dstatus);
        }
      }
    }
    const int64_t HW = (int64_t)H * W;
    k_gap_ntk<T><<<(unsigned)np, 256, 0, st>>>(kc, tc, HW * HW, na, nb, symmetric, pair0, sw2, sb2, K, Th, ldk);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

size_t nk_plain_ws_bytes(const NkGeom& g, int fp64, int64_t chunk) {
  const size_t HW0 = (size_t)g.Hs[0] * g.Ws[0];
  return 2 * (size_t)chunk * HW0 * HW0 * (fp64 ? 8 : 4);
}

cudaError_t nk_launch_myrtle_plain(const NkGeom& g, int fp64, double sw2, double sb2,
                                   const float* Xa, const double* qda, const float* qsa,
                                   int64_t a0, int64_t a1, const float* Xb, const double* qdb,
                                   const float* qsb, int64_t b0, int64_t b1, void* K, int64_t ldk,
                                   int symmetric, void* ws, int64_t chunk, unsigned int* dstatus,
                                   cudaStream_t st, int64_t* launches) {
  if (fp64)
    return run_plain<double>(g, sw2, sb2, Xa, qda, qsa, a0, a1, Xb, qdb, qsb, b0, b1,
                             reinterpret_cast<double*>(K), ldk, symmetric, ws, chunk, dstatus, st, launches);
  return run_plain<float>(g, sw2, sb2, Xa, qda, qsa, a0, a1, Xb, qdb, qsb, b0, b1,
                          reinterpret_cast<float*>(K), ldk, symmetric, ws, chunk, dstatus, st, launches);
}

cudaError_t nk_launch_myrtle_plain_ntk(const NkGeom& g, int fp64, double sw2, double sb2, const float* Xa,
                                       const double* qda, const float* qsa, int64_t a0, int64_t a1,
                                       const float* Xb, const double* qdb, const float* qsb, int64_t b0,
                                       int64_t b1, void* K, void* Th, int64_t ldk, int symmetric, void* ws,
                                       int64_t chunk, unsigned int* dstatus, cudaStream_t st, int64_t* launches) {
  if (fp64)
    return run_plain_ntk<double>(g, sw2, sb2, Xa, qda, qsa, a0, a1, Xb, qdb, qsb, b0, b1,
                                 reinterpret_cast<double*>(K), reinterpret_cast<double*>(Th), ldk, symmetric, ws,
                                 chunk, dstatus, st, launches);
  return run_plain_ntk<float>(g, sw2, sb2, Xa, qda, qsa, a0, a1, Xb, qdb, qsb, b0, b1, reinterpret_cast<float*>(K),
                              reinterpret_cast<float*>(Th), ldk, symmetric, ws, chunk, dstatus, st, launches);
}
