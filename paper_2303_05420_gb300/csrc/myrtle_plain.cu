// Plain layer-wise Myrtle NNGP block (NK_PREC_PLAIN_FP32 / NK_PREC_PLAIN_FP64).
//
// The straightforward GPU form: the full pixel-pair tensor K[pair][p][p'] of
// every layer of the Appendix A Myrtle listing is materialised in HBM and each
// layer is one launch (input covariance, conv, ReLU map, 2x2 pool, global
// average pool + Dense readout).  Pairs are processed in chunks.  It handles
// every architecture nk_block accepts (any filter, identity activation,
// zero-conv stages) and serves as the baseline the fused path is measured
// against.  FP32 uses CUDA's acosf / sqrtf; FP64 uses acos / sqrt.
#include "nk_common.cuh"
#include "nk_map.cuh"

namespace {

// Maps a linear pair index of the block to (i, j).  Symmetric blocks
// enumerate the upper triangle (j >= i) row by row.
__device__ __forceinline__ void pair_of(int64_t idx, int64_t na, int64_t nb, int symmetric,
                                        int64_t* i, int64_t* j) {
  if (!symmetric) {
    *i = idx / nb;
    *j = idx - (*i) * nb;
    return;
  }
  const double m = (double)na;
  double t = (2.0 * m + 1.0) * (2.0 * m + 1.0) - 8.0 * (double)idx;
  int64_t r = (int64_t)floor(((2.0 * m + 1.0) - sqrt(t > 0 ? t : 0)) / 2.0);
  if (r < 0) r = 0;
  if (r > na - 1) r = na - 1;
  // S(r) = r*m - r(r-1)/2 is the first index of row r
  for (int it = 0; it < 4 && r > 0 && r * na - r * (r - 1) / 2 > idx; ++it) --r;
  for (int it = 0; it < 4 && r + 1 < na && (r + 1) * na - (r + 1) * r / 2 <= idx; ++it) ++r;
  *i = r;
  *j = r + (idx - (r * na - r * (r - 1) / 2));
}

template <typename T>
__global__ void k_input_cov(const float* __restrict__ Xa, const float* __restrict__ Xb,
                            int64_t a0, int64_t b0, int64_t na, int64_t nb, int symmetric,
                            int64_t pair0, int64_t npairs, int H, int W, int C, T* __restrict__ out) {
  const int64_t HW = (int64_t)H * W, HW2 = HW * HW;
  const int64_t total = npairs * HW2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pr = e / HW2, rem = e - pr * HW2;
    const int64_t p = rem / HW, pp = rem - p * HW;
    int64_t i, j;
    pair_of(pair0 + pr, na, nb, symmetric, &i, &j);
    const float* x = Xa + (a0 + i) * HW * C + p * C;
    const float* y = Xb + (b0 + j) * HW * C + pp * C;
    T acc = 0;
    for (int c = 0; c < C; ++c) acc += (T)x[c] * (T)y[c];
    out[e] = acc / (T)C;
  }
}

template <typename T>
__global__ void k_conv(const T* __restrict__ in, T* __restrict__ out, int64_t npairs, int H, int W,
                       int filt, T a, T b) {
  const int64_t HW = (int64_t)H * W, HW2 = HW * HW;
  const int64_t total = npairs * HW2;
  const int r = filt / 2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pr = e / HW2, rem = e - pr * HW2;
    const int p = (int)(rem / HW), pp = (int)(rem - (int64_t)p * HW);
    const int i = p / W, j = p % W, k = pp / W, l = pp % W;
    T acc = 0;
    for (int dy = -r; dy <= r; ++dy)
      for (int dx = -r; dx <= r; ++dx) {
        const int i2 = i + dy, j2 = j + dx, k2 = k + dy, l2 = l + dx;
        if (i2 >= 0 && i2 < H && j2 >= 0 && j2 < W && k2 >= 0 && k2 < H && l2 >= 0 && l2 < W)
          acc += in[pr * HW2 + (int64_t)(i2 * W + j2) * HW + k2 * W + l2];
      }
    out[e] = a * acc + b;
  }
}

// ReLU map with self-variances of the pair's two images at this layer.
template <typename T>
__global__ void k_relu(T* __restrict__ K, int64_t npairs, int HW, int64_t na, int64_t nb,
                       int symmetric, int64_t pair0, int64_t a0, int64_t b0,
                       const double* __restrict__ qda, const double* __restrict__ qdb,
                       const float* __restrict__ qsa, const float* __restrict__ qsb, int64_t nq,
                       int qoff, unsigned int* dstatus) {
  const int64_t HW2 = (int64_t)HW * HW, total = npairs * HW2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pr = e / HW2, rem = e - pr * HW2;
    const int p = (int)(rem / HW), pp = (int)(rem - (int64_t)p * HW);
    int64_t i, j;
    pair_of(pair0 + pr, na, nb, symmetric, &i, &j);
    if constexpr (sizeof(T) == 8) {
      const double q1 = qda[(a0 + i) * nq + qoff + p];
      const double q2 = qdb[(b0 + j) * nq + qoff + pp];
      if (!(q1 >= 0.0) || !(q2 >= 0.0)) atomicOr(dstatus, NK_DEV_NUMERICAL);
      K[e] = nk_relu_map_f64(K[e], q1, q2);
    } else {
      const float2 s1 = reinterpret_cast<const float2*>(qsa)[(a0 + i) * nq + qoff + p];
      const float2 s2 = reinterpret_cast<const float2*>(qsb)[(b0 + j) * nq + qoff + pp];
      const float s = s1.y * s2.y;
      float v = 0.f;
      if (s > 0.f) {
        float c = K[e] * (s1.x * s2.x);
        c = fminf(fmaxf(c, -1.f), 1.f);
        v = s * (0.15915494309189533577f) *
            (sqrtf(fmaxf(1.f - c * c, 0.f)) + c * (NK_PI_F - acosf(c)));
      }
      K[e] = v;
    }
  }
}

template <typename T>
__global__ void k_pool(const T* __restrict__ in, T* __restrict__ out, int64_t npairs, int H, int W) {
  const int Ho = H / 2, Wo = W / 2;
  const int64_t HW = (int64_t)H * W, HWo = (int64_t)Ho * Wo;
  const int64_t total = npairs * HWo * HWo;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pr = e / (HWo * HWo), rem = e - pr * HWo * HWo;
    const int P = (int)(rem / HWo), PP = (int)(rem - (int64_t)P * HWo);
    const int I = P / Wo, J = P % Wo, K2 = PP / Wo, L = PP % Wo;
    T acc = 0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        for (int c = 0; c < 2; ++c)
          for (int d = 0; d < 2; ++d)
            acc += in[pr * HW * HW + (int64_t)((2 * I + a) * W + 2 * J + b) * HW +
                      (2 * K2 + c) * W + 2 * L + d];
    out[e] = acc / (T)16;
  }
}

template <typename T>
__global__ void k_gap(const T* __restrict__ in, int64_t HW2, int64_t na, int64_t nb, int symmetric,
                      int64_t pair0, T sw2, T sb2, T* __restrict__ K, int64_t ldk) {
  __shared__ double red[32];
  const int64_t pr = blockIdx.x;
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < HW2; e += blockDim.x) acc += (double)in[pr * HW2 + e];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) {
      int64_t i, j;
      pair_of(pair0 + pr, na, nb, symmetric, &i, &j);
      const T v = (T)((double)sw2 * (acc / (double)HW2) + (double)sb2);
      K[i * ldk + j] = v;
      if (symmetric && i != j) K[j * ldk + i] = v;
    }
  }
}

inline int grid_for(int64_t total) {
  int64_t g = (total + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  if (g < 1) g = 1;
  return (int)g;
}

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
    k_input_cov<T><<<grid_for(np * HW0 * HW0), 256, 0, st>>>(Xa, Xb, a0, b0, na, nb, symmetric,
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
        *launches += (g.act == NK_ACT_RELU) ? 2 : 1;
        k_conv<T><<<grid_for(np * HW * HW), 256, 0, st>>>(cur, nxt, np, H, W, g.filter, a_conv,
                                                          (T)sb2);
        T* t = cur; cur = nxt; nxt = t;
        if (g.act == NK_ACT_RELU)
          k_relu<T><<<grid_for(np * HW * HW), 256, 0, st>>>(cur, np, (int)HW, na, nb, symmetric,
                                                            pair0, a0, b0, qda, qdb, qsa, qsb,
                                                            g.nq, g.layer_qoff[layer], dstatus);
      }
    }
    const int64_t HW = (int64_t)H * W;
    k_gap<T><<<(unsigned)np, 256, 0, st>>>(cur, HW * HW, na, nb, symmetric, pair0, (T)sw2, (T)sb2,
                                           K, ldk);
    cudaError_t e = cudaGetLastError();
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
