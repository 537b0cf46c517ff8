// Plain layer-wise Myrtle kernels shared by the forward (myrtle_plain.cu) and
// the adjoint (myrtle_backward.cu): one thread per pixel-pair element.
#pragma once

#include "nk_common.cuh"
#include "nk_map.cuh"

namespace nkp {

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
  const int HW = H * W, HW2 = HW * HW;
  for (int64_t pr = blockIdx.y; pr < npairs; pr += gridDim.y) {
    int64_t i, j;
    pair_of(pair0 + pr, na, nb, symmetric, &i, &j);
    const float* xa = Xa + (a0 + i) * (int64_t)HW * C;
    const float* xb = Xb + (b0 + j) * (int64_t)HW * C;
    for (int rem = blockIdx.x * blockDim.x + threadIdx.x; rem < HW2; rem += gridDim.x * blockDim.x) {
      const int p = rem / HW, pp = rem - p * HW;
      const float* x = xa + p * C;
      const float* y = xb + pp * C;
      T acc = 0;
      for (int c = 0; c < C; ++c) acc += (T)x[c] * (T)y[c];
      out[pr * (int64_t)HW2 + rem] = acc / (T)C;
    }
  }
}

template <typename T>
__global__ void k_conv(const T* __restrict__ in, T* __restrict__ out, int64_t npairs, int H, int W,
                       int filt, T a, T b, const T* __restrict__ addend) {
  // one pair per blockIdx.y step, 32-bit index arithmetic inside a pair
  const int HW = H * W;
  const int HW2 = HW * HW;
  const int r = filt / 2;
  for (int64_t pr = blockIdx.y; pr < npairs; pr += gridDim.y) {
    const T* src = in + pr * (int64_t)HW2;
    T* dst = out + pr * (int64_t)HW2;
    for (int rem = blockIdx.x * blockDim.x + threadIdx.x; rem < HW2; rem += gridDim.x * blockDim.x) {
      const int p = rem / HW, pp = rem - p * HW;
      const int i = p / W, j = p - i * W, k = pp / W, l = pp - k * W;
      T acc = 0;
      for (int dy = -r; dy <= r; ++dy) {
        const int i2 = i + dy, k2 = k + dy;
        if (i2 < 0 || i2 >= H || k2 < 0 || k2 >= H) continue;
        for (int dx = -r; dx <= r; ++dx) {
          const int j2 = j + dx, l2 = l + dx;
          if (j2 >= 0 && j2 < W && l2 >= 0 && l2 < W) acc += src[(i2 * W + j2) * HW + k2 * W + l2];
        }
      }
      dst[rem] = a * acc + b + (addend ? addend[pr * (int64_t)HW2 + rem] : (T)0);
    }
  }
}

// Launch shape of the per-pair kernels: pairs along y, a pair's pixel pairs
// along x.
inline dim3 pair_grid(int64_t npairs, int64_t HW2) {
  int64_t x = (HW2 + 255) / 256;
  int64_t y = npairs;
  if (y > 65535) y = 65535;
  while (x * y > 152 * 64 && x > 1) x = (x + 1) / 2;
  return dim3((unsigned)std::max<int64_t>(1, x), (unsigned)std::max<int64_t>(1, y));
}

// The same 3x3 SAME conv, streamed: the diagonal stencil factors into a
// 3-tap sum along the (j, l) diagonal of a fixed (i, k) plane and a 3-tap sum
// over the planes (i - 1, k - 1), (i, k), (i + 1, k + 1), with the validity
// masks factoring the same way.  A block walks one (i, k) diagonal of one
// pair; the row-filtered planes of a sliding window of three live in shared
// memory, so each input element is read three times (L1) instead of nine and
// each output once.  smem: 3 W^2 elements of T.
template <typename T>
__global__ void __launch_bounds__(256) k_conv_diag(const T* __restrict__ in, T* __restrict__ out, int64_t npairs,
                                                   int H, int W, T a, T b, const T* __restrict__ addend) {
  extern __shared__ __align__(16) unsigned char conv_sm[];
  T* sh = reinterpret_cast<T*>(conv_sm);
  const int HW = H * W, W2 = W * W;
  const int d = (int)blockIdx.x - (H - 1);  // k - i on this diagonal
  const int i0 = d < 0 ? -d : 0;
  const int i1 = (d > 0 ? H - d : H) - 1;   // last i with k = i + d < H
  for (int64_t pr = blockIdx.y; pr < npairs; pr += gridDim.y) {
    const T* src = in + pr * (int64_t)HW * HW;
    T* dst = out + pr * (int64_t)HW * HW;
    // row-filtered plane (ii, ii + d) into slot ii % 3
    auto load = [&](int ii) {
      const int kk = ii + d;
      T* slot = sh + (ii % 3) * W2;
      for (int e = threadIdx.x; e < W2; e += blockDim.x) {
        const int j = e / W, l = e - j * W;
        T v = src[(int64_t)(ii * W + j) * HW + kk * W + l];
        if (j > 0 && l > 0) v += src[(int64_t)(ii * W + j - 1) * HW + kk * W + l - 1];
        if (j + 1 < W && l + 1 < W) v += src[(int64_t)(ii * W + j + 1) * HW + kk * W + l + 1];
        slot[e] = v;
      }
    };
    __syncthreads();  // the previous pair's planes are no longer read
    load(i0);
    for (int i = i0; i <= i1; ++i) {
      if (i + 1 <= i1) load(i + 1);
      __syncthreads();
      const T* cur = sh + (i % 3) * W2;
      const T* prv = sh + ((i + 2) % 3) * W2;
      const T* nxt = sh + ((i + 1) % 3) * W2;
      const int k = i + d;
      for (int e = threadIdx.x; e < W2; e += blockDim.x) {
        T acc = cur[e];
        if (i > i0) acc += prv[e];
        if (i < i1) acc += nxt[e];
        const int j = e / W, l = e - j * W;
        const int64_t o = (int64_t)(i * W + j) * HW + k * W + l;
        dst[o] = a * acc + b + (addend ? addend[pr * (int64_t)HW * HW + o] : (T)0);
      }
      __syncthreads();  // slot (i + 2) % 3 is refilled next
    }
  }
}

// One 3x3 (or other odd) SAME conv layer on a chunk of pair tensors:
// out = a S(in) + b (+ addend, a tensor of the same shape, when not null).
template <typename T>
inline void conv_layer(const T* in, T* out, int64_t np, int H, int W, int filt, T a, T b, cudaStream_t st,
                       const T* addend = nullptr) {
  const size_t smem = (size_t)3 * W * W * sizeof(T);
  if (filt == 3 && smem <= 200 * 1024) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_conv_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t y = np < 65535 ? np : 65535;
    k_conv_diag<T><<<dim3((unsigned)(2 * H - 1), (unsigned)y), 256, smem, st>>>(in, out, np, H, W, a, b, addend);
  } else {
    k_conv<T><<<pair_grid(np, (int64_t)H * W * H * W), 256, 0, st>>>(in, out, np, H, W, filt, a, b, addend);
  }
}


// Activation of the forward layer-wise form, in place: ReLU or Erf, with or
// without the LayerNorm before it.  FP64 reads the self-variances q and (with
// a norm) the divisors m of both images from qd and maps the normalised
// K / sqrt(m m') with q / m, q' / m'; FP32 uses the factor tables qs of
// nk_self_diag, which carry the norm: ReLU b b' J(K a a') / (2 pi), Erf
// (2/pi) asin(K a a').
template <typename T>
__global__ void k_act(T* K, int64_t npairs, int HW, int64_t na, int64_t nb, int symmetric, int64_t pair0,
                      int64_t a0, int64_t b0, const double* __restrict__ qda, const double* __restrict__ qdb,
                      const float* __restrict__ qsa, const float* __restrict__ qsb, int64_t nq, int qoff,
                      int act, int moff, unsigned int* dstatus) {
  const int HW2 = HW * HW;
  for (int64_t pr = blockIdx.y; pr < npairs; pr += gridDim.y) {
    int64_t i, j;
    pair_of(pair0 + pr, na, nb, symmetric, &i, &j);
    const int64_t ra = (a0 + i) * nq, rb = (b0 + j) * nq;
    for (int rem = blockIdx.x * blockDim.x + threadIdx.x; rem < HW2; rem += gridDim.x * blockDim.x) {
      const int64_t e = pr * (int64_t)HW2 + rem;
      const int p = rem / HW, pp = rem - p * HW;
      if constexpr (sizeof(T) == 8) {
        double q1 = qda[ra + qoff + p], q2 = qdb[rb + qoff + pp];
        if (!(q1 >= 0.0) || !(q2 >= 0.0)) atomicOr(dstatus, NK_DEV_NUMERICAL);
        double k = K[e];
        if (moff >= 0) {
          const double m1 = qda[ra + moff], m2 = qdb[rb + moff];
          k /= sqrt(m1 * m2);
          q1 /= m1;
          q2 /= m2;
        }
        K[e] = (act == NK_ACT_ERF) ? nk_erf_map_f64(k, q1, q2) : nk_relu_map_f64(k, q1, q2);
      } else {
        const float2 s1 = reinterpret_cast<const float2*>(qsa)[ra + qoff + p];
        const float2 s2 = reinterpret_cast<const float2*>(qsb)[rb + qoff + pp];
        const float s = s1.y * s2.y;
        float c = K[e] * (s1.x * s2.x);
        c = fminf(fmaxf(c, -1.f), 1.f);
        float v = 0.f;
        if (act == NK_ACT_ERF) {
          v = s * 0.63661977236758134308f * asinf(c);
        } else if (s > 0.f) {
          v = s * (0.15915494309189533577f) * (sqrtf(fmaxf(1.f - c * c, 0.f)) + c * (NK_PI_F - acosf(c)));
        }
        K[e] = v;
      }
    }
  }
}

// ReLU map with self-variances of the pair's two images at this layer,
// K = map(Kin) (Kin may be K itself).
template <typename T>
__global__ void k_relu(const T* Kin, T* K, int64_t npairs, int HW, int64_t na, int64_t nb,
                       int symmetric, int64_t pair0, int64_t a0, int64_t b0,
                       const double* __restrict__ qda, const double* __restrict__ qdb,
                       const float* __restrict__ qsa, const float* __restrict__ qsb, int64_t nq,
                       int qoff, unsigned int* dstatus) {
  // one pair per blockIdx.y step: its images are found once, not per entry
  const int HW2 = HW * HW;
  for (int64_t pr = blockIdx.y; pr < npairs; pr += gridDim.y) {
   int64_t i, j;
   pair_of(pair0 + pr, na, nb, symmetric, &i, &j);
   for (int rem = blockIdx.x * blockDim.x + threadIdx.x; rem < HW2; rem += gridDim.x * blockDim.x) {
    const int64_t e = pr * (int64_t)HW2 + rem;
    const int p = rem / HW, pp = rem - p * HW;
    if constexpr (sizeof(T) == 8) {
      const double q1 = qda[(a0 + i) * nq + qoff + p];
      const double q2 = qdb[(b0 + j) * nq + qoff + pp];
      if (!(q1 >= 0.0) || !(q2 >= 0.0)) atomicOr(dstatus, NK_DEV_NUMERICAL);
      K[e] = nk_relu_map_f64(Kin[e], q1, q2);
    } else {
      const float2 s1 = reinterpret_cast<const float2*>(qsa)[(a0 + i) * nq + qoff + p];
      const float2 s2 = reinterpret_cast<const float2*>(qsb)[(b0 + j) * nq + qoff + pp];
      const float s = s1.y * s2.y;
      float v = 0.f;
      if (s > 0.f) {
        float c = Kin[e] * (s1.x * s2.x);
        c = fminf(fmaxf(c, -1.f), 1.f);
        v = s * (0.15915494309189533577f) *
            (sqrtf(fmaxf(1.f - c * c, 0.f)) + c * (NK_PI_F - acosf(c)));
      }
      K[e] = v;
    }
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

// Flatten + Dense readout (the CV8 listing): K = sw2 mean_p Kt(p, p) + sb2,
// the pixel pairs p' = p of each pair's last tensor (HW x HW), summed in FP64.
template <typename T>
__global__ void k_flatten(const T* __restrict__ in, int HW, int64_t na, int64_t nb, int symmetric,
                          int64_t pair0, T sw2, T sb2, T* __restrict__ K, int64_t ldk) {
  __shared__ double red[32];
  const int64_t pr = blockIdx.x;
  const int64_t HW2 = (int64_t)HW * HW;
  double acc = 0.0;
  for (int p = threadIdx.x; p < HW; p += blockDim.x) acc += (double)in[pr * HW2 + (int64_t)p * HW + p];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) {
      int64_t i, j;
      pair_of(pair0 + pr, na, nb, symmetric, &i, &j);
      const T v = (T)((double)sw2 * (acc / (double)HW) + (double)sb2);
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

// NTK ReLU step (NTK parameterisation): Kt = map(K) in place and
// Theta_t = Theta * E[relu' relu'] = Theta (pi - arccos c) / (2 pi).
template <typename T>
__global__ void k_relu_ntk(T* K, T* Th, int64_t npairs, int HW, int64_t na, int64_t nb, int symmetric,
                           int64_t pair0, int64_t a0, int64_t b0, const double* __restrict__ qda,
                           const double* __restrict__ qdb, const float* __restrict__ qsa,
                           const float* __restrict__ qsb, int64_t nq, int qoff, unsigned int* dstatus) {
  const int HW2 = HW * HW;
  for (int64_t pr = blockIdx.y; pr < npairs; pr += gridDim.y) {
    int64_t i, j;
    pair_of(pair0 + pr, na, nb, symmetric, &i, &j);
    for (int rem = blockIdx.x * blockDim.x + threadIdx.x; rem < HW2; rem += gridDim.x * blockDim.x) {
      const int64_t e = pr * (int64_t)HW2 + rem;
      const int p = rem / HW, pp = rem - p * HW;
      if constexpr (sizeof(T) == 8) {
        const double q1 = qda[(a0 + i) * nq + qoff + p];
        const double q2 = qdb[(b0 + j) * nq + qoff + pp];
        if (!(q1 >= 0.0) || !(q2 >= 0.0)) atomicOr(dstatus, NK_DEV_NUMERICAL);
        const double s = sqrt(q1 * q2);
        double kd = 0.0, kt = 0.0;
        if (s > 0.0) {
          double c = K[e] / s;
          c = c < -1.0 ? -1.0 : (c > 1.0 ? 1.0 : c);
          const double th = acos(c);
          kt = s * NK_INV_2PI_D * (sqrt(fmax(1.0 - c * c, 0.0)) + c * (NK_PI_D - th));
          kd = (NK_PI_D - th) * NK_INV_2PI_D;
        }
        K[e] = kt;
        Th[e] *= kd;
      } else {
        const float2 s1 = reinterpret_cast<const float2*>(qsa)[(a0 + i) * nq + qoff + p];
        const float2 s2 = reinterpret_cast<const float2*>(qsb)[(b0 + j) * nq + qoff + pp];
        const float s = s1.y * s2.y;
        float kt = 0.f, kd = 0.f;
        if (s > 0.f) {
          float c = K[e] * (s1.x * s2.x);
          c = fminf(fmaxf(c, -1.f), 1.f);
          const float th = acosf(c);
          kt = s * 0.15915494309189533577f * (sqrtf(fmaxf(1.f - c * c, 0.f)) + c * (NK_PI_F - th));
          kd = (NK_PI_F - th) * 0.15915494309189533577f;
        }
        K[e] = kt;
        Th[e] *= kd;
      }
    }
  }
}

// NTK readout: K = sw2 mean(Kt) + sb2, Theta = K + sw2 mean(Theta_t).
template <typename T>
__global__ void k_gap_ntk(const T* __restrict__ Kt, const T* __restrict__ Tt, int64_t HW2, int64_t na, int64_t nb,
                          int symmetric, int64_t pair0, double sw2, double sb2, T* __restrict__ K,
                          T* __restrict__ Th, int64_t ldk) {
  __shared__ double r1[32], r2[32];
  const int64_t pr = blockIdx.x;
  double a = 0.0, b = 0.0;
  for (int64_t e = threadIdx.x; e < HW2; e += blockDim.x) {
    a += (double)Kt[pr * HW2 + e];
    b += (double)Tt[pr * HW2 + e];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r1[threadIdx.x >> 5] = a;
    r2[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    a = (threadIdx.x < (blockDim.x >> 5)) ? r1[threadIdx.x] : 0.0;
    b = (threadIdx.x < (blockDim.x >> 5)) ? r2[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x == 0) {
      int64_t i, j;
      pair_of(pair0 + pr, na, nb, symmetric, &i, &j);
      const double kv = sw2 * (a / (double)HW2) + sb2;
      const double tv = kv + sw2 * (b / (double)HW2);
      K[i * ldk + j] = (T)kv;
      Th[i * ldk + j] = (T)tv;
      if (symmetric && i != j) {
        K[j * ldk + i] = (T)kv;
        Th[j * ldk + i] = (T)tv;
      }
    }
  }
}

}  // namespace nkp
