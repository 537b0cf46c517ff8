// nk_self_diag: per-pixel self-variances q_l(p) = K_l(p, p; x, x) in FP64.
//
// The ReLU map of every activation layer needs q_l at both pixels of a pair
// (stax.Relu after each stax.Conv in the Appendix A Myrtle listing).  The
// diagonal of the self recursion is not closed under pooling: the pooled
// variance at P averages the pre-pool self covariance over the 2x2 block, i.e.
// at pixel offsets D in {-1,0,1}^2.  The conv stencil and the map keep the
// offset D = p' - p fixed, so the self covariance is carried on the offset
// planes |D|_inf <= r_s of each stage, with r = 0 at the last stage that has
// an activation and r_prev = 2 r + 1 across each pool.
//
// One CTA per image (grid-stride over images); planes of the current stage
// live in a per-CTA global workspace (at most 49 planes of H*W doubles), the
// image and the current q in shared memory.
//
// Activations: ReLU (arc-cosine map) or Erf, E[erf(u) erf(v)] =
// (2/pi) asin(2 K / sqrt((1 + 2 q)(1 + 2 q'))).  With a LayerNorm between
// conv and activation (the tuned Myrtle listing), the layer's band is divided
// by m = mean_p q(p) of this image before the activation, which then sees
// the self-variances q / m (the infinite-width limit of normalising over
// pixels and channels); m is written after the layer's q values.
#include "nk_common.cuh"
#include "nk_map.cuh"

namespace {

__global__ void __launch_bounds__(256)
k_self_diag(NkGeom g, double sw2, double sb2, const float* __restrict__ X, int64_t n,
            double* __restrict__ qd, float* __restrict__ qs, double* __restrict__ ws,
            size_t ws_half, unsigned int* dstatus) {
  extern __shared__ double sh[];
  const int H0 = g.Hs[0], W0 = g.Ws[0], C = g.C;
  double* xs = sh;                      // [H0*W0*C]
  double* qsh = sh + (size_t)H0 * W0 * C;  // [H0*W0]
  double* red = qsh + (size_t)H0 * W0;     // [33]: warp sums, then m
  double* bufA = ws + (size_t)blockIdx.x * 2 * ws_half;
  double* bufB = bufA + ws_half;
  const int tid = threadIdx.x, bd = blockDim.x;
  const double a_conv = sw2 / (double)(g.filter * g.filter);
  const int fr = g.filter / 2;

  for (int64_t img = blockIdx.x; img < n; img += gridDim.x) {
    const float* x = X + img * (int64_t)H0 * W0 * C;
    for (int i = tid; i < H0 * W0 * C; i += bd) xs[i] = (double)x[i];
    __syncthreads();
    double* A = bufA;
    double* B = bufB;
    int layer = 0;
    for (int s = 0; s <= g.last_act_stage; ++s) {
      const int H = g.Hs[s], W = g.Ws[s], r = g.radius[s], D = 2 * r + 1;
      const int HW = H * W, np = D * D;
      if (s == 0) {
        // K_0(p, p + D) = (1/C) sum_c x[p, c] x[p + D, c]
        for (int idx = tid; idx < np * HW; idx += bd) {
          const int pl = idx / HW, p = idx - pl * HW;
          const int dy = pl / D - r, dx = pl % D - r;
          const int i = p / W, j = p - (p / W) * W;
          const int i2 = i + dy, j2 = j + dx;
          double v = 0.0;
          if (i2 >= 0 && i2 < H && j2 >= 0 && j2 < W) {
            const double* u = xs + (size_t)(i * W + j) * C;
            const double* w = xs + (size_t)(i2 * W + j2) * C;
            for (int c = 0; c < C; ++c) v += u[c] * w[c];
            v /= (double)C;
          }
          A[idx] = v;
        }
      } else {
        // 2x2 average pool of both images: plane D' at P gathers the
        // previous stage's plane 2D' + b - a at pixel 2P + a.
        const int Wp = g.Ws[s - 1], HWp = g.Hs[s - 1] * Wp;
        const int rp = g.radius[s - 1], Dp = 2 * rp + 1;
        for (int idx = tid; idx < np * HW; idx += bd) {
          const int pl = idx / HW, p = idx - pl * HW;
          const int dy = pl / D - r, dx = pl % D - r;
          const int I = p / W, J = p - (p / W) * W;
          double v = 0.0;
          if (I + dy >= 0 && I + dy < H && J + dx >= 0 && J + dx < W) {
            for (int ay = 0; ay < 2; ++ay)
              for (int ax = 0; ax < 2; ++ax)
                for (int by = 0; by < 2; ++by)
                  for (int bx = 0; bx < 2; ++bx) {
                    const int Dy = 2 * dy + by - ay, Dx = 2 * dx + bx - ax;
                    const int plp = (Dy + rp) * Dp + (Dx + rp);
                    v += A[(size_t)plp * HWp + (2 * I + ay) * Wp + 2 * J + ax];
                  }
            v *= (1.0 / 16.0);
          }
          B[idx] = v;
        }
        double* t = A; A = B; B = t;
      }
      __syncthreads();
      for (int k = 0; k < g.convs[s]; ++k, ++layer) {
        // conv: K(p, p + D) = sw2/f^2 sum_delta Kt(p + delta, p + D + delta) + sb2.
        // A holds zeros wherever p + D leaves the image, so only p + delta
        // needs a range check.
        for (int idx = tid; idx < np * HW; idx += bd) {
          const int pl = idx / HW, p = idx - pl * HW;
          const int dy = pl / D - r, dx = pl % D - r;
          const int i = p / W, j = p - (p / W) * W;
          double v = 0.0;
          if (i + dy >= 0 && i + dy < H && j + dx >= 0 && j + dx < W) {
            double acc = 0.0;
            for (int ey = -fr; ey <= fr; ++ey)
              for (int ex = -fr; ex <= fr; ++ex) {
                const int u = i + ey, w = j + ex;
                if (u >= 0 && u < H && w >= 0 && w < W) acc += A[(size_t)pl * HW + u * W + w];
              }
            v = a_conv * acc + sb2;
          }
          B[idx] = v;
        }
        __syncthreads();
        const int center = r * D + r;
        const int off = g.layer_qoff[layer];
        // LayerNorm divisor m = mean_p q(p) (1 without a norm)
        double m = 1.0;
        if (g.norm == NK_NORM_LAYER) {
          double s = 0.0;
          for (int p = tid; p < HW; p += bd) s += B[(size_t)center * HW + p];
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          if ((tid & 31) == 0) red[tid >> 5] = s;
          __syncthreads();
          if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < (bd >> 5); ++w) t += red[w];
            t /= (double)HW;
            qd[img * (int64_t)g.nq + g.nq_base + layer] = t;
            if (qs) reinterpret_cast<float2*>(qs)[img * (int64_t)g.nq + g.nq_base + layer] = make_float2(0.f, 0.f);
            if (!(t > 0.0)) {
              atomicOr(dstatus, NK_DEV_NUMERICAL);
              t = 1.0;  // results are flagged; keep them finite
            }
            red[32] = t;
          }
          __syncthreads();
          m = red[32];
        }
        for (int p = tid; p < HW; p += bd) {
          const double q = B[(size_t)center * HW + p];
          qsh[p] = q / m;
          qd[img * (int64_t)g.nq + off + p] = q;
          if (!(q >= 0.0)) atomicOr(dstatus, NK_DEV_NUMERICAL);
          if (qs) {
            float2 o = make_float2(0.f, 0.f);
            if (g.act == NK_ACT_ERF) {
              o = make_float2((float)sqrt(2.0 / (m + 2.0 * q)), 1.f);
            } else if (q > 0.0) {
              o = make_float2((float)(1.0 / sqrt(q)), (float)sqrt(q / m));
            }
            reinterpret_cast<float2*>(qs)[img * (int64_t)g.nq + off + p] = o;
          }
        }
        __syncthreads();
        if (g.act == NK_ACT_RELU || g.act == NK_ACT_ERF) {
          const double inv_m = 1.0 / m;
          for (int idx = tid; idx < np * HW; idx += bd) {
            const int pl = idx / HW, p = idx - pl * HW;
            const int dy = pl / D - r, dx = pl % D - r;
            const int i = p / W, j = p - (p / W) * W;
            if (i + dy >= 0 && i + dy < H && j + dx >= 0 && j + dx < W) {
              const double Kn = B[idx] * inv_m, q1 = qsh[p], q2 = qsh[(i + dy) * W + j + dx];
              B[idx] = (g.act == NK_ACT_RELU) ? nk_relu_map_f64(Kn, q1, q2) : nk_erf_map_f64(Kn, q1, q2);
            }
          }
          __syncthreads();
        }
        double* t = A; A = B; B = t;
      }
    }
    __syncthreads();
  }
}

}  // namespace

size_t nk_self_diag_ws_per_cta(const NkGeom& g) {
  size_t m = 0;
  for (int s = 0; s <= g.last_act_stage; ++s) {
    const size_t D = 2 * g.radius[s] + 1;
    const size_t v = D * D * g.Hs[s] * g.Ws[s];
    if (v > m) m = v;
  }
  return 2 * m * sizeof(double);
}

cudaError_t nk_launch_self_diag(const NkGeom& g, double sw2, double sb2, const float* X,
                                int64_t n, double* qd, float* qs, double* ws, int grid,
                                unsigned int* dstatus, cudaStream_t st) {
  if (n <= 0 || g.last_act_stage < 0) return cudaSuccess;
  const size_t half = nk_self_diag_ws_per_cta(g) / sizeof(double) / 2;
  const size_t smem = ((size_t)g.Hs[0] * g.Ws[0] * (g.C + 1) + 33) * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_self_diag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_self_diag<<<grid, 256, smem, st>>>(g, sw2, sb2, X, n, qd, qs, ws, half, dstatus);
  return cudaGetLastError();
}
