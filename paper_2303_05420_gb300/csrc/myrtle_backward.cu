// nk_block_backward: adjoint of the Myrtle NNGP kernel block (plain layer-wise
// form, FP32 or FP64).
//
// For a block K[i][j] = NNGP(Xa[i], Xb[j]) and an upstream gradient dK, it
// accumulates dL/dXa, dL/dXb, dL/dsigma_w^2 and dL/dsigma_b^2 (+=), the
// adjoint of the whole recursion of the Appendix A Myrtle listing:
//   readout  K = sw2 mean(Kt_L) + sb2          -> uniform seed sw2/(H W)^2
//   ReLU map Kt = sqrt(q q')/(2 pi) J(c)        -> dK = dKt J'(c)/(2 pi),
//            dq  = dKt (Kt - K J'(c)/(2 pi)) / (2 q), likewise dq'
//   conv     K = sw2/9 S(Kt_prev) + sb2        -> dKt_prev = sw2/9 S(dK)
//            (S, the diagonal 3x3 stencil with zero padding, is self-adjoint),
//            dsw2 += dK (K - sb2)/sw2, dsb2 += dK
//   pool     Kp(P,P') = 1/16 sum Kt(2P+a,2P'+b) -> dKt = dKp / 16
//   input    K_0 = (1/C) x . x'                 -> dx[p] += (1/C) sum_p' dK_0 x'[p']
// The self-variances q_l(p) = K_l(p,p;x,x) depend on x, sw2 and sb2 through
// the banded self recursion; their gradients dq are reduced per pixel here
// and pushed through the adjoint of that recursion (FP64) at the end.
// Forward pixel-pair tensors of each layer are recomputed per chunk of pairs
// and kept in HBM for the reverse sweep.
#include <algorithm>

#include "myrtle_plain.cuh"

namespace {

using namespace nkp;

// ---------------------------------------------------------------------------
// Per-pair seed: g = dK[i][j] (+ dK[j][i] when the block is symmetric and
// i != j: both entries are the same function); dsw2 += g mean(Kt_L),
// dsb2 += g; the uniform gradient of the last layer's Kt is g sw2 / HW^2.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_pair_seed(const T* __restrict__ dK, int64_t lddk, const T* __restrict__ gapmean,
                            int64_t na, int64_t nb, int sym, int64_t pair0, int64_t np, double sw2,
                            double hw2, T* __restrict__ useed, double* __restrict__ dsw2,
                            double* __restrict__ dsb2) {
  for (int64_t pr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pr < np;
       pr += (int64_t)gridDim.x * blockDim.x) {
    int64_t i, j;
    pair_of(pair0 + pr, na, nb, sym, &i, &j);
    double g = (double)dK[i * lddk + j];
    if (sym && i != j) g += (double)dK[j * lddk + i];
    useed[pr] = (T)(g * sw2 / hw2);
    atomicAdd(dsw2, g * (double)gapmean[pr]);
    atomicAdd(dsb2, g);
  }
}

// mean of each pair's tensor (the forward value before the readout)
template <typename T>
__global__ void k_pair_mean(const T* __restrict__ in, int64_t HW2, T* __restrict__ out) {
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
    if (threadIdx.x == 0) out[pr] = (T)(acc / (double)HW2);
  }
}

template <typename T>
__global__ void k_fill_pairs(T* __restrict__ buf, int64_t np, int64_t HW2, const T* __restrict__ val) {
  const int64_t total = np * HW2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    buf[e] = val[e / HW2];
}

// ReLU-map adjoint, in place on d (dKt in, dK out); h = dKt (Kt - K J'/(2 pi)).
// The FP32 form reads the FP32 (1/sqrt q, sqrt q) tables, as the forward map
// does: no FP64 load, conversion or division per entry (FP64 runs at a small
// fraction of the FP32 rate here and bounded this kernel when it did).
template <typename T>
__global__ void k_map_adj(const T* __restrict__ Kpre, T* __restrict__ d, T* __restrict__ hbuf,
                          int64_t np, int HW, int64_t na, int64_t nb, int sym, int64_t pair0,
                          int64_t a0, int64_t b0, const double* __restrict__ qda,
                          const double* __restrict__ qdb, const float* __restrict__ qsa,
                          const float* __restrict__ qsb, int64_t nq, int qoff, double sb2, double inv_sw2,
                          double* __restrict__ dsw2, double* __restrict__ dsb2) {
  // the conv's sigma terms ride along: dsw2 += dK (K - sb2) / sw2, dsb2 += dK
  // (sums in T over runs of at most 64 entries, added in FP64)
  __shared__ double r1[32], r2[32];
  double sa = 0.0, sbb = 0.0;
  T ta = 0, tb = 0;
  int run = 0;
  const T tsb2 = (T)sb2;
  // one pair per blockIdx.y step: its images are found once, not per entry
  const int HW2 = HW * HW;
  for (int64_t pr = blockIdx.y; pr < np; pr += gridDim.y) {
   int64_t i, j;
   pair_of(pair0 + pr, na, nb, sym, &i, &j);
   for (int rem = blockIdx.x * blockDim.x + threadIdx.x; rem < HW2; rem += gridDim.x * blockDim.x) {
    const int64_t e = pr * (int64_t)HW2 + rem;
    const int p = rem / HW, pp = rem - p * HW;
    T s, rs;  // sqrt(q q'), 1 / sqrt(q q')
    if constexpr (sizeof(T) == 8) {
      s = sqrt(qda[(a0 + i) * nq + qoff + p] * qdb[(b0 + j) * nq + qoff + pp]);
      rs = s > 0.0 ? 1.0 / s : 0.0;
    } else {
      const float2 s1 = reinterpret_cast<const float2*>(qsa)[(a0 + i) * nq + qoff + p];
      const float2 s2 = reinterpret_cast<const float2*>(qsb)[(b0 + j) * nq + qoff + pp];
      s = s1.y * s2.y;
      rs = s1.x * s2.x;
    }
    T dk = 0, h = 0;
    if (s > (T)0) {
      const T K = Kpre[e];
      T c = K * rs;
      c = c < (T)-1 ? (T)-1 : (c > (T)1 ? (T)1 : c);
      const T th = acos(c);
      const T J = sqrt(((T)1 - c * c) > (T)0 ? (T)1 - c * c : (T)0) + c * ((T)NK_PI_D - th);
      const T dJ = (T)NK_PI_D - th;
      const T inv2pi = (T)NK_INV_2PI_D;
      const T Kt = s * inv2pi * J;
      const T g = d[e];
      dk = g * dJ * inv2pi;
      h = g * (Kt - K * dJ * inv2pi);
    }
    d[e] = dk;
    hbuf[e] = h;
    ta += dk * (Kpre[e] - tsb2);
    tb += dk;
    if (++run == 64) {
      sa += (double)ta;
      sbb += (double)tb;
      ta = tb = 0;
      run = 0;
    }
   }
  }
  sa += (double)ta;
  sbb += (double)tb;
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sbb += __shfl_xor_sync(0xffffffffu, sbb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r1[threadIdx.x >> 5] = sa;
    r2[threadIdx.x >> 5] = sbb;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    sa = (threadIdx.x < (blockDim.x >> 5)) ? r1[threadIdx.x] : 0.0;
    sbb = (threadIdx.x < (blockDim.x >> 5)) ? r2[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
      sbb += __shfl_xor_sync(0xffffffffu, sbb, o);
    }
    if (threadIdx.x == 0) {
      atomicAdd(dsw2, sa * inv_sw2);
      atomicAdd(dsb2, sbb);
    }
  }
}

// dq_a[i][p] += sum_p' h(p,p') / (2 q_a(p)): one warp per (pair, p)
template <typename T>
__global__ void k_rowsum_q(const T* __restrict__ hbuf, int64_t np, int HW, int64_t na, int64_t nb,
                           int sym, int64_t pair0, int64_t a0, const double* __restrict__ qda,
                           int64_t nq, int qoff, T* __restrict__ dqa) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t w = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); w < np * HW; w += nw) {
    const int64_t pr = w / HW;
    const int p = (int)(w - pr * HW);
    const T* row = hbuf + (pr * HW + p) * (int64_t)HW;
    T acc = 0;
    for (int k = lane; k < HW; k += 32) acc += row[k];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      int64_t i, j;
      pair_of(pair0 + pr, na, nb, sym, &i, &j);
      const double q = qda[(a0 + i) * nq + qoff + p];
      if (q > 0.0) atomicAdd(dqa + i * nq + qoff + p, (T)((double)acc / (2.0 * q)));
    }
  }
}

// dq_b[j][p'] += sum_p h(p,p') / (2 q_b(p')): one thread per (pair, p')
template <typename T>
__global__ void k_colsum_q(const T* __restrict__ hbuf, int64_t np, int HW, int64_t na, int64_t nb,
                           int sym, int64_t pair0, int64_t b0, const double* __restrict__ qdb,
                           int64_t nq, int qoff, T* __restrict__ dqb) {
  const int64_t total = np * HW;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pr = e / HW;
    const int pp = (int)(e - pr * HW);
    const T* col = hbuf + pr * (int64_t)HW * HW + pp;
    T acc = 0;
    for (int p = 0; p < HW; ++p) acc += col[(int64_t)p * HW];
    int64_t i, j;
    pair_of(pair0 + pr, na, nb, sym, &i, &j);
    const double q = qdb[(b0 + j) * nq + qoff + pp];
    if (q > 0.0) atomicAdd(dqb + j * nq + qoff + pp, (T)((double)acc / (2.0 * q)));
  }
}

// dsw2 += sum d (Kpre - sb2) / sw2 ; dsb2 += sum d
template <typename T>
__global__ void k_sigma_terms(const T* __restrict__ d, const T* __restrict__ Kpre, int64_t total,
                              double sb2, double inv_sw2, double* __restrict__ dsw2,
                              double* __restrict__ dsb2) {
  __shared__ double r1[32], r2[32];
  // sums in T over runs of at most 64 elements, added in FP64 (FP64
  // arithmetic runs at 1/64 of the FP32 rate on this part)
  double a = 0.0, b = 0.0;
  T ta = 0, tb = 0;
  const T tsb2 = (T)sb2;
  int run = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const T g = d[e];
    ta += g * (Kpre[e] - tsb2);
    tb += g;
    if (++run == 64) {
      a += (double)ta;
      b += (double)tb;
      ta = tb = 0;
      run = 0;
    }
  }
  a += (double)ta;
  b += (double)tb;
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
      atomicAdd(dsw2, a * inv_sw2);
      atomicAdd(dsb2, b);
    }
  }
}

// pool adjoint: d_prev(p, p') = d(P, P') / 16 at stage resolution H x W (prev 2H x 2W)
template <typename T>
__global__ void k_pool_adj(const T* __restrict__ d, T* __restrict__ dprev, int64_t np, int H, int W) {
  const int H2 = 2 * H, W2 = 2 * W;
  const int64_t HWp = (int64_t)H2 * W2, HW = (int64_t)H * W;
  const int64_t total = np * HWp * HWp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pr = e / (HWp * HWp), rem = e - pr * HWp * HWp;
    const int p = (int)(rem / HWp), pp = (int)(rem - (int64_t)p * HWp);
    const int P = (p / W2 / 2) * W + (p % W2) / 2;
    const int PP = (pp / W2 / 2) * W + (pp % W2) / 2;
    dprev[e] = d[pr * HW * HW + (int64_t)P * HW + PP] * (T)(1.0 / 16.0);
  }
}

// input adjoint, image a: dXa[i][p][c] += (1/C) sum_p' dK0(p,p') xb[p'][c]
template <typename T>
__global__ void k_seed_adj_a(const T* __restrict__ d0, const float* __restrict__ Xb, int64_t np, int HW,
                             int C, int64_t na, int64_t nb, int sym, int64_t pair0, int64_t a0,
                             int64_t b0, T* __restrict__ dXa) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t w = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); w < np * HW; w += nw) {
    const int64_t pr = w / HW;
    const int p = (int)(w - pr * HW);
    int64_t i, j;
    pair_of(pair0 + pr, na, nb, sym, &i, &j);
    const T* row = d0 + (pr * HW + p) * (int64_t)HW;
    const float* xb = Xb + (b0 + j) * (int64_t)HW * C;
    T acc[4] = {0, 0, 0, 0};
    for (int k = lane; k < HW; k += 32) {
      const T g = row[k];
      for (int c = 0; c < C && c < 4; ++c) acc[c] += g * (T)xb[k * C + c];
    }
    for (int c = 0; c < C && c < 4; ++c) {
      T v = acc[c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) atomicAdd(dXa + ((a0 + i) * (int64_t)HW + p) * C + c, v / (T)C);
    }
  }
}

// input adjoint, image b: dXb[j][p'][c] += (1/C) sum_p dK0(p,p') xa[p][c]
template <typename T>
__global__ void k_seed_adj_b(const T* __restrict__ d0, const float* __restrict__ Xa, int64_t np, int HW,
                             int C, int64_t na, int64_t nb, int sym, int64_t pair0, int64_t a0,
                             int64_t b0, T* __restrict__ dXb) {
  const int64_t total = np * HW;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pr = e / HW;
    const int pp = (int)(e - pr * HW);
    int64_t i, j;
    pair_of(pair0 + pr, na, nb, sym, &i, &j);
    const T* col = d0 + pr * (int64_t)HW * HW + pp;
    const float* xa = Xa + (a0 + i) * (int64_t)HW * C;
    T acc[4] = {0, 0, 0, 0};
    for (int p = 0; p < HW; ++p) {
      const T g = col[(int64_t)p * HW];
      for (int c = 0; c < C && c < 4; ++c) acc[c] += g * (T)xa[p * C + c];
    }
    for (int c = 0; c < C && c < 4; ++c) atomicAdd(dXb + ((b0 + j) * (int64_t)HW + pp) * C + c, acc[c] / (T)C);
  }
}

// ---------------------------------------------------------------------------
// Adjoint of the banded self recursion that produces q_l(p) (FP64).
// One CTA per image.  Forward: the offset planes of every layer (as in
// nk_self_diag), storing each layer's pre-activation planes.  Reverse: the
// external dq_l(p) (from the cross-pair adjoint) enters the D = 0 plane of
// layer l, to which the q-dependence of every self map also feeds back;
// then the conv, pool and input adjoints.
// ---------------------------------------------------------------------------
struct SelfAdjGeom {
  NkGeom g;
  int64_t store_off[NK_MAX_LAYERS];  // doubles, per layer
  int64_t store_total;
  int64_t work;                      // doubles per work buffer
};

__device__ __forceinline__ double J64(double c, double* dJ) {
  c = fmin(fmax(c, -1.0), 1.0);
  const double th = acos(c);
  *dJ = NK_PI_D - th;
  return sqrt(fmax(1.0 - c * c, 0.0)) + c * (NK_PI_D - th);
}

template <typename T>
__global__ void __launch_bounds__(256)
k_self_adj(SelfAdjGeom G, double sw2, double sb2, const float* __restrict__ X, int64_t n, int64_t img0,
           const T* __restrict__ dq, T* __restrict__ dX, double* __restrict__ dsw2,
           double* __restrict__ dsb2, double* __restrict__ ws) {
  extern __shared__ double sh[];
  const NkGeom& g = G.g;
  const int H0 = g.Hs[0], W0 = g.Ws[0], C = g.C;
  double* xs = sh;                                   // [H0*W0*C]
  double* dx = xs + (size_t)H0 * W0 * C;             // [H0*W0*C]
  double* qacc = dx + (size_t)H0 * W0 * C;           // [H0*W0]
  __shared__ double red[2][8];
  double* store = ws + (size_t)blockIdx.x * (G.store_total + 3 * G.work);
  double* bufA = store + G.store_total;
  double* bufB = bufA + G.work;
  double* bufC = bufB + G.work;
  const int tid = threadIdx.x, bd = blockDim.x;
  const double a_conv = sw2 / (double)(g.filter * g.filter);
  const int fr = g.filter / 2;
  const bool relu = (g.act == NK_ACT_RELU);

  for (int64_t img = blockIdx.x; img < n; img += gridDim.x) {
    const float* x = X + (img0 + img) * (int64_t)H0 * W0 * C;
    for (int i = tid; i < H0 * W0 * C; i += bd) {
      xs[i] = (double)x[i];
      dx[i] = 0.0;
    }
    __syncthreads();
    // ---------------- forward, storing pre-activation planes per layer
    double* A = bufA;
    double* B = bufB;
    int layer = 0;
    for (int s = 0; s <= g.last_act_stage; ++s) {
      const int H = g.Hs[s], W = g.Ws[s], r = g.radius[s], D = 2 * r + 1, HW = H * W, np = D * D;
      if (s == 0) {
        for (int idx = tid; idx < np * HW; idx += bd) {
          const int pl = idx / HW, p = idx - pl * HW;
          const int dy = pl / D - r, dx_ = pl % D - r, i = p / W, j = p % W;
          double v = 0.0;
          if (i + dy >= 0 && i + dy < H && j + dx_ >= 0 && j + dx_ < W) {
            for (int c = 0; c < C; ++c) v += xs[p * C + c] * xs[((i + dy) * W + j + dx_) * C + c];
            v /= (double)C;
          }
          A[idx] = v;
        }
      } else {
        const int Wp = g.Ws[s - 1], HWp = g.Hs[s - 1] * Wp, rp = g.radius[s - 1], Dp = 2 * rp + 1;
        for (int idx = tid; idx < np * HW; idx += bd) {
          const int pl = idx / HW, p = idx - pl * HW;
          const int dy = pl / D - r, dx_ = pl % D - r, I = p / W, J = p % W;
          double v = 0.0;
          if (I + dy >= 0 && I + dy < H && J + dx_ >= 0 && J + dx_ < W) {
            for (int ay = 0; ay < 2; ++ay)
              for (int ax = 0; ax < 2; ++ax)
                for (int by = 0; by < 2; ++by)
                  for (int bx = 0; bx < 2; ++bx) {
                    const int plp = (2 * dy + by - ay + rp) * Dp + (2 * dx_ + bx - ax + rp);
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
        double* Kst = store + G.store_off[layer];
        for (int idx = tid; idx < np * HW; idx += bd) {
          const int pl = idx / HW, p = idx - pl * HW;
          const int dy = pl / D - r, dx_ = pl % D - r, i = p / W, j = p % W;
          double v = 0.0;
          if (i + dy >= 0 && i + dy < H && j + dx_ >= 0 && j + dx_ < W) {
            double acc = 0.0;
            for (int ey = -fr; ey <= fr; ++ey)
              for (int ex = -fr; ex <= fr; ++ex) {
                const int u = i + ey, w = j + ex;
                if (u >= 0 && u < H && w >= 0 && w < W) acc += A[(size_t)pl * HW + u * W + w];
              }
            v = a_conv * acc + sb2;
          }
          Kst[idx] = v;
        }
        __syncthreads();
        const int center = r * D + r;
        for (int idx = tid; idx < np * HW; idx += bd) {
          const int pl = idx / HW, p = idx - pl * HW;
          const int dy = pl / D - r, dx_ = pl % D - r, i = p / W, j = p % W;
          double v = 0.0;
          if (i + dy >= 0 && i + dy < H && j + dx_ >= 0 && j + dx_ < W) {
            v = Kst[idx];
            if (relu)
              v = nk_relu_map_f64(v, Kst[(size_t)center * HW + p],
                                  Kst[(size_t)center * HW + (i + dy) * W + j + dx_]);
          }
          A[idx] = v;
        }
        __syncthreads();
      }
    }
    // ---------------- reverse
    // Dg: gradient w.r.t. the current post-activation planes (zero after the
    // last layer: the self recursion is read only through its q's)
    double* Dg = bufB;
    double* E = bufC;
    {
      const int s = g.last_act_stage;
      const int np = (2 * g.radius[s] + 1) * (2 * g.radius[s] + 1);
      for (int idx = tid; idx < np * g.Hs[s] * g.Ws[s]; idx += bd) Dg[idx] = 0.0;
    }
    double lsw = 0.0, lsb = 0.0;
    layer = g.n_layers;
    for (int s = g.last_act_stage; s >= 0; --s) {
      const int H = g.Hs[s], W = g.Ws[s], r = g.radius[s], D = 2 * r + 1, HW = H * W, np = D * D;
      const int center = r * D + r;
      for (int k = g.convs[s] - 1; k >= 0; --k) {
        --layer;
        const double* Kst = store + G.store_off[layer];
        for (int p = tid; p < HW; p += bd) qacc[p] = 0.0;
        __syncthreads();
        // map adjoint
        for (int idx = tid; idx < np * HW; idx += bd) {
          const int pl = idx / HW, p = idx - pl * HW;
          const int dy = pl / D - r, dx_ = pl % D - r, i = p / W, j = p % W;
          double e = 0.0;
          if (i + dy >= 0 && i + dy < H && j + dx_ >= 0 && j + dx_ < W) {
            const double gK = Dg[idx];
            if (!relu) {
              e = gK;
            } else {
              const int p2 = (i + dy) * W + j + dx_;
              const double q1 = Kst[(size_t)center * HW + p], q2 = Kst[(size_t)center * HW + p2];
              const double sq = sqrt(q1 * q2);
              if (sq > 0.0) {
                const double K = Kst[idx];
                double dJ;
                const double J = J64(K / sq, &dJ);
                const double Kt = sq * NK_INV_2PI_D * J;
                e = gK * dJ * NK_INV_2PI_D;
                const double h = gK * (Kt - K * dJ * NK_INV_2PI_D);
                if (h != 0.0) {
                  atomicAdd(qacc + p, h / (2.0 * q1));
                  atomicAdd(qacc + p2, h / (2.0 * q2));
                }
              }
            }
          }
          E[idx] = e;
        }
        __syncthreads();
        // q(p) = K(p,p): the D = 0 plane takes the maps' q terms and the
        // external dq of this layer
        const int off = g.layer_qoff[layer];
        for (int p = tid; p < HW; p += bd)
          E[(size_t)center * HW + p] += qacc[p] + (double)dq[img * (int64_t)g.nq + off + p];
        __syncthreads();
        // sigma terms and conv adjoint (self-adjoint stencil) -> Dg
        for (int idx = tid; idx < np * HW; idx += bd) {
          const int pl = idx / HW, p = idx - pl * HW;
          const int dy = pl / D - r, dx_ = pl % D - r, i = p / W, j = p % W;
          double v = 0.0;
          if (i + dy >= 0 && i + dy < H && j + dx_ >= 0 && j + dx_ < W) {
            const double e = E[idx];
            lsw += e * (Kst[idx] - sb2);
            lsb += e;
            double acc = 0.0;
            for (int ey = -fr; ey <= fr; ++ey)
              for (int ex = -fr; ex <= fr; ++ex) {
                const int u = i - ey, w = j - ex;
                if (u >= 0 && u < H && w >= 0 && w < W) acc += E[(size_t)pl * HW + u * W + w];
              }
            v = a_conv * acc;
          }
          Dg[idx] = v;
        }
        __syncthreads();
      }
      if (s > 0) {
        // pool adjoint: previous-stage plane Dp at u = 2P + a takes
        // Dg(P, D') / 16 with D' = (Dp + a - b)/2 for the b in {0,1} that
        // makes it integral, if |D'| <= r and P + D' in range
        const int Hp = g.Hs[s - 1], Wp = g.Ws[s - 1], HWp = Hp * Wp, rp = g.radius[s - 1];
        const int Dp = 2 * rp + 1, npp = Dp * Dp;
        for (int idx = tid; idx < npp * HWp; idx += bd) {
          const int pl = idx / HWp, u = idx - pl * HWp;
          const int dyp = pl / Dp - rp, dxp = pl % Dp - rp, ui = u / Wp, uj = u % Wp;
          double v = 0.0;
          if (ui + dyp >= 0 && ui + dyp < Hp && uj + dxp >= 0 && uj + dxp < Wp) {
            const int ay = ui & 1, ax = uj & 1, I = ui >> 1, Jj = uj >> 1;
            const int by = (dyp + ay) & 1, bx = (dxp + ax) & 1;
            const int dy = (dyp + ay - by) / 2, dx_ = (dxp + ax - bx) / 2;
            if (dy >= -r && dy <= r && dx_ >= -r && dx_ <= r && I + dy >= 0 && I + dy < H && Jj + dx_ >= 0 &&
                Jj + dx_ < W)
              v = Dg[(size_t)((dy + r) * D + dx_ + r) * HW + I * W + Jj] * (1.0 / 16.0);
          }
          E[idx] = v;
        }
        __syncthreads();
        double* t = Dg; Dg = E; E = t;
      }
    }
    // input adjoint: K_0(p, p+D) = (1/C) sum_c x[p,c] x[p+D,c]
    {
      const int H = H0, W = W0, r = g.radius[0], D = 2 * r + 1, HW = H * W, np = D * D;
      for (int idx = tid; idx < np * HW; idx += bd) {
        const int pl = idx / HW, p = idx - pl * HW;
        const int dy = pl / D - r, dx_ = pl % D - r, i = p / W, j = p % W;
        if (i + dy >= 0 && i + dy < H && j + dx_ >= 0 && j + dx_ < W) {
          const double gk = Dg[idx] / (double)C;
          if (gk != 0.0) {
            const int p2 = (i + dy) * W + j + dx_;
            for (int c = 0; c < C; ++c) {
              atomicAdd(dx + p * C + c, gk * xs[p2 * C + c]);
              atomicAdd(dx + p2 * C + c, gk * xs[p * C + c]);
            }
          }
        }
      }
    }
    __syncthreads();
    if (dX) {
      T* dxo = dX + (img0 + img) * (int64_t)H0 * W0 * C;
      for (int i = tid; i < H0 * W0 * C; i += bd) dxo[i] = (T)((double)dxo[i] + dx[i]);
    }
    // sigma terms: the block's threads -> one atomic each
    for (int o = 16; o > 0; o >>= 1) {
      lsw += __shfl_xor_sync(0xffffffffu, lsw, o);
      lsb += __shfl_xor_sync(0xffffffffu, lsb, o);
    }
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = lsw;
      red[1][tid >> 5] = lsb;
    }
    __syncthreads();
    if (tid == 0) {
      double a1 = 0.0, b1 = 0.0;
      for (int w = 0; w < (bd >> 5); ++w) {
        a1 += red[0][w];
        b1 += red[1][w];
      }
      atomicAdd(dsw2, a1 / sw2);
      atomicAdd(dsb2, b1);
    }
    __syncthreads();
  }
}

template <typename T>
struct BwdPlan {
  int64_t chunk;
  size_t stored_per_pair;  // elements of T
  size_t hw0sq;
  size_t bytes;            // total workspace
  size_t self_bytes;
  SelfAdjGeom sg;
  int self_grid;
};

template <typename T>
BwdPlan<T> plan_backward(const NkGeom& g, int64_t npairs, int64_t na, int64_t nb, int sym, int sm) {
  BwdPlan<T> P = {};
  P.hw0sq = (size_t)g.Hs[0] * g.Ws[0] * g.Hs[0] * g.Ws[0];
  int layer = 0;
  for (int s = 0; s < g.n_stages; ++s)
    for (int k = 0; k < g.convs[s]; ++k, ++layer) {
      const size_t hw = (size_t)g.Hs[s] * g.Ws[s];
      P.stored_per_pair += hw * hw;
    }
  const size_t per_pair = (P.stored_per_pair + 3 * P.hw0sq + 2) * sizeof(T);
  const size_t budget = (size_t)3 << 30;
  P.chunk = (int64_t)std::max<size_t>(1, budget / per_pair);
  if (P.chunk > npairs) P.chunk = npairs;
  // self adjoint
  P.sg.g = g;
  int64_t off = 0;
  int64_t mx = 0;
  layer = 0;
  for (int s = 0; s <= g.last_act_stage; ++s) {
    const int64_t D = 2 * g.radius[s] + 1;
    const int64_t planes = D * D * g.Hs[s] * g.Ws[s];
    mx = std::max(mx, planes);
    for (int k = 0; k < g.convs[s]; ++k, ++layer) {
      P.sg.store_off[layer] = off;
      off += planes;
    }
  }
  P.sg.store_total = off;
  P.sg.work = mx;
  P.self_grid = (int)std::max<int64_t>(1, std::min<int64_t>(std::max(na, sym ? na : nb), sm));
  P.self_bytes = (size_t)P.self_grid * (size_t)(off + 3 * mx) * sizeof(double);
  const size_t nqa = (size_t)na * g.nq, nqb = sym ? 0 : (size_t)nb * g.nq;
  P.bytes = per_pair * P.chunk + (nqa + nqb) * sizeof(T) + P.self_bytes + 4096;
  return P;
}

template <typename T>
cudaError_t run_backward(const NkGeom& g, double sw2, double sb2, const float* Xa, const double* qda,
                         const float* qsa, int64_t a0, int64_t a1, const float* Xb, const double* qdb,
                         const float* qsb, int64_t b0, int64_t b1, const T* dK, int64_t lddk, int sym, T* dXa, T* dXb,
                         double* dsw2, double* dsb2, void* ws, const BwdPlan<T>& P, cudaStream_t st,
                         int64_t* launches, unsigned int* dstatus) {
  const int64_t na = a1 - a0, nb = b1 - b0;
  const int64_t npairs = sym ? na * (na + 1) / 2 : na * nb;
  const int64_t chunk = P.chunk;
  // carve the workspace
  char* w = reinterpret_cast<char*>(ws);
  auto take = [&](size_t bytes) {
    char* p = w;
    w += (bytes + 255) / 256 * 256;
    return p;
  };
  T* stored = reinterpret_cast<T*>(take(P.stored_per_pair * chunk * sizeof(T)));
  T* cur0 = reinterpret_cast<T*>(take(P.hw0sq * chunk * sizeof(T)));
  T* nxt0 = reinterpret_cast<T*>(take(P.hw0sq * chunk * sizeof(T)));
  T* hbuf = reinterpret_cast<T*>(take(P.hw0sq * chunk * sizeof(T)));
  T* useed = reinterpret_cast<T*>(take(chunk * sizeof(T)));
  T* gmean = reinterpret_cast<T*>(take(chunk * sizeof(T)));
  T* dqa = reinterpret_cast<T*>(take((size_t)na * g.nq * sizeof(T)));
  T* dqb = sym ? dqa : reinterpret_cast<T*>(take((size_t)nb * g.nq * sizeof(T)));
  double* sws = reinterpret_cast<double*>(take(P.self_bytes));
  cudaError_t e = cudaMemsetAsync(dqa, 0, (size_t)na * g.nq * sizeof(T), st);
  if (e == cudaSuccess && !sym) e = cudaMemsetAsync(dqb, 0, (size_t)nb * g.nq * sizeof(T), st);
  if (e != cudaSuccess) return e;
  const T a_conv = (T)(sw2 / (double)(g.filter * g.filter));
  const bool relu = (g.act == NK_ACT_RELU);
  int last_conv_stage = 0;
  for (int s = 0; s < g.n_stages; ++s)
    if (g.convs[s] > 0) last_conv_stage = s;
  const double hwl = (double)g.Hs[last_conv_stage] * g.Ws[last_conv_stage];

  for (int64_t pair0 = 0; pair0 < npairs; pair0 += chunk) {
    const int64_t np = std::min<int64_t>(chunk, npairs - pair0);
    // ---- forward, storing each layer's pre-activation tensor
    T* cur = cur0;
    T* nxt = nxt0;
    T* Kst[NK_MAX_LAYERS];
    {
      size_t off = 0;
      int layer = 0;
      for (int s = 0; s < g.n_stages; ++s)
        for (int k = 0; k < g.convs[s]; ++k, ++layer) {
          Kst[layer] = stored + off * np;
          off += (size_t)g.Hs[s] * g.Ws[s] * g.Hs[s] * g.Ws[s];
        }
    }
    ++*launches;
    k_input_cov<T><<<pair_grid(np, (int64_t)P.hw0sq), 256, 0, st>>>(Xa, Xb, a0, b0, na, nb, sym, pair0, np,
                                                                     g.Hs[0], g.Ws[0], g.C, cur);
    int layer = 0;
    for (int s = 0; s <= last_conv_stage; ++s) {
      const int H = g.Hs[s], W = g.Ws[s];
      const int64_t HW = (int64_t)H * W;
      if (s > 0) {
        ++*launches;
        k_pool<T><<<grid_for(np * HW * HW), 256, 0, st>>>(cur, nxt, np, 2 * H, 2 * W);
        T* t = cur; cur = nxt; nxt = t;
      }
      for (int k = 0; k < g.convs[s]; ++k, ++layer) {
        ++*launches;
        conv_layer<T>(cur, Kst[layer], np, H, W, g.filter, a_conv, (T)sb2, st);
        if (relu) {
          // the pre-activation stays in Kst for the reverse sweep
          ++*launches;
          k_relu<T><<<pair_grid(np, HW * HW), 256, 0, st>>>(Kst[layer], nxt, np, (int)HW, na, nb, sym, pair0, a0,
                                                            b0, qda, qdb, qsa, qsb, g.nq, g.layer_qoff[layer],
                                                            dstatus);
        } else {
          e = cudaMemcpyAsync(nxt, Kst[layer], (size_t)np * HW * HW * sizeof(T), cudaMemcpyDeviceToDevice, st);
          if (e != cudaSuccess) return e;
        }
        T* t = cur; cur = nxt; nxt = t;
      }
    }
    // cur: post-activation of the last conv layer; its mean is the readout's
    const int64_t HWl = (int64_t)g.Hs[last_conv_stage] * g.Ws[last_conv_stage];
    ++*launches;
    k_pair_mean<T><<<(unsigned)np, 256, 0, st>>>(cur, HWl * HWl, gmean);
    // ---- reverse
    ++*launches;
    k_pair_seed<T><<<grid_for(np), 256, 0, st>>>(dK, lddk, gmean, na, nb, sym, pair0, np, sw2, hwl * hwl, useed,
                                                 dsw2, dsb2);
    ++*launches;
    k_fill_pairs<T><<<grid_for(np * HWl * HWl), 256, 0, st>>>(cur, np, HWl * HWl, useed);
    for (int s = last_conv_stage; s >= 0; --s) {
      const int H = g.Hs[s], W = g.Ws[s];
      const int64_t HW = (int64_t)H * W;
      for (int k = g.convs[s] - 1; k >= 0; --k) {
        --layer;
        if (relu) {
          *launches += 3;
          k_map_adj<T><<<pair_grid(np, HW * HW), 256, 0, st>>>(Kst[layer], cur, hbuf, np, (int)HW, na, nb, sym,
                                                               pair0, a0, b0, qda, qdb, qsa, qsb, g.nq,
                                                               g.layer_qoff[layer], sb2, 1.0 / sw2, dsw2, dsb2);
          k_rowsum_q<T><<<grid_for(np * HW * 32), 256, 0, st>>>(hbuf, np, (int)HW, na, nb, sym, pair0, a0, qda,
                                                                g.nq, g.layer_qoff[layer], dqa);
          k_colsum_q<T><<<grid_for(np * HW), 256, 0, st>>>(hbuf, np, (int)HW, na, nb, sym, pair0, b0, qdb, g.nq,
                                                           g.layer_qoff[layer], dqb);
        }
        ++*launches;
        if (!relu) {  // with a ReLU the map adjoint has added the sigma terms
          ++*launches;
          k_sigma_terms<T><<<std::min(grid_for(np * HW * HW), 1024), 256, 0, st>>>(cur, Kst[layer], np * HW * HW,
                                                                                 sb2, 1.0 / sw2, dsw2, dsb2);
        }
        conv_layer<T>(cur, nxt, np, H, W, g.filter, a_conv, (T)0, st);
        T* t = cur; cur = nxt; nxt = t;
      }
      if (s > 0) {
        const int64_t HWp = 4 * HW;
        ++*launches;
        k_pool_adj<T><<<grid_for(np * HWp * HWp), 256, 0, st>>>(cur, nxt, np, H, W);
        T* t = cur; cur = nxt; nxt = t;
      }
    }
    const int HW0 = g.Hs[0] * g.Ws[0];
    if (dXa) {
      ++*launches;
      k_seed_adj_a<T><<<grid_for((int64_t)np * HW0 * 32), 256, 0, st>>>(cur, Xb, np, HW0, g.C, na, nb, sym, pair0,
                                                                        a0, b0, dXa);
    }
    T* dXb_eff = sym ? dXa : dXb;
    if (dXb_eff) {
      ++*launches;
      k_seed_adj_b<T><<<grid_for((int64_t)np * HW0), 256, 0, st>>>(cur, Xa, np, HW0, g.C, na, nb, sym, pair0, a0,
                                                                   b0, dXb_eff);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // ---- self-variance adjoint (images a; images b unless symmetric)
  if (relu) {
    const size_t smem = (size_t)g.Hs[0] * g.Ws[0] * (2 * g.C + 1) * sizeof(double);
    e = cudaFuncSetAttribute(k_self_adj<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ++*launches;
    k_self_adj<T><<<std::min<int64_t>(na, P.self_grid), 256, smem, st>>>(P.sg, sw2, sb2, Xa, na, a0, dqa, dXa, dsw2,
                                                                          dsb2, sws);
    if (!sym) {
      ++*launches;
      k_self_adj<T><<<std::min<int64_t>(nb, P.self_grid), 256, smem, st>>>(P.sg, sw2, sb2, Xb, nb, b0, dqb, dXb,
                                                                            dsw2, dsb2, sws);
    }
  }
  return cudaGetLastError();
}

}  // namespace

size_t nk_backward_ws_bytes(const NkGeom& g, int fp64, int64_t npairs, int64_t na, int64_t nb, int sym, int sm) {
  return fp64 ? plan_backward<double>(g, npairs, na, nb, sym, sm).bytes
              : plan_backward<float>(g, npairs, na, nb, sym, sm).bytes;
}

cudaError_t nk_launch_backward(const NkGeom& g, int fp64, double sw2, double sb2, const float* Xa,
                               const double* qda, const float* qsa, int64_t a0, int64_t a1, const float* Xb,
                               const double* qdb, const float* qsb, int64_t b0, int64_t b1, const void* dK,
                               int64_t lddk, int sym, void* dXa, void* dXb, double* dsw2, double* dsb2,
                               void* ws, int sm, cudaStream_t st, int64_t* launches,
                               unsigned int* dstatus) {
  const int64_t na = a1 - a0, nb = b1 - b0;
  const int64_t npairs = sym ? na * (na + 1) / 2 : na * nb;
  if (fp64) {
    auto P = plan_backward<double>(g, npairs, na, nb, sym, sm);
    return run_backward<double>(g, sw2, sb2, Xa, qda, qsa, a0, a1, Xb, qdb, qsb, b0, b1, (const double*)dK, lddk,
                                sym, (double*)dXa, (double*)dXb, dsw2, dsb2, ws, P, st, launches, dstatus);
  }
  auto P = plan_backward<float>(g, npairs, na, nb, sym, sm);
  return run_backward<float>(g, sw2, sb2, Xa, qda, qsa, a0, a1, Xb, qdb, qsb, b0, b1, (const float*)dK, lddk,
                             sym, (float*)dXa, (float*)dXb, dsw2, dsb2, ws, P, st, launches, dstatus);
}
