// nk_block_backward: adjoint of the Myrtle NNGP kernel block (layer-wise form,
// FP32 or FP64).
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
//
// Layer-fused passes.  Every pass over a pixel-pair tensor is one streamed
// 3x3 diagonal stencil (k_conv_fused) whose input transform is applied while
// a plane is loaded: forward, the input covariance (first layer) or the
// previous layer's map of the stored pre-activation; reverse, the map adjoint
// of this layer's stored pre-activation and the incoming gradient, which is
// read from a full tensor, from the next stage's gradient through the pool
// adjoint (index / 2, value / 16), or as the pair's readout constant.  The
// reverse pass also takes the sigma sums and, per plane, the row and column
// sums of the map's q-terms (small partial buffers, reduced per pixel after
// the pass).  Only the pre-activation of each layer is stored (HBM); per pair
// and stage-0 layer that is one write forward, two reads and one write in
// reverse.  The next plane's loads are issued into registers before the
// current plane's barriers, so their latency overlaps the stencil work.
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

// ---------------------------------------------------------------------------
// Layer-fused streamed stencil.
// ---------------------------------------------------------------------------
enum { CIN_COV = 0, CIN_PLAIN = 1, CIN_MAP = 2, CIN_ADJ = 3 };
enum { G_TENSOR = 0, G_POOLED = 1, G_CONST = 2 };

template <typename T>
struct FArgs {
  int64_t np, pair0, na, nb, a0, b0;
  int sym, H, W;
  const T* src;            // CIN_PLAIN / CIN_MAP: input tensor; CIN_ADJ: this layer's pre-activation
  const float* Xa;         // CIN_COV: the images
  const float* Xb;
  int C;
  int relu;                // CIN_MAP / CIN_ADJ: ReLU map (else identity)
  const double* qda;       // self-variances (FP64 form) and their FP32 tables
  const double* qdb;
  const float* qsa;
  const float* qsb;
  int64_t nq;
  int qoff;                // layer offset in the q rows (of the layer whose map is applied)
  const T* gsrc;           // CIN_ADJ: gradient of this layer's post-activation
  int gmode;               // G_TENSOR: same layout; G_POOLED: the next stage's tensor; G_CONST: [np]
  T* out;                  // a S(v) + b of the transformed input v
  T a, b;
  T* prow;                 // CIN_ADJ: [np][H][H][W] per-plane row sums of the q-terms h
  T* pcol;                 //          [np][H][H][W] per-plane column sums
  double sb2, inv_sw2;
  double* dsw2;
  double* dsb2;
};

// The activation's scale factors of pixel p (image a) and p' (image b):
// s = sqrt(q q'), rs = 1 / sqrt(q q').
template <typename T>
__device__ __forceinline__ void act_scale(const FArgs<T>& A, int64_t ia, int64_t ib, int p, int pp, T& s, T& rs) {
  if constexpr (sizeof(T) == 8) {
    s = sqrt(A.qda[ia * A.nq + A.qoff + p] * A.qdb[ib * A.nq + A.qoff + pp]);
    rs = s > 0.0 ? 1.0 / s : 0.0;
  } else {
    const float2 s1 = reinterpret_cast<const float2*>(A.qsa)[ia * A.nq + A.qoff + p];
    const float2 s2 = reinterpret_cast<const float2*>(A.qsb)[ib * A.nq + A.qoff + pp];
    s = s1.y * s2.y;
    rs = s1.x * s2.x;
  }
}

// Raw input of element (p, p') = ((ii, jj), (kk, ll)) of pair pr: k, and
// (reverse) the incoming gradient g.  W is the stage width.
template <typename T, int MODE, int W>
__device__ __forceinline__ void fetch_el(const FArgs<T>& A, int64_t pr, int64_t ia, int64_t ib, int ii, int jj,
                                         int kk, int ll, T& k, T& g) {
  const int HW = A.H * W;
  const int p = ii * W + jj, pp = kk * W + ll;
  if constexpr (MODE == CIN_COV) {
    const float* xa = A.Xa + (ia * HW + p) * (int64_t)A.C;
    const float* xb = A.Xb + (ib * HW + pp) * (int64_t)A.C;
    T acc = 0;
    for (int c = 0; c < A.C; ++c) acc += (T)xa[c] * (T)xb[c];
    k = acc / (T)A.C;
  } else {
    k = A.src[pr * (int64_t)HW * HW + (int64_t)p * HW + pp];
  }
  if constexpr (MODE == CIN_ADJ) {
    if (A.gmode == G_TENSOR) {
      g = A.gsrc[pr * (int64_t)HW * HW + (int64_t)p * HW + pp];
    } else if (A.gmode == G_POOLED) {
      constexpr int Wn = W / 2;
      const int HWn = (A.H >> 1) * Wn;
      const int P = (ii >> 1) * Wn + (jj >> 1), PP = (kk >> 1) * Wn + (ll >> 1);
      g = A.gsrc[pr * (int64_t)HWn * HWn + (int64_t)P * HWn + PP] * (T)(1.0 / 16.0);
    } else {
      g = A.gsrc[pr];
    }
  }
}

// The transform of one element: input covariance / plain value, the map, or
// the map adjoint (h = its q-term, sa / sb the sigma sums).  FP32 evaluates J
// and J' = pi - arccos c by the library's polynomial forms (nk_map.cuh), FP64
// by acos.
template <typename T>
__device__ __forceinline__ void J_dJ(T c, T& J, T& dJ) {
  if constexpr (sizeof(T) == 8) {
    c = c < -1.0 ? -1.0 : (c > 1.0 ? 1.0 : c);
    const double th = acos(c);
    J = sqrt(fmax(1.0 - c * c, 0.0)) + c * (NK_PI_D - th);
    dJ = NK_PI_D - th;
  } else {
    nk_J_dJ_f32(c, J, dJ);
  }
}

template <typename T>
__device__ __forceinline__ T J_only(T c) {
  if constexpr (sizeof(T) == 8) {
    c = c < -1.0 ? -1.0 : (c > 1.0 ? 1.0 : c);
    return sqrt(fmax(1.0 - c * c, 0.0)) + c * (NK_PI_D - acos(c));
  } else {
    return nk_J_f32(c);
  }
}

// s += x with Kahan compensation c (s - c is the compensated sum).
template <typename T>
__device__ __forceinline__ void kahan_add(T& s, T& c, T x) {
  const T y = x - c;
  const T t = s + y;
  c = (t - s) - y;
  s = t;
}

template <typename T, int MODE>
__device__ __forceinline__ T xform(const FArgs<T>& A, int64_t ia, int64_t ib, int p, int pp, T k, T g, T& h, T& sa,
                                   T& sb) {
  if constexpr (MODE == CIN_COV || MODE == CIN_PLAIN) {
    return k;
  } else {
    const T inv2pi = (T)NK_INV_2PI_D;
    if constexpr (MODE == CIN_MAP) {
      if (!A.relu) return k;
      T s, rs;
      act_scale(A, ia, ib, p, pp, s, rs);
      if (!(s > (T)0)) return (T)0;
      return s * inv2pi * J_only<T>(k * rs);
    } else {
      T dk = g;
      h = 0;
      if (A.relu) {
        dk = 0;
        T s, rs;
        act_scale(A, ia, ib, p, pp, s, rs);
        if (s > (T)0) {
          T J, dJ;
          J_dJ<T>(k * rs, J, dJ);
          const T Kt = s * inv2pi * J;
          dk = g * dJ * inv2pi;
          h = g * (Kt - k * dJ * inv2pi);
        }
      }
      sa += dk * (k - (T)A.sb2);
      sb += dk;
      return dk;
    }
  }
}

// Shared memory of k_conv_fused, in elements of T: two buffers (by plane
// parity) of the transformed plane and, reverse, of its q-terms and of the
// column partials of those q-terms.
template <typename T, int MODE, int W, int NPB>
__host__ __device__ constexpr size_t conv_smem_bytes() {
  constexpr int W2 = W * W, CG = W >= 32 ? 256 / W : 1;
  // per pair the two images' factor tables of the layer (H = W): float2 in
  // FP32, the q values (double) in FP64
  constexpr size_t tab = (MODE == CIN_MAP || MODE == CIN_ADJ) ? (size_t)NPB * 2 * W2 * 8 : 0;  // float2 or double
  return (size_t)(2 * NPB * W2 + (MODE == CIN_ADJ ? 2 * NPB * W2 + 2 * NPB * CG * W : 0)) * sizeof(T) + tab;
}

// One block per (group of NPB pairs, diagonal d = k - i of the (i, k)
// image-row planes).  Each thread owns EPT fixed in-plane elements (jj, ll)
// of every plane of the diagonal, so all its addresses are a per-plane base
// plus a per-thread offset.  Per plane s: transform the loaded values (the
// loads of plane s + 2 are then issued), publish them in shared memory (two
// buffers by plane parity, one barrier per plane), row-filter the thread's own
// elements along the (j, l) diagonal (its value plus two neighbours), and
// output plane s - 1 from a register ring of the last three row-filtered
// planes.  Reverse: the q-terms' row sums of a plane are read as float4 runs
// and reduced over the row's lanes by shuffles; column sums are per-warp
// partials finished one plane later (stages narrower than 32 sum with plain
// loops).  The stage is square (H = W, a compile-time constant), and each
// pair's factor tables of the layer (both images, H x W entries each) are
// staged in shared memory once per block.
template <typename T, int MODE, int W, int NPB>
__global__ void __launch_bounds__(256, 3) k_conv_fused(const __grid_constant__ FArgs<T> A) {
  extern __shared__ __align__(16) unsigned char fsm[];
  T* sh = reinterpret_cast<T*>(fsm);
  constexpr int W2 = W * W, EPT = W2 > 256 ? W2 / 256 : 1;
  constexpr bool WIDE = W >= 32;
  constexpr int CG = WIDE ? 256 / W : 1;  // column groups (one per W threads)
  constexpr int H = W, HW = W2;
  constexpr bool TAB = (MODE == CIN_MAP || MODE == CIN_ADJ);
  T* raw = sh;                            // [2][NPB][W2]
  T* hs = raw + 2 * NPB * W2;             // [2][NPB][W2] (reverse only)
  T* cpart = hs + 2 * NPB * W2;           // [2][NPB][CG][W] (reverse only)
  // [NPB][2][HW] factor tables: (1/sqrt q, sqrt q) pairs in FP32, q in FP64;
  // they follow the last buffer this mode has (conv_smem_bytes)
  constexpr int TAB_OFF = MODE == CIN_ADJ ? 4 * NPB * W2 + 2 * NPB * CG * W : 2 * NPB * W2;
  float2* tab2 = reinterpret_cast<float2*>(sh + TAB_OFF);
  double* tabd = reinterpret_cast<double*>(tab2);
  const int tid = threadIdx.x, lane = tid & 31;
  const int d = (int)blockIdx.x - (H - 1);
  const int i0 = d < 0 ? -d : 0;
  const int i1 = (d > 0 ? H - d : H) - 1;
  // the thread's elements: in-plane coordinates, offsets and stencil masks
  int jj_[EPT], ll_[EPT], off_[EPT], offg_[EPT];
  bool in_[EPT];
  T mlo_[EPT], mhi_[EPT];
  constexpr int HWn = (H >> 1) * (W >> 1);
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    const int e = tid + u * 256;
    in_[u] = e < W2;
    jj_[u] = e / W;
    ll_[u] = e % W;
    off_[u] = jj_[u] * HW + ll_[u];
    offg_[u] = (jj_[u] >> 1) * HWn + (ll_[u] >> 1);
    mlo_[u] = (jj_[u] > 0 && ll_[u] > 0) ? (T)1 : (T)0;
    mhi_[u] = (jj_[u] + 1 < W && ll_[u] + 1 < W) ? (T)1 : (T)0;
  }
  // sigma sums (reverse): per plane in T, then in FP64.  FP32 at W = 32 sums
  // a pair group's planes in FP32 with Kahan compensation first, which keeps
  // FP64 instructions (about 1/64 of the FP32 rate) out of the plane loop;
  // the other forms, short of registers or in FP64, add each plane in FP64.
  constexpr bool KAHAN = MODE == CIN_ADJ && W == 32 && sizeof(T) == 4;
  const T sb2 = (T)A.sb2;
  double dsa = 0.0, dsb = 0.0;
  for (int64_t pg = (int64_t)blockIdx.y * NPB; pg < A.np; pg += (int64_t)gridDim.y * NPB) {
    T csa = 0, csb = 0, ksa = 0, ksb = 0;
    int64_t ia[NPB], ib[NPB];
    bool ok[NPB];
#pragma unroll
    for (int b = 0; b < NPB; ++b) {
      ok[b] = pg + b < A.np;
      int64_t i = 0, j = 0;
      if (ok[b]) pair_of(A.pair0 + pg + b, A.na, A.nb, A.sym, &i, &j);
      ia[b] = A.a0 + i;
      ib[b] = A.b0 + j;
    }
    // loads of plane ii into (rk, rg)
    T k0[NPB][EPT], g0[NPB][EPT], k1[NPB][EPT], g1[NPB][EPT];
    auto fetch = [&](int ii, T (&rk)[NPB][EPT], T (&rg)[NPB][EPT]) {
      const int kk = ii + d;
#pragma unroll
      for (int b = 0; b < NPB; ++b) {
        const int64_t pbase = (pg + b) * (int64_t)HW * HW + (int64_t)(ii * W) * HW + kk * W;
#pragma unroll
        for (int u = 0; u < EPT; ++u) {
          rk[b][u] = 0;
          rg[b][u] = 0;
          if (!ok[b] || !in_[u]) continue;
          if constexpr (MODE == CIN_COV) {
            const float* xa = A.Xa + ((ia[b] * HW + ii * W + jj_[u]) * (int64_t)A.C);
            const float* xb = A.Xb + ((ib[b] * HW + kk * W + ll_[u]) * (int64_t)A.C);
            T acc = 0;
            for (int c = 0; c < A.C; ++c) acc += (T)xa[c] * (T)xb[c];
            rk[b][u] = acc / (T)A.C;
          } else {
            rk[b][u] = A.src[pbase + off_[u]];
          }
          if constexpr (MODE == CIN_ADJ) {
            if (A.gmode == G_TENSOR)
              rg[b][u] = A.gsrc[pbase + off_[u]];
            else if (A.gmode == G_POOLED)
              rg[b][u] = A.gsrc[(pg + b) * (int64_t)HWn * HWn + (int64_t)((ii >> 1) * (W >> 1)) * HWn +
                                (kk >> 1) * (W >> 1) + offg_[u]] *
                         (T)(1.0 / 16.0);
            else
              rg[b][u] = A.gsrc[pg + b];
          }
        }
      }
    };
    T rA[NPB][EPT], rB[NPB][EPT], rC[NPB][EPT];  // row-filtered planes s - 2, s - 1, s
#pragma unroll
    for (int b = 0; b < NPB; ++b)
#pragma unroll
      for (int u = 0; u < EPT; ++u) rA[b][u] = rB[b][u] = rC[b][u] = 0;
    auto step = [&](int s, T (&rk)[NPB][EPT], T (&rg)[NPB][EPT]) {
      const int par = s & 1;
      T own[NPB][EPT];
      if (s <= i1) {
        // ---- transform plane s, publish it
        const int kk = s + d;
        T sa = 0, sb = 0;
#pragma unroll
        for (int b = 0; b < NPB; ++b) {
          T* rw = raw + (par * NPB + b) * W2;
          T* hw = hs + (par * NPB + b) * W2;
#pragma unroll
          for (int u = 0; u < EPT; ++u) {
            own[b][u] = 0;
            if (!in_[u]) continue;
            T h = 0;
            T v = rk[b][u];
            if constexpr (MODE == CIN_MAP || MODE == CIN_ADJ) {
              if (A.relu) {
                T sc, rs;
                if constexpr (sizeof(T) == 8) {
                  const double q1 = tabd[(b * 2) * HW + s * W + jj_[u]];
                  const double q2 = tabd[(b * 2 + 1) * HW + kk * W + ll_[u]];
                  sc = sqrt(q1 * q2);
                  rs = sc > 0.0 ? 1.0 / sc : 0.0;
                } else {
                  const float2 s1 = tab2[(b * 2) * HW + s * W + jj_[u]];
                  const float2 s2 = tab2[(b * 2 + 1) * HW + kk * W + ll_[u]];
                  sc = s1.y * s2.y;
                  rs = s1.x * s2.x;
                }
                const T inv2pi = (T)NK_INV_2PI_D;
                if constexpr (MODE == CIN_MAP) {
                  v = sc > (T)0 ? sc * inv2pi * J_only<T>(v * rs) : (T)0;
                } else {
                  T dk = 0;
                  if (sc > (T)0) {
                    T J, dJ;
                    J_dJ<T>(v * rs, J, dJ);
                    dk = rg[b][u] * dJ * inv2pi;
                    h = rg[b][u] * (sc * inv2pi * J - v * dJ * inv2pi);
                  }
                  sa += dk * (v - sb2);
                  sb += dk;
                  v = dk;
                }
              } else if constexpr (MODE == CIN_ADJ) {
                sa += rg[b][u] * (v - sb2);
                sb += rg[b][u];
                v = rg[b][u];
              }
            }
            own[b][u] = v;
            rw[jj_[u] * W + ll_[u]] = v;
            if constexpr (MODE == CIN_ADJ) hw[jj_[u] * W + ll_[u]] = h;
          }
        }
        if constexpr (KAHAN) {
          kahan_add(csa, ksa, sa);
          kahan_add(csb, ksb, sb);
        } else if constexpr (MODE == CIN_ADJ) {
          dsa += (double)sa;
          dsb += (double)sb;
        }
        if (s + 2 <= i1) fetch(s + 2, rk, rg);  // in flight during the next two planes
      }
      __syncthreads();
      if (s <= i1) {
        // ---- row filter of the thread's own elements
#pragma unroll
        for (int b = 0; b < NPB; ++b) {
          const T* rw = raw + (par * NPB + b) * W2;
#pragma unroll
          for (int u = 0; u < EPT; ++u) {
            const int f = jj_[u] * W + ll_[u];
            T v = own[b][u];
            if (in_[u]) {
              if (jj_[u] > 0 && ll_[u] > 0) v += rw[f - W - 1];
              if (jj_[u] + 1 < W && ll_[u] + 1 < W) v += rw[f + W + 1];
            }
            rC[b][u] = v;
          }
        }
        if constexpr (MODE == CIN_ADJ) {
          const int kk = s + d;
          if constexpr (WIDE) {
            // rows: float4 runs, W/4 lanes per row reduced by shuffles
            constexpr int RT = W / 4, RPI = 256 / RT;
            for (int b = 0; b < NPB; ++b) {
              const float4* h4 = reinterpret_cast<const float4*>(hs + (par * NPB + b) * W2);
              const int64_t base = (((pg + b) * H + s) * (int64_t)H + kk) * W;
              for (int r0 = 0; r0 < W; r0 += RPI) {
                const int r = r0 + tid / RT, g = tid % RT;
                T v = 0;
                if constexpr (sizeof(T) == 4) {
                  const float4 x = h4[r * RT + g];
                  v = (x.x + x.y) + (x.z + x.w);
                } else {
                  const T* hb = hs + (par * NPB + b) * W2 + r * W + 4 * g;
                  v = (hb[0] + hb[1]) + (hb[2] + hb[3]);
                }
#pragma unroll
                for (int o = RT / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (g == 0 && ok[b]) A.prow[base + r] = v;
              }
              // columns: this thread's W / CG rows of column tid % W
              const T* hb = hs + (par * NPB + b) * W2;
              const int c = tid % W, cg = tid / W;
              T v = 0;
#pragma unroll
              for (int i = 0; i < W / CG; ++i) v += hb[(cg * (W / CG) + i) * W + c];
              cpart[((par * NPB + b) * CG + cg) * W + c] = v;
            }
          } else {
            // narrow stages: one thread per row / column sum
            for (int t = tid; t < NPB * 2 * W; t += 256) {
              const int b = t / (2 * W), r = t - b * 2 * W;
              if (!ok[b]) continue;
              const T* hb = hs + (par * NPB + b) * W2;
              T v = 0;
              if (r < W) {
                for (int l = 0; l < W; ++l) v += hb[r * W + ((l + r) & (W - 1))];
              } else {
                for (int jj = 0; jj < W; ++jj) v += hb[jj * W + (r - W)];
              }
              const int64_t base = (((pg + b) * H + s) * (int64_t)H + kk) * W;
              if (r < W)
                A.prow[base + r] = v;
              else
                A.pcol[base + r - W] = v;
            }
          }
        }
      }
      if constexpr (MODE == CIN_ADJ && WIDE) {
        // the column sums of plane s - 1 (partials published before this
        // plane's barrier)
        if (s - 1 >= i0) {
          const int io = s - 1, ko = io + d, pp = io & 1;
          for (int t = tid; t < NPB * W; t += 256) {
            const int b = t / W, c = t - b * W;
            if (!ok[b]) continue;
            T v = 0;
#pragma unroll
            for (int g = 0; g < CG; ++g) v += cpart[((pp * NPB + b) * CG + g) * W + c];
            A.pcol[(((pg + b) * H + io) * (int64_t)H + ko) * W + c] = v;
          }
        }
      }
      // ---- output plane s - 1 from the register ring
      if (s - 1 >= i0) {
        const int io = s - 1, ko = io + d;
#pragma unroll
        for (int b = 0; b < NPB; ++b) {
          if (!ok[b]) continue;
          T* dst = A.out + (pg + b) * (int64_t)HW * HW + (int64_t)(io * W) * HW + ko * W;
#pragma unroll
          for (int u = 0; u < EPT; ++u) {
            if (!in_[u]) continue;
            T acc = rB[b][u];
            if (io > i0) acc += rA[b][u];
            if (io < i1) acc += rC[b][u];
            dst[off_[u]] = A.a * acc + A.b;
          }
        }
      }
#pragma unroll
      for (int b = 0; b < NPB; ++b)
#pragma unroll
        for (int u = 0; u < EPT; ++u) {
          rA[b][u] = rB[b][u];
          rB[b][u] = rC[b][u];
        }
    };
    __syncthreads();  // the previous group's buffers are no longer read
    if constexpr (TAB) {
      if (A.relu) {
        for (int t = tid; t < NPB * 2 * HW; t += 256) {
          const int b = t / (2 * HW), r = t - b * 2 * HW, side = r / HW, e = r - side * HW;
          if (!ok[b]) continue;
          const int64_t row = (side == 0 ? ia[b] : ib[b]) * A.nq + A.qoff + e;
          if constexpr (sizeof(T) == 8)
            tabd[(b * 2 + side) * HW + e] = (side == 0 ? A.qda : A.qdb)[row];
          else
            tab2[(b * 2 + side) * HW + e] = reinterpret_cast<const float2*>(side == 0 ? A.qsa : A.qsb)[row];
        }
      }
      __syncthreads();  // the tables are read by every thread's first transform
    }
    fetch(i0, k0, g0);
    if (i0 + 1 <= i1) fetch(i0 + 1, k1, g1);
    int s = i0;
    for (; s + 1 <= i1 + 1; s += 2) {
      step(s, k0, g0);
      step(s + 1, k1, g1);
    }
    if (s <= i1 + 1) step(s, k0, g0);
    if constexpr (KAHAN) {
      dsa += (double)csa - (double)ksa;
      dsb += (double)csb - (double)ksb;
    }
  }
  if constexpr (MODE == CIN_ADJ) {
    __shared__ double r1[8], r2[8];
    for (int o = 16; o > 0; o >>= 1) {
      dsa += __shfl_xor_sync(0xffffffffu, dsa, o);
      dsb += __shfl_xor_sync(0xffffffffu, dsb, o);
    }
    if (lane == 0) {
      r1[tid >> 5] = dsa;
      r2[tid >> 5] = dsb;
    }
    __syncthreads();
    if (tid == 0) {
      double x = 0.0, y = 0.0;
      for (int w = 0; w < 8; ++w) {
        x += r1[w];
        y += r2[w];
      }
      if (x != 0.0 || y != 0.0) {
        atomicAdd(A.dsw2, x * A.inv_sw2);
        atomicAdd(A.dsb2, y);
      }
    }
  }
}

// Forward pool with the map of the previous layer applied on load:
// out(P, P') = 1/16 sum_{a,b} map(src(2P + a, 2P' + b)) at output H x W.
template <typename T>
__global__ void k_pool_map(const FArgs<T> A, int Ho, int Wo) {
  const int Hi = 2 * Ho, Wi = 2 * Wo;
  const int64_t HWi = (int64_t)Hi * Wi, HWo = (int64_t)Ho * Wo;
  const int64_t total = A.np * HWo * HWo;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pr = e / (HWo * HWo), rem = e - pr * HWo * HWo;
    const int P = (int)(rem / HWo), PP = (int)(rem - (int64_t)P * HWo);
    int64_t i, j;
    pair_of(A.pair0 + pr, A.na, A.nb, A.sym, &i, &j);
    const int64_t ia = A.a0 + i, ib = A.b0 + j;
    const int I = P / Wo, J = P % Wo, K2 = PP / Wo, L = PP % Wo;
    T acc = 0, h = 0, sa = 0, sb = 0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        const int p = (2 * I + a) * Wi + 2 * J + b;
        for (int c = 0; c < 2; ++c)
          for (int dd = 0; dd < 2; ++dd) {
            const int pp = (2 * K2 + c) * Wi + 2 * L + dd;
            const T k = A.src[pr * HWi * HWi + (int64_t)p * HWi + pp];
            acc += xform<T, CIN_MAP>(A, ia, ib, p, pp, k, (T)0, h, sa, sb);
          }
      }
    A.out[e] = acc / (T)16;
  }
}

// Forward readout: the pair's mean of map(src) (before sw2 and sb2).
template <typename T>
__global__ void k_map_mean(const FArgs<T> A, T* __restrict__ mean) {
  __shared__ double red[32];
  const int64_t pr = blockIdx.x;
  const int HW = A.H * A.W;
  const int64_t HW2 = (int64_t)HW * HW;
  int64_t i, j;
  pair_of(A.pair0 + pr, A.na, A.nb, A.sym, &i, &j);
  const int64_t ia = A.a0 + i, ib = A.b0 + j;
  double acc = 0.0;
  T run = 0, h = 0, sa = 0, sb = 0;
  int n = 0;
  for (int64_t e = threadIdx.x; e < HW2; e += blockDim.x) {
    const int p = (int)(e / HW), pp = (int)(e - (int64_t)p * HW);
    run += xform<T, CIN_MAP>(A, ia, ib, p, pp, A.src[pr * HW2 + e], (T)0, h, sa, sb);
    if (++n == 64) {
      acc += (double)run;
      run = 0;
      n = 0;
    }
  }
  acc += (double)run;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) mean[pr] = (T)(acc / (double)HW2);
  }
}

// The q-terms per pixel: dq_a[i][p] += sum_k prow(p's plane row, k) / (2 q_a(p)),
// dq_b[j][p'] += sum_i pcol(i, p's plane) / (2 q_b(p')).
template <typename T>
__global__ void k_qsum(const FArgs<T> A, T* __restrict__ dqa, T* __restrict__ dqb) {
  const int H = A.H, W = A.W, HW = H * W;
  const int64_t total = A.np * HW;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 2 * total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const bool col = e >= total;
    const int64_t f = col ? e - total : e;
    const int64_t pr = f / HW;
    const int p = (int)(f - pr * HW);
    const int r = p / W, c = p - r * W;
    int64_t i, j;
    pair_of(A.pair0 + pr, A.na, A.nb, A.sym, &i, &j);
    T acc = 0;
    if (!col) {
      const T* base = A.prow + ((pr * H + r) * (int64_t)H) * W + c;  // (i = r, k, j = c)
      for (int k = 0; k < H; ++k) acc += base[(int64_t)k * W];
      const double q = A.qda[(A.a0 + i) * A.nq + A.qoff + p];
      if (q > 0.0 && acc != (T)0) atomicAdd(dqa + i * A.nq + A.qoff + p, (T)((double)acc / (2.0 * q)));
    } else {
      const T* base = A.pcol + ((pr * H) * (int64_t)H + r) * W + c;  // (i, k = r, l = c)
      for (int ii = 0; ii < H; ++ii) acc += base[(int64_t)ii * H * W];
      const double q = A.qdb[(A.b0 + j) * A.nq + A.qoff + p];
      if (q > 0.0 && acc != (T)0) atomicAdd(dqb + j * A.nq + A.qoff + p, (T)((double)acc / (2.0 * q)));
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

// FP32 input adjoints for C <= 3 with the pair's other image staged in shared
// memory as float4 (one broadcast or consecutive LDS.128 per element instead
// of C scalar loads).  Image b, one thread per column p' of a 256-column
// slab, eight rows' loads in flight:
//   dXb[j][p'][c] += (1/C) sum_p dK0(p,p') xa[p][c];
// image a, one warp per row p of an 8-row group:
//   dXa[i][p][c] += (1/C) sum_p' dK0(p,p') xb[p'][c].
__device__ __forceinline__ void stage_image4(const float* __restrict__ x, int HW, int C, float4* s) {
  for (int p = threadIdx.x; p < HW; p += blockDim.x) {
    const float* v = x + (int64_t)p * C;
    s[p] = make_float4(v[0], C > 1 ? v[1] : 0.f, C > 2 ? v[2] : 0.f, 0.f);
  }
}

__global__ void __launch_bounds__(256) k_seed_adj_b4(const float* __restrict__ d0, const float* __restrict__ Xa,
                                                     int64_t np, int HW, int C, int64_t na, int64_t nb, int sym,
                                                     int64_t pair0, int64_t a0, int64_t b0, float* __restrict__ dXb) {
  extern __shared__ float4 xs4[];
  const int pp = blockIdx.x * 256 + threadIdx.x;
  for (int64_t pr = blockIdx.y; pr < np; pr += gridDim.y) {
    int64_t i, j;
    pair_of(pair0 + pr, na, nb, sym, &i, &j);
    __syncthreads();  // the previous pair's image is no longer read
    stage_image4(Xa + (a0 + i) * (int64_t)HW * C, HW, C, xs4);
    __syncthreads();
    const float* col = d0 + pr * (int64_t)HW * HW + pp;
    float ax = 0.f, ay = 0.f, az = 0.f;
    for (int p = 0; p < HW; p += 8) {
      float g[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) g[u] = __ldcs(col + (int64_t)(p + u) * HW);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 x = xs4[p + u];
        ax = fmaf(g[u], x.x, ax);
        ay = fmaf(g[u], x.y, ay);
        az = fmaf(g[u], x.z, az);
      }
    }
    float* o = dXb + ((b0 + j) * (int64_t)HW + pp) * C;
    const float ic = 1.f / (float)C;
    atomicAdd(o, ax * ic);
    if (C > 1) atomicAdd(o + 1, ay * ic);
    if (C > 2) atomicAdd(o + 2, az * ic);
  }
}

__global__ void __launch_bounds__(256) k_seed_adj_a4(const float* __restrict__ d0, const float* __restrict__ Xb,
                                                     int64_t np, int HW, int C, int64_t na, int64_t nb, int sym,
                                                     int64_t pair0, int64_t a0, int64_t b0, float* __restrict__ dXa) {
  extern __shared__ float4 xs4[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t pr = blockIdx.y; pr < np; pr += gridDim.y) {
    int64_t i, j;
    pair_of(pair0 + pr, na, nb, sym, &i, &j);
    __syncthreads();
    stage_image4(Xb + (b0 + j) * (int64_t)HW * C, HW, C, xs4);
    __syncthreads();
    for (int p = blockIdx.x * 8 + warp; p < HW; p += gridDim.x * 8) {
      const float* row = d0 + (pr * (int64_t)HW + p) * HW;
      float ax = 0.f, ay = 0.f, az = 0.f;
      for (int k = lane; k < HW; k += 128) {
        float g[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) g[u] = __ldcs(row + k + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float4 x = xs4[k + 32 * u];
          ax = fmaf(g[u], x.x, ax);
          ay = fmaf(g[u], x.y, ay);
          az = fmaf(g[u], x.z, az);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
      }
      if (lane == 0) {
        float* out = dXa + ((a0 + i) * (int64_t)HW + p) * C;
        const float ic = 1.f / (float)C;
        atomicAdd(out, ax * ic);
        if (C > 1) atomicAdd(out + 1, ay * ic);
        if (C > 2) atomicAdd(out + 2, az * ic);
      }
    }
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
  int sm;                  // SMs of the device
  size_t patch_bytes;      // FP32 with the tensor-core seed: split patch rows of both image sets
  size_t stored_per_pair;  // elements of T: every layer's pre-activation
  size_t hw0sq;            // elements of the largest (stage-0) pair tensor
  size_t part_per_pair;    // elements of one partial-sum buffer (largest stage)
  size_t bytes;            // total workspace
  size_t self_bytes;
  SelfAdjGeom sg;
  int self_grid;
};

template <typename T>
BwdPlan<T> plan_backward(const NkGeom& g, int64_t npairs, int64_t na, int64_t nb, int sym, int sm) {
  BwdPlan<T> P = {};
  P.hw0sq = (size_t)g.Hs[0] * g.Ws[0] * g.Hs[0] * g.Ws[0];
  P.part_per_pair = (size_t)g.Hs[0] * g.Hs[0] * g.Ws[0];
  int layer = 0;
  for (int s = 0; s < g.n_stages; ++s)
    for (int k = 0; k < g.convs[s]; ++k, ++layer) {
      const size_t hw = (size_t)g.Hs[s] * g.Ws[s];
      P.stored_per_pair += hw * hw;
    }
  const size_t per_pair = (P.stored_per_pair + 2 * P.hw0sq + 2 * P.part_per_pair + 2) * sizeof(T);
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
  P.sm = sm;
  P.patch_bytes = (sizeof(T) == 4 && nk_seed_gemm_supported(g.Hs[0], g.Ws[0], g.C, g.filter))
                      ? nk_seed_patch_bytes(na + (sym ? 0 : nb), g.Hs[0], g.Ws[0])
                      : 0;
  P.bytes = per_pair * P.chunk + (nqa + nqb) * sizeof(T) + P.self_bytes + P.patch_bytes + 4096;
  return P;
}

// One streamed stencil pass (k_conv_fused) over the chunk's pair tensors at
// stage resolution A.H x A.W: two pairs per block at the 32 x 32 stage (four
// at the smaller ones, one at 64 x 64).
template <typename T, int MODE, int W, int NPB>
cudaError_t conv_launch(const FArgs<T>& A, cudaStream_t st) {
  const size_t smem = conv_smem_bytes<T, MODE, W, NPB>();
  const dim3 grid((unsigned)(2 * A.H - 1), (unsigned)std::min<int64_t>((A.np + NPB - 1) / NPB, 65535));
  cudaError_t e = cudaFuncSetAttribute(k_conv_fused<T, MODE, W, NPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_conv_fused<T, MODE, W, NPB><<<grid, 256, smem, st>>>(A);
  return cudaGetLastError();
}

// Stage widths 1 .. 64 (powers of two: the 2x2 pools halve 8 .. 64 pixel
// images); nk_block_backward refuses the others.
template <typename T, int MODE>
cudaError_t conv_pass(const FArgs<T>& A, cudaStream_t st) {
  switch (A.W) {
    case 1: return conv_launch<T, MODE, 1, 4>(A, st);
    case 2: return conv_launch<T, MODE, 2, 4>(A, st);
    case 4: return conv_launch<T, MODE, 4, 4>(A, st);
    case 8: return conv_launch<T, MODE, 8, 4>(A, st);
    case 16: return conv_launch<T, MODE, 16, 4>(A, st);
    case 32: return conv_launch<T, MODE, 32, 1>(A, st);
    case 64: return conv_launch<T, MODE, 64, 1>(A, st);
  }
  return cudaErrorNotSupported;
}

template <typename T>
cudaError_t run_backward(const NkGeom& g, double sw2, double sb2, const float* Xa, const double* qda,
                         const float* qsa, int64_t a0, int64_t a1, const float* Xb, const double* qdb,
                         const float* qsb, int64_t b0, int64_t b1, const T* dK, int64_t lddk, int sym, T* dXa, T* dXb,
                         double* dsw2, double* dsb2, void* ws, const BwdPlan<T>& P, uint32_t wait_limit,
                         cudaStream_t st, int64_t* launches, unsigned int* dstatus) {
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
  T* buf0 = reinterpret_cast<T*>(take(P.hw0sq * chunk * sizeof(T)));
  T* buf1 = reinterpret_cast<T*>(take(P.hw0sq * chunk * sizeof(T)));
  T* prow = reinterpret_cast<T*>(take(P.part_per_pair * chunk * sizeof(T)));
  T* pcol = reinterpret_cast<T*>(take(P.part_per_pair * chunk * sizeof(T)));
  T* useed = reinterpret_cast<T*>(take(chunk * sizeof(T)));
  T* gmean = reinterpret_cast<T*>(take(chunk * sizeof(T)));
  T* dqa = reinterpret_cast<T*>(take((size_t)na * g.nq * sizeof(T)));
  T* dqb = sym ? dqa : reinterpret_cast<T*>(take((size_t)nb * g.nq * sizeof(T)));
  double* sws = reinterpret_cast<double*>(take(P.self_bytes));
  cudaError_t e = cudaMemsetAsync(dqa, 0, (size_t)na * g.nq * sizeof(T), st);
  if (e == cudaSuccess && !sym) e = cudaMemsetAsync(dqb, 0, (size_t)nb * g.nq * sizeof(T), st);
  if (e != cudaSuccess) return e;
  // FP32: the first layer's pre-activation is the patch Gram on the tensor
  // cores (seed_gemm.cu); the patch rows of both image sets are split once
  const bool tc_seed = P.patch_bytes > 0;
  void* patch_a = nullptr;
  void* patch_b = nullptr;
  if (tc_seed) {
    const int64_t HW0 = (int64_t)g.Hs[0] * g.Ws[0];
    patch_a = take(nk_seed_patch_bytes(na, g.Hs[0], g.Ws[0]));
    patch_b = sym ? patch_a : take(nk_seed_patch_bytes(nb, g.Hs[0], g.Ws[0]));
    *launches += sym ? 1 : 2;
    e = nk_seed_patches(Xa + a0 * HW0 * g.C, na, g.Hs[0], g.Ws[0], g.C, patch_a, st);
    if (e == cudaSuccess && !sym) e = nk_seed_patches(Xb + b0 * HW0 * g.C, nb, g.Hs[0], g.Ws[0], g.C, patch_b, st);
    if (e != cudaSuccess) return e;
  }
  const T a_conv = (T)(sw2 / (double)(g.filter * g.filter));
  const bool relu = (g.act == NK_ACT_RELU);
  int last_conv_stage = 0;
  for (int s = 0; s < g.n_stages; ++s)
    if (g.convs[s] > 0) last_conv_stage = s;
  const double hwl = (double)g.Hs[last_conv_stage] * g.Ws[last_conv_stage];

  for (int64_t pair0 = 0; pair0 < npairs; pair0 += chunk) {
    const int64_t np = std::min<int64_t>(chunk, npairs - pair0);
    FArgs<T> A = {};
    A.np = np;
    A.pair0 = pair0;
    A.na = na;
    A.nb = nb;
    A.a0 = a0;
    A.b0 = b0;
    A.sym = sym;
    A.Xa = Xa;
    A.Xb = Xb;
    A.C = g.C;
    A.relu = relu;
    A.qda = qda;
    A.qdb = qdb;
    A.qsa = qsa;
    A.qsb = qsb;
    A.nq = g.nq;
    A.prow = prow;
    A.pcol = pcol;
    A.sb2 = sb2;
    A.inv_sw2 = 1.0 / sw2;
    A.dsw2 = dsw2;
    A.dsb2 = dsb2;
    T* Kst[NK_MAX_LAYERS];
    int lstage[NK_MAX_LAYERS];
    {
      size_t off = 0;
      int layer = 0;
      for (int s = 0; s < g.n_stages; ++s)
        for (int k = 0; k < g.convs[s]; ++k, ++layer) {
          Kst[layer] = stored + off * np;
          lstage[layer] = s;
          off += (size_t)g.Hs[s] * g.Ws[s] * g.Hs[s] * g.Ws[s];
        }
    }
    // ---- forward: store each layer's pre-activation; the map of the
    // previous layer is applied as the next pass loads it
    const T* pend = nullptr;  // tensor the next pass reads (after its map, if pend_layer >= 0)
    int pend_layer = -1;
    int layer = 0;
    for (int s = 0; s <= last_conv_stage; ++s) {
      A.H = g.Hs[s];
      A.W = g.Ws[s];
      if (s > 0) {
        T* pooled = (pend == buf0) ? buf1 : buf0;
        const int64_t HWo = (int64_t)A.H * A.W;
        FArgs<T> B = A;
        B.src = pend;
        B.out = pooled;
        B.relu = relu && pend_layer >= 0;
        B.qoff = pend_layer >= 0 ? g.layer_qoff[pend_layer] : 0;
        ++*launches;
        k_pool_map<T><<<grid_for(np * HWo * HWo), 256, 0, st>>>(B, A.H, A.W);
        pend = pooled;
        pend_layer = -1;
      }
      for (int k = 0; k < g.convs[s]; ++k, ++layer) {
        A.out = Kst[layer];
        A.a = a_conv;
        A.b = (T)sb2;
        ++*launches;
        if (layer == 0 && tc_seed) {
          if constexpr (sizeof(T) == 4)
            e = nk_launch_seed_gemm(patch_a, na, patch_b, nb, sym, pair0, np, g.Hs[0], g.Ws[0], g.C, sw2, sb2,
                                    Kst[0], P.sm, dstatus, wait_limit, st);
        } else if (layer == 0) {
          e = conv_pass<T, CIN_COV>(A, st);
        } else if (pend_layer >= 0) {
          A.src = pend;
          A.qoff = g.layer_qoff[pend_layer];
          e = conv_pass<T, CIN_MAP>(A, st);
        } else {
          A.src = pend;
          e = conv_pass<T, CIN_PLAIN>(A, st);
        }
        if (e != cudaSuccess) return e;
        pend = Kst[layer];
        pend_layer = layer;
      }
    }
    // readout value: the mean of the last layer's post-activation
    {
      FArgs<T> B = A;
      B.H = g.Hs[last_conv_stage];
      B.W = g.Ws[last_conv_stage];
      B.src = pend;
      B.qoff = g.layer_qoff[pend_layer];
      ++*launches;
      k_map_mean<T><<<(unsigned)np, 256, 0, st>>>(B, gmean);
    }
    // ---- reverse
    ++*launches;
    k_pair_seed<T><<<grid_for(np), 256, 0, st>>>(dK, lddk, gmean, na, nb, sym, pair0, np, sw2, hwl * hwl, useed,
                                                 dsw2, dsb2);
    const T* gcur = useed;  // gradient of the current layer's post-activation
    int gmode = G_CONST;
    for (int s = last_conv_stage; s >= 0; --s) {
      A.H = g.Hs[s];
      A.W = g.Ws[s];
      for (int k = g.convs[s] - 1; k >= 0; --k) {
        --layer;
        T* out = (gcur == buf0) ? buf1 : buf0;
        A.src = Kst[layer];
        A.qoff = g.layer_qoff[layer];
        A.gsrc = gcur;
        A.gmode = gmode;
        A.out = out;
        A.a = a_conv;
        A.b = (T)0;
        ++*launches;
        e = conv_pass<T, CIN_ADJ>(A, st);
        if (e != cudaSuccess) return e;
        if (relu) {
          ++*launches;
          k_qsum<T><<<grid_for(2 * np * (int64_t)A.H * A.W), 256, 0, st>>>(A, dqa, dqb);
        }
        gcur = out;
        gmode = G_TENSOR;
      }
      if (s > 0) {
        if (g.convs[s - 1] > 0) {
          gmode = G_POOLED;  // the previous stage's last layer reads it through the pool adjoint
        } else {
          // an empty stage: its input gradient is the pool adjoint itself
          T* out = (gcur == buf0) ? buf1 : buf0;
          const int64_t HWp = 4 * (int64_t)A.H * A.W;
          ++*launches;
          k_pool_adj<T><<<grid_for(np * HWp * HWp), 256, 0, st>>>(gcur, out, np, A.H, A.W);
          gcur = out;
          gmode = G_TENSOR;
        }
      }
    }
    // gcur: gradient of the input covariance K_0
    const int HW0 = g.Hs[0] * g.Ws[0];
    T* dXb_eff = sym ? dXa : dXb;
    // FP32, C <= 3, whole 256-column slabs: the staged float4 forms
    const bool staged = sizeof(T) == 4 && g.C <= 3 && HW0 % 256 == 0;
    const size_t xs_bytes = (size_t)HW0 * sizeof(float4);
    const unsigned pair_grid_y = (unsigned)std::min<int64_t>(np, 65535);
    if (dXa) {
      ++*launches;
      if constexpr (sizeof(T) == 4) {
        if (staged) {
          if (xs_bytes > 48 * 1024)
            cudaFuncSetAttribute(k_seed_adj_a4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs_bytes);
          k_seed_adj_a4<<<dim3((unsigned)(HW0 / 8 < 32 ? HW0 / 8 : 32), pair_grid_y), 256, xs_bytes, st>>>(
              gcur, Xb, np, HW0, g.C, na, nb, sym, pair0, a0, b0, dXa);
        }
      }
      if (!staged)
        k_seed_adj_a<T><<<grid_for((int64_t)np * HW0 * 32), 256, 0, st>>>(gcur, Xb, np, HW0, g.C, na, nb, sym,
                                                                          pair0, a0, b0, dXa);
    }
    if (dXb_eff) {
      ++*launches;
      if constexpr (sizeof(T) == 4) {
        if (staged) {
          if (xs_bytes > 48 * 1024)
            cudaFuncSetAttribute(k_seed_adj_b4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs_bytes);
          k_seed_adj_b4<<<dim3((unsigned)(HW0 / 256), pair_grid_y), 256, xs_bytes, st>>>(
              gcur, Xa, np, HW0, g.C, na, nb, sym, pair0, a0, b0, dXb_eff);
        }
      }
      if (!staged)
        k_seed_adj_b<T><<<grid_for((int64_t)np * HW0), 256, 0, st>>>(gcur, Xa, np, HW0, g.C, na, nb, sym, pair0,
                                                                     a0, b0, dXb_eff);
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
                               void* ws, int sm, uint32_t wait_limit, cudaStream_t st, int64_t* launches,
                               unsigned int* dstatus) {
  const int64_t na = a1 - a0, nb = b1 - b0;
  const int64_t npairs = sym ? na * (na + 1) / 2 : na * nb;
  if (fp64) {
    auto P = plan_backward<double>(g, npairs, na, nb, sym, sm);
    return run_backward<double>(g, sw2, sb2, Xa, qda, qsa, a0, a1, Xb, qdb, qsb, b0, b1, (const double*)dK, lddk,
                                sym, (double*)dXa, (double*)dXb, dsw2, dsb2, ws, P, wait_limit, st, launches,
                                dstatus);
  }
  auto P = plan_backward<float>(g, npairs, na, nb, sym, sm);
  return run_backward<float>(g, sw2, sb2, Xa, qda, qsa, a0, a1, Xb, qdb, qsb, b0, b1, (const float*)dK, lddk,
                             sym, (float*)dXa, (float*)dXb, dsw2, dsb2, ws, P, wait_limit, st, launches,
                             dstatus);
}
