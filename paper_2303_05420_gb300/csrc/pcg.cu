// nk_pcg_solve: Jacobi-preconditioned conjugate gradients for (K + lam I) A = Y
// with R right-hand sides run in lock-step (Section 2, "Iterative solvers":
// CG with a preconditioner; Appendix B.3: CG vectorised over tasks).
//
// The matvec is the only place K occurs (Section 2), and it is bandwidth
// bound: K (N x N float32, symmetric) is streamed once per iteration.  Each
// thread owns 4 consecutive columns i and walks rows j of a row split, using
// K[j][i] = K[i][j] so that every warp reads 512 contiguous bytes of a row;
// the R values P[j][:] are a warp-broadcast load.  FP32 products are summed in
// FP32 over chunks of at most 256 rows and the chunk sums are combined in FP64
// (row-split partials reduced in FP64 by the next kernel).  CG scalars
// (alpha, beta, r.z, p.Ap) are FP64.  NK_PREC_MIXED wraps FP32-matvec inner
// solves in an FP64 iterative-refinement loop whose true residual is formed
// in double-FP32 arithmetic (k_matvec_df: exact FP32 products and two-float
// TwoSum accumulation, about 2^-48 relative per step) on the FP32 units;
// PLAIN_FP64 keeps native FP64 products throughout.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "nk_common.cuh"

namespace {

// per-column CG scalars, sc[slot * R + column]; SC_TOL holds tol^2 of the
// running solve (read on the device, so a captured iteration serves any tol)
enum { SC_RZ = 0, SC_RZN, SC_PQ, SC_RR, SC_YY, SC_ACT, SC_ALPHA, SC_BETA, SC_ITER, SC_TOL, SC_N };

// FP32 form: chunk sums of at most NK_MV_CHUNK rows are added, in FP64, to
// per-thread slots in shared memory (mv_sh[(c * RB + r) * 128 + tid]); keeping
// them out of registers lets four blocks share an SM, each thread holding
// U float4 loads of K in flight.
#define NK_MV_CHUNK 256
#define NK_MV_THREADS 128

// MULTI: more than 16 right-hand sides, one group of 16 per blockIdx.z;
// otherwise all R (<= RB) columns in one group.
template <int RB, bool F64, bool VEC, bool MULTI = false>
__global__ void __launch_bounds__(NK_MV_THREADS, (F64 && RB > 8) ? 2 : 4)
k_matvec(const float* __restrict__ K, int64_t ldk, int64_t N, const void* __restrict__ Pin, int R,
         int rows_per_split, double* __restrict__ Qpart) {
  const int rc0 = MULTI ? (int)blockIdx.z * 16 : 0;
  const int rcnt = MULTI ? min(16, R - rc0) : R;
  using T = typename std::conditional<F64, double, float>::type;
  constexpr int U = F64 ? 2 : (RB > 10 ? 4 : 8);  // rows per unrolled step (registers)
  extern __shared__ double mv_sh[];
  const int tid = threadIdx.x;
  const int64_t i0 = ((int64_t)blockIdx.x * NK_MV_THREADS + tid) * 4;
  const int64_t js = (int64_t)blockIdx.y * rows_per_split;
  const int64_t je = std::min<int64_t>(N, js + rows_per_split);
  const T* P = reinterpret_cast<const T*>(Pin);
  T acc[4][RB];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      acc[c][r] = 0;
      if constexpr (!F64) mv_sh[(c * RB + r) * NK_MV_THREADS + tid] = 0.0;
    }
  const bool full = (i0 + 3 < N);
  int chunk = 0;
  int64_t j = js;
  for (; j + U <= je; j += U) {
    float k[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float* row = K + (j + u) * ldk + i0;
      if (VEC && full) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(row));
        k[u][0] = v.x;
        k[u][1] = v.y;
        k[u][2] = v.z;
        k[u][3] = v.w;
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) k[u][c] = (i0 + c < N) ? __ldg(row + c) : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const T* pr = P + (j + u) * R + rc0;
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        if (r < rcnt) {
          const T p = __ldg(pr + r);
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[c][r] = fma((T)k[u][c], p, acc[c][r]);
        }
      }
    }
    if constexpr (!F64) {
      chunk += U;
      if (chunk >= NK_MV_CHUNK) {
        chunk = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int r = 0; r < RB; ++r) {
            mv_sh[(c * RB + r) * NK_MV_THREADS + tid] += (double)acc[c][r];
            acc[c][r] = 0;
          }
      }
    }
  }
  for (; j < je; ++j) {  // fewer than U rows left (chunk stays below its bound)
    float k[4];
    const float* row = K + j * ldk + i0;
#pragma unroll
    for (int c = 0; c < 4; ++c) k[c] = (i0 + c < N) ? __ldg(row + c) : 0.f;
    const T* pr = P + j * R + rc0;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      if (r < rcnt) {
        const T p = __ldg(pr + r);
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c][r] = fma((T)k[c], p, acc[c][r]);
      }
    }
  }
  double* out = Qpart + (int64_t)blockIdx.y * N * R;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (i0 + c < N) {
#pragma unroll
      for (int r = 0; r < RB; ++r)
        if (r < rcnt) {
          double v = (double)acc[c][r];
          if constexpr (!F64) v += mv_sh[(c * RB + r) * NK_MV_THREADS + tid];
          out[(i0 + c) * R + rc0 + r] = v;
        }
    }
  }
}

template <int RB, bool F64>
constexpr size_t mv_smem() {
  return F64 ? 0 : (size_t)4 * RB * NK_MV_THREADS * sizeof(double);
}

// K @ X for the true residual, with X = Xh + Xl split into two FP32 arrays
// (Xh = fl32(X), Xl = fl32(X - Xh)).  Each product k * xh is taken exactly
// as a pair (p, e) (p = fl32(k xh), e = fma(k, xh, -p)); p enters a
// double-FP32 sum (s, c) through Knuth's TwoSum, and e + k * xl go to the low
// part.  Every step rounds at about 2^-48 relative to the running sum, close
// to FP64, on the FP32 units (64 times the FP64 rate on this part).
template <int RB>
__global__ void __launch_bounds__(NK_MV_THREADS, RB > 8 ? 3 : 4)
k_matvec_df(const float* __restrict__ K, int64_t ldk, int64_t N, const float* __restrict__ Xh,
            const float* __restrict__ Xl, int R, int rows_per_split,
            double* __restrict__ Qpart) {
  constexpr int CPT = 2;  // columns per thread
  const int rc0 = blockIdx.z * 16, rcnt = min(16, R - rc0);  // column group
  const int tid = threadIdx.x;
  const int64_t i0 = ((int64_t)blockIdx.x * NK_MV_THREADS + tid) * CPT;
  const int64_t js = (int64_t)blockIdx.y * rows_per_split;
  const int64_t je = std::min<int64_t>(N, js + rows_per_split);
  float sh[CPT][RB], sl[CPT][RB];
#pragma unroll
  for (int c = 0; c < CPT; ++c)
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      sh[c][r] = 0.f;
      sl[c][r] = 0.f;
    }
  const bool vec = (i0 + CPT - 1 < N) && (ldk % 2 == 0) && ((reinterpret_cast<uintptr_t>(K) & 7) == 0);
  for (int64_t j = js; j < je; ++j) {
    float k[CPT];
    const float* row = K + j * ldk + i0;
    if (vec) {
      const float2 v = __ldg(reinterpret_cast<const float2*>(row));
      k[0] = v.x;
      k[1] = v.y;
    } else {
#pragma unroll
      for (int c = 0; c < CPT; ++c) k[c] = (i0 + c < N) ? __ldg(row + c) : 0.f;
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      if (r < rcnt) {
        const float xh = __ldg(Xh + j * R + rc0 + r);
        const float xl = __ldg(Xl + j * R + rc0 + r);
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          // explicit roundings: no contraction of p into the sum
          const float p = __fmul_rn(k[c], xh);
          const float e = fmaf(k[c], xh, -p);
          const float t = __fadd_rn(sh[c][r], p);  // TwoSum(sh, p)
          const float bp = __fsub_rn(t, sh[c][r]);
          const float err = __fadd_rn(__fsub_rn(sh[c][r], __fsub_rn(t, bp)), __fsub_rn(p, bp));
          sh[c][r] = t;
          sl[c][r] = __fadd_rn(sl[c][r], __fadd_rn(err, fmaf(k[c], xl, e)));
        }
      }
    }
  }
  double* out = Qpart + (int64_t)blockIdx.y * N * R;
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    if (i0 + c < N) {
#pragma unroll
      for (int r = 0; r < RB; ++r)
        if (r < rcnt) out[(i0 + c) * R + rc0 + r] = (double)sh[c][r] + (double)sl[c][r];
    }
  }
}

// Xh = fl32(X), Xl = fl32(X - Xh)
__global__ void k_split_f32(int64_t n, const double* __restrict__ X, float* __restrict__ Xh,
                            float* __restrict__ Xl) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double x = X[e];
    const float h = (float)x;
    Xh[e] = h;
    Xl[e] = (float)(x - (double)h);
  }
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// True in every thread of the block that arrives last in this launch
// (after all other blocks' global writes and atomics are visible); that block
// resets the counter for the next launch.
__device__ __forceinline__ bool last_block(int* done) {
  __shared__ int is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const int total = (int)(gridDim.x * gridDim.y);
    const int old = atomicAdd(done, 1);
    is_last = (old == total - 1);
    if (is_last) atomicExch(done, 0);
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last != 0;
}

// alpha = r.z / p.Ap per running column; clears the sums of the update
__device__ __forceinline__ void finish_alpha(double* sc, int R) {
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const double act = __ldcg(sc + SC_ACT * R + r);
    const double pq = __ldcg(sc + SC_PQ * R + r);
    sc[SC_ALPHA * R + r] = (act != 0.0 && pq != 0.0) ? __ldcg(sc + SC_RZ * R + r) / pq : 0.0;
    sc[SC_RZN * R + r] = 0.0;
    sc[SC_RR * R + r] = 0.0;
  }
}

// Q = sum_s Qpart[s] + lam * P ; sc[PQ][r] += P . Q  (one column r per
// blockIdx.y); with `done`, the last block also forms alpha.
__global__ void k_reduce_dot(const double* __restrict__ Qpart, int S, int64_t N, int R,
                             const double* __restrict__ P, double lam, double* __restrict__ Q,
                             double* __restrict__ sc, int dot_slot, int* done) {
  __shared__ double sh[32];
  const int r = blockIdx.y;
  double part = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    // the S partial loads are independent: keep eight in flight
    const double* src = Qpart + i * R + r;
    const int64_t stride = N * (int64_t)R;
    double q0 = 0.0, q1 = 0.0;
    int s = 0;
    for (; s + 8 <= S; s += 8) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = src[(int64_t)(s + u) * stride];
      q0 += (v[0] + v[1]) + (v[2] + v[3]);
      q1 += (v[4] + v[5]) + (v[6] + v[7]);
    }
    for (; s < S; ++s) q0 += src[(int64_t)s * stride];
    double q = q0 + q1;
    const double p = P[i * R + r];
    q += lam * p;
    Q[i * R + r] = q;
    part += p * q;
  }
  if (dot_slot >= 0) {
    const double s = block_sum(part, sh);
    if (threadIdx.x == 0) atomicAdd(sc + dot_slot * R + r, s);
  }
  if (done && last_block(done)) finish_alpha(sc, R);
}

// Initialise a CG run on right-hand side B (x = 0): r = B, z = M^{-1} r,
// p = z, accumulate r.z and B.B.
__global__ void k_init(const double* __restrict__ B, const double* __restrict__ minv, int64_t N,
                       int R, double* __restrict__ X, double* __restrict__ Rr,
                       double* __restrict__ Z, double* __restrict__ P, float* __restrict__ Pf,
                       double* __restrict__ sc) {
  __shared__ double sh[32];
  const int r = blockIdx.y;
  double rz = 0.0, yy = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i * R + r;
    const double b = B[e];
    const double z = minv[i] * b;
    X[e] = 0.0;
    Rr[e] = b;
    Z[e] = z;
    P[e] = z;
    Pf[e] = (float)z;
    rz += b * z;
    yy += b * b;
  }
  double s = block_sum(rz, sh);
  if (threadIdx.x == 0) atomicAdd(sc + SC_RZ * R + r, s);
  s = block_sum(yy, sh);
  if (threadIdx.x == 0) atomicAdd(sc + SC_YY * R + r, s);
}

// beta, activity and iteration counts for every column; *flag = number of
// columns still running; clears p.Ap for the next iteration.
__device__ __forceinline__ void finish_beta(double* sc, int R, int* flag) {
  int running = 0;
  for (int r0 = 0; r0 < R; r0 += blockDim.x) {
    const int r = r0 + threadIdx.x;
    int act_now = 0;
    if (r < R) {
      const double act = __ldcg(sc + SC_ACT * R + r);
      if (act != 0.0) {
        const double rzn = __ldcg(sc + SC_RZN * R + r);
        const double rz = __ldcg(sc + SC_RZ * R + r);
        sc[SC_BETA * R + r] = (rz != 0.0) ? rzn / rz : 0.0;
        sc[SC_RZ * R + r] = rzn;
        sc[SC_ITER * R + r] += 1.0;
        const bool still = __ldcg(sc + SC_RR * R + r) > sc[SC_TOL * R + r] * sc[SC_YY * R + r];
        sc[SC_ACT * R + r] = still ? 1.0 : 0.0;
        act_now = still ? 1 : 0;
      } else {
        sc[SC_BETA * R + r] = 0.0;
      }
      sc[SC_PQ * R + r] = 0.0;
    }
    running += __syncthreads_count(act_now);
  }
  if (threadIdx.x == 0) *flag = running;
}

// x += alpha p, r -= alpha q, z = M^{-1} r, r.z and r.r; the last block forms
// beta and the activity flags.
// JAC: the Jacobi preconditioner is applied here (z, r.z, and beta in the
// last block); otherwise the preconditioner kernels that follow do it.
template <bool JAC>
__global__ void k_update(const double* __restrict__ minv, int64_t N, int R, double* __restrict__ X,
                         double* __restrict__ Rr, double* __restrict__ Z,
                         const double* __restrict__ P, const double* __restrict__ Q,
                         double* __restrict__ sc, int* done, int* flag) {
  __shared__ double sh[32];
  const int r = blockIdx.y;
  const double alpha = sc[SC_ALPHA * R + r];
  double rz = 0.0, rr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i * R + r;
    X[e] += alpha * P[e];
    const double rn = Rr[e] - alpha * Q[e];
    Rr[e] = rn;
    if constexpr (JAC) {
      const double z = minv[i] * rn;
      Z[e] = z;
      rz += rn * z;
    }
    rr += rn * rn;
  }
  double s;
  if constexpr (JAC) {
    s = block_sum(rz, sh);
    if (threadIdx.x == 0) atomicAdd(sc + SC_RZN * R + r, s);
  }
  s = block_sum(rr, sh);
  if (threadIdx.x == 0) atomicAdd(sc + SC_RR * R + r, s);
  if constexpr (JAC) {
    if (last_block(done)) finish_beta(sc, R, flag);
  }
}

// Initialise a CG run for a preconditioner applied by separate kernels:
// x = 0, r = B, B.B (z, p and r.z follow from the preconditioner kernels).
__global__ void k_init_pc(const double* __restrict__ B, int64_t N, int R, double* __restrict__ X,
                          double* __restrict__ Rr, double* __restrict__ sc) {
  __shared__ double sh[32];
  const int r = blockIdx.y;
  double yy = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i * R + r;
    const double b = B[e];
    X[e] = 0.0;
    Rr[e] = b;
    yy += b * b;
  }
  const double s = block_sum(yy, sh);
  if (threadIdx.x == 0) atomicAdd(sc + SC_YY * R + r, s);
}

__global__ void k_direction(int64_t N, int R, const double* __restrict__ Z, double* __restrict__ P,
                            float* __restrict__ Pf, const double* __restrict__ sc) {
  const int r = blockIdx.y;
  if (sc[SC_ACT * R + r] == 0.0) return;
  const double beta = sc[SC_BETA * R + r];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i * R + r;
    const double p = Z[e] + beta * P[e];
    P[e] = p;
    Pf[e] = (float)p;
  }
}

__global__ void k_minv(const float* __restrict__ K, int64_t ldk, int64_t N, double lam, int jacobi,
                       double* __restrict__ minv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = jacobi ? (double)K[i * ldk + i] + lam : 1.0;
    minv[i] = (d != 0.0) ? 1.0 / d : 1.0;
  }
}

// out = B - Q, per-column ||out||^2 into sc[SC_RR] (used for true residuals)
__global__ void k_resid(const double* __restrict__ B, const double* __restrict__ Q, int64_t N, int R,
                        double* __restrict__ out, double* __restrict__ sc) {
  __shared__ double sh[32];
  const int r = blockIdx.y;
  double rr = 0.0, yy = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i * R + r;
    const double v = B[e] - Q[e];
    out[e] = v;
    rr += v * v;
    yy += B[e] * B[e];
  }
  double s = block_sum(rr, sh);
  if (threadIdx.x == 0) atomicAdd(sc + SC_RR * R + r, s);
  s = block_sum(yy, sh);
  if (threadIdx.x == 0) atomicAdd(sc + SC_YY * R + r, s);
}

// tr(K) in FP64 (one block)
__global__ void k_trace(const float* __restrict__ K, int64_t ldk, int64_t N, double* out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) acc += (double)K[i * ldk + i];
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_add(int64_t n, double* __restrict__ X, const double* __restrict__ D) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    X[e] += D[e];
}

__global__ void k_zero(double* p, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    p[e] = 0.0;
}

__global__ void k_set_active(double* sc, int R, double tol2) {
  const int r = threadIdx.x;
  if (r < R) {
    sc[SC_ACT * R + r] = 1.0;
    sc[SC_TOL * R + r] = tol2;
  }
}

// ---------------------------------------------------------------------------
// Partial pivoted Cholesky preconditioner (Section 2: the paper's own, after
// Wang et al. 2019).  K ~ L^T L from `rank` greedy pivots (the largest
// remaining diagonal d of the Schur complement, lowest index on ties; stop
// once it falls to 1e-12 of K's largest diagonal), M = L^T L + lam I applied
// by the Woodbury identity M^{-1} v = (v - L^T G^{-1} L v) / lam with
// G = lam I + L L^T (rank x rank, FP64).  G^{-1} is formed once per solve
// as W^T W with W = C^{-1}, C the Cholesky factor of G, so that it is
// symmetric positive definite as computed.
// ---------------------------------------------------------------------------
struct PcState {
  int stop;      // the rank is exhausted
  int rank_eff;  // pivots taken
  int piv;       // current pivot
  int pad;
  double invs;   // 1 / sqrt(d[piv])
  double floor;  // 1e-12 * max diag K
};

// argmax of d (lowest index on ties) by one block; sets the next pivot or
// marks the rank exhausted.
__device__ void pc_select(const double* __restrict__ d, int64_t N, PcState* st) {
  __shared__ double sv[32];
  __shared__ int64_t si[32];
  double best = -1.0;
  int64_t bi = 0;
  for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
    const double v = __ldcg(d + j);
    if (v > best) {
      best = v;
      bi = j;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    sv[threadIdx.x >> 5] = best;
    si[threadIdx.x >> 5] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    best = sv[0];
    bi = si[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (sv[w] > best || (sv[w] == best && si[w] < bi)) {
        best = sv[w];
        bi = si[w];
      }
    if (!(best > st->floor)) {
      st->stop = 1;
    } else {
      st->piv = (int)bi;
      st->invs = 1.0 / sqrt(best);
    }
  }
}

__global__ void k_pc_diag(const float* __restrict__ K, int64_t ldk, int64_t N, double* __restrict__ d,
                          PcState* st) {
  __shared__ double sh[32];
  double mx = 0.0;
  for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
    const double v = (double)K[j * ldk + j];
    d[j] = v;
    mx = fmax(mx, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
    st->stop = 0;
    st->rank_eff = 0;
    st->floor = 1e-12 * m;
  }
  __syncthreads();
  pc_select(d, N, st);
}

// row k of L: L[k][j] = (K[i][j] - sum_{m<k} L[m][i] L[m][j]) / sqrt(d[i]);
// d[j] -= L[k][j]^2.  Rows past the exhausted rank are zero.
__global__ void k_pc_row(const float* __restrict__ K, int64_t ldk, int64_t N, double* __restrict__ L,
                         double* __restrict__ d, int k, PcState* st, int* done) {
  const bool stop = st->stop != 0;
  const int i = st->piv;
  const double invs = st->invs;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (!stop) {
      v = (double)K[(int64_t)i * ldk + j];
      for (int m = 0; m < k; ++m) v -= L[(int64_t)m * N + i] * L[(int64_t)m * N + j];
      v *= invs;
      d[j] -= v * v;
    }
    L[(int64_t)k * N + j] = v;
  }
  // the last block picks the next pivot from the updated diagonal
  if (last_block(done) && !stop) {
    if (threadIdx.x == 0) st->rank_eff = k + 1;
    pc_select(d, N, st);
  }
}

// G = lam I + L L^T, lower triangle (one block per (a, b), a >= b)
__global__ void k_pc_gram(const double* __restrict__ L, int r, int64_t N, double lam, double* __restrict__ G) {
  __shared__ double sh[32];
  const int a = blockIdx.x, b = blockIdx.y;
  if (b > a) return;
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < N; j += blockDim.x) s += L[(int64_t)a * N + j] * L[(int64_t)b * N + j];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    if (a == b) s += lam;
    G[a * r + b] = s;
    G[b * r + a] = s;
  }
}

// In place: G -> C (lower Cholesky factor), then Ginv = W^T W with W = C^{-1}
// (one block; rank is small).  Work: W in `work` [r][r].
__global__ void k_pc_factor(double* __restrict__ G, int r, double* __restrict__ W, double* __restrict__ Ginv) {
  for (int k = 0; k < r; ++k) {
    if (threadIdx.x == 0) G[k * r + k] = sqrt(fmax(G[k * r + k], 1e-300));
    __syncthreads();
    const double ckk = G[k * r + k];
    for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) G[i * r + k] /= ckk;
    __syncthreads();
    for (int e = threadIdx.x; e < (r - k - 1) * (r - k - 1); e += blockDim.x) {
      const int i = k + 1 + e / (r - k - 1), j = k + 1 + e % (r - k - 1);
      if (j <= i) G[i * r + j] -= G[i * r + k] * G[j * r + k];
    }
    __syncthreads();
  }
  // W = C^{-1}: column c by forward substitution (one thread per column)
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    for (int i = 0; i < r; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int m = c; m < i; ++m) v -= G[i * r + m] * W[m * r + c];
      W[i * r + c] = (i < c) ? 0.0 : v / G[i * r + i];
    }
  }
  __syncthreads();
  // Ginv[a][b] = sum_m W[m][a] W[m][b]
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int a = e / r, b = e % r;
    double s = 0.0;
    for (int m = (a > b ? a : b); m < r; ++m) s += W[m * r + a] * W[m * r + b];
    Ginv[e] = s;
  }
}

// T[m][col] = sum_j L[m][j] V[j][col] for one m per blockIdx.x and up to 16
// columns per blockIdx.y.
__global__ void k_pc_t(const double* __restrict__ L, int r, int64_t N, const double* __restrict__ V, int R,
                       double* __restrict__ T) {
  __shared__ double sh[32];
  const int m = blockIdx.x;
  const int c0 = blockIdx.y * 16, cn = min(16, R - c0);
  double acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = 0.0;
  for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
    const double l = L[(int64_t)m * N + j];
    const double* v = V + j * R + c0;
#pragma unroll
    for (int c = 0; c < 16; ++c)
      if (c < cn) acc[c] += l * v[c];
  }
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    if (c < cn) {
      const double s = block_sum(acc[c], sh);
      if (threadIdx.x == 0) T[m * R + c0 + c] = s;
    }
  }
}

// U = Ginv T, one thread per entry.
__global__ void k_pc_u(const double* __restrict__ Ginv, int r, const double* __restrict__ T, int R,
                       double* __restrict__ U) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r * R) return;
  const int a = e / R, col = e - a * R;
  double s = 0.0;
  for (int b = 0; b < r; ++b) s += Ginv[a * r + b] * T[b * R + col];
  U[e] = s;
}

// Z = (V - L^T U) / lam and r.z per column.  init: r.z into SC_RZ and P = Z
// (the first direction); otherwise r.z into SC_RZN and the last block forms
// beta and the activity flags.  A block covers 32 rows j and up to 16
// columns (blockIdx.y); its 8 warps split the sum over m (m = warp, warp + 8,
// ...) and warp 0 adds the 8 partial sums, so no thread walks all `rank` terms.
__global__ void __launch_bounds__(256) k_pc_z(const double* __restrict__ L, int r, int64_t N,
                                              const double* __restrict__ V, int R, const double* __restrict__ U,
                                              double lam, double* __restrict__ Z, double* __restrict__ P,
                                              float* __restrict__ Pf, double* __restrict__ sc, int init, int* done,
                                              int* flag) {
  __shared__ double part[8][16][32];
  const int jj = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * 32 + jj;
  const int c0 = blockIdx.y * 16, cn = min(16, R - c0);
  double s[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) s[c] = 0.0;
  if (j < N) {
    for (int m = g; m < r; m += 8) {
      const double l = L[(int64_t)m * N + j];
      const double* u = U + m * R + c0;
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < cn) s[c] += l * u[c];
    }
  }
#pragma unroll
  for (int c = 0; c < 16; ++c) part[g][c][jj] = s[c];
  __syncthreads();
  if (g == 0) {
    const double il = 1.0 / lam;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      if (c >= cn) break;
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < 8; ++w) t += part[w][c][jj];
      double rz = 0.0;
      if (j < N) {
        const int64_t e = j * R + c0 + c;
        const double v = V[e];
        const double z = (v - t) * il;
        Z[e] = z;
        if (init) {
          P[e] = z;
          Pf[e] = (float)z;
        }
        rz = v * z;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rz += __shfl_xor_sync(0xffffffffu, rz, o);
      if (jj == 0) atomicAdd(sc + (init ? SC_RZ : SC_RZN) * R + c0 + c, rz);
    }
  }
  if (!init && last_block(done)) finish_beta(sc, R, flag);
}

struct Pcg {
  int64_t N;
  int R;
  const float* K;
  int64_t ldk;
  double lam;
  int S;             // row splits of the matvec
  int rows_per_split;
  int sm;
  cudaStream_t st;
  double *Rr, *Z, *P, *Q, *Qpart, *minv, *sc, *B2;
  float* Pf;
  float *Xh, *Xl;    // double-FP32 split of the iterate (true residuals)
  int* flag;         // device: active columns after the last iteration
  int* done;         // device: block arrival counters [4] (reset by the last block)
  int64_t* nlaunch;  // handle launch counter
  // pivoted Cholesky preconditioner (pc_rank > 0; else Jacobi / none)
  int pc_rank;
  double *L, *Ginv, *T, *U;
};


template <bool F64>
cudaError_t matvec(const Pcg& c, const void* Pin) {
  const bool vec = (c.ldk % 4 == 0) && ((reinterpret_cast<uintptr_t>(c.K) & 15) == 0);
  const int64_t colthreads = (c.N + 3) / 4;
  dim3 grid((unsigned)((colthreads + NK_MV_THREADS - 1) / NK_MV_THREADS), (unsigned)c.S);
  grid.z = (unsigned)((c.R + 15) / 16);  // all column groups in one launch
  if (c.R > 16) {
    ++*c.nlaunch;
    if (vec)
      k_matvec<16, F64, true, true><<<grid, NK_MV_THREADS, mv_smem<16, F64>(), c.st>>>(
          c.K, c.ldk, c.N, Pin, c.R, c.rows_per_split, c.Qpart);
    else
      k_matvec<16, F64, false, true><<<grid, NK_MV_THREADS, mv_smem<16, F64>(), c.st>>>(
          c.K, c.ldk, c.N, Pin, c.R, c.rows_per_split, c.Qpart);
    return cudaGetLastError();
  }
  const int rmax = c.R;
#define NK_MV(RB)                                                                                  \
  if (rmax <= RB) {                                                                                \
    ++*c.nlaunch;                                                                                  \
    if (vec)                                                                                       \
      k_matvec<RB, F64, true><<<grid, NK_MV_THREADS, mv_smem<RB, F64>(), c.st>>>(                  \
          c.K, c.ldk, c.N, Pin, c.R, c.rows_per_split, c.Qpart);                                   \
    else                                                                                           \
      k_matvec<RB, F64, false><<<grid, NK_MV_THREADS, mv_smem<RB, F64>(), c.st>>>(                 \
          c.K, c.ldk, c.N, Pin, c.R, c.rows_per_split, c.Qpart);                                   \
    return cudaGetLastError();                                                                     \
  }
  NK_MV(1) NK_MV(2) NK_MV(4) NK_MV(8) NK_MV(10) NK_MV(16)
#undef NK_MV
  return cudaGetLastError();
}

// Opt in to the dynamic shared memory of the FP32 matvec forms (above 48 KB
// for 16 right-hand sides); returns the resident blocks per SM of the form
// that R columns use.
int matvec_prepare(int R) {
  const int rcnt = std::min(R, 16);
  int occ = 0;
#define NK_MV_ATTR(RB)                                                                              \
  cudaFuncSetAttribute(k_matvec<RB, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                       (int)mv_smem<RB, false>());                                                  \
  cudaFuncSetAttribute(k_matvec<RB, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                       (int)mv_smem<RB, false>());                                                  \
  if (occ == 0 && rcnt <= RB)                                                                       \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_matvec<RB, false, true>, NK_MV_THREADS,   \
                                                  mv_smem<RB, false>());
  NK_MV_ATTR(1) NK_MV_ATTR(2) NK_MV_ATTR(4) NK_MV_ATTR(8) NK_MV_ATTR(10) NK_MV_ATTR(16)
#undef NK_MV_ATTR
  cudaFuncSetAttribute(k_matvec<16, false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)mv_smem<16, false>());
  cudaFuncSetAttribute(k_matvec<16, false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)mv_smem<16, false>());
  (void)cudaGetLastError();
  return std::max(occ, 1);
}

// Row splits S of the matvec: two to eight waves of blocks, the number of
// blocks chosen so that the last wave is nearly full; at least 32 rows per
// split, and no more splits than keep the FP64 partial sums (S N R words)
// within a quarter of K's bytes unless that would leave the GPU under one
// wave (small systems: latency, not bytes, is what counts).
int choose_splits(int64_t N, int R, int sm, int occ) {
  const int64_t colblocks = ((N + 3) / 4 + NK_MV_THREADS - 1) / NK_MV_THREADS;
  const int64_t groups = (R + 15) / 16;
  const int64_t cap = (int64_t)sm * occ;  // resident blocks
  const int64_t per_split = colblocks * groups;
  const int64_t s_rows = std::max<int64_t>(1, std::min<int64_t>(512, N / 32));
  const int64_t s_lo0 = std::max<int64_t>(1, (2 * cap) / per_split);
  const int64_t s_hi0 = std::max<int64_t>(s_lo0, (8 * cap) / per_split);
  const int64_t s_bytes = std::max<int64_t>(1, N / std::max(4 * R, 32));
  const int64_t s_max = std::min<int64_t>(s_rows, std::max<int64_t>(s_bytes, s_lo0));
  const int64_t s_lo = std::min(s_lo0, s_max), s_hi = std::min(s_hi0, s_max);
  int64_t best = s_lo;
  double best_eff = -1.0;
  for (int64_t S = s_lo; S <= s_hi; ++S) {
    const double waves = (double)(per_split * S) / (double)cap;
    const double eff = waves / std::ceil(waves);
    if (eff > best_eff + 1e-3) {
      best_eff = eff;
      best = S;
    }
  }
  return (int)best;
}

inline dim3 vgrid(const Pcg& c) {
  int64_t b = (c.N + 255) / 256;
  if (b > 4 * (int64_t)c.sm) b = 4 * (int64_t)c.sm;
  return dim3((unsigned)std::max<int64_t>(1, b), (unsigned)c.R);
}

// z = M^{-1} r for the pivoted Cholesky preconditioner, r.z, and (init) the
// first direction or (iteration) beta.
void pc_apply(const Pcg& c, int init) {
  c.nlaunch[0] += 3;
  k_pc_t<<<dim3((unsigned)c.pc_rank, (unsigned)((c.R + 15) / 16)), 256, 0, c.st>>>(c.L, c.pc_rank, c.N, c.Rr,
                                                                                c.R, c.T);
  k_pc_u<<<(unsigned)((c.pc_rank * c.R + 127) / 128), 128, 0, c.st>>>(c.Ginv, c.pc_rank, c.T, c.R, c.U);
  k_pc_z<<<dim3((unsigned)((c.N + 31) / 32), (unsigned)((c.R + 15) / 16)), 256, 0, c.st>>>(
      c.L, c.pc_rank, c.N, c.Rr, c.R, c.U, c.lam, c.Z, c.P, c.Pf, c.sc, init, c.done + 3, c.flag);
}

// Q = (K + lam I) Xc with FP64 products and sums (exact_fp64) or with the
// double-FP32 products and sums of k_matvec_df.
cudaError_t apply_accurate(const Pcg& c, const double* Xc, bool exact_fp64) {
  if (exact_fp64) {
    cudaError_t e = matvec<true>(c, Xc);
    if (e != cudaSuccess) return e;
  } else {
    const int64_t NR = c.N * (int64_t)c.R;
    ++*c.nlaunch;
    k_split_f32<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((NR + 255) / 256, 4 * (int64_t)c.sm)), 256,
                  0, c.st>>>(NR, Xc, c.Xh, c.Xl);
    const int64_t colthreads = (c.N + 1) / 2;  // two columns per thread
    dim3 grid((unsigned)((colthreads + NK_MV_THREADS - 1) / NK_MV_THREADS), (unsigned)c.S);
    grid.z = (unsigned)((c.R + 15) / 16);  // all column groups in one launch
    const int rmax = std::min(16, c.R);
    ++*c.nlaunch;
    if (rmax <= 4)
      k_matvec_df<4><<<grid, NK_MV_THREADS, 0, c.st>>>(c.K, c.ldk, c.N, c.Xh, c.Xl, c.R, c.rows_per_split,
                                                       c.Qpart);
    else if (rmax <= 10)
      k_matvec_df<10><<<grid, NK_MV_THREADS, 0, c.st>>>(c.K, c.ldk, c.N, c.Xh, c.Xl, c.R, c.rows_per_split,
                                                        c.Qpart);
    else
      k_matvec_df<16><<<grid, NK_MV_THREADS, 0, c.st>>>(c.K, c.ldk, c.N, c.Xh, c.Xl, c.R, c.rows_per_split,
                                                        c.Qpart);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  ++*c.nlaunch;
  k_reduce_dot<<<vgrid(c), 256, 0, c.st>>>(c.Qpart, c.S, c.N, c.R, Xc, c.lam, c.Q, c.sc, -1, nullptr);
  return cudaGetLastError();
}

// True residual out = B - (K + lam I) X into sc[RR], sc[YY] (the CG state
// in sc is overwritten).
cudaError_t true_residual(const Pcg& c, const double* B, const double* Xc, double* out, bool exact_fp64) {
  ++*c.nlaunch;
  k_zero<<<1, 256, 0, c.st>>>(c.sc, (int64_t)SC_N * c.R);
  cudaError_t e = apply_accurate(c, Xc, exact_fp64);
  if (e != cudaSuccess) return e;
  ++*c.nlaunch;
  k_resid<<<vgrid(c), 256, 0, c.st>>>(B, c.Q, c.N, c.R, out, c.sc);
  return cudaGetLastError();
}

// One CG iteration for every active column (Section 2, "Iterative solvers").
template <bool F64>
cudaError_t cg_iteration(const Pcg& c, double* Xc) {
  cudaError_t e = F64 ? matvec<true>(c, c.P) : matvec<false>(c, c.Pf);
  if (e != cudaSuccess) return e;
  c.nlaunch[0] += 3;
  k_reduce_dot<<<vgrid(c), 256, 0, c.st>>>(c.Qpart, c.S, c.N, c.R, c.P, c.lam, c.Q, c.sc, SC_PQ, c.done);
  if (c.pc_rank > 0) {
    k_update<false><<<vgrid(c), 256, 0, c.st>>>(c.minv, c.N, c.R, Xc, c.Rr, c.Z, c.P, c.Q, c.sc, c.done + 1,
                                                 c.flag);
    pc_apply(c, 0);
  } else {
    k_update<true><<<vgrid(c), 256, 0, c.st>>>(c.minv, c.N, c.R, Xc, c.Rr, c.Z, c.P, c.Q, c.sc, c.done + 1,
                                                c.flag);
  }
  k_direction<<<vgrid(c), 256, 0, c.st>>>(c.N, c.R, c.Z, c.P, c.Pf, c.sc);
  return cudaGetLastError();
}

// A block of `steps` iterations into Xc, captured once as a CUDA graph and
// replayed (an iteration is six launches of a few microseconds each, as long
// as the matvec itself at N of a few thousand).  Returns null when capture is
// unavailable; the iterations are then launched one by one.
template <bool F64>
cudaGraphExec_t capture_block(const Pcg& c, double* Xc, int steps, int64_t* per_block) {
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  Pcg cc = c;
  cc.st = cs;
  const int64_t before = *c.nlaunch;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    for (int s = 0; s < steps && ok; ++s) ok = cg_iteration<F64>(cc, Xc) == cudaSuccess;
    const bool ended = cudaStreamEndCapture(cs, &g) == cudaSuccess;
    ok = ok && ended && g != nullptr;
  }
  if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  *per_block = *c.nlaunch - before;
  *c.nlaunch = before;
  if (!ok) {
    (void)cudaGetLastError();
    if (ex) cudaGraphExecDestroy(ex);
    return nullptr;
  }
  return ex;
}

#define NK_CHECK_EVERY 8

// CG on (K + lam I) Xc = B from Xc = 0 until every column's recursive
// residual is below tol (relative to ||B||) or maxit iterations; *its = the
// iterations performed (max over columns).  `graph` replays NK_CHECK_EVERY
// iterations into Xc (or is null); hflag is pinned host memory.
template <bool F64>
cudaError_t cg_run(const Pcg& c, const double* B, double* Xc, double tol, int maxit,
                   cudaGraphExec_t graph, int64_t per_block, int* hflag, int* its) {
  *c.nlaunch += 3;
  k_zero<<<1, 256, 0, c.st>>>(c.sc, (int64_t)SC_N * c.R);
  k_set_active<<<1, 256, 0, c.st>>>(c.sc, c.R, tol * tol);
  if (c.pc_rank > 0) {
    k_init_pc<<<vgrid(c), 256, 0, c.st>>>(B, c.N, c.R, Xc, c.Rr, c.sc);
    pc_apply(c, 1);
  } else {
    k_init<<<vgrid(c), 256, 0, c.st>>>(B, c.minv, c.N, c.R, Xc, c.Rr, c.Z, c.P, c.Pf, c.sc);
  }
  cudaError_t e = cudaSuccess;
  int it = 0;
  while (it < maxit) {
    const int steps = std::min(NK_CHECK_EVERY, maxit - it);
    if (graph && steps == NK_CHECK_EVERY) {
      *c.nlaunch += per_block;
      e = cudaGraphLaunch(graph, c.st);
    } else {
      for (int s = 0; s < steps && e == cudaSuccess; ++s) e = cg_iteration<F64>(c, Xc);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hflag, c.flag, sizeof(int), cudaMemcpyDeviceToHost, c.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
    if (e != cudaSuccess) return e;
    it += steps;
    if (*hflag == 0) break;
  }
  std::vector<double> hsc((size_t)SC_N * c.R);
  e = cudaMemcpy(hsc.data(), c.sc, sizeof(double) * SC_N * c.R, cudaMemcpyDeviceToHost);
  int mx = 0;
  for (int r = 0; r < c.R; ++r) mx = std::max(mx, (int)hsc[SC_ITER * c.R + r]);
  *its = mx;
  return e;
}

}  // namespace

// Host orchestration, called by nk_pcg_solve after argument validation.
//
// Mixed form: iterative refinement.  The true residual Y - (K + lam I) A is
// formed with FP64 products; the correction is solved by CG with FP32
// products and FP64 vectors and scalars to a relative tolerance eta; A += D.
// With FP32 products CG's true residual stalls about two decades below its
// right-hand side on these kernels (the recursive residual keeps falling,
// but the products' rounding, not the Krylov space, sets the level), so each
// sweep asks for eta = NK_ETA_FLOOR (or what is left to reach tol, if
// larger): iterations past that level would be spent below the rounding.
#define NK_ETA_FLOOR 3e-2

nk_status nk_pcg_impl(nk_handle* h, const float* K, int64_t ldk, int64_t N, const double* Y, int R,
                      double lam, int precond, nk_prec prec, double tol, int maxit, int refine_max,
                      double* A, int* iters, double* relres, cudaStream_t st) {
  Pcg c = {};
  c.N = N;
  c.R = R;
  c.K = K;
  c.ldk = ldk;
  c.lam = lam;
  c.sm = h->sm_count;
  c.st = st;
  c.nlaunch = &h->launches;
  const int occ = matvec_prepare(R);
  const int S = choose_splits(N, R, c.sm, occ);
  c.S = S;
  c.rows_per_split = (int)((N + S - 1) / S);
  const size_t NR = (size_t)N * R;
  const int pr = (precond == NK_PRECOND_PIVCHOL) ? (int)std::min<int64_t>(std::max(h->pcg_rank, 1), N) : 0;
  const size_t pc_bytes = pr ? ((size_t)pr * N * 8 + 3 * (size_t)pr * pr * 8 + 2 * (size_t)pr * R * 8 +
                                (size_t)N * 8 + 64 + 8 * 256)
                             : 0;
  size_t bytes = NR * 8 * 7 + (size_t)S * NR * 8 + (size_t)N * 8 + SC_N * (size_t)R * 8 + NR * 4 * 3 + 14 * 256 +
                 pc_bytes;
  if (bytes > h->pcg_bytes) {
    if (h->pcg_ws) cudaFree(h->pcg_ws);
    h->pcg_ws = nullptr;
    h->pcg_bytes = 0;
    if (cudaMalloc(&h->pcg_ws, bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      return nk_fail(h, NK_ERR_NO_MEMORY, "pcg workspace of %zu bytes", bytes);
    }
    h->pcg_bytes = bytes;
  }
  char* w = (char*)h->pcg_ws;
  auto take = [&](size_t n) { char* p = w; w += (n + 255) / 256 * 256; return p; };
  c.Rr = (double*)take(NR * 8);
  c.Z = (double*)take(NR * 8);
  c.P = (double*)take(NR * 8);
  c.Q = (double*)take(NR * 8);
  c.B2 = (double*)take(NR * 8);
  double* D = (double*)take(NR * 8);
  c.Qpart = (double*)take((size_t)S * NR * 8);
  c.minv = (double*)take((size_t)N * 8);
  c.sc = (double*)take(SC_N * (size_t)R * 8);
  c.Pf = (float*)take(NR * 4);
  c.Xh = (float*)take(NR * 4);
  c.Xl = (float*)take(NR * 4);
  c.flag = (int*)take(64);
  c.done = c.flag + 4;  // same 64-byte slot: flag, pad, done[4]
  double *pc_G = nullptr, *pc_W = nullptr, *pc_d = nullptr;
  PcState* pc_st = nullptr;
  c.pc_rank = pr;
  if (pr) {
    c.L = (double*)take((size_t)pr * N * 8);
    pc_G = (double*)take((size_t)pr * pr * 8);
    pc_W = (double*)take((size_t)pr * pr * 8);
    c.Ginv = (double*)take((size_t)pr * pr * 8);
    c.T = (double*)take((size_t)pr * R * 8);
    c.U = (double*)take((size_t)pr * R * 8);
    pc_d = (double*)take((size_t)N * 8);
    pc_st = (PcState*)take(64);
  }
  {
    const cudaError_t z = cudaMemsetAsync(c.flag, 0, 64, st);
    if (z != cudaSuccess) return nk_cuda_check(h, z, "pcg counters");
  }

  // pinned host words: the active-column flag and the CG scalars
  void* host = nullptr;
  const size_t host_bytes = 64 + sizeof(double) * SC_N * R;
  const bool pinned = cudaMallocHost(&host, host_bytes) == cudaSuccess;
  if (!pinned) {
    (void)cudaGetLastError();
    host = malloc(host_bytes);
  }
  int* hflag = (int*)host;
  double* hsc = (double*)((char*)host + 64);
  cudaGraphExec_t graph = nullptr;
  auto finish = [&](nk_status s) {
    if (graph) cudaGraphExecDestroy(graph);
    if (pinned)
      cudaFreeHost(host);
    else
      free(host);
    return s;
  };
  auto read_sc = [&]() {
    cudaError_t e = cudaMemcpyAsync(hsc, c.sc, sizeof(double) * SC_N * R, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
  };
  // worst relative true residual after true_residual(); fills relres
  auto worst_rel = [&]() {
    double worst = 0.0;
    for (int r = 0; r < R; ++r) {
      const double yy = hsc[SC_YY * R + r];
      const double rel = yy > 0 ? sqrt(hsc[SC_RR * R + r] / yy) : sqrt(hsc[SC_RR * R + r]);
      if (relres) relres[r] = rel;
      worst = std::max(worst, rel);
    }
    return worst;
  };
  cudaError_t e = cudaSuccess;
  if (lam < 0.0) {
    // relative ridge: lam = |lam| * tr(K) / N
    ++h->launches;
    k_trace<<<1, 256, 0, st>>>(K, ldk, N, c.sc);
    e = cudaMemcpyAsync(hsc, c.sc, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return finish(nk_cuda_check(h, e, "pcg trace"));
    lam = -lam * hsc[0] / (double)N;
    c.lam = lam;
  }
  h->last_lambda = lam;
  ++h->launches;
  k_minv<<<(unsigned)std::min<int64_t>((N + 255) / 256, 4 * c.sm), 256, 0, st>>>(
      K, ldk, N, lam, precond == NK_PRECOND_JACOBI, c.minv);
  if (pr) {
    // partial pivoted Cholesky of K, then G = lam I + L L^T and its inverse
    const unsigned rows_grid = (unsigned)std::min<int64_t>((N + 255) / 256, 4 * c.sm);
    h->launches += pr + 3;
    k_pc_diag<<<1, 1024, 0, st>>>(K, ldk, N, pc_d, pc_st);
    for (int k = 0; k < pr; ++k)
      k_pc_row<<<rows_grid, 256, 0, st>>>(K, ldk, N, c.L, pc_d, k, pc_st, c.done + 2);
    k_pc_gram<<<dim3((unsigned)pr, (unsigned)pr), 256, 0, st>>>(c.L, pr, N, lam, pc_G);
    k_pc_factor<<<1, 256, 0, st>>>(pc_G, pr, pc_W, c.Ginv);
    e = cudaGetLastError();
    if (e != cudaSuccess) return finish(nk_cuda_check(h, e, "pcg preconditioner"));
  }
  const bool f64 = prec == NK_PREC_PLAIN_FP64;
  const bool warm = h->pcg_warm != 0;
  // CG iterates into the correction D when it refines the caller's or its
  // own earlier A (the captured iteration block writes one fixed array)
  double* Xc = (prec == NK_PREC_MIXED || warm) ? D : A;
  int64_t per_block = 0;
  graph = f64 ? capture_block<true>(c, Xc, NK_CHECK_EVERY, &per_block)
              : capture_block<false>(c, Xc, NK_CHECK_EVERY, &per_block);
  bool converged = false;
  int total_it = 0;
  if (prec == NK_PREC_MIXED) {
    if (!warm) {
      ++h->launches;
      k_zero<<<(unsigned)std::min<int64_t>((NR + 255) / 256, 4 * c.sm), 256, 0, st>>>(A, NR);
    }
    for (int outer = 0;; ++outer) {
      if (outer == 0 && !warm) {
        // A = 0: the residual is Y itself
        h->launches += 3;
        k_zero<<<1, 256, 0, st>>>(c.sc, (int64_t)SC_N * R);
        k_zero<<<(unsigned)std::min<int64_t>((NR + 255) / 256, 4 * c.sm), 256, 0, st>>>(c.Q, NR);
        k_resid<<<vgrid(c), 256, 0, st>>>(Y, c.Q, N, R, c.B2, c.sc);
        e = cudaGetLastError();
      } else {
        e = true_residual(c, Y, A, c.B2, false);
      }
      if (e == cudaSuccess) e = read_sc();
      if (e != cudaSuccess) break;
      const double worst = worst_rel();
      if (worst <= tol) {
        converged = true;
        break;
      }
      if (outer >= refine_max || total_it >= maxit) break;
      const double eta = std::min(std::max(0.5 * tol / worst, NK_ETA_FLOOR), 0.5);
      int its = 0;
      e = cg_run<false>(c, c.B2, D, eta, maxit - total_it, graph, per_block, hflag, &its);
      if (e != cudaSuccess) break;
      total_it += its;
      ++h->launches;
      k_add<<<(unsigned)std::min<int64_t>((NR + 255) / 256, 4 * c.sm), 256, 0, st>>>(NR, A, D);
    }
  } else if (warm) {
    // from the caller's A: one correction solve (K + lam I) D = Y - (K + lam I) A
    // to the relative tolerance that brings every column's residual to tol
    e = true_residual(c, Y, A, c.B2, f64);
    if (e == cudaSuccess) e = read_sc();
    const double worst = e == cudaSuccess ? worst_rel() : 0.0;
    if (e == cudaSuccess && worst > tol) {
      const double eta = tol / worst;
      e = f64 ? cg_run<true>(c, c.B2, D, eta, maxit, graph, per_block, hflag, &total_it)
              : cg_run<false>(c, c.B2, D, eta, maxit, graph, per_block, hflag, &total_it);
      if (e == cudaSuccess) {
        ++h->launches;
        k_add<<<(unsigned)std::min<int64_t>((NR + 255) / 256, 4 * c.sm), 256, 0, st>>>(NR, A, D);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = true_residual(c, Y, A, c.B2, f64);
      if (e == cudaSuccess) e = read_sc();
    }
    if (e == cudaSuccess) converged = worst_rel() <= tol;
  } else {
    e = f64 ? cg_run<true>(c, Y, A, tol, maxit, graph, per_block, hflag, &total_it)
            : cg_run<false>(c, Y, A, tol, maxit, graph, per_block, hflag, &total_it);
    if (e == cudaSuccess) e = true_residual(c, Y, A, c.B2, f64);
    if (e == cudaSuccess) e = read_sc();
    if (e == cudaSuccess) converged = worst_rel() <= tol;
  }
  if (e != cudaSuccess) return finish(nk_cuda_check(h, e, "pcg"));
  if (iters) *iters = total_it;
  if (!converged) {
    nk_fail(h, NK_ERR_NOT_CONVERGED, "pcg did not reach tol %.3g in %d iterations", tol, total_it);
    return finish(NK_ERR_NOT_CONVERGED);
  }
  return finish(NK_OK);
}
