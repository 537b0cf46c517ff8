// Fused Myrtle NNGP block (NK_PREC_MIXED): one persistent launch, pixel-pair
// tensors never leave the chip.
//
// What is computed (Appendix A, Myrtle listing; the NNGP definition):
//   K_1(p,p')   = sw2/9 sum_delta (1/C) <x[p+delta], x'[p'+delta]> + sb2
//   Kt_l(p,p')  = sqrt(q q')/(2 pi) J(K_l / sqrt(q q'))           (stax.Relu)
//   K_{l+1}     = sw2/9 sum_delta Kt_l(p+delta, p'+delta) + sb2     (stax.Conv SAME)
//   pool        = 1/16 sum_{a,b in {0,1}^2} Kt(2P+a, 2P'+b)          (stax.AvgPool)
//   K(x,x')     = sw2 mean_{P,P'} Kt(P,P') + sb2                     (GAP + Dense)
//
// Decomposition ("super-planes").  For a shift t = (t_y, t_x) in [0,R)^2 the
// super-plane t holds the R*R pixel pairs (p, p') with p' = (p + t) mod R.
// The conv stencil maps a super-plane to itself (both pixels move by the same
// delta), except across two cuts where p' wraps (column R-1-t_x | R-t_x and
// row R-1-t_y | R-t_y) and at the image border: there the neighbour is a
// zero-padding term.  So the whole stage recursion of a super-plane is a
// stream of R rows of R values, with no halo recomputation, and the R^2
// super-planes cover the R^4 pixel pairs exactly once.
//
// Thread mapping: a warp owns one t_x (warp-uniform, so the column cut is
// uniform) and 16 consecutive t_y; lane = 16 h + (t_y - ty0) with h the
// column half.  Each thread streams the rows of its super-plane, holding its
// R/2 columns in registers; the horizontal 3-tap sum takes one halo value from
// the partner lane (shfl xor 16), the column cut is fixed by a warp-uniform
// switch, and the row cut by a 0/1 factor in the vertical FFMAs.  All layers
// of the stage are pipelined with a one-row delay per layer.  The p-side
// tables (x, 1/sqrt q, sqrt q at row i) are warp-broadcast loads; the p'-side
// ones are a conflict-free gather from tables doubled along columns.
//
// Pooling: super-plane t of stage s feeds super-plane floor/ceil(t/2) of
// stage s+1 (odd shifts split by pixel parity); rows are paired in registers
// and columns paired when t_x is even, the rest goes through shared-memory
// atomics into the next stage's buffer.  At 32x32 that buffer (64K floats)
// is distributed over a 4-CTA cluster by T_x and reached through DSMEM.  The
// last stage is reduced into the global average.
//
// Scale factors sw2/9, 1/(2 pi), 1/16 and 1/C are folded into the p-side
// tables, so a conv is 1.5 adds + 2 FFMA + 1 add per pixel pair and the map
// is ~25 FP32 instructions (nk_map.cuh).
#include "nk_common.cuh"
#include "nk_map.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;
#define NK_FUSED_THREADS 512

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::
                   : "memory");
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned mapa_rank(unsigned a, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ void red_cluster_f32(unsigned a, float v) {
  asm volatile("red.shared::cluster.add.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

__device__ __forceinline__ void st_cluster_f64(unsigned a, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}

// Linear pair index -> (i, j) of the block; the upper triangle row by row
// when symmetric.
__device__ __forceinline__ void pair_ij(int64_t idx, int64_t na, int64_t nb, int sym, int64_t* i,
                                        int64_t* j) {
  if (!sym) {
    *i = idx / nb;
    *j = idx - (*i) * nb;
    return;
  }
  const double m = (double)na;
  double t = (2.0 * m + 1.0) * (2.0 * m + 1.0) - 8.0 * (double)idx;
  int64_t r = (int64_t)floor(((2.0 * m + 1.0) - sqrt(t > 0 ? t : 0)) / 2.0);
  if (r < 0) r = 0;
  if (r > na - 1) r = na - 1;
  for (int it = 0; it < 4 && r > 0 && r * na - r * (r - 1) / 2 > idx; ++it) --r;
  for (int it = 0; it < 4 && r + 1 < na && (r + 1) * na - (r + 1) * r / 2 <= idx; ++it) ++r;
  *i = r;
  *j = r + (idx - (r * na - r * (r - 1) / 2));
}

struct FusedParams {
  const float* Xa;
  const float* Xb;
  const float* qsa;  // float2 pairs (1/sqrt q, sqrt q)
  const float* qsb;
  int64_t a0, na, b0, nb;
  int sym;
  int64_t npairs;
  float* K;
  int64_t ldk;
  int C;
  int nq;
  int qoff[NK_MAX_LAYERS];
  float fold[NK_MAX_LAYERS];  // factor folded into the p-side sqrt(q) of each layer
  float xscale;               // sw2 / (9 C) folded into x
  float sb2;
  double out_scale;           // sw2 / R_gap^4
  double out_bias;            // sb2
};

// ---------------------------------------------------------------------------
// Shared-memory layout (compile-time)
// ---------------------------------------------------------------------------
template <int R0, int N0, int N1, int N2, int CL>
struct Layout {
  static constexpr int SE = 1 + (N1 > 0 ? 1 : 0) + ((N1 > 0 && N2 > 0) ? 1 : 0);
  static constexpr int R1 = R0 / 2, R2 = R0 / 4;
  static constexpr int S0 = 2 * R0 + 1, S1 = 2 * R1 + 1, S2 = 2 * R2 + 1;
  // stage-1 input buffer (pooled stage-0 output), T_x split over the cluster
  static constexpr int TXL1 = R1 / CL;
  static constexpr int B1_sTx = R1 * R1;
  static constexpr int B1_sTy = TXL1 * R1 * R1 + 1;
  static constexpr int B1_size = (SE >= 2) ? R1 * B1_sTy : 0;  // floats
  // stage-2 input buffer, all in rank 0
  static constexpr int TXL2 = R2;
  static constexpr int B2_sTx = R2 * R2;
  static constexpr int B2_sTy = TXL2 * R2 * R2 + 1;
  static constexpr int B2_size = (SE >= 3) ? R2 * B2_sTy : 0;
  // bytes
  static constexpr size_t xs_off = 0;                                    // float4 [R0*R0]
  static constexpr size_t xq_off = xs_off + (size_t)R0 * R0 * 16;        // float4 [R0][S0]
  static constexpr size_t p0_off = xq_off + (size_t)R0 * S0 * 16;        // float2 [N0][R0*R0]
  static constexpr size_t q0_off = p0_off + (size_t)N0 * R0 * R0 * 8;    // float2 [N0][R0][S0]
  static constexpr size_t p1_off = q0_off + (size_t)N0 * R0 * S0 * 8;
  static constexpr size_t q1_off = p1_off + (size_t)N1 * R1 * R1 * 8;
  static constexpr size_t p2_off = q1_off + (size_t)N1 * R1 * S1 * 8;
  static constexpr size_t q2_off = p2_off + (size_t)N2 * R2 * R2 * 8;
  static constexpr size_t b1_off = ((q2_off + (size_t)N2 * R2 * S2 * 8) + 15) / 16 * 16;
  // the stage-2 buffer reuses the stage-0 x' table, dead once stage 0 is done
  static constexpr size_t b2_off = xq_off;
  static_assert((size_t)B2_size * 4 <= (size_t)R0 * S0 * 16, "stage-2 buffer alias");
  static constexpr size_t gap_off = (b1_off + (size_t)B1_size * 4 + 15) / 16 * 16;  // double[8]
  static constexpr size_t red_off = gap_off + 8 * 8;                               // double[32]
  static constexpr size_t bytes = red_off + 32 * 8;
};

// ---------------------------------------------------------------------------
// Thread mapping of a stage at resolution R: a row of the super-plane is split
// into NQ parts of COLS columns; a warp holds TYW = 32 / NQ shifts t_y and the
// NQ parts of each (lane = q * TYW + t_y - ty0).
// ---------------------------------------------------------------------------
template <int R>
struct Split {
  static constexpr int NQ = R >= 4 ? 4 : R;
  static constexpr int COLS = R / NQ;
  static constexpr int TYW = 32 / NQ;
  static constexpr int WPT = R > TYW ? R / TYW : 1;  // warps per t_x
};

// Horizontal 3-tap sum of one row part with halos and the column cut.
template <int COLS, int NQ, int TYW>
__device__ __forceinline__ void hsum(const float (&A)[COLS], float (&Hc)[COLS], int kl, int q) {
  const float fromL = __shfl_up_sync(FULL, A[COLS - 1], TYW);
  const float fromR = __shfl_down_sync(FULL, A[0], TYW);
  const float left = (q > 0) ? fromL : 0.f;
  const float right = (q < NQ - 1) ? fromR : 0.f;
  if constexpr (COLS == 1) {
    Hc[0] = left + A[0] + right;
  } else {
#pragma unroll
    for (int k = 0; k < COLS; k += 2) {
      // pairwise sharing: s = A[k] + A[k+1]
      const float s = A[k] + A[k + 1];
      Hc[k] = (k == 0 ? left : A[k - 1]) + s;
      Hc[k + 1] = s + (k + 2 < COLS ? A[k + 2] : right);
    }
  }
  // column cut between local columns kl and kl + 1 (uniform per part)
#define NK_SEAM(m)                                                                    \
  case m:                                                                             \
    if constexpr ((m) < COLS) {                                                       \
      Hc[m] = ((m) > 0 ? A[(m) > 0 ? (m)-1 : 0] : left) + A[m];                       \
      if constexpr ((m) + 1 < COLS)                                                   \
        Hc[(m) + 1 < COLS ? (m) + 1 : 0] =                                            \
            A[(m) + 1 < COLS ? (m) + 1 : 0] + ((m) + 2 < COLS ? A[(m) + 2 < COLS ? (m) + 2 : 0] : right); \
    }                                                                                 \
    break;
  switch (kl) {
    case -1:
      Hc[0] = A[0] + (COLS > 1 ? A[COLS > 1 ? 1 : 0] : right);
      break;
      NK_SEAM(0) NK_SEAM(1) NK_SEAM(2) NK_SEAM(3) NK_SEAM(4) NK_SEAM(5) NK_SEAM(6) NK_SEAM(7)
    default:
      break;
  }
#undef NK_SEAM
}

// Scatter target of the next stage's buffer (which CTA of the cluster owns
// T_x, and the local float offset).
struct ScatterTo {
  float* buf;      // local base of the buffer (same offset in every CTA)
  int sTy, sTx;    // strides
  int R2;          // next-stage resolution
  int txl;         // T_x per owning CTA
  unsigned rank;   // my rank
};

__device__ __forceinline__ void scatter_add(const ScatterTo& s, int Ty, int Tx, int I, int Kx,
                                            float v) {
  const int owner = Tx / s.txl;
  const int loc = Tx - owner * s.txl;
  float* a = s.buf + Ty * s.sTy + loc * s.sTx + I * s.R2 + Kx;
  if ((unsigned)owner == s.rank) {
    atomicAdd(a, v);
  } else {
    red_cluster_f32(mapa_rank(smem_u32(a), (unsigned)owner), v);
  }
}

template <int COLS>
__device__ __forceinline__ void scatter_row(const ScatterTo& s, int t_x, int Ty, int I, int c0,
                                            const float (&v)[COLS]) {
  const int R2 = s.R2;
  if constexpr (COLS % 2 == 0) {
    if ((t_x & 1) == 0) {
      const int Tx = t_x >> 1;
#pragma unroll
      for (int k = 0; k < COLS; k += 2) scatter_add(s, Ty, Tx, I, (c0 + k) >> 1, v[k] + v[k + 1]);
      return;
    }
  }
  const int TxE = t_x >> 1;                    // even pixel column (odd t_x), or even t_x
  const int TxO = ((t_x + 1) >> 1) & (R2 - 1); // odd pixel column, odd t_x
#pragma unroll
  for (int k = 0; k < COLS; ++k) {
    const int c = c0 + k;
    const int Tx = ((t_x & 1) && (c & 1)) ? TxO : TxE;
    scatter_add(s, Ty, Tx, I, c >> 1, v[k]);
  }
}

// ---------------------------------------------------------------------------
// One warp task: super-planes (t_y in ty0 .. ty0+TYW-1, t_x) of a stage.
// ---------------------------------------------------------------------------
template <int R, int N, bool SEED, bool GAP>
__device__ __forceinline__ void stage_task(int t_x, int ty0, const float4* __restrict__ xs,
                                           const float4* __restrict__ xq,
                                           const float* __restrict__ inb, int in_sTy,
                                           const float2* __restrict__ ptab,
                                           const float2* __restrict__ qtab, float b,
                                           const ScatterTo& sc, double& gap) {
  using SP = Split<R>;
  constexpr int COLS = SP::COLS, NQ = SP::NQ, TYW = SP::TYW;
  constexpr int S = 2 * R + 1;
  const int lane = threadIdx.x & 31;
  const int q = lane / TYW, tyl = lane - q * TYW;
  const bool act = tyl < R;
  const int t_y = (ty0 + tyl) & (R - 1);
  const int c0 = q * COLS;
  const int kl = (t_x == 0) ? -100 : (R - 1 - t_x) - c0;
  const bool tyodd = (t_y & 1) != 0;

  float Hp[N][COLS], Pp[N][COLS], acc[COLS];
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int k = 0; k < COLS; ++k) Hp[j][k] = Pp[j][k] = 0.f;
#pragma unroll
  for (int k = 0; k < COLS; ++k) acc[k] = 0.f;

  for (int t = 0; t < R + N; ++t) {
    float A[COLS];
    if (t < R) {
      if constexpr (SEED) {
        const int pr = (t + t_y) & (R - 1);
        const float4* xa = xs + t * R + c0;
        const float4* xb = xq + pr * S + c0 + t_x;
#pragma unroll
        for (int k = 0; k < COLS; ++k) {
          const float4 u = xa[k], w = xb[k];
          A[k] = fmaf(u.x, w.x, fmaf(u.y, w.y, fmaf(u.z, w.z, u.w * w.w)));
        }
      } else {
        const float* row = inb + t_y * in_sTy + t * R + c0;
#pragma unroll
        for (int k = 0; k < COLS; ++k) A[k] = row[k];
      }
    } else {
#pragma unroll
      for (int k = 0; k < COLS; ++k) A[k] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const int r = t - j;  // row entering layer j at this step
      if (r < 0) break;
      if (r > R) continue;
      float Hc[COLS];
      if (r < R) {
        hsum<COLS, NQ, TYW>(A, Hc, kl, q);
      } else {
#pragma unroll
        for (int k = 0; k < COLS; ++k) Hc[k] = 0.f;
      }
      const float e = (r != R - t_y) ? 1.f : 0.f;  // edge (r-1, r) not cut
      if (r >= 1) {
        const int ro = r - 1;
        const int pr = (ro + t_y) & (R - 1);
        const float2* pt = ptab + (size_t)j * R * R + ro * R + c0;
        const float2* qt = qtab + (size_t)j * R * S + pr * S + c0 + t_x;
#pragma unroll
        for (int k = 0; k < COLS; ++k) {
          const float K = fmaf(e, Hc[k], Pp[j][k]) + b;
          const float2 pv = pt[k], qv = qt[k];
          const float c = K * (pv.x * qv.x);
          // the first layer sees any sign; later correlations are >= 0
          const float J = (SEED && j == 0) ? nk_J_f32(c) : nk_J01_f32(c);
          A[k] = (pv.y * qv.y) * J;
        }
      }
      if (r < R) {
#pragma unroll
        for (int k = 0; k < COLS; ++k) {
          Pp[j][k] = fmaf(e, Hp[j][k], Hc[k]);
          Hp[j][k] = Hc[k];
        }
      }
      if (r == 0) break;
    }
    const int ro = t - N;  // output row of the last layer at this step
    if (ro >= 0 && ro < R) {
      if constexpr (GAP) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < COLS; ++k) s += A[k];
        if (act) gap += (double)s;
      } else {
        if ((ro & 1) == 0) {
#pragma unroll
          for (int k = 0; k < COLS; ++k) acc[k] = A[k];
        } else {
          const int I = ro >> 1;
          float v[COLS];
#pragma unroll
          for (int k = 0; k < COLS; ++k) v[k] = tyodd ? acc[k] : acc[k] + A[k];
          if (act) scatter_row<COLS>(sc, t_x, t_y >> 1, I, c0, v);
          if (act && tyodd) scatter_row<COLS>(sc, t_x, ((t_y + 1) >> 1) & (sc.R2 - 1), I, c0, A);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Per-pair table staging
// ---------------------------------------------------------------------------
template <int R, int NL>
__device__ __forceinline__ void stage_q_tables(const FusedParams& P, int layer0, int64_t ia,
                                               int64_t ib, float2* pt, float2* qt) {
  constexpr int S = 2 * R + 1;
  const float2* qa = reinterpret_cast<const float2*>(P.qsa) + ia * P.nq;
  const float2* qb = reinterpret_cast<const float2*>(P.qsb) + ib * P.nq;
  for (int j = 0; j < NL; ++j) {
    const int L = layer0 + j;
    const float f = P.fold[L];
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
      const float2 v = qa[P.qoff[L] + e];
      pt[j * R * R + e] = make_float2(v.x, v.y * f);
    }
    for (int e = threadIdx.x; e < R * 2 * R; e += blockDim.x) {
      const int row = e / (2 * R), col = e - row * 2 * R;
      qt[j * R * S + row * S + col] = qb[P.qoff[L] + row * R + (col & (R - 1))];
    }
  }
}

template <int R0, int N0, int N1, int N2, int CL>
__global__ void __launch_bounds__(NK_FUSED_THREADS, 1) k_myrtle_fused(const __grid_constant__ FusedParams P) {
  using L = Layout<R0, N0, N1, N2, CL>;
  constexpr int SE = L::SE;
  constexpr int R1 = L::R1, R2 = L::R2;
  extern __shared__ __align__(16) unsigned char smem[];
  float4* xs = reinterpret_cast<float4*>(smem + L::xs_off);
  float4* xq = reinterpret_cast<float4*>(smem + L::xq_off);
  float2* p0 = reinterpret_cast<float2*>(smem + L::p0_off);
  float2* q0 = reinterpret_cast<float2*>(smem + L::q0_off);
  float2* p1 = reinterpret_cast<float2*>(smem + L::p1_off);
  float2* q1 = reinterpret_cast<float2*>(smem + L::q1_off);
  float2* p2 = reinterpret_cast<float2*>(smem + L::p2_off);
  float2* q2 = reinterpret_cast<float2*>(smem + L::q2_off);
  float* b1 = reinterpret_cast<float*>(smem + L::b1_off);
  float* b2 = reinterpret_cast<float*>(smem + L::b2_off);
  double* gap_slots = reinterpret_cast<double*>(smem + L::gap_off);
  double* red = reinterpret_cast<double*>(smem + L::red_off);

  const unsigned rank = (CL > 1) ? cluster_rank() : 0u;
  const int64_t cid = blockIdx.x / CL;
  const int64_t ncl = gridDim.x / CL;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int C = P.C;

  for (int64_t pidx = cid; pidx < P.npairs; pidx += ncl) {
    int64_t i, j;
    pair_ij(pidx, P.na, P.nb, P.sym, &i, &j);
    const int64_t ia = P.a0 + i, ib = P.b0 + j;
    // ---- stage tables
    {
      const float* xa = P.Xa + ia * (int64_t)R0 * R0 * C;
      const float* xb = P.Xb + ib * (int64_t)R0 * R0 * C;
      for (int e = threadIdx.x; e < R0 * R0; e += blockDim.x) {
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        for (int c = 0; c < C; ++c) v[c] = xa[e * C + c] * P.xscale;
        xs[e] = make_float4(v[0], v[1], v[2], v[3]);
      }
      for (int e = threadIdx.x; e < R0 * 2 * R0; e += blockDim.x) {
        const int row = e / (2 * R0), col = e - row * 2 * R0;
        const float* src = xb + (row * R0 + (col & (R0 - 1))) * C;
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        for (int c = 0; c < C; ++c) v[c] = src[c];
        xq[row * L::S0 + col] = make_float4(v[0], v[1], v[2], v[3]);
      }
      stage_q_tables<R0, N0>(P, 0, ia, ib, p0, q0);
      if constexpr (SE >= 2) stage_q_tables<R1, N1>(P, N0, ia, ib, p1, q1);
      if constexpr (SE >= 3) stage_q_tables<R2, N2>(P, N0 + N1, ia, ib, p2, q2);
      for (int e = threadIdx.x; e < L::B1_size; e += blockDim.x) b1[e] = 0.f;
    }
    if constexpr (CL > 1) cluster_sync_all(); else __syncthreads();

    double gap = 0.0;
    // ---- stage 0
    {
      constexpr int NH = Split<R0>::WPT;  // warps per t_x
      constexpr int TXC = R0 / CL;        // t_x per CTA
      ScatterTo sc{b1, L::B1_sTy, L::B1_sTx, R1, L::TXL1, rank};
      for (int task = warp; task < TXC * NH; task += nwarps) {
        const int t_x = (int)rank * TXC + task / NH;
        const int ty0 = (task % NH) * Split<R0>::TYW;
        stage_task<R0, N0, true, SE == 1>(t_x, ty0, xs, xq, nullptr, 0, p0, q0, P.sb2, sc, gap);
      }
    }
    if constexpr (SE >= 3) {
      // b2 aliases xq: zero it only once every warp of this CTA left stage 0
      __syncthreads();
      if (rank == 0)
        for (int e = threadIdx.x; e < L::B2_size; e += blockDim.x) b2[e] = 0.f;
    }
    if constexpr (SE >= 2) {
      if constexpr (CL > 1) cluster_sync_all(); else __syncthreads();
      constexpr int TXC = R1 / CL;
      constexpr int NH = Split<R1>::WPT;
      ScatterTo sc{b2, L::B2_sTy, L::B2_sTx, R2, L::TXL2, rank};
      for (int task = warp; task < TXC * NH; task += nwarps) {
        const int tl = task / NH;
        const int t_x = (int)rank * TXC + tl;
        const float* inb = b1 + tl * L::B1_sTx;
        stage_task<R1, N1, false, SE == 2>(t_x, (task % NH) * Split<R1>::TYW, nullptr, nullptr, inb,
                                           L::B1_sTy, p1, q1, P.sb2, sc, gap);
      }
    }
    if constexpr (SE >= 3) {
      if constexpr (CL > 1) cluster_sync_all(); else __syncthreads();
      if (rank == 0) {
        ScatterTo sc{nullptr, 0, 0, 1, 1, rank};
        constexpr int NH = Split<R2>::WPT;
        for (int task = warp; task < R2 * NH; task += nwarps) {
          const int tl = task / NH;
          const float* inb = b2 + tl * L::B2_sTx;
          stage_task<R2, N2, false, true>(tl, (task % NH) * Split<R2>::TYW, nullptr, nullptr, inb,
                                          L::B2_sTy, p2, q2, P.sb2, sc, gap);
        }
      }
    }
    // ---- global average: warp -> CTA -> cluster rank 0
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gap += __shfl_xor_sync(FULL, gap, o);
    if ((threadIdx.x & 31) == 0) red[warp] = gap;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < nwarps; ++w) s += red[w];
      if constexpr (CL > 1) {
        st_cluster_f64(mapa_rank(smem_u32(gap_slots + rank), 0u), s);
      } else {
        gap_slots[0] = s;
      }
    }
    if constexpr (CL > 1) cluster_sync_all(); else __syncthreads();
    if (rank == 0 && threadIdx.x == 0) {
      double s = 0.0;
      for (int r = 0; r < CL; ++r) s += gap_slots[r];
      const float v = (float)(P.out_scale * s + P.out_bias);
      P.K[i * P.ldk + j] = v;
      if (P.sym && i != j) P.K[j * P.ldk + i] = v;
    }
    // buffers are re-zeroed at the top of the next pair, after every CTA has
    // passed the barrier above
  }
}

template <int R0, int N0, int N1, int N2, int CL>
cudaError_t launch(const FusedParams& P, int sm_count, cudaStream_t st) {
  using L = Layout<R0, N0, N1, N2, CL>;
  auto kern = k_myrtle_fused<R0, N0, N1, N2, CL>;
  const size_t smem = L::bytes;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (CL > 1) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(NK_FUSED_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = sm_count / CL;
  if (CL > 1) {
    cfg.gridDim = dim3(CL, 1, 1);
    int maxc = 0;
    if (cudaOccupancyMaxActiveClusters(&maxc, kern, &cfg) == cudaSuccess && maxc > 0)
      nclusters = maxc;
    else
      (void)cudaGetLastError();
  }
  if (nclusters > P.npairs) nclusters = (int)P.npairs;
  if (nclusters < 1) nclusters = 1;
  cfg.gridDim = dim3((unsigned)(nclusters * CL), 1, 1);
  e = cudaLaunchKernelEx(&cfg, kern, P);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

bool nk_myrtle_fused_supported(const NkGeom& g) {
  if (g.filter != 3 || g.act != NK_ACT_RELU || g.C < 1 || g.C > 4) return false;
  if (g.Hs[0] != g.Ws[0]) return false;
  const int R0 = g.Hs[0];
  if (R0 != 8 && R0 != 16 && R0 != 32) return false;
  int c[3] = {0, 0, 0};
  for (int s = 0; s < g.n_stages; ++s) {
    if (s >= 3) {
      if (g.convs[s] != 0) return false;
      continue;
    }
    c[s] = g.convs[s];
  }
  // zero-conv stages only at the end
  if (c[1] == 0 && c[2] != 0) return false;
  const bool ok = (c[0] == 2 && c[1] == 1 && c[2] == 0) || (c[0] == 2 && c[1] == 1 && c[2] == 1) ||
                  (c[0] == 3 && c[1] == 3 && c[2] == 3) || (c[0] == 1 && c[1] == 0 && c[2] == 0) ||
                  (c[0] == 1 && c[1] == 1 && c[2] == 1);
  if (!ok) return false;
  if (g.n_stages < 3 && c[2] != 0) return false;
  if (R0 == 8 && c[1] > 0 && c[2] > 0 && g.n_stages >= 3) return true;
  return true;
}

cudaError_t nk_launch_myrtle_fused(const NkGeom& g, double sw2, double sb2, const float* Xa,
                                   const float* qsa, int64_t a0, int64_t a1, const float* Xb,
                                   const float* qsb, int64_t b0, int64_t b1, float* K,
                                   int64_t ldk, int symmetric, int sm_count,
                                   unsigned int* dstatus, cudaStream_t st) {
  (void)dstatus;
  if (!nk_myrtle_fused_supported(g)) return cudaErrorNotSupported;
  FusedParams P = {};
  P.Xa = Xa;
  P.Xb = Xb;
  P.qsa = qsa;
  P.qsb = qsb;
  P.a0 = a0;
  P.na = a1 - a0;
  P.b0 = b0;
  P.nb = b1 - b0;
  P.sym = symmetric;
  P.npairs = symmetric ? P.na * (P.na + 1) / 2 : P.na * P.nb;
  if (P.npairs <= 0) return cudaSuccess;
  P.K = K;
  P.ldk = ldk;
  P.C = g.C;
  P.nq = g.nq;
  int c[3] = {g.convs[0], g.n_stages > 1 ? g.convs[1] : 0, g.n_stages > 2 ? g.convs[2] : 0};
  const int SE = 1 + (c[1] > 0) + (c[1] > 0 && c[2] > 0);
  const double a = sw2 / 9.0;
  const double inv2pi = 0.15915494309189533577;
  int layer = 0;
  for (int s = 0; s < SE; ++s) {
    for (int k = 0; k < c[s]; ++k, ++layer) {
      P.qoff[layer] = g.layer_qoff[layer];
      double f;
      if (k + 1 < c[s]) f = a * inv2pi;
      else if (s + 1 < SE) f = a * inv2pi / 16.0;
      else f = inv2pi;
      P.fold[layer] = (float)f;
    }
  }
  P.xscale = (float)(a / g.C);
  P.sb2 = (float)sb2;
  const int Rg = g.Hs[0] >> (SE - 1);
  P.out_scale = sw2 / ((double)Rg * Rg * Rg * Rg);
  P.out_bias = sb2;
  const int R0 = g.Hs[0];
#define NK_DISPATCH(RR, A0, A1, A2, CLL) \
  if (R0 == RR && c[0] == A0 && c[1] == A1 && c[2] == A2) return launch<RR, A0, A1, A2, CLL>(P, sm_count, st);
  NK_DISPATCH(32, 2, 1, 0, 4)
  NK_DISPATCH(32, 2, 1, 1, 4)
  NK_DISPATCH(32, 3, 3, 3, 4)
  NK_DISPATCH(32, 1, 0, 0, 4)
  NK_DISPATCH(32, 1, 1, 1, 4)
  NK_DISPATCH(16, 2, 1, 0, 1)
  NK_DISPATCH(16, 2, 1, 1, 1)
  NK_DISPATCH(16, 3, 3, 3, 1)
  NK_DISPATCH(16, 1, 0, 0, 1)
  NK_DISPATCH(16, 1, 1, 1, 1)
  NK_DISPATCH(8, 2, 1, 0, 1)
  NK_DISPATCH(8, 2, 1, 1, 1)
  NK_DISPATCH(8, 3, 3, 3, 1)
  NK_DISPATCH(8, 1, 0, 0, 1)
  NK_DISPATCH(8, 1, 1, 1, 1)
#undef NK_DISPATCH
  return cudaErrorNotSupported;
}
