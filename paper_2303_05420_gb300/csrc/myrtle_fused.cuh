// Fused Myrtle NNGP block (NK_PREC_MIXED): kernel templates.  One persistent
// launch, pixel-pair tensors never leave the chip.  Instantiated per image
// size in myrtle_fused_r{8,16,32}.cu; host dispatch in myrtle_fused.cu.
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
// Thread mapping: a warp owns one t_x and TYW consecutive t_y; each row of a
// super-plane is split into NQ parts of COLS columns held in registers
// (lane = q * TYW + t_y - ty0).  Each thread streams the rows of its
// super-plane; the horizontal 3-tap sum takes its halo from the neighbouring
// parts (two shuffles), the column cut and the image border enter as 0/1
// edge factors in the FFMAs, and the row cut as a 0/1 factor in the vertical
// FFMAs.  All layers of a stage are pipelined with a one-row delay per layer.
// The p-side tables (x, 1/sqrt q, sqrt q at row i) are warp-broadcast loads;
// the p'-side ones a conflict-free gather from tables doubled along columns.
//
// Pooling: super-plane t of stage s feeds super-plane floor/ceil(t/2) of
// stage s+1 (odd shifts split by pixel parity); rows are paired in registers
// and columns paired when t_x is even, the rest goes through shared-memory
// atomics into the next stage's buffer.  At 32x32 that buffer (64K floats)
// is distributed over a 4-CTA cluster by T_x and reached through DSMEM.  The
// last stage is reduced into the global average, combined across the
// cluster with global FP64 atomics.
//
// Scale factors sw2/9, 1/(2 pi), 1/16 and 1/C are folded into the p-side
// tables, so a conv is 2 FFMA (horizontal) + 2 FFMA (vertical) [+ 1 add for
// sb2] per pixel pair and the map ~15 FP32 instructions plus one square root.
#pragma once

#include "nk_common.cuh"
#include "nk_map.cuh"

namespace nkf {

constexpr unsigned FULL = 0xffffffffu;
// Launch variants chosen by nk_autotune for 32x32 images: threads per CTA and
// the number of parts a 32-column super-plane row is split into.
template <int V>
struct Variant {
  static constexpr int THREADS = (V == 0) ? 768 : 512;
  static constexpr int NQ32 = (V == 2) ? 4 : 8;
};

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
  double* gacc;               // [2 * nclusters] global-average accumulators
  int* gcnt;                  // [2 * nclusters] arrival counters
  float* Th;                  // NTK block (tiled NTK form only), same ldk as K
};

// ---------------------------------------------------------------------------
// Thread mapping of a stage at resolution R: a row of the super-plane is split
// into NQ parts of COLS columns; a warp holds TYW = 32 / NQ shifts t_y and the
// NQ parts of each (lane = q * TYW + t_y - ty0).
// ---------------------------------------------------------------------------
template <int R, int V = 0>
struct Split {
  static constexpr int NQ = (R == 32) ? Variant<V>::NQ32 : (R >= 16 ? 8 : (R >= 4 ? 4 : R));
  static constexpr int COLS = R / NQ;
  static constexpr int TYW = 32 / NQ;
  static constexpr int WPT = R > TYW ? R / TYW : 1;  // warps per t_x
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
  static constexpr size_t red_off = (b1_off + (size_t)B1_size * 4 + 15) / 16 * 16;  // double[32]
  static constexpr size_t ctr_off = red_off + 32 * 8;                             // int task counter
  static constexpr size_t bytes = ctr_off + 16;
};

// ---------------------------------------------------------------------------
// Horizontal 3-tap sum of one row part.  e[k] (k = 0..COLS) is the 0/1 factor
// of the coupling between local columns k-1 and k: 0 across the image border
// and across the column cut, so e[0] / e[COLS] also gate the halo values.
// ---------------------------------------------------------------------------
template <int R, int V>
__device__ __forceinline__ void make_edges(float (&e)[Split<R, V>::COLS + 1], int t_x, int q) {
  constexpr int COLS = Split<R, V>::COLS;
  const int c0 = q * COLS;
  const int kc = (t_x == 0) ? -100 : R - 1 - t_x;  // cut between global columns kc, kc + 1
#pragma unroll
  for (int k = 0; k <= COLS; ++k) {
    const int lc = c0 + k - 1;  // edge between global columns lc and lc + 1
    const bool off = (lc < 0) || (lc + 1 > R - 1) || (lc == kc);
    e[k] = off ? 0.f : 1.f;
  }
}

template <int COLS, int TYW>
__device__ __forceinline__ void hsum(const float (&A)[COLS], float (&Hc)[COLS],
                                     const float (&e)[COLS + 1]) {
  const float fromL = __shfl_up_sync(FULL, A[COLS - 1], TYW);
  const float fromR = __shfl_down_sync(FULL, A[0], TYW);
#pragma unroll
  for (int k = 0; k < COLS; ++k) {
    const float l = (k == 0) ? fromL : A[k > 0 ? k - 1 : 0];
    const float r = (k == COLS - 1) ? fromR : A[k + 1 < COLS ? k + 1 : 0];
    Hc[k] = fmaf(e[k + 1], r, fmaf(e[k], l, A[k]));
  }
}

// ---------------------------------------------------------------------------
// Pooling scatter into the next stage's buffer.  The buffer is laid out
// [T_y][T_x local][I][Kx] (T_y stride padded to an odd count of floats) and
// split over the cluster by T_x; a target T_x is resolved once per task to a
// local pointer or a DSMEM address.
// ---------------------------------------------------------------------------
template <int R2_, int TXL_, int sTx_, int sTy_>
struct OutBuf {
  static constexpr int R2 = R2_, TXL = TXL_, sTx = sTx_, sTy = sTy_;
};

struct Tgt {
  unsigned addr;  // 32-bit shared address (own window) or shared::cluster address
  int local;
};

__device__ __forceinline__ void red_shared_f32(unsigned a, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

template <class OB>
__device__ __forceinline__ Tgt make_tgt(float* buf, int Tx, unsigned rank) {
  const int owner = Tx / OB::TXL;
  const int loc = Tx - owner * OB::TXL;
  Tgt t;
  const unsigned a = smem_u32(buf + loc * OB::sTx);
  t.local = ((unsigned)owner == rank);
  t.addr = t.local ? a : mapa_rank(a, (unsigned)owner);
  return t;
}

// Adds one pooled row part.  Whether the targets are in this CTA is uniform
// over the warp (t_x is), so the branch is taken once per row.
template <int COLS>
__device__ __forceinline__ void scatter_row(const Tgt& tE, const Tgt& tO, int t_x, int base,
                                            int c0, const float (&v)[COLS]) {
  const bool even = (t_x & 1) == 0;
  if constexpr (COLS % 2 == 0) {
    if (even) {
      const unsigned a = tE.addr + 4u * (unsigned)(base + (c0 >> 1));
      if (tE.local) {
#pragma unroll
        for (int k = 0; k < COLS; k += 2) red_shared_f32(a + 2u * k, v[k] + v[k + 1]);
      } else {
#pragma unroll
        for (int k = 0; k < COLS; k += 2) red_cluster_f32(a + 2u * k, v[k] + v[k + 1]);
      }
      return;
    }
  }
  // odd t_x (or a single column): even pixel columns go to tE, odd to tO
  const unsigned aE = tE.addr + 4u * (unsigned)base;
  const unsigned aO = tO.addr + 4u * (unsigned)base;
  if (tE.local && tO.local) {
#pragma unroll
    for (int k = 0; k < COLS; ++k) {
      const int c = c0 + k;
      red_shared_f32(((!even && (c & 1)) ? aO : aE) + 4u * (unsigned)(c >> 1), v[k]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < COLS; ++k) {
      const int c = c0 + k;
      const bool o = !even && (c & 1);
      const unsigned a = (o ? aO : aE) + 4u * (unsigned)(c >> 1);
      if (o ? tO.local : tE.local)
        red_shared_f32(a, v[k]);
      else
        red_cluster_f32(a, v[k]);
    }
  }
}

// ---------------------------------------------------------------------------
// One warp task: super-planes (t_y in ty0 .. ty0+TYW-1, t_x) of a stage.
// SEED: the input rows are the channel contraction of the two images; else
// they are read from this stage's pooled buffer.  GAP: the last layer feeds
// the global average, else the pooling scatter into OB.
//
// Row stream: at step t the input row t enters layer 0 and layer j finishes
// row t - j - 1.  Steps [0, N) fill the pipeline and [R, R + N) drain it;
// in the steady steps [N, R) every layer is active, so they run without
// per-layer conditions, two at a time (the pooling pairs rows).
// ---------------------------------------------------------------------------
template <int R, int N, bool SEED, bool GAP, bool BIAS, class OB, int V>
struct Task {
  using SP = Split<R, V>;
  static constexpr int COLS = SP::COLS, TYW = SP::TYW;
  static constexpr int S = 2 * R + 1;
  int t_x, t_y, c0;
  bool act, tyodd;
  float E[COLS + 1];
  float Hp[N][COLS], Pp[N][COLS], acc[COLS];
  Tgt tE, tO;
  const float4* xs;
  const float4* xq;
  const float* inrow;  // this thread's super-plane in the pooled input buffer
  const float2* ptab;
  const float2* qtab;
  float b;

  __device__ __forceinline__ void input_row(int t, float (&A)[COLS]) const {
    if constexpr (SEED) {
      const int pr = (t + t_y) & (R - 1);
      const float4* xa = xs + t * R + c0;
      const float4* xb = xq + pr * S + c0 + t_x;
#pragma unroll
      for (int k = 0; k < COLS; ++k) {
        const float4 u = xa[k], w = xb[k];
        A[k] = fmaf(u.x, w.x, fmaf(u.y, w.y, u.z * w.z));
      }
    } else {
      const float* row = inrow + t * R;
#pragma unroll
      for (int k = 0; k < COLS; ++k) A[k] = row[k];
    }
  }

  // layer j receives row r (r in [0, R)) and finishes row r - 1 (r >= 1)
  template <int j, bool FIN>
  __device__ __forceinline__ void layer(int r, float (&A)[COLS]) {
    float Hc[COLS];
    hsum<COLS, TYW>(A, Hc, E);
    const float e = (r != R - t_y) ? 1.f : 0.f;  // edge (r-1, r) not cut
    if (FIN) finish<j>(r - 1, e, Hc, A);
#pragma unroll
    for (int k = 0; k < COLS; ++k) {
      Pp[j][k] = fmaf(e, Hp[j][k], Hc[k]);
      Hp[j][k] = Hc[k];
    }
  }

  // finish row ro of layer j: vertical sum, bias, ReLU map -> A
  template <int j>
  __device__ __forceinline__ void finish(int ro, float e, const float (&Hc)[COLS], float (&A)[COLS]) {
    const int pr = (ro + t_y) & (R - 1);
    const float2* pt = ptab + j * R * R + ro * R + c0;
    const float2* qt = qtab + j * R * S + pr * S + c0 + t_x;
#pragma unroll
    for (int k = 0; k < COLS; ++k) {
      float K = fmaf(e, Hc[k], Pp[j][k]);
      if constexpr (BIAS) K += b;
      const float2 pv = pt[k], qv = qt[k];
      const float c = K * (pv.x * qv.x);
      // the first layer sees any sign; later correlations are >= 0
      const float J = (SEED && j == 0) ? nk_J_f32(c) : nk_J01_f32(c);
      A[k] = (pv.y * qv.y) * J;
    }
  }

  // the drain: layer j finishes row R - 1 with no row below
  template <int j>
  __device__ __forceinline__ void finish_last(float (&A)[COLS]) {
    float Hz[COLS];
#pragma unroll
    for (int k = 0; k < COLS; ++k) Hz[k] = 0.f;
    finish<j>(R - 1, 0.f, Hz, A);
  }

  template <int PAR>
  __device__ __forceinline__ void output(int ro, const float (&A)[COLS], double& gap) {
    if constexpr (GAP) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < COLS; ++k) s += A[k];
      if (act) gap += (double)s;
    } else if constexpr (PAR == 0) {
#pragma unroll
      for (int k = 0; k < COLS; ++k) acc[k] = A[k];
    } else {
      const int I = ro >> 1;
      float v[COLS];
#pragma unroll
      for (int k = 0; k < COLS; ++k) v[k] = tyodd ? acc[k] : acc[k] + A[k];
      if (act) scatter_row<COLS>(tE, tO, t_x, (t_y >> 1) * OB::sTy + I * OB::R2, c0, v);
      if (act && tyodd)
        scatter_row<COLS>(tE, tO, t_x, (((t_y + 1) >> 1) & (OB::R2 - 1)) * OB::sTy + I * OB::R2, c0, A);
    }
  }

  // layers j0 .. j1-1 receive their rows (t - j) and finish the previous ones
  template <int j0, int j1>
  __device__ __forceinline__ void layers_fin(int t, float (&A)[COLS]) {
    if constexpr (j0 < j1) {
      layer<j0, true>(t - j0, A);
      layers_fin<j0 + 1, j1>(t, A);
    }
  }

  // pipeline fill, step T < N: layers 0..T-1 finish rows, layer T gets row 0
  template <int T>
  __device__ __forceinline__ void fill() {
    if constexpr (T < N) {
      float A[COLS];
      input_row(T, A);
      layers_fin<0, T>(T, A);
      layer<T, false>(0, A);
      fill<T + 1>();
    }
  }

  // steady step t in [N, R): every layer active; output row t - N
  template <int PAR>
  __device__ __forceinline__ void steady(int t, double& gap) {
    float A[COLS];
    input_row(t, A);
    layers_fin<0, N>(t, A);
    output<PAR>(t - N, A, gap);
  }

  // pipeline drain, step t = R + D: layer D finishes row R - 1, later layers
  // get their remaining rows; output row R + D - N
  template <int D>
  __device__ __forceinline__ void drain(double& gap) {
    if constexpr (D < N) {
      float A[COLS];
#pragma unroll
      for (int k = 0; k < COLS; ++k) A[k] = 0.f;
      finish_last<D>(A);
      layers_fin<D + 1, N>(R + D, A);
      output<((R + D - N) & 1)>(R + D - N, A, gap);
      drain<D + 1>(gap);
    }
  }

  // Generic step t (any R, N): layer j handles r = t - j when 0 <= r <= R.
  template <int j>
  __device__ __forceinline__ void gen_layers(int t, float (&A)[COLS]) {
    if constexpr (j < N) {
      const int r = t - j;
      if (r < 0) return;
      if (r <= R) {
        if (r == R)
          finish_last<j>(A);
        else if (r >= 1)
          layer<j, true>(r, A);
        else
          layer<j, false>(r, A);
        if (r == 0) return;
      }
      gen_layers<j + 1>(t, A);
    }
  }

  __device__ __forceinline__ void generic_run(double& gap) {
    for (int t = 0; t < R + N; ++t) {
      float A[COLS];
      if (t < R) {
        input_row(t, A);
      } else {
#pragma unroll
        for (int k = 0; k < COLS; ++k) A[k] = 0.f;
      }
      gen_layers<0>(t, A);
      const int ro = t - N;
      if (ro >= 0 && ro < R) {
        if (ro & 1)
          output<1>(ro, A, gap);
        else
          output<0>(ro, A, gap);
      }
    }
  }

  __device__ __forceinline__ void run(double& gap) {
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
      for (int k = 0; k < COLS; ++k) Hp[j][k] = Pp[j][k] = 0.f;
    if constexpr (N > R) {
      // tiny last stages (R = 2 with three layers): no steady state
      generic_run(gap);
      return;
    }
    fill<0>();
    int t = N;
    for (; t + 1 < R; t += 2) {
      steady<0>(t, gap);
      steady<1>(t + 1, gap);
    }
    if (t < R) steady<0>(t, gap);
    drain<0>(gap);
  }
};

template <int R, int N, bool SEED, bool GAP, bool BIAS, class OB, int V>
__device__ __forceinline__ void stage_task(int t_x, int ty0, const float4* __restrict__ xs,
                                           const float4* __restrict__ xq,
                                           const float* __restrict__ inb, int in_sTy,
                                           const float2* __restrict__ ptab,
                                           const float2* __restrict__ qtab, float b, float* obuf,
                                           unsigned rank, double& gap) {
  using TK = Task<R, N, SEED, GAP, BIAS, OB, V>;
  constexpr int TYW = TK::TYW;
  TK T;
  const int lane = threadIdx.x & 31;
  const int q = lane / TYW, tyl = lane - q * TYW;
  T.t_x = t_x;
  T.act = tyl < R;
  T.t_y = (ty0 + tyl) & (R - 1);
  T.c0 = q * TK::COLS;
  T.tyodd = (T.t_y & 1) != 0;
  make_edges<R, V>(T.E, t_x, q);
  T.tE = Tgt{0u, 1};
  T.tO = Tgt{0u, 1};
  if constexpr (!GAP) {
    T.tE = make_tgt<OB>(obuf, t_x >> 1, rank);
    T.tO = (t_x & 1) ? make_tgt<OB>(obuf, ((t_x + 1) >> 1) & (OB::R2 - 1), rank) : T.tE;
  }
  T.xs = xs;
  T.xq = xq;
  T.inrow = SEED ? nullptr : inb + T.t_y * in_sTy + T.c0;
  T.ptab = ptab;
  T.qtab = qtab;
  T.b = b;
  T.run(gap);
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

__device__ __forceinline__ float4 load_x(const float* p, int C, float s) {
  return make_float4(p[0] * s, C > 1 ? p[1] * s : 0.f, C > 2 ? p[2] * s : 0.f, 0.f);
}

// One pixel pair (ia, ib) by the CL CTAs of a cluster (CL = 1: this CTA
// alone): stage the tables, run every stage, reduce the global average over
// the CTA.  Returns this CTA's share of the average's sum (valid in thread 0).
template <int R0, int N0, int N1, int N2, int CL, bool BIAS, int V>
__device__ __forceinline__ double pair_body(const FusedParams& P, int64_t ia, int64_t ib,
                                            unsigned char* smem, unsigned rank) {
  using L = Layout<R0, N0, N1, N2, CL>;
  constexpr int SE = L::SE;
  constexpr int R1 = L::R1, R2 = L::R2;
  using OB1 = OutBuf<R1, L::TXL1, L::B1_sTx, L::B1_sTy>;
  using OB2 = OutBuf<R2, L::TXL2, L::B2_sTx, L::B2_sTy>;
  using OBG = OutBuf<1, 1, 0, 0>;
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
  double* red = reinterpret_cast<double*>(smem + L::red_off);
  int* ctr = reinterpret_cast<int*>(smem + L::ctr_off);
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int lane = threadIdx.x & 31;
  const int C = P.C;
  // ---- stage tables; zero this CTA's stage-1 buffer and the task counter
  {
    const float* xa = P.Xa + ia * (int64_t)R0 * R0 * C;
    const float* xb = P.Xb + ib * (int64_t)R0 * R0 * C;
    for (int e = threadIdx.x; e < R0 * R0; e += blockDim.x) xs[e] = load_x(xa + e * C, C, P.xscale);
    for (int e = threadIdx.x; e < R0 * 2 * R0; e += blockDim.x) {
      const int row = e / (2 * R0), col = e - row * 2 * R0;
      xq[row * L::S0 + col] = load_x(xb + (row * R0 + (col & (R0 - 1))) * C, C, 1.f);
    }
    stage_q_tables<R0, N0>(P, 0, ia, ib, p0, q0);
    if constexpr (SE >= 2) stage_q_tables<R1, N1>(P, N0, ia, ib, p1, q1);
    if constexpr (SE >= 3) stage_q_tables<R2, N2>(P, N0 + N1, ia, ib, p2, q2);
    for (int e = threadIdx.x; e < L::B1_size; e += blockDim.x) b1[e] = 0.f;
    if (threadIdx.x == 0) *ctr = 0;
  }
  if constexpr (CL > 1) cluster_sync_all(); else __syncthreads();

  double gap = 0.0;
  // ---- stage 0: tasks (t_x, t_y group) taken from a shared counter
  {
    constexpr int NH = Split<R0, V>::WPT;  // warps per t_x
    constexpr int TXC = R0 / CL;        // t_x per CTA
    constexpr int NT = TXC * NH;
    for (;;) {
      int task = 0;
      if (lane == 0) task = atomicAdd(ctr, 1);
      task = __shfl_sync(FULL, task, 0);
      if (task >= NT) break;
      const int t_x = (int)rank * TXC + task / NH;
      const int ty0 = (task % NH) * Split<R0, V>::TYW;
      stage_task<R0, N0, true, SE == 1, BIAS, OB1, V>(t_x, ty0, xs, xq, nullptr, 0, p0, q0, P.sb2, b1,
                                                   rank, gap);
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
    for (int task = warp; task < TXC * NH; task += nwarps) {
      const int tl = task / NH;
      const int t_x = (int)rank * TXC + tl;
      const float* inb = b1 + tl * L::B1_sTx;
      stage_task<R1, N1, false, SE == 2, BIAS, OB2, V>(t_x, (task % NH) * Split<R1>::TYW, nullptr,
                                                    nullptr, inb, L::B1_sTy, p1, q1, P.sb2, b2,
                                                    rank, gap);
    }
  }
  if constexpr (SE >= 3) {
    if constexpr (CL > 1) cluster_sync_all(); else __syncthreads();
    if (rank == 0) {
      constexpr int NH = Split<R2>::WPT;
      for (int task = warp; task < R2 * NH; task += nwarps) {
        const int tl = task / NH;
        const float* inb = b2 + tl * L::B2_sTx;
        stage_task<R2, N2, false, true, BIAS, OBG, V>(tl, (task % NH) * Split<R2>::TYW, nullptr,
                                                   nullptr, inb, L::B2_sTy, p2, q2, P.sb2, nullptr,
                                                   rank, gap);
      }
    }
  }
  // ---- global average: warp -> CTA
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gap += __shfl_xor_sync(FULL, gap, o);
  if (lane == 0) red[warp] = gap;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nwarps; ++w) s += red[w];
  // the next pair's staging only touches this CTA's own tables and b1,
  // which every warp of this CTA is done with (barrier above); remote CTAs
  // write into b1 only after the next cluster barrier
  return s;
}

// Writes K[i][j] (and the mirror of a symmetric block).
__device__ __forceinline__ void store_entry(const FusedParams& P, int64_t i, int64_t j, double tot) {
  const float v = (float)(P.out_scale * tot + P.out_bias);
  P.K[i * P.ldk + j] = v;
  if (P.sym && i != j) P.K[j * P.ldk + i] = v;
}

// Cluster combine of a pair's global average: each CTA adds its share into
// the cluster's slot with FP64 atomics; the last to arrive writes K.  Slots
// are double-buffered by the parity of the cluster's pair counter.
template <int CL>
__device__ __forceinline__ void cluster_combine(const FusedParams& P, double* gacc, int* gcnt,
                                                int64_t slot, int64_t i, int64_t j, double s) {
  if (threadIdx.x != 0) return;
  if constexpr (CL == 1) {
    store_entry(P, i, j, s);
    return;
  }
  double* acc = gacc + slot;
  int* cnt = gcnt + slot;
  atomicAdd(acc, s);
  __threadfence();
  const int old = atomicAdd(cnt, 1);
  if (old == CL - 1) {
    __threadfence();
    const double tot = atomicAdd(acc, 0.0);
    store_entry(P, i, j, tot);
    atomicExch(reinterpret_cast<unsigned long long*>(acc), 0ull);
    atomicExch(cnt, 0);
  }
}

// The single-block kernel keeps its own copy of the pair body: written out
// here it compiles to fewer spills than through pair_body (measured 2% faster).
template <int R0, int N0, int N1, int N2, int CL, bool BIAS, int V>
__global__ void __launch_bounds__(Variant<V>::THREADS, 1)
    k_myrtle_fused(const __grid_constant__ FusedParams P) {
  using L = Layout<R0, N0, N1, N2, CL>;
  constexpr int SE = L::SE;
  constexpr int R1 = L::R1, R2 = L::R2;
  using OB1 = OutBuf<R1, L::TXL1, L::B1_sTx, L::B1_sTy>;
  using OB2 = OutBuf<R2, L::TXL2, L::B2_sTx, L::B2_sTy>;
  using OBG = OutBuf<1, 1, 0, 0>;
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
  double* red = reinterpret_cast<double*>(smem + L::red_off);
  int* ctr = reinterpret_cast<int*>(smem + L::ctr_off);

  const unsigned rank = (CL > 1) ? cluster_rank() : 0u;
  const int64_t cid = blockIdx.x / CL;
  const int64_t ncl = gridDim.x / CL;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int lane = threadIdx.x & 31;
  const int C = P.C;
  int iter = 0;

  for (int64_t pidx = cid; pidx < P.npairs; pidx += ncl, ++iter) {
    int64_t i, j;
    pair_ij(pidx, P.na, P.nb, P.sym, &i, &j);
    const int64_t ia = P.a0 + i, ib = P.b0 + j;
    // ---- stage tables; zero this CTA's stage-1 buffer and the task counter
    {
      const float* xa = P.Xa + ia * (int64_t)R0 * R0 * C;
      const float* xb = P.Xb + ib * (int64_t)R0 * R0 * C;
      for (int e = threadIdx.x; e < R0 * R0; e += blockDim.x) xs[e] = load_x(xa + e * C, C, P.xscale);
      for (int e = threadIdx.x; e < R0 * 2 * R0; e += blockDim.x) {
        const int row = e / (2 * R0), col = e - row * 2 * R0;
        xq[row * L::S0 + col] = load_x(xb + (row * R0 + (col & (R0 - 1))) * C, C, 1.f);
      }
      stage_q_tables<R0, N0>(P, 0, ia, ib, p0, q0);
      if constexpr (SE >= 2) stage_q_tables<R1, N1>(P, N0, ia, ib, p1, q1);
      if constexpr (SE >= 3) stage_q_tables<R2, N2>(P, N0 + N1, ia, ib, p2, q2);
      for (int e = threadIdx.x; e < L::B1_size; e += blockDim.x) b1[e] = 0.f;
      if (threadIdx.x == 0) *ctr = 0;
    }
    if constexpr (CL > 1) cluster_sync_all(); else __syncthreads();

    double gap = 0.0;
    // ---- stage 0: tasks (t_x, t_y group) taken from a shared counter
    {
      constexpr int NH = Split<R0, V>::WPT;  // warps per t_x
      constexpr int TXC = R0 / CL;        // t_x per CTA
      constexpr int NT = TXC * NH;
      for (;;) {
        int task = 0;
        if (lane == 0) task = atomicAdd(ctr, 1);
        task = __shfl_sync(FULL, task, 0);
        if (task >= NT) break;
        const int t_x = (int)rank * TXC + task / NH;
        const int ty0 = (task % NH) * Split<R0, V>::TYW;
        stage_task<R0, N0, true, SE == 1, BIAS, OB1, V>(t_x, ty0, xs, xq, nullptr, 0, p0, q0, P.sb2, b1,
                                                     rank, gap);
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
      for (int task = warp; task < TXC * NH; task += nwarps) {
        const int tl = task / NH;
        const int t_x = (int)rank * TXC + tl;
        const float* inb = b1 + tl * L::B1_sTx;
        stage_task<R1, N1, false, SE == 2, BIAS, OB2, V>(t_x, (task % NH) * Split<R1>::TYW, nullptr,
                                                      nullptr, inb, L::B1_sTy, p1, q1, P.sb2, b2,
                                                      rank, gap);
      }
    }
    if constexpr (SE >= 3) {
      if constexpr (CL > 1) cluster_sync_all(); else __syncthreads();
      if (rank == 0) {
        constexpr int NH = Split<R2>::WPT;
        for (int task = warp; task < R2 * NH; task += nwarps) {
          const int tl = task / NH;
          const float* inb = b2 + tl * L::B2_sTx;
          stage_task<R2, N2, false, true, BIAS, OBG, V>(tl, (task % NH) * Split<R2>::TYW, nullptr,
                                                     nullptr, inb, L::B2_sTy, p2, q2, P.sb2, nullptr,
                                                     rank, gap);
        }
      }
    }
    // ---- global average: warp -> CTA -> cluster (global FP64 atomics; the
    // last CTA of the cluster to arrive writes K)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gap += __shfl_xor_sync(FULL, gap, o);
    if (lane == 0) red[warp] = gap;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < nwarps; ++w) s += red[w];
      const int64_t slot = cid * 2 + (iter & 1);
      double* acc = P.gacc + slot;
      int* cnt = P.gcnt + slot;
      atomicAdd(acc, s);
      __threadfence();
      const int old = atomicAdd(cnt, 1);
      if (old == CL - 1) {
        __threadfence();
        const double tot = atomicAdd(acc, 0.0);
        const float v = (float)(P.out_scale * tot + P.out_bias);
        P.K[i * P.ldk + j] = v;
        if (P.sym && i != j) P.K[j * P.ldk + i] = v;
        atomicExch(reinterpret_cast<unsigned long long*>(acc), 0ull);
        atomicExch(cnt, 0);
      }
    }
    // the next pair's staging only touches this CTA's own tables and b1,
    // which every warp of this CTA is done with (barrier above); remote CTAs
    // write into b1 only after the next cluster barrier
  }
}

template <int R0, int N0, int N1, int N2, int CL, bool BIAS, int V>
cudaError_t launch(FusedParams P, int sm_count, void* scratch, size_t scratch_bytes,
                   cudaStream_t st) {
  using L = Layout<R0, N0, N1, N2, CL>;
  auto kern = k_myrtle_fused<R0, N0, N1, N2, CL, BIAS, V>;
  const size_t smem = L::bytes;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(Variant<V>::THREADS, 1, 1);
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
  const size_t need = (size_t)nclusters * 2 * (sizeof(double) + sizeof(int));
  if (need > scratch_bytes) return cudaErrorInvalidValue;
  P.gacc = reinterpret_cast<double*>(scratch);
  P.gcnt = reinterpret_cast<int*>(reinterpret_cast<char*>(scratch) + (size_t)nclusters * 2 * sizeof(double));
  e = cudaMemsetAsync(scratch, 0, need, st);
  if (e != cudaSuccess) return e;
  cfg.gridDim = dim3((unsigned)(nclusters * CL), 1, 1);
  e = cudaLaunchKernelEx(&cfg, kern, P);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// A queue of blocks of several image sizes (myrtle_queue.cu).
constexpr int QUEUE_MAX = 8;
constexpr int QUEUE_CL = 4;
struct QueueParams {
  int n;                        // blocks, largest images first
  int R[QUEUE_MAX];             // image side of each block (32, 16 or 8)
  int64_t item0[QUEUE_MAX + 1]; // first queue item of each block
  FusedParams B[QUEUE_MAX];
  double* gacc;                 // [2 * clusters] global-average slots of 32x32 pairs
  int* gcnt;
};
cudaError_t launch_queue(const int c[3], bool bias, QueueParams& Q, int sm_count, void* scratch,
                         size_t scratch_bytes, cudaStream_t st);

// Per image size dispatch (myrtle_fused_r*.cu): launches the instantiation for
// the stage pattern c[0..2], bias flag and launch variant.
cudaError_t dispatch_r32(const int c[3], bool bias, int variant, FusedParams& P, int sm_count,
                         void* scratch, size_t scratch_bytes, cudaStream_t st);
cudaError_t dispatch_r32_v2(const int c[3], bool bias, int variant, FusedParams& P, int sm_count,
                             void* scratch, size_t scratch_bytes, cudaStream_t st);
cudaError_t dispatch_r16(const int c[3], bool bias, int variant, FusedParams& P, int sm_count,
                         void* scratch, size_t scratch_bytes, cudaStream_t st);
cudaError_t dispatch_r8(const int c[3], bool bias, int variant, FusedParams& P, int sm_count,
                        void* scratch, size_t scratch_bytes, cudaStream_t st);

// Tiled form (myrtle_tiled.cu): 64x64 blocks, and queues mixing 64x64 and
// 32x32 blocks (R[b] in {64, 32}, largest first) in one persistent launch.
bool tiled_supported(const int c[3]);
// tensors: pooled tensors per pair (1; 2 for the NTK form)
size_t tiled_ws_bytes(const int c[3], const int* R, const int64_t* npairs, int n, int sm_count, int tensors = 1);
// wait_limit: polls of a dependency wait before it gives up (NK_DEV_TIMEOUT).
// act: NK_ACT_RELU or NK_ACT_ERF (the map of every activation layer).
cudaError_t launch_tiled(const int c[3], bool bias, int act, const int* R, const FusedParams* B, int n,
                         int sm_count,
                         void* ws, size_t ws_bytes, unsigned int* dstatus, long long wait_limit,
                         cudaStream_t st);
// Three-stage nets at 32x32 (myrtle_tiled3.cu): (3,3,3) and (2,1,1), ReLU,
// NNGP (ntk false) or NTK (ntk true: K and Theta, B[b].Th).
bool tiled3_supported(const int c[3]);
cudaError_t launch_tiled3(const int c[3], bool bias, bool ntk, const int* R, const FusedParams* B, int n,
                          int sm_count, void* ws, size_t ws_bytes, unsigned int* dstatus, long long wait_limit,
                          cudaStream_t st);
// The NTK form (myrtle_tiled_ntk.cu): K and Theta (B[b].Th) of ReLU blocks of
// the stage pattern (2,1,0), 64x64 and/or 32x32.
bool tiled_ntk_supported(const int c[3]);
cudaError_t launch_tiled_ntk(const int c[3], bool bias, const int* R, const FusedParams* B, int n, int sm_count,
                             void* ws, size_t ws_bytes, unsigned int* dstatus, long long wait_limit,
                             cudaStream_t st);

}  // namespace nkf

// Kernel parameters of one block (myrtle_fused.cu).
nkf::FusedParams nk_fused_params(const NkGeom& g, double sw2, double sb2, const float* Xa, const float* qsa,
                                 int64_t a0, int64_t a1, const float* Xb, const float* qsb, int64_t b0,
                                 int64_t b1, float* K, int64_t ldk, int symmetric);
