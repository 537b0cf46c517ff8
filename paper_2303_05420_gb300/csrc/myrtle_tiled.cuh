// Tiled fused Myrtle NNGP blocks (NK_PREC_MIXED) for 64x64 images, and for
// queues that mix 64x64 and 32x32 blocks in one persistent launch: the kernel
// templates (instantiated per activation by myrtle_tiled.cu, ReLU, and
// myrtle_tiled_erf.cu, Erf).
//
// Same arithmetic as the super-plane kernel (myrtle_fused.cuh): K_1 from the
// channel contraction, the diagonal 3x3 stencil streamed along the rows of a
// super-plane t = (t_y, t_x) (pairs (p, p') with p' = (p + t) mod R), the
// arc-cosine ReLU map with the scale factors folded into the p-side tables,
// 2x2 pooling into the next stage's super-planes, and the global average.
//
// What changes at 64x64: the pooled stage-1 tensor holds R1^4 = 32^4 floats
// (4 MB) per pair and the per-pair tables of both images (x and the per-layer
// self-variances of the 64x64 stage) no longer fit one CTA's shared memory.
// So a pair is cut into independent stage-0 tasks and one stage-1 task:
//
//  * stage-0 task = (row band of B = 32 rows, group of TY = 16 shifts t_y,
//    group of TX = 8 shifts t_x), 64 or 32 warp tasks of one t_x each.  A
//    band streams its rows plus N0 halo rows on each inner side (the halo
//    outputs are recomputed, not exchanged); the p-side tables cover the
//    band's rows, the p'-side tables the window of rows (r + t_y) mod R and
//    columns (c + t_x) mod R it touches.  At 64x64 with two stage-0 layers
//    the tables take 198 KB; 64 tasks a pair.
//  * the pooled output goes into a per-pair slot in global memory (L2
//    resident: a ring of S slots) by vector atomic adds; rows are paired in
//    registers, columns too when t_x is even.
//  * stage-1 task = the whole R1 = 32 stage of the pair on one CTA, rows read
//    from the slot (L2, bypassing L1) and cleared for the slot's next pair,
//    the last layer reduced into the global average and K written.
//
// Scheduling (tiled_schedule.h): one or two persistent CTAs per SM pull
// items from a global counter.  The items are the stage-0 tasks of every
// pair, block by block, with the stage-1 task of pair k merged in LAG
// stage-0 items (about two waves of the grid) after the last stage-0 task of
// k, so that it rarely waits for them.  The 64x64 and the 32x32 pairs each
// own a ring of S_R slots; a stage-0 task of pair g waits until the slot's
// previous user, pair g - S_R, has been cleared by its stage-1 task, which
// S_R >= LAG / (tasks per pair) + 1 puts earlier in the order (S_R = 2 LAG /
// (tasks per pair) + 2 puts it a LAG earlier, so that it is normally done).
// Every wait is on an item claimed earlier, so the earliest unfinished item
// never waits and the queue drains.  Waits are bounded: on a timeout the
// kernel raises NK_DEV_TIMEOUT and an abort flag that makes every CTA stop
// taking items.  The bound is the handle's wait limit (nk_set_wait_limit;
// 2^22 polls, seconds, by default).
#pragma once

#include <algorithm>

#include "myrtle_fused.cuh"
#include "tiled_schedule.h"

namespace nkf {
namespace tiled {

// Threads per CTA: 512 with one CTA per SM wherever 64x64 blocks are present
// (their tables take 198 KB); 256 with two CTAs per SM for 32x32-only
// launches (97 KB each), so that one CTA's table staging and barriers
// overlap the other's row streams.
constexpr int MAX_WARPS = 16;

// Stage-0 tiling at image side R: rows split into parts of four columns
// (lane = part * TYW + t_y - ty0), as in the 32x32 super-plane kernel.
template <int R>
struct G0 {
  static constexpr int COLS = 4, NQ = R / COLS, TYW = 32 / NQ;
  static constexpr int B = 32;  // rows of a band
  static constexpr int NB = R / B;
  static constexpr int TY = 16, TX = 8;
  static constexpr int NTY = R / TY, NTX = R / TX;
  static constexpr int NT0 = NB * NTY * NTX;  // stage-0 tasks per pair
  static constexpr int YW = TY / TYW;         // warps per t_x within a task
  static constexpr int WT = TX * YW;          // warp tasks per CTA task
  static constexpr int SXP = R + NQ;          // p-side row stride: one pad after each part
  static constexpr int SQ = R + TX - 1;       // p'-side window columns (odd)
  // p'-side window layout.  At 64x64 a warp holds 16 row parts (4 columns
  // apart) of 2 shifts t_y, so row-major tables put the parts' float2 / float4
  // reads on 4 (or 2) bank groups.  There the window is stored column-phase
  // major within a row, column c at (c mod 4) NPH + c / 4, so that for a fixed
  // element k a warp's parts read consecutive entries; the row strides make
  // the two t_y rows fall on the other half of the banks (float2 tables:
  // 72 = 8 mod 16 entries; x', float4: 76 = 4 mod 8).  32x32 keeps the plain
  // rows (conflict-free there).
  static constexpr bool PH = (R == 64);
  static constexpr int NPH = (SQ + 3) / 4;                  // column groups of a phased row
  static constexpr int SQQ = PH ? 4 * NPH : SQ;             // row stride of the q tables
  static constexpr int SQX = PH ? 4 * NPH + 4 : SQ;         // row stride of the x' table
  static_assert(!PH || (SQQ % 16 == 8 && SQX % 8 == 4), "phased strides");
  static_assert(R % B == 0 && COLS % 2 == 0 && SQ % 2 == 1, "tiling");
  static_assert(NT0 == sched::tasks_per_pair(R), "task count of the item order (tiled_schedule.h)");
};

template <int R, int N>
struct L0 {
  using G = G0<R>;
  static constexpr int HALO = (G::NB > 2 ? 2 : (G::NB == 2 ? 1 : 0)) * N;
  static constexpr int NRP = G::B + HALO;  // streamed rows of a band (at most)
  static constexpr int NRQ = NRP + G::TY - 1;
  static constexpr int PL = NRP * G::SXP;  // p-side layer stride (elements)
  static constexpr int QL = NRQ * G::SQQ;  // p'-side layer stride of the q tables
  static constexpr int QLX = NRQ * G::SQX; // p'-side x' table
  static constexpr size_t xs_off = 0;
  static constexpr size_t xq_off = xs_off + (size_t)PL * 16;
  static constexpr size_t p_off = xq_off + (size_t)QLX * 16;
  static constexpr size_t q_off = p_off + (size_t)N * PL * 8;
  static constexpr size_t bytes = q_off + (size_t)N * QL * 8;
};

// Stage-1 tables at side R1 (full images, p' side doubled along columns).
template <int R1, int N>
struct L1 {
  static constexpr int S = 2 * R1 + 1;
  static constexpr int PL = R1 * R1, QL = R1 * S;
  static constexpr size_t p_off = 0;
  static constexpr size_t q_off = (size_t)N * PL * 8;
  static constexpr size_t bytes = q_off + (size_t)N * QL * 8;
};

struct TiledParams {
  int n;                          // blocks, 64x64 first
  int R[QUEUE_MAX];               // image side of each block (64 or 32)
  int nt0[QUEUE_MAX];             // stage-0 tasks per pair of each block
  int64_t g0[QUEUE_MAX + 1];      // first pair index of each block
  int64_t f0[QUEUE_MAX + 1];      // first stage-0 task index of each block
  FusedParams B[QUEUE_MAX];
  int64_t G;                      // pairs
  int64_t G64;                    // pairs of 64x64 blocks (they come first)
  int64_t T0;                     // stage-0 tasks
  int64_t nitems;                 // T0 + G (stage 1 of two-stage nets) or T0
  int64_t LAG;                    // stage-0 tasks between a pair's last one and its stage-1 task
  int S[2];                       // slot rings of the 64x64 and the 32x32 pairs
  int64_t ring_off[2];            // first float of each ring
  int64_t slot_floats[2];         // (R / 2)^4
  float* slots;
  int* cnt0;                      // [G] finished stage-0 tasks
  int* done1;                     // [G] stage 1 finished (slot cleared)
  double* gacc;                   // [G] global-average sums (single-stage nets)
  unsigned long long* next;       // item counter
  int* abort_flag;
  unsigned int* dstatus;
  long long wait_limit;           // polls (~0.25-1 us each) before a wait gives up
};

__device__ __forceinline__ void red_v4(float* a, float x, float y, float z, float w) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(a), "f"(x), "f"(y), "f"(z), "f"(w)
               : "memory");
}
__device__ __forceinline__ void red_v2(float* a, float x, float y) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(a), "f"(x), "f"(y) : "memory");
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0: waits until *p >= v.  False on abort or timeout (which raises
// the abort flag and NK_DEV_TIMEOUT).
__device__ inline bool wait_geq(const TiledParams& Q, const int* p, int v) {
  for (long long it = 0;; ++it) {
    if (ld_acquire(p) >= v) return true;
    if (*(volatile int*)Q.abort_flag) return false;
    if (it > Q.wait_limit) {
      atomicOr(Q.dstatus, NK_DEV_TIMEOUT);
      atomicExch(Q.abort_flag, 1);
      return false;
    }
    __nanosleep(256);
  }
}

// Loads COLS consecutive floats of a slot row (L2 only) and clears them.
// SH: the row is in this CTA's shared memory (the stage-2 tile of a
// three-stage net, cleared before each stage-1 task): plain loads.
template <int COLS, bool SH = false>
__device__ __forceinline__ void take_row(float* p, float (&v)[COLS]) {
  if constexpr (SH) {
#pragma unroll
    for (int k = 0; k < COLS; ++k) v[k] = p[k];
  } else if constexpr (COLS == 4) {
    const float4 u = __ldcg(reinterpret_cast<const float4*>(p));
    v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w;
    __stcg(reinterpret_cast<float4*>(p), make_float4(0.f, 0.f, 0.f, 0.f));
  } else if constexpr (COLS == 2) {
    const float2 u = __ldcg(reinterpret_cast<const float2*>(p));
    v[0] = u.x; v[1] = u.y;
    __stcg(reinterpret_cast<float2*>(p), make_float2(0.f, 0.f));
  } else {
#pragma unroll
    for (int k = 0; k < COLS; ++k) {
      v[k] = __ldcg(p + k);
      __stcg(p + k, 0.f);
    }
  }
}

// ---------------------------------------------------------------------------
// A band of rows [s0, s1) of super-planes (t_y, t_x), rows [b0, b1) output.
// Row stream as in the super-plane kernel: at step t the input row t enters
// layer 0 and layer j finishes row t - j - 1; rows before b0 are the halo
// (their outputs are discarded), and a band that ends at the image border
// drains the pipeline with the zero row below.
//   SEED: input rows are the channel contraction (stage 0), else they are
//         taken from a slot in global memory (stage 1).
//   GAP:  the last layer feeds the global average, else the pooled scatter
//         into the slot of the next stage.
//   WRAP: p'-side tables hold all rows (row index (r + t_y) mod R); else a
//         window starting at row s0 + ty0.
//   NTK:  a tangent row B (the neural tangent kernel's Theta, NTK
//         parameterisation) streams beside the NNGP row A through the same
//         stencil: a conv gives Theta = a S(Theta_t) + K (K with its bias; at
//         the first conv Theta_t = 0, so Theta = K), the ReLU gives Theta_t =
//         Theta (pi - arccos c) / (2 pi), and the layer's folded factor (a /
//         (2 pi), / 16 before a pool) scales B as it scales A, without the
//         sqrt(q q') that A's map carries.  Pools and the global average act
//         on both; the slot holds K's pooled tensor, then Theta's.
// ---------------------------------------------------------------------------
//   SHIN: input rows come from shared memory (the stage-2 tile), not a slot.
template <int R, int NQ, int N, bool SEED, bool GAP, bool BIAS, bool WRAP, int SXP, int SQ, int PL, int QL, int ACT,
          int SQX = SQ, bool PH = false, bool NTK = false, bool SHIN = false>
struct Band {
  static constexpr int COLS = R / NQ, TYW = 32 / NQ;
  static constexpr int R1 = R / 2;
  static constexpr int CT = NTK ? COLS : 1;  // tangent row width (1: unused)
  static constexpr int NTL = NTK ? N : 1;
  int t_x, t_y, c0;
  int s0, s1, b0;
  bool tyodd;
  float E[COLS + 1];
  float Hp[N][COLS], Pp[N][COLS], acc[COLS];
  float nx[COLS];       // prefetched next input row (stage 1)
  float HpT[NTL][CT], PpT[NTL][CT], accT[CT], nxT[CT];  // the tangent row's pipeline
  const float4* xs;     // p-side x, at (r - s0) * SXP + pcol
  const float4* xq;     // p'-side x'
  float* in;            // stage-1 input super-plane in its slot (row stride R)
  float* inT;           // its tangent (NTK)
  const float2* ptab;
  const float2* qtab;
  int pcol, qr0, qc;
  int qo[PH ? COLS : 1];  // phased p'-side offsets of the row part's columns
  float* slot;          // pooled output slot (stage 0 of a two-stage net)
  float* slotT;         // its tangent half (NTK)
  const float* fth;     // folded factor of each layer of this stage (NTK)
  bool dg;              // NTK: the diagonal super-plane t = (0, 0) of an image with itself
  float b;

  // the tangent row enters layer j (not the first conv of stage 0)
  template <int j>
  static constexpr bool tin() { return NTK && !(SEED && j == 0); }

  __device__ __forceinline__ int qrow(int r) const { return WRAP ? ((r + t_y) & (R - 1)) : (r + qr0); }

  __device__ __forceinline__ void input_row(int t, float (&A)[COLS], float (&B)[CT]) {
    if constexpr (SEED) {
      const float4* xa = xs + (t - s0) * SXP + pcol;
      if constexpr (PH) {
        const float4* xb = xq + qrow(t) * SQX;
#pragma unroll
        for (int k = 0; k < COLS; ++k) {
          const float4 u = xa[k], w = xb[qo[k]];
          A[k] = fmaf(u.x, w.x, fmaf(u.y, w.y, u.z * w.z));
        }
      } else {
        const float4* xb = xq + qrow(t) * SQ + qc;
#pragma unroll
        for (int k = 0; k < COLS; ++k) {
          const float4 u = xa[k], w = xb[k];
          A[k] = fmaf(u.x, w.x, fmaf(u.y, w.y, u.z * w.z));
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < COLS; ++k) A[k] = nx[k];
      if constexpr (NTK) {
#pragma unroll
        for (int k = 0; k < COLS; ++k) B[k] = nxT[k];
      }
      if (t + 1 < R) {
        take_row<COLS, SHIN>(in + (t + 1) * R, nx);
        if constexpr (NTK) take_row<COLS, SHIN>(inT + (t + 1) * R, nxT);
      }
    }
  }

  template <int j, bool FIN>
  __device__ __forceinline__ void layer(int r, float (&A)[COLS], float (&B)[CT]) {
    float Hc[COLS], HcT[CT];
    hsum<COLS, TYW>(A, Hc, E);
    if constexpr (tin<j>()) hsum<COLS, TYW>(B, HcT, E);
    const float e = (r != R - t_y) ? 1.f : 0.f;
    if (FIN) finish<j>(r - 1, e, Hc, HcT, A, B);
#pragma unroll
    for (int k = 0; k < COLS; ++k) {
      Pp[j][k] = fmaf(e, Hp[j][k], Hc[k]);
      Hp[j][k] = Hc[k];
    }
    if constexpr (tin<j>()) {
#pragma unroll
      for (int k = 0; k < COLS; ++k) {
        PpT[j][k] = fmaf(e, HpT[j][k], HcT[k]);
        HpT[j][k] = HcT[k];
      }
    }
  }

  template <int j>
  __device__ __forceinline__ void finish(int ro, float e, const float (&Hc)[COLS], const float (&HcT)[CT],
                                         float (&A)[COLS], float (&B)[CT]) {
    const float2* pt = ptab + j * PL + (ro - s0) * SXP + pcol;
    const float2* qt = qtab + j * QL + qrow(ro) * SQ + (PH ? 0 : qc);
#pragma unroll
    for (int k = 0; k < COLS; ++k) {
      float K = fmaf(e, Hc[k], Pp[j][k]);
      if constexpr (BIAS) K += b;
      const float2 pv = pt[k], qv = PH ? qt[qo[k]] : qt[k];
      const float c = K * (pv.x * qv.x);
      float J;
      if constexpr (ACT == NK_ACT_ERF)
        J = nk_asin_f32(c);  // Erf: (2/pi) asin(c), 2/pi folded into the p side
      else
        J = (SEED && j == 0) ? nk_J_f32(c) : nk_J01_f32(c);
      const float sq = pv.y * qv.y;
      A[k] = sq * J;
      if constexpr (NTK) {
        float T = K;
        if constexpr (tin<j>()) T += fmaf(e, HcT[k], PpT[j][k]);
        // pi - arccos c; a zero self-variance on either side gives a zero
        // derivative kernel.  Its slope is infinite at c = 1, where an FP32
        // c short of 1 by d moves it by sqrt(2 d); the pixel pairs (p, p) of
        // an image with itself have c = 1 exactly and take pi.
        const float dJ = (sq != 0.f) ? (dg ? NK_PI_F : NK_HALF_PI_F + nk_asin_f32(c)) : 0.f;
        B[k] = (T * dJ) * fth[j];
      }
    }
  }

  template <int j>
  __device__ __forceinline__ void finish_last(float (&A)[COLS], float (&B)[CT]) {
    float Hz[COLS], HzT[CT];
#pragma unroll
    for (int k = 0; k < COLS; ++k) Hz[k] = 0.f;
#pragma unroll
    for (int k = 0; k < CT; ++k) HzT[k] = 0.f;
    finish<j>(R - 1, 0.f, Hz, HzT, A, B);
  }

  // pooled scatter of one row part into super-plane row (Ty, I) of a slot
  // tensor at `base`
  __device__ __forceinline__ void scatter(float* base, int Ty, int I, const float (&v)[COLS]) const {
    float* aE = base + ((size_t)(Ty * R1 + (t_x >> 1)) * R1 + I) * R1 + (c0 >> 1);
    if (!(t_x & 1)) {
      if constexpr (COLS == 8) {
        red_v4(aE, v[0] + v[1], v[2] + v[3], v[4] + v[5], v[6] + v[7]);
      } else if constexpr (COLS == 4) {
        red_v2(aE, v[0] + v[1], v[2] + v[3]);
      } else {
#pragma unroll
        for (int k = 0; k < COLS; k += 2) atomicAdd(aE + k / 2, v[k] + v[k + 1]);
      }
    } else {
      // even pixel columns keep T_x = t_x >> 1, odd ones go to the next T_x
      float* aO = base + ((size_t)(Ty * R1 + (((t_x + 1) >> 1) & (R1 - 1))) * R1 + I) * R1 + (c0 >> 1);
      if constexpr (COLS == 8) {
        red_v4(aE, v[0], v[2], v[4], v[6]);
        red_v4(aO, v[1], v[3], v[5], v[7]);
      } else if constexpr (COLS == 4) {
        red_v2(aE, v[0], v[2]);
        red_v2(aO, v[1], v[3]);
      } else {
#pragma unroll
        for (int k = 0; k < COLS; k += 2) {
          atomicAdd(aE + k / 2, v[k]);
          atomicAdd(aO + k / 2, v[k + 1]);
        }
      }
    }
  }

  template <int PAR>
  __device__ __forceinline__ void output(int ro, const float (&A)[COLS], const float (&B)[CT], double& gap,
                                         double& gapT) {
    if constexpr (GAP) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < COLS; ++k) s += A[k];
      gap += (double)s;
      if constexpr (NTK) {
        float u = 0.f;
#pragma unroll
        for (int k = 0; k < COLS; ++k) u += B[k];
        gapT += (double)u;
      }
    } else if constexpr (PAR == 0) {
#pragma unroll
      for (int k = 0; k < COLS; ++k) acc[k] = A[k];
      if constexpr (NTK) {
#pragma unroll
        for (int k = 0; k < COLS; ++k) accT[k] = B[k];
      }
    } else {
      const int I = ro >> 1;
      float v[COLS];
#pragma unroll
      for (int k = 0; k < COLS; ++k) v[k] = tyodd ? acc[k] : acc[k] + A[k];
      scatter(slot, t_y >> 1, I, v);
      if (tyodd) scatter(slot, ((t_y + 1) >> 1) & (R1 - 1), I, A);
      if constexpr (NTK) {
        float w[COLS], bt[COLS];
#pragma unroll
        for (int k = 0; k < COLS; ++k) {
          w[k] = tyodd ? accT[k] : accT[k] + B[k];
          bt[k] = B[k];
        }
        scatter(slotT, t_y >> 1, I, w);
        if (tyodd) scatter(slotT, ((t_y + 1) >> 1) & (R1 - 1), I, bt);
      }
    }
  }

  template <int j0, int j1>
  __device__ __forceinline__ void layers_fin(int t, float (&A)[COLS], float (&B)[CT]) {
    if constexpr (j0 < j1) {
      layer<j0, true>(t - j0, A, B);
      layers_fin<j0 + 1, j1>(t, A, B);
    }
  }

  // pipeline fill, step s0 + T for T < N: layers 0..T-1 finish rows, layer T
  // receives its first row s0
  template <int T>
  __device__ __forceinline__ void fill() {
    if constexpr (T < N) {
      float A[COLS], B[CT];
      input_row(s0 + T, A, B);
      layers_fin<0, T>(s0 + T, A, B);
      layer<T, false>(s0, A, B);
      fill<T + 1>();
    }
  }

  template <int PAR>
  __device__ __forceinline__ void steady(int t, double& gap, double& gapT) {
    float A[COLS], B[CT];
    input_row(t, A, B);
    layers_fin<0, N>(t, A, B);
    output<PAR>(t - N, A, B, gap, gapT);
  }

  template <int D>
  __device__ __forceinline__ void drain(double& gap, double& gapT) {
    if constexpr (D < N) {
      float A[COLS], B[CT];
#pragma unroll
      for (int k = 0; k < COLS; ++k) A[k] = 0.f;
#pragma unroll
      for (int k = 0; k < CT; ++k) B[k] = 0.f;
      finish_last<D>(A, B);
      layers_fin<D + 1, N>(R + D, A, B);
      output<((R + D - N) & 1)>(R + D - N, A, B, gap, gapT);
      drain<D + 1>(gap, gapT);
    }
  }

  __device__ __forceinline__ void run(double& gap, double& gapT) {
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
      for (int k = 0; k < COLS; ++k) Hp[j][k] = Pp[j][k] = 0.f;
    if constexpr (NTK) {
#pragma unroll
      for (int j = 0; j < N; ++j)
#pragma unroll
        for (int k = 0; k < CT; ++k) HpT[j][k] = PpT[j][k] = 0.f;
    }
    if constexpr (!SEED) {
      take_row<COLS, SHIN>(in, nx);
      if constexpr (NTK) take_row<COLS, SHIN>(inT, nxT);
    }
    fill<0>();
    int t = s0 + N;
    // halo rows: computed, not output (b0 - s0 is 0 or N)
    for (; t < b0 + N; ++t) {
      float A[COLS], B[CT];
      input_row(t, A, B);
      layers_fin<0, N>(t, A, B);
    }
    // output rows from b0 (even) in pairs
    for (; t + 1 < s1; t += 2) {
      steady<0>(t, gap, gapT);
      steady<1>(t + 1, gap, gapT);
    }
    if (t < s1) steady<0>(t, gap, gapT);
    if (s1 == R) drain<0>(gap, gapT);
  }
};

// 0/1 factors of the couplings between local columns k-1 and k of a row part
// (0 across the image border and the super-plane's column cut).
template <int COLS>
__device__ __forceinline__ void edges(float (&e)[COLS + 1], int R, int t_x, int q) {
  const int c0 = q * COLS;
  const int kc = (t_x == 0) ? -100 : R - 1 - t_x;
#pragma unroll
  for (int k = 0; k <= COLS; ++k) {
    const int lc = c0 + k - 1;
    e[k] = ((lc < 0) || (lc + 1 > R - 1) || (lc == kc)) ? 0.f : 1.f;
  }
}

__device__ __forceinline__ float4 ld_x(const float* p, int C, float s) {
  return make_float4(p[0] * s, C > 1 ? p[1] * s : 0.f, C > 2 ? p[2] * s : 0.f, 0.f);
}

// Block of pair g.
__device__ __forceinline__ int block_of(const TiledParams& Q, int64_t g) { return sched::block_of_pair(Q, g); }

// Slot of pair g (block b) in its resolution's ring, and the pair that used
// it before (-1: none).
__device__ __forceinline__ float* slot_of(const TiledParams& Q, int b, int64_t g, int64_t* prev) {
  int r;
  const int64_t k = sched::slot(Q, b, g, &r, prev);
  return Q.slots + Q.ring_off[r] + k * Q.slot_floats[r];
}

// Theta of the NTK: K + sw2 mean(Theta_t), i.e. the GAP scale applied to the
// sum of both global-average sums (K's bias added once).
__device__ __forceinline__ void store_theta(const FusedParams& P, int64_t i, int64_t j, double tot) {
  const float v = (float)(P.out_scale * tot + P.out_bias);
  P.Th[i * P.ldk + j] = v;
  if (P.sym && i != j) P.Th[j * P.ldk + i] = v;
}

// ---------------------------------------------------------------------------
// Stage-0 task `sub` of pair g (block b).
// ---------------------------------------------------------------------------
template <int R, int N0, int N1, bool BIAS, int NT, int ACT, bool NTK>
__device__ void stage0_task(const TiledParams& Q, int b, int64_t g, int sub, unsigned char* smem, double* red,
                            int* flag) {
  using G = G0<R>;
  using L = L0<R, N0>;
  constexpr bool TWO = N1 > 0;
  const FusedParams& P = Q.B[b];
  int64_t i, j;
  pair_ij(g - Q.g0[b], P.na, P.nb, P.sym, &i, &j);
  const int64_t ia = P.a0 + i, ib = P.b0 + j;
  const int band = sub / (G::NTY * G::NTX);
  const int yg = (sub / G::NTX) % G::NTY;
  const int xg = sub % G::NTX;
  const int b0 = band * G::B;
  const int s0 = b0 - N0 > 0 ? b0 - N0 : 0;
  const int s1 = b0 + G::B + N0 < R ? b0 + G::B + N0 : R;
  const int ty0 = yg * G::TY, tx0 = xg * G::TX;
  int64_t prev = -1;
  float* slot = TWO ? slot_of(Q, b, g, &prev) : nullptr;
  constexpr int64_t R1 = R / 2;
  float* slotT = (TWO && NTK) ? slot + R1 * R1 * R1 * R1 : nullptr;  // the tangent's pooled tensor

  // the slot's previous pair must have been taken by its stage-1 task
  if (threadIdx.x == 0) {
    bool ok = true;
    if (TWO && prev >= 0) ok = wait_geq(Q, Q.done1 + prev, 1);
    *flag = ok ? 1 : 0;
  }
  float4* xs = reinterpret_cast<float4*>(smem + L::xs_off);
  float4* xq = reinterpret_cast<float4*>(smem + L::xq_off);
  float2* pt = reinterpret_cast<float2*>(smem + L::p_off);
  float2* qt = reinterpret_cast<float2*>(smem + L::q_off);
  {
    const int C = P.C;
    const float* xa = P.Xa + ia * (int64_t)R * R * C;
    const float* xb = P.Xb + ib * (int64_t)R * R * C;
    const float2* qa = reinterpret_cast<const float2*>(P.qsa) + ia * P.nq;
    const float2* qb = reinterpret_cast<const float2*>(P.qsb) + ib * P.nq;
    const int np = (s1 - s0) * R;
    for (int e = threadIdx.x; e < np; e += NT) {
      const int r = s0 + e / R, c = e % R;
      const int d = (r - s0) * G::SXP + (c / G::COLS) * (G::COLS + 1) + c % G::COLS;
      xs[d] = ld_x(xa + (r * R + c) * C, C, P.xscale);
#pragma unroll
      for (int l = 0; l < N0; ++l) {
        const float2 v = qa[P.qoff[l] + r * R + c];
        pt[l * L::PL + d] = make_float2(v.x, v.y * P.fold[l]);
      }
    }
    const int nq = (s1 - s0 + G::TY - 1) * G::SQ;
    for (int e = threadIdx.x; e < nq; e += NT) {
      const int wr = e / G::SQ, wc = e - wr * G::SQ;
      const int r = (s0 + ty0 + wr) & (R - 1), c = (tx0 + wc) & (R - 1);
      const int pc = G::PH ? (wc & 3) * G::NPH + (wc >> 2) : wc;  // column position in a window row
      xq[wr * G::SQX + pc] = ld_x(xb + (r * R + c) * C, C, 1.f);
#pragma unroll
      for (int l = 0; l < N0; ++l) qt[l * L::QL + wr * G::SQQ + pc] = qb[P.qoff[l] + r * R + c];
    }
  }
  __syncthreads();
  if (*flag == 0) return;  // aborted (the caller's loop stops)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = lane / G::TYW, tyl = lane - q * G::TYW;
  double gap = 0.0, gapT = 0.0;
  using BT = Band<R, G::NQ, N0, true, !TWO, BIAS, false, G::SXP, G::SQQ, L::PL, L::QL, ACT, G::SQX, G::PH, NTK>;
  static_assert(BT::COLS == G::COLS && BT::TYW == G::TYW, "split");
  for (int w = warp; w < G::WT; w += NT / 32) {
    BT T;
    const int txl = w / G::YW;
    const int tyw = (w % G::YW) * G::TYW + tyl;  // t_y - ty0
    T.t_x = tx0 + txl;
    T.t_y = ty0 + tyw;
    T.c0 = q * G::COLS;
    T.s0 = s0;
    T.s1 = s1;
    T.b0 = b0;
    T.tyodd = (T.t_y & 1) != 0;
    edges<G::COLS>(T.E, R, T.t_x, q);
    T.xs = xs;
    T.xq = xq;
    T.in = nullptr;
    T.ptab = pt;
    T.qtab = qt;
    T.pcol = q * (G::COLS + 1);
    T.qr0 = tyw - s0;
    T.qc = T.c0 + txl;
    if constexpr (G::PH) {
#pragma unroll
      for (int k = 0; k < G::COLS; ++k) {
        const int c = T.qc + k;
        T.qo[k] = (c & 3) * G::NPH + (c >> 2);
      }
    }
    T.slot = slot;
    T.slotT = slotT;
    T.inT = nullptr;
    T.fth = P.fold;
    T.dg = NTK && P.Xa == P.Xb && ia == ib && T.t_x == 0 && T.t_y == 0;
    T.b = P.sb2;
    T.run(gap, gapT);
  }
  if constexpr (TWO) {
    // publish this task's atomic adds, then count it: the barrier orders
    // every thread's adds before thread 0's fence, which releases them
    // together with the count
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(Q.cnt0 + g, 1);
    }
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gap += __shfl_xor_sync(FULL, gap, o);
    if (lane == 0) red[warp] = gap;
    if constexpr (NTK) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) gapT += __shfl_xor_sync(FULL, gapT, o);
      if (lane == 0) red[MAX_WARPS + warp] = gapT;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0, sT = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += red[w];
      atomicAdd(Q.gacc + g, s);
      if constexpr (NTK) {
        for (int w = 0; w < NT / 32; ++w) sT += red[MAX_WARPS + w];
        atomicAdd(Q.gacc + Q.G + g, sT);
      }
      __threadfence();
      const int old = atomicAdd(Q.cnt0 + g, 1);
      if (old == Q.nt0[b] - 1) {
        __threadfence();
        const double tk = atomicAdd(Q.gacc + g, 0.0);
        store_entry(P, i, j, tk);
        if constexpr (NTK) store_theta(P, i, j, tk + atomicAdd(Q.gacc + Q.G + g, 0.0));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Stage-1 task of pair g: the whole R1 stage on this CTA, then K.
// ---------------------------------------------------------------------------
// Shared memory of a stage-1 task: its tables, then (three-stage nets) the
// pooled stage-2 tile of K (and of Theta) and the stage-2 tables.
template <int R1, int N1, int N2, bool NTK>
struct L1x {
  static constexpr int R2 = R1 / 2;
  static constexpr size_t tile_off = (L1<R1, N1>::bytes + 15) / 16 * 16;
  static constexpr size_t tile_floats = N2 > 0 ? (size_t)R2 * R2 * R2 * R2 : 0;
  static constexpr size_t tab2_off = tile_off + (NTK ? 2 : 1) * tile_floats * 4;
  static constexpr size_t bytes = N2 > 0 ? tab2_off + L1<(R2 > 0 ? R2 : 1), N2>::bytes : L1<R1, N1>::bytes;
};

template <int R1, int N0, int N1, bool BIAS, int NT, int ACT, bool NTK, int N2 = 0>
__device__ void stage1_task(const TiledParams& Q, int64_t g, unsigned char* smem, double* red, int* flag) {
  using L = L1<R1, N1>;
  using SP = Split<R1>;
  using X1 = L1x<R1, N1, N2, NTK>;
  const int b = block_of(Q, g);
  const FusedParams& P = Q.B[b];
  int64_t i, j;
  pair_ij(g - Q.g0[b], P.na, P.nb, P.sym, &i, &j);
  const int64_t ia = P.a0 + i, ib = P.b0 + j;
  int64_t prev = -1;
  float* slot = slot_of(Q, b, g, &prev);
  if (threadIdx.x == 0) *flag = wait_geq(Q, Q.cnt0 + g, Q.nt0[b]) ? 1 : 0;
  float2* pt = reinterpret_cast<float2*>(smem + L::p_off);
  float2* qt = reinterpret_cast<float2*>(smem + L::q_off);
  {
    const float2* qa = reinterpret_cast<const float2*>(P.qsa) + ia * P.nq;
    const float2* qb = reinterpret_cast<const float2*>(P.qsb) + ib * P.nq;
    for (int l = 0; l < N1; ++l) {
      const int Lr = N0 + l;
      const float f = P.fold[Lr];
      for (int e = threadIdx.x; e < R1 * R1; e += NT) {
        const float2 v = qa[P.qoff[Lr] + e];
        pt[l * L::PL + e] = make_float2(v.x, v.y * f);
      }
      for (int e = threadIdx.x; e < R1 * 2 * R1; e += NT) {
        const int row = e / (2 * R1), col = e - row * 2 * R1;
        qt[l * L::QL + row * L::S + col] = qb[P.qoff[Lr] + row * R1 + (col & (R1 - 1))];
      }
    }
    if constexpr (N2 > 0) {
      // stage-2 tables, and the stage-2 tile(s) cleared for this pair's pooled adds
      using L2 = L1<X1::R2, N2>;
      constexpr int R2 = X1::R2;
      float2* pt2 = reinterpret_cast<float2*>(smem + X1::tab2_off + L2::p_off);
      float2* qt2 = reinterpret_cast<float2*>(smem + X1::tab2_off + L2::q_off);
      for (int l = 0; l < N2; ++l) {
        const int Lr = N0 + N1 + l;
        const float f = P.fold[Lr];
        for (int e = threadIdx.x; e < R2 * R2; e += NT) {
          const float2 v = qa[P.qoff[Lr] + e];
          pt2[l * L2::PL + e] = make_float2(v.x, v.y * f);
        }
        for (int e = threadIdx.x; e < R2 * 2 * R2; e += NT) {
          const int row = e / (2 * R2), col = e - row * 2 * R2;
          qt2[l * L2::QL + row * L2::S + col] = qb[P.qoff[Lr] + row * R2 + (col & (R2 - 1))];
        }
      }
      float* tile = reinterpret_cast<float*>(smem + X1::tile_off);
      for (size_t e = threadIdx.x; e < (NTK ? 2 : 1) * X1::tile_floats; e += NT) tile[e] = 0.f;
    }
  }
  __syncthreads();
  if (*flag == 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = lane / SP::TYW, tyl = lane - q * SP::TYW;
  double gap = 0.0, gapT = 0.0;
  // stage 1 feeds the global average (two-stage nets) or pools into the
  // stage-2 tile in shared memory (three-stage nets)
  constexpr bool GAP1 = N2 == 0;
  float* tile = N2 > 0 ? reinterpret_cast<float*>(smem + X1::tile_off) : nullptr;
  using BT = Band<R1, SP::NQ, N1, false, GAP1, BIAS, true, R1, L::S, L::PL, L::QL, ACT, L::S, false, NTK>;
  static_assert(BT::COLS == SP::COLS && BT::TYW == SP::TYW, "split");
  static_assert(GAP1 || BT::COLS == 2, "the pooled adds into the shared tile use generic atomics (COLS == 2)");
  constexpr int NH = SP::WPT;
  for (int task = warp; task < R1 * NH; task += NT / 32) {
    BT T;
    T.t_x = task / NH;
    T.t_y = (task % NH) * SP::TYW + tyl;
    T.c0 = q * SP::COLS;
    T.s0 = 0;
    T.s1 = R1;
    T.b0 = 0;
    T.tyodd = (T.t_y & 1) != 0;
    edges<SP::COLS>(T.E, R1, T.t_x, q);
    T.xs = nullptr;
    T.xq = nullptr;
    T.in = slot + ((size_t)(T.t_y * R1 + T.t_x) * R1) * R1 + T.c0;
    T.inT = NTK ? T.in + (size_t)R1 * R1 * R1 * R1 : nullptr;
    T.slotT = (N2 > 0 && NTK) ? tile + X1::tile_floats : nullptr;
    T.fth = P.fold + N0;
    T.dg = NTK && P.Xa == P.Xb && ia == ib && T.t_x == 0 && T.t_y == 0;
    T.ptab = pt;
    T.qtab = qt;
    T.pcol = T.c0;
    T.qr0 = 0;
    T.qc = T.c0 + T.t_x;
    T.slot = tile;
    T.b = P.sb2;
    T.run(gap, gapT);
  }
  if constexpr (N2 > 0) {
    // stage 2 from the pooled tile, on the same CTA
    __syncthreads();
    constexpr int R2 = X1::R2;
    using L2 = L1<R2, N2>;
    using SP2 = Split<R2>;
    using BT2 = Band<R2, SP2::NQ, N2, false, true, BIAS, true, R2, L2::S, L2::PL, L2::QL, ACT, L2::S, false, NTK,
                     true>;
    static_assert(BT2::COLS == SP2::COLS && BT2::TYW == SP2::TYW, "split");
    const int q2 = lane / SP2::TYW, tyl2 = lane - q2 * SP2::TYW;
    constexpr int NH2 = SP2::WPT;
    for (int task = warp; task < R2 * NH2; task += NT / 32) {
      BT2 T;
      T.t_x = task / NH2;
      T.t_y = (task % NH2) * SP2::TYW + tyl2;
      T.c0 = q2 * SP2::COLS;
      T.s0 = 0;
      T.s1 = R2;
      T.b0 = 0;
      T.tyodd = (T.t_y & 1) != 0;
      edges<SP2::COLS>(T.E, R2, T.t_x, q2);
      T.xs = nullptr;
      T.xq = nullptr;
      T.in = tile + ((size_t)(T.t_y * R2 + T.t_x) * R2) * R2 + T.c0;
      T.inT = NTK ? T.in + X1::tile_floats : nullptr;
      T.slotT = nullptr;
      T.fth = P.fold + N0 + N1;
      T.dg = NTK && P.Xa == P.Xb && ia == ib && T.t_x == 0 && T.t_y == 0;
      T.ptab = reinterpret_cast<const float2*>(smem + X1::tab2_off + L2::p_off);
      T.qtab = reinterpret_cast<const float2*>(smem + X1::tab2_off + L2::q_off);
      T.pcol = T.c0;
      T.qr0 = 0;
      T.qc = T.c0 + T.t_x;
      T.slot = nullptr;
      T.b = P.sb2;
      T.run(gap, gapT);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gap += __shfl_xor_sync(FULL, gap, o);
  if (lane == 0) red[warp] = gap;
  if constexpr (NTK) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gapT += __shfl_xor_sync(FULL, gapT, o);
    if (lane == 0) red[MAX_WARPS + warp] = gapT;
  }
  // the cleared slot is published before the flag that frees it (barrier,
  // then thread 0's fence)
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    store_entry(P, i, j, s);
    if constexpr (NTK) {
      double sT = 0.0;
      for (int w = 0; w < NT / 32; ++w) sT += red[MAX_WARPS + w];
      store_theta(P, i, j, s + sT);
    }
    __threadfence();
    atomicExch(Q.done1 + g, 1);
  }
}

template <int N0, int N1, int RMAX, bool NTK = false, int N2 = 0>
struct Smem {
  static_assert(N2 == 0 || RMAX == 32, "three-stage nets: 32x32 images only");
  static constexpr size_t s0 = RMAX == 64 ? std::max(L0<64, N0>::bytes, L0<32, N0>::bytes) : L0<32, N0>::bytes;
  static constexpr size_t s1 =
      N1 > 0 ? (RMAX == 64 ? std::max(L1<32, N1>::bytes, L1<16, N1>::bytes) : L1x<16, N1, N2, NTK>::bytes) : 0;
  static constexpr size_t tables = std::max(s0, s1);
  static constexpr size_t red = (NTK ? 2 : 1) * MAX_WARPS * 8;  // per-warp global-average sums
  static constexpr size_t bytes = tables + red + 16;
};

// NTK instantiations carry the tangent rows (twice the pipeline registers)
// in the same launch shapes (at 128 registers they spill a few bytes).
template <int N0, int N1, bool BIAS, int NT, int RMAX, int ACT, bool NTK = false, int N2 = 0>
__global__ void __launch_bounds__(NT, 512 / NT) k_myrtle_tiled(const __grid_constant__ TiledParams Q) {
  extern __shared__ __align__(16) unsigned char smem[];
  using SM = Smem<N0, N1, RMAX, NTK, N2>;
  constexpr bool TWO = N1 > 0;
  double* red = reinterpret_cast<double*>(smem + SM::tables);
  int* flag = reinterpret_cast<int*>(smem + SM::tables + SM::red);
  long long* item_s = reinterpret_cast<long long*>(smem + SM::tables + SM::red + 8);
  for (;;) {
    if (threadIdx.x == 0) {
      const long long m =
          *(volatile int*)Q.abort_flag ? (long long)Q.nitems : (long long)atomicAdd(Q.next, 1ull);
      long long code = -1;  // stage-0 index k -> 2k; stage-1 pair k -> 2k + 1; -1 done
      if (m < Q.nitems) {
        int64_t k;
        const int st1 = sched::decode(Q, TWO, m, &k);
        code = 2 * k + st1;
      }
      *item_s = code;
    }
    __syncthreads();
    const long long code = *item_s;
    __syncthreads();
    if (code < 0) break;
    const int64_t k = code >> 1;
    if ((code & 1) == 0) {
      int b, sub;
      int64_t g;
      sched::stage0_of(Q, k, &b, &g, &sub);
      if constexpr (RMAX == 64) {
        if (Q.R[b] == 64)
          stage0_task<64, N0, N1, BIAS, NT, ACT, NTK>(Q, b, g, sub, smem, red, flag);
        else
          stage0_task<32, N0, N1, BIAS, NT, ACT, NTK>(Q, b, g, sub, smem, red, flag);
      } else {
        stage0_task<32, N0, N1, BIAS, NT, ACT, NTK>(Q, b, g, sub, smem, red, flag);
      }
    } else if constexpr (TWO) {
      if constexpr (RMAX == 64) {
        if (Q.R[block_of(Q, k)] == 64)
          stage1_task<32, N0, N1, BIAS, NT, ACT, NTK>(Q, k, smem, red, flag);
        else
          stage1_task<16, N0, N1, BIAS, NT, ACT, NTK>(Q, k, smem, red, flag);
      } else {
        stage1_task<16, N0, N1, BIAS, NT, ACT, NTK, N2>(Q, k, smem, red, flag);
      }
    }
    // the next item's staging overwrites the tables
    __syncthreads();
  }
}

template <int N0, int N1, bool BIAS, int NT, int RMAX, int ACT, bool NTK = false, int N2 = 0>
cudaError_t launch_t(TiledParams& Q, const int64_t* npairs, int sm_count, void* ws, size_t ws_bytes,
                     cudaStream_t st) {
  using SM = Smem<N0, N1, RMAX, NTK, N2>;
  auto kern = k_myrtle_tiled<N0, N1, BIAS, NT, RMAX, ACT, NTK, N2>;
  constexpr int tensors = NTK ? 2 : 1;
  static bool attr_set[64] = {false};
  static int per_sm[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NT, SM::bytes);
    if (e != cudaSuccess) return e;
    per_sm[dev] = nb > 0 ? nb : 1;
    attr_set[dev] = true;
  }
  const int grid = std::max(1, sm_count * per_sm[dev]);
  constexpr bool TWO = N1 > 0;
  const sched::Plan p = sched::make_plan(TWO, Q.R, npairs, Q.n, grid, tensors);
  if (p.bytes > ws_bytes) return cudaErrorInvalidValue;
  Q.LAG = p.LAG;
  Q.nitems = Q.T0 + (TWO ? Q.G : 0);
  const size_t G = (size_t)Q.G;
  char* c = reinterpret_cast<char*>(ws);
  for (int r = 0; r < 2; ++r) {
    Q.S[r] = p.S[r];
    Q.slot_floats[r] = p.slot_floats[r];
    Q.ring_off[r] = p.ring_off[r];
  }
  Q.slots = reinterpret_cast<float*>(c);
  Q.gacc = reinterpret_cast<double*>(c + p.slot_bytes);
  Q.cnt0 = reinterpret_cast<int*>(c + p.slot_bytes + tensors * G * sizeof(double));
  Q.done1 = Q.cnt0 + G;
  Q.next = reinterpret_cast<unsigned long long*>(c + p.slot_bytes + G * (2 * sizeof(int) + tensors * sizeof(double)));
  Q.abort_flag = reinterpret_cast<int*>(Q.next + 1);
  cudaError_t e = cudaMemsetAsync(ws, 0, p.bytes, st);
  if (e != cudaSuccess) return e;
  kern<<<grid, NT, SM::bytes, st>>>(Q);
  return cudaGetLastError();
}

// Fills the queue description shared by every instantiation.  False when a
// block is not 64x64 or 32x32 or 64x64 blocks do not come first.
inline bool make_queue(TiledParams& Q, int64_t* np, const int* R, const FusedParams* B, int n,
                       unsigned int* dstatus, long long wait_limit) {
  Q = TiledParams{};
  Q.n = n;
  Q.g0[0] = 0;
  Q.f0[0] = 0;
  for (int b = 0; b < n; ++b) {
    if (R[b] != 64 && R[b] != 32) return false;
    if (b > 0 && R[b] > R[b - 1]) return false;  // 64x64 blocks first
    Q.R[b] = R[b];
    Q.nt0[b] = R[b] == 64 ? G0<64>::NT0 : G0<32>::NT0;
    Q.B[b] = B[b];
    np[b] = B[b].npairs;
    Q.g0[b + 1] = Q.g0[b] + B[b].npairs;
    Q.f0[b + 1] = Q.f0[b] + B[b].npairs * Q.nt0[b];
    if (R[b] == 64) Q.G64 = Q.g0[b + 1];
  }
  Q.G = Q.g0[n];
  Q.T0 = Q.f0[n];
  Q.dstatus = dstatus;
  Q.wait_limit = wait_limit;
  return true;
}

// The instantiations of one activation: stage patterns (2,1,0) (1) (1,1),
// with and without the bias, 256-thread 32x32-only or 512-thread launches.
template <int ACT>
cudaError_t launch_act(const int c[3], bool bias, TiledParams& Q, const int64_t* np, int sm_count, void* ws,
                       size_t ws_bytes, cudaStream_t st) {
  const bool only32 = Q.G64 == 0;
#define NK_T(a, b_)                                                                                    \
  if (c[0] == a && c[1] == b_) {                                                                       \
    if (only32)                                                                                        \
      return bias ? launch_t<a, b_, true, 256, 32, ACT>(Q, np, sm_count, ws, ws_bytes, st)            \
                  : launch_t<a, b_, false, 256, 32, ACT>(Q, np, sm_count, ws, ws_bytes, st);          \
    return bias ? launch_t<a, b_, true, 512, 64, ACT>(Q, np, sm_count, ws, ws_bytes, st)              \
                : launch_t<a, b_, false, 512, 64, ACT>(Q, np, sm_count, ws, ws_bytes, st);            \
  }
  NK_T(2, 1) NK_T(1, 0) NK_T(1, 1)
#undef NK_T
  return cudaErrorNotSupported;
}

}  // namespace tiled
}  // namespace nkf
