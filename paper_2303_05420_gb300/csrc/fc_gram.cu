// nk_fc_block: fully-connected ReLU NNGP kernel block (Appendix A, FC3
// listing) on the tensor cores.
//
//   K_0 = x . x' / d;  K = sw2 K_0 + sb2;  depth times: K <- sw2 relu_map(K) + sb2
//
// The Gram X_a X_b^T is the one dense contraction of the method (d = 3072
// for the CIFAR-shaped inputs).  It runs as a BF16 tcgen05 GEMM with FP32
// accumulation in TMEM on split operands: x = x_hi + x_lo (BF16 each) and
// x . x' ~ hi.lo' + lo.hi' + hi.hi'.  Each row is rewritten once with every
// 32-column block of x as 64 BF16 columns, its high parts then its low parts
// (zero-padded to a multiple of 64), so one 128-byte TMA row of a stage holds
// both parts of 32 columns and feeds all three products: per stage 6 MMAs
// (128 x 256 x 16) on 48 KB of operands.  Persistent CTAs (one per SM) walk
// the 128 x 256 output tiles in a grouped raster (16 tile rows at a time, so
// that concurrent CTAs share B tiles in L2).  Operand tiles (128 x 64 and
// 256 x 64 BF16) arrive by TMA with 128-byte swizzle through a 4-stage
// mbarrier ring (each CTA loads its own tiles); one thread issues the MMAs;
// eight epilogue warps take the finished sums out of TMEM into registers
// (32 rows x 128 columns a warp), release TMEM at once so that the next
// tile's MMAs start, and then apply the whole arc-cosine recursion layer by
// layer over 32 entries at a time (column factors staged in shared memory)
// and store 16 bytes of a K row per lane.  The self-variances q_l of each
// row follow the closed diagonal recursion q_1 = sw2 |x|^2/d + sb2,
// q_{l+1} = sw2 q_l / 2 + sb2 (FP64).  Symmetric blocks run only tiles
// touching the upper triangle and store each entry at (i, j) and (j, i).
//
// Accumulation accuracy.  The tensor core adds each 16-element MMA step to
// the FP32 accumulator with a rounding that always goes toward zero, so for
// a sum of products of one sign (a row with itself or with a near copy of
// itself) the errors add up one way, in proportion to the number of steps
// taken at the full size of the sum: about 2e-5 relative at d = 3072 for one
// accumulator over all 3d products.  Here the small products hi.lo' and
// lo.hi' go to their own accumulator (TMEM columns [0, 256)), whose sum is
// about 2^-8 of the total, and the hi.hi' products to a second one
// ([256, 512)), which the epilogue copies into registers once half of the K
// blocks are in, so that each half is summed from zero (about 4e-6 for near
// copies in a model of the rounding, the level of two alternating chunks).
// The epilogue adds the three sums in FP32.  Self pairs take K_1 from the
// FP64 norm.
//
// Every mbarrier wait of the pipeline is bounded by the handle's wait limit;
// on a timeout the kernel records NK_DEV_TIMEOUT and skips its stores, and
// before exit it waits (with a fixed generous bound) for its own TMA loads
// and MMAs in flight, then frees TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "nk_common.cuh"
#include "nk_map.cuh"
#include "tc_gemm.cuh"

namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int KD = BK / 2;      // columns of x per stage (high and low parts)
constexpr int GROUP_M = 16;     // tile rows per raster group (L2 reuse of B)
constexpr int EPI_WARPS = 8;    // two per TMEM lane quarter, 128 columns each
constexpr int EPI_COLS = BN / 2;
// warpgroup 0: TMA producer (warp 0), MMA issuer (warp 1), two idle warps;
// warpgroups 1 and 2: the epilogue
constexpr int THREADS = 128 + 32 * EPI_WARPS;
// Register split.  Twelve warps on four SM sub-partitions cap a thread at
// 168 registers (three warps per sub-partition), too few for the
// epilogue's 128 drained sums plus the recursion's temporaries (it
// spilled).  The control warpgroup gives registers back and the epilogue
// takes them: 128 x 40 + 256 x 232 = 384 x 168, the launch allocation; per
// sub-partition one control and two epilogue warps, 40 + 2 x 232 = 3 x 168.
// The host refuses the launch unless the kernel was built with exactly
// REG_LAUNCH registers per thread, since an increase beyond the launch
// allocation would never be granted.
constexpr int REG_LAUNCH = 168, REG_CTRL = 40, REG_EPI = 232;
static_assert(128 * REG_CTRL + 32 * EPI_WARPS * REG_EPI <= THREADS * REG_LAUNCH, "register split");
constexpr uint32_t DRAIN_LIMIT = 1u << 26;  // waits for own copies / MMAs before exit
constexpr int MAX_DEPTH = 8;

struct GemmSmem {
  alignas(1024) __nv_bfloat16 A[STAGES][BM * BK];
  alignas(1024) __nv_bfloat16 B[STAGES][BN * BK];
  float2 qb[BN * MAX_DEPTH];             // per-column (1/sqrt q, sqrt q) of the current tile
  float2 qa[BM * MAX_DEPTH];             // per-row (1/sqrt q, sqrt q * sw2/(2 pi))
  uint64_t full[STAGES], empty[STAGES];  // operand ring
  uint64_t tfull, tempty;                // TMEM accumulators: MMA -> epilogue, epilogue -> MMA
  uint64_t hfull, hempty;                // the first half's hi.hi' sum: MMA -> epilogue, epilogue -> MMA
  uint64_t done;
  uint32_t tslot;
};

struct FcParams {
  int64_t M, N;          // rows of A', B'
  int kpad;              // 64 ceil(d / 32): the split columns of a row
  int depth;
  float kscale;          // sw2 / d
  float sb2;
  const float2* qa;      // [M][depth] (1/sqrt q_l, sqrt q_l * sw2/(2 pi))
  const float2* qb;      // [N][depth] (1/sqrt q_l, sqrt q_l)
  float* K;
  int64_t ldk;
  int sym;
  int ntm, ntn;          // tiles along M and N
  unsigned int* dstatus;
  uint32_t wait_limit;   // polls of a pipeline mbarrier wait before it gives up
  // self pairs (same image on both sides: Xa == Xb and a0 + i == b0 + j)
  // take K_1 = sw2 |x|^2/d + sb2 from the FP64 norm instead of the Gram
  int same;
  int64_t selfoff;       // a0 - b0
  const float* q1a;      // [M]
};

// Tile slot t of the grouped raster: GROUP_M tile rows at a time, column by
// column, so that the CTAs running together share B tiles in L2.  False
// when the tile has no entry on or above the diagonal of a symmetric block.
__device__ __forceinline__ bool tile_of(const FcParams& P, int64_t t, int& tm, int& tn) {
  const int64_t per_group = (int64_t)GROUP_M * P.ntn;
  const int g = (int)(t / per_group);
  const int64_t k = t - (int64_t)g * per_group;
  const int rows = min(GROUP_M, P.ntm - g * GROUP_M);
  tm = g * GROUP_M + (int)(k % rows);
  tn = (int)(k / rows);
  return !(P.sym && (int64_t)tn * BN + BN - 1 < (int64_t)tm * BM);
}

__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Barrier over n threads that also returns whether any of them passed v.
__device__ __forceinline__ bool named_any(int id, int n, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// The arc-cosine recursion and the stores of 32 consecutive entries of row i
// (columns n0 + c0 .. n0 + c0 + 31) whose Gram sums are in w.
__device__ __forceinline__ void epi_entries(const FcParams& P, float (&w)[32], const float2* qr,
                                            const float2* qb, int c0, int64_t n0, int64_t i, bool rowok,
                                            float self_k1, bool vec_ok) {
  if (P.same) {
    const int64_t d = i + P.selfoff - (n0 + c0);  // column of the self pair, if among these
#pragma unroll
    for (int e = 0; e < 32; ++e) w[e] = (d == e) ? self_k1 : fmaf(P.kscale, w[e], P.sb2);
  } else {
#pragma unroll
    for (int e = 0; e < 32; ++e) w[e] = fmaf(P.kscale, w[e], P.sb2);
  }
  // layer by layer over the 32 entries (independent chains)
  for (int l = 0; l < P.depth; ++l) {
    const float2 ra = qr[l];
    const float2* qc = qb + c0 * P.depth + l;
    if (l == 0) {
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        const float2 rb = qc[e * P.depth];
        w[e] = fmaf(ra.y * rb.y, nk_J_f32(w[e] * (ra.x * rb.x)), P.sb2);
      }
    } else {
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        const float2 rb = qc[e * P.depth];
        w[e] = fmaf(ra.y * rb.y, nk_J01_f32(w[e] * (ra.x * rb.x)), P.sb2);
      }
    }
  }
  if (!rowok) return;
  const int64_t jb = n0 + c0;
  // mirror of a symmetric block: column stores (j, i), coalesced over i
  if (P.sym) {
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      const int64_t j = jb + e;
      if (j < P.N && j > i) P.K[j * P.ldk + i] = w[e];
    }
  }
  // row stores (i, j): 16 bytes per lane; the two halves of a 32-byte sector
  // come from the same lane in consecutive stores
  float* krow = P.K + i * P.ldk + jb;
#pragma unroll
  for (int e4 = 0; e4 < 32; e4 += 4) {
    const int64_t j = jb + e4;
    if (vec_ok && j + 3 < P.N && (!P.sym || j >= i)) {
      *reinterpret_cast<float4*>(krow + e4) = make_float4(w[e4], w[e4 + 1], w[e4 + 2], w[e4 + 3]);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j + u < P.N && (!P.sym || j + u >= i)) krow[e4 + u] = w[e4 + u];
    }
  }
}

// Persistent kernel, one CTA per SM; CTA c takes tile slots t = c + k * CTAs.
// Warp 0: TMA producer; warp 1: TMEM owner and MMA issuer; warps 4..11:
// epilogue.  TMEM columns [0, 256) hold the small products' sum of the
// current tile, [256, 512) its hi.hi' sum (first half, copied out by the
// epilogue at mid-tile, then the second half).  The epilogue copies a
// finished tile into registers and releases TMEM before its arithmetic, so
// the MMAs of the next tile overlap that arithmetic.
__global__ void __launch_bounds__(THREADS, 1)
k_fc_gram(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
          const __grid_constant__ FcParams P) {
  extern __shared__ __align__(1024) unsigned char raw[];
  GemmSmem& S = *reinterpret_cast<GemmSmem*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = P.kpad / BK;
  // stages whose hi.hi' products form the first half's sum (0: one sum)
  const int H = nk >= 2 ? nk / 2 : 0;
  const int64_t cta = blockIdx.x, ncta = gridDim.x;
  const int64_t nslots = (int64_t)P.ntm * P.ntn;
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&S.full[s], 1);
      tc::mbar_init(&S.empty[s], 1);
    }
    tc::mbar_init(&S.tfull, 1);
    tc::mbar_init(&S.tempty, EPI_WARPS);
    tc::mbar_init(&S.hfull, 1);
    tc::mbar_init(&S.hempty, EPI_WARPS);
    tc::mbar_init(&S.done, 1);
    tc::mbar_fence_init();
    tc::prefetch_tmap(&ta);
    tc::prefetch_tmap(&tb);
  }
  if (warp == 1) tc::tmem_alloc(&S.tslot, 512);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = S.tslot;
  bool ok = true;
  if (warp < 4) tc::setmaxnreg_dec<REG_CTRL>();
  if (warp == 0) {
    if (lane == 0) {
      // TMA producer: the operand ring runs on across tiles
      int64_t kb_all = 0;
      for (int64_t t = cta; t < nslots && ok; t += ncta) {
        int tm, tn;
        if (!tile_of(P, t, tm, tn)) continue;
        for (int kb = 0; kb < nk; ++kb, ++kb_all) {
          const int s = (int)(kb_all % STAGES);
          if (kb_all >= STAGES &&
              !tc::mbar_wait(&S.empty[s], (uint32_t)((kb_all / STAGES) & 1) ^ 1, P.wait_limit)) {
            atomicOr(P.dstatus, NK_DEV_TIMEOUT);
            ok = false;
            break;
          }
          tc::mbar_arrive_expect_tx(&S.full[s], (BM + BN) * BK * 2);
          tc::tma_load_2d(S.A[s], &ta, &S.full[s], kb * BK, tm * BM);
          tc::tma_load_2d(S.B[s], &tb, &S.full[s], kb * BK, tn * BN);
        }
      }
      // every load issued has landed before the CTA may exit
      for (int64_t k = std::max<int64_t>(0, kb_all - STAGES); k < kb_all; ++k)
        if (!tc::mbar_wait(&S.full[k % STAGES], (uint32_t)((k / STAGES) & 1), DRAIN_LIMIT))
          atomicOr(P.dstatus, NK_DEV_TIMEOUT);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
      // Descriptors: the start-address field is the shared-memory byte
      // address / 16 in the low bits, so a stage s and a byte offset o within
      // a 128-byte row move a descriptor by (s * stage bytes + o) / 16 (all
      // addresses stay below 2^18, so the field never carries).  The loop
      // only adds constants to the stage-0 descriptors.
      const uint64_t ad0 = tc::sdesc_k128(tc::smem_addr(S.A[0]));
      const uint64_t bd0 = tc::sdesc_k128(tc::smem_addr(S.B[0]));
      constexpr uint64_t A_STEP = BM * BK * 2 / 16, B_STEP = BN * BK * 2 / 16;
      int64_t kb_all = 0;
      int n = 0;  // tiles of this CTA so far
      for (int64_t t = cta; t < nslots && ok; t += ncta) {
        int tm, tn;
        if (!tile_of(P, t, tm, tn)) continue;
        // the epilogue has taken the previous tile out of TMEM
        if (n >= 1 && !tc::mbar_wait(&S.tempty, (uint32_t)((n - 1) & 1), P.wait_limit)) {
          atomicOr(P.dstatus, NK_DEV_TIMEOUT);
          ok = false;
          break;
        }
        tc::tc_fence_after();
        for (int kb = 0; kb < nk; ++kb, ++kb_all) {
          const int s = (int)(kb_all % STAGES);
          if (!tc::mbar_wait(&S.full[s], (uint32_t)((kb_all / STAGES) & 1), P.wait_limit)) {
            atomicOr(P.dstatus, NK_DEV_TIMEOUT);
            ok = false;
            break;
          }
          tc::tc_fence_after();
          // a 128-byte operand row holds the high parts of 32 columns in
          // bytes [0, 64) (K steps 0, 1: descriptor + 0, + 2) and their low
          // parts in [64, 128) (K steps 2, 3: + 4, + 6)
          const uint64_t ad = ad0 + (uint64_t)s * A_STEP, bd = bd0 + (uint64_t)s * B_STEP;
          const uint32_t ts = tbase, tl = tbase + BN;
          tc::mma_bf16(ts, ad + 0, bd + 4, idesc, kb > 0);  // hi.lo'
          tc::mma_bf16(ts, ad + 2, bd + 6, idesc, 1);
          tc::mma_bf16(ts, ad + 4, bd + 0, idesc, 1);       // lo.hi'
          tc::mma_bf16(ts, ad + 6, bd + 2, idesc, 1);
          if (H > 0 && kb == H) {
            // the epilogue has copied the first half's hi.hi' sum out of TMEM
            if (!tc::mbar_wait(&S.hempty, (uint32_t)(n & 1), P.wait_limit)) {
              atomicOr(P.dstatus, NK_DEV_TIMEOUT);
              ok = false;
              break;
            }
            tc::tc_fence_after();
          }
          tc::mma_bf16(tl, ad + 0, bd + 0, idesc, kb != 0 && kb != H);  // hi.hi'
          tc::mma_bf16(tl, ad + 2, bd + 2, idesc, 1);
          tc::mma_commit(&S.empty[s]);  // the stage may be refilled once these MMAs have read it
          if (kb == H - 1) tc::mma_commit(&S.hfull);
        }
        if (!ok) break;
        tc::mma_commit(&S.tfull);
        ++n;
      }
      // all MMAs issued by this thread complete before TMEM is released
      tc::mma_commit(&S.done);
      if (!tc::mbar_wait(&S.done, 0, DRAIN_LIMIT)) atomicOr(P.dstatus, NK_DEV_TIMEOUT);
    }
  } else if (warp >= 4) {
    tc::setmaxnreg_inc<REG_EPI>();
    // epilogue: TMEM lane quarter q holds tile rows 32q .. 32q+31; the two
    // warps of a quarter take columns [0, 128) and [128, 256)
    const int q = warp & 3;
    const int cbeg = ((warp - 4) >> 2) * EPI_COLS;
    const int et = threadIdx.x - 128;  // 0 .. 32 * EPI_WARPS - 1
    const bool vec_ok = (P.ldk % 4 == 0) && ((reinterpret_cast<uintptr_t>(P.K) & 15) == 0);
    int n = 0;
    for (int64_t t = cta; t < nslots; t += ncta) {
      int tm, tn;
      if (!tile_of(P, t, tm, tn)) continue;
      const int64_t m0 = (int64_t)tm * BM, n0 = (int64_t)tn * BN;
      // row and column factors of this tile into shared memory
      named_sync(1, 32 * EPI_WARPS);
      for (int e = et; e < BN * P.depth; e += 32 * EPI_WARPS) {
        const int64_t j = n0 + e / P.depth;
        S.qb[e] = j < P.N ? P.qb[n0 * P.depth + e] : make_float2(0.f, 0.f);
      }
      for (int e = et; e < BM * P.depth; e += 32 * EPI_WARPS) {
        const int64_t i = m0 + e / P.depth;
        S.qa[e] = i < P.M ? P.qa[m0 * P.depth + e] : make_float2(0.f, 0.f);
      }
      named_sync(1, 32 * EPI_WARPS);
      // this warp's 32 rows x 128 columns
      const uint32_t taddr = tbase + (uint32_t)cbeg + ((uint32_t)(32 * q) << 16);
      float v[EPI_COLS / 32][32];
      if (H > 0) {
        // mid-tile: the first half's hi.hi' sum into registers
        const bool got = tc::mbar_wait(&S.hfull, (uint32_t)(n & 1), P.wait_limit);
        // the epilogue warps leave together (they share named barriers)
        if (named_any(2, 32 * EPI_WARPS, !got)) {
          atomicOr(P.dstatus, NK_DEV_TIMEOUT);
          break;
        }
        tc::tc_fence_after();
#pragma unroll
        for (int c = 0; c < EPI_COLS / 32; ++c) tc::tmem_ld32(taddr + (uint32_t)(BN + 32 * c), v[c]);
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&S.hempty);
      } else {
#pragma unroll
        for (int c = 0; c < EPI_COLS / 32; ++c)
#pragma unroll
          for (int e = 0; e < 32; ++e) v[c][e] = 0.f;
      }
      const bool got = tc::mbar_wait(&S.tfull, (uint32_t)(n & 1), P.wait_limit);
      if (named_any(2, 32 * EPI_WARPS, !got)) {
        atomicOr(P.dstatus, NK_DEV_TIMEOUT);
        break;
      }
      tc::tc_fence_after();
      // (first half + second half of hi.hi') + small products
#pragma unroll
      for (int c = 0; c < EPI_COLS / 32; ++c) {
        float u[32];
        tc::tmem_ld32(taddr + (uint32_t)(BN + 32 * c), u);
#pragma unroll
        for (int e = 0; e < 32; ++e) v[c][e] += u[e];
        tc::tmem_ld32(taddr + (uint32_t)(32 * c), u);
#pragma unroll
        for (int e = 0; e < 32; ++e) v[c][e] += u[e];
      }
      // TMEM is free for the next tile
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&S.tempty);
      const int row = 32 * q + lane;
      const int64_t i = m0 + row;
      const bool rowok = i < P.M;
      const float self_k1 = (rowok && P.same) ? P.q1a[i] : 0.f;
      const float2* qr = S.qa + row * P.depth;
      // one copy of the 32-entry body (the instruction cache is shared with
      // the single-thread TMA and MMA loops): a runtime loop that rotates the
      // register sub-arrays instead of indexing them
      static_assert(EPI_COLS / 32 == 4, "rotation below");
#pragma unroll 1
      for (int c = 0; c < EPI_COLS / 32; ++c) {
        epi_entries(P, v[0], qr, S.qb, cbeg + 32 * c, n0, i, rowok, self_k1, vec_ok);
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          v[0][e] = v[1][e];
          v[1][e] = v[2][e];
          v[2][e] = v[3][e];
        }
      }
      ++n;
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc(tbase, 512);
}

// Split rows: each 32-column block of x becomes 64 BF16 columns, the
// round-to-nearest high parts hi = bf16(x) of its 32 columns, then their low
// parts bf16(x - hi); columns past d are zero (kpad = 64 ceil(d / 32)).
__global__ void k_split_bf16(const float* __restrict__ X, int64_t rows, int d, int kpad,
                             __nv_bfloat16* __restrict__ out) {
  const int64_t total = rows * (int64_t)kpad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / kpad;
    const int k = (int)(e - r * kpad);
    const int c = (k >> 6) * KD + (k & (KD - 1));
    __nv_bfloat16 v = __float2bfloat16_rn(0.f);
    if (c < d) {
      const float x = X[r * d + c];
      const __nv_bfloat16 hi = __float2bfloat16_rn(x);
      v = (k & KD) ? __float2bfloat16_rn(x - __bfloat162float(hi)) : hi;
    }
    out[e] = v;
  }
}

// Per-row self-variances of every layer in FP64 -> (1/sqrt q, sqrt q * f);
// q1 (optional) receives q_1 = sw2 |x|^2/d + sb2.
__global__ void k_fc_q(const float* __restrict__ X, int64_t rows, int d, int depth, double sw2, double sb2,
                       float fold, float2* __restrict__ out, float* __restrict__ q1) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += nw) {
    double s = 0.0;
    for (int k = lane; k < d; k += 32) {
      const double x = X[r * d + k];
      s += x * x;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      double q = sw2 * s / d + sb2;
      if (q1) q1[r] = (float)q;
      for (int l = 0; l < depth; ++l) {
        const float2 o = q > 0.0 ? make_float2((float)(1.0 / sqrt(q)), (float)(sqrt(q) * fold))
                                 : make_float2(0.f, 0.f);
        out[r * depth + l] = o;
        q = sw2 * q / 2.0 + sb2;
      }
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

bool make_map(CUtensorMap* m, void* ptr, int64_t rows, int kpad, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t nk_fc_ws_bytes(int64_t na, int64_t nb, int d, int depth) {
  const int64_t kpad = ((int64_t)d + KD - 1) / KD * BK;
  return ((size_t)na + nb) * kpad * 2 + ((size_t)na + nb) * depth * sizeof(float2) + (size_t)na * 4 + 5 * 1024;
}

cudaError_t nk_launch_fc_block(int depth, double sw2, double sb2, const float* Xa, int64_t a0, int64_t a1,
                               const float* Xb, int64_t b0, int64_t b1, int d, float* K, int64_t ldk, int sym,
                               void* ws, int sm, unsigned int* dstatus, uint32_t wait_limit, cudaStream_t st,
                               int64_t* launches) {
  const int64_t na = a1 - a0, nb = b1 - b0;
  const int kpad = (int)(((int64_t)d + KD - 1) / KD * BK);
  char* w = reinterpret_cast<char*>(ws);
  auto take = [&](size_t bytes) {
    char* p = w;
    w += (bytes + 1023) / 1024 * 1024;
    return p;
  };
  __nv_bfloat16* Ap = reinterpret_cast<__nv_bfloat16*>(take((size_t)na * kpad * 2));
  __nv_bfloat16* Bp = reinterpret_cast<__nv_bfloat16*>(take((size_t)nb * kpad * 2));
  float2* qa = reinterpret_cast<float2*>(take((size_t)na * depth * sizeof(float2)));
  float2* qb = reinterpret_cast<float2*>(take((size_t)nb * depth * sizeof(float2)));
  float* q1a = reinterpret_cast<float*>(take((size_t)na * sizeof(float)));
  const float* xa = Xa + a0 * (int64_t)d;
  const float* xb = Xb + b0 * (int64_t)d;
  auto grid = [](int64_t total) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 32)); };
  // a symmetric block has the same rows on both sides: one split serves both
  *launches += sym ? 3 : 4;
  k_split_bf16<<<grid(na * kpad), 256, 0, st>>>(xa, na, d, kpad, Ap);
  if (!sym) k_split_bf16<<<grid(nb * kpad), 256, 0, st>>>(xb, nb, d, kpad, Bp);
  const double inv2pi = 0.15915494309189533577;
  k_fc_q<<<grid(na * 32), 256, 0, st>>>(xa, na, d, depth, sw2, sb2, (float)(sw2 * inv2pi), qa, q1a);
  k_fc_q<<<grid(nb * 32), 256, 0, st>>>(xb, nb, d, depth, sw2, sb2, 1.f, qb, nullptr);
  CUtensorMap ta, tb;
  if (!make_map(&ta, Ap, na, kpad, BM) || !make_map(&tb, sym ? Ap : Bp, nb, kpad, BN)) return cudaErrorInvalidValue;
  FcParams P = {};
  P.M = na;
  P.N = nb;
  P.kpad = kpad;
  P.depth = depth;
  P.kscale = (float)(sw2 / d);
  P.sb2 = (float)sb2;
  P.qa = qa;
  P.qb = qb;
  P.K = K;
  P.ldk = ldk;
  P.sym = sym;
  P.ntn = (int)((nb + BN - 1) / BN);
  P.ntm = (int)((na + BM - 1) / BM);
  P.same = (Xa == Xb);
  P.selfoff = a0 - b0;
  P.q1a = q1a;
  P.wait_limit = wait_limit;
  const int64_t slots = (int64_t)P.ntm * P.ntn;
  const size_t smem = sizeof(GemmSmem) + 1024;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k_fc_gram);
  if (e != cudaSuccess) return e;
  if (fa.numRegs != REG_LAUNCH) return cudaErrorInvalidConfiguration;  // the register split needs it
  e = cudaFuncSetAttribute(k_fc_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  P.dstatus = dstatus;
  ++*launches;
  const unsigned ctas = (unsigned)std::max<int64_t>(1, std::min<int64_t>(slots, sm));
  k_fc_gram<<<ctas, THREADS, smem, st>>>(ta, tb, P);
  return cudaGetLastError();
}
