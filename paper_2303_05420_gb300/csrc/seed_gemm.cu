// The first layer of the Myrtle recursion as a patch Gram on the tensor
// cores (Appendix A: the first stax.Conv acts on the channel contraction of
// the two images).  With SAME zero padding and the divisor 9 at every pixel,
//
//   K_1(p, p') = sw2 / (9 C) sum_{|dy|,|dx| <= 1} sum_c x(p + d, c) x'(p' + d, c) + sb2
//              = sw2 / (9 C) <P(p), P'(p')> + sb2,
//
// where P(p) is the 3 x 3 x C patch of x around p with zeros outside the
// image (27 values for C = 3).  Over all pixel pairs of an image pair that is
// the GEMM D = P P'^T (HW x HW, K = 9C <= 32), written row-major [p][p'],
// which is the layout in which the adjoint (myrtle_backward.cu) stores the
// first layer's pre-activation.
//
// Operands: each patch, zero-padded to 32 values, is split once into BF16
// parts hi = bf16(v), lo = bf16(v - hi) and stored as one 128-byte row
// [hi 0..31 | lo 0..31] per pixel (k_patch_split).  A tile of 128 rows p x
// 256 columns p' is one TMA stage (16 + 32 KB, 128-byte swizzle) and six
// tcgen05 MMAs (kind::f16, 128 x 256 x 16, FP32 accumulation in TMEM): the
// two small products hi.lo' and lo.hi' first, then hi.hi' (the dropped
// lo.lo' term is 2^-18 of a product).  The sum has only 2 x 27 + 27 terms,
// so the accumulator's rounding does not drift.
//
// Persistent kernel, one CTA per SM: warp 0 issues the TMA loads into a
// 3-stage mbarrier ring, warp 1 owns TMEM (two 128 x 256 FP32 accumulators)
// and issues the MMAs, eight epilogue warps drain one accumulator (32 rows x
// 128 columns a warp, 32 columns at a time) while the MMAs fill the other.
// A tcgen05.ld gives each lane 32 columns of its own row; the warp turns the
// 32 x 32 block around in shared memory so that each store instruction
// writes 128 contiguous bytes of one row (a lane-per-row store wrote 16
// bytes into 32 different rows: eight times the L2 write requests).  The
// output (4 MB per 32 x 32 image pair) makes it an HBM-write-bound kernel.
// Every mbarrier wait is bounded; a timeout sets NK_DEV_TIMEOUT, skips the
// remaining work, and the kernel still waits for its own copies and MMAs and
// frees TMEM before it exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "myrtle_plain.cuh"
#include "tc_gemm.cuh"

namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 3;
constexpr int EPI_WARPS = 8, EPI_COLS = BN / 2;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t DRAIN_LIMIT = 1u << 26;

constexpr int STG = 33;  // row stride of a warp's 32 x 32 staging tile (odd: no bank conflicts)

struct SeedSmem {
  alignas(1024) __nv_bfloat16 A[STAGES][BM * BK];
  alignas(1024) __nv_bfloat16 B[STAGES][BN * BK];
  float stage[EPI_WARPS][32 * STG];  // epilogue: 32 rows x 32 columns, transposed for row-contiguous stores
  uint64_t full[STAGES], empty[STAGES];
  uint64_t tfull[2], tempty[2];  // accumulators: MMA -> epilogue, epilogue -> MMA
  uint64_t done;
  uint32_t tslot;
};

struct SeedParams {
  int64_t np, pair0, na, nb;  // pairs of this chunk, first pair, block shape
  int sym;
  int HW;                     // pixels per image (multiple of 256)
  int tm, tn;                 // tiles per pair along p and p'
  float scale, bias;          // sw2 / (9 C), sb2
  float* out;                 // [np][HW][HW]
  unsigned int* dstatus;
  uint32_t wait_limit;
};

// Patch rows of images [0, n) of X (NHWC, H x W x C, C <= 3): row p of
// image i is [hi(P(p)) | lo(P(p))], 64 BF16, element e = ((dy + 1) 3 +
// (dx + 1)) C + c, zero for e >= 9C and outside the image.
__global__ void k_patch_split(const float* __restrict__ X, int64_t n, int H, int W, int C,
                              __nv_bfloat16* __restrict__ out) {
  const int64_t HW = (int64_t)H * W;
  const int64_t total = n * HW * 32;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(t & 31);
    const int64_t r = t >> 5;  // image * HW + pixel
    const int64_t img = r / HW;
    const int p = (int)(r - img * HW);
    float v = 0.f;
    if (e < 9 * C) {
      const int tap = e / C, c = e - tap * C;
      const int y = p / W + tap / 3 - 1, x = p % W + tap % 3 - 1;
      if (y >= 0 && y < H && x >= 0 && x < W) v = X[((img * HW) + (int64_t)y * W + x) * C + c];
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    out[r * 64 + e] = hi;
    out[r * 64 + 32 + e] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

__device__ __forceinline__ void item_of(const SeedParams& P, int64_t t, int64_t& pr, int& tm, int& tn) {
  const int per = P.tm * P.tn;
  pr = t / per;
  const int r = (int)(t - pr * per);
  tm = r / P.tn;
  tn = r - tm * P.tn;
}

__global__ void __launch_bounds__(THREADS, 1)
k_seed_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
            const __grid_constant__ SeedParams P) {
  extern __shared__ __align__(1024) unsigned char raw[];
  SeedSmem& S = *reinterpret_cast<SeedSmem*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t cta = blockIdx.x, ncta = gridDim.x;
  const int64_t nitems = P.np * P.tm * P.tn;
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&S.full[s], 1);
      tc::mbar_init(&S.empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(&S.tfull[a], 1);
      tc::mbar_init(&S.tempty[a], EPI_WARPS);
    }
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
  if (warp == 0) {
    if (lane == 0) {
      int64_t k = 0;  // items of this CTA so far
      for (int64_t t = cta; t < nitems; t += ncta, ++k) {
        int64_t pr;
        int tm, tn;
        item_of(P, t, pr, tm, tn);
        int64_t i, j;
        nkp::pair_of(P.pair0 + pr, P.na, P.nb, P.sym, &i, &j);
        const int s = (int)(k % STAGES);
        if (k >= STAGES && !tc::mbar_wait(&S.empty[s], (uint32_t)((k / STAGES) & 1) ^ 1, P.wait_limit)) {
          atomicOr(P.dstatus, NK_DEV_TIMEOUT);
          break;
        }
        tc::mbar_arrive_expect_tx(&S.full[s], (BM + BN) * BK * 2);
        tc::tma_load_2d(S.A[s], &ta, &S.full[s], 0, (int)(i * P.HW + tm * BM));
        tc::tma_load_2d(S.B[s], &tb, &S.full[s], 0, (int)(j * P.HW + tn * BN));
      }
      // every load issued has landed before the CTA may exit
      for (int64_t m = std::max<int64_t>(0, k - STAGES); m < k; ++m)
        if (!tc::mbar_wait(&S.full[m % STAGES], (uint32_t)((m / STAGES) & 1), DRAIN_LIMIT))
          atomicOr(P.dstatus, NK_DEV_TIMEOUT);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
      // descriptors of stage 0; a stage s and a byte offset o within a
      // 128-byte row move them by (s * stage bytes + o) / 16
      const uint64_t ad0 = tc::sdesc_k128(tc::smem_addr(S.A[0]));
      const uint64_t bd0 = tc::sdesc_k128(tc::smem_addr(S.B[0]));
      constexpr uint64_t A_STEP = BM * BK * 2 / 16, B_STEP = BN * BK * 2 / 16;
      int64_t k = 0;
      for (int64_t t = cta; t < nitems; t += ncta, ++k) {
        const int acc = (int)(k & 1);
        const int64_t use = k >> 1;  // earlier uses of this accumulator
        if (use >= 1 && !tc::mbar_wait(&S.tempty[acc], (uint32_t)((use - 1) & 1), P.wait_limit)) {
          atomicOr(P.dstatus, NK_DEV_TIMEOUT);
          break;
        }
        const int s = (int)(k % STAGES);
        if (!tc::mbar_wait(&S.full[s], (uint32_t)((k / STAGES) & 1), P.wait_limit)) {
          atomicOr(P.dstatus, NK_DEV_TIMEOUT);
          break;
        }
        tc::tc_fence_after();
        const uint64_t ad = ad0 + (uint64_t)s * A_STEP, bd = bd0 + (uint64_t)s * B_STEP;
        const uint32_t td = tbase + (uint32_t)(acc * BN);
        // hi at bytes 0 and 32 of a row (descriptor + 0, + 2), lo at 64, 96 (+ 4, + 6)
        tc::mma_bf16(td, ad + 0, bd + 4, idesc, 0);  // hi.lo'
        tc::mma_bf16(td, ad + 2, bd + 6, idesc, 1);
        tc::mma_bf16(td, ad + 4, bd + 0, idesc, 1);  // lo.hi'
        tc::mma_bf16(td, ad + 6, bd + 2, idesc, 1);
        tc::mma_bf16(td, ad + 0, bd + 0, idesc, 1);  // hi.hi'
        tc::mma_bf16(td, ad + 2, bd + 2, idesc, 1);
        tc::mma_commit(&S.empty[s]);
        tc::mma_commit(&S.tfull[acc]);
      }
      // all MMAs issued by this thread complete before TMEM is released
      tc::mma_commit(&S.done);
      if (!tc::mbar_wait(&S.done, 0, DRAIN_LIMIT)) atomicOr(P.dstatus, NK_DEV_TIMEOUT);
    }
  } else {
    // epilogue: TMEM lane quarter q holds tile rows 32q .. 32q+31; the two
    // warps of a quarter take columns [0, 128) and [128, 256)
    const int q = warp & 3;
    const int cbeg = ((warp - 2) >> 2) * EPI_COLS;
    int64_t k = 0;
    for (int64_t t = cta; t < nitems; t += ncta, ++k) {
      const int acc = (int)(k & 1);
      const bool got = tc::mbar_wait(&S.tfull[acc], (uint32_t)((k >> 1) & 1), P.wait_limit);
      if (!got) {
        atomicOr(P.dstatus, NK_DEV_TIMEOUT);
        break;
      }
      tc::tc_fence_after();
      int64_t pr;
      int tm, tn;
      item_of(P, t, pr, tm, tn);
      const int row0 = tm * BM + 32 * q;  // this warp's first row
      float* obase = P.out + (pr * P.HW + row0) * (int64_t)P.HW + tn * BN + cbeg + lane;
      const uint32_t taddr = tbase + (uint32_t)(acc * BN + cbeg) + ((uint32_t)(32 * q) << 16);
      float* stg = S.stage[warp - 2];
#pragma unroll 1
      for (int c = 0; c < EPI_COLS / 32; ++c) {
        float v[32];
        tc::tmem_ld32(taddr + (uint32_t)(32 * c), v);
#pragma unroll
        for (int e = 0; e < 32; ++e) stg[lane * STG + e] = fmaf(P.scale, v[e], P.bias);
        __syncwarp();
#pragma unroll 8
        for (int r = 0; r < 32; ++r) obase[(int64_t)r * P.HW + 32 * c] = stg[r * STG + lane];
        __syncwarp();
      }
      // this accumulator is free for the item after next
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&S.tempty[acc]);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc(tbase, 512);
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

bool make_map(CUtensorMap* m, void* ptr, int64_t rows, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)BK, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)BK * 2};
  cuuint32_t box[2] = {BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool nk_seed_gemm_supported(int H, int W, int C, int filter) {
  const int HW = H * W;
  return filter == 3 && C >= 1 && C <= 3 && HW % BN == 0 && HW >= BN && HW <= (1 << 16);
}

size_t nk_seed_patch_bytes(int64_t n_images, int H, int W) {
  return (size_t)n_images * H * W * BK * 2;
}

cudaError_t nk_seed_patches(const float* X, int64_t n, int H, int W, int C, void* patches, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t total = n * H * W * 32;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 32));
  k_patch_split<<<grid, 256, 0, st>>>(X, n, H, W, C, reinterpret_cast<__nv_bfloat16*>(patches));
  return cudaGetLastError();
}

cudaError_t nk_launch_seed_gemm(const void* pa, int64_t na, const void* pb, int64_t nb, int sym, int64_t pair0,
                                int64_t np, int H, int W, int C, double sw2, double sb2, float* out, int sm,
                                unsigned int* dstatus, uint32_t wait_limit, cudaStream_t st) {
  const int HW = H * W;
  if (np <= 0) return cudaSuccess;
  CUtensorMap ta, tb;
  if (!make_map(&ta, const_cast<void*>(pa), na * HW, BM) || !make_map(&tb, const_cast<void*>(pb), nb * HW, BN))
    return cudaErrorInvalidValue;
  SeedParams P = {};
  P.np = np;
  P.pair0 = pair0;
  P.na = na;
  P.nb = nb;
  P.sym = sym;
  P.HW = HW;
  P.tm = HW / BM;
  P.tn = HW / BN;
  P.scale = (float)(sw2 / (9.0 * C));
  P.bias = (float)sb2;
  P.out = out;
  P.dstatus = dstatus;
  P.wait_limit = wait_limit;
  const size_t smem = sizeof(SeedSmem) + 1024;
  cudaError_t e = cudaFuncSetAttribute(k_seed_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t items = np * P.tm * P.tn;
  const unsigned ctas = (unsigned)std::max<int64_t>(1, std::min<int64_t>(items, sm));
  k_seed_gemm<<<ctas, THREADS, smem, st>>>(ta, tb, P);
  return cudaGetLastError();
}
