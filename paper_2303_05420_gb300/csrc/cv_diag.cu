// NNGP blocks of conv networks with a Flatten readout (the CV8 listing of
// Appendix A: eight conv(3x3, SAME) + ReLU layers, Flatten, Dense) by the
// diagonal recursion, NK_PREC_MIXED.
//
// The conv stencil of the NNGP recursion moves both pixels of a pair by the
// same offset, so the offset p' - p of a pixel pair never changes; without
// pools nothing else mixes offsets.  The Flatten readout's Dense weights are
// independent per pixel, so only the pairs p' = p of the last layer enter:
//   K(x, x') = sw2 mean_p Kt_L(p, p) + sb2,
// and the whole recursion closes on the H x W diagonal of each pair:
//   K_1(p) = sw2/(9 C) sum_delta x(p + delta) . x'(p + delta) + sb2,
//   K_{l+1}(p) = sw2/9 sum_delta Kt_l(p + delta) + sb2,   Kt_l = map(K_l),
// with zero padding at the borders and the activation's per-pixel factors
// (nk_self_diag's tables) of both images at the same pixel.  That is H W
// values per pair and layer instead of (H W)^2.
//
// One warp per pair: lane = image column.  The warp's H x 32 diagonal tile
// lives in shared memory (4 KB at H = 32) and every layer sweeps it row by
// row in a rolled loop: the vertical taps are the previous row (carried in a
// register, the value the row had before this layer) and the next row (read
// from the tile), the horizontal taps two shuffles, then the map with the
// per-pixel factors of both images (a coalesced 256-byte load per image and
// row) overwrites the row.  Few registers and a small loop body keep many
// warps resident to hide the factor loads (holding the column in unrolled
// register arrays took 255 registers and one CTA per SM).  FP32 recursion,
// the final mean summed in FP64.  Consecutive warps take consecutive pairs,
// so the warps of a CTA mostly share the image of side a in L1.
#include "myrtle_plain.cuh"

namespace {

constexpr int CV_WARPS = 8;

struct CvParams {
  const float* Xa;
  const float* Xb;
  const float2* qa;  // [n][nq] per-pixel factors (a, b) of side a
  const float2* qb;
  int64_t a0, na, b0, nb, npairs;
  int sym;
  int W, C, L;       // image width (<= 32), channels, conv layers
  int nq;
  int act;
  float xscale;      // sw2 / (9 C)
  float cscale;      // sw2 / 9
  float sb2;
  float fold;        // 1/(2 pi) (ReLU) or 2/pi (Erf)
  double out_scale;  // sw2 / (H W)
  double out_bias;   // sb2
  float* K;
  int64_t ldk;
};

// One layer's sweep over the warp's tile: v <- map(a box3(v) + b) row by row.
// FIRST: the first layer (its correlations may be negative; the later ones,
// after a ReLU, are not).  FULL: all 32 lanes are image columns.
template <int H, int ACT, bool FIRST, bool FULL>
__device__ __forceinline__ void cv_layer(const CvParams& P, float (&v)[H][32], const float2* la, const float2* lb,
                                         int lane, float a) {
  const bool col = FULL || lane < P.W;
  const bool hasr = FULL ? lane < 31 : lane + 1 < P.W;
  float prev = 0.f, cur = v[0][lane];
  float2 fa = col ? la[0] : make_float2(0.f, 0.f), fb = col ? lb[0] : make_float2(0.f, 0.f);
#pragma unroll 2
  for (int r = 0; r < H; ++r) {
    const float next = r + 1 < H ? v[r + 1][lane] : 0.f;
    // the factors of the next row are in flight while this row is mapped
    float2 fa1 = fa, fb1 = fb;
    if (col && r + 1 < H) {
      fa1 = la[(r + 1) * P.W];
      fb1 = lb[(r + 1) * P.W];
    }
    const float s = prev + cur + next;
    const float up = __shfl_up_sync(0xffffffffu, s, 1);
    const float dn = __shfl_down_sync(0xffffffffu, s, 1);
    const float k = fmaf(a, s + (lane > 0 ? up : 0.f) + (hasr ? dn : 0.f), P.sb2);
    const float c = k * (fa.x * fb.x);
    float m;
    if constexpr (ACT == NK_ACT_ERF)
      m = nk_asin_f32(c);
    else
      m = FIRST ? nk_J_f32(c) : nk_J01_f32(c);
    v[r][lane] = col ? (fa.y * fb.y) * P.fold * m : 0.f;
    prev = cur;
    cur = next;
    fa = fa1;
    fb = fb1;
  }
  __syncwarp();
}

template <int H, int ACT, bool FULL>
__global__ void __launch_bounds__(32 * CV_WARPS, 6) k_cv_diag(const __grid_constant__ CvParams P) {
  __shared__ float tile[CV_WARPS][H][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool col = FULL || lane < P.W;
  float (&v)[H][32] = tile[warp];
  const int64_t nw = (int64_t)gridDim.x * CV_WARPS;
  for (int64_t pr = (int64_t)blockIdx.x * CV_WARPS + warp; pr < P.npairs; pr += nw) {
    int64_t i, j;
    nkp::pair_of(pr, P.na, P.nb, P.sym, &i, &j);
    const int64_t ia = P.a0 + i, ib = P.b0 + j;
    const float* xa = P.Xa + ia * (int64_t)H * P.W * P.C;
    const float* xb = P.Xb + ib * (int64_t)H * P.W * P.C;
    // channel contraction at every pixel of the column
#pragma unroll 4
    for (int r = 0; r < H; ++r) {
      float u = 0.f;
      if (col) {
        const float* pa = xa + ((int64_t)r * P.W + lane) * P.C;
        const float* pb = xb + ((int64_t)r * P.W + lane) * P.C;
        for (int c = 0; c < P.C; ++c) u = fmaf(pa[c], pb[c], u);
      }
      v[r][lane] = u;
    }
    __syncwarp();
    const float2* ta = P.qa + ia * (int64_t)P.nq + lane;
    const float2* tb = P.qb + ib * (int64_t)P.nq + lane;
    cv_layer<H, ACT, true, FULL>(P, v, ta, tb, lane, P.xscale);
    for (int l = 1; l < P.L; ++l)
      cv_layer<H, ACT, false, FULL>(P, v, ta + (int64_t)l * H * P.W, tb + (int64_t)l * H * P.W, lane, P.cscale);
    double s = 0.0;
    for (int r = 0; r < H; ++r) s += (double)v[r][lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const float out = (float)(P.out_scale * s + P.out_bias);
      P.K[i * P.ldk + j] = out;
      if (P.sym && i != j) P.K[j * P.ldk + i] = out;
    }
    __syncwarp();
  }
}

template <int H>
cudaError_t cv_launch(const CvParams& P, unsigned grid, cudaStream_t st) {
  const bool full = P.W == 32;
  if (P.act == NK_ACT_ERF) {
    if (full)
      k_cv_diag<H, NK_ACT_ERF, true><<<grid, 32 * CV_WARPS, 0, st>>>(P);
    else
      k_cv_diag<H, NK_ACT_ERF, false><<<grid, 32 * CV_WARPS, 0, st>>>(P);
  } else {
    if (full)
      k_cv_diag<H, NK_ACT_RELU, true><<<grid, 32 * CV_WARPS, 0, st>>>(P);
    else
      k_cv_diag<H, NK_ACT_RELU, false><<<grid, 32 * CV_WARPS, 0, st>>>(P);
  }
  return cudaGetLastError();
}

}  // namespace

bool nk_cv_supported(const NkGeom& g) {
  return g.readout == NK_READOUT_FLATTEN && g.n_stages == 1 && g.filter == 3 &&
         (g.act == NK_ACT_RELU || g.act == NK_ACT_ERF) && g.norm == NK_NORM_NONE && g.C >= 1 && g.C <= 4 &&
         (g.Hs[0] == 8 || g.Hs[0] == 16 || g.Hs[0] == 32) && g.Ws[0] >= 1 && g.Ws[0] <= 32;
}

cudaError_t nk_launch_cv_diag(const NkGeom& g, double sw2, double sb2, const float* Xa, const float* qsa,
                              int64_t a0, int64_t a1, const float* Xb, const float* qsb, int64_t b0, int64_t b1,
                              float* K, int64_t ldk, int symmetric, int sm_count, cudaStream_t st) {
  if (!nk_cv_supported(g)) return cudaErrorNotSupported;
  CvParams P = {};
  P.Xa = Xa;
  P.Xb = Xb;
  P.qa = reinterpret_cast<const float2*>(qsa);
  P.qb = reinterpret_cast<const float2*>(qsb);
  P.a0 = a0;
  P.na = a1 - a0;
  P.b0 = b0;
  P.nb = b1 - b0;
  P.sym = symmetric;
  P.npairs = symmetric ? P.na * (P.na + 1) / 2 : P.na * P.nb;
  if (P.npairs <= 0) return cudaSuccess;
  P.W = g.Ws[0];
  P.C = g.C;
  P.L = g.convs[0];
  P.nq = g.nq;
  P.act = g.act;
  P.xscale = (float)(sw2 / (9.0 * g.C));
  P.cscale = (float)(sw2 / 9.0);
  P.sb2 = (float)sb2;
  P.fold = g.act == NK_ACT_ERF ? 0.63661977236758134308f : 0.15915494309189533577f;
  P.out_scale = sw2 / ((double)g.Hs[0] * g.Ws[0]);
  P.out_bias = sb2;
  P.K = K;
  P.ldk = ldk;
  const int64_t want = (P.npairs + CV_WARPS - 1) / CV_WARPS;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count * 32));
  switch (g.Hs[0]) {
    case 8: return cv_launch<8>(P, grid, st);
    case 16: return cv_launch<16>(P, grid, st);
    default: return cv_launch<32>(P, grid, st);
  }
}
