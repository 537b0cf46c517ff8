// Fused Myrtle NNGP block (NK_PREC_MIXED): host-side argument set-up and
// dispatch to the per-size instantiations (kernel in myrtle_fused.cuh).
#include "myrtle_fused.cuh"

// Stage patterns of the super-plane cluster kernel (ReLU, sides 8, 16, 32).
bool nk_cluster_pattern(const int c[3]) {
  return (c[0] == 2 && c[1] == 1 && c[2] == 0) || (c[0] == 2 && c[1] == 1 && c[2] == 1) ||
         (c[0] == 3 && c[1] == 3 && c[2] == 3) || (c[0] == 1 && c[1] == 0 && c[2] == 0) ||
         (c[0] == 1 && c[1] == 1 && c[2] == 1);
}

// A fused form exists: the tiled form at 64x64, at 32x32 for its patterns
// (ReLU or Erf), or the cluster kernel (ReLU) at 8, 16, 32.  Stages beyond the
// third must be empty (pool then global average equals global average).
bool nk_myrtle_fused_supported(const NkGeom& g) {
  if (g.filter != 3 || (g.act != NK_ACT_RELU && g.act != NK_ACT_ERF) || g.C < 1 || g.C > 3) return false;
  if (g.readout != NK_READOUT_GAP) return false;
  if (g.Hs[0] != g.Ws[0]) return false;
  const int R0 = g.Hs[0];
  if (R0 != 8 && R0 != 16 && R0 != 32 && R0 != 64) return false;
  int c[3] = {0, 0, 0};
  for (int s = 0; s < g.n_stages; ++s) {
    if (s >= 3) {
      if (g.convs[s] != 0) return false;
      continue;
    }
    c[s] = g.convs[s];
  }
  if (R0 == 64) return nkf::tiled_supported(c);
  if (R0 == 32 && nkf::tiled_supported(c)) return true;
  return g.act == NK_ACT_RELU && nk_cluster_pattern(c);
}

// Kernel parameters of one block (everything but the scratch slots).
nkf::FusedParams nk_fused_params(const NkGeom& g, double sw2, double sb2, const float* Xa, const float* qsa,
                                 int64_t a0, int64_t a1, const float* Xb, const float* qsb, int64_t b0,
                                 int64_t b1, float* K, int64_t ldk, int symmetric) {
  nkf::FusedParams P = {};
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
  P.K = K;
  P.ldk = ldk;
  P.C = g.C;
  P.nq = g.nq;
  int c[3] = {g.convs[0], g.n_stages > 1 ? g.convs[1] : 0, g.n_stages > 2 ? g.convs[2] : 0};
  const int SE = 1 + (c[1] > 0) + (c[1] > 0 && c[2] > 0);
  const double a = sw2 / 9.0;
  // the activation's constant: 1/(2 pi) of the arc-cosine map, 2/pi of Erf's
  const double inv2pi = g.act == NK_ACT_ERF ? 0.63661977236758134308 : 0.15915494309189533577;
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
  return P;
}

cudaError_t nk_launch_myrtle_fused(const NkGeom& g, double sw2, double sb2, const float* Xa,
                                   const float* qsa, int64_t a0, int64_t a1, const float* Xb,
                                   const float* qsb, int64_t b0, int64_t b1, float* K,
                                   int64_t ldk, int symmetric, int sm_count, void* scratch,
                                   size_t scratch_bytes, int variant, cudaStream_t st) {
  const int pat[3] = {g.convs[0], g.n_stages > 1 ? g.convs[1] : 0, g.n_stages > 2 ? g.convs[2] : 0};
  if (!nk_myrtle_fused_supported(g) || g.act != NK_ACT_RELU || !nk_cluster_pattern(pat)) return cudaErrorNotSupported;
  nkf::FusedParams P = nk_fused_params(g, sw2, sb2, Xa, qsa, a0, a1, Xb, qsb, b0, b1, K, ldk, symmetric);
  if (P.npairs <= 0) return cudaSuccess;
  int c[3] = {g.convs[0], g.n_stages > 1 ? g.convs[1] : 0, g.n_stages > 2 ? g.convs[2] : 0};
  const int R0 = g.Hs[0];
  const bool bias = (sb2 != 0.0);
  const int v = (R0 == 32) ? variant : 0;
  if (R0 == 32) return nkf::dispatch_r32(c, bias, v, P, sm_count, scratch, scratch_bytes, st);
  if (R0 == 16) return nkf::dispatch_r16(c, bias, v, P, sm_count, scratch, scratch_bytes, st);
  if (R0 == 8) return nkf::dispatch_r8(c, bias, v, P, sm_count, scratch, scratch_bytes, st);
  return cudaErrorNotSupported;
}
