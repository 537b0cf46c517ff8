// Tiled fused Myrtle NTK blocks (NK_PREC_MIXED of nk_block_ntk): the row
// stream of myrtle_tiled.cuh with the tangent rows (Band<..., NTK = true>),
// ReLU, stage pattern (2,1,0).  A translation unit of its own so that the
// build compiles it beside the NNGP ones.
#include "myrtle_tiled.cuh"

namespace nkf {

bool tiled_ntk_supported(const int c[3]) { return c[0] == 2 && c[1] == 1 && c[2] == 0; }

cudaError_t launch_tiled_ntk(const int c[3], bool bias, const int* R, const FusedParams* B, int n, int sm_count,
                             void* ws, size_t ws_bytes, unsigned int* dstatus, long long wait_limit,
                             cudaStream_t st) {
  if (n < 1 || n > QUEUE_MAX || !tiled_ntk_supported(c)) return cudaErrorNotSupported;
  for (int b = 0; b < n; ++b)
    if (!B[b].Th) return cudaErrorInvalidValue;
  tiled::TiledParams Q;
  int64_t np[QUEUE_MAX];
  if (!tiled::make_queue(Q, np, R, B, n, dstatus, wait_limit)) return cudaErrorInvalidValue;
  using namespace tiled;
  if (Q.G64 == 0)
    return bias ? launch_t<2, 1, true, 256, 32, NK_ACT_RELU, true>(Q, np, sm_count, ws, ws_bytes, st)
                : launch_t<2, 1, false, 256, 32, NK_ACT_RELU, true>(Q, np, sm_count, ws, ws_bytes, st);
  return bias ? launch_t<2, 1, true, 512, 64, NK_ACT_RELU, true>(Q, np, sm_count, ws, ws_bytes, st)
              : launch_t<2, 1, false, 512, 64, NK_ACT_RELU, true>(Q, np, sm_count, ws, ws_bytes, st);
}

}  // namespace nkf
