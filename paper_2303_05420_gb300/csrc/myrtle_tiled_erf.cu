// Tiled fused Myrtle NNGP blocks (NK_PREC_MIXED) with the Erf activation,
// E[erf(u) erf(v)] = (2/pi) asin(2 K / sqrt((1 + 2 q)(1 + 2 q'))) at every
// layer (the row stream of myrtle_tiled.cuh with nk_asin_f32 as the map; the
// factors sqrt(2 / (m + 2 q)) and 2/pi come from the tables).  A translation
// unit of its own so that the build compiles it beside the ReLU one.
#include "myrtle_tiled.cuh"

namespace nkf {

cudaError_t launch_tiled_erf(const int c[3], bool bias, tiled::TiledParams& Q, const int64_t* np, int sm_count,
                             void* ws, size_t ws_bytes, cudaStream_t st) {
  return tiled::launch_act<NK_ACT_ERF>(c, bias, Q, np, sm_count, ws, ws_bytes, st);
}

}  // namespace nkf
