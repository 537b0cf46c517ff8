// Tiled fused Myrtle blocks of three-stage nets at 32x32 (Myrtle-10 (3,3,3),
// and (2,1,1)), ReLU, NNGP and NTK: the stage-0 tasks as in the two-stage
// form, and a stage-1 task that pools its 16x16 stage into an 8x8 stage-2
// tile in shared memory and runs stage 2 on the same CTA before the global
// average (myrtle_tiled.cuh, N2 > 0).  The three-layer stage-0 tables take
// 122 KB, so the launch is one CTA of 512 threads per SM.  A translation
// unit of its own so that the build compiles it beside the others.
#include "myrtle_tiled.cuh"

namespace nkf {

bool tiled3_supported(const int c[3]) {
  return (c[0] == 3 && c[1] == 3 && c[2] == 3) || (c[0] == 2 && c[1] == 1 && c[2] == 1);
}

cudaError_t launch_tiled3(const int c[3], bool bias, bool ntk, const int* R, const FusedParams* B, int n,
                          int sm_count, void* ws, size_t ws_bytes, unsigned int* dstatus, long long wait_limit,
                          cudaStream_t st) {
  if (n < 1 || n > QUEUE_MAX || !tiled3_supported(c)) return cudaErrorNotSupported;
  for (int b = 0; b < n; ++b) {
    if (R[b] != 32) return cudaErrorNotSupported;
    if (ntk && !B[b].Th) return cudaErrorInvalidValue;
  }
  tiled::TiledParams Q;
  int64_t np[QUEUE_MAX];
  if (!tiled::make_queue(Q, np, R, B, n, dstatus, wait_limit)) return cudaErrorInvalidValue;
  using namespace tiled;
#define NK_T3(a, b_, c_)                                                                                   \
  if (c[0] == a && c[1] == b_ && c[2] == c_) {                                                             \
    if (ntk)                                                                                               \
      return bias ? launch_t<a, b_, true, 512, 32, NK_ACT_RELU, true, c_>(Q, np, sm_count, ws, ws_bytes, st) \
                  : launch_t<a, b_, false, 512, 32, NK_ACT_RELU, true, c_>(Q, np, sm_count, ws, ws_bytes, st); \
    return bias ? launch_t<a, b_, true, 512, 32, NK_ACT_RELU, false, c_>(Q, np, sm_count, ws, ws_bytes, st)    \
                : launch_t<a, b_, false, 512, 32, NK_ACT_RELU, false, c_>(Q, np, sm_count, ws, ws_bytes, st);  \
  }
  NK_T3(3, 3, 3) NK_T3(2, 1, 1)
#undef NK_T3
  return cudaErrorNotSupported;
}

}  // namespace nkf
