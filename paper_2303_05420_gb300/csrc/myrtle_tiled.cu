// Tiled fused Myrtle NNGP blocks (NK_PREC_MIXED): the ReLU instantiations,
// the tiled form's workspace plan and its launch entry point (the kernel
// templates are in myrtle_tiled.cuh).
#include "myrtle_tiled.cuh"

namespace nkf {

// Stage patterns with a tiled instantiation: stage 0 of one to three convs,
// then at most one conv stage before the global average.
bool tiled_supported(const int c[3]) {
  return (c[0] == 2 && c[1] == 1 && c[2] == 0) || (c[0] == 1 && c[1] == 0 && c[2] == 0) ||
         (c[0] == 1 && c[1] == 1 && c[2] == 0);
}

size_t tiled_ws_bytes(const int c[3], const int* R, const int64_t* npairs, int n, int sm_count, int tensors) {
  // an upper bound of what launch_tiled asks for (it runs one 512-thread or
  // two 256-thread CTAs per SM; four are assumed here)
  return (size_t)sched::make_plan(c[1] > 0, R, npairs, n, 4 * sm_count, tensors).bytes;
}

// Erf instantiations (myrtle_tiled_erf.cu).
cudaError_t launch_tiled_erf(const int c[3], bool bias, tiled::TiledParams& Q, const int64_t* np, int sm_count,
                             void* ws, size_t ws_bytes, cudaStream_t st);

cudaError_t launch_tiled(const int c[3], bool bias, int act, const int* R, const FusedParams* B, int n,
                         int sm_count, void* ws, size_t ws_bytes, unsigned int* dstatus, long long wait_limit,
                         cudaStream_t st) {
  if (n < 1 || n > QUEUE_MAX || !tiled_supported(c)) return cudaErrorNotSupported;
  tiled::TiledParams Q;
  int64_t np[QUEUE_MAX];
  if (!tiled::make_queue(Q, np, R, B, n, dstatus, wait_limit)) return cudaErrorInvalidValue;
  if (act == NK_ACT_ERF) return launch_tiled_erf(c, bias, Q, np, sm_count, ws, ws_bytes, st);
  if (act != NK_ACT_RELU) return cudaErrorNotSupported;
  return tiled::launch_act<NK_ACT_RELU>(c, bias, Q, np, sm_count, ws, ws_bytes, st);
}

}  // namespace nkf
