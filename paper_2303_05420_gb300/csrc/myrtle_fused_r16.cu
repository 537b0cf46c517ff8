// Instantiations of the fused Myrtle kernel for 16x16 images.
#include "myrtle_fused.cuh"

namespace nkf {

cudaError_t dispatch_r16(const int c[3], bool bias, int variant, FusedParams& P, int sm_count,
                         void* scratch, size_t scratch_bytes, cudaStream_t st) {
  if (c[0] == 2 && c[1] == 1 && c[2] == 0 && variant == 0 && bias == true)
    return launch<16, 2, 1, 0, 1, true, 0>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 2 && c[1] == 1 && c[2] == 0 && variant == 0 && bias == false)
    return launch<16, 2, 1, 0, 1, false, 0>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 2 && c[1] == 1 && c[2] == 1 && variant == 0 && bias == true)
    return launch<16, 2, 1, 1, 1, true, 0>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 2 && c[1] == 1 && c[2] == 1 && variant == 0 && bias == false)
    return launch<16, 2, 1, 1, 1, false, 0>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 3 && c[1] == 3 && c[2] == 3 && variant == 0 && bias == true)
    return launch<16, 3, 3, 3, 1, true, 0>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 3 && c[1] == 3 && c[2] == 3 && variant == 0 && bias == false)
    return launch<16, 3, 3, 3, 1, false, 0>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 1 && c[1] == 0 && c[2] == 0 && variant == 0 && bias == true)
    return launch<16, 1, 0, 0, 1, true, 0>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 1 && c[1] == 0 && c[2] == 0 && variant == 0 && bias == false)
    return launch<16, 1, 0, 0, 1, false, 0>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 1 && c[1] == 1 && c[2] == 1 && variant == 0 && bias == true)
    return launch<16, 1, 1, 1, 1, true, 0>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 1 && c[1] == 1 && c[2] == 1 && variant == 0 && bias == false)
    return launch<16, 1, 1, 1, 1, false, 0>(P, sm_count, scratch, scratch_bytes, st);
  return cudaErrorNotSupported;
}

}  // namespace nkf
