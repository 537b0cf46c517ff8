// Instantiations of the fused Myrtle kernel for 32x32 images, launch variant 2.
#include "myrtle_fused.cuh"

namespace nkf {

cudaError_t dispatch_r32_v2(const int c[3], bool bias, int variant, FusedParams& P, int sm_count,
                             void* scratch, size_t scratch_bytes, cudaStream_t st) {
  if (c[0] == 2 && c[1] == 1 && c[2] == 0 && variant == 2 && bias == true)
    return launch<32, 2, 1, 0, 4, true, 2>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 2 && c[1] == 1 && c[2] == 0 && variant == 2 && bias == false)
    return launch<32, 2, 1, 0, 4, false, 2>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 2 && c[1] == 1 && c[2] == 1 && variant == 2 && bias == true)
    return launch<32, 2, 1, 1, 4, true, 2>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 2 && c[1] == 1 && c[2] == 1 && variant == 2 && bias == false)
    return launch<32, 2, 1, 1, 4, false, 2>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 3 && c[1] == 3 && c[2] == 3 && variant == 2 && bias == true)
    return launch<32, 3, 3, 3, 4, true, 2>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 3 && c[1] == 3 && c[2] == 3 && variant == 2 && bias == false)
    return launch<32, 3, 3, 3, 4, false, 2>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 1 && c[1] == 0 && c[2] == 0 && variant == 2 && bias == true)
    return launch<32, 1, 0, 0, 4, true, 2>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 1 && c[1] == 0 && c[2] == 0 && variant == 2 && bias == false)
    return launch<32, 1, 0, 0, 4, false, 2>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 1 && c[1] == 1 && c[2] == 1 && variant == 2 && bias == true)
    return launch<32, 1, 1, 1, 4, true, 2>(P, sm_count, scratch, scratch_bytes, st);
  if (c[0] == 1 && c[1] == 1 && c[2] == 1 && variant == 2 && bias == false)
    return launch<32, 1, 1, 1, 4, false, 2>(P, sm_count, scratch, scratch_bytes, st);
  return cudaErrorNotSupported;
}

}  // namespace nkf
