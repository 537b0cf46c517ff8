// Fused Myrtle blocks of several image sizes in one persistent launch (the
// paper computes blocks of the kernel matrix independently and batches them
// to fill the device, Figure 1).  A queue item is one 32x32 pair (taken by
// the four CTAs of a cluster together) or four 16x16 / 8x8 pairs (one per
// CTA of the cluster).  Items are walked statically, item = cluster +
// k * clusters, largest first, so that the short items fill the tail.
#include <algorithm>

#include "myrtle_fused.cuh"

namespace nkf {

template <int N0, int N1, int N2, bool BIAS>
__global__ void __launch_bounds__(Variant<0>::THREADS, 1)
    k_myrtle_queue(const __grid_constant__ QueueParams Q) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int CL = QUEUE_CL;
  const unsigned rank = cluster_rank();
  const int64_t cid = blockIdx.x / CL;
  const int64_t ncl = gridDim.x / CL;
  const int64_t nitems = Q.item0[Q.n];
  int iter = 0;  // 32x32 pairs of this cluster (slot parity)
  for (int64_t it = cid; it < nitems; it += ncl) {
    int b = 0;
    while (b + 1 < Q.n && it >= Q.item0[b + 1]) ++b;
    const FusedParams& P = Q.B[b];
    const int64_t k = it - Q.item0[b];
    if (Q.R[b] == 32) {
      int64_t i, j;
      pair_ij(k, P.na, P.nb, P.sym, &i, &j);
      const double s = pair_body<32, N0, N1, N2, CL, BIAS, 0>(P, P.a0 + i, P.b0 + j, smem, rank);
      cluster_combine<CL>(P, Q.gacc, Q.gcnt, cid * 2 + (iter & 1), i, j, s);
      ++iter;
    } else {
      // one pair per CTA, no cluster barrier inside
      const int64_t pidx = k * CL + rank;
      if (pidx < P.npairs) {
        int64_t i, j;
        pair_ij(pidx, P.na, P.nb, P.sym, &i, &j);
        double s;
        if (Q.R[b] == 16)
          s = pair_body<16, N0, N1, N2, 1, BIAS, 0>(P, P.a0 + i, P.b0 + j, smem, 0u);
        else
          s = pair_body<8, N0, N1, N2, 1, BIAS, 0>(P, P.a0 + i, P.b0 + j, smem, 0u);
        cluster_combine<1>(P, nullptr, nullptr, 0, i, j, s);
      }
    }
  }
}

template <int N0, int N1, int N2, bool BIAS>
cudaError_t launch_queue_t(QueueParams& Q, int sm_count, void* scratch, size_t scratch_bytes,
                           cudaStream_t st) {
  constexpr int CL = QUEUE_CL;
  auto kern = k_myrtle_queue<N0, N1, N2, BIAS>;
  const size_t smem = std::max(Layout<32, N0, N1, N2, CL>::bytes,
                               std::max(Layout<16, N0, N1, N2, 1>::bytes, Layout<8, N0, N1, N2, 1>::bytes));
  static bool attr_set[64] = {false};
  int adev = 0;
  if (cudaGetDevice(&adev) != cudaSuccess || adev < 0 || adev >= 64) adev = 0;
  cudaError_t e = cudaSuccess;
  if (!attr_set[adev]) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set[adev] = true;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(Variant<0>::THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(CL, 1, 1);
  // resident clusters, looked up once per device (no query inside a capture
  // after the first call)
  static int maxc_of_device[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  int nclusters = sm_count / CL;
  if (maxc_of_device[dev] == 0) {
    int maxc = 0;
    if (cudaOccupancyMaxActiveClusters(&maxc, kern, &cfg) == cudaSuccess && maxc > 0)
      maxc_of_device[dev] = maxc;
    else
      (void)cudaGetLastError();
  }
  if (maxc_of_device[dev] > 0) nclusters = maxc_of_device[dev];
  const int64_t nitems = Q.item0[Q.n];
  if (nclusters > nitems) nclusters = (int)nitems;
  if (nclusters < 1) nclusters = 1;
  const size_t need = (size_t)nclusters * 2 * (sizeof(double) + sizeof(int));
  if (need > scratch_bytes) return cudaErrorInvalidValue;
  Q.gacc = reinterpret_cast<double*>(scratch);
  Q.gcnt = reinterpret_cast<int*>(reinterpret_cast<char*>(scratch) + (size_t)nclusters * 2 * sizeof(double));
  e = cudaMemsetAsync(scratch, 0, need, st);
  if (e != cudaSuccess) return e;
  cfg.gridDim = dim3((unsigned)(nclusters * CL), 1, 1);
  e = cudaLaunchKernelEx(&cfg, kern, Q);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_queue(const int c[3], bool bias, QueueParams& Q, int sm_count, void* scratch,
                         size_t scratch_bytes, cudaStream_t st) {
#define NK_Q(a, b_, d)                                                                          \
  if (c[0] == a && c[1] == b_ && c[2] == d)                                                     \
    return bias ? launch_queue_t<a, b_, d, true>(Q, sm_count, scratch, scratch_bytes, st)       \
                : launch_queue_t<a, b_, d, false>(Q, sm_count, scratch, scratch_bytes, st);
  NK_Q(2, 1, 0) NK_Q(2, 1, 1) NK_Q(3, 3, 3) NK_Q(1, 0, 0) NK_Q(1, 1, 1)
#undef NK_Q
  return cudaErrorNotSupported;
}

}  // namespace nkf
