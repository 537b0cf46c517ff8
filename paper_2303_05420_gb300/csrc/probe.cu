// nk_probe: peak-rate probes of the GPU the library runs on (declared in
// include/nk_probe.h).  The kernels' roofline fractions divide by these.
//
//   FP32 / FP64 FMA: every thread runs 8 independent FMA chains (enough to
//     cover the FMA latency at full occupancy); rate = lane-FMAs per second.
//   L2 / HBM read: every thread streams float4 loads that bypass L1
//     (ld.global.cg) over a buffer, summing them; rate = bytes per second.
//     A buffer of at most 64 MB stays in L2 after a first pass; one of at
//     least 512 MB (four times L2) comes from HBM.
#include <algorithm>

#include "nk_common.cuh"
#include "nk_probe.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_probe_fma(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
  // 32 x 8 FMAs per loop trip: the loop's own three instructions cost about
  // 1 % of the issue slots
#pragma unroll 32
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == (T)-1.2345e6) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(256) k_probe_read(const float4* __restrict__ buf, int64_t n4, int passes,
                                                    float* out) {
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float s = 0.f;
  for (int p = 0; p < passes; ++p) {
    int64_t e = t0;
    for (; e + 3 * nt < n4; e += 4 * nt) {
      const float4 u0 = __ldcg(buf + e), u1 = __ldcg(buf + e + nt), u2 = __ldcg(buf + e + 2 * nt),
                   u3 = __ldcg(buf + e + 3 * nt);
      s += (u0.x + u1.y) + (u2.z + u3.w);
    }
    for (; e < n4; e += nt) s += __ldcg(buf + e).x;
  }
  if (s == -1.2345e6f) out[t0] = s;
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

}  // namespace

extern "C" nk_status nk_probe(int which, int64_t work, double* rate, double* ms, void* stream) {
  if (!rate || !ms) return NK_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return NK_ERR_CUDA;
  const unsigned threads = 256;
  Timer t;
  if (cudaEventCreate(&t.a) != cudaSuccess || cudaEventCreate(&t.b) != cudaSuccess) return NK_ERR_CUDA;
  float elapsed = 0.f;
  if (which == NK_PROBE_FP32_FMA || which == NK_PROBE_FP64_FMA) {
    const bool f64 = which == NK_PROBE_FP64_FMA;
    int iters = (int)(work > 0 ? std::min<int64_t>(work, 1 << 26) : (f64 ? (1 << 11) : (1 << 16)));
    iters = (iters + 31) / 32 * 32;
    const unsigned blocks = (unsigned)sm * 8;  // 2048 threads per SM
    void* out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * threads * 8) != cudaSuccess) return NK_ERR_NO_MEMORY;
    for (int rep = 0; rep < 2; ++rep) {
      e = cudaEventRecord(t.a, st);
      if (f64)
        k_probe_fma<double><<<blocks, threads, 0, st>>>((double*)out, iters, 0.999999, 1e-7);
      else
        k_probe_fma<float><<<blocks, threads, 0, st>>>((float*)out, iters, 0.9999f, 1e-4f);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(t.b, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(t.b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&elapsed, t.a, t.b);
      if (e != cudaSuccess) break;
    }
    cudaFree(out);
    if (e != cudaSuccess) return NK_ERR_CUDA;
    *ms = elapsed;
    *rate = (double)blocks * threads * iters * 8.0 / (elapsed * 1e-3);
    return NK_OK;
  }
  if (which == NK_PROBE_L2_READ || which == NK_PROBE_HBM_READ) {
    const bool l2 = which == NK_PROBE_L2_READ;
    int64_t bytes = work > 0 ? work : (l2 ? ((int64_t)32 << 20) : ((int64_t)1 << 30));
    if (l2 && (bytes < (1 << 20) || bytes > ((int64_t)64 << 20))) return NK_ERR_INVALID_ARG;
    if (!l2 && (bytes < ((int64_t)512 << 20) || bytes > ((int64_t)16 << 30))) return NK_ERR_INVALID_ARG;
    bytes = bytes / 16 * 16;
    const int passes = l2 ? 16 : 1;
    const unsigned blocks = (unsigned)sm * 4;  // 1024 threads per SM, 64 B of loads in flight each
    void* buf = nullptr;
    void* out = nullptr;
    if (cudaMalloc(&buf, (size_t)bytes) != cudaSuccess) return NK_ERR_NO_MEMORY;
    if (cudaMalloc(&out, (size_t)blocks * threads * 4) != cudaSuccess) {
      cudaFree(buf);
      return NK_ERR_NO_MEMORY;
    }
    e = cudaMemsetAsync(buf, 0, (size_t)bytes, st);
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(t.a, st);
      k_probe_read<<<blocks, threads, 0, st>>>((const float4*)buf, bytes / 16, passes, (float*)out);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(t.b, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(t.b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&elapsed, t.a, t.b);
    }
    cudaFree(buf);
    cudaFree(out);
    if (e != cudaSuccess) return NK_ERR_CUDA;
    *ms = elapsed;
    *rate = (double)bytes * passes / (elapsed * 1e-3);
    return NK_OK;
  }
  return NK_ERR_INVALID_ARG;
}
