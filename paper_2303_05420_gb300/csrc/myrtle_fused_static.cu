// nk_block_fused_noalloc: the fused Myrtle kernel block for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a kernel
// block: a serving process whose device memory is reserved up front by its
// own allocator and which forbids new device allocations while it runs, or a
// plugin whose host framework owns all device memory.  nk_block needs an
// nk_handle, and nk_create allocates.  This entry point takes no handle and allocates
// nothing: the only scratch the fused kernel needs -- two per-cluster slots
// holding the global-average sum (8 bytes) and an arrival counter (4 bytes)
// -- lives in a fixed file-scope device array below.
//
// The array is shared by every call in the process on a given device and
// keeps the previous call's contents: the slots a launch uses are cleared
// (stream-ordered memset) before the launch.  Two calls whose kernels overlap
// on the GPU (different streams, no ordering between them) use the same
// slots and race; order them on one stream or serialise them.
#include <cuda.h>
#include <stdio.h>

#include <mutex>

#include "myrtle_fused.cuh"

namespace {

// 16 KB: 2 slots x 12 bytes per cluster covers 682 clusters, far more than
// the SM count of any current GPU (152 SMs on GB300 give at most 152
// clusters of one CTA).
constexpr size_t kNoallocScratchBytes = 16384;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of g_noalloc_scratch for each device ordinal, looked up
// with that device current by the first call on it, and again whenever the
// device's current context is not the one the address was taken in (after a
// cudaDeviceReset the module is loaded anew and the array may move).
// Contexts are told apart by their process-unique ids (cuCtxGetId).  In host
// code the array's name is only a host-side stand-in, never a device
// address.  The table is shared by all host threads, under g_mu.
constexpr int kMaxDevices = 64;
struct ScratchAddr {
  unsigned long long ctx_id;  // 0: none recorded
  void* addr;
};
std::mutex g_mu;
ScratchAddr g_addr[kMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Id of the calling thread's current context; 0 when there is none or the
// driver does not tell (the caller then looks the address up every time).
// Called with g_mu held.
unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = (CtxGetCurrentFn)p;
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)p;
    resolved = true;
  }
  if (!get_cur || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// The scratch array's device address for device `dev` (current).
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = current_ctx_id();
  ScratchAddr& s = g_addr[dev];
  if (id == 0 || s.ctx_id != id || !s.addr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    // the lookup makes the device's primary context current if none was
    id = current_ctx_id();
    s.ctx_id = id;
    s.addr = p;
  }
  *out = s.addr;
  return cudaSuccess;
}

void set_err(char* buf, size_t len, const char* msg) {
  if (buf && len) snprintf(buf, len, "%s", msg);
}

}  // namespace

extern "C" nk_status nk_block_fused_noalloc(const nk_arch* arch, const nk_params* prm,
                                            const float* Xa, const float* qsa, int64_t a0,
                                            int64_t a1, const float* Xb, const float* qsb,
                                            int64_t b0, int64_t b1, int H, int W, int C, float* K,
                                            int64_t ldk, int symmetric, void* stream,
                                            char* err_buf, size_t err_len) {
  char msg[256];
  NkGeom g;
  const char* why = nullptr;
  if (!nk_make_geom(arch, H, W, C, &g, &why)) {
    snprintf(msg, sizeof(msg), "nk_block_fused_noalloc: %s", why);
    set_err(err_buf, err_len, msg);
    return NK_ERR_INVALID_ARG;
  }
  if (!prm || !(prm->sigma_w2 >= 0.0) || !(prm->sigma_b2 >= 0.0) || a0 < 0 || b0 < 0 || a1 < a0 ||
      b1 < b0 || ldk < b1 - b0 || (symmetric && (Xa != Xb || a0 != b0 || a1 != b1))) {
    set_err(err_buf, err_len, "nk_block_fused_noalloc: invalid parameters, ranges, ldk or symmetric flag");
    return NK_ERR_INVALID_ARG;
  }
  if (a1 == a0 || b1 == b0) return NK_OK;
  if (!Xa || !Xb || !qsa || !qsb || !K) {
    set_err(err_buf, err_len, "nk_block_fused_noalloc: NULL pointer");
    return NK_ERR_INVALID_ARG;
  }
  const int pat[3] = {g.convs[0], g.n_stages > 1 ? g.convs[1] : 0, g.n_stages > 2 ? g.convs[2] : 0};
  if (!nk_myrtle_fused_supported(g) || g.act != NK_ACT_RELU || !nk_cluster_pattern(pat)) {
    set_err(err_buf, err_len,
            "nk_block_fused_noalloc: no fused kernel for this architecture / size (see nk_block)");
    return NK_ERR_UNSUPPORTED;
  }
  if (g.Hs[0] == 64) {
    // the 64x64 (tiled) form keeps its pooled stage-1 tensors in a ring of
    // global slots of tens of MB: it needs nk_block and its workspace
    set_err(err_buf, err_len, "nk_block_fused_noalloc: 64x64 images need nk_block (slot workspace)");
    return NK_ERR_UNSUPPORTED;
  }
  int dev = 0, sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    set_err(err_buf, err_len, cudaGetErrorString(e));
    return NK_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_err(err_buf, err_len, "nk_block_fused_noalloc: device ordinal above 63");
    return NK_ERR_INVALID_ARG;
  }
  // set-up once per device (and context), with that device current
  void* scratch = nullptr;
  e = scratch_address(dev, &scratch);
  if (e != cudaSuccess) {
    set_err(err_buf, err_len, cudaGetErrorString(e));
    (void)cudaGetLastError();
    return NK_ERR_CUDA;
  }
  // the launch uses at most one cluster per SM; reject a GPU whose clusters
  // would not fit the fixed array
  const size_t need = (size_t)sm * 2 * (sizeof(double) + sizeof(int));
  if (need > kNoallocScratchBytes) {
    snprintf(msg, sizeof(msg),
             "nk_block_fused_noalloc: %d SMs need %zu bytes of scratch, the fixed array holds %zu",
             sm, need, kNoallocScratchBytes);
    set_err(err_buf, err_len, msg);
    return NK_ERR_INVALID_ARG;
  }
  e = nk_launch_myrtle_fused(g, prm->sigma_w2, prm->sigma_b2, Xa, qsa, a0, a1, Xb, qsb, b0, b1, K, ldk,
                             symmetric, sm, scratch, kNoallocScratchBytes, 0,
                             (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_err(err_buf, err_len, cudaGetErrorString(e));
    (void)cudaGetLastError();
    return NK_ERR_CUDA;
  }
  return NK_OK;
}
