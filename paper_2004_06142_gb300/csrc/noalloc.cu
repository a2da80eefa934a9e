// donof_energy_lagrangian_noalloc: a build that allocates no device memory.
//
// Some callers cannot allocate device memory at the moment they need a build: a host
// framework may own the whole device pool through its own allocator and forbid other
// allocations, or the call may sit in a loop where a cudaMalloc (which can synchronise the
// device and fail under fragmentation) is not acceptable.  For small problems they can use
// this entry point: its scratch is a fixed array in device global memory that exists for
// as long as the library is loaded, so nothing is allocated or freed per call.
#include <cuda.h>

#include <mutex>

#include "common.cuh"

namespace donof {
namespace {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;  // 64 MiB per device
constexpr int kMaxDevices = 64;

// The scratch.  Every GPU that loads the library holds it until the process exits.
// In host code `g_noalloc_scratch` is only a stand-in for the device symbol; its device
// address is obtained with cudaGetSymbolAddress below.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
// Upstream gradient 1.0 for the optional dE/dC (a constant, not scratch).
__device__ double g_noalloc_one = 1.0;

// One lock per device, held for a whole call: the host-side registration of the scratch
// (donof_prepare_B) and the enqueue of the build and adjoint of one call are never
// interleaved with another thread's call on the same device.
std::mutex g_noalloc_mu[kMaxDevices];
void* g_scratch_ptr[kMaxDevices] = {};
double* g_one_ptr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};  // context the addresses belong to

// Unique id of the current context (cuCtxGetId; 0 when it cannot be read).  A device reset
// destroys the primary context, and the module holding the scratch is loaded again, possibly
// elsewhere, in the next one: the cached addresses are then resolved again.
unsigned long long current_context_id() {
  typedef CUresult (*GetCurrentFn)(CUcontext*);
  typedef CUresult (*GetIdFn)(CUcontext, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrentFn)p;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = (GetIdFn)p;
  });
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c ||
      get_id(c, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Set-up, once per device (and again after a reset of its context), with that device
// current: resolve the device addresses of the arrays.  Called with g_noalloc_mu[dev] held.
int noalloc_setup(int dev, void** scratch, double** one) {
  const unsigned long long ctx = current_context_id();
  if (!g_scratch_ptr[dev] || ctx != g_ctx_id[dev]) {
    void* p = nullptr;
    void* q = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return DONOF_ERR_CUDA;
    if (cudaGetSymbolAddress(&q, g_noalloc_one) != cudaSuccess) return DONOF_ERR_CUDA;
    g_scratch_ptr[dev] = p;
    g_one_ptr[dev] = (double*)q;
    g_ctx_id[dev] = ctx;
  }
  *scratch = g_scratch_ptr[dev];
  *one = g_one_ptr[dev];
  return DONOF_OK;
}

int current_device(int* dev) {
  if (cudaGetDevice(dev) != cudaSuccess) return DONOF_ERR_CUDA;
  return (*dev < 0 || *dev >= kMaxDevices) ? DONOF_ERR_UNSUPPORTED : DONOF_OK;
}

}  // namespace
}  // namespace donof

extern "C" int donof_energy_lagrangian_noalloc(const donof_problem* prob, const double* h,
                                               const double* B, const double* C,
                                               const double* gamma, const int32_t* pair_map,
                                               double* E, double* lam, double* dE_dgamma,
                                               double* dE_dC, void* stream) {
  using namespace donof;
  size_t need = 0;
  int rc = donof_workspace_size(prob, &need);
  if (rc != DONOF_OK) return rc;
  if (need > kNoAllocScratchBytes) return DONOF_ERR_WORKSPACE;  // problem too large
  int dev = 0;
  rc = current_device(&dev);
  if (rc != DONOF_OK) return rc;
  std::lock_guard<std::mutex> lk(g_noalloc_mu[dev]);
  void* scratch = nullptr;
  double* one = nullptr;
  rc = noalloc_setup(dev, &scratch, &one);
  if (rc != DONOF_OK) return rc;
  // prepare_B clears the workspace header (status, maxima) before anything reads it; the
  // build clears every accumulator it uses (J, K, G, h C, lambda) itself.
  rc = donof_prepare_B(prob, B, scratch, kNoAllocScratchBytes, stream);
  if (rc != DONOF_OK) return rc;
  rc = donof_energy_lagrangian(prob, h, B, C, gamma, pair_map, scratch, kNoAllocScratchBytes, E,
                               lam, dE_dgamma, stream);
  if (rc != DONOF_OK) return rc;
  if (dE_dC) rc = donof_energy_backward(prob, one, scratch, kNoAllocScratchBytes, dE_dC, nullptr,
                                        stream);
  return rc;
}

extern "C" int donof_noalloc_read_status(int32_t* status, void* stream) {
  using namespace donof;
  if (!status) return DONOF_ERR_INVALID_ARG;
  int dev = 0;
  int rc = current_device(&dev);
  if (rc != DONOF_OK) return rc;
  std::lock_guard<std::mutex> lk(g_noalloc_mu[dev]);
  void* scratch = nullptr;
  double* one = nullptr;
  rc = noalloc_setup(dev, &scratch, &one);
  if (rc != DONOF_OK) return rc;
  // the status word heads the scratch (it is the workspace header of every call)
  return donof_read_status(scratch, status, stream);
}
