// donof_energy_lagrangian_noalloc: a build that allocates no device memory.
//
// Some callers cannot allocate device memory at the moment they need a build: a host
// framework may own the whole device pool through its own allocator and forbid other
// allocations, or the call may sit in a loop where a cudaMalloc (which can synchronise the
// device and fail under fragmentation) is not acceptable.  For small problems they can use
// this entry point: its scratch is a fixed array in device global memory that exists for
// as long as the library is loaded, so nothing is allocated or freed per call.
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

std::mutex g_noalloc_mu;
void* g_scratch_ptr[kMaxDevices] = {};
double* g_one_ptr[kMaxDevices] = {};

// Once per device, with that device current: resolve the device addresses of the arrays.
int noalloc_setup(int dev, void** scratch, double** one) {
  if (dev < 0 || dev >= kMaxDevices) return DONOF_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    void* q = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return DONOF_ERR_CUDA;
    if (cudaGetSymbolAddress(&q, g_noalloc_one) != cudaSuccess) return DONOF_ERR_CUDA;
    g_scratch_ptr[dev] = p;
    g_one_ptr[dev] = (double*)q;
  }
  *scratch = g_scratch_ptr[dev];
  *one = g_one_ptr[dev];
  return DONOF_OK;
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
  if (cudaGetDevice(&dev) != cudaSuccess) return DONOF_ERR_CUDA;
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
