// Batched builds: many independent instances of uneven size (a dissociation scan: the same
// molecule at many geometries) in one call.
//
// Each instance owns a slice of the caller's workspace and runs the single-instance launch
// sequence.  Instances are spread over a pool of internal streams (longest-processing-time
// order, largest estimated cost first), forked from and joined back to the caller's stream
// with events, so that small instances fill the GPU together.  With DONOF_BATCH_GRAPH the
// whole batch is captured once into a CUDA graph keyed by the call's arguments and every
// later call with the same arguments replays it as one graph launch.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace donof {
namespace {

constexpr int kStreams = 16;
constexpr size_t kTableBytes = 256;  // head of the batched workspace: the constant 1.0

struct StreamPool {
  cudaStream_t s[kStreams] = {};
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kStreams] = {};
  bool ready = false;
};

std::mutex g_batch_mu;
std::map<int, StreamPool> g_pools;  // per device

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;  // kernels in one replay
};
std::map<std::vector<unsigned char>, GraphEntry> g_graphs;

int pool_for_device(StreamPool** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DONOF_ERR_CUDA;
  StreamPool& p = g_pools[dev];
  if (!p.ready) {
    for (int i = 0; i < kStreams; ++i) {
      if (cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking) != cudaSuccess)
        return DONOF_ERR_CUDA;
      if (cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming) != cudaSuccess)
        return DONOF_ERR_CUDA;
    }
    if (cudaStreamCreateWithFlags(&p.origin, cudaStreamNonBlocking) != cudaSuccess)
      return DONOF_ERR_CUDA;
    if (cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) != cudaSuccess)
      return DONOF_ERR_CUDA;
    p.ready = true;
  }
  *out = &p;
  return DONOF_OK;
}

size_t instance_offset(int32_t i, const donof_problem* probs) {
  size_t off = kTableBytes;
  for (int32_t k = 0; k < i; ++k) {
    size_t b = 0;
    donof_workspace_size(&probs[k], &b);
    off = align_up(off + b);
  }
  return off;
}

// Relative cost of one build, for the stream assignment.
double est_cost(const donof_problem& p) {
  const double N = p.nbf, Q = p.naux, A = (double)p.npair * (1 + p.ncwo) + p.nsingle;
  return 2.0 * Q * N * A * (N + 2.0 * A) + 4.0 * N * N * A + 2e7;  // + launch overhead
}

// Enqueue every instance on the pool's streams (which already wait on `p.fork`).
int enqueue_all(int32_t ninst, const donof_problem* probs, const donof_instance* inst, char* ws,
                int32_t flags, StreamPool& p) {
  std::vector<int> order(ninst);
  for (int i = 0; i < ninst; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return est_cost(probs[a]) > est_cost(probs[b]); });
  double load[kStreams] = {};
  const double* one = (const double*)ws;
  for (int i : order) {
    int k = (int)(std::min_element(load, load + kStreams) - load);
    load[k] += est_cost(probs[i]);
    char* wsi = ws + instance_offset(i, probs);
    size_t bi = 0;
    donof_workspace_size(&probs[i], &bi);
    const donof_instance& x = inst[i];
    int rc = donof_energy_lagrangian(&probs[i], x.h, x.B, x.C, x.gamma, x.pair_map, wsi, bi, x.E,
                                     x.lam, x.dE_dgamma, p.s[k]);
    if (rc != DONOF_OK) return rc;
    if ((flags & DONOF_BATCH_BACKWARD) && x.dE_dC) {
      rc = donof_energy_backward(&probs[i], one, wsi, bi, x.dE_dC, nullptr, p.s[k]);
      if (rc != DONOF_OK) return rc;
    }
  }
  return DONOF_OK;
}

std::vector<unsigned char> graph_key(int32_t ninst, const donof_problem* probs,
                                     const donof_instance* inst, const void* ws, int32_t flags,
                                     cudaStream_t s) {
  std::vector<unsigned char> k;
  auto put = [&](const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    k.insert(k.end(), c, c + n);
  };
  int dev = 0;
  cudaGetDevice(&dev);
  put(&dev, sizeof dev);
  put(&ninst, sizeof ninst);
  put(&ws, sizeof ws);
  put(&flags, sizeof flags);
  put(probs, sizeof(donof_problem) * (size_t)ninst);
  put(inst, sizeof(donof_instance) * (size_t)ninst);
  return k;
}

}  // namespace
}  // namespace donof

using namespace donof;

extern "C" int donof_batched_workspace_size(int32_t ninst, const donof_problem* probs,
                                            size_t* bytes) {
  if (ninst < 1 || !probs || !bytes) return DONOF_ERR_INVALID_ARG;
  size_t off = kTableBytes;
  for (int32_t k = 0; k < ninst; ++k) {
    size_t b = 0;
    const int rc = donof_workspace_size(&probs[k], &b);
    if (rc != DONOF_OK) return rc;
    off = align_up(off + b);
  }
  *bytes = off;
  return DONOF_OK;
}

extern "C" int donof_prepare_B_batched(int32_t ninst, const donof_problem* probs,
                                       const donof_instance* inst, void* workspace,
                                       size_t workspace_bytes, void* stream) {
  size_t need = 0;
  int rc = donof_batched_workspace_size(ninst, probs, &need);
  if (rc != DONOF_OK) return rc;
  if (!inst || !workspace || workspace_bytes < need || ((uintptr_t)workspace % kAlign) != 0)
    return DONOF_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const double one = 1.0;
  if (cudaMemcpyAsync(workspace, &one, sizeof one, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return DONOF_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DONOF_ERR_CUDA;  // `one` is on the stack
  for (int32_t i = 0; i < ninst; ++i) {
    size_t bi = 0;
    donof_workspace_size(&probs[i], &bi);
    rc = donof_prepare_B(&probs[i], inst[i].B, (char*)workspace + instance_offset(i, probs), bi,
                         stream);
    if (rc != DONOF_OK) return rc;
  }
  return DONOF_OK;
}

extern "C" int donof_energy_lagrangian_batched(int32_t ninst, const donof_problem* probs,
                                               const donof_instance* inst, void* workspace,
                                               size_t workspace_bytes, int32_t flags,
                                               void* stream) {
  size_t need = 0;
  int rc = donof_batched_workspace_size(ninst, probs, &need);
  if (rc != DONOF_OK) return rc;
  if (!inst || !workspace || workspace_bytes < need || ((uintptr_t)workspace % kAlign) != 0)
    return DONOF_ERR_WORKSPACE;
  if (flags & ~(DONOF_BATCH_BACKWARD | DONOF_BATCH_GRAPH)) return DONOF_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(g_batch_mu);
  StreamPool* p = nullptr;
  rc = pool_for_device(&p);
  if (rc != DONOF_OK) return rc;
  char* ws = (char*)workspace;

  if (!(flags & DONOF_BATCH_GRAPH)) {
    if (cudaEventRecord(p->fork, s) != cudaSuccess) return DONOF_ERR_CUDA;
    for (int k = 0; k < kStreams; ++k)
      if (cudaStreamWaitEvent(p->s[k], p->fork, 0) != cudaSuccess) return DONOF_ERR_CUDA;
    rc = enqueue_all(ninst, probs, inst, ws, flags, *p);
    for (int k = 0; k < kStreams; ++k) {
      if (cudaEventRecord(p->join[k], p->s[k]) != cudaSuccess) return DONOF_ERR_CUDA;
      if (cudaStreamWaitEvent(s, p->join[k], 0) != cudaSuccess) return DONOF_ERR_CUDA;
    }
    return rc;
  }

  // graph mode: capture once per distinct argument set, then replay
  std::vector<unsigned char> key = graph_key(ninst, probs, inst, workspace, flags, s);
  auto it = g_graphs.find(key);
  if (it == g_graphs.end()) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(p->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return DONOF_ERR_CUDA;
    const long long l0 = donof_launch_count();
    bool ok = cudaEventRecord(p->fork, p->origin) == cudaSuccess;
    for (int k = 0; ok && k < kStreams; ++k)
      ok = cudaStreamWaitEvent(p->s[k], p->fork, 0) == cudaSuccess;
    rc = ok ? enqueue_all(ninst, probs, inst, ws, flags, *p) : DONOF_ERR_CUDA;
    for (int k = 0; k < kStreams; ++k) {
      cudaEventRecord(p->join[k], p->s[k]);
      cudaStreamWaitEvent(p->origin, p->join[k], 0);
    }
    const cudaError_t ce = cudaStreamEndCapture(p->origin, &graph);
    if (rc != DONOF_OK || ce != cudaSuccess || !graph) {
      if (graph) cudaGraphDestroy(graph);
      return rc != DONOF_OK ? rc : DONOF_ERR_CUDA;
    }
    GraphEntry ge;
    ge.launches = donof_launch_count() - l0;
    const cudaError_t ie = cudaGraphInstantiate(&ge.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return DONOF_ERR_CUDA;
    it = g_graphs.emplace(std::move(key), ge).first;
  } else {
    count_launch((int)it->second.launches);  // the replay launches the captured kernels again
  }
  if (cudaGraphLaunch(it->second.exec, s) != cudaSuccess) return DONOF_ERR_CUDA;
  return DONOF_OK;
}
