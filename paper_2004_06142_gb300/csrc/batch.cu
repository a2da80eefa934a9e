// Batched builds: many independent instances of uneven size (a dissociation scan: the same
// molecule at many geometries) in one call.
//
// Grouped path (every instance mixed precision, all its auxiliary slices in one block): each
// step of the build is one launch for all instances together -- a grouped kernel finds its
// instance and its block within that instance's grid from a table, and the tensor-core
// contractions walk one sequence of work units that spans every instance -- so a batched
// build with its adjoint is 24 launches whatever the number of instances.  The tables (the
// instances' records, the grids of every step, the tensor-core arguments and tensor maps)
// are built on the host and copied into the head of the batched workspace when the call's
// arguments change.
//
// Stream path (any other batch): each instance owns a slice of the caller's workspace and runs
// the single-instance launch sequence on a pool of internal streams (longest-processing-time
// order, largest estimated cost first), forked from and joined back to the caller's stream.
//
// With DONOF_BATCH_GRAPH either path is captured once into a CUDA graph keyed by the call's
// arguments and every later call with the same arguments replays it as one graph launch.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace donof {
namespace {

constexpr int kStreams = 16;
// Head of the batched workspace: the batch's status header (offset 0), the constant 1.0
// (upstream gradient of the adjoints) and the grouped path's tables.
constexpr int kTcKinds = 5;
const int kTcKindList[kTcKinds] = {GK_TC_HC, GK_TC_HALF, GK_TC_B, GK_TC_G, GK_TC_LAM};
struct PlanLayout {
  size_t one, inst, grids, targs[kTcKinds], tmaps[kTcKinds], ustart[kTcKinds], total;
};
PlanLayout plan_layout(int ninst) {
  PlanLayout p{};
  size_t off = align_up(sizeof(DevHeader));
  p.one = off;
  off = align_up(off + sizeof(double));
  p.inst = off;
  off = align_up(off + (size_t)ninst * sizeof(InstRec));
  p.grids = off;
  off = align_up(off + (size_t)GK_COUNT * (4 * (size_t)ninst + 1) * sizeof(int));
  for (int k = 0; k < kTcKinds; ++k) {
    p.targs[k] = off;
    off = align_up(off + (size_t)ninst * tc_args_bytes());
    p.tmaps[k] = off;
    off = align_up(off + (size_t)ninst * tc_maps_bytes());
    p.ustart[k] = off;
    off = align_up(off + ((size_t)ninst + 1) * sizeof(int));
  }
  p.total = off;
  return p;
}

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
  std::vector<char> plan;  // grouped path: the tables the graph reads from the workspace
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

size_t instance_offset(int32_t i, const donof_problem* probs, int32_t ninst) {
  size_t off = plan_layout(ninst).total;
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
  const double* one = (const double*)(ws + plan_layout(ninst).one);
  for (int i : order) {
    int k = (int)(std::min_element(load, load + kStreams) - load);
    load[k] += est_cost(probs[i]);
    char* wsi = ws + instance_offset(i, probs, ninst);
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

// ---------------------------------------------------------------------------------- grouped
// Every instance mixed precision, its auxiliary slices in one block.
bool groupable(int32_t ninst, const donof_problem* probs) {
  for (int32_t i = 0; i < ninst; ++i) {
    if (probs[i].precision != DONOF_MIXED) return false;
    const Dims d = make_dims(&probs[i]);
    if (d.pb != d.Q) return false;
  }
  return true;
}

// The tables of a grouped batch (the bytes of the plan region) and each launch's shape.
struct Plan {
  std::vector<char> bytes;
  int blocks[GK_COUNT] = {};
  dim3 threads[GK_COUNT];
  size_t smem[GK_COUNT] = {};
  int tc_units[kTcKinds] = {};
  size_t tc_smem[kTcKinds] = {};
  int tc_cat[kTcKinds] = {};
};

int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Grid of instance (d, x) in step `kind` (those of the single-instance launchers).
dim3 kind_grid(int kind, const Dims& d, const donof_instance& x, bool backward) {
  const int np = d.Q, sp3 = d.splits < np ? d.splits : np, N = d.N, A = d.A, Ap = d.Ap;
  const bool lam = x.lam != nullptr;
  switch (kind) {
    case GK_ZERO: {  // every range of the instance strided over one grid, 16 words a thread
      const long long words = 1 + 2 + 3LL * A * (d.ng > 0 ? d.ng : 0) * 2 + 4LL * A * A +
                              (lam ? 2LL * N * N : 0);
      return dim3(std::max(1, ceil_div(words, 256 * 16)), 1, 1);
    }
    case GK_OCC: return dim3(1, 1, 1);
    case GK_COEF: return dim3(ceil_div((long long)Ap * Ap, 256), 1, 1);
    case GK_SPLIT_C:  // norms + split, a block per 32 columns of each job (C_act twice, h)
      return dim3(2 * ceil_div(Ap, 32) + ceil_div(N, 32), 1, 1);
    case GK_SUM_HC: return dim3(std::min(1216, ceil_div((long long)N * A, 256)), 1, 1);
    case GK_GRAM_PART: return dim3(ceil_div(N, 32), ceil_div(A, 16), 1);
    case GK_GRAM_FINAL: return dim3(A, 1, 1);
    case GK_HDIAG: return dim3(ceil_div(A, 8), 1, 1);
    case GK_XEXP: return dim3(std::max(1, ceil_div((long long)sp3 * N, 256)), 2, 1);
    case GK_DIAGW: return dim3(ceil_div(np, kDiagWTileSlices), ceil_div(A, kDiagWTileCols), 1);
    case GK_KPART: return dim3(ceil_div(kpart_quads(A), 256), sp3, 1);
    case GK_JKEY:  // the sums a thread per entry; the exponents a warp per (split, row)
      return dim3(ceil_div((long long)A * A, 256) + ceil_div((long long)sp3 * Ap, 8), 1, 1);
    case GK_YQUANT: return dim3(ceil_div(np, 8), 1, 1);  // eight slices a block
    case GK_REDUCEG: return dim3(ceil_div((long long)N * (Ap / 4), 256), 1, 1);
    case GK_EROWS: return dim3(ceil_div(A, 8), 1, 1);
    case GK_EFINAL: return dim3(ceil_div(d.ng + 1, 8), 1, 1);
    case GK_SPLIT_L:  // C (all N columns), G
      return lam ? dim3(ceil_div(N, 32) + ceil_div(Ap, 32), 1, 1) : dim3(0, 1, 1);
    case GK_SUM_L: return lam ? dim3(std::min(1216, ceil_div((long long)N * A, 256)), 1, 1)
                              : dim3(0, 1, 1);
    case GK_BWD: return (backward && x.dE_dC) ? dim3(std::min(608, ceil_div((long long)N * N, 256)), 1, 1)
                                            : dim3(0, 1, 1);
  }
  return dim3(0, 1, 1);
}

int tc_index(int kind) {
  for (int k = 0; k < kTcKinds; ++k)
    if (kTcKindList[k] == kind) return k;
  return -1;
}

int build_plan(int32_t ninst, const donof_problem* probs, const donof_instance* inst, char* ws,
               int32_t flags, Plan& pl) {
  const PlanLayout P = plan_layout(ninst);
  pl.bytes.assign(P.total, 0);
  char* h = pl.bytes.data();
  DevHeader* bhdr = (DevHeader*)ws;  // the batch's status header (device)
  const bool backward = (flags & DONOF_BATCH_BACKWARD) != 0;
  std::vector<Dims> dims(ninst);
  int max_A = 1, max_ng = 1, max_Ap = 16, max_N = 1;
  for (int32_t i = 0; i < ninst; ++i) {
    const Dims d = make_dims(&probs[i]);
    dims[i] = d;
    max_A = std::max(max_A, d.A);
    max_ng = std::max(max_ng, d.ng);
    max_Ap = std::max(max_Ap, d.Ap);
    max_N = std::max(max_N, d.N);
    InstRec r{};
    r.d = d;
    r.L = make_layout(d);
    r.ws = ws + instance_offset(i, probs, ninst);
    const donof_instance& x = inst[i];
    r.h = x.h; r.B = x.B; r.C = x.C; r.gamma = x.gamma; r.pm = x.pair_map;
    r.E = x.E; r.lam = x.lam; r.dEdg = x.dE_dgamma; r.dEdC = backward ? x.dE_dC : nullptr;
    r.Ebar = (const double*)(ws + P.one);
    memcpy(h + P.inst + (size_t)i * sizeof(InstRec), &r, sizeof r);
  }
  // grids of the grouped small kernels
  int* grids = (int*)(h + P.grids);
  for (int k = 0; k < GK_COUNT; ++k) {
    int* start = grids + (size_t)k * (4 * ninst + 1);
    int* gd = start + ninst + 1;
    int tot = 0;
    for (int32_t i = 0; i < ninst; ++i) {
      const dim3 g = tc_index(k) >= 0 ? dim3(0, 1, 1) : kind_grid(k, dims[i], inst[i], backward);
      start[i] = tot;
      gd[3 * i] = (int)std::max(1u, g.x);
      gd[3 * i + 1] = (int)g.y;
      gd[3 * i + 2] = (int)g.z;
      tot += (int)(g.x * g.y * g.z);
    }
    start[ninst] = tot;
    pl.blocks[k] = tot;
    pl.threads[k] = dim3(256);
    pl.smem[k] = 0;
  }
  pl.threads[GK_OCC] = dim3((max_A + 31) / 32 * 32);
  pl.smem[GK_OCC] = (size_t)max_ng * 2 * sizeof(double);
  // 32 x the row groups of the widest instance's column norms (norm_groups in tc.cu)
  pl.threads[GK_SPLIT_C] = pl.threads[GK_SPLIT_L] = dim3(max_N > 256 ? 1024 : 256);
  pl.threads[GK_YQUANT] = dim3(max_Ap / 4, 8);
  // tensor-core records
  for (int t = 0; t < kTcKinds; ++t) {
    const int kind = kTcKindList[t];
    int* ust = (int*)(h + P.ustart[t]);
    int tot = 0;
    for (int32_t i = 0; i < ninst; ++i) {
      const InstRec* r = (const InstRec*)(h + P.inst + (size_t)i * sizeof(InstRec));
      int units = 0;
      if (!tc_group_setup(kind, r->d, r->ws, r->L, h + P.targs[t] + (size_t)i * tc_args_bytes(),
                          h + P.tmaps[t] + (size_t)i * tc_maps_bytes(), units))
        return DONOF_ERR_CUDA;
      if (kind == GK_TC_LAM && !inst[i].lam) units = 0;
      ust[i] = tot;
      tot += units;
    }
    ust[ninst] = tot;
    pl.tc_units[t] = tot;
    pl.tc_smem[t] = tc_group_finish(kind, h + P.targs[t], ninst, &bhdr->status, &bhdr->abort_flag,
                                    pl.tc_cat[t]);
  }
  return DONOF_OK;
}

// Enqueue a grouped batched build (and adjoint) on s; the plan is on the device.
int enqueue_grouped(int32_t ninst, char* ws, int32_t flags, const Plan& pl, cudaStream_t s) {
  const PlanLayout P = plan_layout(ninst);
  const InstRec* inst_dev = (const InstRec*)(ws + P.inst);
  const int* grids = (const int*)(ws + P.grids);
  DevHeader* bhdr = (DevHeader*)ws;
  if (cudaMemsetAsync(&bhdr->abort_flag, 0, sizeof(int32_t), s) != cudaSuccess)
    return DONOF_ERR_CUDA;
  for (int k = 0; k < GK_COUNT; ++k) {
    if (k == GK_BWD && !(flags & DONOF_BATCH_BACKWARD)) continue;
    const int t = tc_index(k);
    cudaError_t e = cudaSuccess;
    if (t >= 0) {
      if (pl.tc_units[t] == 0) continue;
      e = launch_tc_group(k, ws + P.targs[t], ws + P.tmaps[t], (const int*)(ws + P.ustart[t]),
                          ninst, pl.tc_units[t], pl.tc_smem[t], pl.tc_cat[t], s);
    } else {
      if (pl.blocks[k] == 0) continue;
      const int* start = grids + (size_t)k * (4 * ninst + 1);
      const GroupLaunch g{inst_dev, start, start + ninst + 1, ninst};
      const int blocks = pl.blocks[k];
      switch (k) {
        case GK_ZERO: case GK_OCC: case GK_COEF: case GK_HDIAG: case GK_EROWS: case GK_EFINAL:
        case GK_BWD:
          e = launch_fp64_group(k, g, blocks, pl.threads[k].x, pl.smem[k], s);
          break;
        case GK_DIAGW: case GK_KPART: case GK_JKEY: case GK_YQUANT:
          e = launch_mid_group(k, g, blocks, pl.threads[k], s);
          break;
        default:
          e = launch_tc_small_group(k, g, blocks, pl.threads[k].x, s);
      }
    }
    if (e != cudaSuccess) return DONOF_ERR_CUDA;
  }
  return DONOF_OK;
}

// The plan last copied into each batched workspace (so that an unchanged plan is not copied
// again).
std::map<const void*, std::vector<char>> g_uploaded;

int upload_plan(char* ws, const Plan& pl, cudaStream_t s) {
  auto it = g_uploaded.find(ws);
  if (it != g_uploaded.end() && it->second == pl.bytes) return DONOF_OK;
  // earlier work on the stream may still read the old tables
  if (cudaStreamSynchronize(s) != cudaSuccess) return DONOF_ERR_CUDA;
  const size_t hdr = align_up(sizeof(DevHeader));  // the status header and 1.0 stay
  const size_t off = plan_layout(0).inst > hdr ? plan_layout(0).inst : hdr;
  if (cudaMemcpy(ws + off, pl.bytes.data() + off, pl.bytes.size() - off,
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return DONOF_ERR_CUDA;
  g_uploaded[ws] = pl.bytes;
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
  size_t off = plan_layout(ninst).total;
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
  // the batch's status header cleared, the constant 1.0 set
  if (cudaMemsetAsync(workspace, 0, sizeof(DevHeader), s) != cudaSuccess) return DONOF_ERR_CUDA;
  const double one = 1.0;
  if (cudaMemcpyAsync((char*)workspace + plan_layout(ninst).one, &one, sizeof one,
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return DONOF_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DONOF_ERR_CUDA;  // `one` is on the stack
  for (int32_t i = 0; i < ninst; ++i) {
    size_t bi = 0;
    donof_workspace_size(&probs[i], &bi);
    rc = donof_prepare_B(&probs[i], inst[i].B,
                         (char*)workspace + instance_offset(i, probs, ninst), bi, stream);
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
  if (flags & ~(DONOF_BATCH_BACKWARD | DONOF_BATCH_GRAPH | DONOF_BATCH_STREAMS))
    return DONOF_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(g_batch_mu);
  StreamPool* p = nullptr;
  rc = pool_for_device(&p);
  if (rc != DONOF_OK) return rc;
  char* ws = (char*)workspace;
  const bool grouped = !(flags & DONOF_BATCH_STREAMS) && groupable(ninst, probs);

  // the work of one call on stream `o` (grouped: its tables already in the workspace)
  auto enqueue = [&](cudaStream_t o, const Plan* pl) -> int {
    if (grouped) return enqueue_grouped(ninst, ws, flags, *pl, o);
    if (cudaEventRecord(p->fork, o) != cudaSuccess) return DONOF_ERR_CUDA;
    for (int k = 0; k < kStreams; ++k)
      if (cudaStreamWaitEvent(p->s[k], p->fork, 0) != cudaSuccess) return DONOF_ERR_CUDA;
    const int r = enqueue_all(ninst, probs, inst, ws, flags, *p);
    for (int k = 0; k < kStreams; ++k) {
      if (cudaEventRecord(p->join[k], p->s[k]) != cudaSuccess) return DONOF_ERR_CUDA;
      if (cudaStreamWaitEvent(o, p->join[k], 0) != cudaSuccess) return DONOF_ERR_CUDA;
    }
    return r;
  };

  if (!(flags & DONOF_BATCH_GRAPH)) {
    Plan pl;
    if (grouped) {
      rc = build_plan(ninst, probs, inst, ws, flags, pl);
      if (rc == DONOF_OK) rc = upload_plan(ws, pl, s);
      if (rc != DONOF_OK) return rc;
    }
    return enqueue(s, &pl);
  }

  // graph mode: capture once per distinct argument set, then replay
  std::vector<unsigned char> key = graph_key(ninst, probs, inst, workspace, flags, s);
  auto it = g_graphs.find(key);
  if (it == g_graphs.end()) {
    GraphEntry ge;
    Plan pl;
    if (grouped) {  // the tables go into the workspace before the capture
      rc = build_plan(ninst, probs, inst, ws, flags, pl);
      if (rc == DONOF_OK) rc = upload_plan(ws, pl, s);
      if (rc != DONOF_OK) return rc;
      ge.plan = pl.bytes;
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(p->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return DONOF_ERR_CUDA;
    const long long l0 = donof_launch_count();
    rc = enqueue(p->origin, &pl);
    const cudaError_t ce = cudaStreamEndCapture(p->origin, &graph);
    if (rc != DONOF_OK || ce != cudaSuccess || !graph) {
      if (graph) cudaGraphDestroy(graph);
      return rc != DONOF_OK ? rc : DONOF_ERR_CUDA;
    }
    ge.launches = donof_launch_count() - l0;
    const cudaError_t ie = cudaGraphInstantiate(&ge.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return DONOF_ERR_CUDA;
    it = g_graphs.emplace(std::move(key), std::move(ge)).first;
  } else {
    if (!it->second.plan.empty()) {  // another argument set may have replaced the tables
      Plan pl;
      pl.bytes = it->second.plan;
      rc = upload_plan(ws, pl, s);
      if (rc != DONOF_OK) return rc;
    }
    count_launch((int)it->second.launches);  // the replay launches the captured kernels again
  }
  if (cudaGraphLaunch(it->second.exec, s) != cudaSuccess) return DONOF_ERR_CUDA;
  return DONOF_OK;
}
