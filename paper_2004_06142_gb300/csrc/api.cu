// C ABI entry points of libdonof (declared in include/donof.h): argument checks,
// workspace carving and the launch sequence of one build.
//
// One build streams the auxiliary index P in blocks (Sec. III.D: the AO -> MO
// transformation is redone every time the orbitals change).  Per block:
//   X = B C_act  ->  b^P = C_act^T X^P  ->  J, K += ...,  Y^P  ->  G += sum_P X^P Y^P
// and, after the last block, E and dE/dgamma from J, K (Eqs. EPNOF7, Eg, Efg, Efg_s) and
// lambda = C^T G (Eqs. lowdin, lag).  The coefficients of Y depend only on the
// occupations, so G needs no second pass over B.
#include <atomic>
#include <mutex>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace donof {

Dims make_dims(const donof_problem* p) {
  Dims d{};
  d.N = p->nbf;
  d.Q = p->naux;
  d.npair = p->npair;
  d.ncwo = p->ncwo;
  d.nsingle = p->nsingle;
  d.A = p->npair * (1 + p->ncwo) + p->nsingle;
  d.Ap = round_up_int(d.A, 16);
  d.Np = round_up_int(d.N, 8);
  d.ng = p->npair * p->ncwo;
  d.functional = p->functional;
  d.layout = p->b_layout;
  d.precision = p->precision;
  size_t perP;
  if (d.precision == DONOF_FP64) {
    perP = (size_t)d.N * d.A * 8 + 2 * (size_t)d.A * d.A * 8 +
           (d.layout == DONOF_B_PACKED ? (size_t)d.N * d.N * 8 : 0);
  } else {
    perP = (size_t)d.Np * d.Ap * 4 + (size_t)d.Ap * d.Np * 4 + (size_t)d.Ap * d.Ap * (4 + 4 + 4) +
           (size_t)d.Ap * 4 + (size_t)d.A * 8;
  }
  long long pb = d.Q;
  if (p->x_budget_bytes > 0) {
    pb = (long long)(p->x_budget_bytes / perP);
    if (pb < 1) pb = 1;
    if (pb > d.Q) pb = d.Q;
  }
  if (pb > 65535) pb = 65535;  // batch index of the double GEMMs lives in gridDim.z
  d.pb = (int)pb;
  d.nblk = (d.Q + d.pb - 1) / d.pb;
  // split-K of the G contraction: at most 64 slices per split, enough units (row tiles x
  // splits) for 2 waves over the 152 SMs but at least 32 slices per split (short splits
  // only add partials to reduce), and where a few more splits make the units a whole
  // number of waves, those
  const int mt = (d.N + 127) / 128;
  int sp = (d.pb + 63) / 64;
  int want = (2 * 152 + mt - 1) / mt;
  if (want > (d.pb + 31) / 32) want = (d.pb + 31) / 32;
  if (sp < want) sp = want;
  for (int s2 = sp; s2 <= sp + sp / 4; ++s2)
    if ((mt * s2) % 152 == 0) {
      sp = s2;
      break;
    }
  if (sp > d.pb) sp = d.pb;
  d.splits = sp;
  return d;
}

// Split count of the FP64 path's G contraction (contraction over the np slices): about
// four CTAs per SM, at most one split per slice.
int g_splits_fp64(int N, int A, int np) {
  const int bn = dgemm_tile_n(A);
  const long long tiles = (long long)((N + 63) / 64) * ((A + bn - 1) / bn);
  long long ks = (4 * 152 + tiles - 1) / tiles;
  if (ks > np) ks = np;
  if (ks < 1) ks = 1;
  return (int)ks;
}

Layout make_layout(const Dims& d) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + (bytes ? bytes : 1));
    return o;
  };
  const size_t N = d.N, A = d.A, Ap = d.Ap, Np = d.Np, ng = d.ng > 0 ? d.ng : 1, pb = d.pb;
  L.header = take(sizeof(DevHeader));
  L.n = take(A * 8);
  L.sqn = take(A * 8);
  L.phi = take(A * 8);
  L.dn = take(A * ng * 8);
  L.dsq = take(A * ng * 8);
  L.dphi = take(A * ng * 8);
  L.Acoef = take(A * A * 8);
  L.Bcoef = take(A * A * 8);
  L.Hd = take(A * 8);
  L.hC = take(N * A * 8);
  L.J = take(A * A * 8);
  L.K = take(A * A * 8);
  L.G = take(N * A * 8);
  L.dEdg = take(ng * 8);
  L.Epart = take(4 * A * 8);
  {  // split-K partials of the FP64 products with N x A outputs (h C_act, lambda, G)
    size_t ks = 0;
    if (d.precision == DONOF_FP64) {
      ks = (size_t)splitk_count((int)N, (int)A, (int)N);
      const size_t kg = (size_t)g_splits_fp64((int)N, (int)A, (int)pb);
      if (kg > ks) ks = kg;
    }
    L.skp = take(ks > 1 ? ks * N * A * 8 : 0);
  }
  if (d.precision == DONOF_FP64) {
    L.X64 = take(pb * N * A * 8);
    L.b64 = take(pb * A * A * 8);
    L.Y64 = take(pb * A * A * 8);
    L.Bun = d.layout == DONOF_B_PACKED ? take(pb * N * N * 8) : 0;
  } else {
    const size_t Q = d.Q;
    // split B in symmetric lower-triangle tiles, per plane Q x SymTiles::perP halves
    const size_t perP = (size_t)sym_tiles((int)N).perP;
    L.Bhi = take(Q * perP * 2);
    L.Blo = take(Q * perP * 2);
    L.eS = take(N * 4);
    L.rnmax = take(N * 8);
    L.tmax = take(Q * 8);
    L.ChiS = take(Ap * Np * 2);
    L.CloS = take(Ap * Np * 2);
    L.eCs = take(Ap * 4);
    L.gram = take((N + 31) / 32 * A * A * 4);  // chunks of 32 AO indices (k_gram_part)
    L.eB = take(Q * N * 4);
    L.L1max = take(Q * 8);
    L.Chi = take(Ap * Np * 2);
    L.Clo = take(Ap * Np * 2);
    L.eC = take(Ap * 4);
    L.cnorm = take(Ap * 8);
    L.Xhi = take(pb * Np * Ap * 2);  // [P][Ap/8][Np][8]
    L.Xlo = take(pb * Np * Ap * 2);
    L.Xthi = take(pb * Ap * Np * 2);
    L.Xtlo = take(pb * Ap * Np * 2);
    L.eXt = take(pb * Ap * 4);
    L.b32 = take(pb * Ap * Ap * 4);
    L.Yhi = take(pb * Ap * Ap * 2);
    L.Ylo = take(pb * Ap * Ap * 2);
    L.Gpart = take((size_t)d.splits * N * Ap * 4);
    L.D = take(pb * A * 4);
    L.rn2 = take(Q * N * 4);  // fp32
    L.spOf = take(pb * 4);
    L.eX3 = take((size_t)d.splits * N * 4);
    L.W = take(pb * A * 4);
    L.Ksp = take((size_t)d.splits * A * A * 8);
    L.Jsp = take((size_t)d.splits * A * A * 8);
    L.AcF = take(Ap * Ap * 4);
    L.BcF = take(Ap * Ap * 4);
    L.eY = take((size_t)d.splits * Ap * 4);
    L.eCf = take(N * 4);
    L.eG = take(Ap * 4);
    L.hAH = take(4 * N * Np * 2);
    L.hAF = take(4 * N * Np * 2);
    L.cPH = take(4 * Ap * Np * 2);
    L.cPF = take(4 * Ap * Np * 2);
    L.eh = take(N * 4);
    L.hpart = take(4 * N * Ap * 4);
  }
  L.total = off;
  return L;
}

// ---------------------------------------------------------------------------
// Tracing: CUDA-event pairs per phase, and a process-wide kernel launch counter.
// ---------------------------------------------------------------------------
namespace {
std::atomic<long long> g_launches{0};
std::mutex g_prof_mu;
bool g_prof_on = false;
struct PhaseRec {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  bool open = false;
};
PhaseRec g_prof[DONOF_NUM_PHASES];

void prof_clear_locked() {
  for (auto& r : g_prof) {
    for (auto& e : r.ev) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    r.ev.clear();
    r.open = false;
  }
}
}  // namespace

void count_launch(int n) { g_launches += n; }

static bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone;
}

// NVTX range names of the phases (host-side enqueue ranges, for filtering kernels by phase
// in profilers: ncu --nvtx --nvtx-include "donof/half_transform/")
const char* const kPhaseRange[DONOF_NUM_PHASES] = {
    "donof/prep", "donof/half_transform", "donof/mo_3index", "donof/jk_y",
    "donof/g_build", "donof/energy_lambda", "donof/backward", "donof/prepare_B",
    "donof/orbital_update", "donof/occ_opt", "donof/orbital_step"};

void prof_begin(int phase, cudaStream_t s) {
  if (phase >= 0 && phase < DONOF_NUM_PHASES) nvtxRangePushA(kPhaseRange[phase]);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on || phase < 0 || phase >= DONOF_NUM_PHASES || capturing(s)) return;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return;
  if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
  cudaEventRecord(a, s);
  g_prof[phase].ev.emplace_back(a, b);
  g_prof[phase].open = true;
}

void prof_end(int phase, cudaStream_t s) {
  if (phase >= 0 && phase < DONOF_NUM_PHASES) nvtxRangePop();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on || phase < 0 || phase >= DONOF_NUM_PHASES || capturing(s)) return;
  PhaseRec& r = g_prof[phase];
  if (!r.open || r.ev.empty()) return;
  cudaEventRecord(r.ev.back().second, s);
  r.open = false;
}

namespace {

struct Registration {
  const double* B;
  donof_problem prob;
};
std::mutex g_mu;
std::unordered_map<const void*, Registration> g_reg;

bool same_problem(const donof_problem& a, const donof_problem& b) {
  return a.nbf == b.nbf && a.naux == b.naux && a.npair == b.npair && a.ncwo == b.ncwo &&
         a.nsingle == b.nsingle && a.b_layout == b.b_layout && a.precision == b.precision &&
         a.x_budget_bytes == b.x_budget_bytes;
}

int check_problem(const donof_problem* p) {
  if (!p) return DONOF_ERR_INVALID_ARG;
  if (p->nbf < 1 || p->naux < 1 || p->npair < 1 || p->ncwo < 1 || p->nsingle < 0)
    return DONOF_ERR_INVALID_ARG;
  if (p->functional != DONOF_PNOF5 && p->functional != DONOF_PNOF7 &&
      p->functional != DONOF_PNOF7S)
    return DONOF_ERR_INVALID_ARG;
  if (p->b_layout != DONOF_B_DENSE && p->b_layout != DONOF_B_PACKED) return DONOF_ERR_INVALID_ARG;
  if (p->precision != DONOF_FP64 && p->precision != DONOF_MIXED) return DONOF_ERR_INVALID_ARG;
  const long long nact = (long long)p->npair * (1 + p->ncwo) + p->nsingle;
  if (nact > p->nbf) return DONOF_ERR_INVALID_ARG;
  if (p->nbf > 65536 || p->naux > (1 << 24)) return DONOF_ERR_UNSUPPORTED;
  if (p->precision == DONOF_MIXED && round_up_int((int)nact, 16) > 256)
    return DONOF_ERR_UNSUPPORTED;
  return DONOF_OK;
}

int check_ws(const donof_problem* p, const void* ws, size_t bytes) {
  if (!ws || ((uintptr_t)ws % kAlign) != 0) return DONOF_ERR_WORKSPACE;
  const Layout L = make_layout(make_dims(p));
  return bytes >= L.total ? DONOF_OK : DONOF_ERR_WORKSPACE;
}


#define CK(x)                                  \
  do {                                         \
    if ((x) != cudaSuccess) return DONOF_ERR_CUDA; \
  } while (0)

}  // namespace

// C(m, n) += sum_k A(m, k) B(k, n) for an M x N output with a long contraction K: the
// contraction is cut into 64-wide chunks shared by enough CTAs to fill the GPU; each CTA
// writes its partial product to scratch and a second kernel adds the partials to C in a
// fixed order (so C must be initialised, and the result does not depend on scheduling).
namespace {
// 64-wide chunks of the contraction, or 16-wide ones when even all 64-wide chunks would
// leave most SMs idle (small problems: the narrow FP64 pipe makes every CTA's share count)
int splitk_chunk(int M, int N, int K) {
  const int bn = dgemm_tile_n(N);
  const long long tiles = (long long)((M + 63) / 64) * ((N + bn - 1) / bn);
  return tiles * ((K + 63) / 64) < 2 * 152 ? 16 : 64;
}
}  // namespace

int splitk_count(int M, int N, int K) {
  const int bn = dgemm_tile_n(N);
  const long long tiles = (long long)((M + 63) / 64) * ((N + bn - 1) / bn);
  const int chunk = splitk_chunk(M, N, K);
  long long ks = (4 * 152 + tiles - 1) / tiles;  // about four CTAs per SM: latency hiding
  const long long kb = (K + chunk - 1) / chunk;
  if (ks > kb) ks = kb;
  if (ks < 1) ks = 1;
  return (int)ks;
}

DgemmArgs split_k_args(int M, int N, int K, const double* A, long long sAm, long long sAk,
                       const double* B, long long sBk, long long sBn, double* C, long long sCm,
                       long long sCn, double* part) {
  DgemmArgs a{};
  const int chunk = splitk_chunk(M, N, K);
  a.M = M; a.N = N; a.K = chunk; a.KB = (K + chunk - 1) / chunk; a.Ktot = K; a.batch = 1;
  a.ksplit = splitk_count(M, N, K);
  a.A = A; a.sAm = sAm; a.sAk = sAk; a.sAkb = (long long)chunk * sAk;
  a.B = B; a.sBk = sBk; a.sBn = sBn; a.sBkb = (long long)chunk * sBk;
  a.C = C; a.sCm = sCm; a.sCn = sCn;
  a.alpha = 1.0; a.beta = 1.0;
  a.part = part;
  return a;
}
}  // namespace donof

using namespace donof;

extern "C" int donof_workspace_size(const donof_problem* prob, size_t* bytes) {
  const int rc = check_problem(prob);
  if (rc != DONOF_OK) return rc;
  if (!bytes) return DONOF_ERR_INVALID_ARG;
  *bytes = make_layout(make_dims(prob)).total;
  return DONOF_OK;
}

extern "C" int donof_prepare_B(const donof_problem* prob, const double* B, void* workspace,
                               size_t workspace_bytes, void* stream) {
  int rc = check_problem(prob);
  if (rc != DONOF_OK) return rc;
  if (!B) return DONOF_ERR_INVALID_ARG;
  rc = check_ws(prob, workspace, workspace_bytes);
  if (rc != DONOF_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const Dims d = make_dims(prob);
  const Layout L = make_layout(d);
  char* ws = (char*)workspace;
  prof_begin(DONOF_PHASE_PREPARE_B, s);
  CK(cudaMemsetAsync(ws + L.header, 0, sizeof(DevHeader), s));
  if (d.precision == DONOF_MIXED) {
    CK(launch_prepare_split_B(d, B, ws, L, s));
    // the residual-extended planes' zero blocks, which the splits of every build leave alone
    const size_t u = 4 * (size_t)d.N * d.Np * 2, v = 4 * (size_t)d.Ap * d.Np * 2;
    CK(cudaMemsetAsync(ws + L.hAH, 0, u, s));
    CK(cudaMemsetAsync(ws + L.hAF, 0, u, s));
    CK(cudaMemsetAsync(ws + L.cPH, 0, v, s));
    CK(cudaMemsetAsync(ws + L.cPF, 0, v, s));
  }
  prof_end(DONOF_PHASE_PREPARE_B, s);
  std::lock_guard<std::mutex> lk(g_mu);
  g_reg[workspace] = Registration{B, *prob};
  return DONOF_OK;
}

namespace donof {
namespace {
// What one call of the build runs: the whole build; one shard of a build sharded over the
// auxiliary index (its two-electron partial sums J, K and G, nothing after them); or the
// part after the exchange (E, dE/dgamma, lambda from the summed partial sums).
enum BuildMode { kFull = 0, kPartial = 1, kFinish = 2 };

int run_build(const donof_problem* prob, const double* h, const double* B, const double* C,
              const double* gamma, const int32_t* pair_map, void* workspace,
              size_t workspace_bytes, BuildMode mode, double* partial, double* E, double* lam,
              double* dE_dgamma, cudaStream_t s) {
  int rc = check_problem(prob);
  if (rc != DONOF_OK) return rc;
  if (!h || !C || !gamma || !pair_map) return DONOF_ERR_INVALID_ARG;
  if (mode != kPartial && !E) return DONOF_ERR_INVALID_ARG;
  if (mode != kFull && !partial) return DONOF_ERR_INVALID_ARG;
  if (mode != kFinish && !B) return DONOF_ERR_INVALID_ARG;
  rc = check_ws(prob, workspace, workspace_bytes);
  if (rc != DONOF_OK) return rc;
  if (mode != kFinish) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_reg.find(workspace);
    if (it == g_reg.end() || it->second.B != B || !same_problem(it->second.prob, *prob))
      return DONOF_ERR_NOT_PREPARED;
  }
  const Dims d = make_dims(prob);
  const Layout L = make_layout(d);
  char* ws = (char*)workspace;
  const int N = d.N, A = d.A;
  const size_t AA = (size_t)A * A * 8;

  prof_begin(DONOF_PHASE_PREP, s);
  CK(cudaMemsetAsync(&((DevHeader*)(ws + L.header))->abort_flag, 0, sizeof(int32_t), s));
  CK(launch_occupations(d, gamma, pair_map, ws, L, s));
  CK(launch_coefficients(d, pair_map, ws, L, s));
  // hC = h C_act (FP64 DGEMM, or on the tensor cores with residual-extended operands), then
  // H_pp and G = n o hC
  if (d.precision == DONOF_MIXED) {
    CK(launch_split_C(d, C, h, ws, L, mode != kFinish, s));
    rc = run_hc_tc(d, ws, L, s);
    if (rc != DONOF_OK) return rc;
    // bound on ||C_act||_2 for the exponents of X in the G contraction
    if (mode != kFinish) CK(launch_gram_bound(d, C, ws, L, s));
  } else {
    CK(cudaMemsetAsync(ws + L.hC, 0, (size_t)N * A * 8, s));
    CK(launch_dgemm(split_k_args(N, A, N, h, N, 1, C, N, 1, (double*)(ws + L.hC), A, 1,
                                 (double*)(ws + L.skp)), s));
  }
  CK(launch_hdiag_ginit(d, C, ws, L, mode != kPartial, s));
  if (mode == kFinish) {  // the summed two-electron parts of every shard
    CK(cudaMemcpyAsync(ws + L.J, partial, AA, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(ws + L.K, partial + (size_t)A * A, AA, cudaMemcpyDeviceToDevice, s));
    CK(launch_add((double*)(ws + L.G), partial + 2 * (size_t)A * A, (long long)N * A, s));
  } else {
    CK(cudaMemsetAsync(ws + L.J, 0, AA, s));
    CK(cudaMemsetAsync(ws + L.K, 0, AA, s));
  }
  prof_end(DONOF_PHASE_PREP, s);

  for (int p0 = 0; p0 < d.Q && mode != kFinish; p0 += d.pb) {
    const int np = (d.Q - p0) < d.pb ? (d.Q - p0) : d.pb;
    if (d.precision == DONOF_MIXED) {
      rc = run_tc_block(d, p0, np, ws, L, s);
      if (rc != DONOF_OK) return rc;
      continue;
    }
    // ---- FP64 path
    const double* Bblk;
    prof_begin(DONOF_PHASE_HALF_TRANSFORM, s);
    if (d.layout == DONOF_B_PACKED) {
      CK(launch_unpack_B(d, B, p0, np, (double*)(ws + L.Bun), s));
      Bblk = (const double*)(ws + L.Bun);
    } else {
      Bblk = B + (size_t)p0 * N * N;
    }
    double* X = (double*)(ws + L.X64);
    double* b = (double*)(ws + L.b64);
    double* Y = (double*)(ws + L.Y64);
    {  // X[P][mu][q] = sum_nu B[P][mu][nu] C[nu][q]
      DgemmArgs a{};
      a.M = np * N; a.N = A; a.K = N; a.KB = 1; a.batch = 1; a.ksplit = 1;
      a.A = Bblk; a.sAm = N; a.sAk = 1;
      a.B = C; a.sBk = N; a.sBn = 1;
      a.C = X; a.sCm = A; a.sCn = 1;
      a.alpha = 1.0;
      CK(launch_dgemm(a, s));
    }
    prof_end(DONOF_PHASE_HALF_TRANSFORM, s);
    prof_begin(DONOF_PHASE_MO_3INDEX, s);
    {  // b[P][p][q] = sum_mu C[mu][p] X[P][mu][q]
      DgemmArgs a{};
      a.M = A; a.N = A; a.K = N; a.KB = 1; a.batch = np; a.ksplit = 1;
      a.A = C; a.sAm = 1; a.sAk = N;
      a.B = X; a.sBb = (long long)N * A; a.sBk = A; a.sBn = 1;
      a.C = b; a.sCb = (long long)A * A; a.sCm = A; a.sCn = 1;
      a.alpha = 1.0;
      CK(launch_dgemm(a, s));
    }
    prof_end(DONOF_PHASE_MO_3INDEX, s);
    prof_begin(DONOF_PHASE_JK_Y, s);
    CK(launch_jk_accumulate_f64(d, b, np, A, ws, L, s));
    CK(launch_build_Y_f64(d, b, Y, np, ws, L, s));
    prof_end(DONOF_PHASE_JK_Y, s);
    prof_begin(DONOF_PHASE_G_BUILD, s);
    {  // G[mu][p] += sum_P sum_q X[P][mu][q] Y[P][q][p]
      DgemmArgs a{};
      a.M = N; a.N = A; a.K = A; a.KB = np; a.batch = 1;
      a.ksplit = g_splits_fp64(N, A, np);
      a.part = (double*)(ws + L.skp);
      a.A = X; a.sAm = A; a.sAk = 1; a.sAkb = (long long)N * A;
      a.B = Y; a.sBk = A; a.sBn = 1; a.sBkb = (long long)A * A;
      a.C = (double*)(ws + L.G); a.sCm = A; a.sCn = 1;
      a.alpha = 1.0; a.beta = 1.0;
      CK(launch_dgemm(a, s));
    }
    prof_end(DONOF_PHASE_G_BUILD, s);
  }

  if (mode == kPartial) {  // this shard's J, K and two-electron G, for the exchange
    CK(cudaMemcpyAsync(partial, ws + L.J, AA, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(partial + (size_t)A * A, ws + L.K, AA, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(partial + 2 * (size_t)A * A, ws + L.G, (size_t)N * A * 8,
                       cudaMemcpyDeviceToDevice, s));
    return DONOF_OK;
  }

  prof_begin(DONOF_PHASE_ENERGY_LAMBDA, s);
  CK(launch_energy(d, pair_map, ws, L, E, dE_dgamma, s));
  if (lam) {  // lambda_qp = C_q^T G_p (q < N, p < nact), zero for p >= nact
    CK(cudaMemsetAsync(lam, 0, (size_t)N * N * 8, s));
    if (d.precision == DONOF_MIXED) {
      rc = run_lambda_tc(d, C, ws, L, lam, s);
      if (rc != DONOF_OK) return rc;
    } else {
      CK(launch_dgemm(split_k_args(N, A, N, C, 1, N, (const double*)(ws + L.G), A, 1, lam, N, 1,
                                   (double*)(ws + L.skp)),
                      s));
    }
  }
  prof_end(DONOF_PHASE_ENERGY_LAMBDA, s);
  return DONOF_OK;
}
}  // namespace
}  // namespace donof

extern "C" int donof_energy_lagrangian(const donof_problem* prob, const double* h, const double* B,
                                       const double* C, const double* gamma,
                                       const int32_t* pair_map, void* workspace,
                                       size_t workspace_bytes, double* E, double* lam,
                                       double* dE_dgamma, void* stream) {
  return run_build(prob, h, B, C, gamma, pair_map, workspace, workspace_bytes, kFull, nullptr, E,
                   lam, dE_dgamma, (cudaStream_t)stream);
}

extern "C" int donof_partial_size(const donof_problem* prob, size_t* count) {
  const int rc = check_problem(prob);
  if (rc != DONOF_OK) return rc;
  if (!count) return DONOF_ERR_INVALID_ARG;
  const size_t A = (size_t)prob->npair * (1 + prob->ncwo) + prob->nsingle;
  *count = 2 * A * A + (size_t)prob->nbf * A;
  return DONOF_OK;
}

extern "C" int donof_energy_lagrangian_partial(const donof_problem* prob, const double* h,
                                               const double* B, const double* C,
                                               const double* gamma, const int32_t* pair_map,
                                               void* workspace, size_t workspace_bytes,
                                               double* partial, void* stream) {
  return run_build(prob, h, B, C, gamma, pair_map, workspace, workspace_bytes, kPartial, partial,
                   nullptr, nullptr, nullptr, (cudaStream_t)stream);
}

extern "C" int donof_energy_lagrangian_finish(const donof_problem* prob, const double* h,
                                              const double* C, const double* gamma,
                                              const int32_t* pair_map, const double* partial,
                                              void* workspace, size_t workspace_bytes, double* E,
                                              double* lam, double* dE_dgamma, void* stream) {
  return run_build(prob, h, nullptr, C, gamma, pair_map, workspace, workspace_bytes, kFinish,
                   const_cast<double*>(partial), E, lam, dE_dgamma, (cudaStream_t)stream);
}

extern "C" int donof_energy_backward(const donof_problem* prob, const double* Ebar,
                                     const void* workspace, size_t workspace_bytes, double* dE_dC,
                                     double* dE_dgamma, void* stream) {
  int rc = check_problem(prob);
  if (rc != DONOF_OK) return rc;
  if (!Ebar) return DONOF_ERR_INVALID_ARG;
  rc = check_ws(prob, workspace, workspace_bytes);
  if (rc != DONOF_OK) return rc;
  const Dims d = make_dims(prob);
  const Layout L = make_layout(d);
  prof_begin(DONOF_PHASE_BACKWARD, (cudaStream_t)stream);
  CK(launch_backward(d, Ebar, (const char*)workspace, L, dE_dC, dE_dgamma, (cudaStream_t)stream));
  prof_end(DONOF_PHASE_BACKWARD, (cudaStream_t)stream);
  return DONOF_OK;
}

extern "C" int donof_get_jk(const donof_problem* prob, const void* workspace,
                            size_t workspace_bytes, double* J, double* K, void* stream) {
  int rc = check_problem(prob);
  if (rc != DONOF_OK) return rc;
  rc = check_ws(prob, workspace, workspace_bytes);
  if (rc != DONOF_OK) return rc;
  const Dims d = make_dims(prob);
  const Layout L = make_layout(d);
  const size_t bytes = (size_t)d.A * d.A * 8;
  cudaStream_t s = (cudaStream_t)stream;
  if (J) CK(cudaMemcpyAsync(J, (const char*)workspace + L.J, bytes, cudaMemcpyDeviceToDevice, s));
  if (K) CK(cudaMemcpyAsync(K, (const char*)workspace + L.K, bytes, cudaMemcpyDeviceToDevice, s));
  return DONOF_OK;
}

extern "C" int donof_read_status(const void* workspace, int32_t* status, void* stream) {
  if (!workspace || !status) return DONOF_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaStreamSynchronize(s));
  int32_t v = 0;
  CK(cudaMemcpy(&v, workspace, sizeof(int32_t), cudaMemcpyDeviceToHost));
  const int32_t zero = 0;
  CK(cudaMemcpy((void*)workspace, &zero, sizeof(int32_t), cudaMemcpyHostToDevice));
  *status = v;
  return DONOF_OK;
}

// Staging of donof_energy_lagrangian_host: device copies of C, gamma, E, the upstream gradient
// 1, lambda, dE/dgamma and dE/dC, each 256-byte aligned.
namespace donof {
namespace {
struct Stage {
  size_t C, g, E, Ebar, lam, dg, dC, total;
};
Stage stage_layout(const donof_problem* p) {
  Stage st{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + (bytes ? bytes : 1));
    return o;
  };
  const size_t nn = (size_t)p->nbf * p->nbf * 8, ng = (size_t)p->npair * p->ncwo * 8;
  st.C = take(nn);
  st.g = take(ng);
  st.E = take(8);
  st.Ebar = take(8);
  st.lam = take(nn);
  st.dg = take(ng);
  st.dC = take(nn);
  st.total = off;
  return st;
}
}  // namespace
}  // namespace donof

extern "C" int donof_host_staging_size(const donof_problem* prob, size_t* bytes) {
  if (!prob || !bytes) return DONOF_ERR_INVALID_ARG;
  size_t w = 0;
  const int rc = donof_workspace_size(prob, &w);  // validates the problem
  if (rc != DONOF_OK) return rc;
  *bytes = stage_layout(prob).total;
  return DONOF_OK;
}

extern "C" int donof_energy_lagrangian_host(const donof_problem* prob, const double* h,
                                            const double* B, const double* C_host,
                                            const double* gamma_host, const int32_t* pair_map,
                                            void* workspace, size_t workspace_bytes,
                                            void* staging, size_t staging_bytes, double* E_host,
                                            double* lam_host, double* dE_dgamma_host,
                                            double* dE_dC_host, void* stream) {
  if (!prob || !C_host || !gamma_host || !E_host || !staging) return DONOF_ERR_INVALID_ARG;
  size_t need = 0;
  int rc = donof_host_staging_size(prob, &need);
  if (rc != DONOF_OK) return rc;
  if (staging_bytes < need || ((uintptr_t)staging % kAlign) != 0) return DONOF_ERR_WORKSPACE;
  const Stage st = stage_layout(prob);
  char* sg = (char*)staging;
  double* Cd = (double*)(sg + st.C);
  double* gd = (double*)(sg + st.g);
  double* Ed = (double*)(sg + st.E);
  double* Ebar = (double*)(sg + st.Ebar);
  double* lamd = (double*)(sg + st.lam);
  double* dgd = (double*)(sg + st.dg);
  double* dCd = (double*)(sg + st.dC);
  const size_t nn = (size_t)prob->nbf * prob->nbf * 8, ng = (size_t)prob->npair * prob->ncwo * 8;
  cudaStream_t s = (cudaStream_t)stream;
  static const double kOne = 1.0;
  CK(cudaMemcpyAsync(Cd, C_host, nn, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(gd, gamma_host, ng, cudaMemcpyHostToDevice, s));
  if (dE_dC_host) CK(cudaMemcpyAsync(Ebar, &kOne, 8, cudaMemcpyHostToDevice, s));
  rc = donof_energy_lagrangian(prob, h, B, Cd, gd, pair_map, workspace, workspace_bytes, Ed,
                               lam_host ? lamd : nullptr, dE_dgamma_host ? dgd : nullptr, stream);
  if (rc != DONOF_OK) return rc;
  if (dE_dC_host) {
    rc = donof_energy_backward(prob, Ebar, workspace, workspace_bytes, dCd, nullptr, stream);
    if (rc != DONOF_OK) return rc;
  }
  CK(cudaMemcpyAsync(E_host, Ed, 8, cudaMemcpyDeviceToHost, s));
  if (lam_host) CK(cudaMemcpyAsync(lam_host, lamd, nn, cudaMemcpyDeviceToHost, s));
  if (dE_dgamma_host) CK(cudaMemcpyAsync(dE_dgamma_host, dgd, ng, cudaMemcpyDeviceToHost, s));
  if (dE_dC_host) CK(cudaMemcpyAsync(dE_dC_host, dCd, nn, cudaMemcpyDeviceToHost, s));
  int32_t status = DONOF_OK;
  rc = donof_read_status(workspace, &status, stream);  // waits for the stream
  if (rc != DONOF_OK) return rc;
  return status;
}

extern "C" int donof_profile_enable(int32_t enable) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (enable) prof_clear_locked();
  g_prof_on = enable != 0;
  return DONOF_OK;
}

extern "C" int donof_profile_read(int32_t phase, double* total_ms, int32_t* intervals) {
  if (phase < 0 || phase >= DONOF_NUM_PHASES || !total_ms) return DONOF_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  double t = 0.0;
  int n = 0;
  for (auto& e : g_prof[phase].ev) {
    if (cudaEventSynchronize(e.second) != cudaSuccess) return DONOF_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.first, e.second) != cudaSuccess) return DONOF_ERR_CUDA;
    t += ms;
    ++n;
  }
  *total_ms = t;
  if (intervals) *intervals = n;
  return DONOF_OK;
}

extern "C" int64_t donof_launch_count(void) { return (int64_t)g_launches.load(); }

extern "C" const char* donof_status_string(int status) {
  switch (status) {
    case DONOF_OK: return "ok";
    case DONOF_ERR_INVALID_ARG: return "invalid argument";
    case DONOF_ERR_PAIR_MAP: return "pair_map violates the subspace layout";
    case DONOF_ERR_NONFINITE: return "non-finite input or result";
    case DONOF_ERR_WORKSPACE: return "workspace too small or misaligned";
    case DONOF_ERR_CUDA: return "CUDA call failed";
    case DONOF_ERR_TIMEOUT: return "device wait limit exceeded";
    case DONOF_ERR_UNSUPPORTED: return "unsupported problem size";
    case DONOF_ERR_NOT_PREPARED: return "donof_prepare_B not called for this workspace and B";
    default: return "unknown status";
  }
}
