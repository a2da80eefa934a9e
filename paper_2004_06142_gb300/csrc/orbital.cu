// Hand-off to the orbital update (Sec. III.B): the symmetric matrix F of Eq. Fockian from the
// Lagrangian lambda and a given diagonal, its FP64 eigendecomposition, the rotated orbitals
// C V and their FP64 reorthonormalisation (one Newton-Schulz step C (3I - C^T C) / 2).
// The eigendecomposition is this library's own FP64 solver (eigh.cu).
#include <vector>

#include "common.cuh"

namespace donof {
namespace {

// F[q][p] per Eq. Fockian (row-major, symmetric), diagonal from Fdiag.
__global__ void k_fockian(const double* __restrict__ lam, const double* __restrict__ Fdiag, int N,
                          double* F) {
  const long long tot = (long long)N * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(i / N), p = (int)(i % N);
    double v;
    if (q == p) v = Fdiag[p];
    else if (q < p) v = lam[(size_t)q * N + p] - lam[(size_t)p * N + q];
    else v = lam[(size_t)p * N + q] - lam[(size_t)q * N + p];
    F[i] = v;
  }
}

// M = (3 I - S) / 2
__global__ void k_newton_schulz(const double* __restrict__ S, int N, double* M) {
  const long long tot = (long long)N * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / N), c = (int)(i % N);
    M[i] = ((r == c ? 3.0 : 0.0) - S[i]) * 0.5;
  }
}

DgemmArgs plain(int M, int N, int K, const double* A, long long sAm, long long sAk,
                const double* B, long long sBk, long long sBn, double* C, double beta = 0.0) {
  DgemmArgs a{};
  a.M = M; a.N = N; a.K = K; a.KB = 1; a.batch = 1; a.ksplit = 1;
  a.A = A; a.sAm = sAm; a.sAk = sAk;
  a.B = B; a.sBk = sBk; a.sBn = sBn;
  a.C = C; a.sCm = N; a.sCn = 1;
  a.alpha = 1.0; a.beta = beta;
  return a;
}

// M[i][j] = M[j][i] for i < j: the upper triangle from the lower one (a symmetric product
// formed on its lower-triangle tiles only)
__global__ void k_mirror_lower(double* M, int N) {
  const long long tot = (long long)N * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / N), c = (int)(i % N);
    if (r < c) M[i] = M[(size_t)c * N + r];
  }
}

// A symmetric product C_out (+)= A B formed on the lower-triangle tiles, then mirrored.
int sym_product(DgemmArgs a, cudaStream_t s) {
  a.lower = 1;
  if (launch_dgemm(a, s) != cudaSuccess) return DONOF_ERR_CUDA;
  k_mirror_lower<<<152 * 4, 256, 0, s>>>(a.C, a.N);
  count_launch(1);
  return cudaGetLastError() == cudaSuccess ? DONOF_OK : DONOF_ERR_CUDA;
}

}  // namespace
}  // namespace donof

using namespace donof;

extern "C" int donof_orbital_update_workspace_size(int32_t nbf, size_t* bytes) {
  if (nbf < 1 || nbf > kEighMaxN || !bytes) return DONOF_ERR_INVALID_ARG;
  const size_t nn = (size_t)nbf * nbf * 8;
  *bytes = 3 * align_up(nn) + eigh_workspace_bytes(nbf);
  return DONOF_OK;
}

extern "C" int donof_orbital_update(int32_t nbf, const double* lam, const double* Fdiag,
                                    const double* C, void* workspace, size_t workspace_bytes,
                                    double* C_new, double* eps, void* stream) {
  if (!lam || !Fdiag || !C || !C_new || !eps) return DONOF_ERR_INVALID_ARG;
  size_t need = 0;
  int rc = donof_orbital_update_workspace_size(nbf, &need);
  if (rc != DONOF_OK) return rc;
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace % kAlign) != 0)
    return DONOF_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const int N = nbf;
  const size_t nn = align_up((size_t)N * N * 8);
  char* ws = (char*)workspace;
  double* F = (double*)ws;             // F, then its eigenvectors V (row-major)
  double* T = (double*)(ws + nn);      // C V
  double* S = (double*)(ws + 2 * nn);  // T^T T, then (3I - T^T T) / 2
  char* ews = ws + 3 * nn;             // the eigensolver's workspace

  prof_begin(DONOF_PHASE_ORBITAL_UPDATE, s);
  k_fockian<<<152 * 4, 256, 0, s>>>(lam, Fdiag, N, F);
  count_launch(1);
  if (cudaGetLastError() != cudaSuccess) return DONOF_ERR_CUDA;
  // F = V diag(eps) V^T, V over F's storage (row-major, column j = eigenvector j)
  rc = eigh_run(N, F, F, eps, ews, s);
  if (rc != DONOF_OK) return rc;
  // T[mu][j] = sum_i C[mu][i] V[i][j]
  if (launch_dgemm(plain(N, N, N, C, N, 1, F, N, 1, T), s) != cudaSuccess) return DONOF_ERR_CUDA;
  // S = T^T T;  M = (3I - S) / 2;  C_new = T M
  if (sym_product(plain(N, N, N, T, 1, N, T, N, 1, S), s) != DONOF_OK) return DONOF_ERR_CUDA;
  k_newton_schulz<<<152 * 4, 256, 0, s>>>(S, N, S);
  count_launch(1);
  if (cudaGetLastError() != cudaSuccess) return DONOF_ERR_CUDA;
  if (launch_dgemm(plain(N, N, N, T, N, 1, S, N, 1, C_new), s) != cudaSuccess)
    return DONOF_ERR_CUDA;
  prof_end(DONOF_PHASE_ORBITAL_UPDATE, s);
  return DONOF_OK;
}

// ---------------------------------------------------------------------------
// The optimisation procedure around the build (Sec. III.B-D): outer iterations of an
// occupation optimisation at fixed orbitals followed by orbital iterations at fixed
// occupations, each a diagonalisation of F (Eq. Fockian) with the previous eigenvalues on
// its diagonal, its off-diagonal zeta-scaled (Sec. III.B) and DIIS-extrapolated (Sec.
// III.C); converged when max |lambda_qp - lambda_pq| < delta and the energy of an outer
// iteration changed by less than eps_energy.  The host drives the loop and reads two
// device scalars per build; every arithmetic step runs in this library's kernels.
//
// Readings: F^j and its error vector e^j = offdiag F^j are taken to the fixed AO basis
// (C F C^T, C e C^T) so that matrices of different iterations can be combined; with
// lambda = C^T G (G = dE/dC / 4) the energy-lowering assignment of eigenvectors to orbitals
// is by decreasing eigenvalue, and those eigenvalues are the next diagonal; the initial
// diagonal (when requested) is minus the eigenvalues of the symmetrised lambda, whose
// eigenvectors also rotate the start orbitals.
// ---------------------------------------------------------------------------
namespace donof {
namespace {

constexpr int kMaxDepth = 16;
constexpr double kDiisMaxCoefficient = 100.0;

// the history slots in use, oldest first (the newest last)
struct Slots {
  int n;
  int idx[kMaxDepth];
};

struct OptLayout {
  size_t lam, Emo, T1, T2, Fbar, hist, eps, scal, B, c, work;
  size_t skp;  // split-K partials of R_a C^T (nact x N)
  size_t total;
};

int opt_layout(int N, int A, int depth, OptLayout* o) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t r = off;
    off = align_up(off + (bytes ? bytes : 1));
    return r;
  };
  const size_t nn = (size_t)N * N * 8;
  const int m = depth < 1 ? 1 : depth;
  o->lam = take(nn);
  o->Emo = take(nn);
  o->T1 = take(nn);
  o->T2 = take(nn);
  o->Fbar = take(nn);
  o->hist = take(2 * (size_t)m * nn);  // per slot: F_AO, then e_AO
  o->eps = take((size_t)N * 8);
  o->scal = take(8 * 8);                // [0] E, [1] asym bits, [2] E of the occupation step
  o->B = take((size_t)kMaxDepth * kMaxDepth * 8);
  o->c = take((size_t)(kMaxDepth + 2) * 8);  // c[0..n]; the restart flag kept at [kMaxDepth + 1]
  o->work = take(eigh_workspace_bytes(N));  // the eigensolver's workspace
  const int ks = splitk_count(A, N, N);
  o->skp = take(ks > 1 ? (size_t)ks * A * N * 8 : 0);
  o->total = off;
  return DONOF_OK;
}

__global__ void k_asym_max(const double* __restrict__ lam, int N, unsigned long long* out) {
  double m = 0.0;
  const long long tot = (long long)N * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(i / N), p = (int)(i % N);
    if (q < p) m = fmax(m, fabs(lam[i] - lam[(size_t)p * N + q]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (threadIdx.x % 32 == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// Off-diagonal of F (Eq. Fockian), each element above zeta in magnitude divided by ten until
// it is not (Sec. III.B; zeta <= 0: unscaled); zero diagonal.
__global__ void k_fockian_offdiag(const double* __restrict__ lam, int N, double zeta, double* E) {
  const long long tot = (long long)N * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(i / N), p = (int)(i % N);
    double v = 0.0;
    if (q < p) v = lam[(size_t)q * N + p] - lam[(size_t)p * N + q];
    else if (q > p) v = lam[(size_t)p * N + q] - lam[(size_t)q * N + p];
    if (zeta > 0.0)
      while (fabs(v) > zeta) v /= 10.0;
    E[i] = v;
  }
}

// M[q][p] /= 2 for q, p < A (the active block of the first A rows)
__global__ void k_halve_block(double* M, int N, int A) {
  const long long tot = (long long)A * A;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x)
    M[(size_t)(i / A) * N + (i % A)] *= 0.5;
}

// S = Z + Z^T
__global__ void k_sym_sum(const double* __restrict__ Z, int N, double* S) {
  const long long tot = (long long)N * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / N), c = (int)(i % N);
    S[i] = Z[i] + Z[(size_t)c * N + r];
  }
}

// T[mu][p] = C[mu][p] * d[p]
__global__ void k_scale_cols(const double* __restrict__ C, const double* __restrict__ dg, int N,
                             double* T) {
  const long long tot = (long long)N * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x)
    T[i] = C[i] * dg[i % N];
}

// B[new][k] = B[k][new] = <e_new, e_k> for the slots in use (one block per slot, fixed order).
__global__ void __launch_bounds__(1024) k_diis_dots(const double* __restrict__ hist, Slots sl,
                                                    size_t nn, double* Bm, int ldB) {
  __shared__ double red[32];
  const int snew = sl.idx[sl.n - 1];
  const int k = sl.idx[blockIdx.x];
  const double* en = hist + (2 * (size_t)snew + 1) * nn;
  const double* ek = hist + (2 * (size_t)k + 1) * nn;
  double s = 0.0;
  for (size_t i = threadIdx.x; i < nn; i += blockDim.x) s += en[i] * ek[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    Bm[(size_t)snew * ldB + k] = t;
    Bm[(size_t)k * ldB + snew] = t;
  }
}

// Coefficients of Sec. III.C over the slots in use: [[B, -1], [-1, 0]] [c; Lambda] =
// [0; -1] by Gaussian elimination with partial pivoting (one thread).  A singular system,
// or a coefficient above kDiisMaxCoefficient in magnitude, sets the restart flag c[n]
// (the newest matrix is then used alone and the history restarts from it).
__global__ void k_diis_solve(const double* __restrict__ Bm, int ldB, Slots sl, double* c) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double M[kMaxDepth + 1][kMaxDepth + 2];
  const int m = sl.n, n = m + 1;
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) M[i][j] = Bm[(size_t)sl.idx[i] * ldB + sl.idx[j]];
    M[i][m] = -1.0;
    M[i][n] = 0.0;
  }
  for (int j = 0; j < m; ++j) M[m][j] = -1.0;
  M[m][m] = 0.0;
  M[m][n] = -1.0;
  bool restart = false;
  for (int col = 0; col < n && !restart; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
    if (piv != col)
      for (int j = 0; j <= n; ++j) {
        const double t = M[col][j];
        M[col][j] = M[piv][j];
        M[piv][j] = t;
      }
    const double d = M[col][col];
    if (d == 0.0) {
      restart = true;
      break;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = M[r][col] / d;
      if (f != 0.0)
        for (int j = col; j <= n; ++j) M[r][j] -= f * M[col][j];
    }
  }
  if (!restart)
    for (int i = 0; i < m; ++i) {
      c[i] = M[i][n] / M[i][i];
      if (!(fabs(c[i]) <= kDiisMaxCoefficient)) restart = true;
    }
  c[m] = restart ? 1.0 : 0.0;
}

// Fbar = sum_i c_i F_AO^{slot i} (or the newest one alone when the restart flag is set)
__global__ void k_diis_combine(const double* __restrict__ hist, const double* __restrict__ c,
                               Slots sl, size_t nn, double* Fbar) {
  const bool single = c[sl.n] != 0.0;
  const int snew = sl.idx[sl.n - 1];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn;
       i += (size_t)gridDim.x * blockDim.x) {
    double v;
    if (single) {
      v = hist[2 * (size_t)snew * nn + i];
    } else {
      v = 0.0;
      for (int k = 0; k < sl.n; ++k) v += c[k] * hist[2 * (size_t)sl.idx[k] * nn + i];
    }
    Fbar[i] = v;
  }
}

// Eigenvectors (columns of the row-major eigenvector matrix W) in decreasing eigenvalue order
// as the columns of C; the eigenvalues in that order as the next diagonal.
__global__ void k_take_descending(const double* __restrict__ W, const double* __restrict__ eps,
                                  int N, double* C, double* Fdiag) {
  const long long tot = (long long)N * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int mu = (int)(i / N), p = (int)(i % N);
    C[i] = W[(size_t)mu * N + (N - 1 - p)];
    if (mu == 0) Fdiag[p] = eps[N - 1 - p];
  }
}

// S <- (S + S^T) / 2 (the symmetrised lambda); eps -> -eps
__global__ void k_symmetrise(const double* __restrict__ lam, int N, double* S) {
  const long long tot = (long long)N * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(i / N), p = (int)(i % N);
    S[i] = 0.5 * (lam[i] + lam[(size_t)p * N + q]);
  }
}
__global__ void k_negate(const double* __restrict__ x, int n, double* y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    y[i] = -x[i];
}

struct Loop {
  const donof_problem* prob;
  const double *h, *B;
  const int32_t* pm;
  double *C, *gamma, *Fdiag;
  void* bws;
  size_t bbytes;
  char* ows;
  OptLayout L;
  int N;
  cudaStream_t s;
};

bool ok(cudaError_t e) { return e == cudaSuccess; }

// one build at (C, gamma): E and lambda into the loop workspace, asym computed; returns
// DONOF_OK and the host copies of E and asym
int loop_build(Loop& lp, double* E, double* asym) {
  char* o = lp.ows;
  int rc = donof_energy_lagrangian(lp.prob, lp.h, lp.B, lp.C, lp.gamma, lp.pm, lp.bws, lp.bbytes,
                                   (double*)(o + lp.L.scal), (double*)(o + lp.L.lam), nullptr,
                                   lp.s);
  if (rc != DONOF_OK) return rc;
  if (!ok(cudaMemsetAsync(o + lp.L.scal + 8, 0, 8, lp.s))) return DONOF_ERR_CUDA;
  k_asym_max<<<152, 256, 0, lp.s>>>((const double*)(o + lp.L.lam), lp.N,
                                     (unsigned long long*)(o + lp.L.scal + 8));
  count_launch(1);
  if (!ok(cudaGetLastError())) return DONOF_ERR_CUDA;
  double hv[2];
  if (!ok(cudaMemcpyAsync(hv, o + lp.L.scal, 16, cudaMemcpyDeviceToHost, lp.s)) ||
      !ok(cudaStreamSynchronize(lp.s)))
    return DONOF_ERR_CUDA;
  int32_t st = 0;
  rc = donof_read_status(lp.bws, &st, lp.s);
  if (rc != DONOF_OK) return rc;
  if (st != DONOF_OK) return st;
  *E = hv[0];
  *asym = hv[1];
  return DONOF_OK;
}

int loop_occupations(Loop& lp, int max_iter, double gtol) {
  return donof_optimize_occupations(lp.prob, lp.pm, lp.gamma, lp.bws, lp.bbytes, max_iter, gtol,
                                    (double*)(lp.ows + lp.L.scal + 16), nullptr, lp.s);
}

// C <- C (3 I - C^T C) / 2 through T1 (C^T C, then the factor) and T2 (the product)
int loop_reorthonormalise(Loop& lp) {
  const int N = lp.N;
  double* T1 = (double*)(lp.ows + lp.L.T1);
  double* T2 = (double*)(lp.ows + lp.L.T2);
  if (sym_product(plain(N, N, N, lp.C, 1, N, lp.C, N, 1, T1), lp.s) != DONOF_OK)
    return DONOF_ERR_CUDA;
  k_newton_schulz<<<152 * 4, 256, 0, lp.s>>>(T1, N, T1);
  count_launch(1);
  if (!ok(launch_dgemm(plain(N, N, N, lp.C, N, 1, T1, N, 1, T2), lp.s))) return DONOF_ERR_CUDA;
  if (!ok(cudaMemcpyAsync(lp.C, T2, (size_t)N * N * 8, cudaMemcpyDeviceToDevice, lp.s)))
    return DONOF_ERR_CUDA;
  return DONOF_OK;
}

// one diagonalisation step; `active` lists the history slots in use, oldest first, and is
// updated (the new matrix takes a free slot, the oldest is dropped when all are in use);
int loop_orbital_step(Loop& lp, double zeta, int depth, std::vector<int>& active) {
  const int N = lp.N;
  const size_t nn = (size_t)N * N;
  const int slots = depth < 1 ? 1 : depth;
  char* o = lp.ows;
  const int slot = active.empty() ? 0 : (active.back() + 1) % slots;
  if ((int)active.size() == slots) active.erase(active.begin());
  active.push_back(slot);
  double* lam = (double*)(o + lp.L.lam);
  double* Emo = (double*)(o + lp.L.Emo);
  double* T1 = (double*)(o + lp.L.T1);
  double* Fbar = (double*)(o + lp.L.Fbar);
  double* hist = (double*)(o + lp.L.hist);
  double* F_ao = hist + 2 * (size_t)slot * nn;
  double* e_ao = F_ao + nn;
  double* c = (double*)(o + lp.L.c);
  prof_begin(DONOF_PHASE_ORBITAL_STEP, lp.s);
  k_fockian_offdiag<<<152 * 4, 256, 0, lp.s>>>(lam, N, zeta, Emo);
  count_launch(1);
  // e_AO = C Emo C^T.  Emo vanishes between inactive orbitals (lambda_qp = 0 for p >= nact),
  // so Emo = R + R^T with R = [Emo_aa / 2, Emo_ai; 0, 0] (nonzero in the nact active rows
  // only) and e_AO = Z + Z^T with Z = C_a (R_a C^T): two products of rank nact.
  const int A = lp.prob->npair * (1 + lp.prob->ncwo) + lp.prob->nsingle;
  double* W = (double*)(o + lp.L.T2);  // R_a C^T, nact x N
  k_halve_block<<<152, 256, 0, lp.s>>>(Emo, N, A);
  count_launch(1);
  if (!ok(cudaMemsetAsync(W, 0, (size_t)A * N * 8, lp.s)) ||
      !ok(launch_dgemm(split_k_args(A, N, N, Emo, N, 1, lp.C, 1, N, W, N, 1,
                                    (double*)(o + lp.L.skp)),
                       lp.s)) ||
      !ok(launch_dgemm(plain(N, N, A, lp.C, N, 1, W, N, 1, T1), lp.s)))
    return DONOF_ERR_CUDA;
  k_sym_sum<<<152 * 4, 256, 0, lp.s>>>(T1, N, e_ao);
  count_launch(1);
  // F_AO = e_AO + (C diag(Fdiag)) C^T, symmetric
  k_scale_cols<<<152 * 4, 256, 0, lp.s>>>(lp.C, lp.Fdiag, N, T1);
  count_launch(1);
  if (!ok(cudaMemcpyAsync(F_ao, e_ao, nn * 8, cudaMemcpyDeviceToDevice, lp.s)) ||
      sym_product(plain(N, N, N, T1, N, 1, lp.C, 1, N, F_ao, 1.0), lp.s) != DONOF_OK ||
      !ok(cudaMemsetAsync(c + kMaxDepth + 1, 0, 8, lp.s)))
    return DONOF_ERR_CUDA;
  Slots sl{};
  sl.n = (int)active.size();
  for (int i = 0; i < sl.n; ++i) sl.idx[i] = active[i];
  if (depth >= 2) {
    double* Bm = (double*)(o + lp.L.B);
    k_diis_dots<<<sl.n, 1024, 0, lp.s>>>(hist, sl, nn, Bm, kMaxDepth);
    count_launch(1);
  }
  if (depth >= 2 && sl.n >= 2) {
    k_diis_solve<<<1, 32, 0, lp.s>>>((const double*)(o + lp.L.B), kMaxDepth, sl, c);
    k_diis_combine<<<152 * 4, 256, 0, lp.s>>>(hist, c, sl, nn, Fbar);
    count_launch(2);
    // the restart flag, for the host's history
    if (!ok(cudaMemcpyAsync(c + kMaxDepth + 1, c + sl.n, 8, cudaMemcpyDeviceToDevice, lp.s)))
      return DONOF_ERR_CUDA;
  } else {
    if (!ok(cudaMemcpyAsync(Fbar, F_ao, nn * 8, cudaMemcpyDeviceToDevice, lp.s)))
      return DONOF_ERR_CUDA;
  }
  if (!ok(cudaGetLastError())) return DONOF_ERR_CUDA;
  // Fbar symmetric: its row-major storage is its column-major storage
  // Fbar = V diag(eps) V^T, V over Fbar's storage (row-major, column j = eigenvector j)
  int rc = eigh_run(N, Fbar, Fbar, (double*)(o + lp.L.eps), o + lp.L.work, lp.s);
  if (rc != DONOF_OK) return rc;
  k_take_descending<<<152 * 4, 256, 0, lp.s>>>(Fbar, (const double*)(o + lp.L.eps), N, lp.C,
                                               lp.Fdiag);
  count_launch(1);
  if (!ok(cudaGetLastError())) return DONOF_ERR_CUDA;
  rc = loop_reorthonormalise(lp);
  if (rc != DONOF_OK) return rc;
  prof_end(DONOF_PHASE_ORBITAL_STEP, lp.s);
  // the restart decision is needed before the next step: read it now
  double flag = 0.0;
  if (!ok(cudaMemcpyAsync(&flag, c + kMaxDepth + 1, 8, cudaMemcpyDeviceToHost, lp.s)) ||
      !ok(cudaStreamSynchronize(lp.s)))
    return DONOF_ERR_CUDA;
  if (flag != 0.0) active.erase(active.begin(), active.end() - 1);
  return DONOF_OK;
}

// initial step: the symmetrised lambda of the current build rotates C; its eigenvalues,
// negated, are the first diagonal
int loop_initial_diagonal(Loop& lp) {
  const int N = lp.N;
  char* o = lp.ows;
  double* S = (double*)(o + lp.L.Fbar);
  double* T1 = (double*)(o + lp.L.T1);
  k_symmetrise<<<152 * 4, 256, 0, lp.s>>>((const double*)(o + lp.L.lam), N, S);
  count_launch(1);
  const int rc = eigh_run(N, S, S, (double*)(o + lp.L.eps), o + lp.L.work, lp.s);
  if (rc != DONOF_OK) return rc;
  // T1 = C V, V[i][j] = S[i * N + j] (ascending eigenvalues)
  if (!ok(launch_dgemm(plain(N, N, N, lp.C, N, 1, S, N, 1, T1), lp.s)) ||
      !ok(cudaMemcpyAsync(lp.C, T1, (size_t)N * N * 8, cudaMemcpyDeviceToDevice, lp.s)))
    return DONOF_ERR_CUDA;
  k_negate<<<8, 256, 0, lp.s>>>((const double*)(o + lp.L.eps), N, lp.Fdiag);
  count_launch(1);
  return ok(cudaGetLastError()) ? DONOF_OK : DONOF_ERR_CUDA;
}

}  // namespace
}  // namespace donof

extern "C" int donof_optimize_workspace_size(const donof_problem* prob, int32_t diis_depth,
                                             size_t* bytes) {
  if (!prob || !bytes || diis_depth < 0 || diis_depth > kMaxDepth) return DONOF_ERR_INVALID_ARG;
  size_t b = 0;
  int rc = donof_workspace_size(prob, &b);  // validates the problem
  if (rc != DONOF_OK) return rc;
  if (prob->nbf > kEighMaxN) return DONOF_ERR_UNSUPPORTED;
  OptLayout L;
  opt_layout(prob->nbf, prob->npair * (1 + prob->ncwo) + prob->nsingle, diis_depth, &L);
  *bytes = L.total;
  return DONOF_OK;
}

extern "C" int donof_optimize(const donof_problem* prob, const donof_opt_params* prm,
                              const double* h, const double* B, double* C, double* gamma,
                              const int32_t* pair_map, double* Fdiag, int32_t init_diagonal,
                              void* build_ws, size_t build_bytes, void* opt_ws, size_t opt_bytes,
                              donof_opt_result* result, double* energies, int32_t energies_cap,
                              void* stream) {
  if (!prob || !prm || !h || !B || !C || !gamma || !pair_map || !Fdiag || !result)
    return DONOF_ERR_INVALID_ARG;
  if (prm->max_outer < 1 || prm->max_inner < 1 || prm->diis_depth < 0 ||
      prm->diis_depth > kMaxDepth || prm->occ_max_iter < 0 || !(prm->occ_gtol > 0.0) ||
      energies_cap < 0 || (energies_cap > 0 && !energies))
    return DONOF_ERR_INVALID_ARG;
  size_t need = 0;
  int rc = donof_optimize_workspace_size(prob, prm->diis_depth, &need);
  if (rc != DONOF_OK) return rc;
  if (!opt_ws || opt_bytes < need || ((uintptr_t)opt_ws % kAlign) != 0) return DONOF_ERR_WORKSPACE;
  Loop lp;
  lp.prob = prob; lp.h = h; lp.B = B; lp.pm = pair_map;
  lp.C = C; lp.gamma = gamma; lp.Fdiag = Fdiag;
  lp.bws = build_ws; lp.bbytes = build_bytes;
  lp.ows = (char*)opt_ws;
  lp.N = prob->nbf;
  lp.s = (cudaStream_t)stream;
  opt_layout(lp.N, prob->npair * (1 + prob->ncwo) + prob->nsingle, prm->diis_depth, &lp.L);

  int nE = 0;
  auto record = [&](double E) {
    if (nE < energies_cap) energies[nE] = E;
    ++nE;
  };
  double E = 0.0, asym = 0.0;
  result->outer = result->inner = result->builds = result->converged = 0;
  // start: occupations at the given orbitals, then (optionally) the initial diagonal
  rc = loop_build(lp, &E, &asym);
  if (rc != DONOF_OK) return rc;
  result->builds++;
  rc = loop_occupations(lp, prm->occ_max_iter, prm->occ_gtol);
  if (rc != DONOF_OK) return rc;
  if (init_diagonal) {
    rc = loop_build(lp, &E, &asym);
    if (rc != DONOF_OK) return rc;
    result->builds++;
    rc = loop_initial_diagonal(lp);
    if (rc != DONOF_OK) return rc;
  }
  const int depth = prm->diis_depth;
  std::vector<int> active;  // DIIS history slots in use, oldest first
  bool have_outer = false;
  double E_outer = 0.0;
  for (int outer = 1; outer <= prm->max_outer; ++outer) {
    result->outer = outer;
    if (outer > 1) {
      rc = loop_build(lp, &E, &asym);
      if (rc != DONOF_OK) return rc;
      result->builds++;
      rc = loop_occupations(lp, prm->occ_max_iter, prm->occ_gtol);
      if (rc != DONOF_OK) return rc;
    }
    bool have_prev = false;
    double E_prev = 0.0;
    for (int inner = 0; inner < prm->max_inner; ++inner) {
      rc = loop_build(lp, &E, &asym);
      if (rc != DONOF_OK) return rc;
      result->builds++;
      record(E);
      if (asym < prm->delta) break;
      if (have_prev && fabs(E - E_prev) < prm->eps_energy) break;
      E_prev = E;
      have_prev = true;
      rc = loop_orbital_step(lp, prm->zeta, depth, active);
      if (rc != DONOF_OK) return rc;
      result->inner++;
    }
    if (asym < prm->delta && have_outer && fabs(E - E_outer) < prm->eps_energy) {
      result->converged = 1;
      break;
    }
    E_outer = E;
    have_outer = true;
  }
  rc = loop_build(lp, &E, &asym);
  if (rc != DONOF_OK) return rc;
  result->builds++;
  result->E = E;
  result->max_asym = asym;
  result->energies_recorded = nE;
  return DONOF_OK;
}
