// Hand-off to the orbital update (Sec. III.B): the symmetric matrix F of Eq. Fockian from the
// Lagrangian lambda and a given diagonal, its FP64 eigendecomposition, the rotated orbitals
// C V and their FP64 reorthonormalisation (one Newton-Schulz step C (3I - C^T C) / 2).
// The eigensolver is cuSOLVER's divide-and-conquer syevd (a plain library routine, as cuBLAS
// would be for a plain GEMM); everything else runs in this library's kernels.
#include <cusolverDn.h>

#include <map>
#include <mutex>

#include "common.cuh"

namespace donof {
namespace {

std::mutex g_sol_mu;
std::map<int, cusolverDnHandle_t> g_sol;

int solver(cusolverDnHandle_t* h) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DONOF_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_sol_mu);
  auto it = g_sol.find(dev);
  if (it == g_sol.end()) {
    cusolverDnHandle_t s = nullptr;
    if (cusolverDnCreate(&s) != CUSOLVER_STATUS_SUCCESS) return DONOF_ERR_CUDA;
    it = g_sol.emplace(dev, s).first;
  }
  *h = it->second;
  return DONOF_OK;
}

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
                const double* B, long long sBk, long long sBn, double* C) {
  DgemmArgs a{};
  a.M = M; a.N = N; a.K = K; a.KB = 1; a.batch = 1; a.ksplit = 1;
  a.A = A; a.sAm = sAm; a.sAk = sAk;
  a.B = B; a.sBk = sBk; a.sBn = sBn;
  a.C = C; a.sCm = N; a.sCn = 1;
  a.alpha = 1.0; a.beta = 0.0;
  return a;
}

}  // namespace
}  // namespace donof

using namespace donof;

extern "C" int donof_orbital_update_workspace_size(int32_t nbf, size_t* bytes) {
  if (nbf < 1 || !bytes) return DONOF_ERR_INVALID_ARG;
  cusolverDnHandle_t h = nullptr;
  int rc = solver(&h);
  if (rc != DONOF_OK) return rc;
  int lwork = 0;
  if (cusolverDnDsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, nbf,
                                  nullptr, nbf, nullptr, &lwork) != CUSOLVER_STATUS_SUCCESS)
    return DONOF_ERR_CUDA;
  const size_t nn = (size_t)nbf * nbf * 8;
  *bytes = 3 * align_up(nn) + align_up((size_t)lwork * 8) + kAlign;
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
  cusolverDnHandle_t h = nullptr;
  rc = solver(&h);
  if (rc != DONOF_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (cusolverDnSetStream(h, s) != CUSOLVER_STATUS_SUCCESS) return DONOF_ERR_CUDA;
  const int N = nbf;
  const size_t nn = align_up((size_t)N * N * 8);
  char* ws = (char*)workspace;
  double* F = (double*)ws;             // F, then its eigenvectors
  double* T = (double*)(ws + nn);      // C V
  double* S = (double*)(ws + 2 * nn);  // T^T T, then (3I - T^T T) / 2
  int* info = (int*)(ws + 3 * nn);
  double* work = (double*)(ws + 3 * nn + kAlign);
  int lwork = 0;
  if (cusolverDnDsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, N, F, N, eps,
                                  &lwork) != CUSOLVER_STATUS_SUCCESS)
    return DONOF_ERR_CUDA;

  prof_begin(DONOF_PHASE_ORBITAL_UPDATE, s);
  k_fockian<<<152 * 4, 256, 0, s>>>(lam, Fdiag, N, F);
  count_launch(1);
  if (cudaGetLastError() != cudaSuccess) return DONOF_ERR_CUDA;
  // F is symmetric, so its row-major storage is also its column-major storage; on return
  // column j of the column-major result (row j of the row-major view) is eigenvector j.
  if (cusolverDnDsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, N, F, N, eps, work,
                       lwork, info) != CUSOLVER_STATUS_SUCCESS)
    return DONOF_ERR_CUDA;
  // T[mu][j] = sum_i C[mu][i] V[i][j], V[i][j] = F[j * N + i]
  if (launch_dgemm(plain(N, N, N, C, N, 1, F, 1, N, T), s) != cudaSuccess) return DONOF_ERR_CUDA;
  // S = T^T T;  M = (3I - S) / 2;  C_new = T M
  if (launch_dgemm(plain(N, N, N, T, 1, N, T, N, 1, S), s) != cudaSuccess) return DONOF_ERR_CUDA;
  k_newton_schulz<<<152 * 4, 256, 0, s>>>(S, N, S);
  count_launch(1);
  if (cudaGetLastError() != cudaSuccess) return DONOF_ERR_CUDA;
  if (launch_dgemm(plain(N, N, N, T, N, 1, S, N, 1, C_new), s) != cudaSuccess)
    return DONOF_ERR_CUDA;
  prof_end(DONOF_PHASE_ORBITAL_UPDATE, s);
  return DONOF_OK;
}
