// The NOF-MP2 energy terms that need only the integrals of a build (Sec. "Dynamic
// Correlation", Eqs. Etotal, HFL, Esta): the HF-like energy of the natural orbitals and the
// static correlation energy, from H_pp, J_pq, K_pq, n, sqrt n and Phi left in the workspace
// by the last build.  E^dyn (Eq. E2) is not computed: its amplitudes come from modified MP2
// residual equations that the paper cites but does not state.
#include "common.cuh"

namespace donof {
namespace {

constexpr int kThreads = 256;

// Sum over the block in a fixed order: each thread's strided partial, then a fixed tree.
__device__ double block_sum_fixed(double v, double* red) {
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
  __syncthreads();
  return t;  // valid on thread 0
}

// One CTA.  E_hf: pairs (f, g) of the N_Omega strong orbitals, each H_gg and
// (2 J_fg - K_fg) weighted by the occupations of the HF density matrix of Eq. HFL (w = 1 for
// the strong orbital of a pair, 1/2 for a singly occupied one: 2n_g = 2 and 2n_g = 1), and
// the self-interaction J_gg / 4 of every singly occupied g removed; E_sta: pairs (p, q) of
// the active orbitals, the intra-pair term for p != q in one pair subspace (Pi_qp negative
// when exactly one of them is the strong orbital), the inter term for different subspaces.
__global__ void __launch_bounds__(kThreads) k_nofmp2_static(
    Dims d, const int32_t* __restrict__ pm, const double* __restrict__ n,
    const double* __restrict__ sqn, const double* __restrict__ phi, const double* __restrict__ Hd,
    const double* __restrict__ J, const double* __restrict__ K, double* E_hf, double* E_sta) {
  __shared__ double red[kThreads / 32];
  const int A = d.A, npair = d.npair, n_omega = d.npair + d.nsingle;
  double hf = 0.0;
  for (int i = threadIdx.x; i < n_omega * n_omega; i += kThreads) {
    const int f = i / n_omega, g = i % n_omega;
    const double wf = f < npair ? 1.0 : 0.5, wg = g < npair ? 1.0 : 0.5;
    hf += wf * wg * (2.0 * J[(size_t)f * A + g] - K[(size_t)f * A + g]);
    if (f == g) {
      hf += 2.0 * wg * Hd[g];
      if (g >= npair) hf -= J[(size_t)g * A + g] / 4.0;
    }
  }
  double sta = 0.0;
  for (int i = threadIdx.x; i < A * A; i += kThreads) {
    const int p = i / A, q = i % A;
    const int gp = pm[p], gq = pm[q];
    const double kpq = K[(size_t)p * A + q];
    if (gp != gq) {
      sta -= 4.0 * phi[q] * phi[q] * phi[p] * phi[p] * kpq;
    } else if (p != q && gp < npair) {
      const double lq = 1.0 - fabs(1.0 - 2.0 * n[q]), lp = 1.0 - fabs(1.0 - 2.0 * n[p]);
      const double pi = (p < npair || q < npair ? -1.0 : 1.0) * sqn[p] * sqn[q];
      sta += sqrt(lq * lp) * pi * kpq;
    }
  }
  hf = block_sum_fixed(hf, red);
  sta = block_sum_fixed(sta, red);
  if (threadIdx.x == 0) {
    *E_hf = hf;
    *E_sta = sta;
  }
}

}  // namespace
}  // namespace donof

using namespace donof;

extern "C" int donof_nofmp2_static(const donof_problem* prob, const int32_t* pair_map,
                                   const void* workspace, size_t workspace_bytes, double* E_hf,
                                   double* E_sta, void* stream) {
  if (!prob || !pair_map || !E_hf || !E_sta) return DONOF_ERR_INVALID_ARG;
  size_t need = 0;
  const int rc = donof_workspace_size(prob, &need);
  if (rc != DONOF_OK) return rc;
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace % kAlign) != 0)
    return DONOF_ERR_WORKSPACE;
  const Dims d = make_dims(prob);
  const Layout L = make_layout(d);
  const char* ws = (const char*)workspace;
  k_nofmp2_static<<<1, kThreads, 0, (cudaStream_t)stream>>>(
      d, pair_map, (const double*)(ws + L.n), (const double*)(ws + L.sqn),
      (const double*)(ws + L.phi), (const double*)(ws + L.Hd), (const double*)(ws + L.J),
      (const double*)(ws + L.K), E_hf, E_sta);
  count_launch(1);
  return cudaGetLastError() == cudaSuccess ? DONOF_OK : DONOF_ERR_CUDA;
}
