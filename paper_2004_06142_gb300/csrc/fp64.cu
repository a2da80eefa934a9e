// FP64 kernels of the PNOF build: the strided batched DGEMM that carries every
// contraction of the plain-double path (and the small double contractions of the
// mixed path), and the per-orbital / per-pair kernels of both paths:
//   occupations n(gamma) and Jacobians ........ Eqs. soo, woo
//   coefficient matrices of E in J and K ........ Eqs. Eg, Efg, Efg_s
//   J / K accumulation over P, the Y^P operands . Eqs. JKpq (density-fitted)
//   energy and dE/dgamma ........................ Eqs. EPNOF7, Eg, Efg, Efg_s
#include "common.cuh"
#include "occ.cuh"

namespace donof {

// ---------------------------------------------------------------------------
// Strided batched DGEMM, 64 x BN output tile per CTA (BN = 64, or 32 for narrow outputs
// whose width a 64 tile would pad by more), 4 x BN/16 per thread, DFMA.
// ---------------------------------------------------------------------------
namespace {
constexpr int DBM = 64, DBK = 16;

template <int BN>
__global__ void __launch_bounds__(256) k_dgemm(DgemmArgs a) {
  constexpr int NJ = BN / 16;
  __shared__ double As[DBK][DBM + 1];
  __shared__ double Bs[DBK][BN + 1];
  const int bz = blockIdx.z / a.ksplit, ks = blockIdx.z % a.ksplit;
  const long long m0 = (long long)blockIdx.x * DBM;
  const int n0 = blockIdx.y * BN;
  if (a.lower && n0 > m0 + DBM - 1) return;  // tile strictly above the diagonal
  const double* A = a.A + (long long)bz * a.sAb;
  const double* B = a.B + (long long)bz * a.sBb;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const bool a_m_fast = (a.sAm == 1);
  const bool b_n_fast = (a.sBn == 1);
  const int kb0 = (int)((long long)a.KB * ks / a.ksplit);
  const int kb1 = (int)((long long)a.KB * (ks + 1) / a.ksplit);
  double acc[4][NJ];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[i][j] = 0.0;

  for (int kb = kb0; kb < kb1; ++kb) {
    const double* Akb = A + (long long)kb * a.sAkb;
    const double* Bkb = B + (long long)kb * a.sBkb;
    for (int k0 = 0; k0 < a.K; k0 += DBK) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int idx = threadIdx.x + i * 256;
        int mm, kk;
        if (a_m_fast) { mm = idx % DBM; kk = idx / DBM; } else { kk = idx % DBK; mm = idx / DBK; }
        const long long gm = m0 + mm;
        const int gk = k0 + kk;
        const bool kin = gk < a.K && (a.Ktot <= 0 || kb * a.K + gk < a.Ktot);
        As[kk][mm] = (gm < a.M && kin) ? Akb[gm * a.sAm + (long long)gk * a.sAk] : 0.0;
      }
#pragma unroll
      for (int i = 0; i < NJ; ++i) {
        const int idx = threadIdx.x + i * 256;
        int nn, kk;
        if (b_n_fast) { nn = idx % BN; kk = idx / BN; } else { kk = idx % DBK; nn = idx / DBK; }
        const int gn = n0 + nn;
        const int gk = k0 + kk;
        const bool kin = gk < a.K && (a.Ktot <= 0 || kb * a.K + gk < a.Ktot);
        Bs[kk][nn] = (gn < a.N && kin) ? Bkb[(long long)gk * a.sBk + (long long)gn * a.sBn] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < DBK; ++kk) {
        double ra[4], rb[NJ];
#pragma unroll
        for (int i = 0; i < 4; ++i) ra[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < NJ; ++j) rb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < NJ; ++j) acc[i][j] = fma(ra[i], rb[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  double* C = a.C + (long long)bz * a.sCb;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long gm = m0 + ty + 16 * i;
    if (gm >= a.M) continue;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= a.N) continue;
      if (a.ksplit > 1) {
        a.part[((size_t)ks * a.M + gm) * a.N + gn] = a.alpha * acc[i][j];
      } else {
        double* c = C + gm * a.sCm + (long long)gn * a.sCn;
        *c = a.alpha * acc[i][j] + (a.beta != 0.0 ? a.beta * *c : 0.0);
      }
    }
  }
}

// C[m][n] += sum_ks part[ks][m][n], in order of ks
__global__ void k_splitk_reduce(const double* __restrict__ part, int ksplit, int M, int N,
                                double* C, long long sCm, long long sCn) {
  const long long tot = (long long)M * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int k = 0; k < ksplit; ++k) t += part[(size_t)k * tot + i];
    C[(i / N) * sCm + (i % N) * sCn] += t;
  }
}
}  // namespace

cudaError_t launch_dgemm(const DgemmArgs& a, cudaStream_t s) {
  if (a.M <= 0 || a.N <= 0 || a.batch <= 0) return cudaSuccess;
  if (a.ksplit > 1 && (!a.part || a.batch != 1 || a.beta != 1.0)) return cudaErrorInvalidValue;
  const long long mt = (a.M + DBM - 1) / DBM;
  // the narrow tile where it pads the output width less (e.g. 150 -> 160 instead of 192)
  const int bn = dgemm_tile_n(a.N);
  const bool narrow = bn == 32;
  dim3 grid((unsigned)mt, (unsigned)((a.N + bn - 1) / bn), (unsigned)(a.batch * a.ksplit));
  if (narrow)
    k_dgemm<32><<<grid, 256, 0, s>>>(a);
  else
    k_dgemm<64><<<grid, 256, 0, s>>>(a);
  count_launch(1);
  if (a.ksplit > 1) {
    const long long tot = (long long)a.M * a.N;
    const int nb = (int)((tot + 255) / 256 < 152 * 8 ? (tot + 255) / 256 : 152 * 8);
    k_splitk_reduce<<<nb, 256, 0, s>>>(a.part, a.ksplit, a.M, a.N, a.C, a.sCm, a.sCn);
    count_launch(1);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Occupations (Eqs. soo, woo) and their Jacobians with respect to gamma.
// One thread per active orbital; the Jacobians are zeroed by the caller and only their
// nonzero entries are written.  Also validates pair_map and gamma.
// ---------------------------------------------------------------------------
namespace {
// kTable (one CTA): sin and cos of every gamma are formed once into shared memory, so the
// FP64 trigonometry is not repeated per orbital (the narrow FP64 pipe makes it the cost).
template <bool kTable>
__device__ __forceinline__ void k_occupations_body(const Blk& B_, Dims d, const double* __restrict__ gamma,
                              const int32_t* __restrict__ pm, DevHeader* hdr, double* n,
                              double* sqn, double* phi, double* dn, double* dsq, double* dphi) {
  extern __shared__ double trig[];  // kTable: sin[ng], cos[ng]
  const int A = d.A, ng = d.ng, npair = d.npair, ncwo = d.ncwo;
  for (int k = threadIdx.x + B_.x * blockDim.x; k < ng; k += blockDim.x * B_.gx) {
    if (!isfinite(gamma[k])) set_status(hdr, DONOF_ERR_NONFINITE);
    if (kTable) {
      trig[k] = sin(gamma[k]);
      trig[ng + k] = cos(gamma[k]);
    }
  }
  if (kTable) __syncthreads();
  const int p = threadIdx.x + B_.x * blockDim.x;
  if (p >= A) return;
  const int nsub = npair + d.nsingle;  // subspaces: pairs, then the singly occupied orbitals
  const int g = pm[p];
  if (g < 0 || g >= nsub || (p < nsub && g != p) || (p >= nsub && g >= npair)) {
    set_status(hdr, DONOF_ERR_PAIR_MAP);
    return;
  }
  if (p >= npair && p < nsub) {  // Omega_I: n = 1/2, no gamma
    n[p] = 0.5;
    sqn[p] = 0.70710678118654752440;
    phi[p] = 0.5;
    return;
  }
  int rank = 0;
  if (p < npair) {
    int cnt = 0;
    for (int q = nsub; q < A; ++q) cnt += (pm[q] == p);
    if (cnt != ncwo) set_status(hdr, DONOF_ERR_PAIR_MAP);
  } else {
    // rank among the pair's weak orbitals
    for (int q = nsub; q < p; ++q) rank += (pm[q] == g);
    if (rank >= ncwo) {
      set_status(hdr, DONOF_ERR_PAIR_MAP);
      return;
    }
  }
  auto put = [&](int k, double dnk, double dsk, double dpk) {
    dn[(size_t)p * ng + k] = dnk;
    dsq[(size_t)p * ng + k] = dsk;
    dphi[(size_t)p * ng + k] = dpk;
  };
  if (kTable)
    occ_orbital(p, g, rank, npair, ncwo, TrigTable{trig, trig + ng}, n[p], sqn[p], phi[p], put);
  else
    occ_orbital(p, g, rank, npair, ncwo, TrigDirect{gamma}, n[p], sqn[p], phi[p], put);
}
template <bool kTable>
__global__ void k_occupations(Dims d, const double* __restrict__ gamma,
                              const int32_t* __restrict__ pm, DevHeader* hdr, double* n,
                              double* sqn, double* phi, double* dn, double* dsq, double* dphi) {
  k_occupations_body<kTable>(native_blk(), d, gamma, pm, hdr, n, sqn, phi, dn, dsq, dphi);
}
}  // namespace

cudaError_t launch_occupations(const Dims& d, const double* gamma, const int32_t* pm, char* ws,
                               const Layout& L, cudaStream_t s) {
  const size_t jac = (size_t)d.A * d.ng * sizeof(double);
  for (size_t off : {L.dn, L.dsq, L.dphi}) {
    const cudaError_t e = cudaMemsetAsync(ws + off, 0, jac, s);
    if (e != cudaSuccess) return e;
  }
  DevHeader* hdr = (DevHeader*)(ws + L.header);
  double *n = (double*)(ws + L.n), *sqn = (double*)(ws + L.sqn), *phi = (double*)(ws + L.phi);
  double *dn = (double*)(ws + L.dn), *dsq = (double*)(ws + L.dsq), *dphi = (double*)(ws + L.dphi);
  if (d.A <= 1024) {  // one CTA with the sin/cos table (at most 16 KB: ng < nact)
    const int threads = (d.A + 31) / 32 * 32;
    const size_t smem = (size_t)(d.ng > 0 ? d.ng : 1) * 2 * sizeof(double);
    k_occupations<true><<<1, threads, smem, s>>>(d, gamma, pm, hdr, n, sqn, phi, dn, dsq, dphi);
  } else {
    const int threads = 128;
    k_occupations<false><<<(d.A + threads - 1) / threads, threads, 0, s>>>(
        d, gamma, pm, hdr, n, sqn, phi, dn, dsq, dphi);
  }
  count_launch(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// E = 2 sum_p n_p H_pp + sum_pq (Acoef_pq J_pq + Bcoef_pq K_pq):
//   same subspace:      Acoef = 0,         Bcoef = Pi_pq               (Eqs. Eg, intra)
//   different subspace: Acoef = 2 n_p n_q, Bcoef = -n_p n_q - Phi_p Phi_q  (Eq. Efg)
//                                          -n_p n_q                    (PNOF5)
//                                          -n_p n_q - 4 Phi_p^2 Phi_q^2 (Eq. Efg_s)
// ---------------------------------------------------------------------------
namespace {
__device__ __forceinline__ void k_coefficients_body(const Blk& B_, Dims d, const int32_t* __restrict__ pm, const double* __restrict__ n,
                               const double* __restrict__ sqn, const double* __restrict__ phi,
                               double* Ac, double* Bc, float* AcF, float* BcF) {
  // with AcF/BcF (mixed path) also their fp32 copies, [Ap][Ap] with zero padding
  const int A = d.A, W = AcF ? d.Ap : d.A;
  const long long idx = (long long)B_.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)W * W) return;
  const int p = (int)(idx / W), q = (int)(idx % W);
  double a = 0.0, b = 0.0;
  if (p < A && q < A) {
    pair_coefficients(d.functional, d.npair, p, q, pm[p] == pm[q], pm[p] >= d.npair, n[p], n[q],
                      sqn[p], sqn[q], phi[p], phi[q], a, b);
    Ac[(size_t)p * A + q] = a;
    Bc[(size_t)p * A + q] = b;
  }
  if (AcF) {
    AcF[idx] = (float)a;
    BcF[idx] = (float)b;
  }
}
__global__ void k_coefficients(Dims d, const int32_t* __restrict__ pm, const double* __restrict__ n,
                               const double* __restrict__ sqn, const double* __restrict__ phi,
                               double* Ac, double* Bc, float* AcF, float* BcF) {
  k_coefficients_body(native_blk(), d, pm, n, sqn, phi, Ac, Bc, AcF, BcF);
}
}  // namespace

cudaError_t launch_coefficients(const Dims& d, const int32_t* pm, char* ws, const Layout& L,
                                cudaStream_t s) {
  const bool mixed = d.precision == DONOF_MIXED;
  const long long W = mixed ? d.Ap : d.A;
  k_coefficients<<<(unsigned)((W * W + 255) / 256), 256, 0, s>>>(
      d, pm, (const double*)(ws + L.n), (const double*)(ws + L.sqn), (const double*)(ws + L.phi),
      (double*)(ws + L.Acoef), (double*)(ws + L.Bcoef), mixed ? (float*)(ws + L.AcF) : nullptr,
      mixed ? (float*)(ws + L.BcF) : nullptr);
  count_launch(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Packed lower triangle -> dense symmetric slices (FP64 path, per block).
// ---------------------------------------------------------------------------
namespace {
__global__ void k_unpack(const double* __restrict__ Bp, long long np, int N, double* out) {
  const long long npk = (long long)N * (N + 1) / 2;
  const long long tot = np * N * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const long long P = i / ((long long)N * N);
    const int r = (int)((i / N) % N), c = (int)(i % N);
    const int hi = r > c ? r : c, lo = r > c ? c : r;
    out[i] = Bp[P * npk + (long long)hi * (hi + 1) / 2 + lo];
  }
}
}  // namespace

cudaError_t launch_unpack_B(const Dims& d, const double* Bp, int p0, int np, double* out,
                            cudaStream_t s) {
  const long long npk = (long long)d.N * (d.N + 1) / 2;
  k_unpack<<<152 * 8, 256, 0, s>>>(Bp + (long long)p0 * npk, np, d.N, out);
  count_launch(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// H_pp = C_p^T (h C)_p and G_p = n_p (h C)_p.
// ---------------------------------------------------------------------------
namespace {
// one warp per orbital p: H_pp over the lanes' rows mu, and G[mu][p] = n_p (h C)[mu][p]
__device__ __forceinline__ void k_hdiag_ginit_body(const Blk& B_, Dims d, const double* __restrict__ C, const double* __restrict__ hC,
                              const double* __restrict__ n, double* Hd, double* G, double gscale) {
  const int p = B_.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (p >= d.A) return;
  const double np_ = n[p];
  double s = 0.0;
  for (int mu = lane; mu < d.N; mu += 32) {
    const double v = hC[(size_t)mu * d.A + p];
    s += C[(size_t)mu * d.N + p] * v;
    G[(size_t)mu * d.A + p] = gscale * np_ * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) Hd[p] = s;
}
__global__ void k_hdiag_ginit(Dims d, const double* __restrict__ C, const double* __restrict__ hC,
                              const double* __restrict__ n, double* Hd, double* G, double gscale) {
  k_hdiag_ginit_body(native_blk(), d, C, hC, n, Hd, G, gscale);
}
}  // namespace

cudaError_t launch_hdiag_ginit(const Dims& d, const double* C, char* ws, const Layout& L,
                               bool one_electron_G, cudaStream_t s) {
  k_hdiag_ginit<<<(d.A + 7) / 8, 256, 0, s>>>(d, C, (const double*)(ws + L.hC),
                                              (const double*)(ws + L.n), (double*)(ws + L.Hd),
                                              (double*)(ws + L.G), one_electron_G ? 1.0 : 0.0);
  count_launch(1);
  return cudaGetLastError();
}

// y[i] += x[i] (double), i < n: the summed partial sums of a sharded build into the
// workspace's J, K and G.
namespace {
__global__ void k_add(double* __restrict__ y, const double* __restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] += x[i];
}
}  // namespace

cudaError_t launch_add(double* y, const double* x, long long n, cudaStream_t s) {
  const long long nb = (n + 255) / 256;
  k_add<<<(int)(nb < 152 * 8 ? (nb > 0 ? nb : 1) : 152 * 8), 256, 0, s>>>(y, x, n);
  count_launch(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// J_pq += sum_P b[P][p][p] b[P][q][q],  K_pq += sum_P b[P][p][q]^2  (double sums, a thread
// per (p, q) over the block's slices in order, so the sums do not depend on scheduling).
// ---------------------------------------------------------------------------
namespace {
__global__ void k_jk(Dims d, const double* __restrict__ b, int np, int ld, double* J,
                     double* K) {
  const int A = d.A;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)A * A) return;
  const int p = (int)(idx / A), q = (int)(idx % A);
  double sj = 0.0, sk = 0.0;
#pragma unroll 4
  for (int P = 0; P < np; ++P) {
    const double* bp = b + (size_t)P * ld * ld;
    const double dp = bp[(size_t)p * ld + p], dq = bp[(size_t)q * ld + q];
    const double v = bp[(size_t)p * ld + q];
    sj = fma(dp, dq, sj);
    sk = fma(v, v, sk);
  }
  J[idx] += sj;
  K[idx] += sk;
}
}  // namespace

cudaError_t launch_jk_accumulate_f64(const Dims& d, const double* b, int np, int ld, char* ws,
                                     const Layout& L, cudaStream_t s) {
  const long long tot = (long long)d.A * d.A;
  k_jk<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d, b, np, ld, (double*)(ws + L.J),
                                                     (double*)(ws + L.K));
  count_launch(1);
  return cudaGetLastError();
}
// ---------------------------------------------------------------------------
// Y^P[q][p] = Bcoef_qp b^P_qp + delta_qp w^P_p,  w^P_p = sum_r Acoef_pr b^P_rr.
// G_p = n_p (hC)_p + sum_P X^P Y^P  is then (1/4) dE/dC (Eqs. lowdin, Vee-s, Vee-d).
// One CTA per auxiliary slice; ld = leading dimension of b and Y (A or Ap), padding
// entries (q or p >= A) are written as zero.
// ---------------------------------------------------------------------------
namespace {
__global__ void k_build_Y(Dims d, const double* __restrict__ b, double* Y, int np, int ld,
                          const double* __restrict__ Ac, const double* __restrict__ Bc) {
  extern __shared__ double sh[];  // d[ld], w[ld]
  double* dv = sh;
  double* wv = sh + ld;
  const int A = d.A;
  for (int P = blockIdx.x; P < np; P += gridDim.x) {
    const double* bp = b + (size_t)P * ld * ld;
    double* yp = Y + (size_t)P * ld * ld;
    for (int r = threadIdx.x; r < A; r += blockDim.x) dv[r] = bp[(size_t)r * ld + r];
    __syncthreads();
    for (int p = threadIdx.x; p < A; p += blockDim.x) {
      double w = 0.0;
      for (int r = 0; r < A; ++r) w = fma(Ac[(size_t)p * A + r], dv[r], w);
      wv[p] = w;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ld * ld; i += blockDim.x) {
      const int q = i / ld, p = i % ld;
      double v = 0.0;
      if (q < A && p < A) {
        v = Bc[(size_t)q * A + p] * bp[i];
        if (q == p) v += wv[p];
      }
      yp[i] = v;
    }
    __syncthreads();
  }
}
}  // namespace

cudaError_t launch_build_Y_f64(const Dims& d, const double* b, double* Y, int np, char* ws,
                               const Layout& L, cudaStream_t s) {
  const int grid = np < 152 * 4 ? np : 152 * 4;
  k_build_Y<<<grid, 256, 2 * d.A * sizeof(double), s>>>(
      d, b, Y, np, d.A, (const double*)(ws + L.Acoef), (const double*)(ws + L.Bcoef));
  count_launch(1);
  return cudaGetLastError();
}
// ---------------------------------------------------------------------------
// Energy and occupation gradient (double throughout).
//   dE/dn_p     = 2 H_pp + 2 sum_{q not in g(p)} n_q (2 J_pq - K_pq)
//                 [PNOF7s: - 8 (1 - 2 n_p) sum_{q not in g(p)} Phi_q^2 K_pq]
//   dE/dsqrt_np = 2 sum_{q in g(p)} s_pq sqrt(n_q) K_pq   (s_pq the sign of Pi_pq)
//   dE/dPhi_p   = -2 sum_{q not in g(p)} Phi_q K_pq       [PNOF7]
//   dE/dgamma_k = sum_p (dE/dn_p dn_p/dgamma_k + dE/dsqrt_np dsqrt_np/dgamma_k
//                        + dE/dPhi_p dPhi_p/dgamma_k)
// k_energy_rows: one warp per orbital p (its share of E and the three partials);
// k_energy_final: E as a fixed-order sum of the shares, then dE/dgamma (a warp per output).
// ---------------------------------------------------------------------------
namespace {
__device__ __forceinline__ void k_energy_rows_body(const Blk& B_, Dims d, const int32_t* __restrict__ pm, const double* __restrict__ n,
                              const double* __restrict__ sqn, const double* __restrict__ phi,
                              const double* __restrict__ Ac, const double* __restrict__ Bc,
                              const double* __restrict__ Hd, const double* __restrict__ J,
                              const double* __restrict__ K, double* part) {
  const int A = d.A;
  const int p = B_.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (p >= A) return;
  const int g = pm[p];
  double e = 0.0, a_n = 0.0, a_s = 0.0, a_p = 0.0, a_7s = 0.0;
  for (int q = lane; q < A; q += 32) {
    const size_t o = (size_t)p * A + q;
    const double kpq = K[o], jpq = J[o];
    e += Ac[o] * jpq + Bc[o] * kpq;
    if (pm[q] == g) {
      if (g < d.npair) {  // a singly occupied orbital has no intra-subspace term
        const bool plus = (p == q || (p >= d.npair && q >= d.npair));
        a_s += (plus ? 2.0 : -2.0) * sqn[q] * kpq;
      }
    } else {
      a_n += 2.0 * n[q] * (2.0 * jpq - kpq);
      a_p -= 2.0 * phi[q] * kpq;
      a_7s += phi[q] * phi[q] * kpq;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    a_n += __shfl_xor_sync(0xffffffffu, a_n, o);
    a_s += __shfl_xor_sync(0xffffffffu, a_s, o);
    a_p += __shfl_xor_sync(0xffffffffu, a_p, o);
    a_7s += __shfl_xor_sync(0xffffffffu, a_7s, o);
  }
  if (lane == 0) {
    a_n += 2.0 * Hd[p];
    if (d.functional == DONOF_PNOF7S) a_n -= 8.0 * (1.0 - 2.0 * n[p]) * a_7s;
    part[p] = e + 2.0 * n[p] * Hd[p];
    part[A + p] = a_n;
    part[2 * A + p] = a_s;
    part[3 * A + p] = (d.functional == DONOF_PNOF7) ? a_p : 0.0;
  }
}
__global__ void k_energy_rows(Dims d, const int32_t* __restrict__ pm, const double* __restrict__ n,
                              const double* __restrict__ sqn, const double* __restrict__ phi,
                              const double* __restrict__ Ac, const double* __restrict__ Bc,
                              const double* __restrict__ Hd, const double* __restrict__ J,
                              const double* __restrict__ K, double* part) {
  k_energy_rows_body(native_blk(), d, pm, n, sqn, phi, Ac, Bc, Hd, J, K, part);
}

__device__ __forceinline__ void k_energy_final_body(const Blk& B_, Dims d, const double* __restrict__ part,
                                                       const double* __restrict__ dn,
                                                       const double* __restrict__ dsq,
                                                       const double* __restrict__ dphi,
                                                       DevHeader* hdr, double* dEdg_ws,
                                                       double* E_out, double* dEdg_out) {
  // one warp per output (E first, then each dE/dgamma_k), lanes over orbitals, a fixed
  // shuffle tree: the sums do not depend on scheduling
  const int A = d.A;
  const int lane = threadIdx.x % 32, nw = B_.gx * (blockDim.x / 32);
  const int warp = B_.x * (blockDim.x / 32) + threadIdx.x / 32;
  const double* gn = part + A;
  const double* gs = part + 2 * A;
  const double* gp = part + 3 * A;
  for (int k = warp - 1; k < d.ng; k += nw) {
    double t = 0.0;
    if (k < 0) {
      for (int p = lane; p < A; p += 32) t += part[p];
    } else {
      for (int p = lane; p < A; p += 32) {
        const size_t o = (size_t)p * d.ng + k;
        t += gn[p] * dn[o] + gs[p] * dsq[o] + gp[p] * dphi[o];
      }
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) {
      if (k < 0) {
        hdr->E = t;
        if (E_out) *E_out = t;
        if (!isfinite(t)) set_status(hdr, DONOF_ERR_NONFINITE);
      } else {
        dEdg_ws[k] = t;
        if (dEdg_out) dEdg_out[k] = t;
      }
    }
  }
}
__global__ void __launch_bounds__(256) k_energy_final(Dims d, const double* __restrict__ part,
                                                       const double* __restrict__ dn,
                                                       const double* __restrict__ dsq,
                                                       const double* __restrict__ dphi,
                                                       DevHeader* hdr, double* dEdg_ws,
                                                       double* E_out, double* dEdg_out) {
  k_energy_final_body(native_blk(), d, part, dn, dsq, dphi, hdr, dEdg_ws, E_out, dEdg_out);
}
}  // namespace

cudaError_t launch_energy(const Dims& d, const int32_t* pm, char* ws, const Layout& L,
                          double* E_out, double* dEdg_out, cudaStream_t s) {
  double* part = (double*)(ws + L.Epart);
  k_energy_rows<<<(d.A + 7) / 8, 256, 0, s>>>(
      d, pm, (const double*)(ws + L.n), (const double*)(ws + L.sqn), (const double*)(ws + L.phi),
      (const double*)(ws + L.Acoef), (const double*)(ws + L.Bcoef), (const double*)(ws + L.Hd),
      (const double*)(ws + L.J), (const double*)(ws + L.K), part);
  k_energy_final<<<(d.ng + 1 + 7) / 8, 256, 0, s>>>(d, part, (const double*)(ws + L.dn),
                                   (const double*)(ws + L.dsq), (const double*)(ws + L.dphi),
                                   (DevHeader*)(ws + L.header), (double*)(ws + L.dEdg), E_out,
                                   dEdg_out);
  count_launch(2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
namespace {
__device__ __forceinline__ void k_backward_body(const Blk& B_, Dims d, const double* __restrict__ Ebar, const double* __restrict__ G,
                           const double* __restrict__ dEdg, double* dE_dC, double* dE_dgamma) {
  const double eb = *Ebar;
  const long long tot = (long long)d.N * d.N;
  for (long long i = B_.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)B_.gx * blockDim.x) {
    const int p = (int)(i % d.N);
    const long long mu = i / d.N;
    if (dE_dC) dE_dC[i] = (p < d.A) ? 4.0 * eb * G[mu * d.A + p] : 0.0;
    if (dE_dgamma && i < d.ng) dE_dgamma[i] = eb * dEdg[i];
  }
}
__global__ void k_backward(Dims d, const double* __restrict__ Ebar, const double* __restrict__ G,
                           const double* __restrict__ dEdg, double* dE_dC, double* dE_dgamma) {
  k_backward_body(native_blk(), d, Ebar, G, dEdg, dE_dC, dE_dgamma);
}
}  // namespace

cudaError_t launch_backward(const Dims& d, const double* Ebar, const char* ws, const Layout& L,
                            double* dE_dC, double* dE_dgamma, cudaStream_t s) {
  k_backward<<<152 * 4, 256, 0, s>>>(d, Ebar, (const double*)(ws + L.G),
                                     (const double*)(ws + L.dEdg), dE_dC, dE_dgamma);
  count_launch(1);
  return cudaGetLastError();
}

}  // namespace donof

// ---------------------------------------------------------------------------
// Grouped launches of the kernels above (one launch for every instance of a batch; the
// per-instance grids are those of the launchers above, laid out by the GroupLaunch).
// ---------------------------------------------------------------------------
namespace donof {
namespace {
__global__ void k_occupations_group(const GroupLaunch g) {
  Blk b;
  const InstRec& I = g.inst[group_locate(g, b)];
  char* ws = I.ws;
  const Layout& L = I.L;
  k_occupations_body<true>(b, I.d, I.gamma, I.pm, (DevHeader*)(ws + L.header),
                           (double*)(ws + L.n), (double*)(ws + L.sqn), (double*)(ws + L.phi),
                           (double*)(ws + L.dn), (double*)(ws + L.dsq), (double*)(ws + L.dphi));
}
__global__ void k_coefficients_group(const GroupLaunch g) {
  Blk b;
  const InstRec& I = g.inst[group_locate(g, b)];
  char* ws = I.ws;
  const Layout& L = I.L;
  k_coefficients_body(b, I.d, I.pm, (const double*)(ws + L.n), (const double*)(ws + L.sqn),
                      (const double*)(ws + L.phi), (double*)(ws + L.Acoef),
                      (double*)(ws + L.Bcoef), (float*)(ws + L.AcF), (float*)(ws + L.BcF));
}
__global__ void k_hdiag_ginit_group(const GroupLaunch g) {
  Blk b;
  const InstRec& I = g.inst[group_locate(g, b)];
  char* ws = I.ws;
  const Layout& L = I.L;
  k_hdiag_ginit_body(b, I.d, I.C, (const double*)(ws + L.hC), (const double*)(ws + L.n),
                     (double*)(ws + L.Hd), (double*)(ws + L.G), 1.0);
}
__global__ void k_energy_rows_group(const GroupLaunch g) {
  Blk b;
  const InstRec& I = g.inst[group_locate(g, b)];
  char* ws = I.ws;
  const Layout& L = I.L;
  k_energy_rows_body(b, I.d, I.pm, (const double*)(ws + L.n), (const double*)(ws + L.sqn),
                     (const double*)(ws + L.phi), (const double*)(ws + L.Acoef),
                     (const double*)(ws + L.Bcoef), (const double*)(ws + L.Hd),
                     (const double*)(ws + L.J), (const double*)(ws + L.K),
                     (double*)(ws + L.Epart));
}
__global__ void __launch_bounds__(256) k_energy_final_group(const GroupLaunch g) {
  Blk b;
  const InstRec& I = g.inst[group_locate(g, b)];
  char* ws = I.ws;
  const Layout& L = I.L;
  k_energy_final_body(b, I.d, (const double*)(ws + L.Epart), (const double*)(ws + L.dn),
                      (const double*)(ws + L.dsq), (const double*)(ws + L.dphi),
                      (DevHeader*)(ws + L.header), (double*)(ws + L.dEdg), I.E, I.dEdg);
}
__global__ void k_backward_group(const GroupLaunch g) {
  Blk b;
  const InstRec& I = g.inst[group_locate(g, b)];
  k_backward_body(b, I.d, I.Ebar, (const double*)(I.ws + I.L.G),
                  (const double*)(I.ws + I.L.dEdg), I.dEdC, nullptr);
}
// Zero what a build accumulates into or writes only in part: the abort flag, the occupation
// Jacobians, the Gram bound, J, K and lambda.  blockIdx.y of the instance's grid: the range.
__global__ void k_zero_group(const GroupLaunch g) {
  Blk b;
  const InstRec& I = g.inst[group_locate(g, b)];
  const Dims& d = I.d;
  const Layout& L = I.L;
  DevHeader* hdr = (DevHeader*)(I.ws + L.header);
  const size_t jac = (size_t)d.A * (d.ng > 0 ? d.ng : 0) * 8, aa = (size_t)d.A * d.A * 8;
  // the instance's ranges, each strided over all of its threads
  void* const p[8] = {&hdr->abort_flag, I.ws + L.dn, I.ws + L.dsq, I.ws + L.dphi, &hdr->sC2,
                      I.ws + L.J, I.ws + L.K, I.lam};
  const size_t bytes[8] = {4, jac, jac, jac, 8, aa, aa, I.lam ? (size_t)d.N * d.N * 8 : 0};
  const size_t t0 = (size_t)b.x * blockDim.x + threadIdx.x, nt = (size_t)b.gx * blockDim.x;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    uint32_t* w = (uint32_t*)p[r];
    for (size_t i = t0; i < bytes[r] / 4; i += nt) w[i] = 0u;
  }
}
}  // namespace

cudaError_t launch_fp64_group(int kind, const GroupLaunch& g, int blocks, int threads,
                              size_t smem, cudaStream_t s) {
  switch (kind) {
    case GK_ZERO: k_zero_group<<<blocks, threads, 0, s>>>(g); break;
    case GK_OCC: k_occupations_group<<<blocks, threads, smem, s>>>(g); break;
    case GK_COEF: k_coefficients_group<<<blocks, threads, 0, s>>>(g); break;
    case GK_HDIAG: k_hdiag_ginit_group<<<blocks, threads, 0, s>>>(g); break;
    case GK_EROWS: k_energy_rows_group<<<blocks, threads, 0, s>>>(g); break;
    case GK_EFINAL: k_energy_final_group<<<blocks, threads, 0, s>>>(g); break;
    case GK_BWD: k_backward_group<<<blocks, threads, 0, s>>>(g); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch(1);
  return cudaGetLastError();
}
}  // namespace donof
