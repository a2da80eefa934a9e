// Symmetric FP64 eigensolver of the orbital update (Sec. III.B: the new orbitals are the
// eigenvectors of the symmetric matrix F of Eq. Fockian, and its eigenvalues the next
// diagonal).  Laid out for this GPU's narrow FP64 pipe and large L2:
//   1. A = Q T Q^T by Householder reflections in one cooperative launch (one CTA per SM, one
//      grid barrier per column).  Each step forms the next column of the rank-2-updated
//      matrix in every CTA (from one row, by symmetry) and its reflector; every row warp
//      updates its own row of the trailing matrix and takes its part of the next
//      matrix-vector product while a scalar warp forms the reflector's scalars; the matrix
//      stays in L2.  A is first scaled by a power of two (exact) to a largest element in
//      [1/2, 1).
//   2. T is split where an off-diagonal element is at most 16 N eps ||T||_inf (a perturbation
//      of that size moves no eigenvalue by more) and scaled by a power of two to
//      ||T||_inf <= 1; eigenvalues of each block by multisection on Sturm counts, a half-warp
//      per eigenvalue: float rounds, then double rounds from the three-term recurrence of the
//      leading minors with exact power-of-two rescaling.
//   3. Eigenvectors of T from twisted factorisations T - lambda I = N_r D_r N_r^T, two threads
//      per eigenvalue, the twist r where |gamma_r| is smallest; eigenvalues of one block closer
//      than 1e-5 ||T||_inf form clusters: each member's own inverse iteration (all members at
//      once), then a block orthonormalisation inside the cluster (one warp for small
//      clusters, panels on the GEMM kernel for large ones).
//   4. V = Q Z by the compact WY form of blocks of 64 reflectors: the blocks' triangular
//      factors from their Gram matrices, and two FP64 GEMMs per block.
#include <float.h>

#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace donof {
namespace {

constexpr int kRowWarps = 8;                  // warps of a tridiagonal-reduction CTA that own rows
constexpr int kTriWarps = kRowWarps + 1;      // ... and the scalar warp
constexpr int kTriThreads = 32 * kTriWarps;
constexpr int kScalarTid = 32 * kRowWarps;    // lane 0 of the scalar warp
static_assert(kTriWarps <= 16, "block_sum_d sums at most 16 warps");
constexpr int kNb = 64;           // reflectors per WY block
constexpr int kFixCTAs = 32;      // CTAs (one warp each) of the small-cluster kernel
constexpr int kSmallCl = 32;      // clusters up to this size are orthonormalised by one warp
constexpr int kClDesc = 5;        // ints per cluster: first slot, members, block start, block
                                  // length, offset of its vectors in the scratch (large ones)
constexpr int kApplyCols = 8;     // columns of W1 per CTA in the triangular-factor product
// tridiagonal reduction: vector elements per thread held in registers, and the largest n whose
// trailing rows (one per warp) stay in registers, kTriRowRegs elements per lane
constexpr int kTriVec = 5;  // (kTriRegMaxN + kTriThreads - 1) / kTriThreads
constexpr int kTriRegMaxN = 1216;
constexpr int kTriRowRegs = (kTriRegMaxN - 2 + 31) / 32;
constexpr double kClusterTol = 1e-5;
constexpr unsigned long long kBarrierLimitNs = 2000000000ull;

struct EighHdr {
  unsigned int ctr;   // grid-barrier arrivals of the tridiagonal reduction
  int abort;          // set when a barrier wait ran out
  int ncl;            // clusters found
  int maxcl;          // members of the largest cluster
  int nonfinite;      // A holds a NaN or an infinity
  int pad;
  unsigned long long amax_bits;  // max |A_ij| (bit pattern of a non-negative double)
  double scale;       // the power of two applied to A
  double tscale;      // the power of two applied to T: ||T||_inf * tscale in [1/2, 1)
  double tnorm;       // ||T||_inf after that scaling
  double pivmin;      // pivot floor of the twisted factorisations (scaled units)
};

struct EighLayout {
  size_t hdr, A, Yr, Wd, Wp, d, e, ds, es, e2, df, e2f, tau, pbuf, lam, glo, ghi, col, bstart,
      bend, incl, cl, cj, T, G, W1, W2, part, total;
  int nref, nblk;
};

EighLayout eigh_layout(int N) {
  EighLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + (bytes ? bytes : 1));
    return o;
  };
  const size_t n = (size_t)N, nn = n * n;
  L.nref = N > 2 ? N - 2 : 0;
  L.nblk = (L.nref + kNb - 1) / kNb;
  L.hdr = take(sizeof(EighHdr));
  L.A = take(nn * 8);
  L.Yr = take(nn * 8);
  L.Wd = take(nn * 8);
  L.Wp = take(nn * 8);
  L.d = take(n * 8);
  L.e = take(n * 8);
  L.ds = take(n * 8);
  L.es = take(n * 8);
  L.e2 = take(n * 8);
  L.df = take(n * 4);
  L.e2f = take(n * 4);
  L.tau = take(n * 8);
  L.pbuf = take(2 * n * 8);
  L.lam = take(n * 8);
  L.glo = take(n * 8);
  L.ghi = take(n * 8);
  L.col = take(n * 4);
  L.bstart = take(n * 4);
  L.bend = take(n * 4);
  L.incl = take(n * 4);
  L.cl = take((size_t)kClDesc * n * 4);
  L.cj = take(n * 4);
  L.T = take((size_t)L.nblk * kNb * kNb * 8);
  L.G = take((size_t)L.nblk * kNb * kNb * 8);
  L.W1 = take((size_t)kNb * n * 8);
  L.W2 = take((size_t)kNb * n * 8);
  size_t ks = 1;
  for (int b = 0; b < L.nblk; ++b) {
    const int m = L.nref - b * kNb < kNb ? L.nref - b * kNb : kNb;
    const size_t k = (size_t)splitk_count(m, N, N - 1 - b * kNb);
    if (k > ks) ks = k;
  }
  size_t part = ks > 1 ? ks * kNb * n : 0;
  // the large clusters' panel products: (r0 x 32) and (32 x 32) with contraction length <= N
  for (int r0 = 32; r0 < N; r0 += 32) {
    const size_t k = (size_t)splitk_count(r0, 32, N);
    if (k > 1 && k * r0 * 32 > part) part = k * r0 * 32;
  }
  {
    const size_t k = (size_t)splitk_count(32, 32, N);
    if (k > 1 && k * 32 * 32 > part) part = k * 32 * 32;
  }
  L.part = take(part * 8);
  L.total = off;
  return L;
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA in a fixed order (a fixed shuffle tree in each warp, then warp 0 adds the
// warps' sums by a fixed tree): every thread gets the same value.  red holds kTriWarps + 1.
__device__ __forceinline__ double block_sum_d(double v, double* red) {
  v = warp_sum_d(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < kTriWarps ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 8; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[kTriWarps] = t;
  }
  __syncthreads();
  return red[kTriWarps];
}

// Grid barrier of the cooperative launch: arrivals counted in hdr->ctr (zeroed before the
// launch); the wait gives up after kBarrierLimitNs and raises hdr->abort, which ends every
// other CTA's wait at once.  Returns false when the CTA must leave.
__device__ __forceinline__ bool grid_barrier(EighHdr* h, unsigned target, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&h->ctr, 1u);
    const unsigned long long t0 = gtimer();
    int ok = 1;
    while (*(volatile unsigned*)&h->ctr < target) {
      if (*(volatile int*)&h->abort) { ok = 0; break; }
      if (gtimer() - t0 > kBarrierLimitNs) {
        atomicExch(&h->abort, 1);
        ok = 0;
        break;
      }
    }
    __threadfence();
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// ---------------------------------------------------------------------------
// 0. max |A| (and a non-finite check), then the scaled copy
// ---------------------------------------------------------------------------
__global__ void k_eigh_amax(const double* __restrict__ A, long long nn, EighHdr* h) {
  __shared__ unsigned long long red[8];
  unsigned long long m = 0;
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn;
       i += (long long)gridDim.x * blockDim.x) {
    const double a = fabs(A[i]);
    if (!isfinite(a)) bad = 1;
    else m = max(m, (unsigned long long)__double_as_longlong(a));
  }
  for (int o = 16; o; o >>= 1) {
    m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  if ((threadIdx.x & 31) == 0 && bad) h->nonfinite = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = max(m, red[i]);
    atomicMax(&h->amax_bits, m);
  }
}

__device__ __forceinline__ double eigh_scale(const EighHdr* h) {
  const double amax = __longlong_as_double((long long)h->amax_bits);
  if (amax == 0.0 || h->nonfinite) return 1.0;
  int ex = 0;
  frexp(amax, &ex);  // amax = f 2^ex, f in [1/2, 1)
  return ldexp(1.0, -ex);
}

__global__ void k_eigh_scale_copy(const double* __restrict__ A, long long nn, EighHdr* h,
                                  double* __restrict__ out) {
  const double s = eigh_scale(h);
  if (blockIdx.x == 0 && threadIdx.x == 0) h->scale = s;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = A[i] * s;
}

// ---------------------------------------------------------------------------
// 1. Householder tridiagonalisation (cooperative launch, kTriThreads threads, one CTA per SM)
// ---------------------------------------------------------------------------
struct TriArgs {
  int N;
  double* A;     // N x N, row-major, symmetric; trailing rows updated in place
  double* Yr;    // reflector k in row k, columns k+1 .. N-1 (zero elsewhere)
  double* d;     // diagonal of T
  double* e;     // off-diagonal of T (N - 1)
  double* tau;   // tau of reflector k
  double* pbuf;  // two N-vectors: p of the current and the next step
  EighHdr* hdr;
};

__global__ void __launch_bounds__(kTriThreads, 1) k_tridiag(TriArgs a) {
  extern __shared__ double sm[];
  __shared__ double red[kTriWarps + 1];
  __shared__ double sh[3];
  __shared__ int s_flag;
  const int N = a.N, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int G = gridDim.x;
  double* v = sm;           // reflector of the current step (indices k+1 .. N-1)
  double* x = sm + N;       // next column, then its reflector
  double* p = sm + 2 * N;   // p = tau A v of the current step
  double* A = a.A;
  const bool writer = blockIdx.x == 0;
  if (N <= 2) {
    if (writer && tid == 0) {
      a.d[0] = __ldcg(A);
      if (N == 2) {
        a.e[0] = __ldcg(A + 1);
        a.d[1] = __ldcg(A + 3);
      }
    }
    return;
  }
  // rows are dealt to CTAs cyclically (row i to CTA i mod G), then to the CTA's row warps, so
  // the shrinking trailing matrix stays spread over every SM; with N <= G * kRowWarps each row
  // warp owns one row at most and keeps it in registers while it is updated.  The last warp
  // owns no row: its lane 0 forms the reflectors' scalars.
  const bool row_warp = wid < kRowWarps;
  auto row_of = [&](int t) { return blockIdx.x + G * (wid + kRowWarps * t); };
  const bool reg_rows = N <= kTriRegMaxN && N <= G * kRowWarps;
  const int myrow = row_warp ? row_of(0) : N;
  unsigned bar = 0;

  // reflector of x[k0..N) (xn2 = sum over j > k0 of x_j^2): the scalars tau, beta and the
  // scale of u's tail (0 when the column is already reduced: u = e_k0)
  auto hh_scalars = [&](int k0, double xn2) {
    if (tid == kScalarTid) {
      const double al = x[k0];
      double t = 0.0, b = al, sc = 0.0;
      if (xn2 != 0.0) {
        b = -copysign(sqrt(fma(al, al, xn2)), al);
        t = (b - al) / b;
        sc = 1.0 / (al - b);
      }
      sh[0] = t;
      sh[1] = b;
      sh[2] = sc;
    }
  };
  // after a barrier: x[k0+1..) scaled into u's tail, x[k0] = 1; CTA 0 also stores u as row
  // `refl` of Yr
  auto hh_apply = [&](int k0, int refl) {
    const double sc = sh[2];
    double* Yk = a.Yr + (size_t)refl * N;
    for (int j = k0 + tid; j < N; j += kTriThreads) {
      const double u = j == k0 ? 1.0 : x[j] * sc;
      x[j] = u;
      if (writer) Yk[j] = u;
    }
  };

  // reflector 0 from row 0 (column 0)
  double xn = 0.0;
  for (int j = tid; j < N; j += kTriThreads) {
    const double xj = __ldcg(A + j);
    x[j] = xj;
    if (j >= 2) xn = fma(xj, xj, xn);
  }
  hh_scalars(1, block_sum_d(xn, red));
  __syncthreads();
  double tau_c = sh[0], beta = sh[1];
  if (writer && tid == 0) {
    a.d[0] = x[0];
    a.e[0] = beta;
    a.tau[0] = tau_c;
  }
  hh_apply(1, 0);
  __syncthreads();
  if (row_warp) {
    for (int t = 0;; ++t) {
      const int i = row_of(t);
      if (i >= N) break;
      if (i < 1) continue;
      const double* Ar = A + (size_t)i * N;
      double acc = 0.0;
#pragma unroll 4
      for (int j = 1 + lane; j < N; j += 32) acc = fma(__ldcg(Ar + j), x[j], acc);
      acc = warp_sum_d(acc);
      if (lane == 0) a.pbuf[i] = tau_c * acc;
    }
  }
  if (!grid_barrier(a.hdr, (++bar) * G, &s_flag)) return;
  {
    double* t = v;
    v = x;
    x = t;
  }

  for (int k = 0; k <= N - 3; ++k) {
    const double* pk = a.pbuf + (size_t)(k & 1) * N;
    const double* Ak1 = A + (size_t)(k + 1) * N;
    const bool last = k + 1 == N - 2;
    // every load of the step at once: p_k, row k+1, and (register path) the warp's own row
    double pr[kTriVec], ar[kTriVec];
#pragma unroll
    for (int r = 0; r < kTriVec; ++r) {
      const int j = k + 1 + tid + kTriThreads * r;
      pr[r] = 0.0;
      ar[r] = 0.0;
      if (j < N) {
        pr[r] = __ldcg(pk + j);
        ar[r] = __ldcg(Ak1 + j);
      }
    }
    double rr[kTriRowRegs];
    const bool has_row = reg_rows && myrow < N && myrow >= k + 2;
    double* Amy = A + (size_t)(has_row ? myrow : 0) * N;
    if (has_row) {
#pragma unroll
      for (int q = 0; q < kTriRowRegs; ++q) {
        const int j = k + 2 + lane + 32 * q;
        rr[q] = j < N ? __ldcg(Amy + j) : 0.0;
      }
    }
    double acc = 0.0;
#pragma unroll
    for (int r = 0; r < kTriVec; ++r) {
      const int j = k + 1 + tid + kTriThreads * r;
      if (j < N) acc = fma(pr[r], v[j], acc);
    }
    for (int j = k + 1 + tid + kTriThreads * kTriVec; j < N; j += kTriThreads)
      acc = fma(__ldcg(pk + j), v[j], acc);
    // alpha = (tau_k / 2)(p_k . v_k); with w = p - alpha v the update A - v w^T - w v^T is
    // A_ij - v_i p_j - (p_i - 2 alpha v_i) v_j, formed from p and v alone
    const double al = 0.5 * tau_c * block_sum_d(acc, red);
#pragma unroll
    for (int r = 0; r < kTriVec; ++r) {
      const int j = k + 1 + tid + kTriThreads * r;
      if (j < N) p[j] = pr[r];
    }
    for (int j = k + 1 + tid + kTriThreads * kTriVec; j < N; j += kTriThreads)
      p[j] = __ldcg(pk + j);
    __syncthreads();
    // row k+1 of the updated matrix (v[k+1] = 1): its column k+1 below the diagonal
    const double ck1 = fma(-2.0, al, p[k + 1]);
    xn = 0.0;
#pragma unroll
    for (int r = 0; r < kTriVec; ++r) {
      const int j = k + 1 + tid + kTriThreads * r;
      if (j < N) {
        const double xj = fma(-ck1, v[j], ar[r] - pr[r]);
        x[j] = xj;
        if (j >= k + 3) xn = fma(xj, xj, xn);
      }
    }
    for (int j = k + 1 + tid + kTriThreads * kTriVec; j < N; j += kTriThreads) {
      const double xj = fma(-ck1, v[j], __ldcg(Ak1 + j) - p[j]);
      x[j] = xj;
      if (j >= k + 3) xn = fma(xj, xj, xn);
    }
    // register path: the own row's rank-2 update, while the norm is reduced (not at the last
    // step, whose 2 x 2 block is formed from the rows as they stand)
    if (has_row && !last) {
      const double vi = v[myrow], ci = fma(-2.0 * al, vi, p[myrow]);
#pragma unroll
      for (int q = 0; q < kTriRowRegs; ++q) {
        const int j = k + 2 + lane + 32 * q;
        if (j < N) {
          rr[q] = fma(-ci, v[j], fma(-vi, p[j], rr[q]));
          Amy[j] = rr[q];
        }
      }
    }
    const double xn2 = block_sum_d(xn, red);
    if (last) {  // the last 2 x 2 block
      if (writer && tid == 0) {
        a.d[N - 2] = x[N - 2];
        a.e[N - 2] = x[N - 1];
        const double vl = v[N - 1], cl = fma(-2.0 * al, vl, p[N - 1]);
        a.d[N - 1] = __ldcg(A + (size_t)(N - 1) * N + N - 1) - vl * p[N - 1] - cl * vl;
      }
      break;
    }
    // the scalar warp forms the next reflector while the row warps take the dot of their
    // updated row with the unscaled column (u_{k+2} = 1, u_j = sc x_j beyond)
    hh_scalars(k + 2, xn2);
    double rawdot = 0.0, r0 = 0.0;
    if (has_row) {
#pragma unroll
      for (int q = 0; q < kTriRowRegs; ++q) {
        const int j = k + 2 + lane + 32 * q;
        if (j < N) {
          if (q == 0 && lane == 0) r0 = rr[0];
          else rawdot = fma(rr[q], x[j], rawdot);
        }
      }
      rawdot = warp_sum_d(rawdot);
    }
    __syncthreads();
    const double tau_n = sh[0], sc = sh[2];
    beta = sh[1];
    if (writer && tid == 0) {
      a.d[k + 1] = x[k + 1];
      a.e[k + 1] = beta;
      a.tau[k + 1] = tau_n;
    }
    hh_apply(k + 2, k + 1);
    // p_{k+1} = tau A u over the own rows i >= k+2
    double* pn = a.pbuf + (size_t)((k + 1) & 1) * N;
    if (reg_rows) {
      if (has_row && lane == 0) pn[myrow] = tau_n * fma(sc, rawdot, r0);
    } else {
      __syncthreads();  // the scaled reflector
      for (int t = 0; row_warp; ++t) {
        const int i = row_of(t);
        if (i >= N) break;
        if (i < k + 2) continue;
        double* Ar = A + (size_t)i * N;
        const double vi = v[i], ci = fma(-2.0 * al, vi, p[i]);
        double acc2 = 0.0;
        int j = k + 2 + lane;
        for (; j + 96 < N; j += 128) {
          const double a0 = __ldcg(Ar + j), a1 = __ldcg(Ar + j + 32), a2 = __ldcg(Ar + j + 64),
                       a3 = __ldcg(Ar + j + 96);
          const double b0 = fma(-ci, v[j], fma(-vi, p[j], a0));
          const double b1 = fma(-ci, v[j + 32], fma(-vi, p[j + 32], a1));
          const double b2 = fma(-ci, v[j + 64], fma(-vi, p[j + 64], a2));
          const double b3 = fma(-ci, v[j + 96], fma(-vi, p[j + 96], a3));
          Ar[j] = b0;
          Ar[j + 32] = b1;
          Ar[j + 64] = b2;
          Ar[j + 96] = b3;
          acc2 = fma(b0, x[j], acc2);
          acc2 = fma(b1, x[j + 32], acc2);
          acc2 = fma(b2, x[j + 64], acc2);
          acc2 = fma(b3, x[j + 96], acc2);
        }
        for (; j < N; j += 32) {
          const double b0 = fma(-ci, v[j], fma(-vi, p[j], __ldcg(Ar + j)));
          Ar[j] = b0;
          acc2 = fma(b0, x[j], acc2);
        }
        acc2 = warp_sum_d(acc2);
        if (lane == 0) pn[i] = tau_n * acc2;
      }
    }
    if (!grid_barrier(a.hdr, (++bar) * G, &s_flag)) return;
    double* t = v;
    v = x;
    x = t;
    tau_c = tau_n;
  }
}

// ---------------------------------------------------------------------------
// 2. splitting, Gershgorin bounds, bisection.  From here on T is scaled by the power of two
//    ts = 2^-ceil(log2 ||T||_inf), so that ||T||_inf <= 1 (exact), and every kernel reads the
//    scaled arrays.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool dbl_is_zero(double x) {
  return ((unsigned long long)__double_as_longlong(x) << 1) == 0ull;
}
__device__ __forceinline__ int dbl_biased_exp(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }
__device__ __forceinline__ int dbl_sign(double x) { return (int)((unsigned)__double2hiint(x) >> 31); }

// One CTA.  ||T||_inf and the scale ts; the split off-diagonal (es, es^2) and the diagonal
// scaled by ts (double and float copies); the blocks (bstart/bend of every row, found by one
// thread from integer flags); each block's Gershgorin interval (at its first row, one warp
// per block); the twisted factorisations' pivot floor.
__global__ void __launch_bounds__(256) k_tri_prep(int N, const double* __restrict__ d,
                                                  const double* __restrict__ e, EighHdr* h,
                                                  double* ds, double* es, double* e2, float* df,
                                                  float* e2f, int* bstart, int* bend,
                                                  double* glo, double* ghi) {
  extern __shared__ int sflag[];  // [N]: row i ends a block; then the list of block starts
  int* blist = sflag + N;
  __shared__ double red[8];
  __shared__ int s_nb;
  double tn = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double r = fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < N - 1 ? fabs(e[i]) : 0.0);
    tn = fmax(tn, r);
  }
  for (int o = 16; o; o >>= 1) tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tn;
  __syncthreads();
  tn = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tn = fmax(tn, red[i]);
  if (!(tn > 0.0) || !isfinite(tn)) tn = 1.0;  // T = 0 (or not finite: NaN eigenvalues follow)
  int ex = 0;
  frexp(tn, &ex);  // tn = f 2^ex, f in [1/2, 1)
  const double ts = ldexp(1.0, -ex);
  const double thresh = 16.0 * N * DBL_EPSILON * tn;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double di = d[i] * ts;
    ds[i] = di;
    df[i] = (float)di;
    int end = i == N - 1 ? 1 : 0;
    if (i < N - 1) {
      const double ei = fabs(e[i]) <= thresh ? 0.0 : e[i] * ts;
      es[i] = ei;
      e2[i] = ei * ei;
      e2f[i] = (float)(ei * ei);
      end = dbl_is_zero(ei) ? 1 : end;
    }
    sflag[i] = end;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    h->tnorm = tn * ts;
    h->tscale = ts;
    h->pivmin = 0x1p-100;
    int s0 = 0, nb = 0;
    for (int i = 0; i < N; ++i) {
      if (sflag[i]) {
        for (int r = s0; r <= i; ++r) {
          bstart[r] = s0;
          bend[r] = i + 1;
        }
        blist[nb++] = s0;
        s0 = i + 1;
      }
    }
    s_nb = nb;
  }
  __syncthreads();
  const int nb = s_nb, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int b = threadIdx.x >> 5; b < nb; b += nw) {
    const int s0 = blist[b], s1 = b + 1 < nb ? blist[b + 1] : N;
    if (s1 - s0 < 2) continue;  // a 1 x 1 block needs no bisection
    double lo = 0.0, hi = 0.0;
    bool any = false;
    for (int i = s0 + lane; i < s1; i += 32) {
      const double el = i > s0 ? fabs(es[i - 1]) : 0.0;
      const double er = i < s1 - 1 ? fabs(es[i]) : 0.0;
      const double l = ds[i] - el - er, u = ds[i] + el + er;
      lo = any ? fmin(lo, l) : l;
      hi = any ? fmax(hi, u) : u;
      any = true;
    }
    if (!any) {  // lanes beyond the block: neutral values
      lo = ds[s0];
      hi = ds[s0];
    }
    for (int o = 16; o; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      glo[s0] = lo;
      ghi[s0] = hi;
    }
  }
}

// Number of eigenvalues of the (scaled) block [s0, s1) below sig in float: the ratio form
// q_i = (d_i - sig) - e_{i-1}^2 / q_{i-1}, |q_i| floored at piv (a zero pivot counts negative).
__device__ __forceinline__ int sturm_count_f32(const float* __restrict__ d,
                                               const float* __restrict__ e2, int s0, int s1,
                                               float sig) {
  constexpr float piv = 1e-30f;
  float q = d[s0] - sig;
  if (fabsf(q) < piv) q = -piv;
  int cnt = q < 0.0f ? 1 : 0;
  for (int i = s0 + 1; i < s1; ++i) {
    q = (d[i] - sig) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < piv) q = -piv;
    cnt += q < 0.0f ? 1 : 0;
  }
  return cnt;
}

// The same count in double: sign changes of the leading minors
// p_i = (d_i - sig) p_{i-1} - e_{i-1}^2 p_{i-2} (a zero minor counts as a tiny negative ratio),
// the pair (p_{i-1}, p_i) rescaled by 2^-+300 after every eighth row when its larger magnitude
// has left [2^-300, 2^300] (with ||T||_inf <= 1 and the split threshold, eight rows move it by
// at most 2^13 up or 2^-616 down).
__device__ __forceinline__ int sturm_count_f64(const double* __restrict__ d,
                                               const double* __restrict__ e2, int s0, int s1,
                                               double sig) {
  double p0 = 1.0, p1 = d[s0] - sig;
  if (dbl_is_zero(p1)) p1 = -0x1p-60;
  int cnt = dbl_sign(p1);
  int i = s0 + 1;
  while (i < s1) {
    const int iend = min(i + 8, s1);
#pragma unroll 4
    for (; i < iend; ++i) {
      double p2 = fma(d[i] - sig, p1, -(e2[i - 1] * p0));
      if (dbl_is_zero(p2)) p2 = -p1 * 0x1p-60;
      cnt += dbl_sign(p2) ^ dbl_sign(p1);
      p0 = p1;
      p1 = p2;
    }
    const int ex = max(dbl_biased_exp(p0), dbl_biased_exp(p1));
    if (ex > 1023 + 300) {
      p0 *= 0x1p-300;
      p1 *= 0x1p-300;
    } else if (ex < 1023 - 300) {
      p0 *= 0x1p300;
      p1 *= 0x1p300;
    }
  }
  return cnt;
}

// Eigenvalue k = s - bstart[s] of the block holding row s, by multisection: a half-warp per
// eigenvalue, its 16 lanes counting at 16 points of the bracket per round.  Five float rounds
// (brackets of ~2^-20 ||T||), the bracket widened by 4e-6 ||T|| (the float counts are exact
// for a matrix within a few float roundings of T) and its ends checked by double counts (the
// Gershgorin interval again if either fails), then double rounds to the width eps ||T||.
constexpr int kBisThreads = 128;
__global__ void __launch_bounds__(kBisThreads) k_bisect(int N, const double* __restrict__ ds,
                                                        const double* __restrict__ e2,
                                                        const float* __restrict__ df,
                                                        const float* __restrict__ e2f,
                                                        const int* __restrict__ bstart,
                                                        const int* __restrict__ bend,
                                                        const double* __restrict__ glo,
                                                        const double* __restrict__ ghi,
                                                        const EighHdr* h, double* lam) {
  extern __shared__ double sb[];
  double* sd = sb;
  double* se2 = sb + N;
  float* sdf = (float*)(sb + 2 * N);
  float* se2f = sdf + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    sd[i] = ds[i];
    sdf[i] = df[i];
    se2[i] = i < N - 1 ? e2[i] : 0.0;
    se2f[i] = i < N - 1 ? e2f[i] : 0.0f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, j = lane & 15;
  const unsigned hm = 0xffffu << (lane & 16);
  const int s = (blockIdx.x * kBisThreads + threadIdx.x) >> 4;
  if (s >= N) return;  // uniform over the half-warp
  if (h->abort) {
    if (j == 0) lam[s] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  const int s0 = bstart[s], s1 = bend[s], k = s - s0;
  if (s1 - s0 == 1) {
    if (j == 0) lam[s] = sd[s0];
    return;
  }
  const double tn = h->tnorm;
  const double pad = 2.0 * N * DBL_EPSILON * tn;
  const double glo_s = glo[s0] - pad, ghi_s = ghi[s0] + pad;
  double lo = glo_s, hi = ghi_s;
  // narrow [lo, hi] to the points of the lanes: jh the first lane whose count exceeds k, jl
  // the last lane before it whose count does not
  auto narrow = [&](bool above, double base, double step, int off) {
    const unsigned ab = (__ballot_sync(hm, above) >> (lane & 16)) & 0xffffu;
    const unsigned be = (__ballot_sync(hm, !above) >> (lane & 16)) & 0xffffu;
    const int jh = ab ? __ffs(ab) - 1 : 16;
    const unsigned bl = be & ((1u << jh) - 1u);
    const int jl = bl ? 31 - __clz(bl) : -1;
    const double nhi = jh < 16 ? base + (jh + off) * step : hi;
    const double nlo = jl >= 0 ? base + (jl + off) * step : lo;
    hi = nhi;
    lo = nlo;
  };
  for (int r = 0; r < 5; ++r) {
    const double step = (hi - lo) * (1.0 / 17.0);
    const double sg = lo + (j + 1) * step;
    narrow(sturm_count_f32(sdf, se2f, s0, s1, (float)sg) > k, lo, step, 1);
  }
  lo -= 4e-6 * tn;
  hi += 4e-6 * tn;
  {  // 16 points from lo to hi inclusive: the ends verify the float bracket
    const double step = (hi - lo) * (1.0 / 15.0);
    const double sg = lo + j * step;
    const int c = sturm_count_f64(sd, se2, s0, s1, sg);
    const int clo = __shfl_sync(hm, c, lane & 16), chi = __shfl_sync(hm, c, (lane & 16) + 15);
    if (clo <= k && chi > k) {
      narrow(c > k, lo, step, 0);
    } else {
      lo = glo_s;
      hi = ghi_s;
    }
  }
  for (int r = 0; r < 40; ++r) {
    if (!(hi - lo > fmax(DBL_EPSILON * tn, 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi))))) break;
    const double step = (hi - lo) * (1.0 / 17.0);
    const double sg = lo + (j + 1) * step;
    narrow(sturm_count_f64(sd, se2, s0, s1, sg) > k, lo, step, 1);
  }
  if (j == 0) lam[s] = 0.5 * (lo + hi);
}

// Order-preserving integer key of a double (NaN above everything).
__device__ __forceinline__ long long dbl_key(double x) {
  const long long u = __double_as_longlong(x);
  return u >= 0 ? u : (u ^ 0x7fffffffffffffffll);
}

// Rank of every eigenvalue (integer keys, ties by slot), eigenvalues of A in ascending order;
// CTA 0 also lists the clusters: runs of a block's consecutive eigenvalues closer than
// kClusterTol ||T|| (the gaps tested in parallel, the runs found by one thread).
__global__ void __launch_bounds__(256) k_rank_plan(int N, const double* __restrict__ lam,
                                                   const int* __restrict__ bend, EighHdr* h,
                                                   int* col, double* w_out, int* incl, int* cl,
                                                   int* cj, const int* __restrict__ bstart) {
  extern __shared__ long long skey[];
  int* sgap = (int*)(skey + N);
  for (int i = threadIdx.x; i < N; i += blockDim.x) skey[i] = dbl_key(lam[i]);
  __syncthreads();
  const double unscale = 1.0 / (h->tscale * h->scale);  // a power of two
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < N) {
    const long long ks = skey[s];
    int r = 0;
    for (int t = 0; t < N; ++t) {
      const long long kt = skey[t];
      r += (kt < ks || (kt == ks && t < s)) ? 1 : 0;
    }
    const double ls = lam[s];
    if (ls != ls) r = s;  // NaN (a failed reduction): its own slot
    col[s] = r;
    w_out[r] = ls * unscale;
  }
  if (blockIdx.x != 0) return;
  const double tol = kClusterTol * h->tnorm;
  for (int i = threadIdx.x; i < N; i += blockDim.x)
    sgap[i] = (i + 1 < bend[i] && lam[i + 1] - lam[i] < tol) ? 1 : 0;
  __syncthreads();
  if (threadIdx.x != 0) return;
  int ncl = 0, maxcl = 0, off = 0;
  for (int s0 = 0; s0 < N;) {
    int t = s0;
    while (sgap[t]) ++t;  // sgap[bend - 1] = 0 ends every run inside its block
    const int m = t - s0 + 1;
    for (int u = s0; u <= t; ++u) {
      incl[u] = m > 1 ? ncl + 1 : 0;  // cluster id + 1
      cj[u] = u - s0;                 // member index
    }
    if (m > 1) {
      const int a0 = bstart[s0], L = bend[s0] - a0;
      int* c = cl + kClDesc * ncl;
      c[0] = s0;
      c[1] = m;
      c[2] = a0;
      c[3] = L;
      c[4] = off;
      if (m > kSmallCl) off += m * L;  // large clusters keep their vectors in the scratch
      maxcl = max(maxcl, m);
      ++ncl;
    }
    s0 = t + 1;
  }
  h->ncl = ncl;
  h->maxcl = maxcl;
}

// ---------------------------------------------------------------------------
// 3. eigenvectors of T
// ---------------------------------------------------------------------------
// 1/x to double precision by Newton's iteration r <- r (2 - x r) from a float seed (the error
// squares each step: 2^-23, 2^-46, then rounding); 2^-126 < |x| < 2^126.
__device__ __forceinline__ double rcp_nr(double x) {
  double r = (double)__frcp_rn((float)x);
  double t = fma(-x, r, 1.0);
  r = fma(r, t, r);
  t = fma(-x, r, 1.0);
  return fma(r, t, r);
}
// a pivot of magnitude below 2^-100 (||T|| <= 1) becomes -2^-100
__device__ __forceinline__ double pivot_floor(double v) {
  return dbl_biased_exp(v) < 1023 - 100 ? -0x1p-100 : v;
}

// Twisted factorisation of T_b - lambda I for an eigenvalue outside the clusters, two threads
// per eigenvalue.  Thread 0 of the pair runs the forward pivots D+_i (stored in Z's column,
// their reciprocals in Wp), thread 1 the backward pivots D-_i (reciprocals in Wd); then
// gamma_i = D+_i - e_i^2 / D-_{i+1} (each thread half the rows), the twist r where |gamma_r|
// is smallest (first such row), z_r = 1, and thread 0 forms z_i = -e_i z_{i+1} / D+_i above r
// while thread 1 forms z_i = -e_{i-1} z_{i-1} / D-_i below it; normalised to unit length.
// Z[i][col] (row-major, column = rank of the eigenvalue), zero outside the block.
__global__ void __launch_bounds__(32) k_twisted(int N, const double* __restrict__ ds,
                                                const double* __restrict__ es,
                                                const double* __restrict__ e2,
                                                const int* __restrict__ bstart,
                                                const int* __restrict__ bend,
                                                const double* __restrict__ lam,
                                                const int* __restrict__ col,
                                                const int* __restrict__ incl, double* Z,
                                                double* Wp, double* Wd) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = t >> 1, side = t & 1, lane = threadIdx.x;
  const unsigned pm = 3u << (lane & ~1);
  if (s >= N) return;  // uniform over the pair
  const int s0 = bstart[s], s1 = bend[s], c = col[s];
  const size_t ld = (size_t)N;
  if (s1 - s0 == 1) {
    if (side == 0) Z[s0 * ld + c] = 1.0;
    return;
  }
  if (incl[s]) return;
  const double lm = lam[s];
  if (side == 0) {
    double dp = pivot_floor(ds[s0] - lm), rp = rcp_nr(dp);
    Z[s0 * ld + c] = dp;
    Wp[s0 * ld + c] = rp;
    for (int i = s0 + 1; i < s1; ++i) {
      dp = pivot_floor(fma(-e2[i - 1], rp, ds[i] - lm));
      rp = rcp_nr(dp);
      Z[i * ld + c] = dp;
      Wp[i * ld + c] = rp;
    }
  } else {
    double dm = pivot_floor(ds[s1 - 1] - lm), rm = rcp_nr(dm);
    Wd[(s1 - 1) * ld + c] = rm;
    for (int i = s1 - 2; i >= s0; --i) {
      dm = pivot_floor(fma(-e2[i], rm, ds[i] - lm));
      rm = rcp_nr(dm);
      Wd[i * ld + c] = rm;
    }
  }
  __syncwarp(pm);
  // twist: thread 0 the rows [s0, mid), thread 1 [mid, s1)
  const int mid = (s0 + s1) >> 1;
  const int a = side == 0 ? s0 : mid, b = side == 0 ? mid : s1;
  double best = 0.0;
  int r = -1;
  for (int i = a; i < b; ++i) {
    const double g = i < s1 - 1 ? fabs(fma(-e2[i], Wd[(i + 1) * ld + c], Z[i * ld + c]))
                                : fabs(Z[i * ld + c]);
    if (r < 0 || g < best) {
      best = g;
      r = i;
    }
  }
  {
    const double ob = __shfl_xor_sync(pm, best, 1);
    const int orr = __shfl_xor_sync(pm, r, 1);
    // the lower rows win ties; an empty half (r < 0) never wins
    const bool take_other = orr >= 0 && (r < 0 || ob < best || (ob == best && orr < r));
    if (take_other) {
      best = ob;
      r = orr;
    }
  }
  __syncwarp(pm);
  // z: thread 0 upwards from r, thread 1 downwards; rescaled by 2^-500 when above 2^500
  int nres = 0;
  if (side == 0) {
    Z[r * ld + c] = 1.0;
    double z = 1.0;
    for (int i = r - 1; i >= s0; --i) {
      z = -es[i] * z * Wp[i * ld + c];
      if (fabs(z) > 0x1p500) {
        for (int u = i + 1; u <= r; ++u) Z[u * ld + c] *= 0x1p-500;
        z *= 0x1p-500;
        ++nres;
      }
      Z[i * ld + c] = z;
    }
  } else {
    double z = 1.0;
    for (int i = r + 1; i < s1; ++i) {
      z = -es[i - 1] * z * Wd[i * ld + c];
      if (fabs(z) > 0x1p500) {
        for (int u = r + 1; u < i; ++u) Z[u * ld + c] *= 0x1p-500;
        z *= 0x1p-500;
        ++nres;
      }
      Z[i * ld + c] = z;
    }
  }
  __syncwarp(pm);
  // bring both halves to the same scale, then normalise
  const int lo_i = side == 0 ? s0 : r + 1, hi_i = side == 0 ? r + 1 : s1;
  const int other = __shfl_xor_sync(pm, nres, 1);
  for (int q = nres; q < other; ++q)
    for (int i = lo_i; i < hi_i; ++i) Z[i * ld + c] *= 0x1p-500;
  double n2 = 0.0;
  for (int i = lo_i; i < hi_i; ++i) {
    const double zi = Z[i * ld + c];
    n2 = fma(zi, zi, n2);
  }
  n2 += __shfl_xor_sync(pm, n2, 1);
  const double sc = 1.0 / sqrt(n2);
  for (int i = lo_i; i < hi_i; ++i) Z[i * ld + c] *= sc;
}

__device__ __forceinline__ double hash_uniform(unsigned long long key) {
  // splitmix64 (Steele, Lea and Flood, 2014), mapped to [-1, 1)
  unsigned long long z = key + 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1p-52 - 1.0;
}

// Clusters.  Every member first gets two steps of inverse iteration of its own, all members at
// once (a thread each): (T_b - lambda I) = L D L^T without pivoting (pivots floored at 2^-100
// as in the twisted factorisations), from a pseudo-random start, normalised after each step.
// The vectors of a small cluster go to Z's columns and are orthonormalised by one warp (modified
// Gram-Schmidt, twice); those of a large cluster go to rows of a scratch matrix and are
// orthonormalised in panels of 32 (block classical Gram-Schmidt and a Cholesky QR of the
// panel, each twice) on the GEMM kernel, then scattered to Z.  With shifts accurate to eps ||T||
// a member's vector is its eigenvector up to (eps / gap)^2 of its neighbours, so the
// orthonormalisation only mixes members whose eigenvalues are equal at working precision.
__global__ void __launch_bounds__(32) k_cluster_vectors(
    int N, const double* __restrict__ ds, const double* __restrict__ es,
    const int* __restrict__ bstart, const int* __restrict__ bend, const double* __restrict__ lam,
    const int* __restrict__ col, const int* __restrict__ incl, const int* __restrict__ cj,
    const int* __restrict__ cl, double* Z, double* Yc, double* Wrp, double* Wl) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N || incl[t] == 0) return;
  const int* c = cl + kClDesc * (incl[t] - 1);
  const int a0 = bstart[t], L = bend[t] - a0, j = cj[t];
  const size_t ld = (size_t)N;
  const bool large = c[1] > kSmallCl;
  double* y = large ? Yc + (size_t)c[4] + (size_t)j * L : Z + (size_t)a0 * ld + col[t];
  const size_t ys = large ? 1 : ld;
  double* rp = Wrp + (size_t)t * ld;  // reciprocal pivots
  double* lm_ = Wl + (size_t)t * ld;  // multipliers
  const double lm = lam[t];
  double r = rcp_nr(pivot_floor(ds[a0] - lm));
  rp[0] = r;
  for (int i = 0; i + 1 < L; ++i) {
    const double li = es[a0 + i] * r;
    lm_[i] = li;
    r = rcp_nr(pivot_floor(fma(-li, es[a0 + i], ds[a0 + i + 1] - lm)));
    rp[i + 1] = r;
  }
  for (int i = 0; i < L; ++i)
    y[i * ys] = hash_uniform(((unsigned long long)t << 32) + (unsigned long long)i);
  for (int it = 0; it < 2; ++it) {
    // L u = x (in place), w = D^-1 u, L^T y = w
    double u = y[0];
    for (int i = 1; i < L; ++i) {
      u = fma(-lm_[i - 1], u, y[i * ys]);
      y[i * ys] = u;
    }
    double yy = y[(L - 1) * ys] * rp[L - 1];
    y[(L - 1) * ys] = yy;
    double amax = fabs(yy);
    for (int i = L - 2; i >= 0; --i) {
      yy = fma(-lm_[i], yy, y[i * ys] * rp[i]);
      y[i * ys] = yy;
      amax = fmax(amax, fabs(yy));
    }
    const double sa = amax > 0.0 && isfinite(amax) ? 1.0 / amax : 1.0;
    double n2 = 0.0;
    for (int i = 0; i < L; ++i) {
      const double v = y[i * ys] * sa;
      n2 = fma(v, v, n2);
    }
    const double sc = sa / sqrt(n2);
    for (int i = 0; i < L; ++i) y[i * ys] *= sc;
  }
}

// Small clusters (at most kSmallCl members): modified Gram-Schmidt over the members in order,
// twice, on Z's columns; one warp per cluster.
__global__ void __launch_bounds__(32) k_cluster_small(int N, const int* __restrict__ col,
                                                      const int* __restrict__ cl,
                                                      const EighHdr* h, double* Z) {
  const int ncl = h->ncl, lane = threadIdx.x;
  const size_t ld = (size_t)N;
  for (int q = blockIdx.x; q < ncl; q += gridDim.x) {
    const int* c = cl + kClDesc * q;
    const int s = c[0], m = c[1], a0 = c[2], L = c[3];
    if (m > kSmallCl) continue;
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = 0; j < m; ++j) {
        double* zj = Z + (size_t)a0 * ld + col[s + j];
        for (int jj = 0; jj < j; ++jj) {
          const double* zk = Z + (size_t)a0 * ld + col[s + jj];
          double dot = 0.0;
          for (int i = lane; i < L; i += 32) dot = fma(zk[i * ld], zj[i * ld], dot);
          dot = __shfl_sync(0xffffffffu, warp_sum_d(dot), 0);
          for (int i = lane; i < L; i += 32) zj[i * ld] = fma(-dot, zk[i * ld], zj[i * ld]);
          __syncwarp();
        }
        double n2 = 0.0;
        for (int i = lane; i < L; i += 32) n2 = fma(zj[i * ld], zj[i * ld], n2);
        n2 = __shfl_sync(0xffffffffu, warp_sum_d(n2), 0);
        const double sc = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
        for (int i = lane; i < L; i += 32) zj[i * ld] *= sc;
        __syncwarp();
      }
    }
  }
}

// A panel of b <= 32 rows of length L (row-major, leading dimension L): the Cholesky factor
// R^T R of its Gram matrix G (b x b, formed by the GEMM), computed by every CTA, then each
// CTA's columns replaced by R^-T times them (the panel's rows become orthonormal).  A pivot
// that is not positive (a dependent row) is raised to 1e-300 of the diagonal.
__global__ void __launch_bounds__(128) k_chol_apply(int b, int L, const double* __restrict__ G,
                                                    double* P) {
  __shared__ double R[32][33];
  const int tid = threadIdx.x;
  for (int i = tid; i < b * b; i += blockDim.x) R[i / b][i % b] = G[i];
  __syncthreads();
  for (int k = 0; k < b; ++k) {  // right-looking Cholesky, R upper triangular in place
    if (tid == 0) {
      double d = R[k][k];
      if (!(d > 1e-300 * fabs(G[k * b + k]))) d = fmax(1e-300 * fabs(G[k * b + k]), 1e-300);
      R[k][k] = sqrt(d);
    }
    __syncthreads();
    const double rk = R[k][k];
    for (int jj = k + 1 + tid; jj < b; jj += blockDim.x) R[k][jj] /= rk;
    __syncthreads();
    for (int idx = tid; idx < b * b; idx += blockDim.x) {
      const int i = idx / b, jj = idx % b;
      if (i > k && jj >= i) R[i][jj] = fma(-R[k][i], R[k][jj], R[i][jj]);
    }
    __syncthreads();
  }
  const int cidx = blockIdx.x * blockDim.x + tid;
  if (cidx >= L) return;
  double y[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) y[i] = i < b ? P[(size_t)i * L + cidx] : 0.0;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    if (i < b) {
      double v = y[i];
#pragma unroll
      for (int k = 0; k < i; ++k) v = fma(-R[k][i], y[k], v);
      y[i] = v / R[i][i];
    }
  }
#pragma unroll
  for (int i = 0; i < 32; ++i)
    if (i < b) P[(size_t)i * L + cidx] = y[i];
}

// The rows of a large cluster's scratch into Z's columns.
__global__ void k_cluster_scatter(int N, int s, int m, int a0, int L,
                                  const double* __restrict__ Y, const int* __restrict__ col,
                                  double* Z) {
  const long long tot = (long long)m * L;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / L), r = (int)(i % L);
    Z[(size_t)(a0 + r) * N + col[s + j]] = Y[i];
  }
}

// ---------------------------------------------------------------------------
// 4. back-transformation V = Q Z, Q = H_0 ... H_{nref-1} in blocks of kNb reflectors
// ---------------------------------------------------------------------------
// Gram matrices G_b = Y_b^T Y_b of every block (entries c <= c' only), Y_b's column c the
// reflector k0 + c: grid (nblk, kNb / 16, kNb / 16) of 16 x 16 sub-tiles, upper ones only.
__global__ void __launch_bounds__(256) k_gram(int N, int nref, const double* __restrict__ Yr,
                                              double* G) {
  const int b = blockIdx.x, tr = blockIdx.y, tc = blockIdx.z;
  if (tr > tc) return;
  __shared__ double Ys[2][16][65];
  const int k0 = b * kNb;
  const int m = nref - k0 < kNb ? nref - k0 : kNb;
  const int r = threadIdx.x / 16, c = threadIdx.x % 16;
  const int gr = tr * 16 + r, gc = tc * 16 + c;
  double acc = 0.0;
  for (int j0 = k0 + 1; j0 < N; j0 += 64) {
    for (int idx = threadIdx.x; idx < 2 * 16 * 64; idx += 256) {
      const int which = idx / 1024, rr = (idx / 64) % 16, jj = idx % 64;
      const int refl = (which == 0 ? tr : tc) * 16 + rr;
      const int j = j0 + jj;
      Ys[which][rr][jj] = (refl < m && j < N) ? Yr[(size_t)(k0 + refl) * N + j] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int jj = 0; jj < 64; ++jj) acc += Ys[0][r][jj] * Ys[1][c][jj];
    __syncthreads();
  }
  G[(size_t)b * kNb * kNb + gr * kNb + gc] = acc;
}

// Triangular factors T_b (upper): T_ii = tau_i, T[r][i] = -tau_i sum_{c=r}^{i-1} T[r][c] G[c][i]
// (r < i); thread r forms row r.
__global__ void k_tfactor(int nref, const double* __restrict__ tau, const double* __restrict__ G,
                          double* T) {
  const int b = blockIdx.x, r = threadIdx.x;
  const int k0 = b * kNb;
  const int m = nref - k0 < kNb ? nref - k0 : kNb;
  const double* Gb = G + (size_t)b * kNb * kNb;
  double* Tb = T + (size_t)b * kNb * kNb + (size_t)r * kNb;
  for (int i = 0; i < kNb; ++i) {
    double v = 0.0;
    if (r < m && i < m) {
      if (r == i) {
        v = tau[k0 + i];
      } else if (r < i) {
        double acc = 0.0;
        for (int c = r; c < i; ++c) acc += Tb[c] * Gb[c * kNb + i];
        v = -tau[k0 + i] * acc;
      }
    }
    Tb[i] = v;
  }
}

// W2 = T_b W1 (m x N), kApplyCols columns of W1 per CTA, thread r one row.
constexpr size_t kApplySmem = (size_t)(kNb * (kNb + 1) + kNb * kApplyCols) * 8;
__global__ void __launch_bounds__(kNb) k_apply_tfactor(int N, int m, const double* __restrict__ Tb,
                                                       const double* __restrict__ W1, double* W2) {
  extern __shared__ double sa[];
  double(*Ts)[kNb + 1] = (double(*)[kNb + 1])sa;                   // [kNb][kNb + 1]
  double(*Ws)[kApplyCols] = (double(*)[kApplyCols])(sa + kNb * (kNb + 1));  // [kNb][kApplyCols]
  const int r = threadIdx.x, c0 = blockIdx.x * kApplyCols;
  for (int i = 0; i < kNb; ++i) Ts[i][r] = Tb[i * kNb + r];
  for (int cc = 0; cc < kApplyCols; ++cc) {
    const int c = c0 + cc;
    Ws[r][cc] = (r < m && c < N) ? W1[(size_t)r * N + c] : 0.0;
  }
  __syncthreads();
  if (r >= m) return;
  double acc[kApplyCols];
#pragma unroll
  for (int cc = 0; cc < kApplyCols; ++cc) acc[cc] = 0.0;
  for (int c = r; c < m; ++c) {
    const double t = Ts[r][c];
#pragma unroll
    for (int cc = 0; cc < kApplyCols; ++cc) acc[cc] += t * Ws[c][cc];
  }
#pragma unroll
  for (int cc = 0; cc < kApplyCols; ++cc) {
    const int c = c0 + cc;
    if (c < N) W2[(size_t)r * N + c] = acc[cc];
  }
}

struct DevInfo {
  int sms = 0;
};
std::mutex g_dev_mu;
std::map<int, DevInfo> g_dev;

int device_sms(int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DONOF_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  auto it = g_dev.find(dev);
  if (it == g_dev.end()) {
    DevInfo di;
    if (cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return DONOF_ERR_CUDA;
    it = g_dev.emplace(dev, di).first;
  }
  *sms = it->second.sms;
  return DONOF_OK;
}

}  // namespace

size_t eigh_workspace_bytes(int N) { return eigh_layout(N).total; }

int eigh_run(int N, const double* A, double* V, double* w, char* ws, cudaStream_t s) {
  if (N < 1 || N > kEighMaxN || !A || !V || !w || !ws) return DONOF_ERR_INVALID_ARG;
  const EighLayout L = eigh_layout(N);
  EighHdr* hdr = (EighHdr*)(ws + L.hdr);
  double* Aw = (double*)(ws + L.A);
  double* Yr = (double*)(ws + L.Yr);
  double* Wd = (double*)(ws + L.Wd);
  double* Wp = (double*)(ws + L.Wp);
  double* d = (double*)(ws + L.d);
  double* e = (double*)(ws + L.e);
  double* ds = (double*)(ws + L.ds);
  double* es = (double*)(ws + L.es);
  double* e2 = (double*)(ws + L.e2);
  float* df = (float*)(ws + L.df);
  float* e2f = (float*)(ws + L.e2f);
  double* tau = (double*)(ws + L.tau);
  double* lam = (double*)(ws + L.lam);
  double* glo = (double*)(ws + L.glo);
  double* ghi = (double*)(ws + L.ghi);
  int* col = (int*)(ws + L.col);
  int* bstart = (int*)(ws + L.bstart);
  int* bend = (int*)(ws + L.bend);
  int* incl = (int*)(ws + L.incl);
  int* cl = (int*)(ws + L.cl);
  int* cj = (int*)(ws + L.cj);
  double* T = (double*)(ws + L.T);
  double* G = (double*)(ws + L.G);
  double* W1 = (double*)(ws + L.W1);
  double* W2 = (double*)(ws + L.W2);
  double* part = (double*)(ws + L.part);
  const long long nn = (long long)N * N;
  const size_t nnb = (size_t)nn * 8;
  auto ok = [](cudaError_t e) { return e == cudaSuccess; };

  if (!ok(cudaMemsetAsync(hdr, 0, sizeof(EighHdr), s))) return DONOF_ERR_CUDA;
  const int gcopy = (int)((nn + 255) / 256 < 152 * 4 ? (nn + 255) / 256 : 152 * 4);
  k_eigh_amax<<<gcopy, 256, 0, s>>>(A, nn, hdr);
  k_eigh_scale_copy<<<gcopy, 256, 0, s>>>(A, nn, hdr, Aw);
  count_launch(2);
  // V may share A's storage: it is written only after the scaled copy
  if (!ok(cudaMemsetAsync(Yr, 0, nnb, s)) || !ok(cudaMemsetAsync(V, 0, nnb, s)))
    return DONOF_ERR_CUDA;

  // 1. tridiagonal reduction, one CTA per SM, co-resident (cooperative launch)
  int sms = 0;
  int rc = device_sms(&sms);
  if (rc != DONOF_OK) return rc;
  const size_t tri_smem = (size_t)3 * N * 8;
  if (!ok(cudaFuncSetAttribute(k_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tri_smem)))
    return DONOF_ERR_CUDA;
  int occ = 0;
  if (!ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tridiag, kTriThreads, tri_smem)) ||
      occ < 1)
    return DONOF_ERR_CUDA;
  TriArgs ta{N, Aw, Yr, d, e, tau, (double*)(ws + L.pbuf), hdr};
  void* targs[] = {&ta};
  if (!ok(cudaLaunchCooperativeKernel((const void*)k_tridiag, dim3(sms), dim3(kTriThreads), targs,
                                      tri_smem, s)))
    return DONOF_ERR_CUDA;
  count_launch(1);

  // 2. eigenvalues (of T scaled to ||T||_inf <= 1)
  const size_t prep_smem = (size_t)2 * N * 4;
  if (!ok(cudaFuncSetAttribute(k_tri_prep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)prep_smem)))
    return DONOF_ERR_CUDA;
  k_tri_prep<<<1, 256, prep_smem, s>>>(N, d, e, hdr, ds, es, e2, df, e2f, bstart, bend, glo, ghi);
  const size_t bis_smem = (size_t)N * 24;
  if (!ok(cudaFuncSetAttribute(k_bisect, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)bis_smem)))
    return DONOF_ERR_CUDA;
  k_bisect<<<(N * 16 + kBisThreads - 1) / kBisThreads, kBisThreads, bis_smem, s>>>(
      N, ds, e2, df, e2f, bstart, bend, glo, ghi, hdr, lam);
  const size_t rank_smem = (size_t)N * 12;
  if (!ok(cudaFuncSetAttribute(k_rank_plan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)rank_smem)))
    return DONOF_ERR_CUDA;
  k_rank_plan<<<(N + 255) / 256, 256, rank_smem, s>>>(N, lam, bend, hdr, col, w, incl, cl, cj,
                                                      bstart);
  // 3. eigenvectors of T (into V)
  k_twisted<<<(2 * N + 31) / 32, 32, 0, s>>>(N, ds, es, e2, bstart, bend, lam, col, incl, V, Wp,
                                            Wd);
  count_launch(4);
  if (!ok(cudaGetLastError())) return DONOF_ERR_CUDA;
  // clusters: the plan is read on the host (one wait for the stream)
  int hp[2] = {0, 0};
  if (!ok(cudaMemcpyAsync(hp, &hdr->ncl, sizeof(hp), cudaMemcpyDeviceToHost, s)) ||
      !ok(cudaStreamSynchronize(s)))
    return DONOF_ERR_CUDA;
  if (hp[0] > 0) {
    // the scratch: Aw (free after the reduction) for the large clusters' vectors, Wd and Wp rows
    // for the members' factorisations (free after the twisted factorisations)
    k_cluster_vectors<<<(N + 31) / 32, 32, 0, s>>>(N, ds, es, bstart, bend, lam, col, incl, cj, cl,
                                                   V, Aw, Wd, Wp);
    k_cluster_small<<<kFixCTAs, 32, 0, s>>>(N, col, cl, hdr, V);
    count_launch(2);
    if (!ok(cudaGetLastError())) return DONOF_ERR_CUDA;
  }
  if (hp[1] > kSmallCl) {
    std::vector<int> hcl((size_t)kClDesc * hp[0]);
    if (!ok(cudaMemcpyAsync(hcl.data(), cl, hcl.size() * 4, cudaMemcpyDeviceToHost, s)) ||
        !ok(cudaStreamSynchronize(s)))
      return DONOF_ERR_CUDA;
    double* Cc = W1;  // r0 x 32 overlaps of a panel with the rows before it
    double* Gp = W2;  // 32 x 32 Gram matrix of a panel
    for (int q = 0; q < hp[0]; ++q) {
      const int* c = &hcl[(size_t)kClDesc * q];
      const int m = c[1], L = c[3];
      if (m <= kSmallCl) continue;
      double* Y = Aw + c[4];
      for (int r0 = 0; r0 < m; r0 += 32) {
        const int b = m - r0 < 32 ? m - r0 : 32;
        double* P = Y + (size_t)r0 * L;
        for (int pass = 0; pass < 2; ++pass) {
          if (r0 > 0) {
            // Cc = Y[0:r0] P^T, then P -= Cc^T Y[0:r0]
            if (!ok(cudaMemsetAsync(Cc, 0, (size_t)r0 * b * 8, s)) ||
                !ok(launch_dgemm(split_k_args(r0, b, L, Y, L, 1, P, 1, L, Cc, b, 1, part), s)))
              return DONOF_ERR_CUDA;
            DgemmArgs u{};
            u.M = b; u.N = L; u.K = r0; u.KB = 1; u.batch = 1; u.ksplit = 1;
            u.A = Cc; u.sAm = 1; u.sAk = b;
            u.B = Y; u.sBk = L; u.sBn = 1;
            u.C = P; u.sCm = L; u.sCn = 1;
            u.alpha = -1.0; u.beta = 1.0;
            if (!ok(launch_dgemm(u, s))) return DONOF_ERR_CUDA;
          }
          if (!ok(cudaMemsetAsync(Gp, 0, (size_t)b * b * 8, s)) ||
              !ok(launch_dgemm(split_k_args(b, b, L, P, L, 1, P, 1, L, Gp, b, 1, part), s)))
            return DONOF_ERR_CUDA;
          k_chol_apply<<<(L + 127) / 128, 128, 0, s>>>(b, L, Gp, P);
          count_launch(1);
        }
      }
      k_cluster_scatter<<<152 * 4, 256, 0, s>>>(N, c[0], m, c[2], L, Y, col, V);
      count_launch(1);
      if (!ok(cudaGetLastError())) return DONOF_ERR_CUDA;
    }
  }

  // 4. V = Q Z
  if (L.nblk > 0) {
    if (!ok(cudaFuncSetAttribute(k_apply_tfactor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kApplySmem)))
      return DONOF_ERR_CUDA;
    k_gram<<<dim3(L.nblk, kNb / 16, kNb / 16), 256, 0, s>>>(N, L.nref, Yr, G);
    k_tfactor<<<L.nblk, kNb, 0, s>>>(L.nref, tau, G, T);
    count_launch(2);
  }
  for (int b = L.nblk - 1; b >= 0; --b) {
    const int k0 = b * kNb;
    const int m = L.nref - k0 < kNb ? L.nref - k0 : kNb;
    const int R0 = k0 + 1, nR = N - R0;
    // W1 = Y_b^T Z[R0:, :]
    if (!ok(cudaMemsetAsync(W1, 0, (size_t)m * N * 8, s))) return DONOF_ERR_CUDA;
    if (!ok(launch_dgemm(split_k_args(m, N, nR, Yr + (size_t)k0 * N + R0, N, 1, V + (size_t)R0 * N,
                                      N, 1, W1, N, 1, part),
                         s)))
      return DONOF_ERR_CUDA;
    // W2 = T_b W1
    k_apply_tfactor<<<(N + kApplyCols - 1) / kApplyCols, kNb, kApplySmem, s>>>(
        N, m, T + (size_t)b * kNb * kNb, W1, W2);
    count_launch(1);
    // Z[R0:, :] -= Y_b W2
    DgemmArgs u{};
    u.M = nR; u.N = N; u.K = m; u.KB = 1; u.batch = 1; u.ksplit = 1;
    u.A = Yr + (size_t)k0 * N + R0; u.sAm = 1; u.sAk = N;
    u.B = W2; u.sBk = N; u.sBn = 1;
    u.C = V + (size_t)R0 * N; u.sCm = N; u.sCn = 1;
    u.alpha = -1.0; u.beta = 1.0;
    if (!ok(launch_dgemm(u, s))) return DONOF_ERR_CUDA;
  }
  return ok(cudaGetLastError()) ? DONOF_OK : DONOF_ERR_CUDA;
}

}  // namespace donof

using namespace donof;

extern "C" int donof_eigh_workspace_size(int32_t n, size_t* bytes) {
  if (n < 1 || n > kEighMaxN || !bytes) return DONOF_ERR_INVALID_ARG;
  *bytes = eigh_workspace_bytes(n);
  return DONOF_OK;
}

extern "C" int donof_eigh(int32_t n, const double* A, double* V, double* w, void* workspace,
                          size_t workspace_bytes, void* stream) {
  if (n < 1 || n > kEighMaxN || !A || !V || !w) return DONOF_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < eigh_workspace_bytes(n) ||
      ((uintptr_t)workspace % kAlign) != 0)
    return DONOF_ERR_WORKSPACE;
  return eigh_run(n, A, V, w, (char*)workspace, (cudaStream_t)stream);
}

extern "C" int donof_eigh_read_status(const void* workspace, int32_t* status, void* stream) {
  if (!workspace || !status) return DONOF_ERR_INVALID_ARG;
  EighHdr h{};
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return DONOF_ERR_CUDA;
  *status = h.abort ? DONOF_ERR_TIMEOUT : (h.nonfinite ? DONOF_ERR_NONFINITE : DONOF_OK);
  return DONOF_OK;
}
