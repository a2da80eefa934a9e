// Occupation optimisation at fixed orbitals (Sec. III.D, the occupancy step of each
// iteration): minimise E[n(gamma), phi] over the gamma variables.  With the orbitals fixed,
// E depends on gamma only through n, sqrt n and Phi, and the integrals it needs (H_pp,
// J_pq, K_pq) are those left in the workspace by the last build.  n, sqrt n and Phi depend
// on each gamma only through |sin gamma| and |cos gamma|, so the search runs over the box
// [0, pi/2]^ng of representatives: a minimum on a kink of sqrt n = |sin gamma| (an emptied
// weak orbital, a pair split evenly) is then a minimum on a bound, which a projected method
// reaches instead of zigzagging across the kink.
//
// One CTA runs the whole optimisation: projected L-BFGS (memory kMem, two-loop recursion
// on the free variables, initial inverse-Hessian scale s.y / y.y) with a backtracking
// line search on the Armijo condition along the projected path; converged when the
// projected gradient is below gtol.  Each evaluation of E and dE/dgamma is a block-wide
// pass: occupations per orbital (Eqs. soo, woo), the energy rows and the partials dE/dn,
// dE/dsqrt n, dE/dPhi per orbital (one warp each, from three matrix-vector products with J
// and K and a correction over the orbital's own subspace), then the chain rule per pair
// (one thread each, over the pair's members in index order, so the result does not depend
// on thread scheduling).
#include "common.cuh"
#include "occ.cuh"

namespace donof {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kMem = 8;
constexpr double kPi = 3.14159265358979323846;
constexpr double kLo = 0.0, kHi = 0.5 * kPi;  // the box of gamma representatives

struct OccCtx {
  int A, ng, npair, ncwo, functional;
  const int32_t* pm;
  const double* J;
  const double* K;
  const double* Hd;
  // shared memory
  int* rank;
  int* mem;     // members of subspace g at mem[g * msz + k], k < cnt[g], in index order
  int* cnt;
  int msz;      // 1 + ncwo
  double *n, *sqn, *phi, *en, *es, *ep, *epart;
  double *sn, *cs;  // sin and cos of the current gamma's, formed once per evaluation
  double* red;      // kWarps + 1 words
};

// Sum of v over the block, the same value returned to every thread (fixed order).
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();  // red may still be read by a previous call
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += red[w];
    red[kWarps] = t;
  }
  __syncthreads();
  return red[kWarps];
}

__device__ double block_max(double v, double* red) {
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = red[0];
    for (int w = 1; w < kWarps; ++w) t = fmax(t, red[w]);
    red[kWarps] = t;
  }
  __syncthreads();
  return red[kWarps];
}

__device__ double dot(const double* a, const double* b, int m, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += kThreads) s += a[i] * b[i];
  return block_sum(s, red);
}

// E(gamma) and dE/dgamma -> grad (shared), returned E identical on every thread.
__device__ double evaluate(const OccCtx& c, const double* x, double* grad) {
  const int A = c.A;
  for (int k = threadIdx.x; k < c.ng; k += kThreads) {
    c.sn[k] = sin(x[k]);
    c.cs[k] = cos(x[k]);
  }
  __syncthreads();
  const TrigTable tr{c.sn, c.cs};
  for (int p = threadIdx.x; p < A; p += kThreads) {
    if (c.pm[p] >= c.npair) {  // Omega_I: n = 1/2, no gamma
      c.n[p] = 0.5;
      c.sqn[p] = 0.70710678118654752440;
      c.phi[p] = 0.5;
    } else {
      occ_orbital(p, c.pm[p], c.rank[p], c.npair, c.ncwo, tr, c.n[p], c.sqn[p], c.phi[p],
                  [](int, double, double, double) {});
    }
  }
  __syncthreads();
  // Row p of E and the partials dE/dn_p, dE/dsqrt n_p, dE/dPhi_p (one thread per row): the
  // different-subspace form summed over every q by three matrix-vector products,
  //   u = J n, v = K n, w = K Phi (PNOF7) or K Phi^2 (PNOF7s),
  // then the few q of p's own subspace moved from that form to the intra-subspace one
  // (coefficients as in pair_coefficients).  J and K are symmetric, so row p is read as
  // column p: consecutive threads read consecutive words.
  const bool f7 = c.functional == DONOF_PNOF7, f7s = c.functional == DONOF_PNOF7S;
  for (int p = threadIdx.x; p < A; p += kThreads) {
    double u = 0.0, v = 0.0, w = 0.0;
#pragma unroll 4
    for (int q = 0; q < A; ++q) {
      const double jqp = c.J[(size_t)q * A + p], kqp = c.K[(size_t)q * A + p], nq = c.n[q];
      u = fma(jqp, nq, u);
      v = fma(kqp, nq, v);
      if (f7) w = fma(kqp, c.phi[q], w);
      else if (f7s) w = fma(kqp, c.phi[q] * c.phi[q], w);
    }
    const double* Jp = c.J + (size_t)p * A;
    const double* Kp = c.K + (size_t)p * A;
    const int g = c.pm[p];
    const bool single = g >= c.npair;
    const double np_ = c.n[p], sp = c.sqn[p], fp = c.phi[p];
    double e = 2.0 * np_ * u - np_ * v;
    double a_n = 2.0 * (2.0 * u - v), a_s = 0.0, a_p = -2.0 * w, a_7s = w;
    if (f7) e -= fp * w;
    else if (f7s) e -= 4.0 * fp * fp * w;
    for (int k = 0; k < c.cnt[g]; ++k) {
      const int q = c.mem[g * c.msz + k];
      const double jpq = Jp[q], kpq = Kp[q];
      const double nq = c.n[q], sq = c.sqn[q], fq = c.phi[q];
      e -= 2.0 * np_ * nq * jpq - np_ * nq * kpq;
      if (f7) e += fp * fq * kpq;
      else if (f7s) e += 4.0 * fp * fp * fq * fq * kpq;
      a_n -= 2.0 * nq * (2.0 * jpq - kpq);
      a_p += 2.0 * fq * kpq;
      a_7s -= fq * fq * kpq;
      if (!single) {
        const bool plus = (p == q || (p >= c.npair && q >= c.npair));
        e += (plus ? 1.0 : -1.0) * sp * sq * kpq;
        a_s += (plus ? 2.0 : -2.0) * sq * kpq;
      }
    }
    a_n += 2.0 * c.Hd[p];
    if (f7s) a_n -= 8.0 * (1.0 - 2.0 * np_) * a_7s;
    c.epart[p] = e + 2.0 * np_ * c.Hd[p];
    c.en[p] = a_n;
    c.es[p] = a_s;
    c.ep[p] = f7 ? a_p : 0.0;
  }
  __syncthreads();
  // chain rule, one thread per pair: its gamma's are g and the pair's weak block; the
  // members in index order (the threads of a warp handle their k-th members together)
  for (int g = threadIdx.x; g < c.npair; g += kThreads) {
    const int wbase = c.npair + g * (c.ncwo - 1);
    grad[g] = 0.0;
    for (int j = 0; j < c.ncwo - 1; ++j) grad[wbase + j] = 0.0;
    for (int m = 0; m < c.cnt[g]; ++m) {
      const int p = c.mem[g * c.msz + m];
      double nn, sq, ph;
      occ_orbital(p, g, c.rank[p], c.npair, c.ncwo, tr, nn, sq, ph,
                  [&](int k, double dnk, double dsk, double dpk) {
                    grad[k] += c.en[p] * dnk + c.es[p] * dsk + c.ep[p] * dpk;
                  });
    }
  }
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int p = 0; p < A; ++p) t += c.epart[p];
  return block_sum(threadIdx.x == 0 ? t : 0.0, c.red);  // also orders the grad writes
}

__global__ void __launch_bounds__(kThreads, 1)
    k_occ_lbfgs(Dims d, const int32_t* __restrict__ pm, const double* __restrict__ J,
                const double* __restrict__ K, const double* __restrict__ Hd, double* gamma,
                int max_iter, double gtol, DevHeader* hdr, double* E_out, int32_t* iters_out) {
  extern __shared__ double sh[];
  const int A = d.A, ng = d.ng;
  OccCtx c;
  c.A = A; c.ng = ng; c.npair = d.npair; c.ncwo = d.ncwo; c.functional = d.functional;
  c.pm = pm; c.J = J; c.K = K; c.Hd = Hd;
  double* x = sh;
  double* gr = x + ng;
  double* xn = gr + ng;
  double* gn = xn + ng;
  double* dir = gn + ng;
  double* fr = dir + ng;           // 1 for a free variable, 0 for one held on a bound
  double* S = fr + ng;             // [kMem][ng]
  double* Y = S + kMem * ng;       // [kMem][ng]
  double* rho = Y + kMem * ng;     // [kMem]
  double* alpha = rho + kMem;      // [kMem]
  c.n = alpha + kMem;
  c.sqn = c.n + A;
  c.phi = c.sqn + A;
  c.en = c.phi + A;
  c.es = c.en + A;
  c.ep = c.es + A;
  c.epart = c.ep + A;
  c.sn = c.epart + A;              // [ng]
  c.cs = c.sn + ng;                // [ng]
  c.red = c.cs + ng;               // kWarps + 1
  c.rank = (int*)(c.red + kWarps + 1);
  const int nsub = d.npair + d.nsingle;
  c.msz = 1 + d.ncwo;
  c.cnt = c.rank + A;              // [nsub]
  c.mem = c.cnt + nsub;            // [nsub][1 + ncwo]
  if (threadIdx.x == 0) {          // member lists in index order
    for (int g = 0; g < nsub; ++g) c.cnt[g] = 0;
    for (int p = 0; p < A; ++p) {
      const int g = pm[p];
      if (g >= 0 && g < nsub && c.cnt[g] < c.msz) c.mem[g * c.msz + c.cnt[g]++] = p;
    }
  }

  for (int p = threadIdx.x; p < A; p += kThreads) {
    int r = 0;
    const int g = pm[p];
    if (g < 0 || g >= d.npair + d.nsingle) set_status(hdr, DONOF_ERR_PAIR_MAP);
    if (p >= d.npair + d.nsingle)
      for (int q = d.npair + d.nsingle; q < p; ++q) r += (pm[q] == g);
    c.rank[p] = r;
  }
  // the representative in [0, pi/2]: n, sqrt n and Phi depend on each gamma only through
  // |sin gamma| and |cos gamma|
  for (int k = threadIdx.x; k < ng; k += kThreads) {
    double t = fmod(gamma[k], kPi);
    if (t < 0.0) t += kPi;
    x[k] = t > kHi ? kPi - t : t;
  }
  __syncthreads();

  double f = evaluate(c, x, gr);
  int hist = 0, head = 0;  // number of stored pairs, next slot
  int it = 0;
  for (; it < max_iter; ++it) {
    // projected gradient and the free set: a variable on a bound whose gradient points out
    // of the box is held
    double pg = 0.0;
    for (int k = threadIdx.x; k < ng; k += kThreads) {
      const double xk = x[k], gk = gr[k];
      pg = fmax(pg, fabs(fmin(fmax(xk - gk, kLo), kHi) - xk));
      fr[k] = ((xk <= kLo && gk > 0.0) || (xk >= kHi && gk < 0.0)) ? 0.0 : 1.0;
    }
    pg = block_max(pg, c.red);
    if (!(pg >= gtol)) break;  // converged (or non-finite: stop)
    // two-loop recursion on the free variables: dir = -H grad
    for (int k = threadIdx.x; k < ng; k += kThreads) dir[k] = fr[k] * gr[k];
    __syncthreads();
    for (int j = 0; j < hist; ++j) {
      const int s = (head - 1 - j + kMem) % kMem;
      const double a = rho[s] * dot(S + s * ng, dir, ng, c.red);
      if (threadIdx.x == 0) alpha[s] = a;
      for (int k = threadIdx.x; k < ng; k += kThreads) dir[k] -= fr[k] * a * Y[s * ng + k];
      __syncthreads();
    }
    double scale;
    if (hist > 0) {
      const int s = (head - 1 + kMem) % kMem;
      const double yy = dot(Y + s * ng, Y + s * ng, ng, c.red);
      scale = 1.0 / (rho[s] * yy);
    } else {
      const double gg = dot(dir, dir, ng, c.red);
      scale = 1.0 / fmax(sqrt(gg), 1.0);  // first step: at most unit length
    }
    for (int k = threadIdx.x; k < ng; k += kThreads) dir[k] *= scale;
    __syncthreads();
    for (int j = hist - 1; j >= 0; --j) {
      const int s = (head - 1 - j + kMem) % kMem;
      const double b = rho[s] * dot(Y + s * ng, dir, ng, c.red);
      const double a = alpha[s];
      for (int k = threadIdx.x; k < ng; k += kThreads) dir[k] += fr[k] * (a - b) * S[s * ng + k];
      __syncthreads();
    }
    for (int k = threadIdx.x; k < ng; k += kThreads) dir[k] = -dir[k];
    __syncthreads();
    double dg = dot(dir, gr, ng, c.red);
    if (!(dg < 0.0)) {  // not a descent direction: restart from projected steepest descent
      hist = 0;
      double gg = 0.0;
      for (int k = threadIdx.x; k < ng; k += kThreads) gg += fr[k] * gr[k] * gr[k];
      gg = block_sum(gg, c.red);
      const double sc = 1.0 / fmax(sqrt(gg), 1.0);
      for (int k = threadIdx.x; k < ng; k += kThreads) dir[k] = -sc * fr[k] * gr[k];
      __syncthreads();
    }
    // backtracking line search along the projected path (Armijo, c1 = 1e-4); a step whose
    // projection does not descend is shortened like a rejected one
    double t = 1.0, fn = 0.0;
    bool accepted = false;
    for (int ls = 0; ls < 60; ++ls) {
      double pred = 0.0;
      for (int k = threadIdx.x; k < ng; k += kThreads) {
        xn[k] = fmin(fmax(x[k] + t * dir[k], kLo), kHi);
        pred += gr[k] * (xn[k] - x[k]);
      }
      pred = block_sum(pred, c.red);  // also orders the xn writes
      if (pred < 0.0) {
        fn = evaluate(c, xn, gn);
        if (fn <= f + 1e-4 * pred) {
          accepted = true;
          break;
        }
        // at the rounding level of E the Armijo test is noise: a step that does not raise E
        // beyond rounding and shrinks the projected gradient is taken
        if (fn <= f + 4e-16 * fabs(f)) {
          double pgn = 0.0;
          for (int k = threadIdx.x; k < ng; k += kThreads)
            pgn = fmax(pgn, fabs(fmin(fmax(xn[k] - gn[k], kLo), kHi) - xn[k]));
          pgn = block_max(pgn, c.red);
          if (pgn < pg) {
            accepted = true;
            break;
          }
        }
      }
      t *= 0.5;
    }
    if (!accepted) {
      if (hist == 0) break;  // not even projected steepest descent lowers E: stationary
      hist = 0;              // otherwise drop the curvature pairs and retry from there
      continue;
    }
    // history update s = xn - x, y = gn - gr
    const int s = head;
    for (int k = threadIdx.x; k < ng; k += kThreads) {
      S[s * ng + k] = xn[k] - x[k];
      Y[s * ng + k] = gn[k] - gr[k];
    }
    __syncthreads();
    const double sy = dot(S + s * ng, Y + s * ng, ng, c.red);
    if (sy > 1e-300) {
      if (threadIdx.x == 0) rho[s] = 1.0 / sy;
      head = (head + 1) % kMem;
      hist = hist < kMem ? hist + 1 : kMem;
    }
    for (int k = threadIdx.x; k < ng; k += kThreads) {
      x[k] = xn[k];
      gr[k] = gn[k];
    }
    f = fn;
    __syncthreads();
  }
  for (int k = threadIdx.x; k < ng; k += kThreads) gamma[k] = x[k];
  if (threadIdx.x == 0) {
    if (E_out) *E_out = f;
    if (iters_out) *iters_out = it;
    if (!isfinite(f)) set_status(hdr, DONOF_ERR_NONFINITE);
  }
}

size_t occ_smem_bytes(const Dims& d) {
  const size_t ng = d.ng > 0 ? d.ng : 1;
  const size_t nsub = (size_t)d.npair + d.nsingle;
  return (8 * ng + 2 * kMem * ng + 2 * kMem + 7 * (size_t)d.A + kWarps + 1) * sizeof(double) +
         ((size_t)d.A + nsub + nsub * (1 + d.ncwo)) * sizeof(int);
}

}  // namespace
}  // namespace donof

using namespace donof;

extern "C" int donof_optimize_occupations(const donof_problem* prob, const int32_t* pair_map,
                                          double* gamma, void* workspace,
                                          size_t workspace_bytes, int32_t max_iter,
                                          double gtol, double* E, int32_t* iters, void* stream) {
  if (!prob || !pair_map || !gamma || max_iter < 0 || !(gtol > 0.0)) return DONOF_ERR_INVALID_ARG;
  size_t need = 0;
  int rc = donof_workspace_size(prob, &need);
  if (rc != DONOF_OK) return rc;
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace % kAlign) != 0)
    return DONOF_ERR_WORKSPACE;
  const Dims d = make_dims(prob);
  if (d.ng == 0) return DONOF_ERR_UNSUPPORTED;  // no gamma to optimise
  const Layout L = make_layout(d);
  const size_t smem = occ_smem_bytes(d);
  if (smem > 200 * 1024) return DONOF_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  if (cudaFuncSetAttribute(k_occ_lbfgs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return DONOF_ERR_CUDA;
  prof_begin(DONOF_PHASE_OCC_OPT, s);
  k_occ_lbfgs<<<1, kThreads, smem, s>>>(d, pair_map, (const double*)(ws + L.J),
                                        (const double*)(ws + L.K), (const double*)(ws + L.Hd),
                                        gamma, max_iter, gtol, (DevHeader*)(ws + L.header), E,
                                        iters);
  count_launch(1);
  prof_end(DONOF_PHASE_OCC_OPT, s);
  return cudaGetLastError() == cudaSuccess ? DONOF_OK : DONOF_ERR_CUDA;
}
