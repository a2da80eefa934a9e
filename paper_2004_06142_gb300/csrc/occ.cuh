// Occupation numbers of one active orbital from the gamma variables (Eqs. soo, woo) and
// their derivatives, shared by the build's occupation kernel and the occupation optimiser.
//
//   strong orbital g:          n_g = (1 + cos^2 gamma_g) / 2,  sqrt(1 - n_g) = |sin gamma_g| / sqrt 2
//   weak orbital i of pair g:  sqrt(n) = sqrt(1 - n_g) * prod_{j<i} |cos gamma_j| * |sin gamma_i|,
//                              the last weak orbital of the pair without the sine factor
//   Phi = sqrt(n (1 - n))
//
// `rank` is the orbital's rank among the weak orbitals of its pair (ignored for strong
// orbitals); `tr` gives sin and cos of each gamma; `put(k, dn/dgamma_k, dsqrt_n/dgamma_k,
// dPhi/dgamma_k)` receives the nonzero derivatives (pass a no-op to skip them).
#pragma once

#include <cuda_runtime.h>

#include "../../include/donof.h"

namespace donof {

// Sines and cosines of the gamma variables, evaluated on demand or read from a table that
// holds exactly those values (the results are the same bits either way).
struct TrigDirect {
  const double* gamma;
  __device__ double s(int k) const { return sin(gamma[k]); }
  __device__ double c(int k) const { return cos(gamma[k]); }
};
struct TrigTable {
  const double* sn;  // sin(gamma[k])
  const double* cs;  // cos(gamma[k])
  __device__ double s(int k) const { return sn[k]; }
  __device__ double c(int k) const { return cs[k]; }
};

template <typename Trig, typename Put>
__device__ inline void occ_orbital(int p, int g, int rank, int npair, int ncwo, const Trig& tr,
                                   double& n_out, double& sqn_out, double& phi_out, Put put) {
  const double rs2 = 0.70710678118654752440;  // 1/sqrt(2)
  const double cg = tr.c(g), sg = tr.s(g);
  const double sh = fabs(sg) * rs2;  // sqrt(1 - n_g) = sqrt(h_g)
  const double dsh = copysign(1.0, sg) * cg * rs2;
  if (p < npair) {
    const double ng_ = 0.5 * (1.0 + cg * cg);
    const double r = sqrt(ng_);
    const double dng = -cg * sg;
    n_out = ng_;
    sqn_out = r;
    phi_out = r * sh;
    put(g, dng, dng / (2.0 * r), dng / (2.0 * r) * sh + r * dsh);
    return;
  }
  const int i = rank;
  const int wbase = npair + g * (ncwo - 1);
  const bool has_sin = (i < ncwo - 1);
  double prodc = 1.0;
  for (int j = 0; j < i; ++j) prodc *= fabs(tr.c(wbase + j));
  const double si = has_sin ? fabs(tr.s(wbase + i)) : 1.0;
  const double val = sh * prodc * si;
  const double nn = val * val;
  const double om = sqrt(1.0 - nn);
  n_out = nn;
  sqn_out = val;
  phi_out = val * om;
  auto emit = [&](int k, double ds) {
    const double dnk = 2.0 * val * ds;
    put(k, dnk, ds, ds * om - val * dnk / (2.0 * om));
  };
  emit(g, dsh * prodc * si);
  for (int j = 0; j < i; ++j) {
    double rest = sh * si;
    for (int jj = 0; jj < i; ++jj)
      if (jj != j) rest *= fabs(tr.c(wbase + jj));
    emit(wbase + j, -copysign(1.0, tr.c(wbase + j)) * tr.s(wbase + j) * rest);
  }
  if (has_sin)
    emit(wbase + i, copysign(1.0, tr.s(wbase + i)) * tr.c(wbase + i) * sh * prodc);
}

// Coefficients of J_pq and K_pq in E (Eqs. Eg, Efg, Efg_s): same subspace A = 0, B = Pi_pq
// (sign + for p = q or both weak, - when one of them is the strong orbital), none for a
// singly occupied orbital (`single`: the subspace belongs to Omega_I); different
// subspaces A = 2 n_p n_q and B = -n_p n_q [- Phi_p Phi_q (PNOF7) | - 4 Phi_p^2 Phi_q^2 (PNOF7s)].
__device__ inline void pair_coefficients(int functional, int npair, int p, int q, bool same,
                                         bool single, double np_, double nq, double sp,
                                         double sq, double fp, double fq, double& a,
                                         double& b) {
  if (same && single) {  // Omega_I: D_pp,pp = 0, no intra-subspace term
    a = 0.0;
    b = 0.0;
  } else if (same) {
    const bool plus = (p == q || (p >= npair && q >= npair));
    a = 0.0;
    b = (plus ? 1.0 : -1.0) * sp * sq;
  } else {
    a = 2.0 * np_ * nq;
    b = -np_ * nq;
    if (functional == DONOF_PNOF7) b -= fp * fq;
    else if (functional == DONOF_PNOF7S) b -= 4.0 * fp * fp * fq * fq;
  }
}

}  // namespace donof
