"""The parts of the NOF-MP2 energy that need only the integrals of a build (Sec. "Dynamic
Correlation", Eqs. Etotal, HFL, Esta): the HF-like energy of the natural orbitals and the
static correlation energy.  The dynamic part E^dyn (Eq. E2) needs amplitudes from modified
MP2 residual equations that the paper cites but does not state; it is not computed here.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module.  It shares no code with the CUDA library.

Readings (listed in the design notes):

* the strong orbitals of Eq. HFL are the first N_Omega orbitals: g < npair the strong
  orbital of pair g, npair <= g < npair + nsingle the singly occupied ones.  The paper
  defines E_hf as the energy of a closed-shell-like HF density matrix with doubly
  (2n_g = 2) and singly (2n_g = 1) occupied orbitals; its printed formula carries no
  occupation factors, which with singles would count each singly occupied orbital as
  doubly occupied.  Reading: each H_gg and (2 J_fg - K_fg) carries the HF occupations
  w_g = 1 (pairs), 1/2 (singles) of that density matrix, i.e.
  2 sum_g w_g H_gg + sum_{f,g} w_f w_g (2 J_fg - K_fg) - sum_{g singly occupied} J_gg / 4;
  the last sum (as printed) removes the self-interaction w_g^2 J_gg of a singly occupied
  orbital.  Without singles this is the printed formula.  Pinned by the RHF energy (no
  singles), the doublet determinant energy (one single: Slater-Condon rules) and the
  fractional-occupation Roothaan energy of that density matrix (several singles);
* Pi_qp in Eq. Esta is that of Eq. intra (pnof._pi); the first sum of Eq. Esta runs over
  the pair subspaces and over ordered q != p inside each; the second over ordered pairs of
  orbitals in different subspaces (singly occupied ones included, Phi = 1/2 there).
"""
from __future__ import annotations

import math

import numpy as np

from oracle import pnof


def hf_like_energy(Hdiag, J, K, npair, nsingle=0):
    """Eq. HFL with the occupations of its HF density matrix (w_g = 1 for the strong orbitals
    of the pairs, 1/2 for the singly occupied ones):
    2 sum_g w_g H_gg + sum_{f,g} w_f w_g (2 J_fg - K_fg) - sum_{g singly occupied} J_gg / 4,
    f and g over the N_Omega = npair + nsingle strong orbitals."""
    n_omega = npair + nsingle
    w = [1.0 if g < npair else 0.5 for g in range(n_omega)]
    E = 0.0
    for g in range(n_omega):
        E += 2.0 * w[g] * Hdiag[g]
    for f in range(n_omega):
        for g in range(n_omega):
            E += w[f] * w[g] * (2.0 * J[f, g] - K[f, g])
    for g in range(npair, n_omega):
        E -= J[g, g] / 4.0
    return E


def static_correlation(occ, K, pair_map, npair, nsingle=0):
    """Eq. Esta with Lambda_p = 1 - |1 - 2 n_p|.  Returns (E_sta, intra, inter)."""
    n, sq, phi = occ["n"], occ["sqrt_n"], occ["phi"]
    lam = 1.0 - np.abs(1.0 - 2.0 * n)
    members = pnof.subspaces(pair_map, npair, nsingle)
    intra = 0.0
    for g in range(npair):
        for q in members[g]:
            for p in members[g]:
                if q != p:
                    intra += math.sqrt(lam[q] * lam[p]) * pnof._pi(p, q, g, sq) * K[p, q]
    inter = 0.0
    for f in range(len(members)):
        for g in range(len(members)):
            if f == g:
                continue
            for p in members[f]:
                for q in members[g]:
                    inter -= 4.0 * phi[q] ** 2 * phi[p] ** 2 * K[p, q]
    return intra + inter, intra, inter
