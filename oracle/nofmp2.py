"""The parts of the NOF-MP2 energy that need only the integrals of a build (Sec. "Dynamic
Correlation", Eqs. Etotal, HFL, Esta): the HF-like energy of the natural orbitals and the
static correlation energy.  The dynamic part E^dyn (Eq. E2) needs amplitudes from modified
MP2 residual equations that the paper cites but does not state; it is not computed here.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module.  It shares no code with the CUDA library.

Readings (listed in the design notes):

* the strong orbitals of Eq. HFL are the first N_Omega orbitals: g < npair the strong
  orbital of pair g, npair <= g < npair + nsingle the singly occupied ones; Eq. HFL is
  taken as printed, its last sum running over the singly occupied g.  For closed shells
  it is pinned (the RHF energy of the strong orbitals); its singly occupied terms are
  parity unpinned (transcription only);
* Pi_qp in Eq. Esta is that of Eq. intra (pnof._pi); the first sum of Eq. Esta runs over
  the pair subspaces and over ordered q != p inside each; the second over ordered pairs of
  orbitals in different subspaces (singly occupied ones included, Phi = 1/2 there).
"""
from __future__ import annotations

import math

import numpy as np

from oracle import pnof


def hf_like_energy(Hdiag, J, K, npair, nsingle=0):
    """Eq. HFL: 2 sum_g H_gg + sum_{f,g} (2 J_fg - K_fg) - sum_{g singly occupied} J_gg / 4,
    f and g over the N_Omega = npair + nsingle strong orbitals."""
    n_omega = npair + nsingle
    E = 0.0
    for g in range(n_omega):
        E += 2.0 * Hdiag[g]
    for f in range(n_omega):
        for g in range(n_omega):
            E += 2.0 * J[f, g] - K[f, g]
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
