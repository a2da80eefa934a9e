"""Brute-force references that pin the oracle on tiny inputs (nbf <= ~12).

TEST INFRASTRUCTURE.  Only tests may use this module.  None of it shares code
with the CUDA library.

* explicit 4-index ERIs (mu nu|eta delta) = sum_P B^P_{mu nu} B^P_{eta delta},
  transformed to the MO basis one index at a time;
* the closed-shell Roothaan energy and Fock matrix (the Hartree-Fock limit of
  the functional, cf. the HF-like energy of Eq. HFL without singles);
* the APSG expectation value <Psi|H|Psi> in the determinant space, with the
  Hamiltonian of Eq. Ham (PNOF5 is the APSG energy, Sec. II);
* the energy of Eq. ENOF contracted with the reconstructed spin blocks of the
  2RDM, Eqs. intra, interaa and interab (the route the paper collapses into
  Eqs. EPNOF7 / Eg / Efg "after a simple algebra").
"""
from __future__ import annotations

import itertools

import numpy as np


def eri_ao(B: np.ndarray) -> np.ndarray:
    """(mu nu|eta delta), chemists' notation."""
    return np.einsum("Pab,Pcd->abcd", B, B)


def eri_mo(eri: np.ndarray, C: np.ndarray) -> np.ndarray:
    """(pq|rs) = sum C_mu p C_nu q C_eta r C_delta s (mu nu|eta delta), one index at a time."""
    t = np.einsum("abcd,ap->pbcd", eri, C)
    t = np.einsum("pbcd,bq->pqcd", t, C)
    t = np.einsum("pqcd,cr->pqrd", t, C)
    return np.einsum("pqrd,ds->pqrs", t, C)


def jk_from_eri(eri_mo_: np.ndarray, nact: int):
    """J_pq = (pp|qq), K_pq = (pq|qp) over the first nact orbitals."""
    J = np.empty((nact, nact))
    K = np.empty((nact, nact))
    for p in range(nact):
        for q in range(nact):
            J[p, q] = eri_mo_[p, p, q, q]
            K[p, q] = eri_mo_[p, q, q, p]
    return J, K


def roothaan(h: np.ndarray, eri: np.ndarray, C_occ: np.ndarray):
    """Closed-shell RHF energy 1/2 tr[P (h + F)] and Fock matrix F = h + J[P] - K[P]/2,
    P = 2 C_occ C_occ^T."""
    P = 2.0 * C_occ @ C_occ.T
    Jm = np.einsum("abcd,cd->ab", eri, P)
    Km = np.einsum("acbd,cd->ab", eri, P)
    F = h + Jm - 0.5 * Km
    return 0.5 * np.sum(P * (h + F)), F


# ----------------------------------------------------------------------------
# determinant space: spin orbital i = 2 p + s  (s = 0 alpha, 1 beta)
# ----------------------------------------------------------------------------
def _annihilate(det: int, i: int):
    if not (det >> i) & 1:
        return None, 0
    sign = -1 if bin(det & ((1 << i) - 1)).count("1") % 2 else 1
    return det ^ (1 << i), sign


def _create(det: int, i: int):
    if (det >> i) & 1:
        return None, 0
    sign = -1 if bin(det & ((1 << i) - 1)).count("1") % 2 else 1
    return det | (1 << i), sign


def _apply_string(det: int, ops):
    """Apply a product of operators given right-to-left as (kind, index)."""
    sign = 1
    for kind, i in ops:
        det, s = (_create if kind == "c" else _annihilate)(det, i)
        if det is None:
            return None, 0
        sign *= s
    return det, sign


def hamiltonian_expectation(psi: dict, h_mo: np.ndarray, eri_mo_: np.ndarray) -> float:
    """<Psi|H|Psi> with H of Eq. Ham in spin orbitals:
    H = sum_ik H_ki a+_k a_i + 1/2 sum_ijkl <kl|ij> a+_k a+_l a_j a_i,
    <kl|ij> = (k i|l j) times the spin deltas."""
    norb = h_mo.shape[0]
    M = 2 * norb
    out = {}
    for det, c in psi.items():
        for k in range(M):
            for i in range(M):
                if k % 2 != i % 2:
                    continue
                d2, s = _apply_string(det, [("a", i), ("c", k)])
                if d2 is not None:
                    out[d2] = out.get(d2, 0.0) + c * s * h_mo[k // 2, i // 2]
        for k, l, i, j in itertools.product(range(M), repeat=4):
            if k % 2 != i % 2 or l % 2 != j % 2:
                continue
            v = eri_mo_[k // 2, i // 2, l // 2, j // 2]
            if v == 0.0:
                continue
            d2, s = _apply_string(det, [("a", i), ("a", j), ("c", l), ("c", k)])
            if d2 is not None:
                out[d2] = out.get(d2, 0.0) + 0.5 * c * s * v
    return sum(psi.get(d, 0.0) * v for d, v in out.items())


def apsg_wavefunction(members, sqrt_n) -> dict:
    """Psi = prod_g (sum_{p in Omega_g} c_p a+_{p alpha} a+_{p beta}) |0>,
    c_g = +sqrt(n_g), c_p = -sqrt(n_p) for weak p."""
    psi = {0: 1.0}
    for Om in members:
        g = Om[0]
        new = {}
        for det, c in psi.items():
            for p in Om:
                cp = sqrt_n[p] if p == g else -sqrt_n[p]
                d2, s = _apply_string(det, [("c", 2 * p + 1), ("c", 2 * p)])
                if d2 is not None:
                    new[d2] = new.get(d2, 0.0) + c * s * cp
        psi = new
    return psi


# ----------------------------------------------------------------------------
# Eq. ENOF with the reconstructed 2RDM of Eqs. intra, interaa, interab
# ----------------------------------------------------------------------------
def energy_from_2rdm(h_mo, eri_mo_, n, sqrt_n, phi, members, with_phi=True, singles=()) -> float:
    """E = sum_sigma sum_p n_p H_pp + sum over spin blocks of D_{pq,rt} <pq|rt>,
    <pq|rt> = (pr|qt).  D^{ab} enters twice (alpha-beta and beta-alpha), D^{ss}
    once per spin.  ``members`` lists the subspaces of Omega_II; ``singles`` the orbitals
    of Omega_I, each its own subspace, with no intra-subspace alpha-beta element and the
    delta_pt delta_qr form of the Phi block between two of them (Eq. interab)."""
    nact = len(n)
    sub = np.empty(nact, dtype=int)
    strong = set()
    for g, Om in enumerate(members):
        strong.add(Om[0])
        for p in Om:
            sub[p] = g
    single_sub = set()
    for k, s in enumerate(singles):
        sub[s] = len(members) + k
        single_sub.add(len(members) + k)
    phys = lambda p, q, r, t: eri_mo_[p, r, q, t]
    E = 2.0 * sum(n[p] * h_mo[p, p] for p in range(nact))
    Dab = np.zeros((nact,) * 4)
    Dss = np.zeros((nact,) * 4)
    for p, q, r, t in itertools.product(range(nact), repeat=4):
        v = 0.0
        # intra-pair alpha-beta block (Eq. intra), Omega_II only
        if p == q and r == t and sub[p] == sub[r] and sub[p] not in single_sub:
            if p == r or (p not in strong and r not in strong):
                Pi = sqrt_n[p] * sqrt_n[r]
            else:
                Pi = -sqrt_n[p] * sqrt_n[r]
            v += 0.5 * Pi
        # inter-pair alpha-beta block (Eq. interab), f = sub[p], g = sub[q] or sub[r]
        if sub[p] != sub[q] and p == r and q == t:
            v += 0.5 * n[p] * n[q]
        both_single = sub[p] in single_sub and sub[r] in single_sub
        if with_phi and sub[p] != sub[r]:
            if (not both_single and p == q and r == t) or (both_single and p == t and q == r):
                v -= 0.5 * phi[p] * phi[r]
        Dab[p, q, r, t] = v
        # inter-pair parallel-spin block (Eq. interaa)
        if sub[p] != sub[q]:
            Dss[p, q, r, t] = 0.5 * n[p] * n[q] * ((p == r) * (q == t) - (p == t) * (q == r))
    for p, q, r, t in itertools.product(range(nact), repeat=4):
        w = phys(p, q, r, t)
        E += 2.0 * Dab[p, q, r, t] * w + 2.0 * Dss[p, q, r, t] * w
    return E
