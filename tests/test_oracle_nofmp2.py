"""Pins of the oracle's NOF-MP2 reference and static energies (Sec. "Dynamic Correlation",
Eqs. HFL, Esta) against things other than their own formulas (CPU only).

* at integer occupations (every gamma 0: strong orbitals full, weak ones empty) every
  functional's E is the closed-shell HF energy of the strong orbitals, which is Eq. HFL;
  and E^sta vanishes there (Lambda = 0 and Phi = 0 for n in {0, 1});
* the inter-subspace term of Eq. Esta is the PNOF7s functional minus PNOF5 (Eq. Efg_s
  against Eq. Efg without Phi), for any occupations, with and without singly occupied
  orbitals;
* one pair with one weak orbital: n_w <= 1/2, Lambda_g = Lambda_w = 2 n_w and
  Pi_gw = -sqrt(n_g n_w), so the intra-pair term is -4 n_w Phi_w K_gw.
"""
import numpy as np
import pytest

import synth
from oracle import nofmp2, pnof


def _build(prob, d, gamma, functional):
    return pnof.build(d["h"], d["B"], d["C"], gamma, d["pair_map"], prob.npair, prob.ncwo,
                      functional, nsingle=prob.nsingle)


@pytest.mark.parametrize("functional", [pnof.PNOF5, pnof.PNOF7, pnof.PNOF7S])
def test_hf_like_energy_is_every_functional_at_integer_occupations(functional):
    prob = synth.Problem(14, 40, 3, 2, seed=41)
    d = synth.generate(prob)
    ref = _build(prob, d, np.zeros_like(d["gamma"]), functional)
    E_hf = nofmp2.hf_like_energy(ref["Hdiag"], ref["J"], ref["K"], prob.npair)
    assert abs(E_hf - ref["E"]) <= 1e-12 * abs(ref["E"])
    E_sta, intra, inter = nofmp2.static_correlation(ref["occ"], ref["K"], d["pair_map"],
                                                    prob.npair)
    assert E_sta == 0.0 and intra == 0.0 and inter == 0.0


@pytest.mark.parametrize("nsingle", [0, 2])
def test_inter_term_is_pnof7s_minus_pnof5(nsingle):
    prob = synth.Problem(15, 44, 3, 2, seed=42, nsingle=nsingle)
    d = synth.generate(prob)
    e7s = _build(prob, d, d["gamma"], pnof.PNOF7S)
    e5 = _build(prob, d, d["gamma"], pnof.PNOF5)
    _, intra, inter = nofmp2.static_correlation(e5["occ"], e5["K"], d["pair_map"], prob.npair,
                                                nsingle)
    assert inter < 0.0
    assert abs(inter - (e7s["E"] - e5["E"])) <= 1e-12 * abs(e5["E"])


def test_one_pair_one_weak_intra_term():
    prob = synth.Problem(8, 30, 1, 1, seed=43)
    d = synth.generate(prob)
    ref = _build(prob, d, d["gamma"], pnof.PNOF7)
    n, phi, K = ref["occ"]["n"], ref["occ"]["phi"], ref["K"]
    E_sta, intra, inter = nofmp2.static_correlation(ref["occ"], K, d["pair_map"], 1)
    assert inter == 0.0 and n[1] <= 0.5
    assert abs(intra - (-4.0 * n[1] * phi[1] * K[0, 1])) <= 1e-14


def _hf_like_at(prob, d):
    """E_hf of the oracle from the integrals of a build, and the explicit MO integrals."""
    from oracle import brute
    ref = _build(prob, d, d["gamma"], pnof.PNOF7)
    E_hf = nofmp2.hf_like_energy(ref["Hdiag"], ref["J"], ref["K"], prob.npair, prob.nsingle)
    eri = brute.eri_ao(d["B"])
    return E_hf, ref, eri


def test_hf_like_energy_with_one_single_is_the_doublet_determinant():
    # one singly occupied orbital: the HF density matrix with 2n = 2 (pairs) and 2n = 1 (the
    # single) is that of the high-spin doublet determinant, whose energy (Slater-Condon rules
    # over explicit integrals) fixes both the occupation weights of Eq. HFL and its -J_gg/4
    import itertools
    from oracle import brute
    prob = synth.Problem(9, 16, 2, 2, seed=45, nsingle=1)
    d = synth.generate(prob)
    E_hf, ref, eri = _hf_like_at(prob, d)
    g_mo = brute.eri_mo(eri, d["C"])
    h_mo = d["C"].T @ d["h"] @ d["C"]
    so = [(g, s) for g in range(prob.npair) for s in (0, 1)] + [(prob.npair, 0)]
    E_det = sum(h_mo[p, p] for p, _ in so)
    for (p, sp), (q, sq) in itertools.combinations(so, 2):
        E_det += g_mo[p, p, q, q] - (g_mo[p, q, q, p] if sp == sq else 0.0)
    assert abs(E_hf - E_det) <= 1e-11
    # the formula as printed (no occupation factors) is not this energy
    no = prob.npair + 1
    Hd, J, K = ref["Hdiag"], ref["J"], ref["K"]
    printed = (2.0 * Hd[:no].sum() + (2.0 * J[:no, :no] - K[:no, :no]).sum()
               - J[prob.npair, prob.npair] / 4.0)
    assert abs(printed - E_det) > 1e-3


@pytest.mark.parametrize("nsingle", [2, 3])
def test_hf_like_energy_is_the_fractional_roothaan_energy(nsingle):
    # several singly occupied orbitals: the closed-shell-like energy 1/2 tr[P (h + F)] of the
    # HF density matrix P = sum_g 2 w_g C_g C_g^T (w = 1 pairs, 1/2 singles), F = h + J[P] -
    # K[P]/2 from explicit integrals, less the singles' self-interaction J_gg/4
    from oracle import brute
    prob = synth.Problem(10, 18, 2, 1, seed=46, nsingle=nsingle)
    d = synth.generate(prob)
    E_hf, ref, eri = _hf_like_at(prob, d)
    n_omega = prob.npair + nsingle
    w = np.array([1.0] * prob.npair + [0.5] * nsingle)
    C_w = d["C"][:, :n_omega] * np.sqrt(w)[None, :]
    E_rh, _ = brute.roothaan(d["h"], eri, C_w)
    self_int = sum(ref["J"][g, g] for g in range(prob.npair, n_omega)) / 4.0
    assert abs(E_hf - (E_rh - self_int)) <= 1e-11
