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
