"""Pins of the oracle's multiplet terms (Sec. II: N_I singly occupied orbitals in Omega_I,
n = 1/2 each, no intra-subspace term) against things other than itself (CPU only).

* PNOF7 at the limit gamma = 0 (strong orbitals doubly occupied, weak ones empty) with the
  singles half occupied equals the energy of the high-spin single determinant (all singles
  alpha), evaluated by the Slater-Condon rules over spin orbitals from explicit 4-index
  integrals;
* E equals the contraction of the reconstructed 2RDM blocks with explicit integrals
  (Eqs. intra, interaa, interab, with D_pp,pp = 0 in Omega_I and the delta_pt delta_qr form
  of the Phi block between two singles), PNOF5 and PNOF7, at random gamma;
* dE/dgamma, dE/dC and lambda by central finite differences; the Euler identity.
"""
import itertools

import numpy as np
import pytest

import synth
from oracle import brute, pnof


def tiny(nbf=8, naux=12, npair=2, ncwo=1, nsingle=2, seed=0):
    prob = synth.Problem(nbf, naux, npair, ncwo, seed, nsingle=nsingle)
    return prob, synth.generate(prob)


def run(prob, d, functional, gamma=None, C=None):
    return pnof.build(d["h"], d["B"], d["C"] if C is None else C,
                      d["gamma"] if gamma is None else gamma, d["pair_map"], prob.npair,
                      prob.ncwo, functional, nsingle=prob.nsingle)


def _slater_energy(h_mo, g_mo, spin_orbitals):
    """<D|H|D> of one determinant: spin orbitals (spatial index, spin)."""
    E = sum(h_mo[p, p] for p, _ in spin_orbitals)
    for (p, sp), (q, sq) in itertools.combinations(spin_orbitals, 2):
        E += g_mo[p, p, q, q]                    # (pp|qq)
        if sp == sq:
            E -= g_mo[p, q, q, p]                # (pq|qp)
    return E


@pytest.mark.parametrize("nsingle", [1, 2, 3])
def test_high_spin_determinant_limit(nsingle):
    prob, d = tiny(nbf=9, naux=14, npair=2, ncwo=2, nsingle=nsingle, seed=3)
    gamma = np.zeros(prob.ngamma)        # strong n = 1, weak n = 0
    E = run(prob, d, pnof.PNOF7, gamma=gamma)["E"]
    g_mo = brute.eri_mo(brute.eri_ao(d["B"]), d["C"])
    h_mo = d["C"].T @ d["h"] @ d["C"]
    so = [(g, s) for g in range(prob.npair) for s in (0, 1)]
    so += [(prob.npair + k, 0) for k in range(nsingle)]
    assert abs(E - _slater_energy(h_mo, g_mo, so)) < 1e-11


@pytest.mark.parametrize("functional,with_phi", [(pnof.PNOF5, False), (pnof.PNOF7, True)])
def test_energy_equals_2rdm_contraction(functional, with_phi):
    prob, d = tiny(nbf=8, naux=12, npair=2, ncwo=2, nsingle=2, seed=4)
    out = run(prob, d, functional)
    nact = prob.nact
    C_act = d["C"][:, :nact]
    g_mo = brute.eri_mo(brute.eri_ao(d["B"]), C_act)
    h_mo = C_act.T @ d["h"] @ C_act
    occ = out["occ"]
    members = pnof.pair_members(d["pair_map"], prob.npair)
    singles = list(range(prob.npair, prob.npair + prob.nsingle))
    E = brute.energy_from_2rdm(h_mo, g_mo, occ["n"], occ["sqrt_n"], occ["phi"], members,
                               with_phi=with_phi, singles=singles)
    assert abs(out["E"] - E) < 1e-11


@pytest.mark.parametrize("functional", [pnof.PNOF5, pnof.PNOF7, pnof.PNOF7S])
def test_derivatives_by_finite_differences(functional):
    prob, d = tiny(nbf=9, naux=12, npair=2, ncwo=2, nsingle=2, seed=5)
    out = run(prob, d, functional)
    h = 1e-5
    for k in range(prob.ngamma):
        gp, gm = d["gamma"].copy(), d["gamma"].copy()
        gp[k] += h
        gm[k] -= h
        fd = (run(prob, d, functional, gamma=gp)["E"] - run(prob, d, functional, gamma=gm)["E"]) / (2 * h)
        assert abs(out["dE_dgamma"][k] - fd) < 1e-8
    rng = np.random.default_rng(1)
    for _ in range(3):
        D = rng.standard_normal(d["C"].shape)
        fd = (run(prob, d, functional, C=d["C"] + h * D)["E"]
              - run(prob, d, functional, C=d["C"] - h * D)["E"]) / (2 * h)
        assert abs(np.sum(out["dE_dC"] * D) - fd) < 1e-8
    for q, p in [(2, 2), (0, 3), (3, 0), (8, 2), (5, 6)]:   # 2, 3 are the singles
        Cp, Cm = d["C"].copy(), d["C"].copy()
        Cp[:, p] += h * d["C"][:, q]
        Cm[:, p] -= h * d["C"][:, q]
        fd = (run(prob, d, functional, C=Cp)["E"] - run(prob, d, functional, C=Cm)["E"]) / (2 * h)
        assert abs(out["lam"][q, p] - fd / 4) < 1e-9
    euler = np.trace(out["lam"]) + np.sum(out["n"] * out["Hdiag"])
    assert abs(out["E"] - euler) < 1e-12


def test_no_singles_is_unchanged():
    prob, d = tiny(nsingle=0, seed=6)
    a = run(prob, d, pnof.PNOF7)
    b = pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], prob.npair, prob.ncwo,
                   pnof.PNOF7)
    assert a["E"] == b["E"]
