"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or factor, a transposed operand) fails at least one of them:

* J, K: brute-force 4-index ERIs (Eq. Gpmn/JKpq against an explicit (pq|rs));
* E: the Roothaan closed-shell energy at the Hartree-Fock limit, the APSG
  determinant-space energy for PNOF5 (Sec. II), the 2RDM contraction of
  Eqs. intra/interaa/interab for PNOF5 and PNOF7, the PNOF7 = PNOF7s
  coincidence at half occupancy (Sec. V);
* lambda / G: the HF Fock matrix at the HF limit, central finite differences
  of E along C_p -> C_p + eps C_q, the Euler identity;
* dE/dgamma: central finite differences through Eqs. soo/woo.
"""
import math

import numpy as np
import pytest

import synth
from oracle import brute, pnof


def tiny(nbf=6, naux=10, npair=2, ncwo=1, seed=0):
    prob = synth.Problem(nbf, naux, npair, ncwo, seed)
    d = synth.generate(prob)
    return prob, d


def run(prob, d, functional=pnof.PNOF7, gamma=None, C=None, B=None, pair_map=None, h=None):
    return pnof.build(d["h"] if h is None else h, d["B"] if B is None else B,
                      d["C"] if C is None else C, d["gamma"] if gamma is None else gamma,
                      d["pair_map"] if pair_map is None else pair_map,
                      prob.npair, prob.ncwo, functional)


# --------------------------------------------------------------------------- generators
def test_generators_deterministic_and_shaped():
    prob, d = tiny(nbf=9, naux=7, npair=2, ncwo=3, seed=3)
    _, d2 = tiny(nbf=9, naux=7, npair=2, ncwo=3, seed=3)
    for k in d:
        np.testing.assert_array_equal(d[k], d2[k])
    assert d["B"].shape == (7, 9, 9)
    np.testing.assert_array_equal(d["B"], d["B"].transpose(0, 2, 1))
    np.testing.assert_allclose(d["C"].T @ d["C"], np.eye(9), atol=1e-13)
    np.testing.assert_array_equal(d["h"], d["h"].T)
    assert np.all(np.diag(d["h"]) <= -1.0) and np.all(np.diag(d["h"]) >= -10.0)
    assert list(d["pair_map"]) == [0, 1, 0, 0, 0, 1, 1, 1]
    Bp = synth.gen_B(3, 7, 9, packed=True)
    np.testing.assert_array_equal(pnof.unpack_B(Bp, 9), d["B"])


def test_weak_gammas_reproduce_dirichlet_split():
    # the weak gammas are the inverse of Eq. woo for a Dirichlet split of the hole
    npair, ncwo, seed = 3, 4, 5
    gam = synth.gen_gamma(seed, npair, ncwo)
    rng = np.random.default_rng([seed, 3])
    gs = rng.uniform(0.0, 1.45, size=npair)
    occ = pnof.occupations(gam, synth.block_pair_map(npair, ncwo), npair, ncwo)
    for g in range(npair):
        hole = 0.5 * math.sin(gs[g]) ** 2
        split = rng.dirichlet(np.ones(ncwo)) * hole
        weak = occ["n"][npair + g * ncwo: npair + (g + 1) * ncwo]
        np.testing.assert_allclose(weak, split, rtol=1e-12, atol=1e-15)


# --------------------------------------------------------------------------- occupations
@pytest.mark.parametrize("ncwo", [1, 2, 4])
def test_sum_rules(ncwo):
    npair = 3
    rng = np.random.default_rng(1)
    gam = rng.uniform(0.05, 1.5, size=npair * ncwo)
    pm = synth.block_pair_map(npair, ncwo)
    occ = pnof.occupations(gam, pm, npair, ncwo)
    n = occ["n"]
    for g in range(npair):   # Eq. sum1
        assert abs(n[pm == g].sum() - 1.0) < 1e-14
    assert abs(2 * n.sum() - 2 * npair) < 1e-13   # Eq. sumNp
    assert np.all(n[:npair] >= 0.5) and np.all(n[npair:] <= 0.5)
    np.testing.assert_allclose(occ["sqrt_n"] ** 2, n, rtol=1e-14)
    np.testing.assert_allclose(occ["phi"] ** 2, n * (1 - n), rtol=1e-12, atol=1e-16)


def test_occupation_jacobians_fd():
    npair, ncwo = 2, 3
    rng = np.random.default_rng(2)
    gam = rng.uniform(0.1, 1.4, size=npair * ncwo)
    pm = synth.block_pair_map(npair, ncwo)
    occ = pnof.occupations(gam, pm, npair, ncwo)
    hstep = 1e-6
    for k in range(len(gam)):
        gp, gm = gam.copy(), gam.copy()
        gp[k] += hstep
        gm[k] -= hstep
        op, om = pnof.occupations(gp, pm, npair, ncwo), pnof.occupations(gm, pm, npair, ncwo)
        for key, dkey in (("n", "dn"), ("sqrt_n", "dsqrt_n"), ("phi", "dphi")):
            fd = (op[key] - om[key]) / (2 * hstep)
            np.testing.assert_allclose(occ[dkey][:, k], fd, atol=1e-8)


# --------------------------------------------------------------------------- J, K
@pytest.mark.parametrize("packed", [False, True])
def test_jk_against_4index_eri(packed):
    prob, d = tiny(nbf=7, naux=11, npair=2, ncwo=2, seed=4)
    B = synth.gen_B(4, 11, 7, packed=packed)
    out = pnof.build(d["h"], B, d["C"], d["gamma"], d["pair_map"], 2, 2, pnof.PNOF7, packed=packed)
    eri = brute.eri_ao(d["B"])
    mo = brute.eri_mo(eri, d["C"])
    J, K = brute.jk_from_eri(mo, prob.nact)
    np.testing.assert_allclose(out["J"], J, atol=1e-13)
    np.testing.assert_allclose(out["K"], K, atol=1e-13)
    # invariants of the MO integrals
    np.testing.assert_allclose(np.diag(out["J"]), np.diag(out["K"]), atol=1e-14)
    np.testing.assert_allclose(out["J"], out["J"].T, atol=1e-14)
    np.testing.assert_allclose(out["K"], out["K"].T, atol=1e-14)
    assert np.all(out["K"] >= -1e-15)
    assert np.linalg.eigvalsh(out["J"]).min() > -1e-13


# --------------------------------------------------------------------------- energy
@pytest.mark.parametrize("functional", [pnof.PNOF5, pnof.PNOF7, pnof.PNOF7S])
@pytest.mark.parametrize("ncwo", [1, 3])
def test_hartree_fock_limit(functional, ncwo):
    """gamma_g = 0: n_g = 1, weak n = 0; E is the closed-shell Roothaan energy and
    G[:, g] = F C_g with the RHF Fock matrix F (so lambda_qg = (C^T F C)_qg)."""
    prob, d = tiny(nbf=13, naux=12, npair=3, ncwo=ncwo, seed=6)
    gam = d["gamma"].copy()
    gam[: prob.npair] = 0.0
    out = run(prob, d, functional, gamma=gam)
    eri = brute.eri_ao(d["B"])
    E_hf, F = brute.roothaan(d["h"], eri, d["C"][:, : prob.npair])
    assert abs(out["E"] - E_hf) < 1e-12
    FC = F @ d["C"][:, : prob.npair]
    np.testing.assert_allclose(out["G"][:, : prob.npair], FC, atol=1e-12)
    np.testing.assert_allclose(out["G"][:, prob.npair:], 0.0, atol=1e-14)
    np.testing.assert_allclose(out["lam"][:, : prob.npair], d["C"].T @ FC, atol=1e-12)


@pytest.mark.parametrize("ncwo", [1, 2])
def test_pnof5_is_apsg_expectation(ncwo):
    prob, d = tiny(nbf=6, naux=9, npair=2, ncwo=ncwo, seed=7)
    out = run(prob, d, pnof.PNOF5)
    C = d["C"][:, : prob.nact]
    h_mo = C.T @ d["h"] @ C
    mo = brute.eri_mo(brute.eri_ao(d["B"]), C)
    members = pnof.pair_members(d["pair_map"], prob.npair)
    psi = brute.apsg_wavefunction(members, out["occ"]["sqrt_n"])
    assert abs(sum(c * c for c in psi.values()) - 1.0) < 1e-13
    E_apsg = brute.hamiltonian_expectation(psi, h_mo, mo)
    assert abs(out["E"] - E_apsg) < 1e-12


@pytest.mark.parametrize("functional", [pnof.PNOF5, pnof.PNOF7])
def test_energy_equals_2rdm_contraction(functional):
    prob, d = tiny(nbf=7, naux=9, npair=2, ncwo=2, seed=8)
    out = run(prob, d, functional)
    C = d["C"][:, : prob.nact]
    h_mo = C.T @ d["h"] @ C
    mo = brute.eri_mo(brute.eri_ao(d["B"]), C)
    members = pnof.pair_members(d["pair_map"], prob.npair)
    occ = out["occ"]
    E2 = brute.energy_from_2rdm(h_mo, mo, occ["n"], occ["sqrt_n"], occ["phi"], members,
                                with_phi=(functional == pnof.PNOF7))
    assert abs(out["E"] - E2) < 1e-12


def test_pnof7s_coincides_with_pnof7_at_half_occupancy():
    """Sec. V: the PNOF7s inter term equals PNOF7's when all orbitals are half occupied."""
    prob, d = tiny(nbf=8, naux=10, npair=3, ncwo=1, seed=9)
    gam = np.full(prob.ngamma, math.pi / 2)
    e7 = run(prob, d, pnof.PNOF7, gamma=gam)["E"]
    e7s = run(prob, d, pnof.PNOF7S, gamma=gam)["E"]
    e5 = run(prob, d, pnof.PNOF5, gamma=gam)["E"]
    assert abs(e7 - e7s) < 1e-12
    assert abs(e7 - e5) > 1e-3          # the Phi term is switched on and non-trivial there
    g2 = d["gamma"]
    assert abs(run(prob, d, pnof.PNOF7, gamma=g2)["E"] - run(prob, d, pnof.PNOF7S, gamma=g2)["E"]) > 1e-6


def test_single_pair_functionals_agree():
    prob, d = tiny(nbf=6, naux=8, npair=1, ncwo=3, seed=10)
    es = [run(prob, d, f)["E"] for f in (pnof.PNOF5, pnof.PNOF7, pnof.PNOF7S)]
    assert max(es) - min(es) < 1e-13


# --------------------------------------------------------------------------- gradients
@pytest.mark.parametrize("functional", [pnof.PNOF5, pnof.PNOF7, pnof.PNOF7S])
def test_dE_dgamma_fd(functional):
    prob, d = tiny(nbf=13, naux=14, npair=3, ncwo=3, seed=11)
    out = run(prob, d, functional)
    hstep = 1e-5
    for k in range(prob.ngamma):
        gp, gm = d["gamma"].copy(), d["gamma"].copy()
        gp[k] += hstep
        gm[k] -= hstep
        fd = (run(prob, d, functional, gamma=gp)["E"] - run(prob, d, functional, gamma=gm)["E"]) / (2 * hstep)
        assert abs(out["dE_dgamma"][k] - fd) < 1e-8, (k, out["dE_dgamma"][k], fd)


@pytest.mark.parametrize("functional", [pnof.PNOF5, pnof.PNOF7, pnof.PNOF7S])
def test_dE_dC_fd(functional):
    prob, d = tiny(nbf=8, naux=12, npair=2, ncwo=2, seed=12)
    out = run(prob, d, functional)
    rng = np.random.default_rng(0)
    hstep = 1e-5
    for _ in range(3):
        D = rng.standard_normal(d["C"].shape)
        ep = run(prob, d, functional, C=d["C"] + hstep * D)["E"]
        em = run(prob, d, functional, C=d["C"] - hstep * D)["E"]
        assert abs(np.sum(out["dE_dC"] * D) - (ep - em) / (2 * hstep)) < 1e-8


def test_lambda_fd_and_euler_identity():
    """lambda_qp = 1/4 dE/deps along C_p -> C_p + eps C_q; E = sum_p (lambda_pp + n_p H_pp)."""
    prob, d = tiny(nbf=8, naux=12, npair=2, ncwo=2, seed=13)
    out = run(prob, d, pnof.PNOF7)
    hstep = 1e-5
    for q, p in [(0, 0), (3, 1), (1, 4), (7, 2), (5, 5)]:
        Cp, Cm = d["C"].copy(), d["C"].copy()
        Cp[:, p] += hstep * d["C"][:, q]
        Cm[:, p] -= hstep * d["C"][:, q]
        fd = (run(prob, d, pnof.PNOF7, C=Cp)["E"] - run(prob, d, pnof.PNOF7, C=Cm)["E"]) / (2 * hstep)
        assert abs(out["lam"][q, p] - fd / 4) < 1e-9
    euler = np.trace(out["lam"]) + np.sum(out["n"] * out["Hdiag"])
    assert abs(out["E"] - euler) < 1e-12
    np.testing.assert_allclose(out["lam"][:, prob.nact:], 0.0)


# --------------------------------------------------------------------------- invariances
def test_invariances():
    prob, d = tiny(nbf=8, naux=10, npair=2, ncwo=2, seed=14)
    ref = run(prob, d, pnof.PNOF7)
    rng = np.random.default_rng(3)
    # rotation of the auxiliary index
    O, _ = np.linalg.qr(rng.standard_normal((prob.naux, prob.naux)))
    B2 = np.einsum("PQ,Qmn->Pmn", O, d["B"])
    assert abs(run(prob, d, pnof.PNOF7, B=B2)["E"] - ref["E"]) < 1e-12
    # orthogonal AO rotation: h -> U^T h U, B^P -> U^T B^P U, C -> U^T C
    U, _ = np.linalg.qr(rng.standard_normal((prob.nbf, prob.nbf)))
    out = run(prob, d, pnof.PNOF7, h=U.T @ d["h"] @ U, B=np.einsum("am,Pab,bn->Pmn", U, d["B"], U),
              C=U.T @ d["C"])
    assert abs(out["E"] - ref["E"]) < 1e-12
    np.testing.assert_allclose(out["lam"], ref["lam"], atol=1e-12)
    # permutation of the orbitals together with pair_map (weak order within a pair kept)
    perm = np.array([1, 0, 4, 2, 5, 3, 7, 6])     # new orbital i is old orbital perm[i]
    pm_old = d["pair_map"]
    nact = prob.nact
    pm_new = np.array([pm_old[perm[i]] for i in range(nact)], dtype=np.int32)
    # strong orbital of pair g must sit at index g: relabel pairs by their strong index
    relabel = {pm_old[perm[g]]: g for g in range(prob.npair)}
    pm_new = np.array([relabel[x] for x in pm_new], dtype=np.int32)
    gam = d["gamma"].copy()
    gam_new = gam.copy()
    for g_new in range(prob.npair):
        g_old = pm_old[perm[g_new]]
        gam_new[g_new] = gam[g_old]
        w = prob.ncwo - 1
        gam_new[prob.npair + g_new * w: prob.npair + (g_new + 1) * w] = gam[prob.npair + g_old * w: prob.npair + (g_old + 1) * w]
    C2 = d["C"][:, perm]
    out = run(prob, d, pnof.PNOF7, C=C2, pair_map=pm_new, gamma=gam_new)
    assert abs(out["E"] - ref["E"]) < 1e-12
    np.testing.assert_allclose(out["lam"], ref["lam"][np.ix_(perm, perm)], atol=1e-12)


def test_jk_entries_streaming_matches_operator_route():
    prob, d = tiny(nbf=9, naux=13, npair=2, ncwo=2, seed=15)
    out = run(prob, d, pnof.PNOF7)
    pairs = [(0, 0), (1, 4), (5, 2)]
    J, K = pnof.jk_entries(iter(d["B"]), d["C"][:, : prob.nact], pairs)
    for pq in pairs:
        assert abs(J[pq] - out["J"][pq]) < 1e-13
        assert abs(K[pq] - out["K"][pq]) < 1e-13


def test_fockian_first_order_energy_change():
    """Diagonalising F of Eq. Fockian with a widely spaced diagonal rotates the orbitals by
    A_qp = F_qp / (F_pp - F_qq) to first order (Eq. fi1); since dE/dC = 4 G and
    lambda = C^T G, the energy then changes by 4 sum_{q<p} F_qp^2 / (F_pp - F_qq).
    (Eq. ene1 prints the opposite sign with a factor 2: under the paper's own definition of
    lambda in Eq. lag it is a decreasing diagonal that lowers E.)"""
    prob, d = tiny(nbf=10, naux=16, npair=2, ncwo=2, seed=3)
    out = run(prob, d, pnof.PNOF7)
    N = prob.nbf
    F0 = pnof.fockian(out["lam"], np.zeros(N))
    assert np.allclose(F0, F0.T, atol=0)
    for scale in (-200.0, 200.0):
        diag = scale * np.arange(N)
        eps, Cn = pnof.orbital_update(out["lam"], diag, d["C"])
        np.testing.assert_allclose(Cn.T @ Cn, np.eye(N), atol=1e-12)
        np.testing.assert_allclose(np.sort(eps), np.sort(np.linalg.eigvalsh(pnof.fockian(out["lam"], diag))))
        # eigenvector j is close to e_j: restore the orbital order and signs
        V = d["C"].T @ Cn
        idx = np.argmax(np.abs(V), axis=0)
        assert sorted(idx) == list(range(N))
        V2 = np.zeros_like(V)
        for j in range(N):
            V2[:, idx[j]] = V[:, j] * np.sign(V[idx[j], j])
        E1 = run(prob, d, pnof.PNOF7, C=d["C"] @ V2)["E"]
        pred = sum(4 * F0[q, p] ** 2 / (diag[p] - diag[q]) for p in range(N) for q in range(p))
        assert abs((E1 - out["E"]) - pred) < 0.02 * abs(pred), (E1 - out["E"], pred)
        assert np.sign(E1 - out["E"]) == np.sign(scale)


# --------------------------------------------------------------------------- streaming
def test_streamed_build_equals_plain_build():
    # the AO operators of Eq. Gpmn are sums over the auxiliary index: accumulating them over
    # blocks of slices (dense or packed, ragged last block) must give the one-pass build
    prob, d = tiny(nbf=11, naux=23, npair=2, ncwo=2, seed=4)
    ref = run(prob, d)
    mu, nu = synth.packed_index(prob.nbf)
    for bs, packed in ((5, False), (7, True), (23, False)):
        blocks = [d["B"][p0:p0 + bs] for p0 in range(0, prob.naux, bs)]
        if packed:
            blocks = [b[:, mu, nu] for b in blocks]
        seen = []
        out = pnof.build_streamed(d["h"], iter(blocks), d["C"], d["gamma"], d["pair_map"],
                                  prob.npair, prob.ncwo, pnof.PNOF7, on_block=seen.append)
        assert seen[-1] == prob.naux and len(seen) == len(blocks)
        assert abs(out["E"] - ref["E"]) <= 1e-12
        for k in ("lam", "dE_dgamma", "dE_dC", "J", "K"):
            np.testing.assert_allclose(out[k], ref[k], rtol=0, atol=1e-12)
