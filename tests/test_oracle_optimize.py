"""Pins of the oracle's optimisation procedure (Sec. III.B-D) against things other than
itself (CPU only).

* occupation optimisation: for a single pair with one weak orbital every functional reduces
  to a two-configuration wave function, whose optimum is the lowest eigenvalue of a 2 x 2
  matrix; with two weak orbitals the optimum is checked by a dense grid refined by a
  derivative-free method, and bounded below by the lowest eigenvalue of the 3 x 3 matrix;
* the optimum is stationary (or on a kink of sqrt(n) = |sin gamma|, with E rising on both
  sides) and lowers E, for several pairs and every functional.
"""
import numpy as np
import pytest
from scipy.optimize import minimize

import synth
from oracle import optimize, pnof


def _fixed_orbital_integrals(prob, d, C=None):
    ref = pnof.build(d["h"], d["B"], d["C"] if C is None else C, d["gamma"], d["pair_map"],
                     prob.npair, prob.ncwo, pnof.PNOF7)
    return ref["Hdiag"], ref["J"], ref["K"]


def _h_eigvecs(d):
    """Orbitals ordered by the one-electron energy, so that the strong orbital 0 is the
    lowest (the parametrisation has n_strong >= 1/2)."""
    w, V = np.linalg.eigh(d["h"])
    return V


@pytest.mark.parametrize("functional", [pnof.PNOF5, pnof.PNOF7, pnof.PNOF7S])
def test_single_pair_one_weak_is_two_by_two_ci(functional):
    prob = synth.Problem(8, 30, 1, 1, seed=11)
    d = synth.generate(prob)
    C = _h_eigvecs(d)
    Hd, J, K = _fixed_orbital_integrals(prob, d, C)
    # E = c^T M c with c = (sqrt n_g, -sqrt n_w), |c| = 1 (Eq. Eg, one subspace)
    M = np.array([[2 * Hd[0] + J[0, 0], K[0, 1]], [K[0, 1], 2 * Hd[1] + J[1, 1]]])
    assert K[0, 1] > 0 and M[0, 0] < M[1, 1]
    e_min = np.linalg.eigvalsh(M)[0]
    gam, E, _ = optimize.optimize_occupations(Hd, J, K, np.array([0.3]), d["pair_map"], 1, 1,
                                              functional, gtol=1e-12)
    assert abs(E - e_min) < 1e-10, (E, e_min)


def test_single_pair_two_weak_grid_and_bound():
    prob = synth.Problem(8, 30, 1, 2, seed=12)
    d = synth.generate(prob)
    C = _h_eigvecs(d)
    Hd, J, K = _fixed_orbital_integrals(prob, d, C)
    pm = d["pair_map"]
    f = lambda x: optimize.energy_of_gamma(x, Hd, J, K, pm, 1, 2, pnof.PNOF7)[0]
    t = np.linspace(0.0, np.pi / 2, 201)
    grid = np.array([[f(np.array([a, b])) for b in t] for a in t])
    i, j = np.unravel_index(np.argmin(grid), grid.shape)
    nm = minimize(f, np.array([t[i], t[j]]), method="Nelder-Mead",
                  options=dict(xatol=1e-12, fatol=1e-15, maxiter=20000))
    gam, E, _ = optimize.optimize_occupations(Hd, J, K, np.array([0.4, 0.7]), pm, 1, 2,
                                              pnof.PNOF7, gtol=1e-12)
    assert E <= grid.min() + 1e-12
    assert abs(E - nm.fun) < 1e-10, (E, nm.fun)
    # variational bound: one subspace, E = c^T M c with |c| = 1 and a fixed sign pattern
    M = np.diag(2 * Hd[:3] + np.diag(J)[:3]) + (K[:3, :3] - np.diag(np.diag(K)[:3]))
    assert E >= np.linalg.eigvalsh(M)[0] - 1e-12


@pytest.mark.parametrize("functional", [pnof.PNOF5, pnof.PNOF7, pnof.PNOF7S])
def test_optimum_is_stationary_and_lower(functional):
    prob = synth.Problem(30, 90, 3, 2, seed=13)
    d = synth.generate(prob)
    Hd, J, K = _fixed_orbital_integrals(prob, d)
    E0, _ = optimize.energy_of_gamma(d["gamma"], Hd, J, K, d["pair_map"], 3, 2, functional)
    gam, E, _ = optimize.optimize_occupations(Hd, J, K, d["gamma"], d["pair_map"], 3, 2,
                                              functional, gtol=1e-11)
    _, g = optimize.energy_of_gamma(gam, Hd, J, K, d["pair_map"], 3, 2, functional)
    assert E < E0
    # smooth components are stationary; a gamma at a multiple of pi/2 may sit on the kink of
    # sqrt(n) = |sin| (an orbital emptied or a pair split evenly), where E does not fall either way
    at_kink = np.abs(np.remainder(gam + 1e-7, np.pi / 2) - 1e-7) < 1e-7
    assert np.abs(g[~at_kink]).max() < 1e-6
    for k in np.flatnonzero(at_kink):
        for t in (-1e-6, 1e-6):
            x = gam.copy()
            x[k] += t
            assert optimize.energy_of_gamma(x, Hd, J, K, d["pair_map"], 3, 2,
                                            functional)[0] >= E - 1e-12
    # a local minimum: small random steps do not lower E
    rng = np.random.default_rng(0)
    for _ in range(20):
        step = 1e-4 * rng.standard_normal(gam.shape)
        assert optimize.energy_of_gamma(gam + step, Hd, J, K, d["pair_map"], 3, 2,
                                        functional)[0] >= E - 1e-13
