"""Pins of the oracle's orbital iterations (Sec. III.B-D) against things other than itself
(CPU only).

* zeta scaling: every scaled element is the original over a power of ten, the smallest
  power that brings it to or below zeta; the diagonal is untouched;
* DIIS: the two-vector coefficients in closed form, and collinear error vectors cancelling;
* a diagonalisation step with small (scaled) off-diagonal elements lowers E, by the
  first-order amount 4 sum_{q<p} F_qp F'_qp / (F_pp - F_qq) (F' the scaled elements, the
  energy gradient along the rotation C_p -> C_p + k C_q being 4 (lambda_qp - lambda_pq));
* a converged run ends at a point where E is stationary under orbital rotations (central
  finite differences along random generators) and below the start.
"""
import numpy as np
import pytest
from scipy.linalg import expm

import synth
from oracle import optimize, pnof


def test_zeta_scaling_powers_of_ten():
    rng = np.random.default_rng(0)
    F = rng.standard_normal((12, 12)) * 10.0 ** rng.uniform(-3, 3, (12, 12))
    zeta = 0.37
    S = optimize.scale_offdiagonal(F, zeta)
    assert np.array_equal(np.diag(S), np.diag(F))
    off = ~np.eye(12, dtype=bool)
    assert np.all(np.abs(S[off]) <= zeta)
    k = np.rint(np.log10(F[off] / S[off]))
    assert np.all(k >= 0)
    np.testing.assert_allclose(S[off], F[off] / 10.0 ** k, rtol=1e-14)
    # the smallest such power: one power fewer would leave the element above zeta
    big = k > 0
    assert np.all(np.abs(F[off][big]) / 10.0 ** (k[big] - 1) > zeta)
    assert np.array_equal(optimize.scale_offdiagonal(F, 0.0), F)


def test_diis_two_vectors_closed_form():
    rng = np.random.default_rng(1)
    e1, e2 = rng.standard_normal(50), rng.standard_normal(50)
    B = np.array([[e1 @ e1, e1 @ e2], [e2 @ e1, e2 @ e2]])
    c = optimize.diis_coefficients(B)
    c1 = (B[1, 1] - B[0, 1]) / (B[0, 0] - 2 * B[0, 1] + B[1, 1])
    np.testing.assert_allclose(c, [c1, 1 - c1], rtol=1e-12)
    # collinear errors: the combination cancels exactly
    c = optimize.diis_coefficients(np.array([[1.0, 0.3], [0.3, 0.09]]) + 0.0)
    assert abs(c[0] * 1.0 + c[1] * 0.3) < 1e-12 and abs(c.sum() - 1) < 1e-12


def _start(shape, seed, functional=pnof.PNOF7):
    prob = synth.Problem(*shape, seed=seed)
    d = synth.generate(prob)
    ref = pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], prob.npair, prob.ncwo,
                     functional)
    lam = ref["lam"]
    eps, V = np.linalg.eigh(0.5 * (lam + lam.T))
    return prob, d, d["C"] @ V, -eps


@pytest.mark.parametrize("functional", [pnof.PNOF5, pnof.PNOF7, pnof.PNOF7S])
def test_small_steps_lower_energy_first_order(functional):
    prob, d, C, Fdiag = _start((16, 48, 3, 1), 5, functional)
    run = lambda C_: pnof.build(d["h"], d["B"], C_, d["gamma"], d["pair_map"], prob.npair,
                                prob.ncwo, functional)
    zeta = 2e-4  # rotation angles F'/(F_pp - F_qq) below 0.02
    ref = run(C)
    E_prev = ref["E"]
    for step in range(5):
        F = pnof.fockian(ref["lam"], Fdiag)
        Fs = optimize.scale_offdiagonal(F, zeta)
        N = F.shape[0]
        pred = 4.0 * sum(F[q, p] * Fs[q, p] / (F[p, p] - F[q, q])
                         for p in range(N) for q in range(p) if abs(F[q, p]) > 0)
        C, Fdiag = optimize.orbital_step(ref["lam"], Fdiag, C, zeta, [], 0)
        ref = run(C)
        dE = ref["E"] - E_prev
        assert dE < 0, (step, dE)
        assert abs(dE - pred) <= 0.05 * abs(pred), (step, dE, pred)
        E_prev = ref["E"]


def test_converged_point_is_stationary():
    prob = synth.Problem(10, 40, 2, 1, seed=1)
    d = synth.generate(prob)
    res = optimize.optimize(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], prob.npair,
                            prob.ncwo, pnof.PNOF7, zeta=1.0, depth=6, delta=1e-7,
                            eps_energy=1e-11, max_outer=100, max_inner=20)
    assert res["converged"] and res["asym"] < 1e-7
    E0 = pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], 2, 1, pnof.PNOF7)["E"]
    assert res["E"] < E0
    C, gam = res["C"], res["gamma"]
    E = lambda C_: pnof.build(d["h"], d["B"], C_, gam, d["pair_map"], 2, 1, pnof.PNOF7)["E"]
    rng = np.random.default_rng(2)
    h = 1e-4
    for _ in range(4):
        A = rng.standard_normal((10, 10))
        A = (A - A.T) / np.linalg.norm(A - A.T)
        slope = (E(C @ expm(h * A)) - E(C @ expm(-h * A))) / (2 * h)
        assert abs(slope) < 1e-6, slope
