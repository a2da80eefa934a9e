"""Occupation optimisation at fixed orbitals on the GPU (donof_optimize_occupations) against
the oracle's optimiser (Sec. III.D): same start, same fixed orbitals; the optimal energies
agree, the GPU optimum is a point where the oracle's E equals the GPU's E, and for a single
pair with one weak orbital it is the lowest eigenvalue of the 2 x 2 two-configuration
matrix."""
import numpy as np
import pytest

import synth
from oracle import optimize, pnof

from helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_06142_gb300.build as b
    b.build()


def _gpu_opt(prob, d, precision, functional, C=None, gamma0=None):
    import torch
    import paper_2004_06142_gb300 as dn
    b = dn.Builder(prob.nbf, prob.naux, prob.npair, prob.ncwo, functional, dn.B_DENSE, precision)
    b.prepare(to_dev(d["B"]))
    pm = to_dev(d["pair_map"].astype(np.int32))
    g = to_dev(d["gamma"] if gamma0 is None else gamma0).clone()
    b.forward(to_dev(d["h"]), to_dev(d["C"] if C is None else C), g, pm, want_lam=False)
    E, it = b.optimize_occupations(g, pm, max_iter=1000, gtol=1e-10)
    torch.cuda.synchronize()
    assert b.status() == 0
    return E.item(), g.cpu().numpy(), int(it.item())


@pytest.mark.parametrize("shape", [(24, 96, 5, 1), (41, 60, 3, 2), (120, 480, 8, 4)],
                         ids=["plain", "ragged", "differentiation"])
@pytest.mark.parametrize("functional", [pnof.PNOF5, pnof.PNOF7, pnof.PNOF7S])
@pytest.mark.parametrize("precision", [0, 1])
def test_occupation_optimum_matches_oracle(shape, functional, precision):
    prob = synth.Problem(*shape, seed=21)
    d = synth.generate(prob)
    ref = pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], prob.npair, prob.ncwo,
                     functional)
    Hd, J, K = ref["Hdiag"], ref["J"], ref["K"]
    _, E_ref, _ = optimize.optimize_occupations(Hd, J, K, d["gamma"], d["pair_map"], prob.npair,
                                                prob.ncwo, functional, gtol=1e-11)
    E, gam, it = _gpu_opt(prob, d, precision, functional)
    tol = 1e-9 if precision == 0 else 1e-6
    assert E <= ref["E"] + tol
    assert abs(E - E_ref) <= tol, (E, E_ref, it)
    # the oracle's energy at the GPU's optimum is the GPU's energy
    E_at, _ = optimize.energy_of_gamma(gam, Hd, J, K, d["pair_map"], prob.npair, prob.ncwo,
                                       functional)
    assert abs(E_at - E) <= tol


def test_single_pair_two_by_two_ci():
    prob = synth.Problem(16, 64, 1, 1, seed=22)
    d = synth.generate(prob)
    C = np.linalg.eigh(d["h"])[1]
    ref = pnof.build(d["h"], d["B"], C, d["gamma"], d["pair_map"], 1, 1, pnof.PNOF7)
    Hd, J, K = ref["Hdiag"], ref["J"], ref["K"]
    M = np.array([[2 * Hd[0] + J[0, 0], K[0, 1]], [K[0, 1], 2 * Hd[1] + J[1, 1]]])
    E, _, _ = _gpu_opt(prob, d, 0, pnof.PNOF7, C=C, gamma0=np.array([0.2]))
    assert abs(E - np.linalg.eigvalsh(M)[0]) < 1e-10
