"""The hand-off to the orbital update (donof_orbital_update): F of Eq. Fockian from the
Lagrangian and a given diagonal, its double eigendecomposition and the reorthonormalised
rotated orbitals C V.

Eigenvectors are compared through their projectors, which are defined whatever the signs
(and, for a cluster of close eigenvalues, only the cluster's projector is):
sin(theta_j) = sqrt(1 - (v_j . u_j)^2) is the spectral-norm distance between the rank-one
projectors of v_j and u_j, computed as the norm of v_j's component orthogonal to u_j.  Two
comparisons:

  * the library's eigensolver against numpy eigh of the same F (built from the Lagrangian
    the library computed): a backward-stable solver moves eigenvalues by O(N eps ||F||) and
    eigenvector j by that over its gap (Davis-Kahan); the budget is 1e-10 ||F||;
  * the whole hand-off against the oracle's F: the two Lagrangians differ by dF (the mixed
    path's error), so eigenvalues may differ by ||dF||_2 (Weyl) and projectors by
    ||dF||_2 / (gap_j - ||dF||_2) (Davis-Kahan), plus the solver budget.
"""
import numpy as np
import pytest

import synth
from oracle import pnof

from helpers import gpu_build, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_06142_gb300.build as b
    b.build()


def _run_update(lam, Fdiag, C):
    import torch
    import paper_2004_06142_gb300 as dn
    N = C.shape[0]
    C_new = torch.empty(N, N, dtype=torch.float64, device="cuda")
    eps = torch.empty(N, dtype=torch.float64, device="cuda")
    dn.donof_orbital_update(to_dev(lam), to_dev(Fdiag), to_dev(C), C_new, eps)
    torch.cuda.synchronize()
    return eps.cpu().numpy(), C_new.cpu().numpy()


def _gaps(eps):
    """Distance of each eigenvalue to the rest of the spectrum."""
    d = np.diff(eps)
    g = np.full(eps.shape, np.inf)
    g[:-1] = d
    g[1:] = np.minimum(g[1:], d)
    return g


def _sin_theta(V, U):
    """sin of the angle between columns: the norm of v's component orthogonal to u (unit
    columns), accurate to rounding where sqrt(1 - (v.u)^2) would only resolve sqrt(eps)."""
    c = np.sum(V * U, axis=0)
    return np.linalg.norm(V - U * c, axis=0)


def _check_against(eps, Cn, C, F_ref, dF_norm):
    """eps, C_new of the library against eigh(F_ref), F_ref within dF_norm of the F the
    library diagonalised (spectral norm)."""
    eps_ref, V_ref = np.linalg.eigh(F_ref)
    nF = np.linalg.norm(F_ref, 2)
    budget = dF_norm + 1e-10 * nF
    assert np.abs(eps - eps_ref).max() <= budget
    # C orthonormal (synthetic orbitals), so the library's eigenvectors are C^T C_new
    V = C.T @ Cn
    gap = _gaps(eps_ref)
    sep = gap > 2.0 * budget          # separated eigenvalues: rank-one projectors
    assert sep.mean() > 0.99          # the spectra here are (nearly) non-degenerate
    sin = _sin_theta(V[:, sep], V_ref[:, sep])
    assert np.all(sin <= budget / (gap[sep] - budget))
    return eps_ref, V_ref


@pytest.mark.parametrize("shape,precision", [((41, 60, 3, 2), 0), ((120, 480, 8, 4), 0),
                                             ((120, 480, 8, 4), 1)])
def test_orbital_update_against_oracle(shape, precision):
    prob = synth.Problem(*shape, seed=4)
    d = synth.generate(prob)
    ref = pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], prob.npair, prob.ncwo,
                     pnof.PNOF7)
    out = gpu_build(prob, d, precision, pnof.PNOF7, backward=False)
    N = prob.nbf
    Fdiag = -2.0 * np.arange(N) - 5.0          # decreasing: the energy-lowering order
    eps, Cn = _run_update(out["lam"], Fdiag, d["C"])
    np.testing.assert_allclose(Cn.T @ Cn, np.eye(N), rtol=0, atol=1e-12)
    # the solver alone: the F the library diagonalised, from its own Lagrangian
    _check_against(eps, Cn, d["C"], pnof.fockian(out["lam"], Fdiag), 0.0)
    # the hand-off against the oracle: Weyl and Davis-Kahan with the Lagrangians' difference
    F_ref = pnof.fockian(ref["lam"], Fdiag)
    dF = np.linalg.norm(pnof.fockian(out["lam"], Fdiag) - F_ref, 2)
    eps_ref, V_ref = _check_against(eps, Cn, d["C"], F_ref, dF)
    # the energy of the updated orbitals (a function of the orbitals' projectors)
    E_ref = pnof.build(d["h"], d["B"], d["C"] @ V_ref, d["gamma"], d["pair_map"], prob.npair,
                       prob.ncwo, pnof.PNOF7)["E"]
    E_new = gpu_build(prob, dict(d, C=Cn), 0, pnof.PNOF7, backward=False)["E"]
    assert abs(E_new - E_ref) <= (1e-9 if precision == 0 else 1e-5)


def test_orbital_update_headline_shape():
    """The hand-off at the headline shape, nbf 1200 with a Lagrangian of nact = 150 nonzero
    columns (lambda_qp = 0 for p >= nact, as a build returns it): the eigensolver and the
    reorthonormalisation against numpy eigh of the same F."""
    N, A = 1200, 150
    prob = synth.Problem(N, 8, 50, 2, seed=5)
    C = synth.generate(prob, with_B=False)["C"]
    rng = np.random.default_rng([5, 9])
    lam = np.zeros((N, N))
    lam[:, :A] = rng.standard_normal((N, A))
    Fdiag = -2.0 * np.arange(N) - 5.0
    eps, Cn = _run_update(lam, Fdiag, C)
    np.testing.assert_allclose(Cn.T @ Cn, np.eye(N), rtol=0, atol=1e-12)
    _check_against(eps, Cn, C, pnof.fockian(lam, Fdiag), 0.0)
