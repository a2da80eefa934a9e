"""The hand-off to the orbital update (donof_orbital_update): F of Eq. Fockian from the
Lagrangian and a given diagonal, its double eigendecomposition and the reorthonormalised
rotated orbitals, against the oracle (numpy eigh of the oracle's F).  Eigenvectors are
compared up to sign (the spectra here are non-degenerate), together with the orthonormality
of the new orbitals and the energy they give."""
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


@pytest.mark.parametrize("shape,precision", [((41, 60, 3, 2), 0), ((120, 480, 8, 4), 0),
                                             ((120, 480, 8, 4), 1)])
def test_orbital_update_against_oracle(shape, precision):
    import torch
    import paper_2004_06142_gb300 as dn
    prob = synth.Problem(*shape, seed=4)
    d = synth.generate(prob)
    ref = pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], prob.npair, prob.ncwo,
                     pnof.PNOF7)
    out = gpu_build(prob, d, precision, pnof.PNOF7, backward=False)
    N = prob.nbf
    Fdiag = -2.0 * np.arange(N) - 5.0          # decreasing: the energy-lowering order
    eps_ref, C_ref = pnof.orbital_update(ref["lam"], Fdiag, d["C"])
    lam_d, Fd, C_d = to_dev(out["lam"]), to_dev(Fdiag), to_dev(d["C"])
    C_new = torch.empty(N, N, dtype=torch.float64, device="cuda")
    eps = torch.empty(N, dtype=torch.float64, device="cuda")
    dn.donof_orbital_update(lam_d, Fd, C_d, C_new, eps)
    torch.cuda.synchronize()
    eps, Cn = eps.cpu().numpy(), C_new.cpu().numpy()
    tol = 1e-9 if precision == 0 else 1e-4
    np.testing.assert_allclose(eps, eps_ref, rtol=0, atol=tol)
    np.testing.assert_allclose(Cn.T @ Cn, np.eye(N), rtol=0, atol=1e-12)
    sgn = np.sign(np.sum(Cn * C_ref, axis=0))
    np.testing.assert_allclose(Cn * sgn, C_ref, rtol=0, atol=1e-7 if precision == 0 else 1e-3)
    # the energy of the updated orbitals
    E_ref = pnof.build(d["h"], d["B"], C_ref, d["gamma"], d["pair_map"], prob.npair, prob.ncwo,
                       pnof.PNOF7)["E"]
    d2 = dict(d, C=Cn * sgn)
    E_new = gpu_build(prob, d2, 0, pnof.PNOF7, backward=False)["E"]
    assert abs(E_new - E_ref) <= (1e-9 if precision == 0 else 1e-5)
