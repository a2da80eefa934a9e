"""The NOF-MP2 HF-like and static energies (Eqs. HFL, Esta) on the GPU against the oracle,
from the integrals of an FP64 or a mixed build, with and without singly occupied
orbitals."""
import numpy as np
import pytest

import synth
from oracle import nofmp2, pnof

from helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_06142_gb300.build as b
    b.build()


@pytest.mark.parametrize("shape", [(24, 96, 5, 1, 0), (41, 60, 3, 2, 3), (130, 257, 6, 4, 1),
                                   (200, 400, 44, 3, 0)],
                         ids=["plain", "singles", "tail", "wide"])
@pytest.mark.parametrize("precision", [0, 1])
def test_matches_oracle(shape, precision):
    import torch
    import paper_2004_06142_gb300 as dn
    nbf, naux, npair, ncwo, ns = shape
    prob = synth.Problem(nbf, naux, npair, ncwo, seed=44, nsingle=ns)
    d = synth.generate(prob)
    ref = pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], npair, ncwo, pnof.PNOF7,
                     nsingle=ns)
    E_hf_ref = nofmp2.hf_like_energy(ref["Hdiag"], ref["J"], ref["K"], npair, ns)
    E_sta_ref, _, _ = nofmp2.static_correlation(ref["occ"], ref["K"], d["pair_map"], npair, ns)
    b = dn.Builder(nbf, naux, npair, ncwo, dn.PNOF7, dn.B_DENSE, precision, nsingle=ns)
    b.prepare(to_dev(d["B"]))
    pm = to_dev(d["pair_map"].astype(np.int32))
    b.forward(to_dev(d["h"]), to_dev(d["C"]), to_dev(d["gamma"]), pm, want_lam=False)
    E_hf, E_sta = b.nofmp2_static(pm)
    torch.cuda.synchronize()
    assert b.status() == 0
    tol = 1e-10 if precision == 0 else 1e-6
    assert abs(E_hf.item() - E_hf_ref) <= tol
    assert abs(E_sta.item() - E_sta_ref) <= tol
