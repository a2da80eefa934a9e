"""Multiplets on the GPU (Sec. II: nsingle singly occupied orbitals in Omega_I) against the
oracle: the build in both precisions for every functional, the occupation optimiser, and
the device check of the pair_map layout of the singles."""
import numpy as np
import pytest

import synth
from oracle import optimize, pnof

from helpers import gpu_build, to_dev

pytestmark = pytest.mark.gpu

F64_TOL = 1e-10
MIX_E, MIX_G = 1e-6, 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_06142_gb300.build as b
    b.build()


CASES = [(24, 96, 3, 1, 2), (41, 60, 3, 2, 3), (130, 257, 6, 4, 1)]


@pytest.mark.parametrize("case", CASES, ids=["plain", "ragged", "tail"])
@pytest.mark.parametrize("functional", [pnof.PNOF7, pnof.PNOF5, pnof.PNOF7S])
@pytest.mark.parametrize("precision", [0, 1])
def test_build_matches_oracle(case, functional, precision):
    nbf, naux, npair, ncwo, ns = case
    prob = synth.Problem(nbf, naux, npair, ncwo, seed=31, nsingle=ns)
    d = synth.generate(prob)
    ref = pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], npair, ncwo, functional,
                     nsingle=ns)
    out = gpu_build(prob, d, precision, functional)
    te, tg = (F64_TOL, F64_TOL) if precision == 0 else (MIX_E, MIX_G)
    assert out["status"] == 0
    assert abs(out["E"] - ref["E"]) <= te
    for k in ("lam", "dE_dgamma", "dE_dC", "J", "K"):
        np.testing.assert_allclose(out[k], ref[k], rtol=0, atol=tg, err_msg=k)


def test_occupation_optimiser_with_singles():
    import torch
    import paper_2004_06142_gb300 as dn
    prob = synth.Problem(41, 60, 3, 2, seed=32, nsingle=2)
    d = synth.generate(prob)
    ref = pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], 3, 2, pnof.PNOF7,
                     nsingle=2)
    _, E_ref, _ = optimize.optimize_occupations(ref["Hdiag"], ref["J"], ref["K"], d["gamma"],
                                                d["pair_map"], 3, 2, pnof.PNOF7, nsingle=2)
    b = dn.Builder(41, 60, 3, 2, dn.PNOF7, dn.B_DENSE, dn.FP64, nsingle=2)
    b.prepare(to_dev(d["B"]))
    g = to_dev(d["gamma"]).clone()
    pm = to_dev(d["pair_map"].astype(np.int32))
    b.forward(to_dev(d["h"]), to_dev(d["C"]), g, pm, want_lam=False)
    E, _ = b.optimize_occupations(g, pm, max_iter=1000, gtol=1e-10)
    torch.cuda.synchronize()
    assert b.status() == 0
    assert abs(E.item() - E_ref) < 1e-9


def test_single_pair_map_checked():
    prob = synth.Problem(24, 96, 3, 1, seed=33, nsingle=2)
    d = synth.generate(prob)
    bad = d["pair_map"].copy()
    bad[3] = 4            # a single must be its own subspace at its own index
    out = gpu_build(prob, dict(d, pair_map=bad), 0, pnof.PNOF7, backward=False)
    assert out["status"] == -2
