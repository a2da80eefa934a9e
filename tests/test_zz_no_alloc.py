"""The allocation-free build entry point (donof_energy_lagrangian_noalloc).

For callers that cannot allocate device memory when they need a build, the library keeps
a fixed scratch array in device global memory.  This file checks, through the C ABI, that
two calls in a row reproduce the regular entry point's outputs within the parity
tolerances, and that problems too large for the scratch are refused before any device
work.  It sits last in collection order so that a failure here leaves every other test
already run.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = {0: (1e-10, 1e-10), 1: (1e-6, 1e-5)}   # (energy, arrays) for FP64 and mixed


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_06142_gb300.build as b
    b.build()


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape", [(24, 96, 5, 1), (97, 150, 4, 3)])
def test_noalloc_matches_regular_entry_point(precision, shape):
    import torch
    import paper_2004_06142_gb300 as dn
    prob = synth.Problem(*shape, seed=5)
    d = synth.generate(prob)
    h, B, C, g = _dev(d["h"]), _dev(d["B"]), _dev(d["C"]), _dev(d["gamma"])
    pm = _dev(d["pair_map"].astype(np.int32))
    bld = dn.Builder(prob.nbf, prob.naux, prob.npair, prob.ncwo, dn.PNOF7, dn.B_DENSE, precision)
    bld.prepare(B)
    E0, lam0, dg0 = bld.forward(h, C, g, pm)
    dC0, _ = bld.backward(torch.ones(1, dtype=torch.float64, device="cuda"))
    assert bld.status() == 0
    tol_e, tol_a = TOL[precision]
    for _ in range(2):
        E = torch.empty(1, dtype=torch.float64, device="cuda")
        lam = torch.empty(prob.nbf, prob.nbf, dtype=torch.float64, device="cuda")
        dg = torch.empty(prob.ngamma, dtype=torch.float64, device="cuda")
        dC = torch.empty(prob.nbf, prob.nbf, dtype=torch.float64, device="cuda")
        dn.donof_energy_lagrangian_noalloc(bld.prob, h, B, C, g, pm, E, lam, dg, dC)
        torch.cuda.synchronize()
        assert abs(E.item() - E0.item()) <= tol_e
        for a, b in ((lam, lam0), (dg, dg0), (dC, dC0)):
            assert (a - b).abs().max().item() <= tol_a


def test_noalloc_refuses_problems_beyond_its_scratch():
    import torch
    import paper_2004_06142_gb300 as dn
    prob = dn.make_problem(1200, 4800, 50, 2, b_layout=dn.B_PACKED, precision=dn.MIXED)
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    pm = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(dn.DonofError) as e:
        dn.donof_energy_lagrangian_noalloc(prob, x, x, x, x, pm, x)
    assert e.value.code == -4
