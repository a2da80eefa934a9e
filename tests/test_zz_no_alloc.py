"""The allocation-free build entry point (donof_energy_lagrangian_noalloc).

Some callers cannot allocate device memory when they need a build (a host framework that
owns the device pool, a loop where an allocation's synchronisation or failure is not
acceptable); for them the library keeps a fixed scratch array in device global memory.
This file checks, through the C ABI, that two calls in a row reproduce the regular entry
point's outputs within the parity tolerances without changing the device's free memory,
that the device-side checks of a call are reported by donof_noalloc_read_status, and that
problems too large for the scratch are refused before any device work.  It sits last in
collection order so that a failure here leaves every other test already run.
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


def _outputs(prob):
    import torch
    f64, dev = torch.float64, "cuda"
    return (torch.empty(1, dtype=f64, device=dev),
            torch.empty(prob.nbf, prob.nbf, dtype=f64, device=dev),
            torch.empty(prob.ngamma, dtype=f64, device=dev),
            torch.empty(prob.nbf, prob.nbf, dtype=f64, device=dev))


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
    E, lam, dg, dC = _outputs(prob)   # allocated before the calls
    free = []
    for i in range(2):
        for t in (E, lam, dg, dC):
            t.fill_(float("nan"))
        torch.cuda.synchronize()
        if i == 1:  # nothing else allocates between the two readings
            free.append(torch.cuda.mem_get_info()[0])
        dn.donof_energy_lagrangian_noalloc(bld.prob, h, B, C, g, pm, E, lam, dg, dC)
        torch.cuda.synchronize()
        if i == 1:
            free.append(torch.cuda.mem_get_info()[0])
        assert dn.donof_noalloc_read_status() == 0
        assert abs(E.item() - E0.item()) <= tol_e
        for a, b in ((lam, lam0), (dg, dg0), (dC, dC0)):
            assert (a - b).abs().max().item() <= tol_a
    # the first call may load the library's module (and with it the scratch array); the
    # second one allocates nothing
    assert free[1] == free[0]


def test_noalloc_reports_device_side_checks():
    import torch
    import paper_2004_06142_gb300 as dn
    prob = synth.Problem(24, 96, 5, 1, seed=6)
    d = synth.generate(prob)
    h, B, C = _dev(d["h"]), _dev(d["B"]), _dev(d["C"])
    cp = dn.make_problem(prob.nbf, prob.naux, prob.npair, prob.ncwo, dn.PNOF7, dn.B_DENSE,
                         dn.MIXED)
    E, lam, dg, dC = _outputs(prob)
    g_bad = d["gamma"].copy()
    g_bad[1] = np.nan
    dn.donof_energy_lagrangian_noalloc(cp, h, B, C, _dev(g_bad),
                                       _dev(d["pair_map"].astype(np.int32)), E, lam, dg, dC)
    assert dn.donof_noalloc_read_status() == -3          # DONOF_ERR_NONFINITE
    assert dn.donof_noalloc_read_status() == 0           # read clears it
    pm_bad = d["pair_map"].astype(np.int32).copy()
    pm_bad[prob.npair] = 7                               # a weak orbital in no pair
    dn.donof_energy_lagrangian_noalloc(cp, h, B, C, _dev(d["gamma"]), _dev(pm_bad), E, lam, dg,
                                       dC)
    assert dn.donof_noalloc_read_status() == -2          # DONOF_ERR_PAIR_MAP
    # a valid call afterwards starts from a clear status
    dn.donof_energy_lagrangian_noalloc(cp, h, B, C, _dev(d["gamma"]),
                                       _dev(d["pair_map"].astype(np.int32)), E, lam, dg, dC)
    assert dn.donof_noalloc_read_status() == 0
    torch.cuda.synchronize()
    assert np.isfinite(E.item())


def test_noalloc_refuses_problems_beyond_its_scratch():
    import torch
    import paper_2004_06142_gb300 as dn
    prob = dn.make_problem(1200, 4800, 50, 2, b_layout=dn.B_PACKED, precision=dn.MIXED)
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    pm = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(dn.DonofError) as e:
        dn.donof_energy_lagrangian_noalloc(prob, x, x, x, x, pm, x)
    assert e.value.code == -4
