"""The build on host buffers (donof_energy_lagrangian_host): C and gamma copied from host
memory, the build and its adjoint, the outputs copied back, all in one C-ABI call.  Its
results are the device-pointer path's bit for bit, which the parity tests compare with the
oracle."""
import ctypes

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


@pytest.mark.parametrize("precision", [0, 1])
def test_host_buffers_match_device_path(precision):
    import torch
    import paper_2004_06142_gb300 as dn
    prob = synth.Problem(41, 60, 3, 2, seed=6)
    d = synth.generate(prob)
    ref = gpu_build(prob, d, precision, pnof.PNOF7)
    b = dn.Builder(prob.nbf, prob.naux, prob.npair, prob.ncwo, dn.PNOF7, dn.B_DENSE, precision)
    b.prepare(to_dev(d["B"]))
    h, pm = to_dev(d["h"]), to_dev(d["pair_map"].astype(np.int32))
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hC, hg = pin(d["C"]), pin(d["gamma"])
    N, ng = prob.nbf, prob.npair * prob.ncwo
    oE = torch.empty(1, dtype=torch.float64).pin_memory()
    olam = torch.empty(N, N, dtype=torch.float64).pin_memory()
    odg = torch.empty(ng, dtype=torch.float64).pin_memory()
    odC = torch.empty(N, N, dtype=torch.float64).pin_memory()
    staging = dn.alloc_workspace(dn.donof_host_staging_size(b.prob), torch.device("cuda"))
    for _ in range(2):  # the second call reuses the workspace and the staging
        dn.donof_energy_lagrangian_host(b.prob, h, b.B, hC, hg, pm, b.ws, staging, oE, olam, odg,
                                        odC)
        assert oE.item() == ref["E"]
        assert np.array_equal(olam.numpy(), ref["lam"])
        assert np.array_equal(odg.numpy(), ref["dE_dgamma"])
        assert np.array_equal(odC.numpy(), ref["dE_dC"])
    # E alone; a staging buffer that is too small is refused before any device work
    oE.zero_()
    dn.donof_energy_lagrangian_host(b.prob, h, b.B, hC, hg, pm, b.ws, staging, oE)
    assert oE.item() == ref["E"]
    rc = dn.binding.lib().donof_energy_lagrangian_host(
        ctypes.byref(b.prob), ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(b.B.data_ptr()),
        ctypes.c_void_p(hC.data_ptr()), ctypes.c_void_p(hg.data_ptr()),
        ctypes.c_void_p(pm.data_ptr()), ctypes.c_void_p(b.ws.data_ptr()), b.ws.numel(),
        ctypes.c_void_p(staging.data_ptr()), 256, ctypes.c_void_p(oE.data_ptr()), None, None,
        None, None)
    assert rc == -4  # DONOF_ERR_WORKSPACE
