"""Batched builds (donof_energy_lagrangian_batched) on instances of the dissociation-scan
workload: uneven nbf in 40..240, naux = 4 nbf, 5 pairs, Ncwo in 1..4, one seed per instance.

Every instance of a batched call must reproduce the single-instance entry point (the same
kernels, every sum in a fixed order) and the oracle within the parity tolerances, with and
without CUDA-graph capture/replay.
"""
import numpy as np
import pytest

import synth
from oracle import pnof

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_06142_gb300.build as b
    b.build()


def _instances(probs, precision):
    import torch
    import paper_2004_06142_gb300 as dn
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    cprobs, tens, host = [], [], []
    for pr in probs:
        d = synth.generate(pr)
        host.append(d)
        cprobs.append(dn.make_problem(pr.nbf, pr.naux, pr.npair, pr.ncwo, dn.PNOF7, dn.B_DENSE,
                                      precision))
        f64 = torch.float64
        tens.append(dict(h=t(d["h"]), B=t(d["B"]), C=t(d["C"]), gamma=t(d["gamma"]),
                         pair_map=t(d["pair_map"].astype(np.int32)),
                         E=torch.empty(1, dtype=f64, device="cuda"),
                         lam=torch.empty(pr.nbf, pr.nbf, dtype=f64, device="cuda"),
                         dE_dgamma=torch.empty(pr.ngamma, dtype=f64, device="cuda"),
                         dE_dC=torch.empty(pr.nbf, pr.nbf, dtype=f64, device="cuda")))
    return cprobs, tens, host


@pytest.mark.parametrize("precision", [1, 0])
def test_batched_matches_single_and_oracle(precision):
    import torch
    import paper_2004_06142_gb300 as dn
    probs = synth.batch_problems(10 if precision else 5)
    cprobs, tens, host = _instances(probs, precision)
    batch = dn.Batch(cprobs, tens)
    batch.prepare()
    # single-instance reference results through the regular entry points
    single = []
    one = torch.ones(1, dtype=torch.float64, device="cuda")
    for pr, x in zip(probs, tens):
        b = dn.Builder(pr.nbf, pr.naux, pr.npair, pr.ncwo, dn.PNOF7, dn.B_DENSE, precision)
        b.prepare(x["B"])
        E, lam, dg = b.forward(x["h"], x["C"], x["gamma"], x["pair_map"])
        dC, _ = b.backward(one)
        single.append(dict(E=E.item(), lam=lam.cpu().numpy(), dE_dgamma=dg.cpu().numpy(),
                           dE_dC=dC.cpu().numpy()))
    tol_e, tol_a = (1e-6, 1e-5) if precision else (1e-10, 1e-10)
    for flags in (dn.BATCH_BACKWARD, dn.BATCH_BACKWARD | dn.BATCH_GRAPH,
                  dn.BATCH_BACKWARD | dn.BATCH_GRAPH):
        for x in tens:
            for k in ("E", "lam", "dE_dgamma", "dE_dC"):
                x[k].fill_(np.nan)
        batch.run(flags)
        torch.cuda.synchronize()
        for s, x in zip(single, tens):
            assert abs(x["E"].item() - s["E"]) <= 1e-9
            for k in ("lam", "dE_dgamma", "dE_dC"):
                assert np.abs(x[k].cpu().numpy() - s[k]).max() <= 1e-8, k
    # the oracle, on a few instances of the batch
    for i in (0, len(probs) // 2, len(probs) - 1):
        pr, d, x = probs[i], host[i], tens[i]
        ref = pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], pr.npair, pr.ncwo,
                         pnof.PNOF7)
        assert abs(x["E"].item() - ref["E"]) <= tol_e
        assert np.abs(x["lam"].cpu().numpy() - ref["lam"]).max() <= tol_a
        assert np.abs(x["dE_dgamma"].cpu().numpy() - ref["dE_dgamma"]).max() <= tol_a
        assert np.abs(x["dE_dC"].cpu().numpy() - ref["dE_dC"]).max() <= tol_a
