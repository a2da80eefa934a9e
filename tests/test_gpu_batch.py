"""Batched builds (donof_energy_lagrangian_batched) on instances of the dissociation-scan
workload: uneven nbf in 40..240, naux = 4 nbf, 5 pairs, Ncwo in 1..4, one seed per instance.

The grouped path (one launch per step of the build for all instances) and the per-instance
stream path run the same kernel bodies, so they must agree bit for bit, with and without
CUDA-graph capture/replay; every instance must reproduce the single-instance entry point
(the same kernels, every sum in a fixed order) and the oracle within the parity tolerances.
"""
import numpy as np
import pytest

import synth
from oracle import pnof

pytestmark = pytest.mark.gpu

KEYS = ("E", "lam", "dE_dgamma", "dE_dC")


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


def _run(batch, tens, flags):
    import torch
    for x in tens:
        for k in KEYS:
            x[k].fill_(np.nan)
    batch.run(flags)
    torch.cuda.synchronize()
    return [{k: x[k].cpu().numpy().copy() for k in KEYS} for x in tens]


@pytest.mark.parametrize("precision", [1, 0])
def test_batched_matches_single_and_oracle(precision):
    import torch
    import paper_2004_06142_gb300 as dn
    probs = synth.batch_problems(64 if precision else 8)
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
        single.append(dict(E=E.cpu().numpy(), lam=lam.cpu().numpy(), dE_dgamma=dg.cpu().numpy(),
                           dE_dC=dC.cpu().numpy()))
        del b
    BW, GR, ST = dn.BATCH_BACKWARD, dn.BATCH_GRAPH, dn.BATCH_STREAMS
    runs = [_run(batch, tens, f) for f in (BW, BW | GR, BW | GR, BW | ST, BW | ST | GR)]
    assert batch.status() == 0
    for out in runs:
        for s, o in zip(single, out):
            for k in KEYS:
                np.testing.assert_array_equal(o[k], s[k], err_msg=k)
    # every instance against the oracle
    tol_e, tol_a = (1e-6, 1e-5) if precision else (1e-10, 1e-10)
    for pr, d, o in zip(probs, host, runs[0]):
        ref = pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], pr.npair, pr.ncwo,
                         pnof.PNOF7)
        assert abs(o["E"][0] - ref["E"]) <= tol_e, (pr, o["E"][0] - ref["E"])
        for k in ("lam", "dE_dgamma", "dE_dC"):
            assert np.abs(o[k] - ref[k]).max() <= tol_a, (pr, k)


def test_grouped_launch_count():
    # the grouped path: one launch per step of the build for all instances
    import paper_2004_06142_gb300 as dn
    probs = synth.batch_problems(12)
    cprobs, tens, _ = _instances(probs, 1)
    batch = dn.Batch(cprobs, tens)
    batch.prepare()
    batch.run(dn.BATCH_BACKWARD)
    n0 = dn.donof_launch_count()
    batch.run(dn.BATCH_BACKWARD)
    grouped = dn.donof_launch_count() - n0
    n0 = dn.donof_launch_count()
    batch.run(dn.BATCH_BACKWARD | dn.BATCH_STREAMS)
    streams = dn.donof_launch_count() - n0
    assert grouped == 24
    assert streams == 12 * 25
