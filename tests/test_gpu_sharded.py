"""The build sharded over the auxiliary index (donof_energy_lagrangian_partial / _finish) on
one GPU: the shards run one after the other, each on its own slices of B and its own
workspace, their partial sums are added on the device (what the all-reduce does across
GPUs), and the finish must reproduce the oracle and the one-pass build within the parity
tolerances, the adjoint included; every shard's finish gives the same result."""
import numpy as np
import pytest

import synth
from oracle import pnof

from helpers import to_dev

pytestmark = pytest.mark.gpu

TOL = {0: (1e-10, 1e-10), 1: (1e-6, 1e-5)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_06142_gb300.build as b
    b.build()


def _sharded(dn, prob, Bd, layout, precision, nshard, h, C, g, pm):
    import torch
    builders, partial = [], None
    for r in range(nshard):
        P0, P1 = dn.shard_range(prob.naux, r, nshard)
        b = dn.Builder(prob.nbf, P1 - P0, prob.npair, prob.ncwo, dn.PNOF7, layout, precision)
        b.prepare(Bd[P0:P1].contiguous())
        part = b.forward_partial(h, C, g, pm)
        partial = part.clone() if partial is None else partial + part
        builders.append(b)
    outs = []
    one = torch.ones(1, dtype=torch.float64, device="cuda")
    for b in builders:
        E, lam, dg = b.finish(h, C, g, pm, partial)
        dC, _ = b.backward(one)
        J, K = b.jk()
        assert b.status() == 0
        outs.append(dict(E=E.item(), lam=lam.cpu().numpy(), dE_dgamma=dg.cpu().numpy(),
                         dE_dC=dC.cpu().numpy(), J=J.cpu().numpy(), K=K.cpu().numpy()))
    return outs


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape,packed,nshard", [((97, 150, 4, 3), False, 2),
                                                 ((130, 257, 6, 4), True, 3)],
                         ids=["dense-2", "packed-3"])
def test_sharded_build_matches_oracle_and_full_build(precision, shape, packed, nshard):
    import torch
    import paper_2004_06142_gb300 as dn
    prob = synth.Problem(*shape, seed=11)
    d = synth.generate(prob)
    ref = pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], prob.npair, prob.ncwo,
                     pnof.PNOF7)
    Bh = d["B"]
    if packed:
        mu, nu = synth.packed_index(prob.nbf)
        Bh = np.ascontiguousarray(Bh[:, mu, nu])
    layout = dn.B_PACKED if packed else dn.B_DENSE
    Bd = to_dev(Bh)
    h, C, g = to_dev(d["h"]), to_dev(d["C"]), to_dev(d["gamma"])
    pm = to_dev(d["pair_map"].astype(np.int32))
    outs = _sharded(dn, prob, Bd, layout, precision, nshard, h, C, g, pm)
    # the one-pass build on all slices
    full = dn.Builder(prob.nbf, prob.naux, prob.npair, prob.ncwo, dn.PNOF7, layout, precision)
    full.prepare(Bd)
    E, lam, dg = full.forward(h, C, g, pm)
    dC, _ = full.backward(torch.ones(1, dtype=torch.float64, device="cuda"))
    assert full.status() == 0
    tol_e, tol_a = TOL[precision]
    for o in outs:
        # every shard's finish is the same computation on the same summed partial sums
        assert o["E"] == outs[0]["E"]
        np.testing.assert_array_equal(o["lam"], outs[0]["lam"])
        assert abs(o["E"] - ref["E"]) <= tol_e
        assert abs(o["E"] - E.item()) <= tol_e
        for k in ("lam", "dE_dgamma", "dE_dC", "J", "K"):
            assert np.abs(o[k] - ref[k]).max() <= tol_a, k
        for k, v in (("lam", lam), ("dE_dgamma", dg), ("dE_dC", dC)):
            assert np.abs(o[k] - v.cpu().numpy()).max() <= tol_a, k


def test_large_workload_in_two_shards_against_oracle():
    # the large workload (nbf 1200, naux 4800, packed B, mixed) as two shards of 2400 slices,
    # the launch configuration of two GPUs, against the stored oracle values
    import torch
    import paper_2004_06142_gb300 as dn
    from test_gpu_fullsize import _upload_B, load_large_golden
    prob, packed = synth.config_problem("large")
    N, A = prob.nbf, prob.nact
    ref = load_large_golden(prob.seed)
    d = synth.generate(prob, with_B=False)
    dev = torch.device("cuda")
    B = _upload_B(prob, packed, dev)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    h, C, g = t(d["h"]), t(d["C"]), t(d["gamma"])
    pm = t(d["pair_map"].astype(np.int32))
    outs = _sharded(dn, prob, B, dn.B_PACKED, dn.MIXED, 2, h, C, g, pm)
    o = outs[0]
    assert abs(o["E"] - ref["E"][0]) <= 1e-6
    assert np.abs(o["dE_dgamma"] - ref["dE_dgamma"]).max() <= 1e-5
    assert np.abs(o["lam"][:, :A] - ref["lam_act"]).max() <= 1e-5
    assert np.abs(o["dE_dC"][:, :A] - ref["dE_dC_act"]).max() <= 1e-5
    assert np.abs(o["J"] - ref["J"]).max() <= 1e-6 * np.abs(ref["J"]).max()
    assert np.abs(o["K"] - ref["K"]).max() <= 1e-6 * np.abs(ref["K"]).max()
