"""The host side of the build sharded over the auxiliary index (CPU, gloo, world size 2 and
3): every rank takes the slices shard_range gives it, forms its partial sums (J, K and the
two-electron part of G, laid out as donof_energy_lagrangian_partial writes them), the
binding's exchange sums them over the ranks, and every rank finishes.  The partial sums and
the finish are the FP64 oracle's (Sec. III.D: J^q, K^q of Eq. Gpmn, and with them J, K and
G, are sums over the auxiliary index), so the summed result must be the one-pass oracle
build; the CUDA entry points themselves are checked against this on the GPU
(test_gpu_sharded.py)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

import synth
from oracle import pnof
from paper_2004_06142_gb300 import binding

SHAPE = (13, 29, 2, 2)   # nbf, naux, npair, ncwo: naux odd, so the shards are uneven


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def oracle_partial(d, prob, P0, P1):
    """J, K and the two-electron G of slices [P0, P1), flattened in the library's order."""
    Ca = d["C"][:, :prob.nact]
    occ = pnof.occupations(d["gamma"], d["pair_map"], prob.npair, prob.ncwo)
    Jq, Kq = pnof.ao_operators(d["B"][P0:P1], Ca)
    J, K = pnof.mo_jk(Ca, Jq, Kq)
    G2 = pnof.generalized_fock_action(np.zeros_like(d["h"]), Ca, Jq, Kq, occ, d["pair_map"],
                                      prob.npair, pnof.PNOF7)
    return np.concatenate([J.ravel(), K.ravel(), G2.ravel()])


def oracle_finish(d, prob, partial):
    """E and lambda from summed partial sums (the oracle's steps after its sums over P)."""
    A, N = prob.nact, prob.nbf
    J = partial[:A * A].reshape(A, A)
    K = partial[A * A:2 * A * A].reshape(A, A)
    G2 = partial[2 * A * A:].reshape(N, A)
    Ca = d["C"][:, :A]
    occ = pnof.occupations(d["gamma"], d["pair_map"], prob.npair, prob.ncwo)
    Hd = np.einsum("mp,mn,np->p", Ca, d["h"], Ca)
    E = pnof.energy(Hd, J, K, occ, d["pair_map"], prob.npair, pnof.PNOF7)
    G = occ["n"][None, :] * (d["h"] @ Ca) + G2
    return E, d["C"].T @ G


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        prob = synth.Problem(*SHAPE, seed=7)
        d = synth.generate(prob)
        P0, P1 = binding.shard_range(prob.naux, rank, ws)
        part = torch.from_numpy(oracle_partial(d, prob, P0, P1))
        mine = part.clone()
        binding.exchange_partial(part)
        E, lam = oracle_finish(d, prob, part.numpy())
        out[rank] = (P0, P1, mine.numpy(), part.numpy(), E, lam)
    finally:
        tdist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_sharded_build_on_gloo_ranks_is_the_full_build(ws):
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
    prob = synth.Problem(*SHAPE, seed=7)
    d = synth.generate(prob)
    ref = pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], prob.npair, prob.ncwo,
                     pnof.PNOF7)
    # the shards cover the auxiliary index once, in order
    ranges = [out[r][:2] for r in range(ws)]
    assert ranges[0][0] == 0 and ranges[-1][1] == prob.naux
    assert all(ranges[r][1] == ranges[r + 1][0] for r in range(ws - 1))
    assert max(b - a for a, b in ranges) - min(b - a for a, b in ranges) <= 1
    # after the exchange every rank holds the sum of all shards' partials
    total = sum(out[r][2] for r in range(ws))
    for r in range(ws):
        np.testing.assert_allclose(out[r][3], total, rtol=0, atol=1e-14)
        assert abs(out[r][4] - ref["E"]) <= 1e-11
        np.testing.assert_allclose(out[r][5], ref["lam"][:, :prob.nact], rtol=0, atol=1e-12)


def test_exchange_is_a_no_op_without_a_group():
    x = torch.arange(5, dtype=torch.float64)
    assert binding.exchange_partial(x) is x
    assert torch.equal(x, torch.arange(5, dtype=torch.float64))
