"""Shared test plumbing: run one build through the C ABI and return numpy results."""
from __future__ import annotations

import numpy as np

import synth


def to_dev(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def gpu_build(prob: synth.Problem, d: dict, precision: int, functional: int, packed: bool = False,
              budget: int = 0, B=None, backward: bool = True):
    import torch
    import paper_2004_06142_gb300 as dn
    Bh = d["B"] if B is None else B
    if packed and Bh.ndim == 3:
        mu, nu = synth.packed_index(prob.nbf)
        Bh = np.ascontiguousarray(Bh[:, mu, nu])
    b = dn.Builder(prob.nbf, prob.naux, prob.npair, prob.ncwo, functional,
                   dn.B_PACKED if packed else dn.B_DENSE, precision, budget,
                   nsingle=prob.nsingle)
    Bd = to_dev(Bh)
    b.prepare(Bd)
    h, C = to_dev(d["h"]), to_dev(d["C"])
    g = to_dev(d["gamma"])
    pm = to_dev(d["pair_map"].astype(np.int32))
    E, lam, dEdg = b.forward(h, C, g, pm)
    out = dict(E=E.item(), lam=lam.cpu().numpy(), dE_dgamma=dEdg.cpu().numpy())
    J, K = b.jk()
    out["J"], out["K"] = J.cpu().numpy(), K.cpu().numpy()
    if backward:
        Ebar = torch.ones(1, dtype=torch.float64, device="cuda")
        dC, dg = b.backward(Ebar)
        out["dE_dC"] = dC.cpu().numpy()
        out["dE_dgamma_bwd"] = dg.cpu().numpy()
    out["status"] = b.status()
    return out
