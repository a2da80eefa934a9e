"""Writes the FP64 oracle's values for the large workload (tests/golden/large_seed0.npz).

    python tests/golden/make_large_golden.py [--seed 0] [--block 240]

The large workload: nbf 1200, naux 4800, 50 pairs, Ncwo 2 (150 active orbitals), PNOF7,
the seeded synthetic inputs of synth.py.  Dense B would take 55 GB, so the oracle runs its
operator route streamed over blocks of auxiliary slices (oracle.pnof.build_streamed: the
AO operators J^q, K^q of Eq. Gpmn are sums over P, accumulated block by block; J, K, E,
G, lambda and dE/dgamma then follow as in a plain build).  Only oracle/ and synth.py are
used: no value comes from the CUDA library.

Stored (float64): E; dE_dgamma[100]; J, K [150][150]; lam_act = lambda[:, :150] and
dE_dC_act = dE/dC[:, :150] (columns p >= nact of both are zero by definition).
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import pnof  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--block", type=int, default=240)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    prob, _ = synth.config_problem("large", seed=args.seed)
    N, Q, A = prob.nbf, prob.naux, prob.nact
    d = synth.generate(prob, with_B=False)

    def blocks():
        for p0 in range(0, Q, args.block):
            yield synth.gen_B(prob.seed, Q, N, packed=False, p0=p0, p1=min(Q, p0 + args.block))

    t0 = time.time()
    ref = pnof.build_streamed(d["h"], blocks(), d["C"], d["gamma"], d["pair_map"], prob.npair,
                              prob.ncwo, pnof.PNOF7,
                              on_block=lambda n: print(f"  {n}/{Q} slices, {time.time() - t0:.0f} s",
                                                       flush=True))
    out = args.out or os.path.join(HERE, f"large_seed{args.seed}.npz")
    np.savez_compressed(out, E=np.array([ref["E"]]), dE_dgamma=ref["dE_dgamma"], J=ref["J"],
                        K=ref["K"], lam_act=ref["lam"][:, :A], dE_dC_act=ref["dE_dC"][:, :A],
                        shape=np.array([N, Q, prob.npair, prob.ncwo, args.seed]))
    sha = hashlib.sha256(open(out, "rb").read()).hexdigest()
    print(f"E = {ref['E']!r}; wrote {out} (sha256 {sha}) in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
