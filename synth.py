"""Seeded synthetic inputs for the PNOF energy / orbital-Lagrangian build.

This module only draws inputs; it holds none of the method's arithmetic.  The
CUDA path and the FP64 oracle both consume the arrays it returns.

Workload recipe (the shapes of the paper's problem, Sec. III.D: an AO basis of
N_B functions, MO coefficients C, occupations parametrised by gamma, Eqs.
soo/woo), drawn with numpy's PCG64 ``default_rng``:

* ``B[P, mu, nu] = sym(g^P)[mu, nu] * exp(-|mu - nu| / 4) / sqrt(naux)`` with
  ``g^P ~ N(0, 1)`` drawn from its own stream ``default_rng([seed, 0, P])`` and
  ``sym(g) = (g + g^T) / 2``.  Each auxiliary slice has its own stream so any
  slice can be regenerated alone and large cases generate in parallel.
* ``h`` symmetric: upper triangle ``N(0, 0.1) * exp(-|mu - nu| / 4)`` mirrored,
  diagonal ``-U(1, 10)``; stream ``[seed, 1]``.
* ``C = Q`` of ``QR(N(0, 1))`` (nbf x nbf), stream ``[seed, 2]``.
* strong ``gamma_g ~ U(0, 1.45)``; the hole ``1 - n_g`` of pair g is split over
  its weak orbitals by ``Dirichlet(1, ..., 1)``; the weak gammas are the
  inverse of Eq. woo for that split.  Stream ``[seed, 3]``.
* ``pair_map``: strong orbital g at index g, the ``nsingle`` singly occupied orbitals
  of a multiplet at ``npair .. npair + nsingle - 1`` (their own subspaces, pair_map[g] =
  g), weak orbital i of pair g at index ``npair + nsingle + g * ncwo + i`` (block layout).
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

# The five workloads: (name, nbf, naux, npair, ncwo, b_layout).
CONFIGS = {
    "plain": dict(nbf=24, naux=96, npair=5, ncwo=1, packed=False),
    "differentiation": dict(nbf=120, naux=480, npair=8, ncwo=4, packed=False),
    "precision": dict(nbf=500, naux=2000, npair=20, ncwo=3, packed=False),
    "large": dict(nbf=1200, naux=4800, npair=50, ncwo=2, packed=True),
}


@dataclass
class Problem:
    nbf: int
    naux: int
    npair: int
    ncwo: int
    seed: int = 0
    nsingle: int = 0  # singly occupied orbitals (Omega_I), at npair .. npair + nsingle - 1

    @property
    def nact(self) -> int:
        return self.npair * (1 + self.ncwo) + self.nsingle

    @property
    def ngamma(self) -> int:
        return self.npair * self.ncwo


def _band(nbf: int) -> np.ndarray:
    idx = np.arange(nbf)
    return np.exp(-np.abs(idx[:, None] - idx[None, :]) / 4.0)


def b_slice(seed: int, naux: int, nbf: int, P: int, band: np.ndarray | None = None) -> np.ndarray:
    """One auxiliary slice B[P] (nbf x nbf, symmetric, float64)."""
    if band is None:
        band = _band(nbf)
    g = np.random.default_rng([seed, 0, P]).standard_normal((nbf, nbf))
    return 0.5 * (g + g.T) * band / math.sqrt(naux)


def packed_index(nbf: int):
    """Row/column index arrays of the packed lower triangle, mu >= nu, at mu*(mu+1)/2 + nu."""
    mu, nu = np.tril_indices(nbf)
    return mu, nu


def gen_B(seed: int, naux: int, nbf: int, packed: bool = False, p0: int = 0, p1: int | None = None,
          threads: int | None = None) -> np.ndarray:
    """Slices p0..p1 of B, dense [n][nbf][nbf] or packed [n][nbf(nbf+1)/2]."""
    if p1 is None:
        p1 = naux
    band = _band(nbf)
    npk = nbf * (nbf + 1) // 2
    out = np.empty((p1 - p0, npk) if packed else (p1 - p0, nbf, nbf))
    mu, nu = packed_index(nbf) if packed else (None, None)

    def work(P):
        s = b_slice(seed, naux, nbf, P, band)
        if packed:
            out[P - p0] = s[mu, nu]
        else:
            out[P - p0] = s

    nthr = threads or min(16, os.cpu_count() or 1)
    if p1 - p0 <= 4 or nthr == 1:
        for P in range(p0, p1):
            work(P)
    else:
        with ThreadPoolExecutor(nthr) as ex:
            list(ex.map(work, range(p0, p1)))
    return out


def gen_h(seed: int, nbf: int) -> np.ndarray:
    rng = np.random.default_rng([seed, 1])
    off = rng.normal(0.0, 0.1, size=(nbf, nbf)) * _band(nbf)
    h = np.triu(off, 1)
    h = h + h.T
    h[np.diag_indices(nbf)] = -rng.uniform(1.0, 10.0, size=nbf)
    return h


def gen_C(seed: int, nbf: int) -> np.ndarray:
    rng = np.random.default_rng([seed, 2])
    q, _ = np.linalg.qr(rng.standard_normal((nbf, nbf)))
    return np.ascontiguousarray(q)


def block_pair_map(npair: int, ncwo: int, nsingle: int = 0) -> np.ndarray:
    pm = np.empty(npair * (1 + ncwo) + nsingle, dtype=np.int32)
    pm[:npair + nsingle] = np.arange(npair + nsingle)
    w0 = npair + nsingle
    for g in range(npair):
        pm[w0 + g * ncwo: w0 + (g + 1) * ncwo] = g
    return pm


def gen_gamma(seed: int, npair: int, ncwo: int) -> np.ndarray:
    """gamma[0:npair] strong, then (ncwo-1) weak gammas per pair, pair-major."""
    rng = np.random.default_rng([seed, 3])
    gs = rng.uniform(0.0, 1.45, size=npair)
    gam = np.zeros(npair * ncwo)
    gam[:npair] = gs
    if ncwo > 1:
        for g in range(npair):
            hole = 0.5 * math.sin(gs[g]) ** 2
            split = rng.dirichlet(np.ones(ncwo)) * hole
            rest = hole
            for i in range(ncwo - 1):
                ratio = min(1.0, max(0.0, split[i] / rest)) if rest > 0 else 0.0
                gi = math.asin(math.sqrt(ratio))
                gam[npair + g * (ncwo - 1) + i] = gi
                rest *= math.cos(gi) ** 2
    return gam


def generate(prob: Problem, packed: bool = False, with_B: bool = True) -> dict:
    """All inputs of one instance as float64 / int32 numpy arrays."""
    d = dict(
        h=gen_h(prob.seed, prob.nbf),
        C=gen_C(prob.seed, prob.nbf),
        gamma=gen_gamma(prob.seed, prob.npair, prob.ncwo),
        pair_map=block_pair_map(prob.npair, prob.ncwo, prob.nsingle),
    )
    if with_B:
        d["B"] = gen_B(prob.seed, prob.naux, prob.nbf, packed=packed)
    return d


def batch_problems(ninst: int = 64, seed0: int = 0) -> list[Problem]:
    """The dissociation-scan-shaped batch: instance i has seed i,
    nbf ~ U{40..240}, naux = 4 nbf, 5 pairs, ncwo ~ U{1..4} (sizes from stream [i, 4])."""
    out = []
    for i in range(seed0, seed0 + ninst):
        rng = np.random.default_rng([i, 4])
        nbf = int(rng.integers(40, 241))
        ncwo = int(rng.integers(1, 5))
        out.append(Problem(nbf=nbf, naux=4 * nbf, npair=5, ncwo=ncwo, seed=i))
    return out


def config_problem(name: str, seed: int = 0) -> tuple[Problem, bool]:
    c = CONFIGS[name]
    return Problem(c["nbf"], c["naux"], c["npair"], c["ncwo"], seed), c["packed"]
