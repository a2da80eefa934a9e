"""The oracle's occupation map against the occupation numbers the paper prints for water
(Table ONs, Sec. "Illustrative example: water molecule"; fixture
tests/golden/water_ons_table.txt, 2n to three decimals, 5 pairs with N_g = 4).

The printed numbers come from converged calculations on real integrals, which are not
available here, so they pin what holds for any PNOF solution:
  * Eq. sum1 per pair: the strong orbital and its four weak orbitals hold 2n = 2 — the table
    admits a pairing of its weak MOs under which every pair sums to 2 in all six columns;
  * Eqs. soo, woo: with gamma recovered from the printed numbers by inverting the two
    equations as the paper states them (strong: n_g = (1 + cos^2 gamma_g) / 2; weak, in
    index order: n_i = h_g cos^2 gamma_1 ... cos^2 gamma_(i-1) sin^2 gamma_i, the last one
    without sin^2), the oracle's occupations reproduce the table;
  * Eq. sumNp: the oracle's occupations of those gamma add up to N/2 = 5.
"""
import math
import os

import numpy as np

from oracle import pnof

HERE = os.path.dirname(os.path.abspath(__file__))
NPAIR, NCWO = 5, 4
HALF_UNIT = 0.0005  # half a unit of the printed third decimal (2n)


def load_table():
    rows = []
    with open(os.path.join(HERE, "golden", "water_ons_table.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(x) for x in line.split()[1:]])
    return np.array(rows)  # (25 MOs, 6 columns) of 2n


def find_pairing(T):
    """Weak MOs (indices NPAIR..) into NPAIR groups of NCWO, group g for strong MO g, such that
    each pair's 2n sum to 2 in every column within the rounding of its five printed entries.
    Depth-first, the largest entries placed first; None if no pairing exists."""
    tol = (1 + NCWO) * HALF_UNIT + 1e-9
    weak = sorted(range(NPAIR, T.shape[0]), key=lambda w: -T[w].max())
    groups = [[] for _ in range(NPAIR)]
    sums = [T[g].copy() for g in range(NPAIR)]

    def place(i):
        if i == len(weak):
            return all(np.all(np.abs(s - 2.0) <= tol) for s in sums)
        w = weak[i]
        for g in range(NPAIR):
            if len(groups[g]) == NCWO:
                continue
            s = sums[g] + T[w]
            if np.any(s > 2.0 + tol):
                continue
            groups[g].append(w)
            sums[g] = s
            if place(i + 1):
                return True
            groups[g].pop()
            sums[g] = s - T[w]
        return False

    return [sorted(g) for g in groups] if place(0) else None


def gammas_from_ons(n, groups):
    """gamma from per-spin occupations n by inverting Eqs. soo and woo.  The printed weak
    numbers of a pair are first scaled to add up to the pair's hole h_g = 1 - n_g (they
    differ from it by rounding only)."""
    gamma = np.zeros(NPAIR + NPAIR * (NCWO - 1))
    for g in range(NPAIR):
        c2 = min(max(2.0 * n[g] - 1.0, 0.0), 1.0)
        gamma[g] = math.acos(math.sqrt(c2))
        h = 1.0 - n[g]
        nw = np.array([n[w] for w in groups[g]])
        nw = nw * (h / nw.sum()) if nw.sum() > 0 else np.full(NCWO, h / NCWO)
        r = h
        for i in range(NCWO - 1):
            s2 = min(max(nw[i] / r, 0.0), 1.0) if r > 0 else 0.0
            gamma[NPAIR + g * (NCWO - 1) + i] = math.asin(math.sqrt(s2))
            r = max(r - nw[i], 0.0)
    return gamma


def test_table_admits_a_pairing_with_the_pair_sum_rule():
    T = load_table()
    assert T.shape == (NPAIR * (1 + NCWO), 6)
    # every column holds the 10 electrons of water (Eq. sumNp), within rounding
    np.testing.assert_allclose(T.sum(axis=0), 10.0, atol=T.shape[0] * HALF_UNIT)
    groups = find_pairing(T)
    assert groups is not None
    assert sorted(w for g in groups for w in g) == list(range(NPAIR, T.shape[0]))


def test_oracle_occupations_reproduce_the_printed_numbers():
    T = load_table()
    groups = find_pairing(T)
    pair_map = np.zeros(T.shape[0], dtype=np.int64)
    for g in range(NPAIR):
        pair_map[g] = g
        for w in groups[g]:
            pair_map[w] = g
    tol_weak = (1 + NCWO) * HALF_UNIT + HALF_UNIT
    for col in range(T.shape[1]):
        n_printed = T[:, col] / 2.0
        gamma = gammas_from_ons(n_printed, groups)
        n = pnof.occupations(gamma, pair_map, NPAIR, NCWO)["n"]
        # strong orbitals: the inverse is exact
        np.testing.assert_allclose(2.0 * n[:NPAIR], T[:NPAIR, col], rtol=0, atol=1e-12)
        # weak orbitals: within the rounding redistributed by the scaling to h_g
        np.testing.assert_allclose(2.0 * n[NPAIR:], T[NPAIR:, col], rtol=0, atol=tol_weak)
        # Eq. sumNp for the oracle's occupations of these gamma
        assert abs(n.sum() - NPAIR) < 1e-12
