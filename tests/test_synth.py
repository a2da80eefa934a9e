"""The seeded input recipe (synth.py) has the structure the design states: symmetric B slices
with a banded envelope, one random stream per slice (any slice regenerates alone, dense and
packed agree), symmetric h with a negative diagonal, orthogonal C, strong gamma in
[0, 1.45], the block pair_map, and reproducible draws."""
import numpy as np

import synth


def test_b_slices_symmetric_reproducible_and_independent():
    naux, nbf = 7, 13
    B = synth.gen_B(3, naux, nbf)
    assert B.shape == (naux, nbf, nbf)
    np.testing.assert_array_equal(B, np.transpose(B, (0, 2, 1)))
    np.testing.assert_array_equal(B, synth.gen_B(3, naux, nbf))        # same seed, same B
    assert not np.array_equal(B, synth.gen_B(4, naux, nbf))             # another seed
    np.testing.assert_array_equal(synth.gen_B(3, naux, nbf, p0=2, p1=5), B[2:5])
    np.testing.assert_array_equal(synth.gen_B(3, naux, nbf, threads=1), B)
    Bp = synth.gen_B(3, naux, nbf, packed=True)
    mu, nu = synth.packed_index(nbf)
    assert Bp.shape == (naux, nbf * (nbf + 1) // 2)
    np.testing.assert_array_equal(Bp, B[:, mu, nu])
    assert np.all(mu * (mu + 1) // 2 + nu == np.arange(Bp.shape[1]))   # mu*(mu+1)/2 + nu
    # the envelope: far from the diagonal the entries are small against the near ones
    far = np.abs(B[:, 0, -1]).max()
    near = np.abs(B[:, np.arange(nbf), np.arange(nbf)]).max()
    assert far < 0.1 * near


def test_h_c_gamma_and_pair_map():
    prob = synth.Problem(40, 8, 6, 3, seed=5)
    d = synth.generate(prob, with_B=False)
    h, C, gamma, pm = d["h"], d["C"], d["gamma"], d["pair_map"]
    np.testing.assert_array_equal(h, h.T)
    assert np.all(np.diag(h) <= -1.0) and np.all(np.diag(h) >= -10.0)
    np.testing.assert_allclose(C.T @ C, np.eye(40), atol=1e-12)
    assert gamma.shape == (prob.ngamma,)
    assert np.all((gamma[:6] >= 0.0) & (gamma[:6] <= 1.45))
    assert np.all((gamma[6:] >= 0.0) & (gamma[6:] <= np.pi / 2))
    assert pm.dtype == np.int32 and pm.shape == (prob.nact,)
    np.testing.assert_array_equal(pm[:6], np.arange(6))
    np.testing.assert_array_equal(pm[6:], np.repeat(np.arange(6), 3))
    again = synth.generate(prob, with_B=False)
    for k in d:
        np.testing.assert_array_equal(d[k], again[k])


def test_pair_map_with_singles_and_batch_sizes():
    pm = synth.block_pair_map(3, 2, nsingle=2)
    np.testing.assert_array_equal(pm, [0, 1, 2, 3, 4, 0, 0, 1, 1, 2, 2])
    probs = synth.batch_problems(64)
    assert [p.seed for p in probs] == list(range(64))
    assert all(40 <= p.nbf <= 240 and p.naux == 4 * p.nbf and p.npair == 5
               and 1 <= p.ncwo <= 4 for p in probs)
    assert [(p.nbf, p.ncwo) for p in probs] == [(p.nbf, p.ncwo) for p in synth.batch_problems(64)]
