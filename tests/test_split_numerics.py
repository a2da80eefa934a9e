"""The arithmetic of the mixed path's operand splits, emulated on the CPU (numpy), on the
large workload's h and C_act (nbf 1200, nact 150):

  * integer + fraction split of a row x: y = x / 2^e, h = fp16(rint(y)), f = fp16(y - h),
    e the smallest exponent with ||y||_2 < 4096 - sqrt(K)/2 - 2.  Then ||h||_2 < 2^12, so by
    Cauchy-Schwarz every partial sum of h_a . h_b stays below 2^24 and the integer products
    accumulate exactly in fp32, in any order;
  * one split per operand leaves h C_act (and so 2 sum n_p H_pp) with the fraction's
    rounding error, relative ~2^-25 of the row norms: too coarse next to a dominant h;
  * with the residual r = fp16(y - h - f) and the product taken as four K blocks,
    h_U h_V + h_U (r_V + f_V) + f_U (h_V + f_V) + r_U (h_V + f_V), each block in fp32 and
    the blocks added in double, the one-electron energy comes out near double precision.

This checks the arithmetic the kernels are built on, not the kernels (the GPU parity tests
do that); the limits asserted here are the ones the kernels' design relies on.
"""
import math

import numpy as np

import synth
from oracle import pnof

F16, F32 = np.float16, np.float32


def exponents(M, K):
    T = 4096.0 - 0.5 * math.sqrt(K) - 2.0
    nrm = np.sqrt((M * M).sum(axis=1))
    e = np.ceil(np.log2(nrm / T)).astype(int)
    e = np.where(nrm / np.ldexp(1.0, e) >= T, e + 1, e)
    return e


def split(M, e):
    y = M / np.ldexp(1.0, e)[:, None]
    h = np.rint(y).astype(F16).astype(np.float64)
    f = (y - h).astype(F16).astype(np.float64)
    r = (y - h - f).astype(F16).astype(np.float64)
    return y, h, f, r


def large_h_and_c():
    prob = synth.Problem(1200, 8, 50, 2, seed=0)
    d = synth.generate(prob, with_B=False)
    A = prob.npair * (1 + prob.ncwo)
    n = pnof.occupations(d["gamma"], d["pair_map"], prob.npair, prob.ncwo)["n"]
    return d["h"], d["C"][:, :A], n


def test_integer_parts_accumulate_exactly_in_fp32():
    h, Ca, _ = large_h_and_c()
    K = h.shape[1]
    ea, eb = exponents(h, K), exponents(Ca.T, K)
    _, ha, _, _ = split(h, ea)
    _, hb, _, _ = split(Ca.T, eb)
    na = np.sqrt((ha * ha).sum(1))
    nb = np.sqrt((hb * hb).sum(1))
    assert na.max() < 2.0 ** 12 and nb.max() < 2.0 ** 12
    assert na.max() * nb.max() < 2.0 ** 24           # every partial sum below 2^24
    exact = ha @ hb.T
    assert np.array_equal((ha.astype(F32) @ hb.T.astype(F32)).astype(np.float64), exact)
    # the reverse order of the terms too
    assert np.array_equal((ha[:, ::-1].astype(F32) @ hb[:, ::-1].T.astype(F32)).astype(np.float64),
                          exact)


def test_residual_extended_product_reaches_near_double_precision():
    h, Ca, n = large_h_and_c()
    K = h.shape[1]
    ea, eb = exponents(h, K), exponents(Ca.T, K)
    _, ha, fa, ra = split(h, ea)
    _, hb, fb, rb = split(Ca.T, eb)
    sc = np.ldexp(1.0, ea)[:, None] * np.ldexp(1.0, eb)[None, :]
    mm32 = lambda a, b: (a.astype(F32) @ b.T.astype(F32)).astype(np.float64)
    Z = h @ Ca                                        # exact h C_act (double)
    E1 = lambda Zt: 2.0 * float(n @ np.einsum("mp,mp->p", Ca, Zt))
    # one split: integer products exact, the other three together in fp32
    Z1 = (mm32(ha, hb) + (mm32(ha, fb) + mm32(fa, hb) + mm32(fa, fb))) * sc
    # the residual-extended product: four K blocks, each its own fp32 result, summed in double
    Z4 = (mm32(ha, hb) * sc + (mm32(ha, rb + fb) * sc).astype(F32)
          + (mm32(fa, hb + fb) * sc).astype(F32) + (mm32(ra, hb + fb) * sc).astype(F32))
    err1 = abs(E1(Z1) - E1(Z))
    err4 = abs(E1(Z4) - E1(Z))
    assert err1 > 1e-7                                # one split is too coarse here
    assert err4 < 1e-8                                # near double for the one-electron energy
    assert err4 < err1 / 100
    assert np.abs(Z4 - Z).max() < 1e-8 * np.abs(Z).max()
