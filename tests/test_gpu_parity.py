"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP64 path |dE| <= 1e-10 Eh and 1e-10 elementwise on lambda, dE/dgamma,
dE/dC, J, K (double arithmetic with a different contraction order: the differences are
rounding only).  Mixed path (fp16 hi+lo split operands, fp32 tensor-core accumulation,
double cross-tile sums): |dE| <= 1e-6 Eh, gradients <= 1e-5 max-abs, lambda <= 1e-5.
"""
import numpy as np
import pytest

import synth
from oracle import pnof

from helpers import gpu_build

pytestmark = pytest.mark.gpu

F64_TOL = 1e-10
MIX_E, MIX_G = 1e-6, 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_06142_gb300.build as b
    b.build()


def oracle(prob, d, functional, packed=False):
    return pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], prob.npair, prob.ncwo,
                      functional)


def compare(out, ref, tol_e, tol_g, tol_lam, tol_jk=None):
    assert out["status"] == 0
    assert abs(out["E"] - ref["E"]) <= tol_e, (out["E"], ref["E"])
    np.testing.assert_allclose(out["dE_dgamma"], ref["dE_dgamma"], rtol=0, atol=tol_g)
    np.testing.assert_allclose(out["dE_dgamma_bwd"], ref["dE_dgamma"], rtol=0, atol=tol_g)
    np.testing.assert_allclose(out["dE_dC"], ref["dE_dC"], rtol=0, atol=tol_g)
    np.testing.assert_allclose(out["lam"], ref["lam"], rtol=0, atol=tol_lam)
    tj = tol_jk if tol_jk is not None else tol_lam
    np.testing.assert_allclose(out["J"], ref["J"], rtol=0, atol=tj)
    np.testing.assert_allclose(out["K"], ref["K"], rtol=0, atol=tj)


CASES = [
    # name, nbf, naux, npair, ncwo
    ("plain", 24, 96, 5, 1),
    ("ragged", 41, 37, 3, 2),
    ("ragged2", 97, 150, 4, 3),
    ("differentiation", 120, 480, 8, 4),
    ("tail", 130, 257, 6, 4),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("functional", [pnof.PNOF7, pnof.PNOF5, pnof.PNOF7S])
def test_fp64_path(case, functional):
    _, nbf, naux, npair, ncwo = case
    prob = synth.Problem(nbf, naux, npair, ncwo, seed=1)
    d = synth.generate(prob)
    ref = oracle(prob, d, functional)
    out = gpu_build(prob, d, 0, functional)
    compare(out, ref, F64_TOL, F64_TOL, F64_TOL)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("functional", [pnof.PNOF7, pnof.PNOF5, pnof.PNOF7S])
def test_mixed_path(case, functional):
    _, nbf, naux, npair, ncwo = case
    prob = synth.Problem(nbf, naux, npair, ncwo, seed=2)
    d = synth.generate(prob)
    ref = oracle(prob, d, functional)
    out = gpu_build(prob, d, 1, functional)
    compare(out, ref, MIX_E, MIX_G, MIX_G, tol_jk=MIX_G)


def test_mixed_path_few_aux():
    """Fewer auxiliary functions than basis functions (naux = 0.4 nbf, below any density
    fitting basis in use): each slice of B carries more of J, so the representation error of
    the split operands reaches E with less averaging over slices; the E tolerance still holds."""
    prob = synth.Problem(600, 240, 25, 2, seed=3)
    d = synth.generate(prob)
    ref = oracle(prob, d, pnof.PNOF7)
    out = gpu_build(prob, d, 1, pnof.PNOF7)
    compare(out, ref, MIX_E, MIX_G, MIX_G, tol_jk=MIX_G)


def test_mixed_one_electron_part_is_near_double():
    """h scaled by 100 (|h| up to 1e3) so that the one-electron energy 2 sum n_p H_pp
    dominates: h C_act with one integer + fraction split per operand would miss E by about
    3e-5 Eh here (CPU emulation of the split); the residual-extended product by about 7e-8."""
    prob = synth.Problem(300, 200, 10, 2, seed=4)
    d = synth.generate(prob)
    d["h"] = d["h"] * 100.0
    ref = oracle(prob, d, pnof.PNOF7)
    out = gpu_build(prob, d, 1, pnof.PNOF7)
    compare(out, ref, MIX_E, MIX_G, MIX_G, tol_jk=MIX_G)


@pytest.mark.parametrize("shape", [(200, 400, 44, 3), (260, 520, 50, 4), (300, 600, 64, 3)],
                         ids=["nact176", "nact250", "nact256"])
@pytest.mark.parametrize("precision", [0, 1])
def test_wide_active_space(shape, precision):
    """nact above 160 up to the mixed path's limit of 256 (padded width 176, 256 with padding
    rows, 256 exactly): every tensor-core contraction then drains its accumulators 16 columns
    at a time, and at 256 the two accumulators fill the tensor memory."""
    nbf, naux, npair, ncwo = shape
    prob = synth.Problem(nbf, naux, npair, ncwo, seed=7)
    d = synth.generate(prob)
    ref = oracle(prob, d, pnof.PNOF7)
    out = gpu_build(prob, d, precision, pnof.PNOF7)
    tol = (F64_TOL, F64_TOL, F64_TOL) if precision == 0 else (MIX_E, MIX_G, MIX_G)
    compare(out, ref, *tol)


@pytest.mark.parametrize("shape", [(8, 1, 1, 1), (12, 3, 4, 2), (16, 2, 8, 1)],
                         ids=["one_slice", "nact_eq_nbf", "no_inactive_two_slices"])
@pytest.mark.parametrize("precision", [0, 1])
def test_degenerate_shapes(shape, precision):
    """One auxiliary function; every orbital active (nact = nbf, no inactive orbitals)."""
    nbf, naux, npair, ncwo = shape
    prob = synth.Problem(nbf, naux, npair, ncwo, seed=8)
    d = synth.generate(prob)
    ref = oracle(prob, d, pnof.PNOF7)
    out = gpu_build(prob, d, precision, pnof.PNOF7)
    tol = (F64_TOL, F64_TOL, F64_TOL) if precision == 0 else (MIX_E, MIX_G, MIX_G)
    compare(out, ref, *tol)


@pytest.mark.parametrize("precision", [0, 1])
def test_builds_are_bitwise_reproducible(precision):
    """Every sum runs in a fixed order (no atomic accumulation), so two builds of the same
    inputs agree bit for bit, in both precisions."""
    prob = synth.Problem(300, 700, 12, 3, seed=9)
    d = synth.generate(prob)
    a = gpu_build(prob, d, precision, pnof.PNOF7)
    b = gpu_build(prob, d, precision, pnof.PNOF7)
    assert a["E"] == b["E"]
    for k in ("lam", "dE_dgamma", "dE_dC", "J", "K"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("precision", [0, 1])
def test_packed_and_blocked(precision):
    """Packed B and a budget that streams P in several blocks (with a ragged last one)."""
    prob = synth.Problem(57, 203, 4, 2, seed=3)
    d = synth.generate(prob)
    ref = oracle(prob, d, pnof.PNOF7)
    budget = 40 * 57 * 16 * 8 if precision == 0 else 30 * (57 * 16 * 4 + 16 * 64 * 4 + 16 * 16 * 12)
    tol = (F64_TOL, F64_TOL, F64_TOL) if precision == 0 else (MIX_E, MIX_G, MIX_G)
    for packed in (False, True):
        out = gpu_build(prob, d, precision, pnof.PNOF7, packed=packed, budget=budget)
        compare(out, ref, *tol)


def test_autotuned_tiles_keep_parity():
    """After the autotuner has picked tile widths, the mixed path still matches the oracle."""
    import torch
    import paper_2004_06142_gb300 as dn
    from helpers import to_dev
    prob = synth.Problem(130, 257, 6, 4, seed=6)
    d = synth.generate(prob)
    ref = oracle(prob, d, pnof.PNOF7)
    b = dn.Builder(prob.nbf, prob.naux, prob.npair, prob.ncwo, dn.PNOF7, dn.B_DENSE, dn.MIXED)
    b.prepare(to_dev(d["B"]))
    args = (to_dev(d["h"]), to_dev(d["C"]), to_dev(d["gamma"]), to_dev(d["pair_map"].astype(np.int32)))
    b.autotune(*args)
    E, lam, dg = b.forward(*args)
    torch.cuda.synchronize()
    assert b.status() == 0
    assert abs(E.item() - ref["E"]) <= MIX_E
    assert np.abs(lam.cpu().numpy() - ref["lam"]).max() <= MIX_G
    assert np.abs(dg.cpu().numpy() - ref["dE_dgamma"]).max() <= MIX_G
