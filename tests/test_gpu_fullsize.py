"""Parity at the full workload sizes (GPU).

* precision workload (nbf 500, naux 2000, 20 pairs, Ncwo 3): full oracle against both
  GPU paths, element by element;
* large workload (nbf 1200, naux 4800, 50 pairs, Ncwo 2, packed B) in the launch
  configuration bench.py times: both GPU paths element by element against the FP64
  oracle's values stored in tests/golden/large_seed0.npz (written by
  tests/golden/make_large_golden.py, the oracle streamed over blocks of auxiliary
  slices), and properties that hold at any size (J_pp = K_pp, symmetry of J and K, the
  Euler identity E = sum_p (lambda_pp + n_p H_pp));
* differentiation workload (nbf 120, naux 480, 8 pairs, Ncwo 4): the autograd adjoint of
  the FP64 path against central finite differences (h = 1e-5).
"""
import numpy as np
import pytest

import synth
from oracle import pnof

from helpers import gpu_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_06142_gb300.build as b
    b.build()


def test_precision_workload_against_oracle():
    prob, packed = synth.config_problem("precision")
    d = synth.generate(prob, packed=packed)
    ref = pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], prob.npair, prob.ncwo,
                     pnof.PNOF7)
    for precision, tol_e, tol_a in ((0, 1e-10, 1e-10), (1, 1e-6, 1e-5)):
        out = gpu_build(prob, d, precision, pnof.PNOF7)
        assert out["status"] == 0
        assert abs(out["E"] - ref["E"]) <= tol_e, (precision, out["E"] - ref["E"])
        for key in ("lam", "dE_dgamma", "dE_dC", "J", "K"):
            err = np.abs(out[key] - ref[key]).max()
            assert err <= tol_a, (precision, key, err)


def _upload_B(prob, packed, dev):
    import torch
    N, Q = prob.nbf, prob.naux
    npk = N * (N + 1) // 2
    B = torch.empty((Q, npk) if packed else (Q, N, N), dtype=torch.float64, device=dev)
    for p0 in range(0, Q, 240):
        p1 = min(Q, p0 + 240)
        B[p0:p1].copy_(torch.from_numpy(synth.gen_B(prob.seed, Q, N, packed=packed, p0=p0, p1=p1)))
    return B


def load_large_golden(seed=0):
    """The oracle's values for the large workload (E, dE/dgamma, J, K and the active columns
    of lambda and dE/dC), written by tests/golden/make_large_golden.py."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        f"large_seed{seed}.npz")
    z = np.load(path)
    return {k: z[k] for k in z.files}


def test_large_workload_against_oracle_and_invariants():
    import torch
    import paper_2004_06142_gb300 as dn
    prob, packed = synth.config_problem("large")
    N, Q, A = prob.nbf, prob.naux, prob.nact
    ref = load_large_golden(prob.seed)
    assert list(ref["shape"]) == [N, Q, prob.npair, prob.ncwo, prob.seed]
    d = synth.generate(prob, with_B=False)
    dev = torch.device("cuda")
    B = _upload_B(prob, packed, dev)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    h, C, g = t(d["h"]), t(d["C"]), t(d["gamma"])
    pm = t(d["pair_map"].astype(np.int32))
    one = torch.ones(1, dtype=torch.float64, device=dev)
    res = {}
    for precision, budget in ((dn.MIXED, 0), (dn.FP64, 16 << 30)):
        bld = dn.Builder(N, Q, prob.npair, prob.ncwo, dn.PNOF7, dn.B_PACKED, precision, budget)
        bld.prepare(B)
        E, lam, dg = bld.forward(h, C, g, pm)
        dC, _ = bld.backward(one)
        J, K = bld.jk()
        assert bld.status() == 0
        res[precision] = dict(E=E.item(), lam=lam.cpu().numpy(), dg=dg.cpu().numpy(),
                              dC=dC.cpu().numpy(), J=J.cpu().numpy(), K=K.cpu().numpy())
        del bld
        torch.cuda.empty_cache()
    m, f = res[dn.MIXED], res[dn.FP64]
    # both paths against the oracle, element by element
    for r, tol_e, tol_a in ((f, 1e-10, 1e-10), (m, 1e-6, 1e-5)):
        assert abs(r["E"] - ref["E"][0]) <= tol_e, (tol_e, r["E"] - ref["E"][0])
        for key, rk in (("dg", "dE_dgamma"), ("J", "J"), ("K", "K")):
            err = np.abs(r[key] - ref[rk]).max()
            assert err <= tol_a, (tol_e, key, err)
        for key, rk in (("lam", "lam_act"), ("dC", "dE_dC_act")):
            err = np.abs(r[key][:, :A] - ref[rk]).max()
            assert err <= tol_a, (tol_e, key, err)
            assert np.all(r[key][:, A:] == 0.0), key
    # J and K of the mixed path to 1e-6 of their largest entry
    for key in ("J", "K"):
        assert np.abs(m[key] - ref[key]).max() <= 1e-6 * np.abs(ref[key]).max(), key
    # properties that hold at any size
    occ = pnof.occupations(d["gamma"], d["pair_map"], prob.npair, prob.ncwo)
    Ca = d["C"][:, :A]
    Hd = np.einsum("mp,mn,np->p", Ca, d["h"], Ca)
    # (the mixed path's b_pq and b_qp come from different tensor-core sums, so its K is
    # symmetric to the mixed tolerance only; its lambda is within 1e-5 per element, so the
    # Euler identity holds to nact * 1e-5 there)
    for r, tol, tol_sym in ((f, 1e-9, 1e-12), (m, A * 1e-5, 1e-5)):
        np.testing.assert_allclose(np.diag(r["J"]), np.diag(r["K"]), rtol=0, atol=1e-12)
        np.testing.assert_allclose(r["J"], r["J"].T, rtol=0, atol=tol_sym)
        np.testing.assert_allclose(r["K"], r["K"].T, rtol=0, atol=tol_sym)
        assert abs(r["E"] - (np.trace(r["lam"]) + np.sum(occ["n"] * Hd))) <= tol


def test_differentiation_workload_autograd_vs_finite_differences():
    import torch
    import paper_2004_06142_gb300 as dn
    prob, packed = synth.config_problem("differentiation")
    d = synth.generate(prob, packed=packed)
    dev = torch.device("cuda")
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    bld = dn.Builder(prob.nbf, prob.naux, prob.npair, prob.ncwo, dn.PNOF7, dn.B_DENSE, dn.FP64)
    bld.prepare(t(d["B"]))
    h, pm = t(d["h"]), t(d["pair_map"].astype(np.int32))
    C = t(d["C"]).requires_grad_(True)
    g = t(d["gamma"]).requires_grad_(True)
    E, _ = dn.energy(C, g, bld, h, pm)
    E.backward()
    gC, gg = C.grad.cpu().numpy(), g.grad.cpu().numpy()

    def energy(Cx, gx):
        e, _, _ = bld.forward(h, t(Cx), t(gx), pm, want_lam=False)
        return e.item()

    hstep = 1e-5
    for k in range(prob.ngamma):
        gp, gm = d["gamma"].copy(), d["gamma"].copy()
        gp[k] += hstep
        gm[k] -= hstep
        fd = (energy(d["C"], gp) - energy(d["C"], gm)) / (2 * hstep)
        assert abs(gg[k] - fd) <= 1e-7, (k, gg[k], fd)
    rng = np.random.default_rng(1)
    for _ in range(4):
        D = rng.standard_normal(d["C"].shape)
        fd = (energy(d["C"] + hstep * D, d["gamma"]) - energy(d["C"] - hstep * D, d["gamma"])) / (2 * hstep)
        assert abs(np.sum(gC * D) - fd) <= 1e-6 * max(1.0, abs(fd))
    ref = pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], prob.npair, prob.ncwo,
                     pnof.PNOF7)
    assert abs(E.item() - ref["E"]) <= 1e-10
    np.testing.assert_allclose(gC, ref["dE_dC"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(gg, ref["dE_dgamma"], rtol=0, atol=1e-10)
