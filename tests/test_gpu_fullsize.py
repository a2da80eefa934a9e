"""Parity at the full workload sizes (GPU).

* precision workload (nbf 500, naux 2000, 20 pairs, Ncwo 3): full oracle against both
  GPU paths, element by element;
* large workload (nbf 1200, naux 4800, 50 pairs, Ncwo 2, packed B) in the launch
  configuration bench.py times: J_pq and K_pq sampled by the oracle slice by slice,
  the mixed path against the FP64 GPU path, and properties that hold at any size
  (J_pp = K_pp, symmetry of J and K, the Euler identity E = sum_p (lambda_pp + n_p H_pp));
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


def test_large_workload_sampled_and_invariants():
    import torch
    import paper_2004_06142_gb300 as dn
    prob, packed = synth.config_problem("large")
    N, Q, A = prob.nbf, prob.naux, prob.nact
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
    # mixed against the FP64 GPU path
    assert abs(m["E"] - f["E"]) <= 1e-6
    for key in ("lam", "dg", "dC", "J", "K"):
        assert np.abs(m[key] - f[key]).max() <= 1e-5, key
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
        np.testing.assert_allclose(r["lam"][:, A:], 0.0)
    # J, K entries computed by the oracle slice by slice
    pairs = [(0, 0), (0, 57), (3, 120), (49, 50), (149, 149), (100, 7)]
    from concurrent.futures import ThreadPoolExecutor

    def slices():
        with ThreadPoolExecutor(16) as ex:
            for c0 in range(0, Q, 64):
                yield from ex.map(lambda P: synth.b_slice(prob.seed, Q, N, P), range(c0, min(Q, c0 + 64)))

    Jo, Ko = pnof.jk_entries(slices(), Ca, pairs)
    for pq in pairs:
        assert abs(f["J"][pq] - Jo[pq]) <= 1e-10, pq
        assert abs(f["K"][pq] - Ko[pq]) <= 1e-10, pq
        assert abs(m["J"][pq] - Jo[pq]) <= 1e-5, pq
        assert abs(m["K"][pq] - Ko[pq]) <= 1e-5, pq


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
