"""The library's FP64 symmetric eigensolver (donof_eigh), the diagonalisation step of Sec.
III.B, against numpy's LAPACK eigh on the same matrices.

A backward-stable solver gives eigenvalues within O(n eps ||A||) of the exact ones, residuals
||A v_j - w_j v_j|| of that size, and eigenvectors within that over their gap (Davis-Kahan);
the eigenvectors of eigenvalues closer than the solver's cluster threshold are only fixed as
a basis of their cluster's invariant subspace.  Matrices: random dense ones of sizes that
leave ragged ends at every blocking (1, 2, 3, ..., 1200), the Fockian shape of the orbital
update (dense active block, diagonal inactive block), the rank-deficient symmetrised Lagrangian
of the optimisation's first step (a null space of dimension n - 2 nact), exactly repeated
eigenvalues, diagonal and zero matrices, and Wilkinson's W21+ (pairs of eigenvalues equal to
about 1e-14) glued into a larger matrix by small couplings.
"""
import numpy as np
import pytest

from helpers import to_dev

pytestmark = pytest.mark.gpu

EPS = np.finfo(float).eps


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_06142_gb300.build as b
    b.build()


def _eigh(A, ws=None):
    import torch
    import paper_2004_06142_gb300 as dn
    n = A.shape[0]
    Ad = to_dev(A)
    V = torch.empty(n, n, dtype=torch.float64, device="cuda")
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    ws = dn.donof_eigh(Ad, V, w, ws=ws)
    st = dn.donof_eigh_read_status(ws)
    return w.cpu().numpy(), V.cpu().numpy(), st, ws


def _gaps(w):
    d = np.diff(w)
    g = np.full(w.shape, np.inf)
    g[:-1] = d
    g[1:] = np.minimum(g[1:], d)
    return g


def _check(A, w, V, orth_tol=1e-10):
    n = A.shape[0]
    nA = max(np.linalg.norm(A, 2), np.finfo(float).tiny)
    tol = 8.0 * max(n, 8) * EPS * nA
    w_ref, V_ref = np.linalg.eigh(A)
    assert np.all(np.diff(w) >= 0.0)
    assert np.abs(w - w_ref).max() <= tol
    assert np.abs(A @ V - V * w).max() <= tol
    assert np.abs(V.T @ V - np.eye(n)).max() <= orth_tol
    # rank-one projectors of eigenvalues separated by more than the cluster threshold
    gap = _gaps(w_ref)
    sep = gap > 1e-4 * nA
    if sep.any():
        c = np.sum(V[:, sep] * V_ref[:, sep], axis=0)
        sin = np.linalg.norm(V[:, sep] - V_ref[:, sep] * c, axis=0)
        assert np.all(sin <= 4.0 * tol / gap[sep] + 1e-12)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 64, 65, 130, 257, 600, 1200])
def test_random_dense(n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, n))
    A = X + X.T
    w, V, st, _ = _eigh(A)
    assert st == 0
    _check(A, w, V)


def _fockian(n, nact, seed):
    rng = np.random.default_rng(seed)
    lam = np.zeros((n, n))
    lam[:, :nact] = rng.standard_normal((n, nact))
    q, p = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    F = np.where(q < p, lam - lam.T, lam.T - lam)
    np.fill_diagonal(F, -2.0 * np.arange(n) - 5.0)
    return F, lam


@pytest.mark.parametrize("n,nact", [(41, 10), (300, 40), (1200, 150)])
def test_fockian_shape(n, nact):
    F, _ = _fockian(n, nact, 3)
    w, V, st, _ = _eigh(F)
    assert st == 0
    _check(F, w, V)


@pytest.mark.parametrize("n,nact", [(120, 16), (1200, 150)])
def test_rank_deficient_symmetrised_lagrangian(n, nact):
    """(lambda + lambda^T) / 2 with lambda nonzero in nact columns: eigenvalue 0 of
    multiplicity n - 2 nact, whose eigenvectors are any orthonormal basis of the null space."""
    _, lam = _fockian(n, nact, 4)
    S = 0.5 * (lam + lam.T)
    w, V, st, _ = _eigh(S)
    assert st == 0
    _check(S, w, V, orth_tol=1e-11)


def test_repeated_eigenvalues():
    n = 160
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([np.full(40, 1.0), np.full(40, -2.0), rng.standard_normal(80)])
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    w, V, st, _ = _eigh(A)
    assert st == 0
    _check(A, w, V, orth_tol=1e-11)


@pytest.mark.parametrize("kind", ["diagonal", "zero", "identity"])
def test_diagonal_matrices(kind):
    n = 70
    rng = np.random.default_rng(8)
    A = {"diagonal": np.diag(rng.standard_normal(n)), "zero": np.zeros((n, n)),
         "identity": np.eye(n)}[kind]
    w, V, st, _ = _eigh(A)
    assert st == 0
    assert np.abs(w - np.linalg.eigvalsh(A)).max() <= 1e-15
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-14
    assert np.abs(A @ V - V * w).max() <= 1e-15


def test_glued_wilkinson():
    """Five copies of W21+ (eigenvalue pairs equal to ~1e-14) glued by couplings 1e-8 and
    shuffled by a random orthogonal similarity: tight clusters for the inverse-iteration path."""
    m, k = 21, 5
    W = np.diag(np.abs(np.arange(m) - 10.0)) + np.diag(np.ones(m - 1), 1) + np.diag(np.ones(m - 1), -1)
    n = m * k
    T = np.zeros((n, n))
    for b in range(k):
        T[b * m:(b + 1) * m, b * m:(b + 1) * m] = W
        if b:
            T[b * m, b * m - 1] = T[b * m - 1, b * m] = 1e-8
    rng = np.random.default_rng(9)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ T @ Q.T
    A = 0.5 * (A + A.T)
    w, V, st, _ = _eigh(A)
    assert st == 0
    _check(A, w, V, orth_tol=1e-10)


def test_reproducible_and_workspace_reuse():
    rng = np.random.default_rng(11)
    X = rng.standard_normal((333, 333))
    A = X + X.T
    w1, V1, _, ws = _eigh(A)
    w2, V2, _, _ = _eigh(A, ws=ws)
    assert np.array_equal(w1, w2) and np.array_equal(V1, V2)


def test_in_place_and_scaling():
    """V over A's own buffer; a matrix scaled by 2^300 gives the scaled eigenvalues exactly."""
    import torch
    import paper_2004_06142_gb300 as dn
    rng = np.random.default_rng(12)
    X = rng.standard_normal((90, 90))
    A = X + X.T
    w_ref, V_ref, _, _ = _eigh(A)
    Ad = to_dev(A * 2.0 ** 300)
    w = torch.empty(90, dtype=torch.float64, device="cuda")
    ws = dn.donof_eigh(Ad, Ad, w)
    assert dn.donof_eigh_read_status(ws) == 0
    assert np.array_equal(w.cpu().numpy(), w_ref * 2.0 ** 300)
    assert np.array_equal(Ad.cpu().numpy(), V_ref)


def test_nonfinite_input_reported():
    A = np.eye(16)
    A[3, 5] = A[5, 3] = np.nan
    _, _, st, _ = _eigh(A)
    assert st == -3  # DONOF_ERR_NONFINITE


def test_argument_errors():
    import torch
    import paper_2004_06142_gb300 as dn
    lib = dn.binding.lib()
    import ctypes
    nb = ctypes.c_size_t(0)
    assert lib.donof_eigh_workspace_size(0, ctypes.byref(nb)) == -1
    assert lib.donof_eigh_workspace_size(4097, ctypes.byref(nb)) == -1
    assert lib.donof_eigh_workspace_size(10, ctypes.byref(nb)) == 0
    A = torch.eye(10, dtype=torch.float64, device="cuda")
    w = torch.empty(10, dtype=torch.float64, device="cuda")
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    rc = lib.donof_eigh(10, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(A.data_ptr()),
                        ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(small.data_ptr()), 256,
                        None)
    assert rc == -4  # DONOF_ERR_WORKSPACE


@pytest.mark.parametrize("spread", [1e-9, 1e-13])
def test_large_clusters(spread):
    """A block-sized cluster that does not split: 250 eigenvalues within `spread` of 1, 100
    with gaps of 1e-7 near 3 (a chain of resolvable close eigenvalues) and 250 spread over
    [-5, 5], under a random orthogonal similarity: the clusters' members get inverse iteration
    of their own and a block orthonormalisation (the large-cluster path)."""
    n = 600
    rng = np.random.default_rng(13)
    lam = np.concatenate([1.0 + spread * rng.random(250), 3.0 + 1e-7 * np.arange(100),
                          rng.uniform(-5.0, 5.0, 250)])
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    w, V, st, _ = _eigh(A)
    assert st == 0
    _check(A, w, V, orth_tol=1e-11)
