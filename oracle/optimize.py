"""FP64 CPU oracle of the optimisation procedure around the build (Sec. III.D, III.C).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with the
CUDA library and imports nothing from it.

* occupation optimisation at fixed orbitals ...... Sec. III.D ("gamma^{j+1} is obtained for
                                                   fixed NOs by the unconstrained optimisation
                                                   of E[n(gamma), phi^j]", by CG or L-BFGS);
                                                   here scipy's L-BFGS-B as the optimiser
* scaling of F by zeta ........................... Sec. III.B (off-diagonal elements above
                                                   zeta divided by ten until below it)
* DIIS ........................................... Sec. III.C (error vector = off-diagonal
                                                   of F, the bordered linear system for the
                                                   coefficients, F-bar = sum_j c_j F^j)
* orbital iterations and convergence ............. Sec. III.B, III.D (diagonal of F from the
                                                   previous diagonalisation; energy criteria
                                                   and max |lambda_qp - lambda_pq| < delta)
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import minimize

from . import pnof


def energy_of_gamma(gamma, Hdiag, J, K, pair_map, npair, ncwo, functional, nsingle=0):
    """E and dE/dgamma at fixed orbitals (Hdiag, J, K fixed)."""
    occ = pnof.occupations(np.asarray(gamma, dtype=np.float64), pair_map, npair, ncwo, nsingle)
    E = pnof.energy(Hdiag, J, K, occ, pair_map, npair, functional, nsingle)
    g = pnof.occupation_gradient(Hdiag, J, K, occ, pair_map, npair, functional, nsingle)
    return E, g


def fold_gamma(gamma):
    """The representative of gamma in [0, pi/2]: n, sqrt(n) and Phi of Eqs. soo/woo depend on
    each gamma only through |sin gamma| and |cos gamma|, so E is unchanged by gamma -> -gamma
    and gamma -> pi - gamma."""
    t = np.remainder(np.asarray(gamma, dtype=np.float64), np.pi)
    return np.where(t > np.pi / 2, np.pi - t, t)


def optimize_occupations(Hdiag, J, K, gamma0, pair_map, npair, ncwo, functional,
                         gtol=1e-10, maxiter=2000, nsingle=0):
    """argmin_gamma E[n(gamma)] at fixed orbitals; returns (gamma, E, iterations).

    Reading: the minimisation runs over the fundamental box [0, pi/2]^ng (fold_gamma), with
    bounds; a minimum on a kink of sqrt(n) = |sin gamma| (an emptied weak orbital, a pair
    split evenly) is then a bound-constrained minimum, where a projected quasi-Newton method
    converges instead of zigzagging across the kink."""
    fun = lambda x: energy_of_gamma(x, Hdiag, J, K, pair_map, npair, ncwo, functional, nsingle)
    x = fold_gamma(gamma0)
    E, _ = fun(x)
    nit = 0
    bounds = [(0.0, np.pi / 2)] * len(x)
    for _ in range(20):  # restarted until E stops decreasing
        res = minimize(fun, x, jac=True, method="L-BFGS-B", bounds=bounds,
                       options=dict(gtol=gtol, ftol=0.0, maxiter=maxiter, maxcor=8))
        nit += res.nit
        E_new, _ = fun(res.x)
        if not E_new < E:
            break
        x, E = res.x, E_new
    # Newton polish on the free variables (Hessian by central differences of the analytic
    # gradient, minimum-norm steps for flat directions): gamma to near rounding, which the
    # energy alone (flat to second order at the optimum) cannot pin
    for _ in range(6):
        E0, g0 = fun(x)
        free = ~(((x <= 0.0) & (g0 > 0)) | ((x >= np.pi / 2) & (g0 < 0)))
        pg0 = np.abs(np.clip(x - g0, 0.0, np.pi / 2) - x).max()
        if not free.any() or pg0 < 1e-13:
            break
        idx = np.flatnonzero(free)
        H = np.zeros((len(idx), len(idx)))
        hs = 1e-5
        for a, k in enumerate(idx):
            xp, xm = x.copy(), x.copy()
            xp[k] += hs
            xm[k] -= hs
            H[:, a] = (fun(xp)[1][idx] - fun(xm)[1][idx]) / (2 * hs)
        H = 0.5 * (H + H.T)
        step = -np.linalg.lstsq(H, g0[idx], rcond=1e-10)[0]
        xn = x.copy()
        xn[idx] = np.clip(x[idx] + step, 0.0, np.pi / 2)
        En, gn = fun(xn)
        pgn = np.abs(np.clip(xn - gn, 0.0, np.pi / 2) - xn).max()
        if En <= E0 + 1e-14 * abs(E0) and pgn < pg0:
            x, E = xn, En
        else:
            break
    return x, E, nit


# ----------------------------------------------------------------------------
# orbital iterations (Sec. III.B-D)
# ----------------------------------------------------------------------------
def scale_offdiagonal(F, zeta):
    """Sec. III.B: every off-diagonal element above zeta in magnitude is divided by ten
    as many times as it takes to bring it to or below zeta."""
    S = np.array(F, dtype=np.float64)
    if zeta <= 0:
        return S
    N = S.shape[0]
    for q in range(N):
        for p in range(N):
            if q != p:
                while abs(S[q, p]) > zeta:
                    S[q, p] /= 10.0
    return S


def diis_coefficients(Bm):
    """Sec. III.C: minimise sum_ij c_i c_j B_ij subject to sum_j c_j = 1 through the
    bordered system [[B, -1], [-1, 0]] [c; Lambda] = [0; -1].  None when the system is
    singular."""
    m = Bm.shape[0]
    M = np.zeros((m + 1, m + 1))
    M[:m, :m] = Bm
    M[:m, m] = -1.0
    M[m, :m] = -1.0
    rhs = np.zeros(m + 1)
    rhs[m] = -1.0
    try:
        return np.linalg.solve(M, rhs)[:m]
    except np.linalg.LinAlgError:
        return None


DIIS_MAX_COEFFICIENT = 100.0


def max_asymmetry(lam):
    """max_{q,p} |lambda_qp - lambda_pq| (the convergence criterion of Sec. III.D)."""
    return float(np.abs(lam - lam.T).max())


def orbital_step(lam, Fdiag, C, zeta, history, depth):
    """One diagonalisation of F (Eq. Fockian) with the previous eigenvalues as its diagonal.

    Readings: the off-diagonal part is zeta-scaled before use; F^j and its error vector
    e^j = offdiag F^j are taken to the fixed AO basis (C F C^T, C e C^T) so that matrices of
    different iterations can be combined; the DIIS extrapolation uses the last `depth` of
    them (a singular system, or one with a coefficient above DIIS_MAX_COEFFICIENT in
    magnitude, restarts the history from the newest matrix); with lambda = C^T G as defined
    here, the energy-lowering assignment of eigenvectors to orbitals is by decreasing
    eigenvalue, and the eigenvalues in that order are the next diagonal.  Returns the new
    (C, Fdiag)."""
    F = scale_offdiagonal(pnof.fockian(lam, Fdiag), zeta)
    E_mo = F - np.diag(np.diag(F))
    e_ao = C @ E_mo @ C.T
    F_ao = e_ao + C @ np.diag(np.diag(F)) @ C.T
    history.append((F_ao, e_ao))
    del history[:-max(depth, 1)]
    Fbar = F_ao
    if depth >= 2 and len(history) >= 2:
        m = len(history)
        Bm = np.array([[np.sum(history[i][1] * history[j][1]) for j in range(m)]
                       for i in range(m)])
        c = diis_coefficients(Bm)
        if c is None or not np.all(np.abs(c) <= DIIS_MAX_COEFFICIENT):
            # reading: a singular or wildly extrapolating system restarts the history
            del history[:-1]
        else:
            Fbar = sum(c[j] * history[j][0] for j in range(m))
    eps, W = np.linalg.eigh(Fbar)
    order = np.argsort(-eps, kind="stable")
    return W[:, order], eps[order]


def optimize(h, B, C, gamma, pair_map, npair, ncwo, functional, Fdiag=None, zeta=0.1,
             depth=6, delta=1e-6, eps_energy=1e-10, max_outer=50, max_inner=10,
             occ_gtol=1e-10, packed=False, log=None, nsingle=0):
    """The procedure of Sec. III.D: in each outer iteration the occupations are optimised at
    fixed orbitals, then the orbitals by up to `max_inner` diagonalisations of F at fixed
    occupations; converged when max |lambda_qp - lambda_pq| < delta (and the energy changed
    by less than eps_energy over the outer iteration).  With Fdiag None the initial diagonal
    comes from one diagonalisation of the symmetrised lambda (Sec. III.D, initial step),
    which also rotates the start orbitals.  Returns a dict with the final C, gamma, E, the
    asymmetry, the per-build energies and the iteration counts."""
    C = np.array(C, dtype=np.float64)
    gamma = np.array(gamma, dtype=np.float64)
    pair_map = np.asarray(pair_map)
    run = lambda C_, g_: pnof.build(h, B, C_, g_, pair_map, npair, ncwo, functional, packed,
                                    nsingle)
    energies = []
    ref = run(C, gamma)
    gamma, _, _ = optimize_occupations(ref["Hdiag"], ref["J"], ref["K"], gamma, pair_map,
                                       npair, ncwo, functional, occ_gtol, nsingle=nsingle)
    if Fdiag is None:
        ref = run(C, gamma)
        lam = ref["lam"]
        eps, V = np.linalg.eigh(0.5 * (lam + lam.T))
        C = C @ V          # ascending eigenvalues of the symmetrised lambda
        Fdiag = -eps       # in the sign convention of F here: a decreasing diagonal
    Fdiag = np.array(Fdiag, dtype=np.float64)
    history = []
    E_outer = None
    asym = np.inf
    outer = inner_total = 0
    converged = False
    for outer in range(1, max_outer + 1):
        if outer > 1:
            ref = run(C, gamma)
            gamma, _, _ = optimize_occupations(ref["Hdiag"], ref["J"], ref["K"], gamma,
                                               pair_map, npair, ncwo, functional, occ_gtol,
                                               nsingle=nsingle)
        E_prev = None
        for _ in range(max_inner):
            ref = run(C, gamma)
            E = ref["E"]
            energies.append(E)
            asym = max_asymmetry(ref["lam"])
            if log is not None:
                log(outer, E, asym)
            if asym < delta:
                break
            if E_prev is not None and abs(E - E_prev) < eps_energy:
                break
            E_prev = E
            C, Fdiag = orbital_step(ref["lam"], Fdiag, C, zeta, history, depth)
            inner_total += 1
        if asym < delta and E_outer is not None and abs(E - E_outer) < eps_energy:
            converged = True
            break
        E_outer = E
    ref = run(C, gamma)
    return dict(C=C, gamma=gamma, Fdiag=Fdiag, E=ref["E"], asym=max_asymmetry(ref["lam"]),
                energies=energies, outer=outer, inner=inner_total, converged=converged)
