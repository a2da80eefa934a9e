"""FP64 CPU oracle of the PNOF5 / PNOF7 / PNOF7s energy and orbital Lagrangian.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code,
constant or helper with the CUDA library and imports nothing from it.

Plain and slow on purpose: it follows the paper's operator route, not the
contraction order of the GPU kernels.

* occupations from gamma ....................... Sec. III.A, Eqs. soo, sum1-h, woo
* AO Coulomb / exchange operators J^q, K^q ..... Sec. III.D, Eq. Gpmn, with the
                                                 density-fitted ERIs
                                                 (mu nu|eta delta) = sum_P B^P_{mu nu} B^P_{eta delta}
* MO integrals J_pq, K_pq (L = K, real NOs) .... Sec. III.D, Eq. JKpq; Sec. II (L = K)
* energy ....................................... Sec. II, Eqs. EPNOF7, Eg, Efg; Sec. V, Eq. Efg_s
* orbital gradient / Lagrangian ................ Sec. III.B, Eqs. lowdin, Vee-s, Vee-d, lag, gval
* occupation gradient dE/dgamma ................ chain rule through Eqs. soo/woo

Readings of the paper taken here (all listed in the design notes):

* lambda_qp = C_q^T G_p with G = (1/4) dE/dC, i.e. n_p H_qp plus the braces of
  Eqs. Vee-s / Vee-d without their leading factor 4 (Eq. lowdin has 4 lambda on
  its right-hand side, Eq. lag does not show the 1/4).  Stored lam[q, p].
* the sum over f != g in Eq. EPNOF7 runs over ordered pairs; the sum over
  q, p in Omega_g in Eq. Eg includes q = p (Pi_pp K_pp = n_p J_pp).
* Pi_qp = +sqrt(n_q n_p) when q = p or both are weak, -sqrt(n_q n_p) when
  exactly one of them is the strong orbital g (Eq. intra).
* n is per spin in [0, 1]; sqrt(n) >= 0 is taken as the product of |sin| and
  |cos| factors of Eq. woo; derivatives are those of the (0, pi/2) branch.
* the weak orbitals of pair g, in increasing orbital index, are p_1 .. p_Ng
  of Eq. woo; gamma holds the npair strong gammas, then (Ng - 1) weak gammas
  per pair, pair-major.
* orbitals p >= nact are empty (n = 0): their lambda columns are zero.
* multiplets (Sec. II): the N_I singly occupied orbitals of Omega_I sit at indices
  npair .. npair + N_I - 1 (pair_map[g] = g), n = 1/2 fixed; they have no intra-subspace
  term (D_pp,pp = 0), contribute H_gg to E, and enter E_fg with every other subspace.
"""
from __future__ import annotations

import math

import numpy as np

PNOF5 = 5
PNOF7 = 7
PNOF7S = 8


# ----------------------------------------------------------------------------
# occupations (Sec. III.A)
# ----------------------------------------------------------------------------
def pair_members(pair_map: np.ndarray, npair: int):
    """Orbitals of each subspace Omega_g: [g, p_1, ..., p_Ng] (weak ones in increasing index)."""
    members = []
    for g in range(npair):
        weak = [int(p) for p in range(len(pair_map)) if pair_map[p] == g and p != g]
        members.append([g] + sorted(weak))
    return members


def subspaces(pair_map: np.ndarray, npair: int, nsingle: int = 0):
    """All subspaces of Omega: the pairs of Omega_II (pair_members), then the singly
    occupied orbitals of Omega_I, orbital g = npair .. npair + nsingle - 1 each alone."""
    return pair_members(pair_map, npair) + [[g] for g in range(npair, npair + nsingle)]


def occupations(gamma: np.ndarray, pair_map: np.ndarray, npair: int, ncwo: int,
                nsingle: int = 0):
    """n_p, sqrt(n_p), Phi_p = sqrt(n_p (1 - n_p)) and their Jacobians w.r.t. gamma.

    Eq. soo: n_g = (1 + cos^2 gamma_g) / 2, hole h_g = sin^2(gamma_g) / 2.
    Eq. woo: n_{p_i} = h_g cos^2 gamma_{p_1} ... cos^2 gamma_{p_{i-1}} sin^2 gamma_{p_i},
             the last weak orbital without the sin^2 factor.
    """
    nact = len(pair_map)
    ng = len(gamma)
    n = np.zeros(nact)
    sq = np.zeros(nact)
    phi = np.zeros(nact)
    dn = np.zeros((nact, ng))
    dsq = np.zeros((nact, ng))
    dphi = np.zeros((nact, ng))
    members = pair_members(pair_map, npair)
    for g in range(npair):
        tg = gamma[g]
        # strong orbital g
        ng_ = 0.5 * (1.0 + math.cos(tg) ** 2)
        dng = -math.cos(tg) * math.sin(tg)
        s_hole = abs(math.sin(tg)) / math.sqrt(2.0)            # sqrt(h_g) = sqrt(1 - n_g)
        ds_hole = math.copysign(1.0, math.sin(tg)) * math.cos(tg) / math.sqrt(2.0)
        n[g] = ng_
        sq[g] = math.sqrt(ng_)
        dn[g, g] = dng
        dsq[g, g] = dng / (2.0 * sq[g])
        phi[g] = sq[g] * s_hole
        dphi[g, g] = dsq[g, g] * s_hole + sq[g] * ds_hole
        # weak orbitals: sqrt(n_{p_i}) is a product of factors, each depending on one gamma
        weak = members[g][1:]
        for i, p in enumerate(weak):
            factors = [(g, s_hole, ds_hole)]
            for j in range(i):
                k = npair + g * (ncwo - 1) + j
                c = math.cos(gamma[k])
                factors.append((k, abs(c), -math.copysign(1.0, c) * math.sin(gamma[k])))
            if i < len(weak) - 1:
                k = npair + g * (ncwo - 1) + i
                s = math.sin(gamma[k])
                factors.append((k, abs(s), math.copysign(1.0, s) * math.cos(gamma[k])))
            val = 1.0
            for _, f, _ in factors:
                val *= f
            sq[p] = val
            n[p] = val * val
            for a, (k, f, df) in enumerate(factors):
                rest = 1.0
                for b, (_, f2, _) in enumerate(factors):
                    if b != a:
                        rest *= f2
                dsq[p, k] += df * rest
            dn[p] = 2.0 * sq[p] * dsq[p]
            om = math.sqrt(1.0 - n[p])
            phi[p] = sq[p] * om
            dphi[p] = dsq[p] * om - sq[p] * dn[p] / (2.0 * om)
    # Omega_I (Sec. II): each singly occupied orbital has n = 1/2, fixed (no gamma)
    for g in range(npair, npair + nsingle):
        n[g] = 0.5
        sq[g] = math.sqrt(0.5)
        phi[g] = 0.5
    return dict(n=n, sqrt_n=sq, phi=phi, dn=dn, dsqrt_n=dsq, dphi=dphi)


# ----------------------------------------------------------------------------
# integrals (Sec. III.D)
# ----------------------------------------------------------------------------
def unpack_B(Bp: np.ndarray, nbf: int) -> np.ndarray:
    """Packed [naux][nbf(nbf+1)/2] (mu >= nu at mu(mu+1)/2 + nu) -> dense symmetric [naux][nbf][nbf]."""
    naux = Bp.shape[0]
    out = np.zeros((naux, nbf, nbf))
    for mu in range(nbf):
        base = mu * (mu + 1) // 2
        out[:, mu, : mu + 1] = Bp[:, base: base + mu + 1]
        out[:, : mu + 1, mu] = Bp[:, base: base + mu + 1]
    return out


def ao_operators(B: np.ndarray, C_act: np.ndarray):
    """J^q and K^q of Eq. Gpmn for every active orbital q, with DF ERIs.

    J^q_{mu nu} = sum_{eta delta} Gamma^q_{eta delta} (mu nu|eta delta)
                = sum_P B^P_{mu nu} (C_q^T B^P C_q)
    K^q_{mu nu} = sum_{eta delta} Gamma^q_{eta delta} (mu delta|eta nu)
                = sum_P (B^P C_q)_mu (B^P C_q)_nu
    Returns arrays [nact][nbf][nbf].
    """
    naux, nbf, _ = B.shape
    nact = C_act.shape[1]
    Bflat = B.reshape(naux * nbf, nbf)
    BC = (Bflat @ C_act).reshape(naux, nbf, nact)            # (B^P C_q)_mu
    dq = np.einsum("Pmq,mq->Pq", BC, C_act)                  # C_q^T B^P C_q
    Jq = (dq.T @ B.reshape(naux, nbf * nbf)).reshape(nact, nbf, nbf)
    Kq = np.empty((nact, nbf, nbf))
    for q in range(nact):
        x = BC[:, :, q]
        Kq[q] = x.T @ x
    return Jq, Kq


def mo_jk(C_act: np.ndarray, Jq: np.ndarray, Kq: np.ndarray):
    """Eq. JKpq: J_pq = sum Gamma^p J^q, K_pq = sum Gamma^p K^q with Gamma^p = C_p C_p^T,
    i.e. J_pq = C_p^T J^q C_p (and the same for K)."""
    nact = C_act.shape[1]
    J = np.empty((nact, nact))
    K = np.empty((nact, nact))
    for q in range(nact):
        J[:, q] = np.sum(C_act * (Jq[q] @ C_act), axis=0)
        K[:, q] = np.sum(C_act * (Kq[q] @ C_act), axis=0)
    return J, K


def jk_entries(slices, C_act: np.ndarray, pairs):
    """Selected J_pq, K_pq of Eq. JKpq computed slice by slice, for workloads too large to
    hold B: J_pq = sum_P (C_p^T B^P C_p)(C_q^T B^P C_q) = C_p^T J^q C_p and
    K_pq = sum_P (C_p^T B^P C_q)^2 = C_p^T K^q C_p (Eq. Gpmn with DF integrals).
    `slices` yields dense symmetric B^P; `pairs` lists (p, q)."""
    cols = sorted({i for pq in pairs for i in pq})
    J = {pq: 0.0 for pq in pairs}
    K = {pq: 0.0 for pq in pairs}
    for BP in slices:
        BC = BP @ C_act[:, cols]                      # B^P C_i for the sampled orbitals
        loc = {c: k for k, c in enumerate(cols)}
        for (p, q) in pairs:
            dp = C_act[:, p] @ BC[:, loc[p]]
            dq = C_act[:, q] @ BC[:, loc[q]]
            bpq = C_act[:, p] @ BC[:, loc[q]]
            J[(p, q)] += dp * dq
            K[(p, q)] += bpq * bpq
    return J, K


# ----------------------------------------------------------------------------
# energy (Sec. II)
# ----------------------------------------------------------------------------
def _pi(p: int, q: int, g: int, sq: np.ndarray) -> float:
    """Pi_qp of Eq. intra for p, q in the same subspace with strong orbital g."""
    if p == q:
        return sq[p] * sq[q]
    if p == g or q == g:
        return -sq[p] * sq[q]
    return sq[p] * sq[q]


def energy(Hdiag, J, K, occ, pair_map, npair, functional, nsingle=0):
    """E = sum_g E_g + sum_{g in Omega_I} H_gg + sum_{f != g} E_fg (Eqs. EPNOF7, Eg, Efg /
    Efg_s); f, g run over all subspaces, the singly occupied ones included."""
    n, sq, phi = occ["n"], occ["sqrt_n"], occ["phi"]
    members = subspaces(pair_map, npair, nsingle)
    E = 0.0
    for g in range(npair):
        Om = members[g]
        Eg = 2.0 * sum(n[p] * Hdiag[p] for p in Om)
        for q in Om:
            for p in Om:
                Eg += _pi(p, q, g, sq) * K[p, q]
        E += Eg
    for g in range(npair, npair + nsingle):
        E += Hdiag[g]
    for f in range(len(members)):
        for g in range(len(members)):
            if f == g:
                continue
            for p in members[f]:
                for q in members[g]:
                    t = n[q] * n[p] * (2.0 * J[p, q] - K[p, q])
                    if functional == PNOF7:
                        t -= phi[q] * phi[p] * K[p, q]
                    elif functional == PNOF7S:
                        t -= 4.0 * phi[q] ** 2 * phi[p] ** 2 * K[p, q]
                    E += t
    return E


# ----------------------------------------------------------------------------
# orbital gradient and Lagrangian (Sec. III.B)
# ----------------------------------------------------------------------------
def generalized_fock_action(h, C_act, Jq, Kq, occ, pair_map, npair, functional, nsingle=0):
    """G[:, p] = (1/4) dE/dphi_p expanded in the AO basis (Eqs. lowdin, Vee-s, Vee-d):

    G_p = F_p C_p,  F_p = n_p h
        + sum_{q not in Omega_g(p)} [n_q n_p (2 J^q - K^q) - Phi_q Phi_p K^q]   (PNOF7)
        + sum_{q in Omega_g(p)} Pi_qp K^q
    (PNOF5: no Phi term; PNOF7s: -4 Phi_q^2 Phi_p^2 K^q instead.)  F_p is applied to C_p
    term by term: G_p = n_p h C_p + sum_q [a_pq (J^q C)_p + c_pq (K^q C)_p].
    """
    n, sq, phi = occ["n"], occ["sqrt_n"], occ["phi"]
    nbf, nact = C_act.shape
    a = np.zeros((nact, nact))      # coefficient of J^q in F_p
    c = np.zeros((nact, nact))      # coefficient of K^q in F_p
    for p in range(nact):
        gp = int(pair_map[p])
        for q in range(nact):
            gq = int(pair_map[q])
            if gq == gp:
                if gp < npair:  # a singly occupied orbital has no intra-subspace term
                    c[p, q] = _pi(p, q, gp, sq)
            else:
                a[p, q] = 2.0 * n[q] * n[p]
                c[p, q] = -n[q] * n[p]
                if functional == PNOF7:
                    c[p, q] -= phi[q] * phi[p]
                elif functional == PNOF7S:
                    c[p, q] -= 4.0 * phi[q] ** 2 * phi[p] ** 2
    G = n[None, :] * (h @ C_act)
    for q in range(nact):
        G += a[:, q][None, :] * (Jq[q] @ C_act) + c[:, q][None, :] * (Kq[q] @ C_act)
    return G


def occupation_gradient(Hdiag, J, K, occ, pair_map, npair, functional, nsingle=0):
    """dE/dgamma: partial derivatives of E in n, sqrt(n), Phi, then the chain rule
    through Eqs. soo/woo."""
    n, sq, phi = occ["n"], occ["sqrt_n"], occ["phi"]
    nact = len(n)
    dE_dn = np.zeros(nact)
    dE_dsq = np.zeros(nact)
    dE_dphi = np.zeros(nact)
    for p in range(nact):
        gp = int(pair_map[p])
        dE_dn[p] = 2.0 * Hdiag[p]
        for q in range(nact):
            gq = int(pair_map[q])
            if gq == gp:
                if gp < npair:
                    dE_dsq[p] += 2.0 * _pi(p, q, gp, np.ones(nact)) * sq[q] * K[p, q]
            else:
                dE_dn[p] += 2.0 * n[q] * (2.0 * J[p, q] - K[p, q])
                if functional == PNOF7:
                    dE_dphi[p] -= 2.0 * phi[q] * K[p, q]
                elif functional == PNOF7S:
                    dE_dn[p] -= 8.0 * (1.0 - 2.0 * n[p]) * phi[q] ** 2 * K[p, q]
    return dE_dn @ occ["dn"] + dE_dsq @ occ["dsqrt_n"] + dE_dphi @ occ["dphi"]


# ----------------------------------------------------------------------------
# hand-off to the orbital update (Sec. III.B)
# ----------------------------------------------------------------------------
def fockian(lam: np.ndarray, Fdiag: np.ndarray) -> np.ndarray:
    """The symmetric matrix of Eq. Fockian: off-diagonal
    F_qp = theta(p - q)[lambda_qp - lambda_pq] + theta(q - p)[lambda_pq - lambda_qp],
    diagonal given (the paper takes it from the previous diagonalisation)."""
    N = lam.shape[0]
    F = np.zeros((N, N))
    for q in range(N):
        for p in range(N):
            if q < p:
                F[q, p] = lam[q, p] - lam[p, q]
            elif q > p:
                F[q, p] = lam[p, q] - lam[q, p]
    F[np.diag_indices(N)] = Fdiag
    return F


def orbital_update(lam: np.ndarray, Fdiag: np.ndarray, C: np.ndarray):
    """Diagonalise F (eigenvalues ascending) and rotate the orbitals, C_new = C V."""
    eps, V = np.linalg.eigh(fockian(lam, Fdiag))
    return eps, C @ V


def from_operators(h, C, gamma, pair_map, Jq, Kq, npair, ncwo, functional=PNOF7, nsingle=0):
    """Everything of one build after the AO operators J^q, K^q of Eq. Gpmn: J_pq, K_pq
    (Eq. JKpq), E (Eqs. EPNOF7, Eg, Efg / Efg_s), G and lambda = C^T G (Eqs. lowdin, Vee-s,
    Vee-d, lag), dE/dC = 4 G and dE/dgamma (chain rule through Eqs. soo/woo)."""
    h = np.asarray(h, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    nbf = h.shape[0]
    pair_map = np.asarray(pair_map)
    nact = len(pair_map)
    C_act = C[:, :nact]
    occ = occupations(np.asarray(gamma, dtype=np.float64), pair_map, npair, ncwo, nsingle)
    J, K = mo_jk(C_act, Jq, Kq)
    Hdiag = np.einsum("mp,mn,np->p", C_act, h, C_act)
    E = energy(Hdiag, J, K, occ, pair_map, npair, functional, nsingle)
    G = generalized_fock_action(h, C_act, Jq, Kq, occ, pair_map, npair, functional, nsingle)
    lam = np.zeros((nbf, nbf))
    lam[:, :nact] = C.T @ G
    dE_dC = np.zeros((nbf, nbf))
    dE_dC[:, :nact] = 4.0 * G
    dE_dgamma = occupation_gradient(Hdiag, J, K, occ, pair_map, npair, functional, nsingle)
    return dict(E=E, lam=lam, dE_dgamma=dE_dgamma, dE_dC=dE_dC, G=G, J=J, K=K,
                Hdiag=Hdiag, n=occ["n"], occ=occ)


def build(h, B, C, gamma, pair_map, npair, ncwo, functional=PNOF7, packed=False, nsingle=0):
    """One Lagrangian build: E, lambda, dE/dgamma, dE/dC and the intermediates.
    nsingle singly occupied orbitals (Omega_I, n = 1/2) sit at npair .. npair + nsingle - 1
    with pair_map[g] = g.

    B: dense [naux][nbf][nbf] or packed [naux][nbf(nbf+1)/2] (packed=True).
    C: [nbf][nbf], column p = orbital p (Eq. lcao).
    """
    nbf = np.asarray(h).shape[0]
    if packed:
        B = unpack_B(np.asarray(B, dtype=np.float64), nbf)
    B = np.asarray(B, dtype=np.float64)
    C_act = np.asarray(C, dtype=np.float64)[:, :len(pair_map)]
    Jq, Kq = ao_operators(B, C_act)
    return from_operators(h, C, gamma, pair_map, Jq, Kq, npair, ncwo, functional, nsingle)


def build_streamed(h, blocks, C, gamma, pair_map, npair, ncwo, functional=PNOF7, nsingle=0,
                   on_block=None):
    """build() for workloads too large to hold B: `blocks` yields consecutive blocks of
    auxiliary slices, dense [np][nbf][nbf] (or packed [np][nbf(nbf+1)/2], unpacked here).
    J^q and K^q of Eq. Gpmn are sums over the auxiliary index, so ao_operators of each block
    is added to the running J^q, K^q; the rest is build()'s route unchanged.  on_block, when
    given, is called after each block with the number of slices done (progress, timing)."""
    nbf = np.asarray(h).shape[0]
    C_act = np.asarray(C, dtype=np.float64)[:, :len(pair_map)]
    Jq = Kq = None
    done = 0
    for blk in blocks:
        blk = np.asarray(blk, dtype=np.float64)
        if blk.ndim == 2:
            blk = unpack_B(blk, nbf)
        Jb, Kb = ao_operators(blk, C_act)
        if Jq is None:
            Jq, Kq = Jb, Kb
        else:
            Jq += Jb
            Kq += Kb
        done += blk.shape[0]
        if on_block is not None:
            on_block(done)
    return from_operators(h, C, gamma, pair_map, Jq, Kq, npair, ncwo, functional, nsingle)
