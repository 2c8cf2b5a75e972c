"""Seeded synthetic inputs for the stochastic SC-NEVPT2 / SC-MRCI local-estimator path.

This module stands in for the programs that produce the method's inputs in the paper
(the integral program and the CASSCF / selected-CI solver of the Results section):

* one-electron integrals h1 and Cholesky-built two-electron integrals (pq|rs),
* an exact CAS-CI ground state of the active space, or a selected-CI vector for large active
  spaces (the reference phi0),
* core/virtual orbitals made semicanonical (the paper's H_D uses orbitals that
  diagonalise the core and virtual generalised Fock blocks, Sec. II C),
* the random perturber coefficients c_l of the sampling function (Eq. 17).

It contains none of the stochastic method's arithmetic (no local energies, no reach-back
overlaps, no perturber norms).  Both the oracle and the CUDA path take its arrays as plain
inputs; neither imports the other.

Everything is seeded (numpy PCG64) so a workload is a pure function of its parameters.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "System", "make_system", "workload", "pack_eri", "unpack_eri", "n_labels",
    "psi_s_coeffs", "cas_strings", "casci", "sci", "make_sci_system", "WORKLOADS",
]


# --------------------------------------------------------------------------- integrals

def make_integrals(n_core: int, n_act: int, n_virt: int, rank: int, seed: int,
                   offdiag: float = 0.02, chol_sigma: float = 0.012, coulomb=(0.30, 0.45)):
    """Random real h1 (symmetric) and Cholesky factors L[K] (symmetric n x n each).

    h1 diagonal is drawn sorted inside each block: core U[-2,-1], active U[-0.5,0.5],
    virtual U[0.5,3.0]; off-diagonal N(0, offdiag).  eri = sum_K L_K (x) L_K is 8-fold
    symmetric and positive semidefinite as a pair matrix.  The first three factors are
    diagonal with entries in `coulomb` (a Coulomb-like (pp|qq) > 0 background); the rest
    are N(0,1) * exp(-|p-q|/4), symmetrised, scaled by chol_sigma (locality in orbital index).
    """
    n = n_core + n_act + n_virt
    rng = np.random.Generator(np.random.PCG64(seed))
    d = np.concatenate([
        np.sort(rng.uniform(-2.0, -1.0, n_core)),
        np.sort(rng.uniform(-0.5, 0.5, n_act)),
        np.sort(rng.uniform(0.5, 3.0, n_virt)),
    ])
    off = rng.normal(0.0, offdiag, (n, n))
    h1 = 0.5 * (off + off.T)
    h1[np.diag_indices(n)] = d
    idx = np.arange(n)
    decay = np.exp(-np.abs(idx[:, None] - idx[None, :]) / 4.0)
    L = np.zeros((rank, n, n))
    for K in range(rank):
        if K < 3:
            L[K][np.diag_indices(n)] = rng.uniform(coulomb[0], coulomb[1], n)
        else:
            A = rng.normal(0.0, 1.0, (n, n)) * decay
            L[K] = chol_sigma * 0.5 * (A + A.T)
    return h1, L


def pair_index(p: int, q: int) -> int:
    """Compound index of an unordered orbital pair, p >= q -> p(p+1)/2 + q."""
    if p < q:
        p, q = q, p
    return p * (p + 1) // 2 + q


def pack_eri(L: np.ndarray) -> np.ndarray:
    """8-fold packed chemists' integrals: eri[P(P1,P2)] = (pq|rs), P1 = P(p,q) >= P2 = P(r,s)."""
    rank, n, _ = L.shape
    rows, cols = np.tril_indices(n)            # p >= q, row-major over p: P = p(p+1)/2 + q
    Lp = L[:, rows, cols]                      # (rank, npair)
    M = Lp.T @ Lp                              # (npair, npair)
    r2, c2 = np.tril_indices(M.shape[0])
    return np.ascontiguousarray(M[r2, c2])


def unpack_eri(eri: np.ndarray, n: int) -> np.ndarray:
    """Full 4-index (pq|rs) array from the packed form (small n only)."""
    npair = n * (n + 1) // 2
    M = np.zeros((npair, npair))
    r2, c2 = np.tril_indices(npair)
    M[r2, c2] = eri
    M[c2, r2] = eri
    out = np.zeros((n, n, n, n))
    rows, cols = np.tril_indices(n)
    for P in range(npair):
        p, q = rows[P], cols[P]
        blk = np.zeros((n, n))
        blk[rows, cols] = M[P]
        blk[cols, rows] = M[P]
        out[p, q] = blk
        out[q, p] = blk
    return out


# --------------------------------------------------------------------------- CAS-CI

def cas_strings(norb: int, nel: int) -> np.ndarray:
    """Occupation strings (bit masks) of nel electrons in norb orbitals, lexicographic order."""
    return np.array([sum(1 << i for i in c) for c in itertools.combinations(range(norb), nel)],
                    dtype=np.int64)


def _replacement_tables(strs: np.ndarray, norb: int, restrict: bool = False):
    """E_tu = a+_t a_u on a string space: {(t,u): (src, dst, sign)}; sign from the
    number of occupied orbitals the operators pass (orbitals ordered ascending).  With
    restrict, replacements leading out of the given strings are dropped (P E_tu P)."""
    index = {int(s): i for i, s in enumerate(strs)}
    tabs = {}
    for t in range(norb):
        for u in range(norb):
            src, dst, sgn = [], [], []
            for I, s in enumerate(strs):
                s = int(s)
                if not (s >> u) & 1:
                    continue
                s1 = s & ~(1 << u)
                ph = bin(s1 & ((1 << u) - 1)).count("1")
                if (s1 >> t) & 1:
                    continue
                ph += bin(s1 & ((1 << t) - 1)).count("1")
                s2 = s1 | (1 << t)
                if restrict and s2 not in index:
                    continue
                src.append(I)
                dst.append(index[s2])
                sgn.append(-1.0 if ph & 1 else 1.0)
            tabs[(t, u)] = (np.array(src, dtype=np.int64), np.array(dst, dtype=np.int64),
                            np.array(sgn))
    return tabs


def _active_hamiltonian(h1, L, n_core, n_act, e_nuc):
    """Core-averaged active-space Hamiltonian: (E_core, h_eff[t,u], (tu|vw))."""
    c = slice(0, n_core)
    a = slice(n_core, n_core + n_act)
    trLc = np.einsum("kii->k", L[:, c, c])
    Jc = np.einsum("k,kpq->pq", trLc, L)                       # sum_i (pq|ii)
    Kc = np.einsum("kpi,kiq->pq", L[:, :, c], L[:, c, :])      # sum_i (pi|iq)
    e_core = e_nuc + 2.0 * np.trace(h1[c, c]) + 2.0 * np.trace(Jc[c, c]) - np.trace(Kc[c, c])
    heff = h1[a, a] + 2.0 * Jc[a, a] - Kc[a, a]
    La = L[:, a, a]
    eri_a = np.einsum("kpq,krs->pqrs", La, La)
    return e_core, heff, eri_a


class _CasSolver:
    """String-driven sigma vector for the active-space Hamiltonian
    H0 = E_core + sum_tu k_tu E_tu + 1/2 sum_tuvw (tu|vw) E_tu E_vw,
    k_tu = heff_tu - 1/2 sum_v (tv|vu); CI vector stored as C[I_alpha, I_beta]."""

    def __init__(self, e_core, heff, eri_a, na, nb):
        self.n = n = heff.shape[0]
        self.e_core = e_core
        self.heff = heff
        self.eri = eri_a
        self.k = heff - 0.5 * np.einsum("tvvu->tu", eri_a)
        self.sa = cas_strings(n, na)
        self.sb = cas_strings(n, nb)
        self.ta = _replacement_tables(self.sa, n)
        self.tb = self.ta if na == nb else _replacement_tables(self.sb, n)
        self.shape = (len(self.sa), len(self.sb))

    def _Ea(self, t, u, X):
        src, dst, sg = self.ta[(t, u)]
        out = np.zeros_like(X)
        out[dst] = sg[:, None] * X[src]
        return out

    def _Eb(self, t, u, X):
        src, dst, sg = self.tb[(t, u)]
        out = np.zeros_like(X)
        out[:, dst] = sg[None, :] * X[:, src]
        return out

    def E(self, t, u, X):
        return self._Ea(t, u, X) + self._Eb(t, u, X)

    def sigma(self, C):
        n = self.n
        D = np.empty((n, n) + C.shape)
        for t in range(n):
            for u in range(n):
                D[t, u] = self.E(t, u, C)
        G = np.tensordot(self.eri, D, axes=([2, 3], [0, 1]))
        S = self.e_core * C + np.tensordot(self.k, D, axes=([0, 1], [0, 1]))
        for t in range(n):
            for u in range(n):
                S += 0.5 * self.E(t, u, G[t, u])
        return S

    def diagonal(self):
        n = self.n
        oa = np.array([[(s >> t) & 1 for t in range(n)] for s in self.sa], dtype=float)
        ob = np.array([[(s >> t) & 1 for t in range(n)] for s in self.sb], dtype=float)
        J = np.einsum("ttuu->tu", self.eri)
        K = np.einsum("tuut->tu", self.eri)
        hd = np.diag(self.heff)
        one = (oa @ hd)[:, None] + (ob @ hd)[None, :]
        tot = oa[:, None, :] + ob[None, :, :]
        coul = 0.5 * np.einsum("abt,tu,abu->ab", tot, J, tot)
        exa = 0.5 * np.einsum("at,tu,au->a", oa, K, oa)
        exb = 0.5 * np.einsum("bt,tu,bu->b", ob, K, ob)
        return self.e_core + one + coul - exa[:, None] - exb[None, :]

    def rdm1(self, C):
        n = self.n
        nrm = np.vdot(C, C)
        g = np.zeros((n, n))
        for t in range(n):
            for u in range(n):
                g[t, u] = np.vdot(C, self.E(t, u, C)) / nrm
        return g


def _davidson(matvec, diag, x0, tol=1e-11, max_sub=40, max_iter=400):
    x = x0 / np.linalg.norm(x0)
    V = [x]
    AV = [matvec(x)]
    e = None
    for _ in range(max_iter):
        Vm = np.array([v.ravel() for v in V])
        AVm = np.array([v.ravel() for v in AV])
        Hs = Vm @ AVm.T
        Hs = 0.5 * (Hs + Hs.T)
        w, U = np.linalg.eigh(Hs)
        e = w[0]
        x = (U[:, 0] @ Vm).reshape(x0.shape)
        ax = (U[:, 0] @ AVm).reshape(x0.shape)
        r = ax - e * x
        if np.linalg.norm(r) < tol:
            break
        den = diag - e
        den[np.abs(den) < 1e-8] = 1e-8
        t = -r / den
        if len(V) >= max_sub:
            V, AV = [x], [ax]
        for v in V:
            t -= np.vdot(v, t) * v
        for v in V:
            t -= np.vdot(v, t) * v
        nt = np.linalg.norm(t)
        if nt < 1e-14:
            break
        t /= nt
        V.append(t)
        AV.append(matvec(t))
    return e, x / np.linalg.norm(x)


def casci(h1, L, n_core, n_act, na, nb, e_nuc=0.0):
    """Exact lowest Sz-conserving eigenpair of the core-averaged active-space Hamiltonian.

    Returns (energy, C[I_alpha, I_beta], alpha strings, beta strings, gamma (spin-summed 1-RDM)).
    """
    e_core, heff, eri_a = _active_hamiltonian(h1, L, n_core, n_act, e_nuc)
    if n_act == 0:
        C = np.ones((1, 1))
        return e_core, C, np.zeros(1, np.int64), np.zeros(1, np.int64), np.zeros((0, 0))
    s = _CasSolver(e_core, heff, eri_a, na, nb)
    diag = s.diagonal()
    if diag.size <= 400:
        # small spaces: dense diagonalisation of the explicit matrix
        N = diag.size
        Hm = np.zeros((N, N))
        for j in range(N):
            ej = np.zeros(N)
            ej[j] = 1.0
            Hm[:, j] = s.sigma(ej.reshape(s.shape)).ravel()
        w, U = np.linalg.eigh(0.5 * (Hm + Hm.T))
        e, C = w[0], U[:, 0].reshape(s.shape)
    else:
        x0 = np.zeros(s.shape)
        x0.flat[np.argmin(diag)] = 1.0
        x0 += 1e-3 * np.random.Generator(np.random.PCG64(7)).normal(size=s.shape)
        e, C = _davidson(s.sigma, diag, x0)
    if C.flat[np.argmax(np.abs(C))] < 0:
        C = -C
    return e, C, s.sa, s.sb, s.rdm1(C)


# --------------------------------------------------------------------------- selected CI

def _same_spin_hamiltonian(tabs, k, eri_a, nstr):
    """Dense matrix of one spin's part of the active Hamiltonian on the full string space:
    sum_tu k_tu E_tu + 1/2 sum_tuvw (tu|vw) E_tu E_vw (both operators of this spin)."""
    n = k.shape[0]
    Hs = np.zeros((nstr, nstr))
    dmap = np.full((n * n, nstr), -1, dtype=np.int64)
    smap = np.zeros((n * n, nstr))
    for (t, u), (src, dst, sg) in tabs.items():
        np.add.at(Hs, (dst, src), k[t, u] * sg)
        dmap[t * n + u, src] = dst
        smap[t * n + u, src] = sg
    g = eri_a.reshape(n * n, n * n)
    for (v, w), (src, dst, sg) in tabs.items():
        if len(src) == 0:
            continue
        tgt = dmap[:, dst]                                   # (tu, m): E_tu applied after E_vw
        val = 0.5 * g[:, v * n + w][:, None] * smap[:, dst] * sg[None, :]
        ok = tgt >= 0
        np.add.at(Hs, (tgt[ok], np.broadcast_to(src, tgt.shape)[ok]), val[ok])
    return Hs


class _ProductSpaceCI:
    """CI in the product space S x S of selected alpha and beta strings (Sz = 0, n_alpha =
    n_beta), with P H P applied exactly: same-spin parts as dense string-space matrices, the
    opposite-spin part sum (tu|vw) E^a_tu E^b_vw through projected replacement tables."""

    def __init__(self, e_core, heff, eri_a, strs_sel, Hs_sel):
        self.n = n = heff.shape[0]
        self.e_core = e_core
        self.eri = eri_a
        self.Hs = Hs_sel
        self.tab = _replacement_tables(strs_sel, n, restrict=True)
        self.m = m = len(strs_sel)
        occ = np.array([[(int(x) >> t) & 1 for t in range(n)] for x in strs_sel], dtype=float)
        J = np.einsum("ttuu->tu", eri_a)
        hs = np.diag(Hs_sel)
        self.diag = e_core + hs[:, None] + hs[None, :] + occ @ J @ occ.T
        self.g = eri_a.reshape(n * n, n * n)
        self.pairs = [(t, u) for t in range(n) for u in range(n)]

    def sigma(self, C):
        n, m = self.n, self.m
        S = self.e_core * C + self.Hs @ C + C @ self.Hs.T
        D = np.zeros((n * n, m, m))                        # D_vw = C (E^b_vw)^T
        for i, (v, w) in enumerate(self.pairs):
            src, dst, sg = self.tab[(v, w)]
            if len(src):
                D[i][:, dst] = C[:, src] * sg[None, :]
        G = (self.g @ D.reshape(n * n, -1)).reshape(n * n, m, m)
        for i, (t, u) in enumerate(self.pairs):            # sum_tu E^a_tu G_tu
            src, dst, sg = self.tab[(t, u)]
            if len(src):
                S[dst] += sg[:, None] * G[i][src]
        return S

    def rdm1(self, C):
        n = self.n
        g = np.zeros((n, n))
        nrm = np.vdot(C, C)
        for (t, u), (src, dst, sg) in self.tab.items():
            if len(src):
                g[t, u] = (np.vdot(C[dst], sg[:, None] * C[src]) + np.vdot(C[:, dst], sg[None, :] * C[:, src])) / nrm
        return g


def sci(h1, L, n_core, n_act, n_el_spin, n_strings, n_seed_strings=256, e_nuc=0.0, tol=1e-5):
    """Selected CI of the core-averaged active Hamiltonian (Sz = 0) by heat-bath selection of
    strings: solve in the product space of the n_seed_strings strings of lowest same-spin
    energy, score every other string s' by max_s |H_s's| sqrt(w_s) (w_s: the weight of string s
    in that solution), keep the n_strings best, and solve again in their product space
    (n_strings^2 determinants).  Returns (energy, C, strings, strings, gamma)."""
    e_core, heff, eri_a = _active_hamiltonian(h1, L, n_core, n_act, e_nuc)
    strs = cas_strings(n_act, n_el_spin)
    k = heff - 0.5 * np.einsum("tvvu->tu", eri_a)
    Hs = _same_spin_hamiltonian(_replacement_tables(strs, n_act), k, eri_a, len(strs))

    def solve(sel, guess=None):
        ci = _ProductSpaceCI(e_core, heff, eri_a, strs[sel], Hs[np.ix_(sel, sel)])
        x0 = np.zeros((len(sel), len(sel)))
        if guess is None:
            x0.flat[np.argmin(ci.diag)] = 1.0
        else:
            x0 += guess
        x0 += 1e-4 * np.random.Generator(np.random.PCG64(11)).normal(size=x0.shape)
        e, C = _davidson(ci.sigma, ci.diag, x0, tol=tol, max_sub=24, max_iter=80)
        return e, C, ci

    seed_sel = np.sort(np.argsort(np.diag(Hs), kind="stable")[:min(n_seed_strings, len(strs))])
    _, C0, _ = solve(seed_sel)
    w = 0.5 * ((C0 ** 2).sum(1) + (C0 ** 2).sum(0))
    score = (np.abs(Hs[:, seed_sel]) * np.sqrt(w)[None, :]).max(1)
    score[seed_sel] = np.inf
    sel = np.sort(np.argsort(-score, kind="stable")[:min(n_strings, len(strs))])
    pos = np.searchsorted(sel, seed_sel)                 # the seed solution as the starting vector
    guess = np.zeros((len(sel), len(sel)))
    guess[np.ix_(pos, pos)] = C0
    e, C, ci = solve(sel, guess)
    if C.flat[np.argmax(np.abs(C))] < 0:
        C = -C
    return e, C, strs[sel], strs[sel], ci.rdm1(C)


def _to_dets_fast(C, sa, sb, n_core, n_orb):
    """_to_dets for a product space whose occupied orbitals all lie in the first word."""
    W = (n_orb + 63) // 64
    if n_core + max(int(sa.max()), int(sb.max())).bit_length() > 64:
        raise ValueError("core and active orbitals must fit the first word")
    core = np.uint64((1 << n_core) - 1)
    ia, ib = np.indices(C.shape).reshape(2, -1)
    dets = np.zeros((len(ia), 2 * W), dtype=np.uint64)
    dets[:, 0] = core | (sa[ia].astype(np.uint64) << np.uint64(n_core))
    dets[:, W] = core | (sb[ib].astype(np.uint64) << np.uint64(n_core))
    return dets, C.ravel().astype(np.float64)


def make_sci_system(n_core, n_act, n_virt, n_alpha, n_beta, rank, seed, n_strings, *, e_nuc=0.0,
                    n_seed_strings=256, c_seed=None, **integral_kw) -> System:
    """Integrals -> heat-bath selected-CI reference (n_strings^2 determinants) -> semicanonical
    core/virtual -> packed inputs."""
    if n_alpha != n_beta:
        raise ValueError("the selected-CI generator builds Sz = 0 references")
    h1, L = make_integrals(n_core, n_act, n_virt, rank, seed, **integral_kw)
    e, C, sa, sb, gamma = sci(h1, L, n_core, n_act, n_alpha - n_core, n_strings, n_seed_strings, e_nuc)
    h1, L = semicanonicalize(h1, L, n_core, n_act, gamma)
    n = n_core + n_act + n_virt
    dets, coeffs = _to_dets_fast(C, sa, sb, n_core, n)
    nl = n_labels(n_core, n_virt)
    c = psi_s_coeffs(nl, seed + 17 if c_seed is None else c_seed)
    return System(n_core, n_act, n_virt, n_alpha, n_beta, np.ascontiguousarray(h1), pack_eri(L),
                  e_nuc, dets, coeffs, float(e), c, meta=dict(rank=rank, seed=seed, gamma=gamma, L=L, sci=True))


# --------------------------------------------------------------------------- semicanonical

def _generalized_fock(h1, L, n_core, n_act, gamma):
    """F_pq = h_pq + sum_i [2(pq|ii) - (pi|iq)] + sum_tu gamma_tu [(pq|tu) - 1/2 (pt|uq)]."""
    c = slice(0, n_core)
    a = slice(n_core, n_core + n_act)
    trLc = np.einsum("kii->k", L[:, c, c])
    F = h1 + 2.0 * np.einsum("k,kpq->pq", trLc, L) - np.einsum("kpi,kiq->pq", L[:, :, c], L[:, c, :])
    if n_act:
        gL = np.einsum("tu,ktu->k", gamma, L[:, a, a])
        F += np.einsum("k,kpq->pq", gL, L)
        F -= 0.5 * np.einsum("kpt,tu,kuq->pq", L[:, :, a], gamma, L[:, a, :], optimize=True)
    return F


def semicanonicalize(h1, L, n_core, n_act, gamma):
    """Rotate core and virtual orbitals to diagonalise their generalised-Fock blocks.
    Core rotations leave the core density, and virtual rotations the active space, unchanged,
    so the CAS-CI vector is unchanged."""
    n = h1.shape[0]
    F = _generalized_fock(h1, L, n_core, n_act, gamma)
    U = np.eye(n)
    c = slice(0, n_core)
    v = slice(n_core + n_act, n)
    if n_core:
        _, U[c, c] = np.linalg.eigh(F[c, c])
    if n - n_core - n_act:
        _, U[v, v] = np.linalg.eigh(F[v, v])
    h1r = U.T @ h1 @ U
    Lr = np.matmul(np.matmul(U.T, L), U)
    return 0.5 * (h1r + h1r.T), Lr


# --------------------------------------------------------------------------- system

def n_labels(n_core: int, n_virt: int) -> int:
    """Number of perturber labels: (core-hole sets of size <= 2) x (virtual-particle sets of size <= 2)."""
    nh = 1 + 2 * n_core + (2 * n_core) * (2 * n_core - 1) // 2
    npart = 1 + 2 * n_virt + (2 * n_virt) * (2 * n_virt - 1) // 2
    return nh * npart


def psi_s_coeffs(nl: int, seed: int) -> np.ndarray:
    """Sampling-function coefficients (Eq. 17): c_0 = 1, c_l = 0.1 (1 + 0.5 u_l), u_l ~ U[0,1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = 0.1 * (1.0 + 0.5 * rng.random(nl))
    c[0] = 1.0
    return c


@dataclass
class System:
    """One synthetic problem in the library's input format."""
    n_core: int
    n_act: int
    n_virt: int
    n_alpha: int            # total alpha electrons
    n_beta: int
    h1: np.ndarray          # (n, n) row-major, symmetric
    eri: np.ndarray         # 8-fold packed chemists' (pq|rs)
    e_nuc: float
    dets: np.ndarray        # (n_det, 2W) uint64: alpha words then beta words, full-orbital bits
    coeffs: np.ndarray      # (n_det,)
    e_cas: float            # CAS-CI eigenvalue from the generator's own solver
    c: np.ndarray           # (n_labels,) sampling coefficients
    meta: dict = field(default_factory=dict)

    @property
    def n_orb(self) -> int:
        return self.n_core + self.n_act + self.n_virt

    @property
    def W(self) -> int:
        return (self.n_orb + 63) // 64

    @property
    def n_labels(self) -> int:
        return n_labels(self.n_core, self.n_virt)


def _to_dets(C, sa, sb, n_core, n_orb, drop=0.0):
    W = (n_orb + 63) // 64
    core = (1 << n_core) - 1
    ia, ib = np.nonzero(np.abs(C) > drop) if drop > 0 else np.indices(C.shape).reshape(2, -1)
    dets = np.zeros((len(ia), 2 * W), dtype=np.uint64)
    coeffs = C[ia, ib].astype(np.float64)
    for r, (i, j) in enumerate(zip(ia, ib)):
        fa = core | (int(sa[i]) << n_core)
        fb = core | (int(sb[j]) << n_core)
        for w in range(W):
            dets[r, w] = np.uint64((fa >> (64 * w)) & 0xFFFFFFFFFFFFFFFF)
            dets[r, W + w] = np.uint64((fb >> (64 * w)) & 0xFFFFFFFFFFFFFFFF)
    return dets, coeffs


def make_system(n_core, n_act, n_virt, n_alpha, n_beta, rank, seed, *, e_nuc=0.0,
                semicanonical=True, c_seed=None, drop=0.0, **integral_kw) -> System:
    """Integrals -> CAS-CI reference -> semicanonical core/virtual -> packed inputs."""
    h1, L = make_integrals(n_core, n_act, n_virt, rank, seed, **integral_kw)
    na, nb = n_alpha - n_core, n_beta - n_core
    if not (0 <= na <= n_act and 0 <= nb <= n_act):
        raise ValueError("electron count does not fit the active space")
    e, C, sa, sb, gamma = casci(h1, L, n_core, n_act, na, nb, e_nuc)
    if semicanonical:
        h1, L = semicanonicalize(h1, L, n_core, n_act, gamma)
    n = n_core + n_act + n_virt
    dets, coeffs = _to_dets(C, sa, sb, n_core, n, drop)
    nl = n_labels(n_core, n_virt)
    c = psi_s_coeffs(nl, seed + 17 if c_seed is None else c_seed)
    return System(n_core, n_act, n_virt, n_alpha, n_beta, np.ascontiguousarray(h1), pack_eri(L),
                  e_nuc, dets, coeffs, float(e), c,
                  meta=dict(rank=rank, seed=seed, gamma=gamma, L=L))


# --------------------------------------------------------------------------- named workloads

WORKLOADS = {
    # 12 spatial orbitals (2 core, 4 active, 6 virtual), 8 electrons, Sz = 0, Cholesky rank 40,
    # factor scale 0.06 (a multireference CAS: natural occupations well away from 0 and 2),
    # reference = exact CAS(4e,4o) ground state (36 determinants)
    "tiny_12o_cas4": dict(n_core=2, n_act=4, n_virt=6, n_alpha=4, n_beta=4, rank=40, seed=2009,
                          chol_sigma=0.06),
    # 56 spatial orbitals (6 core, 10 active, 40 virtual), 22 electrons, Cholesky rank 168,
    # factor scale 0.05,
    # reference = exact CAS(10e,10o) ground state (63,504 determinants)
    "cas10_56o": dict(n_core=6, n_act=10, n_virt=40, n_alpha=11, n_beta=11, rank=168, seed=2109,
                      chol_sigma=0.05),
    # 104 spatial orbitals (10 core, 14 active, 80 virtual), 34 electrons (CAS(14e,14o)),
    # Cholesky rank 312, factor scale 0.05, reference = heat-bath selected CI on the active
    # Hamiltonian: the product space of 1,000 alpha x 1,000 beta strings (1,000,000 determinants)
    "sci_104o_cas14": dict(n_core=10, n_act=14, n_virt=80, n_alpha=17, n_beta=17, rank=312, seed=2309,
                           chol_sigma=0.05, n_strings=1000),
}

_CACHE: dict = {}


def workload(name: str) -> System:
    """The named seeded workload (memoised in-process)."""
    if name not in _CACHE:
        spec = WORKLOADS[name]
        _CACHE[name] = make_sci_system(**spec) if "n_strings" in spec else make_system(**spec)
    return _CACHE[name]


# --------------------------------------------------------------------------- batched / served workloads

def batch_specs(n_sys: int = 64, seed: int = 2409, total_walkers: int = 32768, max_act: int = 14):
    """Size distribution of the batched workload: 30-120 spatial orbitals, active spaces of 6-14
    orbitals at half filling, 2-10 core orbitals, Cholesky rank 3n.  Active spaces of up to 10
    orbitals take the exact CAS-CI reference (400, 4,900 or 63,504 determinants); 12 and 14 take a
    heat-bath selected-CI reference of 1e5 to 5e5 determinants (n_strings^2, n_strings drawn so).
    Walkers per system are proportional to the reference size (at least 32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    acts = [a for a in (6, 8, 10, 12, 14) if a <= max_act]
    prob = np.array([0.34, 0.26, 0.2, 0.12, 0.08][:len(acts)])
    prob /= prob.sum()
    specs = []
    for k in range(n_sys):
        n = int(rng.integers(30, 121))
        na = int(rng.choice(acts, p=prob))
        nc = int(rng.integers(2, 11))
        nv = n - nc - na
        spec = dict(n_core=nc, n_act=na, n_virt=nv, n_alpha=nc + na // 2, n_beta=nc + na // 2,
                    rank=3 * n, seed=seed + 100 * (k + 1), chol_sigma=0.05)
        if na > 10:
            spec["n_strings"] = int(round(np.sqrt(rng.uniform(1e5, 5e5))))
        specs.append(spec)
    ndet = np.array([s["n_strings"] ** 2 if "n_strings" in s else len(cas_strings(s["n_act"], s["n_act"] // 2)) ** 2
                     for s in specs], dtype=float)
    walkers = np.maximum(32, np.round(total_walkers * ndet / ndet.sum())).astype(int)
    return specs, walkers.tolist()


def _make_from_spec(spec):
    return make_sci_system(**spec) if "n_strings" in spec else make_system(**spec)


def make_systems(specs, processes: int = 0):
    """Generate several systems, in a spawn process pool when processes > 1."""
    if processes and processes > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            return pool.map(_make_from_spec, specs)
    return [_make_from_spec(s) for s in specs]


def scan_systems(spec: dict, n_points: int = 10, lam_max: float = 0.1, seed: int = 7):
    """A 'geometry scan': one orbital partition, Cholesky factors L(lambda) = L0 + lambda dL for
    lambda in [0, lam_max], each with its own CAS-CI reference and semicanonical orbitals."""
    sp = dict(spec)
    nc, na, nv = sp["n_core"], sp["n_act"], sp["n_virt"]
    h1, L0 = make_integrals(nc, na, nv, sp["rank"], sp["seed"], chol_sigma=sp.get("chol_sigma", 0.05))
    rng = np.random.Generator(np.random.PCG64(seed))
    dL = rng.normal(0.0, 1.0, L0.shape) * np.abs(L0).mean()
    dL = 0.5 * (dL + np.transpose(dL, (0, 2, 1)))
    out = []
    nla, nlb = sp["n_alpha"] - nc, sp["n_beta"] - nc
    for k in range(n_points):
        lam = lam_max * k / max(n_points - 1, 1)
        L = L0 + lam * dL
        e, C, sa, sb, gamma = casci(h1, L, nc, na, nla, nlb)
        h1r, Lr = semicanonicalize(h1, L, nc, na, gamma)
        dets, coeffs = _to_dets(C, sa, sb, nc, nc + na + nv)
        c = psi_s_coeffs(n_labels(nc, nv), seed + k)
        out.append(System(nc, na, nv, sp["n_alpha"], sp["n_beta"], np.ascontiguousarray(h1r), pack_eri(Lr), 0.0,
                          dets, coeffs, float(e), c, meta=dict(lam=lam, gamma=gamma, L=Lr)))
    return out
