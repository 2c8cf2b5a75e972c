"""Independent second-quantised operator algebra on tiny determinant spaces (test-only).

Determinants are tuples of occupied spin orbitals in canonical order (alpha 0..n-1, then beta
n..2n-1), |q1 q2 ...> = a+_q1 a+_q2 ... |vac>, q1 < q2 < ....  Operators act by the
anticommutation rules alone: a+_p / a_p pick up (-1)^(number of occupied q < p).  Nothing here
knows Slater-Condon rules, excitation classes or labels, so agreement with the oracle pins
those independently.
"""
from __future__ import annotations

import itertools

import numpy as np


def annihilate(det, p):
    if p not in det:
        return None, 0
    k = det.index(p)
    return det[:k] + det[k + 1:], (-1) ** k


def create(det, p):
    if p in det:
        return None, 0
    k = sum(1 for q in det if q < p)
    return det[:k] + (p,) + det[k:], (-1) ** k


def apply_string(det, ops):
    """ops applied right to left: [(kind, p), ...], kind '+' create, '-' annihilate."""
    sign = 1
    for kind, p in reversed(ops):
        det, s = (create if kind == "+" else annihilate)(det, p)
        if det is None:
            return None, 0
        sign *= s
    return det, sign


def full_space(n, na, nb):
    out = []
    for a in itertools.combinations(range(n), na):
        for b in itertools.combinations(range(n, 2 * n), nb):
            out.append(tuple(a) + tuple(b))
    return out


def to_words(det, n):
    W = (n + 63) // 64
    x = np.zeros(2 * W, np.uint64)
    for so in det:
        s, p = divmod(so, n)
        x[s * W + p // 64] |= np.uint64(1 << (p % 64))
    return x


def from_words(x, n):
    W = (n + 63) // 64
    out = []
    for s in range(2):
        for p in range(n):
            if (int(x[s * W + p // 64]) >> (p % 64)) & 1:
                out.append(s * n + p)
    return tuple(out)


class Hamiltonian:
    """H = E_nuc + sum h_pq a+_p a_q + 1/2 sum <pq|rs> a+_p a+_q a_s a_r over spin orbitals."""

    def __init__(self, h1, eri4, e_nuc=0.0):
        self.n = h1.shape[0]
        self.h1, self.eri4, self.e_nuc = h1, eri4, e_nuc

    def spin(self, so):
        return so // self.n

    def apply(self, vec):
        """vec: {det: amplitude} -> H vec."""
        n, out = self.n, {}
        for det, amp in vec.items():
            out[det] = out.get(det, 0.0) + self.e_nuc * amp
            for q in det:
                for p in range(2 * n):
                    if self.spin(p) != self.spin(q):
                        continue
                    v = self.h1[p % n, q % n]
                    if v == 0.0:
                        continue
                    d2, s = apply_string(det, [("+", p), ("-", q)])
                    if d2 is not None:
                        out[d2] = out.get(d2, 0.0) + v * s * amp
            for r in det:
                for s_ in det:
                    if r == s_:
                        continue
                    for p in range(2 * n):
                        if self.spin(p) != self.spin(r):
                            continue
                        for q in range(2 * n):
                            if self.spin(q) != self.spin(s_):
                                continue
                            v = self.eri4[p % n, r % n, q % n, s_ % n]     # <pq|rs> = (pr|qs)
                            if v == 0.0:
                                continue
                            d2, sg = apply_string(det, [("+", p), ("+", q), ("-", s_), ("-", r)])
                            if d2 is not None:
                                out[d2] = out.get(d2, 0.0) + 0.5 * v * sg * amp
        return out


class DyallHamiltonian:
    """H_D = sum_core eps_i n_i + sum_virt eps_a n_a + (E_core - 2 sum_i eps_i)
       + sum_tu heff_tu a+_t a_u + 1/2 sum_tuvw <tu|vw> a+_t a+_u a_w a_v   (active indices)."""

    def __init__(self, n_core, n_act, n_virt, eps, heff, eri4, e_core):
        self.nc, self.na, self.nv = n_core, n_act, n_virt
        self.n = n_core + n_act + n_virt
        self.eps, self.heff, self.eri4 = eps, heff, eri4
        self.const = e_core - 2.0 * eps[:n_core].sum()

    def cls(self, so):
        p = so % self.n
        return 0 if p < self.nc else (1 if p < self.nc + self.na else 2)

    def apply(self, vec):
        n, nc, out = self.n, self.nc, {}
        act = [so for so in range(2 * n) if self.cls(so) == 1]
        for det, amp in vec.items():
            diag = self.const + sum(self.eps[so % n] for so in det if self.cls(so) != 1)
            out[det] = out.get(det, 0.0) + diag * amp
            for q in det:
                if self.cls(q) != 1:
                    continue
                for p in act:
                    if p // n != q // n:
                        continue
                    d2, s = apply_string(det, [("+", p), ("-", q)])
                    if d2 is not None:
                        out[d2] = out.get(d2, 0.0) + self.heff[p % n - nc, q % n - nc] * s * amp
            for r in det:
                for s_ in det:
                    if r == s_ or self.cls(r) != 1 or self.cls(s_) != 1:
                        continue
                    for p in act:
                        if p // n != r // n:
                            continue
                        for q in act:
                            if q // n != s_ // n:
                                continue
                            v = self.eri4[p % n, r % n, q % n, s_ % n]
                            d2, sg = apply_string(det, [("+", p), ("+", q), ("-", s_), ("-", r)])
                            if d2 is not None:
                                out[d2] = out.get(d2, 0.0) + 0.5 * v * sg * amp
        return out


def dyall_inputs(h1, eri4, n_core, n_act, gamma, e_nuc=0.0):
    """eps (generalised Fock diagonal), heff and E_core written from their definitions."""
    n = h1.shape[0]
    c = range(n_core)
    a = range(n_core, n_core + n_act)
    F = h1.copy()
    for i in c:
        F += 2.0 * eri4[:, :, i, i] - eri4[:, i, i, :]
    for ti, t in enumerate(a):
        for ui, u in enumerate(a):
            F += gamma[ti, ui] * (eri4[:, :, t, u] - 0.5 * eri4[:, t, u, :])
    e_core = e_nuc + sum(2.0 * h1[i, i] for i in c) + sum(
        2.0 * eri4[i, i, j, j] - eri4[i, j, j, i] for i in c for j in c)
    heff = np.array([[h1[t, u] + sum(2.0 * eri4[t, u, i, i] - eri4[t, i, i, u] for i in c) for u in a] for t in a])
    return np.diag(F).copy(), heff.reshape(n_act, n_act), e_core, F
