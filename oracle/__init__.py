"""Plain CPU oracle for the stochastic SC-NEVPT2(s) / SC-MRCI(s) local-estimator path.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / reference leg may import this package.  It shares no code with the CUDA
path (``paper_1909_06935_gb300``) and imports nothing from it.

Layers:
  * ``oracle.c`` (plain C, FP64, OpenMP over walkers): Slater-Condon H and Dyall H_D,
    perturber labels, reference lookup, reach-back overlaps <m|H|phi0> (Eq. 6-7), the local
    quantities of one walker step (Eq. 5, Eq. 16), the continuous-time walk, and brute-force
    deterministic strongly contracted quantities over the whole FOIS (Eq. 2, 14).
  * this module: ctypes marshalling, the finalize step (Eq. 14-15 with screening, jackknife
    error bars), the SC-MRCI(s) energy gradient (Eq. 8-9), its exact counterpart and the
    SC-MRCI eigenproblem in the basis of strongly contracted states, and the AMSGrad update
    (Reddi, Kale, Kumar 2018), written with numpy directly from the equations.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

N_TYPES = 9          # type t = 3h + p of a determinant with h core holes and p virtual electrons


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc -O3 -std=c11: IEEE arithmetic, no FMA contraction; OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.oracle_create.restype = P
            lib.oracle_create.argtypes = [C.c_int] * 5 + [P, P, C.c_double, C.c_int64, P, P, P, C.c_int64,
                                                          C.POINTER(C.c_int)]
            lib.oracle_free.argtypes = [P]
            lib.oracle_setup_info.argtypes = [P, P, P, P, P]
            lib.oracle_label.restype = C.c_int64
            lib.oracle_label.argtypes = [P, P, P]
            lib.oracle_h.restype = C.c_double
            lib.oracle_h.argtypes = [P, P, P]
            lib.oracle_hd.restype = C.c_double
            lib.oracle_hd.argtypes = [P, P, P]
            lib.oracle_psi.restype = C.c_double
            lib.oracle_psi.argtypes = [P, P, P]
            lib.oracle_local.restype = C.c_int64
            lib.oracle_local.argtypes = [P, P, P, C.c_int64, P, P, P]
            lib.oracle_move.restype = C.c_uint32
            lib.oracle_move.argtypes = [P, P, C.c_uint64, C.c_uint32, C.c_uint32, P, P]
            lib.oracle_sample.restype = C.c_int
            lib.oracle_sample.argtypes = [P, C.c_int64, C.c_int64, C.c_int64, C.c_uint64, C.c_int, C.c_int,
                                          P, P, P, P, P, P, P, P]
            lib.oracle_brute.restype = C.c_int
            lib.oracle_brute.argtypes = [P, P, P, P, P]
            lib.oracle_philox.argtypes = [P, P, P]
            lib.oracle_walk_one.restype = C.c_int
            lib.oracle_walk_one.argtypes = [P, C.c_uint32, C.c_int64, C.c_uint64, P]
            lib.oracle_set_hb_eps.argtypes = [P, C.c_double]
            lib.oracle_set_hb_eps.restype = None
            lib.oracle_set_threads.argtypes = [C.c_int]
            lib.oracle_set_threads.restype = None
            lib.oracle_neighbour_ids.restype = C.c_int64
            lib.oracle_neighbour_ids.argtypes = [P, P, C.c_int64, P]
            lib.oracle_neighbours.restype = C.c_int
            lib.oracle_neighbours.argtypes = [P, P, C.c_int64, P, P, P]
            _lib = lib
    return _lib


def set_threads(n: int = 0):
    """Threads of the oracle's parallel loops from now on (0: all cores)."""
    _load().oracle_set_threads(int(n))


def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11) as implemented by the oracle."""
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    _load().oracle_philox(_ptr(c), _ptr(k), _ptr(o))
    return o


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Oracle:
    """One loaded system: integrals, reference, sampling coefficients c (one per label)."""

    def __init__(self, n_core, n_act, n_virt, n_alpha, n_beta, h1, eri, e_nuc, dets, coeffs, c):
        self._lib = _load()
        self.n_core, self.n_act, self.n_virt = n_core, n_act, n_virt
        self.n = n_core + n_act + n_virt
        self.W = (self.n + 63) // 64
        self._keep = [np.ascontiguousarray(h1, np.float64), np.ascontiguousarray(eri, np.float64),
                      np.ascontiguousarray(dets, np.uint64), np.ascontiguousarray(coeffs, np.float64),
                      np.ascontiguousarray(c, np.float64)]
        h1a, eria, detsa, coa, ca = self._keep
        st = C.c_int(0)
        self.n_labels = len(ca)
        self._h = self._lib.oracle_create(n_core, n_act, n_virt, n_alpha, n_beta, _ptr(h1a), _ptr(eria),
                                          float(e_nuc), len(coa), _ptr(detsa), _ptr(coa), _ptr(ca),
                                          len(ca), C.byref(st))
        if not self._h:
            raise ValueError(f"oracle_create failed with status {st.value}")
        self.c = ca
        out = np.zeros(5)
        self.eps = np.zeros(self.n)
        self.gamma = np.zeros((max(n_act, 1), max(n_act, 1)))
        self.heff = np.zeros((max(n_act, 1), max(n_act, 1)))
        self._lib.oracle_setup_info(self._h, _ptr(out), _ptr(self.eps), _ptr(self.gamma), _ptr(self.heff))
        self.e0, self.norm0, self.e_core, self.sum_eps_core = out[:4]
        self.start = int(out[4])

    @classmethod
    def from_system(cls, s, c=None):
        return cls(s.n_core, s.n_act, s.n_virt, s.n_alpha, s.n_beta, s.h1, s.eri, s.e_nuc, s.dets, s.coeffs,
                   s.c if c is None else c)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_free(h)
            self._h = None

    def set_hb_eps(self, eps: float):
        """Heat-bath cutoff (Sec. II D): double excitations with |<ab||ij>| < eps are dropped from the
        walk, the overlaps and the brute force from now on (0: exact).  E0 and the set-up stay exact."""
        self._lib.oracle_set_hb_eps(self._h, float(eps))

    # ---- single determinants
    def _det(self, d):
        return np.ascontiguousarray(d, np.uint64).reshape(2 * self.W)

    def label(self, d):
        hp = np.zeros(2, np.int32)
        l = self._lib.oracle_label(self._h, _ptr(self._det(d)), _ptr(hp))
        return int(l), int(hp[0]), int(hp[1])

    def h(self, a, b) -> float:
        """<b|H|a> (= <a|H|b>)."""
        return self._lib.oracle_h(self._h, _ptr(self._det(a)), _ptr(self._det(b)))

    def hd(self, a, b) -> float:
        return self._lib.oracle_hd(self._h, _ptr(self._det(a)), _ptr(self._det(b)))

    def psi(self, d):
        """(psi_s(d), phi0(d) for a CAS determinant or O(d) = <d|H|phi0> for a FOIS one)."""
        o = C.c_double(0.0)
        v = self._lib.oracle_psi(self._h, _ptr(self._det(d)), C.byref(o))
        return v, o.value

    def local(self, d, max_nb: int = 0):
        """Local quantities of one walker step (Eq. 5, Eq. 16).

        Returns dict(S, EL, num, Hnn, HDnn, psi, label, type, nnb) and, when max_nb > 0,
        neighbour arrays: dets (k, 2W), H, HD, O, psi, Gamma, exc.
        """
        out = np.zeros(10)
        if max_nb:
            nd = np.zeros((max_nb, 2 * self.W), np.uint64)
            nv = np.zeros((max_nb, 5))
            ne = np.zeros(max_nb, np.uint32)
            k = self._lib.oracle_local(self._h, _ptr(self._det(d)), _ptr(out), max_nb, _ptr(nd), _ptr(nv), _ptr(ne))
        else:
            k = self._lib.oracle_local(self._h, _ptr(self._det(d)), _ptr(out), 0, None, None, None)
        r = dict(S=out[0], EL=out[1], num=out[2], Hnn=out[3], HDnn=out[4], psi=out[5], label=int(out[6]),
                 type=int(out[7]), nnb=int(out[8]), terms=int(out[9]))
        if max_nb:
            k = min(k, max_nb)
            r.update(dets=nd[:k], H=nv[:k, 0], HD=nv[:k, 1], O=nv[:k, 2], psi_m=nv[:k, 3], Gamma=nv[:k, 4],
                     exc=ne[:k])
        return r

    def neighbour_ids(self, d):
        """Excitation ids (r1 | r2<<8 | a1<<16 | a2<<24) of every neighbour of d, in the order of
        local(); no overlaps are evaluated."""
        dd = self._det(d)
        n = self._lib.oracle_neighbour_ids(self._h, _ptr(dd), 0, None)
        ids = np.zeros(max(n, 1), np.uint32)
        self._lib.oracle_neighbour_ids(self._h, _ptr(dd), n, _ptr(ids))
        return ids[:n]

    def neighbours(self, d, ids):
        """Per-neighbour quantities of local() for the given excitation ids of d:
        dict(dets, H, HD, O, psi_m, Gamma), evaluated in parallel."""
        dd = self._det(d)
        ii = np.ascontiguousarray(ids, np.uint32)
        dets = np.zeros((len(ii), 2 * self.W), np.uint64)
        vals = np.zeros((len(ii), 5))
        rc = self._lib.oracle_neighbours(self._h, _ptr(dd), len(ii), _ptr(ii), _ptr(dets), _ptr(vals))
        if rc:
            raise ValueError("an id is not a neighbour of the determinant")
        return dict(dets=dets, H=vals[:, 0], HD=vals[:, 1], O=vals[:, 2], psi_m=vals[:, 3], Gamma=vals[:, 4])

    def move(self, d, seed: int, step: int, walker: int):
        nxt = np.zeros(2 * self.W, np.uint64)
        out = np.zeros(4)
        exc = self._lib.oracle_move(self._h, _ptr(self._det(d)), seed, step, walker, _ptr(nxt), _ptr(out))
        return nxt, int(exc), dict(S=out[0], EL=out[1], num=out[2], psi_next=out[3])

    def walk_one(self, walker: int, n_steps: int, seed: int):
        """Trajectory (n_steps x 2W) of one walker from the start determinant."""
        traj = np.zeros((n_steps, 2 * self.W), np.uint64)
        rc = self._lib.oracle_walk_one(self._h, walker, n_steps, seed, _ptr(traj))
        if rc:
            raise RuntimeError(f"oracle_walk_one failed with status {rc}")
        return traj

    # ---- the walk
    def sample(self, n_walkers: int, n_steps: int, burn_in: int, seed: int, n_groups: int,
               threads: int = 0, trajectory: bool = False):
        """Continuous-time walk (Sec. II B); returns the raw group accumulators."""
        L, G = self.n_labels, n_groups
        accN = np.zeros((G, L))
        accU = np.zeros((G, L))
        accW = np.zeros(G)
        accE = np.zeros(G)
        ts = np.zeros(N_TYPES, np.int64)
        accA = np.zeros((G, L))
        accB = np.zeros((G, L))
        traj = np.zeros((n_walkers, n_steps, 2 * self.W), np.uint64) if trajectory else None
        rc = self._lib.oracle_sample(self._h, n_walkers, n_steps, burn_in, seed, G, threads, _ptr(accN),
                                     _ptr(accU), _ptr(accW), _ptr(accE), _ptr(ts), _ptr(accA), _ptr(accB),
                                     _ptr(traj) if trajectory else None)
        if rc:
            raise RuntimeError(f"oracle_sample failed with status {rc}")
        acc = dict(N=accN, U=accU, W=accW, E=accE, A=accA, B=accB, type_steps=ts,
                   walker_steps=n_walkers * max(n_steps - burn_in, 0))
        if trajectory:
            acc["trajectory"] = traj
        return acc

    def finalize(self, acc, tau: float = 1e-10):
        return finalize(acc, self.e0, self.c, self.n_core, self.n_virt, tau)

    # ---- deterministic brute force
    def brute(self, label_matrix: bool = False):
        """Deterministic SC quantities: N_l, D_l = <v_l|H_D|v_l>, <psi_s|psi_s>, <psi_s|H|psi_s>;
        with label_matrix, also H_ll' = <v_l|H|v_l'> (dense; tiny systems only)."""
        Nl = np.zeros(self.n_labels)
        Dl = np.zeros(self.n_labels)
        out = np.zeros(3)
        Hll = np.zeros((self.n_labels, self.n_labels)) if label_matrix else None
        self._lib.oracle_brute(self._h, _ptr(Nl), _ptr(Dl), _ptr(out), _ptr(Hll) if label_matrix else None)
        r = dict(N=Nl, D=Dl, psi_norm=out[0], psi_H_psi=out[1], fois_size=int(out[2]))
        if label_matrix:
            r["H"] = Hll
        return r


# ------------------------------------------------------------------ finalize (Eq. 14-15)

def label_types(n_core: int, n_virt: int) -> np.ndarray:
    """Type t = 3h + p of every label (h core holes, p virtual particles)."""
    nh = 1 + 2 * n_core + (2 * n_core) * (2 * n_core - 1) // 2
    npart = 1 + 2 * n_virt + (2 * n_virt) * (2 * n_virt - 1) // 2

    def size(r, m):
        return 0 if r == 0 else (1 if r <= m else 2)

    hs = np.array([size(r, 2 * n_core) for r in range(nh)])
    ps = np.array([size(r, 2 * n_virt) for r in range(npart)])
    return (3 * hs[:, None] + ps[None, :]).ravel()


def energies(N, U, e0, tau):
    """E^(2) from label sums (Eq. 14-15): for l != 0 with N_l > 0 and N_l/N_0 >= tau,
    E_l = U_l/N_l and E^(2) += (N_l/N_0)/(E0 - E_l).  Returns (per-label e2, kept mask, ratio)."""
    N0 = N[0]
    ratio = np.where(N > 0, N / N0, 0.0)
    keep = (N > 0) & (ratio >= tau)
    keep[0] = False
    El = np.where(keep, U / np.where(N > 0, N, 1.0), 0.0)
    e2 = np.where(keep, ratio / np.where(keep, e0 - El, 1.0), 0.0)
    return e2, keep, ratio


def finalize(acc, e0, c, n_core, n_virt, tau=1e-10):
    """Point estimates and jackknife errors over the G walker groups."""
    N_g, U_g, W_g, E_g = acc["N"], acc["U"], acc["W"], acc["E"]
    G = N_g.shape[0]
    types = label_types(n_core, n_virt)
    N, U = N_g.sum(0), U_g.sum(0)
    Wt, Et = W_g.sum(), E_g.sum()

    def estimates(N, U, Wt, Et):
        e2l, keep, ratio = energies(N, U, e0, tau)
        tn = np.array([ratio[(types == t) & keep].sum() for t in range(N_TYPES)])
        te = np.array([e2l[types == t].sum() for t in range(N_TYPES)])
        return dict(e2=e2l.sum(), e_var=Et / Wt, a0sq=c[0] ** 2 * N[0] / Wt, type_norm=tn, type_e2=te,
                    keep=keep, ratio=ratio)

    full = estimates(N, U, Wt, Et)
    jk = [estimates(N - N_g[g], U - U_g[g], Wt - W_g[g], Et - E_g[g]) for g in range(G)] if G > 1 else []

    def sig(key):
        if not jk:
            return np.nan * np.asarray(full[key])
        v = np.array([j[key] for j in jk])
        return np.sqrt((G - 1) / G * ((v - v.mean(0)) ** 2).sum(0))

    keep = full["keep"]
    screened = (N > 0) & ~keep
    screened[0] = False
    res = dict(
        e0=e0, e2=full["e2"], e2_sigma=float(sig("e2")),
        e_var=full["e_var"], e_var_sigma=float(sig("e_var")),
        a0sq=full["a0sq"], a0sq_sigma=float(sig("a0sq")),
        type_norm=full["type_norm"], type_norm_sigma=sig("type_norm"),
        type_e2=full["type_e2"], type_e2_sigma=sig("type_e2"),
        type_screened=np.array([np.sum(screened & (types == t)) for t in range(N_TYPES)]),
        screened_norm=float(full["ratio"][screened].sum()),
        n_labels_visited=int(np.sum(N[1:] > 0)),
        type_steps=acc.get("type_steps"), walker_steps=acc.get("walker_steps"),
    )
    res["e_mrci_q"] = res["e_var"] + (1.0 - res["a0sq"]) * (res["e_var"] - e0)
    return res


def exact_from_brute(br, e0, c, n_core, n_virt, tau=1e-10):
    """Deterministic SC-NEVPT2 and sampling-function expectations from brute-force sums."""
    N, D = br["N"], br["D"]
    types = label_types(n_core, n_virt)
    e2l, keep, ratio = energies(N, D, e0, tau)
    return dict(
        e2=e2l.sum(),
        type_e2=np.array([e2l[types == t].sum() for t in range(N_TYPES)]),
        type_norm=np.array([ratio[(types == t) & keep].sum() for t in range(N_TYPES)]),
        E_l=np.where(keep, D / np.where(N > 0, N, 1), 0.0),
        e_var=br["psi_H_psi"] / br["psi_norm"],
        a0sq=c[0] ** 2 * N[0] / br["psi_norm"],
        rho_label=(c ** 2) * N / br["psi_norm"],
    )


# ------------------------------------------------------------------ SC-MRCI(s) optimisation (Sec. II B)

def mrci_gradient(acc):
    """Sampled energy gradient of Eq. 8 with the derivative overlaps of Eq. 9,
    g_l = < delta_{l,l_n} / c_l (E_L(n) - E) >, E = <E_L>, from the walk's residence-weighted
    sums A_l = sum w E_L / c_l and B_l = sum w / c_l (all groups).  Like Eq. 8 it leaves out the
    factor 2 of d(<psi|H|psi>/<psi|psi>)/dc_l for a real psi.  Returns (g, E)."""
    Wt, Et = acc["W"].sum(), acc["E"].sum()
    E = Et / Wt
    return (acc["A"].sum(0) - E * acc["B"].sum(0)) / Wt, E


def mrci_gradient_groups(acc):
    """The sampled gradient and its jackknife error over the walker groups."""
    A, B, W, E = acc["A"], acc["B"], acc["W"], acc["E"]
    G = A.shape[0]
    g, _ = mrci_gradient(acc)
    if G < 2:
        return g, np.full_like(g, np.nan)
    At, Bt, Wt, Et = A.sum(0), B.sum(0), W.sum(), E.sum()
    jk = []
    for k in range(G):
        e = (Et - E[k]) / (Wt - W[k])
        jk.append((At - A[k] - e * (Bt - B[k])) / (Wt - W[k]))
    jk = np.array(jk)
    return g, np.sqrt((G - 1) / G * ((jk - jk.mean(0)) ** 2).sum(0))


def exact_gradient(br, c):
    """Exact value of the same gradient for psi = sum_l c_l v_l from the label Hamiltonian
    H_ll' = <v_l|H|v_l'> and the diagonal overlap N_l = <v_l|v_l>:
    g = (H c - E N c) / (c^T N c), E = c^T H c / c^T N c.  Returns (g, E)."""
    H, N = br["H"], br["N"]
    nrm = c @ (N * c)
    E = c @ (H @ c) / nrm
    return (H @ c - E * N * c) / nrm, E


def sc_mrci(br):
    """SC-MRCI eigenproblem in the basis of strongly contracted states (Sec. II B): the lowest
    root of H c = E N c over the labels with N_l > 0.  Returns (E, c) with c_0 = 1."""
    H, N = br["H"], br["N"]
    keep = np.nonzero(N > 0)[0]
    s = 1.0 / np.sqrt(N[keep])
    Ht = s[:, None] * H[np.ix_(keep, keep)] * s[None, :]
    w, V = np.linalg.eigh(0.5 * (Ht + Ht.T))
    c = np.zeros(len(N))
    c[keep] = s * V[:, 0]
    return w[0], c / c[0]


def amsgrad(c, g, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One AMSGrad step (Reddi, Kale, Kumar, ICLR 2018, their Algorithm 2, no bias correction)
    on c_l for l >= 1, with eps in the denominator; c_0 stays fixed.  `state` holds m, v, vhat
    (zero at the start) and is updated in place.  Returns the new c."""
    m, v, vh = state["m"], state["v"], state["vhat"]
    m[1:] = beta1 * m[1:] + (1 - beta1) * g[1:]
    v[1:] = beta2 * v[1:] + (1 - beta2) * g[1:] ** 2
    vh[1:] = np.maximum(vh[1:], v[1:])
    c = c.copy()
    c[1:] -= lr * m[1:] / (np.sqrt(vh[1:]) + eps)
    return c


def amsgrad_state(n):
    return dict(m=np.zeros(n), v=np.zeros(n), vhat=np.zeros(n))
