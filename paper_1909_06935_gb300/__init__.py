"""GB300-native local-estimator path of stochastic SC-NEVPT2(s) / SC-MRCI(s) (arXiv:1909.06935).

Thin ctypes binding over the C ABI in include/mrq.h (library: _build/libmrq.so, built by
``build.build()``).  Arguments are marshalled here; every step of the computation runs in the
library's CUDA kernels.  There is no CPU fallback: loading fails loudly when the library is
missing or no CUDA device is visible.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = ["Context", "SampleParams", "Result", "Local", "Neighbour", "MRQError", "load_library", "NTYPES",
           "TYPE_NAMES", "n_labels", "batch_advance", "sample_batch"]

NTYPES = 9
NOALLOC_SCRATCH_DOUBLES = 1 << 19     # fixed scratch of mrq_finalize_noalloc (include/mrq.h)
TYPE_NAMES = ["CAS", "S_r", "S_rs", "S_i", "S_ir", "S_irs", "S_ij", "S_ijr", "S_ijrs"]   # index 3h + p
SC_NEVPT2, SC_MRCI = 0, 1


class SampleParams(C.Structure):
    _fields_ = [("n_walkers", C.c_int64), ("n_steps", C.c_int64), ("burn_in", C.c_int64), ("seed", C.c_uint64),
                ("n_groups", C.c_int32), ("method", C.c_int32), ("screen_tau", C.c_double),
                ("warps_per_walker", C.c_int32), ("steps_per_check", C.c_int32), ("target_sigma", C.c_double)]


class Result(C.Structure):
    _fields_ = [("e0", C.c_double), ("e2", C.c_double), ("e2_sigma", C.c_double), ("e_var", C.c_double),
                ("e_var_sigma", C.c_double), ("a0sq", C.c_double), ("a0sq_sigma", C.c_double),
                ("e_mrci_q", C.c_double),
                ("type_norm", C.c_double * NTYPES), ("type_norm_sigma", C.c_double * NTYPES),
                ("type_e2", C.c_double * NTYPES), ("type_e2_sigma", C.c_double * NTYPES),
                ("type_screened", C.c_double * NTYPES), ("screened_norm", C.c_double),
                ("n_labels_visited", C.c_double), ("type_steps", C.c_int64 * NTYPES),
                ("walker_steps", C.c_int64), ("total_steps", C.c_int64), ("seconds", C.c_double),
                ("walk_launches", C.c_int64), ("status", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = np.array(v[:]) if hasattr(v, "_length_") else v
        return out


class Local(C.Structure):
    _fields_ = [("S", C.c_double), ("e_local", C.c_double), ("num", C.c_double), ("h_nn", C.c_double),
                ("hd_nn", C.c_double), ("psi", C.c_double), ("label", C.c_int64), ("type", C.c_int64),
                ("n_neighbours", C.c_int64), ("n_candidates", C.c_int64), ("n_probes", C.c_int64),
                ("n_gathers", C.c_int64), ("n_terms", C.c_int64)]


class Neighbour(C.Structure):
    _fields_ = [("det", C.c_uint64 * 4), ("h", C.c_double), ("hd", C.c_double), ("o", C.c_double),
                ("psi", C.c_double), ("gamma", C.c_double), ("exc", C.c_uint32), ("pad", C.c_uint32)]


_NB_DTYPE = np.dtype([("det", np.uint64, 4), ("h", np.float64), ("hd", np.float64), ("o", np.float64),
                      ("psi", np.float64), ("gamma", np.float64), ("exc", np.uint32), ("pad", np.uint32)])
_LOCAL_DTYPE = np.dtype([("S", np.float64), ("e_local", np.float64), ("num", np.float64), ("h_nn", np.float64),
                         ("hd_nn", np.float64), ("psi", np.float64), ("label", np.int64), ("type", np.int64),
                         ("n_neighbours", np.int64), ("n_candidates", np.int64), ("n_probes", np.int64),
                         ("n_gathers", np.int64), ("n_terms", np.int64)])
assert _NB_DTYPE.itemsize == C.sizeof(Neighbour) and _LOCAL_DTYPE.itemsize == C.sizeof(Local)


TUNE_MAX = 16


class TuneResult(C.Structure):
    _fields_ = [("warps_per_walker", C.c_int32), ("steps_per_launch", C.c_int32), ("n_tried", C.c_int32),
                ("tried_warps_per_walker", C.c_int32 * TUNE_MAX), ("tried_steps_per_launch", C.c_int32 * TUNE_MAX),
                ("tried_ms", C.c_double * TUNE_MAX)]

    def as_dict(self):
        n = self.n_tried
        return dict(warps_per_walker=self.warps_per_walker, steps_per_launch=self.steps_per_launch,
                    tried=[(self.tried_warps_per_walker[i], self.tried_steps_per_launch[i], self.tried_ms[i])
                           for i in range(n)])


class SciParams(C.Structure):
    _fields_ = [("n_strings", C.c_int32), ("n_seed_strings", C.c_int32), ("tol", C.c_double),
                ("max_iter", C.c_int32), ("max_sub", C.c_int32), ("semicanonical", C.c_int32),
                ("reserved", C.c_int32)]


class SciResult(C.Structure):
    _fields_ = [("energy", C.c_double), ("seed_energy", C.c_double), ("residual", C.c_double),
                ("fock_offdiag", C.c_double), ("seconds", C.c_double), ("n_det", C.c_int64),
                ("n_strings", C.c_int32), ("n_seed_strings", C.c_int32), ("iters_seed", C.c_int32),
                ("iters", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MRQError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mrq error {code}: {msg}")
        self.code = code


_lib = None


def load_library(build_if_missing: bool = True):
    """Load _build/libmrq.so (building it with nvcc when missing).  Raises when it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"CUDA library not built: {path}")
        _build.build()
    lib = C.CDLL(path)
    P, I64 = C.c_void_p, C.c_int64
    lib.mrq_create.argtypes = [C.POINTER(C.c_void_p), C.c_int]
    lib.mrq_destroy.argtypes = [P]
    lib.mrq_destroy.restype = None
    lib.mrq_last_error.argtypes = [P]
    lib.mrq_last_error.restype = C.c_char_p
    lib.mrq_set_stream.argtypes = [P, P]
    lib.mrq_load_hamiltonian.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P, P, C.c_double]
    lib.mrq_load_reference.argtypes = [P, I64, P, P]
    lib.mrq_set_coeffs.argtypes = [P, I64, P]
    lib.mrq_n_labels.argtypes = [P]
    lib.mrq_n_labels.restype = I64
    lib.mrq_setup_info.argtypes = [P, P, P, P]
    lib.mrq_debug_local.argtypes = [P, I64, P, P, I64, P]
    lib.mrq_walkers_init.argtypes = [P, C.POINTER(SampleParams)]
    lib.mrq_walkers_advance.argtypes = [P, I64]
    lib.mrq_finalize.argtypes = [P, C.POINTER(Result)]
    lib.mrq_finalize_noalloc.argtypes = [P, C.POINTER(Result)]
    lib.mrq_sample.argtypes = [P, C.POINTER(SampleParams), C.POINTER(Result)]
    lib.mrq_read_accumulators.argtypes = [P, P, P, P, P, P]
    lib.mrq_read_walkers.argtypes = [P, P, P]
    lib.mrq_batch_advance.argtypes = [P, C.c_int, I64]
    lib.mrq_set_launch.argtypes = [P, C.c_int, C.c_int, C.c_int]
    lib.mrq_tune_batch.argtypes = [P, C.c_int, I64, P]
    lib.mrq_mrci_gradient.argtypes = [P, P, P]
    lib.mrq_amsgrad_step.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_double]
    lib.mrq_read_coeffs.argtypes = [P, P]
    lib.mrq_read_gradient_sums.argtypes = [P, P, P]
    lib.mrq_sample_batch.argtypes = [P, C.c_int, P, P]
    lib.mrq_debug_race_screen.argtypes = [P, I64, P, P, P, P, P]
    lib.mrq_set_deadline.argtypes = [P, C.c_double]
    lib.mrq_probe_peaks.argtypes = [C.c_int, P]
    lib.mrq_set_l2_window.argtypes = [P, C.c_double]
    lib.mrq_debug_set_limits.argtypes = [P, C.c_int, C.c_int]
    lib.mrq_read_hamiltonian.argtypes = [P, P, P]
    lib.mrq_set_heat_bath_cutoff.argtypes = [P, C.c_double]
    lib.mrq_load_accumulators.argtypes = [P, C.c_int32, P, P, P, P, P, P, P, I64]
    lib.mrq_sci_reference.argtypes = [P, C.POINTER(SciParams), C.POINTER(SciResult), P, P]
    for fn in ("mrq_create", "mrq_set_stream", "mrq_load_hamiltonian", "mrq_load_reference", "mrq_set_coeffs",
               "mrq_setup_info", "mrq_debug_local", "mrq_walkers_init", "mrq_walkers_advance", "mrq_finalize",
               "mrq_finalize_noalloc", "mrq_batch_advance", "mrq_sample_batch", "mrq_mrci_gradient",
               "mrq_amsgrad_step", "mrq_read_coeffs", "mrq_read_gradient_sums", "mrq_sample", "mrq_set_launch",
               "mrq_tune_batch", "mrq_read_accumulators", "mrq_read_walkers", "mrq_debug_race_screen",
               "mrq_set_deadline", "mrq_debug_set_limits", "mrq_probe_peaks",
               "mrq_set_l2_window", "mrq_read_hamiltonian", "mrq_sci_reference", "mrq_load_accumulators", "mrq_set_heat_bath_cutoff"):
        getattr(lib, fn).restype = C.c_int
    _lib = lib
    return lib


def probe_peaks(device: int = 0) -> dict:
    """Measured FP64 FMA rate and random 8-byte read rates (L2- and HBM-resident tables) of the device."""
    lib = load_library()
    out = np.zeros(3)
    rc = lib.mrq_probe_peaks(device, out.ctypes.data_as(C.c_void_p))
    if rc:
        raise MRQError(rc, "mrq_probe_peaks failed")
    return dict(fp64_flops=float(out[0]), l2_gathers_per_s=float(out[1]), hbm_gathers_per_s=float(out[2]))


def n_labels(n_core: int, n_virt: int) -> int:
    nh = 1 + 2 * n_core + (2 * n_core) * (2 * n_core - 1) // 2
    npart = 1 + 2 * n_virt + (2 * n_virt) * (2 * n_virt - 1) // 2
    return nh * npart


def reblock(x, min_blocks: int = 16):
    """Flyvbjerg-Petersen blocking analysis of a correlated time series (the cross-check of the
    jackknife error bars over walker groups): at level k the series is averaged in pairs k times,
    and the standard error of the mean is estimated as if the blocks were independent, with its own
    uncertainty se / sqrt(2 (n_k - 1)).  The estimate grows with k until the blocks are longer than
    the correlation time, then stays on a plateau; the returned `sigma` is the first level (with at
    least min_blocks blocks) whose estimate the next level does not exceed by more than this
    uncertainty, else the largest estimate among the levels with at least min_blocks blocks.
    Returns dict(levels=[(n_blocks, se, d_se), ...], sigma, level)."""
    x = np.asarray(x, dtype=np.float64).ravel()
    levels = []
    while len(x) >= 2:
        n = len(x)
        se = float(np.sqrt(np.mean((x - x.mean()) ** 2) / (n - 1)))
        levels.append((n, se, se / np.sqrt(2.0 * (n - 1))))
        if n % 2:
            x = x[:-1]
        x = 0.5 * (x[0::2] + x[1::2])
    ok = [k for k, lv in enumerate(levels) if lv[0] >= min_blocks]
    if not ok:
        return dict(levels=levels, sigma=float("nan"), level=-1)
    for k in ok[:-1]:
        if levels[k + 1][1] <= levels[k][1] + levels[k][2]:
            return dict(levels=levels, sigma=levels[k][1], level=k)
    k = max(ok, key=lambda i: levels[i][1])
    return dict(levels=levels, sigma=levels[k][1], level=k)


def reblock_ratio(num, den, min_blocks: int = 16):
    """Blocking analysis of R = sum(num) / sum(den) from per-block sums (e.g. E_var = sum w E_L /
    sum w, a0^2 = c0^2 sum w delta_CAS / sum w): the linearised series (num_b - R den_b) / mean(den)
    has the error of R as the standard error of its mean.  Returns reblock()'s dict plus R."""
    num = np.asarray(num, dtype=np.float64).ravel()
    den = np.asarray(den, dtype=np.float64).ravel()
    R = float(num.sum() / den.sum())
    out = reblock((num - R * den) / den.mean(), min_blocks)
    out["R"] = R
    return out


def frozen_core_coeffs(c, n_core: int, n_virt: int):
    """Sampling coefficients of the frozen-core variant (the paper's own implementation, Sec. II D):
    c_l = 0 for every label with a core hole, so that psi_s vanishes on core-excited determinants,
    walkers never reach them and only the (0,1) and (0,2) classes are sampled.  Label
    l = rank(H) n_P + rank(P), so the labels with core holes are l >= n_P."""
    c = np.array(c, dtype=np.float64, copy=True)
    if len(c) != n_labels(n_core, n_virt):
        raise ValueError("coefficient vector does not match the label count")
    n_p = 1 + 2 * n_virt + (2 * n_virt) * (2 * n_virt - 1) // 2
    c[n_p:] = 0.0
    return c


def _addr(a):
    """Address of a host numpy array or a CUDA torch tensor (unified addressing)."""
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _host(a, dtype):
    if hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=dtype)


class Context:
    """One device-resident system (Hamiltonian, reference, coefficients, walkers)."""

    def __init__(self, device: int = 0):
        self._lib = load_library()
        h = C.c_void_p()
        rc = self._lib.mrq_create(C.byref(h), device)
        if rc:
            raise MRQError(rc, "mrq_create failed (no CUDA device?)")
        self._h = h
        self.W = 1
        self.n_core = self.n_act = self.n_virt = 0

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mrq_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc):
        if rc:
            raise MRQError(rc, self._lib.mrq_last_error(self._h).decode())

    def set_stream(self, stream_ptr: int | None):
        self._check(self._lib.mrq_set_stream(self._h, C.c_void_p(stream_ptr or 0)))

    def load_hamiltonian(self, n_core, n_act, n_virt, n_alpha, n_beta, h1, eri, e_core=0.0):
        h1a, eria = _host(h1, np.float64), _host(eri, np.float64)
        self._check(self._lib.mrq_load_hamiltonian(self._h, n_core, n_act, n_virt, n_alpha, n_beta, _addr(h1a),
                                                   _addr(eria), float(e_core)))
        self.n_core, self.n_act, self.n_virt = n_core, n_act, n_virt
        self.n = n_core + n_act + n_virt
        self.W = (self.n + 63) // 64

    def load_reference(self, dets, coeffs):
        d, c = _host(dets, np.uint64), _host(coeffs, np.float64)
        self._check(self._lib.mrq_load_reference(self._h, len(c), _addr(d), _addr(c)))

    def set_coeffs(self, c):
        ca = _host(c, np.float64)
        self._check(self._lib.mrq_set_coeffs(self._h, len(ca), _addr(ca)))

    @property
    def n_labels(self) -> int:
        return int(self._lib.mrq_n_labels(self._h))

    def setup_info(self):
        out = np.zeros(5)
        eps = np.zeros(self.n)
        gam = np.zeros(max(self.n_act, 1) ** 2)
        self._check(self._lib.mrq_setup_info(self._h, _addr(out), _addr(eps), _addr(gam)))
        return dict(e0=out[0], norm0=out[1], e_core=out[2], sum_eps_core=out[3], start=int(out[4]), eps=eps,
                    gamma=gam[: self.n_act ** 2].reshape(self.n_act, self.n_act))

    @classmethod
    def from_system(cls, s, device: int = 0, c=None):
        ctx = cls(device)
        ctx.load_hamiltonian(s.n_core, s.n_act, s.n_virt, s.n_alpha, s.n_beta, s.h1, s.eri, s.e_nuc)
        ctx.load_reference(s.dets, s.coeffs)
        ctx.set_coeffs(s.c if c is None else c)
        return ctx

    def debug_local(self, dets, max_nb: int = 0):
        d = np.ascontiguousarray(dets, np.uint64).reshape(-1, 2 * self.W)
        n = d.shape[0]
        loc = np.zeros(n, _LOCAL_DTYPE)
        nb = np.zeros(n * max_nb, _NB_DTYPE) if max_nb else None
        self._check(self._lib.mrq_debug_local(self._h, n, _addr(d), _addr(loc), max_nb,
                                              _addr(nb) if max_nb else None))
        return loc, (nb.reshape(n, max_nb) if max_nb else None)

    def params(self, n_walkers, n_steps, burn_in=0, seed=1, n_groups=16, screen_tau=1e-10, method=SC_NEVPT2,
               warps_per_walker=0, target_sigma=0.0, steps_per_check=0):
        return SampleParams(n_walkers, n_steps, burn_in, seed, n_groups, method, screen_tau, warps_per_walker,
                            steps_per_check, target_sigma)

    def walkers_init(self, p: SampleParams):
        self._check(self._lib.mrq_walkers_init(self._h, C.byref(p)))

    def walkers_advance(self, n_steps: int):
        self._check(self._lib.mrq_walkers_advance(self._h, n_steps))

    def finalize(self) -> dict:
        r = Result()
        self._check(self._lib.mrq_finalize(self._h, C.byref(r)))
        return r.as_dict()

    def finalize_noalloc(self) -> dict:
        """mrq_finalize without any device allocation (fixed scratch inside the library)."""
        r = Result()
        self._check(self._lib.mrq_finalize_noalloc(self._h, C.byref(r)))
        return r.as_dict()

    def sample(self, p: SampleParams) -> dict:
        r = Result()
        self._check(self._lib.mrq_sample(self._h, C.byref(p), C.byref(r)))
        return r.as_dict()

    def accumulators(self, n_groups: int):
        L = self.n_labels
        N = np.zeros((n_groups, L))
        U = np.zeros((n_groups, L))
        Wg = np.zeros(n_groups)
        E = np.zeros(n_groups)
        ts = np.zeros(NTYPES, np.int64)
        self._check(self._lib.mrq_read_accumulators(self._h, _addr(N), _addr(U), _addr(Wg), _addr(E), _addr(ts)))
        return dict(N=N, U=U, W=Wg, E=E, type_steps=ts)

    def load_accumulators(self, acc, total_steps: int = 0):
        """Replace the accumulators by given per-group sums (dict with N, U, W, E, type_steps and
        optionally A, B), e.g. the concatenated groups of several ranks; finalize() then combines them."""
        N = np.ascontiguousarray(acc["N"], np.float64)
        G = N.shape[0]
        U = np.ascontiguousarray(acc["U"], np.float64)
        Wg = np.ascontiguousarray(acc["W"], np.float64)
        E = np.ascontiguousarray(acc["E"], np.float64)
        ts = np.ascontiguousarray(acc["type_steps"], np.int64)
        A = np.ascontiguousarray(acc["A"], np.float64) if acc.get("A") is not None else None
        B = np.ascontiguousarray(acc["B"], np.float64) if acc.get("B") is not None else None
        if U.shape != N.shape or N.shape[1] != self.n_labels or Wg.shape != (G,) or E.shape != (G,) or ts.shape != (NTYPES,):
            raise ValueError("accumulator shapes do not match the loaded system")
        self._check(self._lib.mrq_load_accumulators(self._h, G, _addr(N), _addr(U), _addr(Wg), _addr(E),
                                                    _addr(A) if A is not None else None,
                                                    _addr(B) if B is not None else None, _addr(ts),
                                                    int(total_steps)))

    def set_launch(self, warps_per_walker=0, steps_per_launch=0, use_graph=False):
        """Walk launch configuration: warps per walker block (0 = chosen from the system's size),
        steps per launch (0 = one launch per advance), CUDA-graph replay of batched reporting
        intervals."""
        self._check(self._lib.mrq_set_launch(self._h, warps_per_walker, steps_per_launch, int(bool(use_graph))))

    def mrci_gradient(self):
        """SC-MRCI(s) gradient (Eq. 8-9) of the last walk and the energy estimate."""
        g = np.zeros(self.n_labels)
        e = C.c_double(0.0)
        self._check(self._lib.mrq_mrci_gradient(self._h, _addr(g), C.byref(e)))
        return g, e.value

    def amsgrad_step(self, lr=0.01, beta1=0.9, beta2=0.999, eps=1e-8):
        """One AMSGrad update of the device coefficients from the last gradient."""
        self._check(self._lib.mrq_amsgrad_step(self._h, lr, beta1, beta2, eps))

    def coeffs(self):
        c = np.zeros(self.n_labels)
        self._check(self._lib.mrq_read_coeffs(self._h, _addr(c)))
        return c

    def gradient_sums(self, n_groups: int):
        """Per-group sums A[g, l] = sum w E_L / c_l and B[g, l] = sum w / c_l of the last walk."""
        a = np.zeros((n_groups, self.n_labels))
        b = np.zeros((n_groups, self.n_labels))
        self._check(self._lib.mrq_read_gradient_sums(self._h, _addr(a), _addr(b)))
        return a, b

    def optimize_mrci(self, n_iter, n_walkers, n_steps, burn_in=20, lr=0.01, seed=1, n_groups=8,
                      beta1=0.9, beta2=0.999, eps=1e-8):
        """SC-MRCI(s) by AMSGrad (Sec. II B): each iteration walks psi = sum_l c_l psi_l with the
        current coefficients, takes the sampled gradient and updates c on the device.  Returns the
        result of every iteration's walk (its e_var is the energy of the c it walked with)."""
        hist = []
        for it in range(n_iter):
            res = self.sample(self.params(n_walkers, n_steps, burn_in=burn_in, seed=seed + it, n_groups=n_groups))
            self.mrci_gradient()
            self.amsgrad_step(lr, beta1, beta2, eps)
            hist.append(res)
        return hist

    def set_l2_window(self, fraction: float):
        """Mark the integral tables persisting in L2 for this context's walks (0 turns it off)."""
        self._check(self._lib.mrq_set_l2_window(self._h, float(fraction)))

    def set_deadline(self, seconds: float):
        """Host waits of this context give up after `seconds` (0: no deadline) with MRQError(-6)."""
        self._check(self._lib.mrq_set_deadline(self._h, float(seconds)))

    def debug_set_limits(self, max_probe: int = 0, cand_cap: int = 0):
        """Lower the hash-probe bound and the candidate-list capacity (0 restores the default)."""
        self._check(self._lib.mrq_debug_set_limits(self._h, int(max_probe), int(cand_cap)))

    def race_screen(self, k53, rate, t_best):
        """The move race's FP32 screen (pass flags) and exact FP64 clocks for (k53, rate, best) triples."""
        k = np.ascontiguousarray(k53, np.uint64)
        r = np.ascontiguousarray(rate, np.float64)
        tb = np.ascontiguousarray(t_best, np.float64)
        if k.shape != r.shape or k.shape != tb.shape:
            raise ValueError("k53, rate and t_best must have the same shape")
        ok = np.zeros(k.shape, np.uint8)
        ex = np.zeros(k.shape, np.float64)
        self._check(self._lib.mrq_debug_race_screen(self._h, k.size, _addr(k), _addr(r), _addr(tb), _addr(ok),
                                                    _addr(ex)))
        return ok.astype(bool), ex

    def set_heat_bath_cutoff(self, eps: float):
        """Drop double excitations with |<ab||ij>| < eps from the walk (0: exact)."""
        self._check(self._lib.mrq_set_heat_bath_cutoff(self._h, float(eps)))

    def read_hamiltonian(self):
        """The loaded integrals (h1 as n x n, the packed eri)."""
        npair = self.n * (self.n + 1) // 2
        h1 = np.zeros((self.n, self.n))
        eri = np.zeros(npair * (npair + 1) // 2)
        self._check(self._lib.mrq_read_hamiltonian(self._h, _addr(h1), _addr(eri)))
        return h1, eri

    def sci_reference(self, n_strings, n_seed_strings=256, tol=1e-5, max_iter=80, max_sub=24,
                      semicanonical=True, want_vectors=True):
        """Build and load the heat-bath selected-CI reference on the device (mrq_sci_reference).
        Returns the result fields, plus the selected strings and the coefficients (n_strings^2)
        when want_vectors."""
        p = SciParams(int(n_strings), int(n_seed_strings), float(tol), int(max_iter), int(max_sub),
                      1 if semicanonical else 0, 0)
        r = SciResult()
        m = n_strings
        strs = np.zeros(m, np.uint32) if want_vectors else None
        cs = np.zeros(m * m) if want_vectors else None
        self._check(self._lib.mrq_sci_reference(self._h, C.byref(p), C.byref(r),
                                                _addr(strs) if want_vectors else None,
                                                _addr(cs) if want_vectors else None))
        out = r.as_dict()
        if want_vectors:
            k = r.n_strings
            out["strings"] = strs[:k].astype(np.int64)
            out["coeffs"] = cs[: k * k].reshape(k, k)
        return out

    def walkers(self, n_walkers: int):
        d = np.zeros((n_walkers, 2 * self.W), np.uint64)
        psi = np.zeros(n_walkers)
        self._check(self._lib.mrq_read_walkers(self._h, _addr(d), _addr(psi)))
        return d, psi


def _ctx_array(ctxs):
    arr = (C.c_void_p * len(ctxs))(*[c._h.value for c in ctxs])
    return arr


def batch_advance(ctxs, n_steps: int):
    """Advance the walkers of several contexts together (one walk launch per determinant width and
    occupancy class)."""
    lib = load_library()
    rc = lib.mrq_batch_advance(C.cast(_ctx_array(ctxs), C.c_void_p), len(ctxs), n_steps)
    if rc:
        raise MRQError(rc, lib.mrq_last_error(ctxs[0]._h).decode())


def tune_batch(ctxs, trial_steps: int = 4):
    """Autotune walkers per block and steps per launch for this batch (on scratch walkers; the
    contexts' state is unchanged) and set the fastest on every context.  Returns the timings."""
    lib = load_library()
    out = TuneResult()
    rc = lib.mrq_tune_batch(C.cast(_ctx_array(ctxs), C.c_void_p), len(ctxs), trial_steps, C.byref(out))
    if rc:
        raise MRQError(rc, lib.mrq_last_error(ctxs[0]._h).decode())
    return out.as_dict()


def sample_batch(ctxs, params):
    """mrq_sample_batch: init, one batched advance, finalize each; returns the result dicts."""
    lib = load_library()
    n = len(ctxs)
    parr = (SampleParams * n)(*params)
    res = (Result * n)()
    rc = lib.mrq_sample_batch(C.cast(_ctx_array(ctxs), C.c_void_p), n, C.cast(parr, C.c_void_p),
                              C.cast(res, C.c_void_p))
    if rc:
        raise MRQError(rc, lib.mrq_last_error(ctxs[0]._h).decode())
    return [r.as_dict() for r in res]


# ------------------------------------------------------------------ request server

class ServerParams(C.Structure):
    _fields_ = [("device", C.c_int32), ("max_active", C.c_int32), ("hbm_budget_bytes", C.c_int64),
                ("steps_per_round", C.c_int64)]


class Request(C.Structure):
    _fields_ = [("n_core", C.c_int32), ("n_act", C.c_int32), ("n_virt", C.c_int32), ("n_alpha", C.c_int32),
                ("n_beta", C.c_int32), ("reserved", C.c_int32), ("e_core", C.c_double), ("h1", C.c_void_p),
                ("eri", C.c_void_p), ("n_det", C.c_int64), ("dets", C.c_void_p), ("coeffs", C.c_void_p),
                ("n_labels", C.c_int64), ("c", C.c_void_p), ("params", SampleParams),
                ("target_sigma", C.c_double), ("max_steps", C.c_int64)]


class RequestStatus(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("steps_done", C.c_int64),
                ("queue_seconds", C.c_double), ("total_seconds", C.c_double), ("result", Result)]


REQ_STATES = ["queued", "running", "done", "failed", "cancelled"]


def _server_lib():
    lib = load_library()
    if not getattr(lib, "_server_typed", False):
        P = C.c_void_p
        lib.mrq_server_create.argtypes = [C.POINTER(C.c_void_p), C.POINTER(ServerParams)]
        lib.mrq_server_submit.argtypes = [P, C.POINTER(Request), C.POINTER(C.c_int64)]
        lib.mrq_server_poll.argtypes = [P, C.c_int64, C.POINTER(RequestStatus)]
        lib.mrq_server_cancel.argtypes = [P, C.c_int64]
        lib.mrq_server_step.argtypes = [P]
        lib.mrq_server_start.argtypes = [P]
        lib.mrq_server_stop.argtypes = [P]
        lib.mrq_server_info.argtypes = [P, P]
        lib.mrq_server_last_error.argtypes = [P]
        lib.mrq_server_last_error.restype = C.c_char_p
        lib.mrq_server_destroy.argtypes = [P]
        lib.mrq_server_destroy.restype = None
        for fn in ("mrq_server_create", "mrq_server_submit", "mrq_server_poll", "mrq_server_cancel",
                   "mrq_server_step", "mrq_server_start", "mrq_server_stop", "mrq_server_info"):
            getattr(lib, fn).restype = C.c_int
        lib._server_typed = True
    return lib


class Server:
    """Request server: continuous batching of sampling requests on one device."""

    def __init__(self, device=0, max_active=16, hbm_budget_bytes=64 << 30, steps_per_round=1):
        self._lib = _server_lib()
        h = C.c_void_p()
        rc = self._lib.mrq_server_create(C.byref(h), C.byref(ServerParams(device, max_active, hbm_budget_bytes,
                                                                          steps_per_round)))
        if rc:
            raise MRQError(rc, "mrq_server_create failed")
        self._h = h
        self._keep = {}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mrq_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def submit(self, s, n_walkers, max_steps, target_sigma=0.0, burn_in=0, seed=1, n_groups=16,
               screen_tau=1e-10, c=None):
        arrays = [np.ascontiguousarray(s.h1, np.float64), np.ascontiguousarray(s.eri, np.float64),
                  np.ascontiguousarray(s.dets, np.uint64), np.ascontiguousarray(s.coeffs, np.float64),
                  np.ascontiguousarray(s.c if c is None else c, np.float64)]
        h1, eri, dets, co, cc = arrays
        req = Request(s.n_core, s.n_act, s.n_virt, s.n_alpha, s.n_beta, 0, float(s.e_nuc), _addr(h1).value,
                      _addr(eri).value, len(co), _addr(dets).value, _addr(co).value, len(cc), _addr(cc).value,
                      SampleParams(n_walkers, 0, burn_in, seed, n_groups, 0, screen_tau, 0, 0, 0.0),
                      float(target_sigma), int(max_steps))
        t = C.c_int64(0)
        rc = self._lib.mrq_server_submit(self._h, C.byref(req), C.byref(t))
        if rc:
            raise MRQError(rc, "mrq_server_submit rejected the request")
        return t.value

    def poll(self, ticket):
        st = RequestStatus()
        rc = self._lib.mrq_server_poll(self._h, ticket, C.byref(st))
        if rc:
            raise MRQError(rc, "unknown ticket")
        return dict(state=REQ_STATES[st.state], status=st.status, steps_done=st.steps_done,
                    queue_seconds=st.queue_seconds, total_seconds=st.total_seconds, result=st.result.as_dict())

    def cancel(self, ticket):
        rc = self._lib.mrq_server_cancel(self._h, ticket)
        if rc:
            raise MRQError(rc, "unknown ticket")

    def step(self):
        rc = self._lib.mrq_server_step(self._h)
        if rc:
            raise MRQError(rc, self._lib.mrq_server_last_error(self._h).decode())

    def start(self):
        self._lib.mrq_server_start(self._h)

    def stop(self):
        self._lib.mrq_server_stop(self._h)

    def info(self):
        out = np.zeros(4, np.int64)
        self._lib.mrq_server_info(self._h, out.ctypes.data_as(C.c_void_p))
        return dict(queued=int(out[0]), active=int(out[1]), bytes=int(out[2]), walker_steps=int(out[3]))
