"""ctypes front end of the plain FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module; the product path
(``paper_1108_0900_gb300``) never does, and the two share no code.  The only
thing both sides consume is the seeded problem description from
``paper_1108_0900_gb300.inputs`` (plain arrays, none of the method's
arithmetic).
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP over walkers / samples)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Problem(ct.Structure):
    _fields_ = [
        ("n_sites", ct.c_int), ("n_up", ct.c_int), ("n_dn", ct.c_int), ("ham", ct.c_int),
        ("n_bonds", ct.c_int), ("bonds", ct.c_void_p), ("bond_t", ct.c_void_p),
        ("U", ct.c_double), ("n_chol", ct.c_int), ("h", ct.c_void_p), ("chol", ct.c_void_p),
        ("n_corr", ct.c_int), ("corr_ptr", ct.c_void_p), ("corr_sites", ct.c_void_p),
        ("corr_class", ct.c_void_p), ("C", ct.c_void_p), ("f", ct.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ct.CDLL(build())
            vp, i64, i32, dbl = ct.c_void_p, ct.c_int64, ct.c_int, ct.c_double
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_pfaffian.argtypes = [i32, vp, vp, vp]
            L.orc_inverse.argtypes = [i32, vp, vp]
            L.orc_inverse.restype = i32
            L.orc_n_params.argtypes = [vp]
            L.orc_n_params.restype = i64
            L.orc_n_corr_params.argtypes = [vp]
            L.orc_n_corr_params.restype = i64
            L.orc_corr_state.argtypes = [vp, vp, i32]
            L.orc_corr_state.restype = i64
            L.orc_log_psi.argtypes = [vp, vp, vp, vp]
            L.orc_logderiv.argtypes = [vp, vp, vp]
            L.orc_logderiv.restype = i32
            L.orc_hamiltonian_element.argtypes = [vp, vp, vp]
            L.orc_hamiltonian_element.restype = dbl
            L.orc_local_energy.argtypes = [vp, vp]
            L.orc_local_energy.restype = dbl
            L.orc_local_energy_abinitio_bruteforce.argtypes = [vp, vp]
            L.orc_local_energy_abinitio_bruteforce.restype = dbl
            L.orc_sample.argtypes = [vp, i32, vp, vp, ct.c_uint64, i32, i32, vp, vp, vp, dbl, vp]
            L.orc_sample.restype = i32
            L.orc_measure.argtypes = [vp, i64, vp, vp, vp]
            L.orc_measure.restype = i32
            L.orc_mean_O.argtypes = [i64, i64, vp, vp]
            L.orc_gradient.argtypes = [i64, i64, vp, vp, vp, vp]
            L.orc_dense_S.argtypes = [i64, i64, vp, vp]
            L.orc_apply_S.argtypes = [i64, i64, vp, vp, vp, dbl, vp]
            L.orc_cg.argtypes = [i64, i64, vp, vp, dbl, dbl, i32, vp, vp, vp]
            L.orc_cg.restype = i32
            L.orc_sr_update.argtypes = [i64, vp, vp, dbl, dbl, vp, vp]
            L.orc_sr_update.restype = dbl
            L.orc_sector_size.argtypes = [vp]
            L.orc_sector_size.restype = i64
            L.orc_enumerate.argtypes = [vp, vp]
            L.orc_enumerate.restype = i64
            L.orc_exact_weights.argtypes = [vp, i64, vp, vp]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ct.c_void_p) if a is not None else None


class Problem:
    """Holds the ctypes problem struct and keeps its arrays alive."""

    def __init__(self, wl):
        self.wl = wl
        self._keep = dict(
            bonds=np.ascontiguousarray(wl.bonds, np.int32),
            bond_t=np.ascontiguousarray(wl.bond_t, np.float64),
            corr_ptr=np.ascontiguousarray(wl.corr_ptr, np.int32),
            corr_sites=np.ascontiguousarray(wl.corr_flat, np.int32),
            corr_class=None if getattr(wl, "corr_class", None) is None
            else np.ascontiguousarray(wl.corr_class, np.int32),
            C=np.ascontiguousarray(wl.C, np.float64),
            f=np.ascontiguousarray(wl.f, np.float64),
            h=None if wl.h is None else np.ascontiguousarray(wl.h, np.float64),
            chol=None if wl.chol is None else np.ascontiguousarray(wl.chol, np.float64),
        )
        k = self._keep
        self.s = _Problem(
            n_sites=wl.n_sites, n_up=wl.n_up, n_dn=wl.n_dn, ham=wl.ham,
            n_bonds=len(k["bonds"]), bonds=_ptr(k["bonds"]), bond_t=_ptr(k["bond_t"]),
            U=float(wl.U), n_chol=0 if wl.chol is None else wl.chol.shape[0],
            h=_ptr(k["h"]), chol=_ptr(k["chol"]),
            n_corr=wl.n_corr, corr_ptr=_ptr(k["corr_ptr"]), corr_sites=_ptr(k["corr_sites"]),
            corr_class=_ptr(k["corr_class"]), C=_ptr(k["C"]), f=_ptr(k["f"]))

    @property
    def ref(self):
        return ct.byref(self.s)

    # --- wavefunction ------------------------------------------------------
    def n_params(self) -> int:
        return int(lib().orc_n_params(self.ref))

    def n_corr_params(self) -> int:
        return int(lib().orc_n_corr_params(self.ref))

    def corr_state(self, occ, c: int) -> int:
        occ = np.ascontiguousarray(occ, np.uint8)
        return int(lib().orc_corr_state(self.ref, _ptr(occ), c))

    def log_psi(self, occ):
        occ = np.ascontiguousarray(occ, np.uint8)
        la = ct.c_double()
        sg = ct.c_int()
        lib().orc_log_psi(self.ref, _ptr(occ), ct.byref(la), ct.byref(sg))
        return la.value, sg.value

    def logderiv(self, occ) -> np.ndarray:
        occ = np.ascontiguousarray(occ, np.uint8)
        O = np.zeros(self.n_params())
        if lib().orc_logderiv(self.ref, _ptr(occ), _ptr(O)) != 0:
            raise ArithmeticError("singular pairing submatrix")
        return O

    def local_energy(self, occ) -> float:
        occ = np.ascontiguousarray(occ, np.uint8)
        return float(lib().orc_local_energy(self.ref, _ptr(occ)))

    def local_energy_bruteforce(self, occ) -> float:
        occ = np.ascontiguousarray(occ, np.uint8)
        return float(lib().orc_local_energy_abinitio_bruteforce(self.ref, _ptr(occ)))

    def hamiltonian_element(self, occ_n, occ_np) -> float:
        a = np.ascontiguousarray(occ_n, np.uint8)
        b = np.ascontiguousarray(occ_np, np.uint8)
        return float(lib().orc_hamiltonian_element(self.ref, _ptr(a), _ptr(b)))

    # --- sampling ------------------------------------------------------------
    def sample(self, occ, step, seed: int, n_burn: int, n_spw: int, close_tol: float = 0.0,
               return_first_close: bool = False):
        """Advance every walker in place; returns (samples, min_margin, accepts)
        and, on request, the index of each walker's first proposal whose
        relative acceptance margin was below close_tol (-1 if none)."""
        assert occ.dtype == np.uint8 and occ.flags.c_contiguous
        assert step.dtype == np.uint64 and step.flags.c_contiguous
        nw, N = occ.shape
        out = np.zeros((nw * n_spw, N), np.uint8)
        mm = np.zeros(nw)
        acc = np.zeros(nw, np.int64)
        fc = np.zeros(nw, np.int64)
        rc = lib().orc_sample(self.ref, nw, _ptr(occ), _ptr(step), ct.c_uint64(seed), n_burn, n_spw,
                              _ptr(out), _ptr(mm), _ptr(acc), float(close_tol), _ptr(fc))
        if rc != 0:
            raise ArithmeticError("walker with zero amplitude")
        if return_first_close:
            return out, mm, acc, fc
        return out, mm, acc

    def measure(self, occ, want_O: bool = True):
        occ = np.ascontiguousarray(occ, np.uint8)
        n_s = occ.shape[0]
        E = np.zeros(n_s)
        O = np.zeros((n_s, self.n_params())) if want_O else None
        if lib().orc_measure(self.ref, n_s, _ptr(occ), _ptr(E), _ptr(O)) != 0:
            raise ArithmeticError("singular pairing submatrix")
        return E, O

    # --- enumeration ---------------------------------------------------------
    def enumerate(self):
        n = int(lib().orc_sector_size(self.ref))
        occ = np.zeros((n, self.wl.N), np.uint8)
        m = int(lib().orc_enumerate(self.ref, _ptr(occ)))
        assert m == n
        w = np.zeros(n)
        lib().orc_exact_weights(self.ref, n, _ptr(occ), _ptr(w))
        return occ, w


# --- free functions ---------------------------------------------------------

def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def pfaffian(A):
    A = np.array(A, np.float64, order="C", copy=True)
    la = ct.c_double()
    sg = ct.c_int()
    lib().orc_pfaffian(A.shape[0], _ptr(A), ct.byref(la), ct.byref(sg))
    return sg.value * np.exp(la.value) if sg.value != 0 else 0.0


def pfaffian_log(A):
    A = np.array(A, np.float64, order="C", copy=True)
    la = ct.c_double()
    sg = ct.c_int()
    lib().orc_pfaffian(A.shape[0], _ptr(A), ct.byref(la), ct.byref(sg))
    return la.value, sg.value


def inverse(A):
    A = np.ascontiguousarray(A, np.float64)
    X = np.zeros_like(A)
    if lib().orc_inverse(A.shape[0], _ptr(A), _ptr(X)) != 0:
        raise ArithmeticError("singular")
    return X


def mean_O(O):
    O = np.ascontiguousarray(O, np.float64)
    out = np.zeros(O.shape[1])
    lib().orc_mean_O(O.shape[0], O.shape[1], _ptr(O), _ptr(out))
    return out


def gradient(O, E):
    O = np.ascontiguousarray(O, np.float64)
    E = np.ascontiguousarray(E, np.float64)
    g = np.zeros(O.shape[1])
    em = ct.c_double()
    lib().orc_gradient(O.shape[0], O.shape[1], _ptr(O), _ptr(E), _ptr(g), ct.byref(em))
    return g, em.value


def dense_S(O):
    O = np.ascontiguousarray(O, np.float64)
    nv = O.shape[1]
    S = np.zeros((nv, nv))
    lib().orc_dense_S(O.shape[0], nv, _ptr(O), _ptr(S))
    return S


def apply_S(O, v, eps, Obar=None):
    O = np.ascontiguousarray(O, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    if Obar is None:
        Obar = mean_O(O)
    out = np.zeros(O.shape[1])
    lib().orc_apply_S(O.shape[0], O.shape[1], _ptr(O), _ptr(np.ascontiguousarray(Obar)), _ptr(v),
                      float(eps), _ptr(out))
    return out


def sr_update(alpha, y, tau, E_mean, Obar):
    """Sec. II.A update after Eq. 2: returns (alpha + x / x_0, x_0) with x = -tau y."""
    alpha = np.ascontiguousarray(alpha, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    Obar = np.ascontiguousarray(Obar, np.float64)
    out = np.zeros_like(alpha)
    x0 = lib().orc_sr_update(alpha.size, _ptr(alpha), _ptr(y), float(tau), float(E_mean), _ptr(Obar), _ptr(out))
    return out, x0


def cg(O, g, eps, tol, max_iter=None):
    O = np.ascontiguousarray(O, np.float64)
    g = np.ascontiguousarray(g, np.float64)
    nv = O.shape[1]
    x = np.zeros(nv)
    it = ct.c_int()
    res = ct.c_double()
    rc = lib().orc_cg(O.shape[0], nv, _ptr(O), _ptr(g), float(eps), float(tol),
                      nv if max_iter is None else int(max_iter), _ptr(x), ct.byref(it), ct.byref(res))
    return x, it.value, res.value, rc == 0
