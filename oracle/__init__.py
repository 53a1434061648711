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
            L.orc_apply_S_compact.argtypes = [vp, i64, vp, vp, i32, vp, vp, i32, vp, dbl, vp, vp]
            L.orc_cg.restype = i32
            L.orc_sr_update.argtypes = [i64, vp, vp, dbl, dbl, vp, vp]
            L.orc_sr_update.restype = dbl
            L.orc_sector_size.argtypes = [vp]
            L.orc_sector_size.restype = i64
            L.orc_enumerate.argtypes = [vp, vp]
            L.orc_enumerate.restype = i64
            L.orc_exact_weights.argtypes = [vp, i64, vp, vp]
            L.orc_lm_apply.argtypes = [vp, i64, vp, vp, i32, vp, vp, dbl, vp, vp, vp]
            L.orc_lm_apply.restype = i32
            L.orc_apply_hop.argtypes = [i32, vp, i32, i32, vp]
            L.orc_apply_hop.restype = i32
            L.orc_set_threads.argtypes = [i32]
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

    # --- linear method (Sec. II.B) -----------------------------------------
    def lm_apply(self, occ, factors, x, weights=None, want_S: bool = True):
        """(Hx, Sx) over the basis {Psi, Psi^1 .. Psi^nv} by Eq. 10 with the
        factored Hamiltonian of Eq. 9 (``factors`` = (L, R, c0) from
        ``lm_factors``); weights None = 1/n_s per sample."""
        occ = np.ascontiguousarray(occ, np.uint8)
        Lf, Rf, c0 = factors
        Lf = np.ascontiguousarray(Lf, np.float64)
        Rf = np.ascontiguousarray(Rf, np.float64)
        x = np.ascontiguousarray(x, np.float64)
        nv1 = self.n_params() + 1
        assert x.shape == (nv1,)
        w = None if weights is None else np.ascontiguousarray(weights, np.float64)
        Hx = np.zeros(nv1)
        Sx = np.zeros(nv1) if want_S else None
        rc = lib().orc_lm_apply(self.ref, occ.shape[0], _ptr(occ), _ptr(w), Lf.shape[0], _ptr(Lf),
                                _ptr(Rf), float(c0), _ptr(x), _ptr(Hx), _ptr(Sx))
        if rc != 0:
            raise ArithmeticError("singular pairing submatrix")
        return Hx, Sx

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


def apply_S_compact(P: "Problem", occ, cstate, pairs, pf, v, eps):
    """Eq. 7 from compact rows (see orc_apply_S_compact): occ [n_s, N] uint8,
    cstate [n_s, n_corr] correlator states, pairs [n_pair, 2] positions
    (a, b) of each stored pairing value, pf [n_s, n_pair] the values, v [nv]
    or [k, nv].  Returns (out with the shape of v, Obar)."""
    occ = np.ascontiguousarray(occ, np.uint8)
    cs = np.ascontiguousarray(cstate, np.int64).reshape(occ.shape[0], -1)
    pairs = np.ascontiguousarray(pairs, np.int32)
    pf = np.ascontiguousarray(pf, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    k = 1 if v.ndim == 1 else v.shape[0]
    nv = v.shape[-1]
    out = np.zeros_like(v)
    Obar = np.zeros(nv)
    lib().orc_apply_S_compact(P.ref, occ.shape[0], _ptr(occ), _ptr(cs), len(pairs), _ptr(pairs), _ptr(pf), k,
                              _ptr(v), float(eps), _ptr(out), _ptr(Obar))
    return out, Obar


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


# --- linear method (Sec. II.B) ------------------------------------------------

def lm_factors(wl):
    """The Hamiltonian in the factored form of Eq. 9,
    H = c0 + sum_mu Lhat_mu Rhat_mu,  Lhat_mu = sum_ij L^mu_ij E_ij,
    E_ij = sum_sigma a+_{i sigma} a_{j sigma}  (spatial n x n matrices).

    A one-body operator K = sum k_ij E_ij commutes with the particle number
    Nhat and Nhat = N in the sector, so K = (K Nhat + Nhat K) / (2N): two terms
    (L, R) = (k / 2N, I) and (I, k / 2N).
    Hubbard: k_ij = -t per bond and direction; U n_up n_dn = (U/2)(E_ii E_ii -
    E_ii) per site, so one term (U/2 e_i e_i^T, e_i e_i^T) per site and
    c0 = -U N / 2.
    Ab initio: a+_p a+_r a_s a_q = E_pq E_rs - delta_qr E_ps (spins summed),
    so the two-body part is 1/2 sum_mu (sum_pq L^mu_pq E_pq)^2 - 1/2 sum_ps J_ps
    E_ps with J_ps = sum_q (pq|qs): terms (L^mu / sqrt 2, L^mu / sqrt 2) and
    k = h - J / 2."""
    n, N = wl.n_sites, wl.n_up + wl.n_dn
    Ls, Rs = [], []
    c0 = 0.0
    I = np.eye(n)
    if wl.ham == 0:
        k = np.zeros((n, n))
        for (i, j), t in zip(wl.bonds, wl.bond_t):
            if i == j:
                continue
            k[i, j] -= t
            k[j, i] -= t
        for i in range(n):
            e = np.zeros((n, n))
            e[i, i] = 1.0
            Ls.append(0.5 * wl.U * e)
            Rs.append(e)
        c0 = -0.5 * wl.U * N
    else:
        chol = np.asarray(wl.chol, np.float64)
        J = np.einsum("mpq,mqs->ps", chol, chol)
        k = np.asarray(wl.h, np.float64) - 0.5 * J
        for Lm in chol:
            Ls.append(Lm / np.sqrt(2.0))
            Rs.append(Lm / np.sqrt(2.0))
    Ls += [k / (2.0 * N), I]
    Rs += [I, k / (2.0 * N)]
    return np.array(Ls), np.array(Rs), float(c0)


def lm_davidson(apply, diag_S, shift_H: float, shift_S: float, tol: float = 1e-8,
                max_iter: int = 300, max_sub: int = 24):
    """Lowest eigenpair of (H + a D) x = lam (S + eps D) x (Eq. 8, shifts on
    the parameter block D = diag(0, 1, .., 1)) by the generalized Davidson
    method: Rayleigh-Ritz on a growing orthonormal basis V, residual
    r = (H + a D) u - theta (S + eps D) u of the lowest Ritz pair, new
    direction r / d with d the diagonal of S + eps D (the matrix-free
    stand-in for diag(H - theta S)), Gram-Schmidt against V (twice); on
    reaching max_sub columns the basis restarts from the current and the
    previous Ritz vectors.  ``apply(v)`` returns (H v, S v).  Starts from
    x = e_0 (the current wavefunction).  Returns (theta, x, iterations,
    relative residual |r| / |theta (S + eps D) u|)."""
    import scipy.linalg
    n = diag_S.shape[0]
    Dm = np.ones(n)
    Dm[0] = 0.0
    d = diag_S + shift_S * Dm

    def op(v):
        Hv, Sv = apply(v)
        return Hv + shift_H * Dm * v, Sv + shift_S * Dm * v

    V = np.zeros((n, 0))
    HV = np.zeros((n, 0))
    SV = np.zeros((n, 0))
    t = np.zeros(n)
    t[0] = 1.0
    u_prev = None
    theta, u, rel = np.nan, t, np.inf
    for it in range(1, max_iter + 1):
        for _ in range(2):
            t = t - V @ (V.T @ t)
        t = t / np.linalg.norm(t)
        Ht, St = op(t)
        V = np.column_stack([V, t])
        HV = np.column_stack([HV, Ht])
        SV = np.column_stack([SV, St])
        h = V.T @ HV
        s = V.T @ SV
        h = 0.5 * (h + h.T)
        s = 0.5 * (s + s.T)
        w, c = scipy.linalg.eigh(h, s)
        theta, cv = w[0], c[:, 0]
        u = V @ cv
        Hu, Su = HV @ cv, SV @ cv
        r = Hu - theta * Su
        rel = np.linalg.norm(r) / abs(theta * np.linalg.norm(Su))
        if rel <= tol:
            return theta, u / u[0], it, rel
        t = -r / d
        if V.shape[1] >= max_sub:
            keep = [u] if u_prev is None else [u, u_prev]
            Q, _ = np.linalg.qr(np.column_stack(keep))
            prods = [op(q) for q in Q.T]
            V = Q
            HV = np.column_stack([a for a, _ in prods])
            SV = np.column_stack([b for _, b in prods])
        u_prev = u
    return theta, u / u[0], max_iter, rel


def lm_update(alpha, x, Sx0: float):
    """Parameter update of the linear method (Sec. II.B): the eigenvector
    x = (x_0, x_1 ..) taken relative to the component along Psi of the basis
    orthogonalised to Psi, (S x)_0 = x_0 + sum_j Obar_j x_j; alpha' =
    alpha + x_{1:} / (S x)_0."""
    return np.asarray(alpha) + np.asarray(x[1:]) / Sx0


def set_threads(n: int):
    """OpenMP threads of the oracle's parallel loops."""
    lib().orc_set_threads(int(n))


def apply_hop(M: int, bits, p: int, q: int):
    """a+_p a_q on a determinant given as occupation bits: (sign, bits')."""
    b = np.ascontiguousarray(bits, np.uint8)
    out = np.zeros(M, np.uint8)
    sg = int(lib().orc_apply_hop(M, _ptr(b), p, q, _ptr(out)))
    return sg, out
