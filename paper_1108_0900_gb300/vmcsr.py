"""Thin Python binding of the vmcsr C ABI (include/vmcsr.h).

Argument marshalling only: every step runs in the CUDA library
``_build/libvmcsr.so``.  Device buffers are torch CUDA tensors and streams are
torch streams; there is no CPU fallback — if the library or a CUDA device is
missing the calls raise.

The functions keep the ABI names (``vmc_create``, ``vmc_sample``,
``sr_gradient``, ``sr_apply_S``, ``sr_cg_solve`` ...).  ``Handle`` bundles a
handle with the sizes the calls need, and ``LogPsi`` is the autograd function
whose backward is the library's adjoint kernel (the derivative ratios of
Eq. 3, recomputed from scratch).
"""
from __future__ import annotations

import ctypes as ct
import os
import re
from typing import Optional

import numpy as np

from . import build as _build

VMC_OK = 0
VMC_HUBBARD, VMC_ABINITIO = 0, 1
VMC_FP64, VMC_FP32 = 0, 1
VMC_STORE_FP64, VMC_STORE_FP32, VMC_STORE_BF16, VMC_STORE_FP32_F32ACC = 0, 1, 2, 3
VMC_CG_FP64, VMC_CG_MIXED, VMC_CG_FP32, VMC_CG_BLOCK4, VMC_CG_MIXED64 = 0, 1, 2, 3, 4
ERRORS = {
    -1: "INVALID_ARG", -2: "OOM", -3: "SINGULAR", -4: "NONFINITE", -5: "NOT_CONVERGED",
    -6: "TIMEOUT", -7: "CUDA", -8: "UNSUPPORTED", -9: "STATE",
}


class VmcError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} {detail}".strip())


class vmc_lattice(ct.Structure):
    _fields_ = [("n_sites", ct.c_int), ("n_bonds", ct.c_int), ("bonds", ct.c_void_p), ("bond_t", ct.c_void_p)]


class vmc_hamiltonian(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("U", ct.c_double), ("n_chol", ct.c_int), ("h", ct.c_void_p),
                ("chol", ct.c_void_p)]


class vmc_ansatz(ct.Structure):
    _fields_ = [("n_up", ct.c_int), ("n_dn", ct.c_int), ("n_corr", ct.c_int), ("corr_ptr", ct.c_void_p),
                ("corr_sites", ct.c_void_p), ("corr_class", ct.c_void_p)]


class vmc_options(ct.Structure):
    _fields_ = [("n_walkers", ct.c_int), ("samples_per_walker", ct.c_int), ("walker_precision", ct.c_int),
                ("keep_fp64_store", ct.c_int), ("keep_lowp_store", ct.c_int), ("refresh_every", ct.c_int),
                ("fp64_refresh", ct.c_int)]


class vmc_sample_stats_t(ct.Structure):
    _fields_ = [("lnpsi_drift_max", ct.c_double), ("lnpsi_drift_mean", ct.c_double), ("refreshed", ct.c_int),
                ("el_refresh_change_max", ct.c_double), ("el_refresh_change_mean", ct.c_double)]


class vmc_lm_info(ct.Structure):
    _fields_ = [("iterations", ct.c_int), ("restarts", ct.c_int), ("converged", ct.c_int),
                ("eigenvalue", ct.c_double), ("rel_residual", ct.c_double), ("Sx0", ct.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class vmc_cg_info(ct.Structure):
    _fields_ = [("iterations", ct.c_int), ("refinements", ct.c_int), ("residual_products", ct.c_int),
                ("converged", ct.c_int), ("true_rel_residual", ct.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def header_functions():
    """Names of the functions declared in include/vmcsr.h."""
    txt = open(os.path.join(_build.INCLUDE, "vmcsr.h")).read()
    return re.findall(r"^\s*(?:int|const char\*)\s+(\w+)\s*\(", txt, flags=re.M)


def lib(build_if_missing: bool = True):
    """Load libvmcsr.so (building it in-tree with nvcc when absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"{path} not built")
        path = _build.build()
    L = ct.CDLL(path)
    vp, i32, i64, dbl, u64 = ct.c_void_p, ct.c_int, ct.c_int64, ct.c_double, ct.c_uint64
    sig = {
        "vmc_create": [vp, vp, vp, vp, vp],
        "vmc_destroy": [vp],
        "vmc_num_params": [vp, vp, vp],
        "vmc_set_params": [vp, vp, vp],
        "vmc_get_params": [vp, vp, vp, vp],
        "sr_update": [vp, vp, dbl, i32, vp, vp],
        "sr_local_moments": [vp, vp, vp, vp, i32, vp],
        "sr_local_product": [vp, vp, vp, i32, vp],
        "lm_apply": [vp, vp, vp, vp, i32, vp],
        "lm_solve": [vp, dbl, dbl, dbl, i32, i32, vp, vp, i32, vp],
        "lm_update": [vp, vp, dbl, vp],
        "vmc_set_walkers": [vp, vp, vp],
        "vmc_get_walkers": [vp, vp, vp, vp],
        "vmc_sample": [vp, i32, u64, vp],
        "vmc_measure": [vp, vp, i64, vp],
        "vmc_num_samples": [vp, vp],
        "vmc_get_samples": [vp, vp, vp, vp, vp, i32, vp],
        "vmc_logpsi": [vp, vp, vp],
        "vmc_logpsi_backward": [vp, vp, vp, vp],
        "sr_gradient": [vp, vp, vp, i32, vp],
        "sr_apply_S": [vp, vp, vp, i32, dbl, i32, vp],
        "sr_cg_solve": [vp, vp, dbl, dbl, i32, i32, vp, vp, vp],
        "vmc_profile": [vp, i32],
        "sr_pairing_product_noalloc": [i64, i32, i32, i32, vp, i64, vp, i64, vp, vp, vp, vp],
        "vmc_profile_read": [vp, i32, vp, vp, vp, vp],
        "vmc_set_wait_limit": [vp, ct.c_uint32],
        "vmc_set_product_path": [vp, i32],
        "sr_autotune": [vp, i32, vp, vp],
        "vmc_set_auto_paths": [vp, i32, i32],
        "vmc_sample_stats": [vp, vp, vp],
        "vmc_sample_batch": [vp, i32, i32, vp, vp],
        "sr_apply_S_batch": [vp, i32, vp, vp, dbl, i32, vp],
        "sr_set_inner_tol": [vp, dbl],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = i32
    L.vmc_error_string.argtypes = [i32]
    L.vmc_error_string.restype = ct.c_char_p
    L.vmc_last_error_detail.argtypes = []
    L.vmc_last_error_detail.restype = ct.c_char_p
    _lib = L
    return L


def _check(rc: int, where: str):
    if rc != VMC_OK:
        detail = lib().vmc_last_error_detail().decode(errors="replace")
        raise VmcError(rc, where, detail)


def _np_ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def _dev_ptr(t):
    if t is None:
        return None
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()
    return ct.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ct.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
# ABI-named wrappers
# ---------------------------------------------------------------------------

def vmc_create(wl, n_walkers=None, samples_per_walker=None, walker_precision=VMC_FP64,
               keep_fp64_store=True, keep_lowp_store=False, refresh_every=0, fp64_refresh=False):
    """Create a handle for a problem description (``inputs.Workload``)."""
    keep = dict(
        bonds=np.ascontiguousarray(wl.bonds, np.int32),
        bond_t=np.ascontiguousarray(wl.bond_t, np.float64),
        corr_ptr=np.ascontiguousarray(wl.corr_ptr, np.int32),
        corr_sites=np.ascontiguousarray(wl.corr_flat, np.int32),
        corr_class=None if getattr(wl, "corr_class", None) is None else np.ascontiguousarray(wl.corr_class, np.int32),
        h=None if wl.h is None else np.ascontiguousarray(wl.h, np.float64),
        chol=None if wl.chol is None else np.ascontiguousarray(wl.chol, np.float64),
    )
    lat = vmc_lattice(wl.n_sites, len(keep["bonds"]), _np_ptr(keep["bonds"]), _np_ptr(keep["bond_t"]))
    ham = vmc_hamiltonian(wl.ham, float(wl.U), 0 if wl.chol is None else wl.chol.shape[0],
                          _np_ptr(keep["h"]), _np_ptr(keep["chol"]))
    ans = vmc_ansatz(wl.n_up, wl.n_dn, wl.n_corr, _np_ptr(keep["corr_ptr"]), _np_ptr(keep["corr_sites"]),
                     _np_ptr(keep["corr_class"]))
    opt = vmc_options(int(n_walkers or wl.n_walkers), int(samples_per_walker or wl.samples_per_walker),
                      int(walker_precision), int(bool(keep_fp64_store)), int(bool(keep_lowp_store)),
                      int(refresh_every), int(bool(fp64_refresh)))
    h = ct.c_void_p()
    _check(lib().vmc_create(ct.byref(lat), ct.byref(ham), ct.byref(ans), ct.byref(opt), ct.byref(h)), "vmc_create")
    return Handle(h, wl, opt)


class Handle:
    def __init__(self, h, wl, opt):
        self.h = h
        self.wl = wl
        self.n_walkers = opt.n_walkers
        self.spw = opt.samples_per_walker
        nv, ncp = ct.c_int64(), ct.c_int64()
        _check(lib().vmc_num_params(h, ct.byref(nv), ct.byref(ncp)), "vmc_num_params")
        self.n_params, self.n_corr_params = nv.value, ncp.value
        self.N = wl.N
        self.P = wl.n_up * (wl.n_up - 1) // 2 + wl.n_dn * (wl.n_dn - 1) // 2 + wl.n_up * wl.n_dn

    def close(self):
        if self.h:
            lib().vmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def vmc_set_params(h: Handle, C, f):
    C = np.ascontiguousarray(C, np.float64)
    f = np.ascontiguousarray(f, np.float64)
    _check(lib().vmc_set_params(h.h, _np_ptr(C), _np_ptr(f)), "vmc_set_params")


def vmc_get_params(h: Handle, stream=None):
    """Current parameters (C, f) as host FP64 arrays."""
    C = np.zeros(h.n_corr_params)
    f = np.zeros(h.n_params - h.n_corr_params)
    _check(lib().vmc_get_params(h.h, _np_ptr(C), _np_ptr(f), _stream(stream)), "vmc_get_params")
    return C, f


def vmc_set_walkers(h: Handle, occ, step=None):
    occ = np.ascontiguousarray(occ, np.uint8)
    st = None if step is None else np.ascontiguousarray(step, np.uint64)
    _check(lib().vmc_set_walkers(h.h, _np_ptr(occ), _np_ptr(st)), "vmc_set_walkers")


def vmc_get_walkers(h: Handle, stream=None):
    occ = np.zeros((h.n_walkers, h.N), np.uint8)
    step = np.zeros(h.n_walkers, np.uint64)
    _check(lib().vmc_get_walkers(h.h, _np_ptr(occ), _np_ptr(step), _stream(stream)), "vmc_get_walkers")
    return occ, step


def save_state(h: Handle, path: str, stream=None, **extra):
    """Checkpoint of an optimisation: the parameters (C, f), every walker's
    configuration and step counter (the counter of its Philox stream), and
    any extra values (e.g. the iteration and the next sampling seed).  With
    the same seed, vmc_sample after load_state reproduces the next batch bit
    for bit.  `path` is an .npz file.  The state is read once the work queued
    on `stream` (the stream the sampling ran on; None = torch's current
    stream) is done."""
    C, f = vmc_get_params(h, stream)
    occ, step = vmc_get_walkers(h, stream)
    np.savez(path, C=C, f=f, occ=occ, step=step, **{k: np.asarray(v) for k, v in extra.items()})


def load_state(h: Handle, path: str) -> dict:
    """Restore a checkpoint written by save_state; returns its extra values.
    The parameter and walker uploads wait for all work queued on the device
    (any stream) before they overwrite anything."""
    d = np.load(path)
    vmc_set_params(h, d["C"], d["f"])
    vmc_set_walkers(h, d["occ"], d["step"])
    return {k: d[k] for k in d.files if k not in ("C", "f", "occ", "step")}


def vmc_sample(h: Handle, n_burn: int, seed: int, stream=None):
    _check(lib().vmc_sample(h.h, int(n_burn), ct.c_uint64(seed), _stream(stream)), "vmc_sample")


def vmc_sample_stats(h: Handle, stream=None) -> dict:
    """Drift of the chains' running ln|Psi| against FP64 from-scratch values
    and, with fp64_refresh, the change of E_L made by the refresh."""
    r = vmc_sample_stats_t()
    _check(lib().vmc_sample_stats(h.h, ct.byref(r), _stream(stream)), "vmc_sample_stats")
    return {k: getattr(r, k) for k, _ in r._fields_}


def vmc_sample_batch(handles, n_burn: int, seeds, stream=None):
    """vmc_sample of every handle (lattices of uneven size) in one launch."""
    n = len(handles)
    hs = (ct.c_void_p * n)(*[h.h for h in handles])
    sd = (ct.c_uint64 * n)(*[int(x) for x in seeds])
    _check(lib().vmc_sample_batch(hs, n, int(n_burn), sd, _stream(stream)), "vmc_sample_batch")


def sr_apply_S_batch(handles, Vs, shift: float, store=VMC_STORE_FP64, stream=None):
    """(S_b + shift I) V_b for every handle b, all stores streamed by one
    launch; Vs: CUDA float64 vectors; returns the products."""
    import torch
    n = len(handles)
    Vs = [v.contiguous() for v in Vs]
    outs = [torch.empty_like(v) for v in Vs]
    hs = (ct.c_void_p * n)(*[h.h for h in handles])
    vp = (ct.c_void_p * n)(*[v.data_ptr() for v in Vs])
    op = (ct.c_void_p * n)(*[o.data_ptr() for o in outs])
    _check(lib().sr_apply_S_batch(hs, n, vp, op, float(shift), int(store), _stream(stream)), "sr_apply_S_batch")
    return outs


def vmc_measure(h: Handle, occ, stream=None):
    occ = np.ascontiguousarray(occ, np.uint8)
    _check(lib().vmc_measure(h.h, _np_ptr(occ), occ.shape[0], _stream(stream)), "vmc_measure")


def vmc_num_samples(h: Handle) -> int:
    n = ct.c_int64()
    _check(lib().vmc_num_samples(h.h, ct.byref(n)), "vmc_num_samples")
    return n.value


def vmc_get_samples(h: Handle, store=VMC_STORE_FP64, stream=None):
    n = vmc_num_samples(h)
    occ = np.zeros((n, h.N), np.uint8)
    E = np.zeros(n)
    cs = np.zeros((n, max(h.wl.n_corr, 1)), np.uint32)
    pf = np.zeros((n, h.P))
    _check(lib().vmc_get_samples(h.h, _np_ptr(occ), _np_ptr(E), _np_ptr(cs), _np_ptr(pf), int(store),
                                 _stream(stream)), "vmc_get_samples")
    return occ, E, cs[:, :h.wl.n_corr], pf


def vmc_logpsi(h: Handle, stream=None):
    import torch
    out = torch.empty(vmc_num_samples(h), dtype=torch.float64, device="cuda")
    _check(lib().vmc_logpsi(h.h, _dev_ptr(out), _stream(stream)), "vmc_logpsi")
    return out


def vmc_logpsi_backward(h: Handle, w=None, stream=None):
    import torch
    if w is None:
        _check(lib().vmc_logpsi_backward(h.h, None, None, _stream(stream)), "vmc_logpsi_backward")
        return None
    w = w.to(dtype=torch.float64, device="cuda").contiguous()
    grad = torch.empty(h.n_params, dtype=torch.float64, device="cuda")
    _check(lib().vmc_logpsi_backward(h.h, _dev_ptr(w), _dev_ptr(grad), _stream(stream)), "vmc_logpsi_backward")
    return grad


def sr_gradient(h: Handle, store=VMC_STORE_FP64, stream=None, stats=True):
    import torch
    g = torch.empty(h.n_params, dtype=torch.float64, device="cuda")
    es = np.zeros(3) if stats else None
    _check(lib().sr_gradient(h.h, _dev_ptr(g), _np_ptr(es), int(store), _stream(stream)), "sr_gradient")
    return g, es


def sr_apply_S(h: Handle, V, shift: float, store=VMC_STORE_FP64, stream=None, out=None):
    """V: CUDA float64 tensor [n_params] or [k, n_params]."""
    import torch
    k = 1 if V.dim() == 1 else V.shape[0]
    V = V.contiguous()
    if out is None:
        out = torch.empty_like(V)
    _check(lib().sr_apply_S(h.h, _dev_ptr(V), _dev_ptr(out), int(k), float(shift), int(store), _stream(stream)),
           "sr_apply_S")
    return out


def sr_cg_solve(h: Handle, g, shift: float, tol: float, max_iter: int, mode=VMC_CG_FP64, stream=None, x=None,
                allow_not_converged=False):
    import torch
    if x is None:
        x = torch.empty_like(g)
    info = vmc_cg_info()
    rc = lib().sr_cg_solve(h.h, _dev_ptr(g), float(shift), float(tol), int(max_iter), int(mode), _dev_ptr(x),
                           ct.byref(info), _stream(stream))
    if not (allow_not_converged and rc == -5):
        _check(rc, "sr_cg_solve")
    return x, info.as_dict()


def sr_update(h: Handle, y, tau: float, store=VMC_STORE_FP64, stream=None):
    """alpha += x / x_0 with x = -tau y (Sec. II.A); returns x_0."""
    x0 = ct.c_double()
    _check(lib().sr_update(h.h, _dev_ptr(y), float(tau), int(store), ct.byref(x0), _stream(stream)), "sr_update")
    return x0.value


def sr_local_moments(h: Handle, store=VMC_STORE_FP64, stream=None):
    """Rank-local (sum O, sum E_L O, sum E_L, n_s) for a sample-sharded solve."""
    import torch
    sO = torch.empty(h.n_params, dtype=torch.float64, device="cuda")
    sEO = torch.empty_like(sO)
    sc = np.zeros(2)
    _check(lib().sr_local_moments(h.h, _dev_ptr(sO), _dev_ptr(sEO), _np_ptr(sc), int(store), _stream(stream)),
           "sr_local_moments")
    return sO, sEO, float(sc[0]), int(sc[1])


def sr_local_product(h: Handle, v, store=VMC_STORE_FP64, stream=None, out=None):
    """Rank-local sum_s (O_s . v) O_s for a sample-sharded solve."""
    import torch
    if out is None:
        out = torch.empty_like(v)
    _check(lib().sr_local_product(h.h, _dev_ptr(v), _dev_ptr(out), int(store), _stream(stream)), "sr_local_product")
    return out


def lm_apply(h: Handle, x, store=VMC_STORE_FP64, want_S: bool = True, stream=None, Hx=None, Sx=None):
    """Linear-method products (Hx, Sx) over the basis {Psi, Psi^1 .. Psi^nv}
    by Eq. 10 (x: device FP64 [n_v + 1]); Sx is None unless want_S."""
    import torch
    if Hx is None:
        Hx = torch.empty_like(x)
    if want_S and Sx is None:
        Sx = torch.empty_like(x)
    _check(lib().lm_apply(h.h, _dev_ptr(x), _dev_ptr(Hx), _dev_ptr(Sx) if want_S else None, int(store),
                          _stream(stream)), "lm_apply")
    return Hx, (Sx if want_S else None)


def lm_solve(h: Handle, shift_H: float, shift_S: float, tol: float, max_iter: int = 500, max_sub: int = 24,
             store=VMC_STORE_FP64, stream=None, allow_not_converged=False):
    """Lowest eigenpair of the shifted Eq. 8 by generalized Davidson; returns
    (x with x_0 = 1, info dict with eigenvalue, residual and Sx0)."""
    import torch
    x = torch.empty(h.n_params + 1, dtype=torch.float64, device="cuda")
    info = vmc_lm_info()
    rc = lib().lm_solve(h.h, float(shift_H), float(shift_S), float(tol), int(max_iter), int(max_sub), _dev_ptr(x),
                        ct.byref(info), int(store), _stream(stream))
    if not (allow_not_converged and rc == -5):
        _check(rc, "lm_solve")
    return x, info.as_dict()


def lm_update(h: Handle, x, Sx0: float, stream=None):
    """alpha += x_{1:} / Sx0 (the linear method's step, Sec. II.B)."""
    _check(lib().lm_update(h.h, _dev_ptr(x), float(Sx0), _stream(stream)), "lm_update")


def lm_optimize(h: Handle, n_iter: int, shift_H: float, shift_S: float, tol: float, store=VMC_STORE_FP64,
                seed: int = 1, max_iter: int = 500, max_sub: int = 24, grow: float = 10.0):
    """The linear-method loop of Sec. II.B with its safeguard: sample, lowest
    eigenpair of the shifted Eq. 8, update, then sample again at the new
    parameters; a step whose energy is higher than before by more than three
    standard errors of the earlier estimate is undone and retried with shift_H * grow
    (the larger diagonal shift rotates the step towards the gradient and
    shortens it).  Returns one record per iteration."""
    vmc_sample(h, 0, seed)
    _, es = sr_gradient(h, store)
    hist = []
    for it in range(n_iter):
        C0, f0 = vmc_get_params(h)
        x, info = lm_solve(h, shift_H, shift_S, tol, max_iter, max_sub, store, allow_not_converged=True)
        lm_update(h, x, info["Sx0"])
        vmc_sample(h, 0, seed + 1 + it)
        _, es_new = sr_gradient(h, store)
        # judged against the error of the energy before the step: a bad step
        # often also inflates the error of the new estimate
        ok = bool(es_new[0] <= es[0] + 3.0 * es[2])
        hist.append({"energy": es, "energy_after": es_new, "lm": info, "shift_H": shift_H, "accepted": ok})
        if ok:
            es = es_new
        else:
            vmc_set_params(h, C0, f0)
            shift_H *= grow
            vmc_sample(h, 0, seed + 100000 + it)
            _, es = sr_gradient(h, store)
    return hist


def sr_optimize(h: Handle, n_iter: int, tau: float, shift: float, tol: float, mode=VMC_CG_FP64, seed: int = 1,
                max_iter: int = 20000, callback=None):
    """The SR loop of Sec. II.A: sample, gradient, CG solve of Eq. 2, update;
    returns one record per iteration (energy statistics before the update,
    CG info, x_0).  The walkers must be set and thermalised."""
    store = VMC_STORE_FP64 if mode in (VMC_CG_FP64, VMC_CG_MIXED64) else VMC_STORE_FP32
    hist = []
    for it in range(n_iter):
        vmc_sample(h, 0, seed + it)
        g, es = sr_gradient(h, store)
        y, info = sr_cg_solve(h, g, shift, tol, max_iter, mode, allow_not_converged=True)
        x0 = sr_update(h, y, tau, store)
        rec = {"iteration": it, "E_mean": float(es[0]), "E_var": float(es[1]), "E_err": float(es[2]),
               "x0": x0, "cg": info}
        hist.append(rec)
        if callback is not None:
            callback(rec)
    return hist


# ---------------------------------------------------------------------------
# autograd: ln|Psi(n_s)| of the stored samples as a function of (C, f)
# ---------------------------------------------------------------------------

def _make_logpsi():
    import torch

    class LogPsi(torch.autograd.Function):
        """ln|Psi_n| = sum_c ln|C_c[idx_c(n)]| + ln|Pf(F[occ, occ])| (Eq. 11)
        for every stored sample; backward maps grad_output w_s to
        sum_s w_s O_s with the library's adjoint kernel (pairing inverse
        recomputed from scratch, FP64)."""

        @staticmethod
        def forward(ctx, handle, C, f):
            vmc_set_params(handle, C.detach().cpu().numpy(), f.detach().cpu().numpy())
            ctx.handle = handle
            ctx.ncp = C.numel()
            ctx.devs = (C.device, C.dtype, f.device, f.dtype)
            return vmc_logpsi(handle)

        @staticmethod
        def backward(ctx, grad_out):
            g = vmc_logpsi_backward(ctx.handle, grad_out)
            dC, tC, df, tf = ctx.devs
            return None, g[:ctx.ncp].to(dC, tC), g[ctx.ncp:].to(df, tf)

    return LogPsi


_LogPsi = None


def LogPsi():
    global _LogPsi
    if _LogPsi is None:
        _LogPsi = _make_logpsi()
    return _LogPsi


VMC_PATH_AUTO, VMC_PATH_SORTED, VMC_PATH_FUSED, VMC_PATH_STAGED, VMC_PATH_GENERIC, VMC_PATH_COMPACT = 0, 1, 2, 3, 4, 5
PATH_NAMES = {0: "auto", 1: "sorted", 2: "fused", 3: "staged", 4: "generic", 5: "compact"}


class vmc_tune_info(ct.Structure):
    _fields_ = [("path", ct.c_int), ("path4", ct.c_int), ("ms", ct.c_double * 6), ("ms4", ct.c_double * 6)]


def vmc_set_product_path(h: Handle, path: int):
    """Product path of the BF16 S products (VMC_PATH_*; AUTO = the autotuner's
    choice, by default the sorted two-pass product)."""
    _check(lib().vmc_set_product_path(h.h, int(path)), "vmc_set_product_path")


def sr_autotune(h: Handle, reps: int = 5, stream=None) -> dict:
    """Time every applicable product path on the handle's samples and make the
    fastest the AUTO choice; returns {"path", "path4", "ms": {name: ms}, "ms4": ...}."""
    info = vmc_tune_info()
    _check(lib().sr_autotune(h.h, int(reps), ct.byref(info), _stream(stream)), "sr_autotune")
    ms = {PATH_NAMES[p]: info.ms[p] for p in range(1, 6) if info.ms[p] > 0}
    ms4 = {PATH_NAMES[p]: info.ms4[p] for p in range(1, 6) if info.ms4[p] > 0}
    return {"path": PATH_NAMES[info.path], "path4": PATH_NAMES[info.path4], "ms": ms, "ms4": ms4}


def tuned(h: Handle, cache_path: str, key: str, reps: int = 5, stream=None) -> dict:
    """The autotuner's choice for workload `key`, cached as JSON in
    `cache_path`: a cached choice is applied to the handle without timing;
    otherwise sr_autotune runs and its result is stored."""
    import json
    cache = {}
    if os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
    names = {v: k for k, v in PATH_NAMES.items()}
    if key in cache:
        ent = cache[key]
        _set_auto(h, names[ent["path"]], names[ent["path4"]])
        return dict(ent, cached=True)
    ent = sr_autotune(h, reps, stream)
    cache[key] = ent
    with open(cache_path, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    return dict(ent, cached=False)


def _set_auto(h: Handle, path: int, path4: int):
    """Apply a cached autotuner choice: one-vector products on `path`,
    two- and four-vector products on `path4`."""
    _check(lib().vmc_set_auto_paths(h.h, int(path), int(path4)), "vmc_set_auto_paths")


def sr_set_inner_tol(h: Handle, floor: float):
    """Floor of the inner relative tolerance of the mixed solves (0: default)."""
    _check(lib().sr_set_inner_tol(h.h, float(floor)), "sr_set_inner_tol")


def vmc_set_wait_limit(h: Handle, tries: int):
    """Tries of every bounded wait on a staged tile in the streaming products
    (default 4,194,304; 0 makes every wait give up: VMC_ERR_TIMEOUT)."""
    _check(lib().vmc_set_wait_limit(h.h, int(tries)), "vmc_set_wait_limit")


def vmc_profile(h: Handle, enable: bool):
    _check(lib().vmc_profile(h.h, int(bool(enable))), "vmc_profile")


def vmc_profile_read(h: Handle, store=VMC_STORE_BF16):
    la, pl = ct.c_int64(), ct.c_int64()
    ms, by = ct.c_double(), ct.c_double()
    _check(lib().vmc_profile_read(h.h, int(store), ct.byref(la), ct.byref(pl), ct.byref(ms), ct.byref(by)),
           "vmc_profile_read")
    return dict(launches_all=la.value, pass_launches=pl.value, pass_ms=ms.value, pass_bytes=by.value)


def sr_pairing_product_noalloc(n_sites: int, n_up: int, n_dn: int, occ, pf, v, t=None, out=None, stream=None):
    """Allocation-free pairing-block product (see include/vmcsr.h).  occ: CUDA
    uint8 [n_s, >=N]; pf: CUDA float32 [n_s, >=P]; v: CUDA float32 [M(M-1)/2].
    Returns (t [n_s] float32, out [M(M-1)/2] float64); pass t / out to reuse
    caller-owned buffers."""
    import torch
    n_s = occ.shape[0]
    M = 2 * n_sites
    if t is None:
        t = torch.empty(n_s, dtype=torch.float32, device=v.device)
    if out is None:
        out = torch.empty(M * (M - 1) // 2, dtype=torch.float64, device=v.device)
    _check(lib().sr_pairing_product_noalloc(n_s, n_sites, n_up, n_dn, _dev_ptr(occ), occ.stride(0), _dev_ptr(pf),
                                            pf.stride(0), _dev_ptr(v), _dev_ptr(t), _dev_ptr(out), _stream(stream)),
           "sr_pairing_product_noalloc")
    return t, out
