"""Host-side checks of the C-ABI library that need no GPU: it builds for
sm_103a, loads, exports every function include/vmcsr.h declares, and its
argument validation rejects bad problems before any CUDA call."""
import ctypes as ct

import numpy as np
import pytest

from paper_1108_0900_gb300 import inputs, vmcsr


@pytest.fixture(scope="module")
def L():
    return vmcsr.lib()


def test_exports_every_declared_function(L):
    names = vmcsr.header_functions()
    assert len(names) >= 17
    for n in names:
        assert hasattr(L, n), n


def test_error_strings(L):
    assert L.vmc_error_string(0) == b"ok"
    for code in range(-1, -10, -1):
        assert L.vmc_error_string(code) not in (b"", b"unknown error")


def _create_rc(wl, **opt):
    keep = dict(b=np.ascontiguousarray(wl.bonds, np.int32), t=np.ascontiguousarray(wl.bond_t, np.float64),
                cp=np.ascontiguousarray(wl.corr_ptr, np.int32), cs=np.ascontiguousarray(wl.corr_flat, np.int32))
    lat = vmcsr.vmc_lattice(wl.n_sites, len(keep["b"]), keep["b"].ctypes.data, keep["t"].ctypes.data)
    ham = vmcsr.vmc_hamiltonian(wl.ham, wl.U, 0, None, None)
    cl = opt.pop("corr_class", None)
    ans = vmcsr.vmc_ansatz(wl.n_up, wl.n_dn, wl.n_corr, keep["cp"].ctypes.data, keep["cs"].ctypes.data,
                           None if cl is None else cl.ctypes.data)
    o = dict(n_walkers=4, samples_per_walker=2, walker_precision=0, keep_fp64_store=1, keep_lowp_store=0,
             refresh_every=0)
    o.update(opt)
    opts = vmcsr.vmc_options(**o)
    h = ct.c_void_p()
    return vmcsr.lib().vmc_create(ct.byref(lat), ct.byref(ham), ct.byref(ans), ct.byref(opts), ct.byref(h))


def test_create_rejects_invalid_problems():
    wl = inputs.hubbard("x", 3, 2, 2, 1, "pair", n_walkers=4)           # odd electron count
    assert _create_rc(wl) == -1
    wl = inputs.hubbard("x", 3, 2, 2, 2, "pair", n_walkers=4)
    assert _create_rc(wl, n_walkers=0) == -1
    assert _create_rc(wl, walker_precision=7) == -1
    big = inputs.hubbard("x", 9, 8, 2, 2, "none", n_walkers=1)        # 72 sites > 64
    assert _create_rc(big) == -1
    dup = inputs.hubbard("x", 3, 2, 2, 2, "pair", n_walkers=1)
    dup.corr_sites = [np.array([0, 0], np.int32)]                       # repeated site
    assert _create_rc(dup) == -1
    ten = inputs.hubbard("x", 4, 4, 2, 2, "none", n_walkers=1)
    ten.corr_sites = [np.arange(10, dtype=np.int32)]                    # 4^10 states: beyond 9 sites
    assert _create_rc(ten) == -1
    mixed = inputs.hubbard("x", 3, 2, 2, 2, "pair", n_walkers=1)
    mixed.corr_sites = [np.array([0, 1], np.int32), np.array([0, 1, 2], np.int32)]
    assert _create_rc(mixed, corr_class=np.zeros(2, np.int32)) == -1   # one class, two sizes
    assert _create_rc(mixed, corr_class=np.array([1, 1], np.int32)) == -1   # class 0 unused
    badbond = inputs.hubbard("x", 3, 2, 2, 2, "pair", n_walkers=1)
    badbond.bonds = np.array([[0, 9]], np.int32)
    badbond.bond_t = np.ones(1)
    assert _create_rc(badbond) == -1


def test_null_handles_are_rejected_before_any_device_work(L):
    """Every entry point that takes a handle checks its arguments first:
    a NULL handle is INVALID_ARG, with no CUDA call made (so this runs
    without a GPU)."""
    import ctypes as ct
    vp = ct.c_void_p
    info = ct.create_string_buffer(256)
    calls = {
        "lm_apply": (vp(), vp(), vp(), vp(), 0, vp()),
        "lm_solve": (vp(), ct.c_double(1.0), ct.c_double(1e-2), ct.c_double(1e-6), 10, 8, vp(), info, 0, vp()),
        "lm_update": (vp(), vp(), ct.c_double(1.0), vp()),
        "sr_update": (vp(), vp(), ct.c_double(0.1), 0, vp(), vp()),
        "sr_local_product": (vp(), vp(), vp(), 0, vp()),
    }
    for name, args in calls.items():
        assert getattr(L, name)(*args) == -1, name
