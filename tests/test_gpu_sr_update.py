"""SR parameter update and optimisation loop (Sec. II.A) on the CUDA path.

sr_update applies alpha_k += x_k / x_0 with x = -tau y and x_0 = 1 - tau <E_L>
- Obar . x on the device; the oracle applies the same update, itself pinned
on the CPU against a dense solve of the whole Eq. 2 system and against the
exact first-order energy change.  Tolerances: FP64 parameters and x_0 1e-12
relative, with the mean of whichever store the gradient was taken over (the
FP32 and BF16 cases rebuild that mean from the store's own values).
"""
import contextlib
import copy

import numpy as np
import pytest

import oracle
from paper_1108_0900_gb300 import inputs
from paper_1108_0900_gb300 import vmcsr as V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


CASES = {
    "hubbard4x4_pair": lambda: inputs.workload("hubbard4x4_pair", n_walkers=24, samples_per_walker=6),
    "tiny2x2": lambda: inputs.hubbard("t", 2, 2, 2, 2, "2x2", seed=5, n_walkers=16, samples_per_walker=4),
    "abinitio24": lambda: inputs.workload("abinitio24", n_walkers=8, samples_per_walker=2),
}


def _measured(wl, prec=V.VMC_FP64):
    P = oracle.Problem(wl)
    occ = wl.init_occ.copy()
    step = np.zeros(wl.n_walkers, np.uint64)
    smp, _, _ = P.sample(occ, step, 77, 3, wl.samples_per_walker)
    E, O = P.measure(smp)
    h = V.vmc_create(wl, walker_precision=prec, keep_fp64_store=True, keep_lowp_store=True)
    V.vmc_set_params(h, wl.C, wl.f)
    V.vmc_measure(h, smp)
    return P, smp, E, O, h


def _with_params(wl, C, f):
    wl2 = copy.copy(wl)
    wl2.C, wl2.f = np.array(C, np.float64), np.array(f, np.float64)
    return wl2


@pytest.mark.parametrize("name", list(CASES))
def test_sr_update_matches_oracle(name):
    wl = CASES[name]()
    P, smp, E, O, h = _measured(wl)
    V.sr_gradient(h, V.VMC_STORE_FP64)
    y = np.random.default_rng(3).standard_normal(wl.n_params)
    tau = 0.02
    x0 = V.sr_update(h, torch.from_numpy(y).cuda(), tau, V.VMC_STORE_FP64)
    C, f = V.vmc_get_params(h)
    alpha = np.concatenate([wl.C, wl.f])
    ref, x0_ref = oracle.sr_update(alpha, y, tau, E.mean(), O.mean(0))
    assert x0 == pytest.approx(x0_ref, rel=1e-12)
    assert rel(np.concatenate([C, f]), ref) <= 1e-13
    # every derived copy moved with the parameters: the library measures the
    # same samples as the oracle holding the new parameters
    wl2 = _with_params(wl, ref[:wl.n_corr_params], ref[wl.n_corr_params:])
    E2, O2 = oracle.Problem(wl2).measure(smp)
    V.vmc_measure(h, smp)
    _, E_g, _, _ = V.vmc_get_samples(h, V.VMC_STORE_FP64)
    assert np.all(np.abs(E_g - E2) <= 1e-10 * np.maximum(1.0, np.abs(E2)))
    h.close()


def _dense_mean(wl, occ, cs, pf):
    """Mean of O over the stored samples, from the store's own values."""
    M, ncp = wl.M, wl.n_corr_params
    Ob = np.zeros(wl.n_params)
    off = np.concatenate([[0], np.cumsum([4 ** len(c) for c in wl.corr_sites])])
    nu, N = wl.n_up, wl.N
    pl = [(a, b) for a in range(nu) for b in range(a + 1, nu)]
    pl += [(a, b) for a in range(nu, N) for b in range(a + 1, N)]
    pl += [(a, b) for a in range(nu) for b in range(nu, N)]
    for s in range(len(occ)):
        for c in range(len(wl.corr_sites)):
            k = off[c] + int(cs[s, c])
            Ob[k] += 1.0 / wl.C[k]
        for e, (a, b) in enumerate(pl):
            p, q = int(occ[s, a]), int(occ[s, b])
            Ob[ncp + p * M - p * (p + 1) // 2 + (q - p - 1)] += pf[s, e]
    return Ob / len(occ)


def test_sr_update_fp32_walkers_and_lowp_means():
    """x_0 uses the mean of the store the gradient was taken over."""
    wl = CASES["hubbard4x4_pair"]()
    P, smp, E, O, h = _measured(wl, prec=V.VMC_FP32)
    y = np.random.default_rng(4).standard_normal(wl.n_params)
    alpha = np.concatenate([wl.C, wl.f])
    for store in (V.VMC_STORE_FP32, V.VMC_STORE_BF16):
        V.vmc_set_params(h, wl.C, wl.f)
        V.vmc_measure(h, smp)
        V.sr_gradient(h, store)
        occ, Es, cs, pf = V.vmc_get_samples(h, store)
        Ob = _dense_mean(wl, occ, cs, pf)
        x0 = V.sr_update(h, torch.from_numpy(y).cuda(), 0.01, store)
        ref, x0_ref = oracle.sr_update(alpha, y, 0.01, Es.mean(), Ob)
        assert x0 == pytest.approx(x0_ref, rel=1e-12)
        C, f = V.vmc_get_params(h)
        assert rel(np.concatenate([C, f]), ref) <= 1e-13
        # FP32 walkers use the updated FP32 copies
        wl2 = _with_params(wl, C, f)
        E2, _ = oracle.Problem(wl2).measure(smp)
        V.vmc_measure(h, smp)
        _, Eg, _, _ = V.vmc_get_samples(h, V.VMC_STORE_FP32)
        assert np.all(np.abs(Eg - E2) <= 5e-3 * np.maximum(1.0, np.abs(E2)))
    h.close()


def test_sr_update_errors_leave_parameters():
    wl = CASES["tiny2x2"]()
    P, smp, E, O, h = _measured(wl)
    y = torch.zeros(wl.n_params, dtype=torch.float64, device="cuda")
    with pytest.raises(V.VmcError) as e:          # no gradient over this store yet
        V.sr_update(h, y, 0.01, V.VMC_STORE_FP64)
    assert e.value.code == -9
    V.sr_gradient(h, V.VMC_STORE_FP64)
    C0, f0 = V.vmc_get_params(h)
    Ob = torch.from_numpy(O.mean(0)).cuda()
    with pytest.raises(V.VmcError) as e:          # x_0 < 0: tau beyond the first-order projector
        V.sr_update(h, -1e6 * Ob / float(Ob @ Ob), 1.0, V.VMC_STORE_FP64)
    assert e.value.code == -4
    C1, f1 = V.vmc_get_params(h)
    assert np.array_equal(C0, C1) and np.array_equal(f0, f1)
    h.close()


def _exact_energy(wl, C, f):
    P = oracle.Problem(_with_params(wl, C, f))
    occ, w = P.enumerate()
    return float(w @ P.measure(occ, want_O=False)[0])


def test_sr_optimize_lowers_the_exact_energy():
    """2x2 lattice at half filling (36 configurations): the exact energy of
    the parameters after a few SR iterations is below the initial one."""
    wl = inputs.hubbard("opt", 2, 2, 2, 2, "2x2", seed=61, n_walkers=64, samples_per_walker=32)
    h = V.vmc_create(wl, walker_precision=V.VMC_FP64, keep_fp64_store=True, keep_lowp_store=True)
    V.vmc_set_params(h, wl.C, wl.f)
    V.vmc_set_walkers(h, wl.init_occ)
    V.vmc_sample(h, 20, 5)
    E0 = _exact_energy(wl, wl.C, wl.f)
    hist = V.sr_optimize(h, 6, tau=0.05, shift=1e-3, tol=1e-8, mode=V.VMC_CG_FP64, seed=100)
    C, f = V.vmc_get_params(h)
    E1 = _exact_energy(wl, C, f)
    assert E1 < E0 - 1e-3, (E0, E1, [r["E_mean"] for r in hist])
    assert all(r["x0"] > 0 for r in hist)
    h.close()


def test_free_fermion_state_is_a_fixed_point():
    """U = 0 with the Slater-determinant pairing of the hopping eigenorbitals
    and all C = 1: every sample has the same E_L, so g = 0, y = 0 and the
    update leaves the parameters where they are (x_0 = 1 - tau E)."""
    wl = inputs.hubbard("u0", 4, 4, 5, 5, "pair", U=0.0, seed=7, n_walkers=16, samples_per_walker=4)
    wl.C[:] = 1.0
    ns, M = wl.n_sites, wl.M
    T = np.zeros((ns, ns))
    for (i, j), t in zip(wl.bonds, wl.bond_t):
        T[i, j] -= t
        T[j, i] -= t
    ev, phi = np.linalg.eigh(T)
    F = phi[:, :5] @ phi[:, :5].T
    f = np.zeros(M * (M - 1) // 2)
    for i in range(ns):
        for j in range(ns):
            p, q = i, ns + j
            f[p * M - p * (p + 1) // 2 + (q - p - 1)] = F[i, j]
    wl.f = f
    P = oracle.Problem(wl)
    cand = inputs.draw_configs(np.random.default_rng(8), 256, ns, 5, 5)
    la = np.array([P.log_psi(o)[0] if P.log_psi(o)[1] != 0 else -np.inf for o in cand])
    occ = np.ascontiguousarray(cand[la > la.max() - 8][:16])
    h = V.vmc_create(wl, walker_precision=V.VMC_FP64, keep_fp64_store=True, keep_lowp_store=True)
    V.vmc_set_params(h, wl.C, wl.f)
    V.vmc_set_walkers(h, occ)
    V.vmc_sample(h, 5, 3)
    V.vmc_sample(h, 0, 9)
    g, es = V.sr_gradient(h, V.VMC_STORE_FP64)
    E = 2 * ev[:5].sum()
    assert es[0] == pytest.approx(E, abs=1e-8) and es[1] <= 1e-14
    gn = float(torch.linalg.vector_norm(g))
    assert gn <= 1e-8
    y, _ = V.sr_cg_solve(h, g, 1e-3, 1e-6, 2000, V.VMC_CG_FP64, allow_not_converged=True)
    tau = 0.05
    x0 = V.sr_update(h, y, tau, V.VMC_STORE_FP64)
    assert x0 == pytest.approx(1 - tau * E, rel=1e-9)
    C, f1 = V.vmc_get_params(h)
    step = np.linalg.norm(np.concatenate([C - 1.0, f1 - f]))
    assert step <= 1.1 * tau * gn / 1e-3 / x0 + 1e-14   # |y| <= |g| / eps
    h.close()


class _SumLocal:
    """Two handles standing for two ranks; summing their local sums is what
    the all-reduce does across processes."""

    def __init__(self, a, b):
        self.a, self.b = a, b

    def moments(self):
        m1, m2 = self.a.moments(), self.b.moments()
        return m1[0] + m2[0], m1[1] + m2[1], m1[2] + m2[2], m1[3] + m2[3]

    def product(self, v):
        return self.a.product(v) + self.b.product(v)


@pytest.mark.parametrize("store", [V.VMC_STORE_FP64, V.VMC_STORE_FP32])
def test_rank_local_sums_add_up_to_the_whole(store):
    from paper_1108_0900_gb300 import shard
    wl = CASES["hubbard4x4_pair"]()
    P = oracle.Problem(wl)
    occ = wl.init_occ.copy()
    step = np.zeros(wl.n_walkers, np.uint64)
    smp, _, _ = P.sample(occ, step, 91, 3, wl.samples_per_walker)
    E, O = P.measure(smp)
    halves = []
    for r in range(2):
        h = V.vmc_create(wl, walker_precision=V.VMC_FP64, keep_fp64_store=True, keep_lowp_store=True)
        V.vmc_set_params(h, wl.C, wl.f)
        V.vmc_measure(h, np.ascontiguousarray(smp[r::2]))
        halves.append(h)
    loc = _SumLocal(*(shard.LibraryLocal(h, store) for h in halves))
    res = shard.sr_step(loc, 0.05, 1e-3, 1e-10, 5000, reduce=lambda t: t)
    g_ref, Em = oracle.gradient(O, E)
    y_ref, _, _, ok = oracle.cg(O, g_ref, 1e-3, 1e-10)
    tol = 1e-8 if store == V.VMC_STORE_FP64 else 1e-5
    assert res["n"] == len(E) and res["E_mean"] == pytest.approx(Em, rel=1e-12)
    assert rel(res["g"].cpu().numpy(), g_ref) <= (1e-10 if store == V.VMC_STORE_FP64 else 1e-6)
    assert rel(res["y"].cpu().numpy(), y_ref) <= tol
    _, x0_ref = oracle.sr_update(np.zeros(wl.n_params), y_ref, 0.05, Em, O.mean(0))
    assert res["x0"] == pytest.approx(x0_ref, rel=tol)
    for h in halves:
        h.close()


@pytest.mark.parametrize("side_stream", [False, True])
def test_checkpoint_resume_reproduces_the_next_batch(tmp_path, side_stream):
    """save_state after an SR update, load_state into a fresh handle, and the
    next vmc_sample with the same seed gives the same samples bit for bit
    (configurations, correlator states, E_L, pairing block).  With
    side_stream, every call runs on a non-blocking torch stream and the
    checkpoint is taken on that stream."""
    wl = inputs.workload("hubbard4x4_pair", n_walkers=32, samples_per_walker=4)
    stream = torch.cuda.Stream() if side_stream else None
    ctx = torch.cuda.stream(stream) if side_stream else contextlib.nullcontext()
    with ctx:
        _checkpoint_roundtrip(tmp_path, wl, stream)


def _checkpoint_roundtrip(tmp_path, wl, stream):

    def fresh():
        return V.vmc_create(wl, walker_precision=V.VMC_FP64, keep_fp64_store=True, keep_lowp_store=False)

    h = fresh()
    V.vmc_set_params(h, wl.C, wl.f)
    V.vmc_set_walkers(h, wl.init_occ)
    V.vmc_sample(h, 5, 11)
    g, _ = V.sr_gradient(h, V.VMC_STORE_FP64)
    y, _ = V.sr_cg_solve(h, g, 1e-3, 1e-8, 5000, V.VMC_CG_FP64)
    V.sr_update(h, y, 0.02, V.VMC_STORE_FP64)
    path = str(tmp_path / "state.npz")
    V.save_state(h, path, stream=stream, next_seed=12, iteration=1)
    V.vmc_sample(h, 0, 12)
    a = V.vmc_get_samples(h, V.VMC_STORE_FP64)
    h2 = fresh()
    extra = V.load_state(h2, path)
    assert int(extra["iteration"]) == 1
    V.vmc_sample(h2, 0, int(extra["next_seed"]))
    b = V.vmc_get_samples(h2, V.VMC_STORE_FP64)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    h.close()
    h2.close()
