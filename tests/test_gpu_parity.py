"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Every input is seeded and synthetic; configurations handed to the library
come from the oracle's own Metropolis chains or from the seeded generator,
never from the CUDA path.  Tolerances (relative, 2-norm per output vector):
  FP64 stages                         1e-10
  FP32 storage, FP32 accumulation     1e-5   (S products)
  FP32 storage, FP64 accumulation     1e-6   (storage rounding 2^-24)
  BF16 storage                        3e-2   (storage rounding 2^-9)
  FP32 walkers (E_L, O)               derived from FP32 inversion: 5e-3
Integers (configurations, correlator states, counters) are compared exactly.
"""
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


def pair_list(wl):
    nu, N = wl.n_up, wl.N
    pl = [(a, b) for a in range(nu) for b in range(a + 1, nu)]
    pl += [(a, b) for a in range(nu, N) for b in range(a + 1, N)]
    pl += [(a, b) for a in range(nu) for b in range(nu, N)]
    return pl


def pf_index(M, p, q):
    return p * M - p * (p + 1) // 2 + (q - p - 1)


def oracle_compact(wl, occ, O):
    """Oracle dense O rows -> the ABI's pairing block order."""
    M, ncp = wl.M, wl.n_corr_params
    pl = pair_list(wl)
    out = np.zeros((len(occ), len(pl)))
    for s, o in enumerate(occ):
        for e, (a, b) in enumerate(pl):
            out[s, e] = O[s, ncp + pf_index(M, int(o[a]), int(o[b]))]
    return out


def oracle_chains(wl, n_burn, spw, seed):
    P = oracle.Problem(wl)
    occ = wl.init_occ.copy()
    step = np.zeros(wl.n_walkers, np.uint64)
    smp, mm, acc = P.sample(occ, step, seed, n_burn, spw)
    return P, smp, mm, occ, step


def make(wl, prec=V.VMC_FP64, keep64=True, keeplow=True, n_walkers=None, spw=None, refresh_every=0):
    h = V.vmc_create(wl, n_walkers=n_walkers, samples_per_walker=spw, walker_precision=prec,
                     keep_fp64_store=keep64, keep_lowp_store=keeplow, refresh_every=refresh_every)
    V.vmc_set_params(h, wl.C, wl.f)
    return h


SMALL = {
    "hubbard4x4_pair": lambda: inputs.workload("hubbard4x4_pair", n_walkers=24, samples_per_walker=6),
    "hubbard4x4_2x2": lambda: inputs.workload("hubbard4x4_2x2", n_walkers=37, samples_per_walker=5),
    "hubbard8x8_2x3_geometry": lambda: inputs.workload("hubbard8x8_2x3", n_walkers=9, samples_per_walker=3),
    "abinitio24": lambda: inputs.workload("abinitio24", n_walkers=8, samples_per_walker=2),
    "tiny2x2": lambda: inputs.hubbard("t", 2, 2, 1, 1, "2x2", seed=5, n_walkers=7, samples_per_walker=4),
    "nocorr3x2": lambda: inputs.hubbard("t", 3, 2, 2, 2, "none", seed=6, n_walkers=11, samples_per_walker=3),
    # translation-invariant correlators: x and y bonds share two blocks; every
    # 2x3 plaquette of the 8x8 lattice reads one block of 4,096 amplitudes
    "hubbard4x4_pair_shared": lambda: inputs.hubbard("s1", 4, 4, 8, 8, "pair", seed=12, n_walkers=24, samples_per_walker=6,
                                         shared=True),
    "hubbard8x8_2x3_shared": lambda: inputs.hubbard("s5", 8, 8, 28, 28, "2x3", seed=13, n_walkers=9, samples_per_walker=3,
                                         shared=True),
    # the paper's 4x4 layout: a 3x3 correlator at every site, one shared block
    # of 4^9 amplitudes per sublattice (524,784 parameters)
    "paper4x4_3x3": lambda: inputs.hubbard("p33", 4, 4, 8, 8, "3x3", seed=14, n_walkers=6, samples_per_walker=3,
                                           shared=True),
}


@pytest.fixture(scope="module", params=list(SMALL))
def case(request):
    wl = SMALL[request.param]()
    P, smp, mm, occ_end, step_end = oracle_chains(wl, 3, wl.samples_per_walker, inputs.seed_sampling_for("hubbard4x4_pair"))
    E, O = P.measure(smp)
    return dict(name=request.param, wl=wl, P=P, smp=smp, E=E, O=O, mm=mm, occ_end=occ_end, step_end=step_end)


# ---------------------------------------------------------------------------
# local energy and derivative ratios on oracle configurations
# ---------------------------------------------------------------------------

def test_measure_fp64(case):
    wl = case["wl"]
    h = make(wl)
    V.vmc_measure(h, case["smp"])
    occ, E, cs, pf = V.vmc_get_samples(h, V.VMC_STORE_FP64)
    assert np.array_equal(occ, case["smp"])
    cs_or = np.array([[case["P"].corr_state(o, c) for c in range(wl.n_corr)] for o in case["smp"]],
                     np.int64).reshape(len(occ), wl.n_corr)
    assert np.array_equal(cs.astype(np.int64), cs_or)
    assert np.all(np.abs(E - case["E"]) <= 1e-10 * np.maximum(1.0, np.abs(case["E"])))
    ref = oracle_compact(wl, case["smp"], case["O"])
    for s in range(len(ref)):
        assert rel(pf[s], ref[s]) <= 1e-10
    # the low-precision copies are the same values rounded
    _, _, _, pf32 = V.vmc_get_samples(h, V.VMC_STORE_FP32)
    _, _, _, pf16 = V.vmc_get_samples(h, V.VMC_STORE_BF16)
    assert np.array_equal(pf32, pf.astype(np.float32).astype(np.float64))
    assert rel(pf16, pf) <= 2 ** -8


def test_measure_fp32_walkers(case):
    wl = case["wl"]
    h = make(wl, prec=V.VMC_FP32)
    V.vmc_measure(h, case["smp"])
    occ, E, cs, pf = V.vmc_get_samples(h, V.VMC_STORE_FP32)
    assert np.array_equal(occ, case["smp"])
    assert np.all(np.abs(E - case["E"]) <= 5e-3 * np.maximum(1.0, np.abs(case["E"])))
    ref = oracle_compact(wl, case["smp"], case["O"])
    errs = [rel(pf[s], ref[s]) for s in range(len(ref))]
    assert max(errs) <= 5e-3


# ---------------------------------------------------------------------------
# Metropolis chains: identical proposals, decisions compared where the
# oracle's acceptance margin exceeds the precision of the kernel
# ---------------------------------------------------------------------------

def _chain_compare(case, prec, margin, max_bad=0.0):
    """Both sides draw the same Philox proposals.  A stored sample is
    compared exactly when every accept/reject decision before it had a
    relative margin |u - r^2| / r^2 above `margin` in the oracle's FP64
    arithmetic (the kernel's ratio error is below that margin); later samples
    of a walker whose chain met a closer decision are only checked for
    validity.  Returns the fraction of samples compared."""
    wl = case["wl"]
    n_burn = 3
    P = oracle.Problem(wl)
    o_occ, o_step = wl.init_occ.copy(), np.zeros(wl.n_walkers, np.uint64)
    smp, _, _, fc = P.sample(o_occ, o_step, inputs.seed_sampling_for("hubbard4x4_pair"), n_burn, wl.samples_per_walker,
                             close_tol=margin, return_first_close=True)
    h = make(wl, prec=prec)
    V.vmc_set_walkers(h, wl.init_occ)
    V.vmc_sample(h, n_burn, inputs.seed_sampling_for("hubbard4x4_pair"))
    occ, E, cs, pf = V.vmc_get_samples(h, V.VMC_STORE_FP64 if prec == V.VMC_FP64 else V.VMC_STORE_FP32)
    wocc, wstep = V.vmc_get_walkers(h)
    assert np.array_equal(wstep, o_step)
    spw, N = wl.samples_per_walker, wl.N
    got = occ.reshape(wl.n_walkers, spw, -1)
    exp = smp.reshape(wl.n_walkers, spw, -1)
    compared = 0
    bad_walkers = []
    for w in range(wl.n_walkers):
        ok = True
        for j in range(spw):
            last = (n_burn + j + 1) * N - 1          # index of the proposal ending sample j
            if fc[w] < 0 or fc[w] > last:
                ok &= bool(np.array_equal(got[w, j], exp[w, j]))
                compared += 1
        if fc[w] < 0:
            ok &= bool(np.array_equal(wocc[w], o_occ[w]))
        if not ok:
            bad_walkers.append(w)
    assert len(bad_walkers) <= max_bad * wl.n_walkers, bad_walkers
    # every stored configuration is inside the sector
    assert np.all((occ[:, :wl.n_up] < wl.n_sites)) and np.all(occ[:, wl.n_up:] >= wl.n_sites)
    assert np.all(np.diff(occ.astype(int), axis=1) > 0)
    return compared / (wl.n_walkers * spw)


def test_sampler_chains_fp64(case):
    frac = _chain_compare(case, V.VMC_FP64, 1e-9)
    assert frac >= 0.9


@pytest.mark.parametrize("refresh,tol", [(1, 1e-10), (0, 1e-7)])
def test_sampler_outputs_fp64(case, refresh, tol):
    """E_L and O written by the sampler itself (not by vmc_measure): on the
    walkers whose FP64 chains equal the oracle's, they must equal the oracle's
    values on its own samples.  With a rebuild before every stored sample the
    inverse is fresh; without it, the rank-2 update drift of one call bounds
    the error."""
    wl = case["wl"]
    n_burn = 3
    P = oracle.Problem(wl)
    o_occ, o_step = wl.init_occ.copy(), np.zeros(wl.n_walkers, np.uint64)
    smp, mm, _ = P.sample(o_occ, o_step, inputs.seed_sampling_for("hubbard4x4_pair"), n_burn, wl.samples_per_walker)
    E_or, O_or = P.measure(smp)
    ref = oracle_compact(wl, smp, O_or)
    h = make(wl, prec=V.VMC_FP64, refresh_every=refresh)
    V.vmc_set_walkers(h, wl.init_occ)
    V.vmc_sample(h, n_burn, inputs.seed_sampling_for("hubbard4x4_pair"))
    occ, E, cs, pf = V.vmc_get_samples(h, V.VMC_STORE_FP64)
    safe = np.repeat(mm > 1e-9, wl.samples_per_walker)
    assert safe.mean() >= 0.9
    assert np.array_equal(occ[safe], smp[safe])
    assert np.all(np.abs(E[safe] - E_or[safe]) <= tol * np.maximum(1.0, np.abs(E_or[safe])))
    for s in np.nonzero(safe)[0]:
        assert rel(pf[s], ref[s]) <= tol


def test_sampler_chains_fp32(case):
    # FP32 inverse after up to ~N^2/3 rank-2 updates: ratio error well below 2e-2
    # An FP32 walker's ratio error is ~u32 kappa(A) plus the drift of the
    # rank-2 updates since its last rebuild; on an ill-conditioned pairing
    # submatrix it can exceed the margin, so a small share of walkers may
    # leave the oracle's chain (they stay inside the sector).
    frac = _chain_compare(case, V.VMC_FP32, 2e-2, max_bad=0.15)
    assert frac > 0


# ---------------------------------------------------------------------------
# gradient and S products
# ---------------------------------------------------------------------------

def test_gradient(case):
    wl = case["wl"]
    h = make(wl)
    V.vmc_measure(h, case["smp"])
    g_or, em = oracle.gradient(case["O"], case["E"])
    g, stats = V.sr_gradient(h, V.VMC_STORE_FP64)
    assert abs(stats[0] - em) <= 1e-12 * max(1, abs(em))
    assert rel(g.cpu().numpy(), g_or) <= 1e-10
    g32, _ = V.sr_gradient(h, V.VMC_STORE_FP32)
    assert rel(g32.cpu().numpy(), g_or) <= 1e-6


@pytest.mark.parametrize("store,tol", [(V.VMC_STORE_FP64, 1e-10), (V.VMC_STORE_FP32, 1e-6),
                                       (V.VMC_STORE_FP32_F32ACC, 1e-5), (V.VMC_STORE_BF16, 3e-2)])
def test_apply_S(case, store, tol):
    wl = case["wl"]
    h = make(wl)
    V.vmc_measure(h, case["smp"])
    V.sr_gradient(h, V.VMC_STORE_FP64)
    rng = np.random.default_rng(7)
    for k in (1, 2, 4):
        v = rng.standard_normal((k, wl.n_params))
        out = V.sr_apply_S(h, torch.from_numpy(v).cuda(), wl.shift, store).cpu().numpy()
        for j in range(k):
            ref = oracle.apply_S(case["O"], v[j], wl.shift)
            assert rel(out[j], ref) <= tol, (k, j)


def test_cg_fp64(case):
    wl = case["wl"]
    h = make(wl)
    V.vmc_measure(h, case["smp"])
    g, _ = V.sr_gradient(h, V.VMC_STORE_FP64)
    x, info = V.sr_cg_solve(h, g, wl.shift, 1e-10, 20 * wl.n_params, V.VMC_CG_FP64)
    assert info["converged"] and info["true_rel_residual"] <= 1e-10
    g_or, _ = oracle.gradient(case["O"], case["E"])
    x_or, it, res, ok = oracle.cg(case["O"], g_or, wl.shift, 1e-12, 20 * wl.n_params)
    assert ok
    # both solve the same SPD system; agreement is bounded by cond * tol
    assert rel(x.cpu().numpy(), x_or) <= 1e-6


@pytest.mark.parametrize("mode", [V.VMC_CG_MIXED, V.VMC_CG_FP32])
def test_cg_mixed_refinement(case, mode):
    wl = case["wl"]
    h = make(wl)
    V.vmc_measure(h, case["smp"])
    g, _ = V.sr_gradient(h, V.VMC_STORE_FP64)
    x, info = V.sr_cg_solve(h, g, wl.shift, 1e-6, 50 * wl.n_params, mode)
    assert info["converged"] and info["true_rel_residual"] <= 1e-6
    # residual against the FP64 store (oracle values) stays at the same level
    g_or, _ = oracle.gradient(case["O"], case["E"])
    r = g_or - oracle.apply_S(case["O"], x.cpu().numpy(), wl.shift)
    assert np.linalg.norm(r) / np.linalg.norm(g_or) <= 2e-6


def test_cg_block4_refinement(case):
    """Enlarged block CG (four parameter-group columns, four-vector BF16
    products) as the inner solve of the flexible outer loop: same tolerance
    and the same residual against the oracle's FP64 store as the one-vector
    mode.  Ansatz with all correlators in one parameter block cannot be split
    four ways (UNSUPPORTED)."""
    wl = case["wl"]
    h = make(wl)
    V.vmc_measure(h, case["smp"])
    g, _ = V.sr_gradient(h, V.VMC_STORE_FP64)
    try:
        x, info = V.sr_cg_solve(h, g, wl.shift, 1e-6, 50 * wl.n_params, V.VMC_CG_BLOCK4)
    except V.VmcError as e:
        split = int(wl.corr_param_off[wl.n_corr // 2]) if wl.n_corr >= 2 else 0
        assert e.code == -8 and not (0 < split < wl.n_corr_params)
        pytest.skip("four-way split needs two correlator blocks")
    assert info["converged"] and info["true_rel_residual"] <= 1e-6
    g_or, _ = oracle.gradient(case["O"], case["E"])
    r = g_or - oracle.apply_S(case["O"], x.cpu().numpy(), wl.shift)
    assert np.linalg.norm(r) / np.linalg.norm(g_or) <= 2e-6


# ---------------------------------------------------------------------------
# log-amplitude and its adjoint
# ---------------------------------------------------------------------------

def test_logpsi_and_backward(case):
    wl = case["wl"]
    h = make(wl)
    V.vmc_measure(h, case["smp"])
    lp = V.vmc_logpsi(h).cpu().numpy()
    ref = np.array([case["P"].log_psi(o)[0] for o in case["smp"]])
    assert np.all(np.abs(lp - ref) <= 1e-10 * np.maximum(1, np.abs(ref)))
    w = np.random.default_rng(3).standard_normal(len(ref))
    grad = V.vmc_logpsi_backward(h, torch.from_numpy(w)).cpu().numpy()
    assert rel(grad, w @ case["O"]) <= 1e-10
    # w = None rewrites the store from scratch: same values
    _, _, _, pf0 = V.vmc_get_samples(h, V.VMC_STORE_FP64)
    V.vmc_logpsi_backward(h, None)
    _, _, _, pf1 = V.vmc_get_samples(h, V.VMC_STORE_FP64)
    assert rel(pf1, pf0) <= 1e-12


def test_autograd_logpsi():
    wl = SMALL["hubbard4x4_pair"]()
    P, smp, *_ = oracle_chains(wl, 2, wl.samples_per_walker, 11)
    h = make(wl)
    V.vmc_measure(h, smp)
    C = torch.tensor(wl.C, dtype=torch.float64, requires_grad=True)
    f = torch.tensor(wl.f, dtype=torch.float64, requires_grad=True)
    lp = V.LogPsi().apply(h, C, f)
    (lp.sum()).backward()
    _, O = P.measure(smp)
    ref = O.sum(0)
    assert rel(C.grad.numpy(), ref[:wl.n_corr_params]) <= 1e-10
    assert rel(f.grad.numpy(), ref[wl.n_corr_params:]) <= 1e-10
    # finite differences of the forward through the library
    hstep = 1e-6
    for k in (0, 17, wl.n_corr_params + 3, wl.n_params - 1):
        dC, df = torch.zeros_like(C), torch.zeros_like(f)
        (dC if k < wl.n_corr_params else df).view(-1)[k if k < wl.n_corr_params else k - wl.n_corr_params] = hstep
        up = V.LogPsi().apply(h, C.detach() + dC, f.detach() + df).sum().item()
        dn = V.LogPsi().apply(h, C.detach() - dC, f.detach() - df).sum().item()
        assert abs((up - dn) / (2 * hstep) - ref[k]) <= 1e-5 * max(1, abs(ref[k]))


# ---------------------------------------------------------------------------
# edge cases and error paths
# ---------------------------------------------------------------------------

def test_errors_and_edges():
    wl = inputs.hubbard("e", 3, 2, 2, 2, "pair", seed=9, n_walkers=5, samples_per_walker=2)
    h = make(wl)
    with pytest.raises(V.VmcError) as e:
        V.vmc_sample(h, 0, 1)                       # walkers not set
    assert e.value.code == -9
    bad = wl.init_occ.copy()
    bad[0, 0], bad[0, 1] = bad[0, 1], bad[0, 0]      # not ascending
    with pytest.raises(V.VmcError):
        V.vmc_set_walkers(h, bad)
    with pytest.raises(V.VmcError) as e:
        V.sr_apply_S(h, torch.zeros(wl.n_params, dtype=torch.float64, device="cuda"), 0.1)  # no samples yet
    assert e.value.code == -9
    # one sample
    V.vmc_measure(h, wl.init_occ[:1])
    assert V.vmc_num_samples(h) == 1
    g, st = V.sr_gradient(h)
    # one sample: zero covariance (up to the rounding of a fused multiply-add)
    assert torch.all(g.abs() <= 1e-14 * max(1.0, abs(st[0])))
    v = torch.randn(wl.n_params, dtype=torch.float64, device="cuda")
    out = V.sr_apply_S(h, v, 0.25)
    assert torch.allclose(out, 0.25 * v, rtol=1e-12, atol=1e-12)
    # singular pairing: all f = 0
    h2 = V.vmc_create(wl)
    V.vmc_set_params(h2, wl.C, np.zeros_like(wl.f))
    with pytest.raises(V.VmcError) as e:
        V.vmc_measure(h2, wl.init_occ)
    assert e.value.code == -3
    # zero correlator amplitude
    C0 = wl.C.copy()
    C0[3] = 0.0
    with pytest.raises(V.VmcError) as e:
        V.vmc_set_params(h2, C0, wl.f)
    assert e.value.code == -3


# ---------------------------------------------------------------------------
# full-size 8x8 / 2x3-plaquette workload (65,536 samples, 270,272 parameters)
# in the launch configuration of the benchmark: sampled outputs against the
# oracle one by one, and invariants that hold at any size
# ---------------------------------------------------------------------------

_FULL = {}


def full_size(prec, name="hubbard8x8_2x3"):
    if (prec, name) not in _FULL:
        wl = inputs.workload(name)
        h = make(wl, prec=prec, keep64=True, keeplow=True)
        cfgs = inputs.draw_configs(np.random.default_rng(555), wl.n_samples, wl.n_sites, wl.n_up, wl.n_dn)
        V.vmc_measure(h, cfgs)
        _FULL.clear()
        _FULL[(prec, name)] = (wl, h, cfgs)
    return _FULL[(prec, name)]


@pytest.mark.parametrize("name,prec,tol", [("hubbard8x8_2x3", V.VMC_FP64, 1e-10), ("hubbard8x8_2x3", V.VMC_FP32, 5e-3),
                                           ("abinitio24", V.VMC_FP64, 1e-10), ("abinitio24", V.VMC_FP32, 5e-3)])
def test_full_size_sampled_outputs(name, prec, tol):
    """Every sample of the full workload is evaluated on the GPU; a random
    subset (and the last sample) is recomputed by the oracle."""
    wl, h, cfgs = full_size(prec, name)
    occ, E, cs, pf = V.vmc_get_samples(h, V.VMC_STORE_FP64 if prec == V.VMC_FP64 else V.VMC_STORE_FP32)
    assert np.array_equal(occ, cfgs)
    P = oracle.Problem(wl)
    pick = np.random.default_rng(1).choice(len(cfgs), 24 if name == "hubbard8x8_2x3" else 8, replace=False)
    pick[-1] = len(cfgs) - 1
    E_or, O_or = P.measure(cfgs[pick])
    ref = oracle_compact(wl, cfgs[pick], O_or)
    for j, s in enumerate(pick):
        assert [P.corr_state(cfgs[s], c) for c in range(wl.n_corr)] == [int(x) for x in cs[s]]
        assert abs(E[s] - E_or[j]) <= tol * max(1.0, abs(E_or[j]))
        assert rel(pf[s], ref[j]) <= tol


def test_full_size_invariants():
    # |Psi|^2-sampled configurations (FP64 walkers): away from the nearly
    # singular pairing submatrices a uniform draw can hit, the identities
    # below hold to FP64 rounding
    # (rebuilding every walker's inverse from scratch before each stored
    # sample, so no rank-2 update drift enters O)
    _FULL.clear()
    wl = inputs.workload("hubbard8x8_2x3")
    h = make(wl, prec=V.VMC_FP64, keep64=True, keeplow=True, refresh_every=1)
    V.vmc_set_walkers(h, wl.init_occ)
    V.vmc_sample(h, 10, inputs.seed_sampling_for("hubbard8x8_2x3"))
    g, stats = V.sr_gradient(h, V.VMC_STORE_FP64)
    ncp = wl.n_corr_params
    eps = wl.shift
    # null vectors: O_s . C_c = 1 and O_s . f = N/2 for every sample
    # FP32 accumulation of the mean term against the FP64 mean leaves ~1e-7
    # relative per pairing entry, ~1e-4 of |eps v| over 8,128 entries
    for store, tol in ((V.VMC_STORE_FP32, 1e-6), (V.VMC_STORE_FP32_F32ACC, 1e-3), (V.VMC_STORE_BF16, 1e-2)):
        for c in (0, 40):
            v = np.zeros(wl.n_params)
            v[c * 4096:(c + 1) * 4096] = wl.C[c * 4096:(c + 1) * 4096]
            vt = torch.from_numpy(v).cuda()
            Sv = V.sr_apply_S(h, vt, eps, store)
            assert rel(Sv.cpu().numpy(), eps * v) <= tol
    vf = np.zeros(wl.n_params)
    vf[ncp:] = wl.f
    rng = np.random.default_rng(2)
    a = torch.from_numpy(rng.standard_normal(wl.n_params)).cuda()
    b = torch.from_numpy(rng.standard_normal(wl.n_params)).cuda()
    Sa = V.sr_apply_S(h, a, eps, V.VMC_STORE_FP32)
    Sb = V.sr_apply_S(h, b, eps, V.VMC_STORE_FP32)
    # O_s . f = N/2 (homogeneity of the pfaffian): S f = eps f, checked in
    # FP64 and against the FP32 store relative to a generic product's size
    scale = torch.linalg.norm(Sa).item() / torch.linalg.norm(a).item() * np.linalg.norm(vf)
    # O_s . f - N/2 is the rounding of sum_ab X_ba A_ab, ~kappa(A) u per sample
    for store, tol in ((V.VMC_STORE_FP64, 1e-9), (V.VMC_STORE_FP32, 1e-6)):
        Sf = V.sr_apply_S(h, torch.from_numpy(vf).cuda(), eps, store).cpu().numpy()
        assert np.linalg.norm(Sf - eps * vf) <= tol * scale
    # symmetry and positivity
    assert abs((b @ Sa - a @ Sb).item()) <= 1e-9 * abs((b @ Sa).item()) + 1e-9
    assert (a @ Sa).item() >= eps * (a @ a).item() * (1 - 1e-9)
    vft = torch.from_numpy(vf).cuda()
    assert abs((g @ vft).item()) <= 1e-6 * torch.linalg.norm(g).item() * np.linalg.norm(vf)


def test_full_size_sampling_run():
    wl = inputs.workload("hubbard8x8_2x3")
    h = make(wl, prec=V.VMC_FP32, keep64=False, keeplow=True)
    V.vmc_set_walkers(h, wl.init_occ)
    V.vmc_sample(h, 2, inputs.seed_sampling_for("hubbard8x8_2x3"))
    occ, E, cs, pf = V.vmc_get_samples(h, V.VMC_STORE_FP32)
    assert np.all(np.isfinite(E)) and np.all(np.isfinite(pf))
    assert np.all(occ[:, :wl.n_up] < wl.n_sites) and np.all(occ[:, wl.n_up:] >= wl.n_sites)
    assert np.all(np.diff(occ.astype(int), axis=1) > 0)
    _, step = V.vmc_get_walkers(h)
    assert np.all(step == (2 + wl.samples_per_walker) * wl.N)


def test_bf16_product_over_several_sample_chunks():
    """The sorted BF16 product splits its parameter-major copy into chunks of
    65,536 samples; with 132,096 samples (two full chunks and a ragged third)
    it must equal the FP64 product of the same stored BF16 values
    (FP32 accumulation: 2e-5)."""
    sp = pytest.importorskip("scipy.sparse")
    wl = inputs.workload("hubbard4x4_pair", n_walkers=16512, samples_per_walker=8)
    n = wl.n_walkers * wl.samples_per_walker
    assert n > 2 * 65536
    cfgs = inputs.draw_configs(np.random.default_rng(31), n, wl.n_sites, wl.n_up, wl.n_dn)
    h = make(wl)
    V.vmc_measure(h, cfgs)
    V.sr_gradient(h, V.VMC_STORE_BF16)
    occ, _, cs, pf = V.vmc_get_samples(h, V.VMC_STORE_BF16)
    M, ncp = wl.M, wl.n_corr_params
    off = np.concatenate([[0], np.cumsum([4 ** len(c) for c in wl.corr_sites])])
    pl = np.array(pair_list(wl))
    p, q = occ[:, pl[:, 0]].astype(np.int64), occ[:, pl[:, 1]].astype(np.int64)
    cols = np.hstack([off[None, :-1] + cs.astype(np.int64), ncp + p * M - p * (p + 1) // 2 + (q - p - 1)])
    vals = np.hstack([1.0 / wl.C[off[None, :-1] + cs.astype(np.int64)], pf])
    O = sp.csr_matrix((vals.ravel(), cols.ravel(), np.arange(0, vals.size + 1, vals.shape[1])),
                      shape=(n, wl.n_params))
    Ob = np.asarray(O.mean(0)).ravel()
    v = np.random.default_rng(8).standard_normal(wl.n_params)
    ref = O.T @ (O @ v) / n - Ob * (Ob @ v) + wl.shift * v
    out = V.sr_apply_S(h, torch.from_numpy(v).cuda(), wl.shift, V.VMC_STORE_BF16).cpu().numpy()
    assert rel(out, ref) <= 2e-5
    h.close()


def test_abinitio_eigenstate_closed_form_at_24_orbitals():
    """The CUDA local energy at 24 orbitals, 12 + 12 electrons, against a
    closed form instead of the oracle: H = Khat^2 / 2 - Jhat / 2 (one
    Cholesky vector K, J = K^2) and Psi the determinants of the 12 lowest
    eigenvectors of K (C = 1) is an eigenstate, so every configuration has
    E_L = kappa^2 / 2 - sum lambda_k^2, kappa = 2 sum lambda_k (singles and
    doubles both contribute)."""
    n, M = 24, 48
    wl = inputs.abinitio("b", n, 12, 12, n_chol=1, seed=79, n_walkers=256, samples_per_walker=4)
    A = np.random.default_rng(9).standard_normal((n, n))
    K = 0.1 * (A + A.T)
    wl.h = np.zeros((n, n))
    wl.chol = K[None].copy()
    wl.C = np.ones_like(wl.C)
    lam, phi = np.linalg.eigh(K)
    F = phi[:, :12] @ phi[:, :12].T
    f = np.zeros(M * (M - 1) // 2)
    for i in range(n):
        for j in range(n):
            p, q = i, n + j
            f[p * M - p * (p + 1) // 2 + (q - p - 1)] = F[i, j]
    wl.f = f
    E0 = 0.5 * (2 * lam[:12].sum()) ** 2 - lam[:12] @ lam[:12]
    h = V.vmc_create(wl, walker_precision=V.VMC_FP64, keep_fp64_store=True, keep_lowp_store=False,
                     refresh_every=1)
    V.vmc_set_params(h, wl.C, wl.f)
    # (a) configurations drawn from |Psi|^2 (FP64 chains, the inverse rebuilt
    # from scratch before every stored sample): every sample at 1e-10
    V.vmc_set_walkers(h, wl.init_occ)
    V.vmc_sample(h, 20, 4242)
    _, E, _, _ = V.vmc_get_samples(h, V.VMC_STORE_FP64)
    err = np.abs(E - E0) / abs(E0)
    assert err.max() <= 1e-10, err.max()
    # (b) uniformly drawn configurations, some with nearly singular pairing
    # blocks: FP64 rounding of the ratios grows with the condition number of
    # the occupied pairing submatrix, and E_L sums about 3 x 10^4 single and
    # double excitation terms, so each sample is held to 1e-12 kappa(A_occ)
    # (about 10^4 unit roundoffs times kappa; a wrong or missing term would
    # leave an O(1) relative error)
    cfgs = inputs.draw_configs(np.random.default_rng(12), wl.n_samples, n, 12, 12)
    V.vmc_measure(h, cfgs)
    _, E, _, _ = V.vmc_get_samples(h, V.VMC_STORE_FP64)
    Fm = np.zeros((M, M))
    Fm[:n, n:] = F
    Fm[n:, :n] = -F.T
    kappa = np.array([np.linalg.cond(Fm[np.ix_(o, o)]) for o in cfgs.astype(np.int64)])
    err = np.abs(E - E0) / abs(E0)
    assert np.all(err <= 1e-12 * np.maximum(kappa, 1.0)), (err / kappa).max()
    h.close()
